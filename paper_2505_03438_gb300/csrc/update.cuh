// update.cuh -- per-particle Stormer-Verlet update and the FP64 block sums
// shared by the force kernels that fuse the update (Sec. 2.1).
#pragma once

#include "ljsel_internal.cuh"

namespace ljsel {

// FP64 block reduction of energy, virial and kinetic energy into Ctrl.
__device__ __forceinline__ void block_sum3(double a, double b, double c, Ctrl *C) {
    __shared__ double s[3][32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) { s[0][warp] = a; s[1][warp] = b; s[2][warp] = c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, y = 0, z = 0;
        for (int k = 0; k < nw; ++k) { x += s[0][k]; y += s[1][k]; z += s[2][k]; }
        if (x != 0.0) atomicAdd(&C->epot, x);
        if (y != 0.0) atomicAdd(&C->virial, y);
        if (z != 0.0) atomicAdd(&C->ekin, z);
    }
}

// FP32 <-> FP64 conversions on the integer pipes (the FP64 pipe of this part
// runs about two operations a clock per SM, the integer pipes 64): exact for
// zero and normal values, double to float rounded to nearest even; results
// in the FP32 subnormal range flush to zero, and non-finite inputs are not
// preserved (the update checks the FP32 forces for them separately, and
// positions and velocities of a running simulation are finite and normal or
// zero).
__device__ __forceinline__ double f32_to_f64(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    // rebias the exponent (1023 - 127 = 896) and move the 23 mantissa bits
    // to the top of the 52
    const unsigned hi = (u & 0x80000000u) | (e ? (((e + 896u) << 20) | ((u & 0x7fffffu) >> 3)) : 0u);
    const unsigned lo = e ? (u << 29) : 0u;
    return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ float f64_to_f32(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu) - 896;
    // the top 23 of the 52 mantissa bits, the round bit and the sticky bits
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
    const unsigned rb = (lo >> 28) & 1u, st = (lo & 0x0fffffffu) != 0u ? 1u : 0u;
    // exponent and mantissa as one field, so that a rounding carry moves
    // into the exponent (and at the top into the infinity pattern)
    unsigned r = ((unsigned)e << 23) + m;
    r += rb & (st | (m & 1u));
    r = e <= 0 ? 0u : (e >= 255 ? 0x7f800000u : r);
    return __uint_as_float((hi & 0x80000000u) | r);
}

// Stormer-Verlet update of one particle (Sec. 2.1) in leapfrog form: the
// stored velocity is at the half step (or, with `half`, at the integer step,
// and the kick is dt/2).  v += (dt/m) F; x += dt v; the working copy is the
// FP32 rounding (to nearest even) of the FP64 position.  Returns |x -
// x_ref|^2 exceedance and the kinetic energy at the integer step (EV).
template <typename R, bool EV>
__device__ __forceinline__ void integrate_one(const Dev<R> &S, int sp, int pp, int half, int i, int t, R fx, R fy,
                                              R fz, double &ke, bool &exceeded, bool &bad) {
    const int n = S.n;
    double *X = S.x[sp];
    double *V = S.v[sp];
    // every load first, so that they are in flight together (the stores
    // below may alias them as far as the compiler knows)
    double vx = V[i], vy = V[n + i], vz = V[2 * n + i];
    const double x0 = X[i], y0 = X[n + i], z0 = X[2 * n + i];
    const V4<R> r = S.xref[i];
    R c = S.tab.inv_mass_dt[t];
    if (half) c *= (R)0.5;
    double dvx, dvy, dvz;
    if constexpr (sizeof(R) == 4) {
        dvx = f32_to_f64(c * fx); dvy = f32_to_f64(c * fy); dvz = f32_to_f64(c * fz);
    } else {
        dvx = c * fx; dvy = c * fy; dvz = c * fz;
    }
    if (EV) {
        double h = half ? 0.0 : 0.5;
        double ux = vx + h * (double)(S.tab.inv_mass_dt[t] * fx);
        double uy = vy + h * (double)(S.tab.inv_mass_dt[t] * fy);
        double uz = vz + h * (double)(S.tab.inv_mass_dt[t] * fz);
        ke += S.tab.half_mass[t] * (ux * ux + uy * uy + uz * uz);
    }
    vx += dvx; vy += dvy; vz += dvz;
    const double dt = S.tab.dt;
    double x = fma(dt, vx, x0);
    double y = fma(dt, vy, y0);
    double z = fma(dt, vz, z0);
    // reflective walls: mirror a crossing back and reverse the velocity component
    if (S.walls[0]) { if (x < 0.0) { x = -x; vx = -vx; } else if (x > S.boxd[0]) { x = 2.0 * S.boxd[0] - x; vx = -vx; } }
    if (S.walls[1]) { if (y < 0.0) { y = -y; vy = -vy; } else if (y > S.boxd[1]) { y = 2.0 * S.boxd[1] - y; vy = -vy; } }
    if (S.walls[2]) { if (z < 0.0) { z = -z; vz = -vz; } else if (z > S.boxd[2]) { z = 2.0 * S.boxd[2] - z; vz = -vz; } }
    V[i] = vx; V[n + i] = vy; V[2 * n + i] = vz;
    X[i] = x; X[n + i] = y; X[2 * n + i] = z;
    V4<R> w;
    if constexpr (sizeof(R) == 4) w = make_pos(f64_to_f32(x), f64_to_f32(y), f64_to_f32(z), t);
    else w = make_pos(x, y, z, t);
    S.pos[pp ^ 1][i] = w;
    R ddx = w.x - r.x, ddy = w.y - r.y, ddz = w.z - r.z;
    R d2 = ddx * ddx + ddy * ddy + ddz * ddz;
    exceeded = exceeded || !(d2 < S.half_skin2);
    bad = bad || !isfinite(fx + fy + fz);
}

__device__ __forceinline__ void report_flags(Ctrl *C, bool exceeded, bool bad) {
    if (__any_sync(0xffffffffu, exceeded) && (threadIdx.x & 31) == 0) C->disp_exceeded = 1;
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) C->nonfinite = 1;
}

}  // namespace ljsel
