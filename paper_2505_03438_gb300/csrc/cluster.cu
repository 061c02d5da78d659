// cluster.cu -- LJ forces over cluster-pair Verlet lists (the GPU form of
// the Verlet-list container, Sec. 2.2.1, with i-clusters x j-clusters).
//
// A group of G = M * k lanes (G <= 32) owns one i-cluster of M particles:
// lane g holds i-member a = g % M and takes j-members b = s, s + k, ... with
// s = g / M.  For every listed j-cluster the group stages the j positions in
// shared memory with one coalesced vector load per lane, evaluates its pairs,
// and at the end sums F_i over the k lanes of each member by warp shuffles.
// N3L on (k = 1): each unordered cluster pair is listed once; lane a visits
// j-members in rotated order b = (a + t) mod n_j so that lanes rarely touch
// the same shared-memory slot, accumulates -F_ij there, and the group adds
// the j forces to global memory once per listed j-cluster.
#include "kernels.cuh"

namespace ljsel {

namespace {

constexpr int CP_THREADS = 128;

template <typename R> struct CpTab {
    R sig2[MAXT2], e24[MAXT2], e48[MAXT2], e4[MAXT2], ushift[MAXT2], lo[MAXT2], hi[MAXT2];
    double rc2d[MAXT2];
};

__device__ __forceinline__ void sadd(float4 *p, float x, float y, float z) {
    atomicAdd(&p->x, x); atomicAdd(&p->y, y); atomicAdd(&p->z, z);
}
__device__ __forceinline__ void sadd(D4 *p, double x, double y, double z) {
    atomicAdd(&p->x, x); atomicAdd(&p->y, y); atomicAdd(&p->z, z);
}
__device__ __forceinline__ void gadd(float4 *F, int j, float4 v) { atomicAdd(F + j, v); }
__device__ __forceinline__ void gadd(D4 *F, int j, const D4 &v) {
    atomicAdd(&F[j].x, v.x); atomicAdd(&F[j].y, v.y); atomicAdd(&F[j].z, v.z);
}

template <typename R>
__device__ __forceinline__ void cp_block_sum3(double a, double b, double c, Ctrl *C) {
    __shared__ double s[3][CP_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { s[0][warp] = a; s[1][warp] = b; s[2][warp] = c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, y = 0, z = 0;
        for (int k = 0; k < CP_THREADS / 32; ++k) { x += s[0][k]; y += s[1][k]; z += s[2][k]; }
        if (x != 0.0) atomicAdd(&C->epot, x);
        if (y != 0.0) atomicAdd(&C->virial, y);
        if (z != 0.0) atomicAdd(&C->ekin, z);
    }
}

template <typename R, bool N3L, int MODE, bool EV, bool MT>
__global__ void __launch_bounds__(CP_THREADS) k_cp(Dev<R> S, int G, int2 *pairs, long long cap) {
    Ctrl *C = S.ctrl;
    if (C->overflow) return;
    __shared__ CpTab<R> T;
    __shared__ V4<R> s_pos[CP_THREADS];
    __shared__ V4<R> s_fj[N3L ? CP_THREADS : 1];
    if (MT) {
        for (int k = threadIdx.x; k < MAXT2; k += blockDim.x) {
            T.sig2[k] = S.tab.sig2[k]; T.e24[k] = S.tab.e24[k]; T.e48[k] = S.tab.e48[k]; T.e4[k] = S.tab.e4[k];
            T.ushift[k] = S.tab.ushift[k]; T.lo[k] = S.tab.rc2lo[k]; T.hi[k] = S.tab.rc2hi[k]; T.rc2d[k] = S.tab.rc2d[k];
        }
    }
    const int M = S.M;
    const int k = G / M;
    const int lane = threadIdx.x & 31;
    const int gl = threadIdx.x % G;              // lane within group
    const int gbase = threadIdx.x - gl;          // first thread of the group in the block
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane - gl));
    const int a = gl % M, s = gl / M;
    if (N3L) s_fj[threadIdx.x] = make_pos((R)0, (R)0, (R)0, 0);
    __syncthreads();
    const int ci = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    const int ncl = *S.ncl_total;
    const bool gvalid = ci < ncl;
    const int pp = C->pos_par, sp = C->state_par;
    const V4<R> *P = S.pos[pp];
    int fi = 0, ni = 0, nent = 0;
    if (gvalid) { fi = S.cl_first[ci]; ni = S.cl_count[ci]; nent = S.cp_count[ci]; }
    const bool ivalid = gvalid && a < ni;
    V4<R> pi = make_pos((R)0, (R)0, (R)0, 0);
    int ti = 0;
    if (ivalid) { pi = ldpos(P, fi + a); ti = type_of(pi); }
    R fx = 0, fy = 0, fz = 0, u = 0, w = 0;
    int np = 0;
    for (int e = 0; e < nent; ++e) {
        const uint32_t ent = S.cp[(size_t)e * S.cp_stride + ci];
        const int cj = (int)(ent & JMASK);
        const uint32_t code = ent >> JBITS;
        const int fj = S.cl_first[cj], nj = S.cl_count[cj];
        if (gl < nj) s_pos[gbase + gl] = ldpos(P, fj + gl);
        __syncwarp(gmask);
        int sx = 0, sy = 0, sz = 0;
        if (code) decode_image(code, sx, sy, sz);
        const bool self = (cj == ci) && code == 0;
        if (ivalid) {
            for (int t = s; t < nj; t += k) {
                const int b = N3L ? (a + t) % nj : t;
                if (self && (N3L ? b <= a : b == a)) continue;
                const V4<R> pj = s_pos[gbase + b];
                R dx, dy, dz;
                if (code == 0) {
                    dx = pi.x - pj.x; dy = pi.y - pj.y; dz = pi.z - pj.z;
                } else {
                    dx = image_dx(pi.x, pj.x, sx, S.box[0], S.box_lo[0]);
                    dy = image_dx(pi.y, pj.y, sy, S.box[1], S.box_lo[1]);
                    dz = image_dx(pi.z, pj.z, sz, S.box[2], S.box_lo[2]);
                }
                const R r2 = r2_of(dx, dy, dz);
                const int tp = MT ? ti * S.tab.ntypes + type_of(pj) : 0;
                R sig2, e24, e48, lo, hi;
                double rc2d;
                if (MT) { sig2 = T.sig2[tp]; e24 = T.e24[tp]; e48 = T.e48[tp]; lo = T.lo[tp]; hi = T.hi[tp]; rc2d = T.rc2d[tp]; }
                else { sig2 = S.tab.sig2[0]; e24 = S.tab.e24[0]; e48 = S.tab.e48[0]; lo = S.tab.rc2lo[0]; hi = S.tab.rc2hi[0]; rc2d = S.tab.rc2d[0]; }
                const bool in = Cut<R>::in(r2, lo, hi, pi, pj, sx, sy, sz, S.boxd, rc2d);
                if (MODE == MODE_PAIRS) {
                    if (in) {
                        const int ia = S.id[sp][fi + a], jb = S.id[sp][fj + b];
                        if (N3L || ia < jb) {
                            unsigned long long slot = atomicAdd(&C->npairs, 1ull);
                            if ((long long)slot < cap) pairs[slot] = make_int2(min(ia, jb), max(ia, jb));
                        }
                    }
                    continue;
                }
                R sr6;
                R fr = lj_fr(r2, sig2, e24, e48, sr6);
                fr = in ? fr : (R)0;
                if (EV) {
                    if (MT) u += in ? T.e4[tp] * sr6 * (sr6 - (R)1) - T.ushift[tp] : (R)0;
                    else { u += in ? sr6 * (sr6 - (R)1) : (R)0; np += in ? 1 : 0; }
                    w += fr * r2;
                }
                fx += fr * dx; fy += fr * dy; fz += fr * dz;
                if (N3L) sadd(&s_fj[gbase + b], -fr * dx, -fr * dy, -fr * dz);
            }
        }
        __syncwarp(gmask);
        if (N3L && MODE != MODE_PAIRS) {
            if (gl < nj) {
                V4<R> f = s_fj[gbase + gl];
                gadd(S.force, fj + gl, f);
                s_fj[gbase + gl] = make_pos((R)0, (R)0, (R)0, 0);
            }
            __syncwarp(gmask);
        }
    }
    if (MODE == MODE_PAIRS) return;
    for (int o = M; o < G; o <<= 1) {
        fx += __shfl_xor_sync(0xffffffffu, fx, o);
        fy += __shfl_xor_sync(0xffffffffu, fy, o);
        fz += __shfl_xor_sync(0xffffffffu, fz, o);
    }
    double ke = 0;
    bool exceeded = false, bad = false;
    if (ivalid && s == 0) {
        const int i = fi + a;
        if (N3L) gadd(S.force, i, make_pos(fx, fy, fz, 0));
        else if (MODE == MODE_FORCE) S.force[i] = make_pos(fx, fy, fz, 0);
        else {
            // Stormer-Verlet update, as in the list and cell kernels
            const int n = S.n;
            double *X = S.x[sp];
            double *V = S.v[sp];
            R c = S.tab.inv_mass_dt[ti];
            const int half = C->half_kick;
            if (half) c *= (R)0.5;
            double vx = V[i], vy = V[n + i], vz = V[2 * n + i];
            if (EV) {
                double h = half ? 0.0 : 0.5;
                double ux = vx + h * (double)(S.tab.inv_mass_dt[ti] * fx);
                double uy = vy + h * (double)(S.tab.inv_mass_dt[ti] * fy);
                double uz = vz + h * (double)(S.tab.inv_mass_dt[ti] * fz);
                ke += S.tab.half_mass[ti] * (ux * ux + uy * uy + uz * uz);
            }
            vx += (double)(c * fx); vy += (double)(c * fy); vz += (double)(c * fz);
            const double dt = S.tab.dt;
            double x = fma(dt, vx, X[i]), y = fma(dt, vy, X[n + i]), z = fma(dt, vz, X[2 * n + i]);
            V[i] = vx; V[n + i] = vy; V[2 * n + i] = vz;
            X[i] = x; X[n + i] = y; X[2 * n + i] = z;
            V4<R> wp = make_pos((R)x, (R)y, (R)z, ti);
            S.pos[pp ^ 1][i] = wp;
            V4<R> r = S.xref[i];
            R ddx = wp.x - r.x, ddy = wp.y - r.y, ddz = wp.z - r.z;
            exceeded = !(ddx * ddx + ddy * ddy + ddz * ddz < S.half_skin2);
            bad = !isfinite(fx + fy + fz);
        }
    }
    if (MODE == MODE_STEP) {
        if (__any_sync(0xffffffffu, exceeded) && lane == 0) C->disp_exceeded = 1;
        if (__any_sync(0xffffffffu, bad) && lane == 0) C->nonfinite = 1;
    }
    if (EV) {
        R e = MT ? u : S.tab.e4[0] * u - S.tab.ushift[0] * (R)np;
        const R scale = N3L ? (R)1 : (R)0.5;
        cp_block_sum3<R>((double)(scale * e), (double)(scale * w), ke, C);
    }
}

template <typename R, bool N3L, int MODE, bool EV, bool MT>
void cp_go(const Dev<R> &S, int G, int2 *pairs, long long cap, cudaStream_t st) {
    long long threads = (long long)S.ncl_cap * G;
    k_cp<R, N3L, MODE, EV, MT><<<div_up(threads, CP_THREADS), CP_THREADS, 0, st>>>(S, G, pairs, cap);
}

template <typename R, bool MT>
void cp_dispatch(const Dev<R> &S, const ljsel_config &cfg, int mode, bool ev, int2 *pairs, long long cap,
                 cudaStream_t st) {
    const bool n3l = cfg.newton3 != 0;
    int G = cfg.threads_per_unit < S.M ? S.M : cfg.threads_per_unit;
    if (n3l) G = S.M;
    if (mode == MODE_PAIRS) { n3l ? cp_go<R, true, MODE_PAIRS, false, MT>(S, G, pairs, cap, st) : cp_go<R, false, MODE_PAIRS, false, MT>(S, G, pairs, cap, st); return; }
    if (n3l) { ev ? cp_go<R, true, MODE_FORCE, true, MT>(S, G, pairs, cap, st) : cp_go<R, true, MODE_FORCE, false, MT>(S, G, pairs, cap, st); return; }
    if (mode == MODE_STEP) { ev ? cp_go<R, false, MODE_STEP, true, MT>(S, G, pairs, cap, st) : cp_go<R, false, MODE_STEP, false, MT>(S, G, pairs, cap, st); return; }
    ev ? cp_go<R, false, MODE_FORCE, true, MT>(S, G, pairs, cap, st) : cp_go<R, false, MODE_FORCE, false, MT>(S, G, pairs, cap, st);
}

}  // namespace

template <typename R> void launch_cp_force(const Dev<R> &S, const ljsel_config &cfg, int mode, bool ev, int2 *pairs,
                                           long long cap, cudaStream_t st);
template <> void launch_cp_force<float>(const Dev<float> &S, const ljsel_config &cfg, int mode, bool ev, int2 *pairs,
                                        long long cap, cudaStream_t st) {
    if (S.tab.ntypes > 1) cp_dispatch<float, true>(S, cfg, mode, ev, pairs, cap, st);
    else cp_dispatch<float, false>(S, cfg, mode, ev, pairs, cap, st);
}
template <> void launch_cp_force<double>(const Dev<double> &S, const ljsel_config &cfg, int mode, bool ev, int2 *pairs,
                                         long long cap, cudaStream_t st) {
    cp_dispatch<double, true>(S, cfg, mode, ev, pairs, cap, st);
}

}  // namespace ljsel
