// batch.cu -- many independent periodic LJ systems (replicas of uneven size)
// stepped together: one launch per kernel stage covers every replica, and
// the whole run of steps is one CUDA graph.
//
// Each replica r has its own cubic-or-not periodic box, its own linked-cell
// grid (side >= r_c + skin, stretched to tile its box, Sec. 2.2.1) and its
// particles.  All replicas share the single-species LJ parameters, cutoff,
// skin and time step.  Replicas are concatenated: particles of replica r
// occupy the slots [p_off[r], p_off[r] + n_r) in input order and keep that
// range after every re-sort, because the global cell index space lists the
// cells of replica 0, then replica 1, ...; so the replica of a slot never
// changes and is looked up from a static table.
//
// Per step (Sec. 2.1, Sec. 2.2.1): IF(rebuild) {plan -> bin -> scan ->
// scatter -> sort + gather -> Verlet lists -> finish}, then the fused force +
// Stormer-Verlet kernel, then the control kernel.  The Verlet-list rule is
// kept per replica: a rebuild event happens as soon as any particle of any
// replica moved skin/2 (or R steps after the last event), and it re-bins and
// re-lists only the replicas that need it -- those with a particle at skin/2,
// or R steps or more since their own last rebuild; the others keep their
// slots, cells and lists.  The force kernel takes a "tile": lanes per particle and CTA
// size, optionally as a persistent grid that strides over the tiles; the
// batch autotuner times the tiles and keeps the fastest.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "system.h"
#include "update.cuh"

using namespace ljsel;

#define CK(call)                                                                                    \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) {                                                                    \
            set_error(std::string("CUDA error in ") + #call + ": " + cudaGetErrorString(e_));       \
            return e_ == cudaErrorMemoryAllocation ? LJSEL_ERR_OOM : LJSEL_ERR_CUDA;                \
        }                                                                                           \
    } while (0)
#define TRY(expr)                         \
    do {                                  \
        ljsel_status s_ = (expr);         \
        if (s_ != LJSEL_OK) return s_;    \
    } while (0)

namespace {

constexpr int SCAN_BLOCK = 1024;

template <typename R> struct RepInfo {
    R box[3];
    R box_lo[3];  // FP32 path: box - (float)box
    double boxd[3];
    float box_dn[3];  // largest float <= L: 0 < (float)x < box_dn proves 0 < x < L
    R inv_side[3];
    int nc[3];
    int cell_off;  // first global cell of the replica
    int p_off;     // first particle slot
    int n;
};

struct BCtrlExtra {
    double *epot, *virial;  // [nrep]
};

template <typename R> struct BDev {
    int ntot, nrep, ncell;
    const RepInfo<R> *rep;
    const int *rep_of;  // [ntot] replica of each slot (static)
    double *x[2], *v[2];
    int *id[2];
    V4<R> *pos[2];  // [ntot + 1], slot ntot is a sentinel
    V4<R> *xref;
    V4<R> *force;
    int *cell_count, *cell_start, *cell_of, *slot_of, *cell_sorted, *tmp_idx, *tmp_key;
    const int *cell_rep;     // [ncell] replica of each cell (static)
    int *rep_flag;           // [nrep] a particle of the replica moved skin/2
    int *rep_do;             // [nrep] the replica is rebuilt in this event
    long long *rep_last;     // [nrep] step of the replica's last rebuild
    int interval;            // R
    uint32_t *nl;
    int *nl_count;
    int nl_cap;
    R rlist2, half_skin2;
    R sig2, e24, e48, e4, ushift, rc2lo, rc2hi, inv_mass_dt;
    double rc2d, dt, half_mass;
    Ctrl *ctrl;
    BCtrlExtra ex;
};

// ---------------------------------------------------------------------------
// Rebuild

// Which replicas this rebuild event covers; resets their flags.
template <typename R> __global__ void k_bplan(BDev<R> S) {
    Ctrl *C = S.ctrl;
    if (!C->rebuild_now) return;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= S.nrep) return;
    const long long now = C->total_steps;
    const bool go = C->rebuild_all || S.rep_flag[r] || now - S.rep_last[r] >= S.interval;
    S.rep_do[r] = go ? 1 : 0;
    if (go) {
        S.rep_flag[r] = 0;
        S.rep_last[r] = now;
        atomicAdd((unsigned long long *)&C->replica_rebuilds, 1ull);
    }
}

// Bin every particle of a replica being rebuilt into its replica's grid.  The FP64 position is first
// wrapped into the replica's box (positions drift out of it between
// rebuilds), so that the image shift a cell stencil implies is the image
// shift of the stored coordinates.
template <typename R> __global__ void k_bbin(BDev<R> S) {
    Ctrl *C = S.ctrl;
    if (!C->rebuild_now) return;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g == 0) { C->need_cap = 0; C->overflow = 0; }
    if (g >= S.ntot) return;
    const int rep = S.rep_of[g];
    if (!S.rep_do[rep]) return;
    const RepInfo<R> &I = S.rep[rep];
    double *X = S.x[C->state_par];
    int c3[3];
    bool bad = false;
    for (int d = 0; d < 3; ++d) {
        double xd = X[d * S.ntot + g];
        // FP64 arithmetic is scarce: the FP64 wrap only for particles whose
        // float rounding does not prove 0 < x < L (rounding is monotonic)
        const float xf = (float)xd;
        if (!(xf > 0.0f && xf < I.box_dn[d])) {
            const double L = I.boxd[d];
            if (!(xd == xd) || fabs(xd) > 4.0 * L) { bad = true; xd = 0.0; }
            if (xd < 0.0) xd += L;
            if (xd >= L) xd -= L;
            if (xd < 0.0 || xd >= L) { xd = xd - L * floor(xd / L); if (xd >= L) xd = 0.0; }
            X[d * S.ntot + g] = xd;
        }
        const int c = (int)floor((R)xd * I.inv_side[d]);
        c3[d] = min(max(c, 0), I.nc[d] - 1);
    }
    if (bad) C->nonfinite = 1;
    const int cell = I.cell_off + (c3[2] * I.nc[1] + c3[1]) * I.nc[0] + c3[0];
    S.cell_of[g] = cell;
    S.slot_of[g] = atomicAdd(&S.cell_count[cell], 1);
}

// Inclusive scan of one value per thread over a CTA (warp shuffles, then
// the warp totals by the first warp).
__device__ __forceinline__ int block_incl_scan(int v, int *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        sh[lane] = w;
    }
    __syncthreads();
    return v + (warp > 0 ? sh[warp - 1] : 0);
}

// Per-replica exclusive scan of the cell counts of the replicas being
// rebuilt: one CTA per replica, starting at the replica's first slot; the
// counts are cleared for the next event.  Other replicas keep their starts.
template <typename R> __global__ void __launch_bounds__(SCAN_BLOCK) k_bscan_rep(BDev<R> S) {
    Ctrl *C = S.ctrl;
    if (!C->rebuild_now) return;
    const int r = blockIdx.x;
    if (r == 0 && threadIdx.x == 0) {
        S.cell_start[S.ncell] = S.ntot;
        C->rebuild_all = 0;  // the plan kernel, which read it, has finished
    }
    if (!S.rep_do[r]) return;
    __shared__ int sh[32];
    __shared__ int total;
    const RepInfo<R> &I = S.rep[r];
    const int c0 = I.cell_off, nc = I.nc[0] * I.nc[1] * I.nc[2];
    int carry = I.p_off;
    for (int base = 0; base < nc; base += SCAN_BLOCK) {
        const int k = base + threadIdx.x;
        const int v = k < nc ? S.cell_count[c0 + k] : 0;
        const int incl = block_incl_scan(v, sh);
        if (k < nc) {
            S.cell_start[c0 + k] = carry + incl - v;
            S.cell_count[c0 + k] = 0;
        }
        if (threadIdx.x == SCAN_BLOCK - 1) total = incl;
        __syncthreads();
        carry += total;
        __syncthreads();
    }
}

template <typename R> __global__ void k_bscatter(BDev<R> S) {
    Ctrl *C = S.ctrl;
    if (!C->rebuild_now) return;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= S.ntot) return;
    if (!S.rep_do[S.rep_of[g]]) return;
    const int cell = S.cell_of[g];
    const int dst = S.cell_start[cell] + S.slot_of[g];
    S.tmp_idx[dst] = g;
    S.tmp_key[dst] = S.id[C->state_par][g];
    S.cell_sorted[dst] = cell;  // the slot's cell: its final occupant is in the same cell
}

// Gather one particle's state into its final slot q of the other state
// buffer (the slot's cell was recorded by the scatter).
template <typename R> __device__ __forceinline__ void bgather(const BDev<R> &S, int sp, int pp, int q, int p) {
    const int n = S.ntot;
    const double *X = S.x[sp], *V = S.v[sp];
    double *Xn = S.x[sp ^ 1], *Vn = S.v[sp ^ 1];
    const double x0 = X[p], x1 = X[n + p], x2 = X[2 * n + p];
    Xn[q] = x0; Xn[n + q] = x1; Xn[2 * n + q] = x2;
    Vn[q] = V[p]; Vn[n + q] = V[n + p]; Vn[2 * n + q] = V[2 * n + p];
    S.id[sp ^ 1][q] = S.id[sp][p];
    const V4<R> w = make_pos((R)x0, (R)x1, (R)x2, 0);
    S.pos[pp][q] = w;
    S.xref[q] = w;
}

// One thread per slot.  A replica not rebuilt keeps its slots: its state is
// carried over to the buffer that becomes current.  In a rebuilt replica the
// slot holds (in scattered order) an element of some cell; its rank among
// the keys (input indices) of that cell is its final place in the cell.
template <typename R> __global__ void k_bsortgather(BDev<R> S) {
    Ctrl *C = S.ctrl;
    if (!C->rebuild_now) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= S.ntot) return;
    const int sp = C->state_par, pp = C->pos_par;
    if (!S.rep_do[S.rep_of[e]]) {
        const int n = S.ntot;
        for (int d = 0; d < 3; ++d) {
            S.x[sp ^ 1][d * n + e] = S.x[sp][d * n + e];
            S.v[sp ^ 1][d * n + e] = S.v[sp][d * n + e];
        }
        S.id[sp ^ 1][e] = S.id[sp][e];
        return;
    }
    const int cell = S.cell_sorted[e];
    const int start = S.cell_start[cell], m = S.cell_start[cell + 1] - start;
    const int key = S.tmp_key[e];
    int rank = 0;
    for (int f = 0; f < m; ++f) rank += S.tmp_key[start + f] < key ? 1 : 0;
    bgather(S, sp, pp, start + rank, S.tmp_idx[e]);
}

// Verlet list of each particle (thread per slot): every j of the 27 stencil
// cells of its replica (periodic images of the replica's box) within the
// list radius.  As for a single system, each (y, z) row of the stencil is
// one run of consecutive slots (cells cx-1 .. cx+1, split only at a periodic
// x edge of the replica), tested four candidates at a time into a 32-bit
// mask per block of 32; only set bits are appended, in slot order (the order
// of a cell-by-cell walk).  Row layout as for a single system: entries
// without an image from the front in 16-byte chunks of four (the last
// padded with the sentinel slot ntot), entries with an image (j | code << 27)
// from the back; nl_count = front count | back count << 16.
template <typename R> __global__ void __launch_bounds__(128) k_bvl_build(BDev<R> S) {
    Ctrl *C = S.ctrl;
    if (!C->rebuild_now) return;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= S.ntot) return;
    if (!S.rep_do[S.rep_of[q]]) return;
    const V4<R> *P = S.pos[C->pos_par];
    const RepInfo<R> &I = S.rep[S.rep_of[q]];
    const V4<R> pi = P[q];
    const int nx = I.nc[0], ny = I.nc[1], nz = I.nc[2];
    const int lc = S.cell_sorted[q] - I.cell_off;
    const int cx = lc % nx, cy = (lc / nx) % ny, cz = lc / (nx * ny);
    const int cap = S.nl_cap;
    uint32_t *row = S.nl + (size_t)q * cap;
    uint4 *row4 = reinterpret_cast<uint4 *>(row);
    uint32_t b0 = 0, b1 = 0, b2 = 0, b3 = 0;
    int nf = 0, nb = 0;
    for (int oz = -1; oz <= 1; ++oz) {
        int wz, sz;
        wrap_cell(cz, oz, nz, wz, sz);
        for (int oy = -1; oy <= 1; ++oy) {
            int wy, sy;
            wrap_cell(cy, oy, ny, wy, sy);
            const int rowc = I.cell_off + (wz * ny + wy) * nx;
            // cells cx-1 .. cx+1 in unwrapped coordinates: left of the box
            // (image -1), inside it, right of it (image +1)
            for (int sx = -1; sx <= 1; ++sx) {
                const int a = sx < 0 ? cx - 1 : (sx == 0 ? max(cx - 1, 0) : max(cx - 1, nx));
                const int b = sx < 0 ? min(cx + 1, -1) : (sx == 0 ? min(cx + 1, nx - 1) : cx + 1);
                if (a > b) continue;
                const int jb = S.cell_start[rowc + a - sx * nx], je = S.cell_start[rowc + b - sx * nx + 1];
                const uint32_t code = encode_image(sx, sy, sz);
                const bool self = code == 0 && jb <= q && q < je;
                const R xs = pi.x - (R)sx * I.box[0], ys = pi.y - (R)sy * I.box[1], zs = pi.z - (R)sz * I.box[2];
                for (int j0 = jb; j0 < je; j0 += 32) {
                    const int m = min(32, je - j0);
                    uint32_t mask = 0;
                    int t = 0;
                    for (; t + 4 <= m; t += 4) {
                        const int j = j0 + t;
                        const V4<R> q0 = ldpos(P, j), q1 = ldpos(P, j + 1), q2 = ldpos(P, j + 2), q3 = ldpos(P, j + 3);
                        const uint32_t bits = (uint32_t)(r2_of(xs - q0.x, ys - q0.y, zs - q0.z) < S.rlist2) |
                                              ((uint32_t)(r2_of(xs - q1.x, ys - q1.y, zs - q1.z) < S.rlist2) << 1) |
                                              ((uint32_t)(r2_of(xs - q2.x, ys - q2.y, zs - q2.z) < S.rlist2) << 2) |
                                              ((uint32_t)(r2_of(xs - q3.x, ys - q3.y, zs - q3.z) < S.rlist2) << 3);
                        mask |= bits << t;
                    }
                    for (; t < m; ++t) {
                        const V4<R> qq = ldpos(P, j0 + t);
                        mask |= (uint32_t)(r2_of(xs - qq.x, ys - qq.y, zs - qq.z) < S.rlist2) << t;
                    }
                    if (self) {  // drop j == q
                        const int rel = q - j0;
                        if (rel >= 0 && rel < 32) mask &= ~(1u << rel);
                    }
                    while (mask) {
                        const int bit = __ffs(mask) - 1;
                        mask &= mask - 1;
                        const uint32_t j = (uint32_t)(j0 + bit);
                        if (code == 0) {
                            b3 = b2; b2 = b1; b1 = b0; b0 = j;
                            ++nf;
                            if ((nf & 3) == 0 && nf + nb <= cap) row4[(nf >> 2) - 1] = make_uint4(b0, b1, b2, b3);
                        } else {
                            if (nb < cap) row[cap - 1 - nb] = j | (code << JBITS);  // inside the row (see the single-system build)
                            ++nb;
                        }
                    }
                }
            }
        }
    }
    const int need = ((nf + 3) & ~3) + nb;
    if (need > cap || nf > 0xffff || nb > 0xffff) {
        atomicMax((unsigned long long *)&C->need_cap, (unsigned long long)need);
        C->overflow = 1;
        S.nl_count[q] = 0;
        return;
    }
    {
        // the longest row of the build (reported by the counters): one
        // atomic per warp over the lanes still here
        const unsigned act = __activemask();
        const unsigned m = __reduce_max_sync(act, (unsigned)need);
        if ((int)(threadIdx.x & 31) == __ffs(act) - 1 && m)
            atomicMax((unsigned long long *)&C->need_cap, (unsigned long long)m);
    }
    if (nf & 3) {
        const uint32_t sent = (uint32_t)S.ntot;
        for (int m = nf & 3; m < 4; ++m) { b3 = b2; b2 = b1; b1 = b0; b0 = sent; }
        row4[nf >> 2] = make_uint4(b0, b1, b2, b3);
    }
    S.nl_count[q] = nf | (nb << 16);
}

// ---------------------------------------------------------------------------
// Forces and the Stormer-Verlet update

enum { BMODE_FORCE = 0, BMODE_STEP = 1, BMODE_PAIRS = 2 };

template <typename R, int G> __device__ __forceinline__ R gsum(R v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Group of G lanes per particle; the grid either covers every particle once
// or (persistent) strides over groups of particles.
template <typename R, int G, int MODE, bool EV>
__global__ void __launch_bounds__(256) k_bforce(BDev<R> S, int2 *pairs3, long long cap, int *pair_rep) {
    Ctrl *C = S.ctrl;
    if (C->overflow) return;
    const int pp = C->pos_par, sp = C->state_par;
    const V4<R> *P = S.pos[pp];
    const int lanes = gridDim.x * blockDim.x;
    const int gid0 = blockIdx.x * blockDim.x + threadIdx.x;
    bool exceeded = false, bad = false;
    // all lanes of a warp run the same number of rounds (shuffles inside)
    const int rounds = (int)(((long long)S.ntot * G + lanes - 1) / lanes);
    for (int rd = 0; rd < rounds; ++rd) {
        const long long gid = (long long)rd * lanes + gid0;
        const int i = (int)(gid / G), sub = (int)(gid % G);
        const bool valid = i < S.ntot;
        R fx = 0, fy = 0, fz = 0, u = 0, w = 0;
        int rep = 0;
        if (valid) {
            rep = S.rep_of[i];
            const RepInfo<R> &I = S.rep[rep];
            const V4<R> pi = P[i];
            const uint32_t *row = S.nl + (size_t)i * S.nl_cap;
            const uint4 *row4 = reinterpret_cast<const uint4 *>(row);
            const int cnt = S.nl_count[i];
            int nq = ((cnt & 0xffff) + 3) >> 2, nb = cnt >> 16;
            if (!lj_check(4 * nq + nb <= S.nl_cap, C, CHECK_BATCH_ENTRY)) { nq = 0; nb = 0; }
            auto pair = [&](int j, int sx, int sy, int sz, R dx, R dy, R dz, const V4<R> &pj) {
                const R r2 = r2_of(dx, dy, dz);
                const bool in = Cut<R>::in(r2, S.rc2lo, S.rc2hi, pi, pj, sx, sy, sz, I.boxd, S.rc2d);
                if (MODE == BMODE_PAIRS) {
                    if (in && S.id[sp][i] < S.id[sp][j]) {
                        const unsigned long long slot = atomicAdd(&C->npairs, 1ull);
                        if ((long long)slot < cap) {
                            pairs3[slot] = make_int2(S.id[sp][i] - I.p_off, S.id[sp][j] - I.p_off);
                            pair_rep[slot] = rep;
                        }
                    }
                    return;
                }
                R sr6;
                R fr = lj_fr(r2, S.sig2, S.e24, S.e48, sr6);
                fr = in ? fr : (R)0;
                fx += fr * dx; fy += fr * dy; fz += fr * dz;
                if (EV) {
                    u += in ? S.e4 * sr6 * (sr6 - (R)1) - S.ushift : (R)0;
                    w += fr * r2;
                }
            };
            // entries without an image: four at a time (padded with the sentinel)
            for (int k = sub; k < nq; k += G) {
                uint4 e = __ldg(row4 + k);
                const unsigned nn = (unsigned)S.ntot;  // the sentinel ntot pads the front
                if (!lj_check(e.x <= nn && e.y <= nn && e.z <= nn && e.w <= nn, C, CHECK_BATCH_ENTRY))
                    e = make_uint4(nn, nn, nn, nn);
                const V4<R> p0 = P[e.x], p1 = P[e.y], p2 = P[e.z], p3 = P[e.w];
                pair((int)e.x, 0, 0, 0, pi.x - p0.x, pi.y - p0.y, pi.z - p0.z, p0);
                pair((int)e.y, 0, 0, 0, pi.x - p1.x, pi.y - p1.y, pi.z - p1.z, p1);
                pair((int)e.z, 0, 0, 0, pi.x - p2.x, pi.y - p2.y, pi.z - p2.z, p2);
                pair((int)e.w, 0, 0, 0, pi.x - p3.x, pi.y - p3.y, pi.z - p3.z, p3);
            }
            // entries with a periodic image: the exact image arithmetic
            for (int k = sub; k < nb; k += G) {
                const uint32_t e = row[S.nl_cap - 1 - k];
                const int j = (int)(e & JMASK);
                if (!lj_check(j < S.ntot, C, CHECK_BATCH_ENTRY)) break;
                int sx, sy, sz;
                decode_image(e >> JBITS, sx, sy, sz);
                const V4<R> pj = P[j];
                pair(j, sx, sy, sz, image_dx(pi.x, pj.x, sx, I.box[0], I.box_lo[0]),
                     image_dx(pi.y, pj.y, sy, I.box[1], I.box_lo[1]), image_dx(pi.z, pj.z, sz, I.box[2], I.box_lo[2]),
                     pj);
            }
        }
        if (MODE == BMODE_PAIRS) continue;
        fx = gsum<R, G>(fx); fy = gsum<R, G>(fy); fz = gsum<R, G>(fz);
        if (EV) { u = gsum<R, G>(u); w = gsum<R, G>(w); }
        if (!valid || sub != 0) continue;
        if (MODE == BMODE_FORCE) {
            S.force[i] = make_pos(fx, fy, fz, 0);
            if (EV) {
                atomicAdd(&S.ex.epot[rep], 0.5 * (double)u);
                atomicAdd(&S.ex.virial[rep], 0.5 * (double)w);
            }
            continue;
        }
        // leapfrog Stormer-Verlet: v += (dt/m) F (dt/2m at the integer step),
        // x += dt v; every load before the stores (which may alias them as
        // far as the compiler knows), the FP32 <-> FP64 conversions on the
        // integer pipes
        const int n = S.ntot;
        double *X = S.x[sp], *V = S.v[sp];
        const double v0x = V[i], v0y = V[n + i], v0z = V[2 * n + i];
        const double x0 = X[i], y0 = X[n + i], z0 = X[2 * n + i];
        const V4<R> r0 = S.xref[i];
        R c = S.inv_mass_dt;
        if (C->half_kick) c *= (R)0.5;
        double vx, vy, vz;
        if constexpr (sizeof(R) == 4) {
            vx = v0x + f32_to_f64(c * fx); vy = v0y + f32_to_f64(c * fy); vz = v0z + f32_to_f64(c * fz);
        } else {
            vx = v0x + c * fx; vy = v0y + c * fy; vz = v0z + c * fz;
        }
        const double x = fma(S.dt, vx, x0), y = fma(S.dt, vy, y0), z = fma(S.dt, vz, z0);
        V[i] = vx; V[n + i] = vy; V[2 * n + i] = vz;
        X[i] = x; X[n + i] = y; X[2 * n + i] = z;
        V4<R> nw;
        if constexpr (sizeof(R) == 4) nw = make_pos(f64_to_f32(x), f64_to_f32(y), f64_to_f32(z), 0);
        else nw = make_pos(x, y, z, 0);
        S.pos[pp ^ 1][i] = nw;
        const R ddx = nw.x - r0.x, ddy = nw.y - r0.y, ddz = nw.z - r0.z;
        if (!(ddx * ddx + ddy * ddy + ddz * ddz < S.half_skin2)) {
            exceeded = true;
            S.rep_flag[rep] = 1;
        }
        bad = bad || !isfinite(fx + fy + fz);
    }
    if (MODE == BMODE_STEP) {
        if (__any_sync(0xffffffffu, exceeded) && (threadIdx.x & 31) == 0) C->disp_exceeded = 1;
        if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) C->nonfinite = 1;
    }
}

template <typename R> __global__ void k_bimport(BDev<R> S, const double *pos, const double *vel, int init) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g > S.ntot) return;
    Ctrl *C = S.ctrl;
    const int sp = C->state_par, pp = C->pos_par, n = S.ntot;
    if (g == S.ntot) {  // sentinel slot of both working buffers
        const V4<R> far = make_pos((R)1e18, (R)1e18, (R)1e18, 0);
        S.pos[0][n] = far;
        S.pos[1][n] = far;
        return;
    }
    if (init) S.id[sp][g] = g;
    const int id = S.id[sp][g];
    double x[3];
    for (int d = 0; d < 3; ++d) {
        if (pos) S.x[sp][d * n + g] = pos[3 * id + d];
        if (vel) S.v[sp][d * n + g] = vel[3 * id + d];
        x[d] = S.x[sp][d * n + g];
    }
    const V4<R> w = make_pos((R)x[0], (R)x[1], (R)x[2], 0);
    S.pos[pp][g] = w;
    S.xref[g] = w;
}

template <typename R> __global__ void k_bexport(BDev<R> S, double *pos, double *vel, double *force, int wrap) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= S.ntot) return;
    const int sp = S.ctrl->state_par, n = S.ntot;
    const int id = S.id[sp][g];
    const RepInfo<R> &I = S.rep[S.rep_of[g]];
    for (int d = 0; d < 3; ++d) {
        if (pos) {
            double x = S.x[sp][d * n + g];
            if (wrap) {
                const double L = I.boxd[d];
                x = x - L * floor(x / L);
                if (x >= L) x = 0.0;
            }
            pos[3 * id + d] = x;
        }
        if (vel) vel[3 * id + d] = S.v[sp][d * n + g];
    }
    if (force) {
        const V4<R> f = S.force[g];
        force[3 * id + 0] = (double)f.x; force[3 * id + 1] = (double)f.y; force[3 * id + 2] = (double)f.z;
    }
}

// v += (dt/2m) F: velocities to the integer step after a force evaluation.
template <typename R> __global__ void k_bsync(BDev<R> S) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= S.ntot) return;
    const int sp = S.ctrl->state_par, n = S.ntot;
    const V4<R> f = S.force[g];
    const R c = S.inv_mass_dt * (R)0.5;
    S.v[sp][g] += (double)(c * f.x);
    S.v[sp][n + g] += (double)(c * f.y);
    S.v[sp][2 * n + g] += (double)(c * f.z);
}

__global__ void k_bcmd(Ctrl *C, int op, long long a) {
    switch (op) {
        case CMD_REBUILD: C->rebuild_now = 1; C->rebuild_all = 1; break;
        case CMD_BEGIN: C->steps_done = 0; C->steps_target = a; break;
        case CMD_RESET_PAIRS: C->npairs = 0; break;
        case CMD_HALF_KICK: C->half_kick = (int)a; break;
        case CMD_CLEAR: C->overflow = 0; C->need_cap = 0; C->disp_exceeded = 0; break;
        case CMD_INTERVAL: C->rebuild_interval = (int)a; break;
    }
}

// ---------------------------------------------------------------------------
// Host side

struct Tile {
    int tpp = 1;         // lanes per particle (1, 2, 4, 8)
    int block = 128;     // threads per CTA (64, 128, 256)
    int persistent = 0;  // CTAs per SM of a persistent grid (0: one lane group per particle)
};

struct BGraph {
    Tile tile;
    int interval = 0;
    std::vector<unsigned char> key;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace

struct ljsel_batch_s {
    ljsel_params params{};
    int precision = 0;
    int nrep = 0, ntot = 0, ncell = 0, nl_cap = 0, interval = 10, nsm = 152;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    Tile tile;
    std::vector<int> counts, p_off, cell_off;
    std::vector<double> boxes;
    Buf b_rep, b_rep_of, b_x[2], b_v[2], b_id[2], b_pos[2], b_xref, b_force, b_cell_count, b_cell_start, b_cell_of,
        b_slot_of, b_cell_sorted, b_tmp_idx, b_tmp_key, b_nl, b_nl_count, b_ctrl, b_ev, b_io, b_cell_rep,
        b_rep_flag, b_rep_do, b_rep_last;
    Ctrl *h_ctrl = nullptr;
    bool synced = true;
    long long retries = 0;
    std::vector<BGraph> graphs;

    ~ljsel_batch_s() {
        for (BGraph &g : graphs) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            if (g.graph) cudaGraphDestroy(g.graph);
        }
        for (Buf *b : bufs()) b->release();
        if (h_ctrl) cudaFreeHost(h_ctrl);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
    std::vector<Buf *> bufs() {
        return {&b_rep, &b_rep_of, &b_x[0], &b_x[1], &b_v[0], &b_v[1], &b_id[0], &b_id[1], &b_pos[0], &b_pos[1],
                &b_xref, &b_force, &b_cell_count, &b_cell_start, &b_cell_of, &b_slot_of, &b_cell_sorted, &b_tmp_idx,
                &b_tmp_key, &b_nl, &b_nl_count, &b_ctrl, &b_ev, &b_io, &b_cell_rep, &b_rep_flag, &b_rep_do, &b_rep_last};
    }
    size_t p4() const { return precision ? sizeof(D4) : sizeof(float4); }

    template <typename R> void fill(BDev<R> &S) const {
        memset(&S, 0, sizeof(S));
        S.ntot = ntot;
        S.nrep = nrep;
        S.ncell = ncell;
        S.rep = (const RepInfo<R> *)b_rep.ptr;
        S.rep_of = (const int *)b_rep_of.ptr;
        for (int k = 0; k < 2; ++k) {
            S.x[k] = (double *)b_x[k].ptr;
            S.v[k] = (double *)b_v[k].ptr;
            S.id[k] = (int *)b_id[k].ptr;
            S.pos[k] = (V4<R> *)b_pos[k].ptr;
        }
        S.xref = (V4<R> *)b_xref.ptr;
        S.force = (V4<R> *)b_force.ptr;
        S.cell_count = (int *)b_cell_count.ptr;
        S.cell_start = (int *)b_cell_start.ptr;
        S.cell_of = (int *)b_cell_of.ptr;
        S.slot_of = (int *)b_slot_of.ptr;
        S.cell_sorted = (int *)b_cell_sorted.ptr;
        S.tmp_idx = (int *)b_tmp_idx.ptr;
        S.tmp_key = (int *)b_tmp_key.ptr;
        S.cell_rep = (const int *)b_cell_rep.ptr;
        S.rep_flag = (int *)b_rep_flag.ptr;
        S.rep_do = (int *)b_rep_do.ptr;
        S.rep_last = (long long *)b_rep_last.ptr;
        S.interval = interval;
        S.nl = (uint32_t *)b_nl.ptr;
        S.nl_count = (int *)b_nl_count.ptr;
        S.nl_cap = nl_cap;
        const double rc = params.rcut[0], sg = params.sigma[0], e = params.eps[0];
        const double rl = (rc + params.skin) * (1.0 + 1.0 / 4096.0);
        S.rlist2 = (R)(rl * rl);
        S.half_skin2 = (R)(0.25 * params.skin * params.skin);
        const double sr = sg / rc, sr6 = sr * sr * sr * sr * sr * sr;
        S.sig2 = (R)(sg * sg);
        S.e24 = (R)(24.0 * e);
        S.e48 = (R)(48.0 * e);
        S.e4 = (R)(4.0 * e);
        S.ushift = params.shift_potential ? (R)(4.0 * e * (sr6 * sr6 - sr6)) : (R)0;
        S.rc2d = rc * rc;
        S.rc2lo = (R)(rc * rc * (1.0 - 1.0 / 16384.0));
        S.rc2hi = (R)(rc * rc * (1.0 + 1.0 / 16384.0));
        S.inv_mass_dt = (R)(params.dt / params.mass[0]);
        S.dt = params.dt;
        S.half_mass = 0.5 * params.mass[0];
        S.ctrl = (Ctrl *)b_ctrl.ptr;
        S.ex.epot = (double *)b_ev.ptr;
        S.ex.virial = (double *)b_ev.ptr + nrep;
    }

    ljsel_status cmd(int op, long long a) {
        k_bcmd<<<1, 1, 0, stream>>>((Ctrl *)b_ctrl.ptr, op, a);
        CK(cudaGetLastError());
        return LJSEL_OK;
    }
    ljsel_status read_ctrl() {
        CK(cudaMemcpyAsync(h_ctrl, b_ctrl.ptr, sizeof(Ctrl), cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        if (h_ctrl->nonfinite) { set_error("non-finite position, velocity or force"); return LJSEL_ERR_NONFINITE; }
        if (h_ctrl->check_failed) {
            set_error("bounds check failed at site " + std::to_string(h_ctrl->check_site) + " (checked build)");
            return LJSEL_ERR_STATE;
        }
        return LJSEL_OK;
    }

    template <typename R> void enqueue_rebuild(const BDev<R> &S, cudaStream_t st) const {
        k_bplan<R><<<div_up(nrep, 256), 256, 0, st>>>(S);
        k_bbin<R><<<div_up(ntot, 256), 256, 0, st>>>(S);
        k_bscan_rep<R><<<nrep, SCAN_BLOCK, 0, st>>>(S);
        k_bscatter<R><<<div_up(ntot, 256), 256, 0, st>>>(S);
        k_bsortgather<R><<<div_up(ntot, 256), 256, 0, st>>>(S);
        k_bvl_build<R><<<div_up(ntot, 128), 128, 0, st>>>(S);
        launch_rebuild_finish(S.ctrl, st);
    }

    template <typename R, int MODE, bool EV>
    void force_launch(const BDev<R> &S, const Tile &t, cudaStream_t st, int2 *pairs = nullptr, long long cap = 0,
                      int *prep = nullptr) const {
        const long long lanes_needed = (long long)ntot * t.tpp;
        int grid = div_up(lanes_needed, t.block);
        if (t.persistent > 0) grid = std::min(grid, nsm * t.persistent);
        grid = std::max(grid, 1);
        switch (t.tpp) {
            case 1: k_bforce<R, 1, MODE, EV><<<grid, t.block, 0, st>>>(S, pairs, cap, prep); break;
            case 2: k_bforce<R, 2, MODE, EV><<<grid, t.block, 0, st>>>(S, pairs, cap, prep); break;
            case 4: k_bforce<R, 4, MODE, EV><<<grid, t.block, 0, st>>>(S, pairs, cap, prep); break;
            default: k_bforce<R, 8, MODE, EV><<<grid, t.block, 0, st>>>(S, pairs, cap, prep); break;
        }
    }

    template <typename R> ljsel_status ensure_structure() {
        for (int attempt = 0; attempt < 8; ++attempt) {
            BDev<R> S;
            fill(S);
            enqueue_rebuild(S, stream);
            CK(cudaGetLastError());
            TRY(read_ctrl());
            if (!h_ctrl->overflow) return LJSEL_OK;
            TRY(grow());
        }
        set_error("batch neighbour lists keep overflowing");
        return LJSEL_ERR_CAPACITY;
    }

    // Row capacity set by the caller; the rows are rebuilt before the next step.
    ljsel_status set_capacity(int cap) {
        nl_cap = (cap + 3) & ~3;
        TRY(b_nl.ensure((size_t)nl_cap * ntot * 4));
        drop_graphs();
        TRY(cmd(CMD_CLEAR, 0));
        TRY(cmd(CMD_REBUILD, 0));
        return LJSEL_OK;
    }

    ljsel_status grow() {
        const long long need = h_ctrl->need_cap;
        nl_cap = (int)((std::max<long long>(need + need / 5 + 8, nl_cap + 16) + 3) & ~3LL);
        retries += 1;
        if (retries > 64) { set_error("batch neighbour lists keep overflowing"); return LJSEL_ERR_CAPACITY; }
        TRY(b_nl.ensure((size_t)nl_cap * ntot * 4));
        drop_graphs();
        TRY(cmd(CMD_CLEAR, 0));
        TRY(cmd(CMD_REBUILD, 0));
        return LJSEL_OK;
    }

    void drop_graphs() {
        for (BGraph &g : graphs) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            if (g.graph) cudaGraphDestroy(g.graph);
        }
        graphs.clear();
    }

    template <typename R> ljsel_status get_graph(cudaGraphExec_t *out) {
        BDev<R> S;
        fill(S);
        const unsigned char *kb = reinterpret_cast<const unsigned char *>(&S);
        for (BGraph &g : graphs)
            if (g.tile.tpp == tile.tpp && g.tile.block == tile.block && g.tile.persistent == tile.persistent &&
                g.interval == interval && g.key.size() == sizeof(S) && memcmp(g.key.data(), kb, sizeof(S)) == 0) {
                *out = g.exec;
                return LJSEL_OK;
            }
        if (!cap_stream) CK(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
        BGraph e;
        e.tile = tile;
        e.interval = interval;
        e.key.assign(kb, kb + sizeof(S));
        cudaGraph_t graph = nullptr;
        CK(cudaGraphCreate(&graph, 0));
        auto fail = [&](cudaError_t err) {
            cudaGraphDestroy(graph);
            set_error(std::string("building the batch step graph failed: ") + cudaGetErrorString(err));
            return LJSEL_ERR_CUDA;
        };
#define G_CK(call)                              \
    do {                                        \
        cudaError_t e_ = (call);                \
        if (e_ != cudaSuccess) return fail(e_); \
    } while (0)
        cudaGraphConditionalHandle h_loop, h_reb;
        G_CK(cudaGraphConditionalHandleCreate(&h_loop, graph, 0, cudaGraphCondAssignDefault));
        G_CK(cudaGraphConditionalHandleCreate(&h_reb, graph, 0, cudaGraphCondAssignDefault));
        G_CK(cudaStreamBeginCaptureToGraph(cap_stream, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        launch_loop_init(S.ctrl, h_reb, h_loop, cap_stream);
        cudaGraph_t tmp = nullptr;
        G_CK(cudaStreamEndCapture(cap_stream, &tmp));
        size_t nn = 0;
        G_CK(cudaGraphGetNodes(graph, nullptr, &nn));
        std::vector<cudaGraphNode_t> nodes(nn);
        G_CK(cudaGraphGetNodes(graph, nodes.data(), &nn));
        if (nn != 1) { cudaGraphDestroy(graph); set_error("unexpected node count in the batch graph"); return LJSEL_ERR_CUDA; }
        cudaGraphNodeParams wp = {};
        wp.type = cudaGraphNodeTypeConditional;
        wp.conditional.handle = h_loop;
        wp.conditional.type = cudaGraphCondTypeWhile;
        wp.conditional.size = 1;
        cudaGraphNode_t wnode;
        G_CK(cudaGraphAddNode(&wnode, graph, nodes.data(), nullptr, 1, &wp));
        cudaGraph_t body = wp.conditional.phGraph_out[0];
        cudaGraphNodeParams ip = {};
        ip.type = cudaGraphNodeTypeConditional;
        ip.conditional.handle = h_reb;
        ip.conditional.type = cudaGraphCondTypeIf;
        ip.conditional.size = 1;
        cudaGraphNode_t inode;
        G_CK(cudaGraphAddNode(&inode, body, nullptr, nullptr, 0, &ip));
        cudaGraph_t rbody = ip.conditional.phGraph_out[0];
        G_CK(cudaStreamBeginCaptureToGraph(cap_stream, rbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        enqueue_rebuild(S, cap_stream);
        G_CK(cudaStreamEndCapture(cap_stream, &tmp));
        G_CK(cudaStreamBeginCaptureToGraph(cap_stream, body, &inode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
        force_launch<R, BMODE_STEP, false>(S, tile, cap_stream);
        launch_control(S.ctrl, h_reb, h_loop, 1, cap_stream);
        G_CK(cudaStreamEndCapture(cap_stream, &tmp));
        G_CK(cudaGraphInstantiate(&e.exec, graph, 0));
#undef G_CK
        e.graph = graph;
        if (graphs.size() >= 32) {
            cudaGraphExecDestroy(graphs.front().exec);
            cudaGraphDestroy(graphs.front().graph);
            graphs.erase(graphs.begin());
        }
        graphs.push_back(e);
        *out = e.exec;
        return LJSEL_OK;
    }

    template <typename R> ljsel_status advance(long long nsteps, bool eager) {
        if (nsteps <= 0) return LJSEL_OK;
        TRY(ensure_structure<R>());
        long long left = nsteps;
        for (int round = 0; round < 16 && left > 0; ++round) {
            TRY(cmd(CMD_BEGIN, left));
            if (params.use_graphs && !eager) {
                cudaGraphExec_t ex = nullptr;
                TRY(get_graph<R>(&ex));
                CK(cudaGraphLaunch(ex, stream));
            } else {
                BDev<R> S;
                fill(S);
                for (long long k = 0; k < left; ++k) {
                    enqueue_rebuild(S, stream);
                    force_launch<R, BMODE_STEP, false>(S, tile, stream);
                    launch_control(S.ctrl, 0, 0, 0, stream);
                }
            }
            CK(cudaGetLastError());
            TRY(read_ctrl());
            left -= h_ctrl->steps_done;
            if (h_ctrl->overflow) {
                TRY(grow());
                TRY(ensure_structure<R>());
            }
        }
        synced = false;
        if (left > 0) { set_error("could not complete the requested steps"); return LJSEL_ERR_CAPACITY; }
        return LJSEL_OK;
    }

    template <typename R> ljsel_status compute(bool ev) {
        TRY(ensure_structure<R>());
        BDev<R> S;
        fill(S);
        CK(cudaMemsetAsync(b_ev.ptr, 0, 2 * (size_t)std::max(nrep, 1) * sizeof(double), stream));
        if (ev) force_launch<R, BMODE_FORCE, true>(S, tile, stream);
        else force_launch<R, BMODE_FORCE, false>(S, tile, stream);
        CK(cudaGetLastError());
        return LJSEL_OK;
    }

    template <typename R> ljsel_status sync_velocities() {
        if (synced) return LJSEL_OK;
        TRY(compute<R>(false));
        BDev<R> S;
        fill(S);
        k_bsync<R><<<div_up(ntot, 256), 256, 0, stream>>>(S);
        TRY(cmd(CMD_HALF_KICK, 1));
        CK(cudaGetLastError());
        synced = true;
        return LJSEL_OK;
    }
};

namespace {

template <typename F> ljsel_status bdispatch(ljsel_batch_s *b, F &&f) {
    if (b->precision) return f((double)0);
    return f((float)0);
}

template <typename R> ljsel_status fill_reps(ljsel_batch_s *b) {
    std::vector<RepInfo<R>> h(b->nrep);
    const double rl = (b->params.rcut[0] + b->params.skin) * (1.0 + 1.0 / 4096.0);
    const double side_min = rl * (1.0 + 1.0 / 4096.0);
    b->cell_off.assign(b->nrep + 1, 0);
    for (int r = 0; r < b->nrep; ++r) {
        RepInfo<R> &I = h[r];
        int nc = 1;
        for (int d = 0; d < 3; ++d) {
            const double L = b->boxes[3 * r + d];
            I.nc[d] = std::max(1, (int)std::floor(L / side_min));
            I.box[d] = (R)L;
            I.box_lo[d] = (R)(L - (double)(R)L);
            I.boxd[d] = L;
            float lf = (float)L;
            if ((double)lf > L) lf = std::nextafter(lf, 0.0f);
            I.box_dn[d] = lf;
            I.inv_side[d] = (R)(I.nc[d] / L);
            nc *= I.nc[d];
        }
        I.cell_off = b->cell_off[r];
        I.p_off = b->p_off[r];
        I.n = b->counts[r];
        b->cell_off[r + 1] = b->cell_off[r] + nc;
    }
    b->ncell = b->cell_off[b->nrep];
    TRY(b->b_rep.ensure(sizeof(RepInfo<R>) * std::max(b->nrep, 1)));
    CK(cudaMemcpy(b->b_rep.ptr, h.data(), sizeof(RepInfo<R>) * b->nrep, cudaMemcpyHostToDevice));
    return LJSEL_OK;
}

}  // namespace

extern "C" {

ljsel_status ljsel_batch_create(const ljsel_params *params, int32_t nrep, const double *boxes, const int64_t *counts,
                                const double *pos, const double *vel, int32_t on_device, void *stream,
                                ljsel_batch *out) {
    set_error("");
    if (!out) { set_error("out is NULL"); return LJSEL_ERR_ARG; }
    *out = nullptr;
    if (!params || nrep < 1 || !boxes || !counts) { set_error("params, nrep >= 1, boxes and counts are required"); return LJSEL_ERR_ARG; }
    if (params->ntypes != 1) { set_error("batched replicas hold a single species (ntypes = 1)"); return LJSEL_ERR_UNSUPPORTED; }
    if (params->walls[0] || params->walls[1] || params->walls[2]) {
        set_error("batched replicas are periodic");
        return LJSEL_ERR_UNSUPPORTED;
    }
    long long ntot = 0;
    for (int r = 0; r < nrep; ++r) {
        if (counts[r] < 0) { set_error("replica counts must be >= 0"); return LJSEL_ERR_ARG; }
        ntot += counts[r];
        ljsel_params p = *params;
        for (int d = 0; d < 3; ++d) p.box[d] = boxes[3 * r + d];
        TRY(validate_params(&p));
    }
    if (ntot < 1 || ntot >= (long long)JMASK) { set_error("total particles must be in [1, 2^27)"); return LJSEL_ERR_ARG; }
    if (!pos || !vel) { set_error("pos and vel are required"); return LJSEL_ERR_ARG; }
    ljsel_batch_s *b = new (std::nothrow) ljsel_batch_s();
    if (!b) { set_error("host allocation failed"); return LJSEL_ERR_OOM; }
    auto fail = [&](ljsel_status st) { delete b; return st; };
    b->params = *params;
    b->precision = params->precision;
    b->nrep = nrep;
    b->ntot = (int)ntot;
    b->stream = (cudaStream_t)stream;
    b->interval = params->skin > 0 ? 10 : 1;
    b->boxes.assign(boxes, boxes + 3 * (size_t)nrep);
    b->counts.resize(nrep);
    b->p_off.assign(nrep + 1, 0);
    for (int r = 0; r < nrep; ++r) {
        b->counts[r] = (int)counts[r];
        b->p_off[r + 1] = b->p_off[r] + (int)counts[r];
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (cudaHostAlloc((void **)&b->h_ctrl, sizeof(Ctrl), cudaHostAllocDefault) != cudaSuccess) {
        set_error("pinned allocation failed");
        return fail(LJSEL_ERR_CUDA);
    }
    memset(b->h_ctrl, 0, sizeof(Ctrl));
    ljsel_status st = bdispatch(b, [&](auto z) { return fill_reps<decltype(z)>(b); });
    if (st != LJSEL_OK) return fail(st);
    // list capacity from the densest replica, with room
    double rho_max = 0;
    for (int r = 0; r < nrep; ++r)
        rho_max = std::max(rho_max, counts[r] / (boxes[3 * r] * boxes[3 * r + 1] * boxes[3 * r + 2]));
    const double rl = params->rcut[0] + params->skin;
    b->nl_cap = ((int)std::min(4.18879 * rl * rl * rl * rho_max * 1.35 + 16, 4096.0) + 3) & ~3;
    const size_t n = (size_t)ntot, n3 = n * 3 * sizeof(double);
    std::vector<int> rep_of(n);
    for (int r = 0; r < nrep; ++r)
        for (int k = b->p_off[r]; k < b->p_off[r + 1]; ++k) rep_of[k] = r;
    const size_t cells1 = (size_t)b->ncell + 1;
    struct { Buf *b; size_t bytes; } plan[] = {
        {&b->b_rep_of, n * 4}, {&b->b_x[0], n3}, {&b->b_x[1], n3}, {&b->b_v[0], n3}, {&b->b_v[1], n3},
        {&b->b_id[0], n * 4}, {&b->b_id[1], n * 4}, {&b->b_pos[0], (n + 1) * b->p4()}, {&b->b_pos[1], (n + 1) * b->p4()},
        {&b->b_xref, n * b->p4()}, {&b->b_force, n * b->p4()}, {&b->b_cell_count, cells1 * 4},
        {&b->b_cell_start, cells1 * 4}, {&b->b_cell_of, n * 4}, {&b->b_slot_of, n * 4}, {&b->b_cell_sorted, n * 4},
        {&b->b_tmp_idx, n * 4}, {&b->b_tmp_key, n * 4}, {&b->b_cell_rep, cells1 * 4},
        {&b->b_rep_flag, (size_t)nrep * 4}, {&b->b_rep_do, (size_t)nrep * 4}, {&b->b_rep_last, (size_t)nrep * 8},
        {&b->b_nl, (size_t)b->nl_cap * n * 4}, {&b->b_nl_count, n * 4}, {&b->b_ctrl, sizeof(Ctrl)},
        {&b->b_ev, 2 * (size_t)nrep * sizeof(double)}};
    for (auto &p : plan)
        if ((st = p.b->ensure(p.bytes)) != LJSEL_OK) return fail(st);
    std::vector<int> cell_rep(cells1, nrep - 1);
    for (int r = 0; r < nrep; ++r)
        for (int c = b->cell_off[r]; c < b->cell_off[r + 1]; ++c) cell_rep[c] = r;
    if (cudaMemcpy(b->b_rep_of.ptr, rep_of.data(), n * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->b_cell_rep.ptr, cell_rep.data(), cells1 * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->b_rep_flag.ptr, 0, (size_t)nrep * 4) != cudaSuccess ||
        cudaMemset(b->b_rep_do.ptr, 0, (size_t)nrep * 4) != cudaSuccess ||
        cudaMemset(b->b_rep_last.ptr, 0, (size_t)nrep * 8) != cudaSuccess ||
        cudaMemset(b->b_cell_count.ptr, 0, cells1 * 4) != cudaSuccess ||
        cudaMemset(b->b_ctrl.ptr, 0, sizeof(Ctrl)) != cudaSuccess ||
        cudaMemset(b->b_nl_count.ptr, 0, n * 4) != cudaSuccess) {
        set_error("batch initialisation copies failed");
        return fail(LJSEL_ERR_CUDA);
    }
    const double *dp = pos, *dv = vel;
    if (!on_device) {
        if ((st = b->b_io.ensure(2 * n3)) != LJSEL_OK) return fail(st);
        if (cudaMemcpy(b->b_io.ptr, pos, n3, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy((char *)b->b_io.ptr + n3, vel, n3, cudaMemcpyHostToDevice) != cudaSuccess) {
            set_error("input copy failed");
            return fail(LJSEL_ERR_CUDA);
        }
        dp = (const double *)b->b_io.ptr;
        dv = (const double *)((char *)b->b_io.ptr + n3);
    }
    st = bdispatch(b, [&](auto z) -> ljsel_status {
        using R = decltype(z);
        BDev<R> S;
        b->fill(S);
        k_bimport<R><<<div_up(b->ntot + 1, 256), 256, 0, b->stream>>>(S, dp, dv, 1);
        CK(cudaGetLastError());
        return LJSEL_OK;
    });
    if (st == LJSEL_OK) st = b->cmd(CMD_INTERVAL, b->interval);
    if (st == LJSEL_OK) st = b->cmd(CMD_REBUILD, 0);
    if (st == LJSEL_OK) st = b->cmd(CMD_HALF_KICK, 1);
    if (st == LJSEL_OK && cudaStreamSynchronize(b->stream) != cudaSuccess) {
        set_error(cudaGetErrorString(cudaGetLastError()));
        st = LJSEL_ERR_CUDA;
    }
    if (st != LJSEL_OK) return fail(st);
    *out = b;
    return LJSEL_OK;
}

ljsel_status ljsel_batch_destroy(ljsel_batch b) {
    if (!b) return LJSEL_OK;
    cudaStreamSynchronize(b->stream);
    delete b;
    return LJSEL_OK;
}

ljsel_status ljsel_batch_set_tile(ljsel_batch b, const ljsel_batch_tile *t) {
    if (!b || !t) { set_error("NULL argument"); return LJSEL_ERR_ARG; }
    const bool ok_tpp = t->threads_per_particle == 1 || t->threads_per_particle == 2 || t->threads_per_particle == 4 ||
                        t->threads_per_particle == 8;
    const bool ok_blk = t->block_threads == 64 || t->block_threads == 128 || t->block_threads == 256;
    if (!ok_tpp || !ok_blk || t->persistent_ctas_per_sm < 0 || t->persistent_ctas_per_sm > 32) {
        set_error("tile: threads_per_particle in {1,2,4,8}, block_threads in {64,128,256}, persistent 0..32");
        return LJSEL_ERR_UNSUPPORTED;
    }
    if (t->rebuild_interval < 1 || (b->params.skin == 0.0 && t->rebuild_interval != 1)) {
        set_error("rebuild_interval must be >= 1 (1 without a skin)");
        return LJSEL_ERR_ARG;
    }
    b->tile.tpp = t->threads_per_particle;
    b->tile.block = t->block_threads;
    b->tile.persistent = t->persistent_ctas_per_sm;
    if (t->rebuild_interval != b->interval) {
        b->interval = t->rebuild_interval;
        TRY(b->cmd(CMD_INTERVAL, b->interval));
    }
    return LJSEL_OK;
}

ljsel_status ljsel_batch_get_tile(ljsel_batch b, ljsel_batch_tile *t) {
    if (!b || !t) { set_error("NULL argument"); return LJSEL_ERR_ARG; }
    t->threads_per_particle = b->tile.tpp;
    t->block_threads = b->tile.block;
    t->persistent_ctas_per_sm = b->tile.persistent;
    t->rebuild_interval = b->interval;
    return LJSEL_OK;
}

ljsel_status ljsel_batch_step(ljsel_batch b, int64_t nsteps) {
    if (!b) { set_error("NULL handle"); return LJSEL_ERR_ARG; }
    if (nsteps < 0) { set_error("nsteps must be >= 0"); return LJSEL_ERR_ARG; }
    return bdispatch(b, [&](auto z) { return b->advance<decltype(z)>(nsteps, false); });
}

ljsel_status ljsel_batch_step_eager(ljsel_batch b, int64_t nsteps) {
    if (!b) { set_error("NULL handle"); return LJSEL_ERR_ARG; }
    if (nsteps < 0) { set_error("nsteps must be >= 0"); return LJSEL_ERR_ARG; }
    return bdispatch(b, [&](auto z) { return b->advance<decltype(z)>(nsteps, true); });
}

ljsel_status ljsel_batch_compute(ljsel_batch b, double *forces, int32_t on_device, double *energy, double *virial) {
    if (!b) { set_error("NULL handle"); return LJSEL_ERR_ARG; }
    return bdispatch(b, [&](auto z) -> ljsel_status {
        using R = decltype(z);
        TRY(b->compute<R>(energy || virial));
        BDev<R> S;
        b->fill(S);
        const size_t n3 = (size_t)b->ntot * 3 * sizeof(double);
        if (forces) {
            double *dst = forces;
            if (!on_device) { TRY(b->b_io.ensure(n3)); dst = (double *)b->b_io.ptr; }
            k_bexport<R><<<div_up(b->ntot, 256), 256, 0, b->stream>>>(S, nullptr, nullptr, dst, 0);
            CK(cudaGetLastError());
            if (!on_device) CK(cudaMemcpyAsync(forces, dst, n3, cudaMemcpyDeviceToHost, b->stream));
        }
        if (energy) CK(cudaMemcpyAsync(energy, b->b_ev.ptr, b->nrep * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
        if (virial)
            CK(cudaMemcpyAsync(virial, (double *)b->b_ev.ptr + b->nrep, b->nrep * sizeof(double), cudaMemcpyDeviceToHost,
                               b->stream));
        TRY(b->read_ctrl());
        return LJSEL_OK;
    });
}

ljsel_status ljsel_batch_get_state(ljsel_batch b, double *pos, double *vel, int32_t on_device) {
    if (!b) { set_error("NULL handle"); return LJSEL_ERR_ARG; }
    return bdispatch(b, [&](auto z) -> ljsel_status {
        using R = decltype(z);
        if (vel) TRY(b->sync_velocities<R>());
        BDev<R> S;
        b->fill(S);
        const size_t n3 = (size_t)b->ntot * 3 * sizeof(double);
        double *dp = pos, *dv = vel;
        if (!on_device) {
            TRY(b->b_io.ensure(2 * n3));
            dp = pos ? (double *)b->b_io.ptr : nullptr;
            dv = vel ? (double *)((char *)b->b_io.ptr + n3) : nullptr;
        }
        k_bexport<R><<<div_up(b->ntot, 256), 256, 0, b->stream>>>(S, dp, dv, nullptr, 1);
        CK(cudaGetLastError());
        if (!on_device) {
            if (pos) CK(cudaMemcpyAsync(pos, dp, n3, cudaMemcpyDeviceToHost, b->stream));
            if (vel) CK(cudaMemcpyAsync(vel, dv, n3, cudaMemcpyDeviceToHost, b->stream));
        }
        CK(cudaStreamSynchronize(b->stream));
        return LJSEL_OK;
    });
}

ljsel_status ljsel_batch_get_work_positions(ljsel_batch b, double *pos) {
    if (!b || !pos) { set_error("NULL argument"); return LJSEL_ERR_ARG; }
    return bdispatch(b, [&](auto z) -> ljsel_status {
        using R = decltype(z);
        TRY(b->read_ctrl());
        const size_t n = (size_t)b->ntot;
        std::vector<V4<R>> w(n);
        std::vector<int> id(n);
        CK(cudaMemcpy(w.data(), b->b_pos[b->h_ctrl->pos_par].ptr, n * sizeof(V4<R>), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(id.data(), b->b_id[b->h_ctrl->state_par].ptr, n * 4, cudaMemcpyDeviceToHost));
        for (size_t g = 0; g < n; ++g) {
            pos[3 * (size_t)id[g] + 0] = (double)w[g].x;
            pos[3 * (size_t)id[g] + 1] = (double)w[g].y;
            pos[3 * (size_t)id[g] + 2] = (double)w[g].z;
        }
        return LJSEL_OK;
    });
}

ljsel_status ljsel_batch_get_pairs(ljsel_batch b, int64_t cap, int32_t *rij, int64_t *count) {
    if (!b || !count || cap < 0 || (cap > 0 && !rij)) { set_error("invalid argument"); return LJSEL_ERR_ARG; }
    return bdispatch(b, [&](auto z) -> ljsel_status {
        using R = decltype(z);
        TRY(b->ensure_structure<R>());
        BDev<R> S;
        b->fill(S);
        int2 *pairs = nullptr;
        int *reps = nullptr;
        if (cap > 0) {
            CK(cudaMalloc(&pairs, (size_t)cap * sizeof(int2)));
            if (cudaMalloc(&reps, (size_t)cap * sizeof(int)) != cudaSuccess) {
                cudaFree(pairs);
                set_error("pair buffer allocation failed");
                return LJSEL_ERR_OOM;
            }
        }
        TRY(b->cmd(CMD_RESET_PAIRS, 0));
        b->force_launch<R, BMODE_PAIRS, false>(S, b->tile, b->stream, pairs, cap, reps);
        cudaError_t e = cudaGetLastError();
        ljsel_status st = e == cudaSuccess ? b->read_ctrl() : LJSEL_ERR_CUDA;
        if (e != cudaSuccess) set_error(cudaGetErrorString(e));
        if (st == LJSEL_OK) {
            *count = (int64_t)b->h_ctrl->npairs;
            const long long m = std::min<long long>(cap, *count);
            if (m > 0) {
                std::vector<int2> hp(m);
                std::vector<int> hr(m);
                if (cudaMemcpy(hp.data(), pairs, m * sizeof(int2), cudaMemcpyDeviceToHost) != cudaSuccess ||
                    cudaMemcpy(hr.data(), reps, m * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
                    set_error("pair copy failed");
                    st = LJSEL_ERR_CUDA;
                } else {
                    for (long long k = 0; k < m; ++k) {
                        rij[3 * k + 0] = hr[k];
                        rij[3 * k + 1] = hp[k].x;
                        rij[3 * k + 2] = hp[k].y;
                    }
                }
            }
        }
        if (pairs) cudaFree(pairs);
        if (reps) cudaFree(reps);
        return st;
    });
}

// Plain stream launches with events around the rebuild chain, the fused
// force + update kernel and the control kernel; the host reads the control
// block every step to launch the rebuild chain only when it runs.
ljsel_status ljsel_batch_profile_steps(ljsel_batch b, int64_t nsteps, ljsel_profile *out) {
    if (!b || !out || nsteps < 0) { set_error("invalid argument"); return LJSEL_ERR_ARG; }
    memset(out, 0, sizeof(*out));
    return bdispatch(b, [&](auto z) -> ljsel_status {
        using R = decltype(z);
        TRY(b->ensure_structure<R>());
        cudaEvent_t ev[5];
        for (auto &e : ev) CK(cudaEventCreate(&e));
        BDev<R> S;
        b->fill(S);
        double tr = 0, tf = 0, tc = 0;
        ljsel_status st = b->cmd(CMD_BEGIN, nsteps);
        for (long long k = 0; k < nsteps && st == LJSEL_OK; ++k) {
            if ((st = b->read_ctrl()) != LJSEL_OK) break;
            if (b->h_ctrl->overflow) {
                if ((st = b->grow()) == LJSEL_OK) st = b->ensure_structure<R>();
                b->fill(S);
                continue;
            }
            const bool reb = b->h_ctrl->rebuild_now != 0;
            if (reb) {
                cudaEventRecord(ev[0], b->stream);
                b->enqueue_rebuild(S, b->stream);
                cudaEventRecord(ev[1], b->stream);
                out->launches += 10;
            }
            cudaEventRecord(ev[2], b->stream);
            b->force_launch<R, BMODE_STEP, false>(S, b->tile, b->stream);
            cudaEventRecord(ev[3], b->stream);
            launch_control(S.ctrl, 0, 0, 0, b->stream);
            cudaEventRecord(ev[4], b->stream);
            out->launches += 2;
            if (cudaEventSynchronize(ev[4]) != cudaSuccess) { set_error("profiling step failed"); st = LJSEL_ERR_CUDA; break; }
            float a = 0, f = 0, c = 0;
            if (reb) { cudaEventElapsedTime(&a, ev[0], ev[1]); out->rebuilds += 1; tr += a; }
            cudaEventElapsedTime(&f, ev[2], ev[3]);
            cudaEventElapsedTime(&c, ev[3], ev[4]);
            tf += f;
            tc += c;
            out->steps += 1;
        }
        for (auto &e : ev) cudaEventDestroy(e);
        if (st != LJSEL_OK) return st;
        b->synced = false;
        out->rebuild_ms = out->rebuilds ? tr / out->rebuilds : 0.0;
        out->force_ms = out->steps ? tf / out->steps : 0.0;
        out->control_ms = out->steps ? tc / out->steps : 0.0;
        out->total_ms = tr + tf + tc;
        return LJSEL_OK;
    });
}

ljsel_status ljsel_batch_set_list_capacity(ljsel_batch b, int64_t entries) {
    if (!b) { set_error("NULL handle"); return LJSEL_ERR_ARG; }
    if (entries < 4 || entries > 65532) { set_error("entries per row must be in 4 .. 65532"); return LJSEL_ERR_ARG; }
    return b->set_capacity((int)entries);
}

ljsel_status ljsel_batch_get_counters(ljsel_batch b, ljsel_counters *c) {
    if (!b || !c) { set_error("NULL argument"); return LJSEL_ERR_ARG; }
    TRY(b->read_ctrl());
    memset(c, 0, sizeof(*c));
    c->steps = b->h_ctrl->total_steps;
    c->rebuilds = b->h_ctrl->rebuilds;
    c->early_rebuilds = b->h_ctrl->early_rebuilds;
    c->longest_row = b->h_ctrl->need_cap;
    c->list_capacity = (int64_t)b->nl_cap * b->ntot;
    c->ncells = b->ncell;
    c->capacity_retries = b->retries;
    c->replica_rebuilds = b->h_ctrl->replica_rebuilds;
    return LJSEL_OK;
}

// Full search over tiles (Sec. 2.2.5 applied to the batch kernel shape):
// each candidate runs trial_steps real steps under the step graph, timed
// with events; the cheapest per step is kept.
ljsel_status ljsel_batch_autotune(ljsel_batch b, int32_t trial_steps, int32_t ncand, const ljsel_batch_tile *cand,
                                  ljsel_batch_tile *chosen, double *costs_ms) {
    if (!b || !chosen || trial_steps < 1 || ncand < 0 || (ncand > 0 && !cand)) {
        set_error("invalid argument");
        return LJSEL_ERR_ARG;
    }
    std::vector<ljsel_batch_tile> list;
    if (ncand > 0) {
        list.assign(cand, cand + ncand);
    } else {
        for (int tpp : {1, 2, 4, 8})
            for (int blk : {128, 256}) list.push_back({tpp, blk, 0, b->interval});
        list.push_back({1, 128, 8, b->interval});
        list.push_back({2, 256, 4, b->interval});
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    double best = 1e300;
    int best_k = -1;
    ljsel_status st = LJSEL_OK;
    for (size_t k = 0; k < list.size(); ++k) {
        double cost = -1.0;
        if (ljsel_batch_set_tile(b, &list[k]) == LJSEL_OK) {
            // one untimed step builds (or finds) the graph of this tile
            st = ljsel_batch_step(b, 1);
            if (st != LJSEL_OK) break;
            cudaEventRecord(e0, b->stream);
            st = ljsel_batch_step(b, trial_steps);
            if (st != LJSEL_OK) break;
            cudaEventRecord(e1, b->stream);
            cudaEventSynchronize(e1);
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            cost = ms / trial_steps;
            if (cost < best) { best = cost; best_k = (int)k; }
        }
        if (costs_ms) costs_ms[k] = cost;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != LJSEL_OK) return st;
    if (best_k < 0) { set_error("no tile could be trialled"); return LJSEL_ERR_UNSUPPORTED; }
    TRY(ljsel_batch_set_tile(b, &list[best_k]));
    *chosen = list[best_k];
    return LJSEL_OK;
}

}  // extern "C"
