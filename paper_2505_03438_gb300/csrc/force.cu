// force.cu -- cutoff Lennard-Jones forces over Verlet lists and linked
// cells (Sec. 2.1, Sec. 2.2.1), the Stormer-Verlet update (Sec. 2.1), the
// per-step control kernel and small data-movement kernels.
//
// Pair arithmetic runs in the working precision R (FP32 on the fast path):
// per candidate 3 displacement subtractions, r^2 by two FMAs, the cutoff
// decision (FP32 outside a narrow band, exact FP64 inside), one approximate
// reciprocal, five multiplies and one FMA for f/r, three FMAs for the force.
// Integration is FP64: v += (dt/m) F, x += dt v, with the FP32 working copy
// rounded from the FP64 position.
#include "kernels.cuh"
#include "update.cuh"

namespace ljsel {

namespace {

constexpr int FORCE_THREADS = 128;

// Shared-memory copy of the per-type-pair table for multi-type systems.
template <typename R> struct STab {
    R sig2[MAXT2], e24[MAXT2], e48[MAXT2], e4[MAXT2], ushift[MAXT2], lo[MAXT2], hi[MAXT2];
    double rc2d[MAXT2];
};

template <typename R>
__device__ __forceinline__ void load_stab(STab<R> &T, const PairTab<R> &P) {
    for (int k = threadIdx.x; k < MAXT2; k += blockDim.x) {
        T.sig2[k] = P.sig2[k]; T.e24[k] = P.e24[k]; T.e48[k] = P.e48[k]; T.e4[k] = P.e4[k];
        T.ushift[k] = P.ushift[k]; T.lo[k] = P.rc2lo[k]; T.hi[k] = P.rc2hi[k]; T.rc2d[k] = P.rc2d[k];
    }
}

// Per-thread accumulators.  Single type: u accumulates sr6 (sr6 - 1) and np
// counts pairs, the energy is e4 * u - ushift * np; multi-type: u is the
// energy itself.
template <typename R> struct Acc {
    R fx = 0, fy = 0, fz = 0, u = 0, w = 0;
    int np = 0;
};

// One candidate pair: decides the cutoff exactly, returns f/r (0 when out of
// range) and accumulates energy and virial when EV.
template <typename R, bool MT, bool EV>
__device__ __forceinline__ R pair_term(const Dev<R> &S, const STab<R> &T, int tp, R r2, const V4<R> &pi,
                                       const V4<R> &pj, int sx, int sy, int sz, Acc<R> &a, bool &in) {
    R sig2, e24, e48, lo, hi;
    double rc2d;
    if (MT) {
        sig2 = T.sig2[tp]; e24 = T.e24[tp]; e48 = T.e48[tp]; lo = T.lo[tp]; hi = T.hi[tp]; rc2d = T.rc2d[tp];
    } else {
        sig2 = S.tab.sig2[0]; e24 = S.tab.e24[0]; e48 = S.tab.e48[0]; lo = S.tab.rc2lo[0]; hi = S.tab.rc2hi[0];
        rc2d = S.tab.rc2d[0];
    }
    in = Cut<R>::in(r2, lo, hi, pi, pj, sx, sy, sz, S.boxd, rc2d);
    R sr6;
    R fr = lj_fr(r2, sig2, e24, e48, sr6);
    fr = in ? fr : (R)0;
    if (EV) {
        if (MT) {
            a.u += in ? T.e4[tp] * sr6 * (sr6 - (R)1) - T.ushift[tp] : (R)0;
        } else {
            a.u += in ? sr6 * (sr6 - (R)1) : (R)0;
            a.np += in ? 1 : 0;
        }
        a.w += fr * r2;
    }
    return fr;
}

template <typename R, bool MT>
__device__ __forceinline__ R energy_of(const Dev<R> &S, const Acc<R> &a) {
    if (MT) return a.u;
    return S.tab.e4[0] * a.u - S.tab.ushift[0] * (R)a.np;
}

__device__ __forceinline__ void add_force(float4 *F, int j, float x, float y, float z) {
    atomicAdd(F + j, make_float4(x, y, z, 0.f));
}
__device__ __forceinline__ void add_force(D4 *F, int j, double x, double y, double z) {
    atomicAdd(&F[j].x, x); atomicAdd(&F[j].y, y); atomicAdd(&F[j].z, z);
}

template <typename R>
__device__ __forceinline__ void export_pair(const Dev<R> &S, int sp, int i, int j, int2 *out, long long cap) {
    int a = S.id[sp][i], b = S.id[sp][j];
    unsigned long long k = atomicAdd(&S.ctrl->npairs, 1ull);
    if ((long long)k < cap) out[k] = make_int2(min(a, b), max(a, b));
}

// ---------------------------------------------------------------------------
// Verlet lists.  Thread group of `tpp` lanes per particle i (sorted index).
// The front of the row (entries without an image, padded with the sentinel)
// is read in 16-byte chunks sub, sub + tpp, ...; the next chunk is loaded
// before the current chunk's four positions are gathered.  The few entries
// with a periodic image, at the back of the row, take the exact image
// arithmetic.  The group sums F_i by shuffles.  Thread 0 of each block first
// asks the L2 to prefetch the block's contiguous list rows and state with
// one bulk-prefetch instruction each.  N3L off: full lists, F_j untouched.
// N3L on: half lists, -F_ij added to F_j with a vector atomic.
__device__ __forceinline__ void l2_prefetch(const void *p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <typename R, bool N3L, int MODE, bool EV, bool MT>
__device__ __forceinline__ void vl_pair(const Dev<R> &S, const STab<R> &T, const V4<R> &pi, int ti, int i, int sp,
                                        int j, int sx, int sy, int sz, R dx, R dy, R dz, const V4<R> &pj, Acc<R> &a,
                                        int2 *pairs, long long cap) {
    const R r2 = r2_of(dx, dy, dz);
    const int tp = MT ? ti * S.tab.ntypes + type_of(pj) : 0;
    bool in;
    const R fr = pair_term<R, MT, EV>(S, T, tp, r2, pi, pj, sx, sy, sz, a, in);
    if (MODE == MODE_PAIRS) {
        if (in && (N3L || S.id[sp][i] < S.id[sp][j])) export_pair(S, sp, i, j, pairs, cap);
        return;
    }
    a.fx += fr * dx; a.fy += fr * dy; a.fz += fr * dz;
    if (N3L && in) add_force(S.force, j, -fr * dx, -fr * dy, -fr * dz);
}

template <typename R, bool N3L, int MODE, bool EV, bool MT>
__global__ void __launch_bounds__(FORCE_THREADS, 8) k_vl(Dev<R> S, int tpp, int2 *pairs, long long cap) {
    Ctrl *C = S.ctrl;
    if (C->overflow) return;
    __shared__ STab<R> T;
    if (MT) { load_stab(T, S.tab); __syncthreads(); }
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gid / tpp, sub = gid - i * tpp;
    const bool valid = i < S.n;
    const int pp = C->pos_par, sp = C->state_par;
    const V4<R> *P = S.pos[pp];
    if (threadIdx.x == 0) {
        const int i0 = (blockIdx.x * blockDim.x) / tpp;
        const int nrow = min(blockDim.x / tpp, S.n - i0);
        if (nrow > 0) {
            l2_prefetch(S.nl + (size_t)i0 * S.nl_cap, (unsigned)(nrow * S.nl_cap * 4));
            // bulk prefetch wants 16-byte aligned start and size: a slice of
            // doubles qualifies when its first index and its length are even
            if (MODE == MODE_STEP && (nrow & 1) == 0) {
                for (int d = 0; d < 3; ++d) {
                    const size_t first = (size_t)d * S.n + i0;
                    if ((first & 1) != 0) continue;
                    l2_prefetch(S.x[sp] + first, (unsigned)(nrow * 8));
                    l2_prefetch(S.v[sp] + first, (unsigned)(nrow * 8));
                }
            }
        }
    }
    V4<R> pi = make_pos((R)0, (R)0, (R)0, 0);
    int nq = 0, nb = 0, ti = 0;
    const uint32_t *rowp = nullptr;
    if (valid) {
        pi = ldpos(P, i);
        const int cnt = S.nl_count[i];
        nq = ((cnt & 0xffff) + 3) >> 2;
        nb = cnt >> 16;
        if (!lj_check(4 * nq + nb <= S.nl_cap, C, CHECK_VL_ROW)) { nq = 0; nb = 0; }
        ti = type_of(pi);
        rowp = S.nl + (size_t)i * S.nl_cap;
    }
    const uint4 *row = reinterpret_cast<const uint4 *>(rowp);
    Acc<R> a;
    uint4 e = sub < nq ? __ldg(row + sub) : make_uint4(0, 0, 0, 0);
    for (int q = sub; q < nq; q += tpp) {
        const uint4 en = q + tpp < nq ? __ldg(row + q + tpp) : e;
        const unsigned nn = (unsigned)S.n;  // the sentinel n pads the front
        if (!lj_check(e.x <= nn && e.y <= nn && e.z <= nn && e.w <= nn, C, CHECK_VL_FRONT)) e = make_uint4(nn, nn, nn, nn);
        const V4<R> p0 = ldpos(P, (int)e.x), p1 = ldpos(P, (int)e.y), p2 = ldpos(P, (int)e.z), p3 = ldpos(P, (int)e.w);
        vl_pair<R, N3L, MODE, EV, MT>(S, T, pi, ti, i, sp, (int)e.x, 0, 0, 0, pi.x - p0.x, pi.y - p0.y, pi.z - p0.z, p0, a, pairs, cap);
        vl_pair<R, N3L, MODE, EV, MT>(S, T, pi, ti, i, sp, (int)e.y, 0, 0, 0, pi.x - p1.x, pi.y - p1.y, pi.z - p1.z, p1, a, pairs, cap);
        vl_pair<R, N3L, MODE, EV, MT>(S, T, pi, ti, i, sp, (int)e.z, 0, 0, 0, pi.x - p2.x, pi.y - p2.y, pi.z - p2.z, p2, a, pairs, cap);
        vl_pair<R, N3L, MODE, EV, MT>(S, T, pi, ti, i, sp, (int)e.w, 0, 0, 0, pi.x - p3.x, pi.y - p3.y, pi.z - p3.z, p3, a, pairs, cap);
        e = en;
    }
    for (int k = sub; k < nb; k += tpp) {
        const uint32_t ent = rowp[S.nl_cap - 1 - k];
        int j = (int)(ent & JMASK);
        if (!lj_check(j < S.n, C, CHECK_VL_BACK)) break;
        int sx, sy, sz;
        decode_image(ent >> JBITS, sx, sy, sz);
        const V4<R> pj = ldpos(P, j);
        vl_pair<R, N3L, MODE, EV, MT>(S, T, pi, ti, i, sp, j, sx, sy, sz,
                                      image_dx(pi.x, pj.x, sx, S.box[0], S.box_lo[0]),
                                      image_dx(pi.y, pj.y, sy, S.box[1], S.box_lo[1]),
                                      image_dx(pi.z, pj.z, sz, S.box[2], S.box_lo[2]), pj, a, pairs, cap);
    }
    if (MODE == MODE_PAIRS) return;
    for (int o = tpp >> 1; o > 0; o >>= 1) {
        a.fx += __shfl_xor_sync(0xffffffffu, a.fx, o);
        a.fy += __shfl_xor_sync(0xffffffffu, a.fy, o);
        a.fz += __shfl_xor_sync(0xffffffffu, a.fz, o);
    }
    double ke = 0;
    bool exceeded = false, bad = false;
    if (valid && sub == 0) {
        if (N3L) add_force(S.force, i, a.fx, a.fy, a.fz);
        else if (MODE == MODE_FORCE) { V4<R> f = make_pos(a.fx, a.fy, a.fz, 0); S.force[i] = f; }
        else integrate_one<R, EV>(S, sp, pp, C->half_kick, i, ti, a.fx, a.fy, a.fz, ke, exceeded, bad);
    }
    if (MODE == MODE_STEP) report_flags(C, exceeded, bad);
    if (EV) {
        const R scale = N3L ? (R)1 : (R)0.5;
        block_sum3((double)(scale * energy_of<R, MT>(S, a)), (double)(scale * a.w), ke, C);
    }
}

// ---------------------------------------------------------------------------
// Linked cells without a list: one thread per particle scans every particle
// of the stencil cells (reach 1 for CSF 1, 2 for CSF 0.5) and applies the
// exact cutoff.  With N3L only j > i is evaluated and F_j gets -F_ij.
template <typename R, bool N3L, int MODE, bool EV, bool MT>
__global__ void __launch_bounds__(FORCE_THREADS) k_lc(Dev<R> S, int2 *pairs, long long cap) {
    Ctrl *C = S.ctrl;
    if (C->overflow) return;
    __shared__ STab<R> T;
    if (MT) { load_stab(T, S.tab); __syncthreads(); }
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < S.n;
    const int pp = C->pos_par, sp = C->state_par;
    const V4<R> *P = S.pos[pp];
    Acc<R> a;
    int ti = 0;
    if (valid) {
        const V4<R> pi = ldpos(P, i);
        ti = type_of(pi);
        const int c = S.cell_sorted[i];
        const int cx = c % S.nc[0], cy = (c / S.nc[0]) % S.nc[1], cz = c / (S.nc[0] * S.nc[1]);
        const int rch = S.reach;
        for (int oz = -rch; oz <= rch; ++oz) {
            int wz, sz;
            if (!stencil_cell(cz, oz, S.nc[2], S.walls[2], wz, sz)) continue;
            for (int oy = -rch; oy <= rch; ++oy) {
                int wy, sy;
                if (!stencil_cell(cy, oy, S.nc[1], S.walls[1], wy, sy)) continue;
                for (int ox = -rch; ox <= rch; ++ox) {
                    int wx, sx;
                    if (!stencil_cell(cx, ox, S.nc[0], S.walls[0], wx, sx)) continue;
                    const int cc = (wz * S.nc[1] + wy) * S.nc[0] + wx;
                    const bool img = (sx | sy | sz) != 0;
                    if (!lj_check(cc >= 0 && cc < S.ncell, C, CHECK_LC_CELL)) continue;
                    int jb = S.cell_start[cc], je = S.cell_start[cc + 1];
                    if (!lj_check(jb >= 0 && jb <= je && je <= S.n, C, CHECK_LC_CELL)) continue;
                    // one pair; the exact image arithmetic only in image cells
                    auto one = [&](int j, R dx, R dy, R dz, const V4<R> &pj) {
                        const R r2 = r2_of(dx, dy, dz);
                        const int tp = MT ? ti * S.tab.ntypes + type_of(pj) : 0;
                        bool in;
                        const R fr = pair_term<R, MT, EV>(S, T, tp, r2, pi, pj, sx, sy, sz, a, in);
                        if (MODE == MODE_PAIRS) {
                            if (in && (N3L || S.id[sp][i] < S.id[sp][j])) export_pair(S, sp, i, j, pairs, cap);
                            return;
                        }
                        a.fx += fr * dx; a.fy += fr * dy; a.fz += fr * dz;
                        if (N3L && in) add_force(S.force, j, -fr * dx, -fr * dy, -fr * dz);
                    };
                    if (!img) {
                        for (int j = N3L ? max(jb, i + 1) : jb; j < je; ++j) {
                            if (!N3L && j == i) continue;
                            const V4<R> pj = ldpos(P, j);
                            one(j, pi.x - pj.x, pi.y - pj.y, pi.z - pj.z, pj);
                        }
                    } else {
                        for (int j = N3L ? max(jb, i + 1) : jb; j < je; ++j) {
                            const V4<R> pj = ldpos(P, j);
                            one(j, image_dx(pi.x, pj.x, sx, S.box[0], S.box_lo[0]),
                                image_dx(pi.y, pj.y, sy, S.box[1], S.box_lo[1]),
                                image_dx(pi.z, pj.z, sz, S.box[2], S.box_lo[2]), pj);
                        }
                    }
                }
            }
        }
    }
    if (MODE == MODE_PAIRS) return;
    double ke = 0;
    bool exceeded = false, bad = false;
    if (valid) {
        if (N3L) add_force(S.force, i, a.fx, a.fy, a.fz);
        else if (MODE == MODE_FORCE) { V4<R> f = make_pos(a.fx, a.fy, a.fz, 0); S.force[i] = f; }
        else integrate_one<R, EV>(S, sp, pp, C->half_kick, i, ti, a.fx, a.fy, a.fz, ke, exceeded, bad);
    }
    if (MODE == MODE_STEP) report_flags(C, exceeded, bad);
    if (EV) {
        const R scale = N3L ? (R)1 : (R)0.5;
        block_sum3((double)(scale * energy_of<R, MT>(S, a)), (double)(scale * a.w), ke, C);
    }
}

// Integration after an N3L force kernel: reads and clears the force buffer.
template <typename R, bool EV>
__global__ void __launch_bounds__(256) k_integrate(Dev<R> S) {
    Ctrl *C = S.ctrl;
    if (C->overflow) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0;
    bool exceeded = false, bad = false;
    if (i < S.n) {
        const int sp = C->state_par, pp = C->pos_par;
        const V4<R> f = S.force[i];
        integrate_one<R, EV>(S, sp, pp, C->half_kick, i, S.type[sp][i], f.x, f.y, f.z, ke, exceeded, bad);
        S.force[i] = make_pos((R)0, (R)0, (R)0, 0);  // after the loads of the update
    }
    report_flags(C, exceeded, bad);
    if (EV) block_sum3(0.0, 0.0, ke, C);
}

// After each step: flip the working-position parity, count, and decide the
// next rebuild (every R steps, or once a particle moved skin/2 since the
// last rebuild).  A step that found the list overflowed is not counted; the
// host reallocates and resumes.
__global__ void k_control(Ctrl *C, cudaGraphConditionalHandle h_rebuild, cudaGraphConditionalHandle h_loop, int graph) {
    bool more = false, need = false;
    if (!C->overflow) {
        C->pos_par ^= 1;
        C->half_kick = 0;
        C->steps_done += 1;
        C->total_steps += 1;
        C->steps_since += 1;
        const bool by_disp = C->disp_exceeded != 0;
        const bool by_count = C->steps_since >= C->rebuild_interval;
        need = by_disp || by_count;
        if (need && !by_count) C->early_rebuilds += 1;
        C->disp_exceeded = 0;
        C->rebuild_now = need ? 1 : 0;
        more = C->steps_done < C->steps_target && !C->nonfinite && !C->timeout;
    }
    if (graph) {
        cudaGraphSetConditional(h_rebuild, (more && need) ? 1u : 0u);
        cudaGraphSetConditional(h_loop, more ? 1u : 0u);
    }
}

__global__ void k_loop_init(Ctrl *C, cudaGraphConditionalHandle h_rebuild, cudaGraphConditionalHandle h_loop) {
    const bool more = C->steps_done < C->steps_target && !C->overflow && !C->nonfinite && !C->timeout;
    cudaGraphSetConditional(h_rebuild, (more && C->rebuild_now) ? 1u : 0u);
    cudaGraphSetConditional(h_loop, more ? 1u : 0u);
}

// ---------------------------------------------------------------------------
template <typename R>
__global__ void k_export_forces(Dev<R> S, double *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    const int sp = S.ctrl->state_par;
    const int id = S.id[sp][i];
    V4<R> f = S.force[i];
    out[3 * id + 0] = (double)f.x; out[3 * id + 1] = (double)f.y; out[3 * id + 2] = (double)f.z;
}

template <typename R>
__global__ void k_export_state(Dev<R> S, double *pos, double *vel, int wrap) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    const int sp = S.ctrl->state_par, n = S.n;
    const int id = S.id[sp][i];
    for (int d = 0; d < 3; ++d) {
        if (pos) {
            double x = S.x[sp][d * n + i];
            if (wrap && !S.walls[d]) {
                double L = S.boxd[d];
                if (x < 0.0) x += L;
                if (x >= L) x -= L;
                if (x < 0.0 || x >= L) { x = x - L * floor(x / L); if (x >= L) x = 0.0; }
            }
            pos[3 * id + d] = x;
        }
        if (vel) vel[3 * id + d] = S.v[sp][d * n + i];
    }
}

template <typename R>
__global__ void k_export_work_pos(Dev<R> S, double *pos) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    const Ctrl *C = S.ctrl;
    const int id = S.id[C->state_par][i];
    V4<R> p = S.pos[C->pos_par][i];
    pos[3 * id + 0] = (double)p.x; pos[3 * id + 1] = (double)p.y; pos[3 * id + 2] = (double)p.z;
}

// Load caller state (input order) into the current sorted slots.  With
// init_ids the slots take the input order (fresh system); otherwise each
// slot keeps its particle.  The working copy is refreshed and a rebuild is
// flagged by the host.
template <typename R>
__global__ void k_import_state(Dev<R> S, const double *pos, const double *vel, const int *types, int init_ids) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    Ctrl *C = S.ctrl;
    const int sp = C->state_par, pp = C->pos_par, n = S.n;
    if (init_ids) {
        S.id[sp][i] = i;
        int t = types ? types[i] : 0;
        if (t < 0 || t >= S.tab.ntypes) {  // reported by the creating call
            C->bad_type = 1;
            t = 0;
        }
        S.type[sp][i] = t;
    }
    const int id = S.id[sp][i];
    double x[3];
    for (int d = 0; d < 3; ++d) {
        if (pos) S.x[sp][d * n + i] = pos[3 * id + d];
        if (vel) S.v[sp][d * n + i] = vel[3 * id + d];
        x[d] = S.x[sp][d * n + i];
    }
    V4<R> w = make_pos((R)x[0], (R)x[1], (R)x[2], S.type[sp][i]);
    S.pos[pp][i] = w;
    S.xref[i] = w;
}

// New positions (input order) for the current slots, keeping the neighbour
// structure: the reference positions of the last rebuild stay, and a
// particle that now lies skin/2 or more from its reference flags a rebuild,
// so the structure is used only while the Verlet-list guarantee holds.
template <typename R>
__global__ void k_move_particles(Dev<R> S, const double *pos) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    Ctrl *C = S.ctrl;
    const int sp = C->state_par, pp = C->pos_par, n = S.n;
    const int id = S.id[sp][i];
    double x[3];
    for (int d = 0; d < 3; ++d) {
        x[d] = pos[3 * id + d];
        S.x[sp][d * n + i] = x[d];
    }
    const V4<R> w = make_pos((R)x[0], (R)x[1], (R)x[2], S.type[sp][i]);
    S.pos[pp][i] = w;
    const V4<R> r = S.xref[i];
    const R dx = w.x - r.x, dy = w.y - r.y, dz = w.z - r.z;
    if (!(dx * dx + dy * dy + dz * dz < S.half_skin2)) C->rebuild_now = 1;
}

// Bring half-step velocities to the integer step: v += (dt/2m) F(x).
template <typename R>
__global__ void k_sync_velocities(Dev<R> S) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    const int sp = S.ctrl->state_par, n = S.n;
    const int t = S.type[sp][i];
    V4<R> f = S.force[i];
    R c = S.tab.inv_mass_dt[t] * (R)0.5;
    S.v[sp][i] += (double)(c * f.x);
    S.v[sp][n + i] += (double)(c * f.y);
    S.v[sp][2 * n + i] += (double)(c * f.z);
}

template <typename R>
__global__ void k_kinetic(Dev<R> S) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double ke = 0;
    if (i < S.n) {
        const int sp = S.ctrl->state_par, n = S.n;
        const int t = S.type[sp][i];
        double vx = S.v[sp][i], vy = S.v[sp][n + i], vz = S.v[sp][2 * n + i];
        ke = S.tab.half_mass[t] * (vx * vx + vy * vy + vz * vz);
    }
    block_sum3(0.0, 0.0, ke, S.ctrl);
}

template <typename R>
__global__ void k_zero_force(Dev<R> S) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < S.n) S.force[i] = make_pos((R)0, (R)0, (R)0, 0);
}

}  // namespace

// ---------------------------------------------------------------------------
template <typename R, bool N3L, int MODE, bool EV, bool MT>
static void vl_go(const Dev<R> &S, int tpp, int2 *pairs, long long cap, cudaStream_t st) {
    long long threads = (long long)S.n * tpp;
    k_vl<R, N3L, MODE, EV, MT><<<div_up(threads, FORCE_THREADS), FORCE_THREADS, 0, st>>>(S, tpp, pairs, cap);
}
template <typename R, bool N3L, int MODE, bool EV, bool MT>
static void lc_go(const Dev<R> &S, int2 *pairs, long long cap, cudaStream_t st) {
    k_lc<R, N3L, MODE, EV, MT><<<div_up(S.n, FORCE_THREADS), FORCE_THREADS, 0, st>>>(S, pairs, cap);
}

template <typename R, bool MT>
static void force_dispatch(const Dev<R> &S, const ljsel_config &cfg, int mode, bool ev, int2 *pairs, long long cap,
                           cudaStream_t st) {
    const bool n3l = cfg.newton3 != 0;
    const int tpp = cfg.threads_per_unit < 1 ? 1 : cfg.threads_per_unit;
    if (cfg.method == LJSEL_METHOD_VL) {
        if (mode == MODE_PAIRS) { n3l ? vl_go<R, true, MODE_PAIRS, false, MT>(S, tpp, pairs, cap, st) : vl_go<R, false, MODE_PAIRS, false, MT>(S, tpp, pairs, cap, st); return; }
        if (n3l) { ev ? vl_go<R, true, MODE_FORCE, true, MT>(S, tpp, pairs, cap, st) : vl_go<R, true, MODE_FORCE, false, MT>(S, tpp, pairs, cap, st); return; }
        if (mode == MODE_STEP) { ev ? vl_go<R, false, MODE_STEP, true, MT>(S, tpp, pairs, cap, st) : vl_go<R, false, MODE_STEP, false, MT>(S, tpp, pairs, cap, st); return; }
        ev ? vl_go<R, false, MODE_FORCE, true, MT>(S, tpp, pairs, cap, st) : vl_go<R, false, MODE_FORCE, false, MT>(S, tpp, pairs, cap, st);
        return;
    }
    // linked cells
    if (mode == MODE_PAIRS) { n3l ? lc_go<R, true, MODE_PAIRS, false, MT>(S, pairs, cap, st) : lc_go<R, false, MODE_PAIRS, false, MT>(S, pairs, cap, st); return; }
    if (n3l) { ev ? lc_go<R, true, MODE_FORCE, true, MT>(S, pairs, cap, st) : lc_go<R, true, MODE_FORCE, false, MT>(S, pairs, cap, st); return; }
    if (mode == MODE_STEP) { ev ? lc_go<R, false, MODE_STEP, true, MT>(S, pairs, cap, st) : lc_go<R, false, MODE_STEP, false, MT>(S, pairs, cap, st); return; }
    ev ? lc_go<R, false, MODE_FORCE, true, MT>(S, pairs, cap, st) : lc_go<R, false, MODE_FORCE, false, MT>(S, pairs, cap, st);
}

template <typename R> void launch_cp_force(const Dev<R> &S, const ljsel_config &cfg, int mode, bool ev, int2 *pairs,
                                           long long cap, cudaStream_t st);

template <> void launch_force<float>(const Dev<float> &S, const ljsel_config &cfg, int mode, bool ev, int2 *pairs,
                                     long long cap, cudaStream_t st) {
    if (cfg.method == LJSEL_METHOD_CLUSTER) { launch_cp_force<float>(S, cfg, mode, ev, pairs, cap, st); return; }
    if (cfg.method == LJSEL_METHOD_VLW) { launch_vlw_force<float>(S, cfg, mode, ev, pairs, cap, st); return; }
    if (S.tab.ntypes > 1) force_dispatch<float, true>(S, cfg, mode, ev, pairs, cap, st);
    else force_dispatch<float, false>(S, cfg, mode, ev, pairs, cap, st);
}
template <> void launch_force<double>(const Dev<double> &S, const ljsel_config &cfg, int mode, bool ev, int2 *pairs,
                                      long long cap, cudaStream_t st) {
    if (cfg.method == LJSEL_METHOD_CLUSTER) { launch_cp_force<double>(S, cfg, mode, ev, pairs, cap, st); return; }
    if (cfg.method == LJSEL_METHOD_VLW) { launch_vlw_force<double>(S, cfg, mode, ev, pairs, cap, st); return; }
    force_dispatch<double, true>(S, cfg, mode, ev, pairs, cap, st);
}

template <typename R> void launch_integrate(const Dev<R> &S, bool ev, cudaStream_t st) {
    if (ev) k_integrate<R, true><<<div_up(S.n, 256), 256, 0, st>>>(S);
    else k_integrate<R, false><<<div_up(S.n, 256), 256, 0, st>>>(S);
}

void launch_control(Ctrl *C, cudaGraphConditionalHandle h_rebuild, cudaGraphConditionalHandle h_loop, int graph,
                    cudaStream_t st) {
    k_control<<<1, 1, 0, st>>>(C, h_rebuild, h_loop, graph);
}
void launch_loop_init(Ctrl *C, cudaGraphConditionalHandle h_rebuild, cudaGraphConditionalHandle h_loop,
                      cudaStream_t st) {
    k_loop_init<<<1, 1, 0, st>>>(C, h_rebuild, h_loop);
}

template <typename R> void launch_export_forces(const Dev<R> &S, double *out, cudaStream_t st) {
    k_export_forces<R><<<div_up(S.n, 256), 256, 0, st>>>(S, out);
}
template <typename R> void launch_export_state(const Dev<R> &S, double *pos, double *vel, int wrap, cudaStream_t st) {
    k_export_state<R><<<div_up(S.n, 256), 256, 0, st>>>(S, pos, vel, wrap);
}
template <typename R> void launch_export_work_pos(const Dev<R> &S, double *pos, cudaStream_t st) {
    k_export_work_pos<R><<<div_up(S.n, 256), 256, 0, st>>>(S, pos);
}
template <typename R> void launch_import_state(const Dev<R> &S, const double *pos, const double *vel, const int *types,
                                               int init_ids, cudaStream_t st) {
    k_import_state<R><<<div_up(S.n, 256), 256, 0, st>>>(S, pos, vel, types, init_ids);
}
template <typename R> void launch_move_particles(const Dev<R> &S, const double *pos, cudaStream_t st) {
    k_move_particles<R><<<div_up(S.n, 256), 256, 0, st>>>(S, pos);
}
template <typename R> void launch_sync_velocities(const Dev<R> &S, cudaStream_t st) {
    k_sync_velocities<R><<<div_up(S.n, 256), 256, 0, st>>>(S);
}
template <typename R> void launch_kinetic(const Dev<R> &S, cudaStream_t st) {
    k_kinetic<R><<<div_up(S.n, 256), 256, 0, st>>>(S);
}
template <typename R> void launch_zero_force(const Dev<R> &S, cudaStream_t st) {
    k_zero_force<R><<<div_up(S.n, 256), 256, 0, st>>>(S);
}

#define INST(R)                                                                                              \
    template void launch_integrate<R>(const Dev<R> &, bool, cudaStream_t);                                   \
    template void launch_export_forces<R>(const Dev<R> &, double *, cudaStream_t);                           \
    template void launch_export_state<R>(const Dev<R> &, double *, double *, int, cudaStream_t);             \
    template void launch_export_work_pos<R>(const Dev<R> &, double *, cudaStream_t);                         \
    template void launch_import_state<R>(const Dev<R> &, const double *, const double *, const int *, int,    \
                                         cudaStream_t);                                                      \
    template void launch_sync_velocities<R>(const Dev<R> &, cudaStream_t);                                   \
    template void launch_move_particles<R>(const Dev<R> &, const double *, cudaStream_t);                    \
    template void launch_kinetic<R>(const Dev<R> &, cudaStream_t);                                           \
    template void launch_zero_force<R>(const Dev<R> &, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace ljsel
