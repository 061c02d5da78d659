// cluster.cu -- LJ forces over cluster lists: the Verlet-list container of
// Sec. 2.2.1 with particles grouped into i-clusters.
//
// Each cell's sorted particles are cut into i-clusters of M consecutive
// particles (M = 2, 4 or 8; the last cluster of a cell may be shorter).  The
// list of an i-cluster holds every particle j outside the cluster that lies
// within r_c + skin of at least one member: the union of the members'
// Verlet lists, so a pair within r_c is always listed.  Pairs inside the
// cluster are evaluated once per cluster, without a list.  A group of T
// lanes owns one i-cluster.  Every lane keeps all M member positions and M
// force accumulators in registers and takes the list entries of the
// cluster's row in 16-byte chunks of four; the j position it loads serves M
// pair evaluations, and neighbouring lanes load neighbouring entries, which
// are mostly runs of consecutive sorted particles.  F_i is summed over the
// group's lanes by warp shuffles (a reduce-scatter: each halving step
// leaves every lane half of the members).  N3L (Sec. 2.1): a row holds only
// particles after the cluster (sorted order), so each unordered pair is
// listed once, and the lane sums -F_ij over the members in registers and
// adds it to F_j with one vector atomic per entry.  Without N3L the group
// fuses the Stormer-Verlet update.
//
// Rows are row-major, row c at cp + c * cp_cap (cp_cap a multiple of four):
// entries without a periodic image from the front, padded with the far
// sentinel particle n to a multiple of four, entries with one (27-bit index
// + 5-bit image code) from the back; cp_count[c] = front | back << 16.
#include <algorithm>

#include "kernels.cuh"
#include "update.cuh"

namespace ljsel {

namespace {

constexpr int CLB_THREADS = 128;  // list build: one warp per i-cluster
constexpr int CL_THREADS = 128;   // force: 128 / T i-clusters per block

template <typename R> struct CTab {
    R sig2[MAXT2], e24[MAXT2], e48[MAXT2], e4[MAXT2], ushift[MAXT2], lo[MAXT2], hi[MAXT2];
    double rc2d[MAXT2];
};

// ---------------------------------------------------------------------------
// List build.  One warp per i-cluster: the members sit in every lane's
// registers; the warp walks the stencil as (y, z) rows of cells whose x
// cells cx - RCH .. cx + RCH form at most three runs of consecutive sorted
// particles (split at a periodic x edge, each run with one image code), 32
// candidates at a time with coalesced loads.  A candidate outside the
// cluster is kept when its squared distance to some member is below
// r_list^2 (plain FP32: the list radius carries a 2^-12 relative margin);
// kept candidates are appended in lane order by ballot and prefix count.
// With N3L only candidates after the cluster's last member are walked.  (A
// periodic image of a member is never within r_list of the cluster: a
// periodic dimension has at least two cells of side >= r_list / 2 with
// L >= 2 r_list.)  A row whose final length exceeds the capacity is
// discarded and flagged; the host grows the rows and rebuilds.  The grid is
// capped (warps stride over the clusters), so that a launch that finds no
// rebuild due costs little.
template <typename R, int M, bool N3L, int RCH>
__global__ void __launch_bounds__(CLB_THREADS) k_cl_build(Dev<R> S) {
    Ctrl *C = S.ctrl;
    if (!C->rebuild_now) return;
    __shared__ unsigned long long s_entries;
    if (threadIdx.x == 0) s_entries = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int ncl = min(*S.ncl_total, S.ncl_cap);
    const int nwarps = (int)((gridDim.x * (unsigned)blockDim.x) >> 5);
    unsigned need = 0;
    for (int c = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5); c < ncl; c += nwarps) {
        const V4<R> *P = S.pos[C->pos_par];
        const int fi = S.cl_first[c], ni = S.cl_count[c];
        R mx[M], my[M], mz[M];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            const V4<R> q = ldpos(P, m < ni ? fi + m : S.n);  // the far sentinel stands in for absent members
            mx[m] = q.x; my[m] = q.y; mz[m] = q.z;
        }
        const int nx = S.nc[0], ny = S.nc[1], nz = S.nc[2];
        const int cell = S.cl_cell[c];
        const int cxy = cell % (nx * ny);
        const int cx = cxy % nx, cy = cxy / nx, cz = cell / (nx * ny);
        const int cap = S.cp_cap;
        uint32_t *row = S.cp + (size_t)c * cap;
        int nf = 0, nb = 0;
        for (int dz = -RCH; dz <= RCH; ++dz) {
            int wz, sz;
            if (!stencil_cell(cz, dz, nz, S.walls[2], wz, sz)) continue;
            for (int dy = -RCH; dy <= RCH; ++dy) {
                int wy, sy;
                if (!stencil_cell(cy, dy, ny, S.walls[1], wy, sy)) continue;
                int xa = cx - RCH, xb = cx + RCH;
                if (S.walls[0]) { xa = max(xa, 0); xb = min(xb, nx - 1); }
                const int rowc = (wz * ny + wy) * nx;
                for (int sx = -1; sx <= 1; ++sx) {
                    const int a = sx < 0 ? xa : (sx == 0 ? max(xa, 0) : max(xa, nx));
                    const int b = sx < 0 ? min(xb, -1) : (sx == 0 ? min(xb, nx - 1) : xb);
                    if (a > b) continue;
                    int jb = S.cell_start[rowc + a - sx * nx];
                    const int je = S.cell_start[rowc + b - sx * nx + 1];
                    if (N3L) jb = max(jb, fi + ni);
                    const uint32_t code = encode_image(sx, sy, sz);
                    const R shx = (R)sx * S.box[0], shy = (R)sy * S.box[1], shz = (R)sz * S.box[2];
                    for (int j0 = jb; j0 < je; j0 += 32) {
                        const int j = j0 + lane;
                        bool keep = false;
                        if (j < je && (N3L || code != 0 || j < fi || j >= fi + ni)) {
                            const V4<R> q = ldpos(P, j);
                            const R qx = q.x + shx, qy = q.y + shy, qz = q.z + shz;
                            R d2 = r2_of(mx[0] - qx, my[0] - qy, mz[0] - qz);
#pragma unroll
                            for (int m = 1; m < M; ++m) {
                                const R r2 = r2_of(mx[m] - qx, my[m] - qy, mz[m] - qz);
                                d2 = r2 < d2 ? r2 : d2;
                            }
                            keep = d2 < S.rlist2;
                        }
                        const unsigned mask = __ballot_sync(0xffffffffu, keep);
                        if (!mask) continue;
                        const int pos = __popc(mask & ((1u << lane) - 1u));
                        if (code == 0) {
                            const int k = nf + pos;
                            if (keep && k < cap) row[k] = (uint32_t)j;
                            nf += __popc(mask);
                        } else {
                            // an image entry only has to stay inside the row: if
                            // the final length fits, back and front cannot meet
                            const int k = nb + pos;
                            if (keep && k < cap) row[cap - 1 - k] = (uint32_t)j | (code << JBITS);
                            nb += __popc(mask);
                        }
                    }
                }
            }
        }
        // the front is read in 16-byte chunks of four: pad it with the far
        // sentinel particle n, whose pairs are never in range
        const int nf4 = (nf + 3) & ~3;
        need = max(need, (unsigned)(nf4 + nb));
        const bool fits = nf4 + nb <= cap && nf4 <= 0xffff && nb <= 0x7fff;
        if (fits && lane < nf4 - nf) row[nf + lane] = (uint32_t)S.n;
        if (lane == 0) {
            if (!fits) {
                C->overflow = 1;
                S.cp_count[c] = 0;
            } else {
                S.cp_count[c] = nf | (nb << 16);
                atomicAdd(&s_entries, (unsigned long long)(nf + nb));
            }
        }
    }
    warp_need_max(C, need);
    __syncthreads();
    if (threadIdx.x == 0 && s_entries) atomicAdd(reinterpret_cast<unsigned long long *>(&C->list_entries), s_entries);
}

// ---------------------------------------------------------------------------
// Shared pieces of the force kernels.
template <typename R, bool MT>
__device__ __forceinline__ void pair_consts(const Dev<R> &S, const CTab<R> &T, int tp, R &sig2, R &e24, R &e48, R &lo,
                                            R &hi, double &rc2d) {
    if (MT) {
        sig2 = T.sig2[tp]; e24 = T.e24[tp]; e48 = T.e48[tp]; lo = T.lo[tp]; hi = T.hi[tp]; rc2d = T.rc2d[tp];
    } else {
        sig2 = S.tab.sig2[0]; e24 = S.tab.e24[0]; e48 = S.tab.e48[0]; lo = S.tab.rc2lo[0]; hi = S.tab.rc2hi[0];
        rc2d = S.tab.rc2d[0];
    }
}

// 16-byte asynchronous global-to-shared copy (through L1) and its group
// bookkeeping.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void vadd(float4 *F, int j, float x, float y, float z) {
    atomicAdd(F + j, make_float4(x, y, z, 0.f));
}
__device__ __forceinline__ void vadd(D4 *F, int j, double x, double y, double z) {
    atomicAdd(&F[j].x, x); atomicAdd(&F[j].y, y); atomicAdd(&F[j].z, z);
}

// Reduce-scatter of the M force accumulators over the group's lanes (T a
// power of two, T >= M): at halving step s the lanes whose bit s is clear
// keep the first half of their current members and take the partner's
// partial sums of them, the others the second half.  Afterwards lane g
// holds the group's total force on member member_of<M>(g), summed over all
// T lanes.
template <int M> __device__ __forceinline__ int member_of(int g) {
    int m = 0;
#pragma unroll
    for (int s = 0, h = M / 2; h >= 1; ++s, h >>= 1) m += ((g >> s) & 1) * h;
    return m;
}
template <typename R, int M>
__device__ __forceinline__ void reduce_scatter(R (&fx)[M], R (&fy)[M], R (&fz)[M], int g, int T) {
#pragma unroll
    for (int s = 0, h = M / 2; h >= 1; ++s, h >>= 1) {
        const bool upper = (g >> s) & 1;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const R sx = upper ? fx[k] : fx[k + h], kx = upper ? fx[k + h] : fx[k];
            const R sy = upper ? fy[k] : fy[k + h], ky = upper ? fy[k + h] : fy[k];
            const R sz = upper ? fz[k] : fz[k + h], kz = upper ? fz[k + h] : fz[k];
            fx[k] = kx + __shfl_xor_sync(0xffffffffu, sx, 1 << s);
            fy[k] = ky + __shfl_xor_sync(0xffffffffu, sy, 1 << s);
            fz[k] = kz + __shfl_xor_sync(0xffffffffu, sz, 1 << s);
        }
    }
    for (int o = M; o < T; o <<= 1) {
        fx[0] += __shfl_xor_sync(0xffffffffu, fx[0], o);
        fy[0] += __shfl_xor_sync(0xffffffffu, fy[0], o);
        fz[0] += __shfl_xor_sync(0xffffffffu, fz[0], o);
    }
}

// ---------------------------------------------------------------------------
// Generic kernel: any precision, any number of types, energy and virial,
// pair export.  One listed particle j against the M members (absent members
// sit at the far sentinel and are never in range).
// With EXCL the entry is the cluster's own member b = j - first member:
// without N3L its pairs with every other member count (each inner pair is
// then seen from both sides, like every other pair), with N3L only those
// with members before it (each inner pair once).
template <typename R, int M, bool N3L, int MODE, bool EV, bool MT, bool EXCL = false>
__device__ __forceinline__ void cl_entry(const Dev<R> &S, const CTab<R> &T, const V4<R> (&pi)[M], const int (&ii)[M],
                                         const int (&ti)[M], int j, const V4<R> &pj, int sx, int sy, int sz,
                                         R (&fx)[M], R (&fy)[M], R (&fz)[M], double &u, double &w, int &np, int sp,
                                         int2 *pairs, long long pcap) {
    R gx = 0, gy = 0, gz = 0;
    const int tj = MT ? type_of(pj) : 0;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        R dx, dy, dz;
        if (sx == 0 && sy == 0 && sz == 0) {
            dx = pi[m].x - pj.x; dy = pi[m].y - pj.y; dz = pi[m].z - pj.z;
        } else {
            dx = image_dx(pi[m].x, pj.x, sx, S.box[0], S.box_lo[0]);
            dy = image_dx(pi[m].y, pj.y, sy, S.box[1], S.box_lo[1]);
            dz = image_dx(pi[m].z, pj.z, sz, S.box[2], S.box_lo[2]);
        }
        const R r2 = r2_of(dx, dy, dz);
        const int tp = MT ? ti[m] * S.tab.ntypes + tj : 0;
        R sig2, e24, e48, lo, hi;
        double rc2d;
        pair_consts<R, MT>(S, T, tp, sig2, e24, e48, lo, hi, rc2d);
        const bool pick = !EXCL || (N3L ? ii[m] < j : ii[m] != j);
        const bool in = pick && Cut<R>::in(r2, lo, hi, pi[m], pj, sx, sy, sz, S.boxd, rc2d);
        if (MODE == MODE_PAIRS) {
            if (in) {
                const int ia = S.id[sp][ii[m]], jb = S.id[sp][j];
                if (N3L || ia < jb) {
                    const unsigned long long k = atomicAdd(&S.ctrl->npairs, 1ull);
                    if ((long long)k < pcap) pairs[k] = make_int2(min(ia, jb), max(ia, jb));
                }
            }
            continue;
        }
        R sr6;
        R fr = lj_fr(r2, sig2, e24, e48, sr6);
        fr = in ? fr : (R)0;
        if (EV) {
            if (MT) u += in ? (double)(T.e4[tp] * sr6 * (sr6 - (R)1) - T.ushift[tp]) : 0.0;
            else { u += in ? (double)(sr6 * (sr6 - (R)1)) : 0.0; np += in ? 1 : 0; }
            w += (double)(fr * r2);
        }
        fx[m] += fr * dx; fy[m] += fr * dy; fz[m] += fr * dz;
        if (N3L) { gx -= fr * dx; gy -= fr * dy; gz -= fr * dz; }
    }
    if (N3L && MODE != MODE_PAIRS && j < S.n && (gx != (R)0 || gy != (R)0 || gz != (R)0)) vadd(S.force, j, gx, gy, gz);
}

template <typename R, int M, bool N3L, int MODE, bool EV, bool MT>
__global__ void __launch_bounds__(CL_THREADS) k_cl(Dev<R> S, int T, int2 *pairs, long long pcap) {
    Ctrl *C = S.ctrl;
    if (C->overflow) return;
    __shared__ CTab<R> Tb;
    if (MT) {
        for (int k = threadIdx.x; k < MAXT2; k += blockDim.x) {
            Tb.sig2[k] = S.tab.sig2[k]; Tb.e24[k] = S.tab.e24[k]; Tb.e48[k] = S.tab.e48[k]; Tb.e4[k] = S.tab.e4[k];
            Tb.ushift[k] = S.tab.ushift[k]; Tb.lo[k] = S.tab.rc2lo[k]; Tb.hi[k] = S.tab.rc2hi[k];
            Tb.rc2d[k] = S.tab.rc2d[k];
        }
        __syncthreads();
    }
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = gid / T, g = gid - c * T;
    const int ncl = min(*S.ncl_total, S.ncl_cap);
    const bool cvalid = c < ncl;
    const int pp = C->pos_par, sp = C->state_par;
    const V4<R> *P = S.pos[pp];
    int fi = 0, ni = 0, nf = 0, nb = 0;
    if (cvalid) {
        fi = S.cl_first[c];
        ni = S.cl_count[c];
        const int cnt = S.cp_count[c];
        nf = cnt & 0xffff;
        nb = cnt >> 16;
        if (!lj_check(fi >= 0 && ni >= 0 && ni <= M && fi + ni <= S.n, C, CHECK_CL_MEMBERS)) { fi = 0; ni = 0; nf = 0; nb = 0; }
        if (!lj_check(((nf + 3) & ~3) + nb <= S.cp_cap, C, CHECK_CL_ROW)) { nf = 0; nb = 0; }
    }
    V4<R> pi[M];
    int ii[M], ti[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        // absent members sit far from the box and from the sentinel particle
        // n of the row padding, so none of their pairs is ever in range
        ii[m] = m < ni ? fi + m : S.n;
        pi[m] = m < ni ? ldpos(P, ii[m]) : make_pos((R)-1e18, (R)-1e18, (R)-1e18, 0);
        ti[m] = type_of(pi[m]);
    }
    R fx[M], fy[M], fz[M];
#pragma unroll
    for (int m = 0; m < M; ++m) { fx[m] = 0; fy[m] = 0; fz[m] = 0; }
    double u = 0, w = 0;  // pair energies and virials (working precision) summed in FP64
    int np = 0;
    // pairs inside the cluster: lane g takes member g as one more entry
    if (g < ni) {
        const V4<R> pb = ldpos(P, fi + g);
        cl_entry<R, M, N3L, MODE, EV, MT, true>(S, Tb, pi, ii, ti, fi + g, pb, 0, 0, 0, fx, fy, fz, u, w, np, sp, pairs,
                                                pcap);
    }
    const int cap = S.cp_cap;
    const uint32_t *row = S.cp + (size_t)(cvalid ? c : 0) * cap;
    const int nq = (nf + 3) >> 2;
    const uint4 *rq = reinterpret_cast<const uint4 *>(row);
    uint4 en = g < nq ? __ldcs(rq + g) : make_uint4(0u, 0u, 0u, 0u);
    for (int q = g; q < nq; q += T) {
        uint4 e = en;
        if (q + T < nq) en = __ldcs(rq + q + T);
        const unsigned nn = (unsigned)S.n;  // the sentinel n pads the front
        if (!lj_check(e.x <= nn && e.y <= nn && e.z <= nn && e.w <= nn, C, CHECK_CL_FRONT)) e = make_uint4(nn, nn, nn, nn);
        const V4<R> p0 = ldpos(P, (int)e.x), p1 = ldpos(P, (int)e.y), p2 = ldpos(P, (int)e.z), p3 = ldpos(P, (int)e.w);
        cl_entry<R, M, N3L, MODE, EV, MT>(S, Tb, pi, ii, ti, (int)e.x, p0, 0, 0, 0, fx, fy, fz, u, w, np, sp, pairs, pcap);
        cl_entry<R, M, N3L, MODE, EV, MT>(S, Tb, pi, ii, ti, (int)e.y, p1, 0, 0, 0, fx, fy, fz, u, w, np, sp, pairs, pcap);
        cl_entry<R, M, N3L, MODE, EV, MT>(S, Tb, pi, ii, ti, (int)e.z, p2, 0, 0, 0, fx, fy, fz, u, w, np, sp, pairs, pcap);
        cl_entry<R, M, N3L, MODE, EV, MT>(S, Tb, pi, ii, ti, (int)e.w, p3, 0, 0, 0, fx, fy, fz, u, w, np, sp, pairs, pcap);
    }
    for (int e = g; e < nb; e += T) {
        const uint32_t ent = __ldcs(row + cap - 1 - e);
        const int j = (int)(ent & JMASK);
        if (!lj_check(j < S.n, C, CHECK_CL_BACK)) break;
        int sx, sy, sz;
        decode_image(ent >> JBITS, sx, sy, sz);
        const V4<R> pj = ldpos(P, j);
        cl_entry<R, M, N3L, MODE, EV, MT>(S, Tb, pi, ii, ti, j, pj, sx, sy, sz, fx, fy, fz, u, w, np, sp, pairs, pcap);
    }
    if (MODE == MODE_PAIRS) return;
    reduce_scatter<R, M>(fx, fy, fz, g, T);
    const int m = member_of<M>(g);
    double ke = 0;
    bool exceeded = false, bad = false;
    if (cvalid && g < M && m < ni) {
        const int i = fi + m;
        if (N3L) vadd(S.force, i, fx[0], fy[0], fz[0]);
        else if (MODE == MODE_FORCE) S.force[i] = make_pos(fx[0], fy[0], fz[0], 0);
        else integrate_one<R, EV>(S, sp, pp, C->half_kick, i, S.type[sp][i], fx[0], fy[0], fz[0], ke, exceeded, bad);
    }
    if (MODE == MODE_STEP) report_flags(C, exceeded, bad);
    if (EV) {
        const double e = MT ? u : (double)S.tab.e4[0] * u - (double)S.tab.ushift[0] * (double)np;
        const double scale = N3L ? 1.0 : 0.5;
        block_sum3(scale * e, scale * w, ke, C);
    }
}

// ---------------------------------------------------------------------------
// The stepping kernel of the FP32 single-type path (no energy, no pair
// export).  Members are evaluated two at a time with packed FP32x2
// arithmetic (one instruction for both halves, each half correctly rounded
// as its scalar counterpart, so r^2 is bit for bit the generic kernel's).
// The cutoff is decided in FP32 first: pairs inside the narrow band around
// r_c^2 are left out, and an entry whose r^2 came near the band is flagged;
// when any lane of the warp flagged one, the lanes re-derive which of their
// pairs were in the band and decide those with the exact FP64 predicate --
// the same decision as the generic kernel, without a divergent call per
// pair.  The positions of a lane's next chunk are copied into its own
// shared-memory stage by cp.async while it evaluates the current chunk (two
// stages, each read back only by the lane that filled it).
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float &half_of(float2 &v, int b) { return b ? v.y : v.x; }
__device__ __forceinline__ float half_of(const float2 &v, int b) { return b ? v.y : v.x; }

struct FastTab {
    float2 a2, nb2;     // 48 eps sigma^12 and -24 eps sigma^6: f/r = s^4 (a s^3 - b) with s = 1 / r^2
    float lo, hi;       // FP32 band around r_c^2 (as in Cut<float>)
    unsigned lo_bits;   // bit pattern of lo; r^2 >= 0 orders like its bit pattern
    unsigned band_bits; // bits(hi) - bits(lo): lo <= r^2 <= hi iff bits(r^2) - bits(lo) <= band_bits (unsigned)
};

// The pairs of one half-pair h of members with one listed particle, given
// their displacements: returns whether r^2 of a counted pair fell in the
// band (such a pair is left out here).  ka / kb: whether each half counts.
template <bool N3L>
__device__ __forceinline__ bool fast_pairs(const float2 &dx, const float2 &dy, const float2 &dz, bool ka, bool kb,
                                           float2 &fx, float2 &fy, float2 &fz, float2 &gx, float2 &gy, float2 &gz,
                                           const FastTab &t) {
    float2 r2 = __fmul2_rn(dx, dx);
    r2 = __ffma2_rn(dy, dy, r2);
    r2 = __ffma2_rn(dz, dz, r2);
    const bool near = (ka && __float_as_uint(r2.x) - t.lo_bits <= t.band_bits) ||
                      (kb && __float_as_uint(r2.y) - t.lo_bits <= t.band_bits);
    // out of range or excluded (the member itself, at distance 0): s = 0
    const float2 sv = make_float2(ka && r2.x < t.lo ? fast_rcp(r2.x) : 0.f, kb && r2.y < t.lo ? fast_rcp(r2.y) : 0.f);
    const float2 s2 = __fmul2_rn(sv, sv);
    const float2 fr = __fmul2_rn(__fmul2_rn(s2, s2), __ffma2_rn(t.a2, __fmul2_rn(s2, sv), t.nb2));
    fx = __ffma2_rn(fr, dx, fx);
    fy = __ffma2_rn(fr, dy, fy);
    fz = __ffma2_rn(fr, dz, fz);
    if (N3L) {
        gx = __ffma2_rn(fr, dx, gx);
        gy = __ffma2_rn(fr, dy, gy);
        gz = __ffma2_rn(fr, dz, gz);
    }
    return near;
}

// One listed particle j against the members: returns whether r^2 of some
// counted pair fell in the band (those pairs are left out here).  With EXCL
// the entry is the cluster's own member b (see cl_entry): member m's half
// counts only when m != b (without N3L) or m < b (with N3L).
template <int M, bool N3L, bool EXCL = false>
__device__ __forceinline__ bool fast_entry(const float4 &pj, const float2 (&mx)[M / 2], const float2 (&my)[M / 2],
                                           const float2 (&mz)[M / 2], float2 (&fx)[M / 2], float2 (&fy)[M / 2],
                                           float2 (&fz)[M / 2], float2 &gx, float2 &gy, float2 &gz,
                                           const FastTab &t, int b = 0) {
    const float2 jx = f2(pj.x), jy = f2(pj.y), jz = f2(pj.z);
    bool near = false;
#pragma unroll
    for (int h = 0; h < M / 2; ++h) {
        const bool ka = !EXCL || (N3L ? 2 * h < b : 2 * h != b);
        const bool kb = !EXCL || (N3L ? 2 * h + 1 < b : 2 * h + 1 != b);
        near |= fast_pairs<N3L>(sub2(mx[h], jx), sub2(my[h], jy), sub2(mz[h], jz), ka, kb, fx[h], fy[h], fz[h], gx, gy,
                                gz, t);
    }
    return near;
}

// image_dx on both halves: x_i - (x_j + s L) from the rounded difference,
// its exact rounding error and the two parts of L, each operation rounded
// as in the scalar form, so both halves equal image_dx bit for bit.
__device__ __forceinline__ float2 image_dx2(const float2 &xi, float xj, int s, float L, float Llo) {
    const float2 j2 = f2(xj);
    const float2 d = sub2(xi, j2);
    const float2 bb = sub2(d, xi);
    const float2 lo = __fadd2_rn(sub2(xi, sub2(d, bb)), sub2(f2(-xj), bb));
    const float sL = s > 0 ? L : -L;
    const float sLlo = s > 0 ? Llo : -Llo;
    const float2 r = __fadd2_rn(sub2(d, f2(sL)), sub2(lo, f2(sLlo)));
    return s == 0 ? d : r;
}

// One listed particle j with periodic image (sx, sy, sz) against the members.
template <int M, bool N3L>
__device__ __forceinline__ bool fast_image_entry(const float4 &pj, int sx, int sy, int sz, const Dev<float> &S,
                                                 const float2 (&mx)[M / 2], const float2 (&my)[M / 2],
                                                 const float2 (&mz)[M / 2], float2 (&fx)[M / 2], float2 (&fy)[M / 2],
                                                 float2 (&fz)[M / 2], float2 &gx, float2 &gy, float2 &gz,
                                                 const FastTab &t) {
    bool near = false;
#pragma unroll
    for (int h = 0; h < M / 2; ++h)
        near |= fast_pairs<N3L>(image_dx2(mx[h], pj.x, sx, S.box[0], S.box_lo[0]),
                                image_dx2(my[h], pj.y, sy, S.box[1], S.box_lo[1]),
                                image_dx2(mz[h], pj.z, sz, S.box[2], S.box_lo[2]), true, true, fx[h], fy[h], fz[h], gx,
                                gy, gz, t);
    return near;
}

// The band pairs of one flagged entry (the pairs the fast path left out:
// lo <= r^2 <= hi), decided exactly; sx..sz its image.
template <int M, bool N3L, bool EXCL = false>
__device__ __forceinline__ void band_entry(const Dev<float> &S, const float4 &pj, int sx, int sy, int sz,
                                           const float2 (&mx)[M / 2], const float2 (&my)[M / 2],
                                           const float2 (&mz)[M / 2], float2 (&fx)[M / 2], float2 (&fy)[M / 2],
                                           float2 (&fz)[M / 2], float &hx, float &hy, float &hz, const FastTab &t,
                                           int b = 0) {
#pragma unroll
    for (int m = 0; m < M; ++m) {
        if (EXCL && (N3L ? m >= b : m == b)) continue;
        const float xi = half_of(mx[m / 2], m & 1), yi = half_of(my[m / 2], m & 1), zi = half_of(mz[m / 2], m & 1);
        const float dx = image_dx(xi, pj.x, sx, S.box[0], S.box_lo[0]);
        const float dy = image_dx(yi, pj.y, sy, S.box[1], S.box_lo[1]);
        const float dz = image_dx(zi, pj.z, sz, S.box[2], S.box_lo[2]);
        const float r2 = r2_of(dx, dy, dz);
        if (r2 < t.lo || !(r2 <= t.hi)) continue;
        if (!exact_in_range(xi, yi, zi, pj.x, pj.y, pj.z, sx, sy, sz, S.boxd, S.tab.rc2d[0])) continue;
        float sr6;
        const float fr = lj_fr(r2, S.tab.sig2[0], S.tab.e24[0], S.tab.e48[0], sr6);
        half_of(fx[m / 2], m & 1) += fr * dx;
        half_of(fy[m / 2], m & 1) += fr * dy;
        half_of(fz[m / 2], m & 1) += fr * dz;
        if (N3L) { hx += fr * dx; hy += fr * dy; hz += fr * dz; }
    }
}

// Register bound by cluster size (measured on the 1M liquid): M = 2, 80
// registers (24 warps per SM) without N3L, 64 (32 warps) with N3L; M = 4, 80
// (24 warps); M = 8, 128 (16 warps).
template <int M, bool N3L, int MODE>
__global__ void __launch_bounds__(CL_THREADS, M == 2 ? (N3L ? 8 : 6) : (M == 4 ? 6 : 4)) k_cl_fast(Dev<float> S, int T) {
    Ctrl *C = S.ctrl;
    if (C->overflow) return;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = gid / T, g = gid - c * T;
    const int ncl = min(*S.ncl_total, S.ncl_cap);
    const bool cvalid = c < ncl;
    const int pp = C->pos_par, sp = C->state_par;
    const float4 *P = S.pos[pp];
    int fi = 0, ni = 0, nf = 0, nb = 0;
    if (cvalid) {
        fi = S.cl_first[c];
        ni = S.cl_count[c];
        const int cnt = S.cp_count[c];
        nf = cnt & 0xffff;
        nb = cnt >> 16;
        if (!lj_check(fi >= 0 && ni >= 0 && ni <= M && fi + ni <= S.n, C, CHECK_CL_MEMBERS)) { fi = 0; ni = 0; nf = 0; nb = 0; }
        if (!lj_check(((nf + 3) & ~3) + nb <= S.cp_cap, C, CHECK_CL_ROW)) { nf = 0; nb = 0; }
    }
    float2 mx[M / 2], my[M / 2], mz[M / 2], fx[M / 2], fy[M / 2], fz[M / 2];
    // absent members sit far from the box and from the sentinel particle n
    // of the row padding, so none of their pairs is ever in range
    const float4 far = make_float4(-1e18f, -1e18f, -1e18f, 0.f);
#pragma unroll
    for (int h = 0; h < M / 2; ++h) {
        const float4 a = 2 * h < ni ? __ldg(P + fi + 2 * h) : far;
        const float4 b = 2 * h + 1 < ni ? __ldg(P + fi + 2 * h + 1) : far;
        mx[h] = make_float2(a.x, b.x);
        my[h] = make_float2(a.y, b.y);
        mz[h] = make_float2(a.z, b.z);
        fx[h] = fy[h] = fz[h] = f2(0.f);
    }
    FastTab t;
    t.a2 = f2(S.tab.a12[0]);
    t.nb2 = f2(-S.tab.b6[0]);
    t.lo = S.tab.rc2lo[0];
    t.hi = S.tab.rc2hi[0];
    t.lo_bits = __float_as_uint(t.lo);
    t.band_bits = __float_as_uint(t.hi) - t.lo_bits;
    const int cap = S.cp_cap;
    const uint32_t *row = S.cp + (size_t)(cvalid ? c : 0) * cap;
    const int nq = (nf + 3) >> 2;
    const uint4 *rq = reinterpret_cast<const uint4 *>(row);
    __shared__ __align__(16) float4 s_stage[2][4][CL_THREADS];
    const int tid = threadIdx.x;
    auto issue = [&](int st, uint4 e) {
        const unsigned nn = (unsigned)S.n;  // the sentinel n pads the front
        if (!lj_check(e.x <= nn && e.y <= nn && e.z <= nn && e.w <= nn, C, CHECK_CL_FRONT)) e = make_uint4(nn, nn, nn, nn);
        cp_async16(&s_stage[st][0][tid], P + e.x);
        cp_async16(&s_stage[st][1][tid], P + e.y);
        cp_async16(&s_stage[st][2][tid], P + e.z);
        cp_async16(&s_stage[st][3][tid], P + e.w);
    };
    int st = 0;
    // one chunk of four entries: the four are evaluated before a single
    // vote, so that their arithmetic can interleave; the band pairs of the
    // flagged entries are then decided exactly.  With N3L each entry's
    // -F_ij goes to F_j at once, and a band pair's with one more atomic.
    auto chunk = [&](const float4 (&pj)[4], const uint4 &e) {
        const unsigned js[4] = {e.x, e.y, e.z, e.w};
        unsigned nm = 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 gx = f2(0.f), gy = f2(0.f), gz = f2(0.f);
            nm |= (fast_entry<M, N3L>(pj[k], mx, my, mz, fx, fy, fz, gx, gy, gz, t) ? 1u : 0u) << k;
            if (N3L) {
                const float hx = gx.x + gx.y, hy = gy.x + gy.y, hz = gz.x + gz.y;
                if (js[k] < (unsigned)S.n && (hx != 0.f || hy != 0.f || hz != 0.f))
                    atomicAdd(S.force + js[k], make_float4(-hx, -hy, -hz, 0.f));
            }
        }
        // the vote runs among the lanes still in the loop (groups of a warp
        // have rows of different length)
        if (__any_sync(__activemask(), nm != 0u) && nm) {
            while (nm) {
                const int k = __ffs(nm) - 1;
                nm &= nm - 1u;
                const float4 q = s_stage[st][k][tid];  // reloaded: pj need not stay in registers
                float bx = 0.f, by = 0.f, bz = 0.f;
                band_entry<M, N3L>(S, q, 0, 0, 0, mx, my, mz, fx, fy, fz, bx, by, bz, t);
                const unsigned j = k == 0 ? js[0] : (k == 1 ? js[1] : (k == 2 ? js[2] : js[3]));
                if (N3L && j < (unsigned)S.n && (bx != 0.f || by != 0.f || bz != 0.f))
                    atomicAdd(S.force + j, make_float4(-bx, -by, -bz, 0.f));
            }
        }
    };
    uint4 e0 = make_uint4(0u, 0u, 0u, 0u), e1 = e0;
    if (g < nq) { e0 = __ldcs(rq + g); issue(0, e0); }
    cp_async_commit();
    if (g + T < nq) e1 = __ldcs(rq + g + T);
    // pairs inside the cluster: lane g takes member g as one more entry
    if (g < ni) {
        const float4 pb = __ldg(P + fi + g);
        float2 gx = f2(0.f), gy = f2(0.f), gz = f2(0.f);
        const bool near = fast_entry<M, N3L, true>(pb, mx, my, mz, fx, fy, fz, gx, gy, gz, t, g);
        float hx = gx.x + gx.y, hy = gy.x + gy.y, hz = gz.x + gz.y;
        if (near) band_entry<M, N3L, true>(S, pb, 0, 0, 0, mx, my, mz, fx, fy, fz, hx, hy, hz, t, g);
        if (N3L && (hx != 0.f || hy != 0.f || hz != 0.f)) atomicAdd(S.force + fi + g, make_float4(-hx, -hy, -hz, 0.f));
    }
    for (int q = g; q < nq; q += T) {
        if (q + T < nq) issue(st ^ 1, e1);
        cp_async_commit();
        const uint4 e = e0;
        e0 = e1;
        if (q + 2 * T < nq) e1 = __ldcs(rq + q + 2 * T);
        cp_async_wait_1();
        const float4 pj[4] = {s_stage[st][0][tid], s_stage[st][1][tid], s_stage[st][2][tid], s_stage[st][3][tid]};
        chunk(pj, e);
        st ^= 1;
    }
    cp_async_wait_all();
    // entries with a periodic image: the same packed arithmetic with the
    // image displacement of image_dx
    for (int e = g; e < nb; e += T) {
        const uint32_t ent = __ldcs(row + cap - 1 - e);
        const int j = (int)(ent & JMASK);
        if (!lj_check(j < S.n, C, CHECK_CL_BACK)) break;
        int sx, sy, sz;
        decode_image(ent >> JBITS, sx, sy, sz);
        const float4 pj = __ldg(P + j);
        float2 gx = f2(0.f), gy = f2(0.f), gz = f2(0.f);
        const bool near = fast_image_entry<M, N3L>(pj, sx, sy, sz, S, mx, my, mz, fx, fy, fz, gx, gy, gz, t);
        float hx = gx.x + gx.y, hy = gy.x + gy.y, hz = gz.x + gz.y;
        if (__any_sync(__activemask(), near) && near)
            band_entry<M, N3L>(S, pj, sx, sy, sz, mx, my, mz, fx, fy, fz, hx, hy, hz, t);
        if (N3L && (hx != 0.f || hy != 0.f || hz != 0.f)) atomicAdd(S.force + j, make_float4(-hx, -hy, -hz, 0.f));
    }
    float ax[M], ay[M], az[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        ax[m] = half_of(fx[m / 2], m & 1);
        ay[m] = half_of(fy[m / 2], m & 1);
        az[m] = half_of(fz[m / 2], m & 1);
    }
    reduce_scatter<float, M>(ax, ay, az, g, T);
    const int m = member_of<M>(g);
    double ke = 0;
    bool exceeded = false, bad = false;
    if (cvalid && g < M && m < ni) {
        const int i = fi + m;
        if (N3L) vadd(S.force, i, ax[0], ay[0], az[0]);
        else if (MODE == MODE_FORCE) S.force[i] = make_float4(ax[0], ay[0], az[0], 0.f);
        else integrate_one<float, false>(S, sp, pp, C->half_kick, i, S.type[sp][i], ax[0], ay[0], az[0], ke, exceeded, bad);
    }
    if (MODE == MODE_STEP) report_flags(C, exceeded, bad);
}

template <int M, bool N3L, int MODE>
void cl_fast_go(const Dev<float> &S, int T, cudaStream_t st) {
    const long long threads = (long long)S.ncl_cap * T;
    k_cl_fast<M, N3L, MODE><<<div_up(threads, CL_THREADS), CL_THREADS, 0, st>>>(S, T);
}

template <int M>
void cl_fast_modes(const Dev<float> &S, const ljsel_config &cfg, int mode, cudaStream_t st) {
    const int T = cfg.threads_per_unit;
    if (cfg.newton3) cl_fast_go<M, true, MODE_FORCE>(S, T, st);
    else if (mode == MODE_STEP) cl_fast_go<M, false, MODE_STEP>(S, T, st);
    else cl_fast_go<M, false, MODE_FORCE>(S, T, st);
}

template <typename R, int M, bool N3L, int MODE, bool EV, bool MT>
void cl_go(const Dev<R> &S, int T, int2 *pairs, long long pcap, cudaStream_t st) {
    const long long threads = (long long)S.ncl_cap * T;
    k_cl<R, M, N3L, MODE, EV, MT><<<div_up(threads, CL_THREADS), CL_THREADS, 0, st>>>(S, T, pairs, pcap);
}

template <typename R, int M, bool MT>
void cl_modes(const Dev<R> &S, const ljsel_config &cfg, int mode, bool ev, int2 *pairs, long long pcap,
              cudaStream_t st) {
    const bool n3l = cfg.newton3 != 0;
    const int T = cfg.threads_per_unit;
    if (mode == MODE_PAIRS) {
        n3l ? cl_go<R, M, true, MODE_PAIRS, false, MT>(S, T, pairs, pcap, st)
            : cl_go<R, M, false, MODE_PAIRS, false, MT>(S, T, pairs, pcap, st);
        return;
    }
    if (n3l) {
        ev ? cl_go<R, M, true, MODE_FORCE, true, MT>(S, T, pairs, pcap, st)
           : cl_go<R, M, true, MODE_FORCE, false, MT>(S, T, pairs, pcap, st);
        return;
    }
    if (mode == MODE_STEP) {
        ev ? cl_go<R, M, false, MODE_STEP, true, MT>(S, T, pairs, pcap, st)
           : cl_go<R, M, false, MODE_STEP, false, MT>(S, T, pairs, pcap, st);
        return;
    }
    ev ? cl_go<R, M, false, MODE_FORCE, true, MT>(S, T, pairs, pcap, st)
       : cl_go<R, M, false, MODE_FORCE, false, MT>(S, T, pairs, pcap, st);
}

template <typename R, bool MT>
void cl_dispatch(const Dev<R> &S, const ljsel_config &cfg, int mode, bool ev, int2 *pairs, long long pcap,
                 cudaStream_t st) {
    switch (S.M) {
        case 2: cl_modes<R, 2, MT>(S, cfg, mode, ev, pairs, pcap, st); break;
        case 4: cl_modes<R, 4, MT>(S, cfg, mode, ev, pairs, pcap, st); break;
        default: cl_modes<R, 8, MT>(S, cfg, mode, ev, pairs, pcap, st); break;
    }
}

template <typename R, int M, bool N3L>
void cl_build_go(const Dev<R> &S, cudaStream_t st) {
    const int blocks = std::min(div_up((long long)S.ncl_cap * 32, CLB_THREADS), 152 * 16);
    if (S.reach == 1) k_cl_build<R, M, N3L, 1><<<blocks, CLB_THREADS, 0, st>>>(S);
    else k_cl_build<R, M, N3L, 2><<<blocks, CLB_THREADS, 0, st>>>(S);
}

}  // namespace

template <typename R> void launch_cp_build(const Dev<R> &S, bool n3l, cudaStream_t st) {
    switch (S.M) {
        case 2: n3l ? cl_build_go<R, 2, true>(S, st) : cl_build_go<R, 2, false>(S, st); break;
        case 4: n3l ? cl_build_go<R, 4, true>(S, st) : cl_build_go<R, 4, false>(S, st); break;
        default: n3l ? cl_build_go<R, 8, true>(S, st) : cl_build_go<R, 8, false>(S, st); break;
    }
}
template void launch_cp_build<float>(const Dev<float> &, bool, cudaStream_t);
template void launch_cp_build<double>(const Dev<double> &, bool, cudaStream_t);

template <typename R> void launch_cp_force(const Dev<R> &S, const ljsel_config &cfg, int mode, bool ev, int2 *pairs,
                                           long long cap, cudaStream_t st);
template <> void launch_cp_force<float>(const Dev<float> &S, const ljsel_config &cfg, int mode, bool ev, int2 *pairs,
                                        long long cap, cudaStream_t st) {
    if (S.tab.ntypes == 1 && !ev && mode != MODE_PAIRS) {
        switch (S.M) {
            case 2: cl_fast_modes<2>(S, cfg, mode, st); break;
            case 4: cl_fast_modes<4>(S, cfg, mode, st); break;
            default: cl_fast_modes<8>(S, cfg, mode, st); break;
        }
        return;
    }
    if (S.tab.ntypes > 1) cl_dispatch<float, true>(S, cfg, mode, ev, pairs, cap, st);
    else cl_dispatch<float, false>(S, cfg, mode, ev, pairs, cap, st);
}
template <> void launch_cp_force<double>(const Dev<double> &S, const ljsel_config &cfg, int mode, bool ev, int2 *pairs,
                                         long long cap, cudaStream_t st) {
    cl_dispatch<double, true>(S, cfg, mode, ev, pairs, cap, st);
}

}  // namespace ljsel
