// rebuild.cu -- neighbour-structure rebuild on the GPU (Sec. 2.2.1).
//
// Linked cells as a counting sort: each particle is binned by its working
// position into cells of side >= (r_c + skin) * CSF (stretched to tile the
// box), cell counts are scanned in one decoupled look-back pass, particles
// are scattered into their cell segments, ordered inside each cell by a
// sub-cell Morton key (ties by input index, so the order is deterministic),
// and the FP64 state is gathered into the new order.  Verlet lists (one
// row per particle) and cluster-pair lists (one row per i-cluster of M
// particles) are then built from the cells with radius r_c + skin.
#include "kernels.cuh"

namespace ljsel {

namespace {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;
constexpr unsigned long long FLAG_A = 1ull << 62;  // tile aggregate published
constexpr unsigned long long FLAG_P = 2ull << 62;  // inclusive prefix published
constexpr unsigned long long VAL_MASK = (1ull << 62) - 1ull;
constexpr int SPIN_LIMIT = 1 << 22;
constexpr int VL_BUILD_THREADS = 128;
constexpr int VL_BUILD_MIN_BLOCKS = 8;  // 32 warps per SM: at most 64 registers a thread
constexpr int VL_WBUILD_THREADS = 256;  // eight particles a block in the warp-per-particle build
// Small systems build their Verlet lists with a warp per particle, larger
// ones with a thread per particle.  The limits are where the two measured
// equal on a liquid at rho 0.8442: about 24k particles when the stencil is
// 27 cells of side r_list (CSF 1), about 8k for 125 cells of half that side
// (CSF 0.5), whose runs of five small cells leave more of a warp's lanes
// idle.  Below them the one-thread build leaves most SMs with one or two
// warps, each walking its candidates one load after another.
#ifndef VL_WARP_BUILD_MAX_N
#define VL_WARP_BUILD_MAX_N 24576
#endif
#ifndef VL_WARP_BUILD_MAX_N_HALF_CELLS
#define VL_WARP_BUILD_MAX_N_HALF_CELLS 8192
#endif

__device__ __forceinline__ unsigned morton3(unsigned x, unsigned y, unsigned z) {
    unsigned k = 0;
    for (int b = 0; b < 3; ++b) k |= (((x >> b) & 1u) << (3 * b)) | (((y >> b) & 1u) << (3 * b + 1)) | (((z >> b) & 1u) << (3 * b + 2));
    return k;
}

template <typename R>
__global__ void k_bin(Dev<R> S, int ntiles) {
    Ctrl *C = S.ctrl;
    if (!C->rebuild_now) return;
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < ntiles) reinterpret_cast<unsigned long long *>(S.scan_partial)[p] = 0ull;
    if (p == 0) {
        C->need_cap = 0;
        C->list_entries = 0;
        C->window_overflow = 0;
        if (S.nstrips) *S.nstrips = 0;
    }
    // every lane stays to the warp-wide match below; lanes past n bin nothing
    const bool valid = p < S.n;
    const int pp = valid ? p : 0;
    const int sp = C->state_par;
    double *X = S.x[sp];
    int c3[3];
    unsigned sub[3];
    bool bad = false;
    for (int d = 0; d < 3; ++d) {
        double xd = X[d * S.n + pp];
        // FP64 arithmetic is scarce on this part: decide "0 < x < L" on the
        // float rounding (rounding is monotonic, so 0 < (float)x < box_dn
        // implies it exactly) and take the FP64 path only for the particles
        // that left the box
        const float xf = (float)xd;
        if (!(xf > 0.0f && xf < S.box_dn[d])) {
            const double L = S.boxd[d];
            if (!(xd == xd) || fabs(xd) > 4.0 * L) { bad = true; xd = 0.0; }
            if (!S.walls[d]) {  // periodic: wrap (between walls positions stay in [0, L])
                if (xd < 0.0) xd += L;
                if (xd >= L) xd -= L;
                if (xd < 0.0 || xd >= L) { xd = xd - L * floor(xd / L); if (xd >= L) xd = 0.0; }
            }
            if (valid) X[d * S.n + p] = xd;
        }
        R w = (R)xd;
        R f = w * S.inv_side[d];
        int c = (int)floor(f);
        c = c < 0 ? 0 : (c > S.nc[d] - 1 ? S.nc[d] - 1 : c);
        int s = (int)((f - (R)c) * (R)8);
        sub[d] = (unsigned)(s < 0 ? 0 : (s > 7 ? 7 : s));
        c3[d] = c;
    }
    if (bad && valid) C->nonfinite = 1;
    const int cell = valid ? (c3[2] * S.nc[1] + c3[1]) * S.nc[0] + c3[0] : -1;
    // slots in the cell: one atomic per distinct cell of the warp (the lanes
    // of a warp are neighbours from the last sort and share one or two cells)
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(0xffffffffu, cell);
    const int leader = __ffs(peers) - 1;
    int base = 0;
    if (valid && lane == leader) base = atomicAdd(&S.cell_count[cell], __popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!valid) return;
    S.cell_of[p] = cell;
    S.slot_of[p] = base + __popc(peers & ((1u << lane) - 1u));
    S.key_of[p] = ((unsigned long long)morton3(sub[0], sub[1], sub[2]) << 32) | (unsigned)S.id[sp][p];
}

__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Exclusive scan of (count, ceil(count / M)) packed as hi/lo 31-bit fields of
// one 64-bit word.  Tiles take tickets in launch order, publish their
// aggregate, then look back over predecessors (which hold earlier tickets and
// so are running or done); every wait is bounded and sets Ctrl::timeout.
template <typename R>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan(Dev<R> S, int M, int ntiles) {
    Ctrl *C = S.ctrl;
    if (!C->rebuild_now) return;
    __shared__ int s_tile;
    __shared__ unsigned long long s_warp[SCAN_THREADS / 32];
    __shared__ unsigned long long s_excl;
    if (threadIdx.x == 0) {
        int t = atomicAdd(&C->scan_ticket, 1);
        if (t == ntiles - 1) C->scan_ticket = 0;
        s_tile = t;
    }
    __syncthreads();
    const int tile = s_tile;
    const int base = tile * SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    unsigned long long item[SCAN_ITEMS];
    unsigned long long run = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int c = base + k;
        int cnt = c < S.ncell ? S.cell_count[c] : 0;
        unsigned long long v = ((unsigned long long)cnt << 31) | (unsigned long long)((cnt + M - 1) / M);
        item[k] = run;
        run += v;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = warp_incl_scan(run);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < SCAN_THREADS / 32 ? s_warp[lane] : 0ull;
        unsigned long long wi = warp_incl_scan(w);
        if (lane < SCAN_THREADS / 32) s_warp[lane] = wi - w;  // exclusive per warp
        if (lane == SCAN_THREADS / 32 - 1) {
            unsigned long long agg = wi;
            volatile unsigned long long *st = reinterpret_cast<volatile unsigned long long *>(S.scan_partial);
            unsigned long long excl = 0;
            if (tile == 0) {
                __threadfence();
                atomicExch(reinterpret_cast<unsigned long long *>(S.scan_partial), FLAG_P | agg);
            } else {
                __threadfence();
                atomicExch(reinterpret_cast<unsigned long long *>(S.scan_partial) + tile, FLAG_A | agg);
                int p = tile - 1;
                while (p >= 0) {
                    const unsigned long long v = spin_until(st + p, FLAG_A | FLAG_P, SPIN_LIMIT);
                    if (!(v & (FLAG_A | FLAG_P))) { C->timeout = 1; break; }
                    excl += v & VAL_MASK;
                    if (v & FLAG_P) break;
                    --p;
                }
                __threadfence();
                atomicExch(reinterpret_cast<unsigned long long *>(S.scan_partial) + tile, FLAG_P | ((excl + agg) & VAL_MASK));
            }
            s_excl = excl;
            if (tile == ntiles - 1) {
                unsigned long long tot = excl + agg;
                S.cell_start[S.ncell] = (int)(tot >> 31);
                S.clcell_start[S.ncell] = (int)(tot & 0x7fffffffull);
                *S.ncl_total = (int)(tot & 0x7fffffffull);
            }
        }
    }
    __syncthreads();
    const unsigned long long off = s_excl + s_warp[warp] + (incl - run);
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        int c = base + k;
        if (c < S.ncell) {
            unsigned long long v = off + item[k];
            S.cell_start[c] = (int)(v >> 31);
            S.clcell_start[c] = (int)(v & 0x7fffffffull);
            S.cell_count[c] = 0;
        }
    }
}

template <typename R>
__global__ void k_scatter(Dev<R> S) {
    Ctrl *C = S.ctrl;
    if (!C->rebuild_now) return;
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= S.n) return;
    const int cell = S.cell_of[p];
    const int dst = S.cell_start[cell] + S.slot_of[p];
    S.tmp_idx[dst] = p;
    S.tmp_key[dst] = S.key_of[p];
    S.cell_sorted[dst] = cell;  // the slot's cell: its final occupant is in the same cell
}

template <typename R>
__device__ __forceinline__ void gather_one(const Dev<R> &S, int sp, int pp, int q, int p) {
    const int n = S.n;
    const double *X = S.x[sp];
    const double *V = S.v[sp];
    double *Xn = S.x[sp ^ 1];
    double *Vn = S.v[sp ^ 1];
    double x0 = X[p], x1 = X[n + p], x2 = X[2 * n + p];
    Xn[q] = x0; Xn[n + q] = x1; Xn[2 * n + q] = x2;
    Vn[q] = V[p]; Vn[n + q] = V[n + p]; Vn[2 * n + q] = V[2 * n + p];
    S.id[sp ^ 1][q] = S.id[sp][p];
    int t = S.type[sp][p];
    S.type[sp ^ 1][q] = t;
    V4<R> w = make_pos((R)x0, (R)x1, (R)x2, t);
    S.pos[pp][q] = w;
    S.xref[q] = w;
}

// One thread per slot of the scattered order: the element's rank among the
// keys of its cell segment is its final place in the cell; the particle
// state is gathered there.  The lanes of a warp cover one or two cells, so
// the key reads are shared.
template <typename R>
__global__ void k_sortgather(Dev<R> S) {
    Ctrl *C = S.ctrl;
    if (!C->rebuild_now) return;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= S.n) return;
    const int sp = C->state_par, pp = C->pos_par;
    const int cell = S.cell_sorted[e];
    const int start = S.cell_start[cell], m = S.cell_start[cell + 1] - start;
    const unsigned long long key = S.tmp_key[e];
    int rank = 0;
    for (int f = 0; f < m; ++f) rank += S.tmp_key[start + f] < key ? 1 : 0;
    const int src = S.tmp_idx[e];
    if (!lj_check(start + rank < S.n && src >= 0 && src < S.n, C, CHECK_SORT_SLOT)) return;
    gather_one(S, sp, pp, start + rank, src);
}

// Verlet-list rows, one thread per sorted particle i: all j with
// r^2 < r_list^2 (working precision) in the stencil of (2 RCH + 1)^3 cells
// (RCH = 1 for CSF 1, 2 for CSF 0.5), j != i; with N3L only the geometric
// half stencil.  The stencil is walked as (y, z) rows of cells; in each row
// the x cells cx - RCH .. cx + RCH form one run of consecutive sorted
// particles, split only at a periodic x edge.  Candidates are tested four at
// a time into a 32-bit mask per block of 32 (in FP32 the sign bits of
// r^2 - r_list^2 are funnel-shifted in); only the set bits are appended.
// The 32 lanes of a warp are 32 consecutive sorted particles and share most
// of their runs (cutting each particle's runs to the reach of the list
// radius tests far fewer candidates but makes the lanes' trip counts differ,
// and measured no faster).  Entries without an image go to the front of the
// row in 16-byte chunks of four, padded with the sentinel index n; entries
// with an image go to the back, one by one.  The list test needs no exact
// image arithmetic: the list radius carries a relative margin of 2^-12, far
// above the rounding of a plain shift, so i is shifted once per run.
template <typename R, bool N3L, int RCH>
__global__ void __launch_bounds__(VL_BUILD_THREADS, VL_BUILD_MIN_BLOCKS) k_vl_build(Dev<R> S) {
    Ctrl *C = S.ctrl;
    if (!C->rebuild_now) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = i < S.n;
    const int ii = act ? i : S.n - 1;
    const V4<R> *P = S.pos[C->pos_par];
    const int nx = S.nc[0], ny = S.nc[1], nz = S.nc[2];
    const int c = S.cell_sorted[ii];
    const int cxy = c % (nx * ny);
    const int cx = cxy % nx, cy = cxy / nx, cz = c / (nx * ny);
    const int cap = S.nl_cap;
    const V4<R> pi = P[ii];
    uint32_t *rowp = S.nl + (size_t)ii * cap;
    uint4 *row = reinterpret_cast<uint4 *>(rowp);
    uint32_t b0 = 0, b1 = 0, b2 = 0, b3 = 0;
    int nf = 0, nb = 0;
    // entries of the current chunk live in a 4-register shift queue and are
    // stored as one 16-byte chunk when four have been found
    auto accept = [&](int j, uint32_t code) {
        if (code == 0) {
            b3 = b2; b2 = b1; b1 = b0; b0 = (uint32_t)j;
            ++nf;
            if ((nf & 3) == 0 && nf + nb <= cap) row[(nf >> 2) - 1] = make_uint4(b0, b1, b2, b3);
        } else {
            // an image entry only has to stay inside the row: if the row's
            // final length fits, the back cannot meet the front; if not, the
            // row is discarded
            if (nb < cap) rowp[cap - 1 - nb] = (uint32_t)j | (code << JBITS);
            ++nb;
        }
    };
    for (int dz = N3L ? 0 : -RCH; dz <= RCH; ++dz) {
        int wz, sz;
        if (!stencil_cell(cz, dz, nz, S.walls[2], wz, sz)) continue;
        for (int dy = -RCH; dy <= RCH; ++dy) {
            // with N3L the half stencil: rows dz > 0, rows (dz = 0, dy > 0),
            // and in i's own row the cells cx (j > i only) to cx + RCH
            if (N3L && dz == 0 && dy < 0) continue;
            const bool own_row = dz == 0 && dy == 0;
            int wy, sy;
            if (!stencil_cell(cy, dy, ny, S.walls[1], wy, sy)) continue;
            int xa = cx - RCH, xb = cx + RCH;
            if (S.walls[0]) { xa = max(xa, 0); xb = min(xb, nx - 1); }
            if (N3L && own_row) xa = cx;
            const int rowc = (wz * ny + wy) * nx;
            // the run [xa, xb] in unwrapped cell coordinates: the part left of
            // the box (image -1), inside it (no image), right of it (image +1)
            for (int sx = -1; sx <= 1; ++sx) {
                const int a = sx < 0 ? xa : (sx == 0 ? max(xa, 0) : max(xa, nx));
                const int b = sx < 0 ? min(xb, -1) : (sx == 0 ? min(xb, nx - 1) : xb);
                if (a > b) continue;
                int jb = S.cell_start[rowc + a - sx * nx];
                const int je = S.cell_start[rowc + b - sx * nx + 1];
                if (N3L && own_row && sx == 0) jb = ii + 1;  // j > i in i's own cell, all j beyond it
                const uint32_t code = encode_image(sx, sy, sz);
                // does this run contain i itself without an image?
                const bool self = !N3L && code == 0 && jb <= ii && ii < je;
                const R xs = pi.x - (R)sx * S.box[0], ys = pi.y - (R)sy * S.box[1], zs = pi.z - (R)sz * S.box[2];
                for (int j0 = jb; j0 < je; j0 += 32) {
                    const int m = min(32, je - j0);
                    uint32_t mask = 0;
                    if constexpr (sizeof(R) == 4) {
                        // the sign bit of r^2 - r_list^2 (set when the
                        // candidate is inside) is shifted into the mask:
                        // candidate t lands at bit m - 1 - t, reversed below
                        const float nrl2 = -(float)S.rlist2;
                        auto below = [&](const V4<R> &q) {
                            const float ex = xs - q.x, ey = ys - q.y, ez = zs - q.z;
                            return __float_as_uint(fmaf(ez, ez, fmaf(ey, ey, fmaf(ex, ex, nrl2))));
                        };
                        int t = 0;
                        for (; t + 4 <= m; t += 4) {
                            const int j = j0 + t;
                            const V4<R> q0 = ldpos(P, j), q1 = ldpos(P, j + 1), q2 = ldpos(P, j + 2), q3 = ldpos(P, j + 3);
                            mask = __funnelshift_l(below(q0), mask, 1);
                            mask = __funnelshift_l(below(q1), mask, 1);
                            mask = __funnelshift_l(below(q2), mask, 1);
                            mask = __funnelshift_l(below(q3), mask, 1);
                        }
                        for (; t < m; ++t) mask = __funnelshift_l(below(ldpos(P, j0 + t)), mask, 1);
                        mask = __brev(mask) >> (32 - m);
                    } else {
                        for (int t = 0; t < m; ++t) {
                            const V4<R> q = ldpos(P, j0 + t);
                            mask |= (uint32_t)(r2_of(xs - q.x, ys - q.y, zs - q.z) < S.rlist2) << t;
                        }
                    }
                    if (self) {  // drop j == i
                        const int rel = ii - j0;
                        if (rel >= 0 && rel < 32) mask &= ~(1u << rel);
                    }
                    if (!act) mask = 0;
                    while (mask) {
                        const int bit = __ffs(mask) - 1;
                        mask &= mask - 1;
                        accept(j0 + bit, code);
                    }
                }
            }
        }
    }
    const int need = ((nf + 3) & ~3) + nb;
    if (act) {
        if (need > cap || nb > 0xffff || nf > 0xffff) {
            C->overflow = 1;
            S.nl_count[i] = 0;
        } else {
            if (nf & 3) {  // sentinel padding of the last chunk
                const uint32_t sent = (uint32_t)S.n;
                for (int k = nf & 3; k < 4; ++k) { b3 = b2; b2 = b1; b1 = b0; b0 = sent; }
                row[nf >> 2] = make_uint4(b0, b1, b2, b3);
            }
            S.nl_count[i] = nf | (nb << 16);
        }
    }
    block_need_max(C, act ? (unsigned)need : 0u);
    block_add_entries(C, (act && need <= cap) ? (unsigned)need : 0u);
}

// The same rows for small systems, one warp per sorted particle i: with
// one thread per particle a system of a few thousand particles fills one
// or two warps an SM, and each thread walks its ~10^3 candidates one load
// after another.  Here lane t tests candidates j0 + t and j0 + 32 + t of a
// run (both loads issued first), a ballot gives the warp the block's mask,
// and each accepted lane stores its own entry.  The k-th entry without an
// image goes where the per-thread build's shift queue puts it (position
// 3 - k mod 4 of chunk k / 4), the k-th image entry to slot cap - 1 - k, and
// the candidates are walked in the same order with the same test, so the
// two builds write identical rows.
template <typename R, bool N3L, int RCH>
__global__ void __launch_bounds__(VL_WBUILD_THREADS) k_vl_build_warp(Dev<R> S) {
    Ctrl *C = S.ctrl;
    if (!C->rebuild_now) return;
    const int lane = threadIdx.x & 31;
    const int i = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const bool act = i < S.n;  // uniform across the warp
    const int ii = act ? i : S.n - 1;
    const V4<R> *P = S.pos[C->pos_par];
    const int nx = S.nc[0], ny = S.nc[1], nz = S.nc[2];
    const int c = S.cell_sorted[ii];
    const int cxy = c % (nx * ny);
    const int cx = cxy % nx, cy = cxy / nx, cz = c / (nx * ny);
    const int cap = S.nl_cap;
    const V4<R> pi = P[ii];
    uint32_t *rowp = S.nl + (size_t)ii * cap;
    const uint32_t lt = (1u << lane) - 1u;
    int nf = 0, nb = 0;
    auto inside = [&](const V4<R> &q, R xs, R ys, R zs) -> bool {
        if constexpr (sizeof(R) == 4) {
            const float ex = xs - q.x, ey = ys - q.y, ez = zs - q.z;
            return (__float_as_uint(fmaf(ez, ez, fmaf(ey, ey, fmaf(ex, ex, -(float)S.rlist2)))) >> 31) != 0;
        } else {
            return r2_of(xs - q.x, ys - q.y, zs - q.z) < S.rlist2;
        }
    };
    auto take = [&](bool in, int j, uint32_t code) {
        const uint32_t mask = __ballot_sync(0xffffffffu, in);
        if (in) {
            const int k = __popc(mask & lt);
            if (code == 0) {
                const int e = nf + k, pos = (e & ~3) + 3 - (e & 3);
                if (pos < cap) rowp[pos] = (uint32_t)j;
            } else {
                const int e = nb + k;
                if (e < cap) rowp[cap - 1 - e] = (uint32_t)j | (code << JBITS);
            }
        }
        if (code == 0) nf += __popc(mask);
        else nb += __popc(mask);
    };
    for (int dz = N3L ? 0 : -RCH; dz <= RCH; ++dz) {
        int wz, sz;
        if (!stencil_cell(cz, dz, nz, S.walls[2], wz, sz)) continue;
        for (int dy = -RCH; dy <= RCH; ++dy) {
            if (N3L && dz == 0 && dy < 0) continue;
            const bool own_row = dz == 0 && dy == 0;
            int wy, sy;
            if (!stencil_cell(cy, dy, ny, S.walls[1], wy, sy)) continue;
            int xa = cx - RCH, xb = cx + RCH;
            if (S.walls[0]) { xa = max(xa, 0); xb = min(xb, nx - 1); }
            if (N3L && own_row) xa = cx;
            const int rowc = (wz * ny + wy) * nx;
            for (int sx = -1; sx <= 1; ++sx) {
                const int a = sx < 0 ? xa : (sx == 0 ? max(xa, 0) : max(xa, nx));
                const int b = sx < 0 ? min(xb, -1) : (sx == 0 ? min(xb, nx - 1) : xb);
                if (a > b) continue;
                int jb = S.cell_start[rowc + a - sx * nx];
                const int je = S.cell_start[rowc + b - sx * nx + 1];
                if (N3L && own_row && sx == 0) jb = ii + 1;
                const uint32_t code = encode_image(sx, sy, sz);
                const bool self = !N3L && code == 0 && jb <= ii && ii < je;
                const R xs = pi.x - (R)sx * S.box[0], ys = pi.y - (R)sy * S.box[1], zs = pi.z - (R)sz * S.box[2];
                for (int j0 = jb; j0 < je; j0 += 64) {
                    const int ja = j0 + lane, jc = j0 + 32 + lane;
                    const bool va = act && ja < je, vc = act && jc < je;
                    const V4<R> qa = ldpos(P, va ? ja : ii), qc = ldpos(P, vc ? jc : ii);
                    take(va && inside(qa, xs, ys, zs) && !(self && ja == ii), ja, code);
                    if (j0 + 32 < je) take(vc && inside(qc, xs, ys, zs) && !(self && jc == ii), jc, code);
                }
            }
        }
    }
    const int need = ((nf + 3) & ~3) + nb;
    if (act) {
        if (need > cap || nb > 0xffff || nf > 0xffff) {
            if (lane == 0) {
                C->overflow = 1;
                S.nl_count[i] = 0;
            }
        } else {
            const int r = nf & 3;
            if (r && lane >= r && lane < 4) rowp[(nf & ~3) + 3 - lane] = (uint32_t)S.n;  // sentinel padding
            if (lane == 0) S.nl_count[i] = nf | (nb << 16);
        }
    }
    block_need_max(C, act ? (unsigned)need : 0u);
    block_add_entries(C, (act && lane == 0 && need <= cap) ? (unsigned)need : 0u);
}

// Clusters: each cell's segment is cut into chunks of M consecutive sorted
// particles (the last may be shorter); one thread per cell writes its
// clusters' first particle, size and cell.
template <typename R>
__global__ void k_cluster_form(Dev<R> S) {
    Ctrl *C = S.ctrl;
    if (!C->rebuild_now) return;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= S.ncell) return;
    const int start = S.cell_start[c], m = S.cell_start[c + 1] - start;
    const int cl0 = S.clcell_start[c];
    for (int k = 0; k * S.M < m; ++k) {
        const int cl = cl0 + k;
        if (cl >= S.ncl_cap) { C->overflow = 1; return; }
        S.cl_first[cl] = start + k * S.M;
        S.cl_count[cl] = min(S.M, m - k * S.M);
        S.cl_cell[cl] = c;
    }
}

__global__ void k_rebuild_finish(Ctrl *C) {
    if (!C->rebuild_now) return;
    C->state_par ^= 1;
    C->steps_since = 0;
    C->rebuilds += 1;
    C->rebuild_now = 0;
}

}  // namespace

template <typename R> void launch_bin(const Dev<R> &S, cudaStream_t st) {
    int ntiles = div_up(S.ncell, SCAN_TILE);
    int n = S.n > ntiles ? S.n : ntiles;
    k_bin<R><<<div_up(n, 256), 256, 0, st>>>(S, ntiles);
}
template <typename R> void launch_scan(const Dev<R> &S, int M, cudaStream_t st) {
    int ntiles = div_up(S.ncell, SCAN_TILE);
    k_scan<R><<<ntiles, SCAN_THREADS, 0, st>>>(S, M < 1 ? 1 : M, ntiles);
}
template <typename R> void launch_scatter(const Dev<R> &S, cudaStream_t st) {
    k_scatter<R><<<div_up(S.n, 256), 256, 0, st>>>(S);
}
template <typename R> void launch_sortgather(const Dev<R> &S, cudaStream_t st) {
    k_sortgather<R><<<div_up(S.n, 256), 256, 0, st>>>(S);
}
template <typename R> void launch_vl_build(const Dev<R> &S, bool n3l, cudaStream_t st) {
    if (S.n <= (S.reach == 1 ? VL_WARP_BUILD_MAX_N : VL_WARP_BUILD_MAX_N_HALF_CELLS)) {
        const int wblocks = div_up(S.n, VL_WBUILD_THREADS / 32);
        if (S.reach == 1) {
            if (n3l) k_vl_build_warp<R, true, 1><<<wblocks, VL_WBUILD_THREADS, 0, st>>>(S);
            else k_vl_build_warp<R, false, 1><<<wblocks, VL_WBUILD_THREADS, 0, st>>>(S);
        } else {
            if (n3l) k_vl_build_warp<R, true, 2><<<wblocks, VL_WBUILD_THREADS, 0, st>>>(S);
            else k_vl_build_warp<R, false, 2><<<wblocks, VL_WBUILD_THREADS, 0, st>>>(S);
        }
        return;
    }
    const int blocks = div_up(S.n, VL_BUILD_THREADS);
    if (S.reach == 1) {
        if (n3l) k_vl_build<R, true, 1><<<blocks, VL_BUILD_THREADS, 0, st>>>(S);
        else k_vl_build<R, false, 1><<<blocks, VL_BUILD_THREADS, 0, st>>>(S);
    } else {
        if (n3l) k_vl_build<R, true, 2><<<blocks, VL_BUILD_THREADS, 0, st>>>(S);
        else k_vl_build<R, false, 2><<<blocks, VL_BUILD_THREADS, 0, st>>>(S);
    }
}
template <typename R> void launch_cluster_form(const Dev<R> &S, cudaStream_t st) {
    k_cluster_form<R><<<div_up(S.ncell, 128), 128, 0, st>>>(S);
}
void launch_rebuild_finish(Ctrl *C, cudaStream_t st) { k_rebuild_finish<<<1, 1, 0, st>>>(C); }

#define INST(R)                                                                 \
    template void launch_bin<R>(const Dev<R> &, cudaStream_t);                  \
    template void launch_scan<R>(const Dev<R> &, int, cudaStream_t);            \
    template void launch_scatter<R>(const Dev<R> &, cudaStream_t);              \
    template void launch_sortgather<R>(const Dev<R> &, cudaStream_t);           \
    template void launch_vl_build<R>(const Dev<R> &, bool, cudaStream_t);       \
    template void launch_cluster_form<R>(const Dev<R> &, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace ljsel
