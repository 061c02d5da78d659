// window.cu -- Verlet lists over shared-memory neighbourhood windows (the
// GPU form of the Verlet-list container of Sec. 2.2.1).
//
// The cell grid (side >= r_c + skin) is cut, inside every (y, z) row of
// cells, into strips of consecutive cells holding at most STRIP_MAX
// particles.  One CTA owns one strip at a time and loads the strip's
// neighbourhood window into shared memory with coalesced loads: the 3 x 3
// adjacent rows, each over the strip's x-range widened by one cell, at most
// WIN_CAP particles.  A particle's 27 stencil cells are then 27 contiguous
// runs of window slots.  List entries are 16-bit window slots (11 bits) plus
// a 5-bit periodic-image code, so the list is half the size of a list of
// particle indices and every neighbour read is a shared-memory load.  Rows
// hold the entries without an image at the front, in 16-byte chunks of
// eight padded with the window's sentinel slot, and the entries with an
// image at the back.
#include "kernels.cuh"

namespace ljsel {

namespace {

constexpr int WIN_SLOTS = 2048;
constexpr int WIN_CAP = WIN_SLOTS - 1;  // slot WIN_CAP holds the far-away sentinel
constexpr int STRIP_MAX = 128;          // particles per strip (the CTA size)
constexpr int STRIP_MAX_CELLS = 62;
constexpr int WIN_CELLS = 9 * (STRIP_MAX_CELLS + 2);
constexpr int WTHREADS = 256;             // two lanes per strip particle

__device__ __forceinline__ int cell_count(const int *cs, int c) { return cs[c + 1] - cs[c]; }

// Number of particles in the window of strip [x0, x1) of row (cy, cz).
template <typename R>
__device__ int window_size_r(const Dev<R> &S, int cy, int cz, int x0, int x1) {
    int tot = 0;
    for (int dz = -1; dz <= 1; ++dz) {
        int wz, sz;
        wrap_cell(cz, dz, S.nc[2], wz, sz);
        for (int dy = -1; dy <= 1; ++dy) {
            int wy, sy;
            wrap_cell(cy, dy, S.nc[1], wy, sy);
            const int rowbase = (wz * S.nc[1] + wy) * S.nc[0];
            if (x0 >= 1 && x1 <= S.nc[0] - 1) {
                tot += S.cell_start[rowbase + x1 + 1] - S.cell_start[rowbase + x0 - 1];
            } else {
                for (int x = x0 - 1; x <= x1; ++x) {
                    int wx = x < 0 ? x + S.nc[0] : (x >= S.nc[0] ? x - S.nc[0] : x);
                    tot += cell_count(S.cell_start, rowbase + wx);
                }
            }
        }
    }
    return tot;
}

// One thread per (y, z) row: cut the row into strips greedily, widening a
// strip while it holds at most STRIP_MAX particles and its window at most
// WIN_CAP.  A single cell whose window is larger cannot be served: the
// window-overflow flag is raised and the configuration is reported as
// unsupported for this system.
template <typename R>
__global__ void k_strip_plan(Dev<R> S) {
    Ctrl *C = S.ctrl;
    if (!C->rebuild_now) return;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int nrow = S.nc[1] * S.nc[2];
    if (r >= nrow) return;
    const int cy = r % S.nc[1], cz = r / S.nc[1];
    const int nx = S.nc[0];
    const int rowbase = r * nx;
    int x0 = 0;
    while (x0 < nx) {
        int x1 = x0 + 1;
        while (x1 < nx && x1 - x0 < STRIP_MAX_CELLS) {
            const int np = S.cell_start[rowbase + x1 + 1] - S.cell_start[rowbase + x0];
            if (np > STRIP_MAX) break;
            if (window_size_r(S, cy, cz, x0, x1 + 1) > WIN_CAP) break;
            ++x1;
        }
        if (window_size_r(S, cy, cz, x0, x1) > WIN_CAP) C->window_overflow = 1;
        const int k = atomicAdd(S.nstrips, 1);
        if (k < S.strip_cap) S.strips[k] = make_int4(r, x0, x1, 0);
        x0 = x1;
    }
}

// Shared-memory layout of one window.
template <typename R, bool G, bool F> struct Win {
    V4<R> pos[WIN_SLOTS];
    int off[WIN_CELLS + 1];  // first slot of each window cell
    int code[WIN_CELLS];     // periodic-image code of each window cell
    int cstart[WIN_CELLS];   // first sorted particle of each window cell
    int gidx[G ? WIN_SLOTS : 1];
    V4<R> frc[F ? WIN_SLOTS : 1];
    unsigned long long mbar;  // completion barrier of the window's bulk copies
    int ncw, W, total, phase;
};

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

template <typename R, bool G, bool F>
__device__ void window_init(Win<R, G, F> &win) {
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&win.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        win.phase = 0;
    }
    __syncthreads();
}

// Bounded wait for the window's copies: returns false (and the caller raises
// the timeout flag) if the barrier phase did not complete.
__device__ __forceinline__ bool mbar_wait(unsigned long long *mbar, int parity) {
    const unsigned a = smem_addr(mbar);
    for (int it = 0; it < (1 << 20); ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Load the window of strip (row, x0, x1) into shared memory (whole block).
// Window cell k = p * (W + 2) + w covers row part p = (dz + 1) * 3 + (dy + 1)
// and column x0 - 1 + w.  Each row part is at most three runs of consecutive
// sorted particles (the two edge cells may be periodic images); threads
// 0..8 issue one asynchronous bulk copy per run into the window, all
// completing on the window's barrier.  Returns false on a wait timeout.
template <typename R, bool G, bool F>
__device__ bool load_window(const Dev<R> &S, Win<R, G, F> &win, int row, int x0, int x1, const V4<R> *P) {
    const int nx = S.nc[0], ny = S.nc[1], nz = S.nc[2];
    const int cy = row % ny, cz = row / ny;
    const int W = x1 - x0, ncw = 9 * (W + 2);
    __shared__ int s_part[WTHREADS];
    // per-window-cell metadata; thread t takes cells t*per .. t*per+per-1
    const int per = (ncw + WTHREADS - 1) / WTHREADS;
    int mysum = 0;
    int cnts[5];
    for (int q = 0; q < per && q < 5; ++q) {
        const int k = threadIdx.x * per + q;
        cnts[q] = 0;
        if (k < ncw) {
            const int p = k / (W + 2), w = k - p * (W + 2);
            const int dz = p / 3 - 1, dy = p % 3 - 1;
            int wz, sz, wy, sy, wx, sx;
            wrap_cell(cz, dz, nz, wz, sz);
            wrap_cell(cy, dy, ny, wy, sy);
            wrap_cell(x0 - 1, w, nx, wx, sx);
            const int c = (wz * ny + wy) * nx + wx;
            win.code[k] = (int)encode_image(sx, sy, sz);
            win.cstart[k] = S.cell_start[c];
            cnts[q] = S.cell_start[c + 1] - S.cell_start[c];
            mysum += cnts[q];
        }
    }
    s_part[threadIdx.x] = mysum;
    __syncthreads();
    // exclusive scan of the per-thread sums (one warp, WTHREADS / 32 each)
    constexpr int PW = WTHREADS / 32;
    if (threadIdx.x < 32) {
        int v[PW], run = 0;
        for (int q = 0; q < PW; ++q) { v[q] = s_part[threadIdx.x * PW + q]; run += v[q]; }
        int incl = run;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, incl, o);
            if ((threadIdx.x & 31) >= o) incl += t;
        }
        int ex = incl - run;
        for (int q = 0; q < PW; ++q) { s_part[threadIdx.x * PW + q] = ex; ex += v[q]; }
        if (threadIdx.x == 31) { win.total = min(incl, WIN_CAP); win.ncw = ncw; win.W = W; }
    }
    __syncthreads();
    {
        int o = s_part[threadIdx.x];
        for (int q = 0; q < per && q < 5; ++q) {
            const int k = threadIdx.x * per + q;
            if (k < ncw) { win.off[k] = o; o += cnts[q]; }
        }
    }
    if (threadIdx.x == 0) {
        win.off[ncw] = win.total;
        // one arrival that expects every byte of the window
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&win.mbar)),
                     "r"((unsigned)(win.total * sizeof(V4<R>)))
                     : "memory");
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        // runs of row part p: [left edge cell][middle cells][right edge cell],
        // merged when consecutive in sorted order
        const int p = threadIdx.x, k0 = p * (W + 2), k1 = k0 + W + 1;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        int k = k0;
        while (k <= k1) {
            int kend = k;
            while (kend < k1 && win.cstart[kend + 1] == win.cstart[kend] + (win.off[kend + 1] - win.off[kend]) &&
                   win.code[kend + 1] == win.code[kend])
                ++kend;
            const int slot = win.off[k];
            const int len = min(win.off[kend + 1], WIN_CAP) - slot;
            if (len > 0) {
                const unsigned bytes = (unsigned)(len * sizeof(V4<R>));
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        smem_addr(&win.pos[slot])),
                    "l"(P + win.cstart[k]), "r"(bytes), "r"(smem_addr(&win.mbar))
                    : "memory");
            }
            k = kend + 1;
        }
    }
    if (G || F) {
        for (int k = threadIdx.x >> 5; k < ncw; k += WTHREADS / 32) {
            const int o = win.off[k], m = min(win.off[k + 1], WIN_CAP) - o, c0 = win.cstart[k];
            for (int t = threadIdx.x & 31; t < m; t += 32) {
                if (G) win.gidx[o + t] = c0 + t;
                if (F) win.frc[o + t] = make_pos((R)0, (R)0, (R)0, 0);
            }
        }
    }
    if (threadIdx.x == 0) {
        win.pos[WIN_CAP] = make_pos((R)1e18, (R)1e18, (R)1e18, 0);
        if (G) win.gidx[WIN_CAP] = -1;
        if (F) win.frc[WIN_CAP] = make_pos((R)0, (R)0, (R)0, 0);
    }
    // one decision for the whole block, so that a timeout ends every thread
    const bool ok = __syncthreads_and(mbar_wait(&win.mbar, win.phase)) != 0;
    if (threadIdx.x == 0) win.phase ^= 1;
    return ok;
}

// 128-bit shift register of eight 16-bit entries.
struct Pack8 {
    uint32_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;
    __device__ __forceinline__ void push(uint32_t e) {
        w3 = __funnelshift_l(w2, w3, 16);
        w2 = __funnelshift_l(w1, w2, 16);
        w1 = __funnelshift_l(w0, w1, 16);
        w0 = (w0 << 16) | (e & 0xffffu);
    }
};

// List build: two lanes per strip particle; the candidates of its 27
// stencil cells are 27 contiguous slot runs of the window, lane 0 takes
// stencil cells 0..13 and lane 1 cells 14..26, each filling its own half of
// the particle's row.  As in the particle-index lists, i is shifted once per
// image cell in plain arithmetic (the list radius carries a 2^-12 relative
// margin).  With N3L only j > i (sorted index).  Counts: one byte per
// segment, nl_count = nf0 | nb0 << 8 | nf1 << 16 | nb1 << 24.
template <typename R, bool N3L>
__global__ void __launch_bounds__(WTHREADS) k_vlw_build(Dev<R> S) {
    Ctrl *C = S.ctrl;
    if (!C->rebuild_now || C->window_overflow) return;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Win<R, false, false> &win = *reinterpret_cast<Win<R, false, false> *>(smem_raw);
    window_init(win);
    const V4<R> *P = S.pos[C->pos_par];
    const int nst = min(*S.nstrips, S.strip_cap);
    const int cap = S.nl_cap, hcap = cap >> 1;
    const int sub = threadIdx.x & 1;
    const unsigned pairmask = 3u << ((threadIdx.x & 31) & ~1);
    unsigned my_need = 0;  // longest row this thread built
    for (int sidx = blockIdx.x; sidx < nst; sidx += gridDim.x) {
        const int4 st = S.strips[sidx];
        __syncthreads();
        if (!load_window<R, false, false>(S, win, st.x, st.y, st.z, P)) { C->timeout = 1; return; }
        const int W = win.W;
        const int rowbase = st.x * S.nc[0];
        const int first = S.cell_start[rowbase + st.y], last = S.cell_start[rowbase + st.z];
        for (int i = first + (threadIdx.x >> 1); i < last; i += WTHREADS / 2) {
            const V4<R> pi = P[i];
            const int ci = S.cell_sorted[i];
            const int wi = ci - rowbase - st.y + 1;  // window column of i's cell
            const int kown = 4 * (W + 2) + wi;
            const int own = win.off[kown] + (i - win.cstart[kown]);
            uint16_t *half16 = S.nl16 + (size_t)i * cap + sub * hcap;
            uint4 *half = reinterpret_cast<uint4 *>(half16);
            Pack8 pk;
            int nf = 0, nb = 0;
            auto accept = [&](int slot, int code) {
                if (code == 0) {
                    pk.push((uint32_t)slot);
                    ++nf;
                    if ((nf & 7) == 0 && nf + nb <= hcap) half[(nf >> 3) - 1] = make_uint4(pk.w0, pk.w1, pk.w2, pk.w3);
                } else {
                    // inside the half row: if its final length fits, the back
                    // cannot meet the front; if not, the row is discarded
                    if (nb < hcap) half16[hcap - 1 - nb] = (uint16_t)(slot | (code << 11));
                    ++nb;
                }
            };
            // candidates in slots [a, b) of one window cell (shifted i: xs, ys, zs)
            auto scan = [&](int a, int b, int code, R xs, R ys, R zs) {
                int slot = a;
                for (; slot + 4 <= b; slot += 4) {
                    const V4<R> q0 = win.pos[slot], q1 = win.pos[slot + 1], q2 = win.pos[slot + 2], q3 = win.pos[slot + 3];
                    const bool t0 = r2_of(xs - q0.x, ys - q0.y, zs - q0.z) < S.rlist2;
                    const bool t1 = r2_of(xs - q1.x, ys - q1.y, zs - q1.z) < S.rlist2;
                    const bool t2 = r2_of(xs - q2.x, ys - q2.y, zs - q2.z) < S.rlist2;
                    const bool t3 = r2_of(xs - q3.x, ys - q3.y, zs - q3.z) < S.rlist2;
                    if (t0 | t1 | t2 | t3) {
                        if (t0) accept(slot, code);
                        if (t1) accept(slot + 1, code);
                        if (t2) accept(slot + 2, code);
                        if (t3) accept(slot + 3, code);
                    }
                }
                for (; slot < b; ++slot) {
                    const V4<R> q = win.pos[slot];
                    if (r2_of(xs - q.x, ys - q.y, zs - q.z) < S.rlist2) accept(slot, code);
                }
            };
            const int c0 = sub ? 14 : 0, c1 = sub ? 27 : 14;
            for (int cc = c0; cc < c1; ++cc) {
                const int p = cc / 3, w = wi - 1 + cc % 3;
                const int k = p * (W + 2) + w;
                const int code = win.code[k];
                int o0 = win.off[k];
                const int o1 = min(win.off[k + 1], WIN_CAP);
                if (N3L) {
                    // a cell other than i's own holds only j < i or only j > i
                    const int cs = win.cstart[k];
                    if (k == kown) o0 = own + 1;
                    else if (cs + (o1 - o0) <= i) continue;
                    else if (cs <= i) o0 += i + 1 - cs;  // i's own cell seen as a periodic image
                }
                int sx, sy, sz;
                decode_image((uint32_t)code, sx, sy, sz);
                const R xs = pi.x - (R)sx * S.box[0], ys = pi.y - (R)sy * S.box[1], zs = pi.z - (R)sz * S.box[2];
                if (!N3L && k == kown) {
                    scan(o0, own, code, xs, ys, zs);
                    scan(own + 1, o1, code, xs, ys, zs);
                } else {
                    scan(o0, o1, code, xs, ys, zs);
                }
            }
            const int need = ((nf + 7) & ~7) + nb;
            const bool bad = need > hcap || nf > 255 || nb > 255;
            if (!bad && (nf & 7)) {
                for (int m = nf & 7; m < 8; ++m) pk.push((uint32_t)WIN_CAP);
                half[nf >> 3] = make_uint4(pk.w0, pk.w1, pk.w2, pk.w3);
            }
            const unsigned mine = bad ? 0u : (unsigned)(nf | (nb << 8));
            const unsigned other = __shfl_xor_sync(pairmask, mine, 1);
            const int obad = __shfl_xor_sync(pairmask, (int)bad, 1);
            if (sub == 0) S.nl_count[i] = (bad || obad) ? 0 : (int)(mine | (other << 16));
            if (bad) C->overflow = 1;
            my_need = max(my_need, (unsigned)(2 * need));
        }
    }
    warp_need_max(C, my_need);
}

template <typename R> struct WTab {
    R sig2[MAXT2], e24[MAXT2], e48[MAXT2], e4[MAXT2], ushift[MAXT2], lo[MAXT2], hi[MAXT2];
    double rc2d[MAXT2];
};

__device__ __forceinline__ void sadd3(float4 &p, float x, float y, float z) {
    atomicAdd(&p.x, x); atomicAdd(&p.y, y); atomicAdd(&p.z, z);
}
__device__ __forceinline__ void sadd3(D4 &p, double x, double y, double z) {
    atomicAdd(&p.x, x); atomicAdd(&p.y, y); atomicAdd(&p.z, z);
}
__device__ __forceinline__ void gadd4(float4 *F, int j, const float4 &v) { atomicAdd(F + j, v); }
__device__ __forceinline__ void gadd4(D4 *F, int j, const D4 &v) {
    atomicAdd(&F[j].x, v.x); atomicAdd(&F[j].y, v.y); atomicAdd(&F[j].z, v.z);
}

template <typename R, bool MT, bool EV> struct WAcc {
    R fx = 0, fy = 0, fz = 0, u = 0, w = 0;
    int np = 0;
};

// Force over window lists: thread per strip particle.  N3L off: fused
// Stormer-Verlet update (MODE_STEP) or forces to the buffer (MODE_FORCE).
// N3L on: -F_ij accumulates in the window's shared force slots and every
// slot is added to global memory once per strip.
template <typename R, bool N3L, int MODE, bool EV, bool MT>
__global__ void __launch_bounds__(WTHREADS) k_vlw(Dev<R> S, int2 *pairs, long long pcap) {
    Ctrl *C = S.ctrl;
    if (C->overflow || C->window_overflow) return;
    constexpr bool G = N3L || MODE == MODE_PAIRS;
    constexpr bool F = N3L && MODE != MODE_PAIRS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Win<R, G, F> &win = *reinterpret_cast<Win<R, G, F> *>(smem_raw);
    window_init(win);
    __shared__ WTab<R> T;
    if (MT) {
        for (int k = threadIdx.x; k < MAXT2; k += blockDim.x) {
            T.sig2[k] = S.tab.sig2[k]; T.e24[k] = S.tab.e24[k]; T.e48[k] = S.tab.e48[k]; T.e4[k] = S.tab.e4[k];
            T.ushift[k] = S.tab.ushift[k]; T.lo[k] = S.tab.rc2lo[k]; T.hi[k] = S.tab.rc2hi[k]; T.rc2d[k] = S.tab.rc2d[k];
        }
    }
    const int pp = C->pos_par, sp = C->state_par;
    const V4<R> *P = S.pos[pp];
    const int nst = min(*S.nstrips, S.strip_cap);
    const int cap = S.nl_cap, hcap = cap >> 1;
    const int sub = threadIdx.x & 1;
    const unsigned pairmask = 3u << ((threadIdx.x & 31) & ~1);
    const int half = C->half_kick;
    R eacc = 0, wacc = 0;
    double ke = 0;
    bool exceeded = false, bad = false;
    for (int sidx = blockIdx.x; sidx < nst; sidx += gridDim.x) {
        const int4 st = S.strips[sidx];
        __syncthreads();
        if (!load_window<R, G, F>(S, win, st.x, st.y, st.z, P)) { C->timeout = 1; return; }
        const int rowbase = st.x * S.nc[0];
        const int first = S.cell_start[rowbase + st.y], last = S.cell_start[rowbase + st.z];
        for (int i = first + (threadIdx.x >> 1); i < last; i += WTHREADS / 2) {
            const V4<R> pi = P[i];
            const int ti = type_of(pi);
            const unsigned cnt = (unsigned)S.nl_count[i] >> (16 * sub);
            const int nq = ((int)(cnt & 0xffu) + 7) >> 3, nb = (int)((cnt >> 8) & 0xffu);
            const uint16_t *half16 = S.nl16 + (size_t)i * cap + sub * hcap;
            const uint4 *row = reinterpret_cast<const uint4 *>(half16);
            WAcc<R, MT, EV> a;
            auto pair = [&](int slot, int sx, int sy, int sz, R dx, R dy, R dz, const V4<R> &pj) {
                const R r2 = r2_of(dx, dy, dz);
                R sig2, e24, e48, lo, hi;
                double rc2d;
                int tp = 0;
                if (MT) {
                    tp = ti * S.tab.ntypes + type_of(pj);
                    sig2 = T.sig2[tp]; e24 = T.e24[tp]; e48 = T.e48[tp]; lo = T.lo[tp]; hi = T.hi[tp]; rc2d = T.rc2d[tp];
                } else {
                    sig2 = S.tab.sig2[0]; e24 = S.tab.e24[0]; e48 = S.tab.e48[0]; lo = S.tab.rc2lo[0];
                    hi = S.tab.rc2hi[0]; rc2d = S.tab.rc2d[0];
                }
                const bool in = Cut<R>::in(r2, lo, hi, pi, pj, sx, sy, sz, S.boxd, rc2d);
                if (MODE == MODE_PAIRS) {
                    if (in) {
                        const int j = win.gidx[slot];
                        const int ia = S.id[sp][i], jb = S.id[sp][j];
                        if (N3L || ia < jb) {
                            unsigned long long k = atomicAdd(&C->npairs, 1ull);
                            if ((long long)k < pcap) pairs[k] = make_int2(min(ia, jb), max(ia, jb));
                        }
                    }
                    return;
                }
                R sr6;
                R fr = lj_fr(r2, sig2, e24, e48, sr6);
                fr = in ? fr : (R)0;
                if (EV) {
                    if (MT) a.u += in ? T.e4[tp] * sr6 * (sr6 - (R)1) - T.ushift[tp] : (R)0;
                    else { a.u += in ? sr6 * (sr6 - (R)1) : (R)0; a.np += in ? 1 : 0; }
                    a.w += fr * r2;
                }
                a.fx += fr * dx; a.fy += fr * dy; a.fz += fr * dz;
                if (F && in) sadd3(win.frc[slot], -fr * dx, -fr * dy, -fr * dz);
            };
            uint4 e = nq > 0 ? row[0] : make_uint4(0, 0, 0, 0);
            for (int q = 0; q < nq; ++q) {
                const uint4 en = q + 1 < nq ? row[q + 1] : e;
                const uint32_t wv[4] = {e.x, e.y, e.z, e.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    int s0 = (int)(wv[h] & 0xffffu), s1 = (int)(wv[h] >> 16);
                    if (!lj_check(s0 < WIN_SLOTS && s1 < WIN_SLOTS, C, CHECK_VLW_SLOT)) { s0 = WIN_CAP; s1 = WIN_CAP; }
                    const V4<R> q0 = win.pos[s0], q1 = win.pos[s1];
                    pair(s0, 0, 0, 0, pi.x - q0.x, pi.y - q0.y, pi.z - q0.z, q0);
                    pair(s1, 0, 0, 0, pi.x - q1.x, pi.y - q1.y, pi.z - q1.z, q1);
                }
                e = en;
            }
            for (int k = 0; k < nb; ++k) {
                const uint32_t ent = half16[hcap - 1 - k];
                const int slot = (int)(ent & 0x7ffu);
                int sx, sy, sz;
                decode_image(ent >> 11, sx, sy, sz);
                const V4<R> pj = win.pos[slot];
                pair(slot, sx, sy, sz, image_dx(pi.x, pj.x, sx, S.box[0], S.box_lo[0]),
                     image_dx(pi.y, pj.y, sy, S.box[1], S.box_lo[1]), image_dx(pi.z, pj.z, sz, S.box[2], S.box_lo[2]),
                     pj);
            }
            a.fx += __shfl_xor_sync(pairmask, a.fx, 1);
            a.fy += __shfl_xor_sync(pairmask, a.fy, 1);
            a.fz += __shfl_xor_sync(pairmask, a.fz, 1);
            if (MODE == MODE_PAIRS) continue;
            if (EV) {
                eacc += MT ? a.u : S.tab.e4[0] * a.u - S.tab.ushift[0] * (R)a.np;
                wacc += a.w;
            }
            if (sub != 0) continue;
            if (F) {
                const int own = win.off[4 * (win.W + 2) + (S.cell_sorted[i] - rowbase - st.y + 1)] +
                                (i - S.cell_start[S.cell_sorted[i]]);
                sadd3(win.frc[own], a.fx, a.fy, a.fz);
            } else if (MODE == MODE_FORCE) {
                S.force[i] = make_pos(a.fx, a.fy, a.fz, 0);
            } else {
                // Stormer-Verlet update (leapfrog form), as in the other list kernels
                const int n = S.n;
                double *X = S.x[sp];
                double *V = S.v[sp];
                R c = S.tab.inv_mass_dt[ti];
                if (half) c *= (R)0.5;
                double vx = V[i], vy = V[n + i], vz = V[2 * n + i];
                if (EV) {
                    double h = half ? 0.0 : 0.5;
                    double ux = vx + h * (double)(S.tab.inv_mass_dt[ti] * a.fx);
                    double uy = vy + h * (double)(S.tab.inv_mass_dt[ti] * a.fy);
                    double uz = vz + h * (double)(S.tab.inv_mass_dt[ti] * a.fz);
                    ke += S.tab.half_mass[ti] * (ux * ux + uy * uy + uz * uz);
                }
                vx += (double)(c * a.fx); vy += (double)(c * a.fy); vz += (double)(c * a.fz);
                const double dt = S.tab.dt;
                const double x = fma(dt, vx, X[i]), y = fma(dt, vy, X[n + i]), z = fma(dt, vz, X[2 * n + i]);
                V[i] = vx; V[n + i] = vy; V[2 * n + i] = vz;
                X[i] = x; X[n + i] = y; X[2 * n + i] = z;
                const V4<R> wp = make_pos((R)x, (R)y, (R)z, ti);
                S.pos[pp ^ 1][i] = wp;
                const V4<R> rf = S.xref[i];
                const R ddx = wp.x - rf.x, ddy = wp.y - rf.y, ddz = wp.z - rf.z;
                exceeded = exceeded || !(ddx * ddx + ddy * ddy + ddz * ddz < S.half_skin2);
                bad = bad || !isfinite(a.fx + a.fy + a.fz);
            }
        }
        if (F) {
            __syncthreads();
            const int tot = min(win.total, WIN_CAP);
            for (int slot = threadIdx.x; slot < tot; slot += blockDim.x) {
                const V4<R> f = win.frc[slot];
                if (f.x != (R)0 || f.y != (R)0 || f.z != (R)0) gadd4(S.force, win.gidx[slot], f);
            }
        }
    }
    if (MODE == MODE_PAIRS) return;
    if (MODE == MODE_STEP) {
        if (__any_sync(0xffffffffu, exceeded) && (threadIdx.x & 31) == 0) C->disp_exceeded = 1;
        if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) C->nonfinite = 1;
    }
    if (EV) {
        __shared__ double s_red[3][WTHREADS / 32];
        const R scale = N3L ? (R)1 : (R)0.5;
        double x = (double)(scale * eacc), y = (double)(scale * wacc), z = ke;
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_down_sync(0xffffffffu, x, o);
            y += __shfl_down_sync(0xffffffffu, y, o);
            z += __shfl_down_sync(0xffffffffu, z, o);
        }
        __syncthreads();
        if ((threadIdx.x & 31) == 0) { s_red[0][threadIdx.x >> 5] = x; s_red[1][threadIdx.x >> 5] = y; s_red[2][threadIdx.x >> 5] = z; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0, b = 0, c = 0;
            for (int k = 0; k < WTHREADS / 32; ++k) { a += s_red[0][k]; b += s_red[1][k]; c += s_red[2][k]; }
            if (a != 0.0) atomicAdd(&C->epot, a);
            if (b != 0.0) atomicAdd(&C->virial, b);
            if (c != 0.0) atomicAdd(&C->ekin, c);
        }
    }
}

int g_sm_count = 0;
int sm_count() {
    if (!g_sm_count) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (g_sm_count <= 0) g_sm_count = 1;
    }
    return g_sm_count;
}

template <typename K> void allow_smem(K kern, size_t bytes) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename R, bool N3L, int MODE, bool EV, bool MT>
void vlw_go(const Dev<R> &S, int2 *pairs, long long pcap, cudaStream_t st) {
    constexpr bool G = N3L || MODE == MODE_PAIRS;
    constexpr bool F = N3L && MODE != MODE_PAIRS;
    const size_t smem = sizeof(Win<R, G, F>);
    const int blocks = sm_count() * (smem > 100000 ? 1 : (smem > 60000 ? 2 : 4));  // 8 warps per CTA
    k_vlw<R, N3L, MODE, EV, MT><<<blocks, WTHREADS, smem, st>>>(S, pairs, pcap);
}

template <typename R, bool MT>
void vlw_dispatch(const Dev<R> &S, const ljsel_config &cfg, int mode, bool ev, int2 *pairs, long long pcap,
                  cudaStream_t st) {
    const bool n3l = cfg.newton3 != 0;
    if (mode == MODE_PAIRS) { n3l ? vlw_go<R, true, MODE_PAIRS, false, MT>(S, pairs, pcap, st) : vlw_go<R, false, MODE_PAIRS, false, MT>(S, pairs, pcap, st); return; }
    if (n3l) { ev ? vlw_go<R, true, MODE_FORCE, true, MT>(S, pairs, pcap, st) : vlw_go<R, true, MODE_FORCE, false, MT>(S, pairs, pcap, st); return; }
    if (mode == MODE_STEP) { ev ? vlw_go<R, false, MODE_STEP, true, MT>(S, pairs, pcap, st) : vlw_go<R, false, MODE_STEP, false, MT>(S, pairs, pcap, st); return; }
    ev ? vlw_go<R, false, MODE_FORCE, true, MT>(S, pairs, pcap, st) : vlw_go<R, false, MODE_FORCE, false, MT>(S, pairs, pcap, st);
}

template <typename R, bool MT> void vlw_prepare_t() {
    allow_smem(k_vlw<R, false, MODE_STEP, false, MT>, sizeof(Win<R, false, false>));
    allow_smem(k_vlw<R, false, MODE_STEP, true, MT>, sizeof(Win<R, false, false>));
    allow_smem(k_vlw<R, false, MODE_FORCE, false, MT>, sizeof(Win<R, false, false>));
    allow_smem(k_vlw<R, false, MODE_FORCE, true, MT>, sizeof(Win<R, false, false>));
    allow_smem(k_vlw<R, true, MODE_FORCE, false, MT>, sizeof(Win<R, true, true>));
    allow_smem(k_vlw<R, true, MODE_FORCE, true, MT>, sizeof(Win<R, true, true>));
    allow_smem(k_vlw<R, false, MODE_PAIRS, false, MT>, sizeof(Win<R, true, false>));
    allow_smem(k_vlw<R, true, MODE_PAIRS, false, MT>, sizeof(Win<R, true, false>));
}

}  // namespace

// Raise the dynamic shared-memory limit of every window kernel (outside any
// stream capture, before the first launch).
void vlw_prepare() {
    static bool done = false;
    if (done) return;
    vlw_prepare_t<float, false>();
    vlw_prepare_t<float, true>();
    vlw_prepare_t<double, true>();
    allow_smem(k_vlw_build<float, false>, sizeof(Win<float, false, false>));
    allow_smem(k_vlw_build<float, true>, sizeof(Win<float, true, false>));
    allow_smem(k_vlw_build<double, false>, sizeof(Win<double, false, false>));
    allow_smem(k_vlw_build<double, true>, sizeof(Win<double, true, false>));
    done = true;
}

template <typename R> void launch_strip_plan(const Dev<R> &S, cudaStream_t st) {
    const int nrow = S.nc[1] * S.nc[2];
    k_strip_plan<R><<<div_up(nrow, 128), 128, 0, st>>>(S);
}

template <typename R> void launch_vlw_build(const Dev<R> &S, bool n3l, cudaStream_t st) {
    const int blocks = sm_count() * 4;
    if (n3l) k_vlw_build<R, true><<<blocks, WTHREADS, sizeof(Win<R, true, false>), st>>>(S);
    else k_vlw_build<R, false><<<blocks, WTHREADS, sizeof(Win<R, false, false>), st>>>(S);
}

template <typename R> void launch_vlw_force(const Dev<R> &S, const ljsel_config &cfg, int mode, bool ev, int2 *pairs,
                                            long long pcap, cudaStream_t st);
template <> void launch_vlw_force<float>(const Dev<float> &S, const ljsel_config &cfg, int mode, bool ev, int2 *pairs,
                                         long long pcap, cudaStream_t st) {
    if (S.tab.ntypes > 1) vlw_dispatch<float, true>(S, cfg, mode, ev, pairs, pcap, st);
    else vlw_dispatch<float, false>(S, cfg, mode, ev, pairs, pcap, st);
}
template <> void launch_vlw_force<double>(const Dev<double> &S, const ljsel_config &cfg, int mode, bool ev,
                                          int2 *pairs, long long pcap, cudaStream_t st) {
    vlw_dispatch<double, true>(S, cfg, mode, ev, pairs, pcap, st);
}

template void launch_strip_plan<float>(const Dev<float> &, cudaStream_t);
template void launch_strip_plan<double>(const Dev<double> &, cudaStream_t);
template void launch_vlw_build<float>(const Dev<float> &, bool, cudaStream_t);
template void launch_vlw_build<double>(const Dev<double> &, bool, cudaStream_t);

}  // namespace ljsel
