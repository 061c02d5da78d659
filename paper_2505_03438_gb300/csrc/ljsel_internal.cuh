// ljsel_internal.cuh -- device data layout and per-pair arithmetic shared by
// the GPU kernels of the library (not by the CPU oracle, which is separate).
//
// Precision split: positions used by the pair arithmetic are a working copy
// (float4 in the FP32 path: x, y, z and the type's bit pattern; a 32-byte
// double quadruple in the FP64 check path); integration state (x, v) is FP64
// structure-of-arrays; energy and virial are summed in FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ljsel.h"

namespace ljsel {

constexpr int MAXT = LJSEL_MAX_TYPES;
constexpr int MAXT2 = MAXT * MAXT;

// A neighbour entry packs the j index (particle or cluster) into the low 27
// bits and an image code into the top 5.  Code 0 means "no periodic image";
// otherwise the code identifies s in {-1,0,1}^3 with x_j image = x_j + s*L.
constexpr uint32_t JBITS = 27;
constexpr uint32_t JMASK = (1u << JBITS) - 1u;

__host__ __device__ inline uint32_t encode_image(int sx, int sy, int sz) {
    int s = (sx + 1) + 3 * (sy + 1) + 9 * (sz + 1) + 14;  // 13 + 14 = 27 -> 0 = no image
    return (uint32_t)(s >= 27 ? s - 27 : s);
}

// Neighbour cell coordinate c + o (|o| <= 2) wrapped into [0, n) with the
// image coefficient s (x_j image = x_j + s L); returns false when the image
// lies two box lengths away (only when n = 1 and |o| = 2).
__host__ __device__ inline bool wrap_cell(int c, int o, int n, int &w, int &s) {
    w = c + o;
    s = 0;
    if (w < 0) { w += n; s = -1; }
    else if (w >= n) { w -= n; s = 1; }
    return w >= 0 && w < n;
}
// The same for a dimension that may be closed by walls: between walls there
// is no image, and a cell beyond the box does not exist (returns false).
__host__ __device__ inline bool stencil_cell(int c, int o, int n, int wall, int &w, int &s) {
    if (wall) {
        w = c + o;
        s = 0;
        return w >= 0 && w < n;
    }
    return wrap_cell(c, o, n, w, s);
}
__host__ __device__ inline void decode_image(uint32_t c, int &sx, int &sy, int &sz) {
    int s = ((int)c + 13) % 27;
    sx = s % 3 - 1;
    sy = (s / 3) % 3 - 1;
    sz = s / 9 - 1;
}

struct __align__(32) D4 {
    double x, y, z, w;
};

template <typename R> struct V4T;
template <> struct V4T<float> { using type = float4; };
template <> struct V4T<double> { using type = D4; };
template <typename R> using V4 = typename V4T<R>::type;

__device__ __forceinline__ int type_of(const float4 &p) { return __float_as_int(p.w); }
__device__ __forceinline__ int type_of(const D4 &p) { return (int)p.w; }
__device__ __forceinline__ float4 make_pos(float x, float y, float z, int t) { return make_float4(x, y, z, __int_as_float(t)); }
__device__ __forceinline__ D4 make_pos(double x, double y, double z, int t) { D4 r; r.x = x; r.y = y; r.z = z; r.w = (double)t; return r; }
__device__ __forceinline__ float4 ldpos(const float4 *p, int i) { return __ldg(p + i); }
__device__ __forceinline__ D4 ldpos(const D4 *p, int i) { return p[i]; }

// Per-type-pair constants in the working precision.  f/r = rinv2 * sr6 *
// (e48 sr6 - e24), U = e4 sr6 (sr6 - 1) - ushift.  The cutoff test uses the
// band [rc2lo, rc2hi] around rc2 to route borderline pairs to the exact FP64
// predicate against rc2d (= rc*rc in double).
template <typename R> struct PairTab {
    R sig2[MAXT2], e24[MAXT2], e48[MAXT2], e4[MAXT2], ushift[MAXT2];
    R rc2lo[MAXT2], rc2hi[MAXT2];
    double rc2d[MAXT2];
    R inv_sig[MAXT2];      // 1 / sigma (parameter derivatives)
    R a12[MAXT2], b6[MAXT2];  // 48 eps sigma^12, 24 eps sigma^6: f/r = s^4 (a12 s^3 - b6), s = 1 / r^2
    R inv_mass_dt[MAXT];   // dt / m per type
    double dt;
    double half_mass[MAXT];
    int ntypes;
};

// Device control block: flags, counters and FP64 sums, one per system.
struct Ctrl {
    int32_t rebuild_now;       // the rebuild kernels of this step run
    int32_t overflow;          // a list build ran out of capacity
    int32_t nonfinite;
    int32_t timeout;
    int32_t disp_exceeded;     // some particle moved >= skin/2 since the last rebuild
    int32_t steps_since;       // steps since the last rebuild
    int32_t pos_par;           // which working-position buffer is current
    int32_t state_par;         // which FP64 state buffer is current
    int32_t half_kick;         // next step kicks by dt/2 (velocities at integer time)
    int32_t rebuild_interval;
    int32_t loop_on;
    int32_t window_overflow;   // a cell's neighbourhood window exceeds its capacity
    int64_t steps_done;        // steps done by the current advance call
    int64_t steps_target;
    int64_t total_steps;
    int64_t rebuilds;
    int64_t early_rebuilds;
    int64_t need_cap;          // largest per-row list length required
    int64_t list_entries;      // entries kept by the last list build (all rows)
    unsigned long long npairs; // pair-export counter
    int32_t scan_ticket;
    int32_t rebuild_all;       // batches: the next rebuild covers every replica
    double epot, virial, ekin; // FP64 sums
    int64_t replica_rebuilds;  // batches: replica rebuilds summed over replicas
    int32_t check_failed;      // checked build: an index fell outside its array
    int32_t check_site;        // checked build: the first failing site (CHECK_* code)
    int32_t bad_type;          // an imported particle type lies outside [0, ntypes)
};

// Bounds checks of the checked build (compiled with -DLJSEL_CHECK): an index
// outside its array is recorded in Ctrl::check_failed, with the site's code
// in Ctrl::check_site, and the caller replaces it by a safe one, so the
// kernel never touches memory outside its buffers; the host then reports
// LJSEL_ERR_STATE.  In the normal build every check is true and compiles away.
enum {
    CHECK_VL_FRONT = 1, CHECK_VL_BACK = 2, CHECK_VL_ROW = 3, CHECK_LC_CELL = 4, CHECK_CL_ROW = 5,
    CHECK_CL_FRONT = 6, CHECK_CL_BACK = 7, CHECK_CL_MEMBERS = 8, CHECK_VLW_SLOT = 9, CHECK_BATCH_ENTRY = 10,
    CHECK_SORT_SLOT = 11, CHECK_BUILD_CELL = 12
};
#ifdef LJSEL_CHECK
__device__ __forceinline__ bool lj_check(bool ok, Ctrl *C, int site) {
    if (!ok) {
        atomicExch(&C->check_failed, 1);
        atomicCAS(&C->check_site, 0, site);
    }
    return ok;
}
#else
__device__ __forceinline__ bool lj_check(bool, Ctrl *, int) { return true; }
#endif

// Everything a kernel needs, passed by value.
template <typename R> struct Dev {
    using P4 = V4<R>;
    int n;
    int ncell;
    int nc[3];
    R inv_side[3];
    R box[3];
    R box_lo[3];          // FP32 path: box - (float)box, for exact image shifts
    double boxd[3];
    float box_dn[3];      // largest float <= L: 0 < (float)x < box_dn proves 0 < x < L
    int reach;            // stencil half-width in cells (1 for CSF 1, 2 for CSF 0.5)
    int walls[3];         // 1: dimension closed by reflective walls
    R rlist2;             // squared list radius (r_c,max + skin, slightly enlarged)
    R half_skin2;         // (skin/2)^2: displacement that forces a rebuild
    // FP64 state, double-buffered by Ctrl::state_par; SoA [3][n]
    double *x[2], *v[2];
    int *id[2];           // original input index
    int *type[2];
    // working positions, double-buffered by Ctrl::pos_par
    P4 *pos[2];
    P4 *xref;             // working positions at the last rebuild
    P4 *force;            // force buffer (N3L accumulation and compute())
    // cells
    int *cell_count;      // [ncell], zero between rebuilds
    int *cell_start;      // [ncell+1]
    int *clcell_start;    // [ncell+1] first cluster of each cell
    int *cell_of;         // [n] cell of particle (old order at binning)
    int *slot_of;         // [n]
    unsigned long long *key_of;  // [n]
    int *tmp_idx;         // [n]
    unsigned long long *tmp_key; // [n]
    int *cell_sorted;     // [n] cell of each sorted particle
    int *scan_partial;    // [nblocks] decoupled look-back state
    // Verlet lists, row-major: row i holds nl_cap entries at nl + i*nl_cap
    // (nl_cap a multiple of 4).  Entries without a periodic image fill the
    // row from the front, followed by entries naming the sentinel particle n
    // up to a multiple of 4, so they are read as 16-byte chunks without
    // bounds checks; entries with an image fill the row from the back.
    // nl_count[i] = front count | (back count << 16).  pos[.][n] is a
    // sentinel far outside the box.
    uint32_t *nl;
    uint16_t *nl16;       // window lists (same buffer as nl, 16-bit entries)
    int *nl_count;
    int nl_cap;
    // window strips: (row, x0, x1, -) per strip; *nstrips of them
    int4 *strips;
    int *nstrips;
    int strip_cap;
    // i-clusters and their lists
    int M;                // cluster size
    int ncl_cap;
    int *cl_first;        // [ncl] first sorted particle
    int *cl_count;        // [ncl]
    int *cl_cell;         // [ncl]
    uint32_t *cp;         // cluster lists, row c at cp + c * cp_cap
    int *cp_count;        // [ncl] front count | back count << 16
    int cp_cap;
    int *ncl_total;       // device scalar: clusters of the current build
    Ctrl *ctrl;
    PairTab<R> tab;
};

// Image-shifted displacement x_i - (x_j + s L) in the FP32 path.  Without an
// image it is one correctly rounded subtraction.  With an image, x_i - x_j is
// split exactly into hi + lo (Knuth's TwoSum), s*L_hi is removed from hi
// (exact by Sterbenz' lemma, since |x_i - x_j| is within [L/2, 2L] for any pair
// that can be in range), and lo - s*L_lo is added: the result carries about
// one rounding at the magnitude of the displacement, not of the box.
__device__ __forceinline__ float image_dx(float xi, float xj, int s, float L, float Llo) {
    float d = __fsub_rn(xi, xj);
    if (s == 0) return d;
    float bb = __fsub_rn(d, xi);
    float lo = __fadd_rn(__fsub_rn(xi, __fsub_rn(d, bb)), __fsub_rn(-xj, bb));
    float sL = s > 0 ? L : -L;
    float sLlo = s > 0 ? Llo : -Llo;
    float t = __fsub_rn(d, sL);
    return __fadd_rn(t, __fsub_rn(lo, sLlo));
}
// FP64 path: the defining arithmetic x_i - (x_j + s L).
__device__ __forceinline__ double image_dx(double xi, double xj, int s, double L, double) {
    return __dsub_rn(xi, __dadd_rn(xj, (double)s * L));
}

// The exact cutoff predicate on working positions promoted to double:
// dx = x_i - (x_j + s L), r^2 = (dx*dx + dy*dy) + dz*dz with every product
// and sum rounded separately, in range iff r^2 < r_c^2.  Out of line and
// taking the FP32 values, so that the common path never pays for it.
static __device__ __noinline__ bool exact_in_range(float fxi, float fyi, float fzi, float fxj, float fyj, float fzj,
                                                   int sx, int sy, int sz, const double *boxd, double rc2d) {
    const double xi = fxi, yi = fyi, zi = fzi, xj = fxj, yj = fyj, zj = fzj;
    double dx = __dsub_rn(xi, __dadd_rn(xj, (double)sx * boxd[0]));
    double dy = __dsub_rn(yi, __dadd_rn(yj, (double)sy * boxd[1]));
    double dz = __dsub_rn(zi, __dadd_rn(zj, (double)sz * boxd[2]));
    double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return r2 < rc2d;
}

// Bounded spin: poll *p until one of the mask bits is set, at most `limit`
// polls with a short sleep between them.  Returns the last value read; the
// caller checks the mask and reports a timeout (never traps).
__device__ __forceinline__ unsigned long long spin_until(const volatile unsigned long long *p, unsigned long long mask,
                                                         int limit) {
    unsigned long long v = 0;
    for (int it = 0; it <= limit; ++it) {
        v = *p;
        if (v & mask) break;
        __nanosleep(32);
    }
    return v;
}

__device__ __forceinline__ float fast_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double fast_rcp(double x) { return 1.0 / x; }

__device__ __forceinline__ float r2_of(float dx, float dy, float dz) { return fmaf(dz, dz, fmaf(dy, dy, dx * dx)); }
__device__ __forceinline__ double r2_of(double dx, double dy, double dz) {
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Largest required list length of a warp or a block, then one atomicMax on
// Ctrl::need_cap: same-address atomics serialise in L2, and one per particle
// (a million per build) cost about as much as the list build itself.
// Every lane of the warp (every thread of the block) must make the call.
__device__ __forceinline__ void warp_need_max(Ctrl *C, unsigned v) {
    const unsigned m = __reduce_max_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(reinterpret_cast<unsigned long long *>(&C->need_cap), (unsigned long long)m);
}
__device__ __forceinline__ void block_need_max(Ctrl *C, unsigned v) {
    __shared__ unsigned s_need;
    if (threadIdx.x == 0) s_need = 0u;
    __syncthreads();
    const unsigned m = __reduce_max_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&s_need, m);
    __syncthreads();
    if (threadIdx.x == 0 && s_need) atomicMax(reinterpret_cast<unsigned long long *>(&C->need_cap), (unsigned long long)s_need);
}

// Entries kept by a list build, summed per block, then one atomicAdd on
// Ctrl::list_entries.  Every thread of the block must make the call.
__device__ __forceinline__ void block_add_entries(Ctrl *C, unsigned v) {
    __shared__ unsigned long long s_sum;
    if (threadIdx.x == 0) s_sum = 0ull;
    __syncthreads();
    const unsigned w = __reduce_add_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(&s_sum, (unsigned long long)w);
    __syncthreads();
    if (threadIdx.x == 0 && s_sum) atomicAdd(reinterpret_cast<unsigned long long *>(&C->list_entries), s_sum);
}

// Decides "r < r_c" for one pair exactly as the FP64 predicate does: in the
// FP32 path outside a relative band of 2^-14 around r_c^2 the FP32 r^2
// (error < 1e-6 relative) decides; inside it, the FP64 predicate.  The FP64
// path evaluates r^2 with the defining arithmetic and decides directly.
template <typename R> struct Cut;
template <> struct Cut<float> {
    __device__ __forceinline__ static bool in(float r2, float lo, float hi, const float4 &pi, const float4 &pj,
                                              int sx, int sy, int sz, const double *boxd, double rc2d) {
        bool in = r2 < lo;
        if (!in && r2 <= hi) in = exact_in_range(pi.x, pi.y, pi.z, pj.x, pj.y, pj.z, sx, sy, sz, boxd, rc2d);
        return in;
    }
};
template <> struct Cut<double> {
    __device__ __forceinline__ static bool in(double r2, double, double, const D4 &, const D4 &, int, int, int,
                                              const double *, double rc2d) {
        return r2 < rc2d;
    }
};

// LJ 12-6 pair terms (Sec. 2.1): returns f/r; adds sr6*(sr6-1) to *u6 when
// the caller accumulates energy.
template <typename R>
__device__ __forceinline__ R lj_fr(R r2, R sig2, R e24, R e48, R &sr6_out) {
    R rinv2 = fast_rcp(r2);
    R sr2 = sig2 * rinv2;
    R sr6 = sr2 * sr2 * sr2;
    sr6_out = sr6;
    return (sr6 * rinv2) * (e48 * sr6 - e24);
}

inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace ljsel
