// noalloc.cu -- a one-shot force evaluation that allocates no memory.
//
// Some callers cannot call cudaMalloc: code inside a framework whose own
// allocator has reserved all device memory and forbids allocations behind
// its back, plug-ins that run inside a host application that owns the
// device, and latency-critical loops that must not take the allocator's
// locks or trigger the implicit synchronization a cudaFree implies.  For
// them, ljsel_compute_forces_noalloc bins the particles into linked cells
// and evaluates the same FP32 LJ pair arithmetic as the library's
// linked-cell kernel, with every intermediate array held in one file-scope
// device array of fixed size (below).  The caller still owns and passes the
// input and output buffers.
//
// The scratch array is static device memory of this shared library: every
// GPU that loads the library holds it until the process exits.  All calls
// share it and it keeps the contents of the last call; each call clears
// what must start at zero (cell counts, the energy sums).  Calls whose work
// overlaps on the GPU (concurrent streams, or several host threads) race
// on the array and give wrong results: serialize them.
#include <mutex>
#include <string>

#include "kernels.cuh"
#include "system.h"

namespace ljsel {
namespace {

constexpr int NA_MAX_N = 1 << 17;      // particles
constexpr int NA_MAX_CELLS = 1 << 17;  // linked cells
constexpr int NA_THREADS = 128;
constexpr int NA_SCAN_THREADS = 1024;

struct NaScratch {
    int cell_count[NA_MAX_CELLS];
    int cell_start[NA_MAX_CELLS + 1];
    int cell_of[NA_MAX_N];
    int slot_of[NA_MAX_N];
    int cell_sorted[NA_MAX_N];
    int id[NA_MAX_N];
    float4 pos[NA_MAX_N];
    double sums[2];  // energy, virial
};

// 5.8 MB of device memory per GPU, held for the life of the process.
static __device__ __align__(256) NaScratch g_noalloc_scratch[1];

struct NaGrid {
    int n, ncell, nc[3], ntypes;
    float inv_side[3];
    float box[3], box_lo[3];
    double boxd[3];
};

__global__ void k_na_clear(NaScratch *S, int ncell) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) S->cell_count[c] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) { S->sums[0] = 0.0; S->sums[1] = 0.0; }
}

// Wrap each position into [0, L) in FP64, round it to FP32 and bin it.
__global__ void k_na_bin(NaScratch *S, NaGrid g, const double *pos) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.n) return;
    int c3[3];
    for (int d = 0; d < 3; ++d) {
        double L = g.boxd[d], x = pos[3 * p + d];
        x = x - L * floor(x / L);
        if (!(x < L)) x = 0.0;
        float w = (float)x;
        int c = (int)floorf(w * g.inv_side[d]);
        c3[d] = c < 0 ? 0 : (c > g.nc[d] - 1 ? g.nc[d] - 1 : c);
    }
    const int cell = (c3[2] * g.nc[1] + c3[1]) * g.nc[0] + c3[0];
    S->cell_of[p] = cell;
    S->slot_of[p] = atomicAdd(&S->cell_count[cell], 1);
}

// One block: exclusive scan of the cell counts (ncell <= NA_MAX_CELLS).
__global__ void __launch_bounds__(NA_SCAN_THREADS) k_na_scan(NaScratch *S, int ncell) {
    __shared__ int s_sum[NA_SCAN_THREADS];
    const int per = (ncell + NA_SCAN_THREADS - 1) / NA_SCAN_THREADS;
    const int b = threadIdx.x * per, e = min(ncell, b + per);
    int t = 0;
    for (int c = b; c < e; ++c) t += S->cell_count[c];
    s_sum[threadIdx.x] = t;
    __syncthreads();
    for (int o = 1; o < NA_SCAN_THREADS; o <<= 1) {
        int v = threadIdx.x >= o ? s_sum[threadIdx.x - o] : 0;
        __syncthreads();
        s_sum[threadIdx.x] += v;
        __syncthreads();
    }
    int run = s_sum[threadIdx.x] - t;
    for (int c = b; c < e; ++c) { S->cell_start[c] = run; run += S->cell_count[c]; }
    if (threadIdx.x == NA_SCAN_THREADS - 1) S->cell_start[ncell] = s_sum[NA_SCAN_THREADS - 1];
}

__global__ void k_na_scatter(NaScratch *S, NaGrid g, const double *pos, const int *types) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.n) return;
    const int cell = S->cell_of[p];
    const int q = S->cell_start[cell] + S->slot_of[p];
    float w[3];
    for (int d = 0; d < 3; ++d) {
        double L = g.boxd[d], x = pos[3 * p + d];
        x = x - L * floor(x / L);
        if (!(x < L)) x = 0.0;
        w[d] = (float)x;
    }
    int t = types ? types[p] : 0;
    t = t < 0 ? 0 : (t >= g.ntypes ? g.ntypes - 1 : t);
    S->pos[q] = make_pos(w[0], w[1], w[2], t);
    S->id[q] = p;
    S->cell_sorted[q] = cell;
}

__device__ __forceinline__ int na_floor_div(int a, int b) { int q = a / b; return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q; }

// Thread per sorted particle, 27 stencil cells, full neighbour set (no N3L),
// the library's pair arithmetic and exact cutoff decision.
__global__ void __launch_bounds__(NA_THREADS) k_na_force(NaScratch *S, NaGrid g, PairTab<float> tab, double *forces) {
    __shared__ double s_red[2][NA_THREADS / 32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float fx = 0.f, fy = 0.f, fz = 0.f, u = 0.f, w = 0.f;
    if (i < g.n) {
        const float4 pi = S->pos[i];
        const int ti = type_of(pi);
        const int c = S->cell_sorted[i];
        const int cx = c % g.nc[0], cy = (c / g.nc[0]) % g.nc[1], cz = c / (g.nc[0] * g.nc[1]);
        for (int oz = -1; oz <= 1; ++oz) {
            int rz = cz + oz, sz = na_floor_div(rz, g.nc[2]);
            int wz = rz - sz * g.nc[2];
            for (int oy = -1; oy <= 1; ++oy) {
                int ry = cy + oy, sy = na_floor_div(ry, g.nc[1]);
                int wy = ry - sy * g.nc[1];
                for (int ox = -1; ox <= 1; ++ox) {
                    int rx = cx + ox, sx = na_floor_div(rx, g.nc[0]);
                    int wx = rx - sx * g.nc[0];
                    const int cc = (wz * g.nc[1] + wy) * g.nc[0] + wx;
                    const bool img = (sx | sy | sz) != 0;
                    for (int j = S->cell_start[cc]; j < S->cell_start[cc + 1]; ++j) {
                        if (j == i && !img) continue;
                        const float4 pj = S->pos[j];
                        const float dx = image_dx(pi.x, pj.x, sx, g.box[0], g.box_lo[0]);
                        const float dy = image_dx(pi.y, pj.y, sy, g.box[1], g.box_lo[1]);
                        const float dz = image_dx(pi.z, pj.z, sz, g.box[2], g.box_lo[2]);
                        const float r2 = r2_of(dx, dy, dz);
                        const int tp = ti * tab.ntypes + type_of(pj);
                        const bool in = Cut<float>::in(r2, tab.rc2lo[tp], tab.rc2hi[tp], pi, pj, sx, sy, sz, g.boxd,
                                                       tab.rc2d[tp]);
                        float sr6;
                        float fr = lj_fr(r2, tab.sig2[tp], tab.e24[tp], tab.e48[tp], sr6);
                        fr = in ? fr : 0.f;
                        fx += fr * dx; fy += fr * dy; fz += fr * dz;
                        u += in ? tab.e4[tp] * sr6 * (sr6 - 1.f) - tab.ushift[tp] : 0.f;
                        w += fr * r2;
                    }
                }
            }
        }
        const int id = S->id[i];
        forces[3 * id + 0] = fx; forces[3 * id + 1] = fy; forces[3 * id + 2] = fz;
    }
    double a = 0.5 * u, b = 0.5 * w;
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) { s_red[0][threadIdx.x >> 5] = a; s_red[1][threadIdx.x >> 5] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, y = 0;
        for (int k = 0; k < NA_THREADS / 32; ++k) { x += s_red[0][k]; y += s_red[1][k]; }
        atomicAdd(&S->sums[0], x);
        atomicAdd(&S->sums[1], y);
    }
}

// Device address of the scratch array, resolved with cudaGetSymbolAddress
// once per CUDA context (the host-side name is only a stand-in, not an
// address).  The cache is keyed by the context's unique id, so that a
// context destroyed by cudaDeviceReset and created again resolves the
// address anew instead of reusing a dangling one.  When the context id is
// not available the address is resolved on every call.
std::mutex g_na_mutex;
struct NaSlot {
    unsigned long long ctx_id = 0;
    NaScratch *addr = nullptr;
};
NaSlot g_na_addr[64];

typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

// Id of the current context through the driver entry points (0 if unknown).
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (CtxGetIdFn)f;
    }
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (!get_cur || !get_id || get_cur(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0ull;
    return id;
}

}  // namespace
}  // namespace ljsel

using namespace ljsel;

extern "C" ljsel_status ljsel_compute_forces_noalloc(const ljsel_params *params, int64_t n, const double *pos,
                                                     const int32_t *types, double *forces, double *energy,
                                                     double *virial, void *stream) {
    set_error("");
    ljsel_status st = validate_params(params);
    if (st != LJSEL_OK) return st;
    if (params->precision != 0) { set_error("the allocation-free path computes in FP32 (precision 0)"); return LJSEL_ERR_UNSUPPORTED; }
    if (params->walls[0] || params->walls[1] || params->walls[2]) {
        set_error("the allocation-free path handles periodic boxes only");
        return LJSEL_ERR_UNSUPPORTED;
    }
    if (!pos || !forces || n < 1) { set_error("pos and forces are required, n >= 1"); return LJSEL_ERR_ARG; }
    if (n > NA_MAX_N) { set_error("n exceeds the allocation-free limit of 131072 particles"); return LJSEL_ERR_CAPACITY; }
    double rcm = 0;
    for (int t = 0; t < params->ntypes * params->ntypes; ++t) rcm = rcm > params->rcut[t] ? rcm : params->rcut[t];
    NaGrid g;
    g.n = (int)n;
    g.ntypes = params->ntypes;
    g.ncell = 1;
    const double side_min = rcm * (1.0 + 1.0 / 4096.0) * (1.0 + 1.0 / 4096.0);
    for (int d = 0; d < 3; ++d) {
        g.nc[d] = (int)floor(params->box[d] / side_min);
        if (g.nc[d] < 1) g.nc[d] = 1;
        if ((long long)g.ncell * g.nc[d] > NA_MAX_CELLS) { set_error("the box needs more than 131072 cells, the allocation-free limit"); return LJSEL_ERR_CAPACITY; }
        g.ncell *= g.nc[d];
        g.inv_side[d] = (float)(g.nc[d] / params->box[d]);
        g.box[d] = (float)params->box[d];
        g.box_lo[d] = (float)(params->box[d] - (double)g.box[d]);
        g.boxd[d] = params->box[d];
    }
    cudaStream_t st_ = (cudaStream_t)stream;
    if (energy || virial) {
        // the sums are read back with a synchronize, which a stream being
        // captured does not allow (it would invalidate the caller's capture)
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st_, &cs) != cudaSuccess) { set_error("invalid stream"); return LJSEL_ERR_ARG; }
        if (cs != cudaStreamCaptureStatusNone) {
            set_error("energy and virial are read back with a stream synchronize, which is not allowed while the "
                      "stream is being captured: pass NULL for both");
            return LJSEL_ERR_STATE;
        }
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { set_error("no current CUDA device"); return LJSEL_ERR_CUDA; }
    NaScratch *S = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mutex);
        const unsigned long long ctx = current_context_id();
        NaSlot &slot = g_na_addr[dev];
        if (!slot.addr || ctx == 0ull || slot.ctx_id != ctx) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) { set_error(std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e)); return LJSEL_ERR_CUDA; }
            slot.addr = (NaScratch *)p;
            slot.ctx_id = ctx;
        }
        S = slot.addr;
    }
    // the pair table of the library's FP32 path
    System tmp;
    tmp.params = *params;
    tmp.n = (int)n;
    Dev<float> D;
    tmp.fill_dev(D);
    k_na_clear<<<div_up(g.ncell, 256) < 1024 ? div_up(g.ncell, 256) : 1024, 256, 0, st_>>>(S, g.ncell);
    k_na_bin<<<div_up(n, 256), 256, 0, st_>>>(S, g, pos);
    k_na_scan<<<1, NA_SCAN_THREADS, 0, st_>>>(S, g.ncell);
    k_na_scatter<<<div_up(n, 256), 256, 0, st_>>>(S, g, pos, types);
    k_na_force<<<div_up(n, NA_THREADS), NA_THREADS, 0, st_>>>(S, g, D.tab, forces);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { set_error(std::string("launch failed: ") + cudaGetErrorString(e)); return LJSEL_ERR_CUDA; }
    if (energy || virial) {
        double sums[2] = {0, 0};
        e = cudaMemcpyAsync(sums, &S->sums[0], sizeof(sums), cudaMemcpyDeviceToHost, st_);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st_);
        if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return LJSEL_ERR_CUDA; }
        if (energy) *energy = sums[0];
        if (virial) *virial = sums[1];
    }
    return LJSEL_OK;
}
