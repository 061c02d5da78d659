// system.cu -- host runtime behind the C ABI in include/ljsel.h.
//
// A System owns the device state of one particle system: FP64 positions and
// velocities, the working-precision copy, the cell grid and the neighbour
// lists of the selected configuration.  Stepping (Sec. 2.1) runs either as
// plain stream launches or as one CUDA graph per configuration:
//
//   init kernel -> WHILE(steps left) {
//       IF(rebuild needed) { bin -> scan -> scatter -> sort+gather -> lists -> finish }
//       force+update kernel(s) -> control kernel (sets both conditions)
//   }
//
// so the decision to rebuild (every R steps, or as soon as a particle has
// moved skin/2, the Verlet-list guarantee of Sec. 2.2.1) is taken on the
// device without a host round trip.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "system.h"

namespace ljsel {

static thread_local std::string g_last_error;

void set_error(const std::string &m) { g_last_error = m; }
const char *last_error() { return g_last_error.c_str(); }

#define LJ_CUDA(call)                                                                              \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) {                                                                   \
            set_error(std::string("CUDA error in ") + #call + ": " + cudaGetErrorString(e_));      \
            return e_ == cudaErrorMemoryAllocation ? LJSEL_ERR_OOM : LJSEL_ERR_CUDA;               \
        }                                                                                          \
    } while (0)

#define LJ_TRY(expr)                         \
    do {                                     \
        ljsel_status s_ = (expr);            \
        if (s_ != LJSEL_OK) return s_;       \
    } while (0)

// ---------------------------------------------------------------------------
// Device buffers

// Device buffers come from the device's default memory pool, which is told
// once per device to keep up to 8 GB of freed memory for reuse: a system
// created after another was destroyed then takes its buffers from the pool
// instead of the driver (a cudaMalloc or cudaFree of a large buffer costs
// tens to hundreds of microseconds and a cudaFree synchronizes the device).
// Allocations and frees are ordered on the legacy default stream and waited
// for, so a buffer is ready on any stream when ensure returns, and a freed
// one is reused only after the work that used it (every caller synchronizes
// its stream before it regrows or releases a buffer).
static ljsel_status pool_once() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LJSEL_OK;
    std::lock_guard<std::mutex> lk(mu);
    if (done[dev]) return LJSEL_OK;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = 8ull << 30;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    done[dev] = true;
    return LJSEL_OK;
}

ljsel_status Buf::ensure(size_t bytes) {
    if (bytes <= size) return LJSEL_OK;
    release();
    pool_once();
    cudaError_t e = cudaMallocAsync(&ptr, bytes ? bytes : 16, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    if (e != cudaSuccess) {
        if (ptr) cudaFreeAsync(ptr, 0);
        ptr = nullptr;
        set_error(std::string("allocation of ") + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? LJSEL_ERR_OOM : LJSEL_ERR_CUDA;
    }
    size = bytes;
    return LJSEL_OK;
}
void Buf::release() {
    if (ptr) cudaFreeAsync(ptr, 0);
    ptr = nullptr;
    size = 0;
}

// ---------------------------------------------------------------------------

static double rc_max(const ljsel_params &p) {
    double m = 0;
    for (int t = 0; t < p.ntypes * p.ntypes; ++t) m = std::max(m, p.rcut[t]);
    return m;
}

ljsel_status validate_params(const ljsel_params *p) {
    if (!p) { set_error("params is NULL"); return LJSEL_ERR_ARG; }
    if (p->ntypes < 1 || p->ntypes > LJSEL_MAX_TYPES) { set_error("ntypes out of range"); return LJSEL_ERR_ARG; }
    if (p->precision != 0 && p->precision != 1) { set_error("precision must be 0 or 1"); return LJSEL_ERR_ARG; }
    if (!(p->skin >= 0) || !(p->dt > 0)) { set_error("skin must be >= 0 and dt > 0"); return LJSEL_ERR_ARG; }
    const int nt = p->ntypes;
    for (int a = 0; a < nt; ++a) {
        if (!(p->mass[a] > 0)) { set_error("masses must be positive"); return LJSEL_ERR_ARG; }
        for (int b = 0; b < nt; ++b) {
            int t = a * nt + b, u = b * nt + a;
            if (!(p->eps[t] >= 0) || !(p->sigma[t] > 0) || !(p->rcut[t] > 0)) { set_error("eps >= 0, sigma > 0, rcut > 0 required"); return LJSEL_ERR_ARG; }
            if (p->eps[t] != p->eps[u] || p->sigma[t] != p->sigma[u] || p->rcut[t] != p->rcut[u]) { set_error("type-pair tables must be symmetric"); return LJSEL_ERR_ARG; }
        }
    }
    const double rl = rc_max(*p) + p->skin;
    for (int d = 0; d < 3; ++d) {
        if (!(p->box[d] > 0) || !std::isfinite(p->box[d])) { set_error("box lengths must be positive"); return LJSEL_ERR_ARG; }
        if (p->walls[d] != 0 && p->walls[d] != 1) { set_error("walls[d] must be 0 or 1"); return LJSEL_ERR_ARG; }
        if (!p->walls[d] && p->box[d] < 2.0 * rl * (1.0 + 1.0 / 1024.0)) {
            set_error("box length below 2 (r_c + skin): minimum image would be ambiguous");
            return LJSEL_ERR_BOX;
        }
    }
    return LJSEL_OK;
}

ljsel_status validate_config(const System &s, const ljsel_config *c) {
    if (!c) { set_error("config is NULL"); return LJSEL_ERR_ARG; }
    if (c->method < 0 || c->method > 3) { set_error("unknown method"); return LJSEL_ERR_UNSUPPORTED; }
    if (c->rebuild_interval < 1) { set_error("rebuild_interval must be >= 1"); return LJSEL_ERR_ARG; }
    if (c->csf != 1.0 && c->csf != 0.5) { set_error("csf must be 1.0 or 0.5"); return LJSEL_ERR_UNSUPPORTED; }
    if (c->newton3 != 0 && c->newton3 != 1) { set_error("newton3 must be 0 or 1"); return LJSEL_ERR_ARG; }
    const int t = c->threads_per_unit;
    if (c->method == LJSEL_METHOD_VL) {
        if (t != 1 && t != 2 && t != 4 && t != 8 && t != 16 && t != 32) { set_error("VL threads_per_unit must be a power of two <= 32"); return LJSEL_ERR_UNSUPPORTED; }
    } else if (c->method == LJSEL_METHOD_CLUSTER) {
        const int M = c->cluster_size;
        if (M != 2 && M != 4 && M != 8) { set_error("cluster_size must be 2, 4 or 8"); return LJSEL_ERR_UNSUPPORTED; }
        if (t < M || t > 32 || (t & (t - 1)) != 0) { set_error("CLUSTER threads_per_unit must be M, 2M, ... <= 32"); return LJSEL_ERR_UNSUPPORTED; }
    } else if (c->method == LJSEL_METHOD_VLW) {
        if (t != 1) { set_error("VLW uses threads_per_unit = 1"); return LJSEL_ERR_UNSUPPORTED; }
        if (c->csf != 1.0) { set_error("VLW uses csf = 1"); return LJSEL_ERR_UNSUPPORTED; }
    } else {
        if (t != 1) { set_error("LC uses threads_per_unit = 1"); return LJSEL_ERR_UNSUPPORTED; }
    }
    const bool walled = s.params.walls[0] || s.params.walls[1] || s.params.walls[2];
    if (walled && c->method == LJSEL_METHOD_VLW) {
        set_error("reflective walls are available with the LC, VL and CLUSTER methods");
        return LJSEL_ERR_UNSUPPORTED;
    }
    if (s.params.skin == 0.0 && c->method != LJSEL_METHOD_LC && c->rebuild_interval != 1) {
        set_error("without a skin the lists must be rebuilt every step (R = 1)");
        return LJSEL_ERR_ARG;
    }
    return LJSEL_OK;
}

// ---------------------------------------------------------------------------

System::~System() {
    drop_graph();
    for (Buf *b : all_bufs()) b->release();
    if (h_ctrl) cudaFreeHost(h_ctrl);
    if (h_stats) cudaFreeHost(h_stats);
    if (ev_a) cudaEventDestroy(ev_a);
    if (ev_b) cudaEventDestroy(ev_b);
    if (cap_stream) cudaStreamDestroy(cap_stream);
}

std::vector<Buf *> System::all_bufs() {
    return {&b_x[0], &b_x[1], &b_v[0], &b_v[1], &b_id[0], &b_id[1], &b_type[0], &b_type[1], &b_pos[0], &b_pos[1],
            &b_xref, &b_force, &b_cell_count, &b_cell_start, &b_clcell_start, &b_cell_of, &b_slot_of, &b_key_of,
            &b_tmp_idx, &b_tmp_key, &b_cell_sorted, &b_scan, &b_nl, &b_nl_count, &b_strips, &b_nstrips, &b_cl_first, &b_cl_count,
            &b_cl_cell, &b_cp, &b_cp_count, &b_ncl, &b_ctrl, &b_io,
            &b_adj_cot, &b_adj_x, &b_adj_v, &b_adj_theta, &b_ckpt, &b_seg, &b_stats};
}

void System::drop_graph() {
    for (GraphEntry &e : gcache) {
        if (e.exec) cudaGraphExecDestroy(e.exec);
        if (e.graph) cudaGraphDestroy(e.graph);
    }
    gcache.clear();
    gexec = nullptr;
}

size_t System::p4() const { return precision ? sizeof(D4) : sizeof(float4); }

// Cell grid of the current configuration: side >= (r_c,max + skin) * CSF,
// slightly enlarged so that FP32 rounding of a position at a cell face can
// never hide a pair; stretched to tile the box (Sec. 2.2.1).
void System::plan_grid() {
    const double rl = rc_max(params) + params.skin;
    rlist = rl * (1.0 + 1.0 / 4096.0);
    const double side_min = rlist * cfg.csf * (1.0 + 1.0 / 4096.0);
    ncell = 1;
    for (int d = 0; d < 3; ++d) {
        nc[d] = std::max(1, (int)std::floor(params.box[d] / side_min));
        side[d] = params.box[d] / nc[d];
        ncell *= nc[d];
    }
    reach = cfg.csf < 1.0 ? 2 : 1;
}

ljsel_status System::alloc_base() {
    const size_t n3 = (size_t)n * 3 * sizeof(double);
    for (int k = 0; k < 2; ++k) {
        LJ_TRY(b_x[k].ensure(n3));
        LJ_TRY(b_v[k].ensure(n3));
        LJ_TRY(b_id[k].ensure((size_t)n * 4));
        LJ_TRY(b_type[k].ensure((size_t)n * 4));
        LJ_TRY(b_pos[k].ensure((size_t)(n + 1) * p4()));
    }
    LJ_TRY(b_xref.ensure((size_t)n * p4()));
    LJ_TRY(b_force.ensure((size_t)n * p4()));
    LJ_CUDA(cudaMemsetAsync(b_force.ptr, 0, (size_t)n * p4(), stream));
    LJ_TRY(b_cell_of.ensure((size_t)n * 4));
    LJ_TRY(b_slot_of.ensure((size_t)n * 4));
    LJ_TRY(b_key_of.ensure((size_t)n * 8));
    LJ_TRY(b_tmp_idx.ensure((size_t)n * 4));
    LJ_TRY(b_tmp_key.ensure((size_t)n * 8));
    LJ_TRY(b_cell_sorted.ensure((size_t)n * 4));
    LJ_TRY(b_ncl.ensure(16));
    LJ_CUDA(cudaMemsetAsync(b_ncl.ptr, 0, 16, stream));
    LJ_TRY(b_ctrl.ensure(sizeof(Ctrl)));
    LJ_CUDA(cudaMemsetAsync(b_ctrl.ptr, 0, sizeof(Ctrl), stream));
    // the sentinel particle n that pads list rows: far outside the box, so
    // every pair with it is out of range and its force term is exactly zero
    for (int k = 0; k < 2; ++k) {
        if (precision) {
            D4 far = {1e18, 1e18, 1e18, 0.0};
            LJ_CUDA(cudaMemcpyAsync((char *)b_pos[k].ptr + (size_t)n * p4(), &far, sizeof(far), cudaMemcpyHostToDevice, stream));
        } else {
            float4 far = make_float4(1e18f, 1e18f, 1e18f, 0.f);
            LJ_CUDA(cudaMemcpyAsync((char *)b_pos[k].ptr + (size_t)n * p4(), &far, sizeof(far), cudaMemcpyHostToDevice, stream));
        }
    }
    LJ_CUDA(cudaStreamSynchronize(stream));
    return LJSEL_OK;
}

// Allocate everything the configuration needs (grow-only) and mark the
// neighbour structure for a rebuild.
ljsel_status System::apply_config() {
    plan_grid();
    const size_t cells1 = (size_t)ncell + 1;
    bool grew = false;
    auto grow = [&](Buf &b, size_t bytes) -> ljsel_status {
        if (bytes > b.size) {
            grew = true;
            ljsel_status st = b.ensure(bytes);
            if (st != LJSEL_OK) return st;
            if (&b == &b_cell_count || &b == &b_nl_count || &b == &b_cp_count)
                LJ_CUDA(cudaMemsetAsync(b.ptr, 0, bytes, stream));
        }
        return LJSEL_OK;
    };
    LJ_TRY(grow(b_cell_count, cells1 * 4));
    LJ_TRY(grow(b_cell_start, cells1 * 4));
    LJ_TRY(grow(b_clcell_start, cells1 * 4));
    LJ_TRY(grow(b_scan, (size_t)(ncell / 4096 + 2) * 8));
    M = cfg.method == LJSEL_METHOD_CLUSTER ? cfg.cluster_size : 1;
    if (cfg.method == LJSEL_METHOD_VL) {
        if (nl_cap <= 0) {
            // mean density estimate of the list row length, with room
            const double vol = params.box[0] * params.box[1] * params.box[2];
            const double rho = n / vol;
            double est = 4.18879 * rlist * rlist * rlist * rho * 1.35 + 16;
            if (cfg.newton3) est = est * 0.5 + 8;
            nl_cap = (int)std::min(est, 4096.0);
        }
        nl_cap = (nl_cap + 3) & ~3;
        LJ_TRY(grow(b_nl, (size_t)nl_cap * n * 4));
        LJ_TRY(grow(b_nl_count, (size_t)n * 4));
    }
    if (cfg.method == LJSEL_METHOD_VLW) {
        vlw_prepare();
        if (nl_cap <= 0) {
            const double vol = params.box[0] * params.box[1] * params.box[2];
            const double rho = n / vol;
            double est = 4.18879 * rlist * rlist * rlist * rho * 1.35 + 24;
            if (cfg.newton3) est = est * 0.5 + 16;
            nl_cap = (int)std::min(est, 4096.0);
        }
        nl_cap = std::min((nl_cap + 15) & ~15, 512);  // two half-rows, at most 255 + 1 entries each
        LJ_TRY(grow(b_nl, (size_t)nl_cap * n * 2));
        LJ_TRY(grow(b_nl_count, (size_t)n * 4));
        LJ_TRY(grow(b_strips, (size_t)ncell * sizeof(int4)));
        LJ_TRY(grow(b_nstrips, 16));
    }
    if (cfg.method == LJSEL_METHOD_CLUSTER) {
        ncl_cap = n / M + ncell + 1;
        if (cp_cap <= 0) {
            // the union of M members' neighbourhoods: a sphere of the list
            // radius widened by about the cluster's radius, with room
            const double vol = params.box[0] * params.box[1] * params.box[2];
            const double rho = n / vol;
            const double grow_r = 0.62 * std::cbrt(M / std::max(rho, 1e-12));
            const double rr = std::min(rlist + grow_r, 2.0 * rlist);
            double est = 4.18879 * rr * rr * rr * rho * 1.3 + 16;
            if (cfg.newton3) est = est * 0.5 + 8;
            cp_cap = (int)std::min(est, 16384.0);
        }
        cp_cap = (cp_cap + 3) & ~3;
        LJ_TRY(grow(b_cl_first, (size_t)ncl_cap * 4));
        LJ_TRY(grow(b_cl_count, (size_t)ncl_cap * 4));
        LJ_TRY(grow(b_cl_cell, (size_t)ncl_cap * 4));
        LJ_TRY(grow(b_cp, (size_t)cp_cap * ncl_cap * 4));
        LJ_TRY(grow(b_cp_count, (size_t)ncl_cap * 4));
    }
    (void)grew;
    gexec = nullptr;  // the next advance looks the configuration up in the graph cache
    structure_dirty = true;
    return LJSEL_OK;
}

template <typename R> void System::fill_dev(Dev<R> &S) const {
    memset(&S, 0, sizeof(S));
    S.n = n;
    S.ncell = ncell;
    for (int d = 0; d < 3; ++d) {
        S.nc[d] = nc[d];
        S.inv_side[d] = (R)(1.0 / side[d]);
        S.box[d] = (R)params.box[d];
        S.box_lo[d] = (R)(params.box[d] - (double)(R)params.box[d]);
        S.boxd[d] = params.box[d];
        float lf = (float)params.box[d];
        if ((double)lf > params.box[d]) lf = std::nextafter(lf, 0.0f);
        S.box_dn[d] = lf;
    }
    S.reach = reach;
    for (int d = 0; d < 3; ++d) S.walls[d] = params.walls[d] ? 1 : 0;
    S.rlist2 = (R)(rlist * rlist);
    const double hs = 0.5 * params.skin;
    S.half_skin2 = (R)(hs * hs);
    for (int k = 0; k < 2; ++k) {
        S.x[k] = (double *)b_x[k].ptr;
        S.v[k] = (double *)b_v[k].ptr;
        S.id[k] = (int *)b_id[k].ptr;
        S.type[k] = (int *)b_type[k].ptr;
        S.pos[k] = (V4<R> *)b_pos[k].ptr;
    }
    S.xref = (V4<R> *)b_xref.ptr;
    S.force = (V4<R> *)b_force.ptr;
    S.cell_count = (int *)b_cell_count.ptr;
    S.cell_start = (int *)b_cell_start.ptr;
    S.clcell_start = (int *)b_clcell_start.ptr;
    S.cell_of = (int *)b_cell_of.ptr;
    S.slot_of = (int *)b_slot_of.ptr;
    S.key_of = (unsigned long long *)b_key_of.ptr;
    S.tmp_idx = (int *)b_tmp_idx.ptr;
    S.tmp_key = (unsigned long long *)b_tmp_key.ptr;
    S.cell_sorted = (int *)b_cell_sorted.ptr;
    S.scan_partial = (int *)b_scan.ptr;
    S.nl = (uint32_t *)b_nl.ptr;
    S.nl16 = (uint16_t *)b_nl.ptr;
    S.strips = (int4 *)b_strips.ptr;
    S.nstrips = (int *)b_nstrips.ptr;
    S.strip_cap = ncell;
    S.nl_count = (int *)b_nl_count.ptr;
    S.nl_cap = nl_cap;
    S.M = M;
    S.ncl_cap = ncl_cap;
    S.cl_first = (int *)b_cl_first.ptr;
    S.cl_count = (int *)b_cl_count.ptr;
    S.cl_cell = (int *)b_cl_cell.ptr;
    S.cp = (uint32_t *)b_cp.ptr;
    S.cp_count = (int *)b_cp_count.ptr;
    S.cp_cap = cp_cap;
    S.ncl_total = (int *)b_ncl.ptr;
    S.ctrl = (Ctrl *)b_ctrl.ptr;
    const int nt = params.ntypes;
    S.tab.ntypes = nt;
    S.tab.dt = params.dt;
    for (int a = 0; a < nt; ++a) {
        S.tab.inv_mass_dt[a] = (R)(params.dt / params.mass[a]);
        S.tab.half_mass[a] = 0.5 * params.mass[a];
        for (int b = 0; b < nt; ++b) {
            const int t = a * nt + b;
            const double e = params.eps[t], sg = params.sigma[t], rc = params.rcut[t];
            const double sr = sg / rc, sr6 = sr * sr * sr * sr * sr * sr;
            const double uc = 4.0 * e * (sr6 * sr6 - sr6);
            S.tab.sig2[t] = (R)(sg * sg);
            S.tab.inv_sig[t] = (R)(1.0 / sg);
            S.tab.e24[t] = (R)(24.0 * e);
            S.tab.e48[t] = (R)(48.0 * e);
            S.tab.e4[t] = (R)(4.0 * e);
            const double sg6 = sg * sg * sg * sg * sg * sg;
            S.tab.a12[t] = (R)(48.0 * e * sg6 * sg6);
            S.tab.b6[t] = (R)(24.0 * e * sg6);
            S.tab.ushift[t] = params.shift_potential ? (R)uc : (R)0;
            S.tab.rc2d[t] = rc * rc;
            S.tab.rc2lo[t] = (R)(rc * rc * (1.0 - 1.0 / 16384.0));
            S.tab.rc2hi[t] = (R)(rc * rc * (1.0 + 1.0 / 16384.0));
        }
    }
}

// Small host-to-device control updates are kernels, so they stay ordered
// with the stream and can be reused inside captures.
namespace {
__global__ void k_cmd(Ctrl *C, int op, long long a) {
    switch (op) {
        case CMD_REBUILD: C->rebuild_now = 1; break;
        case CMD_BEGIN: C->steps_done = 0; C->steps_target = a; break;
        case CMD_RESET_EV: C->epot = 0; C->virial = 0; C->ekin = 0; break;
        case CMD_RESET_PAIRS: C->npairs = 0; break;
        case CMD_HALF_KICK: C->half_kick = (int)a; break;
        case CMD_CLEAR: C->overflow = 0; C->need_cap = 0; C->disp_exceeded = 0; break;
        case CMD_INTERVAL: C->rebuild_interval = (int)a; break;
    }
}
}  // namespace

ljsel_status System::cmd(int op, long long a) {
    k_cmd<<<1, 1, 0, stream>>>((Ctrl *)b_ctrl.ptr, op, a);
    LJ_CUDA(cudaGetLastError());
    return LJSEL_OK;
}

ljsel_status System::read_ctrl() {
    LJ_CUDA(cudaMemcpyAsync(h_ctrl, b_ctrl.ptr, sizeof(Ctrl), cudaMemcpyDeviceToHost, stream));
    LJ_CUDA(cudaStreamSynchronize(stream));
    return LJSEL_OK;
}

ljsel_status System::check_device_errors() {
    if (h_ctrl->check_failed) {
        set_error("bounds check failed at site " + std::to_string(h_ctrl->check_site) + " (checked build)");
        return LJSEL_ERR_STATE;
    }
    if (h_ctrl->nonfinite) { set_error("non-finite position, velocity or force"); return LJSEL_ERR_NONFINITE; }
    if (h_ctrl->timeout) { set_error("a bounded device wait gave up (scan look-back)"); return LJSEL_ERR_TIMEOUT; }
    if (h_ctrl->window_overflow) {
        set_error("a cell's neighbourhood window holds more than 2047 particles: VLW is not available here");
        return LJSEL_ERR_UNSUPPORTED;
    }
    return LJSEL_OK;
}

template <typename R> void System::enqueue_rebuild(const Dev<R> &S, cudaStream_t st) {
    launch_bin(S, st);
    launch_scan(S, M, st);
    launch_scatter(S, st);
    launch_sortgather(S, st);
    if (cfg.method == LJSEL_METHOD_VL) launch_vl_build(S, cfg.newton3 != 0, st);
    if (cfg.method == LJSEL_METHOD_VLW) {
        launch_strip_plan(S, st);
        launch_vlw_build(S, cfg.newton3 != 0, st);
    }
    if (cfg.method == LJSEL_METHOD_CLUSTER) {
        launch_cluster_form(S, st);
        launch_cp_build(S, cfg.newton3 != 0, st);
    }
    launch_rebuild_finish(S.ctrl, st);
}

template <typename R> void System::enqueue_step(const Dev<R> &S, bool ev, cudaStream_t st) {
    if (cfg.newton3) {
        launch_force(S, cfg, MODE_FORCE, ev, nullptr, 0, st);
        launch_integrate(S, ev, st);
    } else {
        launch_force(S, cfg, MODE_STEP, ev, nullptr, 0, st);
    }
}

// Grow the list after an overflow: the failed build recorded the longest row
// it needed.
ljsel_status System::handle_overflow() {
    const long long need = h_ctrl->need_cap;
    const long long cap = (long long)std::max<long long>(need + need / 5 + 8, 16);
    if (cfg.method == LJSEL_METHOD_VL) nl_cap = (int)((cap + 3) & ~3LL);
    else if (cfg.method == LJSEL_METHOD_VLW) {
        if (cap > 512) { set_error("VLW rows hold at most 510 entries; the system is too dense for VLW"); return LJSEL_ERR_UNSUPPORTED; }
        nl_cap = (int)((cap + 15) & ~15LL);
    }
    else if (cfg.method == LJSEL_METHOD_CLUSTER) cp_cap = (int)cap;
    capacity_retries += 1;
    if (capacity_retries > 64) { set_error("neighbour list keeps overflowing"); return LJSEL_ERR_CAPACITY; }
    LJ_TRY(apply_config());
    LJ_TRY(cmd(CMD_CLEAR, 0));
    LJ_TRY(cmd(CMD_REBUILD, 0));
    return LJSEL_OK;
}

// Make the neighbour structure current (rebuild if flagged), retrying after
// capacity overflows.  Leaves the stream synchronized.
template <typename R> ljsel_status System::ensure_structure() {
    for (int attempt = 0; attempt < 8; ++attempt) {
        if (structure_dirty) {
            LJ_TRY(cmd(CMD_INTERVAL, cfg.rebuild_interval));
            LJ_TRY(cmd(CMD_REBUILD, 0));
            structure_dirty = false;
        }
        Dev<R> S;
        fill_dev(S);
        enqueue_rebuild(S, stream);
        LJ_CUDA(cudaGetLastError());
        LJ_TRY(read_ctrl());
        LJ_TRY(check_device_errors());
        if (!h_ctrl->overflow) {
            // Verlet-list rows have a fixed capacity set from the mean density;
            // once a build has measured the longest row, the capacity is fitted
            // to it (with room for its fluctuation), so that the force kernel's
            // prefetch of a block's rows carries little unused capacity.
            const long long need = h_ctrl->need_cap;
            if (cfg.method == LJSEL_METHOD_VL && !cap_fitted && need > 0 && nl_cap > need + need / 8 + 16) {
                cap_fitted = true;
                nl_cap = (int)((need + need / 16 + 8 + 3) & ~3LL);
                LJ_TRY(apply_config());
                LJ_TRY(cmd(CMD_REBUILD, 0));
                continue;
            }
            return LJSEL_OK;
        }
        LJ_TRY(handle_overflow());
    }
    set_error("neighbour structure could not be built");
    return LJSEL_ERR_CAPACITY;
}

template <typename R> ljsel_status System::build_graph() {
    if (!cap_stream) LJ_CUDA(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
    Dev<R> S;
    fill_dev(S);
    GraphEntry e;
    e.cfg = cfg;
    e.key.assign(reinterpret_cast<const unsigned char *>(&S), reinterpret_cast<const unsigned char *>(&S) + sizeof(S));
    cudaGraph_t graph = nullptr;
    LJ_CUDA(cudaGraphCreate(&graph, 0));
    e.graph = graph;
    auto fail = [&](cudaError_t err) {
        cudaGraphDestroy(graph);
        set_error(std::string("building the step graph failed: ") + cudaGetErrorString(err));
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
    // init node
    G_CK(cudaStreamBeginCaptureToGraph(cap_stream, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    launch_loop_init((Ctrl *)b_ctrl.ptr, h_reb, h_loop, cap_stream);
    cudaGraph_t tmp = nullptr;
    G_CK(cudaStreamEndCapture(cap_stream, &tmp));
    size_t nn = 0;
    G_CK(cudaGraphGetNodes(graph, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    G_CK(cudaGraphGetNodes(graph, nodes.data(), &nn));
    if (nn != 1) { cudaGraphDestroy(graph); set_error("unexpected node count while building the step graph"); return LJSEL_ERR_CUDA; }
    // WHILE node
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = h_loop;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    G_CK(cudaGraphAddNode(&wnode, graph, nodes.data(), nullptr, 1, &wp));
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    // IF(rebuild) inside the loop body
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
    // step kernels + control, after the IF node
    G_CK(cudaStreamBeginCaptureToGraph(cap_stream, body, &inode, nullptr, 1, cudaStreamCaptureModeThreadLocal));
    enqueue_step(S, false, cap_stream);
    launch_control((Ctrl *)b_ctrl.ptr, h_reb, h_loop, 1, cap_stream);
    G_CK(cudaStreamEndCapture(cap_stream, &tmp));
    G_CK(cudaGraphInstantiate(&e.exec, graph, 0));
#undef G_CK
    if (gcache.size() >= 48) {  // drop the oldest entry
        cudaGraphExecDestroy(gcache.front().exec);
        cudaGraphDestroy(gcache.front().graph);
        gcache.erase(gcache.begin());
    }
    gcache.push_back(e);
    gexec = e.exec;
    return LJSEL_OK;
}

// Reuse the cached graph of this configuration when the kernel-parameter
// block (every pointer, size and capacity baked into the graph) is unchanged.
template <typename R> ljsel_status System::ensure_graph() {
    if (gexec) return LJSEL_OK;
    Dev<R> S;
    fill_dev(S);
    const unsigned char *kb = reinterpret_cast<const unsigned char *>(&S);
    for (GraphEntry &e : gcache) {
        if (e.key.size() == sizeof(S) && memcmp(e.key.data(), kb, sizeof(S)) == 0 &&
            memcmp(&e.cfg, &cfg, sizeof(cfg)) == 0) {
            gexec = e.exec;
            return LJSEL_OK;
        }
    }
    return build_graph<R>();
}

template <typename R> ljsel_status System::advance(long long nsteps, bool eager) {
    if (nsteps <= 0) return LJSEL_OK;
    LJ_TRY(ensure_structure<R>());
    long long left = nsteps;
    for (int round = 0; round < 16 && left > 0; ++round) {
        LJ_TRY(cmd(CMD_BEGIN, left));
        if (params.use_graphs && !eager) {
            LJ_TRY(ensure_graph<R>());
            LJ_CUDA(cudaGraphLaunch(gexec, stream));
        } else {
            Dev<R> S;
            fill_dev(S);
            for (long long k = 0; k < left; ++k) {
                enqueue_rebuild(S, stream);
                enqueue_step(S, false, stream);
                launch_control(S.ctrl, 0, 0, 0, stream);
            }
        }
        LJ_CUDA(cudaGetLastError());
        LJ_TRY(read_ctrl());
        LJ_TRY(check_device_errors());
        left -= h_ctrl->steps_done;
        if (h_ctrl->overflow) {
            LJ_TRY(handle_overflow());
            LJ_TRY(ensure_structure<R>());
        }
    }
    synced = false;
    if (left > 0) { set_error("could not complete the requested steps"); return LJSEL_ERR_CAPACITY; }
    return LJSEL_OK;
}

// Forces (into the force buffer), energy and virial at the current positions.
template <typename R> ljsel_status System::compute_forces(bool ev) {
    LJ_TRY(ensure_structure<R>());
    Dev<R> S;
    fill_dev(S);
    LJ_TRY(cmd(CMD_RESET_EV, 0));
    if (cfg.newton3) launch_zero_force(S, stream);
    launch_force(S, cfg, MODE_FORCE, ev, nullptr, 0, stream);
    LJ_CUDA(cudaGetLastError());
    return LJSEL_OK;
}

template <typename R> ljsel_status System::sync_velocities() {
    if (synced) return LJSEL_OK;
    LJ_TRY(compute_forces<R>(false));
    Dev<R> S;
    fill_dev(S);
    launch_sync_velocities(S, stream);
    if (cfg.newton3) launch_zero_force(S, stream);
    LJ_TRY(cmd(CMD_HALF_KICK, 1));
    LJ_CUDA(cudaGetLastError());
    synced = true;
    return LJSEL_OK;
}

// Plain stream launches with events around each kernel class; the host
// reads the control block every step to launch the rebuild only when the
// device asked for it, so every timed interval holds real work.
template <typename R> ljsel_status System::profile(long long nsteps, ljsel_profile *out) {
    memset(out, 0, sizeof(*out));
    LJ_TRY(ensure_structure<R>());
    cudaEvent_t ev[6];
    for (auto &e : ev) LJ_CUDA(cudaEventCreate(&e));
    auto done = [&]() { for (auto &e : ev) cudaEventDestroy(e); };
    Dev<R> S;
    fill_dev(S);
    const int chain = 5 + (cfg.method == LJSEL_METHOD_VL ? 1 : 0) + (cfg.method == LJSEL_METHOD_CLUSTER ? 2 : 0) +
                      (cfg.method == LJSEL_METHOD_VLW ? 2 : 0);
    LJ_TRY(cmd(CMD_BEGIN, nsteps));
    double tr = 0, tf = 0, tu = 0, tc = 0;
    for (long long k = 0; k < nsteps; ++k) {
        if (read_ctrl() != LJSEL_OK) { done(); return LJSEL_ERR_CUDA; }
        if (h_ctrl->overflow) {
            ljsel_status st = handle_overflow();
            if (st == LJSEL_OK) st = ensure_structure<R>();
            if (st != LJSEL_OK) { done(); return st; }
            fill_dev(S);
            continue;
        }
        const bool reb = h_ctrl->rebuild_now != 0;
        if (reb) {
            cudaEventRecord(ev[0], stream);
            enqueue_rebuild(S, stream);
            cudaEventRecord(ev[1], stream);
            out->launches += chain;
        }
        cudaEventRecord(ev[2], stream);
        launch_force(S, cfg, cfg.newton3 ? MODE_FORCE : MODE_STEP, false, nullptr, 0, stream);
        cudaEventRecord(ev[3], stream);
        if (cfg.newton3) { launch_integrate(S, false, stream); out->launches += 1; }
        cudaEventRecord(ev[4], stream);
        launch_control(S.ctrl, 0, 0, 0, stream);
        cudaEventRecord(ev[5], stream);
        out->launches += 2;
        cudaError_t e = cudaEventSynchronize(ev[5]);
        if (e != cudaSuccess) { done(); set_error(cudaGetErrorString(e)); return LJSEL_ERR_CUDA; }
        float a = 0, b = 0, c = 0, d = 0;
        if (reb) { cudaEventElapsedTime(&a, ev[0], ev[1]); out->rebuilds += 1; tr += a; }
        cudaEventElapsedTime(&b, ev[2], ev[3]);
        cudaEventElapsedTime(&c, ev[3], ev[4]);
        cudaEventElapsedTime(&d, ev[4], ev[5]);
        tf += b; tu += c; tc += d;
        out->steps += 1;
    }
    done();
    LJ_TRY(read_ctrl());
    LJ_TRY(check_device_errors());
    synced = false;
    out->rebuild_ms = out->rebuilds ? tr / out->rebuilds : 0.0;
    out->force_ms = out->steps ? tf / out->steps : 0.0;
    out->update_ms = (out->steps && cfg.newton3) ? tu / out->steps : 0.0;
    out->control_ms = out->steps ? tc / out->steps : 0.0;
    out->total_ms = tr + tf + tu + tc;
    return LJSEL_OK;
}

// Explicit instantiations of the member templates used by the C ABI.
#define INST(R)                                                        \
    template void System::fill_dev<R>(Dev<R> &) const;                 \
    template void System::enqueue_rebuild<R>(const Dev<R> &, cudaStream_t); \
    template void System::enqueue_step<R>(const Dev<R> &, bool, cudaStream_t); \
    template ljsel_status System::ensure_structure<R>();               \
    template ljsel_status System::build_graph<R>();                    \
    template ljsel_status System::ensure_graph<R>();                   \
    template ljsel_status System::advance<R>(long long, bool);         \
    template ljsel_status System::compute_forces<R>(bool);             \
    template ljsel_status System::sync_velocities<R>();                \
    template ljsel_status System::profile<R>(long long, ljsel_profile *);
INST(float)
INST(double)
#undef INST

}  // namespace ljsel
