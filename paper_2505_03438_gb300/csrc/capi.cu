// capi.cu -- the extern "C" entry points of include/ljsel.h, the live
// statistics of Sec. 4 and the tuning strategies of Sec. 2.2.5 and Sec. 5.1.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kernels.cuh"
#include "system.h"

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

template <typename F> ljsel_status dispatch(System *s, F &&f) {
    if (s->precision) return f((double)0);
    return f((float)0);
}

// Bin counts over CSF-1 cell bins (side >= r_c,max + skin, stretched to the
// box) of the wrapped FP64 positions.
struct BinGrid {
    int nb[3];
    double side[3];
};
// Live statistics on the device (Sec. 4): bin counts from the FP64 state
// (wrapped into the box as ljsel_get_state wraps it), then a histogram of the
// count values with exact integer sums, then one block that reads the mean,
// variance, median, maximum and empty bins off the histogram.  Counts of
// STATS_HMAX or more flag the host path (a copy of all counts).
constexpr int STATS_HMAX = 4096;
struct StatsAcc {
    unsigned long long sum_sq;  // sum over bins of count^2
    unsigned int max;
    unsigned int overflow;      // some count >= STATS_HMAX
};

template <typename R> __global__ void k_stats_bin(Dev<R> S, BinGrid g, int *counts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    const int sp = S.ctrl->state_par, n = S.n;
    int c[3];
    for (int d = 0; d < 3; ++d) {
        double x = S.x[sp][d * n + i];
        if (!S.walls[d]) {
            const double L = S.boxd[d];
            if (x < 0.0) x += L;
            if (x >= L) x -= L;
            if (x < 0.0 || x >= L) { x = x - L * floor(x / L); if (x >= L) x = 0.0; }
        }
        long long k = (long long)floor(x / g.side[d]);
        k %= g.nb[d];
        if (k < 0) k += g.nb[d];
        c[d] = (int)k;
    }
    atomicAdd(&counts[(c[2] * g.nb[1] + c[1]) * g.nb[0] + c[0]], 1);
}

__global__ void k_stats_hist(const int *counts, long long nbins, int *hist, StatsAcc *acc) {
    unsigned long long sq = 0;
    unsigned int mx = 0, over = 0;
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nbins; b += (long long)gridDim.x * blockDim.x) {
        const unsigned int c = (unsigned int)counts[b];
        sq += (unsigned long long)c * c;
        mx = c > mx ? c : mx;
        if (c < (unsigned int)STATS_HMAX) atomicAdd(&hist[c], 1);
        else over = 1;
    }
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_down_sync(0xffffffffu, sq, o);
    mx = __reduce_max_sync(0xffffffffu, mx);
    over = __reduce_or_sync(0xffffffffu, over);
    if ((threadIdx.x & 31) == 0) {
        if (sq) atomicAdd(&acc->sum_sq, sq);
        if (mx) atomicMax(&acc->max, mx);
        if (over) atomicOr(&acc->overflow, over);
    }
}

// out[0] mean, [1] rel_std, [2] median, [3] max, [4] nempty; [5] 1 if the
// histogram overflowed (then out is not valid).
__global__ void k_stats_final(const int *hist, const StatsAcc *acc, long long nbins, long long n, double *out) {
    if (threadIdx.x != 0) return;
    if (acc->overflow) { out[5] = 1.0; return; }
    const double mean = (double)n / (double)nbins;
    // variance = (nbins sum c^2 - n^2) / nbins^2, the numerator exact in integers
    const __int128 num = (__int128)acc->sum_sq * nbins - (__int128)n * n;
    const double var = (double)num / ((double)nbins * (double)nbins);
    auto kth = [&](long long k) {
        long long cum = 0;
        for (int v = 0; v < STATS_HMAX; ++v) {
            cum += hist[v];
            if (cum > k) return v;
        }
        return STATS_HMAX - 1;
    };
    const double med = (nbins % 2) ? (double)kth(nbins / 2) : 0.5 * ((double)kth(nbins / 2 - 1) + (double)kth(nbins / 2));
    out[0] = mean;
    out[1] = mean > 0 ? sqrt(var > 0 ? var : 0.0) / mean : 0.0;
    out[2] = med;
    out[3] = (double)acc->max;
    out[4] = (double)hist[0];
    out[5] = 0.0;
}

// Self-test of the bounded device wait: one thread waits on a flag nothing
// sets, gives up after `polls` polls and records a timeout.
__global__ void k_selftest_wait(Ctrl *C, const unsigned long long *flag, int polls) {
    const unsigned long long v = spin_until(flag, ~0ull, polls);
    if (!v) C->timeout = 1;
}

template <typename R> __global__ void k_scale_velocities(Dev<R> S, double f) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    const int sp = S.ctrl->state_par, n = S.n;
    S.v[sp][i] *= f;
    S.v[sp][n + i] *= f;
    S.v[sp][2 * n + i] *= f;
}

ljsel_config default_config(const ljsel_params &p) {
    ljsel_config c{};
    c.method = LJSEL_METHOD_VL;
    c.cluster_size = 1;
    c.newton3 = 0;
    c.threads_per_unit = 1;
    c.rebuild_interval = p.skin > 0 ? 10 : 1;
    c.csf = 1.0;
    return c;
}

bool same_cfg(const ljsel_config &a, const ljsel_config &b) {
    return a.method == b.method && a.newton3 == b.newton3 && a.threads_per_unit == b.threads_per_unit &&
           a.rebuild_interval == b.rebuild_interval && a.csf == b.csf &&
           (a.method != LJSEL_METHOD_CLUSTER || a.cluster_size == b.cluster_size);
}

// Two configurations use the same neighbour structure when they differ
// only in lanes per unit or in the rebuild interval: the cell grid, the
// sort and the lists do not depend on either.
bool same_structure(const ljsel_config &a, const ljsel_config &b) {
    if (a.method != b.method || a.csf != b.csf) return false;
    if (a.method == LJSEL_METHOD_LC) return true;
    return a.newton3 == b.newton3 && (a.method != LJSEL_METHOD_CLUSTER || a.cluster_size == b.cluster_size);
}

std::vector<ljsel_config> default_candidates(const System &s) {
    std::vector<ljsel_config> v;
    const int R = s.base_interval;
    auto add = [&](int method, int M, int n3, int t, double csf, int r) {
        ljsel_config c{};
        c.method = method; c.cluster_size = M; c.newton3 = n3; c.threads_per_unit = t; c.csf = csf;
        c.rebuild_interval = s.params.skin > 0 ? r : 1;
        if (validate_config(s, &c) == LJSEL_OK) v.push_back(c);
    };
    for (int n3 = 0; n3 <= 1; ++n3)
        for (double csf : {1.0, 0.5}) add(LJSEL_METHOD_LC, 1, n3, 1, csf, R);
    for (int t : {1, 2, 4, 8}) add(LJSEL_METHOD_VL, 1, 0, t, 1.0, R);
    for (int t : {1, 4}) add(LJSEL_METHOD_VL, 1, 1, t, 1.0, R);
    add(LJSEL_METHOD_VL, 1, 0, 1, 1.0, 2 * R);
    add(LJSEL_METHOD_VL, 1, 0, 2, 1.0, 2 * R);
    // half-side cells: the list build tests about 40 % of the candidates
    for (int t : {1, 2, 4}) add(LJSEL_METHOD_VL, 1, 0, t, 0.5, R);
    add(LJSEL_METHOD_VL, 1, 1, 1, 0.5, R);
    add(LJSEL_METHOD_VL, 1, 0, 2, 0.5, 2 * R);
    for (int n3 = 0; n3 <= 1; ++n3) add(LJSEL_METHOD_VLW, 1, n3, 1, 1.0, R);
    add(LJSEL_METHOD_VLW, 1, 0, 1, 1.0, 2 * R);
    // i-clusters of M particles with union lists: T lanes per cluster
    for (int t : {2, 4, 8}) add(LJSEL_METHOD_CLUSTER, 2, 0, t, 1.0, R);
    for (int t : {4, 8, 16}) add(LJSEL_METHOD_CLUSTER, 4, 0, t, 1.0, R);
    for (int t : {8, 16}) add(LJSEL_METHOD_CLUSTER, 8, 0, t, 1.0, R);
    // with the list rebuilt every 2R steps where displacements allow it
    add(LJSEL_METHOD_CLUSTER, 2, 0, 4, 1.0, 2 * R);
    for (int t : {8, 16}) add(LJSEL_METHOD_CLUSTER, 4, 0, t, 1.0, 2 * R);
    add(LJSEL_METHOD_CLUSTER, 2, 1, 4, 1.0, R);
    add(LJSEL_METHOD_CLUSTER, 4, 1, 8, 1.0, R);
    add(LJSEL_METHOD_CLUSTER, 8, 1, 8, 1.0, R);
    return v;
}

// Random forest (Sec. 5.3): structural checks, then the mean over the trees
// of the class probabilities at the leaf each tree reaches.
ljsel_status forest_check(const ljsel_forest *f) {
    if (!f || f->ntrees < 1 || f->nclasses < 1 || f->nfeatures < 1 || f->nfeatures > 8 || f->nnodes < 1 || !f->root ||
        !f->feature || !f->threshold || !f->left || !f->right || !f->value || !f->classes) {
        set_error("malformed forest: counts or NULL arrays");
        return LJSEL_ERR_ARG;
    }
    for (int t = 0; t < f->ntrees; ++t)
        if (f->root[t] < 0 || f->root[t] >= f->nnodes) { set_error("forest root out of range"); return LJSEL_ERR_ARG; }
    for (int k = 0; k < f->nnodes; ++k) {
        const int ft = f->feature[k];
        if (ft == -1) {
            for (int c = 0; c < f->nclasses; ++c) {
                const double v = f->value[(size_t)k * f->nclasses + c];
                if (!(v >= 0.0) || !std::isfinite(v)) { set_error("forest leaf value negative or not finite"); return LJSEL_ERR_ARG; }
            }
        } else if (ft < 0 || ft >= f->nfeatures || f->left[k] < 0 || f->left[k] >= f->nnodes || f->right[k] < 0 ||
                   f->right[k] >= f->nnodes || !std::isfinite(f->threshold[k])) {
            set_error("forest split node out of range");
            return LJSEL_ERR_ARG;
        }
    }
    return LJSEL_OK;
}
ljsel_status forest_predict(int ntrees, int ncls, int nnodes, const int32_t *root, const int32_t *feature,
                            const double *threshold, const int32_t *left, const int32_t *right, const double *value,
                            const double *x, double *proba) {
    for (int c = 0; c < ncls; ++c) proba[c] = 0.0;
    for (int t = 0; t < ntrees; ++t) {
        int k = root[t];
        int steps = 0;
        while (feature[k] >= 0) {
            k = x[feature[k]] <= threshold[k] ? left[k] : right[k];
            if (++steps > nnodes) { set_error("forest path longer than its nodes (a cycle)"); return LJSEL_ERR_ARG; }
        }
        for (int c = 0; c < ncls; ++c) proba[c] += value[(size_t)k * ncls + c];
    }
    for (int c = 0; c < ncls; ++c) proba[c] /= ntrees;
    return LJSEL_OK;
}

// Trial set of one Predictive phase (Sec. 5.1); see ljsel_predictive_trials.
ljsel_status predictive_trials(int32_t ncand, int32_t phase, const int32_t *hist_n, const int32_t *hist_phase,
                               const double *hist_cost, const int32_t *last_trial_phase, const int32_t *blacklisted,
                               int32_t incumbent, double predict_factor, int32_t retrial_phases, int32_t *trial) {
    if (ncand < 0 || incumbent < -1 || incumbent >= ncand || !(predict_factor > 0)) {
        set_error("invalid argument");
        return LJSEL_ERR_ARG;
    }
    if (ncand > 0 && (!hist_n || !hist_phase || !hist_cost || !last_trial_phase || !blacklisted || !trial)) {
        set_error("NULL array");
        return LJSEL_ERR_ARG;
    }
    for (int k = 0; k < ncand; ++k)
        if (hist_n[k] < 0 || hist_n[k] > 2) { set_error("hist_n must be 0, 1 or 2"); return LJSEL_ERR_ARG; }
    if (phase < 2) {  // the first two phases trial everything
        for (int k = 0; k < ncand; ++k) trial[k] = blacklisted[k] ? 0 : 1;
        return LJSEL_OK;
    }
    std::vector<double> pred(ncand, -1.0);
    double best = 1e300;
    for (int k = 0; k < ncand; ++k) {
        if (blacklisted[k] || hist_n[k] == 0) continue;
        const double cb = hist_cost[2 * k + 1];
        double p = cb;
        if (hist_n[k] == 2) {
            const int pa = hist_phase[2 * k], pb = hist_phase[2 * k + 1];
            const double slope = (cb - hist_cost[2 * k]) / (double)std::max(1, pb - pa);
            p = std::max(cb + slope * (double)(phase - pb), 0.5 * cb);
        }
        pred[k] = p;
        best = std::min(best, p);
    }
    for (int k = 0; k < ncand; ++k) {
        if (blacklisted[k]) { trial[k] = 0; continue; }
        const bool unmeasured = pred[k] < 0;
        const bool near = !unmeasured && pred[k] <= predict_factor * best;
        const bool stale = phase - last_trial_phase[k] >= std::max(1, retrial_phases);
        trial[k] = (unmeasured || near || stale || k == incumbent) ? 1 : 0;
    }
    return LJSEL_OK;
}

}  // namespace

extern "C" {

const char *ljsel_last_error(void) { return last_error(); }

ljsel_status ljsel_forest_predict(const ljsel_forest *f, const double *x, double *proba) {
    set_error("");
    if (!x || !proba) { set_error("NULL argument"); return LJSEL_ERR_ARG; }
    TRY(forest_check(f));
    return forest_predict(f->ntrees, f->nclasses, f->nnodes, f->root, f->feature, f->threshold, f->left, f->right,
                          f->value, x, proba);
}

ljsel_status ljsel_set_forest(ljsel_system h, const ljsel_forest *f) {
    System *s = (System *)h;
    if (!s) { set_error("NULL handle"); return LJSEL_ERR_ARG; }
    set_error("");
    TRY(forest_check(f));
    for (int c = 0; c < f->nclasses; ++c) {
        const ljsel_status st = validate_config(*s, &f->classes[c]);
        if (st != LJSEL_OK) return st;
    }
    Forest &F = s->forest;
    F.ntrees = f->ntrees;
    F.ncls = f->nclasses;
    F.nfeat = f->nfeatures;
    F.nnodes = f->nnodes;
    F.root.assign(f->root, f->root + f->ntrees);
    F.feature.assign(f->feature, f->feature + f->nnodes);
    F.left.assign(f->left, f->left + f->nnodes);
    F.right.assign(f->right, f->right + f->nnodes);
    F.threshold.assign(f->threshold, f->threshold + f->nnodes);
    F.value.assign(f->value, f->value + (size_t)f->nnodes * f->nclasses);
    F.classes.assign(f->classes, f->classes + f->nclasses);
    return LJSEL_OK;
}

ljsel_status ljsel_tuner_costs(ljsel_system h, int32_t cap, ljsel_config *cfgs, double *cost, int32_t *phase,
                               int32_t *count) {
    System *s = (System *)h;
    if (!s || !count || (cap > 0 && (!cfgs || !cost))) { set_error("invalid argument"); return LJSEL_ERR_ARG; }
    int k = 0;
    for (const TunerEntry &e : s->tuner) {
        if (e.history.empty()) continue;
        if (k < cap) {
            cfgs[k] = e.cfg;
            cost[k] = e.history.back().second;
            if (phase) phase[k] = e.history.back().first;
        }
        ++k;
    }
    *count = k;
    return LJSEL_OK;
}

ljsel_status ljsel_predictive_trials(int32_t ncand, int32_t phase, const int32_t *hist_n, const int32_t *hist_phase,
                                     const double *hist_cost, const int32_t *last_trial_phase,
                                     const int32_t *blacklisted, int32_t incumbent, double predict_factor,
                                     int32_t retrial_phases, int32_t *trial) {
    set_error("");
    return predictive_trials(ncand, phase, hist_n, hist_phase, hist_cost, last_trial_phase, blacklisted, incumbent,
                             predict_factor, retrial_phases, trial);
}

ljsel_status ljsel_selftest_wait_timeout(int64_t polls) {
    set_error("");
    if (polls < 1 || polls > (1 << 24)) { set_error("polls must be in [1, 2^24]"); return LJSEL_ERR_ARG; }
    void *mem = nullptr;
    CK(cudaMalloc(&mem, sizeof(Ctrl) + 64));
    Ctrl *C = (Ctrl *)mem;
    unsigned long long *flag = (unsigned long long *)((char *)mem + ((sizeof(Ctrl) + 15) & ~(size_t)15));
    Ctrl h{};
    cudaError_t e = cudaMemset(mem, 0, sizeof(Ctrl) + 64);
    if (e == cudaSuccess) {
        k_selftest_wait<<<1, 1>>>(C, flag, (int)polls);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, C, sizeof(Ctrl), cudaMemcpyDeviceToHost);
    cudaFree(mem);
    if (e != cudaSuccess) { set_error(std::string("self-test failed: ") + cudaGetErrorString(e)); return LJSEL_ERR_CUDA; }
    if (h.timeout) { set_error("a bounded device wait gave up (self-test: nothing sets the flag)"); return LJSEL_ERR_TIMEOUT; }
    return LJSEL_OK;
}
int32_t ljsel_abi_version(void) { return LJSEL_ABI_VERSION; }

ljsel_status ljsel_create(const ljsel_params *params, int64_t n, const double *pos, const double *vel,
                          const int32_t *types, int32_t on_device, void *stream, ljsel_system *out) {
    set_error("");
    if (!out) { set_error("out is NULL"); return LJSEL_ERR_ARG; }
    *out = nullptr;
    TRY(validate_params(params));
    if (n < 1 || n >= (int64_t)JMASK) { set_error("n must be in [1, 2^27)"); return LJSEL_ERR_ARG; }
    if (!pos || !vel) { set_error("pos and vel are required"); return LJSEL_ERR_ARG; }
    System *s = new (std::nothrow) System();
    if (!s) { set_error("host allocation failed"); return LJSEL_ERR_OOM; }
    s->params = *params;
    s->n = (int)n;
    s->precision = params->precision;
    s->stream = (cudaStream_t)stream;
    s->cfg = default_config(*params);
    s->base_interval = s->cfg.rebuild_interval;
    auto fail = [&](ljsel_status st) { delete s; return st; };
    if (cudaHostAlloc((void **)&s->h_ctrl, sizeof(Ctrl), cudaHostAllocDefault) != cudaSuccess) {
        set_error("pinned allocation failed");
        return fail(LJSEL_ERR_CUDA);
    }
    memset(s->h_ctrl, 0, sizeof(Ctrl));
    if (cudaEventCreate(&s->ev_a) != cudaSuccess || cudaEventCreate(&s->ev_b) != cudaSuccess) {
        set_error("event creation failed");
        return fail(LJSEL_ERR_CUDA);
    }
    ljsel_status st = s->alloc_base();
    if (st != LJSEL_OK) return fail(st);
    st = s->apply_config();
    if (st != LJSEL_OK) return fail(st);
    // staging of host inputs (the import kernel checks the types)
    const size_t nb = (size_t)n * 3 * sizeof(double);
    const double *dpos = pos, *dvel = vel;
    const int32_t *dtyp = types;
    if (!on_device) {
        st = s->b_io.ensure(2 * nb + (size_t)n * 4);
        if (st != LJSEL_OK) return fail(st);
        char *io = (char *)s->b_io.ptr;
        if (cudaMemcpyAsync(io, pos, nb, cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
            cudaMemcpyAsync(io + nb, vel, nb, cudaMemcpyHostToDevice, s->stream) != cudaSuccess) {
            set_error("input copy failed");
            return fail(LJSEL_ERR_CUDA);
        }
        dpos = (const double *)io;
        dvel = (const double *)(io + nb);
        if (types) {
            if (cudaMemcpyAsync(io + 2 * nb, types, (size_t)n * 4, cudaMemcpyHostToDevice, s->stream) != cudaSuccess) {
                set_error("input copy failed");
                return fail(LJSEL_ERR_CUDA);
            }
            dtyp = (const int32_t *)(io + 2 * nb);
        }
    }
    auto imp = [&](auto z) -> ljsel_status {
        using R = decltype(z);
        Dev<R> S;
        s->fill_dev(S);
        launch_import_state(S, dpos, dvel, dtyp, 1, s->stream);
        return LJSEL_OK;
    };
    dispatch(s, imp);
    st = s->cmd(CMD_INTERVAL, s->cfg.rebuild_interval);
    if (st == LJSEL_OK) st = s->cmd(CMD_REBUILD, 0);
    if (st == LJSEL_OK) st = s->cmd(CMD_HALF_KICK, 1);
    if (st == LJSEL_OK) st = s->read_ctrl();  // synchronizes
    if (st == LJSEL_OK && s->h_ctrl->bad_type) { set_error("a type is outside [0, ntypes)"); st = LJSEL_ERR_ARG; }
    if (st != LJSEL_OK) return fail(st);
    *out = reinterpret_cast<ljsel_system>(s);
    return LJSEL_OK;
}

ljsel_status ljsel_destroy(ljsel_system h) {
    System *s = (System *)h;
    if (!s) return LJSEL_OK;
    cudaStreamSynchronize(s->stream);
    delete s;
    return LJSEL_OK;
}

ljsel_status ljsel_set_config(ljsel_system h, const ljsel_config *cfg) {
    System *s = (System *)h;
    if (!s) { set_error("NULL handle"); return LJSEL_ERR_ARG; }
    TRY(validate_config(*s, cfg));
    ljsel_config c = *cfg;
    if (c.method != LJSEL_METHOD_CLUSTER) c.cluster_size = 1;
    const ljsel_config old = s->cfg;
    // a built structure that the new configuration shares is kept (the
    // Verlet-list guarantee of Sec. 2.2.1 depends on the positions, not on
    // the lanes per unit or the interval); the new interval applies from
    // the current count of steps since the last rebuild
    const bool keep = !s->structure_dirty && same_structure(old, c);
    s->cfg = c;
    // with N3L the force buffer accumulates and must start at zero; without
    // it a force evaluation leaves its result there
    if (c.newton3 && !old.newton3) {
        TRY(dispatch(s, [&](auto z) -> ljsel_status {
            using R = decltype(z);
            Dev<R> S;
            s->fill_dev(S);
            launch_zero_force(S, s->stream);
            CK(cudaGetLastError());
            return LJSEL_OK;
        }));
    }
    TRY(s->apply_config());
    if (keep) {
        s->structure_dirty = false;
        TRY(s->cmd(CMD_INTERVAL, c.rebuild_interval));
    }
    return LJSEL_OK;
}

ljsel_status ljsel_set_list_capacity(ljsel_system h, int64_t entries) {
    System *s = (System *)h;
    if (!s) { set_error("NULL handle"); return LJSEL_ERR_ARG; }
    if (entries < 4 || entries > 65532) { set_error("entries per row must be in 4 .. 65532"); return LJSEL_ERR_ARG; }
    const int e = (int)entries;
    switch (s->cfg.method) {
        case LJSEL_METHOD_VL: s->nl_cap = (e + 3) & ~3; s->cap_fitted = true; break;
        case LJSEL_METHOD_VLW:
            if (e > 512) { set_error("window-list rows hold at most 512 entries"); return LJSEL_ERR_ARG; }
            s->nl_cap = (e + 15) & ~15;
            break;
        case LJSEL_METHOD_CLUSTER: s->cp_cap = (e + 3) & ~3; break;
        default: set_error("linked cells keep no list"); return LJSEL_ERR_STATE;
    }
    return s->apply_config();
}

ljsel_status ljsel_get_config(ljsel_system h, ljsel_config *cfg) {
    System *s = (System *)h;
    if (!s || !cfg) { set_error("NULL argument"); return LJSEL_ERR_ARG; }
    *cfg = s->cfg;
    return LJSEL_OK;
}

ljsel_status ljsel_rebuild(ljsel_system h) {
    System *s = (System *)h;
    if (!s) { set_error("NULL handle"); return LJSEL_ERR_ARG; }
    s->structure_dirty = true;
    return dispatch(s, [&](auto z) { return s->ensure_structure<decltype(z)>(); });
}

ljsel_status ljsel_compute(ljsel_system h, double *forces, int32_t on_device, double *energy, double *virial) {
    System *s = (System *)h;
    if (!s) { set_error("NULL handle"); return LJSEL_ERR_ARG; }
    return dispatch(s, [&](auto z) -> ljsel_status {
        using R = decltype(z);
        // with neither sum wanted the stepping kernels' force path runs (no
        // energy or virial accumulation)
        const bool ev = energy != nullptr || virial != nullptr;
        TRY(s->compute_forces<R>(ev));
        Dev<R> S;
        s->fill_dev(S);
        if (forces) {
            if (on_device) {
                launch_export_forces(S, forces, s->stream);
            } else {
                TRY(s->b_io.ensure((size_t)s->n * 3 * sizeof(double)));
                launch_export_forces(S, (double *)s->b_io.ptr, s->stream);
                CK(cudaMemcpyAsync(forces, s->b_io.ptr, (size_t)s->n * 3 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
            }
        }
        if (s->cfg.newton3) launch_zero_force(S, s->stream);
        CK(cudaGetLastError());
        TRY(s->read_ctrl());
        TRY(s->check_device_errors());
        if (energy) *energy = s->h_ctrl->epot;
        if (virial) *virial = s->h_ctrl->virial;
        return LJSEL_OK;
    });
}

ljsel_status ljsel_thermostat(ljsel_system h, double target, double max_change, double *t_before) {
    System *s = (System *)h;
    if (!s) { set_error("NULL handle"); return LJSEL_ERR_ARG; }
    if (!(target > 0) || !(max_change >= 0)) { set_error("target > 0 and max_change >= 0 required"); return LJSEL_ERR_ARG; }
    return dispatch(s, [&](auto z) -> ljsel_status {
        using R = decltype(z);
        TRY(s->sync_velocities<R>());
        Dev<R> S;
        s->fill_dev(S);
        TRY(s->cmd(CMD_RESET_EV, 0));
        launch_kinetic(S, s->stream);
        CK(cudaGetLastError());
        TRY(s->read_ctrl());
        const bool walled = s->params.walls[0] || s->params.walls[1] || s->params.walls[2];
        const double dof = walled ? 3.0 * s->n : 3.0 * s->n - 3.0;
        const double T = 2.0 * s->h_ctrl->ekin / dof;
        if (t_before) *t_before = T;
        if (!(T > 0)) return LJSEL_OK;
        double dT = target - T;
        dT = std::max(-max_change, std::min(max_change, dT));
        k_scale_velocities<R><<<div_up(s->n, 256), 256, 0, s->stream>>>(S, std::sqrt((T + dT) / T));
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s->stream));
        return LJSEL_OK;
    });
}

ljsel_status ljsel_step(ljsel_system h, int64_t nsteps) {
    System *s = (System *)h;
    if (!s) { set_error("NULL handle"); return LJSEL_ERR_ARG; }
    if (nsteps < 0) { set_error("nsteps must be >= 0"); return LJSEL_ERR_ARG; }
    return dispatch(s, [&](auto z) { return s->advance<decltype(z)>(nsteps); });
}

ljsel_status ljsel_get_state(ljsel_system h, double *pos, double *vel, int32_t on_device) {
    System *s = (System *)h;
    if (!s) { set_error("NULL handle"); return LJSEL_ERR_ARG; }
    return dispatch(s, [&](auto z) -> ljsel_status {
        using R = decltype(z);
        if (vel) TRY(s->sync_velocities<R>());
        Dev<R> S;
        s->fill_dev(S);
        const size_t nb = (size_t)s->n * 3 * sizeof(double);
        if (on_device) {
            launch_export_state(S, pos, vel, 1, s->stream);
        } else {
            TRY(s->b_io.ensure(2 * nb));
            double *dp = pos ? (double *)s->b_io.ptr : nullptr;
            double *dv = vel ? (double *)((char *)s->b_io.ptr + nb) : nullptr;
            launch_export_state(S, dp, dv, 1, s->stream);
            if (pos) CK(cudaMemcpyAsync(pos, dp, nb, cudaMemcpyDeviceToHost, s->stream));
            if (vel) CK(cudaMemcpyAsync(vel, dv, nb, cudaMemcpyDeviceToHost, s->stream));
        }
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s->stream));
        return LJSEL_OK;
    });
}

ljsel_status ljsel_set_state(ljsel_system h, const double *pos, const double *vel, int32_t on_device) {
    System *s = (System *)h;
    if (!s) { set_error("NULL handle"); return LJSEL_ERR_ARG; }
    return dispatch(s, [&](auto z) -> ljsel_status {
        using R = decltype(z);
        const size_t nb = (size_t)s->n * 3 * sizeof(double);
        const double *dp = pos, *dv = vel;
        if (!on_device) {
            TRY(s->b_io.ensure(2 * nb));
            if (pos) { CK(cudaMemcpyAsync(s->b_io.ptr, pos, nb, cudaMemcpyHostToDevice, s->stream)); dp = (const double *)s->b_io.ptr; }
            if (vel) { CK(cudaMemcpyAsync((char *)s->b_io.ptr + nb, vel, nb, cudaMemcpyHostToDevice, s->stream)); dv = (const double *)((char *)s->b_io.ptr + nb); }
        }
        Dev<R> S;
        s->fill_dev(S);
        launch_import_state(S, dp, dv, nullptr, 0, s->stream);
        TRY(s->cmd(CMD_REBUILD, 0));
        TRY(s->cmd(CMD_HALF_KICK, 1));
        s->synced = true;
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s->stream));
        return LJSEL_OK;
    });
}

ljsel_status ljsel_move_particles(ljsel_system h, const double *pos, int32_t on_device) {
    System *s = (System *)h;
    if (!s || !pos) { set_error("NULL argument"); return LJSEL_ERR_ARG; }
    return dispatch(s, [&](auto z) -> ljsel_status {
        using R = decltype(z);
        const size_t nb = (size_t)s->n * 3 * sizeof(double);
        const double *dp = pos;
        if (!on_device) {
            TRY(s->b_io.ensure(nb));
            CK(cudaMemcpyAsync(s->b_io.ptr, pos, nb, cudaMemcpyHostToDevice, s->stream));
            dp = (const double *)s->b_io.ptr;
        }
        Dev<R> S;
        s->fill_dev(S);
        launch_move_particles(S, dp, s->stream);
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s->stream));
        return LJSEL_OK;
    });
}

ljsel_status ljsel_get_work_positions(ljsel_system h, double *pos, int32_t on_device) {
    System *s = (System *)h;
    if (!s || !pos) { set_error("NULL argument"); return LJSEL_ERR_ARG; }
    return dispatch(s, [&](auto z) -> ljsel_status {
        using R = decltype(z);
        Dev<R> S;
        s->fill_dev(S);
        const size_t nb = (size_t)s->n * 3 * sizeof(double);
        if (on_device) {
            launch_export_work_pos(S, pos, s->stream);
        } else {
            TRY(s->b_io.ensure(nb));
            launch_export_work_pos(S, (double *)s->b_io.ptr, s->stream);
            CK(cudaMemcpyAsync(pos, s->b_io.ptr, nb, cudaMemcpyDeviceToHost, s->stream));
        }
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s->stream));
        return LJSEL_OK;
    });
}

ljsel_status ljsel_get_pairs(ljsel_system h, int64_t cap, int32_t *ij, int64_t *count) {
    System *s = (System *)h;
    if (!s || !count || cap < 0 || (cap > 0 && !ij)) { set_error("invalid argument"); return LJSEL_ERR_ARG; }
    return dispatch(s, [&](auto z) -> ljsel_status {
        using R = decltype(z);
        TRY(s->ensure_structure<R>());
        Dev<R> S;
        s->fill_dev(S);
        int2 *buf = nullptr;
        if (cap > 0) CK(cudaMalloc(&buf, (size_t)cap * sizeof(int2)));
        TRY(s->cmd(CMD_RESET_PAIRS, 0));
        launch_force(S, s->cfg, MODE_PAIRS, false, buf, cap, s->stream);
        cudaError_t e = cudaGetLastError();
        ljsel_status st = LJSEL_OK;
        if (e == cudaSuccess) st = s->read_ctrl();
        long long got = (long long)s->h_ctrl->npairs;
        if (e == cudaSuccess && st == LJSEL_OK && cap > 0)
            e = cudaMemcpy(ij, buf, (size_t)std::min<long long>(got, cap) * sizeof(int2), cudaMemcpyDeviceToHost);
        if (buf) cudaFree(buf);
        if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return LJSEL_ERR_CUDA; }
        if (st != LJSEL_OK) return st;
        *count = got;
        return LJSEL_OK;
    });
}

ljsel_status ljsel_get_energy(ljsel_system h, double *epot, double *ekin, double *virial) {
    System *s = (System *)h;
    if (!s) { set_error("NULL handle"); return LJSEL_ERR_ARG; }
    return dispatch(s, [&](auto z) -> ljsel_status {
        using R = decltype(z);
        TRY(s->sync_velocities<R>());
        TRY(s->compute_forces<R>(true));
        Dev<R> S;
        s->fill_dev(S);
        launch_kinetic(S, s->stream);
        if (s->cfg.newton3) launch_zero_force(S, s->stream);
        CK(cudaGetLastError());
        TRY(s->read_ctrl());
        TRY(s->check_device_errors());
        if (epot) *epot = s->h_ctrl->epot;
        if (ekin) *ekin = s->h_ctrl->ekin;
        if (virial) *virial = s->h_ctrl->virial;
        return LJSEL_OK;
    });
}

ljsel_status ljsel_get_stats(ljsel_system h, ljsel_stats *st) {
    System *s = (System *)h;
    if (!s || !st) { set_error("NULL argument"); return LJSEL_ERR_ARG; }
    double rcm = 0;
    for (int t = 0; t < s->params.ntypes * s->params.ntypes; ++t) rcm = std::max(rcm, s->params.rcut[t]);
    const double bin_min = rcm + s->params.skin;
    BinGrid g;
    long long nbins = 1;
    for (int d = 0; d < 3; ++d) {
        g.nb[d] = std::max(1, (int)std::floor(s->params.box[d] / bin_min));
        g.side[d] = s->params.box[d] / g.nb[d];
        nbins *= g.nb[d];
    }
    // device buffer: counts | histogram | accumulators | results
    const size_t cbytes = ((size_t)nbins * 4 + 255) & ~(size_t)255;
    const size_t hbytes = (size_t)STATS_HMAX * 4;
    TRY(s->b_stats.ensure(cbytes + hbytes + 256 + 64));
    int *counts = (int *)s->b_stats.ptr;
    int *hist = (int *)((char *)s->b_stats.ptr + cbytes);
    StatsAcc *acc = (StatsAcc *)((char *)s->b_stats.ptr + cbytes + hbytes);
    double *dres = (double *)((char *)s->b_stats.ptr + cbytes + hbytes + 256);
    const size_t hneed = std::max<size_t>(64, (size_t)nbins * 4);
    if (s->h_stats_cap * 4 < hneed) {
        if (s->h_stats) cudaFreeHost(s->h_stats);
        s->h_stats = nullptr;
        s->h_stats_cap = 0;
        CK(cudaMallocHost((void **)&s->h_stats, hneed));
        s->h_stats_cap = hneed / 4;
    }
    CK(cudaMemsetAsync(s->b_stats.ptr, 0, cbytes + hbytes + 256, s->stream));
    ljsel_status rs = dispatch(s, [&](auto z) -> ljsel_status {
        using R = decltype(z);
        Dev<R> S;
        s->fill_dev(S);
        k_stats_bin<R><<<div_up(s->n, 256), 256, 0, s->stream>>>(S, g, counts);
        return LJSEL_OK;
    });
    if (rs != LJSEL_OK) return rs;
    k_stats_hist<<<(int)std::min<long long>(div_up(nbins, 256), 1024), 256, 0, s->stream>>>(counts, nbins, hist, acc);
    k_stats_final<<<1, 32, 0, s->stream>>>(hist, acc, nbins, s->n, dres);
    CK(cudaGetLastError());
    double *hres = (double *)s->h_stats;
    CK(cudaMemcpyAsync(hres, dres, 6 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    double mean = hres[0], rel_std = hres[1], median = hres[2], mx = hres[3], nempty = hres[4];
    if (hres[5] != 0.0) {
        // a count of STATS_HMAX or more: every count to the host, the median
        // by selection on a copy
        const int *hc = s->h_stats;
        CK(cudaMemcpyAsync(s->h_stats, counts, nbins * 4, cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        mean = (double)s->n / (double)nbins;
        double var = 0;
        int m = 0;
        long long ne = 0;
        for (long long b = 0; b < nbins; ++b) {
            const double d = hc[b] - mean;
            var += d * d;
            m = std::max(m, hc[b]);
            ne += hc[b] == 0;
        }
        var /= (double)nbins;
        std::vector<int> copy(hc, hc + nbins);
        auto kth = [&](long long k) {
            std::nth_element(copy.begin(), copy.begin() + k, copy.end());
            return copy[k];
        };
        median = (nbins % 2) ? (double)kth(nbins / 2) : 0.5 * ((double)kth(nbins / 2 - 1) + (double)kth(nbins / 2));
        rel_std = mean > 0 ? std::sqrt(var) / mean : 0.0;
        mx = m;
        nempty = (double)ne;
    }
    st->mean = mean;
    st->rel_std = rel_std;
    st->median = median;
    st->max = mx;
    st->nbins = (double)nbins;
    st->nempty = nempty;
    st->skin = s->params.skin;
    // the counterpart of the paper's thread count: the threads the GPU keeps
    // resident (SMs x threads per SM), a property of the device, not of the
    // configuration in use
    int dev = 0, per_sm = 0, nsm = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    st->threads = (double)nsm * (double)per_sm;
    return LJSEL_OK;
}

ljsel_status ljsel_get_counters(ljsel_system h, ljsel_counters *c) {
    System *s = (System *)h;
    if (!s || !c) { set_error("NULL argument"); return LJSEL_ERR_ARG; }
    TRY(s->read_ctrl());
    memset(c, 0, sizeof(*c));
    c->steps = s->h_ctrl->total_steps;
    c->rebuilds = s->h_ctrl->rebuilds;
    c->early_rebuilds = s->h_ctrl->early_rebuilds;
    c->ncells = s->ncell;
    c->capacity_retries = s->capacity_retries;
    if (s->cfg.method == LJSEL_METHOD_VL || s->cfg.method == LJSEL_METHOD_VLW) {
        c->list_capacity = (int64_t)s->nl_cap * s->n;  // row-major, nl_cap per particle
        c->list_entries = s->h_ctrl->list_entries;
        c->longest_row = s->h_ctrl->need_cap;
    } else if (s->cfg.method == LJSEL_METHOD_CLUSTER) {
        int ncl = 0;
        CK(cudaMemcpy(&ncl, s->b_ncl.ptr, 4, cudaMemcpyDeviceToHost));
        c->nclusters = ncl;
        c->list_capacity = (int64_t)s->cp_cap * ncl;
        c->list_entries = s->h_ctrl->list_entries;
        c->longest_row = s->h_ctrl->need_cap;
    }
    return LJSEL_OK;
}

ljsel_status ljsel_profile_steps(ljsel_system h, int64_t nsteps, ljsel_profile *out) {
    System *s = (System *)h;
    if (!s || !out || nsteps < 0) { set_error("invalid argument"); return LJSEL_ERR_ARG; }
    return dispatch(s, [&](auto z) { return s->profile<decltype(z)>(nsteps, out); });
}

ljsel_status ljsel_default_candidates(ljsel_system h, int32_t cap, ljsel_config *out, int32_t *count) {
    System *s = (System *)h;
    if (!s || !count || (cap > 0 && !out)) { set_error("invalid argument"); return LJSEL_ERR_ARG; }
    std::vector<ljsel_config> v = default_candidates(*s);
    for (int k = 0; k < (int)v.size() && k < cap; ++k) out[k] = v[k];
    *count = (int32_t)v.size();
    return LJSEL_OK;
}

// ---------------------------------------------------------------------------
// Expert strategy (Sec. 5.2): a fuzzy system whose single input is the mean
// number of particles per CSF-1 cell bin (a Sec. 4 statistic) rates each
// configuration family Good / Okay / Bad; the crisp suitability is the
// centre of gravity of the aggregated output set (Sec. 2.3), and only
// configurations rated at least 0.5 are trialled.  The paper's rule file is
// not available; these rules are ours, written from the full searches of
// the 42 Random Forest training scenarios on this GPU: a Verlet-list
// variant is fastest or within 18 % in every one; cluster lists win or come
// within 1-14 % from about 4 particles per bin up and lose by 10-40 % below;
// window lists (1.2x and more) and linked cells (1.3x and more) never win.
struct Trap {
    double a, b, c, d;  // 0 below a, rising to 1 at b, 1 until c, 0 from d
    double operator()(double x) const {
        if (x < a || x > d) return 0.0;
        if (x < b) return b > a ? (x - a) / (b - a) : 1.0;
        if (x <= c) return 1.0;
        return d > c ? (d - x) / (d - c) : 1.0;
    }
};
static const double INF = 1e300;
static const Trap IN_SPARSE = {-INF, -INF, 1.0, 4.0}, IN_MEDIUM = {1.0, 4.0, 8.0, 12.0}, IN_DENSE = {8.0, 12.0, INF, INF};
static const Trap OUT_BAD = {-INF, -INF, 0.1, 0.4}, OUT_OKAY = {0.2, 0.5, 0.5, 0.8}, OUT_GOOD = {0.6, 0.9, INF, INF};

// consequent term per (family, input term): 0 bad, 1 okay, 2 good
static int expert_rule(const ljsel_config &c, int input_term) {
    static const int VL_[3] = {2, 2, 2}, VLW_[3] = {0, 0, 0}, LC_[3] = {0, 0, 0}, CL_[3] = {0, 1, 1};
    switch (c.method) {
        case LJSEL_METHOD_VL: return VL_[input_term];
        case LJSEL_METHOD_VLW: return VLW_[input_term];
        case LJSEL_METHOD_LC: return LC_[input_term];
        default: return CL_[input_term];
    }
}

static double expert_suitability(const ljsel_config &c, double mean_per_bin) {
    const double w[3] = {IN_SPARSE(mean_per_bin), IN_MEDIUM(mean_per_bin), IN_DENSE(mean_per_bin)};
    const Trap *out[3] = {&OUT_BAD, &OUT_OKAY, &OUT_GOOD};
    double num = 0.0, den = 0.0;
    for (int k = 0; k <= 200; ++k) {
        const double y = k / 200.0;
        double m = 0.0;
        for (int t = 0; t < 3; ++t) m = std::max(m, std::min(w[t], (*out[expert_rule(c, t)])(y)));
        num += m * y;
        den += m;
    }
    return den > 0 ? num / den : 0.0;
}

ljsel_status ljsel_expert_suitability(const ljsel_config *c, double mean_per_bin, double *out) {
    if (!c || !out || !std::isfinite(mean_per_bin)) { set_error("NULL argument or non-finite input"); return LJSEL_ERR_ARG; }
    if (c->method < 0 || c->method > 3) { set_error("unknown method"); return LJSEL_ERR_ARG; }
    *out = expert_suitability(*c, mean_per_bin);
    return LJSEL_OK;
}

// One tuning phase.  Candidates are trialled in the order of their last
// measured cost.  Each trial selects the configuration, builds its
// neighbour structure (timed), then advances opts->trial_steps steps
// (timed); cost per step = build time / R' + step time / trial_steps, the
// weighted average of build and force time of Sec. 2.2.5, with R' = R, or
// min(R, the interval observed since the last phase) when displacements
// forced most of its rebuilds (see i_obs below).  Trials advance the
// simulation (Sec. 1).  With probe_steps > 0 a trial whose first probe_steps
// steps already cost more than probe_factor x the best cost of the phase
// stops there.  Predictive strategy (Sec. 5.1): after two phases a config is
// trialled only if its cost, extrapolated linearly from its last two
// measurements, is within predict_factor of the best prediction, or if it
// has not been trialled for retrial_phases phases; configs measured slower
// than blacklist_factor x the best are dropped for good.  Expert strategy:
// see expert_suitability.
ljsel_status ljsel_autotune(ljsel_system h, const ljsel_tuner_opts *opts, ljsel_config *chosen,
                            ljsel_tuner_report *report) {
    System *s = (System *)h;
    if (!s || !opts) { set_error("NULL argument"); return LJSEL_ERR_ARG; }
    if (opts->trial_steps < 1 || opts->strategy < 0 || opts->strategy > 3 || opts->probe_steps < 0 ||
        opts->forest_top < 0) {
        set_error("invalid tuner options");
        return LJSEL_ERR_ARG;
    }
    if (opts->strategy == 3 && s->forest.ntrees == 0) {
        set_error("the random forest strategy needs a forest (ljsel_set_forest)");
        return LJSEL_ERR_STATE;
    }
    auto t0 = std::chrono::steady_clock::now();
    if (!(opts->skip_within >= 0)) { set_error("skip_within must be >= 0"); return LJSEL_ERR_ARG; }
    // live statistics: the expert input, and the test for skipping a phase
    ljsel_stats st_now{};
    const bool need_stats = opts->strategy == 2 || opts->strategy == 3 || opts->skip_within > 0;
    if (need_stats) TRY(ljsel_get_stats(h, &st_now));
    if (opts->skip_within > 0 && s->have_tuned_stats) {
        auto close = [&](double a, double b) { return std::fabs(a - b) <= opts->skip_within * std::max(std::fabs(b), 1e-12); };
        const ljsel_stats &o = s->tuned_stats;
        if (close(st_now.mean, o.mean) && close(st_now.rel_std, o.rel_std) && close(st_now.max, o.max)) {
            ljsel_tuner_report r = s->last_report;
            r.phase = s->tuner_phase;
            r.ntrialled = 0;
            r.nprobed_out = 0;
            r.overhead_ms = 0;
            r.trial_steps_total = 0;
            r.skipped = 1;
            r.phase_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            s->last_report = r;
            if (chosen) *chosen = s->cfg;
            if (report) *report = r;
            return LJSEL_OK;
        }
    }
    // the rebuild interval the displacements allowed since the last phase
    // (Sec. 2.2.1): when most rebuilds of that window came early (a particle
    // reached skin/2 before R steps), a config's longer R would not space
    // its builds further apart, so the build time of Sec. 2.2.5's weighted
    // cost is divided by min(R, observed interval) instead of R
    TRY(s->read_ctrl());
    double i_obs = 0.0;
    {
        const long long ds = s->h_ctrl->total_steps - s->tune_steps0, dr = s->h_ctrl->rebuilds - s->tune_rebuilds0,
                        de = s->h_ctrl->early_rebuilds - s->tune_early0;
        if (ds >= 20 && dr > 0 && 2 * de >= dr) i_obs = (double)ds / (double)dr;
    }
    auto weight = [&](int R) { return i_obs > 0.0 ? std::min((double)R, i_obs) : (double)R; };
    // the next window starts when this phase ends
    auto end_window = [&]() -> ljsel_status {
        TRY(s->read_ctrl());
        s->tune_steps0 = s->h_ctrl->total_steps;
        s->tune_rebuilds0 = s->h_ctrl->rebuilds;
        s->tune_early0 = s->h_ctrl->early_rebuilds;
        return LJSEL_OK;
    };
    std::vector<ljsel_config> cands;
    if (opts->strategy == 3) {
        cands = s->forest.classes;  // the forest ranks its own classes
    } else if (opts->ncandidates > 0) {
        if (!opts->candidates) { set_error("candidates is NULL"); return LJSEL_ERR_ARG; }
        for (int k = 0; k < opts->ncandidates; ++k) {
            TRY(validate_config(*s, &opts->candidates[k]));
            cands.push_back(opts->candidates[k]);
        }
    } else {
        cands = default_candidates(*s);
    }
    for (const ljsel_config &c : cands) {
        bool found = false;
        for (TunerEntry &e : s->tuner) found = found || same_cfg(e.cfg, c);
        if (!found) s->tuner.push_back(TunerEntry{c, {}, -1, false});
    }
    std::vector<TunerEntry *> ent(cands.size(), nullptr);
    for (size_t k = 0; k < cands.size(); ++k)
        for (TunerEntry &e : s->tuner)
            if (same_cfg(e.cfg, cands[k])) ent[k] = &e;
    const int phase = s->tuner_phase;
    // which candidates to trial
    std::vector<char> trial(cands.size(), 1);
    double expert_x = -1.0;
    if (opts->strategy == 2) {
        const ljsel_stats &st = st_now;
        expert_x = st.mean;
        int any = 0;
        for (size_t k = 0; k < cands.size(); ++k) {
            // suitability >= 0.5 (an "okay" alone has centroid 0.5 up to rounding)
            trial[k] = !ent[k]->blacklisted && expert_suitability(cands[k], st.mean) >= 0.5 - 1e-9;
            any += trial[k];
        }
        if (!any)
            for (size_t k = 0; k < cands.size(); ++k) trial[k] = !ent[k]->blacklisted;
    } else if (opts->strategy == 3) {
        // Random Forest (Sec. 5.3): class probabilities from the Sec. 4
        // statistics; the forest_top most probable classes are trialled
        const Forest &F = s->forest;
        const double x[8] = {st_now.mean, st_now.rel_std, st_now.median, st_now.max,
                             st_now.nbins, st_now.nempty, st_now.skin, st_now.threads};
        std::vector<double> proba(F.ncls, 0.0);
        TRY(forest_predict(F.ntrees, F.ncls, F.nnodes, F.root.data(), F.feature.data(), F.threshold.data(),
                           F.left.data(), F.right.data(), F.value.data(), x, proba.data()));
        std::vector<int> rank(F.ncls);
        for (int c = 0; c < F.ncls; ++c) rank[c] = c;
        std::stable_sort(rank.begin(), rank.end(), [&](int a, int b) { return proba[a] > proba[b]; });
        const int top = std::max(1, opts->forest_top);
        for (size_t k = 0; k < cands.size(); ++k) trial[k] = 0;
        int taken = 0;
        for (int r = 0; r < F.ncls && taken < top; ++r) {
            if (ent[rank[r]]->blacklisted) continue;
            trial[rank[r]] = 1;
            ++taken;
        }
        if (!taken) trial[rank[0]] = 1;  // everything blacklisted: keep the forest's first choice
        expert_x = proba[rank[0]];
        // one suggestion (the paper's forest suggests a configuration): it is
        // selected without a trial, keeping the neighbour structure when the
        // configuration in use shares it
        if (top == 1) {
            const int k = rank[0];
            if (!same_cfg(cands[k], s->cfg)) {
                ljsel_status sc = ljsel_set_config(h, &cands[k]);
                if (sc != LJSEL_OK) return sc;
            }
            ljsel_tuner_report r{};
            s->tuner_phase += 1;
            r.phase = s->tuner_phase;
            r.chosen_index = k;
            const auto &hs = ent[k]->history;
            r.chosen_cost_ms = hs.empty() ? 0.0 : hs.back().second;
            r.expert_input = expert_x;
            r.rebuild_every = i_obs;
            TRY(end_window());
            r.phase_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
            s->tuned_stats = st_now;
            s->have_tuned_stats = true;
            s->last_report = r;
            if (chosen) *chosen = s->cfg;
            if (report) *report = r;
            return LJSEL_OK;
        }
    } else if (opts->strategy == 1) {
        const int nc = (int)cands.size();
        std::vector<int32_t> hn(nc), hp(2 * nc, 0), lt(nc), bl(nc), tr(nc);
        std::vector<double> hc(2 * nc, 0.0);
        int incumbent = -1;
        for (int k = 0; k < nc; ++k) {
            const auto &hs = ent[k]->history;
            hn[k] = (int32_t)std::min<size_t>(2, hs.size());
            for (int q = 0; q < hn[k]; ++q) {
                const auto &e = hs[hs.size() - hn[k] + q];
                const int slot = 2 * k + (hn[k] == 1 ? 1 : q);
                hp[slot] = e.first;
                hc[slot] = e.second;
            }
            lt[k] = ent[k]->last_trial_phase;
            bl[k] = ent[k]->blacklisted ? 1 : 0;
            if (incumbent < 0 && same_cfg(cands[k], s->cfg)) incumbent = k;
        }
        TRY(predictive_trials(nc, phase, hn.data(), hp.data(), hc.data(), lt.data(), bl.data(), incumbent,
                              opts->predict_factor, opts->retrial_phases, tr.data()));
        for (int k = 0; k < nc; ++k) trial[k] = (char)tr[k];
    } else {
        for (size_t k = 0; k < cands.size(); ++k) trial[k] = !ent[k]->blacklisted;
    }
    // trial order: last measured cost ascending, unmeasured ones in set order
    std::vector<size_t> order(cands.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) {
        const bool hx = !ent[x]->history.empty(), hy = !ent[y]->history.empty();
        if (hx != hy) return hx;
        if (!hx) return false;
        return ent[x]->history.back().second < ent[y]->history.back().second;
    });
    std::vector<double> cost(cands.size(), -1.0);
    std::vector<char> probed_out(cands.size(), 0);
    int best_k = -1;
    long long steps_total = 0;
    for (size_t oi = 0; oi < order.size(); ++oi) {
        const size_t k = order[oi];
        if (!trial[k]) continue;
        ljsel_status sc = ljsel_set_config(h, &cands[k]);
        if (sc == LJSEL_ERR_UNSUPPORTED) { ent[k]->blacklisted = true; continue; }
        TRY(sc);
        // every trial builds its own structure, so that the trials' costs
        // compare (a shared structure would reach later trials aged)
        s->structure_dirty = true;
        int done_steps = 0;
        ljsel_status st = dispatch(s, [&](auto z) -> ljsel_status {
            using R = decltype(z);
            float tb = 0, tp = 0, tr = 0, te = 0;
            // timed build (ensure_structure synchronizes; subtract one empty round trip)
            CK(cudaEventRecord(s->ev_a, s->stream));
            TRY(s->ensure_structure<R>());
            CK(cudaEventRecord(s->ev_b, s->stream));
            CK(cudaEventSynchronize(s->ev_b));
            CK(cudaEventElapsedTime(&tb, s->ev_a, s->ev_b));
            CK(cudaEventRecord(s->ev_a, s->stream));
            TRY(s->read_ctrl());
            CK(cudaEventRecord(s->ev_b, s->stream));
            CK(cudaEventSynchronize(s->ev_b));
            CK(cudaEventElapsedTime(&te, s->ev_a, s->ev_b));
            tb = std::max(0.f, tb - te);
            // trials use plain stream launches: instantiating a step graph
            // per candidate would cost more than the trial itself
            const double R_ = weight(std::max(1, cands[k].rebuild_interval));
            int probe = opts->probe_steps > 0 ? std::min(opts->probe_steps, opts->trial_steps) : opts->trial_steps;
            CK(cudaEventRecord(s->ev_a, s->stream));
            TRY(s->advance<R>(probe, true));
            CK(cudaEventRecord(s->ev_b, s->stream));
            CK(cudaEventSynchronize(s->ev_b));
            CK(cudaEventElapsedTime(&tp, s->ev_a, s->ev_b));
            done_steps = probe;
            const double probe_cost = tb / R_ + tp / probe;
            if (probe < opts->trial_steps && best_k >= 0 && probe_cost > opts->probe_factor * cost[best_k]) {
                cost[k] = probe_cost;
                probed_out[k] = 1;
                return LJSEL_OK;
            }
            if (probe < opts->trial_steps) {
                CK(cudaEventRecord(s->ev_a, s->stream));
                TRY(s->advance<R>(opts->trial_steps - probe, true));
                CK(cudaEventRecord(s->ev_b, s->stream));
                CK(cudaEventSynchronize(s->ev_b));
                CK(cudaEventElapsedTime(&tr, s->ev_a, s->ev_b));
                done_steps = opts->trial_steps;
            }
            cost[k] = tb / R_ + (tp + tr) / opts->trial_steps;
            return LJSEL_OK;
        });
        if (st == LJSEL_ERR_UNSUPPORTED) { ent[k]->blacklisted = true; continue; }
        if (st != LJSEL_OK) return st;
        steps_total += done_steps;
        ent[k]->history.push_back({phase, cost[k]});
        if (ent[k]->history.size() > 8) ent[k]->history.erase(ent[k]->history.begin());
        ent[k]->last_trial_phase = phase;
        if (best_k < 0 || cost[k] < cost[best_k]) best_k = (int)k;
    }
    if (best_k < 0) { set_error("no candidate could be trialled"); return LJSEL_ERR_STATE; }
    int nbl = 0, ntr = 0, npo = 0;
    double overhead = 0;
    for (size_t k = 0; k < cands.size(); ++k) {
        if (cost[k] < 0) continue;
        ++ntr;
        npo += probed_out[k];
        const int steps_k = probed_out[k] ? std::min(opts->probe_steps, opts->trial_steps) : opts->trial_steps;
        overhead += (cost[k] - cost[best_k]) * steps_k;
        if (opts->blacklist_factor > 0 && cost[k] > opts->blacklist_factor * cost[best_k]) ent[k]->blacklisted = true;
    }
    for (auto *e : ent) nbl += e->blacklisted;
    TRY(ljsel_set_config(h, &cands[best_k]));
    TRY(end_window());
    s->tuner_phase += 1;
    if (need_stats) {
        s->tuned_stats = st_now;
        s->have_tuned_stats = true;
    }
    auto t1 = std::chrono::steady_clock::now();
    ljsel_tuner_report r{};
    r.phase = s->tuner_phase;
    r.ntrialled = ntr;
    r.nblacklisted = nbl;
    r.chosen_index = best_k;
    r.chosen_cost_ms = cost[best_k];
    r.phase_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
    r.overhead_ms = overhead;
    r.trial_steps_total = steps_total;
    r.nprobed_out = npo;
    r.expert_input = expert_x;
    r.rebuild_every = i_obs;
    s->last_report = r;
    if (chosen) *chosen = cands[best_k];
    if (report) *report = r;
    return LJSEL_OK;
}

}  // extern "C"
