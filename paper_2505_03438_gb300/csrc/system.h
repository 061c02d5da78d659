// system.h -- host-side state of one particle system (behind ljsel_system).
#pragma once

#include <string>
#include <vector>

#include "ljsel_internal.cuh"

namespace ljsel {

void set_error(const std::string &m);
const char *last_error();

struct Buf {
    void *ptr = nullptr;
    size_t size = 0;
    ljsel_status ensure(size_t bytes);
    void release();
};

ljsel_status validate_params(const ljsel_params *p);

// Per-configuration memory of the predictive tuning strategy (Sec. 5.1).
struct TunerEntry {
    ljsel_config cfg;
    std::vector<std::pair<int, double>> history;  // (phase, cost ms/step)
    int last_trial_phase = -1;
    bool blacklisted = false;
};

// A random-forest classifier installed for the Random Forest strategy
// (Sec. 5.3), copied from a caller's ljsel_forest.
struct Forest {
    int ntrees = 0, ncls = 0, nfeat = 0, nnodes = 0;
    std::vector<int32_t> root, feature, left, right;
    std::vector<double> threshold, value;
    std::vector<ljsel_config> classes;
};

// One instantiated step graph, valid for exactly the configuration and
// device layout (the bytes of the kernel-parameter block) it was built for.
struct GraphEntry {
    ljsel_config cfg;
    std::vector<unsigned char> key;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

struct System {
    ljsel_params params{};
    int n = 0;
    int precision = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream used only to capture graphs
    ljsel_config cfg{};
    int base_interval = 10;  // rebuild interval the default candidates start from
    // grid
    int nc[3] = {1, 1, 1};
    double side[3] = {1, 1, 1};
    int ncell = 1;
    int reach = 1;
    double rlist = 0;
    int M = 1;
    // list capacities
    int nl_cap = 0;
    int ncl_cap = 0, cp_cap = 0;
    long long capacity_retries = 0;
    bool cap_fitted = false;  // the Verlet-list row capacity was fitted to a build
    bool structure_dirty = true;
    bool synced = true;  // velocities at the integer step
    // device buffers
    Buf b_x[2], b_v[2], b_id[2], b_type[2], b_pos[2];
    Buf b_xref, b_force;
    Buf b_cell_count, b_cell_start, b_clcell_start, b_cell_of, b_slot_of, b_key_of, b_tmp_idx, b_tmp_key,
        b_cell_sorted, b_scan;
    Buf b_nl, b_nl_count, b_strips, b_nstrips;
    Buf b_cl_first, b_cl_count, b_cl_cell, b_cp, b_cp_count, b_ncl;
    Buf b_ctrl, b_io;
    // gradients: sorted cotangent, caller-order adjoint state, parameter
    // sums, rollout checkpoints and the recomputed segment
    Buf b_adj_cot, b_adj_x, b_adj_v, b_adj_theta, b_ckpt, b_seg;
    struct Rollout {
        long long nsteps = -1, every = 0;
        ljsel_config cfg{};
        ljsel_params params{};
    } rollout;
    Ctrl *h_ctrl = nullptr;  // pinned mirror
    // live statistics: positions and bin counts on the device, the counts'
    // pinned host copy (kept between calls: a tuning phase reads them)
    Buf b_stats;
    int *h_stats = nullptr;
    size_t h_stats_cap = 0;
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    // step graphs, one per (configuration, device layout); gexec is the
    // current configuration's
    std::vector<GraphEntry> gcache;
    cudaGraphExec_t gexec = nullptr;
    // tuner state
    std::vector<TunerEntry> tuner;
    int tuner_phase = 0;
    // counters at the end of the last tuning phase: the window over which the
    // next phase observes the rebuild interval
    long long tune_steps0 = 0, tune_rebuilds0 = 0, tune_early0 = 0;
    Forest forest;  // Random Forest strategy (empty until ljsel_set_forest)
    ljsel_tuner_report last_report{};
    bool have_tuned_stats = false;
    ljsel_stats tuned_stats{};  // live statistics at the last phase that ran trials

    ~System();
    std::vector<Buf *> all_bufs();
    void drop_graph();
    size_t p4() const;
    void plan_grid();
    ljsel_status alloc_base();
    ljsel_status apply_config();
    ljsel_status cmd(int op, long long a);
    ljsel_status read_ctrl();
    ljsel_status check_device_errors();
    ljsel_status handle_overflow();
    template <typename R> void fill_dev(Dev<R> &S) const;
    template <typename R> void enqueue_rebuild(const Dev<R> &S, cudaStream_t st);
    template <typename R> void enqueue_step(const Dev<R> &S, bool ev, cudaStream_t st);
    template <typename R> ljsel_status ensure_structure();
    template <typename R> ljsel_status build_graph();
    template <typename R> ljsel_status ensure_graph();
    template <typename R> ljsel_status advance(long long nsteps, bool eager = false);
    template <typename R> ljsel_status compute_forces(bool ev);
    template <typename R> ljsel_status sync_velocities();
    template <typename R> ljsel_status profile(long long nsteps, ljsel_profile *out);
};

ljsel_status validate_config(const System &s, const ljsel_config *c);

enum { CMD_REBUILD = 1, CMD_BEGIN = 2, CMD_RESET_EV = 3, CMD_RESET_PAIRS = 4, CMD_HALF_KICK = 5, CMD_CLEAR = 6,
       CMD_INTERVAL = 7 };

}  // namespace ljsel
