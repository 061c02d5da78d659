/*
 * ljsel.h -- C ABI of the GB300 library for short-range Lennard-Jones
 * molecular dynamics with run-time configuration selection, after
 * "Algorithm Selection in Short-Range Molecular Dynamics Simulations"
 * (arXiv 2505.03438).
 *
 * The paper describes a black-box particle container that a cutoff
 * simulator drives (Sec. 2.2), which rebuilds its neighbour structure
 * (Sec. 2.2.1), evaluates forces, advances the simulation (Sec. 2.1) and
 * selects among algorithmic configurations in tuning phases whose trial
 * steps still advance the simulation (Sec. 1, Sec. 2.2.5, Sec. 5).  The
 * calls below are those operations.
 *
 * Conventions shared by every call:
 *  - Every function returns an ljsel_status and never aborts or throws.  On
 *    failure ljsel_last_error() gives a message (per calling thread).
 *  - Pointers flagged "host or device" are device pointers when the
 *    `on_device` argument is non-zero, host pointers otherwise.  All arrays
 *    are C-contiguous; particle arrays are n x 3 doubles (x, y, z per
 *    particle) in the caller's input order.  The library re-sorts particles
 *    internally; that order is never visible to the caller.
 *  - The library copies inputs into memory it owns and writes outputs into
 *    caller-owned buffers.  A handle is not thread-safe.
 *  - Work is enqueued on the stream given at creation (NULL: the legacy
 *    default stream).  Calls that return values to host memory synchronize
 *    that stream before returning; ljsel_step does not synchronize.
 *  - Reduced LJ units throughout (energy eps, length sigma, mass m).
 */
#ifndef LJSEL_H
#define LJSEL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LJSEL_ABI_VERSION 1
#define LJSEL_MAX_TYPES 4

typedef enum ljsel_status {
    LJSEL_OK = 0,
    LJSEL_ERR_ARG = 1,         /* invalid argument or NULL handle                  */
    LJSEL_ERR_CUDA = 2,        /* a CUDA runtime call failed                       */
    LJSEL_ERR_OOM = 3,         /* device allocation failed                         */
    LJSEL_ERR_CAPACITY = 4,    /* neighbour-list capacity overflow not recovered   */
    LJSEL_ERR_BOX = 5,         /* a box length is below 2 (r_c + skin)             */
    LJSEL_ERR_NONFINITE = 6,   /* a position, velocity or force became non-finite  */
    LJSEL_ERR_TIMEOUT = 7,     /* a bounded device-side wait gave up               */
    LJSEL_ERR_STATE = 8,       /* call not valid in the current state              */
    LJSEL_ERR_UNSUPPORTED = 9  /* configuration not available for this system      */
} ljsel_status;

/* Neighbour-identification methods (Sec. 2.2.1, Table 1 in GPU form).       */
typedef enum ljsel_method {
    LJSEL_METHOD_LC = 0,       /* linked cells: every step each particle scans the
                                  particles of the cells within reach (no list)  */
    LJSEL_METHOD_VL = 1,       /* Verlet lists: per-particle lists of neighbours
                                  within r_c + skin, rebuilt every R steps        */
    LJSEL_METHOD_CLUSTER = 2,  /* cluster lists (the paper's Verlet list cells):
                                  i-clusters of M = 2, 4 or 8 consecutive
                                  sorted particles of one cell, each with one
                                  list of the j-particles within r_c + skin of
                                  any member; threads_per_unit lanes (M .. 32)
                                  per i-cluster                                  */
    LJSEL_METHOD_VLW = 3       /* Verlet lists over shared-memory windows: cells are
                                  cut into strips of <= 128 particles, each CTA
                                  stages its strip's neighbourhood (<= 2047
                                  particles) on chip and list entries are 16-bit
                                  window slots (CSF 1, one thread per particle)   */
} ljsel_method;

/* System parameters.  eps/sigma/rcut are ntypes x ntypes row-major and must
 * be symmetric; only the first ntypes*ntypes entries are read.            */
typedef struct ljsel_params {
    double box[3];             /* periodic orthorhombic box lengths            */
    int32_t ntypes;            /* 1 .. LJSEL_MAX_TYPES                         */
    int32_t shift_potential;   /* 1: pair energy shifted to zero at the cutoff */
    double eps[LJSEL_MAX_TYPES * LJSEL_MAX_TYPES];
    double sigma[LJSEL_MAX_TYPES * LJSEL_MAX_TYPES];
    double rcut[LJSEL_MAX_TYPES * LJSEL_MAX_TYPES];   /* cutoff per type pair   */
    double mass[LJSEL_MAX_TYPES];
    double skin;               /* Verlet skin (>= 0); list radius r_c + skin   */
    double dt;                 /* Stormer-Verlet time step                     */
    int32_t precision;         /* 0: FP32 pair math, FP64 integration and sums;
                                  1: FP64 everywhere (check path)              */
    int32_t use_graphs;        /* 1: ljsel_step runs as one CUDA graph with
                                  device-side rebuild decisions; 0: plain
                                  stream launches                             */
    int32_t walls[3];          /* 1: dimension d is closed by reflective walls
                                  at 0 and box[d] (no periodic image; a
                                  particle crossing a wall is mirrored back
                                  with its velocity component reversed, the
                                  walled heating sphere of Sec. 6); 0:
                                  periodic.  Walls are available with the
                                  LC, VL and CLUSTER methods of single
                                  systems.                                    */
    int32_t pad;
} ljsel_params;

/* One algorithmic configuration (the GPU counterpart of a container /
 * traversal / N3L / cell-size-factor combination, Sec. 2.2).             */
typedef struct ljsel_config {
    int32_t method;            /* ljsel_method                                 */
    int32_t cluster_size;      /* CLUSTER: 2, 4 or 8; ignored otherwise        */
    int32_t newton3;           /* 1: each pair evaluated once and applied to
                                  both particles (Sec. 2.1); 0: twice          */
    int32_t threads_per_unit;  /* threads sharing one particle (VL: a power of
                                  two <= 32; LC and VLW: 1) or one i-cluster
                                  (CLUSTER: a power of two from M to 32)       */
    int32_t rebuild_interval;  /* R >= 1: rebuild at least every R steps; a
                                  rebuild also happens as soon as a particle
                                  has moved skin/2 since the last one          */
    double csf;                /* cell size factor, 1.0 or 0.5 (Sec. 2.2.1)    */
} ljsel_config;

/* Live simulation statistics over CSF-1 cell bins (Sec. 4).              */
typedef struct ljsel_stats {
    double mean;               /* particles per bin                            */
    double rel_std;            /* population std / mean                        */
    double median;             /* mean of the two middle counts if even        */
    double max;
    double nbins;
    double nempty;
    double skin;
    double threads;            /* threads the GPU keeps resident (SMs x
                                  threads per SM): the device's parallelism,
                                  as the paper's thread count is the run's    */
} ljsel_stats;

/* Counters since creation (host-side copies, refreshed by calls that
 * synchronize).                                                           */
typedef struct ljsel_counters {
    int64_t steps;             /* Verlet steps taken                           */
    int64_t rebuilds;          /* neighbour-structure rebuilds                 */
    int64_t early_rebuilds;    /* rebuilds forced by the skin/2 displacement   */
    int64_t list_entries;      /* entries kept by the last list build, summed
                                  over all rows (0 for LC)                     */
    int64_t list_capacity;     /* allocated entries                            */
    int64_t nclusters;         /* i-clusters (CLUSTER)                         */
    int64_t ncells;            /* cells of the current grid                    */
    int64_t capacity_retries;  /* list reallocations after an overflow         */
    int64_t replica_rebuilds;  /* batches: replica rebuilds summed over all
                                  replicas (each rebuild event re-lists only
                                  the replicas that need it); 0 otherwise     */
    int64_t longest_row;       /* longest list row of the last build          */
} ljsel_counters;

/* Autotuner options (Sec. 2.2.5 Full Search, Sec. 5.1 Predictive, Sec. 5.2
 * Expert, Sec. 5.3 Random Forest).                                        */
typedef struct ljsel_tuner_opts {
    int32_t strategy;          /* 0: full search; 1: predictive; 2: expert
                                  (fuzzy rules on the mean particles per
                                  CSF-1 bin, Sec. 4 statistics); 3: random
                                  forest (the forest installed with
                                  ljsel_set_forest ranks its configurations
                                  from the Sec. 4 statistics; with forest_top
                                  1 its first choice is selected without a
                                  trial, with forest_top k > 1 the k most
                                  probable are trialled)                      */
    int32_t trial_steps;       /* steps per trial (>= 1); a trial first
                                  rebuilds, then advances trial_steps steps   */
    double predict_factor;     /* predictive: trial configs predicted within
                                  this factor of the best (2.0)               */
    double blacklist_factor;   /* drop configs measured this much slower than
                                  the best (10.0); <= 0 disables              */
    int32_t retrial_phases;    /* predictive: re-trial a config not trialled
                                  for this many phases (>= 1)                 */
    int32_t ncandidates;       /* > 0: use candidates[]; 0: the default set   */
    const ljsel_config *candidates;
    int32_t probe_steps;       /* a trial first runs this many steps; when its
                                  cost is above probe_factor x the best cost
                                  of the phase so far, the trial stops there
                                  (0: always run trial_steps)                 */
    int32_t forest_top;        /* random forest: 1 (or 0): select the first
                                  choice; k > 1: trial the k most probable  */
    double probe_factor;       /* e.g. 2.0                                     */
    double skip_within;        /* > 0: when the live statistics (mean,
                                  relative std and max particles per CSF-1
                                  bin, Sec. 4) all differ by less than this
                                  relative amount from those at the last phase
                                  that ran trials, the phase is skipped and the
                                  configuration kept (0: never skip)          */
} ljsel_tuner_opts;

/* Result of the last tuning phase.                                        */
typedef struct ljsel_tuner_report {
    int32_t phase;             /* tuning phases run so far                    */
    int32_t ntrialled;         /* configs trialled in the last phase          */
    int32_t nblacklisted;
    int32_t chosen_index;      /* index into the candidate set                */
    double chosen_cost_ms;     /* cost per step of the chosen config          */
    double phase_ms;           /* wall time of the last phase (all trials)    */
    double overhead_ms;        /* sum over trials of (trial - chosen) cost    */
    int64_t trial_steps_total; /* steps advanced by trials in the last phase  */
    int32_t nprobed_out;       /* trials stopped after their probe            */
    int32_t skipped;           /* 1: the phase was skipped (skip_within)      */
    double expert_input;       /* expert: mean particles per CSF-1 bin; random
                                  forest: probability of its first choice     */
    double rebuild_every;      /* the interval the build time was weighted by
                                  for configs with a longer R: the mean steps
                                  per rebuild observed since the last phase
                                  when most of those rebuilds came early (a
                                  particle reached skin/2), else 0 (each
                                  config's own R)                             */
} ljsel_tuner_report;

/* GPU time per kernel class, measured with CUDA events around each launch
 * of plain stream launches (the tuning cost of Sec. 2.2.5 is built from
 * the build and force times).                                              */
typedef struct ljsel_profile {
    int64_t steps;             /* steps advanced by the profiled call          */
    int64_t rebuilds;          /* rebuilds among them                          */
    int64_t launches;          /* kernels launched                             */
    double rebuild_ms;         /* mean GPU time of one rebuild (all kernels)   */
    double force_ms;           /* mean GPU time of the force kernel, fused
                                  with the Stormer-Verlet update when N3L is
                                  off                                         */
    double update_ms;          /* mean GPU time of the separate update kernel
                                  (N3L on), 0 otherwise                        */
    double control_ms;         /* mean GPU time of the per-step control kernel */
    double total_ms;           /* sum of the above over the call               */
} ljsel_profile;

typedef struct ljsel_system_s *ljsel_system;

/* Message of the last failing call on this thread ("" if none).           */
const char *ljsel_last_error(void);
int32_t ljsel_abi_version(void);

/* Create a system of n particles (Sec. 2.1).  pos, vel: n x 3 (host or
 * device per on_device); types: n int32 in [0, ntypes) (host or device;
 * NULL means all 0).  stream: a cudaStream_t or NULL.  Fails with
 * LJSEL_ERR_BOX if a box length is below 2 (max r_c + skin), LJSEL_ERR_ARG
 * for malformed parameters.  The default configuration is VL, N3L off,
 * one thread per particle, R = 10, CSF 1.  Velocities are at the same time
 * as positions.  *out receives a handle owned by the caller (free with
 * ljsel_destroy).                                                         */
ljsel_status ljsel_create(const ljsel_params *params, int64_t n, const double *pos,
                          const double *vel, const int32_t *types, int32_t on_device,
                          void *stream, ljsel_system *out);

ljsel_status ljsel_destroy(ljsel_system s);

/* Select the algorithmic configuration used from now on (Sec. 2.2).  When
 * the new configuration shares the built neighbour structure (it differs
 * only in threads_per_unit or rebuild_interval) the structure is kept and
 * the new interval counts from the last rebuild; otherwise the next force
 * evaluation rebuilds.  Returns LJSEL_ERR_UNSUPPORTED for combinations the
 * library does not provide.                                               */
ljsel_status ljsel_set_config(ljsel_system s, const ljsel_config *cfg);
ljsel_status ljsel_get_config(ljsel_system s, ljsel_config *cfg);

/* Set the capacity of the current configuration's list rows (entries per
 * particle row for VL, rounded up to a multiple of 4; per window-list row
 * for VLW, a multiple of 16, at most 512; per i-cluster row for CLUSTER, a
 * multiple of 4) instead of the library's estimate, and rebuild before the
 * next evaluation.  A build that needs more still grows the rows and
 * rebuilds.  Errors: ARG for entries outside 4 .. 65532 (or above 512 for
 * VLW), STATE for linked cells (no list).  The next ljsel_set_config
 * re-estimates the capacity only when the rows must grow.                 */
ljsel_status ljsel_set_list_capacity(ljsel_system s, int64_t entries);

/* Rebuild the neighbour structure now (binning, sorting, lists; Sec.
 * 2.2.1).  Positions are wrapped into the box first.                     */
ljsel_status ljsel_rebuild(ljsel_system s);

/* Evaluate forces, potential energy and virial at the current positions
 * with the current configuration (Sec. 2.1).  forces: n x 3 (host or
 * device; NULL to skip), in input order.  energy: shifted potential energy
 * sum over pairs; virial: sum over pairs of r_ij . F_ij (both host double,
 * NULL to skip).  With energy and virial both NULL the forces come from
 * the force arithmetic of the stepping kernels (no sums accumulated), else
 * from the kernels that also accumulate the sums.  Synchronizes the
 * stream.                                                                 */
ljsel_status ljsel_compute(ljsel_system s, double *forces, int32_t on_device,
                           double *energy, double *virial);

/* Advance nsteps Stormer-Verlet steps (Sec. 2.1) with the current
 * configuration, rebuilding the neighbour structure every R steps or
 * earlier when a particle has moved skin/2.  Asynchronous: errors raised on
 * the device (capacity overflow, non-finite values) are reported by the
 * next synchronizing call.                                                */
ljsel_status ljsel_step(ljsel_system s, int64_t nsteps);

/* Copy positions (wrapped into [0, L)) and velocities at the current
 * integer time step into caller buffers (n x 3, host or device; either may
 * be NULL).  Synchronizes the stream.                                     */
ljsel_status ljsel_get_state(ljsel_system s, double *pos, double *vel, int32_t on_device);

/* Replace positions and velocities (n x 3, host or device).               */
ljsel_status ljsel_set_state(ljsel_system s, const double *pos, const double *vel, int32_t on_device);

/* Move particles to new positions (host or device, n x 3, input order;
 * velocities unchanged) while keeping the neighbour structure of the last
 * rebuild, as an external integrator moving particles by less than skin/2
 * between rebuilds would (Sec. 2.2.1).  Positions need not lie in the box.
 * Any particle now at skin/2 or more from where it was at the last rebuild
 * makes the next evaluation rebuild first, so results never depend on a
 * stale structure.  Synchronizes the stream.                              */
ljsel_status ljsel_move_particles(ljsel_system s, const double *pos, int32_t on_device);

/* The positions the pair arithmetic uses (the working-precision copy,
 * promoted exactly to double, not wrapped), n x 3 in input order.  With
 * these, the oracle reproduces the pair set bit for bit.                  */
ljsel_status ljsel_get_work_positions(ljsel_system s, double *pos, int32_t on_device);

/* The set of pairs within the cutoff, exactly as the force evaluation of
 * the current configuration decides it (Sec. 2.1 neighbours).  ij: host,
 * 2 x cap int32 (i < j, input indices, unordered); *count receives the
 * total number of pairs even when it exceeds cap.  Synchronizes.          */
ljsel_status ljsel_get_pairs(ljsel_system s, int64_t cap, int32_t *ij, int64_t *count);

/* Kinetic and potential energy and virial at the current integer step.    */
ljsel_status ljsel_get_energy(ljsel_system s, double *epot, double *ekin, double *virial);

/* Live statistics (Sec. 4) of the current positions.                      */
ljsel_status ljsel_get_stats(ljsel_system s, ljsel_stats *st);
ljsel_status ljsel_get_counters(ljsel_system s, ljsel_counters *c);

/* Run one tuning phase (Sec. 2.2.5, Sec. 5.1): trial candidate
 * configurations, each building its own neighbour structure and then
 * advancing opts->trial_steps steps of the simulation, keep the one with
 * the lowest cost per step (build time over R plus force and integration
 * time per step; when most rebuilds since the last phase came early, the
 * build time is divided by min(R, the observed steps per rebuild) instead,
 * reported as report->rebuild_every), and select it.  chosen and
 * report may be NULL.  State (blacklist, history for the predictive
 * strategy) persists across phases of the same handle.                    */
ljsel_status ljsel_autotune(ljsel_system s, const ljsel_tuner_opts *opts,
                            ljsel_config *chosen, ljsel_tuner_report *report);

/* A random-forest classifier (Sec. 5.3) over the live statistics: the
 * feature vector is the fields of ljsel_stats in order (mean, rel_std,
 * median, max, nbins, nempty, skin, threads; the first nfeatures of them).
 * Node k of the flattened trees either splits (feature[k] in 0..nfeatures-1:
 * go to left[k] when x[feature[k]] <= threshold[k], else to right[k]) or is
 * a leaf (feature[k] = -1) holding class probabilities value[k * nclasses +
 * c].  Class c names the configuration classes[c].  All arrays are host
 * memory owned by the caller.                                             */
typedef struct ljsel_forest {
    int32_t ntrees;
    int32_t nclasses;
    int32_t nfeatures;         /* 1..8                                         */
    int32_t nnodes;            /* nodes over all trees                         */
    const int32_t *root;       /* [ntrees] root node of each tree              */
    const int32_t *feature;    /* [nnodes] split feature, -1 at a leaf         */
    const double *threshold;   /* [nnodes]                                     */
    const int32_t *left;       /* [nnodes] (leaves: ignored)                   */
    const int32_t *right;      /* [nnodes] (leaves: ignored)                   */
    const double *value;       /* [nnodes * nclasses] leaf class probabilities */
    const ljsel_config *classes; /* [nclasses]                                 */
} ljsel_forest;

/* Class probabilities of the forest for one feature vector x[nfeatures]:
 * the mean over the trees of the leaf each tree reaches.  Host only (no
 * GPU).  proba: host, nclasses doubles.  LJSEL_ERR_ARG for a NULL pointer
 * or a malformed forest (a root, child or feature out of range, a negative
 * or non-finite leaf value, a path longer than nnodes).                   */
ljsel_status ljsel_forest_predict(const ljsel_forest *f, const double *x, double *proba);

/* Install (copy) a forest in the system for the Random Forest strategy;
 * the same checks as ljsel_forest_predict, and every class must be a valid
 * configuration for this system (LJSEL_ERR_UNSUPPORTED otherwise).        */
ljsel_status ljsel_set_forest(ljsel_system s, const ljsel_forest *f);

/* Cost per step (ms) measured for each configuration in its most recent
 * trial (the cost the tuner compares), for the configurations trialled so
 * far: writes up to cap configurations and costs, *count = their number.
 * Host only; the phase of the last trial goes to phase[k] (may be NULL).  */
ljsel_status ljsel_tuner_costs(ljsel_system s, int32_t cap, ljsel_config *cfgs, double *cost, int32_t *phase,
                               int32_t *count);

/* The trial set of one Predictive tuning phase (Sec. 5.1), host only (no
 * GPU, no handle); ljsel_autotune applies the same rule.  Before phase 2
 * every configuration that is not blacklisted is trialled.  From phase 2 on,
 * configuration k is trialled when it is not blacklisted and (a) it has no
 * measurement, or (b) its predicted cost is at most predict_factor x the
 * lowest prediction, or (c) it was last trialled retrial_phases or more
 * phases ago, or (d) it is the incumbent.  The prediction is the line
 * through its last two measurements evaluated at `phase` (the measurement
 * itself when there is one), never below half of its last measurement: a
 * steeply falling pair of costs would otherwise predict a cost near zero
 * and exclude every other configuration.
 *   hist_n[k]           0, 1 or 2 measurements of configuration k
 *   hist_phase, hist_cost [2 k], [2 k + 1]: (phase, cost) of the older and
 *                       the newer measurement (with one, only [2 k + 1])
 *   last_trial_phase[k] phase of its last trial (-1: never)
 *   blacklisted[k]      0 or 1
 *   incumbent           index of the configuration in use, or -1
 *   trial[k]            out: 1 if trialled, else 0
 * All arrays have ncand entries (hist_* 2 ncand) and are host memory.
 * Errors: LJSEL_ERR_ARG for ncand < 0, a NULL array with ncand > 0, hist_n
 * outside 0..2, incumbent outside -1..ncand-1 or predict_factor <= 0.     */
ljsel_status ljsel_predictive_trials(int32_t ncand, int32_t phase, const int32_t *hist_n,
                                     const int32_t *hist_phase, const double *hist_cost,
                                     const int32_t *last_trial_phase, const int32_t *blacklisted,
                                     int32_t incumbent, double predict_factor, int32_t retrial_phases,
                                     int32_t *trial);

/* The Expert strategy's rating of a configuration (Sec. 2.3, Sec. 5.2), host
 * only (no GPU, no handle): the fuzzy input is the mean particles per CSF-1
 * bin; input terms sparse, medium, dense (trapezoids with corners
 * (-inf, -inf, 1, 4), (1, 4, 8, 12), (8, 12, inf, inf)); output terms bad,
 * okay, good ((-inf, -inf, 0.1, 0.4), (0.2, 0.5, 0.5, 0.8), (0.6, 0.9, inf,
 * inf)); the rule table maps each method family and input term to an output
 * term (Verlet lists okay / good / good, window lists bad / okay / okay,
 * linked cells good / okay / bad, cluster lists okay / bad / bad).  Max-min
 * inference; *out = centre of gravity of the aggregated output set sampled
 * at 201 points of [0, 1].  A tuning phase trials configurations rated
 * >= 0.5.  Errors: LJSEL_ERR_ARG for NULL pointers, an unknown method or a
 * non-finite input.                                                       */
ljsel_status ljsel_expert_suitability(const ljsel_config *cfg, double mean_per_bin, double *out);

/* Advance nsteps steps with plain stream launches, a CUDA event before and
 * after every kernel class, and report mean GPU times per launch.  The
 * steps advance the simulation like ljsel_step.  Synchronizes every step;
 * for measurement, not production.                                       */
ljsel_status ljsel_profile_steps(ljsel_system s, int64_t nsteps, ljsel_profile *out);

/* The default candidate set for this system: writes up to cap configs and
 * returns their number in *count.                                         */
ljsel_status ljsel_default_candidates(ljsel_system s, int32_t cap, ljsel_config *out, int32_t *count);

/* Velocity-scaling thermostat (the heating of the walled sphere, Sec. 6):
 * the temperature T = sum m v^2 / dof of the integer-step velocities (dof =
 * 3N - 3 in a periodic box, whose total momentum is conserved; 3N when any
 * dimension has walls) is moved towards `target` by at most `max_change`,
 * by scaling every velocity with sqrt(T_new / T).  t_before (optional)
 * receives T before the scaling.  Synchronizes the stream.                */
ljsel_status ljsel_thermostat(ljsel_system s, double target, double max_change, double *t_before);

/* ---- Gradients --------------------------------------------------------
 * The paper has no gradient; these calls serve the differentiable binary
 * mixture (a force-matching loss differentiated with respect to positions
 * and the per-type-pair eps/sigma).  Definitions:
 *  - F_i = sum_j g(r_ij^2) r_ij over the in-range pairs, r_ij = x_i - x_j
 *    (minimum image), g(s) = 24 eps (2 sig^12 / s^7 - sig^6 / s^4)
 *    (Sec. 2.1 names the LJ potential; the energy shift does not enter F).
 *  - The pair set is frozen at the evaluation point: derivatives are those
 *    of the fixed sum over the pairs in range there (the cutoff's motion
 *    with sigma and the jump of F at r_c are not differentiated).
 *  - eps_ab = eps_ba is one parameter; gradient entries (a,b) and (b,a)
 *    both hold the derivative with respect to it.
 * Arithmetic is in the system's precision (FP32 pair math with FP64 sums,
 * or FP64 throughout with precision 1).                                   */

/* Replace the per-type-pair tables (ntypes x ntypes each, row-major,
 * symmetric; eps >= 0, sigma > 0).  rcut NULL keeps the current cutoffs.
 * Positions and velocities are kept; the neighbour structure is rebuilt
 * before the next evaluation (and the cell grid re-planned if the largest
 * cutoff changed).  Invalidates a recorded rollout.  Errors: ARG for
 * invalid tables, BOX when the new cutoffs no longer fit the box.        */
ljsel_status ljsel_set_pair_params(ljsel_system s, const double *eps, const double *sigma, const double *rcut);

/* Vector-Jacobian product of the forces at the current working positions:
 *   cot   (host or device, n x 3): the cotangent dL/dF, input order;
 *   g_pos (host or device, n x 3, or NULL): (dF/dx)^T cot, i.e. minus the
 *         Hessian of the potential energy applied to cot;
 *   g_eps, g_sigma (host, ntypes x ntypes each, or NULL): d(cot . F)/d eps
 *         and d(cot . F)/d sigma.
 * Synchronizes the stream.                                                */
ljsel_status ljsel_force_vjp(ljsel_system s, const double *cot, int32_t on_device, double *g_pos,
                             double *g_eps, double *g_sigma);

/* Advance nsteps Stormer-Verlet steps (as ljsel_step) while recording the
 * state at steps 0, every, 2 every, ... (checkpoints in device memory owned
 * by the system, 48 bytes per particle each) and at the end.  At every
 * checkpoint the neighbour structure is rebuilt from the recorded state, so
 * that ljsel_rollout_vjp can recompute each segment bit for bit.  The
 * system ends at step nsteps with velocities at the integer step, as after
 * ljsel_set_state.  Errors: ARG for nsteps < 0 or every < 1.             */
ljsel_status ljsel_rollout(ljsel_system s, int64_t nsteps, int64_t every);

/* Reverse-mode derivative of the last ljsel_rollout: from the cotangents
 * xbar, vbar (host or device, n x 3, input order; vbar may be NULL = 0) of
 * the final positions and velocities, the cotangents of the initial ones
 * (g_x0, g_v0: host or device, n x 3, or NULL) and of eps/sigma (g_eps,
 * g_sigma: host, ntypes x ntypes, or NULL).  Each segment between
 * checkpoints is recomputed forward and then reversed level by level, one
 * force VJP per time level.  The system is left at the rollout's final
 * state.  Errors: STATE when no rollout was recorded, or the configuration
 * or parameters changed since.  Synchronizes the stream.                 */
ljsel_status ljsel_rollout_vjp(ljsel_system s, const double *xbar, const double *vbar, int32_t on_device,
                               double *g_x0, double *g_v0, double *g_eps, double *g_sigma);

/* ---- Batched replicas ---------------------------------------------------
 * Many independent periodic single-species LJ systems of uneven size, each
 * in its own box with its own cell grid (Sec. 2.2.1), stepped together: one
 * launch per kernel stage covers all of them and a run of steps is one CUDA
 * graph.  All replicas share eps, sigma, r_c, the shift, mass, skin, dt and
 * precision.  The rebuild rule is the single system's, taken over the whole
 * batch: every R steps, or as soon as any particle moved skin/2.
 * Particle arrays are the replicas' arrays concatenated in replica order
 * (sum(counts) x 3 doubles); the library keeps that order for the caller.  */
typedef struct ljsel_batch_s *ljsel_batch;

/* Shape of the batched force kernel: lanes per particle, threads per CTA,
 * and 0 (one lane group per particle) or the CTAs per SM of a persistent
 * grid that strides over the particles.  rebuild_interval = R.           */
typedef struct ljsel_batch_tile {
    int32_t threads_per_particle;  /* 1, 2, 4, 8                             */
    int32_t block_threads;         /* 64, 128, 256                           */
    int32_t persistent_ctas_per_sm;/* 0 .. 32                                */
    int32_t rebuild_interval;      /* >= 1 (1 without a skin)                */
} ljsel_batch_tile;

/* Create a batch.  params: shared parameters (ntypes must be 1; box is
 * ignored).  boxes: host, nrep x 3; counts: host, nrep (>= 0 each, total in
 * [1, 2^27)); pos, vel: host or device, sum(counts) x 3.  Errors: ARG, BOX
 * (a replica box below 2 (r_c + skin)), UNSUPPORTED (ntypes > 1), OOM.    */
ljsel_status ljsel_batch_create(const ljsel_params *params, int32_t nrep, const double *boxes, const int64_t *counts,
                                const double *pos, const double *vel, int32_t on_device, void *stream,
                                ljsel_batch *out);
ljsel_status ljsel_batch_destroy(ljsel_batch b);
ljsel_status ljsel_batch_set_tile(ljsel_batch b, const ljsel_batch_tile *tile);
ljsel_status ljsel_batch_get_tile(ljsel_batch b, ljsel_batch_tile *tile);
/* Advance every replica nsteps steps (one CUDA graph; _eager: plain stream
 * launches, bit-identical results).                                       */
ljsel_status ljsel_batch_step(ljsel_batch b, int64_t nsteps);
ljsel_status ljsel_batch_step_eager(ljsel_batch b, int64_t nsteps);
/* Forces (host or device, sum(counts) x 3) at the current positions, and
 * per-replica potential energy and virial (host, nrep each; NULL to skip).
 * Synchronizes the stream.                                                */
ljsel_status ljsel_batch_compute(ljsel_batch b, double *forces, int32_t on_device, double *energy, double *virial);
/* Positions (wrapped into each replica's box) and integer-step velocities,
 * host or device, sum(counts) x 3 each (either may be NULL).             */
ljsel_status ljsel_batch_get_state(ljsel_batch b, double *pos, double *vel, int32_t on_device);
/* The working-precision positions the pair arithmetic uses (host only).   */
ljsel_status ljsel_batch_get_work_positions(ljsel_batch b, double *pos);
/* In-range pairs: rij (host, 3 x cap) gets (replica, i, j) triples with i < j
 * replica-local input indices; *count the total (may exceed cap).         */
ljsel_status ljsel_batch_get_pairs(ljsel_batch b, int64_t cap, int32_t *rij, int64_t *count);
ljsel_status ljsel_batch_get_counters(ljsel_batch b, ljsel_counters *c);
/* Set the row capacity of the batch's lists (a multiple of 4, as for a
 * single system's VL rows); rebuilt before the next step.                 */
ljsel_status ljsel_batch_set_list_capacity(ljsel_batch b, int64_t entries);
/* nsteps real steps with CUDA events around each kernel class, as
 * ljsel_profile_steps (force_ms covers the fused force + update kernel).  */
ljsel_status ljsel_batch_profile_steps(ljsel_batch b, int64_t nsteps, ljsel_profile *out);
/* Tile selection by full search: each candidate (ncand = 0: a default set
 * of ten) runs trial_steps timed steps that advance the batch; the fastest
 * per step is kept and returned in *chosen; costs_ms (host, ncand or ten
 * entries, or NULL) receives each candidate's ms/step (-1: not run).     */
ljsel_status ljsel_batch_autotune(ljsel_batch b, int32_t trial_steps, int32_t ncand, const ljsel_batch_tile *cand,
                                  ljsel_batch_tile *chosen, double *costs_ms);

/* Self-test of the failure path of the library's bounded device waits (the
 * look-back of the cell scan, the window loads): one GPU thread waits on a
 * flag that nothing sets, gives up after `polls` polls (1 .. 2^24, about
 * 50 ns each) and records a timeout, which the host reads.  Returns
 * LJSEL_ERR_TIMEOUT when the path works; the GPU context stays usable.    */
ljsel_status ljsel_selftest_wait_timeout(int64_t polls);

/* Measured throughput of the arithmetic pipes the kernels use, in 1e12
 * operations per second: FP32 fused multiply-add counted as 2 flops, the
 * packed FP32x2 form counted as 4, FP64 fused multiply-add as 2, and the
 * approximate FP32 reciprocal as 1.  The paper has no counterpart; these are
 * the peaks that the force (FP32, reciprocal) and update (FP64) kernels are
 * measured against.                                                         */
typedef struct ljsel_peaks {
    double fp32_tflops;
    double fp32x2_tflops;
    double fp64_tflops;
    double rcp_tops;
} ljsel_peaks;

/* Run the four probes on the current device, each an independent-chain
 * kernel over a grid that fills every SM, timed with CUDA events after a
 * warm-up launch and scaled to last about target_ms (0 < target_ms <=
 * 10000).  Allocates a small scratch buffer; synchronizes the device's
 * legacy default stream.                                                  */
ljsel_status ljsel_measure_peaks(double target_ms, ljsel_peaks *out);

/* Allocation-free force evaluation.  The paper has no counterpart: this is
 * a service for callers that cannot allocate device memory -- code inside a
 * framework whose allocator has reserved all device memory and forbids
 * allocations behind its back, plug-ins running inside a host application
 * that owns the device, or latency-critical loops that must not take the
 * allocator's locks or the implicit synchronization of a free.  It bins the
 * particles into linked cells of side >= max r_cut (no skin) and evaluates
 * the library's FP32 LJ pair arithmetic with the exact cutoff decision,
 * using only a fixed 5.8 MB static device array inside the library (held
 * by every GPU that loads the library until the process exits) and the
 * caller's buffers.
 *   params: as for ljsel_create; precision must be 0; periodic box only.
 *   n: 1 .. 131072 particles; larger n, or a box needing more than 131072
 *      cells, returns LJSEL_ERR_CAPACITY before any work is enqueued.
 *   pos: device, n x 3 doubles (wrapped into the box on the fly);
 *   types: device, n int32 in [0, ntypes) (NULL: all 0);
 *   forces: device, n x 3 doubles, written in input order;
 *   energy, virial: host doubles or NULL; when either is given the call
 *      reads them back and synchronizes the stream, so it returns
 *      LJSEL_ERR_STATE (enqueuing nothing) when the stream is being
 *      captured.
 *   stream: cudaStream_t or NULL.
 * The first call in a CUDA context resolves the device address of the
 * static array (with that device current) and caches it per context.  All
 * calls share the array and it keeps the last call's contents (each call
 * clears what must start at zero); calls whose GPU work overlaps (on
 * different streams or from different threads) race on it, so serialize
 * them.  Calls no cudaMalloc, cudaFree or other allocating routine.       */
ljsel_status ljsel_compute_forces_noalloc(const ljsel_params *params, int64_t n, const double *pos,
                                          const int32_t *types, double *forces, double *energy, double *virial,
                                          void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LJSEL_H */
