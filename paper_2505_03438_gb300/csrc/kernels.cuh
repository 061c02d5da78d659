// kernels.cuh -- host-side launchers of the library's CUDA kernels.
#pragma once

#include "ljsel_internal.cuh"

namespace ljsel {

// Rebuild pipeline (Sec. 2.2.1): every launcher is a no-op on the device
// unless Ctrl::rebuild_now is set, so the same sequence serves eager streams
// and graph bodies.
template <typename R> void launch_bin(const Dev<R> &S, cudaStream_t st);
template <typename R> void launch_scan(const Dev<R> &S, int M, cudaStream_t st);
template <typename R> void launch_scatter(const Dev<R> &S, cudaStream_t st);
template <typename R> void launch_sortgather(const Dev<R> &S, cudaStream_t st);
template <typename R> void launch_vl_build(const Dev<R> &S, bool n3l, cudaStream_t st);
template <typename R> void launch_cluster_form(const Dev<R> &S, cudaStream_t st);
template <typename R> void launch_cp_build(const Dev<R> &S, bool n3l, cudaStream_t st);
void launch_rebuild_finish(Ctrl *C, cudaStream_t st);
template <typename R> void launch_strip_plan(const Dev<R> &S, cudaStream_t st);
template <typename R> void launch_vlw_build(const Dev<R> &S, bool n3l, cudaStream_t st);
template <typename R> void launch_vlw_force(const Dev<R> &S, const ljsel_config &cfg, int mode, bool ev,
                                            int2 *pairs, long long pairs_cap, cudaStream_t st);
void vlw_prepare();

// Force evaluation.  mode: 0 forces into S.force (+ energy/virial if ev),
// 1 forces fused with the Stormer-Verlet update (N3L off only), 2 export of
// the in-range pair set.
enum { MODE_FORCE = 0, MODE_STEP = 1, MODE_PAIRS = 2 };
template <typename R> void launch_force(const Dev<R> &S, const ljsel_config &cfg, int mode, bool ev,
                                        int2 *pairs_out, long long pairs_cap, cudaStream_t st);
template <typename R> void launch_integrate(const Dev<R> &S, bool ev, cudaStream_t st);

// Per-step control: parity flips, counters, rebuild decision; in graph mode
// it also sets the conditional handles of the rebuild IF and the step WHILE.
void launch_control(Ctrl *C, cudaGraphConditionalHandle h_rebuild, cudaGraphConditionalHandle h_loop, int graph,
                    cudaStream_t st);
void launch_loop_init(Ctrl *C, cudaGraphConditionalHandle h_rebuild, cudaGraphConditionalHandle h_loop,
                      cudaStream_t st);

// Small utilities.
template <typename R> void launch_export_forces(const Dev<R> &S, double *out, cudaStream_t st);
template <typename R> void launch_export_state(const Dev<R> &S, double *pos, double *vel, int wrap, cudaStream_t st);
template <typename R> void launch_export_work_pos(const Dev<R> &S, double *pos, cudaStream_t st);
template <typename R> void launch_import_state(const Dev<R> &S, const double *pos, const double *vel,
                                               const int *types, int init_ids, cudaStream_t st);
template <typename R> void launch_sync_velocities(const Dev<R> &S, cudaStream_t st);
template <typename R> void launch_move_particles(const Dev<R> &S, const double *pos, cudaStream_t st);
template <typename R> void launch_kinetic(const Dev<R> &S, cudaStream_t st);
template <typename R> void launch_zero_force(const Dev<R> &S, cudaStream_t st);
template <typename R> void launch_bin_stats(const Dev<R> &S, const int *counts, int nb, double *out, cudaStream_t st);

}  // namespace ljsel
