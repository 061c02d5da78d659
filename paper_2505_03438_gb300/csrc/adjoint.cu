// adjoint.cu -- gradients of the LJ forces: the force vector-Jacobian
// product (a Hessian-vector product in the positions plus the derivatives
// with respect to the per-type-pair eps and sigma) and the reverse pass of a
// checkpointed Stormer-Verlet rollout (Sec. 2.1 integrator).
//
// The pair set is frozen at the evaluation point: a pair contributes iff the
// force kernels' exact cutoff predicate keeps it.  With s = r^2,
// q = (sigma^2 / s)^3 and r_ij = x_i - x_j (minimum image), the pair force
// on i is g(s) r_ij with
//   g       = (24 eps / s) (2 q^2 - q)
//   dg/ds   = (24 eps / s^2) (4 q - 14 q^2)
//   dg/deps = (24 / s) (2 q^2 - q)
//   dg/dsig = (144 eps / (sigma s)) (4 q^2 - q)
// For a cotangent c (dL/dF) a pair adds u . g r_ij to c . F with
// u = c_i - c_j; its position gradient is w = g u + 2 dg/ds (u . r) r,
// added to particle i and subtracted from j.  Every particle scans its own
// stencil cells (no Newton's third law), so it accumulates its own w; the
// parameter sums see each pair from both ends and are halved when the two
// ordered type slots are folded on the host.
#include <algorithm>
#include <cstring>
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

constexpr int VJP_THREADS = 128;

// Per-type cotangent scale: c_i = scale[type_i] * source_i.
struct CoefTab {
    double c[MAXT];
};

// Cotangent in sorted order.  With vbar set, first advances the velocity
// cotangent through a drift (vbar += dt_x * xbar, caller order) and takes
// it as the source.
template <typename R>
__global__ void k_adj_cot(Dev<R> S, const double *src, double *vbar, const double *xbar, double dt_x, CoefTab co,
                          V4<R> *cot) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > S.n) return;
    if (k == S.n) { cot[k] = make_pos((R)0, (R)0, (R)0, 0); return; }
    const int sp = S.ctrl->state_par;
    const int id = S.id[sp][k], t = S.type[sp][k];
    double v[3];
    for (int d = 0; d < 3; ++d) {
        if (vbar) {
            double a = vbar[3 * id + d];
            if (dt_x != 0.0) a = fma(dt_x, xbar[3 * id + d], a);
            vbar[3 * id + d] = a;
            v[d] = a;
        } else {
            v[d] = src[3 * id + d];
        }
    }
    const double c = co.c[t];
    cot[k] = make_pos((R)(c * v[0]), (R)(c * v[1]), (R)(c * v[2]), 0);
}

// A group of G lanes per particle i (sorted order) over the stencil cells,
// the lanes of a group taking every G-th candidate of each cell; the same
// traversal and the same cutoff decision as the linked-cell force kernel.
// G grows as the system shrinks so that the grid fills the GPU.
// gx (caller order) receives (accumulate ? += : =) the position gradient;
// theta[0..MAXT2) and theta[MAXT2..2 MAXT2) receive the eps and sigma sums
// per ordered type pair (type_i, type_j).
template <typename R, int G>
__device__ __forceinline__ R group_sum(R v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename R, int G>
__global__ void __launch_bounds__(VJP_THREADS) k_vjp(Dev<R> S, const V4<R> *cot, double *gx, int accumulate,
                                                    double *theta) {
    __shared__ double red[2 * MAXT2];
    for (int k = threadIdx.x; k < 2 * MAXT2; k += blockDim.x) red[k] = 0.0;
    __syncthreads();
    const Ctrl *C = S.ctrl;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gid / G, sub = gid % G;
    const bool valid = i < S.n;
    const int pp = C->pos_par, sp = C->state_par, nt = S.tab.ntypes;
    const V4<R> *P = S.pos[pp];
    R ge[MAXT], gs[MAXT];
#pragma unroll
    for (int k = 0; k < MAXT; ++k) { ge[k] = 0; gs[k] = 0; }
    R gxx = 0, gxy = 0, gxz = 0;
    int ti = 0;
    if (valid) {
        const V4<R> pi = ldpos(P, i);
        const V4<R> ci = cot[i];
        ti = type_of(pi);
        const int c = S.cell_sorted[i];
        const int cx = c % S.nc[0], cy = (c / S.nc[0]) % S.nc[1], cz = c / (S.nc[0] * S.nc[1]);
        const int rch = S.reach;
        for (int oz = -rch; oz <= rch; ++oz) {
            int wz, sz;
            if (!stencil_cell(cz, oz, S.nc[2], S.walls[2], wz, sz)) continue;
            for (int oy = -rch; oy <= rch; ++oy) {
                int wy, sy;
                if (!stencil_cell(cy, oy, S.nc[1], S.walls[1], wy, sy)) continue;
                for (int ox = -rch; ox <= rch; ++ox) {
                    int wx, sx;
                    if (!stencil_cell(cx, ox, S.nc[0], S.walls[0], wx, sx)) continue;
                    const int cc = (wz * S.nc[1] + wy) * S.nc[0] + wx;
                    const bool img = (sx | sy | sz) != 0;
                    const int jb = S.cell_start[cc], je = S.cell_start[cc + 1];
                    for (int j = jb + sub; j < je; j += G) {
                        if (!img && j == i) continue;
                        const V4<R> pj = ldpos(P, j);
                        R dx, dy, dz;
                        if (!img) {
                            dx = pi.x - pj.x; dy = pi.y - pj.y; dz = pi.z - pj.z;
                        } else {
                            dx = image_dx(pi.x, pj.x, sx, S.box[0], S.box_lo[0]);
                            dy = image_dx(pi.y, pj.y, sy, S.box[1], S.box_lo[1]);
                            dz = image_dx(pi.z, pj.z, sz, S.box[2], S.box_lo[2]);
                        }
                        const R r2 = r2_of(dx, dy, dz);
                        const int tj = type_of(pj);
                        const int tp = ti * nt + tj;
                        if (!Cut<R>::in(r2, S.tab.rc2lo[tp], S.tab.rc2hi[tp], pi, pj, sx, sy, sz, S.boxd,
                                        S.tab.rc2d[tp]))
                            continue;
                        const R e24 = S.tab.e24[tp];
                        const R rinv2 = fast_rcp(r2);
                        const R sr2 = S.tab.sig2[tp] * rinv2;
                        const R q = sr2 * sr2 * sr2;
                        const R a = rinv2 * q;                      // q / s
                        const R g = a * (S.tab.e48[tp] * q - e24);  // (24 eps / s) (2 q^2 - q)
                        const R dgds = a * rinv2 * e24 * ((R)4 - (R)14 * q);
                        const V4<R> cj = cot[j];
                        const R ux = ci.x - cj.x, uy = ci.y - cj.y, uz = ci.z - cj.z;
                        const R ur = ux * dx + uy * dy + uz * dz;
                        const R k2 = (R)2 * dgds * ur;
                        gxx += g * ux + k2 * dx;
                        gxy += g * uy + k2 * dy;
                        gxz += g * uz + k2 * dz;
                        const R t1 = ur * a;
                        const R de = t1 * ((R)48 * q - (R)24);
                        const R dsg = t1 * (R)6 * e24 * S.tab.inv_sig[tp] * ((R)4 * q - (R)1);
#pragma unroll
                        for (int k = 0; k < MAXT; ++k)
                            if (k == tj) { ge[k] += de; gs[k] += dsg; }
                    }
                }
            }
        }
    }
    gxx = group_sum<R, G>(gxx);
    gxy = group_sum<R, G>(gxy);
    gxz = group_sum<R, G>(gxz);
#pragma unroll
    for (int k = 0; k < MAXT; ++k) {
        ge[k] = group_sum<R, G>(ge[k]);
        gs[k] = group_sum<R, G>(gs[k]);
    }
    if (valid && sub == 0) {
        const int id = S.id[sp][i];
        if (accumulate) {
            gx[3 * id + 0] += (double)gxx; gx[3 * id + 1] += (double)gxy; gx[3 * id + 2] += (double)gxz;
        } else {
            gx[3 * id + 0] = (double)gxx; gx[3 * id + 1] = (double)gxy; gx[3 * id + 2] = (double)gxz;
        }
#pragma unroll
        for (int k = 0; k < MAXT; ++k) {
            if (k < nt) {
                atomicAdd(&red[ti * nt + k], (double)ge[k]);
                atomicAdd(&red[MAXT2 + ti * nt + k], (double)gs[k]);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < nt * nt) {
        atomicAdd(&theta[threadIdx.x], red[threadIdx.x]);
        atomicAdd(&theta[MAXT2 + threadIdx.x], red[MAXT2 + threadIdx.x]);
    }
}

// The same VJP over the Verlet-list rows (configuration VL without N3L:
// full rows, entries without an image in 16-byte chunks padded with the
// sentinel, image entries at the back).  The list holds every pair within
// r_c + skin; the exact cutoff decision keeps the in-range ones, so the mask
// is the force kernels' mask.
template <typename R, int G>
__global__ void __launch_bounds__(VJP_THREADS) k_vjp_vl(Dev<R> S, const V4<R> *cot, double *gx, int accumulate,
                                                       double *theta) {
    __shared__ double red[2 * MAXT2];
    for (int k = threadIdx.x; k < 2 * MAXT2; k += blockDim.x) red[k] = 0.0;
    __syncthreads();
    const Ctrl *C = S.ctrl;
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gid / G, sub = gid % G;
    const bool valid = i < S.n;
    const int pp = C->pos_par, sp = C->state_par, nt = S.tab.ntypes;
    const V4<R> *P = S.pos[pp];
    R ge[MAXT], gs[MAXT];
#pragma unroll
    for (int k = 0; k < MAXT; ++k) { ge[k] = 0; gs[k] = 0; }
    R gxx = 0, gxy = 0, gxz = 0;
    int ti = 0;
    if (valid) {
        const V4<R> pi = ldpos(P, i);
        const V4<R> ci = cot[i];
        ti = type_of(pi);
        const uint32_t *row = S.nl + (size_t)i * S.nl_cap;
        const uint4 *row4 = reinterpret_cast<const uint4 *>(row);
        const int cnt = S.nl_count[i];
        const int nq = ((cnt & 0xffff) + 3) >> 2, nb = cnt >> 16;
        auto pair = [&](int j, int sx, int sy, int sz, R dx, R dy, R dz, const V4<R> &pj) {
            const R r2 = r2_of(dx, dy, dz);
            const int tj = type_of(pj);
            const int tp = ti * nt + tj;
            if (!Cut<R>::in(r2, S.tab.rc2lo[tp], S.tab.rc2hi[tp], pi, pj, sx, sy, sz, S.boxd, S.tab.rc2d[tp])) return;
            const R e24 = S.tab.e24[tp];
            const R rinv2 = fast_rcp(r2);
            const R sr2 = S.tab.sig2[tp] * rinv2;
            const R q = sr2 * sr2 * sr2;
            const R a = rinv2 * q;
            const R g = a * (S.tab.e48[tp] * q - e24);
            const R dgds = a * rinv2 * e24 * ((R)4 - (R)14 * q);
            const V4<R> cj = cot[j];
            const R ux = ci.x - cj.x, uy = ci.y - cj.y, uz = ci.z - cj.z;
            const R ur = ux * dx + uy * dy + uz * dz;
            const R k2 = (R)2 * dgds * ur;
            gxx += g * ux + k2 * dx;
            gxy += g * uy + k2 * dy;
            gxz += g * uz + k2 * dz;
            const R t1 = ur * a;
            const R de = t1 * ((R)48 * q - (R)24);
            const R dsg = t1 * (R)6 * e24 * S.tab.inv_sig[tp] * ((R)4 * q - (R)1);
#pragma unroll
            for (int k = 0; k < MAXT; ++k)
                if (k == tj) { ge[k] += de; gs[k] += dsg; }
        };
        for (int k = sub; k < nq; k += G) {
            const uint4 e = __ldg(row4 + k);
            const V4<R> p0 = ldpos(P, (int)e.x), p1 = ldpos(P, (int)e.y), p2 = ldpos(P, (int)e.z), p3 = ldpos(P, (int)e.w);
            pair((int)e.x, 0, 0, 0, pi.x - p0.x, pi.y - p0.y, pi.z - p0.z, p0);
            pair((int)e.y, 0, 0, 0, pi.x - p1.x, pi.y - p1.y, pi.z - p1.z, p1);
            pair((int)e.z, 0, 0, 0, pi.x - p2.x, pi.y - p2.y, pi.z - p2.z, p2);
            pair((int)e.w, 0, 0, 0, pi.x - p3.x, pi.y - p3.y, pi.z - p3.z, p3);
        }
        for (int k = sub; k < nb; k += G) {
            const uint32_t e = row[S.nl_cap - 1 - k];
            const int j = (int)(e & JMASK);
            int sx, sy, sz;
            decode_image(e >> JBITS, sx, sy, sz);
            const V4<R> pj = ldpos(P, j);
            pair(j, sx, sy, sz, image_dx(pi.x, pj.x, sx, S.box[0], S.box_lo[0]),
                 image_dx(pi.y, pj.y, sy, S.box[1], S.box_lo[1]), image_dx(pi.z, pj.z, sz, S.box[2], S.box_lo[2]), pj);
        }
    }
    gxx = group_sum<R, G>(gxx);
    gxy = group_sum<R, G>(gxy);
    gxz = group_sum<R, G>(gxz);
#pragma unroll
    for (int k = 0; k < MAXT; ++k) {
        ge[k] = group_sum<R, G>(ge[k]);
        gs[k] = group_sum<R, G>(gs[k]);
    }
    if (valid && sub == 0) {
        const int id = S.id[sp][i];
        if (accumulate) {
            gx[3 * id + 0] += (double)gxx; gx[3 * id + 1] += (double)gxy; gx[3 * id + 2] += (double)gxz;
        } else {
            gx[3 * id + 0] = (double)gxx; gx[3 * id + 1] = (double)gxy; gx[3 * id + 2] = (double)gxz;
        }
#pragma unroll
        for (int k = 0; k < MAXT; ++k) {
            if (k < nt) {
                atomicAdd(&red[ti * nt + k], (double)ge[k]);
                atomicAdd(&red[MAXT2 + ti * nt + k], (double)gs[k]);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < nt * nt) {
        atomicAdd(&theta[threadIdx.x], red[threadIdx.x]);
        atomicAdd(&theta[MAXT2 + threadIdx.x], red[MAXT2 + threadIdx.x]);
    }
}

template <typename F> ljsel_status dispatch(System *s, F &&f) {
    if (s->precision) return f((double)0);
    return f((float)0);
}

// Fold the ordered-pair sums into the shared-parameter derivatives.
void fold_theta(const System &s, const double *th, double *g_eps, double *g_sigma) {
    const int nt = s.params.ntypes;
    for (int a = 0; a < nt; ++a)
        for (int b = 0; b < nt; ++b) {
            const int ab = a * nt + b, ba = b * nt + a;
            // a == b: each pair is seen twice in slot (a,a); a != b: once in
            // (a,b) and once in (b,a)
            const double e = 0.5 * (th[ab] + th[ba]);
            const double g = 0.5 * (th[MAXT2 + ab] + th[MAXT2 + ba]);
            if (g_eps) g_eps[ab] = a == b ? 0.5 * th[ab] : e;
            if (g_sigma) g_sigma[ab] = a == b ? 0.5 * th[MAXT2 + ab] : g;
        }
}

template <typename R> ljsel_status ensure_adj_buffers(System *s) {
    const size_t n3 = (size_t)s->n * 3 * sizeof(double);
    TRY(s->b_adj_cot.ensure((size_t)(s->n + 1) * sizeof(V4<R>)));
    TRY(s->b_adj_x.ensure(n3));
    TRY(s->b_adj_v.ensure(n3));
    TRY(s->b_adj_theta.ensure(2 * MAXT2 * sizeof(double)));
    return LJSEL_OK;
}

// One VJP level at the current positions (structure made current first).
template <typename R>
ljsel_status vjp_level(System *s, const double *src, double *vbar, const double *xbar, double dt_x,
                       const CoefTab &co, double *gx, int accumulate) {
    TRY(s->ensure_structure<R>());
    Dev<R> S;
    s->fill_dev(S);
    V4<R> *cot = (V4<R> *)s->b_adj_cot.ptr;
    k_adj_cot<R><<<div_up(s->n + 1, 256), 256, 0, s->stream>>>(S, src, vbar, xbar, dt_x, co, cot);
    double *th = (double *)s->b_adj_theta.ptr;
    // lanes per particle: enough threads for 152 SMs x 2048 resident threads
    int G = 1;
    while (G < 32 && (long long)s->n * G < 152LL * 2048) G *= 2;
    const int grid = div_up((long long)s->n * G, VJP_THREADS);
    // full Verlet-list rows when the configuration has them, else the cells
    const bool rows = s->cfg.method == LJSEL_METHOD_VL && !s->cfg.newton3;
#define VJP_GO(g)                                                                               \
    (rows ? k_vjp_vl<R, g><<<grid, VJP_THREADS, 0, s->stream>>>(S, cot, gx, accumulate, th)     \
          : k_vjp<R, g><<<grid, VJP_THREADS, 0, s->stream>>>(S, cot, gx, accumulate, th))
    switch (G) {
        case 1: VJP_GO(1); break;
        case 2: VJP_GO(2); break;
        case 4: VJP_GO(4); break;
        case 8: VJP_GO(8); break;
        case 16: VJP_GO(16); break;
        default: VJP_GO(32); break;
    }
#undef VJP_GO
    CK(cudaGetLastError());
    return LJSEL_OK;
}

// Load positions (and velocities, if given) in caller order, as a state
// to restart from: velocities at the integer step, rebuild flagged.
template <typename R> ljsel_status load_state(System *s, const double *x, const double *v) {
    Dev<R> S;
    s->fill_dev(S);
    launch_import_state(S, x, v, nullptr, 0, s->stream);
    TRY(s->cmd(CMD_REBUILD, 0));
    TRY(s->cmd(CMD_HALF_KICK, 1));
    s->synced = true;
    CK(cudaGetLastError());
    return LJSEL_OK;
}

template <typename R> ljsel_status save_state(System *s, double *x, double *v) {
    if (v) TRY(s->sync_velocities<R>());
    Dev<R> S;
    s->fill_dev(S);
    launch_export_state(S, x, v, 0, s->stream);
    CK(cudaGetLastError());
    return LJSEL_OK;
}

bool same_params(const ljsel_params &a, const ljsel_params &b) { return memcmp(&a, &b, sizeof(a)) == 0; }
bool same_config(const ljsel_config &a, const ljsel_config &b) { return memcmp(&a, &b, sizeof(a)) == 0; }

}  // namespace

extern "C" {

ljsel_status ljsel_set_pair_params(ljsel_system h, const double *eps, const double *sigma, const double *rcut) {
    System *s = (System *)h;
    if (!s || !eps || !sigma) { set_error("NULL argument"); return LJSEL_ERR_ARG; }
    ljsel_params p = s->params;
    const int nt = p.ntypes;
    for (int k = 0; k < nt * nt; ++k) {
        p.eps[k] = eps[k];
        p.sigma[k] = sigma[k];
        if (rcut) p.rcut[k] = rcut[k];
    }
    TRY(validate_params(&p));
    if (same_params(p, s->params)) return LJSEL_OK;
    double old_max = 0, new_max = 0;
    for (int k = 0; k < nt * nt; ++k) {
        old_max = std::max(old_max, s->params.rcut[k]);
        new_max = std::max(new_max, p.rcut[k]);
    }
    s->params = p;
    s->rollout.nsteps = -1;
    if (new_max != old_max) {
        s->nl_cap = 0;
        s->cp_cap = 0;
        TRY(s->apply_config());
    }
    s->structure_dirty = true;
    return LJSEL_OK;
}

ljsel_status ljsel_force_vjp(ljsel_system h, const double *cot, int32_t on_device, double *g_pos, double *g_eps,
                             double *g_sigma) {
    System *s = (System *)h;
    if (!s || !cot) { set_error("NULL argument"); return LJSEL_ERR_ARG; }
    return dispatch(s, [&](auto z) -> ljsel_status {
        using R = decltype(z);
        TRY(ensure_adj_buffers<R>(s));
        const size_t nb = (size_t)s->n * 3 * sizeof(double);
        const double *dc = cot;
        if (!on_device) {
            TRY(s->b_io.ensure(nb));
            CK(cudaMemcpyAsync(s->b_io.ptr, cot, nb, cudaMemcpyHostToDevice, s->stream));
            dc = (const double *)s->b_io.ptr;
        }
        double *gx = (g_pos && on_device) ? g_pos : (double *)s->b_adj_x.ptr;
        CK(cudaMemsetAsync(s->b_adj_theta.ptr, 0, 2 * MAXT2 * sizeof(double), s->stream));
        CoefTab co{};
        for (int t = 0; t < MAXT; ++t) co.c[t] = 1.0;
        TRY(vjp_level<R>(s, dc, nullptr, nullptr, 0.0, co, gx, 0));
        if (g_pos && !on_device) CK(cudaMemcpyAsync(g_pos, gx, nb, cudaMemcpyDeviceToHost, s->stream));
        double th[2 * MAXT2];
        CK(cudaMemcpyAsync(th, s->b_adj_theta.ptr, sizeof(th), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        TRY(s->read_ctrl());
        TRY(s->check_device_errors());
        fold_theta(*s, th, g_eps, g_sigma);
        return LJSEL_OK;
    });
}

ljsel_status ljsel_rollout(ljsel_system h, int64_t nsteps, int64_t every) {
    System *s = (System *)h;
    if (!s) { set_error("NULL handle"); return LJSEL_ERR_ARG; }
    if (nsteps < 0 || every < 1) { set_error("nsteps must be >= 0 and every >= 1"); return LJSEL_ERR_ARG; }
    return dispatch(s, [&](auto z) -> ljsel_status {
        using R = decltype(z);
        s->rollout.nsteps = -1;
        const size_t n3 = (size_t)s->n * 3;
        const long long nseg = (nsteps + every - 1) / every;
        // per checkpoint: x then v; one more pair for the final state
        TRY(s->b_ckpt.ensure((size_t)(nseg + 1) * 2 * n3 * sizeof(double)));
        double *ck = (double *)s->b_ckpt.ptr;
        for (long long g = 0; g < nseg; ++g) {
            double *cx = ck + (size_t)g * 2 * n3;
            TRY(save_state<R>(s, cx, cx + n3));
            TRY(load_state<R>(s, cx, cx + n3));
            const long long k = std::min<long long>(every, nsteps - g * every);
            TRY(s->advance<R>(k));
        }
        double *ce = ck + (size_t)nseg * 2 * n3;
        TRY(save_state<R>(s, ce, ce + n3));
        CK(cudaStreamSynchronize(s->stream));
        s->rollout.nsteps = nsteps;
        s->rollout.every = every;
        s->rollout.cfg = s->cfg;
        s->rollout.params = s->params;
        return LJSEL_OK;
    });
}

ljsel_status ljsel_rollout_vjp(ljsel_system h, const double *xbar, const double *vbar, int32_t on_device,
                               double *g_x0, double *g_v0, double *g_eps, double *g_sigma) {
    System *s = (System *)h;
    if (!s || !xbar) { set_error("NULL argument"); return LJSEL_ERR_ARG; }
    if (s->rollout.nsteps < 0) { set_error("no rollout recorded"); return LJSEL_ERR_STATE; }
    if (!same_config(s->rollout.cfg, s->cfg) || !same_params(s->rollout.params, s->params)) {
        set_error("configuration or parameters changed since the rollout");
        return LJSEL_ERR_STATE;
    }
    return dispatch(s, [&](auto z) -> ljsel_status {
        using R = decltype(z);
        TRY(ensure_adj_buffers<R>(s));
        const long long N = s->rollout.nsteps, every = s->rollout.every;
        const long long nseg = (N + every - 1) / every;
        const size_t n3 = (size_t)s->n * 3, nb = n3 * sizeof(double);
        double *XB = (double *)s->b_adj_x.ptr, *VB = (double *)s->b_adj_v.ptr;
        CK(cudaMemcpyAsync(XB, xbar, nb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream));
        if (vbar)
            CK(cudaMemcpyAsync(VB, vbar, nb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream));
        else
            CK(cudaMemsetAsync(VB, 0, nb, s->stream));
        CK(cudaMemsetAsync(s->b_adj_theta.ptr, 0, 2 * MAXT2 * sizeof(double), s->stream));
        TRY(s->b_seg.ensure((size_t)(every + 1) * nb));
        double *ck = (double *)s->b_ckpt.ptr, *seg = (double *)s->b_seg.ptr;
        const double dt = s->params.dt;
        CoefTab half{}, full{};
        for (int t = 0; t < s->params.ntypes; ++t) {
            half.c[t] = 0.5 * dt / s->params.mass[t];
            full.c[t] = dt / s->params.mass[t];
        }
        for (long long g = nseg - 1; g >= 0; --g) {
            const long long t0 = g * every, t1 = std::min(N, t0 + every);
            double *cx = ck + (size_t)g * 2 * n3;
            // recompute x_t0 .. x_t1 from the checkpoint exactly as the forward pass ran
            TRY(load_state<R>(s, cx, cx + n3));
            CK(cudaMemcpyAsync(seg, cx, nb, cudaMemcpyDeviceToDevice, s->stream));
            for (long long t = t0 + 1; t <= t1; ++t) {
                TRY(s->advance<R>(1));
                Dev<R> S;
                s->fill_dev(S);
                launch_export_state(S, seg + (size_t)(t - t0) * n3, nullptr, 0, s->stream);
                CK(cudaGetLastError());
            }
            // reverse: level N takes the final kick only; interior levels take
            // the final kick of step t-1 and the first kick of step t (2 c);
            // level 0 the first kick of step 0
            for (long long t = (g == nseg - 1 ? t1 : t1 - 1); t >= t0; --t) {
                TRY(load_state<R>(s, seg + (size_t)(t - t0) * n3, nullptr));
                const bool last = t == N;
                const CoefTab &co = (t == 0 || last) ? half : full;
                TRY(vjp_level<R>(s, nullptr, VB, XB, last ? 0.0 : dt, co, XB, 1));
            }
        }
        // leave the system at the final state of the rollout
        double *ce = ck + (size_t)nseg * 2 * n3;
        TRY(load_state<R>(s, ce, ce + n3));
        if (g_x0) CK(cudaMemcpyAsync(g_x0, XB, nb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream));
        if (g_v0) CK(cudaMemcpyAsync(g_v0, VB, nb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream));
        double th[2 * MAXT2];
        CK(cudaMemcpyAsync(th, s->b_adj_theta.ptr, sizeof(th), cudaMemcpyDeviceToHost, s->stream));
        CK(cudaStreamSynchronize(s->stream));
        TRY(s->read_ctrl());
        TRY(s->check_device_errors());
        fold_theta(*s, th, g_eps, g_sigma);
        return LJSEL_OK;
    });
}

}  // extern "C"
