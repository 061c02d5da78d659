/*
 * ljoracle.c -- plain, slow, FP64 CPU oracle for the cutoff Lennard-Jones
 * hot path of "Algorithm Selection in Short-Range Molecular Dynamics
 * Simulations" (arXiv 2505.03438).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline / reference arm of the benchmark may load this library.  The
 * GPU library shares no code, header, table or helper with it, and never
 * calls it.
 *
 * The paper prints no formulas.  It names the objects this file writes out
 * from their textbook definitions:
 *   - Sec. 2.1: point masses moved by Newton's equations with the
 *     Stormer-Verlet integrator; forces from the Lennard-Jones potential;
 *     pairs farther apart than the cutoff r_c are neglected; Newton's third
 *     law (N3L) lets one evaluation serve both particles of a pair.
 *   - Sec. 2.2.1: linked cells of side r_c + skin scaled by the cell size
 *     factor (CSF) and stretched to tile the domain exactly.
 *   - Sec. 4: live statistics of particles per CSF-1 cell bin.
 * Readings where the paper is silent:
 *   - energy-shifted potential: U_s(r) = U(r) - U(r_c) for r < r_c, force
 *     unshifted;
 *   - "within r_c" is strict: a pair counts iff r^2 < r_c^2, and r^2 is
 *     evaluated as (dx*dx + dy*dy) + dz*dz in double with no fused
 *     multiply-add, where dx = x_i - (x_j + k*L) and k in {-1,0,1} is the
 *     minimum image;
 *   - Stormer-Verlet in velocity (kick-drift-kick) form, positions wrapped
 *     into [0, L) after every drift;
 *   - a dimension may instead be closed by reflective walls at 0 and L (the
 *     walled heating-sphere conditions of Sec. 6): no periodic image in it,
 *     and a particle that crosses a wall after a drift is mirrored back with
 *     its velocity component reversed.
 *
 * Compile with -O2 -ffp-contract=off (the build script does).  Every
 * routine is checked on the CPU against closed forms, invariants, lattice
 * sums, a library neighbour search or a second traversal.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_TYPES 4

typedef struct orc_params {
    double box[3];                              /* periodic box lengths      */
    int32_t ntypes;                             /* 1..ORC_MAX_TYPES          */
    int32_t shift;                              /* 1: U shifted to 0 at r_c  */
    double eps[ORC_MAX_TYPES * ORC_MAX_TYPES];  /* row-major, symmetric      */
    double sigma[ORC_MAX_TYPES * ORC_MAX_TYPES];
    double rcut[ORC_MAX_TYPES * ORC_MAX_TYPES];
    int32_t walls[3];                           /* 1: reflective walls in d  */
} orc_params;

/* ---------------------------------------------------------------------- */
/* Pair terms (Sec. 2.1 names the Lennard-Jones potential as the source of
 * the pair force).  U(r) = 4 eps [(sig/r)^12 - (sig/r)^6];
 * the force on i from j is -dU/dr along r_ij/r, i.e. f_over_r * (r_i - r_j)
 * with f_over_r = 24 eps [2 (sig/r)^12 - (sig/r)^6] / r^2.                */
static void lj_terms(double r2, double eps, double sig, double *f_over_r, double *u)
{
    double s2 = (sig * sig) / r2;
    double s6 = s2 * s2 * s2;
    double s12 = s6 * s6;
    *u = 4.0 * eps * (s12 - s6);
    *f_over_r = 24.0 * eps * (2.0 * s12 - s6) / r2;
}

/* Potential energy at distance r, optionally shifted (reading: shift only
 * the energy; the force is the plain LJ force). Exported for the pins.    */
void orc_lj_pair(double r, double eps, double sig, double rc, int32_t shift,
                 double *f_over_r, double *u)
{
    double f, uu;
    lj_terms(r * r, eps, sig, &f, &uu);
    if (shift) {
        double fc, uc;
        lj_terms(rc * rc, eps, sig, &fc, &uc);
        uu -= uc;
    }
    *f_over_r = f;
    *u = uu;
}

/* Minimum-image coefficient k in {-1, 0, 1} such that x_j + k L is the
 * image of x_j nearest to x_i (positions may sit slightly outside [0, L)). */
static int min_image_k(double xi, double xj, double L)
{
    double d = xi - xj;
    if (d > 0.5 * L) return 1;
    if (d < -0.5 * L) return -1;
    return 0;
}

/* Image coefficient of dimension d: the minimum image in a periodic
 * dimension, none between walls.                                          */
static int image_k(const orc_params *p, int d, double xi, double xj)
{
    return p->walls[d] ? 0 : min_image_k(xi, xj, p->box[d]);
}

/* The defining arithmetic of a displacement component and of r^2.        */
static double image_dx(double xi, double xj, double L, int k)
{
    return xi - (xj + (double)k * L);
}
static double r2_of(double dx, double dy, double dz)
{
    double a = dx * dx;
    double b = dy * dy;
    double c = dz * dz;
    return (a + b) + c;
}

void orc_min_image_r2(double xi, double yi, double zi, double xj, double yj, double zj,
                      const double *box, double *r2_out)
{
    double dx = image_dx(xi, xj, box[0], min_image_k(xi, xj, box[0]));
    double dy = image_dx(yi, yj, box[1], min_image_k(yi, yj, box[1]));
    double dz = image_dx(zi, zj, box[2], min_image_k(zi, zj, box[2]));
    *r2_out = r2_of(dx, dy, dz);
}

static double shift_energy(const orc_params *p, int a, int b)
{
    int t = a * p->ntypes + b;
    if (!p->shift) return 0.0;
    double f, u;
    lj_terms(p->rcut[t] * p->rcut[t], p->eps[t], p->sigma[t], &f, &u);
    return u;
}

/* ---------------------------------------------------------------------- */
/* Brute force O(N^2) over unordered pairs i < j with N3L (Sec. 2.1).      *
 * Returns the number of pairs within the cutoff; the first `cap` of them  *
 * are written to pairs[2*k], pairs[2*k+1] (i < j, input indices).         */
int64_t orc_forces_brute(int64_t n, const double *x, const int32_t *type,
                         const orc_params *p, double *F, double *energy,
                         double *virial, int32_t *pairs, int64_t cap)
{
    int nt = p->ntypes;
    double U = 0.0, W = 0.0;
    int64_t count = 0;
    memset(F, 0, sizeof(double) * 3 * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            int t = type[i] * nt + type[j];
            double dx = image_dx(x[3*i+0], x[3*j+0], p->box[0], image_k(p, 0, x[3*i+0], x[3*j+0]));
            double dy = image_dx(x[3*i+1], x[3*j+1], p->box[1], image_k(p, 1, x[3*i+1], x[3*j+1]));
            double dz = image_dx(x[3*i+2], x[3*j+2], p->box[2], image_k(p, 2, x[3*i+2], x[3*j+2]));
            double r2 = r2_of(dx, dy, dz);
            double rc = p->rcut[t];
            if (!(r2 < rc * rc)) continue;
            double f, u;
            lj_terms(r2, p->eps[t], p->sigma[t], &f, &u);
            F[3*i+0] += f * dx; F[3*i+1] += f * dy; F[3*i+2] += f * dz;
            F[3*j+0] -= f * dx; F[3*j+1] -= f * dy; F[3*j+2] -= f * dz;
            U += u - shift_energy(p, type[i], type[j]);
            W += f * r2;
            if (pairs && count < cap) {
                pairs[2*count] = (int32_t)i;
                pairs[2*count+1] = (int32_t)j;
            }
            ++count;
        }
    }
    if (energy) *energy = U;
    if (virial) *virial = W;
    return count;
}

/* ---------------------------------------------------------------------- */
/* Linked cells (Sec. 2.2.1).  Cell side per dimension is L / floor(L /    *
 * cell_min) >= cell_min, i.e. the minimum side stretched to tile the box.  *
 * Cells are held as Hockney head/next chains.  Every particle i visits    *
 * all cells within reach = ceil(r_c,max / side) (one more when the ratio  *
 * is an exact integer, so that rounding at a cell face cannot lose a      *
 * pair) and accumulates only its own force (no N3L), so the loop over i   *
 * is trivially parallel; pair energy and virial are halved.  The image of *
 * cell c+o is (c+o) mod n with shift s = floor((c+o) / n); images with    *
 * |s| > 1 lie at least one box length away and are skipped.  Positions    *
 * may lie up to a fraction of a cell outside [0, L): particle i is binned *
 * by its wrapped position x_i - m_i L (m_i = floor(x_i / L)), and the     *
 * image coefficient of the pair on the positions as given is then         *
 * k = s + m_i - m_j.                                                      */
static int64_t floor_div(int64_t a, int64_t b) { int64_t q = a / b; if ((a % b != 0) && ((a < 0) != (b < 0))) --q; return q; }

int64_t orc_forces_cells(int64_t n, const double *x, const int32_t *type,
                         const orc_params *p, double cell_min, int32_t nthreads,
                         double *F, double *energy, double *virial,
                         int32_t *pairs, int64_t cap)
{
    int nt = p->ntypes;
    double rcmax = 0.0;
    for (int t = 0; t < nt * nt; ++t) if (p->rcut[t] > rcmax) rcmax = p->rcut[t];
    int64_t nc[3], reach[3];
    double side[3];
    for (int d = 0; d < 3; ++d) {
        nc[d] = (int64_t)floor(p->box[d] / cell_min);
        if (nc[d] < 1) nc[d] = 1;
        side[d] = p->box[d] / (double)nc[d];
        reach[d] = (int64_t)ceil(rcmax / side[d] + 1e-9);
    }
    int64_t ncell = nc[0] * nc[1] * nc[2];
    int64_t *head = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    int64_t *next = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *cidx = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)(n > 0 ? n : 1));
    int64_t *mimg = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)(n > 0 ? n : 1));
    for (int64_t c = 0; c < ncell; ++c) head[c] = -1;
    /* insert in reverse so that each chain lists particles in input order */
    for (int64_t i = n - 1; i >= 0; --i) {
        int64_t c3[3];
        for (int d = 0; d < 3; ++d) {
            int64_t m = p->walls[d] ? 0 : (int64_t)floor(x[3*i+d] / p->box[d]);
            double xw = x[3*i+d] - (double)m * p->box[d];
            int64_t c = (int64_t)floor(xw / side[d]);
            if (c < 0) c = 0;
            if (c > nc[d] - 1) c = nc[d] - 1;
            c3[d] = c;
            cidx[3*i+d] = c;
            mimg[3*i+d] = m;
        }
        int64_t c = (c3[2] * nc[1] + c3[1]) * nc[0] + c3[0];
        next[i] = head[c];
        head[c] = i;
    }
    double U = 0.0, W = 0.0;
    int64_t count = 0;
    memset(F, 0, sizeof(double) * 3 * (size_t)n);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64) reduction(+:U,W)
#endif
    for (int64_t i = 0; i < n; ++i) {
        double fx = 0.0, fy = 0.0, fz = 0.0;
        for (int64_t oz = -reach[2]; oz <= reach[2]; ++oz)
        for (int64_t oy = -reach[1]; oy <= reach[1]; ++oy)
        for (int64_t ox = -reach[0]; ox <= reach[0]; ++ox) {
            int64_t raw[3] = { cidx[3*i+0] + ox, cidx[3*i+1] + oy, cidx[3*i+2] + oz };
            int64_t k[3], cw[3];
            int skip = 0;
            for (int d = 0; d < 3; ++d) {
                k[d] = floor_div(raw[d], nc[d]);
                cw[d] = raw[d] - k[d] * nc[d];
                if (k[d] < -1 || k[d] > 1) skip = 1;
                if (p->walls[d] && k[d] != 0) skip = 1;  /* no image between walls */
            }
            if (skip) continue;
            /* a cell reached twice with the same image would double count;
             * it happens only when 2*reach+1 > n, and then the images differ */
            int64_t c = (cw[2] * nc[1] + cw[1]) * nc[0] + cw[0];
            for (int64_t j = head[c]; j >= 0; j = next[j]) {
                if (j == i && k[0] == 0 && k[1] == 0 && k[2] == 0) continue;
                int t = type[i] * nt + type[j];
                double dx = image_dx(x[3*i+0], x[3*j+0], p->box[0], (int)(k[0] + mimg[3*i+0] - mimg[3*j+0]));
                double dy = image_dx(x[3*i+1], x[3*j+1], p->box[1], (int)(k[1] + mimg[3*i+1] - mimg[3*j+1]));
                double dz = image_dx(x[3*i+2], x[3*j+2], p->box[2], (int)(k[2] + mimg[3*i+2] - mimg[3*j+2]));
                double r2 = r2_of(dx, dy, dz);
                double rc = p->rcut[t];
                if (!(r2 < rc * rc)) continue;
                double f, u;
                lj_terms(r2, p->eps[t], p->sigma[t], &f, &u);
                fx += f * dx; fy += f * dy; fz += f * dz;
                U += 0.5 * (u - shift_energy(p, type[i], type[j]));
                W += 0.5 * f * r2;
                if (i < j) {
                    int64_t slot;
#ifdef _OPENMP
#pragma omp atomic capture
#endif
                    slot = count++;
                    if (pairs && slot < cap) {
                        pairs[2*slot] = (int32_t)i;
                        pairs[2*slot+1] = (int32_t)j;
                    }
                }
            }
        }
        F[3*i+0] = fx; F[3*i+1] = fy; F[3*i+2] = fz;
    }
    free(head); free(next); free(cidx); free(mimg);
    if (energy) *energy = U;
    if (virial) *virial = W;
    return count;
}

/* ---------------------------------------------------------------------- */
/* Stormer-Verlet (Sec. 2.1), velocity form: v += dt/2 F/m; x += dt v;     *
 * wrap; F(x); v += dt/2 F/m.  Forces come from the linked-cell routine.   *
 * epot/ekin/vir receive nsteps+1 samples (step 0 .. nsteps).              */
static void wrap_coord(double *x, double L)
{
    if (!isfinite(*x)) return;
    while (*x < 0.0) *x += L;
    while (*x >= L) *x -= L;
}

/* Reflective walls at 0 and L: mirror the position back into the box and
 * reverse the velocity component.                                         */
static void reflect_coord(double *x, double *v, double L)
{
    if (!isfinite(*x)) return;
    if (*x < 0.0) { *x = -*x; *v = -*v; }
    else if (*x > L) { *x = 2.0 * L - *x; *v = -*v; }
}

static double kinetic(int64_t n, const double *v, const int32_t *type, const double *mass)
{
    double ke = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double m = mass[type[i]];
        ke += 0.5 * m * (v[3*i] * v[3*i] + v[3*i+1] * v[3*i+1] + v[3*i+2] * v[3*i+2]);
    }
    return ke;
}

int32_t orc_verlet_run(int64_t n, double *x, double *v, const int32_t *type,
                       const double *mass, const orc_params *p, double cell_min,
                       double dt, int64_t nsteps, int32_t nthreads,
                       double *epot, double *ekin, double *vir)
{
    double *F = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    if (!F) return 1;
    double U, W;
    orc_forces_cells(n, x, type, p, cell_min, nthreads, F, &U, &W, NULL, 0);
    if (epot) epot[0] = U;
    if (vir) vir[0] = W;
    if (ekin) ekin[0] = kinetic(n, v, type, mass);
    for (int64_t s = 1; s <= nsteps; ++s) {
        for (int64_t i = 0; i < n; ++i) {
            double h = 0.5 * dt / mass[type[i]];
            for (int d = 0; d < 3; ++d) {
                v[3*i+d] += h * F[3*i+d];
                x[3*i+d] += dt * v[3*i+d];
                if (p->walls[d]) reflect_coord(&x[3*i+d], &v[3*i+d], p->box[d]);
                else wrap_coord(&x[3*i+d], p->box[d]);
            }
        }
        orc_forces_cells(n, x, type, p, cell_min, nthreads, F, &U, &W, NULL, 0);
        for (int64_t i = 0; i < n; ++i) {
            double h = 0.5 * dt / mass[type[i]];
            for (int d = 0; d < 3; ++d) v[3*i+d] += h * F[3*i+d];
        }
        if (epot) epot[s] = U;
        if (vir) vir[s] = W;
        if (ekin) ekin[s] = kinetic(n, v, type, mass);
    }
    free(F);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Live simulation statistics (Sec. 4): particles are binned into cells    *
 * that mimic a CSF-1 cell (side >= r_c + skin, stretched to tile the box). *
 * out = {mean, std/mean, median, max, nbins, nempty} of the counts per    *
 * bin.  std is the population standard deviation; the median of an even   *
 * number of bins is the mean of the two middle counts (reading).          */
static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

void orc_bin_stats(int64_t n, const double *x, const double *box, double bin_min, double *out)
{
    int64_t nc[3];
    double side[3];
    for (int d = 0; d < 3; ++d) {
        nc[d] = (int64_t)floor(box[d] / bin_min);
        if (nc[d] < 1) nc[d] = 1;
        side[d] = box[d] / (double)nc[d];
    }
    int64_t nb = nc[0] * nc[1] * nc[2];
    int64_t *cnt = (int64_t *)calloc((size_t)nb, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        int64_t c3[3];
        for (int d = 0; d < 3; ++d) {
            int64_t c = (int64_t)floor(x[3*i+d] / side[d]);
            c3[d] = ((c % nc[d]) + nc[d]) % nc[d];
        }
        cnt[(c3[2] * nc[1] + c3[1]) * nc[0] + c3[0]]++;
    }
    double mean = (double)n / (double)nb;
    double var = 0.0;
    int64_t mx = 0, nempty = 0;
    for (int64_t b = 0; b < nb; ++b) {
        double d = (double)cnt[b] - mean;
        var += d * d;
        if (cnt[b] > mx) mx = cnt[b];
        if (cnt[b] == 0) ++nempty;
    }
    var /= (double)nb;
    qsort(cnt, (size_t)nb, sizeof(int64_t), cmp_i64);
    double median = (nb % 2) ? (double)cnt[nb / 2] : 0.5 * ((double)cnt[nb / 2 - 1] + (double)cnt[nb / 2]);
    out[0] = mean;
    out[1] = mean > 0.0 ? sqrt(var) / mean : 0.0;
    out[2] = median;
    out[3] = (double)mx;
    out[4] = (double)nb;
    out[5] = (double)nempty;
    free(cnt);
}

/* ---------------------------------------------------------------------- */
/* Gradients of the force field (the differentiable binary mixture of the  *
 * workload list; the paper itself has no gradient).  Readings, listed in  *
 * the design notes:                                                       *
 *   - the pair set (the mask r^2 < r_c,ab^2) is frozen at the evaluation  *
 *     point, so derivatives are the almost-everywhere derivatives of a    *
 *     fixed sum, and finite differences use the same frozen set;          *
 *   - eps_ab and sigma_ab are one parameter per unordered type pair; the  *
 *     gradient entry (a,b) and (b,a) both hold the derivative with        *
 *     respect to that shared parameter;                                   *
 *   - the energy shift does not enter the force, so it has no gradient.   *
 * With s = r^2 the force on i from j is g(s) r_ij, r_ij = x_i - (x_j+kL): *
 *   g       = 24 eps (2 sig^12 / s^7 - sig^6 / s^4)                       *
 *   dg/ds   = 24 eps (-14 sig^12 / s^8 + 4 sig^6 / s^5)                   *
 *   dg/deps = 24 (2 sig^12 / s^7 - sig^6 / s^4)                           *
 *   dg/dsig = 24 eps (24 sig^11 / s^7 - 6 sig^5 / s^4)                    *
 * and d(g r)/dr = g I + 2 dg/ds r r^T.                                    */
static void lj_force_derivs(double s, double eps, double sig, double *g, double *dg_ds,
                            double *dg_deps, double *dg_dsig)
{
    double sig2 = sig * sig;
    double sig5 = sig2 * sig2 * sig;
    double sig6 = sig5 * sig;
    double sig11 = sig6 * sig5;
    double sig12 = sig6 * sig6;
    double s2 = s * s;
    double s4 = s2 * s2;
    double s5 = s4 * s;
    double s7 = s4 * s2 * s;
    double s8 = s4 * s4;
    *dg_deps = 24.0 * (2.0 * sig12 / s7 - sig6 / s4);
    *g = eps * *dg_deps;
    *dg_ds = 24.0 * eps * (-14.0 * sig12 / s8 + 4.0 * sig6 / s5);
    *dg_dsig = 24.0 * eps * (24.0 * sig11 / s7 - 6.0 * sig5 / s4);
}

static void pair_dx(const double *x, int64_t i, int64_t j, const orc_params *p, double r[3])
{
    for (int d = 0; d < 3; ++d)
        r[d] = image_dx(x[3*i+d], x[3*j+d], p->box[d], image_k(p, d, x[3*i+d], x[3*j+d]));
}

/* Forces over a given list of unordered pairs (the frozen mask), minimum  *
 * image, no cutoff test.                                                  */
void orc_forces_list(int64_t n, const double *x, const int32_t *type, const orc_params *p,
                     const int32_t *pairs, int64_t npairs, double *F)
{
    int nt = p->ntypes;
    memset(F, 0, sizeof(double) * 3 * (size_t)n);
    for (int64_t k = 0; k < npairs; ++k) {
        int64_t i = pairs[2*k], j = pairs[2*k+1];
        int t = type[i] * nt + type[j];
        double r[3];
        pair_dx(x, i, j, p, r);
        double f, u;
        lj_terms(r2_of(r[0], r[1], r[2]), p->eps[t], p->sigma[t], &f, &u);
        for (int d = 0; d < 3; ++d) {
            F[3*i+d] += f * r[d];
            F[3*j+d] -= f * r[d];
        }
    }
}

/* Vector-Jacobian product of the forces over a frozen pair list.  Given   *
 * the cotangent c = dL/dF (n x 3): gx = (dF/dx)^T c (n x 3; a Hessian-    *
 * vector product, since dF/dx = -Hessian of U), and geps/gsig (ntypes^2)  *
 * = d(c . F)/d eps_ab, d(c . F)/d sig_ab.                                 */
void orc_force_vjp(int64_t n, const double *x, const int32_t *type, const orc_params *p,
                   const int32_t *pairs, int64_t npairs, const double *c,
                   double *gx, double *geps, double *gsig)
{
    int nt = p->ntypes;
    memset(gx, 0, sizeof(double) * 3 * (size_t)n);
    memset(geps, 0, sizeof(double) * (size_t)(nt * nt));
    memset(gsig, 0, sizeof(double) * (size_t)(nt * nt));
    for (int64_t k = 0; k < npairs; ++k) {
        int64_t i = pairs[2*k], j = pairs[2*k+1];
        int a = type[i], b = type[j];
        int t = a * nt + b;
        double r[3], u[3];
        pair_dx(x, i, j, p, r);
        double s = r2_of(r[0], r[1], r[2]);
        double g, dgds, dgde, dgdsig;
        lj_force_derivs(s, p->eps[t], p->sigma[t], &g, &dgds, &dgde, &dgdsig);
        /* the pair adds g r to F_i and -g r to F_j: c . F gets (c_i - c_j) . g r */
        for (int d = 0; d < 3; ++d) u[d] = c[3*i+d] - c[3*j+d];
        double ur = u[0] * r[0] + u[1] * r[1] + u[2] * r[2];
        for (int d = 0; d < 3; ++d) {
            double w = g * u[d] + 2.0 * dgds * ur * r[d];
            gx[3*i+d] += w;
            gx[3*j+d] -= w;
        }
        geps[t] += ur * dgde;
        gsig[t] += ur * dgdsig;
        if (a != b) {
            geps[b * nt + a] += ur * dgde;
            gsig[b * nt + a] += ur * dgdsig;
        }
    }
}

/* In-range pair set at x (linked cells), into a fresh buffer, sorted so  *
 * that every sum over it runs in one fixed order.                         */
static int cmp_pair(const void *a, const void *b)
{
    const int32_t *x = (const int32_t *)a, *y = (const int32_t *)b;
    if (x[0] != y[0]) return (x[0] > y[0]) - (x[0] < y[0]);
    return (x[1] > y[1]) - (x[1] < y[1]);
}

static int32_t *pairs_at(int64_t n, const double *x, const int32_t *type, const orc_params *p,
                         double *F, int64_t *np_out)
{
    double rcmax = 0.0;
    for (int t = 0; t < p->ntypes * p->ntypes; ++t) if (p->rcut[t] > rcmax) rcmax = p->rcut[t];
    int64_t np = orc_forces_cells(n, x, type, p, rcmax, 0, F, NULL, NULL, NULL, 0);
    int32_t *pr = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)(np > 0 ? np : 1));
    orc_forces_cells(n, x, type, p, rcmax, 0, F, NULL, NULL, pr, np);
    qsort(pr, (size_t)np, 2 * sizeof(int32_t), cmp_pair);
    *np_out = np;
    return pr;
}

/* Velocity-form Stormer-Verlet (Sec. 2.1) for a differentiated rollout:   *
 * positions are not wrapped (a shift by L changes no force), and the pair *
 * mask of time level t (t = 0 .. nsteps) is either computed (linked       *
 * cells; appended to masks_out with offsets off_out[t] .. off_out[t+1]    *
 * while it fits in cap pairs) or taken frozen from frozen[off[t] ..       *
 * off[t+1]).  xs, vs (optional) receive x_t, v_t for t = 0 .. nsteps.     *
 * Returns the number of mask pairs over all levels.                       */
int64_t orc_rollout(int64_t n, const double *x0, const double *v0, const int32_t *type,
                    const double *mass, const orc_params *p, double dt, int64_t nsteps,
                    double *xs, double *vs, const int32_t *frozen, const int64_t *off,
                    int32_t *masks_out, int64_t cap, int64_t *off_out)
{
    size_t n3 = 3 * (size_t)n;
    double *x = (double *)malloc(sizeof(double) * (n3 ? n3 : 1));
    double *v = (double *)malloc(sizeof(double) * (n3 ? n3 : 1));
    double *F = (double *)malloc(sizeof(double) * (n3 ? n3 : 1));
    memcpy(x, x0, sizeof(double) * n3);
    memcpy(v, v0, sizeof(double) * n3);
    int64_t used = 0;
    for (int64_t t = 0; t <= nsteps; ++t) {
        /* forces at x_t */
        if (frozen) {
            orc_forces_list(n, x, type, p, frozen + 2 * off[t], off[t+1] - off[t], F);
        } else if (!masks_out && !off_out) {
            double rcmax = 0.0;
            for (int k = 0; k < p->ntypes * p->ntypes; ++k) if (p->rcut[k] > rcmax) rcmax = p->rcut[k];
            orc_forces_cells(n, x, type, p, rcmax, 0, F, NULL, NULL, NULL, 0);
        } else {
            int64_t np;
            int32_t *pr = pairs_at(n, x, type, p, F, &np);
            if (off_out) off_out[t] = used;
            if (masks_out && used + np <= cap) memcpy(masks_out + 2 * used, pr, sizeof(int32_t) * 2 * (size_t)np);
            used += np;
            if (off_out) off_out[t + 1] = used;
            free(pr);
        }
        if (t > 0)  /* second half kick of step t-1 */
            for (int64_t i = 0; i < n; ++i)
                for (int d = 0; d < 3; ++d) v[3*i+d] += 0.5 * dt / mass[type[i]] * F[3*i+d];
        if (xs) memcpy(xs + (size_t)t * n3, x, sizeof(double) * n3);
        if (vs) memcpy(vs + (size_t)t * n3, v, sizeof(double) * n3);
        if (t == nsteps) break;
        /* first half kick and drift of step t */
        for (int64_t i = 0; i < n; ++i)
            for (int d = 0; d < 3; ++d) {
                v[3*i+d] += 0.5 * dt / mass[type[i]] * F[3*i+d];
                x[3*i+d] += dt * v[3*i+d];
            }
    }
    free(x); free(v); free(F);
    return used;
}

/* Reverse-mode derivative of orc_rollout (mask computed per level): given *
 * the cotangents xbar, vbar of x_N, v_N, returns those of x_0, v_0 and of  *
 * eps/sigma.  Each step v_h = v_t + c F(x_t), x_{t+1} = x_t + dt v_h,      *
 * v_{t+1} = v_h + c F(x_{t+1}) (c = dt / 2m) is reversed in the opposite   *
 * order, one force VJP per kick.                                          */
void orc_rollout_vjp(int64_t n, const double *x0, const double *v0, const int32_t *type,
                     const double *mass, const orc_params *p, double dt, int64_t nsteps,
                     const double *xbar, const double *vbar, double *gx0, double *gv0,
                     double *geps, double *gsig)
{
    int nt = p->ntypes;
    size_t n3 = 3 * (size_t)n;
    double *xs = (double *)malloc(sizeof(double) * (n3 ? n3 : 1) * (size_t)(nsteps + 1));
    double *F = (double *)malloc(sizeof(double) * (n3 ? n3 : 1));
    double *cot = (double *)malloc(sizeof(double) * (n3 ? n3 : 1));
    double *g = (double *)malloc(sizeof(double) * (n3 ? n3 : 1));
    double ge[ORC_MAX_TYPES * ORC_MAX_TYPES], gs[ORC_MAX_TYPES * ORC_MAX_TYPES];
    orc_rollout(n, x0, v0, type, mass, p, dt, nsteps, xs, NULL, NULL, NULL, NULL, 0, NULL);
    memcpy(gx0, xbar, sizeof(double) * n3);
    memcpy(gv0, vbar, sizeof(double) * n3);
    memset(geps, 0, sizeof(double) * (size_t)(nt * nt));
    memset(gsig, 0, sizeof(double) * (size_t)(nt * nt));
    for (int64_t t = nsteps - 1; t >= 0; --t) {
        for (int level = 1; level >= 0; --level) {
            /* level 1: the kick v_{t+1} = v_h + c F(x_{t+1}); level 0: the kick
             * v_h = v_t + c F(x_t).  Between them, the drift passes dt * xbar
             * on to the velocity cotangent. */
            const double *xl = xs + (size_t)(t + level) * n3;
            for (int64_t i = 0; i < n; ++i)
                for (int d = 0; d < 3; ++d) cot[3*i+d] = 0.5 * dt / mass[type[i]] * gv0[3*i+d];
            int64_t np;
            int32_t *pr = pairs_at(n, xl, type, p, F, &np);
            orc_force_vjp(n, xl, type, p, pr, np, cot, g, ge, gs);
            free(pr);
            for (size_t k = 0; k < n3; ++k) gx0[k] += g[k];
            for (int k = 0; k < nt * nt; ++k) { geps[k] += ge[k]; gsig[k] += gs[k]; }
            if (level == 1)
                for (size_t k = 0; k < n3; ++k) gv0[k] += dt * gx0[k];
        }
    }
    free(xs); free(F); free(cot); free(g);
}

/* ---------------------------------------------------------------------- */
/* Velocity-scaling thermostat (the heating of the walled sphere, Sec. 6): *
 * the temperature T = sum m v^2 / dof (dof = 3N - 3 in a periodic box,    *
 * whose total momentum is conserved; 3N when any dimension has walls) is  *
 * moved towards the target by at most max_change, by scaling every        *
 * velocity with sqrt(T_new / T).  Returns T before the scaling.           */
double orc_thermostat(int64_t n, double *v, const int32_t *type, const double *mass, const orc_params *p,
                      double target, double max_change)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double m = mass[type[i]];
        s += m * (v[3*i] * v[3*i] + v[3*i+1] * v[3*i+1] + v[3*i+2] * v[3*i+2]);
    }
    int walled = p->walls[0] || p->walls[1] || p->walls[2];
    double dof = walled ? 3.0 * (double)n : 3.0 * (double)n - 3.0;
    double T = s / dof;
    if (!(T > 0.0)) return T;
    double dT = target - T;
    if (dT > max_change) dT = max_change;
    if (dT < -max_change) dT = -max_change;
    double f = sqrt((T + dT) / T);
    for (int64_t k = 0; k < 3 * n; ++k) v[k] *= f;
    return T;
}
