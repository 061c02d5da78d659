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
 * Readings where the paper is silent (all listed in the design notes):
 *   - energy-shifted potential: U_s(r) = U(r) - U(r_c) for r < r_c, force
 *     unshifted;
 *   - "within r_c" is strict: a pair counts iff r^2 < r_c^2, and r^2 is
 *     evaluated as (dx*dx + dy*dy) + dz*dz in double with no fused
 *     multiply-add, where dx = x_i - (x_j + k*L) and k in {-1,0,1} is the
 *     minimum image;
 *   - Stormer-Verlet in velocity (kick-drift-kick) form, positions wrapped
 *     into [0, L) after every drift.
 *
 * Compile with -O2 -ffp-contract=off (the build script does).  "Parity
 * unpinned" applies to nothing in this file: every routine is pinned by the
 * CPU tests against closed forms, invariants, lattice sums, a library
 * neighbour search or a second traversal.
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
            double dx = image_dx(x[3*i+0], x[3*j+0], p->box[0], min_image_k(x[3*i+0], x[3*j+0], p->box[0]));
            double dy = image_dx(x[3*i+1], x[3*j+1], p->box[1], min_image_k(x[3*i+1], x[3*j+1], p->box[1]));
            double dz = image_dx(x[3*i+2], x[3*j+2], p->box[2], min_image_k(x[3*i+2], x[3*j+2], p->box[2]));
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
            int64_t m = (int64_t)floor(x[3*i+d] / p->box[d]);
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
                wrap_coord(&x[3*i+d], p->box[d]);
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
