/*
 * FP64 CPU oracle for the short-ranged Lennard-Jones MD path of van Meel,
 * Arnold, Frenkel, Portegies Zwart and Belleman, "Harvesting graphics power
 * for MD simulations" (arXiv:0709.3225).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA library is checked against.  It shares no code,
 * header, table or constant with the CUDA path, and nothing in the product
 * path may load it: only tests/, the smoke check and the CPU-baseline leg of
 * bench.py do.
 *
 * Everything is IEEE double precision.  Compile with -ffp-contract=off so
 * that every product and sum is rounded on its own (the binning rule below
 * is defined with separately rounded operations).
 *
 * Readings of the paper that this file encodes (each one restated next to
 * the function that uses it):
 *   - pair force: Section 2, LJ pair force equation, read with the missing
 *     1/sigma factor restored, i.e. F(r) = -dU/dr for
 *     U(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6];
 *   - truncation at rc (Section 2, truncated and shifted force): mode 0 plain
 *     truncation, mode 1 energy shift, mode 2 the paper's force shift;
 *   - periodic cubic box, minimum image (implied by the 26 neighbour cells
 *     of Section 3);
 *   - cell count per dimension n = int[L / rc] (Section 3.2, worked example
 *     L = 11 sigma, rc = 2.5 sigma -> n = 4), generalised to a subdivision k:
 *     n = int[k L / rc] with a (2k+1)^3 stencil;
 *   - velocity Verlet (Section 2, last paragraph; the equations are not in
 *     the paper): kick-drift-kick with mass m.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Pair interaction (Section 2: LJ pair force, truncated and shifted force). */

/* Full LJ pair force F_LJ(r) = (24 eps / sigma) [2 (sigma/r)^13 - (sigma/r)^7]
 * (positive = repulsive) and potential U_LJ(r) = 4 eps [(sigma/r)^12 - (sigma/r)^6]. */
static void lj_full(double r, double eps, double sigma, double *F, double *U)
{
    double s = sigma / r;
    double s6 = s * s * s * s * s * s;
    double s7 = s6 * s;
    double s12 = s6 * s6;
    double s13 = s12 * s;
    *F = (24.0 * eps / sigma) * (2.0 * s13 - s7);
    *U = 4.0 * eps * (s12 - s6);
}

/* Truncated pair force and energy at distance r.
 *   mode 0: F = F_LJ, U = U_LJ for r < rc; 0 beyond.
 *   mode 1: energy shift: F = F_LJ, U = U_LJ - U_LJ(rc) for r < rc.
 *   mode 2: force shift of Section 2: F = F_LJ - F_LJ(rc), and the matching
 *           U = U_LJ - U_LJ(rc) + (r - rc) F_LJ(rc), so that F = -dU/dr.
 * The cutoff is strict: r >= rc gives exactly zero. */
void or_pair(double r, double eps, double sigma, double rc, int mode,
             double *F, double *U)
{
    if (!(r < rc)) { *F = 0.0; *U = 0.0; return; }
    double f, u;
    lj_full(r, eps, sigma, &f, &u);
    if (mode == 1 || mode == 2) {
        double fc, uc;
        lj_full(rc, eps, sigma, &fc, &uc);
        u = u - uc;
        if (mode == 2) {
            f = f - fc;
            u = u + (r - rc) * fc;
        }
    }
    *F = f;
    *U = u;
}

/* ------------------------------------------------------------------------ */
/* Box geometry (Section 3 and the worked example of Section 3.2).           */

/* Number of cells per dimension, n = int[k L / rc]. */
int or_ncells(double L, double rc, int k)
{
    return (int)floor(((double)k * L) / rc);
}

/* Wrap one coordinate into the primary box: w = x - L floor(x / L); a value
 * that rounds up to L is moved to w - L. */
static double wrap1(double x, double L)
{
    double q = floor(x / L);
    double w = x - L * q;
    if (w >= L) w = w - L;
    return w;
}

/* Cell coordinate of a wrapped coordinate: c = trunc(w * s) with s = n / L,
 * clamped to [0, n-1]. */
static int cell1(double w, double s, int n)
{
    int c = (int)(w * s);
    if (c >= n) c = n - 1;
    if (c < 0) c = 0;
    return c;
}

/* Minimum-image displacement component. */
static double min_image(double d, double L)
{
    return d - L * nearbyint(d / L);
}

/* ------------------------------------------------------------------------ */
/* Binning: serial counting sort of particles into cells (the CSR form of the
 * cell lists of Section 3.1).                                               */

/* Outputs (caller-allocated): cell_of[n], count[nc^3], start[nc^3 + 1],
 * perm[n].  Within a cell, particles are in increasing index order.  x is
 * (n, 3) row-major and is not modified. */
void or_bin(int64_t n, const double *x, double L, int nc,
            int32_t *cell_of, int32_t *count, int32_t *start, int32_t *perm)
{
    int64_t ncell = (int64_t)nc * nc * nc;
    double s = (double)nc / L;
    for (int64_t c = 0; c < ncell; c++) count[c] = 0;
    for (int64_t i = 0; i < n; i++) {
        int cx = cell1(wrap1(x[3 * i + 0], L), s, nc);
        int cy = cell1(wrap1(x[3 * i + 1], L), s, nc);
        int cz = cell1(wrap1(x[3 * i + 2], L), s, nc);
        int32_t c = (int32_t)(cx + (int64_t)nc * (cy + (int64_t)nc * cz));
        cell_of[i] = c;
        count[c] += 1;
    }
    start[0] = 0;
    for (int64_t c = 0; c < ncell; c++) start[c + 1] = start[c] + count[c];
    int32_t *fill = (int32_t *)calloc((size_t)ncell, sizeof(int32_t));
    for (int64_t i = 0; i < n; i++) {
        int32_t c = cell_of[i];
        perm[start[c] + fill[c]] = (int32_t)i;
        fill[c] += 1;
    }
    free(fill);
}

/* ------------------------------------------------------------------------ */
/* Forces.                                                                   */

/* Eq. (n2_force): f_i = -sum_{j != i} f(|r_j - r_i|) (r_j - r_i)/|r_j - r_i|,
 * i.e. f_i = sum_j F(r_ij) d_ij / r_ij with d_ij = r_i - r_j taken at the
 * minimum image.  O(N^2) brute force over all pairs i < j.
 * Outputs: f (n, 3); e_part[n] = half the pair energies of each particle
 * (may be NULL); *e_pot = sum over pairs of U; *virial = sum over pairs of
 * r F(r). */
void or_forces_brute(int64_t n, const double *x, double L, double eps,
                     double sigma, double rc, int mode, double *f,
                     double *e_part, double *e_pot, double *virial)
{
    double E = 0.0, W = 0.0;
    for (int64_t i = 0; i < 3 * n; i++) f[i] = 0.0;
    if (e_part) for (int64_t i = 0; i < n; i++) e_part[i] = 0.0;
    for (int64_t i = 0; i < n; i++) {
        for (int64_t j = i + 1; j < n; j++) {
            double d[3];
            for (int k = 0; k < 3; k++)
                d[k] = min_image(x[3 * i + k] - x[3 * j + k], L);
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(r2 < rc * rc)) continue;
            double r = sqrt(r2);
            double F, U;
            or_pair(r, eps, sigma, rc, mode, &F, &U);
            for (int k = 0; k < 3; k++) {
                f[3 * i + k] += F * d[k] / r;
                f[3 * j + k] -= F * d[k] / r;
            }
            if (e_part) { e_part[i] += 0.5 * U; e_part[j] += 0.5 * U; }
            E += U;
            W += r * F;
        }
    }
    *e_pot = E;
    *virial = W;
}

/* Cell-list forces (Section 3): each particle interacts with the particles
 * of its own cell and of the surrounding cells of a (2k+1)^3 stencil, all
 * wrapped periodically; the pair vector is the minimum image.  Requires
 * nc >= 2k+1 so that every stencil cell is distinct.  Every particle sums
 * over all its partners (no third-law halving), in the order: stencil cells
 * dz, dy, dx from -k to k, then particles of the cell in index order.
 * Outputs as or_forces_brute.  Returns -1 if nc < 2k+1. */
int or_forces_cells(int64_t n, const double *x, double L, double eps,
                    double sigma, double rc, int mode, int k, double *f,
                    double *e_part, double *e_pot, double *virial)
{
    int nc = or_ncells(L, rc, k);
    if (nc < 2 * k + 1) return -1;
    int64_t ncell = (int64_t)nc * nc * nc;
    int32_t *cell_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *count = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncell);
    int32_t *start = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncell + 1));
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    or_bin(n, x, L, nc, cell_of, count, start, perm);

    double E = 0.0, W = 0.0;
    double rc2 = rc * rc;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : E, W)
    for (int64_t i = 0; i < n; i++) {
        int32_t c = cell_of[i];
        int cx = (int)(c % nc), cy = (int)((c / nc) % nc), cz = (int)(c / ((int64_t)nc * nc));
        double fi[3] = {0.0, 0.0, 0.0};
        double ei = 0.0, wi = 0.0;
        for (int dz = -k; dz <= k; dz++)
            for (int dy = -k; dy <= k; dy++)
                for (int dx = -k; dx <= k; dx++) {
                    int ux = (cx + dx + nc) % nc;
                    int uy = (cy + dy + nc) % nc;
                    int uz = (cz + dz + nc) % nc;
                    int64_t cn = ux + (int64_t)nc * (uy + (int64_t)nc * uz);
                    for (int32_t s = start[cn]; s < start[cn + 1]; s++) {
                        int32_t j = perm[s];
                        if (j == i) continue;
                        double d[3];
                        for (int q = 0; q < 3; q++)
                            d[q] = min_image(x[3 * i + q] - x[3 * (int64_t)j + q], L);
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (!(r2 < rc2)) continue;
                        double r = sqrt(r2);
                        double F, U;
                        or_pair(r, eps, sigma, rc, mode, &F, &U);
                        for (int q = 0; q < 3; q++) fi[q] += F * d[q] / r;
                        ei += 0.5 * U;
                        wi += 0.5 * r * F;
                    }
                }
        for (int q = 0; q < 3; q++) f[3 * i + q] = fi[q];
        if (e_part) e_part[i] = ei;
        E += ei;
        W += wi;
    }
    *e_pot = E;
    *virial = W;
    free(cell_of); free(count); free(start); free(perm);
    return 0;
}

/* Force on ONE particle i by the definition (all j != i, minimum image,
 * strict cutoff).  Used to check sampled outputs of very large systems. */
void or_force_one(int64_t n, const double *x, double L, double eps,
                  double sigma, double rc, int mode, int64_t i, double *fi,
                  double *ei)
{
    double acc[3] = {0.0, 0.0, 0.0};
    double e = 0.0;
    for (int64_t j = 0; j < n; j++) {
        if (j == i) continue;
        double d[3];
        for (int q = 0; q < 3; q++)
            d[q] = min_image(x[3 * i + q] - x[3 * j + q], L);
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (!(r2 < rc * rc)) continue;
        double r = sqrt(r2);
        double F, U;
        or_pair(r, eps, sigma, rc, mode, &F, &U);
        for (int q = 0; q < 3; q++) acc[q] += F * d[q] / r;
        e += 0.5 * U;
    }
    for (int q = 0; q < 3; q++) fi[q] = acc[q];
    *ei = e;
}

/* Smallest |r - rc| over all pairs of particle i within rc + band, as a
 * diagnostic for pairs whose in/out decision is below working precision.
 * Writes 1 to near[i] if particle i has a partner with |r - rc| < band. */
void or_near_cutoff(int64_t n, const double *x, double L, double rc, int k,
                    double band, int32_t *near)
{
    int nc = or_ncells(L, rc + band, k);
    if (nc < 2 * k + 1) nc = 0;
    for (int64_t i = 0; i < n; i++) near[i] = 0;
    if (nc == 0) {
        for (int64_t i = 0; i < n; i++)
            for (int64_t j = 0; j < n; j++) {
                if (j == i) continue;
                double d[3];
                for (int q = 0; q < 3; q++) d[q] = min_image(x[3 * i + q] - x[3 * j + q], L);
                double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                if (fabs(r - rc) < band) near[i] = 1;
            }
        return;
    }
    int64_t ncell = (int64_t)nc * nc * nc;
    int32_t *cell_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *count = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncell);
    int32_t *start = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncell + 1));
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    or_bin(n, x, L, nc, cell_of, count, start, perm);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; i++) {
        int32_t c = cell_of[i];
        int cx = (int)(c % nc), cy = (int)((c / nc) % nc), cz = (int)(c / ((int64_t)nc * nc));
        for (int dz = -k; dz <= k; dz++)
            for (int dy = -k; dy <= k; dy++)
                for (int dx = -k; dx <= k; dx++) {
                    int64_t cn = (cx + dx + nc) % nc + (int64_t)nc * ((cy + dy + nc) % nc + (int64_t)nc * ((cz + dz + nc) % nc));
                    for (int32_t s = start[cn]; s < start[cn + 1]; s++) {
                        int32_t j = perm[s];
                        if (j == i) continue;
                        double d[3];
                        for (int q = 0; q < 3; q++) d[q] = min_image(x[3 * i + q] - x[3 * (int64_t)j + q], L);
                        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                        if (fabs(r - rc) < band) near[i] = 1;
                    }
                }
    }
    free(cell_of); free(count); free(start); free(perm);
}

/* Per-particle sensitivity of the force sum to rounding of the pair
 * vectors, for tolerance bounds in tests (not part of the method):
 *   K_i = sum_j (|dF/dr(r_ij)| + |F(r_ij)| / r_ij),  S_i = sum_j |F(r_ij)|,
 * over partners within rc (brute force over all j).  dF/dr of the LJ force is
 * (24 eps / sigma^2) [7 (sigma/r)^8 - 26 (sigma/r)^14]; the force shift of
 * mode 2 is a constant and does not change it. */
static void stiffness_one(int64_t n, const double *x, double L, double eps, double sigma,
                          double rc, int mode, int64_t i, double *K, double *S)
{
    double k = 0.0, sacc = 0.0;
    for (int64_t j = 0; j < n; j++) {
        if (j == i) continue;
        double d[3];
        for (int q = 0; q < 3; q++) d[q] = min_image(x[3 * i + q] - x[3 * j + q], L);
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        if (!(r2 < rc * rc)) continue;
        double r = sqrt(r2);
        double F, U;
        or_pair(r, eps, sigma, rc, mode, &F, &U);
        double s = sigma / r;
        double s8 = s * s * s * s * s * s * s * s;
        double s14 = s8 * s * s * s * s * s * s;
        double dF = (24.0 * eps / (sigma * sigma)) * (7.0 * s8 - 26.0 * s14);
        k += fabs(dF) + fabs(F) / r;
        sacc += fabs(F);
    }
    *K = k;
    *S = sacc;
}

/* For the m particles listed in idx (all particles when idx is NULL, m = n). */
void or_stiffness(int64_t n, const double *x, double L, double eps,
                  double sigma, double rc, int mode, const int64_t *idx, int64_t m,
                  double *K, double *S)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < m; q++) {
        int64_t i = idx ? idx[q] : q;
        stiffness_one(n, x, L, eps, sigma, rc, mode, i, &K[q], &S[q]);
    }
}

/* ------------------------------------------------------------------------ */
/* Derivatives for the adjoint (not in the paper: the derivative of Eq.
 * (n2_force) with the Section 2 pair force, used for force matching).       */

/* Pair force F(r) of or_pair and its derivatives dF/dr, dF/dsigma, dF/deps
 * (rc fixed).  F_LJ = 24 eps (2 sigma^12 r^-13 - sigma^6 r^-7);
 * dF_LJ/dr = 24 eps (-26 sigma^12 r^-14 + 7 sigma^6 r^-8);
 * dF_LJ/dsigma = 24 eps (24 sigma^11 r^-13 - 6 sigma^5 r^-7);
 * dF/deps = F / eps (computed without dividing).  Mode 2 subtracts the same
 * expressions at rc (except dF/dr).  Zero for r >= rc. */
void or_pair_deriv(double r, double eps, double sigma, double rc, int mode,
                   double *F, double *dFdr, double *dFds, double *dFde)
{
    if (!(r < rc)) { *F = *dFdr = *dFds = *dFde = 0.0; return; }
    double s6 = pow(sigma, 6.0), s12 = s6 * s6;
    double f1 = 24.0 * (2.0 * s12 * pow(r, -13.0) - s6 * pow(r, -7.0));
    double d1 = 24.0 * (-26.0 * s12 * pow(r, -14.0) + 7.0 * s6 * pow(r, -8.0));
    double g1 = 24.0 * (24.0 * s12 / sigma * pow(r, -13.0) - 6.0 * s6 / sigma * pow(r, -7.0));
    if (mode == 2) {
        f1 -= 24.0 * (2.0 * s12 * pow(rc, -13.0) - s6 * pow(rc, -7.0));
        g1 -= 24.0 * (24.0 * s12 / sigma * pow(rc, -13.0) - 6.0 * s6 / sigma * pow(rc, -7.0));
    }
    *F = eps * f1;
    *dFdr = eps * d1;
    *dFds = eps * g1;
    *dFde = f1;
}

/* Vector-Jacobian product of the cell-list forces: with g_i = dL/dF_i,
 *   dx_i  = sum_j J_ij (g_i - g_j),  J_ij = phi I + (phi'(r)/r) d d^T,
 *           phi = F(r)/r, d = x_i - x_j (minimum image), r = |d|;
 *   d_eps = sum_i g_i . dF_i/deps,   d_sigma = sum_i g_i . dF_i/dsigma,
 * over pairs within rc found through the cell list (as or_forces_cells).
 * dx is overwritten; dparam[0] = d_eps, dparam[1] = d_sigma.  Returns -1 on
 * a bad box. */
int or_forces_vjp(int64_t n, const double *x, double L, double eps, double sigma,
                  double rc, int mode, int k, const double *g, double *dx,
                  double *dparam)
{
    int nc = or_ncells(L, rc, k);
    if (nc < 2 * k + 1) return -1;
    int64_t ncell = (int64_t)nc * nc * nc;
    int32_t *cell_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *count = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncell);
    int32_t *start = (int32_t *)malloc(sizeof(int32_t) * (size_t)(ncell + 1));
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    or_bin(n, x, L, nc, cell_of, count, start, perm);
    double de = 0.0, ds = 0.0, rc2 = rc * rc;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : de, ds)
    for (int64_t i = 0; i < n; i++) {
        int32_t c = cell_of[i];
        int cx = (int)(c % nc), cy = (int)((c / nc) % nc), cz = (int)(c / ((int64_t)nc * nc));
        double acc[3] = {0.0, 0.0, 0.0};
        for (int dz = -k; dz <= k; dz++)
            for (int dy = -k; dy <= k; dy++)
                for (int dxc = -k; dxc <= k; dxc++) {
                    int64_t cn = (cx + dxc + nc) % nc + (int64_t)nc * ((cy + dy + nc) % nc + (int64_t)nc * ((cz + dz + nc) % nc));
                    for (int32_t s = start[cn]; s < start[cn + 1]; s++) {
                        int32_t j = perm[s];
                        if (j == i) continue;
                        double d[3], dg[3];
                        for (int q = 0; q < 3; q++) {
                            d[q] = min_image(x[3 * i + q] - x[3 * (int64_t)j + q], L);
                            dg[q] = g[3 * i + q] - g[3 * (int64_t)j + q];
                        }
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        if (!(r2 < rc2)) continue;
                        double r = sqrt(r2);
                        double F, dFdr, dFds, dFde;
                        or_pair_deriv(r, eps, sigma, rc, mode, &F, &dFdr, &dFds, &dFde);
                        double phi = F / r;
                        double dphi_r = (dFdr / r - F / r2) / r;   /* phi'(r) / r */
                        double ddg = d[0] * dg[0] + d[1] * dg[1] + d[2] * dg[2];
                        double gid = g[3 * i] * d[0] + g[3 * i + 1] * d[1] + g[3 * i + 2] * d[2];
                        for (int q = 0; q < 3; q++) acc[q] += phi * dg[q] + dphi_r * ddg * d[q];
                        de += dFde / r * gid;
                        ds += dFds / r * gid;
                    }
                }
        for (int q = 0; q < 3; q++) dx[3 * i + q] = acc[q];
    }
    dparam[0] = de;
    dparam[1] = ds;
    free(cell_of); free(count); free(start); free(perm);
    return 0;
}

/* Adjoint of nsteps velocity-Verlet steps (the or_vv scheme) from (x0, v0):
 * given gx = dL/dx(T), gv = dL/dv(T) at the end, returns dL/dx0, dL/dv0 and
 * adds dL/d(eps, sigma) to dparam.  The forward states are kept (no
 * checkpointing).  Per step, backwards (h = dt / 2m):
 *   lambda_v += (nothing);  lambda_x += h VJP(x_{n+1}, lambda_v)
 *   lambda_v += dt lambda_x
 *   lambda_x += h VJP(x_n, lambda_v)
 * with the parameter parts of both VJPs (times h) added to dparam.  The wrap
 * of positions has derivative 1.  gx / gv are overwritten with dL/dx0,
 * dL/dv0.  Returns -1 on a bad box. */
int or_vv_adjoint(int64_t n, const double *x0, const double *v0, double L,
                  double eps, double sigma, double rc, int mode, int k, double dt,
                  double mass, int nsteps, double *gx, double *gv, double *dparam)
{
    size_t m = (size_t)(3 * n);
    double *xs = (double *)malloc(sizeof(double) * m * (size_t)(nsteps + 1));
    double *v = (double *)malloc(sizeof(double) * (m > 0 ? m : 1));
    double *f = (double *)malloc(sizeof(double) * (m > 0 ? m : 1));
    double *tmp = (double *)malloc(sizeof(double) * (m > 0 ? m : 1));
    double E, W, dp[2];
    memcpy(xs, x0, sizeof(double) * m);
    memcpy(v, v0, sizeof(double) * m);
    if (or_forces_cells(n, xs, L, eps, sigma, rc, mode, k, f, NULL, &E, &W) != 0) return -1;
    for (int s = 0; s < nsteps; s++) {
        double *xn1 = xs + m * (size_t)(s + 1);
        memcpy(xn1, xs + m * (size_t)s, sizeof(double) * m);
        or_vv(n, xn1, v, f, L, eps, sigma, rc, mode, k, dt, mass, 1, NULL, NULL);
    }
    double h = 0.5 * dt / mass;
    for (int s = nsteps - 1; s >= 0; s--) {
        or_forces_vjp(n, xs + m * (size_t)(s + 1), L, eps, sigma, rc, mode, k, gv, tmp, dp);
        for (size_t q = 0; q < m; q++) gx[q] += h * tmp[q];
        dparam[0] += h * dp[0];
        dparam[1] += h * dp[1];
        for (size_t q = 0; q < m; q++) gv[q] += dt * gx[q];
        or_forces_vjp(n, xs + m * (size_t)s, L, eps, sigma, rc, mode, k, gv, tmp, dp);
        for (size_t q = 0; q < m; q++) gx[q] += h * tmp[q];
        dparam[0] += h * dp[0];
        dparam[1] += h * dp[1];
    }
    free(xs); free(v); free(f); free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Observables.                                                              */

/* Kinetic energy (1/2) m sum v^2 in FP64. */
double or_ekin(int64_t n, const double *v, double mass)
{
    double s = 0.0;
    for (int64_t i = 0; i < 3 * n; i++) s += v[i] * v[i];
    return 0.5 * mass * s;
}

/* ------------------------------------------------------------------------ */
/* Velocity Verlet (Section 2, last paragraph; standard kick-drift-kick):
 *   v <- v + (dt / 2m) f;  x <- x + dt v;  x <- wrap(x);  f <- F(x);
 *   v <- v + (dt / 2m) f.
 * On entry f must hold F(x) (as returned by or_forces_cells); on exit it
 * holds the forces at the final positions.  The cell list is rebuilt from
 * scratch at every force evaluation.  k = 0 takes the forces from the
 * Section 2 all-pairs sum instead (or_forces_brute: Eq. n2_force over every
 * pair at the minimum image, no cells).  e_pot/virial receive the values at
 * the final positions.  Returns -1 on a bad box. */
int or_vv(int64_t n, double *x, double *v, double *f, double L, double eps,
          double sigma, double rc, int mode, int k, double dt, double mass,
          int nsteps, double *e_pot, double *virial)
{
    double h = 0.5 * dt / mass;
    double E = 0.0, W = 0.0;
    for (int step = 0; step < nsteps; step++) {
        for (int64_t q = 0; q < 3 * n; q++) {
            v[q] = v[q] + h * f[q];
            x[q] = wrap1(x[q] + dt * v[q], L);
        }
        if (k == 0)
            or_forces_brute(n, x, L, eps, sigma, rc, mode, f, NULL, &E, &W);
        else if (or_forces_cells(n, x, L, eps, sigma, rc, mode, k, f, NULL, &E, &W) != 0)
            return -1;
        for (int64_t q = 0; q < 3 * n; q++) v[q] = v[q] + h * f[q];
    }
    if (e_pot) *e_pot = E;
    if (virial) *virial = W;
    return 0;
}

/* Capped steepest descent for relaxing random starting configurations:
 * nsteps times, forces F at x, each particle moved by d = alpha F_i, scaled
 * down to length dmax when longer, then wrapped (the initial relaxation of
 * the batched-ensemble workload; not in the paper).  x updated in place;
 * f receives the forces at the final positions.  Returns -1 on a bad box. */
int or_relax(int64_t n, double *x, double *f, double L, double eps, double sigma,
             double rc, int mode, int k, int nsteps, double alpha, double dmax)
{
    double E, W;
    for (int s = 0; s < nsteps; s++) {
        if (or_forces_cells(n, x, L, eps, sigma, rc, mode, k, f, NULL, &E, &W) != 0) return -1;
        for (int64_t i = 0; i < n; i++) {
            double d[3], len = 0.0;
            for (int q = 0; q < 3; q++) {
                d[q] = alpha * f[3 * i + q];
                len += d[q] * d[q];
            }
            len = sqrt(len);
            double sc = len > dmax ? dmax / len : 1.0;
            for (int q = 0; q < 3; q++) x[3 * i + q] = wrap1(x[3 * i + q] + sc * d[q], L);
        }
    }
    return or_forces_cells(n, x, L, eps, sigma, rc, mode, k, f, NULL, &E, &W);
}

/* ------------------------------------------------------------------------ */
/* rand48 linear congruential generator (Section 4, Eq. lrand48):
 *   x_{n+1} = (a x_n + c) mod 2^48,  a = 0x5DEECE66D, c = 0xB
 * (the constants of the POSIX/glibc rand48 family).  The 31-bit nonnegative
 * output of lrand48 is the 31 most significant bits, x >> 17 (Section 4: the
 * d most significant bits for a d-bit type); drand48 is x 2^-48 in [0, 1).
 * srand48(s) starts from x_0 = (s << 16) | 0x330E.
 * or_rand48_series writes x_1 .. x_n from x_0, one serial step at a time:
 * the plain definition that the parallel generator must reproduce. */
#define OR_R48_A 0x5DEECE66DULL
#define OR_R48_C 0xBULL
#define OR_R48_MASK ((1ULL << 48) - 1ULL)

uint64_t or_srand48_state(int64_t seed)
{
    return ((((uint64_t)seed) & 0xFFFFFFFFULL) << 16) | 0x330EULL;
}

void or_rand48_series(uint64_t x0, int64_t n, uint64_t *out)
{
    uint64_t x = x0 & OR_R48_MASK;
    for (int64_t i = 0; i < n; i++) {
        x = (OR_R48_A * x + OR_R48_C) & OR_R48_MASK;
        out[i] = x;
    }
}

/* Jump constants of Eq. lrand48m: x_{n+m} = (A x_n + C) mod 2^48 with
 * A = a^m and C = c (a^{m-1} + ... + a + 1), both mod 2^48.  (The paper's
 * Eq. AC prints the sum up to i = m; m terms, i = 0 .. m-1, are what
 * composing the serial step m times gives.)  Computed here by m-fold
 * composition of the affine map, O(m): plain, not fast. */
void or_rand48_jump(int64_t m, uint64_t *A, uint64_t *C)
{
    uint64_t a = 1, c = 0;
    for (int64_t i = 0; i < m; i++) {
        a = (a * OR_R48_A) & OR_R48_MASK;
        c = (c * OR_R48_A + OR_R48_C) & OR_R48_MASK;
    }
    *A = a;
    *C = c;
}

/* ------------------------------------------------------------------------ */
/* Langevin thermostat (the stochastic thermostat that Section 1 names as
 * the setting where single precision suffices; the paper gives no scheme).
 * Reading: the BAOAB splitting of Leimkuhler and Matthews, one step
 *   B: v += (dt/2m) f;   A: x += (dt/2) v;
 *   O: v = c1 v + c2 sqrt(kT/m) xi,  c1 = exp(-gamma dt), c2 = sqrt(1 - c1^2);
 *   A: x += (dt/2) v, wrap;   f = F(x);   B: v += (dt/2m) f,
 * with xi standard normal.  The normals come from the rand48 series u = x 2^-48
 * (drand48): for step s and particle i, with N particles, the four uniforms
 * u_k = drand48 number (4 s + k) N + i + 1 of the series (k = 0 .. 3) give,
 * by the Box-Muller transform,
 *   r1 = sqrt(-2 ln(1 - u0)), t1 = 2 pi u1:  xi_x = r1 cos t1, xi_y = r1 sin t1,
 *   r2 = sqrt(-2 ln(1 - u2)), t2 = 2 pi u3:  xi_z = r2 cos t2
 * (1 - u in (0, 1], so the logarithm is finite).  The series starts at x0
 * (or_srand48_state of the seed); series[] holds x_1 .. x_{4 N nsteps}.
 * On entry f holds F(x); on exit the forces at the final positions.
 * Returns -1 on a bad box. */
int or_langevin(int64_t n, double *x, double *v, double *f, double L, double eps,
                double sigma, double rc, int mode, int k, double dt, double mass,
                double gamma, double kT, int nsteps, const uint64_t *series,
                double *e_pot, double *virial)
{
    const double h = 0.5 * dt / mass;
    const double c1 = exp(-gamma * dt);
    const double c2 = sqrt(1.0 - c1 * c1);
    const double sd = sqrt(kT / mass);
    const double two_pi = 6.283185307179586476925286766559;
    double E = 0.0, W = 0.0;
    for (int s = 0; s < nsteps; s++) {
        const uint64_t *u = series + (int64_t)4 * n * s;
        for (int64_t i = 0; i < n; i++) {
            double xi[3];
            const double u0 = (double)u[i] * 0x1p-48, u1 = (double)u[n + i] * 0x1p-48;
            const double u2 = (double)u[2 * n + i] * 0x1p-48, u3 = (double)u[3 * n + i] * 0x1p-48;
            const double r1 = sqrt(-2.0 * log(1.0 - u0)), t1 = two_pi * u1;
            const double r2 = sqrt(-2.0 * log(1.0 - u2)), t2 = two_pi * u3;
            xi[0] = r1 * cos(t1);
            xi[1] = r1 * sin(t1);
            xi[2] = r2 * cos(t2);
            for (int q = 0; q < 3; q++) {
                const int64_t j = 3 * i + q;
                double vv = v[j] + h * f[j];
                double xx = x[j] + 0.5 * dt * vv;
                vv = c1 * vv + c2 * sd * xi[q];
                xx = xx + 0.5 * dt * vv;
                x[j] = wrap1(xx, L);
                v[j] = vv;
            }
        }
        if (k == 0)
            or_forces_brute(n, x, L, eps, sigma, rc, mode, f, NULL, &E, &W);
        else if (or_forces_cells(n, x, L, eps, sigma, rc, mode, k, f, NULL, &E, &W) != 0)
            return -1;
        for (int64_t q = 0; q < 3 * n; q++) v[q] = v[q] + h * f[q];
    }
    if (e_pot) *e_pot = E;
    if (virial) *virial = W;
    return 0;
}

/* Threads the OpenMP loops may use (no-op without OpenMP); returns the
 * number in effect. */
int or_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}
