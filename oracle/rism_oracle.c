/*
 * rism_oracle.c -- plain FP64 CPU oracle for the 3D-RISM initialization path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * CPU-baseline leg of the benchmark may load this code.  It shares no code,
 * header, table or constant generator with the CUDA library; it is slow on
 * purpose and written so that each function can be checked against the
 * paper by eye.
 *
 * What it evaluates (Wilson, Krasny & Luchko, "Accelerating the 3D-RISM
 * theory of molecular solvation with treecode summation and cut-offs"):
 *   - u_s(r): solute-solvent potential energy, Coulomb + Lennard-Jones
 *     (Sec. 2.1, the potential in the KH closure; LJ form A/r^12 - B/r^6 and
 *     its truncation, Sec. 2.6, eq. (ulj-trunc));
 *   - c_s(r): real-space DCF long-range asymptotics, Sec. 2.2, eq. (dcf-r);
 *   - h_s(r): real-space TCF long-range asymptotics, Sec. 2.2, eq. (tcf-r);
 *   - I_s: the analytic LJ truncation correction integral, Sec. 2.6;
 *   - dL/dR_i, dL/dq_i, dL/dsigma_i, dL/deps_i of L = sum_s sum_r
 *     [G_u u + G_c c + G_h h] (the paper has no gradient; these are the
 *     plain derivatives of the three definitions above);
 *   - T_s: the all-space integral of eq. (excess-chemical-potential-LRA)
 *     (Sec. 2.2), as a double sum over atom pairs of 1D integrals;
 *   - c_s(k), h_s(k): the reciprocal-space asymptotics of eq. (dcf-k) and
 *     eq. (tcf-k) on the grid's reciprocal lattice, with the frequency
 *     cut-off of Sec. 2.5 (its bound eq. (k-space-dcf-err) and root);
 *   - the Taylor coefficients of the cluster-particle treecode (Sec. 2.3,
 *     Sec. 2.4) by the paper's recurrences, and the Taylor approximation of
 *     one cluster's well-separated particles (eq. (taylor_approximation)).
 *
 * Readings of the paper taken here (the paper is silent or ambiguous):
 *   - Gaussian-unit formulas are multiplied by the Coulomb constant k_e
 *     (kcal A / (mol e^2)); beta = 1/(k_B T).
 *   - c carries no dielectric constant; h carries 1/eps_r.
 *   - kappa is the total Debye screening of the ionic solvent species:
 *     kappa^2 = 4 pi beta k_e sum_ions rho_j q_j^2 / eps_r.
 *   - LJ parameters mix by Lorentz-Berthelot: sigma_is = (sigma_i+sigma_s)/2,
 *     eps_is = sqrt(eps_i eps_s), u = 4 eps_is [(sigma/d)^12 - (sigma/d)^6].
 *   - The cut-off keeps pairs with d < r_cut and drops d >= r_cut.
 *   - A grid point exactly on an atom: u = +inf (the r^-12 wall dominates),
 *     c and h take their finite d -> 0 limits.
 *
 * Sums over atoms run in index order with Neumaier compensation.  Build with
 * -ffp-contract=off and without -ffast-math so the compensation survives.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
#define ORC_SQRT_PI 1.77245385090551602730

/* ---------------------------------------------------------------- sums */
typedef struct { double s, c; int pinf, ninf; } nsum_t;

static void ns_init(nsum_t* a) { a->s = 0.0; a->c = 0.0; a->pinf = 0; a->ninf = 0; }

static void ns_add(nsum_t* a, double v)
{
    if (isinf(v)) { if (v > 0) a->pinf = 1; else a->ninf = 1; return; }
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}

static double ns_get(const nsum_t* a)
{
    if (a->pinf && a->ninf) return NAN;
    if (a->pinf) return INFINITY;
    if (a->ninf) return -INFINITY;
    return a->s + a->c;
}

/* ------------------------------------------------------- physical setup */

/* beta = 1/(k_B T), Sec. 2.1 */
double orc_beta(double k_B, double T) { return 1.0 / (k_B * T); }

/* Debye screening of the ionic co-solvent (Sec. 2.2, the kappa_D of
 * eq. (tcf-r)); reading: one total kappa from every ionic site. */
double orc_kappa(int32_t S, const double* qs, const double* rho, const int32_t* is_ion,
                 double beta, double k_e, double eps_r)
{
    double acc = 0.0;
    for (int32_t s = 0; s < S; ++s)
        if (is_ion && is_ion[s]) acc += rho[s] * qs[s] * qs[s];
    return sqrt(4.0 * ORC_PI * beta * k_e * acc / eps_r);
}

/* Lennard-Jones pair energy with Lorentz-Berthelot mixing, in its
 * sigma/epsilon form (A = 4 eps sigma^12, B = 4 eps sigma^6, Sec. 2.6). */
static double lj_pair(double sig_is, double eps_is, double d)
{
    double sr = sig_is / d;
    double sr6 = sr * sr * sr * sr * sr * sr;
    return 4.0 * eps_is * (sr6 * sr6 - sr6);
}

/* Per-pair cut-off from a tolerance (Sec. 2.6): the largest r with
 * |u_LJ(r)| = tol, so that |u| <= tol everywhere beyond it.  Solved by
 * bisection until the bracket stops shrinking. */
double orc_lj_rcut_tol(double sig_is, double eps_is, double tol)
{
    if (eps_is <= 0.0) return 0.0;
    double rmin = pow(2.0, 1.0 / 6.0) * sig_is;
    double lo, hi;
    if (tol < eps_is) {
        /* attractive tail: |u| decreases from eps at rmin to 0 */
        lo = rmin;
        hi = rmin;
        while (fabs(lj_pair(sig_is, eps_is, hi)) > tol) hi *= 2.0;
        for (int it = 0; it < 4000; ++it) {
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (fabs(lj_pair(sig_is, eps_is, mid)) > tol) lo = mid; else hi = mid;
        }
        return hi;
    }
    /* tol >= eps: the repulsive wall, u decreasing from +inf to 0 at sigma */
    lo = 0.5 * sig_is;
    while (lj_pair(sig_is, eps_is, lo) < tol) lo *= 0.5;
    hi = sig_is;
    for (int it = 0; it < 4000; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (lj_pair(sig_is, eps_is, mid) > tol) lo = mid; else hi = mid;
    }
    return hi;
}

/* LJ truncation correction integral of Sec. 2.6:
 * I_s = sum_i 4 pi int_{rc}^inf u_is(r) r^2 dr
 *     = sum_i 4 pi (A_is / (9 rc^9) - B_is / (3 rc^3)).
 * rcut[s*n + i] <= 0 means "no cut-off" and contributes nothing. */
void orc_lj_tail(int64_t n, const double* sigma, const double* eps, int32_t S, const double* sigs,
                 const double* epss, const double* rcut, double* out)
{
    for (int32_t s = 0; s < S; ++s) {
        nsum_t acc;
        ns_init(&acc);
        for (int64_t i = 0; i < n; ++i) {
            double rc = rcut[(int64_t)s * n + i];
            if (!(rc > 0.0)) continue;
            double sg = 0.5 * (sigma[i] + sigs[s]);
            double ep = sqrt(eps[i] * epss[s]);
            double A = 4.0 * ep * pow(sg, 12.0);
            double B = 4.0 * ep * pow(sg, 6.0);
            ns_add(&acc, 4.0 * ORC_PI * (A / (9.0 * pow(rc, 9.0)) - B / (3.0 * pow(rc, 3.0))));
        }
        out[s] = ns_get(&acc);
    }
}

/* ------------------------------------------------ long-range kernels */

typedef struct {
    double eta, kappa, a;   /* a = kappa eta / 2 */
    double ea2;             /* exp(a^2) */
    double bh[10];          /* phi_h(d) = sum_{odd n} bh[n] d^(n-1) for small d */
    double small_x;         /* use the series below this x = d / eta */
} lra_t;

/* Series of the TCF kernel phi_h(d) = e^{a^2}[e^{-kd} erfc(a-x) - e^{kd} erfc(a+x)]/d
 * about d = 0.  The bracket B(d) = e^{a^2}(f(d) - f(-d)) with
 * f(d) = e^{-kappa d} erfc(a - d/eta) is odd, so phi_h = sum_{odd n} B^(n)(0) d^(n-1)/n!.
 * With E(d) = erfc(a - d/eta): e^{a^2} E(0) = erfcx(a) and, for k >= 1,
 * e^{a^2} E^(k)(0) = (2/(eta sqrt(pi))) eta^(1-k) H_{k-1}(a) (physicists' Hermite).
 * Leibniz: f^(n)(0) = sum_k C(n,k) (-kappa)^(n-k) E^(k)(0). */
static void lra_series(lra_t* L)
{
    double H[12];
    H[0] = 1.0;
    H[1] = 2.0 * L->a;
    for (int k = 1; k < 11; ++k) H[k + 1] = 2.0 * L->a * H[k] - 2.0 * k * H[k - 1];
    double Et[12];
    /* e^{a^2} erfc(a) written from its definition; for the small a of
     * physical Debye lengths this is well conditioned. */
    Et[0] = exp(L->a * L->a) * erfc(L->a);
    for (int k = 1; k < 12; ++k) Et[k] = (2.0 / (L->eta * ORC_SQRT_PI)) * pow(L->eta, 1 - k) * H[k - 1];
    for (int n = 0; n < 10; ++n) L->bh[n] = 0.0;
    double fact = 1.0;
    for (int n = 1; n < 10; ++n) {
        fact *= n;
        if ((n & 1) == 0) continue;
        double f = 0.0, binom = 1.0;
        for (int k = 0; k <= n; ++k) {
            if (k > 0) binom = binom * (n - k + 1) / k;
            f += binom * pow(-L->kappa, n - k) * Et[k];
        }
        L->bh[n] = 2.0 * f / fact;
    }
}

static void lra_init(lra_t* L, double eta, double kappa)
{
    L->eta = eta;
    L->kappa = kappa;
    L->a = 0.5 * kappa * eta;
    L->ea2 = exp(L->a * L->a);
    L->small_x = 0.02;
    lra_series(L);
}

/* DCF kernel of eq. (dcfphi): erf(d/eta)/d; d -> 0 limit 2/(eta sqrt(pi)). */
static double phi_c(const lra_t* L, double d)
{
    double x = d / L->eta;
    if (x < L->small_x) {
        /* erf(x)/x = (2/sqrt(pi)) sum_m (-1)^m x^(2m) / (m! (2m+1)) */
        double x2 = x * x;
        double s = 1.0 - x2 / 3.0 + x2 * x2 / 10.0 - x2 * x2 * x2 / 42.0 + x2 * x2 * x2 * x2 / 216.0;
        return 2.0 / (L->eta * ORC_SQRT_PI) * s;
    }
    return erf(x) / d;
}

/* TCF kernel of eq. (tcfpsi) times the e^{kappa^2 eta^2/4} prefactor of
 * eq. (tcf-r). */
static double phi_h(const lra_t* L, double d)
{
    double x = d / L->eta;
    if (x < L->small_x) {
        double d2 = d * d;
        return L->bh[1] + d2 * (L->bh[3] + d2 * (L->bh[5] + d2 * (L->bh[7] + d2 * L->bh[9])));
    }
    double k = L->kappa, a = L->a;
    return L->ea2 * (exp(-k * d) * erfc(a - x) - exp(k * d) * erfc(a + x)) / d;
}

/* g_c(d) = phi_c'(d) / d, finite at d = 0 (used by the gradient). */
static double gphi_c(const lra_t* L, double d)
{
    double eta = L->eta, x = d / eta;
    double C0 = 2.0 / (eta * ORC_SQRT_PI);
    if (x < L->small_x) {
        /* d/dd of C0 sum_m (-1)^m x^(2m)/(m!(2m+1)) divided by d */
        double x2 = x * x;
        double s = -2.0 / 3.0 + x2 * (4.0 / 10.0) - x2 * x2 * (6.0 / 42.0) + x2 * x2 * x2 * (8.0 / 216.0)
                   - x2 * x2 * x2 * x2 * (10.0 / 1320.0);
        return C0 * s / (eta * eta);
    }
    double dphi = C0 * exp(-x * x) / d - erf(x) / (d * d);
    return dphi / d;
}

/* g_h(d) = phi_h'(d) / d, finite at d = 0. */
static double gphi_h(const lra_t* L, double d)
{
    double x = d / L->eta;
    if (x < L->small_x) {
        double d2 = d * d;
        return 2.0 * L->bh[3] + d2 * (4.0 * L->bh[5] + d2 * (6.0 * L->bh[7] + d2 * 8.0 * L->bh[9]));
    }
    double k = L->kappa, a = L->a, eta = L->eta;
    double em = exp(-k * d), ep = exp(k * d);
    double B = L->ea2 * (em * erfc(a - x) - ep * erfc(a + x));
    double Bp = -k * L->ea2 * (em * erfc(a - x) + ep * erfc(a + x))
                + 4.0 / (eta * ORC_SQRT_PI) * exp(-x * x);
    return (Bp / d - B / (d * d)) / d;
}

/* Evaluate the exported kernels at one distance (used by the pin tests). */
void orc_kernels(double eta, double kappa, int64_t m, const double* d, double* pc, double* ph,
                 double* gc, double* gh)
{
    lra_t L;
    lra_init(&L, eta, kappa);
    for (int64_t i = 0; i < m; ++i) {
        if (pc) pc[i] = phi_c(&L, d[i]);
        if (ph) ph[i] = phi_h(&L, d[i]);
        if (gc) gc[i] = gphi_c(&L, d[i]);
        if (gh) gh[i] = gphi_h(&L, d[i]);
    }
}

/* ---------------------------------------------------------- the grids */

/*
 * Fields at grid points.  The grid point with index (i, j, k) sits at
 * origin + h (i, j, k); its flat index is (k ny + j) nx + i.  idx lists the
 * flat indices to evaluate (NULL: all nx ny nz points in order).  Outputs
 * are [S][npts] (npts = number of evaluated points); any of u, c, hh may be
 * NULL.  rcut[s*n + i] <= 0 means no LJ cut-off for that pair.  h is only
 * evaluated when kappa > 0.
 */
int orc_fields(int64_t n, const double* xyz, const double* q, const double* sigma, const double* eps,
               int32_t S, const double* qs, const double* sigs, const double* epss, const double* rcut,
               double beta, double k_e, double eps_r, double eta, double kappa,
               int32_t nx, int32_t ny, int32_t nz, double h, const double* origin,
               int64_t npts, const int64_t* idx, double* u, double* c, double* hh, int32_t nthreads)
{
    lra_t L;
    lra_init(&L, eta, kappa);
    int64_t total = idx ? npts : (int64_t)nx * ny * nz;
    double* sig_is = (double*)malloc(sizeof(double) * (size_t)(S * n + 1));
    double* eps_is = (double*)malloc(sizeof(double) * (size_t)(S * n + 1));
    if (!sig_is || !eps_is) { free(sig_is); free(eps_is); return 1; }
    for (int32_t s = 0; s < S; ++s)
        for (int64_t i = 0; i < n; ++i) {
            sig_is[s * n + i] = 0.5 * (sigma[i] + sigs[s]);
            eps_is[s * n + i] = sqrt(eps[i] * epss[s]);
        }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t p = 0; p < total; ++p) {
        int64_t f = idx ? idx[p] : p;
        int64_t ii = f % nx, jj = (f / nx) % ny, kk = f / ((int64_t)nx * ny);
        double rx = origin[0] + h * (double)ii;
        double ry = origin[1] + h * (double)jj;
        double rz = origin[2] + h * (double)kk;
        nsum_t sc, sh;
        ns_init(&sc);
        ns_init(&sh);
        for (int64_t i = 0; i < n; ++i) {
            double dx = rx - xyz[3 * i + 0], dy = ry - xyz[3 * i + 1], dz = rz - xyz[3 * i + 2];
            double d = sqrt(dx * dx + dy * dy + dz * dz);
            if (c) ns_add(&sc, q[i] * phi_c(&L, d));
            if (hh && kappa > 0.0) ns_add(&sh, q[i] * phi_h(&L, d));
        }
        for (int32_t s = 0; s < S; ++s) {
            if (u) {
                nsum_t su;
                ns_init(&su);
                for (int64_t i = 0; i < n; ++i) {
                    double dx = rx - xyz[3 * i + 0], dy = ry - xyz[3 * i + 1], dz = rz - xyz[3 * i + 2];
                    double d = sqrt(dx * dx + dy * dy + dz * dz);
                    if (d == 0.0) { ns_add(&su, INFINITY); continue; }
                    double e = k_e * qs[s] * q[i] / d;
                    double rc = rcut[s * n + i];
                    if (!(rc > 0.0) || d < rc) e += lj_pair(sig_is[s * n + i], eps_is[s * n + i], d);
                    ns_add(&su, e);
                }
                u[(int64_t)s * total + p] = ns_get(&su);
            }
            if (c) c[(int64_t)s * total + p] = -beta * k_e * qs[s] * ns_get(&sc);
            if (hh) hh[(int64_t)s * total + p] =
                (kappa > 0.0) ? -beta * k_e * qs[s] / (2.0 * eps_r) * ns_get(&sh) : 0.0;
        }
    }
    free(sig_is);
    free(eps_is);
    return 0;
}

/*
 * Gradient of L = sum_s sum_r [G_u,s u_s + G_c,s c_s + G_h,s h_s] with respect
 * to the parameters of the listed atoms.  G_* are full grids [S][nz][ny][nx]
 * (any may be NULL).  For each listed atom a, out[a*8 + 0..7] =
 * dL/dx, dL/dy, dL/dz, dL/dq, dL/dsigma, dL/deps, 0, 0.
 * The cut-off's step at r_cut is not differentiated (it is a delta function).
 * Per z-plane partial sums are combined in plane order, so the result does
 * not depend on the thread count.
 */
int orc_grad(int64_t n, const double* xyz, const double* q, const double* sigma, const double* eps,
             int32_t S, const double* qs, const double* sigs, const double* epss, const double* rcut,
             double beta, double k_e, double eps_r, double eta, double kappa,
             int32_t nx, int32_t ny, int32_t nz, double h, const double* origin,
             const double* gu, const double* gc, const double* gh,
             int64_t natoms, const int64_t* atoms, double* out, int32_t nthreads)
{
    lra_t L;
    lra_init(&L, eta, kappa);
    int64_t M = (int64_t)nx * ny * nz;
    double* part = (double*)calloc((size_t)nz * (size_t)natoms * 6, sizeof(double));
    if (!part) return 1;
    double cfac = -beta * k_e, hfac = -beta * k_e / (2.0 * eps_r);
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int32_t kk = 0; kk < nz; ++kk) {
        for (int64_t a = 0; a < natoms; ++a) {
            int64_t i = atoms[a];
            nsum_t acc[6];
            for (int t = 0; t < 6; ++t) ns_init(&acc[t]);
            for (int32_t jj = 0; jj < ny; ++jj)
                for (int32_t ii = 0; ii < nx; ++ii) {
                    int64_t f = ((int64_t)kk * ny + jj) * nx + ii;
                    double rx = origin[0] + h * (double)ii;
                    double ry = origin[1] + h * (double)jj;
                    double rz = origin[2] + h * (double)kk;
                    double dx = rx - xyz[3 * i + 0], dy = ry - xyz[3 * i + 1], dz = rz - xyz[3 * i + 2];
                    double d = sqrt(dx * dx + dy * dy + dz * dz);
                    if (d == 0.0) continue; /* singular point: not differentiable */
                    double pc = phi_c(&L, d), gcd = gphi_c(&L, d);
                    double ph = kappa > 0.0 ? phi_h(&L, d) : 0.0;
                    double ghd = kappa > 0.0 ? gphi_h(&L, d) : 0.0;
                    /* radial derivative factor: dL/dR_i = -(r - R_i) * sum(...)(dphi/dd)/d */
                    double radial = 0.0, dq = 0.0, dsig = 0.0, deps = 0.0;
                    for (int32_t s = 0; s < S; ++s) {
                        int64_t o = (int64_t)s * M + f;
                        double wu = gu ? gu[o] : 0.0;
                        double wc = gc ? gc[o] * cfac * qs[s] : 0.0;
                        double wh = (gh && kappa > 0.0) ? gh[o] * hfac * qs[s] : 0.0;
                        /* Coulomb: k_e q_s q_i / d, d(1/d)/dd / d = -1/d^3 */
                        dq += wu * k_e * qs[s] / d + wc * pc + wh * ph;
                        radial += q[i] * (wu * k_e * qs[s] * (-1.0 / (d * d * d)) + wc * gcd + wh * ghd);
                        double rc = rcut[s * n + i];
                        if (wu != 0.0 && (!(rc > 0.0) || d < rc)) {
                            double sg = 0.5 * (sigma[i] + sigs[s]);
                            double ep = sqrt(eps[i] * epss[s]);
                            double sr = sg / d, sr6 = sr * sr * sr * sr * sr * sr;
                            /* d/dd of 4 eps (sr^12 - sr^6) = 4 eps (-12 sr^12 + 6 sr^6)/d */
                            radial += wu * 4.0 * ep * (-12.0 * sr6 * sr6 + 6.0 * sr6) / (d * d);
                            /* d/dsigma_is = 4 eps (12 sr^12 - 6 sr^6)/sigma_is, d sigma_is/d sigma_i = 1/2 */
                            dsig += wu * 4.0 * ep * (12.0 * sr6 * sr6 - 6.0 * sr6) / sg * 0.5;
                            /* d/deps_is = u/eps_is, d eps_is/d eps_i = eps_s / (2 eps_is) */
                            deps += wu * 4.0 * (sr6 * sr6 - sr6) * epss[s] / (2.0 * ep);
                        }
                    }
                    /* d d/d R_i = -(r - R_i)/d, so dL/dR_i = -(r - R_i) * radial */
                    ns_add(&acc[0], -dx * radial);
                    ns_add(&acc[1], -dy * radial);
                    ns_add(&acc[2], -dz * radial);
                    ns_add(&acc[3], dq);
                    ns_add(&acc[4], dsig);
                    ns_add(&acc[5], deps);
                }
            for (int t = 0; t < 6; ++t) part[((int64_t)kk * natoms + a) * 6 + t] = ns_get(&acc[t]);
        }
    }
    for (int64_t a = 0; a < natoms; ++a) {
        for (int t = 0; t < 6; ++t) {
            nsum_t acc;
            ns_init(&acc);
            for (int32_t kk = 0; kk < nz; ++kk) ns_add(&acc, part[((int64_t)kk * natoms + a) * 6 + t]);
            out[a * 8 + t] = ns_get(&acc);
        }
        out[a * 8 + 6] = 0.0;
        out[a * 8 + 7] = 0.0;
    }
    free(part);
    return 0;
}

/* ------------------------------------------- all-space LRA integral */

/*
 * The last integral of eq. (excess-chemical-potential-LRA) (Sec. 2.2), per solvent site gamma:
 *   T_gamma = int over all space of [ 1/2 (h_gamma^lr)^2 Theta(Q^U q_gamma) - 1/2 h_gamma^lr c_gamma^lr ] dr,
 * with h^lr of eq. (tcf-r), c^lr of eq. (dcf-r) and Q^U the total solute charge.  The paper computes it "via
 * 1D integrals" and notes its O(N_atom^2) cost (Sec. 4.7).  Both asymptotic functions are sums over atoms of
 * one radial kernel each (phi_h, phi_c above), so the integral is a double sum over atom pairs of
 *   I_hh(R) = int phi_h(|r|) phi_h(|r - R|) dr,    I_hc(R) = int phi_h(|r|) phi_c(|r - R|) dr,
 * R = |R_a - R_b|, and each of these is one 1D integral over the wave number k of the product of the kernels'
 * 3D Fourier transforms (eq. (tcf-k) and eq. (dcf-k) without their prefactors: 8 pi e^{-k^2 eta^2/4}/(k^2 +
 * kappa^2) for phi_h with its e^{kappa^2 eta^2/4} prefactor, 4 pi e^{-k^2 eta^2/4}/k^2 for phi_c):
 *   I(R) = 1/(2 pi^2) int_0^inf k^2 F(k) G(k) sin(kR)/(kR) dk
 *   I_hc(R) = 16 int_0^inf e^{-k^2 eta^2/2} j0(kR) / (k^2 + kappa^2) dk
 *   I_hh(R) = 32 int_0^inf k^2 e^{-k^2 eta^2/2} j0(kR) / (k^2 + kappa^2)^2 dk.
 * The 1D integrals are taken by composite 10-point Gauss-Legendre quadrature up to the wave number where the
 * Gaussian factor falls below 1e-20, on panels no wider than pi/R (half a period of sin(kR)), 0.5/eta, and
 * max(kappa, k)/8 (the Lorentzian factors peak at k = 0 with width kappa).
 */

static const double GL10_X[5] = {0.1488743389816312108848260, 0.4333953941292471907992659,
                                 0.6794095682990244062343274, 0.8650633666889845107320967,
                                 0.9739065285171717200779640};
static const double GL10_W[5] = {0.2955242247147528701738930, 0.2692667193099963550912269,
                                 0.2190863625159820439955349, 0.1494513491505805931457763,
                                 0.0666713443086881375935688};

static double j0s(double x)
{
    if (fabs(x) < 1e-4) { double x2 = x * x; return 1.0 - x2 / 6.0 + x2 * x2 / 120.0; }
    return sin(x) / x;
}

/* I_hc(R), I_hh(R) for m distances (kappa > 0). */
void orc_lra_pair(double eta, double kappa, int64_t m, const double* R, double* Ihc, double* Ihh)
{
    double kmax = sqrt(2.0 * 46.06) / eta; /* e^{-k^2 eta^2 / 2} = 1e-20 */
    double k2 = kappa * kappa;
    for (int64_t i = 0; i < m; ++i) {
        double r = R[i];
        double wmax = 0.5 / eta;
        if (r > 0.0 && ORC_PI / r < wmax) wmax = ORC_PI / r;
        nsum_t shc, shh;
        ns_init(&shc);
        ns_init(&shh);
        double k0 = 0.0;
        while (k0 < kmax) {
            double width = (k0 > kappa ? k0 : kappa) / 8.0;
            if (width > wmax) width = wmax;
            if (k0 + width > kmax) width = kmax - k0;
            double mid = k0 + 0.5 * width, half = 0.5 * width;
            k0 += width;
            for (int g = 0; g < 10; ++g) {
                double k = mid + (g < 5 ? -1.0 : 1.0) * half * GL10_X[g % 5];
                double w = half * GL10_W[g % 5];
                double gau = exp(-0.5 * k * k * eta * eta);
                double den = k * k + k2;
                double j = j0s(k * r);
                ns_add(&shc, w * gau * j / den);
                ns_add(&shh, w * k * k * gau * j / (den * den));
            }
        }
        if (Ihc) Ihc[i] = 16.0 * ns_get(&shc);
        if (Ihh) Ihh[i] = 32.0 * ns_get(&shh);
    }
}

/* Per listed atom a: P_hc[a] = sum_b Q_b I_hc(|R_a - R_b|), P_hh[a] = sum_b Q_b I_hh(...), b over all atoms
 * (b = a included, R = 0). */
int orc_lra_atom_sums(int64_t n, const double* xyz, const double* q, double eta, double kappa, int64_t nlist,
                      const int64_t* atoms, double* Phc, double* Phh, int32_t nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t t = 0; t < nlist; ++t) {
        int64_t a = atoms[t];
        nsum_t shc, shh;
        ns_init(&shc);
        ns_init(&shh);
        for (int64_t b = 0; b < n; ++b) {
            double dx = xyz[3 * a + 0] - xyz[3 * b + 0], dy = xyz[3 * a + 1] - xyz[3 * b + 1];
            double dz = xyz[3 * a + 2] - xyz[3 * b + 2];
            double r = sqrt(dx * dx + dy * dy + dz * dz), ihc, ihh;
            orc_lra_pair(eta, kappa, 1, &r, &ihc, &ihh);
            ns_add(&shc, q[b] * ihc);
            ns_add(&shh, q[b] * ihh);
        }
        Phc[t] = ns_get(&shc);
        Phh[t] = ns_get(&shh);
    }
    return 0;
}

/* T_gamma of every site from the pair sums S_hh = sum_a Q_a P_hh[a], S_hc = sum_a Q_a P_hc[a]:
 * h^lr_gamma = A_gamma sum_a Q_a phi_h, A_gamma = -beta k_e q_gamma / (2 eps_r); c^lr_gamma = B_gamma sum_a Q_a
 * phi_c, B_gamma = -beta k_e q_gamma; Theta(x) = 1 for x > 0, else 0.  Returns S_hh, S_hc in S2[0..1]. */
int orc_lra_integral(int64_t n, const double* xyz, const double* q, int32_t S, const double* qs, double beta,
                     double k_e, double eps_r, double eta, double kappa, double* T, double* S2, int32_t nthreads)
{
    if (!(kappa > 0.0)) {
        for (int32_t s = 0; s < S; ++s) T[s] = 0.0;
        if (S2) { S2[0] = 0.0; S2[1] = 0.0; }
        return 0;
    }
    int64_t* all = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    double* phc = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* phh = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!all || !phc || !phh) { free(all); free(phc); free(phh); return 1; }
    for (int64_t i = 0; i < n; ++i) all[i] = i;
    orc_lra_atom_sums(n, xyz, q, eta, kappa, n, all, phc, phh, nthreads);
    nsum_t shh, shc, qt;
    ns_init(&shh);
    ns_init(&shc);
    ns_init(&qt);
    for (int64_t a = 0; a < n; ++a) {
        ns_add(&shh, q[a] * phh[a]);
        ns_add(&shc, q[a] * phc[a]);
        ns_add(&qt, q[a]);
    }
    double Shh = ns_get(&shh), Shc = ns_get(&shc), Qu = ns_get(&qt);
    for (int32_t s = 0; s < S; ++s) {
        double A = -beta * k_e * qs[s] / (2.0 * eps_r), B = -beta * k_e * qs[s];
        double theta = (Qu * qs[s] > 0.0) ? 1.0 : 0.0;
        T[s] = 0.5 * theta * A * A * Shh - 0.5 * A * B * Shc;
    }
    if (S2) { S2[0] = Shh; S2[1] = Shc; }
    free(all);
    free(phc);
    free(phh);
    return 0;
}

/* ------------------------------------------ reciprocal-space asymptotics */

/*
 * Eq. (dcf-k) and eq. (tcf-k) (Sec. 2.2) on the reciprocal lattice of the grid, with the Coulomb constant k_e
 * of the unit reading:
 *   c_s(k) = -(4 pi beta k_e q_s / k^2) e^{-k^2 eta^2/4} sum_a Q_a e^{i k.(R_a - o)}
 *   h_s(k) = -(4 pi beta k_e q_s / (eps_r (k^2 + kappa^2))) e^{-k^2 eta^2/4} sum_a Q_a e^{i k.(R_a - o)}
 * o = the grid origin, k = 2 pi (m_x/(n_x h), m_y/(n_y h), m_z/(n_z h)) with the frequency layout of a real-to-
 * complex transform: index j_x in [0, n_x/2] is m_x = j_x; along y and z, m = j for j <= (n-1)/2 and j - n
 * above.  The half spectrum is stored [S][n_z][n_y][n_x/2 + 1], re/im interleaved.  c(k = 0) is set to 0 (the
 * 1/k^2 term is not defined there); with kappa = 0 h is 0.  Frequency cut-off (Sec. 2.5): entries with
 * k^2 > kcut^2 are 0 (kcut <= 0: none).  idx lists flat indices into one site's half spectrum (NULL: all).
 */
int orc_kspace(int64_t n, const double* xyz, const double* q, int32_t S, const double* qs, double beta,
               double k_e, double eps_r, double eta, double kappa, int32_t nx, int32_t ny, int32_t nz, double h,
               const double* origin, double kcut, int64_t m, const int64_t* idx, double* c_out, double* h_out,
               int32_t nthreads)
{
    int64_t nxh = nx / 2 + 1;
    int64_t total = idx ? m : nxh * (int64_t)ny * nz;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t p = 0; p < total; ++p) {
        int64_t f = idx ? idx[p] : p;
        int64_t jx = f % nxh, jy = (f / nxh) % ny, jz = f / (nxh * ny);
        double mx = (double)jx;
        double my = (double)(jy <= (ny - 1) / 2 ? jy : jy - ny);
        double mz = (double)(jz <= (nz - 1) / 2 ? jz : jz - nz);
        double kx = 2.0 * ORC_PI * mx / (nx * h), ky = 2.0 * ORC_PI * my / (ny * h), kz = 2.0 * ORC_PI * mz / (nz * h);
        double k2 = kx * kx + ky * ky + kz * kz;
        int keep = !(kcut > 0.0) || k2 <= kcut * kcut;
        double sre = 0.0, sim = 0.0;
        if (keep) {
            nsum_t re, im;
            ns_init(&re);
            ns_init(&im);
            for (int64_t a = 0; a < n; ++a) {
                double ph = kx * (xyz[3 * a + 0] - origin[0]) + ky * (xyz[3 * a + 1] - origin[1]) +
                            kz * (xyz[3 * a + 2] - origin[2]);
                ns_add(&re, q[a] * cos(ph));
                ns_add(&im, q[a] * sin(ph));
            }
            sre = ns_get(&re);
            sim = ns_get(&im);
        }
        double gau = exp(-k2 * eta * eta / 4.0);
        double fc = (keep && k2 > 0.0) ? -4.0 * ORC_PI * beta * k_e * gau / k2 : 0.0;
        double fh = (keep && kappa > 0.0) ? -4.0 * ORC_PI * beta * k_e * gau / (eps_r * (k2 + kappa * kappa)) : 0.0;
        for (int32_t s = 0; s < S; ++s) {
            int64_t o = 2 * ((int64_t)s * total + p);
            if (c_out) { c_out[o] = qs[s] * fc * sre; c_out[o + 1] = qs[s] * fc * sim; }
            if (h_out) { h_out[o] = qs[s] * fh * sre; h_out[o + 1] = qs[s] * fh * sim; }
        }
    }
    return 0;
}

/* The bound of eq. (k-space-dcf-err) (Sec. 2.5) at wave number k, as a true bound for every solute and site:
 * 4 sqrt(2) pi beta k_e max_s |q_s| e^{-k^2 eta^2/4} sum_a |Q_a| / k^2 (the paper prints the signed sum
 * sum_a Q_a, which vanishes for a neutral solute; |sum Q e^{ik.R}| <= sum |Q| is the bound it derives). */
double orc_kspace_bound(double k, double eta, double qmax, double qabs, double beta, double k_e)
{
    return 4.0 * sqrt(2.0) * ORC_PI * beta * k_e * qmax * exp(-k * k * eta * eta / 4.0) * qabs / (k * k);
}

/* The cut-off wave number: the k where the bound equals tol (the bound decreases with k), by bisection. */
double orc_kspace_kcut(double eta, double qmax, double qabs, double beta, double k_e, double tol)
{
    if (!(tol > 0.0) || !(qabs > 0.0) || !(qmax > 0.0)) return 0.0;
    double lo = 1e-6, hi = 1.0;
    while (orc_kspace_bound(hi, eta, qmax, qabs, beta, k_e) > tol) hi *= 2.0;
    if (orc_kspace_bound(lo, eta, qmax, qabs, beta, k_e) <= tol) return lo;
    for (int it = 0; it < 4000; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (orc_kspace_bound(mid, eta, qmax, qabs, beta, k_e) > tol) lo = mid; else hi = mid;
    }
    return hi;
}

/* ----------------------------------------- Taylor cluster-particle expansions */

/*
 * Taylor coefficients a_k(x, y) = (1/k!) d^k/dy^k phi(x, y), |k| <= p, of the cluster-particle treecode of
 * Sec. 2.3 (eq. (taylor_coefficients)), by the recurrences of Sec. 2.3.2 and Sec. 2.4, with r = x - y,
 * rho = |r|, n = |k| >= 1, and a_k = 0 when an index of k is negative:
 *   1/rho (eq. (coulombrecurrence)):
 *     a_k = [ (2 - 1/n) sum_i r_i a_{k-e_i} - (1 - 1/n) sum_i a_{k-2e_i} ] / rho^2
 *   erf(rho/eta)/rho (eq. (dcfrecurrence)), b_k the coefficients of the auxiliary Gaussian
 *   (eq. (dcfauxiliaryrecurrence)) with b_0 = -(eta/sqrt(pi)) e^{-rho^2/eta^2} (the paper does not print it):
 *     b_k = 2/(eta^2 n) [ sum_i r_i b_{k-e_i} - sum_i b_{k-2e_i} ]
 *     a_k = [ (2 - 1/n) sum_i r_i a_{k-e_i} - (1 - 1/n) sum_i a_{k-2e_i} + b_k ] / rho^2
 *   e^{-kappa rho}/rho (eq. (screenedcoulombrecurrence)), b_k the coefficients of e^{-kappa rho}
 *   (eq. (screenedcoulombauxiliaryrecurrence), b_0 = e^{-kappa rho}); the auxiliary term enters with
 *   kappa/n (printed: kappa), which the exact derivatives require:
 *     b_k = (kappa/n) [ sum_i r_i a_{k-e_i} - sum_i a_{k-2e_i} ]
 *     a_k = [ (2 - 1/n) sum_i r_i a_{k-e_i} - (1 - 1/n) sum_i a_{k-2e_i}
 *             + (kappa/n) ( sum_i r_i b_{k-e_i} - sum_i b_{k-2e_i} ) ] / rho^2
 * Coefficients are stored in graded order: level n = |k| in turn, within a level k1 from n down to 0, then k2
 * from n - k1 down to 0: index n(n+1)(n+2)/6 + i(i+1)/2 + (i - k2), i = n - k1.
 */
static int64_t tay_index(int k1, int k2, int k3)
{
    int n = k1 + k2 + k3, i = n - k1;
    return (int64_t)n * (n + 1) * (n + 2) / 6 + (int64_t)i * (i + 1) / 2 + (i - k2);
}

static double tay_get(const double* a, int k1, int k2, int k3)
{
    if (k1 < 0 || k2 < 0 || k3 < 0) return 0.0;
    return a[tay_index(k1, k2, k3)];
}

/* kind 0: 1/rho, 1: erf(rho/eta)/rho, 2: e^{-kappa rho}/rho.  a: C(p+3, 3) coefficients. */
int orc_taylor_coeffs(int32_t kind, int32_t p, double rx, double ry, double rz, double eta, double kappa, double* a)
{
    const double r[3] = {rx, ry, rz};
    double rho2 = rx * rx + ry * ry + rz * rz, rho = sqrt(rho2);
    int64_t nc = (int64_t)(p + 1) * (p + 2) * (p + 3) / 6;
    double* b = (double*)calloc((size_t)nc, sizeof(double));
    if (!b) return 1;
    if (kind == 0) a[0] = 1.0 / rho;
    else if (kind == 1) { a[0] = erf(rho / eta) / rho; b[0] = -(eta / ORC_SQRT_PI) * exp(-rho2 / (eta * eta)); }
    else { a[0] = exp(-kappa * rho) / rho; b[0] = exp(-kappa * rho); }
    for (int n = 1; n <= p; ++n) {
        for (int k1 = n; k1 >= 0; --k1)
            for (int k2 = n - k1; k2 >= 0; --k2) {
                int k3 = n - k1 - k2;
                int k[3] = {k1, k2, k3};
                double s1a = 0.0, s2a = 0.0, s1b = 0.0, s2b = 0.0;
                for (int d = 0; d < 3; ++d) {
                    int m1[3] = {k[0], k[1], k[2]}, m2[3] = {k[0], k[1], k[2]};
                    m1[d] -= 1;
                    m2[d] -= 2;
                    s1a += r[d] * tay_get(a, m1[0], m1[1], m1[2]);
                    s2a += tay_get(a, m2[0], m2[1], m2[2]);
                    s1b += r[d] * tay_get(b, m1[0], m1[1], m1[2]);
                    s2b += tay_get(b, m2[0], m2[1], m2[2]);
                }
                int64_t c = tay_index(k1, k2, k3);
                double v = (2.0 - 1.0 / n) * s1a - (1.0 - 1.0 / n) * s2a;
                if (kind == 1) {
                    b[c] = 2.0 / (eta * eta * n) * (s1b - s2b);
                    v += b[c];
                } else if (kind == 2) {
                    v += kappa / n * (s1b - s2b);
                    b[c] = kappa / n * (s1a - s2a);
                }
                a[c] = v / rho2;
            }
    }
    free(b);
    return 0;
}

/* The Taylor approximation of eq. (taylor_approximation) for one cluster: the moments
 * m_k = sum_j q_j (-1)^{|k|} a_k(x_c, y_j) of the listed particles about the centre x_c, evaluated at the m
 * points x_i as sum_k m_k (x_i - x_c)^k. */
int orc_taylor_eval(int32_t kind, int32_t p, const double* xc, int64_t n, const double* xyz, const double* q,
                    double eta, double kappa, int64_t m, const double* pts, double* out)
{
    int64_t nc = (int64_t)(p + 1) * (p + 2) * (p + 3) / 6;
    double* mom = (double*)calloc((size_t)nc, sizeof(double));
    double* a = (double*)malloc(sizeof(double) * (size_t)nc);
    if (!mom || !a) { free(mom); free(a); return 1; }
    for (int64_t j = 0; j < n; ++j) {
        if (orc_taylor_coeffs(kind, p, xc[0] - xyz[3 * j], xc[1] - xyz[3 * j + 1], xc[2] - xyz[3 * j + 2], eta,
                              kappa, a)) { free(mom); free(a); return 1; }
        for (int nn = 0; nn <= p; ++nn)
            for (int k1 = nn; k1 >= 0; --k1)
                for (int k2 = nn - k1; k2 >= 0; --k2) {
                    int64_t c = tay_index(k1, k2, nn - k1 - k2);
                    mom[c] += q[j] * ((nn & 1) ? -1.0 : 1.0) * a[c];
                }
    }
    for (int64_t i = 0; i < m; ++i) {
        double t[3] = {pts[3 * i] - xc[0], pts[3 * i + 1] - xc[1], pts[3 * i + 2] - xc[2]};
        nsum_t acc;
        ns_init(&acc);
        for (int nn = 0; nn <= p; ++nn)
            for (int k1 = nn; k1 >= 0; --k1)
                for (int k2 = nn - k1; k2 >= 0; --k2) {
                    int k3 = nn - k1 - k2;
                    ns_add(&acc, mom[tay_index(k1, k2, k3)] * pow(t[0], k1) * pow(t[1], k2) * pow(t[2], k3));
                }
        out[i] = ns_get(&acc);
    }
    free(mom);
    free(a);
    return 0;
}
