/*
 * rism3d.h -- C ABI of the GB300 3D-RISM initialization library (librism3d.so).
 *
 * The library computes, on one GPU, the grids that non-periodic 3D-RISM needs
 * before its iterations start (Wilson, Krasny & Luchko, "Accelerating the
 * 3D-RISM theory of molecular solvation with treecode summation and
 * cut-offs"):
 *
 *   u_s(r)  = sum_i k_e q_s q_i / d + sum_i [d < rc_is] (A_is/d^12 - B_is/d^6)
 *             solute-solvent potential energy (Sec. 2.1; LJ form and
 *             truncation of Sec. 2.6, eq. (ulj-trunc)), kcal/mol;
 *   c_s(r)  = -beta k_e q_s sum_i q_i erf(d/eta)/d
 *             real-space DCF long-range asymptotics, Sec. 2.2, eq. (dcf-r);
 *   h_s(r)  = -(beta k_e q_s / (2 eps_r)) sum_i q_i e^{a^2}
 *             [e^{-kappa d} erfc(a - d/eta) - e^{kappa d} erfc(a + d/eta)] / d,
 *             a = kappa eta / 2: real-space TCF asymptotics, Sec. 2.2, eq. (tcf-r);
 *   I_s     = sum_i 4 pi int_{rc_is}^inf u_LJ,is(r) r^2 dr
 *             the analytic LJ truncation correction of Sec. 2.6 (kcal A^3/mol);
 *
 * with d = |r - R_i| over a regular grid r = origin + h (i, j, k), solute
 * atoms R_i (charge q_i, LJ sigma_i, eps_i) and solvent sites s (q_s,
 * sigma_s, eps_s).  Mixing: sigma_is = (sigma_i + sigma_s)/2,
 * eps_is = sqrt(eps_i eps_s), A = 4 eps sigma^12, B = 4 eps sigma^6.
 * The sums are the generic pair sum of Sec. 2.3, eq. (pot); the treecode
 * method evaluates their long-range part with a barycentric-Lagrange
 * particle-cluster treecode (near/far split of eq. (exppot), MAC of
 * Sec. 2.3.1) and the short-range part with cell-list cut-offs.
 *
 * Conventions shared by every entry point:
 *  - Every function returns a status and never aborts or traps.  The text of
 *    the last failure of a context is returned by rism_last_error().
 *  - Grids are FP64, layout [S][nz][ny][nx] (x fastest).  Output pointers are
 *    owned by the caller.  They may be device memory (written asynchronously
 *    on the context's stream; the call returns before the kernels finish) or
 *    host memory (the library computes into its own device buffer, copies
 *    back -- the output grids concurrently, on separate copy streams -- and
 *    synchronises the stream before returning).
 *  - Inputs given as host arrays are copied during the call; the caller keeps
 *    ownership and may free them on return.
 *  - The library never keeps a caller pointer beyond the call.
 *  - Calls on one context must not run concurrently from several host
 *    threads.  Distinct contexts are independent.
 *  - Units: A, e, kcal/mol, K.  c and h are dimensionless.
 */
#ifndef RISM3D_H
#define RISM3D_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define RISM_API __attribute__((visibility("default")))
#else
#define RISM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RISM_OK = 0,
    RISM_E_INVALID = 1,     /* bad argument: NULL, size, NaN/Inf, negative sigma or eps ... */
    RISM_E_STATE = 2,       /* call out of order (no solute or solvent yet) */
    RISM_E_NOMEM = 3,       /* device or host allocation failed */
    RISM_E_CUDA = 4,        /* a CUDA runtime error (text in rism_last_error) */
    RISM_E_TIMEOUT = 5,     /* a bounded device wait ran out; the context stays usable */
    RISM_E_UNSUPPORTED = 6  /* option combination not implemented */
} rism_status;

enum { RISM_METHOD_DIRECT = 0, RISM_METHOD_TREECODE = 1 };
/* FP64: every pair term and sum in double (direct method only: the treecode
 * with FP64 returns RISM_E_UNSUPPORTED, its interpolation error is far above
 * FP32 pair rounding).  FP32: pair terms in single precision with exact
 * lattice-relative distances, sums compensated (float-float). */
enum { RISM_PREC_FP64 = 0, RISM_PREC_FP32 = 1 };
/* LJ truncation (Sec. 2.6): none; one cut-off for all pairs; per-pair
 * cut-off from a tolerance |u_LJ(rc)| = lj_tol. */
enum { RISM_LJ_NONE = 0, RISM_LJ_RCUT = 1, RISM_LJ_TOL = 2 };
/* Far-field approximation of the treecode's target boxes: barycentric-Lagrange
 * Chebyshev proxies (interpolated onto the grid), or the paper's Taylor
 * expansion about the box centre with coefficients from the recurrences of
 * Sec. 2.3.2 and Sec. 2.4 (evaluated at every grid point of the box). */
enum { RISM_APPROX_BARYCENTRIC = 0, RISM_APPROX_TAYLOR = 1 };

#define RISM_MAX_SITES 8

typedef struct rism_ctx rism_ctx;

typedef struct {
    int32_t nx, ny, nz;  /* grid points per axis, 1 <= n <= 65535, at most 2^36 points in all */
    double h;            /* spacing (A), > 0 */
    double origin[3];    /* position of grid point (0,0,0) (A) */
} rism_grid_desc;

typedef struct {
    int32_t method;     /* RISM_METHOD_*; default TREECODE */
    int32_t precision;  /* RISM_PREC_*; default FP32 */
    int32_t degree;     /* barycentric-Lagrange degree n: (n+1)^3 Chebyshev proxies per cluster; default 8 */
    double theta;       /* multipole acceptance: (r_batch + r_cluster)/R < theta; default 0.7 */
    int32_t leaf;       /* max atoms per tree leaf; default 64 */
    int32_t batch[3];   /* target batch (grid sub-box) dims; 0 = library default */
    int32_t lj_mode;    /* RISM_LJ_*; default RCUT */
    double lj_rcut;     /* A, for RISM_LJ_RCUT; default 9 */
    double lj_tol;      /* kcal/mol, for RISM_LJ_TOL; default 1e-6 */
    double eta;         /* charge smearing of eq. (dcf-r)/(tcf-r) (A); default 1 */
    double T;           /* K; default 298 */
    double eps_r;       /* solvent dielectric constant; default 78.44 */
    double kappa;       /* Debye kappa (1/A); < 0 = derive from the ionic sites; default -1 */
    double k_e;         /* Coulomb constant, kcal A/(mol e^2); default 332.0522173 */
    double k_B;         /* Boltzmann constant, kcal/(mol K); default 0.0019872041 */
    double r_short;     /* radius of the short-range erfc remainders (A); 0 = 6 eta (FP64) / 5 eta (FP32) */
    int32_t autotune;   /* 1: time the candidate launch shapes once per problem class and cache the winner */
    int64_t wait_limit; /* polls (each may sleep up to 200 ns) before a bounded device wait gives up;
                           default 1<<24 (a few seconds) */
    int32_t debug_flags;/* test hooks, 0 in production.  Bit 0: the direct kernels skip their first
                           bulk copy, so its wait runs out and the call returns RISM_E_TIMEOUT.
                           Bit 1: time the evaluation kernel with CUDA events (rism_info.eval_ms).
                           Bits 4-5 (treecode, autotune off): v + 1 runs launch shape v (0-2; see
                           rism_info.kernel_variant) instead of shape 0. */
    int32_t target_proxies; /* treecode: 1 (default) = grid boxes of 16^3 points and up also take (n+1)^3
                               Chebyshev proxy targets: a cluster that meets the acceptance criterion for a
                               box is summed at the box's proxies and reaches its grid points by
                               interpolation (cluster-particle form, the paper's orientation of Sec. 2.3.1);
                               0 = only the atom clusters take proxies (particle-cluster form). */
    int32_t approx;     /* RISM_APPROX_*; default BARYCENTRIC.  TAYLOR (treecode with target boxes only):
                           the boxes take the order-`degree` Taylor moments of their accepted atoms (1/d and
                           e^{-kappa d}/d recurrences, Sec. 2.3, eq. (taylor_approximation)) instead of
                           Chebyshev proxies; the reverse mode then runs its far part directly. */
} rism_options;

typedef struct {
    double beta, kappa, r_short;
    int64_t natoms;
    int32_t nsite;
    int32_t tree_nodes, tree_proxied, tree_leaves; /* treecode only; tree_proxied: octree nodes given source
                                                      proxies (0 when target boxes take the far field) */
    int64_t direct_pairs;  /* (grid point, atom) pairs evaluated directly by the last call */
    int64_t proxy_pairs;   /* (grid point, proxy point) pairs of the last call */
    int64_t near_pairs;    /* candidate pairs scanned by the cut-off (cell-list) pass */
    int32_t batch[3];      /* target batch dims in use */
    int32_t kernel_variant;/* launch shape chosen (autotuner or default) */
    int32_t launches;      /* kernels launched by the last compute call */
    float eval_ms;         /* CUDA-event duration of the last evaluation kernel(s) (debug_flags bit 1), else 0 */
    float far_ms, near_ms; /* treecode: the far-field and the near-field + epilogue kernels (debug_flags bit 1) */
    float box_ms;          /* treecode: box-level far field (proxy targets, downward pass, interpolation) */
    int32_t tree_boxes;    /* target boxes whose proxies received at least one cluster */
    int64_t cp_pairs;      /* (proxy target, atom) pairs of the box-level far field */
    int64_t near_tested;   /* treecode near field: (point, atom) pairs distance-tested */
    int64_t lj_pairs;      /* ... of them inside the LJ cut-off (LJ evaluated) */
    int64_t sr_pairs;      /* ... of them inside r_short at d > 0 (short-range remainders evaluated) */
} rism_info;

/* Fill *o with the defaults listed above.  Never fails. */
RISM_API void rism_default_options(rism_options* o);

/* Create a context for one grid.  `stream` is a cudaStream_t (NULL = the
 * legacy default stream) on the current device; every kernel and copy of the
 * context runs on it.  `opts` may be NULL (defaults).  On success *out holds
 * a context the caller frees with rism_destroy.  Errors: RISM_E_INVALID for a
 * bad descriptor or options, RISM_E_NOMEM, RISM_E_CUDA. */
RISM_API rism_status rism_grid_create(const rism_grid_desc* grid, const rism_options* opts, void* stream,
                             rism_ctx** out);

/* Set the solute: n atoms (n >= 0), host arrays xyz [n][3] (A), q [n] (e),
 * sigma [n] (A, >= 0) and eps [n] (kcal/mol, >= 0), all copied.  Uploads the
 * atoms and rebuilds the per-pair tables on the next compute call.
 * RISM_E_INVALID on NULL arrays with n > 0, NaN/Inf or negative sigma/eps. */
RISM_API rism_status rism_set_solute(rism_ctx* ctx, int64_t n, const double* xyz, const double* q, const double* sigma,
                            const double* eps);

/* Set the solvent sites (1 <= nsite <= RISM_MAX_SITES): host arrays q, sigma,
 * eps (copied), bulk site number densities rho (1/A^3, nullable: only needed
 * to derive kappa) and ionic flags is_ion (nullable = none ionic).  With
 * opts.kappa < 0, kappa^2 = 4 pi beta k_e sum_{ionic s} rho_s q_s^2 / eps_r
 * (the kappa_D of eq. (tcf-r), read as the total Debye screening). */
RISM_API rism_status rism_set_solvent(rism_ctx* ctx, int32_t nsite, const double* q, const double* sigma,
                             const double* eps, const double* rho, const int32_t* is_ion);

/* u_s(r) for all sites into u [S][nz][ny][nx]; if lj_tail != NULL the
 * per-site truncation integrals I_s (host array [S]) are written too (zero
 * for RISM_LJ_NONE).  RISM_E_STATE before set_solute/set_solvent. */
RISM_API rism_status rism_potential(rism_ctx* ctx, double* u, double* lj_tail);

/* c_s(r) (eq. (dcf-r)) into c_lr and h_s(r) (eq. (tcf-r)) into h_lr, each
 * [S][nz][ny][nx] and nullable.  h_lr needs kappa > 0 (RISM_E_INVALID
 * otherwise). */
RISM_API rism_status rism_asymptotics(rism_ctx* ctx, double* c_lr, double* h_lr);

/* The whole initialization in one pass over the pairs: u, c_lr, h_lr (each
 * nullable) and lj_tail (host [S], nullable).  Same results as
 * rism_potential + rism_asymptotics, sharing the pair distances. */
RISM_API rism_status rism_init(rism_ctx* ctx, double* u, double* c_lr, double* h_lr, double* lj_tail);

/* Reverse mode of L = sum_s sum_r [G_u,s u_s + G_c,s c_s + G_h,s h_s] (a plain
 * sum over grid points, no volume element).  g_u, g_c, g_h: cotangent grids
 * [S][nz][ny][nx] in device memory (any may be NULL = zero).  Outputs, each
 * nullable, in device memory: d_xyz [n][3] = dL/dR_i (the force on atom i is
 * -d_xyz), d_q [n], d_sigma [n], d_eps [n].  The LJ cut-off's step is not
 * differentiated.  Pair terms are recomputed, never stored.  The paper has no
 * gradient; these are the derivatives of the definitions above. */
RISM_API rism_status rism_potential_backward(rism_ctx* ctx, const double* g_u, const double* g_c, const double* g_h,
                                    double* d_xyz, double* d_q, double* d_sigma, double* d_eps);

/* Many solutes (one context each, all on the same device and with the same
 * method/precision/solvent site count) in one launch sequence on the first
 * context's stream: every context's u, c_lr, h_lr (arrays of `count` device
 * pointers; an array or an element may be NULL).  The work of all solutes is
 * drained from one queue by persistent CTAs, and the sequence is captured in
 * a CUDA graph that is replayed while the set of contexts is unchanged.
 * Output must be device memory. */
RISM_API rism_status rism_potential_batched(rism_ctx* const* ctxs, int32_t count, double* const* u, double* const* c_lr,
                                   double* const* h_lr);

/* Reciprocal-space long-range asymptotics, eq. (dcf-k) and eq. (tcf-k)
 * (Sec. 2.2), times k_e as in the real-space forms:
 *   c_s(k) = -(4 pi beta k_e q_s / k^2) e^{-k^2 eta^2/4} sum_a Q_a e^{i k.(R_a - o)}
 *   h_s(k) = -(4 pi beta k_e q_s / (eps_r (k^2 + kappa^2))) e^{-k^2 eta^2/4} sum_a Q_a e^{i k.(R_a - o)}
 * (A^3), o = grid origin, on the reciprocal lattice of the grid in the half-
 * spectrum layout of a real-to-complex transform: c_k, h_k are
 * [S][nz][ny][nx/2+1] complex values stored as (re, im) FP64 pairs, k =
 * 2 pi (m_x/(nx h), m_y/(ny h), m_z/(nz h)) with m_x = j_x and, along y and
 * z, m = j for j <= (n-1)/2 and j - n above (numpy's rfftn frequency
 * order).  c(0) = 0 (the 1/k^2 term has no value there).  Frequency cut-off
 * of Sec. 2.5: with k_tol > 0 the cut-off k_cut solves the bound of
 * eq. (k-space-dcf-err), 4 sqrt(2) pi beta k_e max_s|q_s| e^{-k^2 eta^2/4}
 * sum_a |Q_a| / k^2 = k_tol (read with |Q_a|: the printed signed sum vanishes
 * for a neutral solute), by Newton's method, and every entry with k^2 > k_cut^2
 * is 0; k_tol <= 0 sums the whole half spectrum.  *k_cut (host, nullable)
 * receives the cut-off (0 = none).  c_k, h_k: device or host memory, each
 * nullable (h_k needs kappa > 0, RISM_E_INVALID otherwise).  The structure
 * factor runs on the GPU with FP32 phase tables reduced exactly modulo one
 * cycle and FP32 products with float-float sums.  Synchronises the
 * context's stream.  RISM_E_STATE before set_solute/set_solvent. */
RISM_API rism_status rism_asymptotics_k(rism_ctx* ctx, double k_tol, double* c_k, double* h_k, double* k_cut);

/* The all-space long-range term of the excess chemical potential: the last
 * integral of eq. (excess-chemical-potential-LRA) (Sec. 2.2), per site s,
 *   T_s = int over all space [ 1/2 (h_s^lr)^2 Theta(Q q_s) - 1/2 h_s^lr c_s^lr ] dr
 * (A^3), with h^lr of eq. (tcf-r), c^lr of eq. (dcf-r), Q the total solute
 * charge and Theta(x) = 1 for x > 0, else 0.  Its contribution to mu_ex is
 * k_B T sum_s rho_s T_s (the caller's assembly, as for lj_tail).  It is a
 * double sum over atom pairs, O(N_atom^2) as Sec. 4.7 notes, of the overlap
 * integrals of the kernels of eqs. (tcf-r)/(dcf-r), evaluated in closed form
 * on the GPU with FP32 pair terms and compensated sums.
 * T: host [S], required.  atom_sums: nullable, device or host [n][2]:
 * per atom a (order of rism_set_solute) P_hc = sum_b Q_b I_hc(|R_a - R_b|)
 * and P_hh = sum_b Q_b I_hh(|R_a - R_b|) (e A, b = a included), so that
 * S_hc = sum_a Q_a P_hc and S_hh = sum_a Q_a P_hh give
 * T_s = 1/2 Theta A_s^2 S_hh - 1/2 A_s B_s S_hc, A_s = -beta k_e q_s/(2 eps_r),
 * B_s = -beta k_e q_s.  Without ionic screening (kappa = 0) h^lr vanishes
 * and T = 0.  Synchronises the context's stream.  RISM_E_STATE before
 * set_solute/set_solvent. */
RISM_API rism_status rism_lra_integral(rism_ctx* ctx, double* T, double* atom_sums);

/* The paper's guide to the accuracy parameters for a residual tolerance of
 * the 3D-RISM solution (Sec. 4.2.1 with Table 3, Sec. 4.3.1, Sec. 4.4.1). */
typedef struct {
    /* Table 3: Taylor order of each kernel,
     *   p_TCF     = max(2, (log10(tolerance) + 5.7) / -0.7)   (h_lr),
     *   p_DCF     = max(2, (log10(tolerance) + 1.9) / -0.8)   (c_lr),
     *   p_Coulomb = max(2, (log10(tolerance) + 1.4) / -0.8)   (u),
     * each rounded up to an integer (the rounding that reproduces the orders
     * Table 2 lists for the guide's solutes at tolerance 1e-6: 2, 6 and 6).
     * With RISM_APPROX_TAYLOR one order serves every moment of a box: set
     * degree to the largest order of the outputs wanted. */
    int32_t p_tcf, p_dcf, p_coulomb;
    double mac;      /* Table 3: acceptance parameter 0.3 (set theta to it) */
    int32_t n0;      /* Table 3: 500 target points per leaf; no counterpart here (the target boxes are fixed
                        16^3-point grid boxes) */
    double k_tol;    /* Sec. 4.3.1: error tolerance of the reciprocal-space cut-off (eq. (k-space-dcf-err),
                        the k_tol of rism_asymptotics_k), 0.04 tolerance^0.9 (the fit to the smaller solutes;
                        the paper found tubulin to need 0.006 tolerance^1.1) */
    double lj_tol;   /* Sec. 4.4.1: LJ cut-off tolerance |u_LJ(r_cut)| (the lj_tol of RISM_LJ_TOL), tolerance / 10,
                        the paper's safe default */
} rism_guide;

/* rism_parameter_guide -- fill *g with the guide's parameters for the
 * residual tolerance `tolerance`.  The paper recommends checking a Taylor
 * order against a run at p + 2, and all of these are starting points.
 * tolerance: finite, 0 < tolerance < 1; g: host memory, non-NULL; else
 * RISM_E_INVALID with *g untouched.  Host arithmetic only; needs no context
 * and no GPU. */
RISM_API rism_status rism_parameter_guide(double tolerance, rism_guide* g);

/* Largest solute accepted by rism_init_noalloc. */
#define RISM_NOALLOC_MAX_ATOMS 8192

/* rism_init_noalloc -- the direct-sum initialization without any device
 * allocation.  The paper has no counterpart: this exists for callers that
 * cannot call cudaMalloc -- plug-ins whose host application owns the device
 * memory and forbids other allocators, and embedded or real-time callers
 * that must not allocate after start-up.  It computes what rism_init
 * computes with method RISM_METHOD_DIRECT (FP32 or FP64 pairs;
 * opts->method must be DIRECT) and calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *
 * Its scratch (the per-atom and per-(atom, site) tables) lives in one
 * file-scope __device__ array of 4,063,488 bytes (RISM_NOALLOC_MAX_ATOMS
 * atoms, RISM_MAX_SITES sites), which every GPU that loads the library holds
 * until the process exits.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress) with the device current.
 * Every call shares the array and leaves its contents behind: calls that
 * overlap on the GPU (several streams, several host threads) race and must
 * be serialised by the caller.
 *
 * grid, opts: as for rism_grid_create (same checks).  n (0 <= n <=
 * RISM_NOALLOC_MAX_ATOMS), xyz [n][3], q, sigma, eps: the solute, device or
 * host memory, copied during the call; host arrays get the checks of
 * rism_set_solute before the GPU is touched, device arrays the same checks
 * on the GPU (RISM_E_INVALID after the call, outputs then unspecified).
 * nsite, qs, sigs, epss, rho (nullable), is_ion (nullable): the solvent,
 * host memory, checked as by rism_set_solvent.  u, c_lr, h_lr: outputs
 * [S][nz][ny][nx], each nullable (h_lr needs kappa > 0); they must be device
 * (or managed) memory -- a host pointer returns RISM_E_INVALID and nothing
 * is launched.  stream: cudaStream_t (NULL = legacy default); the call reads
 * the device error word back into host memory and synchronises the stream
 * before returning.  errbuf (nullable, errlen bytes) receives a message on
 * failure.  n above the maximum returns RISM_E_INVALID without touching the
 * GPU. */
RISM_API rism_status rism_init_noalloc(const rism_grid_desc* grid, const rism_options* opts, int64_t n,
                                       const double* xyz, const double* q, const double* sigma, const double* eps,
                                       int32_t nsite, const double* qs, const double* sigs, const double* epss,
                                       const double* rho, const int32_t* is_ion, double* u, double* c_lr,
                                       double* h_lr, void* stream, char* errbuf, size_t errlen);

/* Counters and derived parameters of the context (after a compute call). */
RISM_API rism_status rism_get_info(const rism_ctx* ctx, rism_info* info);

/* Release the context and its device memory (synchronises its stream).
 * NULL is a no-op. */
RISM_API void rism_destroy(rism_ctx* ctx);

/* Text of the last failure on ctx ("" if none; a static message if ctx is
 * NULL).  Valid until the next call on ctx. */
RISM_API const char* rism_last_error(const rism_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* RISM3D_H */
