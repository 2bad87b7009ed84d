// rism_noalloc.cu -- rism_init_noalloc: the direct-sum initialization without
// any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA stream is
// being captured into a graph (allocation is not a capturable operation),
// plug-ins whose host application owns the device memory pool and forbids
// other allocators, and embedded or real-time callers that must not allocate
// after start-up.  For them this entry point keeps its scratch -- the
// per-atom and per-(atom, site) tables that the context-based API allocates
// with cudaMalloc -- in one file-scope __device__ array of fixed size.  Every
// GPU that loads the library holds that array until the process exits.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "rism_kernels.h"

namespace rism {
namespace {

constexpr int64_t kNoAllocMaxAtoms = RISM_NOALLOC_MAX_ATOMS;
constexpr size_t kAlign = 256;

constexpr size_t round_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Layout of the scratch array for kNoAllocMaxAtoms atoms and kMaxSites sites.
constexpr size_t kOffErr = 0;
constexpr size_t kOffRaw = round_up(sizeof(DevErr));
constexpr size_t kOffGeo = kOffRaw + round_up(sizeof(double) * 6 * kNoAllocMaxAtoms);
constexpr size_t kOffGeoU = kOffGeo + round_up(sizeof(Geo) * kNoAllocMaxAtoms);
constexpr size_t kOffLJd = kOffGeoU + round_up(sizeof(SrcF) * kNoAllocMaxAtoms);
constexpr size_t kOffLJf = kOffLJd + round_up(sizeof(LJd) * kNoAllocMaxAtoms * kMaxSites);
constexpr size_t kScratchBytes = kOffLJf + round_up(sizeof(LJf) * kNoAllocMaxAtoms * kMaxSites);
static_assert(kScratchBytes == 4063488, "the size stated in rism3d.h");

// The scratch itself.  In host code this name is only a stand-in for the
// device object; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[128] = {};  // device address of g_noalloc_scratch per device ordinal

// Once per device, with that device current: look up the array's address.
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

rism_status say(char* buf, size_t len, rism_status s, const char* msg) {
    if (buf && len > 0) {
        std::strncpy(buf, msg, len - 1);
        buf[len - 1] = '\0';
    }
    return s;
}

bool finite_all(const double* a, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

}  // namespace
}  // namespace rism

using namespace rism;

extern "C" RISM_API rism_status rism_init_noalloc(const rism_grid_desc* grid, const rism_options* opts, int64_t n,
                                                  const double* xyz, const double* q, const double* sigma,
                                                  const double* eps, int32_t nsite, const double* qs,
                                                  const double* sigs, const double* epss, const double* rho,
                                                  const int32_t* is_ion, double* u, double* c_lr, double* h_lr,
                                                  void* stream, char* errbuf, size_t errlen) {
    if (!grid || !opts) return say(errbuf, errlen, RISM_E_INVALID, "grid and opts are required");
    if (n < 0 || n > kNoAllocMaxAtoms)
        return say(errbuf, errlen, RISM_E_INVALID,
                   "rism_init_noalloc: atom count outside [0, RISM_NOALLOC_MAX_ATOMS]; use the context API");
    if (n > 0 && (!xyz || !q || !sigma || !eps)) return say(errbuf, errlen, RISM_E_INVALID, "NULL solute array");
    if (nsite < 1 || nsite > kMaxSites || !qs || !sigs || !epss)
        return say(errbuf, errlen, RISM_E_INVALID, "nsite must lie in [1, RISM_MAX_SITES] with q, sigma, eps");
    if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->h > 0.0) || !std::isfinite(grid->h))
        return say(errbuf, errlen, RISM_E_INVALID, "bad grid descriptor");
    const rism_options& o = *opts;
    if (o.method != RISM_METHOD_DIRECT) return say(errbuf, errlen, RISM_E_UNSUPPORTED, "direct method only");
    if (o.precision != RISM_PREC_FP32 && o.precision != RISM_PREC_FP64)
        return say(errbuf, errlen, RISM_E_INVALID, "precision");
    if (!(o.eta > 0 && o.T > 0 && o.eps_r > 0 && o.k_e > 0 && o.k_B > 0) || o.wait_limit < 1)
        return say(errbuf, errlen, RISM_E_INVALID, "eta, T, eps_r, k_e, k_B must be > 0");
    if (o.lj_mode < RISM_LJ_NONE || o.lj_mode > RISM_LJ_TOL ||
        (o.lj_mode == RISM_LJ_RCUT && !(o.lj_rcut > 0)) || (o.lj_mode == RISM_LJ_TOL && !(o.lj_tol > 0)))
        return say(errbuf, errlen, RISM_E_INVALID, "LJ cut-off options");
    if (!finite_all(qs, nsite) || !finite_all(sigs, nsite) || !finite_all(epss, nsite) ||
        (rho && !finite_all(rho, nsite)))
        return say(errbuf, errlen, RISM_E_INVALID, "NaN or Inf in solvent");

    // physical constants (beta, Debye kappa of eq. (tcf-r), d -> 0 limits)
    Phys ph{};
    ph.S = nsite;
    ph.beta = 1.0 / (o.k_B * o.T);
    ph.k_e = o.k_e;
    ph.eps_r = o.eps_r;
    ph.eta = o.eta;
    if (o.kappa >= 0.0) {
        ph.kappa = o.kappa;
    } else {
        double acc = 0.0;
        for (int s = 0; s < nsite; ++s)
            if (is_ion && is_ion[s] && rho) acc += rho[s] * qs[s] * qs[s];
        ph.kappa = std::sqrt(4.0 * M_PI * ph.beta * ph.k_e * acc / ph.eps_r);
    }
    if (h_lr && !(ph.kappa > 0.0)) return say(errbuf, errlen, RISM_E_INVALID, "h_lr needs kappa > 0");
    ph.a = 0.5 * ph.kappa * ph.eta;
    ph.ea2 = std::exp(ph.a * ph.a);
    ph.rs = o.r_short > 0.0 ? o.r_short : (o.precision == RISM_PREC_FP64 ? 6.0 : 5.0) * ph.eta;
    ph.phi_c0 = 2.0 / (ph.eta * std::sqrt(M_PI));
    ph.phi_h0 = 2.0 * (ph.phi_c0 - ph.kappa * ph.ea2 * std::erfc(ph.a));
    for (int s = 0; s < kMaxSites; ++s) ph.qs[s] = s < nsite ? qs[s] : 0.0;
    const GridD g{grid->nx, grid->ny, grid->nz, grid->h, grid->origin[0], grid->origin[1], grid->origin[2]};
    const int smax = nsite <= 2 ? 2 : (nsite <= 4 ? 4 : 8);

    void* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return say(errbuf, errlen, RISM_E_CUDA, cudaGetErrorString(e));
    unsigned char* p = static_cast<unsigned char*>(base);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevTables t;
    t.n = n;
    t.smax = smax;
    t.err = reinterpret_cast<DevErr*>(p + kOffErr);
    t.geo = reinterpret_cast<Geo*>(p + kOffGeo);
    t.srcf = reinterpret_cast<SrcF*>(p + kOffGeoU);
    t.ljd = reinterpret_cast<LJd*>(p + kOffLJd);
    t.ljf = reinterpret_cast<LJf*>(p + kOffLJf);
    double* raw = reinterpret_cast<double*>(p + kOffRaw);

    // The array keeps the previous call's contents: clear the error word.
    if ((e = cudaMemsetAsync(t.err, 0, sizeof(DevErr), st)) != cudaSuccess)
        return say(errbuf, errlen, RISM_E_CUDA, cudaGetErrorString(e));
    if (n > 0) {
        // gather the solute into the [n][6] layout of the setup kernel (strided copies, no allocation;
        // the arrays may be device or host memory)
        const size_t row = 6 * sizeof(double);
        if ((e = cudaMemcpy2DAsync(raw, row, xyz, 3 * sizeof(double), 3 * sizeof(double), n, cudaMemcpyDefault,
                                   st)) != cudaSuccess ||
            (e = cudaMemcpy2DAsync(raw + 3, row, q, sizeof(double), sizeof(double), n, cudaMemcpyDefault, st)) !=
                cudaSuccess ||
            (e = cudaMemcpy2DAsync(raw + 4, row, sigma, sizeof(double), sizeof(double), n, cudaMemcpyDefault, st)) !=
                cudaSuccess ||
            (e = cudaMemcpy2DAsync(raw + 5, row, eps, sizeof(double), sizeof(double), n, cudaMemcpyDefault, st)) !=
                cudaSuccess)
            return say(errbuf, errlen, RISM_E_CUDA, cudaGetErrorString(e));
        if ((e = launch_setup(raw, n, nsite, smax, sigs, epss, o.lj_mode, o.lj_rcut, o.lj_tol, g, t, st)) !=
            cudaSuccess)
            return say(errbuf, errlen, RISM_E_CUDA, cudaGetErrorString(e));
    }
    Outputs out{u, c_lr, h_lr};
    if (u || c_lr || h_lr) {
        if ((e = launch_direct(g, ph, t, o.precision, out, o.wait_limit, 0, o.debug_flags, st)) != cudaSuccess)
            return say(errbuf, errlen, RISM_E_CUDA, cudaGetErrorString(e));
    }
    DevErr he{0, 0};
    if ((e = cudaMemcpyAsync(&he, t.err, sizeof(DevErr), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return say(errbuf, errlen, RISM_E_CUDA, cudaGetErrorString(e));
    if (he.code == DEV_TIMEOUT) return say(errbuf, errlen, RISM_E_TIMEOUT, "a bounded device wait ran out");
    if (he.code != DEV_OK) return say(errbuf, errlen, RISM_E_CUDA, "device error");
    return say(errbuf, errlen, RISM_OK, "");
}
