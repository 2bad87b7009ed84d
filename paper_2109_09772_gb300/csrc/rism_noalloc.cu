// rism_noalloc.cu -- rism_init_noalloc: the direct-sum initialization without
// any device allocation.
//
// Some callers cannot call cudaMalloc: plug-ins whose host application owns
// the device memory pool and forbids other allocators, and embedded or
// real-time callers that must not allocate after start-up (an allocation can
// block, fail late or fragment a pool sized up front).  For them this entry
// point keeps its scratch -- the per-atom and per-(atom, site) tables that the
// context-based API allocates with cudaMalloc -- in one file-scope __device__
// array of fixed size.  Every GPU that loads the library holds that array
// until the process exits.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "rism_kernels.h"
#include "rism_validate.h"

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

// The solute gathered into scratch ([n][6]: x, y, z, q, sigma, eps) must be finite with sigma, eps >= 0, the
// checks rism_set_solute makes on the host; used when the caller's arrays are device memory.  A bad row sets
// the error word (the kernels that follow read no index from these values, so they run to completion).
__global__ void k_check_solute(const double* raw, int64_t n, DevErr* err) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* r = raw + 6 * i;
    bool ok = true;
    for (int k = 0; k < 6; ++k) ok = ok && isfinite(r[k]);
    ok = ok && r[4] >= 0.0 && r[5] >= 0.0;
    if (!ok) report_error(err, DEV_BAD_INPUT, WHERE_INPUT_CHECK);
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
    // ---- everything below is checked before the GPU is touched
    if (!grid || !opts) return say(errbuf, errlen, RISM_E_INVALID, "grid and opts are required");
    if (n < 0 || n > kNoAllocMaxAtoms)
        return say(errbuf, errlen, RISM_E_INVALID,
                   "rism_init_noalloc: atom count outside [0, RISM_NOALLOC_MAX_ATOMS]; use the context API");
    if (n > 0 && (!xyz || !q || !sigma || !eps)) return say(errbuf, errlen, RISM_E_INVALID, "NULL solute array");
    if (const char* m = check_grid_desc(*grid)) return say(errbuf, errlen, RISM_E_INVALID, m);
    const rism_options& o = *opts;
    if (o.method != RISM_METHOD_DIRECT) return say(errbuf, errlen, RISM_E_UNSUPPORTED, "direct method only");
    bool unsupported = false;
    if (const char* m = check_options(o, &unsupported))
        return say(errbuf, errlen, unsupported ? RISM_E_UNSUPPORTED : RISM_E_INVALID, m);
    if (const char* m = check_solvent(nsite, qs, sigs, epss, rho)) return say(errbuf, errlen, RISM_E_INVALID, m);
    // outputs are written by the kernels: they must be device (or managed) memory
    const double* outs[3] = {u, c_lr, h_lr};
    for (const double* p : outs)
        if (p && !is_device_ptr(p))
            return say(errbuf, errlen, RISM_E_INVALID, "rism_init_noalloc: outputs must be device memory");
    // solute arrays in host memory get the host checks of rism_set_solute; device arrays are checked on the GPU
    const double* sol[4] = {xyz, q, sigma, eps};
    const int64_t len[4] = {3 * n, n, n, n};
    bool device_solute = false;
    for (int k = 0; k < 4 && n > 0; ++k) {
        if (is_device_ptr(sol[k])) {
            device_solute = true;
            continue;
        }
        if (!finite_all(sol[k], len[k])) return say(errbuf, errlen, RISM_E_INVALID, "NaN or Inf in solute");
        if (k >= 2)
            for (int64_t i = 0; i < n; ++i)
                if (sol[k][i] < 0.0) return say(errbuf, errlen, RISM_E_INVALID, "negative sigma or eps");
    }

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

    // ---- the GPU part
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
        if (device_solute) {
            k_check_solute<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(raw, n, t.err);
            if ((e = cudaGetLastError()) != cudaSuccess) return say(errbuf, errlen, RISM_E_CUDA, cudaGetErrorString(e));
        }
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
    if (he.code == DEV_BAD_INPUT)
        return say(errbuf, errlen, RISM_E_INVALID, "NaN, Inf or negative sigma/eps in the device solute arrays");
    if (he.code == DEV_TIMEOUT) return say(errbuf, errlen, RISM_E_TIMEOUT, "a bounded device wait ran out");
    if (he.code != DEV_OK) return say(errbuf, errlen, RISM_E_CUDA, "device error");
    return say(errbuf, errlen, RISM_OK, "");
}
