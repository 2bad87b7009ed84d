// rism_validate.h -- host-side argument checks shared by the context API
// (rism_grid_create, rism_set_solute, rism_set_solvent) and the allocation-free
// entry point (rism_init_noalloc), so both accept and refuse the same inputs.
//
// Every check returns nullptr when the argument is acceptable, else a static
// message; nothing here touches the GPU or allocates.
#pragma once

#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "rism3d.h"
#include "rism_tree.h"

namespace rism {

// Largest extent of one grid axis: the launch grids put y and z blocks of a few points on gridDim.y/z (<= 65535).
constexpr int32_t kMaxGridAxis = 65535;
constexpr int64_t kMaxGridPoints = 1LL << 36;

inline bool finite_all(const double* a, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(a[i])) return false;
    return true;
}

inline const char* check_grid_desc(const rism_grid_desc& g) {
    if (g.nx < 1 || g.ny < 1 || g.nz < 1) return "grid dimensions must be >= 1";
    if (g.nx > kMaxGridAxis || g.ny > kMaxGridAxis || g.nz > kMaxGridAxis)
        return "grid dimensions must be <= 65535 per axis";
    if ((int64_t)g.nx * g.ny * g.nz > kMaxGridPoints) return "grid has more than 2^36 points";
    if (!(g.h > 0.0 && std::isfinite(g.h))) return "grid spacing must be finite and > 0";
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(g.origin[k])) return "grid origin must be finite";
    return nullptr;
}

// Options of every method; the status for a refusal is RISM_E_INVALID unless *unsupported is set.
inline const char* check_options(const rism_options& o, bool* unsupported) {
    *unsupported = false;
    if (o.method != RISM_METHOD_DIRECT && o.method != RISM_METHOD_TREECODE) return "method";
    if (o.precision != RISM_PREC_FP64 && o.precision != RISM_PREC_FP32) return "precision";
    if (o.method == RISM_METHOD_TREECODE && o.precision == RISM_PREC_FP64) {
        *unsupported = true;
        return "the treecode computes FP32 pair terms; FP64 needs the direct method";
    }
    if (o.degree < 1 || o.degree > kMaxDegree) return "degree out of range";
    if (!(o.theta > 0.0 && o.theta < 1.0)) return "theta must lie in (0, 1)";
    if (o.leaf < 1) return "leaf must be >= 1";
    for (int k = 0; k < 3; ++k)
        if (o.batch[k] < 0 || o.batch[k] > 64) return "batch dims must lie in [0, 64]";
    if (o.lj_mode < RISM_LJ_NONE || o.lj_mode > RISM_LJ_TOL) return "lj_mode";
    if (o.lj_mode == RISM_LJ_RCUT && !(o.lj_rcut > 0.0 && std::isfinite(o.lj_rcut))) return "lj_rcut must be > 0";
    if (o.lj_mode == RISM_LJ_TOL && !(o.lj_tol > 0.0 && std::isfinite(o.lj_tol))) return "lj_tol must be > 0";
    const double pos[] = {o.eta, o.T, o.eps_r, o.k_e, o.k_B};
    for (double v : pos)
        if (!(v > 0.0 && std::isfinite(v))) return "eta, T, eps_r, k_e, k_B must be finite and > 0";
    if (!std::isfinite(o.kappa)) return "kappa must be finite";
    if (!(o.r_short >= 0.0 && std::isfinite(o.r_short))) return "r_short must be finite and >= 0";
    if (o.wait_limit < 1) return "wait_limit must be >= 1";
    if (o.approx != RISM_APPROX_BARYCENTRIC && o.approx != RISM_APPROX_TAYLOR) return "approx";
    if (o.approx == RISM_APPROX_TAYLOR && (o.method != RISM_METHOD_TREECODE || o.target_proxies == 0)) {
        *unsupported = true;
        return "Taylor moments are a far-field form of the treecode's target boxes (method TREECODE, target_proxies 1)";
    }
    return nullptr;
}

// Solute arrays in host memory: xyz [n][3], q, sigma, eps [n].
inline const char* check_host_solute(int64_t n, const double* xyz, const double* q, const double* sigma,
                                     const double* eps) {
    if (n < 0) return "n < 0";
    if (n > 0 && (!xyz || !q || !sigma || !eps)) return "NULL solute array";
    if (n > (1LL << 31)) return "too many atoms";
    if (n == 0) return nullptr;
    // one pass over the atoms (this runs on every solute update, before the GPU gets the step)
    bool finite = true, nonneg = true;
    for (int64_t i = 0; i < n; ++i) {
        finite &= std::isfinite(xyz[3 * i]) & std::isfinite(xyz[3 * i + 1]) & std::isfinite(xyz[3 * i + 2]) &
                  std::isfinite(q[i]) & std::isfinite(sigma[i]) & std::isfinite(eps[i]);
        nonneg &= (sigma[i] >= 0.0) & (eps[i] >= 0.0);
    }
    if (!finite) return "NaN or Inf in solute";
    if (!nonneg) return "negative sigma or eps";
    return nullptr;
}

// Solvent sites (host memory): q, sigma, eps [nsite], rho [nsite] or NULL.
inline const char* check_solvent(int32_t nsite, const double* q, const double* sigma, const double* eps,
                                 const double* rho) {
    if (nsite < 1 || nsite > RISM_MAX_SITES) return "nsite must lie in [1, RISM_MAX_SITES]";
    if (!q || !sigma || !eps) return "NULL solvent array";
    if (!finite_all(q, nsite) || !finite_all(sigma, nsite) || !finite_all(eps, nsite) ||
        (rho && !finite_all(rho, nsite)))
        return "NaN or Inf in solvent";
    for (int s = 0; s < nsite; ++s) {
        if (sigma[s] < 0.0 || eps[s] < 0.0) return "negative sigma or eps";
        if (rho && rho[s] < 0.0) return "negative density";
    }
    return nullptr;
}

// Kind of memory behind a pointer, as the CUDA runtime sees it (no allocation, no GPU work).
enum class MemKind { kHost, kDevice };
inline MemKind mem_kind(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return MemKind::kHost;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? MemKind::kDevice : MemKind::kHost;
}
inline bool is_device_ptr(const void* p) { return mem_kind(p) == MemKind::kDevice; }

}  // namespace rism
