// rism_kernels.h -- host-side launch interface between the C ABI layer and
// the CUDA kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rism_internal.cuh"

namespace rism {

// Device tables of one solute/solvent pair (owned by the context).
struct DevTables {
    int64_t n = 0;    // atoms
    int smax = 2;     // padded site count (2, 4 or 8)
    Geo* geo = nullptr;   // [n] physical positions + charge
    SrcF* srcf = nullptr; // [n] grid-unit positions (relative to the grid origin, float-float) + charge
    LJd* ljd = nullptr;   // [n][smax]
    LJf* ljf = nullptr;   // [n][smax]
    DevErr* err = nullptr;
};

struct Outputs {
    double* u = nullptr;
    double* c = nullptr;
    double* h = nullptr;
};

// a1: mixing, LJ A/B, per-pair cut-offs, grid-unit positions.
// raw = [n][6] (x, y, z, q, sigma, eps) on the device; site tables on the host (in Phys + arrays).
cudaError_t launch_setup(const double* raw, int64_t n, int S, int smax, const double* sig_s, const double* eps_s,
                         int lj_mode, double lj_rcut, double lj_tol, const GridD& g, DevTables& t,
                         cudaStream_t st);

// a4: I_s = sum_i 4 pi (A/(9 rc^9) - B/(3 rc^3)) into dev_out[S].
cudaError_t launch_lj_tail(const DevTables& t, int S, double* dev_out, cudaStream_t st);

// a2/a3/a5/a6 by direct summation over all atoms (FP64 or FP32 pairs).
cudaError_t launch_direct(const GridD& g, const Phys& ph, const DevTables& t, int precision, Outputs o,
                          long long wait_limit, int variant, int debug_flags, cudaStream_t st);

int direct_variant_count();

}  // namespace rism
