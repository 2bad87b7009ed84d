// rism_lra.h -- the all-space long-range integral of the excess chemical potential (internal launch
// interface; the public entry point is rism_lra_integral in rism3d.h).
#pragma once

#include "rism_kernels.h"

namespace rism {

// Source chunks of the pair kernel for n atoms on a device with `sms` SMs, and the FP64 scratch it needs.
int lra_chunks(int64_t n, int sms);
size_t lra_scratch_doubles(int64_t n, int sms);

// Per-atom overlap sums atom[i] = (P_hc, P_hh) (original atom order) and tot = (S_hh, S_hc, Q) for the solute
// in t; perm[k]: original index of the atom at position k of the pair sum's order (device [n]); ssrc: device
// scratch [n] for the source table in that order; part: lra_scratch_doubles(n, sms) doubles.  kappa must be > 0.
cudaError_t launch_lra(const DevTables& t, const GridD& g, const Phys& ph, int sms, const int* perm, SrcF* ssrc,
                       double* part, double2* atom, double* tot, long long wait_limit, cudaStream_t st);

}  // namespace rism
