// rism_kspace.h -- reciprocal-space long-range asymptotics (internal launch interface; the public entry point
// is rism_asymptotics_k in rism3d.h).
#pragma once

#include "rism_kernels.h"

namespace rism {

struct KspaceSetup {
    int S;
    double beta, k_e, eps_r, eta, kappa;
    double qs[kMaxSites];
    double qmax;   // max_s |q_s|
    double qabs;   // sum_a |Q_a|
    double kcut;   // <= 0: no cut-off
};

// The bound of eq. (k-space-dcf-err) at wave number k (sum |Q_a| and max |q_s|), and the k where it equals tol.
double kspace_bound(double k, const KspaceSetup& s);
double kspace_kcut(const KspaceSetup& s, double tol);

// Device bytes of the per-atom phase tables for n atoms on an nx x ny x nz grid.
size_t kspace_table_bytes(int64_t n, int nx, int ny, int nz);

// c_s(k) and h_s(k) (each nullable) on the half spectrum [S][nz][ny][nx/2+1] as interleaved FP64 complex values.
cudaError_t launch_kspace(const DevTables& t, const GridD& g, const KspaceSetup& s, void* tables, double* c_k,
                          double* h_k, long long wait_limit, cudaStream_t st);

}  // namespace rism
