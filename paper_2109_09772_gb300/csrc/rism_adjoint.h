// rism_adjoint.h -- reverse-mode kernels (internal launch interface).
#pragma once

#include <string>

#include "rism_kernels.h"

namespace rism {

struct AdjointState;
AdjointState* adjoint_create();
void adjoint_destroy(AdjointState* a);
struct TreeState;
// tree: the context's treecode state (nullable); with target boxes on, the far part runs over the grid boxes.
rism_status adjoint_run(AdjointState* a, TreeState* tree, const DevTables& t, const GridD& g, const Phys& ph,
                        const rism_options& o, const double* raw_dev, const double* sig_s, const double* eps_s,
                        const double* g_u, const double* g_c, const double* g_h, double* d_xyz, double* d_q,
                        double* d_sigma, double* d_eps, cudaStream_t st, std::string& err);

}  // namespace rism
