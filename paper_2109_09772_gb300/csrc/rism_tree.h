// rism_tree.h -- barycentric-Lagrange particle-cluster treecode and the
// cell-list near field (internal launch interface).
#pragma once

#include <string>
#include <vector>

#include "rism_kernels.h"

namespace rism {

constexpr int kMaxDegree = 12;

struct TreeState;

struct BatchItem {
    TreeState* tree;
    const DevTables* t;
    GridD g;
    Phys ph;
    Outputs o;
    const double* raw;  // [n][6] solute on the device (uploaded before the launch)
    double sig_s[kMaxSites], eps_s[kMaxSites];
    int lj_mode;
    double lj_rcut, lj_tol;
};

TreeState* tree_create();
void tree_destroy(TreeState* ts);
// Build the tree, proxies, modified charges and interaction lists for the
// current solute tables (called when the solute, solvent or options change).
rism_status tree_prepare(TreeState* ts, const DevTables& t, const GridD& g, const Phys& ph, const rism_options& o,
                         cudaStream_t st, std::string& err);
// Evaluate u, c, h with the treecode far field and the cell-list near field.
rism_status tree_eval(TreeState* ts, const DevTables& t, const GridD& g, const Phys& ph, const rism_options& o,
                      Outputs out, cudaStream_t st, std::string& err, rism_info& info);
// After the stream has been synchronised: copy the counters into info; on a
// far-list overflow grow the buffer and set retry (run prepare + eval again).
rism_status tree_post(TreeState* ts, rism_info& info, bool& retry, std::string& err);
// Many solutes in one persistent, graph-captured launch sequence.
// The whole sequence (per-solute setup and tree kernels, persistent far and
// near kernels) is captured in a CUDA graph and replayed while unchanged.
// After the caller synchronises, tree_post on each item reports overflows
// (retry: run again).
rism_status batch_eval(std::vector<BatchItem>& items, const rism_options& o, cudaStream_t st, DevErr* err,
                       std::string& msg, bool& retry);

}  // namespace rism
