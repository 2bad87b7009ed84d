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
// One solute step as a replayed CUDA graph: upload of the solute from pinned host memory, setup of the
// per-pair tables, tree, lists, box-level far field, far and near kernels, LJ tail and the copies of the
// tail and the counters to pinned host memory.  The sequence is captured on a private stream the first time
// a signature (every pointer, size and constant the launches depend on) is seen and replayed afterwards.
// used = false (nothing enqueued) while the autotuner still has to time this problem class.
struct SoluteStep {
    const double* h_raw;  // pinned [n][6]
    double* d_raw;        // device [n][6]
    int64_t n;
    const double* sig_s;
    const double* eps_s;
    int lj_mode;
    double lj_rcut, lj_tol;
    double* d_tail;       // device [S] or null (no tail)
    double* h_tail;       // pinned [S]
};
rism_status tree_graph_step(TreeState* ts, const DevTables& t, const GridD& g, const Phys& ph, const rism_options& o,
                            Outputs out, const SoluteStep& step, cudaStream_t st, std::string& err, rism_info& info,
                            bool& used);
// Drop the captured solute graph (buffers moved or the retry path ran).
void tree_graph_reset(TreeState* ts);

// Split the far and near kernels of the following evaluations into nslab pairs of launches over z slabs of
// batch layers (1: one launch each), each pair followed by a record of a slab event, so that copies of a
// finished slab's outputs can overlap the rest of the evaluation.  The slab count is part of the solute graph's
// signature.  With slabs, rism_info's far time covers the far and near launches together (near time 0).
rism_status tree_set_slabs(TreeState* ts, int nslab, std::string& err);
// After tree_eval or tree_graph_step enqueued an evaluation with slabs: their number, the grid planes
// [z[k][0], z[k][1]) whose outputs slab k completes, and the event recorded after it; 0 without slabs.
int tree_slabs(const TreeState* ts, const GridD& g, int (*z)[2], cudaEvent_t* ev);
constexpr int kOutSlabsMax = 16;

// Reverse mode, far part, with the grid boxes as source clusters: w holds the per-point weights (A1 of 1/d,
// Ak of e^{-kappa d}/d in .x, .y); part receives per atom (original order) dq, Gx, Gy, Gz in grid units, as
// one chunk of the direct far kernel would.  used = false (nothing done) when target boxes are off or the tree
// is not prepared for the current solute.  Synchronises the stream (list growth).
rism_status tree_adjoint_far(TreeState* ts, const DevTables& t, const GridD& g, const Phys& ph, const rism_options& o,
                             const float4* w, bool dh, double* part, cudaStream_t st, std::string& err, bool& used);

// Original atom indices in Morton (sorted) order of the last tree build, or null before any.
const uint32_t* tree_atom_order(TreeState* ts);

// Many solutes in one persistent, graph-captured launch sequence.
// The whole sequence (per-solute setup and tree kernels, persistent far and
// near kernels) is captured in a CUDA graph and replayed while unchanged.
// After the caller synchronises, tree_post on each item reports overflows
// (retry: run again).
rism_status batch_eval(std::vector<BatchItem>& items, const rism_options& o, cudaStream_t st, DevErr* err,
                       std::string& msg, bool& retry);

}  // namespace rism
