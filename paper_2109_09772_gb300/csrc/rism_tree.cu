// rism_tree.cu -- placeholder until the treecode lands.
#include "rism_tree.h"

namespace rism {
struct TreeState {
    int dummy;
};
TreeState* tree_create() { return new TreeState{}; }
void tree_destroy(TreeState* ts) { delete ts; }
rism_status tree_prepare(TreeState*, const DevTables&, const GridD&, const Phys&, const rism_options&, cudaStream_t,
                         std::string& err) {
    err = "treecode not built";
    return RISM_E_UNSUPPORTED;
}
rism_status tree_eval(TreeState*, const DevTables&, const GridD&, const Phys&, const rism_options&, Outputs,
                      cudaStream_t, std::string& err, rism_info&) {
    err = "treecode not built";
    return RISM_E_UNSUPPORTED;
}
rism_status batch_eval(std::vector<BatchItem>&, const rism_options&, cudaStream_t, DevErr*, std::string& msg) {
    msg = "batched launch not built";
    return RISM_E_UNSUPPORTED;
}
}  // namespace rism
