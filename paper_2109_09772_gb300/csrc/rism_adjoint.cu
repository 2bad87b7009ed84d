// rism_adjoint.cu -- placeholder until the adjoint lands.
#include "rism_adjoint.h"

namespace rism {
struct AdjointState {
    int dummy;
};
AdjointState* adjoint_create() { return new AdjointState{}; }
void adjoint_destroy(AdjointState* a) { delete a; }
rism_status adjoint_run(AdjointState*, const DevTables&, const GridD&, const Phys&, const rism_options&,
                        const double*, const double*, const double*, const double*, double*, double*, double*,
                        double*, cudaStream_t, std::string& err) {
    err = "adjoint not built";
    return RISM_E_UNSUPPORTED;
}
}  // namespace rism
