// Dispatch of the edge-pass launcher on (precision, d); kernels in
// edge_kernels.cuh, instantiated in translation units generated by build.py.
#include "common.cuh"
#include "dispatch.cuh"

namespace pfe {
namespace edgek {
template <typename T, int D>
pfe_status edge_T(pfe_ctx *c, cudaStream_t s);
}  // namespace edgek
using namespace edgek;

pfe_status launch_edge(pfe_ctx *c, cudaStream_t s) {
    if (c->mixed) {
        PFE_DISPATCH_D(c->d, return edge_T<float, D>(c, s));
    } else {
        PFE_DISPATCH_D(c->d, return edge_T<double, D>(c, s));
    }
}

}  // namespace pfe
