// Dispatch of the P-step launcher on (precision, d); kernels in
// pstep_kernels.cuh, instantiated in translation units generated by build.py.
#include "common.cuh"
#include "dispatch.cuh"

namespace pfe {
namespace pstepk {
template <typename T, int D>
pfe_status pstep_T(pfe_ctx *c, cudaStream_t s, int mode);
}  // namespace pstepk
using namespace pstepk;

pfe_status launch_pstep(pfe_ctx *c, cudaStream_t s, int mode) {
    if (c->mixed) {
        PFE_DISPATCH_D(c->d, return pstep_T<float, D>(c, s, mode));
    } else {
        PFE_DISPATCH_D(c->d, return pstep_T<double, D>(c, s, mode));
    }
}

}  // namespace pfe
