// Dispatch of the PCG launchers on (precision, d).  The kernels are in
// pcg_kernels.cuh; they are instantiated in separate translation units
// (generated by build.py) so that the library compiles in parallel.
#include "common.cuh"
#include "dispatch.cuh"

namespace pfe {
namespace pcgk {
template <typename T, int D>
pfe_status init_T(pfe_ctx *c, cudaStream_t s, PcgLaunch L);
template <typename T, int D>
pfe_status body_T(pfe_ctx *c, cudaStream_t s, PcgLaunch L, int iters);
template <typename T, int D>
pfe_status final_T(pfe_ctx *c, cudaStream_t s, PcgLaunch L);
template <typename T, int D>
pfe_status apply_T(pfe_ctx *c, cudaStream_t s, const void *x, void *y);
template <typename T, int D>
pfe_status time_T(pfe_ctx *c, cudaStream_t s, int which, int reps, float *ms, int variant);
}  // namespace pcgk
using namespace pcgk;

pfe_status launch_pcg_init(pfe_ctx *c, cudaStream_t s, PcgLaunch L) {
    if (c->mixed) {
        PFE_DISPATCH_D(c->d, return init_T<float, D>(c, s, L));
    } else {
        PFE_DISPATCH_D(c->d, return init_T<double, D>(c, s, L));
    }
}

pfe_status launch_pcg_body(pfe_ctx *c, cudaStream_t s, PcgLaunch L, int iters) {
    if (c->mixed) {
        PFE_DISPATCH_D(c->d, return body_T<float, D>(c, s, L, iters));
    } else {
        PFE_DISPATCH_D(c->d, return body_T<double, D>(c, s, L, iters));
    }
}

pfe_status launch_pcg_final(pfe_ctx *c, cudaStream_t s, PcgLaunch L) {
    if (c->mixed) {
        PFE_DISPATCH_D(c->d, return final_T<float, D>(c, s, L));
    } else {
        PFE_DISPATCH_D(c->d, return final_T<double, D>(c, s, L));
    }
}

pfe_status launch_apply_A(pfe_ctx *c, cudaStream_t s, const void *x, void *y) {
    if (c->mixed) {
        PFE_DISPATCH_D(c->d, return apply_T<float, D>(c, s, x, y));
    } else {
        PFE_DISPATCH_D(c->d, return apply_T<double, D>(c, s, x, y));
    }
}

}  // namespace pfe

namespace pfe {
pfe_status time_pcg_kernel(pfe_ctx *c, cudaStream_t s, int which, int reps, float *ms, int variant) {
    if (c->mixed) {
        PFE_DISPATCH_D(c->d, return time_T<float, D>(c, s, which, reps, ms, variant));
    } else {
        PFE_DISPATCH_D(c->d, return time_T<double, D>(c, s, which, reps, ms, variant));
    }
}
}  // namespace pfe
