// Dispatch of the Laplacian-eigenmap start on its block size K (a compile-time
// width; kernels in le_kernels.cuh, instantiated in generated translation
// units).
#include "common.cuh"
#include "dispatch.cuh"

namespace pfe {
namespace lek {
template <int K>
pfe_status le_T(pfe_ctx *c, int d, double *yout, int max_iter, double tol, int degree, int *iters_out,
                double *res_out);
}  // namespace lek

// Block of K >= d + 2 + d/4 vectors (guard vectors speed up convergence of the
// d wanted ones), the smallest width built into the library.
int le_block(int d) {
    static const int widths[] = {3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16, 20, 24, 25, 32};
    const int want = d + 2 + d / 4;
    for (int k : widths)
        if (k >= want) return k;
    return d + 2 <= 32 ? 32 : 0;
}

pfe_status launch_le(pfe_ctx *c, int d, double *yout, int max_iter, double tol, int degree, int *iters,
                     double *res) {
    const int K = le_block(d);
    if (K == 0) return PFE_EUNSUPPORTED;
    PFE_DISPATCH_D(K, return lek::le_T<D>(c, d, yout, max_iter, tol, degree, iters, res));
}

}  // namespace pfe
