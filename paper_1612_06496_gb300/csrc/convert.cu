// Copies between the caller's FP64 arrays and the working-precision state
// (state get/set, starting embedding, outputs).  Not on the iteration path.
#include "common.cuh"

namespace pfe {
namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

__global__ void k_to_f32(int64_t cnt, const double *src, float *hi, float *lo) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cnt) return;
    double v = src[k];
    float h = (float)v;
    hi[k] = h;
    if (lo) lo[k] = (float)(v - (double)h);
}

__global__ void k_to_f64(int64_t cnt, const double *src, double *dst) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < cnt) dst[k] = src[k];
}

__global__ void k_from_f32(int64_t cnt, const float *hi, const float *lo, double *dst) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cnt) return;
    dst[k] = (double)hi[k] + (lo ? (double)lo[k] : 0.0);
}

template <typename T>
__global__ void k_bs_gather(int64_t ne, int d, const int *ext_slot, const T *bs, double *dst) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ne * d) return;
    int64_t e = k / d;
    int c = (int)(k % d);
    dst[k] = (double)bs[(int64_t)ext_slot[e] * d + c];
}

template <typename T>
__global__ void k_bs_scatter(int64_t ne, int d, const int *ext_slot, const double *src, T *bs) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ne * d) return;
    int64_t e = k / d;
    int c = (int)(k % d);
    bs[(int64_t)ext_slot[e] * d + c] = (T)src[k];
}

__global__ void k_yhat(int64_t n, int d, const double *P, const double *sqrtdeg, double *dst) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n * d) return;
    dst[k] = P[k] / sqrtdeg[k / d];
}

template <typename T>
__global__ void k_cw(int64_t n, int d, double r, const double *P, const double *B, const double *sqrtdeg, T *cw) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n * d) return;
    cw[k] = (T)(r * sqrtdeg[k / d] * (P[k] - B[k]));
}

}  // namespace

pfe_status launch_cw(pfe_ctx *c, cudaStream_t s) {
    const int64_t cnt = c->g.n * c->d;
    if (c->mixed)
        k_cw<float><<<nblk(cnt, 256), 256, 0, s>>>(c->g.n, c->d, c->r, c->wk.P, c->wk.B, c->g.sqrtdeg,
                                                    (float *)c->wk.Cw);
    else
        k_cw<double><<<nblk(cnt, 256), 256, 0, s>>>(c->g.n, c->d, c->r, c->wk.P, c->wk.B, c->g.sqrtdeg,
                                                     (double *)c->wk.Cw);
    PFE_CUDA_TRY(c, cudaGetLastError());
    return PFE_OK;
}

pfe_status launch_to_work(pfe_ctx *c, cudaStream_t s, const double *src, void *dst, float *dst_lo,
                          int64_t rows) {
    const int64_t cnt = rows * c->d;
    if (cnt == 0) return PFE_OK;
    if (c->mixed)
        k_to_f32<<<nblk(cnt, 256), 256, 0, s>>>(cnt, src, (float *)dst, dst_lo);
    else
        k_to_f64<<<nblk(cnt, 256), 256, 0, s>>>(cnt, src, (double *)dst);
    PFE_CUDA_TRY(c, cudaGetLastError());
    return PFE_OK;
}

pfe_status launch_from_work(pfe_ctx *c, cudaStream_t s, const void *src, const float *src_lo, double *dst,
                            int64_t rows) {
    const int64_t cnt = rows * c->d;
    if (cnt == 0) return PFE_OK;
    if (c->mixed)
        k_from_f32<<<nblk(cnt, 256), 256, 0, s>>>(cnt, (const float *)src, src_lo, dst);
    else
        k_to_f64<<<nblk(cnt, 256), 256, 0, s>>>(cnt, (const double *)src, dst);
    PFE_CUDA_TRY(c, cudaGetLastError());
    return PFE_OK;
}

pfe_status launch_bs_gather(pfe_ctx *c, cudaStream_t s, const void *bs, double *dst, bool) {
    const int64_t cnt = c->g.n_edges * c->d;
    if (cnt == 0) return PFE_OK;
    if (c->mixed)
        k_bs_gather<float><<<nblk(cnt, 256), 256, 0, s>>>(c->g.n_edges, c->d, c->g.ext_slot, (const float *)bs, dst);
    else
        k_bs_gather<double><<<nblk(cnt, 256), 256, 0, s>>>(c->g.n_edges, c->d, c->g.ext_slot, (const double *)bs,
                                                            dst);
    PFE_CUDA_TRY(c, cudaGetLastError());
    return PFE_OK;
}

pfe_status launch_bs_scatter(pfe_ctx *c, cudaStream_t s, const double *src, void *bs) {
    const int64_t cnt = c->g.n_edges * c->d;
    if (cnt == 0) return PFE_OK;
    if (c->mixed)
        k_bs_scatter<float><<<nblk(cnt, 256), 256, 0, s>>>(c->g.n_edges, c->d, c->g.ext_slot, src, (float *)bs);
    else
        k_bs_scatter<double><<<nblk(cnt, 256), 256, 0, s>>>(c->g.n_edges, c->d, c->g.ext_slot, src, (double *)bs);
    PFE_CUDA_TRY(c, cudaGetLastError());
    return PFE_OK;
}

pfe_status launch_yhat(pfe_ctx *c, cudaStream_t s, double *dst) {
    const int64_t cnt = c->g.n * c->d;
    k_yhat<<<nblk(cnt, 256), 256, 0, s>>>(c->g.n, c->d, c->wk.P, c->g.sqrtdeg, dst);
    PFE_CUDA_TRY(c, cudaGetLastError());
    return PFE_OK;
}

bool d_supported(int d) {
    return (d >= 1 && d <= 16) || d == 20 || d == 24 || d == 25 || d == 32;
}

}  // namespace pfe
