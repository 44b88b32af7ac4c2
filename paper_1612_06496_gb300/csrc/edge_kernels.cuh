// Fused edge pass of the split-Bregman inner iteration (Alg. 2 steps 6-7 in
// the compact form):
//   M Y                         (Eq. 7)   E_e = w_e (y_a - y_b), edge e = (a < b)
//   d = Shrink(M Y + b, 1/lam)   (Eq. 9)
//   b' = b + M Y - d             (Eq. 10)
//   RHS = lam M^T (d - b') + r D^{1/2} (P - B)    (Eq. 13, times 2; next solve)
//
// Gather form, no atomics: thread i walks its SELL-32 row; for every incident
// edge it recomputes E, d and b' from the shared old b (both endpoints get
// bit-identical values because E is always formed as w (y_a - y_b) with
// a < b), accumulates (M^T q)_i = sum_e (+-w_e) q_e, and only the first
// endpoint writes b'.  d is never stored: it is consumed where it is made.
#pragma once
#include <type_traits>

#include "common.cuh"

namespace pfe {
namespace edgek {

template <typename T>
struct EdgeArgs {
    int64_t n, n_slices;
    const int *__restrict__ slice_ptr;
    const int *__restrict__ col;
    const int *__restrict__ eid;
    const T *__restrict__ w;
    const T *__restrict__ y;
    const T *__restrict__ bs_old;
    T *__restrict__ bs_new;
    const T *__restrict__ cw;
    T *__restrict__ rhs;
    T lambda, gamma;
};

template <typename T, int D>
__global__ void __launch_bounds__(kBlock) k_edge(EdgeArgs<T> a) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t s = (int64_t)blockIdx.x * kWarps + warp; s < a.n_slices; s += (int64_t)gridDim.x * kWarps) {
        const int64_t i = s * 32 + lane;
        if (i >= a.n) continue;
        const int64_t base = a.slice_ptr[s];
        const int len = (a.slice_ptr[s + 1] - (int)base) >> 5;
        T yi[D], yj[D], bo[D], bn[D], acc[D];
        load_row<T, D>(a.y, i, yi);
#pragma unroll
        for (int c = 0; c < D; ++c) acc[c] = T(0);
        for (int k = 0; k < len; ++k) {
            const int64_t idx = base + (int64_t)k * 32 + lane;
            const int e = a.eid[idx];
            if (e < 0) continue;  // padding slot
            const int j = a.col[idx];
            const T w = a.w[idx];
            const bool first = i < j;  // i is the +w endpoint of edge e
            load_row<T, D>(a.y, j, yj);
            load_row<T, D>(a.bs_old, e, bo);
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const T diff = first ? (yi[c] - yj[c]) : (yj[c] - yi[c]);  // y_a - y_b
                const T t = w * diff + bo[c];                                // (M Y + b)_e
                const T z = shrink<T>(t, a.gamma);                           // d_e
                bn[c] = t - z;                                               // b'_e
                const T v = w * (z - bn[c]);
                acc[c] = first ? acc[c] + v : acc[c] - v;
            }
            if (first) store_row<T, D>(a.bs_new, e, bn);
        }
        T ci[D];
        load_row<T, D>(a.cw, i, ci);
#pragma unroll
        for (int c = 0; c < D; ++c) acc[c] = a.lambda * acc[c] + ci[c];
        store_row<T, D>(a.rhs, i, acc);
    }
}

template <typename T, int D>
pfe_status edge_T(pfe_ctx *c, cudaStream_t s) {
    EdgeArgs<T> a;
    a.n = c->g.n;
    a.n_slices = c->g.n_slices;
    a.slice_ptr = c->g.slice_ptr;
    a.col = c->g.col;
    a.eid = c->g.eid;
    if constexpr (std::is_same_v<T, float>)
        a.w = c->g.w32;
    else
        a.w = c->g.w64;
    a.y = (const T *)c->wk.Y;
    a.bs_old = (const T *)c->wk.Bs[c->bs_cur];
    a.bs_new = (T *)c->wk.Bs[1 - c->bs_cur];
    a.cw = (const T *)c->wk.Cw;
    a.rhs = (T *)c->wk.RHS;
    a.lambda = (T)c->lambda;
    a.gamma = (T)(1.0 / c->lambda);
    k_edge<T, D><<<c->grid_rows, kBlock, 0, s>>>(a);
    PFE_CUDA_TRY(c, cudaGetLastError());
    c->bs_cur = 1 - c->bs_cur;
    return PFE_OK;
}

}  // namespace edgek
}  // namespace pfe

#define PFE_INSTANTIATE(T, D) template pfe_status pfe::edgek::edge_T<T, D>(pfe_ctx *, cudaStream_t);
