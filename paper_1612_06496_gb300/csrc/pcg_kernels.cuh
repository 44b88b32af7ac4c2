// Kernels of the d-column Jacobi-preconditioned conjugate gradients on A Y = RHS, the
// normal equations of Eq. 13 (Sec. III, last paragraph: PCG instead of a
// direct solve).  Each column c runs the textbook recurrences (Barrett et
// al., Templates, PCG) with its own alpha_c, beta_c; a column whose relative
// residual |r_c| / |b_c| reaches tol is frozen (alpha_c = 0).
//
// One iteration is four launches, all persistent-grid row kernels over the
// SELL-32 layout (one thread per row, the d columns of a row interleaved so
// every nonzero is loaded once for all d columns):
//   k_spmm     q = A p                 + block partials of p.q  -> alpha
//   k_update   y += alpha p, r -= alpha q, z = D_A^{-1} r
//                                       + partials of r.z, r.r  -> beta, convergence
//   k_refresh  (every `refresh` iterations) r = b - A y in extended precision
//   k_pupdate  p = z + beta p
// Scalars live in a device control block; the last block of each reduction
// (detected with an atomic ticket, no waiting) finishes the scalar work, so
// the loop needs no host round trip and can run inside a CUDA graph whose
// WHILE node reads the flag set here.
#pragma once
#include <cstring>
#include <type_traits>

#include "common.cuh"

namespace pfe {
namespace pcgk {

template <typename T>
struct SysView {
    int64_t n, n_slices;
    const int *__restrict__ slice_ptr;
    const int *__restrict__ col;
    const T *__restrict__ aoff;
    const T *__restrict__ adiag;
    const T *__restrict__ dinv;
};

template <typename T>
struct PcgArgs {
    SysView<T> A;
    T *x;        // solution (hi part when T = float)
    float *xlo;  // low part (float path only)
    T *r, *p, *q;
    const T *b;
    void *part;  // block partials, Acc<T>::type
    PcgCtl *ctl;
    cudaGraphConditionalHandle cond;
    int use_cond;
};

template <typename T>
SysView<T> sys_view(pfe_ctx *c) {
    SysView<T> v;
    v.n = c->g.n;
    v.n_slices = c->g.n_slices;
    v.slice_ptr = c->g.slice_ptr;
    v.col = c->g.col;
    if constexpr (std::is_same_v<T, float>) {
        v.aoff = c->g.aoff32;
        v.adiag = c->g.adiag32;
        v.dinv = c->g.dinv32;
    } else {
        v.aoff = c->g.aoff64;
        v.adiag = c->g.adiag64;
        v.dinv = c->g.dinv64;
    }
    return v;
}

// ---- device pieces -------------------------------------------------------

template <typename A, typename AT>
__device__ __forceinline__ AT ld_part(const AT *p) {
    if constexpr (std::is_same_v<AT, double>) {
        return __ldcg(p);
    } else {
        float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
        return AT{v.x, v.y};
    }
}

// Sum the NV values over the block; result in sh[0..NV) (valid after return).
template <typename T, int NV>
__device__ __forceinline__ void block_sum(typename Acc<T>::type (&v)[NV], typename Acc<T>::type *sh) {
    using A = Acc<T>;
    using AT = typename A::type;
    __shared__ AT red[kWarps][NV];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
#pragma unroll
        for (int c = 0; c < NV; ++c) A::add(v[c], A::shfl_xor(v[c], m));
    }
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < NV; ++c) red[warp][c] = v[c];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < NV; c += blockDim.x) {
        AT s = red[0][c];
        for (int w = 1; w < kWarps; ++w) A::add(s, red[w][c]);
        sh[c] = s;
    }
    __syncthreads();
}

// Write this block's NV partials; if this is the last block, reduce all
// blocks' partials (fixed order) into out[0..NV) (shared, double) and return true.
template <typename T, int NV>
__device__ __forceinline__ bool grid_sum(typename Acc<T>::type (&v)[NV], void *part_v, unsigned *ticket,
                                         double *out) {
    using A = Acc<T>;
    using AT = typename A::type;
    __shared__ AT sh[NV];
    AT *part = reinterpret_cast<AT *>(part_v);
    block_sum<T, NV>(v, sh);
    for (int c = threadIdx.x; c < NV; c += blockDim.x) part[(int64_t)blockIdx.x * NV + c] = sh[c];
    if (!last_block_arrives(ticket)) return false;
    AT acc[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) acc[c] = A::zero();
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int c = 0; c < NV; ++c) A::add(acc[c], ld_part<A, AT>(part + (int64_t)b * NV + c));
    }
    __syncthreads();  // `sh` is reused below
    block_sum<T, NV>(acc, sh);
    for (int c = threadIdx.x; c < NV; c += blockDim.x) out[c] = A::to_double(sh[c]);
    if (threadIdx.x == 0) *ticket = 0u;
    __syncthreads();
    return true;
}

__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle h, int use, int value) {
    if (use) cudaGraphSetConditional(h, value ? 1u : 0u);
}

// Finish an iteration (or the start of a solve): residual norms -> relres,
// beta, freezing, termination.  Runs on thread 0 of the last block.
static __device__ void finish_scalars(PcgCtl *ctl, const double *rz, const double *rr, int D, bool start,
                               cudaGraphConditionalHandle cond, int use_cond) {
    int any = 0;
    for (int c = 0; c < D; ++c) {
        if (start) {
            ctl->rz[c] = rz[c];
            ctl->beta[c] = 0.0;
            double rel = sqrt(rr[c]) / ctl->bnorm[c];
            ctl->relres[c] = rel;
            if (!(rel == rel) || !(rz[c] == rz[c])) ctl->error = PFE_ENUMERIC;
            ctl->active[c] = rel > ctl->tol;
        } else if (ctl->active[c]) {
            double rel = sqrt(rr[c]) / ctl->bnorm[c];
            ctl->beta[c] = rz[c] / ctl->rz[c];
            ctl->rz[c] = rz[c];
            ctl->relres[c] = rel;
            if (!(rel == rel) || !(rz[c] == rz[c])) ctl->error = PFE_ENUMERIC;
            if (rel <= ctl->tol) ctl->active[c] = 0;
        }
        any |= ctl->active[c];
    }
    ctl->any_active = any;
    int done = (!any) || ctl->error || ctl->iter >= ctl->max_iter;
    if (done) {
        double mr = 0.0;
        for (int c = 0; c < D; ++c) mr = fmax(mr, ctl->relres[c]);
        ctl->tot_iters += ctl->iter;
        ctl->max_solve_iters = max(ctl->max_solve_iters, ctl->iter);
        ctl->n_solves += 1;
        ctl->n_unconv += any ? 1 : 0;
        ctl->last_iters = ctl->iter;
        ctl->last_relres = mr;
        ctl->last_converged = !any;
        ctl->max_relres = fmax(ctl->max_relres, mr);
        const int u = ctl->unroll > 0 ? ctl->unroll : 1;
        ctl->launches += 1 + 4LL * u * ((ctl->iter + u - 1) / u);
    }
    ctl->done = done;
    set_cond(cond, use_cond, !done);
}

// r_i = b_i - (A y)_i with y = hi + lo accumulated in double-FP32 (float
// path) or FP64; returns r_i in working precision.
template <typename T, int D>
__device__ __forceinline__ void true_residual_row(const PcgArgs<T> &a, int64_t s, int lane, int64_t i,
                                                  T (&ri)[D]) {
    const int64_t base = a.A.slice_ptr[s];
    const int len = (a.A.slice_ptr[s + 1] - (int)base) >> 5;
    T bi[D];
    load_row<T, D>(a.b, i, bi);
    if constexpr (std::is_same_v<T, float>) {
        DF acc[D];
        float xh[D], xl[D];
        load_row_rw<float, D>(a.x, i, xh);
        load_row_rw<float, D>(a.xlo, i, xl);
        const float ad = a.A.adiag[i];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            acc[c] = DF{0.f, 0.f};
            df_add_prod(acc[c], ad, xh[c]);
            df_add_f(acc[c], ad * xl[c]);
        }
        for (int k = 0; k < len; ++k) {
            const int64_t idx = base + (int64_t)k * 32 + lane;
            const int j = a.A.col[idx];
            const float av = a.A.aoff[idx];
            load_row_rw<float, D>(a.x, j, xh);
            load_row_rw<float, D>(a.xlo, j, xl);
#pragma unroll
            for (int c = 0; c < D; ++c) {
                df_add_prod(acc[c], av, xh[c]);
                df_add_f(acc[c], av * xl[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < D; ++c) {
            float sh, se;
            two_sum(bi[c], -acc[c].hi, sh, se);
            ri[c] = __fadd_rn(sh, __fsub_rn(se, acc[c].lo));
        }
    } else {
        double acc[D], xv[D];
        load_row_rw<double, D>(a.x, i, xv);
        const double ad = a.A.adiag[i];
#pragma unroll
        for (int c = 0; c < D; ++c) acc[c] = ad * xv[c];
        for (int k = 0; k < len; ++k) {
            const int64_t idx = base + (int64_t)k * 32 + lane;
            const int j = a.A.col[idx];
            const double av = a.A.aoff[idx];
            load_row_rw<double, D>(a.x, j, xv);
#pragma unroll
            for (int c = 0; c < D; ++c) acc[c] = fma(av, xv[c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < D; ++c) ri[c] = bi[c] - acc[c];
    }
}

// ---- kernels -------------------------------------------------------------

// Start of a solve: r = b - A y, p = z = D_A^{-1} r, norms of b, r and r.z.
template <typename T, int D>
__global__ void __launch_bounds__(kBlock) k_pcg_init(PcgArgs<T> a) {
    using A = Acc<T>;
    using AT = typename A::type;
    AT acc[3 * D];  // r.z | r.r | b.b
#pragma unroll
    for (int c = 0; c < 3 * D; ++c) acc[c] = A::zero();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t s = (int64_t)blockIdx.x * kWarps + warp; s < a.A.n_slices; s += (int64_t)gridDim.x * kWarps) {
        const int64_t i = s * 32 + lane;
        if (i >= a.A.n) continue;
        T ri[D], bi[D], zi[D];
        true_residual_row<T, D>(a, s, lane, i, ri);
        load_row<T, D>(a.b, i, bi);
        const T dv = a.A.dinv[i];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            zi[c] = dv * ri[c];
            A::add_prod(acc[c], ri[c], zi[c]);
            A::add_prod(acc[D + c], ri[c], ri[c]);
            A::add_prod(acc[2 * D + c], bi[c], bi[c]);
        }
        store_row<T, D>(a.r, i, ri);
        store_row<T, D>(a.p, i, zi);
    }
    __shared__ double tot[3 * D];
    if (grid_sum<T, 3 * D>(acc, a.part, &a.ctl->ticket[2], tot)) {
        if (threadIdx.x == 0) {
            PcgCtl *ctl = a.ctl;
            ctl->iter = 0;
            ctl->error = 0;
            ctl->refresh_now = 0;
            for (int c = 0; c < D; ++c) {
                double bn = sqrt(tot[2 * D + c]);
                ctl->bnorm[c] = bn > 0.0 ? bn : 1.0;
                ctl->alpha[c] = 0.0;
            }
            finish_scalars(ctl, tot, tot + D, D, true, a.cond, a.use_cond);
        }
    }
}

// q = A p and the column dots p.q -> alpha.
template <typename T, int D>
__global__ void __launch_bounds__(kBlock) k_spmm(PcgArgs<T> a) {
    if (*(volatile int *)&a.ctl->done) return;
    using A = Acc<T>;
    using AT = typename A::type;
    AT pq[D];
#pragma unroll
    for (int c = 0; c < D; ++c) pq[c] = A::zero();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t s = (int64_t)blockIdx.x * kWarps + warp; s < a.A.n_slices; s += (int64_t)gridDim.x * kWarps) {
        const int64_t i = s * 32 + lane;
        if (i >= a.A.n) continue;
        const int64_t base = a.A.slice_ptr[s];
        const int len = (a.A.slice_ptr[s + 1] - (int)base) >> 5;
        T pi[D], acc[D], pj[D];
        load_row<T, D>(a.p, i, pi);
        const T ad = a.A.adiag[i];
#pragma unroll
        for (int c = 0; c < D; ++c) acc[c] = ad * pi[c];
        for (int k = 0; k < len; ++k) {
            const int64_t idx = base + (int64_t)k * 32 + lane;
            const int j = a.A.col[idx];
            const T av = a.A.aoff[idx];
            load_row<T, D>(a.p, j, pj);
#pragma unroll
            for (int c = 0; c < D; ++c) acc[c] = fma(av, pj[c], acc[c]);
        }
        store_row<T, D>(a.q, i, acc);
#pragma unroll
        for (int c = 0; c < D; ++c) A::add_prod(pq[c], pi[c], acc[c]);
    }
    __shared__ double tot[D];
    if (grid_sum<T, D>(pq, a.part, &a.ctl->ticket[0], tot)) {
        if (threadIdx.x == 0) {
            PcgCtl *ctl = a.ctl;
            for (int c = 0; c < D; ++c) {
                if (!ctl->active[c]) {
                    ctl->alpha[c] = 0.0;
                    continue;
                }
                double pqc = tot[c];
                if (!(pqc > 0.0) || !(pqc < INFINITY)) {
                    ctl->error = PFE_ENUMERIC;
                    ctl->alpha[c] = 0.0;
                } else {
                    ctl->alpha[c] = ctl->rz[c] / pqc;
                }
            }
        }
    }
}

// y += alpha p, r -= alpha q, and the dots r.z, r.r of the new residual.
template <typename T, int D>
__global__ void __launch_bounds__(kBlock) k_update(PcgArgs<T> a) {
    if (*(volatile int *)&a.ctl->done) return;
    using A = Acc<T>;
    using AT = typename A::type;
    __shared__ T alpha[D];
    if (threadIdx.x < D) alpha[threadIdx.x] = (T)a.ctl->alpha[threadIdx.x];
    __syncthreads();
    AT acc[2 * D];
#pragma unroll
    for (int c = 0; c < 2 * D; ++c) acc[c] = A::zero();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t s = (int64_t)blockIdx.x * kWarps + warp; s < a.A.n_slices; s += (int64_t)gridDim.x * kWarps) {
        const int64_t i = s * 32 + lane;
        if (i >= a.A.n) continue;
        T xi[D], pi[D], ri[D], qi[D];
        load_row_rw<T, D>(a.x, i, xi);
        load_row_rw<T, D>(a.p, i, pi);
        load_row_rw<T, D>(a.r, i, ri);
        load_row_rw<T, D>(a.q, i, qi);
        const T dv = a.A.dinv[i];
        if constexpr (std::is_same_v<T, float>) {
            float xl[D];
            load_row_rw<float, D>(a.xlo, i, xl);
#pragma unroll
            for (int c = 0; c < D; ++c) {
                // (hi, lo) += alpha * p with the product and sum errors kept in lo
                float dlt = __fmul_rn(alpha[c], pi[c]);
                float de = __fmaf_rn(alpha[c], pi[c], -dlt);
                float sh, se;
                two_sum(xi[c], dlt, sh, se);
                float lo = __fadd_rn(xl[c], __fadd_rn(se, de));
                float h2 = __fadd_rn(sh, lo);  // renormalise
                xl[c] = __fsub_rn(lo, __fsub_rn(h2, sh));
                xi[c] = h2;
                ri[c] = fmaf(-alpha[c], qi[c], ri[c]);
            }
            store_row<float, D>(a.xlo, i, xl);
        } else {
#pragma unroll
            for (int c = 0; c < D; ++c) {
                xi[c] = fma(alpha[c], pi[c], xi[c]);
                ri[c] = fma(-alpha[c], qi[c], ri[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < D; ++c) {
            T z = dv * ri[c];
            A::add_prod(acc[c], ri[c], z);
            A::add_prod(acc[D + c], ri[c], ri[c]);
        }
        store_row<T, D>(a.x, i, xi);
        store_row<T, D>(a.r, i, ri);
    }
    __shared__ double tot[2 * D];
    if (grid_sum<T, 2 * D>(acc, a.part, &a.ctl->ticket[1], tot)) {
        if (threadIdx.x == 0) {
            PcgCtl *ctl = a.ctl;
            ctl->iter += 1;
            if (!ctl->error && ctl->refresh > 0 && (ctl->iter % ctl->refresh) == 0) {
                ctl->refresh_now = 1;  // k_refresh finishes this iteration
            } else {
                finish_scalars(ctl, tot, tot + D, D, false, a.cond, a.use_cond);
            }
        }
    }
}

// Residual replacement: r = b - A y (extended precision), then finish the
// iteration with the true residual.
template <typename T, int D>
__global__ void __launch_bounds__(kBlock) k_refresh(PcgArgs<T> a) {
    if (!*(volatile int *)&a.ctl->refresh_now) return;
    using A = Acc<T>;
    using AT = typename A::type;
    AT acc[2 * D];
#pragma unroll
    for (int c = 0; c < 2 * D; ++c) acc[c] = A::zero();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t s = (int64_t)blockIdx.x * kWarps + warp; s < a.A.n_slices; s += (int64_t)gridDim.x * kWarps) {
        const int64_t i = s * 32 + lane;
        if (i >= a.A.n) continue;
        T ri[D];
        true_residual_row<T, D>(a, s, lane, i, ri);
        const T dv = a.A.dinv[i];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            T z = dv * ri[c];
            A::add_prod(acc[c], ri[c], z);
            A::add_prod(acc[D + c], ri[c], ri[c]);
        }
        store_row<T, D>(a.r, i, ri);
    }
    __shared__ double tot[2 * D];
    if (grid_sum<T, 2 * D>(acc, a.part, &a.ctl->ticket[3], tot)) {
        if (threadIdx.x == 0) {
            a.ctl->refresh_now = 0;
            finish_scalars(a.ctl, tot, tot + D, D, false, a.cond, a.use_cond);
        }
    }
}

// p = z + beta p, z = D_A^{-1} r.
template <typename T, int D>
__global__ void __launch_bounds__(kBlock) k_pupdate(PcgArgs<T> a) {
    if (*(volatile int *)&a.ctl->done) return;
    __shared__ T beta[D];
    if (threadIdx.x < D) beta[threadIdx.x] = (T)a.ctl->beta[threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t s = (int64_t)blockIdx.x * kWarps + warp; s < a.A.n_slices; s += (int64_t)gridDim.x * kWarps) {
        const int64_t i = s * 32 + lane;
        if (i >= a.A.n) continue;
        T ri[D], pi[D];
        load_row_rw<T, D>(a.r, i, ri);
        load_row_rw<T, D>(a.p, i, pi);
        const T dv = a.A.dinv[i];
#pragma unroll
        for (int c = 0; c < D; ++c) pi[c] = fma(beta[c], pi[c], dv * ri[c]);
        store_row<T, D>(a.p, i, pi);
    }
}

// y = A x without dots (pfe_apply_A and kernel timing).
template <typename T, int D>
__global__ void __launch_bounds__(kBlock) k_apply(SysView<T> A, const T *__restrict__ x, T *__restrict__ y) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t s = (int64_t)blockIdx.x * kWarps + warp; s < A.n_slices; s += (int64_t)gridDim.x * kWarps) {
        const int64_t i = s * 32 + lane;
        if (i >= A.n) continue;
        const int64_t base = A.slice_ptr[s];
        const int len = (A.slice_ptr[s + 1] - (int)base) >> 5;
        T acc[D], xj[D];
        load_row<T, D>(x, i, xj);
        const T ad = A.adiag[i];
#pragma unroll
        for (int c = 0; c < D; ++c) acc[c] = ad * xj[c];
        for (int k = 0; k < len; ++k) {
            const int64_t idx = base + (int64_t)k * 32 + lane;
            const int j = A.col[idx];
            const T av = A.aoff[idx];
            load_row<T, D>(x, j, xj);
#pragma unroll
            for (int c = 0; c < D; ++c) acc[c] = fma(av, xj[c], acc[c]);
        }
        store_row<T, D>(y, i, acc);
    }
}

// ---- host side -----------------------------------------------------------

template <typename T>
PcgArgs<T> pcg_args(pfe_ctx *c, PcgLaunch L) {
    PcgArgs<T> a;
    a.A = sys_view<T>(c);
    a.x = (T *)c->wk.Y;
    a.xlo = c->wk.Ylo;
    a.r = (T *)c->wk.R;
    a.p = (T *)c->wk.Pd;
    a.q = (T *)c->wk.Q;
    a.b = (const T *)c->wk.RHS;
    a.part = c->wk.partials;
    a.ctl = c->ctl;
    a.cond = L.cond;
    a.use_cond = L.use_cond;
    return a;
}

template <typename T, int D>
pfe_status init_T(pfe_ctx *c, cudaStream_t s, PcgLaunch L) {
    k_pcg_init<T, D><<<c->grid_rows, kBlock, 0, s>>>(pcg_args<T>(c, L));
    PFE_CUDA_TRY(c, cudaGetLastError());
    return PFE_OK;
}

template <typename T, int D>
pfe_status body_T(pfe_ctx *c, cudaStream_t s, PcgLaunch L, int iters) {
    PcgArgs<T> a = pcg_args<T>(c, L);
    for (int u = 0; u < iters; ++u) {
        k_spmm<T, D><<<c->grid_rows, kBlock, 0, s>>>(a);
        k_update<T, D><<<c->grid_rows, kBlock, 0, s>>>(a);
        k_refresh<T, D><<<c->grid_rows, kBlock, 0, s>>>(a);
        k_pupdate<T, D><<<c->grid_rows, kBlock, 0, s>>>(a);
    }
    PFE_CUDA_TRY(c, cudaGetLastError());
    return PFE_OK;
}

template <typename T, int D>
pfe_status apply_T(pfe_ctx *c, cudaStream_t s, const void *x, void *y) {
    k_apply<T, D><<<c->grid_rows, kBlock, 0, s>>>(sys_view<T>(c), (const T *)x, (T *)y);
    PFE_CUDA_TRY(c, cudaGetLastError());
    return PFE_OK;
}

// Average duration of `reps` back-to-back launches of one PCG kernel on the
// current vectors, bracketed by CUDA events on stream s.  Uses a scratch
// control block (every column active) and scratch copies of y and r, so the
// iteration state is left as it was.  which: 0 = k_spmm, 1 = k_update,
// 2 = k_pupdate.
template <typename T, int D>
pfe_status time_T(pfe_ctx *c, cudaStream_t s, int which, int reps, float *ms) {
    PcgCtl h;
    memset(&h, 0, sizeof(h));
    h.max_iter = 1 << 30;
    h.ncols = D;
    h.tol = 0.0;
    for (int k = 0; k < D; ++k) {
        h.active[k] = 1;
        h.rz[k] = 1.0;
        h.bnorm[k] = 1.0;
        h.alpha[k] = 1e-30;
        h.beta[k] = 0.5;
    }
    const int64_t nd = c->g.n * (int64_t)D;
    PcgCtl *dctl = nullptr;
    T *xs = nullptr, *rs = nullptr;
    float *xls = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    pfe_status st = PFE_OK;
    auto cleanup = [&]() {
        if (dctl) cudaFree(dctl);
        if (xs) cudaFree(xs);
        if (rs) cudaFree(rs);
        if (xls) cudaFree(xls);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (cudaMalloc((void **)&dctl, sizeof(PcgCtl)) != cudaSuccess || cudaMalloc((void **)&xs, nd * sizeof(T)) != cudaSuccess ||
        cudaMalloc((void **)&rs, nd * sizeof(T)) != cudaSuccess ||
        (std::is_same_v<T, float> && cudaMalloc((void **)&xls, nd * sizeof(float)) != cudaSuccess)) {
        cudaGetLastError();
        cleanup();
        c->err = "pfe_time_kernel: scratch allocation failed";
        return PFE_ENOMEM;
    }
    PcgArgs<T> a = pcg_args<T>(c, PcgLaunch{0, 0});
    a.ctl = dctl;
    a.x = xs;
    a.r = rs;
    a.xlo = xls;
    cudaMemcpyAsync(dctl, &h, sizeof(h), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(xs, c->wk.Y, nd * sizeof(T), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(rs, c->wk.R, nd * sizeof(T), cudaMemcpyDeviceToDevice, s);
    if (xls) cudaMemcpyAsync(xls, c->wk.Ylo, nd * sizeof(float), cudaMemcpyDeviceToDevice, s);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto launch = [&]() {
        if (which == 0)
            k_spmm<T, D><<<c->grid_rows, kBlock, 0, s>>>(a);
        else if (which == 1)
            k_update<T, D><<<c->grid_rows, kBlock, 0, s>>>(a);
        else
            k_pupdate<T, D><<<c->grid_rows, kBlock, 0, s>>>(a);
    };
    launch();  // warm-up
    cudaEventRecord(e0, s);
    for (int k = 0; k < reps; ++k) launch();
    cudaEventRecord(e1, s);
    cudaError_t err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err != cudaSuccess) {
        c->err = std::string("pfe_time_kernel: ") + cudaGetErrorString(err);
        st = PFE_ECUDA;
    } else {
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        *ms = t / (float)reps;
    }
    cleanup();
    return st;
}

}  // namespace pcgk
}  // namespace pfe

#define PFE_INSTANTIATE(T, D)                                                                 \
    template pfe_status pfe::pcgk::init_T<T, D>(pfe_ctx *, cudaStream_t, pfe::PcgLaunch);          \
    template pfe_status pfe::pcgk::body_T<T, D>(pfe_ctx *, cudaStream_t, pfe::PcgLaunch, int);     \
    template pfe_status pfe::pcgk::apply_T<T, D>(pfe_ctx *, cudaStream_t, const void *, void *);     \
    template pfe_status pfe::pcgk::time_T<T, D>(pfe_ctx *, cudaStream_t, int, int, float *);
