// P-step and B-step of the SOC iteration (Alg. 1 steps 6-7), in FP64:
//   X = D^{1/2} Y + B
//   P = argmin_{P^T P = I} |P - X|_F = X (X^T X)^{-1/2}   (polar factor)
//   B = B + D^{1/2} Y - P = X - P
//   C = r D^{1/2} (P - B)   (second term of the next right-hand side, Eq. 13)
// The d x d Gram X^T X is reduced over the rows (tall-skinny, one pass, fixed
// order); its inverse square root comes from a cyclic Jacobi
// eigendecomposition on one block.  pfe_init uses the same path with
// X = D^{1/2} Y0, B = 0 to D-orthonormalise the starting embedding.
#pragma once
#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace pfe {
namespace pstepk {

constexpr int kTile = 64;  // rows staged in shared memory per Gram step

template <typename T>
struct PArgs {
    int64_t n;
    const double *__restrict__ sqrtdeg;
    const T *y;             // working Y (hi part for float)
    const float *ylo;       // low part (float) or null
    const double *y0;       // init mode: FP64 start (row-major n x D) instead of y
    double *P, *B;
    T *cw, *rhs;
    T *yw;                  // init mode: Y written back (hi)
    float *ywlo;            // init mode: low part
    double r;
    double *part;           // block partials of the Gram (D*(D+1)/2 per block)
    PstepCtl *ctl;
    int mode;
    Segs sg;                // segments: one Gram and transform each
    double *Tseg;           // nseg x D x D transforms (segment 0: ctl->T for one segment)
    unsigned *tickets;      // nseg Gram tickets
};

template <typename T, int D>
__device__ __forceinline__ void x_row(const PArgs<T> &a, int64_t i, double (&x)[D]) {
    const double sd = a.sqrtdeg[i];
    if (a.mode == PSTEP_INIT) {
#pragma unroll
        for (int c = 0; c < D; ++c) x[c] = sd * a.y0[i * D + c];
        return;
    }
    double bi[D];
    load_row_rw<double, D>(a.B, i, bi);
    if constexpr (std::is_same_v<T, float>) {
        float h[D], l[D];
        load_row_rw<float, D>(a.y, i, h);
        load_row_rw<float, D>(a.ylo, i, l);
#pragma unroll
        for (int c = 0; c < D; ++c) x[c] = fma(sd, (double)h[c] + (double)l[c], bi[c]);
    } else {
        double h[D];
        load_row_rw<double, D>(a.y, i, h);
#pragma unroll
        for (int c = 0; c < D; ++c) x[c] = fma(sd, h[c], bi[c]);
    }
}

template <typename T, int D>
__global__ void __launch_bounds__(kBlock) k_gram(PArgs<T> a) {
    constexpr int NE = D * (D + 1) / 2;
    constexpr int PER = (NE + kBlock - 1) / kBlock;
    __shared__ double tile[kTile][D];
    __shared__ unsigned char ep[NE], eq[NE];
    for (int e = threadIdx.x; e < NE; e += blockDim.x) {
        int p = 0, r = e;
        while (r >= D - p) {
            r -= D - p;
            ++p;
        }
        ep[e] = (unsigned char)p;
        eq[e] = (unsigned char)(p + r);
    }
    double g[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) g[k] = 0.0;
    __syncthreads();
    // this block's segment; its blocks stride over the segment's row tiles
    const BlockSeg bsg = block_seg(a.sg);
    const int64_t ntiles = (bsg.r1 - bsg.r0 + kTile - 1) / kTile;
    for (int64_t t = blockIdx.x - bsg.b0; t < ntiles; t += bsg.nb) {
        const int64_t r0 = bsg.r0 + t * kTile;
        for (int rr = threadIdx.x; rr < kTile; rr += blockDim.x) {
            const int64_t i = r0 + rr;
            double x[D];
            if (i < bsg.r1) {
                x_row<T, D>(a, i, x);
            } else {
#pragma unroll
                for (int c = 0; c < D; ++c) x[c] = 0.0;
            }
#pragma unroll
            for (int c = 0; c < D; ++c) tile[rr][c] = x[c];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = threadIdx.x + k * kBlock;
            if (e < NE) {
                const int p = ep[e], q = eq[e];
                double s = g[k];
                for (int rr = 0; rr < kTile; ++rr) s = fma(tile[rr][p], tile[rr][q], s);
                g[k] = s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = threadIdx.x + k * kBlock;
        if (e < NE) a.part[(int64_t)blockIdx.x * NE + e] = g[k];
    }
    unsigned *ticket = a.sg.nseg == 1 ? &a.ctl->ticket : a.tickets + bsg.seg;
    if (!last_block_arrives(ticket, (unsigned)bsg.nb)) return;
    __shared__ double G[D * D], V[D * D];
    for (int e = threadIdx.x; e < NE; e += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < bsg.nb; ++b) s += __ldcg(a.part + (int64_t)(bsg.b0 + b) * NE + e);
        const int p = ep[e], q = eq[e];
        G[p * D + q] = s;
        G[q * D + p] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // ctl->error was cleared before the launch; any segment may set it
        PstepCtl *ctl = a.ctl;
        const bool first = bsg.seg == 0;
        if (first)
            for (int k = 0; k < D * D; ++k) ctl->G[k] = G[k];
        jacobi_eig(G, V, D);
        double lmax = 0.0, lmin = INFINITY;
        for (int k = 0; k < D; ++k) {
            if (first) ctl->evals[k] = G[k * D + k];
            lmax = fmax(lmax, G[k * D + k]);
            lmin = fmin(lmin, G[k * D + k]);
        }
        if (!(lmin > 1e-13 * lmax) || !(lmax < INFINITY)) {
            atomicMax(&ctl->error, (int)PFE_ESINGULAR);
        } else {
            double *Tout = a.sg.nseg == 1 ? ctl->T : a.Tseg + (int64_t)bsg.seg * D * D;
            for (int p = 0; p < D; ++p)
                for (int q = 0; q < D; ++q) {
                    double s = 0.0;
                    for (int k = 0; k < D; ++k) s += V[p * D + k] * V[q * D + k] / sqrt(G[k * D + k]);
                    Tout[p * D + q] = s;
                }
        }
        *ticket = 0u;
    }
}

template <typename T, int D>
__global__ void __launch_bounds__(kBlock) k_papply(PArgs<T> a) {
    __shared__ double Tm[D * D];
    if (a.ctl->error) return;
    const BlockSeg bsg = block_seg(a.sg);
    const double *Tsrc = a.sg.nseg == 1 ? a.ctl->T : a.Tseg + (int64_t)bsg.seg * D * D;
    for (int k = threadIdx.x; k < D * D; k += blockDim.x) Tm[k] = Tsrc[k];
    __syncthreads();
    for (int64_t i = bsg.r0 + (int64_t)(blockIdx.x - bsg.b0) * blockDim.x + threadIdx.x; i < bsg.r1;
         i += (int64_t)bsg.nb * blockDim.x) {
        double x[D], p[D], b[D];
        x_row<T, D>(a, i, x);
#pragma unroll
        for (int q = 0; q < D; ++q) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) s = fma(x[k], Tm[k * D + q], s);
            p[q] = s;
        }
        const double sd = a.sqrtdeg[i];
        T cw[D];
        if (a.mode == PSTEP_INIT) {
#pragma unroll
            for (int q = 0; q < D; ++q) {
                b[q] = 0.0;
                cw[q] = (T)(a.r * sd * p[q]);
            }
            // Y = D^{-1/2} P
            if constexpr (std::is_same_v<T, float>) {
                float h[D], l[D];
#pragma unroll
                for (int q = 0; q < D; ++q) {
                    const double yv = p[q] / sd;
                    h[q] = (float)yv;
                    l[q] = (float)(yv - (double)h[q]);
                }
                store_row<float, D>(a.yw, i, h);
                store_row<float, D>(a.ywlo, i, l);
            } else {
                double h[D];
#pragma unroll
                for (int q = 0; q < D; ++q) h[q] = p[q] / sd;
                store_row<double, D>(a.yw, i, h);
            }
        } else {
#pragma unroll
            for (int q = 0; q < D; ++q) {
                b[q] = x[q] - p[q];
                cw[q] = (T)(a.r * sd * (p[q] - b[q]));
            }
        }
        if (a.mode == PSTEP_CARRY) {
            T old[D], rh[D];
            load_row_rw<T, D>(a.cw, i, old);
            load_row_rw<T, D>(a.rhs, i, rh);
#pragma unroll
            for (int q = 0; q < D; ++q) rh[q] = rh[q] - old[q] + cw[q];
            store_row<T, D>(a.rhs, i, rh);
        } else {
            store_row<T, D>(a.rhs, i, cw);
        }
        store_row<T, D>(a.cw, i, cw);
        store_row<double, D>(a.P, i, p);
        store_row<double, D>(a.B, i, b);
    }
}

template <typename T, int D>
pfe_status pstep_T(pfe_ctx *c, cudaStream_t s, int mode) {
    PArgs<T> a;
    a.n = c->g.n;
    a.sqrtdeg = c->g.sqrtdeg;
    a.y = (const T *)c->wk.Y;
    a.ylo = c->wk.Ylo;
    a.y0 = c->wk.stage;
    a.P = c->wk.P;
    a.B = c->wk.B;
    a.cw = (T *)c->wk.Cw;
    a.rhs = (T *)c->wk.RHS;
    a.yw = (T *)c->wk.Y;
    a.ywlo = c->wk.Ylo;
    a.r = c->r;
    a.part = c->wk.partials;
    a.ctl = c->pctl;
    a.mode = mode;
    a.sg = seg_view(c);
    a.Tseg = c->seg_T;
    a.tickets = c->seg_pticket;
    const int64_t ntiles = (a.n + kTile - 1) / kTile;
    const int gblocks = (int)std::max<int64_t>(std::min<int64_t>(ntiles, (int64_t)c->num_sms * 2), c->nseg);
    PFE_CUDA_TRY(c, cudaMemsetAsync(&c->pctl->error, 0, sizeof(int), s));
    k_gram<T, D><<<gblocks, kBlock, 0, s>>>(a);
    k_papply<T, D><<<wave_grid(c, G_PAPPLY, k_papply<T, D>, (a.n + kBlock - 1) / kBlock), kBlock, 0, s>>>(a);
    PFE_CUDA_TRY(c, cudaGetLastError());
    return PFE_OK;
}

}  // namespace pstepk
}  // namespace pfe

#define PFE_INSTANTIATE(T, D) template pfe_status pfe::pstepk::pstep_T<T, D>(pfe_ctx *, cudaStream_t, int);
