// Laplacian-eigenmap start (Sec. I; Belkin & Niyogi): the d generalised
// eigenvectors of (D - W) v = mu D v with the smallest mu on the
// D-orthogonal complement of the constant vector, D-normalised, each with its
// largest-magnitude entry positive (ties: the smallest index).
//
// Method: Chebyshev-filtered subspace iteration (Zhou & Saad, 2007) on the
// random-walk matrix P = D^{-1} W, whose eigenvectors are exactly these v
// with eigenvalue theta = 1 - mu and which is self-adjoint in the D inner
// product.  A block of K >= d + 2 vectors is filtered by a degree-m Chebyshev
// polynomial that damps [-1, theta_K] (theta_K: the block's smallest Ritz
// value), then one Gram pass gives V^T D V, V^T D (P V), (P V)^T D (P V) and
// the block's constant-direction coordinates; one thread removes the
// constant direction (P 1 = 1, so the Grams update in closed form),
// orthonormalises (G^{-1/2}), takes the Ritz rotation and the residual norms
// |P v - theta v|_D from the same Grams.  FP64 throughout.
#pragma once
#include <algorithm>
#include <cmath>
#include <string>
#include <type_traits>
#include <vector>

#include "pcg_kernels.cuh"

namespace pfe {
namespace lek {

using pcgk::ldv;
using pcgk::load_slots;
using pcgk::sell_row;
using pcgk::stv;
using pcgk::SubWarp;

constexpr int kChunkLe = 8;
constexpr int kTileLe = 32;  // rows staged per Gram step

struct LeGraph {
    int64_t n;
    int row_len;
    const int *__restrict__ slice_ptr;
    const int *__restrict__ col;
    const double *__restrict__ w;    // per slot w_ij (0 on padding)
    const double *__restrict__ deg;  // d_i
};

// Y_out = alpha P Y_cur + beta Y_cur + gamma Y_prev (rows of K values)
template <int K>
__global__ void __launch_bounds__(kBlock) k_le_cheb(LeGraph g, const double *__restrict__ ycur,
                                                    const double *__restrict__ yprev, double *__restrict__ yout,
                                                    double alpha, double beta, double gamma) {
    using SW = SubWarp<double, K>;
    constexpr int V = SW::V;
    const SW lm;
    const int64_t warp_g = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int64_t warps_total = (int64_t)gridDim.x * kWarps;
    for (int64_t gr = warp_g; gr * SW::RPW < g.n; gr += warps_total) {
        const int64_t i = gr * SW::RPW + lm.r;
        if (!lm.active || i >= g.n) continue;
        const int c0 = lm.cg * V;
        int64_t base;
        int len;
        sell_row(g.slice_ptr, g.row_len, i, base, len);
        double acc[V], yi[V], yp[V];
#pragma unroll
        for (int k = 0; k < V; ++k) acc[k] = 0.0;
        for (int k0 = 0; k0 < len; k0 += kChunkLe) {
            int jj[kChunkLe];
            double wv[kChunkLe], yj[kChunkLe][V];
            load_slots<double, kChunkLe>(g.col, g.w, base, k0, len, (int)i, jj, wv);
#pragma unroll
            for (int u = 0; u < kChunkLe; ++u) ldv<double, V>(ycur + (int64_t)jj[u] * K + c0, yj[u]);
#pragma unroll
            for (int u = 0; u < kChunkLe; ++u)
#pragma unroll
                for (int k = 0; k < V; ++k) acc[k] = fma(wv[u], yj[u][k], acc[k]);
        }
        ldv<double, V>(ycur + i * K + c0, yi);
        if (yprev)
            ldv<double, V>(yprev + i * K + c0, yp);
        else
#pragma unroll
            for (int k = 0; k < V; ++k) yp[k] = 0.0;
        const double s = alpha / g.deg[i];
#pragma unroll
        for (int k = 0; k < V; ++k) acc[k] = fma(s, acc[k], fma(beta, yi[k], gamma * yp[k]));
        stv<double, V>(yout + i * K + c0, acc);
    }
}

// One Rayleigh-Ritz step (device): the reduced Grams from k_le_gram, the
// rotation and Ritz data from k_le_rr.
struct LeRR {
    unsigned ticket;
    int error;         // 1: the block lost rank (Gram not positive definite)
    double G[32 * 32], H[32 * 32], F[32 * 32], s[32];
    double theta[32];  // Ritz values, descending
    double res[32];    // |P v - theta v|_D of the Ritz vectors
    double C[32 * 32]; // rotation: V_new = V C - 1 b^T
    double b[32];
};

// Gram pass: G = V^T D V, H = V^T D (PV), F = (PV)^T D (PV) (upper triangles),
// s = V^T D 1, reduced over the rows by the last block (fixed order).
template <int K>
__global__ void __launch_bounds__(kBlock) k_le_gram(LeGraph g, const double *__restrict__ v,
                                                    const double *__restrict__ pv, double *part, LeRR *rr) {
    constexpr int NE = K * (K + 1) / 2;
    constexpr int NV = 3 * NE + K;  // G, H, F upper triangles, then s
    constexpr int PER = (NV + kBlock - 1) / kBlock;
    __shared__ double tv[kTileLe][K], tp[kTileLe][K], td[kTileLe];
    __shared__ unsigned char ep[NE], eq[NE];
    for (int e = threadIdx.x; e < NE; e += blockDim.x) {
        int p = 0, r = e;
        while (r >= K - p) {
            r -= K - p;
            ++p;
        }
        ep[e] = (unsigned char)p;
        eq[e] = (unsigned char)(p + r);
    }
    double acc[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) acc[k] = 0.0;
    __syncthreads();
    const int64_t ntiles = (g.n + kTileLe - 1) / kTileLe;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t r0 = t * kTileLe;
        for (int e = threadIdx.x; e < kTileLe * K; e += blockDim.x) {
            const int rr_ = e / K, c = e - rr_ * K;
            const int64_t i = r0 + rr_;
            const bool in = i < g.n;
            tv[rr_][c] = in ? v[i * K + c] : 0.0;
            tp[rr_][c] = in ? pv[i * K + c] : 0.0;
            if (c == 0) td[rr_] = in ? g.deg[i] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = threadIdx.x + k * kBlock;
            if (e >= NV) continue;
            double s = acc[k];
            if (e < 3 * NE) {
                const int m = e / NE, f = e - m * NE, p = ep[f], q = eq[f];
                if (m == 0)
                    for (int r = 0; r < kTileLe; ++r) s = fma(td[r] * tv[r][p], tv[r][q], s);
                else if (m == 1)
                    for (int r = 0; r < kTileLe; ++r) s = fma(td[r] * tv[r][p], tp[r][q], s);
                else
                    for (int r = 0; r < kTileLe; ++r) s = fma(td[r] * tp[r][p], tp[r][q], s);
            } else {
                const int p = e - 3 * NE;
                for (int r = 0; r < kTileLe; ++r) s = fma(td[r], tv[r][p], s);
            }
            acc[k] = s;
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = threadIdx.x + k * kBlock;
        if (e < NV) part[(int64_t)blockIdx.x * NV + e] = acc[k];
    }
    if (!last_block_arrives(&rr->ticket)) return;
    for (int e = threadIdx.x; e < NV; e += blockDim.x) {
        double s = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(part + (int64_t)b * NV + e);
        if (e < 3 * NE) {
            const int m = e / NE, f = e - m * NE, p = ep[f], q = eq[f];
            double *M = m == 0 ? rr->G : (m == 1 ? rr->H : rr->F);
            M[p * K + q] = s;
            M[q * K + p] = s;
        } else {
            rr->s[e - 3 * NE] = s;
        }
    }
    if (threadIdx.x == 0) rr->ticket = 0u;
}

// Rayleigh-Ritz on one thread, arrays in (dynamic) shared memory: remove the
// constant direction (V' = V - 1 s^T / vol; P 1 = 1 and 1^T D 1 = vol give
// G' = G - s s^T/vol, H' = H - s s^T/vol), S = G'^{-1/2},
// S H' S = Q diag(theta) Q^T, C = S Q (descending theta), b = C^T s / vol.
template <int K>
__global__ void k_le_rr(double vol, LeRR *rr) {
    extern __shared__ double sm[];
    double *Gm = sm, *Hm = Gm + K * K, *Fm = Hm + K * K, *U = Fm + K * K, *T = U + K * K, *M = T + K * K,
           *Q = M + K * K, *isq = Q + K * K;
    if (threadIdx.x != 0) return;
    for (int p = 0; p < K; ++p)
        for (int q = 0; q < K; ++q) {
            const double o = rr->s[p] * rr->s[q] / vol;
            Gm[p * K + q] = rr->G[p * K + q] - o;
            Hm[p * K + q] = 0.5 * (rr->H[p * K + q] + rr->H[q * K + p]) - o;  // D P = W: symmetric
            Fm[p * K + q] = rr->F[p * K + q] - o;
        }
    for (int k = 0; k < K * K; ++k) T[k] = Gm[k];
    jacobi_eig(T, U, K);  // G' = U diag(T) U^T
    double lmax = 0.0;
    for (int k = 0; k < K; ++k) lmax = fmax(lmax, T[k * K + k]);
    int bad = !(lmax > 0.0) || !(lmax < INFINITY);
    for (int k = 0; k < K; ++k) {
        const double l = T[k * K + k];
        if (!(l > 1e-15 * lmax)) bad = 1;
        isq[k] = l > 0.0 ? 1.0 / sqrt(l) : 0.0;
    }
    rr->error = bad;
    if (bad) return;
    for (int p = 0; p < K; ++p)  // S = G'^{-1/2}
        for (int q = 0; q < K; ++q) {
            double s = 0.0;
            for (int k = 0; k < K; ++k) s += U[p * K + k] * isq[k] * U[q * K + k];
            T[p * K + q] = s;
        }
    for (int p = 0; p < K; ++p)  // U = H' S
        for (int q = 0; q < K; ++q) {
            double s = 0.0;
            for (int k = 0; k < K; ++k) s += Hm[p * K + k] * T[k * K + q];
            U[p * K + q] = s;
        }
    for (int p = 0; p < K; ++p)  // M = S (H' S)
        for (int q = 0; q < K; ++q) {
            double s = 0.0;
            for (int k = 0; k < K; ++k) s += T[p * K + k] * U[k * K + q];
            M[p * K + q] = s;
        }
    jacobi_eig(M, Q, K);  // M = Q diag Q^T
    int ord[K];           // Ritz values descending
    for (int k = 0; k < K; ++k) ord[k] = k;
    for (int a = 1; a < K; ++a)
        for (int b = a; b > 0 && M[ord[b] * K + ord[b]] > M[ord[b - 1] * K + ord[b - 1]]; --b) {
            const int t = ord[b];
            ord[b] = ord[b - 1];
            ord[b - 1] = t;
        }
    for (int p = 0; p < K; ++p)  // C = S Q (columns in descending Ritz order)
        for (int j = 0; j < K; ++j) {
            double s = 0.0;
            for (int k = 0; k < K; ++k) s += T[p * K + k] * Q[k * K + ord[j]];
            rr->C[p * K + j] = s;
        }
    for (int j = 0; j < K; ++j) {
        rr->theta[j] = M[ord[j] * K + ord[j]];
        double bj = 0.0;
        for (int p = 0; p < K; ++p) bj += rr->s[p] * rr->C[p * K + j];
        rr->b[j] = bj / vol;
    }
}

// Residual norms of the Ritz vectors, row by row (the Gram form
// (C^T F' C)_jj - theta_j^2 cancels to about sqrt(eps)):
// P v_j - theta_j v_j = (PV C)_j - theta_j (V C)_j - (1 - theta_j) b_j 1, since P 1 = 1.
template <int K>
__global__ void __launch_bounds__(kBlock) k_le_resid(LeGraph g, const double *__restrict__ v,
                                                     const double *__restrict__ pv, double *part, LeRR *rr) {
    __shared__ double C[K * K], th[K], bb[K], red[kWarps][K];
    for (int k = threadIdx.x; k < K * K; k += blockDim.x) C[k] = rr->C[k];
    if (threadIdx.x < K) {
        th[threadIdx.x] = rr->theta[threadIdx.x];
        bb[threadIdx.x] = rr->b[threadIdx.x];
    }
    __syncthreads();
    double acc[K];
#pragma unroll
    for (int j = 0; j < K; ++j) acc[j] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
        const double di = g.deg[i];
        const double *vi = v + i * K, *pi = pv + i * K;
#pragma unroll 1
        for (int j = 0; j < K; ++j) {
            double r = -(1.0 - th[j]) * bb[j];
            for (int k = 0; k < K; ++k) r = fma(__ldg(pi + k) - th[j] * __ldg(vi + k), C[k * K + j], r);
            acc[j] = fma(di * r, r, acc[j]);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        double x = acc[j];
        for (int m = 16; m > 0; m >>= 1) x += __shfl_xor_sync(0xffffffffu, x, m);
        if (lane == 0) red[warp][j] = x;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double x = 0.0;
        for (int w = 0; w < kWarps; ++w) x += red[w][threadIdx.x];
        part[(int64_t)blockIdx.x * K + threadIdx.x] = x;
    }
    if (!last_block_arrives(&rr->ticket)) return;
    if (threadIdx.x < K) {
        double x = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) x += __ldcg(part + (int64_t)b * K + threadIdx.x);
        rr->res[threadIdx.x] = sqrt(x);
    }
    if (threadIdx.x == 0) rr->ticket = 0u;
}
template <int K>
constexpr size_t le_rr_smem() {
    return sizeof(double) * (7 * K * K + K);
}

// V_out = V C - 1 b^T, one thread per output entry (rows of V read from L1)
template <int K>
__global__ void __launch_bounds__(kBlock) k_le_apply(int64_t n, const double *__restrict__ v, const LeRR *rr,
                                                     double *__restrict__ vout) {
    __shared__ double C[K * K], b[K];
    for (int k = threadIdx.x; k < K * K; k += blockDim.x) C[k] = rr->C[k];
    if (threadIdx.x < K) b[threadIdx.x] = rr->b[threadIdx.x];
    __syncthreads();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * K; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / K;
        const int j = (int)(e - i * K);
        const double *vi = v + i * K;
        double s = -b[j];
        for (int k = 0; k < K; ++k) s = fma(__ldg(vi + k), C[k * K + j], s);
        vout[e] = s;
    }
}

// Start block: a counter-based hash of (row, column) (SplitMix64 finaliser,
// Steele, Lea & Flood 2014) mapped to [-1, 1); no state, same on every run.
__device__ __forceinline__ double hash_unit(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}
template <int K>
__global__ void k_le_start(int64_t n, double *v) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * K; e += (int64_t)gridDim.x * blockDim.x)
        v[e] = hash_unit((uint64_t)e);
}

// Sign rule, column by column: the entry of largest magnitude positive, ties
// to the smallest row.  Block maxima (|v|, row) combined in a fixed order.
struct SignCtl {
    unsigned ticket;
    int pad;
    double sign[32];
};
template <int K>
__global__ void __launch_bounds__(kBlock) k_le_signmax(int64_t n, const double *v, int d, double *pmag, int64_t *prow,
                                                       SignCtl *sc) {
    __shared__ double bm[kBlock];
    __shared__ int64_t br[kBlock];
    for (int c = 0; c < d; ++c) {
        double m = -1.0;
        int64_t r = INT64_MAX;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
            const double a = fabs(v[i * K + c]);
            if (a > m || (a == m && i < r)) {
                m = a;
                r = i;
            }
        }
        bm[threadIdx.x] = m;
        br[threadIdx.x] = r;
        __syncthreads();
        for (int s = kBlock / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) {
                const double m2 = bm[threadIdx.x + s];
                const int64_t r2 = br[threadIdx.x + s];
                if (m2 > bm[threadIdx.x] || (m2 == bm[threadIdx.x] && r2 < br[threadIdx.x])) {
                    bm[threadIdx.x] = m2;
                    br[threadIdx.x] = r2;
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            pmag[(int64_t)blockIdx.x * 32 + c] = bm[0];
            prow[(int64_t)blockIdx.x * 32 + c] = br[0];
        }
        __syncthreads();
    }
    if (!last_block_arrives(&sc->ticket)) return;
    if (threadIdx.x < d) {
        const int c = threadIdx.x;
        double m = -1.0;
        int64_t r = INT64_MAX;
        for (unsigned b = 0; b < gridDim.x; ++b) {
            const double m2 = __ldcg(pmag + (int64_t)b * 32 + c);
            const int64_t r2 = __ldcg(reinterpret_cast<const long long *>(prow) + (int64_t)b * 32 + c);
            if (m2 > m || (m2 == m && r2 < r)) {
                m = m2;
                r = r2;
            }
        }
        sc->sign[c] = (r < n && v[r * K + c] < 0.0) ? -1.0 : 1.0;
    }
    if (threadIdx.x == 0) sc->ticket = 0u;
}

// Y (n x d, row-major) = sign_c * V[:, c] for c < d
template <int K>
__global__ void k_le_out(int64_t n, const double *v, int d, const SignCtl *sc, double *y) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * d; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / d;
        const int c = (int)(e - i * d);
        y[e] = sc->sign[c] * v[i * K + c];
    }
}

// ---- host driver ---------------------------------------------------------------

template <int K>
pfe_status le_T(pfe_ctx *c, int d, double *yout, int max_iter, double tol, int degree, int *iters_out,
                double *res_out) {
    cudaStream_t s = c->stream;
    const int64_t n = c->g.n;
    const LeGraph g{n, c->g.row_len, c->g.slice_ptr, c->g.col, c->g.w64, c->g.deg};
    constexpr int NV = 3 * (K * (K + 1) / 2) + K;
    const int64_t ntiles = (n + kTileLe - 1) / kTileLe;
    const int ggrid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)c->num_sms * 2));
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_le_cheb<K>, kBlock, 0) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    using SW = SubWarp<double, K>;
    const int64_t need = ((n + SW::RPW - 1) / SW::RPW + kWarps - 1) / kWarps;
    const int cgrid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)occ * c->num_sms, need));
    const int sgrid = (int)std::min<int64_t>((n + kBlock - 1) / kBlock, (int64_t)c->num_sms * 2);
    // device work: 4 blocks of n x K, Gram partials, the Ritz block, sign data
    std::vector<void *> mem;
    auto cleanup = [&]() {
        for (void *q : mem) cudaFree(q);
    };
    auto get = [&](size_t bytes) -> void * {
        void *q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        mem.push_back(q);
        return q;
    };
    double *buf[3], *pv, *part, *pmag;
    int64_t *prow;
    LeRR *rr;
    SignCtl *sc;
    const size_t blk = sizeof(double) * (size_t)n * K;
    buf[0] = (double *)get(blk);
    buf[1] = (double *)get(blk);
    buf[2] = (double *)get(blk);
    pv = (double *)get(blk);
    part = (double *)get(sizeof(double) * std::max<size_t>((size_t)ggrid * NV, (size_t)sgrid * K));
    pmag = (double *)get(sizeof(double) * (size_t)sgrid * 32);
    prow = (int64_t *)get(sizeof(int64_t) * (size_t)sgrid * 32);
    rr = (LeRR *)get(sizeof(LeRR));
    sc = (SignCtl *)get(sizeof(SignCtl));
    for (void *q : mem)
        if (!q) {
            cleanup();
            c->err = "Laplacian eigenmap: device allocation failed";
            return PFE_ENOMEM;
        }
    if (mem.size() != 9) {
        cleanup();
        c->err = "Laplacian eigenmap: device allocation failed";
        return PFE_ENOMEM;
    }
    auto fail_cuda = [&](cudaError_t e) {
        cleanup();
        c->err = std::string("Laplacian eigenmap: ") + cudaGetErrorString(e);
        return PFE_ECUDA;
    };
    cudaError_t e = cudaMemsetAsync(rr, 0, sizeof(LeRR), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sc, 0, sizeof(SignCtl), s);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_le_rr<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)le_rr_smem<K>());
    if (e != cudaSuccess) return fail_cuda(e);
    k_le_start<K><<<sgrid, kBlock, 0, s>>>(n, buf[0]);
    int cur = 0;  // buffer holding the current block V
    double hth[32], hres[32];
    int herr = 0, it = 0;
    double bound = 0.0, rmax = INFINITY;
    // one Rayleigh-Ritz step on block buf[src]: Ritz data to the host, the
    // rotated block to buf[dst]
    auto rr_step = [&](int src, int dst) -> cudaError_t {
        k_le_cheb<K><<<cgrid, kBlock, 0, s>>>(g, buf[src], nullptr, pv, 1.0, 0.0, 0.0);  // PV = P V
        k_le_gram<K><<<ggrid, kBlock, 0, s>>>(g, buf[src], pv, part, rr);
        k_le_rr<K><<<1, 1, le_rr_smem<K>(), s>>>(c->vol, rr);
        k_le_resid<K><<<sgrid, kBlock, 0, s>>>(g, buf[src], pv, part, rr);
        cudaError_t e2 = cudaGetLastError();
        if (e2 != cudaSuccess) return e2;
        e2 = cudaMemcpyAsync(&herr, &rr->error, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(hth, rr->theta, sizeof(double) * K, cudaMemcpyDeviceToHost, s);
        if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(hres, rr->res, sizeof(double) * K, cudaMemcpyDeviceToHost, s);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(s);
        if (e2 != cudaSuccess || herr) return e2;
        k_le_apply<K><<<sgrid, kBlock, 0, s>>>(n, buf[src], rr, buf[dst]);
        return cudaGetLastError();
    };
    e = rr_step(0, 1);
    if (e != cudaSuccess) return fail_cuda(e);
    cur = 1;
    for (it = 0; it < max_iter && !herr; ++it) {
        rmax = 0.0;
        for (int j = 0; j < d; ++j) rmax = fmax(rmax, hres[j]);
        if (rmax <= tol) break;
        // Chebyshev filter of degree `degree` damping [-1, bound], bound the
        // block's smallest Ritz value: T_j((P - c) / h) V, c = (bound - 1)/2,
        // h = (bound + 1)/2, by the three-term recurrence
        bound = hth[K - 1];
        const double cc = 0.5 * (bound - 1.0), hh = 0.5 * (bound + 1.0);
        int p0 = cur, p1 = (cur + 1) % 3, p2 = (cur + 2) % 3;
        k_le_cheb<K><<<cgrid, kBlock, 0, s>>>(g, buf[p0], nullptr, buf[p1], 1.0 / hh, -cc / hh, 0.0);
        for (int j = 2; j <= degree; ++j) {
            k_le_cheb<K><<<cgrid, kBlock, 0, s>>>(g, buf[p1], buf[p0], buf[p2], 2.0 / hh, -2.0 * cc / hh, -1.0);
            const int t = p0;
            p0 = p1;
            p1 = p2;
            p2 = t;
        }
        // filtered block in buf[p1]; rotate it into buf[p0] (free)
        e = rr_step(p1, p0);
        if (e != cudaSuccess) return fail_cuda(e);
        cur = p0;
    }
    if (herr) {
        cleanup();
        c->err = "Laplacian eigenmap: the iteration block lost rank";
        return PFE_ENUMERIC;
    }
    rmax = 0.0;
    for (int j = 0; j < d; ++j) rmax = fmax(rmax, hres[j]);
    k_le_signmax<K><<<sgrid, kBlock, 0, s>>>(n, buf[cur], d, pmag, prow, sc);
    k_le_out<K><<<sgrid, kBlock, 0, s>>>(n, buf[cur], d, sc, yout);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail_cuda(e);
    cleanup();
    if (iters_out) *iters_out = it;
    if (res_out) *res_out = rmax;
    if (!(rmax <= tol)) {
        c->err = "Laplacian eigenmap: residual above tol after max_iter iterations";
        return PFE_ENOTCONV;
    }
    return PFE_OK;
}

}  // namespace lek
}  // namespace pfe

#undef PFE_INSTANTIATE
#define PFE_INSTANTIATE(T, D) \
    template pfe_status pfe::lek::le_T<D>(pfe_ctx *, int, double *, int, double, int, int *, double *);
