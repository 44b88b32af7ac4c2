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
#include <cstring>
#include <type_traits>

#include "common.cuh"

namespace pfe {
namespace edgek {

template <typename T>
struct EdgeArgs {
    int64_t n, n_slices;
    int row_len;  // > 0: uniform row length
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
    Segs sg;                // batch: lambda of each row's segment
    const double *seg_lam;  // nseg
    int grid_w, grid_h;     // one grid image: its width and height (0 otherwise)
};

template <typename T, int V>
__device__ __forceinline__ void eldv(const T *__restrict__ p, T (&v)[V]) {
    if constexpr (V * sizeof(T) == 16) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        memcpy(v, &t, 16);
    } else if constexpr (V * sizeof(T) == 8) {
        const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        memcpy(v, &t, 8);
    } else {
#pragma unroll
        for (int k = 0; k < V; ++k) v[k] = __ldg(p + k);
    }
}
template <typename T, int V>
__device__ __forceinline__ void estv(T *p, const T (&v)[V]) {
    if constexpr (V * sizeof(T) == 16) {
        float4 t;
        memcpy(&t, v, 16);
        *reinterpret_cast<float4 *>(p) = t;
    } else if constexpr (V * sizeof(T) == 8) {
        float2 t;
        memcpy(&t, v, 8);
        *reinterpret_cast<float2 *>(p) = t;
    } else {
#pragma unroll
        for (int k = 0; k < V; ++k) p[k] = v[k];
    }
}

template <typename T, int D, bool MS>
__global__ void __launch_bounds__(kBlock) k_edge(EdgeArgs<T> a) {
    // L = D/V lanes per row, V consecutive columns per lane (V = widest of
    // 16/8/4 bytes dividing a row): row loads of y, b and C are contiguous
    // warp accesses and the slot work (edge id, column, weight) is shared
    // by V columns
    constexpr int V = (sizeof(T) == 4 && D % 4 == 0) ? 4 : (D % 2 == 0 ? 2 : 1);
    constexpr int L = D / V, RPW = 32 / L;
    const int lane = threadIdx.x & 31;
    const int rw = lane / L, cg = lane - rw * L, c0 = cg * V;
    const bool active = lane < RPW * L;
    const int64_t warp_g = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int64_t warps_total = (int64_t)gridDim.x * kWarps;
    for (int64_t g = warp_g; g * RPW < a.n; g += warps_total) {
        const int64_t i = g * RPW + rw;
        if (!active || i >= a.n) continue;
        int len;
        int64_t base;
        if (a.row_len > 0) {  // uniform rows (grid graphs): no slice lookup
            len = a.row_len;
            base = i * a.row_len;
        } else {
            const int64_t s = i >> 5;
            const int s0 = a.slice_ptr[s];
            len = (a.slice_ptr[s + 1] - s0) >> 5;
            base = (int64_t)s0 + (i & 31) * (int64_t)len;  // row-major within the slice
        }
        T lam = a.lambda, gam = a.gamma;
        if constexpr (MS) {  // batch: lambda of the row's segment
            const double ls = a.seg_lam[__ldg(a.sg.rseg + i)];
            lam = (T)ls;
            gam = (T)(1.0 / ls);
        }
        T yi[V], acc[V];
        eldv<T, V>(a.y + i * D + c0, yi);
#pragma unroll
        for (int k = 0; k < V; ++k) acc[k] = T(0);
        constexpr int CH = 8;  // slots prefetched together: slot loads, then gathers
        for (int k0 = 0; k0 < len; k0 += CH) {
            int ee[CH], jj[CH];
            T ww[CH], yj[CH][V], bo[CH][V];
#pragma unroll
            for (int g4 = 0; g4 < CH / 4; ++g4) {  // 16-byte loads: len is a multiple of 4
                const int k = k0 + 4 * g4;
                if (k < len) {
                    const int4 e4 = __ldg(reinterpret_cast<const int4 *>(a.eid + base + k));
                    const int4 c4 = __ldg(reinterpret_cast<const int4 *>(a.col + base + k));
                    ee[4 * g4] = e4.x; ee[4 * g4 + 1] = e4.y; ee[4 * g4 + 2] = e4.z; ee[4 * g4 + 3] = e4.w;
                    jj[4 * g4] = c4.x; jj[4 * g4 + 1] = c4.y; jj[4 * g4 + 2] = c4.z; jj[4 * g4 + 3] = c4.w;
#pragma unroll
                    for (int u = 0; u < 4; ++u) ww[4 * g4 + u] = __ldg(a.w + base + k + u);
                } else {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        ee[4 * g4 + u] = -1;
                        jj[4 * g4 + u] = (int)i;
                        ww[4 * g4 + u] = T(0);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                const int e = ee[u] < 0 ? 0 : ee[u];  // padding slots read a valid dummy
                eldv<T, V>(a.y + (int64_t)jj[u] * D + c0, yj[u]);
                eldv<T, V>(a.bs_old + (int64_t)e * D + c0, bo[u]);
            }
#pragma unroll
            for (int u = 0; u < CH; ++u) {
                if (ee[u] < 0) continue;       // padding slot
                const bool first = i < jj[u];  // i is the +w endpoint of edge e
                T bn[V];
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    const T diff = first ? (yi[k] - yj[u][k]) : (yj[u][k] - yi[k]);  // y_a - y_b
                    const T t = ww[u] * diff + bo[u][k];                              // (M Y + b)_e
                    const T z = shrink<T>(t, gam);                                    // d_e
                    bn[k] = t - z;                                                    // b'_e
                    const T v = ww[u] * (z - bn[k]);
                    acc[k] = first ? acc[k] + v : acc[k] - v;
                }
                if (first) estv<T, V>(a.bs_new + (int64_t)ee[u] * D + c0, bn);
            }
        }
        T ci[V];
        eldv<T, V>(a.cw + i * D + c0, ci);
#pragma unroll
        for (int k = 0; k < V; ++k) acc[k] = lam * acc[k] + ci[k];
        estv<T, V>(a.rhs + i * D + c0, acc);
    }
}

// Slots [P0, P1) of a fixed-position row (compile-time range): on a grid the
// lower half [0, K/2) holds the neighbours before i (i is the second endpoint
// of those edges) and the upper half [K/2, K) those after i (i owns the edge
// and writes its b').  Padding slots carry edge id -1.
template <typename T, int D, int V, int P0, int P1, bool FIRST>
__device__ __forceinline__ void edge_half(const EdgeArgs<T> &a, int64_t base, int c0, const T (&yi)[V], T gam,
                                          T (&acc)[V]) {
    constexpr int A0 = P0 & ~3, A1 = (P1 + 3) & ~3, NG = A1 - A0, NS = P1 - P0;
    int ee[NG], jj[NG];
    T ww[NG];
#pragma unroll
    for (int g4 = 0; g4 < NG / 4; ++g4) {
        const int k = A0 + 4 * g4;
        const int4 e4 = __ldg(reinterpret_cast<const int4 *>(a.eid + base + k));
        const int4 c4 = __ldg(reinterpret_cast<const int4 *>(a.col + base + k));
        ee[4 * g4] = e4.x; ee[4 * g4 + 1] = e4.y; ee[4 * g4 + 2] = e4.z; ee[4 * g4 + 3] = e4.w;
        jj[4 * g4] = c4.x; jj[4 * g4 + 1] = c4.y; jj[4 * g4 + 2] = c4.z; jj[4 * g4 + 3] = c4.w;
        if constexpr (sizeof(T) == 4) {
            const float4 w4 = __ldg(reinterpret_cast<const float4 *>(a.w + base + k));
            ww[4 * g4] = w4.x; ww[4 * g4 + 1] = w4.y; ww[4 * g4 + 2] = w4.z; ww[4 * g4 + 3] = w4.w;
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) ww[4 * g4 + u] = __ldg(a.w + base + k + u);
        }
    }
    T yj[NS][V], bo[NS][V];
#pragma unroll
    for (int u = 0; u < NS; ++u) {
        const int q = P0 - A0 + u;
        const int e = ee[q] < 0 ? 0 : ee[q];  // padding slots read a valid dummy
        eldv<T, V>(a.y + (int64_t)jj[q] * D + c0, yj[u]);
        eldv<T, V>(a.bs_old + (int64_t)e * D + c0, bo[u]);
    }
#pragma unroll
    for (int u = 0; u < NS; ++u) {
        const int q = P0 - A0 + u;
        if (ee[q] < 0) continue;  // padding slot
        T bn[V];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const T diff = FIRST ? (yi[k] - yj[u][k]) : (yj[u][k] - yi[k]);  // y_a - y_b
            const T t = ww[q] * diff + bo[u][k];                              // (M Y + b)_e
            const T z = shrink<T>(t, gam);                                    // d_e
            bn[k] = t - z;                                                    // b'_e
            const T v = ww[q] * (z - bn[k]);
            acc[k] = FIRST ? acc[k] + v : acc[k] - v;
        }
        if (FIRST) estv<T, V>(a.bs_new + (int64_t)ee[q] * D + c0, bn);
    }
}

// edge_half on one grid image without the column and edge-id arrays: slot t
// of row i = (x, y) is stencil offset (dx_t, dy_t), its neighbour j = i +
// dy_t W + dx_t when (x + dx_t, y + dy_t) lies in the image (else a padding
// slot), and the edge's b slot follows from the fixed forward positions of
// the graph builder: i K/2 + (t - K/2) for a forward slot (i owns the edge),
// j K/2 + (K - 1 - t - K/2) for a backward one (j owns it through the
// reverse offset K - 1 - t).  Only the weights are loaded; the products are
// those of edge_half, in the same order.
template <typename T, int D, int V, int P0, int P1, bool FIRST, int LEN>
__device__ __forceinline__ void edge_half_grid(const EdgeArgs<T> &a, int i, int x, int y, int c0,
                                               const T (&yi)[V], T gam, T (&acc)[V]) {
    static_assert(sizeof(T) == 4, "the float path");
    constexpr Stencil<LEN> st = make_stencil<LEN>();
    constexpr int KH = LEN / 2;
    constexpr int A0 = P0 & ~3, A1 = (P1 + 3) & ~3, NG = A1 - A0, NS = P1 - P0;
    const int64_t base = (int64_t)i * LEN;
    T ww[NG];
#pragma unroll
    for (int g4 = 0; g4 < NG / 4; ++g4) {
        const float4 w4 = __ldg(reinterpret_cast<const float4 *>(a.w + base + A0 + 4 * g4));
        ww[4 * g4] = w4.x; ww[4 * g4 + 1] = w4.y; ww[4 * g4 + 2] = w4.z; ww[4 * g4 + 3] = w4.w;
    }
    int jj[NS], ee[NS];
    bool ok[NS];
#pragma unroll
    for (int u = 0; u < NS; ++u) {
        const int t = P0 + u;
        const int dx = st.dx[t], dy = st.dy[t];
        ok[u] = (unsigned)(x + dx) < (unsigned)a.grid_w && (unsigned)(y + dy) < (unsigned)a.grid_h;
        const int j = i + dy * a.grid_w + dx;
        jj[u] = ok[u] ? j : i;
        ee[u] = ok[u] ? (FIRST ? i * KH + (t - KH) : j * KH + (LEN - 1 - t - KH)) : 0;  // padding: a valid dummy
    }
    T yj[NS][V], bo[NS][V];
#pragma unroll
    for (int u = 0; u < NS; ++u) {
        eldv<T, V>(a.y + (int64_t)jj[u] * D + c0, yj[u]);
        eldv<T, V>(a.bs_old + (int64_t)ee[u] * D + c0, bo[u]);
    }
#pragma unroll
    for (int u = 0; u < NS; ++u) {
        const int q = P0 - A0 + u;
        if (!ok[u]) continue;  // padding slot
        T bn[V];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const T diff = FIRST ? (yi[k] - yj[u][k]) : (yj[u][k] - yi[k]);  // y_a - y_b
            const T t = ww[q] * diff + bo[u][k];                              // (M Y + b)_e
            const T z = shrink<T>(t, gam);                                    // d_e
            bn[k] = t - z;                                                    // b'_e
            const T v = ww[q] * (z - bn[k]);
            acc[k] = FIRST ? acc[k] + v : acc[k] - v;
        }
        if (FIRST) estv<T, V>(a.bs_new + (int64_t)ee[u] * D + c0, bn);
    }
}

// The edge pass on fixed-position rows of LEN slots (grid graphs): the same
// arithmetic as k_edge, each half of a row as straight-line code.  GRID (one
// grid image, the float path): the columns and edge ids come from the
// stencil (edge_half_grid), so only the weights, y, b, C and the right-hand
// side move.
template <typename T, int D, bool MS, int LEN, bool GRID = false>
__global__ void __launch_bounds__(kBlock, 4) k_edge_fixed(EdgeArgs<T> a) {
    constexpr int V = (sizeof(T) == 4 && D % 4 == 0) ? 4 : (D % 2 == 0 ? 2 : 1);
    constexpr int L = D / V, RPW = 32 / L;
    const int lane = threadIdx.x & 31;
    const int rw = lane / L, cg = lane - rw * L, c0 = cg * V;
    const bool active = lane < RPW * L;
    const int64_t warp_g = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int64_t warps_total = (int64_t)gridDim.x * kWarps;
    for (int64_t g = warp_g; g * RPW < a.n; g += warps_total) {
        const int64_t i = g * RPW + rw;
        if (!active || i >= a.n) continue;
        const int64_t base = i * LEN;
        T lam = a.lambda, gam = a.gamma;
        if constexpr (MS) {  // batch: lambda of the row's segment
            const double ls = a.seg_lam[__ldg(a.sg.rseg + i)];
            lam = (T)ls;
            gam = (T)(1.0 / ls);
        }
        T yi[V], acc[V];
        eldv<T, V>(a.y + i * D + c0, yi);
#pragma unroll
        for (int k = 0; k < V; ++k) acc[k] = T(0);
        if constexpr (GRID) {
            static_assert(!MS, "computed columns: one image");
            const int ii = (int)i, y = ii / a.grid_w, x = ii - y * a.grid_w;
            edge_half_grid<T, D, V, 0, LEN / 2, false, LEN>(a, ii, x, y, c0, yi, gam, acc);
            edge_half_grid<T, D, V, LEN / 2, LEN, true, LEN>(a, ii, x, y, c0, yi, gam, acc);
        } else {
            edge_half<T, D, V, 0, LEN / 2, false>(a, base, c0, yi, gam, acc);
            edge_half<T, D, V, LEN / 2, LEN, true>(a, base, c0, yi, gam, acc);
        }
        T ci[V];
        eldv<T, V>(a.cw + i * D + c0, ci);
#pragma unroll
        for (int k = 0; k < V; ++k) acc[k] = lam * acc[k] + ci[k];
        estv<T, V>(a.rhs + i * D + c0, acc);
    }
}

template <typename T, int D>
pfe_status edge_T(pfe_ctx *c, cudaStream_t s) {
    EdgeArgs<T> a;
    a.n = c->g.n;
    a.n_slices = c->g.n_slices;
    a.row_len = c->g.row_len;
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
    a.sg = seg_view(c);
    a.seg_lam = c->seg_lam;
    const bool one_grid = c->kind == PFE_GRAPH_GRID && c->nseg == 1;
    a.grid_w = one_grid ? (int)c->W : 0;
    a.grid_h = one_grid ? (int)(c->g.n / c->W) : 0;
    constexpr int V = (sizeof(T) == 4 && D % 4 == 0) ? 4 : (D % 2 == 0 ? 2 : 1);
    constexpr int RPW = 32 / (D / V);
    const int64_t need = ((c->g.n + RPW - 1) / RPW + kWarps - 1) / kWarps;
    // fixed-position rows of 12 slots (FP32 radius-2 grids); radius 3 keeps the
    // general kernel (28 slots in straight-line code need 126 registers)
    const int rl = std::is_same_v<T, float> ? c->g.row_len : 0;
    if (c->nseg > 1) {
        if (rl == 12)
            k_edge_fixed<T, D, true, 12><<<wave_grid(c, G_EDGE, k_edge_fixed<T, D, true, 12>, need), kBlock, 0, s>>>(a);
        else
            k_edge<T, D, true><<<wave_grid(c, G_EDGE, k_edge<T, D, true>, need), kBlock, 0, s>>>(a);
    } else {
        if constexpr (std::is_same_v<T, float>) {
            if (rl == 12 && one_grid && c->edge_variant == PFE_EDGE_STENCIL) {
                k_edge_fixed<T, D, false, 12, true><<<wave_grid(c, G_EDGE_GRID, k_edge_fixed<T, D, false, 12, true>,
                                                                need),
                                                      kBlock, 0, s>>>(a);
                PFE_CUDA_TRY(c, cudaGetLastError());
                c->bs_cur = 1 - c->bs_cur;
                return PFE_OK;
            }
        }
        if (rl == 12)
            k_edge_fixed<T, D, false, 12><<<wave_grid(c, G_EDGE, k_edge_fixed<T, D, false, 12>, need), kBlock, 0,
                                            s>>>(a);
        else
            k_edge<T, D, false><<<wave_grid(c, G_EDGE, k_edge<T, D, false>, need), kBlock, 0, s>>>(a);
    }
    PFE_CUDA_TRY(c, cudaGetLastError());
    c->bs_cur = 1 - c->bs_cur;
    return PFE_OK;
}

}  // namespace edgek
}  // namespace pfe

#define PFE_INSTANTIATE(T, D) template pfe_status pfe::edgek::edge_T<T, D>(pfe_ctx *, cudaStream_t);
