// Device helpers shared by the libpfe kernels: double-FP32 accumulation,
// row loads of d-interleaved arrays, block reductions, SELL-32 traversal.
#pragma once

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "internal.h"

namespace pfe {

constexpr int kBlock = 256;             // threads per block of every row kernel
constexpr int kWarps = kBlock / 32;

// ---------------------------------------------------------------------------
// Double-FP32 ("df") accumulators.  GB300 issues FP64 at about 1/60 of the
// FP32 rate, and FP32->FP64 conversions run on the same slow pipe, so bulk
// reductions keep an unevaluated sum hi + lo of two floats.  Products are
// made exact with an FMA (a*b = p + e exactly), sums use Knuth's TwoSum; the
// pair carries about 48 significant bits.  Only O(blocks x d) values are ever
// converted to FP64.
// ---------------------------------------------------------------------------
struct DF {
    float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void df_add_prod(DF &acc, float a, float b) {
    float p = __fmul_rn(a, b);
    float pe = __fmaf_rn(a, b, -p);  // exact: a*b = p + pe
    float s, se;
    two_sum(acc.hi, p, s, se);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(se, pe));
}

__device__ __forceinline__ void df_add_f(DF &acc, float v) {
    float s, se;
    two_sum(acc.hi, v, s, se);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, se);
}

__device__ __forceinline__ void df_add(DF &acc, DF b) {
    float s, se;
    two_sum(acc.hi, b.hi, s, se);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(se, b.lo));
}

__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }

// Accumulator type of each working precision: float data -> DF, double -> double.
template <typename T>
struct Acc;
template <>
struct Acc<float> {
    using type = DF;
    __device__ static __forceinline__ DF zero() { return DF{0.f, 0.f}; }
    __device__ static __forceinline__ void add_prod(DF &a, float x, float y) { df_add_prod(a, x, y); }
    __device__ static __forceinline__ void add(DF &a, DF b) { df_add(a, b); }
    __device__ static __forceinline__ DF shfl_xor(DF a, int m) {
        return DF{__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m)};
    }
    __device__ static __forceinline__ double to_double(DF a) { return df_to_double(a); }
};
template <>
struct Acc<double> {
    using type = double;
    __device__ static __forceinline__ double zero() { return 0.0; }
    __device__ static __forceinline__ void add_prod(double &a, double x, double y) { a = fma(x, y, a); }
    __device__ static __forceinline__ void add(double &a, double b) { a += b; }
    __device__ static __forceinline__ double shfl_xor(double a, int m) {
        return __shfl_xor_sync(0xffffffffu, a, m);
    }
    __device__ static __forceinline__ double to_double(double a) { return a; }
};

// ---------------------------------------------------------------------------
// Row I/O for n x D row-major ("d-interleaved") arrays: the widest aligned
// vector access that divides a row.
// ---------------------------------------------------------------------------
template <typename T, int D>
__device__ __forceinline__ void load_row(const T *__restrict__ base, int64_t i, T (&v)[D]) {
    const T *src = base + i * D;
    constexpr int BYTES = D * (int)sizeof(T);
    if constexpr (BYTES % 16 == 0) {
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
#pragma unroll
        for (int k = 0; k < BYTES / 16; ++k) {
            float4 t = __ldg(s4 + k);
            memcpy(reinterpret_cast<char *>(v) + 16 * k, &t, 16);
        }
    } else if constexpr (BYTES % 8 == 0) {
        const float2 *s2 = reinterpret_cast<const float2 *>(src);
#pragma unroll
        for (int k = 0; k < BYTES / 8; ++k) {
            float2 t = __ldg(s2 + k);
            memcpy(reinterpret_cast<char *>(v) + 8 * k, &t, 8);
        }
    } else {
#pragma unroll
        for (int k = 0; k < D; ++k) v[k] = __ldg(src + k);
    }
}

// Same, through the coherent path (for arrays written earlier in the same kernel
// by other threads is never needed here; used for read-write arrays).
template <typename T, int D>
__device__ __forceinline__ void load_row_rw(const T *base, int64_t i, T (&v)[D]) {
    const T *src = base + i * D;
    constexpr int BYTES = D * (int)sizeof(T);
    if constexpr (BYTES % 16 == 0) {
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
#pragma unroll
        for (int k = 0; k < BYTES / 16; ++k) {
            float4 t = s4[k];
            memcpy(reinterpret_cast<char *>(v) + 16 * k, &t, 16);
        }
    } else if constexpr (BYTES % 8 == 0) {
        const float2 *s2 = reinterpret_cast<const float2 *>(src);
#pragma unroll
        for (int k = 0; k < BYTES / 8; ++k) {
            float2 t = s2[k];
            memcpy(reinterpret_cast<char *>(v) + 8 * k, &t, 8);
        }
    } else {
#pragma unroll
        for (int k = 0; k < D; ++k) v[k] = src[k];
    }
}

template <typename T, int D>
__device__ __forceinline__ void store_row(T *base, int64_t i, const T (&v)[D]) {
    T *dst = base + i * D;
    constexpr int BYTES = D * (int)sizeof(T);
    if constexpr (BYTES % 16 == 0) {
        float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
        for (int k = 0; k < BYTES / 16; ++k) {
            float4 t;
            memcpy(&t, reinterpret_cast<const char *>(v) + 16 * k, 16);
            d4[k] = t;
        }
    } else if constexpr (BYTES % 8 == 0) {
        float2 *d2 = reinterpret_cast<float2 *>(dst);
#pragma unroll
        for (int k = 0; k < BYTES / 8; ++k) {
            float2 t;
            memcpy(&t, reinterpret_cast<const char *>(v) + 8 * k, 8);
            d2[k] = t;
        }
    } else {
#pragma unroll
        for (int k = 0; k < D; ++k) dst[k] = v[k];
    }
}

// ---------------------------------------------------------------------------
// Block reduction of NV accumulators; thread t < NV receives the block total
// of value t (as double).  All threads must call it.  Fixed order, so the
// result does not depend on timing.
// ---------------------------------------------------------------------------
template <typename T, int NV>
__device__ __forceinline__ void block_reduce(typename Acc<T>::type (&v)[NV], double *out_block) {
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
        out_block[c] = A::to_double(s);
    }
}

// "Last block done" detection: every block calls this after writing its
// partials; exactly one block (the last to arrive) gets true and must reset
// the ticket.  No waiting is involved.
__device__ __forceinline__ bool last_block_arrives(unsigned *ticket, unsigned count) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(ticket, 1u);
        am_last = (t == count - 1);
    }
    __syncthreads();
    if (am_last) __threadfence();
    return am_last;
}
__device__ __forceinline__ bool last_block_arrives(unsigned *ticket) { return last_block_arrives(ticket, gridDim.x); }

// Cyclic Jacobi eigendecomposition of the symmetric G (in place -> diagonal),
// V receives the eigenvectors as columns.  Golub & Van Loan, Alg. 8.5.3.
static __device__ __noinline__ void jacobi_eig(double *G, double *V, int D) {
    for (int p = 0; p < D; ++p)
        for (int q = 0; q < D; ++q) V[p * D + q] = (p == q) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int p = 0; p < D; ++p) {
            dia += G[p * D + p] * G[p * D + p];
            for (int q = p + 1; q < D; ++q) off += G[p * D + q] * G[p * D + q];
        }
        if (off <= 1e-32 * dia) break;
        for (int p = 0; p < D - 1; ++p) {
            for (int q = p + 1; q < D; ++q) {
                const double apq = G[p * D + q];
                if (apq == 0.0) continue;
                const double tau = (G[q * D + q] - G[p * D + p]) / (2.0 * apq);
                const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                const double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
                for (int k = 0; k < D; ++k) {  // columns p, q of G J
                    const double gp = G[k * D + p], gq = G[k * D + q];
                    G[k * D + p] = cs * gp - sn * gq;
                    G[k * D + q] = sn * gp + cs * gq;
                }
                for (int k = 0; k < D; ++k) {  // rows p, q of J^T (G J)
                    const double gp = G[p * D + k], gq = G[q * D + k];
                    G[p * D + k] = cs * gp - sn * gq;
                    G[q * D + k] = sn * gp + cs * gq;
                }
                for (int k = 0; k < D; ++k) {  // V J
                    const double vp = V[k * D + p], vq = V[k * D + q];
                    V[k * D + p] = cs * vp - sn * vq;
                    V[k * D + q] = sn * vp + cs * vq;
                }
            }
        }
    }
}

// ---- segments ----------------------------------------------------------------
// The blocks of a grid of G >= nseg blocks are split among the segments in
// proportion to their rows, at least one each: segment s owns blocks
// [seg_first_block(s), seg_first_block(s + 1)).
__device__ __forceinline__ int seg_first_block(const Segs &sg, int s, int G) {
    return s + (int)(((int64_t)(G - sg.nseg) * sg.off[s]) / sg.n);
}
struct BlockSeg {
    int seg, b0, nb;  // segment of this block, its first block and block count
    int64_t r0, r1;   // its rows
};
// MS = false: a single problem known at compile time (no segment lookups).
template <bool MS = true>
__device__ __forceinline__ BlockSeg block_seg(const Segs &sg) {
    BlockSeg o;
    const int G = (int)gridDim.x, b = (int)blockIdx.x;
    if (!MS || sg.nseg == 1) {
        o.seg = 0;
        o.b0 = 0;
        o.nb = G;
        o.r0 = 0;
        o.r1 = sg.n;
        return o;
    }
    int lo = 0, hi = sg.nseg - 1;  // the last segment whose first block is <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg_first_block(sg, mid, G) <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    o.seg = lo;
    o.b0 = seg_first_block(sg, lo, G);
    o.nb = seg_first_block(sg, lo + 1, G) - o.b0;
    o.r0 = sg.off[lo];
    o.r1 = sg.off[lo + 1];
    return o;
}
__device__ __forceinline__ int row_seg(const Segs &sg, int64_t i) { return sg.nseg == 1 ? 0 : __ldg(sg.rseg + i); }

__device__ __forceinline__ double ld_cg(const double *p) { return __ldcg(p); }

// Grid of a grid-stride kernel: exactly one wave of the kernel's own
// occupancy (a second, partial wave would leave most SMs idle while it
// runs), or of the blocks per SM the autotuner chose for the kernel
// (c->kbps[slot]), capped at `need` blocks and rounded down to a multiple of
// `mult`.  Cached per context in c->kgrid[slot].
enum GridSlot {
    G_INIT = 0, G_INIT_F, G_PUPD, G_SPMM, G_UPDATE, G_FSAI_TR, G_XFLUSH, G_REFRESH, G_REFRESH_F,
    G_FSAI_T, G_FSAI_T1, G_FSAI_ZP, G_APPLY, G_EDGE, G_PAPPLY, G_TIME_SPMM, G_TIME_UPDATE, G_SPMM_F1, G_SPMM_F2,
    G_SPMM_F3, G_SPMM_TMA, G_SPMM_STENCIL, G_IC_R, G_IC_DOTS, G_SPMM_G1, G_SPMM_G2, G_EDGE_GRID, G_NSLOTS
};
// Strip width of the stencil SpMM pipeline for d columns, rows of len
// slots (radius 2: 12, radius 3: 28) and p steps in flight: the widest
// multiple of 4 of whole row groups of the float sub-warp mapping (V = 4, 2
// or 1 columns a lane) up to one pass of kWarps warps whose shared memory
// (a ring of 2R + 1 + p row bands, p + 1 rows of matrix values and
// diagonal) fits 41 KB with every copy 16-byte aligned; 0 if none does.
// Stencil of a grid graph with fixed slot positions: slot t of every row is
// the t-th offset (dy, dx), 0 < dx^2 + dy^2 <= R^2, in (dy, dx) order (the
// order the graph builder lists them); 12 slots at radius 2, 28 at radius 3.
template <int LEN>
struct Stencil {
    static constexpr int R = LEN == 12 ? 2 : 3;
    int dx[LEN], dy[LEN];
};
template <int LEN>
constexpr Stencil<LEN> make_stencil() {
    Stencil<LEN> st{};
    constexpr int R = Stencil<LEN>::R;
    int k = 0;
    for (int y = -R; y <= R; ++y)
        for (int x = -R; x <= R; ++x)
            if (x * x + y * y > 0 && x * x + y * y <= R * R && k < LEN) {
                st.dy[k] = y;
                st.dx[k] = x;
                ++k;
            }
    return st;
}
template <int LEN>
constexpr int stencil_count() {
    constexpr int R = Stencil<LEN>::R;
    int k = 0;
    for (int y = -R; y <= R; ++y)
        for (int x = -R; x <= R; ++x) k += (x * x + y * y > 0 && x * x + y * y <= R * R) ? 1 : 0;
    return k;
}

// Level schedule of the incomplete-Cholesky triangular solves on a grid
// image in raster order: pixel (x, y) gets level x + CL y, so every lower
// stencil neighbour (dy < 0, or dy = 0 and dx < 0) has a smaller level and
// the rows of one level are independent.  CL = 1 + the largest dx among the
// offsets with dy = -1 (2 at radius 2, 3 at radius 3).
template <int LEN>
constexpr int ic_level_coef() {
    constexpr Stencil<LEN> st = make_stencil<LEN>();
    int m = 0;
    for (int t = 0; t < LEN; ++t)
        if (st.dy[t] == -1 && st.dx[t] > m) m = st.dx[t];
    return m + 1;
}
template <int LEN>
constexpr bool ic_levels_ok() {
    constexpr Stencil<LEN> st = make_stencil<LEN>();
    constexpr int cl = ic_level_coef<LEN>();
    for (int t = 0; t < LEN / 2; ++t)  // the lower offsets
        if (!(cl * -st.dy[t] - st.dx[t] > 0)) return false;
    return true;
}
// rows of level l of a W x H image: y in [y0, y0 + count), x = l - cl y
__host__ __device__ inline void ic_level_rows(int64_t l, int64_t W, int64_t H, int cl, int64_t &y0, int64_t &count) {
    const int64_t lo = l - (W - 1) <= 0 ? 0 : (l - (W - 1) + cl - 1) / cl;
    const int64_t hi = l / cl < H - 1 ? l / cl : H - 1;
    y0 = lo;
    count = hi >= lo ? hi - lo + 1 : 0;
}
inline int64_t ic_levels(int64_t W, int64_t H, int cl) { return (W - 1) + cl * (H - 1) + 1; }

constexpr int kStencilSteps = 3;  // steps of the stencil SpMM pipeline in flight (5 measured slower)
constexpr int stencil_strip(int d, int len, int p) {
    const int r = len == 12 ? 2 : 3;
    const int v = d % 4 == 0 ? 4 : (d % 2 == 0 ? 2 : 1);
    const int rpw = 32 / (d / v);
    const int q = d % 4 == 0 ? 1 : (d % 2 == 0 ? 2 : 4);  // pixels per 16 bytes
    const int padl = (r % q == 0) ? 0 : q - r % q;
    for (int ts = kWarps * rpw; ts >= rpw; ts -= rpw) {
        const int brows = (ts + 2 * r + padl + q - 1 + q - 1) / q * q;
        const int bytes = 4 * ((2 * r + 1 + p) * brows * d + (p + 1) * ts * len + (p + 1) * ts);
        if (ts % 4 == 0 && bytes <= 41 * 1024) return ts;
    }
    return 0;
}

inline Segs seg_view(const pfe_ctx *c) { return Segs{c->nseg, c->g.n, c->seg_off, c->rseg}; }

// One allocation holds every array of a SegScal: bytes needed, and the
// arrays carved from a base pointer (doubles first, then ints).
inline size_t segscal_bytes(int nseg, int d) {
    return sizeof(double) * 9 * (size_t)nseg * d + sizeof(long long) * (size_t)nseg +
           sizeof(int) * (2 * (size_t)nseg * d + 3 * (size_t)nseg) + sizeof(unsigned) * 4 * (size_t)nseg;
}
inline SegScal segscal_carve(void *base, int nseg, int d) {
    SegScal sc;
    double *dp = reinterpret_cast<double *>(base);
    const size_t nd = (size_t)nseg * d;
    sc.bnorm = dp;
    sc.rz = dp + nd;
    sc.alpha = dp + 2 * nd;
    sc.beta = dp + 3 * nd;
    sc.relres = dp + 4 * nd;
    sc.alpha_prev = dp + 5 * nd;
    sc.rel_ref = dp + 6 * nd;
    sc.rec2 = dp + 7 * nd;
    sc.devr = dp + 8 * nd;
    sc.seg_iters_tot = reinterpret_cast<long long *>(dp + 9 * nd);
    int *ip = reinterpret_cast<int *>(sc.seg_iters_tot + nseg);
    sc.active = ip;
    sc.pending = ip + nd;
    sc.seg_active = ip + 2 * nd;
    sc.seg_iters = ip + 2 * nd + nseg;
    sc.seg_live = ip + 2 * nd + 2 * nseg;
    sc.ticket = reinterpret_cast<unsigned *>(ip + 2 * nd + 3 * nseg);
    return sc;
}

template <typename K>
inline int wave_grid(pfe_ctx *c, int slot, K kernel, int64_t need, int mult = 1, size_t smem = 0) {
    int &g = c->kgrid[slot];
    if (g == 0) {
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kBlock, smem) != cudaSuccess || occ < 1) {
            cudaGetLastError();
            occ = 1;
        }
        int64_t grid = (int64_t)occ * c->num_sms;
        if (c->prm.blocks_per_sm > 0) grid = std::min<int64_t>(grid, (int64_t)c->prm.blocks_per_sm * c->num_sms);
        if (c->kbps[slot] > 0) grid = std::min<int64_t>(grid, (int64_t)c->kbps[slot] * c->num_sms);  // pfe_autotune
        grid = std::min<int64_t>(grid, std::max<int64_t>(need, 1));
        if (mult > 1) grid = std::max<int64_t>(mult, grid / mult * mult);
        // every segment owns at least one block of a row kernel
        if (grid < c->nseg) grid = (c->nseg + std::max(mult, 1) - 1) / std::max(mult, 1) * std::max(mult, 1);
        g = (int)grid;
    }
    return g;
}

template <typename T>
__device__ __forceinline__ T shrink(T t, T gamma) {
    // Alg. 2 Shrink: sign(t) * max(|t| - gamma, 0); NaN propagates.
    T m = fabs(t) - gamma;
    if (m > T(0)) return copysign(m, t);
    return (t != t) ? t : T(0);
}

}  // namespace pfe
