// Kernels of the d-column Jacobi-preconditioned conjugate gradients on
// A Y = RHS, the normal equations of Eq. 13 (Sec. III, last paragraph: PCG in
// place of a direct solve).  Each column c runs the textbook recurrences
// (Barrett et al., Templates, PCG) with its own alpha_c, beta_c; a column
// whose relative residual |r_c| / |b_c| reaches tol is frozen (alpha_c = 0).
//
// Thread mapping of the gather kernels (SubWarp): L = d/V lanes per row, V
// consecutive columns per lane, so every load of a d-interleaved row -- own
// or gathered neighbour -- is one contiguous warp access and a matrix slot
// (col, value) is fetched once per V columns.  The elementwise kernels use a
// flat float4/double2 traversal.
//
// A Jacobi iteration is three launches (plus two that exit at once except
// every `refresh` iterations; the FSAI iteration is listed further down):
//   k_pupdate  p = z + beta p (z = D_A^{-1} r) and y += alpha_prev p_prev (the
//              solution update of the previous iteration, delayed to share
//              this pass), in place
//   k_spmm     q = A p, partials of p.q -> alpha
//   k_update   r -= alpha q, partials of r.z and r.r -> beta, convergence
//   k_xflush   (refresh iterations) y += alpha p
//   k_refresh  (refresh iterations) r = b - A y in extended precision
// and k_xflush once after the loop.  Scalars live in
// a device control block; the last block of each reduction (atomic ticket,
// no waiting) finishes the scalar work, so the loop runs inside a CUDA graph
// whose WHILE node reads the flag set here.
#pragma once
#include <cstring>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "tma.cuh"

namespace pfe {
namespace pcgk {

constexpr int kChunk = 12;  // matrix slots prefetched together by the gather kernels

template <typename T>
struct SysView {
    int64_t n, n_slices;
    int row_len;  // > 0: uniform row length (row i's slots at i * row_len)
    const int *__restrict__ slice_ptr;
    const int *__restrict__ col;
    const T *__restrict__ aoff;
    const T *__restrict__ adiag;
    const T *__restrict__ dinv;
    const float *__restrict__ aofflo;    // FP32 low parts of A's values (the float path's residual replacement)
    const float *__restrict__ adiaglo;
};

template <typename T>
struct PcgArgs {
    SysView<T> A;
    T *x;        // solution (hi part when T = float)
    float *xlo;  // low part (float path only)
    T *r, *q;
    T *p[2];     // direction, double-buffered
    const T *b;
    void *part;  // block partials, Acc<T>::type
    PcgCtl *ctl;
    Segs sg;     // segments (a batch of problems; nseg = 1 for one)
    SegScal sc;  // per-segment scalars [seg * D + c]
    cudaGraphConditionalHandle cond;
    int use_cond;
    int if_pos;  // >= 0: this launch decides the replacement of the body's iteration if_pos (its IF node)
    int grid_w;  // width of the image of a one-image grid graph (0 otherwise)
    // FSAI preconditioner (float path): t = G r; the residual alternates
    // between r2[0] (= r) and r2[1]
    T *t;
    T *r2[2];
    const T *gdiag, *gslot;
    const int *kb;
};

template <typename T>
SysView<T> sys_view(pfe_ctx *c) {
    SysView<T> v;
    v.n = c->g.n;
    v.n_slices = c->g.n_slices;
    v.row_len = c->g.row_len;
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
    v.aofflo = c->g.aofflo32;
    v.adiaglo = c->g.adiaglo32;
    return v;
}

// Sub-warp mapping of a d-interleaved row: V consecutive columns per lane
// (V = the widest of 16/8/4 bytes that divides a row), L = D/V lanes per row,
// RPW = floor(32/L) rows per warp.  Gathered rows are contiguous runs of
// L*V*sizeof(T) bytes and the per-slot scalar work (column index, matrix
// value) is shared by V columns.
template <typename T, int D>
struct SubWarp {
    static constexpr int V = (sizeof(T) == 4 && D % 4 == 0) ? 4 : (D % 2 == 0 ? 2 : 1);
    static constexpr int L = D / V;
    static constexpr int RPW = 32 / L;
    int r, cg;
    bool active;
    __device__ __forceinline__ SubWarp() {
        const int lane = threadIdx.x & 31;
        r = lane / L;
        cg = lane - r * L;
        active = lane < RPW * L;
    }
};

template <typename T, int V>
__device__ __forceinline__ void ldv(const T *__restrict__ p, T (&v)[V]) {
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
// coherent load (array written earlier in the same launch by this thread only)
template <typename T, int V>
__device__ __forceinline__ void ldv_rw(const T *p, T (&v)[V]) {
    if constexpr (V * sizeof(T) == 16) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        memcpy(v, &t, 16);
    } else if constexpr (V * sizeof(T) == 8) {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        memcpy(v, &t, 8);
    } else {
#pragma unroll
        for (int k = 0; k < V; ++k) v[k] = p[k];
    }
}
template <typename T, int V>
__device__ __forceinline__ void stv(T *p, const T (&v)[V]) {
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

// SELL-32 slot addressing of row i (row-major within the slice): slot k is at
// base + k; len is a multiple of 4 and base is 16-byte aligned.  With a
// uniform row length (grid graphs) the address is computed, saving the
// dependent slice lookup ahead of the slot loads.
__device__ __forceinline__ void sell_row(const int *__restrict__ slice_ptr, int row_len, int64_t i, int64_t &base,
                                         int &len) {
    if (row_len > 0) {
        len = row_len;
        base = i * row_len;
        return;
    }
    const int64_t s = i >> 5;
    const int s0 = slice_ptr[s];
    len = (slice_ptr[s + 1] - s0) >> 5;
    base = (int64_t)s0 + (i & 31) * (int64_t)len;
}

// Slots k0 .. k0+CH-1 of a row (CH a multiple of 4): column and value with
// 16-byte vector loads; slots past len give (own row, 0).
template <typename T, int CH>
__device__ __forceinline__ void load_slots(const int *__restrict__ col, const T *__restrict__ val, int64_t base,
                                           int k0, int len, int self, int (&jj)[CH], T (&av)[CH]) {
#pragma unroll
    for (int g4 = 0; g4 < CH / 4; ++g4) {
        const int k = k0 + 4 * g4;
        if (k < len) {
            const int4 cv = __ldg(reinterpret_cast<const int4 *>(col + base + k));
            jj[4 * g4] = cv.x;
            jj[4 * g4 + 1] = cv.y;
            jj[4 * g4 + 2] = cv.z;
            jj[4 * g4 + 3] = cv.w;
            if constexpr (sizeof(T) == 4) {
                const float4 vv = __ldg(reinterpret_cast<const float4 *>(val + base + k));
                av[4 * g4] = vv.x;
                av[4 * g4 + 1] = vv.y;
                av[4 * g4 + 2] = vv.z;
                av[4 * g4 + 3] = vv.w;
            } else {
                const double2 v0 = __ldg(reinterpret_cast<const double2 *>(val + base + k));
                const double2 v1 = __ldg(reinterpret_cast<const double2 *>(val + base + k + 2));
                av[4 * g4] = v0.x;
                av[4 * g4 + 1] = v0.y;
                av[4 * g4 + 2] = v1.x;
                av[4 * g4 + 3] = v1.y;
            }
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                jj[4 * g4 + u] = self;
                av[4 * g4 + u] = T(0);
            }
        }
    }
}

// Slots [P0, P1) of a fixed-length row (base a multiple of 4 slots): the
// widest aligned pieces (4, 2 or 1 slots) that tile the range exactly, so no
// slot outside it is fetched.  4-byte values (the float path).
template <typename T, int P0, int P1, int K = P0>
__device__ __forceinline__ void load_slot_range(const int *__restrict__ col, const T *__restrict__ val, int64_t base,
                                                int (&jj)[P1 - P0], T (&av)[P1 - P0]) {
    static_assert(sizeof(T) == 4, "4-byte slot values");
    if constexpr (K < P1) {
        constexpr int W = (K % 4 == 0 && K + 4 <= P1) ? 4 : (K % 2 == 0 && K + 2 <= P1) ? 2 : 1;
        constexpr int u = K - P0;
        if constexpr (W == 4) {
            const int4 cv = __ldg(reinterpret_cast<const int4 *>(col + base + K));
            const float4 vv = __ldg(reinterpret_cast<const float4 *>(val + base + K));
            jj[u] = cv.x; jj[u + 1] = cv.y; jj[u + 2] = cv.z; jj[u + 3] = cv.w;
            av[u] = vv.x; av[u + 1] = vv.y; av[u + 2] = vv.z; av[u + 3] = vv.w;
        } else if constexpr (W == 2) {
            const int2 cv = __ldg(reinterpret_cast<const int2 *>(col + base + K));
            const float2 vv = __ldg(reinterpret_cast<const float2 *>(val + base + K));
            jj[u] = cv.x; jj[u + 1] = cv.y;
            av[u] = vv.x; av[u + 1] = vv.y;
        } else {
            jj[u] = __ldg(col + base + K);
            av[u] = __ldg(val + base + K);
        }
        load_slot_range<T, P0, P1, K + W>(col, val, base, jj, av);
    }
}

// Values of slots [P0, P1) of a fixed-length row, as load_slot_range without
// the columns.
template <typename T, int P0, int P1, int K = P0>
__device__ __forceinline__ void load_val_range(const T *__restrict__ val, int64_t base, T (&av)[P1 - P0]) {
    static_assert(sizeof(T) == 4, "4-byte slot values");
    if constexpr (K < P1) {
        constexpr int W = (K % 4 == 0 && K + 4 <= P1) ? 4 : (K % 2 == 0 && K + 2 <= P1) ? 2 : 1;
        constexpr int u = K - P0;
        if constexpr (W == 4) {
            const float4 vv = __ldg(reinterpret_cast<const float4 *>(val + base + K));
            av[u] = vv.x; av[u + 1] = vv.y; av[u + 2] = vv.z; av[u + 3] = vv.w;
        } else if constexpr (W == 2) {
            const float2 vv = __ldg(reinterpret_cast<const float2 *>(val + base + K));
            av[u] = vv.x; av[u + 1] = vv.y;
        } else {
            av[u] = __ldg(val + base + K);
        }
        load_val_range<T, P0, P1, K + W>(val, base, av);
    }
}

// Column of slot T of row i of a one-image grid graph of width w and n
// pixels, computed from the stencil (make_stencil: slot T is the T-th offset
// in (dy, dx) order) instead of loaded: i + dy_T w + dx_T,
// clamped into [0, n).  A slot whose neighbour is off the image has value 0
// (padding), so any row serves there; clamping only keeps the address valid
// (a backward slot can only fall below row 0, a forward one past row n - 1).
template <int LEN, int T>
__device__ __forceinline__ int stencil_col(int i, int w, int n) {
    static_assert(stencil_count<LEN>() == LEN, "12 slots: radius 2, 28: radius 3");
    constexpr Stencil<LEN> st = make_stencil<LEN>();
    constexpr int dy = st.dy[T], dx = st.dx[T];
    const int j = i + dy * w + dx;
    if constexpr (T < LEN / 2)
        return max(j, 0);
    else
        return min(j, n - 1);
}
template <int LEN, int P0, int K = P0, int N>
__device__ __forceinline__ void stencil_cols(int i, int w, int n, int (&jj)[N]) {
    if constexpr (K < P0 + N) {
        jj[K - P0] = stencil_col<LEN, K>(i, w, n);
        stencil_cols<LEN, P0, K + 1>(i, w, n, jj);
    }
}

// ---- reductions -------------------------------------------------------------

template <typename A, typename AT>
__device__ __forceinline__ AT ld_part(const AT *p) {
    if constexpr (std::is_same_v<AT, double>) {
        return __ldcg(p);
    } else {
        float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
        return AT{v.x, v.y};
    }
}

// Each lane holds NQ x V accumulators for columns cg*V + v of its row; block
// totals per (quantity, column) land in sh[q*D + c].  Fixed order.
template <typename T, int D, int NQ>
__device__ __forceinline__ void block_sum_cols(typename Acc<T>::type (&v)[NQ][SubWarp<T, D>::V],
                                               typename Acc<T>::type *sh) {
    using A = Acc<T>;
    using AT = typename A::type;
    using SW = SubWarp<T, D>;
    __shared__ AT red[NQ][kWarps][32][SW::V];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int k = 0; k < SW::V; ++k) red[q][warp][lane][k] = v[q][k];
    __syncthreads();
    // two stages (shorter dependent chains than one thread a value): thread
    // (t, w) adds warp w's rows of value t, then thread t adds the warps, in
    // a fixed order
    __shared__ AT wsum[kWarps][NQ * D];
    for (int e = threadIdx.x; e < kWarps * NQ * D; e += blockDim.x) {
        const int w = e / (NQ * D), t = e - w * (NQ * D);
        const int q = t / D, c = t - q * D, cg = c / SW::V, k = c - cg * SW::V;
        AT s = A::zero();
        for (int r = 0; r < SW::RPW; ++r) A::add(s, red[q][w][r * SW::L + cg][k]);
        wsum[w][t] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NQ * D; t += blockDim.x) {
        AT s = wsum[0][t];
        for (int w = 1; w < kWarps; ++w) A::add(s, wsum[w][t]);
        sh[t] = s;
    }
    __syncthreads();
}

// Write this block's NQ*D partials; the last block of the segment to arrive
// reduces the partials of the segment's blocks in a fixed order into
// out[0..NQ*D) (shared) and returns true.
template <typename T, int D, int NQ>
__device__ __forceinline__ bool grid_sum_cols(typename Acc<T>::type (&v)[NQ][SubWarp<T, D>::V], void *part_v,
                                              const BlockSeg &bsg, unsigned *ticket, double *out) {
    using A = Acc<T>;
    using AT = typename A::type;
    constexpr int NV = NQ * D;
    __shared__ AT sh[NV];
    AT *part = reinterpret_cast<AT *>(part_v);
    block_sum_cols<T, D, NQ>(v, sh);
    for (int t = threadIdx.x; t < NV; t += blockDim.x) part[(int64_t)blockIdx.x * NV + t] = sh[t];
    if (!last_block_arrives(ticket, (unsigned)bsg.nb)) return false;
    part += (int64_t)bsg.b0 * NV;
    // last block: G threads per value, thread (v, h) sums blocks h, h+G, ...;
    // the G partials of a value are then added in order (fixed order overall)
    constexpr int G = (kBlock / NV) > 0 ? (kBlock / NV) : 1;
    __shared__ AT pr[G][NV];
    if (threadIdx.x < G * NV) {
        const int v = threadIdx.x % NV, h = threadIdx.x / NV;
        const int nb = bsg.nb;
        AT s = A::zero();
        // sixteen independent loads in flight, then the additions in block order
        for (int b0 = h; b0 < nb; b0 += 16 * G) {
            AT vals[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int b = b0 + u * G;
                vals[u] = b < nb ? ld_part<A, AT>(part + (int64_t)b * NV + v) : A::zero();
            }
#pragma unroll
            for (int u = 0; u < 16; ++u)
                if (b0 + u * G < nb) A::add(s, vals[u]);
        }
        pr[h][v] = s;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NV; t += blockDim.x) {
        AT s = pr[0][t];
        for (int h = 1; h < G; ++h) A::add(s, pr[h][t]);
        out[t] = A::to_double(s);
    }
    if (threadIdx.x == 0) *ticket = 0u;
    __syncthreads();
    return true;
}

// Column sums of non-negative terms x*y (squared norms, r.D^{-1}r): no
// cancellation, so the float path adds each lane's terms in FP32 over runs of
// at most kSqChunk rows (relative error of a run <= (kSqChunk - 1) u) and
// adds the runs to a double-FP32 sum kept in shared memory (one slot per
// thread, so the registers of the gathers stay free): one FMA a term instead
// of the ~10 operations of an exact product.  FP64 adds every term with one
// FMA in registers.  `sh` holds NQ * V * kBlock DF (float path).
constexpr int kSqChunk = 16;
template <typename T, int NQ, int V>
struct SqSum {
    using AT = typename Acc<T>::type;
    static constexpr bool kFloat = std::is_same_v<T, float>;
    AT acc[NQ][V];  // FP64: the sums; float: filled by finish()
    float run[NQ][V];  // float: the current runs
    DF *sh;
    int cnt;
    __device__ __forceinline__ explicit SqSum(DF *shared_base) : sh(shared_base + threadIdx.x), cnt(0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q)
#pragma unroll
            for (int k = 0; k < V; ++k) {
                acc[q][k] = Acc<T>::zero();
                run[q][k] = 0.f;
                if constexpr (kFloat) sh[(q * V + k) * kBlock] = DF{0.f, 0.f};
            }
    }
    __device__ __forceinline__ void add(int q, int k, T x, T y) {
        if constexpr (kFloat)
            run[q][k] = __fmaf_rn(x, y, run[q][k]);
        else
            acc[q][k] = fma(x, y, acc[q][k]);
    }
    __device__ __forceinline__ void flush() {
        if constexpr (kFloat) {
#pragma unroll
            for (int q = 0; q < NQ; ++q)
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    DF d = sh[(q * V + k) * kBlock];
                    df_add_f(d, run[q][k]);
                    sh[(q * V + k) * kBlock] = d;
                    run[q][k] = 0.f;
                }
            cnt = 0;
        }
    }
    // after each row (or group of rows) a lane has added
    __device__ __forceinline__ void row_done() {
        if constexpr (kFloat)
            if (++cnt == kSqChunk) flush();
    }
    // the thread's sums in acc, for grid_sum_cols
    __device__ __forceinline__ void finish() {
        if constexpr (kFloat) {
            flush();
#pragma unroll
            for (int q = 0; q < NQ; ++q)
#pragma unroll
                for (int k = 0; k < V; ++k) acc[q][k] = sh[(q * V + k) * kBlock];
        }
    }
};
template <typename T, int NQ, int V>
constexpr int sqsum_slots() {
    return std::is_same_v<T, float> ? NQ * V * kBlock : 1;
}

// (hi, lo) += alpha * p for the float path (product and sum errors kept in
// lo, renormalised); a plain FMA for FP64.
template <typename T>
__device__ __forceinline__ void axpy_hilo(T &xh, float &xl, T al, T po) {
    if constexpr (std::is_same_v<T, float>) {
        const float dlt = __fmul_rn(al, po);
        const float de = __fmaf_rn(al, po, -dlt);
        float sh, se;
        two_sum(xh, dlt, sh, se);
        const float lo = __fadd_rn(xl, __fadd_rn(se, de));
        const float h2 = __fadd_rn(sh, lo);
        xl = __fsub_rn(lo, __fsub_rn(h2, sh));
        xh = h2;
    } else {
        xh = fma(al, po, xh);
    }
}

__device__ __forceinline__ void set_cond(cudaGraphConditionalHandle h, int use, int value) {
    if (use) cudaGraphSetConditional(h, value ? 1u : 0u);
}

// Whether the replacement kernels of the loop body's iteration a.if_pos run
// (the value of its IF node; graph launches only).
template <typename T>
__device__ __forceinline__ void set_if(const PcgArgs<T> &a, int value) {
    if (a.use_cond && a.if_pos >= 0) cudaGraphSetConditional(a.ctl->ifh[a.if_pos], value ? 1u : 0u);
}

// The finishing steps below run on warp 0 of the last block (all 32 lanes):
// lane c handles column c (or segment c, strided), so the FP64 square roots
// and divisions of the columns run side by side instead of one after the
// other.  Values other blocks wrote in this launch are read with ld.cg (L2):
// the block's L1 may hold lines loaded at its start.
constexpr unsigned kFull = 0xffffffffu;

// Residual replacement (van der Vorst and Ye, "Residual replacement
// strategies for Krylov subspace iterative methods", 2000): the recurrence
// r -= alpha q drifts from b - A y by about eps |r_0| (FP32: 6e-8 |r_0|), so
// with a warm start (|r_0| >> |b|) it can report 1e-6 while b - A y is far
// larger.  Replacing r by b - A y keeps the iteration sound only while that
// drift is small against r: a replacement made after the drift has outgrown
// r makes beta huge, the new direction copies the old one and the iteration
// stalls.  So a column asks for a replacement once its recurrence residual
// has fallen kRefreshDrop below its value at the last one (the drift stays
// below ~eps / kRefreshDrop of r).  A column whose recurrence residual
// reaches tol stops (pending) and is confirmed on the next replacement's true
// residual -- one is made as soon as no column of any problem of a batch is
// left iterating, so the problems of a batch share it -- or, if that
// residual is still above tol, resumes with a restarted direction.  A
// replacement that moved r by more than sqrt(kRestartDev) of its norm
// restarts that column too (beta = 0).  Periodic replacements (every
// `refresh` iterations) come on top; refresh = 0 turns replacement off and
// freezes columns on the recurrence.
constexpr double kRefreshDrop = 1e-3;
constexpr double kRestartDev = 1e-2;

// Per-segment part of finishing iteration `it` (or the start of a solve):
// residual norms -> relres, beta, freezing, replacement requests.  MODE 0:
// the start of a solve (r = b - A y); 1: a replacement iteration (r = b - A y,
// sc.devr holds the replacement's relative deviation); 2: an ordinary
// iteration (recurrence residual).  Ends with a __syncwarp, so lane 0 sees
// every lane's writes.
static __device__ void finish_seg(PcgCtl *ctl, const SegScal &sc, int seg, const double *rz, const double *rr, int D,
                                  int mode, int it) {
    const int lane = threadIdx.x & 31;
    const bool replace = ctl->refresh > 0;
    int live = 0, iterating = 0, want = 0;
    for (int c = lane; c < D; c += 32) {
        const int k = seg * D + c;
        if (mode == 0) {
            sc.rz[k] = rz[c];
            sc.beta[k] = 0.0;
            const double rel = sqrt(rr[c]) / sc.bnorm[k];
            sc.relres[k] = rel;
            sc.rel_ref[k] = rel;
            if (!(rel == rel) || !(rz[c] == rz[c])) atomicMax(&ctl->error, (int)PFE_ENUMERIC);
            sc.active[k] = rel > ctl->tol;
            sc.pending[k] = 0;
        } else if (mode == 1 && (sc.active[k] || sc.pending[k])) {
            const double rel = sqrt(rr[c]) / sc.bnorm[k];
            const bool restart = sc.pending[k] || sc.devr[k] > kRestartDev;
            sc.beta[k] = restart ? 0.0 : rz[c] / sc.rz[k];
            sc.rz[k] = rz[c];
            sc.relres[k] = rel;
            sc.rel_ref[k] = rel;
            if (!(rel == rel) || !(rz[c] == rz[c])) atomicMax(&ctl->error, (int)PFE_ENUMERIC);
            sc.active[k] = rel > ctl->tol;
            sc.pending[k] = 0;
        } else if (mode == 2 && sc.active[k]) {
            const double rel = sqrt(rr[c]) / sc.bnorm[k];
            sc.beta[k] = rz[c] / sc.rz[k];
            sc.rz[k] = rz[c];
            sc.relres[k] = rel;
            if (!(rel == rel) || !(rz[c] == rz[c])) atomicMax(&ctl->error, (int)PFE_ENUMERIC);
            if (rel <= ctl->tol) {
                sc.active[k] = 0;
                sc.pending[k] = replace ? 1 : 0;
            } else if (replace && rel <= kRefreshDrop * sc.rel_ref[k]) {
                want = 1;
            }
        }
        live |= sc.active[k] | sc.pending[k];
        iterating |= sc.active[k];
    }
    live = __any_sync(kFull, live);
    iterating = __any_sync(kFull, iterating);
    want = __any_sync(kFull, want);
    if (lane == 0) {
        if (mode == 0)
            sc.seg_iters[seg] = 0;
        else if (__ldcg(sc.seg_live + seg))
            sc.seg_iters[seg] = it;
        sc.seg_active[seg] = iterating;  // the iteration kernels skip segments with no column iterating
        sc.seg_live[seg] = live;         // the replacement kernels also visit waiting ones
        if (want && mode == 2) ctl->refresh_want = 1;
    }
    __syncwarp();
}

// Lane 0 of warp 0 of a segment's last block, after its segment's work: true
// for the last segment to get here (the one that finishes the iteration).
__device__ __forceinline__ bool last_segment_arrives(PcgCtl *ctl, int k, int nseg) {
    __threadfence();
    const unsigned t = atomicAdd(&ctl->ticket[k], 1u);
    if (t != (unsigned)nseg - 1) return false;
    __threadfence();
    ctl->ticket[k] = 0u;
    return true;
}

// The same decision for the whole warp (lane 0 takes the ticket).
__device__ __forceinline__ bool warp_last_segment(PcgCtl *ctl, int k, int nseg) {
    int last = 0;
    if ((threadIdx.x & 31) == 0) last = last_segment_arrives(ctl, k, nseg);
    last = __shfl_sync(kFull, last, 0);
    __syncwarp();
    return last != 0;
}

template <typename V>
__device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Global part (warp 0, all lanes; the control block is written by lane 0):
// termination (every segment converged, an error, or max_iter) and the
// statistics of a finished solve.
static __device__ void finish_all(PcgCtl *ctl, const SegScal &sc, int nseg, int D, cudaGraphConditionalHandle cond,
                                  int use_cond) {
    const int lane = threadIdx.x & 31;
    int any = 0, iterating = 0;
    for (int s = lane; s < nseg; s += 32) {
        any |= __ldcg(sc.seg_live + s);
        iterating |= __ldcg(sc.seg_active + s);
    }
    any = __any_sync(kFull, any);
    iterating = __any_sync(kFull, iterating);
    int done = 0;
    if (lane == 0) done = (!any) || *(volatile int *)&ctl->error || ctl->iter >= ctl->max_iter;
    done = __shfl_sync(kFull, done, 0);
    // only columns waiting for confirmation left: the next iteration replaces
    if (lane == 0 && !done && !iterating && ctl->refresh > 0) ctl->refresh_want = 1;
    if (done) {
        double mr = 0.0;
        long long tot = 0;
        int mx = 0, nun = 0;
        for (int s = lane; s < nseg; s += 32) {
            const int it = __ldcg(sc.seg_iters + s);
            tot += it;
            sc.seg_iters_tot[s] += it;
            mx = max(mx, it);
            nun += __ldcg(sc.seg_live + s) ? 1 : 0;
            for (int c = 0; c < D; ++c) mr = fmax(mr, __ldcg(sc.relres + (int64_t)s * D + c));
        }
        tot = warp_sum(tot);
        nun = warp_sum(nun);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mx = max(mx, __shfl_xor_sync(kFull, mx, o));
            mr = fmax(mr, __shfl_xor_sync(kFull, mr, o));
        }
        if (lane == 0) {
            ctl->tot_iters += tot;
            ctl->tot_rounds += ctl->iter;
            ctl->tot_refreshes += ctl->refreshes;
            ctl->max_solve_iters = max(ctl->max_solve_iters, mx);
            ctl->n_solves += nseg;
            ctl->n_unconv += nun;
            ctl->last_iters = mx;
            ctl->last_relres = mr;
            ctl->last_converged = !any;
            ctl->max_relres = fmax(ctl->max_relres, mr);
            const int u = ctl->unroll > 0 ? ctl->unroll : 1;
            // launches before and after the loop + the loop body's per
            // iteration; the replacement kernels run on replacement iterations
            // only when they sit in IF nodes, else every iteration
            const long long body_iters = (long long)u * ((ctl->iter + u - 1) / u);
            const bool by_if = use_cond && ctl->n_if > 0;
            ctl->launches += ctl->launch_base + (long long)ctl->launch_per_iter * body_iters +
                             (long long)ctl->launch_cond * (by_if ? (long long)ctl->refreshes : body_iters);
        }
        // the rest of the body's IF nodes stay closed
        if (use_cond)
            for (int k = lane; k < ctl->n_if; k += 32) cudaGraphSetConditional(ctl->ifh[k], 0u);
    }
    if (lane == 0) {
        ctl->done = done;
        set_cond(cond, use_cond, !done);
    }
    __syncwarp();
}

// acc += a * (xh + xl) with a = ah + al: the exact product ah * xh plus the
// cross terms (al * xl is below the pair's precision).
__device__ __forceinline__ void df_add_prod2(DF &acc, float ah, float al, float xh, float xl) {
    df_add_prod(acc, ah, xh);
    df_add_f(acc, __fmaf_rn(al, xh, __fmul_rn(ah, xl)));
}

// (b - A y) on columns c0 .. c0+V-1 of row i.  Float path: y = hi + lo and
// A's FP64 values as FP32 pairs (aoff + aofflo, set when the graph is
// built), accumulated in double-FP32, so the replaced residual is that of the
// FP64 system matrix (not of the FP32 rounding the iteration's q = A p uses)
// to about 2^-44 of |A||y|.  FP64 path: plain FP64.  LEN > 0: uniform rows
// of LEN slots (row i's at i * LEN), loaded as vectors.
template <typename T, int D, int V, int LEN = 0, bool GRID = false>
__device__ __forceinline__ void true_residual(const PcgArgs<T> &a, int64_t i, int c0, T (&out)[V]) {
    T bi[V];
    ldv_rw<T, V>(a.b + i * D + c0, bi);
    if constexpr (std::is_same_v<T, float>) {
        DF acc[V];
        float xh[V], xl[V];
        const float ah = a.A.adiag[i], al = a.A.adiaglo[i];
        ldv_rw<float, V>(a.x + i * D + c0, xh);
        ldv_rw<float, V>(a.xlo + i * D + c0, xl);
#pragma unroll
        for (int k = 0; k < V; ++k) {
            acc[k] = DF{0.f, 0.f};
            df_add_prod2(acc[k], ah, al, xh[k], xl[k]);
        }
        if constexpr (LEN > 0) {
            static_assert(LEN % 4 == 0, "fixed rows hold a multiple of 4 slots");
            const int4 *c4 = reinterpret_cast<const int4 *>(a.A.col + i * LEN);
            const float4 *h4 = reinterpret_cast<const float4 *>(a.A.aoff + i * LEN);
            const float4 *l4 = reinterpret_cast<const float4 *>(a.A.aofflo + i * LEN);
            int jall[GRID ? LEN : 1];  // GRID: every slot's column from the stencil (one grid image)
            if constexpr (GRID) stencil_cols<LEN, 0>((int)i, a.grid_w, (int)a.A.n, jall);
#pragma unroll
            for (int q = 0; q < LEN / 4; ++q) {
                int4 jc;
                if constexpr (GRID)
                    jc = make_int4(jall[4 * q], jall[4 * q + 1], jall[4 * q + 2], jall[4 * q + 3]);
                else
                    jc = __ldg(c4 + q);
                const float4 vh = __ldg(h4 + q), vl = __ldg(l4 + q);
                const int jj[4] = {jc.x, jc.y, jc.z, jc.w};
                const float sh[4] = {vh.x, vh.y, vh.z, vh.w}, sl[4] = {vl.x, vl.y, vl.z, vl.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    ldv_rw<float, V>(a.x + (int64_t)jj[u] * D + c0, xh);
                    ldv_rw<float, V>(a.xlo + (int64_t)jj[u] * D + c0, xl);
#pragma unroll
                    for (int k = 0; k < V; ++k) df_add_prod2(acc[k], sh[u], sl[u], xh[k], xl[k]);
                }
            }
        } else {
            int64_t base;
            int len;
            sell_row(a.A.slice_ptr, a.A.row_len, i, base, len);
            for (int s = 0; s < len; ++s) {
                const int64_t idx = base + s;
                const int j = a.A.col[idx];
                ldv_rw<float, V>(a.x + (int64_t)j * D + c0, xh);
                ldv_rw<float, V>(a.xlo + (int64_t)j * D + c0, xl);
#pragma unroll
                for (int k = 0; k < V; ++k) df_add_prod2(acc[k], a.A.aoff[idx], a.A.aofflo[idx], xh[k], xl[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < V; ++k) {
            float sh, se;
            two_sum(bi[k], -acc[k].hi, sh, se);
            out[k] = __fadd_rn(sh, __fsub_rn(se, acc[k].lo));
        }
    } else {
        int64_t base;
        int len;
        sell_row(a.A.slice_ptr, a.A.row_len, i, base, len);
        double acc[V], xv[V];
        const double ad = a.A.adiag[i];
        ldv_rw<double, V>(a.x + i * D + c0, xv);
#pragma unroll
        for (int k = 0; k < V; ++k) acc[k] = ad * xv[k];
        for (int s = 0; s < len; ++s) {
            const int64_t idx = base + s;
            const double av = a.A.aoff[idx];
            ldv_rw<double, V>(a.x + (int64_t)a.A.col[idx] * D + c0, xv);
#pragma unroll
            for (int k = 0; k < V; ++k) acc[k] = fma(av, xv[k], acc[k]);
        }
#pragma unroll
        for (int k = 0; k < V; ++k) out[k] = bi[k] - acc[k];
    }
}

// Row loop of a row kernel: the block's segment (block_seg), its warps
// stride over the segment's row groups.  LIVE skips segments whose columns
// have all converged.  Inside, PFE_ROW_I defines row i (skips lanes past the
// segment).
#define PFE_ROW_LOOP_(T_, D_, LIVE_, MS_)                                                                  \
    using SW = SubWarp<T_, D_>;                                                                            \
    constexpr int V = SW::V;                                                                               \
    const SW lm;                                                                                           \
    const BlockSeg bsg = block_seg<MS_>(a.sg);                                                             \
    const int64_t warp_g = (int64_t)(blockIdx.x - bsg.b0) * kWarps + (threadIdx.x >> 5);                   \
    const int64_t warps_total = (int64_t)bsg.nb * kWarps;                                                  \
    const int64_t seg_rows = ((MS_) && (LIVE_) && !__ldcg(((LIVE_) == 2 ? a.sc.seg_live : a.sc.seg_active) + bsg.seg)) \
                                 ? 0                                                                                 \
                                 : bsg.r1 - bsg.r0;                                                                  \
    for (int64_t g = warp_g; g * SW::RPW < seg_rows; g += warps_total)
// one problem (FSAI kernels, y = A x)
#define PFE_ROW_LOOP(T_, D_) PFE_ROW_LOOP_(T_, D_, false, false)
// MS: batch (segments) or one problem; LIVE skips converged segments
#define PFE_ROW_LOOP_MS(T_, D_, MS_) PFE_ROW_LOOP_(T_, D_, false, MS_)
#define PFE_ROW_LOOP_LIVE(T_, D_, MS_) PFE_ROW_LOOP_(T_, D_, 1, MS_)
// MS: batch, skipping segments with no column iterating or waiting to be confirmed
#define PFE_ROW_LOOP_REPL(T_, D_, MS_) PFE_ROW_LOOP_(T_, D_, 2, MS_)
#define PFE_ROW_I                                 \
    const int64_t i = bsg.r0 + g * SW::RPW + lm.r; \
    if (!lm.active || i >= bsg.r1) continue

// ---- kernels ----------------------------------------------------------------

// Start of a solve: r = b - A y, norms of b and r, r.z with z = D_A^{-1} r.
// With the FSAI preconditioner (PRE = 1) k_fsai_t makes t = G r and r.z =
// t.t and finishes the start of the solve; k_fsai_zp then sets p = G^T t.
template <typename T, int D, int PRE, bool MS>
__global__ void __launch_bounds__(kBlock) k_pcg_init(PcgArgs<T> a) {
    using A = Acc<T>;
    using AT = typename A::type;
    using SWt = SubWarp<T, D>;
    AT acc[3][SWt::V];  // r.z | r.r | b.b
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int k = 0; k < SWt::V; ++k) acc[q][k] = A::zero();
    PFE_ROW_LOOP_MS(T, D, MS) {
        PFE_ROW_I;
        const int c0 = lm.cg * V;
        T ri[V], bi[V];
        true_residual<T, D, V>(a, i, c0, ri);
        ldv_rw<T, V>(a.b + i * D + c0, bi);
        const T dv = a.A.dinv[i];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const T zi = dv * ri[k];
            A::add_prod(acc[0][k], ri[k], zi);
            A::add_prod(acc[1][k], ri[k], ri[k]);
            A::add_prod(acc[2][k], bi[k], bi[k]);
        }
        stv<T, V>(a.r + i * D + c0, ri);
    }
    // ctl->error was cleared before this launch (segment finishers may set it)
    __shared__ double tot[3 * D];
    if (grid_sum_cols<T, D, 3>(acc, a.part, bsg, &a.sc.ticket[bsg.seg * 4 + 2], tot)) {
        if (threadIdx.x < 32) {
            PcgCtl *ctl = a.ctl;
            const int seg = bsg.seg;
            for (int c = threadIdx.x; c < D; c += 32) {
                double bn = sqrt(tot[2 * D + c]);
                a.sc.bnorm[seg * D + c] = bn > 0.0 ? bn : 1.0;
                a.sc.alpha[seg * D + c] = 0.0;
            }
            __syncwarp();
            if (PRE == 0) finish_seg(ctl, a.sc, seg, tot, tot + D, D, 0, 0);
            if (!MS || warp_last_segment(ctl, 2, a.sg.nseg)) {
                if (threadIdx.x == 0) {
                    ctl->iter = 0;
                    ctl->refresh_now = 0;
                    ctl->p_ready = 1;
                    ctl->xpending = 0;
                    ctl->xheld = 0;
                    ctl->xfold = 0;
                    ctl->refresh_want = 0;
                    ctl->refresh_next = 0;
                    ctl->refreshes = 0;
                    ctl->rounds = 0;
                    if (PRE != 0) ctl->done = 0;  // k_fsai_t finishes the start
                }
                __syncwarp();
                if (PRE == 0) finish_all(ctl, a.sc, a.sg.nseg, D, a.cond, a.use_cond);
            }
        }
    }
}

// float4 / double2 views of flat arrays
template <typename T>
struct Vec;
template <>
struct Vec<float> {
    static constexpr int N = 4;
    using V = float4;
    __device__ static __forceinline__ void get(const V &v, float (&o)[4]) {
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
    __device__ static __forceinline__ V make(const float (&o)[4]) { return make_float4(o[0], o[1], o[2], o[3]); }
};
template <>
struct Vec<double> {
    static constexpr int N = 2;
    using V = double2;
    __device__ static __forceinline__ void get(const V &v, double (&o)[2]) {
        o[0] = v.x; o[1] = v.y;
    }
    __device__ static __forceinline__ V make(const double (&o)[2]) { return make_double2(o[0], o[1]); }
};

// p_new = z + beta p (p = z right after k_pcg_init) with the Jacobi z =
// D_A^{-1} r, into the other direction buffer, and on folding iterations the
// two delayed solution updates y += alpha_prev p_prev + alpha p (p_prev is
// the old content of the buffer p_new goes to; every other iteration holds
// its update, so y is read and written every other iteration).  Elementwise
// (flat float4 / double2 traversal; the grid makes every thread meet fixed
// columns).  (The FSAI iteration makes this update in k_fsai_zp.)
template <typename T, int D, bool MS>
__global__ void __launch_bounds__(kBlock) k_pupdate(PcgArgs<T> a) {
    const PcgCtl *ctl = a.ctl;
    if (*(volatile const int *)&ctl->done) return;
    const int p_ready = ctl->p_ready, fold = ctl->xpending && ctl->xfold;
    // p of the previous iteration in buffer (iter & 1) ^ 1 (its finisher has
    // counted it), the new one into iter & 1
    T *__restrict__ pdst = a.p[ctl->iter & 1];
    const T *__restrict__ psrc = a.p[(ctl->iter & 1) ^ 1];
    constexpr bool multi = MS;  // batch: beta, alpha of each row's segment
    __shared__ T sbeta[D], salpha[D], salpha_prev[D];
    if (threadIdx.x < D) {
        sbeta[threadIdx.x] = p_ready ? T(0) : (T)a.sc.beta[threadIdx.x];
        salpha[threadIdx.x] = (T)a.sc.alpha[threadIdx.x];
        salpha_prev[threadIdx.x] = (T)a.sc.alpha_prev[threadIdx.x];
    }
    __syncthreads();
    using VT = Vec<T>;
    constexpr int VN = VT::N;
    const int64_t nel = a.A.n * D, nvec = nel / VN;
    const int64_t tid = (int64_t)blockIdx.x * kBlock + threadIdx.x, nthr = (int64_t)gridDim.x * kBlock;
    T be[VN], al[VN], ap[VN];
    int cu[VN];
#pragma unroll
    for (int u = 0; u < VN; ++u) {
        const int c = (int)((tid * VN + u) % D);
        cu[u] = c;
        be[u] = sbeta[c];
        al[u] = salpha[c];
        ap[u] = salpha_prev[c];
    }
    using V4 = typename VT::V;
    V4 *p4 = reinterpret_cast<V4 *>(pdst);
    const V4 *ps4 = reinterpret_cast<const V4 *>(psrc);
    const V4 *z4 = reinterpret_cast<const V4 *>(a.r);
    V4 *x4 = reinterpret_cast<V4 *>(a.x);
    float4 *xl4 = reinterpret_cast<float4 *>(a.xlo);  // float path: VN == 4
    for (int64_t v = tid; v < nvec; v += nthr) {
        T pv[VN], zv[VN];
        if constexpr (multi) {
            // element u of this vector is column cu[u] of row v*VN/D + (cu[0] + u)/D
            const int64_t row0 = v * VN / D;
#pragma unroll
            for (int u = 0; u < VN; ++u) {
                const int sgm = __ldg(a.sg.rseg + row0 + (cu[0] + u) / D);
                be[u] = p_ready ? T(0) : (T)a.sc.beta[sgm * D + cu[u]];
                al[u] = (T)a.sc.alpha[sgm * D + cu[u]];
                ap[u] = (T)a.sc.alpha_prev[sgm * D + cu[u]];
            }
        }
        VT::get(ps4[v], pv);
        VT::get(z4[v], zv);
#pragma unroll
        for (int u = 0; u < VN; ++u) zv[u] = a.A.dinv[(v * VN + u) / D] * zv[u];
        if (fold) {
            T xv[VN], pp[VN];
            float xl[VN];
            VT::get(p4[v], pp);
            VT::get(x4[v], xv);
            if constexpr (std::is_same_v<T, float>) {
                const float4 t = xl4[v];
                xl[0] = t.x; xl[1] = t.y; xl[2] = t.z; xl[3] = t.w;
            }
#pragma unroll
            for (int u = 0; u < VN; ++u) {
                axpy_hilo<T>(xv[u], xl[u], ap[u], pp[u]);
                axpy_hilo<T>(xv[u], xl[u], al[u], pv[u]);
            }
            x4[v] = VT::make(xv);
            if constexpr (std::is_same_v<T, float>) xl4[v] = make_float4(xl[0], xl[1], xl[2], xl[3]);
        }
#pragma unroll
        for (int u = 0; u < VN; ++u) pv[u] = p_ready ? zv[u] : zv[u] + be[u] * pv[u];
        p4[v] = VT::make(pv);
    }
    if (tid < nel - nvec * VN) {  // tail elements
        const int64_t e = nvec * VN + tid;
        const int c = (int)(e % D);
        const int sgm = multi ? row_seg(a.sg, e / D) : 0;
        const T bt = p_ready ? T(0) : (multi ? (T)a.sc.beta[sgm * D + c] : sbeta[c]);
        const T at = multi ? (T)a.sc.alpha[sgm * D + c] : salpha[c];
        const T apv = multi ? (T)a.sc.alpha_prev[sgm * D + c] : salpha_prev[c];
        const T z = a.A.dinv[e / D] * a.r[e];
        const T po = psrc[e];
        if (fold) {
            T xh = a.x[e];
            float xl = 0.f;
            if constexpr (std::is_same_v<T, float>) xl = a.xlo[e];
            axpy_hilo<T>(xh, xl, apv, pdst[e]);
            axpy_hilo<T>(xh, xl, at, po);
            a.x[e] = xh;
            if constexpr (std::is_same_v<T, float>) a.xlo[e] = xl;
        }
        pdst[e] = p_ready ? z : z + bt * po;
    }
}

// Last block of a segment: alpha_c = r.z / p.q per column of the segment
// (0 for frozen columns; a non-positive or non-finite p.q is PFE_ENUMERIC).
template <typename T, int D, bool MS>
__device__ __forceinline__ void spmm_finish(const PcgArgs<T> &a, const BlockSeg &bsg, const double *tot) {
    PcgCtl *w = a.ctl;
    const SegScal &sc = a.sc;
    for (int c = threadIdx.x & 31; c < D; c += 32) {
        const int k = bsg.seg * D + c;
        if (!sc.active[k]) {
            sc.alpha[k] = 0.0;
            continue;
        }
        const double pqc = tot[c];
        if (!(pqc > 0.0) || !(pqc < INFINITY)) {
            atomicMax(&w->error, (int)PFE_ENUMERIC);
            sc.alpha[k] = 0.0;
        } else {
            sc.alpha[k] = sc.rz[k] / pqc;
        }
    }
    if ((!MS || warp_last_segment(w, 0, a.sg.nseg)) && (threadIdx.x & 31) == 0) {
        w->p_ready = 0;
        w->xpending = 1;
        // a loop whose iterations stopped advancing (no finisher ran) ends
        // here with PFE_ETIMEOUT instead of running on
        if (++w->rounds > w->max_iter + 2 * kPcgMaxIf + 8) {
            atomicMax(&w->error, (int)PFE_ETIMEOUT);
            w->done = 1;
            set_cond(a.cond, a.use_cond, 0);
            if (a.use_cond)
                for (int k = 0; k < w->n_if; ++k) cudaGraphSetConditional(w->ifh[k], 0u);
        }
    }
}

// q = A p and the column dots p.q -> alpha.  Only p is gathered; the matrix
// slots of a row are fetched kChunk at a time ahead of the gathers.
template <typename T, int D, bool MS>
__global__ void __launch_bounds__(kBlock) k_spmm(PcgArgs<T> a) {
    const PcgCtl *ctl = a.ctl;
    if (*(volatile const int *)&ctl->done) return;
    using A = Acc<T>;
    using AT = typename A::type;
    using SWt = SubWarp<T, D>;
    const T *__restrict__ pp = a.p[ctl->iter & 1];  // FSAI alternates the buffers
    AT pq[1][SWt::V];
#pragma unroll
    for (int k = 0; k < SWt::V; ++k) pq[0][k] = A::zero();
    PFE_ROW_LOOP_LIVE(T, D, MS) {
        PFE_ROW_I;
        const int c0 = lm.cg * V;
        const int64_t ic = i * D + c0;
        int64_t base;
        int len;
        sell_row(a.A.slice_ptr, a.A.row_len, i, base, len);
        T pi[V], acc[V];
        ldv<T, V>(pp + ic, pi);
        const T ad = a.A.adiag[i];
#pragma unroll
        for (int k = 0; k < V; ++k) acc[k] = ad * pi[k];
        for (int k0 = 0; k0 < len; k0 += kChunk) {
            int jj[kChunk];
            T av[kChunk], pj[kChunk][V];
            load_slots<T, kChunk>(a.A.col, a.A.aoff, base, k0, len, (int)i, jj, av);
#pragma unroll
            for (int u = 0; u < kChunk; ++u) ldv<T, V>(pp + (int64_t)jj[u] * D + c0, pj[u]);
#pragma unroll
            for (int u = 0; u < kChunk; ++u)
#pragma unroll
                for (int k = 0; k < V; ++k) acc[k] = fma(av[u], pj[u][k], acc[k]);
        }
        stv<T, V>(a.q + ic, acc);
#pragma unroll
        for (int k = 0; k < V; ++k) A::add_prod(pq[0][k], pi[k], acc[k]);
    }
    __shared__ double tot[D];
    if (grid_sum_cols<T, D, 1>(pq, a.part, bsg, &a.sc.ticket[bsg.seg * 4 + 0], tot))
        if (threadIdx.x < 32) spmm_finish<T, D, MS>(a, bsg, tot);
}

// k_spmm for graphs whose rows all have LEN slots (grid stencils; LEN a
// compile-time constant): the slot loads of ROWS row groups are issued
// together, then their gathers; at least MINB blocks per SM.  GRID (one grid
// image): only the slot values are loaded, the columns are computed from the
// stencil (the same products in the same order).
template <typename T, int D, bool MS, int LEN, int ROWS, int MINB, bool GRID = false>
__global__ void __launch_bounds__(kBlock, MINB) k_spmm_fixed(PcgArgs<T> a) {
    const PcgCtl *ctl = a.ctl;
    if (*(volatile const int *)&ctl->done) return;
    using A = Acc<T>;
    using AT = typename A::type;
    using SW = SubWarp<T, D>;
    constexpr int V = SW::V;
    static_assert(LEN % 4 == 0, "rows are read 4 slots at a time");
    const T *__restrict__ pp = a.p[ctl->iter & 1];  // FSAI alternates the buffers
    AT pq[1][V];
#pragma unroll
    for (int k = 0; k < V; ++k) pq[0][k] = A::zero();
    const SW lm;
    const BlockSeg bsg = block_seg<MS>(a.sg);
    const int64_t warp_g = (int64_t)(blockIdx.x - bsg.b0) * kWarps + (threadIdx.x >> 5);
    const int64_t warps_total = (int64_t)bsg.nb * kWarps;
    const int64_t seg_rows = (MS && !__ldcg(a.sc.seg_active + bsg.seg)) ? 0 : bsg.r1 - bsg.r0;
    const int c0 = lm.cg * V;
    for (int64_t g = warp_g; g * SW::RPW < seg_rows; g += ROWS * warps_total) {
        int64_t ii[ROWS];
        bool ok[ROWS];
        int jj[ROWS][LEN];
        T av[ROWS][LEN];
#pragma unroll
        for (int h = 0; h < ROWS; ++h) {
            ii[h] = bsg.r0 + (g + h * warps_total) * SW::RPW + lm.r;
            ok[h] = lm.active && ii[h] < bsg.r1;
            const int64_t base = (ok[h] ? ii[h] : bsg.r0) * LEN;  // a valid row when idle
            if constexpr (GRID) {
                static_assert(!MS, "computed columns: one image");
                load_val_range<T, 0, LEN>(a.A.aoff, base, av[h]);
                stencil_cols<LEN, 0>((int)(ok[h] ? ii[h] : bsg.r0), a.grid_w, (int)a.A.n, jj[h]);
            } else {
                load_slots<T, LEN>(a.A.col, a.A.aoff, base, 0, LEN, (int)ii[h], jj[h], av[h]);
            }
        }
#pragma unroll
        for (int h = 0; h < ROWS; ++h) {
            if (!ok[h]) continue;
            const int64_t ic = ii[h] * D + c0;
            T pi[V], acc[V], pj[LEN][V];
            ldv<T, V>(pp + ic, pi);
            const T ad = a.A.adiag[ii[h]];
#pragma unroll
            for (int k = 0; k < V; ++k) acc[k] = ad * pi[k];
#pragma unroll
            for (int u = 0; u < LEN; ++u) ldv<T, V>(pp + (int64_t)jj[h][u] * D + c0, pj[u]);
#pragma unroll
            for (int u = 0; u < LEN; ++u)
#pragma unroll
                for (int k = 0; k < V; ++k) acc[k] = fma(av[h][u], pj[u][k], acc[k]);
            stv<T, V>(a.q + ic, acc);
#pragma unroll
            for (int k = 0; k < V; ++k) A::add_prod(pq[0][k], pi[k], acc[k]);
        }
    }
    __shared__ double tot[D];
    if (grid_sum_cols<T, D, 1>(pq, a.part, bsg, &a.sc.ticket[bsg.seg * 4 + 0], tot))
        if (threadIdx.x < 32) spmm_finish<T, D, MS>(a, bsg, tot);
}

// k_spmm for fixed-length rows with the matrix slots staged in shared
// memory by bulk asynchronous copies.  The block walks tiles of TR rows (its
// tiles t, t + gridDim.x, ...); S tiles are requested ahead, so every SM
// keeps S x (its blocks) x TR x LEN x 8 bytes of the slot stream in flight
// while its warps gather p, and a warp's row no longer waits for its slot
// loads before it can gather.  One barrier per tile (it also releases the
// previous tile's stage for refilling).  One problem (no segments).
template <typename T, int D, int LEN, int S>
struct SpmmTma {
    // rows per tile (one pass of the block's warps at d = 10; any d works,
    // some warps idle where a pass holds more rows).  Small tiles leave most
    // of the SM's unified L1/shared memory to L1, which the gathers of p hit.
    static constexpr int TR = 48;
    static constexpr int STAGE = 2 * TR * LEN * 4;  // bytes: columns, then values
    static constexpr int SMEM = S * STAGE;
};

template <typename T, int D, int LEN, int S, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_spmm_tma(PcgArgs<T> a) {
    static_assert(sizeof(T) == 4 && LEN % 4 == 0, "FP32 rows of a multiple of 4 slots (16-byte copies)");
    using P = SpmmTma<T, D, LEN, S>;
    const PcgCtl *ctl = a.ctl;
    if (*(volatile const int *)&ctl->done) return;
    extern __shared__ __align__(16) unsigned char smem_tiles[];
    __shared__ __align__(8) uint64_t bars[S];
    using A = Acc<T>;
    using AT = typename A::type;
    using SW = SubWarp<T, D>;
    constexpr int V = SW::V;
    const T *__restrict__ pp = a.p[ctl->iter & 1];  // FSAI alternates the buffers
    AT pq[1][V];
#pragma unroll
    for (int k = 0; k < V; ++k) pq[0][k] = A::zero();
    const SW lm;
    const BlockSeg bsg = block_seg<false>(a.sg);
    const int64_t n = bsg.r1 - bsg.r0;
    const int64_t ntiles = (n + P::TR - 1) / P::TR;
    const int64_t nmine = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int warp = threadIdx.x >> 5;
    const int c0 = lm.cg * V;
    if (threadIdx.x == 0) {
        for (int q = 0; q < S; ++q) mbar_init(&bars[q], 1);
        mbar_init_fence();
    }
    __syncthreads();
    // thread 0: request this block's tile k into stage k % S (sizes and
    // offsets are multiples of LEN * 4 bytes, a multiple of 16)
    auto issue = [&](int64_t k) {
        const int64_t r0 = bsg.r0 + ((int64_t)blockIdx.x + k * gridDim.x) * P::TR;
        const uint32_t bytes = (uint32_t)(min((int64_t)P::TR, bsg.r1 - r0) * LEN * 4);
        unsigned char *st = smem_tiles + (int)(k % S) * P::STAGE;
        uint64_t *bar = &bars[k % S];
        mbar_arrive_expect_tx(bar, 2 * bytes);
        bulk_copy_g2s(st, a.A.col + r0 * LEN, bytes, bar);
        bulk_copy_g2s(st + P::STAGE / 2, a.A.aoff + r0 * LEN, bytes, bar);
    };
    if (threadIdx.x == 0)
        for (int64_t k = 0; k < S && k < nmine; ++k) issue(k);
    int64_t k = 0;
    bool failed = false;
    for (; k < nmine; ++k) {
        const int st = (int)(k % S);
        const bool got = mbar_wait(&bars[st], (uint32_t)((k / S) & 1));
        // every thread's wait result; every thread is also done with tile
        // k - 1, whose stage is refilled
        if (__syncthreads_or(!got)) {
            failed = true;
            break;
        }
        if (threadIdx.x == 0 && k >= 1 && k - 1 + S < nmine) issue(k - 1 + S);
        const int64_t r0 = bsg.r0 + ((int64_t)blockIdx.x + k * gridDim.x) * P::TR;
        const int rows = (int)min((int64_t)P::TR, bsg.r1 - r0);
        const int *__restrict__ cs = reinterpret_cast<const int *>(smem_tiles + st * P::STAGE);
        const T *__restrict__ vs = reinterpret_cast<const T *>(smem_tiles + st * P::STAGE + P::STAGE / 2);
        for (int g = warp; g * SW::RPW < rows; g += kWarps) {
            const int il = g * SW::RPW + lm.r;
            if (!lm.active || il >= rows) continue;
            const int64_t i = r0 + il;
            int jj[LEN];
            T av[LEN];
#pragma unroll
            for (int g4 = 0; g4 < LEN / 4; ++g4) {
                const int4 cv = *reinterpret_cast<const int4 *>(cs + il * LEN + 4 * g4);
                const float4 vv = *reinterpret_cast<const float4 *>(vs + il * LEN + 4 * g4);
                jj[4 * g4] = cv.x; jj[4 * g4 + 1] = cv.y; jj[4 * g4 + 2] = cv.z; jj[4 * g4 + 3] = cv.w;
                av[4 * g4] = vv.x; av[4 * g4 + 1] = vv.y; av[4 * g4 + 2] = vv.z; av[4 * g4 + 3] = vv.w;
            }
            const int64_t ic = i * D + c0;
            T pi[V], acc[V], pj[LEN][V];
            ldv<T, V>(pp + ic, pi);
            const T ad = a.A.adiag[i];
#pragma unroll
            for (int q = 0; q < V; ++q) acc[q] = ad * pi[q];
#pragma unroll
            for (int u = 0; u < LEN; ++u) ldv<T, V>(pp + (int64_t)jj[u] * D + c0, pj[u]);
#pragma unroll
            for (int u = 0; u < LEN; ++u)
#pragma unroll
                for (int q = 0; q < V; ++q) acc[q] = fma(av[u], pj[u][q], acc[q]);
            stv<T, V>(a.q + ic, acc);
#pragma unroll
            for (int q = 0; q < V; ++q) A::add_prod(pq[0][q], pi[q], acc[q]);
        }
    }
    if (failed) {
        // report, then let the copies this block requested land before it
        // leaves (each wait bounded); the partials still go to the reduction
        if (threadIdx.x == 0) atomicMax(&a.ctl->error, (int)PFE_ETIMEOUT);
        const int64_t refills = max((int64_t)0, min(k - 1, nmine - (int64_t)S));
        const int64_t issued = min(nmine, (int64_t)S) + refills;
        for (int64_t j = k; j < issued; ++j) mbar_wait(&bars[j % S], (uint32_t)((j / S) & 1));
    }
    __shared__ double tot[D];
    if (grid_sum_cols<T, D, 1>(pq, a.part, bsg, &a.sc.ticket[bsg.seg * 4 + 0], tot))
        if (threadIdx.x < 32) spmm_finish<T, D, false>(a, bsg, tot);
}

__device__ __forceinline__ void cp_async_8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait_newest() {  // all but the N newest groups have landed
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Layout of the stencil pipeline of a one-image grid graph of width W: the
// image is cut into vertical strips of TS pixels (the last one narrower) and
// each strip into chunks of image rows; a block walks a chunk top to bottom,
// one image row (a step: up to TS pixels, one pass of its warps) at a time.
// A ring of NSLOT = 2R + 1 + P bands holds image rows y - R .. y + R of the
// vector, each band the strip's pixels plus R (and PADL, for alignment) on
// the left and R (plus rounding) on the right; the next P steps' bands, matrix
// values and diagonals are in flight as bulk asynchronous (TMA) copies that
// one thread requests, completing on one mbarrier per step (P + 1 of them,
// reused).  Every vector element and matrix value is copied from memory once
// per chunk (plus halo rows and columns) and every stencil neighbour is read
// from shared memory at a compile-time offset.
// Needs W * D, W, TS and TS * D multiples of 4 (16-byte aligned copies).
template <typename T, int D, int LEN, int P>
struct StencilPipe {
    static constexpr int R = Stencil<LEN>::R;
    static constexpr int NSLOT = 2 * R + 1 + P, NBAR = P + 1;
    static constexpr int RPW = SubWarp<T, D>::RPW;
    // pixels per 16 bytes of a row of D floats
    static constexpr int Q = D % 4 == 0 ? 1 : (D % 2 == 0 ? 2 : 4);
    // left pad so a band starts on a 16-byte boundary: ((R + PADL) D) % 4 == 0
    static constexpr int PADL = (R % Q == 0) ? 0 : Q - R % Q;
    static constexpr int brows(int ts) { return (ts + 2 * R + PADL + Q - 1 + Q - 1) / Q * Q; }
    static constexpr int TS = stencil_strip(D, LEN, P);  // 0: no aligned layout fits
    static constexpr int BROWS = brows(TS);
    static constexpr int SMEM = 4 * (NSLOT * BROWS * D + NBAR * TS * LEN + NBAR * TS);
    static constexpr bool kAligned = TS > 0 && TS % 4 == 0 && (TS * D) % 4 == 0;
};

// k_spmm for a one-image grid graph in the stencil form: q_i = A_ii p_i +
// sum over the slots t of A_i,t p(i + dy_t W + dx_t), every neighbour read
// from the band ring (the column array is not read: the neighbour of slot t
// is a compile-time offset in its band, and padding slots have A_i,t = 0,
// with pixels outside the image zero-filled).  Summation in slot order: the
// same results as k_spmm_fixed.  nchunk: chunks per strip (the host makes
// strips x chunks <= the grid).  A wait that runs out sets PFE_ETIMEOUT,
// lets the copies already requested land (bounded) and skips the rest.
template <typename T, int D, int LEN, int P, int MINB>
__global__ void __launch_bounds__(kBlock, MINB) k_spmm_stencil(PcgArgs<T> a, int nchunk) {
    static_assert(sizeof(T) == 4 && LEN % 4 == 0 && stencil_count<LEN>() == LEN, "FP32 stencil rows");
    using SP = StencilPipe<T, D, LEN, P>;
    static_assert(SP::kAligned, "strip width");
    constexpr int R = SP::R, TS = SP::TS, NSLOT = SP::NSLOT, NBAR = SP::NBAR, BROWS = SP::BROWS;
    constexpr int PADL = SP::PADL, Q = SP::Q;
    constexpr Stencil<LEN> stn = make_stencil<LEN>();
    const PcgCtl *ctl = a.ctl;
    if (*(volatile const int *)&ctl->done) return;
    extern __shared__ __align__(16) float pipe_smem[];
    __shared__ __align__(8) uint64_t bars[NBAR];
    float *band = pipe_smem;                 // NSLOT x BROWS x D
    float *aof = band + NSLOT * BROWS * D;   // NBAR x TS x LEN
    float *adg = aof + NBAR * TS * LEN;      // NBAR x TS
    using A = Acc<T>;
    using AT = typename A::type;
    using SW = SubWarp<T, D>;
    constexpr int V = SW::V;
    const T *__restrict__ pp = a.p[ctl->iter & 1];  // FSAI alternates the buffers
    AT pq[1][V];
#pragma unroll
    for (int k = 0; k < V; ++k) pq[0][k] = A::zero();
    const SW lm;
    const BlockSeg bsg = block_seg<false>(a.sg);
    const int64_t n = bsg.r1, W = a.grid_w, H = n / W;
    const int64_t NS = (W + TS - 1) / TS, units = NS * (int64_t)nchunk, CH = (H + nchunk - 1) / nchunk;
    const int il = (threadIdx.x >> 5) * SW::RPW + lm.r;  // this lane's pixel of a step
    const int c0 = lm.cg * V;
    if (threadIdx.x == 0) {
        for (int b = 0; b < NBAR; ++b) mbar_init(&bars[b], 1);
        mbar_init_fence();
    }
    __syncthreads();
    uint32_t phase = 0;  // bit b: parity of barrier b's next phase (the same in every thread)
    bool failed = false;
    for (int64_t u = blockIdx.x; u < units && !failed; u += gridDim.x) {
        const int64_t x0 = (u % NS) * TS, y0 = (u / NS) * CH;
        const int w = (int)min((int64_t)TS, W - x0);
        const int64_t L = min(H, y0 + CH) - y0;  // steps (image rows) of this chunk
        if (L <= 0) continue;
        const int m = (w + 2 * R + PADL + Q - 1) / Q * Q;  // pixels copied per band
        // band k: image row y0 - R + k, pixels from x0 - R - PADL (at the image's
        // left and right edges these wrap into the next or previous row: read
        // only by padding slots), into slot k % NSLOT; [lo, hi) is the part in
        // [0, n) (the rest is zero-filled)
        auto band_span = [&](int64_t k, int64_t &jb, int64_t &lo, int64_t &hi) {
            jb = (y0 - R + k) * W + x0 - R - PADL;
            lo = max(jb, (int64_t)0);
            hi = max(lo, min(jb + m, n));
        };
        // thread 0: request step q's group (bands kb0 .. q + 2R, row data of
        // image row y0 + q) on bars[q % NBAR]
        auto issue = [&](int64_t q, int64_t kb0) {
            uint64_t *bar = &bars[q % NBAR];
            const int64_t pix0 = (y0 + q) * W + x0;
            uint32_t bytes = (uint32_t)w * (LEN + 1) * 4;
            for (int64_t k = kb0; k <= q + 2 * R; ++k) {
                int64_t jb, lo, hi;
                band_span(k, jb, lo, hi);
                bytes += (uint32_t)((hi - lo) * D * 4);
            }
            mbar_arrive_expect_tx(bar, bytes);
            // order the block's earlier generic writes to these slots (zero
            // fills) before the copies' writes
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            for (int64_t k = kb0; k <= q + 2 * R; ++k) {
                int64_t jb, lo, hi;
                band_span(k, jb, lo, hi);
                if (hi > lo)
                    bulk_copy_g2s(band + (int)(k % NSLOT) * BROWS * D + (lo - jb) * D, pp + lo * D,
                                  (uint32_t)((hi - lo) * D * 4), bar);
            }
            const int slot = (int)(q % NBAR);
            bulk_copy_g2s(aof + slot * TS * LEN, a.A.aoff + pix0 * LEN, (uint32_t)w * LEN * 4, bar);
            bulk_copy_g2s(adg + slot * TS, a.A.adiag + pix0, (uint32_t)w * 4, bar);
        };
        // every thread: zero the parts of bands kb0 .. q + 2R outside [0, n)
        auto zero_clipped = [&](int64_t q, int64_t kb0) {
            for (int64_t k = kb0; k <= q + 2 * R; ++k) {
                int64_t jb, lo, hi;
                band_span(k, jb, lo, hi);
                if (lo == jb && hi == jb + m) continue;
                float *dst = band + (int)(k % NSLOT) * BROWS * D;
                for (int e = threadIdx.x; e < m * D; e += kBlock) {
                    const int64_t j = jb + e / D;
                    if (j < lo || j >= hi) dst[e] = 0.f;
                }
            }
        };
        const int64_t npro = min(L, (int64_t)P);
        zero_clipped(0, 0);
        for (int64_t q = 1; q < npro; ++q) zero_clipped(q, q + 2 * R);
        if (threadIdx.x == 0) {
            issue(0, 0);
            for (int64_t q = 1; q < npro; ++q) issue(q, q + 2 * R);
        }
        int st = 0;
        const bool lane_on = lm.active && il < w;
        const int lane_off = (il + R + PADL) * D + c0;  // the lane's pixel (dx = 0) within a band slot
        T *qrow = a.q + ((y0 * W + x0 + il) * D + c0);              // its output row at step 0
        for (; st < (int)L; ++st) {
            const int b = st % NBAR;
            // thread 0 waits for step st's copies; the block barrier then also
            // means every thread is done with step st - 1, whose band slot,
            // row-data slot and barrier are reused; every other thread then
            // observes the completed phase itself (no spinning)
            bool got = true;
            if (threadIdx.x == 0) got = mbar_wait(&bars[b], (phase >> b) & 1u);
            if (__syncthreads_or(!got)) {
                failed = true;
                break;
            }
            if (threadIdx.x != 0) mbar_wait(&bars[b], (phase >> b) & 1u);
            phase ^= 1u << b;
            if (st + P < L) {
                zero_clipped(st + P, st + P + 2 * R);
                if (threadIdx.x == 0) issue(st + P, st + P + 2 * R);
            }
            if (lane_on) {
                const float *av = aof + b * TS * LEN + il * LEN;
                const T ad = adg[b * TS + il];
                // the 2R + 1 bands of this step (image rows y - R .. y + R), as
                // 32-bit offsets into shared memory
                int bo[2 * R + 1];
#pragma unroll
                for (int k = 0; k <= 2 * R; ++k) bo[k] = ((st + k) % NSLOT) * (BROWS * D) + lane_off;
                T pi[V], acc[V];
#pragma unroll
                for (int q = 0; q < V; ++q) pi[q] = band[bo[R] + q];
#pragma unroll
                for (int q = 0; q < V; ++q) acc[q] = ad * pi[q];
#pragma unroll
                for (int g4 = 0; g4 < LEN / 4; ++g4) {
                    const float4 a4 = *reinterpret_cast<const float4 *>(av + 4 * g4);
                    const float aw[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const int t = 4 * g4 + h;
                        const int o = bo[stn.dy[t] + R] + stn.dx[t] * D;
#pragma unroll
                        for (int q = 0; q < V; ++q) acc[q] = fma(aw[h], band[o + q], acc[q]);
                    }
                }
                stv<T, V>(qrow, acc);
#pragma unroll
                for (int q = 0; q < V; ++q) A::add_prod(pq[0][q], pi[q], acc[q]);
            }
            qrow += W * D;
        }
        if (failed) {
            // report; let the groups already requested (steps st .. min(L, st + P) - 1) land
            if (threadIdx.x == 0) atomicMax(&a.ctl->error, (int)PFE_ETIMEOUT);
            for (int64_t g = st; g < min(L, (int64_t)st + P); ++g) {
                const int b = (int)(g % NBAR);
                mbar_wait(&bars[b], (phase >> b) & 1u);
                phase ^= 1u << b;
            }
        }
        __syncthreads();  // the next chunk refills every buffer
    }
    __shared__ double tot[D];
    if (grid_sum_cols<T, D, 1>(pq, a.part, bsg, &a.sc.ticket[bsg.seg * 4 + 0], tot))
        if (threadIdx.x < 32) spmm_finish<T, D, false>(a, bsg, tot);
}

template <typename T, int D>
int64_t rows_need(const pfe_ctx *c);

// The SpMM variants (pfe_autotune picks one per context; PFE_SPMM_AUTO
// applies the default rule):
//   PFE_SPMM_GENERAL  any layout, kChunk slots at a time
//   PFE_SPMM_ROW1     fixed row length, one row group per step, >= 6 blocks/SM
//   PFE_SPMM_ROW2     fixed row length, two row groups per step, >= 5 blocks/SM
//   PFE_SPMM_ROW2_4   fixed row length, two row groups per step, >= 4 blocks/SM
//   PFE_SPMM_TMA      fixed row length, slots of row tiles staged by bulk copies
//   PFE_SPMM_STENCIL  one grid image: stencil form, p and A staged by a ring of row bands
// Fixed-length variants exist for the FP32 single-problem path at radius 2
// and 3 (12 and 28 slots) and, one row group per step, for FP32 batches at
// radius 2; elsewhere the general kernel runs.
template <typename T, int D, bool MS, int LEN>
bool launch_spmm_fixed(pfe_ctx *c, cudaStream_t s, const PcgArgs<T> &a, int v) {
    if constexpr (!MS) {
        if (v == PFE_SPMM_STENCIL) {
            constexpr int P = kStencilSteps;
            using SP = StencilPipe<T, D, LEN, P>;
            if constexpr (SP::kAligned) {
                constexpr int MB = 4;  // 64 registers: the pipeline bookkeeping and the row math stay in registers
                auto kern = k_spmm_stencil<T, D, LEN, P, MB>;
                const int64_t W = c->W, H = c->g.n / W, NS = (W + SP::TS - 1) / SP::TS;
                int &grid = c->kgrid[G_SPMM_STENCIL];
                if (grid == 0) {
                    // dynamic shared memory past the default 48 KB less the kernel's static arrays
                    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SP::SMEM);
                    int occ = 0;
                    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kBlock, SP::SMEM) != cudaSuccess ||
                        occ < 1) {
                        cudaGetLastError();
                        occ = 1;
                    }
                    const int64_t maxb = (int64_t)occ * c->num_sms;
                    const int64_t nch = std::max<int64_t>(1, std::min<int64_t>(H, maxb / NS));
                    grid = (int)std::min<int64_t>(maxb, NS * nch);
                }
                const int nchunk = (int)std::max<int64_t>(1, std::min<int64_t>(H, grid / NS));
                kern<<<grid, kBlock, SP::SMEM, s>>>(a, nchunk);
                return true;
            }
        }
        if (v == PFE_SPMM_TMA) {
            constexpr int S = 2;
            using P = SpmmTma<T, D, LEN, S>;
            // with the kernel's static arrays (block reduction, < 8 KB) within
            // the 48 KB a block gets without opting in
            static_assert(P::SMEM <= 40 * 1024, "shared-memory budget");
            const int64_t ntiles = (c->g.n + P::TR - 1) / P::TR;
            constexpr int MB = SubWarp<T, D>::V * (int)sizeof(T) >= 16 ? 4 : 6;  // 40 registers up to 2 columns a lane
            k_spmm_tma<T, D, LEN, S, MB><<<wave_grid(c, G_SPMM_TMA, k_spmm_tma<T, D, LEN, S, MB>, ntiles, 1, P::SMEM),
                                           kBlock, P::SMEM, s>>>(a);
            return true;
        }
    }
    if constexpr (!MS) {
        if (v == PFE_SPMM_GRID1 && a.grid_w > 0) {
            k_spmm_fixed<T, D, MS, LEN, 1, 6, true><<<wave_grid(c, G_SPMM_G1, k_spmm_fixed<T, D, MS, LEN, 1, 6, true>,
                                                                rows_need<T, D>(c)),
                                                      kBlock, 0, s>>>(a);
            return true;
        }
        if (v == PFE_SPMM_GRID2 && a.grid_w > 0) {
            k_spmm_fixed<T, D, MS, LEN, 2, 5, true><<<wave_grid(c, G_SPMM_G2, k_spmm_fixed<T, D, MS, LEN, 2, 5, true>,
                                                                rows_need<T, D>(c)),
                                                      kBlock, 0, s>>>(a);
            return true;
        }
    }
    if (v == PFE_SPMM_ROW1)
        k_spmm_fixed<T, D, MS, LEN, 1, 6><<<wave_grid(c, G_SPMM_F1, k_spmm_fixed<T, D, MS, LEN, 1, 6>,
                                                      rows_need<T, D>(c)),
                                            kBlock, 0, s>>>(a);
    else if (v == PFE_SPMM_ROW2)
        k_spmm_fixed<T, D, MS, LEN, 2, 5><<<wave_grid(c, G_SPMM_F2, k_spmm_fixed<T, D, MS, LEN, 2, 5>,
                                                      rows_need<T, D>(c)),
                                            kBlock, 0, s>>>(a);
    else if (v == PFE_SPMM_ROW2_4)
        k_spmm_fixed<T, D, MS, LEN, 2, 4><<<wave_grid(c, G_SPMM_F3, k_spmm_fixed<T, D, MS, LEN, 2, 4>,
                                                      rows_need<T, D>(c)),
                                            kBlock, 0, s>>>(a);
    else
        return false;
    return true;
}
template <typename T, int D, bool MS>
void launch_spmm(pfe_ctx *c, cudaStream_t s, const PcgArgs<T> &a, int variant = -1) {
    const int v = variant >= 0 ? variant : c->spmm_variant;
    bool done = false;
    if constexpr (std::is_same_v<T, float> && !MS) {
        if (c->g.row_len == 12) done = launch_spmm_fixed<T, D, MS, 12>(c, s, a, v);
        else if (c->g.row_len == 28) done = launch_spmm_fixed<T, D, MS, 28>(c, s, a, v);
    } else if constexpr (std::is_same_v<T, float> && MS) {  // batches: the one-row variant
        if (v == PFE_SPMM_ROW1 && c->g.row_len == 12) {
            k_spmm_fixed<T, D, MS, 12, 1, 6><<<wave_grid(c, G_SPMM_F1, k_spmm_fixed<T, D, MS, 12, 1, 6>,
                                                         rows_need<T, D>(c)),
                                               kBlock, 0, s>>>(a);
            done = true;
        }
    }
    if (!done) k_spmm<T, D, MS><<<wave_grid(c, G_SPMM, k_spmm<T, D, MS>, rows_need<T, D>(c)), kBlock, 0, s>>>(a);
}

// Flat vectorised traversal of an n x D array: thread t handles the VEC
// consecutive elements starting at VEC*t, then strides by VEC * (threads of
// the grid).  The grid is a multiple of D / gcd(D, VEC*kBlock) blocks, so a
// thread always meets the same VEC columns and keeps one accumulator per
// element slot; the tail (n*D mod VEC elements) goes to the first threads.
// r -= alpha q and the dots r.z, r.r of the new residual -> beta, convergence.
// Sub-warp mapping (cheap per-column block sums), two row groups per step.
template <typename T, int D, bool MS>
__global__ void __launch_bounds__(kBlock) k_update(PcgArgs<T> a) {
    if (*(volatile int *)&a.ctl->done) return;
    using SWt = SubWarp<T, D>;
    const BlockSeg bsg = block_seg<MS>(a.sg);
    __shared__ T salpha[D];
    if (threadIdx.x < D) salpha[threadIdx.x] = (T)a.sc.alpha[bsg.seg * D + threadIdx.x];
    __syncthreads();
    __shared__ DF sq_sh[sqsum_slots<T, 2, SWt::V>()];
    SqSum<T, 2, SWt::V> sq(sq_sh);  // r.z (= r.D_A^{-1}r) | r.r
    {
        using SW = SWt;
        constexpr int V = SW::V;
        const SW lm;
        const int64_t warp_g = (int64_t)(blockIdx.x - bsg.b0) * kWarps + (threadIdx.x >> 5);
        const int64_t warps_total = (int64_t)bsg.nb * kWarps;
        const int64_t seg_rows = (!MS || __ldcg(a.sc.seg_active + bsg.seg)) ? bsg.r1 - bsg.r0 : 0;
        const int c0 = lm.cg * V;
        T al[V];
#pragma unroll
        for (int k = 0; k < V; ++k) al[k] = salpha[c0 + k];
        for (int64_t g = warp_g; g * SW::RPW < seg_rows; g += 2 * warps_total) {
            T rv[2][V], qv[2][V], dv[2];
            bool ok[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t i = bsg.r0 + (g + h * warps_total) * SW::RPW + lm.r;
                ok[h] = lm.active && i < bsg.r1;
                const int64_t ic = (ok[h] ? i : 0) * D + c0;
                ldv<T, V>(a.r + ic, rv[h]);
                ldv<T, V>(a.q + ic, qv[h]);
                dv[h] = a.A.dinv[ok[h] ? i : 0];
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!ok[h]) continue;
                const int64_t i = bsg.r0 + (g + h * warps_total) * SW::RPW + lm.r;
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    const T ri = fma(-al[k], qv[h][k], rv[h][k]);
                    sq.add(0, k, ri, dv[h] * ri);
                    sq.add(1, k, ri, ri);
                    rv[h][k] = ri;
                }
                stv<T, V>(a.r + i * D + c0, rv[h]);
            }
            sq.row_done();
        }
    }
    sq.finish();
    __shared__ double tot[2 * D];
    if (grid_sum_cols<T, D, 2>(sq.acc, a.part, bsg, &a.sc.ticket[bsg.seg * 4 + 1], tot)) {
        if (threadIdx.x < 32) {
            PcgCtl *ctl = a.ctl;
            const int it = ctl->iter + 1;
            // an error here can only come from an earlier kernel while a refresh is due
            // (periodic, or asked for by a column at the end of the last iteration)
            int due = 0;
            if (threadIdx.x == 0)
                due = !*(volatile int *)&ctl->error && ctl->refresh > 0 &&
                      ((it % ctl->refresh) == 0 || *(volatile int *)&ctl->refresh_next);
            const bool refresh_due = __shfl_sync(kFull, due, 0) != 0;
            if (!refresh_due) finish_seg(ctl, a.sc, bsg.seg, tot, tot + D, D, 2, it);
            // |r_rec|^2 of the residual the replacement will replace (k_refresh
            // measures how far the true residual lies from it)
            if (refresh_due)
                for (int c = threadIdx.x; c < D; c += 32) a.sc.rec2[bsg.seg * D + c] = tot[D + c];
            // the next k_pupdate holds this iteration's solution update when
            // none is held now (xheld changes only in the last finisher below):
            // each segment keeps its alpha for the fold
            if (!refresh_due && !*(volatile int *)&ctl->xheld)
                for (int c = threadIdx.x; c < D; c += 32) a.sc.alpha_prev[bsg.seg * D + c] = a.sc.alpha[bsg.seg * D + c];
            __syncwarp();
            if (!MS || warp_last_segment(ctl, 1, a.sg.nseg)) {
                if (threadIdx.x == 0) {
                    ctl->iter = it;
                    if (refresh_due) ctl->refresh_now = 1;  // k_xflush + k_refresh finish this iteration
                    set_if(a, refresh_due);
                }
                __syncwarp();
                if (!refresh_due) {
                    finish_all(ctl, a.sc, a.sg.nseg, D, a.cond, a.use_cond);
                    if (threadIdx.x == 0 && !ctl->done) {  // once done the held state stays for the final k_xflush
                        const int fold = ctl->xheld;
                        ctl->xfold = fold;
                        ctl->xheld = !fold;
                    }
                    if (threadIdx.x == 0) {  // every segment's request of this iteration, for the next
                        ctl->refresh_next = ctl->refresh_want;
                        ctl->refresh_want = 0;
                    }
                }
            }
        }
    }
}

// y += alpha p with the direction of the last k_spmm (and y += alpha_prev
// p_prev when an update is held).  In the loop body it runs only on
// replacement iterations; after the loop it applies the final update.  Flat
// float4 / double2 traversal like k_pupdate (the grid makes every thread meet
// fixed columns).
template <typename T, int D, bool MS>
__global__ void __launch_bounds__(kBlock) k_xflush(PcgArgs<T> a, int final_flush, int counted) {
    const PcgCtl *ctl = a.ctl;
    const int xp = *(volatile const int *)&ctl->xpending, xh = *(volatile const int *)&ctl->xheld;
    if (!xp && !xh) return;
    if (!final_flush && !*(volatile const int *)&ctl->refresh_now) return;
    constexpr bool multi = MS;
    __shared__ T salpha[D], salpha_prev[D];
    if (threadIdx.x < D) {
        salpha[threadIdx.x] = xp ? (T)a.sc.alpha[threadIdx.x] : T(0);
        salpha_prev[threadIdx.x] = xh ? (T)a.sc.alpha_prev[threadIdx.x] : T(0);
    }
    __syncthreads();
    // the direction of the last k_spmm: buffer iter & 1 before the iteration's
    // finisher counted it (FSAI refresh iterations), the other one after
    // (counted: Jacobi refresh iterations and the flush after the loop); the
    // direction before it in the other buffer
    const int kc = counted ? ((ctl->iter & 1) ^ 1) : (ctl->iter & 1);
    const T *__restrict__ pc = a.p[kc];
    const T *__restrict__ pprev = a.p[kc ^ 1];
    using VT = Vec<T>;
    constexpr int VN = VT::N;
    const int64_t nel = a.A.n * D, nvec = nel / VN;
    const int64_t tid = (int64_t)blockIdx.x * kBlock + threadIdx.x, nthr = (int64_t)gridDim.x * kBlock;
    T al[VN], ap[VN];
    int cu[VN];
#pragma unroll
    for (int u = 0; u < VN; ++u) {
        cu[u] = (int)((tid * VN + u) % D);
        al[u] = salpha[cu[u]];
        ap[u] = salpha_prev[cu[u]];
    }
    using V4 = typename VT::V;
    const V4 *pc4 = reinterpret_cast<const V4 *>(pc);
    const V4 *pp4 = reinterpret_cast<const V4 *>(pprev);
    V4 *x4 = reinterpret_cast<V4 *>(a.x);
    float4 *xl4 = reinterpret_cast<float4 *>(a.xlo);  // float path: VN == 4
    for (int64_t v = tid; v < nvec; v += nthr) {
        if constexpr (multi) {
            const int64_t row0 = v * VN / D;
#pragma unroll
            for (int u = 0; u < VN; ++u) {
                const int sgm = __ldg(a.sg.rseg + row0 + (cu[0] + u) / D);
                al[u] = xp ? (T)a.sc.alpha[sgm * D + cu[u]] : T(0);
                ap[u] = xh ? (T)a.sc.alpha_prev[sgm * D + cu[u]] : T(0);
            }
        }
        T xv[VN], pv[VN], qv[VN];
        float xl[VN] = {};
        VT::get(x4[v], xv);
        if constexpr (std::is_same_v<T, float>) {
            const float4 t = xl4[v];
            xl[0] = t.x; xl[1] = t.y; xl[2] = t.z; xl[3] = t.w;
        }
        if (xh) {
            VT::get(pp4[v], qv);
#pragma unroll
            for (int u = 0; u < VN; ++u) axpy_hilo<T>(xv[u], xl[u], ap[u], qv[u]);
        }
        if (xp) {
            VT::get(pc4[v], pv);
#pragma unroll
            for (int u = 0; u < VN; ++u) axpy_hilo<T>(xv[u], xl[u], al[u], pv[u]);
        }
        x4[v] = VT::make(xv);
        if constexpr (std::is_same_v<T, float>) xl4[v] = make_float4(xl[0], xl[1], xl[2], xl[3]);
    }
    if (tid < nel - nvec * VN) {  // tail elements
        const int64_t e = nvec * VN + tid;
        const int c = (int)(e % D);
        const int sgm = multi ? row_seg(a.sg, e / D) : 0;
        T xv = a.x[e];
        float xl = 0.f;
        if constexpr (std::is_same_v<T, float>) xl = a.xlo[e];
        if (xh) axpy_hilo<T>(xv, xl, multi ? (T)a.sc.alpha_prev[sgm * D + c] : salpha_prev[c], pprev[e]);
        if (xp) axpy_hilo<T>(xv, xl, multi ? (T)a.sc.alpha[sgm * D + c] : salpha[c], pc[e]);
        a.x[e] = xv;
        if constexpr (std::is_same_v<T, float>) a.xlo[e] = xl;
    }
    // the flags are cleared by whoever reads them next: k_refresh's last
    // block (xpending) and the finisher of the refresh iteration (xheld), or
    // k_pcg_init of the next solve
    if (final_flush) {
        if (last_block_arrives(&a.ctl->ticket[3])) {
            if (threadIdx.x == 0) {
                a.ctl->xpending = 0;
                a.ctl->xheld = 0;
                a.ctl->ticket[3] = 0u;
            }
        }
    }
}

// ---- FSAI preconditioner, z = G^T (G r) --------------------------------------
// With t = G r the PCG dot is r.z = r^T G^T G r = t.t, so it is known as soon
// as t is; z itself is needed only for p = z + beta p.  An FSAI iteration is
//   k_spmm     q = A p, partials of p.q -> alpha
//   k_fsai_tr  r -= alpha q and t = G r in one pass, the dots t.t and r.r ->
//              beta, convergence (skipped on refresh iterations)
//   k_xflush, k_refresh_f, k_fsai_t<1>  (refresh iterations) y += alpha p,
//              r = b - A y, t = G r with the dots
//   k_fsai_zp  z = G^T t fused with p = z + beta p and the delayed y +=
//              alpha p_prev (z is never stored)
// and a solve starts with k_pcg_init<PRE = 1>, k_fsai_t<0>, k_fsai_zp.

// Residual replacement without the preconditioned dots (k_fsai_t<1> makes
// them); it writes the buffer of the new residual (k_fsai_tr does not run on
// replacement iterations).  It also measures how far the true residual lies
// from the recurrence residual r - alpha q it replaces (|r - r_rec|^2 /
// |r_rec|^2 per column -> sc.devr, for the restart test).
template <typename T, int D, int LEN, bool MS, bool GRID = false>
__global__ void __launch_bounds__(kBlock) k_refresh_f(PcgArgs<T> a) {
    if (*(volatile int *)&a.ctl->done || !*(volatile int *)&a.ctl->refresh_now) return;
    const int par = a.ctl->iter & 1;
    const T *__restrict__ rold = a.r2[par];
    T *__restrict__ rdst = a.r2[par ^ 1];
    __shared__ T salpha[D];
    {
        const BlockSeg bs0 = block_seg<MS>(a.sg);
        if (threadIdx.x < D) salpha[threadIdx.x] = (T)a.sc.alpha[bs0.seg * D + threadIdx.x];
    }
    __syncthreads();
    __shared__ DF sq_sh[sqsum_slots<T, 2, SubWarp<T, D>::V>()];
    SqSum<T, 2, SubWarp<T, D>::V> sq(sq_sh);  // |r - r_rec|^2 | |r_rec|^2
    PFE_ROW_LOOP_MS(T, D, MS) {
        PFE_ROW_I;
        const int c0 = lm.cg * V;
        T ri[V], ro[V], qi[V];
        ldv<T, V>(rold + i * D + c0, ro);
        ldv<T, V>(a.q + i * D + c0, qi);
        true_residual<T, D, V, LEN, GRID>(a, i, c0, ri);
        stv<T, V>(rdst + i * D + c0, ri);
#pragma unroll
        for (int k = 0; k < V; ++k) {
            const T rrec = fma(-salpha[c0 + k], qi[k], ro[k]);
            const T dr = ri[k] - rrec;
            sq.add(0, k, dr, dr);
            sq.add(1, k, rrec, rrec);
        }
        sq.row_done();
    }
    sq.finish();
    __shared__ double tot[2 * D];
    if (grid_sum_cols<T, D, 2>(sq.acc, a.part, bsg, &a.sc.ticket[bsg.seg * 4 + 3], tot)) {
        if (threadIdx.x < 32) {
            for (int c = threadIdx.x; c < D; c += 32) {
                const double rec = tot[D + c];
                a.sc.devr[bsg.seg * D + c] = rec > 0.0 ? tot[c] / rec : (tot[c] > 0.0 ? INFINITY : 0.0);
            }
            if (threadIdx.x == 0) a.ctl->xpending = 0;
        }
    }
}

// In FSAI mode the residual is double-buffered: during iteration k (k =
// ctl->iter) the current residual is r2[k & 1] and the new one is written to
// r2[(k + 1) & 1]; the finisher of k_fsai_tr (k_fsai_t<1> on refresh
// iterations) ends the iteration by incrementing k.

// acc += sum of g_k * v(j_k) over the slots k in [lo, hi) among the CH slots
// from k0 on (k0 a multiple of 4; 16-byte slot loads, slots outside the range
// gather the own row with weight 0).  v = src, or src - alpha q with QS.
template <typename T, int D, int V, int CH, bool QS>
__device__ __forceinline__ void gslot_chunk(const int *__restrict__ col, const T *__restrict__ gs, int64_t base,
                                            int k0, int len, int lo, int hi, int self, int c0,
                                            const T *__restrict__ src, const T *__restrict__ qsrc, const T (&al)[V],
                                            T (&acc)[V]) {
    int jj[CH];
    T gv[CH];
    load_slots<T, CH>(col, gs, base, k0, len, self, jj, gv);
#pragma unroll
    for (int u = 0; u < CH; ++u) {
        const int k = k0 + u;
        if (k < lo || k >= hi) {
            jj[u] = self;
            gv[u] = T(0);
        }
    }
    T vj[CH][V];
#pragma unroll
    for (int u = 0; u < CH; ++u) ldv<T, V>(src + (int64_t)jj[u] * D + c0, vj[u]);
    if constexpr (QS) {
        T qj[CH][V];
#pragma unroll
        for (int u = 0; u < CH; ++u) ldv<T, V>(qsrc + (int64_t)jj[u] * D + c0, qj[u]);
#pragma unroll
        for (int u = 0; u < CH; ++u)
#pragma unroll
            for (int k = 0; k < V; ++k) vj[u][k] = fma(-al[k], qj[u][k], vj[u][k]);
    }
#pragma unroll
    for (int u = 0; u < CH; ++u)
#pragma unroll
        for (int k = 0; k < V; ++k) acc[k] = fma(gv[u], vj[u][k], acc[k]);
}

// The FSAI gather kernels are latency-bound: 5 resident blocks of kBlock per SM
// (48 registers a thread) with up to 2 columns a lane, 4 with 4 columns; 6
// (40 registers) for the 12-slot fixed rows with up to 2 columns a lane
// (LEN6 = true: k_fsai_zp, which fits there without spilling; k_fsai_tr,
// with the second gather and the dots, does not).
template <typename T, int D, int LEN = 0, bool LEN6 = false>
constexpr int gather_min_blocks() {
    return SubWarp<T, D>::V * (int)sizeof(T) >= 16 ? 4 : (LEN6 && LEN == 12 ? 6 : 5);
}

// End of an FSAI iteration (or of the start of a solve) from the dots
// tot = [t.t | r.r]: warp 0 of the last block.  MODE 0: start of a solve,
// 1: a refresh iteration (k_xflush applied every pending update), 2: an
// ordinary iteration.
// The solution update y += alpha p of an ordinary iteration is held and
// applied together with the next one (y += alpha_prev p_prev + alpha p in
// one pass of k_fsai_zp, the directions in alternating buffers): the hi/lo
// solution is read and written every other iteration.  Once the solve is
// done the held state stays for the final k_xflush.  MS (a batch): each
// segment's last block finishes its segment; the last segment to get there
// finishes the iteration.
template <typename T, bool MS = false>
__device__ void fsai_finish(const PcgArgs<T> &a, const BlockSeg &bsg, const double *tot, int D, int mode) {
    PcgCtl *ctl = a.ctl;
    finish_seg(ctl, a.sc, bsg.seg, tot, tot + D, D, mode, ctl->iter + 1);
    if (MS && !warp_last_segment(ctl, 1, a.sg.nseg)) return;
    if (threadIdx.x == 0 && mode != 0) ctl->iter += 1;
    if (threadIdx.x == 0 && mode == 1) ctl->refreshes += 1;
    __syncwarp();
    finish_all(ctl, a.sc, a.sg.nseg, D, a.cond, a.use_cond);
    int hold = 0;
    if (threadIdx.x == 0) {
        if (mode != 2) {
            ctl->xheld = 0;
            ctl->xfold = 0;
        } else if (!ctl->done) {
            const int fold = ctl->xheld;
            ctl->xfold = fold;
            ctl->xheld = !fold;
            hold = !fold;
        }
    }
    hold = __shfl_sync(kFull, hold, 0);
    if (hold)
        for (int c = threadIdx.x; c < a.sg.nseg * D; c += 32) a.sc.alpha_prev[c] = a.sc.alpha[c];
    __syncwarp();
}

// All slots in [lo, hi): chunks of kGChunk = 8 slots (the 6 lower or upper
// slots of a radius-2 row in one chunk), then one chunk of 4 if needed.
constexpr int kGChunk = 8;
template <typename T, int D, int V, bool QS>
__device__ __forceinline__ void gslot_range(const int *__restrict__ col, const T *__restrict__ gs, int64_t base,
                                            int len, int lo, int hi, int self, int c0, const T *__restrict__ src,
                                            const T *__restrict__ qsrc, const T (&al)[V], T (&acc)[V]) {
    int k0 = lo & ~3;
    for (; k0 + 4 < hi; k0 += kGChunk)
        gslot_chunk<T, D, V, kGChunk, QS>(col, gs, base, k0, len, lo, hi, self, c0, src, qsrc, al, acc);
    if (k0 < hi) gslot_chunk<T, D, V, 4, QS>(col, gs, base, k0, len, lo, hi, self, c0, src, qsrc, al, acc);
}

// acc += sum of g_k * v(j_k) over the slots k in [P0, P1) of a row with
// compile-time positions (uniform-length rows; padding slots carry g = 0):
// exact-range slot loads, then the gathers.
template <typename T, int D, int V, int P0, int P1, bool QS>
__device__ __forceinline__ void gslot_fixed(const int *__restrict__ col, const T *__restrict__ gs, int64_t base,
                                            int c0, const T *__restrict__ src, const T *__restrict__ qsrc,
                                            const T (&al)[V], T (&acc)[V]) {
    constexpr int NS = P1 - P0;
    int jj[NS];
    T gv[NS];
    load_slot_range<T, P0, P1>(col, gs, base, jj, gv);
    T vj[NS][V];
#pragma unroll
    for (int u = 0; u < NS; ++u) ldv<T, V>(src + (int64_t)jj[u] * D + c0, vj[u]);
    if constexpr (QS) {
        T qj[NS][V];
#pragma unroll
        for (int u = 0; u < NS; ++u) ldv<T, V>(qsrc + (int64_t)jj[u] * D + c0, qj[u]);
#pragma unroll
        for (int u = 0; u < NS; ++u)
#pragma unroll
            for (int k = 0; k < V; ++k) vj[u][k] = fma(-al[k], qj[u][k], vj[u][k]);
    }
#pragma unroll
    for (int u = 0; u < NS; ++u)
#pragma unroll
        for (int k = 0; k < V; ++k) acc[k] = fma(gv[u], vj[u][k], acc[k]);
}

// gslot_fixed on a one-image grid graph with the columns computed from the
// stencil (stencil_col) instead of loaded: the same products in the same
// order, 4 bytes a slot less traffic.
template <typename T, int D, int V, int P0, int P1, int LEN, bool QS>
__device__ __forceinline__ void gslot_grid(const T *__restrict__ gs, int64_t i, int w, int n, int c0,
                                           const T *__restrict__ src, const T *__restrict__ qsrc, const T (&al)[V],
                                           T (&acc)[V]) {
    constexpr int NS = P1 - P0;
    T gv[NS];
    load_val_range<T, P0, P1>(gs, i * LEN, gv);
    int jj[NS];
    stencil_cols<LEN, P0>((int)i, w, n, jj);
    T vj[NS][V];
#pragma unroll
    for (int u = 0; u < NS; ++u) ldv<T, V>(src + (int64_t)jj[u] * D + c0, vj[u]);
    if constexpr (QS) {
        T qj[NS][V];
#pragma unroll
        for (int u = 0; u < NS; ++u) ldv<T, V>(qsrc + (int64_t)jj[u] * D + c0, qj[u]);
#pragma unroll
        for (int u = 0; u < NS; ++u)
#pragma unroll
            for (int k = 0; k < V; ++k) vj[u][k] = fma(-al[k], qj[u][k], vj[u][k]);
    }
#pragma unroll
    for (int u = 0; u < NS; ++u)
#pragma unroll
        for (int k = 0; k < V; ++k) acc[k] = fma(gv[u], vj[u][k], acc[k]);
}

// r' = r - alpha q and t = G r' in one pass: r' is recomputed at each
// gathered lower neighbour from the old r and q (the same FMA its owner
// uses), the owner writes its r' to the other buffer; then the dots t.t
// (= r'.z') and r'.r' and the end of the iteration.  On refresh iterations
// it does nothing (k_refresh_f and k_fsai_t<1> make r and t).
// LEN > 0: uniform rows of LEN slots, lower slots at positions [0, LEN/2);
// GRID: one grid image, the slot columns computed from the stencil; MS: a
// batch (each block in one segment, with its alpha; segments whose columns
// have all converged are skipped).
template <typename T, int D, int LEN, bool GRID, bool MS>
__global__ void __launch_bounds__(kBlock, (gather_min_blocks<T, D>())) k_fsai_tr(PcgArgs<T> a) {
    const PcgCtl *ctl = a.ctl;
    if (*(volatile const int *)&ctl->done) return;
    if (ctl->refresh_now) return;
    __shared__ T salpha[D];
    {
        const BlockSeg bs0 = block_seg<MS>(a.sg);
        if (threadIdx.x < D) salpha[threadIdx.x] = (T)a.sc.alpha[bs0.seg * D + threadIdx.x];
    }
    __syncthreads();
    __shared__ DF sq_sh[sqsum_slots<T, 2, SubWarp<T, D>::V>()];
    SqSum<T, 2, SubWarp<T, D>::V> sq(sq_sh);  // t.t (= r.z) | r.r
    const int par = ctl->iter & 1;
    const T *__restrict__ rold = a.r2[par];
    T *__restrict__ rnew = a.r2[1 - par];
    PFE_ROW_LOOP_LIVE(T, D, MS) {
        PFE_ROW_I;
        const int c0 = lm.cg * V;
        T al[V];
#pragma unroll
        for (int k = 0; k < V; ++k) al[k] = salpha[c0 + k];
        int64_t base;
        int len;
        sell_row(a.A.slice_ptr, a.A.row_len, i, base, len);
        T acc[V], ri[V], qi[V];
        ldv<T, V>(rold + i * D + c0, ri);
        ldv<T, V>(a.q + i * D + c0, qi);
#pragma unroll
        for (int k = 0; k < V; ++k) ri[k] = fma(-al[k], qi[k], ri[k]);
        stv<T, V>(rnew + i * D + c0, ri);
        const T gd = a.gdiag[i];
#pragma unroll
        for (int k = 0; k < V; ++k) acc[k] = gd * ri[k];
        if constexpr (GRID)
            gslot_grid<T, D, V, 0, LEN / 2, LEN, true>(a.gslot, i, a.grid_w, (int)a.A.n, c0, rold, a.q, al, acc);
        else if constexpr (LEN > 0)
            gslot_fixed<T, D, V, 0, LEN / 2, true>(a.A.col, a.gslot, i * LEN, c0, rold, a.q, al, acc);
        else
            gslot_range<T, D, V, true>(a.A.col, a.gslot, base, len, 0, a.kb[i], (int)i, c0, rold, a.q, al, acc);
        stv<T, V>(a.t + i * D + c0, acc);
#pragma unroll
        for (int k = 0; k < V; ++k) {
            sq.add(0, k, acc[k], acc[k]);
            sq.add(1, k, ri[k], ri[k]);
        }
        sq.row_done();
    }
    sq.finish();
    __shared__ double tot[2 * D];
    if (grid_sum_cols<T, D, 2>(sq.acc, a.part, bsg, &a.sc.ticket[bsg.seg * 4 + 1], tot))
        if (threadIdx.x < 32) fsai_finish<T, MS>(a, bsg, tot, D, 2);
}

// t = G r: t_i = G_ii r_i + sum over the lower slots (j < i) of G_ij r_j, with
// the dots t.t (= r.z) and r.r.  MODE 0: the start of a solve (residual in
// r2[0]); MODE 1: only after a residual refresh (residual in the new buffer),
// ending the iteration.
template <typename T, int D, int MODE, int LEN, bool GRID, bool MS>
__global__ void __launch_bounds__(kBlock, (gather_min_blocks<T, D>())) k_fsai_t(PcgArgs<T> a) {
    if (*(volatile int *)&a.ctl->done) return;
    if (MODE == 1 && !*(volatile int *)&a.ctl->refresh_now) return;
    const T *__restrict__ rsrc = MODE == 0 ? a.r2[0] : a.r2[(a.ctl->iter + 1) & 1];
    __shared__ DF sq_sh[sqsum_slots<T, 2, SubWarp<T, D>::V>()];
    SqSum<T, 2, SubWarp<T, D>::V> sq(sq_sh);  // t.t (= r.z) | r.r
    PFE_ROW_LOOP_MS(T, D, MS) {
        PFE_ROW_I;
        const int c0 = lm.cg * V;
        int64_t base;
        int len;
        sell_row(a.A.slice_ptr, a.A.row_len, i, base, len);
        T acc[V], ri[V];
        const T nal[V] = {};
        ldv<T, V>(rsrc + i * D + c0, ri);
        const T gd = a.gdiag[i];
#pragma unroll
        for (int k = 0; k < V; ++k) acc[k] = gd * ri[k];
        if constexpr (GRID)
            gslot_grid<T, D, V, 0, LEN / 2, LEN, false>(a.gslot, i, a.grid_w, (int)a.A.n, c0, rsrc, nullptr, nal, acc);
        else if constexpr (LEN > 0)
            gslot_fixed<T, D, V, 0, LEN / 2, false>(a.A.col, a.gslot, i * LEN, c0, rsrc, nullptr, nal, acc);
        else
            gslot_range<T, D, V, false>(a.A.col, a.gslot, base, len, 0, a.kb[i], (int)i, c0, rsrc, nullptr, nal,
                                        acc);
        stv<T, V>(a.t + i * D + c0, acc);
#pragma unroll
        for (int k = 0; k < V; ++k) {
            sq.add(0, k, acc[k], acc[k]);
            sq.add(1, k, ri[k], ri[k]);
        }
        sq.row_done();
    }
    sq.finish();
    __shared__ double tot[2 * D];
    if (grid_sum_cols<T, D, 2>(sq.acc, a.part, bsg, &a.sc.ticket[bsg.seg * 4 + 1], tot))
        if (threadIdx.x < 32) fsai_finish<T, MS>(a, bsg, tot, D, MODE == 0 ? 0 : 1);
}

// z = G^T t (z_i = G_ii t_i + sum over the upper slots (j > i) of G_ji t_j)
// fused with the direction update p_new = z + beta p (p = z at the start of a
// solve) into the other direction buffer, and on folding iterations the two
// pending solution updates y += alpha_prev p_prev + alpha p (p_prev is the
// old content of the buffer p_new goes to); each thread reads and writes only
// its row's own entries; z is never stored.  Block 0 also decides whether the
// next iteration refreshes the residual.
template <typename T, int D, int LEN, bool GRID, bool MS>
__global__ void __launch_bounds__(kBlock, (gather_min_blocks<T, D, LEN, true>())) k_fsai_zp(PcgArgs<T> a) {
    PcgCtl *ctl = a.ctl;
    if (*(volatile int *)&ctl->done) return;
    const int p_ready = ctl->p_ready, fold = ctl->xpending && ctl->xfold;
    // p of this iteration in buffer iter & 1 before the finisher counted the
    // iteration (at the start of a solve: no old p), the new one in the other
    T *__restrict__ pdst = a.p[ctl->iter & 1];
    const T *__restrict__ psrc = a.p[(ctl->iter & 1) ^ 1];
    __shared__ T sbeta[D], salpha[D], salpha_prev[D];
    {
        const int sk = block_seg<MS>(a.sg).seg * D + threadIdx.x;  // this block's segment
        if (threadIdx.x < D) {
            sbeta[threadIdx.x] = p_ready ? T(0) : (T)a.sc.beta[sk];
            salpha[threadIdx.x] = (T)a.sc.alpha[sk];
            salpha_prev[threadIdx.x] = (T)a.sc.alpha_prev[sk];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {  // periodic, or asked for by a column in this iteration
        ctl->refresh_now = (ctl->refresh > 0 && (((ctl->iter + 1) % ctl->refresh) == 0 || ctl->refresh_want)) ? 1 : 0;
        ctl->refresh_want = 0;
        set_if(a, ctl->refresh_now);
    }
    __syncthreads();
    PFE_ROW_LOOP_MS(T, D, MS) {
        PFE_ROW_I;
        const int c0 = lm.cg * V;
        int64_t base;
        int len;
        sell_row(a.A.slice_ptr, a.A.row_len, i, base, len);
        T acc[V], ti[V], pv[V] = {};
        const T nal[V] = {};
        ldv<T, V>(a.t + i * D + c0, ti);
        const T gd = a.gdiag[i];
#pragma unroll
        for (int k = 0; k < V; ++k) acc[k] = gd * ti[k];
        if constexpr (GRID)
            gslot_grid<T, D, V, LEN / 2, LEN, LEN, false>(a.gslot, i, a.grid_w, (int)a.A.n, c0, a.t, nullptr, nal, acc);
        else if constexpr (LEN > 0)
            gslot_fixed<T, D, V, LEN / 2, LEN, false>(a.A.col, a.gslot, i * LEN, c0, a.t, nullptr, nal, acc);
        else
            gslot_range<T, D, V, false>(a.A.col, a.gslot, base, len, a.kb[i], len, (int)i, c0, a.t, nullptr, nal,
                                        acc);
        const int64_t ic = i * D + c0;
        if (!p_ready) ldv_rw<T, V>(psrc + ic, pv);
        if (fold) {
            T xh[V], pp[V];
            float xl[V] = {};
            ldv_rw<T, V>(pdst + ic, pp);
            ldv_rw<T, V>(a.x + ic, xh);
            if constexpr (std::is_same_v<T, float>) ldv_rw<float, V>(a.xlo + ic, xl);
#pragma unroll
            for (int k = 0; k < V; ++k) {
                axpy_hilo<T>(xh[k], xl[k], salpha_prev[c0 + k], pp[k]);
                axpy_hilo<T>(xh[k], xl[k], salpha[c0 + k], pv[k]);
            }
            stv<T, V>(a.x + ic, xh);
            if constexpr (std::is_same_v<T, float>) stv<float, V>(a.xlo + ic, xl);
        }
#pragma unroll
        for (int k = 0; k < V; ++k) pv[k] = p_ready ? acc[k] : acc[k] + sbeta[c0 + k] * pv[k];
        stv<T, V>(pdst + ic, pv);
    }
}

// ---- incomplete Cholesky IC(0), M^{-1} = L^{-T} L^{-1} --------------------------
// The FSAI iteration with G = L^{-1}: t = L^{-1} r (forward solve), r.z = t.t,
// z = L^{-T} t (backward solve, in place in t) fused with the direction and
// solution updates.  L is held like G (lower entries in a row's lower slots,
// the mirrored upper ones in its upper slots, L_ii in gdiag).  The solves run
// level by level over the raster wavefront (one launch per level, rows of a
// level in parallel, one thread per row and column).  An IC iteration:
//   k_spmm, k_ic_r (r -= alpha q; not on refresh iterations), k_xflush and
//   k_refresh_f (refresh iterations), k_ic_fwd per level, k_ic_dots (t.t,
//   r.r -> beta, convergence; decides the next refresh), k_ic_bwd per level
//   in reverse.  A solve starts with k_pcg_init<PRE = 1>, the forward levels,
//   k_ic_dots (start) and the backward levels.

// r' = r - alpha q into the other residual buffer (elementwise).
template <typename T, int D>
__global__ void __launch_bounds__(kBlock) k_ic_r(PcgArgs<T> a) {
    const PcgCtl *ctl = a.ctl;
    if (*(volatile const int *)&ctl->done) return;
    if (ctl->refresh_now) return;
    const int par = ctl->iter & 1;
    const T *__restrict__ rold = a.r2[par];
    T *__restrict__ rnew = a.r2[1 - par];
    const int64_t nel = a.A.n * D;
    for (int64_t e = (int64_t)blockIdx.x * kBlock + threadIdx.x; e < nel; e += (int64_t)gridDim.x * kBlock)
        rnew[e] = fma(-(T)a.sc.alpha[e % D], a.q[e], rold[e]);
}

// Forward level: t_i = (r_i - sum over the lower slots of L_ij t_j) / L_ii for
// the rows y0 .. y0 + rows - 1 of level `level` (x = level - cl y).
template <typename T, int D, int LEN>
__global__ void __launch_bounds__(kBlock) k_ic_fwd(PcgArgs<T> a, int64_t level, int64_t y0, int64_t rows, int start) {
    const PcgCtl *ctl = a.ctl;
    if (*(volatile const int *)&ctl->done) return;
    constexpr int cl = ic_level_coef<LEN>();
    const int64_t k = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    if (k >= rows * D) return;
    const int64_t y = y0 + k / D, i = y * a.grid_w + (level - cl * y);
    const int c = (int)(k % D);
    const T *__restrict__ src = start ? a.r2[0] : a.r2[(ctl->iter + 1) & 1];
    T acc = src[i * D + c];
#pragma unroll
    for (int t = 0; t < LEN / 2; ++t) {
        const int64_t j = a.A.col[i * LEN + t];
        if (j != i) acc = fma(-a.gslot[i * LEN + t], a.t[j * D + c], acc);
    }
    a.t[i * D + c] = acc / a.gdiag[i];
}

// t.t (= r.z) and r.r over all rows, then the end of the iteration (or of
// the start of the solve) and the refresh decision for the next iteration.
template <typename T, int D>
__global__ void __launch_bounds__(kBlock) k_ic_dots(PcgArgs<T> a, int start) {
    if (*(volatile int *)&a.ctl->done) return;
    const int mode = start ? 0 : (*(volatile int *)&a.ctl->refresh_now ? 1 : 2);
    const T *__restrict__ rsrc = start ? a.r2[0] : a.r2[(a.ctl->iter + 1) & 1];
    __shared__ DF sq_sh[sqsum_slots<T, 2, SubWarp<T, D>::V>()];
    SqSum<T, 2, SubWarp<T, D>::V> sq(sq_sh);  // t.t | r.r
    __syncthreads();
    PFE_ROW_LOOP(T, D) {
        PFE_ROW_I;
        const int c0 = lm.cg * V;
        T ti[V], ri[V];
        ldv_rw<T, V>(a.t + i * D + c0, ti);
        ldv<T, V>(rsrc + i * D + c0, ri);
#pragma unroll
        for (int k = 0; k < V; ++k) {
            sq.add(0, k, ti[k], ti[k]);
            sq.add(1, k, ri[k], ri[k]);
        }
        sq.row_done();
    }
    sq.finish();
    __shared__ double tot[2 * D];
    if (grid_sum_cols<T, D, 2>(sq.acc, a.part, bsg, &a.sc.ticket[bsg.seg * 4 + 1], tot)) {
        if (threadIdx.x < 32) {
            fsai_finish(a, bsg, tot, D, mode);
            if (threadIdx.x == 0) {  // periodic, or asked for by a column in this iteration
                PcgCtl *ctl = a.ctl;
                ctl->refresh_now =
                    (ctl->refresh > 0 && (((ctl->iter + 1) % ctl->refresh) == 0 || ctl->refresh_want)) ? 1 : 0;
                ctl->refresh_want = 0;
                if (!ctl->done) set_if(a, ctl->refresh_now);
            }
        }
    }
}

// Backward level: z_i = (t_i - sum over the upper slots of L_ji z_j) / L_ii
// in place, fused with the row's p_new = z + beta p and, on folding
// iterations, y += alpha_prev p_prev + alpha p (as k_fsai_zp).
template <typename T, int D, int LEN>
__global__ void __launch_bounds__(kBlock) k_ic_bwd(PcgArgs<T> a, int64_t level, int64_t y0, int64_t rows) {
    const PcgCtl *ctl = a.ctl;
    if (*(volatile const int *)&ctl->done) return;
    constexpr int cl = ic_level_coef<LEN>();
    const int64_t k = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    if (k >= rows * D) return;
    const int64_t y = y0 + k / D, i = y * a.grid_w + (level - cl * y);
    const int c = (int)(k % D);
    const int64_t e = i * D + c;
    T acc = a.t[e];
#pragma unroll
    for (int t = LEN / 2; t < LEN; ++t) {
        const int64_t j = a.A.col[i * LEN + t];
        if (j != i) acc = fma(-a.gslot[i * LEN + t], a.t[j * D + c], acc);
    }
    const T z = acc / a.gdiag[i];
    a.t[e] = z;
    const int p_ready = ctl->p_ready, fold = ctl->xpending && ctl->xfold;
    T *__restrict__ pdst = a.p[ctl->iter & 1];
    const T *__restrict__ psrc = a.p[(ctl->iter & 1) ^ 1];
    const T pv = p_ready ? T(0) : psrc[e];
    if (fold) {
        T xh = a.x[e];
        float xl = 0.f;
        if constexpr (std::is_same_v<T, float>) xl = a.xlo[e];
        axpy_hilo<T>(xh, xl, (T)a.sc.alpha_prev[c], pdst[e]);
        axpy_hilo<T>(xh, xl, (T)a.sc.alpha[c], pv);
        a.x[e] = xh;
        if constexpr (std::is_same_v<T, float>) a.xlo[e] = xl;
    }
    pdst[e] = p_ready ? z : z + (T)a.sc.beta[c] * pv;
}

// Residual replacement: r = b - A y (extended precision), then finish the
// iteration with the true residual.  Also |r - r_rec|^2, the squared
// distance of the true residual from the recurrence residual k_update left
// in r (its |r_rec|^2 is in sc.rec2), for the restart test.
template <typename T, int D, bool MS, int LEN, bool GRID = false>
__global__ void __launch_bounds__(kBlock) k_refresh(PcgArgs<T> a) {
    if (!*(volatile int *)&a.ctl->refresh_now) return;
    using A = Acc<T>;
    using AT = typename A::type;
    using SWt = SubWarp<T, D>;
    AT acc[3][SWt::V];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int k = 0; k < SWt::V; ++k) acc[q][k] = A::zero();
    PFE_ROW_LOOP_REPL(T, D, MS) {
        PFE_ROW_I;
        const int c0 = lm.cg * V;
        T ri[V], rr[V];
        ldv_rw<T, V>(a.r + i * D + c0, rr);
        true_residual<T, D, V, LEN, GRID>(a, i, c0, ri);
        const T dv = a.A.dinv[i];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            A::add_prod(acc[0][k], ri[k], dv * ri[k]);
            A::add_prod(acc[1][k], ri[k], ri[k]);
            const T dr = ri[k] - rr[k];
            A::add_prod(acc[2][k], dr, dr);
        }
        stv<T, V>(a.r + i * D + c0, ri);
    }
    __shared__ double tot[3 * D];
    if (grid_sum_cols<T, D, 3>(acc, a.part, bsg, &a.sc.ticket[bsg.seg * 4 + 3], tot)) {
        if (threadIdx.x < 32) {
            PcgCtl *ctl = a.ctl;
            for (int c = threadIdx.x; c < D; c += 32) {
                const int k = bsg.seg * D + c;
                const double rec = a.sc.rec2[k];
                a.sc.devr[k] = rec > 0.0 ? tot[2 * D + c] / rec : (tot[2 * D + c] > 0.0 ? INFINITY : 0.0);
            }
            __syncwarp();
            finish_seg(ctl, a.sc, bsg.seg, tot, tot + D, D, 1, ctl->iter);
            if (!MS || warp_last_segment(ctl, 3, a.sg.nseg)) {
                if (threadIdx.x == 0) {
                    ctl->refresh_now = 0;
                    ctl->xpending = 0;
                    ctl->xheld = 0;  // k_xflush applied every pending update
                    ctl->xfold = 0;
                    ctl->refresh_next = 0;
                    ctl->refresh_want = 0;
                    ctl->refreshes += 1;
                }
                __syncwarp();
                finish_all(ctl, a.sc, a.sg.nseg, D, a.cond, a.use_cond);
            }
        }
    }
}

// y = A x without dots (pfe_apply_A).
template <typename T, int D>
__global__ void __launch_bounds__(kBlock) k_apply(SysView<T> Av, const T *__restrict__ x, T *__restrict__ y) {
    struct {
        SysView<T> A;
        Segs sg;
        SegScal sc;
    } a{Av, Segs{1, Av.n, nullptr, nullptr}, SegScal{}};
    PFE_ROW_LOOP(T, D) {
        PFE_ROW_I;
        const int c0 = lm.cg * V;
        int64_t base;
        int len;
        sell_row(a.A.slice_ptr, a.A.row_len, i, base, len);
        T acc[V], xv[V];
        ldv<T, V>(x + i * D + c0, xv);
        const T ad = a.A.adiag[i];
#pragma unroll
        for (int k = 0; k < V; ++k) acc[k] = ad * xv[k];
        for (int s = 0; s < len; ++s) {
            const int64_t idx = base + s;
            const T av = a.A.aoff[idx];
            ldv<T, V>(x + (int64_t)a.A.col[idx] * D + c0, xv);
#pragma unroll
            for (int k = 0; k < V; ++k) acc[k] = fma(av, xv[k], acc[k]);
        }
        stv<T, V>(y + i * D + c0, acc);
    }
}

// ---- host side -----------------------------------------------------------------

template <typename T>
PcgArgs<T> pcg_args(pfe_ctx *c, PcgLaunch L) {
    PcgArgs<T> a;
    a.A = sys_view<T>(c);
    a.x = (T *)c->wk.Y;
    a.xlo = c->wk.Ylo;
    a.r = (T *)c->wk.R;
    a.p[0] = (T *)c->wk.Pd;
    a.p[1] = (T *)c->wk.Pd2;  // the direction buffers alternate between iterations
    a.q = (T *)c->wk.Q;
    a.b = (const T *)c->wk.RHS;
    a.part = c->wk.partials;
    a.ctl = c->ctl;
    a.sg = seg_view(c);
    a.sc = c->sc;
    a.cond = L.cond;
    a.use_cond = L.use_cond;
    a.if_pos = -1;
    a.grid_w = (c->kind == PFE_GRAPH_GRID && c->nseg == 1) ? (int)c->W : 0;
    a.t = (T *)c->fsai.t;
    a.r2[0] = a.r;
    a.r2[1] = (T *)c->fsai.r1;
    a.gdiag = nullptr;
    a.gslot = nullptr;
    if constexpr (std::is_same_v<T, float>) {
        a.gdiag = c->fsai.gdiag;
        a.gslot = c->fsai.gslot;
    }
    a.kb = c->fsai.kb;
    return a;
}

// blocks that cover every row group once / every vector of a flat traversal once
template <typename T, int D>
int64_t rows_need(const pfe_ctx *c) {
    const int64_t groups = (c->g.n + SubWarp<T, D>::RPW - 1) / SubWarp<T, D>::RPW;
    return (groups + kWarps - 1) / kWarps;
}
template <typename T, int D>
int64_t flat_need(const pfe_ctx *c) {
    return (c->g.n * D / Vec<T>::N + kBlock - 1) / kBlock;
}
// flat kernels that keep per-column state need (grid * kBlock * VEC) % D == 0
template <typename T, int D>
constexpr int flat_mult() {
    int a = D, b = kBlock * Vec<T>::N;
    while (b) {
        const int r = a % b;
        a = b;
        b = r;
    }
    return D / a;
}

// FSAI runs on the float path only (the FP64 path is the plain Jacobi reference)
template <typename T>
bool use_fsai(const pfe_ctx *c) {
    return std::is_same_v<T, float> && c->fsai.enabled;
}

// Launchers.  MS selects the batch (segment) variants of the Jacobi kernels;
// a single problem uses the MS = false ones, which carry no segment lookups.
template <typename T, int D, bool MS>
void init_ms(pfe_ctx *c, cudaStream_t s, const PcgArgs<T> &a) {
    k_pcg_init<T, D, 0, MS><<<wave_grid(c, G_INIT, k_pcg_init<T, D, 0, MS>, rows_need<T, D>(c)), kBlock, 0, s>>>(a);
}
// The replacement kernels of iteration `pos` of the loop body.  Capturing a
// graph with IF nodes (L.n_if > 0): a conditional IF node is appended to the
// capture of stream s (its value is set on the device by the kernel that
// decides the replacement) and its body is captured on the side stream, so
// ordinary iterations launch none of these kernels.  Otherwise they are
// launched on s and return at once outside replacement iterations.
static pfe_status if_begin(pfe_ctx *c, cudaStream_t s, const PcgLaunch &L, int pos, cudaStream_t &ks) {
    ks = s;
    if (L.n_if == 0) return PFE_OK;
    cudaStreamCaptureStatus cst;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    PFE_CUDA_TRY(c, cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, nullptr, &ndeps));
    if (cst != cudaStreamCaptureStatusActive) {
        c->err = "PCG loop body: the stream is not capturing";
        return PFE_ECUDA;
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = L.ifh[pos];
    cp.conditional.type = cudaGraphCondTypeIf;
    cp.conditional.size = 1;
    cudaGraphNode_t n;
    PFE_CUDA_TRY(c, cudaGraphAddNode(&n, g, deps, nullptr, ndeps, &cp));
    PFE_CUDA_TRY(c, cudaStreamUpdateCaptureDependencies(s, &n, nullptr, 1, cudaStreamSetCaptureDependencies));
    PFE_CUDA_TRY(c, cudaStreamBeginCaptureToGraph(L.side, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal));
    ks = L.side;
    return PFE_OK;
}
static pfe_status if_end(pfe_ctx *c, const PcgLaunch &L) {
    if (L.n_if == 0) return PFE_OK;
    PFE_CUDA_TRY(c, cudaGetLastError());
    cudaGraph_t g = nullptr;
    PFE_CUDA_TRY(c, cudaStreamEndCapture(L.side, &g));
    return PFE_OK;
}

// The replacement kernels with the compile-time row length of fixed-length
// layouts (12 or 28 slots), else the general slot loop.
// On one FP32 grid image the replacement residual computes the slot columns
// from the stencil (the same products in the same order as with the column
// array), so no per-iteration kernel of that path reads the column array.
template <typename T, int D, bool MS>
void launch_refresh(pfe_ctx *c, cudaStream_t s, const PcgArgs<T> &a) {
    if constexpr (!MS && std::is_same_v<T, float>) {
        if (a.grid_w > 0 && c->g.row_len == 12) {
            k_refresh<T, D, MS, 12, true><<<wave_grid(c, G_REFRESH, k_refresh<T, D, MS, 12, true>, rows_need<T, D>(c)),
                                            kBlock, 0, s>>>(a);
            return;
        }
        if (a.grid_w > 0 && c->g.row_len == 28) {
            k_refresh<T, D, MS, 28, true><<<wave_grid(c, G_REFRESH, k_refresh<T, D, MS, 28, true>, rows_need<T, D>(c)),
                                            kBlock, 0, s>>>(a);
            return;
        }
    }
    if (c->g.row_len == 12)
        k_refresh<T, D, MS, 12><<<wave_grid(c, G_REFRESH, k_refresh<T, D, MS, 12>, rows_need<T, D>(c)), kBlock, 0, s>>>(a);
    else if (c->g.row_len == 28)
        k_refresh<T, D, MS, 28><<<wave_grid(c, G_REFRESH, k_refresh<T, D, MS, 28>, rows_need<T, D>(c)), kBlock, 0, s>>>(a);
    else
        k_refresh<T, D, MS, 0><<<wave_grid(c, G_REFRESH, k_refresh<T, D, MS, 0>, rows_need<T, D>(c)), kBlock, 0, s>>>(a);
}
template <typename T, int D, bool MS = false>
void launch_refresh_f(pfe_ctx *c, cudaStream_t s, const PcgArgs<T> &a) {
    if constexpr (!MS) {
        if (a.grid_w > 0 && c->g.row_len == 12) {
            k_refresh_f<T, D, 12, MS, true><<<wave_grid(c, G_REFRESH_F, k_refresh_f<T, D, 12, MS, true>,
                                                        rows_need<T, D>(c)),
                                              kBlock, 0, s>>>(a);
            return;
        }
        if (a.grid_w > 0 && c->g.row_len == 28) {
            k_refresh_f<T, D, 28, MS, true><<<wave_grid(c, G_REFRESH_F, k_refresh_f<T, D, 28, MS, true>,
                                                        rows_need<T, D>(c)),
                                              kBlock, 0, s>>>(a);
            return;
        }
    }
    if (c->g.row_len == 12)
        k_refresh_f<T, D, 12, MS><<<wave_grid(c, G_REFRESH_F, k_refresh_f<T, D, 12, MS>, rows_need<T, D>(c)), kBlock, 0,
                                    s>>>(a);
    else if (c->g.row_len == 28)
        k_refresh_f<T, D, 28, MS><<<wave_grid(c, G_REFRESH_F, k_refresh_f<T, D, 28, MS>, rows_need<T, D>(c)), kBlock, 0,
                                    s>>>(a);
    else
        k_refresh_f<T, D, 0, MS><<<wave_grid(c, G_REFRESH_F, k_refresh_f<T, D, 0, MS>, rows_need<T, D>(c)), kBlock, 0,
                                   s>>>(a);
}

template <typename T, int D, bool MS>
pfe_status body_ms(pfe_ctx *c, cudaStream_t s, const PcgArgs<T> &a, const PcgLaunch &L, int u, cudaStream_t &ks) {
    k_pupdate<T, D, MS><<<wave_grid(c, G_PUPD, k_pupdate<T, D, MS>, flat_need<T, D>(c), flat_mult<T, D>()),
                             kBlock, 0, s>>>(a);
    launch_spmm<T, D, MS>(c, s, a);
    k_update<T, D, MS><<<wave_grid(c, G_UPDATE, k_update<T, D, MS>, rows_need<T, D>(c)), kBlock, 0, s>>>(a);
    PFE_TRY(if_begin(c, s, L, u, ks));
    k_xflush<T, D, MS><<<wave_grid(c, G_XFLUSH, k_xflush<T, D, MS>, flat_need<T, D>(c), flat_mult<T, D>()), kBlock, 0, ks>>>(a, 0, 1);
    launch_refresh<T, D, MS>(c, ks, a);
    return if_end(c, L);
}

// The FSAI kernels with the compile-time row length of the layout (FP32 grid
// graphs of radius 2 or 3; else the general kernels).
// which: 0 = k_fsai_tr, 1 = k_fsai_t (start of a solve), 2 = k_fsai_t (after a refresh), 3 = k_fsai_zp
template <typename T, int D, int LEN, bool GRID, bool MS>
void fsai_kernels_len(pfe_ctx *c, cudaStream_t s, const PcgArgs<T> &a, int which) {
    if (which == 0)
        k_fsai_tr<T, D, LEN, GRID, MS><<<wave_grid(c, G_FSAI_TR, k_fsai_tr<T, D, LEN, GRID, MS>, rows_need<T, D>(c)),
                                         kBlock, 0, s>>>(a);
    else if (which == 1)
        k_fsai_t<T, D, 0, LEN, GRID, MS><<<wave_grid(c, G_FSAI_T, k_fsai_t<T, D, 0, LEN, GRID, MS>, rows_need<T, D>(c)),
                                           kBlock, 0, s>>>(a);
    else if (which == 2)
        k_fsai_t<T, D, 1, LEN, GRID, MS><<<wave_grid(c, G_FSAI_T1, k_fsai_t<T, D, 1, LEN, GRID, MS>,
                                                     rows_need<T, D>(c)),
                                           kBlock, 0, s>>>(a);
    else
        k_fsai_zp<T, D, LEN, GRID, MS><<<wave_grid(c, G_FSAI_ZP, k_fsai_zp<T, D, LEN, GRID, MS>, rows_need<T, D>(c)),
                                         kBlock, 0, s>>>(a);
}
// The FSAI kernels on fixed-length rows (12 or 28 slots): slot columns loaded
// (PFE_FSAI_SLOTS) or, on one grid image, computed from the stencil
// (PFE_FSAI_STENCIL; the context's choice, made by pfe_autotune).  A batch
// (MS) reads the slot columns.
template <typename T, int D, bool MS = false>
void launch_fsai(pfe_ctx *c, cudaStream_t s, const PcgArgs<T> &a, int which) {
    const bool grid = !MS && c->fsai_variant == PFE_FSAI_STENCIL && a.grid_w > 0;
    if (c->g.row_len == 12) {
        if (grid)
            fsai_kernels_len<T, D, 12, true, false>(c, s, a, which);
        else
            fsai_kernels_len<T, D, 12, false, MS>(c, s, a, which);
    } else if (c->g.row_len == 28) {
        if (grid)
            fsai_kernels_len<T, D, 28, true, false>(c, s, a, which);
        else
            fsai_kernels_len<T, D, 28, false, MS>(c, s, a, which);
    } else {
        fsai_kernels_len<T, D, 0, false, MS>(c, s, a, which);
    }
}

// The IC(0) triangular solves: one launch per level of the raster wavefront
// (forward: levels ascending into t; backward: descending, z in place).
template <typename T, int D, int LEN>
void ic_solve_len(pfe_ctx *c, cudaStream_t s, const PcgArgs<T> &a, bool fwd, int start) {
    constexpr int cl = ic_level_coef<LEN>();
    const int64_t W = c->W, H = c->g.n / W, L = ic_levels(W, H, cl);
    for (int64_t q = 0; q < L; ++q) {
        const int64_t l = fwd ? q : L - 1 - q;
        int64_t y0 = 0, rows = 0;
        ic_level_rows(l, W, H, cl, y0, rows);
        if (rows == 0) continue;
        const unsigned g = (unsigned)((rows * D + kBlock - 1) / kBlock);
        if (fwd)
            k_ic_fwd<T, D, LEN><<<g, kBlock, 0, s>>>(a, l, y0, rows, start);
        else
            k_ic_bwd<T, D, LEN><<<g, kBlock, 0, s>>>(a, l, y0, rows);
    }
}
template <typename T, int D>
void ic_solve(pfe_ctx *c, cudaStream_t s, const PcgArgs<T> &a, bool fwd, int start) {
    if (c->g.row_len == 12)
        ic_solve_len<T, D, 12>(c, s, a, fwd, start);
    else
        ic_solve_len<T, D, 28>(c, s, a, fwd, start);
}

// One FSAI iteration of the loop body (position u of iters): q = A p, r -=
// alpha q with t = G r, the replacement kernels (IF node), z = G^T t with the
// direction and solution updates.
template <typename T, int D, bool MS>
pfe_status fsai_iter(pfe_ctx *c, cudaStream_t s, const PcgArgs<T> &a, const PcgLaunch &L, int u, int iters,
                     cudaStream_t &ks) {
    launch_spmm<T, D, MS>(c, s, a);
    launch_fsai<T, D, MS>(c, s, a, 0);
    PFE_TRY(if_begin(c, s, L, u, ks));
    k_xflush<T, D, MS><<<wave_grid(c, G_XFLUSH, k_xflush<T, D, MS>, flat_need<T, D>(c), flat_mult<T, D>()), kBlock, 0,
                         ks>>>(a, 0, 0);
    launch_refresh_f<T, D, MS>(c, ks, a);
    launch_fsai<T, D, MS>(c, ks, a, 2);
    PFE_TRY(if_end(c, L));
    PcgArgs<T> az = a;
    az.if_pos = L.n_if > 0 ? (u + 1) % iters : -1;  // decides the next iteration's replacement
    launch_fsai<T, D, MS>(c, s, az, 3);
    return PFE_OK;
}

template <typename T, int D>
pfe_status init_T(pfe_ctx *c, cudaStream_t s, PcgLaunch L) {
    PcgArgs<T> a = pcg_args<T>(c, L);
    // the error flag of the solve starts clear (the segments' finishers only raise it)
    PFE_CUDA_TRY(c, cudaMemsetAsync(&c->ctl->error, 0, sizeof(int), s));
    if constexpr (std::is_same_v<T, float>) {
        if (use_fsai<T>(c) && c->fsai.ic) {
            k_pcg_init<T, D, 1, false><<<wave_grid(c, G_INIT_F, k_pcg_init<T, D, 1, false>, rows_need<T, D>(c)), kBlock,
                                         0, s>>>(a);
            ic_solve<T, D>(c, s, a, true, 1);
            PcgArgs<T> ad = a;
            ad.if_pos = L.n_if > 0 ? 0 : -1;  // decides the replacement of the body's first iteration
            k_ic_dots<T, D><<<wave_grid(c, G_IC_DOTS, k_ic_dots<T, D>, rows_need<T, D>(c)), kBlock, 0, s>>>(ad, 1);
            ic_solve<T, D>(c, s, a, false, 0);
            PFE_CUDA_TRY(c, cudaGetLastError());
            return PFE_OK;
        }
        if (use_fsai<T>(c)) {
            PcgArgs<T> az = a;
            az.if_pos = L.n_if > 0 ? 0 : -1;  // decides the replacement of the body's first iteration
            if (c->nseg > 1) {
                k_pcg_init<T, D, 1, true><<<wave_grid(c, G_INIT_F, k_pcg_init<T, D, 1, true>, rows_need<T, D>(c)),
                                            kBlock, 0, s>>>(a);
                launch_fsai<T, D, true>(c, s, a, 1);
                launch_fsai<T, D, true>(c, s, az, 3);
            } else {
                k_pcg_init<T, D, 1, false><<<wave_grid(c, G_INIT_F, k_pcg_init<T, D, 1, false>, rows_need<T, D>(c)),
                                             kBlock, 0, s>>>(a);
                launch_fsai<T, D>(c, s, a, 1);
                launch_fsai<T, D>(c, s, az, 3);
            }
            PFE_CUDA_TRY(c, cudaGetLastError());
            return PFE_OK;
        }
    }
    if (c->nseg > 1)
        init_ms<T, D, true>(c, s, a);
    else
        init_ms<T, D, false>(c, s, a);
    PFE_CUDA_TRY(c, cudaGetLastError());
    return PFE_OK;
}

template <typename T, int D>
pfe_status body_T(pfe_ctx *c, cudaStream_t s, PcgLaunch L, int iters) {
    PcgArgs<T> a = pcg_args<T>(c, L);
    cudaStream_t ks = s;
    if constexpr (std::is_same_v<T, float>) {
        if (use_fsai<T>(c) && c->fsai.ic) {
            for (int u = 0; u < iters; ++u) {
                launch_spmm<T, D, false>(c, s, a);
                k_ic_r<T, D><<<wave_grid(c, G_IC_R, k_ic_r<T, D>, flat_need<T, D>(c)), kBlock, 0, s>>>(a);
                PFE_TRY(if_begin(c, s, L, u, ks));
                k_xflush<T, D, false><<<wave_grid(c, G_XFLUSH, k_xflush<T, D, false>, flat_need<T, D>(c), flat_mult<T, D>()), kBlock, 0,
                                        ks>>>(a, 0, 0);
                launch_refresh_f<T, D>(c, ks, a);
                PFE_TRY(if_end(c, L));
                ic_solve<T, D>(c, s, a, true, 0);
                PcgArgs<T> ad = a;
                ad.if_pos = L.n_if > 0 ? (u + 1) % iters : -1;  // decides the next iteration's replacement
                k_ic_dots<T, D><<<wave_grid(c, G_IC_DOTS, k_ic_dots<T, D>, rows_need<T, D>(c)), kBlock, 0, s>>>(ad, 0);
                ic_solve<T, D>(c, s, a, false, 0);
            }
            PFE_CUDA_TRY(c, cudaGetLastError());
            return PFE_OK;
        }
        if (use_fsai<T>(c)) {
            for (int u = 0; u < iters; ++u) {
                if (c->nseg > 1)
                    PFE_TRY((fsai_iter<T, D, true>(c, s, a, L, u, iters, ks)));
                else
                    PFE_TRY((fsai_iter<T, D, false>(c, s, a, L, u, iters, ks)));
            }
            PFE_CUDA_TRY(c, cudaGetLastError());
            return PFE_OK;
        }
    }
    for (int u = 0; u < iters; ++u) {
        PcgArgs<T> au = a;
        au.if_pos = L.n_if > 0 ? u : -1;  // k_update decides this iteration's replacement
        if (c->nseg > 1)
            PFE_TRY((body_ms<T, D, true>(c, s, au, L, u, ks)));
        else
            PFE_TRY((body_ms<T, D, false>(c, s, au, L, u, ks)));
    }
    PFE_CUDA_TRY(c, cudaGetLastError());
    return PFE_OK;
}

template <typename T, int D>
pfe_status final_T(pfe_ctx *c, cudaStream_t s, PcgLaunch L) {
    if (c->nseg > 1)
        k_xflush<T, D, true><<<wave_grid(c, G_XFLUSH, k_xflush<T, D, true>, flat_need<T, D>(c), flat_mult<T, D>()), kBlock, 0, s>>>(
            pcg_args<T>(c, L), 1, 1);
    else
        k_xflush<T, D, false><<<wave_grid(c, G_XFLUSH, k_xflush<T, D, false>, flat_need<T, D>(c), flat_mult<T, D>()), kBlock, 0, s>>>(
            pcg_args<T>(c, L), 1, 1);
    PFE_CUDA_TRY(c, cudaGetLastError());
    return PFE_OK;
}

template <typename T, int D>
pfe_status apply_T(pfe_ctx *c, cudaStream_t s, const void *x, void *y) {
    k_apply<T, D><<<wave_grid(c, G_APPLY, k_apply<T, D>, rows_need<T, D>(c)), kBlock, 0, s>>>(sys_view<T>(c), (const T *)x, (T *)y);
    PFE_CUDA_TRY(c, cudaGetLastError());
    return PFE_OK;
}

// Average duration of `reps` back-to-back launches of one PCG kernel on the
// current vectors, bracketed by CUDA events on stream s.  Uses a scratch
// control block (every column active, a steady-state iteration: direction
// update and delayed solution update both on) and scratch copies of y, r and
// the direction buffers, so the iteration state is left as it was.
// which: 0 = k_spmm, 1 = k_update, 2 = k_pupdate folding two solution
// updates, 3 = k_fsai_tr, 4 = k_fsai_zp folding, 5 = k_fsai_zp holding one,
// 6 = k_pupdate holding; on a replacement iteration: 7 = the replacement
// residual (k_refresh, or k_refresh_f with an FSAI factor), 8 = k_xflush
// applying two pending solution updates, 9 = k_fsai_t (t = G r with the dots).
template <typename T, int D>
pfe_status time_T(pfe_ctx *c, cudaStream_t s, int which, int reps, float *ms, int variant) {
    PcgCtl h;
    memset(&h, 0, sizeof(h));
    h.max_iter = 1 << 30;
    h.ncols = D;
    h.tol = 0.0;
    h.p_ready = 0;
    h.xpending = 1;
    h.xfold = (which == 2 || which == 4) ? 1 : 0;  // 2, 4: the folding launch; 5, 6: the holding one
    h.xheld = which == 8 ? 1 : 0;
    h.refresh_now = which >= 7 ? 1 : 0;
    h.refresh = 1 << 30;  // residual replacement on (confirmation logic), never periodic
    // scratch per-segment scalars: every column active
    const int nseg = c->nseg;
    const size_t sc_bytes = segscal_bytes(nseg, D);
    std::vector<unsigned char> hsc(sc_bytes, 0);
    {
        SegScal hs = segscal_carve(hsc.data(), nseg, D);
        for (int k = 0; k < nseg * D; ++k) {
            hs.active[k] = 1;
            hs.rz[k] = 1.0;
            hs.bnorm[k] = 1.0;
            hs.alpha[k] = 1e-30;
            hs.beta[k] = 0.5;
        }
        for (int q = 0; q < nseg; ++q) hs.seg_active[q] = hs.seg_live[q] = 1;
    }
    void *dsc = nullptr;
    const int64_t nd = c->g.n * (int64_t)D;
    const bool fsai = (which >= 3 && which <= 5) || which == 9 || (which == 7 && use_fsai<T>(c) && !c->fsai.ic);
    if (fsai && (!use_fsai<T>(c) || c->fsai.ic)) {
        c->err = "pfe_time_kernel: the FSAI kernels need the FSAI preconditioner on the mixed path";
        return PFE_EUNSUPPORTED;
    }
    PcgCtl *dctl = nullptr;
    T *xs = nullptr, *rs = nullptr, *p0 = nullptr, *p1 = nullptr, *r1s = nullptr, *ts = nullptr;
    float *xls = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    pfe_status st = PFE_OK;
    auto cleanup = [&]() {
        for (void *q : {(void *)dctl, (void *)xs, (void *)rs, (void *)p0, (void *)p1, (void *)xls, (void *)r1s,
                        (void *)ts, dsc})
            if (q) cudaFree(q);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (cudaMalloc((void **)&dctl, sizeof(PcgCtl)) != cudaSuccess || cudaMalloc(&dsc, sc_bytes) != cudaSuccess ||
        cudaMalloc((void **)&xs, nd * sizeof(T)) != cudaSuccess ||
        cudaMalloc((void **)&rs, nd * sizeof(T)) != cudaSuccess || cudaMalloc((void **)&p0, nd * sizeof(T)) != cudaSuccess ||
        cudaMalloc((void **)&p1, nd * sizeof(T)) != cudaSuccess ||
        (std::is_same_v<T, float> && cudaMalloc((void **)&xls, nd * sizeof(float)) != cudaSuccess) ||
        (fsai && (cudaMalloc((void **)&r1s, nd * sizeof(T)) != cudaSuccess ||
                  cudaMalloc((void **)&ts, nd * sizeof(T)) != cudaSuccess))) {
        cudaGetLastError();
        cleanup();
        c->err = "pfe_time_kernel: scratch allocation failed";
        return PFE_ENOMEM;
    }
    PcgArgs<T> a = pcg_args<T>(c, PcgLaunch{0, 0});
    a.ctl = dctl;
    a.sc = segscal_carve(dsc, nseg, D);
    a.x = xs;
    a.r = rs;
    a.xlo = xls;
    a.p[0] = p0;
    a.p[1] = p1;
    a.r2[0] = rs;
    a.r2[1] = r1s;
    a.t = ts;
    cudaMemcpyAsync(dctl, &h, sizeof(h), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dsc, hsc.data(), sc_bytes, cudaMemcpyHostToDevice, s);
    if (fsai) {
        cudaMemcpyAsync(r1s, c->wk.R, nd * sizeof(T), cudaMemcpyDeviceToDevice, s);
        cudaMemcpyAsync(ts, c->wk.R, nd * sizeof(T), cudaMemcpyDeviceToDevice, s);
    }
    cudaMemcpyAsync(xs, c->wk.Y, nd * sizeof(T), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(rs, c->wk.R, nd * sizeof(T), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(p0, c->wk.Pd, nd * sizeof(T), cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(p1, c->wk.Pd, nd * sizeof(T), cudaMemcpyDeviceToDevice, s);
    if (xls) cudaMemcpyAsync(xls, c->wk.Ylo, nd * sizeof(float), cudaMemcpyDeviceToDevice, s);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const bool multi = c->nseg > 1;
    auto launch = [&]() {
        if (which == 0 && multi)
            launch_spmm<T, D, true>(c, s, a, variant);
        else if (which == 0)
            launch_spmm<T, D, false>(c, s, a, variant);
        else if (which == 1 && multi)
            k_update<T, D, true><<<wave_grid(c, G_UPDATE, k_update<T, D, true>, rows_need<T, D>(c)), kBlock, 0, s>>>(a);
        else if (which == 1)
            k_update<T, D, false><<<wave_grid(c, G_UPDATE, k_update<T, D, false>, rows_need<T, D>(c)), kBlock, 0, s>>>(a);
        else if ((which == 2 || which == 6) && multi)
            k_pupdate<T, D, true><<<wave_grid(c, G_PUPD, k_pupdate<T, D, true>, flat_need<T, D>(c),
                                                 flat_mult<T, D>()),
                                       kBlock, 0, s>>>(a);
        else if (which == 2 || which == 6)
            k_pupdate<T, D, false><<<wave_grid(c, G_PUPD, k_pupdate<T, D, false>, flat_need<T, D>(c),
                                                  flat_mult<T, D>()),
                                        kBlock, 0, s>>>(a);
        else if (which == 7 && !fsai) {
            // k_refresh's finisher ends the replacement: mark the next launch as one again
            cudaMemsetAsync(&dctl->refresh_now, 1, sizeof(int), s);
            if (multi)
                launch_refresh<T, D, true>(c, s, a);
            else
                launch_refresh<T, D, false>(c, s, a);
        } else if (which == 8 && multi)
            k_xflush<T, D, true><<<wave_grid(c, G_XFLUSH, k_xflush<T, D, true>, flat_need<T, D>(c), flat_mult<T, D>()),
                                   kBlock, 0, s>>>(a, 0, 0);
        else if (which == 8)
            k_xflush<T, D, false><<<wave_grid(c, G_XFLUSH, k_xflush<T, D, false>, flat_need<T, D>(c),
                                                 flat_mult<T, D>()),
                                       kBlock, 0, s>>>(a, 0, 0);
        else if constexpr (std::is_same_v<T, float>) {
            const int kf = which == 3 ? 0 : which == 9 ? 2 : 3;  // 4, 5: k_fsai_zp
            if (which == 7 && multi)
                launch_refresh_f<T, D, true>(c, s, a);
            else if (which == 7)
                launch_refresh_f<T, D>(c, s, a);
            else if (multi)
                launch_fsai<T, D, true>(c, s, a, kf);
            else
                launch_fsai<T, D>(c, s, a, kf);
        }
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

#define PFE_INSTANTIATE(T, D)                                                                        \
    template pfe_status pfe::pcgk::init_T<T, D>(pfe_ctx *, cudaStream_t, pfe::PcgLaunch);          \
    template pfe_status pfe::pcgk::body_T<T, D>(pfe_ctx *, cudaStream_t, pfe::PcgLaunch, int);     \
    template pfe_status pfe::pcgk::final_T<T, D>(pfe_ctx *, cudaStream_t, pfe::PcgLaunch);         \
    template pfe_status pfe::pcgk::apply_T<T, D>(pfe_ctx *, cudaStream_t, const void *, void *);     \
    template pfe_status pfe::pcgk::time_T<T, D>(pfe_ctx *, cudaStream_t, int, int, float *, int);
