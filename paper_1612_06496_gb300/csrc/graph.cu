// Graph construction on the device (Sec. II heat kernel and degree matrix,
// Sec. II edge operator M, Eq. 13 system matrix A = lambda M^T M + r D).
//
// Layout: SELL-32, row-major within a slice.  Rows are taken 32 at a time;
// slice s stores each row's off-diagonal entries contiguously, padded to the
// slice's longest row rounded up to 4 slots, so that a row's slots are read
// with 16-byte vector loads.  Grid graphs use fixed positions: slot t of
// every row is stencil offset t (a padding slot -- column i, weight 0, edge
// id -1 -- where the offset leaves the image), so every row has the same
// length and a kernel finds row i's slots at i * K without a slice lookup.  Undirected edges (i < j) are stored in a second
// sliced layout over their first endpoint; the split-Bregman edge state b
// (Alg. 2) is indexed by that edge slot.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace pfe {
namespace {

constexpr int kMaxOffsets = 256;

struct Offsets {
    int K;  // total offsets; the first K/2 point backwards, the last K/2 forwards
    int dx[kMaxOffsets], dy[kMaxOffsets];
};

__device__ __forceinline__ double heat_weight(const double *__restrict__ X, int m, int64_t a, int64_t b,
                                              double inv2s2) {
    // w_ab = exp(-|x_a - x_b|^2 / (2 sigma^2)), always evaluated with a < b
    double s = 0.0;
    for (int t = 0; t < m; ++t) {
        double df = X[a * m + t] - X[b * m + t];
        s = fma(df, df, s);
    }
    return exp(-s * inv2s2);
}

// ---- grid graphs --------------------------------------------------------

// Images of a grid graph: image s has H = h[s], W = w[s] and its pixels are
// vertices off[s] .. off[s+1]-1 (one image: nseg = 1, off = {0, n}).
struct GridSegs {
    int nseg;
    const int64_t *off;
    const int *h, *w;
    const int *rseg;
};
__device__ __forceinline__ void grid_pos(const GridSegs &gs, int64_t i, int64_t &vo, int &H, int &W, int &x, int &y) {
    const int s = gs.nseg == 1 ? 0 : gs.rseg[i];
    vo = gs.off[s];
    H = gs.h[s];
    W = gs.w[s];
    const int64_t li = i - vo;
    x = (int)(li % W);
    y = (int)(li / W);
}

__global__ void k_grid_count(int64_t n, int64_t n_slices, GridSegs gs, Offsets off, int *nf_row,
                             int *slice_len, int *fslice_len) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((i >> 5) >= n_slices) return;  // whole warps only
    int nb = 0, nf = 0;
    if (i < n) {
        int64_t vo;
        int H, W, x, y;
        grid_pos(gs, i, vo, H, W, x, y);
        for (int t = 0; t < off.K; ++t) {
            int x2 = x + off.dx[t], y2 = y + off.dy[t];
            if (x2 >= 0 && x2 < W && y2 >= 0 && y2 < H) {
                ++nb;
                if (t >= off.K / 2) ++nf;
            }
        }
        nf_row[i] = nf;
    }
    (void)nb;
    if ((threadIdx.x & 31) == 0) {
        int64_t s = i >> 5;
        // fixed positions: slot t of every row is stencil offset t (K is a
        // multiple of 4: the offsets come in orbits of the 90-degree rotation),
        // and so is the Bregman slot of each forward edge: forward offset t of
        // row i owns b slot i K/2 + (t - K/2) (a slot whose offset leaves the
        // image is unused), so a kernel finds any edge's b slot from the
        // stencil alone
        slice_len[s] = off.K * 32;
        fslice_len[s] = (off.K / 2) * 32;
    }
}

__global__ void k_grid_fill(int64_t n, int64_t n_slices, GridSegs gs, Offsets off, const int64_t *slice_ptr,
                            const int64_t *fslice_ptr, const int64_t *fw_off, const double *__restrict__ X,
                            int m, double inv2s2, int *col, int *eid, double *w64, int *ext_slot, int *ea,
                            int *eb, double *ew, double *deg, double *deg2) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t s = i >> 5;
    if (s >= n_slices) return;
    int lane = (int)(i & 31);
    const int len = (int)((slice_ptr[s + 1] - slice_ptr[s]) >> 5);
    const int64_t base = slice_ptr[s] + (int64_t)lane * len;  // row-major within the slice
    const int flen = (int)((fslice_ptr[s + 1] - fslice_ptr[s]) >> 5);
    int k = 0;
    if (i < n) {
        int64_t vo;
        int H, W, x, y;
        grid_pos(gs, i, vo, H, W, x, y);
        int kf = 0;
        double sw = 0.0, sw2 = 0.0;
        for (int t = 0; t < off.K; ++t) {
            int x2 = x + off.dx[t], y2 = y + off.dy[t];
            int64_t idx = base + t;
            if (x2 < 0 || x2 >= W || y2 < 0 || y2 >= H) {  // off the image: padding slot
                col[idx] = (int)i;
                eid[idx] = -1;
                w64[idx] = 0.0;
                continue;
            }
            int64_t j = vo + (int64_t)y2 * W + x2;
            double w = (j > i) ? heat_weight(X, m, i, j, inv2s2) : heat_weight(X, m, j, i, inv2s2);
            int e;
            if (t >= off.K / 2) {  // forward: i owns the edge, at its slot for offset t
                e = (int)(fslice_ptr[s] + (int64_t)lane * flen + (t - off.K / 2));
                int64_t ext = fw_off[i] + kf;  // external numbering: i's valid forward edges in order
                ext_slot[ext] = e;
                ea[ext] = (int)i;
                eb[ext] = (int)j;
                ew[ext] = w;
                ++kf;
            } else {  // backward: j owns it, at j's slot for the reverse offset
                const int tr = off.K - 1 - t;  // index of the reverse offset
                const int64_t sj = j >> 5;
                const int flj = (int)((fslice_ptr[sj + 1] - fslice_ptr[sj]) >> 5);
                e = (int)(fslice_ptr[sj] + (int64_t)(j & 31) * flj + (tr - off.K / 2));
            }
            col[idx] = (int)j;
            eid[idx] = e;
            w64[idx] = w;
            sw += w;
            sw2 = fma(w, w, sw2);
        }
        deg[i] = sw;
        deg2[i] = sw2;
        k = off.K;
    }
    for (; k < len; ++k) {  // rows past n in the last slice
        int64_t idx = base + k;
        col[idx] = (i < n) ? (int)i : 0;
        eid[idx] = -1;
        w64[idx] = 0.0;
    }
}

// ---- edge-list graphs ---------------------------------------------------

__global__ void k_edges_count(int64_t n, int64_t ne, const int32_t *ei, const int32_t *ej, int *nb_row,
                              int *nf_row, int *err) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ne) return;
    int64_t u = ei[k], v = ej[k];
    if (u < 0 || v < 0 || u >= n || v >= n || u == v) {
        atomicExch(err, 1);
        return;
    }
    int64_t a = u < v ? u : v, b = u < v ? v : u;
    atomicAdd(nb_row + a, 1);
    atomicAdd(nb_row + b, 1);
    atomicAdd(nf_row + a, 1);
}

__global__ void k_slice_max(int64_t n, int64_t n_slices, const int *nb_row, const int *nf_row, int *slice_len,
                            int *fslice_len) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((i >> 5) >= n_slices) return;  // whole warps only
    int nb = i < n ? nb_row[i] : 0, nf = i < n ? nf_row[i] : 0;
    int mb = __reduce_max_sync(0xffffffffu, nb);
    int mf = __reduce_max_sync(0xffffffffu, nf);
    if ((threadIdx.x & 31) == 0) {
        slice_len[i >> 5] = ((mb + 3) & ~3) * 32;  // row length padded to a multiple of 4 slots
        fslice_len[i >> 5] = mf * 32;
    }
}

__global__ void k_edges_scatter(int64_t ne, const int32_t *ei, const int32_t *ej, const int64_t *slice_ptr,
                                int *cursor, int *col, int *tmp_ext) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ne) return;
    int64_t u = ei[k], v = ej[k];
    int64_t a = u < v ? u : v, b = u < v ? v : u;
    int pa = atomicAdd(cursor + a, 1);
    const int la = (int)((slice_ptr[(a >> 5) + 1] - slice_ptr[a >> 5]) >> 5);
    int64_t ia = slice_ptr[a >> 5] + (int64_t)(a & 31) * la + pa;
    col[ia] = (int)b;
    tmp_ext[ia] = (int)k;
    int pb = atomicAdd(cursor + b, 1);
    const int lb = (int)((slice_ptr[(b >> 5) + 1] - slice_ptr[b >> 5]) >> 5);
    int64_t ib = slice_ptr[b >> 5] + (int64_t)(b & 31) * lb + pb;
    col[ib] = (int)a;
    tmp_ext[ib] = (int)k;
}

// Sort each row by column (insertion sort; rows are short), reject duplicate
// pairs, number the forward edges and pad.
__global__ void k_edges_sort(int64_t n, int64_t n_slices, const int64_t *slice_ptr, const int64_t *fslice_ptr, const int *nb_row,
                             int *col, int *tmp_ext, int *eid, int *ext_slot, int *ea, int *eb, int *err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t s = i >> 5;
    if (s >= n_slices) return;
    int lane = (int)(i & 31);
    const int len = (int)((slice_ptr[s + 1] - slice_ptr[s]) >> 5);
    const int64_t base = slice_ptr[s] + (int64_t)lane * len;
    const int flen = (int)((fslice_ptr[s + 1] - fslice_ptr[s]) >> 5);
    int nb = i < n ? nb_row[i] : 0;
    for (int a = 1; a < nb; ++a) {
        int64_t ia = base + a;
        int ca = col[ia], xa = tmp_ext[ia];
        int b = a - 1;
        while (b >= 0) {
            int64_t ib = base + b;
            int cb = col[ib];
            if (cb <= ca) break;
            int64_t ib1 = ib + 1;
            col[ib1] = cb;
            tmp_ext[ib1] = tmp_ext[ib];
            --b;
        }
        int64_t ib1 = base + (b + 1);
        col[ib1] = ca;
        tmp_ext[ib1] = xa;
    }
    int kf = 0, prev = -1;
    for (int k = 0; k < nb; ++k) {
        int64_t idx = base + k;
        int j = col[idx];
        if (j == prev) atomicExch(err, 2);
        prev = j;
        if (j > i) {
            int e = (int)(fslice_ptr[s] + (int64_t)lane * flen + kf);
            int ext = tmp_ext[idx];
            ext_slot[ext] = e;
            ea[ext] = (int)i;
            eb[ext] = j;
            eid[idx] = e;
            ++kf;
        } else {
            eid[idx] = -2;  // resolved by k_edges_backward
        }
    }
    for (int k = nb; k < len; ++k) {
        int64_t idx = base + k;
        col[idx] = i < n ? (int)i : 0;
        eid[idx] = -1;
        tmp_ext[idx] = -1;
    }
}

__global__ void k_edges_backward(int64_t n, const int64_t *slice_ptr, const int *nb_row, const int *tmp_ext,
                                 const int *ext_slot, int *eid, const int *col, const double *__restrict__ X,
                                 int m, double inv2s2, double *w64, double *ew, double *deg, double *deg2) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t s = i >> 5;
    int lane = (int)(i & 31);
    const int len = (int)((slice_ptr[s + 1] - slice_ptr[s]) >> 5);
    const int64_t base = slice_ptr[s] + (int64_t)lane * len;
    int nb = nb_row[i];
    double sw = 0.0, sw2 = 0.0;
    for (int k = 0; k < nb; ++k) {
        int64_t idx = base + k;
        int j = col[idx];
        if (eid[idx] == -2) eid[idx] = ext_slot[tmp_ext[idx]];
        double w = (j > i) ? heat_weight(X, m, i, j, inv2s2) : heat_weight(X, m, j, i, inv2s2);
        if (j > i) ew[tmp_ext[idx]] = w;
        w64[idx] = w;
        sw += w;
        sw2 = fma(w, w, sw2);
    }
    for (int k = nb; k < len; ++k) w64[base + k] = 0.0;
    deg[i] = sw;
    deg2[i] = sw2;
}

// ---- shared -------------------------------------------------------------

// exclusive scan of int32 counts into int64 offsets (out has n + 1 entries)
__global__ void k_scan_block(int64_t n, const int *in, const int64_t *in64, int64_t *out, int64_t *block_sum) {
    __shared__ int64_t wsum[32];
    int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    int64_t v = 0;
    if (i < n) v = in ? (int64_t)in[i] : in64[i];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = wsum[lane];
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    int64_t incl = x + (warp > 0 ? wsum[warp - 1] : 0);
    if (i < n) out[i] = incl - v;
    if (threadIdx.x == 1023) block_sum[blockIdx.x] = incl;
}

__global__ void k_scan_add(int64_t n, int64_t *out, const int64_t *block_off) {
    int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
    if (i < n) out[i] += block_off[blockIdx.x];
}

__global__ void k_sum_f64(int64_t n, const double *v, double *partials, unsigned *ticket, double *result) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += v[i];
    double tmp[1] = {s};
    block_reduce<double, 1>(tmp, partials + blockIdx.x);
    if (last_block_arrives(ticket)) {
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b) t += ld_cg(partials + b);
            *result = t;
            *ticket = 0;
        }
    }
}

__global__ void k_values_slots(int64_t slots, double lam, const double *w64, float *w32, double *aoff64,
                               float *aoff32) {
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= slots) return;
    double w = w64[k];
    double a = -lam * (w * w);
    w32[k] = (float)w;
    aoff64[k] = a;
    aoff32[k] = (float)a;
}

__global__ void k_values_rows(int64_t n, double lam, double r, const double *deg, const double *deg2,
                              double *sqrtdeg, double *adiag64, float *adiag32, double *dinv64, float *dinv32,
                              int *err) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double d = deg[i];
    if (!(d > 0.0)) atomicExch(err, 3);
    double a = lam * deg2[i] + r * d;
    sqrtdeg[i] = sqrt(d);
    adiag64[i] = a;
    adiag32[i] = (float)a;
    dinv64[i] = 1.0 / a;
    dinv32[i] = (float)(1.0 / a);
}

// FP32 low parts of A's values: a = hi + lo with hi = the FP32 value the
// iteration multiplies by and lo = FP32(a - hi), so the residual replacement
// of the FP32 path works with A's FP64 values in FP32 arithmetic.
__global__ void k_values_lo(int64_t count, const double *a64, const float *a32, float *lo32) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    lo32[k] = (float)(a64[k] - (double)a32[k]);
}

// Segment of each row (binary search over the offsets).
__global__ void k_fill_rseg(int64_t n, int nseg, const int64_t *off, int *rseg) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    rseg[i] = lo;
}

// vol_s = sum of d_i over segment s: one block per segment, fixed order.
__global__ void k_seg_sum(const int64_t *off, const double *v, double *out) {
    const int s = blockIdx.x;
    double acc = 0.0;
    for (int64_t i = off[s] + threadIdx.x; i < off[s + 1]; i += blockDim.x) acc += v[i];
    double tmp[1] = {acc};
    __shared__ double res[1];
    block_reduce<double, 1>(tmp, res);
    if (threadIdx.x == 0) out[s] = res[0];
}

// Slot and row values of A with the lambda of each row's segment (batch).
__global__ void k_values_seg(int64_t n, int64_t n_slices, const int *slice_ptr, const int *rseg,
                             const double *seg_lam, double r, const double *w64, float *w32, double *aoff64,
                             float *aoff32, const double *deg, const double *deg2, double *sqrtdeg, double *adiag64,
                             float *adiag32, double *dinv64, float *dinv32, int *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t s = i >> 5;
    if (s >= n_slices) return;
    const double lam = i < n ? seg_lam[rseg[i]] : 0.0;
    const int len = (slice_ptr[s + 1] - slice_ptr[s]) >> 5;
    const int64_t base = (int64_t)slice_ptr[s] + (i & 31) * (int64_t)len;
    for (int k = 0; k < len; ++k) {
        const double w = w64[base + k];
        const double av = -lam * (w * w);
        w32[base + k] = (float)w;
        aoff64[base + k] = av;
        aoff32[base + k] = (float)av;
    }
    if (i >= n) return;
    const double d = deg[i];
    if (!(d > 0.0)) atomicExch(err, 3);
    const double a = lam * deg2[i] + r * d;
    sqrtdeg[i] = sqrt(d);
    adiag64[i] = a;
    adiag32[i] = (float)a;
    dinv64[i] = 1.0 / a;
    dinv32[i] = (float)(1.0 / a);
}

template <typename P>
pfe_status dalloc(pfe_ctx *c, P **p, int64_t count) {
    size_t bytes = (size_t)std::max<int64_t>(count, 1) * sizeof(P);
    if (over_device_cap(c, bytes)) return PFE_ENOMEM;
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e != cudaSuccess) {
        c->err = std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e);
        cudaGetLastError();
        return PFE_ENOMEM;
    }
    c->dev_allocs.push_back(*p);
    c->bytes += (int64_t)bytes;
    return PFE_OK;
}

// temporary device buffer freed at scope exit
struct Tmp {
    void *p = nullptr;
    ~Tmp() {
        if (p) cudaFree(p);
    }
};
template <typename P>
pfe_status talloc(pfe_ctx *c, Tmp &t, P **p, int64_t count) {
    size_t bytes = (size_t)std::max<int64_t>(count, 1) * sizeof(P);
    cudaError_t e = cudaMalloc(&t.p, bytes);
    if (e != cudaSuccess) {
        c->err = std::string("cudaMalloc(tmp ") + std::to_string(bytes) + "): " + cudaGetErrorString(e);
        cudaGetLastError();
        t.p = nullptr;
        return PFE_ENOMEM;
    }
    *p = (P *)t.p;
    return PFE_OK;
}

// out[0..n] = exclusive scan of in[0..n); out[n] = total
pfe_status scan_exclusive(pfe_ctx *c, cudaStream_t s, const int *in, const int64_t *in64, int64_t n,
                          int64_t *out) {
    int64_t nb = (n + 1023) / 1024;
    if (nb == 0) nb = 1;
    Tmp tb, to;
    int64_t *bsum = nullptr, *boff = nullptr;
    PFE_TRY(talloc(c, tb, &bsum, nb));
    PFE_TRY(talloc(c, to, &boff, nb + 1));
    k_scan_block<<<(unsigned)nb, 1024, 0, s>>>(n, in, in64, out, bsum);
    PFE_CUDA_TRY(c, cudaGetLastError());
    if (nb > 1) {
        PFE_TRY(scan_exclusive(c, s, nullptr, bsum, nb, boff));
        k_scan_add<<<(unsigned)nb, 1024, 0, s>>>(n, out, boff);
        PFE_CUDA_TRY(c, cudaGetLastError());
        // total = boff[nb]
        PFE_CUDA_TRY(c, cudaMemcpyAsync(out + n, boff + nb, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    } else {
        PFE_CUDA_TRY(c, cudaMemcpyAsync(out + n, bsum, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    }
    return PFE_OK;
}

__global__ void k_narrow(int64_t n, const int64_t *in, int *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int)in[i];
}

pfe_status read_i64(pfe_ctx *c, cudaStream_t s, const int64_t *d, int64_t *h) {
    PFE_CUDA_TRY(c, cudaMemcpyAsync(h, d, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(c, cudaStreamSynchronize(s));
    return PFE_OK;
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Allocate the slot arrays once the slice pointers are known.
pfe_status alloc_slots(pfe_ctx *c, cudaStream_t s, const int64_t *slice_ptr64, const int64_t *fslice_ptr64) {
    auto &g = c->g;
    int64_t slots = 0, fslots = 0;
    PFE_TRY(read_i64(c, s, slice_ptr64 + g.n_slices, &slots));
    PFE_TRY(read_i64(c, s, fslice_ptr64 + g.n_slices, &fslots));
    if (slots > INT32_MAX || fslots > INT32_MAX) {
        c->err = "graph too large for 32-bit slot indices";
        return PFE_EINVAL;
    }
    g.slots = slots;
    g.fslots = fslots;
    PFE_TRY(dalloc(c, &g.slice_ptr, g.n_slices + 1));
    PFE_TRY(dalloc(c, &g.fslice_ptr, g.n_slices + 1));
    k_narrow<<<nblk(g.n_slices + 1, 256), 256, 0, s>>>(g.n_slices + 1, slice_ptr64, g.slice_ptr);
    k_narrow<<<nblk(g.n_slices + 1, 256), 256, 0, s>>>(g.n_slices + 1, fslice_ptr64, g.fslice_ptr);
    PFE_CUDA_TRY(c, cudaGetLastError());
    PFE_TRY(dalloc(c, &g.col, slots));
    PFE_TRY(dalloc(c, &g.eid, slots));
    PFE_TRY(dalloc(c, &g.w64, slots));
    PFE_TRY(dalloc(c, &g.w32, slots));
    PFE_TRY(dalloc(c, &g.aoff64, slots));
    PFE_TRY(dalloc(c, &g.aoff32, slots));
    PFE_TRY(dalloc(c, &g.aofflo32, slots));
    PFE_TRY(dalloc(c, &g.ext_slot, g.n_edges));
    PFE_TRY(dalloc(c, &g.ea, g.n_edges));
    PFE_TRY(dalloc(c, &g.eb, g.n_edges));
    PFE_TRY(dalloc(c, &g.ew, g.n_edges));
    PFE_TRY(dalloc(c, &g.deg, g.n));
    PFE_TRY(dalloc(c, &g.deg2, g.n));
    PFE_TRY(dalloc(c, &g.sqrtdeg, g.n));
    PFE_TRY(dalloc(c, &g.adiag64, g.n));
    PFE_TRY(dalloc(c, &g.adiag32, g.n));
    PFE_TRY(dalloc(c, &g.adiaglo32, g.n));
    PFE_TRY(dalloc(c, &g.dinv64, g.n));
    PFE_TRY(dalloc(c, &g.dinv32, g.n));
    return PFE_OK;
}

// largest slots-per-row of any slice (host side, for launch sizing)
pfe_status max_row_slots(pfe_ctx *c, cudaStream_t s, const int *slice_len) {
    std::vector<int> h((size_t)c->g.n_slices);
    PFE_CUDA_TRY(c, cudaMemcpyAsync(h.data(), slice_len, sizeof(int) * h.size(), cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(c, cudaStreamSynchronize(s));
    int mx = 0;
    for (int v : h) mx = std::max(mx, v / 32);
    c->g.max_slots_per_row = mx;
    return PFE_OK;
}

}  // namespace

pfe_status build_grid_graph(pfe_ctx *c, const double *dfeat) {
    cudaStream_t s = c->stream;
    auto &g = c->g;
    Offsets off{};
    {
        int R = (int)std::floor(c->radius);
        std::vector<std::pair<int, int>> v;  // (dy, dx) sorted
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx)
                if (dx * dx + dy * dy > 0 && (double)(dx * dx + dy * dy) <= c->radius * c->radius)
                    v.push_back({dy, dx});
        if ((int)v.size() > kMaxOffsets || v.empty()) {
            c->err = "radius gives no or too many stencil offsets";
            return PFE_EINVAL;
        }
        off.K = (int)v.size();
        for (int t = 0; t < off.K; ++t) {
            off.dy[t] = v[t].first;
            off.dx[t] = v[t].second;
        }
    }
    g.n = c->n;
    g.n_slices = (c->n + 31) / 32;
    const int64_t nthreads = g.n_slices * 32;
    Tmp t_nf, t_sl, t_fsl, t_sp, t_fsp, t_fw;
    int *nf_row, *slice_len, *fslice_len;
    int64_t *slice_ptr64, *fslice_ptr64, *fw_off;
    PFE_TRY(talloc(c, t_nf, &nf_row, g.n));
    PFE_TRY(talloc(c, t_sl, &slice_len, g.n_slices));
    PFE_TRY(talloc(c, t_fsl, &fslice_len, g.n_slices));
    PFE_TRY(talloc(c, t_sp, &slice_ptr64, g.n_slices + 1));
    PFE_TRY(talloc(c, t_fsp, &fslice_ptr64, g.n_slices + 1));
    PFE_TRY(talloc(c, t_fw, &fw_off, g.n + 1));
    const GridSegs gs{c->nseg, c->seg_off, c->seg_h, c->seg_w, c->rseg};
    k_grid_count<<<nblk(nthreads, 256), 256, 0, s>>>(g.n, g.n_slices, gs, off, nf_row, slice_len, fslice_len);
    PFE_CUDA_TRY(c, cudaGetLastError());
    PFE_TRY(scan_exclusive(c, s, slice_len, nullptr, g.n_slices, slice_ptr64));
    PFE_TRY(scan_exclusive(c, s, fslice_len, nullptr, g.n_slices, fslice_ptr64));
    PFE_TRY(scan_exclusive(c, s, nf_row, nullptr, g.n, fw_off));
    int64_t ne = 0;
    PFE_TRY(read_i64(c, s, fw_off + g.n, &ne));
    g.n_edges = ne;
    PFE_TRY(max_row_slots(c, s, slice_len));
    PFE_TRY(alloc_slots(c, s, slice_ptr64, fslice_ptr64));
    g.row_len = off.K;  // every row: K slots, slot t = offset t
    const double inv2s2 = 1.0 / (2.0 * c->sigma * c->sigma);
    k_grid_fill<<<nblk(nthreads, 128), 128, 0, s>>>(g.n, g.n_slices, gs, off, slice_ptr64, fslice_ptr64, fw_off,
                                                     dfeat, c->m, inv2s2, g.col, g.eid, g.w64, g.ext_slot, g.ea,
                                                     g.eb, g.ew, g.deg, g.deg2);
    PFE_CUDA_TRY(c, cudaGetLastError());
    PFE_CUDA_TRY(c, cudaStreamSynchronize(s));
    return PFE_OK;
}

pfe_status build_edge_graph(pfe_ctx *c, const double *dfeat, const int32_t *dei, const int32_t *dej) {
    cudaStream_t s = c->stream;
    auto &g = c->g;
    g.n = c->n;
    g.n_slices = (c->n + 31) / 32;
    g.n_edges = c->g.n_edges;
    const int64_t nthreads = g.n_slices * 32;
    Tmp t_nb, t_nf, t_sl, t_fsl, t_sp, t_fsp, t_cur, t_ext, t_err;
    int *nb_row, *nf_row, *slice_len, *fslice_len, *cursor, *tmp_ext, *derr;
    int64_t *slice_ptr64, *fslice_ptr64;
    PFE_TRY(talloc(c, t_nb, &nb_row, g.n));
    PFE_TRY(talloc(c, t_nf, &nf_row, g.n));
    PFE_TRY(talloc(c, t_sl, &slice_len, g.n_slices));
    PFE_TRY(talloc(c, t_fsl, &fslice_len, g.n_slices));
    PFE_TRY(talloc(c, t_sp, &slice_ptr64, g.n_slices + 1));
    PFE_TRY(talloc(c, t_fsp, &fslice_ptr64, g.n_slices + 1));
    PFE_TRY(talloc(c, t_cur, &cursor, g.n));
    PFE_TRY(talloc(c, t_err, &derr, 1));
    PFE_CUDA_TRY(c, cudaMemsetAsync(nb_row, 0, sizeof(int) * g.n, s));
    PFE_CUDA_TRY(c, cudaMemsetAsync(nf_row, 0, sizeof(int) * g.n, s));
    PFE_CUDA_TRY(c, cudaMemsetAsync(cursor, 0, sizeof(int) * g.n, s));
    PFE_CUDA_TRY(c, cudaMemsetAsync(derr, 0, sizeof(int), s));
    k_edges_count<<<nblk(g.n_edges, 256), 256, 0, s>>>(g.n, g.n_edges, dei, dej, nb_row, nf_row, derr);
    k_slice_max<<<nblk(nthreads, 256), 256, 0, s>>>(g.n, g.n_slices, nb_row, nf_row, slice_len, fslice_len);
    PFE_CUDA_TRY(c, cudaGetLastError());
    int herr = 0;
    PFE_CUDA_TRY(c, cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(c, cudaStreamSynchronize(s));
    if (herr) {
        c->err = "edge list has a self-loop or an endpoint outside [0, n)";
        return PFE_EINVAL;
    }
    PFE_TRY(scan_exclusive(c, s, slice_len, nullptr, g.n_slices, slice_ptr64));
    PFE_TRY(scan_exclusive(c, s, fslice_len, nullptr, g.n_slices, fslice_ptr64));
    PFE_TRY(max_row_slots(c, s, slice_len));
    PFE_TRY(alloc_slots(c, s, slice_ptr64, fslice_ptr64));
    PFE_TRY(talloc(c, t_ext, &tmp_ext, g.slots));
    k_edges_scatter<<<nblk(g.n_edges, 256), 256, 0, s>>>(g.n_edges, dei, dej, slice_ptr64, cursor, g.col,
                                                           tmp_ext);
    k_edges_sort<<<nblk(nthreads, 128), 128, 0, s>>>(g.n, g.n_slices, slice_ptr64, fslice_ptr64, nb_row, g.col, tmp_ext,
                                                      g.eid, g.ext_slot, g.ea, g.eb, derr);
    const double inv2s2 = 1.0 / (2.0 * c->sigma * c->sigma);
    k_edges_backward<<<nblk(g.n, 128), 128, 0, s>>>(g.n, slice_ptr64, nb_row, tmp_ext, g.ext_slot, g.eid, g.col,
                                                     dfeat, c->m, inv2s2, g.w64, g.ew, g.deg, g.deg2);
    PFE_CUDA_TRY(c, cudaGetLastError());
    PFE_CUDA_TRY(c, cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(c, cudaStreamSynchronize(s));
    if (herr) {
        c->err = "edge list names the same pair twice";
        return PFE_EINVAL;
    }
    return PFE_OK;
}

__global__ void k_check_edge_segs(int64_t ne, const int *ea, const int *eb, const int *rseg, int *err) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < ne && rseg[ea[k]] != rseg[eb[k]]) atomicExch(err, 1);
}

// A batch's edge list must stay inside the segments.
pfe_status check_edges_in_segments(pfe_ctx *c) {
    cudaStream_t s = c->stream;
    Tmp t_err;
    int *derr, herr = 0;
    PFE_TRY(talloc(c, t_err, &derr, 1));
    PFE_CUDA_TRY(c, cudaMemsetAsync(derr, 0, sizeof(int), s));
    k_check_edge_segs<<<nblk(c->g.n_edges, 256), 256, 0, s>>>(c->g.n_edges, c->g.ea, c->g.eb, c->rseg, derr);
    PFE_CUDA_TRY(c, cudaGetLastError());
    PFE_CUDA_TRY(c, cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(c, cudaStreamSynchronize(s));
    if (herr) {
        c->err = "an edge joins two segments of the batch";
        return PFE_EINVAL;
    }
    return PFE_OK;
}

pfe_status setup_segments(pfe_ctx *c) {
    cudaStream_t s = c->stream;
    const int ns = c->nseg;
    PFE_TRY(dalloc(c, &c->seg_off, ns + 1));
    PFE_TRY(dalloc(c, &c->seg_h, ns));
    PFE_TRY(dalloc(c, &c->seg_w, ns));
    PFE_TRY(dalloc(c, &c->seg_lam, ns));
    PFE_TRY(dalloc(c, &c->rseg, c->n));
    PFE_CUDA_TRY(c, cudaMemcpyAsync(c->seg_off, c->h_seg_off.data(), sizeof(int64_t) * (ns + 1),
                                    cudaMemcpyHostToDevice, s));
    PFE_CUDA_TRY(c, cudaMemcpyAsync(c->seg_h, c->h_seg_h.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
    PFE_CUDA_TRY(c, cudaMemcpyAsync(c->seg_w, c->h_seg_w.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
    k_fill_rseg<<<nblk(c->n, 256), 256, 0, s>>>(c->n, ns, c->seg_off, c->rseg);
    PFE_CUDA_TRY(c, cudaGetLastError());
    PFE_CUDA_TRY(c, cudaStreamSynchronize(s));  // the host tables may go out of scope
    return PFE_OK;
}

pfe_status finish_graph_values(pfe_ctx *c) {
    cudaStream_t s = c->stream;
    auto &g = c->g;
    // vol = sum_i d_i (deterministic block partials), lambda = sqrt(vol) by default
    Tmp t_part, t_tick, t_res, t_err;
    double *part, *res;
    unsigned *tick;
    int *derr;
    const int nb = 256;
    PFE_TRY(talloc(c, t_part, &part, nb));
    PFE_TRY(talloc(c, t_tick, &tick, 1));
    PFE_TRY(talloc(c, t_res, &res, 1));
    PFE_TRY(talloc(c, t_err, &derr, 1));
    PFE_CUDA_TRY(c, cudaMemsetAsync(tick, 0, sizeof(unsigned), s));
    PFE_CUDA_TRY(c, cudaMemsetAsync(derr, 0, sizeof(int), s));
    c->r = c->prm.r;
    if (c->nseg == 1) {
        k_sum_f64<<<nb, kBlock, 0, s>>>(g.n, g.deg, part, tick, res);
        PFE_CUDA_TRY(c, cudaGetLastError());
        double vol = 0;
        PFE_CUDA_TRY(c, cudaMemcpyAsync(&vol, res, sizeof(double), cudaMemcpyDeviceToHost, s));
        PFE_CUDA_TRY(c, cudaStreamSynchronize(s));
        c->vol = vol;
        c->lambda = c->prm.lambda > 0 ? c->prm.lambda : std::sqrt(vol);
        c->h_seg_vol.assign(1, vol);
        c->h_seg_lam.assign(1, c->lambda);
        PFE_CUDA_TRY(c, cudaMemcpyAsync(c->seg_lam, &c->lambda, sizeof(double), cudaMemcpyHostToDevice, s));
        k_values_slots<<<nblk(g.slots, 256), 256, 0, s>>>(g.slots, c->lambda, g.w64, g.w32, g.aoff64, g.aoff32);
        k_values_rows<<<nblk(g.n, 256), 256, 0, s>>>(g.n, c->lambda, c->r, g.deg, g.deg2, g.sqrtdeg, g.adiag64,
                                                     g.adiag32, g.dinv64, g.dinv32, derr);
    } else {
        // one volume and one lambda per segment (image)
        const int ns = c->nseg;
        Tmp t_vol;
        double *dvol;
        PFE_TRY(talloc(c, t_vol, &dvol, ns));
        k_seg_sum<<<ns, kBlock, 0, s>>>(c->seg_off, g.deg, dvol);
        PFE_CUDA_TRY(c, cudaGetLastError());
        c->h_seg_vol.assign(ns, 0.0);
        PFE_CUDA_TRY(c, cudaMemcpyAsync(c->h_seg_vol.data(), dvol, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
        PFE_CUDA_TRY(c, cudaStreamSynchronize(s));
        c->h_seg_lam.assign(ns, 0.0);
        c->vol = 0.0;
        for (int q = 0; q < ns; ++q) {
            c->vol += c->h_seg_vol[q];
            c->h_seg_lam[q] = c->prm.lambda > 0 ? c->prm.lambda : std::sqrt(c->h_seg_vol[q]);
        }
        c->lambda = c->h_seg_lam[0];
        PFE_CUDA_TRY(c, cudaMemcpyAsync(c->seg_lam, c->h_seg_lam.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, s));
        k_values_seg<<<nblk(g.n_slices * 32, 256), 256, 0, s>>>(g.n, g.n_slices, g.slice_ptr, c->rseg, c->seg_lam, c->r,
                                                                 g.w64, g.w32, g.aoff64, g.aoff32, g.deg, g.deg2,
                                                                 g.sqrtdeg, g.adiag64, g.adiag32, g.dinv64, g.dinv32,
                                                                 derr);
    }
    if (g.slots > 0) k_values_lo<<<nblk(g.slots, 256), 256, 0, s>>>(g.slots, g.aoff64, g.aoff32, g.aofflo32);
    k_values_lo<<<nblk(g.n, 256), 256, 0, s>>>(g.n, g.adiag64, g.adiag32, g.adiaglo32);
    PFE_CUDA_TRY(c, cudaGetLastError());
    int herr = 0;
    PFE_CUDA_TRY(c, cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(c, cudaStreamSynchronize(s));
    if (herr) {
        c->err = "a vertex has zero degree (D^{-1/2} undefined)";
        return PFE_EINVAL;
    }
    return PFE_OK;
}

}  // namespace pfe
