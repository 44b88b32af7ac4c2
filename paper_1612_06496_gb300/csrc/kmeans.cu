// Segmentation stage (Sec. IV: k-means clustering on the embeddings), FP64:
// a deterministic maximin start (centroid 0 = row 0, then repeatedly the row
// farthest from its nearest chosen centroid, ties to the smallest row) and
// Lloyd iterations (nearest centroid with ties to the smallest cluster;
// centroids = means of their rows, an empty cluster keeps its centroid)
// until no label changes.  Squared distances accumulate the squared column
// differences in column order with separately rounded products and sums;
// the centroid sums run over contiguous row chunks in row order, combined in
// chunk order.  Every result is reproducible run to run.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace pfe {
namespace {

constexpr int kKmBlock = 256;
constexpr int kMaxK = 64;

__device__ __forceinline__ double sqdist(const double *x, const double *c, int d) {
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        const double df = __dsub_rn(x[j], c[j]);
        s = __dadd_rn(s, __dmul_rn(df, df));
    }
    return s;
}

// (value, index) maximum with ties to the smaller index
__device__ __forceinline__ void amax_merge(double &v, int64_t &i, double v2, int64_t i2) {
    if (v2 > v || (v2 == v && i2 < i)) {
        v = v2;
        i = i2;
    }
}

struct ArgCtl {
    unsigned ticket;
    int pad;
    int64_t row;  // result of the last argmax
};

// One maximin step t >= 1: mind_i = min(mind_i, |x_i - C_{t-1}|^2) (t == 1:
// the distance itself), then C_t = x_r with r = argmax mind.
__global__ void k_km_maximin(int64_t n, int d, const double *__restrict__ X, double *C, int t, double *mind,
                             double *pval, int64_t *pidx, ArgCtl *ac) {
    __shared__ double sc[32];
    for (int j = threadIdx.x; j < d; j += blockDim.x) sc[j] = C[(int64_t)(t - 1) * d + j];
    __syncthreads();
    double bv = -1.0;
    int64_t bi = INT64_MAX;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double dd = sqdist(X + i * d, sc, d);
        const double m = t == 1 ? dd : fmin(mind[i], dd);
        mind[i] = m;
        amax_merge(bv, bi, m, i);
    }
    __shared__ double rv[kKmBlock];
    __shared__ int64_t ri[kKmBlock];
    rv[threadIdx.x] = bv;
    ri[threadIdx.x] = bi;
    __syncthreads();
    for (int s = kKmBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            double v = rv[threadIdx.x];
            int64_t ix = ri[threadIdx.x];
            amax_merge(v, ix, rv[threadIdx.x + s], ri[threadIdx.x + s]);
            rv[threadIdx.x] = v;
            ri[threadIdx.x] = ix;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        pval[blockIdx.x] = rv[0];
        pidx[blockIdx.x] = ri[0];
    }
    if (!last_block_arrives(&ac->ticket)) return;
    __shared__ int64_t row;
    if (threadIdx.x == 0) {
        double v = -1.0;
        int64_t ix = INT64_MAX;
        for (unsigned b = 0; b < gridDim.x; ++b)
            amax_merge(v, ix, __ldcg(pval + b), __ldcg(reinterpret_cast<const long long *>(pidx) + b));
        row = ix < n ? ix : 0;
        ac->row = row;
        ac->ticket = 0u;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < d; j += blockDim.x) C[(int64_t)t * d + j] = X[row * d + j];
}

// Assignment: label_i = argmin_j |x_i - C_j|^2 (ties to the smaller j); counts
// the labels that changed.
__global__ void k_km_assign(int64_t n, int d, int k, const double *__restrict__ X, const double *C, int *labels,
                            unsigned long long *changed) {
    extern __shared__ double scm[];  // k x d centroids
    for (int e = threadIdx.x; e < k * d; e += blockDim.x) scm[e] = C[e];
    __syncthreads();
    unsigned long long ch = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int best = 0;
        double bd = sqdist(X + i * d, scm, d);
        for (int j = 1; j < k; ++j) {
            const double dd = sqdist(X + i * d, scm + j * d, d);
            if (dd < bd) {
                bd = dd;
                best = j;
            }
        }
        if (labels[i] != best) ++ch;
        labels[i] = best;
    }
    for (int m = 16; m > 0; m >>= 1) ch += __shfl_xor_sync(0xffffffffu, ch, m);
    if ((threadIdx.x & 31) == 0 && ch) atomicAdd(changed, ch);
}

// Centroid sums: block b owns rows [b * chunk, (b + 1) * chunk); thread t
// sums column c of cluster j (pairs t, t + blockDim, ...) over its rows in
// row order.  The last block combines the blocks in order and divides.
__global__ void k_km_update(int64_t n, int d, int k, int64_t chunk, const double *__restrict__ X,
                            const int *__restrict__ labels, double *C, double *psum, long long *pcnt,
                            unsigned *ticket) {
    const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(n, r0 + chunk);
    for (int e = threadIdx.x; e < k * d; e += blockDim.x) {
        const int j = e / d, c = e - j * d;
        double s = 0.0;
        long long cnt = 0;
        for (int64_t i = r0; i < r1; ++i)
            if (labels[i] == j) {
                s += X[i * d + c];
                ++cnt;
            }
        psum[(int64_t)blockIdx.x * k * d + e] = s;
        if (c == 0) pcnt[(int64_t)blockIdx.x * k + j] = cnt;
    }
    if (!last_block_arrives(ticket)) return;
    for (int e = threadIdx.x; e < k * d; e += blockDim.x) {
        const int j = e / d;
        double s = 0.0;
        long long cnt = 0;
        for (unsigned b = 0; b < gridDim.x; ++b) {
            s += __ldcg(psum + (int64_t)b * k * d + e);
            cnt += __ldcg(pcnt + (int64_t)b * k + j);
        }
        if (cnt > 0) C[e] = s / (double)cnt;  // an empty cluster keeps its centroid
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

// inertia = sum_i min_j |x_i - C_j|^2, fixed order
__global__ void k_km_inertia(int64_t n, int d, int k, const double *__restrict__ X, const double *C, double *part,
                             unsigned *ticket, double *out) {
    extern __shared__ double scm[];
    for (int e = threadIdx.x; e < k * d; e += blockDim.x) scm[e] = C[e];
    __syncthreads();
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double bd = sqdist(X + i * d, scm, d);
        for (int j = 1; j < k; ++j) bd = fmin(bd, sqdist(X + i * d, scm + j * d, d));
        acc += bd;
    }
    double v[1] = {acc};
    block_reduce<double, 1>(v, part + blockIdx.x);
    if (last_block_arrives(ticket)) {
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(part + b);
            *out = t;
            *ticket = 0u;
        }
    }
}

}  // namespace

pfe_status kmeans_run(pfe_ctx *c, const double *X, int d, int k, const double *C0, int max_iter, int *labels,
                      double *centroids, double *inertia, int *rounds) {
    cudaStream_t s = c->stream;
    const int64_t n = c->n;
    if (d < 1 || d > 32 || k < 1 || k > kMaxK || k > n || max_iter < 1) return PFE_EINVAL;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + kKmBlock - 1) / kKmBlock, (int64_t)c->num_sms * 2));
    const int64_t chunk = (n + grid - 1) / grid;
    const int ugrid = (int)((n + chunk - 1) / chunk);
    std::vector<void *> mem;
    auto get = [&](size_t bytes) -> void * {
        void *q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        mem.push_back(q);
        return q;
    };
    auto cleanup = [&]() {
        for (void *q : mem) cudaFree(q);
    };
    double *dC = (double *)get(sizeof(double) * k * d);
    int *dlab = (int *)get(sizeof(int) * n);
    double *mind = (double *)get(sizeof(double) * n);
    double *pval = (double *)get(sizeof(double) * std::max(grid, ugrid) * (size_t)std::max(1, k * d));
    int64_t *pidx = (int64_t *)get(sizeof(int64_t) * grid);
    long long *pcnt = (long long *)get(sizeof(long long) * ugrid * (size_t)k);
    ArgCtl *ac = (ArgCtl *)get(sizeof(ArgCtl));
    unsigned long long *dch = (unsigned long long *)get(sizeof(unsigned long long) + 64);
    if (mem.size() != 8 || std::find(mem.begin(), mem.end(), nullptr) != mem.end()) {
        cleanup();
        c->err = "pfe_kmeans: device allocation failed";
        return PFE_ENOMEM;
    }
    unsigned *tick = reinterpret_cast<unsigned *>(dch + 1);
    double *dres = reinterpret_cast<double *>(dch) + 2;
    cudaError_t e = cudaMemsetAsync(ac, 0, sizeof(ArgCtl), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dch, 0, sizeof(unsigned long long) + 64, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dlab, 0xff, sizeof(int) * n, s);  // labels -1: every label changes in the first Lloyd round
    if (e == cudaSuccess) {
        if (C0) {
            e = cudaMemcpyAsync(dC, C0, sizeof(double) * k * d, cudaMemcpyDefault, s);
        } else {
            e = cudaMemcpyAsync(dC, X, sizeof(double) * d, cudaMemcpyDeviceToDevice, s);  // centroid 0 = row 0
            for (int t = 1; t < k && e == cudaSuccess; ++t) {
                k_km_maximin<<<grid, kKmBlock, 0, s>>>(n, d, X, dC, t, mind, pval, pidx, ac);
                e = cudaGetLastError();
            }
        }
    }
    const size_t smem = sizeof(double) * k * d;
    int r = 0;
    for (r = 1; r <= max_iter && e == cudaSuccess; ++r) {
        unsigned long long hch = 0;
        e = cudaMemsetAsync(dch, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) break;
        k_km_assign<<<grid, kKmBlock, smem, s>>>(n, d, k, X, dC, dlab, dch);
        k_km_update<<<ugrid, kKmBlock, 0, s>>>(n, d, k, chunk, X, dlab, dC, pval, pcnt, tick);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hch, dch, sizeof(hch), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess || hch == 0) break;
    }
    if (r > max_iter) r = max_iter;
    double hin = 0.0;
    if (e == cudaSuccess) {
        k_km_inertia<<<grid, kKmBlock, smem, s>>>(n, d, k, X, dC, pval, tick + 1, dres);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && labels) e = cudaMemcpyAsync(labels, dlab, sizeof(int) * n, cudaMemcpyDefault, s);
    if (e == cudaSuccess && centroids) e = cudaMemcpyAsync(centroids, dC, sizeof(double) * k * d, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hin, dres, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    if (e != cudaSuccess) {
        c->err = std::string("pfe_kmeans: ") + cudaGetErrorString(e);
        return PFE_ECUDA;
    }
    if (inertia) *inertia = hin;
    if (rounds) *rounds = r;
    return PFE_OK;
}

}  // namespace pfe
