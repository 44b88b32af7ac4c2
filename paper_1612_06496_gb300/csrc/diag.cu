// Diagnostics of an embedding (FP64 reductions, deterministic order):
//   |M Y|_1 = sum over undirected edges (a < b) of w_ab |y_a - y_b|_1, the
//             objective of Eq. 1 (which counts every pair twice);
//   |Y^T D Y - I|_F, the distance from the constraint of Eq. 1, for each
//             problem of a batch (the largest is reported);
//   |b_c - A x_c| / |b_c| per column (and problem of a batch) of a solve of
//             Eq. 13, with the FP64 system matrix whatever the iteration's
//             precision.
#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace pfe {
namespace {

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// one thread per row; slot (i, j) counted when j > i
__global__ void k_obj_l1(int64_t n, const int *slice_ptr, const int *col, const double *w, const double *y, int d,
                         double *part, unsigned *ticket, double *out) {
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = i >> 5;
        const int s0 = slice_ptr[s];
        const int len = (slice_ptr[s + 1] - s0) >> 5;
        const int64_t base = (int64_t)s0 + (i & 31) * (int64_t)len;
        for (int k = 0; k < len; ++k) {
            const int64_t j = col[base + k];
            const double wij = w[base + k];
            if (j <= i || wij == 0.0) continue;
            double t = 0.0;
            for (int c = 0; c < d; ++c) t += fabs(y[i * d + c] - y[j * d + c]);
            acc = fma(wij, t, acc);
        }
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

// Y^T D Y of each segment (rows of a block stay in its segment), then
// |G - I|_F; the largest over the segments by an integer max on the bits of a
// non-negative double (order independent).
constexpr int kTileO = 32;
__global__ void k_obj_gram(Segs sg, const double *deg, const double *y, int d, double *part, unsigned *tickets,
                           unsigned long long *out) {
    extern __shared__ double smo[];
    double *tile = smo;                // kTileO x d
    double *td = tile + kTileO * d;    // kTileO
    const int NE = d * (d + 1) / 2;
    const BlockSeg bsg = block_seg(sg);
    double acc[3] = {0.0, 0.0, 0.0};  // up to 3 entries per thread (NE <= 528 <= 3 * 256 at d <= 32)
    const int64_t ntiles = (bsg.r1 - bsg.r0 + kTileO - 1) / kTileO;
    for (int64_t t = blockIdx.x - bsg.b0; t < ntiles; t += bsg.nb) {
        const int64_t r0 = bsg.r0 + t * kTileO;
        for (int e = threadIdx.x; e < kTileO * d; e += blockDim.x) {
            const int r = e / d, c = e - r * d;
            const int64_t i = r0 + r;
            tile[e] = i < bsg.r1 ? y[i * d + c] : 0.0;
            if (c == 0) td[r] = i < bsg.r1 ? deg[i] : 0.0;
        }
        __syncthreads();
        for (int k = 0; k < 3; ++k) {
            const int e = threadIdx.x + k * blockDim.x;
            if (e >= NE) break;
            int p = 0, rem = e;
            while (rem >= d - p) {
                rem -= d - p;
                ++p;
            }
            const int q = p + rem;
            double s = acc[k];
            for (int r = 0; r < kTileO; ++r) s = fma(td[r] * tile[r * d + p], tile[r * d + q], s);
            acc[k] = s;
        }
        __syncthreads();
    }
    for (int k = 0; k < 3; ++k) {
        const int e = threadIdx.x + k * blockDim.x;
        if (e < NE) part[(int64_t)blockIdx.x * NE + e] = acc[k];
    }
    unsigned *ticket = tickets + bsg.seg;
    if (!last_block_arrives(ticket, (unsigned)bsg.nb)) return;
    if (threadIdx.x == 0) {
        double f = 0.0;
        for (int e = 0; e < NE; ++e) {
            double s = 0.0;
            for (int b = 0; b < bsg.nb; ++b) s += __ldcg(part + (int64_t)(bsg.b0 + b) * NE + e);
            int p = 0, rem = e;
            while (rem >= d - p) {
                rem -= d - p;
                ++p;
            }
            const double dev = s - (rem == 0 ? 1.0 : 0.0);  // diagonal when q == p
            f += (rem == 0 ? 1.0 : 2.0) * dev * dev;
        }
        const double fr = sqrt(f);
        atomicMax(out, (unsigned long long)__double_as_longlong(fr));
        *ticket = 0u;
    }
}

// Residual norms of the columns of B - A X (FP64 values of A): threads own
// one column (block of kRes = d * floor(256 / d) threads; thread t: column
// t % d of rows t / d, t / d + kRes / d, ...), add r^2 and b^2 of their rows,
// the block sums them per column in thread order, and the segment's last
// block adds the blocks' partials in block order: out[seg * d + c] = |r_c| /
// |b_c| (|r_c| where b_c = 0).
__global__ void k_resid(Segs sg, const int *slice_ptr, const int *col, const double *aoff, const double *adiag,
                        const double *B, const double *X, int d, double *part, unsigned *tickets, double *out) {
    extern __shared__ double smr[];  // 2 * blockDim.x
    const BlockSeg bsg = block_seg(sg);
    const int per = blockDim.x / d;  // rows a block holds at once
    const int c = threadIdx.x % d, rr = threadIdx.x / d;
    double r2 = 0.0, b2 = 0.0;
    if (rr < per) {
        for (int64_t i = bsg.r0 + (int64_t)(blockIdx.x - bsg.b0) * per + rr; i < bsg.r1; i += (int64_t)bsg.nb * per) {
            const int64_t s = i >> 5;
            const int s0 = slice_ptr[s];
            const int len = (slice_ptr[s + 1] - s0) >> 5;
            const int64_t base = (int64_t)s0 + (i & 31) * (int64_t)len;
            double ax = adiag[i] * X[i * d + c];
            for (int k = 0; k < len; ++k) ax = fma(aoff[base + k], X[(int64_t)col[base + k] * d + c], ax);
            const double b = B[i * d + c], r = b - ax;
            r2 = fma(r, r, r2);
            b2 = fma(b, b, b2);
        }
    }
    smr[threadIdx.x] = r2;
    smr[blockDim.x + threadIdx.x] = b2;
    __syncthreads();
    if (threadIdx.x < d) {
        double sr = 0.0, sb = 0.0;
        for (int q = 0; q < per; ++q) {
            sr += smr[q * d + threadIdx.x];
            sb += smr[blockDim.x + q * d + threadIdx.x];
        }
        part[(int64_t)blockIdx.x * 2 * d + threadIdx.x] = sr;
        part[(int64_t)blockIdx.x * 2 * d + d + threadIdx.x] = sb;
    }
    if (!last_block_arrives(tickets + bsg.seg, (unsigned)bsg.nb)) return;
    if (threadIdx.x < d) {
        double sr = 0.0, sb = 0.0;
        for (int b = 0; b < bsg.nb; ++b) {
            sr += __ldcg(part + (int64_t)(bsg.b0 + b) * 2 * d + threadIdx.x);
            sb += __ldcg(part + (int64_t)(bsg.b0 + b) * 2 * d + d + threadIdx.x);
        }
        out[bsg.seg * d + threadIdx.x] = sb > 0.0 ? sqrt(sr) / sqrt(sb) : sqrt(sr);
    }
    if (threadIdx.x == 0) tickets[bsg.seg] = 0u;
}

}  // namespace

// Relative residuals |B - A X| / |B| per column (and problem), FP64 A; B, X
// device n x d FP64 arrays; relres: host, nseg * d.
pfe_status diag_residual(pfe_ctx *c, const double *B, const double *X, double *relres) {
    cudaStream_t s = c->stream;
    const int d = c->d;
    const int64_t n = c->g.n;
    const int threads = d * (256 / d);
    const int per = threads / d;
    const int grid = (int)std::max<int64_t>(c->nseg, std::min<int64_t>((n + per - 1) / per, (int64_t)c->num_sms * 8));
    const size_t npart = (size_t)grid * 2 * d, nout = (size_t)c->nseg * d;
    double *buf = nullptr;
    if (cudaMalloc((void **)&buf, (npart + nout + c->nseg) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->err = "pfe_residual: device allocation failed";
        return PFE_ENOMEM;
    }
    double *part = buf, *out = buf + npart;
    unsigned *tick = reinterpret_cast<unsigned *>(out + nout);
    cudaError_t e = cudaMemsetAsync(tick, 0, sizeof(unsigned) * c->nseg, s);
    if (e == cudaSuccess) {
        k_resid<<<grid, threads, 2 * threads * sizeof(double), s>>>(seg_view(c), c->g.slice_ptr, c->g.col, c->g.aoff64,
                                                                    c->g.adiag64, B, X, d, part, tick, out);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(relres, out, nout * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(buf);
    if (e != cudaSuccess) {
        c->err = std::string("pfe_residual: ") + cudaGetErrorString(e);
        return PFE_ECUDA;
    }
    return PFE_OK;
}

// Objective and constraint distance of Y (which = 0: the iterate Y of
// Alg. 2; 1: the embedding Yhat = D^{-1/2} P).
pfe_status diag_objective(pfe_ctx *c, int which, double *l1, double *ortho) {
    cudaStream_t s = c->stream;
    const int d = c->d;
    const int64_t n = c->g.n;
    if (which == 0)
        PFE_TRY(launch_from_work(c, s, c->wk.Y, c->wk.Ylo, c->wk.stage, n));
    else
        PFE_TRY(launch_yhat(c, s, c->wk.stage));
    const int lgrid = (int)std::max<int64_t>(1, std::min<int64_t>(nblk(n, 256), (int64_t)c->num_sms * 4));
    const int ggrid = (int)std::max<int64_t>(c->nseg, std::min<int64_t>(nblk(n, kTileO), (int64_t)c->num_sms * 2));
    const int NE = d * (d + 1) / 2;
    double *buf = nullptr;
    const size_t nbuf = (size_t)std::max<int64_t>(lgrid, (int64_t)ggrid * NE) + 2 + c->nseg;
    if (cudaMalloc((void **)&buf, nbuf * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->err = "pfe_objective: device allocation failed";
        return PFE_ENOMEM;
    }
    double *part = buf, *res = buf + nbuf - 2 - c->nseg;
    unsigned *tick = reinterpret_cast<unsigned *>(res + 2);  // nseg + 1 tickets in the last doubles
    cudaError_t e = cudaMemsetAsync(res, 0, sizeof(double) * (2 + c->nseg), s);
    if (e == cudaSuccess) {
        k_obj_l1<<<lgrid, 256, 0, s>>>(n, c->g.slice_ptr, c->g.col, c->g.w64, c->wk.stage, d, part, tick + c->nseg,
                                       res);
        k_obj_gram<<<ggrid, 256, sizeof(double) * (kTileO * d + kTileO), s>>>(
            seg_view(c), c->g.deg, c->wk.stage, d, part, tick, reinterpret_cast<unsigned long long *>(res + 1));
        e = cudaGetLastError();
    }
    double h[2] = {0.0, 0.0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(buf);
    if (e != cudaSuccess) {
        c->err = std::string("pfe_objective: ") + cudaGetErrorString(e);
        return PFE_ECUDA;
    }
    if (l1) *l1 = h[0];
    if (ortho) *ortho = h[1];
    return PFE_OK;
}

}  // namespace pfe
