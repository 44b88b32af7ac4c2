// pfe_orthonormalize_noalloc: the D-orthonormalisation that pfe_init applies
// to a starting embedding, Yhat = D^{-1/2} polar(D^{1/2} Y), for callers that
// cannot allocate device memory (see include/pfe.h).  Its scratch -- the
// Gram matrix's block partials and a small control block -- lives in one
// file-scope device array of fixed size instead of cudaMalloc'd buffers.
#include <mutex>

#include "pstep_kernels.cuh"
#include "dispatch.cuh"

namespace pfe {
namespace noalloc {

constexpr int kMaxD = 16;            // largest embedding dimension accepted
constexpr int kMaxBlocks = 512;      // largest Gram grid
constexpr int kNEMax = kMaxD * (kMaxD + 1) / 2;
constexpr size_t kPartBytes = (size_t)kMaxBlocks * kNEMax * sizeof(double);
constexpr size_t kCtlOffset = (kPartBytes + 255) / 256 * 256;
constexpr size_t kScratchBytes = kCtlOffset + (sizeof(PstepCtl) + 255) / 256 * 256;

// Shared by every call on a device; holds the last call's contents.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kTileNA = 64;

// block partials of G = X^T X with X_i = sqrt(deg_i) Y_i; the last block sums
// them in a fixed order and computes T = G^{-1/2} (cyclic Jacobi, FP64)
template <int D>
__global__ void __launch_bounds__(kBlock) k_gram_na(const double *__restrict__ Y, const double *__restrict__ deg,
                                                    int64_t n, double *part, PstepCtl *ctl) {
    constexpr int NE = D * (D + 1) / 2;
    constexpr int PER = (NE + kBlock - 1) / kBlock;
    __shared__ double tile[kTileNA][D];
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
    const int64_t ntiles = (n + kTileNA - 1) / kTileNA;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t r0 = t * kTileNA;
        for (int rr = threadIdx.x; rr < kTileNA; rr += blockDim.x) {
            const int64_t i = r0 + rr;
            const double sd = i < n ? sqrt(deg[i]) : 0.0;
#pragma unroll
            for (int c = 0; c < D; ++c) tile[rr][c] = i < n ? sd * Y[i * D + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = threadIdx.x + k * kBlock;
            if (e < NE) {
                const int p = ep[e], q = eq[e];
                double s = g[k];
                for (int rr = 0; rr < kTileNA; ++rr) s = fma(tile[rr][p], tile[rr][q], s);
                g[k] = s;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int e = threadIdx.x + k * kBlock;
        if (e < NE) part[(int64_t)blockIdx.x * NE + e] = g[k];
    }
    if (!last_block_arrives(&ctl->ticket)) return;
    __shared__ double G[D * D], V[D * D];
    for (int e = threadIdx.x; e < NE; e += blockDim.x) {
        double s = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(part + (int64_t)b * NE + e);
        const int p = ep[e], q = eq[e];
        G[p * D + q] = s;
        G[q * D + p] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        jacobi_eig(G, V, D);
        double lmax = 0.0, lmin = INFINITY;
        for (int k = 0; k < D; ++k) {
            lmax = fmax(lmax, G[k * D + k]);
            lmin = fmin(lmin, G[k * D + k]);
        }
        if (!(lmin > 1e-13 * lmax) || !(lmax < INFINITY)) {
            ctl->error = PFE_ESINGULAR;
        } else {
            ctl->error = 0;
            for (int p = 0; p < D; ++p)
                for (int q = 0; q < D; ++q) {
                    double s = 0.0;
                    for (int k = 0; k < D; ++k) s += V[p * D + k] * V[q * D + k] / sqrt(G[k * D + k]);
                    ctl->T[p * D + q] = s;
                }
        }
        ctl->ticket = 0u;
    }
}

// Yhat_i = (sqrt(deg_i) Y_i T) / sqrt(deg_i)
template <int D>
__global__ void __launch_bounds__(kBlock) k_apply_na(const double *__restrict__ Y, const double *__restrict__ deg,
                                                     int64_t n, const PstepCtl *ctl, double *__restrict__ out) {
    __shared__ double Tm[D * D];
    if (ctl->error) return;
    for (int k = threadIdx.x; k < D * D; k += blockDim.x) Tm[k] = ctl->T[k];
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double sd = sqrt(deg[i]);
        double x[D];
#pragma unroll
        for (int c = 0; c < D; ++c) x[c] = sd * Y[i * D + c];
#pragma unroll
        for (int q = 0; q < D; ++q) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < D; ++k) s = fma(x[k], Tm[k * D + q], s);
            out[i * D + q] = s / sd;
        }
    }
}

template <int D>
pfe_status run(const double *Y, const double *deg, int64_t n, double *out, cudaStream_t s, unsigned char *base,
               int blocks) {
    double *part = reinterpret_cast<double *>(base);
    PstepCtl *ctl = reinterpret_cast<PstepCtl *>(base + kCtlOffset);
    // the array keeps the previous call's contents: restart the ticket and flag
    if (cudaMemsetAsync(ctl, 0, 2 * sizeof(unsigned), s) != cudaSuccess) return PFE_ECUDA;
    k_gram_na<D><<<blocks, kBlock, 0, s>>>(Y, deg, n, part, ctl);
    k_apply_na<D><<<blocks, kBlock, 0, s>>>(Y, deg, n, ctl, out);
    if (cudaGetLastError() != cudaSuccess) return PFE_ECUDA;
    int err = 0;
    if (cudaMemcpyAsync(&err, &ctl->error, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return PFE_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PFE_ECUDA;
    return err ? PFE_ESINGULAR : PFE_OK;
}

#define PFE_NA_CASE(DV) \
    case DV:            \
        return run<DV>(Y, deg, n, out, s, base, blocks);

pfe_status dispatch(int d, const double *Y, const double *deg, int64_t n, double *out, cudaStream_t s,
                    unsigned char *base, int blocks) {
    switch (d) {
        PFE_NA_CASE(1) PFE_NA_CASE(2) PFE_NA_CASE(3) PFE_NA_CASE(4) PFE_NA_CASE(5) PFE_NA_CASE(6)
        PFE_NA_CASE(7) PFE_NA_CASE(8) PFE_NA_CASE(9) PFE_NA_CASE(10) PFE_NA_CASE(11) PFE_NA_CASE(12)
        PFE_NA_CASE(13) PFE_NA_CASE(14) PFE_NA_CASE(15) PFE_NA_CASE(16)
        default:
            return PFE_EINVAL;
    }
}

// device address of g_scratch, looked up once per device (with that device current)
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char *g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

bool is_device(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace noalloc
}  // namespace pfe

extern "C" pfe_status pfe_orthonormalize_noalloc(const double *Y, const double *deg, int64_t n, int32_t d,
                                                 double *Yhat, pfe_stream_t stream) {
    using namespace pfe::noalloc;
    if (!Y || !deg || !Yhat || n < 1) return PFE_EINVAL;
    if (d < 1 || d > kMaxD || d > n) return PFE_EINVAL;  // beyond the fixed scratch size
    if (!is_device(Y) || !is_device(deg) || !is_device(Yhat)) return PFE_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PFE_ECUDA;
    unsigned char *base = nullptr;
    int sms = 0;
    {
        std::lock_guard<std::mutex> lk(g_mutex);
        if (!g_addr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return PFE_ECUDA;
            }
            int v = 0;
            if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PFE_ECUDA;
            g_addr[dev] = static_cast<unsigned char *>(ptr);
            g_sms[dev] = v;
        }
        base = g_addr[dev];
        sms = g_sms[dev];
    }
    const int64_t ntiles = (n + kTileNA - 1) / kTileNA;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, std::min(kMaxBlocks, 2 * sms)));
    return dispatch(d, Y, deg, n, Yhat, (cudaStream_t)stream, base, blocks);
}
