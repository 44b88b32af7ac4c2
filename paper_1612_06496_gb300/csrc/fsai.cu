// Learned factorised sparse approximate inverse (FSAI) preconditioner for the
// PCG solve of Eq. 13.  (The paper preconditions with incomplete Cholesky,
// Sec. III; this learned replacement has no counterpart there.)
//
//   M^{-1} = G^T G,  G lower triangular on the pattern of tril(A),
//   G_ij = Gh_ij / sqrt(A_jj),  Gh_ii = softplus(h_diag), Gh_ij = h_off,
//   (h_off, h_diag) = MLP(features of the entry), 4 -> 64 -> 64 -> 2, ReLU.
//
// One network evaluation per pattern entry: n diagonal entries and |E| edge
// entries (edge (a < b) carries G_ba).  Entry features:
//   edge:  (rho_ab, theta_b, theta_a, w_ab),  rho = lam w^2 / sqrt(A_aa A_bb),
//          theta_i = r d_i / A_ii;
//   diag:  (s_i, theta_i, theta_i, 1),  s_i = sum over lower neighbours j of rho_ij^2.
// The 64 x 64 hidden layer runs on the tensor cores (mma.sync m16n8k16, BF16
// operands, FP32 accumulation) in inference and in training; the 4 -> 64 and
// 64 -> 2 layers are FP32.  Training minimises Kaporin's condition number of
// G A G^T, L = log(tr(G A G^T)/n) - (2/n) sum log G_ii, whose gradient on the
// pattern is dL/dG_ij = 2 (A g_i)_j / tr - delta_ij 2/(n G_ii), g_i = row i of G.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace pfe {
namespace fsai {

constexpr int HW = 64;
constexpr int OW1 = 0, OB1 = 4 * HW, OW2 = OB1 + HW, OB2 = OW2 + HW * HW, OW3 = OB2 + HW, OB3 = OW3 + 2 * HW;
static_assert(OB3 + 2 == kNParam, "parameter layout");

constexpr int kMlpWarps = 4;
constexpr int kMlpThreads = 32 * kMlpWarps;

struct View {
    int64_t n, n_edges, n_slices;
    const int *slice_ptr, *col, *eid;
    const int *ea, *eb, *ext_slot;
    const double *ew, *deg, *adiag, *w64, *aoff;
    double lam, r;
    // a batch of problems: lambda of each problem, the problem of each row
    int nseg;
    const double *seg_lam;
    const int *rseg;
    // lambda of row i's problem
    __device__ __forceinline__ double lam_of(int64_t i) const { return nseg > 1 ? seg_lam[rseg[i]] : lam; }
};

View view(pfe_ctx *c) {
    View v;
    v.n = c->g.n;
    v.n_edges = c->g.n_edges;
    v.n_slices = c->g.n_slices;
    v.slice_ptr = c->g.slice_ptr;
    v.col = c->g.col;
    v.eid = c->g.eid;
    v.ea = c->g.ea;
    v.eb = c->g.eb;
    v.ext_slot = c->g.ext_slot;
    v.ew = c->g.ew;
    v.deg = c->g.deg;
    v.adiag = c->g.adiag64;
    v.w64 = c->g.w64;
    v.aoff = c->g.aoff64;
    v.lam = c->lambda;
    v.r = c->r;
    v.nseg = c->nseg;
    v.seg_lam = c->seg_lam;
    v.rseg = c->rseg;
    return v;
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// ---- per-row setup: s_i, the number of lower slots, the edge-slot -> entry map

__global__ void k_rowprep(View g, float *srow, int *kb, int *ent_of_slot) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const int64_t s = i >> 5;
    const int s0 = g.slice_ptr[s];
    const int len = (g.slice_ptr[s + 1] - s0) >> 5;
    const int64_t base = s0 + (i & 31) * (int64_t)len;  // row-major within the slice
    const double aii = g.adiag[i];
    double acc = 0.0;
    // kb = position of the first strictly upper slot (valid slots are sorted by
    // column; padding slots repeat i and may sit anywhere in a fixed-position
    // row): the lower entries are the valid slots before it
    int nb = len;
    for (int k = 0; k < len; ++k) {
        const int64_t idx = base + k;
        const int j = g.col[idx];
        if (j > i) {
            nb = k;
            break;
        }
        if (j == i || g.eid[idx] < 0) continue;  // padding
        const double w = g.w64[idx];
        const double rho = g.lam_of(i) * w * w / sqrt(aii * g.adiag[j]);
        acc = fma(rho, rho, acc);
    }
    srow[i] = (float)acc;
    kb[i] = nb;
}

__global__ void k_entmap(View g, int *ent_of_slot) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.n_edges) return;
    ent_of_slot[g.ext_slot[k]] = (int)k;
}

// features of entry e (e < n: diagonal i = e; else edge k = e - n)
__device__ __forceinline__ void features(const View &g, const float *srow, int64_t e, float f[4], int &head,
                                         float &scale) {
    if (e < g.n) {
        const double a = g.adiag[e];
        const float th = (float)(g.r * g.deg[e] / a);
        f[0] = srow[e];
        f[1] = th;
        f[2] = th;
        f[3] = 1.f;
        head = 1;
        scale = (float)(1.0 / sqrt(a));
    } else {
        const int64_t k = e - g.n;
        const int a = g.ea[k], b = g.eb[k];
        const double aa = g.adiag[a], ab = g.adiag[b], w = g.ew[k];
        f[0] = (float)(g.lam_of(a) * w * w / sqrt(aa * ab));
        f[1] = (float)(g.r * g.deg[b] / ab);
        f[2] = (float)(g.r * g.deg[a] / aa);
        f[3] = (float)w;
        head = 0;
        scale = (float)(1.0 / sqrt(aa));
    }
}

// ---- tensor-core helpers (mma.sync m16n8k16, BF16 x BF16 -> FP32) ----------

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    uint32_t u;
    memcpy(&u, &v, 4);
    return u;
}

__device__ __forceinline__ uint32_t pair_u32(const __nv_bfloat16 *p) {
    uint32_t u;
    memcpy(&u, p, 4);
    return u;
}

__device__ __forceinline__ uint32_t pair_strided(const __nv_bfloat16 *p0, const __nv_bfloat16 *p1) {
    __nv_bfloat162 v;
    v.x = *p0;
    v.y = *p1;
    uint32_t u;
    memcpy(&u, &v, 4);
    return u;
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Shared-memory weights of one block.
struct SmemW {
    float W1[4 * HW], b1[HW], b2[HW], W3[HW * 2], b3[4];
    __nv_bfloat16 W2t[HW * HW];  // [n = h2 unit][k = h1 unit]: B operand of h1 @ W2
    __nv_bfloat16 W2r[HW * HW];  // [n = h1 unit][k = h2 unit]: B operand of da2 @ W2^T
};

__device__ void load_weights(SmemW &s, const float *__restrict__ P) {
    for (int t = threadIdx.x; t < 4 * HW; t += blockDim.x) s.W1[t] = P[OW1 + t];
    for (int t = threadIdx.x; t < HW; t += blockDim.x) {
        s.b1[t] = P[OB1 + t];
        s.b2[t] = P[OB2 + t];
    }
    for (int t = threadIdx.x; t < 2 * HW; t += blockDim.x) s.W3[t] = P[OW3 + t];
    if (threadIdx.x < 2) s.b3[threadIdx.x] = P[OB3 + threadIdx.x];
    for (int t = threadIdx.x; t < HW * HW; t += blockDim.x) {
        const int k = t / HW, n = t % HW;  // W2[k][n], k = h1 unit, n = h2 unit
        const __nv_bfloat16 v = __float2bfloat16_rn(P[OW2 + t]);
        s.W2t[n * HW + k] = v;
        s.W2r[k * HW + n] = v;
    }
}

// Per-warp tile scratch.
struct SmemTile {
    float f[16][4];
    int head[16];
    float scale[16];
    float hv[16];  // raw head value
    __nv_bfloat16 h1[16][HW];
    __nv_bfloat16 da2b[16][HW];
    float h2[16][HW];
    float da2[16][HW];
    float da1[16][HW];
    float dout[16];
};

// Forward of one 16-entry tile.  Leaves h1 (bf16) in smem, a2 (pre-ReLU) in
// the C fragments acc[nt][0..3] (rows gid, gid+8; units 8nt + 2tig + {0,1}).
__device__ __forceinline__ void tile_forward(const SmemW &W, SmemTile &T, float (&acc)[8][4]) {
    const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
    // layer 1 (FP32): lane handles units lane and lane + 32 of all 16 entries
    for (int uu = 0; uu < 2; ++uu) {
        const int u = lane + 32 * uu;
        for (int e = 0; e < 16; ++e) {
            float a = W.b1[u];
#pragma unroll
            for (int k = 0; k < 4; ++k) a = fmaf(T.f[e][k], W.W1[k * HW + u], a);
            T.h1[e][u] = __float2bfloat16_rn(fmaxf(a, 0.f));
        }
    }
    __syncwarp();
    // layer 2 on the tensor cores: a2 = h1 @ W2 + b2
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int u0 = 8 * nt + 2 * tig;
        acc[nt][0] = W.b2[u0];
        acc[nt][1] = W.b2[u0 + 1];
        acc[nt][2] = W.b2[u0];
        acc[nt][3] = W.b2[u0 + 1];
    }
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
        uint32_t a[4];
        const int k0 = 16 * ks + 2 * tig;
        a[0] = pair_u32(&T.h1[gid][k0]);
        a[1] = pair_u32(&T.h1[gid + 8][k0]);
        a[2] = pair_u32(&T.h1[gid][k0 + 8]);
        a[3] = pair_u32(&T.h1[gid + 8][k0 + 8]);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            uint32_t b[2];
            const int n = 8 * nt + gid;
            b[0] = pair_u32(&W.W2t[n * HW + k0]);
            b[1] = pair_u32(&W.W2t[n * HW + k0 + 8]);
            mma_bf16(acc[nt], a, b);
        }
    }
}

// Output heads of the tile rows gid and gid + 8 (valid on lanes with tig == 0).
__device__ __forceinline__ void tile_heads(const SmemW &W, SmemTile &T, const float (&acc)[8][4]) {
    const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
    const int h0 = T.head[gid], h1 = T.head[gid + 8];
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int u0 = 8 * nt + 2 * tig;
        s0 = fmaf(fmaxf(acc[nt][0], 0.f), W.W3[u0 * 2 + h0], s0);
        s0 = fmaf(fmaxf(acc[nt][1], 0.f), W.W3[(u0 + 1) * 2 + h0], s0);
        s1 = fmaf(fmaxf(acc[nt][2], 0.f), W.W3[u0 * 2 + h1], s1);
        s1 = fmaf(fmaxf(acc[nt][3], 0.f), W.W3[(u0 + 1) * 2 + h1], s1);
    }
    s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
    s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
    if (tig == 0) {
        T.hv[gid] = s0 + W.b3[h0];
        T.hv[gid + 8] = s1 + W.b3[h1];
    }
    __syncwarp();
}

__device__ __forceinline__ float softplusf(float x) { return x > 20.f ? x : log1pf(expf(x)); }
__device__ __forceinline__ float sigmoidf(float x) { return 1.f / (1.f + expf(-x)); }

// Inference: G entries for every pattern entry.  gdiag[i] = G_ii, gE[edge
// slot] = G_ba; hraw[e] = the network's head value (training reuses it).
__global__ void __launch_bounds__(kMlpThreads) k_mlp_fwd(View g, const float *srow, const float *__restrict__ P,
                                                         float *gdiag, float *gE, float *hraw) {
    extern __shared__ __align__(16) unsigned char smem[];
    SmemW &W = *reinterpret_cast<SmemW *>(smem);
    SmemTile &T = reinterpret_cast<SmemTile *>(smem + sizeof(SmemW))[threadIdx.x >> 5];
    load_weights(W, P);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t N = g.n + g.n_edges, ntiles = (N + 15) / 16;
    const int64_t warp_g = (int64_t)blockIdx.x * kMlpWarps + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * kMlpWarps;
    for (int64_t t = warp_g; t < ntiles; t += nwarps) {
        if (lane < 16) {
            const int64_t e = t * 16 + lane;
            if (e < N) {
                features(g, srow, e, T.f[lane], T.head[lane], T.scale[lane]);
            } else {
                T.f[lane][0] = T.f[lane][1] = T.f[lane][2] = T.f[lane][3] = 0.f;
                T.head[lane] = 0;
                T.scale[lane] = 0.f;
            }
        }
        __syncwarp();
        float acc[8][4];
        tile_forward(W, T, acc);
        tile_heads(W, T, acc);
        if (lane < 16) {
            const int64_t e = t * 16 + lane;
            if (e < N) {
                const float h = T.hv[lane];
                hraw[e] = h;
                if (e < g.n)
                    gdiag[e] = softplusf(h) * T.scale[lane];
                else
                    gE[g.ext_slot[e - g.n]] = h * T.scale[lane];
            }
        }
        __syncwarp();
    }
}

// ---- the network's inference on the 5th-generation tensor cores (tcgen05) -----
// One CTA of 128 threads takes 128 pattern entries at a time.  Layer 1 (4 ->
// 64, FP32) and the ReLU run one entry per thread and write h1 as BF16 into
// shared memory; the 64 x 64 layer is one 128 x 64 x 64 MMA (tcgen05.mma
// kind::f16, BF16 operands, FP32 accumulator in tensor memory, issued by one
// thread as four K = 16 steps); thread t reads its entry's 64 accumulators
// back from TMEM lane t (tcgen05.ld 32x32b) for the bias, ReLU and the two
// heads.  Operands use the no-swizzle K-major layout: 8-row x 16-byte core
// matrices, the K-adjacent ones 128 bytes apart (leading-dimension offset),
// the next 8 rows 1024 bytes on (stride offset).
constexpr int kTcRows = 128;   // entries per tile: the MMA's M
constexpr int kTcCols = 64;    // TMEM columns of the FP32 accumulator (N = 64)

struct SmemTc {
    __nv_bfloat16 A[kTcRows * HW];  // h1, 16 KB (1024-byte aligned)
    __nv_bfloat16 B[HW * HW];       // W2 as N x K (n = h2 unit, k = h1 unit), 8 KB
    float W1[4 * HW], b1[HW], b2[HW], W3[HW * 2], b3[4];
    unsigned long long mbar;
    unsigned tmem_base;
    int ok;
};
constexpr size_t kSmemTc = sizeof(SmemTc) + 1024;  // + the alignment slack

// byte offset of element (r, k) of an R x 64 BF16 operand in the layout above
__device__ __forceinline__ int tc_off(int r, int k) { return (r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor (tcgen05): start address, leading- and
// stride-dimension byte offsets (all >> 4), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = 64, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(HW >> 3) << 17) |
                              ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ bool tc_mbar_wait(uint32_t mbar, uint32_t parity) {
    // bounded: give up after about a second of device time
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 1000000000ull) return false;
    }
}

__global__ void __launch_bounds__(kTcRows, 4) k_mlp_fwd_tc(View g, const float *srow, const float *__restrict__ P,
                                                          float *gdiag, float *gE, float *hraw, unsigned *err) {
    extern __shared__ unsigned char smem_raw[];
    SmemTc &S = *reinterpret_cast<SmemTc *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5;
    unsigned char *Ab = reinterpret_cast<unsigned char *>(S.A);
    unsigned char *Bb = reinterpret_cast<unsigned char *>(S.B);
    for (int t = tid; t < 4 * HW; t += blockDim.x) S.W1[t] = P[OW1 + t];
    for (int t = tid; t < HW; t += blockDim.x) {
        S.b1[t] = P[OB1 + t];
        S.b2[t] = P[OB2 + t];
    }
    for (int t = tid; t < 2 * HW; t += blockDim.x) S.W3[t] = P[OW3 + t];
    if (tid < 2) S.b3[tid] = P[OB3 + tid];
    for (int t = tid; t < HW * HW; t += blockDim.x) {
        const int k = t / HW, n = t % HW;  // W2[k][n]
        *reinterpret_cast<__nv_bfloat16 *>(Bb + tc_off(n, k)) = __float2bfloat16_rn(P[OW2 + t]);
    }
    const uint32_t mbar = smem_u32(&S.mbar);
    if (tid == 0) {
        S.ok = 1;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {  // 64 TMEM columns for the accumulator
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&S.tmem_base)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // W2 written by the generic proxy
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = S.tmem_base;
    const uint32_t abase = smem_u32(S.A), bbase = smem_u32(S.B);
    const int64_t N = g.n + g.n_edges, ntiles = (N + kTcRows - 1) / kTcRows;
    uint32_t parity = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t e = tile * kTcRows + tid;
        float f[4] = {0.f, 0.f, 0.f, 0.f}, scale = 0.f;
        int head = 0;
        if (e < N) features(g, srow, e, f, head, scale);
        // layer 1 (FP32) into the A operand
#pragma unroll 8
        for (int u = 0; u < HW; ++u) {
            float a = S.b1[u];
#pragma unroll
            for (int k = 0; k < 4; ++k) a = fmaf(f[k], S.W1[k * HW + u], a);
            *reinterpret_cast<__nv_bfloat16 *>(Ab + tc_off(tid, u)) = __float2bfloat16_rn(fmaxf(a, 0.f));
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int ks = 0; ks < HW / 16; ++ks) {  // K = 16 a step: two core matrices along K
                const uint64_t ad = tc_desc(abase + ks * 256, 128, 1024);
                const uint64_t bd = tc_desc(bbase + ks * 256, 128, 1024);
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr),
                    "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(ks)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                         : "memory");
        }
        const bool ok = __syncthreads_and(tc_mbar_wait(mbar, parity)) != 0;
        parity ^= 1u;
        if (!ok) {  // the accumulator never arrived: report, leave (block-uniform)
            if (tid == 0) {
                atomicExch(err, 1u);
                S.ok = 0;
            }
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // epilogue: this thread's entry is TMEM lane 32 warp + lane = row tid
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < HW / 16; ++c) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr + ((uint32_t)(32 * warp) << 16) + (uint32_t)(16 * c)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int u = 16 * c + j;
                s = fmaf(fmaxf(__uint_as_float(r[j]) + S.b2[u], 0.f), S.W3[u * 2 + head], s);
            }
        }
        if (e < N) {
            const float h = s + S.b3[head];
            hraw[e] = h;
            if (e < g.n)
                gdiag[e] = softplusf(h) * scale;
            else
                gE[g.ext_slot[e - g.n]] = h * scale;
        }
        // every thread's TMEM reads are done before the next tile's MMA overwrites
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
    }
    // an MMA still in flight after a time-out gets a second bounded wait
    if (!S.ok && tid == 0) tc_mbar_wait(mbar, parity ^ 1u);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(kTcCols) : "memory");
}

// G values per SELL slot (both orientations of an edge carry G_ba) so that
// the PCG apply kernels read them coalesced.
__global__ void k_gslots(View g, const float *gE, float *gslot) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if ((i >> 5) >= g.n_slices) return;
    const int64_t s = i >> 5;
    const int s0 = g.slice_ptr[s];
    const int len = (g.slice_ptr[s + 1] - s0) >> 5;
    const int64_t base = s0 + (i & 31) * (int64_t)len;  // row-major within the slice
    for (int k = 0; k < len; ++k) {
        const int64_t idx = base + k;
        const int e = g.eid[idx];
        gslot[idx] = e >= 0 ? gE[e] : 0.f;
    }
}

// Kaporin row terms: q_i = g_i^T A g_i and dq_i/dG_ij = 2 (A g_i)_j for the
// entries of row i (j = i and the lower neighbours), with
// (A g_i)_j = lam sum_{k ~ j} w_jk^2 (g_ij - g_ik) + r d_j g_ij,  g_ik = 0 off the row pattern.
constexpr int kMaxLower = 64;
__global__ void k_kaporin_rows(View g, const int *kb, const float *gdiag, const float *gslot, const int *ent_of_slot,
                               float *dq, double *qrow, double *logd) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const int64_t s = i >> 5;
    const int s0 = g.slice_ptr[s];
    const int len_i = (g.slice_ptr[s + 1] - s0) >> 5;
    const int64_t base = s0 + (i & 31) * (int64_t)len_i;
    // the valid lower entries (padding slots skipped), at most kMaxLower
    int cols[kMaxLower + 1], slot_of[kMaxLower];
    float vals[kMaxLower + 1];
    int nl = 0;
    for (int k = 0; k < kb[i] && nl < kMaxLower; ++k) {
        const int64_t idx = base + k;
        if (g.eid[idx] < 0 || g.col[idx] >= i) continue;
        cols[nl] = g.col[idx];
        vals[nl] = gslot[idx];
        slot_of[nl] = k;
        ++nl;
    }
    cols[nl] = (int)i;
    vals[nl] = gdiag[i];
    double q = 0.0;
    for (int m = 0; m <= nl; ++m) {
        const int j = cols[m];
        const double gij = vals[m];
        // (A g_i)_j over row j's slots
        const int64_t sj = (int64_t)j >> 5;
        const int t0 = g.slice_ptr[sj];
        const int lj = (g.slice_ptr[sj + 1] - t0) >> 5;
        const int64_t bj = t0 + (j & 31) * (int64_t)lj;
        double agj = g.r * g.deg[j] * gij;
        for (int k = 0; k < lj; ++k) {
            const int64_t idx = bj + k;
            if (g.eid[idx] < 0) continue;
            const int kk = g.col[idx];
            double gik = 0.0;
            for (int u = 0; u <= nl; ++u)
                if (cols[u] == kk) {
                    gik = vals[u];
                    break;
                }
            const double w = g.w64[idx];
            agj += g.lam_of(j) * w * w * (gij - gik);
        }
        q = fma(gij, agj, q);
        const float d = (float)(2.0 * agj);
        if (m == nl) {
            dq[i] = d;  // diagonal entry i
        } else {
            const int64_t idx = base + slot_of[m];
            dq[g.n + ent_of_slot[g.eid[idx]]] = d;  // edge entry (j, i): G_ij
        }
    }
    qrow[i] = q;
    logd[i] = log((double)gdiag[i]);
}

// Deterministic sum of two n-vectors: out[0] = sum q, out[1] = sum log G_ii.
__global__ void k_sum2(int64_t n, const double *a, const double *b, double *part, unsigned *ticket, double *out) {
    double s[2] = {0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        s[0] += a[i];
        s[1] += b[i];
    }
    block_reduce<double, 2>(s, part + 2 * blockIdx.x);
    if (last_block_arrives(ticket)) {
        if (threadIdx.x < 2) {
            double t = 0.0;
            for (unsigned k = 0; k < gridDim.x; ++k) t += __ldcg(part + 2 * k + threadIdx.x);
            out[threadIdx.x] = t;
        }
        __syncthreads();
        if (threadIdx.x == 0) *ticket = 0u;
    }
}

// ---- right-hand-side residual term: R = (1/m) sum_c |A G^T G b_c - b_c|^2 / |b_c|^2
// over m right-hand sides the method produced (n x m, row-major, FP64).
// u = G b, v = G^T u, w = A v - b, s = 2 mu A w / (m |b|^2) (A symmetric); the
// gradient on G's pattern is dR/dG_ij = u_i s_j + (G s)_i b_j.
constexpr int kMaxRhs = 32;

// out = G x (MODE 0: G_ii and the lower slots [0, kb_i)), G^T x (MODE 1: G_ii
// and the upper slots [kb_i, len), which hold the transposed entries), or
// A x in FP64 (MODE 2); one thread per (row, column).  Padding slots carry 0.
template <int MODE>
__global__ void k_rg_apply(View g, const int *kb, const float *gdiag, const float *gslot, const double *x, int m,
                           double *out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.n * m) return;
    const int64_t i = k / m;
    const int c = (int)(k - i * m);
    const int64_t sl = i >> 5;
    const int s0 = g.slice_ptr[sl];
    const int len = (g.slice_ptr[sl + 1] - s0) >> 5;
    const int64_t base = s0 + (i & 31) * (int64_t)len;
    const int lo = MODE == 1 ? kb[i] : 0, hi = MODE == 0 ? kb[i] : len;
    double acc = (MODE == 2 ? g.adiag[i] : (double)gdiag[i]) * x[k];
    for (int t = lo; t < hi; ++t) {
        const double v = MODE == 2 ? g.aoff[base + t] : (double)gslot[base + t];
        acc = fma(v, x[(int64_t)g.col[base + t] * m + c], acc);
    }
    out[k] = acc;
}

// w -= b, and the column sums |w_c|^2 (out[c]) and |b_c|^2 (out[m + c]):
// block partials, the last block adds them in block order.
__global__ void k_rg_resid(int64_t n, int m, const double *b, double *w, double *part, unsigned *ticket, double *out) {
    double acc[2 * kMaxRhs];
    for (int c = 0; c < 2 * m; ++c) acc[c] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int c = 0; c < m; ++c) {
            const double bv = b[i * m + c], wv = w[i * m + c] - bv;
            w[i * m + c] = wv;
            acc[c] = fma(wv, wv, acc[c]);
            acc[m + c] = fma(bv, bv, acc[m + c]);
        }
    __shared__ double red[256];
    for (int c = 0; c < 2 * m; ++c) {
        red[threadIdx.x] = acc[c];
        __syncthreads();
        for (int h = blockDim.x / 2; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * 2 * m + c] = red[0];
        __syncthreads();
    }
    if (last_block_arrives(ticket)) {
        for (int c = threadIdx.x; c < 2 * m; c += blockDim.x) {
            double t = 0.0;
            for (unsigned k = 0; k < gridDim.x; ++k) t += __ldcg(part + (int64_t)k * 2 * m + c);
            out[c] = t;
        }
        __syncthreads();
        if (threadIdx.x == 0) *ticket = 0u;
    }
}

// s (= A w on entry) *= 2 mu / (m |b_c|^2)
__global__ void k_rg_scale(int64_t n, int m, const double *sq, double mu, double *s) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n * m) return;
    const int c = (int)(k % m);
    s[k] *= 2.0 * mu / ((double)m * sq[m + c]);
}

// Gradient of the term per pattern entry (the entry order of dq): diagonal
// entry i, then edge k = (a_k, b_k), a < b, entry G_{b a}:
//   dR/dG_ij = sum_c u_ic s_jc + (G s)_ic b_jc.
__global__ void k_rg_entries(View g, int m, const double *u, const double *s, const double *gs, const double *b,
                             float *drhs) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= g.n + g.n_edges) return;
    const int64_t i = e < g.n ? e : g.eb[e - g.n], j = e < g.n ? e : g.ea[e - g.n];
    double t = 0.0;
    for (int c = 0; c < m; ++c) t += u[i * m + c] * s[j * m + c] + gs[i * m + c] * b[j * m + c];
    drhs[e] = (float)t;
}

// dL/dh per entry from dq (in place): L = log(Q/n) - (2/n) sum log G_ii
// (+ the right-hand-side term's dL/dG_ij, drhs, when given).
__global__ void k_dloss(View g, const double *sums, const float *gdiag, const float *hraw, float *dq,
                        const float *drhs) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = g.n + g.n_edges;
    if (e >= N) return;
    const double Q = sums[0];
    double dG = dq[e] / Q;
    if (drhs) dG += drhs[e];
    if (e < g.n) {
        dG -= 2.0 / ((double)g.n * gdiag[e]);
        const double h = hraw[e];
        dq[e] = (float)(dG / (1.0 + exp(-h)) / sqrt(g.adiag[e]));  // dG/dh = sigmoid(h)/sqrt(A_ii)
    } else {
        dq[e] = (float)(dG / sqrt(g.adiag[g.ea[e - g.n]]));       // dG/dh = 1/sqrt(A_aa)
    }
}

// Backward through the network for every entry, given dL/dh per entry.
// Block partials of the parameter gradient (kNParam floats per block) are
// reduced by the last block in a fixed order.
__global__ void __launch_bounds__(kMlpThreads) k_mlp_bwd(View g, const float *srow, const float *__restrict__ P,
                                                         const float *dh, float *part, unsigned *ticket,
                                                         float *grad) {
    extern __shared__ __align__(16) unsigned char smem[];
    SmemW &W = *reinterpret_cast<SmemW *>(smem);
    SmemTile *Tall = reinterpret_cast<SmemTile *>(smem + sizeof(SmemW));
    SmemTile &T = Tall[threadIdx.x >> 5];
    float *blk = reinterpret_cast<float *>(smem + sizeof(SmemW) + kMlpWarps * sizeof(SmemTile));  // kNParam
    load_weights(W, P);
    for (int t = threadIdx.x; t < kNParam; t += blockDim.x) blk[t] = 0.f;
    __syncthreads();
    const int lane = threadIdx.x & 31, gid = lane >> 2, tig = lane & 3;
    const int64_t N = g.n + g.n_edges, ntiles = (N + 15) / 16;
    const int64_t warp_g = (int64_t)blockIdx.x * kMlpWarps + (threadIdx.x >> 5);
    const int64_t nwarps = (int64_t)gridDim.x * kMlpWarps;
    float gw2[4][8][4];  // tensor-core accumulator of h1^T da2 (rows h1 unit, cols h2 unit)
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) gw2[mt][nt][0] = gw2[mt][nt][1] = gw2[mt][nt][2] = gw2[mt][nt][3] = 0.f;
    float gw1[4][2] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}}, gb1[2] = {0.f, 0.f};
    float gw3[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, gb2[2] = {0.f, 0.f}, gb3[2] = {0.f, 0.f};
    for (int64_t t = warp_g; t < ntiles; t += nwarps) {
        if (lane < 16) {
            const int64_t e = t * 16 + lane;
            if (e < N) {
                features(g, srow, e, T.f[lane], T.head[lane], T.scale[lane]);
                T.dout[lane] = dh[e];
            } else {
                T.f[lane][0] = T.f[lane][1] = T.f[lane][2] = T.f[lane][3] = 0.f;
                T.head[lane] = 0;
                T.scale[lane] = 0.f;
                T.dout[lane] = 0.f;
            }
        }
        __syncwarp();
        float acc[8][4];
        tile_forward(W, T, acc);
        // da2 = (dout * W3[:, head]) masked by a2 > 0; h2 kept for gW3
        const int h0 = T.head[gid], h1r = T.head[gid + 8];
        const float d0 = T.dout[gid], d1 = T.dout[gid + 8];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
            const int u0 = 8 * nt + 2 * tig;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int u = u0 + q;
                const float a_lo = acc[nt][q], a_hi = acc[nt][2 + q];
                const float g_lo = a_lo > 0.f ? d0 * W.W3[u * 2 + h0] : 0.f;
                const float g_hi = a_hi > 0.f ? d1 * W.W3[u * 2 + h1r] : 0.f;
                T.h2[gid][u] = fmaxf(a_lo, 0.f);
                T.h2[gid + 8][u] = fmaxf(a_hi, 0.f);
                T.da2[gid][u] = g_lo;
                T.da2[gid + 8][u] = g_hi;
                T.da2b[gid][u] = __float2bfloat16_rn(g_lo);
                T.da2b[gid + 8][u] = __float2bfloat16_rn(g_hi);
            }
        }
        __syncwarp();
        // gW2 += h1^T da2 on the tensor cores (K = the 16 entries of the tile)
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            uint32_t a[4];
            const int m0 = 16 * mt + gid;
            const int k0 = 2 * tig;
            a[0] = pair_strided(&T.h1[k0][m0], &T.h1[k0 + 1][m0]);
            a[1] = pair_strided(&T.h1[k0][m0 + 8], &T.h1[k0 + 1][m0 + 8]);
            a[2] = pair_strided(&T.h1[k0 + 8][m0], &T.h1[k0 + 9][m0]);
            a[3] = pair_strided(&T.h1[k0 + 8][m0 + 8], &T.h1[k0 + 9][m0 + 8]);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                uint32_t b[2];
                const int n = 8 * nt + gid;
                b[0] = pair_strided(&T.da2b[k0][n], &T.da2b[k0 + 1][n]);
                b[1] = pair_strided(&T.da2b[k0 + 8][n], &T.da2b[k0 + 9][n]);
                mma_bf16(gw2[mt][nt], a, b);
            }
        }
        // dh1 = da2 @ W2^T on the tensor cores
        float dh1[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) dh1[nt][0] = dh1[nt][1] = dh1[nt][2] = dh1[nt][3] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            uint32_t a[4];
            const int k0 = 16 * ks + 2 * tig;
            a[0] = pair_u32(&T.da2b[gid][k0]);
            a[1] = pair_u32(&T.da2b[gid + 8][k0]);
            a[2] = pair_u32(&T.da2b[gid][k0 + 8]);
            a[3] = pair_u32(&T.da2b[gid + 8][k0 + 8]);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                uint32_t b[2];
                const int n = 8 * nt + gid;
                b[0] = pair_u32(&W.W2r[n * HW + k0]);
                b[1] = pair_u32(&W.W2r[n * HW + k0 + 8]);
                mma_bf16(dh1[nt], a, b);
            }
        }
        // da1 = dh1 masked by a1 > 0 (a1 recomputed in FP32)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int u = 8 * nt + 2 * tig + q;
#pragma unroll
                for (int hr = 0; hr < 2; ++hr) {
                    const int row = gid + 8 * hr;
                    float a1 = W.b1[u];
#pragma unroll
                    for (int k = 0; k < 4; ++k) a1 = fmaf(T.f[row][k], W.W1[k * HW + u], a1);
                    T.da1[row][u] = a1 > 0.f ? dh1[nt][2 * hr + q] : 0.f;
                }
            }
        }
        __syncwarp();
        // FP32 small layers: lane owns units lane and lane + 32
#pragma unroll
        for (int uu = 0; uu < 2; ++uu) {
            const int u = lane + 32 * uu;
            for (int e = 0; e < 16; ++e) {
                const float da1 = T.da1[e][u];
#pragma unroll
                for (int k = 0; k < 4; ++k) gw1[k][uu] = fmaf(T.f[e][k], da1, gw1[k][uu]);
                gb1[uu] += da1;
                gb2[uu] += T.da2[e][u];
                const float hd = T.h2[e][u] * T.dout[e];
                gw3[uu][T.head[e]] += hd;
            }
        }
        if (lane < 2) {
            for (int e = 0; e < 16; ++e)
                if (T.head[e] == lane) gb3[lane] += T.dout[e];
        }
        __syncwarp();
    }
    // warp results -> block sums (fixed warp order)
    for (int w = 0; w < kMlpWarps; ++w) {
        if ((threadIdx.x >> 5) == w) {
#pragma unroll
            for (int mt = 0; mt < 4; ++mt)
#pragma unroll
                for (int nt = 0; nt < 8; ++nt) {
                    const int r0 = 16 * mt + gid, c0 = 8 * nt + 2 * tig;
                    blk[OW2 + r0 * HW + c0] += gw2[mt][nt][0];
                    blk[OW2 + r0 * HW + c0 + 1] += gw2[mt][nt][1];
                    blk[OW2 + (r0 + 8) * HW + c0] += gw2[mt][nt][2];
                    blk[OW2 + (r0 + 8) * HW + c0 + 1] += gw2[mt][nt][3];
                }
#pragma unroll
            for (int uu = 0; uu < 2; ++uu) {
                const int u = lane + 32 * uu;
#pragma unroll
                for (int k = 0; k < 4; ++k) blk[OW1 + k * HW + u] += gw1[k][uu];
                blk[OB1 + u] += gb1[uu];
                blk[OB2 + u] += gb2[uu];
                blk[OW3 + u * 2] += gw3[uu][0];
                blk[OW3 + u * 2 + 1] += gw3[uu][1];
            }
            if (lane < 2) blk[OB3 + lane] += gb3[lane];
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < kNParam; t += blockDim.x) part[(int64_t)blockIdx.x * kNParam + t] = blk[t];
    if (last_block_arrives(ticket)) {
        for (int t = threadIdx.x; t < kNParam; t += blockDim.x) {
            float s = 0.f;
            for (unsigned b = 0; b < gridDim.x; ++b) s += __ldcg(part + (int64_t)b * kNParam + t);
            grad[t] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) *ticket = 0u;
    }
}

__global__ void k_adam(int64_t cnt, float *p, const float *gr, float *m, float *v, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cnt) return;
    const float gk = gr[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

// Classical FSAI (the comparator of the learned factor): for row i with
// pattern S = {lower neighbours of i} + {i} (i last), solve A[S,S] g = e_i by
// an FP64 Cholesky factorisation and scale g by 1/sqrt(g_i).  This G is the
// minimiser of the Kaporin number of G A G^T over the same pattern.
constexpr int kMaxS = 24;
__global__ void k_fsai_classical(View g, const int *kb, float *gdiag, float *gE, int *err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const int64_t s = i >> 5;
    const int s0 = g.slice_ptr[s];
    const int len_i = (g.slice_ptr[s + 1] - s0) >> 5;
    const int64_t base = s0 + (i & 31) * (int64_t)len_i;
    int S[kMaxS], slot_of[kMaxS];
    int nl = 0;  // the valid lower entries (padding slots skipped)
    for (int k = 0; k < kb[i]; ++k) {
        const int64_t idx = base + k;
        if (g.eid[idx] < 0 || g.col[idx] >= i) continue;
        if (nl + 1 >= kMaxS) {
            atomicExch(err, 1);
            return;
        }
        S[nl] = g.col[idx];
        slot_of[nl] = k;
        ++nl;
    }
    const int m = nl + 1;
    S[nl] = (int)i;
    double Ls[kMaxS * kMaxS];
    // A[S,S]: diagonal from A_jj, off-diagonal by searching row S[p]'s slots
    for (int p = 0; p < m; ++p) {
        const int j = S[p];
        const int64_t sj = (int64_t)j >> 5;
        const int t0 = g.slice_ptr[sj];
        const int lj = (g.slice_ptr[sj + 1] - t0) >> 5;
        const int64_t bj = t0 + (j & 31) * (int64_t)lj;
        for (int q = 0; q < m; ++q) {
            double v = 0.0;
            if (q == p) {
                v = g.adiag[j];
            } else {
                const int k = S[q];
                for (int t = 0; t < lj; ++t) {
                    const int64_t idx = bj + t;
                    if (g.eid[idx] >= 0 && g.col[idx] == k) {
                        const double w = g.w64[idx];
                        v = -g.lam_of(j) * w * w;
                        break;
                    }
                }
            }
            Ls[p * kMaxS + q] = v;
        }
    }
    // Cholesky A = L L^T (lower part of Ls)
    for (int p = 0; p < m; ++p) {
        double d = Ls[p * kMaxS + p];
        for (int k = 0; k < p; ++k) d -= Ls[p * kMaxS + k] * Ls[p * kMaxS + k];
        if (!(d > 0.0)) {
            atomicExch(err, 2);
            return;
        }
        d = sqrt(d);
        Ls[p * kMaxS + p] = d;
        for (int q = p + 1; q < m; ++q) {
            double v = Ls[q * kMaxS + p];
            for (int k = 0; k < p; ++k) v -= Ls[q * kMaxS + k] * Ls[p * kMaxS + k];
            Ls[q * kMaxS + p] = v / d;
        }
    }
    // solve L y = e_last, L^T x = y
    double x[kMaxS];
    for (int p = 0; p < m; ++p) {
        double v = (p == m - 1) ? 1.0 : 0.0;
        for (int k = 0; k < p; ++k) v -= Ls[p * kMaxS + k] * x[k];
        x[p] = v / Ls[p * kMaxS + p];
    }
    for (int p = m - 1; p >= 0; --p) {
        double v = x[p];
        for (int k = p + 1; k < m; ++k) v -= Ls[k * kMaxS + p] * x[k];
        x[p] = v / Ls[p * kMaxS + p];
    }
    const double sc = 1.0 / sqrt(x[m - 1]);
    gdiag[i] = (float)(x[m - 1] * sc);
    for (int k = 0; k < nl; ++k) gE[g.eid[base + slot_of[k]]] = (float)(x[k] * sc);
}

__global__ void k_export(View g, const float *gdiag, const float *gE, double *od, double *oe) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < g.n && od) od[k] = gdiag[k];
    if (k < g.n_edges && oe) oe[k] = gE[g.ext_slot[k]];
}

size_t smem_fwd() { return sizeof(SmemW) + kMlpWarps * sizeof(SmemTile); }
size_t smem_bwd() { return sizeof(SmemW) + kMlpWarps * sizeof(SmemTile) + kNParam * sizeof(float); }

}  // namespace fsai

using namespace fsai;

// Allocate the FSAI buffers of a context once.
pfe_status fsai_alloc(pfe_ctx *c) {
    auto &f = c->fsai;
    if (f.gdiag) return PFE_OK;
    const int64_t n = c->g.n, ne = c->g.n_edges, N = n + ne;
    // all or nothing: a failure frees what this call allocated, so a later
    // call starts again from no buffers
    const size_t n_allocs0 = c->dev_allocs.size();
    const int64_t bytes0 = c->bytes;
    bool capped = false;
    auto al = [&](void **p, size_t bytes) -> bool {
        if (over_device_cap(c, bytes)) {
            capped = true;
            return false;
        }
        if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return false;
        }
        c->dev_allocs.push_back(*p);
        c->bytes += (int64_t)bytes;
        return true;
    };
    int nb = std::min<int64_t>((N + 63) / 64, (int64_t)c->num_sms * 2);
    f.mlp_blocks = std::max(1, nb);
    if (!al((void **)&f.gdiag, n * sizeof(float)) || !al((void **)&f.gE, std::max<int64_t>(c->g.fslots, 1) * sizeof(float)) ||
        !al((void **)&f.gslot, c->g.slots * sizeof(float)) || !al((void **)&f.srow, n * sizeof(float)) ||
        !al((void **)&f.kb, n * sizeof(int)) || !al((void **)&f.ent_of_slot, std::max<int64_t>(c->g.fslots, 1) * sizeof(int)) ||
        !al((void **)&f.hraw, N * sizeof(float)) || !al((void **)&f.dq, N * sizeof(float)) ||
        !al((void **)&f.qrow, n * sizeof(double)) || !al((void **)&f.logd, n * sizeof(double)) ||
        !al((void **)&f.sums, 4 * sizeof(double)) || !al((void **)&f.part, 512 * sizeof(double)) ||
        !al((void **)&f.gpart, (size_t)f.mlp_blocks * kNParam * sizeof(float)) ||
        !al((void **)&f.tick, 4 * sizeof(unsigned)) || !al((void **)&f.params, kNParam * sizeof(float)) ||
        !al((void **)&f.grad, kNParam * sizeof(float))) {
        for (size_t k = n_allocs0; k < c->dev_allocs.size(); ++k) cudaFree(c->dev_allocs[k]);
        c->dev_allocs.resize(n_allocs0);
        c->bytes = bytes0;
        f.gdiag = f.gE = f.gslot = f.srow = f.hraw = f.dq = f.gpart = f.params = f.grad = nullptr;
        f.kb = f.ent_of_slot = nullptr;
        f.qrow = f.logd = f.sums = f.part = nullptr;
        f.tick = nullptr;
        if (!capped) c->err = "FSAI buffers: cudaMalloc failed";
        return PFE_ENOMEM;
    }
    cudaStream_t s = c->stream;
    PFE_CUDA_TRY(c, cudaMemsetAsync(f.tick, 0, 4 * sizeof(unsigned), s));
    PFE_CUDA_TRY(c, cudaMemsetAsync(f.gE, 0, std::max<int64_t>(c->g.fslots, 1) * sizeof(float), s));
    View v = view(c);
    k_rowprep<<<nblk(n, 256), 256, 0, s>>>(v, f.srow, f.kb, f.ent_of_slot);
    k_entmap<<<nblk(std::max<int64_t>(ne, 1), 256), 256, 0, s>>>(v, f.ent_of_slot);
    PFE_CUDA_TRY(c, cudaGetLastError());
    PFE_CUDA_TRY(c, cudaFuncSetAttribute(k_mlp_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_fwd()));
    PFE_CUDA_TRY(c, cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemTc));
    PFE_CUDA_TRY(c, cudaFuncSetAttribute(k_mlp_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bwd()));
    return PFE_OK;
}

// G from the parameters in f.params (device, FP32).
pfe_status fsai_infer(pfe_ctx *c) {
    auto &f = c->fsai;
    cudaStream_t s = c->stream;
    View v = view(c);
    if (f.mlp_tc) {
        // 5th-generation tensor cores: one 128-entry tile per CTA step, at
        // most four CTAs (256 TMEM columns) per SM
        unsigned *err = f.tick + 3;
        PFE_CUDA_TRY(c, cudaMemsetAsync(err, 0, sizeof(unsigned), s));
        const int64_t ntiles = (c->g.n + c->g.n_edges + kTcRows - 1) / kTcRows;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)c->num_sms * 4));
        k_mlp_fwd_tc<<<grid, kTcRows, kSmemTc, s>>>(v, f.srow, f.params, f.gdiag, f.gE, f.hraw, err);
        PFE_CUDA_TRY(c, cudaGetLastError());
        unsigned h = 0;
        PFE_CUDA_TRY(c, cudaMemcpyAsync(&h, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        PFE_CUDA_TRY(c, cudaStreamSynchronize(s));
        if (h) {
            c->err = "learned FSAI: the tensor-core accumulator did not arrive";
            return PFE_ETIMEOUT;
        }
    } else {
        k_mlp_fwd<<<f.mlp_blocks, kMlpThreads, smem_fwd(), s>>>(v, f.srow, f.params, f.gdiag, f.gE, f.hraw);
    }
    k_gslots<<<nblk(c->g.n_slices * 32, 256), 256, 0, s>>>(v, f.gE, f.gslot);
    PFE_CUDA_TRY(c, cudaGetLastError());
    return PFE_OK;
}

// Average device time of `reps` launches of the network's inference kernel
// (the current path: tcgen05 or mma.sync) on f.params, CUDA events on the
// context's stream (the outputs are rewritten with the same values).
pfe_status fsai_time_infer(pfe_ctx *c, int reps, float *ms) {
    auto &f = c->fsai;
    cudaStream_t s = c->stream;
    View v = view(c);
    const int64_t ntiles = (c->g.n + c->g.n_edges + kTcRows - 1) / kTcRows;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)c->num_sms * 4));
    unsigned *err = f.tick + 3;
    auto launch = [&]() {
        if (f.mlp_tc)
            k_mlp_fwd_tc<<<grid, kTcRows, kSmemTc, s>>>(v, f.srow, f.params, f.gdiag, f.gE, f.hraw, err);
        else
            k_mlp_fwd<<<f.mlp_blocks, kMlpThreads, smem_fwd(), s>>>(v, f.srow, f.params, f.gdiag, f.gE, f.hraw);
    };
    cudaEvent_t e0, e1;
    PFE_CUDA_TRY(c, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        c->err = "cudaEventCreate failed";
        return PFE_ECUDA;
    }
    PFE_CUDA_TRY(c, cudaMemsetAsync(err, 0, sizeof(unsigned), s));
    launch();
    cudaEventRecord(e0, s);
    for (int k = 0; k < reps; ++k) launch();
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        c->err = "pfe_time_kernel: network inference failed";
        return PFE_ECUDA;
    }
    unsigned h = 0;
    PFE_CUDA_TRY(c, cudaMemcpy(&h, err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (h) {
        c->err = "learned FSAI: the tensor-core accumulator did not arrive";
        return PFE_ETIMEOUT;
    }
    *ms = t / (float)reps;
    return PFE_OK;
}

// Kaporin loss of the current G and its gradient w.r.t. f.params -> f.grad.
pfe_status fsai_loss_grad(pfe_ctx *c, double *loss, const double *B, int m, double mu, double *rterm) {
    auto &f = c->fsai;
    cudaStream_t s = c->stream;
    View v = view(c);
    const int64_t n = c->g.n, N = n + c->g.n_edges;
    const bool rhs = B && m > 0 && mu > 0.0;
    if (rhs && m > kMaxRhs) {
        c->err = "pfe_fsai_loss_grad_rhs: at most 32 right-hand sides";
        return PFE_EINVAL;
    }
    PFE_TRY(fsai_infer(c));
    k_kaporin_rows<<<nblk(n, 128), 128, 0, s>>>(v, f.kb, f.gdiag, f.gslot, f.ent_of_slot, f.dq, f.qrow, f.logd);
    k_sum2<<<256, kBlock, 0, s>>>(n, f.qrow, f.logd, f.part, f.tick, f.sums);
    // the right-hand-side term: five n x m FP64 vectors, N entry gradients,
    // block partials and the 2m column sums (training only, allocated here)
    double *u = nullptr, *vv = nullptr, *w = nullptr, *sv = nullptr, *gs = nullptr, *rpart = nullptr, *sq = nullptr;
    float *drhs = nullptr;
    unsigned *rtick = nullptr;
    struct Free {
        void **ps[9];
        ~Free() {
            for (void **p : ps)
                if (*p) cudaFree(*p);
        }
    } fr{{(void **)&u, (void **)&vv, (void **)&w, (void **)&sv, (void **)&gs, (void **)&rpart, (void **)&sq,
          (void **)&drhs, (void **)&rtick}};
    constexpr int kRgBlocks = 256;
    if (rhs) {
        const size_t nm = sizeof(double) * (size_t)n * m;
        if (cudaMalloc((void **)&u, nm) != cudaSuccess || cudaMalloc((void **)&vv, nm) != cudaSuccess ||
            cudaMalloc((void **)&w, nm) != cudaSuccess || cudaMalloc((void **)&sv, nm) != cudaSuccess ||
            cudaMalloc((void **)&gs, nm) != cudaSuccess ||
            cudaMalloc((void **)&rpart, sizeof(double) * kRgBlocks * 2 * m) != cudaSuccess ||
            cudaMalloc((void **)&sq, sizeof(double) * 2 * m) != cudaSuccess ||
            cudaMalloc((void **)&drhs, sizeof(float) * N) != cudaSuccess ||
            cudaMalloc((void **)&rtick, sizeof(unsigned)) != cudaSuccess) {
            cudaGetLastError();
            c->err = "pfe_fsai_loss_grad_rhs: device allocation failed";
            return PFE_ENOMEM;
        }
        PFE_CUDA_TRY(c, cudaMemsetAsync(rtick, 0, sizeof(unsigned), s));
        const unsigned gnm = nblk(n * m, 256);
        k_rg_apply<0><<<gnm, 256, 0, s>>>(v, f.kb, f.gdiag, f.gslot, B, m, u);     // u = G b
        k_rg_apply<1><<<gnm, 256, 0, s>>>(v, f.kb, f.gdiag, f.gslot, u, m, vv);    // v = G^T u
        k_rg_apply<2><<<gnm, 256, 0, s>>>(v, f.kb, f.gdiag, f.gslot, vv, m, w);    // A v
        k_rg_resid<<<kRgBlocks, 256, 0, s>>>(n, m, B, w, rpart, rtick, sq);        // w = A v - b, norms
        k_rg_apply<2><<<gnm, 256, 0, s>>>(v, f.kb, f.gdiag, f.gslot, w, m, sv);    // A w
        k_rg_scale<<<gnm, 256, 0, s>>>(n, m, sq, mu, sv);                          // s
        k_rg_apply<0><<<gnm, 256, 0, s>>>(v, f.kb, f.gdiag, f.gslot, sv, m, gs);   // G s
        k_rg_entries<<<nblk(N, 256), 256, 0, s>>>(v, m, u, sv, gs, B, drhs);
    }
    k_dloss<<<nblk(N, 256), 256, 0, s>>>(v, f.sums, f.gdiag, f.hraw, f.dq, drhs);
    k_mlp_bwd<<<f.mlp_blocks, kMlpThreads, smem_bwd(), s>>>(v, f.srow, f.params, f.dq, f.gpart, f.tick + 1, f.grad);
    PFE_CUDA_TRY(c, cudaGetLastError());
    double h[2];
    double hs[2 * kMaxRhs] = {};
    PFE_CUDA_TRY(c, cudaMemcpyAsync(h, f.sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (rhs) PFE_CUDA_TRY(c, cudaMemcpyAsync(hs, sq, 2 * m * sizeof(double), cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(c, cudaStreamSynchronize(s));
    *loss = std::log(h[0] / (double)n) - 2.0 / (double)n * h[1];
    double R = 0.0;
    if (rhs) {
        for (int k = 0; k < m; ++k) R += hs[k] / hs[m + k];
        R /= (double)m;
        *loss += mu * R;
    }
    if (rterm) *rterm = R;
    return PFE_OK;
}

// Classical FSAI factor into the FSAI buffers.
pfe_status fsai_classical(pfe_ctx *c) {
    auto &f = c->fsai;
    cudaStream_t s = c->stream;
    View v = view(c);
    int *derr = reinterpret_cast<int *>(f.tick + 2);
    PFE_CUDA_TRY(c, cudaMemsetAsync(derr, 0, sizeof(int), s));
    k_fsai_classical<<<nblk(c->g.n, 64), 64, 0, s>>>(v, f.kb, f.gdiag, f.gE, derr);
    k_gslots<<<nblk(c->g.n_slices * 32, 256), 256, 0, s>>>(v, f.gE, f.gslot);
    PFE_CUDA_TRY(c, cudaGetLastError());
    int h = 0;
    PFE_CUDA_TRY(c, cudaMemcpyAsync(&h, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
    PFE_CUDA_TRY(c, cudaStreamSynchronize(s));
    if (h == 1) {
        c->err = "classical FSAI: a row has more than 23 lower neighbours";
        return PFE_EUNSUPPORTED;
    }
    if (h == 2) {
        c->err = "classical FSAI: a local matrix is not positive definite";
        return PFE_ENUMERIC;
    }
    return PFE_OK;
}

// ---- incomplete Cholesky IC(0) (Sec. III's preconditioner) ------------------
// L lower triangular on the pattern of tril(A) with (L L^T)_ij = A_ij on the
// pattern, row by row: L_ij = (A_ij - sum_k L_ik L_jk) / L_jj for the lower
// neighbours j of i in increasing order, L_ii = sqrt(A_ii - sum_j L_ij^2).  On
// a grid image with fixed slot positions the common lower neighbours k of i
// and j (slot t) are the slot pairs (s, u) with offset_s = offset_t +
// offset_u, a compile-time table; a pair whose slot is padding (outside the
// image) carries L = 0.  Rows of one level of the raster wavefront
// (ic_level_rows) are independent and run in parallel; a launch per level.
template <int LEN>
struct IcPairs {
    int cnt[LEN / 2];
    int s[LEN / 2][LEN / 2], u[LEN / 2][LEN / 2];
};
template <int LEN>
constexpr IcPairs<LEN> make_ic_pairs() {
    constexpr Stencil<LEN> st = make_stencil<LEN>();
    IcPairs<LEN> p{};
    for (int t = 0; t < LEN / 2; ++t) {
        p.cnt[t] = 0;
        for (int s = 0; s < LEN / 2; ++s)  // ascending s: ascending column k
            for (int u = 0; u < LEN / 2; ++u)
                if (st.dy[s] == st.dy[t] + st.dy[u] && st.dx[s] == st.dx[t] + st.dx[u]) {
                    p.s[t][p.cnt[t]] = s;
                    p.u[t][p.cnt[t]] = u;
                    ++p.cnt[t];
                }
    }
    return p;
}

template <int LEN>
__global__ void k_ic_factor(int64_t W, int64_t y0, int64_t rows, int64_t level, int cl, const int *__restrict__ col,
                            const int *__restrict__ eid, const double *__restrict__ aoff,
                            const double *__restrict__ adiag, double *__restrict__ Llow, double *__restrict__ Ldiag,
                            int *err) {
    constexpr int NL = LEN / 2;
    constexpr IcPairs<LEN> pr = make_ic_pairs<LEN>();
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= rows) return;
    const int64_t y = y0 + k, x = level - cl * y;
    const int64_t i = y * W + x;
    double li[NL];
    double sq = 0.0;
#pragma unroll
    for (int t = 0; t < NL; ++t) {
        const int64_t slot = i * LEN + t;
        li[t] = 0.0;
        if (eid[slot] < 0) continue;  // padding
        const int64_t j = col[slot];
        double v = aoff[slot];
#pragma unroll
        for (int q = 0; q < pr.cnt[t]; ++q) v -= li[pr.s[t][q]] * Llow[j * NL + pr.u[t][q]];
        li[t] = v / Ldiag[j];
        sq += li[t] * li[t];
    }
    double piv = adiag[i] - sq;
    if (!(piv > 0.0)) {
        atomicMax(err, 1);
        piv = 1.0;
    }
    Ldiag[i] = sqrt(piv);
#pragma unroll
    for (int t = 0; t < NL; ++t) Llow[i * NL + t] = li[t];
}

// L into the FSAI buffers: gdiag = L_ii, gE[edge] = L_ba (b > a), so that the
// slot copy gives each row its lower entries and, mirrored, the upper ones.
template <int LEN>
__global__ void k_ic_pack(int64_t n, const int *__restrict__ eid, const double *__restrict__ Llow,
                          const double *__restrict__ Ldiag, float *gdiag, float *gE) {
    constexpr int NL = LEN / 2;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    gdiag[i] = (float)Ldiag[i];
    for (int t = 0; t < NL; ++t) {
        const int e = eid[i * LEN + t];
        if (e >= 0) gE[e] = (float)Llow[i * NL + t];
    }
}

template <int LEN>
pfe_status ic0_len(pfe_ctx *c) {
    static_assert(ic_levels_ok<LEN>(), "level schedule");
    auto &f = c->fsai;
    cudaStream_t s = c->stream;
    const int64_t n = c->g.n, W = c->W, H = n / W;
    constexpr int cl = ic_level_coef<LEN>();
    double *Llow = nullptr, *Ldiag = nullptr;
    if (cudaMalloc((void **)&Llow, sizeof(double) * n * (LEN / 2)) != cudaSuccess ||
        cudaMalloc((void **)&Ldiag, sizeof(double) * n) != cudaSuccess) {
        cudaGetLastError();
        if (Llow) cudaFree(Llow);
        c->err = "IC(0): scratch allocation failed";
        return PFE_ENOMEM;
    }
    int *derr = reinterpret_cast<int *>(f.tick + 2);
    cudaError_t e = cudaMemsetAsync(derr, 0, sizeof(int), s);
    const int64_t L = ic_levels(W, H, cl);
    for (int64_t l = 0; l < L && e == cudaSuccess; ++l) {
        int64_t y0 = 0, rows = 0;
        ic_level_rows(l, W, H, cl, y0, rows);
        if (rows == 0) continue;
        k_ic_factor<LEN><<<nblk(rows, 128), 128, 0, s>>>(W, y0, rows, l, cl, c->g.col, c->g.eid, c->g.aoff64,
                                                         c->g.adiag64, Llow, Ldiag, derr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        View v = view(c);
        k_ic_pack<LEN><<<nblk(n, 256), 256, 0, s>>>(n, c->g.eid, Llow, Ldiag, f.gdiag, f.gE);
        k_gslots<<<nblk(c->g.n_slices * 32, 256), 256, 0, s>>>(v, f.gE, f.gslot);
        e = cudaGetLastError();
    }
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(Llow);
    cudaFree(Ldiag);
    if (e != cudaSuccess) {
        c->err = std::string("IC(0): ") + cudaGetErrorString(e);
        return PFE_ECUDA;
    }
    if (h) {
        c->err = "IC(0): a non-positive pivot (the matrix is not an M-matrix)";
        return PFE_ENUMERIC;
    }
    f.ic_cl = cl;
    f.ic_levels = L;
    return PFE_OK;
}

// IC(0) factor of A into the FSAI buffers (one grid image, fixed slot positions).
pfe_status ic0_factor(pfe_ctx *c) {
    if (c->g.row_len == 12) return ic0_len<12>(c);
    if (c->g.row_len == 28) return ic0_len<28>(c);
    c->err = "IC(0) is built for grid images of radius 2 or 3";
    return PFE_EUNSUPPORTED;
}

// G entries as FP64: od[i] = G_ii (n), oe[k] = G_{b_k a_k} for external edge k.
pfe_status fsai_export(pfe_ctx *c, double *od, double *oe) {
    const int64_t m = std::max<int64_t>(c->g.n, c->g.n_edges);
    k_export<<<nblk(m, 256), 256, 0, c->stream>>>(view(c), c->fsai.gdiag, c->fsai.gE, od, oe);
    PFE_CUDA_TRY(c, cudaGetLastError());
    return PFE_OK;
}

pfe_status adam_step(float *p, const float *gr, float *m, float *v, int64_t cnt, int step, double lr, double b1,
                     double b2, double eps, cudaStream_t s) {
    const float c1 = (float)(1.0 - std::pow(b1, step)), c2 = (float)(1.0 - std::pow(b2, step));
    k_adam<<<nblk(cnt, 256), 256, 0, s>>>(cnt, p, gr, m, v, (float)lr, (float)b1, (float)b2, (float)eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? PFE_OK : PFE_ECUDA;
}

}  // namespace pfe
