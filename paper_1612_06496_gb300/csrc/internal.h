// Internal declarations of libpfe: the context, device control blocks and the
// kernel launchers of each translation unit.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/pfe.h"
#include "fsai.h"

#define PFE_DMAX 32

namespace pfe {

// Segments: a batch of independent problems (images) stored as one
// block-diagonal graph; rows [off[s], off[s+1]) belong to segment s.  A single
// problem is one segment.
struct Segs {
    int nseg;
    int64_t n;               // rows in all segments
    const int64_t *off;      // nseg + 1 row offsets (device)
    const int *rseg;         // segment of each row (device)
};

// Per-segment PCG scalars, index [seg * d + c] (device).  Written only by the
// last block of a segment in a reduction kernel.
struct SegScal {
    double *bnorm, *rz, *alpha, *beta, *relres;  // nseg * d
    double *alpha_prev;                           // nseg * d: alpha of a held solution update (FSAI)
    double *rel_ref;                              // nseg * d: relative residual at the last replacement (or the start)
    double *rec2;                                 // nseg * d: |r|^2 of the recurrence residual a replacement replaces
    double *devr;                                 // nseg * d: |r_true - r_rec|^2 / |r_rec|^2 of the last replacement
    int *active;                                  // nseg * d: column still iterating
    int *pending;                                 // nseg * d: reached tol on the recurrence, waiting for a replacement
    int *seg_active;                              // nseg: any column of the segment iterating
    int *seg_live;                                // nseg: any column iterating or waiting to be confirmed
    int *seg_iters;                               // nseg: iterations of the segment in this solve
    long long *seg_iters_tot;                     // nseg: summed over solves until the host clears it
    unsigned *ticket;                             // nseg * 4: per-segment reduction tickets
};

// Most iterations in one captured loop body that get their own conditional
// node for the replacement kernels (a longer body launches them every time).
constexpr int kPcgMaxIf = 8;

// Device-resident control block of one d-column PCG solve (all segments).
// The per-segment finishers of a reduction kernel count themselves on
// `ticket`; the last one finishes the iteration (global flags, statistics).
struct PcgCtl {
    int iter;          // iterations done in the current solve
    int done;          // 1: every column converged, max_iter hit, or an error
    int error;         // pfe_status of a numeric failure (0 = none)
    int refresh_now;   // 1: this iteration ends with a true-residual refresh
    unsigned ticket[4];
    int max_iter, refresh, ncols, any_active;
    double tol;
    // statistics accumulated over solves until the host clears them
    long long tot_iters, tot_rounds, tot_refreshes;
    int max_solve_iters, n_solves, n_unconv, last_iters;
    double max_relres, last_relres;
    int last_converged, unroll;       // unroll: iterations per graph body / host poll
    long long launches;               // PCG kernel launches (early-exited ones included)
    int xheld;                        // FSAI: y += alpha_prev p_prev of the iteration before is also pending
    int p_ready;                      // 1: p was just set by k_pcg_init (no update in k_spmm)
    int xpending;                     // 1: y += alpha p of the last k_spmm not yet applied
    int launch_base, launch_per_iter; // kernel launches outside / per iteration of the loop
    int xfold;                        // FSAI: this iteration's k_fsai_zp applies both pending updates
    int refresh_want;                 // set during an iteration: a column asks for a residual replacement
    int refresh_next;                 // Jacobi: refresh_want latched at the end of an iteration for the next one
    int refreshes;                    // replacement iterations of the current solve
    int rounds;                       // q = A p launches of the current solve (bounds the loop)
    int launch_cond;                  // launches of a replacement iteration that run only then (IF node body)
    int n_if;                         // IF nodes of the captured loop body (0: no graph built)
    cudaGraphConditionalHandle ifh[kPcgMaxIf];  // their handles, by position in the body
};

// Control block of the P-step (Alg. 1 steps 6-7).  G, T and evals are
// those of segment 0 (the only one of a single problem); a batch keeps every
// segment's T in pfe_ctx::seg_T.
struct PstepCtl {
    unsigned ticket;
    int error;
    double G[PFE_DMAX * PFE_DMAX];  // Gram X^T X
    double T[PFE_DMAX * PFE_DMAX];  // (X^T X)^{-1/2}
    double evals[PFE_DMAX];
};

// Graph in SELL-32 form (sliced ELLPACK, slice = 32 consecutive rows = one
// warp).  Off-diagonal slot k of row i lives at slice_ptr[i/32] + 32k + i%32.
// Undirected edges live in a second SELL-32 layout over their first
// endpoint ("forward" edges, j > i): edge slot fslice_ptr[i/32] + 32k + i%32.
struct DevGraph {
    int64_t n = 0, n_slices = 0, slots = 0, n_edges = 0, fslots = 0;
    int max_slots_per_row = 0;
    int row_len = 0;            // > 0: every row has exactly row_len slots (grid graphs), row i at i * row_len
    int *slice_ptr = nullptr;   // n_slices + 1, in slots
    int *fslice_ptr = nullptr;  // n_slices + 1, in edge slots
    int *col = nullptr;         // per slot: neighbour j (padding: i itself)
    int *eid = nullptr;         // per slot: edge slot of (min, max), -1 padding
    double *w64 = nullptr;      // per slot: w_ij
    float *w32 = nullptr;
    double *aoff64 = nullptr;   // per slot: A_ij = -lambda w_ij^2
    float *aoff32 = nullptr;
    float *aofflo32 = nullptr;  // per slot: A_ij - aoff32 rounded to FP32 (aoff32 + aofflo32 = A_ij to ~2^-48)
    double *adiag64 = nullptr;  // A_ii = lambda d2_i + r d_i
    float *adiag32 = nullptr;
    float *adiaglo32 = nullptr;
    double *dinv64 = nullptr;   // 1 / A_ii
    float *dinv32 = nullptr;
    double *deg = nullptr, *deg2 = nullptr, *sqrtdeg = nullptr;
    int *ext_slot = nullptr;    // external edge k -> edge slot
    int *ea = nullptr, *eb = nullptr;  // external edge k endpoints, a < b
    double *ew = nullptr;              // external edge k weight
};

// Work arrays of the iteration for one precision (pointers typed at use).
struct Work {
    void *Y = nullptr;       // n x d: the PCG solution (Y of Alg. 2); FP32 hi part when mixed
    float *Ylo = nullptr;    // mixed: low part of Y (Y = hi + lo)
    void *Bs[2] = {nullptr, nullptr};  // edge slots x d: b of Alg. 2 (double-buffered)
    void *RHS = nullptr;     // n x d: right-hand side of Eq. 13 (times 2)
    void *Cw = nullptr;      // n x d: r D^{1/2} (P - B)
    void *R = nullptr, *Pd = nullptr, *Pd2 = nullptr, *Q = nullptr;  // PCG residual, direction (x2), A*direction
    double *P = nullptr, *B = nullptr;  // n x d FP64 (Alg. 1)
    double *stage = nullptr;            // n x d FP64 staging (init / get / set)
    double *partials = nullptr;         // block partials of reductions
    int64_t partials_len = 0;
};

}  // namespace pfe

struct pfe_ctx {
    pfe_params prm{};
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    int64_t n = 0;
    int m = 0, kind = 0, H = 0, W = 0;
    double radius = 0, sigma = 0, lambda = 0, r = 1, vol = 0;
    // segments (a batch of problems; 1 for a single problem)
    int nseg = 1;
    std::vector<int64_t> h_seg_off;   // nseg + 1 row offsets
    std::vector<int> h_seg_h, h_seg_w;
    std::vector<double> h_seg_lam, h_seg_vol;
    int64_t *seg_off = nullptr;       // device copies
    int *seg_h = nullptr, *seg_w = nullptr;
    int *rseg = nullptr;              // segment of each row
    double *seg_lam = nullptr;        // lambda of each segment
    pfe::SegScal sc{};                // per-segment PCG scalars (allocated by pfe_init)
    double *seg_T = nullptr;          // nseg x d x d P-step transforms
    unsigned *seg_pticket = nullptr;  // nseg P-step tickets
    pfe::DevGraph g;
    int d = 0;
    bool inited = false;
    bool mixed = true;
    int bs_cur = 0;
    pfe::Work wk;
    pfe::PcgCtl *ctl = nullptr;       // device
    pfe::PcgCtl *h_ctl = nullptr;     // pinned host mirror
    pfe::PstepCtl *pctl = nullptr;    // device
    int *h_flag = nullptr;            // pinned host scratch
    int grid_rows = 0;                // blocks of the persistent row kernels (upper bound)
    int kgrid[32] = {0};              // per-kernel grid cache (wave_grid), reset by pfe_init
    int kbps[32] = {0};               // blocks per SM chosen by pfe_autotune per kernel slot (0: occupancy)
    float shape_ms[8][8] = {};        // pfe_autotune: time of each tuned kernel at 1..8 blocks per SM (<= 0: not timed)
    cudaGraph_t pcg_graph = nullptr;
    cudaGraphExec_t pcg_exec = nullptr;
    pfe::FsaiState fsai;
    std::string err;
    std::vector<void *> dev_allocs;   // graph-lifetime allocations
    std::vector<void *> work_allocs;  // d-dependent allocations
    int64_t bytes = 0;       // device memory the context keeps (pfe_info.device_bytes)
    int64_t work_bytes = 0;  // the part of it in work_allocs
    int spmm_variant = PFE_SPMM_ROW1;  // SpMM kernel variant (pfe_autotune)
    int fsai_variant = PFE_FSAI_SLOTS; // FSAI kernels' column form (pfe_autotune)
    int edge_variant = PFE_EDGE_SLOTS; // edge pass: slot columns and edge ids, or from the stencil (pfe_autotune)
    float edge_tune_ms[2] = {-1.f, -1.f};
    float fsai_tune_ms[2] = {-1.f, -1.f};
    int le_iters = 0;                 // last Laplacian-eigenmap computation
    double le_residual = 0.0;
};

namespace pfe {

// NVTX range over one stage of the method (build, init, inner step with its
// PCG and edge pass, P-step, solve, preconditioner set-up), for profilers
// that select kernels by range (ncu --nvtx); a no-op unless a tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// pfe_params.max_device_bytes: true (with the message set) when keeping
// `bytes` more would pass the context's cap; nothing is allocated then.
inline bool over_device_cap(pfe_ctx *c, size_t bytes) {
    const int64_t cap = c->prm.max_device_bytes;
    if (cap <= 0 || c->bytes + (int64_t)bytes <= cap) return false;
    c->err = "max_device_bytes: keeping " + std::to_string(bytes) + " more bytes would pass the cap of " +
             std::to_string(cap) + " (" + std::to_string(c->bytes) + " held)";
    return true;
}

// --- graph.cu
pfe_status build_grid_graph(pfe_ctx *c, const double *dfeat);
pfe_status build_edge_graph(pfe_ctx *c, const double *dfeat, const int32_t *dei, const int32_t *dej);
pfe_status setup_segments(pfe_ctx *c);
// --- kmeans.cu: k-means segmentation of an n x d FP64 device matrix
pfe_status kmeans_run(pfe_ctx *c, const double *X, int d, int k, const double *C0, int max_iter, int *labels,
                      double *centroids, double *inertia, int *rounds);
// --- diag.cu: |M Y|_1 and |Y^T D Y - I|_F (which: 0 = Y, 1 = Yhat)
pfe_status diag_objective(pfe_ctx *c, int which, double *l1, double *ortho);
pfe_status diag_residual(pfe_ctx *c, const double *B, const double *X, double *relres);
// --- le.cu: Laplacian-eigenmap start (n x d FP64, row-major, device)
int le_block(int d);
pfe_status launch_le(pfe_ctx *c, int d, double *yout, int max_iter, double tol, int degree, int *iters,
                     double *res);
pfe_status check_edges_in_segments(pfe_ctx *c);
pfe_status finish_graph_values(pfe_ctx *c);

// --- pcg.cu: one PCG solve A Y = RHS on the context's work arrays
struct PcgLaunch {
    cudaGraphConditionalHandle cond;
    int use_cond;
    // graph capture of the loop body: the kernels of replacement iterations
    // go into one conditional IF node per iteration of the body (n_if > 0),
    // captured on the side stream
    int n_if = 0;
    cudaGraphConditionalHandle ifh[kPcgMaxIf] = {};
    cudaStream_t side = nullptr;
};
pfe_status launch_pcg_init(pfe_ctx *c, cudaStream_t s, PcgLaunch L);
pfe_status launch_pcg_body(pfe_ctx *c, cudaStream_t s, PcgLaunch L, int iters);
pfe_status launch_pcg_final(pfe_ctx *c, cudaStream_t s, PcgLaunch L);
pfe_status launch_apply_A(pfe_ctx *c, cudaStream_t s, const void *x, void *y);
pfe_status time_pcg_kernel(pfe_ctx *c, cudaStream_t s, int which, int reps, float *ms, int variant = -1);

// --- edge.cu: fused edge pass (Eqs. 7, 9, 10) and right-hand side (Eq. 13)
pfe_status launch_edge(pfe_ctx *c, cudaStream_t s);

// --- pstep.cu: Gram, polar factor and the P/B/C update (Alg. 1 steps 6-7)
enum PstepMode { PSTEP_INIT = 0, PSTEP_RESET = 1, PSTEP_CARRY = 2 };
pfe_status launch_pstep(pfe_ctx *c, cudaStream_t s, int mode);

// --- convert.cu: FP64 <-> working precision copies of n x d / edge arrays
pfe_status launch_to_work(pfe_ctx *c, cudaStream_t s, const double *src, void *dst, float *dst_lo,
                          int64_t rows);
pfe_status launch_from_work(pfe_ctx *c, cudaStream_t s, const void *src, const float *src_lo,
                            double *dst, int64_t rows);
pfe_status launch_bs_gather(pfe_ctx *c, cudaStream_t s, const void *bs, double *dst, bool to_ext);
pfe_status launch_bs_scatter(pfe_ctx *c, cudaStream_t s, const double *src, void *bs);
pfe_status launch_yhat(pfe_ctx *c, cudaStream_t s, double *dst);
pfe_status launch_cw(pfe_ctx *c, cudaStream_t s);  // C = r D^{1/2} (P - B)

// supported embedding dimensions
bool d_supported(int d);

}  // namespace pfe

// error helpers
#define PFE_CUDA_TRY(c, call)                                                     \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            (c)->err = std::string(#call) + ": " + cudaGetErrorString(e_);       \
            return PFE_ECUDA;                                                    \
        }                                                                        \
    } while (0)

#define PFE_TRY(call)                 \
    do {                              \
        pfe_status s_ = (call);       \
        if (s_ != PFE_OK) return s_;  \
    } while (0)
