/*
 * pfe.h -- C ABI of libpfe, a CUDA (sm_103a) implementation of the inner
 * loop of piecewise flat embeddings (PFE):
 *
 *     min_Y  sum_{i,j} w_ij |y_i - y_j|_1   s.t.  Y^T D Y = I          (Eq. 1)
 *
 * solved by the SOC / Bregman outer iteration (Alg. 1) around the split
 * Bregman inner iteration (Alg. 2) in its compact form (Eqs. 9, 10, 13),
 * with the d right-hand-side systems of Eq. 13 solved by preconditioned
 * conjugate gradients (Sec. III, last paragraph).
 *
 * Conventions for every entry point:
 *  - Returns a pfe_status; PFE_OK is 0.  No C++ exception crosses the ABI.
 *    pfe_last_error() returns a message for the last failing call on a ctx
 *    (pfe_last_error(NULL): for the calling thread's last failed build).
 *  - Array arguments are plain pointers.  Unless a parameter says otherwise
 *    a pointer may address host memory (pageable or pinned) or device
 *    memory of the context's GPU; the library detects which and copies host
 *    data through its own device buffers.  Arrays are row-major and
 *    contiguous unless a leading dimension is given.
 *  - The caller owns every array it passes; the library never frees or
 *    retains caller memory beyond the call.  The library owns everything it
 *    allocates inside a pfe_ctx until pfe_destroy().
 *  - All device work is queued on the stream given to pfe_build_graph (or
 *    pfe_set_stream).  Calls that return host-visible results synchronise
 *    that stream before returning; the others only enqueue work.
 *  - A context is thread-compatible, not thread-safe: do not use one
 *    context from two threads at once.
 */
#ifndef PFE_H
#define PFE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PFE_API __attribute__((visibility("default")))
#else
#define PFE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pfe_ctx pfe_ctx;
/* A cudaStream_t passed as an opaque pointer; NULL is the legacy default stream. */
typedef void *pfe_stream_t;

typedef enum pfe_status {
    PFE_OK = 0,
    PFE_EINVAL = 1,        /* bad argument (NULL, size, zero-degree vertex, duplicate edge, ...) */
    PFE_ENOMEM = 2,        /* a device or host allocation failed, or would pass max_device_bytes */
    PFE_ECUDA = 3,         /* a CUDA runtime call failed */
    PFE_ENOTCONV = 4,      /* a PCG solve hit max_iter; results are still written */
    PFE_ENUMERIC = 5,      /* NaN/Inf or a non-positive curvature p^T A p in PCG */
    PFE_ESINGULAR = 6,     /* the P-step's Gram matrix is numerically singular */
    PFE_ETIMEOUT = 7,      /* a bounded device wait ran out (a bulk copy of the TMA-staged SpMM never landed), or the
                              PCG loop ran max_iter + 24 rounds without its iterations advancing */
    PFE_EUNSUPPORTED = 8,  /* embedding dimension or option not built into this library */
    PFE_ESTATE = 9         /* call out of order (e.g. pfe_inner_step before pfe_init) */
} pfe_status;

/* Graph kinds (pfe_graph_desc.kind). */
enum { PFE_GRAPH_GRID = 0, PFE_GRAPH_EDGES = 1 };
/* Arithmetic of the iteration (pfe_params.precision). */
enum {
    PFE_FP64 = 0,  /* every array and operation in FP64 */
    PFE_MIXED = 1  /* FP32 edge pass, SpMM and PCG vectors; FP32-pair (about 48-bit)
                      accumulation of dot products and of the PCG solution; FP64
                      Gram, polar step, P, B */
};
/* Preconditioner of the PCG solve (pfe_params.precond); the learned FSAI
 * preconditioner is switched on after construction with pfe_fsai_set(). */
enum { PFE_PRECOND_JACOBI = 0 };
/* How the PCG loop is driven (pfe_params.loop_mode). */
enum {
    PFE_LOOP_GRAPH = 0,  /* CUDA graph with a device-evaluated WHILE node: no host sync */
    PFE_LOOP_HOST = 1    /* host loop that polls a device flag every check_every iterations */
};

/*
 * Data points and graph (Sec. II: points x_i in R^m; heat-kernel weights
 * w_ij = exp(-|x_i - x_j|^2 / (2 sigma^2)); Sec. IV: one vertex per pixel,
 * edges between nearby pixels).
 */
typedef struct pfe_graph_desc {
    int64_t n;               /* number of data points (vertices), >= 2 */
    int32_t m;               /* feature dimension, >= 1 */
    int32_t kind;            /* PFE_GRAPH_GRID or PFE_GRAPH_EDGES */
    const double *features;  /* n x m, row-major FP64 (host or device) */
    /* PFE_GRAPH_GRID: n == H*W, pixel (x, y) is vertex y*W + x, and every
     * pair of pixels with 0 < dx^2 + dy^2 <= radius^2 is an edge. */
    int32_t H, W;
    double radius;           /* in pixels, 1 <= radius <= 8 */
    /* PFE_GRAPH_EDGES: n_edges undirected pairs (ei[k], ej[k]), 0 <= ei, ej < n,
     * ei != ej, no pair listed twice (in either orientation).  int32 arrays,
     * host or device.  Edge k keeps id k in pfe_get_edges(). */
    const int32_t *ei, *ej;
    int64_t n_edges;
    double sigma;            /* heat-kernel width, > 0 */
    /* Batch: nseg >= 2 independent problems (images) in one block-diagonal
     * graph, iterated together (one launch per kernel for all of them), each
     * with its own lambda (sqrt of its own volume by default), PCG scalars,
     * convergence and P-step (Alg. 1 and Alg. 2 applied per problem).  nseg =
     * 0 or 1: one problem, the fields below are not read.  Host arrays:
     *   PFE_GRAPH_GRID:  seg_hw[2s], seg_hw[2s+1] = H_s, W_s of image s; the
     *     pixels of image s follow those of image s-1 and n = sum_s H_s W_s
     *     (H, W are not read);
     *   PFE_GRAPH_EDGES: seg_off[0..nseg], seg_off[0] = 0, seg_off[nseg] = n:
     *     segment s is vertices seg_off[s] .. seg_off[s+1]-1; no edge may join
     *     two segments (PFE_EINVAL).
     * Every segment has >= 2 vertices; nseg <= PFE_MAX_SEGMENTS. */
    int32_t nseg;
    const int32_t *seg_hw;
    const int64_t *seg_off;
} pfe_graph_desc;
#define PFE_MAX_SEGMENTS 4096

typedef struct pfe_params {
    double lambda;        /* split-Bregman penalty (Alg. 2); <= 0 selects sqrt(sum_i d_i) */
    double r;             /* SOC penalty (Alg. 1, Eq. 5), > 0; default 1 */
    int32_t precision;    /* PFE_FP64 or PFE_MIXED; default PFE_MIXED */
    int32_t precond;      /* PFE_PRECOND_JACOBI */
    double tol;           /* PCG stops a column when |b - A y| / |b| <= tol; default 1e-6 */
    int32_t max_iter;     /* PCG iteration cap per solve; default 5000 */
    int32_t refresh;      /* every `refresh` iterations r is recomputed as b - A y in
                             extended precision; 0 = never; default 50 */
    int32_t reset_inner_each_outer; /* 1 (default): b = d = 0 at every outer iteration
                                       (Alg. 2 restarts); 0: carry them over */
    int32_t loop_mode;    /* PFE_LOOP_GRAPH (default) or PFE_LOOP_HOST */
    int32_t check_every;  /* iterations per graph body / host poll; default 4 */
    int32_t blocks_per_sm;/* persistent-grid occupancy of the row kernels; 0 = auto */
    int64_t max_device_bytes; /* cap on the device memory the context keeps (pfe_info.device_bytes):
                                 an allocation that would pass it fails with PFE_ENOMEM and
                                 allocates nothing; temporaries of a single call are not
                                 counted; 0 (default) = no cap */
} pfe_params;

/* Fills *p with the defaults listed above.  Never fails. */
PFE_API void pfe_default_params(pfe_params *p);

typedef struct pfe_info {
    int64_t n;            /* vertices */
    int64_t n_edges;      /* undirected edges |E| (rows of M, Sec. II) */
    int64_t nnz_A;        /* n + 2|E|: nonzeros of lambda M^T M + r D */
    int64_t sell_slots;   /* padded off-diagonal slots actually stored (>= 2|E|) */
    int32_t d;            /* embedding dimension after pfe_init, else 0 */
    int32_t precision;
    double lambda, r;     /* values in use */
    double vol;           /* sum_i d_i */
    int64_t device_bytes; /* bytes of device memory the context holds */
    int32_t nseg;         /* problems in the batch (1 for one problem) */
    int32_t le_iters;     /* iterations of the last Laplacian-eigenmap start (pfe_init, Y0 NULL) */
    double le_residual;   /* its largest residual |P v - theta v|_D */
} pfe_info;

typedef struct pfe_step_stats {
    int32_t pcg_iters;      /* iterations of this step's solve (max over columns) */
    int32_t converged;      /* 1 if every column reached tol */
    double relres_max;      /* max over columns of the final relative residual */
} pfe_step_stats;

typedef struct pfe_solve_stats {
    int64_t pcg_iters_total;  /* sum over solves of the per-solve iteration count */
    int32_t pcg_iters_max;    /* largest per-solve iteration count */
    int32_t n_solves;         /* inner steps run by this call (times the batch's problems) */
    int32_t n_unconverged;    /* solves that stopped at max_iter */
    double relres_max;        /* largest final relative residual of any solve */
    int64_t kernel_launches;  /* libpfe kernels launched by this call's iterations */
    int64_t pcg_rounds;       /* PCG iterations the kernels ran, summed over inner steps: for a
                                 batch the longest problem's count per step (= pcg_iters_total
                                 for one problem) */
    int64_t replacements;     /* of those, iterations that replaced the recurrence residual by
                                 b - A y (periodic, after a 1e3-fold fall, or to confirm tol) */
} pfe_solve_stats;

/*
 * pfe_build_graph -- build the graph and the constant system matrix of Eq. 13.
 *
 * Computes the heat-kernel weights (Sec. II), d_i = sum_j w_ij (Sec. II,
 * Alg. 1 step 2), the edge operator M (one row per undirected edge i < j with
 * +w_ij at i and -w_ij at j, Sec. II) in implicit form, and
 * A = lambda M^T M + r D (twice the matrix of Eq. 13), all on the device.
 * A zero-degree vertex is PFE_EINVAL (D^{-1/2} would not exist).
 * *out receives a new context (NULL on failure).  The feature and edge
 * arrays are read during the call only.  Synchronises `stream`.
 */
PFE_API pfe_status pfe_build_graph(pfe_ctx **out, const pfe_graph_desc *g, const pfe_params *p,
                           pfe_stream_t stream);

/*
 * pfe_init -- set the starting embedding (Alg. 1 step 3).
 *
 * Y0 is n x d FP64 with leading dimension ldY0 >= d (host or device).  The
 * library D-orthonormalises it, Y = D^{-1/2} polar(D^{1/2} Y0) (the P-step
 * map of Alg. 1 step 6 applied to D^{1/2} Y0), then sets P = D^{1/2} Y,
 * B = 0 and the split-Bregman variables b = d = 0 (Alg. 2 step 3).
 * Y0 == NULL starts from the Laplacian eigenmap (pfe_laplacian_eigenmap with
 * its default cap and tolerance; a start short of the tolerance is still
 * used, see pfe_info.le_residual); not for a batch (PFE_EUNSUPPORTED).  d must
 * be one of the dimensions built into the library (1..16, 20, 24, 25, 32),
 * else PFE_EUNSUPPORTED.  PFE_ESINGULAR if D^{1/2} Y0 is rank deficient.
 */
PFE_API pfe_status pfe_init(pfe_ctx *c, int32_t d, const double *Y0, int64_t ldY0);

/*
 * pfe_autotune -- choose the fastest variant of each tunable hot kernel for
 * this context (its graph, d and precision): every candidate is timed with
 * CUDA events over `reps` launches on the current iterate (scratch copies,
 * the iteration state is not modified) and the fastest is kept.  Tunable:
 *  - the SpMM of the PCG iteration (PFE_TUNE_SPMM, variants below; the
 *    fixed-length ones apply to FP32 grid graphs of radius 2 or 3, for a
 *    batch only PFE_SPMM_ROW1 at radius 2);
 *  - with an FSAI factor set (pfe_fsai_set, pfe_fsai_classical) on one FP32
 *    grid image of radius 2 or 3: the column form of the FSAI kernels
 *    (PFE_TUNE_FSAI), timed as one iteration's k_fsai_tr and k_fsai_zp;
 *  - on one FP32 grid image of radius 2: the edge pass's column form
 *    (PFE_TUNE_EDGE), slot arrays or the stencil (Sec. III's memory
 *    argument: the structured grid needs no stored columns).
 * Every variant of a kernel adds the same products in the same order, so
 * the choice changes the time, not the results.  choice[0] receives the
 * chosen SpMM variant and ms[v] (at least PFE_SPMM_NVARIANTS entries; either
 * may be NULL) each variant's average time, -1 where it does not apply;
 * pfe_get_variant reads any kernel's current choice (and the FSAI timings).
 * pfe_set_variant sets a choice directly (e.g. from a cache of earlier
 * tuning): PFE_EUNSUPPORTED where it does not apply.  Needs pfe_init;
 * synchronises.
 */
enum {
    PFE_SPMM_GENERAL = 0, /* any layout: slots fetched 12 at a time, then gathered */
    PFE_SPMM_ROW1 = 1,    /* uniform rows: one row group per step, >= 6 blocks per SM */
    PFE_SPMM_ROW2 = 2,    /* uniform rows: two row groups per step, >= 5 blocks per SM */
    PFE_SPMM_ROW2_4 = 3,  /* uniform rows: two row groups per step, >= 4 blocks per SM */
    PFE_SPMM_TMA = 4,     /* uniform rows: the slots of tiles of rows staged in shared memory by
                             bulk asynchronous (TMA) copies, two tiles ahead (one problem only) */
    PFE_SPMM_STENCIL = 5, /* one grid image whose width is a multiple of 4: the stencil form; a
                             block walks a strip of the image down, a ring of row bands of p and
                             the rows' matrix values staged in shared memory by bulk asynchronous
                             (TMA) copies three rows ahead; the column array is not read and no
                             gather leaves the SM */
    PFE_SPMM_GRID1 = 6,   /* one grid image: uniform rows whose neighbour columns are computed from
                             the stencil (only the matrix values are read), one row group per step */
    PFE_SPMM_GRID2 = 7,   /* the same, two row groups per step */
    PFE_SPMM_NVARIANTS = 8
};
enum { PFE_TUNE_SPMM = 0, PFE_TUNE_FSAI = 1, PFE_TUNE_EDGE = 2, PFE_TUNE_MLP = 3 };
enum {
    PFE_FSAI_SLOTS = 0,   /* FSAI kernels read each slot's column */
    PFE_FSAI_STENCIL = 1  /* one grid image: the columns are computed from the stencil */
};
enum {
    PFE_MLP_MMA_SYNC = 0, /* the network's 64 x 64 layer as warp-level mma.sync m16n8k16 tiles */
    PFE_MLP_TCGEN05 = 1   /* the default: 128 x 64 x 64 tcgen05.mma per 128 entries, FP32 accumulator in
                             tensor memory (inference; training's backward runs mma.sync) */
};
enum {
    PFE_EDGE_SLOTS = 0,   /* edge pass reads each slot's column and edge id */
    PFE_EDGE_STENCIL = 1  /* one FP32 grid image of radius 2: the neighbour and the edge's Bregman
                             slot of every slot are computed from the stencil (only the weights
                             are read) */
};
PFE_API pfe_status pfe_autotune(pfe_ctx *c, int32_t reps, int32_t *choice, double *ms);
PFE_API pfe_status pfe_set_variant(pfe_ctx *c, int32_t kernel, int32_t variant);
/* pfe_get_variant -- the current choice for `kernel` (PFE_TUNE_SPMM,
 * PFE_TUNE_FSAI, PFE_TUNE_EDGE or PFE_TUNE_MLP); for PFE_TUNE_FSAI and
 * PFE_TUNE_EDGE, ms (2 entries, may be NULL) receives the two column forms'
 * times from the last pfe_autotune (-1 if not tuned).  PFE_TUNE_MLP (not
 * tuned: the network runs once per image) selects the tensor-core path of the
 * learned factor's inference; it takes effect at the next pfe_fsai_set or
 * pfe_fsai_loss_grad. */
PFE_API pfe_status pfe_get_variant(pfe_ctx *c, int32_t kernel, int32_t *variant, double *ms);

/*
 * Launch shapes.  Besides the variants above, pfe_autotune chooses the grid
 * of each row kernel that the configured iteration runs -- the SpMM (its
 * current variant, except the stencil form, which sizes its own grid), and
 * k_update and k_pupdate (Jacobi) or k_fsai_tr and k_fsai_zp (an FSAI
 * factor), and the edge pass -- as a number of resident blocks per SM: the
 * kernel's occupancy (the default) and up to three fewer, each timed like
 * the variants, a smaller count kept only when it is at least 2 % faster.
 * The grid groups the rows of a kernel's dot products into block partials,
 * so a tuned shape changes the solves by rounding (each is reproducible).
 *
 * pfe_get_shape -- for `kernel` (PFE_KERNEL_SPMM, _UPDATE, _PUPDATE,
 * _FSAI_TR, _FSAI_ZP or _EDGE): *blocks_per_sm receives the chosen count (0:
 * the kernel's occupancy), and ms (8 entries, may be NULL) the time of one
 * launch at b = 1..8 blocks per SM in ms[b - 1] from the last pfe_autotune
 * (-1 where not timed; k_pupdate and k_fsai_zp: the average of the launches
 * that fold and that hold the solution update).  pfe_set_shape sets the
 * count directly (0 restores the occupancy; counts above it act as it);
 * PFE_EINVAL for another kernel or a count outside 0..8.  The stencil-form
 * SpMM (PFE_SPMM_STENCIL) sizes its own grid: pfe_get_shape reports 0 and
 * no timings for it, pfe_set_shape gives PFE_EUNSUPPORTED.  pfe_init resets
 * every shape to the default.
 */
PFE_API pfe_status pfe_get_shape(pfe_ctx *c, int32_t kernel, int32_t *blocks_per_sm, double *ms);
PFE_API pfe_status pfe_set_shape(pfe_ctx *c, int32_t kernel, int32_t blocks_per_sm);

/*
 * pfe_kmeans -- the segmentation stage of Sec. IV: k-means clustering of the
 * rows of X (n x d row-major FP64, host or device; NULL = the context's
 * embedding D^{-1/2} P, d = its dimension), in FP64.  Start: C0 (k x d, host
 * or device) or, when NULL, the maximin rule: centroid 0 = row 0, then
 * repeatedly the row farthest from its nearest chosen centroid (ties to the
 * smallest row).  Lloyd rounds: every row to its nearest centroid (ties to
 * the smallest cluster), every centroid to the mean of its rows (an empty
 * cluster keeps its centroid), until no label changes or max_iter rounds.
 * Outputs (any may be NULL; host or device): labels[n] (int32), centroids
 * (k x d), *inertia = sum of squared distances to the assigned centroids,
 * *rounds.  Squared distances sum the squared column differences in column
 * order (separately rounded), so results are reproducible.  1 <= d <= 32,
 * 1 <= k <= 64; not for a batch.  Synchronises.
 */
PFE_API pfe_status pfe_kmeans(pfe_ctx *c, const double *X, int32_t d, int32_t k, const double *C0, int32_t max_iter,
                              int32_t *labels, double *centroids, double *inertia, int32_t *rounds);

/*
 * pfe_objective -- diagnostics of the current embedding (FP64 reductions in a
 * fixed order): *l1 = |M Y|_1 = sum over undirected edges a < b of
 * w_ab |y_a - y_b|_1 (Eq. 1 sums every ordered pair, i.e. twice this), and
 * *ortho_err = |Y^T D Y - I|_F, the distance from the constraint of Eq. 1
 * (for a batch: the largest over its problems; l1 sums them).  which:
 * PFE_OBJ_Y the iterate Y of Alg. 2 (not constrained), PFE_OBJ_YHAT the
 * embedding D^{-1/2} P (constrained after every P-step).  Either output may
 * be NULL.  Synchronises; uses the staging buffer.
 */
enum { PFE_OBJ_Y = 0, PFE_OBJ_YHAT = 1 };
PFE_API pfe_status pfe_objective(pfe_ctx *c, int32_t which, double *l1, double *ortho_err);

/*
 * pfe_residual -- how well X solves the linear systems of Eq. 13 (Sec. III:
 * the d systems A x_c = b_c that PCG solves, A = lambda M^T M + r D):
 * relres[s * d + c] = |b_c - A x_c|_2 / |b_c|_2 over the rows of problem s
 * (|b_c - A x_c|_2 where b_c = 0), computed in FP64 with the FP64 values of
 * A whatever the context's precision -- so it states a mixed-precision
 * solve's residual against the problem's matrix, not against the FP32
 * rounding of A that its iteration multiplies by.  B and X: n x d row-major
 * FP64, host or device (host arrays are copied through a temporary device
 * buffer); relres: host, nseg * d.  Sums in a fixed order.  Needs pfe_init
 * (d); synchronises.
 */
PFE_API pfe_status pfe_residual(pfe_ctx *c, const double *B, const double *X, double *relres);

/*
 * pfe_laplacian_eigenmap -- the Laplacian-eigenmap embedding of the graph
 * (Sec. I, the l2 analogue of Eq. 1; Belkin & Niyogi): the d generalised
 * eigenvectors of (D - W) v = mu D v with the smallest mu on the
 * D-orthogonal complement of the constant vector (the trivial solution), in
 * ascending mu, with v^T D v = 1, each signed so that its entry of largest
 * magnitude is positive (ties: the smallest index).  V is n x d row-major FP64
 * (host or device).  Chebyshev-filtered subspace iteration on D^{-1} W in
 * FP64 until every wanted residual |D^{-1} W v - (1 - mu) v|_D <= tol or
 * max_iter rounds (PFE_ENOTCONV, results written); *iters and *residual
 * (either may be NULL) receive the rounds and the largest residual.  Needs
 * n > d + 2 + d/4 and d <= 30; not for a batch.  Synchronises; allocates
 * temporary device memory.
 */
PFE_API pfe_status pfe_laplacian_eigenmap(pfe_ctx *c, int32_t d, double *V, int32_t max_iter, double tol,
                                          int32_t *iters, double *residual);

/*
 * pfe_inner_step -- one split-Bregman iteration (Alg. 2 steps 5-7 in the
 * compact form): solve Eq. 13 for Y by PCG (warm-started from the previous
 * Y), then d = Shrink(M Y + b, 1/lambda) (Eq. 9), b = b + M Y - d (Eq. 10),
 * and the next right-hand side lambda M^T (d - b) + r D^{1/2} (P - B), all
 * fused in one edge pass.  Only enqueues work unless st != NULL, in which
 * case it synchronises and fills *st.  PFE_ENOTCONV / PFE_ENUMERIC are
 * reported by the call that synchronises.
 */
PFE_API pfe_status pfe_inner_step(pfe_ctx *c, pfe_step_stats *st);

/*
 * pfe_pstep -- close an outer iteration: Alg. 1 steps 6-7,
 * P = polar(D^{1/2} Y + B) (orthogonal Procrustes solution, FP64),
 * B = B + D^{1/2} Y - P, then restart the inner variables (b = d = 0) when
 * reset_inner_each_outer is set.  Enqueues only.
 */
PFE_API pfe_status pfe_pstep(pfe_ctx *c);

/*
 * pfe_solve -- run n_outer outer iterations of Alg. 1, each with n_inner
 * inner iterations of Alg. 2, from the current state.  Writes (when non-NULL)
 * Y_out = the last split-Bregman solution Y and Yhat_out = D^{-1/2} P (which
 * satisfies Yhat^T D Yhat = I), both n x d FP64 row-major, host or device.
 * Synchronises once at the end; fills *st when non-NULL.
 */
PFE_API pfe_status pfe_solve(pfe_ctx *c, int32_t n_outer, int32_t n_inner, double *Y_out,
                     double *Yhat_out, pfe_solve_stats *st);

/*
 * pfe_solve_two_stage -- the two-stage schedule of Sec. IV: Stage I is
 * pfe_solve(n_outer, n_inner) (SOC iterations with P-steps); Stage II relaxes
 * the orthogonality constraint -- P and B keep their Stage I values and only
 * penalise it through the r-term -- and runs n_stage2 further split-Bregman
 * iterations (one more call of Alg. 2: b = d = 0 at its start).  The paper's
 * counts: at most 10 x 5 in Stage I, 100 in Stage II.  Y_out receives Stage
 * II's Y, Yhat_out D^{-1/2} P of Stage I; statistics and status as pfe_solve.
 */
PFE_API pfe_status pfe_solve_two_stage(pfe_ctx *c, int32_t n_outer, int32_t n_inner, int32_t n_stage2,
                                       double *Y_out, double *Yhat_out, pfe_solve_stats *st);

/* Frees every library allocation of the context (NULL is allowed). */
PFE_API pfe_status pfe_destroy(pfe_ctx *c);

/* Message of the last failed call on c (never NULL; "" when none).  With
 * c = NULL: the message of the last pfe_build_graph on the calling thread
 * that failed (its context no longer exists), "" if that call succeeded. */
PFE_API const char *pfe_last_error(const pfe_ctx *c);

/* Human-readable name of a status code (static storage). */
PFE_API const char *pfe_status_string(pfe_status s);

/* Sizes and parameters of a context. Never synchronises. */
PFE_API pfe_status pfe_get_info(const pfe_ctx *c, pfe_info *info);

/* Changes the stream later calls enqueue on.  Work already queued on the
 * previous stream is ordered before them (the new stream waits for it on
 * the device; the call does not block the host). */
PFE_API pfe_status pfe_set_stream(pfe_ctx *c, pfe_stream_t stream);

/* Segments of a batch (host arrays, either may be NULL): off[0..nseg] first
 * vertex of each problem (off[nseg] = n), lambda[0..nseg-1] the penalty in
 * use for each.  Never synchronises. */
PFE_API pfe_status pfe_get_segments(const pfe_ctx *c, int64_t *off, double *lambda);

/* Per-problem outcome of the PCG solves (after pfe_init; host arrays, any
 * may be NULL): iters[s] iterations problem s ran in the last solve before
 * all its columns reached tol (or the cap), relres[s*d + c] the final
 * relative residual of its column c, iters_total[s] its iterations summed
 * over the solves of the last pfe_solve call.  Synchronises. */
PFE_API pfe_status pfe_get_segment_stats(pfe_ctx *c, int32_t *iters, double *relres, int64_t *iters_total);

/*
 * State arrays, for checkpoint/resume and for tests (all FP64, row-major,
 * host or device pointers; converted from the working precision):
 *   PFE_ARR_Y     n x d    current Y (last solve, or the start after pfe_init)
 *   PFE_ARR_P     n x d    P of Alg. 1
 *   PFE_ARR_B     n x d    B of Alg. 1
 *   PFE_ARR_BS    |E| x d  split-Bregman b (Alg. 2), rows in pfe_get_edges order
 *   PFE_ARR_RHS   n x d    right-hand side of the next solve (Eq. 13, times 2)
 *   PFE_ARR_DEG   n        d_i = sum_j w_ij
 *   PFE_ARR_DIAG  n        diagonal of A = lambda M^T M + r D
 * pfe_get_array synchronises.  pfe_set_array accepts Y, P, B, BS and RHS;
 * restoring all five after pfe_init(d) resumes an iteration exactly (Y also
 * restores the extended-precision part of the mixed path when set from FP64).
 */
enum { PFE_ARR_Y = 0, PFE_ARR_P = 1, PFE_ARR_B = 2, PFE_ARR_BS = 3, PFE_ARR_RHS = 4,
       PFE_ARR_DEG = 5, PFE_ARR_DIAG = 6 };
PFE_API pfe_status pfe_get_array(pfe_ctx *c, int32_t which, double *dst);
PFE_API pfe_status pfe_set_array(pfe_ctx *c, int32_t which, const double *src);

/*
 * Undirected edges in the library's numbering: a[k] < b[k] and the heat-kernel
 * weight w[k] (any of the three may be NULL).  Each array has n_edges entries
 * (host or device).  For PFE_GRAPH_EDGES input, edge k is input pair k.
 * Synchronises.
 */
PFE_API pfe_status pfe_get_edges(pfe_ctx *c, int32_t *a, int32_t *b, double *w);

/*
 * pfe_apply_A -- Yout = A X for n x d FP64 arrays (host or device), computed
 * by the library's SpMM kernel in the working precision (the product that
 * every PCG iteration performs).  Requires pfe_init (fixes d).  Synchronises.
 */
PFE_API pfe_status pfe_apply_A(pfe_ctx *c, const double *X, double *Yout);

/*
 * pfe_solve_system -- solve A Y = RHS (Eq. 13) by the configured PCG, with Y
 * holding the initial guess on entry and the solution on exit (n x d FP64,
 * host or device).  Does not touch the iteration state except scratch
 * vectors.  Synchronises; fills *st when non-NULL.
 */
PFE_API pfe_status pfe_solve_system(pfe_ctx *c, const double *RHS, double *Y, pfe_step_stats *st);

/*
 * pfe_time_kernel -- average device time of one hot-path kernel, for
 * roofline reporting: `reps` back-to-back launches on the context's current
 * state (after pfe_init), bracketed by CUDA events on the context's stream.
 *   PFE_KERNEL_SPMM     q = A p with the p.q column dots (one per PCG iteration)
 *   PFE_KERNEL_UPDATE   r -= alpha q with the r.z, r.r column dots
 *   PFE_KERNEL_EDGE     fused M Y / Shrink / b update / M^T scatter (Eqs. 7, 9, 10, 13)
 *   PFE_KERNEL_PUPDATE  p_new = D_A^{-1} r + beta p with the two delayed
 *                       solution updates y += alpha_prev p_prev + alpha p
 *                       (every other iteration)
 *   PFE_KERNEL_PUPDATE_HOLD  the same launch on the other iterations, which
 *                       hold the solution update (no pass over y)
 *   PFE_KERNEL_FSAI_TR  r -= alpha q fused with t = G r and the column dots
 *                       t.t (= r.z) and r.r (FSAI preconditioner set)
 *   PFE_KERNEL_FSAI_ZP  z = G^T t fused with p_new = z + beta p and the two
 *                       delayed solution updates y += alpha_prev p_prev +
 *                       alpha p (every other iteration); z is not stored
 *                       (FSAI preconditioner set)
 *   PFE_KERNEL_FSAI_ZP_HOLD  the same launch on the other iterations, which
 *                       hold the solution update (no pass over y)
 *   PFE_KERNEL_REPLACE  the residual replacement r = b - A y with A's FP64
 *                       values (k_refresh; k_refresh_f with an FSAI factor),
 *                       run on replacement iterations only
 *   PFE_KERNEL_XFLUSH   y += alpha_prev p_prev + alpha p, applying the pending
 *                       solution updates ahead of a replacement
 *   PFE_KERNEL_FSAI_T   t = G r with the column dots after a replacement
 *                       (FSAI factor set)
 *   PFE_KERNEL_MLP      the learned factor's network inference over every
 *                       pattern entry, on the path PFE_TUNE_MLP selects
 *                       (after pfe_fsai_set; rewrites G with the same values)
 * The iteration state is not modified (scratch copies and a scratch control
 * block are used; the timed edge passes write the spare b buffer and a
 * scratch right-hand side).  Only
 * the PCG direction p and product q, which every solve re-initialises, are
 * overwritten.  Synchronises; allocates temporary device memory.  Returns
 * PFE_EUNSUPPORTED for an FSAI kernel without the FSAI preconditioner set,
 * PFE_EINVAL for an unknown id.
 */
enum {
    PFE_KERNEL_SPMM = 0,
    PFE_KERNEL_UPDATE = 1,
    PFE_KERNEL_EDGE = 2,
    PFE_KERNEL_PUPDATE = 3,
    PFE_KERNEL_FSAI_TR = 4,
    PFE_KERNEL_FSAI_ZP = 5,
    PFE_KERNEL_FSAI_ZP_HOLD = 6,
    PFE_KERNEL_PUPDATE_HOLD = 7,
    PFE_KERNEL_REPLACE = 8,
    PFE_KERNEL_XFLUSH = 9,
    PFE_KERNEL_FSAI_T = 10,
    PFE_KERNEL_MLP = 11
};
PFE_API pfe_status pfe_time_kernel(pfe_ctx *c, int32_t which, int32_t reps, double *avg_ms);

/*
 * Learned FSAI preconditioner (no counterpart in the paper, which uses an
 * incomplete-Cholesky preconditioner, Sec. III).  The PCG of the mixed path
 * can use M^{-1} = G^T G with G lower triangular on the pattern of
 * tril(A): G_ij = Gh_ij / sqrt(A_jj), Gh_ii = softplus(h_diag),
 * Gh_ij = h_off, where (h_off, h_diag) is a 4 -> 64 -> 64 -> 2 ReLU network
 * evaluated per pattern entry.  Edge entry (b, a), a < b, reads
 * (lam w_ab^2 / sqrt(A_aa A_bb), r d_b / A_bb, r d_a / A_aa, w_ab); diagonal
 * entry i reads (sum over lower neighbours j of the first feature squared,
 * r d_i / A_ii, r d_i / A_ii, 1).  The hidden 64 x 64 layer runs on the
 * tensor cores (BF16 operands, FP32 accumulation).
 *
 * params: pfe_fsai_param_count() FP32 values (host or device), laid out as
 * W1 (4 x 64 row-major), b1 (64), W2 (64 x 64), b2 (64), W3 (64 x 2), b3 (2).
 * A network with W3 = 0 and b3 = (0, softplus^{-1}(1)) gives G = D_A^{-1/2},
 * i.e. exactly the Jacobi preconditioner.
 */
PFE_API int32_t pfe_fsai_param_count(void);

/* Evaluates the network on every pattern entry (G is built once per graph)
 * and makes later PCG solves use G^T G.  On a batch every problem's entries
 * read its own lambda (G is block diagonal like A) and every problem keeps
 * its own PCG scalars and convergence.  params == NULL switches back to
 * Jacobi.  PFE_EUNSUPPORTED on an FP64 context.  Synchronises. */
PFE_API pfe_status pfe_fsai_set(pfe_ctx *c, const float *params);

/* The classical FSAI factor on the same pattern (no network): for each row
 * i with pattern S (i and its lower neighbours), A[S,S] g = e_i solved in
 * FP64 and scaled by 1/sqrt(g_i).  It minimises the Kaporin number over the
 * pattern and bounds what the learned factor can reach.  Switches the PCG to
 * G^T G like pfe_fsai_set.  PFE_EUNSUPPORTED on an FP64 context or when a
 * row has more than 23 lower neighbours.  Synchronises. */
PFE_API pfe_status pfe_fsai_classical(pfe_ctx *c);

/* The paper's preconditioner (Sec. III: conjugate gradients with an
 * incomplete Cholesky factorisation), in its zero-fill form IC(0): L lower
 * triangular on the pattern of tril(A) with (L L^T)_ij = A_ij on the
 * pattern, factored in FP64 on the GPU; later PCG solves use
 * M^{-1} = L^{-T} L^{-1}.  The triangular solves are sequential along a
 * wavefront: they run one launch per level (W + c (H - 1) levels, c = 2 at
 * radius 2 and 3 at radius 3), which is why the FSAI forms are the fast
 * path; IC(0) is the comparator.  L is readable with pfe_fsai_get (L_ii and
 * L_ba per edge).  One grid image of radius 2 or 3 on the mixed-precision
 * path; PFE_EUNSUPPORTED otherwise, PFE_ENUMERIC on a non-positive pivot
 * (not possible for this system matrix, an M-matrix).  pfe_fsai_set(c, NULL)
 * switches back to Jacobi.  Synchronises. */
PFE_API pfe_status pfe_ic0(pfe_ctx *c);

/* Training criterion: Kaporin's condition number of G A G^T,
 *   *loss = log(tr(G A G^T) / n) - (2/n) sum_i log G_ii,
 * and its gradient with respect to params (written to grad when non-NULL,
 * host or device).  Does not change which preconditioner the PCG uses, but
 * G is recomputed from params.  One problem per context (PFE_EUNSUPPORTED
 * on a batch).  Synchronises. */
PFE_API pfe_status pfe_fsai_loss_grad(pfe_ctx *c, const float *params, float *grad, double *loss);

/* pfe_fsai_loss_grad_rhs -- pfe_fsai_loss_grad plus mu times the mean
 * relative residual of the preconditioner on m right-hand sides B of Eq. 13
 * that the method produced (n x m FP64, row-major, host or device; 1 <= m
 * <= 32, every column nonzero):
 *   R = (1/m) sum_c |A G^T G b_c - b_c|^2 / |b_c|^2,   loss = K(G) + mu R,
 * with A in FP64 and the gradient of both terms w.r.t. params (dR/dG_ij =
 * u_i s_j + (G s)_i b_j with u = G b, s = 2 A (A G^T G b - b) / (m |b|^2),
 * on G's pattern).  *rterm (may be NULL) receives R.  mu = 0 or B = NULL
 * is pfe_fsai_loss_grad.  Allocates its scratch vectors (five n x m FP64)
 * for the call.  Synchronises. */
PFE_API pfe_status pfe_fsai_loss_grad_rhs(pfe_ctx *c, const float *params, const double *B, int32_t m, double mu,
                                          float *grad, double *loss, double *rterm);

/* The current G as FP64: gdiag[i] = G_ii (n values), gedge[k] = G_{b_k a_k}
 * for edge k of pfe_get_edges (n_edges values); either may be NULL. */
PFE_API pfe_status pfe_fsai_get(pfe_ctx *c, double *gdiag, double *gedge);

/* One Adam step on device arrays of `count` FP32 values:
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   p -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * step >= 1.  Enqueues on `stream` only. */
PFE_API pfe_status pfe_adam_update(float *params, const float *grad, float *m, float *v, int64_t count,
                                   int32_t step, double lr, double beta1, double beta2, double eps,
                                   pfe_stream_t stream);

/*
 * pfe_orthonormalize_noalloc -- the D-orthonormalisation that pfe_init
 * applies to a starting embedding, Yhat = D^{-1/2} polar(D^{1/2} Y), with no
 * device memory allocated at all.  (There is no counterpart in the paper:
 * this entry point exists for callers, not for the method.)
 *
 * Who needs it: code that cannot call cudaMalloc -- a plug-in inside a host
 * application that owns every device allocation through its own memory pool
 * (a stray cudaMalloc would bypass the pool's accounting or fail against its
 * reservation), or a service that sizes device memory once at start-up and
 * must not grow it later.  Every other libpfe entry point allocates its
 * buffers itself.
 *
 * Y (n x d) and deg (n, every d_i > 0) are FP64 device arrays the caller
 * owns; Yhat (n x d, FP64 device, may not alias Y) receives the result,
 * which satisfies Yhat^T D Yhat = I.  The scratch (the Gram matrix's block
 * partials and a small control block, about 0.6 MB) is a fixed array
 * compiled into the library: every GPU that loads libpfe holds it until the
 * process exits.  Limits: 1 <= d <= 16 and d <= n; larger d, host
 * pointers or NULL give PFE_EINVAL before any work is queued.
 *
 * All calls on a device share that array and it keeps the last call's
 * contents (each call clears the ticket and error word it starts from and
 * rewrites the rest before reading it), so calls that overlap on the GPU --
 * two streams at once, or two threads -- race and must be serialised by the
 * caller.  The first call on each device looks up the array's device
 * address once (with that device current) and keeps it for the life of the
 * process; make that first call before any stream capture, and do not call
 * the entry point again on a device after cudaDeviceReset (the kept address
 * belongs to the context that was reset).  The call queues its work on
 * `stream` and synchronises it to report PFE_ESINGULAR when D^{1/2} Y is
 * numerically rank deficient (Yhat is then left as it was).  It calls no
 * allocating routine.
 */
PFE_API pfe_status pfe_orthonormalize_noalloc(const double *Y, const double *deg, int64_t n, int32_t d,
                                              double *Yhat, pfe_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* PFE_H */
