// The C ABI of libpfe (include/pfe.h): context life cycle, argument checks,
// host/device staging, the PCG loop driver (CUDA graph with a WHILE node, or
// a host poll loop) and the SOC / split-Bregman loop (Alg. 1 around Alg. 2).
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

using namespace pfe;

namespace {

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

pfe_status fail(pfe_ctx *c, pfe_status s, const char *msg) {
    if (c) c->err = msg;
    return s;
}

template <typename P>
pfe_status walloc(pfe_ctx *c, P **p, int64_t count) {
    size_t bytes = (size_t)std::max<int64_t>(count, 1) * sizeof(P);
    *p = nullptr;
    if (over_device_cap(c, bytes)) return PFE_ENOMEM;
    cudaError_t e = cudaMalloc((void **)p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->err = std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e);
        *p = nullptr;
        return PFE_ENOMEM;
    }
    c->work_allocs.push_back((void *)*p);
    c->bytes += (int64_t)bytes;
    c->work_bytes += (int64_t)bytes;
    return PFE_OK;
}

void free_pcg_graph(pfe_ctx *c) {
    if (c->pcg_exec) cudaGraphExecDestroy(c->pcg_exec);
    if (c->pcg_graph) cudaGraphDestroy(c->pcg_graph);
    c->pcg_exec = nullptr;
    c->pcg_graph = nullptr;
}

void free_work(pfe_ctx *c) {
    free_pcg_graph(c);
    for (void *p : c->work_allocs) cudaFree(p);
    c->work_allocs.clear();
    c->bytes -= c->work_bytes;
    c->work_bytes = 0;
    c->wk = Work{};
    c->fsai.t = nullptr;
    c->fsai.r1 = nullptr;
    c->sc = SegScal{};
    c->seg_T = nullptr;
    c->seg_pticket = nullptr;
    c->inited = false;
    c->d = 0;
}

pfe_status sync(pfe_ctx *c) {
    PFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PFE_OK;
}

// Laplacian-eigenmap start of pfe_init: iteration cap, residual tolerance
// (|P v - theta v|_D of each wanted vector) and Chebyshev filter degree.
constexpr int kLeMaxIter = 400;
constexpr double kLeTol = 1e-9;
constexpr int kLeDegree = 10;

// Work vectors of the FSAI iteration: t = G r and the second residual buffer
// (n x d each, work precision float).
pfe_status fsai_vectors(pfe_ctx *c, int64_t nd) {
    float *t, *r1;
    PFE_TRY(walloc(c, &t, nd));
    PFE_TRY(walloc(c, &r1, nd));
    c->fsai.t = t;
    c->fsai.r1 = r1;
    return PFE_OK;
}

// Launches per solve: the init kernels plus the final flush, per iteration
// those that run every iteration, and those of a residual replacement (k_xflush
// and the replacement kernels, which run only on replacement iterations when
// the captured loop puts them in IF nodes; the device adds them up in
// pfe_solve_stats).
void launch_counts(const pfe_ctx *c, int lc[3]) {
    if (c->fsai.enabled && c->fsai.ic) {
        // the triangular solves: one launch per level that holds a row
        int64_t nl = 0;
        const int64_t W = c->W, H = c->g.n / W;
        for (int64_t l = 0; l < c->fsai.ic_levels; ++l) {
            int64_t y0 = 0, rows = 0;
            ic_level_rows(l, W, H, c->fsai.ic_cl, y0, rows);
            nl += rows > 0;
        }
        lc[0] = (int)(2 * nl + 3);
        lc[1] = (int)(2 * nl + 3);
        lc[2] = 2;
        return;
    }
    lc[0] = c->fsai.enabled ? 4 : 2;
    lc[1] = 3;
    lc[2] = c->fsai.enabled ? 3 : 2;
}

pfe_status write_launch_counts(pfe_ctx *c) {
    int lc[3];
    launch_counts(c, lc);
    PFE_CUDA_TRY(c, cudaMemcpyAsync((char *)c->ctl + offsetof(PcgCtl, launch_base), lc, 2 * sizeof(int),
                                    cudaMemcpyHostToDevice, c->stream));
    PFE_CUDA_TRY(c, cudaMemcpyAsync((char *)c->ctl + offsetof(PcgCtl, launch_cond), lc + 2, sizeof(int),
                                    cudaMemcpyHostToDevice, c->stream));
    return PFE_OK;
}

// After the preconditioner changed: drop the captured loop (its body differs
// between preconditioners) and update the launch counts.
pfe_status fsai_switched(pfe_ctx *c) {
    free_pcg_graph(c);
    if (c->inited) PFE_TRY(write_launch_counts(c));
    return sync(c);
}

// Build the CUDA graph {init kernel -> WHILE(body of check_every iterations)}.
// The replacement kernels of each iteration of the body sit in a conditional
// IF node (handles made on the top graph, values set by the kernel that
// decides each replacement, cleared when the solve ends).
pfe_status build_pcg_graph(pfe_ctx *c) {
    free_pcg_graph(c);
    cudaStream_t cs, side;
    PFE_CUDA_TRY(c, cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    if (cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking) != cudaSuccess) {
        cudaStreamDestroy(cs);
        PFE_CUDA_TRY(c, cudaGetLastError());
        return fail(c, PFE_ECUDA, "PCG graph: stream creation failed");
    }
    struct StreamGuard {
        cudaStream_t s, t;
        ~StreamGuard() {
            cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
            for (cudaStream_t q : {s, t})
                if (cudaStreamIsCapturing(q, &st) == cudaSuccess && st != cudaStreamCaptureStatusNone) {
                    cudaGraph_t g = nullptr;
                    cudaStreamEndCapture(q, &g);  // an abandoned capture (error path)
                }
            cudaGetLastError();
            cudaStreamDestroy(s);
            cudaStreamDestroy(t);
        }
    } guard{cs, side};
    cudaGraph_t g = nullptr;
    PFE_CUDA_TRY(c, cudaGraphCreate(&g, 0));
    c->pcg_graph = g;
    cudaGraphConditionalHandle h;
    PFE_CUDA_TRY(c, cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    PcgLaunch L{h, 1};
    const int iters = std::max(1, c->prm.check_every);
    if (iters <= kPcgMaxIf) {
        L.n_if = iters;
        L.side = side;
        for (int k = 0; k < iters; ++k)
            PFE_CUDA_TRY(c, cudaGraphConditionalHandleCreate(&L.ifh[k], g, 0, cudaGraphCondAssignDefault));
    }
    PFE_CUDA_TRY(c, cudaMemcpyAsync((char *)c->ctl + offsetof(PcgCtl, ifh), L.ifh, sizeof(L.ifh),
                                    cudaMemcpyHostToDevice, c->stream));
    PFE_CUDA_TRY(c, cudaMemcpyAsync((char *)c->ctl + offsetof(PcgCtl, n_if), &L.n_if, sizeof(int),
                                    cudaMemcpyHostToDevice, c->stream));
    PFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // L lives on this stack frame
    PFE_CUDA_TRY(c, cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    pfe_status st = launch_pcg_init(c, cs, L);
    cudaGraph_t g2 = g;
    cudaError_t ce = cudaStreamEndCapture(cs, &g2);
    if (st != PFE_OK) return st;
    PFE_CUDA_TRY(c, ce);
    size_t nn = 0;
    PFE_CUDA_TRY(c, cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    PFE_CUDA_TRY(c, cudaGraphGetNodes(g, nodes.data(), &nn));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cn;
    PFE_CUDA_TRY(c, cudaGraphAddNode(&cn, g, nodes.data(), nullptr, nn, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    PFE_CUDA_TRY(c, cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    st = launch_pcg_body(c, cs, L, iters);
    cudaGraph_t b2 = body;
    ce = cudaStreamEndCapture(cs, &b2);
    if (st != PFE_OK) return st;
    PFE_CUDA_TRY(c, ce);
    // the delayed solution update of the last iteration, after the loop
    PFE_CUDA_TRY(c, cudaStreamBeginCaptureToGraph(cs, g, &cn, nullptr, 1, cudaStreamCaptureModeThreadLocal));
    st = launch_pcg_final(c, cs, L);
    cudaGraph_t g3 = g;
    ce = cudaStreamEndCapture(cs, &g3);
    if (st != PFE_OK) return st;
    PFE_CUDA_TRY(c, ce);
    PFE_CUDA_TRY(c, cudaGraphInstantiate(&c->pcg_exec, g, 0));
    return PFE_OK;
}

// One PCG solve A Y = RHS on the work arrays, no host synchronisation in graph mode.
pfe_status run_pcg(pfe_ctx *c, bool force_host) {
    if (!force_host && c->prm.loop_mode == PFE_LOOP_GRAPH) {
        if (!c->pcg_exec) PFE_TRY(build_pcg_graph(c));
        PFE_CUDA_TRY(c, cudaGraphLaunch(c->pcg_exec, c->stream));
        return PFE_OK;
    }
    PcgLaunch L{0, 0};
    PFE_TRY(launch_pcg_init(c, c->stream, L));
    const int chunk = std::max(1, c->prm.check_every);
    const int64_t cap = (int64_t)c->prm.max_iter + 2 * chunk + 8;
    for (int64_t it = 0;; it += chunk) {
        PFE_TRY(launch_pcg_body(c, c->stream, L, chunk));
        PFE_CUDA_TRY(c, cudaMemcpyAsync(c->h_flag, &c->ctl->done, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        PFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        if (*c->h_flag) break;
        if (it > cap) return fail(c, PFE_ECUDA, "PCG control block never reported completion");
    }
    PFE_TRY(launch_pcg_final(c, c->stream, L));
    return PFE_OK;
}

pfe_status read_ctl(pfe_ctx *c) {
    PFE_CUDA_TRY(c, cudaMemcpyAsync(c->h_ctl, c->ctl, sizeof(PcgCtl), cudaMemcpyDeviceToHost, c->stream));
    PFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return PFE_OK;
}

pfe_status clear_stats(pfe_ctx *c) {
    // zero the statistics (tot_iters .. last_converged) and the launch counter
    const size_t off = offsetof(PcgCtl, tot_iters), end = offsetof(PcgCtl, unroll);
    PFE_CUDA_TRY(c, cudaMemsetAsync((char *)c->ctl + off, 0, end - off, c->stream));
    PFE_CUDA_TRY(c, cudaMemsetAsync((char *)c->ctl + offsetof(PcgCtl, launches), 0, sizeof(long long), c->stream));
    if (c->sc.seg_iters_tot)
        PFE_CUDA_TRY(c, cudaMemsetAsync(c->sc.seg_iters_tot, 0, sizeof(long long) * c->nseg, c->stream));
    return PFE_OK;
}

pfe_status check_pstep(pfe_ctx *c) {
    int e = 0;
    PFE_CUDA_TRY(c, cudaMemcpyAsync(c->h_flag, &c->pctl->error, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PFE_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    e = *c->h_flag;
    if (e) return fail(c, PFE_ESINGULAR, "P-step: X^T X is numerically singular");
    return PFE_OK;
}

// The device's PCG error word (host copy must be fresh) as a status.
pfe_status pcg_error(pfe_ctx *c) {
    if (c->h_ctl->error == PFE_ETIMEOUT)
        return fail(c, PFE_ETIMEOUT, "PCG: a bounded device wait ran out, or the loop stopped advancing");
    return fail(c, PFE_ENUMERIC, "PCG: NaN/Inf or non-positive p^T A p");
}

// status of the solves since the last clear_stats (host copy must be fresh)
pfe_status pcg_status(pfe_ctx *c) {
    if (c->h_ctl->error) return pcg_error(c);
    if (c->h_ctl->n_unconv > 0) return fail(c, PFE_ENOTCONV, "PCG: max_iter reached before tol");
    return PFE_OK;
}

size_t elem_size(const pfe_ctx *c) { return c->mixed ? sizeof(float) : sizeof(double); }

pfe_status inner_step_enqueue(pfe_ctx *c) {
    NvtxRange r("pfe inner step");
    {
        NvtxRange r1("pcg");
        PFE_TRY(run_pcg(c, false));
    }
    NvtxRange r2("edge pass");
    PFE_TRY(launch_edge(c, c->stream));
    return PFE_OK;
}

pfe_status pstep_enqueue(pfe_ctx *c) {
    NvtxRange r("pfe P-step");
    const bool reset = c->prm.reset_inner_each_outer != 0;
    PFE_TRY(launch_pstep(c, c->stream, reset ? PSTEP_RESET : PSTEP_CARRY));
    if (reset) {
        const size_t bytes = (size_t)c->g.fslots * c->d * elem_size(c);
        PFE_CUDA_TRY(c, cudaMemsetAsync(c->wk.Bs[c->bs_cur], 0, bytes, c->stream));
    }
    return PFE_OK;
}

}  // namespace

extern "C" {

void pfe_default_params(pfe_params *p) {
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->lambda = 0.0;
    p->r = 1.0;
    p->precision = PFE_MIXED;
    p->precond = PFE_PRECOND_JACOBI;
    p->tol = 1e-6;
    p->max_iter = 5000;
    p->refresh = 50;
    p->reset_inner_each_outer = 1;
    p->loop_mode = PFE_LOOP_GRAPH;
    p->check_every = 4;
    p->blocks_per_sm = 0;
}

const char *pfe_status_string(pfe_status s) {
    switch (s) {
        case PFE_OK: return "PFE_OK";
        case PFE_EINVAL: return "PFE_EINVAL";
        case PFE_ENOMEM: return "PFE_ENOMEM";
        case PFE_ECUDA: return "PFE_ECUDA";
        case PFE_ENOTCONV: return "PFE_ENOTCONV";
        case PFE_ENUMERIC: return "PFE_ENUMERIC";
        case PFE_ESINGULAR: return "PFE_ESINGULAR";
        case PFE_ETIMEOUT: return "PFE_ETIMEOUT";
        case PFE_EUNSUPPORTED: return "PFE_EUNSUPPORTED";
        case PFE_ESTATE: return "PFE_ESTATE";
    }
    return "PFE_?";
}

// Message of the last pfe_build_graph on this thread that failed (its
// context is gone by then, so the message cannot live in one).
static thread_local std::string t_build_err;

const char *pfe_last_error(const pfe_ctx *c) { return c ? c->err.c_str() : t_build_err.c_str(); }

pfe_status pfe_destroy(pfe_ctx *c) {
    if (!c) return PFE_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_work(c);
    for (void *p : c->dev_allocs) cudaFree(p);
    if (c->ctl) cudaFree(c->ctl);
    if (c->pctl) cudaFree(c->pctl);
    if (c->h_ctl) cudaFreeHost(c->h_ctl);
    if (c->h_flag) cudaFreeHost(c->h_flag);
    delete c;
    return PFE_OK;
}

static pfe_status build_graph_impl(pfe_ctx **out, const pfe_graph_desc *gd, const pfe_params *p,
                                   pfe_stream_t stream) {
    if (!out) return PFE_EINVAL;
    *out = nullptr;
    if (!gd || !p) return PFE_EINVAL;
    if (gd->n < 2 || gd->m < 1 || !gd->features || !(gd->sigma > 0.0)) return PFE_EINVAL;
    if (gd->n > (int64_t)INT32_MAX - 64) return PFE_EINVAL;
    const int nseg = gd->nseg > 1 ? gd->nseg : 1;
    if (gd->nseg < 0 || nseg > PFE_MAX_SEGMENTS) return PFE_EINVAL;
    std::vector<int64_t> soff(nseg + 1, 0);
    std::vector<int> sh(nseg, 0), sw(nseg, 0);
    if (gd->kind == PFE_GRAPH_GRID) {
        if (!(gd->radius >= 1.0) || gd->radius > 8.0) return PFE_EINVAL;
        if (nseg == 1) {
            if (gd->H < 1 || gd->W < 1 || (int64_t)gd->H * gd->W != gd->n) return PFE_EINVAL;
            sh[0] = gd->H;
            sw[0] = gd->W;
        } else {
            if (!gd->seg_hw) return PFE_EINVAL;
            for (int q = 0; q < nseg; ++q) {
                sh[q] = gd->seg_hw[2 * q];
                sw[q] = gd->seg_hw[2 * q + 1];
                if (sh[q] < 1 || sw[q] < 1 || (int64_t)sh[q] * sw[q] < 2) return PFE_EINVAL;
                soff[q + 1] = soff[q] + (int64_t)sh[q] * sw[q];
            }
            if (soff[nseg] != gd->n) return PFE_EINVAL;
        }
        soff[nseg] = gd->n;
    } else if (gd->kind == PFE_GRAPH_EDGES) {
        if (nseg > 1) {
            if (!gd->seg_off || gd->seg_off[0] != 0 || gd->seg_off[nseg] != gd->n) return PFE_EINVAL;
            for (int q = 0; q < nseg; ++q) {
                if (gd->seg_off[q + 1] - gd->seg_off[q] < 2) return PFE_EINVAL;
                soff[q + 1] = gd->seg_off[q + 1];
            }
        }
        soff[nseg] = gd->n;
        if (gd->n_edges < 1 || !gd->ei || !gd->ej || gd->n_edges > (int64_t)INT32_MAX / 2) return PFE_EINVAL;
    } else {
        return PFE_EINVAL;
    }
    if (!(p->r > 0.0) || !(p->tol >= 0.0) || p->max_iter < 1 || p->refresh < 0) return PFE_EINVAL;
    if (p->precision != PFE_FP64 && p->precision != PFE_MIXED) return PFE_EINVAL;
    if (p->precond != PFE_PRECOND_JACOBI) return PFE_EUNSUPPORTED;
    if (p->loop_mode != PFE_LOOP_GRAPH && p->loop_mode != PFE_LOOP_HOST) return PFE_EINVAL;

    pfe_ctx *c = new (std::nothrow) pfe_ctx();
    if (!c) return PFE_ENOMEM;
    c->prm = *p;
    c->stream = (cudaStream_t)stream;
    c->n = gd->n;
    c->m = gd->m;
    c->kind = gd->kind;
    c->H = gd->H;
    c->W = gd->W;
    c->radius = gd->radius;
    c->sigma = gd->sigma;
    c->mixed = p->precision == PFE_MIXED;
    c->g.n_edges = gd->kind == PFE_GRAPH_EDGES ? gd->n_edges : 0;
    c->g.n = gd->n;
    c->nseg = nseg;
    c->h_seg_off = soff;
    c->h_seg_h = sh;
    c->h_seg_w = sw;
    auto bail = [&](pfe_status s) {
        t_build_err = c->err;  // kept for pfe_last_error(NULL)
        pfe_destroy(c);
        return s;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) return bail(PFE_ECUDA);
    e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) return bail(PFE_ECUDA);
    if (cudaMalloc((void **)&c->ctl, sizeof(PcgCtl)) != cudaSuccess) return bail(PFE_ENOMEM);
    if (cudaMalloc((void **)&c->pctl, sizeof(PstepCtl)) != cudaSuccess) return bail(PFE_ENOMEM);
    if (cudaMallocHost((void **)&c->h_ctl, sizeof(PcgCtl)) != cudaSuccess) return bail(PFE_ENOMEM);
    if (cudaMallocHost((void **)&c->h_flag, 16) != cudaSuccess) return bail(PFE_ENOMEM);
    if (cudaMemsetAsync(c->ctl, 0, sizeof(PcgCtl), c->stream) != cudaSuccess) return bail(PFE_ECUDA);
    if (cudaMemsetAsync(c->pctl, 0, sizeof(PstepCtl), c->stream) != cudaSuccess) return bail(PFE_ECUDA);

    // stage the inputs on the device when they are host arrays
    const double *dfeat = gd->features;
    double *feat_tmp = nullptr;
    int32_t *ei_tmp = nullptr, *ej_tmp = nullptr;
    struct Frees {
        std::vector<void *> v;
        ~Frees() {
            for (void *q : v) cudaFree(q);
        }
    } frees;
    if (!is_device_ptr(gd->features)) {
        size_t bytes = sizeof(double) * (size_t)gd->n * gd->m;
        if (cudaMalloc((void **)&feat_tmp, bytes) != cudaSuccess) return bail(PFE_ENOMEM);
        frees.v.push_back(feat_tmp);
        if (cudaMemcpyAsync(feat_tmp, gd->features, bytes, cudaMemcpyDefault, c->stream) != cudaSuccess)
            return bail(PFE_ECUDA);
        dfeat = feat_tmp;
    }
    pfe_status st = setup_segments(c);
    if (st != PFE_OK) return bail(st);
    if (gd->kind == PFE_GRAPH_GRID) {
        st = build_grid_graph(c, dfeat);
    } else {
        const int32_t *dei = gd->ei, *dej = gd->ej;
        size_t bytes = sizeof(int32_t) * (size_t)gd->n_edges;
        if (!is_device_ptr(gd->ei)) {
            if (cudaMalloc((void **)&ei_tmp, bytes) != cudaSuccess) return bail(PFE_ENOMEM);
            frees.v.push_back(ei_tmp);
            if (cudaMemcpyAsync(ei_tmp, gd->ei, bytes, cudaMemcpyDefault, c->stream) != cudaSuccess)
                return bail(PFE_ECUDA);
            dei = ei_tmp;
        }
        if (!is_device_ptr(gd->ej)) {
            if (cudaMalloc((void **)&ej_tmp, bytes) != cudaSuccess) return bail(PFE_ENOMEM);
            frees.v.push_back(ej_tmp);
            if (cudaMemcpyAsync(ej_tmp, gd->ej, bytes, cudaMemcpyDefault, c->stream) != cudaSuccess)
                return bail(PFE_ECUDA);
            dej = ej_tmp;
        }
        st = build_edge_graph(c, dfeat, dei, dej);
        if (st == PFE_OK && nseg > 1) st = check_edges_in_segments(c);
    }
    if (st != PFE_OK) return bail(st);
    st = finish_graph_values(c);
    if (st != PFE_OK) return bail(st);
    int bps = p->blocks_per_sm > 0 ? p->blocks_per_sm : 4;
    int64_t want = (int64_t)c->num_sms * bps;
    int64_t need = (c->g.n_slices + kWarps - 1) / kWarps;
    c->grid_rows = (int)std::max<int64_t>(1, std::min(want, need));
    *out = c;
    return PFE_OK;
}

pfe_status pfe_build_graph(pfe_ctx **out, const pfe_graph_desc *gd, const pfe_params *p, pfe_stream_t stream) {
    NvtxRange r("pfe build graph");
    t_build_err.clear();
    const pfe_status st = build_graph_impl(out, gd, p, stream);
    if (st != PFE_OK && t_build_err.empty()) t_build_err = pfe_status_string(st);
    return st;
}

pfe_status pfe_set_stream(pfe_ctx *c, pfe_stream_t stream) {
    if (!c) return PFE_EINVAL;
    const cudaStream_t ns = (cudaStream_t)stream;
    if (ns != c->stream) {
        // work already queued on the old stream stays first: the new stream
        // waits for it on the device (the host does not block)
        cudaEvent_t ev;
        PFE_CUDA_TRY(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        cudaError_t e = cudaEventRecord(ev, c->stream);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ns, ev, 0);
        cudaEventDestroy(ev);  // released once the recorded work completes
        if (e != cudaSuccess) return fail(c, PFE_ECUDA, "pfe_set_stream: ordering the old stream before the new");
    }
    c->stream = ns;
    return PFE_OK;
}

pfe_status pfe_get_info(const pfe_ctx *c, pfe_info *info) {
    if (!c || !info) return PFE_EINVAL;
    info->n = c->n;
    info->n_edges = c->g.n_edges;
    info->nnz_A = c->n + 2 * c->g.n_edges;
    info->sell_slots = c->g.slots;
    info->d = c->d;
    info->precision = c->mixed ? PFE_MIXED : PFE_FP64;
    info->lambda = c->lambda;
    info->r = c->r;
    info->vol = c->vol;
    info->device_bytes = c->bytes;
    info->nseg = c->nseg;
    info->le_iters = c->le_iters;
    info->le_residual = c->le_residual;
    return PFE_OK;
}

// The SpMM variants that apply to a context (the fixed-length kernels need an
// FP32 single-problem graph with 12 or 28 slots per row).
static bool spmm_variant_applies(const pfe_ctx *c, int v) {
    if (v == PFE_SPMM_GENERAL) return true;
    if (!c->mixed || v <= 0 || v >= PFE_SPMM_NVARIANTS) return false;
    if (c->nseg > 1) return v == PFE_SPMM_ROW1 && c->g.row_len == 12;  // batches: one row group per step
    // the stencil form: one grid image whose rows start on 16-byte boundaries
    if (v == PFE_SPMM_STENCIL &&
        (c->kind != PFE_GRAPH_GRID || c->W < 1 || c->W % 4 != 0 || stencil_strip(c->d, c->g.row_len, kStencilSteps) == 0))
        return false;
    // computed columns: one grid image
    if ((v == PFE_SPMM_GRID1 || v == PFE_SPMM_GRID2) && (c->kind != PFE_GRAPH_GRID || c->W < 1)) return false;
    return c->g.row_len == 12 || c->g.row_len == 28;
}

// The FSAI column forms that apply: slot columns always; columns computed
// from the stencil on one FP32 grid image of 12 or 28 slots a row with the
// (learned or classical) FSAI factor set.
static bool fsai_variant_applies(const pfe_ctx *c, int v) {
    if (v == PFE_FSAI_SLOTS) return true;
    return v == PFE_FSAI_STENCIL && c->mixed && c->nseg == 1 && c->kind == PFE_GRAPH_GRID && c->W > 0 &&
           (c->g.row_len == 12 || c->g.row_len == 28);
}

// The edge-pass column forms that apply: slot arrays always; the stencil on
// one FP32 grid image of 12 slots a row.
static bool edge_variant_applies(const pfe_ctx *c, int v) {
    if (v == PFE_EDGE_SLOTS) return true;
    return v == PFE_EDGE_STENCIL && c->mixed && c->nseg == 1 && c->kind == PFE_GRAPH_GRID && c->W > 0 &&
           c->g.row_len == 12;
}

// Average time of `reps` edge passes on the current state.  The passes write
// the spare b buffer (which the next edge pass rewrites) and, instead of the
// right-hand side of the next solve, the FP64 staging buffer (n x d, large
// enough for either precision), so the iteration state is left as it was.
static pfe_status time_edge(pfe_ctx *c, int reps, float *ms) {
    cudaEvent_t e0, e1;
    PFE_CUDA_TRY(c, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(c, PFE_ECUDA, "cudaEventCreate failed");
    }
    const int cur = c->bs_cur;
    void *rhs = c->wk.RHS;
    c->wk.RHS = c->wk.stage;
    pfe_status st = launch_edge(c, c->stream);
    c->bs_cur = cur;
    cudaEventRecord(e0, c->stream);
    for (int k = 0; k < reps && st == PFE_OK; ++k) {
        st = launch_edge(c, c->stream);
        c->bs_cur = cur;
    }
    c->wk.RHS = rhs;
    cudaEventRecord(e1, c->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PFE_OK) return st;
    if (e != cudaSuccess) return fail(c, PFE_ECUDA, cudaGetErrorString(e));
    *ms = t / (float)reps;
    return PFE_OK;
}

static void set_fsai_variant(pfe_ctx *c, int v) {
    c->fsai_variant = v;
    for (int slot : {G_FSAI_TR, G_FSAI_T, G_FSAI_T1, G_FSAI_ZP}) c->kgrid[slot] = 0;  // occupancy differs
    free_pcg_graph(c);
}

// The wave_grid slot of a tunable row kernel in the current configuration
// (-1: the kernel has no tunable shape here).
static int shape_slot(const pfe_ctx *c, int kernel) {
    switch (kernel) {
        case PFE_KERNEL_SPMM: {
            static const int sl[PFE_SPMM_NVARIANTS] = {G_SPMM,     G_SPMM_F1, G_SPMM_F2, G_SPMM_F3,
                                                       G_SPMM_TMA, -1,        G_SPMM_G1, G_SPMM_G2};
            return c->spmm_variant >= 0 && c->spmm_variant < PFE_SPMM_NVARIANTS ? sl[c->spmm_variant] : -1;
        }
        case PFE_KERNEL_UPDATE: return G_UPDATE;
        case PFE_KERNEL_PUPDATE: return G_PUPD;
        case PFE_KERNEL_FSAI_TR: return G_FSAI_TR;
        case PFE_KERNEL_FSAI_ZP: return G_FSAI_ZP;
        case PFE_KERNEL_EDGE: return c->edge_variant == PFE_EDGE_STENCIL ? G_EDGE_GRID : G_EDGE;
        default: return -1;
    }
}
// row of c->shape_ms for a tunable kernel
static int shape_row(int kernel) {
    switch (kernel) {
        case PFE_KERNEL_SPMM: return 0;
        case PFE_KERNEL_UPDATE: return 1;
        case PFE_KERNEL_PUPDATE: return 2;
        case PFE_KERNEL_FSAI_TR: return 3;
        case PFE_KERNEL_FSAI_ZP: return 4;
        case PFE_KERNEL_EDGE: return 5;
        default: return -1;
    }
}

// One launch of a tunable kernel on scratch state (time_pcg_kernel; the
// edge pass by time_edge): the folding and holding launches averaged for
// k_pupdate and k_fsai_zp.
static pfe_status time_shape(pfe_ctx *c, int kernel, int reps, float *ms) {
    float t = 0.f, u = 0.f;
    switch (kernel) {
        case PFE_KERNEL_SPMM: PFE_TRY(time_pcg_kernel(c, c->stream, 0, reps, &t)); break;
        case PFE_KERNEL_UPDATE: PFE_TRY(time_pcg_kernel(c, c->stream, 1, reps, &t)); break;
        case PFE_KERNEL_PUPDATE:
            PFE_TRY(time_pcg_kernel(c, c->stream, 2, reps, &t));
            PFE_TRY(time_pcg_kernel(c, c->stream, 6, reps, &u));
            t = 0.5f * (t + u);
            break;
        case PFE_KERNEL_FSAI_TR: PFE_TRY(time_pcg_kernel(c, c->stream, 3, reps, &t)); break;
        case PFE_KERNEL_FSAI_ZP:
            PFE_TRY(time_pcg_kernel(c, c->stream, 4, reps, &t));
            PFE_TRY(time_pcg_kernel(c, c->stream, 5, reps, &u));
            t = 0.5f * (t + u);
            break;
        case PFE_KERNEL_EDGE: PFE_TRY(time_edge(c, reps, &t)); break;
        default: return PFE_EINVAL;
    }
    *ms = t;
    return PFE_OK;
}

// Launch-shape tuning of one kernel: its occupancy (the default) and up to
// three fewer blocks per SM; a smaller count is kept only when >= 2 % faster.
static pfe_status tune_shape(pfe_ctx *c, int kernel, int reps) {
    const int slot = shape_slot(c, kernel), row = shape_row(kernel);
    if (slot < 0 || row < 0) return PFE_OK;
    for (int b = 0; b < 8; ++b) c->shape_ms[row][b] = -1.f;
    c->kbps[slot] = 0;
    c->kgrid[slot] = 0;
    float t0 = 0.f;
    PFE_TRY(time_shape(c, kernel, reps, &t0));
    const int g0 = c->kgrid[slot];  // the default grid (the kernel's occupancy, or the work if smaller)
    const int occ = std::min(8, std::max(1, (g0 + c->num_sms - 1) / c->num_sms));
    c->shape_ms[row][occ - 1] = t0;
    int best = 0;
    float tbest = t0;
    for (int b = occ - 1; b >= std::max(1, occ - 3); --b) {
        c->kbps[slot] = b;
        c->kgrid[slot] = 0;
        float t = 0.f;
        PFE_TRY(time_shape(c, kernel, reps, &t));
        c->shape_ms[row][b - 1] = t;
        if (t < 0.98f * t0 && t < tbest) {
            tbest = t;
            best = b;
        }
    }
    c->kbps[slot] = best;
    c->kgrid[slot] = 0;
    return PFE_OK;
}

pfe_status pfe_autotune(pfe_ctx *c, int32_t reps, int32_t *choice, double *ms) {
    if (!c || reps < 1) return PFE_EINVAL;
    if (!c->inited) return fail(c, PFE_ESTATE, "pfe_autotune before pfe_init");
    PFE_TRY(sync(c));
    int best = PFE_SPMM_GENERAL;
    float tbest = INFINITY;
    for (int v = 0; v < PFE_SPMM_NVARIANTS; ++v) {
        if (!spmm_variant_applies(c, v)) {
            if (ms) ms[v] = -1.0;
            continue;
        }
        float t = 0.f;
        PFE_TRY(time_pcg_kernel(c, c->stream, 0, reps, &t, v));
        if (ms) ms[v] = t;
        if (t < tbest) {
            tbest = t;
            best = v;
        }
    }
    c->spmm_variant = best;
    free_pcg_graph(c);  // the captured loop holds the previous variant
    if (choice) choice[0] = best;
    // the FSAI kernels' column form, when the FSAI factor is in use: the time
    // of one iteration's k_fsai_tr and k_fsai_zp (folding and holding launches)
    if (c->fsai.enabled && !c->fsai.ic && fsai_variant_applies(c, PFE_FSAI_STENCIL)) {
        float tv[2] = {0.f, 0.f};
        for (int v = 0; v < 2; ++v) {
            set_fsai_variant(c, v);
            for (int which : {3, 4, 5}) {
                float t = 0.f;
                PFE_TRY(time_pcg_kernel(c, c->stream, which, reps, &t));
                tv[v] += which == 3 ? t : 0.5f * t;
            }
        }
        set_fsai_variant(c, tv[1] < tv[0] ? PFE_FSAI_STENCIL : PFE_FSAI_SLOTS);
        c->fsai_tune_ms[0] = tv[0];
        c->fsai_tune_ms[1] = tv[1];
    }
    // the edge pass's column form
    if (edge_variant_applies(c, PFE_EDGE_STENCIL)) {
        for (int v = 0; v < 2; ++v) {
            c->edge_variant = v;
            PFE_TRY(time_edge(c, reps, &c->edge_tune_ms[v]));
        }
        c->edge_variant = c->edge_tune_ms[1] < c->edge_tune_ms[0] ? PFE_EDGE_STENCIL : PFE_EDGE_SLOTS;
    }
    // launch shapes of the kernels the configured iteration runs (single
    // problems: a batch keeps one block or more per segment at occupancy)
    if (c->nseg == 1) {
        const bool fsai = c->fsai.enabled && !c->fsai.ic;
        PFE_TRY(tune_shape(c, PFE_KERNEL_SPMM, reps));
        if (fsai) {
            PFE_TRY(tune_shape(c, PFE_KERNEL_FSAI_TR, reps));
            PFE_TRY(tune_shape(c, PFE_KERNEL_FSAI_ZP, reps));
        } else if (!c->fsai.enabled) {
            PFE_TRY(tune_shape(c, PFE_KERNEL_UPDATE, reps));
            PFE_TRY(tune_shape(c, PFE_KERNEL_PUPDATE, reps));
        }
        PFE_TRY(tune_shape(c, PFE_KERNEL_EDGE, reps));
        free_pcg_graph(c);  // the captured loop holds the grids
    }
    return PFE_OK;
}

pfe_status pfe_get_variant(pfe_ctx *c, int32_t kernel, int32_t *variant, double *ms) {
    if (!c || !variant) return PFE_EINVAL;
    if (kernel == PFE_TUNE_SPMM) {
        *variant = c->spmm_variant;
    } else if (kernel == PFE_TUNE_FSAI) {
        *variant = c->fsai_variant;
        if (ms) {
            ms[0] = c->fsai_tune_ms[0];
            ms[1] = c->fsai_tune_ms[1];
        }
    } else if (kernel == PFE_TUNE_MLP) {
        *variant = c->fsai.mlp_tc ? PFE_MLP_TCGEN05 : PFE_MLP_MMA_SYNC;
    } else if (kernel == PFE_TUNE_EDGE) {
        *variant = c->edge_variant;
        if (ms) {
            ms[0] = c->edge_tune_ms[0];
            ms[1] = c->edge_tune_ms[1];
        }
    } else {
        return PFE_EINVAL;
    }
    return PFE_OK;
}

pfe_status pfe_get_shape(pfe_ctx *c, int32_t kernel, int32_t *blocks_per_sm, double *ms) {
    if (!c || !blocks_per_sm) return PFE_EINVAL;
    const int row = shape_row(kernel);
    if (row < 0) return fail(c, PFE_EINVAL, "pfe_get_shape: not a tunable kernel");
    // the stencil-form SpMM sizes its own grid: the default, nothing timed
    const int slot = shape_slot(c, kernel);
    *blocks_per_sm = slot >= 0 ? c->kbps[slot] : 0;
    if (ms)
        for (int b = 0; b < 8; ++b) ms[b] = (slot >= 0 && c->shape_ms[row][b] > 0.f) ? c->shape_ms[row][b] : -1.0;
    return PFE_OK;
}

pfe_status pfe_set_shape(pfe_ctx *c, int32_t kernel, int32_t blocks_per_sm) {
    if (!c) return PFE_EINVAL;
    const int slot = shape_slot(c, kernel);
    if (shape_row(kernel) < 0 || blocks_per_sm < 0 || blocks_per_sm > 8)
        return fail(c, PFE_EINVAL, "pfe_set_shape: not a tunable kernel, or blocks per SM outside 0..8");
    if (slot < 0) return fail(c, PFE_EUNSUPPORTED, "pfe_set_shape: the stencil-form SpMM sizes its own grid");
    PFE_TRY(sync(c));
    c->kbps[slot] = blocks_per_sm;
    c->kgrid[slot] = 0;
    free_pcg_graph(c);
    return PFE_OK;
}

pfe_status pfe_set_variant(pfe_ctx *c, int32_t kernel, int32_t variant) {
    if (!c) return PFE_EINVAL;
    if (kernel == PFE_TUNE_MLP) {
        if (variant != PFE_MLP_MMA_SYNC && variant != PFE_MLP_TCGEN05) return PFE_EINVAL;
        PFE_TRY(sync(c));
        c->fsai.mlp_tc = variant == PFE_MLP_TCGEN05;
        return PFE_OK;
    }
    if (kernel == PFE_TUNE_EDGE) {
        if (variant < 0 || variant > PFE_EDGE_STENCIL) return PFE_EINVAL;
        if (!edge_variant_applies(c, variant))
            return fail(c, PFE_EUNSUPPORTED, "edge-pass column form does not apply here");
        PFE_TRY(sync(c));
        c->edge_variant = variant;
        return PFE_OK;
    }
    if (kernel == PFE_TUNE_FSAI) {
        if (variant < 0 || variant > PFE_FSAI_STENCIL) return PFE_EINVAL;
        if (!fsai_variant_applies(c, variant))
            return fail(c, PFE_EUNSUPPORTED, "FSAI column form does not apply here");
        PFE_TRY(sync(c));
        set_fsai_variant(c, variant);
        return PFE_OK;
    }
    if (kernel != PFE_TUNE_SPMM || variant < 0 || variant >= PFE_SPMM_NVARIANTS) return PFE_EINVAL;
    if (!spmm_variant_applies(c, variant)) return fail(c, PFE_EUNSUPPORTED, "SpMM variant does not apply here");
    PFE_TRY(sync(c));
    c->spmm_variant = variant;
    free_pcg_graph(c);
    return PFE_OK;
}

pfe_status pfe_kmeans(pfe_ctx *c, const double *X, int32_t d, int32_t k, const double *C0, int32_t max_iter,
                      int32_t *labels, double *centroids, double *inertia, int32_t *rounds) {
    if (!c) return PFE_EINVAL;
    if (!X && !c->inited) return fail(c, PFE_ESTATE, "pfe_kmeans of the embedding before pfe_init");
    if (d < 1 || d > 32 || k < 1 || k > 64 || k > c->n || max_iter < 1)
        return fail(c, PFE_EINVAL, "pfe_kmeans: needs 1 <= d <= 32, 1 <= k <= min(64, n), max_iter >= 1");
    if (c->nseg > 1) return fail(c, PFE_EUNSUPPORTED, "k-means of a batch: cluster each problem separately");
    PFE_TRY(sync(c));
    const double *dX = X;
    double *tmp = nullptr;
    if (!X) {
        if (d != c->d) return fail(c, PFE_EINVAL, "d differs from the embedding dimension");
        PFE_TRY(launch_yhat(c, c->stream, c->wk.stage));
        dX = c->wk.stage;
    } else if (!is_device_ptr(X)) {
        const size_t bytes = sizeof(double) * (size_t)c->n * d;
        if (cudaMalloc((void **)&tmp, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, PFE_ENOMEM, "pfe_kmeans: device allocation failed");
        }
        cudaError_t e = cudaMemcpyAsync(tmp, X, bytes, cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) {
            cudaFree(tmp);
            return fail(c, PFE_ECUDA, cudaGetErrorString(e));
        }
        dX = tmp;
    }
    const pfe_status st = kmeans_run(c, dX, d, k, C0, max_iter, labels, centroids, inertia, rounds);
    if (tmp) cudaFree(tmp);
    return st;
}

pfe_status pfe_objective(pfe_ctx *c, int32_t which, double *l1, double *ortho_err) {
    if (!c || (which != PFE_OBJ_Y && which != PFE_OBJ_YHAT)) return PFE_EINVAL;
    if (!c->inited) return fail(c, PFE_ESTATE, "pfe_objective before pfe_init");
    PFE_TRY(sync(c));
    return diag_objective(c, which, l1, ortho_err);
}

pfe_status pfe_residual(pfe_ctx *c, const double *B, const double *X, double *relres) {
    if (!c || !B || !X || !relres) return PFE_EINVAL;
    if (!c->inited) return fail(c, PFE_ESTATE, "pfe_residual before pfe_init");
    PFE_TRY(sync(c));
    const size_t bytes = (size_t)c->g.n * c->d * sizeof(double);
    const bool hb = !is_device_ptr(B), hx = !is_device_ptr(X);
    double *tmp = nullptr;
    if (hb || hx) {
        if (cudaMalloc((void **)&tmp, (hb + hx) * bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, PFE_ENOMEM, "pfe_residual: device allocation failed");
        }
    }
    const double *Bd = B, *Xd = X;
    cudaError_t e = cudaSuccess;
    if (hb) {
        e = cudaMemcpyAsync(tmp, B, bytes, cudaMemcpyHostToDevice, c->stream);
        Bd = tmp;
    }
    if (hx && e == cudaSuccess) {
        e = cudaMemcpyAsync(tmp + (hb ? c->g.n * c->d : 0), X, bytes, cudaMemcpyHostToDevice, c->stream);
        Xd = tmp + (hb ? c->g.n * c->d : 0);
    }
    pfe_status st = PFE_OK;
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->err = std::string("pfe_residual: ") + cudaGetErrorString(e);
        st = PFE_ECUDA;
    } else {
        st = diag_residual(c, Bd, Xd, relres);
    }
    if (tmp) {
        cudaStreamSynchronize(c->stream);
        cudaFree(tmp);
    }
    return st;
}

pfe_status pfe_laplacian_eigenmap(pfe_ctx *c, int32_t d, double *V, int32_t max_iter, double tol, int32_t *iters,
                                  double *residual) {
    if (!c || !V || d < 1 || max_iter < 0 || !(tol >= 0.0)) return PFE_EINVAL;
    if (c->nseg > 1) return fail(c, PFE_EUNSUPPORTED, "no batched eigenmap: one problem per context");
    if (le_block(d) == 0) return fail(c, PFE_EUNSUPPORTED, "d too large for the eigenmap");
    if (c->n <= le_block(d)) return fail(c, PFE_EINVAL, "too few vertices for the eigenmap");
    PFE_TRY(sync(c));
    double *dv = nullptr;
    const size_t bytes = sizeof(double) * (size_t)c->n * d;
    const bool dev = is_device_ptr(V);
    if (!dev && cudaMalloc((void **)&dv, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, PFE_ENOMEM, "pfe_laplacian_eigenmap: device allocation failed");
    }
    int its = 0;
    double res = 0.0;
    pfe_status st = launch_le(c, d, dev ? V : dv, max_iter, tol, kLeDegree, &its, &res);
    if (!dev) {
        if (st == PFE_OK || st == PFE_ENOTCONV) {
            cudaError_t e = cudaMemcpy(V, dv, bytes, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) st = fail(c, PFE_ECUDA, cudaGetErrorString(e));
        }
        cudaFree(dv);
    }
    if (iters) *iters = its;
    if (residual) *residual = res;
    return st;
}

pfe_status pfe_get_segments(const pfe_ctx *c, int64_t *off, double *lambda) {
    if (!c) return PFE_EINVAL;
    if (off)
        for (int q = 0; q <= c->nseg; ++q) off[q] = c->h_seg_off[q];
    if (lambda)
        for (int q = 0; q < c->nseg; ++q) lambda[q] = c->h_seg_lam[q];
    return PFE_OK;
}

pfe_status pfe_get_segment_stats(pfe_ctx *c, int32_t *iters, double *relres, int64_t *iters_total) {
    if (!c) return PFE_EINVAL;
    if (!c->inited) return fail(c, PFE_ESTATE, "pfe_get_segment_stats before pfe_init");
    PFE_TRY(sync(c));
    if (iters)
        PFE_CUDA_TRY(c, cudaMemcpy(iters, c->sc.seg_iters, sizeof(int) * c->nseg, cudaMemcpyDeviceToHost));
    if (relres)
        PFE_CUDA_TRY(c, cudaMemcpy(relres, c->sc.relres, sizeof(double) * c->nseg * c->d, cudaMemcpyDeviceToHost));
    if (iters_total)
        PFE_CUDA_TRY(c, cudaMemcpy(iters_total, c->sc.seg_iters_tot, sizeof(long long) * c->nseg,
                                   cudaMemcpyDeviceToHost));
    return PFE_OK;
}

static pfe_status init_impl(pfe_ctx *c, int32_t d, const double *Y0, int64_t ldY0) {
    if (d < 1 || d > c->n) return fail(c, PFE_EINVAL, "d must be in [1, n]");
    if (Y0 && ldY0 < d) return fail(c, PFE_EINVAL, "ldY0 < d");
    if (!d_supported(d)) return fail(c, PFE_EUNSUPPORTED, "embedding dimension not built into libpfe");
    const bool le_start = Y0 == nullptr;  // Laplacian-eigenmap start
    if (le_start) {
        if (c->nseg > 1) return fail(c, PFE_EUNSUPPORTED, "a batch takes its start in Y0 (no batched eigenmap)");
        if (le_block(d) == 0) return fail(c, PFE_EUNSUPPORTED, "d too large for the eigenmap start");
        if (c->n <= le_block(d)) return fail(c, PFE_EINVAL, "too few vertices for the eigenmap start");
    }
    free_work(c);
    c->d = d;
    memset(c->kgrid, 0, sizeof(c->kgrid));  // kernels are sized again for this d
    memset(c->kbps, 0, sizeof(c->kbps));    // with their default shapes
    for (auto &r : c->shape_ms)
        for (float &t : r) t = -1.f;
    const int64_t nd = c->n * (int64_t)d;
    const int64_t ed = c->g.fslots * (int64_t)d;
    auto &w = c->wk;
    if (c->mixed) {
        float *y, *bs0, *bs1, *rhs, *cw, *r, *pd, *pd2, *q;
        PFE_TRY(walloc(c, &y, nd));
        PFE_TRY(walloc(c, &w.Ylo, nd));
        PFE_TRY(walloc(c, &bs0, ed));
        PFE_TRY(walloc(c, &bs1, ed));
        PFE_TRY(walloc(c, &rhs, nd));
        PFE_TRY(walloc(c, &cw, nd));
        PFE_TRY(walloc(c, &r, nd));
        PFE_TRY(walloc(c, &pd, nd));
        PFE_TRY(walloc(c, &pd2, nd));
        PFE_TRY(walloc(c, &q, nd));
        w.Y = y; w.Bs[0] = bs0; w.Bs[1] = bs1; w.RHS = rhs; w.Cw = cw; w.R = r; w.Pd = pd; w.Pd2 = pd2; w.Q = q;
    } else {
        double *y, *bs0, *bs1, *rhs, *cw, *r, *pd, *pd2, *q;
        PFE_TRY(walloc(c, &y, nd));
        PFE_TRY(walloc(c, &bs0, ed));
        PFE_TRY(walloc(c, &bs1, ed));
        PFE_TRY(walloc(c, &rhs, nd));
        PFE_TRY(walloc(c, &cw, nd));
        PFE_TRY(walloc(c, &r, nd));
        PFE_TRY(walloc(c, &pd, nd));
        PFE_TRY(walloc(c, &pd2, nd));
        PFE_TRY(walloc(c, &q, nd));
        w.Y = y; w.Bs[0] = bs0; w.Bs[1] = bs1; w.RHS = rhs; w.Cw = cw; w.R = r; w.Pd = pd; w.Pd2 = pd2; w.Q = q;
    }
    if (c->fsai.enabled) PFE_TRY(fsai_vectors(c, nd));
    PFE_TRY(walloc(c, &w.P, nd));
    PFE_TRY(walloc(c, &w.B, nd));
    PFE_TRY(walloc(c, &w.stage, nd));
    // <= 8 resident blocks of 256 threads, and at least one block per segment
    const int64_t part_pcg = std::max<int64_t>((int64_t)c->num_sms * 8, c->nseg) * 3 * PFE_DMAX;
    const int64_t part_gram = std::max<int64_t>((int64_t)c->num_sms * 2, c->nseg) * (PFE_DMAX * (PFE_DMAX + 1) / 2);
    w.partials_len = std::max(part_pcg, part_gram);
    PFE_TRY(walloc(c, &w.partials, w.partials_len));
    {
        unsigned char *scb;
        PFE_TRY(walloc(c, &scb, (int64_t)segscal_bytes(c->nseg, d)));
        c->sc = segscal_carve(scb, c->nseg, d);
        PFE_CUDA_TRY(c, cudaMemsetAsync(scb, 0, segscal_bytes(c->nseg, d), c->stream));
        PFE_TRY(walloc(c, &c->seg_T, (int64_t)c->nseg * d * d));
        PFE_TRY(walloc(c, &c->seg_pticket, c->nseg));
        PFE_CUDA_TRY(c, cudaMemsetAsync(c->seg_pticket, 0, sizeof(unsigned) * c->nseg, c->stream));
    }
    const size_t es = elem_size(c);
    PFE_CUDA_TRY(c, cudaMemsetAsync(w.Bs[0], 0, (size_t)ed * es, c->stream));
    PFE_CUDA_TRY(c, cudaMemsetAsync(w.Bs[1], 0, (size_t)ed * es, c->stream));
    PFE_CUDA_TRY(c, cudaMemsetAsync(w.Pd, 0, (size_t)nd * es, c->stream));
    PFE_CUDA_TRY(c, cudaMemsetAsync(w.Pd2, 0, (size_t)nd * es, c->stream));
    PFE_CUDA_TRY(c, cudaMemsetAsync(w.Q, 0, (size_t)nd * es, c->stream));
    PFE_CUDA_TRY(c, cudaMemsetAsync(w.R, 0, (size_t)nd * es, c->stream));
    c->bs_cur = 0;
    // control block parameters
    PcgCtl h;
    memset(&h, 0, sizeof(h));
    h.max_iter = c->prm.max_iter;
    h.refresh = c->prm.refresh;
    h.ncols = d;
    h.tol = c->prm.tol;
    h.done = 1;
    h.unroll = std::max(1, c->prm.check_every);
    int lc[3];
    launch_counts(c, lc);
    h.launch_base = lc[0];
    h.launch_per_iter = lc[1];
    h.launch_cond = lc[2];
    PFE_CUDA_TRY(c, cudaMemcpyAsync(c->ctl, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
    PFE_CUDA_TRY(c, cudaMemsetAsync(c->pctl, 0, sizeof(PstepCtl), c->stream));
    // Y0 (or the eigenmap) -> stage (contiguous FP64), then D-orthonormalise
    // via the P-step map
    if (le_start) {
        int its = 0;
        double res = 0.0;
        const pfe_status ls = launch_le(c, d, w.stage, kLeMaxIter, kLeTol, kLeDegree, &its, &res);
        c->le_iters = its;
        c->le_residual = res;
        // an eigenmap short of the tolerance is still a valid start
        if (ls != PFE_OK && ls != PFE_ENOTCONV) return ls;
    } else {
        PFE_CUDA_TRY(c, cudaMemcpy2DAsync(w.stage, sizeof(double) * d, Y0, sizeof(double) * ldY0,
                                          sizeof(double) * d, (size_t)c->n, cudaMemcpyDefault, c->stream));
    }
    PFE_TRY(launch_pstep(c, c->stream, PSTEP_INIT));
    PFE_TRY(sync(c));
    PFE_TRY(check_pstep(c));
    c->inited = true;
    return PFE_OK;
}

pfe_status pfe_init(pfe_ctx *c, int32_t d, const double *Y0, int64_t ldY0) {
    if (!c) return PFE_EINVAL;
    NvtxRange r("pfe init");
    const pfe_status st = init_impl(c, d, Y0, ldY0);
    // a failure after the previous state was released leaves no work buffers
    // behind (one rejected by the argument checks keeps that state)
    if (st != PFE_OK && !c->inited) {
        const std::string msg = c->err;
        free_work(c);
        c->err = msg;
    }
    return st;
}

pfe_status pfe_inner_step(pfe_ctx *c, pfe_step_stats *st) {
    if (!c) return PFE_EINVAL;
    if (!c->inited) return fail(c, PFE_ESTATE, "pfe_inner_step before pfe_init");
    PFE_TRY(inner_step_enqueue(c));
    if (st) {
        PFE_TRY(read_ctl(c));
        st->pcg_iters = c->h_ctl->last_iters;
        st->converged = c->h_ctl->last_converged;
        st->relres_max = c->h_ctl->last_relres;
        if (c->h_ctl->error) return pcg_error(c);
        if (!st->converged) return fail(c, PFE_ENOTCONV, "PCG: max_iter reached before tol");
    }
    return PFE_OK;
}

pfe_status pfe_pstep(pfe_ctx *c) {
    if (!c) return PFE_EINVAL;
    if (!c->inited) return fail(c, PFE_ESTATE, "pfe_pstep before pfe_init");
    return pstep_enqueue(c);
}

// Stage I (n_outer SOC iterations of n_inner split-Bregman iterations), then
// Stage II (n_stage2 split-Bregman iterations with P and B held).
static pfe_status solve_stages(pfe_ctx *c, int32_t n_outer, int32_t n_inner, int32_t n_stage2, double *Y_out,
                               double *Yhat_out, pfe_solve_stats *st) {
    if (!c->inited) return fail(c, PFE_ESTATE, "pfe_solve before pfe_init");
    if (n_outer < 0 || n_inner < 0 || n_stage2 < 0) return fail(c, PFE_EINVAL, "negative iteration count");
    NvtxRange r("pfe solve");
    PFE_TRY(clear_stats(c));
    for (int k = 0; k < n_outer; ++k) {
        for (int l = 0; l < n_inner; ++l) PFE_TRY(inner_step_enqueue(c));
        PFE_TRY(pstep_enqueue(c));
    }
    // Stage II is one more call of Alg. 2: b starts at zero (a P-step with
    // reset_inner_each_outer already cleared it)
    if (n_stage2 > 0 && n_outer == 0 && c->prm.reset_inner_each_outer) {
        const size_t bytes = (size_t)c->g.fslots * c->d * elem_size(c);
        PFE_CUDA_TRY(c, cudaMemsetAsync(c->wk.Bs[c->bs_cur], 0, bytes, c->stream));
    }
    for (int l = 0; l < n_stage2; ++l) PFE_TRY(inner_step_enqueue(c));
    const size_t bytes = sizeof(double) * (size_t)c->n * c->d;
    if (Y_out) {
        PFE_TRY(launch_from_work(c, c->stream, c->wk.Y, c->wk.Ylo, c->wk.stage, c->n));
        PFE_CUDA_TRY(c, cudaMemcpyAsync(Y_out, c->wk.stage, bytes, cudaMemcpyDefault, c->stream));
    }
    if (Yhat_out) {
        if (is_device_ptr(Yhat_out)) {
            PFE_TRY(launch_yhat(c, c->stream, Yhat_out));
        } else {
            PFE_TRY(sync(c));  // stage is reused
            PFE_TRY(launch_yhat(c, c->stream, c->wk.stage));
            PFE_CUDA_TRY(c, cudaMemcpyAsync(Yhat_out, c->wk.stage, bytes, cudaMemcpyDefault, c->stream));
        }
    }
    PFE_TRY(read_ctl(c));
    if (st) {
        st->pcg_iters_total = c->h_ctl->tot_iters;
        st->pcg_rounds = c->h_ctl->tot_rounds;
        st->replacements = c->h_ctl->tot_refreshes;
        st->pcg_iters_max = c->h_ctl->max_solve_iters;
        st->n_solves = c->h_ctl->n_solves;
        st->n_unconverged = c->h_ctl->n_unconv;
        st->relres_max = c->h_ctl->max_relres;
        // PCG launches + one edge pass per inner step + Gram and apply per outer step
        st->kernel_launches = c->h_ctl->launches + (int64_t)n_outer * n_inner + n_stage2 + 2LL * n_outer;
    }
    PFE_TRY(check_pstep(c));
    return pcg_status(c);
}

pfe_status pfe_solve(pfe_ctx *c, int32_t n_outer, int32_t n_inner, double *Y_out, double *Yhat_out,
                     pfe_solve_stats *st) {
    if (!c) return PFE_EINVAL;
    return solve_stages(c, n_outer, n_inner, 0, Y_out, Yhat_out, st);
}

pfe_status pfe_solve_two_stage(pfe_ctx *c, int32_t n_outer, int32_t n_inner, int32_t n_stage2, double *Y_out,
                               double *Yhat_out, pfe_solve_stats *st) {
    if (!c) return PFE_EINVAL;
    return solve_stages(c, n_outer, n_inner, n_stage2, Y_out, Yhat_out, st);
}

pfe_status pfe_get_array(pfe_ctx *c, int32_t which, double *dst) {
    if (!c || !dst) return PFE_EINVAL;
    const int64_t n = c->n;
    if (which == PFE_ARR_DEG || which == PFE_ARR_DIAG) {
        const double *src = which == PFE_ARR_DEG ? c->g.deg : c->g.adiag64;
        PFE_CUDA_TRY(c, cudaMemcpyAsync(dst, src, sizeof(double) * n, cudaMemcpyDefault, c->stream));
        return sync(c);
    }
    if (!c->inited) return fail(c, PFE_ESTATE, "state arrays exist after pfe_init");
    const size_t bytes = sizeof(double) * (size_t)n * c->d;
    switch (which) {
        case PFE_ARR_Y:
            PFE_TRY(launch_from_work(c, c->stream, c->wk.Y, c->wk.Ylo, c->wk.stage, n));
            PFE_CUDA_TRY(c, cudaMemcpyAsync(dst, c->wk.stage, bytes, cudaMemcpyDefault, c->stream));
            break;
        case PFE_ARR_RHS:
            PFE_TRY(launch_from_work(c, c->stream, c->wk.RHS, nullptr, c->wk.stage, n));
            PFE_CUDA_TRY(c, cudaMemcpyAsync(dst, c->wk.stage, bytes, cudaMemcpyDefault, c->stream));
            break;
        case PFE_ARR_P:
            PFE_CUDA_TRY(c, cudaMemcpyAsync(dst, c->wk.P, bytes, cudaMemcpyDefault, c->stream));
            break;
        case PFE_ARR_B:
            PFE_CUDA_TRY(c, cudaMemcpyAsync(dst, c->wk.B, bytes, cudaMemcpyDefault, c->stream));
            break;
        case PFE_ARR_BS: {
            const size_t eb = sizeof(double) * (size_t)c->g.n_edges * c->d;
            double *tmp = nullptr;
            if (cudaMalloc((void **)&tmp, std::max<size_t>(eb, 8)) != cudaSuccess) {
                cudaGetLastError();
                return fail(c, PFE_ENOMEM, "staging buffer for b");
            }
            pfe_status s1 = launch_bs_gather(c, c->stream, c->wk.Bs[c->bs_cur], tmp, true);
            cudaError_t e1 = cudaMemcpyAsync(dst, tmp, eb, cudaMemcpyDefault, c->stream);
            cudaError_t e2 = cudaStreamSynchronize(c->stream);
            cudaFree(tmp);
            if (s1 != PFE_OK) return s1;
            if (e1 != cudaSuccess || e2 != cudaSuccess) return fail(c, PFE_ECUDA, "copy of b failed");
            break;
        }
        default:
            return fail(c, PFE_EINVAL, "unknown array id");
    }
    return sync(c);
}

pfe_status pfe_set_array(pfe_ctx *c, int32_t which, const double *src) {
    if (!c || !src) return PFE_EINVAL;
    if (!c->inited) return fail(c, PFE_ESTATE, "state arrays exist after pfe_init");
    const int64_t n = c->n;
    const size_t bytes = sizeof(double) * (size_t)n * c->d;
    switch (which) {
        case PFE_ARR_Y:
            PFE_CUDA_TRY(c, cudaMemcpyAsync(c->wk.stage, src, bytes, cudaMemcpyDefault, c->stream));
            PFE_TRY(launch_to_work(c, c->stream, c->wk.stage, c->wk.Y, c->wk.Ylo, n));
            break;
        case PFE_ARR_RHS:
            PFE_CUDA_TRY(c, cudaMemcpyAsync(c->wk.stage, src, bytes, cudaMemcpyDefault, c->stream));
            PFE_TRY(launch_to_work(c, c->stream, c->wk.stage, c->wk.RHS, nullptr, n));
            break;
        case PFE_ARR_P:
            PFE_CUDA_TRY(c, cudaMemcpyAsync(c->wk.P, src, bytes, cudaMemcpyDefault, c->stream));
            PFE_TRY(launch_cw(c, c->stream));
            break;
        case PFE_ARR_B:
            PFE_CUDA_TRY(c, cudaMemcpyAsync(c->wk.B, src, bytes, cudaMemcpyDefault, c->stream));
            PFE_TRY(launch_cw(c, c->stream));
            break;
        case PFE_ARR_BS: {
            const size_t eb = sizeof(double) * (size_t)c->g.n_edges * c->d;
            double *tmp = nullptr;
            if (cudaMalloc((void **)&tmp, std::max<size_t>(eb, 8)) != cudaSuccess) {
                cudaGetLastError();
                return fail(c, PFE_ENOMEM, "staging buffer for b");
            }
            cudaError_t e1 = cudaMemcpyAsync(tmp, src, eb, cudaMemcpyDefault, c->stream);
            pfe_status s1 = launch_bs_scatter(c, c->stream, tmp, c->wk.Bs[c->bs_cur]);
            cudaError_t e2 = cudaStreamSynchronize(c->stream);
            cudaFree(tmp);
            if (s1 != PFE_OK) return s1;
            if (e1 != cudaSuccess || e2 != cudaSuccess) return fail(c, PFE_ECUDA, "copy of b failed");
            break;
        }
        default:
            return fail(c, PFE_EINVAL, "array id cannot be set");
    }
    return sync(c);
}

pfe_status pfe_get_edges(pfe_ctx *c, int32_t *a, int32_t *b, double *w) {
    if (!c) return PFE_EINVAL;
    const int64_t ne = c->g.n_edges;
    if (a) PFE_CUDA_TRY(c, cudaMemcpyAsync(a, c->g.ea, sizeof(int32_t) * ne, cudaMemcpyDefault, c->stream));
    if (b) PFE_CUDA_TRY(c, cudaMemcpyAsync(b, c->g.eb, sizeof(int32_t) * ne, cudaMemcpyDefault, c->stream));
    if (w) PFE_CUDA_TRY(c, cudaMemcpyAsync(w, c->g.ew, sizeof(double) * ne, cudaMemcpyDefault, c->stream));
    return sync(c);
}

pfe_status pfe_apply_A(pfe_ctx *c, const double *X, double *Yout) {
    if (!c || !X || !Yout) return PFE_EINVAL;
    if (!c->inited) return fail(c, PFE_ESTATE, "pfe_apply_A before pfe_init fixes d");
    const int64_t n = c->n;
    const size_t bytes = sizeof(double) * (size_t)n * c->d;
    PFE_CUDA_TRY(c, cudaMemcpyAsync(c->wk.stage, X, bytes, cudaMemcpyDefault, c->stream));
    PFE_TRY(launch_to_work(c, c->stream, c->wk.stage, c->wk.R, nullptr, n));
    PFE_TRY(launch_apply_A(c, c->stream, c->wk.R, c->wk.Q));
    PFE_TRY(launch_from_work(c, c->stream, c->wk.Q, nullptr, c->wk.stage, n));
    PFE_CUDA_TRY(c, cudaMemcpyAsync(Yout, c->wk.stage, bytes, cudaMemcpyDefault, c->stream));
    return sync(c);
}

pfe_status pfe_solve_system(pfe_ctx *c, const double *RHS, double *Y, pfe_step_stats *st) {
    if (!c || !RHS || !Y) return PFE_EINVAL;
    if (!c->inited) return fail(c, PFE_ESTATE, "pfe_solve_system before pfe_init fixes d");
    const int64_t n = c->n;
    const int64_t nd = n * (int64_t)c->d;
    const size_t bytes = sizeof(double) * (size_t)nd;
    const size_t es = elem_size(c);
    // private solution / right-hand side buffers; the iteration state is untouched
    void *y = nullptr, *b = nullptr;
    float *ylo = nullptr;
    struct F {
        void *p[3];
        ~F() {
            for (void *q : p)
                if (q) cudaFree(q);
        }
    } fr{{nullptr, nullptr, nullptr}};
    if (cudaMalloc(&y, nd * es) != cudaSuccess || (fr.p[0] = y, false) || cudaMalloc(&b, nd * es) != cudaSuccess ||
        (fr.p[1] = b, false) || (c->mixed && cudaMalloc((void **)&ylo, nd * sizeof(float)) != cudaSuccess)) {
        cudaGetLastError();
        return fail(c, PFE_ENOMEM, "pfe_solve_system buffers");
    }
    fr.p[2] = ylo;
    PFE_CUDA_TRY(c, cudaMemcpyAsync(c->wk.stage, RHS, bytes, cudaMemcpyDefault, c->stream));
    PFE_TRY(launch_to_work(c, c->stream, c->wk.stage, b, nullptr, n));
    PFE_CUDA_TRY(c, cudaMemcpyAsync(c->wk.stage, Y, bytes, cudaMemcpyDefault, c->stream));
    PFE_TRY(launch_to_work(c, c->stream, c->wk.stage, y, ylo, n));
    Work saved = c->wk;
    c->wk.Y = y;
    c->wk.Ylo = ylo;
    c->wk.RHS = b;
    pfe_status s = run_pcg(c, true);
    c->wk = saved;
    PFE_TRY(s);
    PFE_TRY(launch_from_work(c, c->stream, y, ylo, c->wk.stage, n));
    PFE_CUDA_TRY(c, cudaMemcpyAsync(Y, c->wk.stage, bytes, cudaMemcpyDefault, c->stream));
    PFE_TRY(read_ctl(c));
    if (st) {
        st->pcg_iters = c->h_ctl->last_iters;
        st->converged = c->h_ctl->last_converged;
        st->relres_max = c->h_ctl->last_relres;
    }
    if (c->h_ctl->error) return pcg_error(c);
    if (!c->h_ctl->last_converged) return fail(c, PFE_ENOTCONV, "PCG: max_iter reached before tol");
    return PFE_OK;
}

pfe_status pfe_time_kernel(pfe_ctx *c, int32_t which, int32_t reps, double *avg_ms) {
    if (!c || !avg_ms || reps < 1) return PFE_EINVAL;
    if (!c->inited) return fail(c, PFE_ESTATE, "pfe_time_kernel before pfe_init");
    PFE_TRY(sync(c));
    float ms = 0.f;
    if (which == PFE_KERNEL_EDGE) {
        PFE_TRY(time_edge(c, reps, &ms));
    } else if (which == PFE_KERNEL_MLP) {
        if (!c->fsai.enabled || c->fsai.ic || !c->fsai.params)
            return fail(c, PFE_EUNSUPPORTED, "pfe_time_kernel: the network needs a learned FSAI factor (pfe_fsai_set)");
        PFE_TRY(fsai_time_infer(c, reps, &ms));
    } else if (which == PFE_KERNEL_SPMM || which == PFE_KERNEL_UPDATE || which == PFE_KERNEL_PUPDATE ||
               which == PFE_KERNEL_FSAI_TR || which == PFE_KERNEL_FSAI_ZP || which == PFE_KERNEL_FSAI_ZP_HOLD ||
               which == PFE_KERNEL_PUPDATE_HOLD || which == PFE_KERNEL_REPLACE || which == PFE_KERNEL_XFLUSH ||
               which == PFE_KERNEL_FSAI_T) {
        if (which == PFE_KERNEL_FSAI_T && (!c->fsai.enabled || c->fsai.ic))
            return fail(c, PFE_EUNSUPPORTED, "pfe_time_kernel: k_fsai_t needs an FSAI factor");
        const int k = which == PFE_KERNEL_PUPDATE        ? 2
                      : which == PFE_KERNEL_FSAI_TR      ? 3
                      : which == PFE_KERNEL_FSAI_ZP      ? 4
                      : which == PFE_KERNEL_FSAI_ZP_HOLD ? 5
                      : which == PFE_KERNEL_PUPDATE_HOLD ? 6
                      : which == PFE_KERNEL_REPLACE      ? 7
                      : which == PFE_KERNEL_XFLUSH       ? 8
                      : which == PFE_KERNEL_FSAI_T       ? 9
                                                         : which;
        PFE_TRY(time_pcg_kernel(c, c->stream, k, reps, &ms));
    } else {
        return fail(c, PFE_EINVAL, "unknown kernel id");
    }
    *avg_ms = ms;
    return PFE_OK;
}

int32_t pfe_fsai_param_count(void) { return kNParam; }

pfe_status pfe_fsai_set(pfe_ctx *c, const float *params) {
    if (!c) return PFE_EINVAL;
    NvtxRange r("pfe learned FSAI set-up");
    PFE_TRY(sync(c));
    if (!params) {
        c->fsai.enabled = false;
    } else {
        if (!c->mixed) return fail(c, PFE_EUNSUPPORTED, "the FSAI preconditioner runs on the mixed-precision path");
        PFE_TRY(fsai_alloc(c));
        PFE_CUDA_TRY(c, cudaMemcpyAsync(c->fsai.params, params, kNParam * sizeof(float), cudaMemcpyDefault,
                                        c->stream));
        PFE_TRY(fsai_infer(c));
        if (c->inited && !c->fsai.t) PFE_TRY(fsai_vectors(c, c->n * (int64_t)c->d));
        c->fsai.enabled = true;
    }
    c->fsai.ic = false;
    return fsai_switched(c);
}

pfe_status pfe_fsai_classical(pfe_ctx *c) {
    if (!c) return PFE_EINVAL;
    NvtxRange r("pfe classical FSAI set-up");
    if (!c->mixed) return fail(c, PFE_EUNSUPPORTED, "the FSAI preconditioner runs on the mixed-precision path");
    PFE_TRY(sync(c));
    PFE_TRY(fsai_alloc(c));
    PFE_TRY(fsai_classical(c));
    if (c->inited && !c->fsai.t) PFE_TRY(fsai_vectors(c, c->n * (int64_t)c->d));
    c->fsai.enabled = true;
    c->fsai.ic = false;
    return fsai_switched(c);
}

pfe_status pfe_ic0(pfe_ctx *c) {
    if (!c) return PFE_EINVAL;
    NvtxRange r("pfe IC(0) set-up");
    if (c->nseg > 1 || c->kind != PFE_GRAPH_GRID || c->W < 1 || (c->g.row_len != 12 && c->g.row_len != 28))
        return fail(c, PFE_EUNSUPPORTED, "IC(0) is built for one grid image of radius 2 or 3");
    if (!c->mixed) return fail(c, PFE_EUNSUPPORTED, "IC(0) runs on the mixed-precision path");
    PFE_TRY(sync(c));
    PFE_TRY(fsai_alloc(c));
    c->fsai.enabled = false;
    PFE_TRY(ic0_factor(c));
    if (c->inited && !c->fsai.t) PFE_TRY(fsai_vectors(c, c->n * (int64_t)c->d));
    c->fsai.enabled = true;
    c->fsai.ic = true;
    return fsai_switched(c);
}

pfe_status pfe_fsai_loss_grad(pfe_ctx *c, const float *params, float *grad, double *loss) {
    if (!c || !params || !loss) return PFE_EINVAL;
    if (c->nseg > 1) return fail(c, PFE_EUNSUPPORTED, "the training loss is built for one problem, not a batch");
    PFE_TRY(fsai_alloc(c));
    PFE_CUDA_TRY(c, cudaMemcpyAsync(c->fsai.params, params, kNParam * sizeof(float), cudaMemcpyDefault, c->stream));
    PFE_TRY(fsai_loss_grad(c, loss));
    if (grad)
        PFE_CUDA_TRY(c, cudaMemcpyAsync(grad, c->fsai.grad, kNParam * sizeof(float), cudaMemcpyDefault, c->stream));
    return sync(c);
}

pfe_status pfe_fsai_loss_grad_rhs(pfe_ctx *c, const float *params, const double *B, int32_t m, double mu,
                                  float *grad, double *loss, double *rterm) {
    if (!c || !params || !loss) return PFE_EINVAL;
    if (c->nseg > 1) return fail(c, PFE_EUNSUPPORTED, "the training loss is built for one problem, not a batch");
    const bool rhs = B && mu > 0.0;
    if (rhs && (m < 1 || m > 32)) return fail(c, PFE_EINVAL, "pfe_fsai_loss_grad_rhs: needs 1 <= m <= 32");
    if (!(mu >= 0.0)) return fail(c, PFE_EINVAL, "pfe_fsai_loss_grad_rhs: mu must be >= 0");
    PFE_TRY(fsai_alloc(c));
    PFE_CUDA_TRY(c, cudaMemcpyAsync(c->fsai.params, params, kNParam * sizeof(float), cudaMemcpyDefault, c->stream));
    const double *dB = B;
    double *tmp = nullptr;
    if (rhs && !is_device_ptr(B)) {
        const size_t bytes = sizeof(double) * (size_t)c->n * m;
        if (cudaMalloc((void **)&tmp, bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, PFE_ENOMEM, "pfe_fsai_loss_grad_rhs: device copy of B");
        }
        if (cudaMemcpyAsync(tmp, B, bytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
            cudaFree(tmp);
            return fail(c, PFE_ECUDA, "pfe_fsai_loss_grad_rhs: copy of B");
        }
        dB = tmp;
    }
    pfe_status st = fsai_loss_grad(c, loss, rhs ? dB : nullptr, rhs ? m : 0, rhs ? mu : 0.0, rterm);
    if (tmp) cudaFree(tmp);
    PFE_TRY(st);
    if (grad)
        PFE_CUDA_TRY(c, cudaMemcpyAsync(grad, c->fsai.grad, kNParam * sizeof(float), cudaMemcpyDefault, c->stream));
    return sync(c);
}

pfe_status pfe_fsai_get(pfe_ctx *c, double *gdiag, double *gedge) {
    if (!c) return PFE_EINVAL;
    if (!c->fsai.gdiag) return fail(c, PFE_ESTATE, "no FSAI factor: call pfe_fsai_set or pfe_fsai_loss_grad first");
    const int64_t n = c->g.n, ne = c->g.n_edges;
    double *tmp = nullptr;
    if (cudaMalloc((void **)&tmp, sizeof(double) * std::max<int64_t>(n + ne, 1)) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, PFE_ENOMEM, "staging buffer for G");
    }
    pfe_status st = fsai_export(c, tmp, tmp + n);
    if (st == PFE_OK && gdiag && cudaMemcpyAsync(gdiag, tmp, sizeof(double) * n, cudaMemcpyDefault, c->stream) != cudaSuccess)
        st = PFE_ECUDA;
    if (st == PFE_OK && gedge && ne > 0 &&
        cudaMemcpyAsync(gedge, tmp + n, sizeof(double) * ne, cudaMemcpyDefault, c->stream) != cudaSuccess)
        st = PFE_ECUDA;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    if (st != PFE_OK) return st;
    if (e != cudaSuccess) return fail(c, PFE_ECUDA, cudaGetErrorString(e));
    return PFE_OK;
}

pfe_status pfe_adam_update(float *params, const float *grad, float *m, float *v, int64_t count, int32_t step,
                           double lr, double beta1, double beta2, double eps, pfe_stream_t stream) {
    if (!params || !grad || !m || !v || count < 1 || step < 1) return PFE_EINVAL;
    if (!is_device_ptr(params) || !is_device_ptr(grad) || !is_device_ptr(m) || !is_device_ptr(v)) return PFE_EINVAL;
    return adam_step(params, grad, m, v, count, step, lr, beta1, beta2, eps, (cudaStream_t)stream);
}

}  // extern "C"
