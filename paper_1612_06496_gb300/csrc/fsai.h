// Learned FSAI preconditioner: buffers of a context and the host-side steps
// (csrc/fsai.cu).
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/pfe.h"

struct pfe_ctx;

namespace pfe {

constexpr int kNParam = 4 * 64 + 64 + 64 * 64 + 64 + 64 * 2 + 2;  // 4610 MLP parameters

struct FsaiState {
    bool enabled = false;      // PCG uses M^{-1} = G^T G instead of Jacobi
    int mlp_blocks = 0;
    float *gdiag = nullptr;    // G_ii
    float *gE = nullptr;       // G_ba per edge slot
    float *gslot = nullptr;    // G value per SELL slot (both orientations)
    float *srow = nullptr;     // diagonal-entry feature s_i
    int *kb = nullptr;         // number of lower (j < i) slots of each row
    int *ent_of_slot = nullptr;// edge slot -> external edge id
    float *hraw = nullptr;     // network head value per entry
    float *dq = nullptr;       // per-entry gradient scratch
    double *qrow = nullptr, *logd = nullptr, *sums = nullptr, *part = nullptr;
    float *gpart = nullptr;    // per-block parameter-gradient partials
    unsigned *tick = nullptr;
    float *params = nullptr;   // network parameters in use (device copy)
    float *grad = nullptr;     // last gradient
    bool mlp_tc = true;        // network inference on tcgen05 (TMEM accumulator); false: mma.sync
    bool ic = false;           // the factor is IC(0)'s L: M^{-1} = L^{-T} L^{-1} (triangular solves)
    int ic_cl = 0;             // IC level schedule: pixel (x, y) has level x + ic_cl y
    int64_t ic_levels = 0;
    void *t = nullptr;   // PCG work vector t = G r (n x d)
    void *r1 = nullptr;  // second residual buffer (n x d)
};

pfe_status fsai_alloc(pfe_ctx *c);
pfe_status fsai_infer(pfe_ctx *c);
pfe_status fsai_time_infer(pfe_ctx *c, int reps, float *ms);
pfe_status fsai_loss_grad(pfe_ctx *c, double *loss, const double *B = nullptr, int m = 0, double mu = 0.0,
                          double *rterm = nullptr);
pfe_status fsai_export(pfe_ctx *c, double *od, double *oe);
pfe_status fsai_classical(pfe_ctx *c);
pfe_status ic0_factor(pfe_ctx *c);
pfe_status adam_step(float *p, const float *gr, float *m, float *v, int64_t cnt, int step, double lr, double b1,
                     double b2, double eps, cudaStream_t s);

}  // namespace pfe
