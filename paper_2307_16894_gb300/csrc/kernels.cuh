// Device data structures shared by the kernels of the hyper-reduced RVE step.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "material.cuh"

namespace podecm {

constexpr int MAX_PHASES = 8;
constexpr int MAX_NPAR = 16;
constexpr int MAX_N = 128;

// per-instance Newton control block
struct Ctl {
    double r0, tol, rn_acc, t;
    int32_t iters, evals, ls, status;
    int32_t active, phase;   // phase 0: start evaluation pending, 1: trial evaluation pending
    int32_t acc_k, pad1;   // acc_k: assemble this instance's stiffness FP32-accurately (BF16/TF32 modes)
};

// model (shared by all instances)
struct Model {
    int d, d2, n, m, n_par, nphase, ncp;
    int mA;                // row stride of the tangent array At (m rounded up to a multiple of 4)
    const double *G_pt;    // [m][d2][n]
    const double *G_T;     // [d2][n][m]
    const float *G32_pt;   // [m][d2][n]
    const float *G32h_T;   // [d2][n][m] FP32 high part of G_T (mixed-precision kinematics), may be null
    const float *G32l_T;   // [d2][n][m] FP32 low part, G_T - G32h_T rounded to FP32
    const float2 *Gdf;     // [d2][m][n rounded up to even] (hi, lo) FP32 split of G in the order of v,
                           // zero padded (double-float residual of the mixed-precision paths), may be null
    const double *w;       // [m]
    const int32_t *phase;  // [m]
    const double *Gmu_T;   // [d2][n_par][m]
    double omega;
};

// one batch (state + work arrays)
struct Batch {
    int64_t B;
    const double *mu;        // [B][n_par]
    double *q_n, *dq_prev;   // [B][n] committed coordinates, last converged increment
    double *cp, *xi;         // [B][ncp][m], [B][m] committed history
    double *q_trial, *q_acc, *dq;   // [B][n]
    Ctl *ctl;                // [B]
    int32_t *list;           // [B] active instances (compacted)
    int32_t *counts;         // [0] = active count, [1] = next count
    double *v;               // [B][d2][m]  wJ vec(P F_mu^-T)
    double *wP;              // [B][d2][m]  wJ P
    void *At;                // [B][d2*d2][mA] pulled-back tangent (double or float)
    double *cp_tr, *xi_tr;   // trial history
    uint8_t *pl;             // [B][m] plastic flags of the last evaluation
    double *r;               // [B][n]
    double *K;               // [B][n][n]
    double *Ubar, *Rbar;     // [B][d2]
    double *U_prev;          // [B][d2] stretch of the last converged step (learned start features), may be null
    double *r0_prev;         // [B] residual norm of the previous-step predictor when last evaluated (+inf
                             // if never), the reference of the learned start; may be null
    const int *err;          // tensor-core pipeline error flag (a bounded wait gave up), may be null
    double *Bsum;            // [B][n d2 + d4]: B = sum_i G_i^T Ahat_i (n x d2) and A0 (d4) of the converged
                             // instances from the tensor cores (k_abar_tc3) when non-null in the
                             // finalize; else the finalize forms them
    const double *geo;       // [B][d2 + 1][m] F_mu^-1 (row-major) and w_i J_mu per point, computed once
                             // per geometry (k_geometry); null: the constitutive kernel forms them
};

// learned Newton start (mlp.cu)
struct MlpDev {
    int n_in, width, depth, n_out, L;
    int64_t nparams;
    float *p32, *m, *v, *grad;
    void *p16;                      // __nv_bfloat16 copy of p32
    float *norm;                    // x_mean[n_in] x_std[n_in] y_mean[n_out] y_std[n_out]
    float *Z, *H, *dH;              // work arrays
    float *loss;
    int64_t cap;
    int wmax;
};

struct StepOpts {
    double tol_rel, tol_abs;
    int max_iter, max_ls, precision, start, polar, want_abar;
    int fp64_residual = 0;          // tensor-core paths: FP64 residual instead of double-float
    int asm_tm = 0, asm_ch = 0;   // assembly tile edge / points per chunk (0 = heuristic)
};

}  // namespace podecm
