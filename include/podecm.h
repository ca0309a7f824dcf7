/*
 * podecm.h -- C ABI of the GB300 hyper-reduced RVE solver.
 *
 * The library solves, for a batch of B independent macro points ("instances"),
 * one load step of the hyper-reduced (POD + empirical cubature) micro problem
 * of Guo, Rokos & Veroy, "A reduced order model for geometrically
 * parameterized two-scale simulations of elasto-plastic microstructures under
 * large deformations" (arXiv 2307.16894):
 *
 *   f_j(a)  = sum_i w_i J_i G_i^T vec(P_i F_mu,i^-T)            Eq. forcevector_ecm
 *   K_jk(a) = sum_i w_i J_i (G_i F_mu^-1)_j : A_i : (G_i F_mu^-1)_k  Eq. stiffnessmatrix_ecm
 *   K da = -f, a += da until ||f|| <= tol                       Eq. red_newton
 *   Pbar = |Omega|^-1 sum_i w_i J_i P_i                          Eq. eff_stress_1
 *   Abar from the d^2 reduced tangent problems                   Eqs. tangent_problem_red, eff_stiffness_1
 *
 * with F_i = Fbar + (G_i a) F_mu,i^-1 and the finite-strain J2 material of
 * Appendix A (multiplicative split, exponential map, log strain, isotropic
 * hardening).  Everything runs in the library's own CUDA kernels on one GPU.
 *
 * Conventions
 *  - d = 2 (plane strain, F33 = 1) or 3.  Second-order tensors are row-major:
 *    vec(T)[a*d + r] = T_ar.  Fourth-order tensors A[(a*d+b)*d*d + c*d+e] =
 *    dP_ab / dF_ce.
 *  - All host pointers are owned by the caller; the library copies what it
 *    keeps.  Device pointers passed to *_device calls are owned by the caller
 *    and must stay valid until the context's stream has passed the call.
 *  - Every call returns a rom_status; no exception crosses the ABI.  The text
 *    of the last error of a context is returned by rom_last_error.
 *    Per-instance solver failures do not fail a call: the call returns ROM_OK
 *    and the failure is reported in rom_step_info.status of that instance,
 *    whose history is then left at the last converged step.
 *  - A context is bound to one device and one CUDA stream and is not
 *    thread-safe; use one context per host thread.
 */
#ifndef PODECM_H
#define PODECM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rom_ctx rom_ctx;      /* library-owned: model data, device buffers, stream */
typedef struct rom_state rom_state;  /* library-owned: per-instance reduced coordinates and history */

typedef enum {
    ROM_OK = 0,
    ROM_E_ARG = 1,            /* invalid argument (sizes, pointers, det F_mu <= 0, ...) */
    ROM_E_STATE = 2,          /* call out of order (e.g. step before basis/cubature/geometry) */
    ROM_E_CUDA = 3,           /* a CUDA runtime call failed */
    ROM_E_NOMEM = 4,          /* device or host allocation failed */
    ROM_E_NOT_CONVERGED = 5,  /* per-instance status: Newton hit max_iter */
    ROM_E_NONFINITE = 6       /* per-instance status: non-finite residual, singular K, det F <= 0 */
} rom_status;

enum { ROM_HARD_LINEAR = 0, ROM_HARD_POWER = 1 };
enum { ROM_PREC_FP64 = 0, ROM_PREC_FP32 = 1, ROM_PREC_TF32 = 2, ROM_PREC_BF16 = 3 };
enum { ROM_START_PLAIN = 0, ROM_START_PREV = 1, ROM_START_MLP = 2 };

/* Material phase (Appendix A, Eqs. j2_1 - j2_10).
 * hard_law = ROM_HARD_LINEAR: sigma_y(xi) = s0 + H_or_k * xi
 * hard_law = ROM_HARD_POWER : sigma_y(xi) = s0 * (1 + H_or_k * xi)^p
 * s0 = +inf makes the phase purely elastic. */
typedef struct {
    double E, nu;
    int32_t hard_law;
    double s0, H_or_k, p;
} rom_phase;

/* Solver options for one load step.
 *  converged iff ||f||_2 <= max(tol_rel * ||f(a0)||_2, tol_abs), a0 = start iterate
 *  (Sec. 2.1 stop rule ||f|| <= eps_newton, made relative);
 *  max_iter: accepted Newton updates before ROM_E_NOT_CONVERGED;
 *  max_ls: backtracking halvings of an update whose residual norm does not
 *          decrease (0 = the plain Newton of Eq. red_newton);
 *  precision: ROM_PREC_FP64 -- everything in FP64;
 *             ROM_PREC_FP32/TF32/BF16 -- return map, yield check, eigen log/exp,
 *             stresses and the convergence test in FP64; the kinematics of 3D models
 *             and the residual of the tensor-core paths in double-float arithmetic
 *             (FP32 pairs, ~48 significant bits; residual error ~1e-12 of
 *             sum |terms|, see fp64_residual); the n x n solve by an FP32 LU with
 *             FP64 residual refinement (n >= 48, FP64 LU fallback) or an FP64 LU;
 *             the tangent in FP32; the stiffness contraction K on the tcgen05 tensor
 *             cores for n <= 64 (FP32 accumulation in tensor memory): FP32 as a TF32
 *             hi/lo split (FP32-accurate), TF32, BF16; for n > 64 FP32 on the CUDA
 *             cores -- an inexact-Newton Jacobian; the converged answer still
 *             satisfies the residual test.  With TF32/BF16 the K used for Abar is one
 *             extra FP32-accurate assembly at the converged iterate;
 *  start: ROM_START_PLAIN a0 = a_n; ROM_START_PREV a0 = a_n + (a_n - a_{n-1});
 *         ROM_START_MLP a0 = a_n + MLP prediction (see rom_mlp_load);
 *  polar_split: 1 = solve on Ubar of Fbar = Rbar Ubar and rotate back (Sec. 4);
 *  want_abar: 1 = compute the effective stiffness;
 *  fp64_residual: 1 = form the residual of the mixed-precision tensor-core paths in
 *         FP64 (one DFMA per multiply-add) instead of double-float FP32 pairs; the
 *         FP64 and CUDA-core paths always form it in FP64.  Default 0.
 * Zero-initialise the struct before setting fields, so that fields added later read 0. */
typedef struct {
    double tol_rel, tol_abs;
    int32_t max_iter;
    int32_t max_ls;
    int32_t precision;
    int32_t start;
    int32_t polar_split;
    int32_t want_abar;
    int32_t fp64_residual;
} rom_opts;

/* Per-instance result of a step. */
typedef struct {
    int32_t iters;    /* accepted Newton updates */
    int32_t evals;    /* residual evaluations after the first (line-search trials included) */
    int32_t status;   /* ROM_OK, ROM_E_NOT_CONVERGED or ROM_E_NONFINITE */
    int32_t n_yield;  /* cubature points that yielded in the accepted state */
    double res0, res; /* ||f|| at the start iterate and at exit */
} rom_step_info;

/* Create a context for dimension dim (2 or 3) on CUDA device `device`, issuing
 * all work on `cuda_stream` (a cudaStream_t; NULL = a new stream owned by the
 * context; pass cudaStreamLegacy for the legacy default stream).  *ctx is set
 * to NULL on failure. */
rom_status rom_create(rom_ctx **ctx, int dim, int device, void *cuda_stream);
/* Wait for the context stream, then free everything the context owns (model copies, work
 * and I/O buffers, the MLP, events) and the stream if the context created it; a stream
 * passed to rom_create stays the caller's.  Destroy the context's states first: a state
 * refers to its context.  NULL: ROM_E_ARG. */
rom_status rom_destroy(rom_ctx *ctx);

/* POD basis gradients at the cubature points (Sec. 3.1, Eq. pod_disp):
 * G[m][d*d][n], G[i][a*d+r][j] = d phi_j,a / d X^p_r at point i.  Host, copied.
 * 1 <= n <= 128, 1 <= m. */
rom_status rom_load_basis(rom_ctx *ctx, int n, int m, const double *G);

/* Empirical cubature rule (Sec. 3.2, Eq. integral_ecm): positive weights w[m],
 * phase index phase[m] into phases[n_phase] (n_phase <= 8) and the parent
 * cell volume |Omega^p| (Eq. eff_stress_1).  Host, copied. */
rom_status rom_load_cubature(rom_ctx *ctx, int m, const double *w, const int32_t *phase, int n_phase,
                             const rom_phase *phases, double omega_vol);

/* Geometry (Sec. 2.1, Eq. weakform-dep-mapped; the geometry step that opens the online stage of Algorithm 1):
 * F_mu,i = I + sum_k mu[b][k] Gmu[i][a*d+r][k] at every point i of instance b.
 * Gmu[m][d*d][n_par] and mu[B][n_par] on the host, copied.  Fails with ROM_E_ARG
 * if any det F_mu <= 0.  1 <= n_par <= 16. */
rom_status rom_set_geometry(rom_ctx *ctx, int64_t B, int n_par, const double *Gmu, const double *mu);

/* Geometry from the reduced auxiliary problem (Sec. 3.4, Eqs. auxiliary_problem and
 * reduced_aux_problem; the geometry step of the online stage of Algorithm 1).  The map is
 * Phi_mu = X + d with d the displacement of a linear-elastic parent domain whose outer boundary
 * is fixed and whose parameterised interior boundary is moved by g(theta)(X) = sum_k theta_k
 * T_k (X - X_c), theta_k = mu_k / mu_ref_k - 1.  Its reduced form: the free part of d lies in
 * the span of n_rb modes psi_j, the prescribed part is the lifting L(theta), and
 *   A_hat d_hat = b_hat(theta),  b_hat = M_deim b(theta)[P],  b(theta)[P] = S theta
 * (discrete empirical interpolation of the forcing b = -K_FD L_D at the rows P; for boundary
 * data linear in theta the rows are S theta exactly).  Per instance the library solves this
 * n_rb x n_rb system on the device and sets
 *   F_mu(X_i) = I + sum_k theta_k GL[i][.][k] + sum_j d_hat_j Gpsi[i][.][j],
 * the map the step kernels use (rom_state / rom_step unchanged; rom_sensitivity is not
 * available with this geometry: it needs at most 3 coefficients).
 *   n_p   geometry parameters, 1 <= n_p <= 8;  n_rb RB modes, 1 <= n_rb <= 8;
 *   n_deim DEIM rows, 1 <= n_deim <= 32;  n_p + n_rb <= 16;
 *   mu_ref[n_p] (> 0), Ahat[n_rb][n_rb], Mdeim[n_rb][n_deim], S[n_deim][n_p],
 *   GL[m][d*d][n_p], Gpsi[m][d*d][n_rb] (gradients at the cubature points, row-major vec),
 *   mu[B][n_p]: all host buffers, copied (the model arrays are read once per call).
 * The solve and a det F_mu > 0 check at every point of every instance run on the device;
 * blocking.  ROM_E_ARG for bad sizes, a singular A_hat, or det F_mu <= 0 anywhere (the text
 * names the first instance and point); ROM_E_STATE before rom_load_basis / rom_load_cubature. */
typedef struct {
    int32_t n_p, n_rb, n_deim;
    const double *mu_ref, *Ahat, *Mdeim, *S, *GL, *Gpsi;
} rom_aux_model;
rom_status rom_set_geometry_aux(rom_ctx *ctx, int64_t B, const rom_aux_model *aux, const double *mu);

/* Per-batch state for B instances: a = 0, C^p^-1 = I, xi = 0 (virgin material).
 * Library-owned device memory (history and the per-step work arrays, rom_state_bytes);
 * ROM_E_STATE before rom_load_basis and rom_load_cubature, ROM_E_NOMEM if it does not fit. */
rom_status rom_state_create(rom_ctx *ctx, int64_t B, rom_state **st);
/* Free the state's device arrays, its captured graph and graph stream (the frees wait for
 * work still using them).  Call before rom_destroy of its context.  NULL: ROM_E_ARG. */
rom_status rom_state_destroy(rom_state *st);

/* Canonical history to/from host buffers: a[B][n], Cpinv[B][m][nc] with
 * nc = 4 (d = 2: C11, C12, C22, C33) or 6 (d = 3: C11, C12, C13, C22, C23, C33)
 * of the inverse plastic right Cauchy-Green tensor C^p^-1 = F^p^-1 F^p^-T,
 * xi[B][m] the equivalent plastic strain.  Any pointer may be NULL (skipped).
 * Blocking. */
rom_status rom_state_export(rom_ctx *ctx, const rom_state *st, double *a, double *Cpinv, double *xi);
rom_status rom_state_import(rom_ctx *ctx, rom_state *st, const double *a, const double *Cpinv, const double *xi);

/* One load step for all B instances (the online Newton loop of Algorithm 1).
 * Fbar[B][d*d] in; Pbar[B][d*d] out; Abar[B][d^4] out (may be NULL if
 * opts->want_abar == 0); info[B] out (may be NULL).  Host buffers; the call
 * copies in, runs, copies out and synchronises.  Converged instances commit
 * their history; the others keep the history of their last converged step. */
rom_status rom_step(rom_ctx *ctx, rom_state *st, const rom_opts *opts, const double *Fbar,
                    double *Pbar, double *Abar, rom_step_info *info);

/* Same with device pointers; asynchronous on the context stream.
 * Tensor-core stiffness (models with n <= 64, every precision but FP64): every pipeline wait inside
 * the kernel is bounded; if one gives up, rom_step (and rom_step_device without graphs)
 * returns ROM_E_CUDA after the Newton passes, and in graph mode the step's Abar entries are
 * NaN (Pbar, info and the history come from the residual test, which no tensor-core result
 * enters, and stay valid). */
rom_status rom_step_device(rom_ctx *ctx, rom_state *st, const rom_opts *opts, const double *Fbar_d,
                           double *Pbar_d, double *Abar_d, rom_step_info *info_d);

/* Shape sensitivities of the effective stress with respect to the geometry parameters
 * (Sec. 2.3, Eq. eff_sensitivities_full) at the converged state of the last rom_step /
 * rom_step_device of `st`: dPbar_ij/dmu_k with mu the coefficients of the affine map
 * F_mu = I + sum_k mu_k Gmu_k given to rom_set_geometry.  The fluctuation sensitivity is the
 * reduced one, K dq_k = -df/dmu_k at fixed a, solved with the factor of K at the solution
 * (K* = K); with the polar split dPbar/dmu = Rbar dPbar(Ubar)/dmu.  Output layout
 * [B][d*d][n_par], entry (b, i*d + j, k); NaN for the instances whose last step did not
 * converge.  Arithmetic: FP64 after a ROM_PREC_FP64 step, FP32 after a mixed-precision step
 * (whose tangent is FP32; the K used is the one of the step: the FP32-accurate re-assembly when
 * the step computed Abar).  At most 3 geometry parameters (ROM_E_ARG otherwise); ROM_E_STATE
 * before the first step.  rom_sensitivity_device: device buffer, asynchronous on the context
 * stream; rom_sensitivity: host buffer, blocking. */
rom_status rom_sensitivity_device(rom_ctx *ctx, rom_state *st, double *dPdmu_d);
rom_status rom_sensitivity(rom_ctx *ctx, rom_state *st, double *dPdmu);

/* Wait for the context stream. */
rom_status rom_sync(rom_ctx *ctx);

/* Text of the last error on this context ("" if none).  Owned by the context. */
const char *rom_last_error(const rom_ctx *ctx);

/* Kernel timing (tracing).  rom_profile(ctx, 1) resets the counters and records
 * CUDA events around every kernel launch of later steps on the context stream;
 * rom_profile(ctx, 0) stops.  rom_profile_read returns, for kernel group
 * 0 start, 1 constitutive (kinematics, return map, tangent), 2 assembly
 * (stiffness; on the CUDA-core path also the force), 3 solve (convergence test, line
 * search, LU), 4 finalize (Pbar, Abar, commit), 5 bookkeeping, 6 learned start
 * (features, MLP inference), 7 force (the residual on the tensor-core paths: double-float,
 * or FP64 with fp64_residual), 8 sensitivity (rom_sensitivity): the
 * summed device time in ms, the number of kernel launches and the algorithmic FLOPs
 * (per active instance and launch: group 1 kinematics 2 m d^2 n; group 2 on the
 * tensor cores 2 m d^4 n + 2 m d^2 n^2 (Y = At G and the full K), on the CUDA cores
 * 2 m d^4 n + m d^2 n (n+1) + 2 m d^2 n (upper triangle of K and the force); group 3
 * 2 n^3/3 + 2 n^2; group 7 2 m d^2 n).  Any pointer may be NULL. */
rom_status rom_profile(rom_ctx *ctx, int enable);

/* Device bytes of a state of B instances (history and per-step work arrays) -- the
 * admission budget of a serving layer. */
rom_status rom_state_bytes(const rom_ctx *ctx, int64_t B, int64_t *bytes);

/* Autotune the CUDA-core stiffness assembly (FP64/FP32 modes): times the tile edges
 * 2/4/8 x points-per-chunk 8/16/32/64 on the state's current tangents (call after at
 * least one step) and keeps the fastest for this context.  Outputs may be NULL. */
rom_status rom_autotune(rom_ctx *ctx, rom_state *st, const rom_opts *opts, int *tile, int *chunk, float *ms);

/* Ragged serving: one load step for G groups (each its own model/context, state, options
 * and device I/O buffers; contexts and states distinct) as ONE CUDA-graph launch: the call
 * captures every group's step (start, learned start, its own device-driven WHILE node over
 * the Newton passes, finalize) on parallel branches of one graph, so groups of different
 * basis size n, cubature size m and Newton iteration count run concurrently, each for as many
 * passes as its instances need.  The graph is launched on ctxs[0]'s stream after the inputs
 * are copied into the states' staging buffers; the outputs are copied back.  group_ms[g] (may
 * be NULL) = time from the launch to the end of group g's branch (an event node).  Abar_d /
 * info_d may be NULL (Abar_d[g] is needed when opts[g].want_abar).  Blocking; the graph is
 * built and released inside the call (a few ms for a handful of groups). */
rom_status rom_serve(int G, rom_ctx *const *ctxs, rom_state *const *sts, const rom_opts *opts,
                     const double *const *Fbar_d, double *const *Pbar_d, double *const *Abar_d,
                     rom_step_info *const *info_d, float *group_ms);

/* Graph mode: with enable = 1, rom_step_device runs each load step as one CUDA-graph launch
 * whose Newton passes execute inside a conditional WHILE node decided on the device (no
 * host synchronisation per pass).  The graph is captured on the first step with given
 * options for a state and reused while the options stay the same; Fbar is copied into and
 * Pbar, Abar, info out of state-owned buffers around the launch.  Profiling (rom_profile)
 * uses the per-launch path.  Default 0. */
rom_status rom_use_graphs(rom_ctx *ctx, int enable);

/* Diagnostics: the reduced stiffness K[B][n][n] of the last evaluated iterate of every
 * instance (as assembled by the selected precision mode; for ROM_PREC_TF32/BF16 and
 * converged instances with want_abar, the FP32 re-assembly used for Abar).  Blocking. */
rom_status rom_debug_stiffness(rom_ctx *ctx, const rom_state *st, double *K);
/* Diagnostics: the pulled-back tangent At of the last evaluated iterate, copied to the host
 * buffer `At` of `bytes` bytes (at most the array's size is copied).  Layout [B][d^4][mA],
 * mA = m rounded up to a multiple of 4, entry (b, (a*d + r)*d*d + c*d + s, i) =
 * w_i J_i sum_{t,u} Finv_i[r][t] dP_i[a][t]/dF[c][u] Finv_i[s][u]; element type double after a
 * ROM_PREC_FP64 step, float otherwise.  Valid for the instances of the last pass.  Blocking. */
rom_status rom_debug_tangent(rom_ctx *ctx, const rom_state *st, void *At, int64_t bytes);
/* Diagnostics: the reduced residual r[B][n] = sum_i w_i J_i G_i^T vec(P_i F_mu,i^-T) of the last
 * evaluated iterate (Eq. of the ECM force vector, Sec. 3.2) and, when `v` is not NULL, the weighted
 * pulled-back stresses v[B][d*d][m] it was formed from (entry (b, a*d + r, i)).  The residual is
 * formed in FP64 after a ROM_PREC_FP64 step and in double-float arithmetic (FP32 pairs) on the
 * mixed-precision tensor-core paths.  Valid for the instances of the last pass.  Blocking. */
rom_status rom_debug_residual(rom_ctx *ctx, const rom_state *st, double *r, double *v);
rom_status rom_profile_read(rom_ctx *ctx, int kernel, double *ms, int64_t *launches, double *flops);

/* ---------------------------------------------------------------------------
 * Learned Newton start (not in the paper, whose Newton start is unspecified).
 * A multilayer perceptron with `depth` hidden layers of `width` units (exact-erf
 * GELU) maps the features of a step
 *     x = [Ubar_k - Ubar_{k-1} (d*d), mu (n_par), a_n (n), a_n - a_{n-1} (n),
 *          mean_i xi_i, max_i xi_i]
 * (n_in = d*d + n_par + 2n + 2; Ubar = stretch of the polar split of Fbar) to the
 * correction of the previous-step increment, da_k - da_{k-1} (n_out = n); the learned
 * start is a_n + da_{k-1} + correction.  Inference uses BF16 weights with FP32
 * accumulation; training keeps an FP32 master copy updated by Adam (beta = 0.9, 0.999,
 * eps = 1e-8) on the mean squared error of the standardised targets.  With
 * opts->start = ROM_START_MLP, rom_step evaluates the residual at the learned start; if
 * it is finite and at most r_ref, the residual of the previous-step predictor
 * a_n + (a_n - a_{n-1}) of the instance's last step that evaluated one, Newton starts
 * from it; otherwise rom_step also evaluates the previous-step predictor (the fallback;
 * one extra residual evaluation, counted in evals), stores its residual as the new r_ref
 * and starts from the smaller of the two.  r_ref is +inf after rom_state_create or an
 * import of a, so the first learned step always evaluates both; steps with
 * ROM_START_PREV also refresh it.  The converged answer does not depend on the start.
 * In this mode the convergence tolerance is relative to r_ref (or to the fallback's
 * residual when it is evaluated), so both starts are held to the same absolute residual.
 *
 * rom_mlp_init: allocate an MLP (random parameters are set by rom_mlp_params);
 *   max_rows = largest batch of rows of any later train/grad/predict call.
 * rom_mlp_params: get (get_host != NULL) and/or set (set_host) the packed FP32
 *   parameters: for every linear map l (n_in -> width -> ... -> width -> n_out)
 *   W_l[out][in] row-major then b_l[out]; rom_mlp_nparams gives their count.
 *   Setting the parameters resets the Adam moments.
 * rom_mlp_norm: x_mean[n_in], x_std[n_in], y_mean[n_out], y_std[n_out] (host);
 *   the network sees (x - x_mean)/x_std and is trained on (y - y_mean)/y_std.
 * rom_mlp_train_step: one Adam step (learning rate lr, step count t >= 1) on the
 *   device batch X_d[N][n_in], Y_d[N][n_out] (raw units); the loss before the
 *   update goes to loss_d[1] (device, may be NULL).  Asynchronous.
 * rom_mlp_loss_grad: loss and gradient (packed like the parameters) without update;
 *   bf16 = 0 uses the FP32 weights.  Device outputs.  Asynchronous.
 * rom_mlp_predict: out_d[N][n_out] (double, raw units) for X_d[N][n_in].  bf16 = 1 with
 *   width 128, n_in <= 256 and n_out <= 128: the whole network on the tcgen05 tensor cores
 *   (one fused kernel per 128 rows, BF16 weights and activations, FP32 accumulation); other
 *   shapes and bf16 = 0 (FP32 weights): CUDA-core kernels with FP32 activations.  Asynchronous.
 * rom_features: the features X_d[B][n_in] (device) of the step Fbar_d[B][d*d] for
 *   the current state of every instance.  Asynchronous. */
rom_status rom_mlp_init(rom_ctx *ctx, int n_in, int width, int depth, int n_out, int64_t max_rows);
rom_status rom_mlp_nparams(rom_ctx *ctx, int64_t *nparams);
rom_status rom_mlp_params(rom_ctx *ctx, float *get_host, const float *set_host);
rom_status rom_mlp_norm(rom_ctx *ctx, const float *norm_host);
rom_status rom_mlp_train_step(rom_ctx *ctx, const float *X_d, const float *Y_d, int64_t N, float lr, int t,
                              float *loss_d);
rom_status rom_mlp_loss_grad(rom_ctx *ctx, const float *X_d, const float *Y_d, int64_t N, int bf16, float *grad_d,
                             float *loss_d);
rom_status rom_mlp_predict(rom_ctx *ctx, const float *X_d, int64_t N, int bf16, double *out_d);
rom_status rom_features(rom_ctx *ctx, rom_state *st, const double *Fbar_d, float *X_d);

/* ---------------------------------------------------------------------------
 * Offline stage on the device (the offline stage of Algorithm 1; Sec. 3.1-3.2).  These calls
 * take no context: device pointers on `cuda_stream` (a cudaStream_t, NULL = legacy default
 * stream), library-owned scratch allocated and freed inside the call, blocking.  FP64
 * arithmetic.  errbuf (errlen bytes, may be NULL) receives the text of an error.
 *
 * rom_pod: POD by the method of snapshots (Eq. pod_disp and the orthonormality relation after
 * it).  S[ns][N] holds the ns snapshots (one per row).  The inner product is u^T M v with M the
 * CSR matrix (rowptr[N+1], col[nnz], val[nnz]; e.g. the V^p Gram matrix of Eq. Vdotproduct),
 * or, with rowptr = NULL, the diagonal wdiag[N] (the L^2 POD of the weighted stress), or the
 * identity (both NULL).  C = S M S^T, C = V diag(lam) V^T (parallel cyclic Jacobi), and
 * Phi[j][.] = sum_a V[a][j] S[a][.] / sqrt(lam_j) for j < n_modes, so Phi M Phi^T = I.
 * lam[ns]: all eigenvalues, descending; sweeps (may be NULL): Jacobi sweeps used.
 * 1 <= n_modes <= ns <= 1024; ROM_E_ARG if n_modes exceeds the numerical rank (eigenvalues
 * above 1e-14 lam_0), ROM_E_NOMEM / ROM_E_CUDA otherwise on failure. */
rom_status rom_pod(void *cuda_stream, int64_t N, int ns, const double *S, const int32_t *rowptr,
                   const int32_t *col, const double *val, const double *wdiag, int n_modes, double *Phi,
                   double *lam, int *sweeps, char *errbuf, size_t errlen);

/* rom_ecm: the empirical cubature greedy (Sec. 3.2, Eq. integral_ecm).  F[P][M] holds P
 * integrands at the M Gauss points of the parent mesh, wq[M] their Gauss weights (device).
 * The integrand space is replaced by an orthonormal basis Z (eigenpairs of F diag(wq) F^T;
 * directions with eigenvalue <= 1e-13 of the largest are dropped) to which the constant
 * function scaled by volume_weight / sqrt(sum wq) is appended; b = Z wq.  Each step adds the
 * point whose column is most aligned with the residual r = b - Z_E w_E (score Z[:,x].r /
 * |Z[:,x]|, ties to the lower index) and refits non-negative weights on the selected set by
 * least squares: a rank-one extension of the Cholesky factor of Z_E^T Z_E when every weight
 * stays positive, else an active-set (Lawson-Hanson) solve; points whose weight is not positive
 * leave the set.  It stops when m points are selected (m >= 1), or, with m < 1, when
 * |r| <= tol |b|, and gives up after 20 m (or 20 M) steps.  Outputs on the host: idx[cap]
 * (point indices in selection order), w[cap], m_out, err (= |r| / |b|, may be NULL), rank (the
 * basis dimension, may be NULL).  1 <= P <= 1024, cap >= m.  ROM_E_NOT_CONVERGED if the greedy
 * stalls (the outputs then hold its last state). */
rom_status rom_ecm(void *cuda_stream, int P, int64_t M, const double *F, const double *wq, int m, double tol,
                   double volume_weight, int cap, int64_t *idx, double *w, int *m_out, double *err, int *rank,
                   char *errbuf, size_t errlen);

/* rom_fe_train: the full-order training solves of the offline stage (Sec. 2.1: Eqs.
 * weakform-dep-mapped, Dweakform-dep and full_newton) for S samples at once, each with its own
 * geometry (F_mu = I + sum_k coef[s][k] Gmu[q][.][k] at the Gauss points) and load path
 * Fbar[s][steps][d*d].  The mesh is given by its elements: edof[ne][nen*d] (global fluctuation
 * dof of each element dof, -1 where fixed), the reference shape-function gradients
 * dN[ngp][nen][d] with respect to X^p and the Gauss weights gw[ngp] (the same for every
 * element of the structured grid), el_phase[ne] into phases[n_phase].  Each load step starts
 * from the previous solution; Newton stops at ||f|| <= max(tol_rel ||f_0||, tol_abs) (at most
 * max_iter iterations, backtracking line search on ||f||, halving up to 10 times), the linear
 * systems are solved by Jacobi-preconditioned conjugate gradients to 1e-12 relative; a step
 * whose Newton fails is split into half increments, at most max_split times.  Outputs (host):
 * w[S][steps][ndof] the fluctuation snapshots, W[S][steps][ne*ngp][d*d] (may be NULL) the
 * weighted stress J P F_mu^-T at the Gauss points, Pbar[S][steps][d*d] (|Omega^p| = 1),
 * iters / substeps [S][steps] (may be NULL).  All host buffers; device work arrays are
 * allocated and freed inside the call; blocking.  ROM_E_NOT_CONVERGED if a step still fails
 * after max_split splits. */
typedef struct {
    int32_t d, ne, nen, ngp, ndof;
    const int32_t *edof;
    const double *dN, *gw;
    const int32_t *el_phase;
} rom_fe_mesh;
rom_status rom_fe_train(const rom_fe_mesh *mesh, int n_phase, const rom_phase *phases, int S, int n_par,
                        const double *Gmu, const double *coef, int steps, const double *Fbar, double tol_rel,
                        double tol_abs, int max_iter, int max_split, double *w, double *W, double *Pbar,
                        int32_t *iters, int32_t *substeps, char *errbuf, size_t errlen);

/* rom_ecm_integrands: the integrands of the cubature fit (Eq. integral_ecm) on the device.
 * Phi[n][ndof] (device): the fluctuation modes; B[L][ne*ngp][d*d] (device): the weighted-stress
 * modes at the Gauss points.  Outputs (device): gradPhi[ne*ngp][d*d][n] = dphi_i/dX^p at every
 * Gauss point (row-major vec, component-major) and F[n*L][ne*ngp] with F[i*L+l][q] =
 * dphi_i/dX^p : B_l at Gauss point q.  The mesh (host arrays, see rom_fe_train) is copied.
 * Blocking. */
rom_status rom_ecm_integrands(void *cuda_stream, const rom_fe_mesh *mesh, int n, const double *Phi, int L,
                              const double *B, double *gradPhi, double *F, char *errbuf, size_t errlen);


/* ---------------------------------------------------------------------------
 * Allocation-free step.  The paper has no counterpart: this is a deployment
 * variant of rom_step_device for callers that cannot call cudaMalloc -- a
 * macro solver running inside a pre-sized memory pool or arena it does not
 * own, or a host application that must not grow its device footprint after
 * start-up (where an allocation could fail or stall the rest of the
 * application).
 *
 * The caller passes every array on the device: the model in the public
 * layouts (G[m][d*d][n], w[m], phase[m], Gmu[m][d*d][n_par]; the phase table
 * phases[n_phase] on the host), the geometry mu[B][n_par], the state -- a[B][n],
 * the last converged increment da_prev[B][n] (zero at the start), the history
 * Cpinv[B][nc][m] (component-major per instance: nc = 4 in 2D (C11, C12, C22,
 * C33), 6 in 3D (C11, C12, C13, C22, C23, C33); identity at the start) and
 * xi[B][m] -- all updated in place for converged instances, and Fbar[B][d*d],
 * Pbar[B][d*d], Abar[B][d^4] (NULL if want_abar = 0), info[B] (may be NULL).
 * The work arrays of the step live in one static device array of
 * ROM_NOALLOC_SCRATCH_BYTES (16 MiB) that every GPU loading the library holds
 * until the process exits; a batch whose work space does not fit (about
 * 10 KB per instance for n = 8, m = 40 in 2D and 42 KB for n = 24, m = 160)
 * is rejected with ROM_E_ARG.  The call allocates nothing: no cudaMalloc,
 * cudaFree or allocating library routine.
 *  - The call synchronises the stream: every Newton pass reads the active
 *    count back to the host, and the phase table is swapped through host
 *    memory.  It must not be called while the stream (or any stream of the
 *    process, in global capture mode) is being captured into a graph.
 *  - The first call on a device looks up the device address of the static
 *    array (cudaGetSymbolAddress, with that device current).
 *  - All calls on a device share the array, and it keeps the previous call's
 *    contents (the call clears what must start at zero).  Calls that overlap
 *    on the GPU -- on different streams or host threads -- race on it; so do
 *    contexts' steps running at the same time, because the call temporarily
 *    installs its phase table in the library's device-wide material table and
 *    restores it at the end.
 *  - precision: ROM_PREC_FP64 or ROM_PREC_FP32; start: PLAIN or PREV.  The
 *    geometry is not validated (det F_mu > 0 is the caller's responsibility).
 *  - Blocking on `cuda_stream` (a cudaStream_t, NULL = legacy default stream).
 *    errbuf (errlen bytes, may be NULL) receives the text of an error. */
#define ROM_NOALLOC_SCRATCH_BYTES (16 * 1024 * 1024)
typedef struct {
    int32_t dim, n, m, n_par, n_phase;
    const double *G, *w;
    const int32_t *phase;
    const double *Gmu;
    const rom_phase *phases;
    double omega_vol;
} rom_noalloc_model;

rom_status rom_step_noalloc(const rom_noalloc_model *model, int64_t B, const double *mu, double *a, double *da_prev,
                            double *Cpinv, double *xi, const rom_opts *opts, const double *Fbar, double *Pbar,
                            double *Abar, rom_step_info *info, void *cuda_stream, char *errbuf, size_t errlen);

#ifdef __cplusplus
}
#endif
#endif
