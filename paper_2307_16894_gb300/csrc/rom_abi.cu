// C ABI of the GB300 hyper-reduced RVE solver (declarations and contracts in
// include/podecm.h).  Host-side bookkeeping only: argument checks, device
// buffers, and the launch sequence of one load step; all arithmetic of the
// step runs in the kernels of kernels.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/podecm.h"
#include "kernels.cuh"

namespace podecm {
void set_phases(const PhaseD *ph, int n, cudaStream_t s);
int launch_start(const Model &M, Batch Bt, const double *Fbar, const StepOpts &o, const double *dq_pred,
                 cudaStream_t s);
int launch_kernel(int which, const Model &M, Batch Bt, const StepOpts &o, int32_t *list_next, cudaStream_t s);
int launch_finalize(const Model &M, Batch Bt, const StepOpts &o, double *Pbar, double *Abar, void *info,
                    cudaStream_t s);
void launch_add_pred(Batch Bt, int n, const double *pred, cudaStream_t s);
void launch_features(const Model &M, Batch Bt, const double *U_prev, float *X, int n_in, cudaStream_t s);
int mlp_alloc(MlpDev &M, int n_in, int width, int depth, int n_out, int64_t cap);
void mlp_free(MlpDev &M);
void mlp_set_params(MlpDev &M, const float *host, cudaStream_t s);
void mlp_get_params(const MlpDev &M, float *host, cudaStream_t s);
void mlp_set_norm(MlpDev &M, const float *host, cudaStream_t s);
void mlp_train_step(MlpDev &M, const float *X, const float *Y, int64_t N, float lr, int t, float *loss_out,
                    cudaStream_t s);
void mlp_loss_grad(MlpDev &M, const float *X, const float *Y, int64_t N, int bf16, float *grad_out, float *loss_out,
                   cudaStream_t s);
void mlp_predict(MlpDev &M, const float *X, int64_t N, int bf16, double *out, cudaStream_t s, int *err);
size_t tc2_image_bytes(int fmt, int n, int m);
void tc2_build_image(int fmt, int n, int m, const double *G, unsigned char *img);
int launch_tc2(int mode, const Model &M, Batch Bt, const unsigned char *img, int *err, int sel, cudaStream_t s);
size_t tc3_image_bytes(int m);
void tc3_build_images(int n, int m, const double *G, unsigned char *img);
int launch_tc3(int mode, const Model &M, Batch Bt, const unsigned char *img, int *err, int sel, cudaStream_t s);
int launch_abar_tc3(const Model &M, Batch Bt, const unsigned char *img, double *Bsum, int *err, cudaStream_t s);
int launch_abar_tcp(const Model &M, Batch Bt, const unsigned char *img, double *Bsum, int *err, cudaStream_t s);

void launch_force(const Model &M, Batch Bt, bool fp64, cudaStream_t s);
void launch_geometry(const Model &M, const double *mu, int64_t B, double *geo, cudaStream_t s);
int launch_sensitivity(const Model &M, Batch Bt, int precision, double *out, cudaStream_t s);
bool separate_force(const Model &M, const StepOpts &o);
void launch_list_converged(Batch Bt, cudaStream_t s);
void launch_flag_final(const Model &M, Batch Bt, const StepOpts &o, int32_t *tmp, cudaStream_t s);
void launch_graph_advance(Batch Bt, const int32_t *list_next, cudaGraphConditionalHandle h, int max_pass,
                          cudaStream_t s);
void launch_reset_pass(Batch Bt, cudaStream_t s);
void launch_all_active(Batch Bt, cudaStream_t s);
int aux_max();
void launch_aux_geometry(int n_p, int n_rb, int n_deim, const double *mu_ref, const double *Ahat,
                         const double *Mdeim, const double *S, int64_t B, const double *mu, double *coef, int *bad,
                         cudaStream_t s);
void launch_geom_check(int d, int m, int nc, int64_t B, const double *coef, const double *Gmu_T,
                       unsigned long long *first_bad, cudaStream_t s);
}  // namespace podecm

using namespace podecm;

#define ROM_NKERNELS 9

struct rom_ctx {
    int dim = 0, device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    int n = 0, m = 0, n_par = 0, nphase = 0;
    bool has_basis = false, has_cub = false, has_geom = false;
    double omega = 1.0;
    int64_t B = 0;
    double *G_pt = nullptr, *G_T = nullptr, *w = nullptr, *Gmu_T = nullptr, *mu = nullptr;
    float *G32 = nullptr;
    float *G32h_T = nullptr, *G32l_T = nullptr;   // double-float split of G_T (mixed-precision kinematics)
    float2 *Gdf = nullptr;                        // double-float split of G in v order (mixed-precision residual)
    int32_t *phase = nullptr;
    // host-call staging
    double *h_stage = nullptr;      // pinned
    size_t h_stage_bytes = 0;
    double *d_Fbar = nullptr, *d_Pbar = nullptr, *d_Abar = nullptr;
    void *d_info = nullptr;
    int64_t io_B = 0;
    int32_t *h_count = nullptr;     // pinned
    // per-kernel profiling (CUDA events around each launch on the context stream)
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    struct Rec { int kid; int ev0, ev1; double flops; int launches; };
    std::vector<Rec> recs;
    double prof_ms[ROM_NKERNELS] = {0};
    int64_t prof_launches[ROM_NKERNELS] = {0};
    double prof_flops[ROM_NKERNELS] = {0};
    // tensor-core assembly: pre-arranged B-operand images of G (BF16, TF32) and an error flag
    unsigned char *tc_img[2] = {nullptr, nullptr};   // 2D tensor-core B-operand images (BF16, TF32)
    unsigned char *tc3_img = nullptr;                 // 3D tensor-core images (tc_assemble3.cu)
    int *d_err = nullptr;
    // per-geometry cache of F_mu^-1 and w J per point [B][d2 + 1][m], built before the first step
    // after the basis, cubature or geometry changed (ensure_geo)
    double *geo = nullptr;
    bool geo_ok = false;
    // learned Newton start
    bool has_mlp = false, mlp_norm = false;
    MlpDev mlp{};
    bool graphs = false;            // rom_step_device through a captured step graph
    int64_t graph_epoch = 0;        // bumped when buffers captured by graphs are reallocated
    int asm_tm = 0, asm_ch = 0;     // autotuned assembly tiles (0 = heuristic)
    float *d_feat = nullptr;        // [B][n_in]
    double *d_pred = nullptr;       // [B][n]
    int64_t feat_B = 0;
};

struct rom_state {
    rom_ctx *ctx = nullptr;
    int64_t B = 0;
    int n = 0, m = 0, d = 0;
    Batch bt{};
    int32_t *list2 = nullptr;
    std::vector<void *> allocs;
    // captured step graph (device-driven Newton loop) and its fixed I/O buffers
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t gstream = nullptr;
    rom_opts gopts{};
    bool g_valid = false;
    int64_t g_epoch = -1;
    double *io_F = nullptr, *io_P = nullptr, *io_A = nullptr;
    void *io_info = nullptr;
    int last_prec = -1;   // precision of the last step (type of the stored tangent), -1 before the first
};

static rom_status fail(rom_ctx *c, rom_status s, const char *fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return fail(ctx, ROM_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static rom_status dalloc(rom_ctx *ctx, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(ctx, e == cudaErrorMemoryAllocation ? ROM_E_NOMEM : ROM_E_CUDA, "cudaMalloc(%zu): %s", bytes,
                    cudaGetErrorString(e));
    }
    return ROM_OK;
}

static void dfree(void *&p) {
    if (p) cudaFree(p);
    p = nullptr;
}

extern "C" {

rom_status rom_create(rom_ctx **out, int dim, int device, void *cuda_stream) {
    if (!out) return ROM_E_ARG;
    *out = nullptr;
    if (dim != 2 && dim != 3) return ROM_E_ARG;
    rom_ctx *ctx = new (std::nothrow) rom_ctx();
    if (!ctx) return ROM_E_NOMEM;
    ctx->dim = dim;
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) { delete ctx; return ROM_E_CUDA; }
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) { delete ctx; return ROM_E_CUDA; }
        ctx->own_stream = true;
    }
    if (cudaMallocHost((void **)&ctx->h_count, 64) != cudaSuccess) { delete ctx; return ROM_E_NOMEM; }
    *out = ctx;
    return ROM_OK;
}

static void free_io(rom_ctx *ctx) {
    void *p;
    p = ctx->d_Fbar; dfree(p); ctx->d_Fbar = nullptr;
    p = ctx->d_Pbar; dfree(p); ctx->d_Pbar = nullptr;
    p = ctx->d_Abar; dfree(p); ctx->d_Abar = nullptr;
    dfree(ctx->d_info);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    ctx->h_stage = nullptr;
    ctx->h_stage_bytes = 0;
    ctx->io_B = 0;
}

rom_status rom_destroy(rom_ctx *ctx) {
    if (!ctx) return ROM_E_ARG;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    void *p;
    p = ctx->G_pt; dfree(p);
    p = ctx->G_T; dfree(p);
    p = ctx->G32; dfree(p);
    p = ctx->G32h_T; dfree(p);
    p = ctx->G32l_T; dfree(p);
    p = ctx->Gdf; dfree(p);
    p = ctx->w; dfree(p);
    p = ctx->Gmu_T; dfree(p);
    p = ctx->mu; dfree(p);
    p = ctx->phase; dfree(p);
    free_io(ctx);
    if (ctx->h_count) cudaFreeHost(ctx->h_count);
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    if (ctx->has_mlp) mlp_free(ctx->mlp);
    p = ctx->d_feat; dfree(p);
    p = ctx->d_pred; dfree(p);
    p = ctx->tc_img[0]; dfree(p);
    p = ctx->tc_img[1]; dfree(p);
    p = ctx->tc3_img; dfree(p);
    p = ctx->geo; dfree(p);
    p = ctx->d_err; dfree(p);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return ROM_OK;
}

rom_status rom_load_basis(rom_ctx *ctx, int n, int m, const double *G) {
    if (!ctx) return ROM_E_ARG;
    if (n < 1 || n > MAX_N || m < 1 || !G) return fail(ctx, ROM_E_ARG, "rom_load_basis: bad n=%d m=%d or G", n, m);
    if (ctx->has_cub && m != ctx->m) return fail(ctx, ROM_E_ARG, "rom_load_basis: m=%d differs from cubature m=%d", m, ctx->m);
    for (size_t k = 0; k < (size_t)m * ctx->dim * ctx->dim * n; ++k)
        if (!std::isfinite(G[k])) return fail(ctx, ROM_E_ARG, "rom_load_basis: non-finite G");
    CK(cudaSetDevice(ctx->device));
    const int d2 = ctx->dim * ctx->dim;
    const size_t cnt = (size_t)m * d2 * n;
    void *p;
    p = ctx->G_pt; dfree(p); ctx->G_pt = nullptr;
    p = ctx->G_T; dfree(p); ctx->G_T = nullptr;
    p = ctx->G32; dfree(p); ctx->G32 = nullptr;
    rom_status s;
    if ((s = dalloc(ctx, (void **)&ctx->G_pt, cnt * 8)) != ROM_OK) return s;
    if ((s = dalloc(ctx, (void **)&ctx->G_T, cnt * 8)) != ROM_OK) return s;
    if ((s = dalloc(ctx, (void **)&ctx->G32, cnt * 4)) != ROM_OK) return s;
    std::vector<double> gt(cnt);
    std::vector<float> g32(cnt);
    for (int i = 0; i < m; ++i)
        for (int c = 0; c < d2; ++c)
            for (int j = 0; j < n; ++j) {
                const double g = G[((size_t)i * d2 + c) * n + j];
                gt[((size_t)c * n + j) * m + i] = g;
                g32[((size_t)i * d2 + c) * n + j] = (float)g;
            }
    CK(cudaMemcpy(ctx->G_pt, G, cnt * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->G_T, gt.data(), cnt * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->G32, g32.data(), cnt * 4, cudaMemcpyHostToDevice));
    p = ctx->G32h_T; dfree(p); ctx->G32h_T = nullptr;
    p = ctx->G32l_T; dfree(p); ctx->G32l_T = nullptr;
    {
        std::vector<float> gh(cnt), gl(cnt);
        for (size_t k = 0; k < cnt; ++k) {
            gh[k] = (float)gt[k];
            gl[k] = (float)(gt[k] - (double)gh[k]);
        }
        if ((s = dalloc(ctx, (void **)&ctx->G32h_T, cnt * 4)) != ROM_OK) return s;
        if ((s = dalloc(ctx, (void **)&ctx->G32l_T, cnt * 4)) != ROM_OK) return s;
        CK(cudaMemcpy(ctx->G32h_T, gh.data(), cnt * 4, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(ctx->G32l_T, gl.data(), cnt * 4, cudaMemcpyHostToDevice));
    }
    p = ctx->Gdf; dfree(p); ctx->Gdf = nullptr;
    {
        const int np = (n + 1) & ~1;   // rows of 16-byte multiples
        std::vector<float2> gdf((size_t)d2 * m * np, make_float2(0.f, 0.f));
        for (int c = 0; c < d2; ++c)
            for (int i = 0; i < m; ++i)
                for (int j = 0; j < n; ++j) {
                    const double g = G[((size_t)i * d2 + c) * n + j];
                    const float h = (float)g;
                    gdf[((size_t)c * m + i) * np + j] = make_float2(h, (float)(g - (double)h));
                }
        if ((s = dalloc(ctx, (void **)&ctx->Gdf, gdf.size() * 8)) != ROM_OK) return s;
        CK(cudaMemcpy(ctx->Gdf, gdf.data(), gdf.size() * 8, cudaMemcpyHostToDevice));
    }
    for (int f = 0; f < 2; ++f) { p = ctx->tc_img[f]; dfree(p); ctx->tc_img[f] = nullptr; }
    p = ctx->tc3_img; dfree(p); ctx->tc3_img = nullptr;
    if (n <= 64 && ctx->dim == 3) {
        std::vector<unsigned char> img(tc3_image_bytes(m));
        tc3_build_images(n, m, G, img.data());
        if ((s = dalloc(ctx, (void **)&ctx->tc3_img, img.size())) != ROM_OK) return s;
        CK(cudaMemcpy(ctx->tc3_img, img.data(), img.size(), cudaMemcpyHostToDevice));
    }
    if (n <= 64) {
        for (int f = 0; f < 2 && ctx->dim == 2; ++f) {
            std::vector<unsigned char> img(tc2_image_bytes(f + 1, n, m));
            tc2_build_image(f + 1, n, m, G, img.data());
            if ((s = dalloc(ctx, (void **)&ctx->tc_img[f], img.size())) != ROM_OK) return s;
            CK(cudaMemcpy(ctx->tc_img[f], img.data(), img.size(), cudaMemcpyHostToDevice));
        }
        if (!ctx->d_err) {
            if ((s = dalloc(ctx, (void **)&ctx->d_err, 16)) != ROM_OK) return s;
            CK(cudaMemset(ctx->d_err, 0, 16));
        }
    }
    ctx->n = n;
    ctx->m = m;
    ctx->has_basis = true;
    ctx->geo_ok = false;
    return ROM_OK;
}

rom_status rom_load_cubature(rom_ctx *ctx, int m, const double *w, const int32_t *phase, int n_phase,
                             const rom_phase *phases, double omega_vol) {
    if (!ctx) return ROM_E_ARG;
    if (m < 1 || !w || !phase || !phases || n_phase < 1 || n_phase > MAX_PHASES || !(omega_vol > 0))
        return fail(ctx, ROM_E_ARG, "rom_load_cubature: bad arguments");
    if (ctx->has_basis && m != ctx->m) return fail(ctx, ROM_E_ARG, "rom_load_cubature: m=%d differs from basis m=%d", m, ctx->m);
    for (int i = 0; i < m; ++i) {
        if (!(w[i] > 0) || !std::isfinite(w[i])) return fail(ctx, ROM_E_ARG, "rom_load_cubature: weight %d not positive", i);
        if (phase[i] < 0 || phase[i] >= n_phase) return fail(ctx, ROM_E_ARG, "rom_load_cubature: phase index %d out of range", i);
    }
    PhaseD ph[MAX_PHASES];
    for (int k = 0; k < n_phase; ++k) {
        const rom_phase &q = phases[k];
        if (!(q.E > 0) || !(q.nu > -1 && q.nu < 0.5) || !(q.s0 > 0) || (q.hard_law != 0 && q.hard_law != 1))
            return fail(ctx, ROM_E_ARG, "rom_load_cubature: bad phase %d", k);
        ph[k].E = q.E; ph[k].nu = q.nu; ph[k].s0 = q.s0; ph[k].k = q.H_or_k; ph[k].p = q.p;
        ph[k].law = q.hard_law;
        ph[k].elastic = std::isinf(q.s0) ? 1 : 0;
        ph[k].G = q.E / (2.0 * (1.0 + q.nu));
        ph[k].lam = q.E * q.nu / ((1.0 + q.nu) * (1.0 - 2.0 * q.nu));
        ph[k].Kb = ph[k].lam + 2.0 * ph[k].G / 3.0;
    }
    CK(cudaSetDevice(ctx->device));
    void *p;
    p = ctx->w; dfree(p); ctx->w = nullptr;
    p = ctx->phase; dfree(p); ctx->phase = nullptr;
    rom_status s;
    if ((s = dalloc(ctx, (void **)&ctx->w, (size_t)m * 8)) != ROM_OK) return s;
    if ((s = dalloc(ctx, (void **)&ctx->phase, (size_t)m * 4)) != ROM_OK) return s;
    CK(cudaMemcpy(ctx->w, w, (size_t)m * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->phase, phase, (size_t)m * 4, cudaMemcpyHostToDevice));
    set_phases(ph, n_phase, ctx->stream);
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->m = m;
    ctx->nphase = n_phase;
    ctx->omega = omega_vol;
    ctx->has_cub = true;
    ctx->geo_ok = false;
    return ROM_OK;
}

rom_status rom_set_geometry(rom_ctx *ctx, int64_t B, int n_par, const double *Gmu, const double *mu) {
    if (!ctx) return ROM_E_ARG;
    if (!ctx->has_basis && !ctx->has_cub) return fail(ctx, ROM_E_STATE, "rom_set_geometry before basis/cubature");
    if (B < 1 || n_par < 1 || n_par > MAX_NPAR || !Gmu || !mu) return fail(ctx, ROM_E_ARG, "rom_set_geometry: bad arguments");
    const int d = ctx->dim, d2 = d * d, m = ctx->m;
    // det F_mu > 0 at every point of every instance (Eq. weakform-dep-mapped needs |det F_mu| > 0)
    for (int64_t b = 0; b < B; ++b)
        for (int i = 0; i < m; ++i) {
            double F[9] = {0};
            for (int a = 0; a < d; ++a)
                for (int r = 0; r < d; ++r) {
                    double s = (a == r) ? 1.0 : 0.0;
                    for (int k = 0; k < n_par; ++k) s += mu[b * n_par + k] * Gmu[((size_t)i * d2 + a * d + r) * n_par + k];
                    F[a * 3 + r] = s;
                }
            if (d == 2) F[8] = 1.0;
            const double det = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                               F[2] * (F[3] * F[7] - F[4] * F[6]);
            if (!(det > 0) || !std::isfinite(det))
                return fail(ctx, ROM_E_ARG, "rom_set_geometry: det F_mu = %g <= 0 at instance %lld point %d", det,
                            (long long)b, i);
        }
    CK(cudaSetDevice(ctx->device));
    std::vector<double> gt((size_t)d2 * n_par * m);
    for (int i = 0; i < m; ++i)
        for (int c = 0; c < d2; ++c)
            for (int k = 0; k < n_par; ++k) gt[((size_t)c * n_par + k) * m + i] = Gmu[((size_t)i * d2 + c) * n_par + k];
    void *p;
    p = ctx->Gmu_T; dfree(p); ctx->Gmu_T = nullptr;
    p = ctx->mu; dfree(p); ctx->mu = nullptr;
    rom_status s;
    if ((s = dalloc(ctx, (void **)&ctx->Gmu_T, gt.size() * 8)) != ROM_OK) return s;
    if ((s = dalloc(ctx, (void **)&ctx->mu, (size_t)B * n_par * 8)) != ROM_OK) return s;
    CK(cudaMemcpy(ctx->Gmu_T, gt.data(), gt.size() * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->mu, mu, (size_t)B * n_par * 8, cudaMemcpyHostToDevice));
    ctx->B = B;
    ctx->n_par = n_par;
    ctx->has_geom = true;
    ctx->geo_ok = false;
    ++ctx->graph_epoch;     // captured step graphs hold the coefficient array
    return ROM_OK;
}

rom_status rom_set_geometry_aux(rom_ctx *ctx, int64_t B, const rom_aux_model *aux, const double *mu) {
    if (!ctx) return ROM_E_ARG;
    if (!ctx->has_basis && !ctx->has_cub) return fail(ctx, ROM_E_STATE, "rom_set_geometry_aux before basis/cubature");
    if (B < 1 || !aux || !mu || !aux->mu_ref || !aux->Ahat || !aux->Mdeim || !aux->S || !aux->GL || !aux->Gpsi)
        return fail(ctx, ROM_E_ARG, "rom_set_geometry_aux: bad arguments");
    const int np = aux->n_p, nr = aux->n_rb, nd = aux->n_deim, nc = np + nr;
    if (np < 1 || np > aux_max() || nr < 1 || nr > aux_max() || nd < 1 || nd > 4 * aux_max() || nc > MAX_NPAR)
        return fail(ctx, ROM_E_ARG, "rom_set_geometry_aux: sizes n_p=%d n_rb=%d n_deim=%d out of range", np, nr, nd);
    for (int k = 0; k < np; ++k)
        if (!(aux->mu_ref[k] > 0) || !std::isfinite(aux->mu_ref[k]))
            return fail(ctx, ROM_E_ARG, "rom_set_geometry_aux: mu_ref[%d] must be positive", k);
    const int d = ctx->dim, d2 = d * d, m = ctx->m;
    CK(cudaSetDevice(ctx->device));
    // Gmu = [grad L_k, grad psi_j] in the kernels' layout [d2][nc][m]
    std::vector<double> gt((size_t)d2 * nc * m);
    for (int i = 0; i < m; ++i)
        for (int c = 0; c < d2; ++c) {
            for (int k = 0; k < np; ++k) gt[((size_t)c * nc + k) * m + i] = aux->GL[((size_t)i * d2 + c) * np + k];
            for (int j = 0; j < nr; ++j) gt[((size_t)c * nc + np + j) * m + i] = aux->Gpsi[((size_t)i * d2 + c) * nr + j];
        }
    // small operators and the parameters in one staging buffer: mu_ref | Ahat | Mdeim | S | mu
    const size_t n_small = (size_t)np + (size_t)nr * nr + (size_t)nr * nd + (size_t)nd * np;
    std::vector<double> sm(n_small);
    size_t o = 0;
    for (int k = 0; k < np; ++k) sm[o++] = aux->mu_ref[k];
    for (int e = 0; e < nr * nr; ++e) sm[o++] = aux->Ahat[e];
    for (int e = 0; e < nr * nd; ++e) sm[o++] = aux->Mdeim[e];
    for (int e = 0; e < nd * np; ++e) sm[o++] = aux->S[e];
    void *p;
    p = ctx->Gmu_T; dfree(p); ctx->Gmu_T = nullptr;
    p = ctx->mu; dfree(p); ctx->mu = nullptr;
    ctx->has_geom = false;
    ctx->geo_ok = false;
    ++ctx->graph_epoch;
    rom_status s;
    double *work = nullptr;       // small operators, then mu [B][np]
    unsigned long long *flags = nullptr;   // [0] first bad point, [1] singular A_hat (as int)
    if ((s = dalloc(ctx, (void **)&ctx->Gmu_T, gt.size() * 8)) != ROM_OK) return s;
    if ((s = dalloc(ctx, (void **)&ctx->mu, (size_t)B * nc * 8)) != ROM_OK) return s;
    if ((s = dalloc(ctx, (void **)&work, (n_small + (size_t)B * np) * 8)) != ROM_OK) return s;
    if ((s = dalloc(ctx, (void **)&flags, 16)) != ROM_OK) { p = work; dfree(p); return s; }
    auto release = [&] { void *q = work; dfree(q); q = flags; dfree(q); };
    const unsigned long long none = (unsigned long long)B * (unsigned long long)m;
    unsigned long long hflags[2] = {none, 0ull};
    cudaError_t e = cudaMemcpy(ctx->Gmu_T, gt.data(), gt.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(work, sm.data(), n_small * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(work + n_small, mu, (size_t)B * np * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(flags, hflags, 16, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { release(); return fail(ctx, ROM_E_CUDA, "rom_set_geometry_aux: %s", cudaGetErrorString(e)); }
    const double *d_ref = work, *d_A = d_ref + np, *d_M = d_A + (size_t)nr * nr, *d_S = d_M + (size_t)nr * nd;
    launch_aux_geometry(np, nr, nd, d_ref, d_A, d_M, d_S, B, work + n_small, ctx->mu,
                        reinterpret_cast<int *>(flags + 1), ctx->stream);
    launch_geom_check(d, m, nc, B, ctx->mu, ctx->Gmu_T, flags, ctx->stream);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hflags, flags, 16, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    release();
    if (e != cudaSuccess) return fail(ctx, ROM_E_CUDA, "rom_set_geometry_aux: %s", cudaGetErrorString(e));
    if ((hflags[1] & 0xffffffffull) != 0) return fail(ctx, ROM_E_ARG, "rom_set_geometry_aux: singular reduced operator A_hat");
    if (hflags[0] < none)
        return fail(ctx, ROM_E_ARG, "rom_set_geometry_aux: det F_mu <= 0 at instance %lld point %d",
                    (long long)(hflags[0] / (unsigned long long)m), (int)(hflags[0] % (unsigned long long)m));
    ctx->B = B;
    ctx->n_par = nc;
    ctx->has_geom = true;
    return ROM_OK;
}

rom_status rom_state_create(rom_ctx *ctx, int64_t B, rom_state **out) {
    if (!ctx || !out) return ROM_E_ARG;
    *out = nullptr;
    if (!ctx->has_basis || !ctx->has_cub) return fail(ctx, ROM_E_STATE, "rom_state_create before basis/cubature");
    if (B < 1 || B > (int64_t)1 << 30) return fail(ctx, ROM_E_ARG, "rom_state_create: bad B");
    CK(cudaSetDevice(ctx->device));
    rom_state *st = new (std::nothrow) rom_state();
    if (!st) return fail(ctx, ROM_E_NOMEM, "host allocation");
    st->ctx = ctx;
    st->B = B;
    st->n = ctx->n;
    st->m = ctx->m;
    st->d = ctx->dim;
    const int d2 = ctx->dim * ctx->dim, n = ctx->n, m = ctx->m;
    const int ncp = ctx->dim == 2 ? 4 : 6;
    Batch &bt = st->bt;
    bt.B = B;
    auto A = [&](void **p, size_t bytes) -> rom_status {
        rom_status s = dalloc(ctx, p, bytes);
        if (s == ROM_OK) st->allocs.push_back(*p);
        return s;
    };
    rom_status s = ROM_OK;
    const size_t Bz = (size_t)B;
    if ((s = A((void **)&bt.q_n, Bz * n * 8)) || (s = A((void **)&bt.dq_prev, Bz * n * 8)) ||
        (s = A((void **)&bt.cp, Bz * ncp * m * 8)) || (s = A((void **)&bt.xi, Bz * m * 8)) ||
        (s = A((void **)&bt.q_trial, Bz * n * 8)) || (s = A((void **)&bt.q_acc, Bz * n * 8)) ||
        (s = A((void **)&bt.dq, Bz * n * 8)) || (s = A((void **)&bt.ctl, Bz * sizeof(Ctl))) ||
        (s = A((void **)&bt.list, Bz * 4)) || (s = A((void **)&st->list2, Bz * 4)) ||
        (s = A((void **)&bt.counts, 64)) || (s = A((void **)&bt.v, Bz * d2 * m * 8)) ||
        (s = A((void **)&bt.wP, Bz * d2 * m * 8)) || (s = A((void **)&bt.At, Bz * d2 * d2 * (size_t)((m + 3) & ~3) * 8)) ||
        (s = A((void **)&bt.cp_tr, Bz * ncp * m * 8)) || (s = A((void **)&bt.xi_tr, Bz * m * 8)) ||
        (s = A((void **)&bt.pl, Bz * m)) || (s = A((void **)&bt.r, Bz * n * 8)) ||
        (s = A((void **)&bt.K, Bz * n * n * 8)) || (s = A((void **)&bt.Bsum, Bz * (n * d2 + d2 * d2) * 8)) ||
        (s = A((void **)&bt.Ubar, Bz * d2 * 8)) ||
        (s = A((void **)&bt.Rbar, Bz * d2 * 8)) || (s = A((void **)&bt.U_prev, Bz * d2 * 8)) ||
        (s = A((void **)&bt.r0_prev, Bz * 8)) ||
        (s = A((void **)&st->io_F, Bz * d2 * 8)) || (s = A((void **)&st->io_P, Bz * d2 * 8)) ||
        (s = A((void **)&st->io_A, Bz * d2 * d2 * 8)) || (s = A(&st->io_info, Bz * sizeof(rom_step_info)))) {
        rom_state_destroy(st);
        return s;
    }
    // virgin state: a = 0, C^p^-1 = I, xi = 0
    std::vector<double> cp(Bz * ncp * m, 0.0);
    const int diag2[4] = {1, 0, 1, 1}, diag3[6] = {1, 0, 0, 1, 0, 1};
    for (size_t b = 0; b < Bz; ++b)
        for (int c = 0; c < ncp; ++c) {
            const double v = ctx->dim == 2 ? diag2[c] : diag3[c];
            for (int i = 0; i < m; ++i) cp[(b * ncp + c) * m + i] = v;
        }
    std::vector<double> eye(Bz * d2, 0.0);
    for (size_t b = 0; b < Bz; ++b)
        for (int a = 0; a < ctx->dim; ++a) eye[b * d2 + a * ctx->dim + a] = 1.0;
    const std::vector<double> inf(Bz, INFINITY);
    cudaError_t e;
    if ((e = cudaMemcpy(bt.U_prev, eye.data(), eye.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(bt.r0_prev, inf.data(), Bz * 8, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(bt.q_n, 0, Bz * n * 8)) != cudaSuccess || (e = cudaMemset(bt.dq_prev, 0, Bz * n * 8)) != cudaSuccess ||
        (e = cudaMemset(bt.xi, 0, Bz * m * 8)) != cudaSuccess ||
        (e = cudaMemcpy(bt.cp, cp.data(), cp.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess) {
        rom_state_destroy(st);
        return fail(ctx, ROM_E_CUDA, "rom_state_create: %s", cudaGetErrorString(e));
    }
    *out = st;
    return ROM_OK;
}

rom_status rom_state_destroy(rom_state *st) {
    if (!st) return ROM_E_ARG;
    if (st->ctx) cudaSetDevice(st->ctx->device);
    if (st->gexec) cudaGraphExecDestroy(st->gexec);
    if (st->gstream) cudaStreamDestroy(st->gstream);
    for (void *p : st->allocs) cudaFree(p);
    delete st;
    return ROM_OK;
}

rom_status rom_state_export(rom_ctx *ctx, const rom_state *st, double *a, double *Cpinv, double *xi) {
    if (!ctx || !st || st->ctx != ctx) return ROM_E_ARG;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    const int n = st->n, m = st->m, ncp = st->d == 2 ? 4 : 6;
    const size_t B = (size_t)st->B;
    if (a) CK(cudaMemcpy(a, st->bt.q_n, B * n * 8, cudaMemcpyDeviceToHost));
    if (xi) CK(cudaMemcpy(xi, st->bt.xi, B * m * 8, cudaMemcpyDeviceToHost));
    if (Cpinv) {
        std::vector<double> t(B * ncp * m);
        CK(cudaMemcpy(t.data(), st->bt.cp, t.size() * 8, cudaMemcpyDeviceToHost));
        for (size_t b = 0; b < B; ++b)
            for (int c = 0; c < ncp; ++c)
                for (int i = 0; i < m; ++i) Cpinv[(b * m + i) * ncp + c] = t[(b * ncp + c) * m + i];
    }
    return ROM_OK;
}

rom_status rom_state_import(rom_ctx *ctx, rom_state *st, const double *a, const double *Cpinv, const double *xi) {
    if (!ctx || !st || st->ctx != ctx) return ROM_E_ARG;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    const int n = st->n, m = st->m, ncp = st->d == 2 ? 4 : 6;
    const size_t B = (size_t)st->B;
    if (a) {
        CK(cudaMemcpy(st->bt.q_n, a, B * n * 8, cudaMemcpyHostToDevice));
        CK(cudaMemset(st->bt.dq_prev, 0, B * n * 8));
        const std::vector<double> inf(B, INFINITY);
        CK(cudaMemcpy(st->bt.r0_prev, inf.data(), B * 8, cudaMemcpyHostToDevice));
    }
    if (xi) CK(cudaMemcpy(st->bt.xi, xi, B * m * 8, cudaMemcpyHostToDevice));
    if (Cpinv) {
        std::vector<double> t(B * ncp * m);
        for (size_t b = 0; b < B; ++b)
            for (int c = 0; c < ncp; ++c)
                for (int i = 0; i < m; ++i) t[(b * ncp + c) * m + i] = Cpinv[(b * m + i) * ncp + c];
        CK(cudaMemcpy(st->bt.cp, t.data(), t.size() * 8, cudaMemcpyHostToDevice));
    }
    return ROM_OK;
}

static rom_status ensure_geo(rom_ctx *ctx);

static rom_status check_step(rom_ctx *ctx, rom_state *st, const rom_opts *opts) {
    if (!ctx || !st || !opts || st->ctx != ctx) return ROM_E_ARG;
    if (!ctx->has_basis || !ctx->has_cub || !ctx->has_geom) return fail(ctx, ROM_E_STATE, "rom_step before basis/cubature/geometry");
    if (st->B != ctx->B) return fail(ctx, ROM_E_STATE, "rom_step: state has B=%lld but geometry B=%lld", (long long)st->B, (long long)ctx->B);
    if (st->n != ctx->n || st->m != ctx->m) return fail(ctx, ROM_E_STATE, "rom_step: state built for another model");
    if (!(opts->tol_rel >= 0) || !(opts->tol_abs >= 0) || opts->max_iter < 0 || opts->max_iter > 1000 ||
        opts->max_ls < 0 || opts->max_ls > 60 || opts->precision < 0 || opts->precision > 3 || opts->start < 0 ||
        opts->start > 2)
        return fail(ctx, ROM_E_ARG, "rom_step: bad options");
    if (opts->start == ROM_START_MLP && (!ctx->has_mlp || !ctx->mlp_norm))
        return fail(ctx, ROM_E_STATE, "rom_step: learned start requested but no MLP (rom_mlp_init, rom_mlp_params, rom_mlp_norm)");
    if (opts->start == ROM_START_MLP && ctx->mlp.n_in != ctx->dim * ctx->dim + ctx->n_par + 2 * ctx->n + 2)
        return fail(ctx, ROM_E_STATE, "rom_step: MLP input size %d does not match d^2 + n_par + 2n + 2", ctx->mlp.n_in);
    if (opts->precision >= ROM_PREC_TF32 && !ctx->tc_img[0] && !ctx->tc3_img)
        return fail(ctx, ROM_E_ARG, "rom_step: tensor-core precision needs n <= 64 (n = %d)", ctx->n);
    return ensure_geo(ctx);
}

static Model make_model(const rom_ctx *ctx) {
    Model M;
    M.d = ctx->dim; M.d2 = ctx->dim * ctx->dim; M.n = ctx->n; M.m = ctx->m; M.n_par = ctx->n_par;
    M.nphase = ctx->nphase; M.ncp = ctx->dim == 2 ? 4 : 6;
    M.mA = (ctx->m + 3) & ~3;
    M.G_pt = ctx->G_pt; M.G_T = ctx->G_T; M.G32_pt = ctx->G32; M.w = ctx->w; M.phase = ctx->phase;
    M.G32h_T = ctx->G32h_T; M.G32l_T = ctx->G32l_T; M.Gdf = ctx->Gdf;
    M.Gmu_T = ctx->Gmu_T; M.omega = ctx->omega;
    return M;
}

// the per-geometry cache (F_mu^-1 and w J per point); the cache belongs to the geometry, so a new
// one is built (and captured graphs re-recorded, graph_epoch) when the model or geometry changed
static rom_status ensure_geo(rom_ctx *ctx) {
    if (ctx->geo_ok) return ROM_OK;
    void *p = ctx->geo;
    dfree(p);
    ctx->geo = nullptr;
    CK(cudaSetDevice(ctx->device));
    rom_status s;
    if ((s = dalloc(ctx, (void **)&ctx->geo, (size_t)ctx->B * (ctx->dim * ctx->dim + 1) * ctx->m * 8)) != ROM_OK)
        return s;
    launch_geometry(make_model(ctx), ctx->mu, ctx->B, ctx->geo, ctx->stream);
    CK(cudaGetLastError());
    ctx->geo_ok = true;
    ++ctx->graph_epoch;
    return ROM_OK;
}

}  // extern "C"

static rom_status ensure_feat(rom_ctx *ctx, int64_t B) {
    if (ctx->feat_B >= B) return ROM_OK;
    ++ctx->graph_epoch;
    void *p;
    p = ctx->d_feat; dfree(p); ctx->d_feat = nullptr;
    p = ctx->d_pred; dfree(p); ctx->d_pred = nullptr;
    rom_status s;
    if ((s = dalloc(ctx, (void **)&ctx->d_feat, (size_t)B * ctx->mlp.n_in * 4)) != ROM_OK) return s;
    if ((s = dalloc(ctx, (void **)&ctx->d_pred, (size_t)B * ctx->mlp.n_out * 8)) != ROM_OK) return s;
    ctx->feat_B = B;
    return ROM_OK;
}

static int prof_event(rom_ctx *ctx, int idx) {
    while ((int)ctx->ev_pool.size() <= idx) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        ctx->ev_pool.push_back(e);
    }
    cudaEventRecord(ctx->ev_pool[idx], ctx->stream);
    return idx;
}

// launch one kernel group `kid` (0 start, 1 constitutive, 2 assemble, 3 solve, 4 finalize, 5 advance,
// 6 learned start, 7 force) of `launches` kernels with optional event timing and an algorithmic
// FLOP count for the roofline
template <typename F>
static int timed(rom_ctx *ctx, int kid, double flops, F &&launch, int launches = 1) {
    int e0 = -1;
    if (ctx->prof) e0 = prof_event(ctx, (int)ctx->recs.size() * 2);
    const int r = launch();
    if (ctx->prof && e0 >= 0) {
        const int e1 = prof_event(ctx, e0 + 1);
        ctx->recs.push_back({kid, e0, e1, flops, launches});
    }
    return r;
}

static void prof_collect(rom_ctx *ctx) {
    if (!ctx->prof || ctx->recs.empty()) return;
    cudaStreamSynchronize(ctx->stream);
    for (const auto &r : ctx->recs) {
        float ms = 0.f;
        if (r.ev1 >= 0 && cudaEventElapsedTime(&ms, ctx->ev_pool[r.ev0], ctx->ev_pool[r.ev1]) == cudaSuccess) {
            ctx->prof_ms[r.kid] += ms;
            ctx->prof_launches[r.kid] += r.launches;
            ctx->prof_flops[r.kid] += r.flops;
        }
    }
    ctx->recs.clear();
}

// the effective-stiffness sums of the converged instances on the tensor cores (3D: k_abar_tc3,
// 2D: k_abar_tcp), for the tensor-core paths of models with n <= 64
static bool tc_sums_path(const rom_ctx *ctx, const Model &M) {
    return M.n_par <= MAX_NPAR && ((M.d == 3 && ctx->tc3_img) || (M.d == 2 && ctx->tc_img[1]));
}
static int launch_abar_sums(const rom_ctx *ctx, const Model &M, Batch bc, double *Bsum, cudaStream_t s) {
    return M.d == 3 ? launch_abar_tc3(M, bc, ctx->tc3_img, Bsum, ctx->d_err, s)
                    : launch_abar_tcp(M, bc, ctx->tc_img[1], Bsum, ctx->d_err, s);
}

// the stiffness K runs on the tensor cores (and the residual in its own kernel, launch_force)
// for models with n <= 64 at every precision but FP64
static bool tc_path(const rom_ctx *ctx, const Model &M, int precision) {
    return precision >= 1 && ((M.d == 3 && ctx->tc3_img) || (M.d == 2 && ctx->tc_img[1]));
}

// K of the active list on the tensor cores (n <= 64): BF16, TF32, or the FP32-accurate TF32 split
// for precision fp32; in BF16 and TF32 the instances that the solve flagged for an accurate
// stiffness get the split assembly.  3D: k_assemble_tc3 / tc4; 2D: k_assemble_tcp with the
// instances packed along M.  FP64 (and n > 64) use the SIMT kernel, which can also produce the
// residual r
static int launch_assembly(rom_ctx *ctx, const Model &M, Batch bt, const StepOpts &o, int32_t *nxt, cudaStream_t s) {
    if (M.d == 3 && ctx->tc3_img && o.precision >= 1) {
        if (o.precision == 1) return launch_tc3(3, M, bt, ctx->tc3_img, ctx->d_err, 0, s);
        const int r = launch_tc3(o.precision == 3 ? 1 : 4, M, bt, ctx->tc3_img, ctx->d_err, 1, s);
        return r ? r : launch_tc3(3, M, bt, ctx->tc3_img, ctx->d_err, 2, s);
    }
    if (M.d == 2 && ctx->tc_img[1] && o.precision >= 1) {
        if (o.precision == 1) return launch_tc2(3, M, bt, ctx->tc_img[1], ctx->d_err, 0, s);
        const int r = o.precision == 3 ? launch_tc2(1, M, bt, ctx->tc_img[0], ctx->d_err, 1, s)
                                       : launch_tc2(2, M, bt, ctx->tc_img[1], ctx->d_err, 1, s);
        return r ? r : launch_tc2(3, M, bt, ctx->tc_img[1], ctx->d_err, 2, s);
    }
    if (o.precision >= 2) return -1;
    return launch_kernel(2, M, bt, o, nxt, s);
}

// the effective stiffness needs K at FP32 accuracy: after a BF16/TF32 solve, the FP32-accurate
// assembly of the converged instances (list rebuilt by launch_list_converged) whose last pass
// assembled a low-precision K.  An instance with the accurate-stiffness flag got the accurate K in
// its last pass (escalated by the solve, or flagged by k_flag_final in the pass that converged
// it); the tensor-core kernels select the others (sel 1).  The residual is not needed here.
static int launch_abar_assembly(rom_ctx *ctx, const Model &M, Batch bc, const StepOpts &o, int32_t *nxt,
                                cudaStream_t s) {
    if (M.d == 3 && ctx->tc3_img) return launch_tc3(3, M, bc, ctx->tc3_img, ctx->d_err, 1, s);
    if (M.d == 2 && ctx->tc_img[1]) return launch_tc2(3, M, bc, ctx->tc_img[1], ctx->d_err, 1, s);
    StepOpts o32 = o;
    o32.precision = 1;
    return launch_assembly(ctx, M, bc, o32, nxt, s);
}

// BF16/TF32 stiffness on the tensor cores with Abar wanted: each Newton pass forms the residual
// first, flags the instances that this pass converges for the accurate assembly and groups them
// (launch_flag_final), then assembles
static bool final_pass_flags(const rom_ctx *ctx, const Model &M, const StepOpts &o) {
    return o.precision >= 2 && o.want_abar && tc_path(ctx, M, o.precision);
}

static rom_status run_step(rom_ctx *ctx, rom_state *st, const rom_opts *opts, const double *Fbar_d, double *Pbar_d,
                           double *Abar_d, void *info_d) {
    st->last_prec = opts->precision;
    StepOpts o;
    o.tol_rel = opts->tol_rel; o.tol_abs = opts->tol_abs; o.max_iter = opts->max_iter; o.max_ls = opts->max_ls;
    o.precision = opts->precision; o.start = opts->start; o.polar = opts->polar_split; o.want_abar = opts->want_abar;
    o.fp64_residual = opts->fp64_residual;
    o.asm_tm = ctx->asm_tm; o.asm_ch = ctx->asm_ch;
    const Model M = make_model(ctx);
    Batch bt = st->bt;
    bt.mu = ctx->mu;
    bt.geo = ctx->geo;
    bt.err = ctx->d_err;
    int32_t *lists[2] = {st->bt.list, st->list2};
    const double n = M.n, m = M.m, d2 = M.d2, d4 = d2 * d2;
    // algorithmic FLOPs per active instance: kinematics and force 2 m d2 n each; Y = At G: 2 m d4 n;
    // K: 2 m d2 n^2 on the tensor cores (full product), m d2 n (n + 1) on the CUDA cores (upper
    // triangle; the SIMT kernel also forms the force); LU + solve: 2 n^3 / 3 + 2 n^2
    const bool tcp = tc_path(ctx, M, o.precision);
    // the residual in its own kernel: always on the tensor-core paths, and on the mixed CUDA-core
    // path when it is formed in double-float arithmetic
    const bool sepf = tcp || separate_force(M, o);
    const double fl_asm = tcp ? 2 * m * d4 * n + 2 * m * d2 * n * n
                              : 2 * m * d4 * n + m * d2 * n * (n + 1) + (sepf ? 0.0 : 2 * m * d2 * n);
    const double fl_kin = 2 * m * d2 * n;
    const double fl_lu = 2 * n * n * n / 3 + 2 * n * n;
    if (ctx->d_err) CK(cudaMemsetAsync(ctx->d_err, 0, 4, ctx->stream));   // tensor-core error flag of this step
    if (timed(ctx, 0, 0.0, [&] { return launch_start(M, bt, Fbar_d, o, nullptr, ctx->stream); }, 2))
        return fail(ctx, ROM_E_ARG, "launch_start");
    if (o.start == ROM_START_MLP) {
        rom_status s2 = ensure_feat(ctx, st->B);
        if (s2 != ROM_OK) return s2;
        timed(ctx, 6, 0.0, [&] {
            launch_features(M, bt, bt.U_prev, ctx->d_feat, ctx->mlp.n_in, ctx->stream);
            mlp_predict(ctx->mlp, ctx->d_feat, st->B, 1, ctx->d_pred, ctx->stream, ctx->d_err);
            launch_add_pred(bt, M.n, ctx->d_pred, ctx->stream);
            return 0;
        }, 3 + 2 * ctx->mlp.L);
    }
    const int max_pass = (opts->max_iter + 1) * (opts->max_ls + 1) + 2;
    const bool fin = final_pass_flags(ctx, M, o);
    int64_t n_act = st->B;
    for (int pass = 0; pass < max_pass; ++pass) {
        bt.list = lists[pass & 1];
        int32_t *nxt = lists[(pass + 1) & 1];
        const double na = (double)n_act;
        auto asm_launch = [&] { return launch_assembly(ctx, M, bt, o, nxt, ctx->stream); };
        auto force_launch = [&] {
            if (sepf) launch_force(M, bt, o.fp64_residual != 0, ctx->stream);
            return 0;
        };
        const int asm_n = (tcp && o.precision >= 2) ? 2 : 1;
        bool bad = timed(ctx, 1, na * fl_kin, [&] { return launch_kernel(1, M, bt, o, nxt, ctx->stream); }) != 0;
        if (fin)
            bad = bad || (sepf && timed(ctx, 7, na * fl_kin, force_launch)) ||
                  timed(ctx, 5, 0.0, [&] { launch_flag_final(M, bt, o, nxt, ctx->stream); return 0; }, 2) ||
                  timed(ctx, 2, na * fl_asm, asm_launch, asm_n);
        else
            bad = bad || timed(ctx, 2, na * fl_asm, asm_launch, asm_n) ||
                  (sepf && timed(ctx, 7, na * fl_kin, force_launch));
        if (bad || timed(ctx, 3, na * fl_lu, [&] { return launch_kernel(3, M, bt, o, nxt, ctx->stream); }) ||
            timed(ctx, 5, 0.0, [&] { return launch_kernel(5, M, bt, o, nxt, ctx->stream); }))
            return fail(ctx, ROM_E_ARG, "rom_step: basis size n=%d not supported by the assembly kernel", M.n);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(ctx->h_count, bt.counts, 4, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        n_act = ctx->h_count[0];
        if (n_act == 0) break;
    }
    // tensor-core paths: the sums B = sum_i G_i^T Ahat_i and A0 of the effective stiffness on the
    // tensor cores as well (over the converged instances); the finalize then reads them
    const bool tc_sums = tcp && tc_sums_path(ctx, M) && o.want_abar;
    if (tcp) {
        if ((o.precision >= 2 && o.want_abar) || tc_sums) {
            Batch bc = bt;
            bc.list = lists[0];
            launch_list_converged(bc, ctx->stream);
            if (o.precision >= 2)
                timed(ctx, 2, 0.0, [&] { return launch_abar_assembly(ctx, M, bc, o, lists[1], ctx->stream); });
            if (tc_sums && timed(ctx, 4, 0.0, [&] { return launch_abar_sums(ctx, M, bc, st->bt.Bsum, ctx->stream); }))
                return fail(ctx, ROM_E_ARG, "rom_step: tensor-core Abar sums not available for this model");
        }
        CK(cudaMemcpyAsync(ctx->h_count + 4, ctx->d_err, 4, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        if (ctx->h_count[4]) {
            cudaMemsetAsync(ctx->d_err, 0, 4, ctx->stream);
            return fail(ctx, ROM_E_CUDA, "rom_step: tensor-core pipeline wait timed out");
        }
    }
    Batch bf = bt;
    bf.Bsum = tc_sums ? st->bt.Bsum : nullptr;
    if (timed(ctx, 4, 0.0, [&] { return launch_finalize(M, bf, o, Pbar_d, Abar_d, info_d, ctx->stream); }))
        return fail(ctx, ROM_E_ARG, "rom_step: n*d*d too large for the finalize kernel");
    CK(cudaGetLastError());
    prof_collect(ctx);
    return ROM_OK;
}

static bool same_opts(const rom_opts &a, const rom_opts &b) {   // field by field: the struct has tail padding
    return a.tol_rel == b.tol_rel && a.tol_abs == b.tol_abs && a.max_iter == b.max_iter && a.max_ls == b.max_ls &&
           a.precision == b.precision && a.start == b.start && a.polar_split == b.polar_split &&
           a.want_abar == b.want_abar && a.fp64_residual == b.fp64_residual;
}
static bool o_needs_recapture(const rom_state *st, const rom_opts *opts) {
    return !st->g_valid || !same_opts(st->gopts, *opts) || st->g_epoch != st->ctx->graph_epoch;
}

// Capture one load step into a CUDA graph whose Newton passes run inside a conditional WHILE
// node: the device decides how many passes to run (no host round trip per pass).  The graph
// reads Fbar from and writes Pbar / Abar / info to buffers owned by the state, so one
// instantiation serves every later step with the same options.
// Record the launches of one load step (start, learned start, the WHILE node over the Newton
// passes, the FP32-accurate Abar assembly, finalize) on `cs`, which must be capturing.  Returns
// a CUDA error (cudaSuccess if recorded) and sets *bad if a launch configuration was refused.
static cudaError_t record_step(rom_ctx *ctx, rom_state *st, const rom_opts *opts, cudaStream_t cs, int *bad_out) {
    StepOpts o;
    o.tol_rel = opts->tol_rel; o.tol_abs = opts->tol_abs; o.max_iter = opts->max_iter; o.max_ls = opts->max_ls;
    o.precision = opts->precision; o.start = opts->start; o.polar = opts->polar_split; o.want_abar = opts->want_abar;
    o.fp64_residual = opts->fp64_residual;
    o.asm_tm = ctx->asm_tm; o.asm_ch = ctx->asm_ch;
    const Model M = make_model(ctx);
    Batch bt = st->bt;
    bt.mu = ctx->mu;
    bt.geo = ctx->geo;
    bt.err = ctx->d_err;
    const int max_pass = (opts->max_iter + 1) * (opts->max_ls + 1) + 2;
    int bad = 0;
    if (ctx->d_err) cudaMemsetAsync(ctx->d_err, 0, 4, cs);   // tensor-core error flag of this step
    bad |= launch_start(M, bt, st->io_F, o, nullptr, cs);
    launch_reset_pass(bt, cs);
    if (o.start == ROM_START_MLP) {
        launch_features(M, bt, bt.U_prev, ctx->d_feat, ctx->mlp.n_in, cs);
        mlp_predict(ctx->mlp, ctx->d_feat, st->B, 1, ctx->d_pred, cs, ctx->d_err);
        launch_add_pred(bt, M.n, ctx->d_pred, cs);
    }
    // conditional WHILE node for the Newton passes
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cg, &deps, nullptr, &ndeps);
    cudaGraphConditionalHandle h{};
    cudaGraphNode_t wnode{};
    cudaGraph_t body = nullptr;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, cg, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&wnode, cg, deps, nullptr, ndeps, &cp);
        if (e == cudaSuccess) body = cp.conditional.phGraph_out[0];
    }
    if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) {
        cudaStream_t bs = nullptr;
        e = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            int32_t *nxt = st->list2;
            const bool sepf = tc_path(ctx, M, o.precision) || separate_force(M, o);
            bad |= launch_kernel(1, M, bt, o, nxt, bs);
            if (final_pass_flags(ctx, M, o)) {
                launch_force(M, bt, o.fp64_residual != 0, bs);
                launch_flag_final(M, bt, o, nxt, bs);
                bad |= launch_assembly(ctx, M, bt, o, nxt, bs);
            } else {
                bad |= launch_assembly(ctx, M, bt, o, nxt, bs);
                if (sepf) launch_force(M, bt, o.fp64_residual != 0, bs);
            }
            bad |= launch_kernel(3, M, bt, o, nxt, bs);
            launch_graph_advance(bt, nxt, h, max_pass, bs);
            cudaGraph_t out = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(bs, &out);
            if (e == cudaSuccess) e = e2;
        }
        if (bs) cudaStreamDestroy(bs);
    }
    const bool tc_sums = tc_path(ctx, M, o.precision) && tc_sums_path(ctx, M) && o.want_abar;
    if (e == cudaSuccess && ((o.precision >= 2 && o.want_abar) || tc_sums)) {
        Batch bc = bt;
        launch_list_converged(bc, cs);
        if (o.precision >= 2) bad |= launch_abar_assembly(ctx, M, bc, o, st->list2, cs);
        if (tc_sums) bad |= launch_abar_sums(ctx, M, bc, st->bt.Bsum, cs);
    }
    Batch bf = bt;
    bf.Bsum = tc_sums ? st->bt.Bsum : nullptr;
    if (e == cudaSuccess) bad |= launch_finalize(M, bf, o, st->io_P, st->io_A, st->io_info, cs);
    *bad_out = bad;
    return e;
}

static rom_status capture_step(rom_ctx *ctx, rom_state *st, const rom_opts *opts) {
    if (st->gexec) { cudaGraphExecDestroy(st->gexec); st->gexec = nullptr; }
    st->g_valid = false;
    if (!st->gstream) CK(cudaStreamCreateWithFlags(&st->gstream, cudaStreamNonBlocking));
    cudaStream_t cs = st->gstream;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int bad = 0;
    cudaError_t e = record_step(ctx, st, opts, cs, &bad);
    cudaError_t e3 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e3;
    if (e != cudaSuccess || bad) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(ctx, ROM_E_CUDA, "rom_step: graph capture failed: %s", e != cudaSuccess ? cudaGetErrorString(e) : "launch configuration");
    }
    e = cudaGraphInstantiate(&st->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(ctx, ROM_E_CUDA, "rom_step: graph instantiate failed: %s", cudaGetErrorString(e));
    st->gopts = *opts;
    st->g_valid = true;
    st->g_epoch = ctx->graph_epoch;
    return ROM_OK;
}

static rom_status run_step_graph(rom_ctx *ctx, rom_state *st, const rom_opts *opts, const double *Fbar_d,
                                 double *Pbar_d, double *Abar_d, void *info_d) {
    st->last_prec = opts->precision;
    if (o_needs_recapture(st, opts)) {
        rom_status s = capture_step(ctx, st, opts);
        if (s != ROM_OK) return s;
    }
    const int d2 = ctx->dim * ctx->dim;
    const size_t B = (size_t)st->B;
    CK(cudaMemcpyAsync(st->io_F, Fbar_d, B * d2 * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaGraphLaunch(st->gexec, ctx->stream));
    CK(cudaMemcpyAsync(Pbar_d, st->io_P, B * d2 * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    if (Abar_d && opts->want_abar) CK(cudaMemcpyAsync(Abar_d, st->io_A, B * d2 * d2 * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    if (info_d) CK(cudaMemcpyAsync(info_d, st->io_info, B * sizeof(rom_step_info), cudaMemcpyDeviceToDevice, ctx->stream));
    return ROM_OK;
}

extern "C" {

rom_status rom_step_device(rom_ctx *ctx, rom_state *st, const rom_opts *opts, const double *Fbar_d, double *Pbar_d,
                           double *Abar_d, rom_step_info *info_d) {
    rom_status s = check_step(ctx, st, opts);
    if (s != ROM_OK) return s;
    if (!Fbar_d || !Pbar_d || (opts->want_abar && !Abar_d)) return fail(ctx, ROM_E_ARG, "rom_step_device: null buffer");
    CK(cudaSetDevice(ctx->device));
    if (ctx->graphs && !ctx->prof) {
        if (opts->start == ROM_START_MLP && (s = ensure_feat(ctx, st->B)) != ROM_OK) return s;
        return run_step_graph(ctx, st, opts, Fbar_d, Pbar_d, Abar_d, info_d);
    }
    return run_step(ctx, st, opts, Fbar_d, Pbar_d, Abar_d, info_d);
}

rom_status rom_step(rom_ctx *ctx, rom_state *st, const rom_opts *opts, const double *Fbar, double *Pbar,
                    double *Abar, rom_step_info *info) {
    rom_status s = check_step(ctx, st, opts);
    if (s != ROM_OK) return s;
    if (!Fbar || !Pbar || (opts->want_abar && !Abar)) return fail(ctx, ROM_E_ARG, "rom_step: null buffer");
    CK(cudaSetDevice(ctx->device));
    const int64_t B = st->B;
    const int d2 = ctx->dim * ctx->dim;
    if (ctx->io_B != B) {
        free_io(ctx);
        if ((s = dalloc(ctx, (void **)&ctx->d_Fbar, (size_t)B * d2 * 8)) || (s = dalloc(ctx, (void **)&ctx->d_Pbar, (size_t)B * d2 * 8)) ||
            (s = dalloc(ctx, (void **)&ctx->d_Abar, (size_t)B * d2 * d2 * 8)) ||
            (s = dalloc(ctx, &ctx->d_info, (size_t)B * sizeof(rom_step_info))))
            return s;
        ctx->io_B = B;
    }
    CK(cudaMemcpyAsync(ctx->d_Fbar, Fbar, (size_t)B * d2 * 8, cudaMemcpyHostToDevice, ctx->stream));
    s = run_step(ctx, st, opts, ctx->d_Fbar, ctx->d_Pbar, ctx->d_Abar, ctx->d_info);
    if (s != ROM_OK) return s;
    CK(cudaMemcpyAsync(Pbar, ctx->d_Pbar, (size_t)B * d2 * 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (Abar && opts->want_abar)
        CK(cudaMemcpyAsync(Abar, ctx->d_Abar, (size_t)B * d2 * d2 * 8, cudaMemcpyDeviceToHost, ctx->stream));
    if (info) CK(cudaMemcpyAsync(info, ctx->d_info, (size_t)B * sizeof(rom_step_info), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return ROM_OK;
}

rom_status rom_sync(rom_ctx *ctx) {
    if (!ctx) return ROM_E_ARG;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    return ROM_OK;
}

const char *rom_last_error(const rom_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

rom_status rom_mlp_init(rom_ctx *ctx, int n_in, int width, int depth, int n_out, int64_t max_rows) {
    if (!ctx) return ROM_E_ARG;
    if (n_in < 1 || n_in > 4096 || width < 1 || width > 4096 || depth < 1 || depth > 16 || n_out < 1 ||
        n_out > 4096 || max_rows < 1)
        return fail(ctx, ROM_E_ARG, "rom_mlp_init: bad shape");
    CK(cudaSetDevice(ctx->device));
    if (ctx->has_mlp) mlp_free(ctx->mlp);
    ctx->has_mlp = false;
    ctx->mlp_norm = false;
    if (mlp_alloc(ctx->mlp, n_in, width, depth, n_out, max_rows)) {
        mlp_free(ctx->mlp);
        return fail(ctx, ROM_E_NOMEM, "rom_mlp_init: allocation failed");
    }
    ctx->has_mlp = true;
    return ROM_OK;
}

rom_status rom_mlp_nparams(rom_ctx *ctx, int64_t *n) {
    if (!ctx || !n) return ROM_E_ARG;
    if (!ctx->has_mlp) return fail(ctx, ROM_E_STATE, "rom_mlp_nparams: no MLP");
    *n = ctx->mlp.nparams;
    return ROM_OK;
}

rom_status rom_mlp_params(rom_ctx *ctx, float *get_host, const float *set_host) {
    if (!ctx) return ROM_E_ARG;
    if (!ctx->has_mlp) return fail(ctx, ROM_E_STATE, "rom_mlp_params: no MLP");
    CK(cudaSetDevice(ctx->device));
    if (set_host) mlp_set_params(ctx->mlp, set_host, ctx->stream);
    if (get_host) mlp_get_params(ctx->mlp, get_host, ctx->stream);
    CK(cudaStreamSynchronize(ctx->stream));
    return ROM_OK;
}

rom_status rom_mlp_norm(rom_ctx *ctx, const float *norm_host) {
    if (!ctx || !norm_host) return ROM_E_ARG;
    if (!ctx->has_mlp) return fail(ctx, ROM_E_STATE, "rom_mlp_norm: no MLP");
    const int nn = 2 * ctx->mlp.n_in + 2 * ctx->mlp.n_out;
    for (int k = 0; k < nn; ++k)
        if (!std::isfinite(norm_host[k])) return fail(ctx, ROM_E_ARG, "rom_mlp_norm: non-finite entry");
    for (int k = 0; k < ctx->mlp.n_in; ++k)
        if (!(norm_host[ctx->mlp.n_in + k] > 0)) return fail(ctx, ROM_E_ARG, "rom_mlp_norm: x_std must be > 0");
    for (int k = 0; k < ctx->mlp.n_out; ++k)
        if (!(norm_host[2 * ctx->mlp.n_in + ctx->mlp.n_out + k] > 0)) return fail(ctx, ROM_E_ARG, "rom_mlp_norm: y_std must be > 0");
    CK(cudaSetDevice(ctx->device));
    mlp_set_norm(ctx->mlp, norm_host, ctx->stream);
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->mlp_norm = true;
    return ROM_OK;
}

rom_status rom_mlp_train_step(rom_ctx *ctx, const float *X_d, const float *Y_d, int64_t N, float lr, int t,
                              float *loss_d) {
    if (!ctx || !X_d || !Y_d) return ROM_E_ARG;
    if (!ctx->has_mlp || !ctx->mlp_norm) return fail(ctx, ROM_E_STATE, "rom_mlp_train_step: MLP or normalisation missing");
    if (N < 1 || N > ctx->mlp.cap || t < 1 || !(lr > 0)) return fail(ctx, ROM_E_ARG, "rom_mlp_train_step: bad N, t or lr");
    CK(cudaSetDevice(ctx->device));
    mlp_train_step(ctx->mlp, X_d, Y_d, N, lr, t, loss_d, ctx->stream);
    CK(cudaGetLastError());
    return ROM_OK;
}

rom_status rom_mlp_loss_grad(rom_ctx *ctx, const float *X_d, const float *Y_d, int64_t N, int bf16, float *grad_d,
                             float *loss_d) {
    if (!ctx || !X_d || !Y_d || !grad_d || !loss_d) return ROM_E_ARG;
    if (!ctx->has_mlp || !ctx->mlp_norm) return fail(ctx, ROM_E_STATE, "rom_mlp_loss_grad: MLP or normalisation missing");
    if (N < 1 || N > ctx->mlp.cap) return fail(ctx, ROM_E_ARG, "rom_mlp_loss_grad: bad N");
    CK(cudaSetDevice(ctx->device));
    mlp_loss_grad(ctx->mlp, X_d, Y_d, N, bf16, grad_d, loss_d, ctx->stream);
    CK(cudaGetLastError());
    return ROM_OK;
}

rom_status rom_mlp_predict(rom_ctx *ctx, const float *X_d, int64_t N, int bf16, double *out_d) {
    if (!ctx || !X_d || !out_d || N < 1) return ROM_E_ARG;
    if (!ctx->has_mlp || !ctx->mlp_norm) return fail(ctx, ROM_E_STATE, "rom_mlp_predict: MLP or normalisation missing");
    CK(cudaSetDevice(ctx->device));
    mlp_predict(ctx->mlp, X_d, N, bf16, out_d, ctx->stream, nullptr);
    CK(cudaGetLastError());
    return ROM_OK;
}

rom_status rom_features(rom_ctx *ctx, rom_state *st, const double *Fbar_d, float *X_d) {
    if (!ctx || !st || !Fbar_d || !X_d || st->ctx != ctx) return ROM_E_ARG;
    if (!ctx->has_basis || !ctx->has_cub || !ctx->has_geom || st->B != ctx->B)
        return fail(ctx, ROM_E_STATE, "rom_features before basis/cubature/geometry");
    CK(cudaSetDevice(ctx->device));
    StepOpts o{};
    o.polar = 1;
    const Model M = make_model(ctx);
    Batch bt = st->bt;
    bt.mu = ctx->mu;
    launch_start(M, bt, Fbar_d, o, nullptr, ctx->stream);
    launch_features(M, bt, bt.U_prev, X_d, ctx->dim * ctx->dim + ctx->n_par + 2 * ctx->n + 2, ctx->stream);
    CK(cudaGetLastError());
    return ROM_OK;
}

rom_status rom_debug_stiffness(rom_ctx *ctx, const rom_state *st, double *K) {
    if (!ctx || !st || !K || st->ctx != ctx) return ROM_E_ARG;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(K, st->bt.K, (size_t)st->B * st->n * st->n * 8, cudaMemcpyDeviceToHost));
    return ROM_OK;
}

rom_status rom_debug_tangent(rom_ctx *ctx, const rom_state *st, void *At, int64_t bytes) {
    if (!ctx || !st || !At || bytes < 0 || st->ctx != ctx) return ROM_E_ARG;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    const size_t have = (size_t)st->B * ctx->dim * ctx->dim * ctx->dim * ctx->dim * (size_t)((st->m + 3) & ~3) * 8;
    CK(cudaMemcpy(At, st->bt.At, std::min((size_t)bytes, have), cudaMemcpyDeviceToHost));
    return ROM_OK;
}

rom_status rom_sensitivity_device(rom_ctx *ctx, rom_state *st, double *dPdmu_d) {
    if (!ctx || !st || !dPdmu_d || st->ctx != ctx) return ROM_E_ARG;
    if (st->last_prec < 0 || !ctx->has_geom) return fail(ctx, ROM_E_STATE, "rom_sensitivity before a step");
    if (ctx->n_par > 3) return fail(ctx, ROM_E_ARG, "rom_sensitivity: at most 3 geometry parameters");
    CK(cudaSetDevice(ctx->device));
    const Model M = make_model(ctx);
    Batch bt = st->bt;
    bt.mu = ctx->mu;
    if (timed(ctx, 8, 0.0, [&] { return launch_sensitivity(M, bt, st->last_prec, dPdmu_d, ctx->stream); }))
        return fail(ctx, ROM_E_ARG, "rom_sensitivity: basis size n=%d too large", M.n);
    CK(cudaGetLastError());
    return ROM_OK;
}

rom_status rom_sensitivity(rom_ctx *ctx, rom_state *st, double *dPdmu) {
    if (!ctx || !st || !dPdmu || st->ctx != ctx) return ROM_E_ARG;
    CK(cudaSetDevice(ctx->device));
    const size_t bytes = (size_t)st->B * ctx->dim * ctx->dim * ctx->n_par * 8;
    double *d = nullptr;
    rom_status s = dalloc(ctx, (void **)&d, bytes);
    if (s != ROM_OK) return s;
    s = rom_sensitivity_device(ctx, st, d);
    if (s == ROM_OK) {
        CK(cudaMemcpyAsync(dPdmu, d, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    void *p = d;
    dfree(p);
    return s;
}

rom_status rom_debug_residual(rom_ctx *ctx, const rom_state *st, double *r, double *v) {
    if (!ctx || !st || !r || st->ctx != ctx) return ROM_E_ARG;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpy(r, st->bt.r, (size_t)st->B * st->n * 8, cudaMemcpyDeviceToHost));
    if (v) CK(cudaMemcpy(v, st->bt.v, (size_t)st->B * ctx->dim * ctx->dim * st->m * 8, cudaMemcpyDeviceToHost));
    return ROM_OK;
}

rom_status rom_state_bytes(const rom_ctx *ctx, int64_t B, int64_t *bytes) {
    if (!ctx || !bytes || B < 1) return ROM_E_ARG;
    const int64_t d2 = ctx->dim * ctx->dim, n = ctx->n, m = ctx->m, ncp = ctx->dim == 2 ? 4 : 6;
    const int64_t per = n * 8 * 5 + (int64_t)sizeof(Ctl) + 8 + 8 + ncp * m * 8 * 2 + m * 8 * 2 + d2 * m * 8 * 2 +
                        d2 * d2 * ((m + 3) & ~3) * 8 + m + n * n * 8 + (n * d2 + d2 * d2) * 8 + d2 * 8 * 4 + d2 * d2 * 8 + 32;
    *bytes = per * B + 64;
    return ROM_OK;
}

rom_status rom_autotune(rom_ctx *ctx, rom_state *st, const rom_opts *opts, int *tile, int *chunk, float *ms) {
    rom_status s = check_step(ctx, st, opts);
    if (s != ROM_OK) return s;
    if (opts->precision >= ROM_PREC_TF32 || (ctx->dim == 3 && ctx->tc3_img) ||
        (opts->precision == ROM_PREC_FP32 && ctx->tc_img[1])) {   // the tensor-core tiles are fixed
        if (tile) *tile = 0;
        if (chunk) *chunk = 0;
        return ROM_OK;
    }
    CK(cudaSetDevice(ctx->device));
    StepOpts o{};
    o.precision = opts->precision;
    const Model M = make_model(ctx);
    Batch bt = st->bt;
    bt.mu = ctx->mu;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float best = 1e30f;
    int bt_tm = 0, bt_ch = 0;
    const int tms[3] = {2, 4, 8}, chs[4] = {8, 16, 32, 64};
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 4; ++c) {
            o.asm_tm = tms[a];
            o.asm_ch = chs[c];
            launch_all_active(bt, ctx->stream);
            if (launch_kernel(2, M, bt, o, st->list2, ctx->stream)) { cudaGetLastError(); continue; }
            float tot = 0.f;
            for (int r = 0; r < 3; ++r) {
                cudaEventRecord(e0, ctx->stream);
                launch_kernel(2, M, bt, o, st->list2, ctx->stream);
                cudaEventRecord(e1, ctx->stream);
                cudaEventSynchronize(e1);
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                tot += t;
            }
            if (cudaGetLastError() != cudaSuccess) continue;
            if (tot / 3 < best) { best = tot / 3; bt_tm = tms[a]; bt_ch = chs[c]; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!bt_tm) return fail(ctx, ROM_E_ARG, "rom_autotune: no valid assembly configuration");
    ctx->asm_tm = bt_tm;
    ctx->asm_ch = bt_ch;
    ++ctx->graph_epoch;
    if (tile) *tile = bt_tm;
    if (chunk) *chunk = bt_ch;
    if (ms) *ms = best;
    return ROM_OK;
}

rom_status rom_serve(int G, rom_ctx *const *ctxs, rom_state *const *sts, const rom_opts *opts,
                     const double *const *Fbar_d, double *const *Pbar_d, double *const *Abar_d,
                     rom_step_info *const *info_d, float *group_ms) {
    if (G < 1 || !ctxs || !sts || !opts || !Fbar_d || !Pbar_d) return ROM_E_ARG;
    rom_ctx *ctx = ctxs[0];
    if (!ctx) return ROM_E_ARG;
    for (int g = 0; g < G; ++g) {
        if (!ctxs[g] || !sts[g] || ctxs[g]->device != ctx->device || sts[g]->ctx != ctxs[g]) return ROM_E_ARG;
        for (int h = 0; h < g; ++h)   // the branches of the graph must not share work buffers
            if (sts[h] == sts[g] || ctxs[h] == ctxs[g])
                return fail(ctx, ROM_E_ARG, "rom_serve: groups %d and %d share a context or state", h, g);
        rom_status s = check_step(ctxs[g], sts[g], &opts[g]);
        if (s != ROM_OK) { ctx->err = ctxs[g]->err; return s; }
        if (opts[g].start == ROM_START_MLP && (s = ensure_feat(ctxs[g], sts[g]->B)) != ROM_OK) { ctx->err = ctxs[g]->err; return s; }
        if (!Fbar_d[g] || !Pbar_d[g] || (opts[g].want_abar && (!Abar_d || !Abar_d[g])))
            return fail(ctx, ROM_E_ARG, "rom_serve: null buffer of group %d", g);
    }
    CK(cudaSetDevice(ctx->device));
    for (int g = 0; g < G; ++g) {
        sts[g]->last_prec = opts[g].precision;
        if (!sts[g]->gstream) CK(cudaStreamCreateWithFlags(&sts[g]->gstream, cudaStreamNonBlocking));
    }
    // one graph for every group: fork from the first group's capture stream, each group's step
    // (its own device-driven WHILE node over the Newton passes) on its own branch, an event node
    // at the end of each branch, join
    std::vector<cudaEvent_t> ev_done(G), ev_join(G);
    cudaEvent_t ev_fork = nullptr, ev_start = nullptr;
    auto destroy_events = [&] {
        for (auto &e : ev_done) if (e) cudaEventDestroy(e);
        for (auto &e : ev_join) if (e) cudaEventDestroy(e);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_start) cudaEventDestroy(ev_start);
    };
    cudaError_t e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&ev_start);
    for (int g = 0; g < G && e == cudaSuccess; ++g) {
        e = cudaEventCreate(&ev_done[g]);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_join[g], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) { destroy_events(); return fail(ctx, ROM_E_CUDA, "rom_serve: %s", cudaGetErrorString(e)); }
    cudaStream_t origin = sts[0]->gstream;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int bad = 0;
    e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(ev_fork, origin);
    for (int g = 0; g < G && e == cudaSuccess; ++g) {
        cudaStream_t cs = sts[g]->gstream;
        if (g > 0) e = cudaStreamWaitEvent(cs, ev_fork, 0);
        int b = 0;
        if (e == cudaSuccess) e = record_step(ctxs[g], sts[g], &opts[g], cs, &b);
        bad |= b;
        if (e == cudaSuccess) e = cudaEventRecordWithFlags(ev_done[g], cs, cudaEventRecordExternal);
        if (e == cudaSuccess && g > 0) {
            e = cudaEventRecord(ev_join[g], cs);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(origin, ev_join[g], 0);
        }
    }
    cudaError_t e2 = cudaStreamEndCapture(origin, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess && !bad) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess || bad) {
        cudaGetLastError();
        destroy_events();
        return fail(ctx, ROM_E_CUDA, "rom_serve: graph of %d groups: %s", G,
                    e != cudaSuccess ? cudaGetErrorString(e) : "launch configuration");
    }
    // inputs into the states' staging buffers, one launch for all groups, outputs back
    cudaStream_t L = ctx->stream;
    for (int g = 0; g < G && e == cudaSuccess; ++g) {
        const int d2 = ctxs[g]->dim * ctxs[g]->dim;
        e = cudaMemcpyAsync(sts[g]->io_F, Fbar_d[g], (size_t)sts[g]->B * d2 * 8, cudaMemcpyDeviceToDevice, L);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev_start, L);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, L);
    for (int g = 0; g < G && e == cudaSuccess; ++g) {
        const int d2 = ctxs[g]->dim * ctxs[g]->dim;
        const size_t B = (size_t)sts[g]->B;
        e = cudaMemcpyAsync(Pbar_d[g], sts[g]->io_P, B * d2 * 8, cudaMemcpyDeviceToDevice, L);
        if (e == cudaSuccess && opts[g].want_abar)
            e = cudaMemcpyAsync(Abar_d[g], sts[g]->io_A, B * d2 * d2 * 8, cudaMemcpyDeviceToDevice, L);
        if (e == cudaSuccess && info_d && info_d[g])
            e = cudaMemcpyAsync(info_d[g], sts[g]->io_info, B * sizeof(rom_step_info), cudaMemcpyDeviceToDevice, L);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(L);
    for (int g = 0; g < G && e == cudaSuccess; ++g)
        if (group_ms) e = cudaEventElapsedTime(&group_ms[g], ev_start, ev_done[g]);
    cudaGraphExecDestroy(exec);
    destroy_events();
    if (e != cudaSuccess) return fail(ctx, ROM_E_CUDA, "rom_serve: %s", cudaGetErrorString(e));
    return ROM_OK;
}

rom_status rom_use_graphs(rom_ctx *ctx, int enable) {
    if (!ctx) return ROM_E_ARG;
    ctx->graphs = enable != 0;
    return ROM_OK;
}

rom_status rom_profile(rom_ctx *ctx, int enable) {
    if (!ctx) return ROM_E_ARG;
    CK(cudaSetDevice(ctx->device));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->recs.clear();
    for (int k = 0; k < ROM_NKERNELS; ++k) { ctx->prof_ms[k] = 0; ctx->prof_launches[k] = 0; ctx->prof_flops[k] = 0; }
    ctx->prof = enable != 0;
    return ROM_OK;
}

rom_status rom_profile_read(rom_ctx *ctx, int kernel, double *ms, int64_t *launches, double *flops) {
    if (!ctx || kernel < 0 || kernel >= ROM_NKERNELS) return ROM_E_ARG;
    if (ms) *ms = ctx->prof_ms[kernel];
    if (launches) *launches = ctx->prof_launches[kernel];
    if (flops) *flops = ctx->prof_flops[kernel];
    return ROM_OK;
}

}  // extern "C"
