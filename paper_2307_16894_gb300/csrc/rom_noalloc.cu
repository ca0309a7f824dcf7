// Allocation-free load step (rom_step_noalloc in include/podecm.h).
//
// Some callers cannot allocate device memory: a solver that runs inside a
// pre-sized memory pool or an arena it does not own, or a host library that
// must not grow the device footprint after start-up (an allocation there can
// fail or stall the rest of the application).  This entry point takes every model, state and output
// array from the caller and keeps the per-instance work arrays of the step
// (trial iterate, Newton control, residual, stiffness, pulled-back tangents,
// trial history, ...) in one file-scope device array of fixed size instead of
// allocating them.  The kernels are the same as those of rom_step_device.
#include <cstdio>
#include <cstring>

#include "../../include/podecm.h"
#include "kernels.cuh"

namespace podecm {
void set_phases(const PhaseD *ph, int n, cudaStream_t s);
cudaError_t get_phases(PhaseD *ph, cudaStream_t s);
int launch_start(const Model &M, Batch Bt, const double *Fbar, const StepOpts &o, const double *dq_pred,
                 cudaStream_t s);
int launch_kernel(int which, const Model &M, Batch Bt, const StepOpts &o, int32_t *list_next, cudaStream_t s);
int launch_finalize(const Model &M, Batch Bt, const StepOpts &o, double *Pbar, double *Abar, void *info,
                    cudaStream_t s);
}  // namespace podecm

using namespace podecm;

// The work arrays of every rom_step_noalloc call on a device live here.  Every GPU
// that loads the library holds these ROM_NOALLOC_SCRATCH_BYTES until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ROM_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch, per device (host-side name is only a stand-in).
static void *g_scratch_addr[64];

// model-layout transposes into the scratch: G [m][d2][n] -> G_T [d2][n][m] and float copy,
// Gmu [m][d2][np] -> Gmu_T [d2][np][m]
__global__ void k_noalloc_layouts(const double *__restrict__ G, const double *__restrict__ Gmu, int m, int d2, int n,
                                  int np, double *G_T, float *G32, double *Gmu_T) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t ng = (int64_t)m * d2 * n;
    if (e < ng) {
        const int j = (int)(e % n);
        const int c = (int)((e / n) % d2);
        const int i = (int)(e / ((int64_t)n * d2));
        const double g = G[e];
        G_T[((int64_t)c * n + j) * m + i] = g;
        G32[e] = (float)g;
    }
    const int64_t nm = (int64_t)m * d2 * np;
    if (e < nm) {
        const int k = (int)(e % np);
        const int c = (int)((e / np) % d2);
        const int i = (int)(e / ((int64_t)np * d2));
        Gmu_T[((int64_t)c * np + k) * m + i] = Gmu[e];
    }
}

static size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

static rom_status err(char *buf, size_t len, rom_status s, const char *msg) {
    if (buf && len) {
        strncpy(buf, msg, len - 1);
        buf[len - 1] = 0;
    }
    return s;
}

extern "C" rom_status rom_step_noalloc(const rom_noalloc_model *model, int64_t B, const double *mu_d, double *a_d,
                                       double *da_prev_d, double *Cpinv_d, double *xi_d, const rom_opts *opts,
                                       const double *Fbar_d, double *Pbar_d, double *Abar_d, rom_step_info *info_d,
                                       void *cuda_stream, char *errbuf, size_t errlen) {
    char msg[256];
    if (!model || !opts || !mu_d || !a_d || !da_prev_d || !Cpinv_d || !xi_d || !Fbar_d || !Pbar_d ||
        (opts->want_abar && !Abar_d) || !model->G || !model->w || !model->phase || !model->Gmu || !model->phases)
        return err(errbuf, errlen, ROM_E_ARG, "rom_step_noalloc: null pointer");
    const int d = model->dim, n = model->n, m = model->m, np = model->n_par;
    if ((d != 2 && d != 3) || n < 1 || n > MAX_N || m < 1 || np < 1 || np > MAX_NPAR || model->n_phase < 1 ||
        model->n_phase > MAX_PHASES || !(model->omega_vol > 0) || B < 1)
        return err(errbuf, errlen, ROM_E_ARG, "rom_step_noalloc: bad model sizes");
    if (!(opts->tol_rel >= 0) || !(opts->tol_abs >= 0) || opts->max_iter < 0 || opts->max_iter > 1000 ||
        opts->max_ls < 0 || opts->max_ls > 60 || opts->precision < 0 || opts->precision > 1 || opts->start < 0 ||
        opts->start > 1)
        return err(errbuf, errlen, ROM_E_ARG, "rom_step_noalloc: bad options (precision fp64/fp32, start plain/prev)");
    const int d2 = d * d, d4 = d2 * d2, ncp = d == 2 ? 4 : 6;
    // scratch carving (every piece 256-byte aligned)
    const size_t Bz = (size_t)B;
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t o = off; off += up256(bytes); return o; };
    const size_t o_GT = take((size_t)m * d2 * n * 8), o_G32 = take((size_t)m * d2 * n * 4);
    const size_t o_GmuT = take((size_t)m * d2 * np * 8), o_counts = take(64);
    const size_t o_qt = take(Bz * n * 8), o_qa = take(Bz * n * 8), o_dq = take(Bz * n * 8);
    const size_t o_ctl = take(Bz * sizeof(Ctl)), o_l1 = take(Bz * 4), o_l2 = take(Bz * 4);
    const size_t o_v = take(Bz * d2 * m * 8), o_wP = take(Bz * d2 * m * 8);
    const size_t o_At = take(Bz * d4 * (size_t)((m + 3) & ~3) * (opts->precision == 0 ? 8 : 4));
    const size_t o_cptr = take(Bz * ncp * m * 8), o_xitr = take(Bz * m * 8), o_pl = take(Bz * m);
    const size_t o_r = take(Bz * n * 8), o_K = take(Bz * n * n * 8), o_U = take(Bz * d2 * 8), o_R = take(Bz * d2 * 8);
    if (off > (size_t)ROM_NOALLOC_SCRATCH_BYTES) {
        snprintf(msg, sizeof msg,
                 "rom_step_noalloc: this batch needs %zu bytes of work space, more than the %d-byte static "
                 "scratch; use fewer instances per call",
                 off, (int)ROM_NOALLOC_SCRATCH_BYTES);
        return err(errbuf, errlen, ROM_E_ARG, msg);
    }
    for (int k = 0; k < model->n_phase; ++k) {
        const rom_phase &q = model->phases[k];
        if (!(q.E > 0) || !(q.nu > -1 && q.nu < 0.5) || !(q.s0 > 0) || (q.hard_law != 0 && q.hard_law != 1))
            return err(errbuf, errlen, ROM_E_ARG, "rom_step_noalloc: bad phase");
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
        return err(errbuf, errlen, ROM_E_CUDA, "rom_step_noalloc: cudaGetDevice failed");
    // one-time set-up on this device (with the device current): the scratch's device address
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            snprintf(msg, sizeof msg, "rom_step_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            return err(errbuf, errlen, ROM_E_CUDA, msg);
        }
        g_scratch_addr[dev] = p;
    }
    unsigned char *S = static_cast<unsigned char *>(g_scratch_addr[dev]);
    cudaStream_t s = (cudaStream_t)cuda_stream;

    Model M;
    M.d = d; M.d2 = d2; M.n = n; M.m = m; M.n_par = np; M.nphase = model->n_phase; M.ncp = ncp;
    M.mA = (m + 3) & ~3;
    M.G_pt = model->G; M.G_T = reinterpret_cast<double *>(S + o_GT); M.G32_pt = reinterpret_cast<float *>(S + o_G32);
    M.w = model->w; M.phase = model->phase; M.Gmu_T = reinterpret_cast<double *>(S + o_GmuT); M.omega = model->omega_vol;
    M.G32h_T = nullptr; M.G32l_T = nullptr;   // FP64 kinematics
    M.Gdf = nullptr;                           // residual in FP64 (k_force)
    Batch bt{};
    bt.B = B; bt.mu = mu_d; bt.q_n = a_d; bt.dq_prev = da_prev_d; bt.cp = Cpinv_d; bt.xi = xi_d;
    bt.q_trial = reinterpret_cast<double *>(S + o_qt); bt.q_acc = reinterpret_cast<double *>(S + o_qa);
    bt.dq = reinterpret_cast<double *>(S + o_dq); bt.ctl = reinterpret_cast<Ctl *>(S + o_ctl);
    bt.list = reinterpret_cast<int32_t *>(S + o_l1); bt.counts = reinterpret_cast<int32_t *>(S + o_counts);
    bt.v = reinterpret_cast<double *>(S + o_v); bt.wP = reinterpret_cast<double *>(S + o_wP);
    bt.At = S + o_At; bt.cp_tr = reinterpret_cast<double *>(S + o_cptr); bt.xi_tr = reinterpret_cast<double *>(S + o_xitr);
    bt.pl = reinterpret_cast<uint8_t *>(S + o_pl); bt.r = reinterpret_cast<double *>(S + o_r);
    bt.K = reinterpret_cast<double *>(S + o_K); bt.Ubar = reinterpret_cast<double *>(S + o_U);
    bt.Rbar = reinterpret_cast<double *>(S + o_R);
    int32_t *list2 = reinterpret_cast<int32_t *>(S + o_l2);

    // the material table lives in constant memory shared with the contexts: save it,
    // install this model's phases, restore it after the step
    PhaseD saved[MAX_PHASES], ph[MAX_PHASES];
    if (get_phases(saved, s) != cudaSuccess) return err(errbuf, errlen, ROM_E_CUDA, "rom_step_noalloc: phase table read");
    for (int k = 0; k < model->n_phase; ++k) {
        const rom_phase &q = model->phases[k];
        ph[k].E = q.E; ph[k].nu = q.nu; ph[k].s0 = q.s0; ph[k].k = q.H_or_k; ph[k].p = q.p; ph[k].law = q.hard_law;
        ph[k].elastic = (q.s0 == INFINITY) ? 1 : 0;
        ph[k].G = q.E / (2.0 * (1.0 + q.nu));
        ph[k].lam = q.E * q.nu / ((1.0 + q.nu) * (1.0 - 2.0 * q.nu));
        ph[k].Kb = ph[k].lam + 2.0 * ph[k].G / 3.0;
    }
    set_phases(ph, model->n_phase, s);
    // the scratch keeps the previous call's contents: clear the active counters
    cudaMemsetAsync(bt.counts, 0, 64, s);
    {
        const int64_t tot = (int64_t)m * d2 * (n > np ? n : np);
        k_noalloc_layouts<<<(int)((tot + 255) / 256), 256, 0, s>>>(model->G, model->Gmu, m, d2, n, np,
                                                                  const_cast<double *>(M.G_T),
                                                                  const_cast<float *>(M.G32_pt),
                                                                  const_cast<double *>(M.Gmu_T));
    }
    StepOpts o;
    o.tol_rel = opts->tol_rel; o.tol_abs = opts->tol_abs; o.max_iter = opts->max_iter; o.max_ls = opts->max_ls;
    o.precision = opts->precision; o.start = opts->start; o.polar = opts->polar_split; o.want_abar = opts->want_abar;
    rom_status st = ROM_OK;
    launch_start(M, bt, Fbar_d, o, nullptr, s);
    int32_t *lists[2] = {bt.list, list2};
    const int max_pass = (opts->max_iter + 1) * (opts->max_ls + 1) + 2;
    int32_t count = 0;
    for (int pass = 0; pass < max_pass; ++pass) {
        Batch b2 = bt;
        b2.list = lists[pass & 1];
        int32_t *nxt = lists[(pass + 1) & 1];
        if (launch_kernel(1, M, b2, o, nxt, s) || launch_kernel(2, M, b2, o, nxt, s) ||
            launch_kernel(3, M, b2, o, nxt, s) || launch_kernel(5, M, b2, o, nxt, s)) {
            st = err(errbuf, errlen, ROM_E_ARG, "rom_step_noalloc: basis size not supported by the assembly kernel");
            break;
        }
        if (cudaMemcpyAsync(&count, bt.counts, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = err(errbuf, errlen, ROM_E_CUDA, "rom_step_noalloc: stream error");
            break;
        }
        if (count == 0) break;
    }
    if (st == ROM_OK && launch_finalize(M, bt, o, Pbar_d, Abar_d, info_d, s))
        st = err(errbuf, errlen, ROM_E_ARG, "rom_step_noalloc: n*d*d too large for the finalize kernel");
    set_phases(saved, MAX_PHASES, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (st == ROM_OK && e != cudaSuccess) {
        snprintf(msg, sizeof msg, "rom_step_noalloc: %s", cudaGetErrorString(e));
        st = err(errbuf, errlen, ROM_E_CUDA, msg);
    }
    return st;
}
