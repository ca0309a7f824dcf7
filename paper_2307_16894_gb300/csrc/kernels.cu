// CUDA kernels of one hyper-reduced load step (arXiv 2307.16894, Sec. 3.2-3.3,
// the online Newton loop of Algorithm 1), batched over independent instances.
//
// One Newton "pass" over the active instances is three launches:
//   k_constitutive : one thread per (instance, cubature point): geometry (F_mu),
//                    kinematics F = Ubar + (G_i a) F_mu^-1, FP64 return map,
//                    tangent, weighted pull-backs v_i = w_i J_i vec(P F_mu^-T) and
//                    At_i = w_i J_i (I x F_mu^-1) A (I x F_mu^-1)^T   [Eqs. forcevector_ecm,
//                    stiffnessmatrix_ecm integrands]
//   k_assemble     : one CTA per instance: f = sum_i G_i^T v_i (FP64) and
//                    K = sum_i G_i^T At_i G_i (FP64 or FP32 CUDA cores)
//   k_solve        : one warp per instance: convergence test, line search,
//                    LU of K (FP64, partial pivoting), da = -K^-1 f      [Eq. red_newton]
// and k_finalize computes Pbar (Eq. eff_stress_1), Abar through the Schur
// complement of the reduced tangent problems (Eqs. tangent_problem_red,
// eff_stiffness_1) and commits the history of converged instances.
#include <algorithm>
#include <cstdio>
#include "kernels.cuh"

namespace podecm {

__constant__ PhaseD c_phases[MAX_PHASES];

void set_phases(const PhaseD *ph, int n, cudaStream_t s) {
    cudaMemcpyToSymbolAsync(c_phases, ph, sizeof(PhaseD) * n, 0, cudaMemcpyHostToDevice, s);
}

// copy the whole phase table back to the host (stream-ordered)
cudaError_t get_phases(PhaseD *ph, cudaStream_t s) {
    return cudaMemcpyFromSymbolAsync(ph, c_phases, sizeof(PhaseD) * MAX_PHASES, 0, cudaMemcpyDeviceToHost, s);
}

// ------------------------------------------------------------------------ start
template <int D>
__global__ void k_start(Model M, Batch Bt, const double *__restrict__ Fbar, StepOpts o,
                        const double *__restrict__ dq_pred) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= Bt.B) return;
    constexpr int D2 = D * D;
    double F[3][3] = {{0}}, R[3][3] = {{0}}, U[3][3] = {{0}};
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) F[i][j] = Fbar[b * D2 + i * D + j];
    if (!o.polar) {
        for (int i = 0; i < D; ++i)
            for (int j = 0; j < D; ++j) { U[i][j] = F[i][j]; R[i][j] = (i == j); }
    } else if (D == 2) {
        const double th = atan2(F[1][0] - F[0][1], F[0][0] + F[1][1]);
        const double c = cos(th), s = sin(th);
        R[0][0] = c; R[0][1] = -s; R[1][0] = s; R[1][1] = c;
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) U[i][j] = R[0][i] * F[0][j] + R[1][i] * F[1][j];
        const double u = 0.5 * (U[0][1] + U[1][0]);
        U[0][1] = U[1][0] = u;
    } else {
        // C = F^T F = N diag(l) N^T ;  U = N diag(sqrt l) N^T ; R = F U^-1
        double C[3][3], N[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += F[k][i] * F[k][j];
                C[i][j] = s;
            }
        jacobi3(C, N);
        double sq[3], isq[3];
        for (int a = 0; a < 3; ++a) { sq[a] = sqrt(C[a][a]); isq[a] = 1.0 / sq[a]; }
        double Ui[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0, si = 0.0;
                for (int a = 0; a < 3; ++a) { s += N[i][a] * sq[a] * N[j][a]; si += N[i][a] * isq[a] * N[j][a]; }
                U[i][j] = s;
                Ui[i][j] = si;
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double s = 0.0;
                for (int k = 0; k < 3; ++k) s += F[i][k] * Ui[k][j];
                R[i][j] = s;
            }
    }
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            Bt.Ubar[b * D2 + i * D + j] = U[i][j];
            Bt.Rbar[b * D2 + i * D + j] = R[i][j];
        }
    const int n = M.n;
    for (int j = 0; j < n; ++j) {
        double q = Bt.q_n[b * n + j];
        if (o.start == 1) q += Bt.dq_prev[b * n + j];
        else if (o.start == 2 && dq_pred) q += dq_pred[b * n + j];
        Bt.q_trial[b * n + j] = q;
        Bt.q_acc[b * n + j] = q;
    }
    Ctl c;
    c.r0 = 0.0; c.tol = 0.0; c.rn_acc = 0.0; c.t = 1.0;
    c.iters = 0; c.evals = 0; c.ls = 0; c.status = 0; c.active = 1; c.acc_k = c.pad1 = 0;
    // learned start: evaluate the predicted point first, then the previous-step point (phase 2 -> 3)
    c.phase = (o.start == 2) ? 2 : 0;
    Bt.ctl[b] = c;
    Bt.list[b] = (int32_t)b;
}

__global__ void k_set_counts(int32_t *counts, int64_t B) {
    counts[0] = (int32_t)B;
    counts[1] = 0;
    counts[4] = 0;   // front / back positions of the final-pass partition (k_flag_final)
    counts[5] = 0;
}

__global__ void k_advance(int32_t *counts) {
    counts[0] = counts[1];
    counts[1] = 0;
}

// ------------------------------------------------------------------ geometry
// a1: F_mu = I + sum_k mu_k Gmu_k(X_i) at cubature point i of instance b (Eq. weakform-dep-mapped);
// returns F_mu^-1 and w_i |det F_mu|
template <int D>
__device__ __forceinline__ void geometry_point(const Model &M, const double *mu, int64_t b, int i, double Fmi[D][D],
                                               double *wJ) {
    const int m = M.m;
    double Fm[D][D];
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int r = 0; r < D; ++r) {
            double s = (a == r) ? 1.0 : 0.0;
            for (int k = 0; k < M.n_par; ++k)
                s += mu[b * M.n_par + k] * M.Gmu_T[((size_t)(a * D + r) * M.n_par + k) * m + i];
            Fm[a][r] = s;
        }
    double J;
    if (D == 2) {
        const double det = Fm[0][0] * Fm[1][1] - Fm[0][1] * Fm[1][0];
        J = fabs(det);
        const double id = 1.0 / det;
        Fmi[0][0] = Fm[1][1] * id; Fmi[0][1] = -Fm[0][1] * id;
        Fmi[1][0] = -Fm[1][0] * id; Fmi[1][1] = Fm[0][0] * id;
    } else {
        double c00 = Fm[1][1] * Fm[2][2] - Fm[1][2] * Fm[2][1];
        double c01 = Fm[1][2] * Fm[2][0] - Fm[1][0] * Fm[2][2];
        double c02 = Fm[1][0] * Fm[2][1] - Fm[1][1] * Fm[2][0];
        const double det = Fm[0][0] * c00 + Fm[0][1] * c01 + Fm[0][2] * c02;
        J = fabs(det);
        const double id = 1.0 / det;
        Fmi[0][0] = c00 * id; Fmi[1][0] = c01 * id; Fmi[2][0] = c02 * id;
        Fmi[0][1] = (Fm[0][2] * Fm[2][1] - Fm[0][1] * Fm[2][2]) * id;
        Fmi[1][1] = (Fm[0][0] * Fm[2][2] - Fm[0][2] * Fm[2][0]) * id;
        Fmi[2][1] = (Fm[0][1] * Fm[2][0] - Fm[0][0] * Fm[2][1]) * id;
        Fmi[0][2] = (Fm[0][1] * Fm[1][2] - Fm[0][2] * Fm[1][1]) * id;
        Fmi[1][2] = (Fm[0][2] * Fm[1][0] - Fm[0][0] * Fm[1][2]) * id;
        Fmi[2][2] = (Fm[0][0] * Fm[1][1] - Fm[0][1] * Fm[1][0]) * id;
    }
    *wJ = M.w[i] * J;
}

// the per-geometry cache geo[b][c][i]: F_mu^-1 entries c < d^2 (row-major), w_i J at c = d^2.  The
// geometry of an instance is fixed over its load steps, so the FP64 work of a1 is done once
// instead of in every Newton pass (FP64 is the constitutive kernel's bound; the cache adds
// (d^2 + 1) x 8 bytes of reads per point and pass)
template <int D>
__global__ void k_geometry(Model M, const double *__restrict__ mu, int64_t B, double *__restrict__ geo) {
    constexpr int D2 = D * D;
    const int m = M.m;
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= B * m) return;
    const int64_t b = gid / m;
    const int i = (int)(gid - b * m);
    double Fmi[D][D], wJ;
    geometry_point<D>(M, mu, b, i, Fmi, &wJ);
    double *gp = geo + (size_t)b * (D2 + 1) * m + i;
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int r = 0; r < D; ++r) gp[(size_t)(a * D + r) * m] = Fmi[a][r];
    gp[(size_t)D2 * m] = wJ;
}

void launch_geometry(const Model &M, const double *mu, int64_t B, double *geo, cudaStream_t s) {
    const int64_t n = B * M.m;
    const unsigned grid = (unsigned)((n + 255) / 256);
    if (M.d == 2) k_geometry<2><<<grid, 256, 0, s>>>(M, mu, B, geo);
    else k_geometry<3><<<grid, 256, 0, s>>>(M, mu, B, geo);
}

// ------------------------------------------------------------------ constitutive
// Mixed-precision kinematics in double-float arithmetic (FP32 pairs, products by TwoProd,
// sums by TwoSum with a compensation term; Ogita, Rump & Oishi 2005): the FP64 pipe of this GPU
// runs 1/64 of the FP32 rate, and the pairs carry ~48 significant bits.  q is split once per
// block into (hi, lo) FP32 pairs in shared memory (a 128-thread block spans at most two
// instances when m >= 128).
constexpr int KIN_DF_SLOTS = 2;

// 3D mixed precision: five 128-thread blocks per SM (at most 102 registers, some spilled to L1)
// hide the FP64 pipe latency better than fewer blocks at more registers (measured: 3 / 4 / 5 / 6
// blocks 444.8 / 452.1 / 436.9 / 439.3 ms of this kernel over 6 load steps at B = 16384)
template <int D, typename TT>
__global__ void __launch_bounds__(128, (D == 3 && sizeof(TT) == 4) ? 5 : 1) k_constitutive(Model M, Batch Bt) {
    constexpr int D2 = D * D;
    constexpr bool DF = sizeof(TT) == 4;
    const int m = M.m, n = M.n;
    const int n_act = Bt.counts[0];
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p = gid / m;
    __shared__ float2 q32s[DF ? KIN_DF_SLOTS * MAX_N : 1];
    const bool use_df = DF && M.G32h_T && m >= 128;
    const int64_t p_first = (int64_t)blockIdx.x * blockDim.x / m;
    if (use_df) {
        for (int e = threadIdx.x; e < KIN_DF_SLOTS * n; e += blockDim.x) {
            const int slot = e / n, j = e - slot * n;
            const int64_t pp = p_first + slot;
            float2 v = make_float2(0.f, 0.f);
            if (pp < n_act) {
                const double q = Bt.q_trial[(int64_t)Bt.list[pp] * n + j];
                v.x = (float)q;
                v.y = (float)(q - (double)v.x);
            }
            q32s[e] = v;
        }
        __syncthreads();
    }
    if (p >= n_act) return;
    const int i = (int)(gid - p * m);
    const int64_t b = Bt.list[p];

    // a1: geometry F_mu = I + sum_k mu_k Gmu_k(X_i): F_mu^-1 and w_i J from the per-geometry cache
    double Fmi[D][D], wJ;
    if (Bt.geo) {
        const double *gp = Bt.geo + (size_t)b * (D2 + 1) * m + i;
#pragma unroll
        for (int a = 0; a < D; ++a)
#pragma unroll
            for (int r = 0; r < D; ++r) Fmi[a][r] = gp[(size_t)(a * D + r) * m];
        wJ = gp[(size_t)D2 * m];
    } else {
        geometry_point<D>(M, Bt.mu, b, i, Fmi, &wJ);
    }

    // a2: kinematics H = G_i a, F = Ubar + H F_mu^-1
    double H[D2];
    if (use_df) {
        const float2 *qs = q32s + (p - p_first) * n;
        float s[D2], er[D2];
#pragma unroll
        for (int c = 0; c < D2; ++c) { s[c] = 0.f; er[c] = 0.f; }
        for (int j = 0; j < n; ++j) {
            const float2 qq = qs[j];
#pragma unroll
            for (int c = 0; c < D2; ++c) {
                const size_t gi = ((size_t)c * n + j) * m + i;
                const float gh = M.G32h_T[gi], gl = M.G32l_T[gi];
                const float pr = __fmul_rn(gh, qq.x);
                float e = fmaf(gh, qq.x, -pr);
                e = fmaf(gh, qq.y, e);
                e = fmaf(gl, qq.x, e);
                const float sn = __fadd_rn(s[c], pr);
                const float bb = __fsub_rn(sn, s[c]);
                const float t = __fadd_rn(__fsub_rn(s[c], __fsub_rn(sn, bb)), __fsub_rn(pr, bb));
                s[c] = sn;
                er[c] = __fadd_rn(er[c], __fadd_rn(t, e));
            }
        }
#pragma unroll
        for (int c = 0; c < D2; ++c) H[c] = f2d_exact(s[c]) + f2d_exact(er[c]);
    } else {
        for (int c = 0; c < D2; ++c) H[c] = 0.0;
        const double *qb = Bt.q_trial + b * n;
        for (int j = 0; j < n; ++j) {
            const double qj = __ldg(qb + j);
#pragma unroll
            for (int c = 0; c < D2; ++c) H[c] += M.G_T[((size_t)c * n + j) * m + i] * qj;
        }
    }
    double F[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 1.0}};
#pragma unroll
    for (int a = 0; a < D; ++a)
#pragma unroll
        for (int bb = 0; bb < D; ++bb) {
            double s = Bt.Ubar[b * D2 + a * D + bb];
#pragma unroll
            for (int r = 0; r < D; ++r) s += H[a * D + r] * Fmi[r][bb];
            F[a][bb] = s;
        }

    // a3: return map (FP64)
    const int ncp = M.ncp;
    const size_t hb = (size_t)b * ncp * m + i;
    double cp[6];
    if (D == 2) {
        cp[0] = Bt.cp[hb]; cp[1] = Bt.cp[hb + m]; cp[2] = 0.0;
        cp[3] = Bt.cp[hb + 2 * (size_t)m]; cp[4] = 0.0; cp[5] = Bt.cp[hb + 3 * (size_t)m];
    } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) cp[k] = Bt.cp[hb + k * (size_t)m];
    }
    const double xi_n = Bt.xi[(size_t)b * m + i];
    const PhaseD &ph = c_phases[M.phase[i]];
    MatState S;
    double P[3][3], Finv[3][3], cpn[6], xin;
    material_value<D, sizeof(TT) == sizeof(double)>(F, cp, xi_n, ph, S, P, Finv, cpn, &xin);
    // a5: weighted pull-backs
    const size_t vb = (size_t)b * D2 * m + i;
#pragma unroll
    for (int a = 0; a < D; ++a) {
        double wp[D];
#pragma unroll
        for (int r = 0; r < D; ++r) {
            wp[r] = wJ * P[a][r];
            Bt.wP[vb + (size_t)(a * D + r) * m] = wp[r];
        }
#pragma unroll
        for (int r = 0; r < D; ++r) {
            double s = 0.0;
#pragma unroll
            for (int bb = 0; bb < D; ++bb) s += wp[bb] * Fmi[r][bb];
            Bt.v[vb + (size_t)(a * D + r) * m] = s;
        }
    }
    if (D == 2) {
        Bt.cp_tr[hb] = cpn[0]; Bt.cp_tr[hb + m] = cpn[1];
        Bt.cp_tr[hb + 2 * (size_t)m] = cpn[3]; Bt.cp_tr[hb + 3 * (size_t)m] = cpn[5];
    } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) Bt.cp_tr[hb + k * (size_t)m] = cpn[k];
    }
    Bt.xi_tr[(size_t)b * m + i] = xin;
    Bt.pl[(size_t)b * m + i] = (uint8_t)S.plastic;

    // a4 + a5: tangent columns At[(a,r),(c,s)] = wJ (dP(e_c x F_mu^-1[s,:]) F_mu^-T)_ar
    TangentData<TT> td;
    tangent_setup<D, TT>(S, ph, F, cp, Finv, P, td);
    TT *At = reinterpret_cast<TT *>(Bt.At);
    const size_t ab = (size_t)b * D2 * D2 * M.mA + i;
    // F_mu^-1 and wJ in the tangent precision, converted once (inside the direction loop the
    // conversions would be redone per direction: on the mixed path they run on the FP64 pipe)
    TT Fmt[3][3];
#pragma unroll
    for (int r = 0; r < D; ++r)
#pragma unroll
        for (int l = 0; l < D; ++l) Fmt[r][l] = TT(Fmi[r][l]);
    const TT wJt = TT(wJ);
#pragma unroll 1
    for (int c = 0; c < D; ++c)
#pragma unroll 1
        for (int s = 0; s < D; ++s) {
            TT f[3] = {TT(0), TT(0), TT(0)};
#pragma unroll
            for (int l = 0; l < D; ++l) f[l] = pick<D, TT>(s, Fmt[0][l], Fmt[1][l], Fmt[D - 1][l]);
            TT dP[3][3];
            tangent_direction<D, TT>(td, c, f, dP);
            const int col = c * D + s;
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int r = 0; r < D; ++r) {
                    TT t = TT(0);
#pragma unroll
                    for (int bb = 0; bb < D; ++bb) t += dP[a][bb] * Fmt[r][bb];
                    At[ab + (size_t)((a * D + r) * D2 + col) * M.mA] = wJt * t;
                }
        }
}

// --------------------------------------------------------------------- assembly
// smem layout: Gs64[CH][D2][np] | Ys[CH][D2][np] (TK) | As[CH][D4] (TK) | vs[CH][D2] | (FP32: Gs32)
template <int D, typename TK, int TM>
__global__ void __launch_bounds__(256) k_assemble(Model M, Batch Bt, int CH, int NG, int do_force) {
    constexpr int D2 = D * D, D4 = D2 * D2;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n_act = Bt.counts[0];
    const int p = blockIdx.x;
    if (p >= n_act) return;
    const int64_t b = Bt.list[p];
    const int n = M.n, m = M.m;
    const int NT = (n + TM - 1) / TM;
    const int np = NT * TM;
    double *Gs = reinterpret_cast<double *>(smem);
    TK *Ys = reinterpret_cast<TK *>(Gs + (size_t)CH * D2 * np);
    TK *As = Ys + (size_t)CH * D2 * np;
    double *vs = reinterpret_cast<double *>(As + (size_t)CH * D4 + 2);   // keep 8-byte alignment
    vs = reinterpret_cast<double *>((reinterpret_cast<uintptr_t>(vs) + 7) & ~uintptr_t(7));
    TK *Gk = reinterpret_cast<TK *>(vs + (size_t)CH * D2);             // used when TK != double

    const int tid = threadIdx.x;
    const int nup = NT * (NT + 1) / 2;
    const int grp = tid / nup;
    const int tl = tid - grp * nup;
    const bool has_tile = grp < NG;
    int ti = 0, tj = 0;
    if (has_tile) {   // tl -> (ti, tj), ti <= tj
        int r = tl;
        ti = 0;
        while (r >= NT - ti) { r -= NT - ti; ++ti; }
        tj = ti + r;
    }
    TK acc[TM][TM];
#pragma unroll
    for (int x = 0; x < TM; ++x)
#pragma unroll
        for (int y = 0; y < TM; ++y) acc[x][y] = TK(0);
    double racc = 0.0;
    const int FG = blockDim.x / n;          // thread groups sharing the force rows
    const int fg = tid / n, fj = tid - (tid / n) * n;
    const TK *At = reinterpret_cast<const TK *>(Bt.At);

    for (int c0 = 0; c0 < m; c0 += CH) {
        const int ch = min(CH, m - c0);
        __syncthreads();
        // load G chunk (rows = (point, component)), zero-padded to np columns; the FP32 copy comes
        // from the FP32 image of G (the same rounding), not from conversions on the FP64 pipe
        for (int e = tid; e < CH * D2 * np; e += blockDim.x) {
            const int row = e / np, col = e - row * np;
            const int ii = row / D2;
            const bool in = ii < ch && col < n;
            const size_t gi = ((size_t)(c0 + ii) * D2 + (row - ii * D2)) * n + col;
            if (sizeof(TK) == sizeof(double) || do_force) Gs[e] = in ? M.G_pt[gi] : 0.0;
            if (sizeof(TK) != sizeof(double)) Gk[e] = in ? TK(M.G32_pt[gi]) : TK(0);
        }
        for (int e = tid; e < CH * D4; e += blockDim.x) {
            const int ce = e / CH, ii = e - ce * CH;
            As[ii * D4 + ce] = (ii < ch) ? At[((size_t)b * D4 + ce) * M.mA + c0 + ii] : TK(0);
        }
        if (do_force)
            for (int e = tid; e < CH * D2; e += blockDim.x) {
                const int c = e / CH, ii = e - c * CH;
                vs[ii * D2 + c] = (ii < ch) ? Bt.v[((size_t)b * D2 + c) * m + c0 + ii] : 0.0;
            }
        __syncthreads();
        // Y[ii][c][k] = sum_e As[ii][c][e] G[ii][e][k]
        const TK *Gsrc = (sizeof(TK) == sizeof(double)) ? reinterpret_cast<const TK *>(Gs) : Gk;
        for (int e = tid; e < CH * D2 * np; e += blockDim.x) {
            const int k = e % np, rc = e / np;
            const int ii = rc / D2, c = rc - ii * D2;
            TK s = TK(0);
#pragma unroll
            for (int q = 0; q < D2; ++q) s += As[ii * D4 + c * D2 + q] * Gsrc[(ii * D2 + q) * np + k];
            Ys[e] = s;
        }
        // force: r_j += sum_rows G[row][j] v[row]  (FP64; rows split over FG thread groups, fixed order)
        if (do_force && fg < FG) {
            for (int row = fg; row < ch * D2; row += FG) racc += Gs[row * np + fj] * vs[row];
        }
        __syncthreads();
        if (has_tile) {
            for (int row = grp; row < ch * D2; row += NG) {
                TK gj[TM], yk[TM];
#pragma unroll
                for (int x = 0; x < TM; ++x) gj[x] = Gsrc[row * np + ti * TM + x];
#pragma unroll
                for (int y = 0; y < TM; ++y) yk[y] = Ys[row * np + tj * TM + y];
#pragma unroll
                for (int x = 0; x < TM; ++x)
#pragma unroll
                    for (int y = 0; y < TM; ++y) acc[x][y] += gj[x] * yk[y];
            }
        }
    }
    __syncthreads();
    // reduce groups in smem (reuse the G buffer): red[g][np][np]
    TK *red = reinterpret_cast<TK *>(smem);
    if (has_tile) {
#pragma unroll
        for (int x = 0; x < TM; ++x)
#pragma unroll
            for (int y = 0; y < TM; ++y) red[((size_t)grp * np + ti * TM + x) * np + tj * TM + y] = acc[x][y];
    }
    __syncthreads();
    double *Kb = Bt.K + (size_t)b * n * n;
    for (int e = tid; e < n * n; e += blockDim.x) {
        const int j = e / n, k = e - j * n;
        const int jj = min(j, k), kk = max(j, k);
        // tile that holds (jj, kk) is upper (ti <= tj); within a diagonal tile both orders exist
        int a = jj, c = kk;
        if ((jj / TM) == (kk / TM)) { a = j; c = k; }
        TK s = TK(0);
        for (int g = 0; g < NG; ++g) s += red[((size_t)g * np + a) * np + c];
        Kb[e] = double(s);
    }
    // reduce the force groups in a fixed order (reuse the buffer after the K gather)
    if (!do_force) return;   // the residual comes from the double-float force kernel
    __syncthreads();
    double *fr = reinterpret_cast<double *>(smem);
    if (fg < FG) fr[fg * n + fj] = racc;
    __syncthreads();
    if (tid < n) {
        double s = 0.0;
        for (int g = 0; g < FG; ++g) s += fr[g * n + tid];
        Bt.r[b * n + tid] = s;
    }
}

// ------------------------------------------------------------------------ solve
// LU with partial pivoting of the n x n row-major matrix A (shared memory) by the whole block,
// the same row operations applied to the nrhs right-hand sides X[r][0..n) (forward
// substitution), then back substitution: X <- A^-1 X.  Pivot = largest |A[i][k]|, ties to the
// lower row; full rows are swapped (L included).  Returns false (uniformly over the block) if a
// pivot is zero or non-finite.
template <typename T>
__device__ bool block_lu_solve(T *A, int n, int lda, T *X, int ldx, int nrhs, int *s_piv) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int tx = tid & 15, ty = tid >> 4, NY = nt >> 4;
    for (int k = 0; k < n; ++k) {
        if (tid < 32) {
            // pivot search in the matrix's own precision (an FP32 matrix compared in FP64 would
            // put conversions and compares on the FP64 pipe)
            T best = T(-1);
            int bi = k;
            for (int i = k + tid; i < n; i += 32) {
                const T v = fabs(A[i * lda + k]);
                if (v > best || (v == best && i < bi)) { best = v; bi = i; }
            }
            for (int off = 16; off > 0; off >>= 1) {
                const T ob = __shfl_xor_sync(0xffffffffu, best, off);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (tid == 0) *s_piv = (!(best > T(0)) || !isfinite(best)) ? -1 : bi;
        }
        __syncthreads();
        const int p = *s_piv;
        if (p < 0) return false;
        if (p != k) {
            for (int j = tid; j < n; j += nt) { const T t = A[k * lda + j]; A[k * lda + j] = A[p * lda + j]; A[p * lda + j] = t; }
            for (int r = tid; r < nrhs; r += nt) { const T t = X[r * ldx + k]; X[r * ldx + k] = X[r * ldx + p]; X[r * ldx + p] = t; }
        }
        __syncthreads();
        const T akk = A[k * lda + k];
        for (int i = k + 1 + tid; i < n; i += nt) A[i * lda + k] /= akk;
        __syncthreads();
        // trailing update and forward substitution (16 x nt/16 thread grid)
        for (int i = k + 1 + ty; i < n; i += NY) {
            const T lik = A[i * lda + k];
            for (int j = k + 1 + tx; j < n; j += 16) A[i * lda + j] -= lik * A[k * lda + j];
            for (int r = tx; r < nrhs; r += 16) X[r * ldx + i] -= lik * X[r * ldx + k];
        }
        __syncthreads();
    }
    for (int k = n - 1; k >= 0; --k) {
        for (int r = tid; r < nrhs; r += nt) X[r * ldx + k] /= A[k * lda + k];
        __syncthreads();
        for (int r = ty; r < nrhs; r += NY)
            for (int i = tx; i < k; i += 16) X[r * ldx + i] -= A[i * lda + k] * X[r * ldx + k];
        __syncthreads();
    }
    return true;
}

// LU with partial pivoting by the whole block without right-hand sides: A <- L\U, piv[k] =
// pivot row of step k (full rows swapped).  Returns false (uniformly) on a zero or non-finite
// pivot.
template <typename T>
__device__ bool block_lu_factor(T *A, int n, int lda, int *piv, int *s_piv) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int tx = tid & 15, ty = tid >> 4, NY = nt >> 4;
    for (int k = 0; k < n; ++k) {
        if (tid < 32) {
            float best = -1.f;
            int bi = k;
            for (int i = k + tid; i < n; i += 32) {
                const float v = fabsf((float)A[i * lda + k]);
                if (v > best || (v == best && i < bi)) { best = v; bi = i; }
            }
            for (int off = 16; off > 0; off >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, off);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (tid == 0) {
                *s_piv = (!(best > 0.f) || !isfinite(best)) ? -1 : bi;
                piv[k] = bi;
            }
        }
        __syncthreads();
        const int p = *s_piv;
        if (p < 0) return false;
        if (p != k)
            for (int j = tid; j < n; j += nt) { const T t = A[k * lda + j]; A[k * lda + j] = A[p * lda + j]; A[p * lda + j] = t; }
        __syncthreads();
        const T akk = A[k * lda + k];
        for (int i = k + 1 + tid; i < n; i += nt) A[i * lda + k] /= akk;
        __syncthreads();
        for (int i = k + 1 + ty; i < n; i += NY) {
            const T lik = A[i * lda + k];
            for (int j = k + 1 + tx; j < n; j += 16) A[i * lda + j] -= lik * A[k * lda + j];
        }
        __syncthreads();
    }
    return true;
}

// y <- A^-1 y with the factors of block_lu_factor, by warp 0 (the others wait at the final barrier)
template <typename T>
__device__ void block_lu_apply(const T *A, int n, int lda, const int *piv, T *y) {
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        if (lane == 0)
            for (int k = 0; k < n; ++k)
                if (piv[k] != k) { const T t = y[k]; y[k] = y[piv[k]]; y[piv[k]] = t; }
        __syncwarp();
        for (int k = 0; k < n; ++k) {
            const T yk = y[k];
            for (int i = k + 1 + lane; i < n; i += 32) y[i] -= A[i * lda + k] * yk;
            __syncwarp();
        }
        for (int k = n - 1; k >= 0; --k) {
            if (lane == 0) y[k] /= A[k * lda + k];
            __syncwarp();
            const T yk = y[k];
            for (int i = lane; i < k; i += 32) y[i] -= A[i * lda + k] * yk;
            __syncwarp();
        }
    }
    __syncthreads();
}

// max over the block of v (>= 0); red = shared scratch of blockDim / 32 doubles
__device__ double block_max(double v, double *red) {
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    __syncthreads();
    return m;
}

// Newton direction x = -K^-1 r into shared x[0..n).  FP64 path: LU of K in FP64 by the block.
// Mixed paths (n >= 16): LU of K rounded to FP32, then iterative refinement with FP64 residuals
// -r - K x (at most 3 corrections, until a correction is below 1e-15 max|x|); a correction that
// does not shrink below half of the previous one sends the solve to the FP64 LU.  The result
// solves the same K to FP64 accuracy either way.  A: n*n doubles of shared scratch.
__device__ bool newton_direction(const Batch &Bt, int64_t b, int n, int precision, double *A, double *x, int *s_piv,
                                 double *red) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const double *Kb = Bt.K + (size_t)b * n * n;
    const double *r = Bt.r + b * n;
    const int lda = n + 1;   // padded rows: column accesses of the factors hit distinct banks
    if (precision >= 1 && n >= 16) {   // mixed paths (below n = 16 the FP64 LU is as fast)
        float *A32 = reinterpret_cast<float *>(A);
        float *y = A32 + (size_t)n * lda;                                 // n floats
        int *piv = reinterpret_cast<int *>(y + n);                        // n ints  (n lda + 2n floats <= 2 n lda)
        // FP64 <-> FP32 by integer operations on the bit patterns (the conversion instructions run
        // on the FP64 pipe); the FP32 factor's truncation is corrected by the FP64 refinement
        for (int e = tid; e < n * n; e += nt) A32[(e / n) * lda + e % n] = to_tangent<float>(Kb[e]);
        for (int j = tid; j < n; j += nt) y[j] = to_tangent<float>(-r[j]);
        __syncthreads();
        bool ok = block_lu_factor<float>(A32, n, lda, piv, s_piv);
        if (ok) {
            block_lu_apply<float>(A32, n, lda, piv, y);
            for (int j = tid; j < n; j += nt) x[j] = widen(y[j]);
            __syncthreads();
            double prev = INFINITY;
            for (int it = 0; it < 3; ++it) {
                // FP64 residual of the current solution, one thread per row (serial sum over the
                // row): every FP64 warp instruction has all its lanes busy, which matters on a part
                // whose FP64 pipe takes 16 cycles per warp instruction whatever the active lanes
                for (int i = tid; i < n; i += nt) {
                    const double *Ki = Kb + (size_t)i * n;
                    double s = 0.0;
                    for (int j = 0; j < n; ++j) s += Ki[j] * x[j];
                    y[i] = to_tangent<float>(-r[i] - s);
                }
                __syncthreads();
                block_lu_apply<float>(A32, n, lda, piv, y);
                double dl = 0.0, xl = 0.0;
                for (int j = tid; j < n; j += nt) { dl = fmax(dl, widen(fabsf(y[j]))); xl = fmax(xl, fabs(x[j])); }
                const double dn = block_max(dl, red), xn = block_max(xl, red);
                if (!(dn <= 0.5 * prev)) { ok = false; break; }
                for (int j = tid; j < n; j += nt) x[j] += widen(y[j]);
                __syncthreads();
                prev = dn;
                if (dn <= 1e-15 * xn) break;
            }
        }
        if (ok) return true;
        __syncthreads();
        // FP64 fallback (rare): the shared-memory region holds only the FP32 factor, so the LU runs
        // in place on K in global memory (K is assembled anew before the next solve, and the K of a
        // converged instance is never factored here)
        double *Kg = Bt.K + (size_t)b * n * n;
        for (int j = tid; j < n; j += nt) x[j] = -r[j];
        __syncthreads();
        return block_lu_solve<double>(Kg, n, n, x, n, 1, s_piv);
    }
    for (int e = tid; e < n * n; e += nt) A[(e / n) * lda + e % n] = Kb[e];
    for (int j = tid; j < n; j += nt) x[j] = -r[j];
    __syncthreads();
    return block_lu_solve<double>(A, n, lda, x, n, 1, s_piv);
}

// shared memory of k_solve: the LU region (FP32 factor with its right-hand side and pivots on the
// mixed paths with n >= 16, else the FP64 matrix), then x [n] doubles and the pivot scratch
__host__ __device__ inline size_t solve_region_bytes(int n, int precision) {
    const size_t f32 = ((size_t)n * (n + 1) + 2 * (size_t)n) * 4;
    const size_t f64 = (size_t)n * (n + 1) * 8;
    return ((precision >= 1 && n >= 16) ? ((f32 + 7) & ~(size_t)7) : f64);
}

constexpr int ESC_ITERS = 4;

// one CTA of SOLVE_THREADS (32 for n <= 32) per active instance: convergence test, line search, start selection
// and the solve of K da = -r (newton_direction); every thread runs the same per-instance state
// machine on the same values, so all branches are uniform over the block
constexpr int SOLVE_THREADS = 128;

// Euclidean norm of the reduced residual r[0..n) by one warp: lane-strided partial sums, then a
// butterfly over the warp (every lane gets the total).  The solve's convergence test and the
// final-pass flag (k_flag_final) both use this function, so they see the same bits.
__device__ __forceinline__ double warp_residual_norm(const double *r, int n, int lane) {
    double s = 0.0;
    for (int j = lane; j < n; j += 32) s += r[j] * r[j];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    return sqrt(s);
}

__global__ void __launch_bounds__(SOLVE_THREADS) k_solve(Model M, Batch Bt, StepOpts o, int32_t *list_next) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double bc_rn;
    __shared__ double red[SOLVE_THREADS / 32];
    __shared__ int s_piv;
    const int n_act = Bt.counts[0];
    const int p = blockIdx.x;
    if (p >= n_act) return;
    const int64_t b = Bt.list[p];
    const int n = M.n, tid = threadIdx.x, nt = blockDim.x;
    double *A = reinterpret_cast<double *>(smem);
    double *x = reinterpret_cast<double *>(smem + solve_region_bytes(n, o.precision));
    const double *r = Bt.r + b * n;
    if (tid < 32) {
        const double v = warp_residual_norm(r, n, tid);
        if (tid == 0) bc_rn = v;
    }
    __syncthreads();
    const double rn = bc_rn;
    Ctl c = Bt.ctl[b];
    double *qt = Bt.q_trial + b * n, *qa = Bt.q_acc + b * n, *dq = Bt.dq + b * n;
    bool accepted = false;
    bool keep_dq = false;   // Newton direction already known (learned start chosen)
    if (c.phase == 0 || c.phase == 4) {
        if (c.phase == 4) c.evals += 1;
        if (c.phase == 0 && o.start == 1 && Bt.r0_prev && tid == 0) Bt.r0_prev[b] = rn;   // previous-step predictor
        c.r0 = rn;
        c.tol = fmax(o.tol_rel * rn, o.tol_abs);
        c.rn_acc = rn;
        c.phase = 1;
        for (int j = tid; j < n; j += nt) qa[j] = qt[j];
        accepted = true;
    } else if (c.phase == 2) {
        // learned start evaluated: its Newton direction, then either start from it (its residual is
        // at most the previous-step predictor's residual of the last step that evaluated one) or
        // also evaluate the previous-step predictor a_n + (a_n - a_{n-1}) and keep the better start
        c.r0 = rn;
        const double rref = Bt.r0_prev ? Bt.r0_prev[b] : INFINITY;
        // an instance that the learned start already converges needs no direction (and its K, the
        // K at the solution, must not be factored in place by the solve's FP64 fallback)
        const bool done = isfinite(rn) && isfinite(rref) && rn <= rref &&
                          (rn <= fmax(o.tol_rel * rref, o.tol_abs) || o.max_iter == 0);
        const bool ok = done || (isfinite(rn) && newton_direction(Bt, b, n, o.precision, A, x, &s_piv, red));
        if (ok && isfinite(rref) && rn <= rref) {
            c.tol = fmax(o.tol_rel * rref, o.tol_abs);
            c.rn_acc = rn;
            if (rn <= c.tol || o.max_iter == 0) {
                c.status = 0;
                c.active = 0;
                for (int j = tid; j < n; j += nt) qa[j] = qt[j];
            } else {
                c.t = 1.0;
                c.ls = 0;
                c.phase = 1;
                for (int j = tid; j < n; j += nt) { dq[j] = x[j]; qa[j] = qt[j]; qt[j] = qa[j] + x[j]; }
            }
            keep_dq = true;
        } else {
            if (!ok) c.r0 = NAN;
            for (int j = tid; j < n; j += nt) {
                dq[j] = ok ? x[j] : 0.0;
                qa[j] = qt[j];
                qt[j] = Bt.q_n[b * n + j] + Bt.dq_prev[b * n + j];
            }
            c.phase = 3;
        }
    } else if (c.phase == 3) {
        c.evals += 1;
        if (Bt.r0_prev && tid == 0) Bt.r0_prev[b] = rn;
        const double rm = c.r0;
        if (!(rm <= rn)) {
            // previous-step predictor wins (or the learned start failed)
            c.r0 = rn;
            c.tol = fmax(o.tol_rel * rn, o.tol_abs);
            c.rn_acc = rn;
            c.phase = 1;
            for (int j = tid; j < n; j += nt) qa[j] = qt[j];
            accepted = true;
        } else {
            // the tolerance stays relative to the previous-step predictor's residual, so that the
            // learned start is held to the same absolute residual as the fallback
            c.r0 = rm;
            c.tol = fmax(o.tol_rel * rn, o.tol_abs);
            c.rn_acc = rm;
            if (rm <= c.tol || o.max_iter == 0) {
                // the stored per-point data belong to the other candidate: re-evaluate here
                for (int j = tid; j < n; j += nt) qt[j] = qa[j];
                c.phase = 4;
            } else {
                c.t = 1.0;
                c.ls = 0;
                c.phase = 1;
                for (int j = tid; j < n; j += nt) qt[j] = qa[j] + dq[j];
                keep_dq = true;
            }
        }
    } else {
        c.evals += 1;
        if (c.ls >= o.max_ls || (isfinite(rn) && rn < c.rn_acc)) {
            for (int j = tid; j < n; j += nt) qa[j] = qt[j];
            c.rn_acc = rn;
            c.iters += 1;
            c.ls = 0;
            accepted = true;
        } else {
            c.ls += 1;
            c.t *= 0.5;
            for (int j = tid; j < n; j += nt) qt[j] = qa[j] + c.t * dq[j];
        }
    }
    if (accepted && !keep_dq) {
        if (!isfinite(c.rn_acc)) { c.status = 6; c.active = 0; }
        else if (c.rn_acc <= c.tol) { c.status = 0; c.active = 0; }
        else if (c.iters >= o.max_iter) { c.status = 5; c.active = 0; }
        else {
            // low-precision stiffness (BF16/TF32): an instance still iterating after ESC_ITERS
            // accepted steps gets the FP32-accurate assembly from its next evaluation on
            if (o.precision >= 2 && c.iters >= ESC_ITERS) c.acc_k = 1;
            __syncthreads();   // qa written above is read below by other threads
            if (!newton_direction(Bt, b, n, o.precision, A, x, &s_piv, red)) { c.status = 6; c.active = 0; }
            else {
                c.t = 1.0;
                c.ls = 0;
                for (int j = tid; j < n; j += nt) { dq[j] = x[j]; qt[j] = qa[j] + x[j]; }
            }
        }
    }
    __syncthreads();
    if (tid == 0) {
        Bt.ctl[b] = c;
        if (c.active) {
            const int pos = atomicAdd(&Bt.counts[1], 1);
            list_next[pos] = (int32_t)b;
        }
    }
}

// Tensor-core paths with a BF16/TF32 stiffness when the effective stiffness is wanted: after the
// residual of a Newton pass and before its assembly, an instance that this pass's solve will find
// converged (a trial evaluation in phase 1 that is accepted and meets ||r|| <= tol: the solve's
// test on the same norm) needs its stiffness only for Abar.  It is flagged for the FP32-accurate
// assembly now, instead of getting a low-precision K that would be discarded and an accurate one
// after the Newton loop.  The list is then reordered, the flagged instances (and those flagged
// earlier by the solve's escalation) last, so that the assembly CTAs, which take consecutive list
// positions, hold instances of one kind.  One warp per list position; tmp holds B entries.
__global__ void k_flag_final(Batch Bt, StepOpts o, int n, int32_t *tmp) {
    const int n_act = Bt.counts[0];
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n_act) return;   // whole warps leave together
    const int32_t b = Bt.list[w];
    const double rn = warp_residual_norm(Bt.r + (int64_t)b * n, n, lane);
    if (lane == 0) {
        Ctl &c = Bt.ctl[b];
        int flag = c.acc_k;
        if (c.phase == 1 && isfinite(rn) && rn <= c.tol && (c.ls >= o.max_ls || rn < c.rn_acc)) flag = 1;
        c.acc_k = flag;
        const int pos = flag ? n_act - 1 - atomicAdd(&Bt.counts[5], 1) : atomicAdd(&Bt.counts[4], 1);
        tmp[pos] = b;
    }
}

// the reordered list back into place; resets the partition positions for the next pass
__global__ void k_take_list(Batch Bt, const int32_t *__restrict__ tmp) {
    const int n_act = Bt.counts[0];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) { Bt.counts[4] = 0; Bt.counts[5] = 0; }
    if (i < n_act) Bt.list[i] = tmp[i];
}

void launch_flag_final(const Model &M, Batch Bt, const StepOpts &o, int32_t *tmp, cudaStream_t s) {
    k_flag_final<<<(int)((Bt.B * 32 + 255) / 256), 256, 0, s>>>(Bt, o, M.n, tmp);
    k_take_list<<<(int)((Bt.B + 255) / 256), 256, 0, s>>>(Bt, tmp);
}

// --------------------------------------------------------------------- finalize
// a11 sums of one instance in FP64: B = sum_i G_i^T Ahat_i [n][D2] and A0 = sum_i Xi_i^T Ahat_i
// [D4]; work = Ah [CHF][D4] | Gs [CHF][D2][n] (doubles).  Ends with Bm, A0 visible to the block.
template <int D>
__device__ void abar_sums_f64(const Model &M, const Batch &Bt, int64_t b, int CHF, double *Bm, double *A0,
                              double *Fm, double *work) {
    constexpr int D2 = D * D, D4 = D2 * D2;
    const int n = M.n, m = M.m, tid = threadIdx.x;
    double *Ah = work;
    double *Gs = Ah + (size_t)CHF * D4;
    const double *At = reinterpret_cast<const double *>(Bt.At);
    double bacc[4] = {0, 0, 0, 0};     // entries tid, tid+256, ... of Bm (n*D2 <= 1152)
    double aacc = 0.0;                 // entry tid of A0 (D4 <= 81)
    for (int c0 = 0; c0 < m; c0 += CHF) {
        const int ch = min(CHF, m - c0);
        __syncthreads();
        for (int e = tid; e < ch * D2; e += blockDim.x) {
            const int ii = e / D2, ar = e - ii * D2;
            const int a = ar / D, r = ar - a * D;
            double s = (a == r) ? 1.0 : 0.0;
            for (int k = 0; k < M.n_par; ++k)
                s += Bt.mu[b * M.n_par + k] * M.Gmu_T[((size_t)ar * M.n_par + k) * m + c0 + ii];
            Fm[ii * D2 + ar] = s;
        }
        for (int e = tid; e < ch * D2 * n; e += blockDim.x)
            Gs[e] = M.G_pt[(size_t)c0 * D2 * n + e];
        __syncthreads();
        for (int e = tid; e < ch * D4; e += blockDim.x) {
            const int ii = e / D4, rem = e - ii * D4;
            const int ar = rem / D2, kl = rem - ar * D2;
            const int k = kl / D, l = kl - k * D;
            double s = 0.0;
            for (int ss = 0; ss < D; ++ss)
                s += At[((size_t)b * D4 + ar * D2 + k * D + ss) * M.mA + c0 + ii] * Fm[ii * D2 + l * D + ss];
            Ah[e] = s;
        }
        __syncthreads();
        for (int q = 0; q < 4; ++q) {
            const int e = tid + q * blockDim.x;
            if (e < n * D2) {
                const int j = e / D2, kl = e - j * D2;
                double s = 0.0;
                for (int ii = 0; ii < ch; ++ii)
                    for (int ar = 0; ar < D2; ++ar) s += Gs[(ii * D2 + ar) * n + j] * Ah[ii * D4 + ar * D2 + kl];
                bacc[q] += s;
            }
        }
        if (tid < D4) {
            const int ij = tid / D2, kl = tid - ij * D2;
            const int ia = ij / D, jb = ij - ia * D;
            double s = 0.0;
            for (int ii = 0; ii < ch; ++ii)
                for (int r = 0; r < D; ++r) s += Fm[ii * D2 + jb * D + r] * Ah[ii * D4 + (ia * D + r) * D2 + kl];
            aacc += s;
        }
    }
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
        const int e = tid + q * blockDim.x;
        if (e < n * D2) Bm[e] = bacc[q];
    }
    if (tid < D4) A0[tid] = aacc;
    __syncthreads();
}

// the same sums from the FP32 tangent of the mixed-precision path, in FP32.  The tangent chunks
// (CHF points) are staged with cp.async one chunk ahead (double-buffered) and Ahat_i = At_i Xi_i
// is formed for the chunk in shared memory.  Thread (tj = tid % JG, pg = tid / JG) accumulates
// B[4 tj .. 4 tj + 3][0..D2) (36 FP32 accumulators in 3D) over the points pg, pg + NPG, ... of
// each chunk, reading G (FP32, shared by all instances and resident in L2) straight from global
// memory, so that each loaded value feeds D2 (G) or 4 (Ahat) multiply-adds; A0 is split over
// D4-thread point groups.  The group sums are added in a fixed order (in FP64).
// work (floats, 16-byte aligned) = As [2][D4][CHF] | Fm32 [2][CHF][D2] | Ah [CHF][D4]; the group
// sums reuse the work area.  CHF must be a multiple of 4.
constexpr int ABAR_JT = 4;   // columns j per thread in the FP32 B sums
__device__ __forceinline__ void cp_async16_f(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

template <int D>
__device__ void abar_sums_f32(const Model &M, const Batch &Bt, int64_t b, int CHF, double *Bm, double *A0,
                              float *work) {
    constexpr int D2 = D * D, D4 = D2 * D2, JT = ABAR_JT;
    const int n = M.n, m = M.m, mA = M.mA, tid = threadIdx.x;
    float *As[2], *Fm32[2];
    As[0] = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(work) + 15) & ~uintptr_t(15));
    As[1] = As[0] + (size_t)D4 * CHF;
    Fm32[0] = As[1] + (size_t)D4 * CHF;
    Fm32[1] = Fm32[0] + (size_t)CHF * D2;
    float *Ah = Fm32[1] + (size_t)CHF * D2;
    const float *At = reinterpret_cast<const float *>(Bt.At);
    const int JG = (n + JT - 1) / JT, NPG = blockDim.x / JG;
    const int tj = tid % JG, pg = tid / JG;
    const bool bact = pg < NPG, vec4 = (n & 3) == 0;
    const int AG = blockDim.x / D4, ag = tid / D4, ae = tid - ag * D4;   // A0: AG point groups
    const int nch = (m + CHF - 1) / CHF;
    auto stage = [&](int c) {
        const int c0 = c * CHF, ch = min(CHF, m - c0), buf = c & 1;
        const int q4 = CHF / 4;
        for (int e = tid; e < D4 * q4; e += blockDim.x) {   // At rows: CHF floats from c0, inside the row
            const int ce = e / q4, qq = e - ce * q4;
            if (c0 + 4 * qq < mA)
                cp_async16_f(As[buf] + (size_t)ce * CHF + 4 * qq, At + ((size_t)b * D4 + ce) * mA + c0 + 4 * qq);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        for (int e = tid; e < ch * D2; e += blockDim.x) {
            const int ii = e / D2, ar = e - ii * D2;
            const int a = ar / D, r = ar - a * D;
            double s = (a == r) ? 1.0 : 0.0;
            for (int k = 0; k < M.n_par; ++k)
                s += Bt.mu[b * M.n_par + k] * M.Gmu_T[((size_t)ar * M.n_par + k) * m + c0 + ii];
            Fm32[buf][ii * D2 + ar] = (float)s;
        }
    };
    float acc[JT][D2];
#pragma unroll
    for (int t = 0; t < JT; ++t)
#pragma unroll
        for (int kl = 0; kl < D2; ++kl) acc[t][kl] = 0.f;
    float aacc = 0.f;
    stage(0);
    for (int c = 0; c < nch; ++c) {
        const int c0 = c * CHF, ch = min(CHF, m - c0), buf = c & 1;
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        if (c + 1 < nch) stage(c + 1);
        const float *as = As[buf], *fm = Fm32[buf];
        for (int e = tid; e < CHF * D4; e += blockDim.x) {   // consecutive threads: consecutive points
            const int ii = e % CHF, rem = e / CHF;
            if (ii >= ch) continue;
            const int ar = rem / D2, kl = rem - ar * D2;
            const int k = kl / D, l = kl - k * D;
            float sacc = 0.f;
#pragma unroll
            for (int ss = 0; ss < D; ++ss)
                sacc = fmaf(as[(ar * D2 + k * D + ss) * CHF + ii], fm[ii * D2 + l * D + ss], sacc);
            Ah[ii * D4 + rem] = sacc;
        }
        __syncthreads();
        if (bact)
            for (int ii = pg; ii < ch; ii += NPG) {
                const float *ah = Ah + ii * D4;
                const float *g = M.G32_pt + (size_t)(c0 + ii) * D2 * n + JT * tj;
#pragma unroll
                for (int ar = 0; ar < D2; ++ar) {
                    float gv[JT];
                    if (vec4) {
                        const float4 t4 = __ldg(reinterpret_cast<const float4 *>(g + (size_t)ar * n));
                        gv[0] = t4.x; gv[1] = t4.y; gv[2] = t4.z; gv[3] = t4.w;
                    } else {
#pragma unroll
                        for (int t = 0; t < JT; ++t) gv[t] = (JT * tj + t < n) ? __ldg(g + (size_t)ar * n + t) : 0.f;
                    }
#pragma unroll
                    for (int kl = 0; kl < D2; ++kl) {
                        const float av = ah[ar * D2 + kl];
#pragma unroll
                        for (int t = 0; t < JT; ++t) acc[t][kl] = fmaf(gv[t], av, acc[t][kl]);
                    }
                }
            }
        if (ag < AG) {
            const int ij = ae / D2, kl = ae - ij * D2;
            const int ia = ij / D, jb = ij - ia * D;
            for (int ii = ag; ii < ch; ii += AG)
#pragma unroll
                for (int r = 0; r < D; ++r) aacc = fmaf(fm[ii * D2 + jb * D + r], Ah[ii * D4 + (ia * D + r) * D2 + kl], aacc);
        }
    }
    __syncthreads();
    float *red = As[0];   // [NPG][n][D2], then [AG][D4]
    if (bact)
#pragma unroll
        for (int t = 0; t < JT; ++t) {
            const int j = JT * tj + t;
            if (j < n)
#pragma unroll
                for (int kl = 0; kl < D2; ++kl) red[((size_t)pg * n + j) * D2 + kl] = acc[t][kl];
        }
    __syncthreads();
    for (int e = tid; e < n * D2; e += blockDim.x) {
        double sacc = 0.0;
        for (int g = 0; g < NPG; ++g) sacc += (double)red[(size_t)g * n * D2 + e];
        Bm[e] = sacc;
    }
    __syncthreads();
    if (ag < AG) red[ag * D4 + ae] = aacc;
    __syncthreads();
    if (tid < D4) {
        double sacc = 0.0;
        for (int g = 0; g < AG; ++g) sacc += (double)red[g * D4 + tid];
        A0[tid] = sacc;
    }
    __syncthreads();
}

// Ahat part of the effective tangent: AU = (A0 - B^T K^-1 B) / |Omega| with the factor of K at
// the solution (K* = K), factored and solved by the block in arithmetic T (FP64 on the FP64
// path; FP32 on the mixed path, whose K, B and A0 carry FP32-level errors already)
template <int D, typename T>
__device__ void schur_abar(const Model &M, const Batch &Bt, int64_t b, const double *Bm, const double *A0,
                           unsigned char *work, double *AU) {
    constexpr int D2 = D * D, D4 = D2 * D2;
    const int n = M.n, tid = threadIdx.x;
    const int ld = n + 1;                    // padded rows and right-hand sides: distinct banks
    T *Aw = reinterpret_cast<T *>(work);     // [n][n + 1]
    T *Zs = Aw + (size_t)n * ld;             // [D2][n + 1]
    int *piv = reinterpret_cast<int *>(Zs + (size_t)ld * D2);
    const double *Kb = Bt.K + (size_t)b * n * n;
    // FP32 copies by integer operations on the bit patterns (mantissa truncation: the FP32 path's
    // K and B carry FP32-level errors already), not by conversion instructions on the FP64 pipe
    for (int e = tid; e < n * n; e += blockDim.x) Aw[(e / n) * ld + e % n] = to_tangent<T>(Kb[e]);
    for (int e = tid; e < n * D2; e += blockDim.x) {
        const int kl = e / n, j = e - kl * n;
        Zs[kl * ld + j] = to_tangent<T>(Bm[j * D2 + kl]);
    }
    __syncthreads();
    const bool ok = block_lu_solve<T>(Aw, n, ld, Zs, ld, D2, piv);
    if (tid < D4) {
        const int ij = tid / D2, kl = tid - ij * D2;
        double s = A0[tid];
        if (ok)
            for (int j = 0; j < n; ++j) s -= Bm[j * D2 + ij] * widen(Zs[(size_t)kl * ld + j]);
        else
            s = NAN;
        AU[tid] = s / M.omega;
    }
    __syncthreads();
}

template <int D, typename TT>
__global__ void __launch_bounds__(256, 4) k_finalize(Model M, Batch Bt, StepOpts o, double *__restrict__ Pbar,
                                                  double *__restrict__ Abar, void *info_v, int CHF) {
    constexpr int D2 = D * D, D4 = D2 * D2;
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t b = blockIdx.x;
    const int n = M.n, m = M.m, tid = threadIdx.x;
    const Ctl c = Bt.ctl[b];
    __shared__ double wred[8][D2 + 1];
    __shared__ double PU[D2], AU[D4], Rb[D2], Ub[D2];
    __shared__ int ny_s;
    const int lane = tid & 31, wid = tid >> 5;
    // n_yield of the last evaluated state and the partial sums of Pbar_U (one pass, fixed order)
    double ps[D2 + 1];
#pragma unroll
    for (int cc = 0; cc <= D2; ++cc) ps[cc] = 0.0;
    for (int i = tid; i < m; i += blockDim.x) {
        ps[D2] += Bt.pl[b * m + i];
#pragma unroll
        for (int cc = 0; cc < D2; ++cc) ps[cc] += Bt.wP[((size_t)b * D2 + cc) * m + i];
    }
#pragma unroll
    for (int cc = 0; cc <= D2; ++cc)
        for (int off = 16; off > 0; off >>= 1) ps[cc] += __shfl_xor_sync(0xffffffffu, ps[cc], off);
    if (lane == 0)
        for (int cc = 0; cc <= D2; ++cc) wred[wid][cc] = ps[cc];
    __syncthreads();
    if (tid <= D2) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wred[w][tid];
        if (tid == D2) ny_s = (int)t;
        else PU[tid] = t / M.omega;
    }
    __syncthreads();
    struct Info { int32_t iters, evals, status, n_yield; double res0, res; };
    Info *info = reinterpret_cast<Info *>(info_v);
    if (tid == 0 && info) {
        Info f;
        f.iters = c.iters; f.evals = c.evals; f.status = c.status; f.n_yield = ny_s;
        f.res0 = c.r0; f.res = c.rn_acc;
        info[b] = f;
    }
    if (c.status != 0) {
        for (int e = tid; e < D2; e += blockDim.x) Pbar[b * D2 + e] = NAN;
        if (Abar && o.want_abar)
            for (int e = tid; e < D4; e += blockDim.x) Abar[b * D4 + e] = NAN;
        return;
    }
    // a10: Pbar_U = |Omega|^-1 sum_i wJ P_i (reduced above)
    if (tid < D2) { Rb[tid] = Bt.Rbar[b * D2 + tid]; Ub[tid] = Bt.Ubar[b * D2 + tid]; }
    __syncthreads();

    if (Abar && o.want_abar && Bt.err && *Bt.err) {
        // a tensor-core assembly of this step gave up on a wait: K at the solution is not
        // trustworthy, so Abar is not produced (Pbar and the history come from exact residuals)
        for (int e = tid; e < D4; e += blockDim.x) Abar[b * D4 + e] = NAN;
    } else if (Abar && o.want_abar) {
        // a11: B = sum_i G_i^T Ahat_i,  A0 = sum_i wJ A_i, Ahat_i = At_i Xi_i (Xi: dH = E_kl F_mu)
        double *Bm = reinterpret_cast<double *>(smem);              // [n][D2]
        double *A0 = Bm + (size_t)n * D2;                          // [D4]
        double *Fm = A0 + D4;                                      // [CHF][D2]
        // FP32 path: the sums' staging area starts at Fm (its FP64 chunk is not used)
        unsigned char *work = reinterpret_cast<unsigned char *>(sizeof(TT) == 8 ? Fm + (size_t)CHF * D2 : Fm);
        if (Bt.Bsum) {
            // B and A0 from the tensor cores (k_abar_tc3: Bsum[b] = [B (n x D2) | A0 (D4)])
            const double *src = Bt.Bsum + (size_t)b * (n * D2 + D4);
            for (int e = tid; e < n * D2; e += blockDim.x) Bm[e] = src[e];
            for (int e = tid; e < D4; e += blockDim.x) A0[e] = src[n * D2 + e];
            __syncthreads();
        } else if (sizeof(TT) == 8) {
            abar_sums_f64<D>(M, Bt, b, CHF, Bm, A0, Fm, reinterpret_cast<double *>(work));
        } else {
            abar_sums_f32<D>(M, Bt, b, CHF, Bm, A0, reinterpret_cast<float *>(Fm));
        }
        // Schur complement with the factor of K at the solution (K* = K)
        if (sizeof(TT) == 8) schur_abar<D, double>(M, Bt, b, Bm, A0, work, AU);
        else schur_abar<D, float>(M, Bt, b, Bm, A0, work, AU);
        // rotate back: Abar = d(R Pbar_U(R^T Fbar))/dFbar
        if (tid < D2) {
            const int k = tid / D, l = tid - k * D;
            double Mm[9] = {0}, W[9] = {0}, dU[9], dPU[9], t[9];
            for (int i = 0; i < D; ++i) Mm[i * D + l] = Rb[k * D + i];
            double trU = 0.0;
            for (int i = 0; i < D; ++i) trU += Ub[i * D + i];
            if (o.polar) {
                if (D == 2) {
                    const double om = (Mm[2] - Mm[1]) / trU;
                    W[1] = -om; W[2] = om;
                } else {
                    const double a0 = Mm[7] - Mm[5], a1 = Mm[2] - Mm[6], a2 = Mm[3] - Mm[1];
                    double S[9];
                    for (int e = 0; e < 9; ++e) S[e] = -Ub[e];
                    S[0] += trU; S[4] += trU; S[8] += trU;
                    const double c00 = S[4] * S[8] - S[5] * S[7], c01 = S[5] * S[6] - S[3] * S[8], c02 = S[3] * S[7] - S[4] * S[6];
                    const double det = S[0] * c00 + S[1] * c01 + S[2] * c02;
                    const double Si[9] = {c00 / det, (S[2] * S[7] - S[1] * S[8]) / det, (S[1] * S[5] - S[2] * S[4]) / det,
                                          c01 / det, (S[0] * S[8] - S[2] * S[6]) / det, (S[2] * S[3] - S[0] * S[5]) / det,
                                          c02 / det, (S[1] * S[6] - S[0] * S[7]) / det, (S[0] * S[4] - S[1] * S[3]) / det};
                    const double w0 = Si[0] * a0 + Si[1] * a1 + Si[2] * a2;
                    const double w1 = Si[3] * a0 + Si[4] * a1 + Si[5] * a2;
                    const double w2 = Si[6] * a0 + Si[7] * a1 + Si[8] * a2;
                    W[1] = -w2; W[2] = w1; W[3] = w2; W[5] = -w0; W[6] = -w1; W[7] = w0;
                }
            }
            for (int i = 0; i < D; ++i)
                for (int j = 0; j < D; ++j) {
                    double s = 0.0;
                    for (int cc = 0; cc < D; ++cc) s += W[i * D + cc] * Ub[cc * D + j];
                    dU[i * D + j] = Mm[i * D + j] - s;
                }
            for (int ij = 0; ij < D2; ++ij) {
                double s = 0.0;
                for (int cc = 0; cc < D2; ++cc) s += AU[ij * D2 + cc] * dU[cc];
                dPU[ij] = s;
            }
            for (int i = 0; i < D; ++i)
                for (int j = 0; j < D; ++j) {
                    double s = dPU[i * D + j];
                    for (int cc = 0; cc < D; ++cc) s += W[i * D + cc] * PU[cc * D + j];
                    t[i * D + j] = s;
                }
            for (int i = 0; i < D; ++i)
                for (int j = 0; j < D; ++j) {
                    double s = 0.0;
                    for (int cc = 0; cc < D; ++cc) s += Rb[i * D + cc] * t[cc * D + j];
                    Abar[b * D4 + (i * D + j) * D2 + tid] = s;
                }
        }
    }
    if (tid < D2) {
        const int i = tid / D, j = tid - i * D;
        double s = 0.0;
        for (int cc = 0; cc < D; ++cc) s += Rb[i * D + cc] * PU[cc * D + j];
        Pbar[b * D2 + tid] = s;
    }
    // a12: commit
    const int ncp = M.ncp;
    for (int e = tid; e < ncp * m; e += blockDim.x) Bt.cp[(size_t)b * ncp * m + e] = Bt.cp_tr[(size_t)b * ncp * m + e];
    for (int e = tid; e < m; e += blockDim.x) Bt.xi[(size_t)b * m + e] = Bt.xi_tr[(size_t)b * m + e];
    for (int j = tid; j < n; j += blockDim.x) {
        const double qa = Bt.q_acc[b * n + j];
        Bt.dq_prev[b * n + j] = qa - Bt.q_n[b * n + j];
        Bt.q_n[b * n + j] = qa;
    }
    if (Bt.U_prev && tid < D2) Bt.U_prev[b * D2 + tid] = Ub[tid];
}

// ---------------------------------------------------------------- graph loop
// device-driven Newton loop: copy the next active list into the current one, then set the
// while-node condition of the captured step graph (more passes iff instances remain active
// and the pass cap is not reached)
__global__ void k_copy_list(const int32_t *__restrict__ src, int32_t *__restrict__ dst, const int32_t *counts,
                            int64_t B) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B && i < counts[1]) dst[i] = src[i];
}

__global__ void k_advance_cond(int32_t *counts, cudaGraphConditionalHandle h, int max_pass) {
    counts[0] = counts[1];
    counts[1] = 0;
    counts[2] += 1;
    cudaGraphSetConditional(h, (counts[0] > 0 && counts[2] < max_pass) ? 1u : 0u);
}

__global__ void k_reset_pass(int32_t *counts) { counts[2] = 0; }

void launch_graph_advance(Batch Bt, const int32_t *list_next, cudaGraphConditionalHandle h, int max_pass,
                          cudaStream_t s) {
    k_copy_list<<<(int)((Bt.B + 255) / 256), 256, 0, s>>>(list_next, Bt.list, Bt.counts, Bt.B);
    k_advance_cond<<<1, 1, 0, s>>>(Bt.counts, h, max_pass);
}

void launch_reset_pass(Batch Bt, cudaStream_t s) { k_reset_pass<<<1, 1, 0, s>>>(Bt.counts); }

__global__ void k_iota_list(Batch Bt) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < Bt.B) Bt.list[b] = (int32_t)b;
    if (b == 0) { Bt.counts[0] = (int32_t)Bt.B; Bt.counts[1] = 0; }
}

void launch_all_active(Batch Bt, cudaStream_t s) {
    k_iota_list<<<(int)((Bt.B + 255) / 256), 256, 0, s>>>(Bt);
}

// compacted list of the converged instances (status OK) into list / counts[0]
__global__ void k_list_converged(Batch Bt) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= Bt.B) return;
    if (Bt.ctl[b].status == 0) {
        const int pos = atomicAdd(&Bt.counts[0], 1);
        Bt.list[pos] = (int32_t)b;
    }
}

void launch_list_converged(Batch Bt, cudaStream_t s) {
    cudaMemsetAsync(Bt.counts, 0, 8, s);
    k_list_converged<<<(int)((Bt.B + 255) / 256), 256, 0, s>>>(Bt);
}

// learned start: q_trial = q_acc = q_n + (q_n - q_{n-1}) + predicted correction
__global__ void k_add_pred(Batch Bt, int n, const double *__restrict__ pred) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Bt.B * n) return;
    const double q = Bt.q_n[e] + Bt.dq_prev[e] + pred[e];
    Bt.q_trial[e] = q;
    Bt.q_acc[e] = q;
}

void launch_add_pred(Batch Bt, int n, const double *pred, cudaStream_t s) {
    const int64_t tot = Bt.B * n;
    k_add_pred<<<(int)((tot + 255) / 256), 256, 0, s>>>(Bt, n, pred);
}

// ----------------------------------------------------------------- host launchers
// the residual of a mixed-precision step comes from the double-float force kernel (launch_force)
// unless the model has no split image of G or the step asks for the FP64 residual
bool separate_force(const Model &M, const StepOpts &o) { return o.precision >= 1 && M.Gdf && !o.fp64_residual; }

template <int D, int TM>
static int launch_assemble(const Model &M, Batch Bt, const StepOpts &o, cudaStream_t s) {
    constexpr int D2 = D * D, D4 = D2 * D2;
    const int NT = (M.n + TM - 1) / TM, np = NT * TM;
    const int nup = NT * (NT + 1) / 2;
    int NG = nup >= 256 ? 1 : 256 / nup;
    const int nthreads = ((NG * nup + 31) / 32) * 32;
    if (nthreads > 256 || nthreads < M.n) return -1;
    const int tksz = o.precision == 0 ? 8 : 4;
    auto smem_for = [&](int CH) {
        size_t bytes = (size_t)CH * D2 * np * 8 + (size_t)CH * D2 * np * tksz + (size_t)CH * D4 * tksz + 16 +
                       (size_t)CH * D2 * 8 + (o.precision == 0 ? 0 : (size_t)CH * D2 * np * tksz);
        const size_t red = (size_t)NG * np * np * tksz;
        return bytes > red ? bytes : red;
    };
    int CH = 64;
    while (CH > 1 && smem_for(CH) > 96 * 1024) CH /= 2;
    if (o.asm_ch > 0) {
        if (smem_for(o.asm_ch) > 200 * 1024) return -1;
        CH = o.asm_ch;
    }
    const size_t sm = smem_for(CH);
    if (o.precision == 0) {
        cudaFuncSetAttribute(k_assemble<D, double, TM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_assemble<D, double, TM><<<(int)Bt.B, nthreads, sm, s>>>(M, Bt, CH, NG, 1);
    } else {
        cudaFuncSetAttribute(k_assemble<D, float, TM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_assemble<D, float, TM><<<(int)Bt.B, nthreads, sm, s>>>(M, Bt, CH, NG, separate_force(M, o) ? 0 : 1);
    }
    return 0;
}

template <int D>
static int launch_kernels_t(int which, const Model &M, Batch Bt, const StepOpts &o, int32_t *list_next,
                            cudaStream_t s) {
    if (which == 1) {
        const int64_t nthr = Bt.B * (int64_t)M.m;
        const int blk = 128;
        const int grid = (int)((nthr + blk - 1) / blk);
        if (o.precision == 0) k_constitutive<D, double><<<grid, blk, 0, s>>>(M, Bt);
        else k_constitutive<D, float><<<grid, blk, 0, s>>>(M, Bt);
        return 0;
    }
    if (which == 2) {
        if (o.asm_tm > 0) {
            const int NT = (M.n + o.asm_tm - 1) / o.asm_tm;
            if (NT * (NT + 1) / 2 > 256) return -1;
            return o.asm_tm == 2 ? launch_assemble<D, 2>(M, Bt, o, s)
                 : o.asm_tm == 4 ? launch_assemble<D, 4>(M, Bt, o, s)
                 : o.asm_tm == 8 ? launch_assemble<D, 8>(M, Bt, o, s) : -1;
        }
        // tile edge TM: the smallest of 2, 4, 8 for which one upper-triangular tile per thread fits 256 threads
        const int tms[3] = {2, 4, 8};
        for (int q = 0; q < 3; ++q) {
            const int TMv = tms[q];
            const int NT = (M.n + TMv - 1) / TMv;
            if (NT * (NT + 1) / 2 <= 256 && (D == 3 || TMv >= 2)) {
                if (D == 3 && TMv == 2 && M.n > 16) continue;   // keep 3D tiles >= 4 for register reuse
                return TMv == 2 ? launch_assemble<D, 2>(M, Bt, o, s)
                     : TMv == 4 ? launch_assemble<D, 4>(M, Bt, o, s)
                                : launch_assemble<D, 8>(M, Bt, o, s);
            }
        }
        return -1;
    }
    if (which == 3) {
        const size_t sms = solve_region_bytes(M.n, o.precision) + (size_t)M.n * 8 + (size_t)M.n * 4 + 16;
        cudaFuncSetAttribute(k_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sms);
        // n <= 32: one warp per instance (its block barriers cost next to nothing and twice as many
        // instances are resident per SM); the arithmetic and its order do not depend on the width
        k_solve<<<(int)Bt.B, M.n <= 32 ? 32 : SOLVE_THREADS, sms, s>>>(M, Bt, o, list_next);
        return 0;
    }
    if (which == 5) {
        k_advance<<<1, 1, 0, s>>>(Bt.counts);
        return 0;
    }
    return -1;
}

// which: 1 constitutive, 2 assemble, 3 solve, 5 advance
int launch_kernel(int which, const Model &M, Batch Bt, const StepOpts &o, int32_t *list_next, cudaStream_t s) {
    return M.d == 2 ? launch_kernels_t<2>(which, M, Bt, o, list_next, s)
                    : launch_kernels_t<3>(which, M, Bt, o, list_next, s);
}

int launch_start(const Model &M, Batch Bt, const double *Fbar, const StepOpts &o, const double *dq_pred,
                 cudaStream_t s) {
    const int blk = 128, grid = (int)((Bt.B + blk - 1) / blk);
    if (M.d == 2) k_start<2><<<grid, blk, 0, s>>>(M, Bt, Fbar, o, dq_pred);
    else k_start<3><<<grid, blk, 0, s>>>(M, Bt, Fbar, o, dq_pred);
    k_set_counts<<<1, 1, 0, s>>>(Bt.counts, Bt.B);
    return 0;
}

// ------------------------------------------------------------------ shape sensitivities
// dPbar/dmu_k (Eq. eff_sensitivities_full) at the converged state of the last step, one CTA per
// instance, in arithmetic T (FP64 after an FP64 step, FP32 after a mixed-precision step, whose
// tangent is FP32).  With M_k = -H F_mu^-1 Gmu_k (so that dF/dmu_k at fixed a = M_k F_mu^-1),
// tr_k = tr(F_mu^-1 Gmu_k) (= d ln|det F_mu| / dmu_k) and the stored pull-backs v, wP and At:
//   dv_k = tr_k v + At vec(M_k) - V Gmu_k^T F_mu^-T            (derivative of v at fixed a)
//   z_k = sum_i G_i^T dv_k,i ;  K dq_k = -z_k                  (reduced fluctuation sensitivity)
//   dPbar_U/dmu_k = |Omega|^-1 sum_i [ tr_k wP + Xi^T At vec(G_i dq_k + M_k) ],  Xi^T y = (I x F_mu) y
//   dPbar/dmu_k = Rbar dPbar_U/dmu_k.
// Points go in chunks of SENS_CH: one thread per point forms dv (shared memory) and its share of
// the tr_k wP and Xi^T At vec(M_k) sums; then thread (j, k) adds G^T dv over the chunk.  The
// partial sums are added in a fixed order.
constexpr int SENS_CH = 256;
constexpr int SENS_THREADS = 256;
constexpr int SENS_MAXP = 3;   // geometry parameters

template <int D, typename T>
__global__ void __launch_bounds__(SENS_THREADS) k_sensitivity(Model M, Batch Bt, double *__restrict__ out) {
    constexpr int D2 = D * D, D4 = D2 * D2;
    constexpr int NA = D2 * SENS_MAXP;   // per-thread partial sums of dPbar_U/dmu_k
    extern __shared__ __align__(16) unsigned char smem[];
    const int64_t b = blockIdx.x;
    const int n = M.n, m = M.m, np = M.n_par, tid = threadIdx.x;
    const int ld = n + 1;
    const Ctl c = Bt.ctl[b];
    if (c.status != 0 || np > SENS_MAXP) {
        for (int e = tid; e < D2 * np; e += blockDim.x) out[b * D2 * np + e] = NAN;
        return;
    }
    // layout: qs [n] | zs [SENS_MAXP][ld] | region (dv chunk | partial sums | LU of K)
    T *qs = reinterpret_cast<T *>(smem);
    T *zs = qs + n;
    T *reg = zs + SENS_MAXP * ld;
    T *dv = reg;                                  // [SENS_CH][SENS_MAXP][D2]
    T *red = reg;                                 // [SENS_CH][NA] (after the chunks)
    T *Ks = reg;                                  // [n][ld] (after the reduction)
    __shared__ int s_piv;
    __shared__ double mu_s[SENS_MAXP];
    const T *At = reinterpret_cast<const T *>(Bt.At);
    const T *Gp = (sizeof(T) == 8) ? reinterpret_cast<const T *>(M.G_pt) : reinterpret_cast<const T *>(M.G32_pt);
    // [d2][n][m] copy of G: per-point sums over j read consecutive points in consecutive threads
    const T *Gt = (sizeof(T) == 8) ? reinterpret_cast<const T *>(M.G_T) : reinterpret_cast<const T *>(M.G32h_T);
    for (int j = tid; j < n; j += blockDim.x) qs[j] = (T)Bt.q_n[b * n + j];
    for (int e = tid; e < SENS_MAXP * ld; e += blockDim.x) zs[e] = T(0);
    if (tid < np) mu_s[tid] = Bt.mu[b * np + tid];
    __syncthreads();

    // per-point geometry (F_mu, its inverse, Gmu_k) of point i
    auto geometry = [&](int i, T Fm[3][3], T Fmi[3][3], T Gk[SENS_MAXP][3][3]) {
        double F[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
        for (int a = 0; a < D; ++a)
            for (int r = 0; r < D; ++r) {
                double s0 = (a == r) ? 1.0 : 0.0;
                for (int k = 0; k < np; ++k) {
                    const double g = M.Gmu_T[((size_t)(a * D + r) * np + k) * m + i];
                    s0 += mu_s[k] * g;
                    Gk[k][a][r] = (T)g;
                }
                F[a][r] = s0;
            }
        double I[3][3];
        if (D == 2) {
            const double id = 1.0 / (F[0][0] * F[1][1] - F[0][1] * F[1][0]);
            I[0][0] = F[1][1] * id; I[0][1] = -F[0][1] * id; I[1][0] = -F[1][0] * id; I[1][1] = F[0][0] * id;
        } else {
            const double c00 = F[1][1] * F[2][2] - F[1][2] * F[2][1], c01 = F[1][2] * F[2][0] - F[1][0] * F[2][2],
                         c02 = F[1][0] * F[2][1] - F[1][1] * F[2][0];
            const double id = 1.0 / (F[0][0] * c00 + F[0][1] * c01 + F[0][2] * c02);
            I[0][0] = c00 * id; I[1][0] = c01 * id; I[2][0] = c02 * id;
            I[0][1] = (F[0][2] * F[2][1] - F[0][1] * F[2][2]) * id;
            I[1][1] = (F[0][0] * F[2][2] - F[0][2] * F[2][0]) * id;
            I[2][1] = (F[0][1] * F[2][0] - F[0][0] * F[2][1]) * id;
            I[0][2] = (F[0][1] * F[1][2] - F[0][2] * F[1][1]) * id;
            I[1][2] = (F[0][2] * F[1][0] - F[0][0] * F[1][2]) * id;
            I[2][2] = (F[0][0] * F[1][1] - F[0][1] * F[1][0]) * id;
        }
        for (int a = 0; a < D; ++a)
            for (int r = 0; r < D; ++r) { Fm[a][r] = (T)F[a][r]; Fmi[a][r] = (T)I[a][r]; }
    };
    // y_k[(a,r)] = sum_{(c,s)} At_i[(a,r),(c,s)] X_k[(c,s)], then acc_k[(a,t)] += sum_r Fm[t][r] y_k[(a,r)]
    // (acc_k at acc + k D2; each At entry read once for all k)
    auto at_apply = [&](int i, const T X[SENS_MAXP][D2], T Fm[3][3], T *acc) {
        for (int ar = 0; ar < D2; ++ar) {
            T y[SENS_MAXP];
#pragma unroll
            for (int k = 0; k < SENS_MAXP; ++k) y[k] = T(0);
#pragma unroll
            for (int cs = 0; cs < D2; ++cs) {
                const T av = At[((size_t)b * D4 + ar * D2 + cs) * M.mA + i];
#pragma unroll
                for (int k = 0; k < SENS_MAXP; ++k) y[k] += av * X[k][cs];
            }
            const int a = ar / D, r = ar - a * D;
#pragma unroll
            for (int k = 0; k < SENS_MAXP; ++k)
#pragma unroll
                for (int t = 0; t < D; ++t) acc[k * D2 + a * D + t] += Fm[t][r] * y[k];
        }
    };

    T acc[NA];
#pragma unroll
    for (int e = 0; e < NA; ++e) acc[e] = T(0);
    const int nch = (m + SENS_CH - 1) / SENS_CH;
    for (int ch = 0; ch < nch; ++ch) {
        const int i0 = ch * SENS_CH, cnt = min(SENS_CH, m - i0);
        if (tid < cnt) {
            const int i = i0 + tid;
            T Fm[3][3], Fmi[3][3], Gk[SENS_MAXP][3][3];
            geometry(i, Fm, Fmi, Gk);
            T H[D2];
#pragma unroll
            for (int cc = 0; cc < D2; ++cc) H[cc] = T(0);
            for (int j = 0; j < n; ++j) {
                const T qj = qs[j];
#pragma unroll
                for (int cc = 0; cc < D2; ++cc) H[cc] += Gt[((size_t)cc * n + j) * m + i] * qj;
            }
            T V[D2], WP[D2];
#pragma unroll
            for (int cc = 0; cc < D2; ++cc) {
                V[cc] = (T)Bt.v[((size_t)b * D2 + cc) * m + i];
                WP[cc] = (T)Bt.wP[((size_t)b * D2 + cc) * m + i];
            }
            // M_k = -H F_mu^-1 Gmu_k and tr_k = tr(F_mu^-1 Gmu_k) for every k, then one pass over
            // the rows of At_i gives y_k = At vec(M_k) for all k (each At entry read once)
            T Mk[SENS_MAXP][D2], trk[SENS_MAXP];
            for (int k = 0; k < SENS_MAXP; ++k) {
                T FG[3][3];
                trk[k] = T(0);
                for (int a = 0; a < D; ++a)
                    for (int r = 0; r < D; ++r) {
                        T s0 = T(0);
                        if (k < np)
                            for (int t = 0; t < D; ++t) s0 += Fmi[a][t] * Gk[k][t][r];
                        FG[a][r] = s0;
                    }
                for (int a = 0; a < D; ++a) trk[k] += FG[a][a];
                for (int a = 0; a < D; ++a)
                    for (int r = 0; r < D; ++r) {
                        T s0 = T(0);
                        for (int t = 0; t < D; ++t) s0 -= H[a * D + t] * FG[t][r];
                        Mk[k][a * D + r] = s0;
                    }
            }
            for (int ar = 0; ar < D2; ++ar) {
                T yk[SENS_MAXP];
#pragma unroll
                for (int k = 0; k < SENS_MAXP; ++k) yk[k] = T(0);
#pragma unroll
                for (int cs = 0; cs < D2; ++cs) {
                    const T av = At[((size_t)b * D4 + ar * D2 + cs) * M.mA + i];
#pragma unroll
                    for (int k = 0; k < SENS_MAXP; ++k) yk[k] += av * Mk[k][cs];
                }
                const int a = ar / D, r = ar - a * D;
                for (int k = 0; k < np; ++k) {
                    // Xi^T image of y into the sums, and dv_k = tr_k v + y - V Gmu_k^T F_mu^-T
                    for (int t = 0; t < D; ++t) acc[k * D2 + a * D + t] += Fm[t][r] * yk[k];
                    T w3 = T(0);
                    for (int s1 = 0; s1 < D; ++s1) {
                        T gf = T(0);
                        for (int t = 0; t < D; ++t) gf += Gk[k][t][s1] * Fmi[r][t];
                        w3 += V[a * D + s1] * gf;
                    }
                    dv[((size_t)tid * SENS_MAXP + k) * D2 + ar] = trk[k] * V[ar] + yk[k] - w3;
                    acc[k * D2 + ar] += trk[k] * WP[ar];
                }
            }
        }
        __syncthreads();
        // z_k[j] += sum over the chunk's points and components of G[i][c][j] dv_k[i][c]
        for (int e = tid; e < n * np; e += blockDim.x) {
            const int k = e / n, j = e - k * n;
            T z = T(0);
            for (int ii = 0; ii < cnt; ++ii)
#pragma unroll
                for (int cc = 0; cc < D2; ++cc)
                    z += Gp[((size_t)(i0 + ii) * D2 + cc) * n + j] * dv[((size_t)ii * SENS_MAXP + k) * D2 + cc];
            zs[k * ld + j] += z;
        }
        __syncthreads();
    }
    // K dq_k = -z_k with the factor of K at the solution (K* = K)
    for (int e = tid; e < np * ld; e += blockDim.x) zs[e] = -zs[e];
    for (int e = tid; e < n * n; e += blockDim.x) Ks[(e / n) * ld + e % n] = (T)Bt.K[(size_t)b * n * n + e];
    __syncthreads();
    const bool ok = block_lu_solve<T>(Ks, n, ld, zs, ld, np, &s_piv);
    __syncthreads();
    // U_k: sum_i Xi^T At vec(G_i dq_k) (into the same accumulators as T)
    for (int i = tid; i < m && ok; i += blockDim.x) {
        T Fm[3][3], Fmi[3][3], Gk[SENS_MAXP][3][3];
        geometry(i, Fm, Fmi, Gk);
        T X[SENS_MAXP][D2];
#pragma unroll
        for (int k = 0; k < SENS_MAXP; ++k)
#pragma unroll
            for (int cc = 0; cc < D2; ++cc) X[k][cc] = T(0);
        for (int j = 0; j < n; ++j) {
            T dj[SENS_MAXP];
#pragma unroll
            for (int k = 0; k < SENS_MAXP; ++k) dj[k] = k < np ? zs[k * ld + j] : T(0);
#pragma unroll
            for (int cc = 0; cc < D2; ++cc) {
                const T g = Gt[((size_t)cc * n + j) * m + i];
#pragma unroll
                for (int k = 0; k < SENS_MAXP; ++k) X[k][cc] += g * dj[k];
            }
        }
        at_apply(i, X, Fm, acc);
    }
    // fixed-order reduction of the per-thread sums: butterfly within each warp, then the warps in
    // order (the LU region is free again)
    __syncthreads();
    const int lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    for (int e = 0; e < NA; ++e) {
        T v = acc[e];
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) red[(size_t)wid * NA + e] = v;
    }
    __syncthreads();
    __shared__ double dPU[D2 * SENS_MAXP];
    if (tid < D2 * np) {
        const int k = tid / D2, at = tid - k * D2;
        double sacc = 0.0;
        for (int w2 = 0; w2 < nw; ++w2) sacc += (double)red[(size_t)w2 * NA + k * D2 + at];
        dPU[tid] = sacc / M.omega;
    }
    __syncthreads();
    // rotate back: dPbar/dmu_k = Rbar dPbar_U/dmu_k
    if (tid < D2 * np) {
        const int k = tid / D2, ij = tid - k * D2, ii = ij / D, jj = ij - ii * D;
        double s0 = 0.0;
        for (int cc = 0; cc < D; ++cc) s0 += Bt.Rbar[b * D2 + ii * D + cc] * dPU[k * D2 + cc * D + jj];
        out[(b * D2 + ij) * np + k] = ok ? s0 : NAN;
    }
}

// shared memory of k_sensitivity: q, the right-hand sides, then max(dv chunk, partial sums, K)
static size_t sensitivity_smem(int D, int n, size_t te) {
    const size_t d2 = (size_t)D * D, na = d2 * SENS_MAXP;
    const size_t region = std::max(std::max((size_t)SENS_CH * SENS_MAXP * d2, (size_t)(SENS_THREADS / 32) * na),
                                   (size_t)n * (n + 1));
    return ((size_t)n + (size_t)SENS_MAXP * (n + 1) + region) * te + 16;
}

int launch_sensitivity(const Model &M, Batch Bt, int precision, double *out, cudaStream_t s) {
    if (M.n_par > SENS_MAXP) return -1;
    const size_t te = precision == 0 ? 8 : 4;
    const size_t sm = sensitivity_smem(M.d, M.n, te);
    if (sm > 200 * 1024) return -1;
#define PODECM_SENS(DD, TT)                                                                                  \
    do {                                                                                                   \
        cudaFuncSetAttribute(k_sensitivity<DD, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        k_sensitivity<DD, TT><<<(int)Bt.B, SENS_THREADS, sm, s>>>(M, Bt, out);                             \
    } while (0)
    if (M.d == 2) {
        if (precision == 0) PODECM_SENS(2, double); else PODECM_SENS(2, float);
    } else {
        if (precision == 0) PODECM_SENS(3, double); else PODECM_SENS(3, float);
    }
#undef PODECM_SENS
    return 0;
}

template <int D>
static int launch_finalize_t(const Model &M, Batch Bt, const StepOpts &o, double *Pbar, double *Abar, void *info,
                             cudaStream_t s) {
    constexpr int D2 = D * D, D4 = D2 * D2;
    const size_t n = M.n;
    if (n * D2 > 1024) return -1;
    const size_t te = o.precision == 0 ? 8 : 4;    // arithmetic of the a11 sums and the Schur solve
    // cubature points per chunk: small chunks keep the shared memory per CTA low (several CTAs per
    // SM hide the latency of this short, barrier-bound kernel)
    auto bytes = [&](int chf) {
        // FP64 path: Bm, A0, Fm [chf][D2], then Ah, Gs; FP32 path: Bm, A0, then (16-byte aligned)
        // As [2][D4][chf], Fm32 [2][chf][D2], Ah [chf][D4], or the group sums [NPG][n][D2]
        if (te == 8) {
            const size_t head = (n * D2 + D4 + (size_t)chf * D2) * 8;
            const size_t sums = ((size_t)chf * D4 + (size_t)chf * D2 * n) * 8;
            const size_t schur = ((n + 1) * n + (n + 1) * D2) * 8 + 16;
            return head + std::max(sums, schur);
        }
        const size_t head = (n * D2 + D4) * 8;
        const size_t npg = 256 / ((n + ABAR_JT - 1) / ABAR_JT);
        const size_t sums = ((size_t)2 * D4 * chf + (size_t)2 * chf * D2 + (size_t)chf * D4) * 4;
        const size_t red = std::max(npg * n * D2, (size_t)256) * 4;
        const size_t schur = ((n + 1) * n + (n + 1) * D2) * 4 + 16;
        return head + 16 + std::max(std::max(sums, red), schur);
    };
    int CHF = te == 8 ? 16 : 32;
    while (CHF > 4 && bytes(CHF) > (te == 8 ? 48 : 64) * 1024) CHF /= 2;
    const size_t sm = bytes(CHF);
    if (o.precision == 0) {
        cudaFuncSetAttribute(k_finalize<D, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_finalize<D, double><<<(int)Bt.B, 256, sm, s>>>(M, Bt, o, Pbar, Abar, info, CHF);
    } else {
        cudaFuncSetAttribute(k_finalize<D, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_finalize<D, float><<<(int)Bt.B, 256, sm, s>>>(M, Bt, o, Pbar, Abar, info, CHF);
    }
    return 0;
}

int launch_finalize(const Model &M, Batch Bt, const StepOpts &o, double *Pbar, double *Abar, void *info,
                    cudaStream_t s) {
    return M.d == 2 ? launch_finalize_t<2>(M, Bt, o, Pbar, Abar, info, s)
                    : launch_finalize_t<3>(M, Bt, o, Pbar, Abar, info, s);
}

}  // namespace podecm
