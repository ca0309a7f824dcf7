// Full-order training solves on the device (the training solves of the offline stage of
// Algorithm 1; Sec. 2.1): the mapped weak form (Eq. weakform-dep-mapped) and its linearisation
// (Eq. Dweakform-dep) on the structured parent grid, Newton (Eq. full_newton) with a
// backtracking line search on ||f||, and step splitting when Newton fails.  S training samples
// (each its own geometry and load path) are solved together.
//   * k_fe_eval: one thread per (sample, element); per Gauss point the deformation gradient
//     F = Fbar + (sum_a w_a (x) dN_a) F_mu^-1, the FP64 return map and consistent tangent of the
//     hot path's material code, the element residual f_a,i = sum_g wJ (P F_mu^-T)_i . dN_a and
//     stiffness K_(a,i)(b,j) = sum_g wJ f_a . dP(e_j (x) f_b) with f_a = F_mu^-T dN_a; element
//     arrays scattered into the sample's residual vector and CSR values with FP64 atomics;
//   * the linear systems K dw = -f by conjugate gradients with a Jacobi preconditioner, batched
//     over the samples (per-sample scalars on the device);
//   * outputs per converged load step: the fluctuation w (the displacement snapshots), the
//     weighted stress W = J P F_mu^-T at every Gauss point (Eq. forcevector_rewritten; the
//     stress snapshots) and Pbar (Eq. eff_stress_full).
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace podecm {

constexpr int FE_MAXEN = 8;                  // nodes per element (Q4: 4, hex8: 8)

struct FeMesh {
    int d, ne, nen, ngp, ndof, nq, n_par;
    const int32_t *edof;     // [ne][nen*d] global dof or -1 (fixed / absent)
    const double *dN;        // [ngp][nen][d]
    const double *gw;        // [ngp]
    const int32_t *phase;    // [ne]
    const int32_t *emap;     // [ne][(nen d)^2] CSR position or -1
    const PhaseD *phases;    // material table
    int64_t nnz;
};

struct FeBatch {
    int S;
    const double *Finv, *J;  // [S][nq][d][d], [S][nq]
    const double *Fbar;      // [S][d*d] target of the current solve
    const double *w;         // [S][ndof] iterate
    const double *cp, *xi;   // [S][nq][6], [S][nq] committed history
    double *cp_tr, *xi_tr;   // trial history of the iterate
    double *f;               // [S][ndof] residual (zeroed by the caller)
    double *K;               // [S][nnz] CSR values (zeroed by the caller), may be null
    double *W;               // [S][nq][d*d] weighted stress J P F_mu^-T
    double *Pbar;            // [S][d*d] sum_g wJ P (zeroed by the caller)
    const uint8_t *active;   // [S] samples to evaluate
};

// geometry F_mu = I + sum_k coef_k Gmu_k at every Gauss point: Finv, J = |det F_mu|
__global__ void k_fe_geom(int d, int nq, int n_par, int S, const double *__restrict__ Gmu, const double *__restrict__ coef,
                          double *__restrict__ Finv, double *__restrict__ J) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)S * nq) return;
    const int s = (int)(t / nq), q = (int)(t - (int64_t)s * nq);
    double F[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int a = 0; a < d; ++a)
        for (int r = 0; r < d; ++r)
            for (int k = 0; k < n_par; ++k) F[a][r] += coef[s * n_par + k] * Gmu[((size_t)q * d * d + a * d + r) * n_par + k];
    const double c00 = F[1][1] * F[2][2] - F[1][2] * F[2][1], c01 = F[1][2] * F[2][0] - F[1][0] * F[2][2],
                 c02 = F[1][0] * F[2][1] - F[1][1] * F[2][0];
    const double det = F[0][0] * c00 + F[0][1] * c01 + F[0][2] * c02;
    const double id = 1.0 / det;
    double I[3][3];
    I[0][0] = c00 * id; I[1][0] = c01 * id; I[2][0] = c02 * id;
    I[0][1] = (F[0][2] * F[2][1] - F[0][1] * F[2][2]) * id;
    I[1][1] = (F[0][0] * F[2][2] - F[0][2] * F[2][0]) * id;
    I[2][1] = (F[0][1] * F[2][0] - F[0][0] * F[2][1]) * id;
    I[0][2] = (F[0][1] * F[1][2] - F[0][2] * F[1][1]) * id;
    I[1][2] = (F[0][2] * F[1][0] - F[0][0] * F[1][2]) * id;
    I[2][2] = (F[0][0] * F[1][1] - F[0][1] * F[1][0]) * id;
    for (int a = 0; a < d; ++a)
        for (int r = 0; r < d; ++r) Finv[(size_t)t * d * d + a * d + r] = I[a][r];
    J[t] = fabs(det);
}

template <int D>
__global__ void __launch_bounds__(128) k_fe_eval(FeMesh Mh, FeBatch Bb, int want_K) {
    constexpr int D2 = D * D;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)Bb.S * Mh.ne) return;
    const int s = (int)(t / Mh.ne), e = (int)(t - (int64_t)s * Mh.ne);
    if (!Bb.active[s]) return;
    const int nen = Mh.nen, nd = nen * D;
    const int32_t *ed = Mh.edof + (size_t)e * nd;
    const double *ws = Bb.w + (size_t)s * Mh.ndof;
    double ue[FE_MAXEN * 3];
    for (int k = 0; k < nd; ++k) ue[k] = ed[k] >= 0 ? ws[ed[k]] : 0.0;
    double fe[FE_MAXEN * 3];
    for (int k = 0; k < nd; ++k) fe[k] = 0.0;
    double *Ke = nullptr;
    double Kloc[(FE_MAXEN * 3) * (FE_MAXEN * 3)];
    if (want_K) {
        Ke = Kloc;
        for (int k = 0; k < nd * nd; ++k) Ke[k] = 0.0;
    }
    const PhaseD ph = Mh.phases[Mh.phase[e]];
    double Ub[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 1.0}};
    for (int a = 0; a < D; ++a)
        for (int r = 0; r < D; ++r) Ub[a][r] = Bb.Fbar[(size_t)s * D2 + a * D + r];
    double Psum[D2];
    for (int c = 0; c < D2; ++c) Psum[c] = 0.0;
    for (int g = 0; g < Mh.ngp; ++g) {
        const int q = e * Mh.ngp + g;
        const size_t sq = (size_t)s * Mh.nq + q;
        const double *dN = Mh.dN + (size_t)g * nen * D;
        double Fmi[D][D];
        for (int a = 0; a < D; ++a)
            for (int r = 0; r < D; ++r) Fmi[a][r] = Bb.Finv[sq * D2 + a * D + r];
        const double wJ = Mh.gw[g] * Bb.J[sq];
        // grad w (row = component) and F = Fbar + grad w F_mu^-1
        double Hg[D][D];
        for (int i = 0; i < D; ++i)
            for (int r = 0; r < D; ++r) {
                double sum = 0.0;
                for (int a = 0; a < nen; ++a) sum += ue[a * D + i] * dN[a * D + r];
                Hg[i][r] = sum;
            }
        double F[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 1.0}};
        for (int i = 0; i < D; ++i)
            for (int c = 0; c < D; ++c) {
                double sum = Ub[i][c];
                for (int r = 0; r < D; ++r) sum += Hg[i][r] * Fmi[r][c];
                F[i][c] = sum;
            }
        double cp[6];
        for (int k = 0; k < 6; ++k) cp[k] = Bb.cp[sq * 6 + k];
        MatState Sm;
        double P[3][3], Finv[3][3], cpn[6], xin;
        material_value<D, true>(F, cp, Bb.xi[sq], ph, Sm, P, Finv, cpn, &xin);
        for (int k = 0; k < 6; ++k) Bb.cp_tr[sq * 6 + k] = cpn[k];
        Bb.xi_tr[sq] = xin;
        // f_a = F_mu^-T dN_a: the pull-back of the shape-function gradients
        double fa[FE_MAXEN][D];
        for (int a = 0; a < nen; ++a)
            for (int c = 0; c < D; ++c) {
                double sum = 0.0;
                for (int r = 0; r < D; ++r) sum += dN[a * D + r] * Fmi[r][c];
                fa[a][c] = sum;
            }
        for (int i = 0; i < D; ++i)
            for (int c = 0; c < D; ++c) {
                double sum = 0.0;
                for (int r = 0; r < D; ++r) sum += P[i][r] * Fmi[c][r];
                Bb.W[sq * D2 + i * D + c] = Bb.J[sq] * sum;
                Psum[i * D + c] += wJ * P[i][c];
            }
        for (int a = 0; a < nen; ++a)
            for (int i = 0; i < D; ++i) {
                double sum = 0.0;
                for (int c = 0; c < D; ++c) sum += P[i][c] * fa[a][c];
                fe[a * D + i] += wJ * sum;
            }
        if (want_K) {
            // dP for the basis directions e_j (x) e_c, then K_(a,i)(b,j) += wJ f_a . dP(e_j (x) f_b)
            TangentData<double> td;
            tangent_setup<D, double>(Sm, ph, F, cp, Finv, P, td);
            double A4[D][D][D][D];   // [j][c][i][rho]
            for (int j = 0; j < D; ++j)
                for (int c = 0; c < D; ++c) {
                    double fdir[3] = {0.0, 0.0, 0.0};
                    fdir[c] = 1.0;
                    double dP[3][3];
                    tangent_direction<D, double>(td, j, fdir, dP);
                    for (int i = 0; i < D; ++i)
                        for (int r = 0; r < D; ++r) A4[j][c][i][r] = dP[i][r];
                }
            for (int b = 0; b < nen; ++b)
                for (int j = 0; j < D; ++j) {
                    double dPb[D][D];
                    for (int i = 0; i < D; ++i)
                        for (int r = 0; r < D; ++r) {
                            double sum = 0.0;
                            for (int c = 0; c < D; ++c) sum += fa[b][c] * A4[j][c][i][r];
                            dPb[i][r] = sum;
                        }
                    const int col = b * D + j;
                    for (int a = 0; a < nen; ++a)
                        for (int i = 0; i < D; ++i) {
                            double sum = 0.0;
                            for (int r = 0; r < D; ++r) sum += dPb[i][r] * fa[a][r];
                            Ke[(a * D + i) * nd + col] += wJ * sum;
                        }
                }
        }
    }
    double *fs = Bb.f + (size_t)s * Mh.ndof;
    for (int k = 0; k < nd; ++k)
        if (ed[k] >= 0) atomicAdd(&fs[ed[k]], fe[k]);
    for (int c = 0; c < D2; ++c) atomicAdd(&Bb.Pbar[(size_t)s * D2 + c], Psum[c]);
    if (want_K) {
        double *Ks = Bb.K + (size_t)s * Mh.nnz;
        const int32_t *em = Mh.emap + (size_t)e * nd * nd;
        for (int k = 0; k < nd * nd; ++k)
            if (em[k] >= 0) atomicAdd(&Ks[em[k]], Ke[k]);
    }
}

// ------------------------------------------------------------------ batched CG pieces
// y[s] = K[s] x[s] (one thread per row)
__global__ void k_fe_spmv(int S, int n, int64_t nnz, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                          const double *__restrict__ K, const double *__restrict__ x, double *__restrict__ y,
                          const uint8_t *__restrict__ run) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)S * n) return;
    const int s = (int)(t / n), r = (int)(t - (int64_t)s * n);
    if (!run[s]) return;
    const double *Ks = K + (size_t)s * nnz;
    const double *xs = x + (size_t)s * n;
    double sum = 0.0;
    for (int32_t k = rowptr[r]; k < rowptr[r + 1]; ++k) sum = fma(Ks[k], xs[col[k]], sum);
    y[t] = sum;
}

// out[s * nout + j] = sum_r a_j[s][r] b_j[s][r] for the nd dot products (one CTA per sample)
__global__ void k_fe_dots(int n, int nd, const double *a0, const double *b0, const double *a1, const double *b1,
                          double *out, const uint8_t *__restrict__ run) {
    __shared__ double red[32], o0, o1;
    const int s = blockIdx.x;
    if (!run[s]) return;
    double s0 = 0.0, s1 = 0.0;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
        const size_t i = (size_t)s * n + r;
        s0 = fma(a0[i], b0[i], s0);
        if (nd > 1) s1 = fma(a1[i], b1[i], s1);
    }
    // two block sums
    for (int k = 0; k < 2; ++k) {
        double v = k == 0 ? s0 : s1;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tsum = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tsum += red[w];
            if (k == 0) o0 = tsum; else o1 = tsum;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[(size_t)s * 2] = o0;
        if (nd > 1) out[(size_t)s * 2 + 1] = o1;
    }
}

// x += alpha p, r -= alpha Ap, z = r / diag  with alpha = rz / pAp per sample
__global__ void k_fe_cg_xr(int S, int n, double *x, double *r, double *z, const double *p, const double *Ap,
                           const double *diag, const double *rz, const double *pAp, const uint8_t *__restrict__ run) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)S * n) return;
    const int s = (int)(t / n);
    if (!run[s]) return;
    const double alpha = rz[(size_t)s * 2] / pAp[(size_t)s * 2];
    x[t] += alpha * p[t];
    r[t] -= alpha * Ap[t];
    z[t] = r[t] / diag[t];
}

// p = z + beta p with beta = rz_new / rz
__global__ void k_fe_cg_p(int S, int n, double *p, const double *z, const double *rz_new, const double *rz,
                          const uint8_t *__restrict__ run) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)S * n) return;
    const int s = (int)(t / n);
    if (!run[s]) return;
    const double beta = rz_new[(size_t)s * 2] / rz[(size_t)s * 2];
    p[t] = z[t] + beta * p[t];
}

// diag[s][r] = K[s][r][r]
__global__ void k_fe_diag(int S, int n, int64_t nnz, const int32_t *__restrict__ dpos, const double *__restrict__ K,
                          double *__restrict__ diag) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)S * n) return;
    const int s = (int)(t / n), r = (int)(t - (int64_t)s * n);
    diag[t] = K[(size_t)s * nnz + dpos[r]];
}

// zero the slices of the masked samples
__global__ void k_fe_zero(int S, int64_t n, double *x, const uint8_t *__restrict__ mask) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)S * n) return;
    if (mask[t / n]) x[t] = 0.0;
}

// dst = src on the masked samples
__global__ void k_fe_copy(int S, int64_t n, const double *src, double *dst, const uint8_t *__restrict__ mask) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)S * n) return;
    if (mask[t / n]) dst[t] = src[t];
}

// r = -f, z = r / diag, p = z, x = 0
__global__ void k_fe_cg_init(int S, int n, const double *f, const double *diag, double *r, double *z, double *p,
                             double *x, const uint8_t *__restrict__ run) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)S * n) return;
    if (!run[t / n]) return;
    r[t] = -f[t];
    z[t] = r[t] / diag[t];
    p[t] = z[t];
    x[t] = 0.0;
}

// wt = w + step[s] dw (samples in `run` only)
__global__ void k_fe_axpy(int S, int n, const double *w, const double *dw, const double *step, double *wt,
                          const uint8_t *__restrict__ run) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)S * n) return;
    const int s = (int)(t / n);
    if (!run[s]) return;
    wt[t] = w[t] + step[s] * dw[t];
}


}  // namespace podecm

// ------------------------------------------------------------------ host driver
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/podecm.h"

using namespace podecm;

namespace {
rom_status fe_fail(char *buf, size_t len, rom_status s, const char *fmt, ...) {
    if (buf && len) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, len, fmt, ap);
        va_end(ap);
    }
    return s;
}
unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

struct DevMem {
    std::vector<void *> ptrs;
    cudaError_t err = cudaSuccess;
    template <class T>
    T *get(size_t count) {
        void *p = nullptr;
        if (err == cudaSuccess) err = cudaMalloc(&p, count ? count * sizeof(T) : 16);
        if (err != cudaSuccess) return nullptr;
        ptrs.push_back(p);
        return static_cast<T *>(p);
    }
    ~DevMem() {
        for (void *p : ptrs) cudaFree(p);
    }
};
}  // namespace

extern "C" rom_status rom_fe_train(const rom_fe_mesh *mesh, int n_phase, const rom_phase *phases, int S, int n_par,
                                   const double *Gmu, const double *coef, int steps, const double *Fbar,
                                   double tol_rel, double tol_abs, int max_iter, int max_split, double *w_out,
                                   double *W_out, double *Pbar_out, int32_t *iters_out, int32_t *substeps_out,
                                   char *errbuf, size_t errlen) {
    if (!mesh || !phases || n_phase < 1 || n_phase > MAX_PHASES || S < 1 || n_par < 1 || !Gmu || !coef || steps < 1 ||
        !Fbar || !w_out || !Pbar_out || max_iter < 1 || max_split < 0)
        return fe_fail(errbuf, errlen, ROM_E_ARG, "rom_fe_train: bad arguments");
    const int d = mesh->d, ne = mesh->ne, nen = mesh->nen, ngp = mesh->ngp, ndof = mesh->ndof;
    if ((d != 2 && d != 3) || ne < 1 || nen < 1 || nen > FE_MAXEN || ngp < 1 || ndof < 1 || !mesh->edof || !mesh->dN ||
        !mesh->gw || !mesh->el_phase)
        return fe_fail(errbuf, errlen, ROM_E_ARG, "rom_fe_train: bad mesh");
    const int nd = nen * d, d2 = d * d, nq = ne * ngp;
    for (int e = 0; e < ne; ++e) {
        if (mesh->el_phase[e] < 0 || mesh->el_phase[e] >= n_phase)
            return fe_fail(errbuf, errlen, ROM_E_ARG, "rom_fe_train: element %d phase out of range", e);
        for (int k = 0; k < nd; ++k)
            if (mesh->edof[(size_t)e * nd + k] >= ndof)
                return fe_fail(errbuf, errlen, ROM_E_ARG, "rom_fe_train: element %d dof out of range", e);
    }
    // material table (the same derived moduli as rom_load_cubature)
    std::vector<PhaseD> ph(n_phase);
    for (int k = 0; k < n_phase; ++k) {
        const rom_phase &q = phases[k];
        if (!(q.E > 0) || !(q.nu > -1 && q.nu < 0.5) || !(q.s0 > 0) || (q.hard_law != 0 && q.hard_law != 1))
            return fe_fail(errbuf, errlen, ROM_E_ARG, "rom_fe_train: bad phase %d", k);
        ph[k].E = q.E; ph[k].nu = q.nu; ph[k].s0 = q.s0; ph[k].k = q.H_or_k; ph[k].p = q.p;
        ph[k].law = q.hard_law;
        ph[k].elastic = std::isinf(q.s0) ? 1 : 0;
        ph[k].G = q.E / (2.0 * (1.0 + q.nu));
        ph[k].lam = q.E * q.nu / ((1.0 + q.nu) * (1.0 - 2.0 * q.nu));
        ph[k].Kb = ph[k].lam + 2.0 * ph[k].G / 3.0;
    }
    // CSR pattern of the assembled stiffness and the element-to-CSR map
    std::vector<std::vector<int32_t>> rows(ndof);
    for (int e = 0; e < ne; ++e)
        for (int A = 0; A < nd; ++A) {
            const int32_t r = mesh->edof[(size_t)e * nd + A];
            if (r < 0) continue;
            for (int B = 0; B < nd; ++B) {
                const int32_t c = mesh->edof[(size_t)e * nd + B];
                if (c >= 0) rows[r].push_back(c);
            }
        }
    std::vector<int32_t> rowptr(ndof + 1, 0), col, dpos(ndof, -1);
    for (int r = 0; r < ndof; ++r) {
        std::sort(rows[r].begin(), rows[r].end());
        rows[r].erase(std::unique(rows[r].begin(), rows[r].end()), rows[r].end());
        rowptr[r + 1] = rowptr[r] + (int32_t)rows[r].size();
        for (size_t k = 0; k < rows[r].size(); ++k) {
            if (rows[r][k] == r) dpos[r] = rowptr[r] + (int32_t)k;
            col.push_back(rows[r][k]);
        }
        if (dpos[r] < 0) return fe_fail(errbuf, errlen, ROM_E_ARG, "rom_fe_train: dof %d belongs to no element", r);
    }
    const int64_t nnz = (int64_t)col.size();
    std::vector<int32_t> emap((size_t)ne * nd * nd, -1);
    for (int e = 0; e < ne; ++e)
        for (int A = 0; A < nd; ++A) {
            const int32_t r = mesh->edof[(size_t)e * nd + A];
            if (r < 0) continue;
            for (int B = 0; B < nd; ++B) {
                const int32_t c = mesh->edof[(size_t)e * nd + B];
                if (c < 0) continue;
                const auto it = std::lower_bound(col.begin() + rowptr[r], col.begin() + rowptr[r + 1], c);
                emap[((size_t)e * nd + A) * nd + B] = (int32_t)(it - col.begin());
            }
        }
    // device data
    DevMem dm;
    int32_t *d_edof = dm.get<int32_t>((size_t)ne * nd), *d_phase = dm.get<int32_t>(ne), *d_emap = dm.get<int32_t>(emap.size());
    int32_t *d_rowptr = dm.get<int32_t>(ndof + 1), *d_col = dm.get<int32_t>(nnz), *d_dpos = dm.get<int32_t>(ndof);
    double *d_dN = dm.get<double>((size_t)ngp * nen * d), *d_gw = dm.get<double>(ngp);
    PhaseD *d_ph = dm.get<PhaseD>(n_phase);
    double *d_Gmu = dm.get<double>((size_t)nq * d2 * n_par), *d_coef = dm.get<double>((size_t)S * n_par);
    double *d_Finv = dm.get<double>((size_t)S * nq * d2), *d_J = dm.get<double>((size_t)S * nq);
    double *d_Fb = dm.get<double>((size_t)S * d2);
    const size_t SN = (size_t)S * ndof;
    double *w_c = dm.get<double>(SN), *w_it = dm.get<double>(SN), *w_t = dm.get<double>(SN), *dw = dm.get<double>(SN);
    double *cp_c = dm.get<double>((size_t)S * nq * 6), *xi_c = dm.get<double>((size_t)S * nq);
    double *cp_tr = dm.get<double>((size_t)S * nq * 6), *xi_tr = dm.get<double>((size_t)S * nq);
    double *f = dm.get<double>(SN), *K = dm.get<double>((size_t)S * nnz), *W = dm.get<double>((size_t)S * nq * d2);
    double *Pb = dm.get<double>((size_t)S * d2);
    double *r = dm.get<double>(SN), *z = dm.get<double>(SN), *p = dm.get<double>(SN), *Ap = dm.get<double>(SN);
    double *diag = dm.get<double>(SN);
    double *s_rz = dm.get<double>((size_t)S * 2), *s_new = dm.get<double>((size_t)S * 2), *s_pap = dm.get<double>((size_t)S * 2);
    double *s_bb = dm.get<double>((size_t)S * 2), *d_step = dm.get<double>(S);
    uint8_t *d_act = dm.get<uint8_t>(S), *d_run = dm.get<uint8_t>(S);
    if (dm.err != cudaSuccess) return fe_fail(errbuf, errlen, ROM_E_NOMEM, "rom_fe_train: %s", cudaGetErrorString(dm.err));
    cudaStream_t st = nullptr;
    std::vector<double> cp0((size_t)S * nq * 6);
    for (size_t q = 0; q < (size_t)S * nq; ++q) {
        double *c = &cp0[q * 6];
        c[0] = 1; c[1] = 0; c[2] = 0; c[3] = 1; c[4] = 0; c[5] = 1;
    }
    cudaError_t e = cudaSuccess;
    auto H2D = [&](void *dst, const void *src, size_t bytes) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    };
    H2D(d_edof, mesh->edof, (size_t)ne * nd * 4);
    H2D(d_phase, mesh->el_phase, (size_t)ne * 4);
    H2D(d_emap, emap.data(), emap.size() * 4);
    H2D(d_rowptr, rowptr.data(), (ndof + 1) * 4);
    H2D(d_col, col.data(), (size_t)nnz * 4);
    H2D(d_dpos, dpos.data(), (size_t)ndof * 4);
    H2D(d_dN, mesh->dN, (size_t)ngp * nen * d * 8);
    H2D(d_gw, mesh->gw, (size_t)ngp * 8);
    H2D(d_ph, ph.data(), (size_t)n_phase * sizeof(PhaseD));
    H2D(d_Gmu, Gmu, (size_t)nq * d2 * n_par * 8);
    H2D(d_coef, coef, (size_t)S * n_par * 8);
    H2D(cp_c, cp0.data(), cp0.size() * 8);
    if (e == cudaSuccess) e = cudaMemsetAsync(xi_c, 0, (size_t)S * nq * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(w_c, 0, SN * 8, st);
    if (e != cudaSuccess) return fe_fail(errbuf, errlen, ROM_E_CUDA, "rom_fe_train: %s", cudaGetErrorString(e));
    k_fe_geom<<<nblk((int64_t)S * nq, 128), 128, 0, st>>>(d, nq, n_par, S, d_Gmu, d_coef, d_Finv, d_J);
    // ---- building blocks on sample masks
    FeMesh Mh{d, ne, nen, ngp, ndof, nq, n_par, d_edof, d_dN, d_gw, d_phase, d_emap, d_ph, nnz};
    std::vector<uint8_t> h_mask(S);
    std::vector<double> h_scal((size_t)S * 2), h_bb((size_t)S * 2);
    auto set_mask = [&](uint8_t *dmask, const std::vector<uint8_t> &m) { H2D(dmask, m.data(), (size_t)S); };
    auto launch_eval = [&](const double *wsrc, int want_K) {
        k_fe_zero<<<nblk((int64_t)S * ndof, 256), 256, 0, st>>>(S, ndof, f, d_act);
        if (want_K) k_fe_zero<<<nblk((int64_t)S * nnz, 256), 256, 0, st>>>(S, nnz, K, d_act);
        k_fe_zero<<<nblk((int64_t)S * d2, 256), 256, 0, st>>>(S, d2, Pb, d_act);
        FeBatch Bb{S, d_Finv, d_J, d_Fb, wsrc, cp_c, xi_c, cp_tr, xi_tr, f, K, W, Pb, d_act};
        if (d == 2) k_fe_eval<2><<<nblk((int64_t)S * ne, 128), 128, 0, st>>>(Mh, Bb, want_K);
        else k_fe_eval<3><<<nblk((int64_t)S * ne, 128), 128, 0, st>>>(Mh, Bb, want_K);
    };
    // ||f_s|| of the masked samples
    auto norms = [&](std::vector<double> &out) {
        k_fe_dots<<<S, 256, 0, st>>>(ndof, 1, f, f, f, f, s_pap, d_act);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_scal.data(), s_pap, (size_t)S * 16, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        for (int s = 0; s < S; ++s) out[s] = std::sqrt(h_scal[(size_t)s * 2]);
    };
    // K dw = -f for the masked samples: Jacobi-preconditioned conjugate gradients (relative 1e-12)
    auto cg = [&](const std::vector<uint8_t> &mask) {
        set_mask(d_act, mask);
        set_mask(d_run, mask);
        k_fe_diag<<<nblk((int64_t)S * ndof, 256), 256, 0, st>>>(S, ndof, nnz, d_dpos, K, diag);
        k_fe_cg_init<<<nblk((int64_t)S * ndof, 256), 256, 0, st>>>(S, ndof, f, diag, r, z, p, dw, d_run);
        k_fe_dots<<<S, 256, 0, st>>>(ndof, 2, r, z, r, r, s_rz, d_run);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_bb.data(), s_rz, (size_t)S * 16, cudaMemcpyDeviceToHost, st);
        std::vector<uint8_t> run = mask;
        double *rz = s_rz, *rn = s_new;
        const int maxit = std::max(200, 20 * ndof);
        for (int it = 0; it < maxit && e == cudaSuccess; ++it) {
            k_fe_spmv<<<nblk((int64_t)S * ndof, 128), 128, 0, st>>>(S, ndof, nnz, d_rowptr, d_col, K, p, Ap, d_run);
            k_fe_dots<<<S, 256, 0, st>>>(ndof, 1, p, Ap, p, p, s_pap, d_run);
            k_fe_cg_xr<<<nblk((int64_t)S * ndof, 256), 256, 0, st>>>(S, ndof, dw, r, z, p, Ap, diag, rz, s_pap, d_run);
            k_fe_dots<<<S, 256, 0, st>>>(ndof, 2, r, z, r, r, rn, d_run);
            k_fe_cg_p<<<nblk((int64_t)S * ndof, 256), 256, 0, st>>>(S, ndof, p, z, rn, rz, d_run);
            std::swap(rz, rn);
            if (it % 8 == 7) {
                e = cudaMemcpyAsync(h_scal.data(), rz, (size_t)S * 16, cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                bool any = false;
                for (int s = 0; s < S; ++s)
                    if (run[s]) {
                        if (!(h_scal[(size_t)s * 2 + 1] > 1e-24 * h_bb[(size_t)s * 2 + 1])) run[s] = 0;
                        any |= run[s] != 0;
                    }
                set_mask(d_run, run);
                if (!any) break;
            }
        }
    };
    auto masked_copy = [&](const double *src, double *dst, int64_t n, const std::vector<uint8_t> &mask) {
        set_mask(d_run, mask);
        k_fe_copy<<<nblk((int64_t)S * n, 256), 256, 0, st>>>(S, n, src, dst, d_run);
    };

    // ---- load steps: per sample a queue of sub-targets; Newton in lockstep over the samples
    std::vector<std::vector<std::vector<double>>> todo(S);
    std::vector<std::vector<int>> level(S);
    std::vector<std::vector<double>> Fprev(S, std::vector<double>(d2, 0.0));
    for (int s = 0; s < S; ++s)
        for (int a = 0; a < d; ++a) Fprev[s][a * d + a] = 1.0;
    std::vector<int> nsub(S), its(S);
    std::vector<double> Fcur((size_t)S * d2), rn0(S), rnv(S), rnt(S), stepv(S);
    for (int k = 0; k < steps && e == cudaSuccess; ++k) {
        for (int s = 0; s < S; ++s) {
            todo[s].assign(1, std::vector<double>(Fbar + ((size_t)s * steps + k) * d2, Fbar + ((size_t)s * steps + k + 1) * d2));
            level[s].assign(1, 0);
            nsub[s] = 0;
        }
        for (;;) {
            std::vector<uint8_t> A(S, 0);
            bool any = false;
            for (int s = 0; s < S; ++s)
                if (!todo[s].empty()) {
                    A[s] = 1;
                    any = true;
                    std::copy(todo[s].back().begin(), todo[s].back().end(), Fcur.begin() + (size_t)s * d2);
                }
            if (!any) break;
            H2D(d_Fb, Fcur.data(), Fcur.size() * 8);
            // Newton on the masked samples from the committed state
            masked_copy(w_c, w_it, ndof, A);
            set_mask(d_act, A);
            launch_eval(w_it, 1);
            norms(rnv);
            if (e != cudaSuccess) break;
            rn0 = rnv;
            std::vector<uint8_t> act = A, ok(S, 0);
            for (int it = 0; it <= max_iter; ++it) {
                bool left = false;
                for (int s = 0; s < S; ++s) {
                    if (!act[s]) continue;
                    if (!std::isfinite(rnv[s])) { act[s] = 0; continue; }
                    if (rnv[s] <= std::max(tol_rel * rn0[s], tol_abs)) { act[s] = 0; ok[s] = 1; its[s] = it; continue; }
                    if (it == max_iter) { act[s] = 0; continue; }
                    left = true;
                }
                if (!left) break;
                cg(act);
                // backtracking line search on ||f|| (halving, up to 10 times; the last trial is
                // taken if none improves)
                std::vector<uint8_t> ls = act;
                for (int s = 0; s < S; ++s) stepv[s] = 1.0;
                for (int t = 0; t < 11 && e == cudaSuccess; ++t) {
                    H2D(d_step, stepv.data(), (size_t)S * 8);
                    set_mask(d_run, ls);
                    k_fe_axpy<<<nblk((int64_t)S * ndof, 256), 256, 0, st>>>(S, ndof, w_it, dw, d_step, w_t, d_run);
                    set_mask(d_act, ls);
                    launch_eval(w_t, 1);
                    norms(rnt);
                    std::vector<uint8_t> take(S, 0);
                    bool pending = false;
                    for (int s = 0; s < S; ++s) {
                        if (!ls[s]) continue;
                        if ((std::isfinite(rnt[s]) && rnt[s] < rnv[s]) || t == 10) {
                            take[s] = 1;
                            rnv[s] = rnt[s];
                            ls[s] = 0;
                        } else {
                            stepv[s] *= 0.5;
                            pending = true;
                        }
                    }
                    masked_copy(w_t, w_it, ndof, take);
                    if (!pending) break;
                }
            }
            if (e != cudaSuccess) break;
            // commit the converged samples; split the increment of the failed ones
            masked_copy(w_it, w_c, ndof, ok);
            masked_copy(cp_tr, cp_c, (int64_t)nq * 6, ok);
            masked_copy(xi_tr, xi_c, nq, ok);
            for (int s = 0; s < S; ++s) {
                if (!A[s]) continue;
                if (ok[s]) {
                    Fprev[s] = todo[s].back();
                    todo[s].pop_back();
                    level[s].pop_back();
                    ++nsub[s];
                    if (todo[s].empty()) {   // load step k of sample s done: its outputs
                        const size_t o = (size_t)s * steps + k;
                        if (e == cudaSuccess) e = cudaMemcpyAsync(w_out + o * ndof, w_c + (size_t)s * ndof, (size_t)ndof * 8, cudaMemcpyDeviceToHost, st);
                        if (e == cudaSuccess && W_out) e = cudaMemcpyAsync(W_out + o * nq * d2, W + (size_t)s * nq * d2, (size_t)nq * d2 * 8, cudaMemcpyDeviceToHost, st);
                        if (e == cudaSuccess) e = cudaMemcpyAsync(Pbar_out + o * d2, Pb + (size_t)s * d2, (size_t)d2 * 8, cudaMemcpyDeviceToHost, st);
                        if (iters_out) iters_out[o] = its[s];
                        if (substeps_out) substeps_out[o] = nsub[s];
                    }
                } else {
                    if (level[s].back() >= max_split) {
                        cudaStreamSynchronize(st);
                        return fe_fail(errbuf, errlen, ROM_E_NOT_CONVERGED,
                                       "rom_fe_train: Newton failed for sample %d at load step %d after %d splits", s, k,
                                       level[s].back());
                    }
                    std::vector<double> mid(d2);
                    for (int c = 0; c < d2; ++c) mid[c] = 0.5 * (Fprev[s][c] + todo[s].back()[c]);
                    const int lv = level[s].back() + 1;
                    todo[s].push_back(mid);
                    level[s].push_back(lv);
                }
            }
        }
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fe_fail(errbuf, errlen, ROM_E_CUDA, "rom_fe_train: %s", cudaGetErrorString(e));
    return ROM_OK;
}
