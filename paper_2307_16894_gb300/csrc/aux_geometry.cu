// Reduced auxiliary geometry problem (Sec. 3.4, Eq. reduced_aux_problem; the geometry step of the
// online stage of Algorithm 1) on the device, one thread per instance:
//   theta = mu / mu_ref - 1                     (shape parameters of the boundary data)
//   b_P   = S theta                             (the forcing at the DEIM rows)
//   b_hat = M_deim b_P                          (DEIM reconstruction projected on the RB modes)
//   A_hat d_hat = b_hat                         (LU with partial pivoting, n_rb <= AUX_MAX)
// The per-instance map coefficients c = [theta, d_hat] then give
//   F_mu(X_i) = I + sum_k theta_k grad L_k(X_i) + sum_j d_hat_j grad psi_j(X_i),
// which the step kernels evaluate as F_mu = I + sum_c c_c Gmu_c with Gmu = [grad L, grad psi].
// A second kernel checks det F_mu > 0 at every point of every instance (the mapped weak form
// needs |det F_mu| > 0) and records the first offending (instance, point).
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace podecm {

constexpr int AUX_MAX = 8;

struct AuxDev {
    int n_p, n_rb, n_deim;
    const double *mu_ref;   // [n_p]
    const double *Ahat;     // [n_rb][n_rb]
    const double *Mdeim;    // [n_rb][n_deim]
    const double *S;        // [n_deim][n_p]
};

__global__ void k_aux_solve(AuxDev a, int64_t B, const double *__restrict__ mu, double *__restrict__ coef,
                            int *__restrict__ bad) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int np = a.n_p, nr = a.n_rb, nd = a.n_deim, nc = np + nr;
    double th[AUX_MAX], bp[4 * AUX_MAX], x[AUX_MAX], A[AUX_MAX * AUX_MAX];
    for (int k = 0; k < np; ++k) th[k] = mu[b * np + k] / a.mu_ref[k] - 1.0;
    for (int p = 0; p < nd; ++p) {
        double s = 0.0;
        for (int k = 0; k < np; ++k) s += a.S[p * np + k] * th[k];
        bp[p] = s;
    }
    for (int j = 0; j < nr; ++j) {
        double s = 0.0;
        for (int p = 0; p < nd; ++p) s += a.Mdeim[j * nd + p] * bp[p];
        x[j] = s;
    }
    for (int e = 0; e < nr * nr; ++e) A[e] = a.Ahat[e];
    // Gaussian elimination with partial pivoting on the n_rb x n_rb reduced operator
    bool ok = true;
    for (int c = 0; c < nr; ++c) {
        int piv = c;
        for (int r = c + 1; r < nr; ++r)
            if (fabs(A[r * nr + c]) > fabs(A[piv * nr + c])) piv = r;
        if (!(fabs(A[piv * nr + c]) > 0.0)) { ok = false; break; }
        if (piv != c) {
            for (int k = 0; k < nr; ++k) { const double t = A[c * nr + k]; A[c * nr + k] = A[piv * nr + k]; A[piv * nr + k] = t; }
            const double t = x[c]; x[c] = x[piv]; x[piv] = t;
        }
        for (int r = c + 1; r < nr; ++r) {
            const double f = A[r * nr + c] / A[c * nr + c];
            for (int k = c; k < nr; ++k) A[r * nr + k] -= f * A[c * nr + k];
            x[r] -= f * x[c];
        }
    }
    if (ok)
        for (int c = nr - 1; c >= 0; --c) {
            double s = x[c];
            for (int k = c + 1; k < nr; ++k) s -= A[c * nr + k] * x[k];
            x[c] = s / A[c * nr + c];
        }
    for (int k = 0; k < np; ++k) coef[b * nc + k] = th[k];
    for (int j = 0; j < nr; ++j) coef[b * nc + np + j] = ok ? x[j] : NAN;
    if (!ok) atomicExch(bad, 1);
}

// det F_mu at point i of instance b; the first (lowest flat index) non-positive or non-finite
// determinant is kept in first_bad (initialised to B * m by the host)
__global__ void k_geom_check(int d, int m, int nc, int64_t B, const double *__restrict__ coef,
                             const double *__restrict__ Gmu_T, unsigned long long *__restrict__ first_bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * m) return;
    const int64_t b = t / m;
    const int i = (int)(t - b * m);
    double F[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    for (int a = 0; a < d; ++a)
        for (int r = 0; r < d; ++r) {
            double s = 0.0;
            for (int k = 0; k < nc; ++k) s += coef[b * nc + k] * Gmu_T[((size_t)(a * d + r) * nc + k) * m + i];
            F[a * 3 + r] += s;
        }
    const double det = F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
                       F[2] * (F[3] * F[7] - F[4] * F[6]);
    if (!(det > 0.0) || !isfinite(det)) atomicMin(first_bad, (unsigned long long)t);
}

int aux_max() { return AUX_MAX; }

void launch_aux_geometry(int n_p, int n_rb, int n_deim, const double *mu_ref, const double *Ahat,
                         const double *Mdeim, const double *S, int64_t B, const double *mu, double *coef, int *bad,
                         cudaStream_t s) {
    AuxDev a{n_p, n_rb, n_deim, mu_ref, Ahat, Mdeim, S};
    const int T = 128;
    k_aux_solve<<<(unsigned)((B + T - 1) / T), T, 0, s>>>(a, B, mu, coef, bad);
}

void launch_geom_check(int d, int m, int nc, int64_t B, const double *coef, const double *Gmu_T,
                       unsigned long long *first_bad, cudaStream_t s) {
    const int T = 256;
    const int64_t n = B * m;
    k_geom_check<<<(unsigned)((n + T - 1) / T), T, 0, s>>>(d, m, nc, B, coef, Gmu_T, first_bad);
}

}  // namespace podecm
