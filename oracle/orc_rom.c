/*
 * ORACLE — test infrastructure only (tests, smoke() and the CPU-baseline leg
 * of bench.py).  Plain FP64 CPU reference; shares no code with the CUDA path.
 *
 * 1. The online hyper-reduced solve (Sec. 3.2-3.3, the online stage of
 *    Algorithm 1), term by term as the equations state:
 *      f_j  = sum_q w_q [ (dphi_j/dX^p F_mu^-1) : P |det F_mu| ]          Eq. forcevector_ecm
 *      K_jk = sum_q w_q [ (dphi_j F_mu^-1) : A : (dphi_k F_mu^-1) |det F_mu| ]  Eq. stiffnessmatrix_ecm
 *      K da = -f,  a += da, until ||f|| <= tol                               Eq. red_newton, Sec. 2.1
 *      Pbar = |Omega^p|^-1 sum_q w_q P |det F_mu|                           Eq. eff_stress_1
 *      K q_kl = b_kl (one solve per component of Fbar)                      Eq. tangent_problem_red
 *      Abar_ijkl = |Omega^p|^-1 sum_q w_q [A : (E_kl + dq_kl/dX^p F_mu^-1)]_ij |det F_mu|
 *                                                                           Eqs. eff_stiffness_1, eff_stress_f11
 *    F = Fbar + (sum_n a_n dphi_n/dX^p) F_mu^-1 (Eq. forcevector_ecm).
 *    A linear solve is a plain LU with partial pivoting.
 *    Shape sensitivities (Eq. eff_sensitivities_full), optional: with
 *      dF_k = (sum_n dq_k,n dphi_n/dX^p) F_mu^-1 + H dF_mu^-1/dmu_k,  H = sum_n a_n dphi_n/dX^p,
 *      K dq_k = -df/dmu_k at fixed a (the reduced counterpart of the fluctuation
 *      sensitivity, same factor K* = K), the derivative of f_j taken term by term,
 *      dPbar_ij/dmu_k = |Omega^p|^-1 sum_q w_q [ A_ijmn dF_k,mn |det F_mu| + P_ij d|det F_mu|/dmu_k ],
 *    given dF_mu^-1/dmu_k and d|det F_mu|/dmu_k at every point (inputs).
 * 2. The macro rotation split Fbar = Rbar Ubar (Sec. 4): the reduced problem
 *    is solved on Ubar and Pbar = Rbar Pbar(Ubar); Abar follows by the
 *    chain rule through the polar decomposition.
 * 3. Element loops of the full-order FE model (Sec. 2.1, Eqs.
 *    weakform-dep-mapped and Dweakform-dep) for the training solves.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include "orc.h"

/* ---------------------------------------------------------------- LU ---- */
static int lu_factor(int n, double *a, int *piv) {
    for (int k = 0; k < n; ++k) {
        int p = k;
        double mx = fabs(a[k * n + k]);
        for (int i = k + 1; i < n; ++i) if (fabs(a[i * n + k]) > mx) { mx = fabs(a[i * n + k]); p = i; }
        piv[k] = p;
        if (mx == 0.0 || !isfinite(mx)) return -1;
        if (p != k) for (int j = 0; j < n; ++j) { double t = a[k * n + j]; a[k * n + j] = a[p * n + j]; a[p * n + j] = t; }
        for (int i = k + 1; i < n; ++i) {
            double l = a[i * n + k] / a[k * n + k];
            a[i * n + k] = l;
            for (int j = k + 1; j < n; ++j) a[i * n + j] -= l * a[k * n + j];
        }
    }
    return 0;
}
static void lu_solve(int n, const double *a, const int *piv, double *b) {
    for (int k = 0; k < n; ++k) { int p = piv[k]; if (p != k) { double t = b[k]; b[k] = b[p]; b[p] = t; } }
    for (int i = 0; i < n; ++i) for (int j = 0; j < i; ++j) b[i] -= a[i * n + j] * b[j];
    for (int i = n - 1; i >= 0; --i) { for (int j = i + 1; j < n; ++j) b[i] -= a[i * n + j] * b[j]; b[i] /= a[i * n + i]; }
}

/* embed a d x d deformation gradient into 3x3 (plane strain: F33 = 1) */
static void embed3(int d, const double *F, double *F3) {
    memset(F3, 0, 9 * sizeof(double));
    for (int i = 0; i < d; ++i) for (int j = 0; j < d; ++j) F3[3 * i + j] = F[d * i + j];
    if (d == 2) F3[8] = 1.0;
}

/* ------------------------------------------------- online reduced step ---- */
typedef struct {
    int d, n, m;
    const double *G, *w, *Finv, *J, *Fbar, *Fp, *xi; const int *phase; const orc_phase *phases;
    double *gF, *Pq, *P33, *Aq, *Fp_tr, *xi_tr; int *pl;
} rom_ws;

/* residual f(a) and stiffness K(a) of Eqs. forcevector_ecm / stiffnessmatrix_ecm at the
 * iterate q; the material update is a trial (history of the last converged step is
 * only read).  Returns ||f||_2 (NaN if any stress is non-finite). */
static double rom_eval(rom_ws *s, const double *q, double *r, double *K, double *T) {
    const int d = s->d, n = s->n, m = s->m, d2 = d * d, d4 = d2 * d2;
    const double *G = s->G, *Finv = s->Finv;
    memset(r, 0, sizeof(double) * n);
    memset(K, 0, sizeof(double) * n * n);
    int bad = 0;
    for (int i = 0; i < m; ++i) {
        double H[9] = {0}, F[9], F3[9];
        for (int a = 0; a < d; ++a)
            for (int rr = 0; rr < d; ++rr) {
                double sum = 0.0;
                for (int j = 0; j < n; ++j) sum += G[((size_t)i * d2 + a * d + rr) * n + j] * q[j];
                H[a * d + rr] = sum;
            }
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) {
                double sum = s->Fbar[a * d + b];
                for (int rr = 0; rr < d; ++rr) sum += H[a * d + rr] * Finv[(size_t)i * d2 + rr * d + b];
                F[a * d + b] = sum;
            }
        embed3(d, F, F3);
        const double *P = s->Pq + (size_t)i * d2;
        const double *A = s->Aq + (size_t)i * d4;
        s->pl[i] = orc_material(d, F3, s->Fp + (size_t)i * 9, s->xi[i], &s->phases[s->phase[i]],
                                s->Pq + (size_t)i * d2, s->Aq + (size_t)i * d4, s->P33 + i,
                                s->Fp_tr + (size_t)i * 9, s->xi_tr + i);
        for (int c = 0; c < d2; ++c) if (!isfinite(P[c])) bad = 1;
        const double wJ = s->w[i] * s->J[i];
        const double *g = s->gF + (size_t)i * n * d2;
        for (int j = 0; j < n; ++j) {
            double sum = 0.0;
            for (int c = 0; c < d2; ++c) sum += g[j * d2 + c] * P[c];
            r[j] += wJ * sum;
        }
        for (int k = 0; k < n; ++k)
            for (int ab = 0; ab < d2; ++ab) {
                double sum = 0.0;
                for (int ce = 0; ce < d2; ++ce) sum += A[ab * d2 + ce] * g[k * d2 + ce];
                T[k * d2 + ab] = sum;
            }
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k) {
                double sum = 0.0;
                for (int ab = 0; ab < d2; ++ab) sum += g[j * d2 + ab] * T[k * d2 + ab];
                K[j * n + k] += wJ * sum;
            }
    }
    double rn = 0.0;
    for (int j = 0; j < n; ++j) rn += r[j] * r[j];
    return bad ? NAN : sqrt(rn);
}

/*
 * Newton on f(a) = 0 (Eq. red_newton).  Globalisation (the paper is silent; it
 * notes that small load steps may be needed): with max_ls > 0 a step a + t da is
 * accepted at the first t in 1, 1/2, 1/4, ... (at most max_ls halvings) with
 * ||f(a + t da)|| < ||f(a)||; after max_ls halvings the last trial is taken.
 * max_ls = 0 is the plain Newton of the paper.  iters = accepted updates,
 * evals = residual evaluations after the first.
 */
int orc_rom_step(int d, int n, int m, const double *G, const double *w, const int *phase,
                 const orc_phase *phases, const double *Finv, const double *J, double omega,
                 const double *Fbar, double *q, double *Fp, double *xi,
                 double tol_rel, double tol_abs, int max_iter, int max_ls,
                 double *Pbar, double *Abar, double *P33bar,
                 int *iters_out, int *evals_out, int *n_yield_out, double *res0_out, double *res_out,
                 int npar, const double *dFinv, const double *dJ, double *dPdmu)
{
    const int d2 = d * d, d4 = d2 * d2;
    rom_ws s = { d, n, m, G, w, Finv, J, Fbar, Fp, xi, phase, phases, NULL, NULL, NULL, NULL, NULL, NULL, NULL };
    s.gF = malloc(sizeof(double) * (size_t)m * n * d2);   /* dphi_j/dX^p F_mu^-1 at each point */
    s.Pq = malloc(sizeof(double) * (size_t)m * d2);
    s.P33 = malloc(sizeof(double) * (size_t)m);
    s.Aq = malloc(sizeof(double) * (size_t)m * d4);
    s.Fp_tr = malloc(sizeof(double) * (size_t)m * 9);
    s.xi_tr = malloc(sizeof(double) * (size_t)m);
    s.pl = malloc(sizeof(int) * (size_t)m);
    double *r = malloc(sizeof(double) * n), *K = malloc(sizeof(double) * n * n), *dq = malloc(sizeof(double) * n);
    double *qt = malloc(sizeof(double) * n);
    double *T = malloc(sizeof(double) * n * d2);
    int *piv = malloc(sizeof(int) * n);
    int status = 5, it = 0, evals = 0;

    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j)
            for (int a = 0; a < d; ++a)
                for (int b = 0; b < d; ++b) {
                    double sum = 0.0;
                    for (int rr = 0; rr < d; ++rr) sum += G[((size_t)i * d2 + a * d + rr) * n + j] * Finv[(size_t)i * d2 + rr * d + b];
                    s.gF[((size_t)i * n + j) * d2 + a * d + b] = sum;
                }

    double rn = rom_eval(&s, q, r, K, T);
    const double r0 = rn;
    const double tol = tol_rel * r0 > tol_abs ? tol_rel * r0 : tol_abs;
    for (it = 0;; ++it) {
        if (!isfinite(rn)) { status = 6; break; }
        if (rn <= tol) { status = 0; break; }
        if (it >= max_iter) { status = 5; break; }
        if (lu_factor(n, K, piv) != 0) { status = 6; break; }
        for (int j = 0; j < n; ++j) dq[j] = -r[j];
        lu_solve(n, K, piv, dq);
        double t = 1.0, rt = 0.0;
        for (int ls = 0;; ++ls) {
            for (int j = 0; j < n; ++j) qt[j] = q[j] + t * dq[j];
            rt = rom_eval(&s, qt, r, K, T);
            ++evals;
            if (ls >= max_ls || (isfinite(rt) && rt < rn)) break;
            t *= 0.5;
        }
        memcpy(q, qt, sizeof(double) * n);
        rn = rt;
    }

    if (iters_out) *iters_out = it;
    if (evals_out) *evals_out = evals;
    if (res0_out) *res0_out = r0;
    if (res_out) *res_out = rn;
    int ny = 0;
    for (int i = 0; i < m; ++i) ny += s.pl[i];
    if (n_yield_out) *n_yield_out = ny;

    if (status == 0 && dPdmu && npar > 0) {
        /* shape sensitivities, Eq. eff_sensitivities_full (dFinv [m][npar][d2], dJ [m][npar]) */
        double *Kf = malloc(sizeof(double) * n * n), *rhs = malloc(sizeof(double) * n);
        memcpy(Kf, K, sizeof(double) * n * n);
        int *pv = malloc(sizeof(int) * n);
        const int fac = lu_factor(n, Kf, pv);
        for (int k = 0; k < npar; ++k) {
            /* rhs = -df/dmu_k at fixed a: the three terms of the derivative of
             * w (dphi_j/dX^p F_mu^-1) : P(F) |det F_mu| with F = Fbar + H F_mu^-1 */
            for (int j = 0; j < n; ++j) rhs[j] = 0.0;
            for (int i = 0; i < m; ++i) {
                const double *Fi = dFinv + ((size_t)i * npar + k) * d2;
                const double *P = s.Pq + (size_t)i * d2, *A = s.Aq + (size_t)i * d4;
                double H[9] = {0}, dF[9], AdF[9];
                for (int c = 0; c < d2; ++c)
                    for (int j = 0; j < n; ++j) H[c] += G[((size_t)i * d2 + c) * n + j] * q[j];
                for (int a = 0; a < d; ++a)
                    for (int b = 0; b < d; ++b) {
                        double t = 0.0;
                        for (int rr = 0; rr < d; ++rr) t += H[a * d + rr] * Fi[rr * d + b];
                        dF[a * d + b] = t;
                    }
                for (int ab = 0; ab < d2; ++ab) {
                    double t = 0.0;
                    for (int c = 0; c < d2; ++c) t += A[ab * d2 + c] * dF[c];
                    AdF[ab] = t;
                }
                const double dJk = dJ[(size_t)i * npar + k];
                for (int j = 0; j < n; ++j) {
                    const double *g = s.gF + ((size_t)i * n + j) * d2;
                    double t1 = 0.0, t2 = 0.0, t3 = 0.0;
                    for (int a = 0; a < d; ++a)
                        for (int b = 0; b < d; ++b) {
                            double gd = 0.0;   /* (dphi_j/dX^p dF_mu^-1/dmu_k)_ab */
                            for (int rr = 0; rr < d; ++rr) gd += G[((size_t)i * d2 + a * d + rr) * n + j] * Fi[rr * d + b];
                            t1 += gd * P[a * d + b];
                        }
                    for (int c = 0; c < d2; ++c) { t2 += g[c] * AdF[c]; t3 += g[c] * P[c]; }
                    rhs[j] -= w[i] * (J[i] * (t1 + t2) + dJk * t3);
                }
            }
            if (fac == 0) lu_solve(n, Kf, pv, rhs);
            for (int ij = 0; ij < d2; ++ij) {
                double sum = 0.0;
                for (int i = 0; i < m; ++i) {
                    const double *Fi = dFinv + ((size_t)i * npar + k) * d2;
                    const double *A = s.Aq + (size_t)i * d4;
                    double H[9] = {0}, Hq[9] = {0}, dF[9];
                    for (int c = 0; c < d2; ++c)
                        for (int j = 0; j < n; ++j) {
                            const double gg = G[((size_t)i * d2 + c) * n + j];
                            H[c] += gg * q[j];
                            Hq[c] += gg * rhs[j];
                        }
                    for (int a = 0; a < d; ++a)
                        for (int b = 0; b < d; ++b) {
                            double t = 0.0;
                            for (int rr = 0; rr < d; ++rr)
                                t += Hq[a * d + rr] * Finv[(size_t)i * d2 + rr * d + b] + H[a * d + rr] * Fi[rr * d + b];
                            dF[a * d + b] = t;
                        }
                    double t = 0.0;
                    for (int c = 0; c < d2; ++c) t += A[ij * d2 + c] * dF[c];
                    sum += w[i] * (J[i] * t + s.Pq[(size_t)i * d2 + ij] * dJ[(size_t)i * npar + k]);
                }
                dPdmu[ij * npar + k] = fac == 0 ? sum / omega : NAN;
            }
        }
        free(Kf); free(rhs); free(pv);
    }
    if (status == 0) {
        /* effective stress, Eq. eff_stress_1 */
        for (int c = 0; c < d2; ++c) {
            double sum = 0.0;
            for (int i = 0; i < m; ++i) sum += w[i] * J[i] * s.Pq[(size_t)i * d2 + c];
            Pbar[c] = sum / omega;
        }
        if (P33bar) {
            double sum = 0.0;
            for (int i = 0; i < m; ++i) sum += w[i] * J[i] * s.P33[i];
            *P33bar = sum / omega;
        }
        /* effective stiffness: d^2 reduced tangent problems on the factor of K at
         * the solution (K* = K, Sec. 3.3), then Eqs. eff_stiffness_1 / eff_stress_f11 */
        if (Abar) {
            int fac = lu_factor(n, K, piv);
            double *qkl = malloc(sizeof(double) * n);
            for (int kl = 0; kl < d2; ++kl) {
                for (int j = 0; j < n; ++j) {
                    double sum = 0.0;
                    for (int i = 0; i < m; ++i) {
                        const double *g = s.gF + ((size_t)i * n + j) * d2;
                        const double *A = s.Aq + (size_t)i * d4;
                        double tt = 0.0;
                        for (int ab = 0; ab < d2; ++ab) tt += g[ab] * A[ab * d2 + kl];
                        sum += w[i] * J[i] * tt;
                    }
                    qkl[j] = -sum;
                }
                if (fac == 0) lu_solve(n, K, piv, qkl);
                for (int ij = 0; ij < d2; ++ij) {
                    double sum = 0.0;
                    for (int i = 0; i < m; ++i) {
                        double dFv[9];
                        /* E_kl + (sum_n q_n dphi_n/dX^p) F_mu^-1 */
                        for (int c = 0; c < d2; ++c) {
                            double tt = (c == kl) ? 1.0 : 0.0;
                            for (int j = 0; j < n; ++j) tt += s.gF[((size_t)i * n + j) * d2 + c] * qkl[j];
                            dFv[c] = tt;
                        }
                        const double *A = s.Aq + (size_t)i * d4;
                        double tt = 0.0;
                        for (int c = 0; c < d2; ++c) tt += A[ij * d2 + c] * dFv[c];
                        sum += w[i] * J[i] * tt;
                    }
                    Abar[ij * d2 + kl] = sum / omega;
                }
            }
            free(qkl);
            if (fac != 0) status = 6;
        }
        /* commit the history of the converged step */
        memcpy(Fp, s.Fp_tr, sizeof(double) * (size_t)m * 9);
        memcpy(xi, s.xi_tr, sizeof(double) * (size_t)m);
    }
    free(s.gF); free(s.Pq); free(s.P33); free(s.Aq); free(s.Fp_tr); free(s.xi_tr); free(s.pl);
    free(r); free(K); free(dq); free(qt); free(T); free(piv);
    return status;
}

/* ------------------------------------------------ polar decomposition ---- */
static void mat3_mul(const double *a, const double *b, double *c) {
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) { double s = 0; for (int k = 0; k < 3; ++k) s += a[3 * i + k] * b[3 * k + j]; c[3 * i + j] = s; }
}
static void mat3_inv(const double *a, double *r) {
    double c[9];
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) {
        int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        c[3 * j + i] = a[3 * i1 + j1] * a[3 * i2 + j2] - a[3 * i1 + j2] * a[3 * i2 + j1];
    }
    double det = a[0] * c[0] + a[1] * c[3] + a[2] * c[6];
    for (int k = 0; k < 9; ++k) r[k] = c[k] / det;
}

/* F = R U with U symmetric positive definite.  2D: closed form.  3D: U = sqrt(F^T F)
 * by the Denman-Beavers iteration, R = F U^-1. */
void orc_polar(int d, const double *F, double *R, double *U) {
    if (d == 2) {
        double th = atan2(F[2] - F[1], F[0] + F[3]);
        double c = cos(th), s = sin(th);
        R[0] = c; R[1] = -s; R[2] = s; R[3] = c;
        /* U = R^T F */
        U[0] = c * F[0] + s * F[2]; U[1] = c * F[1] + s * F[3];
        U[2] = -s * F[0] + c * F[2]; U[3] = -s * F[1] + c * F[3];
        double u = 0.5 * (U[1] + U[2]); U[1] = U[2] = u;
        return;
    }
    double C[9], Ft[9], Y[9], Z[9], Yi[9], Zi[9], Ui[9];
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) Ft[3 * i + j] = F[3 * j + i];
    mat3_mul(Ft, F, C);
    memcpy(Y, C, sizeof Y);
    memset(Z, 0, sizeof Z); Z[0] = Z[4] = Z[8] = 1.0;
    for (int it = 0; it < 100; ++it) {
        mat3_inv(Y, Yi); mat3_inv(Z, Zi);
        double ch = 0, nr = 0;
        for (int k = 0; k < 9; ++k) {
            double yn = 0.5 * (Y[k] + Zi[k]), zn = 0.5 * (Z[k] + Yi[k]);
            ch += (yn - Y[k]) * (yn - Y[k]); nr += yn * yn;
            Y[k] = yn; Z[k] = zn;
        }
        if (ch <= 1e-34 * nr && it > 3) break;
    }
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) U[3 * i + j] = 0.5 * (Y[3 * i + j] + Y[3 * j + i]);
    mat3_inv(U, Ui);
    mat3_mul(F, Ui, R);
}

/* Reduced step on the stretch Ubar of Fbar = Rbar Ubar; Pbar = Rbar Pbar_U and
 * Abar = d(Rbar Pbar_U(Rbar^T Fbar))/dFbar, using dRbar = Rbar W with the axial
 * vector of W solving (tr U I - U) w = axial(M - M^T), M = Rbar^T dFbar.      */
int orc_rom_step_polar(int d, int n, int m, const double *G, const double *w, const int *phase,
                       const orc_phase *phases, const double *Finv, const double *J, double omega,
                       const double *Fbar, double *q, double *Fp, double *xi,
                       double tol_rel, double tol_abs, int max_iter, int max_ls,
                       double *Pbar, double *Abar, double *P33bar,
                       int *iters, int *evals, int *n_yield, double *res0, double *res,
                       int npar, const double *dFinv, const double *dJ, double *dPdmu)
{
    const int d2 = d * d;
    double R[9], U[9], PU[9], AU[81], dPU[27];
    orc_polar(d, Fbar, R, U);
    int st = orc_rom_step(d, n, m, G, w, phase, phases, Finv, J, omega, U, q, Fp, xi,
                          tol_rel, tol_abs, max_iter, max_ls, PU, AU, P33bar, iters, evals, n_yield, res0, res,
                          npar, dFinv, dJ, dPdmu ? dPU : NULL);
    if (st != 0) return st;
    for (int i = 0; i < d; ++i) for (int j = 0; j < d; ++j) {
        double s = 0; for (int k = 0; k < d; ++k) s += R[i * d + k] * PU[k * d + j];
        Pbar[i * d + j] = s;
    }
    /* the rotation does not depend on the geometry: dPbar/dmu = Rbar dPbar_U/dmu */
    if (dPdmu)
        for (int kp = 0; kp < npar; ++kp)
            for (int i = 0; i < d; ++i) for (int j = 0; j < d; ++j) {
                double s = 0; for (int k = 0; k < d; ++k) s += R[i * d + k] * dPU[(k * d + j) * npar + kp];
                dPdmu[(i * d + j) * npar + kp] = s;
            }
    if (!Abar) return st;
    double trU = 0; for (int i = 0; i < d; ++i) trU += U[i * d + i];
    for (int k = 0; k < d; ++k)
        for (int l = 0; l < d; ++l) {
            double M[9] = {0}, W[9] = {0}, dU[9], t[9], dPU[9];
            for (int i = 0; i < d; ++i) M[i * d + l] = R[k * d + i];     /* M = R^T E_kl */
            if (d == 2) {
                double om = (M[2] - M[1]) / trU;
                W[0] = 0; W[1] = -om; W[2] = om; W[3] = 0;
            } else {
                double a[3] = { M[7] - M[5], M[2] - M[6], M[3] - M[1] };
                double S[9], Si[9], om[3];
                for (int i = 0; i < 9; ++i) S[i] = -U[i];
                S[0] += trU; S[4] += trU; S[8] += trU;
                mat3_inv(S, Si);
                for (int i = 0; i < 3; ++i) om[i] = Si[3 * i] * a[0] + Si[3 * i + 1] * a[1] + Si[3 * i + 2] * a[2];
                W[1] = -om[2]; W[2] = om[1]; W[3] = om[2]; W[5] = -om[0]; W[6] = -om[1]; W[7] = om[0];
            }
            for (int i = 0; i < d; ++i) for (int j = 0; j < d; ++j) {
                double s = 0; for (int c = 0; c < d; ++c) s += W[i * d + c] * U[c * d + j];
                dU[i * d + j] = M[i * d + j] - s;
            }
            for (int ij = 0; ij < d2; ++ij) {
                double s = 0; for (int c = 0; c < d2; ++c) s += AU[ij * d2 + c] * dU[c];
                dPU[ij] = s;
            }
            for (int i = 0; i < d; ++i) for (int j = 0; j < d; ++j) {
                double s = dPU[i * d + j];
                for (int c = 0; c < d; ++c) s += W[i * d + c] * PU[c * d + j];
                t[i * d + j] = s;
            }
            for (int i = 0; i < d; ++i) for (int j = 0; j < d; ++j) {
                double s = 0; for (int c = 0; c < d; ++c) s += R[i * d + c] * t[c * d + j];
                Abar[(i * d + j) * d2 + k * d + l] = s;
            }
        }
    return st;
}

/* ------------------------------------------------ threaded batch ----- */
typedef struct {
    int d, n, m, polar;
    const double *G, *w; const int *phase; const orc_phase *phases;
    const double *Finv, *J; double omega;
    const double *Fbar; double *q, *Fp, *xi;
    double tol_rel, tol_abs; int max_iter, max_ls;
    double *Pbar, *Abar, *P33bar; int *iters, *evals, *n_yield, *status; double *res0, *res;
    int npar; const double *dFinv, *dJ; double *dPdmu;
    int B, nthreads, tid;
} rom_batch_args;

static void *rom_batch_worker(void *p) {
    rom_batch_args *a = p;
    const int d2 = a->d * a->d;
    for (int b = a->tid; b < a->B; b += a->nthreads) {
        const double *Finv = a->Finv + (size_t)b * a->m * d2;
        const double *J = a->J + (size_t)b * a->m;
        int (*fn)(int, int, int, const double *, const double *, const int *, const orc_phase *,
                  const double *, const double *, double, const double *, double *, double *, double *,
                  double, double, int, int, double *, double *, double *, int *, int *, int *, double *, double *,
                  int, const double *, const double *, double *)
            = a->polar ? orc_rom_step_polar : orc_rom_step;
        const int np = a->dPdmu ? a->npar : 0;
        a->status[b] = fn(a->d, a->n, a->m, a->G, a->w, a->phase, a->phases, Finv, J, a->omega,
                          a->Fbar + (size_t)b * d2, a->q + (size_t)b * a->n, a->Fp + (size_t)b * a->m * 9,
                          a->xi + (size_t)b * a->m, a->tol_rel, a->tol_abs, a->max_iter, a->max_ls,
                          a->Pbar + (size_t)b * d2, a->Abar ? a->Abar + (size_t)b * d2 * d2 : NULL,
                          a->P33bar ? a->P33bar + b : NULL,
                          a->iters + b, a->evals + b, a->n_yield + b, a->res0 + b, a->res + b,
                          np, np ? a->dFinv + (size_t)b * a->m * np * d2 : NULL, np ? a->dJ + (size_t)b * a->m * np : NULL,
                          np ? a->dPdmu + (size_t)b * d2 * np : NULL);
    }
    return NULL;
}

/* B independent instances, spread over nthreads POSIX threads */
void orc_rom_batch(int B, int nthreads, int polar, int d, int n, int m, const double *G, const double *w,
                   const int *phase, const orc_phase *phases, const double *Finv, const double *J, double omega,
                   const double *Fbar, double *q, double *Fp, double *xi,
                   double tol_rel, double tol_abs, int max_iter, int max_ls,
                   double *Pbar, double *Abar, double *P33bar, int *iters, int *evals, int *n_yield, int *status,
                   double *res0, double *res, int npar, const double *dFinv, const double *dJ, double *dPdmu)
{
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
    rom_batch_args *args = malloc(sizeof(rom_batch_args) * nthreads);
    for (int t = 0; t < nthreads; ++t) {
        rom_batch_args a = { d, n, m, polar, G, w, phase, phases, Finv, J, omega, Fbar, q, Fp, xi,
                             tol_rel, tol_abs, max_iter, max_ls, Pbar, Abar, P33bar, iters, evals, n_yield, status, res0, res,
                             npar, dFinv, dJ, dPdmu, B, nthreads, t };
        args[t] = a;
        pthread_create(&th[t], NULL, rom_batch_worker, &args[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th); free(args);
}

/* ------------------------------------------------ full-order FE ------ */
typedef struct {
    int d, ne, nen, ngp, ndof;
    const int *conn, *dofmap, *el_phase; const orc_phase *phases;
    const double *dN, *gw, *Finv, *J, *Fbar, *wdofs, *Fp, *xi;
    double *fe, *Ke, *Fp_tr, *xi_tr, *Pq, *Aq, *P33q; int *plq;
    int want_K, nthreads, tid;
} fe_args;

static void *fe_worker(void *p) {
    fe_args *a = p;
    const int d = a->d, d2 = d * d, d4 = d2 * d2, nen = a->nen, ngp = a->ngp, ned = nen * d;
    double *gN = malloc(sizeof(double) * nen * d);
    for (int e = a->tid; e < a->ne; e += a->nthreads) {
        double *fe = a->fe + (size_t)e * ned;
        double *Ke = a->want_K ? a->Ke + (size_t)e * ned * ned : NULL;
        memset(fe, 0, sizeof(double) * ned);
        if (Ke) memset(Ke, 0, sizeof(double) * ned * ned);
        const orc_phase *ph = &a->phases[a->el_phase[e]];
        for (int g = 0; g < ngp; ++g) {
            size_t qp = (size_t)e * ngp + g;
            const double *Fi = a->Finv + qp * d2;
            double H[9] = {0}, F[9], F3[9];
            for (int node = 0; node < nen; ++node) {
                int nid = a->conn[e * nen + node];
                for (int c = 0; c < d; ++c) {
                    int dof = a->dofmap[nid * d + c];
                    double u = dof >= 0 ? a->wdofs[dof] : 0.0;
                    for (int rr = 0; rr < d; ++rr) H[c * d + rr] += u * a->dN[(g * nen + node) * d + rr];
                }
                for (int b = 0; b < d; ++b) {
                    double s = 0;
                    for (int rr = 0; rr < d; ++rr) s += a->dN[(g * nen + node) * d + rr] * Fi[rr * d + b];
                    gN[node * d + b] = s;
                }
            }
            for (int i = 0; i < d; ++i) for (int j = 0; j < d; ++j) {
                double s = a->Fbar[i * d + j];
                for (int rr = 0; rr < d; ++rr) s += H[i * d + rr] * Fi[rr * d + j];
                F[i * d + j] = s;
            }
            embed3(d, F, F3);
            double *P = a->Pq + qp * d2, *A = a->Aq + qp * d4;
            a->plq[qp] = orc_material(d, F3, a->Fp + qp * 9, a->xi[qp], ph, P, Ke ? A : NULL, a->P33q + qp,
                                      a->Fp_tr + qp * 9, a->xi_tr + qp);
            const double wJ = a->gw[g] * a->J[qp];
            for (int node = 0; node < nen; ++node)
                for (int i = 0; i < d; ++i) {
                    double s = 0;
                    for (int b = 0; b < d; ++b) s += P[i * d + b] * gN[node * d + b];
                    fe[node * d + i] += wJ * s;
                }
            if (Ke)
                for (int n1 = 0; n1 < nen; ++n1)
                    for (int i = 0; i < d; ++i)
                        for (int n2 = 0; n2 < nen; ++n2)
                            for (int k = 0; k < d; ++k) {
                                double s = 0;
                                for (int b = 0; b < d; ++b)
                                    for (int l = 0; l < d; ++l)
                                        s += gN[n1 * d + b] * A[(i * d + b) * d2 + k * d + l] * gN[n2 * d + l];
                                Ke[(n1 * d + i) * ned + n2 * d + k] += wJ * s;
                            }
        }
    }
    free(gN);
    return NULL;
}

/* Element force vectors fe[ne][nen*d] and stiffness Ke[ne][nen*d][nen*d] of the
 * mapped weak form, plus per-point P, A and trial history.  The caller
 * scatters fe / Ke to global dofs. */
void orc_fe_elements(int d, int ne, int nen, int ngp, const int *conn, const int *dofmap, const int *el_phase,
                     const orc_phase *phases, const double *dN, const double *gw, const double *Finv,
                     const double *J, const double *Fbar, const double *wdofs, const double *Fp, const double *xi,
                     double *fe, double *Ke, double *Fp_tr, double *xi_tr, double *Pq, double *Aq, double *P33q,
                     int *plq, int want_K, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = malloc(sizeof(pthread_t) * nthreads);
    fe_args *args = malloc(sizeof(fe_args) * nthreads);
    for (int t = 0; t < nthreads; ++t) {
        fe_args a = { d, ne, nen, ngp, 0, conn, dofmap, el_phase, phases, dN, gw, Finv, J, Fbar, wdofs, Fp, xi,
                      fe, Ke, Fp_tr, xi_tr, Pq, Aq, P33q, plq, want_K, nthreads, t };
        args[t] = a;
        pthread_create(&th[t], NULL, fe_worker, &args[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th); free(args);
}

/* material at many independent points (for the tests): F3[npt][9] */
void orc_material_batch(int d, int npt, const double *F3, const double *Fp_n, const double *xi_n,
                        const int *phase, const orc_phase *phases, double *P, double *A, double *P33,
                        double *Fp_new, double *xi_new, int *plastic)
{
    const int d2 = d * d;
    for (int i = 0; i < npt; ++i)
        plastic[i] = orc_material(d, F3 + (size_t)i * 9, Fp_n + (size_t)i * 9, xi_n[i], &phases[phase[i]],
                                  P + (size_t)i * d2, A ? A + (size_t)i * d2 * d2 : NULL, P33 ? P33 + i : NULL,
                                  Fp_new + (size_t)i * 9, xi_new + i);
}
