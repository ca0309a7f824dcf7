// Finite-strain J2 material point on the device (Appendix A of arXiv 2307.16894),
// written in the spatial (left Cauchy-Green) form of the same model:
//
//   b_tr = F C^p_n^-1 F^T                       trial elastic left Cauchy-Green tensor
//   b_tr = sum_a lambda_a n_a n_a^T             (FP64 Jacobi eigen-decomposition)
//   eps_a = 1/2 ln lambda_a                      elastic log strain (Eq. j2_7, Hencky)
//   tau_tr,a = lam tr(eps) + 2G eps_a            (Eq. j2_1 in principal Kirchhoff stresses)
//   f = sqrt(3/2) |dev tau_tr| - sigma_y(xi_n)   (Eq. j2_2)
//   radial return in log space, dgamma from g(dg) = q_tr - 3G dg - sigma_y(xi_n + dg) = 0
//   tau_a = tau_tr,a - 2G dg sqrt(3/2) nhat_a    (Eqs. j2_3 - j2_5)
//   P = tau F^-T
//   b_new = sum_a exp(2 eps_a - 2 dg sqrt(3/2) nhat_a) n_a n_a^T,
//   C^p_new^-1 = F^-1 b_new F^-T                 (equivalent to Eq. j2_10)
//
// The exponential update F^p_new = exp(dg r) F^p_n with r coaxial with the trial
// elastic strain returns exactly to eps_tr - dg r in log space, so this form
// and the paper's (F^p) form give the same P and the same C^p^-1 = F^p^-1 F^p^-T.
//
// Consistent tangent (not derived in the paper): for an isotropic function
// tau(b) with principal values tau_a(lambda),
//   d tau' _aa = sum_b (d tau_a / d eps_b) db'_bb / (2 lambda_b),
//   d tau' _ab = (tau_a - tau_b)/(lambda_a - lambda_b) db'_ab   (a != b),
// primes = components in the eigenbasis, with the algorithmic moduli of the
// radial return d tau_a/d eps_b = lam + 2G beta (delta_ab) + 2G(1-beta)/3 ... (see
// moduli()) and (tau_a - tau_b)/(lambda_a - lambda_b) = G beta L(lambda_a, lambda_b),
// L(x, y) = (ln x - ln y)/(x - y) evaluated through log1p (finite at x = y).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace podecm {

struct PhaseD {
    double E, nu, s0, k, p;
    double lam, G, Kb;   // Lame lambda, shear modulus, bulk modulus
    int law;             // 0 linear, 1 power
    int elastic;         // s0 == +inf
};

// sigma_y(xi) and its slope; for the power law also 1 / (1 + k xi) (rbase, if given)
__device__ __forceinline__ double yield_stress(const PhaseD &ph, double xi, double *slope, double *rbase = nullptr) {
    if (ph.elastic) { *slope = 0.0; return INFINITY; }
    if (ph.law == 0) { *slope = ph.k; return ph.s0 + ph.k * xi; }
    // (1 + k xi)^p as exp(p ln(1 + k xi)): two transcendental calls instead of pow()
    const double base = 1.0 + ph.k * xi;
    const double v = ph.s0 * exp(ph.p * log(base));
    const double rb = 1.0 / base;
    *slope = v * ph.p * ph.k * rb;
    if (rbase) *rbase = rb;
    return v;
}

// symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations (FP64).
// a: symmetric matrix (overwritten: diagonal -> eigenvalues), V: eigenvectors in columns.
__device__ __forceinline__ void jacobi3(double a[3][3], double V[3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 12; ++sweep) {
        const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        const double dg = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (off <= 1e-34 * dg) break;
#pragma unroll
        for (int pq = 0; pq < 3; ++pq) {
            const int p = (pq == 2) ? 1 : 0;
            const int q = (pq == 0) ? 1 : 2;
            const int r = 3 - p - q;
            const double apq = a[p][q];
            if (fabs(apq) <= 1e-300) continue;
            const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            const double c = 1.0 / sqrt(t * t + 1.0);
            const double s = t * c;
            a[p][p] -= t * apq;
            a[q][q] += t * apq;
            a[p][q] = a[q][p] = 0.0;
            const double arp = a[r][p], arq = a[r][q];
            a[r][p] = a[p][r] = c * arp - s * arq;
            a[r][q] = a[q][r] = s * arp + c * arq;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double vkp = V[k][p], vkq = V[k][q];
                V[k][p] = c * vkp - s * vkq;
                V[k][q] = s * vkp + c * vkq;
            }
        }
    }
}

// single-precision Jacobi sweeps (rotation angles only need ~1e-7 accuracy here)
__device__ __forceinline__ void jacobi3_f32(float a[3][3], float V[3][3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) V[i][j] = (i == j) ? 1.f : 0.f;
    for (int sweep = 0; sweep < 8; ++sweep) {
        const float off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        const float dg = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (off <= 1e-14f * dg) break;
#pragma unroll
        for (int pq = 0; pq < 3; ++pq) {
            const int p = (pq == 2) ? 1 : 0;
            const int q = (pq == 0) ? 1 : 2;
            const int r = 3 - p - q;
            const float apq = a[p][q];
            if (fabsf(apq) <= 1e-30f) continue;
            const float theta = (a[q][q] - a[p][p]) / (2.f * apq);
            const float t = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
            const float c = rsqrtf(t * t + 1.f);
            const float sn = t * c;
            a[p][p] -= t * apq;
            a[q][q] += t * apq;
            a[p][q] = a[q][p] = 0.f;
            const float arp = a[r][p], arq = a[r][q];
            a[r][p] = a[p][r] = c * arp - sn * arq;
            a[r][q] = a[q][r] = sn * arp + c * arq;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float vkp = V[k][p], vkq = V[k][q];
                V[k][p] = c * vkp - sn * vkq;
                V[k][q] = sn * vkp + c * vkq;
            }
        }
    }
}

// FP64 -> tangent precision.  For FP32 the conversion truncates the mantissa by integer
// operations on the bit pattern (|x| < 2^-126 flushes to zero, beyond the FP32 range gives
// infinity): the tangent only forms the inexact-Newton Jacobian, and the integer pipe is idle
// while the FP64 pipe, which executes the conversion instruction, bounds the kernel.
template <typename T>
__device__ __forceinline__ T to_tangent(double x) { return T(x); }
template <>
__device__ __forceinline__ float to_tangent<float>(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const uint32_t hi = (uint32_t)(u >> 32), lo = (uint32_t)u;
    const int e = (int)((hi >> 20) & 0x7FFu);
    const uint32_t sign = hi & 0x80000000u;
    if (e < 1023 - 126) return __uint_as_float(sign);
    if (e > 1023 + 127) return __uint_as_float(sign | 0x7F800000u);
    return __uint_as_float(sign | ((uint32_t)(e - 896) << 23) | ((hi & 0xFFFFFu) << 3) | (lo >> 29));
}

// FP32 -> FP64 by integer operations on the bit pattern: exact for normal numbers, infinities
// and NaNs (the exponent is rebiased, the mantissa widened); FP32 subnormals flush to zero.  The
// same value as the conversion instruction, without occupying the FP64 pipe.
__device__ __forceinline__ double f2d_exact(float x) {
    const uint32_t u = __float_as_uint(x);
    const uint32_t e = (u >> 23) & 0xFFu;
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    if (e == 0) return __longlong_as_double((long long)sign);
    const unsigned long long ee = (e == 0xFFu) ? 0x7FFull : (unsigned long long)(e + 896u);
    return __longlong_as_double((long long)(sign | (ee << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29)));
}

// 1/x to ~1e-14 relative: the FP32 reciprocal (x converted by integer operations) and one FP64
// Newton step r (2 - x r).  For |x| in [1e-30, 1e30]; used where the result only scales a
// quantity that is tiny against 1 (Jacobi rotation angles), so that 1e-14 relative error is far
// below FP64 rounding of the final values.
__device__ __forceinline__ double rcp_nr(double x) {
    const double r = f2d_exact(__frcp_rn(to_tangent<float>(x)));
    return r * fma(-x, r, 2.0);
}

// 1 / sqrt(x) for x = 1 + d, |d| <= 1e-6: 1 - d/2 + 3 d^2 / 8 (the next term, 5 d^3 / 16, is
// below 3.2e-19); otherwise the library square root and division
__device__ __forceinline__ double rsqrt_near1(double x) {
    const double d = x - 1.0;
    if (fabs(d) <= 1e-6) return fma(d, fma(0.375, d, -0.5), 1.0);
    return 1.0 / sqrt(x);
}

// FP64 value of an FP64 or FP32 number (FP32 widened by integer operations)
__device__ __forceinline__ double widen(double x) { return x; }
__device__ __forceinline__ double widen(float x) { return f2d_exact(x); }

// ln x near 1 and exp x near 0 by their power series (Mercator's series of ln(1 + u) and the
// exponential series), for the Hencky strains of the trial state (eigenvalues of b_tr within a few
// percent of 1) and the plastic update (exponents 2 dg sqrt(3/2) |nhat_a| <= 2 dg): a handful of
// FP64 FMAs instead of the library's range reduction.  ln: u = x - 1 (exact), |u| <= 1/32, terms to
// u^11 / 11 (truncation below 3e-18 relative); exp: |x| <= 1/16, terms to x^9 / 9! (below 3e-18
// relative).  Outside these ranges the library functions.  The same series give the power-law
// yield stress after an increment from the known sigma_y(xi_n) (see power_increment).
__device__ __forceinline__ double log1p_series(double u) {   // |u| <= 1/32
    double p = 1.0 / 11.0;
    p = fma(u, p, -1.0 / 10.0);
    p = fma(u, p, 1.0 / 9.0);
    p = fma(u, p, -1.0 / 8.0);
    p = fma(u, p, 1.0 / 7.0);
    p = fma(u, p, -1.0 / 6.0);
    p = fma(u, p, 1.0 / 5.0);
    p = fma(u, p, -1.0 / 4.0);
    p = fma(u, p, 1.0 / 3.0);
    p = fma(u, p, -0.5);
    p = fma(u, p, 1.0);
    return u * p;
}

__device__ __forceinline__ double log_near1(double x) {
    const double u = x - 1.0;
    if (fabs(u) <= 0.03125) return log1p_series(u);
    return log(x);
}

__device__ __forceinline__ double log1p_near0(double u) {
    if (fabs(u) <= 0.03125) return log1p_series(u);
    return log1p(u);
}

__device__ __forceinline__ double exp_near0(double x) {
    if (fabs(x) <= 0.0625) {
        double p = 1.0 / 362880.0;
        p = fma(x, p, 1.0 / 40320.0);
        p = fma(x, p, 1.0 / 5040.0);
        p = fma(x, p, 1.0 / 720.0);
        p = fma(x, p, 1.0 / 120.0);
        p = fma(x, p, 1.0 / 24.0);
        p = fma(x, p, 1.0 / 6.0);
        p = fma(x, p, 0.5);
        p = fma(x, p, 1.0);
        return fma(x, p, 1.0);
    }
    return exp(x);
}

// power-law yield stress after a plastic increment x from xi_n, from sy_n = sigma_y(xi_n) and
// rb_n = 1 / (1 + k xi_n): 1 + k (xi_n + x) = (1 + k xi_n)(1 + u) with u = k x rb_n, so
// sigma_y(xi_n + x) = sy_n (1 + u)^p = sy_n exp(p ln(1 + u)), and the slope is
// p k sigma_y / (1 + k (xi_n + x)).  Return-map increments keep |u| and |p ln(1 + u)| inside
// the ranges of the short series; larger ones take the library functions.
__device__ __forceinline__ double power_increment(const PhaseD &ph, double sy_n, double rb_n, double x,
                                                  double *slope) {
    const double u = ph.k * x * rb_n;
    const double v = sy_n * exp_near0(ph.p * log1p_near0(u));
    *slope = v * ph.p * ph.k * rb_n / (1.0 + u);
    return v;
}

// FP64-accurate symmetric 3x3 eigen-decomposition: FP32 Jacobi gives approximate
// eigenvectors, which are made exactly orthonormal in FP64 (Gram-Schmidt + cross product; the
// FP32 vectors have norms within ~1e-7 of 1, so their normalisation is a short series) and used
// to rotate b in FP64; FP64 Jacobi sweeps then finish the nearly diagonal matrix (the first
// sweep from off-diagonals ~1e-7 |lambda|, the second from ~1e-14 |lambda|).  Rotation
// t = tan(angle) by the size of e = 2 a_pq / (a_qq - a_pp):
//   |e| <= 1e-8: t = e / 2 and c = 1 (t^2 / 2 < 1.3e-17, below FP64 rounding of 1);
//   |e| <= 1e-3: the series t = e/2 - e^3/8, c = 1 - t^2/2 + 3 t^4/8 (truncation below 1e-16);
//   otherwise the closed form.
// In the first two cases e is formed with rcp_nr (its 1e-14 relative error moves t by less
// than 1e-17 absolute).
// Input b = F C F^T given by F and C (symmetric): b itself is formed only in FP32 for the
// approximate start; the FP64 matrix is Q^T b Q = W^T C W with W = F^T Q.
__device__ __forceinline__ void eig3_mixed(const double F[3][3], const double C[3][3], double lam[3], double N[3][3]) {
    float af[3][3], Vf[3][3];
    {
        float Ff[3][3], Cf[3][3], Zf[3][3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) { Ff[i][j] = to_tangent<float>(F[i][j]); Cf[i][j] = to_tangent<float>(C[i][j]); }
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) Zf[i][j] = Cf[i][0] * Ff[j][0] + Cf[i][1] * Ff[j][1] + Cf[i][2] * Ff[j][2];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = i; j < 3; ++j) af[i][j] = af[j][i] = Ff[i][0] * Zf[0][j] + Ff[i][1] * Zf[1][j] + Ff[i][2] * Zf[2][j];
    }
    jacobi3_f32(af, Vf);   // approximate start only
    double q0[3], q1[3], q2[3];
    {
        double n0 = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) { q0[k] = f2d_exact(Vf[k][0]); n0 += q0[k] * q0[k]; }
        const double i0 = rsqrt_near1(n0);
#pragma unroll
        for (int k = 0; k < 3; ++k) q0[k] *= i0;
        double dt = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) dt += q0[k] * f2d_exact(Vf[k][1]);
        double n1 = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) { q1[k] = f2d_exact(Vf[k][1]) - dt * q0[k]; n1 += q1[k] * q1[k]; }
        const double i1 = rsqrt_near1(n1);
#pragma unroll
        for (int k = 0; k < 3; ++k) q1[k] *= i1;
        q2[0] = q0[1] * q1[2] - q0[2] * q1[1];
        q2[1] = q0[2] * q1[0] - q0[0] * q1[2];
        q2[2] = q0[0] * q1[1] - q0[1] * q1[0];
    }
    const double Q[3][3] = {{q0[0], q1[0], q2[0]}, {q0[1], q1[1], q2[1]}, {q0[2], q1[2], q2[2]}};
    double a[3][3], W[3][3], T[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double sm = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) sm += F[k][i] * Q[k][j];
            W[i][j] = sm;
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double sm = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) sm += C[i][k] * W[k][j];
            T[i][j] = sm;
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            double sm = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) sm += W[k][i] * T[k][j];
            a[i][j] = sm;
            a[j][i] = sm;
        }
    double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int sweep = 0; sweep < 12; ++sweep) {
        const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
        const double dg = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
        if (off <= 1e-34 * dg) break;
#pragma unroll
        for (int pq = 0; pq < 3; ++pq) {
            const int p = (pq == 2) ? 1 : 0;
            const int q = (pq == 0) ? 1 : 2;
            const int r = 3 - p - q;
            const double apq = a[p][q];
            if (fabs(apq) <= 1e-300) continue;
            const double gap = a[q][q] - a[p][p];
            const double ag = fabs(gap);
            double t, c;
            if (fabs(2.0 * apq) <= 1e-8 * ag && ag >= 1e-30 && ag <= 1e30) {
                // tiny angle: a rotation with c = 1
                t = apq * rcp_nr(gap);
                a[p][p] -= t * apq;
                a[q][q] += t * apq;
                a[p][q] = a[q][p] = 0.0;
                const double arp = a[r][p], arq = a[r][q];
                a[r][p] = a[p][r] = fma(-t, arq, arp);
                a[r][q] = a[q][r] = fma(t, arp, arq);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = fma(-t, vkq, vkp);
                    V[k][q] = fma(t, vkp, vkq);
                }
                continue;
            }
            if (fabs(2.0 * apq) <= 1e-3 * ag) {
                const double e = (ag >= 1e-30 && ag <= 1e30) ? 2.0 * apq * rcp_nr(gap) : 2.0 * apq / gap;
                t = 0.5 * e - 0.125 * e * e * e;
                const double t2 = t * t;
                c = 1.0 - 0.5 * t2 + 0.375 * t2 * t2;
            } else {
                const double theta = gap / (2.0 * apq);
                t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                c = 1.0 / sqrt(t * t + 1.0);
            }
            const double sn = t * c;
            a[p][p] -= t * apq;
            a[q][q] += t * apq;
            a[p][q] = a[q][p] = 0.0;
            const double arp = a[r][p], arq = a[r][q];
            a[r][p] = a[p][r] = c * arp - sn * arq;
            a[r][q] = a[q][r] = sn * arp + c * arq;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const double vkp = V[k][p], vkq = V[k][q];
                V[k][p] = c * vkp - sn * vkq;
                V[k][q] = sn * vkp + c * vkq;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        lam[i] = a[i][i];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double sm = 0.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) sm += Q[i][k] * V[k][j];
            N[i][j] = sm;
        }
    }
}

// (ln x - ln y) / (x - y) for x, y > 0, finite and accurate when x ~ y
template <typename T>
__device__ __forceinline__ T log_divided_difference(T x, T y) {
    const T u = y / x - T(1);
    if (fabs(u) < T(1e-8)) return (T(1) - T(0.5) * u) / x;
    return log1p(u) / (u * x);
}

// Result of the value part of the update at one point.
struct MatState {
    double N[3][3];      // eigenvectors of b_tr (columns)
    double lam[3];       // eigenvalues of b_tr
    double tau[3];       // principal Kirchhoff stresses
    double nh[3];        // unit deviatoric direction of the trial log strain
    double beta;         // 1 - 3 G dg / q_tr (1 if elastic)
    double dg, q_tr, hs; // plastic multiplier, trial von Mises, hardening slope at xi_n + dg
    int plastic;
};

// Value part.  F: 3x3 (plane strain: F[2][2] = 1, F[i][2] = F[2][i] = 0), cp: C^p^-1
// (00, 01, 02, 11, 12, 22).  Outputs the state, the first Piola-Kirchhoff stress P = tau F^-T
// (3x3), F^-1, the updated history cp_new, xi_new.  D = 2 uses the block structure.
template <int D, bool FP64_SLOPE = true>
__device__ __forceinline__ void material_value(const double F[3][3], const double cp[6], double xi_n,
                                               const PhaseD &ph, MatState &S, double P[3][3],
                                               double Finv[3][3], double cp_new[6], double *xi_new) {
    // plane strain (D = 2): F, C^p^-1 and every tensor below are block-diagonal, the in-plane
    // 2 x 2 block and the 33 entry (F_33 = 1); only those entries are formed (the FP64 products
    // with the structural zeros would cost FP64 issue slots: x * 0 is not folded under IEEE rules)
    constexpr int K = D == 2 ? 2 : 3;
    const double C[3][3] = {{cp[0], cp[1], cp[2]}, {cp[1], cp[3], cp[4]}, {cp[2], cp[4], cp[5]}};
    if (D == 2) {
        // b = F C F^T (in-plane block; b_33 = c_33): Z = C F^T, b = F Z
        double Z[2][2], b[2][2];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) Z[i][j] = C[i][0] * F[j][0] + C[i][1] * F[j][1];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = i; j < 2; ++j) b[i][j] = b[j][i] = F[i][0] * Z[0][j] + F[i][1] * Z[1][j];
        // one Jacobi rotation diagonalises the in-plane block; axis 3 is principal
        double c = 1.0, s = 0.0;
        const double apq = b[0][1];
        if (fabs(apq) > 1e-300) {
            const double theta = (b[1][1] - b[0][0]) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
            S.lam[0] = b[0][0] - t * apq;
            S.lam[1] = b[1][1] + t * apq;
        } else {
            S.lam[0] = b[0][0];
            S.lam[1] = b[1][1];
        }
        S.lam[2] = cp[5];
        S.N[0][0] = c;  S.N[0][1] = s;  S.N[0][2] = 0.0;
        S.N[1][0] = -s; S.N[1][1] = c;  S.N[1][2] = 0.0;
        S.N[2][0] = 0.0; S.N[2][1] = 0.0; S.N[2][2] = 1.0;
    } else {
        eig3_mixed(F, C, S.lam, S.N);
    }
    double eps[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) eps[a] = 0.5 * log_near1(S.lam[a]);
    const double tr = eps[0] + eps[1] + eps[2];
    const double mean = tr * (1.0 / 3.0);
    double e[3] = {eps[0] - mean, eps[1] - mean, eps[2] - mean};
    const double enorm = sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
    const double G = ph.G;
    S.q_tr = sqrt(6.0) * G * enorm;
    // FP32 copies by integer operations on the bit patterns (the conversion instruction would
    // occupy the FP64 pipe): the power-law constants and the trial state, for the FP32 filter and
    // the FP32 Newton start below
    const bool pw = ph.law == 1 && !ph.elastic;
    const float qf = to_tangent<float>(S.q_tr), xin = to_tangent<float>(xi_n);
    const float s0f = to_tangent<float>(ph.s0), kf = to_tangent<float>(ph.k), pf = to_tangent<float>(ph.p);
    // yield check (Eq. j2_2).  Power law: sigma_y(xi_n) in FP32 (relative error < 1e-6) decides the
    // points more than 1e-5 below the yield surface elastic without the FP64 evaluation; the FP64
    // test decides all others, so the decision is the FP64 test's everywhere
    float syf = 0.f;
    bool maybe_plastic = true;
    if (pw) {
        syf = s0f * expf(pf * logf(1.f + kf * xin));
        maybe_plastic = qf >= syf * (1.f - 1e-5f);
    }
    double h0 = 0.0, sy_n = 0.0, rb_n = 0.0;
    if (maybe_plastic) sy_n = yield_stress(ph, xi_n, &h0, &rb_n);
    S.plastic = maybe_plastic && (S.q_tr - sy_n) > 1e-12 * sy_n;
    S.dg = 0.0;
    S.beta = 1.0;
    S.hs = h0;
    if (S.plastic) {
        // power law: Newton in FP32 first (cheap pipe) to ~1e-7 from the FP32 linearised start,
        // then FP64 Newton steps; from an FP32-accurate start one FP64 step reaches FP64 precision
        // (quadratic convergence, and the hardening curvature is small against 3G), so the FP64
        // loop stops once a step is below 1e-6 |dg| (otherwise at 1e-15 |dg|, as from the FP64
        // linearised start)
        bool conv32 = false;
        float xf = 0.f, hsf = 0.f;
        if (pw) {
            const float g3 = to_tangent<float>(3.0 * G);
            xf = (qf - syf) / (g3 + syf * pf * kf / (1.f + kf * xin));
            for (int it = 0; it < 30; ++it) {
                const float base = 1.f + kf * (xin + xf);
                const float sy = s0f * expf(pf * logf(base));
                hsf = sy * pf * kf / base;
                const float step = (qf - g3 * xf - sy) / (g3 + hsf);
                xf += step;
                if (fabsf(step) <= 1e-6f * fabsf(xf)) { conv32 = isfinite(xf) && xf > 0.f; break; }
            }
        }
        double x = conv32 ? f2d_exact(xf) : (S.q_tr - sy_n) / (3.0 * G + h0);
        double hs = h0;
        if (!FP64_SLOPE && conv32) {
            // FP32 tangent: one FP64 Newton step from the FP32 solution (relative error ~1e-7) on
            // the FP64 residual, with the FP32 slope in the denominator (its ~1e-7 relative error
            // moves the result by ~1e-14 of the step); that slope also serves the FP32 tangent
            hs = f2d_exact(hsf);
            const double sy = sy_n * exp_near0(ph.p * log1p_near0(ph.k * x * rb_n));
            x += (S.q_tr - 3.0 * G * x - sy) / (3.0 * G + hs);
        } else {
            for (int it = 0; it < 60; ++it) {
                const double sy = pw ? power_increment(ph, sy_n, rb_n, x, &hs) : yield_stress(ph, xi_n + x, &hs);
                const double step = (S.q_tr - 3.0 * G * x - sy) / (3.0 * G + hs);
                x += step;
                if (fabs(step) <= 1e-15 * fabs(x)) break;
                if (conv32 && fabs(step) <= 1e-6 * fabs(x)) break;
            }
            if (FP64_SLOPE) {
                if (pw) power_increment(ph, sy_n, rb_n, x, &hs);
                else yield_stress(ph, xi_n + x, &hs);
            } else if (ph.law == 1) {
                // slope for the (FP32) tangent only
                const float base = 1.f + kf * (xin + to_tangent<float>(x));
                hs = f2d_exact(s0f * expf(pf * logf(base)) * pf * kf / base);
            } else {
                hs = ph.k;
            }
        }
        S.dg = x;
        S.hs = hs;
        S.beta = 1.0 - 3.0 * G * x / S.q_tr;
        const double ien = 1.0 / enorm;
#pragma unroll
        for (int a = 0; a < 3; ++a) S.nh[a] = e[a] * ien;
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) S.nh[a] = 0.0;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) S.tau[a] = ph.Kb * tr + 2.0 * G * S.beta * e[a];
    // F^-1 (adjugate)
    if (D == 2) {
        const double det = F[0][0] * F[1][1] - F[0][1] * F[1][0];
        const double id = 1.0 / det;
        Finv[0][0] = F[1][1] * id;
        Finv[0][1] = -F[0][1] * id;
        Finv[1][0] = -F[1][0] * id;
        Finv[1][1] = F[0][0] * id;
        Finv[0][2] = Finv[1][2] = Finv[2][0] = Finv[2][1] = 0.0;
        Finv[2][2] = 1.0;
        if (!(det > 0.0)) Finv[0][0] = NAN;   // det F <= 0: flagged as non-finite stress
    } else {
        double c00 = F[1][1] * F[2][2] - F[1][2] * F[2][1];
        double c01 = F[1][2] * F[2][0] - F[1][0] * F[2][2];
        double c02 = F[1][0] * F[2][1] - F[1][1] * F[2][0];
        const double det = F[0][0] * c00 + F[0][1] * c01 + F[0][2] * c02;
        const double id = 1.0 / det;
        Finv[0][0] = c00 * id;
        Finv[1][0] = c01 * id;
        Finv[2][0] = c02 * id;
        Finv[0][1] = (F[0][2] * F[2][1] - F[0][1] * F[2][2]) * id;
        Finv[1][1] = (F[0][0] * F[2][2] - F[0][2] * F[2][0]) * id;
        Finv[2][1] = (F[0][1] * F[2][0] - F[0][0] * F[2][1]) * id;
        Finv[0][2] = (F[0][1] * F[1][2] - F[0][2] * F[1][1]) * id;
        Finv[1][2] = (F[0][2] * F[1][0] - F[0][0] * F[1][2]) * id;
        Finv[2][2] = (F[0][0] * F[1][1] - F[0][1] * F[1][0]) * id;
        if (!(det > 0.0)) Finv[0][0] = NAN;   // det F <= 0: flagged as non-finite stress
    }
    // M = F^-1 N: P = tau F^-T = N diag(tau_a) N^T F^-T = N diag(tau_a) M^T, and the plastic
    // history below C^p_new^-1 = F^-1 b_new F^-T = M diag(b_new,a) M^T
    double Mx[3][3];
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
        for (int a = 0; a < K; ++a) {
            double s = 0.0;
#pragma unroll
            for (int k = 0; k < K; ++k) s += Finv[i][k] * S.N[k][a];
            Mx[i][a] = s;
        }
#pragma unroll
    for (int i = 0; i < K; ++i) {
        double nt[3];
#pragma unroll
        for (int a = 0; a < K; ++a) nt[a] = S.N[i][a] * S.tau[a];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            double s = 0.0;
#pragma unroll
            for (int a = 0; a < K; ++a) s += nt[a] * Mx[j][a];
            P[i][j] = s;
        }
    }
    if (D == 2) {
        P[0][2] = P[1][2] = P[2][0] = P[2][1] = 0.0;
        P[2][2] = S.tau[2];   // F_33 = 1, N_33 = 1
    }
    if (S.plastic) {
        // b_new = N diag(lambda_a exp(-2 dg sqrt(3/2) nhat_a)) N^T (Eq. j2_10 in the spatial form)
        double ln[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) ln[a] = S.lam[a] * exp_near0(-2.0 * S.dg * 1.2247448713915890491 * S.nh[a]);
        double c[3][3];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            double ml[3];
#pragma unroll
            for (int a = 0; a < K; ++a) ml[a] = Mx[i][a] * ln[a];
#pragma unroll
            for (int j = i; j < K; ++j) {
                double s = 0.0;
#pragma unroll
                for (int a = 0; a < K; ++a) s += ml[a] * Mx[j][a];
                c[i][j] = s;
            }
        }
        if (D == 2) {
            c[0][2] = c[1][2] = 0.0;
            c[2][2] = ln[2];   // F_33 = 1
        }
        cp_new[0] = c[0][0]; cp_new[1] = c[0][1]; cp_new[2] = c[0][2];
        cp_new[3] = c[1][1]; cp_new[4] = c[1][2]; cp_new[5] = c[2][2];
        *xi_new = xi_n + S.dg;
    } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) cp_new[k] = cp[k];
        *xi_new = xi_n;
    }
}

// Tangent data in the eigenbasis (precision T).
template <typename T>
struct TangentData {
    T N[3][3];
    T c[3][3];      // d tau_a / d eps_b
    T th[3];        // theta_01, theta_02, theta_12
    T inv2l[3];     // 1 / (2 lambda_a)
    T Z[3][3];      // C^p^-1 F^T
    T Finv[3][3];   // F^-1
    T P[3][3];      // first Piola-Kirchhoff stress
};

template <int D, typename T>
__device__ __forceinline__ void tangent_setup(const MatState &S, const PhaseD &ph, const double F[3][3],
                                              const double cp[6], const double Finv[3][3],
                                              const double P[3][3], TangentData<T> &td) {
    // all in the tangent precision T (FP64 path: double; mixed path: float on the FP32 pipe)
    const T G = to_tangent<T>(ph.G), beta = to_tangent<T>(S.beta);
    // algorithmic moduli of the radial return in principal log strains
    T cpl = T(0);
    if (S.plastic) cpl = T(6) * G * G * (T(1) / (T(3) * G + to_tangent<T>(S.hs)) - to_tangent<T>(S.dg) / to_tangent<T>(S.q_tr));
    // plane strain: an in-plane direction dF leaves db, and with it every eigenbasis quantity
    // below, in the in-plane block, so only that block of c, Z, N, F^-1 and P is formed
    constexpr int K = D == 2 ? 2 : 3;
    const T nh[3] = {to_tangent<T>(S.nh[0]), to_tangent<T>(S.nh[1]), to_tangent<T>(S.nh[2])};
#pragma unroll
    for (int a = 0; a < K; ++a)
#pragma unroll
        for (int b = 0; b < K; ++b)
            td.c[a][b] = to_tangent<T>(ph.Kb) + T(2) * G * beta * ((a == b ? T(1) : T(0)) - T(1) / T(3)) - cpl * nh[a] * nh[b];
    const T gb = G * beta;
    const T l0 = to_tangent<T>(S.lam[0]), l1 = to_tangent<T>(S.lam[1]), l2 = to_tangent<T>(S.lam[2]);
    td.th[0] = gb * log_divided_difference<T>(l0, l1);
    if (D == 3) {
        td.th[1] = gb * log_divided_difference<T>(l0, l2);
        td.th[2] = gb * log_divided_difference<T>(l1, l2);
    } else {
        // plane strain: db'_a2 = 0 for in-plane directions, so the out-of-plane pairs never enter
        td.th[1] = T(0);
        td.th[2] = T(0);
    }
    td.inv2l[0] = T(0.5) / l0;
    td.inv2l[1] = T(0.5) / l1;
    td.inv2l[2] = D == 2 ? T(0) : T(0.5) / l2;
    T C[3][3], Ft[3][3];
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
        for (int j = 0; j < K; ++j) Ft[i][j] = to_tangent<T>(F[i][j]);
    C[0][0] = to_tangent<T>(cp[0]); C[0][1] = C[1][0] = to_tangent<T>(cp[1]); C[0][2] = C[2][0] = to_tangent<T>(cp[2]);
    C[1][1] = to_tangent<T>(cp[3]); C[1][2] = C[2][1] = to_tangent<T>(cp[4]); C[2][2] = to_tangent<T>(cp[5]);
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
        for (int j = 0; j < K; ++j) {
            T s = T(0);
#pragma unroll
            for (int k = 0; k < K; ++k) s += C[i][k] * Ft[j][k];
            td.Z[i][j] = s;
            td.N[i][j] = to_tangent<T>(S.N[i][j]);
            td.Finv[i][j] = to_tangent<T>(Finv[i][j]);
            td.P[i][j] = to_tangent<T>(P[i][j]);
        }
}

// x_c of (x_0, x_1, x_2) by selects, so that a run-time c indexes no array (an array indexed at
// run time would be placed in local memory)
template <int D, typename T>
__device__ __forceinline__ T pick(int c, T x0, T x1, T x2) {
    return D == 2 ? (c == 0 ? x0 : x1) : (c == 0 ? x0 : (c == 1 ? x1 : x2));
}

// dP for the direction dF = e_c (x) f  (dF_kl = delta_kc f_l).  Only the D x D block is formed.
template <int D, typename T>
__device__ __forceinline__ void tangent_direction(const TangentData<T> &td, int c, const T f[3], T dP[3][3]) {
    T Nc[3], Fc[3];   // row c of N, column c of F^-1
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Nc[a] = pick<D, T>(c, td.N[0][a], td.N[1][a], td.N[2][a]);
        Fc[a] = pick<D, T>(c, td.Finv[a][0], td.Finv[a][1], td.Finv[a][2]);
    }
    // plane strain: dF, db and the eigenbasis components stay in the in-plane block (K = 2)
    constexpr int K = D == 2 ? 2 : 3;
    // g = Z^T f, h = N^T g
    T g[3], h[3];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        T s = T(0);
#pragma unroll
        for (int l = 0; l < D; ++l) s += td.Z[l][j] * f[l];
        g[j] = s;
    }
#pragma unroll
    for (int a = 0; a < K; ++a) {
        T s = T(0);
#pragma unroll
        for (int j = 0; j < K; ++j) s += td.N[j][a] * g[j];
        h[a] = s;
    }
    // db'_ab = N_ca h_b + h_a N_cb
    T dbp[3][3];
#pragma unroll
    for (int a = 0; a < K; ++a)
#pragma unroll
        for (int b = a; b < K; ++b) {
            dbp[a][b] = Nc[a] * h[b] + h[a] * Nc[b];
            dbp[b][a] = dbp[a][b];
        }
    T dt[3][3];
    T w[3];
#pragma unroll
    for (int a = 0; a < K; ++a) w[a] = dbp[a][a] * td.inv2l[a];
#pragma unroll
    for (int a = 0; a < K; ++a) {
        T s = T(0);
#pragma unroll
        for (int b = 0; b < K; ++b) s += td.c[a][b] * w[b];
        dt[a][a] = s;
    }
    dt[0][1] = dt[1][0] = td.th[0] * dbp[0][1];
    if (D == 3) {
        dt[0][2] = dt[2][0] = td.th[1] * dbp[0][2];
        dt[1][2] = dt[2][1] = td.th[2] * dbp[1][2];
    }
    // d tau = N dt N^T (D x D block), then dP = d tau F^-T - (P f) (x) F^-1[:, c]
    T M[3][3];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int b = 0; b < K; ++b) {
            T s = T(0);
#pragma unroll
            for (int a = 0; a < K; ++a) s += td.N[i][a] * dt[a][b];
            M[i][b] = s;
        }
    T dtau[3][3];
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            T s = T(0);
#pragma unroll
            for (int b = 0; b < K; ++b) s += M[i][b] * td.N[j][b];
            dtau[i][j] = s;
        }
    T Pf[3];
#pragma unroll
    for (int i = 0; i < D; ++i) {
        T s = T(0);
#pragma unroll
        for (int l = 0; l < D; ++l) s += td.P[i][l] * f[l];
        Pf[i] = s;
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            T s = T(0);
#pragma unroll
            for (int k = 0; k < D; ++k) s += dtau[i][k] * td.Finv[j][k];
            dP[i][j] = s - Pf[i] * Fc[j];
        }
}

}  // namespace podecm
