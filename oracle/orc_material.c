/*
 * ORACLE — test infrastructure only.  Plain FP64 CPU reference of the
 * finite-strain J2 material point of the paper (Appendix A), used by the
 * tests, by smoke() and by the CPU-baseline leg of bench.py.  It shares no
 * code with the CUDA path.
 *
 * Route (the paper's own, Appendix A):
 *   F = F^el F^pl  (multiplicative split)
 *   C^el = F^elT F^el,  eps = 1/2 ln C^el           (log strain, Eq. j2_7;
 *                                                     factor 1/2 = Hencky reading)
 *   sigma = D : (eps - eps^pl)                       (Eq. j2_1, in log space)
 *   f = ||sigma||_mises - sigma_y(xi)                (Eq. j2_2)
 *   r = sqrt(3/2) dev(sigma)/|dev(sigma)|            (Eq. j2_3)
 *   xi_{k+1} = xi_k + gamma,                         (Eq. j2_4)
 *   F^pl_{k+1} = exp(gamma r) F^pl_k                 (Eq. j2_10)
 *   P = F^el,-T sigma F^pl,-T                        (Eq. j2_9, read as the
 *       pull-back F^el S F^pl,-T with S = sigma : d ln C/dC = C^el,-1 sigma)
 *
 * The matrix logarithm uses the Gregory (inverse hyperbolic tangent) series
 * log X = 2 atanh((X-I)(X+I)^-1) after square roots (Denman-Beavers) bring X
 * near I; the exponential uses Taylor + scaling and squaring (Higham,
 * Functions of Matrices, 2008, ch. 10-11).  Every step is written on dual
 * numbers (value + one directional derivative), so running the material
 * once per direction E_kl gives the consistent tangent A = dP/dF exactly
 * (forward-mode differentiation); the return-map scalar Newton is
 * differentiated by one dual Newton step at the converged root (implicit
 * function theorem).  No eigen-decomposition is used anywhere.
 */
#include <math.h>
#include <string.h>
#include "orc.h"

typedef struct { double v, d; } dual;

static inline dual mk(double v, double d) { dual r; r.v = v; r.d = d; return r; }
static inline dual cst(double v) { return mk(v, 0.0); }
static inline dual add(dual a, dual b) { return mk(a.v + b.v, a.d + b.d); }
static inline dual sub(dual a, dual b) { return mk(a.v - b.v, a.d - b.d); }
static inline dual mul(dual a, dual b) { return mk(a.v * b.v, a.d * b.v + a.v * b.d); }
static inline dual scl(dual a, double s) { return mk(a.v * s, a.d * s); }
static inline dual dvd(dual a, dual b) { double q = a.v / b.v; return mk(q, (a.d - q * b.d) / b.v); }
static inline dual dsqrt(dual a) { double s = sqrt(a.v); return mk(s, a.d / (2.0 * s)); }

typedef struct { dual a[3][3]; } dmat;

static dmat m_zero(void) { dmat r; memset(&r, 0, sizeof r); return r; }
static dmat m_eye(void) { dmat r = m_zero(); for (int i = 0; i < 3; ++i) r.a[i][i] = cst(1.0); return r; }
static dmat m_from(const double *x) { dmat r; for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) r.a[i][j] = cst(x[3 * i + j]); return r; }
static dmat m_add(dmat x, dmat y) { dmat r; for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) r.a[i][j] = add(x.a[i][j], y.a[i][j]); return r; }
static dmat m_sub(dmat x, dmat y) { dmat r; for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) r.a[i][j] = sub(x.a[i][j], y.a[i][j]); return r; }
static dmat m_scl(dmat x, double s) { dmat r; for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) r.a[i][j] = scl(x.a[i][j], s); return r; }
static dmat m_scld(dmat x, dual s) { dmat r; for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) r.a[i][j] = mul(x.a[i][j], s); return r; }
static dmat m_tr(dmat x) { dmat r; for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) r.a[i][j] = x.a[j][i]; return r; }
static dmat m_mul(dmat x, dmat y) {
    dmat r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            dual s = cst(0.0);
            for (int k = 0; k < 3; ++k) s = add(s, mul(x.a[i][k], y.a[k][j]));
            r.a[i][j] = s;
        }
    return r;
}
static dual m_trace(dmat x) { return add(add(x.a[0][0], x.a[1][1]), x.a[2][2]); }
static dual m_det(dmat x) {
    dual c0 = sub(mul(x.a[1][1], x.a[2][2]), mul(x.a[1][2], x.a[2][1]));
    dual c1 = sub(mul(x.a[1][2], x.a[2][0]), mul(x.a[1][0], x.a[2][2]));
    dual c2 = sub(mul(x.a[1][0], x.a[2][1]), mul(x.a[1][1], x.a[2][0]));
    return add(add(mul(x.a[0][0], c0), mul(x.a[0][1], c1)), mul(x.a[0][2], c2));
}
/* inverse by the adjugate (cofactor) formula */
static dmat m_inv(dmat x) {
    dmat c;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
            c.a[j][i] = sub(mul(x.a[i1][j1], x.a[i2][j2]), mul(x.a[i1][j2], x.a[i2][j1]));
        }
    dual det = m_det(x);
    dmat r;
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) r.a[i][j] = dvd(c.a[i][j], det);
    return r;
}
static double m_frob_v(dmat x) { double s = 0; for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) s += x.a[i][j].v * x.a[i][j].v; return sqrt(s); }
static dual m_ddot(dmat x, dmat y) { dual s = cst(0); for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) s = add(s, mul(x.a[i][j], y.a[i][j])); return s; }

/* principal square root of an SPD matrix: Denman-Beavers iteration */
static dmat m_sqrt_db(dmat a) {
    dmat y = a, z = m_eye();
    for (int it = 0; it < 60; ++it) {
        dmat yi = m_inv(y), zi = m_inv(z);
        dmat yn = m_scl(m_add(y, zi), 0.5), zn = m_scl(m_add(z, yi), 0.5);
        double ch = m_frob_v(m_sub(yn, y)) / (m_frob_v(yn) + 1e-300);
        y = yn; z = zn;
        if (ch < 1e-17 && it > 3) break;
    }
    return y;
}

/* log of an SPD matrix: k square roots until ||X-I|| <= 1/4, then
 * log X = 2^k * 2 * sum_j Z^(2j+1)/(2j+1),  Z = (X-I)(X+I)^-1.
 * With ||X-I||_F <= 1/4 every eigenvalue of Z is <= 1/7 in modulus, so 16
 * terms leave a remainder far below double rounding.                      */
static dmat m_log_spd(dmat x) {
    int k = 0;
    dmat I = m_eye();
    while (m_frob_v(m_sub(x, I)) > 0.25 && k < 40) { x = m_sqrt_db(x); ++k; }
    dmat z = m_mul(m_sub(x, I), m_inv(m_add(x, I)));
    dmat z2 = m_mul(z, z), term = z, s = z;
    for (int j = 1; j <= 16; ++j) {
        term = m_mul(term, z2);
        dmat add_ = m_scl(term, 1.0 / (2.0 * j + 1.0));
        s = m_add(s, add_);
        /* stop once the added term (value and derivative) is below double rounding of the sum */
        double tv = 0.0, td = 0.0, sv = 0.0, sd = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                tv += fabs(add_.a[a][b].v); td += fabs(add_.a[a][b].d);
                sv += fabs(s.a[a][b].v); sd += fabs(s.a[a][b].d);
            }
        if (tv <= 1e-18 * sv && td <= 1e-18 * (sd + sv)) break;
    }
    return m_scl(s, 2.0 * ldexp(1.0, k));
}

/* exp of a matrix: scale by 2^-s so that ||X|| <= 1/16, Taylor to 18 terms,
 * square s times. */
static dmat m_exp(dmat x) {
    double nrm = m_frob_v(x);
    int s = 0;
    while (nrm > 0.0625 && s < 60) { nrm *= 0.5; ++s; }
    dmat xs = m_scl(x, ldexp(1.0, -s));
    dmat I = m_eye(), term = I, sum = I;
    for (int j = 1; j <= 18; ++j) {
        term = m_scl(m_mul(term, xs), 1.0 / j);
        sum = m_add(sum, term);
        double tv = 0.0, td = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) { tv += fabs(term.a[a][b].v); td += fabs(term.a[a][b].d); }
        if (tv <= 1e-19 && td <= 1e-19 * (1.0 + tv)) break;
    }
    for (int j = 0; j < s; ++j) sum = m_mul(sum, sum);
    return sum;
}

/* yield stress sigma_y(xi) and its slope (hardening law of the phase) */
double orc_sigma_y(const orc_phase *ph, double xi, double *slope) {
    if (isinf(ph->s0)) { if (slope) *slope = 0.0; return INFINITY; }
    if (ph->hard_law == ORC_HARD_LINEAR) {
        if (slope) *slope = ph->H_or_k;
        return ph->s0 + ph->H_or_k * xi;
    }
    double base = 1.0 + ph->H_or_k * xi;
    double v = ph->s0 * pow(base, ph->p);
    if (slope) *slope = ph->s0 * ph->p * ph->H_or_k * pow(base, ph->p - 1.0);
    return v;
}

/*
 * One material-point update along one direction dF.
 * F, dF, Fp_n, P, dP, Fp_new: 3x3 row-major.  Returns 1 if the point is
 * plastic (f > 1e-12 sigma_y(xi_n)), else 0.
 */
int orc_material_dir(const double *F, const double *dF, const double *Fp_n, double xi_n,
                     const orc_phase *ph, double *P, double *dP, double *Fp_new, double *xi_new)
{
    dmat Fd;
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) Fd.a[i][j] = mk(F[3 * i + j], dF ? dF[3 * i + j] : 0.0);
    const double E = ph->E, nu = ph->nu;
    const double G = E / (2.0 * (1.0 + nu));
    const double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));

    dmat Fpn = m_from(Fp_n);
    dmat Fe_tr = m_mul(Fd, m_inv(Fpn));                 /* trial elastic part */
    dmat Ce_tr = m_mul(m_tr(Fe_tr), Fe_tr);
    dmat eps = m_scl(m_log_spd(Ce_tr), 0.5);           /* Eq. j2_7 (Hencky) */
    dual treps = m_trace(eps);
    dmat sig_tr = m_add(m_scl(m_scld(m_eye(), treps), lam / 1.0), m_scl(eps, 2.0 * G)); /* Eq. j2_1 */
    dual mean = scl(m_trace(sig_tr), 1.0 / 3.0);
    dmat s = m_sub(sig_tr, m_scld(m_eye(), mean));
    dual snorm = dsqrt(m_ddot(s, s));
    dual q_tr = scl(snorm, sqrt(1.5));                  /* von Mises of trial stress */
    double sy_n = orc_sigma_y(ph, xi_n, NULL);
    int plastic = (q_tr.v - sy_n) > 1e-12 * sy_n;       /* Eq. j2_2, j2_6 */

    dmat sig = sig_tr, Fpnew = Fpn;
    double xinew = xi_n;
    if (plastic) {
        /* scalar return map g(dg) = q_tr - 3 G dg - sigma_y(xi_n + dg) = 0 */
        double h0;
        orc_sigma_y(ph, xi_n, &h0);
        double x = (q_tr.v - sy_n) / (3.0 * G + h0);
        for (int it = 0; it < 60; ++it) {
            double hs, sy = orc_sigma_y(ph, xi_n + x, &hs);
            double g = q_tr.v - 3.0 * G * x - sy;
            double step = g / (3.0 * G + hs);
            x += step;
            if (fabs(step) <= 1e-15 * fabs(x)) break;
        }
        /* one dual Newton step at the root gives d(dg) (implicit function thm) */
        double hs, sy = orc_sigma_y(ph, xi_n + x, &hs);
        dual g = sub(sub(q_tr, cst(3.0 * G * x)), cst(sy));
        dual dg = add(cst(x), scl(g, 1.0 / (3.0 * G + hs)));
        dmat r = m_scl(m_scld(s, dvd(cst(1.0), snorm)), sqrt(1.5)); /* Eq. j2_3 */
        sig = m_sub(sig_tr, m_scld(r, scl(dg, 2.0 * G)));
        Fpnew = m_mul(m_exp(m_scld(r, dg)), Fpn);                  /* Eq. j2_10 */
        xinew = xi_n + dg.v;                                        /* Eq. j2_4 */
    }
    dmat Fe = m_mul(Fd, m_inv(Fpnew));
    dmat Pd = m_mul(m_mul(m_tr(m_inv(Fe)), sig), m_tr(m_inv(Fpnew)));  /* Eq. j2_9 (read) */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            if (P) P[3 * i + j] = Pd.a[i][j].v;
            if (dP) dP[3 * i + j] = Pd.a[i][j].d;
            if (Fp_new) Fp_new[3 * i + j] = Fpnew.a[i][j].v;
        }
    if (xi_new) *xi_new = xinew;
    return plastic;
}

/*
 * Material point with the full tangent.  d = 3: A[(3i+j)*9 + 3k+l] = dP_ij/dF_kl.
 * d = 2 (plane strain, F33 = 1): only the in-plane block,
 * A[(2i+j)*4 + 2k+l], P in-plane [4] and P33 separately.
 */
int orc_material(int d, const double *F3, const double *Fp_n, double xi_n, const orc_phase *ph,
                 double *P, double *A, double *P33, double *Fp_new, double *xi_new)
{
    double P3[9], dP[9], dF[9];
    int plastic = orc_material_dir(F3, NULL, Fp_n, xi_n, ph, P3, NULL, Fp_new, xi_new);
    for (int i = 0; i < d; ++i) for (int j = 0; j < d; ++j) P[d * i + j] = P3[3 * i + j];
    if (P33) *P33 = P3[8];
    if (A) {
        for (int k = 0; k < d; ++k)
            for (int l = 0; l < d; ++l) {
                memset(dF, 0, sizeof dF);
                dF[3 * k + l] = 1.0;
                orc_material_dir(F3, dF, Fp_n, xi_n, ph, NULL, dP, NULL, NULL);
                for (int i = 0; i < d; ++i)
                    for (int j = 0; j < d; ++j)
                        A[(d * i + j) * d * d + d * k + l] = dP[3 * i + j];
            }
    }
    return plastic;
}
