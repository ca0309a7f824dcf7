/*
 * ORACLE — test infrastructure only (tests, smoke() and the CPU-baseline leg
 * of bench.py).  Plain FP64 CPU reference of the paper's method; shares no
 * code, header or constant with the CUDA path.
 */
#ifndef ORC_H
#define ORC_H

enum { ORC_HARD_LINEAR = 0, ORC_HARD_POWER = 1 };

/* Material phase.  linear: sigma_y = s0 + H*xi ; power: sigma_y = s0*(1+k*xi)^p.
 * s0 = +inf makes the phase purely elastic. */
typedef struct {
    double E, nu;
    int hard_law;
    double s0, H_or_k, p;
} orc_phase;

double orc_sigma_y(const orc_phase *ph, double xi, double *slope);
int orc_material_dir(const double *F, const double *dF, const double *Fp_n, double xi_n,
                     const orc_phase *ph, double *P, double *dP, double *Fp_new, double *xi_new);
int orc_material(int d, const double *F3, const double *Fp_n, double xi_n, const orc_phase *ph,
                 double *P, double *A, double *P33, double *Fp_new, double *xi_new);

#endif
