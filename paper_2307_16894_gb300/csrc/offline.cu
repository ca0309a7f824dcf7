// Offline stage on the device (the offline stage of Algorithm 1; Sec. 3.1-3.2):
//  * POD by the method of snapshots (Eq. pod_disp and the orthonormality relation after it):
//    C = S^T M S (M the V^p Gram operator, sparse; or a diagonal weight for the L^2 POD of the
//    weighted stress), C = V Lambda V^T, phi_j = S v_j / sqrt(lambda_j);
//  * the empirical cubature greedy (Sec. 3.2, Eq. integral_ecm): an orthonormal basis Z of the
//    integrand space (from the eigenpairs of its weighted Gram matrix), the candidate most
//    aligned with the integration residual, and the positive least-squares weights refit with
//    rank-one updates of a Cholesky factor of the normal matrix (the remark of Sec. 3.2 on the
//    cost of ECM), with an active-set (Lawson-Hanson) pass whenever a weight is not positive.
// Arithmetic: FP64 throughout.  The POD spectrum of the snapshot sets spans up to 14 decades
// (lambda_n / lambda_1 ~ 1e-14 for the 3D family), so the Gram products run on the FP64 pipe;
// a TF32 or BF16 Gram would leave every mode beyond the fourth decade in rounding noise.
#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

namespace podecm {

// ------------------------------------------------------------------ Gram products
// C[a][b] += sum_{x in this CTA's K range} A[a][x] w[x] B[b][x]   (A [na][K], B [nb][K] row-major,
// w optional).  16 x 16 outputs per CTA, K split over gridDim.z, accumulated with FP64 atomics.
constexpr int GT = 16, GK = 64;

__global__ void k_gram(int na, int nb, int64_t K, const double *__restrict__ A, const double *__restrict__ B,
                       const double *__restrict__ w, double *__restrict__ C, int64_t kchunk) {
    __shared__ double As[GT][GK + 1], Bs[GT][GK + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;          // 16 x 16 threads
    const int a0 = blockIdx.y * GT, b0 = blockIdx.x * GT;
    const int64_t k_begin = (int64_t)blockIdx.z * kchunk, k_end = min(K, k_begin + kchunk);
    double acc = 0.0;
    const int tid = ty * GT + tx;
    for (int64_t k0 = k_begin; k0 < k_end; k0 += GK) {
        for (int e = tid; e < GT * GK; e += GT * GT) {
            const int r = e / GK, c = e - r * GK;
            const int64_t k = k0 + c;
            const bool in = k < k_end;
            const double wk = (in && w) ? w[k] : 1.0;
            As[r][c] = (in && a0 + r < na) ? A[(size_t)(a0 + r) * K + k] * wk : 0.0;
            Bs[r][c] = (in && b0 + r < nb) ? B[(size_t)(b0 + r) * K + k] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int c = 0; c < GK; ++c) acc = fma(As[ty][c], Bs[tx][c], acc);
        __syncthreads();
    }
    if (a0 + ty < na && b0 + tx < nb) atomicAdd(&C[(size_t)(a0 + ty) * nb + b0 + tx], acc);
}

// Y[a][row] = sum_j M[row][col_j] X[a][col_j]  (CSR operator applied to every snapshot)
__global__ void k_spmm_csr(int64_t N, int ns, const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                           const double *__restrict__ val, const double *__restrict__ X, double *__restrict__ Y) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y;
    if (row >= N || a >= ns) return;
    double s = 0.0;
    for (int32_t e = rowptr[row]; e < rowptr[row + 1]; ++e) s = fma(val[e], X[(size_t)a * N + col[e]], s);
    Y[(size_t)a * N + row] = s;
}

// ------------------------------------------------------------------ symmetric eigenproblem
// Cyclic parallel Jacobi (round-robin pairing; every round rotates ns/2 disjoint pairs at once:
// C <- J^T C J, V <- V J) in one CTA; C and V in global scratch (L2-resident for ns <= 1024).
// Stops when the off-diagonal Frobenius norm is <= tol * ||C||_F or after max_sweeps.  On exit
// lam holds the eigenvalues in descending order and V's columns are ordered to match.
constexpr int JT = 1024;

__device__ void block_sum2(double v, double *red, double *out) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) *out = t;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(JT) k_jacobi(int n, double *C, double *Vout, double *Vtmp, double *Ct,
                                               double *__restrict__ lam, int *__restrict__ perm, double tol,
                                               int max_sweeps, int *__restrict__ sweeps_out) {
    extern __shared__ double sh[];
    const int np = (n + 1) / 2;               // pairs per round (a dummy index n when n is odd)
    const int nn = 2 * np;
    double *cs = sh, *sn = sh + np;           // rotation of pair k
    int *pa = reinterpret_cast<int *>(sn + np), *pb = pa + np, *partner = pb + np;   // partner[i] for i < nn
    __shared__ double red[32], s_off, s_tot;
    const int tid = threadIdx.x;
    double *V = Vout, *W = Vtmp;              // V <- V J is written to W, then the two swap
    for (int e = tid; e < n * n; e += JT) V[e] = (e / n == e % n) ? 1.0 : 0.0;
    __syncthreads();
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int e = tid; e < n * n; e += JT) {
            const double c = C[e];
            tot += c * c;
            if (e / n != e % n) off += c * c;
        }
        block_sum2(off, red, &s_off);
        block_sum2(tot, red, &s_tot);
        if (s_off <= tol * tol * s_tot) break;
        for (int round = 0; round < nn - 1; ++round) {
            // round-robin schedule: position 0 fixed, positions 1..nn-1 rotate
            for (int k = tid; k < np; k += JT) {
                auto at = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + round) % (nn - 1); };
                int p = at(k), q = at(nn - 1 - k);
                if (p > q) { const int t = p; p = q; q = t; }
                pa[k] = p;
                pb[k] = q;
                double c = 1.0, s = 0.0;
                if (q < n) {
                    const double apq = C[(size_t)p * n + q];
                    if (apq != 0.0) {
                        const double app = C[(size_t)p * n + p], aqq = C[(size_t)q * n + q];
                        const double tau = (aqq - app) / (2.0 * apq);
                        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                    }
                }
                cs[k] = c;
                sn[k] = s;
                partner[p] = k;
                partner[q] = k;
            }
            __syncthreads();
            // rows: Ct = J^T C  (row p' = c p - s q, row q' = s p + c q)
            for (int e = tid; e < n * n; e += JT) {
                const int i = e / n, j = e - i * n;
                const int k = partner[i];
                const int p = pa[k], q = pb[k];
                const double c = cs[k], s = sn[k];
                const double vp = C[(size_t)p * n + j], vq = (q < n) ? C[(size_t)q * n + j] : 0.0;
                Ct[e] = (i == p) ? c * vp - s * vq : s * vp + c * vq;
            }
            __syncthreads();
            // columns: C = Ct J, and V = V J
            for (int e = tid; e < n * n; e += JT) {
                const int i = e / n, j = e - i * n;
                const int k = partner[j];
                const int p = pa[k], q = pb[k];
                const double c = cs[k], s = sn[k];
                const double vp = Ct[(size_t)i * n + p], vq = (q < n) ? Ct[(size_t)i * n + q] : 0.0;
                C[e] = (j == p) ? c * vp - s * vq : s * vp + c * vq;
                const double wp = V[(size_t)i * n + p], wq = (q < n) ? V[(size_t)i * n + q] : 0.0;
                W[e] = (j == p) ? c * wp - s * wq : s * wp + c * wq;
            }
            __syncthreads();
            double *t = V; V = W; W = t;
        }
    }
    // eigenvalues in descending order (stable rank sort: ties keep the lower index first)
    for (int i = tid; i < n; i += JT) {
        const double di = C[(size_t)i * n + i];
        int r = 0;
        for (int j = 0; j < n; ++j) {
            const double dj = C[(size_t)j * n + j];
            r += (dj > di) || (dj == di && j < i);
        }
        lam[r] = di;
        perm[r] = i;
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += JT) {
        const int i = e / n, r = e - i * n;
        Ct[e] = V[(size_t)i * n + perm[r]];
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += JT) Vout[e] = Ct[e];
    if (tid == 0 && sweeps_out) *sweeps_out = sweep;
}

// Phi[j][x] = scale_j * sum_a S[a][x] V[a][j]   (S [ns][N], V [ns][ns], scale_j = 1/sqrt(lam_j))
__global__ void k_combine(int64_t N, int ns, int nm, const double *__restrict__ S, const double *__restrict__ V,
                          const double *__restrict__ lam, double *__restrict__ Phi) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (x >= N || j >= nm) return;
    double s = 0.0;
    for (int a = 0; a < ns; ++a) s = fma(S[(size_t)a * N + x], V[(size_t)a * ns + j], s);
    Phi[(size_t)j * N + x] = s / sqrt(lam[j]);
}


// ------------------------------------------------------------------ rank-revealing Cholesky
// Pivoted lower Cholesky of the symmetric positive semi-definite n x n matrix G (in place, one
// CTA): at step j the largest remaining diagonal entry is moved to position j; the factorisation
// stops (rank = j) when that entry is <= rel * the first pivot.  perm[j] = original row of
// position j; on exit the leading rank columns of G hold L (rows in pivot order).
__global__ void __launch_bounds__(1024) k_pchol(int n, double *G, int *perm, double rel, int *rank_out) {
    __shared__ double rv[32], s_first;
    __shared__ int ri[32], s_p, s_stop;
    const int tid = threadIdx.x;
    for (int i = tid; i < n; i += blockDim.x) perm[i] = i;
    __syncthreads();
    int j = 0;
    for (; j < n; ++j) {
        double bv = -1.0;
        int bi = n;
        for (int i = j + tid; i < n; i += blockDim.x) {
            const double d = G[(size_t)i * n + i];
            if (d > bv || (d == bv && i < bi)) { bv = d; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
        }
        if ((tid & 31) == 0) { rv[tid >> 5] = bv; ri[tid >> 5] = bi; }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (rv[w] > rv[0] || (rv[w] == rv[0] && ri[w] < ri[0])) { rv[0] = rv[w]; ri[0] = ri[w]; }
            if (j == 0) s_first = rv[0];
            s_stop = !(rv[0] > rel * s_first) || !(rv[0] > 0.0);
            s_p = ri[0];
        }
        __syncthreads();
        if (s_stop) break;
        const int p = s_p;
        if (p != j) {   // symmetric swap of rows and columns j, p (the full matrix is kept)
            for (int c = tid; c < n; c += blockDim.x) {
                const double t = G[(size_t)j * n + c]; G[(size_t)j * n + c] = G[(size_t)p * n + c]; G[(size_t)p * n + c] = t;
            }
            __syncthreads();
            for (int r = tid; r < n; r += blockDim.x) {
                const double t = G[(size_t)r * n + j]; G[(size_t)r * n + j] = G[(size_t)r * n + p]; G[(size_t)r * n + p] = t;
            }
            if (tid == 0) { const int t = perm[j]; perm[j] = perm[p]; perm[p] = t; }
            __syncthreads();
        }
        if (tid == 0) G[(size_t)j * n + j] = sqrt(G[(size_t)j * n + j]);
        __syncthreads();
        const double ljj = G[(size_t)j * n + j];
        for (int i = j + 1 + tid; i < n; i += blockDim.x) G[(size_t)i * n + j] /= ljj;
        __syncthreads();
        const int m = n - j - 1;
        for (int e = tid; e < m * m; e += blockDim.x) {
            const int i = j + 1 + e / m, c = j + 1 + e % m;
            G[(size_t)i * n + c] -= G[(size_t)i * n + j] * G[(size_t)c * n + j];   // full trailing block (symmetric)
        }
        __syncthreads();
    }
    if (tid == 0) *rank_out = j;
}

// Z[r][x] = (F[perm[r]][x] - sum_{l<r} L[r][l] Z[l][x]) / L[r][r] for r < k: the orthonormal
// basis L^-1 F_perm (one thread per point; L has leading dimension n)
__global__ void k_trsm_cols(int n, int k, int64_t M, const double *__restrict__ L, const int *__restrict__ perm,
                            const double *__restrict__ F, double *__restrict__ Z) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= M) return;
    for (int r = 0; r < k; ++r) {
        double s = F[(size_t)perm[r] * M + x];
        for (int l = 0; l < r; ++l) s -= L[(size_t)r * n + l] * Z[(size_t)l * M + x];
        Z[(size_t)r * M + x] = s / L[(size_t)r * n + r];
    }
}

// ------------------------------------------------------------------ empirical cubature greedy
// Zx [nr][M]: the orthonormal integrand basis (rows 0..nr-2) and the scaled volume row.
// colnorm[x] = |Zx[:, x]|; bx = Zx wq (the exact integrals); r = bx - Zx[:, sel] w.

// colnorm and the flagged (selected) points
__global__ void k_ecm_colnorm(int nr, int64_t M, const double *__restrict__ Zx, double *__restrict__ cn) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= M) return;
    double s = 0.0;
    for (int r = 0; r < nr; ++r) { const double z = Zx[(size_t)r * M + x]; s = fma(z, z, s); }
    cn[x] = sqrt(s);
}

// bx[r] = sum_x Zx[r][x] wq[x]: one CTA per row
__global__ void k_ecm_rowdot(int nr, int64_t M, const double *__restrict__ Zx, const double *__restrict__ wq,
                             double *__restrict__ bx) {
    __shared__ double red[32], out;
    const int r = blockIdx.x;
    double s = 0.0;
    for (int64_t x = threadIdx.x; x < M; x += blockDim.x) s = fma(Zx[(size_t)r * M + x], wq[x], s);
    block_sum2(s, red, &out);
    if (threadIdx.x == 0) bx[r] = out;
}

// scores c[x] = (Zx[:, x] . res) / colnorm[x] for unselected x; per CTA the maximum and its
// lowest index (ties: the lower index, as a first-maximum argmax)
struct ValIdx { double v; long long i; };
__device__ __forceinline__ ValIdx vi_max(ValIdx a, ValIdx b) {
    if (b.v > a.v || (b.v == a.v && b.i < a.i)) return b;
    return a;
}

__global__ void k_ecm_scores(int nr, int64_t M, const double *__restrict__ Zx, const double *__restrict__ cn,
                             const uint8_t *__restrict__ taken, const double *__restrict__ res, ValIdx *__restrict__ part) {
    extern __shared__ double rs[];                       // res [nr]
    __shared__ ValIdx red[32];
    for (int r = threadIdx.x; r < nr; r += blockDim.x) rs[r] = res[r];
    __syncthreads();
    ValIdx best{-INFINITY, (long long)M};
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < M; x += (int64_t)gridDim.x * blockDim.x) {
        if (taken[x]) continue;
        double s = 0.0;
        for (int r = 0; r < nr; ++r) s = fma(Zx[(size_t)r * M + x], rs[r], s);
        const ValIdx c{s / cn[x], (long long)x};
        best = vi_max(best, c);
    }
    for (int o = 16; o > 0; o >>= 1) {
        ValIdx t;
        t.v = __shfl_xor_sync(0xffffffffu, best.v, o);
        t.i = __shfl_xor_sync(0xffffffffu, best.i, o);
        best = vi_max(best, t);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        ValIdx b = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = vi_max(b, red[w]);
        part[blockIdx.x] = b;
    }
}

// ------------------------------------------------------------------ NNLS refit (one CTA)
// State of the greedy on the device.  Positions 0..n-1 are the selected points in selection
// order; position n is the candidate of the current step.  Hf is the normal matrix of the
// selected columns (A^T A), L the lower Cholesky factor of Hf over the selected set, g = A^T bx.
struct EcmState {
    int nr, cap;
    int64_t M;
    const double *Zx, *bx;
    int *n;                 // [1] selected count
    int *status;            // [1] 0 running, 1 done (target reached), 2 no candidate left, 3 stalled
    long long *idx;         // [cap] point of each position
    double *w;              // [cap] weights
    double *A;              // [cap][nr] columns of the selected points
    double *Hf;             // [cap][cap]
    double *L;              // [cap][cap]
    double *g;              // [cap]
    double *res;            // [nr] bx - A w
    uint8_t *taken;         // [M]
    double *s1, *s2, *s3;   // [cap] scratch vectors
    double *Hp;             // [cap][cap] scratch (passive-set normal matrix)
    int *pos;               // [cap] scratch (passive positions)
};

// y = L^{-1} b (L lower, leading dimension ld, order n); warp 0 computes, the CTA waits
__device__ void fwd_solve(const double *L, int ld, int n, const double *b, double *y) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int l = lane; l < j; l += 32) s = fma(L[(size_t)j * ld + l], y[l], s);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) y[j] = (b[j] - s) / L[(size_t)j * ld + j];
            __syncwarp();
        }
    }
    __syncthreads();
}

// x = L^{-T} y
__device__ void bwd_solve(const double *L, int ld, int n, const double *y, double *x) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        for (int j = n - 1; j >= 0; --j) {
            double s = 0.0;
            for (int l = j + 1 + lane; l < n; l += 32) s = fma(L[(size_t)l * ld + j], x[l], s);
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) x[j] = (y[j] - s) / L[(size_t)j * ld + j];
            __syncwarp();
        }
    }
    __syncthreads();
}

// in-place lower Cholesky of the n x n matrix A (leading dimension ld); returns false if a pivot
// is not positive (the whole CTA gets the same answer)
__device__ bool chol_inplace(double *A, int ld, int n, int *s_bad) {
    if (threadIdx.x == 0) *s_bad = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            const double d = A[(size_t)k * ld + k];
            if (!(d > 0.0)) *s_bad = 1;
            else A[(size_t)k * ld + k] = sqrt(d);
        }
        __syncthreads();
        if (*s_bad) return false;
        const double dk = A[(size_t)k * ld + k];
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[(size_t)i * ld + k] /= dk;
        __syncthreads();
        const int m = n - k - 1;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            const int i = k + 1 + e / m, j = k + 1 + e % m;
            if (j <= i) A[(size_t)i * ld + j] -= A[(size_t)i * ld + k] * A[(size_t)j * ld + k];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < n * n; e += blockDim.x)
        if (e % n > e / n) A[(size_t)(e / n) * ld + e % n] = 0.0;
    __syncthreads();
    return true;
}

// One greedy step: take the best candidate of k_ecm_scores, refit the non-negative weights of
// the selected set plus the candidate, drop points whose weight is not positive, update the
// residual.  The order of the kept points is the selection order.
__global__ void __launch_bounds__(1024) k_ecm_step(EcmState S, const ValIdx *__restrict__ part, int nparts, int target_m,
                                                   double *__restrict__ rnorm2) {
    __shared__ ValIdx red[32];
    __shared__ double dred[32], s_d2, s_tmp;
    __shared__ int s_bad, s_np, s_all, s_t;
    __shared__ long long s_i;
    const int tid = threadIdx.x, nr = S.nr, cap = S.cap;
    if (*S.status != 0) return;
    // best candidate: maximum score, lowest point index on ties
    ValIdx best{-INFINITY, (long long)S.M};
    for (int k = tid; k < nparts; k += blockDim.x) best = vi_max(best, part[k]);
    for (int o = 16; o > 0; o >>= 1) {
        ValIdx t;
        t.v = __shfl_xor_sync(0xffffffffu, best.v, o);
        t.i = __shfl_xor_sync(0xffffffffu, best.i, o);
        best = vi_max(best, t);
    }
    if ((tid & 31) == 0) red[tid >> 5] = best;
    __syncthreads();
    if (tid == 0) {
        ValIdx b = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = vi_max(b, red[w]);
        s_i = (b.v == -INFINITY || b.i >= S.M) ? -1 : b.i;
    }
    __syncthreads();
    const int n = *S.n;
    if (s_i < 0 || n + 1 > cap) {
        if (tid == 0) *S.status = s_i < 0 ? 2 : 3;
        return;
    }
    const long long i = s_i;
    double *An = S.A + (size_t)n * nr;
    for (int r = tid; r < nr; r += blockDim.x) An[r] = S.Zx[(size_t)r * S.M + i];
    if (tid == 0) S.idx[n] = i;
    __syncthreads();
    // normal-matrix row of the candidate and its right-hand side (one warp per entry)
    const int warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    for (int j = warp; j <= n + 1; j += nw) {
        const double *Aj = (j <= n) ? S.A + (size_t)j * nr : S.bx;
        double s = 0.0;
        for (int r = lane; r < nr; r += 32) s = fma(Aj[r], An[r], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            if (j <= n) { S.Hf[(size_t)n * cap + j] = s; S.Hf[(size_t)j * cap + n] = s; }
            else S.g[n] = s;
        }
    }
    __syncthreads();
    // rank-one extension of the Cholesky factor: L_n = [L 0; y^T d], y = L^-1 h, d^2 = h_nn - y.y
    fwd_solve(S.L, cap, n, S.Hf + (size_t)n * cap, S.s1);
    double part2 = 0.0;
    for (int j = tid; j < n; j += blockDim.x) part2 = fma(S.s1[j], S.s1[j], part2);
    block_sum2(part2, dred, &s_d2);
    const double hnn = S.Hf[(size_t)n * cap + n];
    const double d2 = hnn - s_d2;
    const bool appended = d2 > 1e-14 * hnn;
    if (appended) {
        for (int j = tid; j < n; j += blockDim.x) S.L[(size_t)n * cap + j] = S.s1[j];
        if (tid == 0) S.L[(size_t)n * cap + n] = sqrt(d2);
        __syncthreads();
        fwd_solve(S.L, cap, n + 1, S.g, S.s3);
        bwd_solve(S.L, cap, n + 1, S.s3, S.s2);
        if (tid == 0) s_all = 1;
        __syncthreads();
        for (int j = tid; j <= n; j += blockDim.x)
            if (!(S.s2[j] > 0.0)) s_all = 0;
        __syncthreads();
    } else {
        if (tid == 0) s_all = 0;
        __syncthreads();
    }
    int n_new;
    if (appended && s_all) {
        for (int j = tid; j <= n; j += blockDim.x) S.w[j] = S.s2[j];
        if (tid == 0) S.taken[i] = 1;
        n_new = n + 1;
        __syncthreads();
    } else {
        // Lawson-Hanson on the normal equations of the n + 1 candidates, started from the previous
        // weights (feasible) with the candidate at zero.  x = s2, passive flags in s1 (1 = passive).
        const int nc = n + 1;
        double *x = S.s2, *zp = S.s3, *pf = S.s1;
        for (int j = tid; j < nc; j += blockDim.x) { x[j] = (j < n) ? S.w[j] : 0.0; pf[j] = (j < n) ? 1.0 : 0.0; }
        __syncthreads();
        for (int outer = 0; outer < 3 * nc + 8; ++outer) {
            // gradient g - H x on the zero set; the most positive enters the passive set
            if (tid == 0) { s_t = -1; s_tmp = 0.0; }
            __syncthreads();
            for (int j = warp; j < nc; j += nw) {
                if (pf[j] != 0.0) continue;
                double s = 0.0;
                for (int l = lane; l < nc; l += 32) s = fma(S.Hf[(size_t)j * cap + l], x[l], s);
                for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (lane == 0) zp[j] = S.g[j] - s;
            }
            __syncthreads();
            if (tid == 0) {
                double gmax = 0.0;
                for (int j = 0; j < nc; ++j) gmax = fmax(gmax, fabs(S.g[j]));
                for (int j = 0; j < nc; ++j)
                    if (pf[j] == 0.0 && zp[j] > 1e-13 * gmax && (s_t < 0 || zp[j] > s_tmp)) { s_t = j; s_tmp = zp[j]; }
                if (s_t >= 0) pf[s_t] = 1.0;
            }
            __syncthreads();
            if (s_t < 0) break;
            for (int inner = 0; inner < nc + 2; ++inner) {
                // z_P = H_PP^-1 g_P
                if (tid == 0) {
                    int k = 0;
                    for (int j = 0; j < nc; ++j)
                        if (pf[j] != 0.0) S.pos[k++] = j;
                    s_np = k;
                }
                __syncthreads();
                const int np = s_np;
                for (int e = tid; e < np * np; e += blockDim.x)
                    S.Hp[(size_t)(e / np) * cap + e % np] = S.Hf[(size_t)S.pos[e / np] * cap + S.pos[e % np]];
                __syncthreads();
                const bool okc = chol_inplace(S.Hp, cap, np, &s_bad);
                if (!okc) break;
                for (int k = tid; k < np; k += blockDim.x) zp[k] = S.g[S.pos[k]];
                __syncthreads();
                fwd_solve(S.Hp, cap, np, zp, S.res);          // res is rebuilt below: use it as scratch
                bwd_solve(S.Hp, cap, np, S.res, zp);
                if (tid == 0) {
                    // all positive: accept; otherwise step to the boundary and drop the zeros
                    double alpha = 2.0;
                    int kmin = -1;
                    for (int k = 0; k < np; ++k)
                        if (!(zp[k] > 0.0)) {
                            const double xk = x[S.pos[k]];
                            const double a = xk / (xk - zp[k]);
                            if (a < alpha) { alpha = a; kmin = k; }
                        }
                    s_all = kmin < 0;
                    s_tmp = alpha;
                    s_t = kmin;
                }
                __syncthreads();
                if (s_all) {
                    if (tid == 0)
                        for (int j = 0; j < nc; ++j) x[j] = 0.0;
                    __syncthreads();
                    for (int k = tid; k < np; k += blockDim.x) x[S.pos[k]] = zp[k];
                    __syncthreads();
                    break;
                }
                if (tid == 0) {
                    const double alpha = s_tmp;
                    double xmax = 0.0;
                    for (int k = 0; k < np; ++k) {
                        const int j = S.pos[k];
                        x[j] += alpha * (zp[k] - x[j]);
                        xmax = fmax(xmax, x[j]);
                    }
                    x[S.pos[s_t]] = 0.0;                       // the variable that reached the boundary
                    for (int k = 0; k < np; ++k) {
                        const int j = S.pos[k];
                        if (x[j] <= 1e-14 * xmax) { x[j] = 0.0; pf[j] = 0.0; }
                    }
                }
                __syncthreads();
            }
        }
        // keep the positive weights, in selection order
        if (tid == 0) {
            int k = 0;
            for (int j = 0; j < nc; ++j) {
                if (x[j] > 0.0) S.pos[k++] = j;
                else S.taken[S.idx[j]] = 0;
            }
            s_np = k;
        }
        __syncthreads();
        n_new = s_np;
        // compact positions (ascending, so a row never overwrites one still to be read)
        for (int k = 0; k < n_new; ++k) {
            const int j = S.pos[k];
            if (j != k) {
                for (int r = tid; r < nr; r += blockDim.x) S.A[(size_t)k * nr + r] = S.A[(size_t)j * nr + r];
            }
            __syncthreads();
        }
        // rebuild Hf on the kept set (rows and columns compacted) through the scratch matrix
        for (int e = tid; e < n_new * n_new; e += blockDim.x)
            S.Hp[(size_t)(e / n_new) * cap + e % n_new] = S.Hf[(size_t)S.pos[e / n_new] * cap + S.pos[e % n_new]];
        __syncthreads();
        for (int e = tid; e < n_new * n_new; e += blockDim.x) {
            const size_t o = (size_t)(e / n_new) * cap + e % n_new;
            S.Hf[o] = S.Hp[o];
            S.L[o] = S.Hp[o];
        }
        if (tid == 0) {
            for (int k = 0; k < n_new; ++k) {
                const int j = S.pos[k];
                S.idx[k] = S.idx[j];
                S.w[k] = x[j];
                S.g[k] = S.g[j];
                S.taken[S.idx[k]] = 1;
            }
        }
        __syncthreads();
        if (!chol_inplace(S.L, cap, n_new, &s_bad)) {
            if (tid == 0) *S.status = 3;
            return;
        }
    }
    // residual r = bx - A w and its squared norm
    double ss = 0.0;
    for (int r = tid; r < nr; r += blockDim.x) {
        double s = S.bx[r];
        for (int j = 0; j < n_new; ++j) s -= S.A[(size_t)j * nr + r] * S.w[j];
        S.res[r] = s;
        ss = fma(s, s, ss);
    }
    block_sum2(ss, dred, &s_tmp);
    if (tid == 0) {
        *rnorm2 = s_tmp;
        *S.n = n_new;
        if (target_m > 0 && n_new >= target_m) *S.status = 1;
    }
}

}  // namespace podecm

// ------------------------------------------------------------------ host entry points
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/podecm.h"

namespace podecm {

__global__ void k_symmetrize(int n, double *C) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int i = e / n, j = e % n;
    if (j <= i) return;
    const double a = 0.5 * (C[(size_t)i * n + j] + C[(size_t)j * n + i]);
    C[(size_t)i * n + j] = a;
    C[(size_t)j * n + i] = a;
}

__global__ void k_fill(int64_t n, double *x, double v) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) x[e] = v;
}

__global__ void k_scale(int64_t n, double *x, const double *num, double factor) {
    // x *= factor / sqrt(*num)
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) x[e] *= factor / sqrt(*num);
}

namespace {
struct Scratch {
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
    ~Scratch() {
        for (void *p : ptrs) cudaFree(p);
    }
};

rom_status off_fail(char *buf, size_t len, rom_status s, const char *fmt, ...) {
    if (buf && len) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, len, fmt, ap);
        va_end(ap);
    }
    return s;
}

unsigned blocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// C = A diag(w) B^T (na x nb), symmetrised when A == B or sym
void gram(cudaStream_t s, int na, int nb, int64_t K, const double *A, const double *B, const double *w, double *C,
          bool sym) {
    cudaMemsetAsync(C, 0, (size_t)na * nb * 8, s);
    const int64_t kchunk = 4096;
    const dim3 grid(blocks(nb, GT), blocks(na, GT), (unsigned)((K + kchunk - 1) / kchunk));
    k_gram<<<grid, dim3(GT, GT), 0, s>>>(na, nb, K, A, B, w, C, kchunk);
    if (sym) k_symmetrize<<<blocks((int64_t)na * na, 256), 256, 0, s>>>(na, C);
}

// eigenpairs of the symmetric n x n matrix C (overwritten): lam descending, V [n][n] (columns)
void eig(cudaStream_t s, int n, double *C, double *V, double *W, double *Ct, double *lam, int *perm, int *sweeps) {
    const int np = (n + 1) / 2;
    const size_t shm = (size_t)np * 16 + (size_t)(4 * np) * 4;
    k_jacobi<<<1, JT, shm, s>>>(n, C, V, W, Ct, lam, perm, 1e-14, 60, sweeps);
}
}  // namespace
}  // namespace podecm

using namespace podecm;

extern "C" rom_status rom_pod(void *cuda_stream, int64_t N, int ns, const double *S, const int32_t *rowptr,
                              const int32_t *col, const double *val, const double *wdiag, int n_modes, double *Phi,
                              double *lam_out, int *sweeps_out, char *errbuf, size_t errlen) {
    if (N < 1 || ns < 1 || ns > 1024 || n_modes < 1 || n_modes > ns || !S || !Phi || !lam_out || (rowptr && (!col || !val)))
        return off_fail(errbuf, errlen, ROM_E_ARG, "rom_pod: bad arguments (1 <= n_modes <= ns <= 1024)");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    Scratch sc;
    double *C = sc.get<double>((size_t)ns * ns), *V = sc.get<double>((size_t)ns * ns);
    double *W = sc.get<double>((size_t)ns * ns), *Ct = sc.get<double>((size_t)ns * ns);
    double *lam = sc.get<double>(ns);
    int *perm = sc.get<int>(ns), *sw = sc.get<int>(1);
    double *MS = rowptr ? sc.get<double>((size_t)ns * N) : nullptr;
    if (sc.err != cudaSuccess)
        return off_fail(errbuf, errlen, sc.err == cudaErrorMemoryAllocation ? ROM_E_NOMEM : ROM_E_CUDA, "rom_pod: %s",
                        cudaGetErrorString(sc.err));
    if (rowptr) {
        k_spmm_csr<<<dim3(blocks(N, 128), ns), 128, 0, s>>>(N, ns, rowptr, col, val, S, MS);
        gram(s, ns, ns, N, S, MS, nullptr, C, true);
    } else {
        gram(s, ns, ns, N, S, S, wdiag, C, true);
    }
    eig(s, ns, C, V, W, Ct, lam, perm, sw);
    std::vector<double> hl(ns);
    int hs = 0;
    cudaError_t e = cudaMemcpyAsync(hl.data(), lam, (size_t)ns * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, sw, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return off_fail(errbuf, errlen, ROM_E_CUDA, "rom_pod: %s", cudaGetErrorString(e));
    int rank = 0;
    for (int k = 0; k < ns; ++k) rank += hl[k] > hl[0] * 1e-14;
    if (!(hl[0] > 0) || n_modes > rank)
        return off_fail(errbuf, errlen, ROM_E_ARG, "rom_pod: requested %d modes but the snapshot set has rank %d", n_modes,
                        rank);
    k_combine<<<dim3(blocks(N, 128), n_modes), 128, 0, s>>>(N, ns, n_modes, S, V, lam, Phi);
    e = cudaMemcpyAsync(lam_out, lam, (size_t)ns * 8, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return off_fail(errbuf, errlen, ROM_E_CUDA, "rom_pod: %s", cudaGetErrorString(e));
    if (sweeps_out) *sweeps_out = hs;
    return ROM_OK;
}

extern "C" rom_status rom_ecm(void *cuda_stream, int P, int64_t M, const double *F, const double *wq, int m, double tol,
                              double volume_weight, int cap, int64_t *idx_out, double *w_out, int *m_out,
                              double *err_out, int *rank_out, char *errbuf, size_t errlen) {
    if (P < 1 || P > 4096 || M < 1 || !F || !wq || !idx_out || !w_out || !m_out || (m < 1 && !(tol > 0)) ||
        (m > 0 && cap < m) || cap < 1 || !(volume_weight > 0))
        return off_fail(errbuf, errlen, ROM_E_ARG, "rom_ecm: bad arguments (1 <= P <= 4096, m >= 1 or tol > 0, cap >= m)");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    Scratch sc;
    // orthonormal basis of the integrand space: Z = L^-1 F_perm with F W F^T = P^T L L^T P
    // (rank-revealing pivoted Cholesky; directions whose remaining pivot is <= 1e-13 of the first
    // are dropped)
    double *G = sc.get<double>((size_t)P * P);
    int *perm = sc.get<int>(P), *rk = sc.get<int>(1);
    if (sc.err != cudaSuccess)
        return off_fail(errbuf, errlen, ROM_E_NOMEM, "rom_ecm: %s", cudaGetErrorString(sc.err));
    gram(s, P, P, M, F, F, wq, G, true);
    k_pchol<<<1, 1024, 0, s>>>(P, G, perm, 1e-13, rk);
    int k = 0;
    cudaError_t e = cudaMemcpyAsync(&k, rk, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return off_fail(errbuf, errlen, ROM_E_CUDA, "rom_ecm: %s", cudaGetErrorString(e));
    if (k < 1) return off_fail(errbuf, errlen, ROM_E_ARG, "rom_ecm: the integrands vanish");
    const int nr = k + 1;
    double *Zx = sc.get<double>((size_t)nr * M), *cn = sc.get<double>(M), *bx = sc.get<double>(nr);
    const int nparts = (int)std::min<int64_t>(blocks(M, 256), 1216);
    ValIdx *part = sc.get<ValIdx>(nparts);
    EcmState st{};
    st.nr = nr;
    st.cap = cap + 1;                 // one position for the candidate of a step
    st.M = M;
    st.Zx = Zx;
    st.bx = bx;
    st.n = sc.get<int>(1);
    st.status = sc.get<int>(1);
    st.idx = sc.get<long long>(st.cap);
    st.w = sc.get<double>(st.cap);
    st.A = sc.get<double>((size_t)st.cap * nr);
    st.Hf = sc.get<double>((size_t)st.cap * st.cap);
    st.L = sc.get<double>((size_t)st.cap * st.cap);
    st.Hp = sc.get<double>((size_t)st.cap * st.cap);
    st.g = sc.get<double>(st.cap);
    st.s1 = sc.get<double>(st.cap);
    st.s2 = sc.get<double>(st.cap);
    st.s3 = sc.get<double>(st.cap);
    st.pos = sc.get<int>(st.cap);
    st.res = sc.get<double>(nr);
    st.taken = sc.get<uint8_t>(M);
    double *rn2 = sc.get<double>(1);
    if (sc.err != cudaSuccess)
        return off_fail(errbuf, errlen, ROM_E_NOMEM, "rom_ecm: %s", cudaGetErrorString(sc.err));
    k_trsm_cols<<<blocks(M, 128), 128, 0, s>>>(P, k, M, G, perm, F, Zx);
    // the volume row: ones scaled by volume_weight / sqrt(|Omega|), |Omega| = sum wq
    k_fill<<<blocks(M, 256), 256, 0, s>>>(M, Zx + (size_t)k * M, 1.0);
    k_ecm_rowdot<<<nr, 256, 0, s>>>(nr, M, Zx, wq, bx);
    k_scale<<<blocks(M, 256), 256, 0, s>>>(M, Zx + (size_t)k * M, bx + k, volume_weight);
    k_scale<<<1, 1, 0, s>>>(1, bx + k, bx + k, volume_weight);   // bx_k = vol * vw / sqrt(vol)
    k_ecm_colnorm<<<blocks(M, 256), 256, 0, s>>>(nr, M, Zx, cn);
    cudaMemsetAsync(st.n, 0, 4, s);
    cudaMemsetAsync(st.status, 0, 4, s);
    cudaMemsetAsync(st.taken, 0, (size_t)M, s);
    cudaMemcpyAsync(st.res, bx, (size_t)nr * 8, cudaMemcpyDeviceToDevice, s);
    std::vector<double> hb(nr);
    e = cudaMemcpyAsync(hb.data(), bx, (size_t)nr * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return off_fail(errbuf, errlen, ROM_E_CUDA, "rom_ecm: %s", cudaGetErrorString(e));
    double nb = 0.0;
    for (double v : hb) nb += v * v;
    nb = std::sqrt(nb);
    int *hstate = nullptr;        // n, status, then the residual norm^2 as two ints
    e = cudaMallocHost((void **)&hstate, 16);
    if (e != cudaSuccess) return off_fail(errbuf, errlen, ROM_E_NOMEM, "rom_ecm: %s", cudaGetErrorString(e));
    const int64_t limit = 20 * (m > 0 ? (int64_t)m : M);
    int n_sel = 0, status = 0;
    double r2 = nb * nb;
    for (int64_t it = 0; it < limit; ++it) {
        k_ecm_scores<<<nparts, 256, (size_t)nr * 8, s>>>(nr, M, Zx, cn, st.taken, st.res, part);
        k_ecm_step<<<1, 1024, 0, s>>>(st, part, nparts, m > 0 ? m : 0, rn2);
        cudaMemcpyAsync(hstate, st.n, 4, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(hstate + 1, st.status, 4, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(hstate + 2, rn2, 8, cudaMemcpyDeviceToHost, s);
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        n_sel = hstate[0];
        status = hstate[1];
        memcpy(&r2, hstate + 2, 8);
        if (status != 0) break;
        if (m < 1 && std::sqrt(r2) <= tol * nb) break;
    }
    cudaFreeHost(hstate);
    if (e != cudaSuccess) return off_fail(errbuf, errlen, ROM_E_CUDA, "rom_ecm: %s", cudaGetErrorString(e));
    const double err = std::sqrt(r2) / nb;
    *m_out = n_sel;
    if (err_out) *err_out = err;
    if (rank_out) *rank_out = k;
    if (n_sel > cap) return off_fail(errbuf, errlen, ROM_E_ARG, "rom_ecm: more points than cap");
    std::vector<long long> hi(n_sel > 0 ? n_sel : 1);
    e = cudaMemcpyAsync(hi.data(), st.idx, (size_t)n_sel * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w_out, st.w, (size_t)n_sel * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return off_fail(errbuf, errlen, ROM_E_CUDA, "rom_ecm: %s", cudaGetErrorString(e));
    for (int j = 0; j < n_sel; ++j) idx_out[j] = hi[j];
    if (m > 0 && n_sel != m)
        return off_fail(errbuf, errlen, ROM_E_NOT_CONVERGED, "rom_ecm: greedy stalled at %d of %d points (status %d)",
                        n_sel, m, status);
    if (m < 1 && err > tol)
        return off_fail(errbuf, errlen, ROM_E_NOT_CONVERGED, "rom_ecm: greedy stalled at error %.3e > %.3e with %d points",
                        err, tol, n_sel);
    return ROM_OK;
}

// ------------------------------------------------------------------ ECM integrands
namespace podecm {
// gradPhi[q][c][i] = sum_a Phi_i[dof(a, comp)] dN[g][a][r], c = comp * d + r, q = e * ngp + g
__global__ void k_mode_gradients(int d, int ne, int nen, int ngp, int ndof, int n, const int32_t *__restrict__ edof,
                                 const double *__restrict__ dN, const double *__restrict__ Phi, double *__restrict__ gradPhi) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nq = (int64_t)ne * ngp;
    if (t >= nq * n) return;
    const int i = (int)(t / nq);
    const int64_t q = t - (int64_t)i * nq;
    const int e = (int)(q / ngp), g = (int)(q - (int64_t)e * ngp);
    const int d2 = d * d;
    for (int comp = 0; comp < d; ++comp)
        for (int r = 0; r < d; ++r) {
            double s = 0.0;
            for (int a = 0; a < nen; ++a) {
                const int32_t k = edof[(size_t)e * nen * d + a * d + comp];
                if (k >= 0) s = fma(Phi[(size_t)i * ndof + k], dN[((size_t)g * nen + a) * d + r], s);
            }
            gradPhi[((size_t)q * d2 + comp * d + r) * n + i] = s;
        }
}

// F[i * L + l][q] = sum_c gradPhi[q][c][i] B[l][q][c]  (Eq. integral_ecm: the N L products)
__global__ void k_integrands(int d2, int64_t nq, int n, int L, const double *__restrict__ gradPhi,
                             const double *__restrict__ B, double *__restrict__ F) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nq * n * L) return;
    const int row = (int)(t / nq);
    const int64_t q = t - (int64_t)row * nq;
    const int i = row / L, l = row - i * L;
    double s = 0.0;
    for (int c = 0; c < d2; ++c) s = fma(gradPhi[((size_t)q * d2 + c) * n + i], B[((size_t)l * nq + q) * d2 + c], s);
    F[t] = s;
}
}  // namespace podecm

extern "C" rom_status rom_ecm_integrands(void *cuda_stream, const rom_fe_mesh *mesh, int n, const double *Phi, int L,
                                         const double *B, double *gradPhi, double *F, char *errbuf, size_t errlen) {
    if (!mesh || !mesh->edof || !mesh->dN || n < 1 || L < 1 || !Phi || !B || !gradPhi || !F ||
        (mesh->d != 2 && mesh->d != 3) || mesh->ne < 1 || mesh->nen < 1 || mesh->ngp < 1)
        return off_fail(errbuf, errlen, ROM_E_ARG, "rom_ecm_integrands: bad arguments");
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int d = mesh->d, nd = mesh->nen * d;
    const int64_t nq = (int64_t)mesh->ne * mesh->ngp;
    Scratch sc;
    int32_t *edof = sc.get<int32_t>((size_t)mesh->ne * nd);
    double *dN = sc.get<double>((size_t)mesh->ngp * mesh->nen * d);
    if (sc.err != cudaSuccess) return off_fail(errbuf, errlen, ROM_E_NOMEM, "rom_ecm_integrands: %s", cudaGetErrorString(sc.err));
    cudaError_t e = cudaMemcpyAsync(edof, mesh->edof, (size_t)mesh->ne * nd * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dN, mesh->dN, (size_t)mesh->ngp * mesh->nen * d * 8, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return off_fail(errbuf, errlen, ROM_E_CUDA, "rom_ecm_integrands: %s", cudaGetErrorString(e));
    k_mode_gradients<<<blocks(nq * n, 128), 128, 0, s>>>(d, mesh->ne, mesh->nen, mesh->ngp, mesh->ndof, n, edof, dN, Phi,
                                                         gradPhi);
    k_integrands<<<blocks(nq * n * L, 256), 256, 0, s>>>(d * d, nq, n, L, gradPhi, B, F);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return off_fail(errbuf, errlen, ROM_E_CUDA, "rom_ecm_integrands: %s", cudaGetErrorString(e));
    return ROM_OK;
}
