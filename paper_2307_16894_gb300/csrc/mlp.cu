// Learned Newton start: a small MLP that predicts the correction of the previous-step
// increment of the reduced coordinates, da_k - da_{k-1}, from (dUbar, mu, a_n, da_{k-1},
// mean xi, max xi).  Not part of
// the paper (which is silent on the Newton predictor); the converged Newton answer
// does not depend on it.  Hand-written kernels for inference (BF16 weights, FP32
// accumulation, exact-erf GELU) and for training (forward, backward, MSE loss,
// Adam on an FP32 master copy).
//
// Parameter packing (FP32 master copy, also the host format): for layer l = 0 .. L-1
// (L = depth + 1 linear maps: n_in -> width -> ... -> width -> n_out) the weight
// W_l[out_l][in_l] row-major, then the bias b_l[out_l].
#include <cuda_bf16.h>
#include <cstdint>
#include <cmath>

#include "kernels.cuh"
#include "tcgen05.cuh"

namespace podecm {



static __host__ __device__ inline int layer_in(const MlpDev &M, int l) { return l == 0 ? M.n_in : M.width; }
static __host__ __device__ inline int layer_out(const MlpDev &M, int l) { return l == M.L - 1 ? M.n_out : M.width; }
static inline int64_t layer_off(const MlpDev &M, int l) {
    int64_t o = 0;
    for (int k = 0; k < l; ++k) o += (int64_t)layer_out(M, k) * layer_in(M, k) + layer_out(M, k);
    return o;
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

template <typename T>
__device__ __forceinline__ float ldf(const T *p) { return float(*p); }
template <>
__device__ __forceinline__ float ldf<__nv_bfloat16>(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

// C[i][j] (+)= sum_k A(i,k) B(k,j); A(i,k) = TA ? A[k*lda+i] : A[i*lda+k]; B(k,j) = TB ? B[j*ldb+k] : B[k*ldb+j]
template <bool TA, bool TB, typename TBt>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float *__restrict__ A, int lda,
                                              const TBt *__restrict__ B, int ldb, float *__restrict__ C, int ldc,
                                              int accumulate) {
    __shared__ float As[16][64 + 1];
    __shared__ float Bs[16][64 + 1];
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
    float acc[4][4] = {{0}};
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int kk = e / 64, r = e % 64;
            const int i = i0 + r, k = k0 + kk, j = j0 + r;
            As[kk][r] = (i < M && k < K) ? (TA ? A[(int64_t)k * lda + i] : A[(int64_t)i * lda + k]) : 0.f;
            Bs[kk][r] = (j < N && k < K) ? (TB ? ldf(B + (int64_t)j * ldb + k) : ldf(B + (int64_t)k * ldb + j)) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) { a[x] = As[kk][ty * 4 + x]; b[x] = Bs[kk][tx * 4 + x]; }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(a[x], b[y], acc[x][y]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) {
            const int i = i0 + ty * 4 + x, j = j0 + tx * 4 + y;
            if (i < M && j < N) {
                float *c = C + (int64_t)i * ldc + j;
                *c = accumulate ? *c + acc[x][y] : acc[x][y];
            }
        }
}

template <bool TA, bool TB, typename TBt>
static void gemm(int M, int N, int K, const float *A, int lda, const TBt *B, int ldb, float *C, int ldc, int acc,
                 cudaStream_t s) {
    dim3 grid((N + 63) / 64, (M + 63) / 64);
    k_gemm<TA, TB, TBt><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, acc);
}

// Z[i][j] += b[j]; H = gelu(Z) (or H = Z for the output layer)
template <typename TBt>
__global__ void k_bias_act(int N, int C, float *Z, int ldz, const TBt *b, float *H, int ldh, int act) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)N * C) return;
    const int i = (int)(e / C), j = (int)(e % C);
    const float z = Z[(int64_t)i * ldz + j] + ldf(b + j);
    Z[(int64_t)i * ldz + j] = z;
    H[(int64_t)i * ldh + j] = act ? gelu(z) : z;
}

// standardise inputs: H0 = (x - mean)/std
__global__ void k_norm_in(int N, int C, const float *X, const float *mean, const float *std_, float *H, int ldh) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)N * C) return;
    const int i = (int)(e / C), j = (int)(e % C);
    H[(int64_t)i * ldh + j] = (X[e] - mean[j]) / std_[j];
}

// MSE on standardised targets: loss = mean((out - (y - ym)/ys)^2); dOut = 2 (out - t) / (N C)
__global__ void k_mse(int N, int C, const float *out, int ldo, const float *Y, const float *ym, const float *ys,
                      float *dout, int ldd, float *loss) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.f;
    if (e < (int64_t)N * C) {
        const int i = (int)(e / C), j = (int)(e % C);
        const float t = (Y[e] - ym[j]) / ys[j];
        const float r = out[(int64_t)i * ldo + j] - t;
        dout[(int64_t)i * ldd + j] = 2.f * r / (float)((int64_t)N * C);
        l = r * r;
    }
    for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
    if ((threadIdx.x & 31) == 0 && l != 0.f) atomicAdd(loss, l / (float)((int64_t)N * C));
}

// dZ = dH * gelu'(Z) (in place on dH)
__global__ void k_gelu_back(int N, int C, const float *Z, int ldz, float *dH, int ldd) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)N * C) return;
    const int i = (int)(e / C), j = (int)(e % C);
    dH[(int64_t)i * ldd + j] *= gelu_grad(Z[(int64_t)i * ldz + j]);
}

// db[j] = sum_i dZ[i][j]
__global__ void k_colsum(int N, int C, const float *dZ, int ldd, float *db) {
    const int j = blockIdx.x;
    float s = 0.f;
    for (int i = threadIdx.x; i < N; i += blockDim.x) s += dZ[(int64_t)i * ldd + j];
    __shared__ float red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[j] = red[0];
}

__global__ void k_adam(int64_t n, float *p, float *m, float *v, const float *g, __nv_bfloat16 *p16, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.f - b1) * gg;
    const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    const float pn = p[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    p[e] = pn;
    p16[e] = __float2bfloat16(pn);
}

__global__ void k_to_bf16(int64_t n, const float *p, __nv_bfloat16 *q) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) q[e] = __float2bfloat16(p[e]);
}

static inline int nb(int64_t n, int b = 256) { return (int)((n + b - 1) / b); }

// forward pass of N rows of X (raw features); leaves pre-activations in Z and activations
// in H; output (standardised) in H[L].  bf16 = 1: BF16 weights (inference precision).
static void forward(const MlpDev &M, const float *X, int64_t N, int bf16, cudaStream_t s) {
    const int64_t cap = M.cap, w = M.wmax;
    k_norm_in<<<nb(N * M.n_in), 256, 0, s>>>((int)N, M.n_in, X, M.norm, M.norm + M.n_in, M.H, (int)w);
    for (int l = 0; l < M.L; ++l) {
        const int in = layer_in(M, l), out = layer_out(M, l);
        const int64_t off = layer_off(M, l);
        float *Hin = M.H + (int64_t)l * cap * w, *Hout = M.H + (int64_t)(l + 1) * cap * w;
        float *Z = M.Z + (int64_t)l * cap * w;
        if (bf16) gemm<false, true, __nv_bfloat16>((int)N, out, in, Hin, (int)w, reinterpret_cast<__nv_bfloat16 *>(M.p16) + off, in, Z, (int)w, 0, s);
        else gemm<false, true, float>((int)N, out, in, Hin, (int)w, M.p32 + off, in, Z, (int)w, 0, s);
        const int act = l < M.L - 1;
        if (bf16) k_bias_act<<<nb(N * out), 256, 0, s>>>((int)N, out, Z, (int)w, reinterpret_cast<__nv_bfloat16 *>(M.p16) + off + (int64_t)out * in, Hout, (int)w, act);
        else k_bias_act<<<nb(N * out), 256, 0, s>>>((int)N, out, Z, (int)w, M.p32 + off + (int64_t)out * in, Hout, (int)w, act);
    }
}

// loss and gradient (into M.grad) of N rows; returns via M.loss[0]
static void backward(const MlpDev &M, const float *X, const float *Y, int64_t N, int bf16, cudaStream_t s) {
    const int64_t cap = M.cap, w = M.wmax;
    forward(M, X, N, bf16, s);
    cudaMemsetAsync(M.loss, 0, sizeof(float), s);
    float *dA = M.dH, *dB = M.dH + cap * w;
    k_mse<<<nb(N * M.n_out), 256, 0, s>>>((int)N, M.n_out, M.H + (int64_t)M.L * cap * w, (int)w, Y,
                                          M.norm + 2 * M.n_in, M.norm + 2 * M.n_in + M.n_out, dA, (int)w, M.loss);
    for (int l = M.L - 1; l >= 0; --l) {
        const int in = layer_in(M, l), out = layer_out(M, l);
        const int64_t off = layer_off(M, l);
        if (l < M.L - 1) k_gelu_back<<<nb(N * out), 256, 0, s>>>((int)N, out, M.Z + (int64_t)l * cap * w, (int)w, dA, (int)w);
        // dW[out][in] = dZ^T H_in ; db = colsum(dZ)
        gemm<true, false, float>(out, in, (int)N, dA, (int)w, M.H + (int64_t)l * cap * w, (int)w, M.grad + off, in, 0, s);
        k_colsum<<<out, 256, 0, s>>>((int)N, out, dA, (int)w, M.grad + off + (int64_t)out * in);
        if (l > 0) {
            // dH_in[N][in] = dZ[N][out] W[out][in]
            if (bf16) gemm<false, false, __nv_bfloat16>((int)N, in, out, dA, (int)w, reinterpret_cast<__nv_bfloat16 *>(M.p16) + off, in, dB, (int)w, 0, s);
            else gemm<false, false, float>((int)N, in, out, dA, (int)w, M.p32 + off, in, dB, (int)w, 0, s);
            float *t = dA; dA = dB; dB = t;
        }
    }
}

int mlp_alloc(MlpDev &M, int n_in, int width, int depth, int n_out, int64_t cap) {
    M.n_in = n_in; M.width = width; M.depth = depth; M.n_out = n_out; M.L = depth + 1;
    M.nparams = layer_off(M, M.L);
    M.cap = cap;
    M.wmax = width > n_in ? width : n_in;
    if (n_out > M.wmax) M.wmax = n_out;
    const int64_t w = M.wmax;
    if (cudaMalloc(&M.p32, M.nparams * 4) || cudaMalloc(&M.m, M.nparams * 4) || cudaMalloc(&M.v, M.nparams * 4) ||
        cudaMalloc(&M.grad, M.nparams * 4) || cudaMalloc((void **)&M.p16, M.nparams * 2) ||
        cudaMalloc(&M.norm, (2 * n_in + 2 * n_out) * 4) || cudaMalloc(&M.Z, (int64_t)M.L * cap * w * 4) ||
        cudaMalloc(&M.H, (int64_t)(M.L + 1) * cap * w * 4) || cudaMalloc(&M.dH, 2 * cap * w * 4) ||
        cudaMalloc(&M.loss, 16))
        return -1;
    cudaMemset(M.m, 0, M.nparams * 4);
    cudaMemset(M.v, 0, M.nparams * 4);
    return 0;
}

void mlp_free(MlpDev &M) {
    float *ps[] = {M.p32, M.m, M.v, M.grad, M.norm, M.Z, M.H, M.dH, M.loss};
    for (float *p : ps) if (p) cudaFree(p);
    if (M.p16) cudaFree(M.p16);
    M = MlpDev{};
}

int64_t mlp_nparams(const MlpDev &M) { return M.nparams; }

void mlp_set_params(MlpDev &M, const float *host, cudaStream_t s) {
    cudaMemcpyAsync(M.p32, host, M.nparams * 4, cudaMemcpyHostToDevice, s);
    k_to_bf16<<<nb(M.nparams), 256, 0, s>>>(M.nparams, M.p32, reinterpret_cast<__nv_bfloat16 *>(M.p16));
    cudaMemsetAsync(M.m, 0, M.nparams * 4, s);
    cudaMemsetAsync(M.v, 0, M.nparams * 4, s);
}

void mlp_get_params(const MlpDev &M, float *host, cudaStream_t s) {
    cudaMemcpyAsync(host, M.p32, M.nparams * 4, cudaMemcpyDeviceToHost, s);
}

void mlp_set_norm(MlpDev &M, const float *host, cudaStream_t s) {
    cudaMemcpyAsync(M.norm, host, (2 * M.n_in + 2 * M.n_out) * 4, cudaMemcpyHostToDevice, s);
}

// one Adam step on the mini-batch (X, Y) (device, raw features / raw targets)
void mlp_train_step(MlpDev &M, const float *X, const float *Y, int64_t N, float lr, int t, float *loss_out,
                    cudaStream_t s) {
    backward(M, X, Y, N, 1, s);
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    k_adam<<<nb(M.nparams), 256, 0, s>>>(M.nparams, M.p32, M.m, M.v, M.grad, reinterpret_cast<__nv_bfloat16 *>(M.p16), lr, b1, b2, 1e-8f, c1, c2);
    if (loss_out) cudaMemcpyAsync(loss_out, M.loss, 4, cudaMemcpyDeviceToDevice, s);
}

// loss and gradient without update (bf16 = 0: FP32 weights) -> grad_out [nparams], loss_out [1] (device)
void mlp_loss_grad(MlpDev &M, const float *X, const float *Y, int64_t N, int bf16, float *grad_out, float *loss_out,
                   cudaStream_t s) {
    backward(M, X, Y, N, bf16, s);
    cudaMemcpyAsync(grad_out, M.grad, M.nparams * 4, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(loss_out, M.loss, 4, cudaMemcpyDeviceToDevice, s);
}

// de-standardise the output rows into double predictions: out[i][j] = H[L][i][j] * ys + ym
__global__ void k_out(int N, int C, const float *H, int ldh, const float *ym, const float *ys, double *out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)N * C) return;
    const int i = (int)(e / C), j = (int)(e % C);
    out[e] = (double)(H[(int64_t)i * ldh + j] * ys[j] + ym[j]);
}


// ---------------------------------------------------------------- fused inference (tcgen05)
// The whole network for 128 rows per CTA on the tensor cores: the standardised input, rounded
// to BF16, is the A operand (128 rows x K, canonical K-major layout in shared memory); each
// layer's BF16 weight matrix W_l[out][in] is the B operand (rows = out, K = in), placed in
// shared memory in the same layout by the CTA itself; one thread issues the layer's
// tcgen05.mma (kind::f16, M = 128, N = out, K = 16 each) into a 128 x 128 FP32 tensor-memory
// accumulator; the epilogue (thread = row = tensor-memory lane) adds the bias, applies the
// exact-erf GELU and writes the BF16 activations back as the next layer's A operand; the last
// layer adds the bias and undoes the output standardisation.  Same parameters and arithmetic as
// the CUDA-core path, except that the activations between layers are rounded to BF16 (the
// operand type of the MMA).  A bounded wait that gives up writes zero predictions (the
// previous-step predictor) for the CTA's rows and sets the error flag.
namespace mlptc {
constexpr int ROWS = 128;
constexpr int THREADS = 128;
constexpr int MAXL = 8;
struct Geo {
    int L, n_in, n_out, kp0, nout_p;   // layers, sizes, padded input width and output width
    int w_off[MAXL];                   // byte offset of layer l's B image in shared memory
    int a_off, smem;                   // A tile offset, dynamic shared memory
    int64_t p_off[MAXL];               // element offset of layer l in the parameter vector
};
__host__ __device__ inline int l_in(const Geo &g, int l) { return l == 0 ? g.n_in : 128; }
__host__ __device__ inline int l_out(const Geo &g, int l) { return l == g.L - 1 ? g.n_out : 128; }
__host__ __device__ inline int l_kp(const Geo &g, int l) { return l == 0 ? g.kp0 : 128; }
__host__ __device__ inline int l_np(const Geo &g, int l) { return l == g.L - 1 ? g.nout_p : 128; }
// byte offset of element (row r, k) of a BF16 canonical K-major tile whose rows hold kp elements
__host__ __device__ inline int off(int r, int k, int kp) {
    return (r >> 3) * (kp / 8 * 128) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}
}  // namespace mlptc

__global__ void __launch_bounds__(mlptc::THREADS, 1)
    k_mlp_tc(mlptc::Geo g, const __nv_bfloat16 *__restrict__ p16, const float *__restrict__ norm,
             const float *__restrict__ X, int64_t N, double *__restrict__ out, int *err_flag) {
    using namespace tcx;
    using namespace mlptc;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_s;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * ROWS;
    const int kpa = g.kp0 > 128 ? g.kp0 : 128;     // K capacity of the A tile
    unsigned char *A = smem + g.a_off;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(128));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_s = 0;
    }
    // zero the shared memory (padding rows and K slots of every tile), then fill
    for (int e = tid; e < g.smem / 16; e += THREADS) reinterpret_cast<uint4 *>(smem)[e] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    for (int l = 0; l < g.L; ++l) {
        const int in = l_in(g, l), outl = l_out(g, l), kp = l_kp(g, l);
        const __nv_bfloat16 *W = p16 + g.p_off[l];
        unsigned char *img = smem + g.w_off[l];
        if (l > 0) {
            // rows of 128 inputs, 16-byte aligned: 8 weights per copy
            for (int e = tid; e < outl * 16; e += THREADS) {
                const int o = e >> 4, k = (e & 15) * 8;
                *reinterpret_cast<uint4 *>(img + off(o, k, kp)) = *reinterpret_cast<const uint4 *>(W + (int64_t)o * in + k);
            }
        } else {
            for (int e = tid; e < outl * in; e += THREADS) {
                const int o = e / in, k = e - o * in;
                *reinterpret_cast<__nv_bfloat16 *>(img + off(o, k, kp)) = W[e];
            }
        }
    }
    // standardised input rows, rounded to BF16
    const float *mean = norm, *sd = norm + g.n_in;
    for (int e = tid; e < ROWS * g.n_in; e += THREADS) {
        const int r = e / g.n_in, k = e - r * g.n_in;
        if (r0 + r < N) {
            const float v = (X[(r0 + r) * g.n_in + k] - mean[k]) / sd[k];
            *reinterpret_cast<__nv_bfloat16 *>(A + off(r, k, kpa)) = __float2bfloat16(v);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    const int64_t row = r0 + tid;
    for (int l = 0; l < g.L; ++l) {
        const int kp = l_kp(g, l), np = l_np(g, l), outl = l_out(g, l);
        if (tid == 0) {
            const uint32_t idesc = make_idesc(1u, ROWS, np);
            const uint32_t a0 = smem_u32(A), b0 = smem_u32(smem + g.w_off[l]);
            for (int k = 0; k < kp / 16; ++k)
                mma_f16(tmem, make_desc(a0 + k * 256, 128, kpa / 8 * 128), make_desc(b0 + k * 256, 128, kp / 8 * 128),
                        idesc, k > 0 ? 1u : 0u);
            mma_commit(&bar);
        }
        __syncwarp();
        if (!mbar_wait(&bar, (uint32_t)(l & 1), &abort_s)) abort_s = 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
        if (abort_s) break;
        const __nv_bfloat16 *bias = p16 + g.p_off[l] + (int64_t)outl * l_in(g, l);
        const bool last = l == g.L - 1;
        for (int c0 = 0; c0 < np; c0 += 16) {
            uint32_t r[16];
            tmem_ld16(tmem + lane_base + (uint32_t)c0, r);
            tmem_wait_ld();
            if (!last) {
                uint32_t pk[8];
#pragma unroll
                for (int q = 0; q < 16; q += 2) {
                    const float z0 = __uint_as_float(r[q]) + __bfloat162float(bias[c0 + q]);
                    const float z1 = __uint_as_float(r[q + 1]) + __bfloat162float(bias[c0 + q + 1]);
                    pk[q / 2] = pack_bf16(gelu(z0), gelu(z1));
                }
                // row tid, inputs c0 .. c0 + 15 of the next layer: two 16-byte core-matrix rows
                *reinterpret_cast<uint4 *>(A + off(tid, c0, kpa)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                *reinterpret_cast<uint4 *>(A + off(tid, c0 + 8, kpa)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            } else if (row < N) {
                const float *ym = norm + 2 * g.n_in, *ys = ym + g.n_out;
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int j = c0 + q;
                    if (j < g.n_out) {
                        const float z = __uint_as_float(r[q]) + __bfloat162float(bias[j]);
                        out[row * g.n_out + j] = (double)(z * ys[j] + ym[j]);
                    }
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (abort_s) {
        // the previous-step predictor for these rows; a committed MMA may still be in flight
        if (tid == 0) mbar_drain(&bar, 0u), mbar_drain(&bar, 1u);
        if (row < N)
            for (int j = 0; j < g.n_out; ++j) out[row * g.n_out + j] = 0.0;
        if (tid == 0 && err_flag) atomicExch(err_flag, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
    }
}

// the fused kernel's geometry, or false when the network does not fit it (width 128, n_in and
// n_out at most 256 and 128, the whole network in shared memory)
static bool mlp_tc_geo(const MlpDev &M, mlptc::Geo &g) {
    using namespace mlptc;
    if (M.width != 128 || M.L > MAXL || M.n_in > 256 || M.n_out > 128 || M.n_in < 1 || M.n_out < 1) return false;
    g.L = M.L; g.n_in = M.n_in; g.n_out = M.n_out;
    g.kp0 = (M.n_in + 15) / 16 * 16;
    g.nout_p = (M.n_out + 15) / 16 * 16;
    int o = 0;
    for (int l = 0; l < g.L; ++l) {
        g.w_off[l] = o;
        g.p_off[l] = layer_off(M, l);
        o += l_np(g, l) * l_kp(g, l) * 2;
        o = (o + 1023) / 1024 * 1024;
    }
    g.a_off = o;
    o += ROWS * (g.kp0 > 128 ? g.kp0 : 128) * 2;
    g.smem = o;
    return g.smem <= 227 * 1024;
}

// predictions for N rows of raw features X: with BF16 weights on the tensor cores (k_mlp_tc)
// when the network fits it, otherwise on the CUDA cores in chunks of the work capacity
void mlp_predict(MlpDev &M, const float *X, int64_t N, int bf16, double *out, cudaStream_t s, int *err) {
    mlptc::Geo g;
    if (bf16 && mlp_tc_geo(M, g)) {
        cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, g.smem);
        k_mlp_tc<<<(unsigned)((N + mlptc::ROWS - 1) / mlptc::ROWS), mlptc::THREADS, g.smem, s>>>(
            g, reinterpret_cast<const __nv_bfloat16 *>(M.p16), M.norm, X, N, out, err);
        return;
    }
    for (int64_t r0 = 0; r0 < N; r0 += M.cap) {
        const int64_t nr = (N - r0) < M.cap ? (N - r0) : M.cap;
        forward(M, X + r0 * M.n_in, nr, bf16, s);
        k_out<<<nb(nr * M.n_out), 256, 0, s>>>((int)nr, M.n_out, M.H + (int64_t)M.L * M.cap * M.wmax, M.wmax,
                                               M.norm + 2 * M.n_in, M.norm + 2 * M.n_in + M.n_out, out + r0 * M.n_out);
    }
}

// ---------------------------------------------------------------- features
// x = [Ubar_k - Ubar_{k-1} (d2), mu (n_par), a_n (n), a_n - a_{n-1} (n), mean xi, max xi] per instance.
// Ubar_k is the stretch of the polar split of Fbar (computed by k_start); U_prev is
// the stretch of the last converged step of the instance.
__global__ void k_features(Model M, Batch Bt, const double *__restrict__ U_prev, float *__restrict__ X, int n_in) {
    const int64_t b = blockIdx.x;
    const int d2 = M.d2, n = M.n, m = M.m, tid = threadIdx.x;
    __shared__ double s_sum[128], s_max[128];
    double sm = 0.0, mx = 0.0;
    for (int i = tid; i < m; i += blockDim.x) {
        const double x = Bt.xi[b * m + i];
        sm += x;
        mx = fmax(mx, x);
    }
    s_sum[tid] = sm;
    s_max[tid] = mx;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (tid < off) { s_sum[tid] += s_sum[tid + off]; s_max[tid] = fmax(s_max[tid], s_max[tid + off]); }
        __syncthreads();
    }
    float *x = X + b * n_in;
    for (int c = tid; c < d2; c += blockDim.x) x[c] = (float)(Bt.Ubar[b * d2 + c] - U_prev[b * d2 + c]);
    for (int k = tid; k < M.n_par; k += blockDim.x) x[d2 + k] = (float)Bt.mu[b * M.n_par + k];
    for (int j = tid; j < n; j += blockDim.x) {
        x[d2 + M.n_par + j] = (float)Bt.q_n[b * n + j];
        x[d2 + M.n_par + n + j] = (float)Bt.dq_prev[b * n + j];
    }
    if (tid == 0) {
        x[d2 + M.n_par + 2 * n] = (float)(s_sum[0] / m);
        x[d2 + M.n_par + 2 * n + 1] = (float)s_max[0];
    }
}

void launch_features(const Model &M, Batch Bt, const double *U_prev, float *X, int n_in, cudaStream_t s) {
    k_features<<<(int)Bt.B, 128, 0, s>>>(M, Bt, U_prev, X, n_in);
}

}  // namespace podecm
