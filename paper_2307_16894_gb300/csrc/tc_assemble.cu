// Reduced stiffness K_b = sum_i G_i^T At_i G_i (Eq. stiffnessmatrix_ecm) on the 5th-generation
// tensor cores (tcgen05.mma, BF16 or TF32 operands, FP32 accumulation in tensor memory).
//
// Formulation: K_b = Y_b^T G with Y_b = blockdiag_i(At_i) G (rows = (point i, component c)).
// One CTA holds two instances (b0, b1): the MMA is D[128 x 64] += A[128 x K] B[64 x K]^T with
//   A rows 0..63   = Y_b0^T (row j, column (i,c)),  A rows 64..127 = Y_b1^T,
//   B rows j       = G[:, :, j] (column (i,c)),     D rows = K_b0 rows, then K_b1 rows.
// The K dimension runs over chunks of PC cubature points (KC = PC * d^2 columns).  Per chunk:
//   * the A tile (Y^T) is produced by all threads in FP32 from the FP32 tangent At and the
//     FP32 basis copy, rounded to BF16/TF32 and stored in the canonical K-major layout;
//   * the B tile is a pre-arranged image of G (same layout) fetched with one bulk copy
//     (cp.async.bulk, the TMA engine) that completes on an mbarrier;
//   * one thread issues KC/16 (BF16) or KC/8 (TF32) tcgen05.mma and commits them to an
//     mbarrier, so the next chunk's producer work overlaps the tensor cores (2 stages).
// Shared-memory operand layout (no swizzle, K-major): 8-row x 16-byte core matrices; core
// matrices adjacent in K are 128 bytes apart (leading byte offset), 8-row groups are
// SBO = KC * esize / 16 * 128 bytes apart (stride byte offset).
// Every wait is bounded; on timeout the kernel records an error, waits (bounded) for its
// own outstanding MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cstdint>
#include <cstring>

#include "kernels.cuh"

namespace podecm {

namespace tc {

constexpr int MROWS = 128;       // MMA M (two instances x 64 rows)
constexpr int NCOLS = 64;        // MMA N (n padded to 64)
constexpr int THREADS = 256;
constexpr long long WAIT_LIMIT = 20000000;   // try_wait polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;          // descriptor version for tcgen05
    // base offset 0, LBO mode 0, layout type 0 (no swizzle)
    return d;
}

// kind::f16 / kind::tf32 instruction descriptor: D = F32, A/B formats, both K-major, N, M
__host__ __device__ constexpr uint32_t make_idesc(uint32_t ab_format, int M, int N) {
    return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t phase) {
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred P1;\n mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n selp.b32 %0, 1, 0, P1;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

template <int FMT>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    if (FMT == 1) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                tmem_d),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
    }
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// store one rounded element of the A tile (row r, column k) in the canonical layout
template <int FMT>
__device__ __forceinline__ void store_a(unsigned char *tile, int sbo, int r, int k, float v) {
    if (FMT == 1) {
        const int off = (r >> 3) * sbo + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
        *reinterpret_cast<__nv_bfloat16 *>(tile + off) = __float2bfloat16(v);
    } else {
        const int off = (r >> 3) * sbo + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
        *reinterpret_cast<float *>(tile + off) = v;   // the tensor core reads the TF32 part
    }
}

}  // namespace tc

// FMT: 1 = BF16 (PC = 16 points per chunk), 2 = TF32 (PC = 8)
template <int D, int FMT>
__global__ void __launch_bounds__(tc::THREADS, 1)
    k_assemble_tc(Model M, Batch Bt, const unsigned char *__restrict__ Gimg, int nchunks, int *err_flag) {
    using namespace tc;
    constexpr int D2 = D * D, D4 = D2 * D2;
    constexpr int PC = (FMT == 1) ? 16 : 8;
    constexpr int KC = PC * D2;
    constexpr int ES = (FMT == 1) ? 2 : 4;
    constexpr int SBO = KC * ES / 16 * 128;
    constexpr int A_BYTES = (MROWS / 8) * SBO;
    constexpr int B_BYTES = (NCOLS / 8) * SBO;
    constexpr int KSTEP = (FMT == 1) ? 16 : 8;
    constexpr int NK = KC / KSTEP;
    constexpr uint32_t IDESC = make_idesc(FMT == 1 ? 1u : 2u, MROWS, NCOLS);

    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Ast[2] = {smem, smem + A_BYTES};
    unsigned char *Bst[2] = {smem + 2 * A_BYTES, smem + 2 * A_BYTES + B_BYTES};
    float *Gs = reinterpret_cast<float *>(smem + 2 * A_BYTES + 2 * B_BYTES);          // [PC][D2][64]
    float *As = Gs + PC * D2 * NCOLS;                                                   // [2][PC][D4]
    __shared__ __align__(8) uint64_t bar_mma[2], bar_load[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_s;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int n_act = Bt.counts[0];
    const int p0 = 2 * blockIdx.x;
    if (p0 >= n_act) return;
    const bool has1 = (p0 + 1) < n_act;
    const int64_t bI[2] = {Bt.list[p0], has1 ? Bt.list[p0 + 1] : Bt.list[p0]};
    const int n = M.n, m = M.m;
    const float *At = reinterpret_cast<const float *>(Bt.At);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(NCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(&bar_mma[0], 1);
        mbar_init(&bar_mma[1], 1);
        mbar_init(&bar_load[0], 1);
        mbar_init(&bar_load[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_s = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    uint32_t ph_mma[2] = {0, 0}, ph_load[2] = {0, 0};
    int issued[2] = {0, 0};

    for (int c = 0; c < nchunks; ++c) {
        const int s = c & 1;
        if (tid == 0) {
            bool ok = true;
            if (issued[s]) { ok = mbar_wait(&bar_mma[s], ph_mma[s]); ph_mma[s] ^= 1; issued[s] = 0; }
            if (!ok) abort_s = 1;
            else bulk_load(Bst[s], Gimg + (size_t)c * B_BYTES, B_BYTES, &bar_load[s]);
        }
        __syncthreads();
        if (abort_s) break;
        // stage the FP32 basis chunk and the two instances' tangents
        const int c0 = c * PC;
        for (int e = tid; e < PC * D2 * NCOLS; e += THREADS) {
            const int j = e % NCOLS, rc = e / NCOLS;
            const int ii = rc / D2;
            const int q = rc - ii * D2;
            Gs[e] = (j < n && c0 + ii < m) ? M.G32_pt[((size_t)(c0 + ii) * D2 + q) * n + j] : 0.f;
        }
        for (int e = tid; e < 2 * PC * D4; e += THREADS) {
            const int inst = e / (PC * D4), rem = e - inst * PC * D4;
            const int ce = rem / PC, ii = rem - ce * PC;
            const bool valid = (inst == 0 || has1) && (c0 + ii < m);
            As[(inst * PC + ii) * D4 + ce] = valid ? At[((size_t)bI[inst] * D4 + ce) * M.mA + c0 + ii] : 0.f;
        }
        __syncthreads();
        // producer: A[inst*64 + j][ii*D2 + cc] = sum_e At[ii][e][cc] G[ii][e][j]
        for (int e = tid; e < 2 * PC * NCOLS; e += THREADS) {
            const int j = e % NCOLS, r2 = e / NCOLS;
            const int ii = r2 % PC, inst = r2 / PC;
            float g[D2];
#pragma unroll
            for (int q = 0; q < D2; ++q) g[q] = Gs[(ii * D2 + q) * NCOLS + j];
            const float *a = As + (inst * PC + ii) * D4;
#pragma unroll
            for (int cc = 0; cc < D2; ++cc) {
                float y = 0.f;
#pragma unroll
                for (int q = 0; q < D2; ++q) y = fmaf(a[q * D2 + cc], g[q], y);   // Y = At^T G (K, not K^T)
                tc::store_a<FMT>(Ast[s], SBO, inst * 64 + j, ii * D2 + cc, y);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            const bool ok = mbar_wait(&bar_load[s], ph_load[s]);
            ph_load[s] ^= 1;
            if (!ok) {
                abort_s = 1;
            } else {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = smem_u32(Ast[s]), b0 = smem_u32(Bst[s]);
#pragma unroll
                for (int k = 0; k < NK; ++k) {
                    const uint64_t ad = tc::make_desc(a0 + k * 256, 128, SBO);
                    const uint64_t bd = tc::make_desc(b0 + k * 256, 128, SBO);
                    tc::mma<FMT>(tmem, ad, bd, IDESC, (c > 0 || k > 0) ? 1u : 0u);
                }
                tc::mma_commit(&bar_mma[s]);
                issued[s] = 1;
            }
        }
        __syncthreads();
        if (abort_s) break;
    }
    // drain: wait for the outstanding commits (bounded)
    if (tid == 0) {
        for (int s = 0; s < 2; ++s)
            if (issued[s]) {
                if (!mbar_wait(&bar_mma[s], ph_mma[s])) abort_s = 1;
                ph_mma[s] ^= 1;
            }
        if (abort_s && err_flag) atomicExch(err_flag, 1);
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!abort_s && warp < 4) {
        // warp w reads TMEM lanes 32w .. 32w+31 = output rows; 2 x 32 columns
        const int row = warp * 32 + (tid & 31);
        const int inst = row >> 6, j = row & 63;
        float v[64];
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(half * 32);
            uint32_t r[32];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 32; ++q) v[half * 32 + q] = __uint_as_float(r[q]);
        }
        if (j < n && (inst == 0 || has1)) {
            double *Kb = Bt.K + (size_t)bI[inst] * n * n + (size_t)j * n;
            for (int k = 0; k < n; ++k) Kb[k] = (double)v[k];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
}

// force f = sum_i G_i^T v_i in FP64, one CTA per instance; the rows (point, component) are
// split over thread groups in a fixed pattern and the group sums added in a fixed order
__global__ void __launch_bounds__(256) k_force(Model M, Batch Bt) {
    __shared__ double fr[256];
    const int n_act = Bt.counts[0];
    const int p = blockIdx.x;
    if (p >= n_act) return;
    const int64_t b = Bt.list[p];
    const int n = M.n, m = M.m, d2 = M.d2, tid = threadIdx.x;
    const int FG = blockDim.x / n, g = tid / n, j = tid - (tid / n) * n;
    double acc = 0.0;
    if (g < FG)
        for (int row = g; row < m * d2; row += FG) {
            const int i = row / d2, c = row - i * d2;
            acc += M.G_pt[(size_t)row * n + j] * Bt.v[((size_t)b * d2 + c) * m + i];
        }
    if (g < FG) fr[g * n + j] = acc;
    __syncthreads();
    if (tid < n) {
        double s = 0.0;
        for (int q = 0; q < FG; ++q) s += fr[q * n + tid];
        Bt.r[b * n + tid] = s;
    }
}

// Mixed-precision residual r_b = sum_k Gdf[k] v_b[k] (k = (component, point) in the order of v) in
// double-float arithmetic: G is held as an FP32 (hi, lo) pair, each v element is split once when it
// is staged, products are formed by TwoProd with the two cross terms and summed by TwoSum with a
// separate FP32 compensation (Ogita, Rump & Oishi 2005), ~1e-13 relative to sum |terms|.  The FP64
// pipe of this GPU runs at 1/64 of the FP32 rate, so the 12 FP32 operations of one double-float
// multiply-add cost ~5x less than one DFMA.  The instances share G: a CTA of 256 threads takes
// FDF_NI instances and CW columns j (blockIdx.y), thread (j, ig) accumulates FDF_IPT instances.
// Chunks of FDF_RC rows of G (cp.async) and of the v rows of the FDF_NI instances (through
// registers, split on the way) are double-buffered in shared memory, so that the loads of the next
// chunk overlap the arithmetic of this one.  Each thread sums its rows in a fixed order, so the
// result does not depend on the launch.
constexpr int FDF_RC = 32;                 // rows per staged chunk
constexpr int FDF_NI = 16;                 // instances per CTA
constexpr int FDF_LD = FDF_NI * FDF_RC / 256;   // staged v elements per thread and chunk
// CW columns per CTA (64 for n > 32, else 32 so that small bases keep the threads busy):
// 256 / CW column groups, each thread accumulating FDF_NI * CW / 256 instances

__device__ __forceinline__ void df_mac(float &s, float &er, float2 g, float2 v) {
    const float pr = __fmul_rn(g.x, v.x);
    float e = fmaf(g.x, v.x, -pr);
    e = fmaf(g.x, v.y, e);
    e = fmaf(g.y, v.x, e);
    const float sn = __fadd_rn(s, pr);
    const float bb = __fsub_rn(sn, s);
    const float t = __fadd_rn(__fsub_rn(s, __fsub_rn(sn, bb)), __fsub_rn(pr, bb));
    s = sn;
    er = __fadd_rn(er, __fadd_rn(t, e));
}

__device__ __forceinline__ void fdf_cp16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

template <int CW>
__global__ void __launch_bounds__(256) k_force_df(Model M, Batch Bt) {
    constexpr int FDF_IPT = FDF_NI * CW / 256;          // instances per thread
    constexpr int FDF_GLD = FDF_RC * (CW / 2) / 256;    // 16-byte G copies per thread and chunk
    __shared__ __align__(16) float2 gs[2][FDF_RC][CW];
    __shared__ float2 vs[2][FDF_NI][FDF_RC];
    const int n_act = Bt.counts[0];
    const int p0 = blockIdx.x * FDF_NI;
    if (p0 >= n_act) return;
    const int n = M.n, np = (n + 1) & ~1, K = M.m * M.d2;
    const int tid = threadIdx.x, ig = tid / CW, jl = tid % CW;
    const int j0 = blockIdx.y * CW, j = j0 + jl;
    const int nc2 = min(CW, np - j0) / 2;   // 16-byte column pairs of this column block
    const int nch = (K + FDF_RC - 1) / FDF_RC;
    // v staging map: element e = tid + 256 t of a chunk is row e % FDF_RC of instance slot e / FDF_RC
    const double *vrow[FDF_LD];
#pragma unroll
    for (int t = 0; t < FDF_LD; ++t) {
        const int e = tid + 256 * t, slot = e / FDF_RC;
        vrow[t] = (p0 + slot < n_act) ? Bt.v + (size_t)Bt.list[p0 + slot] * K + (e % FDF_RC) : nullptr;
    }
    double pre[FDF_LD];
    auto load = [&](int c) {
#pragma unroll
        for (int t = 0; t < FDF_LD; ++t) {
            const int k = c * FDF_RC + (tid + 256 * t) % FDF_RC;
            pre[t] = (vrow[t] && k < K) ? vrow[t][(size_t)c * FDF_RC] : 0.0;
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int t = 0; t < FDF_LD; ++t) {
            const int e = tid + 256 * t;
            const float h = (float)pre[t];
            vs[buf][e / FDF_RC][e % FDF_RC] = make_float2(h, (float)(pre[t] - (double)h));
        }
    };
    // G rows k0 .. k0 + FDF_RC of this column block (rows of the image are np pairs, 16-byte aligned)
    auto stage_g = [&](int c) {
        const int k0 = c * FDF_RC;
#pragma unroll
        for (int t = 0; t < FDF_GLD; ++t) {
            const int e = tid + 256 * t, row = e / (CW / 2), q = e % (CW / 2);
            if (q < nc2 && k0 + row < K) fdf_cp16(&gs[c & 1][row][2 * q], M.Gdf + (size_t)(k0 + row) * np + j0 + 2 * q);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    float s[FDF_IPT], er[FDF_IPT];
#pragma unroll
    for (int u = 0; u < FDF_IPT; ++u) { s[u] = 0.f; er[u] = 0.f; }
    stage_g(0);
    load(0);
    store(0);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    const bool colok = j < n;
    for (int c = 0; c < nch; ++c) {
        if (c + 1 < nch) {
            stage_g(c + 1);
            load(c + 1);
        }
        const int rows = min(FDF_RC, K - c * FDF_RC);
        const float2 (*vb)[FDF_RC] = vs[c & 1] + ig * FDF_IPT;
        const float2 (*gb)[CW] = gs[c & 1];
        if (colok) {
#pragma unroll 4
            for (int r = 0; r < rows; ++r) {
                const float2 gg = gb[r][jl];
#pragma unroll
                for (int u = 0; u < FDF_IPT; ++u) df_mac(s[u], er[u], gg, vb[u][r]);
            }
        }
        if (c + 1 < nch) store((c + 1) & 1);
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
    }
    if (colok)
#pragma unroll
        for (int u = 0; u < FDF_IPT; ++u) {
            const int p = p0 + ig * FDF_IPT + u;
            if (p < n_act) Bt.r[(size_t)Bt.list[p] * n + j] = (double)s[u] + (double)er[u];
        }
}

// bytes of one B-operand chunk image and the chunk count for a model
void tc_image_shape(int d, int fmt, int m, int *chunk_bytes, int *nchunks) {
    const int d2 = d * d;
    const int PC = fmt == 1 ? 16 : 8;
    const int KC = PC * d2, ES = fmt == 1 ? 2 : 4;
    const int SBO = KC * ES / 16 * 128;
    *chunk_bytes = (tc::NCOLS / 8) * SBO;
    *nchunks = (m + PC - 1) / PC;
}

// host: pre-arranged B-operand image of G[m][d2][n] (n <= 64), chunk-major
void tc_build_image(int d, int fmt, int n, int m, const double *G, unsigned char *img) {
    const int d2 = d * d;
    const int PC = fmt == 1 ? 16 : 8;
    const int KC = PC * d2, ES = fmt == 1 ? 2 : 4;
    const int SBO = KC * ES / 16 * 128;
    int cb, nch;
    tc_image_shape(d, fmt, m, &cb, &nch);
    for (int c = 0; c < nch; ++c) {
        unsigned char *t = img + (size_t)c * cb;
        for (int j = 0; j < tc::NCOLS; ++j)
            for (int k = 0; k < KC; ++k) {
                const int ii = k / d2, q = k % d2, i = c * PC + ii;
                const double g = (j < n && i < m) ? G[((size_t)i * d2 + q) * n + j] : 0.0;
                if (fmt == 1) {
                    const int off = (j >> 3) * SBO + (k >> 3) * 128 + (j & 7) * 16 + (k & 7) * 2;
                    const __nv_bfloat16 h = __float2bfloat16((float)g);
                    memcpy(t + off, &h, 2);
                } else {
                    const int off = (j >> 3) * SBO + (k >> 2) * 128 + (j & 7) * 16 + (k & 3) * 4;
                    const float f = (float)g;
                    memcpy(t + off, &f, 4);
                }
            }
    }
}

template <int D, int FMT>
static int launch_tc_t(const Model &M, Batch Bt, const unsigned char *img, int *err, cudaStream_t s) {
    constexpr int D2 = D * D, D4 = D2 * D2;
    constexpr int PC = (FMT == 1) ? 16 : 8;
    constexpr int KC = PC * D2, ES = (FMT == 1) ? 2 : 4;
    constexpr int SBO = KC * ES / 16 * 128;
    constexpr int A_BYTES = (tc::MROWS / 8) * SBO, B_BYTES = (tc::NCOLS / 8) * SBO;
    const size_t sm = 2 * (size_t)A_BYTES + 2 * (size_t)B_BYTES + (size_t)PC * D2 * tc::NCOLS * 4 + 2 * (size_t)PC * D4 * 4;
    if (M.n > tc::NCOLS) return -1;
    const int nch = (M.m + PC - 1) / PC;
    cudaFuncSetAttribute(k_assemble_tc<D, FMT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_assemble_tc<D, FMT><<<(int)((Bt.B + 1) / 2), tc::THREADS, sm, s>>>(M, Bt, img, nch, err);
    return 0;
}

// residual r = sum_i G_i^T v_i of the listed instances (paths whose stiffness kernel does not
// produce it): double-float when the model carries the split image of G and fp64 is not asked
// for, else FP64
void launch_force(const Model &M, Batch Bt, bool fp64, cudaStream_t s) {
    if (M.Gdf && !fp64) {
        if (M.n > 32) {
            const dim3 grid((unsigned)((Bt.B + FDF_NI - 1) / FDF_NI), (unsigned)((M.n + 63) / 64));
            k_force_df<64><<<grid, 256, 0, s>>>(M, Bt);
        } else {
            const dim3 grid((unsigned)((Bt.B + FDF_NI - 1) / FDF_NI), 1u);
            k_force_df<32><<<grid, 256, 0, s>>>(M, Bt);
        }
    } else {
        k_force<<<(int)Bt.B, 256, 0, s>>>(M, Bt);
    }
}

int launch_tc(int fmt, const Model &M, Batch Bt, const unsigned char *img, int *err, cudaStream_t s) {
    if (M.d == 2) return fmt == 1 ? launch_tc_t<2, 1>(M, Bt, img, err, s) : launch_tc_t<2, 2>(M, Bt, img, err, s);
    return fmt == 1 ? launch_tc_t<3, 1>(M, Bt, img, err, s) : launch_tc_t<3, 2>(M, Bt, img, err, s);
}

}  // namespace podecm
