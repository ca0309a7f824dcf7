// Reduced stiffness of the 3D model, K_b = sum_i G_i^T At_i G_i (Eq. stiffnessmatrix_ecm), on the
// 5th-generation tensor cores, with several instances per CTA sharing every basis tile.
//
// Formulation (per instance b): Y_b = blockdiag_i(At_i^T) G (rows = (point i, component c)), then
// K_b = Y_b^T G, i.e. K[j][l] = sum_i sum_{a,c} G_i[a][j] At_i[a][c] G_i[c][l].  One CTA holds NI = 2 NP instances; instance pair p owns one tensor-memory
// accumulator D_p[128 x 64] (rows 0..63 = K rows of instance 2p, rows 64..127 = instance 2p+1),
// and every MMA of a chunk uses the same B operand (the shared basis tile):
//   D_p += A_p[128 x KC] B[64 x KC]^T,  A_p rows = (instance, j), B rows = l, K = (point, component).
// The K dimension runs over chunks of PC = 4 cubature points; inside a chunk point pt owns KP
// consecutive K slots (its 9 components followed by zero padding: 16 slots in BF16, 12 in TF32),
// so that one producer thread writes the 9 values of a row with 16-byte stores.
//
// Roles (warp specialisation):
//   * producer warps (NPROD threads): thread (instance, point, j-block) keeps the 81 tangent
//     entries of its cubature point in registers, reads the FP32 basis block G_i[:, j..j+3] from
//     shared memory and writes Y^T = (At_i^T G_i)^T for its rows (so that D = K, not K^T, when
//     the FP32 tangent is not exactly symmetric), rounded to BF16 or TF32 (MODE 3
//     writes a TF32 hi/lo pair, see below) into the canonical K-major layout;
//     the tangent of the next chunk is prefetched with cp.async while the current one is used;
//   * one control thread: bulk copies (TMA engine, cp.async.bulk) of the FP32 basis chunk and of
//     the pre-arranged B-operand image into a 2-stage ring, then, once the producers have
//     arrived on the stage's mbarrier, NP x (KC / KSTEP) tcgen05.mma and one tcgen05.commit.
// MODE 1 = BF16 operands, MODE 2 = TF32, MODE 3 = TF32 split: A = A_hi + A_lo, B = B_hi + B_lo
// with A_hi = tf32(A), A_lo = tf32(A - A_hi); the MMA computes A_hi B_hi + A_lo B_hi + A_hi B_lo,
// an FP32-accurate product (the dropped A_lo B_lo term is below FP32 rounding).
// Shared-memory operand layout (no swizzle, K-major): 8-row x 16-byte core matrices, core
// matrices adjacent in K 128 bytes apart (LBO); 8-row groups SBO bytes apart.  The A tiles use
// SBO = (K core blocks) * 128 + 16: the extra 16 bytes spread the producers' 16-byte stores of
// neighbouring row groups over distinct banks.
// Every wait is bounded (wall clock); on timeout the CTA records an error, stops issuing work,
// waits (bounded) for its own outstanding copies and MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cstdint>
#include <cstring>

#include "kernels.cuh"
#include "tcgen05.cuh"

namespace podecm {

namespace tc3 {
using namespace tcx;

constexpr int D2 = 9, D4 = 81;
constexpr int PC = 4;                         // cubature points per chunk
constexpr int NCOLS = 64;                     // MMA N (n padded to 64)
constexpr int GS_BYTES = PC * D2 * NCOLS * 4; // FP32 basis chunk [PC][9][64]

template <int MODE>
struct Cfg {
    static constexpr bool SPLIT = MODE == 3;
    static constexpr int ES = MODE == 1 ? 2 : 4;            // operand element bytes
    static constexpr int KP = MODE == 1 ? 16 : 12;          // K slots per point
    static constexpr int CW = 16 / ES;                      // elements per core-matrix row
    static constexpr int KSTEP = MODE == 1 ? 16 : 8;        // K per tcgen05.mma
    static constexpr int NP = MODE == 1 ? 4 : (MODE == 2 ? 2 : 1);   // instance pairs per CTA
    static constexpr int NI = 2 * NP;
    static constexpr int JT = MODE == 1 ? 8 : 4;            // basis columns per producer thread
    static constexpr int TPI = NCOLS / JT;                  // threads per (instance, point)
    static constexpr int NPROD = NI * PC * TPI;
    static constexpr int THREADS = NPROD + 32;
    static constexpr int KC = PC * KP;
    static constexpr int NKB = KC / CW;                     // core blocks along K
    static constexpr int SBO_A = NKB * 128 + 16;
    static constexpr int A_BYTES = 16 * SBO_A;
    static constexpr int SBO_B = NKB * 128;
    static constexpr int B_BYTES = 8 * SBO_B;
    static constexpr int NK = KC / KSTEP;
    static constexpr int NAT = NP * (SPLIT ? 2 : 1);
    static constexpr int NBT = SPLIT ? 2 : 1;
    static constexpr int STAGE = NAT * A_BYTES + NBT * B_BYTES + GS_BYTES;
    static constexpr int AS_BYTES = NI * D4 * PC * 4;
    static constexpr int SMEM = 2 * STAGE + 2 * AS_BYTES;
    // accumulators: the tensor core adds into FP32 with truncation, so the error of a long
    // chain of MMAs grows with its length; chunk c of pair p goes to accumulator c % NH, and in
    // the split mode the small A_lo B_hi + A_hi B_lo terms go to one more accumulator (NL = 1)
    static constexpr int NL = SPLIT ? 1 : 0;
    static constexpr int NH = 512 / (NP * NCOLS) - NL;
    static constexpr int NACC = NH + NL;
    static constexpr int TMEM_COLS = 512;
    static constexpr uint32_t IDESC = (1u << 4) | ((MODE == 1 ? 1u : 2u) << 7) | ((MODE == 1 ? 1u : 2u) << 10) |
                                      ((uint32_t)(NCOLS >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
};

template <int MODE>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
    if (MODE == 1) mma_f16(tmem_d, adesc, bdesc, Cfg<MODE>::IDESC, acc);
    else mma_tf32(tmem_d, adesc, bdesc, Cfg<MODE>::IDESC, acc);
}

// image offsets (bytes) inside the per-model image buffer
// A operand of the Y-MMA (k_assemble_tc4): for the cubature point pair (2p, 2p+1) of a chunk the
// block-diagonal [G_2p^T 0; 0 G_2p+1^T] as 128 rows (s, j) x 24 K slots (s', q; 9 used per
// point), TF32, canonical K-major layout (SBO 768 B)
constexpr int AY_SBO = 6 * 128;
constexpr int AY_BYTES = 16 * AY_SBO;

struct ImgLayout {
    size_t g32, bf16, tf_hi, tf_lo, ay, total;
    int nch;
};

__host__ __device__ inline ImgLayout img_layout(int m) {
    ImgLayout L;
    L.nch = (m + PC - 1) / PC;
    L.g32 = 0;
    L.bf16 = L.g32 + (size_t)L.nch * GS_BYTES;
    L.tf_hi = L.bf16 + (size_t)L.nch * Cfg<1>::B_BYTES;
    L.tf_lo = L.tf_hi + (size_t)L.nch * Cfg<2>::B_BYTES;
    L.ay = L.tf_lo + (size_t)L.nch * Cfg<2>::B_BYTES;
    L.total = L.ay + (size_t)L.nch * 2 * AY_BYTES;
    return L;
}

}  // namespace tc3

template <int MODE>
__global__ void __launch_bounds__(tc3::Cfg<MODE>::THREADS, 1)
    k_assemble_tc3(Model M, Batch Bt, const unsigned char *__restrict__ img, int *err_flag, int sel) {
    using namespace tc3;
    using C = Cfg<MODE>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_full[2], bar_afull[2], bar_mma[2];
    __shared__ uint32_t tmem_base;
    __shared__ int64_t bI[C::NI];
    __shared__ volatile int abort_s;
    __shared__ int n_sel;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_act = Bt.counts[0];
    const int p0 = C::NI * blockIdx.x;
    if (p0 >= n_act) return;
    const int n = M.n, m = M.m, mA = M.mA;
    const ImgLayout L = img_layout(m);
    const int nch = L.nch;
    const float *At = reinterpret_cast<const float *>(Bt.At);
    const unsigned char *img_g32 = img + L.g32;
    const unsigned char *img_b0 = img + (MODE == 1 ? L.bf16 : L.tf_hi);
    const unsigned char *img_b1 = img + L.tf_lo;
    auto stage_ptr = [&](int s) { return smem + (size_t)s * C::STAGE; };
    auto a_tile = [&](int s, int t) { return stage_ptr(s) + (size_t)t * C::A_BYTES; };
    auto b_tile = [&](int s, int t) { return stage_ptr(s) + (size_t)C::NAT * C::A_BYTES + (size_t)t * C::B_BYTES; };
    auto g_tile = [&](int s) {
        return reinterpret_cast<float *>(stage_ptr(s) + (size_t)C::NAT * C::A_BYTES + (size_t)C::NBT * C::B_BYTES);
    };
    // staged tangents of buffer t at As0 + t * AS_BYTES / 4 (arithmetic, no pointer array in local memory)
    float *const As0 = reinterpret_cast<float *>(smem + 2 * (size_t)C::STAGE);

    // sel: 0 every listed instance, 1 those without the accurate-stiffness flag, 2 those with it
    if (tid == 0) n_sel = 0;
    __syncthreads();
    if (tid < C::NI) {
        int64_t b = -1;
        if (p0 + tid < n_act) {
            b = Bt.list[p0 + tid];
            if (sel != 0 && ((Bt.ctl[b].acc_k != 0) != (sel == 2))) b = -1;
        }
        bI[tid] = b;
        if (b >= 0) atomicAdd(&n_sel, 1);
    }
    __syncthreads();
    if (n_sel == 0) return;
    if (warp == C::NPROD / 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(C::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&bar_full[s], 1);
            mbar_init(&bar_afull[s], C::NPROD);
            mbar_init(&bar_mma[s], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_s = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (tid < C::NPROD) {
        // ------------------------------------------------------------------ producers
        const int jb = tid % C::TPI, pi = tid / C::TPI;
        const int inst = pi / PC, pt = pi % PC;
        const int pair = inst >> 1, half = inst & 1;
        const bool inst_ok = bI[inst] >= 0;
        auto prefetch = [&](int c, int buf) {
            const int c0 = c * PC;
            for (int e = tid; e < C::NI * D4; e += C::NPROD) {
                const int ie = e / D4, ce = e - ie * D4;
                const int64_t be = bI[ie];
                if (be >= 0) cp_async16(As0 + (size_t)buf * (C::AS_BYTES / 4) + (size_t)e * PC, At + ((size_t)be * D4 + ce) * mA + c0);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        prefetch(0, 0);
        int local_abort = 0;
        for (int c = 0; c < nch; ++c) {
            const int s = c & 1;
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            if (bar_or(C::NPROD, local_abort | abort_s)) break;   // also: chunk c's tangents visible
            if (c + 1 < nch) prefetch(c + 1, (c + 1) & 1);
            const uint32_t par = (uint32_t)(c >> 1) & 1u;
            if (!mbar_wait(&bar_full[s], par, &abort_s)) { local_abort = 1; continue; }
            if (c >= 2 && !mbar_wait(&bar_mma[s], par ^ 1u, &abort_s)) { local_abort = 1; continue; }
            float a[D4];
            const bool pt_ok = inst_ok && (c * PC + pt < m);
            const float *asrc = As0 + (size_t)(c & 1) * (C::AS_BYTES / 4) + (size_t)inst * D4 * PC + pt;
#pragma unroll
            for (int e = 0; e < D4; ++e) a[e] = pt_ok ? asrc[e * PC] : 0.f;
            const float *Gs = g_tile(s);
            unsigned char *Ahi = a_tile(s, C::SPLIT ? 2 * pair : pair);
            unsigned char *Alo = a_tile(s, C::SPLIT ? 2 * pair + 1 : pair);
#pragma unroll
            for (int q4 = 0; q4 < C::JT / 4; ++q4) {
                const int j0 = q4 * 4 * C::TPI + jb * 4;
                float4 g[D2];
#pragma unroll
                for (int q = 0; q < D2; ++q) g[q] = *reinterpret_cast<const float4 *>(Gs + (pt * D2 + q) * NCOLS + j0);
                float y[D2][4];
#pragma unroll
                for (int cc = 0; cc < D2; ++cc) {
                    // Y = At^T G: K[j][l] = sum G[q][j] At[q][cc] G[cc][l]; packed FP32 pairs (FFMA2)
                    float2 y01 = make_float2(0.f, 0.f), y23 = make_float2(0.f, 0.f);
#pragma unroll
                    for (int q = 0; q < D2; ++q) {
                        const float av = a[q * D2 + cc];
                        const float2 aa = make_float2(av, av);
                        y01 = __ffma2_rn(aa, make_float2(g[q].x, g[q].y), y01);
                        y23 = __ffma2_rn(aa, make_float2(g[q].z, g[q].w), y23);
                    }
                    y[cc][0] = y01.x; y[cc][1] = y01.y; y[cc][2] = y23.x; y[cc][3] = y23.y;
                }
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    const int r = half * 64 + j0 + jj;
                    const size_t rb = (size_t)(r >> 3) * C::SBO_A + (size_t)(r & 7) * 16;
                    if (MODE == 1) {
                        uint4 v0, v1;
                        v0.x = pack_bf16(y[0][jj], y[1][jj]); v0.y = pack_bf16(y[2][jj], y[3][jj]);
                        v0.z = pack_bf16(y[4][jj], y[5][jj]); v0.w = pack_bf16(y[6][jj], y[7][jj]);
                        v1.x = pack_bf16(y[8][jj], 0.f); v1.y = 0u; v1.z = 0u; v1.w = 0u;
                        *reinterpret_cast<uint4 *>(Ahi + rb + (size_t)(2 * pt) * 128) = v0;
                        *reinterpret_cast<uint4 *>(Ahi + rb + (size_t)(2 * pt + 1) * 128) = v1;
                    } else {
                        uint32_t h[D2];
#pragma unroll
                        for (int cc = 0; cc < D2; ++cc) h[cc] = tf32_bits(y[cc][jj]);
                        *reinterpret_cast<uint4 *>(Ahi + rb + (size_t)(3 * pt) * 128) = make_uint4(h[0], h[1], h[2], h[3]);
                        *reinterpret_cast<uint4 *>(Ahi + rb + (size_t)(3 * pt + 1) * 128) = make_uint4(h[4], h[5], h[6], h[7]);
                        *reinterpret_cast<uint4 *>(Ahi + rb + (size_t)(3 * pt + 2) * 128) = make_uint4(h[8], 0u, 0u, 0u);
                        if (C::SPLIT) {
                            uint32_t l[D2];
#pragma unroll
                            for (int cc = 0; cc < D2; ++cc) l[cc] = tf32_bits(y[cc][jj] - __uint_as_float(h[cc]));
                            *reinterpret_cast<uint4 *>(Alo + rb + (size_t)(3 * pt) * 128) = make_uint4(l[0], l[1], l[2], l[3]);
                            *reinterpret_cast<uint4 *>(Alo + rb + (size_t)(3 * pt + 1) * 128) = make_uint4(l[4], l[5], l[6], l[7]);
                            *reinterpret_cast<uint4 *>(Alo + rb + (size_t)(3 * pt + 2) * 128) = make_uint4(l[8], 0u, 0u, 0u);
                        }
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&bar_afull[s]);
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
    } else if (lane == 0) {
        // ------------------------------------------------------------- control thread
        uint32_t copy_pending = 0, copy_par = 0;   // bit s: a copy into stage s in flight / its parity
        int mma_pending = 0;
        uint32_t mma_par = 0;
        int mma_stage = 0;
        auto issue_copies = [&](int c) {
            const int s = c & 1;
            const uint32_t bytes = GS_BYTES + C::NBT * C::B_BYTES;
            mbar_expect_tx(&bar_full[s], bytes);
            bulk_g2s(g_tile(s), img_g32 + (size_t)c * GS_BYTES, GS_BYTES, &bar_full[s]);
            bulk_g2s(b_tile(s, 0), img_b0 + (size_t)c * C::B_BYTES, C::B_BYTES, &bar_full[s]);
            if (C::SPLIT) bulk_g2s(b_tile(s, 1), img_b1 + (size_t)c * C::B_BYTES, C::B_BYTES, &bar_full[s]);
            copy_pending |= 1u << s;
            copy_par = (copy_par & ~(1u << s)) | (((uint32_t)(c >> 1) & 1u) << s);
        };
        issue_copies(0);
        if (nch > 1) issue_copies(1);
        for (int c = 0; c < nch; ++c) {
            const int s = c & 1;
            const uint32_t par = (uint32_t)(c >> 1) & 1u;
            if (!mbar_wait(&bar_full[s], par, &abort_s)) break;
            copy_pending &= ~(1u << s);
            if (!mbar_wait(&bar_afull[s], par, &abort_s)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int ah_idx = c % C::NH;
#pragma unroll 1
            for (int p = 0; p < C::NP; ++p) {
                // accumulator a of pair p: TMEM columns (a * NP + p) * 64
                const uint32_t dh = tmem + (uint32_t)((ah_idx * C::NP + p) * NCOLS);
                const uint32_t dl = tmem + (uint32_t)((C::NH * C::NP + p) * NCOLS);
                const uint32_t ah = smem_u32(a_tile(s, C::SPLIT ? 2 * p : p));
                const uint32_t bh = smem_u32(b_tile(s, 0));
#pragma unroll
                for (int k = 0; k < C::NK; ++k) {
                    const uint64_t adh = make_desc(ah + k * 256, 128, C::SBO_A);
                    const uint64_t bdh = make_desc(bh + k * 256, 128, C::SBO_B);
                    mma<MODE>(dh, adh, bdh, (c >= C::NH || k > 0) ? 1u : 0u);
                    if (C::SPLIT) {
                        const uint32_t al = smem_u32(a_tile(s, 2 * p + 1));
                        const uint32_t bl = smem_u32(b_tile(s, 1));
                        mma<MODE>(dl, make_desc(al + k * 256, 128, C::SBO_A), bdh, (c > 0 || k > 0) ? 1u : 0u);
                        mma<MODE>(dl, adh, make_desc(bl + k * 256, 128, C::SBO_B), 1u);
                    }
                }
            }
            mma_commit(&bar_mma[s]);
            mma_pending = 1;
            mma_par = par;
            mma_stage = s;
            if (c + 2 < nch) {
                if (!mbar_wait(&bar_mma[s], par, &abort_s)) break;
                issue_copies(c + 2);
            }
        }
        // drain: the last commit covers every MMA issued before it; outstanding copies must land
        if (mma_pending && !mbar_wait(&bar_mma[mma_stage], mma_par, &abort_s)) {
            // a second bounded wait that ignores the abort flag: the MMAs read shared memory
            const unsigned long long t0 = now_ns();
            while (!mbar_test(&bar_mma[mma_stage], mma_par) && now_ns() - t0 < WAIT_NS) {}
        }
        for (int s = 0; s < 2; ++s)
            if ((copy_pending >> s) & 1u) mbar_drain(&bar_full[s], (copy_par >> s) & 1u);
        if (abort_s && err_flag) atomicExch(err_flag, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!abort_s && tid < C::NPROD) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 of the pairs p = w / 4 (mod NPROD / 128)
        const int quad = warp & 3;
        const int row = quad * 32 + lane;
        const int ih = row >> 6, j = row & 63;
        const int n_used = (nch < C::NH ? nch : C::NH) + C::NL;   // accumulators written
        for (int p = warp >> 2; p < C::NP; p += C::NPROD / 128) {
            double v[64];
#pragma unroll
            for (int q = 0; q < 64; ++q) v[q] = 0.0;
#pragma unroll 1
            for (int ai = 0; ai < C::NACC; ++ai) {
                if (ai < C::NH && ai >= n_used - C::NL) continue;   // hi accumulator never written
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)((ai * C::NP + p) * NCOLS + hh * 32);
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
                for (int q = 0; q < 32; ++q) v[hh * 32 + q] += f2d_exact(__uint_as_float(r[q]));   // widening off the FP64 pipe
            }
            }
            const int64_t b = bI[2 * p + ih];
            if (j < n && b >= 0) {
                double *Kb = Bt.K + (size_t)b * n * n + (size_t)j * n;
#pragma unroll
                for (int k = 0; k < NCOLS; ++k)
                    if (k < n) Kb[k] = v[k];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == C::NPROD / 32) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS));
    }
}

// ---------------------------------------------------------------- Y on the tensor cores
// k_assemble_tc4 (TF32): the same K_b = Y_b^T G, but Y = At^T G is formed by the tensor cores as
// well.  For a pair of cubature points (2p, 2p+1) of a chunk, one Y-MMA computes
//   D_Y[(s, j)][(inst, c)] = sum_q G_{2p+s}[q][j] At_{inst, 2p+s}[q][c]      (M 128, N 80, K 24)
// with the block-diagonal A = [G_2p^T 0; 0 G_2p+1^T] (a pre-arranged image) and B = the tangents
// of the 8 instances of the CTA (rows (inst, c), written by the producer warps); converter warps
// read D_Y from tensor memory (lane (s, j) holds 72 values), round them to TF32 and store them as
// rows (inst, j) of the K-GEMM A tiles, and the control thread then issues the K-MMAs of the
// chunk (4 instance pairs, M 128, N 64, K 48) into one tensor-memory accumulator per pair.
// Roles: warps 0-3 converters (tensor-memory lane quadrants), warps 4-7 producers (tangent
// staging with cp.async, both Y-MMA operands: the block-diagonal A is assembled in shared memory
// from the K-GEMM B tile of the chunk, so only that tile comes from L2), warp 8 control (bulk
// copies of the B tiles into a 3-stage ring, MMA issue, commits).  A_K is split into two halves
// (the K slots of point pair 0 and 1): the converters write half h of chunk c + 1 once the K-MMAs
// of chunk c that read it are done, and the control thread issues the K-MMAs of half 0, the
// Y-MMA of the next chunk's first point pair, the K-MMAs of half 1 and the second Y-MMA, so
// that conversion, Y and K overlap.
namespace tc4 {
using tc3::D2;
using tc3::D4;
using tc3::PC;
using tc3::NCOLS;
constexpr int NI = 8, NP = 4;                    // instances, instance pairs per CTA
constexpr int NY = 80;                           // Y-MMA N: 8 instances x 9 components + 8 zero rows
constexpr int BY_SBO = 6 * 128;                  // B_Y: 80 rows x 24 TF32 slots
constexpr int BY_BYTES = 10 * BY_SBO;
constexpr int KP = 12, KC = PC * KP;             // K-MMA K per chunk: 4 points x 12 slots
constexpr int SBO_A = (KC / 4) * 128 + 16;       // A_K rows (inst, j); +16 B spreads row groups over banks
constexpr int A_BYTES = 16 * SBO_A;
constexpr int B_BYTES = tc3::Cfg<2>::B_BYTES;    // the TF32 (hi) B-operand image of G
constexpr int SBO_B = tc3::Cfg<2>::SBO_B;
constexpr int AS_BYTES = NI * D4 * PC * 4;
constexpr int NBK = 3;                           // B tile ring stages
constexpr int OFF_AK = 0;
constexpr int OFF_AY = OFF_AK + NP * A_BYTES;
constexpr int OFF_BK = OFF_AY + 2 * 2 * tc3::AY_BYTES;
constexpr int OFF_BY = OFF_BK + NBK * B_BYTES;
constexpr int OFF_AS = OFF_BY + 2 * BY_BYTES;
constexpr int SMEM = OFF_AS + 2 * AS_BYTES;
constexpr int THREADS = 288;
constexpr int TMEM_Y = 256;                      // D_K[ip] at columns 64 ip, D_Y[pp] at 256 + 128 pp
constexpr uint32_t IDESC_Y = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NY >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
constexpr uint32_t IDESC_K = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NCOLS >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);

}  // namespace tc4

__global__ void __launch_bounds__(tc4::THREADS, 1)
    k_assemble_tc4(Model M, Batch Bt, const unsigned char *__restrict__ img, int *err_flag, int sel) {
    using namespace tc3;
    using namespace tc4;
    extern __shared__ __align__(1024) unsigned char smem[];
    // bar_akh[h] / bar_kh[h]: A_K half h (the K slots of point pair h) written by the converters /
    // the K-MMAs reading it done
    __shared__ __align__(8) uint64_t bar_fbk[NBK], bar_by[2], bar_y[2], bar_yfree[2], bar_akh[2], bar_kh[2];
    __shared__ uint32_t tmem_base;
    __shared__ int64_t bI[NI];
    __shared__ volatile int abort_s;
    __shared__ int n_sel;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_act = Bt.counts[0];
    const int p0 = NI * blockIdx.x;
    if (p0 >= n_act) return;
    const int n = M.n, m = M.m, mA = M.mA;
    const ImgLayout L = img_layout(m);
    const int nch = L.nch;
    const float *At = reinterpret_cast<const float *>(Bt.At);
    float *const As0 = reinterpret_cast<float *>(smem + OFF_AS);   // buffer t at As0 + t * AS_BYTES / 4

    if (tid == 0) n_sel = 0;
    __syncthreads();
    if (tid < NI) {
        int64_t b = -1;
        if (p0 + tid < n_act) {
            b = Bt.list[p0 + tid];
            if (sel != 0 && ((Bt.ctl[b].acc_k != 0) != (sel == 2))) b = -1;
        }
        bI[tid] = b;
        if (b >= 0) atomicAdd(&n_sel, 1);
    }
    __syncthreads();
    if (n_sel == 0) return;
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < NBK; ++s) mbar_init(&bar_fbk[s], 1);
        for (int s = 0; s < 2; ++s) {
            mbar_init(&bar_by[s], 128);
            mbar_init(&bar_y[s], 1);
            mbar_init(&bar_yfree[s], 128);
            mbar_init(&bar_akh[s], 128);
            mbar_init(&bar_kh[s], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_s = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (warp < 4) {
        // ------------------------------------------------------------------ converters
        const int row = tid, sp = row >> 6, j = row & 63;
        int local_abort = 0;
        for (int c = 0; c < nch; ++c) {
            if (bar_or_id(2, 128, local_abort | abort_s)) break;
            const uint32_t par = (uint32_t)c & 1u;
            for (int pp = 0; pp < 2; ++pp) {
                // A_K half pp is free once the K-MMAs of chunk c - 1 that read it are done
                if (c >= 1 && !mbar_wait(&bar_kh[pp], par ^ 1u, &abort_s)) { local_abort = 1; break; }
                if (!mbar_wait(&bar_y[pp], par, &abort_s)) { local_abort = 1; break; }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                uint32_t v[72];
                const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(TMEM_Y + 128 * pp);
                tmem_ld32(ta, v);
                tmem_ld32(ta + 32, v + 32);
                tmem_ld8(ta + 64, v + 64);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                mbar_arrive(&bar_yfree[pp]);
                const int kb = 3 * (2 * pp + sp);
#pragma unroll
                for (int inst = 0; inst < NI; ++inst) {
                    unsigned char *Ak = smem + OFF_AK + (size_t)(inst >> 1) * A_BYTES;
                    const int r = (inst & 1) * 64 + j;
                    const size_t rb = (size_t)(r >> 3) * SBO_A + (size_t)(r & 7) * 16;
                    uint32_t h[D2];
#pragma unroll
                    for (int cc = 0; cc < D2; ++cc) h[cc] = tf32_bits(__uint_as_float(v[inst * D2 + cc]));
                    *reinterpret_cast<uint4 *>(Ak + rb + (size_t)kb * 128) = make_uint4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<uint4 *>(Ak + rb + (size_t)(kb + 1) * 128) = make_uint4(h[4], h[5], h[6], h[7]);
                    *reinterpret_cast<uint4 *>(Ak + rb + (size_t)(kb + 2) * 128) = make_uint4(h[8], 0u, 0u, 0u);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&bar_akh[pp]);
            }
        }
    } else if (warp < 8) {
        // ------------------------------------------------------------------ producers
        const int ptid = tid - 128;
        auto prefetch = [&](int c, int buf) {
            const int c0 = c * PC;
            for (int e = ptid; e < NI * D4; e += 128) {
                const int ie = e / D4, ce = e - ie * D4;
                const int64_t be = bI[ie];
                if (be >= 0) cp_async16(As0 + (size_t)buf * (AS_BYTES / 4) + (size_t)e * PC, At + ((size_t)be * D4 + ce) * mA + c0);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        // the off-diagonal blocks of the Y-MMA A operand stay zero
        for (int e = ptid; e < 2 * 2 * AY_BYTES / 16; e += 128)
            reinterpret_cast<uint4 *>(smem + OFF_AY)[e] = make_uint4(0u, 0u, 0u, 0u);
        prefetch(0, 0);
        int local_abort = 0;
        for (int c = 0; c < nch; ++c) {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            if (bar_or_id(1, 128, local_abort | abort_s)) break;   // also: chunk c's tangents visible
            if (c + 1 < nch) prefetch(c + 1, (c + 1) & 1);
            const float *as = As0 + (size_t)(c & 1) * (AS_BYTES / 4);
            const int kst = c % NBK;
            if (!mbar_wait(&bar_fbk[kst], (uint32_t)(c / NBK) & 1u, &abort_s)) { local_abort = 1; continue; }
            for (int pp = 0; pp < 2; ++pp) {
                // Y-MMA (c - 1, pp) done: B_Y[pp] free, and (with pp = 1) every MMA reading A_Y stage c & 1
                if (c >= 1 && !mbar_wait(&bar_y[pp], (uint32_t)(c - 1) & 1u, &abort_s)) { local_abort = 1; break; }
                if (pp == 0 && c >= 2 && !mbar_wait(&bar_y[1], (uint32_t)(c - 1) & 1u, &abort_s)) { local_abort = 1; break; }
                // A_Y[c & 1][pp]: core matrices of the B tile, rows (s, j) <- B rows j, K blocks of point 2 pp + s
                unsigned char *Ay = smem + OFF_AY + (size_t)((c & 1) * 2 + pp) * AY_BYTES;
                const unsigned char *Bk = smem + OFF_BK + (size_t)kst * B_BYTES;
                for (int e = ptid; e < 2 * 64 * 3; e += 128) {   // consecutive threads: consecutive rows j
                    const int j = e & 63, t = (e >> 6) % 3, sq = (e >> 6) / 3;
                    const uint4 v = *reinterpret_cast<const uint4 *>(Bk + (size_t)(j >> 3) * SBO_B +
                                                                      (size_t)(3 * (2 * pp + sq) + t) * 128 + (size_t)(j & 7) * 16);
                    const int r = sq * 64 + j;
                    *reinterpret_cast<uint4 *>(Ay + (size_t)(r >> 3) * AY_SBO + (size_t)(3 * sq + t) * 128 + (size_t)(r & 7) * 16) = v;
                }
                // B_Y[pp]: row (inst, cc), K slots (s, q) <- At_{inst, 2 pp + s}[q][cc]; one thread per row
                // reads both points of the pair with 8-byte loads (points are the innermost index of the
                // staged tangent)
                unsigned char *By = smem + OFF_BY + (size_t)pp * BY_BYTES;
                for (int nrow = ptid; nrow < NY; nrow += 128) {
                    const int inst = nrow / D2, cc = nrow - inst * D2;
                    const bool vrow = nrow < NI * D2 && bI[inst] >= 0;
                    const bool v0 = vrow && c * PC + 2 * pp < m, v1 = vrow && c * PC + 2 * pp + 1 < m;
                    uint32_t h0[D2], h1[D2];
#pragma unroll
                    for (int q = 0; q < D2; ++q) {
                        float2 t = make_float2(0.f, 0.f);
                        if (vrow) t = *reinterpret_cast<const float2 *>(as + ((size_t)inst * D4 + q * D2 + cc) * PC + 2 * pp);
                        h0[q] = v0 ? tf32_bits(t.x) : 0u;
                        h1[q] = v1 ? tf32_bits(t.y) : 0u;
                    }
                    const size_t rb = (size_t)(nrow >> 3) * BY_SBO + (size_t)(nrow & 7) * 16;
                    *reinterpret_cast<uint4 *>(By + rb) = make_uint4(h0[0], h0[1], h0[2], h0[3]);
                    *reinterpret_cast<uint4 *>(By + rb + 128) = make_uint4(h0[4], h0[5], h0[6], h0[7]);
                    *reinterpret_cast<uint4 *>(By + rb + 256) = make_uint4(h0[8], 0u, 0u, 0u);
                    *reinterpret_cast<uint4 *>(By + rb + 384) = make_uint4(h1[0], h1[1], h1[2], h1[3]);
                    *reinterpret_cast<uint4 *>(By + rb + 512) = make_uint4(h1[4], h1[5], h1[6], h1[7]);
                    *reinterpret_cast<uint4 *>(By + rb + 640) = make_uint4(h1[8], 0u, 0u, 0u);
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(&bar_by[pp]);
            }
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
    } else if (lane == 0) {
        // ------------------------------------------------------------- control thread
        // issue order per chunk c: K-MMAs of half 0 (chunk c), Y-MMA of point pair 0 (chunk c + 1),
        // K-MMAs of half 1, Y-MMA of point pair 1, so that the Y of the next chunk and the
        // conversion of its first half overlap the K-GEMM of this chunk
        uint32_t bk_pend = 0, bk_par = 0;   // bit st: a copy into ring stage st in flight / its parity
        uint64_t *last_bar = nullptr;   // the last commit covers every MMA issued before it
        uint32_t last_par = 0;
        auto copy_bk = [&](int c) {
            const int st = c % NBK;
            mbar_expect_tx(&bar_fbk[st], B_BYTES);
            bulk_g2s(smem + OFF_BK + (size_t)st * B_BYTES, img + L.tf_hi + (size_t)c * B_BYTES, B_BYTES, &bar_fbk[st]);
            bk_pend |= 1u << st;
            bk_par = (bk_par & ~(1u << st)) | (((uint32_t)(c / NBK) & 1u) << st);
        };
        auto issue_y = [&](int c, int pp) -> bool {
            const uint32_t par = (uint32_t)c & 1u;
            if (!mbar_wait(&bar_by[pp], par, &abort_s)) return false;
            if (c >= 1 && !mbar_wait(&bar_yfree[pp], par ^ 1u, &abort_s)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(smem + OFF_AY + (size_t)((c & 1) * 2 + pp) * AY_BYTES);
            const uint32_t b0 = smem_u32(smem + OFF_BY + (size_t)pp * BY_BYTES);
            const uint32_t d = tmem + (uint32_t)(TMEM_Y + 128 * pp);
#pragma unroll
            for (int k = 0; k < 3; ++k)
                mma_tf32(d, make_desc(a0 + k * 256, 128, AY_SBO), make_desc(b0 + k * 256, 128, BY_SBO), IDESC_Y,
                         k > 0 ? 1u : 0u);
            mma_commit(&bar_y[pp]);
            last_bar = &bar_y[pp];
            last_par = par;
            return true;
        };
        auto issue_k = [&](int c, int h) -> bool {
            const uint32_t par = (uint32_t)c & 1u;
            if (!mbar_wait(&bar_akh[h], par, &abort_s)) return false;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t bk0 = smem_u32(smem + OFF_BK + (size_t)(c % NBK) * B_BYTES);
#pragma unroll 1
            for (int ip = 0; ip < NP; ++ip) {
                const uint32_t ak0 = smem_u32(smem + OFF_AK + (size_t)ip * A_BYTES);
                const uint32_t d = tmem + (uint32_t)(ip * NCOLS);
#pragma unroll
                for (int k = 3 * h; k < 3 * h + 3; ++k)
                    mma_tf32(d, make_desc(ak0 + k * 256, 128, SBO_A), make_desc(bk0 + k * 256, 128, SBO_B), IDESC_K,
                             (c > 0 || k > 0) ? 1u : 0u);
            }
            mma_commit(&bar_kh[h]);
            last_bar = &bar_kh[h];
            last_par = par;
            return true;
        };
        for (int c = 0; c < NBK && c < nch; ++c) copy_bk(c);
        bool ok = issue_y(0, 0) && issue_y(0, 1);
        for (int c = 0; ok && c < nch; ++c) {
            const int kst = c % NBK;
            if (!mbar_wait(&bar_fbk[kst], (uint32_t)(c / NBK) & 1u, &abort_s)) break;
            bk_pend &= ~(1u << kst);
            if (c >= 1) {        // B stage (c + 2) % 3 = (c - 1) % 3 is free once the K-MMAs of chunk c - 1 are done
                if (!mbar_wait(&bar_kh[1], (uint32_t)(c - 1) & 1u, &abort_s)) break;
                if (c + 2 < nch) copy_bk(c + 2);
            }
            ok = issue_k(c, 0) && (c + 1 >= nch || issue_y(c + 1, 0)) && issue_k(c, 1) &&
                 (c + 1 >= nch || issue_y(c + 1, 1));
        }
        // drain: outstanding MMAs and copies must complete before the tensor memory is freed
        if (last_bar && !mbar_wait(last_bar, last_par, &abort_s)) {
            const unsigned long long t0 = now_ns();
            while (!mbar_test(last_bar, last_par) && now_ns() - t0 < WAIT_NS) {}
        }
        for (int st = 0; st < NBK; ++st)
            if ((bk_pend >> st) & 1u) mbar_drain(&bar_fbk[st], (bk_par >> st) & 1u);
        if (abort_s && err_flag) atomicExch(err_flag, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!abort_s && warp < 4) {
        // epilogue: warp w reads tensor-memory lanes 32 w .. 32 w + 31 of the four pair accumulators
        const int row = warp * 32 + lane, ih = row >> 6, j = row & 63;
        for (int ip = 0; ip < NP; ++ip) {
            uint32_t v[64];
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ip * NCOLS);
            tmem_ld32(ta, v);
            tmem_ld32(ta + 32, v + 32);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int64_t b = bI[2 * ip + ih];
            if (j < n && b >= 0) {
                double *Kb = Bt.K + (size_t)b * n * n + (size_t)j * n;
#pragma unroll
                for (int k = 0; k < NCOLS; ++k)
                    if (k < n) Kb[k] = f2d_exact(__uint_as_float(v[k]));
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 8) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

// ---------------------------------------------------------------- Abar sums on the tensor cores
// k_abar_tc3: for the converged instances, B_b = sum_i G_i^T Ahat_i (n x 9) with
// Ahat_i[ar][(k,l)] = sum_s At_i[ar][(k,s)] F_mu,i[l][s] (the sums of the effective stiffness,
// Eqs. eff_stiffness / eff_stiffness_ecm), FP32-accurate by the TF32 hi/lo split of
// k_assemble_tc3 MODE 3.  Formulation: B_b^T = Ahat_b^T G with S = 14 instances packed along M,
//   D[(s, kl)][l] += A[(s, kl)][(pt, ar)] G_pt[ar][l],
// whose B operand is the stiffness assembly's TF32 image of G (chunks of 4 points, 12 K slots per
// point, 9 used).  Roles as in k_assemble_tc3: 8 producer warps (tangent pieces staged by
// cp.async, F_mu of the chunk's points, A = Ahat^T rows rounded to TF32 hi and lo), one control
// thread (bulk copies of the B tiles into a 2-stage ring, 18 MMAs and one commit per chunk).
// Chunk c goes to accumulator c % 7, the split's small terms to an eighth; the epilogue adds
// them in FP32 and writes B_b [n][9] in FP64.  The producers also accumulate
// A0_b = sum_i wJ A_i in the F_mu-pushed-forward form A0[(a,j)][(k,l)] =
// sum_i sum_r F_mu[j][r] Ahat_i[(a,r)][(k,l)] (FP32 per thread, FP64 sum of two partials),
// written after B_b: Bsum[b] = [B_b (n x 9) | A0_b (81)].  Every wait is bounded (1 s; error
// flag, drain).
namespace tca {
using tc3::PC;
using tc3::D2;
using tc3::D4;
constexpr int D = 3;
constexpr int S = 14;                              // instances per CTA: rows (s, kl), 126 of 128
constexpr int NPROD = 256, THREADS = NPROD + 32;
constexpr int KP = 12, KC = PC * KP;               // 48 K slots per chunk
constexpr int SBO_A = (KC / 4) * 128 + 16;         // +16 B spreads row groups over banks
constexpr int A_BYTES = 16 * SBO_A;
constexpr int B_BYTES = tc3::Cfg<2>::B_BYTES, SBO_B = tc3::Cfg<2>::SBO_B;
constexpr int NK = KC / 8;                         // 6 K-steps per chunk
constexpr int STAGE = 2 * A_BYTES + 2 * B_BYTES;   // A hi, A lo, B hi, B lo
constexpr int AS_FLOATS = S * D4 * PC;             // staged tangents [S][81][4]
constexpr int FM_FLOATS = S * PC * D2;             // F_mu [S][4][9]
constexpr int GM_FLOATS = D2 * MAX_NPAR * PC;      // geometric-map gradients of a chunk [9 n_par][4]
constexpr int SMEM = 2 * STAGE + 2 * AS_FLOATS * 4 + FM_FLOATS * 4 + 2 * GM_FLOATS * 4;
constexpr int NH = 7, NACC = 8;                    // 64-column accumulators in 512 columns
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(64 >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}  // namespace tca

__global__ void __launch_bounds__(tca::THREADS, 1)
    k_abar_tc3(Model M, Batch Bt, const unsigned char *__restrict__ img, double *__restrict__ Bsum, int *err_flag) {
    using namespace tc3;
    using namespace tca;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_full[2], bar_afull[2], bar_mma[2];
    __shared__ uint32_t tmem_base;
    __shared__ int64_t bI[S];
    __shared__ float muS[S][MAX_NPAR];
    __shared__ volatile int abort_s;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_act = Bt.counts[0];
    const int p0 = S * blockIdx.x;
    if (p0 >= n_act) return;
    const int np = M.n_par;
    const int n = M.n, m = M.m, mA = M.mA;
    const ImgLayout L = img_layout(m);
    const int nch = L.nch;
    const float *At = reinterpret_cast<const float *>(Bt.At);
    auto a_tile = [&](int st, int t) { return smem + (size_t)st * STAGE + (size_t)t * A_BYTES; };
    auto b_tile = [&](int st, int t) { return smem + (size_t)st * STAGE + 2 * (size_t)A_BYTES + (size_t)t * B_BYTES; };
    float *const As0 = reinterpret_cast<float *>(smem + 2 * (size_t)STAGE);   // buffer t at As0 + t * AS_FLOATS
    float *const Fms = As0 + 2 * AS_FLOATS;                                     // [S][PC][9]
    float *const Gm0 = Fms + FM_FLOATS;                                         // buffer t at Gm0 + t * GM_FLOATS

    if (tid < S) bI[tid] = (p0 + tid < n_act) ? (int64_t)Bt.list[p0 + tid] : -1;
    for (int e = tid; e < S * np; e += THREADS) {
        const int s = e / np, k = e - s * np;
        muS[s][k] = (p0 + s < n_act) ? to_tangent<float>(Bt.mu[(int64_t)Bt.list[p0 + s] * np + k]) : 0.f;
    }
    if (warp == NPROD / 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int st = 0; st < 2; ++st) {
            mbar_init(&bar_full[st], 1);
            mbar_init(&bar_afull[st], NPROD);
            mbar_init(&bar_mma[st], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_s = 0;
    }
    // rows 126, 127 and the K slots 9..11 of every point are never produced: zero both A tiles of
    // both stages once (the producers rewrite only the used slots)
    for (int e = tid; e < 4 * A_BYTES / 16; e += THREADS) {
        const int t = e / (A_BYTES / 16), w = e - t * (A_BYTES / 16);
        *reinterpret_cast<uint4 *>(a_tile(t >> 1, t & 1) + (size_t)w * 16) = make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (tid < NPROD) {
        // ------------------------------------------------------------------ producers
        // tangent rows (instance s, component ce) of chunk c: one 16-byte piece of its 4 points;
        // absent instances and points past m as zeros (the columns past m of At are not written);
        // and the chunk's geometric-map gradients Gmu_T[q][k][i] (plain loads, spread over the
        // threads, so that the chunk's F_mu is formed from shared memory)
        auto prefetch = [&](int c, int buf) {
            const int c0 = c * PC;
            for (int e = tid; e < D2 * np * PC; e += NPROD) {
                const int qk = e / PC, pt = e - qk * PC;
                Gm0[(size_t)buf * GM_FLOATS + e] = (c0 + pt < m) ? to_tangent<float>(M.Gmu_T[(size_t)qk * m + c0 + pt]) : 0.f;
            }
            for (int e = tid; e < S * D4; e += NPROD) {
                const int s = e / D4, ce = e - s * D4;
                const int64_t b = bI[s];
                float *dst = As0 + (size_t)buf * AS_FLOATS + (size_t)e * PC;
                if (b >= 0 && c0 + PC <= m) {
                    cp_async16(dst, At + ((size_t)b * D4 + ce) * mA + c0);
                } else {
                    const float *src = At + ((size_t)(b >= 0 ? b : 0) * D4 + ce) * mA + c0;
                    float4 v;
                    v.x = (b >= 0 && c0 + 0 < m) ? src[0] : 0.f;
                    v.y = (b >= 0 && c0 + 1 < m) ? src[1] : 0.f;
                    v.z = (b >= 0 && c0 + 2 < m) ? src[2] : 0.f;
                    v.w = (b >= 0 && c0 + 3 < m) ? src[3] : 0.f;
                    *reinterpret_cast<float4 *>(dst) = v;
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        prefetch(0, 0);
        // thread (point pt, instance s, k): the rows (s, kl = 3 k + l), l = 0..2, of point pt, so
        // that each staged tangent entry serves three rows (168 of the 256 producer threads)
        const bool prod_row = tid < PC * S * D;
        const int ppt = tid / (S * D), rest = tid - ppt * (S * D);
        const int ps = rest / D, pk = rest - ps * D;
        float a0[D][D2];                                   // A0 partial sums of the rows (s, 3 k + l)
#pragma unroll
        for (int l = 0; l < D; ++l)
#pragma unroll
            for (int q = 0; q < D2; ++q) a0[l][q] = 0.f;
        int local_abort = 0;
        for (int c = 0; c < nch; ++c) {
            const int st = c & 1, c0 = c * PC;
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            if (bar_or_id(1, NPROD, local_abort | abort_s)) break;   // also: chunk c's tangents visible
            if (c + 1 < nch) prefetch(c + 1, (c + 1) & 1);
            // F_mu = I + sum_k mu_k Gmu_k at the chunk's points (zeros for absent instances and points)
            const float *gm = Gm0 + (size_t)(c & 1) * GM_FLOATS;
            for (int e = tid; e < S * PC * D2; e += NPROD) {
                const int s = e / (PC * D2), rem = e - s * (PC * D2);
                const int pt = rem / D2, q = rem - pt * D2;
                float v = 0.f;   // F_mu in FP32: it only enters the FP32 Ahat
                if (bI[s] >= 0 && c0 + pt < m) {
                    v = (q % 4 == 0) ? 1.f : 0.f;
                    for (int k = 0; k < np; ++k) v = fmaf(muS[s][k], gm[(q * np + k) * PC + pt], v);
                }
                Fms[(s * PC + pt) * D2 + q] = v;
            }
            bar_or_id(2, NPROD, 0);
            const uint32_t par = (uint32_t)(c >> 1) & 1u;
            if (!mbar_wait(&bar_full[st], par, &abort_s)) { local_abort = 1; continue; }
            if (c >= 2 && !mbar_wait(&bar_mma[st], par ^ 1u, &abort_s)) { local_abort = 1; continue; }
            const float *as = As0 + (size_t)(c & 1) * AS_FLOATS;
            unsigned char *Ahi = a_tile(st, 0), *Alo = a_tile(st, 1);
            // Ahat_{s,pt}[ar][(k,l)] = sum_q At[ar][(k,q)] F_mu[l][q], ar = 0..8, l = 0..2, stored rounded
            // to TF32 hi and lo; A0[(ia, jb)][(k,l)] += sum_r F_mu[jb][r] Ahat[(ia, r)][(k,l)] in FP32
            if (prod_row) {
                const float *fm = Fms + (ps * PC + ppt) * D2;
                float f[D2];
#pragma unroll
                for (int q = 0; q < D2; ++q) f[q] = fm[q];
                const float *a = as + (size_t)ps * D4 * PC + ppt;
                float y[D][D2];
#pragma unroll
                for (int ar = 0; ar < D2; ++ar) {
                    const int ce = ar * D2 + pk * D;
                    const float t0 = a[ce * PC], t1 = a[(ce + 1) * PC], t2 = a[(ce + 2) * PC];
#pragma unroll
                    for (int l = 0; l < D; ++l) y[l][ar] = fmaf(t2, f[l * D + 2], fmaf(t1, f[l * D + 1], t0 * f[l * D]));
                }
#pragma unroll
                for (int l = 0; l < D; ++l) {
#pragma unroll
                    for (int ia = 0; ia < D; ++ia)
#pragma unroll
                        for (int jb = 0; jb < D; ++jb)
                            a0[l][ia * D + jb] = fmaf(f[jb * D + 2], y[l][ia * D + 2],
                                                      fmaf(f[jb * D + 1], y[l][ia * D + 1],
                                                           fmaf(f[jb * D], y[l][ia * D], a0[l][ia * D + jb])));
                    uint32_t h[12], lo[12];
#pragma unroll
                    for (int q = 0; q < 12; ++q) {
                        h[q] = q < D2 ? tf32_bits(y[l][q < D2 ? q : 0]) : 0u;
                        lo[q] = q < D2 ? tf32_bits(y[l][q < D2 ? q : 0] - __uint_as_float(h[q])) : 0u;
                    }
                    const int r = ps * D2 + pk * D + l;
                    const size_t rb = (size_t)(r >> 3) * SBO_A + (size_t)(r & 7) * 16;
#pragma unroll
                    for (int u = 0; u < 3; ++u) {
                        *reinterpret_cast<uint4 *>(Ahi + rb + (size_t)(3 * ppt + u) * 128) =
                            make_uint4(h[4 * u], h[4 * u + 1], h[4 * u + 2], h[4 * u + 3]);
                        *reinterpret_cast<uint4 *>(Alo + rb + (size_t)(3 * ppt + u) * 128) =
                            make_uint4(lo[4 * u], lo[4 * u + 1], lo[4 * u + 2], lo[4 * u + 3]);
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&bar_afull[st]);
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        // A0: the four point partial sums of each row added in a fixed order (the tangent staging
        // area is free once every producer has left the loop)
        const int quit = bar_or_id(1, NPROD, local_abort | abort_s);
        float *red = As0;                                    // [PC][S * 9][9]
        if (prod_row)
#pragma unroll
            for (int l = 0; l < D; ++l)
#pragma unroll
                for (int q = 0; q < D2; ++q) red[((size_t)ppt * S * D2 + ps * D2 + pk * D + l) * D2 + q] = a0[l][q];
        bar_or_id(2, NPROD, 0);
        if (!quit)
            for (int e = tid; e < S * D2 * D2; e += NPROD) {
                const int row = e / D2, q = e - row * D2;        // row = s * 9 + kl
                const int s = row / D2, kl = row - s * D2;
                if (bI[s] < 0) continue;
                double v = 0.0;
#pragma unroll
                for (int pt = 0; pt < PC; ++pt) v += f2d_exact(red[((size_t)pt * S * D2 + row) * D2 + q]);
                Bsum[(size_t)bI[s] * (n * D2 + D4) + (size_t)n * D2 + q * D2 + kl] = v;
            }
    } else if (lane == 0) {
        // ------------------------------------------------------------- control thread
        uint32_t copy_pending = 0, copy_par = 0;
        int mma_pending = 0;
        uint32_t mma_par = 0;
        int mma_stage = 0;
        auto issue_copies = [&](int c) {
            const int st = c & 1;
            mbar_expect_tx(&bar_full[st], 2u * B_BYTES);
            bulk_g2s(b_tile(st, 0), img + L.tf_hi + (size_t)c * B_BYTES, B_BYTES, &bar_full[st]);
            bulk_g2s(b_tile(st, 1), img + L.tf_lo + (size_t)c * B_BYTES, B_BYTES, &bar_full[st]);
            copy_pending |= 1u << st;
            copy_par = (copy_par & ~(1u << st)) | (((uint32_t)(c >> 1) & 1u) << st);
        };
        issue_copies(0);
        if (nch > 1) issue_copies(1);
        for (int c = 0; c < nch; ++c) {
            const int st = c & 1;
            const uint32_t par = (uint32_t)(c >> 1) & 1u;
            if (!mbar_wait(&bar_full[st], par, &abort_s)) break;
            copy_pending &= ~(1u << st);
            if (!mbar_wait(&bar_afull[st], par, &abort_s)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ah = smem_u32(a_tile(st, 0)), al = smem_u32(a_tile(st, 1));
            const uint32_t bh = smem_u32(b_tile(st, 0)), bl = smem_u32(b_tile(st, 1));
            const uint32_t dh = tmem + (uint32_t)((c % NH) * 64), dl = tmem + (uint32_t)(NH * 64);
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                const uint64_t adh = make_desc(ah + k * 256, 128, SBO_A);
                const uint64_t bdh = make_desc(bh + k * 256, 128, SBO_B);
                mma_tf32(dh, adh, bdh, IDESC, (c >= NH || k > 0) ? 1u : 0u);
                mma_tf32(dl, make_desc(al + k * 256, 128, SBO_A), bdh, IDESC, (c > 0 || k > 0) ? 1u : 0u);
                mma_tf32(dl, adh, make_desc(bl + k * 256, 128, SBO_B), IDESC, 1u);
            }
            mma_commit(&bar_mma[st]);
            mma_pending = 1;
            mma_par = par;
            mma_stage = st;
            if (c + 2 < nch) {
                if (!mbar_wait(&bar_mma[st], par, &abort_s)) break;
                issue_copies(c + 2);
            }
        }
        if (mma_pending && !mbar_wait(&bar_mma[mma_stage], mma_par, &abort_s)) mbar_drain(&bar_mma[mma_stage], mma_par);
        for (int st = 0; st < 2; ++st)
            if ((copy_pending >> st) & 1u) mbar_drain(&bar_full[st], (copy_par >> st) & 1u);
        if (abort_s && err_flag) atomicExch(err_flag, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!abort_s && tid < NPROD) {
        // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (rows s * 9 + kl), columns
        // 32 (w / 4) .. + 31 (basis index l); accumulators added in FP32 in a fixed order
        const int row = (warp & 3) * 32 + lane;
        const int s = row / D2, kl = row - s * D2;
        const bool ok = s < S && bI[s] >= 0;
        double *Bb = ok ? Bsum + (size_t)bI[s] * (n * D2 + D4) + kl : nullptr;
        const int nh_used = nch < NH ? nch : NH;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const int c0 = (warp >> 2) * 32 + h * 16;
            float acc[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) acc[q] = 0.f;
#pragma unroll 1
            for (int ai = 0; ai < NACC; ++ai) {
                if (ai >= nh_used && ai < NH) continue;
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(ai * 64 + c0), r);
                tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[q] += __uint_as_float(r[q]);
            }
            if (ok)
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (c0 + q < n) Bb[(size_t)(c0 + q) * D2] = f2d_exact(acc[q]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == NPROD / 32) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

// ------------------------------------------------------------------------ host side

size_t tc3_image_bytes(int m) { return tc3::img_layout(m).total; }

// B-operand images of G[m][9][n] (n <= 64) and the zero-padded FP32 basis chunks, one buffer
void tc3_build_images(int n, int m, const double *G, unsigned char *img) {
    using namespace tc3;
    const ImgLayout L = img_layout(m);
    memset(img, 0, L.total);
    float *g32 = reinterpret_cast<float *>(img + L.g32);
    for (int i = 0; i < m; ++i)
        for (int q = 0; q < D2; ++q)
            for (int j = 0; j < n; ++j) g32[((size_t)i * D2 + q) * NCOLS + j] = (float)G[((size_t)i * D2 + q) * n + j];
    for (int c = 0; c < L.nch; ++c)
        for (int l = 0; l < n; ++l)
            for (int pt = 0; pt < PC; ++pt) {
                const int i = c * PC + pt;
                if (i >= m) continue;
                for (int q = 0; q < D2; ++q) {
                    const double g = G[((size_t)i * D2 + q) * n + l];
                    {   // BF16, KP = 16
                        using C1 = Cfg<1>;
                        const int k = pt * C1::KP + q;
                        const size_t off = (size_t)c * C1::B_BYTES + (size_t)(l >> 3) * C1::SBO_B + (size_t)(k >> 3) * 128 +
                                           (size_t)(l & 7) * 16 + (size_t)(k & 7) * 2;
                        const __nv_bfloat16 h = __float2bfloat16((float)g);
                        memcpy(img + L.bf16 + off, &h, 2);
                    }
                    {   // TF32 hi / lo, KP = 12
                        using C2 = Cfg<2>;
                        const int k = pt * C2::KP + q;
                        const size_t off = (size_t)c * C2::B_BYTES + (size_t)(l >> 3) * C2::SBO_B + (size_t)(k >> 2) * 128 +
                                           (size_t)(l & 7) * 16 + (size_t)(k & 3) * 4;
                        const float f = (float)g;
                        const float hi = tf32_round_host(f);
                        const float lo = tf32_round_host(f - hi);
                        memcpy(img + L.tf_hi + off, &hi, 4);
                        memcpy(img + L.tf_lo + off, &lo, 4);
                    }
                    {   // Y-MMA A operand: point pt of the chunk = point s of pair pt / 2
                        const int pp = pt >> 1, sp = pt & 1;
                        const int r = sp * 64 + l, k = sp * 12 + q;
                        const size_t off = (size_t)(c * 2 + pp) * AY_BYTES + (size_t)(r >> 3) * AY_SBO + (size_t)(k >> 2) * 128 +
                                           (size_t)(r & 7) * 16 + (size_t)(k & 3) * 4;
                        const float t = tf32_round_host((float)g);
                        memcpy(img + L.ay + off, &t, 4);
                    }
                }
            }
}

template <int MODE>
static int launch_tc3_t(const Model &M, Batch Bt, const unsigned char *img, int *err, int sel, cudaStream_t s) {
    using C = tc3::Cfg<MODE>;
    if (M.d != 3 || M.n > tc3::NCOLS || (M.mA & 3)) return -1;
    cudaFuncSetAttribute(k_assemble_tc3<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    const int grid = (int)((Bt.B + C::NI - 1) / C::NI);
    k_assemble_tc3<MODE><<<grid, C::THREADS, C::SMEM, s>>>(M, Bt, img, err, sel);
    return 0;
}

static int launch_tc4(const Model &M, Batch Bt, const unsigned char *img, int *err, int sel, cudaStream_t s) {
    if (M.d != 3 || M.n > tc3::NCOLS || (M.mA & 3)) return -1;
    cudaFuncSetAttribute(k_assemble_tc4, cudaFuncAttributeMaxDynamicSharedMemorySize, tc4::SMEM);
    const int grid = (int)((Bt.B + tc4::NI - 1) / tc4::NI);
    k_assemble_tc4<<<grid, tc4::THREADS, tc4::SMEM, s>>>(M, Bt, img, err, sel);
    return 0;
}

// B_b = sum_i G_i^T Ahat_i [n][9] of the listed (converged) instances on the tensor cores
int launch_abar_tc3(const Model &M, Batch Bt, const unsigned char *img, double *Bsum, int *err, cudaStream_t s) {
    if (M.d != 3 || M.n > tc3::NCOLS || (M.mA & 3) || !Bsum) return -1;
    cudaFuncSetAttribute(k_abar_tc3, cudaFuncAttributeMaxDynamicSharedMemorySize, tca::SMEM);
    const int grid = (int)((Bt.B + tca::S - 1) / tca::S);
    k_abar_tc3<<<grid, tca::THREADS, tca::SMEM, s>>>(M, Bt, img, Bsum, err);
    return 0;
}

// mode 1 BF16, 3 TF32 split (FP32-accurate), 4 TF32 with Y on the tensor cores (k_assemble_tc4;
// it supersedes the TF32 variant of k_assemble_tc3 with Y on the CUDA cores, MODE 2, which is
// not instantiated); sel 0 = all listed instances, 1 = those without, 2 = those with the
// accurate-stiffness flag (Ctl::acc_k)
int launch_tc3(int mode, const Model &M, Batch Bt, const unsigned char *img, int *err, int sel, cudaStream_t s) {
    return mode == 1 ? launch_tc3_t<1>(M, Bt, img, err, sel, s)
         : mode == 3 ? launch_tc3_t<3>(M, Bt, img, err, sel, s)
         : mode == 4 ? launch_tc4(M, Bt, img, err, sel, s) : -1;
}

}  // namespace podecm
