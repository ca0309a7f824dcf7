// Reduced stiffness of the 2D model, K_b = sum_i G_i^T At_i G_i (Eq. stiffnessmatrix_ecm), on the
// 5th-generation tensor cores (tcgen05.mma, FP32 accumulation in tensor memory), with the
// instances of a CTA packed along the MMA's M dimension; and the residual r = sum_i G_i^T v_i
// (Eq. residual_ecm) in FP64 or double-float arithmetic.
//
// Formulation: K_b = Y_b^T G with Y_b[(i, c)][j] = sum_q At_i[q][c] G_i[q][j], so that
// K[j][l] = sum_i sum_{q,c} G_i[q][j] At_i[q][c] G_i[c][l] (K itself, not K^T, when the FP32
// tangent is not exactly symmetric).  A CTA holds S = min(16, floor(128 / n)) instances b_s in
// consecutive n-row slots of one 128-row accumulator:
//   D[128 x NB] += A[128 x K] B[NB x K]^T,   A row s n + j = row j of Y_{b_s}^T,
//   B row l = G[:, :, l],  NB = n rounded up to 16,
// so every MMA serves all S instances with the shared basis tile as its B operand (at n = 24,
// 5 x 24 of the 128 rows carry work).  K runs over chunks of PC cubature points; each point's 4
// components fill 16 bytes of a row in TF32 (PC = 8), two points do in BF16 (PC = 16), so a chunk
// is 128 bytes of K per row in every mode: 8 core matrices, 4 MMAs (K = 8 TF32 / 16 BF16).
//
// Roles: 8 producer warps (256 threads in groups of 8: group item (unit u, instance s, block of
// 8 rows), lane = row j of the block) read the tangent of point(s) u of instance s from a
// cp.async-staged copy (the next chunk's copy overlaps this chunk's work), form Y for row j from
// the FP32 basis chunk, round it and store 16 bytes per row and unit; one control thread issues the bulk copy (cp.async.bulk, the
// TMA engine) of the chunk's image (FP32 basis, pre-arranged B tile(s)) into a 2-stage ring, then,
// once the producers have arrived on the stage's mbarrier, the chunk's MMAs and one commit.
// MODE 1 = BF16 operands, 2 = TF32, 3 = TF32 split: A = A_hi + A_lo, B = B_hi + B_lo with
// A_hi = tf32(A), A_lo = tf32(A - A_hi); the MMAs form A_hi B_hi + A_lo B_hi + A_hi B_lo, an
// FP32-accurate product (the dropped A_lo B_lo term is below FP32 rounding).
// Accumulation: the tensor core adds into FP32 with truncation, so chunk c goes to accumulator
// c % NH (NH of them side by side in tensor memory), the split's small terms to one more, and the
// epilogue adds the accumulators: the chains stay a few MMAs long.
// Every wait is bounded by the wall clock (1 s); on timeout the CTA records an error, stops
// issuing work, waits (bounded) for its own copies and MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <algorithm>
#include <cstdint>
#include <cstring>

#include "kernels.cuh"
#include "tcgen05.cuh"

namespace podecm {

namespace tcp {

constexpr int D2 = 4, D4 = 16;
constexpr int MROWS = 128;            // MMA M
constexpr int MAX_S = 16;             // instances per CTA
constexpr int NU = 8;                 // 16-byte K units per chunk and row
constexpr int SBO_A = NU * 128;       // A and B tiles: 8-row groups 1024 bytes apart
constexpr int SBO_B = NU * 128;
constexpr int A_BYTES = MROWS / 8 * SBO_A;
constexpr int NK = 4;                 // MMAs per chunk (32 bytes of K each)
constexpr int NPROD = 256;
constexpr int THREADS = NPROD + 32;
constexpr int MAXIT = 8;              // producer items per 8-lane group and chunk (at most 7 for n <= 64)

template <int MODE>
struct Cfg {
    static constexpr bool SPLIT = MODE == 3;
    static constexpr int PU = MODE == 1 ? 2 : 1;          // points per 16-byte unit
    static constexpr int PC = NU * PU;                    // points per chunk
    static constexpr int NAT = SPLIT ? 2 : 1;             // A tiles per stage
    static constexpr int ASTR = D4 * PC + 4;              // staged tangent floats per instance (the
                                                          // 4-float pad spreads instances over banks)
    static constexpr int TMEM_COLS = SPLIT ? 256 : 128;
};

// launch geometry of a model (host-computed, passed by value)
struct Geom {
    int S, NB, nch;                 // instances per CTA, MMA N, chunks
    int g32_bytes, b_bytes;         // FP32 basis chunk [PC][4][NB]; one B tile (NB rows x 128 bytes)
    int chunk_bytes, copy_bytes;    // image bytes per chunk; bytes one CTA copies per chunk
    int stage_bytes, as_bytes, smem;
    int AS, NACC, NH;               // accumulator stride (tensor-memory columns), count, hi count
};

template <int MODE>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if (MODE == 1) tcx::mma_f16(d, a, b, idesc, acc);
    else tcx::mma_tf32(d, a, b, idesc, acc);
}

}  // namespace tcp

// sel: 0 every listed instance, 1 those without, 2 those with the accurate-stiffness flag
template <int MODE>
__global__ void __launch_bounds__(tcp::THREADS, 1)
    k_assemble_tcp(Model M, Batch Bt, const unsigned char *__restrict__ img, tcp::Geom g, int *err_flag, int sel) {
    using namespace tcx;
    using namespace tcp;
    using C = Cfg<MODE>;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar_full[2], bar_afull[2], bar_mma[2];
    __shared__ uint32_t tmem_base;
    __shared__ int64_t bI[MAX_S];
    __shared__ volatile int abort_s;
    __shared__ int n_sel;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int n_act = Bt.counts[0];
    const int S = g.S;
    const int p0 = S * blockIdx.x;
    if (p0 >= n_act) return;
    const int n = M.n, m = M.m, mA = M.mA, NB = g.NB, nch = g.nch;
    const float *At = reinterpret_cast<const float *>(Bt.At);
    auto a_tile = [&](int st, int t) { return smem + (size_t)st * g.stage_bytes + (size_t)t * A_BYTES; };
    auto img_tile = [&](int st) { return smem + (size_t)st * g.stage_bytes + (size_t)C::NAT * A_BYTES; };
    // staged tangents of chunk c at As0 + (c & 1) * as_floats (arithmetic, so that no pointer array
    // lands in local memory)
    float *const As0 = reinterpret_cast<float *>(smem + 2 * (size_t)g.stage_bytes);
    const int as_floats = g.as_bytes / 4;

    if (tid == 0) n_sel = 0;
    __syncthreads();
    if (tid < S) {
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
    if (warp == NPROD / 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(C::TMEM_COLS));
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
    // rows S n .. 127 of the A tiles are never produced: zero them once
    const int pad = MROWS - S * n;
    for (int e = tid; e < 2 * C::NAT * pad * NU; e += THREADS) {
        const int u = e % NU, rest = e / NU;
        const int r = S * n + rest % pad, t = rest / pad;
        *reinterpret_cast<uint4 *>(a_tile(t / C::NAT, t % C::NAT) + (size_t)(r >> 3) * SBO_A + u * 128 + (r & 7) * 16) =
            make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (tid < NPROD) {
        // ------------------------------------------------------------------ producers
        const int grp = tid >> 3, j8 = tid & 7;
        // this thread's items (unit u, instance s, block of 8 rows; row blocks fastest, so that the
        // groups of a warp mostly share one tangent and read distinct basis columns), decoded
        // once: staged-tangent index, basis index and A-tile byte offset of row s n + j
        const int NJB = (n + 7) >> 3, n_items = S * NU * NJB;
        int it_a[MAXIT], it_g[MAXIT], it_st[MAXIT];
        uint32_t it_live = 0, it_row = 0;
#pragma unroll
        for (int k = 0; k < MAXIT; ++k) {
            const int it = grp + k * (NPROD / 8);
            const int jb = it % NJB, rest = it / NJB;
            const int s = rest % S, u = rest / S;
            const int j = jb * 8 + j8, r = s * n + j;
            it_a[k] = s * C::ASTR + u * C::PU;
            it_g[k] = u * C::PU * D2 * NB + j;
            it_st[k] = (r >> 3) * SBO_A + u * 128 + (r & 7) * 16;
            if (it < n_items) it_live |= 1u << k;             // uniform over two warps
            if (it < n_items && j < n) it_row |= 1u << k;
        }
        // tangent rows (instance s, component e) of chunk c: PC / 4 pieces of 4 points each; whole
        // pieces by cp.async, the pieces of absent instances and the points past m as zeros
        auto prefetch = [&](int c, int buf) {
            constexpr int PIECES = C::PC / 4;
            const int c0 = c * C::PC;
            for (int e = tid; e < S * D4 * PIECES; e += NPROD) {
                const int h = e % PIECES, row = e / PIECES;
                const int s = row / D4, comp = row - s * D4;
                const int64_t b = bI[s];
                const int p0 = c0 + 4 * h;
                float *dst = As0 + buf * as_floats + s * C::ASTR + comp * C::PC + 4 * h;
                if (b >= 0 && p0 + 4 <= m) {
                    cp_async16(dst, At + ((size_t)b * D4 + comp) * mA + p0);
                } else {
                    const float *src = At + ((size_t)(b >= 0 ? b : 0) * D4 + comp) * mA + p0;
                    float4 v;
                    v.x = (b >= 0 && p0 + 0 < m) ? src[0] : 0.f;
                    v.y = (b >= 0 && p0 + 1 < m) ? src[1] : 0.f;
                    v.z = (b >= 0 && p0 + 2 < m) ? src[2] : 0.f;
                    v.w = (b >= 0 && p0 + 3 < m) ? src[3] : 0.f;
                    *reinterpret_cast<float4 *>(dst) = v;
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        prefetch(0, 0);
        int local_abort = 0;
        for (int c = 0; c < nch; ++c) {
            const int st = c & 1;
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            if (bar_or(NPROD, local_abort | abort_s)) break;   // also: chunk c's tangents visible
            if (c + 1 < nch) prefetch(c + 1, (c + 1) & 1);
            const uint32_t par = (uint32_t)(c >> 1) & 1u;
            if (!mbar_wait(&bar_full[st], par, &abort_s)) { local_abort = 1; continue; }
            if (c >= 2 && !mbar_wait(&bar_mma[st], par ^ 1u, &abort_s)) { local_abort = 1; continue; }
            const float *Gs = reinterpret_cast<const float *>(img_tile(st));
            const float *Ab = As0 + (c & 1) * as_floats;
            unsigned char *Ahi = a_tile(st, 0);
            unsigned char *Alo = a_tile(st, C::NAT - 1);
#pragma unroll
            for (int k = 0; k < MAXIT; ++k) {
                if (!((it_live >> k) & 1u)) break;
                float a[C::PU][D4];
#pragma unroll
                for (int p = 0; p < C::PU; ++p)
#pragma unroll
                    for (int e = 0; e < D4; ++e) a[p][e] = Ab[it_a[k] + e * C::PC + p];
                if ((it_row >> k) & 1u) {
                    float y[C::PU][D2];
#pragma unroll
                    for (int p = 0; p < C::PU; ++p) {
                        const float *gp = Gs + it_g[k] + p * D2 * NB;
                        // Y row j of the point: y[c] = sum_q At[q][c] G[q][j], packed FP32 pairs
                        float2 y01 = make_float2(0.f, 0.f), y23 = make_float2(0.f, 0.f);
#pragma unroll
                        for (int q = 0; q < D2; ++q) {
                            const float gv = gp[q * NB];
                            const float2 gg = make_float2(gv, gv);
                            y01 = __ffma2_rn(make_float2(a[p][q * D2 + 0], a[p][q * D2 + 1]), gg, y01);
                            y23 = __ffma2_rn(make_float2(a[p][q * D2 + 2], a[p][q * D2 + 3]), gg, y23);
                        }
                        y[p][0] = y01.x; y[p][1] = y01.y; y[p][2] = y23.x; y[p][3] = y23.y;
                    }
                    if (MODE == 1) {
                        const uint4 v = make_uint4(pack_bf16(y[0][0], y[0][1]), pack_bf16(y[0][2], y[0][3]),
                                                   pack_bf16(y[C::PU - 1][0], y[C::PU - 1][1]),
                                                   pack_bf16(y[C::PU - 1][2], y[C::PU - 1][3]));
                        *reinterpret_cast<uint4 *>(Ahi + it_st[k]) = v;
                    } else {
                        uint32_t h[D2];
#pragma unroll
                        for (int cc = 0; cc < D2; ++cc) h[cc] = tf32_bits(y[0][cc]);
                        *reinterpret_cast<uint4 *>(Ahi + it_st[k]) = make_uint4(h[0], h[1], h[2], h[3]);
                        if (C::SPLIT) {
                            uint32_t l[D2];
#pragma unroll
                            for (int cc = 0; cc < D2; ++cc) l[cc] = tf32_bits(y[0][cc] - __uint_as_float(h[cc]));
                            *reinterpret_cast<uint4 *>(Alo + it_st[k]) = make_uint4(l[0], l[1], l[2], l[3]);
                        }
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&bar_afull[st]);
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
    } else if (tid == NPROD) {
        // ------------------------------------------------------------- control thread
        uint32_t copy_pending = 0, copy_par = 0;   // bit st: a copy into stage st in flight / its parity
        int mma_pending = 0;
        uint32_t mma_par = 0;
        int mma_stage = 0;
        const uint32_t idesc = make_idesc(MODE == 1 ? 1u : 2u, MROWS, NB);
        auto issue_copies = [&](int c) {
            const int st = c & 1;
            mbar_expect_tx(&bar_full[st], (uint32_t)g.copy_bytes);
            bulk_g2s(img_tile(st), img + (size_t)c * g.chunk_bytes, (uint32_t)g.copy_bytes, &bar_full[st]);
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
            const uint32_t ah = smem_u32(a_tile(st, 0)), al = smem_u32(a_tile(st, C::NAT - 1));
            const uint32_t bh = smem_u32(img_tile(st) + g.g32_bytes), bl = bh + (uint32_t)g.b_bytes;
            const uint32_t dh = tmem + (uint32_t)((c % g.NH) * g.AS), dl = tmem + (uint32_t)(g.NH * g.AS);
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                const uint64_t adh = make_desc(ah + k * 256, 128, SBO_A);
                const uint64_t bdh = make_desc(bh + k * 256, 128, SBO_B);
                tcp::mma<MODE>(dh, adh, bdh, idesc, (c >= g.NH || k > 0) ? 1u : 0u);
                if (C::SPLIT) {
                    tcp::mma<MODE>(dl, make_desc(al + k * 256, 128, SBO_A), bdh, idesc, (c > 0 || k > 0) ? 1u : 0u);
                    tcp::mma<MODE>(dl, adh, make_desc(bl + k * 256, 128, SBO_B), idesc, 1u);
                }
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
        // drain: the last commit covers every MMA issued before it; outstanding copies must land
        if (mma_pending && !mbar_wait(&bar_mma[mma_stage], mma_par, &abort_s)) mbar_drain(&bar_mma[mma_stage], mma_par);
        for (int st = 0; st < 2; ++st)
            if ((copy_pending >> st) & 1u) mbar_drain(&bar_full[st], (copy_par >> st) & 1u);
        if (abort_s && err_flag) atomicExch(err_flag, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!abort_s && tid < NPROD) {
        // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (accumulator rows s n + j)
        // and the 16-column groups w / 4, w / 4 + 2, ...; the accumulators are added in FP32 in a
        // fixed order (the FP64 pipe runs at 1/64 of the FP32 rate) and widened exactly
        const int row = (warp & 3) * 32 + (tid & 31);
        const int s = row / n, j = row - s * n;
        const bool ok = s < S && bI[s] >= 0;
        double *Kb = ok ? Bt.K + (size_t)bI[s] * n * n + (size_t)j * n : nullptr;
        const int nh_used = nch < g.NH ? nch : g.NH;
        for (int c16 = warp >> 2; c16 < NB / 16; c16 += NPROD / 128) {
            float acc[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) acc[q] = 0.f;
            for (int ai = 0; ai < g.NACC; ++ai) {
                if (ai >= nh_used && ai < g.NH) continue;   // accumulator never written
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(ai * g.AS + c16 * 16), r);
                tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[q] += __uint_as_float(r[q]);
            }
            if (ok)
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (c16 * 16 + q < n) Kb[c16 * 16 + q] = f2d_exact(acc[q]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == NPROD / 32) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::TMEM_COLS));
    }
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


// ---------------------------------------------------------------- Abar sums on the tensor cores (2D)
// k_abar_tcp: the 2D counterpart of k_abar_tc3.  For the converged instances B_b = sum_i G_i^T
// Ahat_i (n x 4) and A0_b (16), Ahat_i[ar][(k,l)] = sum_s At_i[ar][(k,s)] F_mu,i[l][s], FP32-accurate
// by the TF32 hi/lo split.  B_b^T = Ahat_b^T G with 32 instances packed along M (rows (s, kl),
// all 128 used), N = n rounded up to 16, K = (point, component) in the chunks of 8 points of the
// packed stiffness kernel's TF32 image of G (its B operand here too).  Producer thread (point,
// instance, k) forms the rows (s, 2k + l), l = 0, 1, and accumulates A0 in FP32; the control
// thread copies the chunk's B tiles (one bulk copy of hi and lo) and issues 12 MMAs per chunk.
// Output Bsum[b] = [B_b (n x 4) | A0_b (16)].  Every wait is bounded (1 s; error flag, drain).
namespace tca2 {
constexpr int D = 2, D2 = 4, D4 = 16;
constexpr int S = 32;                              // instances per CTA (32 x 4 = 128 rows)
constexpr int PC = 8;                              // points per chunk (the TF32 image's chunks)
constexpr int NPROD = 256, THREADS = NPROD + 32;
constexpr int A_BYTES = tcp::A_BYTES;              // 128 rows x 8 units of 16 bytes
constexpr int AS_FLOATS = S * D4 * PC;             // staged tangents [S][16][8]
constexpr int FM_FLOATS = S * PC * D2;             // F_mu [S][8][4]
constexpr int GM_FLOATS = D2 * MAX_NPAR * PC;      // geometric-map gradients of a chunk
}  // namespace tca2

__global__ void __launch_bounds__(tca2::THREADS, 1)
    k_abar_tcp(Model M, Batch Bt, const unsigned char *__restrict__ img, tcp::Geom g, double *__restrict__ Bsum,
               int *err_flag) {
    using namespace tcx;
    using namespace tca2;
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
    const int n = M.n, m = M.m, mA = M.mA, np = M.n_par, NB = g.NB, nch = g.nch;
    const float *At = reinterpret_cast<const float *>(Bt.At);
    const int stage = 2 * A_BYTES + 2 * g.b_bytes;
    auto a_tile = [&](int st, int t) { return smem + (size_t)st * stage + (size_t)t * A_BYTES; };
    auto b_tile = [&](int st) { return smem + (size_t)st * stage + 2 * (size_t)A_BYTES; };   // hi, then lo
    float *const As0 = reinterpret_cast<float *>(smem + 2 * (size_t)stage);   // buffer t at As0 + t * AS_FLOATS
    float *const Fms = As0 + 2 * AS_FLOATS;
    float *const Gm0 = Fms + FM_FLOATS;                                         // buffer t at Gm0 + t * GM_FLOATS

    if (tid < S) bI[tid] = (p0 + tid < n_act) ? (int64_t)Bt.list[p0 + tid] : -1;
    for (int e = tid; e < S * np; e += THREADS) {
        const int s = e / np, k = e - s * np;
        muS[s][k] = (p0 + s < n_act) ? to_tangent<float>(Bt.mu[(int64_t)Bt.list[p0 + s] * np + k]) : 0.f;
    }
    if (warp == NPROD / 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(256));
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
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;

    if (tid < NPROD) {
        // ------------------------------------------------------------------ producers
        // tangent rows (instance s, component ce) of chunk c: two 16-byte pieces of 4 points (zeros
        // for absent instances and points past m), and the chunk's geometric-map gradients
        auto prefetch = [&](int c, int buf) {
            const int c0 = c * PC;
            for (int e = tid; e < S * D4 * 2; e += NPROD) {
                const int h = e & 1, row = e >> 1;
                const int s = row / D4, ce = row - s * D4;
                const int64_t b = bI[s];
                const int q0 = c0 + 4 * h;
                float *dst = As0 + (size_t)buf * AS_FLOATS + (size_t)row * PC + 4 * h;
                if (b >= 0 && q0 + 4 <= m) {
                    cp_async16(dst, At + ((size_t)b * D4 + ce) * mA + q0);
                } else {
                    const float *src = At + ((size_t)(b >= 0 ? b : 0) * D4 + ce) * mA + q0;
                    float4 v;
                    v.x = (b >= 0 && q0 + 0 < m) ? src[0] : 0.f;
                    v.y = (b >= 0 && q0 + 1 < m) ? src[1] : 0.f;
                    v.z = (b >= 0 && q0 + 2 < m) ? src[2] : 0.f;
                    v.w = (b >= 0 && q0 + 3 < m) ? src[3] : 0.f;
                    *reinterpret_cast<float4 *>(dst) = v;
                }
            }
            for (int e = tid; e < D2 * np * PC; e += NPROD) {
                const int qk = e / PC, pt = e - qk * PC;
                Gm0[(size_t)buf * GM_FLOATS + e] = (c0 + pt < m) ? to_tangent<float>(M.Gmu_T[(size_t)qk * m + c0 + pt]) : 0.f;
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        };
        prefetch(0, 0);
        // thread (point pt, instance s, k): rows (s, 2 k + l), l = 0, 1; two such items per thread
        float a0[2][D][D2];
#pragma unroll
        for (int t = 0; t < 2; ++t)
#pragma unroll
            for (int l = 0; l < D; ++l)
#pragma unroll
                for (int q = 0; q < D2; ++q) a0[t][l][q] = 0.f;
        int local_abort = 0;
        for (int c = 0; c < nch; ++c) {
            const int st = c & 1, c0 = c * PC;
            asm volatile("cp.async.wait_group 0;" ::: "memory");
            if (bar_or_id(1, NPROD, local_abort | abort_s)) break;   // also: chunk c's tangents visible
            if (c + 1 < nch) prefetch(c + 1, (c + 1) & 1);
            const float *gm = Gm0 + (size_t)(c & 1) * GM_FLOATS;
            for (int e = tid; e < S * PC * D2; e += NPROD) {
                const int s = e / (PC * D2), rem = e - s * (PC * D2);
                const int pt = rem / D2, q = rem - pt * D2;
                float v = 0.f;
                if (bI[s] >= 0 && c0 + pt < m) {
                    v = (q % 3 == 0) ? 1.f : 0.f;
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
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int it = tid + t * NPROD;                   // < PC * S * D = 512
                const int pt = it / (S * D), rest = it - pt * (S * D);
                const int s = rest / D, k = rest - s * D;
                const float *fm = Fms + (s * PC + pt) * D2;
                const float f0 = fm[0], f1 = fm[1], f2 = fm[2], f3 = fm[3];
                const float *a = as + (size_t)s * D4 * PC + pt;
                float y[D][D2];
#pragma unroll
                for (int ar = 0; ar < D2; ++ar) {
                    const int ce = ar * D2 + k * D;
                    const float t0 = a[ce * PC], t1 = a[(ce + 1) * PC];
                    y[0][ar] = fmaf(t1, f1, t0 * f0);
                    y[1][ar] = fmaf(t1, f3, t0 * f2);
                }
#pragma unroll
                for (int l = 0; l < D; ++l) {
#pragma unroll
                    for (int ia = 0; ia < D; ++ia)
#pragma unroll
                        for (int jb = 0; jb < D; ++jb)
                            a0[t][l][ia * D + jb] = fmaf(fm[jb * D + 1], y[l][ia * D + 1], fmaf(fm[jb * D], y[l][ia * D], a0[t][l][ia * D + jb]));
                    uint32_t h[D2], lo[D2];
#pragma unroll
                    for (int q = 0; q < D2; ++q) {
                        h[q] = tf32_bits(y[l][q]);
                        lo[q] = tf32_bits(y[l][q] - __uint_as_float(h[q]));
                    }
                    const int r = s * D2 + k * D + l;
                    const size_t off = (size_t)(r >> 3) * tcp::SBO_A + (size_t)pt * 128 + (size_t)(r & 7) * 16;
                    *reinterpret_cast<uint4 *>(Ahi + off) = make_uint4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<uint4 *>(Alo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&bar_afull[st]);
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        // A0: the eight point partial sums of each row added in a fixed order
        const int quit = bar_or_id(1, NPROD, local_abort | abort_s);
        float *red = As0;                                    // [PC][S * 4][4]
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int it = tid + t * NPROD;
            const int pt = it / (S * D), rest = it - pt * (S * D);
            const int s = rest / D, k = rest - s * D;
#pragma unroll
            for (int l = 0; l < D; ++l)
#pragma unroll
                for (int q = 0; q < D2; ++q) red[((size_t)pt * S * D2 + s * D2 + k * D + l) * D2 + q] = a0[t][l][q];
        }
        bar_or_id(2, NPROD, 0);
        if (!quit)
            for (int e = tid; e < S * D2 * D2; e += NPROD) {
                const int row = e / D2, q = e - row * D2;        // row = s * 4 + kl
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
        const uint32_t idesc = make_idesc(2u, tcp::MROWS, NB);
        auto issue_copies = [&](int c) {
            const int st = c & 1;
            mbar_expect_tx(&bar_full[st], 2u * g.b_bytes);
            bulk_g2s(b_tile(st), img + (size_t)c * g.chunk_bytes + g.g32_bytes, 2u * g.b_bytes, &bar_full[st]);
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
            const uint32_t bh = smem_u32(b_tile(st)), bl = bh + (uint32_t)g.b_bytes;
            const uint32_t dh = tmem + (uint32_t)((c % g.NH) * g.AS), dl = tmem + (uint32_t)(g.NH * g.AS);
#pragma unroll
            for (int k = 0; k < tcp::NK; ++k) {
                const uint64_t adh = make_desc(ah + k * 256, 128, tcp::SBO_A);
                const uint64_t bdh = make_desc(bh + k * 256, 128, tcp::SBO_B);
                mma_tf32(dh, adh, bdh, idesc, (c >= g.NH || k > 0) ? 1u : 0u);
                mma_tf32(dl, make_desc(al + k * 256, 128, tcp::SBO_A), bdh, idesc, (c > 0 || k > 0) ? 1u : 0u);
                mma_tf32(dl, adh, make_desc(bl + k * 256, 128, tcp::SBO_B), idesc, 1u);
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
        // epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (rows s * 4 + kl) and the
        // 16-column groups w / 4, w / 4 + 2, ...; accumulators added in FP32 in a fixed order
        const int row = (warp & 3) * 32 + lane;
        const int s = row / D2, kl = row - s * D2;
        const bool ok = bI[s] >= 0;
        double *Bb = ok ? Bsum + (size_t)bI[s] * (n * D2 + D4) + kl : nullptr;
        const int nh_used = nch < g.NH ? nch : g.NH;
        for (int c16 = warp >> 2; c16 < NB / 16; c16 += NPROD / 128) {
            float acc[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) acc[q] = 0.f;
            for (int ai = 0; ai < g.NACC; ++ai) {
                if (ai >= nh_used && ai < g.NH) continue;
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(ai * g.AS + c16 * 16), r);
                tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[q] += __uint_as_float(r[q]);
            }
            if (ok)
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (c16 * 16 + q < n) Bb[(size_t)(c16 * 16 + q) * D2] = f2d_exact(acc[q]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == NPROD / 32) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
    }
}

// ------------------------------------------------------------------------ host side

// geometry of the packed 2D kernel for a model (mode 1 BF16, 2 TF32, 3 TF32 split)
static tcp::Geom tcp_geom(int mode, int n, int m) {
    using namespace tcp;
    Geom g{};
    const bool bf = mode == 1, split = mode == 3;
    const int PC = bf ? 16 : 8;
    g.S = std::min(MAX_S, MROWS / n);
    g.NB = (n + 15) / 16 * 16;
    g.nch = (m + PC - 1) / PC;
    g.g32_bytes = PC * D2 * g.NB * 4;
    g.b_bytes = g.NB / 8 * SBO_B;
    g.chunk_bytes = g.g32_bytes + (bf ? 1 : 2) * g.b_bytes;
    g.copy_bytes = g.g32_bytes + (split ? 2 : 1) * g.b_bytes;
    g.stage_bytes = (split ? 2 : 1) * A_BYTES + (g.copy_bytes + 1023) / 1024 * 1024;
    g.as_bytes = g.S * (D4 * PC + 4) * 4;
    g.smem = 2 * g.stage_bytes + 2 * g.as_bytes;
    g.AS = g.NB <= 32 ? 32 : 64;
    g.NACC = (split ? 256 : 128) / g.AS;
    g.NH = g.NACC - (split ? 1 : 0);
    return g;
}

// bytes of the 2D tensor-core image of a model: fmt 1 BF16, 2 TF32 (hi and lo tiles)
size_t tc2_image_bytes(int fmt, int n, int m) {
    const tcp::Geom g = tcp_geom(fmt == 1 ? 1 : 3, n, m);
    return (size_t)g.nch * g.chunk_bytes;
}

// host: per chunk of PC points, the zero-padded FP32 basis [PC][4][NB] and the B-operand tile(s)
// of G[m][4][n] (n <= 64): row l = basis column l, K slot k = (point, component) of the chunk,
// canonical K-major layout; TF32 hi = tf32(g), lo = tf32(g - hi)
void tc2_build_image(int fmt, int n, int m, const double *G, unsigned char *img) {
    using namespace tcp;
    const tcp::Geom g = tcp_geom(fmt == 1 ? 1 : 3, n, m);
    const int PC = fmt == 1 ? 16 : 8;
    memset(img, 0, (size_t)g.nch * g.chunk_bytes);
    for (int c = 0; c < g.nch; ++c) {
        unsigned char *t = img + (size_t)c * g.chunk_bytes;
        for (int pt = 0; pt < PC; ++pt) {
            const int i = c * PC + pt;
            if (i >= m) continue;
            for (int q = 0; q < D2; ++q)
                for (int l = 0; l < n; ++l) {
                    const double v = G[((size_t)i * D2 + q) * n + l];
                    const float f = (float)v;
                    memcpy(t + ((size_t)(pt * D2 + q) * g.NB + l) * 4, &f, 4);
                    const int k = pt * D2 + q;
                    unsigned char *b = t + g.g32_bytes;
                    if (fmt == 1) {
                        const size_t off = (size_t)(l >> 3) * SBO_B + (size_t)(k >> 3) * 128 + (l & 7) * 16 + (k & 7) * 2;
                        const __nv_bfloat16 h = __float2bfloat16(f);
                        memcpy(b + off, &h, 2);
                    } else {
                        const size_t off = (size_t)(l >> 3) * SBO_B + (size_t)(k >> 2) * 128 + (l & 7) * 16 + (k & 3) * 4;
                        const float hi = tcx::tf32_round_host(f);
                        const float lo = tcx::tf32_round_host(f - hi);
                        memcpy(b + off, &hi, 4);
                        memcpy(b + g.b_bytes + off, &lo, 4);
                    }
                }
        }
    }
}

template <int MODE>
static int launch_tcp_t(const Model &M, Batch Bt, const unsigned char *img, int *err, int sel, cudaStream_t s) {
    if (M.d != 2 || M.n < 1 || M.n > 64 || (M.mA & 3)) return -1;
    const tcp::Geom g = tcp_geom(MODE, M.n, M.m);
    if (g.S * tcp::NU * ((M.n + 7) / 8) > tcp::MAXIT * (tcp::NPROD / 8)) return -1;
    cudaFuncSetAttribute(k_assemble_tcp<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, g.smem);
    const int grid = (int)((Bt.B + g.S - 1) / g.S);
    k_assemble_tcp<MODE><<<grid, tcp::THREADS, g.smem, s>>>(M, Bt, img, g, err, sel);
    return 0;
}

// B_b = sum_i G_i^T Ahat_i [n][4] and A0_b [16] of the listed (converged) 2D instances on the
// tensor cores, from the TF32 image (fmt 2) of the packed stiffness kernel
int launch_abar_tcp(const Model &M, Batch Bt, const unsigned char *img, double *Bsum, int *err, cudaStream_t s) {
    using namespace tca2;
    if (M.d != 2 || M.n < 1 || M.n > 64 || (M.mA & 3) || !Bsum || M.n_par > MAX_NPAR) return -1;
    const tcp::Geom g = tcp_geom(3, M.n, M.m);
    const int stage = 2 * A_BYTES + 2 * g.b_bytes;
    const int smem = 2 * stage + 2 * AS_FLOATS * 4 + FM_FLOATS * 4 + 2 * GM_FLOATS * 4;
    cudaFuncSetAttribute(k_abar_tcp, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    const int grid = (int)((Bt.B + S - 1) / S);
    k_abar_tcp<<<grid, THREADS, smem, s>>>(M, Bt, img, g, Bsum, err);
    return 0;
}

// 2D stiffness on the tensor cores: mode 1 BF16 and 2 TF32 (image fmt 1 / 2), 3 TF32 split
// (FP32-accurate, image fmt 2); sel as in k_assemble_tcp
int launch_tc2(int mode, const Model &M, Batch Bt, const unsigned char *img, int *err, int sel, cudaStream_t s) {
    return mode == 1 ? launch_tcp_t<1>(M, Bt, img, err, sel, s)
         : mode == 2 ? launch_tcp_t<2>(M, Bt, img, err, sel, s)
         : mode == 3 ? launch_tcp_t<3>(M, Bt, img, err, sel, s) : -1;
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


}  // namespace podecm
