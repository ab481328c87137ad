// Learned initialiser: a set encoder that maps a sample subset of a dataset
// to the starting hefts, means and variances of EM (in place of k-means
// seeding, which stays the fallback).  Network (row vectors, ReLU):
//   per point  x (D) -> Lp layers of width Hp           (weights W_l [out][in])
//   pool       mean over the P points of the last per-point activations
//   head       Lh layers of width Hh, then a linear layer to G (1 + 2D) outputs
//   outputs    a (G) -> hefts = softmax(a); m (G x D) -> means;
//              r (G x D) -> variances exp(r) + var_floor
// Loss per set (mean over the batch):
//   NLL  = -(1/P) sum_p log sum_g w_g N(x_p | m_g, v_g)           (Eqs. 1, 16)
//   PULL = lambda sum_k w~_k min_g sum_d (m_gd - m~_kd)^2 / v~_kd
// where (w~, m~, v~) is the k-means + EM fit of the plain method on the set.
// The NLL gradient is the EM statistics of the predicted mixture: with
// responsibilities l_{g,p} (Eq. 3),
//   dNLL/da_g  = w_g - (1/P) sum_p l_{g,p}
//   dNLL/dm_gd = -(1/P) sum_p l_{g,p} (x_pd - m_gd) / v_gd
//   dNLL/dr_gd = -(1/2P) sum_p l_{g,p} ((x_pd - m_gd)^2 / v_gd - 1) exp(r_gd) / v_gd.
// Kernels: a tiled BF16 GEMM with FP32 accumulation (optionally transposed
// operands and split-K), bias + ReLU to BF16, ReLU backward, column sums,
// pooling, the loss/gradient kernel and Adam.  FP32 master weights, BF16
// copies feed the GEMMs.
#include <cmath>
#include <algorithm>
#include <cstring>
#include <vector>

#include <cuda.h>

#include "gmm_internal.cuh"
#include "tc_ptx.cuh"

namespace gmm {

namespace {

using namespace ptx;

constexpr int kBM = 64, kBN = 64, kBK = 16;

// C[M][N] (FP32, row stride ldc) (+)= sum_k opA(m,k) opB(n,k).
// opA(m,k) = tA ? A[k*lda + m] : A[m*lda + k];  opB(n,k) = tB ? B[k*ldb + n] : B[n*ldb + k].
// gridDim.z splits K; with splits > 1 (or accumulate) the tile is added with atomics.
__global__ void __launch_bounds__(256) k_gemm_bf16(const __nv_bfloat16 *__restrict__ A, const __nv_bfloat16 *__restrict__ B,
                                                   float *__restrict__ C, int M, int N, int K, int lda, int ldb, int ldc,
                                                   int tA, int tB, int atomic)
{
    __shared__ float As[kBK][kBM + 4];
    __shared__ float Bs[kBK][kBN + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
    const int ks = (K + gridDim.z - 1) / gridDim.z;
    const int kbeg = blockIdx.z * ks, kend = min(K, kbeg + ks);
    float acc[4][4] = {};
    for (int k0 = kbeg; k0 < kend; k0 += kBK) {
        for (int e = threadIdx.x; e < kBK * kBM; e += 256) {
            int kk, mm;
            if (tA) { mm = e % kBM; kk = e / kBM; } else { kk = e % kBK; mm = e / kBK; }
            const int m = m0 + mm, k = k0 + kk;
            float v = 0.f;
            if (m < M && k < kend) v = __bfloat162float(tA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k]);
            As[kk][mm] = v;
        }
        for (int e = threadIdx.x; e < kBK * kBN; e += 256) {
            int kk, nn;
            if (tB) { nn = e % kBN; kk = e / kBN; } else { kk = e % kBK; nn = e / kBK; }
            const int n = n0 + nn, k = k0 + kk;
            float v = 0.f;
            if (n < N && k < kend) v = __bfloat162float(tB ? B[(size_t)k * ldb + n] : B[(size_t)n * ldb + k]);
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
            if (m < M && n < N) {
                if (atomic) atomicAdd(&C[(size_t)m * ldc + n], acc[i][j]);
                else C[(size_t)m * ldc + n] = acc[i][j];
            }
        }
}

// ------------------------------------------------------------------------
// Tensor-core GEMM (tcgen05, BF16 operands, FP32 accumulators in TMEM) for
// the per-point layers: D[M][N] = sum_k A[m][k] B[n][k], A and B row-major
// with K contiguous (K-major), rows a multiple of 8 elements apart.  A CTA
// owns a 128 x BN tile; K advances in 64-wide blocks staged by cp.async into
// 128-byte-swizzled shared memory (kGemmStages stages, all but one block in
// flight ahead of the MMAs), one thread issues the four
// K=16 MMAs of a block and commits them to the stage's mbarrier.  Rows or K
// beyond the operands are zero-filled.  Epilogues (tcgen05.ld, a warp per 32
// rows): 0 FP32 atomics into C (split-K along grid z), 1 bias + ReLU to BF16,
// 2 gradient masked by a stored activation (ReLU backward) to BF16.
// ------------------------------------------------------------------------
struct TcGemm {
    const __nv_bfloat16 *A, *B;
    int M, N, K, lda, ldb;
    int kb_split;                // 64-wide K blocks per CTA along grid z
    int mode;
    float *C; int ldc;
    const float *bias;
    __nv_bfloat16 *out; int ldo;
    const __nv_bfloat16 *ref; int ldr;
    long long budget;            // cycles of a bounded wait
    int *err;                    // set when a wait runs out
};

__device__ __forceinline__ void cp_async16_zf(uint32_t dst, const void *src, int bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes) : "memory");
}

constexpr int kGemmStages = 2;   // K blocks staged at once (two stages keep two CTAs per SM)

template <int BN>
__global__ void __launch_bounds__(128, 1) k_gemm_tc(TcGemm g)
{
    extern __shared__ __align__(1024) unsigned char gt_raw[];
    unsigned char *sb = gt_raw + ((1024u - (smem_u32(gt_raw) & 1023u)) & 1023u);
    constexpr uint32_t kStage = 16384u + (uint32_t)BN * 128u;
    constexpr uint32_t kCols = BN < 32 ? 32 : BN;
    constexpr int NST = kGemmStages;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sb + NST * kStage);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(sb + NST * kStage + 8 * NST);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sb + NST * kStage + 8 * NST + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * BN;
    const int nkb_all = (g.K + 63) / 64;
    const int kb0 = blockIdx.z * g.kb_split, nkb = min(nkb_all, kb0 + g.kb_split) - kb0;
    if (nkb <= 0) return;   // uniform
    if (tid == 0) {
        for (int k = 0; k < NST; ++k) mbar_init(bars + k, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(tslot, kCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    auto load = [&](int kb, int st) {
        unsigned char *sa = sb + st * kStage, *sbb = sa + 16384;
        const int k0 = kb * 64;
        for (int e = tid; e < 128 * 8; e += 128) {
            const int r = e >> 3, c = e & 7, m = m0 + r, k = k0 + 8 * c;
            const bool ok = m < g.M && k < g.K;
            cp_async16_zf(smem_u32(sa + sw128_off(r, c)), ok ? g.A + (size_t)m * g.lda + k : g.A, ok ? 16 : 0);
        }
        for (int e = tid; e < BN * 8; e += 128) {
            const int r = e >> 3, c = e & 7, n = n0 + r, k = k0 + 8 * c;
            const bool ok = n < g.N && k < g.K;
            cp_async16_zf(smem_u32(sbb + sw128_off(r, c)), ok ? g.B + (size_t)n * g.ldb + k : g.B, ok ? 16 : 0);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    const uint32_t idesc = idesc_bf16(128, BN);
    // blocks 0 .. NST-2 in flight before the first MMA; then, per block i, the
    // load of block i + NST - 1 goes to the stage the MMAs of block i - 1 read
    // (after their commit), one cp.async group per block (empty past the end)
    for (int j = 0; j < NST - 1; ++j) {
        if (j < nkb) load(kb0 + j, j);
        else asm volatile("cp.async.commit_group;" ::: "memory");
    }
    for (int i = 0; i < nkb; ++i) {
        const int st = i % NST;
        const int j = i + NST - 1;
        if (j < nkb) {
            if (i >= 1) mbar_wait(bars + (j % NST), (uint32_t)(((i - 1) / NST) & 1), abort_flag, g.budget);
            load(kb0 + j, j % NST);
        } else {
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        asm volatile("cp.async.wait_group %0;" ::"n"(NST - 1) : "memory");   // block i has landed
        fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a = smem_u32(sb + st * kStage), b = a + 16384u;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                tc_mma(tmem, desc_k_sw128(a + kk * 32u), desc_k_sw128(b + kk * 32u), idesc, (i > 0 || kk > 0) ? 1u : 0u);
            tc_commit(bars + st);
        }
    }
    // every MMA has completed once the last block's commit has arrived
    const int ls = (nkb - 1) % NST;
    const uint32_t lp = (uint32_t)(((nkb - 1) / NST) & 1);
    if (!mbar_wait(bars + ls, lp, abort_flag, g.budget)) {
        // bounded drain (ignores the abort flag) before the memory is freed
        const long long d0 = clock64();
        while (!mbar_try_wait(bars + ls, lp) && clock64() - d0 < g.budget) {
        }
        if (tid == 0) atomicExch(g.err, 1);
    }
    tc_fence_after();
    const int row = m0 + 32 * warp + lane;
    const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(tl + (uint32_t)c0, r);
        tmem_wait_ld();
        const int nb = n0 + c0;
        if (row >= g.M || nb >= g.N) continue;
        const bool full = nb + 16 <= g.N;
        if (g.mode == 0) {
            float *c = g.C + (size_t)row * g.ldc + nb;
            if (full && (g.ldc & 3) == 0 && (reinterpret_cast<uintptr_t>(c) & 15u) == 0) {
#pragma unroll
                for (int j = 0; j < 16; j += 4)
                    atomicAdd(reinterpret_cast<float4 *>(c + j),
                              make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                                          __uint_as_float(r[j + 3])));
            } else {
                for (int j = 0; j < 16 && nb + j < g.N; ++j) atomicAdd(c + j, __uint_as_float(r[j]));
            }
        } else {
            __nv_bfloat16 v[16];
            if (g.mode == 1) {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    v[j] = __float2bfloat16_rn(fmaxf(__uint_as_float(r[j]) + (nb + j < g.N ? g.bias[nb + j] : 0.f), 0.f));
            } else {
                const __nv_bfloat16 *h = g.ref + (size_t)row * g.ldr + nb;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float hv = (nb + j < g.N) ? __bfloat162float(h[j]) : 0.f;
                    v[j] = __float2bfloat16_rn(hv > 0.f ? __uint_as_float(r[j]) : 0.f);
                }
            }
            __nv_bfloat16 *o = g.out + (size_t)row * g.ldo + nb;
            if (full && (g.ldo & 7) == 0 && (reinterpret_cast<uintptr_t>(o) & 15u) == 0) {
                reinterpret_cast<uint4 *>(o)[0] = *reinterpret_cast<const uint4 *>(v);
                reinterpret_cast<uint4 *>(o)[1] = *reinterpret_cast<const uint4 *>(v + 8);
            } else {
                for (int j = 0; j < 16 && nb + j < g.N; ++j) o[j] = v[j];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kCols);
}


// ------------------------------------------------------------------------
// Persistent tcgen05 GEMM for the per-point layers' forward and input-
// gradient products (M = points, N = BN <= 256, K <= 256): out[M][N] =
// epilogue(sum_k A[m][k] B[n][k]).  One CTA per SM walks 128-row tiles
// (tile = blockIdx.x + j gridDim.x) with three warp roles:
//   warp 0  loads B (all of K, once) and each tile's 64-wide K blocks of A
//           by tiled TMA (128-byte swizzle, the MMA's K-major layout) into a
//           ring of four stages, each stage freed by the MMAs' commit;
//   warp 1  allocates two TMEM accumulators (2 BN columns) and issues the
//           MMAs of tile j into accumulator j & 1;
//   warps 2-9  the epilogue of tile j from accumulator j & 1 (warp w reads
//           TMEM lanes 32 (w % 4).. and column half (w - 2) / 4), bias +
//           ReLU or the ReLU-backward mask, to BF16, then free the
//           accumulator for tile j + 2,
// so loads, MMAs and the epilogue of consecutive tiles overlap.  K past the
// operands is zero-filled by the TMA.  Every wait is bounded: on expiry the
// CTA raises *err, drains its copies and MMAs, frees its TMEM and returns.
// ------------------------------------------------------------------------
struct TmaGemm {
    int M, N, K;
    int mode;                    // 1: bias + ReLU -> BF16; 2: masked by a stored activation -> BF16
    const float *bias;
    __nv_bfloat16 *out; int ldo;
    const __nv_bfloat16 *ref; int ldr;
    long long budget;
    int *err;
};

constexpr int kTmaStages = 4;
constexpr int kTmaThreads = 320;   // producer warp, MMA warp, eight epilogue warps

template <int BN, int NKB>
__global__ void __launch_bounds__(kTmaThreads, 1) k_gemm_tma(const __grid_constant__ CUtensorMap tmA,
                                                     const __grid_constant__ CUtensorMap tmB, TmaGemm g)
{
    extern __shared__ __align__(1024) unsigned char gm_raw[];
    unsigned char *sb = gm_raw + ((1024u - (smem_u32(gm_raw) & 1023u)) & 1023u);
    constexpr uint32_t kA = 16384u;                 // 128 rows x 128 B
    constexpr uint32_t kB = (uint32_t)BN * 128u;    // BN rows x 128 B per K block
    constexpr int NS = kTmaStages;
    unsigned char *sB = sb;
    unsigned char *sA = sb + NKB * kB;
    uint64_t *full = reinterpret_cast<uint64_t *>(sA + NS * kA);
    uint64_t *empty = full + NS;
    uint64_t *tfull = empty + NS;     // [2]
    uint64_t *tempty = tfull + 2;     // [2]
    uint64_t *bfull = tempty + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bfull + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    float *sbias = reinterpret_cast<float *>(tslot + 4);   // [BN]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (g.M + 127) / 128;
    if (tid == 0) {
        for (int k = 0; k < NS; ++k) { mbar_init(full + k, 1); mbar_init(empty + k, 1); }
        for (int k = 0; k < 2; ++k) { mbar_init(tfull + k, 1); mbar_init(tempty + k, 8); }
        mbar_init(bfull, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(tslot, 2 * BN);
        tmem_relinquish();
    }
    if (g.mode == 1)
        for (int k = tid; k < BN; k += kTmaThreads) sbias[k] = k < g.N ? g.bias[k] : 0.f;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    int issued = 0;   // A loads issued (producer)
    if (warp == 0) {
        if (lane == 0) {
            mbar_expect_tx(bfull, NKB * kB);
            for (int kb = 0; kb < NKB; ++kb) tma_load_2d(sB + kb * kB, &tmB, kb * 64, 0, bfull);
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x)
                for (int kb = 0; kb < NKB; ++kb) {
                    const int s = issued % NS;
                    if (issued >= NS && !mbar_wait(empty + s, (uint32_t)(((issued / NS) - 1) & 1), abort_flag, g.budget))
                        break;
                    mbar_expect_tx(full + s, kA);
                    tma_load_2d(sA + s * kA, &tmA, kb * 64, t * 128, full + s);
                    ++issued;
                }
        }
    } else if (warp == 1) {
        if (lane == 0 && mbar_wait(bfull, 0u, abort_flag, g.budget)) {
            const uint32_t idesc = idesc_bf16(128, BN);
            int used = 0, tc = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort_flag; t += gridDim.x, ++tc) {
                const int acc = tc & 1;
                if (tc >= 2 && !mbar_wait(tempty + acc, (uint32_t)(((tc >> 1) - 1) & 1), abort_flag, g.budget)) break;
                tc_fence_after();
                bool ok = true;
                for (int kb = 0; kb < NKB; ++kb) {
                    const int s = used % NS;
                    if (!mbar_wait(full + s, (uint32_t)((used / NS) & 1), abort_flag, g.budget)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t a = smem_u32(sA + s * kA), b = smem_u32(sB + kb * kB);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        tc_mma(tmem + (uint32_t)(acc * BN), desc_k_sw128(a + kk * 32u), desc_k_sw128(b + kk * 32u), idesc,
                               (kb > 0 || kk > 0) ? 1u : 0u);
                    tc_commit(empty + s);   // the stage is free once these MMAs are done
                    ++used;
                }
                if (!ok) break;
                tc_commit(tfull + acc);     // the accumulator is ready
            }
            // drain: every MMA issued must be complete before TMEM is freed
            if (used > 0) {
                const int s = (used - 1) % NS;
                const uint32_t ph = (uint32_t)(((used - 1) / NS) & 1);
                const long long d0 = clock64();
                while (!mbar_try_wait(empty + s, ph) && clock64() - d0 < g.budget) {
                }
            }
        }
    } else {
        // ---- epilogue warps 2..9: TMEM lane quadrant q = warp % 4, column half
        const int q = warp & 3, ch = (warp - 2) >> 2;
        int tc = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tc) {
            const int acc = tc & 1;
            if (!mbar_wait(tfull + acc, (uint32_t)((tc >> 1) & 1), abort_flag, g.budget)) break;
            tc_fence_after();
            const int row = t * 128 + 32 * q + lane;
            const uint32_t tl = tmem + (uint32_t)(acc * BN) + ((uint32_t)(32 * q) << 16);
            const bool vec_ref = g.mode == 2 && (g.ldr & 7) == 0 && (reinterpret_cast<uintptr_t>(g.ref) & 15u) == 0;
#pragma unroll 1
            // 16 columns of this row -> BF16
            auto emit = [&](int c0, const uint32_t (&r)[16]) {
                if (row >= g.M || c0 >= g.N) return;
                __nv_bfloat16 v[16];
                if (g.mode == 1) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) v[j] = __float2bfloat16_rn(fmaxf(__uint_as_float(r[j]) + sbias[c0 + j], 0.f));
                } else {
                    const __nv_bfloat16 *h = g.ref + (size_t)row * g.ldr + c0;
                    __nv_bfloat16 hv[16];
                    if (vec_ref && c0 + 16 <= g.N) {
                        *reinterpret_cast<uint4 *>(hv) = reinterpret_cast<const uint4 *>(h)[0];
                        *reinterpret_cast<uint4 *>(hv + 8) = reinterpret_cast<const uint4 *>(h)[1];
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) hv[j] = (c0 + j < g.N) ? h[j] : __float2bfloat16_rn(0.f);
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        v[j] = __float2bfloat16_rn(__bfloat162float(hv[j]) > 0.f ? __uint_as_float(r[j]) : 0.f);
                }
                __nv_bfloat16 *o = g.out + (size_t)row * g.ldo + c0;
                if (c0 + 16 <= g.N && (g.ldo & 7) == 0 && (reinterpret_cast<uintptr_t>(o) & 15u) == 0) {
                    reinterpret_cast<uint4 *>(o)[0] = *reinterpret_cast<const uint4 *>(v);
                    reinterpret_cast<uint4 *>(o)[1] = *reinterpret_cast<const uint4 *>(v + 8);
                } else {
                    for (int j = 0; j < 16 && c0 + j < g.N; ++j) o[j] = v[j];
                }
            };
            // 32 columns per TMEM round trip: two loads in flight, one wait
#pragma unroll 1
            for (int c0 = ch * (BN / 2); c0 < (ch + 1) * (BN / 2); c0 += 32) {
                uint32_t ra[16], rb[16];
                tmem_ld16(tl + (uint32_t)c0, ra);
                tmem_ld16(tl + (uint32_t)(c0 + 16), rb);
                tmem_wait_ld();
                emit(c0, ra);
                emit(c0 + 16, rb);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty + acc);
        }
    }
    // drain the producer's copies (bounded, whatever the abort flag) before the
    // shared memory is released: the last load of every stage has landed
    if (warp == 0 && lane == 0) {
        const long long d0 = clock64();
        for (int s = 0; s < NS && s < issued; ++s) {
            const int last = issued - 1 - ((issued - 1 - s) % NS);   // the last load into stage s
            const uint32_t ph = (uint32_t)((last / NS) & 1);
            while (!mbar_try_wait(full + s, ph) && clock64() - d0 < g.budget) {
            }
        }
        while (!mbar_try_wait(bfull, 0u) && clock64() - d0 < g.budget) {
        }
        if (*abort_flag) atomicExch(g.err, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, 2 * BN);
}

// out[c][r] = in[r][c] for a BF16 [R][C] matrix (32 x 32 tiles)
__global__ void k_transpose_bf16(const __nv_bfloat16 *__restrict__ in, __nv_bfloat16 *__restrict__ out, int64_t R, int C)
{
    __shared__ __nv_bfloat16 t[32][34];
    const int64_t r0 = (int64_t)blockIdx.y * 32;
    const int c0 = blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int64_t r = r0 + k;
        const int c = c0 + threadIdx.x;
        if (r < R && c < C) t[k][threadIdx.x] = in[r * C + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k;
        const int64_t r = r0 + threadIdx.x;
        if (r < R && c < C) out[(int64_t)c * R + r] = t[threadIdx.x][k];
    }
}

// out = act(Z + bias) in BF16 (relu != 0) ; also FP32 copy if zf != NULL
__global__ void k_bias_act(const float *__restrict__ Z, const float *__restrict__ bias, __nv_bfloat16 *__restrict__ out,
                           float *__restrict__ zf, int64_t M, int N, int relu)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M * N) return;
    float v = Z[e] + bias[e % N];
    if (relu) v = fmaxf(v, 0.f);
    out[e] = __float2bfloat16_rn(v);
    if (zf) zf[e] = v;
}

// dZ = dH * (H > 0) (ReLU backward through the stored BF16 activation); with
// pool != 0, dH[m][n] = dpool[m / P][n] / P (mean-pool backward).
__global__ void k_relu_bwd(const float *__restrict__ dH, const __nv_bfloat16 *__restrict__ H, __nv_bfloat16 *__restrict__ dZ,
                           int64_t M, int N, int pool_P)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M * N) return;
    float g;
    if (pool_P > 0) {
        const int64_t m = e / N;
        g = dH[(m / pool_P) * N + e % N] / (float)pool_P;
    } else {
        g = dH[e];
    }
    dZ[e] = __float2bfloat16_rn(__bfloat162float(H[e]) > 0.f ? g : 0.f);
}

// db[n] += sum_m dZ[m][n]; blocks over (32 columns, a stride of rows)
__global__ void k_colsum(const __nv_bfloat16 *__restrict__ dZ, float *__restrict__ db, int64_t M, int N)
{
    __shared__ float part[8][33];
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;   // 256 threads: 8 rows at a time
    const int n = blockIdx.x * 32 + lane;
    float s = 0.f;
    if (n < N)
        for (int64_t m = (int64_t)blockIdx.y * 8 + wy; m < M; m += (int64_t)gridDim.y * 8) s += __bfloat162float(dZ[m * N + n]);
    part[wy][lane] = s;
    __syncthreads();
    if (wy == 0 && n < N) {
        float t = 0.f;
        for (int k = 0; k < 8; ++k) t += part[k][lane];
        atomicAdd(&db[n], t);
    }
}

// pooled[b][n] = mean over p of H[b*P + p][n]; also a BF16 copy.  A block
// per (32 columns, set): eight warps take every eighth point, then reduce.
__global__ void k_pool(const __nv_bfloat16 *__restrict__ H, float *__restrict__ pooled, __nv_bfloat16 *__restrict__ pooled_bf,
                       int P, int N)
{
    __shared__ float part[8][33];
    const int b = blockIdx.y, lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int n = blockIdx.x * 32 + lane;
    float s = 0.f;
    if (n < N)
        for (int p = wy; p < P; p += 8) s += __bfloat162float(H[((size_t)b * P + p) * N + n]);
    part[wy][lane] = s;
    __syncthreads();
    if (wy == 0 && n < N) {
        float t = 0.f;
        for (int k = 0; k < 8; ++k) t += part[k][lane];
        t /= (float)P;
        pooled[(size_t)b * N + n] = t;
        pooled_bf[(size_t)b * N + n] = __float2bfloat16_rn(t);
    }
}

__device__ __forceinline__ float bsum_f(float v, float *sh)
{
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
        if (t < s) sh[t] += sh[t + s];
        __syncthreads();
    }
    const float r = sh[0];
    __syncthreads();
    return r;
}

// Loss of each set and its gradient with respect to the network output, in
// three steps (lp = per-set mixture, st = per-set statistics, FP32):
//  k_loss_prep   one block per set: hefts w = softmax(a), constants
//                cst_g = log w_g - 1/2 sum_d log(2 pi v_gd), means m, inverse
//                variances iv = 1/v with v = exp(r) + var_floor, and exp(r);
//                zeroes the statistics and the NLL.
//  k_loss_chunk  one block per (set, 128 points): log-densities and log-sum-
//                exp of each point (Eqs. 15-16), responsibilities (Eq. 3) in
//                shared memory, then the statistics S0_g = sum l, S1_gd =
//                sum l (x - m), S2_gd = sum l (x - m)^2 as a dense reduction
//                over the block's points, added to the set's totals.
//  k_loss_grad   one block per set: dNLL/d(a, m, r) from the statistics, the
//                pull of the predicted means toward the plain method's fit,
//                the loss, and optionally the predicted mixture in FP64.
constexpr int kLossPts = 128;

__global__ void k_loss_prep(const float *__restrict__ out, int D, int G, double var_floor, float *__restrict__ lp,
                            float *__restrict__ st, float *__restrict__ nll)
{
    const int b = blockIdx.x, O = G * (1 + 2 * D), LP = 2 * G + 3 * G * D, ST = G + 2 * G * D;
    const float *o = out + (size_t)b * O;
    float *w = lp + (size_t)b * LP, *cst = w + G, *m = cst + G, *iv = m + G * D, *er = iv + G * D;
    __shared__ float s_max, s_lsum;
    if (threadIdx.x == 0) {
        float mx = -INFINITY;
        for (int g = 0; g < G; ++g) mx = fmaxf(mx, o[g]);
        float sm = 0.f;
        for (int g = 0; g < G; ++g) sm += __expf(o[g] - mx);
        s_max = mx;
        s_lsum = logf(sm);
        nll[b] = 0.f;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < G * D; k += blockDim.x) {
        m[k] = o[G + k];
        const float e = __expf(o[G + G * D + k]);
        er[k] = e;
        iv[k] = 1.f / (e + (float)var_floor);
    }
    for (int k = threadIdx.x; k < ST; k += blockDim.x) st[(size_t)b * ST + k] = 0.f;
    __syncthreads();
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
        const float lw = o[g] - s_max - s_lsum;
        w[g] = __expf(lw);
        float sl = 0.f;
        for (int d = 0; d < D; ++d) sl += logf(iv[g * D + d]);   // = -sum log v
        cst[g] = lw - 0.5f * ((float)D * 1.8378770664093453f - sl);
    }
}

__global__ void __launch_bounds__(kLossPts) k_loss_chunk(const float *__restrict__ pts, int P, int D, int G,
                                                         const float *__restrict__ lp, float *__restrict__ st,
                                                         float *__restrict__ nll)
{
    extern __shared__ float lsm[];
    const int b = blockIdx.x, p0 = blockIdx.y * kLossPts, np = min(kLossPts, P - p0);
    const int LP = 2 * G + 3 * G * D, ST = G + 2 * G * D, GS = G + 1, XS = D | 1;   // odd row strides
    float *cst = lsm;                    // [G]
    float *m = cst + G;                  // [G][D]
    float *iv = m + G * D;               // [G][D]
    float *x = iv + G * D;               // [128][XS]
    float *gam = x + kLossPts * XS;      // [128][G + 1]
    float *red = gam + kLossPts * GS;    // [128]
    const float *lpb = lp + (size_t)b * LP;
    for (int k = threadIdx.x; k < G; k += kLossPts) cst[k] = lpb[G + k];
    for (int k = threadIdx.x; k < 2 * G * D; k += kLossPts) m[k] = lpb[2 * G + k];   // m then iv
    for (int k = threadIdx.x; k < np * D; k += kLossPts) x[(k / D) * XS + k % D] = pts[((size_t)b * P + p0) * D + k];
    __syncthreads();
    float nl = 0.f;
    const int p = threadIdx.x;
    if (p < np) {
        const float *xp = x + p * XS;
        float mx = -INFINITY, sm = 0.f;
        for (int g = 0; g < G; ++g) {
            float q = 0.f;
            for (int d = 0; d < D; ++d) {
                const float t = xp[d] - m[g * D + d];
                q = fmaf(t * t, iv[g * D + d], q);
            }
            const float l = fmaf(-0.5f, q, cst[g]);
            gam[p * GS + g] = l;
            if (l > mx) { sm = sm * __expf(mx - l) + 1.f; mx = l; }
            else if (l > -INFINITY) sm += __expf(l - mx);   // -inf terms add nothing (and -inf - -inf is NaN)
        }
        const float lse = mx + logf(sm);
        nl = -lse;
        for (int g = 0; g < G; ++g) gam[p * GS + g] = __expf(gam[p * GS + g] - lse);   // Eq. 3
    }
    red[threadIdx.x] = nl;
    __syncthreads();
    for (int h = kLossPts / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(&nll[b], red[0]);
    // statistics of the block's points: threads over (g, d)
    float *stb = st + (size_t)b * ST;
    for (int k = threadIdx.x; k < G * D; k += kLossPts) {
        const int g = k / D, d = k - g * D;
        const float mg = m[k];
        float s1 = 0.f, s2 = 0.f;
        for (int q = 0; q < np; ++q) {
            const float t = x[q * XS + d] - mg;
            const float v = gam[q * GS + g] * t;
            s1 += v;
            s2 = fmaf(v, t, s2);
        }
        atomicAdd(&stb[G + k], s1);
        atomicAdd(&stb[G + G * D + k], s2);
    }
    for (int g = threadIdx.x; g < G; g += kLossPts) {
        float s0 = 0.f;
        for (int q = 0; q < np; ++q) s0 += gam[q * GS + g];
        atomicAdd(&stb[g], s0);
    }
}

__global__ void __launch_bounds__(256) k_loss_grad(const float *__restrict__ lp, const float *__restrict__ st,
                                                   const float *__restrict__ nll, int P, int D, int G, double var_floor,
                                                   const double *__restrict__ tgt_m, const double *__restrict__ tgt_v,
                                                   const double *__restrict__ tgt_w, double lambda,
                                                   float *__restrict__ d_out, float *__restrict__ loss,
                                                   double *__restrict__ pm, double *__restrict__ pv,
                                                   double *__restrict__ pw, int B)
{
    __shared__ float sh[256];
    const int b = blockIdx.x, O = G * (1 + 2 * D), LP = 2 * G + 3 * G * D, ST = G + 2 * G * D;
    const float *w = lp + (size_t)b * LP, *m = w + 2 * G, *iv = m + G * D, *er = iv + G * D;
    const float *S0 = st + (size_t)b * ST, *S1 = S0 + G, *S2 = S1 + G * D;
    const float invB = 1.f / (float)B, invP = 1.f / (float)P;
    float *d = d_out + (size_t)b * O;
    for (int g = threadIdx.x; g < G; g += blockDim.x) d[g] = (w[g] - S0[g] * invP) * invB;
    for (int k = threadIdx.x; k < G * D; k += blockDim.x) {
        d[G + k] = -S1[k] * iv[k] * invP * invB;
        d[G + G * D + k] = -0.5f * (S2[k] * iv[k] - S0[k / D]) * er[k] * iv[k] * invP * invB;
    }
    __syncthreads();
    // pull of the predicted means toward the plain method's fit (nearest pairs);
    // the set's targets go to shared memory once (means, inverse variances)
    float pull = 0.f;
    if (lambda > 0.0 && tgt_m) {
        extern __shared__ float tsm[];   // [G][D] target means, [G][D] 1 / target variances
        float *tmf = tsm, *tif = tsm + G * D;
        for (int k = threadIdx.x; k < G * D; k += blockDim.x) {
            tmf[k] = (float)tgt_m[(size_t)b * G * D + k];
            tif[k] = 1.f / (float)tgt_v[(size_t)b * G * D + k];
        }
        __syncthreads();
        for (int k = threadIdx.x; k < G; k += blockDim.x) {
            const float *tm = tmf + k * D, *ti = tif + k * D;
            float best = INFINITY;
            int bg = 0;
            for (int g = 0; g < G; ++g) {
                float q = 0.f;
                for (int dd = 0; dd < D; ++dd) {
                    const float t = m[g * D + dd] - tm[dd];
                    q = fmaf(t * t, ti[dd], q);
                }
                if (q < best) { best = q; bg = g; }
            }
            const float wk = (float)tgt_w[(size_t)b * G + k] * (float)lambda;
            pull += wk * best;
            for (int dd = 0; dd < D; ++dd)
                atomicAdd(&d[G + bg * D + dd], 2.f * wk * (m[bg * D + dd] - tm[dd]) * ti[dd] * invB);
        }
    }
    pull = bsum_f(pull, sh);
    if (threadIdx.x == 0) loss[b] = nll[b] * invP + pull;
    if (pm) {
        for (int k = threadIdx.x; k < G * D; k += blockDim.x) {
            pm[(size_t)b * G * D + k] = (double)m[k];
            pv[(size_t)b * G * D + k] = (double)er[k] + var_floor;
        }
        for (int g = threadIdx.x; g < G; g += blockDim.x) pw[(size_t)b * G + g] = (double)w[g];
    }
}

// Adam (Kingma & Ba, 2015) on the FP32 master weights; BF16 copy refreshed.
__global__ void k_adam(float *__restrict__ wgt, const float *__restrict__ g, float *__restrict__ m1, float *__restrict__ m2,
                       __nv_bfloat16 *__restrict__ wbf, int64_t n, float lr, float b1, float b2, float eps, float c1,
                       float c2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float s = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = s;
    const float w = wgt[i] - lr * (a / c1) / (sqrtf(s / c2) + eps);
    wgt[i] = w;
    wbf[i] = __float2bfloat16_rn(w);
}

__global__ void k_to_bf16(const float *__restrict__ x, __nv_bfloat16 *__restrict__ y, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

// ----------------------------------------------------------------- host
struct InitNet {
    int D, G, Hp, Hh, Lp, Lh, O;
    int64_t n_params = 0;
    std::vector<int64_t> w_off, b_off, w_in, w_out;   // per layer (Lp + Lh + 1 layers)
    float *wgt = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
    __nv_bfloat16 *wbf = nullptr;
    int *err = nullptr;             // device flag: a bounded wait of a tensor-core GEMM ran out
    int64_t step = 0;
    // activation workspace (grown per batch)
    size_t ws_cap = 0;
    unsigned char *ws = nullptr;
};

namespace {

struct Ws {
    __nv_bfloat16 *x;               // [BP][D] input points in BF16
    std::vector<__nv_bfloat16 *> h; // per-point activations [BP][Hp] x Lp
    float *z;                       // FP32 scratch [BP][max(Hp, Hh, O)]
    __nv_bfloat16 *dz;              // BF16 [BP][Hp]
    float *dh;                      // FP32 [BP][Hp]
    float *pooled;                  // [B][Hp]
    std::vector<__nv_bfloat16 *> a; // head activations [B][Hh] x Lh, a[0] = pooled (BF16)
    float *out;                     // [B][O]
    float *dout;                    // [B][O]
    float *loss;                    // [B]
    __nv_bfloat16 *dz2;             // BF16 [BP][Hp] second gradient buffer (tensor-core backward)
    __nv_bfloat16 *dzT;             // BF16 [Hp][BP] transposed gradient
    __nv_bfloat16 *inT;             // BF16 [max(D, Hp)][BP] transposed layer input
    __nv_bfloat16 *wT;              // BF16 [max(D, Hp)][Hp] transposed weights
    float *lpar;                    // [B][2G + 3GD] predicted mixture for the loss
    float *lst;                     // [B][G + 2GD] statistics of the loss
    float *lnll;                    // [B] NLL sums
};

size_t ws_bytes(const InitNet &n, int B, int P)
{
    const int64_t BP = (int64_t)B * P;
    const int64_t wmax = std::max((int64_t)n.Hp, std::max((int64_t)n.Hh, (int64_t)n.O));
    size_t s = 0;
    auto add = [&](size_t b) { s += (b + 255) / 256 * 256; };
    add(2 * BP * n.D);
    for (int l = 0; l < n.Lp; ++l) add(2 * BP * n.Hp);
    add(4 * BP * wmax);
    add(2 * BP * n.Hp);
    add(4 * BP * n.Hp);
    add(4 * (size_t)B * n.Hp);
    for (int l = 0; l <= n.Lh; ++l) add(2 * (size_t)B * std::max(n.Hh, n.Hp));
    add(4 * (size_t)B * n.O);
    add(4 * (size_t)B * n.O);
    add(4 * (size_t)B);
    const int64_t kmax = std::max(n.D, n.Hp);
    add(2 * BP * n.Hp);
    add(2 * BP * n.Hp);
    add(2 * BP * kmax);
    add(2 * (size_t)kmax * n.Hp);
    add(4 * (size_t)B * (2 * n.G + 3 * (size_t)n.G * n.D));
    add(4 * (size_t)B * (n.G + 2 * (size_t)n.G * n.D));
    add(4 * (size_t)B);
    return s;
}

Ws carve(InitNet &n, int B, int P)
{
    const int64_t BP = (int64_t)B * P;
    const int64_t wmax = std::max((int64_t)n.Hp, std::max((int64_t)n.Hh, (int64_t)n.O));
    unsigned char *p = n.ws;
    auto take = [&](size_t b) { unsigned char *q = p; p += (b + 255) / 256 * 256; return q; };
    Ws w;
    w.x = reinterpret_cast<__nv_bfloat16 *>(take(2 * BP * n.D));
    for (int l = 0; l < n.Lp; ++l) w.h.push_back(reinterpret_cast<__nv_bfloat16 *>(take(2 * BP * n.Hp)));
    w.z = reinterpret_cast<float *>(take(4 * BP * wmax));
    w.dz = reinterpret_cast<__nv_bfloat16 *>(take(2 * BP * n.Hp));
    w.dh = reinterpret_cast<float *>(take(4 * BP * n.Hp));
    w.pooled = reinterpret_cast<float *>(take(4 * (size_t)B * n.Hp));
    for (int l = 0; l <= n.Lh; ++l)
        w.a.push_back(reinterpret_cast<__nv_bfloat16 *>(take(2 * (size_t)B * std::max(n.Hh, n.Hp))));
    w.out = reinterpret_cast<float *>(take(4 * (size_t)B * n.O));
    w.dout = reinterpret_cast<float *>(take(4 * (size_t)B * n.O));
    w.loss = reinterpret_cast<float *>(take(4 * (size_t)B));
    const int64_t kmax = std::max(n.D, n.Hp);
    w.dz2 = reinterpret_cast<__nv_bfloat16 *>(take(2 * BP * n.Hp));
    w.dzT = reinterpret_cast<__nv_bfloat16 *>(take(2 * BP * n.Hp));
    w.inT = reinterpret_cast<__nv_bfloat16 *>(take(2 * BP * kmax));
    w.wT = reinterpret_cast<__nv_bfloat16 *>(take(2 * (size_t)kmax * n.Hp));
    w.lpar = reinterpret_cast<float *>(take(4 * (size_t)B * (2 * n.G + 3 * (size_t)n.G * n.D)));
    w.lst = reinterpret_cast<float *>(take(4 * (size_t)B * (n.G + 2 * (size_t)n.G * n.D)));
    w.lnll = reinterpret_cast<float *>(take(4 * (size_t)B));
    return w;
}

cudaError_t gemm(const __nv_bfloat16 *A, const __nv_bfloat16 *B, float *C, int M, int N, int K, int lda, int ldb, int ldc,
                 int tA, int tB, int splits, int accumulate, cudaStream_t s)
{
    dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM, splits);
    if (splits > 1 && !accumulate) return cudaErrorInvalidValue;   // split-K only accumulates onto zeroed C
    k_gemm_bf16<<<grid, 256, 0, s>>>(A, B, C, M, N, K, lda, ldb, ldc, tA, tB, (splits > 1 || accumulate) ? 1 : 0);
    count_launches(1);
    return cudaGetLastError();
}

#define CKE_(x)                                      \
    do {                                             \
        cudaError_t e_ = (x);                        \
        if (e_ != cudaSuccess) return e_;            \
    } while (0)

// C[M][N] (row stride N) = op(A) op(B)^T for the head layers (M = sets, a few
// dozen rows): split along K until the grid fills the GPU; the split parts
// are added with atomics onto the zeroed C.
cudaError_t gemm_small(const __nv_bfloat16 *A, const __nv_bfloat16 *B, float *C, int M, int N, int K, int lda, int ldb,
                       int tA, int tB, cudaStream_t s)
{
    const int tiles = ((N + kBN - 1) / kBN) * ((M + kBM - 1) / kBM);
    const int splits = std::max(1, std::min((K + kBK * 4 - 1) / (kBK * 4), (304 + tiles - 1) / tiles));
    if (splits == 1) return gemm(A, B, C, M, N, K, lda, ldb, N, tA, tB, 1, 0, s);
    CKE_(cudaMemsetAsync(C, 0, sizeof(float) * (size_t)M * N, s));
    return gemm(A, B, C, M, N, K, lda, ldb, N, tA, tB, splits, 1, s);
}

bool tc_usable(const void *A, const void *B, int K, int lda, int ldb)
{
    return ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15u) == 0 && K % 8 == 0 &&
           lda % 8 == 0 && ldb % 8 == 0;
}

// D = A B^T on the tensor cores (see k_gemm_tc); splits > 1 only with mode 0
cudaError_t gemm_tc(const __nv_bfloat16 *A, const __nv_bfloat16 *B, int64_t M, int N, int K, int lda, int ldb, int mode,
                    float *C, int ldc, const float *bias, __nv_bfloat16 *out, int ldo, const __nv_bfloat16 *ref,
                    int ldr, int splits, int *err, cudaStream_t s)
{
    const int nkb = (K + 63) / 64;
    splits = std::max(1, std::min(splits, nkb));
    const int kb_split = (nkb + splits - 1) / splits;
    const int gz = (nkb + kb_split - 1) / kb_split;
    TcGemm g{A, B, (int)M, N, K, lda, ldb, kb_split, mode, C, ldc, bias, out, ldo, ref, ldr, 2000000000LL, err};
    const int BN = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
    const size_t sm = kGemmStages * (16384 + (size_t)BN * 128) + 64 + 1024;
    const dim3 grid((unsigned)((M + 127) / 128), (unsigned)((N + BN - 1) / BN), (unsigned)gz);
#define GTC(BNV)                                                                                           \
    do {                                                                                                   \
        cudaError_t e_ = cudaFuncSetAttribute(k_gemm_tc<BNV>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                              (int)sm);                                                    \
        if (e_ != cudaSuccess) return e_;                                                                  \
        k_gemm_tc<BNV><<<grid, 128, sm, s>>>(g);                                                           \
    } while (0)
    if (BN == 32) GTC(32);
    else if (BN == 64) GTC(64);
    else if (BN == 128) GTC(128);
    else GTC(256);
#undef GTC
    count_launches(1);
    return cudaGetLastError();
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// BF16 [rows][cols] (row stride ld elements) as boxes of 64 columns x box_rows
// rows in the 128-byte swizzle; reads past the matrix return zeros
bool make_map(CUtensorMap *m, const __nv_bfloat16 *base, int64_t rows, int cols, int ld, int box_rows)
{
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2u};
    const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1u, 1u};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n < 1) n = 1;
    }
    return n;
}

// The persistent TMA GEMM for out = epilogue(A B^T) (modes 1, 2 of k_gemm_tc)
// with N = 256 and K <= 256; cudaErrorNotSupported (nothing launched) for
// any other shape, alignment, or without the tensor-map entry point.
cudaError_t gemm_tma(const __nv_bfloat16 *A, const __nv_bfloat16 *B, int64_t M, int N, int K, int lda, int ldb,
                     int mode, const float *bias, __nv_bfloat16 *out, int ldo, const __nv_bfloat16 *ref, int ldr,
                     int *err, cudaStream_t s)
{
    constexpr int BN = 256;
    if (N != BN || K < 1 || K > 256 || K % 8 != 0 || lda % 8 != 0 || ldb % 8 != 0 || M < 1 || M > INT32_MAX ||
        ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15u) != 0 || (mode != 1 && mode != 2))
        return cudaErrorNotSupported;
    CUtensorMap ta, tb;
    if (!make_map(&ta, A, M, K, lda, 128) || !make_map(&tb, B, N, K, ldb, BN)) return cudaErrorNotSupported;
    const int nkb = (K + 63) / 64;
    TmaGemm gg{(int)M, N, K, mode, bias, out, ldo, ref, ldr, 2000000000LL, err};
    const size_t sm = (size_t)nkb * BN * 128 + (size_t)kTmaStages * 16384 + 256 + 4 * BN + 1024;
    const int ntiles = (int)((M + 127) / 128);
    const int grid = std::min(ntiles, sm_count());
#define GTMA(NKB)                                                                                              \
    do {                                                                                                       \
        cudaError_t e_ = cudaFuncSetAttribute(k_gemm_tma<BN, NKB>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                              (int)sm);                                                        \
        if (e_ != cudaSuccess) return e_;                                                                      \
        k_gemm_tma<BN, NKB><<<grid, kTmaThreads, sm, s>>>(ta, tb, gg);                                         \
    } while (0)
    if (nkb == 1) GTMA(1);
    else if (nkb == 2) GTMA(2);
    else if (nkb == 3) GTMA(3);
    else GTMA(4);
#undef GTMA
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t transpose_bf16(const __nv_bfloat16 *in, __nv_bfloat16 *out, int64_t R, int C, cudaStream_t s)
{
    k_transpose_bf16<<<dim3((unsigned)((C + 31) / 32), (unsigned)((R + 31) / 32)), dim3(32, 8), 0, s>>>(in, out, R, C);
    count_launches(1);
    return cudaGetLastError();
}

#define CKE(x)                                       \
    do {                                             \
        cudaError_t e_ = (x);                        \
        if (e_ != cudaSuccess) return e_;            \
    } while (0)

// Forward pass for B sets of P points (pts FP32 [B][P][D], device).
cudaError_t net_forward(InitNet &n, const float *pts, int B, int P, Ws &w, cudaStream_t s)
{
    const int64_t BP = (int64_t)B * P;
    k_to_bf16<<<blocks_for(BP * n.D, 256), 256, 0, s>>>(pts, w.x, BP * n.D);
    const __nv_bfloat16 *in = w.x;
    int kin = n.D;
    for (int l = 0; l < n.Lp; ++l) {
        const __nv_bfloat16 *W = n.wbf + n.w_off[l];
        if (tc_usable(in, W, kin, kin, kin)) {
            // tensor cores, bias + ReLU + BF16 in the epilogue
            const cudaError_t e = gemm_tma(in, W, BP, n.Hp, kin, kin, kin, 1, n.wgt + n.b_off[l], w.h[l], n.Hp, nullptr, 0,
                                           n.err, s);
            if (e == cudaErrorNotSupported)
                CKE(gemm_tc(in, W, BP, n.Hp, kin, kin, kin, 1, nullptr, 0, n.wgt + n.b_off[l], w.h[l], n.Hp, nullptr, 0,
                            1, n.err, s));
            else
                CKE(e);
        } else {
            CKE(gemm(in, W, w.z, (int)BP, n.Hp, kin, kin, kin, n.Hp, 0, 0, 1, 0, s));
            k_bias_act<<<blocks_for(BP * n.Hp, 256), 256, 0, s>>>(w.z, n.wgt + n.b_off[l], w.h[l], nullptr, BP, n.Hp, 1);
        }
        in = w.h[l];
        kin = n.Hp;
    }
    k_pool<<<dim3((n.Hp + 31) / 32, B), 256, 0, s>>>(w.h[n.Lp - 1], w.pooled, w.a[0], P, n.Hp);
    int hin = n.Hp;
    for (int l = 0; l < n.Lh; ++l) {
        const int li = n.Lp + l;
        CKE(gemm_small(w.a[l], n.wbf + n.w_off[li], w.z, B, n.Hh, hin, hin, hin, 0, 0, s));
        k_bias_act<<<blocks_for((int64_t)B * n.Hh, 256), 256, 0, s>>>(w.z, n.wgt + n.b_off[li], w.a[l + 1], nullptr, B,
                                                                       n.Hh, 1);
        hin = n.Hh;
    }
    const int lo = n.Lp + n.Lh;
    CKE(gemm_small(w.a[n.Lh], n.wbf + n.w_off[lo], w.z, B, n.O, hin, hin, hin, 0, 0, s));
    // the BF16 copy of the output is not needed: write it to the free dz buffer
    k_bias_act<<<blocks_for((int64_t)B * n.O, 256), 256, 0, s>>>(w.z, n.wgt + n.b_off[lo], w.dz, w.out, B, n.O, 0);
    count_launches(3 + n.Lp + n.Lh);
    return cudaGetLastError();
}

// Backward pass from w.dout; gradients accumulate into n.grad (zeroed here).
cudaError_t net_backward(InitNet &n, int B, int P, Ws &w, cudaStream_t s)
{
    const int64_t BP = (int64_t)B * P;
    CKE(cudaMemsetAsync(n.grad, 0, sizeof(float) * n.n_params, s));
    // output layer: dW = dout^T a_Lh, db = colsum(dout), dA = dout W
    const int lo = n.Lp + n.Lh;
    int hin = n.Lh > 0 ? n.Hh : n.Hp;
    // dout FP32 -> BF16 for the GEMMs (reuse dz)
    k_to_bf16<<<blocks_for((int64_t)B * n.O, 256), 256, 0, s>>>(w.dout, w.dz, (int64_t)B * n.O);
    CKE(gemm(w.dz, w.a[n.Lh], n.grad + n.w_off[lo], n.O, hin, B, n.O, hin, hin, 1, 1, 1, 1, s));
    k_colsum<<<dim3((n.O + 31) / 32, 1), 256, 0, s>>>(w.dz, n.grad + n.b_off[lo], B, n.O);
    CKE(gemm_small(w.dz, n.wbf + n.w_off[lo], w.dh, B, hin, n.O, n.O, hin, 0, 1, s));
    for (int l = n.Lh - 1; l >= 0; --l) {
        const int li = n.Lp + l;
        const int lin = l == 0 ? n.Hp : n.Hh;
        k_relu_bwd<<<blocks_for((int64_t)B * n.Hh, 256), 256, 0, s>>>(w.dh, w.a[l + 1], w.dz, B, n.Hh, 0);
        CKE(gemm(w.dz, w.a[l], n.grad + n.w_off[li], n.Hh, lin, B, n.Hh, lin, lin, 1, 1, 1, 1, s));
        k_colsum<<<dim3((n.Hh + 31) / 32, 1), 256, 0, s>>>(w.dz, n.grad + n.b_off[li], B, n.Hh);
        CKE(gemm_small(w.dz, n.wbf + n.w_off[li], w.dh, B, lin, n.Hh, n.Hh, lin, 0, 1, s));
    }
    // w.dh now holds d(pooled) [B][Hp]; per-point layers.  cur = dLoss/dZ_l in BF16.
    __nv_bfloat16 *cur = w.dz, *nxt = w.dz2;
    k_relu_bwd<<<blocks_for(BP * n.Hp, 256), 256, 0, s>>>(w.dh, w.h[n.Lp - 1], cur, BP, n.Hp, P);
    for (int l = n.Lp - 1; l >= 0; --l) {
        const int kin = l == 0 ? n.D : n.Hp;
        const __nv_bfloat16 *hin_act = l == 0 ? w.x : w.h[l - 1];
        const __nv_bfloat16 *W = n.wbf + n.w_off[l];
        // dW_l = cur^T in_l: a reduction over the B*P points, split along K
        if (BP % 8 == 0 && tc_usable(w.dzT, w.inT, (int)BP, (int)BP, (int)BP)) {
            CKE(transpose_bf16(cur, w.dzT, BP, n.Hp, s));
            CKE(transpose_bf16(hin_act, w.inT, BP, kin, s));
            CKE(gemm_tc(w.dzT, w.inT, n.Hp, kin, (int)BP, (int)BP, (int)BP, 0, n.grad + n.w_off[l], kin, nullptr, nullptr,
                        0, nullptr, 0, 64, n.err, s));
        } else {
            const int splits = (int)std::min<int64_t>(64, std::max<int64_t>(1, BP / 4096));
            CKE(gemm(cur, hin_act, n.grad + n.w_off[l], n.Hp, kin, (int)BP, n.Hp, kin, kin, 1, 1, splits, 1, s));
        }
        k_colsum<<<dim3((n.Hp + 31) / 32, (unsigned)std::min<int64_t>(256, (BP + 255) / 256)), 256, 0, s>>>(
            cur, n.grad + n.b_off[l], BP, n.Hp);
        if (l == 0) break;
        // dZ_{l-1} = (cur W_l) masked by ReLU'(h_{l-1})
        if (tc_usable(cur, w.wT, n.Hp, n.Hp, n.Hp)) {
            CKE(transpose_bf16(W, w.wT, n.Hp, kin, s));
            const cudaError_t e = gemm_tma(cur, w.wT, BP, kin, n.Hp, n.Hp, n.Hp, 2, nullptr, nxt, kin, w.h[l - 1], kin,
                                           n.err, s);
            if (e == cudaErrorNotSupported)
                CKE(gemm_tc(cur, w.wT, BP, kin, n.Hp, n.Hp, n.Hp, 2, nullptr, 0, nullptr, nxt, kin, w.h[l - 1], kin, 1,
                            n.err, s));
            else
                CKE(e);
            std::swap(cur, nxt);
        } else {
            CKE(gemm(cur, W, w.dh, (int)BP, kin, n.Hp, n.Hp, kin, kin, 0, 1, 1, 0, s));
            k_relu_bwd<<<blocks_for(BP * n.Hp, 256), 256, 0, s>>>(w.dh, w.h[l - 1], cur, BP, n.Hp, 0);
        }
    }
    count_launches(2 + 3 * (n.Lh + n.Lp));
    return cudaGetLastError();
}

cudaError_t ensure_ws(InitNet &n, int B, int P)
{
    const size_t need = ws_bytes(n, B, P);
    if (need <= n.ws_cap) return cudaSuccess;
    if (n.ws) cudaFree(n.ws);
    n.ws = nullptr;
    n.ws_cap = 0;
    CKE(cudaMalloc(&n.ws, need));
    n.ws_cap = need;
    return cudaSuccess;
}

}  // namespace

InitNet *init_net_new(int D, int G, int Hp, int Hh, int Lp, int Lh, uint64_t seed, cudaError_t *err)
{
    InitNet *n = new InitNet();
    n->D = D; n->G = G; n->Hp = Hp; n->Hh = Hh; n->Lp = Lp; n->Lh = Lh; n->O = G * (1 + 2 * D);
    const int L = Lp + Lh + 1;
    int64_t o = 0;
    for (int l = 0; l < L; ++l) {
        const int in = l == 0 ? D : (l < Lp ? Hp : (l == Lp ? Hp : Hh));
        const int out = l < Lp ? Hp : (l < L - 1 ? Hh : n->O);
        n->w_in.push_back(in);
        n->w_out.push_back(out);
        n->w_off.push_back(o);
        o += (int64_t)in * out;
        n->b_off.push_back(o);
        o += out;
    }
    n->n_params = o;
    // He-uniform initial weights from SplitMix64(seed), zero biases; the
    // output layer starts small so the first mixtures are broad
    std::vector<float> h(o, 0.f);
    uint64_t st = seed;
    auto next = [&]() {
        uint64_t z = (st += 0x9e3779b97f4a7c15ULL);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    for (int l = 0; l < L; ++l) {
        const double lim = std::sqrt(6.0 / n->w_in[l]) * (l == L - 1 ? 0.1 : 1.0);
        for (int64_t k = 0; k < n->w_in[l] * n->w_out[l]; ++k) h[n->w_off[l] + k] = (float)((2.0 * next() - 1.0) * lim);
    }
    cudaError_t e = cudaMalloc(&n->wgt, 4 * o);
    if (e == cudaSuccess) e = cudaMalloc(&n->grad, 4 * o);
    if (e == cudaSuccess) e = cudaMalloc(&n->m1, 4 * o);
    if (e == cudaSuccess) e = cudaMalloc(&n->m2, 4 * o);
    if (e == cudaSuccess) e = cudaMalloc(&n->wbf, 2 * o);
    if (e == cudaSuccess) e = cudaMalloc(&n->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(n->err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(n->wgt, h.data(), 4 * o, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(n->m1, 0, 4 * o);
    if (e == cudaSuccess) e = cudaMemset(n->m2, 0, 4 * o);
    if (e == cudaSuccess) {
        k_to_bf16<<<blocks_for(o, 256), 256>>>(n->wgt, n->wbf, o);
        e = cudaGetLastError();
    }
    *err = e;
    return n;
}

void init_net_free(InitNet *n)
{
    if (!n) return;
    void *b[] = {n->wgt, n->grad, n->m1, n->m2, n->wbf, n->ws, n->err};
    for (void *p : b)
        if (p) cudaFree(p);
    delete n;
}

int64_t init_net_n_params(const InitNet *n) { return n->n_params; }

namespace {
__global__ void k_gather_rows(const float *__restrict__ X, int D, const int64_t *__restrict__ idx, int P,
                              float *__restrict__ out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)P * D) return;
    const int64_t p = e / D, d = e - p * D;
    out[e] = X[idx[p] * D + d];
}
}  // namespace

cudaError_t init_net_gather(const float *X, int D, const int64_t *idx, int P, float *out, cudaStream_t s)
{
    k_gather_rows<<<blocks_for((int64_t)P * D, 256), 256, 0, s>>>(X, D, idx, P, out);
    count_launches(1);
    return cudaGetLastError();
}
int init_net_D(const InitNet *n) { return n->D; }
int init_net_G(const InitNet *n) { return n->G; }

cudaError_t init_net_set_weights(InitNet *n, const float *w_host)
{
    CKE(cudaMemcpy(n->wgt, w_host, 4 * n->n_params, cudaMemcpyHostToDevice));
    k_to_bf16<<<blocks_for(n->n_params, 256), 256>>>(n->wgt, n->wbf, n->n_params);
    return cudaGetLastError();
}

cudaError_t init_net_get_adam(const InitNet *n, float *m1_host, float *m2_host, int64_t *step)
{
    if (m1_host) CKE(cudaMemcpy(m1_host, n->m1, 4 * n->n_params, cudaMemcpyDeviceToHost));
    if (m2_host) CKE(cudaMemcpy(m2_host, n->m2, 4 * n->n_params, cudaMemcpyDeviceToHost));
    if (step) *step = n->step;
    return cudaSuccess;
}

cudaError_t init_net_set_adam(InitNet *n, const float *m1_host, const float *m2_host, int64_t step)
{
    CKE(cudaMemcpy(n->m1, m1_host, 4 * n->n_params, cudaMemcpyHostToDevice));
    CKE(cudaMemcpy(n->m2, m2_host, 4 * n->n_params, cudaMemcpyHostToDevice));
    n->step = step;
    return cudaSuccess;
}

cudaError_t init_net_get(const InitNet *n, float *w_host, float *g_host)
{
    if (w_host) CKE(cudaMemcpy(w_host, n->wgt, 4 * n->n_params, cudaMemcpyDeviceToHost));
    if (g_host) CKE(cudaMemcpy(g_host, n->grad, 4 * n->n_params, cudaMemcpyDeviceToHost));
    return cudaSuccess;
}

// Forward (+ loss, + backward if grads, + Adam if lr > 0).  pts: device FP32
// [B][P][D]; targets (device FP64, may be NULL when lambda == 0); predicted
// parameters written to pm/pv/pw (device FP64, may be NULL); mean loss to
// *loss_host.
cudaError_t init_net_run(InitNet *n, const float *pts, int B, int P, const double *tm, const double *tv, const double *tw,
                         double lambda, double var_floor, int grads, double lr, double *pm, double *pv, double *pw,
                         double *loss_host, cudaStream_t s)
{
    CKE(ensure_ws(*n, B, P));
    Ws w = carve(*n, B, P);
    CKE(net_forward(*n, pts, B, P, w, s));
    k_loss_prep<<<B, 256, 0, s>>>(w.out, n->D, n->G, var_floor, w.lpar, w.lst, w.lnll);
    const size_t sm = sizeof(float) * ((size_t)n->G + 2 * (size_t)n->G * n->D + (size_t)kLossPts * (n->D | 1) +
                                       (size_t)kLossPts * (n->G + 1) + kLossPts);
    CKE(cudaFuncSetAttribute(k_loss_chunk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    k_loss_chunk<<<dim3(B, (P + kLossPts - 1) / kLossPts), kLossPts, sm, s>>>(pts, P, n->D, n->G, w.lpar, w.lst, w.lnll);
    const size_t smg = sizeof(float) * 2 * (size_t)n->G * n->D;
    if (smg > 48 * 1024) CKE(cudaFuncSetAttribute(k_loss_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smg));
    k_loss_grad<<<B, 256, smg, s>>>(w.lpar, w.lst, w.lnll, P, n->D, n->G, var_floor, tm, tv, tw, lambda, w.dout, w.loss,
                                    pm, pv, pw, B);
    count_launches(3);
    CKE(cudaGetLastError());
    if (grads) CKE(net_backward(*n, B, P, w, s));
    if (grads && lr > 0.0) {
        ++n->step;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - std::pow(b1, (float)n->step), c2 = 1.f - std::pow(b2, (float)n->step);
        k_adam<<<blocks_for(n->n_params, 256), 256, 0, s>>>(n->wgt, n->grad, n->m1, n->m2, n->wbf, n->n_params, (float)lr,
                                                            b1, b2, 1e-8f, c1, c2);
        count_launches(1);
        CKE(cudaGetLastError());
    }
    int herr = 0;
    CKE(cudaMemcpyAsync(&herr, n->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (loss_host) {
        std::vector<float> l(B);
        CKE(cudaMemcpyAsync(l.data(), w.loss, 4 * (size_t)B, cudaMemcpyDeviceToHost, s));
        CKE(cudaStreamSynchronize(s));
        double t = 0.0;
        for (int b = 0; b < B; ++b) t += l[b];
        *loss_host = t / B;
    } else {
        CKE(cudaStreamSynchronize(s));
    }
    if (herr) {
        cudaMemsetAsync(n->err, 0, sizeof(int), s);
        return cudaErrorLaunchTimeout;   // a bounded wait of a tensor-core GEMM ran out
    }
    return cudaSuccess;
}

}  // namespace gmm
