// Tensor-core (tcgen05, sm_103a) EM pass in three kernels.
//
//  1. k_em_screen_tc -- per 128-sample tile of the CTA's chunk, the E-step
//     contraction on the tensor cores, BF16 operands, FP32 accumulators in
//     TMEM, split into the two halves of the log-density (Eq. 15) expanded
//     about the global centre m (x' = x - m, mu' = mu - m):
//        P1[i][g] = sum_d x'^2 (-1/2 iv_gd)      (K block 0, TMEM columns 0..255)
//        P2[i][g] = sum_d x'   (mu'_gd iv_gd)    (K block 1, TMEM columns 256..511)
//     so l~_g(x_i) = ctc_g + P1 + P2 approximates log w_g N(x_i|g).  With
//     BF16 rounding of both operands, |l~ - l| <= 2^-8 * 1.25 *
//     sum_d (x'^2 iv/2 + |x' mu'| iv) + tiny terms, and by AM-GM
//     sum_d |x' mu'| iv <= sum_d (x'^2 + mu'^2) iv / 2, so
//     |l~ - l| <= K1 |P1| + k2_g with k2_g = 2^-8 * 1.25 * q_g / 2 + ....
//     A Gaussian whose upper bound lies more than T = ln(N * 1e9) nats below
//     the best lower bound has responsibility below 1e-9 / N and is dropped
//     (per Gaussian the dropped mass is below 1e-9, under the 1e-8
//     responsibility sum below which the update keeps a Gaussian's
//     parameters).  Output per (sample, half of the Gaussians): the list of
//     surviving Gaussians (at most kTcCap, else the half is marked dense).
//  2. k_em_exact -- one warp per sample, lanes over dimensions, the
//     parameters in shared memory: the exact FP32 log-density of every
//     candidate (the formula of the CUDA-core form), of every Gaussian of a
//     dense half; log-sum-exp (Eqs. 16-18), log p(x_i) into the CTA's FP64
//     log-likelihood, responsibilities l_{g,i} (Eq. 3) of the candidates.
//  3. k_em_mstep_lists -- one CTA per (sample chunk, half of the Gaussians),
//     the paper's thread t: per 256-sample tile the (sample, Gaussian) pairs
//     are counting-sorted by Gaussian, and the warp that owns a Gaussian sums
//     l, l (x - mu_f), l (x - mu_f)^2 over its pairs in registers (Eqs. 9-11,
//     shifted by the FP32 mean mu_f of the iteration start) and adds them to
//     the CTA's FP32 statistics in shared memory (no atomics on them); the
//     chunk's statistics go to its FP64 partial once.
// Responsibilities exist only for the surviving pairs (a few per sample).
#include <cuda_bf16.h>

#include <cmath>

#include "gmm_internal.cuh"

namespace gmm {

namespace {

constexpr int kEpiThreads = 256;
constexpr int kThreads = kEpiThreads + 32;
constexpr int kTM = 128;          // samples per tile = MMA M
constexpr int kCap = kTcCap;      // candidates per (sample, half) before the dense fallback
constexpr float kK1 = 0.009765625f * 1.25f;   // 2^-7 * 1.25 (multiplies |P1|)
constexpr int kExThreads = 1024;  // exact-recompute kernel: 32 warps, one sample per warp at a time
constexpr int kMsThreads = 512;   // M-step kernel: 16 warps
constexpr int kMsTile = 256;      // samples per M-step tile

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase.  Gives up (and raises the CTA's abort
// flag) after ~1 s, or at once if another thread already aborted.
__device__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag, long long budget)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > budget) { *abort_flag = 1; return false; }
    }
    return true;
}

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major operand in the 128-byte swizzle
// layout: rows of 128 B (64 BF16 along K), 8-row atoms of 1024 B; SBO = 1024
// (next 8 rows), LBO unused for this layout, version field = 1, layout = 2.
__device__ __forceinline__ uint64_t desc_k_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: D F32, A and B BF16, both
// K-major, shape M x N.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of 16-byte chunk c of row r in a 128B-swizzled K-major tile.
__device__ __forceinline__ uint32_t sw128_off(int r, int c)
{
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4));
}


__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float warp_max_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}


__device__ __forceinline__ bool skip_block(const DevStatus *st, int iter)
{
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = (st->halt != 0 || iter > st->stop_after) ? 1 : 0;
    __syncthreads();
    return s_skip != 0;
}

struct TcArgs {
    EmPassArgs a;
    TcLists L;
    int32_t NG;       // Gaussians padded to a multiple of 16 (MMA N)
    int32_t nk;       // K=16 steps per K block: ceil(D/16)
    float screen;     // screening distance in nats, ln(N * 1e9)
};

struct TcSmem {
    uint32_t B, A, cst, ctr, cg, xlo, bars, misc, total;
};

__host__ __device__ inline TcSmem tc_layout(int NG)
{
    TcSmem L;
    uint32_t o = 0;
    L.B = o; o += 2u * NG * 128u;                        // two K blocks of [NG][128 B]
    L.A = o; o += 2u * kTM * 256u;                       // two buffers x two K blocks of [128][128 B]
    L.cst = o; o += 8u * NG;                             // (ctc, k2) per Gaussian
    L.ctr = o; o += 4u * 64u;                            // centre
    L.cg = o; o += (uint32_t)kEpiThreads * kCap;         // candidate list staging, 16 B per thread
    L.xlo = o; o += 4u * kEpiThreads;                    // best lower bound per (sample, half)
    o = (o + 7u) & ~7u;
    L.bars = o; o += 8u * 4u;
    L.misc = o; o += 16u;
    L.total = o;
    return L;
}

// ------------------------------------------------------------------------
// 1. Screening on the tensor cores.  Warp roles: warps 0-7 are the epilogue
// (warp w reads TMEM lanes 32*(w%4).., i.e. samples 32*(w%4).., Gaussians
// 128*(w/4)..), warp 8 allocates TMEM and one of its threads issues the
// MMAs.  The BF16 sample operand is double-buffered, so the MMAs of tile
// t+1 run while tile t is screened.  Every wait is bounded: on expiry the
// CTA records GMM_ERR_TIMEOUT, stops issuing work, drains, frees TMEM and
// returns.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 1) k_em_screen_tc(TcArgs args)
{
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    const EmPassArgs &a = args.a;
    if (skip_block(a.status, a.iter)) return;   // uniform across the block
    const int D = a.D, G = a.G, NG = args.NG, nk = args.nk;
    const TcSmem Ls = tc_layout(NG);
    unsigned char *sbase = tc_raw + ((1024u - (smem_u32(tc_raw) & 1023u)) & 1023u);
    unsigned char *sB = sbase + Ls.B;
    unsigned char *sA = sbase + Ls.A;
    float2 *cst = reinterpret_cast<float2 *>(sbase + Ls.cst);
    float *ctr = reinterpret_cast<float *>(sbase + Ls.ctr);
    uint8_t *cg = reinterpret_cast<uint8_t *>(sbase + Ls.cg);
    float *xlo = reinterpret_cast<float *>(sbase + Ls.xlo);
    uint64_t *bar_afull = reinterpret_cast<uint64_t *>(sbase + Ls.bars);
    uint64_t *bar_lfull = bar_afull + 1;
    uint64_t *bar_lfree = bar_afull + 2;
    uint64_t *bar_drain = bar_afull + 3;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sbase + Ls.misc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sbase + Ls.misc + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long budget = a.wait_cycles;
    const int64_t ntiles = (a.N + kTM - 1) / kTM;
    const int64_t t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
    const int T = (int)(t1 - t0);

    // BF16 operand A of tile `tile` -> A buffer b: row r = [x'^2 | x'] (K blocks 0 | 1), warp per row
    auto build_a = [&](int64_t tile, int b) {
        const int64_t i0 = tile * kTM;
        unsigned char *ab = sA + b * (kTM * 256);
#pragma unroll 4
        for (int i = 0; i < kTM / 8; ++i) {
            const int r = warp + 8 * i;
            const bool v = i0 + r < a.N;
            const float *row = a.X + (i0 + r) * D;
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int d = lane + 32 * hh;
                const float xc = (v && d < D) ? __ldcs(row + d) - ctr[d] : 0.f;
                const uint32_t off = sw128_off(r, d >> 3) + (uint32_t)((d & 7) * 2);
                *reinterpret_cast<__nv_bfloat16 *>(ab + off) = __float2bfloat16_rn(xc * xc);
                *reinterpret_cast<__nv_bfloat16 *>(ab + 16384 + off) = __float2bfloat16_rn(xc);
            }
        }
    };

    if (tid == 0) {
        mbar_init(bar_afull, 1);
        mbar_init(bar_lfull, 1);
        mbar_init(bar_lfree, 1);
        mbar_init(bar_drain, 1);
        *abort_flag = 0;
    }
    if (warp == 8) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    } else {
        for (int k = tid; k < NG * 16; k += kEpiThreads) {
            const int g = k >> 4, kb = (k >> 3) & 1, c = k & 7;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (g < G) v = __ldg(reinterpret_cast<const uint4 *>(a.op.B + (size_t)g * 128 + kb * 64) + c);
            *reinterpret_cast<uint4 *>(sB + (uint32_t)kb * NG * 128u + sw128_off(g, c)) = v;
        }
        for (int g = tid; g < NG; g += kEpiThreads) {
            if (g < G) {
                const float ct = __ldg(a.op.ctc + g);
                // 2^-8 * 1.25 * q/2  +  2^-21 |ctc|  +  1e-4
                const float k2 = 0.00390625f * 1.25f * 0.5f * __ldg(a.op.q + g) + 4.76837158203125e-07f * fabsf(ct) + 1e-4f;
                cst[g] = make_float2(ct, k2);
            } else {
                cst[g] = make_float2(-INFINITY, 0.f);
            }
        }
        for (int d = tid; d < 64; d += kEpiThreads) ctr[d] = d < D ? __ldg(a.center + d) : 0.f;
    }
    __syncthreads();   // centre in place for the first A
    if (warp < 8 && T > 0) {
        build_a(t0, 0);
        fence_proxy_async();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (tid == 0 && T > 0) mbar_arrive(bar_afull);

    unsigned long long st_kept = 0, st_dense = 0, st_n = 0;
    unsigned long long tp[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // phase cycles (thread 0, profiling only)
    long long tmark = clock64();
    auto phase = [&](int k) {
        const long long now = clock64();
        tp[k] += (unsigned long long)(now - tmark);
        tmark = now;
    };
    if (warp == 8) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(kTM, NG);
            const uint32_t aS = smem_u32(sA), bS = smem_u32(sB);
            for (int t = 0; t < T; ++t) {
                if (!mbar_wait(bar_afull, (uint32_t)(t & 1), abort_flag, budget)) break;
                if (t > 0 && !mbar_wait(bar_lfree, (uint32_t)((t - 1) & 1), abort_flag, budget)) break;
                tc_fence_after();
                if (a.skip_mma) continue;   // test hook: the epilogue's wait must run out
                const uint32_t ab = aS + (uint32_t)(t & 1) * (kTM * 256u);
                for (int kb = 0; kb < 2; ++kb)
                    for (int kk = 0; kk < nk; ++kk)
                        tc_mma(tmem + (uint32_t)(kb * 256), desc_k_sw128(ab + kb * 16384u + kk * 32u),
                               desc_k_sw128(bS + (uint32_t)kb * NG * 128u + kk * 32u), idesc, kk > 0 ? 1u : 0u);
                tc_commit(bar_lfull);
            }
            // drain: every MMA issued above must be complete before TMEM is
            // freed, so this wait ignores the abort flag (it is still bounded)
            tc_commit(bar_drain);
            const long long d0 = clock64();
            while (!mbar_try_wait(bar_drain, 0u) && clock64() - d0 < budget) {
            }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3, h = warp >> 2;
        const int s = 32 * q + lane;            // this thread's sample in the tile (TMEM lane)
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
        uint8_t *my = cg + tid * kCap;
        for (int t = 0; t < T; ++t) {
            const int64_t tile = t0 + t;
            const int64_t i0 = tile * kTM;
            const int nvalid = (int)min((int64_t)kTM, a.N - i0);
            // ---- the next tile's BF16 operand
            if (t + 1 < T) {
                build_a(tile + 1, (t + 1) & 1);
                fence_proxy_async();
            }
            phase(0);
            epi_sync();
            if (tid == 0 && t + 1 < T) mbar_arrive(bar_afull);
            phase(1);
            // ---- pass 1: screening bounds from the two TMEM accumulators
            mbar_wait(bar_lfull, (uint32_t)(t & 1), abort_flag, budget);
            tc_fence_after();
            phase(2);
            float ub[128];
            float lo = -INFINITY;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const int g0 = 128 * h + 16 * c;
                if (g0 < NG) {
                    uint32_t p1[16], p2[16];
                    tmem_ld16(tl + (uint32_t)g0, p1);
                    tmem_ld16(tl + 256u + (uint32_t)g0, p2);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float P1 = __uint_as_float(p1[j]), P2 = __uint_as_float(p2[j]);
                        const float2 k = cst[g0 + j];
                        const float l = (P1 + P2) + k.x;
                        const float e = fmaf(fabsf(P1), kK1, k.y);
                        ub[16 * c + j] = l + e;
                        lo = fmaxf(lo, l - e);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) ub[16 * c + j] = -INFINITY;
                }
            }
            tc_fence_before();
            phase(3);
            xlo[tid] = lo;
            epi_sync();
            if (tid == 0) mbar_arrive(bar_lfree);
            lo = fmaxf(xlo[s], xlo[kTM + s]);
            // ---- pass 2: candidate list of this (sample, half) -> global
            const float thr = lo - args.screen;
            const int gend = G - 128 * h;   // only real Gaussians (also when every bound is NaN/-inf)
            int n = 0;
#pragma unroll
            for (int j = 0; j < 128; ++j) {
                if (j < gend && ub[j] >= thr) {
                    if (n < kCap) my[n] = (uint8_t)j;
                    ++n;
                }
            }
            if (s < nvalid) {
                const int64_t rec = (i0 + s) * 2 + h;
                args.L.cnt[rec] = (uint8_t)min(n, 255);
                if (n > 0 && n <= kCap)
                    reinterpret_cast<uint4 *>(args.L.cand)[rec] = *reinterpret_cast<const uint4 *>(my);
                st_n += (h == 0);
                st_kept += (unsigned long long)n;
                st_dense += n > kCap;
            }
            phase(4);
        }
        tc_fence_before();
    }
    __syncthreads();
    if (a.screen_stats && warp < 8) {
        for (int o = 16; o > 0; o >>= 1) {
            st_n += __shfl_xor_sync(0xffffffffu, st_n, o);
            st_kept += __shfl_xor_sync(0xffffffffu, st_kept, o);
            st_dense += __shfl_xor_sync(0xffffffffu, st_dense, o);
        }
        if (lane == 0) {
            atomicAdd(a.screen_stats + 0, st_n);
            atomicAdd(a.screen_stats + 1, st_kept);
            atomicAdd(a.screen_stats + 2, st_dense);
        }
        if (tid == 0)
            for (int k = 0; k < 8; ++k) atomicAdd(a.screen_stats + 3 + k, tp[k]);
    }
    if (tid == 0 && *abort_flag) {
        if (atomicCAS(&a.status->code, 0, (int)GMM_ERR_TIMEOUT) == 0) a.status->fail_iter = a.iter;
        atomicExch(&a.status->halt, 1);
    }
    if (warp == 8) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// ------------------------------------------------------------------------
// 2. Exact log-densities, log-sum-exp and responsibilities of the screened
// candidates.  One CTA per SM, the FP32 operands (s, mu s) and c in shared
// memory; each warp takes one sample at a time, lanes over dimensions
// (D <= 64: dimensions lane and lane + 32).  Lane L of the warp holds the
// candidate in slot L & 15 of half L >> 4.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(kExThreads, 1) k_em_exact(EmPassArgs a, TcLists L)
{
    extern __shared__ __align__(16) unsigned char ex_raw[];
    if (skip_block(a.status, a.iter)) return;
    const int D = a.D, G = a.G;
    float2 *psm = reinterpret_cast<float2 *>(ex_raw);                  // [G][D]
    float *pc = reinterpret_cast<float *>(psm + (size_t)G * D);        // [G]
    float *xbuf = pc + ((G + 3) & ~3);                                 // [32 warps][64]
    __shared__ double s_ll[32];
    for (int k = threadIdx.x; k < G * D; k += blockDim.x) psm[k] = __ldg(a.op.sm + k);
    for (int g = threadIdx.x; g < G; g += blockDim.x) pc[g] = __ldg(a.op.c + g);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *xw = xbuf + warp * 64;
    const int64_t lo = a.N * blockIdx.x / gridDim.x, hi = a.N * (blockIdx.x + 1) / gridDim.x;
    double ll = 0.0;
    for (int64_t i = lo + warp; i < hi; i += kExThreads / 32) {
        const float *row = a.X + i * D;
        const float x0 = lane < D ? __ldg(row + lane) : 0.f;
        const float x1 = lane + 32 < D ? __ldg(row + 32 + lane) : 0.f;
        const int hL = lane >> 4, k = lane & 15;
        const int cnt2 = *reinterpret_cast<const uint16_t *>(L.cnt + 2 * i);
        const int n0 = cnt2 & 255, n1 = cnt2 >> 8;
        const int nh = hL ? n1 : n0;
        const bool valid = nh <= kCap && k < nh;
        const int g = valid ? 128 * hL + L.cand[i * 32 + lane] : 0;
        float logit = -INFINITY;
        unsigned mask = __ballot_sync(0xffffffffu, valid);
        while (mask) {
            int src[4], gg[4];
            bool vv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                vv[u] = mask != 0u;
                src[u] = vv[u] ? __ffs(mask) - 1 : 0;
                if (vv[u]) mask &= mask - 1u;
                gg[u] = __shfl_sync(0xffffffffu, g, src[u]);
            }
            float acc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float2 *p = psm + (size_t)gg[u] * D;
                float r = 0.f;
                if (lane < D) { const float2 q = p[lane]; const float t = fmaf(x0, q.x, -q.y); r = t * t; }
                if (lane + 32 < D) { const float2 q = p[lane + 32]; const float t = fmaf(x1, q.x, -q.y); r = fmaf(t, t, r); }
                acc[u] = r;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (vv[u] && lane == src[u]) logit = fmaf(-0.5f, acc[u], pc[gg[u]]);
        }
        // dense halves (more than kCap candidates): every Gaussian of the
        // half, lanes over Gaussians, online max / sum of exp per lane
        float dm = -INFINITY, ds = 0.f;
        if (n0 > kCap || n1 > kCap) {
            if (lane < D) xw[lane] = x0;
            if (lane + 32 < D) xw[lane + 32] = x1;
            __syncwarp();
            for (int hh = 0; hh < 2; ++hh) {
                if ((hh ? n1 : n0) <= kCap) continue;
                const int ge = min(G, 128 * hh + 128);
                for (int gd = 128 * hh + lane; gd < ge; gd += 32) {
                    const float2 *p = psm + (size_t)gd * D;
                    float r = 0.f;
                    for (int d = 0; d < D; ++d) {
                        const float2 q = p[d];
                        const float t = fmaf(xw[d], q.x, -q.y);
                        r = fmaf(t, t, r);
                    }
                    const float l = fmaf(-0.5f, r, pc[gd]);
                    if (l > dm) { ds = ds * __expf(dm - l) + 1.f; dm = l; }
                    else ds += __expf(l - dm);
                }
            }
            __syncwarp();
        }
        // log-sum-exp over the candidates and the dense halves (Eqs. 16-18)
        const float M = warp_max_f(fmaxf(logit, dm));
        float e = (logit == -INFINITY) ? 0.f : __expf(logit - M);
        if (dm != -INFINITY) e += ds * __expf(dm - M);
        const float lse = M + logf(warp_sum_f(e));
        if (valid) L.gam[i * 32 + lane] = __expf(logit - lse);   // Eq. 3
        if (lane == 0) {
            L.lse[i] = lse;
            ll += (double)lse;
        }
    }
    if (lane == 0) s_ll[warp] = ll;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < kExThreads / 32; ++w) tot += s_ll[w];
        a.ll_partial[blockIdx.x] = tot;
    }
}

// ------------------------------------------------------------------------
// 3. M-step statistics from the responsibility lists.  CTA b handles
// sample chunk b / 2 and half b % 2 of the Gaussians (at most 128).
// Shared memory: the chunk's FP32 statistics [128][1 + 2D] (S0 | S1_d |
// S2_d, shifted by mu_f), the per-tile bins of the counting sort.
// ------------------------------------------------------------------------
struct MsSmem {
    uint32_t slab, cnt, off, fill, pairs, scand, sn, dl, dn, xw, total;
};

__host__ __device__ inline MsSmem ms_layout(int D)
{
    MsSmem L;
    uint32_t o = 0;
    L.slab = o; o += 4u * 128u * (uint32_t)(1 + 2 * D);
    L.cnt = o; o += 4u * 128u;
    L.off = o; o += 4u * 132u;
    L.fill = o; o += 4u * 128u;
    L.scand = o; o += 16u * kMsTile;
    L.pairs = o; o += 2u * kMsTile * kCap;
    L.sn = o; o += (uint32_t)kMsTile;
    L.dl = o; o += 4u * kMsTile;
    L.dn = o; o += 16u;
    L.xw = o; o += 4u * 64u;
    L.total = o;
    return L;
}

__global__ void __launch_bounds__(kMsThreads, 2) k_em_mstep_lists(EmPassArgs a, TcLists L)
{
    extern __shared__ __align__(16) unsigned char ms_raw[];
    if (skip_block(a.status, a.iter)) return;
    const int D = a.D, G = a.G, S = 1 + 2 * D;
    const int h = blockIdx.x & 1, chunk = blockIdx.x >> 1, nchunks = gridDim.x >> 1;
    const int GH = max(0, min(128, G - 128 * h));
    if (GH == 0) return;
    const MsSmem Ls = ms_layout(D);
    float *slab = reinterpret_cast<float *>(ms_raw + Ls.slab);
    int *bcnt = reinterpret_cast<int *>(ms_raw + Ls.cnt);
    int *boff = reinterpret_cast<int *>(ms_raw + Ls.off);
    int *bfill = reinterpret_cast<int *>(ms_raw + Ls.fill);
    uint4 *scand = reinterpret_cast<uint4 *>(ms_raw + Ls.scand);
    uint16_t *pairs = reinterpret_cast<uint16_t *>(ms_raw + Ls.pairs);
    uint8_t *sn = reinterpret_cast<uint8_t *>(ms_raw + Ls.sn);
    int *dl = reinterpret_cast<int *>(ms_raw + Ls.dl);
    int *dn = reinterpret_cast<int *>(ms_raw + Ls.dn);
    float *xw = reinterpret_cast<float *>(ms_raw + Ls.xw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int k = tid; k < 128 * S; k += kMsThreads) slab[k] = 0.f;
    const int64_t lo = a.N * chunk / nchunks, hi = a.N * (chunk + 1) / nchunks;
    const uint8_t *ccnt = L.cnt;
    for (int64_t i0 = lo; i0 < hi; i0 += kMsTile) {
        const int nt = (int)min((int64_t)kMsTile, hi - i0);
        if (tid < 128) { bcnt[tid] = 0; bfill[tid] = 0; }
        if (tid == 0) *dn = 0;
        __syncthreads();
        // ---- this half's list of each sample of the tile; histogram by Gaussian
        if (tid < nt) {
            const int64_t rec = (i0 + tid) * 2 + h;
            const int n = ccnt[rec];
            sn[tid] = (uint8_t)n;
            if (n > kCap) {
                dl[atomicAdd(dn, 1)] = tid;
            } else if (n > 0) {
                scand[tid] = reinterpret_cast<const uint4 *>(L.cand)[rec];
                const uint8_t *cb = reinterpret_cast<const uint8_t *>(scand + tid);
                for (int k = 0; k < n; ++k) atomicAdd(&bcnt[cb[k]], 1);
            }
        }
        __syncthreads();
        // ---- exclusive scan of the 128 bins (warp 0, four bins per lane)
        if (warp == 0) {
            const int4 v = reinterpret_cast<const int4 *>(bcnt)[lane];
            const int tot = v.x + v.y + v.z + v.w;
            int inc = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            const int ex = inc - tot;
            boff[4 * lane] = ex;
            boff[4 * lane + 1] = ex + v.x;
            boff[4 * lane + 2] = ex + v.x + v.y;
            boff[4 * lane + 3] = ex + v.x + v.y + v.z;
            if (lane == 31) boff[128] = inc;
        }
        __syncthreads();
        // ---- scatter the pairs (sample << 4 | slot) into their bins
        if (tid < nt) {
            const int n = sn[tid];
            if (n > 0 && n <= kCap) {
                const uint8_t *cb = reinterpret_cast<const uint8_t *>(scand + tid);
                for (int k = 0; k < n; ++k) {
                    const int gl = cb[k];
                    pairs[boff[gl] + atomicAdd(&bfill[gl], 1)] = (uint16_t)((tid << 4) | k);
                }
            }
        }
        __syncthreads();
        // ---- warp w owns Gaussians w, w + 16, ...: sums in registers, then
        // one read-modify-write of its rows of the CTA's statistics
        for (int gl = warp; gl < GH; gl += kMsThreads / 32) {
            const int pb = boff[gl], pe = boff[gl + 1];
            if (pb == pe) continue;
            const int g = 128 * h + gl;
            const float m0 = lane < D ? __ldg(a.op.mu + (size_t)g * D + lane) : 0.f;
            const float m1 = lane + 32 < D ? __ldg(a.op.mu + (size_t)g * D + 32 + lane) : 0.f;
            float s0 = 0.f, a1 = 0.f, a2 = 0.f, b1 = 0.f, b2 = 0.f;
            for (int p = pb; p < pe; ++p) {
                const int pr = pairs[p];
                const int64_t i = i0 + (pr >> 4);
                const float gm = __ldg(L.gam + i * 32 + 16 * h + (pr & 15));
                const float *row = a.X + i * D;
                if (lane < D) {
                    const float u = __ldg(row + lane) - m0;
                    const float v = gm * u;
                    a1 += v;
                    a2 = fmaf(v, u, a2);
                }
                if (lane + 32 < D) {
                    const float u = __ldg(row + 32 + lane) - m1;
                    const float v = gm * u;
                    b1 += v;
                    b2 = fmaf(v, u, b2);
                }
                s0 += gm;
            }
            float *sg = slab + (size_t)gl * S;
            if (lane == 0) sg[0] += s0;
            if (lane < D) { sg[1 + lane] += a1; sg[1 + D + lane] += a2; }
            if (lane + 32 < D) { sg[33 + lane] += b1; sg[33 + D + lane] += b2; }
        }
        __syncthreads();
        // ---- dense (sample, half) records: warp 0 recomputes every
        // Gaussian of the half exactly and adds the responsibilities > 0
        if (warp == 0) {
            const int nd = *dn;
            for (int r = 0; r < nd; ++r) {
                const int64_t i = i0 + dl[r];
                const float *row = a.X + i * D;
                const float x0 = lane < D ? __ldg(row + lane) : 0.f;
                const float x1 = lane + 32 < D ? __ldg(row + 32 + lane) : 0.f;
                if (lane < D) xw[lane] = x0;
                if (lane + 32 < D) xw[lane + 32] = x1;
                __syncwarp();
                const float ls = __ldg(L.lse + i);
                for (int gb = 0; gb < GH; gb += 32) {
                    const int gl = gb + lane;
                    float gm = 0.f;
                    if (gl < GH) {
                        const float2 *p = a.op.sm + (size_t)(128 * h + gl) * D;
                        float acc = 0.f;
                        for (int d = 0; d < D; ++d) {
                            const float2 q = __ldg(p + d);
                            const float t = fmaf(xw[d], q.x, -q.y);
                            acc = fmaf(t, t, acc);
                        }
                        gm = __expf(fmaf(-0.5f, acc, __ldg(a.op.c + 128 * h + gl)) - ls);
                    }
                    unsigned live = __ballot_sync(0xffffffffu, gm > 0.f);
                    while (live) {
                        const int src = __ffs(live) - 1;
                        live &= live - 1u;
                        const float gv = __shfl_sync(0xffffffffu, gm, src);
                        const int gg = gb + src;
                        const size_t gidx = (size_t)(128 * h + gg) * D;
                        float *sg = slab + (size_t)gg * S;
                        if (lane < D) {
                            const float u = x0 - __ldg(a.op.mu + gidx + lane);
                            const float v = gv * u;
                            sg[1 + lane] += v;
                            sg[1 + D + lane] = fmaf(v, u, sg[1 + D + lane]);
                        }
                        if (lane + 32 < D) {
                            const float u = x1 - __ldg(a.op.mu + gidx + 32 + lane);
                            const float v = gv * u;
                            sg[33 + lane] += v;
                            sg[33 + D + lane] = fmaf(v, u, sg[33 + D + lane]);
                        }
                        if (lane == 0) sg[0] += gv;
                        __syncwarp();
                    }
                }
                __syncwarp();
            }
        }
        __syncthreads();
    }
    // ---- the chunk's statistics of this half -> its FP64 partial
    double *P = a.partial + ((size_t)chunk * G + 128 * h) * S;
    for (int k = tid; k < GH * S; k += kMsThreads) P[k] = (double)slab[k];
}

}  // namespace

bool em_tc_supported(int32_t D, int32_t G)
{
    if (D < 1 || D > 64 || G < 1 || G > 256) return false;
    const int NG = (G + 15) / 16 * 16;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t ex = (size_t)G * D * 8u + 4u * (size_t)((G + 3) & ~3) + 32u * 64u * 4u;
    return tc_layout(NG).total + 1024u + 64u <= (uint32_t)optin && ex <= (size_t)optin &&
           ms_layout(D).total <= (uint32_t)optin;
}

int em_tc_grid(int sms) { return sms; }

size_t em_tc_list_bytes(int64_t N) { return (size_t)N * (32u + 2u + 128u + 4u) + 1024u; }

TcLists em_tc_lists(void *base, int64_t N)
{
    unsigned char *p = static_cast<unsigned char *>(base);
    TcLists L;
    L.gam = reinterpret_cast<float *>(p);                 // [N][2][16] FP32 (16-byte aligned rows)
    p += (size_t)N * 128u;
    L.cand = p;                                           // [N][2][16] Gaussian index within the half
    p += (size_t)N * 32u;
    L.lse = reinterpret_cast<float *>(p);                 // [N]
    p += (size_t)N * 4u;
    L.cnt = p;                                            // [N][2] candidates (> kTcCap: dense)
    return L;
}

cudaError_t launch_em_pass_tc(const EmPassArgs &a, const TcLists &L, int32_t grid, int32_t ms_chunks, cudaStream_t s)
{
    TcArgs t{a, L, (a.G + 15) / 16 * 16, (a.D + 15) / 16, (float)std::log((double)a.N * 1e9)};
    const size_t sm1 = tc_layout(t.NG).total + 1024u;
    cudaError_t e = cudaFuncSetAttribute(k_em_screen_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    if (e != cudaSuccess) return e;
    k_em_screen_tc<<<grid, kThreads, sm1, s>>>(t);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t sm2 = (size_t)a.G * a.D * 8u + 4u * (size_t)((a.G + 3) & ~3) + 32u * 64u * 4u;
    if ((e = cudaFuncSetAttribute(k_em_exact, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2)) != cudaSuccess)
        return e;
    k_em_exact<<<grid, kExThreads, sm2, s>>>(a, L);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t sm3 = ms_layout(a.D).total;
    if ((e = cudaFuncSetAttribute(k_em_mstep_lists, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3)) !=
        cudaSuccess)
        return e;
    k_em_mstep_lists<<<2 * ms_chunks, kMsThreads, sm3, s>>>(a, L);
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace gmm
