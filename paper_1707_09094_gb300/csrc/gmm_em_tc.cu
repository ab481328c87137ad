// Tensor-core (tcgen05, sm_103a) fused EM pass.
//
// Per 128-sample tile of the CTA's contiguous chunk (the paper's thread t):
//  1. E-step contraction on the tensor cores, BF16 operands, FP32 accumulators
//     in TMEM, split into the two halves of the expanded log-density (Eq. 15
//     expanded about the global centre m, x' = x - m, mu' = mu - m):
//        P1[i][g] = sum_d x'^2 (-1/2 iv_gd)      (K block 0, TMEM columns 0..255)
//        P2[i][g] = sum_d x'   (mu'_gd iv_gd)    (K block 1, TMEM columns 256..511)
//     so l~_g(x_i) = ctc_g + P1 + P2 approximates log w_g N(x_i|g).
//  2. Screening with a rigorous bound: with BF16 rounding of both operands,
//     |l~ - l| <= 2^-8 * 1.25 * sum_d (x'^2 iv/2 + |x' mu'| iv) + tiny terms,
//     and by AM-GM sum_d |x' mu'| iv <= sum_d (x'^2 + mu'^2) iv / 2, so
//     |l~ - l| <= K1 |P1| + k2_g with k2_g = 2^-8 * 1.25 * q_g / 2 + ...
//     A Gaussian whose upper bound lies more than T = ln(N * 1e9) nats below
//     the best lower bound (35 nats at N = 2e6) has responsibility below
//     1e-9 / N and is dropped: per Gaussian the dropped mass is below 1e-9,
//     under the 1e-8 responsibility sum below which the update keeps a
//     Gaussian's parameters.
//  3. The few remaining candidates (one to a few per sample on speech-like
//     data) get their log-density recomputed exactly in FP32 on the CUDA
//     cores, one warp per (sample, Gaussian) with lanes over dimensions;
//     log-sum-exp over them (Eqs. 16-18), responsibilities l_{g,i} (Eq. 3),
//     and the M-step statistics (Eqs. 9-11, shifted by the FP32 mean of the
//     iteration start) reduced into the CTA's FP32 slab in L2 with
//     fire-and-forget atomics.  Responsibilities are never stored.
// Pipelining: A (the BF16 sample operand) and the FP32 sample tile (cp.async)
// are double-buffered, so the MMAs of tile t+1 run while tile t is screened,
// recomputed and accumulated.
// Warp roles: warps 0-7 are the epilogue (warp w reads TMEM lanes 32*(w%4)..,
// i.e. samples 32*(w%4).., Gaussians 128*(w/4)..), warp 8 allocates TMEM and
// one of its threads issues the MMAs.  Every wait is bounded: on expiry the
// CTA records GMM_ERR_TIMEOUT, stops issuing work, drains, frees TMEM and
// returns.
#include <cuda_bf16.h>

#include <cmath>

#include "gmm_internal.cuh"

namespace gmm {

namespace {

constexpr int kEpiThreads = 256;
constexpr int kThreads = kEpiThreads + 32;
constexpr int kTM = 128;          // samples per tile = MMA M
constexpr int kCap = 16;          // candidates per (sample, half) before the dense fallback
constexpr int kNB = 8;            // candidates a warp recomputes at once
constexpr float kK1 = 0.009765625f * 1.25f;   // 2^-7 * 1.25 (multiplies |P1|)

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

// Exact FP32 log-density of one Gaussian at one sample by one thread (the
// formula of the CUDA-core form: c_g - 1/2 sum_d (x_d s_gd - mu_gd s_gd)^2);
// x is the sample's row in shared memory.  Used by the dense path.
__device__ __forceinline__ float thread_logit(const float *x, const float2 *__restrict__ p, float c, int D)
{
    float acc = 0.f;
    for (int d = 0; d < D; ++d) {
        const float2 q = __ldg(p + d);
        const float t = fmaf(x[d], q.x, -q.y);
        acc = fmaf(t, t, acc);
    }
    return fmaf(-0.5f, acc, c);
}

// M-step contribution of one (sample, Gaussian) pair with responsibility gm
// (Eqs. 9-11 about the shift tc_shift of the BF16 operand row of g in shared
// memory): one warp; lane k adds (gm u, gm u^2) for dimensions 2k and 2k+1 as
// one 16-byte vector atomic (CUDA's float4 atomicAdd, compute capability
// >= 9.0) into the CTA's slab row [S0, pad x3 | (S1_d, S2_d) for d < DP].
__device__ __forceinline__ void smem_accumulate(float *slab_g, const float *x, const unsigned char *sB, int NG, int g,
                                                const float *ctr, float gm, int D, int DP, int lane)
{
    if (2 * lane < DP) {
        auto term = [&](int d, float &a1, float &a2) {
            float u = 0.f;
            if (d < D) {
                const uint32_t off = sw128_off(g, d >> 3) + (uint32_t)((d & 7) * 2);
                const __nv_bfloat16 b1 = *reinterpret_cast<const __nv_bfloat16 *>(sB + off);
                const __nv_bfloat16 b2 = *reinterpret_cast<const __nv_bfloat16 *>(sB + (uint32_t)NG * 128u + off);
                u = x[d] - tc_shift(ctr[d], b1, b2);
            }
            a1 = gm * u;
            a2 = a1 * u;
        };
        float4 v;
        term(2 * lane, v.x, v.y);
        term(2 * lane + 1, v.z, v.w);
        atomicAdd(reinterpret_cast<float4 *>(slab_g + 4 + 4 * lane), v);
    }
    if (lane == 31) atomicAdd(slab_g, gm);
}

__device__ __forceinline__ void cp_async4(uint32_t dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

struct TcArgs {
    EmPassArgs a;
    float *slab;      // [grid][G][1+2D] FP32 statistics of each CTA
    int32_t NG;       // Gaussians padded to a multiple of 16 (MMA N)
    int32_t nk;       // K=16 steps per K block: ceil(D/16)
    int32_t x_al16;   // X is 16-byte aligned
    float screen;     // screening distance in nats, ln(N * 1e9)
};

struct TcSmem {
    uint32_t B, A, X, xbytes, cst, ctr, cg, cl, cn, dms, xlo, xms, lse, bars, misc, total;
};

__host__ __device__ inline TcSmem tc_layout(int D, int G, int NG)
{
    (void)G;
    TcSmem L;
    uint32_t o = 0;
    L.B = o; o += 2u * NG * 128u;                        // two K blocks of [NG][128 B]
    L.A = o; o += 2u * kTM * 256u;                       // two buffers x two K blocks of [128][128 B]
    L.xbytes = ((uint32_t)kTM * D * 4u + 15u) & ~15u;
    L.X = o; o += 2u * L.xbytes;                         // two FP32 sample tiles
    L.cst = o; o += 8u * NG;                             // (ctc + k2, k2) per Gaussian
    L.ctr = o; o += 4u * 64u;                            // centre
    L.cg = o; o += (uint32_t)kEpiThreads * kCap;         // candidate Gaussian (local index)
    o = (o + 15u) & ~15u;
    L.cl = o; o += 4u * kEpiThreads * kCap;              // exact log-density, then responsibility
    L.cn = o; o += 4u * kEpiThreads;                     // candidates per (sample, half)
    L.dms = o; o += 8u * kEpiThreads;                    // dense path: (max, sum of exp)
    L.xlo = o; o += 4u * kEpiThreads;
    L.xms = o; o += 8u * kEpiThreads;
    L.lse = o; o += 4u * kTM;
    o = (o + 7u) & ~7u;
    L.bars = o; o += 8u * 4u;
    L.misc = o; o += 16u;
    L.total = o;
    return L;
}

__global__ void __launch_bounds__(kThreads, 1) k_em_pass_tc(TcArgs args)
{
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    const EmPassArgs &a = args.a;
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = (a.status->halt != 0 || a.iter > a.status->stop_after) ? 1 : 0;
    __syncthreads();
    if (s_skip) return;   // uniform across the block
    const int D = a.D, G = a.G, NG = args.NG, nk = args.nk, S = 1 + 2 * a.D;
    const TcSmem Ls = tc_layout(D, G, NG);
    unsigned char *sbase = tc_raw + ((1024u - (smem_u32(tc_raw) & 1023u)) & 1023u);
    unsigned char *sB = sbase + Ls.B;
    unsigned char *sA = sbase + Ls.A;
    float *sX = reinterpret_cast<float *>(sbase + Ls.X);
    float2 *cst = reinterpret_cast<float2 *>(sbase + Ls.cst);
    float *ctr = reinterpret_cast<float *>(sbase + Ls.ctr);
    uint8_t *cg = reinterpret_cast<uint8_t *>(sbase + Ls.cg);
    float *cl = reinterpret_cast<float *>(sbase + Ls.cl);
    int *cn = reinterpret_cast<int *>(sbase + Ls.cn);
    float2 *dms = reinterpret_cast<float2 *>(sbase + Ls.dms);
    float *xlo = reinterpret_cast<float *>(sbase + Ls.xlo);
    float2 *xms = reinterpret_cast<float2 *>(sbase + Ls.xms);
    float *slse = reinterpret_cast<float *>(sbase + Ls.lse);
    uint64_t *bar_afull = reinterpret_cast<uint64_t *>(sbase + Ls.bars);
    uint64_t *bar_lfull = bar_afull + 1;
    uint64_t *bar_lfree = bar_afull + 2;
    uint64_t *bar_drain = bar_afull + 3;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sbase + Ls.misc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sbase + Ls.misc + 4);
    float *slab = args.slab + (size_t)blockIdx.x * G * (4 + 2 * ((a.D + 3) & ~3));

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long budget = a.wait_cycles;
    const int DP = (D + 3) & ~3, SP = 4 + 2 * DP;     // padded slab row
    const int64_t ntiles = (a.N + kTM - 1) / kTM;
    const int64_t t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
    const int T = (int)(t1 - t0);

    // FP32 sample tile `tile` -> X buffer b (cp.async, one commit group per call)
    auto load_x = [&](int64_t tile, int b) {
        const int64_t i0 = tile * kTM;
        const int rows = (int)min((int64_t)kTM, a.N - i0);
        const uint32_t bytes = (uint32_t)rows * D * 4u;
        const char *src = reinterpret_cast<const char *>(a.X + i0 * D);
        const uint32_t dst = smem_u32(sbase + Ls.X + b * Ls.xbytes);
        uint32_t done = 0;
        if (args.x_al16) {
            const uint32_t n16 = bytes >> 4;
            for (uint32_t k = tid; k < n16; k += kEpiThreads) cp_async16(dst + 16u * k, src + 16u * k);
            done = n16 << 4;
        }
        for (uint32_t k = done / 4u + tid; k < bytes / 4u; k += kEpiThreads) cp_async4(dst + 4u * k, src + 4u * k);
        cp_async_commit();
    };
    // BF16 operand A of tile `tile` -> A buffer b: row r = [x'^2 | x'] (K blocks 0 | 1), warp per row
    auto build_a = [&](int64_t tile, int b) {
        const int64_t i0 = tile * kTM;
        unsigned char *ab = sA + b * (kTM * 256);
#pragma unroll
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
        for (int k = tid; k < G * SP; k += kEpiThreads) slab[k] = 0.f;
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
        load_x(t0, 0);
        build_a(t0, 0);
        fence_proxy_async();
    }
    __threadfence();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (tid == 0 && T > 0) mbar_arrive(bar_afull);

    double ll = 0.0;
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
        for (int t = 0; t < T; ++t) {
            const int64_t tile = t0 + t;
            const int64_t i0 = tile * kTM;
            const int nvalid = (int)min((int64_t)kTM, a.N - i0);
            // ---- prefetch the next tile: FP32 rows (async) and its BF16 operand
            if (t + 1 < T) {
                load_x(tile + 1, (t + 1) & 1);
                build_a(tile + 1, (t + 1) & 1);
                fence_proxy_async();
            } else {
                cp_async_commit();
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
            // ---- pass 2: candidate list of this (sample, half)
            const float thr = lo - args.screen;
            const int gend = G - 128 * h;   // only real Gaussians (also when every bound is NaN/-inf)
            int n = 0;
            uint8_t *my = cg + tid * kCap;
#pragma unroll
            for (int j = 0; j < 128; ++j) {
                if (j < gend && ub[j] >= thr) {
                    if (n < kCap) my[n] = (uint8_t)j;
                    ++n;
                }
            }
            if (s >= nvalid) n = 0;
            cn[tid] = n;
            if (s < nvalid) { st_n += (h == 0); st_kept += (unsigned long long)n; st_dense += n > kCap; }
            cp_async_wait1();   // this tile's FP32 rows have landed
            epi_sync();
            phase(4);
            const float *xt = sX + (t & 1) * (Ls.xbytes / 4u);
            // ---- exact log-densities: one warp per (sample, candidate), kNB
            // candidates at a time so that their parameter rows load together
            const int my_n = cn[32 * warp + lane];
            const unsigned dense_mask = __ballot_sync(0xffffffffu, my_n > kCap);
            for (int r = 0; r < kCap; ++r) {
                unsigned mask = __ballot_sync(0xffffffffu, my_n > r && my_n <= kCap);
                while (mask) {
                    int jj[kNB], gg[kNB];
                    bool vv[kNB];
#pragma unroll
                    for (int u = 0; u < kNB; ++u) {
                        vv[u] = mask != 0u;
                        jj[u] = vv[u] ? __ffs(mask) - 1 : 0;
                        if (vv[u]) mask &= mask - 1u;
                        gg[u] = vv[u] ? 128 * h + cg[(32 * warp + jj[u]) * kCap + r] : 0;
                    }
                    float2 pp[kNB][2];
                    float cc = 0.f;
#pragma unroll
                    for (int u = 0; u < kNB; ++u) {
                        if (lane == u && vv[u]) cc = __ldg(a.op.c + gg[u]);
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            const int d = lane + 32 * hh;
                            pp[u][hh] = (vv[u] && d < D) ? __ldg(a.op.sm + (size_t)gg[u] * D + d) : make_float2(0.f, 0.f);
                        }
                    }
                    float acc[kNB];
#pragma unroll
                    for (int u = 0; u < kNB; ++u) {
                        const float *x = xt + (32 * q + jj[u]) * D;
                        acc[u] = 0.f;
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            const int d = lane + 32 * hh;
                            if (vv[u] && d < D) {
                                const float tt = fmaf(x[d], pp[u][hh].x, -pp[u][hh].y);
                                acc[u] = fmaf(tt, tt, acc[u]);
                            }
                        }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                        for (int u = 0; u < kNB; ++u) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
                    // lane u writes candidate u (all lanes hold every reduced sum)
#pragma unroll
                    for (int u = 0; u < kNB; ++u)
                        if (lane == u && vv[u]) cl[(32 * warp + jj[u]) * kCap + r] = fmaf(-0.5f, acc[u], cc);
                }
            }
            // dense slots (candidate list overflowed): lanes over Gaussians
            for (unsigned dm = dense_mask; dm; dm &= dm - 1u) {
                const int j = __ffs(dm) - 1;
                const float *x = xt + (32 * q + j) * D;
                float m = -INFINITY, sm = 0.f;
                const int ge = min(G, 128 * h + 128);
                for (int g = 128 * h + lane; g < ge; g += 32) {
                    const float l = thread_logit(x, a.op.sm + (size_t)g * D, __ldg(a.op.c + g), D);
                    if (l > m) { sm = sm * __expf(m - l) + 1.f; m = l; }
                    else sm += __expf(l - m);
                }
                const float M = warp_max_f(m);
                sm = (m == -INFINITY) ? 0.f : sm * __expf(m - M);
                sm = warp_sum_f(sm);
                if (lane == 0) dms[32 * warp + j] = make_float2(M, sm);
            }
            phase(5);
            epi_sync();
            // ---- log-sum-exp per sample over both halves' candidates (Eqs. 16-18)
            float mh = -INFINITY, sh = 0.f;
            const float *myl = cl + tid * kCap;
            if (n <= kCap) {
                for (int k = 0; k < n; ++k) mh = fmaxf(mh, myl[k]);
                for (int k = 0; k < n; ++k) sh += __expf(myl[k] - mh);
            } else {
                const float2 v = dms[tid];
                mh = v.x;
                sh = v.y;
            }
            xms[tid] = make_float2(mh, sh);
            epi_sync();
            const float2 o = xms[(1 - h) * kTM + s];
            const float M = fmaxf(mh, o.x);
            const float Ssum = (mh == -INFINITY ? 0.f : sh * __expf(mh - M)) + (o.x == -INFINITY ? 0.f : o.y * __expf(o.x - M));
            const float lse = M + logf(Ssum);
            if (s < nvalid && h == 0) {
                ll += (double)lse;
                slse[s] = lse;
            }
            if (n <= kCap)
                for (int k = 0; k < n; ++k) cl[tid * kCap + k] = __expf(myl[k] - lse);   // Eq. 3
            epi_sync();
            // ---- M-step accumulation: one warp per (sample, candidate), kNB at a
            // time; the shift comes from the BF16 operand in shared memory
            for (int r = 0; r < kCap; ++r) {
                unsigned mask = __ballot_sync(0xffffffffu, my_n > r && my_n <= kCap);
                while (mask) {
#pragma unroll
                    for (int u = 0; u < kNB; ++u) {
                        if (!mask) break;
                        const int j = __ffs(mask) - 1;
                        mask &= mask - 1u;
                        const int slot = 32 * warp + j;
                        const int g = 128 * h + cg[slot * kCap + r];
                        const float gm = cl[slot * kCap + r];
                        if (gm > 0.f)
                            smem_accumulate(slab + (size_t)g * SP, xt + (32 * q + j) * D, sB, NG, g, ctr, gm, D, DP, lane);
                    }
                }
            }
            for (unsigned dm = dense_mask; dm; dm &= dm - 1u) {
                const int j = __ffs(dm) - 1;
                const float *x = xt + (32 * q + j) * D;
                const float ls = slse[32 * q + j];
                const int ge = min(G, 128 * h + 128);
                for (int g0 = 128 * h; g0 < ge; g0 += 32) {
                    const int g = g0 + lane;
                    const float gml = g < ge ? __expf(thread_logit(x, a.op.sm + (size_t)g * D, __ldg(a.op.c + g), D) - ls) : 0.f;
                    unsigned live = __ballot_sync(0xffffffffu, gml > 0.f);
                    while (live) {
                        const int src = __ffs(live) - 1;
                        live &= live - 1u;
                        const float gmv = __shfl_sync(0xffffffffu, gml, src);
                        smem_accumulate(slab + (size_t)(g0 + src) * SP, x, sB, NG, g0 + src, ctr, gmv, D, DP, lane);
                    }
                }
            }
            phase(6);
            epi_sync();
            phase(7);
        }
        tc_fence_before();
    }
    __threadfence();
    __syncthreads();
    // ---- the CTA's statistics (FP32 slab in L2) -> its FP64 partial
    if (warp < 8) {
        double *P = a.partial + (size_t)blockIdx.x * G * S;
        for (int k = tid; k < G * S; k += kEpiThreads) {
            const int g = k / S, j = k - g * S;
            const int src = j == 0 ? 0 : (j <= D ? 4 + 2 * (j - 1) : 4 + 2 * (j - 1 - D) + 1);
            P[k] = (double)__ldcg(slab + (size_t)g * SP + src);
        }
    }
    double *red = reinterpret_cast<double *>(sbase + Ls.cl);   // candidate storage is free now
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
    for (int o = 16; o > 0; o >>= 1) ll += __shfl_xor_sync(0xffffffffu, ll, o);
    if (lane == 0) red[warp] = ll;
    __syncthreads();
    if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < 9; ++w) tot += red[w];
        a.ll_partial[blockIdx.x] = tot;
        if (*abort_flag) {
            if (atomicCAS(&a.status->code, 0, (int)GMM_ERR_TIMEOUT) == 0) a.status->fail_iter = a.iter;
            atomicExch(&a.status->halt, 1);
        }
    }
    if (warp == 8) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

}  // namespace

bool em_tc_supported(int32_t D, int32_t G)
{
    if (D < 1 || D > 64 || G < 1 || G > 256) return false;
    const int NG = (G + 15) / 16 * 16;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return tc_layout(D, G, NG).total + 1024u + 64u <= (uint32_t)optin;
}

int em_tc_grid(int sms) { return sms; }

size_t em_tc_slab_floats(int32_t D, int32_t G, int grid) { return (size_t)grid * G * (4 + 2 * ((D + 3) & ~3)); }

cudaError_t launch_em_pass_tc(const EmPassArgs &a, float *slab, int32_t grid, cudaStream_t s)
{
    TcArgs t{a, slab, (a.G + 15) / 16 * 16, (a.D + 15) / 16, (reinterpret_cast<uintptr_t>(a.X) & 15u) == 0,
             (float)std::log((double)a.N * 1e9)};
    const size_t sm = tc_layout(a.D, a.G, t.NG).total + 1024u;
    cudaError_t e = cudaFuncSetAttribute(k_em_pass_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_em_pass_tc<<<grid, kThreads, sm, s>>>(t);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gmm
