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
//     A Gaussian whose upper bound lies more than 27.7 nats below the best
//     lower bound has responsibility < 1e-12 and is dropped.
//  3. The few remaining candidates (about one per sample on speech-like data)
//     get their log-density recomputed exactly in FP32 on the CUDA cores (the
//     same formula as the FP32 form); log-sum-exp over them (Eqs. 16-18),
//     responsibilities l_{g,i} (Eq. 3), and the M-step statistics (Eqs. 9-11,
//     shifted by the FP32 mean of the iteration start) accumulated in shared
//     memory.  Responsibilities never leave the SM.
// Warp roles: warps 0-7 are the epilogue (warp w reads TMEM lanes 32*(w%4)..,
// i.e. samples 32*(w%4).., Gaussians 128*(w/4)..), warp 8 allocates TMEM and
// one of its threads issues the MMAs.  Every wait is bounded: on expiry the
// CTA records GMM_ERR_TIMEOUT, stops issuing work, drains, frees TMEM and
// returns.
#include <cuda_bf16.h>

#include "gmm_internal.cuh"

namespace gmm {

namespace {

constexpr int kEpiThreads = 256;
constexpr int kThreads = kEpiThreads + 32;
constexpr int kTM = 128;          // samples per tile = MMA M
constexpr int kCap = 8;           // candidates per thread before the dense fallback
constexpr float kScreenNats = 27.7f;
constexpr float kK1 = 0.009765625f * 1.25f / 1.0f;   // 2^-7 * 1.25 (multiplies |P1|)

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

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&v);
}

// The FP32 log-density of the CUDA-core form, term for term.
template <int DMAX>
__device__ __forceinline__ float exact_logit(const float (&xr)[DMAX], const float2 *__restrict__ p, float c, int D)
{
    float acc = 0.f;
#pragma unroll
    for (int d = 0; d < DMAX; ++d) {
        if (d < D) {
            const float2 q = __ldg(p + d);
            const float t = fmaf(xr[d], q.x, -q.y);
            acc = fmaf(t, t, acc);
        }
    }
    return fmaf(-0.5f, acc, c);
}

template <int DMAX>
__device__ __forceinline__ void load_row(float (&xr)[DMAX], const float *__restrict__ row, bool valid, int D)
{
#pragma unroll
    for (int d = 0; d < DMAX; ++d) xr[d] = (valid && d < D) ? __ldg(row + d) : 0.f;
}

struct TcArgs {
    EmPassArgs a;
    int32_t NG;   // Gaussians padded to a multiple of 16 (MMA N)
    int32_t nk;   // K=16 steps per K block: ceil(D/16)
};

struct TcSmem {
    uint32_t B, A, acc, cst, ctr, xlo, xms, clist, bars, misc, total;
};

__host__ __device__ inline TcSmem tc_layout(int D, int G, int NG)
{
    TcSmem L;
    uint32_t o = 0;
    L.B = o; o += 2u * NG * 128u;                       // two K blocks of [NG][128 B]
    L.A = o; o += kTM * 256u;                            // two K blocks of [128][128 B]
    L.acc = o; o += 4u * (uint32_t)(G + 2 * G * D); o = (o + 15u) & ~15u;
    if (o - L.acc < 128u) o = L.acc + 128u;              // also holds the 9 per-warp log-likelihoods
    L.cst = o; o += 8u * NG;                             // (ctc, k2) per Gaussian
    L.ctr = o; o += 4u * 64u;                            // centre
    L.xlo = o; o += 4u * 2u * kTM;
    L.xms = o; o += 8u * 2u * kTM;
    L.clist = o; o += (uint32_t)kEpiThreads * kCap;
    o = (o + 7u) & ~7u;
    L.bars = o; o += 8u * 4u;
    L.misc = o; o += 16u;
    L.total = o;
    return L;
}

template <int DMAX>
__global__ void __launch_bounds__(kThreads, 1) k_em_pass_tc(TcArgs args)
{
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    const EmPassArgs &a = args.a;
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = (a.status->halt != 0 || a.iter > a.status->stop_after) ? 1 : 0;
    __syncthreads();
    if (s_skip) return;   // uniform across the block
    const int D = a.D, G = a.G, NG = args.NG, nk = args.nk;
    const TcSmem Ls = tc_layout(D, G, NG);
    unsigned char *sbase = tc_raw + ((1024u - (smem_u32(tc_raw) & 1023u)) & 1023u);
    unsigned char *sB = sbase + Ls.B;
    unsigned char *sA = sbase + Ls.A;
    float *S0 = reinterpret_cast<float *>(sbase + Ls.acc);
    float *S1 = S0 + G;
    float *S2 = S1 + (size_t)G * D;
    float2 *cst = reinterpret_cast<float2 *>(sbase + Ls.cst);
    float *ctr = reinterpret_cast<float *>(sbase + Ls.ctr);
    float *xlo = reinterpret_cast<float *>(sbase + Ls.xlo);
    float2 *xms = reinterpret_cast<float2 *>(sbase + Ls.xms);
    uint8_t *clist = reinterpret_cast<uint8_t *>(sbase + Ls.clist);
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
        for (int k = tid; k < G + 2 * G * D; k += kEpiThreads) S0[k] = 0.f;
        // B operand: global [G][128] BF16 rows -> two swizzled K blocks
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
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    double ll = 0.0;
    unsigned long long st_kept = 0, st_dense = 0, st_n = 0;
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
                for (int kb = 0; kb < 2; ++kb)
                    for (int kk = 0; kk < nk; ++kk)
                        tc_mma(tmem + (uint32_t)(kb * 256), desc_k_sw128(aS + kb * 16384u + kk * 32u),
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
        const int s = 32 * q + lane;
        const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
        auto build_a = [&](int64_t tile) {
            const int64_t i0 = tile * kTM;
            const bool v = i0 + s < a.N;
            float xr[DMAX];
            load_row<DMAX>(xr, a.X + (i0 + s) * D, v, D);
            uint32_t w[32];
#pragma unroll
            for (int d = 0; d < DMAX; d += 2) {
                float x0 = (v && d < D) ? xr[d] - ctr[d] : 0.f;
                float x1 = (v && d + 1 < D) ? xr[d + 1] - ctr[d + 1] : 0.f;
                if (h == 0) { x0 *= x0; x1 *= x1; }
                w[d >> 1] = pack_bf16(x0, x1);
            }
            unsigned char *rowp = sA + h * 16384;
#pragma unroll
            for (int c = 0; c < 8; ++c)
                *reinterpret_cast<uint4 *>(rowp + sw128_off(s, c)) =
                    make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
        };
        if (T > 0) build_a(t0);
        fence_proxy_async();
        epi_sync();
        if (tid == 0 && T > 0) mbar_arrive(bar_afull);

        for (int t = 0; t < T; ++t) {
            const int64_t tile = t0 + t;
            const int64_t i = tile * kTM + s;
            const bool valid = i < a.N;
            mbar_wait(bar_lfull, (uint32_t)(t & 1), abort_flag, budget);
            tc_fence_after();
            // ---- pass 1: screening bounds from the two TMEM accumulators
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
            xlo[h * kTM + s] = lo;
            epi_sync();
            if (tid == 0) mbar_arrive(bar_lfree);
            lo = fmaxf(xlo[s], xlo[kTM + s]);
            // ---- pass 2: candidate list
            const float thr = lo - kScreenNats;
            int n = 0;
            uint8_t *my = clist + tid * kCap;
            const int gend = G - 128 * h;   // only real Gaussians (also when every bound is NaN/-inf)
#pragma unroll
            for (int j = 0; j < 128; ++j) {
                if (j < gend && ub[j] >= thr) {
                    if (n < kCap) my[n] = (uint8_t)j;
                    ++n;
                }
            }
            // ---- next tile's A operand (E(t) has finished reading the buffer)
            if (t + 1 < T) build_a(tile + 1);
            fence_proxy_async();
            epi_sync();
            if (tid == 0 && t + 1 < T) mbar_arrive(bar_afull);
            // ---- exact log-densities of the candidates, log-sum-exp, M-step
            float xr[DMAX];
            load_row<DMAX>(xr, a.X + i * D, valid, D);
            float lx[kCap];
            float mh = -INFINITY, sh = 0.f;
            const bool dense = n > kCap;
            if (valid) { st_n += 1; st_kept += (unsigned long long)n; st_dense += dense ? 1ull : 0ull; }
            if (!dense) {
#pragma unroll
                for (int k = 0; k < kCap; ++k) {
                    lx[k] = -INFINITY;
                    if (k < n) {
                        const int g = 128 * h + my[k];
                        lx[k] = exact_logit<DMAX>(xr, a.op.sm + (size_t)g * D, __ldg(a.op.c + g), D);
                        mh = fmaxf(mh, lx[k]);
                    }
                }
#pragma unroll
                for (int k = 0; k < kCap; ++k)
                    if (k < n) sh += __expf(lx[k] - mh);
            } else {
                const int ge = min(G, 128 * h + 128);
                for (int g = 128 * h; g < ge; ++g) {
                    const float l = exact_logit<DMAX>(xr, a.op.sm + (size_t)g * D, __ldg(a.op.c + g), D);
                    if (l > mh) { sh = sh * __expf(mh - l) + 1.f; mh = l; }
                    else sh += __expf(l - mh);
                }
            }
            xms[h * kTM + s] = make_float2(mh, sh);
            epi_sync();
            const float2 o = xms[(1 - h) * kTM + s];
            const float M = fmaxf(mh, o.x);
            const float S = (mh == -INFINITY ? 0.f : sh * __expf(mh - M)) + (o.x == -INFINITY ? 0.f : o.y * __expf(o.x - M));
            const float lse = M + logf(S);
            if (valid) {
                if (h == 0) ll += (double)lse;
                auto accumulate = [&](int g, float l) {
                    const float gm = __expf(l - lse);
                    if (!(gm > 0.f)) return;
                    atomicAdd(&S0[g], gm);
                    const float *mu = a.op.mu + (size_t)g * D;
#pragma unroll
                    for (int d = 0; d < DMAX; ++d) {
                        if (d < D) {
                            const float u = xr[d] - __ldg(mu + d);
                            const float gu = gm * u;
                            atomicAdd(&S1[g * D + d], gu);
                            atomicAdd(&S2[g * D + d], gu * u);
                        }
                    }
                };
                if (!dense) {
#pragma unroll
                    for (int k = 0; k < kCap; ++k)
                        if (k < n) accumulate(128 * h + my[k], lx[k]);
                } else {
                    const int ge = min(G, 128 * h + 128);
                    for (int g = 128 * h; g < ge; ++g)
                        accumulate(g, exact_logit<DMAX>(xr, a.op.sm + (size_t)g * D, __ldg(a.op.c + g), D));
                }
            }
        }
        tc_fence_before();
    }
    __syncthreads();
    // ---- flush the CTA's statistics (same layout as the FP32 form)
    if (warp < 8) {
        const int S = 1 + 2 * D;
        double *P = a.partial + (size_t)blockIdx.x * G * S;
        for (int k = tid; k < G * S; k += kEpiThreads) {
            const int g = k / S, j = k - g * S;
            P[k] = j == 0 ? (double)S0[g] : (j <= D ? (double)S1[g * D + j - 1] : (double)S2[g * D + j - 1 - D]);
        }
    }
    double *red = reinterpret_cast<double *>(sbase + Ls.acc);   // statistics already flushed
    __syncthreads();
    if (a.screen_stats && warp < 8) {
        for (int o = 16; o > 0; o >>= 1) {
            st_n += __shfl_xor_sync(0xffffffffu, st_n, o);
            st_kept += __shfl_xor_sync(0xffffffffu, st_kept, o);
            st_dense += __shfl_xor_sync(0xffffffffu, st_dense, o);
        }
        if (lane == 0) {
            atomicAdd(a.screen_stats + 0, (warp < 4) ? st_n : 0ull);   // each sample counted once (half 0)
            atomicAdd(a.screen_stats + 1, st_kept);
            atomicAdd(a.screen_stats + 2, st_dense);
        }
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
    return tc_layout(D, G, NG).total + 1024u <= (uint32_t)optin;
}

int em_tc_grid(int sms) { return sms; }

cudaError_t launch_em_pass_tc(const EmPassArgs &a, int32_t grid, int32_t split, cudaStream_t s)
{
    if (split) return cudaErrorNotSupported;
    TcArgs t{a, (a.G + 15) / 16 * 16, (a.D + 15) / 16};
    const size_t sm = tc_layout(a.D, a.G, t.NG).total + 1024u;
    cudaError_t e = cudaFuncSetAttribute(k_em_pass_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_em_pass_tc<64><<<grid, kThreads, sm, s>>>(t);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gmm
