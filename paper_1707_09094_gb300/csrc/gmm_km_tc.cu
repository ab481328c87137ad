// Tensor-core (tcgen05, sm_103a) k-means map step for D <= 64, N_G <= 256.
//
// The nearest mean under the distance sum_d w_d (x_d - mu_gd)^2 (Sec. 3,
// map step; w = 1 Euclidean, w = 1/sigma_d^2 Mahalanobis) minimises, in the
// scaled coordinates X = (x - m) sqrt(w), C_g = (mu_g - m) sqrt(w) about the
// global mean m, the score S_g = |C_g|^2 - 2 X.C_g: the distance minus the
// common |X|^2.  Three kernels per iteration:
//
//  1. k_km_prep_tc -- per mean: c' = (mu - m) sqrt(w) in FP32, split into
//     BF16 parts c' = c_hi + c_lo + r; |c'|^2; the FP32 scaled mean
//     mu sqrt(w) and its squared norm (for the exact FP32 distance); the
//     FP32 mean mu_f (shift of the statistics).
//  2. k_km_screen_tc -- per 128-sample tile, the contraction x'.c' on the
//     tensor cores with split BF16 operands (x' = x_hi + x_lo + r):
//        P = x_hi c_hi + x_lo c_hi + x_hi c_lo        (FP32 accumulators in TMEM)
//     and the score s~_g = |c'_g|^2 - 2 P.  Rounding (u = 2^-24, BF16
//     splits: |r| <= 2^-16 |value|; every BF16 product exact in FP32):
//        dropped split terms           <= 3.1 * 2^-16 sum_d |x'_d c'_d|
//        FP32 accumulation (<= 192 products, taken as n * 2^-23)
//                                      <= 2^-15.4 sum_d |x'_d c'_d|
//        FP32 coordinates vs exact     <= 6u |X_d C_d| per term, 6u |C|^2
//        |c'|^2 in FP32 (D <= 64)      <= 2^-18 |c'|^2
//     so with sum_d |x'_d c'_d| <= |x'| |c'| (Cauchy-Schwarz)
//        |s~_g - S_g| <= 2^-12.7 |x'| |c'_g| + 2^-17.6 |c'_g|^2,
//     and e = 2^-12 |x'| max|c'| + 2^-16 (max|c'|^2 + |x'|^2) bounds it for
//     every mean, with room for the FP64 rounding of the distances the
//     definition is evaluated in.  The nearest mean is therefore among the
//     candidates s~_g <= min_h s~_h + 2e.  A sample with one candidate is
//     assigned at once (almost every sample); the others are recorded with
//     their candidates and decided after the CTA's last tile:
//  3. (same kernel, deferred) one warp per such sample: the exact FP32
//     distances sum_d (x_d s_d - mu_gd s_d)^2 of its candidates, lanes over
//     dimensions, under the rounding bound of the CUDA-core form; when the
//     best two are closer than that bound, the candidates that can still
//     win are re-decided in FP64 in the definition's own operation order
//     (lowest index on exact ties); more than 32 candidates, or none (a
//     non-finite sample), re-decide every mean in FP64.
//  4. k_km_stats -- from the assignment, count, sum(x - mu_f) and
//     sum((x - mu_f)^2) per mean into each CTA's FP64 partial: the sums of
//     Eqs. 5-7.
#include <cuda_bf16.h>

#include <climits>
#include <cmath>

#include "gmm_internal.cuh"
#include "tc_ptx.cuh"

namespace gmm {

namespace {

using namespace ptx;

constexpr int kEpi = 512;        // 16 epilogue warps
constexpr int kThr = kEpi + 32;  // + the MMA warp
constexpr int kTM = 128;         // samples per tile = MMA M
constexpr int kCap = 16;         // candidates per (sample, quarter of the means) kept in shared memory
constexpr int kListMax = 32;     // candidates per sample recorded for the deferred decision

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 512;" ::: "memory"); }

__device__ __forceinline__ float wsum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ bool km_skip(const DevStatus *st)
{
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = (st->halt != 0 || 0 > st->stop_after) ? 1 : 0;
    __syncthreads();
    return s_skip != 0;
}

// Rounding bound of an FP32 distance sum_d (xs_d - cs_d)^2 (xs, cs the FP32
// scaled coordinates, any summation order over <= D terms); norms bounds
// |xs|^2 + |cs|^2.  The bound the CUDA-core form decides with.
__device__ __forceinline__ float dist_err(float d, float norms, int D)
{
    return 4.0f * (2.384185791015625e-07f * sqrtf(2.0f * d * norms) + (float)(D + 4) * 5.9604644775390625e-08f * d) +
           1e-30f;
}

// The definition's distance in FP64: sum over d = 0..D-1, in order, of
// w_d (x_d - mu_d)^2, no fused operations.
__device__ __forceinline__ double dist_fp64(const float *__restrict__ x, const double *__restrict__ mu,
                                            const double *__restrict__ w, int D)
{
    double acc = 0.0;
    for (int d = 0; d < D; ++d) {
        const double t = __dsub_rn((double)__ldg(x + d), mu[d]);
        acc = __dadd_rn(acc, __dmul_rn(w[d], __dmul_rn(t, t)));
    }
    return acc;
}

// Warp argmin of (value, index), lowest index on equal values; INT_MAX when
// no lane holds a value below +inf (every distance non-finite).
__device__ __forceinline__ int warp_argmin_fp64(double bv, int bi)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov < bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    return bi;
}

// ------------------------------------------------------------------------
// 1. Operands of one iteration, one block of 64 threads per mean.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(64) k_km_prep_tc(const double *__restrict__ means, const float *__restrict__ sw,
                                                   const float *__restrict__ center, int32_t D, int32_t G, KmTcOps o,
                                                   float *__restrict__ mu_f)
{
    const int g = blockIdx.x, d = threadIdx.x;
    float cp = 0.f, cs = 0.f;
    if (d < D) {
        const double mu = means[(size_t)g * D + d];
        const double s = (double)sw[d];
        cp = (float)((mu - (double)center[d]) * s);
        cs = (float)(mu * s);
        o.cs[(size_t)g * D + d] = cs;
        mu_f[(size_t)g * D + d] = (float)mu;
    }
    const __nv_bfloat16 hi = __float2bfloat16_rn(cp);
    const __nv_bfloat16 lo = __float2bfloat16_rn(cp - __bfloat162float(hi));   // cp - hi is exact in FP32
    o.B[(size_t)g * 128 + d] = hi;
    o.B[(size_t)g * 128 + 64 + d] = lo;
    __shared__ float s_n[2][2];
    const float a = wsum(cp * cp), b = wsum(cs * cs);
    if ((d & 31) == 0) { s_n[d >> 5][0] = a; s_n[d >> 5][1] = b; }
    __syncthreads();
    if (d == 0) {
        o.cn[g] = s_n[0][0] + s_n[1][0];
        o.ncs[g] = s_n[0][1] + s_n[1][1];
    }
}

struct KmTcArgs {
    const float *X;
    int64_t N;
    int32_t D, G, NG, nk;
    KmTcOps o;
    const double *means;   // FP64 means at the iteration start
    const double *w;       // [D] FP64 distance weights
    const float *sw;       // [D] FP32 sqrt(w)
    const float *center;   // [D] FP32 global mean
    int32_t *assign;
    TcLists L;
    DevStatus *status;
    long long wait_cycles;
    int32_t x_al16;
    int32_t x_v2;                // D even and X 8-byte aligned: rows read two dimensions at a time
    unsigned long long *stats;   // [3] samples screened, deferred, re-decided in FP64 (NULL = off)
};

struct KmSmem {
    uint32_t B, A, X, xstride, cn, ctr, swd, cg, cnt, xlo, xn, bars, misc, total;
};

__host__ __device__ inline KmSmem km_layout(int D, int NG)
{
    KmSmem L;
    uint32_t o = 0;
    L.B = o; o += 2u * (uint32_t)NG * 128u;              // K blocks c_hi | c_lo, [NG][128 B] each
    L.A = o; o += 2u * 2u * kTM * 128u;                  // two buffers x (x_hi | x_lo)
    L.xstride = ((4u * kTM * (uint32_t)D) + 127u) & ~127u;
    L.X = o; o += 2u * L.xstride;                        // two staged FP32 sample tiles
    L.cn = o; o += 4u * 256u;                            // |c'|^2 (+inf past the last mean)
    L.ctr = o; o += 4u * 64u;                            // centre
    L.swd = o; o += 4u * 64u;                            // sqrt(w)
    L.cg = o; o += (uint32_t)kEpi * kCap;                // candidate lists per (sample, quarter)
    L.cnt = o; o += 4u * kEpi;                           // their lengths
    L.xlo = o; o += 4u * kEpi;                           // best score per (sample, quarter)
    L.xn = o; o += 2u * kTM * 8u;                        // (|x'|, |x'|^2) per buffer and sample
    o = (o + 7u) & ~7u;
    L.bars = o; o += 8u * 9u;
    L.misc = o; o += 32u;
    L.total = o;
    return L;
}

__device__ __forceinline__ bool tile_bulk(int64_t i0, int64_t N, int x_al16) { return x_al16 && i0 + kTM <= N; }

__device__ __forceinline__ bool x_wait(uint64_t *bar, uint32_t parity, long long budget, volatile int *abort_flag)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > budget) { *abort_flag = 1; return false; }
    }
    return true;
}

// ------------------------------------------------------------------------
// 2./3. Screening on the tensor cores and the exact decision.  Warps 0-15
// are the epilogue (warp w: TMEM lanes / samples 32 (w % 4).., means
// 64 (w / 4)..+63), warp 16 allocates TMEM (two accumulators of 256
// columns) and one of its threads issues the MMAs.  Tile t uses A buffer,
// staged-X buffer and accumulator t & 1, each with its own barriers, so the
// MMAs of tile t+1 run while tile t is screened; each FP32 sample tile is
// staged by a bulk copy two tiles ahead of the operand built from it.
// Every wait is bounded: on expiry the CTA records GMM_ERR_TIMEOUT, stops
// issuing work, drains, frees TMEM and returns.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(kThr, 1) k_km_screen_tc(KmTcArgs a)
{
    extern __shared__ __align__(1024) unsigned char km_raw[];
    if (km_skip(a.status)) return;   // uniform across the block
    const int D = a.D, G = a.G, NG = a.NG, nk = a.nk;
    const KmSmem Ls = km_layout(D, NG);
    unsigned char *sbase = km_raw + ((1024u - (smem_u32(km_raw) & 1023u)) & 1023u);
    unsigned char *sB = sbase + Ls.B;
    unsigned char *sA = sbase + Ls.A;
    float *cn = reinterpret_cast<float *>(sbase + Ls.cn);
    float *ctr = reinterpret_cast<float *>(sbase + Ls.ctr);
    float *swd = reinterpret_cast<float *>(sbase + Ls.swd);
    uint8_t *cg = sbase + Ls.cg;
    int *cnt = reinterpret_cast<int *>(sbase + Ls.cnt);
    float *xlo = reinterpret_cast<float *>(sbase + Ls.xlo);
    float2 *xn = reinterpret_cast<float2 *>(sbase + Ls.xn);
    uint64_t *bar_afull = reinterpret_cast<uint64_t *>(sbase + Ls.bars);   // [2]
    uint64_t *bar_lfull = bar_afull + 2;                                    // [2]
    uint64_t *bar_lfree = bar_afull + 4;                                    // [2]
    uint64_t *bar_x = bar_afull + 6;                                        // [2]
    uint64_t *bar_drain = bar_afull + 8;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sbase + Ls.misc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sbase + Ls.misc + 4);
    int *namb = reinterpret_cast<int *>(sbase + Ls.misc + 8);
    int *n64 = reinterpret_cast<int *>(sbase + Ls.misc + 12);
    int *s_cnmax = reinterpret_cast<int *>(sbase + Ls.misc + 16);   // non-negative floats as ints
    int *s_nmax = reinterpret_cast<int *>(sbase + Ls.misc + 20);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long budget = a.wait_cycles;
    const int64_t ntiles = (a.N + kTM - 1) / kTM;
    const int64_t t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
    const int T = (int)(t1 - t0);
    const TcLists &L = a.L;
    uint32_t xuse0 = 0u, xuse1 = 0u;   // consumed staged tiles per buffer (epilogue threads)
    uint32_t xiss0 = 0u, xiss1 = 0u;   // issued staged tiles per buffer (thread 0)

    auto issue_x = [&](int t) {   // thread 0 only; buffer t & 1
        const int b = t & 1;
        if (b) ++xiss1; else ++xiss0;
        const uint32_t xb = 4u * kTM * (uint32_t)D;
        fence_proxy_async();
        mbar_expect_tx(bar_x + b, xb);
        bulk_g2s(sbase + Ls.X + (uint32_t)b * Ls.xstride, a.X + (t0 + t) * kTM * D, xb, bar_x + b);
    };
    // split BF16 operand of tile t -> A buffer t & 1, row r = x' (K block 0
    // x_hi, block 1 x_lo), warp per row, two dimensions per lane; (|x'|,
    // |x'|^2) per row.  Rows r = warp + 16 k share r & 7, so the swizzled
    // column offset of a lane is the same in every row.
    const uint32_t colo = ((uint32_t)((lane >> 2) ^ (warp & 7)) << 4) | (uint32_t)((lane & 3) * 4);
    const uint32_t rowo = (uint32_t)(warp >> 3) * 1024u + (uint32_t)(warp & 7) * 128u;
    auto build_a = [&](int t) {
        const int bb = t & 1;
        const int64_t i0 = (t0 + t) * kTM;
        const bool staged = tile_bulk(i0, a.N, a.x_al16);
        if (staged && x_wait(bar_x + bb, (bb ? xuse1 : xuse0) & 1u, budget, abort_flag)) {
            if (bb) ++xuse1; else ++xuse0;
        }
        const float *xt = reinterpret_cast<const float *>(sbase + Ls.X + (uint32_t)bb * Ls.xstride);
        unsigned char *ab = sA + bb * (2 * kTM * 128);
        float2 *xnb = xn + bb * kTM;
        const int d0 = 2 * lane;
        const float2 c2 = reinterpret_cast<const float2 *>(ctr)[lane];   // 0 past D
        const float2 s2 = reinterpret_cast<const float2 *>(swd)[lane];   // 0 past D
#pragma unroll 4
        for (int k = 0; k < kTM / 16; ++k) {
            const int r = warp + 16 * k;
            float x0 = 0.f, x1 = 0.f;
            if (i0 + r < a.N && d0 < D) {
                const float *src = staged ? xt + r * D + d0 : a.X + (i0 + r) * D + d0;
                if (a.x_v2) {   // D even and X 8-byte aligned
                    const float2 p = staged ? *reinterpret_cast<const float2 *>(src)
                                            : __ldg(reinterpret_cast<const float2 *>(src));
                    x0 = p.x;
                    x1 = p.y;
                } else {
                    x0 = staged ? src[0] : __ldg(src);
                    if (d0 + 1 < D) x1 = staged ? src[1] : __ldg(src + 1);
                }
            }
            const float xc0 = (x0 - c2.x) * s2.x, xc1 = (x1 - c2.y) * s2.y;
            const __nv_bfloat162 hi = __floats2bfloat162_rn(xc0, xc1);
            const float2 hf = __bfloat1622float2(hi);
            const __nv_bfloat162 lo = __floats2bfloat162_rn(xc0 - hf.x, xc1 - hf.y);   // exact differences
            const uint32_t off = rowo + 2048u * (uint32_t)k + colo;
            *reinterpret_cast<__nv_bfloat162 *>(ab + off) = hi;
            *reinterpret_cast<__nv_bfloat162 *>(ab + kTM * 128 + off) = lo;
            const float ss = wsum(fmaf(xc1, xc1, xc0 * xc0));
            if (lane == 0) xnb[r] = make_float2(sqrtf(ss), ss);
        }
    };
    auto put = [&](int64_t i, int g) { a.assign[i] = g; };

    if (tid == 0) {
        for (int k = 0; k < 9; ++k) mbar_init(bar_afull + k, 1);
        *abort_flag = 0;
        *namb = 0;
        *n64 = 0;
        *s_cnmax = 0;
        *s_nmax = 0;
        fence_mbar_init();
    }
    if (warp == 16) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    } else {
        for (int k = tid; k < NG * 16; k += kEpi) {
            const int g = k >> 4, kb = (k >> 3) & 1, c = k & 7;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (g < G) v = __ldg(reinterpret_cast<const uint4 *>(a.o.B + (size_t)g * 128 + kb * 64) + c);
            *reinterpret_cast<uint4 *>(sB + (uint32_t)kb * NG * 128u + sw128_off(g, c)) = v;
        }
        for (int g = tid; g < 256; g += kEpi) cn[g] = g < G ? __ldg(a.o.cn + g) : INFINITY;
        for (int d = tid; d < 64; d += kEpi) {
            ctr[d] = d < D ? __ldg(a.center + d) : 0.f;
            swd[d] = d < D ? __ldg(a.sw + d) : 0.f;
        }
    }
    __syncthreads();   // barriers initialised, constants in place
    if (warp < 16)
        for (int g = tid; g < G; g += kEpi) {
            atomicMax(s_cnmax, __float_as_int(__ldg(a.o.cn + g)));
            atomicMax(s_nmax, __float_as_int(__ldg(a.o.ncs + g)));
        }
    if (tid == 0)
        for (int k = 0; k < 2 && k < T; ++k)
            if (tile_bulk((t0 + k) * kTM, a.N, a.x_al16)) issue_x(k);
    if (warp < 16 && T > 0) {
        build_a(0);
        fence_proxy_async();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const float cnmax = __int_as_float(*s_cnmax), nmax = __int_as_float(*s_nmax);
    const float cmax = sqrtf(cnmax);
    if (tid == 0 && T > 0) {
        mbar_arrive(bar_afull);
        if (2 < T && tile_bulk((t0 + 2) * kTM, a.N, a.x_al16)) issue_x(2);   // buffer 0 is free again
    }

    if (warp == 16) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(kTM, NG);
            const uint32_t aS = smem_u32(sA), bS = smem_u32(sB);
            for (int t = 0; t < T; ++t) {
                const int b = t & 1;
                const uint32_t u = (uint32_t)(t >> 1);
                if (!mbar_wait(bar_afull + b, u & 1u, abort_flag, budget)) break;
                if (t >= 2 && !mbar_wait(bar_lfree + b, (u - 1u) & 1u, abort_flag, budget)) break;
                tc_fence_after();
                const uint32_t acc = tmem + 256u * (uint32_t)b;
                const uint32_t a0 = aS + (uint32_t)b * (2u * kTM * 128u), a1 = a0 + kTM * 128u;
                const uint32_t b0 = bS, b1 = bS + (uint32_t)NG * 128u;
                for (int kk = 0; kk < nk; ++kk) {
                    const uint32_t ko = (uint32_t)kk * 32u;
                    tc_mma(acc, desc_k_sw128(a0 + ko), desc_k_sw128(b0 + ko), idesc, kk > 0 ? 1u : 0u);
                    tc_mma(acc, desc_k_sw128(a1 + ko), desc_k_sw128(b0 + ko), idesc, 1u);
                    tc_mma(acc, desc_k_sw128(a0 + ko), desc_k_sw128(b1 + ko), idesc, 1u);
                }
                tc_commit(bar_lfull + b);
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
        const int q = warp & 3, c = warp >> 2;   // lane quadrant, quarter of the means
        const int s = 32 * q + lane;             // this thread's sample in the tile (TMEM lane)
        uint8_t *my = cg + tid * kCap;
        unsigned long long st_n = 0;
        for (int t = 0; t < T; ++t) {
            const int b = t & 1;
            const int64_t i0 = (t0 + t) * kTM;
            const int nvalid = (int)min((int64_t)kTM, a.N - i0);
            // ---- the next tile's operand (its A buffer was read by MMA t-1, complete)
            if (t + 1 < T) {
                build_a(t + 1);
                fence_proxy_async();
            }
            epi_sync();
            if (tid == 0 && t + 1 < T) {
                mbar_arrive(bar_afull + ((t + 1) & 1));
                // the staged buffer of tile t+1 is free again: tile t+3 goes there
                if (t + 3 < T && tile_bulk((t0 + t + 3) * kTM, a.N, a.x_al16)) issue_x(t + 3);
            }
            // ---- pass 1: scores of this (sample, quarter) and their minimum
            mbar_wait(bar_lfull + b, (uint32_t)(t >> 1) & 1u, abort_flag, budget);
            tc_fence_after();
            const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16) + 256u * (uint32_t)b + 64u * (uint32_t)c;
            const float4 *cn4 = reinterpret_cast<const float4 *>(cn + 64 * c);   // +inf past the last mean
            // best (m1, at a1) and second best (m2) score of this quarter; the
            // columns past NG hold no product but their score is +inf or NaN
            // (cn = +inf), which no update below takes
            float m1 = INFINITY, m2 = INFINITY;
            int a1 = 0;
            auto upd = [&](int j, uint32_t P, float cj) {
                const float v = fmaf(-2.f, __uint_as_float(P), cj);
                const bool lt = v < m1;
                m2 = fminf(m2, lt ? m1 : v);
                a1 = lt ? j : a1;
                m1 = lt ? v : m1;
            };
#pragma unroll
            for (int cc = 0; cc < 4; cc += 2) {
                if (64 * c + 16 * cc < NG) {   // warp-uniform
                    uint32_t r0[16], r1[16];
                    tmem_ld16(tl + 16u * (uint32_t)cc, r0);
                    tmem_ld16(tl + 16u * (uint32_t)(cc + 1), r1);
                    tmem_wait_ld();
#pragma unroll
                    for (int j4 = 0; j4 < 4; ++j4) {
                        const float4 ca = cn4[4 * cc + j4], cb = cn4[4 * cc + 4 + j4];
                        upd(16 * cc + 4 * j4 + 0, r0[4 * j4 + 0], ca.x);
                        upd(16 * cc + 4 * j4 + 1, r0[4 * j4 + 1], ca.y);
                        upd(16 * cc + 4 * j4 + 2, r0[4 * j4 + 2], ca.z);
                        upd(16 * cc + 4 * j4 + 3, r0[4 * j4 + 3], ca.w);
                        upd(16 * cc + 16 + 4 * j4 + 0, r1[4 * j4 + 0], cb.x);
                        upd(16 * cc + 16 + 4 * j4 + 1, r1[4 * j4 + 1], cb.y);
                        upd(16 * cc + 16 + 4 * j4 + 2, r1[4 * j4 + 2], cb.z);
                        upd(16 * cc + 16 + 4 * j4 + 3, r1[4 * j4 + 3], cb.w);
                    }
                }
            }
            tc_fence_before();
            xlo[tid] = m1;
            epi_sync();
            if (tid == 0) mbar_arrive(bar_lfree + b);
            // ---- pass 2: candidates within 2e of the sample's best score
            const float best = fminf(fminf(xlo[s], xlo[kTM + s]), fminf(xlo[2 * kTM + s], xlo[3 * kTM + s]));
            const float2 nx = xn[b * kTM + s];
            const float e = fmaf(0.000244140625f * nx.x, cmax, 1.52587890625e-05f * (cnmax + nx.y)) + 1e-30f;
            const float thr = best + 2.f * e;
            int n = m1 <= thr ? 1 : 0;   // a1 alone unless the second best is within reach too
            if (n) my[0] = (uint8_t)a1;
            const bool scan = m2 <= thr;
            if (__any_sync(0xffffffffu, scan)) {
                // the accumulator is read again: the MMAs of tile t+2 wait for
                // the next iteration's operand, after every thread has left this one
                tc_fence_after();
                if (scan) n = 0;
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    if (64 * c + 16 * cc < NG) {
                        uint32_t r0[16];
                        tmem_ld16(tl + 16u * (uint32_t)cc, r0);
                        tmem_wait_ld();
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const float v = fmaf(-2.f, __uint_as_float(r0[j]), cn[64 * c + 16 * cc + j]);
                            if (scan && v <= thr) {
                                if (n < kCap) my[n] = (uint8_t)(16 * cc + j);
                                ++n;
                            }
                        }
                    }
                }
                tc_fence_before();
            }
            if (!(thr < INFINITY)) n = kCap + 1;   // no finite bound: every mean
            cnt[tid] = n;
            epi_sync();
            // ---- one candidate: decided; else recorded for the exact decision
            if (tid < kTM && s < nvalid) {
                const int64_t i = i0 + s;
                int nq[4], tot = 0;
                bool over = false;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    nq[k] = cnt[s + kTM * k];
                    tot += nq[k];
                    over |= nq[k] > kCap;
                }
                if (tot == 1) {
                    int g = 0;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        if (nq[k] == 1) g = 64 * k + cg[(s + kTM * k) * kCap];
                    put(i, g);
                } else {
                    if (!over && tot >= 2 && tot <= kListMax) {
                        uint8_t *cl = L.cand + i * 32;
                        int wpos = 0;
                        for (int k = 0; k < 4; ++k) {
                            const int nk = cnt[s + kTM * k];
                            for (int j = 0; j < nk; ++j) cl[wpos++] = (uint8_t)(64 * k + cg[(s + kTM * k) * kCap + j]);
                        }
                        L.cnt[i * 2] = (uint8_t)tot;
                    } else {
                        L.cnt[i * 2] = 255;   // every mean
                    }
                    L.defer[t0 * kTM + atomicAdd(namb, 1)] = (int32_t)i;
                }
                ++st_n;
            }
        }
        tc_fence_before();
        epi_sync();   // every deferred sample is listed
        // ---- deferred samples, one warp each
        const int nd = __shfl_sync(0xffffffffu, *abort_flag ? 0 : *namb, 0);   // one value per warp
        for (int r = warp; r < nd; r += kEpi / 32) {
            const int64_t i = L.defer[t0 * kTM + r];
            const float *xr = a.X + i * D;
            const int tc = L.cnt[i * 2];
            int bi = INT_MAX;
            bool fp64 = true;
            if (tc != 255) {
                const float xs0 = lane < D ? __ldg(xr + lane) * swd[lane] : 0.f;
                const float xs1 = lane + 32 < D ? __ldg(xr + 32 + lane) * swd[lane + 32] : 0.f;
                const float sn = wsum(fmaf(xs1, xs1, xs0 * xs0));
                const uint8_t *cl = L.cand + i * 32;
                float dm = INFINITY;   // lane k: candidate k's FP32 distance
                int gm = INT_MAX;
                for (int k = 0; k < tc; ++k) {
                    const int g = cl[k];
                    const float *cr = a.o.cs + (size_t)g * D;
                    const float u0 = lane < D ? xs0 - __ldg(cr + lane) : 0.f;
                    const float u1 = lane + 32 < D ? xs1 - __ldg(cr + 32 + lane) : 0.f;
                    const float dv = wsum(fmaf(u1, u1, u0 * u0));
                    if (lane == k) { dm = dv; gm = g; }
                }
                float b1 = dm, b2 = INFINITY;
                int a1 = gm;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float ob1 = __shfl_xor_sync(0xffffffffu, b1, o);
                    const float ob2 = __shfl_xor_sync(0xffffffffu, b2, o);
                    const int oa1 = __shfl_xor_sync(0xffffffffu, a1, o);
                    const bool take = ob1 < b1 || (ob1 == b1 && oa1 < a1);
                    const float nb2 = take ? fminf(b1, ob2) : fminf(ob1, b2);
                    if (take) { b1 = ob1; a1 = oa1; }
                    b2 = nb2;
                }
                const float norms = sn + nmax;
                const float e1 = dist_err(b1, norms, D);
                if (b2 - dist_err(b2, norms, D) > b1 + e1) {
                    bi = a1;
                    fp64 = false;
                } else {
                    // candidates that can still win, each on its lane, in FP64
                    double bv = INFINITY;
                    int bl = INT_MAX;
                    if (lane < tc && dm - dist_err(dm, norms, D) <= b1 + e1) {
                        bv = dist_fp64(xr, a.means + (size_t)gm * D, a.w, D);
                        bl = gm;
                    }
                    bi = warp_argmin_fp64(bv, bl);
                }
            } else {
                double bv = INFINITY;
                int bl = INT_MAX;
                for (int g = lane; g < G; g += 32) {
                    const double dv = dist_fp64(xr, a.means + (size_t)g * D, a.w, D);
                    if (dv < bv) { bv = dv; bl = g; }   // ascending g: the first of equal values
                }
                bi = warp_argmin_fp64(bv, bl);
            }
            if (lane == 0) {
                put(i, bi == INT_MAX ? 0 : bi);
                if (fp64) atomicAdd(n64, 1);
            }
        }
        if (a.stats) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) st_n += __shfl_xor_sync(0xffffffffu, st_n, o);
            if (lane == 0 && st_n) atomicAdd(a.stats + 0, st_n);
        }
    }
    __syncthreads();
    // drain: no bulk copy may still be writing into shared memory at exit
    if (tid == 0) {
        for (int bb = 0; bb < 2; ++bb) {
            const uint32_t issued = bb ? xiss1 : xiss0, used = bb ? xuse1 : xuse0;
            const long long d0 = clock64();
            for (uint32_t u = used; u < issued; ++u)
                while (!mbar_try_wait(bar_x + bb, u & 1u) && clock64() - d0 < budget) {
                }
        }
        if (a.stats) {
            atomicAdd(a.stats + 1, (unsigned long long)*namb);
            atomicAdd(a.stats + 2, (unsigned long long)*n64);
        }
        if (*abort_flag) {
            if (atomicCAS(&a.status->code, 0, (int)GMM_ERR_TIMEOUT) == 0) a.status->fail_iter = 0;
            atomicExch(&a.status->halt, 1);
        }
    }
    if (warp == 16) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// ------------------------------------------------------------------------
// 4. Statistics of the assignment: count, sum(x - mu_f), sum((x - mu_f)^2)
// per mean (the sums of Eqs. 5-7, shifted by the FP32 mean mu_f of the
// iteration start).  One CTA per SM over a contiguous run of 128-sample
// tiles, staged (samples and assignments) by bulk copies kStBufs tiles
// ahead; the shifts in shared memory.  Warp w owns the means g = w + 32 k
// and keeps their FP32 sums in registers for the whole run (lanes over
// dimensions): per tile it finds its samples with four ballots over the
// staged assignments and adds each to the sums of its mean.  No atomics and
// one barrier per tile; the sums go to the CTA's FP64 partial at the end.
// ------------------------------------------------------------------------
constexpr int kStThreads = 1024;
constexpr int kStBufs = 4;

struct StArgs {
    const float *X;
    int64_t N;
    int32_t D, G;
    const int32_t *assign;
    const float *mu_f;     // [G][D] FP32 means (the shift)
    double *partial;       // [grid][G][1 + 2D]
    DevStatus *status;
    long long wait_cycles;
    int32_t x_al16;
};

struct StSmem {
    uint32_t mu, cnt, X[kStBufs], asg[kStBufs], bars, misc, total;
};

__host__ __device__ inline StSmem st_layout(int D, int G)
{
    StSmem L;
    uint32_t o = 0;
    L.mu = o; o += 4u * (uint32_t)G * (uint32_t)D;
    L.cnt = o; o += 4u * (uint32_t)G;
    o = (o + 127u) & ~127u;
    for (int b = 0; b < kStBufs; ++b) {
        L.X[b] = o; o += ((4u * kTM * (uint32_t)D) + 127u) & ~127u;
        L.asg[b] = o; o += 4u * kTM;
    }
    L.bars = o; o += 8u * kStBufs;
    L.misc = o; o += 16u;
    L.total = o;
    return L;
}

__global__ void __launch_bounds__(kStThreads, 1) k_km_stats(StArgs a)
{
    extern __shared__ __align__(128) unsigned char st_raw[];
    if (km_skip(a.status)) return;
    const int D = a.D, G = a.G, S = 1 + 2 * D;
    const StSmem Ls = st_layout(D, G);
    float *mus = reinterpret_cast<float *>(st_raw + Ls.mu);
    int *scnt = reinterpret_cast<int *>(st_raw + Ls.cnt);
    uint64_t *bars = reinterpret_cast<uint64_t *>(st_raw + Ls.bars);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(st_raw + Ls.misc);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntiles = (a.N + kTM - 1) / kTM;
    const int64_t t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
    uint32_t iss = 0u;   // bulk tiles issued (thread 0); tile t0 + k goes to buffer k % kStBufs
    auto issue = [&](int64_t tile) {   // thread 0 only
        const int b = (int)((tile - t0) % kStBufs);
        const uint32_t xb = 4u * kTM * (uint32_t)D;
        ++iss;
        fence_proxy_async();
        mbar_expect_tx(bars + b, xb + 4u * kTM);
        bulk_g2s(st_raw + Ls.X[b], a.X + tile * kTM * D, xb, bars + b);
        bulk_g2s(st_raw + Ls.asg[b], a.assign + tile * kTM, 4u * kTM, bars + b);
    };
    for (int k = tid; k < G * D; k += kStThreads) mus[k] = __ldg(a.mu_f + k);
    for (int k = tid; k < G; k += kStThreads) scnt[k] = 0;
    if (tid == 0) {
        for (int b = 0; b < kStBufs; ++b) mbar_init(bars + b, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < kStBufs && t0 + k < t1; ++k)
            if (tile_bulk((t0 + k) * kTM, a.N, a.x_al16)) issue(t0 + k);
    // sums of the owned means (k-th: g = warp + 32 k), dimensions lane and
    // lane + 32; the counts in shared memory
    float s1a[8], s1b[8], s2a[8], s2b[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) s1a[k] = s1b[k] = s2a[k] = s2b[k] = 0.f;
    auto add = [&](int k, const float *xr, const float *mr) {
        const float u0 = lane < D ? xr[lane] - mr[lane] : 0.f;
        const float u1 = lane + 32 < D ? xr[lane + 32] - mr[lane + 32] : 0.f;
        s1a[k] += u0;
        s2a[k] = fmaf(u0, u0, s2a[k]);
        s1b[k] += u1;
        s2b[k] = fmaf(u1, u1, s2b[k]);
    };
    // tile t: wait for its copy (or copy it here), then each warp adds its samples
    auto process = [&](int64_t t) {
        const int b = (int)((t - t0) % kStBufs);
        const uint32_t use = (uint32_t)((t - t0) / kStBufs);
        const int64_t i0 = t * kTM;
        const int nv = (int)min((int64_t)kTM, a.N - i0);
        float *xs = reinterpret_cast<float *>(st_raw + Ls.X[b]);
        int32_t *as = reinterpret_cast<int32_t *>(st_raw + Ls.asg[b]);
        if (tile_bulk(i0, a.N, a.x_al16)) {
            x_wait(bars + b, use & 1u, a.wait_cycles, abort_flag);
        } else {
            for (int k = tid; k < nv * D; k += kStThreads) xs[k] = __ldg(a.X + i0 * D + k);
            for (int k = tid; k < nv; k += kStThreads) as[k] = __ldg(a.assign + i0 + k);
            __syncthreads();   // uniform: every thread processes the same tiles
        }
        // a tile whose copy did not land (the wait ran out) is not read
        const bool skip = __any_sync(0xffffffffu, *abort_flag != 0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int g = !skip && 32 * q + lane < nv ? as[32 * q + lane] : -1;
            const bool mine = g >= 0 && g < G && (g & 31) == warp;
            unsigned m = __ballot_sync(0xffffffffu, mine);
            if (mine) atomicAdd(&scnt[g], 1);
            while (m) {
                const int src = __ffs(m) - 1;
                m &= m - 1u;
                const int gs = __shfl_sync(0xffffffffu, g, src);
                const float *xr = xs + (32 * q + src) * D;
                const float *mr = mus + gs * D;
                switch (gs >> 5) {   // warp-uniform: the sums stay in registers
                case 0: add(0, xr, mr); break;
                case 1: add(1, xr, mr); break;
                case 2: add(2, xr, mr); break;
                case 3: add(3, xr, mr); break;
                case 4: add(4, xr, mr); break;
                case 5: add(5, xr, mr); break;
                case 6: add(6, xr, mr); break;
                default: add(7, xr, mr); break;
                }
            }
        }
    };
    // two tiles between barriers (fewer waits on the slowest warp)
    int64_t tend = t1;   // first tile not consumed (an abort leaves later copies pending)
    for (int64_t t = t0; t < t1; t += 2) {
        process(t);
        if (t + 1 < t1) process(t + 1);
        if (__syncthreads_or(*abort_flag != 0)) {   // uniform
            tend = t;
            break;
        }
        // the buffers of tiles t and t+1 are free again
        if (tid == 0)
            for (int64_t u = t + kStBufs; u < t + kStBufs + 2 && u < t1; ++u)
                if (tile_bulk(u * kTM, a.N, a.x_al16)) issue(u);
    }
    __syncthreads();
    // drain: no bulk copy may still be writing into shared memory at exit.
    // Bulk tiles are issued in order (tiles t0 .. t0 + iss - 1); those from
    // tend on were not consumed.
    if (tid == 0) {
        const long long d0 = clock64();
        for (int64_t t = tend; t < t0 + (int64_t)iss; ++t) {
            const int b = (int)((t - t0) % kStBufs);
            const uint32_t use = (uint32_t)((t - t0) / kStBufs);
            while (!mbar_try_wait(bars + b, use & 1u) && clock64() - d0 < a.wait_cycles) {
            }
        }
    }
    double *P = a.partial + (size_t)blockIdx.x * G * S;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int g = warp + 32 * k;
        if (g < G) {
            double *pg = P + (size_t)g * S;
            if (lane == 0) pg[0] = (double)scnt[g];
            if (lane < D) { pg[1 + lane] = (double)s1a[k]; pg[1 + D + lane] = (double)s2a[k]; }
            if (lane + 32 < D) { pg[33 + lane] = (double)s1b[k]; pg[33 + D + lane] = (double)s2b[k]; }
        }
    }
    if (tid == 0 && *abort_flag) {
        if (atomicCAS(&a.status->code, 0, (int)GMM_ERR_TIMEOUT) == 0) a.status->fail_iter = 0;
        atomicExch(&a.status->halt, 1);
    }
}

}  // namespace

bool km_tc_supported(int32_t D, int32_t G)
{
    if (D < 1 || D > 64 || G < 1 || G > 256 || !em_tc_supported(D, G)) return false;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int NG = (G + 15) / 16 * 16;
    return km_layout(D, NG).total + 1024u + 1024u <= (uint32_t)optin && st_layout(D, G).total + 1024u <= (uint32_t)optin;
}

namespace {
size_t al256k(size_t n) { return (n + 255u) & ~(size_t)255u; }
}

size_t km_tc_ops_bytes(int32_t D, int32_t G)
{
    const size_t g = (size_t)G;
    return al256k(256u * g) + 2u * al256k(4u * g) + al256k(4u * g * (size_t)D) + 256u;
}

KmTcOps km_tc_ops(void *base, int32_t D, int32_t G)
{
    const size_t g = (size_t)G;
    unsigned char *p = static_cast<unsigned char *>(base);
    KmTcOps o;
    o.B = reinterpret_cast<__nv_bfloat16 *>(p);  p += al256k(256u * g);
    o.cn = reinterpret_cast<float *>(p);         p += al256k(4u * g);
    o.ncs = reinterpret_cast<float *>(p);        p += al256k(4u * g);
    o.cs = reinterpret_cast<float *>(p);
    (void)D;
    return o;
}

cudaError_t launch_km_pass_tc(const float *X, int64_t N, int32_t D, int32_t G, const double *means,
                              const double *w, const float *sw, const float *center, KmTcOps o, Operands op,
                              double *partial, int32_t grid, int32_t *assign, const TcLists &L, DevStatus *status,
                              long long wait_cycles, unsigned long long *stats, cudaStream_t s)
{
    k_km_prep_tc<<<G, 64, 0, s>>>(means, sw, center, D, G, o, op.mu);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int NG = (G + 15) / 16 * 16;
    KmTcArgs k{X, N, D, G, NG, (D + 15) / 16, o, means, w, sw, center, assign, L, status, wait_cycles,
               (reinterpret_cast<uintptr_t>(X) & 15u) == 0 ? 1 : 0,
               (D % 2 == 0 && (reinterpret_cast<uintptr_t>(X) & 7u) == 0) ? 1 : 0, stats};
    const size_t sm = km_layout(D, NG).total + 1024u;
    if ((e = cudaFuncSetAttribute(k_km_screen_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
        cudaSuccess)
        return e;
    k_km_screen_tc<<<grid, kThr, sm, s>>>(k);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    StArgs st{X, N, D, G, assign, op.mu, partial, status, wait_cycles, k.x_al16};
    const size_t sm4 = st_layout(D, G).total;
    if ((e = cudaFuncSetAttribute(k_km_stats, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm4)) != cudaSuccess)
        return e;
    k_km_stats<<<grid, kStThreads, sm4, s>>>(st);
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace gmm
