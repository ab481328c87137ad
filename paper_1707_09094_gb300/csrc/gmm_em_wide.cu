// Tensor-core (tcgen05, sm_103a) EM pass for shapes beyond the one-tile
// form: D up to 128 and N_G up to 4096, e.g. the precision workload
// (N_G = 1024, D = 128, standard deviations down to 0.1, means many of them
// away from the centre).  Per iteration:
//
//  0. k_wide_prep -- per Gaussian, the log-density (Eq. 15) expanded about
//     the global centre m (x' = x - m, mu' = mu - m):
//        l_g(x) = ctc_g + sum_d x'^2 a_gd + sum_d x' b_gd,
//        a = -1/2 iv, b = mu' iv, ctc_g = c_g - 1/2 q_g, q_g = sum_d mu'^2 iv;
//     each FP32 operand split into BF16 parts v_h = bf16(v),
//     v_l = bf16(v - v_h), stored as the shared-memory image of the MMA's B
//     operand: pieces of 128 Gaussians x 64 K (16 KB, 128-byte swizzle), per
//     block of 128 Gaussians the parts a_h | a_l | b_h | b_l of nkb = D'/64
//     pieces each; and the screening constants (ctc - k2, ctc + k2).
//  1. k_wide_screen -- per 128-sample tile, the A operand x'^2 and x' split
//     the same way (t_h | t_l | x_h | x_l), and for each block of 128
//     Gaussians the split products
//        P1 = sum_d (t_h a_h + t_l a_h + t_h a_l)   (t = x'^2)
//        P2 = sum_d (x_h b_h + x_l b_h + x_h b_l)
//     on the tensor cores into two FP32 TMEM accumulators, block after
//     block.  Each sample keeps its best lower bound so far
//     lb_g = P1 + P2 + ctc_g - (K1 |P1| + k2_g) and lists the Gaussians
//     whose upper bound lies within T = ln(N * 1e9) nats of it, dropping
//     entries as that bound rises; after the last block the list holds the
//     Gaussians that can reach a responsibility of 1e-9 / N: at most 64.
//     A sample with more (a start far from converged, where many broad
//     Gaussians overlap) goes with the other such samples, gathered in sample
//     order, to the register-blocked FP32 form (every Gaussian), whose
//     statistics and log-likelihood partials follow this pass's own.
//  2. k_wide_exact -- a warp per sample, lanes over dimensions: the exact
//     FP32 log-density c_g - 1/2 sum_d (x_d s_gd - mu_gd s_gd)^2 of each
//     candidate, log-sum-exp (Eqs. 16-18), log p(x_i) into the CTA's FP64
//     log-likelihood, and the responsibilities (Eq. 3) of at least exp(-T)
//     into the sample's record (at most 64, one per candidate).
//  3. k_wide_mstep -- grid (sample chunk) x (block of 192 Gaussians): per
//     1024-sample tile the records that fall in the block, compacted in
//     sample order; the warp that owns a Gaussian (g mod 32) adds l, l (x - mu_f),
//     l (x - mu_f)^2 (Eqs. 9-11 about the FP32 mean mu_f) to the block's FP32
//     sums in shared memory, which move to the chunk's FP64 partial after at
//     most 128 additions.  The register-blocked FP32 form's records of kept
//     responsibilities go through the same M-step.
//
// Screening bound.  A split operand leaves |v - v_h - v_l| <= 2^-18 |v| with
// |v_l| <= 2^-9 |v|, so the three kept products of a pair miss at most
// 3.1 * 2^-18 |a b|; a product of two BF16 values is exact in FP32, and
// accumulating n <= 384 of them in FP32 adds at most n 2^-23 of their summed
// magnitudes.  The FP32 operands and the exact kernel's own FP32 value add
// ~2^-22 relative errors in |P1|, q_g and r_g = sum_d m_d^2 iv_gd.  With
// sum_d |x' b_d| <= |P1| + q_g / 2 (AM-GM) the screen's value is within
// K1 |P1| + k2_g of the exact kernel's, K1 = 2^-11 and
// k2_g = 2^-12 q_g + 2^-18 r_g + 2^-20 |ctc_g| + 1e-3: at least four times
// the sum of those terms.  A Gaussian dropped by the screen therefore holds
// an exact responsibility below 1e-9 / N, which the exact kernel drops too.
#include <cuda_bf16.h>

#include <cmath>

#include "gmm_internal.cuh"
#include "tc_ptx.cuh"

namespace gmm {

namespace {

using namespace ptx;

constexpr int kWTM = 128;               // samples per tile (MMA M)
constexpr int kWGB = 128;               // Gaussians per screening block (MMA N)
constexpr int kWEpi = 512;              // epilogue threads: 16 warps, four per TMEM lane quadrant
constexpr int kWThreads = kWEpi + 64;   // + the MMA warp + the operand-loading warp
constexpr int kWStages = 3;             // B operand ring
constexpr uint32_t kWPiece = 16384;     // one operand piece: 128 rows x 64 K in BF16
constexpr int kWCap = 64;               // candidates per sample before the dense fallback
constexpr int kWKeep = kRecSlots;       // responsibilities per sample record
constexpr float kWK1 = 4.8828125e-4f;   // 2^-11
constexpr int kWxThreads = 512;         // exact kernel: 16 warps
constexpr int kWmThreads = 1024;        // M-step kernel: 32 warps
constexpr int kWmTile = 1024;           // samples per M-step tile (one per thread)
constexpr int kWmBG = 192;              // Gaussians per M-step block (FP32 sums: 192 KB of shared memory)
constexpr int kWmFlush = 128;           // FP32 additions per sum between FP64 flushes
constexpr int kWmEnt = 2048;            // list entries per window of an M-step tile
constexpr int kWMaxG = 4096;

__device__ __forceinline__ void wepi_sync() { asm volatile("bar.sync 1, 512;" ::: "memory"); }

__device__ __forceinline__ bool wide_skip(const DevStatus *st, int iter)
{
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = (st->halt != 0 || iter > st->stop_after) ? 1 : 0;
    __syncthreads();
    return s_skip != 0;
}

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t *>(&v); }

// v -> (bf16(v), bf16(v - bf16(v))) for two values at once
__device__ __forceinline__ void split2(float v0, float v1, uint32_t &hi, uint32_t &lo)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
    const float2 hf = __bfloat1622float2(h);
    hi = bf2_bits(h);
    lo = bf2_bits(__floats2bfloat162_rn(v0 - hf.x, v1 - hf.y));
}

// ------------------------------------------------------------------------
// 0. Operands.  One block of 128 threads per Gaussian slot g < NGp (the
// padded slots get zero rows and -inf bounds).
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_wide_prep(int32_t D, int32_t G, int32_t nkb, const double *__restrict__ par,
                                                   const float *__restrict__ center, unsigned char *__restrict__ img,
                                                   float2 *__restrict__ bnd)
{
    __shared__ double sh[3][4];
    const int g = blockIdx.x, j = g / kWGB, r = g % kWGB, DP = 64 * nkb;
    const bool real = g < G;
    double qs = 0.0, rs = 0.0, ls = 0.0;
    unsigned char *base = img + (size_t)j * 4 * nkb * kWPiece;
    for (int d = threadIdx.x; d < DP; d += blockDim.x) {
        float av = 0.f, bv = 0.f;
        if (real && d < D) {
            const double v = par[(size_t)G * D + (size_t)g * D + d], mu = par[(size_t)g * D + d];
            const double iv = 1.0 / v, cd = (double)center[d], mc = mu - cd;
            av = (float)(-0.5 * iv);
            bv = (float)(mc * iv);
            qs += mc * mc * iv;
            rs += cd * cd * iv;
            ls += log(v);
        }
        const __nv_bfloat16 ah = __float2bfloat16_rn(av), bh = __float2bfloat16_rn(bv);
        const __nv_bfloat16 al = __float2bfloat16_rn(av - __bfloat162float(ah));
        const __nv_bfloat16 bl = __float2bfloat16_rn(bv - __bfloat162float(bh));
        const int k = d >> 6, e = d & 63;
        const uint32_t o = sw128_off(r, e >> 3) + 2u * (uint32_t)(e & 7);
        *reinterpret_cast<__nv_bfloat16 *>(base + (size_t)(0 * nkb + k) * kWPiece + o) = ah;
        *reinterpret_cast<__nv_bfloat16 *>(base + (size_t)(1 * nkb + k) * kWPiece + o) = al;
        *reinterpret_cast<__nv_bfloat16 *>(base + (size_t)(2 * nkb + k) * kWPiece + o) = bh;
        *reinterpret_cast<__nv_bfloat16 *>(base + (size_t)(3 * nkb + k) * kWPiece + o) = bl;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        qs += __shfl_xor_sync(0xffffffffu, qs, o);
        rs += __shfl_xor_sync(0xffffffffu, rs, o);
        ls += __shfl_xor_sync(0xffffffffu, ls, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh[0][w] = qs;
        sh[1][w] = rs;
        sh[2][w] = ls;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!real) {
            bnd[g] = make_float2(-INFINITY, -INFINITY);
            return;
        }
        const double q = sh[0][0] + sh[0][1] + sh[0][2] + sh[0][3];
        const double rr = sh[1][0] + sh[1][1] + sh[1][2] + sh[1][3];
        const double l = sh[2][0] + sh[2][1] + sh[2][2] + sh[2][3];
        const double c = log(par[2 * (size_t)G * D + g]) - 0.5 * (double)D * kLog2Pi - 0.5 * l;
        const double ctc = c - 0.5 * q;
        const double k2 = q * 0x1p-12 + rr * 0x1p-18 + fabs(ctc) * 0x1p-20 + 1e-3;
        bnd[g] = make_float2((float)(ctc - k2), (float)(ctc + k2));
    }
}

// ------------------------------------------------------------------------
// 1. Screening on the tensor cores.
// ------------------------------------------------------------------------
struct WideArgs {
    EmPassArgs a;
    const unsigned char *img;   // [NGp / 128][4 nkb][16 KB] operand pieces
    const float2 *bnd;          // [NGp] (ctc - k2, ctc + k2)
    uint8_t *cnt;               // [N] candidates (255: every Gaussian)
    uint16_t *cand;             // [N][kWCap] candidate Gaussians, ascending
    int32_t nb, nkb;            // Gaussian blocks of 128; 64-wide K pieces per part
    float screen;               // T = ln(N * 1e9)
    int32_t x_v8;               // D % 4 == 0 and X 16-byte aligned: 16-byte sample loads
};

struct WSmem {
    uint32_t A, R, lst, lcnt, xlo, sbnd, ctr, bars, misc, total;
};

__host__ __device__ inline WSmem w_layout(int nkb)
{
    WSmem L;
    uint32_t o = 0;
    L.A = o; o += 4u * (uint32_t)nkb * kWPiece;   // t_h | t_l | x_h | x_l, nkb pieces each
    L.R = o; o += (uint32_t)kWStages * kWPiece;   // B ring
    L.lst = o; o += 4u * kWTM * kWCap;            // (Gaussian, upper bound) per sample
    L.lcnt = o; o += 4u * kWTM;                   // entries per sample (past kWCap: some lost)
    L.xlo = o; o += 8u * kWEpi;                   // block maxima of the lower bounds, two buffers
    L.sbnd = o; o += 2u * 8u * kWGB;              // screening constants of a block, two buffers
    L.ctr = o; o += 4u * 128u;
    L.bars = o; o += 8u * (6 + 2 * kWStages);
    L.misc = o; o += 16u;
    L.total = o;
    return L;
}

// Warp roles: warps 0-15 are the epilogue (warp w reads TMEM lanes
// 32 (w % 4).. -- samples 32 (w % 4).. of the tile -- and Gaussians
// 32 (w / 4)..+31 of each block) and build the A operand of the next tile;
// warp 16 allocates TMEM and one of its threads issues the MMAs; one thread of
// warp 17 streams the B pieces through the ring by bulk copies and prefetches
// the next sample tile into L2.  TMEM: two buffers of (P1 | P2), 256
// columns each, so the MMAs of one block run while the epilogue reads the
// previous one.  Every wait is bounded: on expiry the CTA records
// GMM_ERR_TIMEOUT, stops issuing work, drains its copies and MMAs, frees
// TMEM and returns.
__global__ void __launch_bounds__(kWThreads, 1) k_wide_screen(WideArgs w)
{
    extern __shared__ __align__(1024) unsigned char w_raw[];
    const EmPassArgs &a = w.a;
    if (wide_skip(a.status, a.iter)) return;   // uniform across the block
    const int D = a.D, G = a.G, nb = w.nb, nkb = w.nkb, DP = 64 * nkb, npc = 4 * nkb;
    const WSmem Ls = w_layout(nkb);
    unsigned char *sb = w_raw + ((1024u - (smem_u32(w_raw) & 1023u)) & 1023u);
    unsigned char *sA = sb + Ls.A, *sR = sb + Ls.R;
    uint32_t *lst = reinterpret_cast<uint32_t *>(sb + Ls.lst);
    int *lcnt = reinterpret_cast<int *>(sb + Ls.lcnt);
    float *xlo = reinterpret_cast<float *>(sb + Ls.xlo);
    float2 *sbnd = reinterpret_cast<float2 *>(sb + Ls.sbnd);
    float *ctr = reinterpret_cast<float *>(sb + Ls.ctr);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sb + Ls.bars);
    uint64_t *b_afull = bar, *b_tfull = bar + 1, *b_tfree = bar + 3, *b_drain = bar + 5;
    uint64_t *b_bfull = bar + 6, *b_bfree = bar + 6 + kWStages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sb + Ls.misc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sb + Ls.misc + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long budget = a.wait_cycles;
    const int64_t ntiles = (a.N + kWTM - 1) / kWTM;
    const int64_t t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
    const int T = (int)(t1 - t0);

    // A operand of `tile`: item = (row, 8 consecutive dimensions), which is
    // one 16-byte chunk of each of the four parts
    auto build_a = [&](int64_t tile) {
        const int64_t i0 = tile * kWTM;
        const int nch = DP / 8;
        for (int it = tid; it < kWTM * nch; it += kWEpi) {
            const int r = it / nch, ch = it - r * nch, d0 = 8 * ch;
            const int64_t i = i0 + r;
            float x[8];
            if (i < a.N && w.x_v8 && d0 + 8 <= D) {
                const float4 *src = reinterpret_cast<const float4 *>(a.X + i * D + d0);
                const float4 u = __ldg(src), v = __ldg(src + 1);
                x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w;
                x[4] = v.x; x[5] = v.y; x[6] = v.z; x[7] = v.w;
#pragma unroll
                for (int e = 0; e < 8; ++e) x[e] -= ctr[d0 + e];
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) x[e] = (i < a.N && d0 + e < D) ? __ldg(a.X + i * D + d0 + e) - ctr[d0 + e] : 0.f;
            }
            uint32_t th[4], tl[4], xh[4], xl[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                split2(x[2 * e] * x[2 * e], x[2 * e + 1] * x[2 * e + 1], th[e], tl[e]);
                split2(x[2 * e], x[2 * e + 1], xh[e], xl[e]);
            }
            const int k = d0 >> 6;
            const uint32_t off = sw128_off(r, (d0 & 63) >> 3);
            *reinterpret_cast<uint4 *>(sA + (uint32_t)(0 * nkb + k) * kWPiece + off) = make_uint4(th[0], th[1], th[2], th[3]);
            *reinterpret_cast<uint4 *>(sA + (uint32_t)(1 * nkb + k) * kWPiece + off) = make_uint4(tl[0], tl[1], tl[2], tl[3]);
            *reinterpret_cast<uint4 *>(sA + (uint32_t)(2 * nkb + k) * kWPiece + off) = make_uint4(xh[0], xh[1], xh[2], xh[3]);
            *reinterpret_cast<uint4 *>(sA + (uint32_t)(3 * nkb + k) * kWPiece + off) = make_uint4(xl[0], xl[1], xl[2], xl[3]);
        }
    };

    if (tid == 0) {
        for (int k = 0; k < 6 + 2 * kWStages; ++k) mbar_init(bar + k, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    for (int d = tid; d < 128; d += kWThreads) ctr[d] = d < D ? __ldg(a.center + d) : 0.f;
    for (int k = tid; k < kWGB; k += kWThreads) sbnd[k] = __ldg(w.bnd + k);   // block 0: the first job's
    for (int k = tid; k < kWTM; k += kWThreads) lcnt[k] = 0;
    if (warp == 16) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    __syncthreads();   // barriers initialised, centre in place
    if (warp < 16 && T > 0) {
        build_a(t0);
        fence_proxy_async();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (tid == 0 && T > 0) mbar_arrive(b_afull);

    if (warp == 16) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(kWTM, kWGB);
            const uint32_t aS = smem_u32(sA), rS = smem_u32(sR);
            uint32_t q = 0, pc = 0;
            bool ok = true;
            unsigned long long w_a = 0, w_b = 0;   // cycles waiting for A / a TMEM buffer, for B pieces (profiling)
            long long c0 = clock64();
            for (int t = 0; t < T && ok; ++t) {
                c0 = clock64();
                if (!mbar_wait(b_afull, (uint32_t)(t & 1), abort_flag, budget)) break;
                w_a += (unsigned long long)(clock64() - c0);
                tc_fence_after();
                if (a.skip_mma) break;   // test hook: the epilogue's wait must run out
                for (int j = 0; j < nb && ok; ++j, ++q) {
                    const uint32_t buf = q & 1u;
                    c0 = clock64();
                    if (q >= 2 && !mbar_wait(b_tfree + buf, ((q >> 1) - 1u) & 1u, abort_flag, budget)) {
                        ok = false;
                        break;
                    }
                    w_a += (unsigned long long)(clock64() - c0);
                    tc_fence_after();
                    const uint32_t d1 = tmem + buf * 256u, d2 = d1 + 128u;
                    for (int p = 0; p < npc; ++p, ++pc) {
                        const uint32_t slot = pc % kWStages;
                        c0 = clock64();
                        if (!mbar_wait(b_bfull + slot, (pc / kWStages) & 1u, abort_flag, budget)) {
                            ok = false;
                            break;
                        }
                        w_b += (unsigned long long)(clock64() - c0);
                        tc_fence_after();
                        const int part = p / nkb, k = p - part * nkb;
                        const uint32_t bs = rS + slot * kWPiece;
                        const uint32_t dst = part < 2 ? d1 : d2;
                        const uint32_t ah = aS + (uint32_t)((part < 2 ? 0 : 2) * nkb + k) * kWPiece;   // t_h | x_h
                        const uint32_t al = aS + (uint32_t)((part < 2 ? 1 : 3) * nkb + k) * kWPiece;   // t_l | x_l
                        const bool first = (part == 0 || part == 2) && k == 0;
                        for (int kk = 0; kk < 4; ++kk)
                            tc_mma(dst, desc_k_sw128(ah + 32u * kk), desc_k_sw128(bs + 32u * kk), idesc,
                                   (first && kk == 0) ? 0u : 1u);
                        if ((part & 1) == 0)   // a hi part of B meets both parts of A
                            for (int kk = 0; kk < 4; ++kk)
                                tc_mma(dst, desc_k_sw128(al + 32u * kk), desc_k_sw128(bs + 32u * kk), idesc, 1u);
                        tc_commit(b_bfree + slot);
                    }
                    if (ok) tc_commit(b_tfull + buf);
                }
            }
            if (a.screen_stats) {
                atomicAdd(a.screen_stats + 9, w_a);
                atomicAdd(a.screen_stats + 10, w_b);
            }
            // drain: every MMA issued above completes before TMEM is freed
            // (this wait ignores the abort flag; it is still bounded)
            tc_commit(b_drain);
            const long long d0 = clock64();
            while (!mbar_try_wait(b_drain, 0u) && clock64() - d0 < budget) {
            }
        }
        __syncwarp();
    } else if (warp == 17) {
        // ------------------------------------------------------------ operand loader
        if (lane == 0) {
            uint32_t pc = 0;
            bool ok = true;
            for (int t = 0; t < T && ok; ++t) {
                const int64_t nt = t0 + t + 1;   // the next tile, prefetched into L2 for its A build
                if (t + 1 < T && w.x_v8 && (nt + 1) * kWTM <= a.N)
                    prefetch_l2(a.X + nt * kWTM * D, (uint32_t)(kWTM * D * 4));
                for (int j = 0; j < nb && ok; ++j)
                    for (int p = 0; p < npc; ++p, ++pc) {
                        const uint32_t slot = pc % kWStages;
                        if (pc >= (uint32_t)kWStages &&
                            !mbar_wait(b_bfree + slot, ((pc / kWStages) - 1u) & 1u, abort_flag, budget)) {
                            ok = false;
                            break;
                        }
                        mbar_expect_tx(b_bfull + slot, kWPiece);
                        bulk_g2s(sR + slot * kWPiece, w.img + ((size_t)j * npc + p) * kWPiece, kWPiece, b_bfull + slot);
                    }
            }
            // drain: copies still in flight (at most one per ring slot)
            const long long d0 = clock64();
            for (uint32_t u = pc > (uint32_t)kWStages ? pc - kWStages : 0u; u < pc; ++u)
                while (!mbar_try_wait(b_bfull + (u % kWStages), (u / kWStages) & 1u) && clock64() - d0 < budget) {
                }
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        const int qd = warp & 3, qq = warp >> 2;  // TMEM lane quadrant; quarter of each block's columns
        const int s = 32 * qd + lane;             // this thread's sample in the tile (TMEM lane)
        const int ts = tid & 127;                 // thread of quarter c of this sample: ts + 128 c
        const uint32_t tl = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(32 * qq);
        uint32_t *sl = lst + s * kWCap;           // the sample's list: g | (bf16 upper bound rounded up) << 16
        unsigned long long st_n = 0, st_c = 0, st_d = 0;
        unsigned long long tp[6] = {0, 0, 0, 0, 0, 0};   // phase cycles of thread 0 (profiling)
        long long tmark = clock64();
        auto phase = [&](int k) {
            const long long now = clock64();
            tp[k] += (unsigned long long)(now - tmark);
            tmark = now;
        };
        // the sample's owner thread keeps the entries whose bound reaches thr
        auto prune = [&](int n, float thr) -> int {
            int k = 0;
            for (int e = 0; e < n; ++e) {
                const uint32_t v = sl[e];
                if (__uint_as_float(v & 0xFFFF0000u) >= thr) sl[k++] = v;
            }
            return k;
        };
        uint32_t q = 0;
        for (int t = 0; t < T; ++t) {
            const int64_t i0 = (t0 + t) * kWTM;
            const int nvalid = (int)min((int64_t)kWTM, a.N - i0);
            float mrun = -INFINITY;   // best lower bound so far of this sample (the same on its four threads)
            bool lost = false;        // owner: entries were lost to a full list
            for (int j = 0; j < nb; ++j, ++q) {
                const uint32_t buf = q & 1u;
                // the next job's constants (block (j + 1) mod nb), stored into the
                // other buffer once the load has landed (after this job's bounds)
                float2 nbnd = make_float2(0.f, 0.f);
                if (tid < kWGB) nbnd = __ldg(w.bnd + (j + 1 < nb ? j + 1 : 0) * kWGB + tid);
                phase(4);
                mbar_wait(b_tfull + buf, (q >> 1) & 1u, abort_flag, budget);
                tc_fence_after();
                phase(0);
                if (j == nb - 1 && t + 1 < T) {
                    // every MMA of this tile is complete: A takes the next tile
                    build_a(t0 + t + 1);
                    fence_proxy_async();
                    wepi_sync();
                    if (tid == 0) mbar_arrive(b_afull);
                    phase(1);
                }
                const uint32_t tb = tl + buf * 256u;
                const float2 *cb = sbnd + buf * kWGB + 32 * qq;
                float ub[32];
                float lmax = -INFINITY;
#pragma unroll
                for (int cc = 0; cc < 2; ++cc) {
                    uint32_t p1[16], p2[16];
                    tmem_ld16(tb + 16u * cc, p1);
                    tmem_ld16(tb + 128u + 16u * cc, p2);
                    tmem_wait_ld();
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const float P1 = __uint_as_float(p1[e]), P2 = __uint_as_float(p2[e]);
                        const float2 c = cb[16 * cc + e];
                        const float base = P1 + P2, k = kWK1 * fabsf(P1);
                        lmax = fmaxf(lmax, base + c.x - k);
                        ub[16 * cc + e] = base + c.y + k;
                    }
                }
                tc_fence_before();
                phase(2);
                if (tid < kWGB) sbnd[(buf ^ 1u) * kWGB + tid] = nbnd;
                xlo[buf * kWEpi + tid] = lmax;
                wepi_sync();
                if (tid == 0) mbar_arrive(b_tfree + buf);
                const float *xb = xlo + buf * kWEpi;
                mrun = fmaxf(mrun, fmaxf(fmaxf(xb[ts], xb[ts + 128]), fmaxf(xb[ts + 256], xb[ts + 384])));
                const float thr = mrun - w.screen;
                if (qq == 0 && lcnt[s] > kWCap - 32) {   // room for this block's entries
                    const int n0 = lcnt[s];
                    lost = lost || n0 > kWCap;
                    lcnt[s] = prune(min(n0, kWCap), thr);
                }
                wepi_sync();
                phase(3);
                const int g0 = j * kWGB + 32 * qq;
#pragma unroll
                for (int e = 0; e < 32; ++e) {
                    if (ub[e] >= thr && g0 + e < G) {
                        const int k = atomicAdd(lcnt + s, 1);
                        if (k < kWCap) {
                            // bf16 of the bound rounded up: truncation moves a negative value up
                            const uint32_t u = __float_as_uint(ub[e]);
                            const uint32_t h = (u >> 16) + (((u >> 31) == 0u && (u & 0xFFFFu) != 0u) ? 1u : 0u);
                            sl[k] = (uint32_t)(g0 + e) | (h << 16);
                        }
                    }
                }
            }
            // ---- the owner prunes the list at the final bound, sorts it by Gaussian
            // and writes the sample's record
            phase(4);
            wepi_sync();
            if (qq == 0) {
                const int n0 = lcnt[s];
                lost = lost || n0 > kWCap;
                int n = prune(min(n0, kWCap), mrun - w.screen);
                if (s < nvalid) {
                    const int64_t i = i0 + s;
                    if (lost || n == 0) {
                        w.cnt[i] = 255;   // every Gaussian (none listed only when every bound is NaN)
                        ++st_d;
                    } else {
                        for (int e = 1; e < n; ++e) {   // insertion sort by Gaussian index
                            const uint32_t v = sl[e];
                            int k = e - 1;
                            while (k >= 0 && (sl[k] & 0xFFFFu) > (v & 0xFFFFu)) {
                                sl[k + 1] = sl[k];
                                --k;
                            }
                            sl[k + 1] = v;
                        }
                        uint2 *dst = reinterpret_cast<uint2 *>(w.cand + i * kWCap);   // four per 8-byte store
                        for (int e = 0; e < n; e += 4) {
                            uint32_t v[4];
#pragma unroll
                            for (int k = 0; k < 4; ++k) v[k] = e + k < n ? (sl[e + k] & 0xFFFFu) : 0u;
                            dst[e >> 2] = make_uint2(v[0] | (v[1] << 16), v[2] | (v[3] << 16));
                        }
                        w.cnt[i] = (uint8_t)n;
                    }
                    ++st_n;
                    st_c += (unsigned long long)n;
                }
                lcnt[s] = 0;
            }
            wepi_sync();   // the lists are rewritten by the next tile
            phase(5);
        }
        tc_fence_before();
        if (a.screen_stats) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                st_n += __shfl_xor_sync(0xffffffffu, st_n, o);
                st_c += __shfl_xor_sync(0xffffffffu, st_c, o);
                st_d += __shfl_xor_sync(0xffffffffu, st_d, o);
            }
            if (lane == 0 && qq == 0) {
                atomicAdd(a.screen_stats + 0, st_n);
                atomicAdd(a.screen_stats + 1, st_c);
                atomicAdd(a.screen_stats + 2, st_d);
            }
            if (tid == 0)
                for (int k = 0; k < 6; ++k) atomicAdd(a.screen_stats + 3 + k, tp[k]);
        }
    }
    __syncthreads();
    if (tid == 0 && *abort_flag) {
        if (atomicCAS(&a.status->code, 0, (int)GMM_ERR_TIMEOUT) == 0) a.status->fail_iter = a.iter;
        atomicExch(&a.status->halt, 1);
    }
    if (warp == 16) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// ------------------------------------------------------------------------
// 2. Exact log-densities of the candidates, log-sum-exp, records.
// ------------------------------------------------------------------------
struct WxArgs {
    EmPassArgs a;
    const uint8_t *cnt;
    const uint16_t *cand;
    uint8_t *rc;       // [N] kept responsibilities in the record
    uint16_t *rg;      // [N][kWKeep] their Gaussians
    float *rgam;       // [N][kWKeep] and values
    float screen;
    int32_t x_v4;      // D % 4 == 0 and X 16-byte aligned
    int32_t s_v4;      // D even and the operand array 16-byte aligned
};

// Dimensions 4 lane .. 4 lane + 3 of sample i (zeros past D).
__device__ __forceinline__ void wide_x(const float *__restrict__ X, int64_t i, int D, int lane, bool v4, float (&x)[4])
{
    const int d0 = 4 * lane;
    if (v4 && d0 + 4 <= D) {
        const float4 u = __ldg(reinterpret_cast<const float4 *>(X + i * D + d0));
        x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w;
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) x[e] = d0 + e < D ? __ldg(X + i * D + d0 + e) : 0.f;
    }
}

// Exact FP32 log-density c_g - 1/2 sum_d (x_d s_gd - mu_gd s_gd)^2 with the
// lanes over dimensions (each lane four), summed by a butterfly: every lane
// returns the same value.
__device__ __forceinline__ float wide_logit(const Operands &op, int D, int g, const float (&x)[4], int lane, bool v4)
{
    const int d0 = 4 * lane;
    float r = 0.f;
    if (d0 < D) {
        const float2 *q = op.sm + (size_t)g * D + d0;
        float2 s[4];
        if (v4 && d0 + 4 <= D) {
            const float4 u = __ldg(reinterpret_cast<const float4 *>(q)), v = __ldg(reinterpret_cast<const float4 *>(q) + 1);
            s[0] = make_float2(u.x, u.y); s[1] = make_float2(u.z, u.w);
            s[2] = make_float2(v.x, v.y); s[3] = make_float2(v.z, v.w);
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) s[e] = d0 + e < D ? __ldg(q + e) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float t = fmaf(x[e], s[e].x, -s[e].y);
            r = fmaf(t, t, r);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    return fmaf(-0.5f, r, __ldg(op.c + g));
}

// One warp per sample over a contiguous sample range per CTA; the CTA's FP64
// log-likelihood is summed per warp in sample order, then over the warps.
__global__ void __launch_bounds__(kWxThreads) k_wide_exact(WxArgs w)
{
    const EmPassArgs &a = w.a;
    if (wide_skip(a.status, a.iter)) return;
    __shared__ double s_ll[kWxThreads / 32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int nw = kWxThreads / 32;
    const int D = a.D, G = a.G;
    const bool xv4 = w.x_v4 != 0, sv4 = w.s_v4 != 0;
    const float keep = -w.screen;
    const int64_t i0 = a.N * blockIdx.x / gridDim.x, i1 = a.N * (blockIdx.x + 1) / gridDim.x;
    double ll = 0.0;
    for (int64_t i = i0 + warp; i < i1; i += nw) {
        float x[4];
        wide_x(a.X, i, D, lane, xv4, x);
        const int n = w.cnt[i];   // <= kWCap, or 255: left to the FP32 form
        float lse = 0.f;
        int m = 0;
        if (n <= kWCap) {
            // candidate k on lane k % 32, slot k / 32
            int gc[4];
            float lc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                gc[u] = 32 * u + lane < n ? min((int)w.cand[i * kWCap + 32 * u + lane], G - 1) : 0;
                lc[u] = -INFINITY;
            }
            for (int k = 0; k < n; ++k) {
                const int u = k >> 5;
                const int gsrc = u == 0 ? gc[0] : (u == 1 ? gc[1] : (u == 2 ? gc[2] : gc[3]));
                const float l = wide_logit(a.op, D, __shfl_sync(0xffffffffu, gsrc, k & 31), x, lane, sv4);
                if (lane == (k & 31)) {
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        if (v == u) lc[v] = l;
                }
            }
            float M = fmaxf(fmaxf(lc[0], lc[1]), fmaxf(lc[2], lc[3]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) M = fmaxf(M, __shfl_xor_sync(0xffffffffu, M, o));
            float S = 0.f;
            if (M != -INFINITY)
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (lc[u] != -INFINITY) S += __expf(lc[u] - M);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) S += __shfl_xor_sync(0xffffffffu, S, o);
            lse = M + logf(S);
            // kept pairs in candidate order
            unsigned bal[4];
            bool kp[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                kp[u] = 32 * u + lane < n && lc[u] - lse >= keep;
                bal[u] = __ballot_sync(0xffffffffu, kp[u]);
                m += __popc(bal[u]);
            }
            if (m <= kWKeep) {
                const unsigned below = (1u << lane) - 1u;
                int base = 0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (kp[u]) {
                        const int rank = base + __popc(bal[u] & below);
                        w.rg[i * kWKeep + rank] = (uint16_t)gc[u];
                        w.rgam[i * kWKeep + rank] = __expf(lc[u] - lse);
                    }
                    base += __popc(bal[u]);
                }
            }
        }
        if (lane == 0) {
            w.rc[i] = (uint8_t)min(m, kWKeep);   // m <= n <= kWKeep; 0 for a sample left to the FP32 form
            ll += (double)lse;
        }
    }
    if (lane == 0) s_ll[warp] = ll;
    __syncthreads();
    if (tid == 0) {
        double v = 0.0;
        for (int k = 0; k < nw; ++k) v += s_ll[k];
        a.ll_partial[blockIdx.x] = v;
    }
}

// ------------------------------------------------------------------------
// 3. M-step from the records.
// ------------------------------------------------------------------------
struct WmArgs {
    EmPassArgs a;
    const uint8_t *rc;
    const uint16_t *rg;
    const float *rgam;
    int32_t n_gb, n_chunks;
};

struct WmSmem {
    uint32_t S12, ent, scan, total;
};

__host__ __device__ inline WmSmem wm_layout()
{
    WmSmem L;
    uint32_t o = 0;
    L.S12 = o; o += 4u * kWmBG * 256u;          // [kWmBG][S1: 128 | S2: 128]
    L.ent = o; o += 8u * kWmEnt;                // (sample | g_local << 16, responsibility)
    L.scan = o; o += 4u * 32u;
    L.total = o;
    return L;
}

__global__ void __launch_bounds__(kWmThreads, 1) k_wide_mstep(WmArgs w)
{
    extern __shared__ __align__(16) unsigned char wm_raw[];
    const EmPassArgs &a = w.a;
    if (wide_skip(a.status, a.iter)) return;
    const WmSmem Ls = wm_layout();
    float *S12 = reinterpret_cast<float *>(wm_raw + Ls.S12);
    uint2 *ent = reinterpret_cast<uint2 *>(wm_raw + Ls.ent);
    int *scan = reinterpret_cast<int *>(wm_raw + Ls.scan);
    constexpr int nw = kWmThreads / 32;          // warp w owns the Gaussians g_local = w + nw j
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int D = a.D, G = a.G, S = 1 + 2 * D;
    const int gb = blockIdx.x % w.n_gb, chunk = blockIdx.x / w.n_gb, g0 = gb * kWmBG;
    double *P = a.partial + (size_t)chunk * G * S;
    for (int k = tid; k < kWmBG * 256; k += kWmThreads) S12[k] = 0.f;
    // lane j < kWmBG / nw keeps, for the warp's Gaussian g_local = warp + nw j:
    // the sum of l, the FP32 additions since the last flush, whether flushed once
    float s0r = 0.f;
    int cnr = 0, flr = 0;
    // FP32 sums of this warp's Gaussian gl -> the chunk's FP64 partial
    auto flush = [&](int gl) {
        const int g = g0 + gl, j = gl / nw;
        const float s0 = __shfl_sync(0xffffffffu, s0r, j);
        const bool add = __shfl_sync(0xffffffffu, flr, j) != 0;
        if (g < G) {
            double *row = P + (size_t)g * S;
            float *s1 = S12 + gl * 256, *s2 = s1 + 128;
            for (int d = lane; d < D; d += 32) {
                row[1 + d] = add ? row[1 + d] + (double)s1[d] : (double)s1[d];
                row[1 + D + d] = add ? row[1 + D + d] + (double)s2[d] : (double)s2[d];
                s1[d] = 0.f;
                s2[d] = 0.f;
            }
            if (lane == 0) row[0] = add ? row[0] + (double)s0 : (double)s0;
        }
        if (lane == j) {
            s0r = 0.f;
            cnr = 0;
            flr = 1;
        }
        __syncwarp();
    };
    // one pair, lanes over dimensions d = lane + 32 u: v = x - mu_f (loads
    // first, so a batch of pairs has its loads in flight together), then the
    // sums in list order
    auto load_pair = [&](int64_t i, int gl, float (&v)[4]) {
        const int g = g0 + gl;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int d = lane + 32 * u;
            v[u] = d < D ? __ldg(a.X + i * D + d) - __ldg(a.op.mu + (size_t)g * D + d) : 0.f;
        }
    };
    auto acc_pair = [&](int gl, float gam, const float (&v)[4]) {
        float *s1 = S12 + gl * 256, *s2 = s1 + 128;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int d = lane + 32 * u;
            if (d < D) {
                const float gv = gam * v[u];
                s1[d] += gv;
                s2[d] = fmaf(gv, v[u], s2[d]);
            }
        }
        const int j = gl / nw;
        if (lane == j) {
            s0r += gam;
            ++cnr;
        }
        if (__shfl_sync(0xffffffffu, cnr, j) >= kWmFlush) flush(gl);
    };
    const int64_t ntiles = (a.N + kWmTile - 1) / kWmTile;
    const int64_t tb0 = ntiles * chunk / w.n_chunks, tb1 = ntiles * (chunk + 1) / w.n_chunks;
    __syncthreads();
    for (int64_t t = tb0; t < tb1; ++t) {
        const int64_t i0 = t * kWmTile, i = i0 + tid;
        int nm = 0, rcv = 0;
        const uint16_t *rgi = w.rg + i * kWKeep;
        if (i < a.N) {
            const int r = w.rc[i];
            rcv = r == 255 ? 0 : min(r, kWKeep);   // 255: the sample's statistics come from elsewhere
            for (int k8 = 0; k8 < rcv; k8 += 8) {   // eight slots per 16-byte load
                const uint4 u = __ldg(reinterpret_cast<const uint4 *>(rgi + k8));
                const uint32_t uw[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int g = (int)((uw[k >> 1] >> (16 * (k & 1))) & 0xFFFFu);
                    nm += (k8 + k < rcv && g < G && g / kWmBG == gb);
                }
            }
        }
        // exclusive prefix sum of the pairs over the tile, in sample order
        int pn = nm;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int a1 = __shfl_up_sync(0xffffffffu, pn, o);
            if (lane >= o) pn += a1;
        }
        if (lane == 31) scan[warp] = pn;
        __syncthreads();
        int bp = 0, tp = 0;
#pragma unroll
        for (int k = 0; k < nw; ++k) {
            if (k < warp) bp += scan[k];
            tp += scan[k];
        }
        const int pos0 = bp + pn - nm;
        // ---- the pairs in windows of kWmEnt list entries; owner warps take the
        // pairs of Gaussians g_local = warp (mod 32), in list order
        for (int r0 = 0; r0 < tp; r0 += kWmEnt) {
            if (nm > 0 && pos0 < r0 + kWmEnt && pos0 + nm > r0) {
                int p = pos0;
                for (int k = 0; k < rcv; ++k) {
                    const int g = __ldg(rgi + k);
                    if (g < G && g / kWmBG == gb) {
                        if (p >= r0 && p < r0 + kWmEnt)
                            ent[p - r0] = make_uint2((uint32_t)tid | ((uint32_t)(g - g0) << 16),
                                                     __float_as_uint(__ldg(w.rgam + i * kWKeep + k)));
                        ++p;
                    }
                }
            }
            __syncthreads();
            const int ne = min(kWmEnt, tp - r0);
            for (int e0 = 0; e0 < ne; e0 += 32) {
                const bool own = e0 + lane < ne && (int)((ent[e0 + lane].x >> 16) % nw) == warp;
                unsigned mask = __ballot_sync(0xffffffffu, own);
                while (mask) {   // up to four of this warp's pairs at a time
                    int idx[4];
                    float v[4][4];
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        idx[b] = -1;
                        if (mask) {
                            idx[b] = e0 + __ffs(mask) - 1;
                            mask &= mask - 1u;
                        }
                    }
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        if (idx[b] >= 0) {
                            const uint2 en = ent[idx[b]];
                            load_pair(i0 + (int)(en.x & 0xFFFFu), (int)(en.x >> 16), v[b]);
                        }
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        if (idx[b] >= 0) {
                            const uint2 en = ent[idx[b]];
                            acc_pair((int)(en.x >> 16), __uint_as_float(en.y), v[b]);
                        }
                }
            }
            __syncthreads();   // the window (and scan) are rewritten
        }
        if (tp == 0) __syncthreads();   // scan is rewritten by the next tile
    }
    // final flush of this warp's rows (rows never touched are written as zeros)
    for (int gl = warp; gl < kWmBG; gl += nw) flush(gl);
}

// ------------------------------------------------------------------------
// Samples with more candidates than a list holds go to the register-blocked
// FP32 form (every Gaussian, the same log-densities to FP32 rounding): their
// indices are compacted in sample order and their rows gathered into Xd.
// Per 1024 samples: the count, then the offsets, then the rows.
// ------------------------------------------------------------------------
constexpr int kWdBlock = 1024;

__global__ void __launch_bounds__(kWdBlock) k_wide_dcount(const uint8_t *__restrict__ cnt, int64_t N,
                                                          int32_t *__restrict__ bcnt)
{
    const int64_t i = (int64_t)blockIdx.x * kWdBlock + threadIdx.x;
    const int f = __syncthreads_count(i < N && cnt[i] == 255);
    if (threadIdx.x == 0) bcnt[blockIdx.x] = f;
}

// Exclusive prefix sum of the nblk counts in place (one CTA), the total to *n_dense.
__global__ void __launch_bounds__(1024) k_wide_dscan(int32_t *__restrict__ bcnt, int32_t nblk, int64_t *__restrict__ n_dense)
{
    __shared__ int32_t s_w[32];
    __shared__ int64_t s_base;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_base = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nblk; b0 += 1024) {
        const int b = b0 + tid;
        const int v = b < nblk ? bcnt[b] : 0;
        int x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_w[warp] = x;
        __syncthreads();
        int wb = 0, tot = 0;
        for (int k = 0; k < 32; ++k) {
            if (k < warp) wb += s_w[k];
            tot += s_w[k];
        }
        const int64_t base = s_base;
        if (b < nblk) bcnt[b] = (int32_t)(base + wb + x - v);
        __syncthreads();
        if (tid == 0) s_base = base + tot;
        __syncthreads();
    }
    if (tid == 0) *n_dense = s_base;
}

__global__ void __launch_bounds__(kWdBlock) k_wide_dgather(const uint8_t *__restrict__ cnt, const float *__restrict__ X,
                                                           int64_t N, int32_t D, const int32_t *__restrict__ boff,
                                                           float *__restrict__ Xd, const float *__restrict__ v,
                                                           float *__restrict__ vd)
{
    __shared__ int32_t s_w[32];
    __shared__ int64_t s_idx[kWdBlock];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i = (int64_t)blockIdx.x * kWdBlock + tid;
    const int f = (i < N && cnt[i] == 255) ? 1 : 0;
    int x = f;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    int wb = 0, tot = 0;
    for (int k = 0; k < 32; ++k) {
        if (k < warp) wb += s_w[k];
        tot += s_w[k];
    }
    if (f) {
        s_idx[wb + x - 1] = i;
        if (v) vd[boff[blockIdx.x] + wb + x - 1] = v[i];   // a per-sample value travels with the row
    }
    __syncthreads();
    const int64_t o0 = boff[blockIdx.x];
    for (int k = warp; k < tot; k += kWdBlock / 32) {   // a warp per row
        const int64_t src = s_idx[k];
        for (int d = lane; d < D; d += 32) Xd[(o0 + k) * D + d] = __ldg(X + src * D + d);
    }
}

}  // namespace

bool em_wide_supported(int32_t D, int32_t G)
{
    if (D < 1 || D > 128 || G < 1 || G > kWMaxG || !em_blocked_supported(D, G)) return false;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return w_layout((D + 63) / 64).total + 1024u + 1024u <= (uint32_t)optin;
}

namespace {
int wide_mchunks(int64_t N, int32_t G, int sms)
{
    const int n_gb = (G + kWmBG - 1) / kWmBG;
    int64_t c = (4LL * sms + n_gb - 1) / n_gb;                 // about four waves of one CTA per SM
    const int64_t tiles = (N + kWmTile - 1) / kWmTile;
    c = c < tiles ? c : tiles;
    return (int)(c < 1 ? 1 : c);
}

int wide_xgrid(int64_t N, int sms)
{
    const int64_t g = 2LL * sms, w = (N + 15) / 16;            // at least 16 samples per CTA
    return (int)(g < w ? g : (w < 1 ? 1 : w));
}

size_t wal256(size_t n) { return (n + 255u) & ~(size_t)255u; }
}  // namespace

int em_wide_partials(int64_t N, int32_t G, int sms) { return wide_mchunks(N, G, sms) + em_blocked_chunks(G, sms); }

int em_wide_ll_partials(int64_t N, int sms) { return wide_xgrid(N, sms) + (int)((N + 127) / 128); }

size_t em_wide_ws_bytes(int64_t N, int32_t D, int32_t G)
{
    const size_t n = (size_t)N, nkb = (size_t)((D + 63) / 64), ngp = (size_t)((G + kWGB - 1) / kWGB) * kWGB;
    const size_t nblk = (n + kWdBlock - 1) / kWdBlock;
    return wal256(ngp / kWGB * 4 * nkb * kWPiece) + wal256(8u * ngp) + wal256(n) + wal256(2u * kWCap * n) +
           wal256(n) + wal256(2u * kWKeep * n) + wal256(4u * kWKeep * n) + wal256(4u * nblk) + wal256(8u) +
           wal256(4u * n * (size_t)D) + wal256(4u * n) + wal256(8u * n * (size_t)em_blocked_gblocks(G)) + 256u;
}

WideWs em_wide_ws(void *base, int64_t N, int32_t D, int32_t G)
{
    const size_t n = (size_t)N, nkb = (size_t)((D + 63) / 64), ngp = (size_t)((G + kWGB - 1) / kWGB) * kWGB;
    const size_t nblk = (n + kWdBlock - 1) / kWdBlock;
    unsigned char *p = static_cast<unsigned char *>(base);
    WideWs w;
    w.img = p;                                    p += wal256(ngp / kWGB * 4 * nkb * kWPiece);
    w.bnd = reinterpret_cast<float2 *>(p);        p += wal256(8u * ngp);
    w.cnt = p;                                    p += wal256(n);
    w.cand = reinterpret_cast<uint16_t *>(p);     p += wal256(2u * kWCap * n);
    w.rc = p;                                     p += wal256(n);
    w.rg = reinterpret_cast<uint16_t *>(p);       p += wal256(2u * kWKeep * n);
    w.rgam = reinterpret_cast<float *>(p);        p += wal256(4u * kWKeep * n);
    w.bcnt = reinterpret_cast<int32_t *>(p);      p += wal256(4u * nblk);
    w.n_dense = reinterpret_cast<int64_t *>(p);   p += wal256(8u);
    w.Xd = reinterpret_cast<float *>(p);          p += wal256(4u * n * (size_t)D);
    w.lse_d = reinterpret_cast<float *>(p);       p += wal256(4u * n);
    w.part_d = reinterpret_cast<float2 *>(p);
    return w;
}

int record_mstep_chunks(int64_t N, int32_t G, int sms) { return wide_mchunks(N, G, sms); }

cudaError_t launch_record_mstep(const EmPassArgs &a, const uint8_t *rc, const uint16_t *rg, const float *rgam, int sms,
                                cudaStream_t s)
{
    const int mch = wide_mchunks(a.N, a.G, sms), n_gb = (a.G + kWmBG - 1) / kWmBG;
    WmArgs m{a, rc, rg, rgam, n_gb, mch};
    const size_t sm3 = wm_layout().total;
    cudaError_t e = cudaFuncSetAttribute(k_wide_mstep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3);
    if (e != cudaSuccess) return e;
    k_wide_mstep<<<mch * n_gb, kWmThreads, sm3, s>>>(m);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gather_marked(const uint8_t *flag, const float *X, const float *v, int64_t N, int32_t D, int32_t *bcnt,
                                 int64_t *n_marked, float *Xd, float *vd, cudaStream_t s)
{
    const int nblk = (int)((N + kWdBlock - 1) / kWdBlock);
    k_wide_dcount<<<nblk, kWdBlock, 0, s>>>(flag, N, bcnt);
    k_wide_dscan<<<1, 1024, 0, s>>>(bcnt, nblk, n_marked);
    k_wide_dgather<<<nblk, kWdBlock, 0, s>>>(flag, X, N, D, bcnt, Xd, v, vd);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_em_wide(const EmPassArgs &a, const double *par, const WideWs &ws, int sms, cudaStream_t s)
{
    const int nkb = (a.D + 63) / 64, nb = (a.G + kWGB - 1) / kWGB;
    const float scr = (float)std::log((double)(a.N_total > a.N ? a.N_total : a.N) * 1e9);
    const bool x16 = (reinterpret_cast<uintptr_t>(a.X) & 15u) == 0;
    const int xv4 = (x16 && a.D % 4 == 0) ? 1 : 0;
    const int sv4 = ((reinterpret_cast<uintptr_t>(a.op.sm) & 15u) == 0 && a.D % 2 == 0) ? 1 : 0;
    const int mch = wide_mchunks(a.N, a.G, sms), xg = wide_xgrid(a.N, sms);
    k_wide_prep<<<nb * kWGB, 128, 0, s>>>(a.D, a.G, nkb, par, a.center, ws.img, ws.bnd);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    WideArgs w{a, ws.img, ws.bnd, ws.cnt, ws.cand, nb, nkb, scr, xv4};
    const size_t sm1 = w_layout(nkb).total + 1024u;
    if ((e = cudaFuncSetAttribute(k_wide_screen, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1)) != cudaSuccess)
        return e;
    const int64_t ntiles = (a.N + kWTM - 1) / kWTM;
    const int g1 = (int)(ntiles < sms ? ntiles : sms);
    k_wide_screen<<<g1, kWThreads, sm1, s>>>(w);
    // the samples left to the FP32 form, in sample order
    const int nblk = (int)((a.N + kWdBlock - 1) / kWdBlock);
    k_wide_dcount<<<nblk, kWdBlock, 0, s>>>(ws.cnt, a.N, ws.bcnt);
    k_wide_dscan<<<1, 1024, 0, s>>>(ws.bcnt, nblk, ws.n_dense);
    k_wide_dgather<<<nblk, kWdBlock, 0, s>>>(ws.cnt, a.X, a.N, a.D, ws.bcnt, ws.Xd, nullptr, nullptr);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    WxArgs x{a, ws.cnt, ws.cand, ws.rc, ws.rg, ws.rgam, scr, xv4, sv4};
    k_wide_exact<<<xg, kWxThreads, 0, s>>>(x);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const int n_gb = (a.G + kWmBG - 1) / kWmBG;
    WmArgs m{a, ws.rc, ws.rg, ws.rgam, n_gb, mch};
    const size_t sm3 = wm_layout().total;
    if ((e = cudaFuncSetAttribute(k_wide_mstep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3)) != cudaSuccess)
        return e;
    k_wide_mstep<<<mch * n_gb, kWmThreads, sm3, s>>>(m);
    count_launches(7);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the FP32 form over the gathered samples: statistics after the pass's
    // own partials, log-likelihood partials after the exact kernel's
    EmPassArgs d = a;
    d.X = ws.Xd;
    d.partial = a.partial + (size_t)mch * a.G * (1 + 2 * a.D);
    d.ll_partial = a.ll_partial + xg;
    return launch_em_blocked(d, ws.lse_d, ws.part_d, em_blocked_chunks(a.G, sms), s, ws.n_dense);
}

}  // namespace gmm
