// Tensor-core (tcgen05, sm_103a) EM pass in three kernels.
//
//  1. k_em_screen_tc -- per 128-sample tile of the CTA's chunk, the E-step
//     contraction on the tensor cores, BF16 operands, FP32 accumulators in
//     TMEM, split into the two halves of the log-density (Eq. 15) expanded
//     about the global centre m (x' = x - m, mu' = mu - m):
//        P1[i][g] = sum_d x'^2 (-1/2 iv_gd)      (K block 0, TMEM columns 0..255)
//        P2[i][g] = sum_d x'   (mu'_gd iv_gd)    (K block 1, TMEM columns 256..511)
//     so l~_g(x_i) = ctc_g + P1 + P2 approximates log w_g N(x_i|g).  Each
//     operand rounded to BF16 (8-bit significand) is within 2^-8 of its FP32
//     value, so each product is within 2^-7 + 2^-16 of the exact one; the
//     FP32 accumulation of 64 exact products adds at most 64 * 2^-23 of the
//     sum of their magnitudes.  Hence
//        |l~ - l| <= 2^-7 * 1.01 * sum_d (x'^2 iv/2 + |x' mu'| iv) + tiny terms,
//     and by AM-GM sum_d |x' mu'| iv <= sum_d (x'^2 + mu'^2) iv / 2 = |P1| + q_g/2
//     (q_g = sum_d mu'^2 iv), so |l~ - l| <= K1 |P1| + k2_g with
//     K1 = 2^-6 * 1.25 and k2_g = 2^-7 * 1.25 * q_g / 2 + 2^-21 |ctc_g| + 1e-4.
//     A Gaussian whose upper bound lies more than T = ln(N * 1e9) nats below
//     the best lower bound has responsibility below 1e-9 / N and is dropped
//     (per Gaussian the dropped mass is below 1e-9, under the 1e-8
//     responsibility sum below which the update keeps a Gaussian's
//     parameters).  Output per (sample, half of the Gaussians): the list of
//     surviving Gaussians (at most kTcCap, else the half is marked dense).
//  2. k_em_exact -- one CTA per SM over a contiguous run of 128-sample tiles,
//     the FP32 operands in shared memory, one lane per (sample, candidate)
//     pair: the exact FP32 log-density of every candidate (the formula of
//     the CUDA-core form), of every Gaussian of a dense half; log-sum-exp
//     (Eqs. 16-18), log p(x_i) into the CTA's FP64 log-likelihood,
//     responsibilities l_{g,i} (Eq. 3) of the candidates that matter.
//  3. k_em_mstep_lists -- the same CTA runs (the paper's thread t): per
//     128-sample tile the (sample, Gaussian) pairs are counting-sorted by
//     Gaussian, and the warp that owns a Gaussian sums l, l (x - mu_f),
//     l (x - mu_f)^2 over its pairs in registers (Eqs. 9-11, shifted by the
//     FP32 mean mu_f of the iteration start) and adds them to the CTA's FP32
//     statistics in shared memory (no atomics on them); the chunk's
//     statistics go to its FP64 partial once.
// Responsibilities exist only for the surviving pairs (a few per sample).
#include <cuda_bf16.h>

#include <cmath>

#include "gmm_internal.cuh"
#include "tc_ptx.cuh"

namespace gmm {

namespace {

using namespace ptx;

constexpr int kEpiThreads = 512;  // screening kernel: 16 epilogue warps
constexpr int kThreads = kEpiThreads + 32;
constexpr int kTM = 128;          // samples per tile = MMA M
constexpr int kCap = kTcCap;      // candidates per (sample, half) before the dense fallback
constexpr float kK1 = 0.015625f * 1.25f;      // 2^-6 * 1.25 (multiplies |P1|)
constexpr int kExThreads = 1024;  // exact-recompute kernel: 32 warps, one sample per warp at a time
constexpr int kMsThreads = 1024;  // M-step kernel: 32 warps

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 512;" ::: "memory"); }

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}



__device__ __forceinline__ bool skip_block(const DevStatus *st, int iter)
{
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = (st->halt != 0 || iter > st->stop_after) ? 1 : 0;
    __syncthreads();
    return s_skip != 0;
}

constexpr int kST = 128;   // samples per staged tile of the exact and M-step kernels

// A staged tile is copied by the bulk engine when it is a whole tile of a
// 16-byte-aligned X; the last, partial tile (or an unaligned X) is copied by
// the threads themselves.
__device__ __forceinline__ bool tile_is_bulk(int64_t i0, int64_t N, int x_al16)
{
    return x_al16 && i0 + kST <= N;
}

// Bounded wait on a staged tile: true when it landed.  On expiry the status
// word records GMM_ERR_TIMEOUT (the block then stops consuming tiles).
__device__ __forceinline__ bool stage_wait(uint64_t *bar, uint32_t parity, long long budget, volatile int *abort_flag)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort_flag) return false;
        if (clock64() - t0 > budget) { *abort_flag = 1; return false; }
    }
    return true;
}

struct TcArgs {
    EmPassArgs a;
    TcLists L;
    int32_t NG;       // Gaussians padded to a multiple of 16 (MMA N)
    int32_t nk;       // K=16 steps per K block: ceil(D/16)
    float screen;     // screening distance in nats, ln(N * 1e9)
    int32_t x_al16;   // X is 16-byte aligned: whole tiles are staged by bulk copies
    int32_t x_v2;     // D even and X 8-byte aligned: rows are read two dimensions at a time
};

struct TcSmem {
    uint32_t B, A, X, xstride, cst, ctr, cg, xlo, cn, bars, misc, total;
};

__host__ __device__ inline TcSmem tc_layout(int D, int NG)
{
    TcSmem L;
    uint32_t o = 0;
    L.B = o; o += 2u * NG * 128u;                        // two K blocks of [NG][128 B]
    L.A = o; o += 2u * kTM * 256u;                       // two buffers x two K blocks of [128][128 B]
    L.xstride = ((4u * kTM * (uint32_t)D) + 127u) & ~127u;
    L.X = o; o += 2u * L.xstride;                        // two staged FP32 sample tiles
    L.cst = o; o += 8u * NG;                             // ctc - k2 [NG] | ctc + k2 [NG]
    L.ctr = o; o += 4u * 64u;                            // centre
    L.cg = o; o += (uint32_t)kEpiThreads * kCap;         // candidate list staging, 16 B per thread
    L.xlo = o; o += 4u * kEpiThreads;                    // best lower bound per (sample, quarter)
    L.cn = o; o += 8u * kEpiThreads;                     // candidate bit mask per (sample, quarter)
    o = (o + 7u) & ~7u;
    L.bars = o; o += 8u * 6u;
    L.misc = o; o += 16u;
    L.total = o;
    return L;
}

// ------------------------------------------------------------------------
// 1. Screening on the tensor cores.  Warp roles: warps 0-15 are the
// epilogue (warp w reads TMEM lanes 32*(w%4).., i.e. samples 32*(w%4)..,
// and Gaussians 64*(w/4)..64*(w/4)+63 of both accumulators), warp 16
// allocates TMEM and one of its threads issues the MMAs.  Each FP32 sample
// tile is staged by a bulk copy three tiles ahead; the BF16 operand of tile
// t+1 is built from it (double-buffered) while the MMAs of tile t+1 follow
// the screening of tile t.  Output per (sample, half of the Gaussians): the
// candidates of its two quarters merged into one list of at most kTcCap,
// else the half is marked dense.  Every wait is bounded: on expiry the CTA
// records GMM_ERR_TIMEOUT, stops issuing work, drains, frees TMEM and returns.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads, 1) k_em_screen_tc(TcArgs args)
{
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    const EmPassArgs &a = args.a;
    if (skip_block(a.status, a.iter)) return;   // uniform across the block
    const int D = a.D, G = a.G, NG = args.NG, nk = args.nk;
    const TcSmem Ls = tc_layout(D, NG);
    unsigned char *sbase = tc_raw + ((1024u - (smem_u32(tc_raw) & 1023u)) & 1023u);
    unsigned char *sB = sbase + Ls.B;
    unsigned char *sA = sbase + Ls.A;
    float *clb = reinterpret_cast<float *>(sbase + Ls.cst);   // lower-bound constant per Gaussian
    float *cub = clb + NG;                                       // upper-bound constant
    float *ctr = reinterpret_cast<float *>(sbase + Ls.ctr);
    uint8_t *cg = reinterpret_cast<uint8_t *>(sbase + Ls.cg);
    float *xlo = reinterpret_cast<float *>(sbase + Ls.xlo);
    uint2 *cm = reinterpret_cast<uint2 *>(sbase + Ls.cn);
    uint64_t *bar_afull = reinterpret_cast<uint64_t *>(sbase + Ls.bars);
    uint64_t *bar_lfull = bar_afull + 1;
    uint64_t *bar_lfree = bar_afull + 2;
    uint64_t *bar_drain = bar_afull + 3;
    uint64_t *bar_x = bar_afull + 4;   // [2] staged sample tiles
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sbase + Ls.misc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(sbase + Ls.misc + 4);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long budget = a.wait_cycles;
    const int64_t ntiles = (a.N + kTM - 1) / kTM;
    const int64_t t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
    const int T = (int)(t1 - t0);
    uint32_t xuse0 = 0u, xuse1 = 0u;   // consumed bulk tiles per buffer (epilogue threads)
    uint32_t xiss0 = 0u, xiss1 = 0u;   // issued bulk tiles per buffer (thread 0)

    auto issue_x = [&](int64_t tile) {   // thread 0 only; buffer tile & 1
        const int b = (int)(tile & 1);
        if (b) ++xiss1; else ++xiss0;
        const uint32_t xb = 4u * kTM * (uint32_t)D;
        fence_proxy_async();
        mbar_expect_tx(bar_x + b, xb);
        bulk_g2s(sbase + Ls.X + (uint32_t)b * Ls.xstride, a.X + tile * kTM * D, xb, bar_x + b);
    };
    // BF16 operand A of tile `tile` -> A buffer b: row r = [x'^2 | x'] (K
    // blocks 0 | 1), warp per row, from the staged tile (or from global for
    // a tile that is not staged)
    // Rows r = warp + 16 i share r & 7, so a lane's swizzled column offset
    // (two dimensions per lane) is the same in every row it writes.
    const uint32_t colo = ((uint32_t)((lane >> 2) ^ (warp & 7)) << 4) | (uint32_t)((lane & 3) * 4);
    const uint32_t rowo = (uint32_t)(warp >> 3) * 1024u + (uint32_t)(warp & 7) * 128u;
    auto build_a = [&](int64_t tile, int b) {
        const int64_t i0 = tile * kTM;
        unsigned char *ab = sA + b * (kTM * 256);
        const bool staged = tile_is_bulk(i0, a.N, args.x_al16);
        if (staged) {
            const int xb = (int)(tile & 1);
            if (stage_wait(bar_x + xb, (xb ? xuse1 : xuse0) & 1u, budget, abort_flag)) {
                if (xb) ++xuse1; else ++xuse0;
            }
        }
        const float *xt = reinterpret_cast<const float *>(sbase + Ls.X + (uint32_t)(tile & 1) * Ls.xstride);
        const int d0 = 2 * lane;
        const float2 c2 = reinterpret_cast<const float2 *>(ctr)[lane];   // 0 past D
#pragma unroll 4
        for (int i = 0; i < kTM / 16; ++i) {
            const int r = warp + 16 * i;
            float x0 = 0.f, x1 = 0.f;
            if (i0 + r < a.N && d0 < D) {
                const float *src = staged ? xt + r * D + d0 : a.X + (i0 + r) * D + d0;
                if (args.x_v2) {   // D even and X 8-byte aligned
                    const float2 p = staged ? *reinterpret_cast<const float2 *>(src)
                                            : __ldg(reinterpret_cast<const float2 *>(src));
                    x0 = p.x - c2.x;
                    x1 = p.y - c2.y;
                } else {
                    x0 = (staged ? src[0] : __ldg(src)) - c2.x;
                    if (d0 + 1 < D) x1 = (staged ? src[1] : __ldg(src + 1)) - c2.y;
                }
            }
            const uint32_t off = rowo + 2048u * (uint32_t)i + colo;
            *reinterpret_cast<__nv_bfloat162 *>(ab + off) = __floats2bfloat162_rn(x0 * x0, x1 * x1);
            *reinterpret_cast<__nv_bfloat162 *>(ab + 16384 + off) = __floats2bfloat162_rn(x0, x1);
        }
    };

    if (tid == 0) {
        for (int k = 0; k < 6; ++k) mbar_init(bar_afull + k, 1);
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 16) {
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
                // 2^-7 * 1.25 * q/2  +  2^-21 |ctc|  +  1e-4
                const float k2 = 0.0078125f * 1.25f * 0.5f * __ldg(a.op.q + g) + 4.76837158203125e-07f * fabsf(ct) + 1e-4f;
                clb[g] = ct - k2;
                cub[g] = ct + k2;
            } else {
                clb[g] = -INFINITY;
                cub[g] = -INFINITY;
            }
        }
        for (int d = tid; d < 64; d += kEpiThreads) ctr[d] = d < D ? __ldg(a.center + d) : 0.f;
    }
    __syncthreads();   // barriers initialised, centre in place
    if (tid == 0)
        for (int k = 0; k < 2 && k < T; ++k)
            if (tile_is_bulk((t0 + k) * kTM, a.N, args.x_al16)) issue_x(t0 + k);
    if (warp < 16 && T > 0) {
        build_a(t0, 0);
        fence_proxy_async();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    if (tid == 0 && T > 0) {
        mbar_arrive(bar_afull);
        if (2 < T && tile_is_bulk((t0 + 2) * kTM, a.N, args.x_al16)) issue_x(t0 + 2);
    }

    unsigned long long st_kept = 0, st_dense = 0, st_n = 0;
    unsigned long long tp[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // phase cycles (thread 0, profiling only)
    long long tmark = clock64();
    auto phase = [&](int k) {
        const long long now = clock64();
        tp[k] += (unsigned long long)(now - tmark);
        tmark = now;
    };
    if (warp == 16) {
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
        const int q = warp & 3, c = warp >> 2;  // lane quadrant, Gaussian quarter
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
            if (tid == 0) {
                if (t + 1 < T) mbar_arrive(bar_afull);
                // the staged buffer of tile t+1 is free again: tile t+3 goes there
                if (t + 3 < T && tile_is_bulk((tile + 3) * kTM, a.N, args.x_al16)) issue_x(tile + 3);
            }
            phase(1);
            // ---- pass 1: screening bounds from the two TMEM accumulators
            mbar_wait(bar_lfull, (uint32_t)(t & 1), abort_flag, budget);
            tc_fence_after();
            phase(2);
            // P1 = sum x'^2 (-iv/2) is a sum of non-positive products, so |P1| = -P1
            // and the bounds l -+ e are linear in (P1, P2):
            //   lb = (1 + K1) P1 + P2 + (ctc - k2),  ub = (1 - K1) P1 + P2 + (ctc + k2)
            // evaluated two Gaussians per packed FP32 instruction.  Pass 1 takes
            // the best lower bound; pass 2 reads the accumulators again for the
            // upper bounds (the MMAs of the next tile wait for this tile's pass 2).
            float lo = -INFINITY;
            const float2 kp = make_float2(1.f + kK1, 1.f + kK1), km = make_float2(1.f - kK1, 1.f - kK1);
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const int g0 = 64 * c + 16 * cc;
                if (g0 < NG) {
                    uint32_t p1[16], p2[16];
                    tmem_ld16(tl + (uint32_t)g0, p1);
                    tmem_ld16(tl + 256u + (uint32_t)g0, p2);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 16; j += 4) {
                        const float4 cl = *reinterpret_cast<const float4 *>(clb + g0 + j);
                        const float2 la = __fadd2_rn(
                            __ffma2_rn(make_float2(__uint_as_float(p1[j]), __uint_as_float(p1[j + 1])), kp,
                                       make_float2(__uint_as_float(p2[j]), __uint_as_float(p2[j + 1]))),
                            make_float2(cl.x, cl.y));
                        const float2 lb = __fadd2_rn(
                            __ffma2_rn(make_float2(__uint_as_float(p1[j + 2]), __uint_as_float(p1[j + 3])), kp,
                                       make_float2(__uint_as_float(p2[j + 2]), __uint_as_float(p2[j + 3]))),
                            make_float2(cl.z, cl.w));
                        lo = fmaxf(lo, fmaxf(fmaxf(la.x, la.y), fmaxf(lb.x, lb.y)));
                    }
                }
            }
            phase(3);
            xlo[tid] = lo;
            epi_sync();
            lo = fmaxf(fmaxf(xlo[s], xlo[kTM + s]), fmaxf(xlo[2 * kTM + s], xlo[3 * kTM + s]));
            // ---- pass 2: candidate list of this (sample, quarter), as a bit mask first
            const float thr = lo - args.screen;
            const int gend = G - 64 * c;   // only real Gaussians (also when every bound is NaN/-inf)
            uint32_t m0 = 0u, m1 = 0u;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const int g0 = 64 * c + 16 * cc;
                if (g0 < NG) {
                    uint32_t p1[16], p2[16];
                    tmem_ld16(tl + (uint32_t)g0, p1);
                    tmem_ld16(tl + 256u + (uint32_t)g0, p2);
                    tmem_wait_ld();
                    uint32_t bits = 0u;
#pragma unroll
                    for (int j = 0; j < 16; j += 4) {
                        const float4 cu = *reinterpret_cast<const float4 *>(cub + g0 + j);
                        const float2 ua = __fadd2_rn(
                            __ffma2_rn(make_float2(__uint_as_float(p1[j]), __uint_as_float(p1[j + 1])), km,
                                       make_float2(__uint_as_float(p2[j]), __uint_as_float(p2[j + 1]))),
                            make_float2(cu.x, cu.y));
                        const float2 ubb = __fadd2_rn(
                            __ffma2_rn(make_float2(__uint_as_float(p1[j + 2]), __uint_as_float(p1[j + 3])), km,
                                       make_float2(__uint_as_float(p2[j + 2]), __uint_as_float(p2[j + 3]))),
                            make_float2(cu.z, cu.w));
                        if (ua.x >= thr) bits |= 1u << j;
                        if (ua.y >= thr) bits |= 1u << (j + 1);
                        if (ubb.x >= thr) bits |= 1u << (j + 2);
                        if (ubb.y >= thr) bits |= 1u << (j + 3);
                    }
                    if (cc < 2) m0 |= bits << (16 * cc);
                    else m1 |= bits << (16 * (cc - 2));
                }
            }
            tc_fence_before();
            m0 &= gend >= 32 ? 0xffffffffu : (gend > 0 ? (1u << gend) - 1u : 0u);
            m1 &= gend >= 64 ? 0xffffffffu : (gend > 32 ? (1u << (gend - 32)) - 1u : 0u);
            cm[tid] = make_uint2(m0, m1);
            epi_sync();
            if (tid == 0) mbar_arrive(bar_lfree);   // every thread's TMEM reads of this tile are done
            // ---- the two quarters of a half -> one record (threads of even quarters)
            if ((c & 1) == 0 && s < nvalid) {
                const int h = c >> 1;
                const uint2 pm = cm[tid + 128];
                const int n = __popc(m0) + __popc(m1), nb = __popc(pm.x) + __popc(pm.y);
                const int tot = n + nb;
                const int64_t rec = (i0 + s) * 2 + h;
                args.L.cnt[rec] = (uint8_t)(n > kCap || nb > kCap ? 255 : tot);
                if (tot > 0 && tot <= kCap) {
                    int k = 0;
                    for (uint32_t m = m0; m != 0u; m &= m - 1u) my[k++] = (uint8_t)(__ffs(m) - 1);
                    for (uint32_t m = m1; m != 0u; m &= m - 1u) my[k++] = (uint8_t)(31 + __ffs(m));
                    for (uint32_t m = pm.x; m != 0u; m &= m - 1u) my[k++] = (uint8_t)(63 + __ffs(m));
                    for (uint32_t m = pm.y; m != 0u; m &= m - 1u) my[k++] = (uint8_t)(95 + __ffs(m));
                    reinterpret_cast<uint4 *>(args.L.cand)[rec] = *reinterpret_cast<const uint4 *>(my);
                }
                st_n += (h == 0);
                st_kept += (unsigned long long)tot;
                st_dense += tot > kCap;
            }
            phase(4);
        }
        tc_fence_before();
    }
    __syncthreads();
    // drain: no bulk copy may still be writing into shared memory at exit
    if (tid == 0)
        for (int bb = 0; bb < 2; ++bb) {
            const uint32_t issued = bb ? xiss1 : xiss0, used = bb ? xuse1 : xuse0;
            const long long d0 = clock64();
            for (uint32_t u = used; u < issued; ++u)
                while (!mbar_try_wait(bar_x + bb, u & 1u) && clock64() - d0 < budget) {
                }
        }
    if (a.screen_stats && warp < 16) {
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
    if (warp == 16) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

struct ExArgs {
    EmPassArgs a;
    TcLists L;
    float screen;     // ln(N * 1e9): responsibilities below exp(-screen) are dropped
    int32_t x_al16;
    int32_t wp;       // exact kernel: pair slots per warp (a multiple of 32)
};

struct ExSmem {
    uint32_t psm, pc, X[2], cand[2], cnt[2], wl, wg, ws, bars, misc, total;
};

// The operands (s = 1/sigma, mu s) are one [G][DS] float2 array whose row
// stride DS is the smallest value >= D with DS = 2 (mod 4): rows start on
// 16-byte boundaries (two dimensions per 128-bit load) and DS/2 is odd, so
// the eight lanes of one 128-bit load phase that read different Gaussians at
// one d hit different banks.
__host__ __device__ inline int ex_stride(int D) { return D + ((6 - (D & 3)) & 3); }

__host__ __device__ inline ExSmem ex_layout(int D, int G, int wp)
{
    ExSmem L;
    const uint32_t DS = (uint32_t)ex_stride(D);
    uint32_t o = 0;
    L.psm = o; o += 8u * (uint32_t)G * DS;
    L.pc = o; o += 4u * (uint32_t)G;
    o = (o + 127u) & ~127u;
    for (int b = 0; b < 2; ++b) {
        L.X[b] = o; o += ((4u * kST * (uint32_t)D) + 127u) & ~127u;
        L.cand[b] = o; o += 32u * kST;
        L.cnt[b] = o; o += 2u * kST;
    }
    L.wl = o; o += 4u * 32u * (uint32_t)wp;
    L.wg = o; o += 32u * (uint32_t)wp;
    L.ws = o; o += 32u * (uint32_t)wp;
    L.bars = o; o += 16u;
    L.misc = o; o += 16u;
    L.total = o;
    return L;
}

// ------------------------------------------------------------------------
// 2. Exact log-densities, log-sum-exp and responsibilities of the screened
// candidates.  One CTA per SM owns a contiguous run of 128-sample tiles; the
// FP32 operands (s, mu s) and c sit in shared memory, and each tile's
// samples, candidate lists and counts are staged by bulk copies two tiles
// ahead.  Warp w takes samples 4w..4w+3 of a tile, with no block barrier
// inside the tile:
//  * its (sample, Gaussian) pairs -- the screened candidates, or every
//    Gaussian of a dense half -- one lane per pair, each lane the whole
//    exact FP32 log-density over D (the formula of the CUDA-core form);
//  * eight lanes per sample: log-sum-exp (Eqs. 16-18), log p(x_i) into the
//    CTA's FP64 log-likelihood, and the pairs whose responsibility (Eq. 3)
//    is at least exp(-screen) -- the screen's own bound: every dropped pair
//    carries less than 1e-9 / N -- kept in pair order: the first kTcKeep in
//    the sample's record, the rest in the CTA's spill list.
// Four samples with more than kWarpPairs pairs (dense halves) are done one
// sample at a time, lanes over dimensions, to the same results.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(kExThreads, 1) k_em_exact(ExArgs args)
{
    extern __shared__ __align__(128) unsigned char ex_raw[];
    const EmPassArgs &a = args.a;
    const TcLists &L = args.L;
    if (skip_block(a.status, a.iter)) return;
    const int D = a.D, G = a.G, DS = ex_stride(D);
    const int WP = args.wp;
    const ExSmem Ls = ex_layout(D, G, WP);
    float2 *psm = reinterpret_cast<float2 *>(ex_raw + Ls.psm);
    float *pc = reinterpret_cast<float *>(ex_raw + Ls.pc);
    uint64_t *bars = reinterpret_cast<uint64_t *>(ex_raw + Ls.bars);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(ex_raw + Ls.misc);
    int *nspill = reinterpret_cast<int *>(ex_raw + Ls.misc + 4);
    __shared__ double s_ll[32];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    float *wl = reinterpret_cast<float *>(ex_raw + Ls.wl) + warp * WP;
    uint8_t *wg = ex_raw + Ls.wg + warp * WP;
    uint8_t *wsm = ex_raw + Ls.ws + warp * WP;
    const int64_t ntiles = (a.N + kST - 1) / kST;
    const int64_t t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
    const float keep = -args.screen;
    int64_t *sp_ig = L.sp_ig + (size_t)blockIdx.x * kTcSpill;
    float *sp_gam = L.sp_gam + (size_t)blockIdx.x * kTcSpill;

    uint32_t iss0 = 0u, iss1 = 0u;   // issued bulk tiles per buffer (thread 0)
    auto issue = [&](int64_t tile, int b) {   // thread 0 only
        const int64_t i0 = tile * kST;
        const uint32_t xb = 4u * kST * (uint32_t)D;
        const uint32_t bo = (uint32_t)b * (Ls.X[1] - Ls.X[0]);
        if (b) ++iss1; else ++iss0;
        fence_proxy_async();
        mbar_expect_tx(bars + b, xb + 32u * kST + 2u * kST);
        bulk_g2s(ex_raw + Ls.X[0] + bo, a.X + i0 * D, xb, bars + b);
        bulk_g2s(ex_raw + Ls.cand[0] + bo, L.cand + i0 * 32, 32u * kST, bars + b);
        bulk_g2s(ex_raw + Ls.cnt[0] + bo, L.cnt + i0 * 2, 2u * kST, bars + b);
    };
    // one kept pair of sample i at rank r (pair order): record slot or spill
    auto put = [&](int64_t i, int r, int g, float gam, int spill_base, bool spill_ok) {
        if (r < kTcKeep) {
            L.gam[i * kTcKeep + r] = gam;
            L.kg[i * kTcKeep + r] = (uint8_t)g;
        } else if (spill_base >= 0) {
            const int e = spill_base + r - kTcKeep;
            if (e < kTcSpill) {
                sp_ig[e] = i * 256 + g;
                sp_gam[e] = spill_ok ? gam : 0.f;   // a failed reservation leaves null entries
            }
        }
    };

    if (tid == 0) {
        mbar_init(bars, 1);
        mbar_init(bars + 1, 1);
        *abort_flag = 0;
        *nspill = 0;
        fence_mbar_init();
    }
    for (int k = tid; k < G * D; k += kExThreads) {
        const int g = k / D, d = k - g * D;
        psm[g * DS + d] = __ldg(a.op.sm + k);
    }
    for (int g = tid; g < G; g += kExThreads) pc[g] = __ldg(a.op.c + g);
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < 2 && t0 + k < t1; ++k)
            if (tile_is_bulk((t0 + k) * kST, a.N, args.x_al16)) issue(t0 + k, k);
    double ll = 0.0;
    uint32_t use0 = 0u, use1 = 0u;
    const int j8 = lane & 7, k8 = lane >> 3;     // eight lanes per sample in the finish step
    for (int64_t t = t0; t < t1; ++t) {
        const int b = (int)((t - t0) & 1);
        const int64_t i0 = t * kST;
        const int nv = (int)min((int64_t)kST, a.N - i0);
        const uint32_t bo = (uint32_t)b * (Ls.X[1] - Ls.X[0]);
        float *xs = reinterpret_cast<float *>(ex_raw + Ls.X[0] + bo);
        uint8_t *cs = ex_raw + Ls.cand[0] + bo;
        uint8_t *ns = ex_raw + Ls.cnt[0] + bo;
        if (tile_is_bulk(i0, a.N, args.x_al16)) {
            if (stage_wait(bars + b, (b ? use1 : use0) & 1u, a.wait_cycles, abort_flag)) {
                if (b) ++use1; else ++use0;
            }
        } else {
            for (int k = tid; k < nv * D; k += kExThreads) xs[k] = __ldg(a.X + i0 * D + k);
            for (int k = tid; k < nv * 32; k += kExThreads) cs[k] = L.cand[i0 * 32 + k];
            for (int k = tid; k < nv * 2; k += kExThreads) ns[k] = L.cnt[i0 * 2 + k];
        }
        __syncthreads();
        if (*abort_flag) break;   // uniform: nothing sets the flag between the barrier and here
        const int sb = 4 * warp;  // this warp's first sample in the tile
        // ---- pairs of the four samples: counts, offsets (lanes 0..3)
        int n0 = 0, n1 = 0, c0 = 0, c1 = 0;
        if (lane < 4 && sb + lane < nv) {
            n0 = ns[2 * (sb + lane)];
            n1 = ns[2 * (sb + lane) + 1];
            c0 = n0 > kCap ? min(128, G) : n0;
            c1 = n1 > kCap ? max(0, min(128, G - 128)) : n1;
        }
        const int tot = c0 + c1;
        const int t_0 = __shfl_sync(0xffffffffu, tot, 0), t_1 = __shfl_sync(0xffffffffu, tot, 1);
        const int t_2 = __shfl_sync(0xffffffffu, tot, 2), t_3 = __shfl_sync(0xffffffffu, tot, 3);
        const int o1 = t_0, o2 = o1 + t_1, o3 = o2 + t_2, T = o3 + t_3;
        if (T <= WP) {
            // ---- one lane per pair, in rounds of 32 pairs.  Within a round the
            // pairs are dealt to lanes in the order (rank among the pairs with
            // the same g mod 8, g mod 8): the eight lanes of a 128-bit load
            // phase then mostly read operand rows in distinct bank groups.
            for (int p0 = 0; p0 < T; p0 += 32) {
                const int pl = p0 + lane;
                int sil = 0, gl = 0;
                if (pl < T) {
                    const int k = (pl >= o1) + (pl >= o2) + (pl >= o3);
                    const int j = pl - (k == 0 ? 0 : (k == 1 ? o1 : (k == 2 ? o2 : o3)));
                    sil = sb + k;
                    const int m0 = ns[2 * sil], m1 = ns[2 * sil + 1];
                    const int d0 = m0 > kCap ? min(128, G) : m0;
                    if (j < d0) gl = m0 > kCap ? j : cs[sil * 32 + j];
                    else gl = 128 + (m1 > kCap ? j - d0 : cs[sil * 32 + 16 + (j - d0)]);
                }
                const int key = pl < T ? (gl & 7) : 8;   // lanes past the last pair sort last
                const int rk = __popc(__match_any_sync(0xffffffffu, key) & ((1u << lane) - 1u));
                int pos = 0;
#pragma unroll
                for (int kk = 0; kk < 9; ++kk) {
                    const int ck = __popc(__ballot_sync(0xffffffffu, key == kk));
                    pos += min(ck, rk) + (kk < key && ck > rk ? 1 : 0);
                }
                wsm[p0 + pos] = (uint8_t)lane;   // p0 + 31 < WP: T <= WP and WP is a multiple of 32
                __syncwarp();
                const int src = wsm[p0 + lane];
                const int p = p0 + src;
                const int si = __shfl_sync(0xffffffffu, sil, src), g = __shfl_sync(0xffffffffu, gl, src);
                if (p >= T) continue;
                // ---- exact log-density of the pair over all D
                const float *xr = xs + si * D;
                const float2 *q = psm + g * DS;
                float r0 = 0.f, r1 = 0.f;
                if ((D & 3) == 0) {   // 16-byte aligned rows: four dimensions per three 128-bit loads
                    const float4 *x4 = reinterpret_cast<const float4 *>(xr);
                    const float4 *q4 = reinterpret_cast<const float4 *>(q);
#pragma unroll 3
                    for (int d4 = 0; d4 < D / 4; ++d4) {
                        const float4 xv = x4[d4], qa = q4[2 * d4], qb = q4[2 * d4 + 1];
                        const float ta = fmaf(xv.x, qa.x, -qa.y), tb = fmaf(xv.y, qa.z, -qa.w);
                        const float tc = fmaf(xv.z, qb.x, -qb.y), td = fmaf(xv.w, qb.z, -qb.w);
                        r0 = fmaf(ta, ta, r0);
                        r1 = fmaf(tb, tb, r1);
                        r0 = fmaf(tc, tc, r0);
                        r1 = fmaf(td, td, r1);
                    }
                } else if ((D & 1) == 0) {   // 8-byte aligned rows: two dimensions per load
                    const float2 *x2 = reinterpret_cast<const float2 *>(xr);
#pragma unroll 4
                    for (int d2 = 0; d2 < D / 2; ++d2) {
                        const float2 xv = x2[d2], qa = q[2 * d2], qb = q[2 * d2 + 1];
                        const float ta = fmaf(xv.x, qa.x, -qa.y), tb = fmaf(xv.y, qb.x, -qb.y);
                        r0 = fmaf(ta, ta, r0);
                        r1 = fmaf(tb, tb, r1);
                    }
                } else {
                    for (int d = 0; d < D; ++d) {
                        const float2 qa = q[d];
                        const float ta = fmaf(xr[d], qa.x, -qa.y);
                        r0 = fmaf(ta, ta, r0);
                    }
                }
                wl[p] = fmaf(-0.5f, r0 + r1, pc[g]);
                wg[p] = (uint8_t)g;
            }
            __syncwarp();
            // ---- eight lanes per sample: log-sum-exp, kept pairs in order
            const int si = sb + k8;
            const int pb = k8 == 0 ? 0 : (k8 == 1 ? o1 : (k8 == 2 ? o2 : o3));
            const int pn = (k8 == 0 ? o1 : (k8 == 1 ? o2 : (k8 == 2 ? o3 : T))) - pb;
            float M = -INFINITY;
            for (int q = j8; q < pn; q += 8) M = fmaxf(M, wl[pb + q]);
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) M = fmaxf(M, __shfl_xor_sync(0xffffffffu, M, o));
            float Ssum = 0.f;
            if (M != -INFINITY)
                for (int q = j8; q < pn; q += 8) Ssum += __expf(wl[pb + q] - M);
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) Ssum += __shfl_xor_sync(0xffffffffu, Ssum, o);
            const float lse = M + logf(Ssum);
            // kept pairs: ranks by rounds of eight, in pair order
            int m = 0;
            const int rounds = (pn + 7) >> 3;
            const int rmax = __reduce_max_sync(0xffffffffu, rounds);
            for (int r = 0; r < rmax; ++r) {
                const int q = 8 * r + j8;
                const float rl = q < pn ? wl[pb + q] - lse : -INFINITY;
                const bool kp = q < pn && rl >= keep;
                const unsigned bal = __ballot_sync(0xffffffffu, kp);
                const unsigned grp = (bal >> (8 * k8)) & 0xFFu;
                if (kp) {
                    const int rank = m + __popc(grp & ((1u << j8) - 1u));
                    if (rank < kTcKeep) put(i0 + si, rank, wg[pb + q], __expf(rl), -1, true);
                }
                m += __popc(grp);
            }
            // spill: reserve the CTA list's slots for ranks >= kTcKeep
            int sbase = -1;
            bool sok = true;
            if (j8 == 0 && si < nv && m > kTcKeep) {
                sbase = atomicAdd(nspill, m - kTcKeep);
                sok = sbase + (m - kTcKeep) <= kTcSpill;
            }
            sbase = __shfl_sync(0xffffffffu, sbase, 8 * k8);
            sok = __shfl_sync(0xffffffffu, (int)sok, 8 * k8) != 0;
            if (__any_sync(0xffffffffu, sbase >= 0)) {   // warp-uniform
                int mm = 0;
                for (int r = 0; r < rmax; ++r) {
                    const int q = 8 * r + j8;
                    const float rl = q < pn ? wl[pb + q] - lse : -INFINITY;
                    const bool kp = q < pn && rl >= keep;
                    const unsigned grp = (__ballot_sync(0xffffffffu, kp) >> (8 * k8)) & 0xFFu;
                    if (kp && sbase >= 0) {
                        const int rank = mm + __popc(grp & ((1u << j8) - 1u));
                        if (rank >= kTcKeep) put(i0 + si, rank, wg[pb + q], __expf(rl), sbase, sok);
                    }
                    mm += __popc(grp);
                }
            }
            if (j8 == 0 && si < nv) {
                L.km[i0 + si] = (uint8_t)(m > kTcKeep ? (sok ? kTcKeep : 255) : m);
                L.lse[i0 + si] = lse;
                ll += (double)lse;
            }
            __syncwarp();
        } else {
            // ---- more pairs than the warp's slots (dense halves): one sample
            // at a time, one lane per pair in rounds of 32, two passes
            for (int k = 0; k < 4; ++k) {
                const int si = sb + k;
                if (si >= nv) break;
                const float *xr = xs + si * D;
                const int m0 = ns[2 * si], m1 = ns[2 * si + 1];
                const int d0 = m0 > kCap ? min(128, G) : m0;
                const int cnt = d0 + (m1 > kCap ? max(0, min(128, G - 128)) : m1);
                auto gsel = [&](int j) -> int {
                    if (j < d0) return m0 > kCap ? j : cs[si * 32 + j];
                    return 128 + (m1 > kCap ? j - d0 : cs[si * 32 + 16 + (j - d0)]);
                };
                auto logit = [&](int g) -> float {
                    const float2 *q = psm + g * DS;
                    float r0 = 0.f;
                    for (int d = 0; d < D; ++d) {
                        const float2 qa = q[d];
                        const float tt = fmaf(xr[d], qa.x, -qa.y);
                        r0 = fmaf(tt, tt, r0);
                    }
                    return fmaf(-0.5f, r0, pc[g]);
                };
                // pass 1: online max / sum of exp per lane, then over the warp
                float mx = -INFINITY, sm = 0.f;
                for (int j = lane; j < cnt; j += 32) {
                    const float l = logit(gsel(j));
                    if (l > mx) { sm = sm * __expf(mx - l) + 1.f; mx = l; }
                    else if (l > -INFINITY) sm += __expf(l - mx);   // -inf terms add nothing (and -inf - -inf is NaN)
                }
                float M = mx;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) M = fmaxf(M, __shfl_xor_sync(0xffffffffu, M, o));
                float Ssum = (mx == -INFINITY) ? 0.f : sm * __expf(mx - M);
                Ssum = warp_sum_f(Ssum);
                const float lse = M + logf(Ssum);
                // pass 2: kept pairs in pair order
                int m = 0;
                for (int j0 = 0; j0 < cnt; j0 += 32) {
                    const int j = j0 + lane;
                    const float rl = j < cnt ? logit(gsel(j)) - lse : -INFINITY;
                    m += __popc(__ballot_sync(0xffffffffu, j < cnt && rl >= keep));
                }
                int sbase = -1;
                bool sok = true;
                if (lane == 0 && m > kTcKeep) {
                    sbase = atomicAdd(nspill, m - kTcKeep);
                    sok = sbase + (m - kTcKeep) <= kTcSpill;
                }
                sbase = __shfl_sync(0xffffffffu, sbase, 0);
                sok = __shfl_sync(0xffffffffu, (int)sok, 0) != 0;
                int r = 0;
                for (int j0 = 0; j0 < cnt; j0 += 32) {
                    const int j = j0 + lane;
                    const int g = j < cnt ? gsel(j) : 0;
                    const float rl = j < cnt ? logit(g) - lse : -INFINITY;
                    const bool kp = j < cnt && rl >= keep;
                    const unsigned bal = __ballot_sync(0xffffffffu, kp);
                    if (kp) put(i0 + si, r + __popc(bal & ((1u << lane) - 1u)), g, __expf(rl), sbase, sok);
                    r += __popc(bal);
                }
                if (lane == 0) {
                    L.km[i0 + si] = (uint8_t)(m > kTcKeep ? (sok ? kTcKeep : 255) : m);
                    L.lse[i0 + si] = lse;
                    ll += (double)lse;
                }
            }
        }
        __syncthreads();   // every warp is done with buffer b
        if (tid == 0 && t + 2 < t1 && tile_is_bulk((t + 2) * kST, a.N, args.x_al16)) issue(t + 2, b);
    }
    // drain: no bulk copy may still be writing into shared memory at exit
    if (tid == 0)
        for (int bb = 0; bb < 2; ++bb) {
            const uint32_t issued = bb ? iss1 : iss0;
            const uint32_t used = bb ? use1 : use0;
            const long long d0 = clock64();
            for (uint32_t u = used; u < issued; ++u)
                while (!mbar_try_wait(bars + bb, u & 1u) && clock64() - d0 < a.wait_cycles) {
                }
        }
    for (int o = 16; o > 0; o >>= 1) ll += __shfl_xor_sync(0xffffffffu, ll, o);
    if (lane == 0) s_ll[warp] = ll;
    __syncthreads();
    if (tid == 0) {
        double tot = 0.0;
        for (int w = 0; w < kExThreads / 32; ++w) tot += s_ll[w];
        a.ll_partial[blockIdx.x] = tot;
        L.sp_n[blockIdx.x] = min(*nspill, kTcSpill);
        if (*abort_flag) {
            if (atomicCAS(&a.status->code, 0, (int)GMM_ERR_TIMEOUT) == 0) a.status->fail_iter = a.iter;
            atomicExch(&a.status->halt, 1);
        }
    }
}

// ------------------------------------------------------------------------
// 3. M-step statistics from the compacted responsibility records.  CTA b
// owns the same run of 128-sample tiles as CTA b of the exact kernel (the
// paper's thread t) and the FP32 statistics [G][1 + 2D] (S0 | S1_d | S2_d,
// shifted by the FP32 means mu_f) of its samples in shared memory.  Each
// tile's samples and records are staged by bulk copies two tiles ahead; its
// (sample, Gaussian) pairs are counting-sorted by Gaussian, and the warp that
// owns a Gaussian (g = warp + 32 k; its mu_f row in registers for the whole
// kernel) sums its pairs in registers and adds them to the Gaussian's row:
// no atomics on the statistics.  Then the CTA's spill list (kept pairs
// beyond kTcKeep) is added with shared-memory atomics, and the samples the
// spill list had no room for are recomputed over every Gaussian.
// ------------------------------------------------------------------------
struct MsSmem {
    uint32_t slab, cnt, off, fill, pairs, X[2], kg[2], gam[2], km[2], ovl, misc, bars, total;
};

__host__ __device__ inline MsSmem ms_layout(int D, int G)
{
    MsSmem L;
    uint32_t o = 0;
    L.slab = o; o += 4u * (uint32_t)G * (uint32_t)(1 + 2 * D);
    o = (o + 15u) & ~15u;
    L.cnt = o; o += 4u * 256u;
    L.off = o; o += 4u * 260u;
    L.fill = o; o += 4u * 256u;
    L.pairs = o; o += 2u * kST * kTcKeep;
    o = (o + 127u) & ~127u;
    for (int b = 0; b < 2; ++b) {
        L.X[b] = o; o += ((4u * kST * (uint32_t)D) + 127u) & ~127u;
        L.gam[b] = o; o += 4u * kST * kTcKeep;
        L.kg[b] = o; o += (uint32_t)kST * kTcKeep;
        L.km[b] = o; o += (uint32_t)kST;
    }
    L.ovl = o; o += 4u * kST;
    L.misc = o; o += 16u;
    L.bars = o; o += 16u;
    L.total = o;
    return L;
}

__global__ void __launch_bounds__(kMsThreads, 1) k_em_mstep_lists(ExArgs args)
{
    extern __shared__ __align__(128) unsigned char ms_raw[];
    const EmPassArgs &a = args.a;
    const TcLists &L = args.L;
    if (skip_block(a.status, a.iter)) return;
    const int D = a.D, G = a.G, S = 1 + 2 * D;
    const MsSmem Ls = ms_layout(D, G);
    float *slab = reinterpret_cast<float *>(ms_raw + Ls.slab);
    int *bcnt = reinterpret_cast<int *>(ms_raw + Ls.cnt);
    int *boff = reinterpret_cast<int *>(ms_raw + Ls.off);
    int *bfill = reinterpret_cast<int *>(ms_raw + Ls.fill);
    uint16_t *pairs = reinterpret_cast<uint16_t *>(ms_raw + Ls.pairs);
    int *ovl = reinterpret_cast<int *>(ms_raw + Ls.ovl);
    int *novl = reinterpret_cast<int *>(ms_raw + Ls.misc);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(ms_raw + Ls.misc + 4);
    uint64_t *bars = reinterpret_cast<uint64_t *>(ms_raw + Ls.bars);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t ntiles = (a.N + kST - 1) / kST;
    const int64_t t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
    const float keep = -args.screen;

    // shifts of the Gaussians this warp owns (g = warp + 32 k), kept in registers
    float mu0[8], mu1[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int g = warp + 32 * k;
        mu0[k] = (g < G && lane < D) ? __ldg(a.op.mu + (size_t)g * D + lane) : 0.f;
        mu1[k] = (g < G && lane + 32 < D) ? __ldg(a.op.mu + (size_t)g * D + 32 + lane) : 0.f;
    }
    // one pair (responsibility gv of Gaussian g at sample row x0|x1) with atomics
    auto add_atomic = [&](int g, float gv, float x0, float x1) {
        float *sg = slab + (size_t)g * S;
        if (lane < D) {
            const float u = x0 - __ldg(a.op.mu + (size_t)g * D + lane);
            const float v = gv * u;
            atomicAdd(sg + 1 + lane, v);
            atomicAdd(sg + 1 + D + lane, v * u);
        }
        if (lane + 32 < D) {
            const float u = x1 - __ldg(a.op.mu + (size_t)g * D + 32 + lane);
            const float v = gv * u;
            atomicAdd(sg + 33 + lane, v);
            atomicAdd(sg + 33 + D + lane, v * u);
        }
        if (lane == 0) atomicAdd(sg, gv);
    };

    uint32_t iss0 = 0u, iss1 = 0u;   // issued bulk tiles per buffer (thread 0)
    auto issue = [&](int64_t tile, int b) {   // thread 0 only
        const int64_t i0 = tile * kST;
        const uint32_t xb = 4u * kST * (uint32_t)D;
        const uint32_t bo = (uint32_t)b * (Ls.X[1] - Ls.X[0]);
        if (b) ++iss1; else ++iss0;
        fence_proxy_async();
        mbar_expect_tx(bars + b, xb + 5u * kST * kTcKeep + kST);
        bulk_g2s(ms_raw + Ls.X[0] + bo, a.X + i0 * D, xb, bars + b);
        bulk_g2s(ms_raw + Ls.gam[0] + bo, L.gam + i0 * kTcKeep, 4u * kST * kTcKeep, bars + b);
        bulk_g2s(ms_raw + Ls.kg[0] + bo, L.kg + i0 * kTcKeep, (uint32_t)kST * kTcKeep, bars + b);
        bulk_g2s(ms_raw + Ls.km[0] + bo, L.km + i0, (uint32_t)kST, bars + b);
    };
    if (tid == 0) {
        mbar_init(bars, 1);
        mbar_init(bars + 1, 1);
        *abort_flag = 0;
        *novl = 0;
        fence_mbar_init();
    }
    for (int k = tid; k < G * S; k += kMsThreads) slab[k] = 0.f;
    for (int k = tid; k < 256; k += kMsThreads) { bcnt[k] = 0; bfill[k] = 0; }
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < 2 && t0 + k < t1; ++k)
            if (tile_is_bulk((t0 + k) * kST, a.N, args.x_al16)) issue(t0 + k, k);
    uint32_t use0 = 0u, use1 = 0u;
    for (int64_t t = t0; t < t1; ++t) {
        const int b = (int)((t - t0) & 1);
        const int64_t i0 = t * kST;
        const int nv = (int)min((int64_t)kST, a.N - i0);
        const uint32_t bo = (uint32_t)b * (Ls.X[1] - Ls.X[0]);
        float *xs = reinterpret_cast<float *>(ms_raw + Ls.X[0] + bo);
        float *gms = reinterpret_cast<float *>(ms_raw + Ls.gam[0] + bo);
        uint8_t *kgs = ms_raw + Ls.kg[0] + bo;
        uint8_t *kms = ms_raw + Ls.km[0] + bo;
        if (tile_is_bulk(i0, a.N, args.x_al16)) {
            if (stage_wait(bars + b, (b ? use1 : use0) & 1u, a.wait_cycles, abort_flag)) {
                if (b) ++use1; else ++use0;
            }
        } else {
            for (int k = tid; k < nv * D; k += kMsThreads) xs[k] = __ldg(a.X + i0 * D + k);
            for (int k = tid; k < nv; k += kMsThreads) {
                const int m = L.km[i0 + k];
                kms[k] = (uint8_t)m;
                for (int j = 0; j < kTcKeep && m <= kTcKeep && j < m; ++j) {
                    kgs[k * kTcKeep + j] = L.kg[(i0 + k) * kTcKeep + j];
                    gms[k * kTcKeep + j] = L.gam[(i0 + k) * kTcKeep + j];
                }
            }
        }
        __syncthreads();
        if (*abort_flag) break;   // uniform: nothing sets the flag between the barrier and here
        // ---- histogram of the tile's pairs by Gaussian
        for (int e = tid; e < nv * kTcKeep; e += kMsThreads) {
            const int si = e / kTcKeep, slot = e - si * kTcKeep;
            const int m = kms[si];
            if (m == 255) {
                if (slot == 0) ovl[atomicAdd(novl, 1)] = si;
            } else if (slot < m) {
                atomicAdd(&bcnt[kgs[e]], 1);
            }
        }
        __syncthreads();
        // ---- exclusive scan of the 256 bins (warp 0, eight bins per lane)
        if (warp == 0) {
            int v[8], tot = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) { v[j] = bcnt[8 * lane + j]; tot += v[j]; }
            int inc = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            int run = inc - tot;
#pragma unroll
            for (int j = 0; j < 8; ++j) { boff[8 * lane + j] = run; run += v[j]; }
            if (lane == 31) boff[256] = inc;
        }
        __syncthreads();
        // ---- scatter the pairs (sample * kTcKeep + slot) into their bins
        for (int e = tid; e < nv * kTcKeep; e += kMsThreads) {
            const int si = e / kTcKeep, slot = e - si * kTcKeep;
            const int m = kms[si];
            if (m != 255 && slot < m) {
                const int g = kgs[e];
                pairs[boff[g] + atomicAdd(&bfill[g], 1)] = (uint16_t)e;
            }
        }
        __syncthreads();
        // ---- warp w owns Gaussians w + 32 k: sums in registers, then one
        // read-modify-write of the Gaussian's row
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int g = warp + 32 * k;
            if (g < G) {
                const int pb = boff[g], pe = boff[g + 1];
                if (pb < pe) {
                    float s0 = 0.f, a1 = 0.f, a2 = 0.f, b1 = 0.f, b2 = 0.f;
                    for (int p = pb; p < pe; ++p) {
                        const int e = pairs[p];
                        const float gm = gms[e];
                        const float *xr = xs + (e / kTcKeep) * D;
                        if (lane < D) {
                            const float u = xr[lane] - mu0[k];
                            const float v = gm * u;
                            a1 += v;
                            a2 = fmaf(v, u, a2);
                        }
                        if (lane + 32 < D) {
                            const float u = xr[lane + 32] - mu1[k];
                            const float v = gm * u;
                            b1 += v;
                            b2 = fmaf(v, u, b2);
                        }
                        s0 += gm;
                    }
                    float *sg = slab + (size_t)g * S;
                    if (lane == 0) sg[0] += s0;
                    if (lane < D) { sg[1 + lane] += a1; sg[1 + D + lane] += a2; }
                    if (lane + 32 < D) { sg[33 + lane] += b1; sg[33 + D + lane] += b2; }
                }
            }
        }
        __syncthreads();
        // ---- samples the spill list had no room for: every Gaussian, one
        // warp per sample, shared-memory atomics (never taken in practice)
        const int nd = *novl;
        for (int r = warp; r < nd; r += kMsThreads / 32) {
            const int si = ovl[r];
            const float *xr = xs + si * D;
            const float x0 = lane < D ? xr[lane] : 0.f;
            const float x1 = lane + 32 < D ? xr[lane + 32] : 0.f;
            const float ls = __ldg(L.lse + i0 + si);
            for (int g = 0; g < G; ++g) {
                const float2 *pp = a.op.sm + (size_t)g * D;
                float acc = 0.f;
                if (lane < D) { const float2 q = __ldg(pp + lane); const float tt = fmaf(x0, q.x, -q.y); acc = tt * tt; }
                if (lane + 32 < D) { const float2 q = __ldg(pp + 32 + lane); const float tt = fmaf(x1, q.x, -q.y); acc = fmaf(tt, tt, acc); }
                acc = warp_sum_f(acc);
                const float rl = fmaf(-0.5f, acc, __ldg(a.op.c + g)) - ls;
                if (rl >= keep) add_atomic(g, __expf(rl), x0, x1);   // the same rule as the kept pairs
            }
        }
        for (int k = tid; k < 256; k += kMsThreads) { bcnt[k] = 0; bfill[k] = 0; }
        __syncthreads();   // every warp is done with buffer b, the bins and the list
        if (tid == 0) {
            *novl = 0;
            if (t + 2 < t1 && tile_is_bulk((t + 2) * kST, a.N, args.x_al16)) issue(t + 2, b);
        }
    }
    // drain: no bulk copy may still be writing into shared memory at exit
    if (tid == 0)
        for (int bb = 0; bb < 2; ++bb) {
            const uint32_t issued = bb ? iss1 : iss0;
            const uint32_t used = bb ? use1 : use0;
            const long long d0 = clock64();
            for (uint32_t u = used; u < issued; ++u)
                while (!mbar_try_wait(bars + bb, u & 1u) && clock64() - d0 < a.wait_cycles) {
                }
        }
    __syncthreads();
    // ---- the spill list of this CTA's samples (kept pairs beyond kTcKeep)
    if (!*abort_flag) {
        const int ns = L.sp_n[blockIdx.x];
        const int64_t *sp_ig = L.sp_ig + (size_t)blockIdx.x * kTcSpill;
        const float *sp_gam = L.sp_gam + (size_t)blockIdx.x * kTcSpill;
        for (int e = warp; e < ns; e += kMsThreads / 32) {
            const float gv = sp_gam[e];
            if (!(gv > 0.f)) continue;
            const int64_t ig = sp_ig[e];
            const int64_t i = ig >> 8;
            const int g = (int)(ig & 255);
            const float *xr = a.X + i * D;
            add_atomic(g, gv, lane < D ? __ldg(xr + lane) : 0.f, lane + 32 < D ? __ldg(xr + 32 + lane) : 0.f);
        }
    }
    __syncthreads();
    // ---- the CTA's statistics -> its FP64 partial
    double *P = a.partial + (size_t)blockIdx.x * G * S;
    for (int k = tid; k < G * S; k += kMsThreads) P[k] = (double)slab[k];
    if (tid == 0 && *abort_flag) {
        if (atomicCAS(&a.status->code, 0, (int)GMM_ERR_TIMEOUT) == 0) a.status->fail_iter = a.iter;
        atomicExch(&a.status->halt, 1);
    }
}

}  // namespace

namespace {
int optin_smem()
{
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return optin;
}
// pair slots per warp of the exact kernel: what shared memory leaves, up to 256
int ex_wp(int D, int G)
{
    const long long rest = (long long)optin_smem() - 2048 - (long long)ex_layout(D, G, 0).total;
    const long long wp = rest / (6 * 32);
    return (int)(wp >= 256 ? 256 : (wp / 32) * 32);
}
}  // namespace

bool em_tc_supported(int32_t D, int32_t G)
{
    if (D < 1 || D > 64 || G < 1 || G > 256) return false;
    const int NG = (G + 15) / 16 * 16;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // dynamic layouts plus the kernels' static shared memory
    return tc_layout(D, NG).total + 1024u + 2048u <= (uint32_t)optin && ex_wp(D, G) >= 32 &&
           ms_layout(D, G).total + 2048u <= (uint32_t)optin;
}

int em_tc_grid(int sms) { return sms; }

namespace {
size_t al256(size_t n) { return (n + 255u) & ~(size_t)255u; }
}

size_t em_tc_list_bytes(int64_t N, int grid)
{
    const size_t n = (size_t)N, sp = (size_t)grid * kTcSpill;
    return al256(4u * n * kTcKeep) + al256(n * kTcKeep) + al256(32u * n) + al256(4u * n) + al256(2u * n) +
           al256(n) + al256(8u * sp) + al256(4u * sp) + al256(4u * (size_t)grid) + al256(4u * n) + 256u;
}

TcLists em_tc_lists(void *base, int64_t N, int grid)
{
    const size_t n = (size_t)N, sp = (size_t)grid * kTcSpill;
    unsigned char *p = static_cast<unsigned char *>(base);
    TcLists L;
    L.gam = reinterpret_cast<float *>(p);       p += al256(4u * n * kTcKeep);
    L.kg = p;                                   p += al256(n * kTcKeep);
    L.cand = p;                                 p += al256(32u * n);
    L.lse = reinterpret_cast<float *>(p);       p += al256(4u * n);
    L.cnt = p;                                  p += al256(2u * n);
    L.km = p;                                   p += al256(n);
    L.sp_ig = reinterpret_cast<int64_t *>(p);   p += al256(8u * sp);
    L.sp_gam = reinterpret_cast<float *>(p);    p += al256(4u * sp);
    L.sp_n = reinterpret_cast<int32_t *>(p);    p += al256(4u * (size_t)grid);
    L.defer = reinterpret_cast<int32_t *>(p);
    return L;
}

cudaError_t launch_em_pass_tc(const EmPassArgs &a, const TcLists &L, int32_t grid, int32_t ms_grid, cudaStream_t s)
{
    const float scr = (float)std::log((double)(a.N_total > a.N ? a.N_total : a.N) * 1e9);
    const int al = (reinterpret_cast<uintptr_t>(a.X) & 15u) == 0;
    TcArgs t{a, L, (a.G + 15) / 16 * 16, (a.D + 15) / 16, scr, al,
             (a.D % 2 == 0 && (reinterpret_cast<uintptr_t>(a.X) & 7u) == 0) ? 1 : 0};
    const size_t sm1 = tc_layout(a.D, t.NG).total + 1024u;
    cudaError_t e = cudaFuncSetAttribute(k_em_screen_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    if (e != cudaSuccess) return e;
    k_em_screen_tc<<<grid, kThreads, sm1, s>>>(t);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ExArgs x{a, L, scr, al, ex_wp(a.D, a.G)};
    const size_t sm2 = ex_layout(a.D, a.G, x.wp).total;
    if ((e = cudaFuncSetAttribute(k_em_exact, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2)) != cudaSuccess)
        return e;
    k_em_exact<<<grid, kExThreads, sm2, s>>>(x);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t sm3 = ms_layout(a.D, a.G).total;
    if ((e = cudaFuncSetAttribute(k_em_mstep_lists, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3)) !=
        cudaSuccess)
        return e;
    k_em_mstep_lists<<<ms_grid, kMsThreads, sm3, s>>>(x);
    count_launches(3);
    return cudaGetLastError();
}

}  // namespace gmm
