// Register-blocked FP32 EM pass for shapes whose per-CTA statistics do not
// fit in shared memory next to all N_G operands (e.g. N_G = 1024, D = 128).
// The iteration is the paper's map step (Sec. 2.1) split over blocks of 64
// Gaussians:
//   k_blk_lse     grid (sample chunk) x (Gaussian block): FP32 log-densities
//                 log w_g N(x_i | g) of the block (Eq. 15, the direct form
//                 sum_d (x_d s_gd - mu_gd s_gd)^2 in two FMA chains of D/2
//                 terms each), reduced per sample to a partial log-sum-exp
//                 (max, sum of exp) over the block (Eqs. 16-18);
//   k_blk_combine log p(x_i) = merge of the blocks' partials; the CTA's FP64
//                 log-likelihood;
//   k_blk_em      the same log-densities again, responsibilities
//                 l_{g,i} = exp(log w_g N - log p(x_i)) (Eq. 3), those below
//                 1e-9 / N set to 0 (every Gaussian loses less than 1e-9 of
//                 mass), and the block's shifted statistics sum l,
//                 sum l (x - mu_f), sum l (x - mu_f)^2 (Eqs. 9-11 about the
//                 FP32 mean mu_f of the iteration start) into the rows of the
//                 chunk's FP64 partial.
// Both log-density kernels hold the block's operands (s, mu s) in shared
// memory and stream the chunk's samples in tiles staged by cp.async two-deep;
// each thread computes a register block of samples x 4 Gaussians, so a
// 128-bit shared load feeds 8-16 FMAs.  FP32 sums: a statistic is summed over
// at most 64 samples in registers, then over at most 64 tiles in shared
// memory, then in FP64.
#include <cmath>

#include "gmm_internal.cuh"
#include "gmm_km_exact.cuh"

namespace gmm {

namespace {

constexpr int kBG = 64;        // Gaussians per block
constexpr int kBThreads = 256; // threads per CTA: a 16 x 16 grid of register blocks
constexpr int kBFlush = 64;    // tiles summed in shared memory between FP64 flushes

__device__ __forceinline__ bool blk_skip(const DevStatus *st, int iter)
{
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = (st && (st->halt != 0 || iter > st->stop_after)) ? 1 : 0;   // no status: inference
    __syncthreads();
    return s_skip != 0;
}

// Padded widths: D8 = D rounded up to 8 (zero dimensions add nothing); the
// sample-row stride XS and operand-row stride OS are odd multiples of 16
// bytes, so rows read together by a load phase lie in distinct bank groups.
__host__ __device__ inline int blk_d8(int D) { return (D + 7) & ~7; }
__host__ __device__ inline int blk_odd16(int n) { return ((n / 4) & 1) ? n : n + 4; }   // n a multiple of 4
__host__ __device__ inline int blk_xs(int D) { return blk_odd16(blk_d8(D)); }
__host__ __device__ inline int blk_os(int D) { return blk_odd16(2 * blk_d8(D)); }
constexpr int kGS = kBG + 4;   // responsibility-tile row stride
constexpr int kMacc = 17;      // float4 slots of shared-memory sums per M-step thread: 8 S1, 8 S2, 1 S0

struct BlkArgs {
    EmPassArgs a;
    int32_t n_gb;        // Gaussian blocks: ceil(G / 64)
    int32_t n_chunks;    // sample chunks
    int32_t x_v4;        // D % 4 == 0 and X 16-byte aligned: rows staged 16 bytes at a time
    float2 *part;        // [n_gb][N] (max, sum of exp) per sample and block
    float *lse;          // [N] log p(x_i)
    double *out;         // inference: log p(x_i) in FP64 here instead of lse and the log-likelihood
    const int64_t *n_dev;   // non-null: the samples actually present (device), at most N (part's stride)
    // candidate records (non-null rec_n): per (block, sample) the Gaussians
    // whose log-density lies within `screen` of the block's best
    uint8_t *rec_n;         // [n_gb][N] count (> kBRec: some not recorded)
    uint16_t *rec_g;        // [n_gb][N][kBRec]
    float *rec_l;           // [n_gb][N][kBRec] their log-densities
    float screen;           // ln(N * 1e9)
    // per-sample records of the kept responsibilities (k_blk_combine_rec)
    uint8_t *rc;            // [N] count (255: the sample goes through k_blk_em)
    uint16_t *rg;           // [N][kRecSlots]
    float *rgam;            // [N][kRecSlots]
};
constexpr int kBRec = 8;    // recorded candidates per (block, sample)

// Samples present: a.N, or fewer when the count is known only on the device.
__device__ __forceinline__ int64_t blk_n(const BlkArgs &b) { return b.n_dev ? *b.n_dev : b.a.N; }

__host__ __device__ inline size_t blk_smem(int D, int TS, bool em)
{
    size_t f = (size_t)kBG * blk_os(D) + kBG + 2 * (size_t)TS * blk_xs(D) + TS;
    if (em) f += (size_t)TS * kGS + 4 * (size_t)kMacc * kBThreads;
    return f * sizeof(float);
}

__device__ __forceinline__ void cp_async16(float *dst, const float *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(float *dst, const float *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// (m, s) partial log-sum-exp merge; -inf terms add nothing
__device__ __forceinline__ float2 lse_merge(float2 p, float2 q)
{
    const float M = fmaxf(p.x, q.x);
    if (M == -INFINITY) return make_float2(-INFINITY, 0.f);
    return make_float2(M, p.y * __expf(p.x - M) + q.y * __expf(q.x - M));
}

// Operands of Gaussian block gb -> shared memory: row g holds, per pair of
// dimensions (2p, 2p+1), (s_2p, s_2p+1, -mu_2p s_2p, -mu_2p+1 s_2p+1) over D8
// dimensions (zeros past D; zero rows and c = -inf past G), the packed-FP32
// operands of two dimensions.
__device__ void blk_stage_operands(const EmPassArgs &a, int g0, float *op, float *cg)
{
    const int D = a.D, D8 = blk_d8(D), OS = blk_os(D);
    for (int k = threadIdx.x; k < kBG * D8; k += kBThreads) {
        const int g = k / D8, d = k - g * D8;
        float2 q = make_float2(0.f, 0.f);
        if (g0 + g < a.G && d < D) q = __ldg(a.op.sm + (size_t)(g0 + g) * D + d);
        op[g * OS + 4 * (d >> 1) + (d & 1)] = q.x;
        op[g * OS + 4 * (d >> 1) + 2 + (d & 1)] = -q.y;
    }
    for (int g = threadIdx.x; g < kBG; g += kBThreads) cg[g] = g0 + g < a.G ? __ldg(a.op.c + g0 + g) : -INFINITY;
}

// Sample tile t (TS rows) -> buffer xb: cp.async for the rows that exist,
// zeros for the rest; the zero columns D..D8-1 are written once beforehand.
template <int TS>
__device__ void blk_stage_tile(const BlkArgs &b, int64_t N, int64_t t, float *xb)
{
    const EmPassArgs &a = b.a;
    const int D = a.D, XS = blk_xs(D);
    const int64_t i0 = t * TS;
    const int nv = (int)min((int64_t)TS, N - i0);
    if (b.x_v4) {
        const int q4 = D / 4;
        for (int k = threadIdx.x; k < TS * q4; k += kBThreads) {
            const int r = k / q4, c = k - r * q4;
            if (r < nv) cp_async16(xb + r * XS + 4 * c, a.X + (i0 + r) * D + 4 * c);
            else *reinterpret_cast<float4 *>(xb + r * XS + 4 * c) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    } else {
        for (int k = threadIdx.x; k < TS * D; k += kBThreads) {
            const int r = k / D, c = k - r * D;
            if (r < nv) cp_async4(xb + r * XS + c, a.X + (i0 + r) * D + c);
            else xb[r * XS + c] = 0.f;
        }
    }
}

// FP32 log-densities of this thread's register block: samples sg + 16 k
// (k < RS), Gaussians gg + 16 j (j < 4); two FMA chains per pair (dimensions
// 0, 2 mod 4 and 1, 3 mod 4), the direct form of the CUDA-core pass, two
// dimensions per packed FP32 instruction (each half an IEEE fma: the same
// values as scalar FMAs).
template <int RS>
__device__ __forceinline__ void blk_logits(const float *xb, const float *op, const float *cg, int XS, int OS, int D8,
                                           int sg, int gg, float (&l)[RS][4])
{
    float2 acc[RS][4];
#pragma unroll
    for (int k = 0; k < RS; ++k)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[k][j] = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int d4 = 0; d4 < D8 / 4; ++d4) {
        float4 xv[RS];
#pragma unroll
        for (int k = 0; k < RS; ++k) xv[k] = *reinterpret_cast<const float4 *>(xb + (sg + 16 * k) * XS + 4 * d4);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float4 qa = *reinterpret_cast<const float4 *>(op + (gg + 16 * j) * OS + 8 * d4);
            const float4 qb = *reinterpret_cast<const float4 *>(op + (gg + 16 * j) * OS + 8 * d4 + 4);
            const float2 sa = make_float2(qa.x, qa.y), ma = make_float2(qa.z, qa.w);
            const float2 sb = make_float2(qb.x, qb.y), mb = make_float2(qb.z, qb.w);
#pragma unroll
            for (int k = 0; k < RS; ++k) {
                const float2 t01 = __ffma2_rn(make_float2(xv[k].x, xv[k].y), sa, ma);
                const float2 t23 = __ffma2_rn(make_float2(xv[k].z, xv[k].w), sb, mb);
                acc[k][j] = __ffma2_rn(t01, t01, acc[k][j]);
                acc[k][j] = __ffma2_rn(t23, t23, acc[k][j]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float c = cg[gg + 16 * j];
#pragma unroll
        for (int k = 0; k < RS; ++k) l[k][j] = fmaf(-0.5f, acc[k][j].x + acc[k][j].y, c);
    }
}

// ------------------------------------------------------------------------
// Phase 1: partial log-sum-exp of each sample over one block of Gaussians.
// Thread (sg, gg): warp w, lane l -> sg = 8 (w & 1) + (l & 7),
// gg = 4 (w >> 1) + (l >> 3).
// ------------------------------------------------------------------------
template <int RS>
__global__ void __launch_bounds__(kBThreads, 1) k_blk_lse(BlkArgs b)
{
    constexpr int TS = 16 * RS;
    extern __shared__ __align__(16) float bsm[];
    const EmPassArgs &a = b.a;
    if (blk_skip(a.status, a.iter)) return;
    if (blk_n(b) == 0) return;   // nothing to write (uniform)
    const int D = a.D, D8 = blk_d8(D), XS = blk_xs(D), OS = blk_os(D);
    const int gb = blockIdx.x % b.n_gb, chunk = blockIdx.x / b.n_gb;   // the chunk's blocks run side by side
    float *op = bsm, *cg = op + kBG * OS, *xt = cg + kBG;
    float2 *red = reinterpret_cast<float2 *>(xt + 2 * TS * XS);   // [4][TS] partials of the four Gaussian quarters
    float *mb = reinterpret_cast<float *>(red + 4 * TS);           // [TS] block maximum per sample (records)
    int *cntb = reinterpret_cast<int *>(mb + TS);                  // [TS] candidates recorded per sample
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int sg = 8 * (w & 1) + (lane & 7), gg = 4 * (w >> 1) + (lane >> 3);
    const bool rec = b.rec_n != nullptr;
    for (int s = tid; s < TS; s += kBThreads) cntb[s] = 0;
    blk_stage_operands(a, gb * kBG, op, cg);
    for (int k = tid; k < 2 * TS * (XS - D); k += kBThreads) {   // zero columns D..XS-1 of both buffers
        const int r = k / (XS - D);
        xt[r * XS + D + (k - r * (XS - D))] = 0.f;
    }
    const int64_t N = blk_n(b);
    const int64_t ntiles = (N + TS - 1) / TS;
    const int64_t t0 = ntiles * chunk / b.n_chunks, t1 = ntiles * (chunk + 1) / b.n_chunks;
    __syncthreads();
    if (t0 < t1) blk_stage_tile<TS>(b, N, t0, xt);
    cp_commit();
    for (int64_t t = t0; t < t1; ++t) {
        const int bi = (int)((t - t0) & 1);
        if (t + 1 < t1) blk_stage_tile<TS>(b, N, t + 1, xt + (1 - bi) * TS * XS);
        cp_commit();
        cp_wait<1>();
        __syncthreads();
        float l[RS][4];
        blk_logits<RS>(xt + bi * TS * XS, op, cg, XS, OS, D8, sg, gg, l);
        // per sample: this thread's four Gaussians, then the warp's four
        // Gaussian groups (lanes ^ 8, ^ 16), then the four warps' quarters
#pragma unroll
        for (int k = 0; k < RS; ++k) {
            const float m = fmaxf(fmaxf(l[k][0], l[k][1]), fmaxf(l[k][2], l[k][3]));
            float s = 0.f;
            if (m != -INFINITY)
#pragma unroll
                for (int j = 0; j < 4; ++j) s += l[k][j] > -INFINITY ? __expf(l[k][j] - m) : 0.f;
            float2 p = make_float2(m, s);
            p = lse_merge(p, make_float2(__shfl_xor_sync(0xffffffffu, p.x, 8), __shfl_xor_sync(0xffffffffu, p.y, 8)));
            p = lse_merge(p, make_float2(__shfl_xor_sync(0xffffffffu, p.x, 16), __shfl_xor_sync(0xffffffffu, p.y, 16)));
            if (lane < 8) red[(w >> 1) * TS + sg + 16 * k] = p;
        }
        __syncthreads();
        const int64_t i0 = t * TS;
        for (int s = tid; s < TS; s += kBThreads) {
            float2 p = make_float2(-INFINITY, 0.f);
            if (i0 + s < N) {
                p = red[s];
#pragma unroll
                for (int q = 1; q < 4; ++q) p = lse_merge(p, red[q * TS + s]);
                b.part[(size_t)gb * a.N + i0 + s] = p;
            }
            if (rec) mb[s] = p.x;
        }
        if (rec) {   // uniform
            // candidates: log-density within `screen` of the block's best (a
            // superset of those within it of the best over all blocks)
            __syncthreads();
#pragma unroll
            for (int k = 0; k < RS; ++k) {
                const int s = sg + 16 * k;
                if (i0 + s < N) {
                    const float thr = mb[s] - b.screen;
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        if (l[k][j] >= thr) {   // -inf logits (past N_G) never pass
                            const int slot = atomicAdd(cntb + s, 1);
                            if (slot < kBRec) {
                                const size_t o = ((size_t)gb * a.N + i0 + s) * kBRec + slot;
                                b.rec_g[o] = (uint16_t)(gb * kBG + gg + 16 * j);
                                b.rec_l[o] = l[k][j];
                            }
                        }
                }
            }
            __syncthreads();
            for (int s = tid; s < TS; s += kBThreads) {
                if (i0 + s < N) b.rec_n[(size_t)gb * a.N + i0 + s] = (uint8_t)min(cntb[s], 255);
                cntb[s] = 0;
            }
        }
        // the next iteration restages buffer bi only after its barrier, which
        // every thread reaches after it is done with red and buffer bi
    }
    cp_wait<0>();
}

// log p(x_i) from the blocks' partials; FP64 log-likelihood per 128 samples.
__global__ void __launch_bounds__(128) k_blk_combine(BlkArgs b)
{
    __shared__ double sh[128];
    const EmPassArgs &a = b.a;
    if (blk_skip(a.status, a.iter)) return;
    const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
    double v = 0.0;
    if (i < blk_n(b)) {
        float2 p = b.part[i];
        for (int q = 1; q < b.n_gb; ++q) p = lse_merge(p, b.part[(size_t)q * a.N + i]);
        if (b.out) {   // the inference kernel's form: max + log(sum) in FP64
            b.out[i] = (double)p.x + log((double)p.y);
            return;
        }
        const float ls = p.x + logf(p.y);
        b.lse[i] = ls;
        v = (double)ls;
        if (b.rc) {
            // the recorded candidates whose responsibility reaches exp(-screen),
            // block after block, each block's in Gaussian order
            int m = 0;
            bool over = false;
            for (int q = 0; q < b.n_gb; ++q) {
                const size_t base = (size_t)q * a.N + i;
                const int n = b.rec_n[base];
                if (n > kBRec) {
                    over = true;
                    continue;
                }
                int eg[kBRec];
                float el[kBRec];
#pragma unroll
                for (int e = 0; e < kBRec; ++e) {
                    eg[e] = e < n ? (int)b.rec_g[base * kBRec + e] : 0xFFFF;
                    el[e] = e < n ? b.rec_l[base * kBRec + e] : -INFINITY;
                }
                int last = -1;
                for (int r = 0; r < n; ++r) {
                    int bg = 0x10000;
                    float bl = -INFINITY;
#pragma unroll
                    for (int e = 0; e < kBRec; ++e)
                        if (eg[e] > last && eg[e] < bg) {
                            bg = eg[e];
                            bl = el[e];
                        }
                    last = bg;
                    const float rl = bl - ls;
                    if (rl >= -b.screen) {
                        if (m < kRecSlots) {
                            b.rg[i * kRecSlots + m] = (uint16_t)bg;
                            b.rgam[i * kRecSlots + m] = __expf(rl);
                        }
                        ++m;
                    }
                }
            }
            b.rc[i] = (uint8_t)((over || m > kRecSlots) ? 255 : m);
        }
    }
    if (b.out) return;   // the block's threads past N
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = 64; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) a.ll_partial[blockIdx.x] = sh[0];
}

// ------------------------------------------------------------------------
// Phase 2: responsibilities and statistics of one block of Gaussians over one
// sample chunk.  E-step threads as in phase 1 (RS = 4: 64-sample tiles); the
// responsibilities go to a [64 samples][64 Gaussians] tile.  M-step thread
// t < 16 NDG (NDG = D8 / 8 dimension groups): Gaussians 4 (t / NDG) + j,
// dimensions 8 (t % NDG) + e; the threads of a warp skip a sample together
// when none of their Gaussians holds a responsibility there.
// ------------------------------------------------------------------------
__global__ void __launch_bounds__(kBThreads, 1) k_blk_em(BlkArgs b)
{
    constexpr int RS = 4, TS = 16 * RS;
    extern __shared__ __align__(16) float bsm[];
    const EmPassArgs &a = b.a;
    if (blk_skip(a.status, a.iter)) return;
    const int D = a.D, G = a.G, D8 = blk_d8(D), XS = blk_xs(D), OS = blk_os(D), S = 1 + 2 * D;
    const int gb = blockIdx.x % b.n_gb, chunk = blockIdx.x / b.n_gb, g0 = gb * kBG;
    float *op = bsm, *cg = op + kBG * OS, *xt = cg + kBG, *lt = xt + 2 * TS * XS, *gam = lt + TS;
    // shared-memory FP32 sums, slot q of thread t at macc[q * kBThreads + t]:
    // q = 2 j + h: S1 of Gaussian j, dimensions 4 h..4 h+3 of the group;
    // 8 + 2 j + h: S2; 16: S0 of the four Gaussians
    float4 *macc = reinterpret_cast<float4 *>(gam + TS * kGS);
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int sg = 8 * (w & 1) + (lane & 7), gg = 4 * (w >> 1) + (lane >> 3);
    const int NDG = D8 / 8;
    const bool mact = tid < 16 * NDG;
    const int mq = mact ? tid / NDG : 0, dg = mact ? tid - mq * NDG : 0;
    const float keep = (float)(1e-9 / (double)(a.N_total > a.N ? a.N_total : a.N));
    blk_stage_operands(a, g0, op, cg);
    for (int k = tid; k < 2 * TS * (XS - D); k += kBThreads) {
        const int r = k / (XS - D);
        xt[r * XS + D + (k - r * (XS - D))] = 0.f;
    }
    for (int q = 0; q < kMacc; ++q) macc[q * kBThreads + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    // this thread's M-step shifts, negated: -mu_f (0 past G or D), pairs of dimensions
    float2 nmu[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int g = g0 + 4 * mq + j, d = 8 * dg + 2 * e;
            nmu[j][e] = make_float2((mact && g < G && d < D) ? -__ldg(a.op.mu + (size_t)g * D + d) : 0.f,
                                    (mact && g < G && d + 1 < D) ? -__ldg(a.op.mu + (size_t)g * D + d + 1) : 0.f);
        }
    double *P = a.partial + (size_t)chunk * G * S;
    int flushes = 0, since = 0;
    // shared-memory sums -> FP64 partial rows of this block (the first flush writes)
    auto flush = [&]() {
        if (mact) {
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 f0 = macc[16 * kBThreads + tid];
            const float s0v[4] = {f0.x, f0.y, f0.z, f0.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int g = g0 + 4 * mq + j;
                if (g >= G) continue;
                double *row = P + (size_t)g * S;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float4 f1 = macc[(2 * j + h) * kBThreads + tid], f2 = macc[(8 + 2 * j + h) * kBThreads + tid];
                    const float v1[4] = {f1.x, f1.y, f1.z, f1.w}, v2[4] = {f2.x, f2.y, f2.z, f2.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int d = 8 * dg + 4 * h + e;
                        if (d >= D) continue;
                        row[1 + d] = flushes ? row[1 + d] + (double)v1[e] : (double)v1[e];
                        row[1 + D + d] = flushes ? row[1 + D + d] + (double)v2[e] : (double)v2[e];
                    }
                    macc[(2 * j + h) * kBThreads + tid] = z;
                    macc[(8 + 2 * j + h) * kBThreads + tid] = z;
                }
                if (dg == 0) row[0] = flushes ? row[0] + (double)s0v[j] : (double)s0v[j];
            }
            macc[16 * kBThreads + tid] = z;
        }
        ++flushes;
        since = 0;
    };
    const int64_t N = blk_n(b);
    const int64_t ntiles = (N + TS - 1) / TS;
    const int64_t t0 = ntiles * chunk / b.n_chunks, t1 = ntiles * (chunk + 1) / b.n_chunks;
    __syncthreads();
    if (t0 < t1) {
        blk_stage_tile<TS>(b, N, t0, xt);
        for (int s = tid; s < TS; s += kBThreads) lt[s] = t0 * TS + s < N ? b.lse[t0 * TS + s] : 0.f;
    }
    cp_commit();
    for (int64_t t = t0; t < t1; ++t) {
        const int bi = (int)((t - t0) & 1);
        float *xb = xt + bi * TS * XS;
        cp_wait<0>();
        __syncthreads();
        // ---- E: log-densities -> responsibilities (0 below keep; 0 past N)
        {
            float l[RS][4];
            blk_logits<RS>(xb, op, cg, XS, OS, D8, sg, gg, l);
            const int64_t i0 = t * TS;
#pragma unroll
            for (int k = 0; k < RS; ++k) {
                const int s = sg + 16 * k;
                const float ls = lt[s];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float gm = i0 + s < N ? __expf(l[k][j] - ls) : 0.f;
                    gam[s * kGS + gg + 16 * j] = gm >= keep ? gm : 0.f;
                }
            }
        }
        __syncthreads();
        // the next tile's samples (other buffer) and log p, while the M-step
        // runs: the E-step is done with lt
        if (t + 1 < t1) {
            blk_stage_tile<TS>(b, N, t + 1, xt + (1 - bi) * TS * XS);
            for (int s = tid; s < TS; s += kBThreads) lt[s] = (t + 1) * TS + s < N ? b.lse[(t + 1) * TS + s] : 0.f;
        }
        cp_commit();
        // ---- M: this thread's 4 Gaussians x 8 dimensions over the tile's
        // samples, two dimensions per packed FP32 instruction
        float2 s1[4][4], s2[4][4];
        float s0[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            s0[j] = 0.f;
#pragma unroll
            for (int e = 0; e < 4; ++e) { s1[j][e] = make_float2(0.f, 0.f); s2[j][e] = make_float2(0.f, 0.f); }
        }
        // samples where one of the warp's Gaussians holds a responsibility
        // (the warp's active M-step threads cover Gaussian quads mqa..mqb), a
        // 64-bit mask, then two samples at a time
        uint64_t amask;
        {
            const int mqa = (int)__reduce_min_sync(0xffffffffu, mact ? (unsigned)mq : 0xFFFFu);
            const int mqb = (int)__reduce_max_sync(0xffffffffu, mact ? (unsigned)mq : 0u);
            bool on[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                bool v = false;
                for (int q = mqa; q <= mqb; ++q) {
                    const float4 g4 = *reinterpret_cast<const float4 *>(gam + (lane + 32 * h) * kGS + 4 * q);
                    v = v || g4.x > 0.f || g4.y > 0.f || g4.z > 0.f || g4.w > 0.f;
                }
                on[h] = v;   // sample lane + 32 h, whatever this lane's own M-step role
            }
            amask = (uint64_t)__ballot_sync(0xffffffffu, on[0]) | ((uint64_t)__ballot_sync(0xffffffffu, on[1]) << 32);
        }
        auto msample = [&](int s) {
            const float4 g4 = *reinterpret_cast<const float4 *>(gam + s * kGS + 4 * mq);
            const float4 xa = *reinterpret_cast<const float4 *>(xb + s * XS + 8 * dg);
            const float4 xc = *reinterpret_cast<const float4 *>(xb + s * XS + 8 * dg + 4);
            const float2 xe[4] = {make_float2(xa.x, xa.y), make_float2(xa.z, xa.w), make_float2(xc.x, xc.y),
                                  make_float2(xc.z, xc.w)};
            const float gj[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                s0[j] += gj[j];
                const float2 gg2 = make_float2(gj[j], gj[j]);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float2 u = __fadd2_rn(xe[e], nmu[j][e]);
                    const float2 v = __fmul2_rn(gg2, u);
                    s1[j][e] = __fadd2_rn(s1[j][e], v);
                    s2[j][e] = __ffma2_rn(v, u, s2[j][e]);
                }
            }
        };
        while (amask) {
            const int sa = __ffsll((long long)amask) - 1;
            amask &= amask - 1;
            msample(sa);
            if (amask) {
                const int sb = __ffsll((long long)amask) - 1;
                amask &= amask - 1;
                msample(sb);
            }
        }
        if (mact) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    float4 f1 = macc[(2 * j + h) * kBThreads + tid], f2 = macc[(8 + 2 * j + h) * kBThreads + tid];
                    f1.x += s1[j][2 * h].x; f1.y += s1[j][2 * h].y; f1.z += s1[j][2 * h + 1].x; f1.w += s1[j][2 * h + 1].y;
                    f2.x += s2[j][2 * h].x; f2.y += s2[j][2 * h].y; f2.z += s2[j][2 * h + 1].x; f2.w += s2[j][2 * h + 1].y;
                    macc[(2 * j + h) * kBThreads + tid] = f1;
                    macc[(8 + 2 * j + h) * kBThreads + tid] = f2;
                }
            float4 f0 = macc[16 * kBThreads + tid];
            f0.x += s0[0]; f0.y += s0[1]; f0.z += s0[2]; f0.w += s0[3];
            macc[16 * kBThreads + tid] = f0;
        }
        if (++since == kBFlush) flush();
        __syncthreads();   // buffer bi and gam are free
    }
    cp_wait<0>();
    flush();   // also writes the rows of a chunk with no tiles (zeros)
}


// ------------------------------------------------------------------------
// k-means map step (Sec. 3 with Sec. 2.1's chunking) for shapes beyond the
// tiled CUDA-core form (D > 64 or N_G > 256), register-blocked like the EM
// form, over blocks of 64 means:
//   k_bkm_norms    max |cs_g|^2 over all means (the near-tie bound's norm);
//   k_bkm_dist     grid (sample chunk) x (block of means): FP32 distances
//                  sum_d (xs_d - cs_gd)^2 in scaled coordinates xs = x sqrt(w),
//                  cs = mu sqrt(w) (two FMA chains, as the thread-per-sample
//                  form), each sample's best, runner-up and argmin over the
//                  block -> part [block][N];
//   k_bkm_combine  per sample the blocks' results merged, then the exact
//                  decision: the FP32 winner where the runner-up minus its
//                  rounding bound exceeds the winner plus its bound, else
//                  every mean re-decided in FP64 (lowest index on ties) ->
//                  assign[N];
//   k_bkm_stats    grid as k_bkm_dist: count, sum (x - mu_f), sum (x - mu_f)^2
//                  of the block's means over the chunk's samples (mu_f the
//                  old mean rounded to FP32), into the chunk's FP64 partial.
// ------------------------------------------------------------------------
struct BkmArgs {
    const float *X;
    int64_t N;
    int32_t D, G;
    const double *means;    // means at the start of the iteration
    const double *w;        // [D] FP64 distance weights
    const float *sw;        // [D] FP32 sqrt(w)
    float2 *part;           // [n_gb][N] (best, runner-up) of each block
    uint8_t *arg;           // [n_gb][N] the block's argmin (index within the block)
    float *nmax;            // [1] max |cs_g|^2
    float *snorm;           // [N] |xs_i|^2 (written by the first block's CTAs)
    int32_t *defer;         // [N] samples left to the FP64 re-decision; defer_n their count
    int32_t *defer_n;
    int32_t *assign;        // [N]
    double *partial;        // [n_chunks][G][1 + 2D]
    int32_t n_gb, n_chunks, x_v4;
    const DevStatus *status;
};

__global__ void __launch_bounds__(256) k_bkm_norms(BkmArgs b)
{
    __shared__ float s_m[256];
    if (blk_skip(b.status, 0)) return;
    float mx = 0.f;
    for (int g = threadIdx.x; g < b.G; g += 256) {
        float n = 0.f;
        for (int d = 0; d < b.D; ++d) {
            const float c = (float)(b.means[(size_t)g * b.D + d] * (double)b.sw[d]);
            n = fmaf(c, c, n);
        }
        mx = fmaxf(mx, n);
    }
    s_m[threadIdx.x] = mx;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s_m[threadIdx.x] = fmaxf(s_m[threadIdx.x], s_m[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *b.nmax = s_m[0];
        *b.defer_n = 0;
    }
}

// (best, runner-up, argmin) merge; the lower index wins an exact tie
struct Best2 {
    float b1, b2;
    int a1;
};
__device__ __forceinline__ Best2 best2_merge(Best2 p, Best2 q)
{
    if (q.b1 < p.b1 || (q.b1 == p.b1 && q.a1 < p.a1)) return Best2{q.b1, fminf(p.b1, q.b2), q.a1};
    return Best2{p.b1, fminf(p.b2, q.b1), p.a1};
}

__host__ __device__ inline size_t bkm_dist_smem(int D)
{
    return sizeof(float) * ((size_t)kBG * blk_xs(D) + blk_d8(D) + 2 * 128 * (size_t)blk_xs(D)) +
           sizeof(float4) * 4 * 128;
}

template <int RS>
__global__ void __launch_bounds__(kBThreads, 1) k_bkm_dist(BkmArgs b)
{
    constexpr int TS = 16 * RS;
    extern __shared__ __align__(16) float bsm[];
    if (blk_skip(b.status, 0)) return;
    const int D = b.D, D8 = blk_d8(D), XS = blk_xs(D), CS = XS;   // mean rows as sample rows
    const int gb = blockIdx.x % b.n_gb, chunk = blockIdx.x / b.n_gb, g0 = gb * kBG;
    float *ncs = bsm;                    // [64][CS] -cs (0 past D)
    float *swd = ncs + kBG * CS;         // [D8]
    float *xt = swd + D8;                // [2][TS][XS] scaled samples
    float4 *red = reinterpret_cast<float4 *>(xt + 2 * TS * XS);   // [4][TS]
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int sg = 8 * (w & 1) + (lane & 7), gg = 4 * (w >> 1) + (lane >> 3);
    for (int k = tid; k < kBG * D8; k += kBThreads) {
        const int g = k / D8, d = k - g * D8;
        ncs[g * CS + d] = (g0 + g < b.G && d < D) ? -(float)(b.means[(size_t)(g0 + g) * D + d] * (double)b.sw[d]) : 0.f;
    }
    for (int d = tid; d < D8; d += kBThreads) swd[d] = d < D ? b.sw[d] : 0.f;
    for (int k = tid; k < 2 * TS * (XS - D); k += kBThreads) {
        const int r = k / (XS - D);
        xt[r * XS + D + (k - r * (XS - D))] = 0.f;
    }
    const int64_t ntiles = (b.N + TS - 1) / TS;
    const int64_t t0 = ntiles * chunk / b.n_chunks, t1 = ntiles * (chunk + 1) / b.n_chunks;
    auto stage = [&](int64_t t, float *xb) {
        const int64_t i0 = t * TS;
        const int nv = (int)min((int64_t)TS, b.N - i0);
        if (b.x_v4) {
            const int q4 = D / 4;
            for (int k = tid; k < TS * q4; k += kBThreads) {
                const int r = k / q4, c = k - r * q4;
                if (r < nv) cp_async16(xb + r * XS + 4 * c, b.X + (i0 + r) * D + 4 * c);
                else *reinterpret_cast<float4 *>(xb + r * XS + 4 * c) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        } else {
            for (int k = tid; k < TS * D; k += kBThreads) {
                const int r = k / D, c = k - r * D;
                if (r < nv) cp_async4(xb + r * XS + c, b.X + (i0 + r) * D + c);
                else xb[r * XS + c] = 0.f;
            }
        }
    };
    __syncthreads();
    if (t0 < t1) stage(t0, xt);
    cp_commit();
    for (int64_t t = t0; t < t1; ++t) {
        const int bi = (int)((t - t0) & 1);
        float *xb = xt + bi * TS * XS;
        if (t + 1 < t1) stage(t + 1, xt + (1 - bi) * TS * XS);
        cp_commit();
        cp_wait<1>();
        __syncthreads();
        for (int k = tid; k < TS * D; k += kBThreads) {   // xs = x sqrt(w), in place
            const int r = k / D, d = k - r * D;
            xb[r * XS + d] *= swd[d];
        }
        __syncthreads();
        if (gb == 0) {   // |xs|^2 per sample for the near-tie bound (any order: the bound has a 4x margin)
            const int64_t i0 = t * TS;
            for (int r = w; r < TS; r += kBThreads / 32) {
                float v = 0.f;
                for (int d = lane; d < D8; d += 32) v = fmaf(xb[r * XS + d], xb[r * XS + d], v);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0 && i0 + r < b.N) b.snorm[i0 + r] = v;
            }
        }
        float2 acc[RS][4];
#pragma unroll
        for (int k = 0; k < RS; ++k)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[k][j] = make_float2(0.f, 0.f);
#pragma unroll 2
        for (int d4 = 0; d4 < D8 / 4; ++d4) {
            float4 xv[RS];
#pragma unroll
            for (int k = 0; k < RS; ++k) xv[k] = *reinterpret_cast<const float4 *>(xb + (sg + 16 * k) * XS + 4 * d4);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float4 c = *reinterpret_cast<const float4 *>(ncs + (gg + 16 * j) * CS + 4 * d4);
                const float2 ca = make_float2(c.x, c.y), cb = make_float2(c.z, c.w);
#pragma unroll
                for (int k = 0; k < RS; ++k) {
                    const float2 t01 = __fadd2_rn(make_float2(xv[k].x, xv[k].y), ca);
                    const float2 t23 = __fadd2_rn(make_float2(xv[k].z, xv[k].w), cb);
                    acc[k][j] = __ffma2_rn(t01, t01, acc[k][j]);
                    acc[k][j] = __ffma2_rn(t23, t23, acc[k][j]);
                }
            }
        }
        // per sample: best two over this thread's means (ascending), the
        // warp's four mean groups (lanes ^ 8, ^ 16), the four warp pairs
#pragma unroll
        for (int k = 0; k < RS; ++k) {
            Best2 p{INFINITY, INFINITY, 0};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int g = gg + 16 * j;
                if (g0 + g < b.G) p = best2_merge(p, Best2{acc[k][j].x + acc[k][j].y, INFINITY, g});
            }
#pragma unroll
            for (int o = 8; o <= 16; o <<= 1) {
                Best2 q{__shfl_xor_sync(0xffffffffu, p.b1, o), __shfl_xor_sync(0xffffffffu, p.b2, o),
                        __shfl_xor_sync(0xffffffffu, p.a1, o)};
                p = best2_merge(p, q);
            }
            if (lane < 8) red[(w >> 1) * TS + sg + 16 * k] = make_float4(p.b1, p.b2, __int_as_float(p.a1), 0.f);
        }
        __syncthreads();
        const int64_t i0 = t * TS;
        for (int s = tid; s < TS; s += kBThreads) {
            if (i0 + s < b.N) {
                const float4 r0 = red[s];
                Best2 p{r0.x, r0.y, __float_as_int(r0.z)};
#pragma unroll
                for (int q = 1; q < 4; ++q) {
                    const float4 rq = red[q * TS + s];
                    p = best2_merge(p, Best2{rq.x, rq.y, __float_as_int(rq.z)});
                }
                b.part[(size_t)gb * b.N + i0 + s] = make_float2(p.b1, p.b2);
                b.arg[(size_t)gb * b.N + i0 + s] = (uint8_t)p.a1;
            }
        }
    }
    cp_wait<0>();
}

__global__ void __launch_bounds__(128) k_bkm_combine(BkmArgs b)
{
    if (blk_skip(b.status, 0)) return;
    const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
    if (i >= b.N) return;
    Best2 p{INFINITY, INFINITY, 0};
    for (int q = 0; q < b.n_gb; ++q) {   // blocks in ascending order: lower index wins ties
        const float2 v = b.part[(size_t)q * b.N + i];
        p = best2_merge(p, Best2{v.x, v.y, q * kBG + b.arg[(size_t)q * b.N + i]});
    }
    const float norms = b.snorm[i] + *b.nmax;
    b.assign[i] = p.a1;
    // near tie: the FP64 re-decision runs in k_bkm_recheck, a warp per sample
    // (inline, one thread's FP64 pass over every mean held a whole wave of
    // blocks: 358 ms per c3 iteration for 0.06 % of the samples)
    if (b.G > 1 && !(p.b2 - km_err(p.b2, norms, b.D) > p.b1 + km_err(p.b1, norms, b.D)))
        b.defer[atomicAdd(b.defer_n, 1)] = (int32_t)i;
}

// FP64 re-decision of the deferred samples: the definition
// sum_d w_d (x_d - mu_gd)^2 in order d = 0..D-1 without fused operations
// (the thread-per-sample form's km_recheck_fp64), lanes over the means, the
// lowest index among equal values.
__global__ void __launch_bounds__(256) k_bkm_recheck(BkmArgs b)
{
    if (blk_skip(b.status, 0)) return;
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int n = *b.defer_n;
    for (int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < n; e += nw) {
        const int64_t i = b.defer[e];
        const float *x = b.X + i * b.D;
        double best = INFINITY;
        int a = 0x7fffffff;
        for (int g = lane; g < b.G; g += 32) {
            const double *mu = b.means + (size_t)g * b.D;
            double acc = 0.0;
            for (int d = 0; d < b.D; ++d) {
                const double t = __dsub_rn((double)x[d], mu[d]);
                acc = __dadd_rn(acc, __dmul_rn(b.w[d], __dmul_rn(t, t)));
            }
            if (acc < best) { best = acc; a = g; }   // ascending g: the lane's lowest index on ties
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oa = __shfl_xor_sync(0xffffffffu, a, o);
            if (ob < best || (ob == best && oa < a)) { best = ob; a = oa; }
        }
        if (lane == 0) b.assign[i] = a;
    }
}

__host__ __device__ inline size_t bkm_stats_smem(int D)
{
    return sizeof(float) * 2 * 64 * (size_t)blk_xs(D) + sizeof(int) * 2 * 64 + sizeof(float4) * 18 * kBThreads +
           sizeof(int) * (2 * 64 + 4);
}

__global__ void __launch_bounds__(kBThreads, 1) k_bkm_stats(BkmArgs b)
{
    constexpr int TS = 64, UPT = 8;   // samples per tile; units per thread at most (64 means x D8/4 <= 2048)
    extern __shared__ __align__(16) float bsm[];
    if (blk_skip(b.status, 0)) return;
    const int D = b.D, G = b.G, D8 = blk_d8(D), XS = blk_xs(D), S = 1 + 2 * D, NQ = D8 / 4;
    const int gb = blockIdx.x % b.n_gb, chunk = blockIdx.x / b.n_gb, g0 = gb * kBG;
    float *xt = bsm;                                                // [2][64][XS]
    int *asg = reinterpret_cast<int *>(xt + 2 * TS * XS);           // [2][64]
    float4 *macc = reinterpret_cast<float4 *>(asg + 2 * TS);        // [18][256] per-thread sums
    int *lst = reinterpret_cast<int *>(macc + 18 * kBThreads);       // [2][64] in-block samples of the tile, per warp
    int *wcnt = lst + 2 * TS;                                         // [2] their counts
    const int tid = threadIdx.x;
    const int nu = kBG * NQ;   // units (mean of the block, 4 dimensions)
    // this thread's units u = tid + 256 r: shifts mu_f (FP32 old means)
    float4 mu[UPT];
#pragma unroll
    for (int r = 0; r < UPT; ++r) {
        const int u = tid + kBThreads * r, gl = u / NQ, d = 4 * (u - gl * NQ), g = g0 + gl;
        const bool on = u < nu && g < G;
        mu[r] = make_float4(on && d < D ? (float)b.means[(size_t)g * D + d] : 0.f,
                            on && d + 1 < D ? (float)b.means[(size_t)g * D + d + 1] : 0.f,
                            on && d + 2 < D ? (float)b.means[(size_t)g * D + d + 2] : 0.f,
                            on && d + 3 < D ? (float)b.means[(size_t)g * D + d + 3] : 0.f);
    }
    for (int q = 0; q < 18; ++q) macc[q * kBThreads + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = tid; k < 2 * TS * (XS - D); k += kBThreads) {
        const int r = k / (XS - D);
        xt[r * XS + D + (k - r * (XS - D))] = 0.f;
    }
    double *P = b.partial + (size_t)chunk * G * S;
    int flushes = 0, since = 0;
    auto flush = [&]() {
#pragma unroll
        for (int r = 0; r < UPT; ++r) {
            const int u = tid + kBThreads * r, gl = u / NQ, q = u - gl * NQ, d = 4 * q, g = g0 + gl;
            if (u >= nu || g >= G) continue;
            const float4 s1 = macc[(2 * r) * kBThreads + tid], s2 = macc[(2 * r + 1) * kBThreads + tid];
            const float v1[4] = {s1.x, s1.y, s1.z, s1.w}, v2[4] = {s2.x, s2.y, s2.z, s2.w};
            double *row = P + (size_t)g * S;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (d + e >= D) continue;
                row[1 + d + e] = flushes ? row[1 + d + e] + (double)v1[e] : (double)v1[e];
                row[1 + D + d + e] = flushes ? row[1 + D + d + e] + (double)v2[e] : (double)v2[e];
            }
            macc[(2 * r) * kBThreads + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
            macc[(2 * r + 1) * kBThreads + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        // counts: unit r of a thread with q == 0 keeps its mean's count in
        // component r & 3 of slot 16 + (r >> 2)
#pragma unroll
        for (int r = 0; r < UPT; ++r) {
            const int u = tid + kBThreads * r, gl = u / NQ, q = u - gl * NQ, g = g0 + gl;
            if (u >= nu || g >= G || q != 0) continue;
            float4 &c4 = macc[(16 + (r >> 2)) * kBThreads + tid];
            const float c = (r & 3) == 0 ? c4.x : ((r & 3) == 1 ? c4.y : ((r & 3) == 2 ? c4.z : c4.w));
            double *row = P + (size_t)g * S;
            row[0] = flushes ? row[0] + (double)c : (double)c;
        }
        macc[16 * kBThreads + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
        macc[17 * kBThreads + tid] = make_float4(0.f, 0.f, 0.f, 0.f);
        ++flushes;
        since = 0;
    };
    const int64_t ntiles = (b.N + TS - 1) / TS;
    const int64_t t0 = ntiles * chunk / b.n_chunks, t1 = ntiles * (chunk + 1) / b.n_chunks;
    auto stage = [&](int64_t t, int bi) {
        float *xb = xt + bi * TS * XS;
        const int64_t i0 = t * TS;
        const int nv = (int)min((int64_t)TS, b.N - i0);
        if (b.x_v4) {
            const int q4 = D / 4;
            for (int k = tid; k < TS * q4; k += kBThreads) {
                const int r = k / q4, c = k - r * q4;
                if (r < nv) cp_async16(xb + r * XS + 4 * c, b.X + (i0 + r) * D + 4 * c);
                else *reinterpret_cast<float4 *>(xb + r * XS + 4 * c) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        } else {
            for (int k = tid; k < TS * D; k += kBThreads) {
                const int r = k / D, c = k - r * D;
                if (r < nv) cp_async4(xb + r * XS + c, b.X + (i0 + r) * D + c);
                else xb[r * XS + c] = 0.f;
            }
        }
        for (int s = tid; s < TS; s += kBThreads) asg[bi * TS + s] = s < nv ? b.assign[i0 + s] : -1;
    };
    __syncthreads();
    if (t0 < t1) stage(t0, 0);
    cp_commit();
    for (int64_t t = t0; t < t1; ++t) {
        const int bi = (int)((t - t0) & 1);
        const float *xb = xt + bi * TS * XS;
        const int *ab = asg + bi * TS;
        if (t + 1 < t1) stage(t + 1, 1 - bi);
        cp_commit();
        cp_wait<1>();
        __syncthreads();
        // the tile's samples assigned to this block's means, in sample order
        if (tid < TS) {   // warps 0 and 1: samples 0..31, 32..63
            const int gl = ab[tid] - g0;
            const bool in = ab[tid] >= 0 && gl >= 0 && gl < kBG;
            const unsigned bal = __ballot_sync(0xffffffffu, in);
            if ((tid & 31) == 0) wcnt[tid >> 5] = __popc(bal);
            if (in) lst[(tid >> 5) * TS + __popc(bal & ((1u << (tid & 31)) - 1u))] = tid;
        }
        __syncthreads();
        const int n0 = wcnt[0], n1 = wcnt[1];
#pragma unroll
        for (int r = 0; r < UPT; ++r) {
            const int u = tid + kBThreads * r;
            if (u >= nu) continue;
            const int gl = u / NQ, d = 4 * (u - gl * NQ), g = g0 + gl;
            float4 s1 = make_float4(0.f, 0.f, 0.f, 0.f), s2 = s1;
            float cnt = 0.f;
            for (int e = 0; e < n0 + n1; ++e) {
                const int s = e < n0 ? lst[e] : lst[TS + e - n0];
                if (ab[s] != g) continue;
                const float4 xv = *reinterpret_cast<const float4 *>(xb + s * XS + d);
                const float u0 = xv.x - mu[r].x, u1 = xv.y - mu[r].y, u2 = xv.z - mu[r].z, u3 = xv.w - mu[r].w;
                s1.x += u0; s1.y += u1; s1.z += u2; s1.w += u3;
                s2.x = fmaf(u0, u0, s2.x); s2.y = fmaf(u1, u1, s2.y); s2.z = fmaf(u2, u2, s2.z); s2.w = fmaf(u3, u3, s2.w);
                cnt += 1.f;
            }
            float4 &a1 = macc[(2 * r) * kBThreads + tid], &a2 = macc[(2 * r + 1) * kBThreads + tid];
            a1.x += s1.x; a1.y += s1.y; a1.z += s1.z; a1.w += s1.w;
            a2.x += s2.x; a2.y += s2.y; a2.z += s2.z; a2.w += s2.w;
            float4 &c4 = macc[(16 + (r >> 2)) * kBThreads + tid];
            if ((r & 3) == 0) c4.x += cnt;
            else if ((r & 3) == 1) c4.y += cnt;
            else if ((r & 3) == 2) c4.z += cnt;
            else c4.w += cnt;
        }
        if (++since == kBFlush) flush();
        __syncthreads();   // buffer bi is free
    }
    cp_wait<0>();
    flush();   // also writes the rows of a chunk with no tiles (zeros)
}

}  // namespace

bool em_blocked_supported(int32_t D, int32_t G)
{
    if (D < 1 || D > 128 || G < 1) return false;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return blk_smem(D, 128, false) + 4 * 128 * sizeof(float2) + 2 * 128 * 4 + 1024 <= (size_t)optin &&
           blk_smem(D, 64, true) + 1024 <= (size_t)optin;
}

int em_blocked_gblocks(int32_t G) { return (G + kBG - 1) / kBG; }

// Sample chunks: the fewest that make (chunks x Gaussian blocks) a whole
// number of waves of one CTA per SM (up to 4 waves), else one wave's worth.
int em_blocked_chunks(int32_t G, int sms)
{
    const int nb = em_blocked_gblocks(G);
    for (int m = 1; m <= 4; ++m)
        if ((m * sms) % nb == 0) return m * sms / nb;
    const int c = sms / nb;
    return c > 0 ? c : 1;
}

cudaError_t launch_em_blocked(const EmPassArgs &a, float *lse, float2 *part, int32_t n_chunks, cudaStream_t s,
                              const int64_t *n_dev)
{
    BlkArgs b{a, em_blocked_gblocks(a.G), n_chunks,
              (a.D % 4 == 0 && (reinterpret_cast<uintptr_t>(a.X) & 15u) == 0) ? 1 : 0, part, lse, nullptr, n_dev};
    const size_t sm1 = blk_smem(a.D, 128, false) + 4 * 128 * sizeof(float2) + 2 * 128 * 4;
    const size_t sm3 = blk_smem(a.D, 64, true);
    cudaError_t e = cudaFuncSetAttribute(k_blk_lse<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    if (e != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_blk_em, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3)) != cudaSuccess)
        return e;
    const int grid = b.n_gb * n_chunks;
    k_blk_lse<8><<<grid, kBThreads, sm1, s>>>(b);
    k_blk_combine<<<(int)((a.N + 127) / 128), 128, 0, s>>>(b);
    k_blk_em<<<grid, kBThreads, sm3, s>>>(b);
    count_launches(3);
    return cudaGetLastError();
}

size_t em_rec_ws_bytes(int64_t N, int32_t D, int32_t G)
{
    const size_t n = (size_t)N, nb = (size_t)em_blocked_gblocks(G), nblk = (n + 1023) / 1024;
    auto al = [](size_t x) { return (x + 255u) & ~(size_t)255u; };
    return al(nb * n) + al(2u * nb * n * kBRec) + al(4u * nb * n * kBRec) + al(n) + al(2u * n * kRecSlots) +
           al(4u * n * kRecSlots) + al(4u * nblk) + al(8u) + al(4u * n * (size_t)D) + al(4u * n) + al(8u * nb * n) + 256u;
}

RecWs em_rec_ws(void *base, int64_t N, int32_t D, int32_t G)
{
    const size_t n = (size_t)N, nb = (size_t)em_blocked_gblocks(G), nblk = (n + 1023) / 1024;
    auto al = [](size_t x) { return (x + 255u) & ~(size_t)255u; };
    unsigned char *p = static_cast<unsigned char *>(base);
    RecWs w;
    w.rec_n = p;                                   p += al(nb * n);
    w.rec_g = reinterpret_cast<uint16_t *>(p);     p += al(2u * nb * n * kBRec);
    w.rec_l = reinterpret_cast<float *>(p);        p += al(4u * nb * n * kBRec);
    w.rc = p;                                      p += al(n);
    w.rg = reinterpret_cast<uint16_t *>(p);        p += al(2u * n * kRecSlots);
    w.rgam = reinterpret_cast<float *>(p);         p += al(4u * n * kRecSlots);
    w.bcnt = reinterpret_cast<int32_t *>(p);       p += al(4u * nblk);
    w.n_mark = reinterpret_cast<int64_t *>(p);     p += al(8u);
    w.Xd = reinterpret_cast<float *>(p);           p += al(4u * n * (size_t)D);
    w.lse_d = reinterpret_cast<float *>(p);        p += al(4u * n);
    w.part_d = reinterpret_cast<float2 *>(p);
    return w;
}

int em_rec_partials(int64_t N, int32_t G, int sms) { return record_mstep_chunks(N, G, sms) + em_blocked_chunks(G, sms); }

cudaError_t launch_em_blocked_rec(const EmPassArgs &a, float *lse, float2 *part, const RecWs &ws, int sms, cudaStream_t s)
{
    const int nch = em_blocked_chunks(a.G, sms), n_gb = em_blocked_gblocks(a.G);
    const float scr = (float)std::log((double)(a.N_total > a.N ? a.N_total : a.N) * 1e9);
    BlkArgs b{a, n_gb, nch, (a.D % 4 == 0 && (reinterpret_cast<uintptr_t>(a.X) & 15u) == 0) ? 1 : 0, part, lse, nullptr,
              nullptr, ws.rec_n, ws.rec_g, ws.rec_l, scr, ws.rc, ws.rg, ws.rgam};
    const size_t sm1 = blk_smem(a.D, 128, false) + 4 * 128 * sizeof(float2) + 2 * 128 * 4;
    const size_t sm3 = blk_smem(a.D, 64, true);
    cudaError_t e = cudaFuncSetAttribute(k_blk_lse<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    if (e != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_blk_em, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3)) != cudaSuccess)
        return e;
    // log-sum-exp partials and the candidates per block; log p, the
    // log-likelihood and the kept responsibilities per sample
    k_blk_lse<8><<<n_gb * nch, kBThreads, sm1, s>>>(b);
    k_blk_combine<<<(int)((a.N + 127) / 128), 128, 0, s>>>(b);
    count_launches(2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // samples whose records overflowed, gathered with their log p
    if ((e = launch_gather_marked(ws.rc, a.X, lse, a.N, a.D, ws.bcnt, ws.n_mark, ws.Xd, ws.lse_d, s)) != cudaSuccess)
        return e;
    // statistics from the records, then those samples' from their recomputed
    // responsibilities (partials after the records')
    if ((e = launch_record_mstep(a, ws.rc, ws.rg, ws.rgam, sms, s)) != cudaSuccess) return e;
    EmPassArgs d = a;
    d.X = ws.Xd;
    d.partial = a.partial + (size_t)record_mstep_chunks(a.N, a.G, sms) * a.G * (1 + 2 * a.D);
    BlkArgs bd{d, n_gb, nch, a.D % 4 == 0 ? 1 : 0, ws.part_d, ws.lse_d, nullptr, ws.n_mark};
    k_blk_em<<<n_gb * nch, kBThreads, sm3, s>>>(bd);
    count_launches(1);
    return cudaGetLastError();
}

bool km_blocked_supported(int32_t D, int32_t G)
{
    if (D < 1 || D > 128 || G < 1) return false;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return bkm_dist_smem(D) + 1024 <= (size_t)optin && bkm_stats_smem(D) + 1024 <= (size_t)optin;
}

cudaError_t launch_km_blocked(const float *X, int64_t N, int32_t D, int32_t G, const double *means,
                              const double *w, const float *sw, float2 *part, uint8_t *arg, float *nmax,
                              float *snorm, int32_t *defer, int32_t *assign, double *partial, int32_t n_chunks,
                              const DevStatus *status, cudaStream_t s)
{
    BkmArgs b{X, N, D, G, means, w, sw, part, arg, nmax, snorm, defer, defer + N, assign, partial, em_blocked_gblocks(G),
              n_chunks,
              (D % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0) ? 1 : 0, status};
    const size_t smd = bkm_dist_smem(D), sms = bkm_stats_smem(D);
    cudaError_t e = cudaFuncSetAttribute(k_bkm_dist<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smd);
    if (e != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_bkm_stats, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sms)) != cudaSuccess)
        return e;
    const int grid = b.n_gb * n_chunks;
    k_bkm_norms<<<1, 256, 0, s>>>(b);
    k_bkm_dist<8><<<grid, kBThreads, smd, s>>>(b);
    k_bkm_combine<<<(int)((N + 127) / 128), 128, 0, s>>>(b);
    k_bkm_recheck<<<grid, 256, 0, s>>>(b);
    k_bkm_stats<<<grid, kBThreads, sms, s>>>(b);
    count_launches(5);
    return cudaGetLastError();
}

// Inference: log p(x_i) of the mixture (Sec. 4.1 log_p) by the phase-1
// kernels: partial log-sum-exps per block of 64 Gaussians, merged in FP64.
cudaError_t launch_log_p_blocked(const float *X, int64_t N, int32_t D, int32_t G, Operands op, double *out,
                                 float2 *part, int sms, cudaStream_t s)
{
    EmPassArgs a{};
    a.X = X;
    a.N = N;
    a.D = D;
    a.G = G;
    a.op = op;
    a.N_total = N;
    const int n_chunks = em_blocked_chunks(G, sms);
    BlkArgs b{a, em_blocked_gblocks(G), n_chunks, (D % 4 == 0 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0) ? 1 : 0,
              part, nullptr, out};
    const size_t sm1 = blk_smem(D, 128, false) + 4 * 128 * sizeof(float2) + 2 * 128 * 4;
    cudaError_t e = cudaFuncSetAttribute(k_blk_lse<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1);
    if (e != cudaSuccess) return e;
    k_blk_lse<8><<<b.n_gb * n_chunks, kBThreads, sm1, s>>>(b);
    k_blk_combine<<<(int)((N + 127) / 128), 128, 0, s>>>(b);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace gmm
