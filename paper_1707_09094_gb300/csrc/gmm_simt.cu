// CUDA-core kernels of the library: global statistics, k-means assignment +
// accumulation, the plain FP32 fused EM pass, the FP64 reduce/update
// ("finalize") kernels, operand preparation and inference.
//
// Data layout in HBM (row-major):
//   X        float [N][D]
//   lambda   double [G*D means | G*D dcovs | G hefts]   (ping-pong pair)
//   partial  double [n_partial][G][1 + 2D]: per-CTA map results of Sec. 2.1
//            (index 0 = L~_g, 1..D = sum l (x - shift), D+1..2D = sum l (x - shift)^2)
// Every reduction over CTAs runs in CTA order in FP64, so results do not
// depend on scheduling.
#include <atomic>
#include <mutex>
#include <cfloat>
#include <cmath>

#include "gmm_internal.cuh"
#include "gmm_km_exact.cuh"

namespace gmm {

namespace {

#ifndef GMM_EM_WARPS
#define GMM_EM_WARPS 16
#endif
constexpr int kWarps = GMM_EM_WARPS;   // warps of a CTA of the FP32 EM passes
constexpr int kEmThreads = kWarps * 32;
#ifndef GMM_EM_GSTEP
#define GMM_EM_GSTEP 4
#endif
constexpr int kEmGs = GMM_EM_GSTEP;   // Gaussians per warp step of the FP32 E-step
constexpr int kTile = 32;      // samples per tile of the FP32 EM pass
constexpr int kTP = kTile + 1; // padded row stride of the tile buffers
constexpr int kKmThreads = 128;

// Whether this block must skip its work: one thread reads the status block
// and shares the answer, so that every thread of the block agrees even if
// another block raises the halt flag meanwhile.
__device__ __forceinline__ bool block_skip(const DevStatus *st, int iter)
{
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = (st->halt != 0 || iter > st->stop_after) ? 1 : 0;
    __syncthreads();
    return s_skip != 0;
}

__device__ __forceinline__ float warp_max(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ float warp_sum(float v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Fixed-order block reduction of one double per thread (thread 0 returns it).
__device__ double block_sum_d(double v, double *sh)
{
    int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
        if (t < s) sh[t] += sh[t + s];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

__device__ void set_error(DevStatus *st, int code, int iter)
{
    if (atomicCAS(&st->code, 0, code) == 0) st->fail_iter = iter;
    atomicExch(&st->halt, 1);
}

// p[0] + p[stride] + ... + p[(n-1) stride], added in that order, with eight
// loads in flight at a time
__device__ __forceinline__ double sum_in_order(const double *__restrict__ p, int n, size_t stride)
{
    double s = 0.0;
    int c = 0;
    for (; c + 8 <= n; c += 8) {
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = p[(size_t)(c + u) * stride];
#pragma unroll
        for (int u = 0; u < 8; ++u) s += v[u];
    }
    for (; c < n; ++c) s += p[(size_t)c * stride];
    return s;
}

// ------------------------------------------------------------------------
// Global per-dimension mean and variance (Eq. 20's global covariance).
// Pass 1 sums x, pass 2 sums (x - mean)^2.  Each thread keeps an unevaluated
// float-float sum (hi + lo, about 44 significant bits: Knuth's error-free
// two-sum with renormalisation), so the pass runs on the FP32 pipes at HBM
// speed; the per-thread sums are combined in FP64 per CTA, then in CTA
// order.  blockDim = R*D: thread (r, d) walks rows r, r+R*grid, ... of
// column d.
// ------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// (hi, lo) += (v, ve), renormalised so that |lo| <= ulp(hi) / 2
__device__ __forceinline__ void ff_add(float &hi, float &lo, float v, float ve)
{
    float s, e;
    two_sum(hi, v, s, e);
    e = __fadd_rn(e, __fadd_rn(lo, ve));
    hi = __fadd_rn(s, e);
    lo = __fsub_rn(e, __fsub_rn(hi, s));
}

template <int PASS>
__global__ void k_gstats(const float *__restrict__ X, int64_t N, int32_t D,
                         const double *__restrict__ gmean, double *__restrict__ partial)
{
    extern __shared__ double shd[];
    const int R = blockDim.x / D;
    const int t = threadIdx.x;
    float hi = 0.f, lo = 0.f;
    if (t < R * D) {
        const int d = t % D, r = t / D;
        const double m = PASS == 2 ? gmean[d] : 0.0;
        const float mh = (float)m, ml = (float)(m - (double)mh);   // m = mh + ml to ~2^-48
        for (int64_t i = (int64_t)blockIdx.x * R + r; i < N; i += (int64_t)gridDim.x * R) {
            const float v = X[i * D + d];
            if (PASS == 1) {
                ff_add(hi, lo, v, 0.f);
            } else {
                float q, qe;
                two_sum(v, -mh, q, qe);          // v - mh exactly
                qe = __fsub_rn(qe, ml);          // (q, qe) = v - m
                const float p = __fmul_rn(q, q);
                float pe = __fmaf_rn(q, q, -p);  // q*q - p exactly
                pe = __fmaf_rn(__fadd_rn(q, q), qe, pe);
                ff_add(hi, lo, p, pe);
            }
        }
    }
    shd[t] = (double)hi + (double)lo;
    __syncthreads();
    if (t < D) {
        double s = 0.0;
        for (int r = 0; r < R; ++r) s += shd[r * D + t];
        partial[(size_t)blockIdx.x * D + t] = s;
    }
}

template <int PASS>
__global__ void __launch_bounds__(128) k_gstats_final(const double *__restrict__ partial, int n_partial, int64_t N,
                                                      int32_t D, double var_floor, int32_t dist, double *gmean,
                                                      double *gvar_floored, double *wdist, float *sw, float *center)
{
    // one block per dimension: strided partial sums, then a fixed-order tree
    __shared__ double red[128];
    const int d = blockIdx.x, t = threadIdx.x;
    double s = 0.0;
    for (int c = t; c < n_partial; c += 128) s += partial[(size_t)c * D + d];
    red[t] = s;
    __syncthreads();
    for (int w = 64; w > 0; w >>= 1) {
        if (t < w) red[t] += red[t + w];
        __syncthreads();
    }
    if (t != 0) return;
    s = red[0];
    if (PASS == 1) {
        gmean[d] = s / (double)N;
        center[d] = (float)(s / (double)N);
    } else {
        double v = s / (double)N;
        v = v > var_floor ? v : var_floor;
        gvar_floored[d] = v;
        double w = dist == GMM_MAHA ? 1.0 / v : 1.0;
        wdist[d] = w;
        sw[d] = (float)sqrt(w);
    }
}

__global__ void k_gather_seeds(const float *__restrict__ X, int32_t D, int32_t G,
                               const int64_t *__restrict__ idx, double *par)
{
    int g = blockIdx.x;
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
        par[(size_t)g * D + d] = (double)X[idx[g] * D + d];
        par[(size_t)G * D + (size_t)g * D + d] = 1.0;
    }
    if (threadIdx.x == 0) par[2 * (size_t)G * D + g] = 1.0 / (double)G;
}

struct KmArgs {
    const float *X;
    int64_t N;
    int32_t D, DP, G, GS;
    const double *means;   // lambda (means at the start of the iteration)
    const double *w;       // [D] FP64 distance weights
    const float *sw;       // [D] FP32 sqrt(w)
    double *partial;       // [grid][G][1+2D] FP64 per-CTA statistics (output)
    int32_t *assign;
    const DevStatus *status;
};

// Tiled form of the k-means map step for D <= 64, N_G <= 256 (one CTA per
// SM, its contiguous chunk of samples).  With scaled coordinates
// xs = x sqrt(w), cs = mu sqrt(w) the nearest mean minimises the expanded
// score s_g = |cs_g|^2 - 2 xs.cs_g (the distance minus the common |xs|^2):
// one FMA per (sample, mean, dimension).  Shared memory holds the scaled
// means with an odd row stride, their squared norms, the chunk's FP32
// statistics [G][1 + 2D] (count, sum(x - mu_f), sum((x - mu_f)^2), shifted
// by the FP32 old mean mu_f) and a 128-sample tile of scaled rows.  Warp w
// takes samples 8w..8w+7 of the tile, lane l the means l, l+32, ...: 64
// scores per thread in registers.
// Rounding bound of a computed score (xs, cs each within 3u of the exact
// scaled values, u = 2^-24; FMA accumulation over D terms; the final
// subtraction): |s~ - s| <= (D + 8) u (|cs|^2 + 2 |xs| |cs|) to first order,
// taken here with a factor 2 and the largest |cs|^2 of all means.  If the
// runner-up minus the winner exceeds twice that bound the FP32 winner is the
// exact winner; otherwise the means whose score is within twice the bound of
// the best (no other mean can win) are re-decided in FP64, each on its own
// lane, as sum_d w_d (x_d - mu_d)^2 in order d = 0..D-1 without fused
// operations, lowest index on exact ties (the oracle's definition).  The
// statistics go to shared memory with atomics (one mean per sample), and
// the chunk's FP32 statistics to its FP64 partial at the end.
constexpr int kKmTileThreads = 512;
constexpr int kKmTileS = 128;   // samples per tile: 16 warps x 8

__host__ __device__ inline int km_tile_cs(int D) { return D | 1; }

__host__ __device__ inline size_t km_tile_smem(int D, int G)
{
    const size_t cs = (size_t)km_tile_cs(D);
    return sizeof(float) * ((size_t)G * cs + (size_t)G + (size_t)G * (1 + 2 * D) + (size_t)kKmTileS * 64u + 64u) + 64u;
}

template <int NJ>   // means per lane: ceil(N_G / 32) rounded up to a power of two
__global__ void __launch_bounds__(kKmTileThreads, 1) k_km_tile(KmArgs a)
{
    extern __shared__ __align__(16) unsigned char kmt_smem[];
    if (block_skip(a.status, 0)) return;
    const int D = a.D, G = a.G, CS = km_tile_cs(D), S = 1 + 2 * D;
    float *cent = reinterpret_cast<float *>(kmt_smem);        // [G][CS]
    float *cnorm = cent + (size_t)G * CS;                       // [G]
    float *slab = cnorm + G;                                    // [G][S]
    float *xsc = slab + (size_t)G * S;                          // [128][64] scaled rows
    float *swd = xsc + kKmTileS * 64;                           // [64] sqrt(w)
    __shared__ float s_nmax;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int d = tid; d < 64; d += kKmTileThreads) swd[d] = d < D ? a.sw[d] : 0.f;
    for (int k = tid; k < G * S; k += kKmTileThreads) slab[k] = 0.f;
    if (tid == 0) s_nmax = 0.f;
    __syncthreads();
    for (int k = tid; k < G * D; k += kKmTileThreads) {
        const int g = k / D, d = k - g * D;
        cent[g * CS + d] = (float)(a.means[k] * (double)swd[d]);
    }
    __syncthreads();
    for (int g = tid; g < G; g += kKmTileThreads) {
        float n = 0.f;
        for (int d = 0; d < D; ++d) n = fmaf(cent[g * CS + d], cent[g * CS + d], n);
        cnorm[g] = n;
        atomicMax(reinterpret_cast<int *>(&s_nmax), __float_as_int(n));   // n >= 0
    }
    __syncthreads();
    const float nmax = s_nmax;
    const float kE = 2.0f * (float)(D + 8) * 5.9604644775390625e-08f;
    const int64_t i0 = a.N * blockIdx.x / gridDim.x, i1 = a.N * (blockIdx.x + 1) / gridDim.x;
    float cn[NJ];
    int ro[NJ];   // row offsets; lanes past the last mean read its row (their score is +inf)
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        const int g = lane + 32 * j;
        cn[j] = g < G ? cnorm[g] : INFINITY;
        ro[j] = min(g, G - 1) * CS;
    }
    for (int64_t base = i0; base < i1; base += kKmTileS) {
        const int nv = (int)min((int64_t)kKmTileS, i1 - base);
        for (int k = tid; k < nv * D; k += kKmTileThreads) {
            const int r = k / D, d = k - r * D;
            xsc[r * 64 + d] = __ldg(a.X + base * D + k) * swd[d];
        }
        __syncthreads();
        const int sb = 8 * warp;
        if (sb < nv) {
            float acc[8][NJ];
#pragma unroll
            for (int k = 0; k < 8; ++k)
#pragma unroll
                for (int j = 0; j < NJ; ++j) acc[k][j] = 0.f;
            const float *xrow = xsc + sb * 64;
#pragma unroll 2
            for (int d = 0; d < D; ++d) {
                float xv[8], c[NJ];
#pragma unroll
                for (int k = 0; k < 8; ++k) xv[k] = xrow[k * 64 + d];
#pragma unroll
                for (int j = 0; j < NJ; ++j) c[j] = cent[ro[j] + d];
#pragma unroll
                for (int k = 0; k < 8; ++k)
#pragma unroll
                    for (int j = 0; j < NJ; ++j) acc[k][j] = fmaf(xv[k], c[j], acc[k][j]);
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int si = sb + k;   // warp-uniform
                float b1 = INFINITY, b2 = INFINITY;
                int a1 = 0x7fffffff;
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    const float v = fmaf(-2.f, acc[k][j], cn[j]);
                    const int g = lane + 32 * j;
                    if (v < b1) { b2 = b1; b1 = v; a1 = g; }
                    else if (v < b2) { b2 = v; }
                }
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
                if (si >= nv) continue;
                float sn = 0.f;
                for (int d = lane; d < D; d += 32) sn = fmaf(xrow[k * 64 + d], xrow[k * 64 + d], sn);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sn += __shfl_xor_sync(0xffffffffu, sn, o);
                const float E = kE * (nmax + 2.f * sqrtf(sn * nmax)) + 1e-30f;
                const int64_t i = base + si;
                const float *x = a.X + i * D;
                int best = a1;
                if (G > 1 && !(b2 - b1 > 2.f * E)) {
                    // FP64 re-decision among the means whose score is within 2E
                    // of the best (every other mean is provably farther), each on
                    // its own lane in the oracle's operation order
                    double bv = INFINITY;
                    int bi = 0x7fffffff;
                    const float lim = b1 + 2.f * E;
#pragma unroll
                    for (int j = 0; j < NJ; ++j) {
                        const int g = lane + 32 * j;
                        if (g < G && fmaf(-2.f, acc[k][j], cn[j]) <= lim) {
                            const double *mu = a.means + (size_t)g * D;
                            double accd = 0.0;
                            for (int d = 0; d < D; ++d) {
                                const double t = __dsub_rn((double)__ldg(x + d), mu[d]);
                                accd = __dadd_rn(accd, __dmul_rn(a.w[d], __dmul_rn(t, t)));
                            }
                            if (accd < bv || (accd == bv && g < bi)) { bv = accd; bi = g; }
                        }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                        if (ov < bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
                    }
                    best = bi;
                }
                if (lane == 0) a.assign[i] = best;
                // statistics of the mean this sample joins
                float *sg = slab + (size_t)best * S;
                const double *mu = a.means + (size_t)best * D;
                for (int d = lane; d < D; d += 32) {
                    const float u = __ldg(x + d) - (float)mu[d];
                    atomicAdd(sg + 1 + d, u);
                    atomicAdd(sg + 1 + D + d, u * u);
                }
                if (lane == 0) atomicAdd(sg, 1.f);
            }
        }
        __syncthreads();   // the tile buffer is reused
    }
    double *P = a.partial + (size_t)blockIdx.x * G * S;
    for (int k = tid; k < G * S; k += kKmTileThreads) P[k] = (double)slab[k];
}

// k-means reduce + update (Sec. 3 (ii); Eqs. 5-7 with Eq. 19 for the last
// iteration).  One block per Gaussian, partials summed in CTA order.
__global__ void k_km_finalize(const double *__restrict__ partial, int n_partial, int64_t N, int32_t D,
                              int32_t G, double *par, double var_floor, int32_t final_iter,
                              double *counts, const DevStatus *status)
{
    if (block_skip(status, 0)) return;
    extern __shared__ double red[];   // [1+2D]
    const int g = blockIdx.x, S = 1 + 2 * D;
    for (int j = threadIdx.x; j < S; j += blockDim.x) red[j] = sum_in_order(partial + (size_t)g * S + j, n_partial, (size_t)G * S);
    __syncthreads();
    const double cnt = red[0];
    if (threadIdx.x == 0) counts[g] = cnt;
    if (cnt > 0.0) {
        double *means = par, *dcovs = par + (size_t)G * D, *hefts = par + 2 * (size_t)G * D;
        for (int d = threadIdx.x; d < D; d += blockDim.x) {
            const double shift = (double)(float)means[(size_t)g * D + d];
            const double m1 = red[1 + d] / cnt;
            if (final_iter) {
                double v = red[1 + D + d] / cnt - m1 * m1;
                dcovs[(size_t)g * D + d] = v > var_floor ? v : var_floor;
            }
            means[(size_t)g * D + d] = shift + m1;
        }
        if (final_iter && threadIdx.x == 0) hefts[g] = cnt / (double)N;
    }
}


// Dead-mean resurrection (Sec. 3.1), reading documented in the oracle: the
// most popular mean (largest count, lowest index) gives its lowest-index
// samples, in increasing order, to the dead means in increasing index order
// (cycling when there are more dead means than such samples).  Last
// iteration: a dead mean gets the floored global variance and heft 1/N, and
// the hefts are renormalised.  One block of 1024 threads.
__global__ void __launch_bounds__(1024) k_km_dead_fix(const float *__restrict__ X,
                                                      const int32_t *__restrict__ assign, int64_t N,
                                                      int32_t D, int32_t G, double *par,
                                                      const double *__restrict__ counts,
                                                      const double *__restrict__ gvar_floored,
                                                      int32_t final_iter, DevStatus *status)
{
    extern __shared__ int64_t members[];   // [G]
    __shared__ int s_pop, s_ndead, s_found;
    __shared__ int s_warp[32];
    if (block_skip(status, 0)) return;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // most populous mean (lowest index among equal counts) and dead means, block-wide
    {
        double best = -1.0;
        int pop = 0x7fffffff, nd = 0;
        for (int g = tid; g < G; g += blockDim.x) {
            const double c = counts[g];
            if (c > best) { best = c; pop = g; }   // ascending g: the first of equal counts
            nd += !(c > 0.0);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int op = __shfl_xor_sync(0xffffffffu, pop, o);
            if (ob > best || (ob == best && op < pop)) { best = ob; pop = op; }
            nd += __shfl_xor_sync(0xffffffffu, nd, o);
        }
        __shared__ double s_best[32];
        __shared__ int s_popw[32], s_ndw[32];
        if (lane == 0) { s_best[wid] = best; s_popw[wid] = pop; s_ndw[wid] = nd; }
        __syncthreads();
        if (tid == 0) {
            double b = -1.0;
            int p = 0x7fffffff, n = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                if (s_best[w] > b || (s_best[w] == b && s_popw[w] < p)) { b = s_best[w]; p = s_popw[w]; }
                n += s_ndw[w];
            }
            s_pop = p == 0x7fffffff ? 0 : p; s_ndead = n; s_found = 0;
            status->n_dead = n;
        }
        __syncthreads();
    }
    const int nd = s_ndead;
    if (nd == 0) return;
    const int pop = s_pop;
    const int64_t n_pop = (int64_t)counts[pop];
    int need = (int)min((int64_t)nd, n_pop);
    // ordered scan of the assignments for the popular mean's first `need` samples
    for (int64_t base = 0; base < N; base += blockDim.x) {
        if (s_found >= need) break;
        const int64_t i = base + tid;
        const int f = (i < N && assign[i] == pop) ? 1 : 0;
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) s_warp[wid] = __popc(bal);
        __syncthreads();
        int off = 0, tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { if (w < wid) off += s_warp[w]; tot += s_warp[w]; }
        const int pos = s_found + off + __popc(bal & ((1u << lane) - 1u));
        if (f && pos < need) members[pos] = i;
        __syncthreads();
        if (tid == 0) s_found += tot;
        __syncthreads();
    }
    if (s_found < need) need = s_found;   // counts and assignments disagree: use what was found
    if (need < 1) return;
    double *means = par, *dcovs = par + (size_t)G * D, *hefts = par + 2 * (size_t)G * D;
    int j = 0;
    for (int g = 0; g < G; ++g) {
        if (counts[g] > 0.0) continue;
        const int64_t s = members[j % need];
        ++j;
        for (int d = tid; d < D; d += blockDim.x) {
            means[(size_t)g * D + d] = (double)X[s * D + d];
            if (final_iter) dcovs[(size_t)g * D + d] = gvar_floored[d];
        }
        if (final_iter && tid == 0) hefts[g] = 1.0 / (double)N;
    }
    if (final_iter) {
        __syncthreads();
        __shared__ double s_hsum;
        if (tid == 0) {
            double h = 0.0;
            for (int g = 0; g < G; ++g) h += hefts[g];
            s_hsum = h;
        }
        __syncthreads();
        for (int g = tid; g < G; g += blockDim.x) hefts[g] /= s_hsum;
    }
}

// ------------------------------------------------------------------------
// Operands of the E-step from lambda (Eq. 15 with a diagonal covariance):
//   FP32 form   l_g(x) = c_g - 1/2 sum_d (x_d s_gd - mu_gd s_gd)^2,
//               s = 1/sigma, c_g = log w_g - D/2 log 2pi - 1/2 sum_d log sigma^2_gd
//   tensor form the same expanded about the global centre m (x' = x - m,
//               mu' = mu - m): l_g = ctc_g + P1 + P2 with
//               P1 = sum_d x'^2 (-1/2 iv_gd), P2 = sum_d x' (mu'_gd iv_gd),
//               ctc_g = c_g - 1/2 q_g, q_g = sum_d mu'^2 iv; packed K-major
//               [G][128] BF16: columns 0..63 hold -1/2 iv (the x'^2 block),
//               64..127 hold mu' iv (the x' block), zero padded (D <= 64).
// One block per Gaussian; called by k_em_prep and by k_em_finalize.
// ------------------------------------------------------------------------
__device__ void prep_operands(int g, int D, int G, const double *mu, const double *var, double w,
                              const Operands &op, const float *center, int build_tc, double *sh)
{
    double lsum = 0.0, qsum = 0.0;
    build_tc = build_tc && D <= 64;
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
        const double v = var[d], m = mu[d];
        const double s = 1.0 / sqrt(v);
        op.sm[(size_t)g * D + d] = make_float2((float)s, (float)(m * s));
        op.mu[(size_t)g * D + d] = (float)m;
        lsum += log(v);
        if (build_tc) {
            const double iv = 1.0 / v;
            const double mc = m - (double)center[d];
            qsum += mc * mc * iv;
            op.B[(size_t)g * 128 + d] = __float2bfloat16_rn((float)(-0.5 * iv));
            op.B[(size_t)g * 128 + 64 + d] = __float2bfloat16_rn((float)(mc * iv));
        }
    }
    if (build_tc)
        for (int k = threadIdx.x; k < 128; k += blockDim.x)
            if ((k & 63) >= D) op.B[(size_t)g * 128 + k] = __float2bfloat16_rn(0.f);
    lsum = block_sum_d(lsum, sh);
    qsum = block_sum_d(qsum, sh);
    if (threadIdx.x == 0) {
        const double c0 = -0.5 * (double)D * kLog2Pi - 0.5 * lsum;
        const double lw = log(w);
        op.c[g] = (float)(lw + c0);
        op.c0[g] = (float)c0;
        if (build_tc) {
            op.ctc[g] = (float)(lw + c0 - 0.5 * qsum);
            op.q[g] = (float)qsum;
        }
    }
}

__global__ void k_em_prep(int32_t D, int32_t G, const double *__restrict__ par, Operands op,
                          const float *__restrict__ center, int32_t build_tc)
{
    __shared__ double sh[128];
    const int g = blockIdx.x;
    prep_operands(g, D, G, par + (size_t)g * D, par + (size_t)G * D + (size_t)g * D,
                  par[2 * (size_t)G * D + g], op, center, build_tc, sh);
}

// ------------------------------------------------------------------------
// Plain FP32 fused EM pass (the CUDA-core form): per 32-sample tile
//   E  logits l_g(x_i) for every Gaussian (warp w: Gaussians g = w mod 8,
//      lane = sample), into shared memory only;
//   LSE warp-shuffle log-sum-exp per sample (Eqs. 16-18: max + sum of exp),
//      log p(x_i) added to the CTA's FP64 log-likelihood, responsibilities
//      l_{g,i} = exp(l_g - log p) (Eq. 3) written over the logits;
//   M  thread-owned (g, d) pairs accumulate sum l (x - mu_f) and
//      sum l (x - mu_f)^2 (Eqs. 9-11 shifted by the FP32 mean mu_f of the
//      iteration start, which keeps FP32 sums small); FP32 in shared memory
//      for the CTA's chunk, flushed once to the FP64 partial of the CTA.
// Each CTA owns one contiguous chunk of tiles: the paper's thread t.
// ------------------------------------------------------------------------
template <int DMAX>
__global__ void __launch_bounds__(kEmThreads, 1) k_em_pass_simt(EmPassArgs a)
{
    extern __shared__ __align__(16) float em_smem[];
    if (block_skip(a.status, a.iter)) return;
    const int D = a.D, G = a.G;
    float *xT = em_smem;                          // [D][kTP]
    float *L = xT + (size_t)D * kTP;              // [G][kTP]
    float *S0 = L + (size_t)G * kTP;              // [G]
    float *S1 = S0 + G;                           // [G*D]
    float *S2 = S1 + (size_t)G * D;               // [G*D]
    int *act = reinterpret_cast<int *>(S2 + (size_t)G * D);   // [G] Gaussians that matter in the tile
    __shared__ double s_ll[kWarps];
    __shared__ int s_nact;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    // responsibilities below 1e-9 / N (the tensor-core form's rule) carry less
    // than 1e-9 per Gaussian in total: a Gaussian none of whose tile
    // responsibilities reaches it is left out of the tile's M-step
    const float keep = (float)(1e-9 / (double)(a.N_total > a.N ? a.N_total : a.N));

    for (int k = tid; k < G; k += kEmThreads) S0[k] = 0.f;
    for (int k = tid; k < G * D; k += kEmThreads) { S1[k] = 0.f; S2[k] = 0.f; }

    const int64_t ntiles = (a.N + kTile - 1) / kTile;
    const int64_t t0 = ntiles * blockIdx.x / gridDim.x, t1 = ntiles * (blockIdx.x + 1) / gridDim.x;
    double ll = 0.0;
    for (int64_t tile = t0; tile < t1; ++tile) {
        const int64_t i0 = tile * kTile;
        const int n = (int)min((int64_t)kTile, a.N - i0);
        __syncthreads();
        const float *Xt = a.X + i0 * D;
        for (int k = tid; k < kTile * D; k += kEmThreads) {
            const int i = k / D, d = k - i * D;
            xT[d * kTP + i] = i < n ? Xt[k] : 0.f;
        }
        __syncthreads();
        // ---- E: logits
        {
            float xr[DMAX];
#pragma unroll
            for (int d = 0; d < DMAX; ++d) xr[d] = d < D ? xT[d * kTP + lane] : 0.f;
            // kEmGs Gaussians per step, two dimensions per 128-bit operand load
            // (even D): 2 kEmGs independent FMA chains per thread
            for (int g0 = w; g0 < G; g0 += kEmGs * kWarps) {
                float acc[kEmGs], acc2[kEmGs];
#pragma unroll
                for (int u = 0; u < kEmGs; ++u) { acc[u] = 0.f; acc2[u] = 0.f; }
                if ((D & 1) == 0) {
#pragma unroll
                    for (int d = 0; d < DMAX; d += 2) {
                        if (d < D) {
#pragma unroll
                            for (int u = 0; u < kEmGs; ++u) {
                                const int g = g0 + u * kWarps;
                                if (g < G) {
                                    const float4 q = __ldg(reinterpret_cast<const float4 *>(a.op.sm + (size_t)g * D + d));
                                    const float t0 = fmaf(xr[d], q.x, -q.y), t1 = fmaf(xr[d + 1], q.z, -q.w);
                                    acc[u] = fmaf(t0, t0, acc[u]);
                                    acc2[u] = fmaf(t1, t1, acc2[u]);
                                }
                            }
                        }
                    }
                } else {
#pragma unroll
                    for (int d = 0; d < DMAX; ++d) {
                        if (d < D) {
#pragma unroll
                            for (int u = 0; u < kEmGs; ++u) {
                                const int g = g0 + u * kWarps;
                                if (g < G) {
                                    const float2 q = __ldg(a.op.sm + (size_t)g * D + d);
                                    const float t = fmaf(xr[d], q.x, -q.y);
                                    acc[u] = fmaf(t, t, acc[u]);
                                }
                            }
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < kEmGs; ++u) {
                    const int g = g0 + u * kWarps;
                    if (g < G) L[g * kTP + lane] = fmaf(-0.5f, acc[u] + acc2[u], __ldg(a.op.c + g));
                }
            }
        }
        __syncthreads();
        // ---- LSE + responsibilities
        for (int s = w; s < kTile; s += kWarps) {
            float m = -INFINITY;
            for (int g = lane; g < G; g += 32) m = fmaxf(m, L[g * kTP + s]);
            m = warp_max(m);
            float sum = 0.f;
            for (int g = lane; g < G; g += 32) sum += __expf(L[g * kTP + s] - m);
            sum = warp_sum(sum);
            const float lse = m + logf(sum);
            const bool ok = s < n;
            for (int g = lane; g < G; g += 32) L[g * kTP + s] = ok ? __expf(L[g * kTP + s] - lse) : 0.f;
            if (lane == 0 && ok) ll += (double)lse;
        }
        if (tid == 0) s_nact = 0;
        __syncthreads();
        for (int g = tid; g < G; g += kEmThreads) {
            float mx = 0.f;
            for (int i = 0; i < kTile; ++i) mx = fmaxf(mx, L[g * kTP + i]);
            if (mx >= keep) act[atomicAdd(&s_nact, 1)] = g;
        }
        __syncthreads();
        const int na = s_nact;
        // ---- M: thread-owned (g, d) accumulators over the Gaussians that matter
        // four (g, d) pairs per step: eight independent FMA chains per thread
        for (int p0 = tid; p0 < na * D; p0 += 4 * kEmThreads) {
            int gq[4], dq[4];
            float mu[4], r1[4], r2[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int p = min(p0 + u * kEmThreads, na * D - 1);
                const int ga = p / D;
                gq[u] = act[ga];
                dq[u] = p - ga * D;
                mu[u] = __ldg(a.op.mu + (size_t)gq[u] * D + dq[u]);
                r1[u] = 0.f;
                r2[u] = 0.f;
            }
#pragma unroll 4
            for (int i = 0; i < kTile; ++i) {
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float gm = L[gq[u] * kTP + i];
                    const float uu = xT[dq[u] * kTP + i] - mu[u];
                    r1[u] = fmaf(gm, uu, r1[u]);
                    r2[u] = fmaf(gm * uu, uu, r2[u]);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int p = p0 + u * kEmThreads;
                if (p < na * D) {
                    const int q = gq[u] * D + dq[u];
                    S1[q] += r1[u];
                    S2[q] += r2[u];
                }
            }
        }
        for (int k = tid; k < na; k += kEmThreads) {
            const int g = act[k];
            float r0 = 0.f;
            for (int i = 0; i < kTile; ++i) r0 += L[g * kTP + i];
            S0[g] += r0;
        }
    }
    __syncthreads();
    const int S = 1 + 2 * D;
    double *P = a.partial + (size_t)blockIdx.x * G * S;
    for (int k = tid; k < G * S; k += kEmThreads) {
        const int g = k / S, j = k - g * S;
        P[k] = j == 0 ? (double)S0[g] : (j <= D ? (double)S1[g * D + j - 1] : (double)S2[g * D + j - 1 - D]);
    }
    if (lane == 0) s_ll[w] = ll;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int k = 0; k < kWarps; ++k) t += s_ll[k];
        a.ll_partial[blockIdx.x] = t;
    }
}

// Log-likelihood reduce and the stopping rule: ll_hist[iter] =
// log p(X | lambda_iter) / N; with em_tol > 0, iteration iter >= 1 whose gain
// is below em_tol is the last one.  Fixed order whatever the scheduling: thread
// t sums its contiguous run of partials in order, then a fixed pairwise tree
// (a sequential sum of the 15,625 partials of a 2e6-sample two-phase pass took
// 0.25 ms in one thread).
__global__ void __launch_bounds__(256) k_em_ll(const double *__restrict__ ll_partial, int n_partial, int64_t N,
                                               int32_t iter, double em_tol, double *ll_hist, DevStatus *status)
{
    __shared__ double sh[256];
    __shared__ int s_skip;
    if (threadIdx.x == 0) s_skip = (status->halt != 0 || iter > status->stop_after) ? 1 : 0;
    __syncthreads();
    if (s_skip) return;
    const int t = threadIdx.x;
    const int j0 = (int)((int64_t)n_partial * t / 256), j1 = (int)((int64_t)n_partial * (t + 1) / 256);
    double v = 0.0;
    for (int j = j0; j < j1; ++j) v += ll_partial[j];
    sh[t] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (t < o) sh[t] += sh[t + o];
        __syncthreads();
    }
    if (t != 0) return;
    const double m = sh[0] / (double)N;
    ll_hist[iter] = m;
    if (!isfinite(m)) { set_error(status, GMM_ERR_NONFINITE, iter); return; }
    status->n_done = iter + 1;
    if (em_tol > 0.0 && iter >= 1 && m - ll_hist[iter - 1] < em_tol) status->stop_after = iter;
}

// EM reduce + update (Eqs. 12-14, Eq. 5; floor of Sec. 2.2), then the
// operands of the next E-step.  One block per Gaussian; CTA-order FP64 sums.
// A Gaussian whose responsibility sum L_g is below 1e-8 keeps its mean and
// covariance (its heft is L_g / N): below that mass the re-estimate is a ratio
// of underflowing sums.  A non-finite result stops the call with GMM_ERR_NONFINITE and
// leaves par_in (the last finite parameters) untouched.
__global__ void k_em_finalize(EmFinalizeArgs a)
{
    extern __shared__ double red[];   // [1+2D]
    __shared__ double sh[128];
    __shared__ int s_bad;
    if (block_skip(a.status, a.iter)) return;
    const int g = blockIdx.x, D = a.D, G = a.G, S = 1 + 2 * D;
    for (int j = threadIdx.x; j < S; j += blockDim.x) red[j] = sum_in_order(a.partial + (size_t)g * S + j, a.n_partial, (size_t)G * S);
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    const double Lg = red[0];
    const double *mi = a.par_in + (size_t)g * D, *vi = a.par_in + (size_t)G * D + (size_t)g * D;
    double *mo = a.par_out + (size_t)g * D, *vo = a.par_out + (size_t)G * D + (size_t)g * D;
    const double w = Lg / (double)a.N;
    const bool live = Lg >= 1e-8;   // below this mass the Gaussian keeps its parameters
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
        double mu = mi[d], v = vi[d];
        if (live) {
            const double shift = (double)a.op.mu[(size_t)g * D + d];   // the passes' FP32 shift
            const double m1 = red[1 + d] / Lg;
            mu = shift + m1;
            v = red[1 + D + d] / Lg - m1 * m1;
            v = v > a.var_floor ? v : a.var_floor;
        }
        if (!isfinite(mu) || !isfinite(v)) s_bad = 1;
        mo[d] = mu;
        vo[d] = v;
    }
    if (threadIdx.x == 0) {
        a.par_out[2 * (size_t)G * D + g] = w;
        if (!isfinite(w)) s_bad = 1;
    }
    __syncthreads();
    if (s_bad) { if (threadIdx.x == 0) set_error(a.status, GMM_ERR_NONFINITE, a.iter); return; }
    prep_operands(g, D, G, mo, vo, w, a.op, a.center, a.build_tc, sh);
}

// ------------------------------------------------------------------------
// Inference (Sec. 4.1): log_p with the FP32 operands (online log-sum-exp per
// thread, one sample per thread), and assign.
// ------------------------------------------------------------------------
template <int DMAX>
__global__ void __launch_bounds__(128) k_log_p(const float *__restrict__ X, int64_t N, int32_t D, int32_t G,
                                               Operands op, int32_t gsel, double *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float xr[DMAX];
#pragma unroll
    for (int d = 0; d < DMAX; ++d) xr[d] = d < D ? X[i * D + d] : 0.f;
    auto logit = [&](int g) {
        const float2 *p = op.sm + (size_t)g * D;
        float acc = 0.f;
#pragma unroll
        for (int d = 0; d < DMAX; ++d)
            if (d < D) { const float2 q = __ldg(p + d); const float t = fmaf(xr[d], q.x, -q.y); acc = fmaf(t, t, acc); }
        return -0.5f * acc;
    };
    if (gsel >= 0) { out[i] = (double)logit(gsel) + (double)op.c0[gsel]; return; }
    float m = -INFINITY, s = 0.f;
    for (int g = 0; g < G; ++g) {
        const float l = logit(g) + __ldg(op.c + g);
        if (l > m) { s = s * __expf(m - l) + 1.f; m = l; }
        else if (l > -INFINITY) s += __expf(l - m);   // -inf terms add nothing (and -inf - -inf is NaN)
    }
    out[i] = (double)m + log((double)s);
}

template <int DMAX>
__global__ void __launch_bounds__(128) k_assign(const float *__restrict__ X, int64_t N, int32_t D, int32_t G,
                                                const double *__restrict__ means, Operands op, int32_t mode,
                                                int32_t *__restrict__ out, const double *__restrict__ w_ones)
{
    __shared__ float s_nmax;
    if (threadIdx.x == 0) s_nmax = 0.f;
    __syncthreads();
    if (mode == GMM_EUCL) {
        float nm = 0.f;
        for (int g = threadIdx.x; g < G; g += blockDim.x) {
            float n = 0.f;
            for (int d = 0; d < D; ++d) { const float v = op.mu[(size_t)g * D + d]; n = fmaf(v, v, n); }
            nm = fmaxf(nm, n);
        }
        atomicMax(reinterpret_cast<int *>(&s_nmax), __float_as_int(nm));
        __syncthreads();
    }
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float xr[DMAX];
    float snorm = 0.f;
#pragma unroll
    for (int d = 0; d < DMAX; ++d) { xr[d] = d < D ? X[i * D + d] : 0.f; snorm = fmaf(xr[d], xr[d], snorm); }
    if (mode == GMM_EUCL) {
        float b1 = INFINITY, b2 = INFINITY;
        int a1 = 0;
        for (int g = 0; g < G; ++g) {
            const float *c = op.mu + (size_t)g * D;
            float acc = 0.f;
#pragma unroll
            for (int d = 0; d < DMAX; ++d)
                if (d < D) { const float t = xr[d] - __ldg(c + d); acc = fmaf(t, t, acc); }
            if (acc < b1) { b2 = b1; b1 = acc; a1 = g; }
            else if (acc < b2) b2 = acc;
        }
        const float norms = snorm + s_nmax;
        int best = a1;
        if (G > 1 && !(b2 - km_err(b2, norms, D) > b1 + km_err(b1, norms, D)))
            best = km_recheck_fp64(X + i * D, D, G, means, w_ones);
        out[i] = best;
    } else {
        float bl = -INFINITY;
        int best = 0;
        for (int g = 0; g < G; ++g) {
            const float2 *p = op.sm + (size_t)g * D;
            float acc = 0.f;
#pragma unroll
            for (int d = 0; d < DMAX; ++d)
                if (d < D) { const float2 q = __ldg(p + d); const float t = fmaf(xr[d], q.x, -q.y); acc = fmaf(t, t, acc); }
            const float l = fmaf(-0.5f, acc, __ldg(op.c + g));
            if (l > bl) { bl = l; best = g; }
        }
        out[i] = best;
    }
}

__global__ void k_status_reset(DevStatus *st)
{
    st->code = 0; st->halt = 0; st->stop_after = 0x7fffffff; st->n_done = 0;
    st->fail_iter = -1; st->n_dead = 0;
}

__global__ void k_sum_fp64(const double *__restrict__ v, int64_t n, double *out)
{
    __shared__ double sh[1024];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += v[i];
    s = block_sum_d(s, sh);
    if (threadIdx.x == 0) *out = s;
}

__global__ void k_hist(const int32_t *__restrict__ a, int64_t N, int32_t G, unsigned long long *counts)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        const int g = a[i];
        if (g >= 0 && g < G) atomicAdd(counts + g, 1ull);
    }
}

int dmax_for(int D) { return D <= 16 ? 16 : D <= 32 ? 32 : D <= 64 ? 64 : 128; }

// ------------------------------------------------------------------------
// Allocation-free avg_log_p.  Scratch: one FP64 partial sum per 128-sample
// block plus the grand total, in a fixed device array that every GPU loading
// this library holds until the process exits (512 KiB + 8 B).  Every slot a
// call reads is written by the same call, so nothing has to be cleared; two
// calls whose kernels overlap on the GPU (different streams) race on it.
// ------------------------------------------------------------------------
constexpr int kNoAllocMaxBlocks = 65536;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxBlocks + 1];

template <int DMAX>
__global__ void __launch_bounds__(128) k_log_p_blocksum(const float *__restrict__ X, int64_t N, int32_t D, int32_t G,
                                                        Operands op, int32_t gsel, double *__restrict__ partial)
{
    __shared__ double sh[128];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (i < N) {
        float xr[DMAX];
#pragma unroll
        for (int d = 0; d < DMAX; ++d) xr[d] = d < D ? X[i * D + d] : 0.f;
        auto logit = [&](int g) {
            const float2 *p = op.sm + (size_t)g * D;
            float acc = 0.f;
#pragma unroll
            for (int d = 0; d < DMAX; ++d)
                if (d < D) { const float2 q = __ldg(p + d); const float t = fmaf(xr[d], q.x, -q.y); acc = fmaf(t, t, acc); }
            return -0.5f * acc;
        };
        if (gsel >= 0) {
            v = (double)logit(gsel) + (double)op.c0[gsel];
        } else {
            float m = -INFINITY, s = 0.f;
            for (int g = 0; g < G; ++g) {
                const float l = logit(g) + __ldg(op.c + g);
                if (l > m) { s = s * __expf(m - l) + 1.f; m = l; }
                else if (l > -INFINITY) s += __expf(l - m);   // -inf terms add nothing (and -inf - -inf is NaN)
            }
            v = (double)m + log((double)s);
        }
    }
    v = block_sum_d(v, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = v;
}

}  // namespace

// Device address of the scratch array on the current device.  The symbol's
// host-side name is only a stand-in: the address has to be looked up once per
// device, with that device current, before a kernel may be given it.
static std::mutex g_noalloc_mu;
static double *g_noalloc_dev[256] = {};

static cudaError_t noalloc_scratch(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_dev[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_dev[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_dev[dev];
    return cudaSuccess;
}

int64_t avg_log_p_noalloc_max_n() { return (int64_t)kNoAllocMaxBlocks * 128; }

cudaError_t launch_avg_log_p_noalloc(const float *X, int64_t N, int32_t D, int32_t G, Operands op, int32_t g,
                                     double *sum_host, cudaStream_t s)
{
    if (N < 1 || N > avg_log_p_noalloc_max_n()) return cudaErrorInvalidValue;
    double *scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) return e;
    const int blocks = (int)((N + 127) / 128);
    const int dm = dmax_for(D);
    if (dm == 16) k_log_p_blocksum<16><<<blocks, 128, 0, s>>>(X, N, D, G, op, g, scratch);
    else if (dm == 32) k_log_p_blocksum<32><<<blocks, 128, 0, s>>>(X, N, D, G, op, g, scratch);
    else if (dm == 64) k_log_p_blocksum<64><<<blocks, 128, 0, s>>>(X, N, D, G, op, g, scratch);
    else k_log_p_blocksum<128><<<blocks, 128, 0, s>>>(X, N, D, G, op, g, scratch);
    k_sum_fp64<<<1, 1024, 0, s>>>(scratch, blocks, scratch + kNoAllocMaxBlocks);
    count_launches(2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(sum_host, scratch + kNoAllocMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
        return e;
    return cudaStreamSynchronize(s);
}

// ------------------------------------------------------------------------
// Spread seeding (static_spread / random_spread, Sec. 4.1): greedy
// farthest-first traversal.  Pass g marks seed idx[g] as chosen (mind = -1),
// lowers every other sample's distance to its nearest seed by its distance to
// idx[g] (Eq. 20 with the k-means weights, FP64, d = 0..D-1 without fused
// operations: the oracle's order) and reduces the largest (lowest index on a
// tie) per block; the pick kernel reduces the blocks in order into idx[g+1].
// ------------------------------------------------------------------------
struct SpreadArgs {
    const float *X;
    int64_t N;
    int32_t D;
    const double *w;
    int64_t *idx;
    double *mind;      // [N]
    double *pv;        // [blocks] best distance per block
    int64_t *pi;       // [blocks] its sample
    int32_t g;
    int32_t init;
};

__global__ void __launch_bounds__(256) k_spread_pass(SpreadArgs a)
{
    __shared__ double sv[256];
    __shared__ int64_t si[256];
    const int64_t cur = a.idx[a.g];
    const float *xc = a.X + cur * a.D;
    double bv = -INFINITY;
    int64_t bi = INT64_MAX;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.N; i += (int64_t)gridDim.x * blockDim.x) {
        double md = a.init ? INFINITY : a.mind[i];
        if (i == cur) {
            md = -1.0;
        } else if (md >= 0.0) {
            const float *x = a.X + i * a.D;
            double acc = 0.0;
            for (int d = 0; d < a.D; ++d) {
                const double t = __dsub_rn((double)x[d], (double)xc[d]);
                acc = __dadd_rn(acc, __dmul_rn(a.w[d], __dmul_rn(t, t)));
            }
            if (acc < md) md = acc;
        }
        a.mind[i] = md;
        if (md >= 0.0 && (md > bv || (md == bv && i < bi))) { bv = md; bi = i; }
    }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            const double ov = sv[threadIdx.x + h];
            const int64_t oi = si[threadIdx.x + h];
            if (ov > sv[threadIdx.x] || (ov == sv[threadIdx.x] && oi < si[threadIdx.x])) {
                sv[threadIdx.x] = ov;
                si[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a.pv[blockIdx.x] = sv[0];
        a.pi[blockIdx.x] = si[0];
    }
}

__global__ void k_spread_pick(SpreadArgs a, int nb)
{
    if (threadIdx.x != 0) return;
    double bv = -INFINITY;
    int64_t bi = INT64_MAX;
    for (int b = 0; b < nb; ++b)
        if (a.pv[b] > bv || (a.pv[b] == bv && a.pi[b] < bi)) { bv = a.pv[b]; bi = a.pi[b]; }
    a.idx[a.g + 1] = bi;
}

// ------------------------------------------------------------------------
// generate (Sec. 4.1, M.generate(N)): sample i takes the SplitMix64 outputs
// i*K .. i*K+K-1 of a generator started at state `seed` (counter-based: output
// k = mix(seed + (k+1) * 0x9e3779b97f4a7c15)), u = ((r >> 11) + 0.5) 2^-53;
// the first picks the Gaussian (first g with u < cumulative heft / total,
// else the last), pairs (u1, u2) give Box-Muller normals for dimensions
// 2j, 2j+1; x = mean + sqrt(dcov) z, stored as float.
// ------------------------------------------------------------------------
__device__ __forceinline__ double counter_uniform(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

__global__ void __launch_bounds__(256) k_generate(const double *__restrict__ par, int32_t G, int32_t D, int64_t N,
                                                  uint64_t seed, float *__restrict__ out)
{
    extern __shared__ double cdf[];   // [G] cumulative hefts / total
    const double *mu = par, *var = par + (size_t)G * D, *h = par + 2 * (size_t)G * D;
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int g = 0; g < G; ++g) tot = __dadd_rn(tot, h[g]);
        double c = 0.0;
        for (int g = 0; g < G; ++g) {
            c = __dadd_rn(c, h[g]);
            cdf[g] = __ddiv_rn(c, tot);
        }
    }
    __syncthreads();
    const int64_t K = 1 + 2 * (int64_t)((D + 1) / 2);
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k0 = (uint64_t)(i * K);
        const double u = counter_uniform(seed, k0);
        int lab = G - 1;
        for (int g = 0; g < G; ++g)
            if (u < cdf[g]) { lab = g; break; }
        for (int j = 0; 2 * j < D; ++j) {
            const double u1 = counter_uniform(seed, k0 + 1 + 2 * (uint64_t)j);
            const double u2 = counter_uniform(seed, k0 + 2 + 2 * (uint64_t)j);
            const double r = sqrt(-2.0 * log(u1));
            const double a = two_pi * u2;
            const double z0 = r * cos(a), z1 = r * sin(a);
            const int d = 2 * j;
            out[i * D + d] = (float)(mu[(size_t)lab * D + d] + sqrt(var[(size_t)lab * D + d]) * z0);
            if (d + 1 < D) out[i * D + d + 1] = (float)(mu[(size_t)lab * D + d + 1] + sqrt(var[(size_t)lab * D + d + 1]) * z1);
        }
    }
}

// ======================================================================== host
static std::atomic<long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(std::memory_order_relaxed); }

size_t em_simt_smem(int32_t D, int32_t G)
{
    return sizeof(float) * ((size_t)D * kTP + (size_t)G * kTP + (size_t)G + 2 * (size_t)G * D) + sizeof(int) * (size_t)G;
}

bool em_simt_supported(int32_t D, int32_t G)
{
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return D >= 1 && D <= GMM_MAX_DIMS && em_simt_smem(D, G) <= (size_t)optin;
}

int em_simt_grid(int32_t D, int32_t G, int sms)
{
    const size_t sm = em_simt_smem(D, G);
    int per = (int)((200u * 1024u) / (sm + 2048));
    per = per < 1 ? 1 : (per > 4 ? 4 : per);
    return sms * per;
}

static bool km_tile_fits(int32_t D, int32_t G)
{
    if (D > 64 || G > 256) return false;   // 8 means per lane
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return km_tile_smem(D, G) + 2048u <= (size_t)optin;
}

bool km_tile_supported(int32_t D, int32_t G) { return km_tile_fits(D, G); }

int km_grid(int32_t D, int32_t G, int sms)
{
    if (km_tile_fits(D, G)) return sms;   // tiled form: one CTA per SM
    return em_blocked_chunks(G, sms);     // register-blocked form: one partial per sample chunk
}

cudaError_t launch_global_stats(const float *X, int64_t N, int32_t D, double var_floor, int32_t dist,
                                double *partial, int32_t grid, double *gmean, double *gvar_floored,
                                double *wdist, float *sw, float *center, cudaStream_t s)
{
    const int R = D >= 256 ? 1 : 256 / D;
    const int threads = ((R * D + 31) / 32) * 32;
    const size_t sm = sizeof(double) * threads;
    k_gstats<1><<<grid, threads, sm, s>>>(X, N, D, nullptr, partial);
    k_gstats_final<1><<<D, 128, 0, s>>>(partial, grid, N, D, var_floor, dist, gmean, gvar_floored, wdist, sw,
                                         center);
    k_gstats<2><<<grid, threads, sm, s>>>(X, N, D, gmean, partial);
    k_gstats_final<2><<<D, 128, 0, s>>>(partial, grid, N, D, var_floor, dist, gmean, gvar_floored, wdist, sw,
                                         center);
    count_launches(4);
    return cudaGetLastError();
}

cudaError_t launch_gather_seeds(const float *X, int32_t D, int32_t G, const int64_t *idx, double *par,
                                cudaStream_t s)
{
    k_gather_seeds<<<G, 128, 0, s>>>(X, D, G, idx, par);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_km_pass(const float *X, int64_t N, int32_t D, int32_t G, const double *par,
                           const double *wdist, const float *sw, double *partial, int32_t grid, int32_t *assign,
                           DevStatus *status, cudaStream_t s)
{
    if (!km_tile_fits(D, G)) return cudaErrorInvalidConfiguration;   // the register-blocked form's shapes
    KmArgs a{X, N, D, (D + 3) & ~3, G, G, par, wdist, sw, partial, assign, status};
    const size_t smt = km_tile_smem(D, G);
#define KMT_LAUNCH(NJ)                                                                              \
    do {                                                                                            \
        cudaFuncSetAttribute(k_km_tile<NJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smt); \
        k_km_tile<NJ><<<grid, kKmTileThreads, smt, s>>>(a);                                         \
    } while (0)
    if (G <= 32) KMT_LAUNCH(1);
    else if (G <= 64) KMT_LAUNCH(2);
    else if (G <= 128) KMT_LAUNCH(4);
    else KMT_LAUNCH(8);
#undef KMT_LAUNCH
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_km_finalize(const double *partial, int32_t n_partial, int64_t N, int32_t D, int32_t G,
                               double *par, double var_floor, int32_t final_iter, double *counts,
                               const float *X, const int32_t *assign, const double *gvar_floored,
                               DevStatus *status, cudaStream_t s)
{
    k_km_finalize<<<G, 128, sizeof(double) * (1 + 2 * D), s>>>(partial, n_partial, N, D, G, par, var_floor,
                                                               final_iter, counts, status);
    const size_t sm = sizeof(int64_t) * (size_t)G;
    if (sm > 48 * 1024)
        cudaFuncSetAttribute(k_km_dead_fix, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_km_dead_fix<<<1, 1024, sm, s>>>(X, assign, N, D, G, par, counts, gvar_floored, final_iter, status);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_em_prep(int32_t D, int32_t G, const double *par, Operands op, const float *center,
                           int32_t build_tc, cudaStream_t s)
{
    k_em_prep<<<G, 128, 0, s>>>(D, G, par, op, center, build_tc);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_em_pass_simt(const EmPassArgs &a, int32_t grid, cudaStream_t s)
{
    const size_t sm = em_simt_smem(a.D, a.G);
    const int dm = dmax_for(a.D);
#define EM_LAUNCH(DM)                                                                                   \
    do {                                                                                                \
        cudaFuncSetAttribute(k_em_pass_simt<DM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm); \
        k_em_pass_simt<DM><<<grid, kEmThreads, sm, s>>>(a);                                             \
    } while (0)
    if (dm == 16) EM_LAUNCH(16);
    else if (dm == 32) EM_LAUNCH(32);
    else if (dm == 64) EM_LAUNCH(64);
    else EM_LAUNCH(128);
#undef EM_LAUNCH
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_em_finalize(const EmFinalizeArgs &a, cudaStream_t s)
{
    k_em_ll<<<1, 256, 0, s>>>(a.ll_partial, a.n_ll_partial, a.N, a.iter, a.em_tol, a.ll_hist, a.status);
    k_em_finalize<<<a.G, 128, sizeof(double) * (1 + 2 * a.D), s>>>(a);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_log_p(const float *X, int64_t N, int32_t D, int32_t G, Operands op, int32_t g,
                         double *out, cudaStream_t s)
{
    const int blocks = (int)((N + 127) / 128);
    const int dm = dmax_for(D);
    if (dm == 16) k_log_p<16><<<blocks, 128, 0, s>>>(X, N, D, G, op, g, out);
    else if (dm == 32) k_log_p<32><<<blocks, 128, 0, s>>>(X, N, D, G, op, g, out);
    else if (dm == 64) k_log_p<64><<<blocks, 128, 0, s>>>(X, N, D, G, op, g, out);
    else k_log_p<128><<<blocks, 128, 0, s>>>(X, N, D, G, op, g, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_assign(const float *X, int64_t N, int32_t D, int32_t G, const double *par, Operands op,
                          int32_t mode, int32_t *out, const float *sw_ones, const double *w_ones,
                          DevStatus *status, cudaStream_t s)
{
    (void)sw_ones; (void)status;
    const int blocks = (int)((N + 127) / 128);
    const int dm = dmax_for(D);
    if (dm == 16) k_assign<16><<<blocks, 128, 0, s>>>(X, N, D, G, par, op, mode, out, w_ones);
    else if (dm == 32) k_assign<32><<<blocks, 128, 0, s>>>(X, N, D, G, par, op, mode, out, w_ones);
    else if (dm == 64) k_assign<64><<<blocks, 128, 0, s>>>(X, N, D, G, par, op, mode, out, w_ones);
    else k_assign<128><<<blocks, 128, 0, s>>>(X, N, D, G, par, op, mode, out, w_ones);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_status_reset(DevStatus *st, cudaStream_t s)
{
    k_status_reset<<<1, 1, 0, s>>>(st);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_sum_fp64(const double *v, int64_t n, double *out, cudaStream_t s)
{
    k_sum_fp64<<<1, 1024, 0, s>>>(v, n, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_hist(const int32_t *a, int64_t N, int32_t G, unsigned long long *counts, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * G, s);
    if (e != cudaSuccess) return e;
    if (N > 0) k_hist<<<(int)((N + 255) / 256), 256, 0, s>>>(a, N, G, counts);
    count_launches(N > 0 ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace gmm

namespace gmm {
cudaError_t launch_spread_seeds(const float *X, int64_t N, int32_t D, int32_t G, const double *w, int64_t *idx,
                                double *work, int32_t blocks, cudaStream_t s)
{
    SpreadArgs a{X, N, D, w, idx, work, work + N, reinterpret_cast<int64_t *>(work + N + blocks), 0, 1};
    for (int32_t g = 0; g + 1 < G; ++g) {
        a.g = g;
        a.init = g == 0;
        k_spread_pass<<<blocks, 256, 0, s>>>(a);
        k_spread_pick<<<1, 32, 0, s>>>(a, blocks);
    }
    count_launches(2 * (G > 1 ? G - 1 : 0));
    return cudaGetLastError();
}
}  // namespace gmm

namespace gmm {
namespace {
__global__ void k_f64_to_f32(const double *__restrict__ in, int64_t n, float *__restrict__ out)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = __double2float_rn(in[k]);
}
}  // namespace

cudaError_t launch_f64_to_f32(const double *in, int64_t n, float *out, int sms, cudaStream_t s)
{
    const int64_t blocks = (n + 255) / 256;
    k_f64_to_f32<<<(int)(blocks < 8 * sms ? (blocks > 0 ? blocks : 1) : 8 * sms), 256, 0, s>>>(in, n, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_generate(const double *par, int32_t G, int32_t D, int64_t N, uint64_t seed, float *out, int sms,
                            cudaStream_t s)
{
    const size_t sm = sizeof(double) * (size_t)G;
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_generate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    const int64_t want = (N + 255) / 256;
    const int blocks = (int)(want < 8 * (int64_t)sms ? (want > 0 ? want : 1) : 8 * sms);
    k_generate<<<blocks, 256, sm, s>>>(par, G, D, N, seed, out);
    count_launches(1);
    return cudaGetLastError();
}
}  // namespace gmm
