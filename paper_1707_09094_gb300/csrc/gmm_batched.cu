// Batched form: many independent k-means + EM fits (uneven N, D, N_G) in one
// CUDA graph.  The data passes are persistent kernels over a work list of
// (fit, sample chunk) items -- each item is one "thread" of the paper's
// MapReduce (Sec. 2.1) -- taken from a global counter, so long and short fits
// share the GPU; each item writes its own FP64 partial, and per-(fit,
// Gaussian) reduce/update kernels combine a fit's items in item order (so the
// result does not depend on which CTA took which item).  Arithmetic is that of
// the FP32 CUDA-core form (D <= 64, N_G <= 128 per fit).
#include <cmath>

#include "gmm_internal.cuh"

namespace gmm {

namespace {

constexpr int kBT = 32;            // samples per tile
constexpr int kBTP = kBT + 1;
constexpr int kBThreads = 256;
constexpr int kBWarps = 8;
constexpr int kBDM = 64;           // register tile of a sample (D <= 64)

__device__ __forceinline__ double bsum_d(double v, double *sh)
{
    const int t = threadIdx.x;
    sh[t] = v;
    __syncthreads();
    for (int s = blockDim.x >> 1; s > 0; s >>= 1) {
        if (t < s) sh[t] += sh[t + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ float wmax(float v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float wsum(float v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Next work item for the whole block (thread 0 draws, everyone reads).
__device__ __forceinline__ int next_item(int *counter, int *slot)
{
    __syncthreads();
    if (threadIdx.x == 0) *slot = atomicAdd(counter, 1);
    __syncthreads();
    return *slot;
}

__device__ __forceinline__ bool fit_stopped(const BFitStatus &st, int iter)
{
    return st.halt != 0 || iter > st.stop_after;
}

// ------------------------------------------------------------------ global stats
// One block per fit: per-dimension mean and variance (two passes, FP64), the
// Mahalanobis weights 1/max(var, floor) (or 1) and the centring.
__global__ void __launch_bounds__(256) k_b_gstats(BFit *fits, double var_floor, int dist)
{
    __shared__ double sh[256];
    BFit &f = fits[blockIdx.x];
    const int D = f.D;
    const int64_t N = f.N;
    for (int d = 0; d < D; ++d) {
        double s = 0.0;
        for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s += (double)f.X[i * D + d];
        s = bsum_d(s, sh);
        const double mean = s / (double)N;
        double q = 0.0;
        for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
            const double t = (double)f.X[i * D + d] - mean;
            q += t * t;
        }
        q = bsum_d(q, sh);
        if (threadIdx.x == 0) {
            double v = q / (double)N;
            v = v > var_floor ? v : var_floor;
            f.gvar[d] = v;
            f.w[d] = dist == GMM_MAHA ? 1.0 / v : 1.0;
            f.sw[d] = (float)sqrt(f.w[d]);
            f.center[d] = (float)mean;
        }
    }
}

// One block per (fit, Gaussian): means = the seed samples, unit covariances,
// uniform hefts.
__global__ void k_b_seed(BFit *fits, const int32_t *comp_fit, const int32_t *comp_g)
{
    BFit &f = fits[comp_fit[blockIdx.x]];
    const int g = comp_g[blockIdx.x], D = f.D, G = f.G;
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
        f.par[(size_t)g * D + d] = (double)f.X[f.seed_idx[g] * D + d];
        f.par[(size_t)G * D + (size_t)g * D + d] = 1.0;
    }
    if (threadIdx.x == 0) f.par[2 * (size_t)G * D + g] = 1.0 / (double)G;
}

// ------------------------------------------------------------------ k-means
// Item = (fit, chunk): nearest mean per sample in FP32 (scaled coordinates)
// with the exact FP64 recheck of near ties, assignment, and the shifted hard
// statistics in shared memory (FP32 atomics), flushed to the item's partial.
__device__ __forceinline__ float b_km_err(float d, float norms, int D)
{
    return 4.0f * (2.384185791015625e-07f * sqrtf(2.0f * d * norms) + (float)(D + 4) * 5.9604644775390625e-08f * d)
           + 1e-30f;
}

__global__ void __launch_bounds__(128) k_b_km_pass(BFit *fits, const BItem *items, const int32_t *order, int n_items,
                                                  int *counter, double *partial)
{
    extern __shared__ __align__(16) float bsm[];
    __shared__ int s_item;
    __shared__ float s_nmax;
    while (true) {
        const int k = next_item(counter, &s_item);
        if (k >= n_items) break;
        const int it = order[k];
        const BItem item = items[it];
        BFit &f = fits[item.fit];
        if (f.status->halt) continue;
        const int D = f.D, G = f.G, DP = (D + 3) & ~3;
        float *cent = bsm;                          // [G][DP]
        float *S1 = cent + (size_t)G * DP;          // [G][D]
        float *S2 = S1 + (size_t)G * D;
        float *cnt = S2 + (size_t)G * D;            // [G]
        for (int k = threadIdx.x; k < G * DP; k += blockDim.x) {
            const int g = k / DP, d = k - g * DP;
            cent[k] = d < D ? (float)(f.par[(size_t)g * D + d] * (double)f.sw[d]) : 0.f;
        }
        for (int k = threadIdx.x; k < G * D; k += blockDim.x) { S1[k] = 0.f; S2[k] = 0.f; }
        for (int g = threadIdx.x; g < G; g += blockDim.x) cnt[g] = 0.f;
        if (threadIdx.x == 0) s_nmax = 0.f;
        __syncthreads();
        for (int g = threadIdx.x; g < G; g += blockDim.x) {
            float n = 0.f;
            for (int d = 0; d < D; ++d) n = fmaf(cent[g * DP + d], cent[g * DP + d], n);
            atomicMax(reinterpret_cast<int *>(&s_nmax), __float_as_int(n));
        }
        __syncthreads();
        const float nmax = s_nmax;
        for (int64_t base = item.i0; base < item.i1; base += blockDim.x) {
            const int64_t i = base + threadIdx.x;
            if (i >= item.i1) continue;
            float xr[kBDM], xs[kBDM];
            float snorm = 0.f;
#pragma unroll
            for (int d = 0; d < kBDM; ++d) {
                const float v = d < D ? f.X[i * D + d] : 0.f;
                xr[d] = v;
                xs[d] = d < D ? v * f.sw[d] : 0.f;
                snorm = fmaf(xs[d], xs[d], snorm);
            }
            float b1 = INFINITY, b2 = INFINITY;
            int a1 = 0;
            for (int g = 0; g < G; ++g) {
                const float4 *c4 = reinterpret_cast<const float4 *>(cent + g * DP);
                float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
                for (int q = 0; q < kBDM / 4; ++q) {
                    if (q * 4 < DP) {
                        const float4 c = c4[q];
                        const float t0 = xs[4 * q] - c.x, t1 = xs[4 * q + 1] - c.y;
                        const float t2 = xs[4 * q + 2] - c.z, t3 = xs[4 * q + 3] - c.w;
                        acc0 = fmaf(t0, t0, acc0); acc1 = fmaf(t1, t1, acc1);
                        acc0 = fmaf(t2, t2, acc0); acc1 = fmaf(t3, t3, acc1);
                    }
                }
                const float acc = acc0 + acc1;
                if (acc < b1) { b2 = b1; b1 = acc; a1 = g; }
                else if (acc < b2) b2 = acc;
            }
            int best = a1;
            const float norms = snorm + nmax;
            if (G > 1 && !(b2 - b_km_err(b2, norms, D) > b1 + b_km_err(b1, norms, D))) {
                double bd = INFINITY;
                for (int g = 0; g < G; ++g) {
                    double acc = 0.0;
                    for (int d = 0; d < D; ++d) {
                        const double t = __dsub_rn((double)f.X[i * D + d], f.par[(size_t)g * D + d]);
                        acc = __dadd_rn(acc, __dmul_rn(f.w[d], __dmul_rn(t, t)));
                    }
                    if (acc < bd) { bd = acc; best = g; }
                }
            }
            f.assign[i] = best;
            atomicAdd(&cnt[best], 1.f);
#pragma unroll
            for (int d = 0; d < kBDM; ++d) {
                if (d < D) {
                    const float u = xr[d] - (float)f.par[(size_t)best * D + d];
                    atomicAdd(&S1[best * D + d], u);
                    atomicAdd(&S2[best * D + d], u * u);
                }
            }
        }
        __syncthreads();
        const int S = 1 + 2 * D;
        double *P = partial + item.poff;
        for (int k = threadIdx.x; k < G * S; k += blockDim.x) {
            const int g = k / S, j = k - g * S;
            P[k] = j == 0 ? (double)cnt[g] : (j <= D ? (double)S1[g * D + j - 1] : (double)S2[g * D + j - 1 - D]);
        }
    }
}

// One block per (fit, Gaussian): k-means reduce + update over the fit's items.
__global__ void k_b_km_finalize(BFit *fits, const int32_t *comp_fit, const int32_t *comp_g, const BItem *items,
                                const double *partial, double var_floor, int final_iter)
{
    __shared__ double red[1 + 2 * kBDM];
    BFit &f = fits[comp_fit[blockIdx.x]];
    if (f.status->halt) return;
    const int g = comp_g[blockIdx.x], D = f.D, G = f.G, S = 1 + 2 * D;
    for (int j = threadIdx.x; j < S; j += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < f.n_items; ++k) s += partial[items[f.item0 + k].poff + (size_t)g * S + j];
        red[j] = s;
    }
    __syncthreads();
    const double cnt = red[0];
    if (threadIdx.x == 0) f.counts[g] = cnt;
    if (cnt > 0.0) {
        double *means = f.par, *dcovs = f.par + (size_t)G * D, *hefts = f.par + 2 * (size_t)G * D;
        for (int d = threadIdx.x; d < D; d += blockDim.x) {
            const double shift = (double)(float)means[(size_t)g * D + d];
            const double m1 = red[1 + d] / cnt;
            if (final_iter) {
                const double v = red[1 + D + d] / cnt - m1 * m1;
                dcovs[(size_t)g * D + d] = v > var_floor ? v : var_floor;
            }
            means[(size_t)g * D + d] = shift + m1;
        }
        if (final_iter && threadIdx.x == 0) hefts[g] = cnt / (double)f.N;
    }
}

// One block per fit: dead means (same rule as the single-fit path).
__global__ void __launch_bounds__(256) k_b_km_dead_fix(BFit *fits, int final_iter)
{
    __shared__ int s_pop, s_nd, s_found;
    __shared__ int s_warp[8];
    __shared__ int64_t s_members[128];
    __shared__ double s_h;
    BFit &f = fits[blockIdx.x];
    if (f.status->halt) return;
    const int D = f.D, G = f.G, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tid == 0) {
        int pop = 0, nd = 0;
        for (int g = 0; g < G; ++g) {
            if (f.counts[g] > f.counts[pop]) pop = g;
            if (!(f.counts[g] > 0.0)) ++nd;
        }
        s_pop = pop; s_nd = nd; s_found = 0;
    }
    __syncthreads();
    if (s_nd == 0) return;
    const int pop = s_pop;
    int need = (int)min((int64_t)s_nd, (int64_t)f.counts[pop]);
    for (int64_t base = 0; base < f.N; base += blockDim.x) {
        if (s_found >= need) break;
        const int64_t i = base + tid;
        const int fl = (i < f.N && f.assign[i] == pop) ? 1 : 0;
        const unsigned bal = __ballot_sync(0xffffffffu, fl);
        if (lane == 0) s_warp[wid] = __popc(bal);
        __syncthreads();
        int off = 0, tot = 0;
        for (int w = 0; w < 8; ++w) { if (w < wid) off += s_warp[w]; tot += s_warp[w]; }
        const int pos = s_found + off + __popc(bal & ((1u << lane) - 1u));
        if (fl && pos < need) s_members[pos] = i;
        __syncthreads();
        if (tid == 0) s_found += tot;
        __syncthreads();
    }
    if (s_found < need) need = s_found;
    if (need < 1) return;
    double *means = f.par, *dcovs = f.par + (size_t)G * D, *hefts = f.par + 2 * (size_t)G * D;
    int j = 0;
    for (int g = 0; g < G; ++g) {
        if (f.counts[g] > 0.0) continue;
        const int64_t s = s_members[j % need];
        ++j;
        for (int d = tid; d < D; d += blockDim.x) {
            means[(size_t)g * D + d] = (double)f.X[s * D + d];
            if (final_iter) dcovs[(size_t)g * D + d] = f.gvar[d];
        }
        if (final_iter && tid == 0) hefts[g] = 1.0 / (double)f.N;
    }
    if (final_iter) {
        __syncthreads();
        if (tid == 0) {
            double h = 0.0;
            for (int g = 0; g < G; ++g) h += hefts[g];
            s_h = h;
        }
        __syncthreads();
        for (int g = tid; g < G; g += blockDim.x) hefts[g] /= s_h;
    }
}

// ------------------------------------------------------------------ EM
__device__ void b_prep(BFit &f, int g, const double *par, double *sh)
{
    const int D = f.D, G = f.G;
    double lsum = 0.0;
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
        const double v = par[(size_t)G * D + (size_t)g * D + d], m = par[(size_t)g * D + d];
        const double s = 1.0 / sqrt(v);
        f.sm[(size_t)g * D + d] = make_float2((float)s, (float)(m * s));
        f.mu[(size_t)g * D + d] = (float)m;
        lsum += log(v);
    }
    lsum = bsum_d(lsum, sh);
    if (threadIdx.x == 0) f.c[g] = (float)(log(par[2 * (size_t)G * D + g]) - 0.5 * (double)D * kLog2Pi - 0.5 * lsum);
}

__global__ void __launch_bounds__(128) k_b_em_prep(BFit *fits, const int32_t *comp_fit, const int32_t *comp_g)
{
    __shared__ double sh[128];
    BFit &f = fits[comp_fit[blockIdx.x]];
    b_prep(f, comp_g[blockIdx.x], f.par, sh);
}

// Item = (fit, chunk): the fused FP32 E+M pass of the single-fit form over
// the chunk's 32-sample tiles, statistics in shared memory, flushed to the
// item's FP64 partial; per-item FP64 log-likelihood.
__global__ void __launch_bounds__(kBThreads) k_b_em_pass(BFit *fits, const BItem *items, const int32_t *order,
                                                        int n_items, int *counter, double *partial, double *llp,
                                                        int iter)
{
    extern __shared__ __align__(16) float bsm[];
    __shared__ int s_item;
    __shared__ double s_ll[kBWarps];
    __shared__ int s_nact;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    while (true) {
        const int k = next_item(counter, &s_item);
        if (k >= n_items) break;
        const int it = order[k];
        const BItem item = items[it];
        BFit &f = fits[item.fit];
        if (fit_stopped(*f.status, iter)) continue;
        const int D = f.D, G = f.G;
        float *xT = bsm;                          // [D][kBTP]
        float *L = xT + (size_t)D * kBTP;         // [G][kBTP]
        float *S0 = L + (size_t)G * kBTP;         // [G]
        float *S1 = S0 + G;                       // [G*D]
        float *S2 = S1 + (size_t)G * D;           // [G*D]
        int *act = reinterpret_cast<int *>(S2 + (size_t)G * D);   // [G] Gaussians that matter in the tile
        // the single-fit rule: responsibilities below 1e-9 / N are left out
        const float keep = (float)(1e-9 / (double)f.N);
        for (int k = tid; k < G; k += kBThreads) S0[k] = 0.f;
        for (int k = tid; k < G * D; k += kBThreads) { S1[k] = 0.f; S2[k] = 0.f; }
        double ll = 0.0;
        for (int64_t i0 = item.i0; i0 < item.i1; i0 += kBT) {
            const int n = (int)min((int64_t)kBT, item.i1 - i0);
            __syncthreads();
            const float *Xt = f.X + i0 * D;
            for (int k = tid; k < kBT * D; k += kBThreads) {
                const int i = k / D, d = k - i * D;
                xT[d * kBTP + i] = i < n ? Xt[k] : 0.f;
            }
            __syncthreads();
            {
                float xr[kBDM];
#pragma unroll
                for (int d = 0; d < kBDM; ++d) xr[d] = d < D ? xT[d * kBTP + lane] : 0.f;
                for (int g0 = w; g0 < G; g0 += 4 * kBWarps) {
                    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
                    for (int d = 0; d < kBDM; ++d) {
                        if (d < D) {
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int g = g0 + u * kBWarps;
                                if (g < G) {
                                    const float2 q = __ldg(f.sm + (size_t)g * D + d);
                                    const float t = fmaf(xr[d], q.x, -q.y);
                                    acc[u] = fmaf(t, t, acc[u]);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int g = g0 + u * kBWarps;
                        if (g < G) L[g * kBTP + lane] = fmaf(-0.5f, acc[u], __ldg(f.c + g));
                    }
                }
            }
            __syncthreads();
            for (int s = w; s < kBT; s += kBWarps) {
                float m = -INFINITY;
                for (int g = lane; g < G; g += 32) m = fmaxf(m, L[g * kBTP + s]);
                m = wmax(m);
                float sum = 0.f;
                for (int g = lane; g < G; g += 32) sum += __expf(L[g * kBTP + s] - m);
                sum = wsum(sum);
                const float lse = m + logf(sum);
                const bool ok = s < n;
                for (int g = lane; g < G; g += 32) L[g * kBTP + s] = ok ? __expf(L[g * kBTP + s] - lse) : 0.f;
                if (lane == 0 && ok) ll += (double)lse;
            }
            if (tid == 0) s_nact = 0;
            __syncthreads();
            for (int g = tid; g < G; g += kBThreads) {
                float mx = 0.f;
                for (int i = 0; i < kBT; ++i) mx = fmaxf(mx, L[g * kBTP + i]);
                if (mx >= keep) act[atomicAdd(&s_nact, 1)] = g;
            }
            __syncthreads();
            const int na = s_nact;
            for (int p0 = tid; p0 < na * D; p0 += 4 * kBThreads) {
                int gq[4], dq[4];
                float mu[4], r1[4], r2[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int p = min(p0 + u * kBThreads, na * D - 1);
                    const int ga = p / D;
                    gq[u] = act[ga];
                    dq[u] = p - ga * D;
                    mu[u] = __ldg(f.mu + (size_t)gq[u] * D + dq[u]);
                    r1[u] = 0.f;
                    r2[u] = 0.f;
                }
#pragma unroll 4
                for (int i = 0; i < kBT; ++i) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float gm = L[gq[u] * kBTP + i];
                        const float uu = xT[dq[u] * kBTP + i] - mu[u];
                        r1[u] = fmaf(gm, uu, r1[u]);
                        r2[u] = fmaf(gm * uu, uu, r2[u]);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int p = p0 + u * kBThreads;
                    if (p < na * D) {
                        const int q = gq[u] * D + dq[u];
                        S1[q] += r1[u];
                        S2[q] += r2[u];
                    }
                }
            }
            for (int kk = tid; kk < na; kk += kBThreads) {
                const int g = act[kk];
                float r0 = 0.f;
                for (int i = 0; i < kBT; ++i) r0 += L[g * kBTP + i];
                S0[g] += r0;
            }
        }
        __syncthreads();
        const int S = 1 + 2 * D;
        double *P = partial + item.poff;
        for (int k = tid; k < G * S; k += kBThreads) {
            const int g = k / S, j = k - g * S;
            P[k] = j == 0 ? (double)S0[g] : (j <= D ? (double)S1[g * D + j - 1] : (double)S2[g * D + j - 1 - D]);
        }
        if (lane == 0) s_ll[w] = ll;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int k = 0; k < kBWarps; ++k) t += s_ll[k];
            llp[it] = t;
        }
    }
}

// One thread per fit: log-likelihood of the iteration and the em_tol rule.
__global__ void k_b_em_ll(BFit *fits, int n_fits, const BItem *items, const double *llp, int iter, double em_tol)
{
    const int fi = blockIdx.x * blockDim.x + threadIdx.x;
    if (fi >= n_fits) return;
    BFit &f = fits[fi];
    BFitStatus &st = *f.status;
    if (fit_stopped(st, iter)) return;
    // item indices of fit fi are item0 .. item0 + n_items - 1 (items are grouped by fit)
    double s = 0.0;
    for (int k = 0; k < f.n_items; ++k) s += llp[f.item0 + k];
    const double m = s / (double)f.N;
    f.ll_hist[iter] = m;
    if (!isfinite(m)) { st.code = GMM_ERR_NONFINITE; st.fail_iter = iter; st.halt = 1; return; }
    st.n_done = iter + 1;
    if (em_tol > 0.0 && iter >= 1 && m - f.ll_hist[iter - 1] < em_tol) st.stop_after = iter;
}

// One block per (fit, Gaussian): EM reduce + update (Eqs. 12-14, floor) and
// the next E-step's operands; ping-pong parameter buffers per fit.
__global__ void __launch_bounds__(128) k_b_em_finalize(BFit *fits, const int32_t *comp_fit, const int32_t *comp_g,
                                                       const BItem *items, const double *partial, double var_floor,
                                                       int iter)
{
    __shared__ double red[1 + 2 * kBDM];
    __shared__ double sh[128];
    __shared__ int s_skip, s_bad;
    BFit &f = fits[comp_fit[blockIdx.x]];
    if (threadIdx.x == 0) { s_skip = (f.status->halt != 0 || iter > f.status->stop_after); s_bad = 0; }
    __syncthreads();
    if (s_skip) return;
    const int g = comp_g[blockIdx.x], D = f.D, G = f.G, S = 1 + 2 * D;
    for (int j = threadIdx.x; j < S; j += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < f.n_items; ++k) s += partial[items[f.item0 + k].poff + (size_t)g * S + j];
        red[j] = s;
    }
    __syncthreads();
    const double *pin = (iter & 1) ? f.par2 : f.par;
    double *pout = (iter & 1) ? f.par : f.par2;
    const double Lg = red[0];
    const bool live = Lg >= 1e-8;
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
        double mu = pin[(size_t)g * D + d], v = pin[(size_t)G * D + (size_t)g * D + d];
        if (live) {
            const double m1 = red[1 + d] / Lg;
            mu = (double)f.mu[(size_t)g * D + d] + m1;
            v = red[1 + D + d] / Lg - m1 * m1;
            v = v > var_floor ? v : var_floor;
        }
        if (!isfinite(mu) || !isfinite(v)) s_bad = 1;
        pout[(size_t)g * D + d] = mu;
        pout[(size_t)G * D + (size_t)g * D + d] = v;
    }
    if (threadIdx.x == 0) pout[2 * (size_t)G * D + g] = Lg / (double)f.N;
    __syncthreads();
    if (s_bad) {
        if (threadIdx.x == 0) { f.status->code = GMM_ERR_NONFINITE; f.status->fail_iter = iter; f.status->halt = 1; }
        return;
    }
    b_prep(f, g, pout, sh);
}

}  // namespace

size_t b_em_smem(int D, int G)
{
    return sizeof(float) * ((size_t)D * kBTP + (size_t)G * kBTP + G + 2 * (size_t)G * D) + sizeof(int) * (size_t)G;
}

size_t b_km_smem(int D, int G)
{
    const int DP = (D + 3) & ~3;
    return sizeof(float) * ((size_t)G * DP + 2 * (size_t)G * D + G);
}

// Shared-memory limits of the two persistent kernels; set outside any stream
// capture, before the first launch.
cudaError_t b_prepare(size_t em_smem, size_t km_smem)
{
    cudaError_t e = cudaFuncSetAttribute(k_b_em_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)em_smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_b_km_pass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)km_smem);
    return e;
}

cudaError_t launch_b_gstats(BFit *fits, int n_fits, double var_floor, int dist, cudaStream_t s)
{
    k_b_gstats<<<n_fits, 256, 0, s>>>(fits, var_floor, dist);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_b_seed(BFit *fits, const int32_t *comp_fit, const int32_t *comp_g, int n_comp, cudaStream_t s)
{
    k_b_seed<<<n_comp, 64, 0, s>>>(fits, comp_fit, comp_g);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_b_km_iter(BFit *fits, int n_fits, const int32_t *comp_fit, const int32_t *comp_g, int n_comp,
                             const BItem *items, const int32_t *order, int n_items, int *counter, double *partial,
                             size_t smem, int grid, double var_floor, int final_iter, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_b_km_pass<<<grid, 128, smem, s>>>(fits, items, order, n_items, counter, partial);
    k_b_km_finalize<<<n_comp, 128, 0, s>>>(fits, comp_fit, comp_g, items, partial, var_floor, final_iter);
    k_b_km_dead_fix<<<n_fits, 256, 0, s>>>(fits, final_iter);
    count_launches(3);
    return cudaGetLastError();
}

cudaError_t launch_b_em_prep(BFit *fits, const int32_t *comp_fit, const int32_t *comp_g, int n_comp, cudaStream_t s)
{
    k_b_em_prep<<<n_comp, 128, 0, s>>>(fits, comp_fit, comp_g);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_b_em_pass(BFit *fits, const BItem *items, const int32_t *order, int n_items, int *counter,
                             double *partial, double *llp, size_t smem, int grid, int iter, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    k_b_em_pass<<<grid, kBThreads, smem, s>>>(fits, items, order, n_items, counter, partial, llp, iter);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_b_em_finish(BFit *fits, int n_fits, const int32_t *comp_fit, const int32_t *comp_g, int n_comp,
                               const BItem *items, const double *partial, const double *llp, double var_floor,
                               double em_tol, int iter, cudaStream_t s)
{
    k_b_em_ll<<<(n_fits + 127) / 128, 128, 0, s>>>(fits, n_fits, items, llp, iter, em_tol);
    k_b_em_finalize<<<n_comp, 128, 0, s>>>(fits, comp_fit, comp_g, items, partial, var_floor, iter);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace gmm
