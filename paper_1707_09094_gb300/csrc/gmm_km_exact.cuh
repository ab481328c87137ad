// Exact nearest-mean decision shared by the CUDA-core k-means forms
// (gmm_simt.cu, gmm_blocked.cu) and assign: the FP32 distance's rounding
// bound and the FP64 re-decision of near ties.
#pragma once
#include <cuda_runtime.h>

namespace gmm {

// ------------------------------------------------------------------------
// Nearest mean (Eq. 19) with an exact FP64 recheck of near ties.
// FP32 distances use scaled coordinates xs = x*sqrt(w), cs = mu*sqrt(w).
// Rounding bound of one FP32 distance d (x, mu rounded to FP32, t = xs - cs
// rounded, FMA accumulation): |err| <= 2^-22 sqrt(2 d (|xs|^2 + |cs|^2))
// + (D + 4) 2^-24 d.  If the runner-up minus its bound still exceeds the
// winner plus its bound, the FP32 winner is the exact winner; otherwise all
// Gaussians are re-evaluated in FP64 exactly as sum_d w_d (x_d - mu_d)^2 in
// order d = 0..D-1 without fused operations, lowest index on exact ties.
// ------------------------------------------------------------------------
__device__ __forceinline__ float km_err(float d, float norms, int D)
{
    return 4.0f * (2.384185791015625e-07f * sqrtf(2.0f * d * norms) + (float)(D + 4) * 5.9604644775390625e-08f * d)
           + 1e-30f;
}

__device__ inline int km_recheck_fp64(const float *__restrict__ x, int D, int G, const double *__restrict__ means,
                               const double *__restrict__ w)
{
    double best = INFINITY;
    int a = 0;
    for (int g = 0; g < G; ++g) {
        const double *mu = means + (size_t)g * D;
        double acc = 0.0;
        for (int d = 0; d < D; ++d) {
            double t = __dsub_rn((double)x[d], mu[d]);
            acc = __dadd_rn(acc, __dmul_rn(w[d], __dmul_rn(t, t)));
        }
        if (acc < best) { best = acc; a = g; }
    }
    return a;
}

}  // namespace gmm
