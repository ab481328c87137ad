/*
 * gmm_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle for
 * diagonal-covariance GMM training by k-means + EM, written from the paper
 * "An Open Source C++ Implementation of Multi-Threaded Gaussian Mixture
 * Models, k-Means and Expectation Maximisation" (arXiv 1707.09094).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or helper with
 * the CUDA library; the two meet only through plain arrays.
 *
 * Conventions
 *   X      float  [N][D]  one sample per row (the paper stores one sample per
 *                         column of a D x N matrix; the bytes are the same).
 *   means  double [G][D]  dcovs double [G][D]   hefts double [G]
 *   All arithmetic is IEEE double, round-to-nearest.  The file is compiled
 *   with -ffp-contract=off so that no multiply-add is fused behind our back.
 *
 * Every function names the passage of the paper it follows.  Where the paper
 * is silent the reading taken is stated inline (tag "reading").
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_NONFINITE (-2)
#define ORC_ERR_OOM (-5)

static const double ORC_LOG_2PI = 1.83787706640934548356065947281123527;

/* ------------------------------------------------------------------------ */
/* Log density of one diagonal Gaussian: Eq. 15 (log of Eq. 2) with the     */
/* determinant a product and the inverse a reciprocal of the diagonal       */
/* (Sec. 4, items (i) and (ii)).  Direct form: sum of (x-mu)^2 / sigma^2.   */
/* ------------------------------------------------------------------------ */
double orc_log_gauss(const float *x, const double *mu, const double *dcov, int32_t D)
{
    double log_det = 0.0, maha = 0.0;
    for (int32_t d = 0; d < D; ++d) {
        double t = (double)x[d] - mu[d];
        log_det += log(dcov[d]);
        maha += (t * t) / dcov[d];
    }
    return -(0.5 * (double)D * ORC_LOG_2PI + 0.5 * log_det) - 0.5 * maha;
}

/* Eq. 17-18: log(exp(la) + exp(lb)) = la + log(1 + exp(lb - la)) after
 * swapping so that la >= lb.  Both -inf gives -inf.  (log1p is used for
 * log(1 + .); it is the same quantity, evaluated without forming 1 + tiny.) */
double orc_log_add(double la, double lb)
{
    if (la < lb) { double t = la; la = lb; lb = t; }
    if (lb == -INFINITY) return la;
    return la + log1p(exp(lb - la));
}

/* log(w_g N(x|g)) for every g; Eq. 16's summands. */
static void orc_log_terms(const float *x, int32_t D, int32_t G, const double *means,
                          const double *dcovs, const double *hefts, double *t)
{
    for (int32_t g = 0; g < G; ++g)
        t[g] = log(hefts[g]) + orc_log_gauss(x, means + (size_t)g * D, dcovs + (size_t)g * D, D);
}

/* Eq. 16 evaluated as the paper does: a running pairwise log-add over g. */
static double orc_log_mix_pairwise(const double *t, int32_t G)
{
    double acc = t[0];
    for (int32_t g = 1; g < G; ++g) acc = orc_log_add(acc, t[g]);
    return acc;
}

/* Eq. 16 evaluated the other textbook way (max + sum of exp), used only to
 * cross-check the pairwise form. */
static double orc_log_mix_maxsum(const double *t, int32_t G)
{
    double m = -INFINITY;
    for (int32_t g = 0; g < G; ++g) if (t[g] > m) m = t[g];
    if (m == -INFINITY) return -INFINITY;
    double s = 0.0;
    for (int32_t g = 0; g < G; ++g) s += exp(t[g] - m);
    return m + log(s);
}

/* log p(x_i | lambda) (Eq. 1 in log form, Eq. 16), or with g >= 0 the log
 * density of Gaussian g alone (reading of `log_p(X, g)`: the likelihood
 * "according to Gaussian g" is N(x | mu_g, Sigma_g), without its heft).
 * maxsum != 0 selects the cross-check evaluation of Eq. 16. */
int orc_log_p(const float *X, int64_t N, int32_t D, int32_t G, const double *means,
              const double *dcovs, const double *hefts, int32_t g, int32_t maxsum, double *out)
{
    if (N < 0 || D < 1 || G < 1 || g >= G || g < -1) return ORC_ERR_ARG;
    double *t = (double *)malloc(sizeof(double) * (size_t)G);
    if (!t) return ORC_ERR_OOM;
    for (int64_t i = 0; i < N; ++i) {
        const float *x = X + (size_t)i * D;
        if (g >= 0) {
            out[i] = orc_log_gauss(x, means + (size_t)g * D, dcovs + (size_t)g * D, D);
        } else {
            orc_log_terms(x, D, G, means, dcovs, hefts, t);
            out[i] = maxsum ? orc_log_mix_maxsum(t, G) : orc_log_mix_pairwise(t, G);
        }
    }
    free(t);
    return ORC_OK;
}

/* avg_log_p (Sec. 4.1): the mean over samples of log_p. */
int orc_avg_log_p(const float *X, int64_t N, int32_t D, int32_t G, const double *means,
                  const double *dcovs, const double *hefts, int32_t g, double *out)
{
    if (N < 1) return ORC_ERR_ARG;
    double *lp = (double *)malloc(sizeof(double) * (size_t)N);
    if (!lp) return ORC_ERR_OOM;
    int rc = orc_log_p(X, N, D, G, means, dcovs, hefts, g, 0, lp);
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i) s += lp[i];
    *out = s / (double)N;
    free(lp);
    return rc;
}

/* Eq. 3: the a-posteriori probability l_{g,i} of every Gaussian for every
 * sample, computed in the log domain (Sec. 2.2): exp(log w_g N_g - log p). */
int orc_posteriors(const float *X, int64_t N, int32_t D, int32_t G, const double *means,
                   const double *dcovs, const double *hefts, double *post /* [N][G] */)
{
    double *t = (double *)malloc(sizeof(double) * (size_t)G);
    if (!t) return ORC_ERR_OOM;
    for (int64_t i = 0; i < N; ++i) {
        orc_log_terms(X + (size_t)i * D, D, G, means, dcovs, hefts, t);
        double lp = orc_log_mix_pairwise(t, G);
        for (int32_t g = 0; g < G; ++g) post[(size_t)i * G + g] = exp(t[g] - lp);
    }
    free(t);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Global diagonal covariance for the Mahalanobis distance (Eq. 20 and the   */
/* paragraph after it): per-dimension mean and variance over all samples,   */
/* divided by N (reading: the ML estimate, as in Eq. 7), two passes.        */
/* ------------------------------------------------------------------------ */
int orc_global_stats(const float *X, int64_t N, int32_t D, double *mean, double *var)
{
    if (N < 1 || D < 1) return ORC_ERR_ARG;
    for (int32_t d = 0; d < D; ++d) { mean[d] = 0.0; var[d] = 0.0; }
    for (int64_t i = 0; i < N; ++i)
        for (int32_t d = 0; d < D; ++d) mean[d] += (double)X[(size_t)i * D + d];
    for (int32_t d = 0; d < D; ++d) mean[d] /= (double)N;
    for (int64_t i = 0; i < N; ++i)
        for (int32_t d = 0; d < D; ++d) {
            double t = (double)X[(size_t)i * D + d] - mean[d];
            var[d] += t * t;
        }
    for (int32_t d = 0; d < D; ++d) var[d] /= (double)N;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* random_subset seeding (Sec. 4.1, `seed_mode`).  The paper names no RNG.   */
/* Reading: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom  */
/* number generators", OOPSLA 2014) drives a partial Fisher-Yates shuffle of */
/* the sample indices; the first G shuffled indices are the seeds (distinct). */
/* ------------------------------------------------------------------------ */
static uint64_t orc_splitmix64(uint64_t *state)
{
    uint64_t z = (*state += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

int orc_seed_random_subset(int64_t N, int32_t G, uint64_t seed, int64_t *idx_out)
{
    if (G < 1 || (int64_t)G > N) return ORC_ERR_ARG;
    int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    if (!perm) return ORC_ERR_OOM;
    for (int64_t i = 0; i < N; ++i) perm[i] = i;
    uint64_t st = seed;
    for (int32_t j = 0; j < G; ++j) {
        uint64_t r = orc_splitmix64(&st) % (uint64_t)(N - j);
        int64_t k = j + (int64_t)r;
        int64_t tmp = perm[j]; perm[j] = perm[k]; perm[k] = tmp;
        idx_out[j] = perm[j];
    }
    free(perm);
    return ORC_OK;
}

double orc_km_dist(const float *x, const double *mu, const double *w, int32_t D);

/* static_subset (Sec. 4.1, seed_mode): "a subset of the training samples
 * (repeatable)".  Reading: N_G samples at evenly spaced indices
 * floor(g * N / N_G), g = 0..N_G-1 -- repeatable and free of random numbers. */
int orc_seed_static_subset(int64_t N, int32_t G, int64_t *idx_out)
{
    if (G < 1 || (int64_t)G > N) return ORC_ERR_ARG;
    for (int32_t g = 0; g < G; ++g) idx_out[g] = (int64_t)(((__int128)g * N) / G);
    return ORC_OK;
}

/* static_spread / random_spread (Sec. 4.1, seed_mode): "a maximally spread
 * subset of training samples", repeatable or from a random start, inspired
 * by k-means++.  Reading: greedy farthest-first traversal.  The first seed is
 * sample `first`; each next seed is the sample whose distance (Eq. 20 with
 * the k-means weights w: Mahalanobis or Euclidean, in the order of
 * orc_km_dist) to its nearest chosen seed is largest, the lowest index on an
 * exact tie; chosen samples are never chosen again (so the seeds are
 * distinct even when samples repeat). */
int orc_seed_spread(const float *X, int64_t N, int32_t D, int32_t G, const double *w, int64_t first,
                    int64_t *idx_out)
{
    if (G < 1 || (int64_t)G > N || first < 0 || first >= N) return ORC_ERR_ARG;
    double *mind = (double *)malloc(sizeof(double) * (size_t)N);
    double *mu = (double *)malloc(sizeof(double) * (size_t)D);
    if (!mind || !mu) { free(mind); free(mu); return ORC_ERR_OOM; }
    for (int64_t i = 0; i < N; ++i) mind[i] = INFINITY;
    int64_t cur = first;
    for (int32_t g = 0; g < G; ++g) {
        idx_out[g] = cur;
        mind[cur] = -1.0;   /* chosen */
        if (g + 1 == G) break;
        for (int32_t d = 0; d < D; ++d) mu[d] = (double)X[(size_t)cur * D + d];
        int64_t best = -1;
        double bv = -INFINITY;
        for (int64_t i = 0; i < N; ++i) {
            if (mind[i] < 0.0) continue;
            double dd = orc_km_dist(X + (size_t)i * D, mu, w, D);
            if (dd < mind[i]) mind[i] = dd;
            if (mind[i] > bv) { bv = mind[i]; best = i; }
        }
        cur = best;
    }
    free(mind);
    free(mu);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* k-means (Sec. 3): the hard-assignment special case of EM, Eq. 19.         */
/* ------------------------------------------------------------------------ */

/* dist(mu_g, x) = sum_d w_d (x_d - mu_gd)^2 : Eq. 20 with a diagonal global
 * covariance (w_d = 1 / sigma^2_global,d), or the squared Euclidean distance
 * (Sec. 3.1) when every w_d = 1.  Fixed order d = 0..D-1, no fused ops. */
double orc_km_dist(const float *x, const double *mu, const double *w, int32_t D)
{
    double acc = 0.0;
    for (int32_t d = 0; d < D; ++d) {
        double t = (double)x[d] - mu[d];
        acc = acc + w[d] * (t * t);
    }
    return acc;
}

/* Eq. 19: index of the nearest mean; the lowest index wins an exact tie
 * (reading: the paper is silent on ties).  Also returns the two smallest
 * distances so that callers can tell near-ties apart. */
int orc_km_assign(const float *X, int64_t N, int32_t D, int32_t G, const double *means,
                  const double *w, int32_t *assign, double *d_best, double *d_second)
{
    /* the map step of Sec. 3: every sample independently (OpenMP threads
     * over samples; no result depends on the thread count) */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < N; ++i) {
        const float *x = X + (size_t)i * D;
        double b1 = INFINITY, b2 = INFINITY;
        int32_t a = 0;
        for (int32_t g = 0; g < G; ++g) {
            double dg = orc_km_dist(x, means + (size_t)g * D, w, D);
            if (dg < b1) { b2 = b1; b1 = dg; a = g; }
            else if (dg < b2) { b2 = dg; }
        }
        assign[i] = a;
        if (d_best) d_best[i] = b1;
        if (d_second) d_second[i] = b2;
    }
    return ORC_OK;
}

/*
 * Full k-means initialisation (Sec. 3, Sec. 3.1).
 *   means  in: the seed means; out: the k-means estimate of the means.
 *   dcovs, hefts out: the first EM estimate from the hard statistics of the
 *          last iteration (Eqs. 5-7 with l from Eq. 19, Sec. 3).
 *   w      the distance weights (Eq. 20 or all ones).
 *   gvar_floored  per-dimension floored global variance (used for the
 *          covariance of a mean that is still dead after the last iteration).
 * Each iteration: (i) distances and Eq. 19 assignment, (ii) each mean becomes
 * the average of its samples (Sec. 3), then every "dead" mean (no samples)
 * is made equal to a vector assigned to the most popular mean (Sec. 3.1).
 * Reading of that heuristic (the paper does not say which vector): popular =
 * largest count, lowest index on ties; the dead means, in increasing index
 * order, take the 1st, 2nd, ... lowest-index samples of the popular mean
 * (cycling if there are more dead means than such samples).  After the last
 * iteration a dead mean gets the floored global variance and a heft of 1/N,
 * and the hefts are renormalised to sum to one.
 */
int orc_kmeans(const float *X, int64_t N, int32_t D, int32_t G, const double *w,
               const double *gvar_floored, double *means, double *dcovs, double *hefts,
               int32_t km_iter, double var_floor, int32_t *assign_last)
{
    if (N < 1 || D < 1 || G < 1 || (int64_t)G > N || km_iter < 1) return ORC_ERR_ARG;
    size_t GD = (size_t)G * D;
    int32_t *a = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    double *cnt = (double *)malloc(sizeof(double) * G);
    double *s1 = (double *)malloc(sizeof(double) * GD);
    double *s2 = (double *)malloc(sizeof(double) * GD);
    if (!a || !cnt || !s1 || !s2) { free(a); free(cnt); free(s1); free(s2); return ORC_ERR_OOM; }

    for (int32_t it = 0; it < km_iter; ++it) {
        orc_km_assign(X, N, D, G, means, w, a, NULL, NULL);
        for (int32_t g = 0; g < G; ++g) cnt[g] = 0.0;
        memset(s1, 0, sizeof(double) * GD);
        memset(s2, 0, sizeof(double) * GD);
        for (int64_t i = 0; i < N; ++i) {
            const float *x = X + (size_t)i * D;
            int32_t g = a[i];
            cnt[g] += 1.0;
            for (int32_t d = 0; d < D; ++d) {
                double v = (double)x[d];
                s1[(size_t)g * D + d] += v;
                s2[(size_t)g * D + d] += v * v;
            }
        }
        /* (ii) new means = average of the assigned samples */
        int32_t pop = 0, n_dead = 0;
        for (int32_t g = 0; g < G; ++g) {
            if (cnt[g] > 0.0) {
                for (int32_t d = 0; d < D; ++d) means[(size_t)g * D + d] = s1[(size_t)g * D + d] / cnt[g];
            } else {
                ++n_dead;
            }
            if (cnt[g] > cnt[pop]) pop = g;
        }
        /* dead-mean resurrection (Sec. 3.1) */
        if (n_dead > 0) {
            int64_t n_pop = (int64_t)cnt[pop], k = 0;
            int64_t *members = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_pop);
            if (!members) { free(a); free(cnt); free(s1); free(s2); return ORC_ERR_OOM; }
            for (int64_t i = 0; i < N && k < n_pop; ++i) if (a[i] == pop) members[k++] = i;
            int64_t j = 0;
            for (int32_t g = 0; g < G; ++g) {
                if (cnt[g] > 0.0) continue;
                int64_t s = members[j % n_pop];
                ++j;
                for (int32_t d = 0; d < D; ++d) means[(size_t)g * D + d] = (double)X[(size_t)s * D + d];
            }
            free(members);
        }
        if (it == km_iter - 1) {
            /* Eqs. 5-7 with hard l (Sec. 3): hefts, and diagonal covariances in
             * the one-pass form of Eq. 8, floored (Sec. 2.2). */
            double hsum = 0.0;
            for (int32_t g = 0; g < G; ++g) {
                if (cnt[g] > 0.0) {
                    hefts[g] = cnt[g] / (double)N;
                    for (int32_t d = 0; d < D; ++d) {
                        double mu = means[(size_t)g * D + d];
                        double v = s2[(size_t)g * D + d] / cnt[g] - mu * mu;
                        dcovs[(size_t)g * D + d] = v > var_floor ? v : var_floor;
                    }
                } else {
                    hefts[g] = 1.0 / (double)N;
                    for (int32_t d = 0; d < D; ++d) dcovs[(size_t)g * D + d] = gvar_floored[d];
                }
                hsum += hefts[g];
            }
            if (n_dead > 0)
                for (int32_t g = 0; g < G; ++g) hefts[g] /= hsum;
        }
    }
    if (assign_last) memcpy(assign_last, a, sizeof(int32_t) * (size_t)N);
    free(a); free(cnt); free(s1); free(s2);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* EM (Sec. 2) in the MapReduce form of Sec. 2.1.                           */
/* ------------------------------------------------------------------------ */

/*
 * One EM iteration, n_chunks "threads" (Sec. 2.1):
 *   map   : chunk t accumulates L~_g (Eq. 9), mu~_g (Eq. 10) and the diagonal
 *           of Sigma~_g (Eq. 11) over its contiguous samples, with l_{g,j}
 *           from Eq. 3 evaluated in the log domain (Eqs. 15-18);
 *   reduce: Eqs. 12-14 sum the chunks in order t = 1..N_T and divide;
 *   update: hefts by Eq. 5, variances by the one-pass form of Eq. 8 / Eq. 14,
 *           floored after the iteration (Sec. 2.2).
 * Eqs. 12-14 define the new mean and covariance for every L_g > 0, and so
 * does this function.  Reading for L_g == 0 (every responsibility underflowed;
 * the paper is silent): the heft becomes 0 and the mean and covariance are
 * kept, which only avoids 0/0.
 * *mean_ll receives log p(X | lambda_old) / N, the likelihood of the
 * parameters the E-step used.
 */
static int orc_em_one(const float *X, int64_t N, int32_t D, int32_t G, double *means,
                      double *dcovs, double *hefts, double var_floor, int32_t n_chunks,
                      double *mean_ll)
{
    size_t GD = (size_t)G * D;
    size_t per = (size_t)G * (1 + 2 * (size_t)D);      /* L~, mu~, Sigma~ per chunk */
    double *acc = (double *)calloc((size_t)n_chunks * per, sizeof(double));
    double *chunk_ll = (double *)calloc((size_t)n_chunks, sizeof(double));
    if (!acc || !chunk_ll) { free(acc); free(chunk_ll); return ORC_ERR_OOM; }

#ifdef _OPENMP
#pragma omp parallel for schedule(static, 1)
#endif
    for (int32_t t = 0; t < n_chunks; ++t) {
        int64_t i0 = (int64_t)((double)N * t / n_chunks);
        int64_t i1 = (int64_t)((double)N * (t + 1) / n_chunks);
        double *Lt = acc + (size_t)t * per;
        double *Mt = Lt + G;
        double *St = Mt + GD;
        double *lt = (double *)malloc(sizeof(double) * (size_t)G);
        double ll = 0.0;
        for (int64_t i = i0; i < i1; ++i) {
            const float *x = X + (size_t)i * D;
            orc_log_terms(x, D, G, means, dcovs, hefts, lt);
            double lp = orc_log_mix_pairwise(lt, G);
            ll += lp;
            for (int32_t g = 0; g < G; ++g) {
                double l = exp(lt[g] - lp);                         /* Eq. 3 */
                Lt[g] += l;                                          /* Eq. 9 */
                for (int32_t d = 0; d < D; ++d) {
                    double v = (double)x[d];
                    Mt[(size_t)g * D + d] += l * v;                  /* Eq. 10 */
                    St[(size_t)g * D + d] += l * (v * v);            /* Eq. 11, diagonal */
                }
            }
        }
        chunk_ll[t] = ll;
        free(lt);
    }

    /* reduce, Eqs. 12-14, chunks in order */
    double *L = (double *)calloc(per, sizeof(double));
    if (!L) { free(acc); free(chunk_ll); return ORC_ERR_OOM; }
    double *M = L + G, *S = M + GD;
    double ll = 0.0;
    for (int32_t t = 0; t < n_chunks; ++t) {
        const double *src = acc + (size_t)t * per;
        for (size_t k = 0; k < per; ++k) L[k] += src[k];
        ll += chunk_ll[t];
    }
    *mean_ll = ll / (double)N;

    int rc = ORC_OK;
    for (int32_t g = 0; g < G; ++g) {
        hefts[g] = L[g] / (double)N;                                  /* Eq. 5 */
        if (!(L[g] > 0.0)) continue;                                  /* 0/0 guard only */
        for (int32_t d = 0; d < D; ++d) {
            double mu = M[(size_t)g * D + d] / L[g];                  /* Eq. 13 */
            double v = S[(size_t)g * D + d] / L[g] - mu * mu;         /* Eq. 14 */
            v = v > var_floor ? v : var_floor;                        /* floor, Sec. 2.2 */
            means[(size_t)g * D + d] = mu;
            dcovs[(size_t)g * D + d] = v;
            if (!isfinite(mu) || !isfinite(v)) rc = ORC_ERR_NONFINITE;
        }
    }
    if (!isfinite(*mean_ll)) rc = ORC_ERR_NONFINITE;
    free(acc); free(chunk_ll); free(L);
    return rc;
}

/*
 * em_iter EM iterations from the given parameters.  ll_hist[k] = mean log
 * likelihood of the parameters used by iteration k.  Stopping (Sec. 2, last
 * paragraph before Sec. 2.1; `em_iter` is a maximum): with em_tol > 0 the loop
 * ends after an iteration k >= 1 whose ll_hist[k] - ll_hist[k-1] < em_tol
 * (that iteration's update is kept).  *n_done = iterations run.
 */
int orc_em_iterate(const float *X, int64_t N, int32_t D, int32_t G, double *means, double *dcovs,
                   double *hefts, int32_t em_iter, double var_floor, double em_tol,
                   int32_t n_chunks, double *ll_hist, int32_t *n_done)
{
    if (N < 1 || D < 1 || G < 1 || n_chunks < 1 || em_iter < 0) return ORC_ERR_ARG;
    int32_t k = 0;
    for (; k < em_iter; ++k) {
        double ll = 0.0;
        int rc = orc_em_one(X, N, D, G, means, dcovs, hefts, var_floor, n_chunks, &ll);
        if (ll_hist) ll_hist[k] = ll;
        if (rc != ORC_OK) { if (n_done) *n_done = k + 1; return rc; }
        if (em_tol > 0.0 && k >= 1 && ll_hist && ll_hist[k] - ll_hist[k - 1] < em_tol) { ++k; break; }
    }
    if (n_done) *n_done = k;
    return ORC_OK;
}

/*
 * One EM iteration with the covariance of Eq. 7 evaluated directly (two
 * passes: means first, then the weighted scatter about the new means).  Used
 * only to bound the cancellation of the one-pass form of Eq. 8.
 */
int orc_em_step_twopass(const float *X, int64_t N, int32_t D, int32_t G, double *means,
                        double *dcovs, double *hefts, double var_floor)
{
    size_t GD = (size_t)G * D;
    double *post = (double *)malloc(sizeof(double) * (size_t)N * G);
    double *L = (double *)calloc((size_t)G, sizeof(double));
    double *M = (double *)calloc(GD, sizeof(double));
    double *S = (double *)calloc(GD, sizeof(double));
    if (!post || !L || !M || !S) { free(post); free(L); free(M); free(S); return ORC_ERR_OOM; }
    orc_posteriors(X, N, D, G, means, dcovs, hefts, post);
    for (int64_t i = 0; i < N; ++i)
        for (int32_t g = 0; g < G; ++g) {
            double l = post[(size_t)i * G + g];
            L[g] += l;                                                    /* Eq. 4 */
            for (int32_t d = 0; d < D; ++d) M[(size_t)g * D + d] += l * (double)X[(size_t)i * D + d];
        }
    for (int32_t g = 0; g < G; ++g)
        for (int32_t d = 0; d < D; ++d) M[(size_t)g * D + d] /= L[g];    /* Eq. 6 */
    for (int64_t i = 0; i < N; ++i)
        for (int32_t g = 0; g < G; ++g) {
            double l = post[(size_t)i * G + g];
            for (int32_t d = 0; d < D; ++d) {
                double t = (double)X[(size_t)i * D + d] - M[(size_t)g * D + d];
                S[(size_t)g * D + d] += l * (t * t);                      /* Eq. 7, diagonal */
            }
        }
    for (int32_t g = 0; g < G; ++g) {
        hefts[g] = L[g] / (double)N;                                      /* Eq. 5 */
        if (!(L[g] > 0.0)) continue;                                      /* 0/0 guard only */
        for (int32_t d = 0; d < D; ++d) {
            double v = S[(size_t)g * D + d] / L[g];
            means[(size_t)g * D + d] = M[(size_t)g * D + d];
            dcovs[(size_t)g * D + d] = v > var_floor ? v : var_floor;
        }
    }
    free(post); free(L); free(M); free(S);
    return ORC_OK;
}

/*
 * One EM iteration (exactly orc_em_iterate with em_iter = 1, var_floor and
 * n_chunks as there) together with a bound on how far an FP32 evaluation of
 * the same iteration may land from it.  This is a parity tolerance, not part
 * of the method: the CUDA library evaluates the E-step of Eq. 15 in FP32 as
 *     l~ = fl(c_g) - 1/2 sum_d fl(x_d s_d - m_d)^2,  s = fl(1/sigma), m = fl(mu/sigma),
 * forms log p (Eq. 16) and l_{g,i} (Eq. 3) with FP32 exp/log, leaves out
 * responsibilities whose total per Gaussian is below `drop`, and sums
 * Eqs. 9-11 in FP32 about the FP32 start means f (at most n_acc additions into
 * any FP32 accumulator) before the FP64 reduce of Eqs. 12-14.
 * First-order bounds with u = 2^-24, from the exact FP64 quantities
 * t_d = (x_d - mu_d) / sigma_d and a_d = (|x_d| + |mu_d|) / sigma_d:
 *   logit   e_ig = u (|c_g| + |l_ig| + sum_d |t_d| a_d + (1 + D/2) sum_d t_d^2)
 *                  + 4 u^2 sum_d (a_d + |t_d|)^2
 *           (the last term is the square of the rounding of x s - mu s itself,
 *           one or two roundings of size u (a_d + |t_d|); it matters only when
 *           sigma is tiny against |x| + |mu|)
 *   log p   E_i = sum_h l_hi e_ih carried from the logits, and its own rounding
 *           r_i = sum_h l_hi u |l_ih - max_h l_ih| + (n_lse + 8) u + u |log p_i| + 2^-20 + G drop / N
 *           (n_lse: the longest chain of FP32 additions in the sum of Eq. 16)
 *   l_{g,i} relative error, since log l_{g,i} = l_ig - log p_i moves by
 *           (1 - l_gi) dl_ig - sum_{h != g} l_hi dl_ih plus the roundings:
 *           delta_ig = (E_i - l_gi e_ig) + (1 - l_gi) e_ig + r_i + u |l_ig - log p_i| + 2^-21
 * and, with rho = n_acc u, L_g, mu', v' the new parameters and R_gd the largest
 * |x_id - mu'_gd|:
 *   b_w[g]    = (sum_i l delta + drop + rho L_g) / N
 *   b_mu[g,d] = (sum_i l delta |x - mu'| + drop R + 2 rho sum_i l |x - f|) / L_g
 *   b_var[g,d]= (sum_i l delta |(x - mu')^2 - v'| + drop (R^2 + v')
 *                + 2 rho (sum_i l (x - f)^2 + 2 |mu' - f| sum_i l |x - f|)) / L_g
 * (the first terms are the first-order change of a weighted mean / variance
 * when each weight l_{g,i} moves by a relative delta_ig).  A Gaussian with
 * L_g == 0 gets zero bounds (its parameters are kept on both sides).
 * means/dcovs/hefts are updated in place; *mean_ll as in orc_em_iterate.
 */
int orc_em_fp32_budget(const float *X, int64_t N, int32_t D, int32_t G, double *means, double *dcovs,
                       double *hefts, double var_floor, int32_t n_chunks, int32_t n_acc, int32_t n_lse, double drop,
                       double *mean_ll, double *b_mu, double *b_var, double *b_w)
{
    if (N < 1 || D < 1 || G < 1 || n_chunks < 1 || n_acc < 1 || n_lse < 1 || !(drop >= 0.0)) return ORC_ERR_ARG;
    const double u = 1.0 / 16777216.0;
    size_t GD = (size_t)G * D;
    double *m0 = (double *)malloc(sizeof(double) * GD), *v0 = (double *)malloc(sizeof(double) * GD);
    double *h0 = (double *)malloc(sizeof(double) * (size_t)G);
    if (!m0 || !v0 || !h0) { free(m0); free(v0); free(h0); return ORC_ERR_OOM; }
    memcpy(m0, means, sizeof(double) * GD);
    memcpy(v0, dcovs, sizeof(double) * GD);
    memcpy(h0, hefts, sizeof(double) * (size_t)G);
    int rc = orc_em_one(X, N, D, G, means, dcovs, hefts, var_floor, n_chunks, mean_ll);
    if (rc != ORC_OK) { free(m0); free(v0); free(h0); return rc; }

    /* per Gaussian of the start: sigma_gd and the constant of Eq. 15 */
    double *sd = (double *)malloc(sizeof(double) * GD), *cst = (double *)malloc(sizeof(double) * (size_t)G);
    /* per chunk: Bw [G], Bm, Bv, Am, Av, R [G][D] */
    size_t per = (size_t)G + 5 * GD;
    double *acc = (double *)calloc((size_t)n_chunks * per, sizeof(double));
    if (!acc || !sd || !cst) { free(acc); free(sd); free(cst); free(m0); free(v0); free(h0); return ORC_ERR_OOM; }
    for (int32_t g = 0; g < G; ++g) {
        cst[g] = log(h0[g]) - 0.5 * (double)D * ORC_LOG_2PI;
        for (int32_t d = 0; d < D; ++d) {
            sd[(size_t)g * D + d] = sqrt(v0[(size_t)g * D + d]);
            cst[g] -= 0.5 * log(v0[(size_t)g * D + d]);
        }
    }
#ifdef _OPENMP
#pragma omp parallel for schedule(static, 1)
#endif
    for (int32_t t = 0; t < n_chunks; ++t) {
        int64_t i0 = (int64_t)((double)N * t / n_chunks);
        int64_t i1 = (int64_t)((double)N * (t + 1) / n_chunks);
        double *Bw = acc + (size_t)t * per, *Bm = Bw + G, *Bv = Bm + GD, *Am = Bv + GD, *Av = Am + GD, *R = Av + GD;
        double *l = (double *)malloc(sizeof(double) * (size_t)G);
        double *e = (double *)malloc(sizeof(double) * (size_t)G);
        for (int64_t i = i0; i < i1; ++i) {
            const float *x = X + (size_t)i * D;
            double mx = -INFINITY;
            for (int32_t g = 0; g < G; ++g) {
                const double *mu = m0 + (size_t)g * D, *sg = sd + (size_t)g * D;
                double t2 = 0.0, ta = 0.0, q2 = 0.0;
                for (int32_t d = 0; d < D; ++d) {
                    double td = ((double)x[d] - mu[d]) / sg[d];
                    double ad = (fabs((double)x[d]) + fabs(mu[d])) / sg[d];
                    t2 += td * td;
                    ta += fabs(td) * ad;
                    q2 += (ad + fabs(td)) * (ad + fabs(td));
                }
                l[g] = cst[g] - 0.5 * t2;                       /* Eq. 15 */
                e[g] = l[g] == -INFINITY ? 0.0
                                         : u * (fabs(cst[g]) + fabs(l[g]) + ta + (1.0 + 0.5 * (double)D) * t2) + 4.0 * u * u * q2;
                if (l[g] > mx) mx = l[g];
            }
            if (mx == -INFINITY) continue;
            double se = 0.0;
            for (int32_t g = 0; g < G; ++g) se += exp(l[g] - mx);
            const double lse = mx + log(se);                    /* Eq. 16 */
            /* E = sum_h l_h e_h (the logit errors carried into log p), rnd = the
             * rounding of log p itself */
            double E = 0.0, rnd = (double)(n_lse + 8) * u + u * fabs(lse) + 1.0 / 1048576.0 + (double)G * drop / (double)N;
            for (int32_t g = 0; g < G; ++g)
                if (l[g] > -INFINITY) {
                    const double gam = exp(l[g] - lse);
                    E += gam * e[g];
                    rnd += gam * u * fabs(l[g] - mx);
                }
            for (int32_t g = 0; g < G; ++g) {
                const double gam = exp(l[g] - lse);
                const double *mu1 = means + (size_t)g * D, *v1 = dcovs + (size_t)g * D;
                for (int32_t d = 0; d < D; ++d) {
                    double r = fabs((double)x[d] - mu1[d]);
                    if (r > R[(size_t)g * D + d]) R[(size_t)g * D + d] = r;
                }
                if (gam == 0.0) continue;
                /* log l_{g,i} = l_g - log p: its logit error enters with weight
                 * 1 - gam, the others' through log p */
                const double del = (E - gam * e[g]) + (1.0 - gam) * e[g] + rnd + u * fabs(l[g] - lse) + 1.0 / 2097152.0;
                const double gd = gam * del;
                Bw[g] += gd;
                for (int32_t d = 0; d < D; ++d) {
                    const double xd = (double)x[d];
                    const double r = xd - mu1[d];
                    const double q = xd - (double)(float)m0[(size_t)g * D + d];
                    Bm[(size_t)g * D + d] += gd * fabs(r);
                    Bv[(size_t)g * D + d] += gd * fabs(r * r - v1[d]);
                    Am[(size_t)g * D + d] += gam * fabs(q);
                    Av[(size_t)g * D + d] += gam * (q * q);
                }
            }
        }
        free(l);
        free(e);
    }
    /* reduce the chunks (R by maximum) and form the bounds */
    double *tot = (double *)calloc(per, sizeof(double));
    if (!tot) { free(acc); free(sd); free(cst); free(m0); free(v0); free(h0); return ORC_ERR_OOM; }
    for (int32_t t = 0; t < n_chunks; ++t) {
        const double *src = acc + (size_t)t * per;
        for (size_t k = 0; k < (size_t)G + 4 * GD; ++k) tot[k] += src[k];
        for (size_t k = (size_t)G + 4 * GD; k < per; ++k) if (src[k] > tot[k]) tot[k] = src[k];
    }
    const double *Bw = tot, *Bm = Bw + G, *Bv = Bm + GD, *Am = Bv + GD, *Av = Am + GD, *R = Av + GD;
    const double rho = (double)n_acc * u;
    for (int32_t g = 0; g < G; ++g) {
        const double L = hefts[g] * (double)N;
        b_w[g] = (Bw[g] + drop + rho * L) / (double)N;
        for (int32_t d = 0; d < D; ++d) {
            const size_t k = (size_t)g * D + d;
            if (!(L > 0.0)) { b_mu[k] = 0.0; b_var[k] = 0.0; continue; }
            const double sh = fabs(means[k] - (double)(float)m0[k]);
            b_mu[k] = (Bm[k] + drop * R[k] + 2.0 * rho * Am[k]) / L;
            b_var[k] = (Bv[k] + drop * (R[k] * R[k] + dcovs[k]) + 2.0 * rho * (Av[k] + 2.0 * sh * Am[k])) / L;
        }
    }
    free(tot); free(acc); free(sd); free(cst); free(m0); free(v0); free(h0);
    return ORC_OK;
}

/*
 * Per sample, a bound on how far an FP32 evaluation of log p(x_i) (Eq. 16
 * with the log-densities of Eq. 15 as the CUDA forms compute them) may land
 * from the FP64 value: E_i + r_i of orc_em_fp32_budget (first order, plus the
 * square of the rounding of x s - mu s).  A parity tolerance, not part of the
 * method.
 */
int orc_log_p_fp32_bound(const float *X, int64_t N, int32_t D, int32_t G, const double *means, const double *dcovs,
                         const double *hefts, int32_t n_lse, double *out)
{
    if (N < 0 || D < 1 || G < 1 || n_lse < 1) return ORC_ERR_ARG;
    const double u = 1.0 / 16777216.0;
    size_t GD = (size_t)G * D;
    double *sd = (double *)malloc(sizeof(double) * GD), *cst = (double *)malloc(sizeof(double) * (size_t)G);
    if (!sd || !cst) { free(sd); free(cst); return ORC_ERR_OOM; }
    for (int32_t g = 0; g < G; ++g) {
        cst[g] = log(hefts[g]) - 0.5 * (double)D * ORC_LOG_2PI;
        for (int32_t d = 0; d < D; ++d) {
            sd[(size_t)g * D + d] = sqrt(dcovs[(size_t)g * D + d]);
            cst[g] -= 0.5 * log(dcovs[(size_t)g * D + d]);
        }
    }
    int rc = ORC_OK;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < N; ++i) {
        const float *x = X + (size_t)i * D;
        double *l = (double *)malloc(sizeof(double) * (size_t)G), *e = (double *)malloc(sizeof(double) * (size_t)G);
        if (!l || !e) { free(l); free(e); rc = ORC_ERR_OOM; continue; }
        double mx = -INFINITY;
        for (int32_t g = 0; g < G; ++g) {
            const double *mu = means + (size_t)g * D, *sg = sd + (size_t)g * D;
            double t2 = 0.0, ta = 0.0, q2 = 0.0;
            for (int32_t d = 0; d < D; ++d) {
                double td = ((double)x[d] - mu[d]) / sg[d];
                double ad = (fabs((double)x[d]) + fabs(mu[d])) / sg[d];
                t2 += td * td;
                ta += fabs(td) * ad;
                q2 += (ad + fabs(td)) * (ad + fabs(td));
            }
            l[g] = cst[g] - 0.5 * t2;
            e[g] = l[g] == -INFINITY ? 0.0
                                     : u * (fabs(cst[g]) + fabs(l[g]) + ta + (1.0 + 0.5 * (double)D) * t2) + 4.0 * u * u * q2;
            if (l[g] > mx) mx = l[g];
        }
        double se = 0.0;
        for (int32_t g = 0; g < G; ++g) se += exp(l[g] - mx);
        const double lse = mx + log(se);
        double b = (double)(n_lse + 8) * u + u * fabs(lse) + 1.0 / 1048576.0;
        for (int32_t g = 0; g < G; ++g)
            if (l[g] > -INFINITY) b += exp(l[g] - lse) * (e[g] + u * fabs(l[g] - mx));
        out[i] = b;
        free(l);
        free(e);
    }
    free(sd);
    free(cst);
    return rc;
}

/*
 * assign(X, dist_mode) (Sec. 4.1): eucl (mode 0) = nearest mean in squared
 * Euclidean distance; prob (mode 2) = the Gaussian with the largest
 * log(w_g N(x|g)) (the "inverse likelihood" distance).  Lowest index on ties.
 */
int orc_assign(const float *X, int64_t N, int32_t D, int32_t G, const double *means,
               const double *dcovs, const double *hefts, int32_t mode, int32_t *out)
{
    if (mode == 0) {
        double *w = (double *)malloc(sizeof(double) * (size_t)D);
        if (!w) return ORC_ERR_OOM;
        for (int32_t d = 0; d < D; ++d) w[d] = 1.0;
        orc_km_assign(X, N, D, G, means, w, out, NULL, NULL);
        free(w);
        return ORC_OK;
    }
    if (mode != 2) return ORC_ERR_ARG;
    double *t = (double *)malloc(sizeof(double) * (size_t)G);
    if (!t) return ORC_ERR_OOM;
    for (int64_t i = 0; i < N; ++i) {
        orc_log_terms(X + (size_t)i * D, D, G, means, dcovs, hefts, t);
        int32_t best = 0;
        for (int32_t g = 1; g < G; ++g) if (t[g] > t[best]) best = g;
        out[i] = best;
    }
    free(t);
    return ORC_OK;
}

/*
 * learn(data, n_gaus, dist_mode, seed_mode, km_iter, em_iter, var_floor)
 * (Sec. 4.1).  dist_mode: 0 eucl, 1 maha.  seed_mode: 0 keep_existing (the
 * given means/dcovs/hefts are the start), 1 random_subset (seed), 2
 * static_subset, 3 static_spread, 4 random_spread (seed).
 * Flow: global statistics (Mahalanobis weights, floored) -> seeds -> k-means
 * (if km_iter > 0) -> EM (em_iter iterations).  With km_iter == 0 and
 * random_subset the start is the plain initialisation of Sec. 3 first
 * paragraph: means = the seed samples, unit covariances, uniform hefts.
 */
int orc_learn(const float *X, int64_t N, int32_t D, int32_t G, int32_t dist_mode,
              int32_t seed_mode, uint64_t seed, int32_t km_iter, int32_t em_iter,
              double var_floor, double em_tol, int32_t n_chunks, double *means,
              double *dcovs, double *hefts, double *ll_hist, int32_t *n_em_done)
{
    if (N < 1 || D < 1 || G < 1 || (int64_t)G > N || km_iter < 0 || em_iter < 0 ||
        !(var_floor >= 0.0) || (dist_mode != 0 && dist_mode != 1) ||
        seed_mode < 0 || seed_mode > 4)
        return ORC_ERR_ARG;
    double *gm = (double *)malloc(sizeof(double) * D), *gv = (double *)malloc(sizeof(double) * D);
    double *w = (double *)malloc(sizeof(double) * D);
    if (!gm || !gv || !w) { free(gm); free(gv); free(w); return ORC_ERR_OOM; }
    orc_global_stats(X, N, D, gm, gv);
    for (int32_t d = 0; d < D; ++d) {
        gv[d] = gv[d] > var_floor ? gv[d] : var_floor;
        w[d] = dist_mode == 1 ? 1.0 / gv[d] : 1.0;
    }
    int rc = ORC_OK;
    if (seed_mode != 0) {
        int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * G);
        if (!idx) { free(gm); free(gv); free(w); return ORC_ERR_OOM; }
        if (seed_mode == 1) rc = orc_seed_random_subset(N, G, seed, idx);
        else if (seed_mode == 2) rc = orc_seed_static_subset(N, G, idx);
        else {
            int64_t first = 0;   /* static_spread: sample 0; random_spread: random_subset's first draw */
            if (seed_mode == 4) rc = orc_seed_random_subset(N, 1, seed, &first);
            if (rc == ORC_OK) rc = orc_seed_spread(X, N, D, G, w, first, idx);
        }
        for (int32_t g = 0; g < G && rc == ORC_OK; ++g) {
            for (int32_t d = 0; d < D; ++d) {
                means[(size_t)g * D + d] = (double)X[(size_t)idx[g] * D + d];
                dcovs[(size_t)g * D + d] = 1.0;
            }
            hefts[g] = 1.0 / (double)G;
        }
        free(idx);
    }
    if (rc == ORC_OK && km_iter > 0)
        rc = orc_kmeans(X, N, D, G, w, gv, means, dcovs, hefts, km_iter, var_floor, NULL);
    if (rc == ORC_OK && em_iter > 0)
        rc = orc_em_iterate(X, N, D, G, means, dcovs, hefts, em_iter, var_floor, em_tol,
                            n_chunks, ll_hist, n_em_done);
    else if (n_em_done)
        *n_em_done = 0;
    free(gm); free(gv); free(w);
    return rc;
}

/* Host threads of the OpenMP MapReduce loops (only the CPU-baseline timing
 * changes it; results do not depend on it beyond the order of chunk sums). */
void orc_set_threads(int32_t n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* generate (Sec. 4.1, M.generate(N)): N random samples of the model.       */
/* Reading (the paper gives no generator): uniforms from SplitMix64 used as  */
/* a counter-based generator -- output k for seed s is the SplitMix64 mix of */
/* s + (k + 1) * 0x9e3779b97f4a7c15, i.e. the k-th output of a generator     */
/* started at state s -- as u = ((r >> 11) + 0.5) 2^-53 in (0, 1).  Sample i */
/* uses outputs i*K .. i*K + K - 1, K = 1 + 2 ceil(D / 2): the first picks  */
/* the Gaussian (the first g with u < cumulative heft / total heft, else the */
/* last), then pairs (u1, u2) give Box-Muller normals sqrt(-2 ln u1) (cos,   */
/* sin)(2 pi u2) for dimensions 2j, 2j+1; x = mean + sqrt(dcov) z, stored as */
/* float.                                                                    */
/* ------------------------------------------------------------------------ */
static double orc_counter_uniform(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    z ^= z >> 31;
    return ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

int orc_generate(const double *means, const double *dcovs, const double *hefts, int32_t G, int32_t D,
                 int64_t N, uint64_t seed, float *out, int32_t *labels)
{
    if (G < 1 || D < 1 || N < 0) return ORC_ERR_ARG;
    double tot = 0.0;
    for (int32_t g = 0; g < G; ++g) tot += hefts[g];
    const int64_t K = 1 + 2 * (int64_t)((D + 1) / 2);
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t i = 0; i < N; ++i) {
        const uint64_t k0 = (uint64_t)(i * K);
        const double u = orc_counter_uniform(seed, k0);
        int32_t lab = G - 1;
        double c = 0.0;
        for (int32_t g = 0; g < G; ++g) {
            c += hefts[g];
            if (u < c / tot) { lab = g; break; }
        }
        if (labels) labels[i] = lab;
        for (int32_t j = 0; 2 * j < D; ++j) {
            const double u1 = orc_counter_uniform(seed, k0 + 1 + 2 * (uint64_t)j);
            const double u2 = orc_counter_uniform(seed, k0 + 2 + 2 * (uint64_t)j);
            const double r = sqrt(-2.0 * log(u1));
            for (int32_t h = 0; h < 2 && 2 * j + h < D; ++h) {
                const int32_t d = 2 * j + h;
                const double z = r * (h == 0 ? cos(two_pi * u2) : sin(two_pi * u2));
                out[(size_t)i * D + d] = (float)(means[(size_t)lab * D + d] + sqrt(dcovs[(size_t)lab * D + d]) * z);
            }
        }
    }
    return ORC_OK;
}
