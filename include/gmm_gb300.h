/*
 * gmm_gb300.h -- C ABI of the GB300 (sm_103a) library for training and using
 * diagonal-covariance Gaussian mixture models by k-means + EM, following
 * arXiv 1707.09094 ("An Open Source C++ Implementation of Multi-Threaded
 * Gaussian Mixture Models, k-Means and Expectation Maximisation").
 *
 * Layouts (all row-major, C order):
 *   X      const float  [N][D]   one sample per row.  The paper stores one
 *                                sample per column of a D x N matrix; the
 *                                bytes in memory are identical.
 *   means  double [G][D]         the paper's `means`, one Gaussian per row
 *   dcovs  double [G][D]         diagonal covariances, one Gaussian per row
 *   hefts  double [G]            mixture weights (Eq. 1, sum to one)
 *
 * Pointers: every X / out argument may be a host pointer or a device pointer
 * of the current CUDA device; the library tells them apart with
 * cudaPointerGetAttributes.  Host inputs are copied to a device staging area
 * owned by the model; host outputs are written after a device->host copy.
 * The caller owns every buffer it passes; the library keeps no caller pointer
 * after a call returns.  A model owns its parameters and workspace (device
 * memory) until gmm_destroy.
 *
 * Errors: every call returns a gmm_status; 0 is success (the paper's `learn`
 * returns a bool, Sec. 4.1).  gmm_last_error() gives a thread-local message.
 * On failure a model keeps the last valid parameters.  Calls on one model
 * are not thread-safe; distinct models are independent.
 *
 * Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).
 * Calls return after the work they queued has finished (they synchronise the
 * stream), so host outputs are valid on return.
 */
#ifndef GMM_GB300_H
#define GMM_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gmm_model gmm_model;

typedef enum {
    GMM_OK = 0,
    GMM_ERR_ARG = -1,         /* invalid argument or shape                    */
    GMM_ERR_NONFINITE = -2,   /* a NaN/Inf appeared (e.g. in X); model kept   */
    GMM_ERR_CUDA = -3,        /* a CUDA call failed                           */
    GMM_ERR_TIMEOUT = -4,     /* a bounded device wait gave up                */
    GMM_ERR_OOM = -5,         /* device or host allocation failed             */
    GMM_ERR_STATE = -6,       /* model has no parameters / shape mismatch     */
    GMM_ERR_UNSUPPORTED = -7  /* shape outside what the kernels handle        */
} gmm_status;

/* Distances (Sec. 3.1, Sec. 4.1 `dist_mode`): EUCL squared Euclidean, MAHA
 * squared Mahalanobis with a global diagonal covariance (Eq. 20), PROB the
 * "probabilistic distance" of `assign` (largest log w_g N(x|g)). */
typedef enum { GMM_EUCL = 0, GMM_MAHA = 1, GMM_PROB = 2 } gmm_dist;

/* Seeding (Sec. 4.1 `seed_mode`): KEEP_EXISTING starts from the model's
 * parameters; RANDOM_SUBSET takes n_gaus distinct random samples as means
 * (SplitMix64(seed) driving a partial Fisher-Yates shuffle of 0..N-1);
 * STATIC_SUBSET the samples floor(g N / n_gaus) (repeatable); STATIC_SPREAD
 * and RANDOM_SPREAD a maximally spread subset: greedy farthest-first under the
 * k-means distance (dist), lowest index on ties, starting at sample 0 or at
 * RANDOM_SUBSET's first draw for `seed` (N_G passes over X, FP64 distances).
 * With km_iter = 0 the seeds are the means, with unit variances and uniform
 * hefts. */
typedef enum {
    GMM_KEEP_EXISTING = 0,
    GMM_RANDOM_SUBSET = 1,
    GMM_STATIC_SUBSET = 2,
    GMM_STATIC_SPREAD = 3,
    GMM_RANDOM_SPREAD = 4
} gmm_seed;

/* Arithmetic of the E-step log-density (Eq. 15) in the fused EM pass.
 *   FP32   CUDA cores: direct sum of (x - mu)^2 / sigma^2 for every (sample,
 *          Gaussian), log-sum-exp, M-step (FP32 sums shifted by the
 *          iteration's means, reduced in FP64) over the Gaussians holding a
 *          responsibility >= 1e-9 / N somewhere in a 32-sample tile.
 *   BF16   tcgen05 tensor cores: the expanded log-density (x'^2 and x' blocks,
 *          data centred by the global mean) with FP32 accumulation screens
 *          every Gaussian with a rigorous rounding bound; the Gaussians that
 *          can hold a responsibility >= 1e-9 / N are recomputed exactly in
 *          FP32, and those whose exact responsibility reaches 1e-9 / N enter
 *          log-sum-exp and the M-step.  (For every Gaussian the
 *          responsibility left out sums to less than 1e-9.)  D <= 64 and
 *          n_gaus <= 256: BF16 operands, all Gaussians in one tile.  Up to
 *          D = 128 and n_gaus = 4096: operands split into BF16 hi + lo parts
 *          (three products), blocks of 128 Gaussians; a sample with more
 *          than 64 candidates is evaluated by the register-blocked FP32
 *          kernels instead.
 * Sufficient statistics are reduced in FP64 in every mode.  There is no TF32
 * E-step, and no E-step that uses a reduced-precision contraction directly:
 * that loses ~2^-9 (BF16), ~2^-11 (TF32) or ~2^-16 (split BF16) of terms that
 * reach 10^3-10^4 nats when a Gaussian's mean lies many of its standard
 * deviations from the global centre, far more than the FP32 form's
 * responsibilities allow; as a screen the bound only widens the candidate
 * set. */
typedef enum { GMM_FP32 = 0, GMM_BF16 = 1 } gmm_prec;

typedef struct {
    int32_t dist;       /* gmm_dist for seeding/k-means: EUCL or MAHA (default MAHA) */
    int32_t seed_mode;  /* gmm_seed (default RANDOM_SUBSET)                           */
    uint64_t seed;      /* RNG seed for RANDOM_SUBSET (default 0)                     */
    double em_tol;      /* > 0: stop EM once the mean log-likelihood gains < em_tol   */
    int32_t prec;       /* gmm_prec of the EM E-step (default FP32)                   */
    int32_t print;      /* non-zero: print per-iteration progress to stderr           */
    void *stream;       /* cudaStream_t, NULL = default stream                        */
} gmm_learn_opts;

/* Per-call limits of the kernels: D <= GMM_MAX_DIMS everywhere.  The FP32
 * EM form runs one fused pass when its per-CTA statistics (4 n_gaus (2D+1)
 * bytes plus tile buffers) fit in shared memory and n_gaus <= 128, and
 * otherwise the register-blocked two-phase form.  The tensor-core EM pass
 * needs n_gaus <= 4096 (else GMM_ERR_UNSUPPORTED). */
#define GMM_MAX_DIMS 128

/* Create an empty model (no parameters) on the current CUDA device. */
gmm_status gmm_create(gmm_model **out);

/* Free a model and everything it owns.  NULL is ignored. */
void gmm_destroy(gmm_model *m);

/* Fill *o with the defaults listed in gmm_learn_opts. */
void gmm_default_opts(gmm_learn_opts *o);

/*
 * learn(data, n_gaus, dist_mode, seed_mode, km_iter, em_iter, var_floor,
 * print_mode) of Sec. 4.1.  Steps: global per-dimension mean and variance of
 * X (Eq. 20's global covariance, also the centring used by the tensor-core
 * forms); seeding; km_iter iterations of k-means (Sec. 3, Eq. 19; dead means
 * resurrected from the most popular mean's samples, Sec. 3.1), whose last
 * iteration's hard statistics give the first hefts/means/dcovs (Eqs. 5-7 with
 * Eq. 19); then em_iter EM iterations (Eqs. 3-14 in the log domain,
 * Eqs. 15-18), each one fused data pass plus an FP64 reduce/update, with the
 * variance floor applied after every iteration (Sec. 2.2).  With km_iter == 0
 * and RANDOM_SUBSET the start is means = seeds, dcovs = 1, hefts = 1/n_gaus
 * (Sec. 3, first paragraph).  opts NULL = defaults.
 * X: [N][D] host or device.  Requires 1 <= n_gaus <= N, 1 <= D <= 128,
 * var_floor >= 0 and finite; KEEP_EXISTING requires parameters of shape
 * (n_gaus, D).  GMM_ERR_NONFINITE if an update produced NaN/Inf (the model
 * keeps the last finite parameters).
 */
gmm_status gmm_learn(gmm_model *m, const float *X, int64_t N, int32_t D, int32_t n_gaus,
                     int32_t km_iter, int32_t em_iter, double var_floor,
                     const gmm_learn_opts *opts);

/*
 * n_iter EM iterations (Sec. 2 / 2.1) from the model's current parameters on
 * X, i.e. learn() with KEEP_EXISTING and km_iter = 0 without recomputing the
 * global statistics when X is the data the model last learned on (the
 * tensor-core forms centre the data by the stored global mean; pass
 * recompute_center != 0 for new data).  Appends to the log-likelihood
 * history read by gmm_get_stats.  This is the call the EM throughput
 * benchmark times.
 */
gmm_status gmm_em_iterate(gmm_model *m, const float *X, int64_t N, int32_t n_iter,
                          double var_floor, int32_t prec, int32_t recompute_center,
                          void *stream);

/*
 * k-means (Sec. 3) alone: from the model's current means (KEEP_EXISTING) run
 * km_iter iterations with distance `dist` (EUCL or MAHA; MAHA weights come
 * from the global variance of X, floored by var_floor); on return the model
 * holds the hard-statistics estimate (hefts, means, dcovs) of the last
 * iteration and, if assign_out != NULL, assign_out[N] (int32, host or device)
 * receives that iteration's assignments (Eq. 19, lowest index on exact ties).
 */
gmm_status gmm_kmeans(gmm_model *m, const float *X, int64_t N, int32_t km_iter, int32_t dist,
                      double var_floor, int32_t *assign_out, void *stream);

/*
 * Batched learn(): n_fits independent fits (their own X, N, D, n_gaus) with
 * the same km_iter, em_iter, var_floor and opts, run as one CUDA graph whose
 * data passes are persistent kernels over a work list of (fit, sample chunk)
 * items (Sec. 2.1's chunks, scheduled largest first across all fits).  Fit f
 * seeds with random_subset from opts->seed + f; arithmetic is the FP32 form
 * with FP64 reductions, so each fit matches gmm_learn on its own data.  The
 * chunk size and CTAs per SM of the EM pass are picked by an autotuner per
 * shape bucket (timed on the first batch of that bucket; kept in memory and,
 * if the environment variable GMM_AUTOTUNE_CACHE names a file, there).
 * Requires 1 <= D <= 64 and 1 <= n_gaus <= min(N, 128) per fit; opts->prec
 * must be GMM_FP32 and opts->seed_mode GMM_RANDOM_SUBSET.  X[f] may be host
 * or device memory.  On return models[f] holds fit f's parameters and history.
 */
gmm_status gmm_learn_batched(gmm_model *const *models, int32_t n_fits, const float *const *X, const int64_t *N,
                             const int32_t *D, const int32_t *n_gaus, int32_t km_iter, int32_t em_iter,
                             double var_floor, const gmm_learn_opts *opts);

/*
 * log_p(X) / log_p(X, g) of Sec. 4.1: out[i] = log p(x_i | lambda) (Eq. 16)
 * for g = -1, or log N(x_i | mu_g, Sigma_g) (Eq. 15, without the heft) for
 * 0 <= g < n_gaus.  out: double [N], host or device.
 */
gmm_status gmm_log_p(const gmm_model *m, const float *X, int64_t N, int32_t g, double *out,
                     void *stream);

/* avg_log_p(X[, g]) of Sec. 4.1: *out (host double) = mean over i of log_p. */
gmm_status gmm_avg_log_p(const gmm_model *m, const float *X, int64_t N, int32_t g, double *out,
                         void *stream);

/*
 * gmm_avg_log_p_noalloc: the same value as gmm_avg_log_p (mean of log_p over
 * X) for callers that must not allocate device memory.  The paper has no
 * counterpart: it exists for code that cannot call cudaMalloc at the moment
 * it needs the number -- for example inside a framework whose caching
 * allocator already holds all free device memory (a cudaMalloc would fail or
 * force the framework to release its cache), or in a service that fixes its
 * memory footprint up front.  gmm_avg_log_p stages a per-sample
 * buffer of N doubles in the model; this entry point instead reduces per
 * 128-sample block into a fixed array of 65537 doubles (512 KiB) compiled
 * into the library, which every GPU that loads the library keeps until the
 * process exits.  It allocates nothing and calls no allocating routine.
 *   X    device pointer, float [N][D] (host pointers are rejected: staging
 *        them would need an allocation); 1 <= N <= 8,388,608, larger N
 *        returns GMM_ERR_UNSUPPORTED.
 *   out  host double, written on return (the call synchronises `stream`).
 * The first call on each device looks up the device address of the array
 * (cudaGetSymbolAddress, with that device current) and keeps it for the
 * life of the process.  A
 * cudaDeviceReset (or any other teardown of the device's primary context)
 * invalidates the kept address: this entry point must not be called after
 * one.  All calls share the array and every call
 * overwrites the slots it reads, so nothing needs clearing; calls whose
 * kernels overlap on the GPU (concurrent streams or threads) race on it and
 * must be serialised by the caller.
 */
gmm_status gmm_avg_log_p_noalloc(const gmm_model *m, const float *X, int64_t N, int32_t g, double *out,
                                 void *stream);

/*
 * assign(X, dist_mode) of Sec. 4.1: out[i] (int32 [N], host or device) = the
 * closest Gaussian.  EUCL: argmin ||x - mu_g||^2 (exact: FP32 with an FP64
 * recheck of near ties); PROB: argmax log(w_g N(x|g)) in FP32.  Lowest index
 * on ties.
 */
gmm_status gmm_assign(const gmm_model *m, const float *X, int64_t N, int32_t mode, int32_t *out,
                      void *stream);

/* raw_hist / norm_hist of Sec. 4.1: counts (int64 [n_gaus]) or normalised
 * counts (double [n_gaus]) of assign(X, mode); host pointers. */
gmm_status gmm_raw_hist(const gmm_model *m, const float *X, int64_t N, int32_t mode,
                        int64_t *counts, void *stream);
gmm_status gmm_norm_hist(const gmm_model *m, const float *X, int64_t N, int32_t mode,
                         double *hist, void *stream);

/*
 * Learned initialiser (a set encoder trained on the plain method's fits).
 * Network: per point D -> point_layers x hidden_point (ReLU), mean-pool over
 * the P points, head_layers x hidden_head (ReLU), linear to n_gaus (1 + 2D)
 * outputs: softmax -> hefts, means, exp(.) + var_floor -> dcovs.  All
 * products run in BF16 with FP32 accumulation (FP32 master weights, Adam).
 * Loss of a set: the mean negative log-likelihood of its points under the
 * predicted mixture (Eqs. 1, 16), plus lambda * sum_k w~_k min_g
 * sum_d (m_gd - m~_kd)^2 / v~_kd pulling the predicted means to the plain
 * method's fit (w~, m~, v~) when targets are given.
 */
typedef struct gmm_init_net gmm_init_net;

/* D <= 64, n_gaus <= 64; weights drawn from SplitMix64(seed). */
gmm_status gmm_init_net_create(gmm_init_net **out, int32_t D, int32_t n_gaus, int32_t hidden_point,
                               int32_t hidden_head, int32_t point_layers, int32_t head_layers, uint64_t seed);
void gmm_init_net_destroy(gmm_init_net *n);
int64_t gmm_init_net_num_params(const gmm_init_net *n);

/* Copy the FP32 weights and/or the last gradients to host arrays (NULL = skip);
 * layout: per layer W [out][in] then b [out], layers in order. */
gmm_status gmm_init_net_get_weights(const gmm_init_net *n, float *weights, float *grads);
gmm_status gmm_init_net_set_weights(gmm_init_net *n, const float *weights);

/* Training checkpoint: Adam's first and second moments (host float arrays of
 * num_params, the weights' layout; NULL = skip on get) and its step count
 * (the bias corrections use it).  With the weights, this resumes training
 * where it stopped.  GMM_ERR_ARG for NULL pointers (set) or step < 0. */
gmm_status gmm_init_net_get_adam(const gmm_init_net *n, float *m1, float *m2, int64_t *step);
gmm_status gmm_init_net_set_adam(gmm_init_net *n, const float *m1, const float *m2, int64_t step);

/*
 * One pass over a batch of B sets of P points (pts: device float [B][P][D]).
 * mode 0: forward + loss; 1: also gradients; 2: also one Adam step (lr).
 * Targets (device double [B][n_gaus][D], [B][n_gaus][D], [B][n_gaus]) are
 * needed when lambda > 0.  pred_* (device, may be NULL) receive the predicted
 * parameters; *loss (host) the batch-mean loss.
 */
gmm_status gmm_init_net_step(gmm_init_net *n, const float *pts, int32_t B, int32_t P, const double *tgt_means,
                             const double *tgt_dcovs, const double *tgt_hefts, double lambda, double var_floor,
                             int32_t mode, double lr, double *pred_means, double *pred_dcovs, double *pred_hefts,
                             double *loss, void *stream);

/* Seed model m for EM from P random samples of X (SplitMix64(seed) subset):
 * the network's predicted hefts, means and dcovs become m's parameters.
 * GMM_ERR_NONFINITE if the prediction is not finite (callers fall back to
 * k-means seeding). */
gmm_status gmm_init_net_seed_model(const gmm_init_net *n, gmm_model *m, const float *X, int64_t N, int32_t P,
                                   uint64_t seed, double var_floor, void *stream);

/* generate (Sec. 4.1, M.generate(N)): N random samples of the model into out
 * (float [N][D], host or device pointer, owned by the caller).  Sample i
 * takes SplitMix64 outputs i*K .. i*K + K - 1 of a generator started at
 * state `seed` (K = 1 + 2 ceil(D/2); output k is computed directly from
 * seed + (k+1) * 0x9e3779b97f4a7c15, so samples are independent of N and of
 * the launch): the first picks the Gaussian by its heft (inverse CDF), pairs
 * give Box-Muller normals; x = mean + sqrt(dcov) z.  Errors: GMM_ERR_STATE
 * without parameters, GMM_ERR_ARG for N < 0 or out == NULL with N > 0. */
gmm_status gmm_generate(const gmm_model *m, int64_t N, uint64_t seed, float *out, void *stream);

/* FP64 sample data (the double-precision input of the paper's gmm_diag,
 * Sec. 4.1).  The library computes on FP32 samples: gmm_x_from_f64 rounds
 * X64[0..count) to the nearest FP32 values (ties to even) into X32[0..count),
 * on `stream` (NULL = the default stream), and X32 is then passed to any call
 * that takes X.  Both pointers are device memory owned by the caller; a host
 * array is converted on the host instead.  Values beyond the FP32 range become
 * +-inf, which the calls that take X report as GMM_ERR_NONFINITE.
 * GMM_ERR_ARG for count < 0, a NULL or host pointer (count > 0). */
gmm_status gmm_x_from_f64(const double *X64, int64_t count, float *X32, void *stream);

/* save / load (Sec. 4.1, M.save / M.load): the model's parameters in a file
 * of this library's format -- 8 bytes "GMMDIAG1", int32 D, int32 n_gaus
 * (little-endian), then FP64 means [n_gaus][D], dcovs [n_gaus][D], hefts
 * [n_gaus].  load checks the header, the sizes, and that every value is
 * finite, every dcov > 0 and every heft >= 0; on any failure the model is
 * unchanged and GMM_ERR_ARG is returned (the paper's `false`). */
gmm_status gmm_save(const gmm_model *m, const char *path);
gmm_status gmm_load(gmm_model *m, const char *path);

/* Read the parameters (host pointers; any may be NULL).  D / n_gaus receive
 * the shape.  GMM_ERR_STATE if the model has none. */
gmm_status gmm_get_params(const gmm_model *m, int32_t *D, int32_t *n_gaus, double *means,
                          double *dcovs, double *hefts);

/* set_params of Sec. 4.1 (host pointers): the shape may differ from the
 * model's.  Requires dcovs > 0, hefts >= 0 (not renormalised). */
gmm_status gmm_set_params(gmm_model *m, int32_t D, int32_t n_gaus, const double *means,
                          const double *dcovs, const double *hefts);

/* Per-EM-iteration mean log-likelihood of the parameters each E-step used
 * (host double ll_hist[cap]); *n receives how many are stored (up to cap). */
gmm_status gmm_get_stats(const gmm_model *m, double *ll_hist, int32_t cap, int32_t *n);

/* Measurement hooks (no counterpart in the paper).  gmm_profile(m, 1)
 * resets the counters and makes later calls on m record CUDA events, on the
 * stream the kernels are launched on, around every launch of the fused data
 * pass (EM or k-means); gmm_profile(m, 0) stops recording.
 * gmm_profile_read returns the summed device time of those launches (ms),
 * their number, and the number of library kernels launched since the reset.
 * Any output pointer may be NULL. */
gmm_status gmm_profile(gmm_model *m, int32_t enable);
gmm_status gmm_profile_read(const gmm_model *m, double *pass_ms, int64_t *pass_launches,
                            int64_t *kernel_launches);

/* Failure-detection test hooks (no counterpart in the paper).
 *   GMM_DEBUG_WAIT_CYCLES  (value > 0) budget, in SM clock cycles, of every
 *                          bounded wait inside the tensor-core pass (default
 *                          2e9, about one second); 0 restores the default.
 *   GMM_DEBUG_SKIP_MMA     value != 0 makes the tensor-core pass issue no
 *                          MMA, so its epilogue waits for data that never
 *                          arrives: the wait runs out, the pass records
 *                          GMM_ERR_TIMEOUT, frees its tensor memory and the
 *                          call returns GMM_ERR_TIMEOUT with the model kept.
 * Used by the test-suite only. */
#define GMM_DEBUG_WAIT_CYCLES 1
#define GMM_DEBUG_SKIP_MMA 2
/*   GMM_DEBUG_KM_FORM      0 (default): k-means assigns on the tensor cores
 *                          where D <= 64 and N_G <= 256 (same assignments:
 *                          both forms decide the nearest mean exactly);
 *                          1: on the CUDA cores. */
#define GMM_DEBUG_KM_FORM 3
/*   GMM_DEBUG_FP32_FORM    0 (default): the FP32 EM pass runs the one-pass
 *                          form for N_G <= 128 where all N_G operands and
 *                          statistics fit in one CTA's shared memory, else
 *                          the register-blocked two-phase form; 1: the
 *                          one-pass form wherever it fits; 2: the
 *                          register-blocked form for every shape; 3: the
 *                          same with the log-densities recomputed in the
 *                          second phase instead of recorded in the first
 *                          (the same results to FP32 rounding). */
#define GMM_DEBUG_FP32_FORM 4
/*   GMM_DEBUG_TC_FORM      0 (default): the BF16 EM pass runs the one-tile
 *                          tensor-core form for D <= 64 and N_G <= 256, else
 *                          the blocked split-BF16 form; 1: the blocked form
 *                          for every shape it supports (the same results to
 *                          FP32 rounding). */
#define GMM_DEBUG_TC_FORM 5
gmm_status gmm_debug_set(gmm_model *m, int32_t key, int64_t value);

/* Screening counters of the tensor-core pass, summed since the last
 * gmm_profile(m, 1): GMM_STAT_SCREENED samples screened, GMM_STAT_KEPT
 * (sample, Gaussian) pairs kept for the exact recompute, GMM_STAT_DENSE
 * (sample, half of the Gaussians) lists that overflowed (exact pass over
 * every Gaussian of the half). */
#define GMM_STAT_SCREENED 3
#define GMM_STAT_KEPT 4
#define GMM_STAT_DENSE 5
/* GMM_STAT_PHASE0 + k (k = 0..7): SM cycles one epilogue thread of each CTA
 * of the screening kernel spent in phase k of a tile (0 building the next
 * tile's BF16 operand, 1 barrier, 2 MMA wait, 3 lower bounds (first read of
 * the accumulators), 4 upper bounds and candidate masks (second read) and the
 * records; 5-7 unused), summed over CTAs. */
#define GMM_STAT_PHASE0 6
/* Tensor-core k-means, summed over its passes: GMM_STAT_KM_SCREENED samples
 * screened, GMM_STAT_KM_DEFERRED samples the screen left with more than one
 * candidate (decided by exact FP32 distances), GMM_STAT_KM_FP64 samples
 * re-decided in FP64. */
#define GMM_STAT_KM_SCREENED 14
#define GMM_STAT_KM_DEFERRED 15
#define GMM_STAT_KM_FP64 16
gmm_status gmm_debug_get(const gmm_model *m, int32_t key, int64_t *value);

/* Thread-local text of the last error ("" if none). */
const char *gmm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GMM_GB300_H */
