// Internal declarations shared by the CUDA translation units of the library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "gmm_gb300.h"

namespace gmm {

constexpr double kLog2Pi = 1.83787706640934548356065947281123527;
constexpr int kRecSlots = 64;   // kept responsibilities per sample record (record M-step)

// Device-side status block, one per model.  Kernels never trap: they record
// what went wrong here and return, and the host reads it after the stream
// has drained.
struct DevStatus {
    int32_t code;        // 0 ok, else a gmm_status
    int32_t halt;        // set on error: later kernels of the same call no-op
    int32_t stop_after;  // last EM iteration to run (em_tol convergence)
    int32_t n_done;      // EM iterations completed
    int32_t fail_iter;   // iteration that produced a non-finite value
    int32_t n_dead;      // dead means seen by the last k-means iteration
    int32_t pad[2];
};

// Operands of the E-step derived from lambda (written by the prep/finalize
// kernels, read by the fused passes and the inference kernels).
struct Operands {
    float2 *sm;          // [G][D]  (s, mu*s) with s = 1/sqrt(sigma^2)      (FP32 form)
    float *mu;           // [G][D]  FP32 copy of the means: shift of the FP32 M-step
    float *c;            // [G]     log w - D/2 log 2pi - 1/2 sum log sigma^2
    float *c0;           // [G]     same without log w  (log_p(X, g))
    __nv_bfloat16 *B;    // [G][128] tensor-core E operand, K-major
    float *ctc;          // [G]     constant of the centred tensor-core logits
    float *q;            // [G]     sum_d mu'^2 / sigma^2 (centred), for the screening bound
    int32_t KP;          // K of the tensor-core operand: two 64-wide blocks (x'^2 half, x' half)
};

struct EmPassArgs {
    const float *X;
    int64_t N;
    int32_t D, G;
    Operands op;
    const float *center;     // [D] FP32 global mean (tensor-core centring)
    double *partial;         // [grid][G][1+2D]
    double *ll_partial;      // [grid]
    DevStatus *status;
    int32_t iter;
    long long wait_cycles;   // budget of bounded waits (tensor-core pass)
    int32_t skip_mma;        // test hook: issue no MMA
    unsigned long long *screen_stats;   // [3] screened, kept, dense (NULL = off)
    int64_t N_total;         // samples of the whole iteration (N of one chunk when X arrives in chunks)
};

struct EmFinalizeArgs {
    const double *partial;
    const double *ll_partial;
    int32_t n_partial;       // partials of the statistics
    int32_t n_ll_partial;    // partials of the log-likelihood
    int64_t N;
    int32_t D, G;
    const double *par_in;    // [G*D means | G*D dcovs | G hefts]
    double *par_out;
    double var_floor;
    int32_t shift_mode;      // reserved (0): the statistics are shifted by the FP32 means op.mu
    Operands op;
    const float *center;
    DevStatus *status;
    int32_t iter;
    double em_tol;
    double *ll_hist;         // device history
    int32_t build_tc;        // also build the tensor-core operands
};

// Count of library kernels launched (process-wide, all models).
void count_launches(int n);
long long launches_total();

// ---- launchers implemented in gmm_simt.cu
cudaError_t launch_global_stats(const float *X, int64_t N, int32_t D, double var_floor, int32_t dist,
                                double *partial, int32_t grid, double *gmean, double *gvar_floored,
                                double *wdist, float *sw, float *center, cudaStream_t s);
cudaError_t launch_gather_seeds(const float *X, int32_t D, int32_t G, const int64_t *idx,
                                double *par, cudaStream_t s);
// tiled CUDA-core k-means map step (km_tile_supported shapes: D <= 64, N_G <= 256)
bool km_tile_supported(int32_t D, int32_t G);
cudaError_t launch_km_pass(const float *X, int64_t N, int32_t D, int32_t G, const double *par,
                           const double *wdist, const float *sw, double *partial, int32_t grid, int32_t *assign,
                           DevStatus *status, cudaStream_t s);
cudaError_t launch_km_finalize(const double *partial, int32_t n_partial, int64_t N, int32_t D,
                               int32_t G, double *par, double var_floor, int32_t final_iter,
                               double *counts, const float *X, const int32_t *assign,
                               const double *gvar_floored, DevStatus *status, cudaStream_t s);
cudaError_t launch_em_prep(int32_t D, int32_t G, const double *par, Operands op, const float *center,
                           int32_t build_tc, cudaStream_t s);
cudaError_t launch_em_pass_simt(const EmPassArgs &a, int32_t grid, cudaStream_t s);
cudaError_t launch_em_finalize(const EmFinalizeArgs &a, cudaStream_t s);
// ---- register-blocked FP32 form (gmm_blocked.cu): blocks of 64 Gaussians,
// partial log-sum-exp per (block, sample) in part [gblocks][N]
bool em_blocked_supported(int32_t D, int32_t G);
int em_blocked_gblocks(int32_t G);
int em_blocked_chunks(int32_t G, int sms);
// n_dev (optional, device): the samples actually present, at most a.N (a.N is
// the stride of part and lse and sizes the launch)
cudaError_t launch_em_blocked(const EmPassArgs &a, float *lse, float2 *part, int32_t n_chunks, cudaStream_t s,
                              const int64_t *n_dev = nullptr);
// The same form with the log-densities computed once: the first phase also
// records each block's candidates, the merge turns them into per-sample
// records of the kept responsibilities, the M-step reads those; samples whose
// records overflow go through the recomputing second phase.  Statistics
// partials [em_rec_partials][G][1 + 2D]; log-likelihood partials per 128
// samples as launch_em_blocked.
struct RecWs {
    uint8_t *rec_n;          // [n_gb][N]
    uint16_t *rec_g;         // [n_gb][N][8]
    float *rec_l;            // [n_gb][N][8]
    uint8_t *rc;             // [N]
    uint16_t *rg;            // [N][kRecSlots]
    float *rgam;             // [N][kRecSlots]
    int32_t *bcnt;           // ceil(N / 1024)
    int64_t *n_mark;         // [1]
    float *Xd;               // [N][D]
    float *lse_d;            // [N]
    float2 *part_d;          // [n_gb][N]
};
size_t em_rec_ws_bytes(int64_t N, int32_t D, int32_t G);
RecWs em_rec_ws(void *base, int64_t N, int32_t D, int32_t G);
int em_rec_partials(int64_t N, int32_t G, int sms);
cudaError_t launch_em_blocked_rec(const EmPassArgs &a, float *lse, float2 *part, const RecWs &ws, int sms, cudaStream_t s);
// k-means map step for shapes beyond the tiled form: assign [N] (exact
// nearest mean) and the statistics into partial [n_chunks][G][1 + 2D];
// part [gblocks][N], arg [gblocks][N], nmax [1], snorm [N] and defer [N + 1]
// are work space
bool km_blocked_supported(int32_t D, int32_t G);
cudaError_t launch_km_blocked(const float *X, int64_t N, int32_t D, int32_t G, const double *means,
                              const double *w, const float *sw, float2 *part, uint8_t *arg, float *nmax,
                              float *snorm, int32_t *defer, int32_t *assign, double *partial, int32_t n_chunks,
                              const DevStatus *status, cudaStream_t s);
// log p(x_i) of the mixture into out [N] (FP64); part as above
cudaError_t launch_log_p_blocked(const float *X, int64_t N, int32_t D, int32_t G, Operands op, double *out,
                                 float2 *part, int sms, cudaStream_t s);
cudaError_t launch_log_p(const float *X, int64_t N, int32_t D, int32_t G, Operands op, int32_t g,
                         double *out, cudaStream_t s);
cudaError_t launch_assign(const float *X, int64_t N, int32_t D, int32_t G, const double *par,
                          Operands op, int32_t mode, int32_t *out, const float *sw_ones,
                          const double *w_ones, DevStatus *status, cudaStream_t s);
cudaError_t launch_status_reset(DevStatus *st, cudaStream_t s);
cudaError_t launch_sum_fp64(const double *v, int64_t n, double *out, cudaStream_t s);
cudaError_t launch_hist(const int32_t *a, int64_t N, int32_t G, unsigned long long *counts,
                        cudaStream_t s);
int64_t avg_log_p_noalloc_max_n();
cudaError_t launch_avg_log_p_noalloc(const float *X, int64_t N, int32_t D, int32_t G, Operands op, int32_t g,
                                     double *sum_host, cudaStream_t s);
int em_simt_grid(int32_t D, int32_t G, int sms);
int km_grid(int32_t D, int32_t G, int sms);
cudaError_t launch_f64_to_f32(const double *in, int64_t n, float *out, int sms, cudaStream_t s);
size_t em_simt_smem(int32_t D, int32_t G);
bool em_simt_supported(int32_t D, int32_t G);

// ---- batched form (gmm_batched.cu)
struct BFitStatus {
    int32_t code, halt, stop_after, n_done, fail_iter, pad[3];
};

struct BFit {
    const float *X;
    int64_t N;
    int32_t D, G;
    double *par, *par2;        // ping-pong [G*D means | G*D dcovs | G hefts]
    float2 *sm;                // E-step operands
    float *mu, *c;
    double *gvar, *w;          // floored global variance, distance weights
    float *sw, *center;
    double *counts;
    int32_t *assign;
    const int64_t *seed_idx;
    double *ll_hist;           // [em_iter]
    BFitStatus *status;
    int32_t item0, n_items;    // this fit's items are item0 .. item0+n_items-1
};

struct BItem {
    int32_t fit, pad;
    int64_t i0, i1;            // sample range of the item
    size_t poff;               // offset of its FP64 partial [G][1+2D]
};

size_t b_em_smem(int D, int G);
cudaError_t b_prepare(size_t em_smem, size_t km_smem);
size_t b_km_smem(int D, int G);
cudaError_t launch_b_gstats(BFit *fits, int n_fits, double var_floor, int dist, cudaStream_t s);
cudaError_t launch_b_seed(BFit *fits, const int32_t *comp_fit, const int32_t *comp_g, int n_comp, cudaStream_t s);
cudaError_t launch_b_km_iter(BFit *fits, int n_fits, const int32_t *comp_fit, const int32_t *comp_g, int n_comp,
                             const BItem *items, const int32_t *order, int n_items, int *counter, double *partial,
                             size_t smem, int grid, double var_floor, int final_iter, cudaStream_t s);
cudaError_t launch_b_em_prep(BFit *fits, const int32_t *comp_fit, const int32_t *comp_g, int n_comp, cudaStream_t s);
cudaError_t launch_b_em_pass(BFit *fits, const BItem *items, const int32_t *order, int n_items, int *counter,
                             double *partial, double *llp, size_t smem, int grid, int iter, cudaStream_t s);
cudaError_t launch_b_em_finish(BFit *fits, int n_fits, const int32_t *comp_fit, const int32_t *comp_g, int n_comp,
                               const BItem *items, const double *partial, const double *llp, double var_floor,
                               double em_tol, int iter, cudaStream_t s);

// ---- learned initialiser (gmm_init_net.cu)
struct InitNet;
InitNet *init_net_new(int D, int G, int Hp, int Hh, int Lp, int Lh, uint64_t seed, cudaError_t *err);
void init_net_free(InitNet *n);
int64_t init_net_n_params(const InitNet *n);
int init_net_D(const InitNet *n);
int init_net_G(const InitNet *n);
cudaError_t init_net_gather(const float *X, int D, const int64_t *idx, int P, float *out, cudaStream_t s);
cudaError_t init_net_set_weights(InitNet *n, const float *w_host);
cudaError_t init_net_get(const InitNet *n, float *w_host, float *g_host);
cudaError_t init_net_get_adam(const InitNet *n, float *m1_host, float *m2_host, int64_t *step);
cudaError_t init_net_set_adam(InitNet *n, const float *m1_host, const float *m2_host, int64_t step);
cudaError_t init_net_run(InitNet *n, const float *pts, int B, int P, const double *tm, const double *tv, const double *tw,
                         double lambda, double var_floor, int grads, double lr, double *pm, double *pv, double *pw,
                         double *loss_host, cudaStream_t s);

// Spread seeding: idx[0] set by the caller, idx[1..G-1] written on the device;
// work holds N + 2 * blocks doubles.
cudaError_t launch_spread_seeds(const float *X, int64_t N, int32_t D, int32_t G, const double *w, int64_t *idx,
                                double *work, int32_t blocks, cudaStream_t s);

// generate: N samples of the model (par = [means | dcovs | hefts]) into out (device)
cudaError_t launch_generate(const double *par, int32_t G, int32_t D, int64_t N, uint64_t seed, float *out, int sms,
                            cudaStream_t s);

// ---- launchers implemented in gmm_em_tc.cu
constexpr int kTcCap = 16;   // candidates per (sample, half of the Gaussians) before the dense fallback
constexpr int kTcKeep = 16;  // responsibilities kept per sample before the full-recompute fallback
struct TcLists {             // per-sample records between the three kernels of the tensor-core pass
    float *gam;              // [N][kTcKeep] responsibilities that matter (compacted)
    uint8_t *kg;             // [N][kTcKeep] their Gaussians (N_G <= 256)
    uint8_t *cand;           // [N][2][kTcCap] screened candidates (index within the half)
    float *lse;              // [N] log p(x_i)
    uint8_t *cnt;            // [N][2] candidates per half (> kTcCap: every Gaussian of the half)
    uint8_t *km;             // [N] kept responsibilities in the record (255: recompute every Gaussian)
    int64_t *sp_ig;          // [grid][kTcSpill] kept pairs beyond kTcKeep: sample * 256 + Gaussian
    float *sp_gam;           //                  and their responsibilities (0: unused entry)
    int32_t *sp_n;           // [grid] entries of each CTA's spill list
    int32_t *defer;          // [N] k-means: samples left to the exact decision (CTA b's in its own sample range)
};
constexpr int kTcSpill = 16384;   // spill entries per CTA

// Tensor-core k-means operands, rebuilt from the FP64 means every iteration.
struct KmTcOps {
    __nv_bfloat16 *B;        // [G][128] c' = (mu - m) sqrt(w) split as BF16 hi (0..63) | lo (64..127)
    float *cn;               // [G] |c'|^2
    float *cs;               // [G][D] mu sqrt(w) (FP32, uncentred: the exact FP32 distance)
    float *ncs;              // [G] |mu sqrt(w)|^2
};
bool km_tc_supported(int32_t D, int32_t G);
size_t km_tc_ops_bytes(int32_t D, int32_t G);
KmTcOps km_tc_ops(void *base, int32_t D, int32_t G);
// One k-means iteration's map step on the tensor cores: operands, assignment
// (assign[N]; L holds the screen's candidate lists), statistics into partial
// [grid][G][1 + 2D] (shifted by the FP32 means written to op.mu).
cudaError_t launch_km_pass_tc(const float *X, int64_t N, int32_t D, int32_t G, const double *means,
                              const double *w, const float *sw, const float *center, KmTcOps o, Operands op,
                              double *partial, int32_t grid, int32_t *assign, const TcLists &L, DevStatus *status,
                              long long wait_cycles, unsigned long long *stats, cudaStream_t s);

bool em_tc_supported(int32_t D, int32_t G);
int em_tc_grid(int sms);
size_t em_tc_list_bytes(int64_t N, int grid);
TcLists em_tc_lists(void *base, int64_t N, int grid);
cudaError_t launch_em_pass_tc(const EmPassArgs &a, const TcLists &L, int32_t grid, int32_t ms_chunks, cudaStream_t s);

// ---- tensor-core EM pass for D <= 128, N_G <= 4096 (gmm_em_wide.cu)
struct WideWs {              // work space, grown once per model
    unsigned char *img;      // split BF16 operand pieces of the screen
    float2 *bnd;             // screening constants per Gaussian
    uint8_t *cnt;            // [N] candidates per sample (255: more than a list holds)
    uint16_t *cand;          // [N][64] candidate Gaussians
    uint8_t *rc;             // [N] kept responsibilities in the record
    uint16_t *rg;            // [N][64] their Gaussians
    float *rgam;             // [N][64] and values
    int32_t *bcnt;           // per 1024 samples: samples left to the FP32 form, then their offsets
    int64_t *n_dense;        // [1] samples left to the FP32 form
    float *Xd;               // [N][D] their rows, gathered in sample order
    float *lse_d;            // [N] their log p(x_i)
    float2 *part_d;          // [ceil(G / 64)][N] their partial log-sum-exps
};
bool em_wide_supported(int32_t D, int32_t G);
// statistics partials [em_wide_partials][G][1 + 2D] and log-likelihood
// partials [em_wide_ll_partials] of one pass
int em_wide_partials(int64_t N, int32_t G, int sms);
int em_wide_ll_partials(int64_t N, int sms);
size_t em_wide_ws_bytes(int64_t N, int32_t D, int32_t G);
WideWs em_wide_ws(void *base, int64_t N, int32_t D, int32_t G);
// One EM iteration's pass from par (the iteration's parameters; op holds
// their FP32 operands) into a.partial and a.ll_partial.
cudaError_t launch_em_wide(const EmPassArgs &a, const double *par, const WideWs &ws, int sms, cudaStream_t s);
// M-step from per-sample records (rc [N] counts, rg/rgam [N][kRecSlots]
// Gaussians and responsibilities) into a.partial [record_mstep_chunks][G][1 + 2D]

int record_mstep_chunks(int64_t N, int32_t G, int sms);
cudaError_t launch_record_mstep(const EmPassArgs &a, const uint8_t *rc, const uint16_t *rg, const float *rgam, int sms,
                                cudaStream_t s);
// the samples whose flag is 255, in sample order: their rows into Xd, v[i]
// into vd (when v is given), their count into *n_marked; bcnt holds
// ceil(N / 1024) ints of work space
cudaError_t launch_gather_marked(const uint8_t *flag, const float *X, const float *v, int64_t N, int32_t D, int32_t *bcnt,
                                 int64_t *n_marked, float *Xd, float *vd, cudaStream_t s);

}  // namespace gmm
