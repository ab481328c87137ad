// C ABI of the library (declared in include/gmm_gb300.h): argument checks,
// the model object and its device workspace, host<->device staging, and the
// order in which the kernels of one call are queued on the caller's stream.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <unordered_map>
#include <vector>

#include "gmm_internal.cuh"

using gmm::DevStatus;
using gmm::Operands;

namespace {

// Device counters of gmm_profile: words 0-10 the EM screening kernel's,
// words 11-13 the tensor-core k-means pass's (screened, deferred, FP64).
constexpr int kStatWords = 14;
constexpr int kStatKm = 11;

thread_local std::string g_err;

gmm_status fail(gmm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CK(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail(GMM_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                        __FILE__, __LINE__);                                                     \
    } while (0)

template <class T>
cudaError_t grow(T *&p, size_t &cap, size_t n)
{
    if (n <= cap && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&p), (n ? n : 1) * sizeof(T));
    if (e == cudaSuccess) cap = n;
    return e;
}

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): state advances by the
// golden-gamma constant, output is the variant-13 mix of the state.
uint64_t splitmix64_next(uint64_t &state)
{
    uint64_t z = (state += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// random_subset seeding: the first G entries of a partial Fisher-Yates
// shuffle of 0..N-1 driven by SplitMix64(seed); the untouched identity
// permutation is kept implicit (only swapped slots are stored).
std::vector<int64_t> random_subset(int64_t N, int32_t G, uint64_t seed)
{
    std::unordered_map<int64_t, int64_t> moved;
    auto at = [&](int64_t k) {
        auto it = moved.find(k);
        return it == moved.end() ? k : it->second;
    };
    std::vector<int64_t> out(G);
    uint64_t st = seed;
    for (int32_t j = 0; j < G; ++j) {
        const int64_t k = j + (int64_t)(splitmix64_next(st) % (uint64_t)(N - j));
        const int64_t vj = at(j), vk = at(k);
        moved[j] = vk;
        moved[k] = vj;
        out[j] = vk;
    }
    return out;
}

}  // namespace

struct gmm_model {
    int device = 0;
    int sms = 0;
    int32_t D = 0, G = 0;
    bool has_params = false;
    bool ops_valid = false;
    double *par[2] = {nullptr, nullptr};
    size_t par_cap[2] = {0, 0};
    int cur = 0;
    // E-step operands
    Operands op{};
    float2 *op_sm = nullptr; size_t op_sm_cap = 0;
    float *op_mu = nullptr; size_t op_mu_cap = 0;
    float *op_c = nullptr; size_t op_c_cap = 0;
    __nv_bfloat16 *op_B = nullptr; size_t op_B_cap = 0;
    // global statistics
    double *gstat = nullptr; size_t gstat_cap = 0;   // gmean | gvar_floored | wdist | wones  [4][D]
    float *fstat = nullptr; size_t fstat_cap = 0;    // sw | center  [2][D]
    bool has_center = false;
    int32_t center_D = 0;
    // workspace
    double *partial = nullptr; size_t partial_cap = 0;
    uint8_t *kmarg = nullptr; size_t kmarg_cap = 0;           // register-blocked k-means: argmin per block | max norm
    unsigned char *tclist = nullptr; size_t tclist_cap = 0;   // tensor-core pass: per-sample records
    unsigned char *wide = nullptr; size_t wide_cap = 0;       // tensor-core pass beyond D 64 / N_G 256
    unsigned char *recws = nullptr; size_t recws_cap = 0;     // FP32 two-phase form: candidate and kept records
    unsigned char *kmop = nullptr; size_t kmop_cap = 0;       // tensor-core k-means operands
    double *spread = nullptr; size_t spread_cap = 0;          // spread seeding: distances + block partials
    cudaStream_t cstream = nullptr;                           // host-input copies that overlap the first pass
    std::vector<cudaEvent_t> cev;                             // [0] start, [1..] chunk copies
    float *lse = nullptr; size_t lse_cap = 0;
    float2 *lsep = nullptr; size_t lsep_cap = 0;               // register-blocked form: [Gaussian blocks][N] partials
    double *llp = nullptr; size_t llp_cap = 0;
    double *lld = nullptr; size_t lld_cap = 0;
    double *counts = nullptr; size_t counts_cap = 0;
    int32_t *assign = nullptr; size_t assign_cap = 0;
    float *xstage = nullptr; size_t xstage_cap = 0;
    double *dstage = nullptr; size_t dstage_cap = 0;
    int64_t *idx = nullptr; size_t idx_cap = 0;
    unsigned long long *hist = nullptr; size_t hist_cap = 0;
    DevStatus *status = nullptr;
    std::vector<double> ll_hist;
    // measurement hooks
    bool profiling = false;
    std::vector<cudaEvent_t> ev;      // pairs around fused-pass launches (pending)
    size_t ev_used = 0;
    double pass_ms = 0.0;
    long long pass_launches = 0;
    long long launch_base = 0;
    // failure-detection test hooks
    long long wait_cycles = 2000000000LL;
    int skip_mma = 0;
    int km_form = 0;                        // 0: tensor cores where supported, 1: CUDA cores
    int fp32_form = 0;                      // 0: by shape, 1: one-pass where it fits, 2: register-blocked, 3: same, recomputed second phase
    int tc_form = 0;                        // 0: by shape, 1: the D <= 128 / N_G <= 4096 pass for every shape
    unsigned long long *sstats = nullptr;   // screening counters (device, [kStatWords])

    double *means() const { return par[cur]; }
    double *gmean() const { return gstat; }
    double *gvar() const { return gstat + D; }
    double *wdist() const { return gstat + 2 * (size_t)D; }
    double *wones() const { return gstat + 3 * (size_t)D; }
    float *sw() const { return fstat; }
    float *center() const { return fstat + D; }
};

namespace {

// Event pair around one fused-pass launch when profiling is on.
gmm_status prof_begin(gmm_model *m, cudaStream_t s, size_t *slot)
{
    if (!m->profiling) return GMM_OK;
    if (m->ev_used + 2 > m->ev.size()) {
        for (int k = 0; k < 64; ++k) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            m->ev.push_back(e);
        }
    }
    *slot = m->ev_used;
    m->ev_used += 2;
    CK(cudaEventRecord(m->ev[*slot], s));
    return GMM_OK;
}

gmm_status prof_end(gmm_model *m, cudaStream_t s, size_t slot)
{
    if (!m->profiling) return GMM_OK;
    CK(cudaEventRecord(m->ev[slot + 1], s));
    return GMM_OK;
}

// After the stream has drained: add up the recorded pairs.
gmm_status prof_collect(gmm_model *m)
{
    for (size_t k = 0; k + 1 < m->ev_used; k += 2) {
        float ms = 0.f;
        CK(cudaEventSynchronize(m->ev[k + 1]));
        CK(cudaEventElapsedTime(&ms, m->ev[k], m->ev[k + 1]));
        m->pass_ms += ms;
        m->pass_launches += 1;
    }
    m->ev_used = 0;
    return GMM_OK;
}

gmm_status ensure_shape(gmm_model *m, int32_t D, int32_t G)
{
    const size_t np = 2 * (size_t)G * D + G;
    CK(grow(m->par[0], m->par_cap[0], np));
    CK(grow(m->par[1], m->par_cap[1], np));
    const int32_t KP = 128;
    CK(grow(m->op_sm, m->op_sm_cap, (size_t)G * D));
    CK(grow(m->op_mu, m->op_mu_cap, (size_t)G * D));
    CK(grow(m->op_c, m->op_c_cap, 4 * (size_t)G));
    CK(grow(m->op_B, m->op_B_cap, (size_t)G * KP));
    m->op.sm = m->op_sm;
    m->op.mu = m->op_mu;
    m->op.c = m->op_c;
    m->op.c0 = m->op_c + G;
    m->op.ctc = m->op_c + 2 * (size_t)G;
    m->op.q = m->op_c + 3 * (size_t)G;
    m->op.B = m->op_B;
    m->op.KP = KP;
    if (m->D != D) m->has_center = false;
    CK(grow(m->gstat, m->gstat_cap, 4 * (size_t)D));
    CK(grow(m->fstat, m->fstat_cap, 2 * (size_t)D));
    if (!m->status) CK(cudaMalloc(&m->status, sizeof(DevStatus)));
    m->D = D;
    m->G = G;
    return GMM_OK;
}

// Device view of X: the caller's pointer if it is device memory, else a copy
// in the model's staging buffer.
gmm_status stage_x(gmm_model *m, const float *X, int64_t N, int32_t D, cudaStream_t s, const float **Xd)
{
    if (is_device_ptr(X)) { *Xd = X; return GMM_OK; }
    CK(grow(m->xstage, m->xstage_cap, (size_t)N * D));
    CK(cudaMemcpyAsync(m->xstage, X, sizeof(float) * (size_t)N * D, cudaMemcpyHostToDevice, s));
    *Xd = m->xstage;
    return GMM_OK;
}

gmm_status read_status(gmm_model *m, cudaStream_t s, DevStatus *out)
{
    CK(cudaMemcpyAsync(out, m->status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return GMM_OK;
}

gmm_status run_global_stats(gmm_model *m, const float *Xd, int64_t N, double var_floor, int32_t dist,
                            cudaStream_t s)
{
    const int grid = m->sms * 4;
    CK(grow(m->partial, m->partial_cap, (size_t)grid * m->D));
    CK(gmm::launch_global_stats(Xd, N, m->D, var_floor, dist, m->partial, grid, m->gmean(), m->gvar(),
                                m->wdist(), m->sw(), m->center(), s));
    m->has_center = true;
    m->center_D = m->D;
    return GMM_OK;
}

gmm_status run_kmeans(gmm_model *m, const float *Xd, int64_t N, int32_t km_iter, double var_floor,
                      cudaStream_t s)
{
    const int32_t D = m->D, G = m->G, S = 1 + 2 * D;
    const bool tc = m->km_form == 0 && m->has_center && m->center_D == D && gmm::km_tc_supported(D, G);
    const bool blk = !tc && !gmm::km_tile_supported(D, G);   // register-blocked CUDA-core form
    if (blk && !gmm::km_blocked_supported(D, G))
        return fail(GMM_ERR_UNSUPPORTED, "k-means: shared memory too small for D=%d, G=%d", D, G);
    const int grid = tc ? m->sms : gmm::km_grid(D, G, m->sms);
    CK(grow(m->partial, m->partial_cap, (size_t)grid * G * S));
    const size_t nb = (size_t)gmm::em_blocked_gblocks(G) * (size_t)N;
    if (tc) {
        CK(grow(m->tclist, m->tclist_cap, gmm::em_tc_list_bytes(N, grid)));
        CK(grow(m->kmop, m->kmop_cap, gmm::km_tc_ops_bytes(D, G)));
        m->ops_valid = false;   // the pass writes the FP32 means into the E-step operands
    } else if (blk) {
        CK(grow(m->lsep, m->lsep_cap, nb));                          // (best, runner-up) per block
        // argmin per block | max |cs|^2 | |xs|^2 [N] | deferred samples [N] and their count
        CK(grow(m->kmarg, m->kmarg_cap, ((nb + 15) & ~(size_t)15) + 16 + 8 * (size_t)N + 16));
    }
    CK(grow(m->assign, m->assign_cap, (size_t)N));
    CK(grow(m->counts, m->counts_cap, (size_t)G));
    for (int32_t it = 0; it < km_iter; ++it) {
        const int32_t np = grid;
        size_t slot = 0;
        gmm_status prc = prof_begin(m, s, &slot);
        if (prc != GMM_OK) return prc;
        if (tc)
            CK(gmm::launch_km_pass_tc(Xd, N, D, G, m->par[m->cur], m->wdist(), m->sw(), m->center(),
                                      gmm::km_tc_ops(m->kmop, D, G), m->op, m->partial, grid, m->assign,
                                      gmm::em_tc_lists(m->tclist, N, grid), m->status, m->wait_cycles,
                                      m->profiling ? m->sstats + kStatKm : nullptr, s));
        else if (blk)
            CK(gmm::launch_km_blocked(Xd, N, D, G, m->par[m->cur], m->wdist(), m->sw(), m->lsep, m->kmarg,
                                      reinterpret_cast<float *>(m->kmarg + ((nb + 15) & ~(size_t)15)),
                                      reinterpret_cast<float *>(m->kmarg + ((nb + 15) & ~(size_t)15) + 16),
                                      reinterpret_cast<int32_t *>(m->kmarg + ((nb + 15) & ~(size_t)15) + 16 + 4 * (size_t)N),
                                      m->assign, m->partial, grid, m->status, s));
        else
            CK(gmm::launch_km_pass(Xd, N, D, G, m->par[m->cur], m->wdist(), m->sw(), m->partial, grid, m->assign,
                                   m->status, s));
        if ((prc = prof_end(m, s, slot)) != GMM_OK) return prc;
        CK(gmm::launch_km_finalize(m->partial, np, N, D, G, m->par[m->cur], var_floor, it == km_iter - 1,
                                   m->counts, Xd, m->assign, m->gvar(), m->status, s));
    }
    return GMM_OK;
}

gmm_status run_prep(gmm_model *m, cudaStream_t s)
{
    const int build_tc = m->has_center && m->center_D == m->D;
    CK(gmm::launch_em_prep(m->D, m->G, m->par[m->cur], m->op, m->has_center ? m->center() : nullptr, build_tc, s));
    m->ops_valid = true;
    return GMM_OK;
}

// Host X arriving in sample chunks (tile-aligned bounds, one copy event per
// chunk): the first EM iteration runs its pass chunk by chunk, each after its
// copy, so the copies of later chunks overlap the pass over earlier ones.
struct ChunkPlan {
    std::vector<int64_t> bounds;     // C + 1 sample bounds
    std::vector<cudaEvent_t> ready;  // C events recorded on the copy stream
};

// em_iter EM iterations from par[cur]; iteration k reads par[(cur+k)&1] and
// writes par[(cur+k+1)&1].  The status block tells which buffer is final.
gmm_status run_em(gmm_model *m, const float *Xd, int64_t N, int32_t em_iter, double var_floor, double em_tol,
                  int32_t prec, int32_t print, cudaStream_t s, const ChunkPlan *cp = nullptr)
{
    const int32_t D = m->D, G = m->G, S = 1 + 2 * D;
    const bool tc = prec == GMM_BF16;
    // tensor cores: the one-tile pass for D <= 64 and N_G <= 256, else the
    // split-BF16 screen over blocks of Gaussians (D <= 128, N_G <= 4096)
    const bool wide = tc && (m->tc_form == 1 || !gmm::em_tc_supported(D, G));
    if (wide && !gmm::em_wide_supported(D, G))
        return fail(GMM_ERR_UNSUPPORTED, "tensor-core E-step needs D <= 128 and n_gaus <= 4096 (D=%d, G=%d)", D, G);
    // FP32: the one-pass form for N_G <= 128 while all N_G operands and
    // statistics fit in one CTA's shared memory, else the register-blocked
    // two-phase form (faster from N_G = 256: 11.0 against 12.7 ms per
    // iteration at N = 2e6, D = 60)
    const bool one_pass_fits = gmm::em_simt_supported(D, G);
    const bool two_phase = !tc && (m->fp32_form >= 2 || !one_pass_fits || (m->fp32_form == 0 && G > 128));
    if (two_phase && !gmm::em_blocked_supported(D, G))
        return fail(GMM_ERR_UNSUPPORTED, "FP32 E-step: shared memory too small for D=%d, G=%d", D, G);
    if (tc && !(m->has_center && m->center_D == D))
        return fail(GMM_ERR_STATE, "tensor-core E-step needs the global centre (run learn or recompute_center)");
    // one-pass forms: one partial per CTA; two-phase form: one per sample chunk
    // (and one log-likelihood partial per 128-sample block of the lse pass)
    const bool rec = two_phase && m->fp32_form != 3;   // records of the kept responsibilities (else recompute)
    const int grid = wide ? gmm::em_wide_partials(N, G, m->sms)
                          : (tc ? gmm::em_tc_grid(m->sms)
                                : (two_phase ? (rec ? gmm::em_rec_partials(N, G, m->sms) : gmm::em_blocked_chunks(G, m->sms))
                                             : gmm::em_simt_grid(D, G, m->sms)));
    if ((two_phase || wide) && cp) {   // these forms take all of X at once
        CK(cudaStreamWaitEvent(s, cp->ready.back(), 0));
        cp = nullptr;
    }
    const int nch = cp ? (int)cp->ready.size() : 1;
    const int n_llp = two_phase ? (int)((N + 127) / 128) : (wide ? gmm::em_wide_ll_partials(N, m->sms) : grid);
    CK(grow(m->partial, m->partial_cap, (size_t)nch * grid * G * S));
    if (two_phase) CK(grow(m->lse, m->lse_cap, (size_t)N));
    if (two_phase) CK(grow(m->lsep, m->lsep_cap, (size_t)gmm::em_blocked_gblocks(G) * (size_t)N));
    if (tc && !wide) CK(grow(m->tclist, m->tclist_cap, gmm::em_tc_list_bytes(N, grid)));
    if (wide) CK(grow(m->wide, m->wide_cap, gmm::em_wide_ws_bytes(N, D, G)));
    if (rec) CK(grow(m->recws, m->recws_cap, gmm::em_rec_ws_bytes(N, D, G)));
    CK(grow(m->llp, m->llp_cap, (size_t)nch * n_llp));
    CK(grow(m->lld, m->lld_cap, (size_t)(em_iter > 0 ? em_iter : 1)));
    CK(gmm::launch_status_reset(m->status, s));
    if (em_iter == 0) return GMM_OK;
    const int base = m->cur;
    CK(gmm::launch_em_prep(D, G, m->par[base], m->op, m->center(), tc ? 1 : (m->has_center && m->center_D == D), s));
    for (int32_t k = 0; k < em_iter; ++k) {
        const int chunks = (k == 0 && cp) ? nch : 1;
        size_t slot = 0;
        gmm_status prc = prof_begin(m, s, &slot);
        if (prc != GMM_OK) return prc;
        for (int c = 0; c < chunks; ++c) {
            const int64_t b0 = chunks > 1 ? cp->bounds[c] : 0, b1 = chunks > 1 ? cp->bounds[c + 1] : N;
            if (chunks > 1) CK(cudaStreamWaitEvent(s, cp->ready[c], 0));
            gmm::EmPassArgs pa{Xd + b0 * D, b1 - b0, D, G, m->op, m->center(), m->partial + (size_t)c * grid * G * S,
                               m->llp + (size_t)c * n_llp, m->status, k, m->wait_cycles, m->skip_mma,
                               m->profiling ? m->sstats : nullptr, N};
            if (wide)
                CK(gmm::launch_em_wide(pa, m->par[(base + k) & 1], gmm::em_wide_ws(m->wide, N, D, G), m->sms, s));
            else if (tc) CK(gmm::launch_em_pass_tc(pa, gmm::em_tc_lists(m->tclist, b1 - b0, grid), grid, grid, s));
            else if (rec) CK(gmm::launch_em_blocked_rec(pa, m->lse, m->lsep, gmm::em_rec_ws(m->recws, N, D, G), m->sms, s));
            else if (two_phase) CK(gmm::launch_em_blocked(pa, m->lse, m->lsep, grid, s));
            else CK(gmm::launch_em_pass_simt(pa, grid, s));
        }
        if ((prc = prof_end(m, s, slot)) != GMM_OK) return prc;
        gmm::EmFinalizeArgs fa{m->partial, m->llp, chunks * grid, chunks * n_llp, N, D, G, m->par[(base + k) & 1], m->par[(base + k + 1) & 1],
                               var_floor, 0, m->op, m->center(), m->status, k, em_tol, m->lld,
                               tc ? 1 : (m->has_center && m->center_D == D)};
        CK(gmm::launch_em_finalize(fa, s));
    }
    DevStatus st;
    gmm_status rc = read_status(m, s, &st);
    if (rc != GMM_OK) return rc;
    if ((rc = prof_collect(m)) != GMM_OK) return rc;
    std::vector<double> ll(em_iter);
    CK(cudaMemcpy(ll.data(), m->lld, sizeof(double) * em_iter, cudaMemcpyDeviceToHost));
    if (st.code != 0) {
        m->cur = (base + (st.fail_iter < 0 ? 0 : st.fail_iter)) & 1;
        for (int k = 0; k < st.n_done && k < em_iter; ++k) m->ll_hist.push_back(ll[k]);
        m->ops_valid = false;
        return fail((gmm_status)st.code, st.code == GMM_ERR_TIMEOUT ? "EM iteration %d: a bounded device wait ran out"
                                                                     : "EM iteration %d produced a non-finite value",
                    st.fail_iter);
    }
    m->cur = (base + st.n_done) & 1;
    for (int k = 0; k < st.n_done; ++k) {
        m->ll_hist.push_back(ll[k]);
        if (print) fprintf(stderr, "gmm: EM iteration %d: mean log-likelihood %.10g\n", k + 1, ll[k]);
    }
    return GMM_OK;
}

gmm_status validate_x(const float *X, int64_t N, int32_t D)
{
    if (!X) return fail(GMM_ERR_ARG, "X is NULL");
    if (N < 1) return fail(GMM_ERR_ARG, "N must be >= 1 (got %lld)", (long long)N);
    if (D < 1 || D > GMM_MAX_DIMS) return fail(GMM_ERR_UNSUPPORTED, "D must be in [1, %d] (got %d)", GMM_MAX_DIMS, D);
    return GMM_OK;
}

cudaStream_t as_stream(void *p) { return reinterpret_cast<cudaStream_t>(p); }

}  // namespace

extern "C" {

const char *gmm_last_error(void) { return g_err.c_str(); }

void gmm_default_opts(gmm_learn_opts *o)
{
    if (!o) return;
    o->dist = GMM_MAHA;
    o->seed_mode = GMM_RANDOM_SUBSET;
    o->seed = 0;
    o->em_tol = 0.0;
    o->prec = GMM_FP32;
    o->print = 0;
    o->stream = nullptr;
}

gmm_status gmm_create(gmm_model **out)
{
    if (!out) return fail(GMM_ERR_ARG, "out is NULL");
    *out = nullptr;
    gmm_model *m = new (std::nothrow) gmm_model();
    if (!m) return fail(GMM_ERR_OOM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&m->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&m->sms, cudaDevAttrMultiProcessorCount, m->device);
    if (e == cudaSuccess) e = cudaMalloc(&m->status, sizeof(DevStatus));
    if (e != cudaSuccess) {
        delete m;
        return fail(GMM_ERR_CUDA, "no usable CUDA device: %s", cudaGetErrorString(e));
    }
    *out = m;
    return GMM_OK;
}

void gmm_destroy(gmm_model *m)
{
    if (!m) return;
    for (cudaEvent_t e : m->ev) cudaEventDestroy(e);
    for (cudaEvent_t e : m->cev) cudaEventDestroy(e);
    if (m->cstream) cudaStreamDestroy(m->cstream);
    if (m->sstats) cudaFree(m->sstats);
    void *bufs[] = {m->par[0], m->par[1], m->op_sm, m->op_mu, m->op_c, m->op_B, m->gstat, m->fstat,
                    m->partial, m->kmarg, m->lse, m->llp, m->lld, m->counts, m->assign, m->xstage, m->dstage, m->idx,
                    m->hist, m->status, m->tclist, m->kmop, m->spread, m->lsep, m->wide, m->recws};
    for (void *p : bufs)
        if (p) cudaFree(p);
    delete m;
}

gmm_status gmm_learn(gmm_model *m, const float *X, int64_t N, int32_t D, int32_t n_gaus, int32_t km_iter,
                     int32_t em_iter, double var_floor, const gmm_learn_opts *opts)
{
    if (!m) return fail(GMM_ERR_ARG, "model is NULL");
    gmm_learn_opts o;
    gmm_default_opts(&o);
    if (opts) o = *opts;
    gmm_status rc = validate_x(X, N, D);
    if (rc != GMM_OK) return rc;
    if (n_gaus < 1 || (int64_t)n_gaus > N) return fail(GMM_ERR_ARG, "need 1 <= n_gaus <= N (n_gaus=%d, N=%lld)", n_gaus, (long long)N);
    if (km_iter < 0 || em_iter < 0) return fail(GMM_ERR_ARG, "km_iter and em_iter must be >= 0");
    if (!(var_floor >= 0.0) || !std::isfinite(var_floor)) return fail(GMM_ERR_ARG, "var_floor must be finite and >= 0");
    if (o.dist != GMM_EUCL && o.dist != GMM_MAHA) return fail(GMM_ERR_ARG, "dist must be EUCL or MAHA");
    if (o.seed_mode < GMM_KEEP_EXISTING || o.seed_mode > GMM_RANDOM_SPREAD) return fail(GMM_ERR_ARG, "bad seed_mode");
    if (o.prec < GMM_FP32 || o.prec > GMM_BF16) return fail(GMM_ERR_ARG, "bad prec");
    if (o.seed_mode == GMM_KEEP_EXISTING && !(m->has_params && m->D == D && m->G == n_gaus))
        return fail(GMM_ERR_STATE, "keep_existing needs parameters of shape (%d, %d)", n_gaus, D);
    cudaStream_t s = as_stream(o.stream);
    if (o.seed_mode != GMM_KEEP_EXISTING || m->D != D || m->G != n_gaus) {
        rc = ensure_shape(m, D, n_gaus);
        if (rc != GMM_OK) return rc;
    }
    const float *Xd = nullptr;
    if ((rc = stage_x(m, X, N, D, s, &Xd)) != GMM_OK) return rc;
    CK(gmm::launch_status_reset(m->status, s));
    if ((rc = run_global_stats(m, Xd, N, var_floor, o.dist, s)) != GMM_OK) return rc;
    if (o.seed_mode != GMM_KEEP_EXISTING) {
        std::vector<int64_t> idx;
        if (o.seed_mode == GMM_RANDOM_SUBSET) {
            idx = random_subset(N, n_gaus, o.seed);
        } else if (o.seed_mode == GMM_STATIC_SUBSET) {
            for (int32_t g = 0; g < n_gaus; ++g) idx.push_back((int64_t)(((__int128)g * N) / n_gaus));
        } else {   // spread: the first seed here, the rest on the device
            idx.assign((size_t)n_gaus, 0);
            idx[0] = o.seed_mode == GMM_STATIC_SPREAD ? 0 : random_subset(N, 1, o.seed)[0];
        }
        CK(grow(m->idx, m->idx_cap, (size_t)n_gaus));
        CK(cudaMemcpyAsync(m->idx, idx.data(), sizeof(int64_t) * n_gaus, cudaMemcpyHostToDevice, s));
        if (o.seed_mode == GMM_STATIC_SPREAD || o.seed_mode == GMM_RANDOM_SPREAD) {
            const int blocks = 2 * m->sms;
            CK(grow(m->spread, m->spread_cap, (size_t)N + 2u * blocks));
            CK(gmm::launch_spread_seeds(Xd, N, D, n_gaus, m->wdist(), m->idx, m->spread, blocks, s));
        }
        m->cur = 0;
        CK(gmm::launch_gather_seeds(Xd, D, n_gaus, m->idx, m->par[0], s));
        CK(cudaStreamSynchronize(s));   // idx is a host vector
        m->has_params = true;
    }
    m->ll_hist.clear();
    if (km_iter > 0 && (rc = run_kmeans(m, Xd, N, km_iter, var_floor, s)) != GMM_OK) return rc;
    if ((rc = run_em(m, Xd, N, em_iter, var_floor, o.em_tol, o.prec, o.print, s)) != GMM_OK) return rc;
    if ((rc = run_prep(m, s)) != GMM_OK) return rc;
    DevStatus st;
    if ((rc = read_status(m, s, &st)) != GMM_OK) return rc;
    if ((rc = prof_collect(m)) != GMM_OK) return rc;
    if (st.code != 0) return fail((gmm_status)st.code, "learn failed with device status %d", st.code);
    return GMM_OK;
}

gmm_status gmm_em_iterate(gmm_model *m, const float *X, int64_t N, int32_t n_iter, double var_floor, int32_t prec,
                          int32_t recompute_center, void *stream)
{
    if (!m) return fail(GMM_ERR_ARG, "model is NULL");
    if (!m->has_params) return fail(GMM_ERR_STATE, "model has no parameters");
    gmm_status rc = validate_x(X, N, m->D);
    if (rc != GMM_OK) return rc;
    if (n_iter < 0 || !(var_floor >= 0.0) || !std::isfinite(var_floor)) return fail(GMM_ERR_ARG, "bad n_iter/var_floor");
    if (prec < GMM_FP32 || prec > GMM_BF16) return fail(GMM_ERR_ARG, "bad prec");
    cudaStream_t s = as_stream(stream);
    const float *Xd = nullptr;
    const bool need_center = recompute_center || !(m->has_center && m->center_D == m->D);
    ChunkPlan plan;
    constexpr int kChunks = 4;
    if (!is_device_ptr(X) && !need_center && n_iter >= 1 && N >= (int64_t)kChunks * 65536) {
        // host X in four tile-aligned chunks on a copy stream; the first
        // iteration's pass follows them chunk by chunk
        const size_t D = (size_t)m->D;
        CK(grow(m->xstage, m->xstage_cap, (size_t)N * D));
        if (!m->cstream) CK(cudaStreamCreateWithFlags(&m->cstream, cudaStreamNonBlocking));
        while (m->cev.size() < kChunks + 1) {
            cudaEvent_t e;
            CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            m->cev.push_back(e);
        }
        CK(cudaEventRecord(m->cev[0], s));               // earlier work on s that reads xstage
        CK(cudaStreamWaitEvent(m->cstream, m->cev[0], 0));
        for (int c = 0; c <= kChunks; ++c) plan.bounds.push_back(c == kChunks ? N : (N * c / kChunks) / 128 * 128);
        for (int c = 0; c < kChunks; ++c) {
            const int64_t b0 = plan.bounds[c], b1 = plan.bounds[c + 1];
            CK(cudaMemcpyAsync(m->xstage + b0 * D, X + b0 * D, sizeof(float) * (size_t)(b1 - b0) * D,
                               cudaMemcpyHostToDevice, m->cstream));
            CK(cudaEventRecord(m->cev[1 + c], m->cstream));
            plan.ready.push_back(m->cev[1 + c]);
        }
        Xd = m->xstage;   // the first pass waits for each chunk; the last wait covers every later use
    } else if ((rc = stage_x(m, X, N, m->D, s, &Xd)) != GMM_OK) {
        return rc;
    }
    if (need_center) {
        CK(gmm::launch_status_reset(m->status, s));
        if ((rc = run_global_stats(m, Xd, N, var_floor, GMM_MAHA, s)) != GMM_OK) return rc;
    }
    if ((rc = run_em(m, Xd, N, n_iter, var_floor, 0.0, prec, 0, s, plan.ready.empty() ? nullptr : &plan)) != GMM_OK)
        return rc;
    return run_prep(m, s);
}

gmm_status gmm_kmeans(gmm_model *m, const float *X, int64_t N, int32_t km_iter, int32_t dist, double var_floor,
                      int32_t *assign_out, void *stream)
{
    if (!m) return fail(GMM_ERR_ARG, "model is NULL");
    if (!m->has_params) return fail(GMM_ERR_STATE, "model has no parameters (means to start from)");
    gmm_status rc = validate_x(X, N, m->D);
    if (rc != GMM_OK) return rc;
    if (km_iter < 1) return fail(GMM_ERR_ARG, "km_iter must be >= 1");
    if (dist != GMM_EUCL && dist != GMM_MAHA) return fail(GMM_ERR_ARG, "dist must be EUCL or MAHA");
    if ((int64_t)m->G > N) return fail(GMM_ERR_ARG, "n_gaus > N");
    if (!(var_floor >= 0.0) || !std::isfinite(var_floor)) return fail(GMM_ERR_ARG, "bad var_floor");
    cudaStream_t s = as_stream(stream);
    const float *Xd = nullptr;
    if ((rc = stage_x(m, X, N, m->D, s, &Xd)) != GMM_OK) return rc;
    CK(gmm::launch_status_reset(m->status, s));
    if ((rc = run_global_stats(m, Xd, N, var_floor, dist, s)) != GMM_OK) return rc;
    if ((rc = run_kmeans(m, Xd, N, km_iter, var_floor, s)) != GMM_OK) return rc;
    if ((rc = run_prep(m, s)) != GMM_OK) return rc;
    if (assign_out) {
        CK(cudaMemcpyAsync(assign_out, m->assign, sizeof(int32_t) * (size_t)N, cudaMemcpyDefault, s));
    }
    DevStatus st;
    if ((rc = read_status(m, s, &st)) != GMM_OK) return rc;
    if ((rc = prof_collect(m)) != GMM_OK) return rc;
    if (st.code != 0) return fail((gmm_status)st.code, "k-means failed with device status %d", st.code);
    return GMM_OK;
}

namespace {
// log p(x_i) into od (device): for the mixture with N_G > 128 by the
// register-blocked partial log-sum-exps (the FP32 EM form's first phase),
// else one sample per thread
cudaError_t run_log_p(gmm_model *m, const float *Xd, int64_t N, int32_t g, double *od, cudaStream_t s)
{
    if (g < 0 && m->G > 128 && gmm::em_blocked_supported(m->D, m->G)) {
        cudaError_t e = grow(m->lsep, m->lsep_cap, (size_t)gmm::em_blocked_gblocks(m->G) * (size_t)N);
        if (e != cudaSuccess) return e;
        return gmm::launch_log_p_blocked(Xd, N, m->D, m->G, m->op, od, m->lsep, m->sms, s);
    }
    return gmm::launch_log_p(Xd, N, m->D, m->G, m->op, g, od, s);
}
}  // namespace

gmm_status gmm_log_p(const gmm_model *mc, const float *X, int64_t N, int32_t g, double *out, void *stream)
{
    gmm_model *m = const_cast<gmm_model *>(mc);
    if (!m || !out) return fail(GMM_ERR_ARG, "NULL argument");
    if (!m->has_params) return fail(GMM_ERR_STATE, "model has no parameters");
    gmm_status rc = validate_x(X, N, m->D);
    if (rc != GMM_OK) return rc;
    if (g < -1 || g >= m->G) return fail(GMM_ERR_ARG, "g out of range");
    cudaStream_t s = as_stream(stream);
    if (!m->ops_valid && (rc = run_prep(m, s)) != GMM_OK) return rc;
    const float *Xd = nullptr;
    if ((rc = stage_x(m, X, N, m->D, s, &Xd)) != GMM_OK) return rc;
    double *od = out;
    const bool dev_out = is_device_ptr(out);
    if (!dev_out) {
        CK(grow(m->dstage, m->dstage_cap, (size_t)N));
        od = m->dstage;
    }
    CK(run_log_p(m, Xd, N, g, od, s));
    if (!dev_out) CK(cudaMemcpyAsync(out, od, sizeof(double) * (size_t)N, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return GMM_OK;
}

gmm_status gmm_avg_log_p(const gmm_model *mc, const float *X, int64_t N, int32_t g, double *out, void *stream)
{
    gmm_model *m = const_cast<gmm_model *>(mc);
    if (!m || !out) return fail(GMM_ERR_ARG, "NULL argument");
    if (!m->has_params) return fail(GMM_ERR_STATE, "model has no parameters");
    gmm_status rc = validate_x(X, N, m->D);
    if (rc != GMM_OK) return rc;
    if (g < -1 || g >= m->G) return fail(GMM_ERR_ARG, "g out of range");
    cudaStream_t s = as_stream(stream);
    if (!m->ops_valid && (rc = run_prep(m, s)) != GMM_OK) return rc;
    const float *Xd = nullptr;
    if ((rc = stage_x(m, X, N, m->D, s, &Xd)) != GMM_OK) return rc;
    CK(grow(m->dstage, m->dstage_cap, (size_t)N + 1));
    // one sample per thread, as the allocation-free average, which returns this value
    CK(gmm::launch_log_p(Xd, N, m->D, m->G, m->op, g, m->dstage, s));
    CK(gmm::launch_sum_fp64(m->dstage, N, m->dstage + N, s));
    double sum = 0.0;
    CK(cudaMemcpyAsync(&sum, m->dstage + N, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    *out = sum / (double)N;
    return GMM_OK;
}

gmm_status gmm_avg_log_p_noalloc(const gmm_model *mc, const float *X, int64_t N, int32_t g, double *out,
                                 void *stream)
{
    gmm_model *m = const_cast<gmm_model *>(mc);
    if (!m || !out) return fail(GMM_ERR_ARG, "NULL argument");
    if (!m->has_params) return fail(GMM_ERR_STATE, "model has no parameters");
    gmm_status rc = validate_x(X, N, m->D);
    if (rc != GMM_OK) return rc;
    if (g < -1 || g >= m->G) return fail(GMM_ERR_ARG, "g out of range");
    if (!is_device_ptr(X)) return fail(GMM_ERR_ARG, "X must be device memory (this call stages nothing)");
    if (N > gmm::avg_log_p_noalloc_max_n())
        return fail(GMM_ERR_UNSUPPORTED, "N=%lld exceeds the allocation-free limit of %lld samples", (long long)N,
                    (long long)gmm::avg_log_p_noalloc_max_n());
    cudaStream_t s = as_stream(stream);
    if (!m->ops_valid && (rc = run_prep(m, s)) != GMM_OK) return rc;
    double sum = 0.0;
    CK(gmm::launch_avg_log_p_noalloc(X, N, m->D, m->G, m->op, g, &sum, s));
    *out = sum / (double)N;
    return GMM_OK;
}

static gmm_status assign_dev(gmm_model *m, const float *X, int64_t N, int32_t mode, cudaStream_t s, int32_t **ad)
{
    gmm_status rc = validate_x(X, N, m->D);
    if (rc != GMM_OK) return rc;
    if (mode != GMM_EUCL && mode != GMM_PROB) return fail(GMM_ERR_ARG, "assign mode must be EUCL or PROB");
    if (!m->ops_valid && (rc = run_prep(m, s)) != GMM_OK) return rc;
    const float *Xd = nullptr;
    if ((rc = stage_x(m, X, N, m->D, s, &Xd)) != GMM_OK) return rc;
    CK(grow(m->assign, m->assign_cap, (size_t)N));
    // unit weights for the exact Euclidean recheck
    std::vector<double> ones(m->D, 1.0);
    CK(cudaMemcpyAsync(m->wones(), ones.data(), sizeof(double) * m->D, cudaMemcpyHostToDevice, s));
    CK(gmm::launch_assign(Xd, N, m->D, m->G, m->par[m->cur], m->op, mode, m->assign, nullptr, m->wones(),
                          m->status, s));
    CK(cudaStreamSynchronize(s));   // `ones` is a host vector
    *ad = m->assign;
    return GMM_OK;
}

gmm_status gmm_assign(const gmm_model *mc, const float *X, int64_t N, int32_t mode, int32_t *out, void *stream)
{
    gmm_model *m = const_cast<gmm_model *>(mc);
    if (!m || !out) return fail(GMM_ERR_ARG, "NULL argument");
    if (!m->has_params) return fail(GMM_ERR_STATE, "model has no parameters");
    cudaStream_t s = as_stream(stream);
    int32_t *ad = nullptr;
    gmm_status rc = assign_dev(m, X, N, mode, s, &ad);
    if (rc != GMM_OK) return rc;
    CK(cudaMemcpyAsync(out, ad, sizeof(int32_t) * (size_t)N, cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
    return GMM_OK;
}

gmm_status gmm_raw_hist(const gmm_model *mc, const float *X, int64_t N, int32_t mode, int64_t *counts, void *stream)
{
    gmm_model *m = const_cast<gmm_model *>(mc);
    if (!m || !counts) return fail(GMM_ERR_ARG, "NULL argument");
    if (!m->has_params) return fail(GMM_ERR_STATE, "model has no parameters");
    cudaStream_t s = as_stream(stream);
    int32_t *ad = nullptr;
    gmm_status rc = assign_dev(m, X, N, mode, s, &ad);
    if (rc != GMM_OK) return rc;
    CK(grow(m->hist, m->hist_cap, (size_t)m->G));
    CK(gmm::launch_hist(ad, N, m->G, m->hist, s));
    std::vector<unsigned long long> h(m->G);
    CK(cudaMemcpyAsync(h.data(), m->hist, sizeof(unsigned long long) * m->G, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int g = 0; g < m->G; ++g) counts[g] = (int64_t)h[g];
    return GMM_OK;
}

gmm_status gmm_norm_hist(const gmm_model *mc, const float *X, int64_t N, int32_t mode, double *hist, void *stream)
{
    if (!mc || !hist) return fail(GMM_ERR_ARG, "NULL argument");
    std::vector<int64_t> c(mc->G > 0 ? mc->G : 1);
    gmm_status rc = gmm_raw_hist(mc, X, N, mode, c.data(), stream);
    if (rc != GMM_OK) return rc;
    for (int g = 0; g < mc->G; ++g) hist[g] = (double)c[g] / (double)N;
    return GMM_OK;
}

gmm_status gmm_get_params(const gmm_model *m, int32_t *D, int32_t *n_gaus, double *means, double *dcovs,
                          double *hefts)
{
    if (!m) return fail(GMM_ERR_ARG, "model is NULL");
    if (D) *D = m->has_params ? m->D : 0;
    if (n_gaus) *n_gaus = m->has_params ? m->G : 0;
    if (!m->has_params) return (means || dcovs || hefts) ? fail(GMM_ERR_STATE, "model has no parameters") : GMM_OK;
    const size_t GD = (size_t)m->G * m->D;
    const double *p = m->par[m->cur];
    if (means) CK(cudaMemcpy(means, p, sizeof(double) * GD, cudaMemcpyDeviceToHost));
    if (dcovs) CK(cudaMemcpy(dcovs, p + GD, sizeof(double) * GD, cudaMemcpyDeviceToHost));
    if (hefts) CK(cudaMemcpy(hefts, p + 2 * GD, sizeof(double) * m->G, cudaMemcpyDeviceToHost));
    return GMM_OK;
}

gmm_status gmm_set_params(gmm_model *m, int32_t D, int32_t n_gaus, const double *means, const double *dcovs,
                          const double *hefts)
{
    if (!m || !means || !dcovs || !hefts) return fail(GMM_ERR_ARG, "NULL argument");
    if (D < 1 || D > GMM_MAX_DIMS || n_gaus < 1) return fail(GMM_ERR_ARG, "bad shape (D=%d, n_gaus=%d)", D, n_gaus);
    const size_t GD = (size_t)n_gaus * D;
    for (size_t k = 0; k < GD; ++k)
        if (!(dcovs[k] > 0.0) || !std::isfinite(dcovs[k]) || !std::isfinite(means[k]))
            return fail(GMM_ERR_ARG, "dcovs must be finite and > 0, means finite");
    for (int g = 0; g < n_gaus; ++g)
        if (!(hefts[g] >= 0.0) || !std::isfinite(hefts[g])) return fail(GMM_ERR_ARG, "hefts must be finite and >= 0");
    gmm_status rc = ensure_shape(m, D, n_gaus);
    if (rc != GMM_OK) return rc;
    m->cur = 0;
    CK(cudaMemcpy(m->par[0], means, sizeof(double) * GD, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->par[0] + GD, dcovs, sizeof(double) * GD, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(m->par[0] + 2 * GD, hefts, sizeof(double) * n_gaus, cudaMemcpyHostToDevice));
    m->has_params = true;
    m->ops_valid = false;
    m->ll_hist.clear();
    return run_prep(m, nullptr);
}

gmm_status gmm_generate(const gmm_model *mc, int64_t N, uint64_t seed, float *out, void *stream)
{
    if (!mc) return fail(GMM_ERR_ARG, "model is NULL");
    if (!mc->has_params) return fail(GMM_ERR_STATE, "model has no parameters");
    if (N < 0 || (N > 0 && !out)) return fail(GMM_ERR_ARG, "need N >= 0 and an output buffer");
    if (N == 0) return GMM_OK;
    gmm_model *m = const_cast<gmm_model *>(mc);   // staging buffer only
    cudaStream_t s = as_stream(stream);
    const size_t n = (size_t)N * m->D;
    if (is_device_ptr(out)) {
        CK(gmm::launch_generate(m->par[m->cur], m->G, m->D, N, seed, out, m->sms, s));
        return GMM_OK;
    }
    CK(grow(m->xstage, m->xstage_cap, n));
    CK(gmm::launch_generate(m->par[m->cur], m->G, m->D, N, seed, m->xstage, m->sms, s));
    CK(cudaMemcpyAsync(out, m->xstage, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return GMM_OK;
}

gmm_status gmm_x_from_f64(const double *X64, int64_t count, float *X32, void *stream)
{
    if (count < 0) return fail(GMM_ERR_ARG, "count must be >= 0");
    if (count == 0) return GMM_OK;
    if (!X64 || !X32) return fail(GMM_ERR_ARG, "NULL pointer");
    if (!is_device_ptr(X64) || !is_device_ptr(X32))
        return fail(GMM_ERR_ARG, "gmm_x_from_f64 takes device memory (convert host arrays on the host)");
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(gmm::launch_f64_to_f32(X64, count, X32, sms, as_stream(stream)));
    return GMM_OK;
}

gmm_status gmm_save(const gmm_model *m, const char *path)
{
    if (!m || !path) return fail(GMM_ERR_ARG, "NULL argument");
    if (!m->has_params) return fail(GMM_ERR_STATE, "model has no parameters");
    const int32_t D = m->D, G = m->G;
    const size_t GD = (size_t)G * D;
    std::vector<double> buf(2 * GD + G);
    gmm_status rc = gmm_get_params(m, nullptr, nullptr, buf.data(), buf.data() + GD, buf.data() + 2 * GD);
    if (rc != GMM_OK) return rc;
    FILE *f = fopen(path, "wb");
    if (!f) return fail(GMM_ERR_ARG, "cannot open %s for writing", path);
    bool ok = fwrite("GMMDIAG1", 1, 8, f) == 8 && fwrite(&D, sizeof(D), 1, f) == 1 && fwrite(&G, sizeof(G), 1, f) == 1 &&
              fwrite(buf.data(), sizeof(double), buf.size(), f) == buf.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? GMM_OK : fail(GMM_ERR_ARG, "cannot write %s", path);
}

gmm_status gmm_load(gmm_model *m, const char *path)
{
    if (!m || !path) return fail(GMM_ERR_ARG, "NULL argument");
    FILE *f = fopen(path, "rb");
    if (!f) return fail(GMM_ERR_ARG, "cannot open %s", path);
    char magic[8];
    int32_t D = 0, G = 0;
    bool ok = fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "GMMDIAG1", 8) == 0 && fread(&D, sizeof(D), 1, f) == 1 &&
              fread(&G, sizeof(G), 1, f) == 1 && D >= 1 && D <= GMM_MAX_DIMS && G >= 1 && G <= (1 << 24);
    std::vector<double> buf;
    if (ok) {
        const size_t GD = (size_t)G * D;
        buf.resize(2 * GD + G);
        ok = fread(buf.data(), sizeof(double), buf.size(), f) == buf.size();
    }
    fclose(f);
    if (!ok) return fail(GMM_ERR_ARG, "%s is not a model file of this library", path);
    const size_t GD = (size_t)G * D;
    return gmm_set_params(m, D, G, buf.data(), buf.data() + GD, buf.data() + 2 * GD);
}

gmm_status gmm_profile(gmm_model *m, int32_t enable)
{
    if (!m) return fail(GMM_ERR_ARG, "model is NULL");
    m->profiling = enable != 0;
    if (!m->sstats) CK(cudaMalloc(&m->sstats, kStatWords * sizeof(unsigned long long)));
    CK(cudaMemset(m->sstats, 0, kStatWords * sizeof(unsigned long long)));
    m->ev_used = 0;
    m->pass_ms = 0.0;
    m->pass_launches = 0;
    m->launch_base = gmm::launches_total();
    return GMM_OK;
}

gmm_status gmm_profile_read(const gmm_model *m, double *pass_ms, int64_t *pass_launches, int64_t *kernel_launches)
{
    if (!m) return fail(GMM_ERR_ARG, "model is NULL");
    if (pass_ms) *pass_ms = m->pass_ms;
    if (pass_launches) *pass_launches = m->pass_launches;
    if (kernel_launches) *kernel_launches = gmm::launches_total() - m->launch_base;
    return GMM_OK;
}

gmm_status gmm_debug_set(gmm_model *m, int32_t key, int64_t value)
{
    if (!m) return fail(GMM_ERR_ARG, "model is NULL");
    if (key == GMM_DEBUG_WAIT_CYCLES) {
        if (value < 0) return fail(GMM_ERR_ARG, "wait budget must be >= 0");
        m->wait_cycles = value > 0 ? (long long)value : 2000000000LL;
    } else if (key == GMM_DEBUG_SKIP_MMA) {
        m->skip_mma = value != 0;
    } else if (key == GMM_DEBUG_KM_FORM) {
        if (value < 0 || value > 1) return fail(GMM_ERR_ARG, "k-means form must be 0 or 1");
        m->km_form = (int)value;
    } else if (key == GMM_DEBUG_FP32_FORM) {
        if (value < 0 || value > 3) return fail(GMM_ERR_ARG, "FP32 form must be 0, 1, 2 or 3");
        m->fp32_form = (int)value;
    } else if (key == GMM_DEBUG_TC_FORM) {
        if (value < 0 || value > 1) return fail(GMM_ERR_ARG, "tensor-core form must be 0 or 1");
        m->tc_form = (int)value;
    } else {
        return fail(GMM_ERR_ARG, "unknown debug key %d", key);
    }
    return GMM_OK;
}

gmm_status gmm_debug_get(const gmm_model *m, int32_t key, int64_t *value)
{
    if (!m || !value) return fail(GMM_ERR_ARG, "NULL argument");
    if (key < GMM_STAT_SCREENED || key >= GMM_STAT_SCREENED + kStatWords) return fail(GMM_ERR_ARG, "unknown key %d", key);
    unsigned long long v[kStatWords] = {0};
    if (m->sstats) CK(cudaMemcpy(v, m->sstats, sizeof v, cudaMemcpyDeviceToHost));
    *value = (int64_t)v[key - GMM_STAT_SCREENED];
    return GMM_OK;
}

gmm_status gmm_get_stats(const gmm_model *m, double *ll_hist, int32_t cap, int32_t *n)
{
    if (!m) return fail(GMM_ERR_ARG, "model is NULL");
    const int32_t k = (int32_t)m->ll_hist.size() < cap ? (int32_t)m->ll_hist.size() : cap;
    for (int32_t i = 0; i < k; ++i) ll_hist[i] = m->ll_hist[i];
    if (n) *n = k;
    return GMM_OK;
}

}  // extern "C"

// ============================================================== batched form
namespace {

// Autotuner of the batched EM pass: per shape bucket (largest D rounded up to
// 16, largest n_gaus rounded up to a power of two, log2 of the total sample
// count) the fastest (samples per work item, CTAs per SM) among a fixed set of
// candidates, timed with CUDA events on the real batch.  Results live in
// memory and, when GMM_AUTOTUNE_CACHE names a file, are appended to / read
// from it as lines "bucket chunk per_sm ms".
std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune;
bool g_tune_loaded = false;

std::string tune_bucket(int dmax, int gmax, int64_t ntot)
{
    int gq = 1;
    while (gq < gmax) gq <<= 1;
    int nq = 0;
    while ((int64_t(1) << (nq + 1)) <= ntot) ++nq;
    std::ostringstream o;
    o << "D" << ((dmax + 15) / 16 * 16) << "_G" << gq << "_N2^" << nq;
    return o.str();
}

void tune_load()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = std::getenv("GMM_AUTOTUNE_CACHE");
    if (!path) return;
    std::ifstream f(path);
    std::string key;
    int chunk, per_sm;
    double ms;
    while (f >> key >> chunk >> per_sm >> ms) g_tune[key] = {chunk, per_sm};
}

void tune_store(const std::string &key, int chunk, int per_sm, double ms)
{
    g_tune[key] = {chunk, per_sm};
    const char *path = std::getenv("GMM_AUTOTUNE_CACHE");
    if (!path) return;
    std::ofstream f(path, std::ios::app);
    f << key << " " << chunk << " " << per_sm << " " << ms << "\n";
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct BatchHost {
    std::vector<gmm::BFit> fits;
    std::vector<gmm::BItem> items;
    std::vector<int32_t> order;
    size_t partial_doubles = 0;
};

// Work items of `chunk` samples, grouped by fit; `order` lists them largest
// first (the persistent kernels draw items in that order).
void build_items(BatchHost &h, int chunk)
{
    h.items.clear();
    h.partial_doubles = 0;
    for (size_t f = 0; f < h.fits.size(); ++f) {
        gmm::BFit &F = h.fits[f];
        F.item0 = (int32_t)h.items.size();
        const size_t pd = (size_t)F.G * (1 + 2 * F.D);
        for (int64_t i0 = 0; i0 < F.N; i0 += chunk) {
            gmm::BItem it{};
            it.fit = (int32_t)f;
            it.i0 = i0;
            it.i1 = std::min<int64_t>(F.N, i0 + chunk);
            it.poff = h.partial_doubles;
            h.partial_doubles += pd;
            h.items.push_back(it);
        }
        F.n_items = (int32_t)h.items.size() - F.item0;
    }
    h.order.resize(h.items.size());
    for (size_t k = 0; k < h.items.size(); ++k) h.order[k] = (int32_t)k;
    std::stable_sort(h.order.begin(), h.order.end(), [&](int32_t a, int32_t b) {
        const gmm::BItem &A = h.items[a], &B = h.items[b];
        const gmm::BFit &FA = h.fits[A.fit], &FB = h.fits[B.fit];
        return (double)(A.i1 - A.i0) * FA.G * FA.D > (double)(B.i1 - B.i0) * FB.G * FB.D;
    });
}

}  // namespace

extern "C" gmm_status gmm_learn_batched(gmm_model *const *models, int32_t n_fits, const float *const *X,
                                        const int64_t *N, const int32_t *D, const int32_t *n_gaus, int32_t km_iter,
                                        int32_t em_iter, double var_floor, const gmm_learn_opts *opts)
{
    if (!models || !X || !N || !D || !n_gaus || n_fits < 1) return fail(GMM_ERR_ARG, "bad batch arguments");
    gmm_learn_opts o;
    gmm_default_opts(&o);
    if (opts) o = *opts;
    if (o.seed_mode != GMM_RANDOM_SUBSET) return fail(GMM_ERR_UNSUPPORTED, "batched learn seeds with random_subset");
    if (o.prec != GMM_FP32) return fail(GMM_ERR_UNSUPPORTED, "batched learn runs the FP32 form");
    if (o.dist != GMM_EUCL && o.dist != GMM_MAHA) return fail(GMM_ERR_ARG, "dist must be EUCL or MAHA");
    if (km_iter < 0 || em_iter < 0 || !(var_floor >= 0.0) || !std::isfinite(var_floor))
        return fail(GMM_ERR_ARG, "bad km_iter/em_iter/var_floor");
    int dmax = 1, gmax = 1;
    int64_t ntot = 0;
    for (int f = 0; f < n_fits; ++f) {
        if (!models[f] || !X[f]) return fail(GMM_ERR_ARG, "fit %d: NULL model or X", f);
        if (D[f] < 1 || D[f] > 64) return fail(GMM_ERR_UNSUPPORTED, "fit %d: batched fits need 1 <= D <= 64", f);
        if (n_gaus[f] < 1 || n_gaus[f] > 128 || (int64_t)n_gaus[f] > N[f])
            return fail(GMM_ERR_ARG, "fit %d: need 1 <= n_gaus <= min(N, 128)", f);
        dmax = std::max(dmax, D[f]);
        gmax = std::max(gmax, n_gaus[f]);
        ntot += N[f];
    }
    int dev = 0, sms = 0, optin = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    size_t em_sm = 0, km_sm = 0;
    for (int f = 0; f < n_fits; ++f) {
        em_sm = std::max(em_sm, gmm::b_em_smem(D[f], n_gaus[f]));
        km_sm = std::max(km_sm, gmm::b_km_smem(D[f], n_gaus[f]));
    }
    const int km_per_sm = km_sm * 2 + 4096 <= (size_t)(228 * 1024) ? 2 : 1;
    if (em_sm > (size_t)optin || km_sm > (size_t)optin) return fail(GMM_ERR_UNSUPPORTED, "batch shapes exceed shared memory");
    CK(gmm::b_prepare(em_sm, km_sm));

    // ---- device arena: per-fit buffers, descriptors, seeds, staged X
    BatchHost h;
    h.fits.resize(n_fits);
    std::vector<size_t> off(n_fits);
    size_t bytes = 0;
    std::vector<std::vector<int64_t>> seeds(n_fits);
    std::vector<bool> host_x(n_fits);
    for (int f = 0; f < n_fits; ++f) {
        const size_t G = n_gaus[f], Df = D[f], np = 2 * G * Df + G;
        off[f] = bytes;
        bytes += align_up(8 * np, 256) * 2 + align_up(8 * G * Df, 256) + align_up(4 * G * Df, 256) +
                 align_up(4 * G, 256) + align_up(8 * Df, 256) * 2 + align_up(4 * Df, 256) * 2 + align_up(8 * G, 256) +
                 align_up(4 * (size_t)N[f], 256) + align_up(8 * G, 256) + align_up(8 * (size_t)std::max(em_iter, 1), 256) +
                 align_up(sizeof(gmm::BFitStatus), 256);
        host_x[f] = !is_device_ptr(X[f]);
        if (host_x[f]) bytes += align_up(4 * (size_t)N[f] * Df, 256);
        seeds[f] = random_subset(N[f], n_gaus[f], o.seed + (uint64_t)f);
    }
    unsigned char *arena = nullptr;
    CK(cudaMalloc(&arena, bytes ? bytes : 1));
    struct ArenaGuard { unsigned char *p; ~ArenaGuard() { if (p) cudaFree(p); } } guard{arena};
    cudaStream_t s = nullptr;
    CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    struct StreamGuard { cudaStream_t s; ~StreamGuard() { if (s) cudaStreamDestroy(s); } } sguard{s};
    std::vector<gmm::BFitStatus> st0(n_fits);
    std::vector<int32_t> comp_fit, comp_g;
    for (int f = 0; f < n_fits; ++f) {
        const size_t G = n_gaus[f], Df = D[f], np = 2 * G * Df + G;
        unsigned char *p = arena + off[f];
        auto take = [&](size_t n) { unsigned char *q = p; p += align_up(n, 256); return q; };
        gmm::BFit &F = h.fits[f];
        F.N = N[f];
        F.D = D[f];
        F.G = n_gaus[f];
        F.par = reinterpret_cast<double *>(take(8 * np));
        F.par2 = reinterpret_cast<double *>(take(8 * np));
        F.sm = reinterpret_cast<float2 *>(take(8 * G * Df));
        F.mu = reinterpret_cast<float *>(take(4 * G * Df));
        F.c = reinterpret_cast<float *>(take(4 * G));
        F.gvar = reinterpret_cast<double *>(take(8 * Df));
        F.w = reinterpret_cast<double *>(take(8 * Df));
        F.sw = reinterpret_cast<float *>(take(4 * Df));
        F.center = reinterpret_cast<float *>(take(4 * Df));
        F.counts = reinterpret_cast<double *>(take(8 * G));
        F.assign = reinterpret_cast<int32_t *>(take(4 * (size_t)N[f]));
        int64_t *sidx = reinterpret_cast<int64_t *>(take(8 * G));
        F.seed_idx = sidx;
        F.ll_hist = reinterpret_cast<double *>(take(8 * (size_t)std::max(em_iter, 1)));
        F.status = reinterpret_cast<gmm::BFitStatus *>(take(sizeof(gmm::BFitStatus)));
        if (host_x[f]) {
            float *xs = reinterpret_cast<float *>(take(4 * (size_t)N[f] * Df));
            CK(cudaMemcpyAsync(xs, X[f], 4 * (size_t)N[f] * Df, cudaMemcpyHostToDevice, s));
            F.X = xs;
        } else {
            F.X = X[f];
        }
        CK(cudaMemcpyAsync(sidx, seeds[f].data(), 8 * G, cudaMemcpyHostToDevice, s));
        st0[f] = gmm::BFitStatus{0, 0, 0x7fffffff, 0, -1, {0, 0, 0}};
        for (int g = 0; g < F.G; ++g) { comp_fit.push_back(f); comp_g.push_back(g); }
    }
    const int n_comp = (int)comp_fit.size();
    // descriptors and tables in a second allocation (sized after items are known)
    gmm::BFit *d_fits = nullptr;
    int32_t *d_comp = nullptr;
    int *d_counter = nullptr;
    CK(cudaMalloc(&d_fits, sizeof(gmm::BFit) * n_fits));
    struct FreeGuard { void *p; ~FreeGuard() { if (p) cudaFree(p); } } g1{d_fits};
    CK(cudaMalloc(&d_comp, sizeof(int32_t) * 2 * n_comp));
    FreeGuard g2{d_comp};
    CK(cudaMalloc(&d_counter, sizeof(int)));
    FreeGuard g3{d_counter};
    CK(cudaMemcpyAsync(d_comp, comp_fit.data(), 4 * n_comp, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(d_comp + n_comp, comp_g.data(), 4 * n_comp, cudaMemcpyHostToDevice, s));
    gmm::BItem *d_items = nullptr;
    int32_t *d_order = nullptr;
    double *d_partial = nullptr, *d_llp = nullptr;
    size_t cap_items = 0, cap_partial = 0;
    FreeGuard g4{nullptr}, g5{nullptr}, g6{nullptr}, g7{nullptr};
    auto upload = [&](int chunk) -> gmm_status {
        build_items(h, chunk);
        if (h.items.size() > cap_items) {
            if (d_items) cudaFree(d_items);
            if (d_order) cudaFree(d_order);
            if (d_llp) cudaFree(d_llp);
            cap_items = h.items.size();
            CK(cudaMalloc(&d_items, sizeof(gmm::BItem) * cap_items));
            CK(cudaMalloc(&d_order, sizeof(int32_t) * cap_items));
            CK(cudaMalloc(&d_llp, sizeof(double) * cap_items));
            g4.p = d_items; g5.p = d_order; g6.p = d_llp;
        }
        if (h.partial_doubles > cap_partial) {
            if (d_partial) cudaFree(d_partial);
            cap_partial = h.partial_doubles;
            CK(cudaMalloc(&d_partial, sizeof(double) * cap_partial));
            g7.p = d_partial;
        }
        CK(cudaMemcpyAsync(d_items, h.items.data(), sizeof(gmm::BItem) * h.items.size(), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_order, h.order.data(), sizeof(int32_t) * h.items.size(), cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(d_fits, h.fits.data(), sizeof(gmm::BFit) * n_fits, cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));   // host vectors are reused by the next call
        return GMM_OK;
    };
    auto reset_status = [&]() -> gmm_status {
        for (int f = 0; f < n_fits; ++f)
            CK(cudaMemcpyAsync(h.fits[f].status, &st0[f], sizeof(gmm::BFitStatus), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
        return GMM_OK;
    };
    gmm_status rc;

    // ---- autotune the EM pass for this shape bucket
    int chunk = 8192, per_sm = 1;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load();
        const std::string key = tune_bucket(dmax, gmax, ntot);
        auto hit = g_tune.find(key);
        if (hit != g_tune.end()) {
            chunk = hit->second.first;
            per_sm = hit->second.second;
        } else if (em_iter > 0) {
            if ((rc = upload(8192)) != GMM_OK) return rc;
            if ((rc = reset_status()) != GMM_OK) return rc;
            CK(gmm::launch_b_gstats(d_fits, n_fits, var_floor, o.dist, s));
            CK(gmm::launch_b_seed(d_fits, d_comp, d_comp + n_comp, n_comp, s));
            CK(gmm::launch_b_em_prep(d_fits, d_comp, d_comp + n_comp, n_comp, s));
            cudaEvent_t e0, e1;
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            double best = 1e300;
            const int chunks[3] = {2048, 8192, 32768};
            for (int ci = 0; ci < 3; ++ci)
                for (int ps = 1; ps <= 2; ++ps) {
                    if (ps == 2 && em_sm * 2 + 4096 > (size_t)(228 * 1024)) continue;
                    if ((rc = upload(chunks[ci])) != GMM_OK) return rc;
                    float ms = 0.f, tot = 0.f;
                    for (int rep = 0; rep < 2; ++rep) {
                        CK(cudaEventRecord(e0, s));
                        CK(gmm::launch_b_em_pass(d_fits, d_items, d_order, (int)h.items.size(), d_counter, d_partial,
                                                 d_llp, em_sm, sms * ps, 0, s));
                        CK(cudaEventRecord(e1, s));
                        CK(cudaEventSynchronize(e1));
                        CK(cudaEventElapsedTime(&ms, e0, e1));
                        if (rep) tot += ms;
                    }
                    if (tot < best) { best = tot; chunk = chunks[ci]; per_sm = ps; }
                }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            tune_store(key, chunk, per_sm, best);
        }
    }

    // ---- the whole fit as one CUDA graph
    if ((rc = upload(chunk)) != GMM_OK) return rc;
    if ((rc = reset_status()) != GMM_OK) return rc;
    const int n_items = (int)h.items.size();
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = cudaSuccess;
    auto cap = [&](cudaError_t e) { if (ce == cudaSuccess) ce = e; };
    cap(gmm::launch_b_gstats(d_fits, n_fits, var_floor, o.dist, s));
    cap(gmm::launch_b_seed(d_fits, d_comp, d_comp + n_comp, n_comp, s));
    for (int it = 0; it < km_iter; ++it)
        cap(gmm::launch_b_km_iter(d_fits, n_fits, d_comp, d_comp + n_comp, n_comp, d_items, d_order, n_items,
                                  d_counter, d_partial, km_sm, sms * km_per_sm, var_floor, it == km_iter - 1, s));
    cap(gmm::launch_b_em_prep(d_fits, d_comp, d_comp + n_comp, n_comp, s));
    for (int it = 0; it < em_iter; ++it) {
        cap(gmm::launch_b_em_pass(d_fits, d_items, d_order, n_items, d_counter, d_partial, d_llp, em_sm, sms * per_sm,
                                  it, s));
        cap(gmm::launch_b_em_finish(d_fits, n_fits, d_comp, d_comp + n_comp, n_comp, d_items, d_partial, d_llp,
                                    var_floor, o.em_tol, it, s));
    }
    cudaError_t ee = cudaStreamEndCapture(s, &graph);
    if (ce != cudaSuccess) { if (graph) cudaGraphDestroy(graph); CK(ce); }
    CK(ee);
    struct GraphGuard { cudaGraph_t g; cudaGraphExec_t x; ~GraphGuard() { if (x) cudaGraphExecDestroy(x); if (g) cudaGraphDestroy(g); } } gg{graph, nullptr};
    CK(cudaGraphInstantiate(&exec, graph, 0));
    gg.x = exec;
    CK(cudaGraphLaunch(exec, s));
    CK(cudaStreamSynchronize(s));

    // ---- results into the models
    std::vector<gmm::BFitStatus> st(n_fits);
    int32_t first_bad = -1;
    for (int f = 0; f < n_fits; ++f) {
        CK(cudaMemcpy(&st[f], h.fits[f].status, sizeof(gmm::BFitStatus), cudaMemcpyDeviceToHost));
        gmm_model *m = models[f];
        const gmm::BFit &F = h.fits[f];
        if ((rc = ensure_shape(m, F.D, F.G)) != GMM_OK) return rc;
        int done = st[f].code ? std::max(st[f].fail_iter, 0) : st[f].n_done;
        const double *src = (done & 1) ? F.par2 : F.par;
        const size_t np = 2 * (size_t)F.G * F.D + F.G;
        CK(cudaMemcpy(m->par[0], src, 8 * np, cudaMemcpyDeviceToDevice));
        m->cur = 0;
        m->has_params = true;
        m->ops_valid = false;
        m->has_center = false;
        std::vector<double> ll(std::max(st[f].n_done, 0));
        if (!ll.empty()) CK(cudaMemcpy(ll.data(), F.ll_hist, 8 * ll.size(), cudaMemcpyDeviceToHost));
        m->ll_hist = ll;
        if (st[f].code && first_bad < 0) first_bad = f;
        if (o.print)
            for (size_t k = 0; k < ll.size(); ++k)
                fprintf(stderr, "gmm: fit %d EM iteration %zu: mean log-likelihood %.10g\n", f, k + 1, ll[k]);
    }
    for (int f = 0; f < n_fits; ++f)
        if ((rc = run_prep(models[f], nullptr)) != GMM_OK) return rc;
    CK(cudaDeviceSynchronize());
    if (first_bad >= 0)
        return fail((gmm_status)st[first_bad].code, "fit %d failed at EM iteration %d", first_bad, st[first_bad].fail_iter);
    return GMM_OK;
}

// ============================================================== learned initialiser
struct gmm_init_net {
    gmm::InitNet *net;
};

extern "C" gmm_status gmm_init_net_create(gmm_init_net **out, int32_t D, int32_t n_gaus, int32_t hidden_point,
                                          int32_t hidden_head, int32_t point_layers, int32_t head_layers, uint64_t seed)
{
    if (!out) return fail(GMM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (D < 1 || D > 64 || n_gaus < 1 || n_gaus > 64 || hidden_point < 1 || hidden_head < 1 || point_layers < 1 ||
        head_layers < 0)
        return fail(GMM_ERR_ARG, "bad network shape");
    cudaError_t e = cudaSuccess;
    gmm::InitNet *n = gmm::init_net_new(D, n_gaus, hidden_point, hidden_head, point_layers, head_layers, seed, &e);
    if (e != cudaSuccess) {
        gmm::init_net_free(n);
        return fail(GMM_ERR_CUDA, "network allocation failed: %s", cudaGetErrorString(e));
    }
    *out = new gmm_init_net{n};
    return GMM_OK;
}

extern "C" void gmm_init_net_destroy(gmm_init_net *n)
{
    if (!n) return;
    gmm::init_net_free(n->net);
    delete n;
}

extern "C" int64_t gmm_init_net_num_params(const gmm_init_net *n) { return n ? gmm::init_net_n_params(n->net) : 0; }

extern "C" gmm_status gmm_init_net_get_weights(const gmm_init_net *n, float *weights, float *grads)
{
    if (!n) return fail(GMM_ERR_ARG, "net is NULL");
    CK(gmm::init_net_get(n->net, weights, grads));
    return GMM_OK;
}

extern "C" gmm_status gmm_init_net_get_adam(const gmm_init_net *n, float *m1, float *m2, int64_t *step)
{
    if (!n) return fail(GMM_ERR_ARG, "net is NULL");
    CK(gmm::init_net_get_adam(n->net, m1, m2, step));
    return GMM_OK;
}

extern "C" gmm_status gmm_init_net_set_adam(gmm_init_net *n, const float *m1, const float *m2, int64_t step)
{
    if (!n || !m1 || !m2) return fail(GMM_ERR_ARG, "NULL argument");
    if (step < 0) return fail(GMM_ERR_ARG, "step must be >= 0");
    CK(gmm::init_net_set_adam(n->net, m1, m2, step));
    return GMM_OK;
}

extern "C" gmm_status gmm_init_net_set_weights(gmm_init_net *n, const float *weights)
{
    if (!n || !weights) return fail(GMM_ERR_ARG, "NULL argument");
    CK(gmm::init_net_set_weights(n->net, weights));
    CK(cudaDeviceSynchronize());
    return GMM_OK;
}

extern "C" gmm_status gmm_init_net_step(gmm_init_net *n, const float *pts, int32_t B, int32_t P, const double *tgt_means,
                                        const double *tgt_dcovs, const double *tgt_hefts, double lambda,
                                        double var_floor, int32_t mode, double lr, double *pred_means,
                                        double *pred_dcovs, double *pred_hefts, double *loss, void *stream)
{
    if (!n || !pts) return fail(GMM_ERR_ARG, "NULL argument");
    if (B < 1 || P < 1 || mode < 0 || mode > 2) return fail(GMM_ERR_ARG, "bad B/P/mode");
    if (!is_device_ptr(pts)) return fail(GMM_ERR_ARG, "pts must be device memory");
    if (lambda > 0.0 && !(tgt_means && tgt_dcovs && tgt_hefts)) return fail(GMM_ERR_ARG, "lambda > 0 needs targets");
    if (!(var_floor > 0.0)) return fail(GMM_ERR_ARG, "var_floor must be > 0");
    CK(gmm::init_net_run(n->net, pts, B, P, tgt_means, tgt_dcovs, tgt_hefts, lambda, var_floor, mode >= 1,
                         mode == 2 ? lr : 0.0, pred_means, pred_dcovs, pred_hefts, loss, as_stream(stream)));
    return GMM_OK;
}

extern "C" gmm_status gmm_init_net_seed_model(const gmm_init_net *nc, gmm_model *m, const float *X, int64_t N, int32_t P,
                                              uint64_t seed, double var_floor, void *stream)
{
    if (!nc || !m || !X) return fail(GMM_ERR_ARG, "NULL argument");
    gmm::InitNet *n = nc->net;
    const int D = gmm::init_net_D(n), G = gmm::init_net_G(n);
    if (N < P || P < 1) return fail(GMM_ERR_ARG, "need 1 <= P <= N");
    cudaStream_t s = as_stream(stream);
    gmm_status rc = ensure_shape(m, D, G);
    if (rc != GMM_OK) return rc;
    const float *Xd = nullptr;
    if ((rc = stage_x(m, X, N, D, s, &Xd)) != GMM_OK) return rc;
    std::vector<int64_t> idx = random_subset(N, P, seed);
    int64_t *d_idx = nullptr;
    float *d_pts = nullptr;
    double *d_par = nullptr;
    CK(cudaMalloc(&d_idx, 8 * (size_t)P));
    struct F { void *p; ~F() { if (p) cudaFree(p); } } f1{d_idx};
    CK(cudaMalloc(&d_pts, 4 * (size_t)P * D));
    F f2{d_pts};
    CK(cudaMalloc(&d_par, 8 * (2 * (size_t)G * D + G)));
    F f3{d_par};
    CK(cudaMemcpyAsync(d_idx, idx.data(), 8 * (size_t)P, cudaMemcpyHostToDevice, s));
    CK(gmm::init_net_gather(Xd, D, d_idx, P, d_pts, s));
    double loss = 0.0;
    CK(gmm::init_net_run(n, d_pts, 1, P, nullptr, nullptr, nullptr, 0.0, var_floor, 0, 0.0, d_par,
                         d_par + (size_t)G * D, d_par + 2 * (size_t)G * D, &loss, s));
    std::vector<double> h(2 * (size_t)G * D + G);
    CK(cudaMemcpy(h.data(), d_par, 8 * h.size(), cudaMemcpyDeviceToHost));
    for (double v : h)
        if (!std::isfinite(v)) return fail(GMM_ERR_NONFINITE, "the network produced non-finite parameters");
    return gmm_set_params(m, D, G, h.data(), h.data() + (size_t)G * D, h.data() + 2 * (size_t)G * D);
}
