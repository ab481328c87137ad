"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances (the FP32 CUDA-core path):
  k-means assignments  bit-exact, except samples whose two nearest oracle
                       distances differ by < 1e-6 relative
  EM parameters        1e-4 relative, with absolute floors 1e-4 * global std
                       (means), 1e-4 * global variance (dcovs), 1e-4 / G (hefts).
                       The floor on dcovs covers Gaussians that collapse onto a
                       sample: their FP64 one-pass variance is ~0 (floored),
                       FP32 sums resolve it only to ~1e-7 of the squared shift.
                       Where the oracle's FP32 error budget of the iteration
                       (oracle.em_fp32_budget: first-order bounds of an FP32
                       E-step and FP32 statistics sums, propagated through
                       Eqs. 3 and 12-14), doubled for second-order terms,
                       exceeds that tolerance, the budget is the tolerance.
                       It does so only for Gaussians fed by far, low
                       responsibilities (about < 10 samples' worth on c2).
                       A Gaussian whose responsibility sum the library found
                       below 1e-8 keeps its mean and covariance there (the
                       library's reading for vanishing mass); only its heft is
                       compared.
  one k-means step     1e-6 relative (FP32 shifted sums, FP64 reduce)
  log-likelihoods      1e-6 relative (FP32 logits, FP64 sums)
Multi-iteration runs amplify the FP32 differences of weakly supported
Gaussians from one iteration to the next, so parameters are compared one
iteration at a time from the same state (em_step_check) and trajectories by
their log-likelihoods.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1707_09094_gb300 import GMM, GMM_EUCL, GMM_KEEP_EXISTING, GMM_MAHA, GMM_PROB, GmmError, synth

pytestmark = pytest.mark.gpu

RTOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1707_09094_gb300 import build
    build.build()


def dev(X):
    return torch.from_numpy(np.ascontiguousarray(X)).cuda()


def assert_close(got, ref, rtol, atol, what):
    """|got - ref| <= atol + rtol |ref| element-wise (atol may be an array)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    err = np.abs(got - ref)
    lim = np.broadcast_to(np.asarray(atol, np.float64), ref.shape) + rtol * np.abs(ref)
    bad = ~(err <= lim)
    if bad.any():
        k = np.unravel_index(np.argmax(np.where(bad, err / np.maximum(lim, 1e-300), 0)), ref.shape)
        raise AssertionError("%s: %d of %d outside tolerance; worst at %s: got %r ref %r (limit %.3g)"
                             % (what, bad.sum(), bad.size, k, got[k], ref[k], lim[k]))


BUDGET_K = 2.0      # first-order FP32 budget, doubled for the neglected second-order terms
FROZEN_MASS = 1e-8  # below this responsibility sum the library keeps a Gaussian's mean and covariance


def assert_params(got, ref, X, rtol=RTOL, budget=None):
    """Parameters within tolerance: |got - ref| <= max(rtol |ref| + floor,
    BUDGET_K * budget) element-wise, budget = (b_means, b_dcovs, b_hefts) of
    oracle.em_fp32_budget (None: the base tolerance alone).  Means and dcovs
    of Gaussians the library froze (responsibility sum N w < 1e-8 in `got`)
    are not compared."""
    m, v, h = got
    M, V, H = ref
    gstd = X.astype(np.float64).std(axis=0)
    G = M.shape[0]
    live = (h * X.shape[0] >= FROZEN_MASS)[:, None]
    am, av, ah = (rtol * gstd)[None, :], (rtol * gstd ** 2)[None, :], rtol / G
    if budget is not None:
        bm, bv, bw = budget
        am = np.maximum(am + rtol * np.abs(M), BUDGET_K * bm) - rtol * np.abs(M)
        av = np.maximum(av + rtol * np.abs(V), BUDGET_K * bv) - rtol * np.abs(V)
        ah = np.maximum(ah + rtol * np.abs(H), BUDGET_K * bw) - rtol * np.abs(H)
    assert_close(np.where(live, m, M), M, rtol, am, "means")
    assert_close(np.where(live, v, V), V, rtol, av, "dcovs")
    assert_close(h, H, rtol, ah, "hefts")


def em_step_check(g, X, Xd, prec="fp32", var_floor=1e-10, n_acc=0, recompute_center=False):
    """One EM iteration of model g on Xd against the oracle's iteration from
    g's current parameters (the same FP64 values), within the FP32 budget."""
    start = g.get_params()
    M, V, H, ll, budget = oracle.em_fp32_budget(X, *start, var_floor, n_acc=n_acc)
    n0 = len(g.ll_history())
    g.em_iterate(Xd, 1, prec=prec, var_floor=var_floor, recompute_center=recompute_center)
    assert_params(g.get_params(), (M, V, H), X, budget=budget)
    np.testing.assert_allclose(g.ll_history()[n0:], [ll], rtol=1e-6)
    return M, V, H, budget


def near_tie_mask(b1, b2, rel=1e-6):
    return (b2 - b1) < rel * np.maximum(np.abs(b2), 1e-300)


def km_weights(X, dist, var_floor):
    _, gv = oracle.global_stats(X)
    gv = np.maximum(gv, var_floor)
    return (1.0 / gv if dist == GMM_MAHA else np.ones_like(gv)), gv


# ------------------------------------------------------------ seeding
def test_random_subset_seeds_match_oracle():
    X, _, _ = synth.make("c1", N=20000)
    g = GMM().learn(dev(X), 8, km_iter=0, em_iter=0, seed=77)
    m, v, h = g.get_params()
    idx = oracle.seed_random_subset(X.shape[0], 8, 77)
    np.testing.assert_array_equal(m, X[idx].astype(np.float64))
    assert (v == 1.0).all() and np.allclose(h, 1 / 8)


# ------------------------------------------------------------ k-means
@pytest.mark.parametrize("dist", [GMM_MAHA, GMM_EUCL])
@pytest.mark.parametrize("shape", [(100000, 10, 8), (5003, 13, 5), (129, 3, 3), (4097, 60, 37)])
def test_kmeans_one_iteration_exact(shape, dist):
    N, D, G = shape
    X, _, _ = synth.make("c1", N=N, D=D, G=G, seed=11 + N)
    seeds = synth.seeds_subset(X, G, 5)
    w, gv = km_weights(X, dist, 1e-10)
    M, V, H, A = oracle.kmeans(X, seeds, w, gv, 1, 1e-10)
    _, b1, b2 = oracle.km_assign(X, seeds, w)
    g = GMM().set_params(seeds, np.ones_like(seeds), np.full(G, 1.0 / G))
    a = g.kmeans(dev(X), 1, dist_mode=dist).cpu().numpy()
    ok = ~near_tie_mask(b1, b2)
    np.testing.assert_array_equal(a[ok], A[ok])
    if ok.all():
        assert_params(g.get_params(), (M, V, H), X, rtol=1e-6)


def test_kmeans_ten_iterations_c1():
    X, _, _ = synth.make("c1")
    seeds = synth.seeds_subset(X, 8, 9)
    w, gv = km_weights(X, GMM_MAHA, 1e-10)
    M, V, H, A = oracle.kmeans(X, seeds, w, gv, 10, 1e-10)
    g = GMM().set_params(seeds, np.ones_like(seeds), np.full(8, 1.0 / 8))
    a = g.kmeans(dev(X), 10).cpu().numpy()
    # the last iteration's distances, from the oracle's means before it
    Mprev = oracle.kmeans(X, seeds, w, gv, 9, 1e-10)[0]
    _, b1, b2 = oracle.km_assign(X, Mprev, w)
    ok = ~near_tie_mask(b1, b2)
    np.testing.assert_array_equal(a[ok], A[ok])
    assert_params(g.get_params(), (M, V, H), X)


def test_kmeans_dead_mean_resurrection_gpu():
    X = np.array([[0.0], [0.1], [0.2], [10.0], [10.1]], np.float32)
    seeds = np.array([[0.1], [10.05], [1e6]])
    g = GMM().set_params(seeds, np.ones_like(seeds), np.full(3, 1 / 3))
    g.kmeans(dev(X), 1, dist_mode=GMM_EUCL, var_floor=1e-10)
    w, gv = km_weights(X, GMM_EUCL, 1e-10)
    M, V, H, A = oracle.kmeans(X, seeds, w, gv, 1, 1e-10)
    m, v, h = g.get_params()
    np.testing.assert_allclose(m, M, rtol=1e-12)
    np.testing.assert_allclose(v, V, rtol=1e-6)
    np.testing.assert_allclose(h, H, rtol=1e-15)


# ------------------------------------------------------------ EM (FP32 form)
def _start(X, G, seed):
    seeds = synth.seeds_subset(X, G, seed)
    w, gv = km_weights(X, GMM_MAHA, 1e-10)
    return oracle.kmeans(X, seeds, w, gv, 5, 1e-10)[:3]


@pytest.mark.parametrize("shape", [(100000, 10, 8), (7, 3, 2), (33, 1, 3), (1000, 13, 1), (2049, 60, 40),
                                   (3001, 64, 17)])
def test_em_iterations_match_oracle(shape):
    N, D, G = shape
    X, _, _ = synth.make("c1", N=N, D=D, G=G, seed=3 + N)
    start = _start(X, G, 2) if G > 1 and N > 50 else (synth.seeds_subset(X, G, 1), np.ones((G, D)),
                                                      np.full(G, 1.0 / G))
    n_iter = 3
    M, V, H, ll = oracle.em_iterate(X, *start, n_iter, 1e-10)
    g = GMM().set_params(*start)
    g.em_iterate(dev(X), n_iter, var_floor=1e-10, recompute_center=True)
    assert_params(g.get_params(), (M, V, H), X)
    np.testing.assert_allclose(g.ll_history(), ll, rtol=1e-6, atol=1e-6)


def test_single_gaussian_closed_form_gpu():
    rng = np.random.default_rng(4)
    X = rng.normal(3.0, 2.0, (20011, 6)).astype(np.float32)
    g = GMM().set_params(np.zeros((1, 6)), np.ones((1, 6)), np.ones(1))
    g.em_iterate(dev(X), 1, recompute_center=True)
    m, v, h = g.get_params()
    Xd = X.astype(np.float64)
    np.testing.assert_allclose(m[0], Xd.mean(axis=0), rtol=1e-6)
    np.testing.assert_allclose(v[0], Xd.var(axis=0), rtol=1e-5)
    assert h[0] == pytest.approx(1.0, abs=1e-12)


def test_learn_end_to_end_c1_matches_oracle():
    X, _, _ = synth.make("c1")
    g = GMM().learn(dev(X), 8, km_iter=10, em_iter=10, seed=1001, var_floor=1e-10)
    M, V, H, ll = oracle.learn(X, 8, seed=1001, km_iter=10, em_iter=10, var_floor=1e-10)
    assert_params(g.get_params(), (M, V, H), X)
    np.testing.assert_allclose(g.ll_history(), ll, rtol=1e-6)
    assert (np.diff(g.ll_history()) >= -1e-6).all()


def test_learn_accepts_host_input_and_em_tol():
    X, _, _ = synth.make("c1", N=30000)
    g = GMM().learn(X, 8, km_iter=5, em_iter=50, seed=3, em_tol=1e-6)
    M, V, H, ll = oracle.learn(X, 8, seed=3, km_iter=5, em_iter=50, em_tol=1e-6)
    assert len(g.ll_history()) == len(ll)
    assert_params(g.get_params(), (M, V, H), X)


def test_variance_floor_and_constant_dimension():
    X, _, _ = synth.make("c1", N=20000)
    X[:, 2] = 1.5
    g = GMM().learn(dev(X), 8, km_iter=3, em_iter=3, seed=5, var_floor=1e-3)
    _, v, _ = g.get_params()
    assert (v >= 1e-3).all()
    np.testing.assert_allclose(v[:, 2], 1e-3)


def test_nonfinite_input_is_reported_and_model_kept():
    X, _, _ = synth.make("c1", N=5000)
    g = GMM().learn(dev(X), 4, km_iter=2, em_iter=2, seed=1)
    before = g.get_params()
    Xb = X.copy()
    Xb[17, 3] = np.nan
    with pytest.raises(GmmError) as e:
        g.em_iterate(dev(Xb), 2)
    assert e.value.status == -2
    after = g.get_params()
    for a, b in zip(before, after):
        np.testing.assert_array_equal(a, b)


def test_argument_errors():
    X, _, _ = synth.make("c1", N=100)
    with pytest.raises(GmmError) as e:
        GMM().learn(dev(X), 101)
    assert e.value.status == -1
    with pytest.raises(GmmError) as e:
        GMM().learn(dev(X), 4, seed_mode=GMM_KEEP_EXISTING)
    assert e.value.status == -6


# ------------------------------------------------------------ inference
@pytest.mark.parametrize("shape", [(10000, 10, 8), (333, 60, 256), (65, 1, 1), (1000, 128, 5)])
def test_log_p_and_assign_match_oracle(shape):
    N, D, G = shape
    X, _, mix = synth.make("c1", N=N, D=D, G=G, seed=21 + D)
    m, v, h = mix.means, mix.stds ** 2, mix.hefts
    g = GMM().set_params(m, v, h)
    Xd = dev(X)
    lp = g.log_p(Xd).cpu().numpy()
    ref = oracle.log_p(X, m, v, h)
    np.testing.assert_allclose(lp, ref, rtol=1e-6, atol=1e-5)
    for k in (0, G - 1):
        np.testing.assert_allclose(g.log_p(Xd, k).cpu().numpy(), oracle.log_p(X, m, v, h, g=k), rtol=1e-6, atol=1e-5)
    assert g.avg_log_p(Xd) == pytest.approx(ref.mean(), rel=1e-6)
    a_e = g.assign(Xd, GMM_EUCL).cpu().numpy()
    _, b1, b2 = oracle.km_assign(X, m, np.ones(D))
    ok = ~near_tie_mask(b1, b2)
    np.testing.assert_array_equal(a_e[ok], oracle.assign(X, m, v, h, 0)[ok])
    a_p = g.assign(Xd, GMM_PROB).cpu().numpy()
    lt = np.stack([np.log(h[k]) + oracle.log_p(X, m, v, h, g=k) for k in range(G)], axis=1)
    srt = np.sort(lt, axis=1)
    ok = (srt[:, -1] - srt[:, -2]) > 1e-4 * np.abs(srt[:, -1]) + 1e-4 if G > 1 else np.ones(N, bool)
    np.testing.assert_array_equal(a_p[ok], oracle.assign(X, m, v, h, 2)[ok])
    hist = g.raw_hist(Xd, GMM_EUCL)
    np.testing.assert_array_equal(hist, np.bincount(a_e, minlength=G))
    np.testing.assert_allclose(g.norm_hist(Xd, GMM_EUCL), hist / N)


@pytest.mark.parametrize("shape", [(4000, 6, 5), (3000, 128, 300)])
def test_zero_heft_gaussian_first(shape):
    """A Gaussian with heft exactly 0 (log w = -inf; EM produces one when no
    sample of the data gives it any responsibility) placed first: log p,
    avg_log_p, the allocation-free average, prob assignment and an EM
    iteration (the one-pass form, and the two-phase form for the 128 x 300
    shape) all equal the oracle's, which takes log 0 = -inf exactly."""
    import ctypes
    from paper_1707_09094_gb300 import _lib
    N, D, G = shape
    X, _, mix = synth.make("c1", N=N, D=D, G=G, seed=12)
    h = mix.hefts.copy()
    h[0] = 0.0
    h /= h.sum()
    m, v = mix.means, mix.stds ** 2
    Xd = dev(X)
    g = GMM().set_params(m, v, h)
    ref = oracle.log_p(X, m, v, h)
    np.testing.assert_allclose(g.log_p(Xd).cpu().numpy(), ref, rtol=1e-6, atol=1e-5)
    assert g.avg_log_p(Xd) == pytest.approx(ref.mean(), rel=1e-6)
    out = ctypes.c_double()
    assert _lib.load().gmm_avg_log_p_noalloc(g._h, ctypes.c_void_p(Xd.data_ptr()), N, -1, ctypes.byref(out),
                                            None) == 0
    assert out.value == pytest.approx(ref.mean(), rel=1e-6)
    assert (g.assign(Xd, GMM_PROB).cpu().numpy() != 0).all()
    M, V, H, ll = oracle.em_iterate(X, m, v, h, 1, 1e-10)
    g.em_iterate(Xd, 1, recompute_center=True)
    np.testing.assert_allclose(g.ll_history(), ll, rtol=1e-6)
    assert g.get_params()[2][0] == 0.0 and H[0] == 0.0


# ------------------------------------------------------------ full size (c2)
@pytest.fixture(scope="module")
def c2():
    X, lab, mix = synth.make("c2")
    return X, dev(X), mix


@pytest.mark.parametrize("form", [0, 1])
def test_c2_full_size_em_iteration_fp32(c2, form):
    """One FP32 EM iteration at the benchmark's full size (N=2e6, D=60,
    G=256), compared with the oracle run over the same data (MapReduce
    chunks across the host cores): the default FP32 form at this shape (the
    register-blocked one) and the one-pass form (GMM_DEBUG_FP32_FORM = 1)."""
    from paper_1707_09094_gb300._lib import GMM_DEBUG_FP32_FORM
    X, Xd, mix = c2
    start = (mix.means, mix.stds ** 2 * 1.2, mix.hefts)
    start = tuple(np.array(a, dtype=np.float64) for a in start)
    g = GMM().set_params(*start).debug_set(GMM_DEBUG_FP32_FORM, form)
    em_step_check(g, X, Xd, recompute_center=True)


def test_c2_full_size_log_p_sampled(c2):
    X, Xd, mix = c2
    m, v, h = mix.means, mix.stds ** 2, mix.hefts
    g = GMM().set_params(m, v, h)
    lp = g.log_p(Xd).cpu().numpy()
    idx = np.random.default_rng(0).choice(X.shape[0], 4000, replace=False)
    np.testing.assert_allclose(lp[idx], oracle.log_p(X[idx], m, v, h), rtol=1e-6, atol=1e-5)


# ------------------------------------------------------------ large N_G * D
@pytest.mark.parametrize("form", [2, 3])
@pytest.mark.parametrize("shape", [(100000, 10, 8), (20000, 60, 256), (3001, 64, 17), (160, 16, 16), (30, 3, 2),
                                   (5000, 33, 65)])
def test_register_blocked_form_on_small_shapes(shape, form):
    """The register-blocked two-phase form forced onto shapes the one-pass
    form would take: N_G below one 64-Gaussian block, partial blocks, D not a
    multiple of 4 or 8, a single short tile; with the log-densities recorded
    in the first phase (GMM_DEBUG_FP32_FORM = 2) and recomputed in the second
    (3).  Each iteration equals the oracle's."""
    from paper_1707_09094_gb300._lib import GMM_DEBUG_FP32_FORM
    N, D, G = shape
    X, _, _ = synth.make("c1", N=N, D=D, G=G, seed=11 + N)
    start = _start(X, G, 4)
    Xd = dev(X)
    g = GMM().set_params(*start).debug_set(GMM_DEBUG_FP32_FORM, form)
    g.em_iterate(Xd, 0, recompute_center=True)
    for _ in range(2):
        em_step_check(g, X, Xd)


@pytest.mark.parametrize("part", [1.0, 0.3])
def test_register_blocked_records_overflow(part):
    """Overlapping Gaussians: a sample near 100 overlapping means has more
    candidates in a 64-Gaussian block than its record holds (8), so it is
    gathered and its responsibilities are recomputed in the second phase;
    all samples (part 1.0) or 30 % of them (0.3, the rest near 60 others).
    Each iteration equals the oracle's."""
    from paper_1707_09094_gb300._lib import GMM_DEBUG_FP32_FORM
    rng = np.random.default_rng(9)
    N, D = 6000, 8
    X = rng.normal(0, 1, (N, D)).astype(np.float32)
    n_near = int(part * N)
    X[:n_near] += 40.0
    means = 40.0 + rng.normal(0, 0.05, (100, D))
    if part < 1.0:
        means = np.concatenate([means, rng.normal(0, 0.5, (60, D))])
    G = means.shape[0]
    g = GMM().set_params(means, np.ones((G, D)), np.full(G, 1.0 / G)).debug_set(GMM_DEBUG_FP32_FORM, 2)
    Xd = dev(X)
    g.em_iterate(Xd, 0, recompute_center=True)
    for _ in range(2):
        em_step_check(g, X, Xd)


@pytest.mark.parametrize("shape", [(6000, 128, 300), (8000, 100, 600), (30000, 17, 2500)])
def test_two_phase_em_matches_oracle(shape):
    """Shapes whose per-CTA statistics exceed shared memory run the two-phase
    FP32 form (partial log-sum-exps per block of 64 Gaussians and their merge,
    then responsibilities and statistics per block; D = 17 takes the
    unaligned staging path, N_G = 2500 a partial last block).  Started from
    k-means (>= 10 samples per Gaussian, as the paper recommends): from unit
    variances in 100+ dimensions the log-densities reach thousands of nats and
    FP32 resolves responsibilities only to ~1e-3."""
    N, D, G = shape
    X, _, _ = synth.make("c1", N=N, D=D, G=G, seed=7 + G)
    start = _start(X, G, 3)
    M, V, H, ll = oracle.em_iterate(X, *start, 2, 1e-10)
    Xd = dev(X)
    g = GMM().set_params(*start)
    g.em_iterate(Xd, 2, recompute_center=True)
    rtol = 1e-6 if N >= 10 * G else 1e-5
    np.testing.assert_allclose(g.ll_history(), ll, rtol=rtol)
    # parameters, one iteration at a time from the same state
    g = GMM().set_params(*start)
    g.em_iterate(Xd, 0, recompute_center=True)
    for _ in range(2):
        em_step_check(g, X, Xd)


@pytest.mark.parametrize("dist", [GMM_MAHA, GMM_EUCL])
@pytest.mark.parametrize("shape", [(5000, 128, 300), (3001, 100, 40), (4000, 17, 400), (777, 65, 64), (90, 70, 3)])
def test_kmeans_register_blocked_exact(shape, dist):
    """Shapes beyond the tiled form (D > 64 or N_G > 256) take the
    register-blocked k-means (blocks of 64 means, partial best two per block,
    merged, near ties re-decided in FP64): the assignment equals the FP64
    argmin away from near ties, and the updated parameters the oracle's."""
    N, D, G = shape
    X, _, _ = synth.make("c1", N=N, D=D, G=G, seed=9 + N)
    seeds = synth.seeds_subset(X, G, 4)
    w, gv = km_weights(X, dist, 1e-10)
    M, V, H, A = oracle.kmeans(X, seeds, w, gv, 1, 1e-10)
    _, b1, b2 = oracle.km_assign(X, seeds, w)
    g = GMM().set_params(seeds, np.ones_like(seeds), np.full(G, 1.0 / G))
    a = g.kmeans(dev(X), 1, dist_mode=dist).cpu().numpy()
    ok = ~near_tie_mask(b1, b2)
    np.testing.assert_array_equal(a[ok], A[ok])
    if ok.all():
        assert_params(g.get_params(), (M, V, H), X, rtol=1e-6)


def test_c3_full_size_fp32_properties_and_sampled_log_p():
    """N=1e7, D=128, N_G=1024 (the precision workload) through learn(): the
    per-iteration log-likelihood never decreases, hefts sum to one, the floor
    holds, and sampled per-sample log-densities match the oracle's under the
    learned parameters."""
    X, _, _ = synth.make("c3")
    Xd = dev(X)
    g = GMM().learn(Xd, 1024, km_iter=2, em_iter=3, seed=1003, var_floor=1e-10)
    ll = g.ll_history()
    assert len(ll) == 3 and np.isfinite(ll).all()
    assert (np.diff(ll) >= -1e-6 * np.abs(ll[1:])).all()
    m, v, h = g.get_params()
    assert h.sum() == pytest.approx(1.0, abs=1e-6)   # FP32 responsibility sums over 1e7 samples
    assert (v >= 1e-10).all()
    idx = np.random.default_rng(1).choice(X.shape[0], 300, replace=False)
    lp = g.log_p(Xd).cpu().numpy()[idx]
    np.testing.assert_allclose(lp, oracle.log_p(X[idx], m, v, h), rtol=1e-5, atol=1e-4)
    del Xd
    torch.cuda.empty_cache()


def test_c3_prefix_em_iteration_matches_oracle():
    """The precision workload's shape and value distributions (D=128,
    N_G=1024, means ~ N(0, 3^2), sigma log-uniform on [0.1, 10]) on 200,000
    samples: from a k-means start, one EM iteration against the oracle's
    iteration from the same parameters, every Gaussian within 1e-4 or its
    FP32 budget, the log-likelihood within 1e-6."""
    X, _, _ = synth.make("c3", N=200_000)
    Xd = dev(X)
    g = GMM().learn(Xd, 1024, km_iter=3, em_iter=0, seed=1003, var_floor=1e-10)
    em_step_check(g, X, Xd)


# ------------------------------------------------------------ other seed modes (Sec. 4.1)
@pytest.mark.parametrize("dist", [GMM_MAHA, GMM_EUCL])
@pytest.mark.parametrize("mode", ["static_subset", "static_spread", "random_spread"])
def test_seed_modes_match_oracle(mode, dist):
    """The same seed samples as the oracle (the spread modes' FP64 distances
    are taken in the oracle's order, so the farthest-first choices agree
    exactly), then a short learn from them within the FP32 tolerances."""
    from paper_1707_09094_gb300 import GMM_RANDOM_SPREAD, GMM_STATIC_SPREAD, GMM_STATIC_SUBSET
    sm = {"static_subset": GMM_STATIC_SUBSET, "static_spread": GMM_STATIC_SPREAD,
          "random_spread": GMM_RANDOM_SPREAD}[mode]
    X, _, _ = synth.make("c1", N=20000, seed=31)
    g = GMM().learn(dev(X), 8, dist_mode=dist, seed_mode=sm, km_iter=0, em_iter=0, seed=11)
    M, V, H, _ = oracle.learn(X, 8, dist_mode=dist, seed_mode=sm, seed=11, km_iter=0, em_iter=0)
    m, v, h = g.get_params()
    np.testing.assert_array_equal(m, M)
    np.testing.assert_array_equal(v, V)
    np.testing.assert_array_equal(h, H)
    Xd = dev(X)
    g2 = GMM().learn(Xd, 8, dist_mode=dist, seed_mode=sm, km_iter=3, em_iter=3, seed=11)
    M2, V2, H2, ll = oracle.learn(X, 8, dist_mode=dist, seed_mode=sm, seed=11, km_iter=3, em_iter=3)
    np.testing.assert_allclose(g2.ll_history(), ll, rtol=1e-6)
    # k-means from these seeds, then the EM iterations one at a time
    g3 = GMM().learn(Xd, 8, dist_mode=dist, seed_mode=sm, km_iter=3, em_iter=0, seed=11)
    M3, V3, H3, _ = oracle.learn(X, 8, dist_mode=dist, seed_mode=sm, seed=11, km_iter=3, em_iter=0)
    assert_params(g3.get_params(), (M3, V3, H3), X)
    for _ in range(3):
        em_step_check(g3, X, Xd)


def test_spread_seeds_many_gaussians():
    X, _, _ = synth.make("c1", N=200_000, D=10, G=64, seed=32)
    from paper_1707_09094_gb300 import GMM_STATIC_SPREAD
    g = GMM().learn(dev(X), 64, seed_mode=GMM_STATIC_SPREAD, km_iter=0, em_iter=0)
    _, gv = oracle.global_stats(X)
    idx = oracle.seed_spread(X, 64, 1.0 / np.maximum(gv, 1e-10), 0)
    np.testing.assert_array_equal(g.get_params()[0], X[idx].astype(np.float64))


# ------------------------------------------------------------ generate, save, load (Sec. 4.1)
def test_generate_matches_oracle_and_save_load_roundtrip(tmp_path):
    """The same counter-based uniforms on both sides: labels identical and
    values equal up to the last bits of the math library (FP64 log, cos, sin
    rounded to float); host and device outputs equal; save + load restores
    the parameters exactly; a bad file is rejected and leaves the model."""
    _, _, mix = synth.make("c1", N=1000)
    g = GMM().set_params(mix.means, mix.stds ** 2, mix.hefts)
    Y = g.generate(100_000, seed=7).cpu().numpy()
    Yr, _ = oracle.generate(mix.means, mix.stds ** 2, mix.hefts, 100_000, seed=7)
    np.testing.assert_allclose(Y, Yr, rtol=1e-6, atol=1e-6)
    np.testing.assert_array_equal(g.generate(1000, seed=7, device=None), Y[:1000])
    path = tmp_path / "model.gmm"
    g.save(path)
    h = GMM().load(path)
    for a, b in zip(g.get_params(), h.get_params()):
        np.testing.assert_array_equal(a, b)
    bad = tmp_path / "bad.gmm"
    bad.write_bytes(b"GMMDIAG0" + bytes(16))
    with pytest.raises(GmmError) as e:
        h.load(bad)
    assert e.value.status == -1
    for a, b in zip(g.get_params(), h.get_params()):
        np.testing.assert_array_equal(a, b)


# ------------------------------------------------------------ FP64 sample data
def test_fp64_samples_round_to_fp32_on_the_device():
    """The paper's double input: CUDA float64 samples are rounded to nearest
    FP32 by the library's kernel (compared bit for bit with numpy's rounding,
    including overflow to inf and subnormals), and a fit on them equals the
    fit on the rounded samples."""
    import ctypes
    from paper_1707_09094_gb300 import _lib
    rng = np.random.default_rng(1)
    v = np.concatenate([rng.normal(0, 3, 10000), [1e300, -1e300, 1e-310, 3.4e38, 1.0 + 2.0 ** -30, np.nan]])
    t = torch.from_numpy(v).cuda()
    out = torch.empty(v.size, dtype=torch.float32, device="cuda")
    _lib.check(_lib.load().gmm_x_from_f64(ctypes.c_void_p(t.data_ptr()), v.size, ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(0)), "gmm_x_from_f64")
    torch.cuda.synchronize()
    with np.errstate(over="ignore"):
        ref = v.astype(np.float32)
    got = out.cpu().numpy()
    fin = ~np.isnan(ref)
    np.testing.assert_array_equal(got[fin].view(np.uint32), ref[fin].view(np.uint32))
    assert np.isnan(got[~fin]).all()

    X, _, _ = synth.make("c1", N=20000)
    X64 = X.astype(np.float64) + rng.normal(0, 1e-6, X.shape)
    X32 = X64.astype(np.float32)
    M, V, H, ll = oracle.learn(X32, 8, seed=5, km_iter=3, em_iter=3, var_floor=1e-10)
    for Xin in (torch.from_numpy(X64).cuda(), X64):
        g = GMM().learn(Xin, 8, km_iter=3, em_iter=3, seed=5, var_floor=1e-10)
        assert_params(g.get_params(), (M, V, H), X32)
