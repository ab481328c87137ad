"""Pins for the FP64 oracle: it is checked against what the paper and the
mathematics fix -- closed forms, invariants, library routines and brute force
on tiny inputs -- never against itself or the CUDA path."""
import os

import numpy as np
import pytest
import scipy.optimize
import scipy.stats

import oracle
from paper_1707_09094_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _rand_model(rng, G, D, spread=3.0):
    means = rng.normal(0, spread, (G, D))
    dcovs = rng.uniform(0.3, 2.0, (G, D))
    hefts = rng.dirichlet(np.ones(G))
    return means, dcovs, hefts


# ---------------------------------------------------------------- Eq. 2 / 15
def test_log_gauss_matches_scipy_and_bruteforce():
    rng = np.random.default_rng(1)
    for D in (1, 3, 7):
        mu = rng.normal(0, 2, D)
        var = rng.uniform(0.2, 3.0, D)
        x = rng.normal(0, 2, D).astype(np.float32)
        got = oracle.log_gauss(x, mu, var)
        ref = scipy.stats.multivariate_normal(mean=mu, cov=np.diag(var)).logpdf(x.astype(np.float64))
        assert got == pytest.approx(ref, rel=1e-13, abs=1e-13)
        # Eq. 2 written out, non-log, in long double
        xl = x.astype(np.longdouble)
        dens = np.prod(1.0 / np.sqrt(2 * np.pi * var.astype(np.longdouble))) * \
            np.exp(-0.5 * np.sum((xl - mu) ** 2 / var))
        assert got == pytest.approx(float(np.log(dens)), rel=1e-12, abs=1e-12)


# ------------------------------------------------------------- Eqs. 16-18
def test_log_add_closed_forms():
    assert oracle.log_add(np.log(2.0), np.log(3.0)) == pytest.approx(np.log(5.0), rel=1e-15)
    assert oracle.log_add(np.log(3.0), np.log(2.0)) == pytest.approx(np.log(5.0), rel=1e-15)
    assert oracle.log_add(-np.inf, 1.5) == 1.5
    assert oracle.log_add(1.5, -np.inf) == 1.5
    assert oracle.log_add(-np.inf, -np.inf) == -np.inf
    # far apart: the smaller one vanishes, no overflow from exp of a big gap
    assert oracle.log_add(-1000.0, 0.0) == 0.0
    assert oracle.log_add(800.0, 800.0) == pytest.approx(800.0 + np.log(2.0), rel=1e-15)


def test_mixture_log_p_bruteforce_and_cross_forms():
    rng = np.random.default_rng(2)
    for (N, D, G) in ((20, 1, 1), (30, 2, 3), (40, 4, 4)):
        m, v, h = _rand_model(rng, G, D, spread=1.0)
        X = rng.normal(0, 1.5, (N, D)).astype(np.float32)
        lp = oracle.log_p(X, m, v, h)
        lp2 = oracle.log_p(X, m, v, h, maxsum=True)
        np.testing.assert_allclose(lp, lp2, rtol=1e-14, atol=1e-14)
        # Eq. 1 with Eq. 2, non-log, long double
        Xl = X.astype(np.longdouble)
        dens = np.zeros(N, np.longdouble)
        for g in range(G):
            norm = np.prod(1.0 / np.sqrt(2 * np.pi * v[g].astype(np.longdouble)))
            dens += h[g] * norm * np.exp(-0.5 * np.sum((Xl - m[g]) ** 2 / v[g], axis=1))
        np.testing.assert_allclose(lp, np.log(dens).astype(np.float64), rtol=1e-12, atol=1e-12)
        # per-Gaussian form: N(x|g) without heft
        for g in range(G):
            ref = scipy.stats.multivariate_normal(mean=m[g], cov=np.diag(v[g])).logpdf(
                X.astype(np.float64))
            np.testing.assert_allclose(oracle.log_p(X, m, v, h, g=g), np.atleast_1d(ref),
                                       rtol=1e-12, atol=1e-12)
        assert oracle.avg_log_p(X, m, v, h) == pytest.approx(lp.mean(), rel=1e-14)


def test_log_p_underflow_robust():
    # Far-away samples: direct densities underflow to 0 in double, the log
    # domain form stays finite (Sec. 2.2).
    m = np.array([[0.0], [1.0]])
    v = np.array([[1e-4], [1e-4]])
    h = np.array([0.5, 0.5])
    X = np.array([[500.0]], np.float32)
    lp = oracle.log_p(X, m, v, h)
    assert np.isfinite(lp).all()
    ref = np.logaddexp(np.log(0.5) + scipy.stats.norm(0, 1e-2).logpdf(500.0),
                       np.log(0.5) + scipy.stats.norm(1, 1e-2).logpdf(500.0))
    assert lp[0] == pytest.approx(ref, rel=1e-12)


# ------------------------------------------------------------------- Eq. 3
def test_posteriors_sum_to_one_and_bruteforce():
    rng = np.random.default_rng(3)
    G, D, N = 4, 3, 50
    m, v, h = _rand_model(rng, G, D, spread=1.0)
    X = rng.normal(0, 1.5, (N, D)).astype(np.float32)
    post = oracle.posteriors(X, m, v, h)
    np.testing.assert_allclose(post.sum(axis=1), 1.0, atol=1e-15 * G * 4)
    assert (post >= 0).all() and (post <= 1).all()
    Xl = X.astype(np.longdouble)
    num = np.zeros((N, G), np.longdouble)
    for g in range(G):
        norm = np.prod(1.0 / np.sqrt(2 * np.pi * v[g].astype(np.longdouble)))
        num[:, g] = h[g] * norm * np.exp(-0.5 * np.sum((Xl - m[g]) ** 2 / v[g], axis=1))
    ref = (num / num.sum(axis=1, keepdims=True)).astype(np.float64)
    np.testing.assert_allclose(post, ref, rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------- Eqs. 4-14
def test_single_gaussian_is_sample_mean_and_variance():
    rng = np.random.default_rng(4)
    X = (rng.normal(3.0, 2.0, (5000, 6))).astype(np.float32)
    m0 = np.zeros((1, 6)); v0 = np.ones((1, 6)); h0 = np.ones(1)
    m, v, h, ll = oracle.em_iterate(X, m0, v0, h0, 1, 1e-10)
    Xd = X.astype(np.float64)
    np.testing.assert_allclose(m[0], Xd.mean(axis=0), rtol=1e-12)
    np.testing.assert_allclose(v[0], Xd.var(axis=0, ddof=0), rtol=1e-10)
    assert h[0] == pytest.approx(1.0, abs=1e-15)
    # the likelihood reported is that of the starting parameters
    ref = scipy.stats.multivariate_normal(mean=np.zeros(6), cov=np.eye(6)).logpdf(Xd).mean()
    assert ll[0] == pytest.approx(ref, rel=1e-12)


def test_mstep_is_weighted_mean_and_variance():
    rng = np.random.default_rng(5)
    G, D, N = 3, 4, 3000
    m0, v0, h0 = _rand_model(rng, G, D, spread=2.0)
    X = rng.normal(0, 2.0, (N, D)).astype(np.float32)
    post = oracle.posteriors(X, m0, v0, h0)
    m, v, h, _ = oracle.em_iterate(X, m0, v0, h0, 1, 0.0)
    Xd = X.astype(np.float64)
    for g in range(G):
        mu = np.average(Xd, axis=0, weights=post[:, g])
        var = np.average((Xd - mu) ** 2, axis=0, weights=post[:, g])
        np.testing.assert_allclose(m[g], mu, rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(v[g], var, rtol=1e-9)
    np.testing.assert_allclose(h, post.mean(axis=0), rtol=1e-12)
    assert h.sum() == pytest.approx(1.0, abs=1e-13)


def test_one_pass_matches_two_pass_within_cancellation_bound():
    X, _, _ = synth.make("c1", N=4000)
    rng = np.random.default_rng(6)
    G = 8
    m0 = X[rng.choice(X.shape[0], G, replace=False)].astype(np.float64)
    v0 = np.ones((G, X.shape[1])); h0 = np.full(G, 1.0 / G)
    m1, v1, h1, _ = oracle.em_iterate(X, m0, v0, h0, 1, 1e-10)
    m2, v2, h2 = oracle.em_step_twopass(X, m0, v0, h0, 1e-10)
    np.testing.assert_allclose(m1, m2, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(h1, h2, rtol=1e-12)
    eps = np.finfo(np.float64).eps
    bound = 64 * eps * (m2 ** 2 + v2)      # one-pass error ~ eps * E[x^2]
    assert (np.abs(v1 - v2) <= bound).all()


def test_mapreduce_chunks_equal_single_pass():
    X, _, _ = synth.make("c1", N=5000)
    rng = np.random.default_rng(7)
    m0 = X[rng.choice(5000, 8, replace=False)].astype(np.float64)
    v0 = np.ones((8, 10)); h0 = np.full(8, 1 / 8)
    a = oracle.em_iterate(X, m0, v0, h0, 3, 1e-10, n_chunks=1)
    b = oracle.em_iterate(X, m0, v0, h0, 3, 1e-10, n_chunks=7)
    for u, w in zip(a, b):
        np.testing.assert_allclose(u, w, rtol=1e-11, atol=1e-13)


def test_em_loglik_non_decreasing_and_floor():
    X, _, _ = synth.make("c1", N=20000)
    rng = np.random.default_rng(8)
    m0 = X[rng.choice(20000, 8, replace=False)].astype(np.float64)
    v0 = np.ones((8, 10)); h0 = np.full(8, 1 / 8)
    m, v, h, ll = oracle.em_iterate(X, m0, v0, h0, 15, 1e-10)
    assert (np.diff(ll) >= -1e-12 * np.abs(ll[1:])).all()
    # the final parameters are at least as good as the last E-step's
    assert oracle.avg_log_p(X, m, v, h) >= ll[-1] - 1e-12 * abs(ll[-1])
    assert h.sum() == pytest.approx(1.0, abs=1e-12)
    # floor: a constant dimension gets exactly the floor
    Xc = X.copy(); Xc[:, 3] = 1.25
    _, vc, _, _ = oracle.em_iterate(Xc, m0, v0, h0, 3, 1e-3)
    assert (vc >= 1e-3).all()
    assert np.allclose(vc[:, 3], 1e-3)


def _q_function(X, post, m, v, h):
    """Appendix A's Q(theta | theta_old) for diagonal Gaussians, FP64."""
    Xd = X.astype(np.float64)
    q = 0.0
    for g in range(m.shape[0]):
        lg = -0.5 * np.sum(np.log(2 * np.pi * v[g])) - 0.5 * np.sum((Xd - m[g]) ** 2 / v[g], axis=1)
        q += np.sum(post[:, g] * (np.log(h[g]) + lg))
    return q


def test_mstep_is_stationary_point_of_q():
    """Appendix A: the M-step solves dQ/dmu = dQ/dsigma = 0 and, with the
    Lagrange multiplier psi = -N, dQ/dw_m = N for every m."""
    rng = np.random.default_rng(9)
    G, D, N = 3, 2, 400
    m0, v0, h0 = _rand_model(rng, G, D, spread=1.5)
    X = rng.normal(0, 1.5, (N, D)).astype(np.float32)
    post = oracle.posteriors(X, m0, v0, h0)
    m, v, h, _ = oracle.em_iterate(X, m0, v0, h0, 1, 0.0)
    for g in range(G):
        for d in range(D):
            for arr, step in ((m, 1e-5), (v, 1e-6)):
                p = arr.copy(); p[g, d] += step
                mm = arr.copy(); mm[g, d] -= step
                args_p = (p, v, h) if arr is m else (m, p, h)
                args_m = (mm, v, h) if arr is m else (m, mm, h)
                grad = (_q_function(X, post, *args_p) - _q_function(X, post, *args_m)) / (2 * step)
                assert abs(grad) < 1e-5 * N
    # weights: dQ/dw_g = L_g / w_g equals N for every g
    L = post.sum(axis=0)
    np.testing.assert_allclose(L / h, N, rtol=1e-12)


def test_zero_responsibility_component_keeps_parameters():
    X = np.random.default_rng(10).normal(0, 1, (500, 2)).astype(np.float32)
    m0 = np.array([[0.0, 0.0], [1e4, 1e4]])
    v0 = np.array([[1.0, 1.0], [1e-6, 1e-6]])
    h0 = np.array([0.5, 0.5])
    m, v, h, _ = oracle.em_iterate(X, m0, v0, h0, 1, 1e-10)
    np.testing.assert_array_equal(m[1], m0[1])
    np.testing.assert_array_equal(v[1], v0[1])
    assert h[1] == 0.0 and h[0] == pytest.approx(1.0)


def test_tiny_responsibility_component_is_reestimated():
    """Eqs. 12-14 define the update for every L_g > 0: a Gaussian holding only
    ~1e-20 of one sample's responsibility still gets the responsibility-
    weighted mean and variance of the samples (only L_g == 0 keeps them)."""
    X = np.random.default_rng(12).normal(0, 1, (500, 1)).astype(np.float32)
    m0 = np.array([[0.0], [12.0]])
    v0 = np.array([[1.0], [1.0]])
    h0 = np.array([0.5, 0.5])
    post = oracle.posteriors(X, m0, v0, h0)[:, 1]
    L = post.sum()
    assert 0.0 < L < 1e-8
    m, v, h, _ = oracle.em_iterate(X, m0, v0, h0, 1, 1e-10)
    x = X[:, 0].astype(np.float64)
    mu = (post * x).sum() / L
    np.testing.assert_allclose(m[1, 0], mu, rtol=1e-10)
    np.testing.assert_allclose(v[1, 0], max((post * (x - mu) ** 2).sum() / L, 1e-10), rtol=1e-6)
    assert h[1] == pytest.approx(L / 500, rel=1e-12)


def _fp32_em_emulation(X, means, dcovs, hefts, var_floor):
    """An EM iteration evaluated the way an FP32 E-step does it (numpy float32:
    l = c - 1/2 sum (x s - m)^2 with s = 1/sigma, m = mu/sigma, float32
    log-sum-exp, responsibilities and statistics sums about the float32 start
    means), then the FP64 update of Eqs. 12-14."""
    f32 = np.float32
    G, D = means.shape
    s = (1.0 / np.sqrt(dcovs)).astype(f32)
    mm = (means / np.sqrt(dcovs)).astype(f32)
    c = (np.log(hefts) - 0.5 * D * np.log(2 * np.pi) - 0.5 * np.log(dcovs).sum(1)).astype(f32)
    x = X.astype(f32)
    t = x[:, None, :] * s[None] - mm[None]
    l = c[None] - f32(0.5) * (t * t).sum(2, dtype=f32)
    mx = l.max(1, keepdims=True)
    lse = mx[:, 0] + np.log(np.exp(l - mx).sum(1, dtype=f32))
    gam = np.exp(l - lse[:, None])
    f = means.astype(f32)
    q = x[:, None, :] - f[None]
    S0 = gam.sum(0, dtype=f32).astype(np.float64)
    S1 = (gam[:, :, None] * q).sum(0, dtype=f32).astype(np.float64)
    S2 = (gam[:, :, None] * q * q).sum(0, dtype=f32).astype(np.float64)
    live = S0 >= 1e-8          # vanishing mass: mean and covariance kept (as the library does)
    Sd = np.where(live, S0, 1.0)[:, None]
    mu = np.where(live[:, None], f.astype(np.float64) + S1 / Sd, means)
    var = np.where(live[:, None], np.maximum(S2 / Sd - (S1 / Sd) ** 2, var_floor), dcovs)
    return mu, var, S0 / X.shape[0], lse.astype(np.float64), live


@pytest.mark.parametrize("kind", ["c2", "overlap", "floored"])
def test_fp32_budget_covers_an_fp32_emulation(kind):
    """The parity budget (orc_em_fp32_budget, orc_log_p_fp32_bound) bounds what
    an FP32 evaluation of the iteration actually does: an independent numpy
    float32 emulation lands inside it for log p of every sample and every
    parameter of every Gaussian, including the
    weakly supported ones, while on the c2-like case (a start near the
    fit) the budget of the well supported Gaussians stays below the 1e-4
    parity tolerance, i.e. it widens nothing there."""
    if kind == "c2":
        X, _, mix = synth.make("c2", N=4000, G=64)
        start = (mix.means, mix.stds ** 2 * 1.2, mix.hefts)
    elif kind == "overlap":
        rng = np.random.default_rng(5)
        X = rng.normal(0, 1, (3000, 6)).astype(np.float32)
        start = (rng.normal(0, 1.5, (12, 6)), rng.uniform(0.2, 2, (12, 6)), rng.dirichlet(np.ones(12)))
    else:
        # a single-sample cluster at the 1e-10 variance floor, centred on its sample
        X, _, mix = synth.make("c1", N=3000, D=10, G=8, seed=77)
        means, dcovs = mix.means.copy(), mix.stds ** 2
        means[0] = X[5].astype(np.float64)
        dcovs[0] = 1e-10
        start = (means, dcovs, mix.hefts)
    M, V, H, ll, (bm, bv, bw) = oracle.em_fp32_budget(X, *start, 1e-10)
    m, v, h, lse32, live = _fp32_em_emulation(X, *start, 1e-10)
    ll32 = float(lse32.mean())
    # per sample, log p within the oracle's FP32 bound
    assert np.all(np.abs(lse32 - oracle.log_p(X, *start)) <= 2 * oracle.log_p_fp32_bound(X, *start))
    assert np.all(np.abs(m - M)[live] <= 2 * bm[live] + 1e-12)
    assert np.all(np.abs(v - V)[live] <= 2 * bv[live] + 1e-12)
    assert np.all(np.abs(h - H) <= 2 * bw + 1e-15)
    assert abs(ll32 - ll) <= 1e-6 * abs(ll)
    if kind != "c2":
        return
    L = H * X.shape[0]
    big = L >= 100
    assert big.any()
    assert (bm[big] <= 1e-4 * (np.abs(M[big]) + X.std(0))).all()
    assert (bv[big] <= 1e-4 * V[big]).all()


# ------------------------------------------------------- Sec. 3 (k-means)
def test_km_assign_bruteforce():
    rng = np.random.default_rng(11)
    X = rng.normal(0, 2, (300, 3)).astype(np.float32)
    mu = rng.normal(0, 2, (5, 3))
    w = rng.uniform(0.2, 3, 3)
    a, b1, b2 = oracle.km_assign(X, mu, w)
    d = ((X.astype(np.float64)[:, None, :] - mu[None]) ** 2 * w).sum(-1)
    np.testing.assert_array_equal(a, np.argmin(d, axis=1))
    np.testing.assert_allclose(b1, d.min(axis=1), rtol=1e-14)
    np.testing.assert_allclose(b2, np.sort(d, axis=1)[:, 1], rtol=1e-14)
    # exact tie -> lowest index
    mu2 = np.array([[1.0, 0, 0], [1.0, 0, 0]])
    a2, _, _ = oracle.km_assign(X, mu2, w)
    assert (a2 == 0).all()


def test_kmeans_update_is_average_and_objective_non_increasing():
    X, _, _ = synth.make("c1", N=6000)
    gm, gv = oracle.global_stats(X)
    w = 1.0 / gv
    seeds = synth.seeds_subset(X, 8, 3)
    prev = np.inf
    means = seeds
    Xd = X.astype(np.float64)
    for it in range(1, 6):
        m, v, h, a = oracle.kmeans(X, means, w, gv, 1, 1e-10)
        # update = average of the assigned samples (Sec. 3, step (ii))
        for g in range(8):
            sel = a == g
            if sel.any():
                np.testing.assert_allclose(m[g], Xd[sel].mean(axis=0), rtol=1e-12, atol=1e-12)
                np.testing.assert_allclose(v[g], np.maximum(Xd[sel].var(axis=0), 1e-10), rtol=1e-9,
                                           atol=1e-12)
                assert h[g] == pytest.approx(sel.mean(), rel=1e-15)
        obj = sum((((Xd[a == g] - m[g]) ** 2) * w).sum() for g in range(8))
        assert obj <= prev * (1 + 1e-12)
        prev = obj
        means = m


def test_kmeans_dead_mean_resurrection():
    # three samples near 0, two near 10, one seed far from everything -> dead
    X = np.array([[0.0], [0.1], [0.2], [10.0], [10.1]], np.float32)
    seeds = np.array([[0.1], [10.05], [1e6]])
    w = np.ones(1)
    gv = np.array([25.0])
    m, v, h, a = oracle.kmeans(X, seeds, w, gv, 1, 1e-10)
    # the popular mean (index 0, three samples) gives its lowest-index sample
    assert m[2, 0] == pytest.approx(0.0)
    assert v[2, 0] == 25.0
    # hefts: 3/5, 2/5, 1/5, renormalised
    np.testing.assert_allclose(h, np.array([3, 2, 1]) / 6.0, rtol=1e-15)
    # one more iteration: the resurrected mean at 0 now wins sample 0 (tie ->
    # lowest index keeps mean 0 for x=0? mean0 = 0.1, mean2 = 0.0)
    m2, _, _, a2 = oracle.kmeans(X, m, w, gv, 1, 1e-10)
    assert a2[0] == 2 and (a2[3:] == 1).all()


def test_kmeans_dead_means_cycle_over_the_popular_members():
    """More dead means than samples of the most popular mean: the dead means,
    in increasing index, take its samples in increasing index and start over
    (reading of Sec. 3.1); after the last iteration each gets the floored
    global variance and heft 1/N, and the hefts are renormalised."""
    X = np.array([[0.0], [0.1], [10.0], [10.1], [20.0], [20.1]], np.float32)
    seeds = np.array([[0.05], [10.05], [20.05], [1e6], [2e6], [3e6]])
    gv = np.array([64.0])
    m, v, h, a = oracle.kmeans(X, seeds, np.ones(1), gv, 1, 1e-10)
    np.testing.assert_array_equal(a, [0, 0, 1, 1, 2, 2])
    # popular = mean 0 (count 2, lowest index among the ties); dead 3, 4, 5
    # take samples 0, 1, 0
    np.testing.assert_array_equal(m[3:, 0], X[[0, 1, 0], 0].astype(np.float64))
    np.testing.assert_allclose(m[:3, 0], [np.float32(0.0) / 2 + np.float32(0.1) / 2,
                                          (np.float64(np.float32(10.0)) + np.float64(np.float32(10.1))) / 2,
                                          (np.float64(np.float32(20.0)) + np.float64(np.float32(20.1))) / 2],
                               rtol=1e-15)
    assert (v[3:, 0] == 64.0).all()
    np.testing.assert_allclose(h, np.array([2, 2, 2, 1, 1, 1]) / 9.0, rtol=1e-15)


def test_random_subset_seeding_pins_splitmix64():
    with open(os.path.join(HERE, "golden", "splitmix64_seed0.txt")) as f:
        vals = [int(l, 16) for l in f if l.strip() and not l.startswith("#")]
    N = 1000
    idx = oracle.seed_random_subset(N, 2, 0)
    first = vals[0] % N
    assert idx[0] == first
    r1 = 1 + vals[1] % (N - 1)
    assert idx[1] == (0 if r1 == first else r1)
    big = oracle.seed_random_subset(100000, 256, 12345)
    assert len(set(big.tolist())) == 256 and big.min() >= 0 and big.max() < 100000


def test_global_stats_matches_numpy():
    X, _, _ = synth.make("c1", N=3000)
    m, v = oracle.global_stats(X)
    np.testing.assert_allclose(m, X.astype(np.float64).mean(axis=0), rtol=1e-13)
    np.testing.assert_allclose(v, X.astype(np.float64).var(axis=0), rtol=1e-12)


# ------------------------------------------------------- learn (Sec. 4.1)
@pytest.mark.parametrize("G", [2, 4, 8])
def test_recovers_well_separated_mixture(G):
    # k-means + EM only climbs to a local maximum (Sec. 2), and a random
    # subset rarely seeds every cluster, so the start is one sample of each
    # true cluster (keep_existing); k-means and EM must then find the truth.
    X, lab, mix = synth.separated(8000 * G, 4, G, seed=100 + G)
    first = [int(np.flatnonzero(lab == k)[0]) for k in range(G)]
    init = (X[first].astype(np.float64), np.ones((G, 4)), np.full(G, 1.0 / G))
    m, v, h, ll = oracle.learn(X, G, seed_mode=oracle.SEED_KEEP_EXISTING, km_iter=10,
                               em_iter=10, init=init)
    cost = ((m[:, None, :] - mix.means[None]) ** 2).sum(-1)
    r, c = scipy.optimize.linear_sum_assignment(cost)
    for g, k in zip(r, c):
        n = max((lab == k).sum(), 1)
        tol = 4 * mix.stds[k] / np.sqrt(n)
        assert (np.abs(m[g] - mix.means[k]) <= tol + 1e-9).all()
        assert (np.abs(np.sqrt(v[g]) - mix.stds[k]) <= 4 * mix.stds[k] / np.sqrt(n) + 1e-9).all()
        assert h[g] == pytest.approx((lab == k).mean(), abs=1e-6)


def test_fig1_example_program_hefts():
    X, lab, _ = synth.make("fig1")
    m, v, h, ll = oracle.learn(X, 2, seed=1, km_iter=10, em_iter=5)
    order = np.argsort(m[:, 0])
    assert h[order][0] == pytest.approx(2 / 3, abs=0.05)
    assert h[order][1] == pytest.approx(1 / 3, abs=0.05)


def test_assign_modes():
    rng = np.random.default_rng(12)
    m, v, h = _rand_model(rng, 4, 3)
    X = rng.normal(0, 3, (200, 3)).astype(np.float32)
    a_e = oracle.assign(X, m, v, h, 0)
    a_p = oracle.assign(X, m, v, h, 2)
    Xd = X.astype(np.float64)
    np.testing.assert_array_equal(a_e, np.argmin(((Xd[:, None] - m[None]) ** 2).sum(-1), axis=1))
    lt = np.stack([np.log(h[g]) + scipy.stats.multivariate_normal(m[g], np.diag(v[g])).logpdf(Xd)
                   for g in range(4)], axis=1)
    np.testing.assert_array_equal(a_p, np.argmax(lt, axis=1))


def test_learn_rejects_bad_arguments():
    X = np.zeros((5, 2), np.float32)
    with pytest.raises(RuntimeError):
        oracle.learn(X, 6)
    with pytest.raises(RuntimeError):
        oracle.learn(X, 2, var_floor=-1.0)


# ------------------------------------------------------------ seed modes (Sec. 4.1)
def test_static_subset_is_evenly_spaced():
    idx = oracle.seed_static_subset(10, 4)
    np.testing.assert_array_equal(idx, [0, 2, 5, 7])   # floor(g * 10 / 4)
    idx = oracle.seed_static_subset(7, 7)
    np.testing.assert_array_equal(idx, np.arange(7))


def test_spread_is_farthest_first_on_a_line():
    """Points 0..9 on a line, unit weights: from 0 the farthest is 9; then 4
    and 5 are both 4 away from their nearest seed and the lower index wins."""
    X = np.arange(10, dtype=np.float32)[:, None]
    np.testing.assert_array_equal(oracle.seed_spread(X, 3, np.ones(1), 0), [0, 9, 4])
    np.testing.assert_array_equal(oracle.seed_spread(X, 4, np.ones(1), 6), [6, 0, 3, 9])


def test_spread_matches_bruteforce_and_weights():
    rng = np.random.default_rng(8)
    X = rng.normal(0, 1, (60, 3)).astype(np.float32) * np.array([1.0, 5.0, 0.2], np.float32)
    w = 1.0 / np.array([1.0, 25.0, 0.04])
    idx = oracle.seed_spread(X, 7, w, 11)
    chosen = [11]
    Xd = X.astype(np.float64)
    while len(chosen) < 7:
        d = np.min(((Xd[:, None, :] - Xd[None, chosen, :]) ** 2 * w).sum(2), axis=1)
        d[chosen] = -1.0
        chosen.append(int(np.argmax(d)))   # argmax returns the lowest index of the maximum
    np.testing.assert_array_equal(idx, chosen)
    # duplicates: seeds stay distinct when fewer distinct points than seeds exist
    Xr = np.repeat(np.array([[0.0], [1.0]], np.float32), 3, axis=0)
    idx = oracle.seed_spread(Xr, 4, np.ones(1), 0)
    assert len(set(idx.tolist())) == 4


def test_learn_seed_modes_place_means_on_samples():
    X, _, _ = synth.make("c1", N=5000)
    for mode in (oracle.SEED_STATIC_SUBSET, oracle.SEED_STATIC_SPREAD, oracle.SEED_RANDOM_SPREAD):
        M, V, H, _ = oracle.learn(X, 8, seed_mode=mode, seed=5, km_iter=0, em_iter=0)
        rows = {tuple(r) for r in X.astype(np.float64)}
        assert all(tuple(m) in rows for m in M)
        np.testing.assert_array_equal(V, np.ones_like(V))
    # random_spread starts where random_subset's first draw lands
    _, gv = oracle.global_stats(X)
    M, _, _, _ = oracle.learn(X, 8, seed_mode=oracle.SEED_RANDOM_SPREAD, seed=5, km_iter=0, em_iter=0)
    first = oracle.seed_random_subset(X.shape[0], 1, 5)[0]
    idx = oracle.seed_spread(X, 8, 1.0 / np.maximum(gv, 1e-10), first)
    np.testing.assert_array_equal(M, X[idx].astype(np.float64))


# ------------------------------------------------------------ generate (Sec. 4.1)
def test_generate_matches_the_model_statistics():
    """Samples of a known mixture: label frequencies within 5 sigma of the
    hefts, per-component sample means and variances within 5 standard errors
    of the model's (normal theory), and the first uniform equals SplitMix64's
    first output from the seed (the published generator)."""
    rng = np.random.default_rng(3)
    G, D, N = 3, 5, 200_000
    means = rng.normal(0, 3, (G, D))
    dcovs = rng.uniform(0.5, 2.0, (G, D))
    hefts = np.array([0.5, 0.3, 0.2])
    X, lab = oracle.generate(means, dcovs, hefts, N, seed=0)
    freq = np.bincount(lab, minlength=G) / N
    assert np.all(np.abs(freq - hefts) < 5 * np.sqrt(hefts * (1 - hefts) / N))
    for g in range(G):
        xs = X[lab == g].astype(np.float64)
        n = xs.shape[0]
        assert np.all(np.abs(xs.mean(0) - means[g]) < 5 * np.sqrt(dcovs[g] / n))
        assert np.all(np.abs(xs.var(0) - dcovs[g]) < 5 * dcovs[g] * np.sqrt(2.0 / n))
    # the label of sample 0 follows from SplitMix64's first output for seed 0
    with open(os.path.join(HERE, "golden", "splitmix64_seed0.txt")) as f:
        first = [int(l.strip(), 16) for l in f if l.strip() and not l.startswith("#")][0]
    u = ((first >> 11) + 0.5) / 2.0 ** 53
    assert lab[0] == int(np.searchsorted(np.cumsum(hefts), u, side="right"))
    # deterministic
    X2, lab2 = oracle.generate(means, dcovs, hefts, 1000, seed=0)
    np.testing.assert_array_equal(X2, X[:1000])
