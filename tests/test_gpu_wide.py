"""GPU parity of the blocked tensor-core EM pass (split-BF16 screen over blocks
of 128 Gaussians, exact FP32 recompute of the candidates, M-step from the
kept responsibilities) against the FP64 oracle.

The pass runs by itself wherever D > 64 or N_G > 256 (up to D = 128,
N_G = 4096), and on smaller shapes through the GMM_DEBUG_TC_FORM hook.  Its
screen drops only Gaussians whose responsibility is provably below 1e-9 / N,
so it is held to the FP32 tolerances of test_gpu_parity.py: 1e-4 relative on
parameters (or the oracle's FP32 budget where larger) and 1e-6 on the
log-likelihood."""
import numpy as np
import pytest
import torch

import oracle
from paper_1707_09094_gb300 import GMM, GMM_MAHA, GmmError, synth
from paper_1707_09094_gb300._lib import GMM_DEBUG_SKIP_MMA, GMM_DEBUG_TC_FORM, GMM_DEBUG_WAIT_CYCLES
from test_gpu_parity import assert_params, dev, em_step_check, km_weights

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1707_09094_gb300 import build
    build.build()


def _start(X, G, seed):
    seeds = synth.seeds_subset(X, G, seed)
    if G == 1 or X.shape[0] < 50:
        return seeds, np.ones_like(seeds), np.full(G, 1.0 / G)
    w, gv = km_weights(X, GMM_MAHA, 1e-10)
    return oracle.kmeans(X, seeds, w, gv, 5, 1e-10)[:3]


# (N, D, G): forced onto the blocked form below D 64 / N_G 256; by shape above.
# Ragged tiles and blocks, D not a multiple of 4 or 8, one and two K pieces.
SHAPES = [(100000, 10, 8), (7, 3, 2), (33, 1, 3), (2049, 60, 40), (3001, 64, 17), (129, 16, 16),
          (300, 5, 200), (5000, 100, 40), (4000, 20, 300), (3000, 128, 130), (1000, 127, 9), (6000, 65, 257)]


def wide_step(g, X, Xd):
    """One tensor-core iteration of g against the oracle's iteration from g's
    parameters: each parameter within 1e-4 or its FP32 budget; the mean
    log-likelihood within 1e-6 or twice the mean of the oracle's per-sample
    FP32 bound on log p (Gaussians collapsed onto the variance floor make
    x s and mu s large, and FP32 then resolves their samples' log p only to
    that bound)."""
    start = g.get_params()
    M, V, H, ll, budget = oracle.em_fp32_budget(X, *start, 1e-10)
    lim = max(1e-6 * abs(ll), 2.0 * float(np.mean(oracle.log_p_fp32_bound(X, *start))))
    g.em_iterate(Xd, 1, prec="bf16")
    assert_params(g.get_params(), (M, V, H), X, budget=budget)
    assert abs(g.ll_history()[-1] - ll) <= lim, (g.ll_history()[-1], ll, lim)


@pytest.mark.parametrize("shape", SHAPES)
def test_wide_em_matches_oracle(shape):
    """Three iterations from a k-means start, each against the oracle's."""
    N, D, G = shape
    X, _, _ = synth.make("c1", N=N, D=D, G=G, seed=5 + N + D)
    Xd = dev(X)
    g = GMM().set_params(*_start(X, G, 2))
    g.debug_set(GMM_DEBUG_TC_FORM, 1)
    g.em_iterate(Xd, 0, recompute_center=True)
    for _ in range(3):
        wide_step(g, X, Xd)


@pytest.mark.parametrize("case", ["spread48", "all40", "all100"])
def test_wide_candidate_lists_and_fp32_handoff(case):
    """Heavily overlapping Gaussians.  spread48: 48 of 128 Gaussians, 12 in each
    quarter of the block's columns, are candidates of every sample (the
    exact kernel takes two per lane), the other 80 lie far away; all40: the
    40 Gaussians of a model, all in the first quarter of the block's columns,
    are candidates of every sample (one list per sample, up to 64); all100:
    100 candidates, more than a list holds, so every sample goes to the
    register-blocked FP32 form, whose statistics and log-likelihood join the
    pass's."""
    rng = np.random.default_rng(3)
    N, D = 4000, 8
    X = rng.normal(0, 1, (N, D)).astype(np.float32)
    if case == "spread48":
        G = 128
        means = 30.0 + rng.normal(0, 1, (G, D))
        near = np.concatenate([np.arange(12) + 32 * k for k in range(4)])
        means[near] = rng.normal(0, 0.05, (near.size, D))
    else:
        G = 40 if case == "all40" else 100
        means = rng.normal(0, 0.05, (G, D))
    start = (means, np.ones((G, D)), np.full(G, 1.0 / G))
    M, V, H, ll = oracle.em_iterate(X, *start, 2, 1e-10)
    g = GMM().set_params(*start)
    g.debug_set(GMM_DEBUG_TC_FORM, 1)
    g.profile(True)
    g.em_iterate(dev(X), 2, prec="bf16", recompute_center=True)
    n, kept, nd = g.screen_stats()
    assert n == 2 * N and nd == (2 * N if case == "all100" else 0)
    if case != "all100":
        assert kept == 2 * N * (48 if case == "spread48" else 40)
    assert_params(g.get_params(), (M, V, H), X)
    np.testing.assert_allclose(g.ll_history(), ll, rtol=1e-6)


def test_wide_some_samples_to_fp32_form():
    """A mixture where part of the samples have more than 64 candidates: those
    go to the FP32 form, the rest stay on the tensor-core path, and the
    iteration matches the oracle's."""
    rng = np.random.default_rng(5)
    N, D, G = 6000, 8, 160
    X = rng.normal(0, 1, (N, D)).astype(np.float32)
    X[: N // 3] += 40.0   # a third of the samples near the 100 overlapping means, the rest near 60 others
    means = np.concatenate([40.0 + rng.normal(0, 0.05, (100, D)), rng.normal(0, 0.5, (60, D))])
    start = (means, np.ones((G, D)), np.full(G, 1.0 / G))
    M, V, H, ll = oracle.em_iterate(X, *start, 2, 1e-10)
    g2 = GMM().set_params(*start)
    g2.debug_set(GMM_DEBUG_TC_FORM, 1)
    g2.profile(True)
    g2.em_iterate(dev(X), 2, prec="bf16", recompute_center=True)
    n, kept, nd = g2.screen_stats()
    assert 0 < nd < n
    assert_params(g2.get_params(), (M, V, H), X)
    np.testing.assert_allclose(g2.ll_history(), ll, rtol=1e-6)


def test_wide_matches_one_tile_form():
    """On a shape both tensor-core forms take, three iterations of each from the
    same start agree to FP32 summation noise."""
    X, _, _ = synth.make("c2", N=200_000)
    Xd = dev(X)
    start = GMM().learn(Xd, 256, km_iter=5, em_iter=0, seed=1002).get_params()
    lls = []
    for form in (0, 1):
        g = GMM().set_params(*start)
        g.debug_set(GMM_DEBUG_TC_FORM, form)
        g.em_iterate(Xd, 3, prec="bf16", recompute_center=True)
        lls.append(np.array(g.ll_history()))
    np.testing.assert_allclose(lls[1], lls[0], rtol=1e-6)


def test_c3_prefix_tensor_core_iterations_match_oracle():
    """The precision workload's shape and value distributions (D=128,
    N_G=1024, means ~ N(0, 3^2), sigma log-uniform on [0.1, 10]) on 200,000
    samples: from a k-means start, two tensor-core EM iterations, each against
    the oracle's iteration from the same parameters: every Gaussian within
    1e-4 or its FP32 budget, the log-likelihood within 1e-6."""
    X, _, _ = synth.make("c3", N=200_000)
    Xd = dev(X)
    g = GMM().learn(Xd, 1024, km_iter=3, em_iter=0, seed=1003, var_floor=1e-10)
    g.em_iterate(Xd, 0, recompute_center=True)
    g.profile(True)
    for _ in range(2):
        em_step_check(g, X, Xd, prec="bf16")
    n, kept, dense = g.screen_stats()
    print("\nc3 prefix: %.3f candidates per sample, %d dense" % (kept / n, dense))
    assert n == 2 * X.shape[0]


def test_c3_full_size_tensor_core_form():
    """N=1e7, D=128, N_G=1024 on the tensor cores: from the k-means start of
    the bench, three iterations; the log-likelihood does not decrease and
    matches the FP32 register-blocked form's to FP32 summation noise, and
    sampled per-sample log-densities match the oracle's."""
    X, _, _ = synth.make("c3")
    Xd = dev(X)
    start = GMM().learn(Xd, 1024, km_iter=2, em_iter=0, seed=1003, var_floor=1e-10).get_params()
    lls = {}
    for prec in ("bf16", "fp32"):
        g = GMM().set_params(*start)
        g.em_iterate(Xd, 3, prec=prec, var_floor=1e-10, recompute_center=True)
        lls[prec] = np.array(g.ll_history())
        if prec == "bf16":
            m, v, h = g.get_params()
            assert h.sum() == pytest.approx(1.0, abs=1e-6)
            idx = np.random.default_rng(2).choice(X.shape[0], 300, replace=False)
            lp = g.log_p(Xd).cpu().numpy()[idx]
            np.testing.assert_allclose(lp, oracle.log_p(X[idx], m, v, h), rtol=1e-5, atol=1e-4)
    ll = lls["bf16"]
    assert (np.diff(ll) >= -1e-6 * np.abs(ll[1:])).all()
    np.testing.assert_allclose(ll, lls["fp32"], rtol=1e-6)
    del Xd
    torch.cuda.empty_cache()


def test_wide_unaligned_and_host_input_match_aligned():
    """An X that starts 4 bytes into its buffer (scalar sample loads, no L2
    prefetch of whole tiles) and a host X (copied in chunks behind the first
    pass in the one-tile form; taken whole here) give the aligned device
    result, to FP32 summation order."""
    X, _, _ = synth.make("c1", N=50_000, D=100, G=300, seed=22)
    flat = torch.zeros(X.size + 1, dtype=torch.float32, device="cuda")
    flat[1:] = torch.from_numpy(X.ravel()).cuda()
    Xu = flat[1:].view(X.shape)
    assert Xu.data_ptr() % 16 == 4
    Xa = dev(X)
    start = GMM().learn(Xa, 300, km_iter=5, em_iter=0, seed=3).get_params()
    runs = []
    for Xin in (Xa, Xu, X):
        g = GMM().set_params(*start)
        g.em_iterate(Xin, 3, prec="bf16", recompute_center=True)
        runs.append(g)
    for b in runs[1:]:
        np.testing.assert_allclose(b.ll_history(), runs[0].ll_history(), rtol=1e-7)
        assert_params(b.get_params(), runs[0].get_params(), X, rtol=1e-6)


def test_wide_bounded_wait_times_out_and_context_survives():
    """Failure detection without a fault, blocked form: the MMA thread issues
    nothing, the epilogue's and the operand loader's bounded waits run out,
    the screen drains its copies, frees its tensor memory and records
    GMM_ERR_TIMEOUT; the later kernels of the pass stand down, the model is
    kept and the context stays usable."""
    X, _, _ = synth.make("c1", N=4096, D=80, G=8, seed=2)
    Xd = dev(X)
    g = GMM().learn(Xd, 8, km_iter=2, em_iter=1, seed=1)
    before = g.get_params()
    g.debug_set(GMM_DEBUG_WAIT_CYCLES, 2_000_000).debug_set(GMM_DEBUG_SKIP_MMA, 1)
    with pytest.raises(GmmError) as e:
        g.em_iterate(Xd, 1, prec="bf16")
    assert e.value.status == -4
    for p, q in zip(before, g.get_params()):
        np.testing.assert_array_equal(p, q)
    g.debug_set(GMM_DEBUG_SKIP_MMA, 0).debug_set(GMM_DEBUG_WAIT_CYCLES, 0)
    g.em_iterate(Xd, 1, prec="bf16")
    torch.cuda.synchronize()
    assert np.isfinite(g.ll_history()).all()
