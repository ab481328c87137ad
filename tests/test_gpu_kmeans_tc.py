"""Tensor-core k-means (split-BF16 screen + exact decision) against the FP64
oracle and against the CUDA-core form.

Both forms decide the nearest mean exactly -- the definition's FP64 distance
sum_d w_d (x_d - mu_d)^2 in order d = 0..D-1, lowest index on exact ties --
so the assignments of one step are compared bit for bit on every sample, ties
included.  The statistics are FP32 sums shifted by the FP32 old means and
reduced in FP64: 1e-6 relative after one step (the tolerance of the CUDA-core
form).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1707_09094_gb300 import GMM, GMM_EUCL, GMM_MAHA, synth
from paper_1707_09094_gb300._lib import GMM_DEBUG_KM_FORM

pytestmark = pytest.mark.gpu

TC, CUDA_CORES = 0, 1


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1707_09094_gb300 import build
    build.build()


def dev(X):
    return torch.from_numpy(np.ascontiguousarray(X)).cuda()


def km_weights(X, dist, var_floor=1e-10):
    _, gv = oracle.global_stats(X)
    gv = np.maximum(gv, var_floor)
    return (1.0 / gv if dist == GMM_MAHA else np.ones_like(gv)), gv


def close(got, ref, X, rtol):
    """Parameters within rtol, absolute floors rtol * global std (means),
    rtol * global variance (dcovs), rtol / G (hefts)."""
    gstd = X.astype(np.float64).std(axis=0)
    G = ref[0].shape[0]
    for a, b, atol, what in ((got[0], ref[0], rtol * gstd[None, :], "means"),
                             (got[1], ref[1], rtol * gstd[None, :] ** 2, "dcovs"),
                             (got[2], ref[2], rtol / G, "hefts")):
        err = np.abs(np.asarray(a) - np.asarray(b))
        lim = atol + rtol * np.abs(b)
        assert (err <= lim).all(), "%s: %d outside tolerance, worst %.3g" % (what, (err > lim).sum(),
                                                                            float((err / lim).max()))


def step(X, seeds, iters, dist, form, profile=False):
    G = seeds.shape[0]
    g = GMM().set_params(seeds, np.ones_like(seeds), np.full(G, 1.0 / G))
    g.debug_set(GMM_DEBUG_KM_FORM, form)
    if profile:
        g.profile(True)
    a = g.kmeans(dev(X), iters, dist_mode=dist).cpu().numpy()
    return g, a


@pytest.mark.parametrize("dist", [GMM_MAHA, GMM_EUCL])
@pytest.mark.parametrize("shape", [(100000, 10, 8), (5003, 13, 5), (129, 3, 3), (4097, 60, 37),
                                   (20000, 64, 256), (3001, 1, 2), (777, 33, 200), (1000, 7, 1)])
def test_tc_kmeans_step_bit_exact(shape, dist):
    """Several 128-sample tiles and a ragged tail; D from 1 to 64, N_G from 1
    to 256 (one to sixteen 16-wide MMA column blocks)."""
    N, D, G = shape
    X, _, _ = synth.make("c1", N=N, D=D, G=max(G, 2), seed=31 + N + D)
    seeds = synth.seeds_subset(X, G, 5)
    w, gv = km_weights(X, dist)
    M, V, H, A = oracle.kmeans(X, seeds, w, gv, 1, 1e-10)
    g, a = step(X, seeds, 1, dist, TC)
    np.testing.assert_array_equal(a, A)
    close(g.get_params(), (M, V, H), X, 1e-6)


def test_tc_kmeans_exact_ties_and_duplicate_means():
    """Integer samples against half-integer means: many samples are at
    exactly equal distance from several means (the FP64 definition decides,
    lowest index first); two means are copies of a third."""
    rng = np.random.default_rng(3)
    X = rng.integers(-4, 5, size=(30000, 6)).astype(np.float32)
    seeds = rng.integers(-3, 4, size=(12, 6)).astype(np.float64) + 0.5
    seeds[5] = seeds[2]
    seeds[9] = seeds[2]
    w, _ = km_weights(X, GMM_EUCL)
    A, b1, b2 = oracle.km_assign(X, seeds, w)
    assert (b1 == b2).sum() > 1000   # the case is really exercised
    g, a = step(X, seeds, 1, GMM_EUCL, TC, profile=True)
    np.testing.assert_array_equal(a, A)
    screened, deferred, fp64 = g.km_screen_stats()
    assert screened == X.shape[0] and deferred >= (b1 == b2).sum() and fp64 >= (b1 == b2).sum()


def test_tc_kmeans_many_equal_candidates():
    """Forty copies of one mean: more candidates than a sample's list holds,
    so those samples re-decide every mean in FP64."""
    X, _, _ = synth.make("c1", N=6000, D=8, G=4, seed=2)
    seeds = synth.seeds_subset(X, 100, 7)
    seeds[10:50] = seeds[10]
    w, _ = km_weights(X, GMM_MAHA)
    A, _, _ = oracle.km_assign(X, seeds, w)
    assert (A == 10).sum() > 0
    _, a = step(X, seeds, 1, GMM_MAHA, TC)
    np.testing.assert_array_equal(a, A)


def test_tc_kmeans_unaligned_input():
    """X not 16-byte aligned: every tile is read by the threads, no bulk copies."""
    X, _, _ = synth.make("c1", N=9001, D=10, G=8, seed=4)
    seeds = synth.seeds_subset(X, 8, 3)
    w, gv = km_weights(X, GMM_MAHA)
    M, V, H, A = oracle.kmeans(X, seeds, w, gv, 1, 1e-10)
    buf = torch.empty(X.size + 1, dtype=torch.float32, device="cuda")
    Xd = buf[1:].view(X.shape)
    Xd.copy_(torch.from_numpy(X))
    g = GMM().set_params(seeds, np.ones_like(seeds), np.full(8, 1.0 / 8))
    a = g.kmeans(Xd, 1).cpu().numpy()
    np.testing.assert_array_equal(a, A)
    close(g.get_params(), (M, V, H), X, 1e-6)


def test_tc_kmeans_ten_iterations_agree_with_cuda_core_form():
    X, _, _ = synth.make("c1", N=50000, D=24, G=32, seed=8)
    seeds = synth.seeds_subset(X, 32, 1)
    g0, a0 = step(X, seeds, 10, GMM_MAHA, TC)
    g1, a1 = step(X, seeds, 10, GMM_MAHA, CUDA_CORES)
    assert (a0 != a1).mean() < 1e-4   # FP32 sums in another order can move near-ties of later steps
    close(g0.get_params(), g1.get_params(), X, 1e-5)


@pytest.fixture(scope="module")
def c2():
    X, _, _ = synth.make("c2")
    return X, dev(X)


def test_tc_kmeans_c2_full_size(c2):
    """N=2e6, D=60, N_G=256 in the benchmark's launch configuration: the
    assignment equals the CUDA-core form's on every sample and the oracle's
    on a sample of 20000; the statistics agree with the CUDA-core form."""
    X, Xd = c2
    seeds = synth.seeds_subset(X, 256, 5)
    ga = GMM().set_params(seeds, np.ones_like(seeds), np.full(256, 1.0 / 256))
    ga.profile(True)
    a0 = ga.kmeans(Xd, 1).cpu().numpy()
    gb = GMM().set_params(seeds, np.ones_like(seeds), np.full(256, 1.0 / 256))
    gb.debug_set(GMM_DEBUG_KM_FORM, CUDA_CORES)
    a1 = gb.kmeans(Xd, 1).cpu().numpy()
    np.testing.assert_array_equal(a0, a1)
    idx = np.random.default_rng(0).choice(X.shape[0], 20000, replace=False)
    w, _ = km_weights(X, GMM_MAHA)
    A, _, _ = oracle.km_assign(X[idx], seeds, w)
    np.testing.assert_array_equal(a0[idx], A)
    close(ga.get_params(), gb.get_params(), X, 1e-6)
    screened, deferred, fp64 = ga.km_screen_stats()
    assert screened == X.shape[0]
    assert deferred < 0.05 * X.shape[0] and fp64 < 1e-3 * X.shape[0]
