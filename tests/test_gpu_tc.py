"""GPU parity of the tensor-core (tcgen05) EM pass against the FP64 oracle and
against the FP32 CUDA-core pass.

The tensor-core pass screens Gaussians with BF16 products under a rigorous
rounding bound and recomputes the survivors exactly in FP32, so it must meet
the FP32 tolerances of test_gpu_parity.py (1e-4 relative on parameters, 1e-6
on log-likelihoods); against the FP32 pass on the same data it agrees to
FP32 summation-order noise.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1707_09094_gb300 import GMM, GMM_MAHA, GmmError, synth
from paper_1707_09094_gb300._lib import GMM_DEBUG_SKIP_MMA, GMM_DEBUG_WAIT_CYCLES
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


@pytest.mark.parametrize("shape", [(100000, 10, 8), (7, 3, 2), (33, 1, 3), (1000, 13, 1), (2049, 60, 40),
                                   (3001, 64, 17), (20000, 60, 256), (129, 16, 16), (300, 5, 200)])
def test_tc_em_matches_oracle(shape):
    N, D, G = shape
    X, _, _ = synth.make("c1", N=N, D=D, G=G, seed=3 + N)
    start = _start(X, G, 2)
    M, V, H, ll = oracle.em_iterate(X, *start, 3, 1e-10)
    g = GMM().set_params(*start)
    g.em_iterate(dev(X), 3, prec="bf16", recompute_center=True)
    assert_params(g.get_params(), (M, V, H), X)
    # Fewer than the 10 samples per Gaussian the paper recommends (Sec. 4.1)
    # lets Gaussians collapse onto the variance floor; their constants
    # -1/2 sum log sigma^2 are then large and FP32 resolves log p to ~1e-5.
    rtol = 1e-6 if N >= 10 * G else 1e-5
    np.testing.assert_allclose(g.ll_history(), ll, rtol=rtol, atol=1e-6)


def test_tc_dense_fallback_many_candidates():
    """Heavily overlapping Gaussians: every sample keeps more candidates than
    the per-thread list holds, which exercises the exact dense path."""
    rng = np.random.default_rng(3)
    N, D, G = 4000, 8, 40
    X = rng.normal(0, 1, (N, D)).astype(np.float32)
    start = (rng.normal(0, 0.05, (G, D)), np.ones((G, D)), np.full(G, 1.0 / G))
    M, V, H, ll = oracle.em_iterate(X, *start, 2, 1e-10)
    g = GMM().set_params(*start)
    g.em_iterate(dev(X), 2, prec="bf16", recompute_center=True)
    assert_params(g.get_params(), (M, V, H), X)
    np.testing.assert_allclose(g.ll_history(), ll, rtol=1e-6)


def test_tc_spill_list_full_falls_back_to_recompute():
    """Every sample keeps ~40 responsibilities: 16 go to its record, the rest
    to its CTA's spill list; at N = 150,000 the lists overflow and the
    samples without room are recomputed over every Gaussian in the M-step.
    All three routes must give the oracle's iteration."""
    rng = np.random.default_rng(4)
    N, D, G = 150_000, 8, 40
    X = rng.normal(0, 1, (N, D)).astype(np.float32)
    start = (rng.normal(0, 0.05, (G, D)), np.ones((G, D)), np.full(G, 1.0 / G))
    M, V, H, ll = oracle.em_iterate(X, *start, 2, 1e-10)
    g = GMM().set_params(*start)
    g.em_iterate(dev(X), 2, prec="bf16", recompute_center=True)
    assert_params(g.get_params(), (M, V, H), X)
    np.testing.assert_allclose(g.ll_history(), ll, rtol=1e-6)


def test_tc_learn_end_to_end_c1():
    X, _, _ = synth.make("c1")
    g = GMM().learn(dev(X), 8, km_iter=10, em_iter=10, seed=1001, prec="bf16")
    M, V, H, ll = oracle.learn(X, 8, seed=1001, km_iter=10, em_iter=10)
    assert_params(g.get_params(), (M, V, H), X)
    np.testing.assert_allclose(g.ll_history(), ll, rtol=1e-6)


@pytest.fixture(scope="module")
def c2_km():
    """The benchmark's state: c2 at full size (N=2e6, D=60, N_G=256),
    k-means-initialised (10 iterations, random_subset seed 1002)."""
    X, _, mix = synth.make("c2")
    Xd = dev(X)
    start = GMM().learn(Xd, 256, km_iter=10, em_iter=0, seed=1002).get_params()
    return X, Xd, mix, start


def test_tc_headline_c2_matches_oracle(c2_km):
    """The headline form at the headline size: from the benchmark's k-means
    start, two BF16 tensor-core EM iterations, each compared with the
    oracle's iteration (all host cores) from the same parameters: every
    Gaussian's parameters within 1e-4 or its FP32 budget, the log-likelihood
    within 1e-6."""
    X, Xd, _, start = c2_km
    g = GMM().set_params(*start)
    g.em_iterate(Xd, 0, recompute_center=True)
    for _ in range(2):
        em_step_check(g, X, Xd, prec="bf16")


def test_tc_matches_fp32_pass_at_full_size(c2_km):
    """3 EM iterations in each form from the same start agree in their
    log-likelihood trajectories to FP32 summation noise, and the results are
    judged equal by the same evaluator (the parameters of each form are held
    to the oracle one iteration at a time by the tests above)."""
    X, Xd, mix, _ = c2_km
    start = (mix.means, mix.stds ** 2 * 1.2, mix.hefts)
    a = GMM().set_params(*start)
    a.em_iterate(Xd, 3, prec="fp32", recompute_center=True)
    b = GMM().set_params(*start)
    b.em_iterate(Xd, 3, prec="bf16", recompute_center=True)
    np.testing.assert_allclose(b.ll_history(), a.ll_history(), rtol=1e-7)
    assert abs(a.avg_log_p(Xd) - b.avg_log_p(Xd)) < 1e-5


def test_tc_bounded_wait_times_out_and_context_survives():
    """Failure detection without a fault: the MMA issuer is told to issue
    nothing, the epilogue's bounded wait runs out, the pass frees its tensor
    memory and reports GMM_ERR_TIMEOUT; the model and the CUDA context stay
    usable."""
    X, _, _ = synth.make("c1", N=4096)
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


def test_tc_rejects_unsupported_shapes():
    """The tensor-core forms take D <= 128 and N_G <= 4096 (D <= 64 and
    N_G <= 256 in one tile, the rest in blocks of Gaussians)."""
    G = 4097
    X, _, _ = synth.make("c1", N=8200, D=3, G=4, seed=1)
    g = GMM().set_params(X[:G].astype(np.float64), np.ones((G, 3)), np.full(G, 1.0 / G))
    with pytest.raises(GmmError) as e:
        g.em_iterate(dev(X), 1, prec="bf16", recompute_center=True)
    assert e.value.status == -7


def test_tc_unaligned_input_matches_aligned():
    """The staged kernels copy whole 128-sample tiles with the bulk engine
    only when X is 16-byte aligned; an X that starts 4 bytes into its buffer
    takes the per-thread copy for every tile and must give the same results
    (same arithmetic; only the order of FP32 additions within a Gaussian's
    bin may differ)."""
    X, _, _ = synth.make("c1", N=50_000, seed=21)
    flat = torch.zeros(X.size + 1, dtype=torch.float32, device="cuda")
    flat[1:] = torch.from_numpy(X.ravel()).cuda()
    Xu = flat[1:].view(X.shape)
    assert Xu.data_ptr() % 16 == 4
    Xa = dev(X)
    start = GMM().learn(Xa, 8, km_iter=5, em_iter=0, seed=3).get_params()
    a = GMM().set_params(*start)
    a.em_iterate(Xa, 3, prec="bf16", recompute_center=True)
    b = GMM().set_params(*start)
    b.em_iterate(Xu, 3, prec="bf16", recompute_center=True)
    np.testing.assert_allclose(a.ll_history(), b.ll_history(), rtol=1e-7)
    # FP32 addition order: 1e-6 relative, with a floor of 1e-6 of the data's scale
    assert_params(b.get_params(), a.get_params(), X, rtol=1e-6)


def test_tc_and_fp32_converge_alike_under_em_tol():
    """Convergence-driven runs (em_tol = 1e-6, at most 250 iterations) on two
    Table-1-shaped synthetic sets: the tensor-core form stops within a few
    iterations of the FP32 form (their mean-LL gains differ by FP32 noise
    where they cross em_tol) and at the same mean log-likelihood."""
    for r, (N, D, G) in enumerate([(6497, 11, 30), (37749, 32, 50)]):
        rng = np.random.default_rng(2100 + r)
        X, _ = synth._draw(rng, synth.mixture_c1(rng, D, G), N)
        Xd = dev(X)
        a = GMM().learn(Xd, G, km_iter=10, em_iter=250, em_tol=1e-6, seed=5, prec="fp32")
        b = GMM().learn(Xd, G, km_iter=10, em_iter=250, em_tol=1e-6, seed=5, prec="bf16")
        assert abs(len(a.ll_history()) - len(b.ll_history())) <= 3   # the stop test sees LL gains near em_tol
        assert abs(a.avg_log_p(Xd) - b.avg_log_p(Xd)) < 1e-5


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_host_input_in_chunks_matches_device_input(prec):
    """Host X of >= 262,144 samples reaches the GPU in four chunks whose copies
    overlap the first EM iteration's pass; the result equals the device-input
    run up to FP32 addition order, over several iterations."""
    X, _, _ = synth.make("c1", N=300_001, seed=41)
    Xd = dev(X)
    start = GMM().learn(Xd, 8, km_iter=3, em_iter=0, seed=2).get_params()
    a = GMM().set_params(*start)
    a.em_iterate(Xd, 0, recompute_center=True)
    a.em_iterate(Xd, 3, prec=prec)
    b = GMM().set_params(*start)
    b.em_iterate(Xd, 0, recompute_center=True)
    Xh = torch.from_numpy(X).pin_memory()
    b.em_iterate(Xh, 3, prec=prec)
    b.em_iterate(X, 2, prec=prec)            # pageable host memory too
    a.em_iterate(Xd, 2, prec=prec)
    np.testing.assert_allclose(b.ll_history(), a.ll_history(), rtol=1e-7)
    assert_params(b.get_params(), a.get_params(), X, rtol=1e-6)
