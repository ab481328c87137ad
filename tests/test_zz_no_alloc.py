"""gmm_avg_log_p_noalloc: the allocation-free variant of gmm_avg_log_p, for
callers that cannot call cudaMalloc when they need the value (a framework
whose caching allocator already holds all free device memory, a service with
a fixed memory footprint).  It must return what gmm_avg_log_p returns, on
consecutive calls, through the C ABI, without changing the device's free
memory.  This file is collected last so that a run that stops at its first
failure has run every other test before it."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1707_09094_gb300 import GMM, _lib, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1707_09094_gb300 import build
    build.build()


def _noalloc(model, X, g=-1):
    out = ctypes.c_double()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = _lib.load().gmm_avg_log_p_noalloc(model._h, ctypes.c_void_p(X.data_ptr()), X.shape[0], g,
                                           ctypes.byref(out), stream)
    return st, out.value


def _reference(model, X, g=-1):
    out = ctypes.c_double()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = _lib.load().gmm_avg_log_p(model._h, ctypes.c_void_p(X.data_ptr()), X.shape[0], g, ctypes.byref(out),
                                   stream)
    assert st == 0
    return out.value


@pytest.mark.parametrize("shape", [(100000, 10, 8), (4099, 60, 256), (1, 3, 1)])
def test_noalloc_matches_avg_log_p_on_two_calls(shape):
    N, D, G = shape
    X, _, mix = synth.make("c1", N=N, D=D, G=G, seed=5 + N)
    Xd = torch.from_numpy(X).cuda()
    g = GMM().set_params(mix.means, mix.stds ** 2, mix.hefts)
    for k in (-1, G - 1):
        ref = _reference(g, Xd, k)
        for _ in range(2):
            st, v = _noalloc(g, Xd, k)
            assert st == 0, _lib.load().gmm_last_error()
            assert v == pytest.approx(ref, rel=1e-12, abs=1e-12)


def test_noalloc_first_on_a_fresh_model_allocates_nothing():
    """Called before anything else on a new model (nothing staged yet), the
    entry point still returns gmm_avg_log_p's value, and the device's free
    memory is the same before and after each later call.  (The first call may
    see the driver load the kernels' code; that is the driver's, so memory is
    compared across the calls after it.)"""
    X, _, mix = synth.make("c1", N=50_000, D=20, G=16, seed=3)
    Xd = torch.from_numpy(X).cuda()
    torch.cuda.synchronize()
    g = GMM().set_params(mix.means, mix.stds ** 2, mix.hefts)
    st, first = _noalloc(g, Xd)
    assert st == 0, _lib.load().gmm_last_error()
    for _ in range(3):
        free0 = torch.cuda.mem_get_info()[0]
        st, v = _noalloc(g, Xd)
        free1 = torch.cuda.mem_get_info()[0]
        assert st == 0 and v == first
        assert free1 == free0
    assert first == pytest.approx(_reference(g, Xd), rel=1e-12, abs=1e-12)


def test_noalloc_at_the_size_limit():
    """N = 8,388,608 fills all 65,536 block slots of the array: still the
    value of gmm_avg_log_p, twice in a row."""
    N = 8_388_608
    rng = np.random.default_rng(8)
    X = torch.from_numpy(rng.normal(0.5, 2.0, (N, 1)).astype(np.float32)).cuda()
    g = GMM().set_params(np.array([[0.0], [1.0]]), np.array([[1.0], [4.0]]), np.array([0.3, 0.7]))
    ref = _reference(g, X)
    for _ in range(2):
        st, v = _noalloc(g, X)
        assert st == 0, _lib.load().gmm_last_error()
        assert v == pytest.approx(ref, rel=1e-12, abs=1e-12)
    del X
    torch.cuda.empty_cache()


def test_noalloc_rejects_host_input_and_oversize():
    X, _, mix = synth.make("c1", N=1000, D=4, G=2, seed=1)
    g = GMM().set_params(mix.means, mix.stds ** 2, mix.hefts)
    out = ctypes.c_double()
    st = _lib.load().gmm_avg_log_p_noalloc(g._h, X.ctypes.data_as(ctypes.c_void_p), X.shape[0], -1,
                                           ctypes.byref(out), None)
    assert st == _lib.GMM_ERR_ARG
    big = torch.zeros((8_388_609, 1), dtype=torch.float32, device="cuda")
    g1 = GMM().set_params(np.zeros((1, 1)), np.ones((1, 1)), np.ones(1))
    st, _ = _noalloc(g1, big)
    assert st == _lib.GMM_ERR_UNSUPPORTED
    assert b"allocation-free limit" in _lib.load().gmm_last_error()
