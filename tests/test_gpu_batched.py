"""Batched form: many independent fits of uneven N, D, N_G in one graph.

Each fit must match the single-fit gmm_learn on its own data (same seeds) and
the FP64 oracle, within the FP32 tolerances of test_gpu_parity.py."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1707_09094_gb300 import GMM, learn_batched, synth
from test_gpu_parity import assert_params, dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1707_09094_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def fits():
    out = []
    for j in range(14):
        X, _, mix = synth.batched_fit(j, n_lo=1000, n_hi=30000)
        out.append((X, mix.means.shape[0]))
    return out


def test_batched_matches_single_fit_and_oracle(fits, tmp_path, monkeypatch):
    """Log-likelihood trajectories equal the single fits' and the oracle's;
    the parameters of the last iteration equal the oracle's iteration from
    the batched run's own previous state (a batched run is deterministic:
    per-item FP64 partials in fixed order), within the FP32 budget of an
    item of up to 32,768 samples."""
    monkeypatch.setenv("GMM_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    Xs = [dev(X) for X, _ in fits]
    Gs = [G for _, G in fits]
    models = learn_batched(Xs, Gs, km_iter=5, em_iter=5, seed=100)
    before = learn_batched(Xs, Gs, km_iter=5, em_iter=4, seed=100)
    for j, ((X, G), m, p) in enumerate(zip(fits, models, before)):
        single = GMM().learn(Xs[j], G, km_iter=5, em_iter=5, seed=100 + j)
        np.testing.assert_allclose(m.ll_history(), single.ll_history(), rtol=1e-6)
        np.testing.assert_allclose(m.ll_history()[:4], p.ll_history(), rtol=0, atol=0)
        M, V, H, ll, budget = oracle.em_fp32_budget(X, *p.get_params(), 1e-10,
                                                    n_acc=oracle.fp32_accumulations(X.shape[0], chunk=32768))
        assert_params(m.get_params(), (M, V, H), X, budget=budget)
        np.testing.assert_allclose(m.ll_history()[4], ll, rtol=1e-6)
        if j < 4:
            ll_ref = oracle.learn(X, G, seed=100 + j, km_iter=5, em_iter=5)[3]
            np.testing.assert_allclose(m.ll_history(), ll_ref, rtol=1e-6)
    # the autotuner recorded its choice for this shape bucket
    lines = open(tmp_path / "tune.txt").read().split("\n")
    assert any(l.startswith("D64_") for l in lines)


def test_batched_host_inputs_and_per_fit_em_tol(fits):
    """Host inputs and em_tol: each fit stops where the oracle stops, along
    the same log-likelihood trajectory."""
    Xs = [X for X, _ in fits[:6]]
    Gs = [G for _, G in fits[:6]]
    models = learn_batched(Xs, Gs, km_iter=3, em_iter=40, seed=7, em_tol=1e-4)
    lens = []
    for j, m in enumerate(models):
        ll = oracle.learn(Xs[j], Gs[j], seed=7 + j, km_iter=3, em_iter=40, em_tol=1e-4)[3]
        assert len(m.ll_history()) == len(ll)
        np.testing.assert_allclose(m.ll_history(), ll, rtol=1e-6)
        lens.append(len(ll))
    assert len(set(lens)) > 1   # fits stop at different iterations


def test_batched_rejects_unsupported():
    X = np.zeros((100, 70), np.float32)
    with pytest.raises(Exception):
        learn_batched([X], [4])
