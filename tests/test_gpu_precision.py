"""Precision report: the error of every result of one EM iteration against the
FP64 oracle, per E-step form, on prefixes of the c2 workload (N = 50,000,
D = 60, N_G = 256) and the c3 workload (N = 20,000, D = 128, N_G = 1024) from
a k-means start.

Results compared: log p(x_i) under the E-step's parameters (lse_i, the FP32
E-step formula), the mean log-likelihood of the iteration, and the updated
means, variances and weights (the sufficient statistics S0, S1, S2 enter
only through them).  The
relative errors are printed (pytest -s) and held to the parity tolerances:
1e-4 on parameters (floors 1e-4 * global std / variance / 1 / N_G, or the
oracle's FP32 budget where larger), 1e-6 on the mean log-likelihood, and
on each log p(x_i) 3 (1e-5 + 1e-6 |log p|) -- the FP32 evaluation sums
log-density terms of a few hundred nats (u * 500 is 3e-5) -- or twice the
oracle's per-sample FP32 bound where larger (samples of single-sample
clusters at the 1e-10 variance floor: there x s and mu s reach 1e5 |x|)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1707_09094_gb300 import GMM, GMM_MAHA, synth
from test_gpu_parity import assert_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1707_09094_gb300 import build
    build.build()


def rel_err(got, ref, floor):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    return float(np.max(np.abs(got - ref) / (np.abs(ref) + floor)))


@pytest.mark.parametrize("kind,N,G,forms", [("c2", 50000, 256, ("fp32", "bf16")), ("c3", 20000, 1024, ("fp32", "bf16"))])
def test_precision_report(kind, N, G, forms):
    """Per form and result, the relative error of one GPU EM iteration against
    the oracle's.  On c3 (D=128, N_G=1024, sigma down to 0.1) the FP32
    form is the register-blocked two-phase one and the tensor-core form the
    blocked split-BF16 screen with exact FP32 candidates."""
    X, _, _ = synth.make(kind, N=N)
    _, gv = oracle.global_stats(X)
    gv = np.maximum(gv, 1e-10)
    seeds = synth.seeds_subset(X, G, 7)
    start = oracle.kmeans(X, seeds, 1.0 / gv, gv, 3, 1e-10)[:3]
    M, V, H, ll1, budget = oracle.em_fp32_budget(X, *start, 1e-10)
    ll = [ll1]
    lp_ref = oracle.log_p(X, *start)   # log p(x_i) of the E-step's parameters (lse_i)
    lp_lim = np.maximum(3.0 * (1e-5 + 1e-6 * np.abs(lp_ref)), 2.0 * oracle.log_p_fp32_bound(X, *start))
    gstd = np.sqrt(X.astype(np.float64).var(axis=0))
    Xd = torch.from_numpy(X).cuda()
    rows = []
    for prec in forms:
        g = GMM().set_params(*start)
        g.em_iterate(Xd, 1, prec=prec, recompute_center=True)
        m, v, h = g.get_params()
        lp = GMM().set_params(*start).log_p(Xd).cpu().numpy()
        big = H * N >= 10   # the table: Gaussians with >= 10 samples' worth (the assertion: all, by the budget)
        r = {"form": prec,
             "means": rel_err(m[big], M[big], gstd[None, :]),
             "dcovs": rel_err(v[big], V[big], gstd[None, :] ** 2),
             "hefts": rel_err(h, H, 1.0 / G),
             "LL": abs(g.ll_history()[0] - ll[0]) / abs(ll[0]),
             "log p(x_i)": rel_err(lp, lp_ref, 1.0),
             "log p limit": float(np.max(np.abs(lp - lp_ref) / lp_lim))}
        rows.append(r)
        k = int(np.argmax(np.abs(lp - lp_ref) / lp_lim))
        print("\n%s worst log p: got %.9g ref %.9g" % (prec, lp[k], lp_ref[k]))
        assert_params((m, v, h), (M, V, H), X, budget=budget)
        assert r["LL"] <= 1e-6 and r["log p limit"] <= 1.0, r
    keys = ["means", "dcovs", "hefts", "LL", "log p(x_i)"]
    print("\n%s prefix, N=%d, N_G=%d" % (kind, N, G))
    print("| form | " + " | ".join(keys) + " |\n|---|" + "---:|" * len(keys))
    for r in rows:
        print("| %s | " % r["form"] + " | ".join("%.1e" % r[k] for k in keys) + " |")
