"""Learned initialiser on the GPU: loss and gradients of the BF16 kernels
against the FP64 network oracle, and a short training run."""
import numpy as np
import pytest
import torch

from oracle import init_net as orc
from paper_1707_09094_gb300 import InitNet

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1707_09094_gb300 import build
    build.build()


@pytest.mark.parametrize("cfg", [dict(D=4, G=3, Hp=16, Hh=32, Lp=2, Lh=1, B=3, P=96, tol=0.05),
                                 dict(D=32, G=32, Hp=64, Hh=64, Lp=3, Lh=3, B=2, P=256, tol=0.12)])
def test_gradients_match_oracle(cfg):
    """BF16 operands with FP32 accumulation against the FP64 network oracle.

    Every GEMM rounds both operands to BF16 (unit roundoff 2^-8), forward
    and backward, so the gradient error grows with depth: the whole vector
    must lie within `tol` (relative norm: 5% for the 3-layer net, 12% for
    the 7-layer one) and point the same way (cosine > 0.995); each layer's
    block must have cosine > 0.98, which a dropped term or a transposed
    operand in any one layer's backward pass fails."""
    D, G, Hp, Hh, Lp, Lh, B, P = (cfg[k] for k in ("D", "G", "Hp", "Hh", "Lp", "Lh", "B", "P"))
    net = InitNet(D, G, Hp, Hh, Lp, Lh, seed=3)
    w = net.get_weights().astype(np.float64)
    rng = np.random.default_rng(4)
    pts = rng.normal(0, 1.5, (B, P, D)).astype(np.float32)
    tgt = (rng.normal(0, 1, (B, G, D)), rng.uniform(0.5, 2, (B, G, D)), rng.dirichlet(np.ones(G), B))
    loss, _ = net.step(torch.from_numpy(pts).cuda(), [torch.from_numpy(t).cuda() for t in tgt], lam=0.2,
                       var_floor=1e-3, mode=1)
    g = net.get_grads().astype(np.float64)
    ref_loss, ref_g, _ = orc.loss_and_grad(w, pts, G, D, Hp, Hh, Lp, Lh, 1e-3, tgt, lam=0.2)
    assert loss == pytest.approx(ref_loss, rel=1e-2)

    def cmp(a, b):
        return np.linalg.norm(a - b) / np.linalg.norm(b), a @ b / (np.linalg.norm(a) * np.linalg.norm(b))

    per_layer, o = [], 0
    for (fo, fi) in orc.layer_shapes(D, G, Hp, Hh, Lp, Lh):
        n = fo * fi + fo
        per_layer.append(cmp(g[o:o + n], ref_g[o:o + n]))
        o += n
    rel, cos = cmp(g, ref_g)
    assert rel < cfg["tol"] and cos > 0.995, (rel, cos, per_layer)
    assert all(c > 0.98 for _, c in per_layer), per_layer


def test_training_reduces_loss():
    rng = np.random.default_rng(5)
    D, G, P = 4, 3, 128
    net = InitNet(D, G, 32, 32, 2, 1, seed=1)
    pts = torch.from_numpy(rng.normal(0, 1, (8, P, D)).astype(np.float32) * 2 + 1).cuda()
    first, _ = net.step(pts, mode=0, var_floor=1e-3)
    for _ in range(200):
        net.step(pts, mode=2, lr=3e-3, var_floor=1e-3)
    last, _ = net.step(pts, mode=0, var_floor=1e-3)
    assert last < first - 0.5


def test_learned_seeds_gain_over_kmeans_seeding_at_the_initialiser_shape():
    """The initialiser workload's shape (D=32, N_G=32, 4096 points per set, the
    per-point 32-256-256-256 / mean pool / 256-512-512-512 network) trained on
    32,768 mixtures fitted by the plain method, then 24 held-out mixtures of
    N = 1e6 samples each fitted to convergence (em_tol 1e-6) three ways.  The
    gain, paired per set: the network's means used as k-means seeds (3
    iterations) reach a higher final mean log-likelihood than the paper's
    k-means seeding (random subset, 10 iterations) -- the mean difference
    lies above zero by more than 1.645 standard errors (a one-sided 95 %
    bound) -- in fewer data passes on average.  The network's start used directly (no k-means) converges in
    the fewest passes but to a lower likelihood at this shape; that is
    reported, not asserted."""
    from paper_1707_09094_gb300 import init_train
    r = init_train.c5_experiment(n_train=32768, epochs=2.0, n_eval=24, eval_n=1_000_000, lr=3e-3, lam=1.0,
                                 hybrid_km=3)
    print("\nk-means: LL %.4f, %.1f passes; learned+k-means(3): LL %.4f (%+.3f +- %.3f), %.1f passes, "
          "better on %d/%d; learned alone: LL %.4f (%+.3f +- %.3f), %.1f passes"
          % (r["ll_kmeans"], r["passes_kmeans"], r["ll_hybrid"], r["hybrid_diff_mean"], r["hybrid_diff_se"],
             r["passes_hybrid"], r["hybrid_better"], len(r["rows"]), r["ll_learned"], r["ll_diff_mean"],
             r["ll_diff_se"], r["passes_learned"]))
    assert r["loss_last"] < r["loss_first"]
    assert all(row["learned_ok"] for row in r["rows"])
    assert r["hybrid_diff_mean"] - 1.645 * r["hybrid_diff_se"] > 0.0, r   # one-sided 95 % paired bound
    assert r["passes_hybrid"] < r["passes_kmeans"], r


def test_checkpoint_resumes_training(tmp_path):
    """Weights + Adam moments + step count saved after 5 steps and loaded into a
    fresh net reproduce the next steps' losses (FP32 atomics in the weight
    gradients reorder sums, hence the tolerance)."""
    rng = np.random.default_rng(8)
    D, G = 8, 4
    pts = torch.from_numpy(rng.normal(0, 1.5, (4, 128, D)).astype(np.float32)).cuda()
    tgt = [torch.from_numpy(t).cuda() for t in (rng.normal(0, 1, (4, G, D)), rng.uniform(0.5, 2, (4, G, D)),
                                                 rng.dirichlet(np.ones(G), 4))]
    a = InitNet(D, G, 32, 32, 2, 2, seed=1)
    for _ in range(5):
        a.step(pts, tgt, lam=0.1, mode=2, lr=1e-2)
    path = str(tmp_path / "ckpt.npz")
    a.save_checkpoint(path)
    assert a.get_state()["adam_step"] == 5
    b = InitNet(D, G, 32, 32, 2, 2, seed=99).load_checkpoint(path)
    for _ in range(3):
        la, _ = a.step(pts, tgt, lam=0.1, mode=2, lr=1e-2)
        lb, _ = b.step(pts, tgt, lam=0.1, mode=2, lr=1e-2)
        assert lb == pytest.approx(la, rel=1e-4)
    np.testing.assert_allclose(b.get_weights(), a.get_weights(), rtol=1e-3, atol=1e-5)
