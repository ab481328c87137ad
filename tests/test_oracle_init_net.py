"""Pins of the FP64 network oracle: reverse-mode gradients against central
finite differences, and the loss of a one-Gaussian output against scipy."""
import numpy as np
import scipy.stats

from oracle import init_net as net


def _setup(seed=0, D=3, G=2, Hp=5, Hh=4, Lp=2, Lh=1, B=2, P=7):
    rng = np.random.default_rng(seed)
    shapes = net.layer_shapes(D, G, Hp, Hh, Lp, Lh)
    n = sum(o * i + o for o, i in shapes)
    w = rng.normal(0, 0.5, n)
    pts = rng.normal(0, 1.5, (B, P, D))
    tgt = (rng.normal(0, 1, (B, G, D)), rng.uniform(0.5, 2, (B, G, D)), rng.dirichlet(np.ones(G), B))
    return w, pts, tgt, (G, D, Hp, Hh, Lp, Lh)


def test_gradient_matches_finite_differences():
    w, pts, tgt, (G, D, Hp, Hh, Lp, Lh) = _setup()
    loss, g, _ = net.loss_and_grad(w, pts, G, D, Hp, Hh, Lp, Lh, 1e-3, tgt, lam=0.3)
    rng = np.random.default_rng(1)
    for k in rng.choice(w.size, 40, replace=False):
        e = np.zeros_like(w)
        e[k] = 1e-6
        lp = net.loss_and_grad(w + e, pts, G, D, Hp, Hh, Lp, Lh, 1e-3, tgt, lam=0.3)[0]
        lm = net.loss_and_grad(w - e, pts, G, D, Hp, Hh, Lp, Lh, 1e-3, tgt, lam=0.3)[0]
        fd = (lp - lm) / 2e-6
        assert abs(fd - g[k]) <= 1e-5 * max(1.0, abs(fd)), (k, fd, g[k])


def test_single_gaussian_loss_is_gaussian_nll():
    rng = np.random.default_rng(2)
    D, P = 3, 50
    x = rng.normal(0, 1, (P, D))
    out = np.concatenate([[0.7], rng.normal(0, 1, D), rng.normal(0, 0.3, D)])
    loss, _ = net.set_loss_and_grad(out, x, 1, D, 1e-3, None, 0.0)
    m = out[1:1 + D]
    v = np.exp(out[1 + D:]) + 1e-3
    ref = -scipy.stats.multivariate_normal(m, np.diag(v)).logpdf(x).mean()
    assert abs(loss - ref) < 1e-12 * abs(ref)
