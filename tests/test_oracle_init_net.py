"""Pins of the FP64 network oracle: reverse-mode gradients against central
finite differences, the loss of a one-Gaussian output against scipy, the
forward pass of a hand-set net against values worked out by hand, and the
pull term on a constructed case."""
import numpy as np
import pytest
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


def _hand_net():
    """A 1-point-layer, 1-head-layer net (D=1, G=2, 2 hidden units each) with
    hand-set weights, so that each stage's output is known by hand:
      point layer  h(x) = (relu(x), relu(-x))           W = [[1], [-1]], b = 0
      mean pool    over the points x = 2, -4: ((2, 0) + (0, 4)) / 2 = (1, 2)
                   (a sum pool would give (2, 4))
      head layer   z = relu((1*1 + 0*2, 1*1 - 1*2 + 0.5)) = relu((1, -0.5)) = (1, 0)
                   (without the ReLU: (1, -0.5))
      output       out = Wo z + bo = (1, 0, 3, -1, 0, ln 2): the second column
                   of Wo is all ones, so a missing head ReLU shifts every
                   output by -0.5
    giving hefts softmax(1, 0), means (3, -1), variances (e^0, e^ln2) + floor."""
    W0, b0 = np.array([[1.0], [-1.0]]), np.zeros(2)
    W1, b1 = np.array([[1.0, 0.0], [1.0, -1.0]]), np.array([0.0, 0.5])
    Wo = np.column_stack([[1.0, 0.0, 3.0, -1.0, 0.0, 0.0], np.ones(6)])
    bo = np.array([0.0, 0.0, 0.0, 0.0, 0.0, np.log(2.0)])
    w = np.concatenate([W0.ravel(), b0, W1.ravel(), b1, Wo.ravel(), bo])
    pts = np.array([[[2.0], [-4.0]]])
    return w, pts


def test_forward_with_hand_set_weights():
    """The forward pass against values worked out by hand (the mixture NLL
    from scipy's normal density): pins the ReLUs, the mean pool over P > 1
    points, the head and the output mapping of several Gaussians."""
    w, pts = _hand_net()
    loss, _, out = net.loss_and_grad(w, pts, 2, 1, 2, 2, 1, 1, 0.0)
    np.testing.assert_allclose(out[0], [1.0, 0.0, 3.0, -1.0, 0.0, np.log(2.0)], rtol=0, atol=1e-15)
    w0 = np.e / (np.e + 1.0)
    x = np.array([2.0, -4.0])
    p = w0 * scipy.stats.norm.pdf(x, 3.0, 1.0) + (1 - w0) * scipy.stats.norm.pdf(x, -1.0, np.sqrt(2.0))
    assert loss == pytest.approx(-np.log(p).mean(), rel=1e-13)
    # the variance floor is added to exp(r)
    loss_f = net.loss_and_grad(w, pts, 2, 1, 2, 2, 1, 1, 0.5)[0]
    p = w0 * scipy.stats.norm.pdf(x, 3.0, np.sqrt(1.5)) + (1 - w0) * scipy.stats.norm.pdf(x, -1.0, np.sqrt(2.5))
    assert loss_f == pytest.approx(-np.log(p).mean(), rel=1e-13)


def test_pull_term_on_a_constructed_case():
    """PULL = lambda sum_k w~_k min_g sum_d (m_gd - m~_kd)^2 / v~_kd with the
    hand net's means (3, -1): target 0 at 2.5 (variance 0.25, weight 0.6) is
    nearest to mean 0 at distance 1; target 1 at 0 (variance 4, weight 0.4)
    to mean 1 at distance 0.25; lambda = 2 gives 2 (0.6 + 0.1) = 1.4 on top of
    the NLL."""
    w, pts = _hand_net()
    tgt = (np.array([[[2.5], [0.0]]]), np.array([[[0.25], [4.0]]]), np.array([[0.6, 0.4]]))
    base = net.loss_and_grad(w, pts, 2, 1, 2, 2, 1, 1, 0.0)[0]
    loss = net.loss_and_grad(w, pts, 2, 1, 2, 2, 1, 1, 0.0, tgt, lam=2.0)[0]
    assert loss - base == pytest.approx(1.4, rel=1e-13)
