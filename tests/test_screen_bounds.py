"""The rounding bounds the tensor-core screens rely on, checked on the CPU
against emulated BF16 arithmetic (round to nearest even of the top 16 bits of
an FP32 value, products exact in FP32, FP32 accumulation).

EM screen (Eq. 15 expanded about the global centre): l~ = ctc + P1~ + P2~ with
P1 = sum x'^2 (-iv/2) and P2 = sum x' mu' iv on BF16 operands; the kernel
assumes |l~ - l| <= K1 |P1~| + k2 with K1 = 2^-6 * 1.25 and
k2 = 2^-7 * 1.25 * q/2 + 2^-21 |ctc| + 1e-4, q = sum mu'^2 iv.

k-means screen: s~ = |c'|^2 - 2 (x_hi c_hi + x_lo c_hi + x_hi c_lo) on split
BF16 operands; the kernel assumes |s~ - s| <= 2^-12 |x'| max|c'| +
2^-16 (max|c'|^2 + |x'|^2).

Random inputs and adversarial ones (every operand losing most of the 2^-8
a BF16 rounding can take, all errors of one sign) must stay inside the
bounds; the adversarial EM case also shows that half the EM constants
would not."""
import numpy as np

K1 = 2.0 ** -6 * 1.25
K2Q = 2.0 ** -7 * 1.25


def bf16(a):
    b = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b >> 16) & 1) + 0x7FFF
    return ((b + r) & 0xFFFF0000).astype(np.uint32).view(np.float32)


def em_case(xc, iv, muc, ctc=0.0):
    """(|l~ - l|, kernel bound, bound with half the constants) for one
    (sample, Gaussian) pair; xc, iv, muc: FP32 vectors of x', 1/sigma^2, mu'."""
    xc, iv, muc = (np.asarray(v, np.float32) for v in (xc, iv, muc))
    a1 = bf16(xc * xc)
    b1 = bf16(np.float32(-0.5) * iv)
    a2 = bf16(xc)
    b2 = bf16(muc * iv)
    p1 = np.float32(0.0)
    p2 = np.float32(0.0)
    for k in range(xc.size):   # FP32 accumulation of exact FP32 products
        p1 = np.float32(p1 + np.float32(a1[k] * b1[k]))
        p2 = np.float32(p2 + np.float32(a2[k] * b2[k]))
    x, v, m = (np.asarray(t, np.float64) for t in (xc, iv, muc))
    P1 = np.sum(x * x * (-0.5 * v))
    P2 = np.sum(x * m * v)
    q = np.sum(m * m * v)
    err = abs((float(p1) + float(p2)) - (P1 + P2))
    bound = K1 * abs(float(p1)) + K2Q * q / 2 + 2.0 ** -21 * abs(ctc) + 1e-4
    half = K1 / 2 * abs(float(p1)) + K2Q / 2 * q / 2 + 2.0 ** -21 * abs(ctc) + 1e-4
    return err, bound, half


def below_midpoint(n, rng, lo=0.5, hi=4.0):
    """FP32 values whose BF16 rounding error is almost 2^-8 relative, rounding down."""
    e = rng.integers(int(np.log2(lo)), int(np.log2(hi)), n).astype(np.float64)
    top = 1.0 + rng.integers(0, 128, n) / 128.0   # a BF16 value in [1, 2)
    return ((top + 2.0 ** -8 - 2.0 ** -20) * 2.0 ** e).astype(np.float32)


def test_em_bound_random():
    rng = np.random.default_rng(0)
    for _ in range(300):
        D = int(rng.integers(1, 65))
        xc = rng.normal(0, rng.uniform(0.1, 30), D)
        iv = 1.0 / rng.uniform(0.01, 9, D)
        muc = rng.normal(0, rng.uniform(0.1, 30), D)
        err, bound, _ = em_case(xc, iv, muc, ctc=rng.normal(0, 300))
        assert err <= bound, (err, bound)


def adversarial_dims(D, rng, frac=0.65):
    """(x', iv): D dimensions in which x', x'^2, -iv/2 and x' iv all lose at
    least frac * 2^-8 of their magnitude to BF16 rounding."""
    out_x, out_iv = [], []
    while len(out_x) < D:
        x = rng.uniform(0.3, 3.0, 200000).astype(np.float32)
        iv = rng.uniform(0.2, 5.0, 200000).astype(np.float32)
        vals = [x, x * x, np.float32(-0.5) * iv, -(x * iv)]
        ok = np.ones(x.size, bool)
        for v in vals:
            ok &= (np.abs(bf16(v)) - np.abs(v)) <= -frac * 2.0 ** -8 * np.abs(v)
        out_x.extend(x[ok].tolist())
        out_iv.extend(iv[ok].tolist())
    return np.array(out_x[:D], np.float32), np.array(out_iv[:D], np.float32)


def test_em_bound_adversarial_and_half_constants_fail():
    """mu' = -x': every product of the expansion loses magnitude, so the errors of
    P1 (2^-7 |P1| at most) and P2 (2^-7 * 2 |P1| at most) add up."""
    rng = np.random.default_rng(1)
    worst_half = 0.0
    for _ in range(5):
        xc, iv = adversarial_dims(64, rng)
        err, bound, half = em_case(xc, iv, -xc)
        assert err <= bound, (err, bound)
        worst_half = max(worst_half, err / half)
    assert worst_half > 1.0   # half the constants undercount the rounding of a product of two BF16 operands


def km_case(x, c_all, g):
    """(|s~_g - s_g|, kernel bound) for sample x' and means c' (FP32)."""
    x = np.asarray(x, np.float32)
    c = np.asarray(c_all[g], np.float32)
    xh = bf16(x)
    xl = bf16(x - xh)
    ch = bf16(c)
    cl = bf16(c - ch)
    p = np.float32(0.0)
    for k in range(x.size):
        for t in (xh[k] * ch[k], xl[k] * ch[k], xh[k] * cl[k]):
            p = np.float32(p + np.float32(t))
    cn = np.float32(0.0)
    for k in range(c.size):
        cn = np.float32(cn + np.float32(c[k] * c[k]))
    s_tilde = float(np.float32(cn - np.float32(2.0) * p))
    xd, cd = x.astype(np.float64), c.astype(np.float64)
    s_exact = float(cd @ cd - 2.0 * (xd @ cd))
    cn_all = (np.asarray(c_all, np.float64) ** 2).sum(1)
    xn = float(np.sqrt(xd @ xd))
    bound = 2.0 ** -12 * xn * np.sqrt(cn_all.max()) + 2.0 ** -16 * (cn_all.max() + xd @ xd) + 1e-30
    return abs(s_tilde - s_exact), bound


def test_kmeans_bound_random_and_adversarial():
    rng = np.random.default_rng(2)
    for _ in range(200):
        D = int(rng.integers(1, 65))
        G = int(rng.integers(1, 9))
        x = rng.normal(0, rng.uniform(0.1, 50), D)
        cs = rng.normal(0, rng.uniform(0.1, 50), (G, D))
        for g in range(G):
            err, bound = km_case(x, cs, g)
            assert err <= bound, (err, bound)
    for _ in range(30):
        D = 64
        x = below_midpoint(D, rng)
        cs = below_midpoint(D, rng)[None, :]
        err, bound = km_case(x, cs, 0)
        assert err <= bound, (err, bound)


# ---------------------------------------------------------------- blocked (split-BF16) EM screen
# The blocked tensor-core pass splits every FP32 operand v into BF16 parts
# v_h = bf16(v), v_l = bf16(v - v_h) and accumulates t_h a_h + t_l a_h + t_h a_l
# (t = x'^2) and x_h b_h + x_l b_h + x_h b_l in FP32; it assumes the result is
# within K1s |P1~| + k2s of the exact kernel's FP32 value
# c - 1/2 sum_d (x_d s_d - (mu s)_d)^2, with K1s = 2^-11 and
# k2s = 2^-12 q + 2^-18 r + 2^-20 |ctc| + 1e-3 (r = sum_d m_d^2 iv_d).
K1S = 2.0 ** -11


def _split(v):
    h = bf16(v)
    return h, bf16(np.asarray(v, np.float32) - h)


def _seq_sum32(p):
    """Sequential FP32 accumulation along the last axis (the MMA chain's
    order is not known; any order obeys the same bound)."""
    return np.add.accumulate(np.asarray(p, np.float32), axis=-1, dtype=np.float32)[..., -1]


def split_em_case(x, m, mu, var, w):
    """x: [P][D] FP32 samples, m: [D] FP32 centre, mu/var: [P][D] FP64 Gaussian
    parameters (one per pair), w: [P] weights.  Returns (|screen - exact|, bound)."""
    x = np.asarray(x, np.float32)
    D = x.shape[1]
    xc = (x - m[None, :]).astype(np.float32)                    # x' in FP32
    t = (xc * xc).astype(np.float32)
    iv = 1.0 / var
    a = (-0.5 * iv).astype(np.float32)
    b = ((mu - m[None, :].astype(np.float64)) * iv).astype(np.float32)
    th, tl = _split(t)
    xh, xl = _split(xc)
    ah, al = _split(a)
    bh, bl = _split(b)
    p1 = _seq_sum32(np.concatenate([th * ah, tl * ah, th * al], axis=1).astype(np.float32))
    p2 = _seq_sum32(np.concatenate([xh * bh, xl * bh, xh * bl], axis=1).astype(np.float32))
    mc = mu - m[None, :].astype(np.float64)
    q = np.sum(mc * mc * iv, axis=1)
    r = np.sum(m[None, :].astype(np.float64) ** 2 * iv, axis=1)
    c = np.log(w) - 0.5 * D * np.log(2 * np.pi) - 0.5 * np.sum(np.log(var), axis=1)
    ctc = (c - 0.5 * q).astype(np.float32)
    screen = (p1 + p2).astype(np.float32) + ctc
    # the exact kernel: s = 1/sigma, mu s in FP32, t = fma(x, s, -mu s), sum of t^2, c - r/2
    s = (1.0 / np.sqrt(var)).astype(np.float32)
    ms = (mu * (1.0 / np.sqrt(var))).astype(np.float32)
    td = (x.astype(np.float64) * s - ms).astype(np.float32)       # one rounding, as an FMA
    rr = _seq_sum32((td * td).astype(np.float32))
    exact = (c.astype(np.float32) - np.float32(0.5) * rr).astype(np.float32)
    k2 = 2.0 ** -12 * q + 2.0 ** -18 * r + 2.0 ** -20 * np.abs(ctc.astype(np.float64)) + 1e-3
    err = np.abs(screen.astype(np.float64) - exact.astype(np.float64))
    return err, K1S * np.abs(p1.astype(np.float64)) + k2


def test_split_em_bound_c3_like():
    """Pairs shaped like the precision workload (means ~ N(0, 3^2), sigma
    log-uniform on [0.1, 10], D = 128): samples of the pair's own Gaussian
    and of other Gaussians, centre near the data mean."""
    rng = np.random.default_rng(7)
    P, D = 2000, 128
    mu = rng.normal(0, 3, (P, D))
    sd = np.exp(rng.uniform(np.log(0.1), np.log(10), (P, D)))
    own = rng.random(P) < 0.5
    other_mu = rng.normal(0, 3, (P, D))
    other_sd = np.exp(rng.uniform(np.log(0.1), np.log(10), (P, D)))
    x = np.where(own[:, None], mu + sd * rng.normal(size=(P, D)), other_mu + other_sd * rng.normal(size=(P, D)))
    m = rng.normal(0, 0.3, D).astype(np.float32)
    err, bound = split_em_case(x.astype(np.float32), m, mu, sd ** 2, rng.uniform(1e-4, 1e-2, P))
    assert (err <= bound).all(), float(np.max(err / bound))
    assert np.max(err / bound) < 0.5   # the constants hold with room to spare


def test_split_em_bound_wide_ranges():
    """Variances from 1e-4 to 1e2, centres far from the data, D from 1 to 128."""
    rng = np.random.default_rng(8)
    for _ in range(40):
        D = int(rng.integers(1, 129))
        P = 200
        mu = rng.normal(0, rng.uniform(0.1, 30), (P, D))
        var = np.exp(rng.uniform(np.log(1e-4), np.log(1e2), (P, D)))
        x = (mu + np.sqrt(var) * rng.normal(size=(P, D)) * rng.uniform(0.1, 20)).astype(np.float32)
        m = rng.normal(0, rng.uniform(0.1, 30), D).astype(np.float32)
        err, bound = split_em_case(x, m, mu, var, rng.uniform(1e-6, 1, P))
        assert (err <= bound).all(), float(np.max(err / bound))
