"""Host-side check of the rule the record-keeping EM forms rely on (no GPU):
a Gaussian whose log-density lies within T of the best over all Gaussians
also lies within T of the best of its own block, so recording per block the
candidates within T of the block's best and then keeping those within T of
log p(x) (log-sum-exp over every Gaussian) keeps exactly the pairs the
direct rule l_g - log p(x) >= -T keeps, whenever no block's record overflows;
and the responsibilities of the dropped pairs sum to less than N_G e^-T."""
import numpy as np


def _lse(l):
    m = l.max(axis=1, keepdims=True)
    return (m + np.log(np.exp(l - m).sum(axis=1, keepdims=True)))[:, 0]


def records_keep(l, block, T, cap):
    """Kept pairs through block records: (mask, overflowed samples)."""
    N, G = l.shape
    lse = _lse(l)
    keep = np.zeros_like(l, dtype=bool)
    over = np.zeros(N, dtype=bool)
    for b0 in range(0, G, block):
        lb = l[:, b0:b0 + block]
        cand = lb >= lb.max(axis=1, keepdims=True) - T
        over |= cand.sum(axis=1) > cap
        keep[:, b0:b0 + block] = cand & (lb - lse[:, None] >= -T)
    return keep, over


def test_block_records_keep_exactly_the_direct_pairs():
    rng = np.random.default_rng(0)
    T = np.log(1e6 * 1e9)
    for G, block in [(256, 64), (1024, 64), (100, 64), (7, 64)]:
        # log-densities with a few close Gaussians per sample and a long tail
        l = rng.normal(-2000, 600, (4000, G))   # well-separated: a block's other Gaussians lie far below
        near = rng.integers(0, G, (4000, 4))
        for k in range(4):
            l[np.arange(4000), near[:, k]] = rng.normal(0, 15, 4000)
        keep, over = records_keep(l, block, T, cap=8)
        direct = l - _lse(l)[:, None] >= -T
        ok = ~over
        np.testing.assert_array_equal(keep[ok], direct[ok])
        assert ok.mean() > 0.9
        # every dropped pair's responsibility is below e^-T
        gam = np.exp(l - _lse(l)[:, None])
        assert (gam[~direct] < np.exp(-T)).all()


def test_overflow_is_flagged_not_dropped():
    """A block with more candidates than its record holds flags the sample
    (it is then recomputed over every Gaussian), whatever the other blocks hold."""
    T = 30.0
    l = np.full((3, 128), -1000.0)
    l[0, :10] = 0.0            # 10 equal candidates in block 0: past a cap of 8
    l[1, [0, 70]] = 0.0        # one in each block
    l[2, :64] = np.linspace(0, -29, 64)   # all of block 0 within T
    keep, over = records_keep(l, 64, T, cap=8)
    assert over.tolist() == [True, False, True]
    assert keep[1].sum() == 2
