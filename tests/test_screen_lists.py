"""Host-side model of the candidate lists kept by the blocked tensor-core
screen (no GPU): the blocks of 128 Gaussians are visited once; each sample
keeps its best lower bound so far and appends every Gaussian whose upper
bound reaches that bound minus T, stored with the bound rounded up to BF16;
when the list passes 32 entries, and after the last block, entries whose
stored bound falls below the current bound minus T are dropped; a list that
would pass 64 entries marks the sample for the FP32 form.  The model checks
that the final list is exactly the set {g : ub_g >= max_g lb_g - T} up to the
BF16 rounding of the stored bound, in Gaussian order, whenever the sample
is not marked."""
import numpy as np

CAP, PRUNE_AT, BLOCK = 64, 32, 128


def bf16_up(v):
    """The screen's encoding: the top 16 bits of the FP32 value, rounded up."""
    u = np.float32(v).view(np.uint32)
    h = int(u) >> 16
    if (int(u) >> 31) == 0 and (int(u) & 0xFFFF) != 0:
        h += 1
    return np.uint32(h << 16).view(np.float32)


def screen_list(lb, ub, T):
    """Candidates of one sample as the screen keeps them: (sorted list, marked)."""
    G = lb.size
    mrun, lst, lost = -np.inf, [], False
    for b0 in range(0, G, BLOCK):
        blk = slice(b0, min(G, b0 + BLOCK))
        mrun = max(mrun, float(lb[blk].max()))
        thr = mrun - T
        if len(lst) > CAP - 32:   # the owner's prune before the block's appends
            lost = lost or len(lst) > CAP
            lst = [e for e in lst[:CAP] if e[1] >= thr]
        for g in range(b0, min(G, b0 + BLOCK)):
            if ub[g] >= thr:
                lst.append((g, float(bf16_up(ub[g]))))
    lost = lost or len(lst) > CAP
    final = [e for e in lst[:CAP] if e[1] >= mrun - T]
    return sorted(g for g, _ in final), lost or not final, mrun


def test_lists_equal_the_candidate_set():
    rng = np.random.default_rng(11)
    T = float(np.log(1e7 * 1e9))
    marked = 0
    for trial in range(400):
        G = int(rng.choice([128, 300, 1024, 4096]))
        # log-densities with a long tail, a few near the best, the best in a random block
        l = rng.normal(-3000, 800, G).astype(np.float32)
        close = rng.integers(0, G, int(rng.integers(1, 20)))
        l[close] = rng.normal(0, 15, close.size).astype(np.float32)
        err = np.abs(rng.normal(0, 2, G)).astype(np.float32) + 1.0   # the screen's bound K1 |P1| + k2
        lb, ub = (l - err).astype(np.float32), (l + err).astype(np.float32)
        got, lost, mrun = screen_list(lb, ub, T)
        assert mrun == float(lb.max())
        if lost:
            marked += 1
            continue
        want = [g for g in range(G) if ub[g] >= lb.max() - T]
        # a stored bound rounds up, so entries just below the line may stay: a superset by at most
        # those within one BF16 step of it
        assert set(want) <= set(got)
        extra = set(got) - set(want)
        assert all(float(bf16_up(ub[g])) >= lb.max() - T for g in extra)
        assert got == sorted(got)
    assert marked < 40


def test_overflow_marks_the_sample():
    T = 30.0
    G = 256
    lb = np.full(G, -1000.0, np.float32)
    ub = lb + 1.0
    lb[:70], ub[:70] = -1.0, 1.0          # 70 candidates, all within T of the best
    got, lost, _ = screen_list(lb, ub, T)
    assert lost
    lb[:60], ub[:60] = -1.0, 1.0
    lb[60:70], ub[60:70] = -1000.0, -999.0
    got, lost, _ = screen_list(lb, ub, T)
    assert not lost and got == list(range(60))


def test_rising_bound_drops_early_entries():
    """Entries admitted against an early, low best lower bound are dropped once
    a later block raises it: 40 near-equal Gaussians in block 0, the best in
    block 3 far above them."""
    T = 30.0
    G = 512
    lb = np.full(G, -5000.0, np.float32)
    lb[:40] = -100.0
    lb[400] = 0.0
    ub = lb + 1.0
    got, lost, mrun = screen_list(lb, ub, T)
    assert not lost and mrun == 0.0 and got == [400]
