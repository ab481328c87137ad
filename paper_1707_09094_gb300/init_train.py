"""Training and evaluation of the learned initialiser (set encoder).

Training sets: seeded synthetic diagonal mixtures (the c1 distributions of
synth.py at the requested D and N_G), P points sampled from each; the target
of a set is the plain method's own fit of those points -- k-means (10
iterations) + EM (10 iterations) through the batched form.  Training runs the
library's BF16 forward/backward kernels and Adam (gmm_init_net_step).

Evaluation on held-out mixtures with many samples: EM to convergence
(em_tol) from (a) the network's prediction on P sampled points, (b) the
paper's k-means seeding (random subset, 10 iterations) and (c) the network's
means as k-means seeds (3 iterations); reported per set: data passes
(k-means + EM iterations), final mean log-likelihood.  Seeding policies:
`learned_kmeans_em` is (c) with (b) as the fallback when the prediction is
not finite; `learned_or_kmeans` uses the prediction directly and -- with
judge=True -- keeps whichever of (a) and (b) reaches the higher final EM
log-likelihood (the paper's objective is the judge).
"""
from __future__ import annotations

import time

import numpy as np

from . import GMM, GMM_KEEP_EXISTING, GmmError, InitNet, learn_batched, synth


def make_sets(n_sets: int, D: int, G: int, P: int, seed0: int, fit: bool = True, km_iter: int = 10,
              em_iter: int = 10, var_floor: float = 1e-3):
    """Return (pts float32 [n][P][D], targets (means, dcovs, hefts) or None)."""
    import torch
    pts = np.empty((n_sets, P, D), np.float32)
    for s in range(n_sets):
        rng = np.random.default_rng(seed0 + s)
        mix = synth.mixture_c1(rng, D, G)
        X, _ = synth._draw(rng, mix, P)
        pts[s] = X
    if not fit:
        return pts, None
    tm = np.empty((n_sets, G, D)); tv = np.empty((n_sets, G, D)); tw = np.empty((n_sets, G))
    dev = torch.from_numpy(pts).cuda()
    step = 4096
    for s0 in range(0, n_sets, step):
        chunk = [dev[s] for s in range(s0, min(n_sets, s0 + step))]
        models = learn_batched(chunk, G, km_iter=km_iter, em_iter=em_iter, seed=seed0 + s0, var_floor=var_floor)
        for k, m in enumerate(models):
            tm[s0 + k], tv[s0 + k], tw[s0 + k] = m.get_params()
    return pts, (tm, tv, tw)


def train(net: InitNet, pts, targets, steps: int, batch: int = 64, lr: float = 1e-3, lam: float = 0.1,
          var_floor: float = 1e-3, seed: int = 0, log_every: int = 0):
    """Adam training on random batches; returns the loss history."""
    import torch
    rng = np.random.default_rng(seed)
    P_dev = torch.from_numpy(pts).cuda()
    T = None if targets is None else [torch.from_numpy(np.ascontiguousarray(t)).cuda() for t in targets]
    hist = []
    for it in range(steps):
        idx = torch.from_numpy(rng.choice(pts.shape[0], batch, replace=False)).cuda()
        xb = P_dev.index_select(0, idx).contiguous()
        tb = None if T is None else [t.index_select(0, idx).contiguous() for t in T]
        loss, _ = net.step(xb, tb, lam=lam if tb is not None else 0.0, var_floor=var_floor, mode=2, lr=lr)
        hist.append(loss)
        if log_every and it % log_every == 0:
            print("step %d loss %.4f" % (it, loss), flush=True)
    return np.array(hist)


def em_from(model: GMM, X, max_iter: int, em_tol: float, var_floor: float):
    """EM to convergence from the model's current parameters; (iterations, final mean LL)."""
    G = model.n_gaus
    model.learn(X, G, seed_mode=GMM_KEEP_EXISTING, km_iter=0, em_iter=max_iter, em_tol=em_tol, var_floor=var_floor)
    return len(model.ll_history()), model.avg_log_p(X)


def evaluate(net: InitNet, X_list, P: int, max_iter: int = 300, em_tol: float = 1e-6, var_floor: float = 1e-3,
             seed: int = 0, km_iter: int = 10, hybrid_km: int = 0):
    """Per set: k-means seeding vs learned seeding, EM to convergence.  With
    hybrid_km > 0 also the learned means refined by hybrid_km k-means
    iterations before EM (k-means seeded by the network instead of by a
    random subset)."""
    rows = []
    for j, X in enumerate(X_list):
        G = net.n_gaus
        t0 = time.perf_counter()
        base = GMM().learn(X, G, km_iter=km_iter, em_iter=max_iter, em_tol=em_tol, seed=seed + j,
                           var_floor=var_floor)
        base_ll, base_it = base.avg_log_p(X), len(base.ll_history())
        t1 = time.perf_counter()
        g = GMM()
        try:
            net.seed_model(g, X, P=P, seed=seed + j, var_floor=var_floor)
            init_ll = g.avg_log_p(X)
            it, ll = em_from(g, X, max_iter, em_tol, var_floor)
            ok = True
        except GmmError:
            it, ll, init_ll, ok = 0, -np.inf, -np.inf, False
        t2 = time.perf_counter()
        row = {"kmeans_passes": km_iter + base_it, "kmeans_em_iters": base_it, "kmeans_ll": base_ll,
               "learned_em_iters": it, "learned_passes": it, "learned_ll": ll, "learned_init_ll": init_ll,
               "learned_ok": ok, "kmeans_s": t1 - t0, "learned_s": t2 - t1}
        if hybrid_km > 0 and ok:
            h = GMM()
            net.seed_model(h, X, P=P, seed=seed + j, var_floor=var_floor)
            h.learn(X, G, seed_mode=GMM_KEEP_EXISTING, km_iter=hybrid_km, em_iter=max_iter, em_tol=em_tol,
                    var_floor=var_floor)
            row.update({"hybrid_km": hybrid_km, "hybrid_passes": hybrid_km + len(h.ll_history()),
                        "hybrid_ll": h.avg_log_p(X)})
        rows.append(row)
    return rows


def learned_kmeans_em(net: InitNet, X, P: int = 4096, km_iter: int = 3, em_iter: int = 250, em_tol: float = 1e-6,
                      var_floor: float = 1e-3, seed: int = 0, fallback_km_iter: int = 10):
    """Seeding with the network: its predicted means seed k-means (km_iter
    iterations, Sec. 3) in place of a random subset, then EM to convergence.
    Falls back to the paper's k-means seeding (random subset, fallback_km_iter
    iterations) when the prediction is not finite.  Returns (model, policy)."""
    G = net.n_gaus
    g = GMM()
    try:
        net.seed_model(g, X, P=P, seed=seed, var_floor=var_floor)
        g.learn(X, G, seed_mode=GMM_KEEP_EXISTING, km_iter=km_iter, em_iter=em_iter, em_tol=em_tol,
                var_floor=var_floor)
        if np.isfinite(g.ll_history()).all():
            return g, "learned+kmeans"
    except GmmError:
        pass
    base = GMM().learn(X, G, km_iter=fallback_km_iter, em_iter=em_iter, em_tol=em_tol, seed=seed, var_floor=var_floor)
    return base, "kmeans"


def learned_or_kmeans(net: InitNet, X, P: int = 4096, em_iter: int = 300, em_tol: float = 1e-6,
                      var_floor: float = 1e-3, seed: int = 0, judge: bool = False, km_iter: int = 10):
    """Seeding policy: learned start, k-means start as the fallback (and, with
    judge=True, as the competitor: the higher final log-likelihood wins)."""
    G = net.n_gaus
    g = GMM()
    try:
        net.seed_model(g, X, P=P, seed=seed, var_floor=var_floor)
        em_from(g, X, em_iter, em_tol, var_floor)
        ok = np.isfinite(g.ll_history()).all()
    except GmmError:
        ok = False
    if ok and not judge:
        return g, "learned"
    base = GMM().learn(X, G, km_iter=km_iter, em_iter=em_iter, em_tol=em_tol, seed=seed, var_floor=var_floor)
    if not ok or base.avg_log_p(X) > g.avg_log_p(X):
        return base, "kmeans"
    return g, "learned"


def fit_sets_dev(pts, G: int, seed0: int, km_iter: int = 10, em_iter: int = 10, var_floor: float = 1e-3,
                 chunk: int = 4096):
    """The plain method's fit of every set of the device tensor pts [n][P][D]
    (batched k-means + EM, fit s seeded seed0 + s); device FP64 targets."""
    import torch
    n, _, D = pts.shape
    tm = torch.empty((n, G, D), dtype=torch.float64, device=pts.device)
    tv = torch.empty((n, G, D), dtype=torch.float64, device=pts.device)
    tw = torch.empty((n, G), dtype=torch.float64, device=pts.device)
    for s0 in range(0, n, chunk):
        s1 = min(n, s0 + chunk)
        models = learn_batched([pts[s] for s in range(s0, s1)], G, km_iter=km_iter, em_iter=em_iter,
                               seed=seed0 + s0, var_floor=var_floor)
        ps = [m.get_params() for m in models]
        tm[s0:s1] = torch.from_numpy(np.stack([p[0] for p in ps])).to(pts.device)
        tv[s0:s1] = torch.from_numpy(np.stack([p[1] for p in ps])).to(pts.device)
        tw[s0:s1] = torch.from_numpy(np.stack([p[2] for p in ps])).to(pts.device)
        del models
    return tm, tv, tw


def train_dev(net: InitNet, pts, targets, epochs: float, batch: int = 16, lr: float = 1e-3, lr_final: float = 1e-4,
              lam: float = 0.1, var_floor: float = 1e-3, seed: int = 0):
    """Adam over shuffled batches of the device-resident sets (learning rate
    decayed geometrically from lr to lr_final); returns the loss history."""
    import torch
    n = pts.shape[0]
    rng = np.random.default_rng(seed)
    steps = max(1, int(round(epochs * n / batch)))
    order = np.concatenate([rng.permutation(n) for _ in range(int(np.ceil(epochs)) + 1)])
    hist = np.empty(steps)
    for it in range(steps):
        idx = torch.from_numpy(order[it * batch:(it + 1) * batch]).to(pts.device)
        xb = pts.index_select(0, idx)
        tb = [t.index_select(0, idx) for t in targets]
        lr_t = lr * (lr_final / lr) ** (it / max(steps - 1, 1))
        hist[it], _ = net.step(xb, tb, lam=lam, var_floor=var_floor, mode=2, lr=lr_t)
    return hist


def c5_experiment(n_train: int = 200_000, epochs: float = 2.0, n_eval: int = 64, eval_n: int = 1_000_000,
                  D: int = 32, G: int = 32, P: int = 4096, batch: int = 16, var_floor: float = 1e-3,
                  em_tol: float = 1e-6, max_iter: int = 250, seed_train: int = 5_000_000, seed_eval: int = 9_000_000,
                  chunk: int = 4096, lr: float = 1e-3, lam: float = 0.1, hybrid_km: int = 0, log=None):
    """The learned-initialiser workload: a set encoder (per point D-256-256-256,
    mean pool, 256-512-512-512-G(1+2D)) trained on n_train seeded c1-style
    mixtures of P points fitted by the plain method (batched k-means 10 + EM
    10), then evaluated on n_eval held-out mixtures of eval_n samples: EM to
    convergence (em_tol, at most max_iter iterations) from the learned start
    and from k-means seeding (10 iterations).  Returns the per-set rows and
    paired summaries (data passes, final mean log-likelihood)."""
    import torch
    out = {"n_train": n_train, "epochs": epochs, "D": D, "G": G, "P": P, "eval_sets": n_eval, "eval_n": eval_n,
           "lr": lr, "lambda": lam, "hybrid_km": hybrid_km}
    t0 = time.perf_counter()
    pts = torch.empty((n_train, P, D), dtype=torch.float32, device="cuda")
    for s0 in range(0, n_train, chunk):
        s1 = min(n_train, s0 + chunk)
        mixes = [synth.mixture_c1(np.random.default_rng(seed_train + s), D, G) for s in range(s0, s1)]
        pts[s0:s1] = synth.draw_sets_torch(mixes, P, seed=seed_train + s0)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    tgt = fit_sets_dev(pts, G, seed_train, var_floor=var_floor, chunk=chunk)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    if log:
        log("c5: %d sets drawn in %.1f s, fitted in %.1f s" % (n_train, t1 - t0, t2 - t1))
    net = InitNet(D, G, 256, 512, 3, 3, seed=0)
    hist = train_dev(net, pts, tgt, epochs, batch=batch, lr=lr, lr_final=lr / 10, lam=lam, var_floor=var_floor)
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    del pts, tgt
    torch.cuda.empty_cache()
    if log:
        log("c5: %d training steps in %.1f s, loss %.3f -> %.3f" % (hist.size, t3 - t2, hist[:100].mean(),
                                                                     hist[-100:].mean()))
    rows = []
    for j in range(n_eval):
        mix = synth.mixture_c1(np.random.default_rng(seed_eval + j), D, G)
        X = synth.draw_sets_torch([mix], eval_n, seed=seed_eval + j)[0].contiguous()
        rows += evaluate(net, [X], P=P, max_iter=max_iter, em_tol=em_tol, var_floor=var_floor, seed=seed_eval + j,
                         hybrid_km=hybrid_km)
        del X
    t4 = time.perf_counter()
    out.update(summarise(rows))
    out.update({"train_steps": int(hist.size), "loss_first": float(hist[:100].mean()),
                "loss_last": float(hist[-100:].mean()), "draw_s": t1 - t0, "fit_s": t2 - t1, "train_s": t3 - t2,
                "eval_s": t4 - t3, "rows": rows})
    return out


def summarise(rows):
    """Paired comparison of the learned start with k-means seeding: mean data
    passes to convergence (k-means iterations count as passes), mean final
    log-likelihood, and the mean paired difference learned - k-means with its
    standard error."""
    km = np.array([r["kmeans_ll"] for r in rows])
    ln = np.array([r["learned_ll"] for r in rows])
    d = ln - km
    se = float(d.std(ddof=1) / np.sqrt(d.size)) if d.size > 1 else float("nan")
    pk = np.array([r["kmeans_passes"] for r in rows], np.float64)
    pl = np.array([r["learned_passes"] for r in rows], np.float64)
    extra = {}
    if rows and "hybrid_ll" in rows[0]:
        hy = np.array([r["hybrid_ll"] for r in rows])
        dh = hy - km
        extra = {"passes_hybrid": float(np.mean([r["hybrid_passes"] for r in rows])), "ll_hybrid": float(hy.mean()),
                 "hybrid_diff_mean": float(dh.mean()),
                 "hybrid_diff_se": float(dh.std(ddof=1) / np.sqrt(dh.size)) if dh.size > 1 else float("nan"),
                 "hybrid_better": int((dh > 1e-6).sum()), "hybrid_worse": int((dh < -1e-6).sum())}
    return {**extra, "passes_kmeans": float(pk.mean()), "passes_learned": float(pl.mean()),
            "passes_saved": float((pk - pl).mean()), "ll_kmeans": float(km.mean()), "ll_learned": float(ln.mean()),
            "ll_diff_mean": float(d.mean()), "ll_diff_se": se, "learned_better": int((d > 1e-6).sum()),
            "kmeans_better": int((d < -1e-6).sum()), "ll_judged": float(np.maximum(km, ln).mean())}


def step_bench(B: int = 16, P: int = 4096, D: int = 32, G: int = 32, steps: int = 10, warmup: int = 3):
    """Time Adam training steps of the set encoder (per point D-256-256-256,
    mean pool, 256-512-512-512-G(1+2D)) on synthetic sets; returns ms/step."""
    import torch
    net = InitNet(D, G, 256, 512, 3, 3, seed=0)
    gen = torch.Generator(device="cuda").manual_seed(7)
    pts = torch.randn((B, P, D), device="cuda", generator=gen) * 2.0
    tgt = (torch.randn((B, G, D), device="cuda", generator=gen, dtype=torch.float64),
           torch.rand((B, G, D), device="cuda", generator=gen, dtype=torch.float64) + 0.5,
           torch.full((B, G), 1.0 / G, device="cuda", dtype=torch.float64))
    for _ in range(warmup):
        net.step(pts, tgt, lam=0.1, mode=2)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(steps):
        net.step(pts, tgt, lam=0.1, mode=2)
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / max(steps, 1)


def _main(argv=None):
    import argparse
    import json
    ap = argparse.ArgumentParser(prog="python -m paper_1707_09094_gb300.init_train")
    sub = ap.add_subparsers(dest="cmd", required=True)
    b = sub.add_parser("step-bench", help="time training steps")
    b.add_argument("--sets", type=int, default=16)
    b.add_argument("--points", type=int, default=4096)
    b.add_argument("--steps", type=int, default=10)
    b.add_argument("--warmup", type=int, default=3)
    c = sub.add_parser("c5", help="the learned-initialiser workload (D=32, N_G=32, 4096 points per set)")
    c.add_argument("--sets", type=int, default=200_000)
    c.add_argument("--epochs", type=float, default=2.0)
    c.add_argument("--eval", type=int, default=64)
    c.add_argument("--eval-n", type=int, default=1_000_000)
    c.add_argument("--out", default=None, help="write the result (JSON) here")
    t = sub.add_parser("train", help="train on fitted synthetic sets, evaluate against k-means seeding")
    t.add_argument("--D", type=int, default=8)
    t.add_argument("--G", type=int, default=8)
    t.add_argument("--points", type=int, default=512)
    t.add_argument("--sets", type=int, default=4000)
    t.add_argument("--steps", type=int, default=1500)
    t.add_argument("--eval", type=int, default=16)
    t.add_argument("--eval-n", type=int, default=100_000)
    t.add_argument("--save", default=None, help="write the trained weights (float32 .npy)")
    a = ap.parse_args(argv)
    from . import build
    build.build()
    if a.cmd == "step-bench":
        ms = step_bench(a.sets, a.points, steps=a.steps, warmup=a.warmup)
        print(json.dumps({"ms_per_step": ms, "sets": a.sets, "points_per_set": a.points}))
        return 0
    if a.cmd == "c5":
        r = c5_experiment(a.sets, a.epochs, a.eval, a.eval_n, log=lambda m: print(m, flush=True))
        summ = {k: v for k, v in r.items() if k != "rows"}
        print(json.dumps(summ))
        if a.out:
            with open(a.out, "w") as f:
                json.dump(r, f)
        return 0
    import torch
    pts, tgt = make_sets(a.sets, a.D, a.G, a.points, seed0=5_000_000)
    net = InitNet(a.D, a.G, 128, 256, 3, 3, seed=0)
    hist = train(net, pts, tgt, steps=a.steps)
    Xs = []
    for j in range(a.eval):
        rng = np.random.default_rng(9_000_000 + j)
        X, _ = synth._draw(rng, synth.mixture_c1(rng, a.D, a.G), a.eval_n)
        Xs.append(torch.from_numpy(X).cuda())
    rows = evaluate(net, Xs, P=a.points)
    km = np.array([r["kmeans_ll"] for r in rows])
    ln = np.array([r["learned_ll"] for r in rows])
    print(json.dumps({"loss_first": float(hist[:50].mean()), "loss_last": float(hist[-50:].mean()),
                      "passes_kmeans": float(np.mean([r["kmeans_passes"] for r in rows])),
                      "passes_learned": float(np.mean([r["learned_passes"] for r in rows])),
                      "ll_kmeans": float(km.mean()), "ll_learned": float(ln.mean()),
                      "ll_judged": float(np.maximum(km, ln).mean())}))
    if a.save:
        np.save(a.save, net.get_weights())
    return 0


if __name__ == "__main__":
    raise SystemExit(_main())
