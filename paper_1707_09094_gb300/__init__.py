"""GB300 (sm_103a) diagonal-GMM training by k-means + EM (arXiv 1707.09094).

The computation runs in the CUDA library built from ``csrc/`` (C ABI in
``include/gmm_gb300.h``); this package only marshals arguments.  Inputs may
be torch tensors (CUDA or CPU) or numpy arrays; PyTorch supplies device
memory and the current stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _lib
from ._lib import (GMM_BF16, GMM_EUCL, GMM_FP32, GMM_KEEP_EXISTING, GMM_MAHA, GMM_PROB,  # noqa: F401
                   GMM_RANDOM_SPREAD, GMM_RANDOM_SUBSET, GMM_STATIC_SPREAD, GMM_STATIC_SUBSET,
                   GmmError)

PREC = {"fp32": GMM_FP32, "bf16": GMM_BF16}


def _torch():
    import torch
    return torch


def _stream_ptr(X):
    torch = _torch()
    if isinstance(X, torch.Tensor) and X.is_cuda:
        return ctypes.c_void_p(torch.cuda.current_stream(X.device).cuda_stream)
    return ctypes.c_void_p(0)


def _as_input(X):
    """(pointer, N, D, keepalive) for a float32 [N][D] tensor/array.  FP64
    samples (the paper's double input) are rounded to FP32: CUDA tensors by
    the library's conversion kernel, host data on the host."""
    torch = _torch()
    if isinstance(X, torch.Tensor):
        if X.dim() != 2 or X.dtype not in (torch.float32, torch.float64):
            raise ValueError("X must be a float32 or float64 [N][D] tensor")
        X = X.contiguous()
        if X.dtype == torch.float64:
            if not X.is_cuda:
                return _as_input(X.numpy())
            X32 = torch.empty(X.shape, dtype=torch.float32, device=X.device)
            _lib.check(_lib.load().gmm_x_from_f64(ctypes.c_void_p(X.data_ptr()), X.numel(),
                                                  ctypes.c_void_p(X32.data_ptr()), _stream_ptr(X)),
                       "gmm_x_from_f64")
            X = X32
        return ctypes.c_void_p(X.data_ptr()), X.shape[0], X.shape[1], X
    A = np.ascontiguousarray(X, dtype=np.float32)
    if A.ndim != 2:
        raise ValueError("X must be [N][D]")
    return A.ctypes.data_as(ctypes.c_void_p), A.shape[0], A.shape[1], A


def _out_like(X, n, dtype):
    torch = _torch()
    if isinstance(X, torch.Tensor) and X.is_cuda:
        t = torch.empty(n, dtype={np.float64: torch.float64, np.int32: torch.int32}[dtype], device=X.device)
        return ctypes.c_void_p(t.data_ptr()), t
    a = np.empty(n, dtype)
    return a.ctypes.data_as(ctypes.c_void_p), a


class GMM:
    """A diagonal-covariance GMM held on the GPU (the paper's gmm_diag)."""

    def __init__(self):
        lib = _lib.load()
        h = ctypes.c_void_p()
        _lib.check(lib.gmm_create(ctypes.byref(h)), "gmm_create")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.load().gmm_destroy(h)
            self._h = None

    # --------------------------------------------------------------- training
    def learn(self, X, n_gaus, dist_mode=GMM_MAHA, seed_mode=GMM_RANDOM_SUBSET, km_iter=10, em_iter=10,
              var_floor=1e-10, print_mode=False, seed=0, em_tol=0.0, prec="fp32"):
        ptr, N, D, keep = _as_input(X)
        o = _lib.gmm_learn_opts()
        _lib.load().gmm_default_opts(ctypes.byref(o))
        o.dist, o.seed_mode, o.seed, o.em_tol = dist_mode, seed_mode, seed & (2**64 - 1), em_tol
        o.prec, o.print, o.stream = PREC.get(prec, prec), int(print_mode), _stream_ptr(X)
        _lib.check(_lib.load().gmm_learn(self._h, ptr, N, D, n_gaus, km_iter, em_iter, var_floor, ctypes.byref(o)),
                   "gmm_learn")
        del keep
        return self

    def em_iterate(self, X, n_iter, var_floor=1e-10, prec="fp32", recompute_center=False):
        ptr, N, D, keep = _as_input(X)
        _lib.check(_lib.load().gmm_em_iterate(self._h, ptr, N, n_iter, var_floor, PREC.get(prec, prec),
                                              int(recompute_center), _stream_ptr(X)), "gmm_em_iterate")
        del keep
        return self

    def kmeans(self, X, km_iter, dist_mode=GMM_MAHA, var_floor=1e-10, return_assign=True):
        ptr, N, D, keep = _as_input(X)
        optr, out = _out_like(X, N, np.int32) if return_assign else (ctypes.c_void_p(0), None)
        _lib.check(_lib.load().gmm_kmeans(self._h, ptr, N, km_iter, dist_mode, var_floor, optr, _stream_ptr(X)),
                   "gmm_kmeans")
        del keep
        return out

    # -------------------------------------------------------------- inference
    def log_p(self, X, g=-1):
        ptr, N, D, keep = _as_input(X)
        optr, out = _out_like(X, N, np.float64)
        _lib.check(_lib.load().gmm_log_p(self._h, ptr, N, g, optr, _stream_ptr(X)), "gmm_log_p")
        del keep
        return out

    def avg_log_p(self, X, g=-1):
        ptr, N, D, keep = _as_input(X)
        v = ctypes.c_double()
        _lib.check(_lib.load().gmm_avg_log_p(self._h, ptr, N, g, ctypes.byref(v), _stream_ptr(X)), "gmm_avg_log_p")
        del keep
        return v.value

    def assign(self, X, dist_mode=GMM_EUCL):
        ptr, N, D, keep = _as_input(X)
        optr, out = _out_like(X, N, np.int32)
        _lib.check(_lib.load().gmm_assign(self._h, ptr, N, dist_mode, optr, _stream_ptr(X)), "gmm_assign")
        del keep
        return out

    def raw_hist(self, X, dist_mode=GMM_EUCL):
        ptr, N, D, keep = _as_input(X)
        out = np.empty(self.n_gaus, np.int64)
        _lib.check(_lib.load().gmm_raw_hist(self._h, ptr, N, dist_mode, out.ctypes.data_as(ctypes.c_void_p),
                                            _stream_ptr(X)), "gmm_raw_hist")
        del keep
        return out

    def norm_hist(self, X, dist_mode=GMM_EUCL):
        ptr, N, D, keep = _as_input(X)
        out = np.empty(self.n_gaus, np.float64)
        _lib.check(_lib.load().gmm_norm_hist(self._h, ptr, N, dist_mode, out.ctypes.data_as(ctypes.c_void_p),
                                             _stream_ptr(X)), "gmm_norm_hist")
        del keep
        return out

    # ------------------------------------------------------------- parameters
    def _shape(self):
        D, G = ctypes.c_int32(), ctypes.c_int32()
        _lib.check(_lib.load().gmm_get_params(self._h, ctypes.byref(D), ctypes.byref(G), None, None, None),
                   "gmm_get_params")
        return D.value, G.value

    @property
    def n_dims(self):
        return self._shape()[0]

    @property
    def n_gaus(self):
        return self._shape()[1]

    def get_params(self):
        D, G = self._shape()
        m = np.empty((G, D)); v = np.empty((G, D)); h = np.empty(G)
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        _lib.check(_lib.load().gmm_get_params(self._h, None, None, vp(m), vp(v), vp(h)), "gmm_get_params")
        return m, v, h

    @property
    def means(self):
        return self.get_params()[0]

    @property
    def dcovs(self):
        return self.get_params()[1]

    @property
    def hefts(self):
        return self.get_params()[2]

    def set_params(self, means, dcovs, hefts):
        m = np.ascontiguousarray(means, np.float64)
        v = np.ascontiguousarray(dcovs, np.float64)
        h = np.ascontiguousarray(hefts, np.float64)
        G, D = m.shape
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        _lib.check(_lib.load().gmm_set_params(self._h, D, G, vp(m), vp(v), vp(h)), "gmm_set_params")
        return self

    def reset(self, n_dims, n_gaus):
        """reset() of Sec. 4.1: zero means, unit covariances, uniform hefts."""
        return self.set_params(np.zeros((n_gaus, n_dims)), np.ones((n_gaus, n_dims)),
                               np.full(n_gaus, 1.0 / n_gaus))

    def generate(self, N, seed=0, device="cuda"):
        """M.generate(N) of Sec. 4.1: N samples of the model as a float32 [N][D]
        tensor on `device` ("cuda") or a numpy array (device=None)."""
        D = self.get_params()[0].shape[1]
        if device is None:
            out = np.empty((N, D), np.float32)
            ptr = out.ctypes.data_as(ctypes.c_void_p)
            stream = None
        else:
            torch = _torch()
            out = torch.empty((N, D), dtype=torch.float32, device=device)
            ptr = ctypes.c_void_p(out.data_ptr())
            stream = _stream_ptr(out)
        _lib.check(_lib.load().gmm_generate(self._h, N, seed & (2**64 - 1), ptr, stream), "gmm_generate")
        return out

    def save(self, path):
        """M.save(filename) of Sec. 4.1."""
        _lib.check(_lib.load().gmm_save(self._h, os.fsencode(path)), "gmm_save")
        return self

    def load(self, path):
        """M.load(filename) of Sec. 4.1."""
        _lib.check(_lib.load().gmm_load(self._h, os.fsencode(path)), "gmm_load")
        return self

    def profile(self, enable=True):
        """Start (reset) or stop event timing of the fused-pass launches."""
        _lib.check(_lib.load().gmm_profile(self._h, int(enable)), "gmm_profile")
        return self

    def profile_read(self):
        """(summed pass time in ms, pass launches, library kernel launches)."""
        ms, n, k = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
        _lib.check(_lib.load().gmm_profile_read(self._h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(k)),
                   "gmm_profile_read")
        return ms.value, n.value, k.value

    def debug_set(self, key, value):
        """Test hooks (GMM_DEBUG_WAIT_CYCLES, GMM_DEBUG_SKIP_MMA, GMM_DEBUG_KM_FORM, GMM_DEBUG_FP32_FORM,
        GMM_DEBUG_TC_FORM)."""
        _lib.check(_lib.load().gmm_debug_set(self._h, key, int(value)), "gmm_debug_set")
        return self

    def screen_stats(self):
        """(samples screened, candidates kept, dense fallbacks) of the tensor-core pass since profile()."""
        out = []
        for k in (_lib.GMM_STAT_SCREENED, _lib.GMM_STAT_KEPT, _lib.GMM_STAT_DENSE):
            v = ctypes.c_int64()
            _lib.check(_lib.load().gmm_debug_get(self._h, k, ctypes.byref(v)), "gmm_debug_get")
            out.append(v.value)
        return tuple(out)

    def km_screen_stats(self):
        """(samples screened, deferred to the exact FP32 decision, re-decided in FP64) of the
        tensor-core k-means since profile()."""
        out = []
        for k in (_lib.GMM_STAT_KM_SCREENED, _lib.GMM_STAT_KM_DEFERRED, _lib.GMM_STAT_KM_FP64):
            v = ctypes.c_int64()
            _lib.check(_lib.load().gmm_debug_get(self._h, k, ctypes.byref(v)), "gmm_debug_get")
            out.append(v.value)
        return tuple(out)

    def phase_cycles(self):
        """Per-phase SM cycles of the tensor-core pass since profile() (summed over CTAs)."""
        out = []
        for k in range(8):
            v = ctypes.c_int64()
            _lib.check(_lib.load().gmm_debug_get(self._h, 6 + k, ctypes.byref(v)), "gmm_debug_get")
            out.append(v.value)
        return out

    def ll_history(self, cap=4096):
        out = np.empty(cap)
        n = ctypes.c_int32()
        _lib.check(_lib.load().gmm_get_stats(self._h, out.ctypes.data_as(ctypes.c_void_p), cap, ctypes.byref(n)),
                   "gmm_get_stats")
        return out[: n.value].copy()


def learn_batched(Xs, n_gaus, km_iter=10, em_iter=10, var_floor=1e-10, dist_mode=GMM_MAHA, seed=0, em_tol=0.0,
                  print_mode=False):
    """Batched learn(): one GMM per array/tensor in Xs (fit f seeds from seed + f).
    n_gaus is an int or a sequence.  Returns the list of fitted GMM objects."""
    n = len(Xs)
    gs = list(n_gaus) if hasattr(n_gaus, "__len__") else [int(n_gaus)] * n
    models = [GMM() for _ in range(n)]
    keep, ptrs, Ns, Ds = [], [], [], []
    for X in Xs:
        p, N, D, k = _as_input(X)
        keep.append(k); ptrs.append(p.value); Ns.append(N); Ds.append(D)
    arr = lambda t, v: (t * len(v))(*v)  # noqa: E731
    o = _lib.gmm_learn_opts()
    _lib.load().gmm_default_opts(ctypes.byref(o))
    o.dist, o.seed, o.em_tol, o.print = dist_mode, seed & (2**64 - 1), em_tol, int(print_mode)
    hs = arr(ctypes.c_void_p, [m._h.value for m in models])
    _lib.check(_lib.load().gmm_learn_batched(hs, n, arr(ctypes.c_void_p, ptrs), arr(ctypes.c_int64, Ns),
                                             arr(ctypes.c_int32, Ds), arr(ctypes.c_int32, gs), km_iter, em_iter,
                                             var_floor, ctypes.byref(o)), "gmm_learn_batched")
    del keep
    return models


class InitNet:
    """Learned initialiser (set encoder) on the GPU; see gmm_init_net_* in the C header."""

    def __init__(self, D=32, n_gaus=32, hidden_point=256, hidden_head=512, point_layers=3, head_layers=3, seed=0):
        h = ctypes.c_void_p()
        _lib.check(_lib.load().gmm_init_net_create(ctypes.byref(h), D, n_gaus, hidden_point, hidden_head,
                                                   point_layers, head_layers, seed & (2**64 - 1)),
                   "gmm_init_net_create")
        self._h, self.D, self.n_gaus = h, D, n_gaus

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.load().gmm_init_net_destroy(h)
            self._h = None

    @property
    def num_params(self):
        return int(_lib.load().gmm_init_net_num_params(self._h))

    def get_weights(self):
        w = np.empty(self.num_params, np.float32)
        _lib.check(_lib.load().gmm_init_net_get_weights(self._h, w.ctypes.data_as(ctypes.c_void_p), None), "get")
        return w

    def get_grads(self):
        g = np.empty(self.num_params, np.float32)
        _lib.check(_lib.load().gmm_init_net_get_weights(self._h, None, g.ctypes.data_as(ctypes.c_void_p)), "get")
        return g

    def set_weights(self, w):
        w = np.ascontiguousarray(w, np.float32)
        _lib.check(_lib.load().gmm_init_net_set_weights(self._h, w.ctypes.data_as(ctypes.c_void_p)), "set")
        return self

    def get_state(self):
        """Training checkpoint: weights, Adam moments and step count."""
        n = self.num_params
        m1, m2, t = np.empty(n, np.float32), np.empty(n, np.float32), ctypes.c_int64()
        _lib.check(_lib.load().gmm_init_net_get_adam(self._h, m1.ctypes.data_as(ctypes.c_void_p),
                                                     m2.ctypes.data_as(ctypes.c_void_p), ctypes.byref(t)),
                   "gmm_init_net_get_adam")
        return {"weights": self.get_weights(), "adam_m1": m1, "adam_m2": m2, "adam_step": t.value}

    def set_state(self, state):
        self.set_weights(state["weights"])
        m1 = np.ascontiguousarray(state["adam_m1"], np.float32)
        m2 = np.ascontiguousarray(state["adam_m2"], np.float32)
        _lib.check(_lib.load().gmm_init_net_set_adam(self._h, m1.ctypes.data_as(ctypes.c_void_p),
                                                     m2.ctypes.data_as(ctypes.c_void_p), int(state["adam_step"])),
                   "gmm_init_net_set_adam")
        return self

    def save_checkpoint(self, path):
        np.savez(path, **self.get_state())

    def load_checkpoint(self, path):
        with np.load(path) as z:
            return self.set_state({k: z[k] for k in z.files})

    def step(self, pts, targets=None, lam=0.0, var_floor=1e-3, mode=0, lr=1e-3, want_pred=False):
        """pts: CUDA float32 tensor [B][P][D]; targets: (means, dcovs, hefts) CUDA float64 tensors or None.
        Returns (loss, pred) with pred = (means, dcovs, hefts) CUDA tensors when want_pred."""
        torch = _torch()
        B, P, D = pts.shape
        tp = [ctypes.c_void_p(0)] * 3 if targets is None else [ctypes.c_void_p(t.data_ptr()) for t in targets]
        pred = None
        pp = [ctypes.c_void_p(0)] * 3
        if want_pred:
            G = self.n_gaus
            pred = (torch.empty((B, G, D), dtype=torch.float64, device=pts.device),
                    torch.empty((B, G, D), dtype=torch.float64, device=pts.device),
                    torch.empty((B, G), dtype=torch.float64, device=pts.device))
            pp = [ctypes.c_void_p(t.data_ptr()) for t in pred]
        loss = ctypes.c_double()
        _lib.check(_lib.load().gmm_init_net_step(self._h, ctypes.c_void_p(pts.data_ptr()), B, P, tp[0], tp[1], tp[2],
                                                 lam, var_floor, mode, lr, pp[0], pp[1], pp[2], ctypes.byref(loss),
                                                 _stream_ptr(pts)), "gmm_init_net_step")
        return loss.value, pred

    def seed_model(self, model, X, P=4096, seed=0, var_floor=1e-3):
        ptr, N, D, keep = _as_input(X)
        _lib.check(_lib.load().gmm_init_net_seed_model(self._h, model._h, ptr, N, P, seed & (2**64 - 1), var_floor,
                                                       _stream_ptr(X)), "gmm_init_net_seed_model")
        del keep
        return model
