"""Python names for the format-selection entry points (include/ffspmv_select.h).

Argument marshalling only: the features, the exhaustive search, the network's
forward/backward/Adam/inference all run in libffspmv.so.
"""
from __future__ import annotations

import ctypes

import numpy as np

from ._api import _ptr, stream_ptr
from ._lib import (MLP_HIDDEN, MLP_IN, MLP_OUT, MLP_PARAMS, NUM_BIN_FEATURES, NUM_BINS,
                   NUM_FEATURES, NUM_FORMATS, SELECTOR_WEIGHTS, Options, check, lib,
                   options_default)

FORMAT_NAMES = ["ELL_R", "CSR/1", "CSR/2", "CSR/4", "CSR/8", "CSR/16", "CSR/32", "CSR-CTA",
                "CSR-split", "COO"]


def _torch():
    import torch
    return torch


def matrix_features(A, stream=None):
    """(float[16], float[17][6]) features of an object with nrows, ncols,
    row_ptr, col, val, modulus, computed by the device kernels."""
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    rp = torch.from_numpy(np.ascontiguousarray(A.row_ptr, dtype=np.int64)).to(dev)
    cl = torch.from_numpy(np.ascontiguousarray(A.col, dtype=np.int32)).to(dev)
    vl = torch.from_numpy(np.ascontiguousarray(A.val, dtype=np.uint32).view(np.int32)).to(dev)
    f = torch.empty(NUM_FEATURES, dtype=torch.float32, device=dev)
    bf = torch.empty((NUM_BINS, NUM_BIN_FEATURES), dtype=torch.float32, device=dev)
    check(lib().ffspmv_matrix_features(A.nrows, A.ncols, _ptr(rp), _ptr(cl), _ptr(vl),
                                       int(A.modulus), _ptr(f), _ptr(bf), stream_ptr(stream)),
          "ffspmv_matrix_features")
    return f.cpu().numpy(), bf.cpu().numpy()


def tune_bins(A, max_rows=16384, max_nnz=1 << 21, reps=5):
    """The exhaustive per-bin search: dict with times[17][10] (ms per call, NaN
    = invalid), pm_times[17][2], sample_nnz[17], best[17][3]."""
    times = np.zeros((NUM_BINS, NUM_FORMATS), dtype=np.float32)
    pm = np.zeros((NUM_BINS, 2), dtype=np.float32)
    snnz = np.zeros(NUM_BINS, dtype=np.int64)
    best = np.zeros((NUM_BINS, 3), dtype=np.int32)
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(A.col, dtype=np.int32)
    vl = np.ascontiguousarray(A.val, dtype=np.uint32)
    check(lib().ffspmv_tune_bins(A.nrows, A.ncols, int(rp[-1]), _ptr(rp), _ptr(cl), _ptr(vl),
                                 int(A.modulus), int(max_rows), int(max_nnz), int(reps),
                                 _ptr(times), _ptr(pm), _ptr(snnz), _ptr(best)),
          "ffspmv_tune_bins")
    return {"times": times, "pm_times": pm, "sample_nnz": snnz, "best": best}


def selector_choose(A, with_layout=False):
    """best[17][3] from the installed selector network (inference kernel);
    with_layout: (best, layout), layout one of LAYOUT_BINNED (heuristic
    table), LAYOUT_NETBINS (binned, the network's table) or LAYOUT_PANEL."""
    best = np.zeros((NUM_BINS, 3), dtype=np.int32)
    layout = np.zeros(1, dtype=np.int32)
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(A.col, dtype=np.int32)
    vl = np.ascontiguousarray(A.val, dtype=np.uint32)
    check(lib().ffspmv_selector_choose(A.nrows, A.ncols, int(rp[-1]), _ptr(rp), _ptr(cl),
                                       _ptr(vl), int(A.modulus), _ptr(best), _ptr(layout)),
          "ffspmv_selector_choose")
    return (best, int(layout[0])) if with_layout else best


def heuristic_choose(A, use_pm1=-1):
    """best[17][3] of the heuristic table for A."""
    best = np.zeros((NUM_BINS, 3), dtype=np.int32)
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    vl = np.ascontiguousarray(A.val, dtype=np.uint32)
    check(lib().ffspmv_heuristic_choose(A.nrows, _ptr(rp), _ptr(vl), int(A.modulus), int(use_pm1),
                                        _ptr(best)), "ffspmv_heuristic_choose")
    return best


def selector_load(params):
    """Install selector weights (float32[MLP_PARAMS]); None uninstalls."""
    if params is None:
        check(lib().ffspmv_selector_load(None, 0), "ffspmv_selector_load")
        return
    w = np.ascontiguousarray(params, dtype=np.float32)
    check(lib().ffspmv_selector_load(_ptr(w), int(w.size)), "ffspmv_selector_load")


def create_binned(A, best, options=None, **opts):
    """A handle whose binned plan uses the per-bin choice best[17][3]."""
    from ._api import Matrix
    if options is None:
        options = options_default(**opts)
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    cl = np.ascontiguousarray(A.col, dtype=np.int32)
    vl = np.ascontiguousarray(A.val, dtype=np.uint32)
    b = np.ascontiguousarray(best, dtype=np.int32)
    h = ctypes.c_void_p()
    check(lib().spmv_create_binned(ctypes.byref(h), A.nrows, A.ncols, int(rp[-1]), _ptr(rp),
                                   _ptr(cl), _ptr(vl), int(A.modulus), _ptr(b),
                                   ctypes.byref(options), None), "spmv_create_binned")
    M = Matrix.__new__(Matrix)
    M.nrows, M.ncols, M.modulus, M.options, M.handle = A.nrows, A.ncols, A.modulus, options, h
    return M


class MLP:
    """The selector network on the device: parameters, Adam moments and the
    forward / loss / backward / Adam kernels of the library."""

    def __init__(self, params=None, seed=0):
        torch = _torch()
        self.dev = torch.device("cuda", torch.cuda.current_device())
        if params is None:
            params = init_params(seed)
        self.p = torch.from_numpy(np.ascontiguousarray(params, dtype=np.float32)).to(self.dev)
        self.m = torch.zeros_like(self.p)
        self.v = torch.zeros_like(self.p)
        self.g = torch.zeros_like(self.p)
        self.step_count = 0

    def forward(self, x):
        torch = _torch()
        x = x.contiguous()
        B = x.shape[0]
        act = torch.empty((B, 2 * MLP_HIDDEN), dtype=torch.float32, device=self.dev)
        out = torch.empty((B, MLP_OUT), dtype=torch.float32, device=self.dev)
        check(lib().ffspmv_mlp_forward(_ptr(self.p), _ptr(x), B, _ptr(act), _ptr(out),
                                       stream_ptr()), "ffspmv_mlp_forward")
        return out, act

    def loss_and_grad(self, x, target, mask):
        torch = _torch()
        out, act = self.forward(x)
        dout = torch.empty_like(out)
        loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        check(lib().ffspmv_mlp_loss(_ptr(out), _ptr(target.contiguous()), _ptr(mask.contiguous()),
                                    x.shape[0], _ptr(dout), _ptr(loss), stream_ptr()),
              "ffspmv_mlp_loss")
        check(lib().ffspmv_mlp_backward(_ptr(self.p), _ptr(x.contiguous()), x.shape[0], _ptr(act),
                                        _ptr(dout), _ptr(self.g), stream_ptr()),
              "ffspmv_mlp_backward")
        return loss, self.g

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        check(lib().ffspmv_mlp_adam(_ptr(self.p), _ptr(self.g), _ptr(self.m), _ptr(self.v),
                                    self.step_count, lr, b1, b2, eps, stream_ptr()),
              "ffspmv_mlp_adam")

    def params(self):
        return self.p.detach().cpu().numpy().copy()


def init_params(seed=0):
    """He-uniform weights, zero biases, in the flat layout of ffspmv_select.h."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((MLP_IN, MLP_HIDDEN), (MLP_HIDDEN, MLP_HIDDEN), (MLP_HIDDEN, MLP_OUT)):
        lim = np.sqrt(6.0 / fan_in)
        parts.append(rng.uniform(-lim, lim, (fan_out, fan_in)).astype(np.float32).ravel())
        parts.append(np.zeros(fan_out, dtype=np.float32))
    p = np.concatenate(parts)
    assert p.size == MLP_PARAMS
    return p


__all__ = ["matrix_features", "tune_bins", "selector_choose", "heuristic_choose",
           "selector_load", "create_binned",
           "MLP", "init_params", "FORMAT_NAMES", "SELECTOR_WEIGHTS"]
