"""Python binding of the tuner C ABI in include/kt.h (argument marshalling only)."""
from __future__ import annotations

import ctypes

import numpy as np

from . import nla as _nla

KT_EXHAUSTIVE, KT_MODEL_TOPK, KT_RANDOM = 0, 1, 2
KT_TRAIL_LEFT, KT_TRAIL_RIGHT, KT_GESVD = 0, 1, 2
KT_TIME, KT_ENERGY = 0, 1
FEATURES = 15


class Problem(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int), ("m", ctypes.c_int), ("n", ctypes.c_int), ("dtype", ctypes.c_int),
                ("update", ctypes.c_int), ("band", ctypes.c_int), ("reps", ctypes.c_int),
                ("objective", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("best", _nla.Cfg), ("best_ms", ctypes.c_double), ("median_ms", ctypes.c_double),
                ("default_ms", ctypes.c_double), ("evaluated", ctypes.c_int), ("valid", ctypes.c_int),
                ("failed", ctypes.c_int), ("best_lq", _nla.Cfg)]

    def as_dict(self):
        return {"best": self.best.as_tuple(), "best_ms": self.best_ms, "median_ms": self.median_ms,
                "default_ms": self.default_ms, "evaluated": self.evaluated, "valid": self.valid,
                "failed": self.failed, "best_lq": self.best_lq.as_tuple()}


_bound = False


def lib():
    global _bound
    L = _nla.lib()
    if not _bound:
        c, i, d, sz = ctypes.c_char_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        fp = ctypes.POINTER(ctypes.c_float)
        L.kt_space_size.restype = i
        L.kt_space_get.argtypes = [i, ctypes.POINTER(_nla.Cfg)]
        L.kt_cfg_valid.argtypes = [i, i, ctypes.POINTER(_nla.Cfg)]
        L.kt_cfg_valid.restype = i
        L.kt_random_subset.argtypes = [i, i, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_int)]
        L.kt_tune.argtypes = [ctypes.POINTER(Problem), i, d, c, c, ctypes.c_ulonglong, ctypes.POINTER(Result)]
        L.kt_load_config.argtypes = [c]
        L.kt_write_table.argtypes = [c, i, i, i, i, i, ctypes.POINTER(_nla.Cfg), d]
        L.kt_features.argtypes = [i, i, i, i, i, ctypes.POINTER(_nla.Cfg), fp]
        L.kt_mlp_train.argtypes = [fp, fp, i, i, i, ctypes.c_float, ctypes.c_ulonglong, c, fp]
        L.kt_mlp_predict.argtypes = [c, fp, i, fp]
        L.kt_mlp_param_count.restype = sz
        L.kt_mlp_work_bytes.argtypes = [i]
        L.kt_mlp_work_bytes.restype = sz
        vp = ctypes.c_void_p
        L.kt_mlp_forward_backward.argtypes = [vp, vp, vp, i, vp, vp, vp, sz, vp]
        L.kt_mlp_adam_step.argtypes = [vp, vp, vp, vp, sz, i, ctypes.c_float, vp]
        L.kt_energy_open.argtypes = [c]
        L.kt_energy_read.argtypes = [ctypes.POINTER(ctypes.c_ulonglong)]
        L.kt_energy_read_index.argtypes = [ctypes.c_uint, ctypes.POINTER(ctypes.c_ulonglong)]
        for f in ("kt_space_get", "kt_random_subset", "kt_tune", "kt_load_config", "kt_write_table", "kt_features",
                  "kt_mlp_train", "kt_mlp_predict", "kt_mlp_forward_backward", "kt_mlp_adam_step",
                  "kt_energy_open", "kt_energy_read", "kt_energy_read_index"):
            getattr(L, f).restype = i
        _bound = True
    return L


def _b(s):
    return None if s is None else str(s).encode()


def space():
    L = lib()
    out = []
    c = _nla.Cfg()
    for k in range(L.kt_space_size()):
        _nla._check(L.kt_space_get(k, ctypes.byref(c)))
        out.append(c.as_tuple())
    return out


def cfg_valid(kernel, dtype, cfg):
    c = _nla.Cfg.make(*cfg)
    return bool(lib().kt_cfg_valid(int(kernel), int(dtype), ctypes.byref(c)))


def random_subset(count, k, seed):
    out = (ctypes.c_int * max(k, 1))()
    _nla._check(lib().kt_random_subset(int(count), int(k), int(seed), out))
    return [out[i] for i in range(min(k, count))]


def features(kernel, m, n, dtype, update, cfg):
    c = _nla.Cfg.make(*cfg)
    out = (ctypes.c_float * FEATURES)()
    _nla._check(lib().kt_features(int(kernel), int(m), int(n), int(dtype), int(update), ctypes.byref(c), out))
    return np.array(out[:], dtype=np.float32)


def tune(kernel, m, n, dtype, update=0, band=0, reps=0, strategy=KT_EXHAUSTIVE, budget_frac=0.05, cache=None,
         model=None, seed=0, objective=0):
    p = Problem(int(kernel), int(m), int(n), int(dtype), int(update), int(band), int(reps), int(objective))
    r = Result()
    _nla._check(lib().kt_tune(ctypes.byref(p), int(strategy), float(budget_frac), _b(cache), _b(model), int(seed),
                              ctypes.byref(r)))
    return r.as_dict()


def load_config(path):
    _nla._check(lib().kt_load_config(_b(path)))


def write_table(path, side, m, n, dtype, update, cfg, ms):
    c = _nla.Cfg.make(*cfg)
    _nla._check(lib().kt_write_table(_b(path), int(side), int(m), int(n), int(dtype), int(update), ctypes.byref(c),
                                     float(ms)))


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def mlp_train(X, y, epochs=60, batch=256, lr=1e-3, seed=0, model_path="kt_mlp.bin"):
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    loss = ctypes.c_float(0)
    _nla._check(lib().kt_mlp_train(_fptr(X), _fptr(y), X.shape[0], int(epochs), int(batch), float(lr), int(seed),
                                   _b(model_path), ctypes.byref(loss)))
    return float(loss.value)


def mlp_predict(model_path, X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.zeros(X.shape[0], dtype=np.float32)
    _nla._check(lib().kt_mlp_predict(_b(model_path), _fptr(X), X.shape[0], _fptr(y)))
    return y


def mlp_param_count():
    return int(lib().kt_mlp_param_count())


def mlp_forward_backward(params, X, y, stream=None):
    """params, X, y: CUDA float32 tensors; returns (pred, grads)."""
    import torch

    rows = X.shape[0]
    grads = torch.empty_like(params)
    pred = torch.empty(rows, dtype=torch.float32, device=X.device)
    work = torch.empty(int(lib().kt_mlp_work_bytes(rows)), dtype=torch.uint8, device=X.device)
    vp = ctypes.c_void_p
    _nla._check(lib().kt_mlp_forward_backward(vp(params.data_ptr()), vp(X.data_ptr()), vp(y.data_ptr()), rows,
                                              vp(pred.data_ptr()), vp(grads.data_ptr()), vp(work.data_ptr()),
                                              work.numel(), _nla._stream_ptr(stream)))
    return pred, grads


def mlp_adam_step(params, grads, m, v, t, lr, stream=None):
    vp = ctypes.c_void_p
    _nla._check(lib().kt_mlp_adam_step(vp(params.data_ptr()), vp(grads.data_ptr()), vp(m.data_ptr()),
                                       vp(v.data_ptr()), params.numel(), int(t), float(lr), _nla._stream_ptr(stream)))


def energy_open(nvml_path=None):
    _nla._check(lib().kt_energy_open(_b(nvml_path)))


def energy_read(index=None):
    """Energy counter (millijoules) of the current CUDA device, or of NVML device `index`."""
    v = ctypes.c_ulonglong(0)
    if index is None:
        _nla._check(lib().kt_energy_read(ctypes.byref(v)))
    else:
        _nla._check(lib().kt_energy_read_index(int(index), ctypes.byref(v)))
    return int(v.value)
