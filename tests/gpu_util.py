"""Helpers shared by the GPU parity tests: host/device conversion and error
measures. Inputs come from paper_2603_09668_gb300.inputs; expected values come
from the oracle only."""
import numpy as np
import torch

from paper_2603_09668_gb300 import binding as B


def dev():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch.device("cuda:0")


def to_dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(dev())


def state_to_dev(st):
    return B.MpmState(*(to_dev(np.asarray(a, np.float32)) for a in st))


def state_to_np(st):
    return tuple(a.detach().cpu().numpy().astype(np.float64) for a in st)


def f64(st):
    return tuple(np.asarray(a, np.float64) for a in st)


def max_rel(a, b):
    """max |a - b| / max |b| (0/0 -> 0)."""
    den = np.abs(b).max()
    num = np.abs(a - b).max()
    return 0.0 if num == 0 else num / max(den, 1e-30)


def rel_l2(a, b):
    den = np.linalg.norm(b)
    num = np.linalg.norm(a - b)
    return 0.0 if num == 0 else num / max(den, 1e-30)


def wind_dev(values_np, t_total):
    return B.WindField(to_dev(values_np.astype(np.float32)), float(t_total))


def wind_ref(values_np, t_total):
    v = np.asarray(values_np, np.float64)
    return (v, v.shape[1], v.shape[0], float(t_total))
