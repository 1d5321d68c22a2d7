"""Shared helpers of the GPU parity tests (imported by tests marked gpu)."""
import numpy as np


def make_ctx():
    import torch
    from paper_2104_12522_gb300 import build
    build.build()
    import paper_2104_12522_gb300 as bart
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return bart.Context(0)


def opacity_errors(got, ref, floor=1e-6):
    """Max relative error over points above floor * row max, and the worst
    per-row relative L2 error.  Arrays [..., n_nu]."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    rowmax = ref.max(axis=-1, keepdims=True)
    mask = ref > floor * rowmax
    rel = np.abs(got - ref)[mask] / ref[mask]
    num = np.sqrt(np.sum((got - ref) ** 2, axis=-1))
    den = np.sqrt(np.sum(ref ** 2, axis=-1))
    l2 = np.max(num[den > 0] / den[den > 0]) if np.any(den > 0) else 0.0
    return (float(rel.max()) if rel.size else 0.0), float(l2)


def max_rel(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(got - ref) / np.abs(ref)))
