"""Helpers of the GPU parity tests: device copies and the parity metric."""
import numpy as np

from paper_2110_01792_gb300 import inputs as I


def dev(arrs, dtype=None):
    import torch
    out = []
    for a in arrs:
        t = torch.from_numpy(np.ascontiguousarray(a))
        if dtype is not None:
            t = t.to(dtype)
        out.append(t.cuda())
    return out


def host(ts):
    return [t.double().cpu().numpy() for t in ts]


def interior(lay, a):
    return np.concatenate([lay.interior(a, b).ravel() for b in range(lay.nbox)])


def max_rel_err(lay, got, ref):
    """max |x - x_ref| / max(|x_ref|, RMS(x_ref)) over interior cells, per field."""
    out = []
    for g, r in zip(got, ref):
        gi, ri = interior(lay, g), interior(lay, r)
        floor = max(float(np.sqrt(np.mean(ri ** 2))), 1e-300)
        out.append(float(np.max(np.abs(gi - ri) / np.maximum(np.abs(ri), floor))))
    return out


def rel_l1(lay, got, ref):
    out = []
    for g, r in zip(got, ref):
        gi, ri = interior(lay, g), interior(lay, r)
        out.append(float(np.abs(gi - ri).sum() / np.abs(ri).sum()))
    return out
