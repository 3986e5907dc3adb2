"""The C-ABI library loads and exports every entry point include/qk.h declares
(no compute call: runs without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(qk_[a-z_0-9]+)\s*\(", txt)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = _declared()
    for want in ("qk_init_patches", "qk_fill_ghosts", "qk_hydro_stage", "qk_rad_stage",
                 "qk_rad_matter_exchange", "qk_step", "qk_conserved_sums", "qk_destroy"):
        assert want in names


def test_library_exports_every_declared_symbol():
    from paper_2110_01792_gb300 import build as B
    try:
        path = B.build()
    except (RuntimeError, FileNotFoundError) as e:  # no nvcc on this host
        pytest.skip(f"cannot build libqk: {e}")
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def _qk():
    from paper_2110_01792_gb300 import build as B
    try:
        B.build()
    except (RuntimeError, FileNotFoundError) as e:
        pytest.skip(f"cannot build libqk: {e}")
    from paper_2110_01792_gb300 import qk
    return qk


def _init(qk, boxes, dom, ng=4, prec=0, **prm):
    arr = (qk.Box * max(1, len(boxes)))()
    for i, (lo, n, off) in enumerate(boxes):
        for d in range(3):
            arr[i].lo[d] = lo[d]
            arr[i].n[d] = n[d]
        arr[i].offset = off
    p = qk.make_params(**dict(dict(hydro_only=1, dx=0.1), **prm))
    h = ctypes.c_void_p()
    dn = (ctypes.c_int32 * 3)(*dom)
    rc = qk.lib().qk_init_patches(ctypes.byref(h), ctypes.byref(p), arr, len(boxes), dn, ng, prec)
    msg = qk.lib().qk_last_error(None).decode()
    if rc == 0:
        qk.lib().qk_destroy(h)
    return rc, msg


def test_init_rejects_invalid_patch_sets():
    """qk_init_patches validates before touching the GPU: empty sets, gaps,
    overlaps, boxes outside the domain, shared field ranges, too few ghost
    cells, unknown precision and invalid parameters are QK_EINVAL with a
    message (runs on CPU)."""
    qk = _qk()
    vol = lambda n, g=4: (n[0] + 2 * g) * (n[1] + 2 * g) * (n[2] + 2 * g)
    a = ((0, 0, 0), (8, 8, 8), 0)
    b = ((8, 0, 0), (8, 8, 8), vol((8, 8, 8)))
    cases = [
        ([], (16, 8, 8), {}, "no boxes"),
        ([a], (16, 8, 8), {}, "cover"),                      # gap
        ([a, ((4, 0, 0), (8, 8, 8), vol((8, 8, 8)))], (16, 8, 8), {}, "overlap"),
        ([a, ((8, 0, 0), (16, 8, 8), vol((8, 8, 8)))], (16, 8, 8), {}, "outside"),
        ([a, ((8, 0, 0), (8, 8, 8), 10)], (16, 8, 8), {}, "field range"),
        ([a, b], (16, 8, 8), {"ng": 2}, "nghost"),
        ([a, b], (16, 8, 8), {"prec": 7}, "precision"),
        ([a, b], (16, 8, 8), {"gamma": 1.0, "c_v": 1.0}, "gamma"),
        ([a, b], (16, 8, 8), {"hydro_only": 0, "chat": 0.0}, "chat"),
        ([((0, 0, 0), (0, 8, 8), 0)], (16, 8, 8), {}, "empty extent"),
    ]
    for boxes, dom, kw, word in cases:
        ng = kw.pop("ng", 4)
        prec = kw.pop("prec", 0)
        rc, msg = _init(qk, boxes, dom, ng, prec, **kw)
        assert rc == qk.EINVAL, (word, rc, msg)
        assert word.split()[0] in msg.lower() or word in msg.lower(), (word, msg)


def test_init_shard_rejects_invalid_ownership():
    """qk_init_shard checks the owner array and the rank before touching the
    GPU: NULL owner, owners outside [0, nranks), a rank outside the range, a
    rank that owns no patch, and overlapping field ranges among the patches
    this rank owns are QK_EINVAL with a message (runs on CPU)."""
    qk = _qk()
    vol = (8 + 8) * (8 + 8) * (8 + 8)
    boxes = [((0, 0, 0), (8, 8, 8), 0), ((8, 0, 0), (8, 8, 8), vol)]
    arr = (qk.Box * 2)()
    for i, (lo, n, off) in enumerate(boxes):
        for d in range(3):
            arr[i].lo[d] = lo[d]
            arr[i].n[d] = n[d]
        arr[i].offset = off
    p = qk.make_params(hydro_only=1, dx=0.1)
    dn = (ctypes.c_int32 * 3)(16, 8, 8)
    L = qk.lib()

    def init(owner, nranks, rank, offsets=None):
        if offsets is not None:
            for i, o in enumerate(offsets):
                arr[i].offset = o
        h = ctypes.c_void_p()
        own = None if owner is None else (ctypes.c_int32 * 2)(*owner)
        rc = L.qk_init_shard(ctypes.byref(h), ctypes.byref(p), arr, 2, dn, 4, 0, own, nranks, rank)
        if rc == 0:
            L.qk_destroy(h)
        return rc, L.qk_last_error(None).decode()

    cases = [
        ((None, 2, 0, None), "owner is null"),
        (([0, 2], 2, 0, None), "outside"),
        (([0, 1], 2, 2, None), "rank 2 of 2"),
        (([0, 0], 2, 1, None), "owns no patch"),
        (([0, 0], 1, 0, [0, 10]), "field range"),
    ]
    for (owner, nranks, rank, offs), word in cases:
        rc, msg = init(owner, nranks, rank, offs)
        assert rc == qk.EINVAL, (word, rc, msg)
        assert word in msg.lower(), (word, msg)



def test_lo16_host_encoding_round_trip():
    """The host form of the 16-bit low parts keeps hi + lo to ~2^-39 of the
    value over a wide range of magnitudes and signs, with |k| <= 2^14."""
    from paper_2110_01792_gb300 import qk
    rng = np.random.Generator(np.random.Philox(5))
    x = rng.lognormal(0.0, 8.0, 200000) * rng.choice([-1.0, 1.0], 200000)
    hi = x.astype(np.float32)
    k = qk.lo16_encode(hi, x - hi.astype(np.float64))
    back = hi.astype(np.float64) + qk.lo16_decode(hi, k)
    assert np.abs(k).max() <= 2 ** 14
    assert np.max(np.abs(back - x) / np.abs(x)) <= 2.0 ** -38
