"""The allocation-free conservation sums (qk_conserved_sums_noalloc).

That entry point exists for callers that cannot call cudaMalloc where they
need the conservation totals (a diagnostics hook under a fixed device-memory
budget, code under an external device allocator, code without a qk context).
It keeps its working memory in a fixed static device array of the library.
Here it is called through the C ABI twice in a row, on two different patch
sets and precisions, and each result must equal qk_conserved_sums of a
regular context on the same fields bit for bit (same kernels, same reduction
order).  A warm call must leave the device's free memory and the caching
allocator's counters unchanged.  One more case fills the static patch table to
its limit (exactly 4096 patches).  This file is collected last so that a
failure here does not hide the rest of the suite.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2110_01792_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2110_01792_gb300 import qk
    L = qk.lib()
    fn = L.qk_conserved_sums_noalloc
    fn.argtypes = [C.POINTER(qk.Params), C.POINTER(qk.Box), C.c_int32, C.c_int32, C.c_int32,
                   C.c_int64, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                   C.POINTER(C.c_double), C.c_void_p, C.c_char_p, C.c_int32]
    fn.restype = C.c_int
    return torch, qk, fn


def _state(lay, seed, with_rad):
    prob = I.rhd_lognormal(layout=lay, seed=seed)
    rng = np.random.Generator(np.random.Philox(seed))
    for b in range(lay.nbox):
        rho = lay.interior(prob.U[0], b)
        for d in range(3):
            lay.interior(prob.U[1 + d], b)[...] = rho * 0.2 * rng.standard_normal(rho.shape)
        for d in range(3):
            lay.interior(prob.R[1 + d], b)[...] = 5.0 * rng.standard_normal(rho.shape)
    return prob.U, (prob.R if with_rad else None), dict(prob.params, dx=1.0 / lay.dom_n[0])


def _boxes(qk, lay):
    arr = (qk.Box * lay.nbox)()
    for b in range(lay.nbox):
        for d in range(3):
            arr[b].lo[d] = int(lay.lo[b][d])
            arr[b].n[d] = int(lay.n[b][d])
        arr[b].offset = int(lay.off[b])
    return arr


def _ptrs(ts):
    return (C.c_void_p * len(ts))(*[t.data_ptr() for t in ts])


def _noalloc(qk, fn, lay, prm, prec, dU, dR, stream):
    out = (C.c_double * qk.NSUMS)()
    err = C.create_string_buffer(256)
    params = qk.make_params(**prm)
    rc = fn(C.byref(params), _boxes(qk, lay), lay.nbox, lay.ng, prec, lay.field_len, _ptrs(dU),
            _ptrs(dR) if dR is not None else None, out, C.c_void_p(stream), err, 256)
    assert rc == qk.OK, err.value.decode()
    return np.array(out[:])


def _memory(torch):
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    st = torch.cuda.memory_stats()
    return free, st.get("allocation.all.allocated", 0), st.get("reserved_bytes.all.current", 0)


def test_noalloc_sums_match_context_sums_on_two_calls(env):
    torch, qk, fn = env
    cases = [
        (I.make_layout([[0, 0, 0], [13, 0, 0], [0, 7, 0]],
                       [[13, 7, 11], [6, 17, 11], [13, 10, 11]], (19, 17, 11), 4),
         21, qk.FP64, True),
        (I.patch_tiling(dom_n=(48, 40, 32), seed=5, ng=3, edges=(8, 16, 24)), 22,
         qk.FP32_MIXED, False),
    ]
    stream = torch.cuda.current_stream().cuda_stream
    for lay, seed, prec, with_rad in cases:
        U, R, prm = _state(lay, seed, with_rad)
        tdt = torch.float64 if prec == qk.FP64 else torch.float32
        dU = [torch.from_numpy(a).cuda().to(tdt) for a in U]
        dR = None if R is None else [torch.from_numpy(a).cuda().to(tdt) for a in R]
        ctx = qk.Context(lay, prm, prec)
        ref = ctx.conserved_sums(dU, dR)
        ctx.close()
        got = _noalloc(qk, fn, lay, prm, prec, dU, dR, stream)
        np.testing.assert_array_equal(got, ref)
        # a warm call allocates nothing: free device memory and the caching
        # allocator's counters stay where they were
        before = _memory(torch)
        again = _noalloc(qk, fn, lay, prm, prec, dU, dR, stream)
        after = _memory(torch)
        assert after == before, (before, after)
        np.testing.assert_array_equal(again, ref)


def test_noalloc_sums_at_the_patch_limit(env):
    """Exactly QK_NOALLOC_MAX_BOXES = 4096 patches (16^3 boxes of 4^3 cells in a
    64^3 periodic domain): the largest patch-table copy, table build and
    prefix the static layout holds."""
    torch, qk, fn = env
    lo = [[4 * i, 4 * j, 4 * k] for k in range(16) for j in range(16) for i in range(16)]
    lay = I.make_layout(lo, [[4, 4, 4]] * 4096, (64, 64, 64), 3)
    assert lay.nbox == 4096
    U, R, prm = _state(lay, 31, True)
    dU = [torch.from_numpy(a).cuda() for a in U]
    dR = [torch.from_numpy(a).cuda() for a in R]
    ctx = qk.Context(lay, prm, qk.FP64)
    ref = ctx.conserved_sums(dU, dR)
    ctx.close()
    stream = torch.cuda.current_stream().cuda_stream
    got = _noalloc(qk, fn, lay, prm, qk.FP64, dU, dR, stream)
    np.testing.assert_array_equal(got, ref)


def test_noalloc_rejects_too_many_patches(env):
    torch, qk, fn = env
    lay = I.single_box(4, 4, 4)
    dU = [torch.zeros(lay.field_len, dtype=torch.float64, device="cuda") for _ in range(5)]
    n = 4097
    boxes = (qk.Box * n)()
    for b in range(n):
        for d in range(3):
            boxes[b].n[d] = 1
    out = (C.c_double * qk.NSUMS)()
    err = C.create_string_buffer(256)
    params = qk.make_params(hydro_only=1, dx=0.25)
    rc = fn(C.byref(params), boxes, n, 4, qk.FP64, lay.field_len, _ptrs(dU), None, out, None,
            err, 256)
    assert rc == qk.EINVAL and b"4096" in err.value


def test_noalloc_rejects_a_patch_beyond_the_field_length(env):
    """A patch table that does not fit the field arrays is refused before any
    launch (the sums kernel would read past the caller's arrays)."""
    torch, qk, fn = env
    lay = I.single_box(4, 4, 4)
    dU = [torch.zeros(lay.field_len, dtype=torch.float64, device="cuda") for _ in range(5)]
    boxes = _boxes(qk, lay)
    out = (C.c_double * qk.NSUMS)()
    err = C.create_string_buffer(256)
    params = qk.make_params(hydro_only=1, dx=0.25)
    rc = fn(C.byref(params), boxes, 1, 4, qk.FP64, lay.field_len - 1, _ptrs(dU), None, out,
            None, err, 256)
    assert rc == qk.EINVAL and b"field_len" in err.value
    boxes[0].offset = 1
    rc = fn(C.byref(params), boxes, 1, 4, qk.FP64, lay.field_len, _ptrs(dU), None, out, None,
            err, 256)
    assert rc == qk.EINVAL
