"""Python binding of libqk (include/qk.h): argument marshalling only.

Every computation runs in the CUDA kernels of ``libqk.so``; this module turns
torch CUDA tensors into device pointers and the current torch stream into a
cudaStream_t.  It never computes a step itself and has no CPU path: if the
library is missing it raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# QK_FMAD=0 selects the diagnostic build without FMA contraction
# (build.build(fmad=False)); the default is the production library.
LIB_PATH = os.path.join(_HERE, "_build" if os.environ.get("QK_FMAD", "1") != "0"
                        else "_build_nofmad", "libqk.so")

OK, EINVAL, ECUDA, ENOCONV, ENEGATIVE = 0, 1, 2, 3, 4
FP64, FP32_MIXED = 0, 1
LAUNCH_BATCHED, LAUNCH_PER_PATCH = 0, 1
LO_F32, LO_I16 = 1, 2
NSUMS = 13
_lib = None


class QKError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"qk error {code}: {msg}")
        self.code = code


class Params(C.Structure):
    """Mirror of qk_params."""
    _fields_ = [
        ("gamma", C.c_double), ("cfl", C.c_double), ("a_r", C.c_double),
        ("c", C.c_double), ("chat", C.c_double), ("c_v", C.c_double),
        ("kappa_P", C.c_double), ("kappa_R", C.c_double), ("alpha_eos", C.c_double),
        ("eps_newton", C.c_double), ("dx", C.c_double * 3),
        ("kappa_mode", C.c_int32), ("eos", C.c_int32), ("max_iter", C.c_int32),
        ("nsub_max", C.c_int32), ("tau_correction", C.c_int32), ("hydro_only", C.c_int32),
        ("recon", C.c_int32), ("flattening", C.c_int32), ("closure", C.c_int32),
        ("bc_lo", C.c_int32 * 3), ("bc_hi", C.c_int32 * 3),
    ]


CLOSURE_LEVERMORE, CLOSURE_MINERBO, CLOSURE_EDDINGTON = 0, 1, 2
PART_ALL, PART_INTERIOR, PART_BOUNDARY = 0, 1, 2
BC_PERIODIC, BC_REFLECT, BC_OUTFLOW, BC_DIRICHLET = 0, 1, 2, 3


class Box(C.Structure):
    """Mirror of qk_box."""
    _fields_ = [("lo", C.c_int32 * 3), ("n", C.c_int32 * 3), ("offset", C.c_int64)]


def lib():
    """Load libqk.so (built by ``paper_2110_01792_gb300.build``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libqk.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    P = C.POINTER
    L.qk_init_patches.argtypes = [P(vp), P(Params), P(Box), i32, P(i32), i32, i32]
    L.qk_init_patches.restype = C.c_int
    L.qk_destroy.argtypes = [vp]
    L.qk_destroy.restype = None
    L.qk_last_error.argtypes = [vp]
    L.qk_last_error.restype = C.c_char_p
    L.qk_field_len.argtypes = [vp]
    L.qk_field_len.restype = i64
    L.qk_num_cells.argtypes = [vp]
    L.qk_num_cells.restype = i64
    L.qk_set_params.argtypes = [vp, P(Params)]
    L.qk_set_graph.argtypes = [vp, i32]
    L.qk_set_launch_mode.argtypes = [vp, i32]
    L.qk_set_fused_exchange.argtypes = [vp, i32]
    L.qk_set_launch_config.argtypes = [vp, P(i32)]
    L.qk_rad_stage2_exchange.argtypes = [vp, P(vp), P(vp), P(vp), P(vp), dbl, vp]
    L.qk_autotune.argtypes = [vp, P(vp), P(vp), P(i32), vp]
    L.qk_fill_ghosts.argtypes = [vp, P(vp), i32, vp]
    L.qk_hydro_stage.argtypes = [vp, i32, P(vp), P(vp), P(vp), dbl, vp]
    L.qk_rad_stage.argtypes = [vp, i32, P(vp), P(vp), P(vp), vp, dbl, vp]
    L.qk_rad_matter_exchange.argtypes = [vp, P(vp), P(vp), dbl, vp]
    L.qk_timestep.argtypes = [vp, P(vp), P(dbl), vp]
    L.qk_step.argtypes = [vp, P(vp), P(vp), P(dbl), P(i32), vp]
    L.qk_conserved_sums.argtypes = [vp, P(vp), P(vp), P(dbl), vp]
    L.qk_step_info.argtypes = [vp, P(dbl), vp]
    L.qk_status.argtypes = [vp, P(C.c_uint32), P(i64), P(i32), i32, vp]
    L.qk_init_shard.argtypes = [P(vp), P(Params), P(Box), i32, P(i32), i32, i32, P(i32), i32, i32]
    L.qk_halo_info.argtypes = [vp, i32, P(i64), P(i64), P(i32)]
    L.qk_halo_pack.argtypes = [vp, i32, P(vp), i32, i32, vp, vp]
    L.qk_halo_unpack.argtypes = [vp, i32, P(vp), i32, i32, vp, vp]
    L.qk_fill_ghosts_range.argtypes = [vp, P(vp), i32, i32, vp]
    L.qk_fill_plan.argtypes = [P(Params), P(Box), i32, P(i32), i32, P(i64), i64, P(i64), P(i64)]
    L.qk_set_dirichlet.argtypes = [vp, P(vp), P(vp), vp]
    L.qk_set_source.argtypes = [vp, vp]
    L.qk_set_tile_part.argtypes = [vp, i32]
    L.qk_init_level.argtypes = [P(vp), P(Params), P(Box), i32, P(i32), i32, i32]
    L.qk_amr_init.argtypes = [P(vp), vp, vp]
    L.qk_amr_destroy.argtypes = [vp]
    L.qk_amr_destroy.restype = None
    L.qk_amr_last_error.argtypes = [vp]
    L.qk_amr_last_error.restype = C.c_char_p
    L.qk_amr_info.argtypes = [vp, P(i64), P(i64), P(i64)]
    L.qk_amr_interp.argtypes = [vp, P(vp), P(vp), dbl, P(vp), i32, i32, vp]
    L.qk_amr_register.argtypes = [vp, i32, i32, P(vp), vp, dbl, vp]
    L.qk_amr_sync.argtypes = [vp, P(vp), P(vp), P(vp), P(vp), vp]
    L.qk_tile_counts.argtypes = [vp, P(i32), P(i32)]
    L.qk_signal_speed.argtypes = [vp, P(vp), P(dbl), vp]
    L.qk_set_timestep.argtypes = [vp, dbl, P(dbl), vp]
    L.qk_eval_math.argtypes = [vp, i64, vp, vp, vp]
    L.qk_eval_convert.argtypes = [vp, vp, vp, vp, i64, vp]
    L.qk_fma_probe.argtypes = [i32, i64, vp, i64, P(dbl), vp]
    L.qk_step_compensated.argtypes = [vp, P(vp), P(vp), P(vp), P(vp), P(dbl), P(i32), vp]
    L.qk_step_host.argtypes = [vp, P(vp), P(vp), P(dbl), P(i32), vp]
    L.qk_conserved_sums_compensated.argtypes = [vp, P(vp), P(vp), P(vp), P(vp), P(dbl), vp]
    L.qk_set_lo_format.argtypes = [vp, i32]
    for f in ("qk_init_level", "qk_amr_init", "qk_amr_info", "qk_amr_interp", "qk_amr_register",
              "qk_amr_sync", "qk_set_tile_part", "qk_tile_counts", "qk_fill_plan", "qk_fill_ghosts_range", "qk_set_dirichlet", "qk_set_source",
              "qk_init_shard", "qk_halo_info", "qk_halo_pack", "qk_halo_unpack",
              "qk_signal_speed", "qk_set_timestep", "qk_set_params", "qk_set_graph", "qk_set_launch_mode", "qk_set_fused_exchange", "qk_rad_stage2_exchange", "qk_set_launch_config", "qk_autotune",
              "qk_fill_ghosts", "qk_hydro_stage", "qk_rad_stage",
              "qk_rad_matter_exchange", "qk_timestep", "qk_step", "qk_conserved_sums",
              "qk_status", "qk_step_info", "qk_eval_math", "qk_eval_convert", "qk_fma_probe",
              "qk_step_compensated", "qk_step_host",
              "qk_conserved_sums_compensated", "qk_set_lo_format"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


def eval_math(x, rcp=None, sqrt_out=None, stream=None):
    """The library's FP64 reciprocal and square root of the device doubles `x`
    into the device arrays `rcp` / `sqrt_out` (either may be None)."""
    rc = lib().qk_eval_math(C.c_void_p(int(x.data_ptr())), int(x.numel()),
                            C.c_void_p(int(rcp.data_ptr())) if rcp is not None else None,
                            C.c_void_p(int(sqrt_out.data_ptr())) if sqrt_out is not None else None,
                            _stream(stream))
    if rc != OK:
        raise QKError(rc, "qk_eval_math failed")


def lo16_encode(hi, lo):
    """Host form of the 16-bit low parts (LO_I16): for float32 hi and the
    residual lo (|lo| <= ulp(hi)/2), k = rint(lo 2^(38 - E)) as int16, E the
    binary exponent of hi (zero where lo or hi is zero or below the normal
    float range)."""
    hi = np.asarray(hi, dtype=np.float32)
    lo = np.asarray(lo, dtype=np.float64)
    _, e = np.frexp(hi)
    E = e.astype(np.int64) - 1
    k = np.rint(np.ldexp(lo, (38 - E).astype(np.int32)))
    k = np.where((np.abs(lo) < 2.0 ** -126) | (hi == 0), 0.0, k)
    return np.clip(k, -32767, 32767).astype(np.int16)


def lo16_decode(hi, k):
    """The low parts held by LO_I16 arrays: lo = k 2^(E - 38) (float64)."""
    hi = np.asarray(hi, dtype=np.float32)
    _, e = np.frexp(hi)
    E = e.astype(np.int64) - 1
    return np.ldexp(np.asarray(k, dtype=np.float64), (E - 38).astype(np.int32))


_CFG_NAMES = ("hydro1", "hydro2", "rad1", "rad2")


def _decode_cfg(vals):
    """threads | schedule << 16 | shape << 17 -> {kernel: (threads, schedule)},
    schedule "strided" / "contiguous" on 8^3 tiles, or "columns" / "columns2"
    (16 x 16 columns; "columns2": registers held to two CTAs per SM)."""
    out = {}
    for n, v in zip(_CFG_NAMES, vals):
        v = int(v)
        if (v >> 17) & 1:
            sched = "columns2" if (v >> 16) & 1 else "columns"
        else:
            sched = "contiguous" if (v >> 16) & 1 else "strided"
        out[n] = (v & 0xffff, sched)
    return out


def _encode_cfg(c):
    th, sched = c
    return int(th) | ({"strided": 0, "contiguous": 1 << 16, "columns": 1 << 17,
                       "columns2": 3 << 16}[sched])


def eval_convert(f_in=None, d_out=None, d_in=None, f_out=None, stream=None):
    """The library's float -> double widening of `f_in` into `d_out` and
    double -> float truncation of `d_in` into `f_out` (device tensors)."""
    n = int((f_in if f_in is not None else d_in).numel())
    ptr = lambda t: C.c_void_p(int(t.data_ptr())) if t is not None else None
    rc = lib().qk_eval_convert(ptr(f_in), ptr(d_out), ptr(d_in), ptr(f_out), n, _stream(stream))
    if rc != OK:
        raise QKError(rc, "qk_eval_convert failed")


def fma_probe(fp64: bool, iters: int, sink, stream=None) -> float:
    """Launch the library's FMA throughput probe on `stream` (the caller times
    it); `sink` is a device tensor of at least 256 doubles / floats.  Returns
    the launch's flop count."""
    fl = C.c_double(0.0)
    rc = lib().qk_fma_probe(1 if fp64 else 0, int(iters), C.c_void_p(int(sink.data_ptr())),
                            int(sink.numel()), C.byref(fl), _stream(stream))
    if rc != OK:
        raise QKError(rc, "qk_fma_probe failed")
    return fl.value


def make_params(**kw) -> Params:
    p = Params()
    p.gamma = kw.get("gamma", 5.0 / 3.0)
    p.cfl = kw.get("cfl", 0.3)
    p.a_r = kw.get("a_r", 1.0)
    p.c = kw.get("c", 100.0)
    p.chat = kw.get("chat", 10.0)
    p.c_v = kw["c_v"] if "c_v" in kw else (1.0 / (p.gamma - 1.0) if p.gamma != 1.0 else 0.0)
    p.kappa_P = kw.get("kappa_P", 1.0)
    p.kappa_R = kw.get("kappa_R", 1.0)
    p.alpha_eos = kw.get("alpha_eos", 0.0)
    p.eps_newton = kw.get("eps_newton", 1e-10)
    dx = kw.get("dx", (1.0, 1.0, 1.0))
    if np.isscalar(dx):
        dx = (dx, dx, dx)
    for i in range(3):
        p.dx[i] = float(dx[i])
    p.kappa_mode = int(kw.get("kappa_mode", 0))
    p.eos = int(kw.get("eos", 0))
    p.max_iter = int(kw.get("max_iter", 400))
    p.nsub_max = int(kw.get("nsub_max", 10))
    p.tau_correction = int(kw.get("tau_correction", 1))
    p.hydro_only = int(kw.get("hydro_only", 0))
    p.recon = int(kw.get("recon", 0))
    p.flattening = int(kw.get("flattening", 0))
    p.closure = int(kw.get("closure", 0))
    lo = kw.get("bc_lo", (0, 0, 0))
    hi = kw.get("bc_hi", (0, 0, 0))
    for i in range(3):
        p.bc_lo[i] = int(lo[i])
        p.bc_hi[i] = int(hi[i])
    return p


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptrs(fields, n):
    if fields is None:
        return None
    assert len(fields) == n, f"expected {n} fields"
    return (C.c_void_p * n)(*[int(f.data_ptr()) for f in fields])


def _boxes(layout):
    nb = layout.nbox
    boxes = (Box * nb)()
    for b in range(nb):
        for d in range(3):
            boxes[b].lo[d] = int(layout.lo[b][d])
            boxes[b].n[d] = int(layout.n[b][d])
        boxes[b].offset = int(layout.off[b])
    return boxes


def fill_plan(layout, params: dict):
    """The ghost-fill descriptors of a patch set (host only, no GPU): an
    (ncopies, 11) int64 array of copies (dst, src, ex, ey, ez, dsx, dsy, flip,
    sx, sy, sz) and an (nregions, 7) array of Dirichlet regions (dst, -, ex,
    ey, ez, dsx, dsy)."""
    L = lib()
    prm = make_params(**params)
    dom = (C.c_int32 * 3)(*[int(v) for v in layout.dom_n])
    nc, nd = C.c_int64(), C.c_int64()
    rc = L.qk_fill_plan(C.byref(prm), _boxes(layout), layout.nbox, dom, int(layout.ng), None, 0,
                        C.byref(nc), C.byref(nd))
    if rc != OK:
        raise QKError(rc, L.qk_last_error(None).decode())
    out = np.zeros((nc.value + nd.value, 12), dtype=np.int64)
    rc = L.qk_fill_plan(C.byref(prm), _boxes(layout), layout.nbox, dom, int(layout.ng),
                        out.ctypes.data_as(C.POINTER(C.c_int64)), len(out), C.byref(nc),
                        C.byref(nd))
    if rc != OK:
        raise QKError(rc, L.qk_last_error(None).decode())
    return out[out[:, 11] == 0, :11], out[out[:, 11] == 1, :7]


class Context:
    """A patch set on the current CUDA device (wraps qk_init_patches).

    With ``owner`` (owner rank of every patch) and ``rank``, the context is
    this rank's shard of the patch set (qk_init_shard): ``layout`` then holds
    the whole patch set with this rank's patches placed in its own field
    arrays (see ``shard.rank_layout``)."""

    def __init__(self, layout, params: dict, precision: int = FP64, owner=None, rank: int = 0,
                 level: bool = False):
        self._L = lib()
        nb = layout.nbox
        boxes = _boxes(layout)
        dom = (C.c_int32 * 3)(*[int(v) for v in layout.dom_n])
        self.params = make_params(**params)
        self.precision = precision
        self.layout = layout
        h = C.c_void_p()
        self.rank, self.nranks = 0, 1
        if level:
            rc = self._L.qk_init_level(C.byref(h), C.byref(self.params), boxes, nb, dom,
                                       int(layout.ng), int(precision))
        elif owner is None:
            rc = self._L.qk_init_patches(C.byref(h), C.byref(self.params), boxes, nb, dom,
                                         int(layout.ng), int(precision))
        else:
            own = np.ascontiguousarray(owner, dtype=np.int32)
            assert own.shape == (nb,)
            self.rank, self.nranks = int(rank), int(own.max()) + 1
            rc = self._L.qk_init_shard(C.byref(h), C.byref(self.params), boxes, nb, dom,
                                       int(layout.ng), int(precision),
                                       own.ctypes.data_as(C.POINTER(C.c_int32)),
                                       self.nranks, self.rank)
        if rc != OK:
            raise QKError(rc, self._L.qk_last_error(None).decode())
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._L.qk_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != OK:
            raise QKError(rc, self._L.qk_last_error(self._h).decode())

    @property
    def field_len(self):
        return int(self._L.qk_field_len(self._h))

    @property
    def num_cells(self):
        return int(self._L.qk_num_cells(self._h))

    def set_params(self, **kw):
        self.params = make_params(**kw)
        self._check(self._L.qk_set_params(self._h, C.byref(self.params)))

    def set_launch_mode(self, per_patch: bool):
        """Batched (one launch per stage over all patches) or one launch per patch."""
        self._check(self._L.qk_set_launch_mode(self._h, 1 if per_patch else 0))

    def autotune(self, U, R=None, stream=None):
        """Pick the fastest launch configuration of each stage kernel on this
        state; returns {kernel: (threads per CTA, schedule)}."""
        out = (C.c_int32 * 4)()
        self._check(self._L.qk_autotune(self._h, _ptrs(U, 5), _ptrs(R, 4) if R is not None else None,
                                        out, _stream(stream)))
        return _decode_cfg(out[:])

    def set_launch_config(self, cfg):
        """Set the four stage kernels' launch configurations, given as
        {kernel: (threads, schedule)} like autotune's result."""
        arr = (C.c_int32 * 4)(*[_encode_cfg(cfg[n]) for n in _CFG_NAMES])
        self._check(self._L.qk_set_launch_config(self._h, arr))

    def set_lo_format(self, fmt: int):
        """Storage of the low parts of compensated states: LO_F32 (float
        arrays) or LO_I16 (int16 arrays, ~39-bit values in 6 bytes)."""
        self._check(self._L.qk_set_lo_format(self._h, int(fmt)))

    def set_fused_exchange(self, enable: bool):
        self._check(self._L.qk_set_fused_exchange(self._h, 1 if enable else 0))

    def set_graph(self, enable: bool):
        self._check(self._L.qk_set_graph(self._h, 1 if enable else 0))

    def fill_ghosts(self, fields, first=0, stream=None):
        """Ghost fill of fields holding state fields first, first+1, ... of
        (rho, m_x, m_y, m_z, E, E_r, F_x, F_y, F_z)."""
        self._check(self._L.qk_fill_ghosts_range(self._h, _ptrs(fields, len(fields)), int(first),
                                                 len(fields), _stream(stream)))

    def set_dirichlet(self, U, R=None, stream=None):
        """Record the states the ghost cells beyond Dirichlet faces hold now."""
        self._check(self._L.qk_set_dirichlet(self._h, _ptrs(U, 5),
                                             _ptrs(R, 4) if R is not None else None,
                                             _stream(stream)))

    def set_source(self, j):
        """Emissivity field of the exchange (a tensor kept alive by the caller), or None."""
        self._source = j
        self._check(self._L.qk_set_source(self._h, C.c_void_p(int(j.data_ptr())) if j is not None
                                          else None))

    def hydro_stage(self, stage, U0, U1, Uout, dt, stream=None):
        self._check(self._L.qk_hydro_stage(self._h, stage, _ptrs(U0, 5), _ptrs(U1, 5),
                                           _ptrs(Uout, 5), float(dt), _stream(stream)))

    def rad_stage(self, stage, R0, R1, Rout, rho, dt, stream=None):
        self._check(self._L.qk_rad_stage(self._h, stage, _ptrs(R0, 4), _ptrs(R1, 4),
                                         _ptrs(Rout, 4), C.c_void_p(int(rho.data_ptr())),
                                         float(dt), _stream(stream)))

    def rad_stage2_exchange(self, R0, R1, Rout, U, dt, stream=None):
        """Radiation stage 2 with the exchange fused into its epilogue."""
        self._check(self._L.qk_rad_stage2_exchange(self._h, _ptrs(R0, 4), _ptrs(R1, 4),
                                                   _ptrs(Rout, 4), _ptrs(U, 5), float(dt),
                                                   _stream(stream)))

    def exchange(self, U, R, dt, stream=None):
        self._check(self._L.qk_rad_matter_exchange(self._h, _ptrs(U, 5), _ptrs(R, 4), float(dt),
                                                   _stream(stream)))

    def timestep(self, U, stream=None):
        out = (C.c_double * 4)()
        self._check(self._L.qk_timestep(self._h, _ptrs(U, 5), out, _stream(stream)))
        return out[0], int(out[1]), out[2], out[3]

    def step(self, U, R=None, want_dt=False, stream=None, lo=None):
        """One full update.  `lo` = (U_lo, R_lo) selects the compensated FP32
        step (qk_step_compensated): the state is U + U_lo, R + R_lo."""
        dt = C.c_double(0.0)
        ns = C.c_int32(0)
        rp = _ptrs(R, 4) if R is not None else None
        if lo is None:
            rc = self._L.qk_step(self._h, _ptrs(U, 5), rp, C.byref(dt) if want_dt else None,
                                 C.byref(ns) if want_dt else None, _stream(stream))
        else:
            Ul, Rl = lo
            rc = self._L.qk_step_compensated(
                self._h, _ptrs(U, 5), rp, _ptrs(Ul, 5), _ptrs(Rl, 4) if R is not None else None,
                C.byref(dt) if want_dt else None, C.byref(ns) if want_dt else None,
                _stream(stream))
        self._check(rc)
        return (dt.value, ns.value) if want_dt else None

    def step_host(self, U, R=None, want_dt=False, stream=None):
        """One full update of a state held in host memory (qk_step_host): U,
        R are CPU tensors (pinned for full copy speed) or numpy arrays of the
        context's precision, updated in place; returns after the copy back."""
        def hp(fields, n):
            assert len(fields) == n, f"expected {n} fields"
            out = (C.c_void_p * n)()
            for i, f in enumerate(fields):
                out[i] = f.ctypes.data if isinstance(f, np.ndarray) else int(f.data_ptr())
            return out
        dt = C.c_double(0.0)
        ns = C.c_int32(0)
        rc = self._L.qk_step_host(self._h, hp(U, 5), hp(R, 4) if R is not None else None,
                                  C.byref(dt) if want_dt else None,
                                  C.byref(ns) if want_dt else None, _stream(stream))
        self._check(rc)
        return (dt.value, ns.value) if want_dt else None

    def step_info(self, stream=None):
        """(dt, N_sub, dt_rad, smax) of the last timestep, total substeps, total steps."""
        out = (C.c_double * 6)()
        self._check(self._L.qk_step_info(self._h, out, _stream(stream)))
        return tuple(out[:])

    def conserved_sums(self, U, R=None, stream=None, lo=None):
        """qk_conserved_sums; `lo` = (U_lo, R_lo) sums a compensated state."""
        out = (C.c_double * NSUMS)()
        rp = _ptrs(R, 4) if R is not None else None
        if lo is None:
            rc = self._L.qk_conserved_sums(self._h, _ptrs(U, 5), rp, out, _stream(stream))
        else:
            Ul, Rl = lo
            rc = self._L.qk_conserved_sums_compensated(
                self._h, _ptrs(U, 5), rp, _ptrs(Ul, 5), _ptrs(Rl, 4) if R is not None else None,
                out, _stream(stream))
        self._check(rc)
        return np.array(out[:])

    def status(self, reset=False, stream=None):
        fl = C.c_uint32()
        fb = C.c_int64()
        mi = C.c_int32()
        rc = self._L.qk_status(self._h, C.byref(fl), C.byref(fb), C.byref(mi), 1 if reset else 0,
                               _stream(stream))
        return rc, int(fl.value), int(fb.value), int(mi.value)

    # ---- sharded contexts (one rank of a multi-GPU run) ----
    def halo_cells(self, peer):
        """(cells per field sent to peer, cells per field received from peer)."""
        s, r = C.c_int64(), C.c_int64()
        self._check(self._L.qk_halo_info(self._h, int(peer), C.byref(s), C.byref(r), None))
        return int(s.value), int(r.value)

    def halo_pack(self, peer, fields, buf, first=0, stream=None):
        self._check(self._L.qk_halo_pack(self._h, int(peer), _ptrs(fields, len(fields)),
                                         int(first), len(fields),
                                         C.c_void_p(int(buf.data_ptr())), _stream(stream)))

    def halo_unpack(self, peer, fields, buf, first=0, stream=None):
        self._check(self._L.qk_halo_unpack(self._h, int(peer), _ptrs(fields, len(fields)),
                                           int(first), len(fields),
                                           C.c_void_p(int(buf.data_ptr())), _stream(stream)))

    def signal_speed(self, U, stream=None):
        """max(|v| + c_s) over this context's cells."""
        out = C.c_double(0.0)
        self._check(self._L.qk_signal_speed(self._h, _ptrs(U, 5), C.byref(out), _stream(stream)))
        return out.value

    def set_timestep(self, smax, stream=None):
        """(dt, N_sub, dt_rad, smax) from the global signal speed."""
        out = (C.c_double * 4)()
        self._check(self._L.qk_set_timestep(self._h, float(smax), out, _stream(stream)))
        return out[0], int(out[1]), out[2], out[3]

    def set_tile_part(self, part):
        """Tiles processed by later stage calls: PART_ALL, PART_INTERIOR or PART_BOUNDARY."""
        self._check(self._L.qk_set_tile_part(self._h, int(part)))

    def tile_counts(self):
        """(interior tiles, boundary tiles) of this context."""
        i, b = C.c_int32(), C.c_int32()
        self._check(self._L.qk_tile_counts(self._h, C.byref(i), C.byref(b)))
        return int(i.value), int(b.value)


def _ptrs9(fields):
    arr = (C.c_void_p * 9)()
    for i, f in enumerate(fields):
        arr[i] = int(f.data_ptr()) if f is not None else None
    return arr


class Amr:
    """Two refinement levels (wraps qk_amr_init): `coarse` covers the domain,
    `fine` (a Context made with level=True) refines part of it by 2."""

    def __init__(self, coarse: Context, fine: Context):
        self._L = lib()
        self.coarse, self.fine = coarse, fine
        h = C.c_void_p()
        rc = self._L.qk_amr_init(C.byref(h), coarse._h, fine._h)
        if rc != OK:
            raise QKError(rc, self._L.qk_amr_last_error(None).decode())
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._L.qk_amr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != OK:
            raise QKError(rc, self._L.qk_amr_last_error(self._h).decode())

    def info(self):
        """(fine ghost cells interpolated, coarse-fine faces, coarse cells under the fine region)."""
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        self._check(self._L.qk_amr_info(self._h, C.byref(a), C.byref(b), C.byref(c)))
        return int(a.value), int(b.value), int(c.value)

    def interp(self, c_old, c_new, alpha, fine_fields, first, stream=None):
        self._check(self._L.qk_amr_interp(self._h, _ptrs9(c_old), _ptrs9(c_new), float(alpha),
                                          _ptrs(fine_fields, len(fine_fields)), int(first),
                                          len(fine_fields), _stream(stream)))

    def register(self, level, kind, fields, rho, weight, stream=None):
        self._check(self._L.qk_amr_register(self._h, int(level), int(kind),
                                            _ptrs(fields, len(fields)),
                                            C.c_void_p(int(rho.data_ptr())) if rho is not None
                                            else None, float(weight), _stream(stream)))

    def sync(self, cU, cR, fU, fR, stream=None):
        self._check(self._L.qk_amr_sync(self._h, _ptrs(cU, 5), _ptrs(cR, 4) if cR is not None
                                        else None, _ptrs(fU, 5),
                                        _ptrs(fR, 4) if fR is not None else None,
                                        _stream(stream)))
