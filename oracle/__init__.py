"""FP64 CPU oracle for the per-cell uniform-patch RHD update (arXiv:2110.01792).

TEST INFRASTRUCTURE ONLY: this package is the parity reference and the timed
CPU baseline.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.  It
shares no code with the CUDA library and the CUDA library never calls it.

The arithmetic lives in ``qk_oracle.c`` (plain C, compiled with
``-ffp-contract=off`` so that x86-64 and aarch64 hosts give identical bits);
this module only builds it, loads it with ``ctypes`` and marshals numpy arrays.

Parity status per function (the pins live in ``tests/test_oracle_*.py``):
  hydro stage, PPM, HLLC, RK2, timestep ... pinned (contact, uniform state,
      exact Riemann, sound-wave order and the paper's printed errors,
      conservation, x<->y symmetry, direction invariance)
  Levermore closure ........................ pinned (chi limits, trace, streaming)
  radiation stage .......................... pinned (free-streaming translation
      and order, diffusion-limit Gaussian, conservation)
  exchange ................................. pinned (closed form eq.
      rsla_temperature, T_eq ratio, invariants, bisection)
  parity unpinned: the readings the paper leaves open (MC slope in the
      extremum branch, radiation wavespeed, optical-depth correction form,
      Newton stopping rule) are pinned only as far as the pins above reach.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

NHYD, NRAD, NSUMS = 5, 4, 13
OK, EINVAL, ENOCONV, ENEGATIVE = 0, 1, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (with OpenMP for
    the host-thread cell loops where the compiler has it, else serial)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
        if r.returncode != 0:
            subprocess.run(base, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def set_threads(n: int) -> int:
    """Host threads of the oracle's cell loops (z-planes over OpenMP threads;
    results are bit-identical to one thread).  Returns the number in effect:
    1 when the oracle was built without OpenMP."""
    return int(lib().or_set_threads(int(n)))


class Params(C.Structure):
    """Mirror of ``or_params`` in qk_oracle.c (physical and numerical constants)."""
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


BC_PERIODIC, BC_REFLECT, BC_OUTFLOW, BC_DIRICHLET = 0, 1, 2, 3
CLOSURE_LEVERMORE, CLOSURE_MINERBO, CLOSURE_EDDINGTON = 0, 1, 2


def make_params(**kw) -> Params:
    """Build oracle parameters from a dict using the library's parameter names."""
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


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.POINTER
            vp = C.c_void_p
            L.or_grid_create.restype = vp
            L.or_grid_create.argtypes = [C.c_int32, P(C.c_int32), P(C.c_int32), P(C.c_int64),
                                         P(C.c_int32), C.c_int32]
            L.or_grid_destroy.argtypes = [vp]
            L.or_fill_ghosts.argtypes = [vp, vp]
            L.or_ppm_cell.argtypes = [P(C.c_double), P(C.c_double), P(C.c_double)]
            L.or_plm_cell.argtypes = [P(C.c_double), P(C.c_double), P(C.c_double)]
            L.or_hllc.argtypes = [P(C.c_double), P(C.c_double), C.c_int, C.c_double, P(C.c_double)]
            L.or_hydro_stage.argtypes = [vp, P(Params), C.c_int, vp, vp, vp, C.c_double,
                                         C.c_int64, vp]
            L.or_rad_stage.argtypes = [vp, P(Params), C.c_int, vp, vp, vp, vp, C.c_double,
                                       C.c_int64, vp]
            L.or_max_signal_speed.restype = C.c_double
            L.or_max_signal_speed.argtypes = [vp, P(Params), vp]
            L.or_timestep.argtypes = [vp, P(Params), vp, P(C.c_double)]
            L.or_timestep_from_speed.argtypes = [P(Params), C.c_double, P(C.c_double)]
            L.or_eddington_tensor.argtypes = [C.c_int, P(C.c_double), P(C.c_double)]
            L.or_eddington_factor.restype = C.c_double
            L.or_eddington_factor.argtypes = [C.c_int, C.c_double]
            L.or_exchange_energy_src.restype = C.c_int
            L.or_exchange_energy_src.argtypes = [P(Params), C.c_double, C.c_double, C.c_double,
                                                 C.c_double, C.c_double, P(C.c_double),
                                                 P(C.c_double)]
            L.or_hydro_face_flux.argtypes = [vp, P(Params), vp, C.c_int32, P(C.c_int32),
                                             C.c_int32, P(C.c_double)]
            L.or_rad_face_flux.argtypes = [vp, P(Params), vp, vp, C.c_int32, P(C.c_int32),
                                           C.c_int32, P(C.c_double)]
            L.or_set_dirichlet.restype = C.c_int
            L.or_set_dirichlet.argtypes = [vp, P(Params), vp]
            L.or_fill_ghosts_bc.restype = C.c_int
            L.or_fill_ghosts_bc.argtypes = [vp, P(Params), vp, C.c_int, C.c_int]
            L.or_exchange_energy.restype = C.c_int
            L.or_exchange_energy.argtypes = [P(Params), C.c_double, C.c_double, C.c_double,
                                             C.c_double, P(C.c_double), P(C.c_double)]
            L.or_exchange.argtypes = [vp, P(Params), vp, vp, C.c_double, C.c_int64, vp,
                                      vp, P(C.c_int64)]
            L.or_relax_cell.argtypes = [P(Params), C.c_double, C.c_double, C.c_double,
                                        C.c_double, C.c_int64, vp, vp]
            L.or_step.argtypes = [vp, P(Params), vp, vp, vp, vp, P(C.c_double), P(C.c_int64)]
            L.or_conserved_sums.argtypes = [vp, P(Params), vp, vp, P(C.c_double)]
            L.or_set_threads.restype = C.c_int
            L.or_set_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def _dptr(a: np.ndarray) -> int:
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data


def _ptr_array(fields):
    arr = (C.c_void_p * len(fields))(*[_dptr(f) for f in fields])
    return arr


class Grid:
    """A set of patches tiling a periodic domain, with the SoA field layout
    (patch b at element ``off[b]``, (n+2g)^3 cells, x fastest)."""

    def __init__(self, lo, n, off, dom_n, ng):
        self.lo = np.ascontiguousarray(lo, dtype=np.int32).reshape(-1, 3)
        self.n = np.ascontiguousarray(n, dtype=np.int32).reshape(-1, 3)
        self.off = np.ascontiguousarray(off, dtype=np.int64).reshape(-1)
        self.dom_n = np.ascontiguousarray(dom_n, dtype=np.int32).reshape(3)
        self.ng = int(ng)
        L = lib()
        P = C.POINTER
        self._h = L.or_grid_create(len(self.off), self.lo.ctypes.data_as(P(C.c_int32)),
                                   self.n.ctypes.data_as(P(C.c_int32)),
                                   self.off.ctypes.data_as(P(C.c_int64)),
                                   self.dom_n.ctypes.data_as(P(C.c_int32)), self.ng)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().or_grid_destroy(h)
            self._h = None

    @property
    def handle(self):
        return self._h


def _cells_arg(cells):
    if cells is None:
        return 0, None, None
    c = np.ascontiguousarray(cells, dtype=np.int32).reshape(-1, 4)
    return len(c), c.ctypes.data, c


def fill_ghosts(grid: Grid, f: np.ndarray) -> None:
    lib().or_fill_ghosts(grid.handle, _dptr(f))


def ppm_cell(stencil):
    s = (C.c_double * 5)(*[float(x) for x in stencil])
    qL, qR = C.c_double(), C.c_double()
    lib().or_ppm_cell(s, C.byref(qL), C.byref(qR))
    return qL.value, qR.value


def plm_cell(stencil):
    s = (C.c_double * 5)(*[float(x) for x in stencil])
    qL, qR = C.c_double(), C.c_double()
    lib().or_plm_cell(s, C.byref(qL), C.byref(qR))
    return qL.value, qR.value


def hllc(wL, wR, d, gamma):
    a = (C.c_double * 5)(*[float(x) for x in wL])
    b = (C.c_double * 5)(*[float(x) for x in wR])
    F = (C.c_double * 5)()
    lib().or_hllc(a, b, int(d), float(gamma), F)
    return np.array(F[:])


def eddington_tensor(f, closure=0):
    a = (C.c_double * 3)(*[float(x) for x in f])
    T = (C.c_double * 9)()
    lib().or_eddington_tensor(int(closure), a, T)
    return np.array(T[:]).reshape(3, 3)


def eddington_factor(f, closure=0):
    return lib().or_eddington_factor(int(closure), float(f))


def hydro_face_flux(grid, p, U, b, c, d):
    """Hydro flux through the low face of patch b's cell c along axis d."""
    out = (C.c_double * NHYD)()
    cc = (C.c_int32 * 3)(*[int(v) for v in c])
    lib().or_hydro_face_flux(grid.handle, C.byref(p), _ptr_array(U), int(b), cc, int(d), out)
    return np.array(out[:])


def rad_face_flux(grid, p, R, rho, b, c, d):
    """Radiation flux through the low face of patch b's cell c along axis d."""
    out = (C.c_double * NRAD)()
    cc = (C.c_int32 * 3)(*[int(v) for v in c])
    lib().or_rad_face_flux(grid.handle, C.byref(p), _ptr_array(R), _dptr(rho), int(b), cc,
                           int(d), out)
    return np.array(out[:])


def set_dirichlet(grid, p, U, R):
    """Record the boundary states held in the ghost cells beyond Dirichlet faces
    (all 9 fields); returns the status (OR_EINVAL when two ghost cells of the
    same boundary position disagree)."""
    return lib().or_set_dirichlet(grid.handle, C.byref(p), _ptr_array(list(U) + list(R)))


def fill_ghosts_bc(grid, p, fields, fid0=0):
    """Ghost cells of fields (field ids fid0, fid0+1, ...) under the boundary conditions."""
    return lib().or_fill_ghosts_bc(grid.handle, C.byref(p), _ptr_array(fields), len(fields),
                                   int(fid0))


def hydro_stage(grid, p, stage, U0, U1, Uout, dt, cells=None):
    n, ptr, keep = _cells_arg(cells)
    lib().or_hydro_stage(grid.handle, C.byref(p), int(stage), _ptr_array(U0),
                         _ptr_array(U1) if U1 is not None else None, _ptr_array(Uout),
                         float(dt), n, ptr)


def rad_stage(grid, p, stage, R0, R1, Rout, rho, dt, cells=None):
    n, ptr, keep = _cells_arg(cells)
    lib().or_rad_stage(grid.handle, C.byref(p), int(stage), _ptr_array(R0),
                       _ptr_array(R1) if R1 is not None else None, _ptr_array(Rout),
                       _dptr(rho), float(dt), n, ptr)


def max_signal_speed(grid, p, U):
    return lib().or_max_signal_speed(grid.handle, C.byref(p), _ptr_array(U))


def timestep(grid, p, U):
    out = (C.c_double * 3)()
    lib().or_timestep(grid.handle, C.byref(p), _ptr_array(U), out)
    return out[0], int(out[1]), out[2]


def timestep_from_speed(p, smax):
    out = (C.c_double * 3)()
    lib().or_timestep_from_speed(C.byref(p), float(smax), out)
    return out[0], int(out[1]), out[2]


def exchange_energy(p, rho, Eg0, Er0, dt, S=0.0):
    Eg, Er = C.c_double(), C.c_double()
    it = lib().or_exchange_energy_src(C.byref(p), float(rho), float(Eg0), float(Er0), float(dt),
                                      float(S), C.byref(Eg), C.byref(Er))
    return Eg.value, Er.value, it


def exchange(grid, p, U, R, dt, cells=None, src=None):
    n, ptr, keep = _cells_arg(cells)
    info = (C.c_int64 * 4)()
    rc = lib().or_exchange(grid.handle, C.byref(p), _ptr_array(U), _ptr_array(R), float(dt),
                           n, ptr, _dptr(src) if src is not None else None, info)
    return rc, tuple(info[:])


def relax_cell(p, rho, Eg, Er, dt, nsteps):
    Egh = np.zeros(nsteps)
    Erh = np.zeros(nsteps)
    rc = lib().or_relax_cell(C.byref(p), float(rho), float(Eg), float(Er), float(dt),
                             int(nsteps), _dptr(Egh), _dptr(Erh))
    return rc, Egh, Erh


def step(grid, p, U, R=None, scratch=None, src=None):
    """One hydro step plus its radiation substeps; returns (rc, (dt, nsub, dt_rad), info).
    src: optional emissivity field j (radiation source of the exchange)."""
    if scratch is None:
        scratch = [np.zeros_like(U[0]) for _ in range(NHYD + NRAD)]
    out = (C.c_double * 3)()
    info = (C.c_int64 * 4)()
    rc = lib().or_step(grid.handle, C.byref(p), _ptr_array(U),
                       _ptr_array(R) if R is not None else None, _ptr_array(scratch),
                       _dptr(src) if src is not None else None, out, info)
    return rc, (out[0], int(out[1]), out[2]), tuple(info[:])


def conserved_sums(grid, p, U, R=None):
    out = (C.c_double * NSUMS)()
    lib().or_conserved_sums(grid.handle, C.byref(p), _ptr_array(U),
                            _ptr_array(R) if R is not None else None, out)
    return np.array(out[:])
