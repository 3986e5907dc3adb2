"""The ghost-fill plan of the library, replayed on the host (no GPU): the
copy descriptors and Dirichlet regions that qk_init_patches uploads, applied
with the kernel's own index formulas, must stay inside the field arrays,
write every ghost cell exactly once and never an interior cell, and
reproduce the oracle's boundary-resolved ghost values bit for bit."""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2110_01792_gb300 import inputs as I
from tests import problems as P

PER, REF, OUT, DIR = 0, 1, 2, 3
VEC = P.VEC_AXIS


def _qk():
    from paper_2110_01792_gb300 import build as B
    try:
        B.build()
    except (RuntimeError, FileNotFoundError) as e:
        pytest.skip(f"cannot build libqk: {e}")
    from paper_2110_01792_gb300 import qk
    return qk


def _layouts():
    return [P.two_patches((11, 9, 7)), P.two_patches((5, 4, 6)),
            I.make_layout([[0, 0, 0], [13, 0, 0], [0, 7, 0]],
                          [[13, 7, 11], [6, 17, 11], [13, 10, 11]], (19, 17, 11), 4),
            I.patch_tiling(dom_n=(48, 40, 32), seed=5, ng=4, edges=(8, 16, 24))]


def _replay(lay, copies, dirs, fields, fid0, interior):
    """Apply the plan to host arrays exactly as the fill kernels index them;
    every source must be an interior cell (the kernel reads and writes the
    same arrays, so a ghost source would race); returns the per-element write
    count."""
    n = lay.field_len
    writes = np.zeros(n, dtype=np.int64)
    src_vals = [f.copy() for f in fields]
    for (dst, src, ex, ey, ez, dsx, dsy, flip, sx, sy, sz) in copies:
        z, y, x = np.meshgrid(np.arange(ez), np.arange(ey), np.arange(ex), indexing="ij")
        d = dst + (z * dsy + y) * dsx + x
        s = src + x * sx + y * sy + z * sz
        assert d.min() >= 0 and d.max() < n and s.min() >= 0 and s.max() < n
        assert interior[s].all()
        np.add.at(writes, d.ravel(), 1)
        for k, f in enumerate(fields):
            ax = VEC.get(fid0 + k, -1)
            sign = -1.0 if ax >= 0 and (flip >> ax) & 1 else 1.0
            f[d] = sign * src_vals[k][s]
    for (dst, _, ex, ey, ez, dsx, dsy) in dirs:
        z, y, x = np.meshgrid(np.arange(ez), np.arange(ey), np.arange(ex), indexing="ij")
        d = dst + (z * dsy + y) * dsx + x
        assert d.min() >= 0 and d.max() < n
        np.add.at(writes, d.ravel(), 1)
        # restore: the recorded state is what the caller's ghost cells held
    return writes


BC_SETS = [((PER,) * 3, (PER,) * 3), ((REF, OUT, PER), (REF, OUT, PER)),
           ((DIR, REF, OUT), (DIR, REF, OUT)), ((OUT, DIR, REF), (DIR, REF, REF)),
           ((DIR,) * 3, (DIR,) * 3), ((REF,) * 3, (OUT,) * 3)]


@pytest.mark.parametrize("bcs", BC_SETS, ids=lambda b: "".join(map(str, b[0] + b[1])))
def test_fill_plan_reproduces_the_oracle(bcs):
    qk = _qk()
    bc_lo, bc_hi = bcs
    for lay in _layouts():
        if any(lay.dom_n[d] < lay.ng for d in range(3) if REF in (bc_lo[d], bc_hi[d])):
            continue
        prm = dict(hydro_only=1, dx=0.1, bc_lo=bc_lo, bc_hi=bc_hi)
        copies, dirs = qk.fill_plan(lay, prm)
        rng = np.random.Generator(np.random.Philox(7))
        # ghost cells: a consistent function of position where Dirichlet, noise elsewhere
        ext = [rng.standard_normal(tuple(m + 2 * lay.ng for m in lay.dom_n[::-1])) for _ in range(9)]
        fields = [np.full(lay.field_len, np.nan) for _ in range(9)]
        for f, e in zip(fields, ext):
            for b in range(lay.nbox):
                idx = []
                for d in range(3):
                    x = np.arange(lay.lo[b][d] - lay.ng, lay.lo[b][d] + lay.n[b][d] + lay.ng)
                    if bc_lo[d] == PER:
                        x = np.mod(x, lay.dom_n[d])
                    idx.append(x + lay.ng)
                lay.full(f, b)[...] = e[np.ix_(idx[2], idx[1], idx[0])]
        g = O.Grid(lay.lo, lay.n, lay.off, lay.dom_n, lay.ng)
        p = O.make_params(**prm)
        if DIR in bc_lo + bc_hi:
            assert O.set_dirichlet(g, p, fields[:5], fields[5:]) == 0
        else:
            assert len(dirs) == 0
        ref = [f.copy() for f in fields]
        assert O.fill_ghosts_bc(g, p, ref[:5], 0) == 0
        assert O.fill_ghosts_bc(g, p, ref[5:], 5) == 0
        got = [f.copy() for f in fields]
        # ghost cells outside any Dirichlet region are overwritten by copies;
        # scramble them first so that a missing copy shows
        mask_dir = np.zeros(lay.field_len, dtype=bool)
        for (dst, _, ex, ey, ez, dsx, dsy) in dirs:
            z, y, x = np.meshgrid(np.arange(ez), np.arange(ey), np.arange(ex), indexing="ij")
            mask_dir[(dst + (z * dsy + y) * dsx + x).ravel()] = True
        interior = np.zeros(lay.field_len, dtype=bool)
        for b in range(lay.nbox):
            lay.interior(interior, b)[...] = True
        for f in got:
            f[~interior & ~mask_dir] = 1e300
        w1 = _replay(lay, copies, dirs, got[:5], 0, interior)
        w2 = _replay(lay, copies, dirs, got[5:], 5, interior)
        assert np.array_equal(w1, w2)
        inside = np.zeros(lay.field_len, dtype=bool)
        for b in range(lay.nbox):
            inside[lay.off[b]:lay.off[b] + int(np.prod(lay.n[b] + 2 * lay.ng))] = True
        assert np.all(w1[interior] == 0)
        assert np.all(w1[inside & ~interior] == 1)
        for a, r in zip(got, ref):
            for b in range(lay.nbox):
                assert np.array_equal(lay.full(a, b), lay.full(r, b))


def test_fill_plan_validation():
    """Invalid boundary combinations are rejected on the host: a periodic face
    paired with a non-periodic one, unknown types, a reflecting axis shorter
    than the ghost width, an unknown closure."""
    qk = _qk()
    lay = P.two_patches((11, 9, 3))
    for kw, word in ((dict(bc_lo=(PER, 0, 0), bc_hi=(REF, 0, 0)), "periodic"),
                     (dict(bc_lo=(7, 0, 0), bc_hi=(7, 0, 0)), "unknown boundary"),
                     (dict(bc_lo=(0, 0, REF), bc_hi=(0, 0, REF)), "reflecting"),
                     (dict(closure=5), "closure")):
        with pytest.raises(qk.QKError) as e:
            qk.fill_plan(lay, dict(hydro_only=1, dx=0.1, **kw))
        assert word in str(e.value).lower(), (word, str(e.value))
