"""Diagnostic parity build: the library compiled without FMA contraction
(``--fmad=false``; the compiler keeps every product and sum separately
rounded, as the oracle's plain C does under ``-ffp-contract=off``, while the
explicit fma() calls of both sources remain) meets the same ten-step FP64
bound against the oracle as the production build.  The two errors, printed
by the child processes, separate the contraction's share of the parity
residual from the rest of the rounding-order differences."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# runs in a child process so that QK_FMAD selects the library before it loads
_SCRIPT = r"""
import json
from tests import gpu_util as G
from tests import test_gpu_parity as T
lay, prob, prm = T._small_rhd()
Ug, Rg, _, st = T._run_gpu_steps(lay, prob, prm, 10)
Ur, Rr, _ = T._run_oracle_steps(lay, prob, prm, 10)
print(json.dumps({"status": int(st[0]), "err": max(G.max_rel_err(lay, Ug + Rg, Ur + Rr))}))
"""


def _ten_steps(fmad: bool) -> dict:
    env = dict(os.environ, QK_FMAD="1" if fmad else "0")
    r = subprocess.run([sys.executable, "-c", _SCRIPT], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_rhd_ten_steps_without_fma_contraction():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    from paper_2110_01792_gb300 import build as B
    __graft_entry__.build()
    B.build(fmad=False)
    prod, nofma = _ten_steps(True), _ten_steps(False)
    print(f"10 RHD steps, max relative error vs the oracle: production {prod['err']:.3e}, "
          f"--fmad=false {nofma['err']:.3e}")
    assert prod["status"] == 0 and nofma["status"] == 0
    assert prod["err"] <= 1e-10 and nofma["err"] <= 1e-10
