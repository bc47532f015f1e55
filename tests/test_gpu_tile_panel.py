"""The FP32 factorization with tile-pivoted panels (H2SP_PANEL=tile).

The pivot of each column is searched only in its panel's 64-row diagonal tile
(oracle.factor.getrf_tile), so a panel needs no search or row exchange below
the tile.  On the 2D -log r workload (N = 65,536, one right-hand side), an FP32
emulation of the block LU gives the same preconditioner quality: 5 GMRES
steps against 4 with partial pivoting over the supernode.  The switch is read
once per process, so each case runs in a child process.
Bars: GMRES on the FP64 H^2 product reaches 1e-10, and the solution agrees
with the oracle's FP64 direct solve to the accuracy that residual implies.

On a GB300 the 4,096- and 3,001-point cases pass in 4 GMRES steps, but the
16,384-point case stagnates at a relative residual of 3.3e-10 after 80 steps
(GMRES(20)), while supernode pivoting converges there.  That case is marked
as an expected failure; it is why tile pivoting is not the default.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1705_04601_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import factor as ofa  # noqa: E402
from oracle import sparsify as osp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_CHILD = r"""
import json, sys
import numpy as np
import torch
from paper_1705_04601_gb300 import synth, h2sp as H
n, leaf, tol, seed = int(sys.argv[1]), int(sys.argv[2]), float(sys.argv[3]), int(sys.argv[4])
h, b = synth.make_small(n, kernel="log", leaf=leaf, tol=tol, seed=seed, nrhs=3)
hd = H.h2sp_sparsify(H.H2Input(h))
H.h2sp_factor(hd, H.H2SP_FP32)
bt = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()
xt = torch.empty_like(bt)
info = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_GMRES, tol=1e-10, maxit=80, restart=20)
torch.cuda.synchronize()
np.save(sys.argv[5], xt.cpu().numpy().T)
print(json.dumps({"status": int(info.status), "iters": int(info.iters), "res": float(info.rel_residual)}))
hd.close()
"""


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1705_04601_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA is required for the gpu tests")


@pytest.mark.parametrize("n,leaf,tol,seed", [
    (4096, 64, 1e-8, 1), (3001, 23, 1e-7, 8),
    pytest.param(16384, 64, 1e-6, 9, marks=pytest.mark.xfail(
        reason="tile pivoting: GMRES(20) stagnates at 3.3e-10 after 80 steps on a GB300", strict=False))])
def test_tile_panel_preconditioner_reaches_1e10(tmp_path, n, leaf, tol, seed):
    out = str(tmp_path / "x.npy")
    env = dict(os.environ, H2SP_PANEL="tile", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", _CHILD, str(n), str(leaf), str(tol), str(seed), out], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    info = json.loads(r.stdout.strip().splitlines()[-1])
    print("tile panel n=%d: %s" % (n, info))
    assert info["status"] == 0 and info["res"] <= 1e-10
    h, b = synth.make_small(n, kernel="log", leaf=leaf, tol=tol, seed=seed, nrhs=3)
    sp = osp.sparsify(h)
    xo = ofa.solve(h, sp, ofa.factor(h, sp, pivot="tile"), b)
    xg = np.load(out)
    assert np.linalg.norm(xg - xo) <= 1e-6 * np.linalg.norm(xo)
