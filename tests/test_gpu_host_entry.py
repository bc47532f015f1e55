"""h2sp_solve_host: the whole path (sparsify, factor, solve) from host
buffers in one C-ABI call, against the same steps through the device-pointer
entry points and against the oracle's H^2 product."""
import numpy as np
import pytest

from paper_1705_04601_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_04601_gb300 import h2sp as H  # noqa: E402
from oracle import factor as ofa  # noqa: E402
from oracle import h2 as oh2  # noqa: E402
from oracle import sparsify as osp  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1705_04601_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA is required for the gpu tests")


def _host_cols(b):
    """(n, nrhs) numpy -> Fortran-ordered copy and its address."""
    bf = np.asfortranarray(b, dtype=np.float64)
    return bf, bf.ctypes.data


@pytest.mark.parametrize("with_analysis", [True, False])
def test_host_entry_fp64_direct_matches_oracle(with_analysis):
    h, b = synth.make_small(1024, kernel="log", leaf=32, tol=1e-8, seed=1, nrhs=3)
    an = H.h2sp_analyze(H.H2Input(h, device=None)) if with_analysis else None
    inp = H.H2Input(h, device="host")
    bf, bp = _host_cols(b)
    x = np.zeros((h.n, 3), order="F")
    info = H.h2sp_solve_host(an, inp, bp, h.n, x.ctypes.data, h.n, 3, flags=0, prec=H.H2SP_FP64,
                             mode=H.H2SP_DIRECT)
    assert info.status == H.H2SP_OK
    sp = osp.sparsify(h)
    xo = ofa.solve(h, sp, ofa.factor(h, sp), b)
    assert np.linalg.norm(x - xo) <= 1e-10 * np.linalg.norm(xo)


def test_host_entry_mixed_gmres_matches_device_path():
    h, _ = synth.make_workload("inv3d_sphere_n262144", n=8192)
    b = np.random.default_rng(5).standard_normal((h.n, 2))
    an = H.h2sp_analyze(H.H2Input(h, device=None))
    # pinned host copies of the numbers, as a caller that stages its data would keep them
    host = {nm: torch.from_numpy(np.ascontiguousarray(getattr(h, nm))).pin_memory()
            for nm in ("leaf_basis", "transfer", "coupling", "near_block")}
    inp = H.H2Input(h, device="host", host=host)
    bf, bp = _host_cols(b)
    x = np.zeros((h.n, 2), order="F")
    info = H.h2sp_solve_host(an, inp, bp, h.n, x.ctypes.data, h.n, 2, flags=H.H2SP_SPARSIFY_FP32,
                             prec=H.H2SP_FP32_CHOL, mode=H.H2SP_GMRES, tol=1e-10)
    assert info.status == H.H2SP_OK and info.rel_residual <= 1e-10
    r = np.linalg.norm(b - oh2.Matvec(h)(x), axis=0) / np.linalg.norm(b, axis=0)
    assert r.max() <= 2e-10
    # the device-pointer path on the same inputs
    hd = H.h2sp_sparsify_analyzed(an, H.H2Input(h), flags=H.H2SP_SPARSIFY_FP32)
    H.h2sp_factor(hd, H.H2SP_FP32_CHOL)
    bt = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()
    xt = torch.empty_like(bt)
    info2 = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_GMRES, tol=1e-10, maxit=60, restart=20)
    assert info2.status == H.H2SP_OK
    xd = xt.cpu().numpy().T
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    hd.close()


def test_host_entry_rejects_another_structure():
    h, b = synth.make_small(1024, kernel="log", leaf=32, tol=1e-8, seed=1, nrhs=1)
    h2, _ = synth.make_small(1024, kernel="log", leaf=32, tol=1e-8, seed=3, nrhs=1)
    an = H.h2sp_analyze(H.H2Input(h2, device=None))
    inp = H.H2Input(h, device="host")
    bf, bp = _host_cols(b)
    x = np.zeros((h.n, 1), order="F")
    with pytest.raises(H.H2spError) as e:
        H.h2sp_solve_host(an, inp, bp, h.n, x.ctypes.data, h.n, 1, prec=H.H2SP_FP64, mode=H.H2SP_DIRECT)
    assert e.value.status == H.H2SP_EINVAL
