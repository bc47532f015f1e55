"""Failure detection on the GPU without a fault: a bounded device wait that
runs out.

The triangular sweeps synchronise their row blocks by flags (one cooperative
launch per level and direction); every wait is bounded.  With a short poll
limit (H2SP_OPTION_WAIT_POLLS) and the forward sweeps awaiting an epoch that
no block publishes (H2SP_OPTION_TEST_STALE_EPOCH), every wait on another
block gives up, raises the solve's error word and leaves: the solve returns
H2SP_ETIMEOUT.  The same handle then solves correctly, and the device keeps
working for a new handle.
"""
import numpy as np
import pytest

from paper_1705_04601_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_04601_gb300 import h2sp as H  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1705_04601_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA is required for the gpu tests")


@pytest.mark.parametrize("prec", [H.H2SP_FP64, H.H2SP_FP32])
def test_sweep_wait_runs_out_and_the_handle_recovers(prec):
    h, b = synth.make_small(4096, kernel="log", leaf=64, tol=1e-8, seed=1, nrhs=2)
    hd = H.h2sp_sparsify(H.H2Input(h))
    H.h2sp_factor(hd, prec)
    bt = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()
    x0 = torch.empty_like(bt)
    info = H.h2sp_solve(hd, bt, x0, mode=H.H2SP_DIRECT)
    assert info.status == H.H2SP_OK
    H.h2sp_set_option(hd, H.H2SP_OPTION_WAIT_POLLS, 2000)
    H.h2sp_set_option(hd, H.H2SP_OPTION_TEST_STALE_EPOCH, 1)
    x1 = torch.empty_like(bt)
    with pytest.raises(H.H2spError) as e:
        H.h2sp_solve(hd, bt, x1, mode=H.H2SP_DIRECT)
    assert e.value.status == H.H2SP_ETIMEOUT
    # the option cleared itself: the same handle solves again, to the same x
    # up to the order of the atomic additions of the boundary rows (FP32
    # factors: to the FP32 direct solve's accuracy)
    x2 = torch.empty_like(bt)
    info = H.h2sp_solve(hd, bt, x2, mode=H.H2SP_DIRECT)
    assert info.status == H.H2SP_OK
    torch.cuda.synchronize()
    tol = 1e-10 if prec == H.H2SP_FP64 else 1e-3
    assert float((x0 - x2).norm() / x0.norm()) <= tol
    # and GMRES to 1e-10 still works on it
    info = H.h2sp_solve(hd, bt, x2, mode=H.H2SP_GMRES, tol=1e-10, maxit=60, restart=20)
    assert info.status == H.H2SP_OK and info.rel_residual <= 1e-10
    hd.close()
    # a new handle on the same device
    hd2 = H.h2sp_sparsify(H.H2Input(h))
    H.h2sp_factor(hd2, prec)
    info = H.h2sp_solve(hd2, bt, x2, mode=H.H2SP_IR, tol=1e-10, maxit=30)
    assert info.status == H.H2SP_OK and info.rel_residual <= 1e-10
    hd2.close()


def test_wait_option_values_checked():
    h, _ = synth.make_small(512, kernel="log", leaf=32, tol=1e-8, seed=2, nrhs=1)
    hd = H.h2sp_sparsify(H.H2Input(h))
    for opt, val in [(H.H2SP_OPTION_WAIT_POLLS, 0), (H.H2SP_OPTION_WAIT_POLLS, 1 << 40), (99, 1)]:
        with pytest.raises(H.H2spError) as e:
            H.h2sp_set_option(hd, opt, val)
        assert e.value.status == H.H2SP_EINVAL
    hd.close()
