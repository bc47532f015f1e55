"""The allocation-free H^2 product, h2sp_h2_matvec_static, through the C ABI.

This entry point serves callers that cannot allocate device memory where they
call it: code running while someone else owns or budgets the memory pool, an
allocation-free real-time loop, or a plug-in whose host forbids cudaMalloc.
Its two coefficient workspaces live in a static device array inside the
library, so it must give exactly the product h2sp_apply(H2SP_OP_H2) gives,
call after call, and refuse matrices whose workspace would not fit.

This file is collected last on purpose: it should pass both alone in a fresh
process and after every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1705_04601_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_04601_gb300 import h2sp as H  # noqa: E402

STATIC_DOUBLES = 1 << 21


def _static_matvec(hd, x, y):
    n = x.shape[1]
    return H.lib().h2sp_h2_matvec_static(hd.ptr, int(x.shape[0]), ctypes.c_void_p(x.data_ptr()), n,
                                         ctypes.c_void_p(y.data_ptr()), n,
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_static_workspace_product_matches_apply_on_two_calls():
    from paper_1705_04601_gb300 import build
    build.build()
    h, _ = synth.make_small(4096, kernel="log", leaf=64, tol=1e-8, seed=1)
    hd = H.h2sp_sparsify(H.H2Input(h))
    rng = np.random.default_rng(20)
    for call in range(2):
        nrhs = 20 if call == 0 else 3   # 20 columns take two 16-column passes
        x = torch.from_numpy(rng.standard_normal((nrhs, h.n))).cuda()
        ref = torch.empty_like(x)
        H.h2sp_apply(hd, H.H2SP_OP_H2, x, ref)
        y = torch.full_like(x, float("nan"))
        assert _static_matvec(hd, x, y) == H.H2SP_OK
        torch.cuda.synchronize()
        assert bool(torch.isfinite(y).all())
        assert float((y - ref).norm()) <= 1e-12 * float(ref.norm())
    hd.close()


def test_static_workspace_rejects_a_matrix_that_does_not_fit():
    # raw Chebyshev ranks (16 per cluster) on many small leaves: the workspace
    # 2 * 16 * sum(ranks) exceeds the static array
    h, _ = synth.make_small(24000, kernel="log", leaf=12, tol=None, seed=5)
    assert 2 * 16 * int(h.rank.sum()) > STATIC_DOUBLES
    hd = H.h2sp_sparsify(H.H2Input(h))
    x = torch.ones(1, h.n, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    assert _static_matvec(hd, x, y) == H.H2SP_EUNSUPPORTED
    assert "static array" in H.lib().h2sp_last_cuda_error().decode()
    hd.close()
