"""GPU parity for blocks above 64 rows (3D leaves of up to 128 points, upper
levels stacked from up to eight sons), through the C ABI.

These items take the streaming kernels: k_householder_large,
k_transform_large, k_apply_qt_large / k_apply_q_large and
k_h2_leaf_out_large.  The bars are those of test_gpu_parity.py:
* per block of S, ||S_gpu - S_oracle||_F <= 1e-10 ||row block of S_oracle||_F;
* per cluster, ||Q_gpu - Q_oracle||_F <= 1e-10 ||Q||_F;
* applies and products within 1e-12 (scaled by sqrt(n) / 8);
* the FP64 direct solve within 1e-10 of the oracle's;
* FP32 factors + GMRES reach 1e-10 on the FP64 H^2 product.

"""
import numpy as np
import pytest

from paper_1705_04601_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_04601_gb300 import h2sp as H  # noqa: E402
from oracle import factor as ofa  # noqa: E402
from oracle import h2 as oh2  # noqa: E402
from oracle import sparsify as osp  # noqa: E402

TOL = 1e-10

# 1/r on the jittered Fibonacci sphere (leaf <= 128; level blocks up to 91 rows)
# and Yukawa in the unit cube (leaves up to 113 points)
_CASES = {
    "sphere8k": ("inv3d_sphere_n262144", 8192),
    "cube6k": ("yukawa3d_n1048576", 6000),
}
_cache = {}


def case(name):
    if name not in _cache:
        wl, n = _CASES[name]
        h, _ = synth.make_workload(wl, n=n)
        b = np.random.default_rng(11).standard_normal((h.n, 3))
        _cache[name] = (h, b, osp.sparsify(h))
    return _cache[name]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1705_04601_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA is required for the gpu tests")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, np.float64).reshape(a.shape[0], -1).T)).cuda()


def host(t):
    return t.cpu().numpy().T


@pytest.mark.parametrize("name", list(_CASES))
def test_large_blocks_S_and_Q_match_oracle(name):
    h, b, sp = case(name)
    assert max(int(sp.sch.m[c]) for c in range(h.ncl) if sp.sch.level[c] < max(sp.sch.lstop, 1)) > 64
    hd = H.h2sp_sparsify(H.H2Input(h))
    S = H.h2sp_export_S(hd)
    vbr = osp.to_vbr(sp)
    assert np.array_equal(S["brow_ptr"], vbr.brow_ptr) and np.array_equal(S["bcol_idx"], vbr.bcol_idx)
    ns = vbr.node_size
    for i in range(ns.size):
        lo, hi = int(vbr.brow_ptr[i]), int(vbr.brow_ptr[i + 1])
        if hi == lo:
            continue
        a, e = int(vbr.val_off[lo]), int(vbr.val_off[hi - 1] + ns[i] * ns[vbr.bcol_idx[hi - 1]])
        ref_row = np.linalg.norm(vbr.vals[a:e])
        for z in range(lo, hi):
            j = int(vbr.bcol_idx[z])
            o, sz = int(vbr.val_off[z]), int(ns[i] * ns[j])
            d = np.linalg.norm(S["vals"][o:o + sz] - vbr.vals[o:o + sz])
            assert d <= TOL * max(ref_row, 1e-300), (i, j, d, ref_row)
    for t in sp.Q:
        Qg = H.h2sp_export_Q(hd, t)
        assert np.linalg.norm(Qg - sp.Q[t]) <= TOL * np.linalg.norm(sp.Q[t]), t
    hd.close()


@pytest.mark.parametrize("name", list(_CASES))
def test_large_blocks_applies_and_products(name):
    h, b, sp = case(name)
    hd = H.h2sp_sparsify(H.H2Input(h))
    bt = dev(b)
    out = torch.empty_like(bt)
    for op, ref in [(H.H2SP_OP_UT, osp.apply_T(sp, h, b, col=False)), (H.H2SP_OP_V, osp.apply_N(sp, h, b, col=True)),
                    (H.H2SP_OP_S, osp.dense_S(sp) @ b), (H.H2SP_OP_H2, oh2.Matvec(h)(b))]:
        H.h2sp_apply(hd, op, bt, out)
        torch.cuda.synchronize()
        g = host(out)
        assert np.linalg.norm(g - ref) <= 1e-12 * np.linalg.norm(ref) * max(1.0, np.sqrt(h.n) / 8), op
    hd.close()


@pytest.mark.parametrize("name", list(_CASES))
def test_large_blocks_fp64_direct_and_fp32_gmres(name):
    h, b, sp = case(name)
    hd = H.h2sp_sparsify(H.H2Input(h))
    bt = dev(b)
    xt = torch.empty_like(bt)
    H.h2sp_factor(hd, H.H2SP_FP64)
    H.h2sp_solve(hd, bt, xt, mode=H.H2SP_DIRECT)
    torch.cuda.synchronize()
    xo = ofa.solve(h, sp, ofa.factor(h, sp), b)
    assert np.linalg.norm(host(xt) - xo) <= TOL * np.linalg.norm(xo)
    H.h2sp_factor(hd, H.H2SP_FP32)
    info = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_GMRES, tol=1e-10, maxit=60, restart=20)
    assert info.status == H.H2SP_OK and info.rel_residual <= 1e-10
    torch.cuda.synchronize()
    r = np.linalg.norm(b - oh2.Matvec(h)(host(xt)), axis=0) / np.linalg.norm(b, axis=0)
    assert r.max() <= 2e-10
    hd.close()


@pytest.mark.parametrize("name", list(_CASES))
@pytest.mark.parametrize("nrhs", [1, 2, 4, 5, 16])
def test_h2_product_for_each_count_of_right_hand_sides(name, nrhs):
    """The FP64 H^2 product takes the few-right-hand-side kernels up to 4
    columns and the 16-column ones above; both within 1e-12 of the oracle."""
    h, _, _ = case(name)
    b = np.random.default_rng(100 + nrhs).standard_normal((h.n, nrhs))
    hd = H.h2sp_sparsify(H.H2Input(h))
    bt = dev(b)
    out = torch.empty_like(bt)
    H.h2sp_apply(hd, H.H2SP_OP_H2, bt, out)
    torch.cuda.synchronize()
    ref = oh2.Matvec(h)(b)
    g = host(out).reshape(ref.shape)
    assert np.linalg.norm(g - ref) <= 1e-12 * np.linalg.norm(ref) * max(1.0, np.sqrt(h.n) / 8)
    hd.close()
