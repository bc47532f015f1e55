"""GPU parity of the CUDA path against the CPU oracle, through the C ABI.

Bars:
* integer structure (S node order, VBR pattern, elimination structure): equal;
* FP64 values: per block of S, ||S_gpu - S_oracle||_F <= 1e-10 ||row block of S_oracle||_F;
  per cluster, ||Q_gpu - Q_oracle||_F <= 1e-10 ||Q||_F; solutions
  ||x_gpu - x_oracle|| <= 1e-10 ||x_oracle|| for the FP64 direct solve;
* the FP32-factor preconditioned refinement reaches a relative residual of
  1e-10 on the FP64 H^2 product and then agrees with the FP64 solution to
  the accuracy that residual implies.
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

_CASES = {
    "log1k": dict(n=1024, kernel="log", leaf=32, tol=1e-8, seed=1),
    "log4k": dict(n=4096, kernel="log", leaf=64, tol=1e-8, seed=1),
    "skew1k": dict(n=1024, kernel="log_skew", leaf=32, tol=1e-8, seed=2),
    "raw1k": dict(n=1024, kernel="log", leaf=32, tol=None, seed=3),
    "tiny": dict(n=48, kernel="log", leaf=64, tol=1e-8, seed=6),
    "ragged": dict(n=3001, kernel="log", leaf=23, tol=1e-7, seed=8),
    "inv3d": dict(n=1500, kernel="inv", leaf=40, tol=1e-6, seed=5, dim=3),
}
_cache = {}


def case(name):
    if name not in _cache:
        s = _CASES[name]
        h, b = synth.make_small(s["n"], kernel=s["kernel"], leaf=s["leaf"], tol=s["tol"], seed=s["seed"],
                                dim=s.get("dim", 2), nrhs=3)
        sp = osp.sparsify(h)
        _cache[name] = (h, b, sp)
    return _cache[name]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1705_04601_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA is required for the gpu tests")


def dev(a):
    """(n, nrhs) numpy -> (nrhs, n) cuda tensor (column-major n x nrhs)."""
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, np.float64).reshape(a.shape[0], -1).T)).cuda()


def host(t):
    return t.cpu().numpy().T


def sparsified(name):
    h, b, sp = case(name)
    inp = H.H2Input(h)
    hd = H.h2sp_sparsify(inp)
    return h, b, sp, hd


@pytest.mark.parametrize("name", list(_CASES))
def test_S_and_Q_match_oracle(name):
    h, b, sp, hd = sparsified(name)
    S = H.h2sp_export_S(hd)
    vbr = osp.to_vbr(sp)
    assert np.array_equal(S["brow_ptr"], vbr.brow_ptr)
    assert np.array_equal(S["bcol_idx"], vbr.bcol_idx)
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
        if not h.symmetric_bases:
            Qcg = H.h2sp_export_Q(hd, t, col=True)
            assert np.linalg.norm(Qcg - sp.Qc[t]) <= TOL * np.linalg.norm(sp.Qc[t]), t
    hd.close()


@pytest.mark.parametrize("name", ["log1k", "skew1k", "tiny", "ragged", "inv3d"])
def test_applies_and_products(name):
    h, b, sp, hd = sparsified(name)
    n = h.n
    bt = dev(b)
    out = torch.empty_like(bt)
    for op, ref in [(H.H2SP_OP_UT, osp.apply_T(sp, h, b, col=False)), (H.H2SP_OP_VT, osp.apply_T(sp, h, b, col=True)),
                    (H.H2SP_OP_U, osp.apply_N(sp, h, b, col=False)), (H.H2SP_OP_V, osp.apply_N(sp, h, b, col=True)),
                    (H.H2SP_OP_S, osp.dense_S(sp) @ b), (H.H2SP_OP_H2, oh2.Matvec(h)(b))]:
        H.h2sp_apply(hd, op, bt, out)
        torch.cuda.synchronize()
        g = host(out)
        assert np.linalg.norm(g - ref) <= 1e-12 * np.linalg.norm(ref) * max(1.0, np.sqrt(n) / 8), op
    hd.close()


@pytest.mark.parametrize("name", ["log1k", "log4k", "skew1k", "raw1k", "tiny", "ragged", "inv3d"])
def test_fp64_direct_solve_matches_oracle(name):
    h, b, sp, hd = sparsified(name)
    H.h2sp_factor(hd, H.H2SP_FP64)
    fa = ofa.factor(h, sp)
    xo = ofa.solve(h, sp, fa, b)
    bt = dev(b)
    xt = torch.empty_like(bt)
    H.h2sp_solve(hd, bt, xt, mode=H.H2SP_DIRECT)
    torch.cuda.synchronize()
    xg = host(xt)
    assert np.linalg.norm(xg - xo) <= TOL * np.linalg.norm(xo)
    # S^{-1} directly
    c = osp.apply_T(sp, h, b)
    ct = dev(c)
    yt = torch.empty_like(ct)
    H.h2sp_apply(hd, H.H2SP_OP_SINV, ct, yt)
    torch.cuda.synchronize()
    yo = ofa.solve_S(fa, c)
    assert np.linalg.norm(host(yt) - yo) <= TOL * np.linalg.norm(yo)
    hd.close()


@pytest.mark.parametrize("name", ["log4k", "skew1k", "ragged"])
def test_fp32_refinement_reaches_1e10(name):
    h, b, sp, hd = sparsified(name)
    H.h2sp_factor(hd, H.H2SP_FP32)
    bt = dev(b)
    xt = torch.empty_like(bt)
    info = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_IR, tol=1e-10, maxit=30)
    assert info.status == H.H2SP_OK and info.rel_residual <= 1e-10
    xg = host(xt)
    A = oh2.dense(h)
    res = np.linalg.norm(b - A @ xg, axis=0) / np.linalg.norm(b, axis=0)
    assert res.max() <= 2e-10
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(xg - xd) <= 1e-7 * np.linalg.norm(xd)
    hd.close()


@pytest.mark.parametrize("nrhs", [1, 16, 20])
def test_many_rhs_chunks(nrhs):
    h, _, sp, hd = sparsified("log1k")
    rng = np.random.default_rng(nrhs)
    b = rng.standard_normal((h.n, nrhs))
    H.h2sp_factor(hd, H.H2SP_FP64)
    fa = ofa.factor(h, sp)
    xo = ofa.solve(h, sp, fa, b)
    bt = dev(b)
    xt = torch.empty_like(bt)
    H.h2sp_solve(hd, bt, xt, mode=H.H2SP_DIRECT)
    torch.cuda.synchronize()
    assert np.linalg.norm(host(xt) - xo) <= TOL * np.linalg.norm(xo)
    hd.close()


def test_singular_pivot_reported():
    """A zero close matrix and zero bases give S = 0: the factor must report a singular pivot."""
    h, _, sp = case("log1k")
    import copy
    h0 = copy.copy(h)
    h0.near_block = np.zeros_like(h.near_block)
    h0.coupling = np.zeros_like(h.coupling)
    hd = H.h2sp_sparsify(H.H2Input(h0))
    with pytest.raises(H.H2spError) as e:
        H.h2sp_factor(hd, H.H2SP_FP64)
    assert e.value.status == H.H2SP_ESINGULAR
    hd.close()


# ---------------------------------------------------------------------------
# full size: the 2D log kernel with 65,536 points, leaf <= 64, tol 1e-6, 16 RHS
# ---------------------------------------------------------------------------


@pytest.fixture(scope="module")
def full():
    h, b = synth.make_workload("log2d_n65536")
    sp = osp.sparsify(h)
    return h, b, sp


def test_full_size_S_parity(full):
    h, b, sp = full
    hd = H.h2sp_sparsify(H.H2Input(h))
    S = H.h2sp_export_S(hd)
    vbr = osp.to_vbr(sp)
    assert np.array_equal(S["brow_ptr"], vbr.brow_ptr) and np.array_equal(S["bcol_idx"], vbr.bcol_idx)
    ns = vbr.node_size
    rng = np.random.default_rng(0)
    rows = rng.choice(ns.size, size=min(400, ns.size), replace=False)
    for i in rows:
        lo, hi = int(vbr.brow_ptr[i]), int(vbr.brow_ptr[i + 1])
        a = int(vbr.val_off[lo])
        e = int(vbr.val_off[hi - 1] + ns[i] * ns[vbr.bcol_idx[hi - 1]])
        assert np.linalg.norm(S["vals"][a:e] - vbr.vals[a:e]) <= TOL * np.linalg.norm(vbr.vals[a:e])
    hd.close()


def test_full_size_fp64_direct_and_mixed_refinement(full):
    h, b, sp = full
    mv = oh2.Matvec(h)
    hd = H.h2sp_sparsify(H.H2Input(h))
    bt = dev(b)
    xt = torch.empty_like(bt)
    H.h2sp_factor(hd, H.H2SP_FP64)
    H.h2sp_solve(hd, bt, xt, mode=H.H2SP_DIRECT)
    torch.cuda.synchronize()
    xd = host(xt)
    r = np.linalg.norm(b - mv(xd), axis=0) / np.linalg.norm(b, axis=0)
    assert r.max() <= 1e-9   # one FP64 direct solve (blocked, inverted 64x64 diagonal blocks)
    info = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_IR, tol=1e-10, maxit=10)
    assert info.status == H.H2SP_OK and info.iters <= 3
    x64 = host(xt)
    r = np.linalg.norm(b - mv(x64), axis=0) / np.linalg.norm(b, axis=0)
    assert r.max() <= 1e-10
    H.h2sp_factor(hd, H.H2SP_FP32)
    info = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_IR, tol=1e-10, maxit=30)
    assert info.status == H.H2SP_OK
    x32 = host(xt)
    r = np.linalg.norm(b - mv(x32), axis=0) / np.linalg.norm(b, axis=0)
    assert r.max() <= 2e-10
    assert np.linalg.norm(x32 - x64) <= 1e-6 * np.linalg.norm(x64)
    hd.close()


# ---------------------------------------------------------------------------
# batched form: independent systems on random ellipses in one forest
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_forest_matches_individual_systems(prec):
    systems, f, b = synth.make_batched(6, 600, 3000, leaf=32, tol=1e-8, nrhs=2)
    hd = H.h2sp_sparsify(H.H2Input(f))
    bt = dev(b)
    xt = torch.empty_like(bt)
    if prec == "fp64":
        H.h2sp_factor(hd, H.H2SP_FP64)
        H.h2sp_solve(hd, bt, xt, mode=H.H2SP_DIRECT)
    else:
        H.h2sp_factor(hd, H.H2SP_FP32)
        info = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_IR, tol=1e-10, maxit=30)
        assert info.status == H.H2SP_OK and info.rel_residual <= 1e-10
    torch.cuda.synchronize()
    xg = host(xt)
    o = 0
    for s in systems:
        bs = b[o:o + s.n]
        sp = osp.sparsify(s)
        xo = ofa.solve(s, sp, ofa.factor(s, sp), bs)
        tol = TOL if prec == "fp64" else 1e-7
        assert np.linalg.norm(xg[o:o + s.n] - xo) <= tol * np.linalg.norm(xo)
        if prec == "fp32":  # every system meets the residual bound on its own
            r = np.linalg.norm(bs - oh2.Matvec(s)(xg[o:o + s.n]), axis=0) / np.linalg.norm(bs, axis=0)
            assert r.max() <= 2e-10
        o += s.n
    hd.close()


@pytest.mark.parametrize("name", ["log4k", "ragged"])
def test_fp32_factor_direct_accuracy(name):
    """One FP32-factor direct solve is accurate to the level of an FP32 dense
    LU with partial pivoting of the same matrix (computed here by LAPACK in
    float32).  The block LU pivots only inside each supernode and its
    extend-add rounds in a run-dependent order, so it may lose up to a small
    factor more; a TF32-only trailing update would lose about 1000x."""
    import os
    import scipy.linalg as sl
    h, b, sp, hd = sparsified(name)
    H.h2sp_factor(hd, H.H2SP_FP32)
    bt = dev(b)
    xt = torch.empty_like(bt)
    H.h2sp_solve(hd, bt, xt, mode=H.H2SP_DIRECT)
    torch.cuda.synchronize()
    xo = ofa.solve(h, sp, ofa.factor(h, sp), b)
    err = np.linalg.norm(host(xt) - xo) / np.linalg.norm(xo)
    lu32 = sl.lu_factor(oh2.dense(h).astype(np.float32))
    x32 = sl.lu_solve(lu32, b.astype(np.float32)).astype(np.float64)
    err32 = np.linalg.norm(x32 - xo) / np.linalg.norm(xo)
    print("fp32 direct rel err (%s, GEMM=%s): %.3e (dense FP32 LU: %.3e)"
          % (name, os.environ.get("H2SP_GEMM", "tc"), err, err32))
    assert err <= 25 * err32
    hd.close()


@pytest.mark.parametrize("name,prec", [("log4k", "fp32"), ("skew1k", "fp32"), ("ragged", "fp64")])
def test_gmres_reaches_1e10(name, prec):
    """Right-preconditioned restarted GMRES on the FP64 H^2 product (§5.5)."""
    h, b, sp, hd = sparsified(name)
    H.h2sp_factor(hd, H.H2SP_FP32 if prec == "fp32" else H.H2SP_FP64)
    bt = dev(b)
    xt = torch.empty_like(bt)
    info = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_GMRES, tol=1e-10, maxit=60, restart=20)
    assert info.status == H.H2SP_OK and info.rel_residual <= 1e-10
    xg = host(xt)
    A = oh2.dense(h)
    res = np.linalg.norm(b - A @ xg, axis=0) / np.linalg.norm(b, axis=0)
    assert res.max() <= 2e-10
    hd.close()


@pytest.mark.parametrize("name", ["log4k", "skew1k"])
def test_sparsify_analyzed_matches_sparsify(name):
    """The numeric phase on a shared host analysis gives the same S, Q and
    solution as the full h2sp_sparsify, also after the analysis handle is gone."""
    h, b, sp = case(name)
    inp = H.H2Input(h)
    full = H.h2sp_sparsify(inp)
    an = H.h2sp_analyze(H.H2Input(h, device=None))
    hd = H.h2sp_sparsify_analyzed(an, inp)
    an.close()
    Sf = H.h2sp_export_S(full)
    Sa = H.h2sp_export_S(hd)
    assert np.array_equal(Sf["brow_ptr"], Sa["brow_ptr"]) and np.array_equal(Sf["bcol_idx"], Sa["bcol_idx"])
    assert np.array_equal(Sf["vals"], Sa["vals"])
    H.h2sp_factor(hd, H.H2SP_FP64)
    bt = dev(b)
    xt = torch.empty_like(bt)
    H.h2sp_solve(hd, bt, xt, mode=H.H2SP_DIRECT)
    torch.cuda.synchronize()
    xo = ofa.solve(h, sp, ofa.factor(h, sp), b)
    assert np.linalg.norm(host(xt) - xo) / np.linalg.norm(xo) <= 1e-10
    full.close()
    hd.close()


@pytest.mark.parametrize("name", ["log1k", "skew1k", "ragged", "inv3d"])
def test_fp32_sparsification_matches_oracle(name):
    """H2SP_SPARSIFY_FP32: the Householder completions stay FP64, so every Q
    meets the FP64 bar (1e-10); the sandwich products run in FP32 with Q
    rounded to FP32, so each block row of S carries the rounding of two
    64-term FP32 products per level (about 2 x 64 x 6e-8 = 8e-6 per level in
    the worst case, a few e-7 typically) summed over at most 6 levels: 1e-4
    of the row-block norm.  The pattern is integer work and must be
    identical."""
    h, b, sp = case(name)
    hd = H.h2sp_sparsify(H.H2Input(h), flags=H.H2SP_SPARSIFY_FP32)
    assert H.h2sp_query(hd)["sparsify_prec"] == H.H2SP_FP32
    S = H.h2sp_export_S(hd)
    vbr = osp.to_vbr(sp)
    assert np.array_equal(S["brow_ptr"], vbr.brow_ptr) and np.array_equal(S["bcol_idx"], vbr.bcol_idx)
    ns = vbr.node_size
    worst = 0.0
    for i in range(ns.size):
        lo, hi = int(vbr.brow_ptr[i]), int(vbr.brow_ptr[i + 1])
        if hi == lo:
            continue
        a, e = int(vbr.val_off[lo]), int(vbr.val_off[hi - 1] + ns[i] * ns[vbr.bcol_idx[hi - 1]])
        ref_row = max(np.linalg.norm(vbr.vals[a:e]), 1e-300)
        worst = max(worst, np.linalg.norm(S["vals"][a:e] - vbr.vals[a:e]) / ref_row)
    print("fp32 products (%s): S row-block rel %.2e" % (name, worst))
    assert worst <= 1e-4
    for t in sp.Q:
        assert np.linalg.norm(H.h2sp_export_Q(hd, t) - sp.Q[t]) <= TOL * np.linalg.norm(sp.Q[t]), t
        if not h.symmetric_bases:
            Qcg = H.h2sp_export_Q(hd, t, col=True)
            assert np.linalg.norm(Qcg - sp.Qc[t]) <= TOL * np.linalg.norm(sp.Qc[t]), t
    hd.close()


@pytest.mark.parametrize("name,mode", [("log4k", "gmres"), ("skew1k", "gmres"), ("ragged", "gmres"),
                                       ("log4k", "ir")])
def test_fp32_sparsify_and_factor_reach_1e10(name, mode):
    """The preconditioner built from an FP32 S and FP32 factors (U and V
    FP64) still drives GMRES / refinement on the FP64 H^2 residual to 1e-10
    (§5.5), and the solution agrees with the dense FP64 solve to what that
    residual implies."""
    h, b, sp = case(name)
    hd = H.h2sp_sparsify(H.H2Input(h), flags=H.H2SP_SPARSIFY_FP32)
    H.h2sp_factor(hd, H.H2SP_FP32)
    bt = dev(b)
    xt = torch.empty_like(bt)
    if mode == "gmres":
        info = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_GMRES, tol=1e-10, maxit=60, restart=20)
    else:
        info = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_IR, tol=1e-10, maxit=30)
    print("fp32 sparsify + fp32 factor (%s, %s): %d iterations, residual %.2e" %
          (name, mode, info.iters, info.rel_residual))
    assert info.status == H.H2SP_OK and info.rel_residual <= 1e-10
    A = oh2.dense(h)
    xg = host(xt)
    res = np.linalg.norm(b - A @ xg, axis=0) / np.linalg.norm(b, axis=0)
    assert res.max() <= 2e-10
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(xg - xd) <= 1e-7 * np.linalg.norm(xd)
    hd.close()


def test_fp32_sparsify_products_stay_fp64_vectors():
    """With an FP32 S the applies still take and return FP64 vectors: U^T, V,
    U, V^T and the H^2 product do not touch S and keep the FP64 bar; S x
    differs from the oracle's by the FP32 rounding of S only (<= 1e-4)."""
    h, b, sp = case("skew1k")
    n = h.n
    hd = H.h2sp_sparsify(H.H2Input(h), flags=H.H2SP_SPARSIFY_FP32)
    bt = dev(b)
    out = torch.empty_like(bt)
    for op, ref in [(H.H2SP_OP_UT, osp.apply_T(sp, h, b, col=False)), (H.H2SP_OP_VT, osp.apply_T(sp, h, b, col=True)),
                    (H.H2SP_OP_U, osp.apply_N(sp, h, b, col=False)), (H.H2SP_OP_V, osp.apply_N(sp, h, b, col=True)),
                    (H.H2SP_OP_S, osp.dense_S(sp) @ b), (H.H2SP_OP_H2, oh2.Matvec(h)(b))]:
        H.h2sp_apply(hd, op, bt, out)
        torch.cuda.synchronize()
        rel = np.linalg.norm(host(out) - ref) / np.linalg.norm(ref)
        bound = 1e-4 if op == H.H2SP_OP_S else 1e-12 * max(1.0, np.sqrt(n) / 8)
        assert rel <= bound, (op, rel)
    hd.close()


def test_fp32_factor_backward_error():
    """The FP32 block LU of S is a backward-stable factorization, also on the
    large top fronts here (panels on thread-block clusters, block-end updates
    on the tensor cores): y = S^{-1} c from the FP32 factors has a normwise
    backward error ||c - S y|| / (||S||_F ||y|| + ||c||) of FP32 order
    (u = 6e-8 times a modest growth), required <= 1e-5; a wrong pivot row, a
    stale update or a misplaced row gives O(1e-2) or more."""
    n = 16384
    h, _ = synth.make_workload("log2d_n65536", n=n)
    hd = H.h2sp_sparsify(H.H2Input(h))
    H.h2sp_factor(hd, H.H2SP_FP32)
    c = np.random.default_rng(5).standard_normal((n, 4))
    ct = dev(c)
    yt = torch.empty_like(ct)
    rt = torch.empty_like(ct)
    H.h2sp_apply(hd, H.H2SP_OP_SINV, ct, yt)
    H.h2sp_apply(hd, H.H2SP_OP_S, yt, rt)
    torch.cuda.synchronize()
    nS = np.linalg.norm(H.h2sp_export_S(hd)["vals"])
    y, r = host(yt), c - host(rt)
    eta = (np.linalg.norm(r, axis=0) / (nS * np.linalg.norm(y, axis=0) + np.linalg.norm(c, axis=0))).max()
    print("fp32 factor backward error (n=%d): %.2e" % (n, eta))
    assert eta <= 1e-5
    hd.close()


@pytest.mark.parametrize("name,prec,flags", [("log4k", "fp32", 1), ("skew1k", "fp32", 0), ("log1k", "fp64", 0)])
def test_refactor_replays_on_new_numbers(name, prec, flags):
    """h2sp_refactor: after new numbers are written into the borrowed arrays
    (here the close blocks and couplings doubled in place, so A becomes 2A
    exactly), the captured sparsification + factorization gives the solution
    of 2 A x = b: the dense solution halved, on the first call (capture) and
    on the second (replay)."""
    h, b, sp = case(name)
    inp = H.H2Input(h)
    hd = H.h2sp_sparsify(inp, flags=flags)
    P = H.H2SP_FP32 if prec == "fp32" else H.H2SP_FP64
    with pytest.raises(H.H2spError) as e:
        H.h2sp_refactor(hd)
    assert e.value.status == H.H2SP_ESTATE
    H.h2sp_factor(hd, P)
    A = oh2.dense(h)
    xd = np.linalg.solve(A, b)
    bt = dev(b)
    xt = torch.empty_like(bt)
    for scale in (2.0, 4.0):
        inp.dev["near_block"].mul_(2.0)
        inp.dev["coupling"].mul_(2.0)
        H.h2sp_refactor(hd)
        if prec == "fp32":
            info = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_GMRES, tol=1e-10, maxit=60, restart=20)
            assert info.status == H.H2SP_OK and info.rel_residual <= 1e-10
            bound = 1e-7
        else:
            H.h2sp_solve(hd, bt, xt, mode=H.H2SP_DIRECT)
            bound = 1e-9
        torch.cuda.synchronize()
        xg = host(xt)
        err = np.linalg.norm(xg - xd / scale) / np.linalg.norm(xd / scale)
        print("refactor (%s, %s, x%g): rel err %.2e" % (name, prec, scale, err))
        assert err <= bound
    if prec == "fp32":
        # a factorization in the other precision replaces the captured one
        H.h2sp_factor(hd, H.H2SP_FP64)
        H.h2sp_refactor(hd)
        assert H.h2sp_query(hd)["factor_prec"] == H.H2SP_FP64
        info = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_GMRES, tol=1e-10, maxit=60, restart=20)
        assert info.status == H.H2SP_OK and info.rel_residual <= 1e-10
        torch.cuda.synchronize()
        err = np.linalg.norm(host(xt) - xd / 4.0) / np.linalg.norm(xd / 4.0)
        assert err <= 1e-7
    hd.close()


# ---------------------------------------------------------------------------
# log-determinant from the factors (§5.3)
# ---------------------------------------------------------------------------


def _logdet_terms(fa):
    """Sum of |log|u_jj|| over the oracle's pivots: the scale the rounding of the pivots is relative to."""
    return sum(float(np.sum(np.abs(np.log(np.abs(np.diag(lu)))))) for lu, _ in fa.lu)


@pytest.mark.parametrize("name", ["log1k", "skew1k", "inv3d", "tiny", "ragged"])
def test_logdet_matches_oracle(name):
    """log|det A| and sign(det S) from the GPU factors equal the oracle's.
    Both are invariants of S, so they agree whatever pivots each side chose.
    FP64 factors: within 1e-10 of the sum of the terms' magnitudes.  FP32
    factors: within 1e-5 of it; a dense FP32 getrf of the same S (LAPACK)
    stays within 4e-7 on these cases."""
    h, b, sp, hd = sparsified(name)
    fa = ofa.factor(h, sp)
    lo, so = ofa.logdet(fa)
    terms = max(1.0, _logdet_terms(fa))
    H.h2sp_factor(hd, H.H2SP_FP64)
    ld, sg = H.h2sp_logdet(hd)
    print("logdet %s: oracle %.12g, fp64 diff %.2e" % (name, lo, ld[0] - lo))
    assert ld.shape == (1,) and sg.shape == (1,)
    assert abs(ld[0] - lo) <= 1e-10 * terms
    assert sg[0] == so
    H.h2sp_factor(hd, H.H2SP_FP32)
    ld32, sg32 = H.h2sp_logdet(hd)
    print("logdet %s: fp32 diff %.2e" % (name, ld32[0] - lo))
    assert abs(ld32[0] - lo) <= 1e-5 * terms
    assert sg32[0] == so
    hd.close()


def test_logdet_per_system_of_a_forest():
    """Batched form: one value per independent system, each equal to the
    oracle's for that system alone."""
    systems, f, b = synth.make_batched(5, 500, 2500, leaf=32, tol=1e-8, nrhs=1)
    hd = H.h2sp_sparsify(H.H2Input(f))
    H.h2sp_factor(hd, H.H2SP_FP64)
    ld, sg = H.h2sp_logdet(hd)
    assert ld.shape == (len(systems),)
    for w, s in enumerate(systems):
        sp = osp.sparsify(s)
        fa = ofa.factor(s, sp)
        lo, so = ofa.logdet(fa)
        assert abs(ld[w] - lo) <= 1e-10 * max(1.0, _logdet_terms(fa))
        assert sg[w] == so
    hd.close()


# ---------------------------------------------------------------------------
# the small configurations of the workloads, as generated for the bench
# ---------------------------------------------------------------------------


def test_config_log2d_n4096_fp64_direct():
    """2D -log r, N = 4,096 uniform points, leaf <= 64, Chebyshev 4x4
    recompressed to 1e-8, one right-hand side: the FP64 path end to end (S
    pattern equal, S and Q blocks within 1e-10, the direct solve within 1e-10
    of the oracle's)."""
    h, b = synth.make_workload("log2d_n4096")
    sp = osp.sparsify(h)
    hd = H.h2sp_sparsify(H.H2Input(h))
    S = H.h2sp_export_S(hd)
    vbr = osp.to_vbr(sp)
    assert np.array_equal(S["node_size"], vbr.node_size)
    assert np.array_equal(S["brow_ptr"], vbr.brow_ptr) and np.array_equal(S["bcol_idx"], vbr.bcol_idx)
    ns = vbr.node_size
    for i in range(ns.size):
        lo, hi = int(vbr.brow_ptr[i]), int(vbr.brow_ptr[i + 1])
        if hi == lo:
            continue
        a, e = int(vbr.val_off[lo]), int(vbr.val_off[hi - 1] + ns[i] * ns[vbr.bcol_idx[hi - 1]])
        assert np.linalg.norm(S["vals"][a:e] - vbr.vals[a:e]) <= TOL * np.linalg.norm(vbr.vals[a:e])
    for t in sp.Q:
        assert np.linalg.norm(H.h2sp_export_Q(hd, t) - sp.Q[t]) <= TOL * np.linalg.norm(sp.Q[t]), t
    H.h2sp_factor(hd, H.H2SP_FP64)
    bt = dev(b)
    xt = torch.empty_like(bt)
    H.h2sp_solve(hd, bt, xt, mode=H.H2SP_DIRECT)
    torch.cuda.synchronize()
    xo = ofa.solve(h, sp, ofa.factor(h, sp), b)
    assert np.linalg.norm(host(xt) - xo) <= TOL * np.linalg.norm(xo)
    hd.close()


def test_batched_ellipses_fp32_refinement_and_graph_replay():
    """Batched form: 16 systems with N_k uniform in [2048, 8192] on random
    ellipses, leaf <= 64, tol 1e-6.  FP32 factors + FP64 refinement bring every
    system to 1e-10 (checked on each system's own oracle H^2 product); after the
    close blocks and couplings are doubled in place, h2sp_refactor (graph
    replay) and the same refinement bring the doubled systems to 1e-10."""
    systems, f, b = synth.make_batched(16, 2048, 8192, leaf=64, tol=1e-6, nrhs=2)
    inp = H.H2Input(f)
    hd = H.h2sp_sparsify(inp)
    H.h2sp_factor(hd, H.H2SP_FP32)
    bt = dev(b)
    xt = torch.empty_like(bt)
    mvs = [oh2.Matvec(s) for s in systems]
    for scale in (1.0, 2.0):
        if scale != 1.0:
            inp.dev["near_block"].mul_(scale)
            inp.dev["coupling"].mul_(scale)
            H.h2sp_refactor(hd)
        info = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_IR, tol=1e-10, maxit=30)
        assert info.status == H.H2SP_OK and info.rel_residual <= 1e-10
        torch.cuda.synchronize()
        xg = host(xt)
        o = 0
        for s, mv in zip(systems, mvs):
            bs = b[o:o + s.n]
            r = np.linalg.norm(bs - scale * mv(xg[o:o + s.n]), axis=0) / np.linalg.norm(bs, axis=0)
            assert r.max() <= 2e-10, (scale, o, r.max())
            o += s.n
    hd.close()


def test_batched_256_systems_persistent_form():
    """256 independent ellipse systems (N_k in [256, 1024]) in one forest: the
    persistent form (h2sp_refactor graph replay + FP64 refinement) brings every
    system to 1e-10 on its own oracle H^2 product, and the FP64 direct solve of
    sampled systems equals their oracle's."""
    systems, f, b = synth.make_batched(256, 256, 1024, leaf=64, tol=1e-6, nrhs=1)
    inp = H.H2Input(f)
    an = H.h2sp_analyze(H.H2Input(f, device=None))
    assert H.h2sp_query(an)["nsys"] == 256
    hd = H.h2sp_sparsify_analyzed(an, inp, flags=H.H2SP_SPARSIFY_FP32)
    H.h2sp_factor(hd, H.H2SP_FP32)
    bt = dev(b)
    xt = torch.empty_like(bt)
    for rep in range(2):
        if rep:
            H.h2sp_refactor(hd)
        info = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_IR, tol=1e-10, maxit=30)
        assert info.status == H.H2SP_OK and info.rel_residual <= 1e-10
    torch.cuda.synchronize()
    xg = host(xt)
    o = 0
    for s in systems:
        bs = b[o:o + s.n]
        r = np.linalg.norm(bs - oh2.Matvec(s)(xg[o:o + s.n])) / np.linalg.norm(bs)
        assert r <= 2e-10, (o, r)
        o += s.n
    # the captured refinement (one graph launch per call) after another refactorization
    H.h2sp_refactor(hd)
    xc = torch.empty_like(bt)
    for _ in range(2):
        info = H.h2sp_solve_captured(hd, bt, xc, steps=8)
        assert info.status == H.H2SP_OK and info.rel_residual <= 1e-10
    torch.cuda.synchronize()
    xg = host(xc)
    o = 0
    for s in systems:
        bs = b[o:o + s.n]
        assert np.linalg.norm(bs - oh2.Matvec(s)(xg[o:o + s.n])) <= 2e-10 * np.linalg.norm(bs)
        o += s.n
    hd.close()
    hd64 = H.h2sp_sparsify_analyzed(an, inp)
    H.h2sp_factor(hd64, H.H2SP_FP64)
    H.h2sp_solve(hd64, bt, xt, mode=H.H2SP_DIRECT)
    torch.cuda.synchronize()
    xg = host(xt)
    offs = np.cumsum([0] + [s.n for s in systems])
    for k in (0, 77, 255):
        s = systems[k]
        sp = osp.sparsify(s)
        xo = ofa.solve(s, sp, ofa.factor(s, sp), b[offs[k]:offs[k + 1]])
        assert np.linalg.norm(xg[offs[k]:offs[k + 1]] - xo) <= TOL * np.linalg.norm(xo)
    hd64.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_captured_refinement_replays_with_new_right_hand_sides(prec):
    """h2sp_solve_captured: the fixed-step refinement captured once and
    replayed; a new b written into the same buffer is solved by the replay
    (the sweeps' flags are reset inside the graph), and after a refactor with
    doubled numbers the replay uses the new factors."""
    h, b, sp, hd = sparsified("log4k")
    H.h2sp_factor(hd, H.H2SP_FP64 if prec == "fp64" else H.H2SP_FP32)
    A = oh2.dense(h)
    bt = dev(b)
    xt = torch.empty_like(bt)
    steps = 1 if prec == "fp64" else 8
    for rep in range(3):
        if rep:
            bt.copy_(dev(np.random.default_rng(50 + rep).standard_normal(b.shape)))
        info = H.h2sp_solve_captured(hd, bt, xt, steps=steps)
        assert info.status == H.H2SP_OK and info.rel_residual <= 1e-10, (rep, info.rel_residual)
        torch.cuda.synchronize()
        bh = host(bt)
        r = np.linalg.norm(bh - A @ host(xt), axis=0) / np.linalg.norm(bh, axis=0)
        assert r.max() <= 2e-10
    # the same numbers doubled, refactored: the replay solves 2A x = b
    inp = hd.inp
    inp.dev["near_block"].mul_(2.0)
    inp.dev["coupling"].mul_(2.0)
    H.h2sp_refactor(hd)
    info = H.h2sp_solve_captured(hd, bt, xt, steps=steps)
    assert info.status == H.H2SP_OK and info.rel_residual <= 1e-10
    torch.cuda.synchronize()
    bh = host(bt)
    assert np.linalg.norm(bh - 2.0 * A @ host(xt)) <= 2e-10 * np.linalg.norm(bh) * np.sqrt(b.shape[1])
    inp.dev["near_block"].mul_(0.5)
    inp.dev["coupling"].mul_(0.5)
    hd.close()
