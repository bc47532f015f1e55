"""GPU construction of the H^2 matrix (h2sp_construct): the interpolation
parameters and close blocks against the host generator's (same formulas,
rounding-level agreement), the recompressed matrix against the kernel matrix
itself (error at the tolerance, like the host generator's), and the
sparsify / factor / GMRES path run on the GPU-built matrix."""
import numpy as np
import pytest

from paper_1705_04601_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_04601_gb300 import h2sp as H  # noqa: E402
from oracle import h2 as oh2  # noqa: E402

_CASES = {
    # name: (points maker, kernel, leaf, order)
    "log2d": (lambda: (np.random.default_rng(11).random((2048, 2)), np.zeros(2), np.ones(2)), "log", 32, 4),
    "sphere3d": (lambda: synth.workload_points("inv3d_sphere_n262144", n=4096)[:3], "inv", 64, 4),
    "yukawa3d": (lambda: (np.random.default_rng(12).random((3000, 3)), np.zeros(3), np.ones(3)), "yukawa", 64, 3),
    "gauss3d": (lambda: (np.random.default_rng(13).random((2000, 3)), np.zeros(3), np.ones(3)), "gauss", 40, 4),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1705_04601_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA is required for the gpu tests")


def _gpu(name, tol):
    mk, kernel, leaf, p = _CASES[name]
    pts, lo, hi = mk()
    diag = synth.default_diag(kernel, pts.shape[0], pts.shape[1])
    tree, tp = synth.tree_arrays(pts, leaf, lo, hi)
    c = H.h2sp_construct(tree, torch.from_numpy(tp).cuda(), kernel, diag, order=p, tol=tol)
    return c, tree, tp, (pts, kernel, leaf, p, lo, hi, diag)


def _as_h2(c, tree, tp, kernel, diag):
    """The GPU-built matrix as the host container (numbers copied back)."""
    d = c.desc()
    ncl = tree["parent"].size
    nleaf = int(tree["level_ptr"][tree["depth"] + 1] - tree["level_ptr"][tree["depth"]])
    nfar, nnear = int(tree["far_ptr"][-1]), int(tree["near_ptr"][-1])
    arr = lambda p, n, t: np.ctypeslib.as_array(p, shape=(n,)).astype(t).copy()
    return synth.H2Matrix(
        n=int(d.n), dim=tp.shape[1], depth=int(d.depth), level_ptr=tree["level_ptr"], parent=tree["parent"],
        begin=tree["begin"], size=tree["size"], rank=arr(d.rank, ncl, np.int32),
        leaf_basis=c.copy(0), leaf_basis_off=arr(d.leaf_basis_off, nleaf, np.int64),
        transfer=c.copy(1), transfer_off=arr(d.transfer_off, ncl, np.int64),
        far_ptr=tree["far_ptr"], far_col=tree["far_col"], coupling=c.copy(2),
        coupling_off=arr(d.coupling_off, max(nfar, 1), np.int64)[:nfar],
        near_ptr=tree["near_ptr"], near_col=tree["near_col"], near_block=c.copy(3),
        near_off=arr(d.near_off, nnear, np.int64), points=tp, kernel=kernel, diag=float(diag))


@pytest.mark.parametrize("name", list(_CASES))
def test_raw_interpolation_matches_host_generator(name):
    c, tree, tp, (pts, kernel, leaf, p, lo, hi, diag) = _gpu(name, 0.0)
    h = synth.build_h2(pts, kernel, leaf, p=p, tol=None, lo=lo, hi=hi, diag=diag)
    g = _as_h2(c, tree, tp, kernel, diag)
    assert np.array_equal(g.rank, h.rank)
    for k in ("leaf_basis_off", "transfer_off", "coupling_off", "near_off"):
        assert np.array_equal(getattr(g, k), getattr(h, k)), k
    for k in ("leaf_basis", "transfer", "coupling", "near_block"):
        a, b = getattr(g, k), getattr(h, k)
        assert a.shape == b.shape, k
        assert np.max(np.abs(a - b)) <= 1e-12 * max(np.max(np.abs(b)), 1.0), (k, np.max(np.abs(a - b)))
    c.close()


@pytest.mark.parametrize("name", ["log2d", "sphere3d", "yukawa3d"])
def test_recompressed_matrix_is_within_tolerance(name):
    tol = 1e-6
    c, tree, tp, (pts, kernel, leaf, p, lo, hi, diag) = _gpu(name, tol)
    g = _as_h2(c, tree, tp, kernel, diag)
    h = synth.build_h2(pts, kernel, leaf, p=p, tol=tol, lo=lo, hi=hi, diag=diag)
    # the kernel matrix itself, in tree order
    A = synth.KERNELS[kernel](tp, tp)
    np.fill_diagonal(A, diag)
    nA = np.linalg.norm(A)
    eg = np.linalg.norm(oh2.dense(g) - A) / nA
    eh = np.linalg.norm(oh2.dense(h) - A) / nA
    # the raw interpolation, for scale
    print("%s: GPU recompressed %.2e, host recompressed %.2e; ranks %d / %d" % (
        name, eg, eh, int(g.rank.sum()), int(h.rank.sum())))
    assert eg <= 3.0 * eh + 1e-12
    # the same ranks up to ties at the threshold
    diff = np.abs(g.rank.astype(int) - h.rank.astype(int))
    assert diff.max() <= 2 and np.count_nonzero(diff) <= max(2, g.rank.size // 50)
    # orthonormal leaf bases
    for lf in range(g.nleaf):
        t = int(g.level_ptr[g.depth]) + lf
        k, m = int(g.rank[t]), int(g.size[t])
        if k == 0:
            continue
        R = g.leaf_basis[g.leaf_basis_off[lf]:g.leaf_basis_off[lf] + m * k].reshape(k, m).T
        assert np.linalg.norm(R.T @ R - np.eye(k)) <= 1e-12
    c.close()


def test_gpu_built_matrix_solves_to_1e10():
    """sphere N = 8,192: built on the GPU (Chebyshev 4^3, tol 1e-6), sparsified,
    FP32 block Cholesky, GMRES on its FP64 H^2 product to 1e-10; the residual
    is checked with the host H^2 product of the same (GPU-built) matrix."""
    pts, lo, hi, cfg = synth.workload_points("inv3d_sphere_n262144", n=8192)
    diag = synth.default_diag("inv", pts.shape[0], 3)
    tree, tp = synth.tree_arrays(pts, cfg["leaf"], lo, hi)
    c = H.h2sp_construct(tree, torch.from_numpy(tp).cuda(), "inv", diag, order=4, tol=cfg["tol"])
    hd = H.h2sp_sparsify(c, flags=H.H2SP_SPARSIFY_FP32)
    H.h2sp_factor(hd, H.H2SP_FP32_CHOL)
    b = np.random.default_rng(3).standard_normal((tp.shape[0], 1))
    bt = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()
    xt = torch.empty_like(bt)
    info = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_GMRES, tol=1e-10, maxit=60, restart=20)
    assert info.status == H.H2SP_OK and info.rel_residual <= 1e-10
    torch.cuda.synchronize()
    g = _as_h2(c, tree, tp, "inv", diag)
    x = xt.cpu().numpy().T
    r = np.linalg.norm(b - oh2.Matvec(g)(x)) / np.linalg.norm(b)
    assert r <= 2e-10
    hd.close()
    c.close()


def test_construct_rejects_bad_arguments():
    mk, kernel, leaf, p = _CASES["log2d"]
    pts, lo, hi = mk()
    tree, tp = synth.tree_arrays(pts, leaf, lo, hi)
    x = torch.from_numpy(tp).cuda()
    for kw in (dict(order=9), dict(tol=1e-9)):
        args = dict(order=4, tol=0.0)
        args.update(kw)
        with pytest.raises(H.H2spError) as e:
            H.h2sp_construct(tree, x, "log", 1.0, **args)
        assert e.value.status == H.H2SP_EINVAL
    bad = dict(tree)
    bad["far_col"] = bad["far_col"].copy()
    if bad["far_col"].size:
        bad["far_col"][0] = tree["parent"].size + 5
        with pytest.raises(H.H2spError) as e:
            H.h2sp_construct(tree | {"far_col": bad["far_col"]}, x, "log", 1.0)
        assert e.value.status == H.H2SP_EINVAL
