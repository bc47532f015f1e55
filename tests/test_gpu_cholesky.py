"""GPU block Cholesky (h2sp_factor with H2SP_FP64_CHOL / H2SP_FP32_CHOL)
against the oracle's block Cholesky (oracle.factor.cholesky), through the C ABI.

For a symmetric positive definite S the Cholesky factor is unique, so the
GPU factor is compared element by element: per supernode, the factored front
(stored in the LU form, unit L and U = D L^T) gives L_chol = L D^1/2, whose
first s columns must equal the oracle's [L11; L21] within 1e-10 of their
norm (FP64).  Also within the FP64 bars of the LU path: the direct solve,
S^-1 and log det S.  The FP32 factor preconditions GMRES to 1e-10 on the FP64
H^2 product, and one FP32 direct solve stays within a small factor of a dense
FP32 LAPACK Cholesky of the same matrix.  An indefinite S (the -log r kernel)
is reported as a non-positive pivot.

Cases: the Gaussian kernel with 2 on the diagonal (§5.2's SPD example) in 2D,
ragged 2D and 3D, and 1/r on the jittered Fibonacci sphere (blocks above 64
rows, fronts of several 256-column outer blocks).
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
    "gauss1k": dict(n=1024, kernel="gauss", leaf=32, tol=1e-8, seed=4),
    "gauss_ragged": dict(n=3001, kernel="gauss", leaf=23, tol=1e-8, seed=8),
    "gauss3d": dict(n=2000, kernel="gauss", leaf=40, tol=1e-8, seed=6, dim=3),
    "sphere8k": dict(workload="inv3d_sphere_n262144", n=8192),
}
_cache = {}


def case(name):
    if name not in _cache:
        c = _CASES[name]
        if "workload" in c:
            h, _ = synth.make_workload(c["workload"], n=c["n"])
        else:
            h, _ = synth.make_small(c["n"], kernel=c["kernel"], leaf=c["leaf"], tol=c["tol"], seed=c["seed"],
                                    dim=c.get("dim", 2), nrhs=3)
        b = np.random.default_rng(21).standard_normal((h.n, 3))
        sp = osp.sparsify(h)
        _cache[name] = (h, b, sp, ofa.cholesky(h, sp))
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


def chol_of_front(F, s):
    """L_chol's first s columns from a front in the LU form (unit L, U = D L^T)."""
    d = np.sqrt(np.diag(F)[:s])
    L = np.tril(F[:, :s], -1)
    L[np.arange(s), np.arange(s)] = 1.0
    return L * d[None, :]


@pytest.mark.parametrize("name", list(_CASES))
def test_fp64_cholesky_factor_matches_oracle(name):
    h, b, sp, ch = case(name)
    hd = H.h2sp_sparsify(H.H2Input(h))
    H.h2sp_factor(hd, H.H2SP_FP64_CHOL)
    q = H.h2sp_query(hd)
    assert q["factor_chol"] == 1 and q["nsupernodes"] == len(ch.L11)
    for k in range(q["nsupernodes"]):
        F, s = H.h2sp_export_front(hd, k)
        ref = np.vstack([ch.L11[k], ch.L21[k]]) if ch.L21[k].size else ch.L11[k]
        assert F.shape[0] == ref.shape[0] and s == ref.shape[1], k
        got = chol_of_front(F, s)
        assert np.linalg.norm(got - ref) <= TOL * np.linalg.norm(ref), (k, np.linalg.norm(got - ref))
    hd.close()


@pytest.mark.parametrize("name", list(_CASES))
def test_fp64_cholesky_solve_and_logdet(name):
    h, b, sp, ch = case(name)
    hd = H.h2sp_sparsify(H.H2Input(h))
    H.h2sp_factor(hd, H.H2SP_FP64_CHOL)
    bt = dev(b)
    xt = torch.empty_like(bt)
    H.h2sp_solve(hd, bt, xt, mode=H.H2SP_DIRECT)
    torch.cuda.synchronize()
    c = osp.apply_T(sp, h, b, col=False)
    xo = osp.apply_N(sp, h, ofa.solve_S_chol(ch, c), col=True)
    assert np.linalg.norm(host(xt) - xo) <= TOL * np.linalg.norm(xo)
    # S^-1 itself, on the S-space vector
    ct = dev(c)
    yt = torch.empty_like(ct)
    H.h2sp_apply(hd, H.H2SP_OP_SINV, ct, yt)
    torch.cuda.synchronize()
    yo = ofa.solve_S_chol(ch, c)
    assert np.linalg.norm(host(yt) - yo) <= TOL * np.linalg.norm(yo)
    ld, sign = H.h2sp_logdet(hd)
    ref = ofa.logdet_chol(ch)
    scale = 2.0 * sum(float(np.sum(np.abs(np.log(np.diag(L))))) for L in ch.L11)
    assert abs(ld[0] - ref) <= TOL * scale and sign[0] == 1
    hd.close()


@pytest.mark.parametrize("name", list(_CASES))
def test_fp32_cholesky_preconditions_gmres_to_1e10(name):
    h, b, sp, ch = case(name)
    hd = H.h2sp_sparsify(H.H2Input(h), flags=H.H2SP_SPARSIFY_FP32)
    H.h2sp_factor(hd, H.H2SP_FP32_CHOL)
    bt = dev(b)
    xt = torch.empty_like(bt)
    info = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_GMRES, tol=1e-10, maxit=60, restart=20)
    assert info.status == H.H2SP_OK and info.rel_residual <= 1e-10
    torch.cuda.synchronize()
    r = np.linalg.norm(b - oh2.Matvec(h)(host(xt)), axis=0) / np.linalg.norm(b, axis=0)
    assert r.max() <= 2e-10
    hd.close()


@pytest.mark.parametrize("name", ["gauss1k", "gauss_ragged", "gauss3d"])
def test_fp32_cholesky_direct_accuracy(name):
    """One FP32 block-Cholesky direct solve is accurate to a small multiple of
    a dense FP32 LAPACK Cholesky of the same matrix."""
    import scipy.linalg as sl
    h, b, sp, ch = case(name)
    hd = H.h2sp_sparsify(H.H2Input(h))
    H.h2sp_factor(hd, H.H2SP_FP32_CHOL)
    bt = dev(b)
    xt = torch.empty_like(bt)
    H.h2sp_solve(hd, bt, xt, mode=H.H2SP_DIRECT)
    torch.cuda.synchronize()
    A = oh2.dense(h)
    xd = np.linalg.solve(A, b)
    err = np.linalg.norm(host(xt) - xd) / np.linalg.norm(xd)
    c32 = sl.cho_factor(A.astype(np.float32), lower=True)
    x32 = sl.cho_solve(c32, b.astype(np.float32)).astype(np.float64)
    err32 = np.linalg.norm(x32 - xd) / np.linalg.norm(xd)
    print("%s: block Cholesky FP32 %.2e, dense FP32 %.2e" % (name, err, err32))
    assert err <= 25.0 * max(err32, 1e-7)
    hd.close()


def test_cholesky_reports_indefinite_S():
    """-log r in the unit square (diameter sqrt 2 > 1): S is indefinite, the
    oracle's Cholesky refuses it, and so must the GPU's."""
    h, _ = synth.make_small(1024, kernel="log", leaf=32, tol=1e-8, seed=1, nrhs=1)
    sp = osp.sparsify(h)
    with pytest.raises(np.linalg.LinAlgError):
        ofa.cholesky(h, sp)
    hd = H.h2sp_sparsify(H.H2Input(h))
    with pytest.raises(H.H2spError) as e:
        H.h2sp_factor(hd, H.H2SP_FP64_CHOL)
    assert e.value.status == H.H2SP_ESINGULAR
    # the handle factors again with the LU afterwards
    H.h2sp_factor(hd, H.H2SP_FP64)
    hd.close()


def test_cholesky_rejects_column_bases():
    h, _ = synth.make_small(1024, kernel="log_skew", leaf=32, tol=1e-8, seed=2, nrhs=1)
    hd = H.h2sp_sparsify(H.H2Input(h))
    with pytest.raises(H.H2spError) as e:
        H.h2sp_factor(hd, H.H2SP_FP32_CHOL)
    assert e.value.status == H.H2SP_EINVAL
    hd.close()


def test_cholesky_then_lu_then_cholesky_same_handle():
    """Switching factorizations on one handle: the FP32 Cholesky, the FP64 LU
    (the front buffer grows) and the FP32 Cholesky again solve alike."""
    h, b, sp, ch = case("gauss1k")
    hd = H.h2sp_sparsify(H.H2Input(h))
    bt = dev(b)
    xs = []
    for prec in (H.H2SP_FP32_CHOL, H.H2SP_FP64, H.H2SP_FP32_CHOL):
        H.h2sp_factor(hd, prec)
        xt = torch.empty_like(bt)
        info = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_IR, tol=1e-10, maxit=30)
        assert info.status == H.H2SP_OK and info.rel_residual <= 1e-10
        xs.append(host(xt))
    assert np.linalg.norm(xs[0] - xs[2]) <= 1e-9 * np.linalg.norm(xs[1])
    hd.close()


def test_schedules_give_the_same_factor():
    """Every candidate schedule of the autotuner (128 x 128 or 128 x 256
    tiles and tiles per CTA of the block-end update, SMs left to the panel
    stream, look-ahead) factors S to
    the same L up to FP32 rounding order, and the tuner returns one of them."""
    from paper_1705_04601_gb300 import tune as T
    h, b, sp, ch = case("sphere8k")
    an = H.h2sp_analyze(H.H2Input(h, device=None))
    inp = H.H2Input(h)
    ref = None
    for sched in [T.DEFAULT, {"tiles_per_cta": 8, "panel_sms": 16, "lookahead": 1},
                  {"tiles_per_cta": 32, "panel_sms": 8, "lookahead": 0}, dict(T.DEFAULT, wide=0),
                  dict(T.DEFAULT, wide=2), {"tiles_per_cta": 3, "panel_sms": 8, "lookahead": 1, "wide": 1},
                  {"tiles_per_cta": 5, "panel_sms": 16, "lookahead": 1, "wide": 2}]:
        hd = H.h2sp_sparsify_analyzed(an, inp)
        T.apply(hd, sched)
        H.h2sp_factor(hd, H.H2SP_FP32_CHOL)
        # the entries a factored front defines: its factored columns, the U12
        # rows and the lower triangle of the contribution block (the rest of
        # the front is work space, which the schedules may leave differently)
        F = []
        for k in range(len(ch.L11)):
            Fk, s = H.h2sp_export_front(hd, k)
            F.append(np.concatenate([Fk[:, :s].ravel(), Fk[:s, s:].ravel(), np.tril(Fk[s:, s:]).ravel()]))
        if ref is None:
            ref = F
        else:
            for a, r in zip(F, ref):
                assert np.linalg.norm(a - r) <= 1e-5 * np.linalg.norm(r)
        hd.close()
    sched, ms = T.tune(an, inp, flags=0, repeats=1)
    assert ms > 0 and set(sched) == set(T.DEFAULT)
    assert all(sched[n] in T.CANDIDATES[n] for n in sched)


@pytest.mark.parametrize("name", ["gauss3d", "sphere8k"])
@pytest.mark.parametrize("prec,bound", [("H2SP_BF16_CHOL", 1e-2), ("H2SP_BF16X3_CHOL", 2e-4)])
def test_bf16_cholesky_preconditions_gmres_to_1e10(name, prec, bound):
    """H2SP_BF16_CHOL: the block-end updates in BF16 with a power-of-two scale
    per 128-row tile of L21 (FP32 accumulation); H2SP_BF16X3_CHOL: the same
    with each scaled entry split into a BF16 hi and lo part and three BF16
    products.  The factor is an approximation of the FP64 one -- its error
    against the oracle's factor is printed and bounded (8 significant bits:
    1e-2; about 16: 2e-4) -- and it preconditions FP64 GMRES to 1e-10."""
    h, b, sp, ch = case(name)
    hd = H.h2sp_sparsify(H.H2Input(h), flags=H.H2SP_SPARSIFY_FP32)
    H.h2sp_factor(hd, getattr(H, prec))
    q = H.h2sp_query(hd)
    num = den = 0.0
    for k in range(q["nsupernodes"]):
        F, s = H.h2sp_export_front(hd, k)
        ref = np.vstack([ch.L11[k], ch.L21[k]]) if ch.L21[k].size else ch.L11[k]
        num += np.linalg.norm(chol_of_front(F, s) - ref) ** 2
        den += np.linalg.norm(ref) ** 2
    rel = np.sqrt(num / den)
    print("%s: %s factor vs the FP64 oracle: %.2e" % (name, prec, rel))
    assert rel <= bound
    bt = dev(b)
    xt = torch.empty_like(bt)
    info = H.h2sp_solve(hd, bt, xt, mode=H.H2SP_GMRES, tol=1e-10, maxit=100, restart=30)
    print("%s: GMRES steps %d" % (name, info.iters))
    assert info.status == H.H2SP_OK and info.rel_residual <= 1e-10
    torch.cuda.synchronize()
    r = np.linalg.norm(b - oh2.Matvec(h)(host(xt)), axis=0) / np.linalg.norm(b, axis=0)
    assert r.max() <= 2e-10
    hd.close()
