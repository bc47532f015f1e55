"""Pins of the CPU oracle against what the paper and the mathematics fix.

No GPU.  Each pin is chosen so that a plausible slip in the oracle (a dropped
term, a wrong sign or index, a transposed operand, a wrong permutation) fails
at least one of them:

* Householder completion vs LAPACK's QR (scipy), plus closed forms;
* U, V orthogonal and built from block-diagonal and permutation factors
  (§1, Eq. main_uv);
* S equals U^T A V computed densely and U S V^T equals A (exactness of the
  sparsification, §5 "does not worsen the accuracy");
* the block pattern of S follows the rule of §3 and U^T A V vanishes outside it;
* symmetric A gives U = V and symmetric S; SPD A gives SPD S (Proposition 2.1);
* the block LU solve agrees with dense LAPACK solves of S and of A;
* the symbolic elimination agrees with brute-force boolean elimination;
* the number of nonzeros per row of S stays bounded as N grows (§5.1);
* IR / GMRES with the factored S reach 1e-10 (§5.5);
* log|det A| from the pivots of S equals LAPACK's slogdet of the dense A and
  of the dense S, with the sign of det S (§5.3);
* the threshold incomplete LU (ILUt) of §5.5 matches a hand-worked example,
  is the exact LU without dropping, keeps no entry below its row threshold,
  and preconditions §5.5's example as the paper describes;
* the block Cholesky of an SPD S reproduces S, equals LAPACK's dense
  Cholesky factor of S in elimination order (the factor is unique), solves
  like a dense solve, and refuses an indefinite S.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from paper_1705_04601_gb300 import synth
from oracle import factor as ofa
from oracle import h2 as oh2
from oracle import householder as ohh
from oracle import ilu as oilu
from oracle import iterate as oit
from oracle import sparsify as osp

_CACHE = {}


def case(name):
    if name in _CACHE:
        return _CACHE[name]
    spec = {
        "log1k": dict(n=1024, kernel="log", leaf=32, tol=1e-8, seed=1),
        "log4k": dict(n=4096, kernel="log", leaf=64, tol=1e-8, seed=1),
        "skew1k": dict(n=1024, kernel="log_skew", leaf=32, tol=1e-8, seed=2),
        "raw1k": dict(n=1024, kernel="log", leaf=32, tol=None, seed=3),
        "gauss1k": dict(n=1024, kernel="gauss", leaf=32, tol=1e-8, seed=4),
        "inv3d": dict(n=1500, kernel="inv", leaf=40, tol=1e-6, seed=5, dim=3),
        "tiny": dict(n=48, kernel="log", leaf=64, tol=1e-8, seed=6),
        "small": dict(n=256, kernel="log", leaf=16, tol=1e-8, seed=7),
        "gauss3d": dict(n=1500, kernel="gauss", leaf=40, tol=1e-8, seed=10, dim=3),
        # 3D leaves above 64 points (octree leaf <= 128), as the streaming kernels take them
        "yukawa3d": dict(n=3000, kernel="yukawa", leaf=128, tol=1e-6, seed=13, dim=3),
    }[name]
    h, b = synth.make_small(spec["n"], kernel=spec["kernel"], leaf=spec["leaf"], tol=spec["tol"],
                            seed=spec["seed"], dim=spec.get("dim", 2), nrhs=2)
    sp = osp.sparsify(h)
    A = oh2.dense(h)
    _CACHE[name] = (h, b, sp, A)
    return _CACHE[name]


# --------------------------------------------------------------------------
# Householder completion (§4.2)
# --------------------------------------------------------------------------


@pytest.mark.parametrize("m,k", [(16, 5), (40, 16), (7, 7), (5, 9), (30, 1), (12, 0)])
def test_householder_matches_lapack(m, k):
    rng = np.random.default_rng(m * 100 + k)
    W = rng.standard_normal((m, k))
    Q, Rr = ohh.householder_complete(W)
    kp = min(m, k)
    assert Q.shape == (m, m) and Rr.shape == (kp, k)
    assert np.abs(Q.T @ Q - np.eye(m)).max() < 1e-14
    assert np.abs(Q[:, :kp] @ Rr - W).max(initial=0.0) < 1e-13 * max(1.0, np.abs(W).max(initial=0.0))
    if k:
        Ql, Rl = sla.qr(W, mode="full")          # dgeqrf + dorgqr
        assert np.abs(Ql - Q).max() < 1e-13
        assert np.abs(Rl[:kp] - Rr).max() < 1e-13


def test_householder_closed_forms():
    # one column (3, 4): beta = -5, v = (1, 0.5), tau = 1.6
    Q, Rr = ohh.householder_complete(np.array([[3.0], [4.0]]))
    assert np.allclose(Rr, [[-5.0]], atol=1e-15)
    assert np.allclose(Q, [[-0.6, -0.8], [-0.8, 0.6]], atol=1e-15)
    # a column that is already e1 * alpha leaves H = I (tau = 0)
    Q, Rr = ohh.householder_complete(np.array([[-2.0], [0.0], [0.0]]))
    assert np.array_equal(Q, np.eye(3)) and Rr[0, 0] == -2.0
    # zero alpha takes sign(0) = +1, i.e. beta = -||x||
    Q, Rr = ohh.householder_complete(np.array([[0.0], [2.0]]))
    assert np.isclose(Rr[0, 0], -2.0)


# --------------------------------------------------------------------------
# sparsification A = U S V^T (§2, §4)
# --------------------------------------------------------------------------

CASES = ["log1k", "log4k", "skew1k", "raw1k", "gauss1k", "inv3d", "small", "tiny", "yukawa3d"]


@pytest.mark.parametrize("name", CASES)
def test_factors_orthogonal_and_exact(name):
    h, b, sp, A = case(name)
    n = h.n
    U = osp.apply_N(sp, h, np.eye(n), col=False)
    V = osp.apply_N(sp, h, np.eye(n), col=True)
    assert np.abs(U.T @ U - np.eye(n)).max() < 1e-13
    assert np.abs(V.T @ V - np.eye(n)).max() < 1e-13
    S = osp.dense_S(sp)
    nA = np.linalg.norm(A)
    assert np.linalg.norm(S - U.T @ A @ V) / nA < 1e-12
    assert np.linalg.norm(U @ S @ V.T - A) / nA < 1e-12
    # applies agree with the explicit matrices
    assert np.abs(osp.apply_T(sp, h, b, col=False) - U.T @ b).max() < 1e-12 * np.abs(b).max()
    assert np.abs(osp.apply_T(sp, h, b, col=True) - V.T @ b).max() < 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("name", ["log1k", "skew1k", "small"])
def test_U_is_block_diagonal_times_permutation(name):
    """Column j of U (an entry of S node (l, t)) is supported on cluster t's points only."""
    h, b, sp, A = case(name)
    sch = sp.sch
    U = osp.apply_N(sp, h, np.eye(h.n), col=False)
    for v in range(sch.node_size.size):
        t = int(sch.node_cluster[v])
        lo, hi = int(h.begin[t]), int(h.begin[t] + h.size[t])
        cols = U[:, sch.node_off[v]:sch.node_off[v + 1]]
        assert np.abs(cols[:lo]).max(initial=0.0) == 0.0
        assert np.abs(cols[hi:]).max(initial=0.0) == 0.0


@pytest.mark.parametrize("name", ["log1k", "log4k", "skew1k", "inv3d", "small", "yukawa3d"])
def test_pattern_rule(name):
    h, b, sp, A = case(name)
    sch = sp.sch
    pat = osp.pattern_rule(h, sch)
    assert pat == set(sp.blocks.keys())
    # U^T A V vanishes outside the predicted pattern
    U = osp.apply_N(sp, h, np.eye(h.n), col=False)
    V = osp.apply_N(sp, h, np.eye(h.n), col=True)
    Sd = U.T @ A @ V
    mask = np.zeros_like(Sd, dtype=bool)
    for (i, j) in pat:
        mask[sch.node_off[i]:sch.node_off[i + 1], sch.node_off[j]:sch.node_off[j + 1]] = True
    assert np.abs(Sd[~mask]).max(initial=0.0) <= 1e-13 * np.abs(A).max()
    # and the pattern is not trivially dense: fewer than half of the node pairs
    nn = sch.node_size.size
    if h.n >= 4096 and h.dim == 2:
        assert len(pat) < 0.5 * nn * nn


def test_symmetric_gives_U_equal_V_and_symmetric_S():
    h, b, sp, A = case("log1k")
    assert all(np.array_equal(sp.Q[t], sp.Qc[t]) for t in sp.Q)
    S = osp.dense_S(sp)
    assert np.abs(S - S.T).max() < 1e-12 * np.abs(S).max()


def test_spd_gives_spd_S():
    h, b, sp, A = case("gauss1k")
    S = osp.dense_S(sp)
    Ss = 0.5 * (S + S.T)
    assert np.abs(S - S.T).max() < 1e-12 * np.abs(S).max()
    np.linalg.cholesky(Ss)      # raises if S is not positive definite
    assert np.linalg.eigvalsh(Ss).min() > 0


def test_no_far_field_keeps_A():
    h, b, sp, A = case("tiny")
    assert sp.sch.lstop == 0
    assert np.array_equal(osp.dense_S(sp), A)


def test_sizes_add_up():
    h, b, sp, A = case("log4k")
    sch = sp.sch
    assert int(sch.node_off[-1]) == h.n
    for l in range(sch.lstop):
        for t in sch.clusters[l]:
            assert sch.kp[t] == min(h.rank[t], sch.m[t])
            assert sch.d[t] == sch.m[t] - sch.kp[t]


def test_nnz_per_row_bounded_in_n():
    """§5.1: the number of nonzeros per row of S does not grow with N."""
    per_row = []
    for n in (1024, 4096, 16384):
        h, _ = synth.make_small(n, kernel="log", leaf=32, tol=1e-6, seed=11)
        sp = osp.sparsify(h)
        nnz = sum(v.size for v in sp.blocks.values())
        per_row.append(nnz / n)
    assert per_row[2] < 1.5 * per_row[1] and per_row[1] < 1.5 * per_row[0] + 200


def test_vbr_roundtrip():
    h, b, sp, A = case("log1k")
    vbr = osp.to_vbr(sp)
    S = osp.dense_S(sp)
    no = vbr.node_off
    for i in range(vbr.node_size.size):
        for z in range(int(vbr.brow_ptr[i]), int(vbr.brow_ptr[i + 1])):
            j = int(vbr.bcol_idx[z])
            r, c = int(vbr.node_size[i]), int(vbr.node_size[j])
            blk = vbr.vals[vbr.val_off[z]:vbr.val_off[z] + r * c].reshape(c, r).T
            assert np.array_equal(blk, S[no[i]:no[i + 1], no[j]:no[j + 1]])
        cols = vbr.bcol_idx[vbr.brow_ptr[i]:vbr.brow_ptr[i + 1]]
        assert np.all(np.diff(cols) > 0)


# --------------------------------------------------------------------------
# H^2 definition
# --------------------------------------------------------------------------


@pytest.mark.parametrize("name", ["log1k", "skew1k", "inv3d"])
def test_h2_approximates_kernel_and_matvec(name):
    h, b, sp, A = case(name)
    K = synth.KERNELS[h.kernel](h.points, h.points)
    np.fill_diagonal(K, h.diag)
    assert np.linalg.norm(A - K) / np.linalg.norm(K) < 1e-3
    mv = oh2.Matvec(h)
    assert np.linalg.norm(mv(b) - A @ b) / np.linalg.norm(A @ b) < 1e-13


# --------------------------------------------------------------------------
# ordering, symbolic and numeric block LU, solve (Eq. sp0)
# --------------------------------------------------------------------------


@pytest.mark.parametrize("name", ["log1k", "log4k", "skew1k", "raw1k", "inv3d", "small", "tiny", "yukawa3d"])
def test_block_lu_solve_matches_dense(name):
    h, b, sp, A = case(name)
    fa = ofa.factor(h, sp)
    c = osp.apply_T(sp, h, b)
    y = ofa.solve_S(fa, c)
    S = osp.dense_S(sp)
    yd = np.linalg.solve(S, c)
    assert np.linalg.norm(y - yd) / np.linalg.norm(yd) < 1e-10
    x = ofa.solve(h, sp, fa, b)
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-10


@pytest.mark.parametrize("name", ["small", "log1k", "skew1k"])
def test_symbolic_matches_boolean_elimination(name):
    """Boundary sets equal the structure of brute-force boolean elimination."""
    h, b, sp, A = case(name)
    sym = ofa.symbolic(h, sp)
    nn = sp.sch.node_size.size
    G = np.zeros((nn, nn), dtype=bool)
    for (i, j) in sp.blocks:
        G[i, j] = G[j, i] = True
    pos = np.empty(nn, dtype=np.int64)
    pos[sym.order] = np.arange(nn)
    P = G[np.ix_(sym.order, sym.order)].copy()
    for v in range(nn):                      # node-by-node elimination
        nb = np.nonzero(P[v, v + 1:])[0] + v + 1
        P[np.ix_(nb, nb)] = True
    for k in range(sym.sn_ptr.size - 1):
        lo, hi = int(sym.sn_ptr[k]), int(sym.sn_ptr[k + 1])
        later = set(np.nonzero(P[lo:hi, hi:].any(axis=0))[0] + hi)
        assert later == set(int(pos[w]) for w in sym.boundary[k])


@pytest.mark.parametrize("name", ["log1k", "log4k", "inv3d"])
def test_closure_nested_dissection(name):
    """Nodes coupled in S (or by fill) have closures on one root path, and
    same-depth supernodes never touch each other's boundaries."""
    h, b, sp, A = case(name)
    sym = ofa.symbolic(h, sp)
    dep = ofa._depths(h)

    def comparable(a, b_):
        return ofa.lca(h, dep, a, b_) in (a, b_)
    for (i, j) in sp.blocks:
        assert comparable(sym.closure[i], sym.closure[j])
    for k in range(sym.sn_ptr.size - 1):
        for w in sym.boundary[k]:
            assert comparable(sym.sn_closure[k], sym.closure[w])
            assert dep[sym.closure[w]] < sym.sn_depth[k]


def test_singular_pivot_block_is_reported():
    h, b, sp, A = case("small")
    sym = ofa.symbolic(h, sp)
    v = int(sym.order[0])
    bad = dict(sp.blocks)
    bad[(v, v)] = np.zeros_like(bad[(v, v)])
    for key in list(bad):
        if v in key:
            bad[key] = np.zeros_like(bad[key])
    sp2 = osp.Sparsified(sp.sch, sp.Q, sp.Qc, sp.Rr, sp.Rrc, bad)
    with pytest.raises(np.linalg.LinAlgError):
        ofa.factor(h, sp2, sym)


# --------------------------------------------------------------------------
# iterative solves (§5.5)
# --------------------------------------------------------------------------


# --------------------------------------------------------------------------
# log-determinant from the block LU (§5.3)
# --------------------------------------------------------------------------

_LOGDET_CASES = ["log1k", "log4k", "skew1k", "inv3d", "small", "tiny", "gauss1k"]


@pytest.mark.parametrize("name", _LOGDET_CASES)
def test_logdet_matches_dense_slogdet(name):
    """|det A| = |det S| since U and V are orthogonal; det A = det S when the
    bases are symmetric (V = U).  Both dense determinants come from LAPACK."""
    h, b, sp, A = case(name)
    fa = ofa.factor(h, sp)
    ld, sign = ofa.logdet(fa)
    # rounding of the pivots scales with the sum of the magnitudes of the terms
    terms = sum(float(np.sum(np.abs(np.log(np.abs(np.diag(lu)))))) for lu, _ in fa.lu)
    tol = 1e-10 * max(1.0, terms)
    sa, la = np.linalg.slogdet(A)
    ss, ls = np.linalg.slogdet(osp.dense_S(sp))
    assert abs(ld - la) <= tol
    assert abs(ld - ls) <= tol
    assert sign == int(ss)
    if h.col_leaf_basis is None:
        assert sign == int(sa)


def test_logdet_cases_exercise_both_sign_terms():
    """The cases above hold odd and even counts of interchanges and of
    negative pivots, and both signs of det S, so dropping either sign term of
    the oracle flips the sign of at least one case."""
    swaps, negs, signs = set(), set(), set()
    for name in _LOGDET_CASES:
        h, b, sp, A = case(name)
        fa = ofa.factor(h, sp)
        swaps.add(sum(int(np.count_nonzero(p != np.arange(p.size))) for _, p in fa.lu) % 2)
        negs.add(sum(int(np.count_nonzero(np.diag(lu) < 0.0)) for lu, _ in fa.lu) % 2)
        signs.add(ofa.logdet(fa)[1])
    assert swaps == {0, 1} and negs == {0, 1} and signs == {-1, 1}


def test_refinement_and_gmres_reach_1e10():
    h, b, sp, A = case("log4k")
    fa = ofa.factor(h, sp)
    mv = oh2.Matvec(h)
    pre = lambda r: ofa.solve(h, sp, fa, r)
    x, hist = oit.refine(mv, pre, b, tol=1e-10)
    assert hist[-1] <= 1e-10
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-9
    # a deliberately weakened preconditioner (S perturbed) still converges under GMRES
    S = osp.dense_S(sp)
    rng = np.random.default_rng(0)
    Sp = S * (1.0 + 1e-3 * rng.standard_normal(S.shape))
    lu = sla.lu_factor(Sp)
    pre2 = lambda r: osp.apply_N(sp, h, sla.lu_solve(lu, osp.apply_T(sp, h, r)), col=True)
    xg, hg = oit.gmres(mv, pre2, b[:, 0], tol=1e-10, restart=20, maxit=100)
    assert hg[-1] <= 1e-10
    assert np.linalg.norm(xg - xd[:, 0]) / np.linalg.norm(xd[:, 0]) < 1e-8
    assert len(hg) > 2


# --------------------------------------------------------------------------
# block Cholesky of an SPD S (§5.3-5.4, Proposition 2.1)
# --------------------------------------------------------------------------


def _dense_chol(fa, n):
    """The block factors as one dense lower factor in the original row order,
    and the scalar elimination order."""
    sym = fa.sym
    Ld = np.zeros((n, n))
    perm = []
    for k in range(sym.sn_ptr.size - 1):
        rows = ofa._rows(fa.node_off, [int(v) for v in sym.order[sym.sn_ptr[k]:sym.sn_ptr[k + 1]]])
        brows = ofa._rows(fa.node_off, [int(w) for w in sym.boundary[k]])
        Ld[np.ix_(rows, rows)] = fa.L11[k]
        if brows.size:
            Ld[np.ix_(brows, rows)] = fa.L21[k]
        perm.extend(rows.tolist())
    return Ld, np.array(perm)


@pytest.mark.parametrize("name", ["gauss1k", "gauss3d"])
def test_block_cholesky_matches_dense(name):
    h, b, sp, A = case(name)
    S = osp.dense_S(sp)
    fa = ofa.cholesky(h, sp)
    Ld, perm = _dense_chol(fa, h.n)
    assert np.linalg.norm(Ld @ Ld.T - S) <= 1e-12 * np.linalg.norm(S)
    Lp = Ld[np.ix_(perm, perm)]
    assert np.abs(np.triu(Lp, 1)).max() == 0.0           # lower triangular in elimination order
    Lref = np.linalg.cholesky(S[np.ix_(perm, perm)])      # unique for an SPD matrix
    assert np.linalg.norm(Lp - Lref) <= 1e-10 * np.linalg.norm(Lref)
    c = osp.apply_T(sp, h, b)
    y = ofa.solve_S_chol(fa, c)
    yd = np.linalg.solve(S, c)
    assert np.linalg.norm(y - yd) <= 1e-10 * np.linalg.norm(yd)
    sgn, ld = np.linalg.slogdet(A)
    assert sgn > 0 and abs(ofa.logdet_chol(fa) - ld) <= 1e-10 * max(1.0, abs(ld))


def test_block_cholesky_refuses_an_indefinite_S():
    h, b, sp, A = case("log1k")     # -log r on [0,1]^2: S has a negative eigenvalue
    assert np.linalg.eigvalsh(osp.dense_S(sp)).min() < 0
    with pytest.raises(np.linalg.LinAlgError):
        ofa.cholesky(h, sp)


# --------------------------------------------------------------------------
# pivot search restricted to the 64-row diagonal tile (FP32 preconditioner)
# --------------------------------------------------------------------------


def test_getrf_tile_with_one_tile_is_lapack_getrf():
    rng = np.random.default_rng(3)
    for n in (1, 7, 64, 150):
        F = rng.standard_normal((n, n))
        lu, piv = ofa.getrf_tile(F, nb=max(n, 1))
        lur, pivr = sla.lu_factor(F)
        assert np.array_equal(piv, pivr)
        assert np.abs(lu - lur).max() <= 1e-12 * max(1.0, np.abs(lur).max())


def test_getrf_tile_reconstructs_and_searches_only_its_tile():
    rng = np.random.default_rng(4)
    n = 150
    F = rng.standard_normal((n, n))
    F[100, 0] = 1e3          # the column maximum lies outside the first 64-row tile
    lu, piv = ofa.getrf_tile(F, nb=64)
    assert piv[0] == int(np.argmax(np.abs(F[:64, 0])))
    assert np.all(piv >= np.arange(n)) and np.all(piv < np.minimum((np.arange(n) // 64 + 1) * 64, n))
    P = np.arange(n)
    for j, p in enumerate(piv):
        P[[j, p]] = P[[p, j]]
    L = np.tril(lu, -1) + np.eye(n)
    U = np.triu(lu)
    assert np.linalg.norm(L @ U - F[P]) <= 1e-13 * np.linalg.norm(F) * n


@pytest.mark.parametrize("name", ["log1k", "log4k", "skew1k"])
def test_tile_pivoted_block_lu_solves(name):
    h, b, sp, A = case(name)
    fa = ofa.factor(h, sp, pivot="tile")
    c = osp.apply_T(sp, h, b)
    y = ofa.solve_S(fa, c)
    yd = np.linalg.solve(osp.dense_S(sp), c)
    assert np.linalg.norm(y - yd) <= 1e-9 * np.linalg.norm(yd)
    lo, so = ofa.logdet(fa)
    sa, la = np.linalg.slogdet(A)
    assert abs(lo - la) <= 1e-9 * max(1.0, abs(la))
    if h.col_leaf_basis is None:
        assert so == int(sa)


# --------------------------------------------------------------------------
# threshold incomplete LU (ILUt), the preconditioner of §5.5
# --------------------------------------------------------------------------


def test_ilut_hand_example():
    """A 3 x 3 arrow matrix worked by hand.  Row 1: multiplier 1/4, then
    u11 = 4 - 1/4 = 3.75 and the fill u12 = -1/4.  With tau = 0.1 the
    threshold of row 1 is 0.1 * ||(1, 4, 0)|| = 0.412 > 1/4, so the multiplier
    itself is dropped and row 1 of U stays (0, 4, 0)."""
    A = np.array([[4.0, 1.0, 1.0], [1.0, 4.0, 0.0], [1.0, 0.0, 4.0]])
    L, U = oilu.ilut(A, 0.01)
    assert L[1, 0] == 0.25 and U[1, 1] == 3.75 and U[1, 2] == -0.25
    assert L[2, 0] == 0.25 and abs(L[2, 1] - (-0.25 / 3.75)) < 1e-15
    assert abs(U[2, 2] - (4.0 - 0.25 - 0.25 * 0.25 / 3.75)) < 1e-14
    L, U = oilu.ilut(A, 0.1)
    assert L[1, 0] == 0.0 and np.array_equal(U[1], [0.0, 4.0, 0.0])


def test_ilut_without_dropping_is_the_exact_lu():
    h, b, sp, A = case("log1k")
    fa = oilu.factor_ilut(h, sp, 0.0)
    Ap = osp.dense_S(sp)[np.ix_(fa.perm, fa.perm)]
    assert np.array_equal(fa.L, np.tril(fa.L)) and np.all(np.diag(fa.L) == 1.0)
    assert np.array_equal(fa.U, np.triu(fa.U))
    assert np.linalg.norm(fa.L @ fa.U - Ap) <= 1e-12 * np.linalg.norm(Ap)   # the LU without pivoting is unique
    c = osp.apply_T(sp, h, b)
    yd = np.linalg.solve(osp.dense_S(sp), c)
    assert np.linalg.norm(oilu.solve_S_ilu(fa, c) - yd) <= 1e-9 * np.linalg.norm(yd)


def test_ilut_keeps_no_entry_below_the_row_threshold():
    h, b, sp, A = case("small")
    tau = 1e-2
    fa = oilu.factor_ilut(h, sp, tau)
    Ap = osp.dense_S(sp)[np.ix_(fa.perm, fa.perm)]
    thr = tau * np.linalg.norm(Ap, axis=1)
    off_l = np.abs(np.tril(fa.L, -1))
    off_u = np.abs(np.triu(fa.U, 1))
    assert np.all((off_l == 0) | (off_l >= thr[:, None]))
    assert np.all((off_u == 0) | (off_u >= thr[:, None]))
    full = oilu.factor_ilut(h, sp, 0.0)
    assert np.count_nonzero(fa.L) + np.count_nonzero(fa.U) < np.count_nonzero(full.L) + np.count_nonzero(full.U)


def test_ilut_preconditions_the_example_of_section_5_5():
    """§5.5's matrix (3D points, 1 on the diagonal, |r|/d inside d, d/|r|
    beyond): GMRES on the H^2 product preconditioned by the ILUt of S reaches
    1e-10 at the paper's drop tolerances 1e-2 and 2e-2.  As §5.5 describes,
    the larger d (worse conditioned) needs more steps, and the larger tau
    gives sparser factors and more steps."""
    steps, nnz = {}, {}
    for kern in ("ifmm_d1e-3", "ifmm_d1e-2"):
        h, b = synth.make_small(1500, kernel=kern, leaf=40, tol=1e-6, seed=12, dim=3, nrhs=1)
        sp = osp.sparsify(h)
        mv = oh2.Matvec(h)
        for tau in (1e-2, 2e-2):
            fa = oilu.factor_ilut(h, sp, tau)
            cnt = [0]

            def pre(v, fa=fa, h=h, sp=sp):
                cnt[0] += 1
                return oilu.precondition(h, sp, fa, v)

            x, hist = oit.gmres(mv, pre, b[:, 0], tol=1e-10, restart=30, maxit=300)
            assert oit.rel_residual(mv, b[:, 0], x) <= 2e-10
            steps[kern, tau] = cnt[0]
            nnz[kern, tau] = np.count_nonzero(fa.L) + np.count_nonzero(fa.U)
    for kern in ("ifmm_d1e-3", "ifmm_d1e-2"):
        assert nnz[kern, 2e-2] < nnz[kern, 1e-2] and steps[kern, 2e-2] >= steps[kern, 1e-2]
    for tau in (1e-2, 2e-2):
        assert steps["ifmm_d1e-2", tau] > steps["ifmm_d1e-3", tau]
