"""Host-side checks of the C ABI (no GPU needed).

* libh2sp.so loads and exports every function include/h2sp.h declares;
* h2sp_analyze (host planning only, no CUDA call) reproduces the oracle's
  integer structure bit for bit: S node order and sizes, the VBR pattern of
  S, closures, elimination order, supernodes and their boundaries;
* malformed descriptors are rejected with H2SP_EINVAL before any launch.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1705_04601_gb300 import h2sp as H
from paper_1705_04601_gb300 import synth
from oracle import factor as ofa
from oracle import sparsify as osp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1705_04601_gb300 import build
    build.build()


def test_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "h2sp.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"\b(h2sp_[a-z_A-Z0-9]+)\s*\(", hdr))
    assert len(names) >= 12
    L = ctypes.CDLL(H.LIB_PATH)
    for nm in sorted(names):
        assert hasattr(L, nm), nm
    assert names == set(H.SIGNATURES), names ^ set(H.SIGNATURES)


_CASES = {
    "log1k": dict(n=1024, kernel="log", leaf=32, tol=1e-8, seed=1),
    "log4k": dict(n=4096, kernel="log", leaf=64, tol=1e-8, seed=1),
    "skew1k": dict(n=1024, kernel="log_skew", leaf=32, tol=1e-8, seed=2),
    "raw1k": dict(n=1024, kernel="log", leaf=32, tol=None, seed=3),
    "tiny": dict(n=48, kernel="log", leaf=64, tol=1e-8, seed=6),
    "inv3d": dict(n=1500, kernel="inv", leaf=40, tol=1e-6, seed=5, dim=3),
    "log16k": dict(n=16384, kernel="log", leaf=64, tol=1e-6, seed=9),
    # 3D with blocks above 64 rows: 1/r on the jittered Fibonacci sphere (leaf <= 128,
    # levels up to 91 rows) and Yukawa in the cube (leaves up to 113 points)
    "sphere8k": dict(workload="inv3d_sphere_n262144", n=8192),
    "cube6k": dict(workload="yukawa3d_n1048576", n=6000),
}


def _make(name):
    s = _CASES[name]
    if "workload" in s:
        return synth.make_workload(s["workload"], n=s["n"])[0]
    h, _ = synth.make_small(s["n"], kernel=s["kernel"], leaf=s["leaf"], tol=s["tol"], seed=s["seed"],
                            dim=s.get("dim", 2))
    return h


@pytest.mark.parametrize("name", list(_CASES))
def test_analyze_matches_oracle_structure(name):
    h = _make(name)
    sp = osp.sparsify(h)
    sym = ofa.symbolic(h, sp)
    vbr = osp.to_vbr(sp)
    hd = H.h2sp_analyze(H.H2Input(h, device=None))
    q = H.h2sp_query(hd)
    assert q["lstop"] == sp.sch.lstop
    assert q["nnodes"] == sp.sch.node_size.size
    S = H.h2sp_export_S(hd, values=False)
    assert np.array_equal(S["node_size"], sp.sch.node_size)
    assert np.array_equal(S["brow_ptr"], vbr.brow_ptr)
    assert np.array_equal(S["bcol_idx"], vbr.bcol_idx)
    assert np.array_equal(S["val_off"], vbr.val_off)
    st = H.h2sp_export_structure(hd)
    assert np.array_equal(st["node_level"], sp.sch.node_level)
    assert np.array_equal(st["node_cluster"], sp.sch.node_cluster)
    assert np.array_equal(st["closure"], sym.closure)
    assert np.array_equal(st["order"], sym.order)
    assert np.array_equal(st["sn_ptr"], sym.sn_ptr)
    assert st["bnd_ptr"][-1] == sum(len(b) for b in sym.boundary)
    for k, b in enumerate(sym.boundary):
        assert np.array_equal(st["bnd"][st["bnd_ptr"][k]:st["bnd_ptr"][k + 1]], b)
    assert q["factor_flops"] == pytest.approx(sym.flops, rel=1e-12)
    hd.close()


def _bad(h, **changes):
    inp = H.H2Input(h, device=None)
    for k, v in changes.items():
        inp.arrs[k] = v
    return inp


def test_malformed_descriptors_are_rejected():
    h = _make("log1k")
    base = H.H2Input(h, device=None)
    # unsorted close list
    nc = base.arrs["near_col"].copy()
    lo, hi = int(h.near_ptr[3]), int(h.near_ptr[4])
    nc[lo:hi] = nc[lo:hi][::-1]
    bad = [
        dict(near_col=nc),
        dict(parent=np.where(np.arange(h.ncl) == 5, 7, base.arrs["parent"]).astype(np.int32)),
        dict(size=np.where(np.arange(h.ncl) == h.ncl - 1, h.size[-1] + 1, h.size).astype(np.int64)),
        dict(rank=np.where(np.arange(h.ncl) == 3, -1, h.rank).astype(np.int32)),
        dict(level_ptr=np.array([0, 2] + list(h.level_ptr[2:]), np.int32)),
    ]
    for ch in bad:
        with pytest.raises(H.H2spError) as e:
            H.h2sp_analyze(_bad(h, **ch))
        assert e.value.status == H.H2SP_EINVAL
    # a far list that crosses depths
    fc = base.arrs["far_col"].copy()
    fc[0] = 0
    with pytest.raises(H.H2spError) as e:
        H.h2sp_analyze(_bad(h, far_col=fc))
    assert e.value.status == H.H2SP_EINVAL


def test_oversized_blocks_are_reported_unsupported():
    h, _ = synth.make_small(2000, kernel="log", leaf=1000, tol=1e-8, seed=3)
    assert h.size[h.level_ptr[h.depth]:].max() > 384
    with pytest.raises(H.H2spError) as e:
        H.h2sp_analyze(H.H2Input(h, device=None))
    assert e.value.status == H.H2SP_EUNSUPPORTED


def test_device_calls_on_an_analyzed_handle_are_refused():
    h = _make("log1k")
    hd = H.h2sp_analyze(H.H2Input(h, device=None))
    st = H.lib().h2sp_factor(hd.ptr, 0, None)
    assert st == H.H2SP_ESTATE
    hd.close()


def test_forest_plan_is_block_diagonal():
    """Batched form: several roots = independent systems; S never couples two of them."""
    systems, f, _ = synth.make_batched(5, 400, 1500, leaf=32, tol=1e-8)
    hd = H.h2sp_analyze(H.H2Input(f, device=None))
    st = H.h2sp_export_structure(hd)
    S = H.h2sp_export_S(hd, values=False)
    nroots = int(f.level_ptr[1])
    assert nroots == 5
    root = np.zeros(f.ncl, dtype=np.int64)
    for c in range(f.ncl):
        root[c] = c if c < nroots else root[f.parent[c]]
    node_root = root[st["node_cluster"]]
    for i in range(len(S["node_size"])):
        cols = S["bcol_idx"][S["brow_ptr"][i]:S["brow_ptr"][i + 1]]
        assert np.all(node_root[cols] == node_root[i])
    # every supernode lies in one system; its closure is a cluster of that system
    for k in range(len(st["sn_ptr"]) - 1):
        nodes = st["order"][st["sn_ptr"][k]:st["sn_ptr"][k + 1]]
        assert len(set(node_root[nodes])) == 1
        assert root[st["closure"][nodes[0]]] == node_root[nodes[0]]
    assert int(S["node_size"].sum()) == f.n
    hd.close()


def test_forest_rejects_pairs_across_systems():
    systems, f, _ = synth.make_batched(3, 400, 800, leaf=32, tol=1e-8)
    inp = H.H2Input(f, device=None)
    nc = inp.arrs["near_col"].copy()
    last = int(f.level_ptr[-1]) - 1          # a leaf of the last system
    nc[0] = last                              # first leaf (system 0) now "close" to it
    inp.arrs["near_col"] = np.sort(nc[:int(f.near_ptr[1])]).tolist() + nc[int(f.near_ptr[1]):].tolist()
    inp.arrs["near_col"] = np.array(inp.arrs["near_col"], dtype=np.int32)
    with pytest.raises(H.H2spError) as e:
        H.h2sp_analyze(inp)
    assert e.value.status == H.H2SP_EINVAL


def _with_fake_numbers(inp):
    """Descriptor of `inp` with non-null numeric pointers that must never be
    dereferenced (the calls below fail on the host before any launch)."""
    d = inp.desc()
    buf = (ctypes.c_double * 4)()
    for nm in ("leaf_basis", "transfer", "coupling", "near_block"):
        setattr(d, nm, ctypes.addressof(buf))
    return d, buf


def test_sparsify_analyzed_rejects_a_different_structure():
    h = _make("log1k")
    an = H.h2sp_analyze(H.H2Input(h, device=None))
    out = H._vp()
    o = H.Opts(0)
    # another point set: different lists
    h2, _ = synth.make_small(1024, kernel="log", leaf=32, tol=1e-8, seed=11)
    d2, keep2 = _with_fake_numbers(H.H2Input(h2, device=None))
    assert H.lib().h2sp_sparsify_analyzed(an.ptr, ctypes.byref(d2), ctypes.byref(o), None,
                                          ctypes.byref(out)) == H.H2SP_EINVAL
    # same lists, one close-block offset changed: only the fingerprint sees it
    inp = H.H2Input(h, device=None)
    inp.arrs["near_off"] = inp.arrs["near_off"].copy()
    inp.arrs["near_off"][5] += 1
    d3, keep3 = _with_fake_numbers(inp)
    assert H.lib().h2sp_sparsify_analyzed(an.ptr, ctypes.byref(d3), ctypes.byref(o), None,
                                          ctypes.byref(out)) == H.H2SP_EINVAL
    # missing numbers
    d4 = H.H2Input(h, device=None).desc()
    assert H.lib().h2sp_sparsify_analyzed(an.ptr, ctypes.byref(d4), ctypes.byref(o), None,
                                          ctypes.byref(out)) == H.H2SP_EINVAL
    assert not out
    an.close()


def test_unknown_option_bits_are_rejected():
    """h2sp_opts.flags accepts H2SP_SPARSIFY_FP32 only; any other bit is
    refused on the host before planning or launching."""
    h = _make("log1k")
    inp = H.H2Input(h, device=None)
    d, keep = _with_fake_numbers(inp)
    out = H._vp()
    for bad in (2, 4, 1 << 30, -1):
        o = H.Opts(bad)
        assert H.lib().h2sp_sparsify(ctypes.byref(d), ctypes.byref(o), None, ctypes.byref(out)) == H.H2SP_EINVAL
        an = H.h2sp_analyze(H.H2Input(h, device=None))
        assert H.lib().h2sp_sparsify_analyzed(an.ptr, ctypes.byref(d), ctypes.byref(o), None,
                                              ctypes.byref(out)) == H.H2SP_EINVAL
        an.close()
    assert not out


def test_analysis_handle_reports_no_sparsify_precision():
    h = _make("log1k")
    an = H.h2sp_analyze(H.H2Input(h, device=None))
    st = H.h2sp_query(an)
    assert st["sparsify_prec"] == -1 and st["factor_prec"] == -1
    an.close()


def test_refactor_needs_a_factorized_handle():
    """h2sp_refactor on a null handle is EINVAL; on an analysis-only handle
    (no device buffers, no factorization to repeat) it is ESTATE, decided on
    the host before any CUDA call."""
    assert H.lib().h2sp_refactor(None, None) == H.H2SP_EINVAL
    h = _make("log1k")
    an = H.h2sp_analyze(H.H2Input(h, device=None))
    assert H.lib().h2sp_refactor(an.ptr, None) == H.H2SP_ESTATE
    an.close()


def test_logdet_needs_factors():
    """h2sp_logdet: a null handle or output array is EINVAL; an analysis-only
    handle has no factors (ESTATE), decided on the host before any CUDA call."""
    d = ctypes.c_double(0.0)
    assert H.lib().h2sp_logdet(None, ctypes.byref(d), None, None) == H.H2SP_EINVAL
    h = _make("log1k")
    an = H.h2sp_analyze(H.H2Input(h, device=None))
    assert H.lib().h2sp_logdet(an.ptr, None, None, None) == H.H2SP_EINVAL
    assert H.lib().h2sp_logdet(an.ptr, ctypes.byref(d), None, None) == H.H2SP_ESTATE
    an.close()


def test_query_counts_independent_systems():
    systems, f, _ = synth.make_batched(4, 400, 1200, leaf=32, tol=1e-8)
    an = H.h2sp_analyze(H.H2Input(f, device=None))
    assert H.h2sp_query(an)["nsys"] == 4 == len(systems)
    an.close()
    an = H.h2sp_analyze(H.H2Input(_make("tiny"), device=None))
    assert H.h2sp_query(an)["nsys"] == 1
    an.close()


@pytest.mark.parametrize("name", ["sphere8k", "cube6k"])
def test_large_blocks_plan_small_items_first(name):
    """Blocks above 64 rows are planned (up to 384): the structure matches the
    oracle (test above) and the planner's audit accepts the item lists, whose
    small items lead each level."""
    h = _make(name)
    sp = osp.sparsify(h)
    assert max(int(sp.sch.m[c]) for c in range(h.ncl) if sp.sch.level[c] < max(sp.sch.lstop, 1)) > 64
    hd = H.h2sp_analyze(H.H2Input(h, device=None))
    assert H.h2sp_query(hd)["lstop"] == sp.sch.lstop
    hd.close()


def test_plain_c_consumer(tmp_path):
    """The ABI from C: include/h2sp.h compiles as C99 (and as C++), and a C
    program linked against libh2sp.so analyses a hand-built two-leaf structure
    and checks the sizes, the S pattern of §3 and the state errors."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lib_dir = os.path.dirname(H.LIB_PATH)
    exe = str(tmp_path / "analyze_tiny")
    src = os.path.join(ROOT, "tests", "c_abi", "analyze_tiny.c")
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), src,
                        "-L", lib_dir, "-lh2sp", "-Wl,-rpath," + lib_dir, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
    if shutil.which("g++") is not None:
        r = subprocess.run(["g++", "-std=c++17", "-fsyntax-only", "-Wall", "-Werror", "-x", "c++",
                            os.path.join(ROOT, "include", "h2sp.h")], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_sparsification_work_is_linear_in_n():
    """§5.2: the sparsification costs O(N) for a fixed accuracy.  The
    planner's algorithmic flop count per point and the nonzeros of S per point
    stay within a factor 1.5 across N = 4,096 .. 32,768 (2D -log r, leaf <= 64,
    basis tol 1e-6), while the factorization work per point grows with N."""
    per_n = []
    for n in (4096, 16384, 32768):
        h, _ = synth.make_workload("log2d_n65536", n=n)
        an = H.h2sp_analyze(H.H2Input(h, device=None))
        q = H.h2sp_query(an)
        per_n.append((q["sparsify_flops"] / n, q["nnz"] / n, q["factor_flops"] / n))
        an.close()
    sf = [a for a, _, _ in per_n]
    nz = [b for _, b, _ in per_n]
    ff = [c for _, _, c in per_n]
    assert max(sf) / min(sf) <= 1.5
    assert max(nz) / min(nz) <= 1.5
    assert ff[0] < ff[1] < ff[2]


def test_solve_rejects_bad_right_hand_side_counts():
    """h2sp_solve takes 1 <= nrhs <= 64; other counts, or a null handle, are
    H2SP_EINVAL before anything is touched."""
    o = H.SolveOpts(int(H.H2SP_DIRECT), 1e-10, 10, 20)
    dummy = ctypes.c_void_p(16)
    for nrhs in (0, -1, 65):
        assert H.lib().h2sp_solve(None, ctypes.byref(o), nrhs, dummy, 1, dummy, 1, None, None) == H.H2SP_EINVAL
    h = _make("tiny")
    an = H.h2sp_analyze(H.H2Input(h, device=None))
    for nrhs in (0, 65):
        assert H.lib().h2sp_solve(an.ptr, ctypes.byref(o), nrhs, dummy, h.n, dummy, h.n, None, None) == H.H2SP_EINVAL
    assert H.lib().h2sp_solve(an.ptr, ctypes.byref(o), 1, dummy, h.n, dummy, h.n, None, None) == H.H2SP_ESTATE
    an.close()


def test_empty_and_null_descriptors_are_rejected():
    """An empty matrix (N = 0), a descriptor without levels, a NULL
    descriptor or a NULL output handle are EINVAL, and no handle comes back."""
    h = _make("tiny")
    inp = H.H2Input(h, device=None)
    out = ctypes.c_void_p()
    d = inp.desc()
    d.n = 0
    assert H.lib().h2sp_analyze(ctypes.byref(d), ctypes.byref(out)) == H.H2SP_EINVAL and not out.value
    d = inp.desc()
    d.depth = -1
    assert H.lib().h2sp_analyze(ctypes.byref(d), ctypes.byref(out)) == H.H2SP_EINVAL and not out.value
    d = inp.desc()
    d.level_ptr = None
    assert H.lib().h2sp_analyze(ctypes.byref(d), ctypes.byref(out)) == H.H2SP_EINVAL and not out.value
    assert H.lib().h2sp_analyze(None, ctypes.byref(out)) == H.H2SP_EINVAL and not out.value
    assert H.lib().h2sp_analyze(ctypes.byref(inp.desc()), None) == H.H2SP_EINVAL
    # the same descriptor, intact, is accepted: a single leaf, no far field (S = A)
    an = H.h2sp_analyze(inp)
    assert H.h2sp_query(an)["n"] == h.n
    an.close()
