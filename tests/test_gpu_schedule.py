"""The level schedule of §2.2-2.3 on the device (integer kernels): block
sizes m, k', the stacking offsets, the level-vector offsets, the S node order
and offsets and the close lists Near_l, bit-exact against the oracle's
schedule; and the plan h2sp_sparsify builds from them is the host analysis's
plan to the integer."""
import numpy as np
import pytest

from paper_1705_04601_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1705_04601_gb300 import h2sp as H  # noqa: E402
from oracle import sparsify as osp  # noqa: E402

_CASES = {
    "log1k": lambda: synth.make_small(1024, kernel="log", leaf=32, tol=1e-8, seed=1, nrhs=1)[0],
    # ranks above the leaf sizes: k' = min(k, m) clips
    "raw1k": lambda: synth.make_small(1024, kernel="log", leaf=16, tol=None, seed=2, nrhs=1)[0],
    "gauss_ragged": lambda: synth.make_small(3001, kernel="gauss", leaf=23, tol=1e-8, seed=8, nrhs=1)[0],
    "gauss3d": lambda: synth.make_small(2000, kernel="gauss", leaf=40, tol=1e-8, seed=6, dim=3, nrhs=1)[0],
    "deep2d": lambda: synth.make_small(4096, kernel="log", leaf=8, tol=1e-6, seed=3, nrhs=1)[0],
    "sphere8k": lambda: synth.make_workload("inv3d_sphere_n262144", n=8192)[0],
    "log2d_16k": lambda: synth.make_workload("log2d_n65536", n=16384)[0],
    "forest": lambda: synth.make_forest([synth.make_small(n, kernel="log", leaf=32, tol=1e-8, seed=s, nrhs=1)[0]
                                         for n, s in ((700, 1), (1500, 2), (300, 3), (2048, 4))]),
}
_cache = {}


def make(name):
    if name not in _cache:
        _cache[name] = _CASES[name]()
    return _cache[name]


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1705_04601_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA is required for the gpu tests")


@pytest.mark.parametrize("name", list(_CASES))
def test_device_schedule_matches_oracle(name):
    h = make(name)
    sch = osp.schedule(h)
    an = H.h2sp_analyze(H.H2Input(h, device=None))
    got = H.h2sp_export_schedule(an, h.ncl)
    assert got["lstop"] == sch.lstop
    for k in ("m", "kp", "off", "xoff"):
        assert np.array_equal(got[k], getattr(sch, k)), k
    assert np.array_equal(got["node_off"], sch.node_off)
    assert np.array_equal(got["node_cluster"], sch.node_cluster)
    D = h.depth
    for l in range(1, sch.lstop + 1):
        lo, hi = int(h.level_ptr[D - l]), int(h.level_ptr[D - l + 1])
        ptr, col = H.h2sp_export_near(an, l, hi - lo)
        rows = np.repeat(np.arange(lo, hi, dtype=np.int64), np.diff(ptr))
        pairs = np.stack([rows, col.astype(np.int64)], axis=1)
        assert np.array_equal(pairs, sch.near[l].reshape(-1, 2)), l
    for bad in (0, sch.lstop + 1):
        with pytest.raises(H.H2spError) as e:
            H.h2sp_export_near(an, bad, 1)
        assert e.value.status == H.H2SP_EINVAL
    an.close()


@pytest.mark.parametrize("name", ["log1k", "raw1k", "sphere8k", "forest"])
def test_sparsify_plan_from_device_schedule_equals_host_analysis(name):
    """h2sp_sparsify plans from the device schedule, h2sp_analyze from the
    host's; every integer of the two plans agrees."""
    h = make(name)
    an = H.h2sp_analyze(H.H2Input(h, device=None))
    hd = H.h2sp_sparsify(H.H2Input(h))
    qa, qd = H.h2sp_query(an), H.h2sp_query(hd)
    for k in ("n", "depth", "lstop", "nnodes", "nnzb", "nnz", "nsupernodes", "max_front", "front_elems"):
        assert qa[k] == qd[k], k
    assert qa["factor_flops"] == qd["factor_flops"]
    a, d = H.h2sp_export_structure(an), H.h2sp_export_structure(hd)
    for k in a:
        assert np.array_equal(a[k], d[k]), k
    sa, sd = H.h2sp_export_S(an, values=False), H.h2sp_export_S(hd, values=False)
    for k in ("node_size", "brow_ptr", "bcol_idx", "val_off"):
        assert np.array_equal(sa[k], sd[k]), k
    hd.close()
    an.close()
