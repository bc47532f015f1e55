"""The seeded synthetic inputs: the same name and seed give bit-identical
inputs, another seed gives other inputs, and the generators keep the stated
recipe (unit cube, jittered unit sphere, ellipse sizes in their range)."""
import dataclasses

import numpy as np

from paper_1705_04601_gb300 import synth


def _arrays(h):
    return {f.name: getattr(h, f.name) for f in dataclasses.fields(h)
            if isinstance(getattr(h, f.name), np.ndarray)}


def test_workloads_are_reproducible():
    for name, n in [("log2d_n4096", 1024), ("inv3d_sphere_n262144", 2048), ("yukawa3d_n1048576", 1000)]:
        h1, b1 = synth.make_workload(name, n=n)
        h2, b2 = synth.make_workload(name, n=n)
        assert np.array_equal(b1, b2)
        a1, a2 = _arrays(h1), _arrays(h2)
        assert a1.keys() == a2.keys()
        for k in a1:
            assert np.array_equal(a1[k], a2[k]), (name, k)
        h3, b3 = synth.make_workload(name, n=n, seed=12345)
        assert not np.array_equal(b1, b3)


def test_point_recipes():
    p, lo, hi, cfg = synth.workload_points("yukawa3d_n1048576", n=5000)
    assert p.shape == (5000, 3) and np.all(p >= 0.0) and np.all(p < 1.0)
    assert np.all(lo == 0.0) and np.all(hi == 1.0)
    p, lo, hi, cfg = synth.workload_points("inv3d_sphere_n262144", n=5000)
    r = np.linalg.norm(p, axis=1)
    # Fibonacci lattice on the unit sphere, each coordinate jittered by at most 1e-3
    assert p.shape == (5000, 3) and np.all(np.abs(r - 1.0) <= np.sqrt(3.0) * 1e-3 + 1e-12)
    assert np.all(p > lo) and np.all(p < hi)
    # the lattice covers the sphere: every octant holds about an eighth of the points
    counts = np.bincount(((p[:, 0] > 0) * 4 + (p[:, 1] > 0) * 2 + (p[:, 2] > 0)).astype(int), minlength=8)
    assert counts.min() > 0.10 * 5000 and counts.max() < 0.15 * 5000
    pa, *_ = synth.workload_points("inv3d_sphere_n262144", n=5000)
    assert np.array_equal(p, pa)


def test_ellipse_systems_sizes():
    systems, forest, b = synth.make_batched(4, 300, 600, leaf=64, tol=1e-6)
    sizes = [h.n for h in systems]
    assert len(systems) == 4 and all(300 <= s <= 600 for s in sizes)
    assert forest.n == sum(sizes) and b.shape == (forest.n, 1)
    systems2, _, b2 = synth.make_batched(4, 300, 600, leaf=64, tol=1e-6)
    assert [h.n for h in systems2] == sizes and np.array_equal(b, b2)
