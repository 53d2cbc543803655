"""The seeded synthetic inputs follow the stated recipe: sizes, materials,
layer structure and the design sweep's distributions of the five workloads
(an isotropic cube, a single coating, a crystalline stack, a 256-mirror
sweep and a large mirror)."""
import math

import numpy as np

import workloads as W


def geometric(z):
    d = [-v for v in z]
    r = [d[i + 1] / d[i] for i in range(len(d) - 1)]
    return np.allclose(r, r[0], rtol=1e-12)


def test_plain_box():
    d = W.plain_box()
    assert W.n_dof(d) == 12288 and d["degree"] == 3
    assert d["x_breaks"][0] == -10 and d["x_breaks"][-1] == 10 and len(d["x_breaks"]) == 5
    assert d["slab_z"][0] == 0 and d["slab_z"][-1] == -20 and len(d["slab_z"]) == 5
    assert d["bc_side"] == "fixed" and d["bc_bottom"] == "fixed" and d["penalty_C"] == 1.5
    assert d["materials"] == [{"kind": "iso", "Y": 72e9, "nu": 0.17}]
    assert d["beam"] == {"r0": 1.0, "F0": 1.0}


def test_single_coating():
    d = W.single_coating()
    assert 1.9e6 < W.n_dof(d) < 2.1e6 and d["degree"] == 6
    assert d["R"] == 10 and d["slab_z"][-1] == -10
    assert math.isclose(-d["slab_z"][1], 0.02)
    assert d["materials"][0] == {"kind": "iso", "Y": 140e9, "nu": 0.23}
    assert d["materials"][1] == {"kind": "iso", "Y": 72e9, "nu": 0.17}
    assert d["slab_log"][0] == 0 and all(d["slab_log"][1:])
    assert geometric(d["slab_z"][1:])


def test_crystalline_multilayer():
    d = W.crystalline_multilayer()
    assert 7.5e6 < W.n_dof(d) < 8.5e6 and d["degree"] == 5
    th = -np.diff(d["slab_z"][:41])
    assert np.allclose(th, 4e-4, rtol=1e-9)
    assert d["slab_layer"][:40] == list(range(40))
    a, b = d["materials"][0], d["materials"][1]
    assert (a["c11"], a["c12"], a["c44"]) == (119.9e9, 53.8e9, 59.4e9)
    assert (b["c11"], b["c12"], b["c44"]) == (120.5e9, 57.0e9, 58.9e9)
    assert all(m["kind"] == "cubic" for m in d["materials"][:40])


def test_large_mirror():
    d = W.large_mirror()
    assert 5.5e7 < W.n_dof(d) < 6.5e7 and d["degree"] == 8
    assert d["R"] == 20 and d["slab_z"][-1] == -20
    th = -np.diff(d["slab_z"][:21])
    assert np.allclose(th, 1e-3, rtol=1e-9)
    Ys = [m["Y"] for m in d["materials"][:20]]
    assert Ys == [72e9, 140e9] * 10


def test_design_sweep_distributions_and_seeding():
    ds = W.design_sweep(256)
    assert len(ds) == 256
    deg = [d["degree"] for d in ds]
    assert set(deg) == {4, 5, 6, 7, 8}
    for d in ds:
        L = len(d["materials"]) - 1
        assert 1 <= L <= 20
        th = -np.diff(d["slab_z"][:L + 1])
        assert th.min() >= 1e-4 * (1 - 1e-12) and th.max() <= 5e-2 * (1 + 1e-12)
        assert 0.5 <= d["beam"]["r0"] <= 2.0 and d["R"] == 10
    assert set(len(d["materials"]) - 1 for d in ds) >= set(range(2, 20))
    assert W.design_sweep(256) == ds
    assert W.design_sweep(2, first=5) == [W.sweep_instance(5), W.sweep_instance(6)]
    assert W.design_sweep(1, first=256)[0] != ds[0]


def test_random_field_is_seeded():
    d = W.plain_box()
    u1, u2, u3 = W.random_field(d, 3), W.random_field(d, 3), W.random_field(d, 4)
    assert u1.shape == (W.n_dof(d),) and np.array_equal(u1, u2) and not np.array_equal(u1, u3)
    assert u1.min() >= -1 and u1.max() <= 1
