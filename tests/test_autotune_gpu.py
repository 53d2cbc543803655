"""Autotuning of the FP32 operator kernel: the two occupancy variants give
bit-identical applies and solves, on one mesh and on a batch of mixed
degrees, and the tuner times both and records its choice per degree."""
import numpy as np
import pytest

import workloads as W

from cases import box_layers, box_tiny, cyl_small

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_06893_gb300 import build
    build.build()


def rand(n, seed=0):
    rng = np.random.default_rng(seed)
    return torch.tensor(rng.uniform(-1, 1, size=n), dtype=torch.float32, device="cuda")


@pytest.mark.parametrize("desc", [box_tiny(2), box_layers(4), cyl_small(5, 1), cyl_small(6, 1),
                                  cyl_small(7, 1), box_tiny(8)],
                         ids=["p2", "p4", "p5", "p6", "p7", "p8"])
def test_variants_apply_bit_identical(desc):
    from paper_2111_06893_gb300 import thermonoise
    ctx = thermonoise.setup(desc)
    p = desc["degree"]
    u = rand(ctx.ndof)
    ys = []
    for v in (0, 1):
        ctx.set_apply_variant(p, v)
        assert ctx.apply_tuning()[p]["variant"] == v
        ys.append(ctx.apply_operator(u))
    assert torch.equal(ys[0], ys[1])
    y64 = ctx.apply_operator(u.double())
    err = float((ys[0].double() - y64).abs().max() / y64.abs().max())
    assert err < 2e-5, err


def test_variants_batch_bit_identical():
    from paper_2111_06893_gb300 import thermonoise
    descs = [box_tiny(2), cyl_small(3, 1), box_layers(4), W.sweep_instance(3), cyl_small(6, 1), box_tiny(8)]
    bc = thermonoise.Context().build_batch(descs)
    u = rand(bc.ndof, seed=1)
    ys = []
    for v in (0, 1):
        for p in sorted({d["degree"] for d in descs}):
            bc.set_apply_variant(p, v)
        ys.append(bc.apply_operator(u))
    assert torch.equal(ys[0], ys[1])


def test_variants_mixed_solve_bit_identical():
    from paper_2111_06893_gb300 import thermonoise
    desc = cyl_small(5, 1)
    ctx = thermonoise.setup(desc)
    us = []
    for v in (0, 1):
        ctx.set_apply_variant(5, v)
        u, rep = ctx.solve(mode="mixed", rtol=1e-12, energy_rtol=1e-12)
        us.append(u.clone())
    assert torch.equal(us[0], us[1])


def test_tuner_times_both_variants_and_resets_with_the_mesh():
    from paper_2111_06893_gb300 import thermonoise
    desc = cyl_small(6, 1)
    ctx = thermonoise.setup(desc)
    assert ctx.apply_tuning() == {}
    ctx.apply_operator(rand(ctx.ndof))
    t = ctx.apply_tuning()
    assert set(t) == {6}
    us0, us1 = t[6]["us"]
    assert us0 > 0 and us1 > 0
    assert t[6]["variant"] == (1 if us1 < 0.98 * us0 else 0)
    ctx.set_apply_variant(6, -1)
    assert ctx.apply_tuning() == {}
    ctx.solve(mode="mixed", rtol=1e-8)  # the mixed solve times it again
    assert set(ctx.apply_tuning()) == {6}
    ctx.build_mesh(desc)
    assert ctx.apply_tuning() == {}
    with pytest.raises(thermonoise.ThermonoiseError):
        ctx.set_apply_variant(9, 0)
    with pytest.raises(thermonoise.ThermonoiseError):
        ctx.set_apply_variant(6, 2)
