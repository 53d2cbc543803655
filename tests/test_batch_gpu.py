"""A batch of mirrors of uneven degree and element count: every mirror's block
of the batched operator / preconditioner equals the single-mirror result
bitwise, and the batched solve gives each mirror's energies (oracle parity)."""
import numpy as np
import pytest

import workloads as W
from oracle import Mesh, Operator, observables as ob

from cases import box_layers, box_tiny, cyl_small

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_06893_gb300 import build
    build.build()


def batch_descs():
    return [box_tiny(2), cyl_small(3, 1), box_layers(4), cyl_small(4, 1, thick=(0.03,)),
            W.sweep_instance(3), box_tiny(5)]


def test_batch_blocks_equal_single_mirror_results():
    from paper_2111_06893_gb300 import thermonoise
    descs = batch_descs()
    bc = thermonoise.Context().build_batch(descs)
    off = bc.dof_off
    rng = np.random.default_rng(0)
    for dtype in (torch.float64, torch.float32):
        u = torch.tensor(rng.uniform(-1, 1, size=int(off[-1])), dtype=dtype, device="cuda")
        y = bc.apply_operator(u)
        z = bc.precond_apply(u, precond="zline")
        zg = bc.precond_apply(u, precond="zgroup")
        for i, d in enumerate(descs):
            sc = thermonoise.setup(d)
            ui = u[off[i]:off[i + 1]].clone()
            assert torch.equal(y[off[i]:off[i + 1]], sc.apply_operator(ui)), (i, dtype)
            assert torch.equal(z[off[i]:off[i + 1]], sc.precond_apply(ui, precond="zline")), (i, dtype)
            assert torch.equal(zg[off[i]:off[i + 1]], sc.precond_apply(ui, precond="zgroup")), (i, dtype)


def test_batched_solve_energies_match_oracle():
    from paper_2111_06893_gb300 import thermonoise
    descs = batch_descs()[:4]
    bc = thermonoise.Context().build_batch(descs)
    Uos = []
    for d in descs:
        op = Operator(Mesh(d))
        Uos.append(ob.layer_energies(op, ob.solve_dense(op.assemble(), op.rhs())))
    for mode, pc in (("f64", "zline"), ("mixed", "zline"), ("f64", "zgroup"), ("mixed", "zgroup")):
        u, rep = bc.solve(mode=mode, rtol=1e-12, energy_rtol=1e-12, precond=pc)
        U = bc.layer_energies(u)
        for i, Uo in enumerate(Uos):
            Ui = U[bc.layer_off[i]:bc.layer_off[i + 1]]
            assert np.max(np.abs(Ui - Uo) / Uo) < 1e-9, (mode, pc, i, Ui, Uo, rep)


def test_batched_gradients_equal_single_mirror_gradients():
    from paper_2111_06893_gb300 import thermonoise
    descs = batch_descs()[:3]
    bc = thermonoise.Context().build_batch(descs)
    u, _ = bc.solve(mode="f64", rtol=1e-13, energy_rtol=1e-14, raise_on_error=False)
    nl = int(bc.layer_off[-1])
    w = np.random.default_rng(2).uniform(0.5, 2.0, size=nl)
    gb = bc.energy_grad(u, w, mode="f64", rtol=1e-13, raise_on_error=False)
    for i, d in enumerate(descs):
        sc = thermonoise.setup(d)
        ui, _ = sc.solve(mode="f64", rtol=1e-13, energy_rtol=1e-14, raise_on_error=False)
        wi = w[bc.layer_off[i]:bc.layer_off[i + 1]]
        gs = sc.energy_grad(ui, wi, mode="f64", rtol=1e-13, raise_on_error=False)
        gi = gb["instances"][i]
        scale = np.abs(gs["slab_z"]).max()
        assert np.max(np.abs(gi["slab_z"] - gs["slab_z"])) <= 1e-7 * scale, (i, gi["slab_z"], gs["slab_z"])
        assert abs(gi["r0"] - gs["r0"]) <= 1e-7 * abs(gs["r0"])
        assert np.max(np.abs(gi["moduli"] - gs["moduli"])) <= 1e-7 * np.abs(gs["moduli"]).max()
