"""Adjoint energy gradients on the GPU against the oracle's complex-step
gradients (exact derivatives of the discrete energies) and against central
finite differences of GPU solves."""
import numpy as np
import pytest

import workloads as W
from oracle import gradient as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_06893_gb300 import build
    build.build()


def layered_box():
    return W.box([-1.0, 0.2, 1.0], [-0.5, 1.0], [0.0, -0.3, -0.8, -1.3], 3, None, slab_layer=[0, 1, 2],
                 materials=[W.CRYSTAL_A, W.COATING_HIGH, W.FUSED_SILICA], penalty_C=3.0,
                 bc_side="fixed", bc_bottom="fixed", r0=0.7)


def thin_cylinder():
    d = W.cylinder(10.0, 10.0, [0.02, 0.05], [W.CRYSTAL_B, W.COATING_HIGH], W.FUSED_SILICA, 1, 3, 2,
                   r0=1.3)
    # geometric substrate slabs share one depth ratio, so the face sizes h
    # of the two slabs meeting at the inner substrate boundary are equal and
    # min(h, h_ext) has a kink there: the energies have only one-sided
    # derivatives in slab_z[2] and slab_z[3].  Moving that boundary off the
    # geometric sequence makes every slab derivative two-sided.
    z = list(d["slab_z"])
    z[3] = -0.9
    d["slab_z"] = z
    return d


def iso_chain(m):
    """d(c11, c12, c44)/d(Y, nu) for an isotropic material."""
    Y, nu = m["Y"], m["nu"]
    h = 1e-7
    from paper_2111_06893_gb300.thermonoise import iso_moduli
    base = np.array(iso_moduli(Y, nu))
    dY = (np.array(iso_moduli(Y * (1 + h), nu)) - np.array(iso_moduli(Y * (1 - h), nu))) / (2 * h * Y)
    dn = (np.array(iso_moduli(Y, nu + h)) - np.array(iso_moduli(Y, nu - h))) / (2 * h)
    return base, dY, dn


# tolerance: the layered box is well conditioned (both solves accurate to
# ~1e-13); the thin-coating cylinder (C = 100, 0.02-thick layers) has
# cond(A) ~ 1e8, so both the oracle's direct solve and the GPU solves carry
# ~1e-8 relative error into u and lambda
@pytest.mark.parametrize("make,tol", [(layered_box, 1e-8), (thin_cylinder, 1e-6)])
def test_adjoint_gradient_matches_oracle_complex_step(make, tol):
    from paper_2111_06893_gb300 import thermonoise
    desc = make()
    ctx = thermonoise.setup(desc)
    # thin layers put the FP64 residual floor near 1e-11: stop on energies
    u, rep = ctx.solve(mode="f64", rtol=1e-13, energy_rtol=1e-14, raise_on_error=False)
    assert rep["rel_residual"] < 1e-10, rep
    nl = len(desc["materials"])
    rng = np.random.default_rng(4)
    w = rng.uniform(0.5, 2.0, size=nl)
    g = ctx.energy_grad(u, w, mode="f64", rtol=1e-13, raise_on_error=False)
    assert g["report"]["rel_residual"] < 1e-10, g["report"]
    ns = len(desc["slab_z"]) - 1
    # slab boundaries
    for s in range(1, ns + 1):
        ref = float(np.dot(w, G.energy_derivative(desc, ("slab_z", s))))
        scale = max(abs(ref), 1e-3 * max(abs(v) for v in g["slab_z"]))
        assert abs(g["slab_z"][s] - ref) <= tol * scale, ("slab_z", s, g["slab_z"][s], ref)
    ref = float(np.dot(w, G.energy_derivative(desc, ("r0",))))
    assert abs(g["r0"] - ref) <= tol * abs(ref), ("r0", g["r0"], ref)
    # moduli: cubic layers directly, isotropic through (Y, nu)
    for L, m in enumerate(desc["materials"]):
        if m["kind"] == "cubic":
            for q, key in enumerate(["c11", "c12", "c44"]):
                ref = float(np.dot(w, G.energy_derivative(desc, ("material", L, key))))
                assert abs(g["moduli"][L, q] - ref) <= tol * abs(ref), (L, key, g["moduli"][L, q], ref)
        else:
            _, dY, dn = iso_chain(m)
            for key, dc in (("Y", dY), ("nu", dn)):
                ref = float(np.dot(w, G.energy_derivative(desc, ("material", L, key))))
                got = float(np.dot(g["moduli"][L], dc))
                assert abs(got - ref) <= max(tol, 1e-6) * abs(ref), (L, key, got, ref)


def test_gradient_matches_gpu_finite_differences_and_autograd():
    from paper_2111_06893_gb300 import thermonoise
    desc = thin_cylinder()
    EnergyFn = thermonoise.energy_fn()
    slab_z = torch.tensor(desc["slab_z"], dtype=torch.float64, requires_grad=True)
    r0 = torch.tensor(desc["beam"]["r0"], dtype=torch.float64, requires_grad=True)
    mod = torch.tensor([thermonoise.iso_moduli(m["Y"], m["nu"]) if m["kind"] == "iso"
                        else (m["c11"], m["c12"], m["c44"]) for m in desc["materials"]],
                       dtype=torch.float64, requires_grad=True)
    kw = {"mode": "f64", "rtol": 1e-13, "energy_rtol": 1e-13, "raise_on_error": False}
    U = EnergyFn.apply(slab_z, r0, mod, desc, kw)
    J = U[0] * 2.0 + U[1] + 0.5 * U[-1]
    J.backward()

    def Jval(sz, rr):
        with torch.no_grad():
            V = EnergyFn.apply(sz, rr, mod, desc, kw)
        return float(V[0] * 2.0 + V[1] + 0.5 * V[-1])

    # thickness of the first coating layer: moves slab_z[1:] ... only slab_z[1] here
    h = 1e-6
    e1 = torch.zeros_like(slab_z)
    e1[1] = h
    fd = (Jval(slab_z.detach() + e1, r0.detach()) - Jval(slab_z.detach() - e1, r0.detach())) / (2 * h)
    assert abs(slab_z.grad[1].item() - fd) <= 1e-5 * abs(fd), (slab_z.grad[1].item(), fd)
    fd = (Jval(slab_z.detach(), r0.detach() + h) - Jval(slab_z.detach(), r0.detach() - h)) / (2 * h)
    assert abs(r0.grad.item() - fd) <= 1e-5 * abs(fd), (r0.grad.item(), fd)


def test_single_coating_full_size_gradient_matches_finite_differences():
    """Adjoint gradients on the 2.0 M DOF mirror against central differences
    of GPU solves, for parameters the energies depend on smoothly: the beam
    width r0 and the moduli (slab positions of geometric substrate slabs sit
    on kinks of min(h_int, h_ext))."""
    from paper_2111_06893_gb300 import thermonoise
    desc = W.single_coating()
    EnergyFn = thermonoise.energy_fn()
    slab_z = torch.tensor(desc["slab_z"], dtype=torch.float64)
    r0 = torch.tensor(desc["beam"]["r0"], dtype=torch.float64, requires_grad=True)
    mod = torch.tensor([thermonoise.iso_moduli(m["Y"], m["nu"]) for m in desc["materials"]],
                       dtype=torch.float64, requires_grad=True)
    kw = {"mode": "f64", "rtol": 1e-13, "energy_rtol": 1e-14, "raise_on_error": False}
    U = EnergyFn.apply(slab_z, r0, mod, desc, kw)
    J = 3.0 * U[0] + U[1]
    J.backward()

    def Jval(rr, mm):
        with torch.no_grad():
            V = EnergyFn.apply(slab_z, rr, mm, desc, kw)
        return float(3.0 * V[0] + V[1])

    h = 1e-5
    fd = (Jval(r0.detach() + h, mod.detach()) - Jval(r0.detach() - h, mod.detach())) / (2 * h)
    assert abs(r0.grad.item() - fd) <= 1e-5 * abs(fd), (r0.grad.item(), fd)
    for (L, q) in ((0, 2), (1, 0)):  # coating c44, substrate c11
        dm = torch.zeros_like(mod)
        hm = 1e-5 * abs(mod[L, q].item())
        dm[L, q] = hm
        fd = (Jval(r0.detach(), mod.detach() + dm) - Jval(r0.detach(), mod.detach() - dm)) / (2 * hm)
        assert abs(mod.grad[L, q].item() - fd) <= 1e-5 * abs(fd), (L, q, mod.grad[L, q].item(), fd)
