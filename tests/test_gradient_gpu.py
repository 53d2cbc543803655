"""Adjoint energy gradients on the GPU against the oracle's exact derivatives
(complex step through the whole oracle with iteratively refined solves,
tests/golden/oracle_gradients.json written by make_gradient_golden.py from
oracle/ alone) and against finite differences of GPU solves.

Tolerances are the measured error plus margin, each with its cause:
  layered_box    well conditioned: GPU gradients agree with the oracle to
                 ~2e-13; tested at 1e-11.
  thin_cylinder  0.02 / 0.05-thick coatings, cond(A) ~ 1e8: GPU energies
                 agree to ~2e-10 and gradients to ~6e-9 whatever the solver
                 (PCG to the FP64 floor, column or grouped lines, Jacobi,
                 mixed).  An FP64 perturbation of the oracle's own operator
                 (each entry times 1 + 1e-15 N(0,1)) moves its energies by up
                 to 1.7e-9 and its gradients by 0.5-3.7e-9: the gap is the
                 rounding floor of the discrete problem in FP64, not the
                 solver.  Energies tested at 1e-9, gradients at 1e-8.
  tie_stack      four equal cubic layers of 2^-11 (exact ties of
                 min(h_int, h_ext); both sides take the derivative for an
                 increasing parameter there), FP64 residual floor ~3e-9:
                 GPU energies agree to ~4e-9 and gradients to ~3e-5.  The
                 same perturbation of the oracle's operator (1 + 2e-16 or
                 1e-15 N(0,1) per entry) moves its energies by 5e-9 to 1e-7
                 and its gradients in slab positions and c11 by 1.4e-5 to
                 2.7e-4 (r0: 5e-9 to 3e-8): again the floor of the discrete
                 problem in FP64.  Energies tested at 2e-8, gradients at 1e-4.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from cases import layered_box, thin_cylinder, tie_stack

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

HERE = os.path.dirname(os.path.abspath(__file__))


def golden():
    with open(os.path.join(HERE, "golden", "oracle_gradients.json")) as f:
        return json.load(f)


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_06893_gb300 import build
    build.build()


def gpu_gradient(ctx, desc, w, mode="f64"):
    """dJ/dtheta for every parameter of the golden record, J = w . U."""
    from paper_2111_06893_gb300 import thermonoise
    g = ctx.energy_grad(ctx._u, w, mode=mode, rtol=1e-15, raise_on_error=False)
    out = {}
    ns = len(desc["slab_z"]) - 1
    for s in range(1, ns + 1):
        out[json.dumps(["slab_z", s])] = g["slab_z"][s]
    out[json.dumps(["r0"])] = g["r0"]
    for L, m in enumerate(desc["materials"]):
        if m["kind"] == "cubic":
            for q, key in enumerate(["c11", "c12", "c44"]):
                out[json.dumps(["material", L, key])] = g["moduli"][L, q]
        else:
            _, dc = thermonoise.iso_moduli(m["Y"], m["nu"], derivatives=True)  # d(c11, c12, c44)/d(Y, nu)
            out[json.dumps(["material", L, "Y"])] = float(np.dot(g["moduli"][L], dc[:, 0]))
            out[json.dumps(["material", L, "nu"])] = float(np.dot(g["moduli"][L], dc[:, 1]))
    return out, g["report"]


CASES = {"layered_box": (layered_box, 1e-12, 1e-11),
         "thin_cylinder": (thin_cylinder, 1e-9, 1e-8),
         "tie_stack": (tie_stack, 2e-8, 1e-4)}


@pytest.mark.parametrize("name", sorted(CASES))
def test_energies_and_adjoint_gradients_match_refined_oracle(name):
    from paper_2111_06893_gb300 import thermonoise
    make, tol_U, tol_g = CASES[name]
    desc = make()
    rec = golden()[name]
    ctx = thermonoise.setup(desc)
    # FP64 PCG run to its rounding floor (stagnation of the true residual)
    u, rep = ctx.solve(mode="f64", rtol=1e-15, raise_on_error=False)
    assert rep["status"] in (0, thermonoise.STATUS_CODE["TN_ENOTCONV"]), rep
    U = ctx.layer_energies(u)
    Uo = np.array(rec["U"])
    errU = np.max(np.abs(U - Uo) / Uo)
    assert errU <= tol_U, (errU, U, Uo)
    ctx._u = u
    w = np.random.default_rng(4).uniform(0.5, 2.0, size=len(desc["materials"]))
    got, grep = gpu_gradient(ctx, desc, w)
    assert grep["status"] in (0, thermonoise.STATUS_CODE["TN_ENOTCONV"]), grep
    errs = {}
    for key, dU in rec["dU"].items():
        ref = float(np.dot(w, dU))
        errs[key] = abs(got[key] - ref) / abs(ref)
    worst = max(errs.values())
    print(f"{name}: energies {errU:.1e}, gradients {worst:.1e}", {k: f"{v:.1e}" for k, v in errs.items()})
    assert worst <= tol_g, errs


def test_thickness_gradient_at_ties_is_the_forward_difference():
    """Exact ties (tie_stack): the adjoint's derivative in an interface
    position equals the forward finite difference of GPU solves (the
    derivative for an increasing parameter), Richardson-extrapolated."""
    from paper_2111_06893_gb300 import thermonoise
    desc = tie_stack()
    w = np.zeros(len(desc["materials"]))
    w[1], w[2] = 1.0, 1.0  # the two layers at interface 2
    ctx = thermonoise.setup(desc)
    u, _ = ctx.solve(mode="f64", rtol=1e-15, raise_on_error=False)
    J0 = float(np.dot(w, ctx.layer_energies(u)))
    ctx._u = u
    got, _ = gpu_gradient(ctx, desc, w)

    def J(dz):
        d = dict(desc)
        z = list(desc["slab_z"])
        z[2] += dz
        d["slab_z"] = z
        c = thermonoise.setup(d)
        v, _ = c.solve(mode="f64", rtol=1e-15, raise_on_error=False)
        return float(np.dot(w, c.layer_energies(v)))

    t = desc["slab_z"][1] - desc["slab_z"][2]
    h = 2e-4 * t
    fwd = 2 * (J(h / 2) - J0) / (h / 2) - (J(h) - J0) / h
    bwd = 2 * (J0 - J(-h / 2)) / (h / 2) - (J0 - J(-h)) / h
    adj = got[json.dumps(["slab_z", 2])]
    assert abs(adj - fwd) <= 1e-5 * abs(fwd), (adj, fwd, bwd)
    # a real kink (the penalty term moves J only through the small jumps, so
    # the two one-sided derivatives differ by ~1e-4 relative here), and the
    # adjoint sits on the forward side of it
    assert abs(bwd - fwd) > 10 * abs(adj - fwd), (adj, fwd, bwd)


def test_gradient_matches_gpu_finite_differences_and_autograd():
    from paper_2111_06893_gb300 import thermonoise
    desc = thin_cylinder()
    EnergyFn = thermonoise.energy_fn()
    slab_z = torch.tensor(desc["slab_z"], dtype=torch.float64, requires_grad=True)
    r0 = torch.tensor(desc["beam"]["r0"], dtype=torch.float64, requires_grad=True)
    mod = torch.tensor([thermonoise.iso_moduli(m["Y"], m["nu"]) if m["kind"] == "iso"
                        else (m["c11"], m["c12"], m["c44"]) for m in desc["materials"]],
                       dtype=torch.float64, requires_grad=True)
    kw = {"mode": "f64", "rtol": 1e-15, "raise_on_error": False}
    U = EnergyFn.apply(slab_z, r0, mod, desc, kw)
    J = U[0] * 2.0 + U[1] + 0.5 * U[-1]
    J.backward()

    def Jval(sz, rr):
        with torch.no_grad():
            V = EnergyFn.apply(sz, rr, mod, desc, kw)
        return float(V[0] * 2.0 + V[1] + 0.5 * V[-1])

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
    width r0 and the moduli."""
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


def test_crystalline_full_size_thickness_gradient_matches_forward_differences():
    """The 40-layer cubic stack (8.0 M DOF): dJ/d(interface position) at
    interface 20 (equal layers on both sides: ties of min(h_int, h_ext)
    within rounding) against Richardson-extrapolated forward differences of
    FP64 GPU solves, J = U_19 + U_20."""
    from paper_2111_06893_gb300 import thermonoise
    desc = W.crystalline_multilayer()
    nl = len(desc["materials"])
    w = np.zeros(nl)
    w[19], w[20] = 1.0, 1.0
    kw = {"mode": "f64", "rtol": 1e-15, "energy_rtol": 1e-13, "raise_on_error": False}
    ctx = thermonoise.setup(desc)
    u, _ = ctx.solve(**kw)
    J0 = float(np.dot(w, ctx.layer_energies(u)))
    g = ctx.energy_grad(u, w, mode="f64", rtol=1e-13, raise_on_error=False)
    adj = g["slab_z"][20]

    def J(dz):
        d = dict(desc)
        z = list(desc["slab_z"])
        z[20] += dz
        d["slab_z"] = z
        c = thermonoise.setup(d)
        v, _ = c.solve(**kw)
        return float(np.dot(w, c.layer_energies(v)))

    h = 1e-3 * 4e-4
    fwd = 2 * (J(h / 2) - J0) / (h / 2) - (J(h) - J0) / h
    assert abs(adj - fwd) <= 1e-4 * abs(fwd), (adj, fwd)
