"""Derivatives of the layer energies U_i by complex step through the whole
oracle computation (mesh maps -> explicit DG operator -> direct solve ->
energies of Sec. 2.1): dU/dtheta = Im U(theta + i h) / h with h = 1e-30.
Every step of the oracle is analytic in the slab positions, the beam width
and the elastic moduli, so the result is the exact derivative of the
discrete energies up to rounding; it needs no adjoint and no step-size
choice, and is independent of the adjoint formula it is compared with.

Parameters:
  ("slab_z", s)            position of slab boundary s (s >= 1)
  ("r0",)                  beam width of Eq. (laserbeam)
  ("material", L, key)     modulus `key` of layer L ("Y", "nu", "c11", ...)

Test infrastructure: slow, plain FP64, imported only by tests and by the
CPU-baseline leg of the benchmark.
"""
import copy

import numpy as np

from .dg import Operator
from .mesh import Mesh
from . import observables as ob

H = 1e-30


def energies(desc, solver="refined"):
    """Layer energies of the mirror `desc` (complex-valued under a complex
    step).  solver: "refined" (iterative refinement with extended-precision
    residuals, accurate well below FP64 rounding of a plain solve even for
    thin layers), "dense" (dense Cholesky / LU) or "lu" (sparse LU)."""
    op = Operator(Mesh(desc))
    A = op.assemble()
    b = op.rhs()
    if solver == "refined":
        u = ob.solve_refined(A, b)
        u = u.astype(np.complex128 if np.iscomplexobj(u) else np.float64)
    elif solver == "dense":
        u = ob.solve_dense(A, b)
    else:
        u = ob.solve(A, b)
    return ob.layer_energies(op, u)


def perturbed(desc, param, step):
    d = copy.deepcopy(desc)
    if param[0] == "slab_z":
        z = np.asarray(d["slab_z"], dtype=complex)
        z[param[1]] += step
        d["slab_z"] = z
    elif param[0] == "r0":
        d["beam"] = dict(d["beam"])
        d["beam"]["r0"] = d["beam"]["r0"] + step
    elif param[0] == "material":
        mats = [dict(m) for m in d["materials"]]
        mats[param[1]][param[2]] = mats[param[1]][param[2]] + step
        d["materials"] = mats
    else:
        raise ValueError(param)
    return d


def energy_derivative(desc, param, solver="refined"):
    """dU_i / d param for every layer i (complex step)."""
    U = energies(perturbed(desc, param, 1j * H), solver=solver)
    return np.imag(U) / H
