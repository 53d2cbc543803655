"""Solve and post-process (Secs. 2.1 and 2.3).

* ``solve``: the linear system A u = b of Eq. (matrix_eqn), solved directly
  (sparse LU) so that the oracle has no iteration error.
* ``layer_energies``: U = -1/2 int S_ij T^ij dV with T = -Y S (Sec. 2.1),
  i.e. 1/2 int S : Y : S, evaluated per material layer with the element's own
  (unlifted) strain S = D_(k u_l) at its LGL nodes and LGL weights.
* ``layer_energy_parts``: the same energies split by elastic modulus
  (dilatational, tetragonal and shear strain subspaces of the stiffness).
* ``noise_psd``: the fluctuation-dissipation relation, Eq. (thermalnoise),
  with the quasistatic loss of Eq. (wdiss) summed over layers.  Taken as a
  dissipated power (energy per cycle 2 pi U phi, times f) this reads
  S_q = 4 k_B T sum_i phi_i U_i / (pi f F0^2); only this constant is a
  reading, S_q proportional to sum_i phi_i U_i is the paper's.
* ``half_space_energy``: closed-form energy of an isotropic half-space under
  the pressure profile of Eq. (laserbeam), (1 - nu^2) F0^2 / (2 sqrt(2 pi) Y r0),
  and the same number by quadrature of the Boussinesq surface response.
* ``thin_coating_energy``: the coating's energy to first order in its
  thickness on an isotropic half-space (the limit behind the approximate
  noise formula Eq. (approx_analytic)), from the substrate's surface strain.

Test infrastructure: slow, plain FP64, imported only by tests and by the
CPU-baseline leg of the benchmark.
"""
import math

import numpy as np
import scipy.sparse.linalg as spla
from scipy import integrate, special

from .materials import lame_from_young

BOLTZMANN = 1.380649e-23


def solve(A, b):
    return spla.splu(A.tocsc()).solve(b)


def element_energy(op, e, u):
    mesh = op.mesh
    n, nloc = mesh.n, 3 * mesh.n
    ue = u[e * nloc:(e + 1) * nloc].reshape(3, n)
    G = op.grad_matrices(e)
    grad = np.stack([G[a] @ ue.T for a in range(3)], axis=1)  # (n, a, l) = du_l/dx^a
    S = 0.5 * (grad + grad.transpose(0, 2, 1))
    dens = np.einsum("pij,ijkl,pkl->p", S, op.Ye(e), S)
    return 0.5 * np.sum(mesh.geometry(e)["wJ"] * dens)


def layer_energies(op, u):
    """U_i per layer id (coating layers top-down, the substrate last)."""
    U = np.zeros(op.mesh.n_layers, dtype=np.result_type(op.dtype, u))
    for e in range(op.mesh.E):
        U[op.mesh.layer(e)] += element_energy(op, e, u)
    return U


def _kelvin(S):
    """Strain tensors (..., 3, 3) as Kelvin 6-vectors (S11, S22, S33,
    sqrt2 S23, sqrt2 S13, sqrt2 S12), in which S : Y : S = s . C s."""
    r2 = np.sqrt(2.0)
    return np.stack([S[..., 0, 0], S[..., 1, 1], S[..., 2, 2], r2 * S[..., 1, 2], r2 * S[..., 0, 2],
                     r2 * S[..., 0, 1]], axis=-1)


def _kelvin_matrix(Y):
    idx = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    sc = [1.0, 1.0, 1.0, np.sqrt(2.0), np.sqrt(2.0), np.sqrt(2.0)]
    return np.array([[sc[a] * sc[b] * Y[idx[a] + idx[b]] for b in range(6)] for a in range(6)])


def layer_energy_parts(op, u):
    """[n_layers, 3]: the layer energies split by elastic modulus, for loss
    angles attached to the independent moduli (Sec. 2.1 notes that a
    material can carry several).  Reading: the energy density 1/2 s . C s of
    the cubic-aligned (or isotropic) stiffness in Kelvin notation splits with
    the orthogonal projectors onto its invariant subspaces -- dilatation
    (1, 1, 1, 0, 0, 0)/sqrt3, the rest of the diagonal strains (tetragonal),
    and the shear strains -- which C leaves invariant, so that the three
    parts 1/2 s . P C P s add up to the energy."""
    v0 = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0]) / np.sqrt(3.0)
    P_dil = np.outer(v0, v0)
    P_tet = np.diag([1.0, 1.0, 1.0, 0.0, 0.0, 0.0]) - P_dil
    P_shr = np.diag([0.0, 0.0, 0.0, 1.0, 1.0, 1.0])
    mesh = op.mesh
    n, nloc = mesh.n, 3 * mesh.n
    out = np.zeros((mesh.n_layers, 3))
    for e in range(mesh.E):
        ue = u[e * nloc:(e + 1) * nloc].reshape(3, n)
        G = op.grad_matrices(e)
        grad = np.stack([G[a] @ ue.T for a in range(3)], axis=1)
        S = 0.5 * (grad + grad.transpose(0, 2, 1))
        s6 = _kelvin(S)
        C = _kelvin_matrix(op.Ye(e))
        wJ = mesh.geometry(e)["wJ"]
        for j, P in enumerate((P_dil, P_tet, P_shr)):
            dens = np.einsum("pa,ab,pb->p", s6, P @ C @ P, s6)
            out[mesh.layer(e), j] += 0.5 * np.sum(wJ * dens)
    return out


def noise_psd(U, phi, kB_T, f, F0):
    return 4.0 * kB_T * float(np.dot(phi, U)) / (math.pi * f * F0 ** 2)


def half_space_energy(Y, nu, F0, r0):
    return (1.0 - nu ** 2) * F0 ** 2 / (2.0 * math.sqrt(2.0 * math.pi) * Y * r0)


def half_space_energy_quadrature(Y, nu, F0, r0):
    """U = (1 - nu^2) / (2 pi Y) int_0^inf |p_hat(k)|^2 dk, from the surface
    response w_hat = 2 (1 - nu^2) p_hat / (Y k) of a half-space, with p_hat
    the Hankel transform of F0 p(r) computed by quadrature."""
    def p(r):
        return F0 * math.exp(-r * r / r0 ** 2) / (math.pi * r0 ** 2)

    def p_hat(k):
        val, _ = integrate.quad(lambda r: 2 * math.pi * r * p(r) * special.j0(k * r),
                                0.0, 12.0 * r0, limit=200)
        return val

    val, _ = integrate.quad(lambda k: p_hat(k) ** 2, 0.0, 16.0 / r0, limit=200)
    return (1.0 - nu ** 2) / (2.0 * math.pi * Y) * val


def thin_coating_energy(Yc, nuc, Ys, nus, d, F0, r0):
    """Energy of an isotropic coating (Yc, nuc) of thickness d << r0 on an
    isotropic half-space (Ys, nus) loaded by the beam pressure p(r) of
    Eq. (laserbeam), to first order in d.

    A thin coating follows the substrate's in-plane surface strain
    (continuous displacement) and carries the normal traction -p and no
    shear traction.  On a half-space a normal surface load moves the
    surface sideways by the gradient of a potential whose in-plane
    Laplacian is -(1 - 2 nus)(1 + nus) p / Ys (Boussinesq's point load gives
    the inward surface displacement (1 - 2 nu)(1 + nu) P / (2 pi Y r);
    loads superpose), so the in-plane strain trace there is e = -a p with
    a = (1 - 2 nus)(1 + nus) / Ys, and for a gradient field the integral of
    eps_ab eps_ab over the surface equals that of e^2.  The coating's Hooke
    law with sigma_zz = -p fixes eps_zz = -(1 - lam_c a) p / (lam_c + 2 mu_c),
    every term of the energy density is then a multiple of p^2, and
    int p^2 dA = F0^2 / (2 pi r0^2)."""
    lam, mu = lame_from_young(Yc, nuc)
    a = (1.0 - 2.0 * nus) * (1.0 + nus) / Ys
    e = -a                                  # in-plane strain trace per unit p
    ezz = -(1.0 - lam * a) / (lam + 2.0 * mu)  # normal strain per unit p
    two_w = lam * (e + ezz) * e + 2.0 * mu * e * e - ezz  # sigma : eps per unit p^2
    return 0.5 * d * two_w * F0 ** 2 / (2.0 * math.pi * r0 ** 2)


def solve_cg(op, A, b, rtol=1e-12, maxiter=20000):
    """A u = b by conjugate gradients preconditioned with the exact inverse of
    each element's diagonal block: the oracle's iterative solve for systems
    too large to factor (its result carries the iteration error rtol)."""
    import scipy.sparse as sp
    nl = 3 * op.mesh.n
    blocks = [sp.csr_matrix(np.linalg.inv(A[e * nl:(e + 1) * nl, e * nl:(e + 1) * nl].toarray()))
              for e in range(op.mesh.E)]
    Minv = sp.block_diag(blocks, format="csr")
    u, info = spla.cg(A, b, rtol=rtol, atol=0.0, M=Minv, maxiter=maxiter)
    if info != 0:
        raise RuntimeError(f"oracle CG did not converge (info={info})")
    return u


def solve_dense(A, b):
    """A u = b by dense Cholesky (fails loudly if A is not positive definite);
    complex-symmetric systems (complex-step derivatives) by dense LU."""
    import scipy.linalg as sl
    if np.iscomplexobj(A.data) or np.iscomplexobj(b):
        return sl.lu_solve(sl.lu_factor(A.toarray(), check_finite=False), b)
    c = sl.cho_factor(A.toarray(), lower=True, overwrite_a=True, check_finite=False)
    return sl.cho_solve(c, b)


def solve_refined(A, b, max_steps=12, info=None):
    """A u = b for the FP64 matrix A to well below FP64 rounding of a plain
    factorisation: classical iterative refinement (Wilkinson), x += A^-1 r
    with the residual r = b - A x formed in extended precision
    (np.longdouble: 64-bit significand on x86, IEEE quad on Arm) and the
    correction from one sparse LU of A in FP64.  Each step shrinks the error
    by about cond(A) eps64; it stops once a correction no longer shrinks.
    Thin coating layers give cond(A) ~ 1e8, where a plain FP64 solve keeps
    ~1e-9 relative error in the energies; this solve is the reference the
    GPU results are graded against there.  Complex systems (complex-step
    derivatives) are refined the same way in complex extended precision.
    Returns the solution in extended precision; info (a dict) receives the
    relative size of every correction."""
    cplx = np.iscomplexobj(A.data) or np.iscomplexobj(b)
    ext = np.clongdouble if cplx else np.longdouble
    work = np.complex128 if cplx else np.float64
    lu = spla.splu(A.tocsc().astype(work))
    Ae = A.tocsr().astype(ext)
    be = np.asarray(b).astype(ext)
    x = lu.solve(np.asarray(b, dtype=work)).astype(ext)
    steps = []
    for _ in range(max_steps):
        r = be - Ae @ x
        d = lu.solve(r.astype(work))
        x = x + d.astype(ext)
        steps.append(float(np.max(np.abs(d)) / np.max(np.abs(x))))
        if steps[-1] < 1e-17 or (len(steps) >= 3 and steps[-1] > 0.5 * steps[-3]):
            break
    if info is not None:
        info["corrections"] = steps
    return x
