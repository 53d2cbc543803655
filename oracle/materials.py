"""Constitutive relations Y^{ijkl} (Sec. 2.1).

Isotropic: Eq. (constrel_iso) with the Lame parameter and shear modulus
obtained from Young's modulus and the Poisson ratio by inverting the
footnote to Eq. (constrel_iso).  Cubic crystal: Eq. (constrel_cryst), with the
crystal axes along x, y, z.

Test infrastructure: slow, plain FP64, imported only by tests and by the
CPU-baseline leg of the benchmark.
"""
import numpy as np


def lame_from_young(Y, nu):
    """lambda, mu from Y = mu (3 lambda + 2 mu) / (lambda + mu) and
    nu = lambda / (2 (lambda + mu))."""
    mu = Y / (2.0 * (1.0 + nu))
    lam = 2.0 * mu * nu / (1.0 - 2.0 * nu)
    return lam, mu


def young_from_lame(lam, mu):
    """The footnote's forward relations (also giving the bulk modulus)."""
    K = lam + 2.0 * mu / 3.0
    Y = 9.0 * K * mu / (3.0 * K + mu)
    nu = (3.0 * K - 2.0 * mu) / (2.0 * (3.0 * K + mu))
    return Y, nu, K


def iso_tensor(lam, mu):
    d = np.eye(3)
    return (lam * np.einsum("ij,kl->ijkl", d, d)
            + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))


def cubic_tensor(c11, c12, c44):
    Y = np.zeros((3, 3, 3, 3), dtype=np.result_type(c11, c12, c44, float))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    if i == j == k == l:
                        Y[i, j, k, l] = c11
                    elif i == j and k == l and i != k:
                        Y[i, j, k, l] = c12
                    elif (i == k and j == l and i != j) or (i == l and j == k and i != j):
                        Y[i, j, k, l] = c44
    return Y


def tensor(mat):
    if mat["kind"] == "iso":
        return iso_tensor(*lame_from_young(mat["Y"], mat["nu"]))
    if mat["kind"] == "cubic":
        return cubic_tensor(mat["c11"], mat["c12"], mat["c44"])
    raise ValueError(mat["kind"])
