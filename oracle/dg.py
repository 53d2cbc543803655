"""The DG operator of Sec. 2.2, written out as explicit element matrices.

Discretisation (Sec. 2.2.2, Eqs. (massmat)-(liftop), (dg_residuals)):
nodal Lagrange basis on LGL points, LGL quadrature everywhere, so the mass
matrix is diagonal, M = w detJ, and the lifting operator is diagonal on face
nodes, L = w^Sigma J^Sigma / (w detJ).  The auxiliary strain is lifted with
the flux of Eq. (numfluxaux), the primal flux is the generalized internal
penalty flux of Eq. (numfluxprimal) with the averaged constitutive relation
Y_* of Eq. (constrel_avg), and the penalty is Eq. (penalty) with p the
polynomial degree and h = 2 detJ / J^Sigma at each face node (minimum over the
two sides).  Boundary conditions enter through exterior values, Eq. (bc).

This module builds the operator in the weak form that integrates the
divergence of Eq. (dg_residuals) by parts:

  a(v, u) = sum_e sum_p w_p detJ_p grad v : Y : grad u
          - sum_faces sum_q w^S_q J^S_q ( [[v]] . n.{Y grad u}
                                         + n.{Y grad v} . [[u]]
                                         - sigma [[v]] . (n.Y_*.n) [[u]] )

with [[u]] = u_int - u_ext, n the outward normal of the interior side and
{.} the average.  On affine elements LGL quadrature satisfies summation by
parts and this equals the strong form of Eq. (dg_residuals) exactly
(``strong_residual`` below follows the paper's strong form step by step, and
a test shows the two agree); on curved elements the weak form is the one
that stays exactly symmetric.  Dirichlet faces use u_ext = 2 u_b - u_int and
the interior stress; Neumann faces use the prescribed traction and no jump.

Sign conventions: T = -Y S (Eq. (Hooke)), so the operator is positive
definite and the beam load n_i T^ij_b = n^j p(r) on z = 0 gives
b = -sum_top w^S J^S p(r) n.

Test infrastructure: slow, plain FP64, imported only by tests and by the
CPU-baseline leg of the benchmark.
"""
import numpy as np
import scipy.sparse as sp

from . import materials


class Operator:
    def __init__(self, mesh):
        self.mesh = mesh
        N = mesh.N
        I = np.eye(N)
        D = mesh.D
        # logical derivative matrices on the element (node p = (k N + j) N + i)
        self.Dlog = [np.kron(I, np.kron(I, D)), np.kron(I, np.kron(D, I)),
                     np.kron(D, np.kron(I, I))]
        self.Y = [materials.tensor(m) for m in mesh.desc["materials"]]
        self.C = mesh.desc["penalty_C"]
        self.dtype = np.result_type(mesh.slab_z, *[Y.dtype for Y in self.Y], mesh.desc["beam"]["r0"], float)
        self._G = {}

    # ------------------------------------------------------------ pieces
    def grad_matrices(self, e):
        """G[a][r, q] = d psi_q / dx^a at node r (chain rule through J^-1)."""
        if e in self._G:
            return self._G[e]
        Jinv = self.mesh.geometry(e)["Jinv"]
        G = [sum(Jinv[:, m, a][:, None] * self.Dlog[m] for m in range(3))
             for a in range(3)]
        if len(self._G) > 2048:
            self._G.clear()
        self._G[e] = G
        return G

    def Ye(self, e):
        return self.Y[self.mesh.layer(e)]

    def volume_matrix(self, e):
        """K[(c,q),(d,r)] = sum_p w_p detJ_p dpsi_q/dx^a Y^{acbd} dpsi_r/dx^b."""
        G = self.grad_matrices(e)
        wJ = self.mesh.geometry(e)["wJ"]
        Y = self.Ye(e)
        n = self.mesh.n
        K = np.zeros((3, n, 3, n), dtype=self.dtype)
        for a in range(3):
            for b in range(3):
                Mab = G[a].T @ (wJ[:, None] * G[b])
                for c in range(3):
                    for d in range(3):
                        if Y[a, c, b, d] != 0.0:
                            K[c, :, d, :] += Y[a, c, b, d] * Mab
        return K.reshape(3 * n, 3 * n)

    def value_op(self, F):
        """V[(c,q),(c,F[q])] = 1: face values of the three components."""
        n, m = self.mesh.n, len(F)
        V = np.zeros((3 * m, 3 * n))
        for c in range(3):
            V[c * m + np.arange(m), c * n + F] = 1.0
        return V

    def traction_op(self, e, F, nvec):
        """(Tr u)_j(q) = n_a(q) Y^{ajbl} du_l/dx^b at node F[q] of element e
        (unlifted derivative, as in Eq. (numfluxprimal))."""
        G = self.grad_matrices(e)
        Y = self.Ye(e)
        n, m = self.mesh.n, len(F)
        Tr = np.zeros((3, m, 3, n), dtype=self.dtype)
        for j in range(3):
            for l in range(3):
                for b in range(3):
                    coef = np.einsum("qa,a->q", nvec, Y[:, j, b, l])
                    if np.any(coef != 0.0):
                        Tr[j, :, l, :] += coef[:, None] * G[b][F, :]
        return Tr.reshape(3 * m, 3 * n)

    def penalty_op(self, nvec, Ystar, sigma):
        """Pen[(j,q),(l,q)] = sigma(q) n_a Y_*^{ajbl} n_b."""
        m = len(sigma)
        Mq = np.einsum("qa,ajbl,qb->qjl", nvec, Ystar, nvec) * sigma[:, None, None]
        P = np.zeros((3, m, 3, m), dtype=self.dtype)
        for j in range(3):
            for l in range(3):
                P[j, np.arange(m), l, np.arange(m)] = Mq[:, j, l]
        return P.reshape(3 * m, 3 * m)

    def sigma(self, h):
        p = self.mesh.p
        return self.C * (p + 1) ** 2 / h

    @staticmethod
    def h_min(h1, h2):
        """min(h_int, h_ext) of Eq. (penalty), node by node.  For real h it
        is the minimum.  Under a complex step (derivatives) two sides whose
        real parts agree to 1e-12 relative count as a tie (equal layer
        thicknesses meet there, computed from slab positions with rounding):
        the value is the smaller real part and the derivative the smaller of
        the two, i.e. the derivative for an increasing parameter, which is
        the same seen from both elements of the face."""
        if not (np.iscomplexobj(h1) or np.iscomplexobj(h2)):
            return np.minimum(h1, h2)
        h1 = np.asarray(h1, dtype=complex)
        h2 = np.asarray(h2, dtype=complex)
        r1, r2 = h1.real, h2.real
        tie = np.abs(r1 - r2) <= 1e-12 * np.maximum(np.abs(r1), np.abs(r2))
        tied = np.minimum(r1, r2) + 1j * np.minimum(h1.imag, h2.imag)
        return np.where(tie, tied, np.where(r1 < r2, h1, h2))

    # ---------------------------------------------------------- the rows
    def element_rows(self, e):
        """Blocks {e2: A[e-rows, e2-cols]} of the weak-form operator."""
        mesh = self.mesh
        blocks = {e: self.volume_matrix(e)}
        for f in range(6):
            bc = mesh.boundary_condition(e, f)
            if bc == "neumann":
                continue
            fg = mesh.face_geometry(e, f)
            F, nvec = fg["F"], fg["n"]
            W = np.tile(fg["W"], 3)
            V = self.value_op(F)
            Tr = self.traction_op(e, F, nvec)
            if bc == "dirichlet":
                Pen = self.penalty_op(nvec, self.Ye(e), self.sigma(fg["h"]))
                blocks[e] += (-(V.T @ (W[:, None] * Tr)) - (Tr.T @ (W[:, None] * V))
                              + 2.0 * V.T @ (W[:, None] * Pen @ V))
                continue
            e2, f2 = int(mesh.neighbour[e, f]), int(mesh.nb_face[e, f])
            perm = mesh.face_perm(e, f)
            F2 = mesh.face_nodes(f2)[perm]
            h2 = mesh.face_geometry(e2, f2)["h"][perm]
            sig = self.sigma(self.h_min(fg["h"], h2))
            Ystar = 0.5 * (self.Ye(e) + self.Ye(e2))
            Pen = self.penalty_op(nvec, Ystar, sig)
            V2 = self.value_op(F2)
            Tr2 = self.traction_op(e2, F2, nvec)
            blocks[e] += (-0.5 * (V.T @ (W[:, None] * Tr)) - 0.5 * (Tr.T @ (W[:, None] * V))
                          + V.T @ (W[:, None] * Pen @ V))
            off = (-0.5 * (V.T @ (W[:, None] * Tr2)) + 0.5 * (Tr.T @ (W[:, None] * V2))
                   - V.T @ (W[:, None] * Pen @ V2))
            blocks[e2] = blocks.get(e2, 0.0) + off
        return blocks

    def assemble(self):
        """The global sparse matrix A of Eq. (matrix_eqn)."""
        mesh = self.mesh
        nloc = 3 * mesh.n
        rows, cols, vals = [], [], []
        ii, jj = np.meshgrid(np.arange(nloc), np.arange(nloc), indexing="ij")
        for e in range(mesh.E):
            for e2, B in self.element_rows(e).items():
                nz = B != 0.0
                rows.append(e * nloc + ii[nz])
                cols.append(e2 * nloc + jj[nz])
                vals.append(B[nz])
        rows, cols, vals = (np.concatenate(a) for a in (rows, cols, vals))
        return sp.csr_matrix((vals, (rows, cols)), shape=(mesh.ndof, mesh.ndof))

    def apply_element(self, e, u):
        """Rows of element e of A u, without assembling the rest."""
        nloc = 3 * self.mesh.n
        y = np.zeros(nloc, dtype=np.result_type(self.dtype, u))
        for e2, B in self.element_rows(e).items():
            y += B @ u[e2 * nloc:(e2 + 1) * nloc]
        return y

    # ------------------------------------------------------- right side
    def rhs(self, dirichlet=None, neumann=None):
        """b = -residual(u = 0): the beam pressure on the top (Neumann,
        n_i T^ij_b = n^j p(r) with p of Eq. (laserbeam)) plus, for tests, any
        inhomogeneous data: dirichlet(x) -> u_b on fixed faces and
        neumann(x, n, where) -> n_i T^ij_b on free faces."""
        mesh = self.mesh
        beam = mesh.desc["beam"]
        r0, F0 = beam["r0"], beam["F0"]
        nloc = 3 * mesh.n
        b = np.zeros(mesh.ndof, dtype=self.dtype)
        for e in range(mesh.E):
            be = np.zeros(nloc, dtype=self.dtype)
            for f in range(6):
                bc = mesh.boundary_condition(e, f)
                if bc == "interior":
                    continue
                fg = mesh.face_geometry(e, f)
                F, nvec, x = fg["F"], fg["n"], fg["xyz"]
                W = np.tile(fg["W"], 3)
                V = self.value_op(F)
                if bc == "neumann":
                    where = mesh.bkind[e, f]
                    if neumann is not None:
                        t = neumann(x, nvec, where)
                    elif where == "top":
                        r2 = x[:, 0] ** 2 + x[:, 1] ** 2
                        p = F0 * np.exp(-r2 / r0 ** 2) / (np.pi * r0 ** 2)
                        t = nvec * p[:, None]
                    else:
                        t = np.zeros_like(x)
                    be -= V.T @ (W * t.T.ravel())
                elif dirichlet is not None:
                    ub = dirichlet(x).T.ravel()
                    Tr = self.traction_op(e, F, nvec)
                    Pen = self.penalty_op(nvec, self.Ye(e), self.sigma(fg["h"]))
                    be += -(Tr.T @ (W * ub)) + 2.0 * V.T @ (W * (Pen @ ub))
            b[e * nloc:(e + 1) * nloc] = be
        return b

    # ---------------------------------------------- the paper's strong form
    def strong_residual(self, u):
        """Eq. (dg_residuals) evaluated step by step for homogeneous boundary
        data: S = D_(k u_l) + L((n_(k u_l))^* - n_(k u_l)), then
        -MD_i Y S - ML ((n_i Y S)^* - n_i Y S), with the fluxes of Eq. (numflux)
        and the exterior values of Eq. (bc)."""
        mesh = self.mesh
        n, nloc = mesh.n, 3 * mesh.n
        out = np.zeros(mesh.ndof)
        for e in range(mesh.E):
            ue = u[e * nloc:(e + 1) * nloc].reshape(3, n)
            G = self.grad_matrices(e)
            geo = mesh.geometry(e)
            Y = self.Ye(e)
            grad = np.stack([G[a] @ ue.T for a in range(3)], axis=1)  # (n, a, l)
            S = 0.5 * (grad + grad.transpose(0, 2, 1))
            lift = np.zeros((n, 3, 3))
            flux_terms = []
            for f in range(6):
                bc = mesh.boundary_condition(e, f)
                fg = mesh.face_geometry(e, f)
                F, nvec, Wf = fg["F"], fg["n"], fg["W"]
                tr_int = np.einsum("qa,ajbl,qbl->qj", nvec, Y, grad[F])
                if bc == "interior":
                    e2, f2 = int(mesh.neighbour[e, f]), int(mesh.nb_face[e, f])
                    perm = mesh.face_perm(e, f)
                    F2 = mesh.face_nodes(f2)[perm]
                    u2 = u[e2 * nloc:(e2 + 1) * nloc].reshape(3, n)
                    G2 = self.grad_matrices(e2)
                    grad2 = np.stack([G2[a][F2] @ u2.T for a in range(3)], axis=1)
                    Y2 = self.Ye(e2)
                    jump = ue[:, F].T - u2[:, F2].T
                    nu_star_minus = -0.5 * jump  # {u} - u_int
                    h2 = mesh.face_geometry(e2, f2)["h"][perm]
                    sig = self.sigma(self.h_min(fg["h"], h2))
                    Ystar = 0.5 * (Y + Y2)
                    tr_ext = np.einsum("qa,ajbl,qbl->qj", nvec, Y2, grad2)
                    pen = sig[:, None] * np.einsum("qa,ajbl,qb,ql->qj", nvec, Ystar, nvec, jump)
                    flux_star = 0.5 * (tr_int + tr_ext) - pen
                elif bc == "dirichlet":
                    nu_star_minus = -ue[:, F].T  # u_b - u_int with u_b = 0
                    sig = self.sigma(fg["h"])
                    pen = sig[:, None] * np.einsum("qa,ajbl,qb,ql->qj", nvec, Y, nvec, ue[:, F].T)
                    flux_star = tr_int - 2.0 * pen
                else:
                    nu_star_minus = np.zeros((len(F), 3))
                    flux_star = np.zeros((len(F), 3))  # n_i T^ij_b = 0
                g = 0.5 * (np.einsum("qk,ql->qkl", nvec, nu_star_minus)
                           + np.einsum("ql,qk->qkl", nvec, nu_star_minus))
                np.add.at(lift, F, g * (Wf / geo["wJ"][F])[:, None, None])
                flux_terms.append((F, nvec, Wf, flux_star))
            S = S + lift
            YS = np.einsum("ijkl,pkl->pij", Y, S)
            res = np.zeros((n, 3))
            for i in range(3):
                res -= geo["wJ"][:, None] * (G[i] @ YS[:, i, :])
            for F, nvec, Wf, flux_star in flux_terms:
                nYS = np.einsum("qi,qij->qj", nvec, YS[F])
                np.add.at(res, F, -Wf[:, None] * (flux_star - nYS))
            out[e * nloc:(e + 1) * nloc] = res.T.ravel()
        return out
