"""Domain decomposition and element geometry (Sec. 2.2.1 and Fig. 1).

The mirror is a box or a cylinder cut into hexahedral elements.  The cylinder
cross-section is a central square enveloped by four wedges, surrounded by four
outer wedges (Fig. 1, top); in z it is cut into slabs that follow the material
layers, with a logarithmic map in depth inside the substrate slabs.  Each
element carries a map x(xi) from the reference cube [-1, 1]^3; its Jacobian
J^i_j = dx^i / dxi^j, determinant and inverse are taken here by complex-step
differentiation of the map, so that no derivative is written out by hand.

Neighbours are found from physical coordinates (face centres and face nodes),
not from the element numbering, and boundary faces are classified by where
they lie (top z = 0, bottom, sides).

Every element map here is a cross-section map (X, Y)(xi, eta) times a
vertical map Z(zeta).  ``geometry`` takes the 2x2 cross-section Jacobian by
complex step and dZ/dzeta from its closed form, so that the whole oracle stays
analytic in the slab positions and can itself be differentiated by complex
step (gradients); ``jacobian`` (full 3-D complex step) pins the two against
each other.

Test infrastructure: slow, plain FP64, imported only by tests and by the
CPU-baseline leg of the benchmark.
"""
import numpy as np
from scipy.spatial import cKDTree

from .lgl import diff_matrix, lgl_nodes_weights

_CSTEP = 1e-30


def _rot(r, X, Y):
    """Rotation by r * 90 degrees, written with exact integer coefficients."""
    if r == 0:
        return X, Y
    if r == 1:
        return -Y, X
    if r == 2:
        return -X, -Y
    return Y, -X


class Mesh:
    def __init__(self, desc):
        self.desc = desc
        self.p = int(desc["degree"])
        self.N = self.p + 1
        self.n = self.N ** 3
        self.nodes, self.weights = lgl_nodes_weights(self.N)
        self.D = diff_matrix(self.nodes)
        self.kind = desc["kind"]
        if self.kind == "box":
            self.nx = len(desc["x_breaks"]) - 1
            self.ny = len(desc["y_breaks"]) - 1
            self.ncol = self.nx * self.ny
        elif self.kind == "cylinder":
            self.k = int(desc["k"])
            self.ncol = 9 * self.k ** 2
        else:
            raise ValueError(desc["kind"])
        self.slab_z = np.asarray(desc["slab_z"])
        self.nslab = len(self.slab_z) - 1
        self.E = self.ncol * self.nslab
        self.ndof = 3 * self.n * self.E
        self.n_layers = len(desc["materials"])
        # logical coordinates of the element nodes, node p = (k N + j) N + i
        g = self.nodes
        kk, jj, ii = np.meshgrid(np.arange(self.N), np.arange(self.N),
                                 np.arange(self.N), indexing="ij")
        self.ijk = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)
        self.xi_nodes = g[self.ijk]  # (n, 3): (xi, eta, zeta) per node
        self.wvol = (self.weights[self.ijk[:, 0]] * self.weights[self.ijk[:, 1]]
                     * self.weights[self.ijk[:, 2]])
        self._geo = {}
        self._build_topology()

    # ------------------------------------------------------------------ maps
    def element_of(self, e):
        return divmod(e, self.ncol)  # (slab, column)

    def layer(self, e):
        return int(self.desc["slab_layer"][e // self.ncol])

    def _map_xy(self, c, xi, eta):
        d = self.desc
        if self.kind == "box":
            ix, jy = c % self.nx, c // self.nx
            x0, x1 = d["x_breaks"][ix], d["x_breaks"][ix + 1]
            y0, y1 = d["y_breaks"][jy], d["y_breaks"][jy + 1]
            return x0 + 0.5 * (1 + xi) * (x1 - x0), y0 + 0.5 * (1 + eta) * (y1 - y0)
        k = self.k
        blk, cl = divmod(c, k * k)
        bi, ai = divmod(cl, k)
        xb = -1.0 + (2.0 * ai + 1.0 + xi) / k
        eb = -1.0 + (2.0 * bi + 1.0 + eta) / k
        a, R1, R = d["a"], d["R1"], d["R"]
        if blk == 0:
            return a * xb, a * eb
        th = np.pi * eb / 4.0
        if blk <= 4:  # inner wedge: square face blended into the circle R1
            X = 0.5 * (1 - xb) * a + 0.5 * (1 + xb) * R1 * np.cos(th)
            Y = 0.5 * (1 - xb) * a * eb + 0.5 * (1 + xb) * R1 * np.sin(th)
            return _rot(blk - 1, X, Y)
        rad = 0.5 * (1 - xb) * R1 + 0.5 * (1 + xb) * R  # outer wedge: annulus
        return _rot(blk - 5, rad * np.cos(th), rad * np.sin(th))

    def _map_z(self, s, zeta):
        zt, zb = self.slab_z[s], self.slab_z[s + 1]
        if self.desc["slab_log"][s]:
            st, sb = -zt, -zb  # depths, both > 0
            return -np.exp(0.5 * (1 + zeta) * np.log(st) + 0.5 * (1 - zeta) * np.log(sb))
        return 0.5 * (1 + zeta) * zt + 0.5 * (1 - zeta) * zb

    def _dmap_z(self, s, zeta):
        """dZ/dzeta of the slab map, written out."""
        zt, zb = self.slab_z[s], self.slab_z[s + 1]
        if self.desc["slab_log"][s]:
            st, sb = -zt, -zb
            depth = np.exp(0.5 * (1 + zeta) * np.log(st) + 0.5 * (1 - zeta) * np.log(sb))
            return 0.5 * depth * (np.log(sb) - np.log(st))
        return 0.5 * (zt - zb) + 0.0 * zeta

    def map(self, e, xi):
        """x(xi) for element e; xi has shape (..., 3); works for complex xi."""
        s, c = self.element_of(e)
        X, Y = self._map_xy(c, xi[..., 0], xi[..., 1])
        Z = self._map_z(s, xi[..., 2])
        return np.stack(np.broadcast_arrays(X, Y, Z), axis=-1)

    def jacobian(self, e, xi):
        """J[..., a, m] = dx^a / dxi^m by complex step."""
        xi = np.asarray(xi, dtype=complex)
        cols = []
        for m in range(3):
            dx = np.zeros(3, dtype=complex)
            dx[m] = 1j * _CSTEP
            cols.append(np.imag(self.map(e, xi + dx)) / _CSTEP)
        return np.stack(cols, axis=-1)

    def jacobian_split(self, e, xi):
        """J from a complex step of the cross-section map and dZ/dzeta."""
        s, c = self.element_of(e)
        xi = np.asarray(xi, dtype=float)
        J = np.zeros(xi.shape[:-1] + (3, 3), dtype=np.result_type(self.slab_z, float))
        for m_ in range(2):
            d = np.zeros(3, dtype=complex)
            d[m_] = 1j * _CSTEP
            xc = xi + d
            X, Y = self._map_xy(c, xc[..., 0], xc[..., 1])
            J[..., 0, m_] = np.imag(X) / _CSTEP
            J[..., 1, m_] = np.imag(Y) / _CSTEP
        J[..., 2, 2] = self._dmap_z(s, xi[..., 2])
        return J

    def geometry(self, e):
        """Nodal coordinates, Jacobian, det, inverse and quadrature weight w detJ."""
        if e in self._geo:
            return self._geo[e]
        xi = self.xi_nodes
        s, c = self.element_of(e)
        X, Y = self._map_xy(c, xi[:, 0], xi[:, 1])
        Z = self._map_z(s, xi[:, 2])
        xyz = np.stack(np.broadcast_arrays(X, Y, Z), axis=-1)
        if not np.iscomplexobj(self.slab_z):
            xyz = np.real(xyz)
        J = self.jacobian_split(e, xi)
        detJ = np.linalg.det(J)
        Jinv = np.linalg.inv(J)  # Jinv[p, m, a] = dxi^m / dx^a
        geo = {"xyz": xyz, "J": J, "detJ": detJ, "Jinv": Jinv,
               "wJ": self.wvol * detJ}
        if len(self._geo) > 4096:
            self._geo.clear()
        self._geo[e] = geo
        return geo

    # -------------------------------------------------------------- faces
    def face_nodes(self, f):
        """Node indices of face f = 2 d + s (d: xi/eta/zeta; s: -1 or +1 side)."""
        d, s = divmod(f, 2)
        end = self.N - 1 if s else 0
        return np.nonzero(self.ijk[:, d] == end)[0]

    def face_weights(self, f):
        """Tangential LGL weights w^Sigma of the face nodes."""
        d = f // 2
        t = [m for m in range(3) if m != d]
        F = self.face_nodes(f)
        return self.weights[self.ijk[F, t[0]]] * self.weights[self.ijk[F, t[1]]]

    def face_geometry(self, e, f):
        """Unit outward normal n_i, surface Jacobian J^Sigma and the size
        h = 2 detJ / J^Sigma orthogonal to the face, at the face nodes."""
        geo = self.geometry(e)
        d, s = divmod(f, 2)
        F = self.face_nodes(f)
        row = geo["Jinv"][F, d, :]  # grad xi^d
        mag = np.sqrt(np.sum(row * row, axis=1))
        sign = 1.0 if s else -1.0
        n = sign * row / mag[:, None]
        Jsig = geo["detJ"][F] * mag
        h = 2.0 * geo["detJ"][F] / Jsig
        return {"F": F, "n": n, "Jsig": Jsig, "h": h, "xyz": geo["xyz"][F],
                "W": self.face_weights(f) * Jsig}

    def _build_topology(self):
        centres = np.zeros((self.E, 6, 3))
        for e in range(self.E):
            for f in range(6):
                d, s = divmod(f, 2)
                xi = np.zeros(3, dtype=complex)
                xi[d] = 1.0 if s else -1.0
                centres[e, f] = np.real(self.map(e, xi))
        flat = centres.reshape(-1, 3)
        flat = np.real(flat)
        scale = max(1.0, float(np.max(np.abs(flat))))
        tree = cKDTree(flat)
        pairs = tree.query_pairs(r=1e-9 * scale, output_type="ndarray")
        self.neighbour = -np.ones((self.E, 6), dtype=np.int64)
        self.nb_face = -np.ones((self.E, 6), dtype=np.int64)
        for a, b in pairs:
            ea, fa = divmod(int(a), 6)
            eb, fb = divmod(int(b), 6)
            if ea == eb:
                raise RuntimeError("degenerate element")
            if self.neighbour[ea, fa] >= 0 or self.neighbour[eb, fb] >= 0:
                raise RuntimeError("non-conforming face")
            self.neighbour[ea, fa], self.nb_face[ea, fa] = eb, fb
            self.neighbour[eb, fb], self.nb_face[eb, fb] = ea, fa
        zmax, zmin = np.real(self.slab_z[0]), np.real(self.slab_z[-1])
        tol = 1e-9 * scale
        self.bkind = np.full((self.E, 6), "", dtype=object)
        for e in range(self.E):
            for f in range(6):
                if self.neighbour[e, f] >= 0:
                    continue
                z = centres[e, f, 2]
                if abs(z - zmax) < tol and f == 5:
                    self.bkind[e, f] = "top"
                elif abs(z - zmin) < tol and f == 4:
                    self.bkind[e, f] = "bottom"
                else:
                    self.bkind[e, f] = "side"
        self._perm = {}

    def face_perm(self, e, f):
        """perm such that node face_nodes(f2)[perm[q]] of the neighbour
        coincides with node face_nodes(f)[q] of e."""
        key = (e, f)
        if key in self._perm:
            return self._perm[key]
        e2, f2 = int(self.neighbour[e, f]), int(self.nb_face[e, f])
        x1 = np.real(self.geometry(e)["xyz"][self.face_nodes(f)])
        x2 = np.real(self.geometry(e2)["xyz"][self.face_nodes(f2)])
        dist, perm = cKDTree(x2).query(x1)
        scale = max(1.0, float(np.max(np.abs(x1))))
        if np.max(dist) > 1e-9 * scale or len(set(perm.tolist())) != len(perm):
            raise RuntimeError("face nodes do not match")
        self._perm[key] = perm
        return perm

    def boundary_condition(self, e, f):
        """'interior', 'neumann' or 'dirichlet' for face f of element e:
        the top carries the beam pressure (Neumann), sides and bottom follow
        the description (fixed = Dirichlet u = 0, free = zero traction)."""
        if self.neighbour[e, f] >= 0:
            return "interior"
        where = self.bkind[e, f]
        if where == "top":
            return "neumann"
        tag = self.desc["bc_side"] if where == "side" else self.desc["bc_bottom"]
        return "dirichlet" if tag == "fixed" else "neumann"
