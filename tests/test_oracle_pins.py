"""Pins of the FP64 oracle to facts outside itself (no GPU).

Each test ties a part of the oracle to a closed form, a textbook identity, an
invariant of the mathematics or a brute-force evaluation, so that a dropped
term, a wrong sign or a transposed index in the oracle fails one of them.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import Mesh, Operator, observables as ob
from oracle import lgl, materials


# --------------------------------------------------------------- LGL basis

def test_lgl_closed_forms():
    x, w = lgl.lgl_nodes_weights(3)
    assert np.allclose(x, [-1, 0, 1], atol=1e-15)
    assert np.allclose(w, [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    x, w = lgl.lgl_nodes_weights(4)
    s = 1 / math.sqrt(5)
    assert np.allclose(x, [-1, -s, s, 1], atol=1e-15)
    assert np.allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15)
    x, w = lgl.lgl_nodes_weights(5)
    s = math.sqrt(3 / 7)
    assert np.allclose(x, [-1, -s, 0, s, 1], atol=1e-15)
    assert np.allclose(w, [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10], atol=1e-15)


@pytest.mark.parametrize("N", range(2, 11))
def test_lgl_quadrature_exactness(N):
    x, w = lgl.lgl_nodes_weights(N)
    assert abs(w.sum() - 2.0) < 1e-14
    for deg in range(0, 2 * N - 2):
        exact = 0.0 if deg % 2 else 2.0 / (deg + 1)
        assert abs(np.dot(w, x ** deg) - exact) < 1e-13
    deg = 2 * N - 2  # first degree LGL does not integrate exactly
    assert abs(np.dot(w, x ** deg) - 2.0 / (deg + 1)) > 1e-6


@pytest.mark.parametrize("N", range(2, 11))
def test_diff_matrix_exact_on_polynomials(N):
    x, _ = lgl.lgl_nodes_weights(N)
    D = lgl.diff_matrix(x)
    for k in range(N):
        d = k * x ** (k - 1) if k else np.zeros_like(x)
        assert np.max(np.abs(D @ x ** k - d)) < 1e-12 * max(1, k * N)
    # cardinality of the Lagrange basis
    assert np.allclose(lgl.interp_matrix(x, x), np.eye(N), atol=1e-14)


# --------------------------------------------------------------- materials

def test_lame_roundtrip_footnote():
    for Y, nu in [(72e9, 0.17), (140e9, 0.23), (1.0, 0.3)]:
        lam, mu = materials.lame_from_young(Y, nu)
        Y2, nu2, K = materials.young_from_lame(lam, mu)
        assert abs(Y2 / Y - 1) < 1e-14 and abs(nu2 - nu) < 1e-14
        assert abs(K - (lam + 2 * mu / 3)) < 1e-14 * Y
        # nu = lambda / (2 (lambda + mu)) written the other way
        assert abs(lam / (2 * (lam + mu)) - nu) < 1e-14


def test_stiffness_symmetries_and_cubic_reduces_to_iso():
    lam, mu = 3.1, 1.7
    Yi = materials.iso_tensor(lam, mu)
    Yc = materials.cubic_tensor(lam + 2 * mu, lam, mu)
    assert np.max(np.abs(Yi - Yc)) < 1e-15
    Yc = materials.cubic_tensor(119.9, 53.8, 59.4)
    for Yt in (Yi, Yc):
        assert np.allclose(Yt, Yt.transpose(1, 0, 2, 3))
        assert np.allclose(Yt, Yt.transpose(0, 1, 3, 2))
        assert np.allclose(Yt, Yt.transpose(2, 3, 0, 1))
    # Voigt form of the cubic tensor
    assert Yc[0, 0, 0, 0] == 119.9 and Yc[0, 0, 1, 1] == 53.8 and Yc[0, 1, 0, 1] == 59.4
    assert Yc[0, 0, 0, 1] == 0.0


# ---------------------------------------------------------------- geometry

def small_cylinder(degree=4, k=1, thick=(0.05,), n_sub=2, mats=None, **kw):
    mats = mats or [W.COATING_HIGH] * len(thick)
    return W.cylinder(10.0, 10.0, list(thick), mats, W.FUSED_SILICA, k, degree, n_sub, **kw)


def test_geometry_volume_and_top_area():
    d = W.box([-1, 0.5, 2], [0, 1, 3, 4], [0, -0.5, -2], 3, W.FUSED_SILICA)
    m = Mesh(d)
    vol = sum(m.geometry(e)["wJ"].sum() for e in range(m.E))
    assert abs(vol - 3 * 4 * 2) < 1e-12
    d = small_cylinder(degree=8, k=2)
    m = Mesh(d)
    vol = sum(m.geometry(e)["wJ"].sum() for e in range(m.E))
    assert abs(vol / (math.pi * 100 * 10) - 1) < 1e-8
    top = sum(m.face_geometry(e, 5)["W"].sum() for e in range(m.E) if m.bkind[e, 5] == "top")
    assert abs(top / (math.pi * 100) - 1) < 1e-8


def test_complex_step_jacobian_against_finite_differences():
    m = Mesh(small_cylinder(degree=3, k=2))
    rng = np.random.default_rng(3)
    for e in [0, 5, 17, 30, m.E - 1]:
        xi = rng.uniform(-1, 1, size=3)
        J = m.jacobian(e, xi)
        for j in range(3):
            h = np.zeros(3)
            h[j] = 1e-6
            fd = (np.real(m.map(e, (xi + h).astype(complex)))
                  - np.real(m.map(e, (xi - h).astype(complex)))) / 2e-6
            assert np.allclose(J[:, j], fd, rtol=1e-7, atol=1e-7)


def test_faces_conform():
    m = Mesh(small_cylinder(degree=3, k=2))
    for e in range(m.E):
        for f in range(6):
            if m.neighbour[e, f] < 0:
                continue
            e2, f2 = m.neighbour[e, f], m.nb_face[e, f]
            perm = m.face_perm(e, f)
            g1, g2 = m.face_geometry(e, f), m.face_geometry(e2, f2)
            assert np.allclose(g1["n"], -g2["n"][perm], atol=1e-12)
            assert np.allclose(g1["W"], g2["W"][perm], rtol=1e-12)
    kinds = set(m.bkind[m.neighbour < 0].tolist())
    assert kinds == {"top", "bottom", "side"}


# ------------------------------------------------------------- operator

def test_operator_symmetric_positive_definite_curved_two_materials():
    d = small_cylinder(degree=3, k=1, thick=(0.05, 0.1), mats=[W.COATING_HIGH, W.CRYSTAL_A])
    op = Operator(Mesh(d))
    A = op.assemble()
    assert abs(A - A.T).max() <= 1e-13 * abs(A).max()
    Ad = A.toarray()
    np.linalg.cholesky(Ad)  # raises if not positive definite


def test_strong_form_equals_weak_form_on_affine_mesh():
    d = W.box([-2, 0, 1], [-1, 1], [0, -0.3, -1, -2], 3, None,
              slab_layer=[0, 1, 2], materials=[W.COATING_HIGH, W.CRYSTAL_B, W.FUSED_SILICA],
              bc_side="fixed", bc_bottom="free")
    op = Operator(Mesh(d))
    u = W.random_field(d, 7)
    y = op.assemble() @ u
    r = op.strong_residual(u)
    assert np.max(np.abs(r - y)) < 1e-12 * np.max(np.abs(y))


def test_strong_and_weak_form_differ_on_curved_mesh():
    d = small_cylinder(degree=3, k=1)
    op = Operator(Mesh(d))
    u = W.random_field(d, 7)
    y = op.assemble() @ u
    r = op.strong_residual(u)
    rel = np.max(np.abs(r - y)) / np.max(np.abs(y))
    assert 1e-10 < rel < 1.0


def test_null_space_translations_and_rotations():
    # curved mesh, all faces free: rigid translations are annihilated
    d = small_cylinder(degree=3, k=1, bc_bottom="free")
    m = Mesh(d)
    A = Operator(m).assemble()
    scale = abs(A).max()
    for c in range(3):
        t = np.zeros((m.E, 3, m.n))
        t[:, c, :] = 1.0
        assert np.max(np.abs(A @ t.ravel())) < 1e-12 * scale
    # affine mesh, two materials, all free: infinitesimal rotations too
    d = W.box([-2, 0, 1], [-1, 1], [0, -0.3, -1], 3, None, slab_layer=[0, 1],
              materials=[W.COATING_HIGH, W.FUSED_SILICA], bc_side="free", bc_bottom="free")
    m = Mesh(d)
    A = Operator(m).assemble()
    scale = abs(A).max()
    xyz = np.stack([m.geometry(e)["xyz"] for e in range(m.E)])  # (E, n, 3)
    for w in np.eye(3):
        rot = np.cross(w, xyz)  # (E, n, 3)
        u = rot.transpose(0, 2, 1).ravel()
        assert np.max(np.abs(A @ u)) < 1e-11 * scale * np.max(np.abs(u))


def test_manufactured_linear_field_is_reproduced_exactly():
    d = W.box([-1, 0, 1.5], [-1, 0.5, 1], [0, -0.7, -2], 2, W.CRYSTAL_A,
              bc_side="fixed", bc_bottom="fixed", F0=0.0)
    m = Mesh(d)
    op = Operator(m)
    Gm = np.array([[0.3, -0.2, 0.5], [0.1, 0.4, -0.3], [-0.6, 0.2, 0.7]]) * 1e-3
    c0 = np.array([0.01, -0.02, 0.03])

    def exact(x):
        return x @ Gm.T + c0  # u_l = G_lk x_k + c_l

    S = 0.5 * (Gm + Gm.T)  # S_kl = d_(k u_l)
    stress = np.einsum("ijkl,kl->ij", op.Y[0], S)

    def neumann(x, n, where):
        return -n @ stress  # n_i T^ij with T = -Y S

    A = op.assemble()
    b = op.rhs(dirichlet=exact, neumann=neumann)
    u = ob.solve_dense(A, b)
    ue = np.stack([exact(m.geometry(e)["xyz"]).T for e in range(m.E)]).ravel()
    assert np.max(np.abs(u - ue)) < 1e-10 * np.max(np.abs(ue))
    U = ob.layer_energies(op, u).sum()
    vol = 2.5 * 2.0 * 2.0
    assert abs(U / (0.5 * np.einsum("ij,ij", S, stress) * vol) - 1) < 1e-10


def test_manufactured_layered_column_with_discontinuous_materials():
    """u = (0, 0, g(z)) with g' = -P / Y^zzzz per layer: continuous u and
    traction across layers with different Y (the consistency argument of
    Sec. 2.2.3), reproduced to roundoff."""
    mats = [W.COATING_HIGH, W.CRYSTAL_A, W.FUSED_SILICA]
    zb = [0.0, -0.2, -0.5, -1.5, -2.5]
    d = W.box([-1, 0, 1], [-1, 1], zb, 3, None, slab_layer=[0, 1, 2, 2], materials=mats,
              bc_side="fixed", bc_bottom="fixed", F0=0.0)
    m = Mesh(d)
    op = Operator(m)
    P = 2.5e7
    czz = [op.Y[i][2, 2, 2, 2] for i in range(3)]
    layer_of = [0, 1, 2, 2]

    def g(z):
        out = np.zeros_like(z)
        for i, zv in np.ndenumerate(z):
            val = 0.0
            for s in range(len(zb) - 1, -1, -1):  # from the bottom upwards
                if s == len(zb) - 1:
                    continue
                top, bot = zb[s], zb[s + 1]
                slope = -P / czz[layer_of[s]]
                lo = bot
                hi = min(top, zv)
                if hi > lo:
                    val += slope * (hi - lo)
            out[i] = val
        return out

    def exact(x):
        return np.stack([0 * x[:, 0], 0 * x[:, 0], g(x[:, 2])], axis=1)

    def neumann(x, n, where):
        return n * P  # n_i T^ij = n^j P: uniform pressure on the top

    A = op.assemble()
    b = op.rhs(dirichlet=exact, neumann=neumann)
    u = ob.solve_dense(A, b)
    ue = np.stack([exact(m.geometry(e)["xyz"]).T for e in range(m.E)]).ravel()
    assert np.max(np.abs(u - ue)) < 1e-10 * np.max(np.abs(ue))


def test_brute_force_quadrature_one_element():
    """v^T K u from the LGL element matrix equals the exact integral of
    grad v : Y : grad u (Gauss-Legendre, 12 points) for polynomial u, v whose
    integrand LGL integrates exactly (degree <= 2N - 3 per variable)."""
    d = W.box([0.0, 2.0], [0.0, 1.0], [0.0, -3.0], 3, W.CRYSTAL_B)
    m = Mesh(d)
    op = Operator(m)
    K = op.volume_matrix(0)
    xyz = m.geometry(0)["xyz"]
    cu = np.random.default_rng(1).normal(size=(3, 8))
    cv = np.random.default_rng(2).normal(size=(3, 8))
    # u_l = sum of monomials x^a y^b z^c with a, b, c <= 1 (trilinear), v: degree <= 2
    mons_u = [(a, b, c) for a in range(2) for b in range(2) for c in range(2)]
    mons_v = [(2, 0, 1), (0, 2, 1), (1, 1, 2), (2, 1, 0), (1, 0, 0), (0, 1, 2), (0, 0, 2), (2, 2, 2)]

    def field(coef, mons, x):
        return np.stack([sum(coef[l, t] * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** c
                             for t, (a, b, c) in enumerate(mons)) for l in range(3)], axis=1)

    def grad(coef, mons, x):
        g = np.zeros((len(x), 3, 3))  # [q, k, l] = d u_l / d x_k
        for l in range(3):
            for t, (a, b, c) in enumerate(mons):
                cc = coef[l, t]
                g[:, 0, l] += cc * a * x[:, 0] ** max(a - 1, 0) * x[:, 1] ** b * x[:, 2] ** c
                g[:, 1, l] += cc * b * x[:, 0] ** a * x[:, 1] ** max(b - 1, 0) * x[:, 2] ** c
                g[:, 2, l] += cc * c * x[:, 0] ** a * x[:, 1] ** b * x[:, 2] ** max(c - 1, 0)
        return g

    u = field(cu, mons_u, xyz).T.ravel()
    v = field(cv, mons_v, xyz).T.ravel()
    lhs = v @ K @ u
    gx, gw = np.polynomial.legendre.leggauss(12)
    X, Yg, Z = np.meshgrid(1 + gx, 0.5 + 0.5 * gx, -1.5 + 1.5 * gx, indexing="ij")
    Wq = np.einsum("i,j,k->ijk", gw, gw, gw).ravel() * (1 * 0.5 * 1.5)
    pts = np.stack([X.ravel(), Yg.ravel(), Z.ravel()], axis=1)
    Yt = op.Y[0]
    dens = np.einsum("qij,ijkl,qkl->q", grad(cv, mons_v, pts), Yt, grad(cu, mons_u, pts))
    rhs = np.sum(Wq * dens)
    assert abs(lhs - rhs) < 1e-11 * abs(rhs)


# --------------------------------------------------------- load and energy

def test_beam_load_normalisation_and_sign():
    d = W.cylinder(10.0, 10.0, [0.05], [W.COATING_HIGH], W.FUSED_SILICA, 3, 7, 2, r0=1.3, F0=2.0)
    op = Operator(Mesh(d))
    b = op.rhs().reshape(op.mesh.E, 3, op.mesh.n)
    Fz = b[:, 2, :].sum()
    assert abs(Fz / (-2.0 * (1 - math.exp(-100 / 1.3 ** 2))) - 1) < 1e-6
    assert np.max(np.abs(b[:, :2, :])) == 0.0


def test_half_space_closed_form_matches_quadrature():
    for Y, nu, F0, r0 in [(72e9, 0.17, 1.0, 1.0), (140e9, 0.23, 2.0, 0.7)]:
        assert abs(ob.half_space_energy_quadrature(Y, nu, F0, r0)
                   / ob.half_space_energy(Y, nu, F0, r0) - 1) < 1e-7


def _graded(L, h0=0.5):
    v = [h0]
    while v[-1] < L:
        v.append(v[-1] * 2)
    v[-1] = L
    return [-x for x in v[::-1]] + [0.0] + v


def test_half_space_limit():
    """Clamped graded boxes of half-width L = 4 and 8 (p = 2): the energy
    error decays like 1/L and the Richardson-extrapolated energy is the
    half-space closed form (1 - nu^2) F0^2 / (2 sqrt(2 pi) Y r0)."""
    Uh = ob.half_space_energy(72e9, 0.17, 1.0, 1.0)
    E = {}
    for L in (4, 8):
        br = _graded(L)
        zb = [0.0] + [-x for x in br[len(br) // 2 + 1:]]
        d = W.box(br, br, zb, 2, W.FUSED_SILICA, penalty_C=1.5)
        op = Operator(Mesh(d))
        A = op.assemble()
        b = op.rhs()
        u = ob.solve_cg(op, A, b, rtol=1e-10)
        E[L] = ob.layer_energies(op, u).sum()
        uz = u.reshape(op.mesh.E, 3, op.mesh.n)[:, 2, :]
        assert uz.min() < 0 and abs(uz.min()) > abs(uz.max())  # pressed in
    assert E[4] < E[8] < Uh
    extrap = 2 * E[8] - E[4]
    assert abs(extrap / Uh - 1) < 0.01


def test_noise_psd_independent_of_force_and_levin_half_space():
    d = small_cylinder(degree=3, k=1)
    op = Operator(Mesh(d))
    A = op.assemble()
    S = []
    for F0 in (1.0, 3.0):
        d["beam"]["F0"] = F0
        b = op.rhs()
        U = ob.layer_energies(op, ob.solve_dense(A, b))
        S.append(ob.noise_psd(U, [1e-4, 1e-6], 300 * ob.BOLTZMANN, 100.0, F0))
    assert abs(S[1] / S[0] - 1) < 1e-12
    # half-space: S = 2 kT (1 - nu^2) phi / (pi^(3/2) f w Y) with w = sqrt(2) r0
    Y, nu, r0, phi, kT, f = 72e9, 0.17, 1.0, 1e-6, 300 * ob.BOLTZMANN, 100.0
    Sq = ob.noise_psd([ob.half_space_energy(Y, nu, 1.0, r0)], [phi], kT, f, 1.0)
    levin = 2 * kT * (1 - nu ** 2) * phi / (math.pi ** 1.5 * f * math.sqrt(2) * r0 * Y)
    assert abs(Sq / levin - 1) < 1e-13


def test_thin_coating_energy_and_psd_reproduce_the_approximate_formula():
    """Eq. (approx_analytic): the paper's thin-coating noise for amorphous
    layers on a half-space (beam width w = sqrt(2) r0, one coating loss
    angle).  The oracle's route to the same number is independent of it: the
    coating energy from the substrate's surface strain, then the PSD
    constant of the fluctuation-dissipation reading.  Agreement for unlike
    materials pins both the energy derivation and the constant 4/pi."""
    kT, f, d, r0, phi = 300 * ob.BOLTZMANN, 100.0, 3e-3, 1.3, 4e-4
    for Yc, nuc, Ys, nus in ((140e9, 0.23, 72e9, 0.17), (72e9, 0.17, 72e9, 0.17),
                             (100e9, 0.32, 72e9, 0.17), (60e9, 0.0, 200e9, 0.35)):
        for F0 in (1.0, 2.5):
            U = ob.thin_coating_energy(Yc, nuc, Ys, nus, d, F0, r0)
            S = ob.noise_psd([U], [phi], kT, f, F0)
            paper = (kT / (math.pi ** 2 * f) * (1 - nus ** 2) / (r0 * Ys) * d / r0
                     * phi / (Ys * Yc * (1 - nuc ** 2) * (1 - nus ** 2))
                     * (Yc ** 2 * (1 + nus) ** 2 * (1 - 2 * nus) ** 2 + Ys ** 2 * (1 + nuc) ** 2 * (1 - 2 * nuc)))
            assert abs(S / paper - 1) < 1e-13, (Yc, nuc, Ys, nus, S / paper)


def test_layer_energy_sum_approaches_half_b_dot_u_with_degree():
    """Sec. 2.1 energy, read as the element's own unlifted strain energy:
    its layer sum differs from the discrete energy 1/2 b.u by the jump and
    penalty terms, a gap that must vanish as the degree grows (a wrong
    factor or a lifted/unlifted mix-up in the density would leave it)."""
    gaps = []
    for p in (2, 3, 4, 5):
        d = W.box([-2.0, 0.0, 2.0], [-2.0, 0.0, 2.0], [0.0, -1.0, -2.5], p, W.FUSED_SILICA,
                  penalty_C=3.0, bc_side="fixed", bc_bottom="fixed", r0=0.8)
        op = Operator(Mesh(d))
        b = op.rhs()
        u = ob.solve(op.assemble(), b)
        E = 0.5 * float(b @ u)
        gaps.append(abs(ob.layer_energies(op, u).sum() - E) / E)
    assert all(g1 < g0 for g0, g1 in zip(gaps, gaps[1:])), gaps
    assert gaps[0] > 1e-3 and gaps[-1] < 1e-4, gaps


def test_split_jacobian_matches_full_complex_step():
    """The geometry's Jacobian (complex step of the cross-section map, closed
    form dZ/dzeta) equals the full 3-D complex-step Jacobian of the map."""
    m = Mesh(W.cylinder(10.0, 10.0, [0.05, 0.3], [W.COATING_HIGH, W.FUSED_SILICA], W.FUSED_SILICA,
                        2, 4, 3))
    rng = np.random.default_rng(5)
    for e in [0, 7, 40, m.E - 1]:
        xi = rng.uniform(-1, 1, size=(6, 3))
        assert np.allclose(m.jacobian_split(e, xi), m.jacobian(e, xi), rtol=1e-13, atol=1e-13)


def test_complex_step_energy_gradients_match_central_differences():
    """The oracle's reference gradients (complex step through mesh, operator,
    solve and energies) against central finite differences of full solves."""
    from oracle import gradient as G
    d = W.box([-1.0, 0.2], [-0.5, 1.0], [0.0, -0.3, -1.3], 2, None, slab_layer=[0, 1],
              materials=[W.CRYSTAL_A, W.FUSED_SILICA], penalty_C=3.0, bc_side="fixed", bc_bottom="fixed")
    for p, h, tol in [(("slab_z", 1), 1e-6, 1e-7), (("r0",), 1e-6, 1e-8),
                      (("material", 0, "c11"), 1e-6 * 119.9e9, 1e-6), (("material", 1, "nu"), 1e-6, 1e-5)]:
        cs = G.energy_derivative(d, p)
        fd = np.real(G.energies(G.perturbed(d, p, h)) - G.energies(G.perturbed(d, p, -h))) / (2 * h)
        assert np.max(np.abs(cs - fd)) <= tol * np.max(np.abs(cs)), (p, cs, fd)


# ------------------------------------------------ refined solve, tie rule

def test_refined_solve_recovers_exact_integer_solution():
    """solve_refined on Pascal matrices (integer, SPD, cond 4e9 and 2e7) with
    integer solutions: the refined solution is exact to well below what a
    plain FP64 factorisation reaches; under a complex step the imaginary
    part (a derivative) is recovered too."""
    import scipy.linalg as sl
    import scipy.sparse as sp
    rng = np.random.default_rng(0)
    A = sl.pascal(10).astype(float)
    x = rng.integers(-3, 4, size=10).astype(float)
    b = A @ x
    plain = np.linalg.solve(A, b)
    xr = ob.solve_refined(sp.csr_matrix(A), b)
    assert np.max(np.abs(plain - x)) > 1e-9  # the plain solve is visibly off
    assert np.max(np.abs(np.asarray(xr, dtype=float) - x)) < 1e-10
    A = sl.pascal(8).astype(float)
    x = rng.integers(-3, 4, size=8).astype(float)
    y = rng.integers(-3, 4, size=8).astype(float)
    B = sl.toeplitz(np.arange(8) % 5).astype(float)
    h = 1e-30
    xc = ob.solve_refined(sp.csr_matrix(A + 1j * h * B), A @ x + 1j * h * (B @ x + A @ y))
    assert np.max(np.abs(np.real(xc).astype(float) - x)) < 1e-12
    assert np.max(np.abs(np.imag(xc).astype(float) / h - y)) < 2e-9


@pytest.mark.parametrize("dz_bottom", [0.0, -1e-14])
def test_tie_of_face_sizes_takes_the_forward_derivative(dz_bottom):
    """Two slabs of equal thickness (exactly, or within rounding): the
    complex-step derivative in the shared boundary equals the forward
    difference (derivative for an increasing parameter), not the backward
    one, which differs because min(h_int, h_ext) has a kink there."""
    from oracle import gradient as G
    desc = W.box([-1.0, 1.0], [-1.0, 1.0], [0.0, -0.5, -1.0 + dz_bottom], 2, W.FUSED_SILICA,
                 penalty_C=3.0, bc_side="fixed", bc_bottom="fixed", r0=0.7)
    cs = G.energy_derivative(desc, ("slab_z", 1))[0]

    def U(dz):
        d = dict(desc)
        z = list(desc["slab_z"])
        z[1] += dz
        d["slab_z"] = z
        return G.energies(d)[0]

    U0, h = U(0.0), 1e-5
    fwd = 2 * (U(h / 2) - U0) / (h / 2) - (U(h) - U0) / h
    bwd = 2 * (U0 - U(-h / 2)) / (h / 2) - (U0 - U(-h)) / h
    assert abs(cs - fwd) < 1e-6 * abs(fwd), (cs, fwd)
    assert abs(bwd - fwd) > 1e-3 * abs(fwd), (bwd, fwd)


# ------------------------------------------------- energy split by modulus

def _one_element_box(material):
    return W.box([-0.5, 0.7], [-0.4, 0.9], [0.0, -1.1], 2, material, penalty_C=3.0,
                 bc_side="free", bc_bottom="free")


@pytest.mark.parametrize("material", [W.CRYSTAL_A, W.COATING_HIGH])
def test_energy_parts_of_pure_strain_modes(material):
    """Linear fields with a pure dilatational, tetragonal or shear strain on
    one element: the parts are the closed forms 3/2 (c11 + 2 c12) V,
    (c11 - c12) V and 2 c44 V, the other parts vanish."""
    desc = _one_element_box(material)
    mesh = Mesh(desc)
    op = Operator(mesh)
    x = np.array([mesh.geometry(0)["xyz"][:, a] for a in range(3)])  # node coordinates
    V = 1.2 * 1.3 * 1.1
    Y = materials.tensor(material)
    c11, c12, c44 = Y[0, 0, 0, 0], Y[0, 0, 1, 1], Y[0, 1, 0, 1]
    fields = {0: (x[0], x[1], x[2]), 1: (x[0], -x[1], 0 * x[2]), 2: (x[1], x[0], 0 * x[2])}
    expect = {0: 1.5 * (c11 + 2 * c12) * V, 1: (c11 - c12) * V, 2: 2 * c44 * V}
    for mode, comps in fields.items():
        u = np.concatenate([np.asarray(c, dtype=float) for c in comps])
        P = ob.layer_energy_parts(op, u)[0]
        for j in range(3):
            ref = expect[mode] if j == mode else 0.0
            assert abs(P[j] - ref) <= 1e-12 * expect[mode], (mode, j, P[j], ref)


def test_energy_parts_add_up_to_layer_energies():
    desc = W.cylinder(10.0, 10.0, [0.05, 0.02], [W.CRYSTAL_A, W.COATING_HIGH], W.FUSED_SILICA, 1, 3, 2)
    op = Operator(Mesh(desc))
    u = W.random_field(desc, 3)
    P = ob.layer_energy_parts(op, u)
    U = ob.layer_energies(op, u)
    assert np.all(P >= -1e-12 * U[:, None])
    assert np.max(np.abs(P.sum(axis=1) - U) / U) < 1e-13
