"""Parity of the CUDA path with the FP64 oracle on the same seeded inputs.

Tolerances: FP64 operator applies 1e-11 relative to max|y| (element by
element), energies 1e-9 relative; FP32 applies 2e-5 relative to max|y|
(single rounding of the fields and geometry plus FP32 accumulation over
~10^2 terms per output).
"""
import functools

import numpy as np
import pytest

import workloads as W
from oracle import Mesh, Operator, observables as ob

from cases import CASES

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_06893_gb300 import build
    build.build()


@functools.lru_cache(maxsize=None)
def oracle_case(name):
    desc = CASES[name]()
    op = Operator(Mesh(desc))
    A = op.assemble()
    return desc, op, A


def gpu_ctx(desc):
    from paper_2111_06893_gb300 import thermonoise
    return thermonoise.setup(desc)


def to_dev(x, dtype=torch.float64):
    return torch.tensor(np.asarray(x), dtype=dtype, device="cuda")


@pytest.mark.parametrize("name", sorted(CASES))
def test_apply_f64_matches_oracle(name):
    desc, op, A = oracle_case(name)
    ctx = gpu_ctx(desc)
    assert ctx.ndof == op.mesh.ndof
    for seed in (0, 1):
        u = W.random_field(desc, seed)
        y = ctx.apply_operator(to_dev(u)).cpu().numpy()
        yo = A @ u
        err = np.max(np.abs(y - yo)) / np.max(np.abs(yo))
        assert err < 1e-11, (name, seed, err)


@pytest.mark.parametrize("name", ["plain_box", "box_layers_p4", "cyl_small_p4_k2", "cyl_thin_p5"])
def test_apply_f32_matches_oracle(name):
    desc, op, A = oracle_case(name)
    ctx = gpu_ctx(desc)
    u = W.random_field(desc, 3)
    u32 = u.astype(np.float32)
    y = ctx.apply_operator(to_dev(u32, torch.float32)).cpu().numpy().astype(np.float64)
    yo = A @ u32.astype(np.float64)
    err = np.max(np.abs(y - yo)) / np.max(np.abs(yo))
    assert err < 2e-5, (name, err)


@pytest.mark.parametrize("name", ["plain_box", "box_layers_p4", "cyl_small_p4_k2", "cyl_small_p7_k1_fixed"])
def test_rhs_and_diagonal_match_oracle(name):
    desc, op, A = oracle_case(name)
    ctx = gpu_ctx(desc)
    b = ctx.rhs().cpu().numpy()
    bo = op.rhs()
    assert np.max(np.abs(b - bo)) <= 1e-14 * np.max(np.abs(bo))
    d = ctx.diagonal().cpu().numpy()
    do = A.diagonal()
    assert np.max(np.abs(d - do) / np.abs(do)) < 1e-12


@pytest.mark.parametrize("name", ["box_layers_p4", "cyl_small_p4_k2", "cyl_thin_p5"])
def test_energies_match_oracle_on_random_field(name):
    desc, op, A = oracle_case(name)
    ctx = gpu_ctx(desc)
    u = W.random_field(desc, 5)
    U = ctx.layer_energies(to_dev(u))
    Uo = ob.layer_energies(op, u)
    assert np.max(np.abs(U - Uo) / np.abs(Uo)) < 1e-12


def line_index_sets(m):
    """DOF indices of every vertical line of nodes: column c, cross-section
    node (i, j), all slabs top-down, three components, all k (the ordering
    inside a line does not matter for the block solve)."""
    N, n = m.N, m.n
    sets = []
    for c in range(m.ncol):
        for j in range(N):
            for i in range(N):
                idx = [((s * m.ncol + c) * 3 + comp) * n + (k * N + j) * N + i
                       for s in range(m.nslab) for comp in range(3) for k in range(N)]
                sets.append(np.array(idx))
    return sets


def group_index_sets(m):
    """DOF indices of every group of vertical lines that pass through one
    point of the cross-section (matching nodes of neighbouring columns),
    found from the physical coordinates of the oracle's nodes."""
    from scipy.spatial import cKDTree
    lines = line_index_sets(m)
    N = m.N
    pts = []
    for c in range(m.ncol):
        xyz = np.real(m.geometry(c)["xyz"])  # element of column c in the top slab
        for j in range(N):
            for i in range(N):
                pts.append(xyz[j * N + i][:2])  # node (i, j, k = 0)
    pts = np.array(pts)
    parent = list(range(len(pts)))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    scale = max(1.0, float(np.abs(pts).max()))
    for a, b in cKDTree(pts).query_pairs(1e-9 * scale):
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)
    groups = {}
    for t in range(len(pts)):
        groups.setdefault(find(t), []).append(t)
    return [np.concatenate([lines[q] for q in g]) for g in groups.values()], [len(g) for g in groups.values()]


@pytest.mark.parametrize("name", ["box_layers_p4", "cyl_small_p4_k2", "cyl_thin_p5", "cyl_small_p7_k1_fixed"])
def test_zgroup_preconditioner_matches_oracle_group_blocks(name):
    """z = A_GG^-1 r on every group of lines through one cross-section point,
    A_GG the principal sub-matrix of the oracle's assembled operator."""
    desc, op, A = oracle_case(name)
    A = A.tocsr()
    ctx = gpu_ctx(desc)
    r = W.random_field(desc, 23)
    z = ctx.precond_apply(to_dev(r), precond="zgroup").cpu().numpy()
    z32 = ctx.precond_apply(to_dev(r, torch.float32), precond="zgroup").cpu().numpy().astype(np.float64)
    sets, sizes = group_index_sets(op.mesh)
    assert sum(len(S) for S in sets) == len(r)
    assert max(sizes) >= 3  # edge and corner groups are exercised
    worst_bwd = worst_fwd = worst32 = 0.0
    for S in sets:
        B = A[S][:, S].toarray()
        zo = np.linalg.solve(B, r[S])
        scale = np.abs(B).max() * np.abs(z[S]).max()
        worst_bwd = max(worst_bwd, np.abs(B @ z[S] - r[S]).max() / scale)
        worst32 = max(worst32, np.abs(B @ z32[S] - r[S]).max() / (np.abs(B).max() * np.abs(z32[S]).max()))
        worst_fwd = max(worst_fwd, np.abs(z[S] - zo).max() / np.abs(zo).max())
    assert worst_bwd < 1e-13, worst_bwd
    assert worst32 < 1e-5, worst32
    assert worst_fwd < 1e-6, worst_fwd


def test_zgroup_cuts_iterations_on_thin_layers():
    """The grouped lines take the face-penalty coupling of neighbouring
    columns into the blocks: on a thin-layer mirror PCG needs far fewer
    iterations than with single lines (CPU estimate with the oracle's
    matrices: 976 -> 118 to 1e-8)."""
    desc, op, A = oracle_case("cyl_thin_p5")
    ctx = gpu_ctx(desc)
    its = {}
    for pc in ("zline", "zgroup"):
        _, rep = ctx.solve(mode="f64", rtol=1e-8, precond=pc)
        its[pc] = rep["inner_iters"]
    assert its["zgroup"] < 0.4 * its["zline"], its


@pytest.mark.parametrize("name", ["box_layers_p4", "cyl_small_p4_k2", "cyl_thin_p5", "cyl_small_p7_k1_fixed"])
def test_zline_preconditioner_matches_oracle_line_blocks(name):
    """z = A_LL^-1 r on every vertical line, A_LL the principal sub-matrix of
    the oracle's assembled operator on the line's DOFs."""
    desc, op, A = oracle_case(name)
    A = A.tocsr()
    ctx = gpu_ctx(desc)
    r = W.random_field(desc, 21)
    z = ctx.precond_apply(to_dev(r), precond="zline").cpu().numpy()
    z32 = ctx.precond_apply(to_dev(r, torch.float32), precond="zline").cpu().numpy().astype(np.float64)
    worst_bwd = worst_fwd = worst32 = 0.0
    for S in line_index_sets(op.mesh):
        B = A[S][:, S].toarray()
        zo = np.linalg.solve(B, r[S])
        scale = np.abs(B).max() * np.abs(z[S]).max()
        worst_bwd = max(worst_bwd, np.abs(B @ z[S] - r[S]).max() / scale)
        worst32 = max(worst32, np.abs(B @ z32[S] - r[S]).max() / (np.abs(B).max() * np.abs(z32[S]).max()))
        worst_fwd = max(worst_fwd, np.abs(z[S] - zo).max() / np.abs(zo).max())
    assert worst_bwd < 1e-13, worst_bwd
    assert worst32 < 1e-5, worst32
    assert worst_fwd < 1e-6, worst_fwd


@pytest.mark.parametrize("mode", ["f64", "mixed"])
@pytest.mark.parametrize("precond", ["jacobi", "zline", "zgroup"])
def test_solve_plain_box_energies_match_oracle_direct_solve(mode, precond):
    desc, op, A = oracle_case("plain_box")
    uo = ob.solve_dense(A, op.rhs())
    Uo = ob.layer_energies(op, uo)
    ctx = gpu_ctx(desc)
    u, rep = ctx.solve(mode=mode, rtol=1e-12, energy_rtol=1e-12, precond=precond)
    assert rep["rel_residual"] <= 1e-12 or rep["energy_change"] <= 1e-12
    U = ctx.layer_energies(u)
    assert np.max(np.abs(U - Uo) / Uo) < 1e-9, (U, Uo)
    un = u.cpu().numpy()
    assert np.max(np.abs(un - uo)) < 1e-9 * np.max(np.abs(uo))
    if mode == "mixed":
        assert rep["applies_f32"] > rep["applies_f64"]


def test_solve_layered_cylinder_matches_oracle():
    desc, op, A = oracle_case("cyl_small_p4_k1")
    uo = ob.solve_dense(A, op.rhs())
    Uo = ob.layer_energies(op, uo)
    ctx = gpu_ctx(desc)
    for mode, pc in (("f64", "zline"), ("mixed", "zline"), ("f64", "zgroup"), ("mixed", "zgroup")):
        u, rep = ctx.solve(mode=mode, rtol=1e-13, energy_rtol=1e-12, precond=pc)
        U = ctx.layer_energies(u)
        assert np.max(np.abs(U - Uo) / Uo) < 1e-9, (mode, pc, U, Uo, rep)
    from paper_2111_06893_gb300 import noise_psd
    phi = [1e-4, 4e-4, 1e-6]
    S = noise_psd(U, phi, 4.14e-21, 100.0, desc["beam"]["F0"])
    So = ob.noise_psd(Uo, phi, 4.14e-21, 100.0, desc["beam"]["F0"])
    assert abs(S / So - 1) < 1e-9


def test_apply_is_deterministic():
    desc, op, A = oracle_case("cyl_small_p4_k2")
    ctx = gpu_ctx(desc)
    u = to_dev(W.random_field(desc, 9))
    y1 = ctx.apply_operator(u).clone()
    y2 = ctx.apply_operator(u)
    assert torch.equal(y1, y2)


def test_single_coating_full_size_sampled_rows():
    """The 2.0 M DOF single-coating mirror (p = 6): sampled element rows of
    A u against the oracle's element-by-element rows, FP64 and FP32."""
    desc = W.single_coating()
    ctx = gpu_ctx(desc)
    m = Mesh(desc)
    op = Operator(m)
    u = W.random_field(desc, 11)
    y = ctx.apply_operator(to_dev(u)).cpu().numpy()
    y32 = ctx.apply_operator(to_dev(u, torch.float32)).cpu().numpy()
    nl = 3 * m.n
    rng = np.random.default_rng(0)
    sample = sorted(set([0, m.ncol - 1, m.ncol, m.E - 1, 40, 80]
                        + rng.integers(0, m.E, size=6).tolist()))
    scale = 0.0
    rows = {}
    for e in sample:
        rows[e] = op.apply_element(e, u)
        scale = max(scale, np.max(np.abs(rows[e])))
    for e in sample:
        err = np.max(np.abs(y[e * nl:(e + 1) * nl] - rows[e])) / scale
        assert err < 1e-11, (e, err)
        err32 = np.max(np.abs(y32[e * nl:(e + 1) * nl] - rows[e])) / scale
        assert err32 < 2e-5, (e, err32)


def test_single_coating_full_size_sampled_line_groups():
    """The grouped-line solve on the 2.0 M DOF mirror: for one group of each
    size (1 to 4 lines), z = A_GG^-1 r against the group's principal
    sub-matrix assembled from the oracle's element rows; and the whole
    preconditioner is symmetric positive definite at full size."""
    from scipy.spatial import cKDTree
    desc = W.single_coating()
    ctx = gpu_ctx(desc)
    m = Mesh(desc)
    op = Operator(m)
    N, n, S = m.N, m.n, m.nslab
    r = W.random_field(desc, 31)
    z = ctx.precond_apply(to_dev(r), precond="zgroup").cpu().numpy()
    z32 = ctx.precond_apply(to_dev(r, torch.float32), precond="zgroup").cpu().numpy().astype(np.float64)
    # groups of lines by the physical position of their nodes
    lines, pts = [], []
    for c in range(m.ncol):
        xyz = np.real(m.geometry(c)["xyz"])
        for j in range(N):
            for i in range(N):
                lines.append((c, i, j))
                pts.append(xyz[j * N + i][:2])
    pts = np.array(pts)
    parent = list(range(len(pts)))

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for a, b in cKDTree(pts).query_pairs(1e-9 * max(1.0, float(np.abs(pts).max()))):
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[max(ra, rb)] = min(ra, rb)
    groups = {}
    for t_ in range(len(pts)):
        groups.setdefault(find(t_), []).append(lines[t_])
    pick = {}
    for g in groups.values():
        pick.setdefault(len(g), g)
    assert sorted(pick) == [1, 2, 3, 4]
    cache = {}

    def rows(e):
        if e not in cache:
            cache[e] = op.element_rows(e)
        return cache[e]

    for g, members in sorted(pick.items()):
        # DOFs of the group: line, slab, component, k
        idx, per_elem = [], {}  # per_elem[e] = (local indices in e, positions in the group)
        for (c, i, j) in members:
            for s in range(S):
                e = s * m.ncol + c
                for comp in range(3):
                    for k in range(N):
                        loc = comp * n + (k * N + j) * N + i
                        per_elem.setdefault(e, ([], []))
                        per_elem[e][0].append(loc)
                        per_elem[e][1].append(len(idx))
                        idx.append(e * 3 * n + loc)
        B = np.zeros((len(idx), len(idx)))
        for e, (locs, pos) in per_elem.items():
            for e2, blk in rows(e).items():
                if e2 in per_elem:
                    locs2, pos2 = per_elem[e2]
                    B[np.ix_(pos, pos2)] = blk[np.ix_(locs, locs2)]
        idx = np.array(idx)
        bwd = np.abs(B @ z[idx] - r[idx]).max() / (np.abs(B).max() * np.abs(z[idx]).max())
        bwd32 = np.abs(B @ z32[idx] - r[idx]).max() / (np.abs(B).max() * np.abs(z32[idx]).max())
        assert bwd < 1e-13, (g, bwd)
        assert bwd32 < 1e-5, (g, bwd32)
    # symmetric positive definite: (M^-1 a) . b = a . (M^-1 b), a . M^-1 a > 0
    a = W.random_field(desc, 32)
    za = ctx.precond_apply(to_dev(a), precond="zgroup").cpu().numpy()
    assert abs(za @ r - a @ z) <= 1e-10 * np.sqrt((za @ a) * (z @ r))
    assert za @ a > 0 and z @ r > 0


def test_single_coating_full_size_sampled_element_energies():
    """Layer energies on the 2.0 M DOF mirror for a field that is nonzero on a
    few sampled elements only: each layer's energy is then the sum of those
    elements' energies, which the oracle computes element by element."""
    desc = W.single_coating()
    ctx = gpu_ctx(desc)
    m = Mesh(desc)
    op = Operator(m)
    nl = 3 * m.n
    rng = np.random.default_rng(5)
    sample = sorted(set([0, m.ncol - 1, m.ncol + 3, m.E - 1] + rng.integers(0, m.E, size=6).tolist()))
    full = W.random_field(desc, 12)
    u = np.zeros_like(full)
    for e in sample:
        u[e * nl:(e + 1) * nl] = full[e * nl:(e + 1) * nl]
    U = ctx.layer_energies(to_dev(u))
    Uo = np.zeros_like(U)
    for e in sample:
        Uo[m.layer(e)] += ob.element_energy(op, e, u)
    for L in range(len(U)):
        if Uo[L] == 0.0:
            assert U[L] == 0.0
        else:
            assert abs(U[L] - Uo[L]) <= 1e-12 * abs(Uo[L]), (L, U[L], Uo[L])


def test_invalid_arguments_are_rejected_before_launch():
    from paper_2111_06893_gb300 import thermonoise
    desc = CASES["box_tiny_p2"]()
    ctx = gpu_ctx(desc)
    u = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    lib = thermonoise.load()
    assert lib.tn_apply_operator(ctx._h, 7, u.data_ptr(), u.data_ptr()) == thermonoise.TN_EINVAL_CODE
    v = torch.zeros(ctx.ndof + 1, dtype=torch.float64, device="cuda")
    assert lib.tn_apply_operator(ctx._h, 0, v[1:].data_ptr(), u.data_ptr()) == thermonoise.TN_EINVAL_CODE
    bad = dict(desc)
    bad["degree"] = 12
    with pytest.raises(thermonoise.ThermonoiseError, match="TN_EINVAL"):
        thermonoise.Context().build_mesh(bad)
    with pytest.raises(thermonoise.ThermonoiseError, match="TN_ESTATE"):
        c2 = thermonoise.Context()
        c2.apply_operator(u)


@pytest.mark.parametrize("name", ["box_layers_p4", "cyl_small_p4_k2", "cyl_thin_p5"])
def test_energy_parts_match_oracle_on_random_field(name):
    """tn_layer_energy_parts against the oracle's projector split (dilatational,
    tetragonal, shear) of every layer, and the parts add up to the energies."""
    from paper_2111_06893_gb300 import thermonoise
    desc = CASES[name]()
    op = Operator(Mesh(desc))
    u = W.random_field(desc, 5)
    Po = ob.layer_energy_parts(op, u)
    ctx = thermonoise.setup(desc)
    ut = torch.tensor(u, dtype=torch.float64, device="cuda")
    P = ctx.layer_energy_parts(ut)
    U = ctx.layer_energies(ut)
    scale = U[:, None]
    assert np.max(np.abs(P - Po) / scale) < 1e-12, (P, Po)
    assert np.max(np.abs(P.sum(axis=1) - U) / U) < 1e-13


def test_energy_parts_of_a_batch_match_single_mirrors():
    from paper_2111_06893_gb300 import thermonoise
    descs = [CASES["box_layers_p4"](), CASES["cyl_small_p4_k1"](), CASES["box_tiny_p2"]()]
    bc = thermonoise.Context().build_batch(descs)
    u = torch.tensor(np.random.default_rng(7).uniform(-1, 1, size=int(bc.dof_off[-1])), dtype=torch.float64,
                     device="cuda")
    P = bc.layer_energy_parts(u)
    lo = bc.layer_off
    for i, d in enumerate(descs):
        sc = thermonoise.setup(d)
        Pi = sc.layer_energy_parts(u[bc.dof_off[i]:bc.dof_off[i + 1]].clone())
        assert np.array_equal(P[lo[i]:lo[i + 1]], Pi), i


def test_finite_size_ratio_matches_oracle():
    """The finite-size study's quantity on a small mirror (R = H = 5 r0,
    d = 0.04 r0, near-beam square and wedges of 2 and 4 r0): the solved
    coating noise over the approximate formula, GPU (mixed solve,
    tn_thin_coating_psd) against the oracle (refined direct solve, its own
    first-order thin-coating energy), to 1e-9."""
    from paper_2111_06893_gb300 import thermonoise
    desc = W.cylinder(5.0, 5.0, [0.04], [W.COATING_HIGH], W.FUSED_SILICA, 1, 3, 3, a=2.0, R1=4.0)
    op = Operator(Mesh(desc))
    uo = np.asarray(ob.solve_refined(op.assemble(), op.rhs()), dtype=np.float64)
    Uo = ob.layer_energies(op, uo)[0]
    c, s_ = W.COATING_HIGH, W.FUSED_SILICA
    ratio_o = Uo / ob.thin_coating_energy(c["Y"], c["nu"], s_["Y"], s_["nu"], 0.04, 1.0, 1.0)
    ctx = thermonoise.setup(desc)
    u, _ = ctx.solve(mode="mixed", rtol=1e-13, energy_rtol=1e-12, raise_on_error=False)
    kT, f, phi = 300 * ob.BOLTZMANN, 100.0, 4e-4
    S = thermonoise.noise_psd(ctx.layer_energies(u)[:1], np.array([phi]), kT, f, 1.0)
    ratio = S / thermonoise.thin_coating_psd(kT, f, 1.0, 0.04, s_, c, phi)
    assert abs(ratio - ratio_o) <= 1e-9 * ratio_o, (ratio, ratio_o)
