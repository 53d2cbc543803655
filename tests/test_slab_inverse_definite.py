"""The grouped-line preconditioner stores the inverse S_s^-1 of every slab's
Schur complement explicitly, rounded to FP32 for the inner solves.  An
explicit inverse stays positive definite after rounding only while its
condition number is far below 1 / (M eps32) ~ 1e5 (M <= 108 rows per slab
block).  Pinned here on the oracle's assembled operator for the thin-layer
test meshes: every group of lines through one cross-section point (the
same blocks as the GPU's), block Cholesky along the slabs in FP64, and the
eigenvalues of the FP32-rounded S_s^-1."""
import numpy as np
import pytest
from scipy.spatial import cKDTree

from oracle import Mesh, Operator

from cases import thin_cylinder, tie_stack


def slab_blocks_of_groups(m):
    """Per group of lines: the DOF indices of slab s as one array per slab."""
    N, n = m.N, m.n
    pts, lines = [], []
    for c in range(m.ncol):
        xyz = np.real(m.geometry(c)["xyz"])
        for j in range(N):
            for i in range(N):
                pts.append(xyz[j * N + i][:2])
                lines.append((c, i, j))
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
        groups.setdefault(find(t), []).append(lines[t])
    out = []
    for members in groups.values():
        per_slab = []
        for s in range(m.nslab):
            idx = [((s * m.ncol + c) * 3 + comp) * n + (k * N + j) * N + i
                   for (c, i, j) in members for comp in range(3) for k in range(N)]
            per_slab.append(np.array(idx))
        out.append(per_slab)
    return out


@pytest.mark.parametrize("make", [thin_cylinder, tie_stack], ids=["thin_cylinder", "tie_stack"])
def test_fp32_slab_inverses_stay_positive_definite(make):
    m = Mesh(make())
    A = Operator(m).assemble().tocsr()
    groups = slab_blocks_of_groups(m)
    sizes = {len(g[0]) // (3 * m.N) for g in groups}
    assert sizes >= {1, 2}, sizes
    worst_cond, worst_shift = 0.0, 0.0
    # one group of every size, and every slab along it
    seen = set()
    for per_slab in groups:
        g = len(per_slab[0]) // (3 * m.N)
        if g in seen:
            continue
        seen.add(g)
        Sinv_prev = None
        for s, idx in enumerate(per_slab):
            D = A[idx][:, idx].toarray()
            if s > 0:
                O = A[per_slab[s - 1]][:, idx].toarray()  # rows slab s - 1, columns slab s
                D = D - O.T @ Sinv_prev @ O
            ev = np.linalg.eigvalsh(D)
            assert ev[0] > 0.0, (g, s)
            Sinv = np.linalg.inv(D)
            Sinv = 0.5 * (Sinv + Sinv.T)
            ev64 = np.linalg.eigvalsh(Sinv)
            ev32 = np.linalg.eigvalsh(Sinv.astype(np.float32).astype(np.float64))
            worst_cond = max(worst_cond, ev[-1] / ev[0])
            worst_shift = max(worst_shift, abs(ev32[0] - ev64[0]) / ev64[0])
            Sinv_prev = Sinv
    print(f"worst cond(S_s) {worst_cond:.3g}, largest relative shift of the smallest eigenvalue "
          f"of S_s^-1 by FP32 rounding {worst_shift:.3g}")
    assert worst_cond < 1e5, worst_cond
    # rounding to FP32 moves the smallest eigenvalue of the inverse by a
    # tiny fraction of itself: the stored inverse is definite with margin
    assert worst_shift < 1e-2, worst_shift
