"""The allocation-free energy entry point (tn_layer_energies_noalloc), for
callers that cannot allocate device memory when they ask for energies, gives
the same per-layer energies as tn_layer_energies on two calls in a row.
Collected last on purpose; it also passes when run alone."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2111_06893_gb300 import build
    build.build()


def test_noalloc_energies_match_the_allocating_entry_point_twice():
    from paper_2111_06893_gb300 import thermonoise
    lib = thermonoise.load()
    desc = W.cylinder(10.0, 10.0, [0.05, 0.02], [W.COATING_HIGH, W.CRYSTAL_A], W.FUSED_SILICA, 1, 4, 2)
    ctx = thermonoise.setup(desc)
    nl = len(desc["materials"])
    dp = C.POINTER(C.c_double)
    for seed in (1, 2):  # two calls in a row, different fields
        u = torch.tensor(W.random_field(desc, seed), dtype=torch.float64, device="cuda")
        U_ref = ctx.layer_energies(u)
        U = np.zeros(nl)
        st = lib.tn_layer_energies_noalloc(ctx._h, C.c_void_p(u.data_ptr()), U.ctypes.data_as(dp))
        assert st == thermonoise.TN_OK, lib.tn_last_error().decode()
        assert np.max(np.abs(U - U_ref) / np.abs(U_ref)) < 1e-12, (seed, U, U_ref)


def test_noalloc_rejects_meshes_beyond_its_limit():
    from paper_2111_06893_gb300 import thermonoise
    lib = thermonoise.load()
    desc = W.box([0.0] + [float(i + 1) for i in range(300)], [0.0, 1.0], [0.0, -1.0], 2, W.FUSED_SILICA)
    desc["y_breaks"] = [float(j) for j in range(220)]  # 300 x 219 columns > 65536 elements
    ctx = thermonoise.setup(desc)
    u = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda")
    U = np.zeros(1)
    st = lib.tn_layer_energies_noalloc(ctx._h, C.c_void_p(u.data_ptr()), U.ctypes.data_as(C.POINTER(C.c_double)))
    assert st == thermonoise.TN_EINVAL_CODE
    assert b"at most 65536 elements" in lib.tn_last_error()


def test_noalloc_energies_at_the_element_limit():
    """A mesh of exactly 65536 elements (128 x 128 columns, four slabs of two
    materials): the per-element scratch is full and the layer sums sit right
    after it."""
    from paper_2111_06893_gb300 import thermonoise
    lib = thermonoise.load()
    xb = [float(i) / 16.0 for i in range(129)]
    desc = W.box(xb, xb, [0.0, -0.05, -0.1, -1.0, -4.0], 2, None, r0=2.0, slab_layer=[0, 0, 1, 1],
                 materials=[W.COATING_HIGH, W.FUSED_SILICA])
    ctx = thermonoise.setup(desc)
    assert ctx.ndof == 3 * 27 * 65536
    dp = C.POINTER(C.c_double)
    u = torch.tensor(W.random_field(desc, 5), dtype=torch.float64, device="cuda")
    U_ref = ctx.layer_energies(u)
    U = np.zeros(2)
    st = lib.tn_layer_energies_noalloc(ctx._h, C.c_void_p(u.data_ptr()), U.ctypes.data_as(dp))
    assert st == thermonoise.TN_OK, lib.tn_last_error().decode()
    assert np.max(np.abs(U - U_ref) / np.abs(U_ref)) < 1e-12, (U, U_ref)
