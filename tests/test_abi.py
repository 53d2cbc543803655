"""The C-ABI library builds, loads and exports every declared entry point
(no GPU needed); host-only entry points and argument checks run on CPU."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2111_06893_gb300 import build, thermonoise
    build.build()
    return thermonoise.load()


def declared_symbols():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            src = open(os.path.join(inc, fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(tn_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    from paper_2111_06893_gb300 import thermonoise
    names = declared_symbols()
    assert len(names) >= 13
    for name in names:
        assert hasattr(lib, name), name
    assert set(thermonoise.SYMBOLS) <= set(names)


def test_noise_psd_host_entry_point(lib):
    from oracle import observables as ob
    from paper_2111_06893_gb300 import thermonoise
    U = np.array([1.5e-13, 2.0e-12])
    phi = np.array([4e-4, 1e-6])
    kT = 300 * ob.BOLTZMANN
    S = thermonoise.noise_psd(U, phi, kT, 100.0, 2.0)
    assert math.isclose(S, ob.noise_psd(U, phi, kT, 100.0, 2.0), rel_tol=1e-15)
    with pytest.raises(thermonoise.ThermonoiseError):
        thermonoise.noise_psd(U, phi, -1.0, 100.0, 2.0)


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    st = lib.tn_create(C.byref(h), 0, None)
    assert st != 0 and not h.value
    assert len(lib.tn_last_error()) > 0


def test_null_arguments_rejected(lib):
    assert lib.tn_build_mesh(None, None) == -1
    assert lib.tn_apply_operator(None, 0, None, None) == -1
    assert lib.tn_solve(None, None, None, None) == -1
    lib.tn_destroy(None)


def test_apply_tuning_entry_points_reject_null_context(lib):
    var = (C.c_int * 7)()
    assert lib.tn_apply_tuning(None, var, None) != 0
    assert lib.tn_set_apply_variant(None, 6, 0) != 0


def test_iso_moduli_host_entry_point(lib):
    """tn_iso_moduli against the oracle's Lame conversion (written from the
    other direction of the footnote to Eq. (constrel_iso)) and its
    derivatives against complex steps of the oracle's formula."""
    from oracle import materials
    from paper_2111_06893_gb300 import thermonoise
    for Y, nu in [(72e9, 0.17), (140e9, 0.23), (3.0, -0.4)]:
        (c11, c12, c44), dc = thermonoise.iso_moduli(Y, nu, derivatives=True)
        lam, mu = materials.lame_from_young(Y, nu)
        assert np.allclose([c11, c12, c44], [lam + 2 * mu, lam, mu], rtol=1e-14, atol=0)
        h = 1e-30
        for j, (dY, dn) in enumerate([(1j * h, 0.0), (0.0, 1j * h)]):
            l2, m2 = materials.lame_from_young(Y + dY, nu + dn)
            ref = np.imag([l2 + 2 * m2, l2, m2]) / h
            assert np.allclose(dc[:, j], ref, rtol=1e-13, atol=0), (j, dc[:, j], ref)
    with pytest.raises(thermonoise.ThermonoiseError):
        thermonoise.iso_moduli(72e9, 0.5)


def test_thin_coating_psd_host_entry_point(lib):
    """Eq. (approx_analytic) in the library against the oracle's first-order
    thin-coating energy turned into a PSD (the two are pinned to each other
    for unlike materials in the oracle pins)."""
    from oracle import observables as ob
    from paper_2111_06893_gb300 import thermonoise
    import workloads as W
    kT, f, r0, d, phi = 300 * ob.BOLTZMANN, 100.0, 1.3, 0.02, 4e-4
    for sub, coat in [(W.FUSED_SILICA, W.COATING_HIGH), (W.COATING_HIGH, W.FUSED_SILICA)]:
        S = thermonoise.thin_coating_psd(kT, f, r0, d, sub, coat, phi)
        U = ob.thin_coating_energy(coat["Y"], coat["nu"], sub["Y"], sub["nu"], d, 1.0, r0)
        ref = ob.noise_psd(np.array([U]), np.array([phi]), kT, f, 1.0)
        assert math.isclose(S, ref, rel_tol=1e-13), (S, ref)
    with pytest.raises(thermonoise.ThermonoiseError):
        thermonoise.thin_coating_psd(kT, f, r0, -d, W.FUSED_SILICA, W.COATING_HIGH, phi)
