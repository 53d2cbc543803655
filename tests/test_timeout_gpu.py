"""Bounded device waits (tn_solve_opts.device_wait_limit_s): a line solve
whose staged factor copy has not landed within the limit ends its kernel
after a bounded wait for the copies it has in flight, and the solve returns
TN_ETIMEOUT; the context stays usable.  The limit is run out by setting it
to 1 ns on the 2.0 M DOF single-coating mirror, whose 205 MB of factors
stream from HBM, so that a copy takes far longer than a tick of the GPU's
global timer: every wait is for real copies that do land (no wait is made to
hang)."""
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


@pytest.mark.parametrize("precond", ["zgroup", "zline"])
@pytest.mark.parametrize("mode", ["f64", "mixed"])
def test_wait_limit_runs_out_and_context_stays_usable(precond, mode):
    from paper_2111_06893_gb300 import thermonoise
    desc = W.single_coating()
    ctx = thermonoise.setup(desc)
    u_ok, rep_ok = ctx.solve(mode=mode, rtol=1e-9, precond=precond)
    U_ok = ctx.layer_energies(u_ok)
    status = None
    for _ in range(3):  # a wait that happens to find its copy landed does not time out
        _, rep = ctx.solve(mode=mode, rtol=1e-9, precond=precond, raise_on_error=False,
                           device_wait_limit_s=1e-9)
        status = rep["status"]
        if status == thermonoise.STATUS_CODE["TN_ETIMEOUT"]:
            break
    assert status == thermonoise.STATUS_CODE["TN_ETIMEOUT"], rep
    assert "gave up waiting" in thermonoise.load().tn_last_error().decode()
    # the same context solves again with the default limit
    u2, rep2 = ctx.solve(mode=mode, rtol=1e-9, precond=precond)
    assert rep2["status"] == 0
    U2 = ctx.layer_energies(u2)
    assert np.max(np.abs(U2 - U_ok) / U_ok) < 1e-9


def test_wait_limit_is_validated():
    from paper_2111_06893_gb300 import thermonoise
    desc = W.cylinder(10.0, 10.0, [0.02], [W.COATING_HIGH], W.FUSED_SILICA, 1, 3, 2)
    ctx = thermonoise.setup(desc)
    with pytest.raises(thermonoise.ThermonoiseError) as ei:
        ctx.solve(mode="f64", device_wait_limit_s=-1.0)
    assert ei.value.status == thermonoise.TN_EINVAL_CODE
