"""Stored oracle records (tests/golden/oracle_energies.json, written by
tests/golden/make_golden.py from the oracle alone): the oracle still
reproduces them (CPU, the fast case; the GPU solves of the same meshes are
compared with the live oracle in test_parity_gpu.py)."""
import json
import math
import os

import numpy as np
import workloads as W
from cases import box_layers, box_tiny, cyl_small

HERE = os.path.dirname(os.path.abspath(__file__))
with open(os.path.join(HERE, "golden", "oracle_energies.json")) as f:
    GOLDEN = json.load(f)

CASES = {
    "box_tiny_p3": lambda: box_tiny(3),
    "box_layers_p4": lambda: box_layers(4),
    "cyl_small_p4_k1": lambda: cyl_small(4, 1),
    "plain_box": W.plain_box,
}


def test_oracle_reproduces_its_record():
    from oracle import Mesh, Operator, observables as ob
    op = Operator(Mesh(CASES["box_tiny_p3"]()))
    U = ob.layer_energies(op, ob.solve(op.assemble(), op.rhs()))
    ref = np.array(GOLDEN["box_tiny_p3"]["layer_energies"])
    assert np.max(np.abs(U - ref) / ref) < 1e-12
    d = W.plain_box()
    mat = d["materials"][-1]
    hs = ob.half_space_energy(mat["Y"], mat["nu"], d["beam"]["F0"], d["beam"]["r0"])
    assert math.isclose(hs, GOLDEN["half_space_plain_box"], rel_tol=1e-15)


def test_records_cover_every_case():
    assert set(CASES) <= set(GOLDEN)
    for name in CASES:
        U = GOLDEN[name]["layer_energies"]
        assert len(U) == len(CASES[name]()["materials"]) and min(U) > 0



def test_oracle_reproduces_its_gradient_record():
    """tests/golden/oracle_gradients.json (make_gradient_golden.py, oracle/
    alone): the layered box's energies and every derivative recomputed."""
    import json as _json
    from cases import layered_box
    from oracle import gradient as G
    path = os.path.join(HERE, "golden", "oracle_gradients.json")
    with open(path) as f:
        rec = _json.load(f)
    assert {"layered_box", "thin_cylinder", "tie_stack"} <= set(rec)
    desc = layered_box()
    r = rec["layered_box"]
    assert np.max(np.abs(G.energies(desc) - np.array(r["U"])) / np.array(r["U"])) < 1e-12
    for key, dU in r["dU"].items():
        d = G.energy_derivative(desc, tuple(_json.loads(key)))
        assert np.max(np.abs(d - np.array(dU))) <= 1e-10 * np.max(np.abs(dU)), key
