"""Writes oracle_energies.json: layer energies of small seeded meshes,
computed by the FP64 oracle alone (explicit operator, direct sparse solve,
Sec. 2.1 energies), plus the oracle's closed-form half-space energy for the
isotropic cube workload's material and beam.  These are regression records
of the oracle, not pins: the pins are the closed forms and invariants of
test_oracle_pins.py.  Run from the repository root:

    python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))                    # tests/ (cases)
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))   # repository root

import workloads as W  # noqa: E402
from cases import box_layers, box_tiny, cyl_small  # noqa: E402
from oracle import Mesh, Operator, observables as ob  # noqa: E402

CASES = {
    "box_tiny_p3": lambda: box_tiny(3),
    "box_layers_p4": lambda: box_layers(4),
    "cyl_small_p4_k1": lambda: cyl_small(4, 1),
    "plain_box": W.plain_box,
}


def compute():
    out = {}
    for name, make in CASES.items():
        desc = make()
        op = Operator(Mesh(desc))
        u = ob.solve(op.assemble(), op.rhs())
        out[name] = {"layer_energies": [float(x) for x in ob.layer_energies(op, u)]}
    d = W.plain_box()
    mat = d["materials"][-1]
    out["half_space_plain_box"] = ob.half_space_energy(mat["Y"], mat["nu"], d["beam"]["F0"], d["beam"]["r0"])
    return out


if __name__ == "__main__":
    path = os.path.join(HERE, "oracle_energies.json")
    with open(path, "w") as f:
        json.dump(compute(), f, indent=1, sort_keys=True)
        f.write("\n")
    print("wrote", path)
