"""Writes oracle_gradients.json: the oracle's layer energies and their exact
derivatives (complex step through the whole oracle, iteratively refined
solves with extended-precision residuals, oracle/gradient.py) for the
gradient test meshes of tests/cases.py:

  layered_box    three materials in a clamped box (well conditioned)
  thin_cylinder  two thin coatings (0.02, 0.05) on a cylinder, cond(A) ~ 1e8
  tie_stack      four equal cubic layers of 2^-11: exact ties of
                 min(h_int, h_ext) at every coating interface

For every parameter (slab boundaries s >= 1, the beam width r0, and per
layer c11, c12, c44 for cubic or Y, nu for isotropic materials) the record
holds dU_i/dtheta for every layer i.  Regression records of the oracle,
computed by oracle/ alone; the oracle's complex-step derivatives are pinned
against central finite differences in test_oracle_pins.py.  Run from the
repository root (about half an hour on 8 cores):

    python tests/golden/make_gradient_golden.py [case ...]
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))                    # tests/ (cases)
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))   # repository root

import numpy as np  # noqa: E402

from cases import layered_box, thin_cylinder, tie_stack  # noqa: E402
from oracle import gradient as G  # noqa: E402

CASES = {"layered_box": layered_box, "thin_cylinder": thin_cylinder, "tie_stack": tie_stack}
PATH = os.path.join(HERE, "oracle_gradients.json")


def parameters(desc):
    ps = [["slab_z", s] for s in range(1, len(desc["slab_z"]))] + [["r0"]]
    for L, m in enumerate(desc["materials"]):
        for key in (["c11", "c12", "c44"] if m["kind"] == "cubic" else ["Y", "nu"]):
            ps.append(["material", L, key])
    return ps


def compute(name):
    desc = CASES[name]()
    rec = {"U": [float(v) for v in G.energies(desc)], "dU": {}}
    for p in parameters(desc):
        t0 = time.time()
        d = G.energy_derivative(desc, tuple(p))
        rec["dU"][json.dumps(p)] = [float(v) for v in d]
        print(name, p, f"{time.time() - t0:.0f} s", flush=True)
    return rec


if __name__ == "__main__":
    names = sys.argv[1:] or list(CASES)
    out = {}
    if os.path.exists(PATH):
        with open(PATH) as f:
            out = json.load(f)
    for name in names:
        out[name] = compute(name)
        with open(PATH, "w") as f:
            json.dump(out, f, indent=1, sort_keys=True)
            f.write("\n")
    print("wrote", PATH)
