"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module holds data only: mesh descriptions (plain numbers: element break
points, slab boundaries, layer/material tables, boundary-condition tags, beam
parameters) and seeded random vectors.  It contains none of the method's
arithmetic (no element maps, Jacobians, basis functions or DG terms); each side
interprets a description with its own code.

Description layout (a plain dict, the same for both sides):

  kind         "box" or "cylinder"
  degree       polynomial degree p; N = p + 1 LGL points per dimension
  x_breaks,
  y_breaks     (box) element boundaries along x and y
  R, a, R1, k  (cylinder) outer radius, half-width of the central square,
               radius of the circle between inner and outer wedges, and the
               k x k split of each of the nine cross-section blocks
  slab_z       n_slabs + 1 z values from the top surface z = 0 downwards
  slab_layer   layer id of each slab (coating layers top-down, substrate last)
  slab_log     1 where the slab uses the logarithmic map in depth
  materials    one entry per layer id: {"kind": "iso", "Y", "nu"} or
               {"kind": "cubic", "c11", "c12", "c44"} (Pa)
  penalty_C    the constant C of the penalty sigma = C (p+1)^2 / h
  bc_side      "fixed" (u = 0) or "free" (zero traction) on x/y sides / mantle
  bc_bottom    "fixed" or "free" on the bottom z = slab_z[-1]
  beam         {"r0": beam width, "F0": total force}; the top z = 0 always
               carries the Gaussian pressure of the beam

Element ordering: e = s * n_columns + c, slab s counted from the top, column
c counted in the cross-section.  Box columns: c = jy * n_x + ix.  Cylinder
columns: block-major over the nine blocks [square, inner wedges at 0, 90, 180,
270 degrees, outer wedges at 0, 90, 180, 270 degrees], inside a block
c_local = b * k + a with a counting along the block's first logical axis.
Field layout: u[(e * 3 + comp) * N^3 + (kz * N + jy) * N + ix].
"""
import math

import numpy as np

GPA = 1.0e9


def iso(Y, nu):
    return {"kind": "iso", "Y": float(Y), "nu": float(nu)}


def cubic(c11, c12, c44):
    return {"kind": "cubic", "c11": float(c11), "c12": float(c12), "c44": float(c44)}


FUSED_SILICA = iso(72 * GPA, 0.17)
COATING_HIGH = iso(140 * GPA, 0.23)
CRYSTAL_A = cubic(119.9 * GPA, 53.8 * GPA, 59.4 * GPA)
CRYSTAL_B = cubic(120.5 * GPA, 57.0 * GPA, 58.9 * GPA)


def substrate_slabs(d, H, n):
    """Slab boundaries in depth from d (bottom of the coating) to H, geometric
    so that every slab spans the same ratio of depths (log map inside)."""
    if n < 1:
        raise ValueError("need at least one substrate slab")
    if d <= 0.0:
        raise ValueError("a logarithmic substrate map needs a coating above it")
    return [d * (H / d) ** (i / n) for i in range(n + 1)]


def layered_vertical(thicknesses, H, n_sub):
    """slab_z / slab_layer / slab_log for coating layers (one slab each,
    top-down) above a substrate of total height H split into n_sub slabs."""
    depth = [0.0]
    for t in thicknesses:
        depth.append(depth[-1] + float(t))
    sub = substrate_slabs(depth[-1], H, n_sub)
    depth = depth + sub[1:]
    nl = len(thicknesses)
    slab_layer = list(range(nl)) + [nl] * n_sub
    slab_log = [0] * nl + [1] * n_sub
    return [-s for s in depth], slab_layer, slab_log


def box(x_breaks, y_breaks, z_breaks, degree, material, penalty_C=1.5,
        bc_side="fixed", bc_bottom="fixed", r0=1.0, F0=1.0, slab_layer=None,
        materials=None):
    nz = len(z_breaks) - 1
    return {
        "kind": "box", "degree": int(degree),
        "x_breaks": [float(v) for v in x_breaks],
        "y_breaks": [float(v) for v in y_breaks],
        "slab_z": [float(v) for v in z_breaks],
        "slab_layer": list(slab_layer) if slab_layer is not None else [0] * nz,
        "slab_log": [0] * nz,
        "materials": list(materials) if materials is not None else [material],
        "penalty_C": float(penalty_C),
        "bc_side": bc_side, "bc_bottom": bc_bottom,
        "beam": {"r0": float(r0), "F0": float(F0)},
    }


def cylinder(R, H, thicknesses, coat_materials, substrate, k, degree, n_sub,
             penalty_C=100.0, bc_side="free", bc_bottom="fixed", r0=1.0,
             F0=1.0, a=None, R1=None):
    slab_z, slab_layer, slab_log = layered_vertical(thicknesses, H, n_sub)
    return {
        "kind": "cylinder", "degree": int(degree),
        "R": float(R), "a": float(a if a is not None else R / 5.0),
        "R1": float(R1 if R1 is not None else R / 2.0), "k": int(k),
        "slab_z": slab_z, "slab_layer": slab_layer, "slab_log": slab_log,
        "materials": list(coat_materials) + [substrate],
        "penalty_C": float(penalty_C),
        "bc_side": bc_side, "bc_bottom": bc_bottom,
        "beam": {"r0": float(r0), "F0": float(F0)},
    }


def n_columns(desc):
    if desc["kind"] == "box":
        return (len(desc["x_breaks"]) - 1) * (len(desc["y_breaks"]) - 1)
    return 9 * desc["k"] ** 2


def n_elements(desc):
    return n_columns(desc) * (len(desc["slab_z"]) - 1)


def n_dof(desc):
    N = desc["degree"] + 1
    return 3 * N ** 3 * n_elements(desc)


# --------------------------------------------------------------------------
# The five workloads (plain method box, single coating, crystalline multilayer,
# batched design sweep, large mirror).  Lengths in units of the beam width.
# --------------------------------------------------------------------------

def plain_box():
    """Isotropic box [-10,10]^2 x [-20,0], 4x4x4 straight hexes, p = 3,
    penalty 1.5, u = 0 on the five faces other than z = 0 (12 288 DOF)."""
    br = [-10.0, -5.0, 0.0, 5.0, 10.0]
    return box(br, br, [0.0, -5.0, -10.0, -15.0, -20.0], 3, FUSED_SILICA,
               penalty_C=1.5, bc_side="fixed", bc_bottom="fixed")


def single_coating(k=3, degree=6, n_sub=23):
    """Cylinder R = H = 10, one 0.02-thick isotropic coating (140 GPa, 0.23)
    on fused silica, p = 6: 81 columns x 24 slabs, 2.0 M DOF."""
    return cylinder(10.0, 10.0, [0.02], [COATING_HIGH], FUSED_SILICA, k,
                    degree, n_sub)


def crystalline_multilayer(k=5, degree=5, n_layers=40, n_sub=15):
    """Cylinder R = H = 10, 40 alternating cubic layers of 4e-4 each, p = 5,
    one element per layer: 225 columns x 55 slabs, 8.0 M DOF."""
    mats = [CRYSTAL_A if i % 2 == 0 else CRYSTAL_B for i in range(n_layers)]
    return cylinder(10.0, 10.0, [4e-4] * n_layers, mats, FUSED_SILICA, k,
                    degree, n_sub)


def large_mirror(k=10, degree=8, n_layers=20, n_sub=10):
    """Cylinder R = H = 20, 20 alternating isotropic layers of 1e-3, p = 8:
    900 columns x 30 slabs, 59 M DOF."""
    mats = [FUSED_SILICA if i % 2 == 0 else COATING_HIGH for i in range(n_layers)]
    return cylinder(20.0, 20.0, [1e-3] * n_layers, mats, FUSED_SILICA, k,
                    degree, n_sub)


def sweep_instance(seed):
    """One mirror of the batched design sweep: layer count U{1..20},
    thicknesses log-uniform in [1e-4, 5e-2], r0 ~ U[0.5, 2], p ~ U{4..8},
    R = H = 10, k = 1, four substrate slabs."""
    rng = np.random.default_rng(seed)
    L = int(rng.integers(1, 21))
    th = np.exp(rng.uniform(math.log(1e-4), math.log(5e-2), size=L))
    r0 = float(rng.uniform(0.5, 2.0))
    p = int(rng.integers(4, 9))
    mats = [COATING_HIGH if i % 2 == 0 else FUSED_SILICA for i in range(L)]
    return cylinder(10.0, 10.0, [float(t) for t in th], mats, FUSED_SILICA, 1,
                    p, 4, r0=r0)


def design_sweep(n=256, first=0):
    """Mirrors first .. first + n - 1 of the seeded sweep."""
    return [sweep_instance(s) for s in range(first, first + n)]


def random_field(desc, seed=0):
    """u uniform in [-1, 1] in the field layout above."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=n_dof(desc))
