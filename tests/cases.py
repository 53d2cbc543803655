"""Named mesh descriptions used by the parity tests (plain data from
workloads; no method arithmetic)."""
import workloads as W


def box_tiny(degree=3):
    return W.box([-1.0, 0.2], [-0.5, 1.0], [0.0, -1.3], degree, W.FUSED_SILICA,
                 penalty_C=1.5, bc_side="fixed", bc_bottom="fixed")


def box_layers(degree=4, bc_side="fixed", bc_bottom="free"):
    return W.box([-2.0, -0.5, 0.7, 2.0], [-1.0, 0.3, 1.5], [0.0, -0.05, -0.3, -1.0, -2.5], degree,
                 None, slab_layer=[0, 1, 2, 2], materials=[W.CRYSTAL_A, W.COATING_HIGH, W.FUSED_SILICA],
                 penalty_C=3.0, bc_side=bc_side, bc_bottom=bc_bottom, r0=0.8, F0=1.7)


def cyl_small(degree=4, k=2, thick=(0.05, 0.02), n_sub=2, bc_side="free", bc_bottom="fixed"):
    mats = [W.CRYSTAL_B if i % 2 else W.COATING_HIGH for i in range(len(thick))]
    return W.cylinder(10.0, 10.0, list(thick), mats, W.FUSED_SILICA, k, degree, n_sub,
                      penalty_C=100.0, bc_side=bc_side, bc_bottom=bc_bottom, r0=1.2, F0=1.0)


def cyl_thin(degree=5):
    """Crystalline-like stack: 4 cubic layers of 4e-4 (extreme aspect ratio)."""
    mats = [W.CRYSTAL_A if i % 2 == 0 else W.CRYSTAL_B for i in range(4)]
    return W.cylinder(10.0, 10.0, [4e-4] * 4, mats, W.FUSED_SILICA, 1, degree, 2)


CASES = {
    "box_tiny_p2": lambda: box_tiny(2),
    "box_tiny_p8": lambda: box_tiny(8),
    "plain_box": W.plain_box,
    "box_layers_p4": lambda: box_layers(4),
    "box_layers_allfree_p3": lambda: box_layers(3, "free", "free"),
    "box_layers_allfixed_p5": lambda: box_layers(5, "fixed", "fixed"),
    "cyl_small_p4_k2": lambda: cyl_small(4, 2),
    "cyl_small_p4_k1": lambda: cyl_small(4, 1),
    "cyl_small_p6_k1": lambda: cyl_small(6, 1),
    "cyl_small_p7_k1_fixed": lambda: cyl_small(7, 1, bc_side="fixed"),
    "cyl_thin_p5": cyl_thin,
}


def layered_box():
    """Three materials (cubic, isotropic coating, substrate) in a clamped box."""
    return W.box([-1.0, 0.2, 1.0], [-0.5, 1.0], [0.0, -0.3, -0.8, -1.3], 3, None, slab_layer=[0, 1, 2],
                 materials=[W.CRYSTAL_A, W.COATING_HIGH, W.FUSED_SILICA], penalty_C=3.0,
                 bc_side="fixed", bc_bottom="fixed", r0=0.7)


def thin_cylinder():
    """Two thin coatings (cubic 0.02, isotropic 0.05) on a cylinder, p = 3.
    The geometric substrate slabs share one depth ratio, so the two slabs
    meeting at the inner substrate boundary would have equal face sizes h
    there (a kink of min(h_int, h_ext)); that boundary is moved off the
    geometric sequence so that every slab derivative is two-sided."""
    d = W.cylinder(10.0, 10.0, [0.02, 0.05], [W.CRYSTAL_B, W.COATING_HIGH], W.FUSED_SILICA, 1, 3, 2,
                   r0=1.3)
    z = list(d["slab_z"])
    z[3] = -0.9
    d["slab_z"] = z
    return d


def tie_stack(degree=3):
    """The crystalline multilayer in miniature: four alternating cubic layers
    of equal thickness 2^-11 (~4.9e-4; dyadic, so that the slab positions and
    thicknesses are exact and both sides of every coating interface have the
    same face size h bit for bit: exact ties of min(h_int, h_ext)) on fused
    silica, one element per layer, p = 3.  The substrate boundary is moved off
    the geometric sequence (no tie there)."""
    t = 2.0 ** -11
    mats = [W.CRYSTAL_A if i % 2 == 0 else W.CRYSTAL_B for i in range(4)]
    d = W.cylinder(10.0, 10.0, [t] * 4, mats, W.FUSED_SILICA, 1, degree, 2, r0=1.3)
    z = list(d["slab_z"])
    z[5] = -0.15
    d["slab_z"] = z
    return d
