"""Python binding of the thermonoise C ABI (include/thermonoise.h).

Argument marshalling only: every step runs in the CUDA library.  PyTorch
supplies device memory (tensors) and the CUDA stream.  There is no CPU
fallback: if the shared library is missing or no GPU is present the calls
raise.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libthermonoise.so")

TN_OK = 0
TN_EINVAL_CODE = -1
TN_MESH_BOX, TN_MESH_CYLINDER = 0, 1
TN_BC_FREE, TN_BC_FIXED = 0, 1
TN_F64, TN_F32 = 0, 1
TN_ISO, TN_CUBIC = 0, 1
TN_SOLVE_F64, TN_SOLVE_MIXED_F32 = 0, 1
TN_PC_JACOBI, TN_PC_ZLINE, TN_PC_ZGROUP = 0, 1, 2
PRECONDS = {"jacobi": TN_PC_JACOBI, "zline": TN_PC_ZLINE, "zgroup": TN_PC_ZGROUP}
STATUS = {0: "TN_OK", -1: "TN_EINVAL", -2: "TN_ENOMEM", -3: "TN_ECUDA", -4: "TN_ENOTCONV",
          -5: "TN_EBREAKDOWN", -6: "TN_ETIMEOUT", -7: "TN_ESTATE"}
STATUS_CODE = {v: k for k, v in STATUS.items()}

# every entry point declared in include/thermonoise.h
SYMBOLS = ["tn_create", "tn_destroy", "tn_last_error", "tn_build_mesh", "tn_ndof",
           "tn_set_materials", "tn_set_beam", "tn_apply_operator", "tn_rhs", "tn_diagonal",
           "tn_solve", "tn_layer_energies", "tn_noise_psd", "tn_precond_apply", "tn_energy_grad", "tn_batch_create", "tn_batch_set",
           "tn_batch_offsets", "tn_batch_energy_grad", "tn_layer_energies_noalloc", "tn_precond_factor_bytes",
           "tn_apply_tuning", "tn_set_apply_variant", "tn_iso_moduli", "tn_fma_peak",
           "tn_layer_energy_parts", "tn_thin_coating_psd"]


class MeshDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("degree", C.c_int), ("nx", C.c_int), ("ny", C.c_int),
                ("x_breaks", C.POINTER(C.c_double)), ("y_breaks", C.POINTER(C.c_double)),
                ("R", C.c_double), ("a", C.c_double), ("R1", C.c_double), ("k", C.c_int),
                ("n_slabs", C.c_int), ("slab_z", C.POINTER(C.c_double)),
                ("slab_layer", C.POINTER(C.c_int)), ("slab_log", C.POINTER(C.c_int)),
                ("n_layers", C.c_int), ("penalty_C", C.c_double), ("bc_side", C.c_int),
                ("bc_bottom", C.c_int)]


class Material(C.Structure):
    _fields_ = [("kind", C.c_int), ("Y", C.c_double), ("nu", C.c_double),
                ("c11", C.c_double), ("c12", C.c_double), ("c44", C.c_double)]


class SolveOpts(C.Structure):
    _fields_ = [("mode", C.c_int), ("precond", C.c_int), ("rtol", C.c_double),
                ("inner_rtol", C.c_double), ("max_iter", C.c_int), ("max_outer", C.c_int),
                ("use_x0", C.c_int), ("check_every", C.c_int), ("inner_max", C.c_int),
                ("fcg_window", C.c_int), ("energy_rtol", C.c_double),
                ("device_wait_limit_s", C.c_double)]


class SolveReport(C.Structure):
    _fields_ = [("status", C.c_int), ("outer_iters", C.c_int), ("inner_iters", C.c_int),
                ("applies_f64", C.c_int), ("applies_f32", C.c_int), ("launches", C.c_int64),
                ("rel_residual", C.c_double), ("energy_change", C.c_double),
                ("seconds", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ThermonoiseError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load():
    """Load libthermonoise.so (fails loudly if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2111_06893_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i64p, dp = C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double)
    sig = {
        "tn_create": (C.c_int, [C.POINTER(vp), C.c_int, vp]),
        "tn_destroy": (None, [vp]),
        "tn_last_error": (C.c_char_p, []),
        "tn_build_mesh": (C.c_int, [vp, C.POINTER(MeshDesc)]),
        "tn_ndof": (C.c_int, [vp, i64p]),
        "tn_set_materials": (C.c_int, [vp, C.c_int, C.POINTER(Material)]),
        "tn_set_beam": (C.c_int, [vp, C.c_double, C.c_double]),
        "tn_apply_operator": (C.c_int, [vp, C.c_int, vp, vp]),
        "tn_rhs": (C.c_int, [vp, vp]),
        "tn_diagonal": (C.c_int, [vp, vp]),
        "tn_solve": (C.c_int, [vp, C.POINTER(SolveOpts), vp, C.POINTER(SolveReport)]),
        "tn_layer_energies": (C.c_int, [vp, vp, dp]),
        "tn_noise_psd": (C.c_int, [dp, dp, C.c_int, C.c_double, C.c_double, C.c_double, dp]),
        "tn_iso_moduli": (C.c_int, [C.c_double, C.c_double, dp, dp]),
        "tn_fma_peak": (C.c_int, [C.c_int, C.c_int, dp]),
        "tn_thin_coating_psd": (C.c_int, [C.c_double] * 9 + [dp]),
        "tn_precond_apply": (C.c_int, [vp, C.c_int, C.c_int, vp, vp]),
        "tn_precond_factor_bytes": (C.c_int, [vp, C.c_int, C.POINTER(C.c_longlong)]),
        "tn_energy_grad": (C.c_int, [vp, C.POINTER(SolveOpts), vp, dp, vp, dp, dp, dp,
                                     C.POINTER(SolveReport)]),
        "tn_layer_energies_noalloc": (C.c_int, [vp, vp, dp]),
        "tn_layer_energy_parts": (C.c_int, [vp, vp, dp]),
        "tn_batch_create": (C.c_int, [vp, C.c_int]),
        "tn_batch_set": (C.c_int, [vp, C.c_int, C.POINTER(MeshDesc), C.c_int, C.POINTER(Material),
                                   C.c_double, C.c_double]),
        "tn_batch_offsets": (C.c_int, [vp, i64p, C.POINTER(C.c_int)]),
        "tn_batch_energy_grad": (C.c_int, [vp, C.POINTER(SolveOpts), vp, dp, vp, dp, dp, dp,
                                           C.POINTER(SolveReport)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status):
    if status != TN_OK:
        raise ThermonoiseError(status, load().tn_last_error().decode())


def _dptr(arr, ctype):
    arr = np.ascontiguousarray(arr, dtype=np.float64 if ctype is C.c_double else np.int32)
    return arr, arr.ctypes.data_as(C.POINTER(ctype))


def mesh_struct(desc):
    """tn_mesh_desc from a workload description (keeps the arrays alive)."""
    keep = []
    d = MeshDesc()
    d.kind = TN_MESH_BOX if desc["kind"] == "box" else TN_MESH_CYLINDER
    d.degree = int(desc["degree"])
    if desc["kind"] == "box":
        xb, px = _dptr(desc["x_breaks"], C.c_double)
        yb, py = _dptr(desc["y_breaks"], C.c_double)
        keep += [xb, yb]
        d.nx, d.ny, d.x_breaks, d.y_breaks = len(xb) - 1, len(yb) - 1, px, py
    else:
        d.R, d.a, d.R1, d.k = desc["R"], desc["a"], desc["R1"], int(desc["k"])
    sz, pz = _dptr(desc["slab_z"], C.c_double)
    sl, pl = _dptr(desc["slab_layer"], C.c_int)
    lg, pg = _dptr(desc["slab_log"], C.c_int)
    keep += [sz, sl, lg]
    d.n_slabs, d.slab_z, d.slab_layer, d.slab_log = len(sz) - 1, pz, pl, pg
    d.n_layers = len(desc["materials"])
    d.penalty_C = float(desc["penalty_C"])
    d.bc_side = TN_BC_FIXED if desc["bc_side"] == "fixed" else TN_BC_FREE
    d.bc_bottom = TN_BC_FIXED if desc["bc_bottom"] == "fixed" else TN_BC_FREE
    return d, keep


def material_array(mats):
    arr = (Material * len(mats))()
    for i, m in enumerate(mats):
        if m["kind"] == "iso":
            arr[i].kind, arr[i].Y, arr[i].nu = TN_ISO, m["Y"], m["nu"]
        else:
            arr[i].kind = TN_CUBIC
            arr[i].c11, arr[i].c12, arr[i].c44 = m["c11"], m["c12"], m["c44"]
    return arr


class Context:
    """One tn_ctx on a CUDA device; work goes on torch's current stream of
    that device unless a stream is given."""

    def __init__(self, device=0, stream=None):
        import torch
        self._torch = torch
        lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("thermonoise needs a CUDA GPU; there is no CPU path")
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        _check(lib.tn_create(C.byref(h), device, C.c_void_p(self.stream.cuda_stream)))
        self._h = h
        self.desc = None

    def close(self):
        if getattr(self, "_h", None):
            load().tn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- set-up
    def build_mesh(self, desc):
        d, keep = mesh_struct(desc)
        _check(load().tn_build_mesh(self._h, C.byref(d)))
        del keep
        self.desc = desc
        self.descs = None
        return self

    def set_materials(self, mats):
        arr = material_array(mats)
        _check(load().tn_set_materials(self._h, len(mats), arr))
        return self

    def set_beam(self, r0, F0):
        _check(load().tn_set_beam(self._h, float(r0), float(F0)))
        return self

    def build_batch(self, descs):
        """Hold many mirrors at once (see tn_batch_create); returns self."""
        lib = load()
        _check(lib.tn_batch_create(self._h, len(descs)))
        for i, d in enumerate(descs):
            md, keep = mesh_struct(d)
            mats = material_array(d["materials"])
            _check(lib.tn_batch_set(self._h, i, C.byref(md), len(d["materials"]), mats,
                                    float(d["beam"]["r0"]), float(d["beam"]["F0"])))
            del keep
        n = len(descs)
        doff = (C.c_int64 * (n + 1))()
        loff = (C.c_int * (n + 1))()
        _check(lib.tn_batch_offsets(self._h, doff, loff))
        self.descs = list(descs)
        self.desc = None
        self.dof_off = np.array(doff[:], dtype=np.int64)
        self.layer_off = np.array(loff[:], dtype=np.int64)
        self.desc = {"materials": [None] * int(self.layer_off[-1])}
        return self

    @property
    def ndof(self):
        n = C.c_int64()
        _check(load().tn_ndof(self._h, C.byref(n)))
        return n.value

    def _vec(self, dtype):
        return self._torch.empty(self.ndof, dtype=dtype, device=self.device)

    def _check_tensor(self, t, dtype, name):
        if not (t.is_cuda and t.dtype == dtype and t.is_contiguous() and t.numel() == self.ndof):
            raise ValueError(f"{name}: need a contiguous {dtype} CUDA tensor of {self.ndof} values")

    # ---- operator and data
    def apply_operator(self, u, y=None):
        torch = self._torch
        prec = TN_F64 if u.dtype == torch.float64 else TN_F32
        if y is None:
            y = torch.empty_like(u)
        self._check_tensor(u, u.dtype, "u")
        self._check_tensor(y, u.dtype, "y")
        _check(load().tn_apply_operator(self._h, prec, C.c_void_p(u.data_ptr()), C.c_void_p(y.data_ptr())))
        return y

    def apply_tuning(self):
        """{degree: {"variant": 0 | 1, "us": [variant 0, variant 1]}} for the
        degrees whose FP32 operator variant is settled (timed by the first
        FP32 apply or mixed solve, or fixed by set_apply_variant)."""
        var = (C.c_int * 7)()
        us = (C.c_double * 14)()
        _check(load().tn_apply_tuning(self._h, var, us))
        return {p: {"variant": var[p - 2], "us": [us[2 * (p - 2)], us[2 * (p - 2) + 1]]}
                for p in range(2, 9) if var[p - 2] >= 0}

    def set_apply_variant(self, degree, variant):
        """Fix the FP32 operator variant (0 or 1) of one degree; -1: time it again."""
        _check(load().tn_set_apply_variant(self._h, int(degree), int(variant)))

    def rhs(self, out=None):
        out = self._vec(self._torch.float64) if out is None else out
        self._check_tensor(out, self._torch.float64, "b")
        _check(load().tn_rhs(self._h, C.c_void_p(out.data_ptr())))
        return out

    def diagonal(self, out=None):
        out = self._vec(self._torch.float64) if out is None else out
        self._check_tensor(out, self._torch.float64, "d")
        _check(load().tn_diagonal(self._h, C.c_void_p(out.data_ptr())))
        return out

    def precond_apply(self, r, z=None, precond="zline"):
        torch = self._torch
        prec = TN_F64 if r.dtype == torch.float64 else TN_F32
        if z is None:
            z = torch.empty_like(r)
        self._check_tensor(r, r.dtype, "r")
        self._check_tensor(z, r.dtype, "z")
        _check(load().tn_precond_apply(self._h, PRECONDS[precond], prec, C.c_void_p(r.data_ptr()),
                                       C.c_void_p(z.data_ptr())))
        return z

    @staticmethod
    def _opts(mode, rtol, inner_rtol, max_iter, max_outer, check_every, precond, energy_rtol):
        o = SolveOpts()
        o.mode = TN_SOLVE_F64 if mode == "f64" else TN_SOLVE_MIXED_F32
        o.precond = PRECONDS[precond]
        o.rtol, o.inner_rtol = rtol, inner_rtol
        o.max_iter, o.max_outer, o.check_every = max_iter, max_outer, check_every
        o.energy_rtol = energy_rtol
        o.inner_max = 300  # adjoint solves: inner runs stop at inner_rtol; 300 only bounds them
        o.use_x0 = 0
        return o

    def _precond(self, precond):
        """None: grouped lines (one mirror or a batch)."""
        return "zgroup" if precond is None else precond

    def precond_factor_bytes(self, precond=None):
        """FP32 factor bytes one FP32 application of the preconditioner reads."""
        b = C.c_longlong(0)
        _check(load().tn_precond_factor_bytes(self._h, PRECONDS[self._precond(precond)], C.byref(b)))
        return int(b.value)

    def energy_grad(self, u, w, mode="f64", rtol=1e-12, inner_rtol=0.05, max_iter=200000, max_outer=60,
                    check_every=25, precond=None, raise_on_error=True):
        """Adjoint gradient of J = sum_i w_i U_i at the solution u: returns
        dJ/dslab_z (n_slabs + 1), dJ/dr0, dJ/d(c11, c12, c44) per layer."""
        precond = self._precond(precond)
        self._check_tensor(u, self._torch.float64, "u")
        nl = len(self.desc["materials"])
        w = np.ascontiguousarray(w, dtype=np.float64)
        if w.shape != (nl,):
            raise ValueError(f"w needs {nl} values")
        batched = getattr(self, "descs", None) is not None
        descs = self.descs if batched else [self.desc]
        ns = sum(len(d["slab_z"]) for d in descs)
        gz = np.zeros(ns)
        gr = np.zeros(len(descs))
        gm = np.zeros(3 * nl)
        o = self._opts(mode, rtol, inner_rtol, max_iter, max_outer, check_every, precond, 0.0)
        rep = SolveReport()
        dp = C.POINTER(C.c_double)
        fn = load().tn_batch_energy_grad if batched else load().tn_energy_grad
        st = fn(self._h, C.byref(o), C.c_void_p(u.data_ptr()), w.ctypes.data_as(dp), None,
                gz.ctypes.data_as(dp), gr.ctypes.data_as(dp), gm.ctypes.data_as(dp), C.byref(rep))
        if raise_on_error:
            _check(st)
        if not batched:
            return {"slab_z": gz, "r0": float(gr[0]), "moduli": gm.reshape(nl, 3), "report": rep.as_dict()}
        out, zo = [], 0
        for i, d in enumerate(descs):
            nz = len(d["slab_z"])
            lo, hi = int(self.layer_off[i]), int(self.layer_off[i + 1])
            out.append({"slab_z": gz[zo:zo + nz], "r0": float(gr[i]), "moduli": gm.reshape(nl, 3)[lo:hi]})
            zo += nz
        return {"instances": out, "report": rep.as_dict()}

    def solve(self, mode="f64", rtol=1e-12, inner_rtol=1e-3, max_iter=200000, max_outer=5000,
              x0=None, check_every=25, out=None, raise_on_error=True, precond=None,
              energy_rtol=0.0, inner_max=None, fcg_window=16, device_wait_limit_s=0.0):
        """precond None: grouped lines.  inner_max None: the library's
        default, 40 FP32 iterations per flexible-CG step with grouped lines
        and 300 otherwise (measured best on the single-coating, crystalline
        and design-sweep workloads)."""
        precond = self._precond(precond)
        o = SolveOpts()
        o.mode = TN_SOLVE_F64 if mode == "f64" else TN_SOLVE_MIXED_F32
        o.precond = PRECONDS[precond]
        o.rtol, o.inner_rtol = rtol, inner_rtol
        o.max_iter, o.max_outer, o.check_every = max_iter, max_outer, check_every
        o.energy_rtol = energy_rtol
        o.inner_max, o.fcg_window = inner_max or 0, fcg_window
        o.device_wait_limit_s = device_wait_limit_s
        u = out if out is not None else self._vec(self._torch.float64)
        o.use_x0 = 0
        if x0 is not None:
            u.copy_(x0)
            o.use_x0 = 1
        rep = SolveReport()
        st = load().tn_solve(self._h, C.byref(o), C.c_void_p(u.data_ptr()), C.byref(rep))
        if raise_on_error:
            _check(st)
        return u, rep.as_dict()

    def layer_energies(self, u):
        self._check_tensor(u, self._torch.float64, "u")
        n = len(self.desc["materials"])
        U = np.zeros(n)
        _check(load().tn_layer_energies(self._h, C.c_void_p(u.data_ptr()),
                                        U.ctypes.data_as(C.POINTER(C.c_double))))
        return U

    def layer_energy_parts(self, u):
        """[n_layers, 3]: dilatational, tetragonal and shear parts of every
        layer energy (tn_layer_energy_parts)."""
        self._check_tensor(u, self._torch.float64, "u")
        n = len(self.desc["materials"])
        P = np.zeros(3 * n)
        _check(load().tn_layer_energy_parts(self._h, C.c_void_p(u.data_ptr()),
                                            P.ctypes.data_as(C.POINTER(C.c_double))))
        return P.reshape(n, 3)


def noise_psd(U, phi, kB_T, f, F0):
    U = np.ascontiguousarray(U, dtype=np.float64)
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    if U.shape != phi.shape:
        raise ValueError("U and phi need the same length")
    out = C.c_double()
    _check(load().tn_noise_psd(U.ctypes.data_as(C.POINTER(C.c_double)),
                               phi.ctypes.data_as(C.POINTER(C.c_double)), len(U), kB_T, f, F0,
                               C.byref(out)))
    return out.value


def thin_coating_psd(kB_T, f, r0, d, substrate, coating, phi_c):
    """Eq. (approx_analytic) through tn_thin_coating_psd; substrate and
    coating are isotropic material dicts {"Y", "nu"}."""
    out = C.c_double()
    _check(load().tn_thin_coating_psd(float(kB_T), float(f), float(r0), float(d), float(substrate["Y"]),
                                      float(substrate["nu"]), float(coating["Y"]), float(coating["nu"]),
                                      float(phi_c), C.byref(out)))
    return out.value


def fma_peak(device=0, precision="f32"):
    """Measured FMA peak of the CUDA cores in flop/s (tn_fma_peak)."""
    out = C.c_double()
    _check(load().tn_fma_peak(int(device), TN_F32 if precision == "f32" else TN_F64, C.byref(out)))
    return out.value


def setup(desc, device=0, stream=None):
    """Context with mesh, materials and beam of a workload description."""
    ctx = Context(device, stream)
    ctx.build_mesh(desc)
    ctx.set_materials(desc["materials"])
    ctx.set_beam(desc["beam"]["r0"], desc["beam"]["F0"])
    return ctx


def iso_moduli(Y, nu, derivatives=False):
    """(c11, c12, c44) of an isotropic material from the library
    (tn_iso_moduli); with derivatives=True also the 3 x 2 matrix
    d(c11, c12, c44)/d(Y, nu)."""
    c = (C.c_double * 3)()
    dc = (C.c_double * 6)()
    _check(load().tn_iso_moduli(float(Y), float(nu), c, dc))
    cs = (c[0], c[1], c[2])
    if not derivatives:
        return cs
    return cs, np.array(dc[:], dtype=np.float64).reshape(3, 2)


def _energy_fn_class():
    import torch

    class EnergyFn(torch.autograd.Function):
        """U = EnergyFn.apply(slab_z, r0, moduli, desc, solve_kw): per-layer
        energies of the mirror `desc` with slab boundary positions slab_z
        (n_slabs + 1, slab_z[0] = 0), beam width r0 and moduli
        [n_layers, 3] = (c11, c12, c44); backward runs the adjoint
        (tn_energy_grad), which reuses the forward operator."""

        @staticmethod
        def forward(ctx, slab_z, r0, moduli, desc, solve_kw):
            d = dict(desc)
            d["slab_z"] = [float(v) for v in slab_z.detach().cpu().tolist()]
            d["beam"] = {"r0": float(r0.detach()), "F0": desc["beam"]["F0"]}
            mats = [{"kind": "cubic", "c11": float(c[0]), "c12": float(c[1]), "c44": float(c[2])}
                    for c in moduli.detach().cpu().tolist()]
            d["materials"] = mats
            tc = setup(d)
            kw = dict(solve_kw or {})
            u, _ = tc.solve(**kw)
            U = tc.layer_energies(u)
            ctx.tc, ctx.u, ctx.kw = tc, u, kw
            return torch.tensor(U, dtype=torch.float64)

        @staticmethod
        def backward(ctx, gU):
            kw = {k: v for k, v in ctx.kw.items() if k in ("mode", "rtol", "inner_rtol", "precond",
                                                         "max_iter", "max_outer", "check_every",
                                                         "raise_on_error")}
            g = ctx.tc.energy_grad(ctx.u, gU.detach().cpu().numpy(), **kw)
            return (torch.tensor(g["slab_z"], dtype=torch.float64), torch.tensor(g["r0"], dtype=torch.float64),
                    torch.tensor(g["moduli"], dtype=torch.float64), None, None)

    return EnergyFn


_ENERGY_FN = None


def energy_fn():
    """The torch.autograd.Function computing per-layer energies (see above)."""
    global _ENERGY_FN
    if _ENERGY_FN is None:
        _ENERGY_FN = _energy_fn_class()
    return _ENERGY_FN
