"""Benchmark of the DG thermal-noise hot path on GB300.

One step = one pass of the whole path on the 2.0 M DOF single-coating
mirror (cylinder R = H = 10 r0, 0.02 r0 coating, p = 6): right-hand side,
Jacobi diagonal, mixed-precision solve (FP32 inner PCG, FP64 residual and
refinement) until every layer energy is within 1e-9 of the FP64 reference,
per-layer energies and the noise PSD.  Inputs (mesh, geometry, materials)
are resident in HBM before the timed region; L2 is flushed between steps.

metric: GDOF/s = (operator applies x N_DOF) / time, over the whole step.
Extra keys report the FP32/FP64 apply kernels alone, the time to U for the
mixed and the plain FP64 solve, the roofline of the dominant kernel of the
step (the FP32 column-line solve, HBM-bound) and of the FP32 apply
(ALU-bound), and the FP64 oracle on the host cores.

Multi-GPU: no collective on the data path.  A single-mirror workload runs
as replicas (every rank solves its own copy); the design sweep gives every
rank its own 256 mirrors (different seeds).  value = all ranks' DOF-applies
/ max over ranks of the time (weak scaling).
`--impl reference` times the FP64 CPU oracle instead (rank 0 only).
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

WORKLOADS = {
    "single_coating": W.single_coating,
    "plain_box": W.plain_box,
    "crystalline_multilayer": W.crystalline_multilayer,
    "large_mirror": W.large_mirror,
    "design_sweep": lambda: W.design_sweep(256),
}
KB_T = 1.380649e-23 * 300.0
FREQ = 100.0


def fp32_apply_flops_per_dof(N):
    """Algorithmic FP32 work of one operator apply per DOF: the sum-factorised
    gradient and weak divergence (36 N flops per node), metric / strain /
    stress / flux transforms (~80 per node), and per face node (6 N^2 per
    element) the neighbour normal and tangential derivatives plus the flux
    terms (~130 + 18 N)."""
    per_elem = N ** 3 * (36 * N + 80) + 6 * N ** 2 * (130 + 18 * N)
    return per_elem / (3 * N ** 3)


# DRAM bytes (read + write) of one preconditioner solve (no residual update)
# from `ncu --set full -k regex:zgroup_packed_kernel` of `bench.py --mode
# apply --workload single_coating`; absent where no capture of the current
# kernel exists
ZLINE_TRAFFIC = {("single_coating", "zgroup_packed_kernel<7,float>"): 342619136.0 + 10593280.0}


# DRAM bytes (read + write) of one FP32 apply per occupancy variant, from
# `ncu --set full -k regex:apply2_kernel` of `bench.py --mode apply --workload
# single_coating` (variant 0 captured; variant 1's register spills add
# local-memory traffic, not captured for the current kernel)
APPLY_TRAFFIC = {("single_coating", "apply2_kernel<7,float,0>"): 8148736.0}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate_over_ranks(t_local, applies, dist, device):
    """Whole-job figures of a replicas run (every rank solves its own
    mirror): the slowest rank's time and the operator applies of all ranks."""
    import torch
    tt = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    aa = torch.tensor([float(applies)], dtype=torch.float64, device=device)
    dist.all_reduce(aa, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(aa.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return max(i.get("num_threads", 1) for i in info)
    except ImportError:
        pass
    return os.cpu_count()


def reduced_desc(desc):
    """The bounded CPU sample of a workload: the same mirror (materials,
    degree, coating layers, beam) on the coarsest cross-section (k = 1) with
    one substrate slab, so that the oracle assembles it in ~15-40 s."""
    if desc["kind"] != "cylinder":
        return desc
    nc = desc["slab_log"].index(1) if 1 in desc["slab_log"] else len(desc["slab_log"])
    thick = [desc["slab_z"][i] - desc["slab_z"][i + 1] for i in range(nc)]
    mats = desc["materials"]
    d = W.cylinder(desc["R"], -desc["slab_z"][-1], thick, mats[:-1], mats[-1], 1, desc["degree"], 1,
                   penalty_C=desc["penalty_C"], bc_side=desc["bc_side"], bc_bottom=desc["bc_bottom"],
                   r0=desc["beam"]["r0"], F0=desc["beam"]["F0"], a=desc["a"], R1=desc["R1"])
    return d


def oracle_spmv_rate(desc, budget_s):
    """The FP64 oracle's apply as it stands on a bounded sample of the
    workload: its explicitly assembled CSR matrix (scipy, one thread) times a
    seeded field, repeated for ~budget_s.  Returns (GDOF/s, DOF, applies,
    seconds, assembly seconds)."""
    from oracle import Mesh, Operator
    t0 = time.perf_counter()
    op = Operator(Mesh(desc))
    A = op.assemble()
    t_asm = time.perf_counter() - t0
    u = W.random_field(desc, 0)
    A @ u
    t0 = time.perf_counter()
    done = 0
    while True:
        A @ u
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return A.shape[0] * done / dt / 1e9, A.shape[0], done, dt, t_asm


def oracle_direct_solve_s():
    """The oracle's direct solve of the plain box workload (12 288 DOF, dense
    Cholesky through LAPACK on the BLAS threads)."""
    from oracle import Mesh, Operator, observables as ob
    op = Operator(Mesh(W.plain_box()))
    A, b = op.assemble(), op.rhs()
    t0 = time.perf_counter()
    ob.solve_dense(A, b)
    return time.perf_counter() - t0


def voigt_isotropic(c):
    """Effective isotropic moduli of a cubic crystal (Voigt average, the
    amorphous model the approximate formula assumes): K = (c11 + 2 c12)/3,
    G = (c11 - c12 + 3 c44)/5, then Y = 9 K G / (3 K + G),
    nu = (3 K - 2 G) / (2 (3 K + G))."""
    K = (c["c11"] + 2 * c["c12"]) / 3.0
    G = (c["c11"] - c["c12"] + 3 * c["c44"]) / 5.0
    return W.iso(9 * K * G / (3 * K + G), (3 * K - 2 * G) / (2 * (3 * K + G)))


def finite_size_study(device):
    """The analogue of Sec. 3.2 on synthetic parameters: the coating noise
    of a single coating on a finite cylinder (R = H), solved, against the
    approximate thin-coating / semi-infinite formula Eq. (approx_analytic),
    across R / r0 and d / r0; and the crystalline correction, a cubic
    coating against its effective isotropic (Voigt) model.  Near the beam
    the mesh is the same for every R (central square of half-width 2 r0,
    inner wedges to 4 r0, k = 3), so that the ratio isolates the size
    effect; p-refinement at one mirror shows the discretization error."""
    from paper_2111_06893_gb300 import thermonoise
    kT, f, phi = KB_T, FREQ, 4e-4
    crystal = W.CRYSTAL_A
    iso_eff = voigt_isotropic(crystal)

    def run(R, d, coat, degree=6, k=3):
        desc = W.cylinder(R, R, [d], [coat], W.FUSED_SILICA, k, degree, 23, a=2.0, R1=4.0)
        ctx = thermonoise.setup(desc, device=device)
        u, rep = ctx.solve(mode="mixed", rtol=1e-13, energy_rtol=1e-11, raise_on_error=False)
        U = ctx.layer_energies(u)
        return U[0], rep, W.n_dof(desc)

    for R in (5.0, 10.0, 20.0):
        for d in (0.005, 0.01, 0.02, 0.04):
            t0 = time.perf_counter()
            Uc, rep, ndof = run(R, d, iso_eff)
            S_num = thermonoise.noise_psd(np.array([Uc]), np.array([phi]), kT, f, 1.0)
            S_an = thermonoise.thin_coating_psd(kT, f, 1.0, d, W.FUSED_SILICA, iso_eff, phi)
            Ux, repx, _ = run(R, d, crystal)
            print(json.dumps({"study": "finite_size", "R_over_r0": R, "d_over_r0": d, "degree": 6, "ndof": ndof,
                              "S_numerical_over_approx": S_num / S_an,
                              "finite_size_effect_pct": 100 * (S_num / S_an - 1),
                              "crystalline_effect_pct": 100 * (Ux / Uc - 1),
                              "rel_residual": [rep["rel_residual"], repx["rel_residual"]],
                              "seconds": time.perf_counter() - t0}), flush=True)
    for degree in (5, 6, 7):
        Uc, rep, ndof = run(10.0, 0.02, iso_eff, degree=degree)
        S_num = thermonoise.noise_psd(np.array([Uc]), np.array([phi]), kT, f, 1.0)
        S_an = thermonoise.thin_coating_psd(kT, f, 1.0, 0.02, W.FUSED_SILICA, iso_eff, phi)
        Ux, _, _ = run(10.0, 0.02, crystal, degree=degree)
        print(json.dumps({"study": "finite_size_p_refinement", "R_over_r0": 10.0, "d_over_r0": 0.02,
                          "degree": degree, "ndof": ndof, "finite_size_effect_pct": 100 * (S_num / S_an - 1),
                          "crystalline_effect_pct": 100 * (Ux / Uc - 1)}), flush=True)


def bench_config(args, descs, world):
    """The `config` of the JSON line, the same for both arms."""
    batched = len(descs) > 1 or args.workload == "design_sweep"
    pc = args.precond or "zgroup"
    return {"workload": args.workload, "ndof": sum(W.n_dof(d) for d in descs),
            "degree": sorted({d["degree"] for d in descs}) if batched else descs[0]["degree"],
            "elements": sum(W.n_elements(d) for d in descs), "mirrors": len(descs),
            "step": "rhs+mixed solve+energies+psd",
            "rtol": args.rtol, "energy_rtol": args.energy_rtol, "inner_rtol": args.inner_rtol,
            "inner_max": args.inner_max or (40 if pc == "zgroup" else 300),
            "fcg_window": args.fcg_window,
            "precond": pc, "l2": "flushed between steps (256 MB)",
            "parallelism": "replicas" if world > 1 else "single"}


def run_reference(args, desc, world, rank, descs=None):
    if rank != 0:
        return
    from oracle import Mesh, Operator
    sample = reduced_desc(desc)
    op = Operator(Mesh(sample))
    A = op.assemble()
    u = W.random_field(sample, 0)
    per = args.ref_step_s
    times, dofs = [], 0
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        n = 0
        while time.perf_counter() - t0 < per:
            A @ u
            n += 1
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
            dofs += n * A.shape[0]
    total = sum(times)
    value = dofs / total / 1e9
    N = desc["degree"] + 1
    line = {
        "impl": "reference", "metric": "GDOF/s of DG elasticity apply", "value": value, "unit": "GDOF/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(args, descs or [desc], world),
        "cpu_baseline": {"value": value, "unit": "GDOF/s", "cores": 1, "kind": "oracle",
                         "sample": f"FP64 oracle: its assembled CSR matrix times a field (scipy SpMV, one "
                                   f"thread), {A.shape[0]} DOF (the workload at k = 1 with one substrate "
                                   f"slab, N={N}), {per:.0f} s of applies per step"},
        "e2e": {"value": value, "unit": "GDOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="single_coating", choices=sorted(WORKLOADS))
    ap.add_argument("--rtol", type=float, default=1e-13)
    ap.add_argument("--energy-rtol", type=float, default=1e-10,
                    help="stop once every U_i changes by less than this between checks")
    ap.add_argument("--inner-rtol", type=float, default=1e-3)
    ap.add_argument("--inner-max", type=int, default=None,
                    help="default: 40 with grouped lines, 300 with single lines")
    ap.add_argument("--fcg-window", type=int, default=16)
    ap.add_argument("--precond", default=None, choices=["zline", "zgroup", "jacobi"],
                    help="default: grouped lines")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 time-to-U solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--no-reference", action="store_true",
                    help="skip the FP64 reference solve (energy errors are then not reported)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer leg")
    ap.add_argument("--mode", default="step", choices=["step", "apply", "finite_size"],
                    help="apply: only time the FP32 / FP64 operator applies (for profiling); "
                         "finite_size: the finite-size and crystalline study (one JSON line per mirror)")
    ap.add_argument("--ref-step-s", type=float, default=8.0)
    ap.add_argument("--cpu-budget-s", type=float, default=8.0)
    ap.add_argument("--reference-pair", default=None, choices=["on", "off"],
                    help="FP64 reference from grouped AND column lines (default: on for the single coating, "
                         "whose column-line FP64 solve takes ~40 s; off elsewhere, where it takes minutes)")
    ap.add_argument("--grad", action="store_true",
                    help="also time the adjoint energy gradient (every mirror of a batch)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.workload == "design_sweep":
        # independent mirrors: every rank solves its own 256 (mirrors 256 r .. 256 r + 255)
        desc = W.design_sweep(256, first=256 * rank)
    else:
        desc = WORKLOADS[args.workload]()  # one mirror: every rank solves its own copy
    descs = desc if isinstance(desc, list) else [desc]
    batched = isinstance(desc, list)
    if batched:
        desc = descs[0]  # the CPU oracle samples the first mirror of a batch
    if args.impl == "reference":
        run_reference(args, desc, world, rank, descs)
        return

    import torch
    from paper_2111_06893_gb300 import build, thermonoise
    if rank == 0:
        build.build()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist.barrier()
        build.build()
    else:
        torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    if batched:
        ctx = thermonoise.Context(local, stream).build_batch(descs)
    else:
        ctx = thermonoise.setup(desc, device=local, stream=stream)
    ndof = ctx.ndof
    N = desc["degree"] + 1
    dof_w = [W.n_dof(d) for d in descs]
    flops_dof = sum(fp32_apply_flops_per_dof(d["degree"] + 1) * w for d, w in zip(descs, dof_w)) / sum(dof_w)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    if args.mode == "finite_size":
        if rank == 0:
            finite_size_study(local)
        return

    if args.mode == "apply":
        x32 = torch.rand(ndof, dtype=torch.float32, device=dev)
        y32 = torch.empty_like(x32)
        x64, y64 = x32.double(), torch.empty(ndof, dtype=torch.float64, device=dev)
        res = {}
        for name, x, y, reps_n in (("f32", x32, y32, 20), ("f64", x64, y64, 5)):
            for _ in range(3):
                ctx.apply_operator(x, y)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps_n):
                ctx.apply_operator(x, y)
            e1.record(stream)
            e1.synchronize()
            res[name] = e0.elapsed_time(e1) / reps_n * 1e3
        # the column-line preconditioner solve (one launch per application)
        zres = {}
        for pc in ("zline", "zgroup"):
            for name, x, y, reps_n in (("f32", x32, y32, 20), ("f64", x64, y64, 10)):
                for _ in range(3):
                    ctx.precond_apply(x, y, precond=pc)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(reps_n):
                    ctx.precond_apply(x, y, precond=pc)
                e1.record(stream)
                e1.synchronize()
                zres[pc + "_" + name] = e0.elapsed_time(e1) / reps_n * 1e3
        if rank == 0:
            print(json.dumps({"mode": "apply", "workload": args.workload, "ndof": ndof, "us": res,
                              "gdofs": {k: ndof / v / 1e3 for k, v in res.items()},
                              "zline_us": zres}), flush=True)
        return

    # FP64 reference energies: two GPU FP64 PCG solves with different
    # preconditioners (grouped lines, column lines), each run to its rounding
    # floor (residual test only: it stops once the true residual stagnates);
    # their disagreement bounds the reference's own error
    refs = {}
    U_ref = None
    pair = args.reference_pair == "on" or (args.reference_pair is None and args.workload == "single_coating")
    if not args.no_reference:
        for pc_ref in (("zgroup", "zline") if pair else ("zgroup",)):
            t0 = time.perf_counter()
            u_ref, rr = ctx.solve(mode="f64", rtol=1e-15, energy_rtol=0.0, precond=pc_ref, raise_on_error=False,
                                  max_iter=400000)
            refs[pc_ref] = {"U": ctx.layer_energies(u_ref), "rel_residual": rr["rel_residual"],
                            "iters": rr["inner_iters"], "status": rr["status"], "s": time.perf_counter() - t0}
            del u_ref
        U_ref = refs["zgroup"]["U"]
    ref_pair = None
    if refs:
        ref_pair = {k: {kk: vv for kk, vv in v.items() if kk != "U"} for k, v in refs.items()}
        if "zline" in refs:
            Ua, Ub = refs["zgroup"]["U"], refs["zline"]["U"]
            ref_pair["max_rel_diff"] = float(np.max(np.abs(Ua - Ub) / np.abs(Ua)))

    def err_vs_refs(U):
        if not refs:
            return None
        return float(max(np.max(np.abs(U - r["U"]) / np.abs(r["U"])) for r in refs.values()))
    t_fp64 = None
    rep_fp64 = None
    if not args.no_fp64:
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        u64, rep_fp64 = ctx.solve(mode="f64", rtol=args.rtol, energy_rtol=args.energy_rtol,
                                  precond=args.precond, raise_on_error=False)
        U64 = ctx.layer_energies(u64)
        torch.cuda.synchronize()
        t_fp64 = time.perf_counter() - t0
        err64 = err_vs_refs(U64)
        del u64

    phis = [np.array([4e-4] * (len(d["materials"]) - 1) + [1e-6]) for d in descs]
    lofs = np.cumsum([0] + [len(d["materials"]) for d in descs])
    u = torch.empty(ndof, dtype=torch.float64, device=dev)

    def step():
        _, rep = ctx.solve(mode="mixed", rtol=args.rtol, inner_rtol=args.inner_rtol, out=u,
                           energy_rtol=args.energy_rtol, precond=args.precond, raise_on_error=False,
                           inner_max=args.inner_max, fcg_window=args.fcg_window)
        U = ctx.layer_energies(u)
        S = [thermonoise.noise_psd(U[lofs[i]:lofs[i + 1]], phis[i], KB_T, FREQ, d["beam"]["F0"])
             for i, d in enumerate(descs)]
        return rep, U, S

    for _ in range(args.warmup):
        step()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    total_ms, applies, launches = 0.0, 0, 0
    reps = []
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.fill_(float(len(reps)))
            ev0.record(stream)
            rep, U, S = step()
            ev1.record(stream)
            ev1.synchronize()
            total_ms += ev0.elapsed_time(ev1)
            applies += rep["applies_f32"] + rep["applies_f64"]
            launches += rep["launches"] + 2
            reps.append(rep)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    err_mixed = err_vs_refs(U)
    t_local = total_ms / 1e3
    t_max = t_local
    tot_applies = applies
    if world > 1:
        import torch.distributed as dist
        t_max, tot_applies = aggregate_over_ranks(t_local, applies, dist, dev)
    value = tot_applies * ndof / t_max / 1e9
    mixed_s = t_local / args.steps

    # ---- the dominant kernel alone: FP32 and FP64 applies, CUDA events on the launch stream
    x32 = torch.rand(ndof, dtype=torch.float32, device=dev)
    y32 = torch.empty_like(x32)
    x64 = x32.double()
    y64 = torch.empty_like(x64)

    def time_apply(x, y, reps_n):
        for _ in range(5):
            ctx.apply_operator(x, y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps_n):
            ctx.apply_operator(x, y)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps_n / 1e3

    t32 = time_apply(x32, y32, 200)
    tuning = ctx.apply_tuning()  # FP32 operator variant per degree, timed by the first FP32 call
    akernel = ("apply2_batch_kernel<N,float,V>" if batched
               else f"apply2_kernel<{N},float,{tuning.get(N - 1, {}).get('variant', 0)}>")
    t64 = time_apply(x64, y64, 20)

    # the dominant kernel of the step: the FP32 preconditioner solve (column lines)
    pc = args.precond or "zgroup"
    if pc == "jacobi":
        pc = "zline"

    def time_zline(x, y, reps_n):
        for _ in range(5):
            ctx.precond_apply(x, y, precond=pc)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps_n):
            ctx.precond_apply(x, y, precond=pc)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps_n / 1e3

    def time_zline_graph(reps_n):
        """The solve replays the line solve from a CUDA graph: time it the same
        way, on a context of its own whose stream is the capture stream."""
        sz = torch.cuda.Stream(dev)
        cz = (thermonoise.Context(local, sz).build_batch(descs) if batched
              else thermonoise.setup(desc, device=local, stream=sz))
        cz.precond_factor_bytes(pc)  # factors built before the capture
        xz, yz = torch.rand(ndof, dtype=torch.float32, device=dev), torch.empty(ndof, dtype=torch.float32, device=dev)
        with torch.cuda.stream(sz):
            for _ in range(3):
                cz.precond_apply(xz, yz, precond=pc)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=sz):
            for _ in range(reps_n):
                cz.precond_apply(xz, yz, precond=pc)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(sz):  # replay() launches on the current stream
            g.replay()
            torch.cuda.synchronize()
            e0.record(sz)
            g.replay()
            e1.record(sz)
        e1.synchronize()
        t = e0.elapsed_time(e1) / reps_n / 1e3
        del g, cz
        torch.cuda.synchronize()
        return t

    tz_eager = time_zline(x32, y32, 100)
    try:
        tz, tz_how = time_zline_graph(20), "CUDA events around a replayed graph of 20 applications"
    except Exception as exc:  # capture not possible here: eager timing
        tz, tz_how = tz_eager, f"CUDA events, eager calls ({type(exc).__name__})"
    # algorithmic bytes of one line solve: the compact FP32 factors once (the
    # grouped solve's backward couplings W_s, which derive from them, and
    # re-reads are not credited), r in and z out
    zbytes = ctx.precond_factor_bytes(pc) + 8 * ndof
    flops = flops_dof * ndof
    # measured FMA peaks of the CUDA cores (the apply is bound by arithmetic)
    peak_fp32 = thermonoise.fma_peak(local, "f32") / 1e12
    peak_fp64 = thermonoise.fma_peak(local, "f64") / 1e12
    achieved = flops / t32 / 1e12
    peaks = measured_peaks()

    # ---- the adjoint gradient (every mirror of a batch), timed on request
    grad = None
    if args.grad:
        w_all = np.concatenate(phis)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = ctx.energy_grad(u, w_all, mode="mixed", rtol=1e-10, inner_rtol=1e-3, raise_on_error=False)
        torch.cuda.synchronize()
        grad = {"seconds": time.perf_counter() - t0, "adjoint": g["report"],
                "w": "phi of the noise PSD (J = sum_i phi_i U_i)", "mode": "mixed adjoint solve to rtol 1e-10"}

    # ---- end to end through the C ABI with host buffers
    u_host = torch.empty(ndof, dtype=torch.float64, pin_memory=True)
    h2d = 0
    for d in descs:
        Nd = d["degree"] + 1
        h2d += (W.n_columns(d) * (7 * Nd * Nd * 8 + 8 * 4) + (len(d["slab_z"]) - 1) * (2 * Nd * 8 + 4)
                + len(d["materials"]) * 24)
    d2h = ndof * 8 + int(lofs[-1]) * 8
    e2e_times = [(float("nan"), 0)]
    for it in range(0 if args.no_e2e else 2):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if batched:
            ctx.build_batch(descs)
        else:
            ctx.build_mesh(desc)
            ctx.set_materials(desc["materials"])
            ctx.set_beam(desc["beam"]["r0"], desc["beam"]["F0"])
        _, rep_e = ctx.solve(mode="mixed", rtol=args.rtol, inner_rtol=args.inner_rtol, out=u,
                             energy_rtol=args.energy_rtol, precond=args.precond, raise_on_error=False,
                             inner_max=args.inner_max, fcg_window=args.fcg_window)
        u_host.copy_(u, non_blocking=True)
        U_e = ctx.layer_energies(u)
        for i, d in enumerate(descs):
            thermonoise.noise_psd(U_e[lofs[i]:lofs[i + 1]], phis[i], KB_T, FREQ, d["beam"]["F0"])
        torch.cuda.synchronize()
        e2e_times.append((time.perf_counter() - t0, rep_e["applies_f32"] + rep_e["applies_f64"]))
    e2e_value = e2e_times[-1][1] * ndof / e2e_times[-1][0] / 1e9 if not args.no_e2e else None

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu and world == 1:
        rate, sdof, napp, dt, t_asm = oracle_spmv_rate(reduced_desc(desc), budget_s=args.cpu_budget_s)
        t_direct = oracle_direct_solve_s()
        cpu = {"value": rate, "unit": "GDOF/s", "cores": 1, "kind": "oracle",
               "sample": f"FP64 oracle's assembled CSR matrix times a field (scipy SpMV, one thread): "
                         f"{napp} applies of {sdof} DOF (this workload at k = 1 with one substrate slab; "
                         f"assembly {t_asm:.0f} s, untimed) in {dt:.1f} s",
               "direct_solve_plain_box_s": t_direct, "direct_solve_cores": blas_threads(),
               "direct_solve": "dense Cholesky of the 12 288-DOF plain box (LAPACK on the BLAS threads)"}
    clocks = clk.summary()
    hbm_peak = peaks.get("hbm_gbs") or 6800.0
    peak_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks.get("hbm_gbs") else "fallback 6.8 TB/s"
    if pc == "zgroup":
        zkernel = (f"zgroup_packed_kernel<{'N' if batched else N},float>"
                   + (", one launch per degree" if batched else ""))
    else:
        zkernel = ("zline_solve_batch_kernel<N,float,float,0>" if batched
                   else f"zline_solve_kernel<{N},float,float,0>")
    line = {
        "metric": "GDOF/s of DG elasticity apply", "value": value, "unit": "GDOF/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": bench_config(args, descs, world),
        "time_to_U_s": {"mixed": mixed_s, "fp64": t_fp64,
                        "mixed_energy_rel_err": err_mixed,
                        "fp64_energy_rel_err": err64 if t_fp64 is not None else None},
        "solve": {"inner_iters": reps[-1]["inner_iters"], "outer_iters": reps[-1]["outer_iters"],
                  "applies_f32": reps[-1]["applies_f32"], "applies_f64": reps[-1]["applies_f64"],
                  "rel_residual": reps[-1]["rel_residual"], "status": reps[-1]["status"],
                  "fp64_iters": rep_fp64["inner_iters"] if rep_fp64 else None,
                  "fp64_status": rep_fp64["status"] if rep_fp64 else None,
                  "reference_pair": ref_pair},
        "apply_kernel": {"f32_us": t32 * 1e6, "f64_us": t64 * 1e6,
                         "f32_gdofs": ndof / t32 / 1e9, "f64_gdofs": ndof / t64 / 1e9,
                         "autotune": {f"p{p}": v for p, v in tuning.items()}},
        "roofline": {"bound": "hbm", "achieved": zbytes / tz / 1e9, "peak": hbm_peak, "unit": "GB/s",
                     "frac": zbytes / tz / 1e9 / hbm_peak,
                     "traffic": ZLINE_TRAFFIC.get((args.workload, zkernel)),
                     "kernel": zkernel, "us": tz * 1e6, "us_eager": tz_eager * 1e6, "timing": tz_how,
                     "algorithmic_bytes": zbytes, "bytes": "compact FP32 factors (S_s^-1 packed, O_s factors) once + r in + z out",
                     "peak_source": peak_src},
        "roofline_apply": {"bound": "alu", "achieved": achieved, "peak": peak_fp32, "unit": "TFLOP/s",
                           "frac": achieved / peak_fp32,
                           "traffic": None if batched else APPLY_TRAFFIC.get((args.workload, akernel)),
                           "kernel": akernel,
                           "flops_per_dof": flops_dof,
                           "hbm_GBps_algorithmic": 8 * ndof / t32 / 1e9,
                           "hbm_frac_algorithmic": 8 * ndof / t32 / 1e9 / hbm_peak,
                           "peak_source": "measured: tn_fma_peak FP32 (FMA chains, CUDA events)"},
        "roofline_apply_f64": {"bound": "alu", "achieved": flops / t64 / 1e12, "peak": peak_fp64,
                               "unit": "TFLOP/s", "frac": flops / t64 / 1e12 / peak_fp64,
                               "kernel": f"apply2_kernel<{N},double,0>" if not batched else "apply2_batch_kernel<N,double,0>",
                               "peak_source": "measured: tn_fma_peak FP64 (FMA chains, CUDA events)"},
        "gradient": grad,
        "e2e": {"value": e2e_value, "unit": "GDOF/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "seconds": e2e_times[-1][0]},
        "gpu_launches": launches,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
