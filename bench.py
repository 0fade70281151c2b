#!/usr/bin/env python3
"""Benchmark: GB300 MGRIT on the PWM-driven annular machine.

Default workload (cfg1; one "step" of this benchmark = one complete MGRIT solve
to tolerance): fine mesh the 24 x 48 annulus refined twice (18,240 interior
DOFs), linear materials, three-phase triangle-carrier PWM at 20 kHz,
J0 = 1e6 A/m^2, T = 20 ms, N = 4096 backward-Euler steps; 3-level MGRIT, m = 16,
FCF relaxation, coarse time levels on the 1,104-DOF base mesh (direct spatial
coarsening), FP64 arithmetic form.  The MGRIT tolerance is chosen so that the
maximal relative L2 error per time point against GPU sequential stepping is
<= 1e-6; the error reached is reported.

--workload picks another of the synthetic workloads (one JSON line each, same
keys): cfg0 (1,104 DOFs, N = 256, 2-level F-relaxation), cfg2 (73,344 DOFs,
N = 16,384; the FP32+FP64-refinement form timed beside the FP64 form), cfg3
(18,240 DOFs with the Brauer law, J0 = 3e6, N = 8,192, Newton steps).

value = fine time steps resolved per second of MGRIT wall time (N / t_MGRIT),
summed over ranks (independent replicas, one per GPU).  Also reported: GPU
sequential stepping wall time on the same GB300 and the speedup, the live
roofline of the dominant kernel (the level-0 batched step solve), end-to-end
throughput through the host-buffer entry point, sampled clocks, the error
against the CPU oracle on the leading time points, and the CPU oracle's
sequential stepping on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload cfg0|cfg1|cfg2|cfg3]
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MGRIT wall time vs GPU sequential stepping at <=1e-6 rel err; SpMM/CG HBM GB/s"
UNIT = "time-steps/s"
WORKLOAD = "cfg1: 18,240-DOF annulus, N=4096, T=20 ms, 3-level MGRIT m=16 FCF, coarse levels on 1,104 DOFs"
N_STEPS, T_END, F_CARRIER = 4096, 20e-3, 20e3
# the workloads --workload selects: (synth.workloads name, description, leading time
# points the CPU oracle computes for the error check)
BENCH_WORKLOADS = {
    "cfg0": ("cfg0_linear_l0_N256",
             "cfg0: 1,104-DOF annulus, N=256, T=5 ms, 5 kHz PWM, 2-level MGRIT m=16 F-relaxation", 256),
    "cfg1": ("cfg1_linear_l2_N4096", WORKLOAD, 4096),
    "cfg2": ("cfg2_mixed_l3_N16384",
             "cfg2: 73,344-DOF annulus, N=16384, T=20 ms, 3-level MGRIT m=16 FCF, delayed spatial coarsening "
             "(level 1 on 73,344 DOFs, coarsest on 18,240), FP32+FP64-refinement form (FP64 form timed beside it)",
             256),
    "cfg3": ("cfg3_nonlinear_l2_N8192",
             "cfg3: 18,240-DOF annulus, Brauer law, J0=3e6, N=8192, T=20 ms, 3-level MGRIT m=16 FCF, "
             "coarse levels on 1,104 DOFs, Newton to 1e-8", 0),
}
# cfg3: sequential Newton stepping is timed on this many leading steps and its
# time extrapolated to N (a full run takes about half an hour); they are also the
# error reference.  The MGRIT tolerance is fixed (a calibration ladder of full
# nonlinear solves would take too long) and nested iterations give the first guess.
NONLINEAR_SEQ_PREFIX = 128
NONLINEAR_TOL = 1e-7
ERR_TARGET = 1e-6   # metric: maximal relative L2 error per time point vs sequential stepping
ERR_MARGIN = 0.5    # calibrate to half the target
TOL_LADDER = (1e-3, 3e-4, 1e-4, 3e-5, 1e-5, 3e-6, 1e-6, 3e-7, 1e-7, 1e-8)
# MGRIT solves the steps of iteration k to max(1e-13, STEP_TOL_RATIO x relative residual)
STEP_TOL_RATIO = 3e-4
# step-solve tolerances tried for the sequential baseline, loosest first
SEQ_TOL_LADDER = (1e-6, 1e-7, 1e-8, 1e-9, 1e-10, 1e-11, 1e-13)
# smoothing of the sequential baseline's single-column steps: 4 Chebyshev sweeps on
# [lam/20, lam] measured 3 % faster there than the library default (5 on [lam/30, lam])
SEQ_SMOOTHING = dict(smooth=4, cheb_ratio=20.0)
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "graph_step_l2x256_fp64.md")


# the sources of the batched-step graph (its kernels, their device helpers and the
# shared definitions): the roofline launch's DRAM counters are valid only for them
STEP_SOURCES = ("batch.cu", "internal.h", "vec.cuh")


def csrc_sha1() -> str:
    """Hash of the batched step's sources: DRAM counters are valid only for the kernels they measured."""
    import hashlib

    h = hashlib.sha1()
    d = os.path.join(ROOT, "paper_1912_03106_gb300", "csrc")
    for f in STEP_SOURCES:
        h.update(f.encode())
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()


def last_traffic_capture():
    """The committed ncu summary's DRAM bytes per batched-step launch and the hash of
    the sources it was taken on, or None if the summary is missing."""
    try:
        fields = {}
        for line in open(TRAFFIC_FILE):
            if ":" in line and line.strip().startswith(("csrc_sha1", "traffic_bytes_per_launch")):
                k, v = line.strip().split(":", 1)
                fields.setdefault(k.strip(), v.strip())
        return {"bytes_per_launch": float(fields["traffic_bytes_per_launch"]), "csrc_sha1": fields["csrc_sha1"]}
    except (OSError, KeyError, ValueError):
        return None


def measured_traffic():
    """DRAM bytes per batched-step launch from the committed ncu summary, or None if
    the summary is missing or was taken on other sources."""
    cap = last_traffic_capture()
    return cap["bytes_per_launch"] if cap and cap["csrc_sha1"] == csrc_sha1() else None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=96, help="oracle steps timed for the CPU baseline")
    ap.add_argument("--profile-step", type=int, default=0, metavar="K",
                    help="only run batched steps of K columns on the 18,240-DOF mesh (for profilers)")
    ap.add_argument("--precision", type=int, default=0, help="with --profile-step: 0 FP64, 1 FP32+refinement")
    ap.add_argument("--path", type=int, default=0, help="with --profile-step: 0 auto, 1 cluster, 2 graph")
    ap.add_argument("--reps", type=int, default=2, help="with --profile-step: number of steps")
    ap.add_argument("--level", type=int, default=2, help="with --profile-step: mesh level 0..3 (18,240 DOFs = 2)")
    ap.add_argument("--halo-fusion", type=int, default=0,
                    help="with --profile-step: halo-fused multigrid kernels (0 library choice, 1 off, 2 on, "
                         "3 on with the sweeps' input staged in shared memory)")
    ap.add_argument("--base-cores", type=int, default=0,
                    help="with --profile-step: dense base solve on CUDA (1) or tensor (2) cores, 0 library choice")
    ap.add_argument("--tol", type=float, default=0.0,
                    help="with --profile-step: step tolerance (cg_tol and refine_tol; 0: library default)")
    ap.add_argument("--no-autotune", action="store_true", help="use the library's default launch shapes")
    ap.add_argument("--instances", type=int, default=0, metavar="M",
                    help="only the batching workload: M uneven instances, concurrent vs one by one")
    ap.add_argument("--workload", default="cfg1", choices=sorted(BENCH_WORKLOADS),
                    help="synthetic workload (default cfg1, the headline)")
    ap.add_argument("--oracle-points", type=int, default=-1,
                    help="leading time points checked against the CPU oracle (-1: the workload's default)")
    ap.add_argument("--no-sc", action="store_true",
                    help="every MGRIT level on the fine mesh (no spatial coarsening)")
    ap.add_argument("--no-e2e", action="store_true",
                    help="skip the end-to-end solves through host buffers (each nonlinear solve takes minutes)")
    return ap.parse_args()


def step_inputs(ctx, ids, k, level=2):
    """Seeded start states for batched steps of k columns on a mesh level (the
    18,240-DOF level 2 by default): the launch the roofline times and the one the
    DRAM counters were taken on."""
    import torch

    n = ctx.mg_num_dofs(ids[level])
    gen = torch.Generator(device="cuda").manual_seed(0)
    x_in = 0.01 * torch.randn((n, k), dtype=torch.float64, device="cuda", generator=gen)
    return x_in, torch.zeros((n, k), dtype=torch.float64, device="cuda")


def profile_step(args):
    """Batched backward-Euler steps of K columns on one mesh level, nothing else: a
    short, fixed program for kernel profilers (one untimed step, then --reps steps
    timed with CUDA events).  Iteration limits count as success."""
    import torch

    import synth
    from synth.model import PwmSpec, machine_model
    from paper_1912_03106_gb300 import api

    ctx = api.Context(0)
    ids = api.setup_machine(ctx, synth.mesh_hierarchy(max(3, args.level + 1)),
                            machine_model(pwm=PwmSpec(J0=1e6, f_carrier=F_CARRIER)))
    k = args.profile_step
    x_in, out = step_inputs(ctx, ids, k, args.level)
    so = api.solver_opts(precision=args.precision, path=args.path, halo_fusion=args.halo_fusion,
                         base_cores=args.base_cores)
    if args.tol > 0.0:
        so.cg_tol = so.refine_tol = args.tol

    def step():
        return ctx.mg_step(ids[args.level], N_STEPS, T_END, x_in, out, i0=1, istride=1 if k > 1 else 0,
                           solver=so, allow=(-5,))[1]

    st = step()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(ctx.stream)
    iters = 0
    for _ in range(args.reps):
        st = step()
        iters += st["cg_iters"]
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.reps)
    it_col = iters / max(1, args.reps) / k
    ns = [ctx.mg_num_dofs(ids[lv]) for lv in range(args.level, -1, -1)]  # multigrid depths
    kb = 8 if args.precision == 0 else 4
    per_col = step_bytes_per_column_iteration(ns, nu=so.smooth, krylov_bytes=kb)
    alg = it_col * (k * per_col + matrix_bytes_per_iteration(ns, nu=so.smooth)) + k * ns[0] * 8 * 9
    survey = survey_bytes_per_unit(args.precision) * ns[0] * k * it_col
    print(json.dumps({"profile_step": k, "level": args.level, "dofs": ns[0], "precision": args.precision,
                      "tol": so.cg_tol if args.precision == 0 else so.refine_tol,
                      "ms": ms, "pcg_iters_per_column": it_col, "survey_bytes": survey,
                      "survey_gbs": survey / ms / 1e6, "all_pass_bytes": alg, "all_pass_gbs": alg / ms / 1e6}))


def instances_run(args):
    """The batching workload: M seeded uneven machine instances (meshes of 1,104 /
    4,512 / 18,240 / 73,344 DOFs, N of 1,024 / 4,096 / 16,384 steps over 20 ms,
    5/10/20 kHz carriers, J0 uniform in [0.5e6, 3e6] A/m^2, half of the
    1,104-DOF ones with the Brauer law), each a 3-level FCF MGRIT solve (m = 16
    on its own mesh, relative tolerance 1e-7 with inexact step solves; linear
    instances in the FP32+refinement form, Brauer-law instances with FP64 Newton
    steps).  All instances are solved by one mg_batch_solve under a work budget of
    the free device memory (their outputs, 101 GB for 64 instances, are allocated
    first); one by one, each alone with its work buffers freed afterwards, is timed
    on one instance of every (mesh, N, law) class and scaled by the class sizes.
    Aggregate step-solves per second of both; two small linear instances are
    compared with the CPU oracle's sequential stepping at every time point."""
    import collections

    import numpy as np
    import torch

    import synth
    from synth.model import PwmSpec, machine_model
    from synth.workloads import instances
    from oracle.problem import MachineProblem, rel_err_per_point
    from paper_1912_03106_gb300 import api

    meshes = synth.mesh_hierarchy(4)
    insts = instances(args.instances, seed=0, mesh_levels=(0, 1, 2, 3), Ns=(1024, 4096, 16384), T=20.0e-3,
                      nonlinear_fraction=0.5, nonlinear_levels=(0,))
    setups = []
    for inst in insts:
        model = machine_model(nonlinear=inst.nonlinear, pwm=PwmSpec(J0=inst.J0, f_carrier=inst.f_carrier))
        ctx = api.Context(0, stream=torch.cuda.Stream())
        ids = api.setup_machine(ctx, meshes[:inst.mesh_level + 1], model)
        lv = ids[inst.mesh_level]
        n = ctx.mg_num_dofs(lv)
        opts = api.mgrit_opts(levels=3, m=(16, 16), space_level=(lv, lv, lv), relax=1, tol=1e-7, max_iter=40,
                              step_tol_ratio=STEP_TOL_RATIO, nested=inst.nonlinear,
                              solver=api.solver_opts(precision=0 if inst.nonlinear else 1))
        setups.append((ctx, opts, torch.zeros(n, dtype=torch.float64, device="cuda"),
                       torch.zeros((inst.N + 1, n), dtype=torch.float64, device="cuda")))
    torch.cuda.synchronize()
    ctxs, a0s, outs, optss = [s_[0] for s_ in setups], [s_[2] for s_ in setups], [s_[3] for s_ in setups], \
        [s_[1] for s_ in setups]
    Ns, Ts = [i.N for i in insts], [i.T for i in insts]
    # warm-up: step operators and PWM tables (one relaxation each; work buffers freed)
    warm = []
    for o in optss:
        w_ = api.L.mg_opts.from_buffer_copy(o)
        w_.max_iter = 0
        warm.append(w_)
    api.mg_batch_solve(ctxs, Ns, Ts, a0s, outs, warm, work_budget=-1)
    free_gb = torch.cuda.mem_get_info()[0] / 1e9
    t0 = time.perf_counter()
    rc, status, stats = api.mg_batch_solve(ctxs, Ns, Ts, a0s, outs, optss, work_budget=-1)
    t_conc = time.perf_counter() - t0
    solves = sum(s_["step_solves"] for s_ in stats)
    print(json.dumps({"phase": "concurrent", "status": rc, "statuses": sorted(set(status)), "step_solves": solves,
                      "concurrent_s": t_conc, "concurrent_step_solves_per_s": solves / t_conc,
                      "iters": [s_["iters"] for s_ in stats]}), file=sys.stderr, flush=True)
    # oracle: two small linear instances at every time point
    checks = []
    for idx in [i for i, inst in enumerate(insts) if not inst.nonlinear and inst.mesh_level <= 1 and
                inst.N == 1024][:2]:
        inst = insts[idx]
        model = machine_model(pwm=PwmSpec(J0=inst.J0, f_carrier=inst.f_carrier))
        ref = MachineProblem(meshes[:inst.mesh_level + 1], model, inst.N, inst.T, (inst.mesh_level,), ()).sequential()
        checks.append({"instance": idx, "dofs": int(a0s[idx].numel()), "N": inst.N,
                       "max_rel_err": float(rel_err_per_point(outs[idx].cpu().numpy(), ref).max())})
    # one by one: one instance per class, alone, scaled by the class sizes
    classes = collections.OrderedDict()
    for i, inst in enumerate(insts):
        classes.setdefault((int(a0s[i].numel()), inst.N, inst.nonlinear), []).append(i)
    t_seq, per_class = 0.0, []
    for (n, N_, nl), members in classes.items():
        i = members[0]
        ctx = ctxs[i]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r, st = ctx.mg_solve(Ns[i], Ts[i], a0s[i], outs[i], optss[i], allow=(-7, -10))
        torch.cuda.synchronize()
        dt_ = time.perf_counter() - t0
        ctx.mg_release_work()
        t_seq += dt_ * len(members)
        per_class.append({"dofs": n, "N": N_, "nonlinear": nl, "count": len(members), "alone_s": round(dt_, 3),
                          "step_solves": st["step_solves"], "status": r})
        print(json.dumps({"phase": "alone", **per_class[-1]}), file=sys.stderr, flush=True)
    print(json.dumps({"instances": len(insts), "status": rc, "statuses": sorted(set(status)),
                      "work_budget_gb": round(0.95 * free_gb, 1), "outputs_gb": round(
                          sum(o.numel() for o in outs) * 8 / 1e9, 1),
                      "step_solves": solves, "concurrent_s": t_conc, "one_by_one_s": t_seq,
                      "one_by_one": "each class timed alone once, scaled by its size", "classes": per_class,
                      "concurrent_step_solves_per_s": solves / t_conc, "one_by_one_step_solves_per_s": solves / t_seq,
                      "speedup": t_seq / t_conc, "iters": [s_["iters"] for s_ in stats], "oracle_check": checks}))
    for s_ in setups:
        s_[0].close()


def workload_config(dofs, world, key="cfg1"):
    """The workload keys both arms report (the MGRIT arm adds its solver settings).
    dofs: interior DOFs of each mesh level."""
    from synth.workloads import workload

    w = workload(BENCH_WORKLOADS[key][0])
    n_fine = dofs[w.fine_level]
    traj_mb = (w.N + 1) * n_fine * 8 / 1e6
    return {"workload": BENCH_WORKLOADS[key][1], "dofs": n_fine, "N": w.N, "T_s": w.T, "levels": w.levels,
            "m": list(w.m), "relax": "FCF" if w.relax else "F",
            "space_levels": [dofs[s_] for s_ in w.space_levels],
            "error_target": ERR_TARGET,
            "l2_flush": ("inputs larger than L2 (%.0f MB trajectory per solve)" % traj_mb) if traj_mb > 129 else
                        ("trajectory of %.1f MB fits the 129 MB L2: each solve timed alone after a 256 MB write "
                         "that flushes L2" % traj_mb),
            "parallelism": f"replicas x{world}"}


def max_over_ranks(t, world, device):
    """The slowest rank's time: the whole job ends with it (t itself on one rank)."""
    if world <= 1:
        return t
    import torch
    import torch.distributed as td

    tt = torch.tensor([t], dtype=torch.float64, device=device)
    td.all_reduce(tt, op=td.ReduceOp.MAX)
    return float(tt)


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- algorithmic bytes
def step_bytes_per_column_iteration(ns, W=7, nu=5, base_tile=16, krylov_bytes=8):
    """Algorithmic bytes one column moves per PCG iteration of the batched step kernel.

    ns: rows per multigrid depth (finest first).  Each vector pass of the V-cycle
    with one smoothing sweep per launch counts once (two sweeps per launch move
    fewer: their intermediate residual stays on the SM; a gathered vector counts as
    one read), the ELL matrix (4-byte column index +
    4-byte value per entry, 8-byte values for the FP64 operator) once per phase
    for the whole launch, not per column, so it is added by the caller.
    """
    n0 = ns[0]
    kb = krylov_bytes
    b = 0.0
    b += n0 * (4 + 4 * kb)  # A: z read, p, q read and written
    b += n0 * 6 * kb  # B: x, p, r, q read; x, r written
    nd = len(ns)
    for d in range(nd - 1):
        n, nc = ns[d], ns[d + 1]
        rb = kb if d == 0 else 4
        b += n * (rb + 8)  # first smoothing sweep: r read, x and s written
        b += (nu - 1) * n * 16  # further sweeps: s, x read; x, s written
        b += n * 4 + nc * 4  # restriction: s read, coarse r written
        b += n * 12 + nc * 4  # prolongation: coarse x read, x read/written, y written
        b += n * 12  # residual update: y read, s read/written
        b += (nu - 1) * n * 16 + n * 12 + (n0 * kb if d == 0 else 0)  # post sweeps (+ r for (r, z))
    nb = ns[-1]
    b += nb * 8 + nb * nb * 4 / base_tile  # coarsest: r read, x written, dense inverse per tile
    return b


def matrix_bytes_per_iteration(ns, W=7, nu=5):
    b = ns[0] * W * 12  # FP64 operator in phase A
    for d in range(len(ns) - 1):
        b += ns[d] * W * 8 * (nu + 1 + nu - 1)  # smoothing sweeps + residual update (FP32)
    return b


# ---------------------------------------------------------------- our arm
def survey_bytes_per_unit(precision):
    """Algorithmic bytes of one unknown x column x PCG iteration in the survey's
    unit (fused PCG iteration: ~9 vector passes of 8 B, plus the ELL matrix over a
    32-column tile): 76 B in the FP64 form, 38 B with FP32 Krylov vectors."""
    return 76.0 if precision == 0 else 38.0


def workload_setup(key, local):
    """Context, mesh ids and MGRIT options of a bench workload (synth.workloads)."""
    import torch

    import synth
    from synth.model import PwmSpec, machine_model
    from synth.workloads import workload
    from paper_1912_03106_gb300 import api

    w = workload(BENCH_WORKLOADS[key][0])
    meshes = synth.mesh_hierarchy(w.fine_level + 1)
    model = machine_model(nonlinear=w.nonlinear, pwm=PwmSpec(J0=w.J0, f_carrier=w.f_carrier))
    stream = torch.cuda.current_stream(local)
    ctx = api.Context(local, stream)
    ids = api.setup_machine(ctx, meshes, model)
    return w, meshes, model, ctx, ids, stream


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    from paper_1912_03106_gb300 import api

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as td

        td.init_process_group("nccl", device_id=dev)
    key = args.workload
    w, meshes, model, ctx, ids, stream = workload_setup(key, local)
    fine = ids[w.fine_level]
    n = ctx.mg_num_dofs(fine)
    N, T = w.N, w.T
    space = tuple(ids[w.fine_level if args.no_sc else s_] for s_ in w.space_levels)

    def make_opts(tol, precision=w.precision, ratio=STEP_TOL_RATIO):
        return api.mgrit_opts(levels=w.levels, m=w.m, space_level=space, relax=w.relax, tol=tol, max_iter=60,
                              step_tol_ratio=ratio, solver=api.solver_opts(precision=precision),
                              nested=w.nonlinear)

    a0 = torch.zeros(n, dtype=torch.float64, device=dev)
    out = torch.empty((N + 1, n), dtype=torch.float64, device=dev)

    # launch shapes: the library's autotuner, once per (mesh, columns) the solve and
    # the sequential baseline use (linear meshes only)
    tuned = {}
    if not args.no_autotune and not w.nonlinear:
        shapes, stride = [(w.fine_level, 1)], 1
        for l, m_l in enumerate(w.m):
            shapes.append((w.space_levels[l], N // stride // m_l))
            stride *= m_l
        shapes.append((w.space_levels[-1], 1))
        for lvl, kk in dict.fromkeys(shapes):
            so, ms = ctx.mg_autotune(ids[lvl], N, T, kk)
            tuned["%d_DOFs_x%d" % (ctx.mg_num_dofs(ids[lvl]), kk)] = {
                "path": "graph" if so.path == 2 else "cluster", "tile": so.tile, "cluster": so.cluster,
                "rows_per_block": so.rows_per_block, "coarse_rows_per_block": so.coarse_rows_per_block,
                "base_tiles": so.base_tiles, "halo_fusion": so.halo_fusion, "base_cores": so.base_cores,
                "ms": round(ms, 4)}

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as td

            td.barrier()

    # error reference: sequential stepping with every step solved to 1e-13 (linear);
    # nonlinear: sequential Newton stepping on the leading NONLINEAR_SEQ_PREFIX steps
    # (also the timed sequential sample)
    if w.nonlinear:
        Kp = NONLINEAR_SEQ_PREFIX
        ref = torch.empty((Kp + 1, n), dtype=torch.float64, device=dev)
        ctx.mg_sequential(fine, 8, T * 8 / N, a0, ref[:9])  # warm-up: plans
        torch.cuda.synchronize()
        e0_, e1_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0_.record(stream)
        _, seq_st = ctx.mg_sequential(fine, Kp, T * Kp / N, a0, ref)
        e1_.record(stream)
        torch.cuda.synchronize()
        seq_prefix_s = e0_.elapsed_time(e1_) / 1e3
        ref_note = "GPU sequential Newton stepping (Newton to 1e-8) on the first %d steps" % Kp
    else:
        ref = torch.empty((N + 1, n), dtype=torch.float64, device=dev)
        ref_note = "GPU sequential stepping, every step solved to 1e-13"
        ctx.mg_sequential(fine, N, T, a0, ref)

    def max_rel_err(b):
        hi = ref.shape[0]  # the whole trajectory, or the reference's leading steps
        diff = torch.linalg.vector_norm(b[1:hi] - ref[1:hi], dim=1) / torch.linalg.vector_norm(ref[1:hi], dim=1)
        return float(diff.max())

    # warm-up doubles as calibration: the loosest relative residual tolerance of the
    # ladder whose solution is within ERR_MARGIN * ERR_TARGET of the reference
    def calibrate(precision):
        tol = TOL_LADDER[-1]
        calib = []
        for t_try in TOL_LADDER:
            ctx.mg_solve(N, T, a0, out, make_opts(t_try, precision), allow=(-7, -10))
            e = max_rel_err(out)
            calib.append((t_try, e))
            if e <= ERR_MARGIN * ERR_TARGET:
                tol = t_try
                break
        return tol, calib

    if w.nonlinear:
        tol, calib = NONLINEAR_TOL, []
    else:
        tol, calib = calibrate(w.precision)
    opts = make_opts(tol)
    for _ in range(args.warmup):
        ctx.mg_solve(N, T, a0, out, opts)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    stats = []
    # a trajectory that fits the 129 MB L2 would be timed warm: then each solve is
    # timed on its own, after a write of 256 MB that flushes the L2
    flush = torch.empty(32 << 20, dtype=torch.float64, device=dev) if (N + 1) * n * 8 <= 129e6 else None
    with ClockSampler(local) as clocks:
        barrier()
        t0 = time.perf_counter()
        if flush is None:
            e0.record(stream)
            for _ in range(args.steps):
                _, st = ctx.mg_solve(N, T, a0, out, opts)
                stats.append(st)
            e1.record(stream)
            barrier()
            dev_s = e0.elapsed_time(e1) / 1e3
        else:
            dev_s = 0.0
            for _ in range(args.steps):
                flush.fill_(1.0)
                e0.record(stream)
                _, st = ctx.mg_solve(N, T, a0, out, opts)
                e1.record(stream)
                torch.cuda.synchronize()
                dev_s += e0.elapsed_time(e1) / 1e3
                stats.append(st)
            barrier()
        wall = time.perf_counter() - t0
    t_step = dev_s / args.steps
    mgrit_out = out.clone()  # the last timed solve
    t_step = max_over_ranks(t_step, world, dev)
    value = world * N / t_step

    # the other arithmetic form, calibrated and timed the same way (FP32+refinement
    # workloads: the FP64 form beside it)
    alt = None
    if w.precision == 1:
        tol_a, calib_a = calibrate(0)
        opts_a = make_opts(tol_a, 0)
        ctx.mg_solve(N, T, a0, out, opts_a)
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            _, st_a = ctx.mg_solve(N, T, a0, out, opts_a)
        e1.record(stream)
        barrier()
        ta = e0.elapsed_time(e1) / 1e3 / args.steps
        alt = {"form": "fp64", "wall_s": ta, "time_steps_per_s": N / ta, "mgrit_tol_rel": tol_a,
               "iters": st_a["iters"], "pcg_iters": st_a["cg_iters"], "tolerance_calibration": calib_a,
               "max_rel_err_vs_reference": max_rel_err(out), "step_solves_per_s": st_a["step_solves"] / ta}

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e:
        a0_h = torch.zeros(n, dtype=torch.float64).pin_memory()
        out_h = torch.empty((N + 1, n), dtype=torch.float64).pin_memory()
        a0_np, out_np = a0_h.numpy(), out_h.numpy()
        if not w.nonlinear:  # warm (a nonlinear solve takes minutes; its plans exist already)
            ctx.mg_solve_host(N, T, a0_np, out_np, opts)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.mg_solve_host(N, T, a0_np, out_np, opts)
        barrier()
        e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, world, dev)
        e2e = {"value": world * N / e2e_s, "unit": UNIT, "h2d_bytes_per_step": n * 8,
               "d2h_bytes_per_step": (N + 1) * n * 8,
               "max_rel_err_vs_reference": max_rel_err(torch.as_tensor(out_np).to(dev))}
        del out_h

    roof = roofline(ctx, ids, w, stream)

    # GPU sequential stepping, the baseline: its steps solved to the loosest tolerance
    # of a ladder that keeps the trajectory within ERR_MARGIN * ERR_TARGET of the
    # reference (the calibration runs warm it up), then timed once; nonlinear: the
    # default Newton tolerance, timed on the leading steps and extrapolated to N
    if w.nonlinear:
        Kp = NONLINEAR_SEQ_PREFIX
        seq_s = seq_prefix_s * N / Kp
        seq_tol, seq_calib = None, []
        seq_err = 0.0  # it is the reference
        seq_note = "timed on the first %d steps, extrapolated to N = %d" % (Kp, N)
    else:
        seq = torch.empty((N + 1, n), dtype=torch.float64, device=dev)
        seq_tol = SEQ_TOL_LADDER[-1]
        seq_calib = []
        for c_try in SEQ_TOL_LADDER:
            ctx.mg_sequential(fine, N, T, a0, seq, solver=api.solver_opts(cg_tol=c_try, **SEQ_SMOOTHING))
            e = max_rel_err(seq)
            seq_calib.append((c_try, e))
            if e <= ERR_MARGIN * ERR_TARGET:
                seq_tol = c_try
                break
        seq_so = api.solver_opts(cg_tol=seq_tol, **SEQ_SMOOTHING)
        barrier()
        e0.record(stream)
        _, seq_st = ctx.mg_sequential(fine, N, T, a0, seq, solver=seq_so)
        e1.record(stream)
        torch.cuda.synchronize()
        seq_s = e0.elapsed_time(e1) / 1e3
        seq_err = max_rel_err(seq)
        seq_note = "full run"
        del seq

    max_err = max_rel_err(mgrit_out)
    oracle = oracle_check(args, key, w, meshes, model, mgrit_out, ref) if rank == 0 else None

    st = stats[-1]
    dso = api.solver_opts()
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": t_step * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if w.precision == 0 else "f32+f64",
        "data": "synthetic",
        "config": dict(workload_config([ctx.mg_num_dofs(i) for i in ids], world, key), mgrit_tol_rel=tol,
                       precond="multigrid V(%d,%d), Chebyshev smoothing on [lam/%g, lam], FP32, dense base inverse"
                               % (dso.smooth, dso.smooth, dso.cheb_ratio)),
        "mgrit": {"form": "fp64" if w.precision == 0 else "fp32+fp64-refinement", "wall_s": t_step,
                  "iters": st["iters"], "res_hist": st["res_hist"], "step_tol_ratio": STEP_TOL_RATIO,
                  "tolerance_calibration": calib, "max_rel_err_vs_reference": max_err,
                  "step_solves": st["step_solves"], "batched_steps": st["batched_steps"], "pcg_iters": st["cg_iters"],
                  "newton_iters": st["newton_iters"], "step_solves_per_s": st["step_solves"] / t_step},
        "gpu_sequential": {"wall_s": seq_s, "time_steps_per_s": N / seq_s, "pcg_iters": seq_st["cg_iters"],
                           "newton_iters": seq_st["newton_iters"], "step_cg_tol": seq_tol,
                           "smoothing": SEQ_SMOOTHING, "tolerance_calibration": seq_calib,
                           "max_rel_err_vs_reference": seq_err, "timing": seq_note},
        "speedup_vs_gpu_sequential": seq_s / t_step,
        "error_reference": ref_note,
        "spatial_coarsening": not args.no_sc,
        "oracle_check": oracle,
        "e2e": e2e,
        "roofline": roof,
        "clocks": clocks.summary(),
        "gpu_launches": int(sum(s_["launches"] for s_ in stats)),
        "autotune": tuned,
        "wall_check_s": wall,
    }
    if alt is not None:
        line["mgrit_fp64"] = alt
    if rank == 0:
        if world == 1:
            line["cpu_baseline"] = cpu_baseline(args, key)
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        import torch.distributed as td

        td.destroy_process_group()


def oracle_check(args, key, w, meshes, model, got, ref):
    """The CPU oracle's sequential stepping (banded Cholesky, FP64) on the leading
    time points; the maximal relative error per time point of the timed MGRIT
    solve and of the GPU reference against it."""
    import numpy as np

    K = BENCH_WORKLOADS[key][2] if args.oracle_points < 0 else args.oracle_points
    K = min(K, w.N)
    if K <= 0 or w.nonlinear:
        return None
    from oracle.problem import MachineProblem, rel_err_per_point

    t0 = time.perf_counter()
    P = MachineProblem(meshes, model, w.N, w.T, (w.fine_level,), ())
    phi = P.levels[0].phi
    u = [np.zeros(P.n)]
    for i in range(1, K + 1):
        u.append(phi(u[-1], i))
    u = np.array(u)
    g = got[:K + 1].cpu().numpy()
    r = ref[:K + 1].cpu().numpy()
    return {"points": K, "max_rel_err_mgrit": float(rel_err_per_point(g, u).max()),
            "max_rel_err_reference": float(rel_err_per_point(r, u).max()), "oracle_s": time.perf_counter() - t0}


def roofline(ctx, ids, w, stream):
    """Time the dominant launch (one batched step of the level-0 batch width on the
    fine mesh from the seeded start states of step_inputs, in the workload's
    arithmetic form, the library's own graph-path shape as in its DRAM capture)
    with CUDA events.  achieved: the survey's unit (76 B per unknown x column x PCG
    iteration in the FP64 form, 38 B with FP32 Krylov vectors) over the launch
    time; achieved_all_passes: every vector pass of the multigrid-preconditioned
    iteration, as bench's byte model counts it."""
    import torch

    from paper_1912_03106_gb300 import api

    if w.nonlinear:
        return {"bound": "hbm", "kernel": "batched Newton step", "achieved": None, "peak": None, "unit": "GB/s",
                "frac": None, "traffic": None,
                "note": "no byte model for the Newton step; the linear workloads carry the PCG roofline"}
    lvl = w.fine_level
    n = ctx.mg_num_dofs(ids[lvl])
    k = w.N // w.m[0]
    x_in, x_out = step_inputs(ctx, ids, k, lvl)
    so = api.solver_opts(path=2 if k >= 16 else 0, precision=w.precision)
    ctx.mg_step(ids[lvl], w.N, w.T, x_in, x_out, i0=1, istride=1, solver=so)
    reps = 5
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    iters = 0
    for _ in range(reps):
        _, st = ctx.mg_step(ids[lvl], w.N, w.T, x_in, x_out, i0=1, istride=1, solver=so)
        iters += st["cg_iters"]
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / reps
    it_per_col = iters / reps / k
    ns = [ctx.mg_num_dofs(ids[d]) for d in range(lvl, -1, -1)]
    kb = 8 if w.precision == 0 else 4
    per_col = step_bytes_per_column_iteration(ns, nu=so.smooth, krylov_bytes=kb)
    mat = matrix_bytes_per_iteration(ns, nu=so.smooth)
    bytes_all = it_per_col * (k * per_col + mat) + k * n * 8 * 9
    bytes_survey = survey_bytes_per_unit(w.precision) * n * k * it_per_col
    peak = None
    src = "fallback"
    try:
        peak = json.load(open(PEAKS_FILE))["hbm_gbs"]
        src = "measured"
    except (OSError, KeyError, ValueError):
        peak = 6800.0
    achieved = bytes_survey / t / 1e9
    achieved_all = bytes_all / t / 1e9
    resident = n * k * 8 < 129e6
    return {"bound": "hbm",
            "kernel": "batched step, %d DOFs x %d columns, %s form" % (
                n, k, "FP64" if w.precision == 0 else "FP32+refinement") + (
                " (one graph of per-phase kernels)" if k >= 16 else " (cluster-persistent kernel)"),
            "achieved": achieved, "peak": peak, "peak_source": src, "unit": "GB/s", "frac": achieved / peak,
            "achieved_all_passes": achieved_all, "frac_all_passes": achieved_all / peak,
            "traffic": measured_traffic() if (lvl == 2 and k == 256 and w.precision == 0) else None,
            "traffic_last_capture": (dict(last_traffic_capture() or {}, sources_now=csrc_sha1())
                                     if (lvl == 2 and k == 256 and w.precision == 0) else None),
            "launch_ms": t * 1e3, "pcg_iters_per_column": it_per_col,
            "algorithmic_bytes_per_launch": bytes_survey, "all_pass_bytes_per_launch": bytes_all,
            "l2_resident": resident}


ORACLE_THREADS = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}


def cpu_baseline(args, key="cfg1"):
    """The oracle's sequential stepping (banded Cholesky, FP64; Newton with banded
    Cholesky for the Brauer law) on a bounded sample of the workload, in a
    subprocess whose BLAS runs on one thread."""
    from synth.workloads import workload

    w = workload(BENCH_WORKLOADS[key][0])
    sample = min(w.N, 4 if w.nonlinear else args.cpu_sample)
    env = dict(os.environ, **ORACLE_THREADS)
    code = (
        "import sys, time, json; sys.path.insert(0, %r)\n"
        "import numpy as np, synth\n"
        "from synth.model import PwmSpec, machine_model\n"
        "from synth.workloads import workload\n"
        "from oracle.problem import MachineProblem\n"
        "w = workload(%r)\n"
        "ms = synth.mesh_hierarchy(w.fine_level + 1)\n"
        "model = machine_model(nonlinear=w.nonlinear, pwm=PwmSpec(J0=w.J0, f_carrier=w.f_carrier))\n"
        "P = MachineProblem(ms, model, w.N, w.T, (w.fine_level,), (), nonlinear=w.nonlinear)\n"
        "phi = P.levels[0].phi\n"
        "u = np.zeros(P.n); phi(u, 1); t = time.perf_counter()\n"
        "for i in range(1, %d + 1): u = phi(u, i)\n"
        "dt = time.perf_counter() - t\n"
        "print(json.dumps({'steps': %d, 'seconds': dt, 'n': int(P.n)}))\n"
    ) % (ROOT, w.name, sample, sample)
    try:
        r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
        res = json.loads(r.stdout.strip().splitlines()[-1])
        how = ("damped Newton, each correction by banded Cholesky" if w.nonlinear else
               "banded Cholesky factored once (factorisation not timed)")
        return {"value": res["steps"] / res["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"first {res['steps']} of {w.N} backward-Euler steps of the {res['n']:,}-DOF model, "
                          f"sequential, {how}; BLAS on one thread"}
    except Exception as e:  # pragma: no cover
        return {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}


# ---------------------------------------------------------------- reference arm (the oracle)
def run_reference(args, rank, world):
    """The oracle's sequential stepping timed on the host: the reference arm.  Its
    BLAS is pinned to one thread (set in main() before numpy loads)."""
    if rank != 0:
        return
    import numpy as np

    import synth
    from synth.model import PwmSpec, machine_model
    from synth.workloads import workload
    from oracle.problem import MachineProblem

    key = getattr(args, "workload", "cfg1")
    w = workload(BENCH_WORKLOADS[key][0])
    ms = synth.mesh_hierarchy(w.fine_level + 1)
    model = machine_model(nonlinear=w.nonlinear, pwm=PwmSpec(J0=w.J0, f_carrier=w.f_carrier))
    P = MachineProblem(ms, model, w.N, w.T, (w.fine_level,), (), nonlinear=w.nonlinear)
    phi = P.levels[0].phi
    sample = min(w.N, 2 if w.nonlinear else 32)

    def step():
        u = np.zeros(P.n)
        t = time.perf_counter()
        for i in range(1, sample + 1):
            u = phi(u, i)
        return time.perf_counter() - t

    for _ in range(args.warmup):
        step()
    times = [step() for _ in range(args.steps)]
    t_step = sum(times) / len(times)
    value = sample / t_step
    threads = os.environ.get("OPENBLAS_NUM_THREADS", "")
    cores = int(threads) if threads.isdigit() else (
        len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count())
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": workload_config([len(m_.interior_nodes()) for m_ in ms], world, key),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{sample} sequential backward-Euler steps of the {P.n:,}-DOF model per step, "
                                   f"BLAS on {cores} thread(s)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.instances:
        instances_run(args)
        return
    if args.profile_step:
        profile_step(args)
        return
    rank, world, local = dist_info()
    if args.impl == "reference":
        os.environ.update(ORACLE_THREADS)  # before numpy is first imported
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
