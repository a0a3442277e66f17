#!/usr/bin/env python
"""Benchmark of the GYM leapfrog on GB300: field DoF-updates/s.

Workload (default): PEC cube, N = 32 cubes per side split into Kuhn tets (196,608 tets), order
k = 2, per-tet permittivity i.i.d. U[1,4) (seed 2000), mu = 1, one Gaussian-modulated z-dipole
(centre frequency pi sqrt 5, width 20 steps) at a point U[0.2,0.8)^3 (seed 2001), dt = 0.5 tau_CFL,
2000 leapfrog steps per run, FP32 fields.  One benchmark step is one whole 2000-step run from the
zero state; value = (N1 + N2) * 2000 / run time, summed over ranks (independent replicas).

Batched mode (--rhs R, R a power of two): R independent excitations as R right-hand-side columns
of one context, one Gaussian-pulse dipole per column at U[0.2,0.8)^3 points (seed 3001) with
normalised-Gaussian orientations (seed 3002); value = (N1 + N2) * R * steps / run time.

Run:  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--rhs R]
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "field DoF-updates/s on 1 GB300 (FP32/batched vs FP64) at stated L2 error/energy drift"
UNIT = "DoF-updates/s"


def workload(n=32, k=2, leapfrog_steps=2000, rhs=1):
    if rhs == 1:
        x0 = synth.source_positions(2001, 1)
        d = np.array([[0.0, 0.0, 1.0]])
    else:
        x0 = synth.source_positions(3001, rhs)
        d = synth.unit_vectors(3002, rhs)
    return dict(n=n, k=k, eps=synth.tet_eps(2000, n, 1.0, 4.0), x0=x0[0], xs=x0, d=d[0], ds=d, rhs=rhs,
                omega=np.pi * np.sqrt(5.0), width=20.0, steps=leapfrog_steps)


def source_for(W, dt, column=None):
    """The workload's dipoles (one per column); column = r gives column r's dipole alone, on column 0."""
    sigma = W["width"] * dt
    cols = range(W["rhs"]) if column is None else [column]
    return [dict(x=W["xs"][r], d=W["ds"][r], amp=1.0, omega=W["omega"], t0=4 * sigma, sigma=sigma,
                 rhs=r if column is None else 0) for r in cols]


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one curl-rows Q1-apply launch of
# the default workload, from the ncu capture summarised in profiles/k_qapply_s_cavity_N32_k2_fp32.md.
# The kernel has changed since (the programmatic-dependent-launch prologue, no memory operation
# added), so the line reports traffic as null and this figure as the last capture, of the kernel
# without that prologue; set QAPPLY_TRAFFIC_CURRENT once a capture of the current kernel exists.
QAPPLY_TRAFFIC_BYTES = 834.205184e6 + 9.822208e6
QAPPLY_TRAFFIC_CURRENT = False


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
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
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            P = json.load(f)
        return float(P["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ CPU oracle timing
def oracle_model(n=5, k=2):
    """The FP64 CPU oracle's operators for a bounded sample of the workload: the same recipe
    (eps seed 2000, z-dipole seed 2001, dt = 0.5 tau_CFL) on an n^3 cube.  The set-up (SPAI) is
    not part of the timed leapfrog."""
    from oracle import spai as SP
    from oracle.fem import FEM
    from oracle.gym import GYM
    from oracle.mesh import KuhnMesh
    W = workload(n=n, k=k, leapfrog_steps=0)
    f = FEM(KuhnMesh(n, k), eps=W["eps"])
    M1 = f.M1()
    Q, _ = SP.gym_q1(f, M1)
    g = GYM(f.C(), f.M2(), Q, M1)
    return dict(f=f, g=g, dt=0.5 * g.tau_cfl(), W=W, n=n, k=k)


def _oracle_leapfrog(model, steps):
    """Time `steps` leapfrog steps of the oracle from rest with the workload's dipole; seconds."""
    from oracle.gym import DipoleSource
    f, g, W, dt = model["f"], model["g"], model["W"], model["dt"]
    src = [dict(x=W["x0"], d=W["d"], amp=1.0, omega=W["omega"], width_steps=W["width"])]
    J = DipoleSource(f, src, dt)
    e = np.zeros(f.mesh.N1)
    b = np.zeros(f.mesh.N2)
    t0 = time.perf_counter()
    g.run(e, b, dt, steps, source=J)
    return time.perf_counter() - t0


def _replica(args):
    path, steps = args
    import pickle
    with open(path, "rb") as fh:
        model = pickle.load(fh)
    return _oracle_leapfrog(model, steps)


def oracle_sample(model, steps, procs=1):
    """DoF-updates/s of the oracle as it stands: one process, or `procs` spawned replicas of the
    same sample running at once (the oracle itself is single-threaded).  Returns (rate, wall s)."""
    f = model["f"]
    units = (f.mesh.N1 + f.mesh.N2) * steps
    if procs == 1:
        el = _oracle_leapfrog(model, steps)
        return units / el, el
    import multiprocessing as mp
    import pickle
    import tempfile
    with tempfile.NamedTemporaryFile(suffix=".pkl", delete=False) as fh:
        pickle.dump(model, fh)
        path = fh.name
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            pool.map(_replica, [(path, 10)] * procs)          # import and unpickle in every worker
            t0 = time.perf_counter()
            pool.map(_replica, [(path, steps)] * procs)
            el = time.perf_counter() - t0
    finally:
        os.unlink(path)
    return procs * units / el, el


def cpu_baseline_line(args):
    """Single-thread and all-core rates of the oracle on the bounded sample, plus the first
    (FP64, N = 4, k = 1, 1000 steps) workload timed in full."""
    ncores = os.cpu_count() or 1
    model = oracle_model(n=args.cpu_n)
    v1, el1 = oracle_sample(model, args.cpu_steps)
    vN, elN = oracle_sample(model, args.cpu_steps, procs=ncores)
    f = model["f"]
    c1 = oracle_model(n=4, k=1)
    t_c1 = _oracle_leapfrog(c1, 1000)
    sample = (f"FP64 CPU oracle (scipy sparse), same recipe on a {args.cpu_n}^3 cube, k=2 "
              f"(N1={f.mesh.N1}, N2={f.mesh.N2}, Q1 nnz {model['g'].Q1.nnz}), {args.cpu_steps} leapfrog steps; "
              f"value = {ncores} concurrent single-threaded replicas on {ncores} host cores; the rate per DoF "
              f"of this sample stands in for the N=32 cavity (not measured at that size)")
    return dict(value=vN, unit=UNIT, cores=ncores, kind="oracle", sample=sample,
                single_thread=dict(value=v1, cores=1, seconds=el1), all_cores_seconds=elN,
                first_workload_in_full=dict(workload="N=4, k=1, FP64, 1000 steps", seconds=t_c1,
                                            value=(c1["f"].mesh.N1 + c1["f"].mesh.N2) * 1000 / t_c1))


def run_reference(args, rank, world):
    if rank != 0:
        return
    ncores = os.cpu_count() or 1
    model = oracle_model(n=args.cpu_n)
    vals = []
    for i in range(args.warmup + args.steps):
        v, el = oracle_sample(model, args.cpu_steps, procs=ncores)
        if i >= args.warmup:
            vals.append((v, el))
    value = float(np.mean([v for v, _ in vals]))
    ms = float(np.mean([el for _, el in vals]) * 1e3)
    f = model["f"]
    sample = (f"FP64 CPU oracle (scipy sparse), same recipe on a {args.cpu_n}^3 cube, k=2 "
              f"(N1={f.mesh.N1}, N2={f.mesh.N2}), {args.cpu_steps} leapfrog steps per step, "
              f"{ncores} concurrent single-threaded replicas on {ncores} host cores")
    line = dict(impl="reference", metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64", data="synthetic",
                config=dict(workload="PEC cube N=32, k=2, eps~U[1,4) seed 2000, z-dipole, 2000 steps "
                                     f"(oracle timed on a bounded N={args.cpu_n} sample)"),
                cpu_baseline=dict(value=value, unit=UNIT, cores=ncores, kind="oracle", sample=sample),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ replica aggregation
def aggregate(units_per_rank, seconds_local, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas: every rank did `units_per_rank`; the job
    time is the maximum over ranks.  Returns (value, job seconds)."""
    import torch
    t = float(seconds_local)
    world = 1
    if dist is not None and dist.is_available() and dist.is_initialized():
        world = dist.get_world_size()
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return world * units_per_rank / t, t


# ------------------------------------------------------------------ GPU arm
def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2301_01753_gb300 as Y
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    W = workload(n=args.n, k=args.order, leapfrog_steps=args.leapfrog_steps, rhs=args.rhs)
    R = args.rhs
    # a stream of our own: the context launches on it and the timing events are recorded on it
    stream = torch.cuda.Stream(device=local_rank)
    torch.cuda.set_stream(stream)
    prec = dict(fp32=Y.YGM_FP32, fp64=Y.YGM_FP64, tf32=Y.YGM_FP32_TC_TF32, tf32x3=Y.YGM_FP32_TC_3XTF32)[args.precision]
    tb = time.perf_counter()
    # the timed context also records the conserved energy every 100 steps (row A-5)
    ctx = Y.Context(W["n"], W["k"], eps=W["eps"], precision=prec, device=local_rank, stream=stream.cuda_stream,
                    energy_every=args.energy_every, n_rhs=R)
    setup_s = time.perf_counter() - tb
    dt = 0.5 * ctx.tau_cfl
    src = source_for(W, dt)
    tdt = torch.float64 if prec == Y.YGM_FP64 else torch.float32
    ze = torch.zeros(ctx.N1 * R, dtype=tdt, device="cuda")
    zb = torch.zeros(ctx.N2 * R, dtype=tdt, device="cuda")
    units = (ctx.N1 + ctx.N2) * R * W["steps"]

    def one_run():
        ctx.set_state(ze, zb)
        ctx.step(W["steps"], dt, src)

    for _ in range(args.warmup):
        one_run()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    l0 = ctx.launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            one_run()
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms_total = ev0.elapsed_time(ev1)
    launches = ctx.launch_count() - l0
    ms = ms_total / args.steps
    # per-kernel device times from one more run with CUDA events around every launch (kept out
    # of the timed region above: the event records would add to its time)
    ctx.kernel_timing(True)
    ctx.kernel_times()
    one_run()
    kt = ctx.kernel_times()
    ctx.kernel_timing(False)
    value, t_job = aggregate(units * args.steps, ms_total * 1e-3, dist, device="cuda")

    # end to end through the public API with host buffers (pinned): H2D state in, D2H state out
    he = torch.zeros(ctx.N1 * R, dtype=tdt).pin_memory().numpy()
    hb = torch.zeros(ctx.N2 * R, dtype=tdt).pin_memory().numpy()
    oe = torch.empty(ctx.N1 * R, dtype=tdt).pin_memory().numpy()
    ob = torch.empty(ctx.N2 * R, dtype=tdt).pin_memory().numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.set_state(he, hb)
        ctx.step(W["steps"], dt, src)
        ctx.get_state(synced=True, out_e=oe, out_b=ob)
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e_val, _ = aggregate(units, e2e_s, dist, device="cuda")
    rs = 8 if prec == Y.YGM_FP64 else 4

    # roofline of the dominant kernel (Q1 apply), from the instrumented run.  Algorithmic bytes of
    # one launch = the distinct Q1 values its rows use (a symmetric pair once) + e read + x
    # written.  Steps with an energy read-out compute every row; the others only the
    # curl-carrying rows (C x reads nothing else).
    qms, qn = kt["k_qapply"]
    n_all = kt["k_energy"][1]                  # one all-rows Q1 apply per energy read-out
    n_act = qn - n_all
    ra, ua, sa = ctx.qapply_counts(False)
    rf, uf, sf = ctx.qapply_counts(True)
    alg_total = rs * (n_act * (ua + R * (ctx.N1 + ra)) + n_all * (uf + R * (ctx.N1 + rf)))
    streamed_total = rs * (n_act * (sa + R * (ctx.N1 + ra)) + n_all * (sf + R * (ctx.N1 + rf)))
    alg_bytes = alg_total / max(qn, 1)
    q_avg_s = (qms / max(qn, 1)) * 1e-3
    peak, peak_kind = peaks()
    achieved = alg_bytes / q_avg_s / 1e9
    streamed_gbs = streamed_total / max(qn, 1) / q_avg_s / 1e9
    q_unique = uf
    step_kernels = {k: dict(ms_per_launch=(v[0] / v[1] if v[1] else None), launches=v[1]) for k, v in kt.items()}

    # accuracy at the stated configuration: FP32 vs the FP64 GPU path (same operators, one run),
    # and the discrete energy drift after the pulse has passed
    acc = None
    if rank == 0 and not args.no_accuracy:
        # FP64 single-column reference run(s): column 0 (and the last column when batched)
        # same operators (copied host set-up, nothing recomputed), FP64 state and arithmetic
        ref = ctx.like(precision=Y.YGM_FP64, n_rhs=1, energy_every=100, stream=stream.cuda_stream)
        ctx.set_state(ze, zb)
        ctx.step(W["steps"], dt, src)
        W32 = ctx.energy_history().reshape(-1, R)
        e32, b32 = ctx.get_state(synced=True)
        e32, b32 = e32.reshape(ctx.N1, R), b32.reshape(ctx.N2, R)
        cols = [0] if R == 1 else [0, R - 1]
        errs_e, errs_b, drift64, drift32, t64 = [], [], [], [], None
        for r in cols:
            ref.set_state(np.zeros(ref.N1), np.zeros(ref.N2))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ref.step(W["steps"], dt, source_for(W, dt, column=r))
            e64, b64 = ref.get_state(synced=True)
            if t64 is None:
                t64 = time.perf_counter() - t0
            Wh = ref.energy_history()
            errs_e.append(float(np.linalg.norm(e32[:, r] - e64) / np.linalg.norm(e64)))
            errs_b.append(float(np.linalg.norm(b32[:, r] - b64) / np.linalg.norm(b64)))
            # the pulse has passed after 4 sigma + t0 = 160 steps; records 3.. are source-free
            drift64.append(float(np.max(np.abs(Wh[3:] - Wh[3])) / Wh[3]) if len(Wh) > 4 else None)
            w = W32[:, r]
            drift32.append(float(np.max(np.abs(w[3:] - w[3])) / w[3]) if len(w) > 4 else None)
        acc = dict(columns_checked=cols, rel_l2_e_vs_fp64_gpu=max(errs_e), rel_l2_b_vs_fp64_gpu=max(errs_b),
                   fp64_gpu_vs_oracle=("every output of one step of this cavity within 1e-12 of the FP64 oracle "
                                       "(its Q1 rows evaluated locally): tests/test_gpu_2_fullsize.py"),
                   energy_drift_fp64_after_pulse=max((d for d in drift64 if d is not None), default=None),
                   energy_every=100,
                   note="drift = max |W_n - W_300| / W_300 over n >= 300 (pulse over); FP64 reference = "
                        "single-column FP64 GPU run of the same column's source",
                   energy_drift_fp32_after_pulse=max((d for d in drift32 if d is not None), default=None),
                   fp64_gpu_value=(ref.N1 + ref.N2) * W["steps"] / t64, fp64_gpu_ms_per_run=t64 * 1e3)
        ref.close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_line(args)
    if rank == 0:
        line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
                    ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None,
                    dtype="f64" if prec == Y.YGM_FP64 else "f32", data="synthetic",
                    config=dict(workload=(f"PEC cube N={W['n']} (6N^3={6 * W['n'] ** 3} Kuhn tets), k={W['k']}, "
                                          f"eps~U[1,4) seed 2000, z-dipole seed 2001, dt=0.5 tau_CFL, "
                                          f"{W['steps']} leapfrog steps per step") if R == 1 else
                                         (f"batched: PEC cube N={W['n']} (6N^3={6 * W['n'] ** 3} Kuhn tets), "
                                          f"k={W['k']}, eps~U[1,4) seed 2000, {R} RHS columns, one dipole each "
                                          f"(positions seed 3001, orientations seed 3002), dt=0.5 tau_CFL, "
                                          f"{W['steps']} leapfrog steps per step"),
                                n_rhs=R,
                                N1=ctx.N1, N2=ctx.N2, dofs=ctx.N1 + ctx.N2, leapfrog_steps=W["steps"],
                                q1_nnz=ctx.q1_nnz, q1=ctx.q1_info(), dt=dt, setup_s=setup_s,
                                parallelism=f"replicas{world}" if world > 1 else "single",
                                l2_policy="inputs larger than L2 (Q1 %.0f MB > 129 MB L2)" % (rs * q_unique / 1e6)),
                    e2e=dict(value=e2e_val, unit=UNIT, h2d_bytes_per_step=rs * (ctx.N1 + ctx.N2) * R,
                             d2h_bytes_per_step=rs * (ctx.N1 + ctx.N2) * R),
                    gpu_launches=launches,
                    roofline=dict(bound="hbm", achieved=achieved, peak=peak, unit="GB/s", frac=achieved / peak,
                                  traffic=(QAPPLY_TRAFFIC_BYTES if (QAPPLY_TRAFFIC_CURRENT and R == 1 and W["n"] == 32
                                                                    and W["k"] == 2 and prec == Y.YGM_FP32) else None),
                                  traffic_unit="bytes per launch (ncu, profiles/k_qapply_s_cavity_N32_k2_fp32.md)",
                                  traffic_last_capture=(QAPPLY_TRAFFIC_BYTES if (R == 1 and W["n"] == 32 and W["k"] == 2
                                                                                 and prec == Y.YGM_FP32) else None),
                                  traffic_last_capture_note="k_qapply_s before its two-instruction PDL prologue "
                                                            "(griddepcontrol); no memory operation changed since",
                                  kernel="k_qapply_s" if R == 1 else "k_qapply_p",
                                  bytes_per_launch=alg_bytes,
                                  launches=dict(curl_rows_only=n_act, all_rows=n_all),
                                  streamed_gbs=streamed_gbs,
                                  note="bytes: distinct Q1 values (symmetric pair once) + e + x; streamed_gbs "
                                       "counts the full-row Q1 entries the kernel actually reads",
                                  peak_source=f"{peak_kind} hbm_gbs"),
                    kernels=step_kernels, clocks=clk.summary(), accuracy=acc, cpu_baseline=cpu)
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "tf32", "tf32x3"],
                    help="tf32 / tf32x3: batched C^T M2 on tensor cores (needs --rhs 32, 64 or 128)")
    ap.add_argument("--n", type=int, default=32)
    ap.add_argument("--order", type=int, default=2)
    ap.add_argument("--leapfrog-steps", type=int, default=2000)
    ap.add_argument("--cpu-steps", type=int, default=5000,
                    help="leapfrog steps of the timed FP64 oracle sample (about 5 s on one core)")
    ap.add_argument("--cpu-n", type=int, default=5, help="cubes per side of the oracle sample")
    ap.add_argument("--energy-every", type=int, default=100)
    ap.add_argument("--rhs", type=int, default=1, help="right-hand-side columns (batched excitations)")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
