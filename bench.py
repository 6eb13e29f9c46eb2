"""Benchmark of the QDS field step on B300.

Workload (default): the batched vacuum two-colour scan - 512 independent
EM + axion + axion-regenerated-field solves of uneven size (nx 512..4096,
nr 32..256, 2..4 modes, from seed 2), FP32 with the axion and regenerated
fields carried as phi/g and E1/g^2, moving window.  One "step" advances every
instance by one time step.  The state (36 GB in FP32) is far larger than L2.
The FP64 plain path is timed on the same workload, and FP32 is compared with
FP64 over the full 1000 steps on a sample of the instances; the FP64 CPU
oracle is timed on a bounded sample on the host cores.  With N GPUs the 512
instances are split into N disjoint subsets of equal cost (strong scaling).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl qds|reference]
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QDS cell-mode updates/s FP32-batched vs FP64-plain; % HBM roofline"
UNIT = "cell-mode updates/s"
# algorithmic bytes per cell-mode per step: the 15 complex state words
# (T_r+-, T_th+-, E_x, B_x; phi, T_a+-; and the regenerated group) read once
# and written once (phi_prev and the tile halos excluded)
WORDS = 15
BYTES_PER_UNIT = {"f32": 2 * WORDS * 8, "f64": 2 * WORDS * 16}


from paper_2609_03550_b300.ranks import env_rank  # noqa: E402


# The transposed step's algorithmic bytes per cell-mode (FP32): it reads the
# forward EM fields (6 complex words), the adjoint after the step (EM and
# axion, 9), the currents j_x, j_theta (2), and writes the adjoint before the
# step (9): 26 complex words of 8 bytes.
ADJ_BYTES_PER_UNIT = 26 * 8


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def kernel_hash():
    """Hash of the device code of the step's pass kernels (the headers that
    define them); launch code on the host does not change their counters."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2609_03550_b300", "csrc")
    for f in ("qds_common.cuh", "qds_stages.cuh", "qds_kernels.cuh", "qds_march.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload, prec):
    """DRAM bytes per step from an ncu capture summarised under profiles/,
    used only while the kernel source is the one that was profiled."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        e = d.get(f"{workload}/{prec}")
        if e and e.get("kernel_hash") == kernel_hash():
            return e["bytes_per_step"]
    except Exception:
        pass
    return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def build_solver(wls, flags, device, autotune=False):
    import torch
    from paper_2609_03550_b300 import qds as Q
    params = [Q.Params(w.nx, w.nr, w.M, w.dr, g=w.g, m_a=w.m_a, flags=flags) for w in wls]
    s = Q.QDSSolver(params, device=device)
    s.timings = {}
    if autotune:
        s.autotune()  # before the initial state is set: the trial steps advance the state
    for i, w in enumerate(wls):
        s.set_state(w.initial_state(device=device), i=i)
    torch.cuda.synchronize()
    return s


def time_steps(s, K, stream):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    s.step(K, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def phase_matched_scales(wl, T):
    """Amplitudes the two-colour pair of workload wl would drive in T time
    units if phase matched (manufactured resonance: a source S0 cos(kx - wt)
    grows phi as g S0 t / (2 w)): phi ~ g A1 A2 T / (2 dw), A1, A2 the peak
    pulse fields, dw = w1 - w2; the regenerated fields ~ g A1 dw phi T / 2."""
    l1, l2 = wl.lasers[0], wl.lasers[1]
    w1, w2 = 2 * math.pi / l1.lam, 2 * math.pi / l2.lam
    A1, A2 = l1.a0 * w1, l2.a0 * w2
    phi = wl.g * A1 * A2 * T / (2 * (w1 - w2))
    return phi, wl.g * A1 * (w1 - w2) * phi * T / 2


def accuracy(wls, flags, device, steps):
    """FP32 against FP64 on the GPU after ``steps`` steps of the given
    instances (the FP64 GPU path matches the oracle to 1e-12 in the tests):
    relative L2 of the EM fields; for the axion and regenerated groups the
    amplitude error (max |diff| / max |FP64|) and the error against the
    phase-matched scales (the vacuum pulses leave only a residue of axion,
    ~1e-4 of that scale or less); worst over the instances."""
    import numpy as np
    import torch
    from paper_2609_03550_b300 import qds as Q
    s64 = build_solver(wls, flags, device)
    s32 = build_solver(wls, flags | Q.FP32, device)
    s64.step(steps)
    s32.step(steps)
    torch.cuda.synchronize()
    worst = {"em_rel_l2": 0.0, "axion_rel_l2": 0.0, "arem_rel_l2": 0.0, "axion_amplitude": 0.0,
             "arem_amplitude": 0.0, "axion_vs_phase_matched_scale": 0.0, "arem_vs_phase_matched_scale": 0.0,
             "fp64_axion_vs_phase_matched_scale": 0.0}
    for i, w in enumerate(wls):
        a = s32.get_state(i).cpu().numpy()
        b = s64.get_state(i).cpu().numpy()
        n = w.M * w.nx * w.nr
        s_phi, s_e1 = phase_matched_scales(w, steps * w.h)
        for name, lo, hi, sc in (("em", 0, 6, None), ("axion", 6, 9, s_phi), ("arem", 9, 15, s_e1)):
            d, r = a[lo * n:hi * n] - b[lo * n:hi * n], b[lo * n:hi * n]
            worst[f"{name}_rel_l2"] = max(worst[f"{name}_rel_l2"], float(np.linalg.norm(d) / np.linalg.norm(r)))
            if sc is not None:
                worst[f"{name}_amplitude"] = max(worst[f"{name}_amplitude"],
                                                 float(np.abs(d).max() / np.abs(r).max()))
                dd = np.abs(d[:n]).max() if name == "axion" else np.abs(d).max()  # axion: phi itself
                worst[f"{name}_vs_phase_matched_scale"] = max(worst[f"{name}_vs_phase_matched_scale"], float(dd / sc))
        worst["fp64_axion_vs_phase_matched_scale"] = max(worst["fp64_axion_vs_phase_matched_scale"],
                                                         float(np.abs(b[6 * n:7 * n]).max() / s_phi))
    del s32, s64
    torch.cuda.empty_cache()
    worst.update({"steps": steps, "instances": [w.name for w in wls], "against": "FP64 on the GPU",
                  "bounds": {"em_rel_l2": 1e-5, "axion_vs_phase_matched_scale": 1e-4,
                             "arem_vs_phase_matched_scale": 1e-4},
                  "note": "vacuum pulses: the axion is a residue of the vanishing vacuum source; the amplitude "
                          "errors of physically generated axion (two-colour + bunch) are in tests/test_gpu_precision.py"})
    return worst


def cpu_baseline(wls, flags, budget_s):
    """The FP64 oracle on the host cores over a bounded sample of the same
    workload: whole instances in order, one step each, until budget_s."""
    import numpy as np  # noqa: F401
    import oracle
    units, t_total, used = 0, 0.0, []
    for w in wls:
        st = oracle.State(w.M, w.nx, w.nr, w.initial_state())
        p = dict(nx=w.nx, nr=w.nr, M=w.M, h=1.0, dr=w.dr, g=w.g, m_a=w.m_a, flags=flags & 31)
        t0 = time.perf_counter()
        oracle.step(p, st)
        t_total += time.perf_counter() - t0
        units += w.cell_modes()
        used.append(w.name)
        if t_total >= budget_s:
            break
    cores = oracle.set_threads(0)
    # the same on one thread, over a quarter of the time budget
    oracle.set_threads(1)
    u1, t1 = 0, 0.0
    for w in wls:
        st = oracle.State(w.M, w.nx, w.nr, w.initial_state())
        p = dict(nx=w.nx, nr=w.nr, M=w.M, h=1.0, dr=w.dr, g=w.g, m_a=w.m_a, flags=flags & 31)
        t0 = time.perf_counter()
        oracle.step(p, st)
        t1 += time.perf_counter() - t0
        u1 += w.cell_modes()
        if t1 >= budget_s / 4:
            break
    oracle.set_threads(cores)
    return {"value": units / t_total, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one FP64 step of each of the first {len(used)} instances ({units} cell-modes, {t_total:.1f} s)",
            "value_1_thread": u1 / t1, "sample_1_thread": f"{u1} cell-modes, {t1:.1f} s"}


def adjoint_bench(device, steps, every):
    """Gradient of the axion energy around the pulses after ``steps`` steps of
    the two-colour + bunch run (FP32, 4096 x 128, modes 0..2) with respect to
    the laser-2 radial profile, omega2 and g, by run_qds (checkpoints every
    ``every`` steps, recompute, transposed steps).  Reports the forward and
    backward times and the identity dL/dg = 2 L / g (the axion grows from
    zero and is linear in g).  The run is timed after one untimed run."""
    import torch
    from paper_2609_03550_b300 import adjoint as A
    from paper_2609_03550_b300 import inputs as I
    from paper_2609_03550_b300 import qds as Q
    wl = I.adjoint_run(steps=steps)
    ex = wl.extra
    p = Q.Params(wl.nx, wl.nr, wl.M, wl.dr, g=wl.g, m_a=wl.m_a,
                 flags=Q.AXION | Q.AREM | Q.MOVING_WINDOW | Q.FP32)
    src = I.DeviceBunchSources(wl, device, torch.complex64)
    spec = A.RunSpec(p, steps, every=every, sources=src, device=str(device))
    prof = torch.tensor(ex["profile2"], dtype=torch.complex128, device=device, requires_grad=True)
    om = torch.tensor(ex["omega2"], dtype=torch.float64, device=device, requires_grad=True)
    g = torch.tensor(wl.g, dtype=torch.float64, device=device, requires_grad=True)
    base = wl.initial_state(device=device)
    # one untimed run first: the device memory of the checkpoints and of the
    # re-run segments is touched for the first time there
    for timed in (False, True):
        for t in (prof, om, g):
            t.grad = None
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ev[0].record()
        s0 = A.laser2_state(base, p, prof, om, ex["x0"], ex["fwhm"])
        L = A.axion_energy(A.run_qds(s0, g, spec), p, *ex["window"])
        ev[1].record()
        L.backward()
        ev[2].record()
        torch.cuda.synchronize()
    fwd, bwd = ev[0].elapsed_time(ev[1]) / 1e3, ev[1].elapsed_time(ev[2]) / 1e3
    Lv, gg = float(L.detach()), float(g.grad)
    units = wl.cell_modes() * steps
    # the transposed step alone (qds_adjoint_step_w with the snapshots at the
    # start and the end of the step), as the backward pass runs it
    s = Q.QDSSolver(p, device=device)
    s.set_state(base)
    jx, jr, jt = src(0)
    s.step(3, jx=jx, jr=jr, jth=jt)
    snap, k0 = s.save_working(em_only=True)
    s.step(1, jx=jx, jr=jr, jth=jt)
    nxt, _ = s.save_working(em_only=True)
    gen = torch.Generator(device=device)
    gen.manual_seed(5)
    plane = wl.M * wl.nx * wl.nr
    lam = torch.randn(p.state_elems(), dtype=torch.complex64, device=device, generator=gen)
    lam[9 * plane:15 * plane] = 0
    lam_b = torch.zeros_like(lam)
    dg = torch.zeros(1, dtype=torch.float64, device=device)
    bufs = [lam, lam_b]
    for i in range(3):
        s.adjoint_step_w(snap, k0, bufs[i % 2], bufs[(i + 1) % 2], jx=jx, jth=jt, dLdg=dg, fwd_next=nxt)
    reps, batches = 20, 5
    times = []
    for _ in range(batches):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(reps):
            s.adjoint_step_w(snap, k0, bufs[i % 2], bufs[(i + 1) % 2], jx=jx, jth=jt, dLdg=dg, fwd_next=nxt)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / reps / 1e3)
    t_adj = statistics.median(times)
    peak, peak_kind = measured_peak()
    achieved = wl.cell_modes() * ADJ_BYTES_PER_UNIT / t_adj / 1e9
    transposed = {"ms": t_adj * 1e3, "launches": 3, "cell_modes": wl.cell_modes(),
                  "bytes_per_cell_mode": ADJ_BYTES_PER_UNIT,
                  "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                               "frac": achieved / peak, "peak_kind": peak_kind},
                  "timing": f"median of {batches} runs of {reps} calls after 3 (ms per call: "
                            + ", ".join(f"{t * 1e3:.4f}" for t in times) + "), CUDA events; inputs larger than L2"}
    return {"workload": wl.name, "steps": steps, "checkpoint_every": spec.interval(), "dtype": "f32",
            "params": "laser-2 radial profile (%d complex), omega2, g" % wl.nr,
            "loss": "axion energy in window cells [%d, %d)" % ex["window"], "L": Lv,
            "forward_s": fwd, "backward_s": bwd, "backward_over_forward": bwd / fwd,
            "value": units / (fwd + bwd), "unit": "cell-mode updates/s (forward + gradient)",
            "dLdg_vs_2L_over_g": abs(gg - 2 * Lv / wl.g) / abs(gg),
            "grad_finite": bool(torch.isfinite(prof.grad).all()) and math.isfinite(float(om.grad)) and math.isfinite(gg),
            "transposed_step": transposed,
            "checks": "gradients vs oracle central differences and oracle Jacobian columns: tests/test_gpu_adjoint.py"}


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    from paper_2609_03550_b300 import inputs as I
    wls = I.batched_scan()
    flags = 1 | 2 | 4
    import oracle
    # each step: one oracle step over a bounded sample (instance 0)
    w = wls[0]
    st = oracle.State(w.M, w.nx, w.nr, w.initial_state())
    p = dict(nx=w.nx, nr=w.nr, M=w.M, h=1.0, dr=w.dr, g=w.g, flags=flags)
    for _ in range(args.warmup):
        oracle.step(p, st)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.step(p, st)
    dt = time.perf_counter() - t0
    v = w.cell_modes() * args.steps / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", len(os.sched_getaffinity(0))))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": "batched_vacuum_two_colour_scan_512_seed2",
                                           "sample": f"instance 0 ({w.nx}x{w.nr}x{w.M})"},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"FP64 oracle steps of instance 0 ({w.cell_modes()} cell-modes per step)"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_qds(args):
    import torch
    from paper_2609_03550_b300.ranks import Ranks, job_throughput, shard
    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    ranks = Ranks("nccl", device)
    barrier, max_over_ranks = ranks.barrier, ranks.max

    from paper_2609_03550_b300 import inputs as I
    from paper_2609_03550_b300 import qds as Q
    scan = I.batched_scan()[: args.instances]
    total_units = sum(w.cell_modes() for w in scan)
    mine = shard([w.cell_modes() for w in scan], world)[rank]  # this rank's instances
    wls = [scan[i] for i in mine]
    units = sum(w.cell_modes() for w in wls)
    flags = Q.AXION | Q.AREM | Q.MOVING_WINDOW
    stream = torch.cuda.current_stream(device)

    # ---------------- FP32 batched ----------------
    s = build_solver(wls, flags | Q.FP32, device, autotune=not args.no_autotune)
    tile = s.tile()
    tile["step_mode"] = s.step_mode_name()
    tile["autotune_ms_per_step"] = {f"{['default', 'flat', 'march'][m]} rows={r} cols={c}": round(t, 3)
                                    for (m, r, c), t in s.timings.items()}
    launches_per_step = s.step_launches()
    s.step(args.warmup, stream=stream)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    reps = []
    for _ in range(args.repeats):
        barrier()
        reps.append(max_over_ranks(time_steps(s, args.steps, stream)))
    barrier()
    clk = clocks.stop()
    t32 = statistics.median(reps)
    step32 = t32 / args.steps
    status = s.status()

    # ---------------- end to end through the public API ----------------
    # per step: advance every instance, compute every instance's energies
    # (EM, axion, regenerated, exchange) and read them back to pinned host
    # memory; the undriven vacuum workload has no per-step inputs.
    diag_dev = torch.empty((len(wls), 4), dtype=torch.float64, device=device)
    diag_host = torch.empty((len(wls), 4), dtype=torch.float64, pin_memory=True)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.step(1, stream=stream)
        s.diagnostics_all(diag_dev, stream=stream)
        diag_host.copy_(diag_dev, non_blocking=True)
        stream.synchronize()
    te2e = max_over_ranks(time.perf_counter() - t0)
    e2e_finite = bool(torch.isfinite(diag_host).all())
    del s
    torch.cuda.empty_cache()

    # ---------------- accuracy of FP32 against FP64 ----------------
    acc = None
    if not args.no_accuracy:
        sample = [w for w in wls if w.name in {f"scan_{i}" for i in range(args.accuracy_instances)}]
        if sample:
            acc = accuracy(sample, flags, device, sample[0].steps)

    # ---------------- FP64 plain on the same workload ----------------
    fp64 = None
    if not args.no_fp64:
        s64 = build_solver(wls, flags, device)
        s64.step(1, stream=stream)
        barrier()
        t64 = max_over_ranks(time_steps(s64, args.fp64_steps, stream))
        step64 = t64 / args.fp64_steps
        fp64 = {"value": job_throughput(total_units, step64), "unit": UNIT, "ms_per_step": 1e3 * step64,
                "steps": args.fp64_steps, "dtype": "f64", "step_mode": s64.step_mode_name(),
                "hbm_gbs_algorithmic": units * BYTES_PER_UNIT["f64"] / step64 / 1e9,
                "fp32_speedup": step64 / step32,
                "fp32_accuracy_at_this_speedup": None if acc is None else
                {k: acc[k] for k in ("em_rel_l2", "axion_vs_phase_matched_scale", "arem_vs_phase_matched_scale",
                                     "axion_amplitude", "arem_amplitude")}}
        del s64
        torch.cuda.empty_cache()

    adj = None
    if world == 1 and not args.no_adjoint:
        adj = adjoint_bench(device, args.adjoint_steps, args.adjoint_every)
        torch.cuda.empty_cache()

    if rank != 0:
        ranks.close()
        return
    peak, peak_kind = measured_peak()
    achieved = units * BYTES_PER_UNIT["f32"] / step32 / 1e9
    traffic = recorded_traffic("batched_scan", "f32")
    cpu = None
    if world == 1 and not args.no_cpu:
        cpu = cpu_baseline(wls, flags, args.cpu_seconds)
    out = {
        "metric": METRIC, "value": job_throughput(total_units, step32), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * step32,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "batched_vacuum_two_colour_scan_512_seed2" if len(scan) == 512
                   else f"batched_vacuum_two_colour_scan_first{len(scan)}_seed2", "instances": len(scan),
                   "cell_modes_per_step": total_units, "modes": "2..4", "nx": "513..4085", "nr": "32..254",
                   "precision": "FP32, phi/g and E1/g^2", "parallelism": f"instances split over {world} GPU(s)",
                   "l2": f"inputs larger than L2 ({units * BYTES_PER_UNIT['f32'] / 2e9:.1f} GB FP32 state per GPU)",
                   "timing": f"median of {args.repeats} timed runs of {args.steps} steps (ms per step: "
                             + ", ".join(f"{1e3 * t / args.steps:.2f}" for t in reps) + ")",
                   "tile": tile},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "the kernels of one step, all mode counts (the step reads and writes the state "
                               "once in algorithmic terms)",
                     "bytes_per_unit": BYTES_PER_UNIT["f32"], "peak_kind": peak_kind},
        "accuracy": acc,
        "device_status": status,
        "fp64_plain": fp64,
        "e2e": {"value": total_units * args.steps / te2e, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": int(diag_host.numel() * 8), "finite": e2e_finite,
                "per_step": "step + energies of all instances + device-to-host read (the vacuum scan has no "
                            "per-step inputs)"},
        "gpu_launches": args.steps * launches_per_step,
        "adjoint": adj,
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    print(json.dumps(out), flush=True)
    ranks.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="qds", choices=["qds", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--instances", type=int, default=512, help="first N instances (profiling runs only)")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default step mode (profiling runs)")
    ap.add_argument("--repeats", type=int, default=5, help="timed runs of --steps steps (the median is reported)")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--accuracy-instances", type=int, default=8,
                    help="FP32 vs FP64 over the full run on the scan's first N instances")
    ap.add_argument("--adjoint-steps", type=int, default=8000)
    ap.add_argument("--adjoint-every", type=int, default=90)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "qds":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_qds(args)


if __name__ == "__main__":
    main()
