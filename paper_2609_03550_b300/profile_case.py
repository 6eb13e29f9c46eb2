"""A short run of the benchmark workload for profilers: the first N
instances of the batched scan (or the gradient workload with its per-step
currents, or that workload's transposed step), a chosen precision and step
implementation, a few steps.

    python -m paper_2609_03550_b300.profile_case --instances 8 --precision f32 --mode march --steps 3
    python -m paper_2609_03550_b300.profile_case --workload gradient --steps 90
    python -m paper_2609_03550_b300.profile_case --workload transpose --steps 4

It prints the cell-modes per step and the device status, and exits non-zero
if the device reports an error.
"""
import argparse
import sys

import torch

from . import inputs as I
from . import qds as Q


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="scan", choices=["scan", "gradient", "transpose"])
    ap.add_argument("--instances", type=int, default=8)
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--mode", default="default", choices=["default", "flat", "march"])
    ap.add_argument("--rows", type=int, default=0)
    ap.add_argument("--cols", type=int, default=0)
    ap.add_argument("--steps", type=int, default=3)
    a = ap.parse_args(argv)
    dev = "cuda:0"
    prec = Q.FP32 if a.precision == "f32" else 0
    mode = {"default": Q.STEP_DEFAULT, "flat": Q.STEP_FLAT, "march": Q.STEP_MARCH}[a.mode]
    flags = Q.AXION | Q.AREM | Q.MOVING_WINDOW | prec
    if a.workload == "scan":
        wls = I.batched_scan()[: a.instances]
        s = Q.QDSSolver([Q.Params(w.nx, w.nr, w.M, w.dr, g=w.g, m_a=w.m_a, flags=flags) for w in wls], device=dev)
        s.set_tile(a.rows, a.cols)
        s.set_step_mode(mode)
        for i, w in enumerate(wls):
            s.set_state(w.initial_state(device=dev), i=i)
        s.step(a.steps)
        units = sum(w.cell_modes() for w in wls)
    elif a.workload == "transpose":
        # qds_adjoint_step_w, --steps times, at the state after three driven
        # steps (the snapshots at the start and the end of the fourth)
        wl = I.adjoint_run(steps=4)
        p = Q.Params(wl.nx, wl.nr, wl.M, wl.dr, g=wl.g, m_a=wl.m_a, flags=flags)
        s = Q.QDSSolver(p, device=dev)
        s.set_state(wl.initial_state(device=dev))
        src = I.DeviceBunchSources(wl, dev, torch.complex64 if prec else torch.complex128)
        jx, jr, jt = src(0)
        s.step(3, jx=jx, jr=jr, jth=jt)
        snap, k0 = s.save_working(em_only=True)
        s.step(1, jx=jx, jr=jr, jth=jt)
        nxt, _ = s.save_working(em_only=True)
        gen = torch.Generator(device=dev)
        gen.manual_seed(1)
        plane = wl.M * wl.nx * wl.nr
        lam = torch.randn(p.state_elems(), dtype=s.rdtype, device=dev, generator=gen)
        lam[9 * plane:15 * plane] = 0
        bufs = [lam, torch.zeros_like(lam)]
        dg = torch.zeros(1, dtype=torch.float64, device=dev)
        for i in range(a.steps):
            s.adjoint_step_w(snap, k0, bufs[i % 2], bufs[(i + 1) % 2], jx=jx, jth=jt, dLdg=dg, fwd_next=nxt)
        units = wl.cell_modes()
    else:
        wl = I.adjoint_run(steps=a.steps)
        s = Q.QDSSolver(Q.Params(wl.nx, wl.nr, wl.M, wl.dr, g=wl.g, m_a=wl.m_a, flags=flags), device=dev)
        s.set_tile(a.rows, a.cols)
        s.set_step_mode(mode)
        s.set_state(wl.initial_state(device=dev))
        src = I.DeviceBunchSources(wl, dev, torch.complex64 if prec else torch.complex128)
        s.set_sources(0, *src.fill(0, a.steps), per_step=True)
        s.step(a.steps)
        units = wl.cell_modes()
    torch.cuda.synchronize()
    st = s.status()
    print(f"cell-modes per step {units}, steps {a.steps}, status {st}")
    return 0 if st == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
