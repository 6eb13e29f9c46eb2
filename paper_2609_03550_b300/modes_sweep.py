"""Time the mode products (qds_mode_products) by the convolution sums and by
the theta-grid FFTs over the mode count, on many points, for the crossover
of Sec. 3.3 (the direct sums cost O(M^2) per point, the transforms
O(N log N) with N >= 3M - 2).

    python -m paper_2609_03550_b300.modes_sweep [--points 1048576] [--pairs 3]

Prints one line per mode count: ns per point for each method and FP32 /
FP64, and the maximum difference of the two methods relative to the
largest output."""
import argparse
import sys

import torch

from . import qds as Q


def time_ms(fn, reps=10):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--points", type=int, default=1 << 20)
    ap.add_argument("--pairs", type=int, default=3)
    ap.add_argument("--modes", default="2,4,8,12,16,24,32,48,64")
    a = ap.parse_args(argv)
    g = torch.Generator(device="cuda").manual_seed(3)
    print("M  N_theta  direct_f32 theta_f32 direct_f64 theta_f64 (ns per point)  max|diff|/max")
    for M in [int(x) for x in a.modes.split(",")]:
        row = [M, Q.lib().qds_mode_products_theta_points(M)]
        diff = 0.0
        for dt in (torch.complex64, torch.complex128):
            A = torch.randn((a.pairs, M, a.points), dtype=dt, device="cuda", generator=g)
            B = torch.randn((a.pairs, M, a.points), dtype=dt, device="cuda", generator=g)
            A[:, 0] = A[:, 0].real
            B[:, 0] = B[:, 0].real
            w = [1.0, 0.5, -0.5, 0.25][: a.pairs]
            outs = []
            for method in (Q.MODES_DIRECT, Q.MODES_THETA):
                out = torch.empty((M, a.points), dtype=dt, device="cuda")
                ms = time_ms(lambda: Q.mode_products(A, B, w, method=method, out=out))
                row.append(ms * 1e6 / a.points)
                outs.append(out)
            if dt == torch.complex128:
                diff = float((outs[0] - outs[1]).abs().max() / outs[0].abs().max())
            del A, B, outs
        print(f"{row[0]:3d} {row[1]:5d}  " + "  ".join(f"{v:9.3f}" for v in row[2:]) + f"  {diff:.1e}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
