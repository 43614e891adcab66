"""A small, self-contained run of the sweep kernels for profiling.

  python -m paper_1411_5512_gb300.profile_case [--L 128] [--samples 128] [--sweeps 4]
                                               [--rule 0] [--batch] [--cpt N] [--T 0.7]
                                               [--measure | --c4-radial]

One job of `samples` samples at side L (p_neg = 0.5, T = 0.7), quenched and swept
`sweeps` times through the plain path (or through a one-job batch with --batch,
whose launch shape --cpt sets: 1, 2 or 4).
At L = 128 and 128 samples the state is 168 MB, above the 126 MB L2, so DRAM
counters stay meaningful while the device footprint stays small.
"""
import argparse
import sys


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=128)
    ap.add_argument("--samples", type=int, default=128)
    ap.add_argument("--sweeps", type=int, default=4)
    ap.add_argument("--rule", type=int, default=0)
    ap.add_argument("--batch", action="store_true")
    ap.add_argument("--cpt", type=int, default=0, help="batch launch shape (0 = default)")
    ap.add_argument("--T", type=float, default=0.7)
    ap.add_argument("--measure", action="store_true", help="schedule t_w = t = {0, 1, 2, 4}")
    ap.add_argument("--c4-radial", action="store_true",
                    help="then the four-point sums over every vector of the last snapshot")
    a = ap.parse_args(argv)
    import torch

    from paper_1411_5512_gb300 import job

    j = job.EAJob(a.L, 0.5, 100, a.samples)
    if a.measure:
        j.set_schedule([0, 1, 2, 4], [0, 1, 2, 4])
    elif a.c4_radial:
        j.set_schedule([a.sweeps], [0])
    j.quench(a.T, a.rule)
    if a.batch:
        b = job.EABatch()
        b.configure(a.cpt, 0)
        b.add(j)
        b.sweep(a.sweeps)
        b.close()
    else:
        j.sweep(a.sweeps)
    if a.c4_radial:
        j.c4_radial(a.sweeps)
    torch.cuda.synchronize()
    print("ok", j.time)
    j.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
