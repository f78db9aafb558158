"""Small, self-terminating workloads of the library for ncu captures.

usage: python -m paper_1510_07799_gb300.profile_rhs [precision] [N] [repeats] [steps] [crossing] [tails]
Runs `repeats` rhs evaluations (default 2) of a seeded vertex at N (default
128, the U=3, T=0.005 workload parameters) and prints the phase timings of the
last one; with a fourth argument `steps` > 0 it then advances a flow of the
same workload by that many Dormand-Prince step attempts (one captured graph
per step), so that a launch list shows the kernels of the flow step.  Further
arguments `crossing` and `tails` make the context assert the crossing
symmetry (FRG_CROSSING) and add the frequency-box tails (FRG_TAILS), as
`bench.py --crossing` and `--tails` do.
With N = batch64 it advances the 64-point batch context by `steps` attempts
(no single-point evaluations) and prints the time of the last 10.
"""
import sys

import torch

from . import build, frg, inputs


def batch(prec, steps):
    build.build()
    ctx = frg.Context(inputs.batch_points(), precision=prec)
    ctx.advance(max(steps - 10, 0))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ctx.advance(min(steps, 10))
    e1.record()
    torch.cuda.synchronize()
    print("batch64: %d step attempts in %.3f ms" % (min(steps, 10), e0.elapsed_time(e1)))
    ctx.close()


def main():
    prec = sys.argv[1] if len(sys.argv) > 1 else "3xtf32"
    if len(sys.argv) > 2 and sys.argv[2] == "batch64":
        batch(prec, int(sys.argv[4]) if len(sys.argv) > 4 else 14)
        return
    N = int(sys.argv[2]) if len(sys.argv) > 2 else 128
    reps = int(sys.argv[3]) if len(sys.argv) > 3 else 2
    steps = int(sys.argv[4]) if len(sys.argv) > 4 else 0
    cross = "crossing" in sys.argv[5:]
    tails = "tails" in sys.argv[5:]
    build.build()
    w = inputs.Workload("profile", N=N, U=3.0, T=0.005, eps_d=-1.5)
    mask = frg.CH_ALL | (frg.CROSSING if cross else 0) | (frg.TAILS if tails else 0)
    ctx = frg.Context([w], precision=prec, channel_mask=mask)
    V = torch.from_numpy(inputs.random_vertex(N, w.U, 1)).cuda()
    s = torch.from_numpy(inputs.random_sigma(N, 2)).cuda()
    dg = torch.empty_like(V)
    ds = torch.empty_like(s)
    ph = None
    for _ in range(reps):
        ph = ctx.rhs_timed(0, 0.02, V, s, dg, ds)
    torch.cuda.synchronize()
    print("phases ms (bubble+sigma, regather, contraction, combine):", [round(x, 4) for x in ph[:4]])
    if steps > 0:
        st = ctx.advance(steps)[0]
        torch.cuda.synchronize()
        print("flow: %d step attempts, %d rhs evaluations" % (st.accepted + st.rejected, st.rhs_evals))
    ctx.close()


if __name__ == "__main__":
    main()
