"""Benchmark: vertex right-hand-side evaluations per second of the one-loop SIAM
fRG flow at N_f = 128 on one GB300 (and N independent replicas for --gpus N).

One benchmark step = one whole N_f = 128 flow through the C ABI, from the bare
vertex at Lambda0 = 1e3 down to Lambda_f = 1e-3 (about 80 Dormand-Prince step
attempts, each six rhs evaluations -- bubble weights, channel contractions,
self-energy -- plus the stage sums, the error norm and the step controller),
i.e. every row of the hot path.  value = rhs evaluations actually performed in
the timed flows / device time (CUDA events, max over ranks), summed over ranks.
The default line also carries the other workloads' figures under "configs"
(64-point batch, N_f = 256, N_f = 64 flows), each bounded to seconds.

Arms:
  default            the CUDA library (precision --precision)
  --impl reference   the FP64 CPU oracle as it stands, timed on the host cores on
                     a bounded sample of the same workload (rows of the vertex)

Secondary workloads (--workload; each prints its own JSON line, not the
headline):
  batch64    64 parameter points with N_f in {32, 48, 64, 96} integrated in one
             context (one captured graph per step over all points): full flows
             per second, next to 64 sequential plain-FP64 GPU flows
  siam_N256  the largest single flow, N_f = 256: rhs evaluations per second,
             phase times and the error of one rhs against the FP64 GPU path on
             the same state
  siam_N64   full flows per second at N_f = 64 (off particle-hole symmetry):
             the plain FP64 GPU path and the 3xTF32 path, next to the oracle's
             flow on the host cores (one flow, --no-oracle skips it)
  siam_N64_iflow  the same with the interaction-flow cutoff (Lambda = 1/g from
             1e12 down to the full model at 1)
Options of the headline workload: --tails (frequency-box tails), --reversal
(the frequency-reversal reduction asserted for every input, half storage),
--no-reversal (flows compute every transfer), --crossing (the crossing
reduction of the channel products, FRG_CROSSING, which every flow from the
bare vertex may assert).  By default a split-precision
flow uses the reversal reduction automatically (every flow from the bare vertex
is exactly reversal-symmetric); the line then also reports the same flows
computing every transfer under "every_transfer".
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "vertex-rhs evals/s at N_f=128: split-TF32 vs FP64 on one GB300 @≤1e-6 rel"
UNIT = "rhs evals/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
FP64_NOMINAL_TFLOPS = 1.25  # GB300 nominal FP64 rate (CUDA cores)
DTYPES = {"fp64": "f64", "3xtf32": "tf32x3", "bf16x3": "bf16x3"}


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        p["_source"] = "measured"
        return p
    except Exception:
        p = dict(FALLBACK_PEAKS)
        p["_source"] = "fallback"
        return p


def profiled_traffic(kind):
    """DRAM bytes per rhs of the contraction launches from the committed ncu
    summary, or None if the kernel source changed since it was captured."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "contraction_%s_N128.md" % kind)
    try:
        kv = {}
        for line in open(path):
            if ":" in line and not line.startswith(("|", "#", " ", "`")):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        src = os.path.join(ROOT, kv["source"])
        if hashlib.sha256(open(src, "rb").read()).hexdigest() != kv["source_sha256"]:
            return None
        return float(kv["dram_bytes_per_rhs"])
    except Exception:
        return None


def executed_tensor_flops(N, NT=128, mrows=64, ks=16, half=False, products=3):
    """Tensor-core flops the split kernel issues per rhs: per tile (64 complex
    rows x NT columns) and k-step of 16 complex k, `products` slice products
    (3xTF32: 3, BF16x3: 6) of M = 128 real rows (real form of the left operand)
    x N = NT x K = 32; ragged transfers padded to whole tiles and k-steps (the
    direct channel has two K halves)."""
    tot = 0
    for ch in range(3):
        for m in range(-(N - 1), 1 if half else N):
            D = N - abs(m)
            nk = (2 if ch == 1 else 1) * -(-D // ks)
            tiles = -(-D // mrows) * -(-N // min(NT, -(-N // 16) * 16))
            tot += tiles * nk * products * 2 * 128 * (2 * min(NT, -(-N // 16) * 16)) * ks
    return tot


def contraction_macs(N, half=False):
    """Useful complex multiply-adds of the three channel contractions per rhs:
    4 N sum_m D_m^2 with D_m = N - |m| (pp: D x D x N, dph: D x 2D x N,
    xph: D x D x N per transfer); with the reversal reduction only the
    transfers m <= 0 (about half) are contracted."""
    return 4 * N * sum((N - abs(m)) ** 2 for m in range(-(N - 1), 1 if half else N))


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.path:
            return None
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_over_ranks(ms, evals, device=None):
    """Whole-job figures of N independent replicas (one flow per rank, no
    data-path collective): the slowest rank's time and the evaluations of all
    ranks.  With one rank (or no process group) the inputs come back."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    ev = torch.tensor([float(evals)], dtype=torch.float64, device=device)
    try:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            dist.all_reduce(ev, op=dist.ReduceOp.SUM)
    except ImportError:
        pass
    return float(t.item()), float(ev.item())


def oracle_rows_per_call(threads, N=128):
    """Vertex rows i1 per oracle call: the oracle's OpenMP loop runs over the
    rows of a call, so a call takes two rows per thread (every core busy)."""
    return max(1, min(N, 2 * threads))


def cpu_baseline(seconds=12.0, mask=0xF):
    """The FP64 oracle as it stands on the host cores, on whole rows i1 of the
    N=128 vertex (a bounded sample), scaled to rhs evaluations per second."""
    import numpy as np
    import oracle
    from paper_1510_07799_gb300 import inputs
    w = inputs.SIAM_N128
    m = oracle.Model(U=w.U, T=w.T, eps_d=w.eps_d, Delta=w.Delta, N=w.N)
    V = inputs.random_vertex(w.N, w.U, seed=11)
    sig = inputs.random_sigma(w.N, seed=12, amp=0.05)
    N_rows = oracle_rows_per_call(oracle.max_threads(), w.N)
    rows, t0 = 0, time.perf_counter()
    i = 0
    while True:
        a = (i * N_rows) % w.N
        oracle.rhs_rows(m, 0.02, V, sig, a, a + N_rows, mask=mask)
        rows += N_rows
        i += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    res = {"value": (rows / w.N) / el, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
           "host_cpus": os.cpu_count(),
           "sample": "%d vertex rows i1 (of %d) of one rhs evaluation at N_f=%d (channel mask 0x%x), %d rows "
                     "per call, repeated for %.1f s; scaled by rows/N" % (rows, w.N, w.N, mask, N_rows, el)}
    # the same sample on one thread (a quarter of the time budget)
    oracle.set_threads(1)
    try:
        rows1, t0 = 0, time.perf_counter()
        while True:
            a = rows1 % w.N
            oracle.rhs_rows(m, 0.02, V, sig, a, a + 1, mask=mask)
            rows1 += 1
            el1 = time.perf_counter() - t0
            if el1 >= seconds / 4:
                break
    finally:
        oracle.set_threads(0)  # back to the OpenMP default
    res["value_1thread"] = (rows1 / w.N) / el1
    res["sample_1thread"] = "%d vertex rows on one thread in %.1f s" % (rows1, el1)
    res["speedup_vs_1thread"] = res["value"] / res["value_1thread"]
    return res


def run_reference(args):
    world, rank, _ = dist_init()
    if rank != 0:
        return 0
    import oracle  # noqa: F401
    from oracle import build as oracle_build
    oracle_build.build()
    import numpy as np
    import oracle as orc
    from paper_1510_07799_gb300 import inputs
    w = inputs.SIAM_N128
    m = orc.Model(U=w.U, T=w.T, eps_d=w.eps_d, Delta=w.Delta, N=w.N)
    V = inputs.random_vertex(w.N, w.U, seed=11)
    sig = inputs.random_sigma(w.N, seed=12, amp=0.05)
    # one step = two vertex rows per host thread of one rhs evaluation
    rows = oracle_rows_per_call(orc.max_threads(), w.N)
    for i in range(args.warmup):
        orc.rhs_rows(m, 0.02, V, sig, 0, rows)
    t0 = time.perf_counter()
    for i in range(args.steps):
        a = (i * rows) % w.N
        orc.rhs_rows(m, 0.02, V, sig, a, a + rows)
    el = time.perf_counter() - t0
    value = args.steps * rows / w.N / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w.name, "N_f": w.N, "step": "oracle rhs on %d of %d vertex rows" % (rows, w.N)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": orc.max_threads(), "kind": "oracle",
                             "sample": "%d rows of %d per step, %d steps" % (rows, w.N, args.steps)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def run_ours(args):
    import numpy as np
    import torch
    world, rank, local = dist_init()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1510_07799_gb300 import build as cuda_build
    cuda_build.build()
    from paper_1510_07799_gb300 import frg, inputs
    w = inputs.SIAM_N128
    N = w.N
    prec = args.precision
    mask = frg.CH_ALL | (frg.TAILS if args.tails else 0) | (frg.REVERSAL if args.reversal else 0) | \
        (frg.NO_REVERSAL if args.no_reversal else 0) | (frg.CROSSING if args.crossing else 0)
    # the reversal reduction is in effect for split-precision flows unless turned off
    reduced = prec != "fp64" and not args.no_reversal
    ctx = frg.Context([w], precision=prec, channel_mask=mask)
    tune = ctx.autotune() if prec != "fp64" else None
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---- whole flows (the headline value): every step integrates the N = 128
    # flow from the bare vertex at Lambda0 down to Lambda_f
    bare = torch.full((N, N, N), w.U, dtype=torch.complex128, device=dev)

    def one_flow():
        ctx.set_state(0, bare, None, w.Lambda0)
        st = ctx.flow()[0]
        if st.status != 0 or not st.done:
            raise RuntimeError("flow failed: %s" % (st,))
        return st

    for _ in range(args.warmup):
        one_flow()
    barrier()
    torch.cuda.synchronize()
    l0 = frg.kernel_launches()
    evals = attempts = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            st = one_flow()
            evals += st.rhs_evals
            attempts += st.accepted + st.rejected
        e1.record(stream)
        torch.cuda.synchronize()
    barrier()
    launches = frg.kernel_launches() - l0
    ms = e0.elapsed_time(e1)
    ms_max, ev_all = reduce_over_ranks(ms, evals, device=dev)
    value = ev_all / (ms_max / 1e3)

    # ---- per-phase timing of single rhs evaluations on the same stream
    g, s, lam, _ = ctx.get_state(0)
    dg = torch.empty_like(g)
    ds = torch.empty_like(s)
    for _ in range(2):
        ctx.rhs_timed(0, lam, g, s, dg, ds)
    phases = np.array([ctx.rhs_timed(0, lam, g, s, dg, ds) for _ in range(args.rhs_reps)])
    ph = phases.mean(axis=0)
    pk = peaks()
    # the per-phase split above is of stand-alone rhs evaluations (every
    # transfer unless --reversal asserts the symmetry)
    macs = contraction_macs(N, half=args.reversal)
    if prec == "fp64":
        flops = 8.0 * macs
        achieved = flops / (ph[2] * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_NOMINAL_TFLOPS, "traffic": None,
                "kernel": "k_contract_fp64 (pp, dph, xph launches of one rhs)",
                "peak_source": "nominal GB300 FP64 rate (no measured FP64 peak)",
                "algorithmic": "8 flops x %d useful complex MACs per rhs" % macs}
    else:
        flops = 8.0 * macs
        bf = prec == "bf16x3"
        # the products run in the slices' own type: BF16 at the measured bf16
        # rate, TF32 at half of it (nominal tf32/bf16 ratio)
        tc_peak = pk["bf16_tflops"] * (1.0 if bf else 0.5)
        nprod = 6 if bf else 3
        achieved = flops / (ph[2] * 1e-3) / 1e12
        executed = executed_tensor_flops(N, half=args.reversal, products=nprod) / (ph[2] * 1e-3) / 1e12
        roof = {"bound": "tensor", "achieved": achieved, "peak": tc_peak, "unit": "TFLOP/s",
                "frac": achieved / tc_peak,
                "traffic": None if args.reversal else profiled_traffic("bf16x3" if bf else "tf32"),
                "traffic_unit": "DRAM bytes per rhs (contraction launch, ncu, cold cache)",
                "kernel": "tcgen05 channel contractions of one rhs",
                "peak_source": ("%s bf16 burst" if bf else "%s bf16 burst x 0.5 (nominal tf32/bf16 ratio)") % pk["_source"],
                "algorithmic": "8 flops x %d useful complex MACs per rhs (useful, not executed)" % macs,
                "executed_tflops": executed,
                "executed_frac": executed / tc_peak,
                "executed_note": "tensor-core flops issued (%d slice products, real form of the complex product, whole tiles "
                                 "and k-steps), for comparison with the tensor pipe's own rate; not the roofline value"
                                 % nprod}
    roof["phases_ms"] = {"bubble_and_sigma": ph[0], "regather": ph[1], "contraction": ph[2], "combine": ph[3]}
    if args.tails:
        roof["phases_ms"]["tails_add"] = ph[4]

    # ---- end to end through the host-buffer entry point: pinned host buffers,
    # the pipelined call (input copy, evaluation and output copy of successive
    # calls overlap); every call copies its input in and its result out
    hg = g.cpu().pin_memory().numpy()
    hs = s.cpu().pin_memory().numpy()
    reps = max(2, args.e2e_reps)
    outs = [(torch.empty(hg.shape, dtype=torch.complex128).pin_memory().numpy(),
             torch.empty(hs.shape, dtype=torch.complex128).pin_memory().numpy()) for _ in range(reps)]
    for og, os_ in outs[:2]:
        ctx.rhs_host_async(0, lam, hg, hs, og, os_)
    ctx.sync()
    t0 = time.perf_counter()
    for og, os_ in outs:
        ctx.rhs_host_async(0, lam, hg, hs, og, os_)
    ctx.sync()
    e2e_s = (time.perf_counter() - t0) / reps
    nb = (hg.nbytes + hs.nbytes)
    e2e = {"value": world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": nb, "d2h_bytes_per_step": nb,
           "what": "frg_rhs_host_async with pinned host buffers (%d calls in flight, then frg_sync), copies "
                   "inside the timed region" % reps}
    e2e["link"] = host_link(torch, nb)
    bound = min(e2e["link"]["h2d_concurrent_gbs"], e2e["link"]["d2h_concurrent_gbs"]) * 1e9 / nb
    e2e["link"]["bound_rhs_per_s"] = bound
    e2e["link"]["frac"] = e2e["value"] / world / bound

    # the plain FP64 GPU path on the same state (the metric's comparison arm)
    fp64_gpu = None
    if prec != "fp64":
        with frg.Context([w], precision="fp64", channel_mask=mask) as c64:
            for _ in range(2):
                c64.rhs_timed(0, lam, g, s, dg, ds)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            reps = 3
            for _ in range(reps):
                c64.rhs(0, lam, g, s, dg, ds)
            torch.cuda.synchronize()
            r64 = reps / (time.perf_counter() - t0)
        fp64_gpu = {"value": r64, "unit": UNIT, "what": "plain FP64 GPU rhs on the same state",
                    "speedup_split_vs_fp64": (1e3 / sum(ph)) / r64}

    # the same flows computing every transfer (no reversal reduction)
    every = None
    if reduced and rank == 0 and world == 1 and not args.headline_only:
        with frg.Context([w], precision=prec, channel_mask=(mask & ~frg.REVERSAL) | frg.NO_REVERSAL) as cf:
            if prec != "fp64":
                cf.autotune()
            ev_f = 0
            cf.set_state(0, bare, None, w.Lambda0)
            cf.flow()
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for _ in range(3):
                cf.set_state(0, bare, None, w.Lambda0)
                st = cf.flow()[0]
                ev_f += st.rhs_evals
            f1.record(stream)
            torch.cuda.synchronize()
            every = {"value": ev_f / (f0.elapsed_time(f1) / 1e3), "unit": UNIT, "flows": 3,
                     "what": "the same whole flows with FRG_NO_REVERSAL (every transfer of every channel)"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[prec], "data": "synthetic",
            "config": {"workload": w.name + ("+tails" if args.tails else "") + ("+reversal" if args.reversal else ""),
                       "crossing_reduction": "asserted (FRG_CROSSING; flows from the bare vertex)"
                       if args.crossing and prec != "fp64" else "off",
                       "reversal_reduction": ("asserted (FRG_REVERSAL)" if args.reversal else
                                              "automatic (states reversal-symmetric)" if reduced else "off"),
                       "N_f": N, "U": w.U, "T": w.T,
                       "eps_d": w.eps_d, "channel_mask": mask,
                       "precision": prec, "rhs_evals_timed": evals, "step_attempts_timed": attempts,
                       "ms_per_step_attempt": ms_max / max(attempts, 1),
                       "flows_per_s": world * args.steps / (ms_max / 1e3),
                       "step": "one whole flow from the bare vertex, Lambda 1e3 -> 1e-3 (every step attempt: "
                               "6 rhs + stage sums + error norm + controller)",
                       "l2": "working set > L2 (state, 7 stage derivatives, stage input: %.0f MB)"
                             % ((2 * 16 + 7 * (8 if prec != 'fp64' else 16) + 16) * N ** 3 / 1e6),
                       "parallelism": "replicas" if world > 1 else "single", "autotune": tune},
            "roofline": roof, "e2e": e2e, "gpu_launches": launches, "every_transfer": every,
            "clocks": clk.summary(), "fp64_gpu": fp64_gpu}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(seconds=args.cpu_seconds, mask=mask & 0x1F)
    if rank == 0 and world == 1 and not args.headline_only:
        # the other workloads, each bounded to seconds (not the headline)
        t0 = time.perf_counter()
        line["configs"] = {
            "batch64": measure_batch(prec, warmup=1, steps=3, crossing=args.crossing),
            "siam_N256": measure_n256(prec, warmup=3, steps=20),
            "siam_N64": measure_n64(False, warmup=1, steps=3, with_oracle=not args.no_oracle),
        }
        line["configs"]["wall_s"] = time.perf_counter() - t0
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def reset_flows(ctx, pts, torch):
    """Every point back to the bare vertex, Sigma = 0 at Lambda0."""
    for i, p in enumerate(pts):
        g = torch.full((p.N,) * 3, p.U, dtype=torch.complex128, device="cuda")
        ctx.set_state(i, g, None, p.Lambda0)


def host_link(torch, nbytes, reps=6):
    """Copy-engine bandwidth of the host link for one call's bytes (pinned host
    buffers, CUDA events): each direction alone, and both at once on two
    streams, as the pipelined host-buffer calls overlap them."""
    hin = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    hout = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    din = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    dout = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def timed(fn, stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            fn()
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
        return e0, e1

    def gbs(ev):
        return reps * nbytes / (ev[0].elapsed_time(ev[1]) / 1e3) / 1e9

    h2d = timed(lambda: din.copy_(hin, non_blocking=True), s1)
    torch.cuda.synchronize()
    d2h = timed(lambda: hout.copy_(dout, non_blocking=True), s2)
    torch.cuda.synchronize()
    out = {"h2d_gbs": gbs(h2d), "d2h_gbs": gbs(d2h)}
    a = timed(lambda: din.copy_(hin, non_blocking=True), s1)
    b = timed(lambda: hout.copy_(dout, non_blocking=True), s2)
    torch.cuda.synchronize()
    out.update({"h2d_concurrent_gbs": gbs(a), "d2h_concurrent_gbs": gbs(b), "bytes": nbytes,
                "what": "pinned copies of one call's bytes, each direction alone and both at once on two streams"})
    return out


def measure_batch(prec, warmup, steps, fp64_baseline=True, crossing=False):
    """64 points, uneven N_f, one context: full flows per second (from the bare
    vertex, so the split precisions may assert the crossing reduction)."""
    import torch
    from paper_1510_07799_gb300 import build as cuda_build
    cuda_build.build()
    from paper_1510_07799_gb300 import frg, inputs
    pts = inputs.batch_points()
    ctx = frg.Context(pts, precision=prec, channel_mask=frg.CH_ALL | (frg.CROSSING if crossing else 0))
    tune = ctx.autotune() if prec != "fp64" else None
    stream = torch.cuda.current_stream()
    times, evals = [], []
    for k in range(warmup + steps):
        reset_flows(ctx, pts, torch)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = ctx.flow()
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= warmup:
            times.append(e0.elapsed_time(e1) / 1e3)
            evals.append(sum(x.rhs_evals for x in st))
    ctx.close()
    tb = sum(times) / len(times)
    # 64 sequential plain-FP64 GPU flows, one context each
    t64, ev64 = 0.0, 0
    if fp64_baseline:
        for p in pts:
            with frg.Context([p], precision="fp64") as c:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st = c.flow()[0]
                torch.cuda.synchronize()
                t64 += time.perf_counter() - t0
                ev64 += st.rhs_evals
    line = {"metric": "full flows/s, 64-point batch (N_f 32/48/64/96) in one context", "value": len(pts) / tb,
            "unit": "flows/s", "n_gpus": 1, "steps": steps, "warmup": warmup,
            "ms_per_step": 1e3 * tb, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[prec], "data": "synthetic",
            "config": {"workload": "batch64", "seed": inputs.BATCH_SEED, "points": len(pts),
                       "N_f": {str(n): sum(1 for p in pts if p.N == n) for n in inputs.BATCH_SIZES},
                       "precision": prec, "step": "one full flow of all 64 points (Lambda 1e3 -> 1e-3)",
                       "rhs_evals_per_step": int(sum(evals) / len(evals)), "autotune": tune},
            "fp64_sequential": None if not fp64_baseline else {
                "value": len(pts) / t64, "unit": "flows/s", "rhs_evals": ev64,
                "what": "64 plain-FP64 GPU flows, one context each, one after the other"}}
    if fp64_baseline:
        line["speedup_vs_fp64_sequential"] = line["value"] / line["fp64_sequential"]["value"]
    return line


def run_batch(args):
    print(json.dumps(measure_batch(args.precision, args.warmup, args.steps, not args.no_fp64_baseline,
                                   args.crossing)))
    return 0


def measure_n256(prec, warmup, steps, rhs_reps=5):
    """The largest single flow: rhs evaluations per second at N_f = 256, and
    the error of the split rhs against the FP64 GPU path on the same state."""
    import numpy as np
    import torch
    from paper_1510_07799_gb300 import build as cuda_build
    cuda_build.build()
    from paper_1510_07799_gb300 import frg, inputs
    w = inputs.SIAM_N256
    ctx = frg.Context([w], precision=prec)
    tune = ctx.autotune() if prec != "fp64" else None
    stream = torch.cuda.current_stream()
    ctx.advance(warmup)
    torch.cuda.synchronize()
    st0 = ctx.stats()[0]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        e0.record(stream)
        ctx.advance(steps)
        e1.record(stream)
        torch.cuda.synchronize()
    st1 = ctx.stats()[0]
    ms = e0.elapsed_time(e1)
    evals = st1.rhs_evals - st0.rhs_evals
    g, s, lam, _ = ctx.get_state(0)
    dg, ds = torch.empty_like(g), torch.empty_like(s)
    for _ in range(2):
        ctx.rhs_timed(0, lam, g, s, dg, ds)
    ph = np.array([ctx.rhs_timed(0, lam, g, s, dg, ds) for _ in range(rhs_reps)]).mean(axis=0)
    ctx.close()
    with frg.Context([w], precision="fp64") as c64:
        fg, fs = torch.empty_like(g), torch.empty_like(s)
        c64.rhs(0, lam, g, s, fg, fs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c64.rhs(0, lam, g, s, fg, fs)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0

    def nrel(a, b):
        return float((a - b).abs().max() / b.abs().max())

    pk = peaks()
    macs = contraction_macs(w.N)
    bf = prec == "bf16x3"
    tc_peak = pk["bf16_tflops"] * (1.0 if bf else 0.5)
    achieved = 8.0 * macs / (ph[2] * 1e-3) / 1e12
    line = {"metric": "vertex-rhs evals/s at N_f=256 (largest single flow)", "value": evals / (ms / 1e3),
            "unit": UNIT, "n_gpus": 1, "steps": steps, "warmup": warmup,
            "ms_per_step": ms / max(1, (st1.accepted + st1.rejected) - (st0.accepted + st0.rejected)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[prec],
            "data": "synthetic",
            "config": {"workload": w.name, "N_f": w.N, "U": w.U, "T": w.T, "eps_d": w.eps_d,
                       "precision": prec, "rhs_evals_timed": evals, "autotune": tune},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": tc_peak, "unit": "TFLOP/s",
                         "frac": achieved / tc_peak, "kernel": "tcgen05 channel contractions of one rhs",
                         "executed_tflops": executed_tensor_flops(w.N, products=6 if bf else 3) / (ph[2] * 1e-3) / 1e12,
                         "peak_source": ("%s bf16 burst" if bf else "%s bf16 burst x 0.5") % pk["_source"],
                         "phases_ms": {"bubble_and_sigma": ph[0], "regather": ph[1], "contraction": ph[2],
                                       "combine": ph[3]}},
            "error_vs_fp64_gpu": {"gamma": nrel(dg, fg), "sigma": nrel(ds, fs),
                                  "state": "flow state at Lambda=%.4g after %d warm-up steps" % (lam, warmup)},
            "fp64_gpu": {"value": 1.0 / t64, "unit": UNIT,
                         "speedup_split_vs_fp64": (1e3 / sum(ph)) * t64},
            "clocks": clk.summary()}
    return line


def run_n256(args):
    print(json.dumps(measure_n256(args.precision, args.warmup, args.steps, args.rhs_reps)))
    return 0


def measure_n64(iflow, warmup, steps, with_oracle=True):
    """Full flows per second at N_f = 64: plain FP64 and 3xTF32 on the GPU,
    and the FP64 oracle on the host cores; parity of the final vertex."""
    import numpy as np
    import torch
    from paper_1510_07799_gb300 import build as cuda_build
    cuda_build.build()
    from paper_1510_07799_gb300 import frg, inputs
    w = inputs.SIAM_N64_IFLOW if iflow else inputs.SIAM_N64
    res = {}
    finals = {}
    for prec in ("fp64", "3xtf32"):
        times, evals = [], []
        for k in range(warmup + steps):
            with frg.Context([w], precision=prec) as ctx:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st = ctx.flow()[0]
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                if k >= warmup:
                    times.append(dt)
                    evals.append(st.rhs_evals)
                g, s, _, _ = ctx.get_state(0)
                finals[prec] = g.cpu().numpy()
        t = sum(times) / len(times)
        res[prec] = {"flows_per_s": 1.0 / t, "rhs_evals_per_s": evals[-1] / t, "rhs_evals": evals[-1]}
    scheme = "interaction flow, Lambda = 1/g 1e12 -> 1" if w.cutoff else "Omega scheme, Lambda 1e3 -> 1e-3"
    line = {"metric": "full flows/s at N_f=64 (off particle-hole symmetry%s)" % (", interaction flow" if w.cutoff else ""),
            "value": res["fp64"]["flows_per_s"],
            "unit": "flows/s", "n_gpus": 1, "steps": steps, "warmup": warmup,
            "ms_per_step": 1e3 / res["fp64"]["flows_per_s"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "N_f": w.N, "U": w.U, "T": w.T, "eps_d": w.eps_d,
                       "cutoff": w.cutoff, "step": "one full flow (%s, rtol 1e-8)" % scheme},
            "fp64_gpu": res["fp64"], "tf32x3_gpu": res["3xtf32"],
            "tf32x3_vs_fp64_gamma": float(np.max(np.abs(finals["3xtf32"] - finals["fp64"]))
                                          / np.max(np.abs(finals["fp64"])))}
    if with_oracle:
        import oracle as orc
        from oracle import build as oracle_build
        oracle_build.build()
        m = orc.Model(U=w.U, T=w.T, eps_d=w.eps_d, Delta=w.Delta, N=w.N, cutoff=w.cutoff)
        t0 = time.perf_counter()
        g0, _, st0 = orc.flow(m, Lambda0=w.Lambda0, Lambda_f=w.Lambda_f, rtol=w.rtol, atol=w.atol)
        dt = time.perf_counter() - t0
        line["oracle_cpu"] = {"flows_per_s": 1.0 / dt, "rhs_evals_per_s": st0.rhs_evals / dt,
                              "rhs_evals": int(st0.rhs_evals), "cores": orc.max_threads(), "kind": "oracle",
                              "sample": "one full flow"}
        line["fp64_vs_oracle_gamma"] = float(np.max(np.abs(finals["fp64"] - g0)) / np.max(np.abs(g0)))
    return line


def run_n64(args):
    print(json.dumps(measure_n64(args.workload == "siam_N64_iflow", args.warmup, args.steps, not args.no_oracle)))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default=None, choices=list(DTYPES))
    ap.add_argument("--rhs-reps", type=int, default=5)
    ap.add_argument("--e2e-reps", type=int, default=12)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="siam_N128",
                    choices=["siam_N128", "batch64", "siam_N256", "siam_N64", "siam_N64_iflow"])
    ap.add_argument("--no-oracle", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="only the N_f = 128 headline (no batch64 / N_f = 256 / N_f = 64 figures under 'configs')")
    ap.add_argument("--no-fp64-baseline", action="store_true")
    ap.add_argument("--tails", action="store_true",
                    help="headline workload with the frequency-box tail option (channel_mask | FRG_TAILS)")
    ap.add_argument("--no-reversal", action="store_true",
                    help="flows compute every transfer (channel_mask | FRG_NO_REVERSAL)")
    ap.add_argument("--crossing", action="store_true",
                    help="headline workload with the crossing reduction of the products (channel_mask | "
                         "FRG_CROSSING; the flows start from the crossing-symmetric bare vertex)")
    ap.add_argument("--reversal", action="store_true",
                    help="headline workload with the frequency-reversal reduction (channel_mask | FRG_REVERSAL): "
                         "the contraction computes half of the transfers of each channel")
    args = ap.parse_args()
    args.precision_explicit = args.precision is not None
    if args.precision is None:
        args.precision = "3xtf32"
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch(args)
    if args.workload == "siam_N256":
        return run_n256(args)
    if args.workload in ("siam_N64", "siam_N64_iflow"):
        return run_n64(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
