"""GPU parity of the split-precision tensor-core path (tcgen05) against the FP64
CPU oracle, through the C ABI.

Tolerance: the contraction operands are the vertex rounded to FP32 times the
bubble weights, split into TF32 hi/lo or three BF16 slices, with FP32
accumulation in TMEM; the normwise relative error of one rhs evaluation is
bounded by RHS_TOL below, and of a full flow by FLOW_TOL (the 1e-6 acceptance
bar for the mixed form)."""
import json
import os

import numpy as np
import pytest

import flow_ref
import oracle
import rhs_bar
from paper_1510_07799_gb300 import frg, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
# One rhs: 3xTF32 errors grow with the contraction length (the tensor core's
# FP32 accumulator does not round to nearest; the cross products have their own
# accumulator and the k-chunks are fed in increasing magnitude), BF16x3 slices on
# a per-transfer fixed grid (absolute error 2^-24 of the operand bound).
# The 3xTF32 bar is the 1e-6 acceptance bar of the mixed form itself.
RHS_TOL = {frg.TF32X3: 1e-6, frg.BF16X3: 5e-5}
FLOW_TOL = {frg.TF32X3: 1e-6, frg.BF16X3: 1e-6}
PRECS = [frg.TF32X3, frg.BF16X3]


def nrel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def model(w):
    return oracle.Model(U=w.U, T=w.T, eps_d=w.eps_d, Delta=w.Delta, N=w.N)


def gpu_rhs(ctx, point, Lam, V, sig):
    g = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    s = torch.from_numpy(np.ascontiguousarray(sig)).cuda()
    dg = torch.full_like(g, complex(np.nan, np.nan))
    ds = torch.full_like(s, complex(np.nan, np.nan))
    ctx.rhs(point, Lam, g, s, dg, ds)
    torch.cuda.synchronize()
    return dg.cpu().numpy(), ds.cpu().numpy()


@pytest.mark.parametrize("crossing", [True, False])
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [2, 4, 16, 34, 64, 100])
@pytest.mark.parametrize("mask", [0xF, 0x1, 0x2, 0x4])
def test_split_rhs_matches_oracle(N, mask, prec, crossing):
    """Every channel mask, on vertices with and without crossing symmetry: the
    split path reads every operand of the three channel sums as the entry the
    sum names (the direct channel's V(k1,p,p-t) and V(p-t,k2,k2-t) from the
    skewed layout), so it is the same function of the vertex as the oracle's
    literal sums.  Error against the whole rhs of the same input (rhs_bar)."""
    w = inputs.Workload("t", N=N, U=1.7, T=0.03, eps_d=-0.85 + 0.3)
    V = inputs.random_vertex(N, w.U, seed=N + (0 if crossing else 500), crossing=crossing)
    sig = inputs.random_sigma(N, seed=100 + N)
    with frg.Context([w], precision=prec, channel_mask=mask) as ctx:
        for Lam in (0.01, 0.4, 7.0):
            dg, ds = gpu_rhs(ctx, 0, Lam, V, sig)
            rg, rs = oracle.rhs(model(w), Lam, V, sig, mask=mask)
            ng, _ = rhs_bar.full_norms(model(w), Lam, V, sig, key=("split", N, crossing))
            e = rhs_bar.err(dg, rg, ng)
            print("prec=%d N=%d mask=%x crossing=%d Lam=%g err=%.3e (of the channel subset itself: %.3e)" % (
                prec, N, mask, crossing, Lam, e, nrel(dg, rg)))
            assert e < RHS_TOL[prec]


@pytest.mark.parametrize("crossing", [True, False])
@pytest.mark.parametrize("prec", PRECS)
def test_split_rhs_full_size_sampled_entries(prec, crossing):
    w = inputs.SIAM_N128
    V = inputs.random_vertex(w.N, w.U, seed=11, crossing=crossing)
    sig = inputs.random_sigma(w.N, seed=12, amp=0.05)
    Lam = 0.02
    with frg.Context([w], precision=prec) as ctx:
        dg, ds = gpu_rhs(ctx, 0, Lam, V, sig)
    rng = np.random.default_rng(5)
    idx = rng.integers(0, w.N, (3000, 3))
    idx[:4] = [[0, 0, 0], [w.N - 1] * 3, [w.N // 2] * 3, [0, w.N - 1, 0]]
    ref = oracle.rhs_entries(model(w), Lam, V, sig, idx)
    got = dg[idx[:, 0], idx[:, 1], idx[:, 2]]
    e = nrel(got, ref)
    print("prec=%d N=128 crossing=%d sampled rel=%.3e" % (prec, crossing, e))
    assert e < RHS_TOL[prec]


_FP64_FLOWS = {}


def fp64_gpu_flow(name):
    """Final vertex and self-energy of the plain FP64 GPU flow of a workload
    (the path that matches the oracle's flows within 1e-10 with the oracle's
    own step sequence): the whole-vertex reference where the oracle's final
    vertex is stored only on a sample (grids above 16)."""
    if name not in _FP64_FLOWS:
        with frg.Context([inputs.WORKLOADS[name]]) as ctx:
            st = ctx.flow()[0]
            g, s, _, _ = ctx.get_state(0)
        assert st.status == 0 and st.done == 1
        _FP64_FLOWS[name] = (g.cpu().numpy(), s.cpu().numpy())
    return _FP64_FLOWS[name]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", ["siam_N16_U1_T0.05_ph", "siam_N64_U2_T0.01_asym0.5",
                                  "siam_N128_U3_T0.005_ph"])
def test_split_flow_matches_oracle_reference(name, prec):
    """Final vertex, self-energy and effective interaction of a whole flow:
    against the oracle (every entry at N = 16, its stored sample above), and at
    N = 64 and 128 every entry against the plain FP64 GPU flow."""
    with open(os.path.join(HERE, "golden", "oracle_flow_%s.json" % name)) as f:
        ref = json.load(f)
    w = inputs.WORKLOADS[name]
    with frg.Context([w], precision=prec) as ctx:
        st = ctx.flow()[0]
        g, s, lam, _ = ctx.get_state(0)
        obs = ctx.observables(0)
    assert st.status == 0 and st.done == 1
    g = g.cpu().numpy()
    if w.N > 16:
        fg, fs = fp64_gpu_flow(name)
        e_all = nrel(g, fg)
        print("prec=%d flow %s every entry vs the FP64 GPU flow: gamma %.3e sigma %.3e" % (
            prec, name, e_all, nrel(s.cpu().numpy(), fs)))
        assert e_all < FLOW_TOL[prec] and nrel(s.cpu().numpy(), fs) < FLOW_TOL[prec]
    eg = flow_ref.gamma_error(g, ref)
    rsig = np.array(ref["sigma_re"]) + 1j * np.array(ref["sigma_im"])
    es = nrel(s.cpu().numpy(), rsig)
    eu = abs(obs["U_eff"] - complex(*ref["observables"]["U_eff"])) / abs(complex(*ref["observables"]["U_eff"]))
    print("prec=%d flow %s errors gamma %.3e sigma %.3e ueff %.3e evals %d vs %d" % (
        prec, name, eg, es, eu, st.rhs_evals, ref["stats"]["rhs_evals"]))
    assert eg < FLOW_TOL[prec] and es < FLOW_TOL[prec] and eu < FLOW_TOL[prec]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("mask", [0x8, 0x8 | frg.TAILS])
@pytest.mark.parametrize("rev", [0, frg.NO_REVERSAL])
def test_split_flow_without_vertex_channels_matches_oracle(prec, mask, rev):
    """No vertex channel: the self-energy flows alone (with the tails the
    vertex also takes the tail constants).  The step control of the split
    paths still takes the embedded error estimate (the scatter-add that writes
    the vertex derivative of k7 completes it), so the flow matches the
    oracle's within the flow bar with about the oracle's number of steps."""
    w = inputs.Workload("t", N=16, U=1.3, T=0.04, eps_d=-0.65 + 0.25)
    rg, rs, rst = oracle.flow(model(w), Lambda0=w.Lambda0, Lambda_f=w.Lambda_f, rtol=w.rtol, atol=w.atol,
                              mask=mask)
    with frg.Context([w], precision=prec, channel_mask=mask | rev) as ctx:
        st = ctx.flow()[0]
        g, s, _, _ = ctx.get_state(0)
    print("prec=%d mask=%#x steps %d+%d vs oracle %d+%d" % (prec, mask, st.accepted, st.rejected, rst.accepted,
                                                             rst.rejected))
    assert st.status == 0 and st.done == 1
    assert nrel(g.cpu().numpy(), rg) < FLOW_TOL[prec] and nrel(s.cpu().numpy(), rs) < FLOW_TOL[prec]
    assert abs(st.accepted - rst.accepted) <= max(2, rst.accepted // 10)


@pytest.mark.parametrize("prec", [frg.FP64] + PRECS)
@pytest.mark.parametrize("N", [2, 16, 100])
def test_zero_interaction_flows_nothing(prec, N):
    """U = 0 (a degenerate case): every diagram and the self-energy rhs vanish,
    so the whole flow keeps the vertex and the self-energy exactly zero in
    every precision (the split slicing of an all-zero operand included)."""
    w = inputs.Workload("u0", N=N, U=0.0, T=0.05, eps_d=0.2)
    with frg.Context([w], precision=prec) as ctx:
        st = ctx.flow()[0]
        g, s, lam, _ = ctx.get_state(0)
    assert st.status == 0 and st.done == 1 and abs(lam / w.Lambda_f - 1.0) < 1e-12
    assert torch.count_nonzero(g).item() == 0 and torch.count_nonzero(s).item() == 0


@pytest.mark.parametrize("prec", PRECS)
def test_split_batched_points_equal_single_point_runs(prec):
    """Uneven grid sizes in one context: every tile's sum runs in a fixed order
    whichever CTA the schedule gives it to, so each point's flow is bitwise the
    flow of a context that holds only that point."""
    pts = [inputs.Workload("a", N=16, U=1.0, T=0.05, eps_d=-0.5),
           inputs.Workload("b", N=34, U=2.5, T=0.02, eps_d=-1.0),
           inputs.Workload("c", N=48, U=0.7, T=0.08, eps_d=0.1)]
    with frg.Context(pts, precision=prec) as ctx:
        stb = ctx.flow()
        batched = [ctx.get_state(i)[:2] for i in range(len(pts))]
    for i, w in enumerate(pts):
        with frg.Context([w], precision=prec) as ctx:
            st = ctx.flow()[0]
            g, s, _, _ = ctx.get_state(0)
        assert torch.equal(g, batched[i][0]) and torch.equal(s, batched[i][1])
        assert st.rhs_evals == stb[i].rhs_evals and st.accepted == stb[i].accepted


def test_split_batched_rhs_matches_oracle():
    """One rhs of each point of a mixed-size context against the oracle."""
    pts = [inputs.Workload("a", N=32, U=1.3, T=0.03, eps_d=-0.2),
           inputs.Workload("b", N=48, U=3.1, T=0.011, eps_d=-1.9),
           inputs.Workload("c", N=96, U=0.6, T=0.07, eps_d=-0.5)]
    with frg.Context(pts, precision=frg.TF32X3) as ctx:
        for i, w in enumerate(pts):
            V = inputs.random_vertex(w.N, w.U, seed=40 + i)
            sig = inputs.random_sigma(w.N, seed=50 + i)
            dg, ds = gpu_rhs(ctx, i, 0.05, V, sig)
            rg, rs = oracle.rhs(model(w), 0.05, V, sig)
            assert nrel(dg, rg) < RHS_TOL[frg.TF32X3] and nrel(ds, rs) < RHS_TOL[frg.TF32X3]


def test_split_rhs_largest_grid_n256():
    """N = 256 (the largest grid): both split precisions against the plain FP64
    GPU path on the whole rhs, and against the oracle on sampled entries."""
    w = inputs.SIAM_N256
    V = inputs.random_vertex(w.N, w.U, seed=21)
    sig = inputs.random_sigma(w.N, seed=22, amp=0.05)
    Lam = 0.01
    with frg.Context([w]) as ctx:
        fg, fs = gpu_rhs(ctx, 0, Lam, V, sig)
    rng = np.random.default_rng(6)
    idx = rng.integers(0, w.N, (2000, 3))
    idx[:4] = [[0, 0, 0], [w.N - 1] * 3, [w.N // 2] * 3, [0, w.N - 1, 0]]
    ref = oracle.rhs_entries(model(w), Lam, V, sig, idx)
    assert nrel(fg[idx[:, 0], idx[:, 1], idx[:, 2]], ref) < 1e-12
    for prec in PRECS:
        with frg.Context([w], precision=prec) as ctx:
            dg, ds = gpu_rhs(ctx, 0, Lam, V, sig)
        e_full = nrel(dg, fg)
        e_samp = nrel(dg[idx[:, 0], idx[:, 1], idx[:, 2]], ref)
        print("prec=%d N=256 vs fp64 gpu %.3e, vs oracle sampled %.3e, sigma %.3e" % (
            prec, e_full, e_samp, nrel(ds, fs)))
        # the split path's self-energy sums the FP32 stage input in FP64
        assert e_full < RHS_TOL[prec] and e_samp < RHS_TOL[prec] and nrel(ds, fs) < RHS_TOL[prec]


def test_autotuned_plan_keeps_the_results():
    """The autotuner only redistributes the same per-element sums: a tuned
    context's rhs and flow stay within the split bars of the oracle."""
    pts = [inputs.Workload("a", N=32, U=1.3, T=0.03, eps_d=-0.2),
           inputs.Workload("b", N=96, U=2.2, T=0.02, eps_d=-1.4)]
    with frg.Context(pts, precision=frg.TF32X3) as ctx:
        tune = ctx.autotune()
        assert tune["candidates"] >= 3 and tune["nt_cap"] in (32, 64, 128) and tune["ms"] > 0
        for i, w in enumerate(pts):
            V = inputs.random_vertex(w.N, w.U, seed=60 + i)
            sig = inputs.random_sigma(w.N, seed=70 + i)
            dg, ds = gpu_rhs(ctx, i, 0.03, V, sig)
            rg, rs = oracle.rhs(model(w), 0.03, V, sig)
            assert nrel(dg, rg) < RHS_TOL[frg.TF32X3] and nrel(ds, rs) < RHS_TOL[frg.TF32X3]
        st = ctx.flow()
        assert all(s.status == 0 and s.done for s in st)


@pytest.mark.parametrize("prec", [frg.FP64, frg.TF32X3])
def test_pipelined_host_calls_equal_synchronous_calls(prec):
    """frg_rhs_host_async: several evaluations in flight (two device slots, two
    copy streams) give bitwise the results of one-by-one frg_rhs_host calls."""
    w = inputs.Workload("t", N=24, U=1.6, T=0.03, eps_d=-0.4)
    ins = [(inputs.random_vertex(w.N, w.U, seed=90 + i), inputs.random_sigma(w.N, seed=95 + i), 0.02 + 0.1 * i)
           for i in range(5)]
    with frg.Context([w], precision=prec) as ctx:
        ref = []
        for V, sig, lam in ins:
            og, os_ = np.empty_like(V), np.empty_like(sig)
            ctx.rhs_host(0, lam, V, sig, og, os_)
            ref.append((og, os_))
        outs = [(np.full_like(V, np.nan), np.full_like(sig, np.nan)) for V, sig, _ in ins]
        for (V, sig, lam), (og, os_) in zip(ins, outs):
            ctx.rhs_host_async(0, lam, V, sig, og, os_)
        ctx.sync()
    for (og, os_), (rg, rs) in zip(outs, ref):
        assert np.array_equal(og, rg) and np.array_equal(os_, rs)
