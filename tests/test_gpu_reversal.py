"""GPU parity of the frequency-reversal reduction (channel_mask | FRG_REVERSAL)
against the FP64 CPU oracle, through the C ABI.

With the bit set the split contraction computes the transfers m <= N - 1 of
each channel and the scatter-add takes the others from the mirrored entries,
which is exact for reversal-symmetric states (every flow from the bare
vertex).  Tolerances are those of the split paths."""
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
RHS_TOL = {frg.FP64: 1e-12, frg.TF32X3: 1e-6, frg.BF16X3: 5e-5}
FLOW_TOL = 1e-6
REV = frg.REVERSAL


def nrel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def model(w):
    return oracle.Model(U=w.U, T=w.T, eps_d=w.eps_d, Delta=w.Delta, N=w.N)


def symmetric_state(N, U, seed):
    V = inputs.random_vertex(N, U, seed=seed)
    V = 0.5 * (V + np.conj(V[::-1, ::-1, ::-1]))
    s = inputs.random_sigma(N, seed=seed + 1)
    return V, 0.5 * (s + np.conj(s[::-1]))


def gpu_rhs(ctx, Lam, V, sig):
    g = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    s = torch.from_numpy(np.ascontiguousarray(sig)).cuda()
    dg = torch.full_like(g, complex(np.nan, np.nan))
    ds = torch.full_like(s, complex(np.nan, np.nan))
    ctx.rhs(0, Lam, g, s, dg, ds)
    torch.cuda.synchronize()
    return dg.cpu().numpy(), ds.cpu().numpy()


@pytest.mark.parametrize("prec", [frg.TF32X3, frg.BF16X3, frg.FP64])
@pytest.mark.parametrize("N", [2, 4, 16, 34, 100])
@pytest.mark.parametrize("mask", [0xF, 0x1, 0x2, 0x4, 0xF | frg.TAILS])
def test_reversal_rhs_matches_oracle(prec, N, mask):
    """The reduced rhs is within the path's own rhs bar of the oracle, like the
    same path computing every transfer (FP64: normwise against the oracle's rhs
    with the same mask; split precisions: against the whole rhs of the same
    input and options, rhs_bar)."""
    if N == 100 and prec == frg.FP64:
        pytest.skip("the FP64 path computes every transfer; covered at smaller N")
    w = inputs.Workload("t", N=N, U=1.7, T=0.03, eps_d=-0.85 + 0.3)
    V, sig = symmetric_state(N, w.U, seed=7 * N)
    with frg.Context([w], precision=prec, channel_mask=mask | REV) as ctx, \
            frg.Context([w], precision=prec, channel_mask=mask) as full:
        for Lam in (0.01, 0.4, 7.0):
            dg, ds = gpu_rhs(ctx, Lam, V, sig)
            fg, fs = gpu_rhs(full, Lam, V, sig)
            rg, rs = oracle.rhs(model(w), Lam, V, sig, mask=mask)
            ng, ns = (np.max(np.abs(rg)), np.max(np.abs(rs))) if prec == frg.FP64 else \
                rhs_bar.full_norms(model(w), Lam, V, sig, extra_mask=mask & frg.TAILS,
                                   key=("reversal", N))
            e, ef = rhs_bar.err(dg, rg, ng), rhs_bar.err(fg, rg, ng)
            print("reversal prec=%d N=%d mask=%x Lam=%g err=%.3e (every transfer: %.3e)" % (
                prec, N, mask, Lam, e, ef))
            assert e < RHS_TOL[prec] and ef < RHS_TOL[prec], (Lam, e, ef)
            assert rhs_bar.err(ds, rs, ns) < RHS_TOL[prec]


@pytest.mark.parametrize("prec", [frg.TF32X3, frg.BF16X3])
def test_reversal_output_is_exactly_symmetric(prec):
    """Without tails every mirrored entry is the exact conjugate of the
    computed one (same summation order on both sides)."""
    N = 34
    w = inputs.Workload("t", N=N, U=1.7, T=0.03, eps_d=-0.85 + 0.3)
    V, sig = symmetric_state(N, w.U, seed=3)
    with frg.Context([w], precision=prec, channel_mask=0xF | REV) as ctx:
        dg, _ = gpu_rhs(ctx, 0.4, V, sig)
    assert np.array_equal(dg, np.conj(dg[::-1, ::-1, ::-1]))


@pytest.mark.parametrize("name", ["siam_N16_U1_T0.05_ph", "siam_N64_U2_T0.01_asym0.5",
                                  "siam_N128_U3_T0.005_ph"])
def test_reversal_flow_matches_oracle_reference(name):
    with open(os.path.join(HERE, "golden", "oracle_flow_%s.json" % name)) as f:
        ref = json.load(f)
    w = inputs.WORKLOADS[name]
    with frg.Context([w], precision=frg.TF32X3, channel_mask=0xF | REV) as ctx:
        st = ctx.flow()[0]
        g, s, _, _ = ctx.get_state(0)
        obs = ctx.observables(0)
    assert st.status == 0 and st.done == 1
    g = g.cpu().numpy()
    # the state stays exactly reversal-symmetric along the flow
    assert np.array_equal(g, np.conj(g[::-1, ::-1, ::-1]))
    eg = flow_ref.gamma_error(g, ref)
    rsig = np.array(ref["sigma_re"]) + 1j * np.array(ref["sigma_im"])
    es = nrel(s.cpu().numpy(), rsig)
    ru = complex(*ref["observables"]["U_eff"])
    eu = abs(obs["U_eff"] - ru) / abs(ru)
    print("reversal flow %s errors gamma %.3e sigma %.3e ueff %.3e evals %d vs %d" % (
        name, eg, es, eu, st.rhs_evals, ref["stats"]["rhs_evals"]))
    assert eg < FLOW_TOL and es < FLOW_TOL and eu < FLOW_TOL


def test_reversal_in_a_mixed_size_batch_equals_single_point_runs():
    pts = [inputs.Workload("a", N=16, U=1.2, T=0.04, eps_d=-0.6 + 0.2),
           inputs.Workload("b", N=34, U=2.0, T=0.03, eps_d=-1.0 - 0.4)]
    with frg.Context(pts, precision=frg.TF32X3, channel_mask=0xF | REV) as ctx:
        stb = ctx.advance(4)
        batched = [ctx.get_state(i)[:2] for i in range(len(pts))]
    for i, w in enumerate(pts):
        with frg.Context([w], precision=frg.TF32X3, channel_mask=0xF | REV) as ctx:
            st = ctx.advance(4)[0]
            g, s, _, _ = ctx.get_state(0)
        assert torch.equal(g, batched[i][0]) and torch.equal(s, batched[i][1])
        assert st.rhs_evals == stb[i].rhs_evals


@pytest.mark.parametrize("cutoff", [0, 1])
def test_all_options_together_match_the_fp64_path(cutoff):
    """3xTF32 with the reversal reduction and the tails, on either cutoff,
    against the FP64 path with the tails (itself at 1e-15 of the oracle):
    a full N = 16 flow off particle-hole symmetry within the 1e-6 bar."""
    kw = dict(Lambda0=1e12, Lambda_f=1.0) if cutoff else {}
    w = inputs.Workload("t", N=16, U=1.0, T=0.05, eps_d=-0.5 + 0.3, cutoff=cutoff, **kw)
    with frg.Context([w], precision=frg.FP64, channel_mask=0xF | frg.TAILS) as c64:
        st64 = c64.flow()[0]
        g64, s64, _, _ = c64.get_state(0)
    with frg.Context([w], precision=frg.TF32X3, channel_mask=0xF | frg.TAILS | REV) as c:
        st = c.flow()[0]
        g, s, _, _ = c.get_state(0)
    assert st64.status == 0 and st.status == 0
    assert nrel(g.cpu().numpy(), g64.cpu().numpy()) < FLOW_TOL
    assert nrel(s.cpu().numpy(), s64.cpu().numpy()) < FLOW_TOL
    gn = g.cpu().numpy()
    assert nrel(gn, np.conj(gn[::-1, ::-1, ::-1])) < 1e-15


@pytest.mark.parametrize("prec", [frg.TF32X3, frg.BF16X3])
@pytest.mark.parametrize("mask", [0xF, 0x8, 0x8 | frg.TAILS, 0xF | frg.TAILS])
def test_half_storage_flow_matches_full_storage(prec, mask):
    """In a flow the reversal reduction keeps half of the vertex (stage
    derivatives and float-pair state for i1 < N/2) and writes the other half as
    conjugates.  Against the same flow without the reduction (whole storage,
    every transfer): the final state agrees within the split
    paths' bound and is exactly symmetric, also when no vertex channel is on
    (the zero-vertex and tail-addition kernels then write the derivatives)."""
    w = inputs.Workload("t", N=16, U=1.3, T=0.04, eps_d=-0.65 + 0.25)
    with frg.Context([w], precision=prec, channel_mask=mask | REV) as ch, \
            frg.Context([w], precision=prec, channel_mask=mask) as cf:
        sh = ch.flow()[0]
        sf = cf.flow()[0]
        gh, s_h, lh, _ = ch.get_state(0)
        gf, s_f, lf, _ = cf.get_state(0)
    assert sh.status == 0 and sf.status == 0 and sh.done == 1 and sf.done == 1 and lh == lf
    gh, gf = gh.cpu().numpy(), gf.cpu().numpy()
    assert np.array_equal(gh, np.conj(gh[::-1, ::-1, ::-1]))
    assert nrel(gh, gf) < FLOW_TOL and nrel(s_h.cpu().numpy(), s_f.cpu().numpy()) < FLOW_TOL


def test_half_storage_symmetrises_a_state_from_its_canonical_half():
    """A state set with frg_set_state enters a reduced flow through its entries
    with i1 < N/2: an asymmetric state flows like its canonical half's
    symmetric completion."""
    N = 16
    w = inputs.Workload("t", N=N, U=1.0, T=0.05, eps_d=-0.5 + 0.2)
    V, sig = symmetric_state(N, w.U, seed=41)
    V = 0.2 * (V - w.U) + w.U  # a mild perturbation of the bare vertex
    Va = V.copy()
    Va[N // 2:] += 0.05  # break the symmetry in the mirrored half only
    out = []
    for state in (V, Va):
        with frg.Context([w], precision=frg.TF32X3, channel_mask=0xF | REV) as c:
            c.set_state(0, torch.from_numpy(state).cuda(), torch.from_numpy(sig).cuda(), 20.0)
            st = c.advance(3)[0]
            assert st.status == 0 and st.accepted >= 1
            out.append(c.get_state(0)[0].cpu().numpy())
    assert np.array_equal(out[0], out[1])


def _flow_state(prec, mask, w, state=None):
    with frg.Context([w], precision=prec, channel_mask=mask) as ctx:
        if state is not None:
            g, s = state
            ctx.set_state(0, torch.from_numpy(g).cuda(), torch.from_numpy(s).cuda(), w.Lambda0)
        st = ctx.flow()[0]
        g, s, _, _ = ctx.get_state(0)
    assert st.status == 0 and st.done == 1
    return g.cpu().numpy(), s.cpu().numpy(), st


@pytest.mark.parametrize("prec", [frg.TF32X3, frg.BF16X3])
def test_default_flows_use_the_reduction(prec):
    """A split-precision context uses the reversal reduction by default while
    its states are reversal-symmetric: a flow from the bare vertex is bitwise
    the flow of a context that asserts the symmetry (FRG_REVERSAL, half
    storage), stays exactly symmetric, and is within the flow bar of the same
    flow computing every transfer (FRG_NO_REVERSAL)."""
    w = inputs.Workload("t", N=34, U=2.2, T=0.02, eps_d=-1.1 + 0.3)
    g, s, st = _flow_state(prec, frg.CH_ALL, w)
    gf, sf, stf = _flow_state(prec, frg.CH_ALL | REV, w)
    gn, sn, _ = _flow_state(prec, frg.CH_ALL | frg.NO_REVERSAL, w)
    assert np.array_equal(g, gf) and np.array_equal(s, sf) and st.rhs_evals == stf.rhs_evals
    assert np.array_equal(g, np.conj(g[::-1, ::-1, ::-1])) and np.array_equal(s, np.conj(s[::-1]))
    assert nrel(g, gn) < FLOW_TOL and nrel(s, sn) < FLOW_TOL


def test_a_state_without_the_symmetry_switches_the_flows_to_every_transfer():
    """frg_set_state checks the symmetry exactly: an asymmetric state makes the
    context's flows compute every transfer (bitwise the FRG_NO_REVERSAL flow);
    a symmetric state brings the reduction back (bitwise the FRG_REVERSAL
    flow); frg_rhs computes every transfer on any input."""
    w = inputs.Workload("t", N=24, U=1.4, T=0.03, eps_d=-0.7 + 0.2, Lambda0=2.0)
    Va = inputs.random_vertex(w.N, w.U, seed=5, amp=0.1, crossing=False)
    sa = inputs.random_sigma(w.N, seed=6, amp=0.01)
    Vs, ss = symmetric_state(w.N, w.U, seed=7)
    with frg.Context([w], precision=frg.TF32X3) as ctx:
        for state, ref_mask in (((Va, sa), frg.NO_REVERSAL), ((Vs, ss), REV), ((Va, sa), frg.NO_REVERSAL)):
            ctx.set_state(0, torch.from_numpy(state[0]).cuda(), torch.from_numpy(state[1]).cuda(), w.Lambda0)
            st = ctx.flow()[0]
            g, s, _, _ = ctx.get_state(0)
            gr, sr, str_ = _flow_state(frg.TF32X3, frg.CH_ALL | ref_mask, w, state)
            assert st.status == 0 and st.rhs_evals == str_.rhs_evals
            assert np.array_equal(g.cpu().numpy(), gr) and np.array_equal(s.cpu().numpy(), sr)
        # a stand-alone rhs on an asymmetric input: every transfer
        with frg.Context([w], precision=frg.TF32X3, channel_mask=frg.CH_ALL | frg.NO_REVERSAL) as full:
            dg, ds = gpu_rhs(ctx, 0.3, Va, sa)
            fg, fs = gpu_rhs(full, 0.3, Va, sa)
        assert np.array_equal(dg, fg) and np.array_equal(ds, fs)


def test_observables_and_state_of_a_reduced_flow_agree():
    """Under the reduction the seventh stage kernel writes the FP64 state's
    canonical half only; frg_observables and frg_get_state fill in the other
    half first: U_eff (the vertex at i1 = i2 = i3 = N/2, in the mirrored half)
    equals the returned state's entry, with and without a get_state before."""
    w = inputs.Workload("t", N=24, U=1.6, T=0.03, eps_d=-0.8 + 0.2)
    with frg.Context([w], precision=frg.TF32X3) as ctx:
        ctx.advance(5)
        obs = ctx.observables(0)
        g, _, _, _ = ctx.get_state(0)
        obs2 = ctx.observables(0)
    g = g.cpu().numpy()
    h = w.N // 2
    assert obs["U_eff"] == g[h, h, h] and obs2["U_eff"] == g[h, h, h]
    assert np.array_equal(g, np.conj(g[::-1, ::-1, ::-1]))


def test_a_batch_switching_to_every_transfer_keeps_the_other_points_whole():
    """Two points flow under the reduction; an asymmetric state set on the
    second switches the context to every transfer.  The first point continues
    from its whole state (frg_set_state fills in the mirrored half of every
    point first): close to the flow that takes its state at the switch into a
    context computing every transfer (that context starts without the split
    paths' tolerance floors of the error norm, so its steps differ slightly;
    a stale half would be off by the vertex's whole change since the
    start)."""
    w0 = inputs.Workload("a", N=24, U=1.4, T=0.03, eps_d=-0.7 + 0.2)
    w1 = inputs.Workload("b", N=24, U=1.2, T=0.04, eps_d=-0.6 + 0.1)
    Va = inputs.random_vertex(w1.N, w1.U, seed=15, amp=0.1, crossing=False)
    sa = inputs.random_sigma(w1.N, seed=16, amp=0.01)
    with frg.Context([w0, w1], precision=frg.TF32X3) as ctx:
        ctx.advance(6)
        g0, s0, lam0, h0 = ctx.get_state(0)
    with frg.Context([w0, w1], precision=frg.TF32X3) as ctx:
        ctx.advance(6)  # no whole-state read before the switch
        ctx.set_state(1, torch.from_numpy(Va).cuda(), torch.from_numpy(sa).cuda(), w1.Lambda0)
        ctx.advance(5)
        gb, sb, lamb, _ = ctx.get_state(0)
    with frg.Context([w0], precision=frg.TF32X3, channel_mask=frg.CH_ALL | frg.NO_REVERSAL) as ref:
        ref.set_state(0, g0, s0, lam0, h0)
        ref.advance(5)
        gr, sr, lamr, _ = ref.get_state(0)
    eg = nrel(gb.cpu().numpy(), gr.cpu().numpy())
    es = nrel(sb.cpu().numpy(), sr.cpu().numpy())
    print("switch: vertex %.2e, self-energy %.2e, Lambda %.17g vs %.17g" % (eg, es, lamb, lamr))
    assert abs(lamb - lamr) <= 1e-4 * lamr and eg < 1e-7 and es < 1e-4
