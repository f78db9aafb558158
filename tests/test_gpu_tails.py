"""GPU parity of the frequency-box tail option (channel_mask | FRG_TAILS)
against the FP64 CPU oracle, through the C ABI.

The oracle evaluates the tails literally (internal sums over the whole window
of FRG_TAIL_FACTOR * N indices); the library adds them as FP64 constants per
transfer.  Tolerances as for the box-only paths: FP64 rhs 1e-12 and flows
1e-10 with the oracle's step sequence; split paths within their rhs bounds and
flows within 1e-6."""
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
FLOW_TOL = {frg.FP64: 1e-10, frg.TF32X3: 1e-6, frg.BF16X3: 1e-6}


def nrel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def model(w):
    return oracle.Model(U=w.U, T=w.T, eps_d=w.eps_d, Delta=w.Delta, N=w.N)


def gpu_rhs(ctx, Lam, V, sig):
    g = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    s = torch.from_numpy(np.ascontiguousarray(sig)).cuda()
    dg = torch.full_like(g, complex(np.nan, np.nan))
    ds = torch.full_like(s, complex(np.nan, np.nan))
    ctx.rhs(0, Lam, g, s, dg, ds)
    torch.cuda.synchronize()
    return dg.cpu().numpy(), ds.cpu().numpy()


def test_library_constants_match_the_oracle():
    assert frg.TAILS == oracle.MASK_TAILS and frg.TAIL_FACTOR == oracle.TAIL_FACTOR


@pytest.mark.parametrize("prec", [frg.FP64, frg.TF32X3, frg.BF16X3])
@pytest.mark.parametrize("N", [2, 4, 16, 34])
@pytest.mark.parametrize("mask", [0xF, 0x1, 0x2, 0x4, 0x8])
def test_tails_rhs_matches_oracle(prec, N, mask):
    """FP64: normwise against the oracle's rhs with the same mask; split
    precisions: against the whole rhs of the same input (rhs_bar)."""
    w = inputs.Workload("t", N=N, U=1.7, T=0.03, eps_d=-0.85 + 0.3)
    V = inputs.random_vertex(N, w.U, seed=3 * N)
    sig = inputs.random_sigma(N, seed=200 + N)
    m = mask | frg.TAILS
    with frg.Context([w], precision=prec, channel_mask=m) as ctx:
        for Lam in (0.01, 0.4, 7.0):
            dg, ds = gpu_rhs(ctx, Lam, V, sig)
            rg, rs = oracle.rhs(model(w), Lam, V, sig, mask=m)
            ng, ns = (np.max(np.abs(rg)), np.max(np.abs(rs))) if prec == frg.FP64 else \
                rhs_bar.full_norms(model(w), Lam, V, sig, extra_mask=frg.TAILS, key=("tails", N))
            if mask & 7:
                assert rhs_bar.err(dg, rg, ng) < RHS_TOL[prec], (Lam, rhs_bar.err(dg, rg, ng))
            else:
                assert np.max(np.abs(dg)) == 0.0
            if mask & 8:
                assert rhs_bar.err(ds, rs, ns) < RHS_TOL[prec]
            else:
                assert np.max(np.abs(ds)) == 0.0


def test_tails_change_the_rhs():
    """The option is live: with the tails the pp/xph rhs and the self-energy
    (off particle-hole symmetry) differ from the box-only rhs."""
    N = 16
    w = inputs.Workload("t", N=N, U=1.7, T=0.03, eps_d=-0.85 + 0.3)
    V = inputs.random_vertex(N, w.U, seed=5)
    sig = inputs.random_sigma(N, seed=6)
    with frg.Context([w], channel_mask=0xF) as c0, frg.Context([w], channel_mask=0x1F) as c1:
        dg0, ds0 = gpu_rhs(c0, 0.4, V, sig)
        dg1, ds1 = gpu_rhs(c1, 0.4, V, sig)
    assert nrel(dg1, dg0) > 1e-4 and nrel(ds1, ds0) > 1e-4


@pytest.mark.parametrize("prec", [frg.FP64, frg.TF32X3])
def test_tails_flow_matches_oracle_reference(prec):
    name = "siam_N16_U1_T0.05_asym0.3"
    with open(os.path.join(HERE, "golden", "oracle_flow_%s_mask1f.json" % name)) as f:
        ref = json.load(f)
    assert ref["mask"] == 0x1F
    w = inputs.WORKLOADS[name]
    with frg.Context([w], precision=prec, channel_mask=0x1F) as ctx:
        st = ctx.flow()[0]
        g, s, lam, _ = ctx.get_state(0)
        obs = ctx.observables(0)
    assert st.status == 0 and st.done == 1
    g = g.cpu().numpy()
    eg = flow_ref.gamma_error(g, ref)
    rsig = np.array(ref["sigma_re"]) + 1j * np.array(ref["sigma_im"])
    es = nrel(s.cpu().numpy(), rsig)
    ru = complex(*ref["observables"]["U_eff"])
    eu = abs(obs["U_eff"] - ru) / abs(ru)
    print("prec=%d tails flow errors gamma %.3e sigma %.3e ueff %.3e evals %d vs %d" % (
        prec, eg, es, eu, st.rhs_evals, ref["stats"]["rhs_evals"]))
    assert eg < FLOW_TOL[prec] and es < FLOW_TOL[prec] and eu < FLOW_TOL[prec]
    if prec == frg.FP64:
        assert st.accepted == ref["stats"]["accepted"] and st.rejected == ref["stats"]["rejected"]
        assert st.rhs_evals == ref["stats"]["rhs_evals"]


def test_tails_in_a_mixed_size_batch_equal_single_point_runs():
    pts = [inputs.Workload("a", N=16, U=1.2, T=0.04, eps_d=-0.6 + 0.2),
           inputs.Workload("b", N=34, U=2.0, T=0.03, eps_d=-1.0 - 0.4)]
    with frg.Context(pts, channel_mask=0x1F) as ctx:
        stb = ctx.advance(4)
        batched = [ctx.get_state(i)[:2] for i in range(len(pts))]
    for i, w in enumerate(pts):
        with frg.Context([w], channel_mask=0x1F) as ctx:
            st = ctx.advance(4)[0]
            g, s, _, _ = ctx.get_state(0)
        assert torch.equal(g, batched[i][0]) and torch.equal(s, batched[i][1])
        assert st.rhs_evals == stb[i].rhs_evals


def test_concurrent_tail_kernels_leave_the_contraction_intact():
    """With the tails the tail kernels share the SMs with the contraction; the
    rhs must equal the in-order evaluation (frg_rhs_timed, no side stream)
    bit for bit.  Idle pauses between calls change the relative timing of the
    two streams (a missing proxy fence once let a tensor-map copy overtake the
    transform's reads of its raw stage in exactly this setting)."""
    import time
    N = 100
    w = inputs.Workload("t", N=N, U=1.7, T=0.03, eps_d=-0.85 + 0.3)
    V = inputs.random_vertex(N, w.U, seed=717)
    sig = inputs.random_sigma(N, seed=718)
    g = torch.from_numpy(V).cuda()
    s = torch.from_numpy(sig).cuda()
    with frg.Context([w], precision=frg.TF32X3, channel_mask=0x1F) as ctx:
        for Lam in (0.01, 0.4, 7.0, 0.4, 7.0, 0.01):
            time.sleep(0.7)
            a, sa = torch.empty_like(g), torch.empty_like(s)
            b, sb = torch.empty_like(g), torch.empty_like(s)
            ctx.rhs(0, Lam, g, s, a, sa)
            torch.cuda.synchronize()
            ctx.rhs_timed(0, Lam, g, s, b, sb)
            torch.cuda.synchronize()
            assert torch.equal(a, b) and torch.equal(sa, sb), Lam
