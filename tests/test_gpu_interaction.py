"""GPU parity of the interaction-flow cutoff (frg_params.cutoff =
FRG_CUTOFF_INTERACTION: Theta = 1/sqrt(Lambda), Lambda = 1/g from 1e12 down to
the full model at 1) against the FP64 CPU oracle, through the C ABI.

The cutoff changes only the propagators (and so the bubble weights and the
self-energy kernel); every channel kernel is shared with the Omega scheme.
Tolerances as for the Omega scheme: FP64 rhs 1e-12 and flows 1e-10 with the
oracle's step sequence; split paths within their rhs bounds and flows 1e-6."""
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
    return oracle.Model(U=w.U, T=w.T, eps_d=w.eps_d, Delta=w.Delta, N=w.N, cutoff=w.cutoff)


def gpu_rhs(ctx, Lam, V, sig):
    g = torch.from_numpy(np.ascontiguousarray(V)).cuda()
    s = torch.from_numpy(np.ascontiguousarray(sig)).cuda()
    dg = torch.full_like(g, complex(np.nan, np.nan))
    ds = torch.full_like(s, complex(np.nan, np.nan))
    ctx.rhs(0, Lam, g, s, dg, ds)
    torch.cuda.synchronize()
    return dg.cpu().numpy(), ds.cpu().numpy()


def iflow(N):
    return inputs.Workload("t", N=N, U=1.7, T=0.03, eps_d=-0.85 + 0.3, Lambda0=1e12, Lambda_f=1.0, cutoff=1)


@pytest.mark.parametrize("prec", [frg.FP64, frg.TF32X3, frg.BF16X3])
@pytest.mark.parametrize("N", [2, 4, 16, 34])
@pytest.mark.parametrize("mask", [0xF, 0x1, 0x2, 0x4, 0x8, 0xF | frg.TAILS])
def test_interaction_rhs_matches_oracle(prec, N, mask):
    """FP64: normwise against the oracle's rhs with the same mask; split
    precisions: against the whole rhs of the same input and options (rhs_bar)."""
    w = iflow(N)
    V = inputs.random_vertex(N, w.U, seed=5 * N)
    sig = inputs.random_sigma(N, seed=300 + N)
    with frg.Context([w], precision=prec, channel_mask=mask) as ctx:
        for Lam in (1e6, 30.0, 1.0):
            dg, ds = gpu_rhs(ctx, Lam, V, sig)
            rg, rs = oracle.rhs(model(w), Lam, V, sig, mask=mask)
            ng, ns = (np.max(np.abs(rg)), np.max(np.abs(rs))) if prec == frg.FP64 else \
                rhs_bar.full_norms(model(w), Lam, V, sig, extra_mask=mask & frg.TAILS,
                                   key=("iflow", N))
            if mask & 7:
                assert rhs_bar.err(dg, rg, ng) < RHS_TOL[prec], (Lam, rhs_bar.err(dg, rg, ng))
            if mask & 8:
                assert rhs_bar.err(ds, rs, ns) < RHS_TOL[prec]


def test_cutoff_changes_the_rhs():
    N = 16
    w1 = iflow(N)
    w0 = inputs.Workload("t", N=N, U=w1.U, T=w1.T, eps_d=w1.eps_d)
    V = inputs.random_vertex(N, w1.U, seed=8)
    sig = inputs.random_sigma(N, seed=9)
    with frg.Context([w0]) as c0, frg.Context([w1]) as c1:
        a, sa = gpu_rhs(c0, 1.0, V, sig)
        b, sb = gpu_rhs(c1, 1.0, V, sig)
    assert nrel(a, b) > 1e-2 and nrel(sa, sb) > 1e-2


@pytest.mark.parametrize("prec", [frg.FP64, frg.TF32X3])
@pytest.mark.parametrize("name", ["siam_N16_U1_T0.05_asym0.3_iflow", "siam_N64_U2_T0.01_asym0.5_iflow"])
def test_interaction_flow_matches_oracle_reference(name, prec):
    with open(os.path.join(HERE, "golden", "oracle_flow_%s.json" % name)) as f:
        ref = json.load(f)
    w = inputs.WORKLOADS[name]
    assert ref["params"]["cutoff"] == 1 and w.cutoff == 1
    with frg.Context([w], precision=prec) as ctx:
        st = ctx.flow()[0]
        g, s, lam, _ = ctx.get_state(0)
        obs = ctx.observables(0)
    assert st.status == 0 and st.done == 1 and abs(lam - 1.0) < 1e-15
    g = g.cpu().numpy()
    eg = flow_ref.gamma_error(g, ref)
    rsig = np.array(ref["sigma_re"]) + 1j * np.array(ref["sigma_im"])
    es = nrel(s.cpu().numpy(), rsig)
    ro = ref["observables"]
    eu = abs(obs["U_eff"] - complex(*ro["U_eff"])) / abs(complex(*ro["U_eff"]))
    ez = abs(obs["Z"] - ro["Z"])
    print("prec=%d interaction flow %s errors gamma %.3e sigma %.3e ueff %.3e Z %.1e evals %d vs %d" % (
        prec, name, eg, es, eu, ez, st.rhs_evals, ref["stats"]["rhs_evals"]))
    assert max(eg, es, eu, ez) < FLOW_TOL[prec]
    if prec == frg.FP64:
        assert st.accepted == ref["stats"]["accepted"] and st.rejected == ref["stats"]["rejected"]
        assert st.rhs_evals == ref["stats"]["rhs_evals"]


def test_interaction_rhs_without_allocation():
    N = 16
    w = iflow(N)
    V = inputs.random_vertex(N, w.U, seed=17)
    sig = inputs.random_sigma(N, seed=18)
    g = torch.from_numpy(V).cuda()
    s = torch.from_numpy(sig).cuda()
    dg, ds = torch.empty_like(g), torch.empty_like(s)
    frg.rhs_noalloc(frg.Params.from_workload(w), 3.0, g, s, dg, ds)
    torch.cuda.synchronize()
    rg, rs = oracle.rhs(model(w), 3.0, V, sig)
    assert nrel(dg.cpu().numpy(), rg) < RHS_TOL[frg.FP64] and nrel(ds.cpu().numpy(), rs) < RHS_TOL[frg.FP64]
