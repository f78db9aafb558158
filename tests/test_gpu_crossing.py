"""GPU parity of the crossing reduction of the split-precision channel products
(channel_mask | FRG_CROSSING), through the C ABI.

Crossing symmetry V(i1,i2,i3) = V(i2,i1,i4) pairs the entries of each
channel's product at one transfer (pp directly, the two particle-hole channels
composed with frequency reversal); with the reversal reduction's transfers the
contraction skips one rectangle of partners in every transfer with more than 64
valid rows and writes it from the entries it computed.  On inputs with both
symmetries the rhs matches the oracle within the split bar and the unreduced
rhs within rounding; flows from the bare vertex (crossing-symmetric in exact
arithmetic) match the FP64 GPU flow and the oracle's reference within the 1e-6
flow bar."""
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
RHS_TOL = {frg.TF32X3: 1e-6, frg.BF16X3: 5e-5}
FLOW_TOL = 1e-6
RC = frg.REVERSAL | frg.CROSSING


def nrel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def model(w):
    return oracle.Model(U=w.U, T=w.T, eps_d=w.eps_d, Delta=w.Delta, N=w.N)


def symmetric_state(N, U, seed):
    """A vertex with both symmetries (the crossing-symmetric seeded vertex
    averaged with its reversed conjugate: the two maps commute) and a
    reversal-symmetric self-energy."""
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


def test_inputs_have_both_symmetries():
    N = 66
    V, s = symmetric_state(N, 1.3, 5)
    i1, i2, i3 = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    i4 = i1 + i2 - i3
    ok = (i4 >= 0) & (i4 < N)
    assert np.max(np.abs(V[ok] - V[i2[ok], i1[ok], i4[ok]])) < 1e-15
    assert np.array_equal(V, np.conj(V[::-1, ::-1, ::-1])) and np.array_equal(s, np.conj(s[::-1]))


@pytest.mark.parametrize("prec", [frg.TF32X3, frg.BF16X3])
@pytest.mark.parametrize("N,mask", [(66, 0xF), (66, 0x1), (66, 0x2), (66, 0x4), (100, 0xF), (100, 0x1),
                                    (100, 0x2), (100, 0x4), (98, 0xF), (128, 0xF)])
def test_crossing_rhs_matches_oracle(prec, N, mask):
    """Reduced rhs against the oracle (split bar, rhs_bar) and against the
    reversal-reduced rhs without crossing on the same input; the self-energy
    rhs does not involve the products and is unchanged bit for bit."""
    w = inputs.Workload("t", N=N, U=1.7, T=0.03, eps_d=-0.85 + 0.3)
    V, sig = symmetric_state(N, w.U, 11 * N)
    lams = (0.01, 0.4, 7.0) if N < 128 else (0.4,)
    with frg.Context([w], precision=prec, channel_mask=mask | RC) as c, \
            frg.Context([w], precision=prec, channel_mask=mask | frg.REVERSAL) as c0:
        for Lam in lams:
            dg, ds = gpu_rhs(c, Lam, V, sig)
            dg0, ds0 = gpu_rhs(c0, Lam, V, sig)
            rg, _ = oracle.rhs(model(w), Lam, V, sig, mask=mask)
            ng = float(np.max(np.abs(rg))) if mask == 0xF else \
                rhs_bar.full_norms(model(w), Lam, V, sig, key=("crossing", N))[0]
            e, e0 = rhs_bar.err(dg, rg, ng), rhs_bar.err(dg, dg0, ng)
            print("prec=%d N=%d mask=%#x Lam=%g: vs oracle %.2e, vs unreduced %.2e" % (prec, N, mask, Lam, e, e0))
            assert np.isfinite(dg).all()
            assert e < RHS_TOL[prec] and e0 < RHS_TOL[prec]
            assert np.array_equal(ds, ds0)


@pytest.mark.parametrize("prec", [frg.TF32X3, frg.BF16X3])
def test_crossing_flow_matches_fp64_and_oracle_reference(prec):
    """The precision workload's whole flow from the bare vertex with the
    crossing reduction (and the automatic reversal reduction): every entry of
    the final vertex against the plain FP64 GPU flow, the oracle's stored
    sample, self-energy and effective interaction within the flow bar."""
    name = "siam_N128_U3_T0.005_ph"
    w = inputs.WORKLOADS[name]
    with open(os.path.join(HERE, "golden", "oracle_flow_%s.json" % name)) as f:
        ref = json.load(f)
    with frg.Context([w]) as c64:
        s64 = c64.flow()[0]
        g64, sg64, _, _ = c64.get_state(0)
    with frg.Context([w], precision=prec, channel_mask=0xF | frg.CROSSING) as ctx:
        st = ctx.flow()[0]
        g, s, _, _ = ctx.get_state(0)
        obs = ctx.observables(0)
    assert s64.status == 0 and st.status == 0 and st.done == 1
    g = g.cpu().numpy()
    e_all = nrel(g, g64.cpu().numpy())
    es = nrel(s.cpu().numpy(), sg64.cpu().numpy())
    eg = flow_ref.gamma_error(g, ref)
    ru = complex(*ref["observables"]["U_eff"])
    eu = abs(obs["U_eff"] - ru) / abs(ru)
    print("prec=%d crossing flow: every entry vs FP64 %.2e, sigma %.2e, oracle sample %.2e, U_eff %.2e, evals %d" % (
        prec, e_all, es, eg, eu, st.rhs_evals))
    assert max(e_all, es, eg, eu) < FLOW_TOL


def test_crossing_flow_off_symmetry_matches_the_unreduced_flow():
    """Off particle-hole symmetry at a grid of 100 frequencies (transfers of
    even and odd row counts): the reduced flow against the flow without the
    crossing reduction and the FP64 GPU flow."""
    w = inputs.Workload("c", N=100, U=2.0, T=0.01, eps_d=-1.0 + 0.4)
    with frg.Context([w]) as c64:
        c64.flow()
        g64, s64, _, _ = c64.get_state(0)
    out = {}
    for mask in (0xF, 0xF | frg.CROSSING):
        with frg.Context([w], precision=frg.TF32X3, channel_mask=mask) as c:
            st = c.flow()[0]
            assert st.status == 0 and st.done == 1
            out[mask] = [x.cpu().numpy() for x in c.get_state(0)[:2]]
    g, s = out[0xF | frg.CROSSING]
    print("N=100 crossing flow: vs unreduced %.2e, vs FP64 %.2e" % (nrel(g, out[0xF][0]), nrel(g, g64.cpu().numpy())))
    assert nrel(g, out[0xF][0]) < FLOW_TOL and nrel(g, g64.cpu().numpy()) < FLOW_TOL
    assert nrel(s, s64.cpu().numpy()) < FLOW_TOL


@pytest.mark.parametrize("prec,extra", [(frg.FP64, 0), (frg.TF32X3, frg.NO_REVERSAL)])
def test_crossing_bit_is_inert_where_every_transfer_is_computed(prec, extra):
    """The FP64 path and flows without the reversal reduction compute every
    entry: the bit changes nothing, bit for bit."""
    w = inputs.Workload("c", N=66, U=1.3, T=0.04, eps_d=-0.65 + 0.25)
    res = []
    for mask in (0xF | extra, 0xF | extra | frg.CROSSING):
        with frg.Context([w], precision=prec, channel_mask=mask) as c:
            c.advance(3)
            res.append(c.get_state(0)[:2])
    assert torch.equal(res[0][0], res[1][0]) and torch.equal(res[0][1], res[1][1])


def test_crossing_in_a_mixed_size_batch_equals_single_point_runs():
    """Points with and without reduced transfers (N above and below 64) share
    one schedule; each equals its own run bit for bit."""
    pts = [inputs.Workload("a", N=128, U=1.2, T=0.02, eps_d=-0.6 + 0.2),
           inputs.Workload("b", N=48, U=2.0, T=0.03, eps_d=-1.0 - 0.4),
           inputs.Workload("c", N=90, U=1.5, T=0.025, eps_d=-0.75)]
    with frg.Context(pts, precision=frg.TF32X3, channel_mask=0xF | frg.CROSSING) as ctx:
        stb = ctx.advance(3)
        batched = [ctx.get_state(i)[:2] for i in range(len(pts))]
    for i, w in enumerate(pts):
        with frg.Context([w], precision=frg.TF32X3, channel_mask=0xF | frg.CROSSING) as ctx:
            st = ctx.advance(3)[0]
            g, s, _, _ = ctx.get_state(0)
        assert torch.equal(g, batched[i][0]) and torch.equal(s, batched[i][1])
        assert st.rhs_evals == stb[i].rhs_evals
