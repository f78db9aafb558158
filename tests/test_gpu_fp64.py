"""GPU parity of the plain-FP64 CUDA path against the FP64 CPU oracle, through
the C ABI.  Tolerance: the FP64 path differs from the oracle only by summation
order, so the rhs agrees to 1e-12 relative max-norm and full flows to 1e-10
(the acceptance bar of the FP64 path)."""
import json
import os

import numpy as np
import pytest

import flow_ref
import oracle
from paper_1510_07799_gb300 import frg, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
RHS_TOL = 1e-12
FLOW_TOL = 1e-10


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
@pytest.mark.parametrize("N", [2, 4, 6, 16, 34, 64])
@pytest.mark.parametrize("mask", [0xF, 0x1, 0x2, 0x4, 0x8])
def test_rhs_matches_oracle(N, mask, crossing):
    """Every channel mask, on vertices with and without crossing symmetry: the
    channel sums (paper Sec. 2, Eq. 1; Sec. 4) are defined for any vertex, and
    the FP64 path evaluates every operand as the entry the sum names."""
    w = inputs.Workload("t", N=N, U=1.7, T=0.03, eps_d=-0.85 + 0.3)
    V = inputs.random_vertex(N, w.U, seed=N + mask + (0 if crossing else 500), crossing=crossing)
    sig = inputs.random_sigma(N, seed=100 + N)
    with frg.Context([w], channel_mask=mask) as ctx:
        for Lam in (0.01, 0.4, 7.0):
            dg, ds = gpu_rhs(ctx, 0, Lam, V, sig)
            rg, rs = oracle.rhs(model(w), Lam, V, sig, mask=mask)
            if mask & 7:
                assert nrel(dg, rg) < RHS_TOL
            else:
                assert np.max(np.abs(dg)) == 0.0
            if mask & 8:
                assert nrel(ds, rs) < RHS_TOL
            else:
                assert np.max(np.abs(ds)) == 0.0


def test_rhs_host_buffers_match_device_buffers():
    w = inputs.Workload("t", N=20, U=2.0, T=0.02, eps_d=-0.7)
    V = inputs.random_vertex(w.N, w.U, seed=3)
    sig = inputs.random_sigma(w.N, seed=4)
    with frg.Context([w]) as ctx:
        dg, ds = gpu_rhs(ctx, 0, 0.3, V, sig)
        hg = np.empty_like(V)
        hs = np.empty_like(sig)
        ctx.rhs_host(0, 0.3, V, sig, hg, hs)
        assert np.array_equal(hg, dg) and np.array_equal(hs, ds)


def test_rhs_full_size_sampled_entries():
    """N = 128 in the benchmark's launch configuration: sampled entries against
    the oracle's entry-by-entry evaluation; self-energy in full."""
    w = inputs.SIAM_N128
    V = inputs.random_vertex(w.N, w.U, seed=11)
    sig = inputs.random_sigma(w.N, seed=12, amp=0.05)
    Lam = 0.02
    with frg.Context([w]) as ctx:
        dg, ds = gpu_rhs(ctx, 0, Lam, V, sig)
    rng = np.random.default_rng(5)
    idx = rng.integers(0, w.N, (3000, 3))
    idx[:4] = [[0, 0, 0], [w.N - 1] * 3, [w.N // 2] * 3, [0, w.N - 1, 0]]
    ref = oracle.rhs_entries(model(w), Lam, V, sig, idx)
    got = dg[idx[:, 0], idx[:, 1], idx[:, 2]]
    assert nrel(got, ref) < RHS_TOL
    _, rs = oracle.rhs(oracle.Model(U=w.U, T=w.T, eps_d=w.eps_d, Delta=w.Delta, N=w.N), Lam,
                       V, sig, mask=0x8)
    assert nrel(ds, rs) < RHS_TOL


def load_golden(name):
    with open(os.path.join(HERE, "golden", "oracle_flow_%s.json" % name)) as f:
        return json.load(f)


@pytest.mark.parametrize("name", ["siam_N16_U1_T0.05_ph", "siam_N64_U2_T0.01_asym0.5",
                                  "siam_N128_U3_T0.005_ph"])
def test_full_flow_matches_oracle_reference(name):
    ref = load_golden(name)
    w = inputs.WORKLOADS[name]
    with frg.Context([w]) as ctx:
        st = ctx.flow()[0]
        g, s, lam, _ = ctx.get_state(0)
        obs = ctx.observables(0)
    assert st.status == 0 and st.done == 1 and abs(lam - w.Lambda_f) < 1e-15
    g = g.cpu().numpy()
    s = s.cpu().numpy()
    assert flow_ref.gamma_error(g, ref) < FLOW_TOL
    rsig = np.array(ref["sigma_re"]) + 1j * np.array(ref["sigma_im"])
    assert nrel(s, rsig) < FLOW_TOL
    ro = ref["observables"]
    assert abs(obs["U_eff"] - complex(*ro["U_eff"])) / abs(complex(*ro["U_eff"])) < FLOW_TOL
    assert abs(obs["Z"] - ro["Z"]) < FLOW_TOL
    # same step sequence as the oracle's controller
    assert st.accepted == ref["stats"]["accepted"] and st.rejected == ref["stats"]["rejected"]
    assert st.rhs_evals == ref["stats"]["rhs_evals"]


def test_full_flow_matches_live_oracle_off_symmetry():
    w = inputs.Workload("t", N=24, U=2.5, T=0.02, eps_d=-1.25 - 0.6)
    g0, s0, st0 = oracle.flow(model(w))
    with frg.Context([w]) as ctx:
        st = ctx.flow()[0]
        g, s, _, _ = ctx.get_state(0)
    assert nrel(g.cpu().numpy(), g0) < FLOW_TOL
    assert nrel(s.cpu().numpy(), s0) < FLOW_TOL
    assert st.rhs_evals == st0.rhs_evals


def test_first_step_costs_seven_evaluations():
    with frg.Context([inputs.SIAM_N16]) as ctx:
        st = ctx.advance(1)[0]
    assert st.rhs_evals == 7 and st.accepted + st.rejected == 1


def test_checkpoint_resume_is_bitwise():
    w = inputs.SIAM_N16
    with frg.Context([w]) as ctx:
        ctx.flow()
        gA, sA, _, _ = ctx.get_state(0)
    with frg.Context([w]) as ctx:
        ctx.advance(20)
        g, s, lam, h = ctx.get_state(0)
    assert lam > w.Lambda_f
    with frg.Context([w]) as ctx2:
        ctx2.set_state(0, g, s, lam, h)
        ctx2.flow()
        gB, sB, lamB, _ = ctx2.get_state(0)
    assert torch.equal(gA, gB) and torch.equal(sA, sB)


def test_repeat_runs_are_bitwise_identical():
    w = inputs.Workload("t", N=18, U=1.5, T=0.04, eps_d=-0.4)
    out = []
    for _ in range(2):
        with frg.Context([w]) as ctx:
            ctx.flow()
            out.append(ctx.get_state(0)[:2])
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])


def test_batched_points_equal_single_point_runs():
    pts = [inputs.Workload("a", N=8, U=1.0, T=0.05, eps_d=-0.5),
           inputs.Workload("b", N=20, U=2.5, T=0.02, eps_d=-1.0),
           inputs.Workload("c", N=14, U=0.7, T=0.08, eps_d=0.1)]
    with frg.Context(pts) as ctx:
        stb = ctx.flow()
        batched = [ctx.get_state(i)[:2] for i in range(3)]
    for i, w in enumerate(pts):
        with frg.Context([w]) as ctx:
            st = ctx.flow()[0]
            g, s, _, _ = ctx.get_state(0)
        assert torch.equal(g, batched[i][0]) and torch.equal(s, batched[i][1])
        assert st.rhs_evals == stb[i].rhs_evals


def test_non_finite_state_is_reported():
    w = inputs.SIAM_N16
    V = np.full((w.N,) * 3, w.U, np.complex128)
    V[3, 4, 5] = np.nan
    with frg.Context([w]) as ctx:
        ctx.set_state(0, torch.from_numpy(V).cuda(), None, 1.0)
        with pytest.raises(frg.FrgError) as e:
            ctx.flow()
        assert e.value.code == frg.ENONFINITE


def test_step_limit_is_reported():
    w = inputs.SIAM_N16
    p = frg.Params.from_workload(w)
    p.max_steps = 3
    with frg.Context([p]) as ctx:
        with pytest.raises(frg.FrgError) as e:
            ctx.flow()
        assert e.value.code == frg.ENOTCONV
        st = ctx.stats()[0]
        assert st.accepted + st.rejected == 3 and st.done == 1
