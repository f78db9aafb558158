"""The allocation-free rhs entry point (frg_rhs_noalloc) against the context
path (frg_rhs), on the GPU, through the C ABI.

Callers that cannot allocate device memory when they need an rhs (latency-
critical loops, processes whose device memory belongs to another allocator)
use frg_rhs_noalloc, whose workspace is a fixed device array inside the
library.  Both entry points run the same FP64 kernels, so they agree to the
FP64 parity bar of the other tests; two calls in a row check that nothing of
one call leaks into the next through the shared array.  This file is collected
last so that a failure here does not hide the other tests."""
import numpy as np
import pytest

import oracle
from paper_1510_07799_gb300 import frg, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12  # FP64 rhs parity bar used by the other GPU tests


def nrel(a, b):
    return float((a - b).abs().max() / b.abs().max())


def case(N, seed):
    w = inputs.Workload("noalloc", N=N, U=1.9, T=0.03, eps_d=-0.95 + 0.35)
    V = torch.from_numpy(inputs.random_vertex(N, w.U, seed=seed)).cuda()
    S = torch.from_numpy(inputs.random_sigma(N, seed=seed + 1)).cuda()
    return w, V, S


def test_noalloc_rhs_matches_context_rhs_on_consecutive_calls():
    for N, seeds in ((48, (1, 2)), (64, (3, 3)), (10, (4, 5))):
        # two calls in a row on the shared array (a different, then a repeated input)
        runs = []
        for seed in seeds:
            w, V, S = case(N, seed)
            Lam = 0.05 * seed
            dg, ds = torch.empty_like(V), torch.empty_like(S)
            frg.rhs_noalloc(w, Lam, V, S, dg, ds)
            runs.append((w, Lam, V, S, dg, ds))
        torch.cuda.synchronize()
        for w, Lam, V, S, dg, ds in runs:
            with frg.Context([w]) as ctx:
                rg, rs = torch.empty_like(V), torch.empty_like(S)
                ctx.rhs(0, Lam, V, S, rg, rs)
                torch.cuda.synchronize()
            assert nrel(dg, rg) < TOL and nrel(ds, rs) < TOL


@pytest.mark.parametrize("mask", [0x1, 0x2, 0x4, 0x8, 0x7, 0xF])
@pytest.mark.parametrize("with_sigma", [True, False])
def test_noalloc_channel_masks_and_absent_self_energy(mask, with_sigma):
    """channel_mask applies (mask 0x8 alone takes the zero-vertex branch), and
    a NULL self-energy input means Sigma = 0: the same as the context path
    with the same mask and no self-energy."""
    w, V, S = case(24, 30 + mask)
    sig = S if with_sigma else None
    dg, ds = torch.full_like(V, np.nan), torch.full_like(S, np.nan)
    frg.rhs_noalloc(w, 0.2, V, sig, dg, ds, channel_mask=mask)
    with frg.Context([w], channel_mask=mask) as ctx:
        rg, rs = torch.full_like(V, np.nan), torch.full_like(S, np.nan)
        ctx.rhs(0, 0.2, V, sig, rg, rs)
        torch.cuda.synchronize()
    for got, ref, on in ((dg, rg, mask & 7), (ds, rs, mask & 8)):
        if on:
            assert nrel(got, ref) < TOL
        else:
            assert float(got.abs().max()) == 0.0 and float(ref.abs().max()) == 0.0


def test_noalloc_matches_oracle_at_its_largest_grid():
    """N = 64 (the array's limit), Omega cutoff, off particle-hole symmetry, a
    vertex without crossing symmetry: against the FP64 CPU oracle's literal
    sums, whole vertex and self-energy, with and without a self-energy input."""
    w, V, S = case(64, 41)
    Vh = inputs.random_vertex(64, w.U, seed=41, crossing=False)
    V = torch.from_numpy(Vh).cuda()
    m = oracle.Model(U=w.U, T=w.T, eps_d=w.eps_d, Delta=w.Delta, N=w.N)
    for sig in (S, None):
        dg, ds = torch.full_like(V, np.nan), torch.full_like(S, np.nan)
        frg.rhs_noalloc(w, 0.07, V, sig, dg, ds)
        torch.cuda.synchronize()
        sh = sig.cpu().numpy() if sig is not None else np.zeros(64, complex)
        rg, rs = oracle.rhs(m, 0.07, Vh, sh)
        eg = np.max(np.abs(dg.cpu().numpy() - rg)) / np.max(np.abs(rg))
        es = np.max(np.abs(ds.cpu().numpy() - rs)) / np.max(np.abs(rs))
        assert eg < TOL and es < TOL, (eg, es)


def test_noalloc_rejects_sizes_beyond_its_array():
    for N, mask in ((frg.NOALLOC_MAX_N + 2, frg.CH_ALL), (7, frg.CH_ALL), (16, frg.CH_ALL | frg.TAILS),
                    (16, frg.CH_ALL | frg.REVERSAL), (16, frg.CH_ALL | frg.CROSSING)):
        w, V, S = case(N, 7)
        dg, ds = torch.full_like(V, 1.0), torch.full_like(S, 1.0)
        with pytest.raises(frg.FrgError) as e:
            frg.rhs_noalloc(w, 0.1, V, S, dg, ds, channel_mask=mask)
        assert e.value.code == frg.EINVAL
        torch.cuda.synchronize()
        assert bool((dg == 1.0).all()) and bool((ds == 1.0).all())  # nothing was written
