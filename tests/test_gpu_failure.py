"""Failure detection on the GPU without a GPU fault.

Every wait of the tensor-core pipeline is bounded: a wait that runs out records
the failure in the context's device error word, every role of the kernel leaves
its loop, and the host reports FRG_ETIMEOUT.  The self-test entry point runs one
such wait on a barrier that nothing completes (a short limit), so the failure
path is exercised without hanging or faulting the device; the context must stay
usable afterwards."""
import time

import numpy as np
import pytest

import oracle
from paper_1510_07799_gb300 import frg, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_stays_usable():
    w = inputs.Workload("t", N=16, U=1.2, T=0.04, eps_d=-0.3)
    with frg.Context([w], precision=frg.TF32X3) as ctx:
        t0 = time.perf_counter()
        with pytest.raises(frg.FrgError) as e:
            ctx.selftest_wait(50.0)
        assert e.value.code == frg.ETIMEOUT
        assert "bounded device-side wait" in str(e.value)
        assert time.perf_counter() - t0 < 10.0
        # the error word was cleared: the next evaluation runs normally
        V = inputs.random_vertex(w.N, w.U, seed=81)
        sig = inputs.random_sigma(w.N, seed=82)
        g = torch.from_numpy(V).cuda()
        s = torch.from_numpy(sig).cuda()
        dg, ds = torch.empty_like(g), torch.empty_like(s)
        ctx.rhs(0, 0.1, g, s, dg, ds)
        torch.cuda.synchronize()
        rg, rs = oracle.rhs(oracle.Model(U=w.U, T=w.T, eps_d=w.eps_d, Delta=w.Delta, N=w.N), 0.1, V, sig)
        dg = dg.cpu().numpy()
        assert np.max(np.abs(dg - rg)) / np.max(np.abs(rg)) < 1e-6
        # and a flow runs to the end
        st = ctx.flow()[0]
        assert st.status == 0 and st.done == 1


def test_selftest_rejects_bad_limits():
    with frg.Context([inputs.SIAM_N16]) as ctx:
        with pytest.raises(frg.FrgError) as e:
            ctx.selftest_wait(-1.0)
        assert e.value.code == frg.EINVAL
