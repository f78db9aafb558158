"""Physics checks of the GPU flows that do not go through the oracle.

With a single vertex channel and the self-energy flow switched off, the
one-loop flow is a geometric (ladder) series with a closed form on every
entry whose four frequencies lie in the box:
  pp alone:  V = U / (1 + U dB_pp(s)),   dB_pp(s) = T sum_p [G(p) G(s-p)] from Lambda0 to Lambda_f
  xph alone: V = U / (1 + U dB_ph(Q)),   dB_ph(Q) = T sum_p [G(p) G(p+Q)] ...
  dph alone: V = U (its spin sum 2VV - VV - VV vanishes for a constant vertex)
with the free regulated propagator G (closed_forms.py).  Both the plain FP64
path and the 3xTF32 tensor-core path must reproduce them: FP64 to the ODE
tolerance, 3xTF32 to its 1e-6 flow bar."""
import numpy as np
import pytest

import closed_forms as cf
from paper_1510_07799_gb300 import frg, inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {frg.FP64: 2e-8, frg.TF32X3: 1e-6}


@pytest.mark.parametrize("prec", [frg.FP64, frg.TF32X3])
@pytest.mark.parametrize("mask,U", [(frg.CH_PP, 2.5), (0x4, 1.2), (0x2, 2.0)])
def test_single_channel_ladder_flow_hits_the_closed_form(prec, mask, U):
    N, T, D, shift = 12, 0.05, 1.0, 0.5
    w = inputs.Workload("ladder", N=N, U=U, T=T, eps_d=-U / 2 + shift, Delta=D)
    p = frg.Params.from_workload(w)
    if prec == frg.FP64:
        p.rtol, p.atol = 1e-11, 1e-14
    with frg.Context([p], precision=prec, channel_mask=mask) as ctx:
        st = ctx.flow()[0]
        g, s, lam, _ = ctx.get_state(0)
    assert st.status == 0 and st.done == 1
    g = g.cpu().numpy()
    assert float(s.abs().max()) == 0.0  # the self-energy flow is off
    _, dBpp, dBph = cf.second_order_vertex(N, T, shift, D, 1.0, w.Lambda0, w.Lambda_f)
    if mask == frg.CH_PP:
        ref = U / (1 + U * dBpp)
    elif mask == 0x4:
        ref = U / (1 + U * dBph)
    else:
        ref = np.full(g.shape, U, np.complex128)
    mk = inputs.all_in_box_mask(N)
    err = float(np.max(np.abs(g[mk] - ref[mk])) / np.max(np.abs(ref[mk])))
    assert err < TOL[prec]
    if mask != 0x2:
        assert float(np.max(np.abs(ref[mk] - U)) / U) > 0.05  # far from the bare value
