"""Error measure of one split-precision rhs evaluation against the oracle.

The acceptance bar of the split precisions concerns the right-hand side the
flow integrates, F[V] = dV/dl with every channel on (paper Sec. 2, Eq. 1).  A
test that switches channels off looks at one term of that sum, and a term can be
a small difference of large products (the direct particle-hole combination
2VV - VV - VV cancels exactly at the bare vertex), so its error is measured
against the size of the whole rhs of the same input: max |gpu - oracle| over
the entries, divided by max |F[V]| (the oracle's rhs with every channel of the
same options on).  With every channel on this is the plain normwise relative
error."""
import numpy as np

import oracle

_FULL = {}


def full_norms(model, Lam, V, sig, extra_mask=0, key=None):
    """max |dV/dl| and max |dSigma/dl| of the oracle's whole rhs (channels and
    self-energy on, plus the option bits in extra_mask); cached under key."""
    k = None if key is None else (key, Lam, extra_mask)
    if k is not None and k in _FULL:
        return _FULL[k]
    rg, rs = oracle.rhs(model, Lam, V, sig, mask=0xF | extra_mask)
    out = (float(np.max(np.abs(rg))), float(np.max(np.abs(rs))))
    if k is not None:
        _FULL[k] = out
    return out


def err(got, ref, norm):
    """max |got - ref| / norm."""
    return float(np.max(np.abs(np.asarray(got) - np.asarray(ref))) / max(norm, 1e-300))
