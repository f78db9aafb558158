"""Reading the oracle's stored flow results (tests/golden/oracle_flow_*.json,
written by tests/golden/make_oracle_reference.py, which calls only oracle/).

A golden file holds the whole final vertex for small grids (full_re/full_im)
and a seeded sample of entries for every grid; gamma_error compares a GPU final
vertex against the whole stored vertex when it is there, else on the sample,
normwise: max |g - ref| / max |ref| (the norm of the whole oracle vertex)."""
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def load(name):
    with open(os.path.join(HERE, "golden", "oracle_flow_%s.json" % name)) as f:
        return json.load(f)


def full_vertex(ref):
    """The whole final oracle vertex (N, N, N), or None when only sampled."""
    if not ref.get("full_re"):
        return None
    N = ref["params"]["N"]
    return (np.array(ref["full_re"]) + 1j * np.array(ref["full_im"])).reshape(N, N, N)


def gamma_error(g, ref):
    """Normwise relative error of the final vertex g against the oracle's:
    every entry where the golden file has the whole vertex, else its sample."""
    g = np.asarray(g)
    full = full_vertex(ref)
    if full is not None:
        return float(np.max(np.abs(g - full)) / ref["gamma_norm_inf"])
    idx = np.array(ref["sample_idx"])
    rv = np.array(ref["sample_re"]) + 1j * np.array(ref["sample_im"])
    return float(np.max(np.abs(g[idx[:, 0], idx[:, 1], idx[:, 2]] - rv)) / ref["gamma_norm_inf"])
