"""Write oracle reference values for full flows into tests/golden/.

Runs only the FP64 CPU oracle (oracle/) on a named workload from the input
module, flowing from Lambda0 to Lambda_f, and stores a seeded sample of the final
vertex (and, for grids up to FULL_MAX_N, the whole final vertex), the whole
self-energy, the observables, the norms needed for normwise relative errors,
and the integrator statistics.  Nothing here touches the CUDA path.

usage: python tests/golden/make_oracle_reference.py <workload-name> [samples] [mask]
(mask: the channel mask in hex, default 0xF; a mask other than 0xF is part of
the output file's name)
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1510_07799_gb300 import inputs  # noqa: E402

SAMPLE_SEED = 20151025
FULL_MAX_N = 16  # whole final vertex stored up to this grid (N^3 entries)


def sample_indices(N, count, seed=SAMPLE_SEED):
    """Seeded sample of vertex entries, always including the lowest-frequency
    entry (the effective interaction) and its crossing/reversal partners."""
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, N, (count, 3))
    h = N // 2
    extra = np.array([[h, h, h], [h - 1, h - 1, h - 1], [0, 0, 0], [N - 1, N - 1, N - 1],
                      [h, h - 1, h], [h - 1, h, h - 1]])
    return np.concatenate([extra, idx]).astype(np.int64)


def main():
    name = sys.argv[1]
    count = int(sys.argv[2]) if len(sys.argv) > 2 else 2048
    mask = int(sys.argv[3], 16) if len(sys.argv) > 3 else 0xF
    w = inputs.WORKLOADS[name]
    m = oracle.Model(U=w.U, T=w.T, eps_d=w.eps_d, Delta=w.Delta, N=w.N, cutoff=w.cutoff)
    t0 = time.time()
    g, s, st = oracle.flow(m, Lambda0=w.Lambda0, Lambda_f=w.Lambda_f, rtol=w.rtol,
                           atol=w.atol, mask=mask)
    wall = time.time() - t0
    if st.status != 0:
        raise SystemExit("oracle flow failed: %s" % st)
    idx = sample_indices(w.N, count)
    vals = g[idx[:, 0], idx[:, 1], idx[:, 2]]
    obs = oracle.observables(m, w.Lambda_f, g, s)
    out = {
        "workload": name,
        "mask": mask,
        "what": "oracle FP64 flow from Lambda0 to Lambda_f; sampled final vertex (whole vertex "
                "in full_re/full_im, flat index ((i1*N)+i2)*N+i3, when N <= %d)" % FULL_MAX_N,
        "params": {"N": w.N, "U": w.U, "T": w.T, "eps_d": w.eps_d, "Delta": w.Delta,
                   "Lambda0": w.Lambda0, "Lambda_f": w.Lambda_f, "rtol": w.rtol,
                   "atol": w.atol, "cutoff": w.cutoff},
        "stats": {"accepted": st.accepted, "rejected": st.rejected,
                  "rhs_evals": st.rhs_evals, "first_step_evals": st.first_step_evals,
                  "wall_s": wall, "threads": oracle.max_threads()},
        "gamma_norm_inf": float(np.max(np.abs(g))),
        "sigma_norm_inf": float(np.max(np.abs(s))),
        "gamma_mean": [float(g.real.mean()), float(g.imag.mean())],
        "sample_idx": idx.tolist(),
        "sample_re": [float(x) for x in vals.real],
        "sample_im": [float(x) for x in vals.imag],
        "full_re": [float(x) for x in g.real.reshape(-1)] if w.N <= FULL_MAX_N else None,
        "full_im": [float(x) for x in g.imag.reshape(-1)] if w.N <= FULL_MAX_N else None,
        "sigma_re": [float(x) for x in s.real],
        "sigma_im": [float(x) for x in s.imag],
        "observables": {"sigma_lowest": [obs["sigma_lowest"].real, obs["sigma_lowest"].imag],
                        "Z": obs["Z"], "U_eff": [obs["U_eff"].real, obs["U_eff"].imag],
                        "n": obs["n"]},
    }
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        "oracle_flow_%s%s.json" % (name, "" if mask == 0xF else "_mask%x" % mask))
    with open(path, "w") as f:
        json.dump(out, f, indent=0, separators=(",", ":"))
        f.write("\n")
    print(path, st, "%.1fs" % wall)


if __name__ == "__main__":
    main()
