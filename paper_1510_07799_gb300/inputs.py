"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds the workload definitions (model parameters, grid sizes, the
seeded parameter batch) and seeded random vertex/self-energy states.  It holds
none of the flow's arithmetic: no propagators, bubbles, channel sums or
integrator.  Both the CUDA path and the CPU oracle consume what it produces.

Vertex arrays are complex128 of shape (N, N, N), index [i1, i2, i3] with
i = n + N/2 the fermionic Matsubara index n in [-N/2, N/2); the fourth index is
i4 = i1 + i2 - i3.  Workloads (frequency box N, interaction U, temperature T,
level eps_d, hybridisation Delta = 1, Lambda from 1e3 down to 1e-3):
"""
import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    N: int
    U: float
    T: float
    eps_d: float
    Delta: float = 1.0
    Lambda0: float = 1e3
    Lambda_f: float = 1e-3
    rtol: float = 1e-8
    atol: float = 1e-10
    cutoff: int = 0  # 0: Omega scheme; 1: interaction flow (Lambda = 1/g from Lambda0 down to 1)


# Plain FP64 single flow, particle-hole symmetric.
SIAM_N16 = Workload("siam_N16_U1_T0.05_ph", N=16, U=1.0, T=0.05, eps_d=-0.5)
# Off particle-hole symmetry (eps_d = -U/2 + 0.5).
SIAM_N64 = Workload("siam_N64_U2_T0.01_asym0.5", N=64, U=2.0, T=0.01, eps_d=-1.0 + 0.5)
# Precision workload, particle-hole symmetric.
SIAM_N128 = Workload("siam_N128_U3_T0.005_ph", N=128, U=3.0, T=0.005, eps_d=-1.5)
# Largest single flow (eps_d = -U/2 + 0.25).
SIAM_N256 = Workload("siam_N256_U3_T0.002_asym0.25", N=256, U=3.0, T=0.002,
                     eps_d=-1.5 + 0.25)

# Small flow off particle-hole symmetry (eps_d = -U/2 + 0.3), used with the
# frequency-box tail option (whose self-energy tail vanishes at ph symmetry).
SIAM_N16_ASYM = Workload("siam_N16_U1_T0.05_asym0.3", N=16, U=1.0, T=0.05, eps_d=-0.5 + 0.3)

# Interaction flow (cutoff 1): Lambda = 1/g from 1e12 down to 1, the full model;
# off particle-hole symmetry.
SIAM_N16_IFLOW = Workload("siam_N16_U1_T0.05_asym0.3_iflow", N=16, U=1.0, T=0.05, eps_d=-0.5 + 0.3,
                          Lambda0=1e12, Lambda_f=1.0, cutoff=1)
SIAM_N64_IFLOW = Workload("siam_N64_U2_T0.01_asym0.5_iflow", N=64, U=2.0, T=0.01, eps_d=-1.0 + 0.5,
                          Lambda0=1e12, Lambda_f=1.0, cutoff=1)

WORKLOADS = {w.name: w for w in (SIAM_N16, SIAM_N64, SIAM_N128, SIAM_N256, SIAM_N16_ASYM, SIAM_N16_IFLOW,
                                 SIAM_N64_IFLOW)}

BATCH_SEED = 1510077
BATCH_SIZES = (32, 48, 64, 96)


def batch_points(count: int = 64, seed: int = BATCH_SEED):
    """The batched workload: `count` parameter points drawn from one PCG64
    stream: U ~ U[0.5, 4], T ~ U[0.01, 0.1], eps_d = -U/2 + U[-1, 1]; grid
    sizes N from (32, 48, 64, 96) in equal shares, permuted by the same stream."""
    rng = np.random.default_rng(seed)
    pts = []
    U = rng.uniform(0.5, 4.0, count)
    T = rng.uniform(0.01, 0.1, count)
    de = rng.uniform(-1.0, 1.0, count)
    per = count // len(BATCH_SIZES)
    sizes = []
    for n in BATCH_SIZES:
        sizes += [n] * per
    sizes += [BATCH_SIZES[-1]] * (count - len(sizes))
    sizes = rng.permutation(np.array(sizes))
    for i in range(count):
        pts.append(Workload("batch%02d" % i, N=int(sizes[i]), U=float(U[i]),
                            T=float(T[i]), eps_d=float(-U[i] / 2 + de[i])))
    return pts


def _crossing_partner(N):
    """Flat index of the crossing partner (i2, i1, i4) of every (i1, i2, i3)
    whose fourth index lies in the box, and the mask of such entries."""
    i1, i2, i3 = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    i4 = i1 + i2 - i3
    ok = (i4 >= 0) & (i4 < N)
    part = (i2 * N + i1) * N + np.clip(i4, 0, N - 1)
    return part.reshape(-1), ok.reshape(-1)


def all_in_box_mask(N):
    """Boolean (N, N, N) mask of entries whose fourth index i4 lies in the box."""
    i1, i2, i3 = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    i4 = i1 + i2 - i3
    return (i4 >= 0) & (i4 < N)


def random_vertex(N: int, U: float, seed: int, amp: float = 0.3, smooth: bool = True,
                  crossing: bool = True):
    """Seeded complex vertex: U plus a smooth part in the three transfer
    frequencies plus noise.  With crossing=True (the default) it is symmetric
    under crossing (i1,i2,i3)->(i2,i1,i4) on entries whose fourth index is in
    the box, as every SU(2) vertex is; with crossing=False the noise is left as
    drawn, so the vertex breaks crossing (and frequency-reversal) symmetry
    everywhere -- the channel sums are defined for any vertex and the parity
    tests also feed such inputs."""
    rng = np.random.default_rng(seed)
    i1, i2, i3 = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    s = (i1 + i2 - (N - 1)).astype(np.float64)  # bosonic index, centred
    t = (i3 - i1).astype(np.float64)
    q = (i2 - i3).astype(np.float64)
    v = np.full((N, N, N), U, np.complex128)
    if smooth:
        w = max(N / 8.0, 1.0)
        a, b, c = rng.uniform(0.2, 1.0, 3)
        v += amp * U * (a / (1 + (s / w) ** 2) - b / (1 + (q / w) ** 2)
                        + 0.5 * c / (1 + (t / w) ** 2))
    v += amp * U * 0.2 * (rng.standard_normal((N, N, N))
                          + 1j * rng.standard_normal((N, N, N)))
    if not crossing:
        return v
    flat = v.reshape(-1)
    part, ok = _crossing_partner(N)
    sym = flat.copy()
    sym[ok] = 0.5 * (flat[ok] + flat[part[ok]])
    return sym.reshape(N, N, N)


def random_sigma(N: int, seed: int, amp: float = 0.1):
    """Seeded complex self-energy of shape (N,)."""
    rng = np.random.default_rng(seed)
    return amp * (rng.standard_normal(N) + 1j * rng.standard_normal(N))


def bare_state(N: int, U: float):
    """Initial state of the flow: vertex = U everywhere, self-energy = 0."""
    return np.full((N, N, N), U, np.complex128), np.zeros(N, np.complex128)
