"""The seeded synthetic inputs (CPU): the workloads' parameters, the 64-point
batch recipe and the random vertices the parity tests and the benchmark use."""
import numpy as np
import pytest

from paper_1510_07799_gb300 import inputs


def test_workload_parameters():
    """The single-flow workloads: grid, U, T and the level shift eps~ =
    eps_d + U/2 (0 at particle-hole symmetry)."""
    expect = {  # name: (N, U, T, eps~, cutoff)
        inputs.SIAM_N16: (16, 1.0, 0.05, 0.0, 0),
        inputs.SIAM_N64: (64, 2.0, 0.01, 0.5, 0),
        inputs.SIAM_N128: (128, 3.0, 0.005, 0.0, 0),
        inputs.SIAM_N256: (256, 3.0, 0.002, 0.25, 0),
        inputs.SIAM_N64_IFLOW: (64, 2.0, 0.01, 0.5, 1),
    }
    for w, (N, U, T, et, cut) in expect.items():
        assert (w.N, w.U, w.T, w.cutoff) == (N, U, T, cut)
        assert abs(w.eps_d + w.U / 2 - et) < 1e-15
        assert w.name in inputs.WORKLOADS


def test_batch_recipe():
    """64 points from one seeded PCG64 stream: U in [0.5, 4], T in [0.01, 0.1],
    eps_d + U/2 in [-1, 1], each grid size of (32, 48, 64, 96) 16 times;
    the same seed gives the same batch, another seed another one."""
    pts = inputs.batch_points()
    assert len(pts) == 64
    U = np.array([p.U for p in pts])
    T = np.array([p.T for p in pts])
    et = np.array([p.eps_d + p.U / 2 for p in pts])
    assert U.min() >= 0.5 and U.max() <= 4.0
    assert T.min() >= 0.01 and T.max() <= 0.1
    assert et.min() >= -1.0 and et.max() <= 1.0
    sizes, counts = np.unique([p.N for p in pts], return_counts=True)
    assert list(sizes) == [32, 48, 64, 96] and list(counts) == [16] * 4
    again = inputs.batch_points()
    assert [(p.N, p.U, p.T, p.eps_d) for p in again] == [(p.N, p.U, p.T, p.eps_d) for p in pts]
    other = inputs.batch_points(seed=inputs.BATCH_SEED + 1)
    assert [p.U for p in other] != [p.U for p in pts]


@pytest.mark.parametrize("N", [4, 7, 16])
def test_random_vertex_is_seeded_and_crossing_symmetric(N):
    """V(i1, i2, i3) = V(i2, i1, i4) wherever i4 = i1 + i2 - i3 is in the
    box; the same seed gives the same array; values scatter around U."""
    U = 1.5
    V = inputs.random_vertex(N, U, seed=3)
    assert V.shape == (N, N, N) and V.dtype == np.complex128
    assert np.array_equal(V, inputs.random_vertex(N, U, seed=3))
    assert not np.array_equal(V, inputs.random_vertex(N, U, seed=4))
    for i1 in range(N):
        for i2 in range(N):
            for i3 in range(N):
                i4 = i1 + i2 - i3
                if 0 <= i4 < N:
                    assert V[i1, i2, i3] == V[i2, i1, i4]
    assert abs(np.mean(V) - U) < U
    assert np.max(np.abs(V.imag)) > 0


@pytest.mark.parametrize("N", [4, 16])
def test_random_vertex_without_crossing_breaks_both_symmetries(N):
    """crossing=False leaves the seeded noise as drawn: crossing and frequency
    reversal with conjugation fail on almost every in-box entry, so a path
    that read an operand through either symmetry would see other values."""
    U = 1.5
    V = inputs.random_vertex(N, U, seed=3, crossing=False)
    assert np.array_equal(V, inputs.random_vertex(N, U, seed=3, crossing=False))
    i1, i2, i3 = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    i4 = i1 + i2 - i3
    ok = (i4 >= 0) & (i4 < N) & ((i1 != i2) | (i3 != i4))
    crossed = V[i2[ok], i1[ok], i4[ok]]
    assert np.mean(V[ok] != crossed) > 0.99
    assert np.mean(V != np.conj(V[::-1, ::-1, ::-1])) > 0.99


def test_bare_state_and_random_sigma():
    g, s = inputs.bare_state(6, 2.0)
    assert np.array_equal(g, np.full((6, 6, 6), 2.0 + 0j)) and np.array_equal(s, np.zeros(6, complex))
    a = inputs.random_sigma(8, seed=1)
    assert a.shape == (8,) and np.array_equal(a, inputs.random_sigma(8, seed=1))
