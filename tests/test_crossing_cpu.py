"""Host logic of the crossing reduction (FRG_CROSSING), no GPU: the tile rules
of the library (frg_cross_tile) cover every entry of a reduced transfer's
product exactly once, and every entry a tile writes for a partner is the image
of the entry it computed under crossing symmetry V(k1,k2,k3) = V(k2,k1,k4)
(composed with frequency reversal, n -> -n-1 with conjugation, for the two
particle-hole channels), written out on the vertex indices here.

Products of one transfer (index sets of the library's channel geometry):
  pp  transfer s = m:       rows k1 (k2 = s - k1),  columns k3
  dph transfer t = m-(N-1): rows k1 (k3 = k1 + t),  columns k2
  xph transfer Q = m-(N-1): rows k3 (k2 = k3 + Q),  columns k1
with the reversal reduction's transfers m <= N - 1."""
import numpy as np
import pytest

from paper_1510_07799_gb300 import frg

MROWS = 64


def vertex_index(ch, N, m, r, c):
    """(k1, k2, k3) of entry (row r counted from the transfer's first valid
    row, column c) of channel ch's product at transfer m <= N - 1."""
    if ch == 0:
        s = m
        k1 = r  # first valid row 0 for s <= N - 1
        return k1, s - k1, c
    t = m - (N - 1)
    if ch == 1:
        k1 = r - t  # first valid row -t
        return k1, c, k1 + t
    Q = t
    k3 = r - Q
    return c, k3 + Q, k3


def entry_of(ch, N, m, k):
    """Inverse of vertex_index: (row, column) of vertex index k in the product
    of transfer m, or None when k does not belong to it."""
    k1, k2, k3 = k
    if ch == 0:
        return (k1, k3) if k1 + k2 == m else None
    t = m - (N - 1)
    if ch == 1:
        return (k1 + t, k2) if k3 - k1 == t else None
    return (k3 + t, k1) if k2 - k3 == t else None


def partner(ch, N, k):
    """Crossing image of vertex index k (pp), composed with frequency reversal
    (dph, xph): the entry whose product value is the same (pp) or the
    conjugate (dph, xph)."""
    k1, k2, k3 = k
    k4 = k1 + k2 - k3
    c = (k2, k1, k4)
    if ch == 0:
        return c
    M = N - 1
    return (M - c[0], M - c[1], M - c[2])


def in_box(N, k):
    k1, k2, k3 = k
    return all(0 <= x < N for x in (k1, k2, k3, k1 + k2 - k3))


@pytest.mark.parametrize("N", [66, 80, 98, 100, 126, 128])
def test_reduced_tiles_write_every_entry_once(N):
    nt = (N + 15) // 16 * 16
    for ch in range(3):
        for m in range(MROWS, N):
            D = m + 1
            count = np.zeros((D, N), int)
            for rt in range(2):
                c0, w, own_lo, own_hi, m_lo, m_hi, m_row = frg.cross_tile(ch, N, nt, m, rt)
                if w == 0:
                    continue
                assert c0 % 2 == 0 and w % 16 == 0 and w <= 128  # aligned tensor-map x, MMA width
                assert c0 <= own_lo and own_hi <= min(N, c0 + w)  # own entries are computed
                rows = range(rt * MROWS, min(D, rt * MROWS + MROWS))
                for r in rows:
                    for c in range(max(c0, 0), min(N, c0 + w)):
                        if own_lo <= c < own_hi:
                            count[r, c] += 1
                        if m_lo <= c < m_hi and r <= m_row:
                            k = vertex_index(ch, N, m, r, c)
                            assert in_box(N, k)
                            p = partner(ch, N, k)
                            assert in_box(N, p), (ch, m, r, c)  # paired entries only
                            rc = entry_of(ch, N, m, p)
                            assert rc is not None, (ch, m, r, c)  # the partner is in the same product
                            pr, pc = rc
                            assert 0 <= pr < D and 0 <= pc < N
                            # written from a computed entry, never onto one this tile owns
                            assert not (rt * MROWS <= pr < rt * MROWS + MROWS and own_lo <= pc < own_hi)
                            count[pr, pc] += 1
            assert (count == 1).all(), (N, ch, m, np.argwhere(count != 1)[:4])


def test_entries_without_a_partner_are_computed():
    """An entry whose crossing image leaves the box (its fourth frequency
    outside) has no partner: every such entry is among a tile's own ones."""
    N, nt = 100, 112
    for ch in range(3):
        for m in range(MROWS, N):
            D = m + 1
            own = np.zeros((D, N), bool)
            for rt in range(2):
                c0, w, own_lo, own_hi, _, _, _ = frg.cross_tile(ch, N, nt, m, rt)
                for r in range(rt * MROWS, min(D, rt * MROWS + MROWS)):
                    own[r, max(own_lo, c0):min(own_hi, c0 + w)] = w > 0
            for r in range(D):
                for c in range(N):
                    k = vertex_index(ch, N, m, r, c)
                    if in_box(N, k) and not in_box(N, partner(ch, N, k)):
                        assert own[r, c], (ch, m, r, c)


@pytest.mark.parametrize("bad", [dict(ch=3), dict(rt=2), dict(N=130, nt=128), dict(m=63), dict(m=100),
                                 dict(nt=120), dict(N=99)])
def test_invalid_arguments_are_rejected(bad):
    a = dict(ch=0, N=100, nt=112, m=80, rt=0)
    a.update(bad)
    with pytest.raises(frg.FrgError) as e:
        frg.cross_tile(a["ch"], a["N"], a["nt"], a["m"], a["rt"])
    assert e.value.code == frg.EINVAL
