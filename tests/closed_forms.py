"""Closed-form references for the oracle's pins (test side).

Free propagator of the wide-band SIAM with the Omega-scheme regulator,
G_L(w) = Theta_L(w) G0(w), Theta_L = w^2/(w^2+L^2), G0 = 1/(iw - et + i Delta sgn w),
and the bubbles built from it.  The propagator itself is pinned separately
(Lorentzian spectral representation, limits, finite differences).
"""
import numpy as np


def freqs(N, T):
    n = np.arange(N) - N // 2
    return (2 * n + 1) * np.pi * T


def g_free(N, T, et, Delta, Lam, cutoff=0):
    """Free propagator; cutoff 0: Omega scheme, 1: interaction flow
    (Theta = 1/sqrt(Lambda), Lambda = 1/g)."""
    w = freqs(N, T)
    th = 1.0 / np.sqrt(Lam) if cutoff else w ** 2 / (w ** 2 + Lam ** 2)
    return th / (1j * w - et + 1j * Delta * np.sign(w))


def bubble_pp(G, T):
    """B_pp[s] = T sum_{p, s-p in box} G(p) G(s-p), s = 0..2N-2."""
    N = G.size
    B = np.zeros(2 * N - 1, np.complex128)
    for s in range(2 * N - 1):
        for p in range(N):
            q = s - p
            if 0 <= q < N:
                B[s] += G[p] * G[q]
    return T * B


def bubble_ph(G, T):
    """B_ph[Q + N - 1] = T sum_{p, p+Q in box} G(p) G(p+Q), Q = -(N-1)..N-1."""
    N = G.size
    B = np.zeros(2 * N - 1, np.complex128)
    for Q in range(-(N - 1), N):
        for p in range(N):
            r = p + Q
            if 0 <= r < N:
                B[Q + N - 1] += G[p] * G[r]
    return T * B


def transfer_indices(N):
    i1, i2, i3 = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    s = i1 + i2
    Q = i2 - i3 + N - 1
    return s, Q


def second_order_vertex(N, T, et, Delta, U, Lam0, Lamf, cutoff=0):
    G0 = g_free(N, T, et, Delta, Lam0, cutoff)
    G1 = g_free(N, T, et, Delta, Lamf, cutoff)
    dBpp = bubble_pp(G1, T) - bubble_pp(G0, T)
    dBph = bubble_ph(G1, T) - bubble_ph(G0, T)
    s, Q = transfer_indices(N)
    return U - U ** 2 * dBpp[s] - U ** 2 * dBph[Q], dBpp[s], dBph[Q]


def first_order_sigma(N, T, et, Delta, U, Lam0, Lamf, cutoff=0):
    G0 = g_free(N, T, et, Delta, Lam0, cutoff)
    G1 = g_free(N, T, et, Delta, Lamf, cutoff)
    return np.full(N, U * T * np.sum(G1 - G0), np.complex128)


# ---------------------------------------------- frequency-box tails ----
# With the tail option the internal sums run over a window of W = factor * N
# Matsubara indices centred on the box, [lo, lo + W) with lo = -(W - N) / 2.

def window(N, factor):
    W = factor * N
    return -(W - N) // 2, W


def g_free_window(N, factor, T, et, Delta, Lam):
    lo, W = window(N, factor)
    n = np.arange(lo, lo + W) - N // 2
    w = (2 * n + 1) * np.pi * T
    th = w ** 2 / (w ** 2 + Lam ** 2)
    return th / (1j * w - et + 1j * Delta * np.sign(w))


def bubble_pp_window(Gw, N, factor, T):
    """B_pp[s] = T sum_{p, s-p in the window} G(p) G(s-p), s = 0..2N-2."""
    lo, W = window(N, factor)
    B = np.zeros(2 * N - 1, np.complex128)
    for s in range(2 * N - 1):
        for p in range(lo, lo + W):
            q = s - p
            if lo <= q < lo + W:
                B[s] += Gw[p - lo] * Gw[q - lo]
    return T * B


def bubble_ph_window(Gw, N, factor, T):
    """B_ph[Q + N - 1] = T sum_{p, p+Q in the window} G(p) G(p+Q)."""
    lo, W = window(N, factor)
    B = np.zeros(2 * N - 1, np.complex128)
    for Q in range(-(N - 1), N):
        for p in range(lo, lo + W):
            r = p + Q
            if lo <= r < lo + W:
                B[Q + N - 1] += Gw[p - lo] * Gw[r - lo]
    return T * B


def second_order_vertex_window(N, factor, T, et, Delta, U, Lam0, Lamf):
    G0 = g_free_window(N, factor, T, et, Delta, Lam0)
    G1 = g_free_window(N, factor, T, et, Delta, Lamf)
    dBpp = bubble_pp_window(G1, N, factor, T) - bubble_pp_window(G0, N, factor, T)
    dBph = bubble_ph_window(G1, N, factor, T) - bubble_ph_window(G0, N, factor, T)
    s, Q = transfer_indices(N)
    return U - U ** 2 * dBpp[s] - U ** 2 * dBph[Q]


def first_order_sigma_window(N, factor, T, et, Delta, U, Lam0, Lamf):
    G0 = g_free_window(N, factor, T, et, Delta, Lam0)
    G1 = g_free_window(N, factor, T, et, Delta, Lamf)
    return np.full(N, U * T * np.sum(G1 - G0), np.complex128)
