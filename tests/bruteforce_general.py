"""Brute-force spin-resolved one-loop fRG right-hand side (test reference).

This is the general one-loop flow of an antisymmetric two-particle vertex
gamma(1'2'; 12), multi-index x = (spin, frequency), at second level of the
hierarchy with the three-particle vertex dropped, written out over every spin
and frequency label without using SU(2) or any channel reduction:

  d gamma(1'2';12)/dL = T sum_{3,4} [ -1/2 gamma(1'2';34) Lb(3,4) gamma(34;12)
                                       + gamma(1'4;13) Lb(3,4) gamma(32';42)
                                       - gamma(2'4;13) Lb(3,4) gamma(31';42) ]
  d Sigma(1)/dL = T sum_3 S(3) gamma(13;13)

with Lb(3,4) = S(3)G(4) + G(3)S(4) (propagators diagonal in spin), the
internal pair restricted to frequencies inside the box.  The two coefficients
(-1/2 for the particle-particle term, +1 for the particle-hole term, whose
exchange partner enters with the opposite sign so that the result stays
antisymmetric) are the ones for which the flow reproduces second-order
perturbation theory of the Hubbard-type interaction U n_up n_dn; the tests
check that property directly (bare vertex -> -U^2 d(B_pp + B_ph)/dL, and
Hartree for the self-energy).

The spin-resolved vertex is built from the up-down function V through the
SU(2) decomposition gamma = V(1'2';12) d(s1',s1) d(s2',s2)
- V(2'1';12) d(s1',s2) d(s2',s1), with V(1'2';12) = V(k1=w1, k2=w2, k3=w1')
read from the stored array when all four frequencies are in the box and the
bare U otherwise.  Pure-Python loops: use only on tiny grids (N <= 8).

With lo != 0 the internal pair runs over the frequency window
[lo, lo + len(G)) instead of the box (the frequency-box tail option); G and S
are then given on that window, G[w - lo].
"""
import numpy as np

UP, DN = 0, 1


class GeneralVertex:
    def __init__(self, V, U):
        self.V = np.asarray(V)
        self.N = self.V.shape[0]
        self.U = U

    def vf(self, o1, o2, i1, i2):
        """V(1'2';12) for frequency indices (out1, out2; in1, in2)."""
        N = self.N
        if o1 + o2 != i1 + i2:
            return 0.0
        for x in (o1, o2, i1, i2):
            if x < 0 or x >= N:
                return self.U
        return self.V[i1, i2, o1]

    def __call__(self, s1p, w1p, s2p, w2p, s1, w1, s2, w2):
        val = 0.0
        if s1p == s1 and s2p == s2:
            val += self.vf(w1p, w2p, w1, w2)
        if s1p == s2 and s2p == s1:
            val -= self.vf(w2p, w1p, w1, w2)
        return val


def general_rhs_entry(gv, G, S, T, ext, lo=0):
    """d gamma/dL at external labels ext = (s1',w1',s2',w2',s1,w1,s2,w2)."""
    s1p, w1p, s2p, w2p, s1, w1, s2, w2 = ext
    hi = lo + len(G)
    acc = 0.0
    for sa in (UP, DN):
        for sb in (UP, DN):
            for wa in range(lo, hi):
                # particle-particle: 3=(sa,wa), 4=(sb,wb), wa+wb = w1+w2
                wb = w1 + w2 - wa
                if lo <= wb < hi:
                    lb = S[wa - lo] * G[wb - lo] + G[wa - lo] * S[wb - lo]
                    acc += -0.5 * gv(s1p, w1p, s2p, w2p, sa, wa, sb, wb) * lb * \
                        gv(sa, wa, sb, wb, s1, w1, s2, w2)
                # direct particle-hole: gamma(1'4;13) gamma(32';42),
                # w1' + w4 = w1 + w3
                wb = w1 + wa - w1p
                if lo <= wb < hi:
                    lb = S[wa - lo] * G[wb - lo] + G[wa - lo] * S[wb - lo]
                    acc += gv(s1p, w1p, sb, wb, s1, w1, sa, wa) * lb * \
                        gv(sa, wa, s2p, w2p, sb, wb, s2, w2)
                # exchanged particle-hole: gamma(2'4;13) gamma(31';42),
                # w2' + w4 = w1 + w3
                wb = w1 + wa - w2p
                if lo <= wb < hi:
                    lb = S[wa - lo] * G[wb - lo] + G[wa - lo] * S[wb - lo]
                    acc -= gv(s2p, w2p, sb, wb, s1, w1, sa, wa) * lb * \
                        gv(sa, wa, s1p, w1p, sb, wb, s2, w2)
    return T * acc


def general_sigma_entry(gv, S, T, w, lo=0):
    """d Sigma_up(w)/dL."""
    acc = 0.0
    for sa in (UP, DN):
        for wa in range(lo, lo + len(S)):
            acc += S[wa - lo] * gv(UP, w, sa, wa, UP, w, sa, wa)
    return T * acc


def reduced_from_general(V, U, G, S, T, Lam, lo=0):
    """(dV/dl, dSigma/dl) obtained from the general formula: the up-down
    component d gamma(k3 up, k4 dn; k1 up, k2 dn)/dl for every stored entry."""
    gv = GeneralVertex(V, U)
    N = gv.N
    dV = np.zeros((N, N, N), np.complex128)
    for i1 in range(N):
        for i2 in range(N):
            for i3 in range(N):
                i4 = i1 + i2 - i3
                dV[i1, i2, i3] = Lam * general_rhs_entry(
                    gv, G, S, T, (UP, i3, DN, i4, UP, i1, DN, i2), lo)
    dS = np.array([Lam * general_sigma_entry(gv, S, T, w, lo) for w in range(N)])
    return dV, dS
