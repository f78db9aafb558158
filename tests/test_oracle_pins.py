"""Pins of the FP64 CPU oracle against facts fixed outside the oracle.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, a wrong index, a transposed operand, a mistyped coefficient) makes
at least one of them fail:
  * propagator:   Lorentzian spectral representation of the wide-band G0,
                  regulator limits, S = dG/dLambda by finite differences;
  * U = 0:        nothing flows;
  * O(U^2):       second-order perturbation theory for the vertex (Cooper
                  screening + transverse particle-hole), O(U) Hartree for Sigma,
                  with the U^3 / U^2 scaling of the remainder;
  * ladders:      exact single-channel solutions U/(1 + U dB);
  * brute force:  the general spin-resolved one-loop rhs on tiny grids;
  * symmetries:   crossing, frequency reversal, particle-hole reality;
  * integrator:   Dormand-Prince order conditions, fifth-order convergence,
                  closed-form linear ODEs, seven evaluations for the first step
                  (the paper, Sec. 4).
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle import Model
from paper_1510_07799_gb300 import inputs

import bruteforce_general as bf
import closed_forms as cf


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


# ------------------------------------------------------------ propagator ----

def test_free_propagator_is_lorentzian_hilbert_transform():
    """Wide-band G0(iw) = int d eps A(eps)/(iw - eps) with a Lorentzian A of
    half-width Delta centred at et.  At Lambda -> 0 the regulated G -> G0."""
    m = Model(U=2.0, T=0.03, eps_d=-1.0 + 0.4, Delta=0.7, N=8)
    et = m.eps_d + m.U / 2
    G, _ = oracle.propagators(m, 1e-9)
    for i, w in enumerate(cf.freqs(m.N, m.T)):
        A = lambda e: (m.Delta / np.pi) / ((e - et) ** 2 + m.Delta ** 2)
        re = integrate.quad(lambda e: A(e) * (-e) / (w ** 2 + e ** 2), -np.inf, np.inf,
                            epsabs=1e-13, epsrel=1e-12)[0]
        im = integrate.quad(lambda e: A(e) * (-w) / (w ** 2 + e ** 2), -np.inf, np.inf,
                            epsabs=1e-13, epsrel=1e-12)[0]
        assert abs(G[i] - complex(re, im)) < 1e-9


def test_regulator_limits():
    m = Model(U=1.0, T=0.05, eps_d=-0.3, Delta=1.0, N=10)
    G_big, _ = oracle.propagators(m, 1e8)
    assert np.max(np.abs(G_big)) < 1e-12
    w = cf.freqs(m.N, m.T)
    G_at_w, _ = oracle.propagators(m, abs(w[m.N // 2]))
    G0, _ = oracle.propagators(m, 0.0)
    # Theta(w = Lambda) = 1/2 at the frequency equal to the scale
    assert abs(G_at_w[m.N // 2] - 0.5 * G0[m.N // 2]) < 1e-14


@pytest.mark.parametrize("Lam", [0.05, 0.7, 3.0])
def test_single_scale_is_scale_derivative(Lam):
    """S = dG/dLambda at fixed Sigma (central differences)."""
    m = Model(U=1.5, T=0.04, eps_d=-0.2, Delta=1.0, N=12)
    sig = inputs.random_sigma(m.N, seed=11, amp=0.2)
    _, S = oracle.propagators(m, Lam, sig)
    h = 1e-5 * Lam
    Gp, _ = oracle.propagators(m, Lam + h, sig)
    Gm, _ = oracle.propagators(m, Lam - h, sig)
    fd = (Gp - Gm) / (2 * h)
    assert rel(S, fd) < 1e-8


# ------------------------------------------------------------------ U = 0 ----

def test_u_zero_stays_trivial():
    m = Model(U=0.0, T=0.05, eps_d=0.3, Delta=1.0, N=8)
    g, s, st = oracle.flow(m)
    assert st.status == 0
    assert np.max(np.abs(g)) == 0.0 and np.max(np.abs(s)) == 0.0


# --------------------------------------------------- perturbation theory ----

@pytest.mark.parametrize("eps_shift", [0.0, 0.6])
def test_second_order_perturbation_theory(eps_shift):
    """Gamma - [U - U^2 dB_pp(s) - U^2 dB_ph(Q)] = O(U^3) on every entry and
    Sigma - U T sum [G] = O(U^2); the remainders shrink by 8x / 4x when U halves."""
    N, T, D = 8, 0.05, 1.0
    L0, Lf = 1e3, 1e-2
    devs, sdevs = [], []
    Us = [0.04, 0.02, 0.01]
    for U in Us:
        m = Model(U=U, T=T, eps_d=-U / 2 + eps_shift, Delta=D, N=N)
        g, s, st = oracle.flow(m, Lambda0=L0, Lambda_f=Lf, rtol=1e-12, atol=1e-16)
        assert st.status == 0
        ref, _, _ = cf.second_order_vertex(N, T, eps_shift, D, U, L0, Lf)
        sref = cf.first_order_sigma(N, T, eps_shift, D, U, L0, Lf)
        devs.append(np.max(np.abs(g - ref)))
        sdevs.append(np.max(np.abs(s - sref)))
    # second order itself is resolved: |U^2 dB| >> remainder
    _, dBpp, dBph = cf.second_order_vertex(N, T, eps_shift, D, 1.0, L0, Lf)
    assert np.max(np.abs(dBpp)) > 1e-2 and np.max(np.abs(dBph)) > 1e-2
    for a, b in zip(devs, devs[1:]):
        assert 6.5 < a / b < 9.5, devs
    for a, b in zip(sdevs, sdevs[1:]):
        assert 3.2 < a / b < 4.8, sdevs
    if eps_shift == 0.0:
        # the O(U) Hartree term vanishes at particle-hole symmetry
        sref = cf.first_order_sigma(N, T, 0.0, D, 1.0, L0, Lf)
        assert np.max(np.abs(sref)) < 1e-15


# ----------------------------------------------------------- observables ----

def test_observables_of_the_bare_state():
    """Bare vertex, no self-energy: U_eff = U, Z = 1, Sigma(pi T) = 0."""
    N, U = 8, 1.7
    m = Model(U=U, T=0.04, eps_d=-U / 2 + 0.3, Delta=1.0, N=N)
    o = oracle.observables(m, 1e-3, np.full((N, N, N), U, np.complex128), np.zeros(N, np.complex128))
    assert o["U_eff"] == U and o["Z"] == 1.0 and o["sigma_lowest"] == 0.0


def test_quasiparticle_weight_of_a_linear_self_energy():
    """Fermi-liquid form Sigma(i w_n) = -i a_n w_n: Z = 1 / (1 + a) at the lowest
    positive Matsubara frequency w = pi T (index N/2); a different a_n on every
    frequency pins which one the observable reads."""
    N, T = 10, 0.03
    m = Model(U=1.0, T=T, eps_d=-0.5, Delta=1.0, N=N)
    w = cf.freqs(N, T)
    a = 0.1 + 0.05 * np.arange(N)
    sig = -1j * a * w
    o = oracle.observables(m, 1e-3, np.full((N, N, N), 1.0, np.complex128), sig)
    i0 = N // 2
    assert abs(w[i0] - np.pi * T) < 1e-15
    assert abs(o["Z"] - 1.0 / (1.0 + a[i0])) < 1e-14
    assert o["sigma_lowest"] == sig[i0]


def test_effective_interaction_of_the_pp_ladder():
    """U_eff is the vertex at n1 = n2 = n3 = 0 (all external frequencies pi T):
    after a pp-only flow it equals the ladder value U / (1 + U dB_pp(s)) at
    s = i1 + i2 = N, the bosonic transfer of two frequencies pi T."""
    N, T, D, U = 10, 0.05, 1.0, 2.5
    m = Model(U=U, T=T, eps_d=-U / 2, Delta=D, N=N)
    g, s, st = oracle.flow(m, mask=0x1, rtol=1e-11, atol=1e-14)
    o = oracle.observables(m, 1e-3, g, s)
    _, dBpp, _ = cf.second_order_vertex(N, T, 0.0, D, 1.0, 1e3, 1e-3)
    ref = U / (1 + U * dBpp)
    i0 = N // 2
    assert abs(o["U_eff"] - ref[i0, i0, i0]) / abs(ref[i0, i0, i0]) < 2e-8
    assert abs(ref[i0, i0, i0] - U) / U > 0.05


# ------------------------------------------------------- ladder solutions ----

def _aib(N):
    return inputs.all_in_box_mask(N)


@pytest.mark.parametrize("eps_shift", [0.0, 0.5])
def test_pp_ladder_closed_form(eps_shift):
    """pp channel alone, Sigma frozen: V depends only on s and equals
    U / (1 + U dB_pp(s)) on every entry whose four frequencies are in the box."""
    N, T, D, U = 10, 0.05, 1.0, 2.5
    m = Model(U=U, T=T, eps_d=-U / 2 + eps_shift, Delta=D, N=N)
    g, s, st = oracle.flow(m, mask=0x1, rtol=1e-11, atol=1e-14)
    assert st.status == 0 and np.max(np.abs(s)) == 0.0
    _, dBpp, _ = cf.second_order_vertex(N, T, eps_shift, D, 1.0, 1e3, 1e-3)
    ref = U / (1 + U * dBpp)
    mk = _aib(N)
    assert rel(g[mk], ref[mk]) < 2e-8
    assert rel(ref[mk], U) > 0.05  # far from the bare value: the test has teeth


@pytest.mark.parametrize("eps_shift", [0.0, 0.5])
def test_xph_ladder_closed_form(eps_shift):
    N, T, D, U = 10, 0.05, 1.0, 1.2
    m = Model(U=U, T=T, eps_d=-U / 2 + eps_shift, Delta=D, N=N)
    g, s, st = oracle.flow(m, mask=0x4, rtol=1e-11, atol=1e-14)
    assert st.status == 0
    _, _, dBph = cf.second_order_vertex(N, T, eps_shift, D, 1.0, 1e3, 1e-3)
    ref = U / (1 + U * dBph)
    mk = _aib(N)
    assert rel(g[mk], ref[mk]) < 2e-8
    assert rel(ref[mk], U) > 0.05


def test_dph_alone_keeps_bare_vertex():
    N, U = 8, 2.0
    m = Model(U=U, T=0.05, eps_d=-U / 2 + 0.3, Delta=1.0, N=N)
    g, s, st = oracle.flow(m, mask=0x2)
    assert st.status == 0
    assert np.max(np.abs(g - U)) < 1e-14


# ------------------------------------------------------------ brute force ----

@pytest.mark.parametrize("N,seed,eps_shift", [(4, 1, 0.0), (6, 2, 0.4), (8, 3, -0.7)])
def test_reduced_rhs_matches_spin_resolved_general_formula(N, seed, eps_shift):
    U, T, Lam = 1.3, 0.07, 0.37
    m = Model(U=U, T=T, eps_d=-U / 2 + eps_shift, Delta=1.0, N=N)
    V = inputs.random_vertex(N, U, seed=seed, amp=0.4)
    sig = inputs.random_sigma(N, seed=seed + 100, amp=0.15)
    dg, ds = oracle.rhs(m, Lam, V, sig)
    G, S = oracle.propagators(m, Lam, sig)
    dgb, dsb = bf.reduced_from_general(V, U, G, S, T, Lam)
    assert rel(dg, dgb) < 1e-13
    assert rel(ds, dsb) < 1e-13


def test_general_formula_coefficients_reproduce_perturbation_theory():
    """At the bare vertex the general formula gives -U^2 d(B_pp + B_ph)/dL for
    the up-down component and U T sum S for Sigma (the two conditions that fix
    its coefficients)."""
    N, U, T, Lam = 6, 0.9, 0.06, 0.5
    m = Model(U=U, T=T, eps_d=-U / 2 + 0.3, Delta=1.0, N=N)
    G, S = oracle.propagators(m, Lam)
    gv = bf.GeneralVertex(np.full((N, N, N), U, np.complex128), U)
    h = 1e-6
    Gp, _ = oracle.propagators(m, Lam + h)
    Gm, _ = oracle.propagators(m, Lam - h)
    dBpp = (cf.bubble_pp(Gp, T) - cf.bubble_pp(Gm, T)) / (2 * h)
    dBph = (cf.bubble_ph(Gp, T) - cf.bubble_ph(Gm, T)) / (2 * h)
    for (i1, i2, i3) in [(0, 0, 0), (1, 4, 2), (5, 5, 3), (2, 3, 5), (0, 5, 1)]:
        i4 = i1 + i2 - i3
        val = bf.general_rhs_entry(gv, G, S, T, (bf.UP, i3, bf.DN, i4, bf.UP, i1, bf.DN, i2))
        ref = -U ** 2 * (dBpp[i1 + i2] + dBph[i2 - i3 + N - 1])
        assert abs(val - ref) < 1e-7 * max(1.0, abs(ref))
    for w in range(N):
        assert abs(bf.general_sigma_entry(gv, S, T, w) - U * T * np.sum(S)) < 1e-14


def test_general_formula_is_antisymmetric_and_su2():
    N, U, T, Lam = 4, 1.1, 0.08, 0.6
    m = Model(U=U, T=T, eps_d=-U / 2 + 0.2, Delta=1.0, N=N)
    V = inputs.random_vertex(N, U, seed=5, amp=0.5)
    G, S = oracle.propagators(m, Lam)
    gv = bf.GeneralVertex(V, U)
    rng = np.random.default_rng(9)
    for _ in range(12):
        w1, w2, w1p = rng.integers(0, N, 3)
        w2p = w1 + w2 - w1p
        if not 0 <= w2p < N:
            continue
        sp = rng.integers(0, 2, 4)
        a = bf.general_rhs_entry(gv, G, S, T, (sp[0], w1p, sp[1], w2p, sp[2], w1, sp[3], w2))
        b = bf.general_rhs_entry(gv, G, S, T, (sp[1], w2p, sp[0], w1p, sp[2], w1, sp[3], w2))
        assert abs(a + b) < 1e-13
        # SU(2): up-up component = up-down minus its exchange
        uu = bf.general_rhs_entry(gv, G, S, T, (0, w1p, 0, w2p, 0, w1, 0, w2))
        ud = bf.general_rhs_entry(gv, G, S, T, (0, w1p, 1, w2p, 0, w1, 1, w2))
        ud_x = bf.general_rhs_entry(gv, G, S, T, (0, w2p, 1, w1p, 0, w1, 1, w2))
        assert abs(uu - (ud - ud_x)) < 1e-13


# ------------------------------------------------------------- symmetries ----

def _crossing_err(g):
    N = g.shape[0]
    e = 0.0
    for i1 in range(N):
        for i2 in range(N):
            for i3 in range(N):
                i4 = i1 + i2 - i3
                if 0 <= i4 < N:
                    e = max(e, abs(g[i1, i2, i3] - g[i2, i1, i4]))
    return e


@pytest.mark.parametrize("eps_shift", [0.0, 0.5])
def test_flow_symmetries(eps_shift):
    N, U = 12, 2.0
    m = Model(U=U, T=0.05, eps_d=-U / 2 + eps_shift, Delta=1.0, N=N)
    g, s, st = oracle.flow(m)
    assert st.status == 0
    mk = _aib(N)
    scale = np.max(np.abs(g))
    assert _crossing_err(g) < 1e-12 * scale
    # frequency reversal n -> -n-1 (i -> N-1-i) with complex conjugation
    rev = np.conj(g[::-1, ::-1, ::-1])
    assert np.max(np.abs((g - rev)[mk])) < 1e-12 * scale
    assert np.max(np.abs(s - np.conj(s[::-1]))) < 1e-14
    if eps_shift == 0.0:
        assert np.max(np.abs(g.imag)) < 1e-14 * scale
        assert np.max(np.abs(s.real)) < 1e-15
    else:
        assert np.max(np.abs(g.imag)) > 1e-3
        assert np.max(np.abs(s.real)) > 1e-3


# ------------------------------------------------------------- integrator ----

def test_dp5_order_conditions():
    c, a, b, bs = oracle.dp5_tableau()
    A = np.zeros((7, 7))
    A[:, :6] = a
    assert np.allclose(A.sum(axis=1), c, atol=1e-15, rtol=0)
    assert np.allclose(A[6], b, atol=0, rtol=0)  # first same as last
    ac = A @ c
    conds5 = [
        (b.sum(), 1), (b @ c, 1 / 2), (b @ c ** 2, 1 / 3), (b @ ac, 1 / 6),
        (b @ c ** 3, 1 / 4), (b @ (c * ac), 1 / 8), (b @ (A @ c ** 2), 1 / 12),
        (b @ (A @ ac), 1 / 24), (b @ c ** 4, 1 / 5), (b @ (c ** 2 * ac), 1 / 10),
        (b @ ac ** 2, 1 / 20), (b @ (c * (A @ c ** 2)), 1 / 15),
        (b @ (c * (A @ ac)), 1 / 30), (b @ (A @ c ** 3), 1 / 20),
        (b @ (A @ (c * ac)), 1 / 40), (b @ (A @ (A @ c ** 2)), 1 / 60),
        (b @ (A @ (A @ ac)), 1 / 120)]
    for got, want in conds5:
        assert abs(got - want) < 1e-14
    for got, want in [(bs.sum(), 1), (bs @ c, 1 / 2), (bs @ c ** 2, 1 / 3),
                      (bs @ ac, 1 / 6), (bs @ c ** 3, 1 / 4), (bs @ (c * ac), 1 / 8),
                      (bs @ (A @ c ** 2), 1 / 12), (bs @ (A @ ac), 1 / 24)]:
        assert abs(got - want) < 1e-14
    # the embedded pair differs (otherwise the error estimate is void)
    assert np.max(np.abs(b - bs)) > 1e-3


def _lin(lmb):
    M = np.array([[lmb.real, -lmb.imag], [lmb.imag, lmb.real]])
    return lambda t, y: M @ y


def test_dp5_fifth_order_convergence():
    lmb = complex(-1.0, 2.0)
    exact = np.exp(lmb)
    errs = []
    for n in (8, 16, 32):
        y, st = oracle.dp5_integrate(_lin(lmb), [1.0, 0.0], 0.0, 1.0, fixed_h=1.0 / n)
        errs.append(abs(complex(y[0], y[1]) - exact))
        assert st.accepted == n and st.rhs_evals == 6 * n + 1
    for a, b in zip(errs, errs[1:]):
        assert 4.6 < math.log2(a / b) < 5.4, errs


@pytest.mark.parametrize("lmb", [complex(-2.0, 0.0), complex(0.0, 3.0), complex(-0.5, -5.0)])
def test_dp5_adaptive_linear_closed_form(lmb):
    y, st = oracle.dp5_integrate(_lin(lmb), [1.0, 0.0], 0.0, 2.0, rtol=1e-9, atol=1e-12,
                                 h0=0.01)
    assert st.status == 0 and abs(st.Lambda - 2.0) == 0.0
    assert abs(complex(y[0], y[1]) - np.exp(2 * lmb)) < 5e-8 * max(1, abs(np.exp(2 * lmb)))
    # backwards in t reproduces the inverse map
    y2, st2 = oracle.dp5_integrate(_lin(lmb), y, 2.0, 0.0, rtol=1e-9, atol=1e-12, h0=-0.01)
    assert abs(complex(y2[0], y2[1]) - 1.0) < 5e-7


def test_first_step_costs_seven_rhs_evaluations():
    """The paper (Sec. 4): the first step of the explicit stepper needs seven
    complete rhs evaluations."""
    m = Model(U=1.0, T=0.05, eps_d=-0.5, Delta=1.0, N=6)
    _, _, st = oracle.flow(m)
    assert st.first_step_evals == 7
    # afterwards first-same-as-last: six new evaluations per attempted step
    assert st.rhs_evals == 7 + 6 * (st.accepted + st.rejected - 1)


# -------------------------------------------------- internal consistency ----

def test_entry_and_row_evaluations_agree_with_full_rhs():
    N, U = 10, 1.7
    m = Model(U=U, T=0.04, eps_d=-U / 2 + 0.3, Delta=1.0, N=N)
    V = inputs.random_vertex(N, U, seed=21)
    sig = inputs.random_sigma(N, seed=22)
    dg, _ = oracle.rhs(m, 0.8, V, sig)
    rng = np.random.default_rng(4)
    idx = rng.integers(0, N, (50, 3))
    e = oracle.rhs_entries(m, 0.8, V, sig, idx)
    assert np.array_equal(e, dg[idx[:, 0], idx[:, 1], idx[:, 2]])
    r = oracle.rhs_rows(m, 0.8, V, sig, 3, 7)
    assert np.array_equal(r[3:7], dg[3:7]) and np.all(r[:3] == 0) and np.all(r[7:] == 0)


# ----------------------------------------------- frequency-box tails ----
# With mask bit MASK_TAILS the internal sums run over a window of
# TAIL_FACTOR * N Matsubara indices centred on the box (Sigma = 0 outside the
# box, bare-U vertices as soon as an index leaves the box).

TAILS = oracle.MASK_TAILS


def window_propagators(m, Lam, sigma):
    """(Gw, Sw, lo) on the tail window: the window's frequencies are exactly
    those of a box of W = TAIL_FACTOR * N indices, so the oracle's propagators
    of that larger model (with the self-energy padded by zeros) are the window's."""
    N = m.N
    W = oracle.TAIL_FACTOR * N
    lo = -(W - N) // 2
    sw = np.zeros(W, np.complex128)
    sw[-lo:-lo + N] = sigma
    mw = Model(U=m.U, T=m.T, eps_d=m.eps_d, Delta=m.Delta, N=W)
    Gw, Sw = oracle.propagators(mw, Lam, sw)
    return Gw, Sw, lo


def tail_constants(m, Lam, sigma):
    """Every vertex with an internal index outside the box is the bare U, so
    the window's extra terms are U^2 times bubble sums per transfer (pp and
    xph), 2U^2 - U^2 - U^2 = 0 for dph, and U times a sum of S for Sigma."""
    N = m.N
    Gw, Sw, lo = window_propagators(m, Lam, sigma)
    W = Gw.size
    box = lambda i: 0 <= i < N
    win = lambda i: lo <= i < lo + W
    lb = lambda a, b: Sw[a - lo] * Gw[b - lo] + Gw[a - lo] * Sw[b - lo]
    cpp = np.zeros(2 * N - 1, np.complex128)
    cxph = np.zeros(2 * N - 1, np.complex128)
    for s in range(2 * N - 1):
        for p in range(lo, lo + W):
            q = s - p
            if win(q) and not (box(p) and box(q)):
                cpp[s] += lb(p, q)
    for Q in range(-(N - 1), N):
        for p in range(lo, lo + W):
            r = p + Q
            if win(r) and not (box(p) and box(r)):
                cxph[Q + N - 1] += lb(p, r)
    csig = sum(Sw[p - lo] for p in range(lo, lo + W) if not box(p))
    return cpp, cxph, csig


@pytest.mark.parametrize("mask", [0xF, 0x1, 0x2, 0x4, 0x8])
def test_tails_add_a_constant_per_transfer(mask):
    N, U, T, Lam = 8, 1.4, 0.06, 0.45
    m = Model(U=U, T=T, eps_d=-U / 2 + 0.35, Delta=1.0, N=N)
    V = inputs.random_vertex(N, U, seed=11, amp=0.4)
    sig = inputs.random_sigma(N, seed=12, amp=0.2)
    dg0, ds0 = oracle.rhs(m, Lam, V, sig, mask)
    dg1, ds1 = oracle.rhs(m, Lam, V, sig, mask | TAILS)
    cpp, cxph, csig = tail_constants(m, Lam, sig)
    s, Q = cf.transfer_indices(N)
    ref = np.zeros((N, N, N), np.complex128)
    if mask & 1:
        ref += -Lam * T * U ** 2 * cpp[s]
    if mask & 4:
        ref += -Lam * T * U ** 2 * cxph[Q]
    sref = np.full(N, Lam * T * U * csig if mask & 8 else 0.0, np.complex128)
    scale = max(np.max(np.abs(dg0)), 1e-3)
    assert np.max(np.abs((dg1 - dg0) - ref)) < 1e-13 * scale
    assert np.max(np.abs((ds1 - ds0) - sref)) < 1e-15
    if mask & 5:
        assert np.max(np.abs(ref)) > 1e-3 * scale  # the tails are resolved
    if mask & 8:
        assert abs(csig) > 1e-6  # off particle-hole symmetry the Hartree tail is nonzero


@pytest.mark.parametrize("N,seed,eps_shift", [(4, 21, 0.0), (6, 22, 0.5)])
def test_tails_match_spin_resolved_general_formula(N, seed, eps_shift):
    U, T, Lam = 1.2, 0.08, 0.3
    m = Model(U=U, T=T, eps_d=-U / 2 + eps_shift, Delta=1.0, N=N)
    V = inputs.random_vertex(N, U, seed=seed, amp=0.4)
    sig = inputs.random_sigma(N, seed=seed + 100, amp=0.15)
    dg, ds = oracle.rhs(m, Lam, V, sig, 0xF | TAILS)
    Gw, Sw, lo = window_propagators(m, Lam, sig)
    dgb, dsb = bf.reduced_from_general(V, U, Gw, Sw, T, Lam, lo)
    assert rel(dg, dgb) < 1e-13
    assert rel(ds, dsb) < 1e-13 or np.max(np.abs(ds - dsb)) < 1e-16


@pytest.mark.parametrize("eps_shift", [0.0, 0.6])
def test_tails_second_order_perturbation_theory(eps_shift):
    """With the tails the O(U^2) vertex and the O(U) Hartree term take the
    bubbles over the whole window."""
    N, T, D, F = 8, 0.05, 1.0, oracle.TAIL_FACTOR
    L0, Lf = 1e3, 1e-2
    devs, sdevs = [], []
    for U in [0.04, 0.02, 0.01]:
        m = Model(U=U, T=T, eps_d=-U / 2 + eps_shift, Delta=D, N=N)
        g, s, st = oracle.flow(m, Lambda0=L0, Lambda_f=Lf, rtol=1e-12, atol=1e-16, mask=0xF | TAILS)
        assert st.status == 0
        ref = cf.second_order_vertex_window(N, F, T, eps_shift, D, U, L0, Lf)
        sref = cf.first_order_sigma_window(N, F, T, eps_shift, D, U, L0, Lf)
        devs.append(np.max(np.abs(g - ref)))
        sdevs.append(np.max(np.abs(s - sref)))
        # the window changes the second-order result: the box-only reference misses it
        box_ref, _, _ = cf.second_order_vertex(N, T, eps_shift, D, U, L0, Lf)
        assert np.max(np.abs(ref - box_ref)) > 20 * devs[-1]
    for a, b in zip(devs, devs[1:]):
        assert 6.5 < a / b < 9.5, devs
    if eps_shift != 0.0:
        for a, b in zip(sdevs, sdevs[1:]):
            assert 3.2 < a / b < 4.8, sdevs


def test_tails_keep_the_flow_symmetries():
    N, U = 8, 2.0
    m = Model(U=U, T=0.05, eps_d=-U / 2 + 0.5, Delta=1.0, N=N)
    g, s, st = oracle.flow(m, mask=0xF | TAILS)
    assert st.status == 0
    scale = np.max(np.abs(g))
    assert _crossing_err(g) < 1e-12 * scale
    mk = _aib(N)
    rev = np.conj(g[::-1, ::-1, ::-1])
    assert np.max(np.abs((g - rev)[mk])) < 1e-12 * scale
    assert np.max(np.abs(s - np.conj(s[::-1]))) < 1e-14
    mp = Model(U=U, T=0.05, eps_d=-U / 2, Delta=1.0, N=N)
    gp, sp, st = oracle.flow(mp, mask=0xF | TAILS)
    assert st.status == 0
    assert np.max(np.abs(gp.imag)) < 1e-14 * np.max(np.abs(gp))
    assert np.max(np.abs(sp.real)) < 1e-15


# ------------------------------------------------- frequency reversal ----

@pytest.mark.parametrize("mask", [0xF, 0x1, 0x2, 0x4, 0x8, 0xF | TAILS])
def test_rhs_keeps_the_reversal_symmetry_on_every_entry(mask):
    """For V(N-1-i1, N-1-i2, N-1-i3) = conj V(i1, i2, i3) and
    Sigma(N-1-i) = conj Sigma(i) the rhs has the same symmetry, channel by
    channel, on every stored entry (also those whose fourth index leaves the
    box): what the library's reversal reduction rests on."""
    N, U = 10, 1.3
    m = Model(U=U, T=0.05, eps_d=-U / 2 + 0.4, Delta=1.0, N=N)
    V = inputs.random_vertex(N, U, seed=31)
    V = 0.5 * (V + np.conj(V[::-1, ::-1, ::-1]))
    s = inputs.random_sigma(N, seed=32)
    s = 0.5 * (s + np.conj(s[::-1]))
    dg, ds = oracle.rhs(m, 0.3, V, s, mask)
    if mask & 7:
        assert rel(dg, np.conj(dg[::-1, ::-1, ::-1])) < 1e-14
        assert np.max(np.abs(dg)) > 1e-3
    if mask & 8:
        assert np.max(np.abs(ds - np.conj(ds[::-1]))) < 1e-14 * max(np.max(np.abs(ds)), 1e-3)
    # a vertex without the symmetry gives an rhs without it
    W = inputs.random_vertex(N, U, seed=33)
    dw, _ = oracle.rhs(m, 0.3, W, s, 0xF)
    assert rel(dw, np.conj(dw[::-1, ::-1, ::-1])) > 1e-3


# ------------------------------------------------------ interaction flow ----
# cutoff = 1: Theta = 1/sqrt(Lambda) (the bare propagator sqrt(g) G0, g = 1/Lambda),
# flowing from Lambda0 = 1/g0 >> 1 down to Lambda = 1, the full model.
IF_L0, IF_LF = 1e12, 1.0


@pytest.mark.parametrize("Lam", [1e6, 40.0, 1.0, 0.3])
def test_interaction_flow_single_scale_is_scale_derivative(Lam):
    m = Model(U=1.5, T=0.04, eps_d=-0.2, Delta=1.0, N=12, cutoff=1)
    sig = inputs.random_sigma(m.N, seed=13, amp=0.2)
    G, S = oracle.propagators(m, Lam, sig)
    h = 1e-5 * Lam
    Gp, _ = oracle.propagators(m, Lam + h, sig)
    Gm, _ = oracle.propagators(m, Lam - h, sig)
    assert rel(S, (Gp - Gm) / (2 * h)) < 1e-8
    # at Lambda = 1 the regulated propagator is the full one
    if Lam == 1.0:
        w = cf.freqs(m.N, m.T)
        full = 1.0 / (1j * w - (m.eps_d + m.U / 2) + 1j * m.Delta * np.sign(w) - sig)
        assert rel(G, full) < 1e-14


@pytest.mark.parametrize("eps_shift", [0.0, 0.6])
def test_interaction_flow_second_order_perturbation_theory(eps_shift):
    N, T, D = 8, 0.05, 1.0
    devs, sdevs = [], []
    for U in [0.04, 0.02, 0.01]:
        m = Model(U=U, T=T, eps_d=-U / 2 + eps_shift, Delta=D, N=N, cutoff=1)
        g, s, st = oracle.flow(m, Lambda0=IF_L0, Lambda_f=IF_LF, rtol=1e-12, atol=1e-16)
        assert st.status == 0
        ref, _, _ = cf.second_order_vertex(N, T, eps_shift, D, U, IF_L0, IF_LF, cutoff=1)
        sref = cf.first_order_sigma(N, T, eps_shift, D, U, IF_L0, IF_LF, cutoff=1)
        devs.append(np.max(np.abs(g - ref)))
        sdevs.append(np.max(np.abs(s - sref)))
    _, dBpp, dBph = cf.second_order_vertex(N, T, eps_shift, D, 1.0, IF_L0, IF_LF, cutoff=1)
    assert np.max(np.abs(dBpp)) > 1e-2 and np.max(np.abs(dBph)) > 1e-2
    for a, b in zip(devs, devs[1:]):
        assert 6.5 < a / b < 9.5, devs
    if eps_shift != 0.0:
        for a, b in zip(sdevs, sdevs[1:]):
            assert 3.2 < a / b < 4.8, sdevs


def test_interaction_flow_pp_ladder_closed_form():
    N, T, D, U = 10, 0.05, 1.0, 2.5
    m = Model(U=U, T=T, eps_d=-U / 2 + 0.4, Delta=D, N=N, cutoff=1)
    g, s, st = oracle.flow(m, mask=0x1, Lambda0=IF_L0, Lambda_f=IF_LF, rtol=1e-11, atol=1e-14)
    assert st.status == 0 and np.max(np.abs(s)) == 0.0
    _, dBpp, _ = cf.second_order_vertex(N, T, 0.4, D, 1.0, IF_L0, IF_LF, cutoff=1)
    ref = U / (1 + U * dBpp)
    mk = _aib(N)
    assert rel(g[mk], ref[mk]) < 2e-8
    assert rel(ref[mk], U) > 0.05


def test_interaction_and_omega_schemes_agree_to_second_order():
    """Both cutoffs end at the full propagator, so their final vertex and
    self-energy coincide through O(U^2) (perturbation theory does not know the
    regulator); the one-loop truncation makes them differ at O(U^3)."""
    dg, ds = [], []
    for U in [0.5, 0.25, 0.125]:
        kw = dict(U=U, T=0.05, eps_d=-U / 2 + 0.3, Delta=1.0, N=8)
        gi, si, st1 = oracle.flow(Model(cutoff=1, **kw), Lambda0=IF_L0, Lambda_f=IF_LF, rtol=1e-11, atol=1e-15)
        go, so, st2 = oracle.flow(Model(cutoff=0, **kw), Lambda0=1e8, Lambda_f=1e-8, rtol=1e-11, atol=1e-15)
        assert st1.status == 0 and st2.status == 0
        dg.append(np.max(np.abs(gi - go)))
        ds.append(np.max(np.abs(si - so)))
        assert np.max(np.abs(gi - U)) > 20 * dg[-1]  # the vertex did flow
    for a, b in zip(dg, dg[1:]):
        assert 6.5 < a / b < 9.5, dg
    for a, b in zip(ds, ds[1:]):
        assert 6.0 < a / b < 10.0, ds


def test_interaction_flow_rhs_matches_spin_resolved_general_formula():
    N, U, T, Lam = 6, 1.3, 0.07, 3.7
    m = Model(U=U, T=T, eps_d=-U / 2 + 0.4, Delta=1.0, N=N, cutoff=1)
    V = inputs.random_vertex(N, U, seed=41, amp=0.4)
    sig = inputs.random_sigma(N, seed=42, amp=0.15)
    dg, ds = oracle.rhs(m, Lam, V, sig)
    G, S = oracle.propagators(m, Lam, sig)
    dgb, dsb = bf.reduced_from_general(V, U, G, S, T, Lam)
    assert rel(dg, dgb) < 1e-13 and rel(ds, dsb) < 1e-13
