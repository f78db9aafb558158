"""ctypes wrapper around the plain-C FP64 oracle (frg_oracle.c).

Test infrastructure only: used by tests/, the smoke check and the CPU-baseline
leg of the benchmark.  Arrays are numpy complex128, vertex index
[i1, i2, i3] with i = n + N/2 the fermionic Matsubara index.
"""
import ctypes as C
import dataclasses

import numpy as np

from . import build as _build

_lib = None

# Channel-mask bits: 1 pp, 2 dph, 4 xph, 8 self-energy flow, 16 frequency-box
# tails (internal sums over a window of TAIL_FACTOR * N Matsubara indices
# centred on the box, bare-U vertices and Sigma = 0 outside the box).
MASK_TAILS = 0x10
TAIL_FACTOR = 16


class _Model(C.Structure):
    _fields_ = [("U", C.c_double), ("T", C.c_double), ("eps_d", C.c_double),
                ("Delta", C.c_double), ("N", C.c_int), ("cutoff", C.c_int)]


class _Stats(C.Structure):
    _fields_ = [("t", C.c_double), ("h", C.c_double), ("accepted", C.c_long),
                ("rejected", C.c_long), ("rhs_evals", C.c_long),
                ("status", C.c_int), ("first_step_evals", C.c_long)]


RHS_FN = C.CFUNCTYPE(C.c_int, C.c_double, C.POINTER(C.c_double),
                     C.POINTER(C.c_double), C.c_void_p)


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        mp = C.POINTER(_Model)
        lib.oracle_rhs.argtypes = [mp, C.c_double, dp, dp, C.c_int, dp, dp]
        lib.oracle_rhs_rows.argtypes = [mp, C.c_double, dp, dp, C.c_int, C.c_int,
                                        C.c_int, dp, dp]
        lib.oracle_rhs_entries.argtypes = [mp, C.c_double, dp, dp, C.c_int, C.c_int,
                                           C.POINTER(C.c_int), dp]
        lib.oracle_flow.argtypes = [mp, C.c_int, C.c_double, C.c_double, C.c_double,
                                    C.c_double, C.c_double, C.c_long, dp, dp,
                                    C.POINTER(_Stats)]
        lib.oracle_propagators.argtypes = [mp, C.c_double, dp, dp, dp]
        lib.oracle_observables.argtypes = [mp, C.c_double, dp, dp, dp]
        lib.oracle_dp5_tableau.argtypes = [dp, dp, dp, dp]
        lib.oracle_dp5.argtypes = [C.c_long, dp, C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.c_double, C.c_long, C.c_double,
                                   RHS_FN, C.c_void_p, C.POINTER(_Stats)]
        lib.oracle_set_threads.argtypes = [C.c_int]
        lib.oracle_max_threads.restype = C.c_int
        _lib = lib
    return _lib


@dataclasses.dataclass(frozen=True)
class Model:
    """SIAM parameters: interaction U, temperature T, level eps_d,
    hybridisation Delta, N fermionic frequencies per axis (N even); cutoff 0
    for the Omega scheme, 1 for the interaction flow."""
    U: float
    T: float
    eps_d: float
    Delta: float
    N: int
    cutoff: int = 0

    def c(self):
        return _Model(self.U, self.T, self.eps_d, self.Delta, self.N, self.cutoff)


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _c128(a, shape):
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if a.shape != shape:
        raise ValueError("expected shape %s, got %s" % (shape, a.shape))
    return a


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def propagators(m: Model, Lam: float, sigma=None):
    """(G, S) at scale Lam on the N in-box frequencies."""
    lib = _load()
    sg = _c128(np.zeros(m.N) if sigma is None else sigma, (m.N,))
    G = np.zeros(m.N, np.complex128)
    S = np.zeros(m.N, np.complex128)
    mc = m.c()
    lib.oracle_propagators(C.byref(mc), Lam, _dp(sg), _dp(G), _dp(S))
    return G, S


def rhs(m: Model, Lam: float, gamma, sigma, mask: int = 0xF):
    """(dgamma/dl, dsigma/dl) at scale Lam, l = ln Lam."""
    N = m.N
    g = _c128(gamma, (N, N, N))
    s = _c128(sigma, (N,))
    dg = np.zeros((N, N, N), np.complex128)
    ds = np.zeros(N, np.complex128)
    mc = m.c()
    rc = _load().oracle_rhs(C.byref(mc), Lam, _dp(g), _dp(s), int(mask), _dp(dg), _dp(ds))
    if rc:
        raise RuntimeError("oracle_rhs failed (%d)" % rc)
    return dg, ds


def rhs_rows(m: Model, Lam: float, gamma, sigma, k1_begin: int, k1_end: int,
             mask: int = 0xF):
    """dgamma/dl for rows i1 in [k1_begin, k1_end) only (used to time a bounded
    sample); returns the full-size array with the other rows zero."""
    N = m.N
    g = _c128(gamma, (N, N, N))
    s = _c128(sigma, (N,))
    dg = np.zeros((N, N, N), np.complex128)
    mc = m.c()
    rc = _load().oracle_rhs_rows(C.byref(mc), Lam, _dp(g), _dp(s), int(mask),
                                 int(k1_begin), int(k1_end), _dp(dg), None)
    if rc:
        raise RuntimeError("oracle_rhs_rows failed (%d)" % rc)
    return dg


def rhs_entries(m: Model, Lam: float, gamma, sigma, idx, mask: int = 0xF):
    """dgamma/dl at the listed (i1, i2, i3) entries (idx shape (k, 3))."""
    N = m.N
    g = _c128(gamma, (N, N, N))
    s = _c128(sigma, (N,))
    idx = np.ascontiguousarray(idx, dtype=np.int32).reshape(-1, 3)
    out = np.zeros(idx.shape[0], np.complex128)
    mc = m.c()
    rc = _load().oracle_rhs_entries(C.byref(mc), Lam, _dp(g), _dp(s), int(mask),
                                    idx.shape[0], idx.ctypes.data_as(C.POINTER(C.c_int)),
                                    _dp(out))
    if rc:
        raise RuntimeError("oracle_rhs_entries failed (%d)" % rc)
    return out


@dataclasses.dataclass
class FlowStats:
    Lambda: float
    h: float
    accepted: int
    rejected: int
    rhs_evals: int
    status: int
    first_step_evals: int


def flow(m: Model, gamma0=None, sigma0=None, Lambda0=1e3, Lambda_f=1e-3,
         rtol=1e-8, atol=1e-10, h0=-0.01, mask=0xF, max_steps=200000):
    """Integrate the flow from Lambda0 to Lambda_f; returns (gamma, sigma, stats).
    Default initial state: gamma = U, sigma = 0."""
    N = m.N
    g = (np.full((N, N, N), m.U, np.complex128) if gamma0 is None
         else _c128(gamma0, (N, N, N)).copy())
    s = np.zeros(N, np.complex128) if sigma0 is None else _c128(sigma0, (N,)).copy()
    st = _Stats()
    mc = m.c()
    _load().oracle_flow(C.byref(mc), int(mask), Lambda0, Lambda_f, rtol, atol, h0,
                        int(max_steps), _dp(g), _dp(s), C.byref(st))
    import math
    stats = FlowStats(math.exp(st.t), st.h, st.accepted, st.rejected, st.rhs_evals,
                      st.status, st.first_step_evals)
    return g, s, stats


def observables(m: Model, Lam: float, gamma, sigma):
    """dict with sigma_lowest (complex), Z, U_eff (complex), n (informational)."""
    N = m.N
    g = _c128(gamma, (N, N, N))
    s = _c128(sigma, (N,))
    out = np.zeros(6)
    mc = m.c()
    _load().oracle_observables(C.byref(mc), Lam, _dp(g), _dp(s), _dp(out))
    return {"sigma_lowest": complex(out[0], out[1]), "Z": out[2],
            "U_eff": complex(out[3], out[4]), "n": out[5]}


def dp5_tableau():
    """(c[7], a[7,6], b[7], bstar[7]) as held by the oracle."""
    c = np.zeros(7)
    a = np.zeros(42)
    b = np.zeros(7)
    bs = np.zeros(7)
    _load().oracle_dp5_tableau(_dp(c), _dp(a), _dp(b), _dp(bs))
    return c, a.reshape(7, 6), b, bs


def dp5_integrate(f, y0, t0, t1, rtol=1e-8, atol=1e-10, h0=0.01, fixed_h=0.0,
                  max_steps=1000000):
    """Integrate a real vector ODE y' = f(t, y) with the oracle's DP5 driver.
    f maps (t, numpy array) -> numpy array.  Returns (y, stats)."""
    y = np.ascontiguousarray(y0, dtype=np.float64).copy()
    n = y.size

    def cb(t, yp, dp, _ctx):
        yy = np.ctypeslib.as_array(yp, shape=(n,))
        d = np.ctypeslib.as_array(dp, shape=(n,))
        d[:] = f(t, yy.copy())
        return 0

    fn = RHS_FN(cb)
    st = _Stats()
    _load().oracle_dp5(n, _dp(y), t0, t1, h0, rtol, atol, int(max_steps), fixed_h,
                       fn, None, C.byref(st))
    stats = FlowStats(st.t, st.h, st.accepted, st.rejected, st.rhs_evals, st.status,
                      st.first_step_evals)
    return y, stats
