"""Thin ctypes binding to the C ABI of include/frg.h (argument marshalling only).

Every step of the computation runs in the CUDA library built from csrc/; this
module only converts Python/torch arguments to pointers and sizes.  There is
no fallback: if the library is missing or fails to load, every call raises.

Vertex tensors are complex128 of shape (N, N, N) (index [i1, i2, i3], i = n + N/2),
self-energy tensors complex128 of shape (N,).
"""
import ctypes as C
import dataclasses
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libfrg.so")

FP64, TF32X3, BF16X3 = 0, 1, 2
PRECISIONS = {"fp64": FP64, "3xtf32": TF32X3, "bf16x3": BF16X3}
CH_PP, CH_DPH, CH_XPH, CH_SIGMA, CH_ALL = 0x1, 0x2, 0x4, 0x8, 0xF
TAILS, TAIL_FACTOR = 0x10, 16  # frequency-box tails option of channel_mask (FRG_TAILS)
REVERSAL = 0x20  # frequency-reversal reduction asserted for every input (FRG_REVERSAL)
NO_REVERSAL = 0x40  # no reversal reduction in flows (FRG_NO_REVERSAL; default: while the states are symmetric)
CROSSING = 0x80  # crossing symmetry asserted for every input: crossing-reduced products (FRG_CROSSING)
CUTOFF_OMEGA, CUTOFF_INTERACTION = 0, 1  # frg_params.cutoff

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ENOTCONV, ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
ERRNAMES = {EINVAL: "FRG_EINVAL", ENOMEM: "FRG_ENOMEM", ECUDA: "FRG_ECUDA",
            ENONFINITE: "FRG_ENONFINITE", ENOTCONV: "FRG_ENOTCONV", ETIMEOUT: "FRG_ETIMEOUT"}

EXPORTED = ("frg_init", "frg_destroy", "frg_last_error", "frg_rhs", "frg_rhs_host", "frg_flow",
            "frg_advance", "frg_observables", "frg_get_state", "frg_set_state", "frg_stats",
            "frg_rhs_timed", "frg_kernel_launches", "frg_rhs_noalloc", "frg_autotune", "frg_selftest_wait", "frg_rhs_host_async", "frg_sync",
            "frg_cross_tile")
NOALLOC_MAX_N = 64


class FrgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRNAMES.get(code, "error"), code, msg))
        self.code = code


class _Params(C.Structure):
    _fields_ = [("U", C.c_double), ("T", C.c_double), ("eps_d", C.c_double),
                ("Delta", C.c_double), ("N_f", C.c_int), ("Lambda0", C.c_double),
                ("Lambda_f", C.c_double), ("rtol", C.c_double), ("atol", C.c_double),
                ("h0", C.c_double), ("max_steps", C.c_long), ("precision", C.c_int),
                ("channel_mask", C.c_int), ("cutoff", C.c_int)]


class _Stats(C.Structure):
    _fields_ = [("Lambda", C.c_double), ("h", C.c_double), ("accepted", C.c_long),
                ("rejected", C.c_long), ("rhs_evals", C.c_long), ("status", C.c_int),
                ("done", C.c_int)]


class _Tune(C.Structure):
    _fields_ = [("nt_cap", C.c_int), ("epi_cost", C.c_int), ("candidates", C.c_int),
                ("ms", C.c_float), ("ms_default", C.c_float)]


class _Obs(C.Structure):
    _fields_ = [("sigma_lowest_re", C.c_double), ("sigma_lowest_im", C.c_double),
                ("Z", C.c_double), ("U_eff_re", C.c_double), ("U_eff_im", C.c_double),
                ("n", C.c_double)]


@dataclasses.dataclass
class Params:
    U: float
    T: float
    eps_d: float
    N_f: int
    Delta: float = 1.0
    Lambda0: float = 1e3
    Lambda_f: float = 1e-3
    rtol: float = 1e-8
    atol: float = 1e-10
    h0: float = -0.01
    max_steps: int = 100000
    cutoff: int = 0  # CUTOFF_OMEGA or CUTOFF_INTERACTION

    @classmethod
    def from_workload(cls, w):
        return cls(U=w.U, T=w.T, eps_d=w.eps_d, N_f=w.N, Delta=w.Delta, Lambda0=w.Lambda0,
                   Lambda_f=w.Lambda_f, rtol=w.rtol, atol=w.atol, cutoff=getattr(w, "cutoff", 0))


@dataclasses.dataclass
class Stats:
    Lambda: float
    h: float
    accepted: int
    rejected: int
    rhs_evals: int
    status: int
    done: int


_lib = None


def load():
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FrgError(ECUDA, "CUDA library %s is missing: build it first "
                              "(python -c 'import __graft_entry__ as g; g.build()')" % LIB_PATH)
    lib = C.CDLL(LIB_PATH)
    vp, dp = C.c_void_p, C.POINTER(C.c_double)
    lib.frg_init.argtypes = [C.POINTER(_Params), C.c_int, vp, C.POINTER(vp)]
    lib.frg_destroy.argtypes = [vp]
    lib.frg_destroy.restype = None
    lib.frg_last_error.argtypes = [vp]
    lib.frg_last_error.restype = C.c_char_p
    lib.frg_rhs.argtypes = [vp, C.c_int, C.c_double, vp, vp, vp, vp]
    lib.frg_rhs_host.argtypes = [vp, C.c_int, C.c_double, dp, dp, dp, dp]
    lib.frg_flow.argtypes = [vp, C.POINTER(_Stats)]
    lib.frg_advance.argtypes = [vp, C.c_long, C.POINTER(_Stats)]
    lib.frg_stats.argtypes = [vp, C.POINTER(_Stats)]
    lib.frg_observables.argtypes = [vp, C.c_int, C.POINTER(_Obs)]
    lib.frg_get_state.argtypes = [vp, C.c_int, vp, vp, dp, dp]
    lib.frg_set_state.argtypes = [vp, C.c_int, vp, vp, C.c_double, C.c_double]
    lib.frg_rhs_timed.argtypes = [vp, C.c_int, C.c_double, vp, vp, vp, vp, C.POINTER(C.c_float)]
    lib.frg_rhs_noalloc.argtypes = [C.POINTER(_Params), C.c_double, vp, vp, vp, vp, vp]
    lib.frg_autotune.argtypes = [vp, C.POINTER(_Tune)]
    lib.frg_selftest_wait.argtypes = [vp, C.c_double]
    lib.frg_rhs_host_async.argtypes = [vp, C.c_int, C.c_double, dp, dp, dp, dp]
    lib.frg_sync.argtypes = [vp]
    lib.frg_cross_tile.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int)]
    lib.frg_kernel_launches.argtypes = []
    lib.frg_kernel_launches.restype = C.c_long
    _lib = lib
    return lib


def cross_tile(ch, N, nt, m, rt):
    """Crossing-reduced tile geometry (frg_cross_tile): (c0, width, own_lo,
    own_hi, partner_lo, partner_hi, partner_row_max)."""
    out = (C.c_int * 7)()
    rc = load().frg_cross_tile(ch, N, nt, m, rt, out)
    if rc != OK:
        raise FrgError(rc, "frg_cross_tile: invalid arguments")
    return tuple(out)


def kernel_launches():
    """Kernels launched by the library in this process so far."""
    return int(load().frg_kernel_launches())


def rhs_noalloc(params, Lambda, gamma, sigma, dgamma, dsigma, channel_mask=CH_ALL, stream=None):
    """FP64 rhs of one point through frg_rhs_noalloc (no context, no device
    allocation; N_f <= NOALLOC_MAX_N).  Tensors as for Context.rhs; asynchronous
    on `stream` (default: torch's current stream)."""
    lib = load()
    p = params if isinstance(params, Params) else Params.from_workload(params)
    N = p.N_f
    for t, shp, name in ((gamma, (N, N, N), "gamma"), (sigma, (N,), "sigma"),
                         (dgamma, (N, N, N), "dgamma"), (dsigma, (N,), "dsigma")):
        if t is not None:
            _check_dev(t, shp, name)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    cp = _Params(p.U, p.T, p.eps_d, p.Delta, p.N_f, p.Lambda0, p.Lambda_f, p.rtol, p.atol, p.h0,
                 p.max_steps, FP64, channel_mask, getattr(p, "cutoff", 0))
    rc = lib.frg_rhs_noalloc(C.byref(cp), Lambda, _ptr(gamma), _ptr(sigma), _ptr(dgamma),
                             _ptr(dsigma), C.c_void_p(stream))
    if rc != OK:
        raise FrgError(rc, "frg_rhs_noalloc failed (N_f must be even and <= %d)" % NOALLOC_MAX_N)


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _check_dev(t, shape, name):
    import torch
    if t is None:
        return
    if not (t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()
            and tuple(t.shape) == tuple(shape)):
        raise ValueError("%s must be a contiguous complex128 CUDA tensor of shape %s"
                         % (name, tuple(shape)))


class Context:
    """A set of parameter points sharing one precision and channel mask."""

    def __init__(self, points, precision=FP64, channel_mask=CH_ALL, stream=None):
        lib = load()
        if isinstance(precision, str):
            precision = PRECISIONS[precision]
        pts = [p if isinstance(p, Params) else Params.from_workload(p) for p in points]
        arr = (_Params * len(pts))()
        for i, p in enumerate(pts):
            arr[i] = _Params(p.U, p.T, p.eps_d, p.Delta, p.N_f, p.Lambda0, p.Lambda_f, p.rtol,
                             p.atol, p.h0, p.max_steps, precision, channel_mask, p.cutoff)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self._stream = stream
        h = C.c_void_p()
        rc = lib.frg_init(arr, len(pts), C.c_void_p(stream), C.byref(h))
        if rc != OK:
            raise FrgError(rc, "frg_init failed")
        self._h = h
        self.points = pts
        self.precision = precision
        self.n = len(pts)

    def _chk(self, rc):
        if rc != OK:
            raise FrgError(rc, load().frg_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            load().frg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def N(self, point):
        return self.points[point].N_f

    def rhs(self, point, Lambda, gamma, sigma, dgamma, dsigma):
        N = self.N(point)
        _check_dev(gamma, (N, N, N), "gamma")
        _check_dev(sigma, (N,), "sigma")
        _check_dev(dgamma, (N, N, N), "dgamma")
        _check_dev(dsigma, (N,), "dsigma")
        self._chk(load().frg_rhs(self._h, point, Lambda, _ptr(gamma), _ptr(sigma), _ptr(dgamma),
                                 _ptr(dsigma)))

    def rhs_timed(self, point, Lambda, gamma, sigma, dgamma, dsigma):
        """Like rhs(); returns the phase durations in ms (bubble weights with the
        self-energy, operand regather, channel contractions, combine, and 0)
        measured with CUDA events on the context stream."""
        N = self.N(point)
        _check_dev(gamma, (N, N, N), "gamma")
        _check_dev(dgamma, (N, N, N), "dgamma")
        _check_dev(dsigma, (N,), "dsigma")
        ms = (C.c_float * 5)()
        self._chk(load().frg_rhs_timed(self._h, point, Lambda, _ptr(gamma), _ptr(sigma),
                                       _ptr(dgamma), _ptr(dsigma), ms))
        return list(ms)

    def rhs_host(self, point, Lambda, gamma, sigma, dgamma, dsigma):
        """Host numpy complex128 buffers (copies inside the call)."""
        import numpy as np
        N = self.N(point)
        for a, shp in ((gamma, (N, N, N)), (dgamma, (N, N, N)), (dsigma, (N,))):
            if a.dtype != np.complex128 or not a.flags.c_contiguous or a.shape != shp:
                raise ValueError("host buffers must be contiguous complex128 arrays")
        dp = C.POINTER(C.c_double)
        sp = None if sigma is None else sigma.ctypes.data_as(dp)
        self._chk(load().frg_rhs_host(self._h, point, Lambda, gamma.ctypes.data_as(dp), sp,
                                      dgamma.ctypes.data_as(dp), dsigma.ctypes.data_as(dp)))

    def rhs_host_async(self, point, Lambda, gamma, sigma, dgamma, dsigma):
        """Pipelined host-buffer evaluation (returns at once; the buffers must
        stay alive and the outputs unread until sync())."""
        import numpy as np
        N = self.N(point)
        for a, shp in ((gamma, (N, N, N)), (dgamma, (N, N, N)), (dsigma, (N,))):
            if a.dtype != np.complex128 or not a.flags.c_contiguous or a.shape != shp:
                raise ValueError("host buffers must be contiguous complex128 arrays")
        dp = C.POINTER(C.c_double)
        sp = None if sigma is None else sigma.ctypes.data_as(dp)
        self._chk(load().frg_rhs_host_async(self._h, point, Lambda, gamma.ctypes.data_as(dp), sp,
                                            dgamma.ctypes.data_as(dp), dsigma.ctypes.data_as(dp)))

    def sync(self):
        self._chk(load().frg_sync(self._h))

    def _stats(self, arr):
        return [Stats(s.Lambda, s.h, s.accepted, s.rejected, s.rhs_evals, s.status, s.done)
                for s in arr]

    def flow(self):
        arr = (_Stats * self.n)()
        self._chk(load().frg_flow(self._h, arr))
        return self._stats(arr)

    def advance(self, max_attempts):
        arr = (_Stats * self.n)()
        self._chk(load().frg_advance(self._h, int(max_attempts), arr))
        return self._stats(arr)

    def stats(self):
        arr = (_Stats * self.n)()
        self._chk(load().frg_stats(self._h, arr))
        return self._stats(arr)

    def autotune(self):
        """Time the candidate contraction plans on the current state and keep
        the fastest (split precisions); returns the choice."""
        t = _Tune()
        self._chk(load().frg_autotune(self._h, C.byref(t)))
        return {"nt_cap": t.nt_cap, "epi_cost": t.epi_cost, "candidates": t.candidates,
                "ms": t.ms, "ms_default": t.ms_default}

    def selftest_wait(self, limit_ms=50.0):
        """Run one bounded pipeline wait that must run out; raises FrgError
        with code ETIMEOUT when the failure path works."""
        self._chk(load().frg_selftest_wait(self._h, float(limit_ms)))

    def observables(self, point):
        o = _Obs()
        self._chk(load().frg_observables(self._h, point, C.byref(o)))
        return {"sigma_lowest": complex(o.sigma_lowest_re, o.sigma_lowest_im), "Z": o.Z,
                "U_eff": complex(o.U_eff_re, o.U_eff_im), "n": o.n}

    def get_state(self, point):
        import torch
        N = self.N(point)
        g = torch.empty((N, N, N), dtype=torch.complex128, device="cuda")
        s = torch.empty((N,), dtype=torch.complex128, device="cuda")
        lam, h = C.c_double(), C.c_double()
        self._chk(load().frg_get_state(self._h, point, _ptr(g), _ptr(s), C.byref(lam), C.byref(h)))
        return g, s, lam.value, h.value

    def set_state(self, point, gamma, sigma, Lambda, h=0.0):
        N = self.N(point)
        _check_dev(gamma, (N, N, N), "gamma")
        _check_dev(sigma, (N,), "sigma")
        self._chk(load().frg_set_state(self._h, point, _ptr(gamma), _ptr(sigma), Lambda, h))
