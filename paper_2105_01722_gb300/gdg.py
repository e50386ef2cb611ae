"""Thin ctypes binding of libgdg (include/gdg.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts torch
tensors to device pointers and the current torch stream to a cudaStream_t.
It raises if libgdg.so is missing: there is no fallback.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# the index-checking build (gdg_checks.cuh) when the environment asks for it
LIB_PATH = os.path.join(_HERE, "libgdg_checks.so" if os.environ.get("GDG_CHECKS") == "1" else "libgdg.so")

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, ETIMEOUT, ENONFINITE, EUNSUPPORTED, EHALO = 0, -1, -2, -3, -4, -5, -6, -7, -8
BC_DIRICHLET, BC_PERIODIC = 0, 1
FLUX_CENTRAL, FLUX_UPWIND, FLUX_ALTERNATING = 0, 1, 2
COEF_CONST, COEF_NODAL = 0, 1
SOLVE_DIAG, SOLVE_PCG, SOLVE_INVERSE = 0, 1, 2
PC_FDM, PC_NONE, PC_IC0 = 0, 1, 2
FP64, MIXED, TF32, BF16 = 0, 1, 2, 3
ROUTE_MODAL, ROUTE_NODAL = 0, 1
OP_M, OP_S = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)


class Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("n_elem", ctypes.c_int * 3), ("N", ctypes.c_int), ("p", ctypes.c_int),
        ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("bc", ctypes.c_int * 3),
        ("flux", ctypes.c_int), ("xi", ctypes.c_double), ("coef", ctypes.c_int), ("c2", ctypes.c_double),
        ("x_nodes", _dp), ("y_nodes", _dp), ("c2_nodes", _dp), ("nquad", ctypes.c_int),
        ("solver", ctypes.c_int), ("precond", ctypes.c_int), ("pcg_rtol", ctypes.c_double),
        ("pcg_maxit", ctypes.c_int), ("precision", ctypes.c_int), ("route", ctypes.c_int),
        ("refine_max", ctypes.c_int), ("refine_rtol", ctypes.c_double), ("rows", ctypes.c_int * 2),
    ]


class PcgStats(ctypes.Structure):
    _fields_ = [("max_iters", ctypes.c_int), ("mean_iters", ctypes.c_double),
                ("max_rel_resid", ctypes.c_double), ("unconverged", ctypes.c_int),
                ("max_sweeps", ctypes.c_int), ("mean_sweeps", ctypes.c_double),
                ("guessed", ctypes.c_longlong), ("fell_back", ctypes.c_longlong)]


_LIB = None

# int (*gdg_halo_fn)(void *user, void *stream)
HALO_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p)

EXPORTS = {
    "gdg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "gdg_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "gdg_basis_1d": (ctypes.c_int, [ctypes.c_int, ctypes.c_int] + [ctypes.c_void_p] * 8),
    "gdg_create": (ctypes.c_int, [ctypes.POINTER(Problem), ctypes.POINTER(ctypes.c_void_p)]),
    "gdg_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "gdg_state_len": (ctypes.c_longlong, [ctypes.c_void_p]),
    "gdg_rhs": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_double] + [ctypes.c_void_p] * 3),
    "gdg_mass_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]),
    "gdg_pcg": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.POINTER(PcgStats), ctypes.c_void_p]),
    "gdg_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                ctypes.c_double, ctypes.c_int, ctypes.c_void_p]),
    "gdg_step_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_void_p]),
    "gdg_energy": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "gdg_residuals": (ctypes.c_int, [ctypes.c_void_p] * 6),
    "gdg_mlp_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.c_void_p]),
    "gdg_mlp_partial_len": (ctypes.c_longlong, [ctypes.c_int]),
    "gdg_mlp_backward": (ctypes.c_int, [ctypes.c_void_p] * 5 + [ctypes.c_int] + [ctypes.c_void_p] * 4),
    "gdg_mlp_adam": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_int, ctypes.c_float, ctypes.c_void_p,
                                                           ctypes.c_void_p]),
    "gdg_mlp_to_bf16": (ctypes.c_int, [ctypes.c_void_p] * 3),
    "gdg_mlp_rows": (ctypes.c_int, [ctypes.c_void_p] * 6),
    "gdg_mlp_attach": (ctypes.c_int, [ctypes.c_void_p] * 3),
    "gdg_mlp_detach": (ctypes.c_int, [ctypes.c_void_p]),
    "gdg_batch_create": (ctypes.c_int, [ctypes.POINTER(Problem), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "gdg_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "gdg_batch_state_len": (ctypes.c_longlong, [ctypes.c_void_p, ctypes.c_int]),
    "gdg_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                      ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_void_p]),
    "gdg_batch_tuning": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_int)] * 6),
    "gdg_check_status": (ctypes.c_int, [ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                         ctypes.c_int]),
    "gdg_check_selftest": (ctypes.c_int, [ctypes.c_longlong, ctypes.c_longlong, ctypes.c_void_p]),
    "gdg_batch_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "gdg_batch_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(PcgStats),
                                       ctypes.POINTER(PcgStats)]),
    "gdg_rhs_static": (ctypes.c_int, [ctypes.POINTER(Problem)] + [ctypes.c_void_p] * 5),
    "gdg_step_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(PcgStats), ctypes.POINTER(PcgStats)]),
    "gdg_profile_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "gdg_set_stage_variant": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "gdg_get_stage_variant": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "gdg_set_wait_limit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "gdg_set_point_source": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double]),
    "gdg_profile_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.POINTER(ctypes.c_double)]),
    "gdg_probe_fp64": (ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                      ctypes.c_void_p]),
    "gdg_halo_len": (ctypes.c_longlong, [ctypes.c_void_p]),
    "gdg_set_halo": (ctypes.c_int, [ctypes.c_void_p] * 5 + [HALO_FN, ctypes.c_void_p]),
}

K_STAGE, K_TRACES, K_TRANSFORM, K_RHS, K_PCG, K_OTHER = range(6)
K_NAMES = ("stage", "traces", "transform", "rhs", "pcg", "other")


def lib():
    """Load libgdg.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libgdg.so is not built (run __graft_entry__.build()); "
                               "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in EXPORTS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


class GdgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (%d): %s" % (lib().gdg_status_string(status).decode(), status, msg))
        self.status = status


def basis_1d(p, N):
    """Host basis builder: dict of M, S, phiL, phiR, dphiL, dphiR, Psi, lam."""
    n1 = N + 1
    out = {k: np.zeros((n1, n1)) for k in ("M", "S", "Psi")}
    out.update({k: np.zeros(n1) for k in ("phiL", "phiR", "dphiL", "dphiR", "lam")})
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    st = lib().gdg_basis_1d(p, N, ptr(out["M"]), ptr(out["S"]), ptr(out["phiL"]), ptr(out["phiR"]),
                            ptr(out["dphiL"]), ptr(out["dphiR"]), ptr(out["Psi"]), ptr(out["lam"]))
    if st != OK:
        raise GdgError(st, "gdg_basis_1d(p=%d, N=%d)" % (p, N))
    return out


def make_problem(dim, n, N, p, lo=(0.0, 0.0), hi=(1.0, 1.0), bc=(BC_DIRICHLET, BC_DIRICHLET),
                 flux=FLUX_UPWIND, xi=0.0, c2=1.0, coef=COEF_CONST, x_nodes=None, y_nodes=None,
                 c2_nodes=None, nquad=0, solver=None, precond=PC_FDM, pcg_rtol=1e-10, pcg_maxit=200,
                 precision=FP64, route=ROUTE_MODAL, refine_max=8, refine_rtol=1e-5, rows=(0, 0)):
    pb = Problem()
    pb.dim = dim
    n = tuple(n) + (1,) * (3 - len(n))
    lo = tuple(lo) + (0.0,) * (3 - len(lo))
    hi = tuple(hi) + (1.0,) * (3 - len(hi))
    bc = tuple(bc) + (BC_DIRICHLET,) * (3 - len(bc))
    for k in range(3):
        pb.n_elem[k], pb.lo[k], pb.hi[k], pb.bc[k] = n[k], lo[k], hi[k], bc[k]
    pb.N, pb.p = N, p
    pb.flux, pb.xi, pb.coef, pb.c2 = flux, xi, coef, c2
    keep = []
    for name, arr in (("x_nodes", x_nodes), ("y_nodes", y_nodes), ("c2_nodes", c2_nodes)):
        if arr is not None:
            a = np.ascontiguousarray(arr, dtype=np.float64)
            keep.append(a)
            setattr(pb, name, a.ctypes.data_as(_dp))
    pb.nquad = nquad
    pb.solver = (SOLVE_DIAG if coef == COEF_CONST else SOLVE_PCG) if solver is None else solver
    pb.precond, pb.pcg_rtol, pb.pcg_maxit = precond, pcg_rtol, pcg_maxit
    pb.precision, pb.route = precision, route
    pb.refine_max, pb.refine_rtol = refine_max, refine_rtol
    pb.rows[0], pb.rows[1] = int(rows[0]), int(rows[1])
    pb._keep = keep   # host arrays must outlive gdg_create
    return pb


def _ptr(t, n=None):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError("expected %d elements, got %d" % (n, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


MLP_IN, MLP_HID, MLP_OUT, MLP_NPARAM, MLP_NWEIGHT = 162, 64, 81, 19857, 19648


def _fptr(t, n=None):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous float32 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError("expected %d elements, got %d" % (n, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def _uptr(t):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.int16 or not t.is_cuda or not t.is_contiguous() \
            or t.numel() != MLP_NWEIGHT:
        raise ValueError("expected %d int16 (BF16 bit patterns) on the device" % MLP_NWEIGHT)
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def check_status(reset=False):
    """Index-check failures of the GDG_CHECKS build since the last reset:
    dict(count, site, index, bound) of the first failure; raises GdgError
    (GDG_EUNSUPPORTED) on the ordinary build."""
    c, si, i, b = ctypes.c_longlong(), ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong()
    st = lib().gdg_check_status(ctypes.byref(c), ctypes.byref(si), ctypes.byref(i), ctypes.byref(b), int(reset))
    if st != OK:
        raise GdgError(st, "gdg_check_status")
    return dict(count=c.value, site=si.value, index=i.value, bound=b.value)


def check_selftest(index, bound, stream=None):
    """Check index against [0, bound) on the device (records site 99 if it fails)."""
    st = lib().gdg_check_selftest(int(index), int(bound), _stream(stream))
    if st != OK:
        raise GdgError(st, "gdg_check_selftest")


def probe_fp64(iters, sink, stream=None):
    """gdg_probe_fp64: launch the FP64 FMA-chain probe on `stream` (sink: a
    float64 CUDA tensor of at least one element); returns the launch's flop
    count.  Time it with CUDA events on the same stream."""
    flops = ctypes.c_double()
    st = lib().gdg_probe_fp64(int(iters), _ptr(sink[:1]), ctypes.byref(flops), _stream(stream))
    if st != OK:
        raise GdgError(st, "gdg_probe_fp64")
    return flops.value


def rhs_static(problem, u, v, du, dv, stream=None):
    """gdg_rhs_static: the constant-coefficient right-hand side without any
    allocation (no context; scratch in the library's static device array)."""
    n = (problem.N + 1) ** problem.dim
    for d in range(problem.dim):
        n *= problem.n_elem[d]
    st = lib().gdg_rhs_static(ctypes.byref(problem), _ptr(u, n), _ptr(v, n), _ptr(du, n), _ptr(dv, n),
                              _stream(stream))
    if st != OK:
        raise GdgError(st, "gdg_rhs_static")


class Context:
    """A gdg_ctx on the current CUDA device."""

    def __init__(self, problem):
        self._h = ctypes.c_void_p()
        st = lib().gdg_create(ctypes.byref(problem), ctypes.byref(self._h))
        if st != OK:
            raise GdgError(st, "gdg_create")
        self.problem = problem
        self.n = lib().gdg_state_len(self._h)

    def close(self):
        if self._h:
            lib().gdg_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st, what):
        if st != OK:
            raise GdgError(st, "%s: %s" % (what, lib().gdg_last_error(self._h).decode()))

    def rhs(self, u, v, du, dv, stream=None, t=0.0):
        """gdg_rhs at time t (which matters only with a point source)."""
        self._check(lib().gdg_rhs(self._h, _ptr(u, self.n), _ptr(v, self.n), float(t), _ptr(du, self.n),
                                  _ptr(dv, self.n), _stream(stream)), "gdg_rhs")

    def mass_solve(self, which, b, x, stream=None):
        self._check(lib().gdg_mass_solve(self._h, which, _ptr(b, self.n), _ptr(x, self.n),
                                         _stream(stream)), "gdg_mass_solve")

    def pcg(self, which, b, x, stream=None, allow_noconv=False):
        stats = PcgStats()
        st = lib().gdg_pcg(self._h, which, _ptr(b, self.n), _ptr(x, self.n), ctypes.byref(stats),
                           _stream(stream))
        if not (allow_noconv and st == ENOCONV):
            self._check(st, "gdg_pcg")
        return dict(max_iters=stats.max_iters, mean_iters=stats.mean_iters,
                    max_rel_resid=stats.max_rel_resid, unconverged=stats.unconverged,
                    max_sweeps=stats.max_sweeps, mean_sweeps=stats.mean_sweeps, status=st)

    def halo_len(self):
        """Doubles per halo side buffer (-1 without halo sides)."""
        return lib().gdg_halo_len(self._h)

    def set_halo(self, send_lo, send_hi, recv_lo, recv_hi, exchange):
        """gdg_set_halo: caller-owned float64 CUDA buffers of halo_len()
        doubles (None for a side without a halo) and exchange(stream_ptr) ->
        None, called between stages; an exception in it fails the call with
        GDG_EHALO."""
        n = self.halo_len()

        def cb(user, stream):
            try:
                exchange(stream)
                return 0
            except Exception as exc:     # reported through the status code
                self._halo_error = exc
                return 1

        self._halo_cb = HALO_FN(cb)     # keep the callback alive with the context
        self._halo_bufs = (send_lo, send_hi, recv_lo, recv_hi)
        ptr = lambda t: None if t is None else _ptr(t, n)
        self._check(lib().gdg_set_halo(self._h, ptr(send_lo), ptr(send_hi), ptr(recv_lo), ptr(recv_hi),
                                       self._halo_cb, None), "gdg_set_halo")

    def step_stats(self):
        """PCG statistics of the solves inside step()/rhs() since the last call."""
        su, sv = PcgStats(), PcgStats()
        self._check(lib().gdg_step_stats(self._h, ctypes.byref(su), ctypes.byref(sv)), "gdg_step_stats")
        f = lambda s: dict(max_iters=s.max_iters, mean_iters=s.mean_iters, unconverged=s.unconverged,
                           max_sweeps=s.max_sweeps, mean_sweeps=s.mean_sweeps, guessed=s.guessed,
                           fell_back=s.fell_back)
        return f(su), f(sv)

    def residuals(self, u, v, ru, rv, stream=None):
        self._check(lib().gdg_residuals(self._h, _ptr(u, self.n), _ptr(v, self.n), _ptr(ru, self.n),
                                        _ptr(rv, self.n), _stream(stream)), "gdg_residuals")

    def mlp_rows(self, ru, y, X, T, stream=None):
        """Training rows (features X, targets T) of every element; y may be None."""
        ne = self.n // 81
        self._check(lib().gdg_mlp_rows(self._h, _ptr(ru, self.n), _ptr(y, self.n) if y is not None else None,
                                       _fptr(X, ne * MLP_IN), _fptr(T, ne * MLP_OUT) if T is not None else None,
                                       _stream(stream)), "gdg_mlp_rows")

    def mlp_attach(self, net):
        self._check(lib().gdg_mlp_attach(self._h, _uptr(net.wbf16), _fptr(net.params, MLP_NPARAM)),
                    "gdg_mlp_attach")

    def mlp_detach(self):
        self._check(lib().gdg_mlp_detach(self._h), "gdg_mlp_detach")

    def step(self, u, v, t0, dt, nsteps, stream=None):
        self._check(lib().gdg_step(self._h, _ptr(u, self.n), _ptr(v, self.n), t0, dt, nsteps,
                                   _stream(stream)), "gdg_step")

    def step_host(self, u, v, t0, dt, nsteps, stream=None):
        """u, v: C-contiguous float64 host arrays (numpy or pinned torch CPU tensors)."""
        def hp(a):
            if isinstance(a, np.ndarray):
                assert a.dtype == np.float64 and a.flags.c_contiguous and a.size == self.n
                return ctypes.c_void_p(a.ctypes.data)
            assert a.dtype.is_floating_point and a.is_contiguous() and a.numel() == self.n
            return ctypes.c_void_p(a.data_ptr())
        self._check(lib().gdg_step_host(self._h, hp(u), hp(v), t0, dt, nsteps, _stream(stream)),
                    "gdg_step_host")

    def set_stage_variant(self, variant):
        """2-D constant coefficient: 0 one thread per line, 1 two, 2 one per line
        and field, 3 persistent step, -1 timed choice."""
        self._check(lib().gdg_set_stage_variant(self._h, int(variant)), "gdg_set_stage_variant")

    def set_point_source(self, element, r, s, amplitude, omega):
        """f = amplitude sin(omega t) delta(x - x_s), x_s at reference (r, s) of element."""
        self._check(lib().gdg_set_point_source(self._h, int(element), float(r), float(s), float(amplitude),
                                               float(omega)), "gdg_set_point_source")

    def set_wait_limit(self, seconds):
        """Bound on any device-side wait (seconds of wall time)."""
        self._check(lib().gdg_set_wait_limit(self._h, float(seconds)), "gdg_set_wait_limit")

    def stage_variant(self):
        out = ctypes.c_int()
        self._check(lib().gdg_get_stage_variant(self._h, ctypes.byref(out)), "gdg_get_stage_variant")
        return out.value

    def profile(self, on):
        self._check(lib().gdg_profile_enable(self._h, 1 if on else 0), "gdg_profile_enable")

    def profile_read(self):
        """{kind name: (launches, total ms)} of the launches recorded since profile(True)."""
        out = {}
        for k, name in enumerate(K_NAMES):
            n, ms = ctypes.c_longlong(), ctypes.c_double()
            self._check(lib().gdg_profile_read(self._h, k, ctypes.byref(n), ctypes.byref(ms)),
                        "gdg_profile_read")
            if n.value:
                out[name] = (n.value, ms.value)
        return out

    def energy(self, u, v, stream=None):
        E = ctypes.c_double()
        self._check(lib().gdg_energy(self._h, _ptr(u, self.n), _ptr(v, self.n), ctypes.byref(E),
                                     _stream(stream)), "gdg_energy")
        return E.value


class Batch:
    """A gdg_batch: independent problems advanced by shared persistent launches."""

    def __init__(self, problems):
        arr = (Problem * len(problems))(*problems)
        self._problems = problems     # keep host arrays alive through create
        self._h = ctypes.c_void_p()
        st = lib().gdg_batch_create(arr, len(problems), ctypes.byref(self._h))
        if st != OK:
            raise GdgError(st, "gdg_batch_create")
        self.count = len(problems)
        self.lens = [lib().gdg_batch_state_len(self._h, i) for i in range(self.count)]

    def close(self):
        if self._h:
            lib().gdg_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, us, vs, dts, nsteps, stream=None):
        U = (ctypes.c_void_p * self.count)(*[_ptr(u, n).value for u, n in zip(us, self.lens)])
        V = (ctypes.c_void_p * self.count)(*[_ptr(v, n).value for v, n in zip(vs, self.lens)])
        D = (ctypes.c_double * self.count)(*dts)
        st = lib().gdg_batch_step(self._h, U, V, D, nsteps, _stream(stream))
        if st != OK:
            raise GdgError(st, "gdg_batch_step")

    def tuning(self):
        t, b, e, g, r, c = (ctypes.c_int() for _ in range(6))
        lib().gdg_batch_tuning(self._h, *(ctypes.byref(x) for x in (t, b, e, g, r, c)))
        return dict(threads_per_block=t.value, blocks_per_sm=b.value, tile_elements=e.value,
                    register_budget=g.value, registers_per_thread=r.value, items_per_turn=c.value)

    def set_tuning(self, register_budget, blocks_per_sm, items_per_turn=1):
        """Pin the launch shape (blocks_per_sm = 0: tune again at the next step)."""
        st = lib().gdg_batch_set_tuning(self._h, register_budget, blocks_per_sm, items_per_turn)
        if st != OK:
            raise GdgError(st, "gdg_batch_set_tuning")

    def stats(self, i):
        su, sv = PcgStats(), PcgStats()
        st = lib().gdg_batch_stats(self._h, i, ctypes.byref(su), ctypes.byref(sv))
        if st != OK:
            raise GdgError(st, "gdg_batch_stats")
        f = lambda s: dict(max_iters=s.max_iters, mean_iters=s.mean_iters, unconverged=s.unconverged,
                           max_sweeps=s.max_sweeps, mean_sweeps=s.mean_sweeps)
        return f(su), f(sv)


class Mlp:
    """Network parameters on the device (FP32 master + BF16 working weights)
    and the library's training kernels.  Only argument marshalling here."""

    def __init__(self, params, device="cuda"):
        import torch
        self.params = torch.as_tensor(params, dtype=torch.float32, device=device).contiguous()
        assert self.params.numel() == MLP_NPARAM
        self.wbf16 = torch.zeros(MLP_NWEIGHT, dtype=torch.int16, device=device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.step_count = 0
        self._partial = None
        st = lib().gdg_mlp_to_bf16(_fptr(self.params), _uptr(self.wbf16), _stream())
        if st != OK:
            raise GdgError(st, "gdg_mlp_to_bf16")

    def forward(self, X, Y, stream=None):
        B = X.numel() // MLP_IN
        st = lib().gdg_mlp_forward(_uptr(self.wbf16), _fptr(self.params), _fptr(X, B * MLP_IN), B,
                                   _fptr(Y, B * MLP_OUT), _stream(stream))
        if st != OK:
            raise GdgError(st, "gdg_mlp_forward")

    def backward(self, X, T, idx=None, stream=None):
        """Loss (device tensor) and self.grad for rows idx (int32 device tensor) or all rows."""
        import torch
        B = idx.numel() if idx is not None else X.numel() // MLP_IN
        need = lib().gdg_mlp_partial_len(B)
        if self._partial is None or self._partial.numel() < need:
            self._partial = torch.empty(need, dtype=torch.float32, device=X.device)
        ip = ctypes.c_void_p(idx.data_ptr()) if idx is not None else None
        st = lib().gdg_mlp_backward(_uptr(self.wbf16), _fptr(self.params), _fptr(X), _fptr(T), ip, B,
                                    ctypes.c_void_p(self._partial.data_ptr()), _fptr(self.grad),
                                    _fptr(self.loss), _stream(stream))
        if st != OK:
            raise GdgError(st, "gdg_mlp_backward")
        return self.loss

    def adam(self, lr, stream=None):
        self.step_count += 1
        st = lib().gdg_mlp_adam(_fptr(self.params), _fptr(self.m), _fptr(self.v), _fptr(self.grad),
                                self.step_count, ctypes.c_float(lr), _uptr(self.wbf16), _stream(stream))
        if st != OK:
            raise GdgError(st, "gdg_mlp_adam")
