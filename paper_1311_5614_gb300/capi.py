"""ctypes binding of the C ABI in ``include/ib.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does
nothing but check and convert arguments: torch CUDA tensors are passed as raw
device pointers, numpy arrays as host pointers, the problem's CUDA stream is
torch's current stream at set-up.  All arithmetic runs in ``libibmg.so``.
If the library has not been built, loading it raises immediately; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libibmg.so")

IB_OK = 0
IB_ERR_INVALID_ARG = 1
IB_ERR_CUDA = 2
IB_ERR_OOM = 3
IB_ERR_NOT_CONVERGED = 4
IB_ERR_BREAKDOWN = 5
IB_ERR_SINGULAR = 6
IB_ERR_TIMEOUT = 7
STATUS_NAMES = {0: "IB_OK", 1: "IB_ERR_INVALID_ARG", 2: "IB_ERR_CUDA", 3: "IB_ERR_OOM",
                4: "IB_ERR_NOT_CONVERGED", 5: "IB_ERR_BREAKDOWN", 6: "IB_ERR_SINGULAR",
                7: "IB_ERR_TIMEOUT"}

DELTA = {"peskin4": 0, "cos4": 1}
PRECISION = {"fp64": 0, "fp32": 1, "mixed": 2}
JACOBIAN = {"clamped": 0, "exact": 1}
WALLS = {"periodic": 0, "noslip": 1}
TIME_METHOD = {"implicit": 0, "explicit": 1}


class ib_params(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32), ("L", ctypes.c_double), ("rho", ctypes.c_double),
                ("mu", ctypes.c_double), ("dt", ctypes.c_double), ("delta", ctypes.c_int32),
                ("box", ctypes.c_int32), ("nu1", ctypes.c_int32), ("nu2", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("jacobian", ctypes.c_int32), ("tol", ctypes.c_double),
                ("max_iters", ctypes.c_int32), ("escalate", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("walls", ctypes.c_int32), ("lid", ctypes.c_double), ("time_method", ctypes.c_int32)]


class ib_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("rel_res_true", ctypes.c_double), ("rel_res_est", ctypes.c_double),
                ("t_setup_ms", ctypes.c_double), ("t_solve_ms", ctypes.c_double),
                ("n_struct_boxes", ctypes.c_int32), ("status", ctypes.c_int32),
                ("escalated_at", ctypes.c_int32), ("learned_used", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class IBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(code, code), msg))
        self.code = code


_lib = None

_P = ctypes.c_void_p
_SIGS = {
    "ib_default_params": (None, [ctypes.POINTER(ib_params)]),
    "ib_setup": (ctypes.c_int, [ctypes.POINTER(ib_params), ctypes.c_int32, _P, ctypes.c_int32, _P, _P,
                                _P, _P, ctypes.POINTER(_P)]),
    "ib_update_points": (ctypes.c_int, [_P, _P]),
    "ib_apply": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "ib_vcycle": (ctypes.c_int, [_P, _P, _P]),
    "ib_rhs": (ctypes.c_int, [_P, _P, _P]),
    "ib_solve_step": (ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ib_stats)]),
    "ib_solve_step_newton": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int32, ctypes.c_double,
                                            ctypes.POINTER(ib_stats), ctypes.POINTER(ctypes.c_double)]),
    "ib_solve": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ib_stats)]),
    "ib_num_levels": (ctypes.c_int, [_P]),
    "ib_level_size": (ctypes.c_int, [_P, ctypes.c_int32]),
    "ib_num_struct_boxes": (ctypes.c_int, [_P, ctypes.c_int32]),
    "ib_tail_grid": (ctypes.c_int, [_P, ctypes.c_int32]),
    "ib_tail_cluster": (ctypes.c_int, [_P, ctypes.c_int32]),
    "ib_box_form": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32]),
    "ib_launch_count": (ctypes.c_int64, [_P, ctypes.c_int32]),
    "ib_profile": (ctypes.c_int, [_P, ctypes.c_int32]),
    "ib_profile_read": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "ib_vcycle_timer": (ctypes.c_int, [_P, ctypes.c_int32]),
    "ib_vcycle_timer_read": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(ctypes.c_double)]),
    "ib_apply_noalloc": (ctypes.c_int, [ctypes.POINTER(ib_params), ctypes.c_int32, _P, ctypes.c_int32, _P,
                                        _P, _P, _P, _P, _P]),
    "ib_setup_batch": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "ib_solve_step_batch": (ctypes.c_int, [_P, _P, _P, _P, _P]),
    "ib_batch_size": (ctypes.c_int, [_P]),
    "ib_batch_problem": (_P, [_P, ctypes.c_int32]),
    "ib_destroy_batch": (None, [_P]),
    "ib_unet_num_params": (ctypes.c_int64, []),
    "ib_unet_create": (ctypes.c_int, [ctypes.c_int32, _P, _P, ctypes.POINTER(_P)]),
    "ib_unet_set_params": (ctypes.c_int, [_P, _P]),
    "ib_unet_get_params": (ctypes.c_int, [_P, _P]),
    "ib_unet_forward": (ctypes.c_int, [_P, _P, _P]),
    "ib_unet_loss_grad": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(ctypes.c_double), _P]),
    "ib_unet_train_step": (ctypes.c_int, [_P, _P, _P, ctypes.c_float, ctypes.POINTER(ctypes.c_double)]),
    "ib_unet_destroy": (None, [_P]),
    "ib_set_learned_stage": (ctypes.c_int, [_P, _P]),
    "ib_learned_pair": (ctypes.c_int, [_P, _P, _P, _P]),
    "ib_learned_chain": (ctypes.c_int, [_P, _P, _P, _P]),
    "ib_destroy": (None, [_P]),
    "ib_last_error": (ctypes.c_char_p, []),
    "ib_version": (ctypes.c_char_p, []),
}


def lib():
    """Load ``libibmg.so`` (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libibmg.so is not built (run __graft_entry__.build()): " + LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code):
    if code != IB_OK:
        raise IBError(code, lib().ib_last_error().decode())


def _dev_ptr(t, numel, name):
    import torch

    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise TypeError("%s must be a contiguous float64 tensor" % name)
    if t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), numel))
    return ctypes.c_void_p(t.data_ptr())


def ib_default_params():
    p = ib_params()
    lib().ib_default_params(ctypes.byref(p))
    return p


def make_params(N, L=1.0, rho=1.0, mu=1.0, dt=1e-2, delta="peskin4", box=1, nu1=1, nu2=1,
                precision="fp64", jacobian="clamped", tol=1e-8, max_iters=100, escalate=True, restart=0,
                walls="periodic", lid=0.0, time_method="implicit"):
    p = ib_default_params()
    p.N, p.L, p.rho, p.mu, p.dt = int(N), float(L), float(rho), float(mu), float(dt)
    p.delta = DELTA[delta] if isinstance(delta, str) else int(delta)
    p.box, p.nu1, p.nu2 = int(box), int(nu1), int(nu2)
    p.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
    p.jacobian = JACOBIAN[jacobian] if isinstance(jacobian, str) else int(jacobian)
    p.tol, p.max_iters = float(tol), int(max_iters)
    p.escalate = 1 if escalate else 0
    p.restart = int(restart)
    p.walls = WALLS[walls] if isinstance(walls, str) else int(walls)
    p.lid = float(lid)
    p.time_method = TIME_METHOD[time_method] if isinstance(time_method, str) else int(time_method)
    return p


def ib_setup(params, X, springs, kappa, rest, stream=None):
    """Create a problem from host arrays; returns the opaque handle (c_void_p)."""
    import torch

    X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, 2)
    springs = np.ascontiguousarray(springs, dtype=np.int32).reshape(-1, 2)
    kappa = np.ascontiguousarray(kappa, dtype=np.float64).ravel()
    rest = np.ascontiguousarray(rest, dtype=np.float64).ravel()
    if kappa.size != springs.shape[0] or rest.size != springs.shape[0]:
        raise ValueError("kappa and rest need one value per spring")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    out = ctypes.c_void_p()
    _check(lib().ib_setup(ctypes.byref(params), X.shape[0], X.ctypes.data_as(_P),
                          springs.shape[0], springs.ctypes.data_as(_P), kappa.ctypes.data_as(_P),
                          rest.ctypes.data_as(_P), ctypes.c_void_p(stream), ctypes.byref(out)))
    return out


def ib_update_points(prob, X_dev, n_points):
    _check(lib().ib_update_points(prob, _dev_ptr(X_dev, 2 * n_points, "X")))


def ib_apply(prob, level, w, y):
    n = ib_level_size(prob, level)
    _check(lib().ib_apply(prob, int(level), _dev_ptr(w, 3 * n * n, "w"), _dev_ptr(y, 3 * n * n, "y")))


def ib_vcycle(prob, b, w):
    n = ib_level_size(prob, 0)
    _check(lib().ib_vcycle(prob, _dev_ptr(b, 3 * n * n, "b"), _dev_ptr(w, 3 * n * n, "w")))


def ib_rhs(prob, u_n, b):
    n = ib_level_size(prob, 0)
    _check(lib().ib_rhs(prob, _dev_ptr(u_n, 2 * n * n, "u_n"), _dev_ptr(b, 3 * n * n, "b")))


def ib_solve_step(prob, u_n, up, X, n_points, raise_on_not_converged=False):
    """One implicit step; returns the ib_stats as a dict (status included)."""
    n = ib_level_size(prob, 0)
    st = ib_stats()
    code = lib().ib_solve_step(prob, _dev_ptr(u_n, 2 * n * n, "u_n"), _dev_ptr(up, 3 * n * n, "up"),
                               _dev_ptr(X, 2 * n_points, "X") if n_points else None, ctypes.byref(st))
    if code != IB_OK and (code != IB_ERR_NOT_CONVERGED or raise_on_not_converged):
        _check(code)
    return st.as_dict()


def ib_solve_step_newton(prob, u_n, up, X, n_points, max_newton=20, tol_newton=1e-9,
                         raise_on_not_converged=False):
    """One implicit step with the spring force at the new positions (Newton's method);
    returns the ib_stats as a dict plus newton_iters and newton_change."""
    n = ib_level_size(prob, 0)
    st = ib_stats()
    nw = (ctypes.c_double * 2)()
    code = lib().ib_solve_step_newton(prob, _dev_ptr(u_n, 2 * n * n, "u_n"), _dev_ptr(up, 3 * n * n, "up"),
                                      _dev_ptr(X, 2 * n_points, "X") if n_points else None, int(max_newton),
                                      float(tol_newton), ctypes.byref(st), nw)
    if code != IB_OK and (code != IB_ERR_NOT_CONVERGED or raise_on_not_converged):
        _check(code)
    d = st.as_dict()
    d["newton_iters"] = int(nw[0])
    d["newton_change"] = float(nw[1])
    return d


def ib_solve(prob, b, x, raise_on_not_converged=False):
    """Solve A_0 x = b with the current hierarchy; returns the ib_stats as a dict."""
    n = ib_level_size(prob, 0)
    st = ib_stats()
    code = lib().ib_solve(prob, _dev_ptr(b, 3 * n * n, "b"), _dev_ptr(x, 3 * n * n, "x"), ctypes.byref(st))
    if code != IB_OK and (code != IB_ERR_NOT_CONVERGED or raise_on_not_converged):
        _check(code)
    return st.as_dict()


def ib_num_levels(prob):
    return lib().ib_num_levels(prob)


def ib_level_size(prob, level):
    return lib().ib_level_size(prob, int(level))


def ib_num_struct_boxes(prob, level):
    return lib().ib_num_struct_boxes(prob, int(level))


IB_NOALLOC_MAX_POINTS = 65536


def ib_apply_noalloc(params, X, springs, kappa, rest, w, y, stream=None):
    """y = A_0 w without a problem handle and without any device allocation.

    For callers that cannot allocate device memory (no cudaMalloc stalls inside a
    time step, or all memory owned by the caller's own pool).  X, springs (int32),
    kappa, rest, w and y are CUDA tensors; the scratch is the library's static
    device array, so concurrent calls on one GPU race and must be serialised.
    """
    import torch

    n = int(params.N)
    npts = 0 if X is None else X.numel() // 2
    ns = 0 if springs is None else springs.numel() // 2
    if springs is not None and (springs.dtype != torch.int32 or not springs.is_cuda or
                                not springs.is_contiguous()):
        raise TypeError("springs must be a contiguous int32 CUDA tensor")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    _check(lib().ib_apply_noalloc(
        ctypes.byref(params), npts, _dev_ptr(X, 2 * npts, "X") if npts else None, ns,
        ctypes.c_void_p(springs.data_ptr()) if ns else None,
        _dev_ptr(kappa, ns, "kappa") if ns else None, _dev_ptr(rest, ns, "rest") if ns else None,
        _dev_ptr(w, 3 * n * n, "w"), _dev_ptr(y, 3 * n * n, "y"), ctypes.c_void_p(stream)))


KERNEL_CLASSES = ("stokes", "box", "interp", "spread", "transfer", "coarse", "krylov", "setup", "other")


def ib_launch_count(prob, kclass=-1):
    return int(lib().ib_launch_count(prob, int(kclass)))


def ib_profile(prob, enable):
    _check(lib().ib_profile(prob, 1 if enable else 0))


def ib_profile_read(prob, kclass):
    """(launches, total_ms, algorithmic_bytes) of one kernel class since ib_profile."""
    n = ctypes.c_int64()
    ms = ctypes.c_double()
    by = ctypes.c_double()
    _check(lib().ib_profile_read(prob, int(kclass), ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by)))
    return int(n.value), float(ms.value), float(by.value)


def ib_vcycle_timer(prob, enable):
    _check(lib().ib_vcycle_timer(prob, 1 if enable else 0))


def ib_vcycle_timer_read(prob, precision):
    """(V-cycles timed, their total device ms) for the V-cycle of one precision."""
    n, ms = ctypes.c_int64(), ctypes.c_double()
    _check(lib().ib_vcycle_timer_read(prob, PRECISION[precision], ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


def ib_destroy(prob):
    if prob:
        lib().ib_destroy(prob)


def ib_last_error():
    return lib().ib_last_error().decode()


def ib_version():
    return lib().ib_version().decode()


def ib_setup_batch(params_list, X_list, springs_list, kappa_list, rest_list, stream=None):
    """Create a batch of independent problems from per-problem host arrays."""
    import torch

    n = len(params_list)
    P = (ib_params * n)(*params_list)
    pt = np.zeros(n + 1, dtype=np.int32)
    sp = np.zeros(n + 1, dtype=np.int32)
    for k in range(n):
        pt[k + 1] = pt[k] + np.asarray(X_list[k]).reshape(-1, 2).shape[0]
        sp[k + 1] = sp[k] + np.asarray(springs_list[k]).reshape(-1, 2).shape[0]
    X = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64).reshape(-1, 2) for x in X_list]))
    S = np.ascontiguousarray(np.concatenate([np.asarray(x, np.int32).reshape(-1, 2) for x in springs_list]))
    K = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64).ravel() for x in kappa_list]))
    R = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float64).ravel() for x in rest_list]))
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    out = ctypes.c_void_p()
    _check(lib().ib_setup_batch(n, P, pt.ctypes.data_as(_P), X.ctypes.data_as(_P), sp.ctypes.data_as(_P),
                                S.ctypes.data_as(_P), K.ctypes.data_as(_P), R.ctypes.data_as(_P),
                                ctypes.c_void_p(stream), ctypes.byref(out)))
    return out, pt, sp


def ib_solve_step_batch(batch, u_n_all, up_all, X_all, nprob, raise_on_not_converged=False):
    """One implicit step of every problem; returns the per-problem stats dicts."""
    st = (ib_stats * nprob)()

    def ptr(t):
        return None if t is None else ctypes.c_void_p(t.data_ptr())

    code = lib().ib_solve_step_batch(batch, ptr(u_n_all), ptr(up_all), ptr(X_all), st)
    if code != IB_OK and (code != IB_ERR_NOT_CONVERGED or raise_on_not_converged):
        _check(code)
    return [s.as_dict() for s in st]


class IBBatch:
    """Independent problems solved together (each on its own stream)."""

    def __init__(self, problems, **kw):
        """kw: parameters for every problem; a list or tuple gives one value per problem."""
        plist = []
        for k, p in enumerate(problems):
            d = dict(L=p.L, rho=p.rho, mu=p.mu, dt=p.dt, delta=p.delta, box=p.box, nu1=p.nu1, nu2=p.nu2,
                     tol=p.tol, max_iters=p.max_iters, jacobian="clamped" if p.clamped else "exact")
            d.update({key: (v[k] if isinstance(v, (list, tuple)) else v) for key, v in kw.items()})
            plist.append(make_params(p.N, **d))
        self.params = plist
        self.sizes = [p.N for p in problems]
        self.handle, self.pt_off, self.sp_off = ib_setup_batch(
            plist, [p.X for p in problems], [p.springs for p in problems], [p.kappa for p in problems],
            [p.rest for p in problems])
        self.up_off = np.concatenate([[0], np.cumsum([3 * n * n for n in self.sizes])]).astype(np.int64)
        self.nprob = len(problems)

    def solve_step(self, u_n_all, up_all, X_all, raise_on_not_converged=False):
        return ib_solve_step_batch(self.handle, u_n_all, up_all, X_all, self.nprob, raise_on_not_converged)

    def problem(self, k):
        return lib().ib_batch_problem(self.handle, int(k))

    def close(self):
        if self.handle:
            lib().ib_destroy_batch(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _f32_ptr(t, numel, name):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError("%s must be a contiguous float32 CUDA tensor" % name)
    if t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), numel))
    return ctypes.c_void_p(t.data_ptr())


def ib_unet_num_params():
    return int(lib().ib_unet_num_params())


class UNet:
    """The learned stage's network (parameters on the device; FP32 master, BF16 copy)."""

    def __init__(self, N, params=None, stream=None):
        import torch

        self.N = int(N)
        self.n_params = ib_unet_num_params()
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        host = None
        if params is not None:
            host = np.ascontiguousarray(params, dtype=np.float32)
            if host.size != self.n_params:
                raise ValueError("expected %d parameters" % self.n_params)
        out = ctypes.c_void_p()
        _check(lib().ib_unet_create(self.N, host.ctypes.data_as(_P) if host is not None else None,
                                    ctypes.c_void_p(stream), ctypes.byref(out)))
        self.handle = out

    def set_params(self, params):
        host = np.ascontiguousarray(params, dtype=np.float32)
        _check(lib().ib_unet_set_params(self.handle, host.ctypes.data_as(_P)))

    def get_params(self):
        host = np.empty(self.n_params, dtype=np.float32)
        _check(lib().ib_unet_get_params(self.handle, host.ctypes.data_as(_P)))
        return host

    def forward(self, x, y):
        n = self.N * self.N
        _check(lib().ib_unet_forward(self.handle, _f32_ptr(x, 4 * n, "x"), _f32_ptr(y, 3 * n, "y")))
        return y

    def loss_grad(self, x, t):
        n = self.N * self.N
        L = ctypes.c_double()
        g = np.empty(self.n_params, dtype=np.float32)
        _check(lib().ib_unet_loss_grad(self.handle, _f32_ptr(x, 4 * n, "x"), _f32_ptr(t, 3 * n, "t"),
                                       ctypes.byref(L), g.ctypes.data_as(_P)))
        return float(L.value), g

    def train_step(self, x, t, lr):
        n = self.N * self.N
        L = ctypes.c_double()
        _check(lib().ib_unet_train_step(self.handle, _f32_ptr(x, 4 * n, "x"), _f32_ptr(t, 3 * n, "t"),
                                        ctypes.c_float(lr), ctypes.byref(L)))
        return float(L.value)

    def close(self):
        if self.handle:
            lib().ib_unet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class IBSolver:
    """Owns one problem handle; methods forward to the functions above."""

    def __init__(self, N, X, springs, kappa, rest, **kw):
        self.params = make_params(N, **kw)
        self.N = int(N)
        self.n_points = int(np.asarray(X).reshape(-1, 2).shape[0])
        self.handle = ib_setup(self.params, X, springs, kappa, rest)

    @classmethod
    def from_problem(cls, prob, **overrides):
        kw = dict(L=prob.L, rho=prob.rho, mu=prob.mu, dt=prob.dt, delta=prob.delta, box=prob.box,
                  nu1=prob.nu1, nu2=prob.nu2, tol=prob.tol, max_iters=prob.max_iters,
                  jacobian="clamped" if prob.clamped else "exact")
        kw.update(overrides)
        return cls(prob.N, prob.X, prob.springs, prob.kappa, prob.rest, **kw)

    @property
    def n_levels(self):
        return ib_num_levels(self.handle)

    def level_size(self, level):
        return ib_level_size(self.handle, level)

    def struct_boxes(self, level):
        return ib_num_struct_boxes(self.handle, level)

    def tail_grid(self, precision="fp32"):
        return lib().ib_tail_grid(self.handle, PRECISION[precision])

    def tail_cluster(self, precision="fp32"):
        return lib().ib_tail_cluster(self.handle, PRECISION[precision])

    def box_forms(self, precision="fp32"):
        """Box-kernel form chosen by the set-up autotuner on each smoothing level (see ib_box_form)."""
        return [lib().ib_box_form(self.handle, PRECISION[precision], l) for l in range(self.n_levels - 1)]

    def apply(self, level, w, y):
        ib_apply(self.handle, level, w, y)
        return y

    def vcycle(self, b, w):
        ib_vcycle(self.handle, b, w)
        return w

    def rhs(self, u_n, b):
        ib_rhs(self.handle, u_n, b)
        return b

    def update_points(self, X_dev):
        ib_update_points(self.handle, X_dev, self.n_points)

    def solve_step(self, u_n, up, X, raise_on_not_converged=False):
        return ib_solve_step(self.handle, u_n, up, X, self.n_points, raise_on_not_converged)

    def solve_step_newton(self, u_n, up, X, max_newton=20, tol_newton=1e-9, raise_on_not_converged=False):
        """One implicit step with the spring force at X^{n+1}, by Newton's method."""
        return ib_solve_step_newton(self.handle, u_n, up, X, self.n_points, max_newton, tol_newton,
                                    raise_on_not_converged)

    def solve(self, b, x, raise_on_not_converged=False):
        """x = A_0^{-1} b by MG-preconditioned FGMRES (the points do not move)."""
        return ib_solve(self.handle, b, x, raise_on_not_converged)

    def set_learned_stage(self, net):
        _check(lib().ib_set_learned_stage(self.handle, net.handle if net is not None else None))

    def learned_pair(self, x, in4, target):
        n = self.N * self.N
        _check(lib().ib_learned_pair(self.handle, _dev_ptr(x, 3 * n, "x"), _f32_ptr(in4, 4 * n, "in4"),
                                     _f32_ptr(target, 3 * n, "target")))

    def learned_chain(self, e, in4, target):
        n = self.N * self.N
        _check(lib().ib_learned_chain(self.handle, _dev_ptr(e, 3 * n, "e"), _f32_ptr(in4, 4 * n, "in4"),
                                      _f32_ptr(target, 3 * n, "target")))

    def launch_count(self, kclass=-1):
        return ib_launch_count(self.handle, kclass)

    def profile(self, enable):
        ib_profile(self.handle, enable)

    def profile_read(self):
        return {name: ib_profile_read(self.handle, i) for i, name in enumerate(KERNEL_CLASSES)}

    def vcycle_timer(self, enable):
        ib_vcycle_timer(self.handle, enable)

    def vcycle_timer_read(self, precision):
        return ib_vcycle_timer_read(self.handle, precision)

    def close(self):
        if self.handle:
            ib_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
