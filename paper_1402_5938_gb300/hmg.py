"""Thin ctypes binding of libhmg (include/hmg.h): argument marshalling only.

Every function takes and returns the same things as its C counterpart; device vectors are
passed as CUDA tensors (float64, contiguous, on the problem's device) and the stream is
the current PyTorch stream unless one is given. No numerical work happens in Python.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libhmg.so")

HMG_OK, HMG_EINVAL, HMG_ENOMEM, HMG_ENOCONV, HMG_EDEVICE, HMG_ETIMEOUT, HMG_EBUSY, HMG_ENAN = 0, -1, -2, -3, -4, -5, -6, -7
HIER = {"h": 0, "p": 1}
SMOOTHER = {"jacobi": 0, "cheb": 1, "l1jacobi": 2, "blockjacobi": 3}
MODE = {"mg": 0, "pcg": 1}
PREC = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3}
ARITH = {"fp64": 0, "df64": 1}  # arithmetic of the finest level's FP64 operator


class HmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"hmg status {status}: {msg}")
        self.status = status


# void mu_fn(size_t n, const double* xyz, double* mu, void* user)
MU_FN = ctypes.CFUNCTYPE(None, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                         ctypes.c_void_p)


class Desc(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int), ("nelem", ctypes.c_int * 3), ("order", ctypes.c_int),
        ("warp_amp", ctypes.c_double), ("mu_a", ctypes.c_double), ("mu_b", ctypes.c_double),
        ("mu_k", ctypes.c_double), ("hier", ctypes.c_int), ("n_hlevels", ctypes.c_int),
        ("smoother", ctypes.c_int), ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int),
        ("omega", ctypes.c_double), ("arnoldi_iters", ctypes.c_int),
        ("cheb_lo_frac", ctypes.c_double), ("cheb_safety", ctypes.c_double),
        ("arnoldi_seed", ctypes.c_ulonglong), ("smooth_prec", ctypes.c_int), ("solve_graph", ctypes.c_int),
        ("node_xyz", ctypes.POINTER(ctypes.c_double)), ("mu_fn", MU_FN), ("mu_user", ctypes.c_void_p),
        ("fp64_arith", ctypes.c_int),
    ]


_lib = None

# name -> (restype, argtypes)
_P, _D, _I, _V = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_void_p
_SIGS = {
    "hmg_desc_default": (_I, [ctypes.POINTER(Desc)]),
    "hmg_setup": (_I, [ctypes.POINTER(Desc), _V, ctypes.POINTER(_P)]),
    "hmg_destroy": (_I, [_P]),
    "hmg_nlevels": (_I, [_P]),
    "hmg_ndof": (ctypes.c_size_t, [_P, _I]),
    "hmg_level_variants": (_I, [_P, _I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "hmg_level_info": (_I, [_P, _I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_size_t)]),
    "hmg_device_bytes": (ctypes.c_size_t, [_P]),
    "hmg_node_coords": (_I, [_P, _I, _V, _V]),
    "hmg_rhs": (_I, [_P, _V, _V, _V]),
    "hmg_apply": (_I, [_P, _I, _V, _V, _V]),
    "hmg_apply_f32": (_I, [_P, _I, _V, _V, _V]),
    "hmg_diag_inv": (_I, [_P, _I, _V, _V]),
    "hmg_lambda_max": (_I, [_P, _I, ctypes.POINTER(_D)]),
    "hmg_prolong": (_I, [_P, _I, _V, _V, _V]),
    "hmg_restrict": (_I, [_P, _I, _V, _V, _V]),
    "hmg_smooth": (_I, [_P, _I, _V, _V, _I, _I, _V]),
    "hmg_vcycle": (_I, [_P, _V, _V, _V]),
    "hmg_solve": (_I, [_P, _I, _V, _V, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), _V]),
    "hmg_solve_low_order": (_I, [_P, _P, _V, _V, _D, _I, _D, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_longlong),
                                 ctypes.POINTER(_D), _V]),
    "hmg_apply_host": (_I, [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(_D), _V]),
    "hmg_solve_host": (_I, [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(_D), _D, _I, ctypes.POINTER(_I),
                            ctypes.POINTER(_D), _V]),
    "hmg_measure_peak": (_I, [_I, ctypes.POINTER(_D)]),
    "hmg_restrict_noalloc": (_I, [_I, ctypes.POINTER(ctypes.c_int), _I, _I, _I, _V, _V, _V]),
    "hmg_solve_batched": (_I, [ctypes.POINTER(_P), _I, _I, ctypes.POINTER(_V), ctypes.POINTER(_V), _D, _I,
                               ctypes.POINTER(_I), ctypes.POINTER(ctypes.POINTER(_D)), ctypes.POINTER(_I), _V]),
    "hmg_desc_ndof": (ctypes.c_size_t, [ctypes.POINTER(Desc)]),
    "hmg_estimate_bytes": (_I, [ctypes.POINTER(Desc), ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    "hmg_server_create": (_I, [_I, ctypes.c_size_t, _I, ctypes.POINTER(_P)]),
    "hmg_server_submit": (_I, [_P, ctypes.POINTER(Desc), ctypes.POINTER(_D), _D, _I, _I, ctypes.POINTER(ctypes.c_ulonglong)]),
    "hmg_server_poll": (_I, [_P, ctypes.c_ulonglong, ctypes.POINTER(_D), ctypes.POINTER(_I), ctypes.POINTER(_D),
                             ctypes.POINTER(_D)]),
    "hmg_server_wait": (_I, [_P, ctypes.c_ulonglong, _D, ctypes.POINTER(_D), ctypes.POINTER(_I), ctypes.POINTER(_D),
                             ctypes.POINTER(_D)]),
    "hmg_server_stats": (_I, [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                              ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(_I)]),
    "hmg_server_destroy": (_I, [_P]),
    "hmg_selftest_bounded_wait": (_I, [ctypes.c_uint, ctypes.POINTER(_I)]),
    "hmg_batch_create": (_I, [ctypes.POINTER(_P), _I, _I, _I, ctypes.POINTER(_P)]),
    "hmg_batch_solve": (_I, [_P, ctypes.POINTER(_V), ctypes.POINTER(_V), _D, _I, ctypes.POINTER(_I),
                             ctypes.POINTER(ctypes.POINTER(_D)), ctypes.POINTER(_I), _V]),
    "hmg_batch_info": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_longlong)]),
    "hmg_batch_destroy": (_I, [_P]),
    "hmg_fine_applies": (ctypes.c_longlong, [_P]),
    "hmg_launch_count": (ctypes.c_longlong, []),
    "hmg_status_string": (ctypes.c_char_p, [_I]),
    "hmg_last_error": (ctypes.c_char_p, []),
    "hmg_host_basis": (_I, [_I, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "hmg_host_hessenberg_max_real_eig": (_I, [ctypes.POINTER(_D), _I, ctypes.POINTER(_D)]),
}


def lib():
    """Load libhmg.so (built in-tree by __graft_entry__.build()); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != HMG_OK:
        raise HmgError(status, lib().hmg_last_error().decode())


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(stream)
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t, n=None, dtype=None):
    import torch
    if not (t.is_cuda and t.dtype == (dtype or torch.float64) and t.is_contiguous()):
        raise TypeError(f"expected a contiguous {dtype or torch.float64} CUDA tensor")
    if n is not None and t.numel() < n:
        raise ValueError(f"tensor has {t.numel()} entries, the level needs {n}")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(a, n):
    """Pointer to n contiguous float64 host values (numpy array or CPU tensor)."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("expected a contiguous float64 numpy array")
        if a.size < n:
            raise ValueError(f"array has {a.size} entries, the level needs {n}")
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    import torch
    if not (isinstance(a, torch.Tensor) and not a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()):
        raise TypeError("expected a contiguous float64 host array or CPU tensor")
    if a.numel() < n:
        raise ValueError(f"tensor has {a.numel()} entries, the level needs {n}")
    return ctypes.cast(ctypes.c_void_p(a.data_ptr()), ctypes.POINTER(ctypes.c_double))


def measure_peak(what):
    """hmg_measure_peak: measured TFLOP/s of 'fp64' FMA, 'fp32' FMA, 'fp64_mma' or 'fp64_both' (FMA and
    MMA warps at once) on the current device."""
    v = ctypes.c_double()
    _check(lib().hmg_measure_peak({"fp64": 0, "fp32": 1, "fp64_mma": 2, "fp64_both": 3}[what], ctypes.byref(v)))
    return v.value


def make_desc(prob: dict) -> Desc:
    """hmg_desc from a workload dictionary (see synth.problem)."""
    d = Desc()
    _check(lib().hmg_desc_default(ctypes.byref(d)))
    d.dim = prob["dim"]
    E = list(prob["nelem"]) + [1] * (3 - len(prob["nelem"]))
    d.nelem = (ctypes.c_int * 3)(*E)
    d.order = prob["order"]
    d.warp_amp = prob.get("warp_amp", 0.0)
    d.mu_a, d.mu_b, d.mu_k = prob.get("mu_a", 1.0), prob.get("mu_b", 0.0), prob.get("mu_k", 2.0)
    d.hier = HIER[prob.get("hier", "h")]
    d.n_hlevels = prob.get("n_hlevels", 3)
    d.smoother = SMOOTHER[prob.get("smoother", "cheb")]
    d.nu_pre, d.nu_post = prob.get("nu_pre", 3), prob.get("nu_post", 3)
    d.omega = prob.get("omega", 2.0 / 3.0)
    d.arnoldi_iters = prob.get("arnoldi_iters", 10)
    d.cheb_lo_frac = prob.get("cheb_lo_frac", 0.25)
    d.cheb_safety = prob.get("cheb_safety", 1.0)
    d.arnoldi_seed = prob.get("arnoldi_seed", 0)
    d.smooth_prec = PREC[prob.get("smooth_prec", "fp64")]
    d.solve_graph = int(prob.get("solve_graph", 1))
    d.fp64_arith = ARITH[prob.get("fp64_arith", "fp64")]
    keep = []
    if prob.get("node_xyz") is not None:
        xyz = np.ascontiguousarray(prob["node_xyz"], dtype=np.float64)
        keep.append(xyz)
        d.node_xyz = xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    if prob.get("mu_fn") is not None:
        f, dim = prob["mu_fn"], d.dim

        def _mu(n, xyz, mu, user):
            try:
                x = np.ctypeslib.as_array(xyz, shape=(dim * n,)).reshape(dim, n)
                np.ctypeslib.as_array(mu, shape=(n,))[:] = np.asarray(f(x), dtype=np.float64).reshape(n)
            except Exception:  # reported by the library as a non-finite coefficient
                np.ctypeslib.as_array(mu, shape=(n,))[:] = np.nan
        cb = MU_FN(_mu)
        keep.append(cb)
        d.mu_fn = cb
    d._keep = keep  # the arrays and the callback must outlive hmg_setup
    return d


class Problem:
    """Owner of one hmg_problem handle (device-resident hierarchy)."""

    def __init__(self, prob: dict, stream=None):
        self.desc = make_desc(prob)
        h = ctypes.c_void_p()
        _check(lib().hmg_setup(ctypes.byref(self.desc), _stream(stream), ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().hmg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # introspection
    def nlevels(self):
        return lib().hmg_nlevels(self.h)

    def ndof(self, level=0):
        return lib().hmg_ndof(self.h, level)

    def level_info(self, level):
        E = (ctypes.c_int * 3)()
        p = ctypes.c_int()
        n = ctypes.c_size_t()
        _check(lib().hmg_level_info(self.h, level, E, ctypes.byref(p), ctypes.byref(n)))
        return tuple(E), p.value, n.value

    def device_bytes(self):
        return lib().hmg_device_bytes(self.h)

    def level_variants(self, level):
        """(FP64 apply variant, V-cycle operator variant) the autotuner chose on `level`."""
        a, b = ctypes.c_int(), ctypes.c_int()
        _check(lib().hmg_level_variants(self.h, level, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def fine_applies(self):
        return lib().hmg_fine_applies(self.h)

    # operations (same names as the C ABI without the prefix)
    def node_coords(self, level, xyz, stream=None):
        _check(lib().hmg_node_coords(self.h, level, _ptr(xyz, self.desc.dim * self.ndof(level)), _stream(stream)))

    def rhs(self, f, b, stream=None):
        n = self.ndof(0)
        _check(lib().hmg_rhs(self.h, _ptr(f, n), _ptr(b, n), _stream(stream)))

    def apply(self, level, x, y, stream=None):
        n = self.ndof(level)
        _check(lib().hmg_apply(self.h, level, _ptr(x, n), _ptr(y, n), _stream(stream)))

    def apply_f32(self, level, x, y, stream=None):
        import torch
        n = self.ndof(level)
        _check(lib().hmg_apply_f32(self.h, level, _ptr(x, n, torch.float32), _ptr(y, n, torch.float32),
                                   _stream(stream)))

    def diag_inv(self, level, out, stream=None):
        _check(lib().hmg_diag_inv(self.h, level, _ptr(out, self.ndof(level)), _stream(stream)))

    def lambda_max(self, level):
        v = ctypes.c_double()
        _check(lib().hmg_lambda_max(self.h, level, ctypes.byref(v)))
        return v.value

    def prolong(self, level, xc, xf, stream=None):
        _check(lib().hmg_prolong(self.h, level, _ptr(xc, self.ndof(level + 1)), _ptr(xf, self.ndof(level)),
                                 _stream(stream)))

    def restrict(self, level, rf, rc, stream=None):
        _check(lib().hmg_restrict(self.h, level, _ptr(rf, self.ndof(level)), _ptr(rc, self.ndof(level + 1)),
                                  _stream(stream)))

    def smooth(self, level, b, x, steps, zero_guess=False, stream=None):
        n = self.ndof(level)
        _check(lib().hmg_smooth(self.h, level, _ptr(b, n), _ptr(x, n), int(steps), int(bool(zero_guess)),
                                _stream(stream)))

    def vcycle(self, r, z, stream=None):
        n = self.ndof(0)
        _check(lib().hmg_vcycle(self.h, _ptr(r, n), _ptr(z, n), _stream(stream)))

    def solve(self, mode, b, u, rtol=1e-8, maxit=1000, stream=None, raise_on_noconv=False):
        """Returns (status, iterations, residual history as a numpy array)."""
        n = self.ndof(0)
        it = ctypes.c_int()
        hist = (ctypes.c_double * (maxit + 1))()
        st = lib().hmg_solve(self.h, MODE[mode], _ptr(b, n), _ptr(u, n), float(rtol), int(maxit),
                             ctypes.byref(it), hist, _stream(stream))
        if st not in (HMG_OK, HMG_ENOCONV, HMG_ENAN) or (raise_on_noconv and st != HMG_OK):
            _check(st)
        return st, it.value, np.array(hist[: it.value + 1])


    def apply_host(self, level, x_host, y_host, stream=None):
        """hmg_apply_host: y_host = A_k x_host with host buffers (numpy float64 arrays or CPU
        tensors, contiguous, hmg_ndof(level) entries; page-locked tensors copy fastest)."""
        n = self.ndof(level)
        _check(lib().hmg_apply_host(self.h, level, _host_ptr(x_host, n), _host_ptr(y_host, n), _stream(stream)))

    def solve_host(self, mode, f_host, u_host, rtol=1e-8, maxit=1000, stream=None):
        """hmg_solve_host: nodal f on the host -> u on the host. Returns (status, iterations, history)."""
        n = self.ndof(0)
        it = ctypes.c_int()
        hist = (ctypes.c_double * (maxit + 1))()
        st = lib().hmg_solve_host(self.h, MODE[mode], _host_ptr(f_host, n), _host_ptr(u_host, n), float(rtol),
                                  int(maxit), ctypes.byref(it), hist, _stream(stream))
        if st not in (HMG_OK, HMG_ENOCONV, HMG_ENAN):
            _check(st)
        return st, it.value, np.array(hist[: it.value + 1])

    def solve_low_order(self, low, b, u, rtol=1e-8, maxit=1000, inner_rtol=1e-12, stream=None):
        """hmg_solve_low_order: PCG preconditioned by the low-order problem `low` (a Problem of
        order 1 on this problem's nodes). Returns (status, iterations, inner iterations, history)."""
        n = self.ndof(0)
        it = ctypes.c_int()
        inner = ctypes.c_longlong()
        hist = (ctypes.c_double * (maxit + 1))()
        st = lib().hmg_solve_low_order(self.h, low.h, _ptr(b, n), _ptr(u, n), float(rtol), int(maxit),
                                       float(inner_rtol), ctypes.byref(it), ctypes.byref(inner), hist,
                                       _stream(stream))
        if st not in (HMG_OK, HMG_ENOCONV, HMG_ENAN):
            _check(st)
        return st, it.value, inner.value, np.array(hist[: it.value + 1])


def solve_batched(problems, mode, bs, us, rtol=1e-8, maxit=1000, stream=None):
    """hmg_solve_batched: returns (statuses, iterations, histories) for the n problems."""
    n = len(problems)
    H = (_P * n)(*[p.h for p in problems])
    B = (_V * n)(*[_ptr(b, p.ndof(0)) for p, b in zip(problems, bs)])
    U = (_V * n)(*[_ptr(u, p.ndof(0)) for p, u in zip(problems, us)])
    its = (_I * n)()
    sts = (_I * n)()
    hists = [(_D * (maxit + 1))() for _ in range(n)]
    HP = (ctypes.POINTER(_D) * n)(*[ctypes.cast(h, ctypes.POINTER(_D)) for h in hists])
    st = lib().hmg_solve_batched(H, n, MODE[mode], B, U, float(rtol), int(maxit), its, HP, sts, _stream(stream))
    if st not in (HMG_OK, HMG_ENOCONV):
        _check(st)
    return list(sts), list(its), [np.array(h[: its[i] + 1]) for i, h in enumerate(hists)]


def noalloc_lengths(dim, nelem_fine, order_fine, order_coarse, halve_mesh):
    """(fine, coarse) node counts of hmg_restrict_noalloc's level pair: prod_a (E_a p_f + 1) and
    prod_a (E_a' p_c + 1) over the first dim axes, E_a' = E_a / 2 when the mesh is halved."""
    nf = nc = 1
    for a in range(int(dim)):
        e = int(nelem_fine[a])
        nf *= e * int(order_fine) + 1
        nc *= (e // 2 if halve_mesh else e) * int(order_coarse) + 1
    return nf, nc


class BatchPlan:
    """hmg_batch_*: a plan that solves `problems` together, one graph launch per solve."""

    def __init__(self, problems, mode="pcg", maxit_cap=1000):
        self.problems = list(problems)
        n = len(self.problems)
        H = (_P * n)(*[p.h for p in self.problems])
        h = ctypes.c_void_p()
        _check(lib().hmg_batch_create(H, n, MODE[mode], int(maxit_cap), ctypes.byref(h)))
        self.h, self.cap = h, int(maxit_cap)

    def info(self):
        """(groups, kernels launched per loop iteration)."""
        g, k = ctypes.c_int(), ctypes.c_longlong()
        _check(lib().hmg_batch_info(self.h, ctypes.byref(g), ctypes.byref(k)))
        return g.value, k.value

    def solve(self, bs, us, rtol=1e-8, maxit=None, stream=None):
        """Returns (statuses, iterations, histories)."""
        maxit = self.cap if maxit is None else int(maxit)
        n = len(self.problems)
        B = (_V * n)(*[_ptr(b, p.ndof(0)) for p, b in zip(self.problems, bs)])
        U = (_V * n)(*[_ptr(u, p.ndof(0)) for p, u in zip(self.problems, us)])
        its, sts = (_I * n)(), (_I * n)()
        hists = [(_D * (maxit + 1))() for _ in range(n)]
        HP = (ctypes.POINTER(_D) * n)(*[ctypes.cast(x, ctypes.POINTER(_D)) for x in hists])
        st = lib().hmg_batch_solve(self.h, B, U, float(rtol), maxit, its, HP, sts, _stream(stream))
        if st not in (HMG_OK, HMG_ENOCONV, HMG_ENAN):
            _check(st)
        return list(sts), list(its), [np.array(x[: its[i] + 1]) for i, x in enumerate(hists)]

    def close(self):
        if getattr(self, "h", None):
            lib().hmg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def restrict_noalloc(dim, nelem_fine, order_fine, order_coarse, halve_mesh, rf, rc, stream=None):
    """hmg_restrict_noalloc: r_c = P^T r_f for a structured mesh given by its sizes, using
    only the library's fixed device storage (no handle, no allocation). rf and rc must hold
    the fine and coarse levels' node counts (noalloc_lengths); shorter tensors raise ValueError."""
    E = list(nelem_fine) + [1] * (3 - len(nelem_fine))
    nf, nc = noalloc_lengths(dim, E, order_fine, order_coarse, halve_mesh)
    _check(lib().hmg_restrict_noalloc(int(dim), (ctypes.c_int * 3)(*E), int(order_fine), int(order_coarse),
                                      int(bool(halve_mesh)), _ptr(rf, nf), _ptr(rc, nc), _stream(stream)))


def launch_count():
    """Kernels launched by libhmg so far in this process."""
    return lib().hmg_launch_count()


def host_basis(order):
    n = order + 1
    r, g, w = (ctypes.c_double * n)(), (ctypes.c_double * n)(), (ctypes.c_double * n)()
    _check(lib().hmg_host_basis(order, r, g, w))
    return np.array(r), np.array(g), np.array(w)


def host_hessenberg_max_real_eig(H):
    H = np.ascontiguousarray(H, dtype=np.float64)
    m = H.shape[0]
    out = ctypes.c_double()
    st = lib().hmg_host_hessenberg_max_real_eig(H.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), m,
                                                ctypes.byref(out))
    _check(st)
    return out.value


def desc_ndof(prob: dict) -> int:
    d = make_desc(prob)
    return lib().hmg_desc_ndof(ctypes.byref(d))


def estimate_bytes(prob: dict):
    """(resident, peak) device bytes of hmg_setup for this workload (no device touched)."""
    d = make_desc(prob)
    r, pk = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().hmg_estimate_bytes(ctypes.byref(d), ctypes.byref(r), ctypes.byref(pk)))
    return r.value, pk.value


class Server:
    """hmg_server: continuous batching of independent solves (see include/hmg.h)."""

    def __init__(self, device=0, hbm_budget=8 << 30, max_slots=4):
        h = ctypes.c_void_p()
        _check(lib().hmg_server_create(int(device), int(hbm_budget), int(max_slots), ctypes.byref(h)))
        self.h = h

    def submit(self, prob: dict, f_host, rtol=1e-8, mode="pcg", maxit=1000):
        d = make_desc(prob)
        f = np.ascontiguousarray(f_host, dtype=np.float64)
        if f.size != lib().hmg_desc_ndof(ctypes.byref(d)):
            raise ValueError("right-hand side length does not match the problem")
        t = ctypes.c_ulonglong()
        _check(lib().hmg_server_submit(self.h, ctypes.byref(d), f.ctypes.data_as(ctypes.POINTER(_D)), float(rtol),
                                       MODE[mode], int(maxit), ctypes.byref(t)))
        return t.value, f.size

    def _result(self, fn, ticket, n, *extra):
        u = np.zeros(n)
        it, res, lat = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        st = fn(self.h, ctypes.c_ulonglong(ticket), *extra, u.ctypes.data_as(ctypes.POINTER(_D)), ctypes.byref(it),
                ctypes.byref(res), ctypes.byref(lat))
        return st, u, it.value, res.value, lat.value

    def poll(self, ticket, n):
        """(status, u, iterations, final relative residual, latency s); status HMG_EBUSY if not done."""
        return self._result(lib().hmg_server_poll, ticket, n)

    def wait(self, ticket, n, timeout_s=600.0):
        return self._result(lib().hmg_server_wait, ticket, n, ctypes.c_double(timeout_s))

    def stats(self):
        c, h, r, q = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_size_t(), ctypes.c_int()
        _check(lib().hmg_server_stats(self.h, ctypes.byref(c), ctypes.byref(h), ctypes.byref(r), ctypes.byref(q)))
        return dict(completed=c.value, cache_hits=h.value, resident_bytes=r.value, queued=q.value)

    def close(self):
        if getattr(self, "h", None):
            lib().hmg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
