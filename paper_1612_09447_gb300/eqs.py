"""ctypes binding of ``libeqs.so`` (the C ABI declared in include/eqs.h).

Each ``eqs_*`` function here has the C function's name and arguments and only
marshals them: host arrays are numpy arrays, device buffers are CUDA torch
tensors (passed by data pointer).  A non-zero status raises ``EqsError``
carrying ``eqs_last_error``.  There is no fallback: if the library is
missing, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libeqs.so")

EQS_OK, EQS_ERR_ARG, EQS_ERR_MESH, EQS_ERR_CUDA = 0, -1, -2, -3
EQS_ERR_NOCONV, EQS_ERR_TIMEOUT, EQS_ERR_NAN, EQS_ERR_STATE = -4, -5, -6, -7
EQS_PREC_FP64, EQS_PREC_MIXED = 0, 1
EQS_GUESS_PREV, EQS_GUESS_MLP, EQS_GUESS_ZERO, EQS_GUESS_SPE = 0, 1, 2, 3
EQS_GUESS_POD, EQS_GUESS_POD2, EQS_GUESS_SPE_MLP = 4, 5, 6
EQS_MAX_STAGES = 64
EQS_KERNEL_SPE_GRAM, EQS_KERNEL_ELEM, EQS_KERNEL_PCG_PQ = 0, 1, 2
EQS_KERNEL_ENS_SPE_GRAM, EQS_KERNEL_ENS_ELEM, EQS_KERNEL_ENS_PCG_PQ = 16, 17, 18


class EqsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"eqs status {status}: {msg}")
        self.status = status


class eqs_material(C.Structure):
    _fields_ = [("eps_r", C.c_double), ("kappa_lo", C.c_double), ("kappa_hi", C.c_double),
                ("E0", C.c_double), ("w", C.c_double)]


class eqs_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("theta", C.c_double), ("coarse_max", C.c_int),
                ("max_levels", C.c_int), ("cheb_degree", C.c_int), ("cheb_alpha", C.c_double),
                ("rtol", C.c_double), ("max_iter", C.c_int), ("guess", C.c_int),
                ("flexible", C.c_int), ("persistent", C.c_int), ("blocks_per_sm", C.c_int),
                ("spe_n", C.c_int), ("host_loop", C.c_int), ("barrier_polls", C.c_longlong),
                ("split_m", C.c_int), ("pod_k", C.c_int), ("pod_m", C.c_int),
                ("pod_min_iters", C.c_int), ("fill_lanes", C.c_int), ("coarse_split", C.c_int),
                ("defer_sums", C.c_int)]


class eqs_batch_stats(C.Structure):
    _fields_ = [("n_inst", C.c_int), ("s", C.c_int), ("total_iters", C.c_int64),
                ("max_iters", C.c_int), ("max_relres", C.c_double), ("status", C.c_int),
                ("launches", C.c_int64)]


EQS_ENS_W = 4


class eqs_ens_stats(C.Structure):
    _fields_ = [("s", C.c_int), ("total_iters", C.c_int * EQS_ENS_W), ("passes", C.c_int),
                ("max_iters", C.c_int), ("max_relres", C.c_double), ("status", C.c_int),
                ("launches", C.c_int64)]


class eqs_adapt_stats(C.Structure):
    _fields_ = [("h_used", C.c_double), ("h_next", C.c_double), ("err", C.c_double), ("s", C.c_int),
                ("tries", C.c_int), ("total_iters", C.c_int)]


class eqs_step_stats(C.Structure):
    _fields_ = [("s", C.c_int), ("total_iters", C.c_int), ("max_iters", C.c_int),
                ("iters", C.c_int * EQS_MAX_STAGES), ("max_relres", C.c_double),
                ("status", C.c_int), ("launches", C.c_int64), ("guess_kept", C.c_int)]


_lib = None


def lib():
    """Load libeqs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"{_LIB_PATH} is missing: run __graft_entry__.build() first")
        _lib = C.CDLL(_LIB_PATH)
        _declare(_lib)
    return _lib


def _declare(L):
    P, I64, I, D = C.c_void_p, C.c_int64, C.c_int, C.c_double
    sig = {
        "eqs_opts_default": (None, [C.POINTER(eqs_opts)]),
        "eqs_mesh_create": (I, [P, I64, P, I64, P, C.POINTER(C.c_void_p)]),
        "eqs_mesh_create_p2": (I, [P, I64, P, I64, P, C.POINTER(C.c_void_p)]),
        "eqs_set_materials": (I, [P, P, I, P]),
        "eqs_set_dirichlet": (I, [P, D, D, D]),
        "eqs_amg_setup": (I, [P, C.POINTER(eqs_opts)]),
        "eqs_apply_K": (I, [P, P, P]),
        "eqs_apply_K_static": (I, [P, P, P]),
        "eqs_solve_M": (I, [P, P, P, I, D, P]),
        "eqs_vcycle": (I, [P, P, P]),
        "eqs_spmv_M": (I, [P, P, P]),
        "eqs_spmv_M32": (I, [P, P, P]),
        "eqs_rkc_step": (I, [P, P, D, D, I, C.POINTER(eqs_step_stats)]),
        "eqs_rkc_dt_bound": (D, [P, I]),
        "eqs_get_step_stats": (I, [P, C.POINTER(eqs_step_stats)]),
        "eqs_set_stream": (I, [P, P]),
        "eqs_get_sizes": (I, [P, P, P, P]),
        "eqs_amg_info": (I, [P, P, P, P]),
        "eqs_amg_aggregates": (I, [P, I, P]),
        "eqs_set_guess": (I, [P, I]),
        "eqs_guess_set_params": (I, [P, P, I]),
        "eqs_guess_get_params": (I, [P, P, I]),
        "eqs_guess_record": (I, [P, I64]),
        "eqs_guess_train": (I, [P, I, I, C.c_float, C.c_uint64, P, P]),
        "eqs_guess_grad": (I, [P, P, P, I, P, P]),
        "eqs_guess_eval": (I, [P, P, P]),
        "eqs_guess_eval_spe": (I, [P, P, P, P, P]),
        "eqs_guess_train_batches": (I, [P, P, P, I, I, C.c_float, P]),
        "eqs_spe_eval": (I, [P, P, P, I, P]),
        "eqs_batch_create": (I, [P, I, I, C.POINTER(C.c_void_p)]),
        "eqs_batch_rkc_step": (I, [P, P, D, D, I, C.POINTER(eqs_batch_stats)]),
        "eqs_batch_get_stats": (I, [P, C.POINTER(eqs_batch_stats), P]),
        "eqs_batch_info": (I, [P, P, P]),
        "eqs_batch_set_barrier_polls": (I, [P, C.c_longlong]),
        "eqs_batch_destroy": (I, [P]),
        "eqs_batch_last_error": (C.c_char_p, [P]),
        "eqs_ens_rkc_step": (I, [P, P, P, D, D, I, C.POINTER(eqs_ens_stats)]),
        "eqs_ens_apply_K": (I, [P, P, P]),
        "eqs_ens_get_step_stats": (I, [P, C.POINTER(eqs_ens_stats)]),
        "eqs_ens_solve_M": (I, [P, P, P, P]),
        "eqs_pod_eval": (I, [P, P, I, P, P]),
        "eqs_launch_kernel": (I, [P, I]),
        "eqs_convert_check": (I, [P, I, P]),
        "eqs_ens_spe_eval": (I, [P, P, P, P, P]),
        "eqs_pod_info": (I, [P, P, P, P, P, P]),
        "eqs_rkc_adaptive_step": (I, [P, P, D, D, D, D, I, C.POINTER(eqs_adapt_stats)]),
        "eqs_destroy": (I, [P]),
        "eqs_last_error": (C.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _check(status, ctx=None):
    if status != EQS_OK:
        raise EqsError(status, lib().eqs_last_error(ctx).decode())


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(C.c_void_p)


def _dev(t):
    """Device pointer of a CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


# ------------------------------------------------------------- C entry points
def eqs_opts_default():
    o = eqs_opts()
    lib().eqs_opts_default(C.byref(o))
    return o


def eqs_mesh_create(xyz, tets, node_tag):
    """Linear (n_tets x 4) or quadratic (n_tets x 10) tetrahedral mesh."""
    xyz, pxyz = _host(xyz, np.float64)
    tets, ptets = _host(tets, np.int32)
    tag, ptag = _host(node_tag, np.uint8)
    out = C.c_void_p()
    create = lib().eqs_mesh_create_p2 if tets.ndim == 2 and tets.shape[1] == 10 else lib().eqs_mesh_create
    _check(create(pxyz, len(xyz), ptets, len(tets), ptag, C.byref(out)))
    return out


def eqs_set_materials(ctx, tet_mat, materials):
    tm, ptm = _host(tet_mat, np.uint8)
    arr = (eqs_material * len(materials))()
    for k, m in enumerate(materials):
        t = m.as_tuple() if hasattr(m, "as_tuple") else tuple(m)
        arr[k] = eqs_material(*t)
    _check(lib().eqs_set_materials(ctx, ptm, len(materials), arr), ctx)


def eqs_set_dirichlet(ctx, V0, freq_hz, phase=0.0):
    _check(lib().eqs_set_dirichlet(ctx, V0, freq_hz, phase), ctx)


def eqs_amg_setup(ctx, opts=None):
    _check(lib().eqs_amg_setup(ctx, C.byref(opts) if opts is not None else None), ctx)


def eqs_apply_K(ctx, x, y):
    _check(lib().eqs_apply_K(ctx, _dev(x), _dev(y)), ctx)


def eqs_apply_K_static(ctx, x, y):
    _check(lib().eqs_apply_K_static(ctx, _dev(x), _dev(y)), ctx)


def eqs_solve_M(ctx, rhs, z, nrhs=1, rtol=0.0):
    iters = (C.c_int * nrhs)()
    st = lib().eqs_solve_M(ctx, _dev(rhs), _dev(z), nrhs, rtol, iters)
    _check(st, ctx)
    return list(iters)


def eqs_vcycle(ctx, r, z):
    _check(lib().eqs_vcycle(ctx, _dev(r), _dev(z)), ctx)


def eqs_spmv_M(ctx, x, y):
    _check(lib().eqs_spmv_M(ctx, _dev(x), _dev(y)), ctx)


def eqs_spmv_M32(ctx, x, y):
    _check(lib().eqs_spmv_M32(ctx, _dev(x), _dev(y)), ctx)


def eqs_rkc_step(ctx, x, t, dt, s, want_stats=True):
    st = eqs_step_stats() if want_stats else None
    _check(lib().eqs_rkc_step(ctx, _dev(x), t, dt, s, C.byref(st) if st is not None else None), ctx)
    return st


def eqs_rkc_adaptive_step(ctx, x, t, h_try, atol, rtol, s_max=EQS_MAX_STAGES):
    """One accepted adaptive RKC step from t (x: CUDA float64 node vector)."""
    st = eqs_adapt_stats()
    _check(lib().eqs_rkc_adaptive_step(ctx, _dev(x), t, h_try, atol, rtol, s_max, C.byref(st)), ctx)
    return st


def eqs_get_step_stats(ctx):
    st = eqs_step_stats()
    _check(lib().eqs_get_step_stats(ctx, C.byref(st)), ctx)
    return st


def eqs_rkc_dt_bound(ctx, s):
    return lib().eqs_rkc_dt_bound(ctx, s)


def eqs_set_stream(ctx, stream_ptr):
    _check(lib().eqs_set_stream(ctx, C.c_void_p(stream_ptr) if stream_ptr else None), ctx)


def eqs_get_sizes(ctx):
    n, nf, nt = C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().eqs_get_sizes(ctx, C.byref(n), C.byref(nf), C.byref(nt)), ctx)
    return n.value, nf.value, nt.value


def eqs_amg_info(ctx):
    nl = C.c_int()
    rows = (C.c_int64 * 16)()
    nnz = (C.c_int64 * 16)()
    _check(lib().eqs_amg_info(ctx, C.byref(nl), rows, nnz), ctx)
    return [rows[i] for i in range(nl.value)], [nnz[i] for i in range(nl.value)]


def eqs_amg_aggregates(ctx, level, n_rows):
    out = np.empty(n_rows, dtype=np.int32)
    _check(lib().eqs_amg_aggregates(ctx, level, out.ctypes.data_as(C.c_void_p)), ctx)
    return out


def eqs_set_guess(ctx, mode):
    _check(lib().eqs_set_guess(ctx, mode), ctx)


def eqs_guess_set_params(ctx, theta):
    th, pth = _host(theta, np.float32)
    _check(lib().eqs_guess_set_params(ctx, pth, len(th)), ctx)


def eqs_guess_get_params(ctx):
    out = np.empty(1377, dtype=np.float32)
    _check(lib().eqs_guess_get_params(ctx, out.ctypes.data_as(C.c_void_p), len(out)), ctx)
    return out


def eqs_guess_record(ctx, capacity):
    _check(lib().eqs_guess_record(ctx, int(capacity)), ctx)


def eqs_guess_train(ctx, iters, batch, lr, seed):
    lf, ll = C.c_float(), C.c_float()
    _check(lib().eqs_guess_train(ctx, iters, batch, lr, seed, C.byref(lf), C.byref(ll)), ctx)
    return lf.value, ll.value


def eqs_guess_grad(ctx, X, T):
    X, pX = _host(X, np.float32)
    T, pT = _host(T, np.float32)
    g = np.empty(1377, dtype=np.float32)
    loss = C.c_float()
    _check(lib().eqs_guess_grad(ctx, pX, pT, len(T), g.ctypes.data_as(C.c_void_p), C.byref(loss)), ctx)
    return g, loss.value


def eqs_guess_train_batches(ctx, X, T, lr):
    """X: (n_batches, B, 8), T: (n_batches, B) host arrays; returns the losses."""
    X, pX = _host(X, np.float32)
    T, pT = _host(T, np.float32)
    nb, B = T.shape
    if X.shape != (nb, B, 8):
        raise ValueError("X must be (n_batches, B, 8)")
    losses = np.empty(nb, dtype=np.float32)
    _check(lib().eqs_guess_train_batches(ctx, pX, pT, B, nb, lr, losses.ctypes.data_as(C.c_void_p)), ctx)
    return losses


def eqs_guess_eval_spe(ctx, x0, H, R, z0):
    _check(lib().eqs_guess_eval_spe(ctx, _dev(x0), _dev(H), _dev(R), _dev(z0)), ctx)


def eqs_guess_eval(ctx, H, z0):
    _check(lib().eqs_guess_eval(ctx, _dev(H), _dev(z0)), ctx)


def _bcheck(status, b=None):
    if status != EQS_OK:
        raise EqsError(status, lib().eqs_batch_last_error(b).decode())


def eqs_batch_create(ctxs, rows_per_block=1024):
    arr = (C.c_void_p * len(ctxs))(*[c.value if isinstance(c, C.c_void_p) else c for c in ctxs])
    out = C.c_void_p()
    _bcheck(lib().eqs_batch_create(arr, len(ctxs), rows_per_block, C.byref(out)))
    return out


def eqs_batch_rkc_step(b, xs, t, dt, s, want_stats=True):
    arr = (C.c_void_p * len(xs))(*[x.data_ptr() for x in xs])
    st = eqs_batch_stats() if want_stats else None
    _bcheck(lib().eqs_batch_rkc_step(b, arr, t, dt, s, C.byref(st) if st is not None else None), b)
    return st


def eqs_batch_get_stats(b, n):
    st = eqs_batch_stats()
    per = (C.c_int64 * n)()
    _bcheck(lib().eqs_batch_get_stats(b, C.byref(st), per), b)
    return st, list(per)


def eqs_batch_info(b):
    tb, rpb = C.c_int(), C.c_int()
    _bcheck(lib().eqs_batch_info(b, C.byref(tb), C.byref(rpb)), b)
    return tb.value, rpb.value


def eqs_batch_set_barrier_polls(b, polls):
    _bcheck(lib().eqs_batch_set_barrier_polls(b, polls), b)


def eqs_batch_destroy(b):
    if b:
        lib().eqs_batch_destroy(b)


def eqs_pod_eval(ctx, X, K, b, x0):
    _check(lib().eqs_pod_eval(ctx, _dev(X), K, _dev(b), _dev(x0)), ctx)


def eqs_pod_info(ctx):
    cnt, m, rb, ad = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    lam = (C.c_double * 16)()
    _check(lib().eqs_pod_info(ctx, C.byref(cnt), C.byref(m), C.byref(rb), C.byref(ad), lam), ctx)
    return {"count": cnt.value, "modes": m.value, "rebuilds": rb.value, "adds": ad.value,
            "lam": list(lam)}


def eqs_spe_eval(ctx, X, b, n, x0):
    _check(lib().eqs_spe_eval(ctx, _dev(X), _dev(b), n, _dev(x0)), ctx)


def eqs_ens_rkc_step(ctx, x, v0_scale, t, dt, s, want_stats=True):
    """One RKC step of the 4-trajectory ensemble; x: CUDA float64 tensor of
    shape (4, n_nodes) (trajectory c in row c), v0_scale: 4 drive scales."""
    st = eqs_ens_stats() if want_stats else None
    v, vp = _host(v0_scale, np.float64)
    if v.size != EQS_ENS_W:
        raise ValueError("v0_scale needs 4 values")
    _check(lib().eqs_ens_rkc_step(ctx, _dev(x), vp, t, dt, s, C.byref(st) if st is not None else None), ctx)
    return st


def eqs_ens_apply_K(ctx, X, Y):
    """Y = K(X) X for four columns; X, Y: CUDA float64 tensors of shape
    (4, n_nodes) (column c in row c)."""
    _check(lib().eqs_ens_apply_K(ctx, _dev(X), _dev(Y)), ctx)


def eqs_ens_get_step_stats(ctx):
    st = eqs_ens_stats()
    _check(lib().eqs_ens_get_step_stats(ctx, C.byref(st)), ctx)
    return st


def eqs_ens_solve_M(ctx, rhs, z):
    """Blocked solve of 4 columns: rhs, z CUDA float64 tensors (4, n_free);
    z holds the start vectors and receives the solutions."""
    it = (C.c_int * EQS_ENS_W)()
    _check(lib().eqs_ens_solve_M(ctx, _dev(rhs), _dev(z), it), ctx)
    return list(it)


def eqs_ens_spe_eval(ctx, X, b, x0, r0):
    """X: CUDA float64 (6, 4, n_free) history (newest first); b, x0, r0: (4, n_free)."""
    _check(lib().eqs_ens_spe_eval(ctx, _dev(X), _dev(b), _dev(x0), _dev(r0)), ctx)


def eqs_convert_check(f, f_wide):
    """f (CUDA float32) -> f_wide (CUDA float64) with the kernels' widening."""
    _check(lib().eqs_convert_check(_dev(f), f.numel(), _dev(f_wide)))


def eqs_launch_kernel(ctx, kernel):
    _check(lib().eqs_launch_kernel(ctx, kernel), ctx)


def eqs_destroy(ctx):
    if ctx:
        lib().eqs_destroy(ctx)


def eqs_last_error(ctx=None):
    return lib().eqs_last_error(ctx).decode()


# ---------------------------------------------------------- convenience
class Solver:
    """One EQS instance on the GPU: mesh + materials + drive + AMG setup.

    ``problem`` has xyz, tets, node_tag, tet_mat, materials, V0, freq, phase
    (eqs_inputs.Problem).  Vectors are CUDA float64 tensors."""

    def __init__(self, problem, precision=EQS_PREC_FP64, rtol=1e-8, **opt):
        import torch

        self.ctx = None
        unknown = sorted(set(opt) - {f[0] for f in eqs_opts._fields_})
        if unknown:  # a misspelt option must not pass silently as a plain attribute
            raise TypeError(f"unknown solver option(s): {', '.join(unknown)}")
        self.torch = torch
        self.p = problem
        self.ctx = eqs_mesh_create(problem.xyz, problem.tets, problem.node_tag)
        eqs_set_materials(self.ctx, problem.tet_mat, problem.materials)
        eqs_set_dirichlet(self.ctx, problem.V0, problem.freq, problem.phase)
        o = eqs_opts_default()
        o.precision = precision
        o.rtol = rtol
        for k, v in opt.items():
            setattr(o, k, v)
        self.opts = o
        eqs_amg_setup(self.ctx, o)
        self.n, self.nf, self.nt = eqs_get_sizes(self.ctx)

    def close(self):
        if self.ctx:
            eqs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def zeros(self, n=None):
        return self.torch.zeros(n or self.n, dtype=self.torch.float64, device="cuda")

    def apply_K(self, x):
        y = self.torch.empty_like(x)
        eqs_apply_K(self.ctx, x, y)
        return y

    def spmv_M(self, x):
        y = self.torch.empty_like(x)
        eqs_spmv_M(self.ctx, x, y)
        return y

    def vcycle(self, r):
        z = self.torch.empty_like(r)
        eqs_vcycle(self.ctx, r, z)
        return z

    def solve_M(self, rhs, z0=None, rtol=0.0):
        nrhs = 1 if rhs.dim() == 1 else rhs.shape[0]
        z = self.torch.zeros_like(rhs) if z0 is None else z0.clone()
        iters = eqs_solve_M(self.ctx, rhs.contiguous(), z, nrhs, rtol)
        return z, iters

    def step(self, x, t, dt, s, stats=True):
        return eqs_rkc_step(self.ctx, x, t, dt, s, stats)

    def last_stats(self):
        return eqs_get_step_stats(self.ctx)

    def dt_bound(self, s):
        return eqs_rkc_dt_bound(self.ctx, s)

    def amg_info(self):
        return eqs_amg_info(self.ctx)
