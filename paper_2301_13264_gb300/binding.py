"""ctypes binding of libccsd_gb300.so (see include/ccsd.h).

Argument marshalling only: every function forwards to the C entry point of the
same name.  Arrays may be numpy arrays (host memory) or torch tensors (host or
CUDA memory); they must be contiguous float64.  The library raises no Python
fallback: if it is not built, loading fails with an error.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libccsd_gb300.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_STATE, ERR_NOT_CONVERGED, ERR_COMPLEX_ROOT, ERR_DEGENERATE, ERR_NOT_HF, \
    ERR_TIMEOUT = range(10)
PREC_FP64, PREC_MIXED, PREC_FP64_TC = 0, 1, 2
GEMM_FP64, GEMM_SPLIT, GEMM_FP64_TC = 0, 1, 2


# device-allocator callbacks of ccsd_options: alloc(bytes, stream, ctx) -> pointer or NULL,
# free(pointer, stream, ctx)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class Options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("splits", ctypes.c_int),
        ("relax_orbitals", ctypes.c_int),
        ("tol_res", ctypes.c_double),
        ("tol_eom", ctypes.c_double),
        ("tol_lin", ctypes.c_double),
        ("tol_degen", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("diis_dim", ctypes.c_int),
        ("davidson_block", ctypes.c_int),
        ("davidson_max_sub", ctypes.c_int),
        ("guess", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("tc_min_flops", ctypes.c_double),
        ("refine", ctypes.c_int),
        ("tol_switch", ctypes.c_double),
        ("autotune", ctypes.c_int),
        ("fp64_tc", ctypes.c_int),
        ("alloc", ALLOC_FN),
        ("free", FREE_FN),
        ("alloc_ctx", ctypes.c_void_p),
    ]


class ProfileData(ctypes.Structure):
    _fields_ = [
        ("launches", ctypes.c_longlong),
        ("tc_launches", ctypes.c_longlong),
        ("tc_ms", ctypes.c_double),
        ("tc_flops", ctypes.c_double),
        ("tc_issued_flops", ctypes.c_double),
        ("fp64_launches", ctypes.c_longlong),
        ("fp64_ms", ctypes.c_double),
        ("fp64_flops", ctypes.c_double),
        ("top_launches", ctypes.c_longlong),
        ("top_ms", ctypes.c_double),
        ("top_flops", ctypes.c_double),
        ("top_issued_flops", ctypes.c_double),
        ("ladder_launches", ctypes.c_longlong),
        ("ladder_ms", ctypes.c_double),
        ("ladder_flops", ctypes.c_double),
        ("ladder_issued_flops", ctypes.c_double),
    ]


class CCSDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built ({LIB_PATH}); run paper_2301_13264_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.ccsd_default_options.argtypes = [ctypes.POINTER(Options)]
        L.ccsd_default_options.restype = None
        L.ccsd_create.argtypes = [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(Options),
                                  ctypes.POINTER(_P)]
        L.ccsd_solve_ground.argtypes = [_P, _D, ctypes.POINTER(ctypes.c_int)]
        L.eom_solve_right.argtypes = [_P, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_int)]
        L.eom_solve_left.argtypes = [_P, ctypes.c_int, _D, ctypes.POINTER(ctypes.c_int)]
        L.ccsd_jacobian_transform.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P, _P]
        L.ccsd_residual.argtypes = [_P, _P, _P, _D]
        L.ccsd_get_amplitudes.argtypes = [_P, _P, _P]
        L.ccsd_set_amplitudes.argtypes = [_P, _P, _P, _D]
        L.ccsd_get_states.argtypes = [_P, ctypes.c_int, _D, _P, _P]
        L.ccsd_coupling_densities.argtypes = [_P, ctypes.c_int, ctypes.c_int, _P, _P]
        L.ccsd_derivative_coupling.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _D]
        L.ccsd_stats.argtypes = [_P, _D, _D, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong)]
        L.ccsd_profile_start.argtypes = [_P]
        L.ccsd_profile_start.restype = ctypes.c_int
        L.ccsd_profile_stop.argtypes = [_P, ctypes.POINTER(ProfileData)]
        L.ccsd_profile_stop.restype = ctypes.c_int
        L.ccsd_profile_records.argtypes = [_P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.ccsd_profile_records.restype = ctypes.c_int
        L.ccsd_strerror.argtypes = [ctypes.c_int]
        L.ccsd_strerror.restype = ctypes.c_char_p
        L.ccsd_last_error.argtypes = [_P]
        L.ccsd_last_error.restype = ctypes.c_char_p
        L.ccsd_destroy.argtypes = [_P]
        L.ccsd_destroy.restype = None
        L.ccsd_describe_program.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.c_size_t]
        L.ccsd_describe_program.restype = ctypes.c_longlong
        for name in ("ccsd_create", "ccsd_solve_ground", "eom_solve_right", "eom_solve_left",
                     "ccsd_jacobian_transform", "ccsd_residual", "ccsd_get_amplitudes", "ccsd_set_amplitudes", "ccsd_get_states",
                     "ccsd_coupling_densities", "ccsd_derivative_coupling", "ccsd_stats"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(x):
    """Raw pointer of a contiguous float64 numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous float64")
        return ctypes.c_void_p(x.ctypes.data)
    # torch tensor
    import torch
    if x.dtype != torch.float64 or not x.is_contiguous():
        raise ValueError("tensors must be contiguous float64")
    return ctypes.c_void_p(x.data_ptr())


def _check(h, status):
    if status != OK:
        msg = lib().ccsd_last_error(h).decode() if h else (lib().ccsd_strerror(status).decode() + ": " +
                                                         lib().ccsd_last_error(None).decode())
        raise CCSDError(status, msg)


def ccsd_default_options(**kw) -> Options:
    opt = Options()
    lib().ccsd_default_options(ctypes.byref(opt))
    names = {n for n, _ in Options._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown option {k!r}")
        if k == "stream" and v is not None and not isinstance(v, int):
            v = v.cuda_stream  # torch.cuda.Stream
        setattr(opt, k, v)
    return opt


def ccsd_create(eps, h, B, o, v, naux, options: Options | None = None):
    handle = _P()
    st = lib().ccsd_create(_ptr(eps), _ptr(h), _ptr(B), o, v, naux,
                           ctypes.byref(options) if options is not None else None, ctypes.byref(handle))
    _check(None, st)
    return handle


def ccsd_solve_ground(h):
    e = ctypes.c_double()
    it = ctypes.c_int()
    _check(h, lib().ccsd_solve_ground(h, ctypes.byref(e), ctypes.byref(it)))
    return e.value, it.value


def eom_solve_right(h, nroots):
    w = (ctypes.c_double * nroots)()
    it = ctypes.c_int()
    _check(h, lib().eom_solve_right(h, nroots, w, ctypes.byref(it)))
    return list(w), it.value


def eom_solve_left(h, nroots):
    w = (ctypes.c_double * nroots)()
    it = ctypes.c_int()
    _check(h, lib().eom_solve_left(h, nroots, w, ctypes.byref(it)))
    return list(w), it.value


def ccsd_jacobian_transform(h, side, nvec, x, y):
    _check(h, lib().ccsd_jacobian_transform(h, side, nvec, _ptr(x), _ptr(y)))


def ccsd_residual(h, t, omega):
    e = ctypes.c_double()
    _check(h, lib().ccsd_residual(h, _ptr(t), _ptr(omega), ctypes.byref(e)))
    return e.value


def ccsd_set_amplitudes(h, t, lam=None):
    e = ctypes.c_double()
    _check(h, lib().ccsd_set_amplitudes(h, _ptr(t), _ptr(lam), ctypes.byref(e)))
    return e.value


def ccsd_get_amplitudes(h, t=None, lam=None):
    _check(h, lib().ccsd_get_amplitudes(h, _ptr(t), _ptr(lam)))


def ccsd_get_states(h, nroots, right=None, left=None):
    r0 = (ctypes.c_double * nroots)()
    _check(h, lib().ccsd_get_states(h, nroots, r0, _ptr(right), _ptr(left)))
    return list(r0)


def ccsd_coupling_densities(h, k, l, D, Z=None):
    _check(h, lib().ccsd_coupling_densities(h, k, l, _ptr(D), _ptr(Z)))


def ccsd_derivative_coupling(h, k, l, ndir, dh, dB):
    F = (ctypes.c_double * ndir)()
    _check(h, lib().ccsd_derivative_coupling(h, k, l, ndir, _ptr(dh), _ptr(dB), F))
    return list(F)


def ccsd_gradient_densities(h, k, D, Z=None):
    _check(h, lib().ccsd_gradient_densities(h, k, _ptr(D), _ptr(Z)))


def ccsd_energy_gradient(h, k, ndir, dh, dB):
    g = (ctypes.c_double * ndir)()
    _check(h, lib().ccsd_energy_gradient(h, k, ndir, _ptr(dh), _ptr(dB), g))
    return list(g)


def ccsd_branching_plane(h, k, l, ndir, dh, dB):
    """(g, h, G) as three lists of ndir values: grad(E_l - E_k), (E_l - E_k) F_kl and the
    Bearpark-Robb-Schlegel direction."""
    out = (ctypes.c_double * (3 * ndir))()
    _check(h, lib().ccsd_branching_plane(h, k, l, ndir, _ptr(dh), _ptr(dB), out))
    v = list(out)
    return v[:ndir], v[ndir:2 * ndir], v[2 * ndir:]


def ccsd_left_norm(h, k):
    N = ctypes.c_double()
    _check(h, lib().ccsd_left_norm(h, k, ctypes.byref(N)))
    return N.value


def ccsd_normalized_coupling(h, k, l, ndir, dh, dB):
    F = (ctypes.c_double * ndir)()
    _check(h, lib().ccsd_normalized_coupling(h, k, l, ndir, _ptr(dh), _ptr(dB), F))
    return list(F)


def ccsd_transition_density(h, k, l, D):
    _check(h, lib().ccsd_transition_density(h, k, l, _ptr(D)))


def ccsd_connection_term(h, k, l, ndir, W):
    O = (ctypes.c_double * ndir)()
    _check(h, lib().ccsd_connection_term(h, k, l, ndir, _ptr(W), O))
    return list(O)


def ccsd_derivative_coupling_noalloc(h, k, l, ndir, dh, dB):
    """Allocation-free variant; dh and dB must be device tensors, densities held."""
    F = (ctypes.c_double * ndir)()
    L = lib()
    if not getattr(L.ccsd_derivative_coupling_noalloc, "argtypes", None):
        L.ccsd_derivative_coupling_noalloc.argtypes = [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _D]
        L.ccsd_derivative_coupling_noalloc.restype = ctypes.c_int
    _check(h, L.ccsd_derivative_coupling_noalloc(h, k, l, ndir, _ptr(dh), _ptr(dB), F))
    return list(F)


def ccsd_stats(h):
    f64, ftc = ctypes.c_double(), ctypes.c_double()
    g, gt = ctypes.c_longlong(), ctypes.c_longlong()
    _check(h, lib().ccsd_stats(h, ctypes.byref(f64), ctypes.byref(ftc), ctypes.byref(g), ctypes.byref(gt)))
    return {"flops_fp64": f64.value, "flops_tc": ftc.value, "gemms": g.value, "tc_gemms": gt.value}


def ccsd_gemm(form, A, B, C=None, alpha=1.0, beta=0.0, splits=3, reps=1):
    """C = alpha A B^T + beta C in one arithmetic form (GEMM_FP64, GEMM_SPLIT, GEMM_FP64_TC).

    A (M x K), B (N x K), C (M x N): C-contiguous float64 host arrays; C is allocated when None.
    Returns (C, ms) with ms the mean device time of one of `reps` repetitions."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K:
        raise ValueError("A and B must share K")
    if C is None:
        C = np.zeros((M, N))
    ms = ctypes.c_double()
    L = lib()
    L.ccsd_gemm.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                            _P, _P, ctypes.c_double, _P, ctypes.c_int, _D]
    L.ccsd_gemm.restype = ctypes.c_int
    _check(None, L.ccsd_gemm(form, splits, M, N, K, alpha, _ptr(A), _ptr(B), beta, _ptr(C), reps,
                             ctypes.byref(ms)))
    return C, ms.value


def ccsd_set_wait_budget(h, cycles: int):
    """Budget of each tensor-core pipeline wait in GPU clock cycles (0: the default)."""
    L = lib()
    L.ccsd_set_wait_budget.argtypes = [_P, ctypes.c_longlong]
    _check(h, L.ccsd_set_wait_budget(h, int(cycles)))


def ccsd_inject_stall(h):
    """Test hook: the handle's next split-bf16 tensor-core GEMM issues no loads and times out."""
    _check(h, lib().ccsd_inject_stall(h))


def ccsd_profile_start(h):
    _check(h, lib().ccsd_profile_start(h))


def ccsd_profile_stop(h) -> dict:
    d = ProfileData()
    _check(h, lib().ccsd_profile_stop(h, ctypes.byref(d)))
    return {name: getattr(d, name) for name, _ in ProfileData._fields_}


class ProfileRecord(ctypes.Structure):
    _fields_ = [("label", ctypes.c_char * 160), ("engine", ctypes.c_int), ("ladder", ctypes.c_int),
                ("batch", ctypes.c_longlong), ("m", ctypes.c_longlong), ("n", ctypes.c_longlong),
                ("k", ctypes.c_longlong), ("ms", ctypes.c_double), ("flops", ctypes.c_double),
                ("issued_flops", ctypes.c_double)]


def ccsd_profile_records(h) -> list:
    """The GEMM launches of the last ccsd_profile_stop, in launch order, as dicts."""
    n = ctypes.c_int(0)
    _check(h, lib().ccsd_profile_records(h, None, 0, ctypes.byref(n)))
    recs = (ProfileRecord * max(n.value, 1))()
    _check(h, lib().ccsd_profile_records(h, recs, n.value, ctypes.byref(n)))
    out = []
    for r in recs[: n.value]:
        d = {name: getattr(r, name) for name, _ in ProfileRecord._fields_}
        d["label"] = r.label.decode()
        out.append(d)
    return out


def ccsd_destroy(h):
    if h:
        lib().ccsd_destroy(h)


def ccsd_describe_program(which: str) -> str:
    n = lib().ccsd_describe_program(which.encode(), None, 0)
    if n < 0:
        raise ValueError(f"unknown program {which}")
    buf = ctypes.create_string_buffer(n + 1)
    lib().ccsd_describe_program(which.encode(), buf, n + 1)
    return buf.value.decode()


def vector_dim(o: int, v: int) -> int:
    return o * v + o * o * v * v


# ---- learned doubles guess -------------------------------------------------

MLP_PARAMS = 17160
MLP_TRAINABLE = MLP_PARAMS - 7


def _fptr(x, n=None):
    """Raw pointer of a contiguous float32 numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float32 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous float32")
        if n is not None and x.size < n:
            raise ValueError(f"array needs at least {n} elements")
        return ctypes.c_void_p(x.ctypes.data)
    import torch
    if x.dtype != torch.float32 or not x.is_contiguous():
        raise ValueError("tensors must be contiguous float32")
    if n is not None and x.numel() < n:
        raise ValueError(f"tensor needs at least {n} elements")
    return ctypes.c_void_p(x.data_ptr())


def _mlp_fn(name, argtypes):
    f = getattr(lib(), name)
    if not getattr(f, "argtypes", None):
        f.argtypes = argtypes
        f.restype = ctypes.c_int
    return f


def ccsd_mlp_train(X, T, steps, batch=4096, lr=2e-3, seed=0):
    """Train a model on rows X[n, 3] -> T[n]; returns (model float32[MLP_PARAMS], final loss)."""
    n = T.shape[0]
    model = np.zeros(MLP_PARAMS, dtype=np.float32)
    loss = ctypes.c_float()
    f = _mlp_fn("ccsd_mlp_train", [_P, _P, ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                   ctypes.c_ulonglong, _P, ctypes.POINTER(ctypes.c_float)])
    _check(None, f(_fptr(X, 3 * n), _fptr(T, n), n, steps, batch, lr, seed, _fptr(model), ctypes.byref(loss)))
    return model, loss.value


def ccsd_mlp_predict(model, X, out):
    n = out.shape[0]
    f = _mlp_fn("ccsd_mlp_predict", [_P, _P, ctypes.c_longlong, _P])
    _check(None, f(_fptr(model, MLP_PARAMS), _fptr(X, 3 * n), n, _fptr(out, n)))


def ccsd_mlp_gradient(model, X, T):
    """(loss, gradient float32[MLP_TRAINABLE]) of the training loss over all rows."""
    n = T.shape[0]
    grad = np.zeros(MLP_TRAINABLE, dtype=np.float32)
    loss = ctypes.c_float()
    f = _mlp_fn("ccsd_mlp_gradient", [_P, _P, _P, ctypes.c_longlong, _P, ctypes.POINTER(ctypes.c_float)])
    _check(None, f(_fptr(model, MLP_PARAMS), _fptr(X, 3 * n), _fptr(T, n), n, _fptr(grad), ctypes.byref(loss)))
    return loss.value, grad


def ccsd_guess_features(h, X):
    """Fill X (float32, o*o*v*v*3 elements, [i][j][a][b][3]) with the handle's features."""
    f = _mlp_fn("ccsd_guess_features", [_P, _P])
    _check(h, f(h, _fptr(X)))


def ccsd_set_guess_model(h, model):
    f = _mlp_fn("ccsd_set_guess_model", [_P, _P])
    _check(h, f(h, None if model is None else _fptr(model, MLP_PARAMS)))


GUESS_AMPLITUDES, GUESS_MULTIPLIERS = 0, 1


def ccsd_set_multiplier_guess_model(h, model):
    """Learned start for the multiplier solves (None: the Jacobi start)."""
    f = _mlp_fn("ccsd_set_multiplier_guess_model", [_P, _P])
    _check(h, f(h, None if model is None else _fptr(model, MLP_PARAMS)))


def ccsd_guess_targets(h, which, X, T):
    """Fill X[n2][3] (float32) with a start's features and T[n2] with converged - start doubles."""
    f = _mlp_fn("ccsd_guess_targets", [_P, ctypes.c_int, _P, _P])
    _check(h, f(h, which, _fptr(X), _fptr(T)))


def ccsd_guess_doubles(h, which, model, x2):
    """x2[n2] (float64) = the start's doubles, corrected by `model` when given."""
    f = _mlp_fn("ccsd_guess_doubles", [_P, ctypes.c_int, _P, _P])
    _check(h, f(h, which, None if model is None else _fptr(model, MLP_PARAMS), _ptr(x2)))


def ccsd_solve_iterations(h):
    g, l, z = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(h, lib().ccsd_solve_iterations(h, ctypes.byref(g), ctypes.byref(l), ctypes.byref(z)))
    return {"ground": g.value, "lambda": l.value, "zeta": z.value}


# ---- batches of systems -----------------------------------------------------

def _batch_fn(name, argtypes, restype=ctypes.c_int):
    f = getattr(lib(), name)
    if not getattr(f, "argtypes", None):
        f.argtypes = argtypes
        f.restype = restype
    return f


def _bcheck(b, status):
    if status != OK:
        f = _batch_fn("ccsd_batch_last_error", [_P], ctypes.c_char_p)
        msg = f(b).decode() if b else lib().ccsd_strerror(status).decode()
        raise CCSDError(status, msg)


def ccsd_batch_create(handles, nvec=8):
    arr = (_P * len(handles))(*[h.value if isinstance(h, _P) else h for h in handles])
    out = _P()
    f = _batch_fn("ccsd_batch_create", [ctypes.c_int, ctypes.POINTER(_P), ctypes.c_int, ctypes.POINTER(_P)])
    _bcheck(None, f(len(handles), arr, nvec, ctypes.byref(out)))
    return out


def ccsd_batch_transform(b, side, xs, ys):
    """ys[s] = transform of xs[s] ([nvec][dim_s] float64 arrays, host or device) for every system."""
    n = len(xs)
    xa = (_P * n)(*[_ptr(x).value for x in xs])
    ya = (_P * n)(*[_ptr(y).value for y in ys])
    f = _batch_fn("ccsd_batch_transform", [_P, ctypes.c_int, ctypes.POINTER(_P), ctypes.POINTER(_P)])
    _bcheck(b, f(b, side, xa, ya))


def ccsd_batch_eom_solve(b, side, nroots, nsys):
    w = np.zeros(nsys * nroots)
    it = (ctypes.c_int * nsys)()
    f = _batch_fn("ccsd_batch_eom_solve", [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_int)])
    _bcheck(b, f(b, side, nroots, _ptr(w), it))
    return w.reshape(nsys, nroots), list(it)


def ccsd_batch_stats(b):
    la, ca, na = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    f = _batch_fn("ccsd_batch_stats", [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_longlong)])
    _bcheck(b, f(b, ctypes.byref(la), ctypes.byref(ca), ctypes.byref(na)))
    return {"launches": la.value, "captures": ca.value, "nodes": na.value}


def ccsd_batch_destroy(b):
    if b:
        _batch_fn("ccsd_batch_destroy", [_P], None)(b)


# ---- Hartree-Fock orbitals (relaxed mode) -------------------------------------

def ccsd_scf(eps, h, B, o, v, naux, tol=1e-12, rotated=True):
    """Nearest Hartree-Fock orbitals: (U[n,n], h'[n,n], B'[naux,n,n], iterations) as numpy arrays."""
    n = o + v
    U = np.zeros((n, n))
    hr = np.zeros((n, n)) if rotated else None
    Br = np.zeros((naux, n, n)) if rotated else None
    it = ctypes.c_int()
    f = _mlp_fn("ccsd_scf", [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _P, _P, _P,
                             ctypes.POINTER(ctypes.c_int)])
    _check(None, f(_ptr(eps), _ptr(h), _ptr(B), o, v, naux, tol, _ptr(U), _ptr(hr), _ptr(Br), ctypes.byref(it)))
    return U, hr, Br, it.value


def ccsd_rotate_integrals(U, h, B, o, v, naux):
    n = o + v
    hr, Br = np.zeros((n, n)), np.zeros((naux, n, n))
    f = _mlp_fn("ccsd_rotate_integrals", [_P, _P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P])
    _check(None, f(_ptr(U), _ptr(h), _ptr(B), o, v, naux, _ptr(hr), _ptr(Br)))
    return hr, Br


def ccsd_get_orbital_multipliers(h, k, l, o, v):
    kb = np.zeros((o, v))
    f = _mlp_fn("ccsd_get_orbital_multipliers", [_P, ctypes.c_int, ctypes.c_int, _P])
    _check(h, f(h, k, l, _ptr(kb)))
    return kb
