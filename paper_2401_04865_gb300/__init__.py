"""Python binding of the GB300 immersed-boundary PME library (``libibpme.so``).

Argument marshalling only: every function here forwards to the C entry point
of the same name declared in ``include/ibpme.h``; all arithmetic runs in the
library's CUDA kernels.  Arrays may be torch tensors (CUDA or CPU) or numpy
arrays; they must be C-contiguous with the dtype the header states (float64,
int32 for body offsets).  There is no CPU fallback: if the library is missing
the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libibpme.so")

IBPME_OK = 0
IBPME_ERR_ARG = 1
IBPME_ERR_CUDA = 2
IBPME_ERR_CUFFT = 3
IBPME_ERR_OOM = 4
IBPME_ERR_NOT_CONVERGED = 5
IBPME_ERR_UNEQUAL_RADII = 6
IBPME_ERR_TIMEOUT = 7
IBPME_ERR_NONFINITE = 8
IBPME_FP64 = 0
IBPME_MIXED = 1
IBPME_GUESS_ZERO = 0
IBPME_GUESS_USER = 1
IBPME_GUESS_LEARNED = 2
IBPME_GUESS_LEARNED_STEP = 3
IBPME_PRECOND_BODY = 0
IBPME_PRECOND_NONE = 1

_d, _i, _p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p


class ibpme_params(ctypes.Structure):
    _fields_ = [("box", _d * 3), ("mesh", _i * 3), ("xi", _d), ("eta", _d), ("r_cut", _d), ("P", _i),
                ("tol", _d), ("bead_radius", _d), ("eps_f", _d), ("precision", _i), ("max_rhs", _i),
                ("n_radius_classes", _i), ("class_radius", _d * 4)]


class ibpme_bodies(ctypes.Structure):
    _fields_ = [("n_bodies", _i), ("body_offsets", _p), ("X", _p), ("Q", _p)]


class ibpme_solve_opts(ctypes.Structure):
    _fields_ = [("rtol", _d), ("restart", _i), ("max_iter", _i), ("guess", _i), ("mlp", _p), ("precision", _i),
                ("precond", _i)]


class ibpme_solve_stats(ctypes.Structure):
    _fields_ = [("iters", _i), ("outer", _i), ("matvecs_fp64", _i), ("rel_residual", _d), ("time_ms", _d),
                ("fell_back", _i), ("init_rel_residual", _d)]


class ibpme_bd_params(ctypes.Structure):
    _fields_ = [("dt", _d), ("gamma", _d), ("kT", _d), ("seed", ctypes.c_ulonglong), ("step", ctypes.c_longlong)]


class IbpmeError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where} failed with status {status}: {msg}")
        self.status = status


_lib = None

# entry points of include/ibpme.h: name -> (restype, argtypes)
SIGNATURES = {
    "pme_setup": (_i, [ctypes.POINTER(_p), ctypes.POINTER(ibpme_params), _p]),
    "pme_destroy": (_i, [_p]),
    "ibpme_set_stream": (_i, [_p, _p]),
    "ibpme_get_params": (_i, [_p, ctypes.POINTER(ibpme_params)]),
    "ibpme_last_error": (ctypes.c_char_p, []),
    "ibpme_set_radius_classes": (_i, [_p, _i, _p]),
    "ibpme_rpy_mobility": (_i, [_p, _i, _p, _p, _d, _p]),
    "ibpme_rigid_mobility": (_i, [_p, _i, _p, ctypes.POINTER(ibpme_bodies), _p, _d,
                                  ctypes.POINTER(ibpme_solve_opts), _p, _p, ctypes.POINTER(ibpme_solve_stats)]),
    "pme_spread": (_i, [_p, _i, _p, _p, _i, _p]),
    "pme_field": (_i, [_p, _i, _p, _p, _i, _p, _p]),
    "induced_charge_solve": (_i, [_p, _i, _p, ctypes.POINTER(ibpme_bodies), _p, _i,
                                  ctypes.POINTER(ibpme_solve_opts), _p, _p, _p,
                                  ctypes.POINTER(ibpme_solve_stats)]),
    "induced_charge_solve_batch": (_i, [_p, _i, _p, ctypes.POINTER(ibpme_bodies), _i, _p, _p, _i,
                                        ctypes.POINTER(ibpme_solve_opts), _p, _p, _p, _p]),
    "body_force_torque": (_i, [_p, _i, _p, _p, ctypes.POINTER(ibpme_bodies), _p, _p, _p, _p, _p]),
    "ibpme_bd_step": (_i, [_p, _i, _p, ctypes.POINTER(ibpme_bodies), _p, ctypes.POINTER(ibpme_bd_params),
                           _p, _p]),
    "ibpme_bd_advance": (_i, [_p, _i, _p, ctypes.POINTER(ibpme_bodies), _p, ctypes.POINTER(ibpme_solve_opts),
                              ctypes.POINTER(ibpme_bd_params), _p, _p, _p, _p, _p, _p, _p, _p,
                              ctypes.POINTER(ibpme_solve_stats)]),
    "pme_spread_noalloc": (_i, [ctypes.POINTER(ibpme_params), _i, _p, _p, _i, _p, _p]),
    "ibpme_capacitance": (_i, [_p, _i, _p, ctypes.POINTER(ibpme_bodies), ctypes.POINTER(ibpme_solve_opts), _p,
                               ctypes.POINTER(ibpme_solve_stats)]),
    "ibpme_mlp_create": (_i, [ctypes.POINTER(_p), ctypes.c_ulonglong]),
    "ibpme_mlp_destroy": (_i, [_p]),
    "ibpme_mlp_get": (_i, [_p, _p]),
    "ibpme_mlp_set": (_i, [_p, _p]),
    "ibpme_mlp_forward": (_i, [_p, _i, _p, _p, _p]),
    "ibpme_mlp_forward_tc": (_i, [_p, _i, _p, _p, _p]),
    "ibpme_mlp_gradient": (_i, [_p, _i, _p, _p, _p, _p, _p]),
    "ibpme_mlp_train": (_i, [_p, _i, _p, _p, _i, _i, ctypes.c_float, ctypes.c_ulonglong, _p, _p]),
    "ibpme_features": (_i, [_p, _i, _p, ctypes.POINTER(ibpme_bodies), _p, _i, _p, _p, _p]),
    "ibpme_kernel_launches": (ctypes.c_longlong, []),
    "ibpme_profile": (_i, [ctypes.c_uint]),
    "ibpme_profile_read": (_i, [_i, _p, _p]),
    "ibpme_stage_name": (ctypes.c_char_p, [_i]),
}

STAGES = ["near_build", "near_apply", "spread", "fft_forward", "scale", "fft_inverse", "gather", "krylov",
          "bodies", "spread64", "fft_forward64", "scale64", "fft_inverse64", "gather64", "near_apply32",
          "near_field", "rpy_near"]


def load(path: str | None = None):
    """Load libibpme.so (built in-tree by ``__graft_entry__.build()``); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"the CUDA library {path} is not built; run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    return load().ibpme_last_error().decode(errors="replace")


def _check(status: int, where: str, ok=(IBPME_OK,)):
    if status not in ok:
        raise IbpmeError(status, where, last_error())
    return status


def ptr(a, dtype=np.float64):
    """Raw address of a contiguous torch tensor / numpy array (None -> NULL)."""
    if a is None:
        return None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            want = {np.float64: torch.float64, np.float32: torch.float32, np.int32: torch.int32}[dtype]
            if a.dtype != want:
                raise TypeError(f"expected {want}, got {a.dtype}")
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            return a.data_ptr()
    except ImportError:
        pass
    if isinstance(a, np.ndarray):
        if a.dtype != np.dtype(dtype):
            raise TypeError(f"expected {np.dtype(dtype)}, got {a.dtype}")
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if isinstance(a, int):
        return a
    raise TypeError(f"unsupported array type {type(a)}")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


IBPME_MAX_RADIUS_CLASSES = 4


def make_params(box, mesh=(0, 0, 0), tol=1e-6, bead_radius=0.1, eps_f=1.0, precision=IBPME_FP64, max_rhs=3,
                xi=0.0, eta=0.0, r_cut=0.0, P=0, class_radius=()) -> ibpme_params:
    p = ibpme_params()
    for d in range(3):
        p.box[d] = float(box[d])
        p.mesh[d] = int(mesh[d])
    p.xi, p.eta, p.r_cut, p.P = float(xi), float(eta), float(r_cut), int(P)
    p.tol, p.bead_radius, p.eps_f = float(tol), float(bead_radius), float(eps_f)
    p.precision, p.max_rhs = int(precision), int(max_rhs)
    if len(class_radius) > IBPME_MAX_RADIUS_CLASSES:
        raise ValueError("at most %d radius classes" % IBPME_MAX_RADIUS_CLASSES)
    p.n_radius_classes = len(class_radius)
    for i, r in enumerate(class_radius):
        p.class_radius[i] = float(r)
    return p


class Bodies:
    """ibpme_bodies plus references to the arrays it points to."""

    def __init__(self, body_offsets, X, Q):
        self.arrays = (body_offsets, X, Q)
        self.c = ibpme_bodies(int(len(body_offsets) - 1), ptr(body_offsets, np.int32), ptr(X), ptr(Q))


def pme_setup(params: ibpme_params, stream=None):
    lib = load()
    ctx = _p()
    _check(lib.pme_setup(ctypes.byref(ctx), ctypes.byref(params), _stream_handle(stream)), "pme_setup")
    return ctx


def pme_destroy(ctx):
    return _check(load().pme_destroy(ctx), "pme_destroy")


def ibpme_set_stream(ctx, stream):
    return _check(load().ibpme_set_stream(ctx, _stream_handle(stream)), "ibpme_set_stream")


def ibpme_set_radius_classes(ctx, n, cls):
    """Bind the radius class of each of n beads (host int array; None or n = 0 unbinds)."""
    arr = None if cls is None else np.ascontiguousarray(np.asarray(cls).reshape(-1), dtype=np.int32)
    if arr is not None and arr.shape[0] != int(n):
        raise ValueError("one class per bead expected")
    return _check(load().ibpme_set_radius_classes(ctx, int(n), ptr(arr, np.int32)), "ibpme_set_radius_classes")


def ibpme_rpy_mobility(ctx, n, x, F, mu, U):
    """U [n][3] = periodic RPY mobility (viscosity mu) times the forces F [n][3] at x [n][3]."""
    return _check(load().ibpme_rpy_mobility(ctx, int(n), ptr(x), ptr(F), float(mu), ptr(U)), "ibpme_rpy_mobility")


def ibpme_rigid_mobility(ctx, n, x, bodies: Bodies, FL, mu, opts: ibpme_solve_opts | None, W, f_out=None):
    """Rigid-body mobility problem: FL [n_bodies][6] (F, L) -> W [n_bodies][6] (U, Omega) and the bead
    constraint forces f_out [n][3].  Returns (status, stats); raises on any status other than OK /
    NOT_CONVERGED."""
    st = ibpme_solve_stats()
    status = load().ibpme_rigid_mobility(ctx, int(n), ptr(x), ctypes.byref(bodies.c), ptr(FL), float(mu),
                                         ctypes.byref(opts) if opts is not None else None, ptr(W), ptr(f_out),
                                         ctypes.byref(st))
    if status not in (IBPME_OK, IBPME_ERR_NOT_CONVERGED):
        _check(status, "ibpme_rigid_mobility")
    return status, st


def ibpme_get_params(ctx) -> ibpme_params:
    out = ibpme_params()
    _check(load().ibpme_get_params(ctx, ctypes.byref(out)), "ibpme_get_params")
    return out


def pme_spread(ctx, n, x, q, nrhs, grid_out=None):
    gdt = np.float32 if (grid_out is not None and getattr(grid_out, "dtype", None) in (np.float32, _torch_f32())) \
        else np.float64
    return _check(load().pme_spread(ctx, int(n), ptr(x), ptr(q), int(nrhs), ptr(grid_out, gdt)), "pme_spread")


IBPME_NOALLOC_MAX_BEADS = 262144
IBPME_MLP_IN = 12
IBPME_MLP_HIDDEN = 64
IBPME_MLP_NPARAM = 64 * IBPME_MLP_IN + 64 + 64 * 64 + 64 + 64 + 1


def ibpme_mlp_create(seed=0):
    m = _p()
    _check(load().ibpme_mlp_create(ctypes.byref(m), int(seed)), "ibpme_mlp_create")
    return m


def ibpme_mlp_destroy(m):
    return _check(load().ibpme_mlp_destroy(m), "ibpme_mlp_destroy")


def ibpme_mlp_get(m, params):
    return _check(load().ibpme_mlp_get(m, ptr(params, np.float32)), "ibpme_mlp_get")


def ibpme_mlp_set(m, params):
    return _check(load().ibpme_mlp_set(m, ptr(params, np.float32)), "ibpme_mlp_set")


def ibpme_mlp_forward(m, n, feat, y, stream=None):
    return _check(load().ibpme_mlp_forward(m, int(n), ptr(feat, np.float32), ptr(y, np.float32),
                                           _stream_handle(stream)), "ibpme_mlp_forward")


def ibpme_mlp_forward_tc(m, n, feat, y, stream=None):
    """Tensor-core inference (BF16 hidden layer, FP32 accumulation)."""
    return _check(load().ibpme_mlp_forward_tc(m, int(n), ptr(feat, np.float32), ptr(y, np.float32),
                                              _stream_handle(stream)), "ibpme_mlp_forward_tc")


def ibpme_mlp_gradient(m, n, feat, target, grad, loss=None, stream=None):
    return _check(load().ibpme_mlp_gradient(m, int(n), ptr(feat, np.float32), ptr(target, np.float32),
                                            ptr(grad, np.float32), ptr(loss, np.float32), _stream_handle(stream)),
                  "ibpme_mlp_gradient")


def ibpme_mlp_train(m, n, feat, target, batch=4096, epochs=1, lr=1e-3, seed=0, stream=None):
    loss = np.zeros(1, dtype=np.float32)
    _check(load().ibpme_mlp_train(m, int(n), ptr(feat, np.float32), ptr(target, np.float32), int(batch),
                                  int(epochs), float(lr), int(seed), ptr(loss, np.float32), _stream_handle(stream)),
           "ibpme_mlp_train")
    return float(loss[0])


def ibpme_features(ctx, n, x, bodies: "Bodies", E0, nrhs, feat, q=None, target=None):
    return _check(load().ibpme_features(ctx, int(n), ptr(x), ctypes.byref(bodies.c), ptr(E0), int(nrhs),
                                        ptr(feat, np.float32), ptr(q), ptr(target, np.float32)), "ibpme_features")


def pme_spread_noalloc(params: ibpme_params, n, x, q, nrhs, grid_out, stream=None):
    """Spreading with no context and no device allocation (device arrays only)."""
    gdt = np.float32 if getattr(grid_out, "dtype", None) in (np.float32, _torch_f32()) else np.float64
    return _check(load().pme_spread_noalloc(ctypes.byref(params), int(n), ptr(x), ptr(q), int(nrhs),
                                            ptr(grid_out, gdt), _stream_handle(stream)), "pme_spread_noalloc")


def _torch_f32():
    try:
        import torch
        return torch.float32
    except ImportError:
        return None


def pme_field(ctx, n, x, q, nrhs, psi, E=None):
    return _check(load().pme_field(ctx, int(n), ptr(x), ptr(q), int(nrhs), ptr(psi), ptr(E)), "pme_field")


def make_opts(rtol=1e-6, restart=50, max_iter=3000, guess=IBPME_GUESS_ZERO, precision=-1, mlp=None,
              precond=IBPME_PRECOND_BODY) -> ibpme_solve_opts:
    handle = mlp.value if isinstance(mlp, ctypes.c_void_p) else mlp
    return ibpme_solve_opts(float(rtol), int(restart), int(max_iter), int(guess), handle, int(precision),
                            int(precond))


def induced_charge_solve(ctx, n, x, bodies: Bodies, E0, nrhs, opts: ibpme_solve_opts | None, q_out, psi_out=None,
                         S_out=None):
    """Returns (status, stats); raises on any status other than OK / NOT_CONVERGED."""
    st = ibpme_solve_stats()
    status = load().induced_charge_solve(ctx, int(n), ptr(x), ctypes.byref(bodies.c), ptr(E0), int(nrhs),
                                         ctypes.byref(opts) if opts is not None else None, ptr(q_out), ptr(psi_out),
                                         ptr(S_out), ctypes.byref(st))
    _check(status, "induced_charge_solve", ok=(IBPME_OK, IBPME_ERR_NOT_CONVERGED))
    return status, st


def induced_charge_solve_batch(ctx, n, x, bodies: Bodies, cfg_bodies, E0, nrhs, opts: ibpme_solve_opts | None,
                               q_out, psi_out=None, S_out=None):
    """Independent configurations (bodies cfg_bodies[k]..cfg_bodies[k+1]-1) in one call.
    Returns (status, [stats per configuration]); raises like induced_charge_solve."""
    cb = np.ascontiguousarray(np.asarray(cfg_bodies, dtype=np.int32))
    ncfg = int(cb.size) - 1
    st = (ibpme_solve_stats * max(ncfg, 1))()
    status = load().induced_charge_solve_batch(ctx, int(n), ptr(x), ctypes.byref(bodies.c), ncfg, cb.ctypes.data,
                                               ptr(E0), int(nrhs), ctypes.byref(opts) if opts is not None else None,
                                               ptr(q_out), ptr(psi_out), ptr(S_out), st)
    _check(status, "induced_charge_solve_batch", ok=(IBPME_OK, IBPME_ERR_NOT_CONVERGED))
    return status, list(st)[:ncfg]


def body_force_torque(ctx, n, x, q, bodies: Bodies, E0, f_bead, F, L, U=None):
    return _check(load().body_force_torque(ctx, int(n), ptr(x), ptr(q), ctypes.byref(bodies.c), ptr(E0),
                                           ptr(f_bead), ptr(F), ptr(L), ptr(U)), "body_force_torque")


def ibpme_bd_step(ctx, n, x, bodies: Bodies, f_bead, dt, gamma=1.0, kT=1.0, seed=0, step=0, x_out=None,
                  X_out=None):
    bd = ibpme_bd_params(float(dt), float(gamma), float(kT), int(seed), int(step))
    return _check(load().ibpme_bd_step(ctx, int(n), ptr(x), ctypes.byref(bodies.c), ptr(f_bead),
                                       ctypes.byref(bd), ptr(x_out), ptr(X_out)), "ibpme_bd_step")


def ibpme_bd_advance(ctx, n, x, bodies: Bodies, E0, opts: ibpme_solve_opts | None, q_io, dt, gamma=1.0, kT=1.0,
                     seed=0, step=0, F=None, L=None, x_out=None, X_out=None, psi_out=None, f_bead=None, U=None):
    """Solve, forces and one BD step in one call.  Returns (status, stats); raises on
    any status other than OK / NOT_CONVERGED."""
    bd = ibpme_bd_params(float(dt), float(gamma), float(kT), int(seed), int(step))
    st = ibpme_solve_stats()
    status = load().ibpme_bd_advance(ctx, int(n), ptr(x), ctypes.byref(bodies.c), ptr(E0),
                                     ctypes.byref(opts) if opts is not None else None, ctypes.byref(bd), ptr(q_io),
                                     ptr(psi_out), ptr(f_bead), ptr(F), ptr(L), ptr(U), ptr(x_out), ptr(X_out),
                                     ctypes.byref(st))
    _check(status, "ibpme_bd_advance", ok=(IBPME_OK, IBPME_ERR_NOT_CONVERGED))
    return status, st


def ibpme_capacitance(ctx, n, x, bodies: Bodies, C_out, opts: ibpme_solve_opts | None = None):
    """Grand capacitance tensor C [4 N_b][4 N_b] into C_out.  Returns (status, stats);
    raises on any status other than OK / NOT_CONVERGED."""
    st = ibpme_solve_stats()
    status = load().ibpme_capacitance(ctx, int(n), ptr(x), ctypes.byref(bodies.c),
                                      ctypes.byref(opts) if opts is not None else None, ptr(C_out),
                                      ctypes.byref(st))
    _check(status, "ibpme_capacitance", ok=(IBPME_OK, IBPME_ERR_NOT_CONVERGED))
    return status, st


def ibpme_kernel_launches() -> int:
    return int(load().ibpme_kernel_launches())


def ibpme_profile(stage_mask: int):
    return _check(load().ibpme_profile(int(stage_mask)), "ibpme_profile")


def ibpme_profile_read():
    """{stage name: (total ms, timed launches)} for every stage."""
    ms = np.zeros(len(STAGES))
    cnt = np.zeros(len(STAGES), dtype=np.int64)
    _check(load().ibpme_profile_read(len(STAGES), ms.ctypes.data, cnt.ctypes.data), "ibpme_profile_read")
    return {STAGES[i]: (float(ms[i]), int(cnt[i])) for i in range(len(STAGES))}


def ibpme_stage_name(stage: int) -> str:
    return load().ibpme_stage_name(int(stage)).decode()
