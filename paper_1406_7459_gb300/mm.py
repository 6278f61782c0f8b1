"""ctypes binding of libmm.so with the C ABI's names (include/mm.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Device arrays are torch CUDA tensors (float32, contiguous, 3*N
elements, SoA planes with x fastest); host arrays are numpy float32.  Each
call raises ``MMError`` on a nonzero status.  There is no CPU fallback: if
the library is missing, the first call raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libmm.so")

MM_OK = 0
MM_EINVAL = -1
MM_ENOMEM = -2
MM_ECUDA = -3
MM_ENONFINITE = -4
MM_ETIMEOUT = -5
MM_EUNSUPPORTED = -6
MM_ELIMIT = -7

MM_STEP_AUTO = 0
MM_STEP_GRAPH = 1
MM_STEP_PERSISTENT = 2
MM_TILED_GATHER = 1
MM_TILED_SCATTER = 2

MM_INTEGRATOR_EULER = 0
MM_INTEGRATOR_HEUN = 1
MM_INTEGRATOR_RK4 = 2

# every function declared in include/mm.h, with (restype, argtypes)
_c_int, _c_double, _vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
_PROTOS = {
    "mm_create": (_c_int, [ctypes.POINTER(_vp), ctypes.POINTER(_c_int), ctypes.POINTER(_c_double),
                           _c_double, _c_double, _c_double, _c_double, _c_double, _vp]),
    "mm_destroy": (_c_int, [_vp]),
    "mm_set_field": (_c_int, [_vp, ctypes.POINTER(_c_double)]),
    "mm_set_integrator": (_c_int, [_vp, _c_int]),
    "mm_set_m": (_c_int, [_vp, _vp]),
    "mm_get_m": (_c_int, [_vp, _vp]),
    "mm_demag_field": (_c_int, [_vp, _vp, _vp]),
    "mm_effective_field": (_c_int, [_vp, _vp, _vp]),
    "mm_step": (_c_int, [_vp, _c_int, _c_double]),
    "mm_step_host": (_c_int, [_vp, _vp, _c_int, _c_double, _vp]),
    "mm_set_step_path": (_c_int, [_vp, _c_int]),
    "mm_get_step_path": (_c_int, [_vp]),
    "mm_set_tiled_copies": (_c_int, [_vp, _c_int]),
    "mm_get_tiled_copies": (_c_int, [_vp]),
    "mm_set_wait_limit": (_c_int, [_vp, ctypes.c_longlong]),
    "mm_run_adaptive": (_c_int, [_vp, _c_double, ctypes.POINTER(_c_double), _c_double, _c_int,
                                 ctypes.POINTER(_c_double)]),
    "mm_energy": (_c_int, [_vp, ctypes.POINTER(_c_double)]),
    "mm_sync": (_c_int, [_vp]),
    "mm_last_error": (ctypes.c_char_p, [_vp]),
    "mm_plan_info": (_c_int, [_vp, ctypes.POINTER(_c_int)]),
    "mm_tensor_octant": (_c_int, [_vp, _vp]),
    "mm_kernel_spectrum": (_c_int, [_vp, _vp]),
    "mm_time_passes": (_c_int, [_vp, _c_int, _c_double, _vp, ctypes.c_ulonglong,
                                ctypes.POINTER(ctypes.c_float)]),
    "mm_demag_field_noalloc": (_c_int, [ctypes.POINTER(_c_int), _vp, ctypes.c_longlong, _vp, _vp, _vp]),
    "mm_batch_create": (_c_int, [ctypes.POINTER(_vp), _c_int, ctypes.POINTER(_c_int), ctypes.POINTER(_c_double),
                                 ctypes.POINTER(_c_double), ctypes.POINTER(_c_double),
                                 ctypes.POINTER(_c_double), ctypes.POINTER(_c_double),
                                 ctypes.POINTER(_c_double), _vp]),
    "mm_batch_destroy": (_c_int, [_vp]),
    "mm_batch_set_field": (_c_int, [_vp, ctypes.POINTER(_c_double)]),
    "mm_batch_set_m": (_c_int, [_vp, _vp]),
    "mm_batch_get_m": (_c_int, [_vp, _vp]),
    "mm_batch_step": (_c_int, [_vp, _c_int, _c_double]),
    "mm_batch_set_path": (_c_int, [_vp, _c_int]),
    "mm_batch_set_wait_limit": (_c_int, [_vp, ctypes.c_longlong]),
    "mm_batch_sync": (_c_int, [_vp]),
    "mm_batch_cells": (ctypes.c_longlong, [_vp]),
    "mm_batch_launch_form": (_c_int, [_vp]),
    "mm_batch_autotune": (_c_int, [_vp, _c_double, ctypes.POINTER(_c_int), ctypes.POINTER(ctypes.c_float)]),
    "mm_fno_create": (_c_int, [ctypes.POINTER(_vp), _c_int, _c_int, _c_int, _c_int, _c_int, _c_int,
                               ctypes.c_ulonglong, _vp]),
    "mm_fno_destroy": (_c_int, [_vp]),
    "mm_fno_param_count": (ctypes.c_longlong, [_vp]),
    "mm_fno_set_params": (_c_int, [_vp, _vp]),
    "mm_fno_get_params": (_c_int, [_vp, _vp]),
    "mm_fno_forward": (_c_int, [_vp, _c_int, _vp, _vp]),
    "mm_fno_grad": (_c_int, [_vp, _c_int, _vp, _vp, ctypes.POINTER(_c_double), _vp]),
    "mm_fno_train_step": (_c_int, [_vp, _c_int, _vp, _vp, ctypes.c_float, ctypes.POINTER(_c_double)]),
    "mm_step_surrogate": (_c_int, [_vp, _vp, _c_int, _c_double, _c_int, _c_double, ctypes.POINTER(_c_double)]),
    "mm_gemm_bf16": (_c_int, [_vp, _vp, _vp, _c_int, _c_int, _c_int] + [ctypes.c_longlong] * 6 +
                     [_c_int] + [ctypes.c_longlong] * 3 + [ctypes.c_float, ctypes.c_float, _c_int, _vp]),
}

_lib = None


class MMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libmm error %d: %s" % (code, msg))
        self.code = code


def lib():
    """Load libmm.so once; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libmm.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _PROTOS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def mm_last_error(ctx=None):
    return lib().mm_last_error(ctx).decode()


def _check(rc):
    if rc < 0:
        raise MMError(rc, mm_last_error())
    return rc


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(x, n=None, dtype=np.float32):
    """Raw pointer of a torch tensor (any device) or a numpy array."""
    if isinstance(x, np.ndarray):
        if x.dtype != dtype or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy array must be C-contiguous %s" % np.dtype(dtype))
        if n is not None and x.size != n:
            raise ValueError("expected %d elements, got %d" % (n, x.size))
        return x.ctypes.data
    import torch
    want = {np.float32: torch.float32, np.float64: torch.float64}[dtype]
    if x.dtype != want or not x.is_contiguous():
        raise ValueError("tensor must be contiguous %s" % want)
    if n is not None and x.numel() != n:
        raise ValueError("expected %d elements, got %d" % (n, x.numel()))
    return x.data_ptr()


class Context:
    """Owned handle of an mm_ctx plus its sizes."""

    def __init__(self, handle, grid):
        self.handle = handle
        self.grid = tuple(grid)
        self.N = grid[0] * grid[1] * grid[2]

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.mm_destroy(h)


def mm_create(grid, cell, Ms, A, Ku, alpha, gamma, stream=None):
    g = (ctypes.c_int * 3)(*[int(v) for v in grid])
    c = (ctypes.c_double * 3)(*[float(v) for v in cell])
    out = _vp()
    _check(lib().mm_create(ctypes.byref(out), g, c, Ms, A, Ku, alpha, gamma, _vp(_stream_handle(stream))))
    return Context(out, tuple(int(v) for v in grid))


def mm_destroy(ctx):
    h, ctx.handle = ctx.handle, None
    if h:
        _check(lib().mm_destroy(h))


def mm_set_integrator(ctx, method):
    if isinstance(method, str):
        method = {"euler": MM_INTEGRATOR_EULER, "heun": MM_INTEGRATOR_HEUN, "rk4": MM_INTEGRATOR_RK4}[method]
    _check(lib().mm_set_integrator(ctx.handle, int(method)))


def mm_set_field(ctx, H_ext):
    h = (ctypes.c_double * 3)(*[float(v) for v in H_ext])
    _check(lib().mm_set_field(ctx.handle, h))


def mm_set_m(ctx, M):
    _check(lib().mm_set_m(ctx.handle, _vp(_ptr(M, 3 * ctx.N))))


def mm_get_m(ctx, out):
    _check(lib().mm_get_m(ctx.handle, _vp(_ptr(out, 3 * ctx.N))))
    return out


def mm_demag_field(ctx, M, H):
    _check(lib().mm_demag_field(ctx.handle, _vp(_ptr(M, 3 * ctx.N)), _vp(_ptr(H, 3 * ctx.N))))
    return H


def mm_effective_field(ctx, M, H):
    _check(lib().mm_effective_field(ctx.handle, _vp(_ptr(M, 3 * ctx.N)), _vp(_ptr(H, 3 * ctx.N))))
    return H


def mm_step(ctx, n, dt):
    _check(lib().mm_step(ctx.handle, int(n), float(dt)))


def mm_step_host(ctx, M_in, n, dt, M_out):
    """n steps from the host array M_in (numpy float32 or a CPU torch tensor,
    3*N) into the host array M_out (may be M_in)."""
    N3 = 3 * ctx.N
    _check(lib().mm_step_host(ctx.handle, _vp(_ptr(M_in, N3)), int(n), float(dt), _vp(_ptr(M_out, N3))))
    return M_out


def mm_set_step_path(ctx, path):
    _check(lib().mm_set_step_path(ctx.handle, int(path)))


def mm_get_step_path(ctx):
    return _check(lib().mm_get_step_path(ctx.handle))


def mm_set_tiled_copies(ctx, mask):
    _check(lib().mm_set_tiled_copies(ctx.handle, int(mask)))


def mm_get_tiled_copies(ctx):
    return _check(lib().mm_get_tiled_copies(ctx.handle))


def mm_set_wait_limit(ctx, polls):
    _check(lib().mm_set_wait_limit(ctx.handle, int(polls)))


def mm_run_adaptive(ctx, t_span, dt, tol, max_steps=100000):
    """Adaptive Dormand-Prince run over t_span seconds.  Returns (complete,
    dt_next, stats) with stats = dict(accepted, rejected, evaluations, t);
    complete is False when max_steps ran out first (MM_ELIMIT)."""
    d = ctypes.c_double(float(dt))
    st = (ctypes.c_double * 4)()
    rc = lib().mm_run_adaptive(ctx.handle, float(t_span), ctypes.byref(d), float(tol), int(max_steps), st)
    if rc != MM_ELIMIT:
        _check(rc)
    stats = dict(accepted=int(st[0]), rejected=int(st[1]), evaluations=int(st[2]), t=float(st[3]))
    return rc == MM_OK, d.value, stats


def mm_energy(ctx):
    E = (ctypes.c_double * 5)()
    _check(lib().mm_energy(ctx.handle, E))
    return np.array(list(E))


def mm_sync(ctx):
    _check(lib().mm_sync(ctx.handle))


def mm_plan_info(ctx):
    L = (ctypes.c_int * 3)()
    launches = _check(lib().mm_plan_info(ctx.handle, L))
    return tuple(L), launches


def mm_tensor_octant(ctx):
    nx, ny, nz = ctx.grid
    out = np.zeros((6, nz, ny, nx), np.float64)
    _check(lib().mm_tensor_octant(ctx.handle, _vp(_ptr(out, None, np.float64))))
    return out


def mm_kernel_spectrum(ctx, out=None):
    """Copy of the stored tensor spectrum; into `out` (torch or numpy,
    float32, (Lx/2+1)*(Lz/2+1)*(Ly/2+1)*6 elements) when given."""
    (Lx, Ly, Lz), _ = mm_plan_info(ctx)
    n = (Lx // 2 + 1) * (Lz // 2 + 1) * (Ly // 2 + 1) * 6
    if out is None:
        out = np.zeros((Lx // 2 + 1, Lz // 2 + 1, Ly // 2 + 1, 6), np.float32)
    _check(lib().mm_kernel_spectrum(ctx.handle, _vp(_ptr(out, n))))
    return out


def mm_time_passes(ctx, reps, dt, flush=None):
    """Mean per-pass durations (ms) over `reps` steps; `flush` is an optional
    torch CUDA tensor overwritten before each step."""
    ms = (ctypes.c_float * 3)()
    fptr = flush.data_ptr() if flush is not None else None
    fbytes = flush.numel() * flush.element_size() if flush is not None else 0
    _check(lib().mm_time_passes(ctx.handle, int(reps), float(dt), _vp(fptr), fbytes, ms))
    return tuple(ms)


def mm_demag_field_noalloc(grid, Kt, M, H, stream=None):
    """Demag field without any device allocation (see include/mm.h): Kt is
    the device copy of mm_kernel_spectrum for the same grid and cell."""
    g = (ctypes.c_int * 3)(*[int(v) for v in grid])
    n = 3 * int(grid[0]) * int(grid[1]) * int(grid[2])
    kt_elems = int(Kt.numel() if hasattr(Kt, "numel") else Kt.size)
    _check(lib().mm_demag_field_noalloc(g, _vp(_ptr(Kt)), kt_elems, _vp(_ptr(M, n)), _vp(_ptr(H, n)),
                                        _vp(_stream_handle(stream))))
    return H


class Batch:
    """Owned handle of an mm_batch."""

    def __init__(self, handle, grids):
        self.handle = handle
        self.grids = [tuple(g) for g in grids]
        self.sizes = [3 * g[0] * g[1] * g[2] for g in self.grids]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.total = int(self.offsets[-1])

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.mm_batch_destroy(h)


def _darr(v):
    v = [float(x) for x in v]
    return (ctypes.c_double * len(v))(*v)


def mm_batch_create(grids, cells, Ms, A, Ku, alpha, gamma, stream=None):
    n = len(grids)
    g = (ctypes.c_int * (3 * n))(*[int(v) for gr in grids for v in gr])
    c = _darr([v for ce in cells for v in ce])
    out = _vp()
    _check(lib().mm_batch_create(ctypes.byref(out), n, g, c, _darr(Ms), _darr(A), _darr(Ku), _darr(alpha),
                                 _darr(gamma), _vp(_stream_handle(stream))))
    return Batch(out, grids)


def mm_batch_destroy(b):
    h, b.handle = b.handle, None
    if h:
        _check(lib().mm_batch_destroy(h))


def mm_batch_set_field(b, H):
    _check(lib().mm_batch_set_field(b.handle, _darr([v for h in H for v in h])))


def mm_batch_set_m(b, M):
    _check(lib().mm_batch_set_m(b.handle, _vp(_ptr(M, b.total))))


def mm_batch_get_m(b, out):
    _check(lib().mm_batch_get_m(b.handle, _vp(_ptr(out, b.total))))
    return out


def mm_batch_step(b, n, dt):
    _check(lib().mm_batch_step(b.handle, int(n), float(dt)))


def mm_batch_sync(b):
    _check(lib().mm_batch_sync(b.handle))


def mm_batch_set_path(b, path):
    _check(lib().mm_batch_set_path(b.handle, int(path)))


def mm_batch_set_wait_limit(b, polls):
    _check(lib().mm_batch_set_wait_limit(b.handle, int(polls)))


def mm_batch_cells(b):
    return int(lib().mm_batch_cells(b.handle))


def mm_batch_launch_form(b):
    """0: graph step; 1: persistent launch replayed from a graph; 2: persistent
    launch issued directly; -1 before any step."""
    return int(lib().mm_batch_launch_form(b.handle))


def mm_batch_autotune(b, dt):
    choice = (ctypes.c_int * 4)()
    ms = (ctypes.c_float * 16)()
    _check(lib().mm_batch_autotune(b.handle, float(dt), choice, ms))
    return tuple(choice), list(ms)


class Fno:
    """Owned handle of an mm_fno."""

    def __init__(self, handle, H, W, width, modes, layers):
        self.handle = handle
        self.H, self.W, self.width, self.modes, self.layers = H, W, width, modes, layers

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.mm_fno_destroy(h)


def mm_fno_create(H, W, width=32, modes=16, layers=4, max_batch=8, seed=0, stream=None):
    out = _vp()
    _check(lib().mm_fno_create(ctypes.byref(out), H, W, width, modes, layers, max_batch, seed,
                               _vp(_stream_handle(stream))))
    return Fno(out, H, W, width, modes, layers)


def mm_fno_destroy(f):
    h, f.handle = f.handle, None
    if h:
        _check(lib().mm_fno_destroy(h))


def mm_fno_param_count(f):
    return int(lib().mm_fno_param_count(f.handle))


def mm_fno_set_params(f, p):
    _check(lib().mm_fno_set_params(f.handle, _vp(_ptr(p, mm_fno_param_count(f)))))


def mm_fno_get_params(f, out=None):
    if out is None:
        out = np.zeros(mm_fno_param_count(f), np.float32)
    _check(lib().mm_fno_get_params(f.handle, _vp(_ptr(out, mm_fno_param_count(f)))))
    return out


def mm_fno_forward(f, x, y):
    b = x.numel() // (3 * f.H * f.W)
    _check(lib().mm_fno_forward(f.handle, b, _vp(_ptr(x)), _vp(_ptr(y))))
    return y


def mm_fno_grad(f, x, t, grad=None):
    b = x.numel() // (3 * f.H * f.W)
    loss = _c_double()
    _check(lib().mm_fno_grad(f.handle, b, _vp(_ptr(x)), _vp(_ptr(t)), ctypes.byref(loss),
                             _vp(_ptr(grad) if grad is not None else None)))
    return loss.value


def mm_fno_train_step(f, x, t, lr):
    b = x.numel() // (3 * f.H * f.W)
    loss = _c_double()
    _check(lib().mm_fno_train_step(f.handle, b, _vp(_ptr(x)), _vp(_ptr(t)), float(lr), ctypes.byref(loss)))
    return loss.value


def mm_step_surrogate(ctx, f, n, dt, refresh=8, tol=1e-3):
    st = (ctypes.c_double * 4)()
    _check(lib().mm_step_surrogate(ctx.handle, f.handle, int(n), float(dt), int(refresh), float(tol), st))
    return {"surrogate_steps": int(st[0]), "exact_steps": int(st[1]), "max_residual": st[2],
            "fell_back": bool(st[3])}


def fno_param_dict(flat, width, modes, layers):
    """Split the flat parameter vector into named arrays (the layout of
    include/mm.h), as float64 for comparisons."""
    C, m, L = width, modes, layers
    flat = np.asarray(flat, np.float64)
    shapes = [("P", (C, 5)), ("p", (C,)), ("R_re", (L, C, C, 2 * m, m)), ("R_im", (L, C, C, 2 * m, m)),
              ("W", (L, C, C)), ("b", (L, C)), ("Q", (3, C)), ("q", (3,))]
    out, o = {}, 0
    for name, shp in shapes:
        n = int(np.prod(shp))
        out[name] = flat[o:o + n].reshape(shp)
        o += n
    return out


def mm_gemm_bf16(A, B, C, M, N, K, strides, batch=1, batch_strides=(0, 0, 0), alpha=1.0, beta=0.0, atomic=False,
                 stream=None):
    """C[z] = alpha A[z] B[z] + beta C[z] (or C[z] += alpha A[z] B[z] with
    atomic) on the tensor cores.  A, B: bfloat16 CUDA tensors, C: float32
    CUDA tensor; strides = (sam, sak, sbk, sbn, scm, scn) and batch_strides =
    (zA, zB, zC) in elements.  Synchronises the stream."""
    import torch
    for t, want in ((A, torch.bfloat16), (B, torch.bfloat16), (C, torch.float32)):
        if t.dtype != want or not t.is_cuda:
            raise ValueError("A, B must be bfloat16 and C float32 CUDA tensors")
    sam, sak, sbk, sbn, scm, scn = (int(v) for v in strides)
    zA, zB, zC = (int(v) for v in batch_strides)
    _check(lib().mm_gemm_bf16(_vp(A.data_ptr()), _vp(B.data_ptr()), _vp(C.data_ptr()), int(M), int(N), int(K),
                              sam, sak, sbk, sbn, scm, scn, int(batch), zA, zB, zC, float(alpha), float(beta),
                              1 if atomic else 0, _vp(_stream_handle(stream))))
    return C
