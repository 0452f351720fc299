"""Thin ctypes binding of libapfc (the C ABI declared in include/apfc.h).

Argument marshalling only: every step of the time integration runs in the
CUDA library.  The binding refuses to run when the library is missing; there
is no CPU fallback.

Buffers may be numpy arrays (host memory, ``APFC_HOST``) or torch CUDA
tensors (device memory, ``APFC_DEVICE``), complex128 and C-contiguous.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libapfc.so")

APFC_OK, APFC_EINVAL, APFC_ENOMEM, APFC_ECUDA, APFC_ENOCONV, APFC_ENAN, APFC_ESTATE, APFC_ETOOBIG = range(8)
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "ENAN", 6: "ESTATE", 7: "ETOOBIG"}
APFC_STATIC_MAX_DOF = 262144
APFC_HOST, APFC_DEVICE = 0, 1
APFC_C128, APFC_C64 = 0, 1
APFC_LATTICE_CUSTOM, APFC_LATTICE_HEX2D, APFC_LATTICE_BCC3D = 0, 1, 2
APFC_FP64, APFC_FP32_REFINED = 0, 1
APFC_BICGSTAB = 0
APFC_TAU_FOLD, APFC_TAU_PLAIN = 0, 1
APFC_MAX_J = 8
APFC_BATCH_GRAPH = 1
APFC_ALU_FMA64, APFC_ALU_FMA32, APFC_ALU_CVT64 = 0, 1, 2
APFC_GUESS_PREV, APFC_GUESS_EXTRAP = 0, 1


class ApfcError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"apfc status {STATUS_NAMES.get(status, status)}: {msg}")


class Lattice(C.Structure):
    _fields_ = [("lattice", C.c_int), ("dim", C.c_int), ("J", C.c_int), ("k", (C.c_double * 3) * APFC_MAX_J)]


class Params(C.Structure):
    _fields_ = [("dB", C.c_double), ("Bx", C.c_double), ("t", C.c_double), ("v", C.c_double)]


class Grid(C.Structure):
    _fields_ = [("n", C.c_int * 3), ("h", C.c_double * 3)]


class Opts(C.Structure):
    _fields_ = [
        ("precision", C.c_int),
        ("krylov", C.c_int),
        ("max_iter", C.c_int),
        ("cheb_degree", C.c_int),
        ("tau_mode", C.c_int),
        ("max_refine", C.c_int),
        ("check_every", C.c_int),
        ("fused", C.c_int),
        ("tol", C.c_double),
        ("tol_inner", C.c_double),
        ("tile", C.c_int),
        ("tile_rows", C.c_int),
        ("picard_iters", C.c_int),
        ("jacobian", C.c_int),
        ("tile_t", C.c_int),
        ("guess", C.c_int),
    ]


class Adapt(C.Structure):
    _fields_ = [("n", C.c_double), ("h_int", C.c_double), ("h_max", C.c_double), ("eps", C.c_double),
                ("A_min", C.c_double)]


class Stats(C.Structure):
    _fields_ = [
        ("steps", C.c_longlong),
        ("iters_total", C.c_longlong),
        ("iters_last", C.c_int),
        ("refine_last", C.c_int),
        ("resid_last", C.c_double),
    ]


EXPORTS = {
    "apfc_default_opts": (C.c_int, [C.POINTER(Opts)]),
    "apfc_uniform_amplitude": (C.c_int, [C.POINTER(Lattice), C.POINTER(Params), C.POINTER(C.c_double)]),
    "apfc_init": (
        C.c_int,
        [C.POINTER(C.c_void_p), C.POINTER(Lattice), C.POINTER(Params), C.POINTER(Grid), C.POINTER(Opts), C.c_void_p],
    ),
    "apfc_set_opts": (C.c_int, [C.c_void_p, C.POINTER(Opts)]),
    "apfc_set_amplitudes": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "apfc_get_amplitudes": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "apfc_get_zeta": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "apfc_step": (C.c_int, [C.c_void_p, C.c_double, C.c_int]),
    "apfc_autotune": (
        C.c_int, [C.c_void_p, C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)]
    ),
    "apfc_energy": (C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    "apfc_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    "apfc_last_error": (C.c_char_p, [C.c_void_p]),
    "apfc_destroy": (None, [C.c_void_p]),
    "apfc_apply_operator": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_int]),
    "apfc_apply_preconditioner": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_int]),
    "apfc_nonlinear_rhs": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_int]),
    "apfc_kernel_count": (C.c_int, []),
    "apfc_kernel_name": (C.c_char_p, [C.c_int]),
    "apfc_profile_start": (C.c_int, [C.c_void_p, C.c_int]),
    "apfc_profile_read": (
        C.c_int,
        [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.POINTER(C.c_double),
         C.POINTER(C.c_longlong)],
    ),
    "apfc_profile_stop": (C.c_int, [C.c_void_p]),
    "apfc_measure_alu_rate": (C.c_int, [C.c_int, C.c_void_p, C.POINTER(C.c_double)]),
    "apfc_apply_preconditioner_static": (
        C.c_int,
        [C.POINTER(Lattice), C.POINTER(Params), C.POINTER(Grid), C.c_int, C.c_int, C.c_double, C.c_void_p,
         C.c_void_p, C.c_void_p],
    ),
    "apfc_set_params": (C.c_int, [C.c_void_p, C.POINTER(Params)]),
    "apfc_adjoint_step": (
        C.c_int,
        [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_int],
    ),
    "apfc_energy_gradient": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_int]),
    "apfc_rollout_forward": (C.c_int, [C.c_void_p, C.c_double, C.c_int, C.c_int]),
    "apfc_rollout_backward": (
        C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_int]
    ),
    "apfc_rotation_field": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "apfc_batch_init": (
        C.c_int,
        [C.POINTER(C.c_void_p), C.POINTER(Lattice), C.POINTER(Params), C.c_int, C.POINTER(C.c_int),
         C.POINTER(C.c_int), C.c_double, C.c_double, C.POINTER(Opts), C.c_int, C.c_void_p],
    ),
    "apfc_batch_set_opts": (C.c_int, [C.c_void_p, C.POINTER(Opts)]),
    "apfc_batch_get_opts": (C.c_int, [C.c_void_p, C.POINTER(Opts)]),
    "apfc_batch_set_amplitudes": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "apfc_batch_get_amplitudes": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "apfc_batch_step": (C.c_int, [C.c_void_p, C.c_double, C.c_int]),
    "apfc_batch_energy": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "apfc_batch_stats": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(Stats)]),
    "apfc_batch_autotune": (
        C.c_int,
        [C.c_void_p, C.c_double, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double)],
    ),
    "apfc_batch_graph_replays": (C.c_longlong, [C.c_void_p]),
    "apfc_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "apfc_batch_destroy": (None, [C.c_void_p]),
    "apfc_batch_profile_start": (C.c_int, [C.c_void_p, C.c_int]),
    "apfc_batch_profile_read": (
        C.c_int,
        [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.POINTER(C.c_double),
         C.POINTER(C.c_longlong)],
    ),
    "apfc_batch_profile_stop": (C.c_int, [C.c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libapfc.so (built by ``paper_1902_09761_gb300.build``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libapfc.so is not built ({path}); run __graft_entry__.build() first")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


# ---------------------------------------------------------------------------
# Plain wrappers with the C names
# ---------------------------------------------------------------------------


def make_lattice(k, kind: int) -> Lattice:
    k = np.asarray(k, dtype=float)
    L = Lattice()
    L.lattice = kind
    L.J, L.dim = k.shape
    for j in range(L.J):
        for d in range(L.dim):
            L.k[j][d] = float(k[j, d])
    return L


def make_params(dB, Bx, t, v) -> Params:
    return Params(dB, Bx, t, v)


def make_grid(shape, h) -> Grid:
    """shape in array order ((ny, nx) or (nz, ny, nx)); h in (x, y[, z]) order."""
    dim = len(shape)
    g = Grid()
    for d in range(3):
        g.n[d] = int(shape[dim - 1 - d]) if d < dim else 1
        g.h[d] = float(h[d]) if d < dim else 1.0
    return g


def apfc_default_opts(**kw) -> Opts:
    o = Opts()
    _check(load().apfc_default_opts(C.byref(o)))
    for key, val in kw.items():
        setattr(o, key, val)
    return o


def apfc_uniform_amplitude(lattice: Lattice, params: Params) -> float:
    phi = C.c_double()
    _check(load().apfc_uniform_amplitude(C.byref(lattice), C.byref(params), C.byref(phi)))
    return phi.value


def _check(status, ctx=None, init=False):
    if status != APFC_OK:
        # a failed apfc_init has no context: the library keeps this thread's init failure
        msg = load().apfc_last_error(ctx).decode() if (ctx or init) else ""
        raise ApfcError(status, msg)


def _check_batch(status, h=None, init=False):
    if status != APFC_OK:
        # a failed apfc_batch_init has no handle: the library keeps this thread's init failure
        msg = load().apfc_batch_last_error(h).decode() if (h or init) else ""
        raise ApfcError(status, msg)


def _ptr(buf, writable=False, c64_ok=False):
    """(pointer, where, keepalive) of a numpy array or torch tensor of complex128 (or, where
    the entry point takes a dtype, complex64; see _dtype)."""
    if isinstance(buf, np.ndarray):
        ok = buf.dtype == np.complex128 or (c64_ok and buf.dtype == np.complex64)
        if not ok or not buf.flags["C_CONTIGUOUS"]:
            raise TypeError("numpy buffers must be C-contiguous complex128" + (" or complex64" if c64_ok else ""))
        if writable and not buf.flags["WRITEABLE"]:
            raise TypeError("output buffer is read-only")
        return buf.ctypes.data_as(C.c_void_p), APFC_HOST, buf
    import torch  # device buffers only

    if not isinstance(buf, torch.Tensor):
        raise TypeError("buffer must be a numpy array or a torch tensor")
    ok = buf.dtype == torch.complex128 or (c64_ok and buf.dtype == torch.complex64)
    if not ok or not buf.is_contiguous():
        raise TypeError("torch buffers must be contiguous complex128" + (" or complex64" if c64_ok else ""))
    if buf.is_cuda:
        return C.c_void_p(buf.data_ptr()), APFC_DEVICE, buf
    if writable:
        raise TypeError("host output must be a numpy array")
    arr = buf.numpy()
    return arr.ctypes.data_as(C.c_void_p), APFC_HOST, arr


def _dtype(buf) -> int:
    """APFC_C64 for complex64 buffers, else APFC_C128."""
    return APFC_C64 if str(buf.dtype).endswith("complex64") else APFC_C128


class Context:
    """One APFC simulation on one CUDA stream (owns the library context)."""

    def __init__(self, k, kind, params, shape, h, opts: Opts | None = None, stream=None):
        lib = load()
        self.shape = tuple(int(s) for s in shape)
        self.k = np.asarray(k, dtype=float)
        self.J, self.dim = self.k.shape
        self.lattice = make_lattice(self.k, kind)
        self.params = params if isinstance(params, Params) else make_params(*params)
        self.grid = make_grid(self.shape, h)
        self.opts = opts if opts is not None else apfc_default_opts()
        handle = C.c_void_p()
        st = lib.apfc_init(
            C.byref(handle), C.byref(self.lattice), C.byref(self.params), C.byref(self.grid), C.byref(self.opts),
            C.c_void_p(stream) if stream else None,
        )
        _check(st, init=True)
        self._h = handle

    # -- lifecycle ---------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            load().apfc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- state -------------------------------------------------------------
    @property
    def amp_shape(self):
        return (self.J,) + self.shape

    @property
    def block_shape(self):
        return (self.J, 2) + self.shape

    def set_opts(self, opts: Opts):
        _check(load().apfc_set_opts(self._h, C.byref(opts)), self._h)
        self.opts = opts

    def set_amplitudes(self, eta):
        """Copy amplitudes in: complex128 or complex64 (converted on the device)."""
        p, where, keep = _ptr(eta, c64_ok=True)
        _check(load().apfc_set_amplitudes(self._h, p, where, _dtype(eta)), self._h)

    def get_amplitudes(self, out=None, dtype=np.complex128):
        """Copy amplitudes out into `out` (complex128 or complex64), or a new host array of dtype."""
        out = np.empty(self.amp_shape, dtype) if out is None else out
        p, where, keep = _ptr(out, True, c64_ok=True)
        _check(load().apfc_get_amplitudes(self._h, p, where, _dtype(out)), self._h)
        return out

    def get_zeta(self, out=None):
        out = np.empty(self.amp_shape, np.complex128) if out is None else out
        p, where, keep = _ptr(out, True)
        _check(load().apfc_get_zeta(self._h, p, where), self._h)
        return out

    def step(self, dt: float, n: int = 1):
        _check(load().apfc_step(self._h, float(dt), int(n)), self._h)

    def try_step(self, dt: float, n: int = 1) -> int:
        """apfc_step returning the raw status instead of raising."""
        return load().apfc_step(self._h, float(dt), int(n))

    def autotune(self, dt: float) -> dict:
        """apfc_autotune: time one step per candidate segment height and t-kernel variant,
        keep the fastest."""
        rows, tt, ms = C.c_int(), C.c_int(), C.c_double()
        _check(load().apfc_autotune(self._h, float(dt), C.byref(rows), C.byref(tt), C.byref(ms)), self._h)
        return {"tile_rows": rows.value, "tile_t": tt.value, "ms_per_step": ms.value}

    def energy(self) -> float:
        F = C.c_double()
        _check(load().apfc_energy(self._h, C.byref(F)), self._h)
        return F.value

    def stats(self) -> dict:
        s = Stats()
        _check(load().apfc_stats(self._h, C.byref(s)), self._h)
        return {name: getattr(s, name) for name, _ in Stats._fields_}

    def last_error(self) -> str:
        return load().apfc_last_error(self._h).decode()

    # -- measurement -------------------------------------------------------
    def profile_start(self, timed: str | int | None = None):
        """timed: a kernel name or id, None (no event timing) or "all" (every kernel)."""
        if timed == "all":
            tid = -2
        else:
            tid = -1 if timed is None else (timed if isinstance(timed, int) else kernel_ids()[timed])
        _check(load().apfc_profile_start(self._h, tid), self._h)

    def profile_read(self, kernel: str | int) -> dict:
        kid = kernel if isinstance(kernel, int) else kernel_ids()[kernel]
        ms, n, b, tot = C.c_double(), C.c_longlong(), C.c_double(), C.c_longlong()
        _check(load().apfc_profile_read(self._h, kid, C.byref(ms), C.byref(n), C.byref(b), C.byref(tot)), self._h)
        return {"ms": ms.value, "launches": n.value, "bytes": b.value, "all_launches": tot.value}

    def profile_stop(self):
        _check(load().apfc_profile_stop(self._h), self._h)

    # -- operator-level entry points --------------------------------------
    def _binary(self, fn, dt, x, shape, out):
        out = np.empty(shape, np.complex128) if out is None else out
        px, wx, kx = _ptr(x)
        py, wy, ky = _ptr(out, True)
        if wx != wy:
            raise TypeError("input and output must both be host or both be device buffers")
        _check(fn(self._h, float(dt), px, py, wx), self._h)
        return out

    def apply_operator(self, dt, x, out=None):
        return self._binary(load().apfc_apply_operator, dt, x, self.block_shape, out)

    def apply_preconditioner(self, dt, b, out=None):
        return self._binary(load().apfc_apply_preconditioner, dt, b, self.block_shape, out)

    def nonlinear_rhs(self, dt, eta, out=None):
        return self._binary(load().apfc_nonlinear_rhs, dt, eta, self.amp_shape, out)

    # -- parameters and adjoint --------------------------------------------
    def set_params(self, params):
        self.params = params if isinstance(params, Params) else make_params(*params)
        _check(load().apfc_set_params(self._h, C.byref(self.params)), self._h)

    def _same_side(self, *bufs):
        ptrs = [_ptr(b, i == len(bufs) - 1) for i, b in enumerate(bufs)]
        if len({w for _, w, _ in ptrs}) != 1:
            raise TypeError("buffers must all be host or all be device buffers")
        return ptrs

    def adjoint_step(self, dt, eta_n, eta_np1, lam_np1, out=None):
        """(grad wrt eta^n, dL/d dB) of one step, given grad wrt eta^{n+1}."""
        out = np.empty(self.amp_shape, np.complex128) if out is None else out
        (a, w, ka), (b, _, kb), (c, _, kc), (d, _, kd) = self._same_side(eta_n, eta_np1, lam_np1, out)
        g = C.c_double()
        _check(load().apfc_adjoint_step(self._h, float(dt), a, b, c, d, C.byref(g), w), self._h)
        return out, g.value

    def energy_gradient(self, eta, out=None):
        """(grad of F wrt eta, dF/d dB)."""
        out = np.empty(self.amp_shape, np.complex128) if out is None else out
        (a, w, ka), (d, _, kd) = self._same_side(eta, out)
        g = C.c_double()
        _check(load().apfc_energy_gradient(self._h, a, d, C.byref(g), w), self._h)
        return out, g.value

    def rotation_field(self, adapt: dict | None = None, device=None):
        """(omega, A, h) of the current state as numpy arrays (host) or torch tensors (device=...).

        omega has shape (ncomp,) + grid; h is None without ``adapt`` (keys n, h_int, h_max, eps, A_min)."""
        nc = 1 if self.dim == 2 else 3
        a = Adapt(**adapt) if adapt is not None else None
        if device is None:
            om = np.empty((nc,) + self.shape)
            am = np.empty(self.shape)
            hm = np.empty(self.shape) if a is not None else None
            ptr = lambda v: v.ctypes.data_as(C.c_void_p) if v is not None else None  # noqa: E731
            where = APFC_HOST
        else:
            import torch

            om = torch.empty((nc,) + self.shape, dtype=torch.float64, device=device)
            am = torch.empty(self.shape, dtype=torch.float64, device=device)
            hm = torch.empty(self.shape, dtype=torch.float64, device=device) if a is not None else None
            ptr = lambda v: C.c_void_p(v.data_ptr()) if v is not None else None  # noqa: E731
            where = APFC_DEVICE
        _check(load().apfc_rotation_field(self._h, ptr(om), ptr(am), ptr(hm), C.byref(a) if a else None, where),
               self._h)
        return om, am, hm

    def rollout_forward(self, dt: float, n: int, every: int):
        _check(load().apfc_rollout_forward(self._h, float(dt), int(n), int(every)), self._h)

    def rollout_backward(self, lam_n, out=None):
        """(grad wrt eta^0, dL/d dB) of the recorded rollout, given grad wrt eta^n."""
        out = np.empty(self.amp_shape, np.complex128) if out is None else out
        (a, w, ka), (d, _, kd) = self._same_side(lam_n, out)
        g = C.c_double()
        _check(load().apfc_rollout_backward(self._h, a, d, C.byref(g), w), self._h)
        return out, g.value


def apfc_apply_preconditioner_static(lattice: Lattice, params: Params, grid: Grid, cheb_degree: int, tau_mode: int,
                                     dt: float, b_ptr: int, x_ptr: int, stream: int | None = None) -> int:
    """Preconditioner apply without any device allocation (device pointers; returns the status)."""
    return load().apfc_apply_preconditioner_static(
        C.byref(lattice), C.byref(params), C.byref(grid), int(cheb_degree), int(tau_mode), float(dt),
        C.c_void_p(b_ptr), C.c_void_p(x_ptr), C.c_void_p(stream) if stream else None,
    )


class Batch:
    """Independent 2D runs of one lattice, parameter set and spacing on grids of
    different sizes, stepped together (owns the library batch)."""

    def __init__(self, k, kind, params, shapes, h, opts: Opts | None = None, graph: bool = True, stream=None):
        lib = load()
        self.k = np.asarray(k, dtype=float)
        self.J, self.dim = self.k.shape
        self.shapes = [tuple(int(v) for v in s) for s in shapes]  # (ny, nx) per run
        self.R = len(self.shapes)
        self.lattice = make_lattice(self.k, kind)
        self.params = params if isinstance(params, Params) else make_params(*params)
        if opts is None:
            opts = apfc_default_opts(precision=APFC_FP32_REFINED)
        ny = (C.c_int * self.R)(*[s[0] for s in self.shapes])
        nx = (C.c_int * self.R)(*[s[1] for s in self.shapes])
        handle = C.c_void_p()
        st = lib.apfc_batch_init(
            C.byref(handle), C.byref(self.lattice), C.byref(self.params), self.R, nx, ny, float(h[1]), float(h[0]),
            C.byref(opts), APFC_BATCH_GRAPH if graph else 0, C.c_void_p(stream) if stream else None,
        )
        _check_batch(st, init=True)
        self._h = handle

    def close(self):
        if getattr(self, "_h", None):
            load().apfc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def amp_shape(self, run):
        return (self.J,) + self.shapes[run]

    @property
    def opts(self) -> Opts:
        o = Opts()
        _check_batch(load().apfc_batch_get_opts(self._h, C.byref(o)), self._h)
        return o

    def set_opts(self, opts: Opts):
        _check_batch(load().apfc_batch_set_opts(self._h, C.byref(opts)), self._h)

    def set_amplitudes(self, run, eta):
        p, where, keep = _ptr(eta)
        _check_batch(load().apfc_batch_set_amplitudes(self._h, int(run), p, where), self._h)

    def get_amplitudes(self, run, out=None):
        out = np.empty(self.amp_shape(run), np.complex128) if out is None else out
        p, where, keep = _ptr(out, True)
        _check_batch(load().apfc_batch_get_amplitudes(self._h, int(run), p, where), self._h)
        return out

    def step(self, dt: float, n: int = 1):
        _check_batch(load().apfc_batch_step(self._h, float(dt), int(n)), self._h)

    def try_step(self, dt: float, n: int = 1) -> int:
        return load().apfc_batch_step(self._h, float(dt), int(n))

    def energy(self, run) -> float:
        F = C.c_double()
        _check_batch(load().apfc_batch_energy(self._h, int(run), C.byref(F)), self._h)
        return F.value

    def stats(self, run) -> dict:
        s = Stats()
        _check_batch(load().apfc_batch_stats(self._h, int(run), C.byref(s)), self._h)
        return {name: getattr(s, name) for name, _ in Stats._fields_}

    def autotune(self, dt: float) -> dict:
        t, r, ms = C.c_int(), C.c_int(), C.c_double()
        _check_batch(load().apfc_batch_autotune(self._h, float(dt), C.byref(t), C.byref(r), C.byref(ms)), self._h)
        return {"tile": t.value, "tile_rows": r.value, "ms_per_iter": ms.value}

    def graph_replays(self) -> int:
        return load().apfc_batch_graph_replays(self._h)

    def last_error(self) -> str:
        return load().apfc_batch_last_error(self._h).decode()

    def profile_start(self, timed: str | int | None = None):
        if timed == "all":
            tid = -2
        else:
            tid = -1 if timed is None else (timed if isinstance(timed, int) else kernel_ids()[timed])
        _check_batch(load().apfc_batch_profile_start(self._h, tid), self._h)

    def profile_read(self, kernel: str | int) -> dict:
        kid = kernel if isinstance(kernel, int) else kernel_ids()[kernel]
        ms, n, b, tot = C.c_double(), C.c_longlong(), C.c_double(), C.c_longlong()
        _check_batch(
            load().apfc_batch_profile_read(self._h, kid, C.byref(ms), C.byref(n), C.byref(b), C.byref(tot)), self._h
        )
        return {"ms": ms.value, "launches": n.value, "bytes": b.value, "all_launches": tot.value}

    def profile_stop(self):
        _check_batch(load().apfc_batch_profile_stop(self._h), self._h)


def measure_alu_rate(kind: int, stream: int | None = None) -> float:
    """Arithmetic rate of the current GPU: FLOP/s of FP64 (APFC_ALU_FMA64) or FP32 (APFC_ALU_FMA32)
    FMAs, or FP64 <-> FP32 conversions/s (APFC_ALU_CVT64)."""
    out = C.c_double()
    _check(load().apfc_measure_alu_rate(int(kind), C.c_void_p(stream) if stream else None, C.byref(out)))
    return out.value


def kernel_ids() -> dict:
    """{name: id} of the library's kernels (apfc_kernel_name)."""
    lib = load()
    return {lib.apfc_kernel_name(i).decode(): i for i in range(lib.apfc_kernel_count())}


def apfc_init(k, kind, params, shape, h, opts=None, stream=None) -> Context:
    return Context(k, kind, params, shape, h, opts, stream)


def apfc_step(ctx: Context, dt: float, n: int = 1):
    ctx.step(dt, n)


def apfc_energy(ctx: Context) -> float:
    return ctx.energy()
