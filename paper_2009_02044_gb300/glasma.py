"""Python binding of the C ABI in include/glasma.h (ctypes).

Argument marshalling only: every step of the method runs in the CUDA
kernels of libglasma.so.  PyTorch provides the device memory (through the
caching allocator, passed to the library as its allocator callbacks) and
the CUDA stream.  If the shared library is missing the import fails loudly;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libglasma.so")

GLASMA_OK = 0
ERRORS = {
    -1: "INVALID_ARG", -2: "CUDA", -3: "OOM", -4: "NONFINITE",
    -5: "PARTICLE_EXIT", -6: "NOT_CONVERGED", -7: "TIMEOUT", -8: "CHECKSUM",
    -9: "INTERNAL",
}
FP64, FP32 = 0, 1
LEAPFROG, IMPLICIT = 0, 1
KERNELS = {"auto": 0, "staple": 1, "plaquette": 2, "plaquette_256": 3,
           "staple_pairs": 4, "staple_staged": 5}


class GlasmaError(RuntimeError):
    def __init__(self, status, fn, msg):
        self.status = status
        self.code = ERRORS.get(status, str(status))
        super().__init__("%s failed: %s (%s)" % (fn, self.code, msg))


class glasma_params(C.Structure):
    _fields_ = [("nc", C.c_int), ("nz", C.c_int), ("nx", C.c_int),
                ("ny", C.c_int), ("a_t", C.c_double), ("a_z", C.c_double),
                ("dt", C.c_double), ("sigma_l", C.c_double),
                ("g2mu", C.c_double), ("m_ir", C.c_double),
                ("uv_cutoff", C.c_double), ("z_offset", C.c_double),
                ("seed", C.c_ulonglong), ("precision", C.c_int),
                ("scheme", C.c_int), ("implicit_max_iter", C.c_int),
                ("implicit_tol", C.c_double), ("n_sheets", C.c_int)]


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class glasma_allocator(C.Structure):
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("user", C.c_void_p)]


class glasma_info(C.Structure):
    _fields_ = [("sites", C.c_longlong), ("step_n", C.c_longlong),
                ("nc", C.c_int), ("precision", C.c_int), ("scheme", C.c_int),
                ("window_a", C.c_int * 2), ("window_b", C.c_int * 2),
                ("state_device_bytes", C.c_size_t),
                ("kernel_launches", C.c_int), ("implicit_iters", C.c_int)]


_lib = None


def load_library(path=LIB_PATH):
    """Load libglasma.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            "libglasma.so not found at %s: build it first "
            "(python -m paper_2009_02044_gb300.build)" % path)
    lib = C.CDLL(path)
    P = C.c_void_p
    dp = C.POINTER(C.c_double)
    sig = {
        "glasma_init_mv": (C.c_int, [C.POINTER(glasma_params), dp, P,
                                     C.POINTER(glasma_allocator),
                                     C.POINTER(C.c_void_p)]),
        "glasma_step": (C.c_int, [P, C.c_int]),
        "glasma_gauss_residual": (C.c_int, [P, dp, dp, dp]),
        "glasma_tmunu": (C.c_int, [P, dp, dp]),
        "glasma_free": (None, [P]),
        "glasma_strerror": (C.c_char_p, [C.c_int]),
        "glasma_last_error_message": (C.c_char_p, []),
        "glasma_get_fields": (C.c_int, [P, dp, dp, dp, dp,
                                        C.POINTER(C.c_longlong)]),
        "glasma_set_fields": (C.c_int, [P, dp, dp, dp, dp, dp, C.c_longlong]),
        "glasma_state_bytes": (C.c_int, [P, C.POINTER(C.c_size_t)]),
        "glasma_get_state": (C.c_int, [P, P, C.c_size_t]),
        "glasma_set_state": (C.c_int, [P, P, C.c_size_t]),
        "glasma_get_info": (C.c_int, [P, C.POINTER(glasma_info)]),
        "glasma_set_step_kernel": (C.c_int, [P, C.c_int, C.c_int]),
        "glasma_set_staging_wait": (C.c_int, [P, C.c_longlong, C.c_int]),
        "glasma_slab_init": (C.c_int, [C.POINTER(glasma_params), dp, C.c_int,
                                       C.c_int, P, C.POINTER(glasma_allocator),
                                       C.POINTER(C.c_void_p)]),
        "glasma_slab_info": (C.c_int, [P] + [C.POINTER(C.c_int)] * 5),
        "glasma_slab_set_windows": (C.c_int, [P, C.c_int, C.c_int, C.c_int,
                                              C.c_int]),
        "glasma_slab_message_bytes": (C.c_int, [P, C.c_int,
                                                C.POINTER(C.c_size_t)]),
        "glasma_slab_pack": (C.c_int, [P, C.c_int, P]),
        "glasma_slab_unpack": (C.c_int, [P, C.c_int, P]),
        "glasma_implicit_begin": (C.c_int, [P]),
        "glasma_implicit_sweep": (C.c_int, [P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "glasma_implicit_end": (C.c_int, [P]),
        "glasma_gauss_residual_static": (
            C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                      C.c_double, C.c_double, P, P, P, C.c_int, C.c_int, P,
                      C.c_int, C.c_int, P, dp, dp, dp]),
        "glasma_tmunu_device": (C.c_int, [P, P]),
        "glasma_rest_frame": (C.c_int, [P, C.c_int, C.c_longlong, P, P]),
        "glasma_sample_grid": (C.c_int, [P, C.c_int, C.c_int, C.c_int, C.c_int,
                                         C.c_double, C.c_double, C.c_double,
                                         C.c_double, P, P, C.c_longlong,
                                         C.c_int, P, P]),
        "glasma_implicit_converged": (C.c_int, [dp, dp, C.c_int, C.c_double, C.c_int,
                                                 C.POINTER(C.c_int)]),
        "glasma_fit_gaussian": (C.c_int, [dp, dp, C.c_int, C.c_double, dp, dp,
                                          dp]),
        "glasma_adjoint_energy": (C.c_int, [C.POINTER(glasma_params), dp,
                                            C.c_int, C.c_double, C.c_int, P,
                                            C.POINTER(glasma_allocator), dp,
                                            dp]),
        "glasma_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int,
                                          C.POINTER(C.c_void_p)]),
        "glasma_batch_step": (C.c_int, [P, C.c_int]),
        "glasma_batch_tune": (C.c_int, [P, C.c_int, C.POINTER(C.c_int),
                                        C.POINTER(C.c_int)]),
        "glasma_batch_set_shape": (C.c_int, [P, C.c_int, C.c_int]),
        "glasma_batch_set_barrier": (C.c_int, [P, C.c_longlong, C.c_int]),
        "glasma_batch_free": (None, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status, fn):
    if status != GLASMA_OK:
        msg = load_library().glasma_last_error_message().decode()
        raise GlasmaError(status, fn, msg)


def _dptr(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(cfg):
    """glasma_params from a config dict (keys as in glasma_inputs)."""
    p = glasma_params()
    p.nc = int(cfg["nc"])
    p.nz, p.nx, p.ny = int(cfg["nz"]), int(cfg["nx"]), int(cfg["ny"])
    p.a_t = float(cfg.get("a_t", 1.0))
    p.a_z = float(cfg.get("a_z", 1.0))
    p.dt = float(cfg["dt"])
    p.sigma_l = float(cfg["sigma_l"])
    p.g2mu = float(cfg["g2mu"])
    p.m_ir = float(cfg["m_ir"])
    p.uv_cutoff = float(cfg.get("uv_cutoff", 0.0))
    p.z_offset = float(cfg.get("z_offset", 0.0))
    p.seed = int(cfg.get("seed", 0))
    prec = cfg.get("precision", "fp64")
    p.precision = FP32 if prec in ("fp32", FP32) else FP64
    sch = cfg.get("scheme", "leapfrog")
    p.scheme = IMPLICIT if sch in ("implicit", IMPLICIT) else LEAPFROG
    p.implicit_max_iter = int(cfg.get("implicit_max_iter", 50))
    p.implicit_tol = float(cfg.get("implicit_tol", 1e-14))
    p.n_sheets = int(cfg.get("n_sheets", 1))
    return p


# --- PyTorch as the device-memory provider --------------------------------

_live_blocks = {}


def _torch_allocator():
    import torch

    @_ALLOC_FN
    def _alloc(nbytes, stream, user):
        try:
            ptr = torch.cuda.caching_allocator_alloc(
                int(nbytes), torch.cuda.current_device(),
                int(stream or 0) or torch.cuda.current_stream())
        except Exception:
            return None
        _live_blocks[ptr] = nbytes
        return ptr

    @_FREE_FN
    def _free(ptr, nbytes, stream, user):
        if ptr in _live_blocks:
            del _live_blocks[ptr]
            torch.cuda.caching_allocator_delete(ptr)

    a = glasma_allocator()
    a.alloc = _alloc
    a.free = _free
    a.user = None
    return a, (_alloc, _free)


# --- the C calls, same names ------------------------------------------------

def glasma_init_mv(cfg, rho=None, stream=None, torch_memory=True):
    """Create a context with the MV initial state; returns an opaque handle.

    rho: None (draw from cfg['seed'] on the device) or float64 array
    [2][nc^2-1][ny][nx].  stream: a torch.cuda.Stream, a raw cudaStream_t
    integer or None (torch's current stream)."""
    return _create(cfg, rho, stream, torch_memory, None)


def glasma_slab_init(cfg, z0, z1, rho=None, stream=None, torch_memory=True):
    """Context of the global slices [z0, z1) of the event cfg describes,
    with its halo slices (see include/glasma.h); the handle's `slab` holds
    (z0, z1, local slices, lo, hi)."""
    return _create(cfg, rho, stream, torch_memory, (int(z0), int(z1)))


def _create(cfg, rho, stream, torch_memory, slab):
    lib = load_library()
    p = make_params(cfg)
    if rho is not None:
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        na = p.nc * p.nc - 1
        want = (2, na, p.ny, p.nx)
        if p.n_sheets > 1:
            want = (p.n_sheets,) + want
        if rho.shape != want:
            raise ValueError("rho must have shape %s" % (want,))
    keep = None
    alloc_ptr = None
    if torch_memory:
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        a, keep = _torch_allocator()
        alloc_ptr = C.byref(a)
        keep = (a, keep)
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    out = C.c_void_p()
    if slab is None:
        st = lib.glasma_init_mv(C.byref(p), _dptr(rho), C.c_void_p(s or 0),
                                alloc_ptr, C.byref(out))
        _check(st, "glasma_init_mv")
        return Handle(out, p, keep)
    st = lib.glasma_slab_init(C.byref(p), _dptr(rho), slab[0], slab[1],
                              C.c_void_p(s or 0), alloc_ptr, C.byref(out))
    _check(st, "glasma_slab_init")
    h = Handle(out, p, keep)
    v = [C.c_int() for _ in range(5)]
    _check(lib.glasma_slab_info(out, *[C.byref(x) for x in v]),
           "glasma_slab_info")
    h.slab = tuple(x.value for x in v)
    return h


class Handle:
    """Owns one glasma_ctx*; frees it when closed or collected."""

    def __init__(self, ptr, params, keep):
        self.ptr = ptr
        self.params = params
        self._keep = keep
        self.slab = None      # (z0, z1, local slices, lo, hi) of a slab

    @property
    def local_nz(self):
        """Slices of the context's own lattice (a slab's with its halos)."""
        return self.params.nz if self.slab is None else self.slab[2]

    @property
    def rows(self):
        """T^{mu nu} rows glasma_tmunu returns (the owned slices)."""
        return self.params.nz if self.slab is None else self.slab[1] - self.slab[0]

    @property
    def na(self):
        return self.params.nc * self.params.nc - 1

    def close(self):
        if self.ptr is not None and self.ptr.value:
            load_library().glasma_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def glasma_step(h, n_steps):
    _check(load_library().glasma_step(h.ptr, int(n_steps)), "glasma_step")


def glasma_gauss_residual(h):
    m, r, q = C.c_double(), C.c_double(), C.c_double()
    _check(load_library().glasma_gauss_residual(h.ptr, C.byref(m), C.byref(r),
                                                C.byref(q)),
           "glasma_gauss_residual")
    return m.value, r.value, q.value


def glasma_tmunu(h):
    tab = np.empty((h.rows, 4))
    H = C.c_double()
    _check(load_library().glasma_tmunu(h.ptr, _dptr(tab), C.byref(H)),
           "glasma_tmunu")
    return tab, H.value


def glasma_get_fields(h):
    p = h.params
    nz = h.local_nz
    V = nz * p.ny * p.nx
    na, nc = h.na, p.nc
    U = np.empty((3, nz, p.ny, p.nx, nc, nc, 2))
    E = np.empty((3, nz, p.ny, p.nx, na))
    QA = np.empty((nz, p.ny, p.nx, na))
    QB = np.empty((nz, p.ny, p.nx, na))
    n = C.c_longlong()
    _check(load_library().glasma_get_fields(h.ptr, _dptr(U), _dptr(E),
                                            _dptr(QA), _dptr(QB), C.byref(n)),
           "glasma_get_fields")
    assert U.size == 3 * V * nc * nc * 2
    return U[..., 0] + 1j * U[..., 1], E, QA, QB, n.value


def glasma_set_fields(h, U, E, QA=None, QB=None, U_prev=None, step_n=0):
    def links(u):
        if u is None:
            return None
        u = np.asarray(u)
        return np.ascontiguousarray(np.stack([u.real, u.imag], -1),
                                    dtype=np.float64)
    E = np.ascontiguousarray(E, dtype=np.float64)
    QA = None if QA is None else np.ascontiguousarray(QA, dtype=np.float64)
    QB = None if QB is None else np.ascontiguousarray(QB, dtype=np.float64)
    Ul, Upl = links(U), links(U_prev)
    _check(load_library().glasma_set_fields(h.ptr, _dptr(Ul), _dptr(E),
                                            _dptr(QA), _dptr(QB), _dptr(Upl),
                                            int(step_n)),
           "glasma_set_fields")


def glasma_state_bytes(h):
    n = C.c_size_t()
    _check(load_library().glasma_state_bytes(h.ptr, C.byref(n)),
           "glasma_state_bytes")
    return n.value


def glasma_get_state(h):
    buf = np.empty(glasma_state_bytes(h), dtype=np.uint8)
    _check(load_library().glasma_get_state(h.ptr, buf.ctypes.data_as(C.c_void_p),
                                           buf.nbytes), "glasma_get_state")
    return buf


def glasma_set_state(h, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint8)
    _check(load_library().glasma_set_state(h.ptr, buf.ctypes.data_as(C.c_void_p),
                                           buf.nbytes), "glasma_set_state")


def glasma_get_info(h):
    info = glasma_info()
    _check(load_library().glasma_get_info(h.ptr, C.byref(info)),
           "glasma_get_info")
    return info


def glasma_set_step_kernel(h, kernel="auto", zlen=0):
    """Leapfrog step kernel of the context: "auto", "staple", "plaquette",
    "plaquette_256", "staple_pairs" (FP32) or "staple_staged" (FP32 SU(3),
    nx = 32 or 64); zlen = z slices per block of the plaquette kernel
    (0 = automatic)."""
    _check(load_library().glasma_set_step_kernel(h.ptr, KERNELS[kernel],
                                                 int(zlen)),
           "glasma_set_step_kernel")


def glasma_set_staging_wait(h, wait_cycles=1 << 31, stall=False):
    """Spin budget (SM cycles) of one wait of the staged step kernel, and
    the stall that makes a wait run out (for testing the timeout path)."""
    _check(load_library().glasma_set_staging_wait(h.ptr, int(wait_cycles),
                                                  1 if stall else 0),
           "glasma_set_staging_wait")


def glasma_slab_set_windows(h, window_a, window_b):
    """Whole-lattice charge windows (first global slice, slices) of A, B."""
    _check(load_library().glasma_slab_set_windows(
        h.ptr, int(window_a[0]), int(window_a[1]), int(window_b[0]),
        int(window_b[1])), "glasma_slab_set_windows")


def glasma_slab_message_bytes(h, direction):
    n = C.c_size_t()
    _check(load_library().glasma_slab_message_bytes(h.ptr, int(direction),
                                                    C.byref(n)),
           "glasma_slab_message_bytes")
    return n.value


def glasma_slab_pack(h, direction, dev_ptr):
    _check(load_library().glasma_slab_pack(h.ptr, int(direction),
                                           C.c_void_p(dev_ptr)),
           "glasma_slab_pack")


def glasma_slab_unpack(h, direction, dev_ptr):
    _check(load_library().glasma_slab_unpack(h.ptr, int(direction),
                                             C.c_void_p(dev_ptr)),
           "glasma_slab_unpack")


def glasma_implicit_begin(h):
    """Begin an improved step driven sweep by sweep (see include/glasma.h)."""
    _check(load_library().glasma_implicit_begin(h.ptr), "glasma_implicit_begin")


def glasma_implicit_sweep(h):
    """One sweep; returns (max |dE|, max |E|) over the owned slices."""
    d, e = C.c_double(), C.c_double()
    _check(load_library().glasma_implicit_sweep(h.ptr, C.byref(d), C.byref(e)),
           "glasma_implicit_sweep")
    return d.value, e.value


def glasma_implicit_end(h):
    """Commit the step begun by glasma_implicit_begin."""
    _check(load_library().glasma_implicit_end(h.ptr), "glasma_implicit_end")


def glasma_free(h):
    h.close()


def glasma_strerror(status):
    return load_library().glasma_strerror(int(status)).decode()


def glasma_gauss_residual_static(nc, precision, nz, ny, nx, a_t, a_z, U, E,
                                 QA=None, zA0=0, WA=0, QB=None, zB0=0, WB=0,
                                 stream=None):
    """Gauss residual of caller-owned device fields with no device
    allocation (see include/glasma.h).  U, E, QA, QB are raw device
    addresses (ints) in the library's layout; returns (max, rms, rho_max)."""
    m, r, q = C.c_double(), C.c_double(), C.c_double()
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    prec = FP32 if precision in ("fp32", FP32) else FP64
    _check(load_library().glasma_gauss_residual_static(
        int(nc), prec, int(nz), int(ny), int(nx), float(a_t), float(a_z),
        C.c_void_p(U), C.c_void_p(E), C.c_void_p(QA), int(zA0), int(WA),
        C.c_void_p(QB), int(zB0), int(WB), C.c_void_p(s or 0),
        C.byref(m), C.byref(r), C.byref(q)), "glasma_gauss_residual_static")
    return m.value, r.value, q.value


class Batch:
    """Owns one glasma_batch* over borrowed contexts (kept alive here)."""

    def __init__(self, ptr, handles):
        self.ptr = ptr
        self.handles = list(handles)

    def close(self):
        if self.ptr is not None and self.ptr.value:
            load_library().glasma_batch_free(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def glasma_batch_create(handles):
    """One batch over Handles that share nc, precision, dt, a_t, a_z and
    the stream (leapfrog scheme)."""
    arr = (C.c_void_p * len(handles))(*[h.ptr.value for h in handles])
    out = C.c_void_p()
    _check(load_library().glasma_batch_create(arr, len(handles), C.byref(out)),
           "glasma_batch_create")
    return Batch(out, handles)


def glasma_batch_step(b, n_steps):
    _check(load_library().glasma_batch_step(b.ptr, int(n_steps)),
           "glasma_batch_step")


BATCH_MODES = {"graph": 0, "persistent": 1, "per_event": 2}


def glasma_batch_tune(b, steps=10):
    """Time every mode and block shape on the batch; returns the kept
    (block_sites, mode name).  The events' states are left as they were."""
    bx, mode = C.c_int(), C.c_int()
    _check(load_library().glasma_batch_tune(b.ptr, int(steps), C.byref(bx),
                                            C.byref(mode)),
           "glasma_batch_tune")
    names = {v: k for k, v in BATCH_MODES.items()}
    return bx.value, names[mode.value]


def glasma_batch_set_shape(b, mode, block_sites=64):
    """mode: "graph", "persistent" or "per_event"."""
    _check(load_library().glasma_batch_set_shape(b.ptr, BATCH_MODES[mode],
                                                 int(block_sites)),
           "glasma_batch_set_shape")


def glasma_batch_set_barrier(b, wait_cycles, extra_arrivals=0):
    _check(load_library().glasma_batch_set_barrier(b.ptr, int(wait_cycles),
                                                   int(extra_arrivals)),
           "glasma_batch_set_barrier")


def glasma_batch_free(b):
    b.close()


def _stream_ptr(stream):
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    return C.c_void_p(s or 0)


def glasma_tmunu_device(h, dev_out):
    """T^{mu nu} table [nz][4] into device memory at address dev_out (an
    int, e.g. tensor.data_ptr()), on the context's stream, no sync."""
    _check(load_library().glasma_tmunu_device(h.ptr, C.c_void_p(dev_out)),
           "glasma_tmunu_device")


def glasma_rest_frame(tabs, n_events, n_points, out, stream=None):
    """Event mean and local rest frame (device addresses; see
    include/glasma.h): tabs [n_events][n_points][4] -> out
    [n_points][8]."""
    _check(load_library().glasma_rest_frame(
        C.c_void_p(tabs), int(n_events), int(n_points), C.c_void_p(out),
        _stream_ptr(stream)), "glasma_rest_frame")


def glasma_sample_grid(grid, n_t, nz, stride, comp, t0, dts, z0, az, x, y,
                       n_pts, out, coords="milne", stream=None):
    """Bilinear samples of grid [n_t][nz][stride] component comp at
    (tau, eta_s) (coords "milne") or (t, z) (coords "lab") points; device
    addresses."""
    _check(load_library().glasma_sample_grid(
        C.c_void_p(grid), int(n_t), int(nz), int(stride), int(comp),
        float(t0), float(dts), float(z0), float(az), C.c_void_p(x),
        C.c_void_p(y), int(n_pts), {"milne": 0, "lab": 1}[coords],
        C.c_void_p(out), _stream_ptr(stream)), "glasma_sample_grid")


def glasma_implicit_converged(dmax, emax, tol=1e-14, precision="fp32"):
    """Whether the improved scheme's iteration stops after the last of the
    sweeps whose max |dE| and max |E| are given (host computation)."""
    d = np.ascontiguousarray(dmax, dtype=np.float64)
    e = np.ascontiguousarray(emax, dtype=np.float64)
    if d.size == 0 or d.size != e.size:
        raise ValueError("dmax and emax need the same, non-zero length")
    out = C.c_int()
    prec = FP32 if precision in ("fp32", FP32) else FP64
    _check(load_library().glasma_implicit_converged(
        _dptr(d), _dptr(e), d.size - 1, float(tol), prec, C.byref(out)),
        "glasma_implicit_converged")
    return bool(out.value)


def glasma_fit_gaussian(x, f, frac=0.1):
    """(amp, mu, sigma) of the Gaussian fitted to host arrays x, f."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    amp, mu, sig = C.c_double(), C.c_double(), C.c_double()
    _check(load_library().glasma_fit_gaussian(
        _dptr(x), _dptr(f), len(x), float(frac), C.byref(amp), C.byref(mu),
        C.byref(sig)), "glasma_fit_gaussian")
    return amp.value, mu.value, sig.value


def glasma_adjoint_energy(cfg, rho, n_steps, half_width, checkpoint_every=20,
                          stream=None, grad=True, torch_memory=True):
    """O = a_z sum_{|z - z_c| < half_width} eps(z) after n_steps from the
    MV charges rho [2][3][ny][nx] (SU(2), FP64, leapfrog) and, if grad,
    dO/drho from the hand-written adjoint (include/glasma.h).
    Returns (O, gradient array or None)."""
    lib = load_library()
    p = make_params(cfg)
    r = None
    if rho is not None:
        r = np.ascontiguousarray(rho, dtype=np.float64)
        if r.shape != (2, 3, p.ny, p.nx):
            raise ValueError("rho must have shape (2, 3, %d, %d)" % (p.ny, p.nx))
    keep = None
    alloc_ptr = None
    if torch_memory:
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        a, keep = _torch_allocator()
        alloc_ptr = C.byref(a)
    s = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    val = C.c_double()
    g = np.zeros((2, 3, p.ny, p.nx)) if grad else None
    st = lib.glasma_adjoint_energy(C.byref(p), _dptr(r), int(n_steps),
                                   float(half_width), int(checkpoint_every),
                                   C.c_void_p(s or 0), alloc_ptr,
                                   C.byref(val), _dptr(g))
    del keep
    _check(st, "glasma_adjoint_energy")
    return val.value, g


def mid_rapidity_energy(rho, cfg, n_steps, half_width, checkpoint_every=20):
    """The observable as a differentiable torch function of rho (float64
    tensor [2][3][ny][nx] on any device): forward runs the simulation, the
    backward pass calls the CUDA adjoint."""
    import torch

    class _MidEnergy(torch.autograd.Function):
        @staticmethod
        def forward(ctx, r):
            host = r.detach().to("cpu", torch.float64).numpy()
            val, _ = glasma_adjoint_energy(cfg, host, n_steps, half_width,
                                           checkpoint_every, grad=False)
            ctx.host = host
            return r.new_tensor(val)

        @staticmethod
        def backward(ctx, go):
            _, g = glasma_adjoint_energy(cfg, ctx.host, n_steps, half_width,
                                         checkpoint_every, grad=True)
            return go * torch.from_numpy(g).to(go.device, go.dtype)

    return _MidEnergy.apply(rho)
