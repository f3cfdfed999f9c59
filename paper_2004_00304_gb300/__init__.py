"""GB300-native coupled lattice Boltzmann / MPCD time stepper.

A thin ctypes binding over the C ABI of ``liblbmpcd.so`` (declared in
``include/lbmpcd.h``).  Every step of the method runs in the library's CUDA
kernels; this module only marshals arguments.  There is no CPU fallback:
importing the binding without a built library, or creating a handle without a
CUDA device, raises.

The entry points keep the ABI's names: :func:`lbmpcd_create`,
:func:`lbmpcd_set_region`, :func:`lbmpcd_step`, :func:`lbmpcd_get_fields`,
:func:`lbmpcd_set_state`, :func:`lbmpcd_destroy`; :class:`Lbmpcd` wraps them.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbmpcd.so")

D2Q9, D3Q19 = 9, 19
FP64, FP32, FP16DEV = 0, 1, 2
FIELDS = dict(RHO=0, U=1, POPS=2, PART_POS=3, PART_VEL=4, PART_CELL=5, SHIFT=6,
              CELL_COUNT=7, WINDOW_MEAN=8, DIAG=9, PART_HOME=10, CELL_VCM=11, PART_ID=12,
              CLOSURE_IN=13, CLOSURE_OUT=14, CLOSURE_TARGET=15, CELL_LIST=17)
INT_FIELDS = {"PART_CELL", "CELL_COUNT", "PART_HOME", "PART_ID", "CELL_LIST"}
LAUNCH_LB_TMA = 1   # LBMPCD_LAUNCH_LB_TMA
LAUNCH_SERIAL = 2   # LBMPCD_LAUNCH_SERIAL
ERRORS = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "TIMEOUT", -5: "STATE", -6: "CAPACITY"}


class LbmpcdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class lbmpcd_params(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("tau", ctypes.c_double), ("force", ctypes.c_double * 3),
                ("refine", ctypes.c_int), ("ppc", ctypes.c_int), ("alpha", ctypes.c_double),
                ("kT", ctypes.c_double), ("mass", ctypes.c_double),
                ("coupling_width", ctypes.c_int), ("precision", ctypes.c_int),
                ("feedback", ctypes.c_int), ("window", ctypes.c_int),
                ("resample_density", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("collision", ctypes.c_int), ("redraw", ctypes.c_int)]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load liblbmpcd.so (build it with ``paper_2004_00304_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"liblbmpcd.so not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp, ci, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    L.lbmpcd_create.argtypes = [ctypes.POINTER(lbmpcd_params), ci, vp, ctypes.POINTER(vp)]
    L.lbmpcd_set_region.argtypes = [vp, ci, ctypes.POINTER(ci), ctypes.POINTER(ci)]
    L.lbmpcd_set_region_piece.argtypes = [vp, ci, ctypes.POINTER(ci), ctypes.POINTER(ci), ci, ci, ci, ci]
    L.lbmpcd_set_particles.argtypes = [vp, ci, ctypes.c_longlong, vp, vp, vp, vp]
    L.lbmpcd_step.argtypes = [vp, ci]
    L.lbmpcd_get_fields.argtypes = [vp, ci, ci, vp, sz, ci]
    L.lbmpcd_set_state.argtypes = [vp, ci, ci, vp, sz, ci]
    L.lbmpcd_field_size.argtypes = [vp, ci, ci]
    L.lbmpcd_field_size.restype = ctypes.c_longlong
    L.lbmpcd_step_profiled.argtypes = [vp, ci, ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_longlong)]
    L.lbmpcd_tc_gemm_bf16.argtypes = [vp, vp, vp, ci, ci, ci, ctypes.c_float, ctypes.c_float, vp, vp]
    ll, fp = ctypes.c_longlong, ctypes.POINTER(ctypes.c_float)
    L.lbmpcd_net_num_params.restype = ll
    L.lbmpcd_net_num_params.argtypes = []
    L.lbmpcd_net_create.argtypes = [ci, vp, ctypes.POINTER(vp)]
    L.lbmpcd_net_get_params.argtypes = [vp, vp, ll, ci, ci]
    L.lbmpcd_net_set_params.argtypes = [vp, vp, ll, ci]
    L.lbmpcd_net_forward.argtypes = [vp, vp, ci, vp]
    L.lbmpcd_net_backward.argtypes = [vp, vp, vp, ci, fp]
    L.lbmpcd_net_train_step.argtypes = [vp, vp, vp, ci, ctypes.c_float, fp]
    L.lbmpcd_net_destroy.argtypes = [vp]
    L.lbmpcd_net_forward_noalloc.argtypes = [vp, vp, ci, vp, vp]
    L.lbmpcd_set_closure.argtypes = [vp, vp, ll, ci, ci]
    L.lbmpcd_set_launch_mode.argtypes = [vp, ci, ci, ci]
    L.lbmpcd_set_wait_limit.argtypes = [vp, ctypes.c_uint]
    L.lbmpcd_autotune.argtypes = [vp, ci, ctypes.POINTER(ci)]
    L.lbmpcd_population_bytes.argtypes = [vp]
    L.lbmpcd_get_columns.argtypes = [vp, ci, ci, ci, vp, ci]
    L.lbmpcd_set_columns.argtypes = [vp, ci, ci, ci, vp, ci]
    L.lbmpcd_net_destroy.restype = None
    L.lbmpcd_destroy.argtypes = [vp]
    L.lbmpcd_destroy.restype = None
    L.lbmpcd_last_error.argtypes = [vp]
    L.lbmpcd_last_error.restype = ctypes.c_char_p
    _lib = L
    return L


EXPORTED = ["lbmpcd_create", "lbmpcd_set_region", "lbmpcd_step", "lbmpcd_step_profiled",
            "lbmpcd_get_fields", "lbmpcd_set_state", "lbmpcd_field_size", "lbmpcd_destroy",
            "lbmpcd_last_error", "lbmpcd_tc_gemm_bf16", "lbmpcd_net_num_params", "lbmpcd_net_create",
            "lbmpcd_net_get_params", "lbmpcd_net_set_params", "lbmpcd_net_forward", "lbmpcd_net_backward",
            "lbmpcd_net_train_step", "lbmpcd_net_destroy", "lbmpcd_net_forward_noalloc",
            "lbmpcd_set_closure", "lbmpcd_set_launch_mode", "lbmpcd_set_wait_limit", "lbmpcd_autotune",
            "lbmpcd_population_bytes", "lbmpcd_get_columns", "lbmpcd_set_columns", "lbmpcd_set_region_piece",
            "lbmpcd_set_particles"]


def make_params(d: dict) -> lbmpcd_params:
    p = lbmpcd_params()
    p.lattice = int(d.get("lattice", 9))
    p.nx, p.ny, p.nz = int(d["nx"]), int(d["ny"]), int(d.get("nz", 1))
    p.tau = float(d["tau"])
    f = list(d.get("force", (0.0, 0.0, 0.0))) + [0.0, 0.0, 0.0]
    p.force = (ctypes.c_double * 3)(*[float(x) for x in f[:3]])
    p.refine = int(d.get("refine", 1))
    p.ppc = int(d.get("ppc", 10))
    p.alpha = float(d.get("alpha", math.radians(130.0)))
    p.kT = float(d.get("kT", 1e-4))
    p.mass = float(d.get("mass", 1.0))
    p.coupling_width = int(d.get("coupling_width", 2))
    p.precision = int(d.get("precision", FP32))
    p.feedback = int(d.get("feedback", 0))
    p.window = int(d.get("window", 100))
    p.resample_density = int(d.get("resample_density", 0))
    p.seed = int(d.get("seed", 1))
    p.collision = int(d.get("collision", 0))
    p.redraw = int(d.get("redraw", 0))
    return p


def _check(h, rc: int):
    if rc != 0:
        msg = load_library().lbmpcd_last_error(h)
        raise LbmpcdError(rc, msg.decode() if msg else "")


def lbmpcd_create(params, n_replicas: int = None, stream=None):
    """Create a handle; ``params`` is a dict or a list of dicts (one per replica).
    ``stream`` is a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
    L = load_library()
    plist = params if isinstance(params, (list, tuple)) else [params]
    n = len(plist) if n_replicas is None else int(n_replicas)
    arr = (lbmpcd_params * n)(*[make_params(p) for p in plist[:n]])
    sptr = getattr(stream, "cuda_stream", stream) or 0
    h = ctypes.c_void_p()
    rc = L.lbmpcd_create(arr, n, ctypes.c_void_p(int(sptr)), ctypes.byref(h))
    _check(None, rc)
    return h


def lbmpcd_set_region(h, replica: int, lo, hi):
    lo3 = (ctypes.c_int * 3)(*[int(v) for v in lo])
    hi3 = (ctypes.c_int * 3)(*[int(v) for v in hi])
    _check(h, load_library().lbmpcd_set_region(h, int(replica), lo3, hi3))


def lbmpcd_set_region_piece(h, replica: int, lo, hi, own, keep):
    """A piece of a region divided over x-slabs: lo / hi the whole region in
    this handle's LB columns (may reach beyond the lattice), own = (own_lo,
    own_hi) the owned LB columns, keep = (keep_lo, keep_hi) the region cell
    columns (mod the region's width) whose particles the handle keeps."""
    lo3 = (ctypes.c_int * 3)(*[int(v) for v in lo])
    hi3 = (ctypes.c_int * 3)(*[int(v) for v in hi])
    _check(h, load_library().lbmpcd_set_region_piece(h, int(replica), lo3, hi3, int(own[0]), int(own[1]),
                                                     int(keep[0]), int(keep[1])))


def lbmpcd_set_particles(h, replica: int, home, off, vel, pid):
    """Replace the pooled particles of a region piece (home int32 [n][3],
    offsets and velocities binary64 [n][3], ids int32 [n], host arrays)."""
    home = np.ascontiguousarray(home, dtype=np.int32).reshape(-1, 3)
    off = np.ascontiguousarray(off, dtype=np.float64).reshape(-1, 3)
    vel = np.ascontiguousarray(vel, dtype=np.float64).reshape(-1, 3)
    pid = np.ascontiguousarray(pid, dtype=np.int32).reshape(-1)
    n = pid.size
    if not (home.shape[0] == off.shape[0] == vel.shape[0] == n):
        raise ValueError("home, off, vel and pid must describe the same particles")
    _check(h, load_library().lbmpcd_set_particles(h, int(replica), n, home.ctypes.data, off.ctypes.data,
                                                  vel.ctypes.data, pid.ctypes.data))


def lbmpcd_step(h, nsteps: int):
    _check(h, load_library().lbmpcd_step(h, int(nsteps)))


def lbmpcd_step_profiled(h, nsteps: int):
    """Run nsteps with a CUDA event pair around every kernel; returns
    ({phase: milliseconds}, number of kernel launches)."""
    ms = (ctypes.c_double * 6)()
    nl = ctypes.c_longlong(0)
    _check(h, load_library().lbmpcd_step_profiled(h, int(nsteps), ms, ctypes.byref(nl)))
    return dict(zip(("prep", "lb_pull", "particle_pass", "cell_pass", "sort", "closure"), list(ms))), int(nl.value)


def lbmpcd_set_closure(h, theta, interval: int = 1):
    """Load the learned closure's parameters (numpy float32 vector or a
    float32 CUDA tensor) with the network evaluated every ``interval`` steps;
    None unloads them (sampling only)."""
    L = load_library()
    if theta is None:
        _check(h, L.lbmpcd_set_closure(h, None, 0, 0, 1))
    elif hasattr(theta, "data_ptr"):
        t = theta.contiguous()
        _check(h, L.lbmpcd_set_closure(h, ctypes.c_void_p(t.data_ptr()), t.numel(), int(t.is_cuda), int(interval)))
    else:
        arr = np.ascontiguousarray(theta, dtype=np.float32)
        _check(h, L.lbmpcd_set_closure(h, ctypes.c_void_p(arr.ctypes.data), arr.size, 0, int(interval)))


def lbmpcd_field_size(h, replica: int, field: str) -> int:
    n = load_library().lbmpcd_field_size(h, int(replica), FIELDS[field])
    if n < 0:
        _check(h, int(n))
    return int(n)


def lbmpcd_get_fields(h, replica: int, field: str, out=None):
    """Copy a field out; ``out`` may be a numpy array (host) or a torch CUDA tensor
    of the right size and dtype (float64 / int32); returns the filled array."""
    n = lbmpcd_field_size(h, replica, field)
    is_int = field in INT_FIELDS
    if out is None:
        out = np.empty(n, dtype=np.int32 if is_int else np.float64)
    if isinstance(out, np.ndarray):
        assert out.flags.c_contiguous and out.size == n
        ptr, nbytes, on_dev = out.ctypes.data, out.nbytes, 0
    else:   # torch tensor
        assert out.is_contiguous() and out.numel() == n
        ptr, nbytes, on_dev = out.data_ptr(), out.numel() * out.element_size(), int(out.is_cuda)
    _check(h, load_library().lbmpcd_get_fields(h, int(replica), FIELDS[field], ctypes.c_void_p(ptr),
                                               nbytes, on_dev))
    return out


def lbmpcd_set_state(h, replica: int, field: str, value):
    is_int = field in INT_FIELDS
    if isinstance(value, np.ndarray) or not hasattr(value, "data_ptr"):
        arr = np.ascontiguousarray(value, dtype=np.int32 if is_int else np.float64).ravel()
        ptr, nbytes, on_dev = arr.ctypes.data, arr.nbytes, 0
    else:
        arr = value.contiguous()
        ptr, nbytes, on_dev = arr.data_ptr(), arr.numel() * arr.element_size(), int(arr.is_cuda)
    _check(h, load_library().lbmpcd_set_state(h, int(replica), FIELDS[field], ctypes.c_void_p(ptr),
                                              nbytes, on_dev))


def _raw_buffer(buf):
    """(address, bytes, on_device) of a contiguous numpy array or torch tensor."""
    if isinstance(buf, np.ndarray):
        if not buf.flags.c_contiguous:
            raise ValueError("buffer must be contiguous")
        return buf.ctypes.data, buf.nbytes, 0
    if not buf.is_contiguous():
        raise ValueError("buffer must be contiguous")
    return buf.data_ptr(), buf.numel() * buf.element_size(), int(buf.is_cuda)


def lbmpcd_tc_gemm_bf16(A, B, C, alpha=1.0, beta=0.0, err=None, stream=None):
    """C = alpha A B^T + beta C on the tensor cores; A (M, K) and B (N, K) bf16
    CUDA tensors, C (M, N) float32 CUDA tensor, err an int32 CUDA tensor."""
    M, K = A.shape
    N = B.shape[0]
    sptr = getattr(stream, "cuda_stream", stream) or 0
    rc = load_library().lbmpcd_tc_gemm_bf16(ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(B.data_ptr()),
                                             ctypes.c_void_p(C.data_ptr()), M, N, K, float(alpha), float(beta),
                                             ctypes.c_void_p(err.data_ptr()), ctypes.c_void_p(int(sptr)))
    if rc != 0:
        raise LbmpcdError(rc, "tc_gemm_bf16")


NET_STATIC_MAX_PATCHES = 8   # LBMPCD_NET_STATIC_MAX_PATCHES


def _check_net_tensor(name, t, shape):
    """A float32, contiguous CUDA tensor of the given shape (the C side only
    sees its address, so a short or strided buffer would be read out of
    bounds on the device)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{name}: expected a torch tensor")
    if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous float32 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: expected shape {tuple(shape)}, got {tuple(t.shape)}")


def lbmpcd_net_forward_noalloc(theta, x, y, stream=None):
    """Network forward with the library's static scratch (no allocation):
    theta (n_params,) float32, x (P, 16, 16, 24) and y (P, 16, 16, 3) float32
    contiguous CUDA tensors on the current device, P <= NET_STATIC_MAX_PATCHES
    (a larger P is passed on so that the library reports ERR_CAPACITY).
    Raises ValueError for a tensor of the wrong type, shape or device."""
    import torch
    if not isinstance(x, torch.Tensor) or x.dim() != 4:
        raise ValueError("x: expected a (P, 16, 16, 24) tensor")
    P = int(x.shape[0])
    _check_net_tensor("theta", theta, (int(load_library().lbmpcd_net_num_params()),))
    _check_net_tensor("x", x, (P, 16, 16, 24))
    _check_net_tensor("y", y, (P, 16, 16, 3))
    cur = torch.cuda.current_device()
    for name, t in (("theta", theta), ("x", x), ("y", y)):
        if t.device.index != cur:
            raise ValueError(f"{name}: on cuda:{t.device.index}, the current device is cuda:{cur}")
    sptr = getattr(stream, "cuda_stream", stream) or 0
    rc = load_library().lbmpcd_net_forward_noalloc(ctypes.c_void_p(theta.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                                    int(x.shape[0]), ctypes.c_void_p(y.data_ptr()),
                                                    ctypes.c_void_p(int(sptr)))
    if rc != 0:
        raise LbmpcdError(rc, "net_forward_noalloc")


def lbmpcd_destroy(h):
    if h:
        load_library().lbmpcd_destroy(h)


class Net:
    """The learned closure network (device tensors are torch CUDA tensors)."""

    def __init__(self, max_patches: int, stream=None):
        L = load_library()
        h = ctypes.c_void_p()
        sptr = getattr(stream, "cuda_stream", stream) or 0
        rc = L.lbmpcd_net_create(int(max_patches), ctypes.c_void_p(int(sptr)), ctypes.byref(h))
        if rc != 0:
            raise LbmpcdError(rc, "net_create")
        self._h = h
        self.n = int(L.lbmpcd_net_num_params())

    def _rc(self, rc, what):
        if rc != 0:
            raise LbmpcdError(rc, what)

    def set_params(self, theta):
        arr = np.ascontiguousarray(theta, dtype=np.float32)
        self._rc(load_library().lbmpcd_net_set_params(self._h, arr.ctypes.data, arr.size, 0), "set_params")

    def get_params(self, which: int = 0) -> np.ndarray:
        out = np.empty(self.n, dtype=np.float32)
        self._rc(load_library().lbmpcd_net_get_params(self._h, out.ctypes.data, out.size, which, 0), "get_params")
        return out

    def forward(self, x, y):
        P = x.shape[0]
        self._rc(load_library().lbmpcd_net_forward(self._h, ctypes.c_void_p(x.data_ptr()), P,
                                                   ctypes.c_void_p(y.data_ptr())), "forward")

    def backward(self, x, t) -> float:
        loss = ctypes.c_float()
        self._rc(load_library().lbmpcd_net_backward(self._h, ctypes.c_void_p(x.data_ptr()),
                                                    ctypes.c_void_p(t.data_ptr()), x.shape[0],
                                                    ctypes.byref(loss)), "backward")
        return float(loss.value)

    def train_step(self, x, t, lr: float) -> float:
        loss = ctypes.c_float()
        self._rc(load_library().lbmpcd_net_train_step(self._h, ctypes.c_void_p(x.data_ptr()),
                                                      ctypes.c_void_p(t.data_ptr()), x.shape[0], float(lr),
                                                      ctypes.byref(loss)), "train_step")
        return float(loss.value)

    def close(self):
        if getattr(self, "_h", None):
            load_library().lbmpcd_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Lbmpcd:
    """Owning wrapper of one handle (all replicas)."""

    def __init__(self, params, stream=None):
        self.params = list(params) if isinstance(params, (list, tuple)) else [params]
        self._h = lbmpcd_create(self.params, stream=stream)

    def set_region(self, replica: int, x0: int, x1: int):
        p = self.params[replica]
        lbmpcd_set_region(self._h, replica, (x0, 0, 0), (x1, p["ny"], p.get("nz", 1)))

    def set_region_piece(self, replica: int, x0: int, x1: int, own, keep):
        p = self.params[replica]
        lbmpcd_set_region_piece(self._h, replica, (x0, 0, 0), (x1, p["ny"], p.get("nz", 1)), own, keep)

    def set_particles(self, replica: int, home, off, vel, pid):
        lbmpcd_set_particles(self._h, replica, home, off, vel, pid)

    def set_strip(self, replica: int, y1: int):
        """Near-wall strip (Sec. 3.3): all columns, LB rows [1, y1), coupling
        buffer along y1."""
        p = self.params[replica]
        lbmpcd_set_region(self._h, replica, (0, 0, 0), (p["nx"], y1, p.get("nz", 1)))

    def step(self, n: int = 1):
        lbmpcd_step(self._h, n)

    def step_profiled(self, n: int):
        return lbmpcd_step_profiled(self._h, n)

    def set_closure(self, theta, interval: int = 1):
        lbmpcd_set_closure(self._h, theta, interval)

    def set_launch_mode(self, mode: int, blocks_per_sm: int = 0, lb_tma: bool = False, serial: bool = False):
        """0: per-kernel launches in 64-step graphs (overlapped unless serial;
        blocks_per_sm caps the particle pass there); 1: one persistent kernel
        per chunk (blocks_per_sm: its blocks per SM).  lb_tma: TMA-staged LB
        rows (D2Q9 binary32)."""
        flags = (LAUNCH_LB_TMA if lb_tma else 0) | (LAUNCH_SERIAL if serial else 0)
        _check(self._h, load_library().lbmpcd_set_launch_mode(self._h, int(mode), int(blocks_per_sm), flags))

    def set_wait_limit(self, polls: int = 0):
        """Polls before a grid-barrier wait of the persistent form gives up
        (0: the library's default); lbmpcd_step then returns ERR_TIMEOUT."""
        _check(self._h, load_library().lbmpcd_set_wait_limit(self._h, int(polls)))

    def autotune(self, steps: int = 256) -> dict:
        """Time the launch forms on a copy of this handle and keep the fastest."""
        out = (ctypes.c_int * 5)()
        _check(self._h, load_library().lbmpcd_autotune(self._h, int(steps), out))
        return dict(mode=out[0], blocks_per_sm=out[1], lb_nodes_per_thread=out[2], lb_tma=bool(out[3] & LAUNCH_LB_TMA),
                    serial=bool(out[3] & LAUNCH_SERIAL), candidates=out[4])

    def get(self, field: str, replica: int = 0, out=None):
        return lbmpcd_get_fields(self._h, replica, field, out)

    def population_bytes(self) -> int:
        return int(load_library().lbmpcd_population_bytes(self._h))

    def column_bytes(self, ncols: int, replica: int = 0) -> int:
        p = self.params[replica]
        q = int(p.get("lattice", 9))
        return q * int(p.get("nz", 1)) * int(p["ny"]) * int(ncols) * self.population_bytes()

    def get_columns(self, x: int, ncols: int, out, replica: int = 0):
        """Raw populations of LB columns [x, x + ncols) into ``out`` (a
        contiguous numpy array or torch tensor of column_bytes(ncols) bytes,
        any dtype); returns out."""
        ptr, nbytes, on_dev = _raw_buffer(out)
        if nbytes != self.column_bytes(ncols, replica):
            raise ValueError("column buffer has the wrong size")
        _check(self._h, load_library().lbmpcd_get_columns(self._h, int(replica), int(x), int(ncols),
                                                          ctypes.c_void_p(ptr), on_dev))
        return out

    def set_columns(self, x: int, ncols: int, src, replica: int = 0):
        """Load raw populations of LB columns [x, x + ncols) from ``src``
        (layout and size of get_columns)."""
        ptr, nbytes, on_dev = _raw_buffer(src)
        if nbytes != self.column_bytes(ncols, replica):
            raise ValueError("column buffer has the wrong size")
        _check(self._h, load_library().lbmpcd_set_columns(self._h, int(replica), int(x), int(ncols),
                                                          ctypes.c_void_p(ptr), on_dev))

    def set(self, field: str, value, replica: int = 0):
        lbmpcd_set_state(self._h, replica, field, value)

    def close(self):
        if getattr(self, "_h", None):
            lbmpcd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
