"""Plain FP64 CPU oracle of the coupled LB-MPCD step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and it
shares no code with the CUDA path: the arithmetic lives in ``oracle.c`` and is
reached here through ctypes.

The oracle follows the paper (Montessori et al., coupled lattice
Boltzmann-multiparticle collision method): Eq. 1-2 for the LB step, Eq. 3 for
MPCD streaming, Eq. 4 for the SRD collision, Sec. 2.3 / Algorithms 1-2 for the
coupling; the readings it takes where the paper is silent are listed at the
top of ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_SO_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")   # all-cores timing build
_lib = None
_lib_omp = None

FIELDS = dict(RHO=0, U=1, POPS=2, PART_POS=3, PART_VEL=4, PART_CELL=5, SHIFT=6,
              CELL_COUNT=7, WINDOW_MEAN=8, DIAG=9, PART_HOME=10, CELL_VCM=11, PART_ID=12,
              CLOSURE_IN=13, CLOSURE_TARGET=15, PI=16, CELL_LIST=17)
_INT_FIELDS = {"PART_CELL", "CELL_COUNT", "PART_HOME", "PART_ID", "CELL_LIST"}


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (plain gcc, no FMA contraction),
    the parity oracle, and _build/liboracle_omp.so, the same source with its
    OpenMP pragmas enabled (LB nodes, particle streaming and redraw spread over
    the host cores), used only to time the oracle on all cores."""
    src = os.path.join(_HERE, "oracle.c")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    newest = max(os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h")))
    for so, extra in ((_SO, []), (_SO_OMP, ["-fopenmp"])):
        if force or not os.path.exists(so) or os.path.getmtime(so) < newest:
            tmp = so + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC"] + extra +
                                  ["-shared", "-o", tmp, src, "-lm"])
            os.replace(tmp, so)
    return _SO


class Params(ctypes.Structure):
    _fields_ = [("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("tau", ctypes.c_double), ("force", ctypes.c_double * 3),
                ("refine", ctypes.c_int), ("ppc", ctypes.c_int), ("alpha", ctypes.c_double),
                ("kT", ctypes.c_double), ("mass", ctypes.c_double),
                ("coupling_width", ctypes.c_int), ("precision", ctypes.c_int),
                ("feedback", ctypes.c_int), ("window", ctypes.c_int),
                ("resample_density", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("collision", ctypes.c_int), ("redraw", ctypes.c_int)]


def lib(omp: bool = False):
    """The parity oracle, or with omp=True its all-cores timing build."""
    global _lib, _lib_omp
    if (_lib_omp if omp else _lib) is None:
        build()
        L = ctypes.CDLL(_SO_OMP if omp else _SO)
        vp = ctypes.c_void_p
        L.orc_create.restype = vp
        L.orc_create.argtypes = [ctypes.POINTER(Params), ctypes.c_int]
        L.orc_set_region.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        L.orc_set_strip.argtypes = [vp, ctypes.c_int]
        L.orc_step.argtypes = [vp, ctypes.c_int]
        L.orc_field_size.restype = ctypes.c_long
        L.orc_field_size.argtypes = [vp, ctypes.c_int]
        L.orc_get_field.argtypes = [vp, ctypes.c_int, vp]
        L.orc_set_field.argtypes = [vp, ctypes.c_int, vp]
        L.orc_destroy.argtypes = [vp]
        L.orc_num_particles.restype = ctypes.c_long
        L.orc_num_particles.argtypes = [vp]
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_num_threads.argtypes = []
        L.orc_step_count.restype = ctypes.c_long
        L.orc_step_count.argtypes = [vp]
        L.orc_philox4x32_10.argtypes = [vp, vp, vp]
        L.orc_box_muller.argtypes = [ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
        L.orc_feq.argtypes = [ctypes.c_int, ctypes.c_double, vp, vp]
        L.orc_lattice_table.argtypes = [ctypes.c_int, vp, vp]
        L.orc_bin_offset.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int]
        L.orc_srd_rotate_2d.argtypes = [ctypes.c_double] * 5 + [ctypes.c_int] + \
            [ctypes.POINTER(ctypes.c_double)] * 2
        L.orc_srd_rotate_3d.argtypes = [vp, vp, vp, ctypes.c_double, vp]
        L.orc_random_axis.argtypes = [ctypes.c_uint32, ctypes.c_uint32, vp]
        L.orc_u_fine.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
        L.orc_closure_patches.restype = ctypes.c_long
        L.orc_closure_patches.argtypes = [vp]
        L.orc_closure_impose.argtypes = [vp, vp]
        if omp:
            _lib_omp = L
        else:
            _lib = L
    return _lib_omp if omp else _lib


def num_threads(omp: bool = True) -> int:
    """Threads the oracle's parallel loops use (1 for the parity build)."""
    return int(lib(omp).orc_num_threads())


def make_params(d: dict) -> Params:
    p = Params()
    p.lattice = int(d.get("lattice", 9))
    p.nx, p.ny, p.nz = int(d["nx"]), int(d["ny"]), int(d.get("nz", 1))
    p.tau = float(d["tau"])
    f = list(d.get("force", (0.0, 0.0, 0.0))) + [0.0, 0.0, 0.0]
    p.force = (ctypes.c_double * 3)(*[float(x) for x in f[:3]])
    p.refine = int(d.get("refine", 1))
    p.ppc = int(d.get("ppc", 10))
    p.alpha = float(d.get("alpha", np.deg2rad(130.0)))
    p.kT = float(d.get("kT", 1e-4))
    p.mass = float(d.get("mass", 1.0))
    p.coupling_width = int(d.get("coupling_width", 2))
    p.precision = int(d.get("precision", 0))
    p.feedback = int(d.get("feedback", 0))
    p.window = int(d.get("window", 100))
    p.resample_density = int(d.get("resample_density", 0))
    p.seed = int(d.get("seed", 1))
    p.collision = int(d.get("collision", 0))
    p.redraw = int(d.get("redraw", 0))
    return p


class OracleSim:
    """One replica of the coupled system, stepped by the FP64 oracle."""

    def __init__(self, params: dict, replica: int = 0, omp: bool = False):
        """omp: run on the all-cores timing build (same arithmetic; the
        per-node and per-particle loops are shared out among threads)."""
        self.params = dict(params)
        self._p = make_params(params)
        self._L = lib(omp)
        self._h = self._L.orc_create(ctypes.byref(self._p), int(replica))
        if not self._h:
            raise ValueError("oracle rejected the parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_destroy(h)
            self._h = None

    def set_region(self, x0: int, x1: int) -> None:
        if self._L.orc_set_region(self._h, int(x0), int(x1)) != 0:
            raise ValueError("bad region")

    def set_strip(self, y1: int) -> None:
        """Near-wall strip (Sec. 3.3): all columns, LB rows [1, y1), buffer along y1."""
        if self._L.orc_set_strip(self._h, int(y1)) != 0:
            raise ValueError("bad strip")

    def step(self, n: int = 1) -> None:
        self._L.orc_step(self._h, int(n))

    @property
    def num_particles(self) -> int:
        return int(self._L.orc_num_particles(self._h))

    @property
    def step_count(self) -> int:
        return int(self._L.orc_step_count(self._h))

    def get(self, field: str) -> np.ndarray:
        fid = FIELDS[field]
        n = int(self._L.orc_field_size(self._h, fid))
        out = np.empty(n, dtype=np.int32 if field in _INT_FIELDS else np.float64)
        self._L.orc_get_field(self._h, fid, out.ctypes.data)
        return out

    def u_fine(self, X: int, Y: int, Z: int = 0) -> np.ndarray:
        out = np.zeros(3)
        self._L.orc_u_fine(self._h, int(X), int(Y), int(Z), out.ctypes.data)
        return out

    @property
    def closure_patches(self) -> int:
        return int(self._L.orc_closure_patches(self._h))

    def closure_impose(self, y) -> None:
        """a8 of the learned closure for the step just taken, from the network
        output y of shape (P, 16, 16, 3): the LB update of the next step
        imposes it on the inner-buffer nodes."""
        arr = np.ascontiguousarray(y, dtype=np.float64).ravel()
        if arr.size != self.closure_patches * 768:
            raise ValueError("closure output has the wrong size")
        if self._L.orc_closure_impose(self._h, arr.ctypes.data) != 0:
            raise ValueError("no closure sampling on this replica")

    def set_closure(self, theta, interval: int = 1) -> None:
        """Network parameters for step_with_closure: the network runs on steps
        n0, n0 + interval, ... with n0 = max(7, the current step count)."""
        self._cl = (np.asarray(theta, dtype=np.float64), int(interval), max(7, self.step_count))
        self._cl_y = None

    def step_with_closure(self, n: int = 1) -> None:
        """n steps with the learned closure in the loop: on evaluation steps the
        network (oracle/closure.py, bf16 rounding emulated as on the GPU) maps
        the step's input to the predicted fields; from the first evaluation on
        every step imposes the latest prediction."""
        from . import closure
        theta, K, first = self._cl
        for _ in range(int(n)):
            s = self.step_count
            self.step(1)
            if s >= first and (s - first) % K == 0:
                x = self.get("CLOSURE_IN").reshape(-1, 16, 16, 24)
                self._cl_y, _ = closure.forward(theta, x, emulate_bf16=True)
            if s >= first:
                self.closure_impose(self._cl_y)

    def set(self, field: str, value) -> None:
        fid = FIELDS[field]
        n = int(self._L.orc_field_size(self._h, fid))
        arr = np.ascontiguousarray(value, dtype=np.int32 if field in _INT_FIELDS else np.float64).ravel()
        if arr.size != n:
            raise ValueError(f"{field}: expected {n} elements, got {arr.size}")
        if self._L.orc_set_field(self._h, fid, arr.ctypes.data) != 0:
            raise ValueError(f"{field} cannot be set")


# ---- building blocks, for the pin tests -------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, dtype=np.uint32)
    lib().orc_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def box_muller(w0: int, w1: int):
    z0, z1 = ctypes.c_double(), ctypes.c_double()
    lib().orc_box_muller(int(w0), int(w1), ctypes.byref(z0), ctypes.byref(z1))
    return z0.value, z1.value


def lattice(lat: int):
    c = np.zeros(19 * 3, dtype=np.int32)
    w = np.zeros(19)
    q = lib().orc_lattice_table(int(lat), c.ctypes.data, w.ctypes.data)
    return c[: 3 * q].reshape(q, 3), w[:q]


def feq(lat: int, rho: float, u) -> np.ndarray:
    uu = np.zeros(3)
    uu[: len(u)] = u
    out = np.zeros(19)
    lib().orc_feq(int(lat), float(rho), uu.ctypes.data, out.ctypes.data)
    return out[: (9 if lat == 9 else 19)]


def bin_offset(off: float, sh: float, precision: int) -> int:
    return int(lib().orc_bin_offset(float(off), float(sh), int(precision)))


def srd_rotate_2d(v, vcm, alpha: float, sign: int):
    ox, oy = ctypes.c_double(), ctypes.c_double()
    lib().orc_srd_rotate_2d(float(v[0]), float(v[1]), float(vcm[0]), float(vcm[1]),
                            float(alpha), int(sign), ctypes.byref(ox), ctypes.byref(oy))
    return np.array([ox.value, oy.value])


def srd_rotate_3d(v, vcm, axis, alpha: float) -> np.ndarray:
    a = np.ascontiguousarray(v, dtype=np.float64)
    b = np.ascontiguousarray(vcm, dtype=np.float64)
    c = np.ascontiguousarray(axis, dtype=np.float64)
    out = np.zeros(3)
    lib().orc_srd_rotate_3d(a.ctypes.data, b.ctypes.data, c.ctypes.data, float(alpha), out.ctypes.data)
    return out


def random_axis(w0: int, w1: int) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_random_axis(int(w0), int(w1), out.ctypes.data)
    return out
