"""GB300 imaginary-time FDTD solver for the 3-D Schroedinger equation.

Python binding of the C ABI in ``include/fdtd.h`` (library ``libfdtd.so``,
hand-written sm_103a CUDA).  This module only marshals arguments: every step
of the method runs in the library's kernels.  PyTorch supplies the device
workspace and the CUDA stream.  Importing the package raises if the CUDA
library has not been built; there is no CPU fallback.

Method (Strickland & Yager-Elorriaga, arXiv:0904.0939):
  * Eq. updateeq -- imaginary-time update psi <- A psi + (B dtau / 2m) sum D.PsiHat
  * Eq. energysum -- energy functional, <r^2>, binding energy (Eq. bindingenergy)
  * Sec. IV -- symmetric / antisymmetric initial conditions (S_i, A_i)
  * Sec. VI -- multi-resolution bootstrap (trilinear transfer to 2N)
  * gradients of E and <r^2> w.r.t. V through the unrolled evolution
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# FDTD_LIB selects another build of the library, e.g. the bounds-checking
# libfdtd_checked.so (python paper_0904_0939_gb300/_build.py --checked)
LIB_PATH = os.environ.get("FDTD_LIB") or os.path.join(_HERE, "libfdtd.so")

OK, NOT_CONVERGED = 0, 1
ERR_INVALID_ARG, ERR_UNSTABLE_DT, ERR_NONFINITE, ERR_CUDA = -1, -2, -3, -4
ERR_TIMEOUT, ERR_SHAPE, ERR_WORKSPACE, ERR_STATE, ERR_IO = -5, -6, -7, -8, -9
F64, F32, BF16 = 0, 1, 2
C64, C32 = 3, 4  # complex potentials: interleaved (re, im) pairs of doubles / floats
MEM_HOST, MEM_DEVICE = 0, 1
DIST_UNIFORM, DIST_GAUSSIAN = 0, 1
PARITY_NONE, PARITY_S, PARITY_A = 0, 1, 2


def parity_mask(px: int = 0, py: int = 0, pz: int = 0) -> int:
    """Two bits per axis: 0 none, 1 S_i, 2 A_i (Sec. IV)."""
    return px | (py << 2) | (pz << 4)


class FdtdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"fdtd error {code}: {msg}")
        self.code = code


class LatticeDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("precision", ctypes.c_int32), ("length", ctypes.c_double),
                ("mass", ctypes.c_double), ("dtau", ctypes.c_double), ("v_inf", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("check_every", ctypes.c_int32), ("tol_relative", ctypes.c_int32), ("tol", ctypes.c_double),
                ("temporal_depth", ctypes.c_int32), ("backward_steps", ctypes.c_int32),
                ("batched", ctypes.c_int32), ("reimpose_parity", ctypes.c_int32),
                ("stencil_kernel", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("zchunk", ctypes.c_int32), ("wait_limit_us", ctypes.c_int32),
                ("snapshots", ctypes.c_int32), ("graphs", ctypes.c_int32), ("boundary", ctypes.c_int32),
                ("tile_x", ctypes.c_int32), ("tile_y", ctypes.c_int32)]


class Obs(ctypes.Structure):
    _fields_ = [("energy", ctypes.c_double), ("binding_energy", ctypes.c_double), ("norm", ctypes.c_double),
                ("r2", ctypes.c_double), ("r_rms", ctypes.c_double), ("v_expect", ctypes.c_double),
                ("delta_e", ctypes.c_double), ("energy_imag", ctypes.c_double), ("steps", ctypes.c_int64),
                ("converged", ctypes.c_int32), ("checks", ctypes.c_int32)]

    def to_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("stencil_launches", ctypes.c_int64),
                ("stencil_ms", ctypes.c_double), ("stencil_site_updates", ctypes.c_int64),
                ("stencil_bytes", ctypes.c_double), ("graph_launches", ctypes.c_int64),
                ("stencil_timed_launches", ctypes.c_int64)]


EXPORTED = ["fdtd_default_options", "fdtd_workspace_size", "fdtd_create", "fdtd_destroy", "fdtd_last_error",
            "fdtd_set_potential", "fdtd_set_potential_async", "fdtd_init_symmetric", "fdtd_set_psi", "fdtd_get_psi", "fdtd_evolve",
            "fdtd_last_check", "fdtd_observables", "fdtd_upsample", "fdtd_backward", "fdtd_get_stats",
            "fdtd_reset_stats", "fdtd_set_profiling", "fdtd_observables_noalloc", "fdtd_tuned_config",
            "fdtd_tuned_kernel",
            "fdtd_check_history", "fdtd_save_psi", "fdtd_load_psi", "fdtd_bounds_violations",
            "fdtd_snapshot_save", "fdtd_snapshot_load", "fdtd_project_out", "fdtd_combine",
            "fdtd_slab_workspace_size", "fdtd_slab_create", "fdtd_slab_destroy", "fdtd_slab_steps",
            "fdtd_slab_steps_range", "fdtd_slab_sums",
            "fdtd_slab_scale", "fdtd_check_sums"]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, u64, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "fdtd_default_options": [P(Options)],
        "fdtd_workspace_size": [P(LatticeDesc), i32, P(Options), P(ctypes.c_size_t)],
        "fdtd_create": [P(LatticeDesc), i32, P(Options), vp, ctypes.c_size_t, vp, P(vp)],
        "fdtd_destroy": [vp],
        "fdtd_set_potential": [vp, i32, vp, i32, i32],
        "fdtd_set_potential_async": [vp, i32, vp, i32, i32],
        "fdtd_init_symmetric": [vp, i32, u64, i32, i32],
        "fdtd_set_psi": [vp, i32, vp, i32, i32, i32],
        "fdtd_get_psi": [vp, i32, vp, i32, i32],
        "fdtd_evolve": [vp, i64, P(i64)],
        "fdtd_last_check": [vp, i32, P(Obs)],
        "fdtd_observables": [vp, i32, P(Obs)],
        "fdtd_upsample": [vp, i32, vp, i32],
        "fdtd_backward": [vp, i32, i64, d, d, vp, i32, i32, P(Obs)],
        "fdtd_get_stats": [vp, P(Stats)],
        "fdtd_reset_stats": [vp],
        "fdtd_set_profiling": [vp, i32],
        "fdtd_tuned_config": [vp, i32, P(ctypes.c_int), P(ctypes.c_int)],
        "fdtd_tuned_kernel": [vp, i32, P(ctypes.c_int), P(ctypes.c_int)],
        "fdtd_check_history": [vp, i32, P(d), i32, P(ctypes.c_int)],
        "fdtd_save_psi": [vp, i32, ctypes.c_char_p],
        "fdtd_bounds_violations": [vp, P(i64)],
        "fdtd_load_psi": [vp, i32, ctypes.c_char_p],
        "fdtd_snapshot_save": [vp, i32, i32],
        "fdtd_snapshot_load": [vp, i32, i32],
        "fdtd_project_out": [vp, i32, P(ctypes.c_int), i32],
        "fdtd_combine": [vp, i32, P(ctypes.c_int), P(ctypes.c_double), i32],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.fdtd_observables_noalloc.argtypes = [vp, vp, i32, i32, d, d, vp, vp]
    lib.fdtd_observables_noalloc.restype = ctypes.c_int
    lib.fdtd_last_error.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    lib.fdtd_last_error.restype = i32
    return lib


lib = _load()


def default_options(**kw) -> Options:
    o = Options()
    lib.fdtd_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@dataclass
class Lattice:
    """One lattice: n sites per axis, box length, storage precision."""
    n: int
    length: float
    precision: int = F32
    mass: float = 1.0
    dtau: float = 0.0
    v_inf: float = 0.0

    def desc(self) -> LatticeDesc:
        return LatticeDesc(self.n, self.precision, self.length, self.mass, self.dtau, self.v_inf)

    @property
    def a(self) -> float:
        return self.length / self.n

    @property
    def tau_step(self) -> float:
        return self.dtau if self.dtau > 0 else self.a * self.a / 4.0


def last_error(handle=None) -> str:
    """The library's message for the last error on `handle` (None: handle creation)."""
    size = lib.fdtd_last_error(handle, None, 0)
    buf = ctypes.create_string_buffer(size + 1)
    lib.fdtd_last_error(handle, buf, size + 1)
    return buf.value.decode(errors="replace")


def _check(rc: int, handle=None, allow_soft: bool = False) -> int:
    if rc < 0 or (rc > 0 and not allow_soft):
        raise FdtdError(rc, last_error(handle))
    return rc


def _buffer(arr, want_dtype=None):
    """(pointer, dtype code, mem kind, keepalive) for a numpy array or torch
    tensor: float64 / float32 are passed as they are, complex128 / complex64
    as interleaved pairs (C64 / C32), anything else is converted to float64."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(arr, torch.Tensor):
        t = arr.contiguous()
        codes = {torch.float64: F64, torch.float32: F32, torch.complex128: C64, torch.complex64: C32}
        if t.dtype not in codes:
            t = t.double()
        return ctypes.c_void_p(t.data_ptr()), codes[t.dtype], (MEM_DEVICE if t.is_cuda else MEM_HOST), t
    a = np.ascontiguousarray(arr)
    codes = {np.dtype(np.float64): F64, np.dtype(np.float32): F32, np.dtype(np.complex128): C64,
             np.dtype(np.complex64): C32}
    if a.dtype not in codes:
        a = a.astype(np.float64)
    return ctypes.c_void_p(a.ctypes.data), codes[a.dtype], MEM_HOST, a


class Solver:
    """A handle on the C library for one or more lattices.

    The workspace is one torch uint8 CUDA tensor of fdtd_workspace_size()
    bytes; all work runs on `stream` (default: torch's current stream)."""

    def __init__(self, lattices, options: Options | None = None, device=None, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise FdtdError(ERR_CUDA, "no CUDA device: the FDTD solver runs on the GPU only")
        self.lattices = list(lattices) if isinstance(lattices, (list, tuple)) else [lattices]
        self.options = options if options is not None else default_options()
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        arr = (LatticeDesc * len(self.lattices))(*[l.desc() for l in self.lattices])
        self._descs = arr
        size = ctypes.c_size_t()
        _check(lib.fdtd_workspace_size(arr, len(self.lattices), ctypes.byref(self.options), ctypes.byref(size)))
        self.workspace_bytes = size.value
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.workspace = torch.empty(size.value, dtype=torch.uint8, device=self.device)
            h = ctypes.c_void_p()
            _check(lib.fdtd_create(arr, len(self.lattices), ctypes.byref(self.options),
                                   ctypes.c_void_p(self.workspace.data_ptr()), size.value,
                                   ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.handle = h
        self._in_flight = []  # buffers of potentials enqueued without waiting

    def close(self):
        if getattr(self, "handle", None):
            lib.fdtd_destroy(self.handle)  # waits for the stream
            self.handle = None
            self._in_flight = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ctx(self):
        import torch

        return torch.cuda.device(self.device)

    def _sized(self, arr, lat: int, what: str):
        """The C ABI reads or writes exactly n^3 elements: check the buffer."""
        if not 0 <= lat < len(self.lattices):
            raise FdtdError(ERR_INVALID_ARG, f"{what}: lattice index {lat} out of range")
        n = self.lattices[lat].n
        size = arr.numel() if hasattr(arr, "numel") else np.asarray(arr).size
        if size != n**3:
            raise FdtdError(ERR_SHAPE, f"{what}: expected {n}^3 = {n**3} values, got {size}")
        return arr

    # --- calls ---------------------------------------------------------------
    def set_potential(self, v, lat: int = 0, wait: bool = True):
        """Load V.  wait=False enqueues the copy and its checks on the
        handle's stream and returns (fdtd_set_potential_async): v is kept
        referenced until the next call that waits for the stream, which
        also reports the checks (host tensors should be pinned)."""
        ptr, code, mem, keep = _buffer(self._sized(v, lat, "set_potential"))
        with self._ctx():
            if wait:
                _check(lib.fdtd_set_potential(self.handle, lat, ptr, code, mem), self.handle)
                self._in_flight.clear()
            else:
                _check(lib.fdtd_set_potential_async(self.handle, lat, ptr, code, mem), self.handle)
                self._in_flight.append((v, keep))

    def init_symmetric(self, seed: int, mask: int = 0, lat: int = 0, dist: int = DIST_UNIFORM):
        with self._ctx():
            _check(lib.fdtd_init_symmetric(self.handle, lat, seed, mask, dist), self.handle)

    def set_psi(self, psi, lat: int = 0, mask: int = 0):
        ptr, code, mem, keep = _buffer(self._sized(psi, lat, "set_psi"))
        with self._ctx():
            _check(lib.fdtd_set_psi(self.handle, lat, ptr, code, mem, mask), self.handle)

    def get_psi(self, lat: int = 0, dtype=None, out=None):
        """psi as a dense (n, n, n) array [z][y][x] (float64 by default,
        complex128 for complex lattices); `out` may be a CUDA tensor."""
        n = self.lattices[lat].n
        if out is None:
            if dtype is None:
                dtype = np.complex128 if self.lattices[lat].precision in (C64, C32) else np.float64
            out = np.empty((n, n, n), dtype=dtype)
        ptr, code, mem, keep = _buffer(self._sized(out, lat, "get_psi"))
        with self._ctx():
            _check(lib.fdtd_get_psi(self.handle, lat, ptr, code, mem), self.handle)
        return out

    def evolve(self, max_steps: int) -> tuple[int, bool]:
        """Run until every lattice converges or max_steps; returns (steps, converged)."""
        done = ctypes.c_int64()
        with self._ctx():
            rc = _check(lib.fdtd_evolve(self.handle, max_steps, ctypes.byref(done)), self.handle, allow_soft=True)
        self._in_flight.clear()  # the call waited for the stream
        return done.value, rc == OK

    def last_check(self, lat: int = 0) -> dict:
        o = Obs()
        with self._ctx():
            _check(lib.fdtd_last_check(self.handle, lat, ctypes.byref(o)), self.handle)
        return o.to_dict()

    def observables(self, lat: int = 0) -> dict:
        o = Obs()
        with self._ctx():
            _check(lib.fdtd_observables(self.handle, lat, ctypes.byref(o)), self.handle)
        self._in_flight.clear()
        return o.to_dict()

    def upsample_from(self, src: "Solver", lat_src: int = 0, lat: int = 0):
        with self._ctx():
            _check(lib.fdtd_upsample(src.handle, lat_src, self.handle, lat), self.handle)
        self._in_flight.clear()

    def backward(self, T: int, w_e: float = 1.0, w_r: float = 0.0, lat: int = 0, out=None):
        """dL/dV for L = w_e E + w_r <r^2> after T steps; returns (gV, obs)."""
        n = self.lattices[lat].n
        if out is None:
            out = np.empty((n, n, n), dtype=np.float64)
        ptr, code, mem, keep = _buffer(self._sized(out, lat, "backward"))
        o = Obs()
        with self._ctx():
            _check(lib.fdtd_backward(self.handle, lat, T, w_e, w_r, ptr, code, mem, ctypes.byref(o)), self.handle)
        self._in_flight.clear()
        return out, o.to_dict()

    # --- snapshots (Sec. III) and combinations (Sec. VI) -----------------------
    def snapshot_save(self, slot: int, lat: int = 0):
        with self._ctx():
            _check(lib.fdtd_snapshot_save(self.handle, lat, slot), self.handle)

    def snapshot_load(self, slot: int, lat: int = 0):
        with self._ctx():
            _check(lib.fdtd_snapshot_load(self.handle, lat, slot), self.handle)

    def project_out(self, slots, lat: int = 0):
        """psi <- psi minus its components along the snapshot slots, renormalised."""
        arr = (ctypes.c_int * max(1, len(slots)))(*slots)
        with self._ctx():
            _check(lib.fdtd_project_out(self.handle, lat, arr, len(slots)), self.handle)
        self._in_flight.clear()

    def combine(self, slots, weights, lat: int = 0):
        """psi <- sum_k weights[k] * slot_k, renormalised."""
        a = (ctypes.c_int * len(slots))(*slots)
        w = (ctypes.c_double * len(weights))(*weights)
        with self._ctx():
            _check(lib.fdtd_combine(self.handle, lat, a, w, len(slots)), self.handle)
        self._in_flight.clear()

    def bounds_violations(self) -> int:
        """Out-of-allocation accesses counted by a bounds-checking build."""
        c = ctypes.c_int64()
        _check(lib.fdtd_bounds_violations(self.handle, ctypes.byref(c)), self.handle)
        return c.value

    def save(self, path, lat: int = 0):
        """Write psi of lattice `lat` to a checkpoint file (fdtd_save_psi)."""
        with self._ctx():
            _check(lib.fdtd_save_psi(self.handle, lat, os.fsencode(path)), self.handle)

    def load(self, path, lat: int = 0):
        """Start lattice `lat` from a checkpoint file, at the same or a
        2^k-times coarser resolution (fdtd_load_psi)."""
        with self._ctx():
            _check(lib.fdtd_load_psi(self.handle, lat, os.fsencode(path)), self.handle)

    HISTORY_FIELDS = ("t", "E", "E_b", "norm", "r2", "V", "delta_e", "S0")

    def history(self, lat: int = 0, cap: int = 4096) -> np.ndarray:
        """Per-check records of the last evolve, oldest first: an array of
        shape (k, 8) with columns HISTORY_FIELDS."""
        buf = np.zeros((cap, 8), dtype=np.float64)
        count = ctypes.c_int()
        with self._ctx():
            _check(lib.fdtd_check_history(self.handle, lat, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), cap,
                                          ctypes.byref(count)), self.handle)
        return buf[: min(count.value, cap, 4096)].copy()

    def tuned_config(self, lat: int = 0) -> tuple[int, int]:
        """(temporal depth, span in tile planes per block) the stencil uses for
        lattice `lat`; span 0 means the one-step z-marching kernel (no TMA)."""
        d, z = ctypes.c_int(), ctypes.c_int()
        with self._ctx():
            _check(lib.fdtd_tuned_config(self.handle, lat, ctypes.byref(d), ctypes.byref(z)), self.handle)
        self._in_flight.clear()
        return d.value, z.value

    def tuned_kernel(self, lat: int = 0) -> tuple[int, int]:
        """(tile width in x, tile height in y) of the TMA stencil for lattice
        `lat`; (0, 0) when the one-step kernel is in use."""
        t, r = ctypes.c_int(), ctypes.c_int()
        with self._ctx():
            _check(lib.fdtd_tuned_kernel(self.handle, lat, ctypes.byref(t), ctypes.byref(r)), self.handle)
        self._in_flight.clear()
        return t.value, r.value

    def stats(self) -> dict:
        s = Stats()
        _check(lib.fdtd_get_stats(self.handle, ctypes.byref(s)), self.handle)
        return {f: getattr(s, f) for f, _ in s._fields_}

    def reset_stats(self):
        _check(lib.fdtd_reset_stats(self.handle), self.handle)

    def set_profiling(self, on: bool):
        _check(lib.fdtd_set_profiling(self.handle, int(bool(on))), self.handle)


def solve(v, n: int, length: float, precision: int = F32, mask: int = 0, seed: int = 904939,
          max_steps: int = 1_000_000, options: Options | None = None, v_inf: float = 0.0):
    """Ground state of one sector from a random start (Secs. III-V)."""
    s = Solver(Lattice(n, length, precision, v_inf=v_inf), options)
    s.set_potential(v)
    s.init_symmetric(seed, mask)
    steps, conv = s.evolve(max_steps)
    return s, s.last_check()


def multires(levels, potentials, mask: int = 0, seed: int = 904939, options: Options | None = None,
             max_steps: int = 1_000_000, v_inf=0.0):
    """Multi-resolution bootstrap (Sec. VI): solve on levels[0] from a random
    start, then transfer each converged field to the next (2N, same L)
    lattice and continue.  Returns the list of (solver, last_check)."""
    out = []
    prev = None
    for i, (lat, v) in enumerate(zip(levels, potentials)):
        s = Solver(lat, options)
        s.set_potential(v)
        if prev is None:
            s.init_symmetric(seed, mask)
        else:
            s.upsample_from(prev)
        s.evolve(max_steps)
        out.append((s, s.last_check()))
        prev = s
    return out


def observables_noalloc(psi, v, length: float, mass: float = 1.0, out=None, stream=None):
    """Lattice sums of a caller-held CUDA field without any allocation in the
    library (fdtd_observables_noalloc).  psi and v are contiguous CUDA
    tensors of n^3 values on one device, both float64 or both float32; out
    is a contiguous float64 CUDA tensor of at least 8 values on that device
    (allocated here if not given).  Returns out:
    [E, <r^2>, <V>, sum psi^2 a^3, S0, SH, Sr, SV].

    Everything the C entry cannot check on a raw pointer (dtype, device,
    layout, length of out) is checked here before the call; the kernels are
    enqueued on `stream` (default: the current stream of psi's device) and
    the call does not synchronise."""
    import torch

    for name, t in (("psi", psi), ("v", v)):
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise FdtdError(ERR_INVALID_ARG, f"observables_noalloc: {name} must be a CUDA tensor")
        if t.dtype not in (torch.float32, torch.float64):
            raise FdtdError(ERR_INVALID_ARG, f"observables_noalloc: {name} must be float32 or float64, not {t.dtype}")
        if not t.is_contiguous():
            raise FdtdError(ERR_INVALID_ARG, f"observables_noalloc: {name} must be contiguous")
    if psi.dtype != v.dtype or psi.device != v.device:
        raise FdtdError(ERR_INVALID_ARG, "observables_noalloc: psi and v need one dtype and one device")
    n = round(psi.numel() ** (1.0 / 3.0))
    if n < 1 or psi.numel() != n**3 or v.numel() != n**3:
        raise FdtdError(ERR_SHAPE, "observables_noalloc: psi and v must hold n^3 values each")
    if out is None:
        out = torch.empty(8, dtype=torch.float64, device=psi.device)
    elif (not isinstance(out, torch.Tensor) or out.dtype != torch.float64 or out.device != psi.device
          or not out.is_contiguous() or out.numel() < 8):
        raise FdtdError(ERR_INVALID_ARG,
                        "observables_noalloc: out must be a contiguous float64 tensor of >= 8 values on psi's device")
    code = F64 if psi.dtype == torch.float64 else F32
    st = stream if stream is not None else torch.cuda.current_stream(psi.device)
    with torch.cuda.device(psi.device):
        _check(lib.fdtd_observables_noalloc(ctypes.c_void_p(psi.data_ptr()), ctypes.c_void_p(v.data_ptr()), code, n,
                                            float(length), float(mass), ctypes.c_void_p(out.data_ptr()),
                                            ctypes.c_void_p(st.cuda_stream)))
    if st != torch.cuda.current_stream(psi.device):
        # the kernels read psi and v (and write out) later on another stream:
        # keep the caching allocator from handing their memory out meanwhile
        for t in (psi, v, out):
            t.record_stream(st)
    return out


def energy_fn():
    """The torch.autograd.Function (E, <r^2>) = F(V) of T unrolled update
    steps (Eq. updateeq) with the checks of fdtd_evolve, whose backward is
    fdtd_backward (sqrt(T) checkpointing, the adjoint step).

    ``EnergyFn.apply(v, solver, T, psi0=None, seed=0, mask=0)``:
      v       the potential, n^3 values (any float tensor; on the GPU or the
              host); V_theta built from parameters theta in torch gives
              dL/dtheta through torch's own chain rule
      solver  a Solver of one lattice created with options tol <= 0 (the
              forward must run exactly T steps: a tolerance would stop it at
              convergence, and the gradient would belong to another T) and
              backward_steps >= T
      psi0    the start field (n^3 values, e.g. the oscillator Gaussian);
              None draws the seeded symmetric random start (seed, mask)
      mask    the symmetry mask imposed on the start and at every check
    Returns two float64 scalars on v's device: E and <r^2> at step T."""
    import torch

    class EnergyFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, v, solver, T, psi0=None, seed=0, mask=0):
            T = int(T)
            if len(solver.lattices) != 1:
                raise FdtdError(ERR_INVALID_ARG, "EnergyFn: the solver must hold exactly one lattice")
            if T < 1:
                raise FdtdError(ERR_INVALID_ARG, "EnergyFn: T must be >= 1")
            if solver.options.tol > 0:
                raise FdtdError(ERR_INVALID_ARG, "EnergyFn: the solver needs options.tol <= 0 so that the forward "
                                "runs exactly T steps (a tolerance would end it early at convergence)")
            if solver.options.batched:
                raise FdtdError(ERR_INVALID_ARG, "EnergyFn: batched handles have no backward pass")
            if solver.options.backward_steps < T:
                raise FdtdError(ERR_WORKSPACE, f"EnergyFn: options.backward_steps = {solver.options.backward_steps} "
                                f"< T = {T}: create the solver with backward_steps >= T")
            solver.set_potential(v.detach())
            if psi0 is not None:
                solver.set_psi(psi0.detach() if isinstance(psi0, torch.Tensor) else psi0, mask=mask)
            else:
                solver.init_symmetric(seed, mask)
            steps, _ = solver.evolve(T)
            o = solver.last_check()
            if steps != T or o["steps"] != T:
                raise FdtdError(ERR_STATE, f"EnergyFn: the forward ran {steps} steps, not T = {T}")
            ctx.solver, ctx.T = solver, T
            ctx.shape, ctx.dtype, ctx.device = v.shape, v.dtype, v.device
            return (torch.tensor(o["energy"], dtype=torch.float64, device=v.device),
                    torch.tensor(o["r2"], dtype=torch.float64, device=v.device))

        @staticmethod
        def backward(ctx, g_e, g_r):
            dev = ctx.device if ctx.device.type == "cuda" else ctx.solver.device
            out = torch.empty(ctx.shape, dtype=torch.float64, device=dev)
            # the loss weights are the incoming gradients of the two outputs
            ctx.solver.backward(ctx.T, float(g_e), float(g_r), out=out)
            return out.to(device=ctx.device, dtype=ctx.dtype), None, None, None, None, None

    return EnergyFn
