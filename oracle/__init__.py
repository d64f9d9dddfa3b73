"""Plain FP64 CPU oracle of the imaginary-time FDTD method (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use this package; the product path
(``paper_0904_0939_gb300``) never imports, loads or calls it, and the two
share no code.  The arithmetic lives in ``fdtd_oracle.c``; this wrapper only
marshals numpy arrays.

Arrays seen from Python are dense interior fields of shape (N, N, N) indexed
[z][y][x] (x fastest, C order, float64).  The C side stores the paper's
padded (N+2)^3 lattice (Sec. V) and the wrapper pads/unpads with zeros.

Every function cites the passage of the paper it follows:
  init_random          Sec. III (random initial wavefunction) + SplitMix64
  impose_parity        Sec. IV (S_i / A_i operators)
  step                 Sec. III, Eq. updateeq (A, B, D . PsiHat)
  observables          Sec. III, Eq. energysum (sign of Sec. II's H); <r^2>
  evolve               Sec. III renormalisation, Sec. IV re-imposition,
                       Sec. V convergence check
  upsample             Sec. VI / VII.G multi-resolution transfer (trilinear)
  adjoint_step, grad_v_accum, backward
                       adjoint of Eq. updateeq (gradients w.r.t. V)
  project_out          Sec. III snapshot projection of lower states
  combine              Sec. VI linear combination of states as a start
  set_boundary /
  periodic_boundary    Sec. III remark on other boundary conditions:
                       periodic ones (default: the zero shell)
  cstep, cobservables, cevolve
                       complex potentials (Sec. VIII outlook): Eq. updateeq
                       with complex A, B; Hermitian Rayleigh quotient
                       (fdtd_oracle_complex.c)
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liboracle.so")

_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        from .build import build_oracle

        build_oracle()
    lib = ctypes.CDLL(LIB_PATH)
    d, i, i64, u64 = ctypes.c_double, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
    P = ctypes.POINTER(ctypes.c_double)
    lib.oracle_set_boundary.argtypes = [i]
    lib.oracle_set_boundary.restype = None
    lib.oracle_splitmix64_mix.argtypes = [u64]
    lib.oracle_splitmix64_mix.restype = u64
    lib.oracle_splitmix64_output.argtypes = [u64, u64]
    lib.oracle_splitmix64_output.restype = u64
    lib.oracle_draw_uniform.argtypes = [u64, u64, u64]
    lib.oracle_draw_uniform.restype = d
    lib.oracle_draw_gaussian.argtypes = [u64, u64, u64]
    lib.oracle_draw_gaussian.restype = d
    lib.oracle_init_random.argtypes = [i, u64, u64, i, P]
    lib.oracle_init_random.restype = None
    lib.oracle_impose_parity.argtypes = [i, i, P]
    lib.oracle_impose_parity.restype = i
    lib.oracle_impose_parity_adjoint.argtypes = [i, i, P]
    lib.oracle_impose_parity_adjoint.restype = i
    lib.oracle_step.argtypes = [i, d, d, d, P, P, P]
    lib.oracle_step.restype = None
    lib.oracle_observables.argtypes = [i, d, d, P, P, P]
    lib.oracle_observables.restype = None
    lib.oracle_scale.argtypes = [i, d, P]
    lib.oracle_scale.restype = None
    lib.oracle_evolve.argtypes = [i, d, d, d, P, P, P, i64, i64, d, i, i, d, P, P, i64]
    lib.oracle_evolve.restype = i64
    lib.oracle_upsample.argtypes = [i, P, P]
    lib.oracle_upsample.restype = None
    lib.oracle_adjoint_step.argtypes = [i, d, d, d, P, P, P]
    lib.oracle_adjoint_step.restype = None
    lib.oracle_grad_v_accum.argtypes = [i, d, d, d, P, P, P, P]
    lib.oracle_grad_v_accum.restype = None
    lib.oracle_backward.argtypes = [i, d, d, d, P, P, i64, i64, i, d, d, P, P]
    lib.oracle_backward.restype = ctypes.c_int
    lib.oracle_cstep.argtypes = [i, d, d, d, P, P, P, P, P, P]
    lib.oracle_cstep.restype = None
    lib.oracle_cobservables.argtypes = [i, d, d, P, P, P, P, P]
    lib.oracle_cobservables.restype = None
    lib.oracle_cevolve.argtypes = [i, d, d, d, P, P, P, P, P, P, i64, i64, d, i, i, d, P]
    lib.oracle_cevolve.restype = i64
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _dense(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.float64)


def pad(psi: np.ndarray) -> np.ndarray:
    """Dense (N,N,N) -> padded (N+2)^3 with a zero shell (Sec. V)."""
    return np.ascontiguousarray(np.pad(_dense(psi), 1))


def unpad(p: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(p[1:-1, 1:-1, 1:-1])


def _n_of(psi: np.ndarray) -> int:
    n = psi.shape[0]
    assert psi.shape == (n, n, n), psi.shape
    return n


# --- boundary ---------------------------------------------------------------

def set_boundary(periodic: bool) -> None:
    """Zero shell (default, Sec. III) or periodic boundaries for every later call."""
    _load().oracle_set_boundary(int(bool(periodic)))


class periodic_boundary:
    """Context manager: periodic boundaries inside the block."""

    def __enter__(self):
        set_boundary(True)
        return self

    def __exit__(self, *exc):
        set_boundary(False)
        return False


# --- random numbers -------------------------------------------------------

def splitmix64_mix(z: int) -> int:
    return int(_load().oracle_splitmix64_mix(z))


def splitmix64_output(seed: int, d: int) -> int:
    """Output number d (0-based) of the SplitMix64 stream seeded with seed."""
    return int(_load().oracle_splitmix64_output(seed, d))


def draw_uniform(seed: int, lat: int, n: int) -> float:
    return float(_load().oracle_draw_uniform(seed, lat, n))


def draw_gaussian(seed: int, lat: int, n: int) -> float:
    return float(_load().oracle_draw_gaussian(seed, lat, n))


def init_random(n: int, seed: int, lat: int = 0, dist: int = 0) -> np.ndarray:
    """Random initial wavefunction (Sec. III); dist 0 = U[-1,1), 1 = N(0,1)."""
    p = np.zeros((n + 2,) * 3)
    _load().oracle_init_random(n, seed, lat, dist, _ptr(p))
    return unpad(p)


def init_symmetric(n: int, seed: int, mask: int, lat: int = 0, dist: int = 0) -> np.ndarray:
    """Random initial condition with the symmetry mask imposed (Sec. IV)."""
    return impose_parity(init_random(n, seed, lat, dist), mask)


def impose_parity(psi: np.ndarray, mask: int) -> np.ndarray:
    n = _n_of(psi)
    p = pad(psi)
    if _load().oracle_impose_parity(n, mask, _ptr(p)) != 0:
        raise ValueError(f"invalid parity mask {mask}")
    return unpad(p)


def impose_parity_adjoint(lam: np.ndarray, mask: int) -> np.ndarray:
    n = _n_of(lam)
    p = pad(lam)
    if _load().oracle_impose_parity_adjoint(n, mask, _ptr(p)) != 0:
        raise ValueError(f"invalid parity mask {mask}")
    return unpad(p)


# --- update and sums ------------------------------------------------------

def step(psi: np.ndarray, v: np.ndarray, a: float, dtau: float, mass: float = 1.0) -> np.ndarray:
    """One application of Eq. updateeq."""
    n = _n_of(psi)
    vin = _dense(v)
    src, dst = pad(psi), np.zeros((n + 2,) * 3)
    _load().oracle_step(n, a, dtau, mass, _ptr(vin), _ptr(src), _ptr(dst))
    return unpad(dst)


def steps(psi: np.ndarray, v: np.ndarray, a: float, dtau: float, count: int, mass: float = 1.0) -> np.ndarray:
    """`count` plain updates without renormalisation or checks."""
    n = _n_of(psi)
    vin = _dense(v)
    src, dst = pad(psi), np.zeros((n + 2,) * 3)
    lib = _load()
    for _ in range(count):
        lib.oracle_step(n, a, dtau, mass, _ptr(vin), _ptr(src), _ptr(dst))
        src, dst = dst, src
    return unpad(src)


def observables(psi: np.ndarray, v: np.ndarray, a: float, mass: float = 1.0) -> dict:
    """Lattice sums of Eq. energysum and <r^2>; returns S0, SH, Sr, SV, E, r2."""
    n = _n_of(psi)
    out = np.zeros(4)
    _load().oracle_observables(n, a, mass, _ptr(_dense(v)), _ptr(pad(psi)), _ptr(out))
    s0, sh, sr, sv = out
    return {"S0": s0, "SH": sh, "Sr": sr, "SV": sv, "E": sh / s0, "r2": sr / s0, "V": sv / s0}


def evolve(psi, v, a, dtau, max_steps, check_every=100, tol=0.0, tol_relative=False, mask=0,
           v_inf=0.0, mass=1.0, hist_cap=100000):
    """Imaginary-time evolution with checks (Secs. III-V); returns (psi, rec, hist)."""
    n = _n_of(psi)
    p = pad(psi)
    tmp = np.zeros_like(p)
    rec = np.zeros(8)
    hist = np.zeros((hist_cap, 4))
    nchk = _load().oracle_evolve(n, a, dtau, mass, _ptr(_dense(v)), _ptr(p), _ptr(tmp),
                                 int(max_steps), int(check_every), float(tol), int(bool(tol_relative)),
                                 int(mask), float(v_inf), _ptr(rec), _ptr(hist), hist_cap)
    if nchk < 0:
        raise ValueError("bad evolve arguments")
    r = {"E": rec[0], "Eb": rec[1], "S0": rec[2], "r2": rec[3], "V": rec[4], "dE": rec[5],
         "steps": int(rec[6]), "converged": bool(rec[7])}
    return unpad(p), r, hist[: min(nchk, hist_cap)]


def upsample(psi_c: np.ndarray) -> np.ndarray:
    """Trilinear transfer Nc^3 -> (2 Nc)^3 at fixed L (Sec. VI)."""
    nc = _n_of(psi_c)
    dst = np.zeros((2 * nc + 2,) * 3)
    _load().oracle_upsample(nc, _ptr(pad(psi_c)), _ptr(dst))
    return unpad(dst)


# --- adjoint --------------------------------------------------------------

def adjoint_step(lam, v, a, dtau, mass=1.0):
    """Transpose of one update step applied to lam."""
    n = _n_of(lam)
    dst = np.zeros((n + 2,) * 3)
    _load().oracle_adjoint_step(n, a, dtau, mass, _ptr(_dense(v)), _ptr(pad(lam)), _ptr(dst))
    return unpad(dst)


def grad_v_accum(psi, lam_next, v, a, dtau, mass=1.0, gv=None):
    n = _n_of(psi)
    g = np.zeros((n, n, n)) if gv is None else _dense(gv).copy()
    _load().oracle_grad_v_accum(n, a, dtau, mass, _ptr(_dense(v)), _ptr(pad(psi)), _ptr(pad(lam_next)),
                                _ptr(g))
    return g


def project_out(psi, states, a):
    """Sec. III: |psi> - |phi><phi|psi> / <phi|phi> for each phi in `states`,
    one after another, then scaled to sum psi^2 a^3 = 1."""
    out = np.array(psi, dtype=np.float64, copy=True)
    for phi in states:
        phi = np.asarray(phi, dtype=np.float64)
        out = out - phi * (np.sum(phi * out) / np.sum(phi * phi))
    return out / np.sqrt(np.sum(out * out) * a**3)


def combine(states, weights, a):
    """Sec. VI: sum_k weights[k] states[k], scaled to sum psi^2 a^3 = 1."""
    out = sum(w * np.asarray(s, dtype=np.float64) for s, w in zip(states, weights))
    return out / np.sqrt(np.sum(out * out) * a**3)


def backward(psi0, v, a, dtau, T, check_every=100, mask=0, w_e=1.0, w_r=0.0, mass=1.0):
    """d(w_e E + w_r <r^2>)/dV after T unrolled steps from psi0; returns (gV, obs)."""
    n = _n_of(psi0)
    g = np.zeros((n, n, n))
    obs = np.zeros(4)
    rc = _load().oracle_backward(n, a, dtau, mass, _ptr(_dense(v)), _ptr(pad(psi0)), int(T),
                                 int(check_every), int(mask), float(w_e), float(w_r), _ptr(g), _ptr(obs))
    if rc != 0:
        raise MemoryError("oracle_backward could not allocate its trajectory")
    return g, {"E": obs[0], "r2": obs[1], "S0": obs[2], "loss": obs[3]}


# --- complex potentials ------------------------------------------------------

def _parts(x):
    x = np.asarray(x)
    return _dense(x.real), _dense(x.imag) if np.iscomplexobj(x) else np.zeros(x.shape)


def cstep(psi, v, a, dtau, mass=1.0):
    """One application of Eq. updateeq with a complex potential."""
    n = _n_of(np.asarray(psi))
    vr, vi = _parts(v)
    pr, pi = _parts(psi)
    pr, pi = pad(pr), pad(pi)
    outr, outi = np.zeros_like(pr), np.zeros_like(pi)
    _load().oracle_cstep(n, a, dtau, mass, _ptr(vr), _ptr(vi), _ptr(pr), _ptr(pi), _ptr(outr), _ptr(outi))
    return unpad(outr) + 1j * unpad(outi)


def cobservables(psi, v, a, mass=1.0) -> dict:
    """Sums with the Hermitian inner product: S0, SH (complex), Sr, SV
    (complex), and E = SH/S0, <r^2>, <V>."""
    n = _n_of(np.asarray(psi))
    vr, vi = _parts(v)
    pr, pi = _parts(psi)
    out = np.zeros(6)
    _load().oracle_cobservables(n, a, mass, _ptr(vr), _ptr(vi), _ptr(pad(pr)), _ptr(pad(pi)), _ptr(out))
    s0, sh, sr, sv = out[0], out[1] + 1j * out[2], out[3], out[4] + 1j * out[5]
    return {"S0": s0, "SH": sh, "Sr": sr, "SV": sv, "E": sh / s0, "r2": sr / s0, "V": sv / s0}


def cevolve(psi, v, a, dtau, max_steps, check_every=100, tol=0.0, tol_relative=False, mask=0, v_inf=0.0,
            mass=1.0):
    """Complex-potential evolution with checks (Secs. III-V); returns (psi, rec)."""
    n = _n_of(np.asarray(psi))
    vr, vi = _parts(v)
    pr, pi = _parts(psi)
    pr, pi = pad(pr), pad(pi)
    tr, ti = np.zeros_like(pr), np.zeros_like(pi)
    rec = np.zeros(10)
    nchk = _load().oracle_cevolve(n, a, dtau, mass, _ptr(vr), _ptr(vi), _ptr(pr), _ptr(pi), _ptr(tr), _ptr(ti),
                                  int(max_steps), int(check_every), float(tol), int(bool(tol_relative)), int(mask),
                                  float(v_inf), _ptr(rec))
    if nchk < 0:
        raise ValueError("bad evolve arguments")
    r = {"E": rec[0] + 1j * rec[1], "Eb": rec[2] + 1j * rec[1], "S0": rec[3], "r2": rec[4],
         "V": rec[5] + 1j * rec[6], "dE": rec[7], "steps": int(rec[8]), "converged": bool(rec[9])}
    return unpad(pr) + 1j * unpad(pi), r


def cupsample(psi_c):
    """The trilinear transfer (Sec. VI) of the real and imaginary parts."""
    p = np.asarray(psi_c)
    return upsample(p.real) + 1j * upsample(p.imag) if np.iscomplexobj(p) else upsample(p)
