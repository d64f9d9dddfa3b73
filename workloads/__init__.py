"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the CUDA path, the oracle, the tests and the
benchmark.  It holds no arithmetic of the FDTD method itself (no update,
sum, symmetry operator or interpolation): only the lattice geometry
convention, closed-form potentials V(r) evaluated on lattice sites, and the
seeded draws of workload parameters.  All values are float64 numpy arrays of
shape (N, N, N) indexed [z][y][x].

Geometry: interior site i = 1..N along an axis sits at x_i = (i - (N+1)/2) a
with a = L / N (Sec. III: L = N a; Sec. VII: r is the distance from the
centre of the lattice).  For even N no site falls on the centre, which keeps
the Coulomb singularity off the lattice (Sec. III).

Potentials (paper citations):
  harmonic        V = w^2 r^2 / 2                      Sec. VII.D, Eq. hopot
  coulomb_paper   V = 0 (r < a), -1/r + 1/a (r >= a)   Sec. VII.C, Eq. coulombpot
  coulomb_soft    V = -Z / sqrt(r^2 + a^2)             regulated variant
  anisotropic     V = (x^2 + 2 y^2 + 3 z^2)/2 + sum of seeded Gaussians
  dodecahedron    V = -100 inside the regular dodecahedron of Sec. VII.E
  v_theta         V = r^2/2 + sum_k theta_k G_k(r)     differentiable workload
  complex_oscillator  V = w2 r^2 / 2 with complex w2    complex potentials (Sec. VIII)
  absorbing_layer W = eta sum_axes ((|x| - x0)/w)^2 beyond x0 = L/2 - w: the
                  imaginary part -W of an absorbing boundary layer
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 904939


def spacing(n: int, length: float) -> float:
    return float(length) / float(n)


def axis(n: int, length: float) -> np.ndarray:
    a = spacing(n, length)
    return (np.arange(1, n + 1, dtype=np.float64) - 0.5 * (n + 1)) * a


def grid(n: int, length: float):
    """(z, y, x) coordinate arrays broadcastable to (N, N, N)."""
    x = axis(n, length)
    return x[:, None, None], x[None, :, None], x[None, None, :]


def radius2(n: int, length: float) -> np.ndarray:
    z, y, x = grid(n, length)
    return x * x + y * y + z * z


def harmonic(n: int, length: float, omega: float = 1.0) -> np.ndarray:
    return 0.5 * omega * omega * radius2(n, length)


def coulomb_soft(n: int, length: float, charge: float = 1.0) -> np.ndarray:
    a = spacing(n, length)
    return -charge / np.sqrt(radius2(n, length) + a * a)


def coulomb_paper(n: int, length: float) -> np.ndarray:
    a = spacing(n, length)
    r = np.sqrt(radius2(n, length))
    return np.where(r < a, 0.0, -1.0 / np.maximum(r, a) + 1.0 / a)


def coulomb_paper_device(n: int, length: float, device, dtype=None):
    """coulomb_paper() evaluated on a torch device, for lattices too large to
    build quickly in numpy (1024^3)."""
    import torch

    dtype = dtype or torch.float64
    a = spacing(n, length)
    ax = torch.as_tensor(axis(n, length), dtype=torch.float64, device=device)
    r = torch.sqrt(ax[:, None, None] ** 2 + ax[None, :, None] ** 2 + ax[None, None, :] ** 2)
    return torch.where(r < a, torch.zeros_like(r), -1.0 / torch.clamp(r, min=a) + 1.0 / a).to(dtype)


def gaussian_bumps(n: int, length: float, centres, widths, amplitudes) -> np.ndarray:
    """sum_k amp_k exp(-|r - c_k|^2 / (2 w_k^2)), built from per-axis factors."""
    ax = axis(n, length)
    out = np.zeros((n, n, n))
    for (cx, cy, cz), w, amp in zip(centres, widths, amplitudes):
        s = 2.0 * w * w
        ex, ey, ez = (np.exp(-((ax - c) ** 2) / s) for c in (cx, cy, cz))
        out += amp * ez[:, None, None] * (ey[:, None] * ex[None, :])[None, :, :]
    return out


def gaussian_params(seed: int, count: int, half_box: float, amp_range, width_range):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(-half_box, half_box, size=(count, 3))
    widths = rng.uniform(width_range[0], width_range[1], size=count)
    amps = rng.uniform(amp_range[0], amp_range[1], size=count)
    return centres, widths, amps


def anisotropic(n: int, length: float, seed: int = BASE_SEED, count: int = 32) -> np.ndarray:
    """(x^2 + 2y^2 + 3z^2)/2 plus `count` Gaussians with amplitude U[-0.5,0.5],
    width U[0.5,2] and centres uniform in [-L/4, L/4]^3."""
    z, y, x = grid(n, length)
    base = 0.5 * (x * x + 2.0 * y * y + 3.0 * z * z)
    c, w, amp = gaussian_params(seed, count, length / 4.0, (-0.5, 0.5), (0.5, 2.0))
    return base + gaussian_bumps(n, length, c, w, amp)


def anisotropic_device(n: int, length: float, device, seed: int = BASE_SEED, count: int = 32, dtype=None):
    """anisotropic() evaluated on a torch device (same seeded parameters,
    same per-axis construction); for lattices too large to build quickly in
    numpy."""
    import torch

    dtype = dtype or torch.float64
    ax = torch.as_tensor(axis(n, length), dtype=torch.float64, device=device)
    v = 0.5 * (ax[None, None, :] ** 2 + 2.0 * ax[None, :, None] ** 2 + 3.0 * ax[:, None, None] ** 2)
    c, w, amp = gaussian_params(seed, count, length / 4.0, (-0.5, 0.5), (0.5, 2.0))
    for (cx, cy, cz), wk, ak in zip(c, w, amp):
        s = 2.0 * wk * wk
        ex, ey, ez = (torch.exp(-((ax - float(cc)) ** 2) / s) for cc in (cx, cy, cz))
        v += float(ak) * ez[:, None, None] * (ey[:, None] * ex[None, :])[None, :, :]
    return v.to(dtype)


def theta_basis(n: int, length: float, seed: int = BASE_SEED + 5, count: int = 16):
    """Basis G_k(r) = exp(-|r - c_k|^2 / (2 s_k^2)), c_k in [-L/4, L/4]^3,
    s_k in U[0.5, 1.5], and a seeded theta_k in U[-1, 1].
    Returns (G[count, N, N, N], theta[count])."""
    c, s, th = gaussian_params(seed, count, length / 4.0, (-1.0, 1.0), (0.5, 1.5))
    g = np.empty((count, n, n, n))
    for k in range(count):
        g[k] = gaussian_bumps(n, length, c[k:k + 1], s[k:k + 1], [1.0])
    return g, th


def v_theta(n: int, length: float, theta, basis) -> np.ndarray:
    return 0.5 * radius2(n, length) + np.tensordot(np.asarray(theta, dtype=np.float64), basis, axes=1)


def complex_oscillator(n: int, length: float, omega2: complex) -> np.ndarray:
    """V = omega2 r^2 / 2 with a complex omega2 (complex128 array)."""
    return 0.5 * complex(omega2) * radius2(n, length).astype(np.complex128)


def absorbing_layer(n: int, length: float, width: float, strength: float) -> np.ndarray:
    """W(r) = strength * sum over axes of ((|x| - x0) / width)^2 where |x| > x0
    = L/2 - width, else 0: the magnitude of a negative imaginary potential
    -i W that absorbs what reaches the last `width` of the box on each side
    (a complex absorbing layer; V = V_R - i W)."""
    x0 = 0.5 * length - width
    ax = axis(n, length)
    f = np.where(np.abs(ax) > x0, ((np.abs(ax) - x0) / width) ** 2, 0.0)
    return strength * (f[:, None, None] + f[None, :, None] + f[None, None, :])


PHI = 0.5 * (1.0 + math.sqrt(5.0))


def dodecahedron_vertices(printed: bool = False) -> np.ndarray:
    """20 vertices of the dodecahedron of Sec. VII.E, Eq. dodecahedronpotential:
    (+-1/phi, +-1/phi, +-1/phi), (0, +-1/phi^2, +-1), (+-1/phi^2, +-1, 0) and a
    third group that the paper prints as (+-1/phi^2, 0, +-1).  That printed
    group does not close a regular solid; the regular dodecahedron the text
    names needs the cyclic permutation (+-1, 0, +-1/phi^2), which is the
    default here (printed=True gives the list as printed)."""
    p, q = 1.0 / PHI, 1.0 / (PHI * PHI)
    v = []
    for sx in (-1, 1):
        for sy in (-1, 1):
            for sz in (-1, 1):
                v.append((sx * p, sy * p, sz * p))
    for s1 in (-1, 1):
        for s2 in (-1, 1):
            v.append((0.0, s1 * q, s2 * 1.0))
            v.append((s1 * q, s2 * 1.0, 0.0))
            v.append((s1 * q, 0.0, s2 * 1.0) if printed else (s2 * 1.0, 0.0, s1 * q))
    return np.array(v)


def dodecahedron(n: int, depth: float = -100.0, printed: bool = False) -> np.ndarray:
    """V = depth inside the convex hull of the 20 vertices, 0 outside.
    Lattice index 1 maps to the coordinate -1 and index N to +1 on every
    axis (Sec. VII.E)."""
    from scipy.spatial import ConvexHull

    verts = dodecahedron_vertices(printed)
    hull = ConvexHull(verts)
    u = -1.0 + 2.0 * (np.arange(1, n + 1, dtype=np.float64) - 1.0) / (n - 1.0)
    z, y, x = u[:, None, None], u[None, :, None], u[None, None, :]
    inside = np.ones((n, n, n), dtype=bool)
    for eq in hull.equations:  # eq[:3] . p + eq[3] <= 0 inside
        inside &= (eq[0] * x + eq[1] * y + eq[2] * z + eq[3]) <= 1e-12
    return np.where(inside, depth, 0.0)


# --- workload recipes --------------------------------------------------------

SYMMETRIC_ALL = 0b010101          # S_x S_y S_z
ODD_X = 0b000010                  # A_x
ODD_Y = 0b001000                  # A_y
ODD_Z = 0b100000                  # A_z


@dataclass
class Lattice:
    """One lattice: size, box, potential recipe, symmetry sector."""
    n: int
    length: float
    kind: str = "harmonic"
    param: float = 1.0
    mask: int = 0
    seed: int = BASE_SEED
    v_inf: float = 0.0
    meta: dict = field(default_factory=dict)

    @property
    def a(self) -> float:
        return spacing(self.n, self.length)

    @property
    def dtau(self) -> float:
        return self.a * self.a / 4.0

    def potential(self) -> np.ndarray:
        if self.kind == "harmonic":
            return harmonic(self.n, self.length, self.param)
        if self.kind == "coulomb_soft":
            return coulomb_soft(self.n, self.length, self.param)
        if self.kind == "coulomb_paper":
            return coulomb_paper(self.n, self.length)
        if self.kind == "anisotropic":
            return anisotropic(self.n, self.length, self.seed)
        if self.kind == "dodecahedron":
            return dodecahedron(self.n)
        raise ValueError(self.kind)


def config_small_ho() -> Lattice:
    """32^3, L = 10, V = r^2/2, dtau = a^2/4, uniform random start."""
    return Lattice(32, 10.0, "harmonic", 1.0, 0)


def config_coulomb_levels(mask: int = SYMMETRIC_ALL):
    """Soft-core Coulomb, L = 40, levels 64^3 -> 128^3 -> 256^3."""
    return [Lattice(n, 40.0, "coulomb_soft", 1.0, mask) for n in (64, 128, 256)]


def config_anisotropic_levels():
    """Anisotropic oscillator + 32 Gaussians, L = 16, 128^3 -> 256^3 -> 512^3."""
    return [Lattice(n, 16.0, "anisotropic", 1.0, 0) for n in (128, 256, 512)]


def config_batch(seed: int = BASE_SEED + 3, count: int = 64):
    """`count` independent lattices: N in {48, 64, 96, 128, 160}; harmonic
    (omega in U[0.5, 2], L = 12/sqrt(omega)) or soft-core Coulomb (Z in
    U[0.5, 2], L = 24/Z for the even sector, 48/Z for an odd sector); sector
    drawn from {S_x S_y S_z, A_x, A_y, A_z}."""
    rng = np.random.default_rng(seed)
    sizes = (48, 64, 96, 128, 160)
    sectors = (SYMMETRIC_ALL, ODD_X, ODD_Y, ODD_Z)
    out = []
    for b in range(count):
        n = int(sizes[rng.integers(0, len(sizes))])
        mask = int(sectors[rng.integers(0, len(sectors))])
        if rng.uniform() < 0.5:
            om = float(rng.uniform(0.5, 2.0))
            out.append(Lattice(n, 12.0 / math.sqrt(om), "harmonic", om, mask, seed + b))
        else:
            zc = float(rng.uniform(0.5, 2.0))
            length = (24.0 if mask == SYMMETRIC_ALL else 48.0) / zc
            out.append(Lattice(n, length, "coulomb_soft", zc, mask, seed + b))
    return out


def config_theta(n: int = 128, length: float = 10.0, seed: int = BASE_SEED + 5):
    """V_theta = r^2/2 + sum_{k<16} theta_k exp(-|r - c_k|^2 / (2 s_k^2))."""
    g, th = theta_basis(n, length, seed)
    return g, th
