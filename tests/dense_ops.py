"""Dense matrices for tiny lattices, built independently of the oracle.

The 3-D operators are assembled from 1-D matrices with Kronecker products
(numpy C order, axes [z][y][x]), a construction that shares nothing with the
oracle's site loops.  Used only by the tests to pin the oracle.
"""
import numpy as np


def second_difference_1d(n: int, a: float, periodic: bool = False) -> np.ndarray:
    """D = [1, -2, 1] / a^2 on n sites with zero values beyond both ends, or
    on a ring of n sites (circulant) when periodic."""
    d = np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
    if periodic:
        d[0, n - 1] += 1.0
        d[n - 1, 0] += 1.0
    return d / (a * a)


def laplacian_3d(n: int, a: float, periodic: bool = False) -> np.ndarray:
    t, i = second_difference_1d(n, a, periodic), np.eye(n)
    return np.kron(np.kron(i, i), t) + np.kron(np.kron(i, t), i) + np.kron(np.kron(t, i), i)


def hamiltonian(v: np.ndarray, a: float, mass: float = 1.0, periodic: bool = False) -> np.ndarray:
    """H = -(1/2m) Lap + diag(V) on the lattice (Sec. II with Sec. III's D)."""
    n = v.shape[0]
    return -laplacian_3d(n, a, periodic) / (2.0 * mass) + np.diag(v.reshape(-1))


def weight(v: np.ndarray, dtau: float) -> np.ndarray:
    return 1.0 + 0.5 * dtau * v.reshape(-1)


def update_matrix(v: np.ndarray, a: float, dtau: float, mass: float = 1.0, periodic: bool = False) -> np.ndarray:
    """The FDTD step as a matrix: (1 + dtau V/2) psi' = (1 - dtau V/2) psi + (dtau/2m) Lap psi,
    i.e. psi' = W^-1 [(2 - W) + (dtau/2m) Lap] psi with W = 1 + dtau V / 2."""
    n = v.shape[0]
    w = weight(v, dtau)
    rhs = np.diag(2.0 - w) + dtau / (2.0 * mass) * laplacian_3d(n, a, periodic)
    return rhs / w[:, None]


def interpolation_1d(nc: int, periodic: bool = False) -> np.ndarray:
    """Linear interpolation from nc cell-centred coarse sites to 2 nc fine
    sites of the same box, zero beyond the ends (or wrapping around a ring
    when periodic): the fine site j sits at coarse index position j/2 + 1/4."""
    nf = 2 * nc
    p = np.zeros((nf, nc))
    for j in range(1, nf + 1):
        xi = 0.5 * j + 0.25
        lo = int(np.floor(xi))
        w = xi - lo
        for idx, wt in ((lo, 1.0 - w), (lo + 1, w)):
            if periodic:
                p[j - 1, (idx - 1) % nc] += wt
            elif 1 <= idx <= nc:
                p[j - 1, idx - 1] += wt
    return p
