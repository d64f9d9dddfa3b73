"""Pins of the oracle's periodic boundaries (the paper's remark that other
boundary conditions are easily implemented, Sec. III): dense circulant
operators assembled independently, exact plane waves, translation
invariance, and a separable crystal potential against a 1-D dense
generalised eigenproblem."""
import math

import numpy as np
import pytest
from scipy.linalg import eigh

import workloads as wl
from dense_ops import hamiltonian, interpolation_1d, second_difference_1d, update_matrix, weight


@pytest.fixture()
def per(orc):
    orc.set_boundary(True)
    yield orc
    orc.set_boundary(False)


@pytest.mark.parametrize("n", [3, 4, 5, 7])
def test_periodic_step_matches_circulant_pde(per, n):
    rng = np.random.default_rng(10 + n)
    a, dtau, mass = 0.4, 0.03, 1.3
    v = rng.uniform(-2.0, 4.0, (n, n, n))
    psi = rng.standard_normal((n, n, n))
    want = (update_matrix(v, a, dtau, mass, periodic=True) @ psi.reshape(-1)).reshape(n, n, n)
    got = per.step(psi, v, a, dtau, mass)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * np.abs(want).max())
    # and it is not the zero-shell operator
    dirichlet = (update_matrix(v, a, dtau, mass) @ psi.reshape(-1)).reshape(n, n, n)
    assert np.abs(got - dirichlet).max() > 1e-3


def test_periodic_plane_wave_is_exact(per):
    """Constant V: cos(2 pi (p i + q j + r k) / N + phi) is an eigenvector of
    the ring Laplacian with eigenvalue -(4/a^2) sum sin^2(pi m / N); one step
    multiplies it by A - B dtau/(2m) lambda and its energy is V0 + lambda/2m."""
    n, a, dtau, v0, mass = 10, 0.3, 0.02, 1.7, 0.8
    p, q, r, phi = 1, 3, 2, 0.4
    i = np.arange(1, n + 1)
    mode = np.cos(2 * math.pi * (r * i[:, None, None] + q * i[None, :, None] + p * i[None, None, :]) / n + phi)
    lam = 4.0 / a**2 * sum(math.sin(math.pi * m / n) ** 2 for m in (p, q, r))
    A = (1 - dtau * v0 / 2) / (1 + dtau * v0 / 2)
    B = 1 / (1 + dtau * v0 / 2)
    got = per.step(mode, np.full((n, n, n), v0), a, dtau, mass)
    np.testing.assert_allclose(got, (A - B * dtau / (2 * mass) * lam) * mode, rtol=0, atol=1e-14)
    assert per.observables(mode, np.full((n, n, n), v0), a, mass)["E"] == pytest.approx(v0 + lam / (2 * mass),
                                                                                         rel=1e-13)


def test_periodic_step_commutes_with_cyclic_shifts(per):
    n, a, dtau = 7, 0.5, 0.05
    rng = np.random.default_rng(21)
    v = rng.uniform(-1, 2, (n, n, n))
    psi = rng.standard_normal((n, n, n))
    base = per.step(psi, v, a, dtau)
    for shift in [(1, 0, 0), (0, 3, 0), (2, 5, 6)]:
        got = per.step(np.roll(psi, shift, (0, 1, 2)), np.roll(v, shift, (0, 1, 2)), a, dtau)
        np.testing.assert_array_equal(got, np.roll(base, shift, (0, 1, 2)))


def test_periodic_observables_match_dense(per):
    n, a, mass = 5, 0.6, 0.7
    rng = np.random.default_rng(5)
    v = rng.uniform(-1, 2, (n, n, n))
    psi = rng.standard_normal((n, n, n))
    f = psi.reshape(-1)
    obs = per.observables(psi, v, a, mass)
    assert obs["SH"] == pytest.approx(f @ hamiltonian(v, a, mass, periodic=True) @ f, rel=1e-12)
    assert obs["S0"] == pytest.approx(f @ f, rel=1e-14)


def test_periodic_constant_potential_ground_state_is_uniform(per):
    n, L, v0 = 8, 4.0, -0.3
    a = L / n
    psi, rec, _ = per.evolve(per.init_random(n, 5), np.full((n, n, n), v0), a, a * a / 4, 200000, 100, 1e-14)
    assert rec["converged"]
    assert rec["E"] == pytest.approx(v0, abs=1e-11)
    assert np.std(psi) <= 1e-6 * np.abs(np.mean(psi))


def test_periodic_crystal_ground_state_matches_1d_generalised_eigenproblem(per):
    """V depends on x only (a cosine 'crystal' of period L): the converged
    field is uniform in y and z, and along x it is the lowest generalised
    eigenvector of (H_1d, 1 + dtau V/2) on the ring; the oracle reports its
    Rayleigh quotient <H>."""
    n, L, v0 = 12, 6.0, 1.5
    a = L / n
    dtau = a * a / 4
    xs = wl.axis(n, L)
    v1 = v0 * np.cos(2 * math.pi * xs / L)
    v = np.broadcast_to(v1[None, None, :], (n, n, n)).copy()
    psi, rec, _ = per.evolve(per.init_random(n, 9), v, a, dtau, 400000, 100, 1e-14)
    assert rec["converged"]
    h1 = -second_difference_1d(n, a, periodic=True) / 2.0 + np.diag(v1)
    w1 = weight(v1, dtau)
    _, vecs = eigh(h1, np.diag(w1))
    g = vecs[:, 0]
    assert rec["E"] == pytest.approx(g @ h1 @ g / (g @ g), abs=1e-10)
    prof = psi[0, 0, :]
    np.testing.assert_allclose(psi, np.broadcast_to(prof, psi.shape), rtol=0, atol=1e-6 * np.abs(prof).max())
    assert rec["E"] < v0  # bound below the barrier tops, above the minimum -v0
    assert rec["E"] > -v0


def test_periodic_upsample_matches_ring_interpolation(per):
    nc = 5
    f = np.random.default_rng(2).standard_normal((nc, nc, nc))
    p = interpolation_1d(nc, periodic=True)
    want = (np.kron(np.kron(p, p), p) @ f.reshape(-1)).reshape((2 * nc,) * 3)
    np.testing.assert_allclose(per.upsample(f), want, atol=1e-14)
    np.testing.assert_allclose(per.upsample(np.full((nc,) * 3, 2.5)), 2.5, atol=1e-14)


def test_periodic_adjoint_is_the_transpose(per):
    n, a = 5, 0.5
    dtau = a * a / 4
    rng = np.random.default_rng(11)
    v = rng.uniform(-1, 3, (n, n, n))
    y = rng.standard_normal((n, n, n))
    mt = update_matrix(v, a, dtau, periodic=True).T
    np.testing.assert_allclose(per.adjoint_step(y, v, a, dtau).reshape(-1), mt @ y.reshape(-1), atol=1e-13)


def test_periodic_backward_matches_central_differences(per):
    n, L, T, ce = 6, 4.0, 30, 10
    a = L / n
    dtau = a * a / 4
    z, y, x = wl.grid(n, L)
    v = np.ascontiguousarray(np.broadcast_to(0.5 * np.cos(2 * math.pi * x / L) + 0.2 * np.sin(2 * math.pi * y / L),
                                             (n, n, n)))
    psi0 = per.init_random(n, 13)
    g, obs = per.backward(psi0, v, a, dtau, T, ce, 0, 1.0, 0.0)

    def loss(vv):
        _, rec, _ = per.evolve(psi0, vv, a, dtau, T, ce, 0.0, False, 0)
        return rec["E"]

    assert obs["loss"] == pytest.approx(loss(v), rel=1e-13)
    h = 1e-4
    for site in [(0, 0, 0), (3, 5, 1), (5, 2, 4)]:
        vp, vm = v.copy(), v.copy()
        vp[site] += h
        vm[site] -= h
        assert g[site] == pytest.approx((loss(vp) - loss(vm)) / (2 * h), rel=1e-5, abs=1e-9)
