"""Pins of the oracle's complex-potential functions (CPU, no GPU).

Each pin ties the complex update, sums or evolution to something other than
the oracle itself: the real oracle (already pinned) when V is real, an exact
Fourier mode under a uniform complex V, the dense complex Hamiltonian and
iteration matrix at 5^3, and the continuum complex oscillator, whose ground
level 3 omega / 2 continues analytically to complex omega^2.
"""
import numpy as np
import pytest

import workloads as wl


def rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def test_real_potential_reduces_to_the_real_update(orc):
    """V real: the real and imaginary parts evolve as two independent real
    fields (linearity); one step and 60 steps with checks."""
    n, L = 9, 4.0
    a = L / n
    v = wl.harmonic(n, L) + 0.2 * wl.grid(n, L)[0]
    pr, pi = orc.init_random(n, 1), orc.init_random(n, 2)
    got = orc.cstep(pr + 1j * pi, v + 0j, a, a * a / 4)
    assert rel(got.real, orc.step(pr, v, a, a * a / 4)) <= 1e-14
    assert rel(got.imag, orc.step(pi, v, a, a * a / 4)) <= 1e-14
    # evolution: E of a real start equals the real oracle's, Im E = 0
    psi, rec = orc.cevolve(pr + 0j, v + 0j, a, a * a / 4, 60, 20)
    ref, rrec, _ = orc.evolve(pr, v, a, a * a / 4, 60, 20)
    assert rel(psi.real, ref) <= 1e-13 and np.max(np.abs(psi.imag)) == 0.0
    assert rec["E"].real == pytest.approx(rrec["E"], rel=1e-13) and rec["E"].imag == 0.0


@pytest.mark.parametrize("p", [(1, 1, 1), (2, 1, 3)])
def test_fourier_mode_under_a_uniform_complex_potential(orc, p):
    """V = v0 + i w0 everywhere and psi a sine mode with lattice Laplacian
    eigenvalue -mu/a^2: one step multiplies psi by exactly
    (1 - h - c mu) / (1 + h), h = dtau V / 2, c = dtau / (2 m a^2)."""
    n, L, mass = 7, 3.5, 1.3
    a = L / n
    dtau = a * a / 5
    v0 = 0.7 - 0.4j
    idx = np.arange(1, n + 1)
    sx, sy, sz = (np.sin(np.pi * q * idx / (n + 1)) for q in p)
    psi = (sz[:, None, None] * sy[None, :, None] * sx[None, None, :]) * (0.3 + 0.8j)
    mu = 4.0 * sum(np.sin(np.pi * q / (2 * (n + 1))) ** 2 for q in p)
    h = dtau * v0 / 2
    c = dtau / (2 * mass * a * a)
    lam = (1 - h - c * mu) / (1 + h)
    got = orc.cstep(psi, np.full((n, n, n), v0), a, dtau, mass)
    assert rel(got, lam * psi) <= 1e-13


def dense_hamiltonian(n, a, v, mass=1.0):
    """-(1/2m) Lap + diag(V) on the N^3 interior with zero outside, [z][y][x] order."""
    I = np.eye(n)
    d = (np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1) - 2 * I) / (a * a)
    lap = np.kron(np.kron(d, I), I) + np.kron(np.kron(I, d), I) + np.kron(np.kron(I, I), d)
    return -lap / (2 * mass) + np.diag(np.asarray(v, dtype=np.complex128).ravel())


def test_sums_against_the_dense_hamiltonian(orc):
    """E = psi^H H psi / psi^H psi with the dense complex H, <V> and <r^2>
    from the field directly, Im of the kinetic part zero."""
    n, L = 5, 3.0
    a = L / n
    rng = np.random.default_rng(4)
    v = wl.harmonic(n, L) - 1j * wl.absorbing_layer(n, L, 1.0, 2.0) + 0.3j
    psi = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    H = dense_hamiltonian(n, a, v)
    f = psi.ravel()
    s = orc.cobservables(psi, v, a)
    e = np.vdot(f, H @ f) / np.vdot(f, f)
    assert abs(s["E"] - e) <= 1e-12 * abs(e)
    w = np.abs(psi) ** 2
    assert abs(s["V"] - np.sum(v * w) / np.sum(w)) <= 1e-13 * abs(s["V"])
    assert s["r2"] == pytest.approx(np.sum(wl.radius2(n, L) * w) / np.sum(w), rel=1e-13)
    assert s["E"].imag == pytest.approx(s["V"].imag, rel=1e-12)


def test_evolution_converges_to_the_dominant_eigenvector(orc):
    """At 5^3 the iteration matrix M = W^-1 (W - dtau H), W = 1 + dtau V/2,
    is formed densely; the evolved state is its dominant eigenvector and E is
    that vector's Rayleigh quotient."""
    n, L = 5, 3.0
    a = L / n
    dtau = a * a / 4
    v = wl.harmonic(n, L) - 1j * wl.absorbing_layer(n, L, 1.0, 1.5)
    H = dense_hamiltonian(n, a, v)
    W = np.diag(1 + dtau * np.asarray(v).ravel() / 2)
    M = np.linalg.solve(W, W - dtau * H)
    lam, vec = np.linalg.eig(M)
    top = vec[:, np.argmax(np.abs(lam))]
    want = np.vdot(top, H @ top) / np.vdot(top, top)
    psi, rec = orc.cevolve(orc.init_random(n, 3) + 0j, v, a, dtau, 20000, 50, 1e-14)
    assert rec["converged"]
    assert abs(rec["E"] - want) <= 1e-10 * abs(want)
    f = psi.ravel()
    overlap = abs(np.vdot(top, f)) / (np.linalg.norm(top) * np.linalg.norm(f))
    assert overlap == pytest.approx(1.0, abs=1e-10)
    assert want.imag < 0  # the absorbing layer gives the level a negative imaginary part


def test_complex_oscillator_approaches_three_halves_omega(orc):
    """V = w2 r^2/2 with w2 = 1 + 0.4i: the continuum ground level is
    (3/2) sqrt(w2); the lattice level approaches it as O(a^2) (the error
    falls by about four when a halves)."""
    L, w2 = 8.0, 1.0 + 0.4j
    exact = 1.5 * np.sqrt(w2)
    err = []
    for n in (16, 32):
        a = L / n
        v = wl.complex_oscillator(n, L, w2)
        start = np.exp(-0.5 * wl.radius2(n, L)) + 0j
        _, rec = orc.cevolve(start, v, a, a * a / 4, 200000, 100, 1e-12, True)
        assert rec["converged"]
        err.append(abs(rec["E"] - exact))
    assert err[1] < 0.1
    assert 3.0 < err[0] / err[1] < 5.0


def test_absorbing_layer_generator():
    """W is zero inside the box minus the layer, quadratic in the depth into
    the layer, additive over axes."""
    n, L, width, eta = 10, 10.0, 2.0, 3.0
    w = wl.absorbing_layer(n, L, width, eta)
    ax = wl.axis(n, L)
    inner = np.abs(ax) <= 0.5 * L - width
    assert np.all(w[np.ix_(inner, inner, inner)] == 0.0)
    depth = (np.abs(ax[0]) - (0.5 * L - width)) / width
    assert w[0, 0, 0] == pytest.approx(3 * eta * depth**2)
    assert w[0, n // 2, n // 2] == pytest.approx(eta * depth**2)
    assert np.all(w >= 0)


def test_symmetry_mask_acts_on_both_parts(orc):
    """The A_x mask (Sec. IV) at every check of a complex evolution: both
    parts come out exactly odd in x; with a real V each part equals the real
    oracle's masked evolution of that part (the checks' scale factor is
    shared, so the parts are compared after normalising each)."""
    n, L = 8, 4.0
    a = L / n
    v = wl.harmonic(n, L) - 0.3j * wl.absorbing_layer(n, L, 1.0, 1.0)
    start = orc.init_random(n, 5) + 1j * orc.init_random(n, 6)
    psi, _ = orc.cevolve(start, v, a, a * a / 4, 30, 10, mask=wl.ODD_X)
    for part in (psi.real, psi.imag):
        np.testing.assert_array_equal(part[:, :, ::-1], -part)
    vr = wl.harmonic(n, L)
    psi, _ = orc.cevolve(start, vr + 0j, a, a * a / 4, 30, 10, mask=wl.ODD_X)
    for got, part in ((psi.real, start.real), (psi.imag, start.imag)):
        ref, _, _ = orc.evolve(part, vr, a, a * a / 4, 30, 10, mask=wl.ODD_X)
        assert rel(got / np.linalg.norm(got), ref / np.linalg.norm(ref)) <= 1e-13
