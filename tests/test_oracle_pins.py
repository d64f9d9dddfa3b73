"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics.

Each test pins one oracle function to something other than itself: published
generator outputs, the discretised PDE assembled as a dense matrix by
Kronecker products (Eqs. time + space of Sec. III, a route independent of
the A/B form of Eq. updateeq), exact discrete eigenmodes, dense generalised
eigenpairs, continuum closed forms reached at O(a^2), affine exactness of
interpolation, transpose identities and central finite differences.
"""
import math
import os

import numpy as np
import pytest

import workloads as wl
from dense_ops import hamiltonian, interpolation_1d, laplacian_3d, update_matrix, weight
from conftest import GOLDEN


# ----------------------------------------------------------------- generator

def test_splitmix64_published_vectors(orc):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_vectors.txt")) if l[0] != "#"]
    assert len(rows) == 7
    for seed, idx, val in rows:
        assert orc.splitmix64_output(int(seed), int(idx)) == int(val)


def test_uniform_draws_distribution(orc):
    from scipy import stats

    x = np.array([orc.draw_uniform(11, 0, n) for n in range(20000)])
    assert x.min() >= -1.0 and x.max() < 1.0
    assert stats.kstest(x, stats.uniform(loc=-1, scale=2).cdf).pvalue > 1e-3
    assert abs(np.corrcoef(x[:-1], x[1:])[0, 1]) < 0.03
    # separate lattices draw from disjoint, uncorrelated blocks
    y = np.array([orc.draw_uniform(11, 1, n) for n in range(20000)])
    assert abs(np.corrcoef(x, y)[0, 1]) < 0.03


def test_gaussian_draws_distribution(orc):
    from scipy import stats

    g = np.array([orc.draw_gaussian(5, 2, n) for n in range(20000)])
    assert stats.kstest(g, "norm").pvalue > 1e-3
    assert abs(g.mean()) < 0.03 and abs(g.std() - 1.0) < 0.03


def test_init_random_site_order(orc):
    n = 5
    p = orc.init_random(n, 77, 3, 0)
    # dense index n = ((k-1) N + (j-1)) N + (i-1): z slowest, x fastest
    assert p[2, 1, 4] == orc.draw_uniform(77, 3, (2 * n + 1) * n + 4)
    assert p.shape == (n, n, n)


# ----------------------------------------------------------------- update

@pytest.mark.parametrize("n", [4, 5, 7])
def test_step_matches_discretised_pde(orc, n):
    rng = np.random.default_rng(n)
    L = 3.0
    a = L / n
    dtau = 0.2 * a * a
    v = rng.uniform(-2.0, 4.0, size=(n, n, n))
    psi = rng.standard_normal((n, n, n))
    got = orc.step(psi, v, a, dtau, mass=1.3)
    want = (update_matrix(v, a, dtau, mass=1.3) @ psi.reshape(-1)).reshape(n, n, n)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13 * np.abs(want).max())


def test_step_exact_fourier_mode(orc):
    """Constant V: sin modes are exact eigenvectors of the lattice Laplacian
    with eigenvalue -(4/a^2) sum_i sin^2(pi p_i / (2(N+1)))."""
    n, a, dtau, v0, mass = 9, 0.3, 0.02, 1.7, 0.8
    p, q, r = 1, 3, 2
    idx = np.arange(1, n + 1)
    mode = (np.sin(math.pi * r * idx / (n + 1))[:, None, None] * np.sin(math.pi * q * idx / (n + 1))[None, :, None]
            * np.sin(math.pi * p * idx / (n + 1))[None, None, :])
    lam = 4.0 / a**2 * sum(math.sin(math.pi * m / (2 * (n + 1))) ** 2 for m in (p, q, r))
    A = (1 - dtau * v0 / 2) / (1 + dtau * v0 / 2)
    B = 1 / (1 + dtau * v0 / 2)
    factor = A - B * dtau / (2 * mass) * lam
    got = orc.step(mode, np.full((n, n, n), v0), a, dtau, mass)
    np.testing.assert_allclose(got, factor * mode, rtol=0, atol=1e-14)
    obs = orc.observables(mode, np.full((n, n, n), v0), a, mass)
    assert obs["E"] == pytest.approx(v0 + lam / (2 * mass), rel=1e-13)


# ----------------------------------------------------------------- sums

def test_observables_match_dense(orc):
    n, L = 6, 4.0
    a = L / n
    rng = np.random.default_rng(3)
    v = rng.uniform(-1, 2, size=(n, n, n))
    psi = rng.standard_normal((n, n, n))
    h = hamiltonian(v, a, mass=0.7)
    f = psi.reshape(-1)
    obs = orc.observables(psi, v, a, mass=0.7)
    assert obs["S0"] == pytest.approx(f @ f, rel=1e-14)
    assert obs["SH"] == pytest.approx(f @ h @ f, rel=1e-12)
    assert obs["SV"] == pytest.approx(f @ (v.reshape(-1) * f), rel=1e-13)
    # r measured from the box centre: independent of which potential is used
    pos = (np.arange(n) - (n - 1) / 2.0) * a
    zz, yy, xx = np.meshgrid(pos, pos, pos, indexing="ij")
    assert obs["Sr"] == pytest.approx(np.sum((xx**2 + yy**2 + zz**2) * psi**2), rel=1e-13)


# ----------------------------------------------------------------- fixed point

@pytest.mark.parametrize("kind", ["harmonic", "skewed"])
def test_converged_state_is_generalised_eigenvector(orc, kind):
    """psi' = (I - dtau W^-1 H) psi: the iteration converges to the lowest
    generalised eigenvector of (H, W), W = 1 + dtau V / 2."""
    from scipy.linalg import eigh

    n, L = 8, 4.0
    a = L / n
    dtau = a * a / 4
    z, y, x = wl.grid(n, L)
    v = wl.harmonic(n, L)
    if kind == "skewed":
        v = v + 0.3 * x + 0.6 * y * y - 0.2 * z + 0.1 * x * z
    h = hamiltonian(v, a)
    w = weight(v, dtau)
    evals, evecs = eigh(h, np.diag(w))
    g = evecs[:, 0]
    e_ref = g @ h @ g / (g @ g)
    psi0 = orc.init_random(n, 1, 0, 0)
    psi, rec, _ = orc.evolve(psi0, v, a, dtau, 20000, 50, 1e-15, False)
    assert rec["converged"]
    assert rec["E"] == pytest.approx(e_ref, abs=1e-11)
    u = psi.reshape(-1) / np.linalg.norm(psi)
    gg = g / np.linalg.norm(g) * np.sign(g @ u)
    assert np.max(np.abs(u - gg)) < 1e-6
    # and the generalised eigenvalue is the fixed point of the update matrix
    m = update_matrix(v, a, dtau)
    assert np.max(np.abs(m @ gg - (1 - dtau * evals[0]) * gg)) < 1e-12


# ----------------------------------------------------------------- closed forms

def _ground(orc, v, n, L, mask=0, tol=1e-13, max_steps=200000):
    a = L / n
    psi0 = orc.init_symmetric(n, 21, mask, 0, 0)
    _, rec, _ = orc.evolve(psi0, v, a, a * a / 4, max_steps, 100, tol, False, mask)
    assert rec["converged"]
    return rec


def test_harmonic_oscillator_a_squared_convergence(orc):
    """3-D oscillator: E0 = 3/2 and <r^2> = 3/2 in the continuum; the lattice
    error is O(a^2), so halving a divides it by ~4."""
    L = 8.0
    es, rs = [], []
    for n in (16, 32, 64):
        rec = _ground(orc, wl.harmonic(n, L), n, L)
        es.append(rec["E"] - 1.5)
        rs.append(rec["r2"] - 1.5)
    assert abs(es[-1]) < 3e-3 and abs(rs[-1]) < 3e-2
    assert 3.5 < es[0] / es[1] < 4.5 and 3.5 < es[1] / es[2] < 4.5
    assert 3.0 < rs[0] / rs[1] < 5.0 and 3.0 < rs[1] / rs[2] < 5.0


def test_anisotropic_oscillator_closed_form(orc):
    """V = (x^2 + 2 y^2 + 3 z^2)/2: E0 = (1 + sqrt2 + sqrt3)/2 and
    <r^2> = (1 + 1/sqrt2 + 1/sqrt3)/2; distinct axes catch any x/y/z mix-up."""
    L = 8.0
    e_exact = 0.5 * (1 + math.sqrt(2) + math.sqrt(3))
    r_exact = 0.5 * (1 + 1 / math.sqrt(2) + 1 / math.sqrt(3))
    errs = []
    for n in (16, 32):
        z, y, x = wl.grid(n, L)
        rec = _ground(orc, 0.5 * (x * x + 2 * y * y + 3 * z * z), n, L)
        errs.append(rec["E"] - e_exact)
        assert rec["r2"] == pytest.approx(r_exact, rel=0.05)
    assert abs(errs[1]) < 2e-2
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_odd_sector_gives_first_excited_oscillator_state(orc):
    """A_x removes the even ground state: E -> 5/2, <r^2> -> 5/2 (Sec. IV)."""
    L = 8.0
    r16, r32 = (_ground(orc, wl.harmonic(n, L), n, L, mask=wl.ODD_X) for n in (16, 32))
    assert r32["E"] == pytest.approx(2.5, rel=1e-2)
    assert r32["r2"] == pytest.approx(2.5, rel=3e-2)
    assert 3.5 < (r16["E"] - 2.5) / (r32["E"] - 2.5) < 4.5


def test_paper_coulomb_binding_energy(orc):
    """Eq. coulombpot with binding energy E - V_inf, V_inf = 1/a (Eq.
    bindingenergy): the 1s level E0 = -1/2 (Sec. VII.C), here on a coarse
    lattice (a = 0.25), so only to a few per cent."""
    import json

    gold = json.load(open(os.path.join(GOLDEN, "paper_values.json")))["coulomb_levels"]
    n, L = 64, 16.0
    a = L / n
    v = wl.coulomb_paper(n, L)
    psi0 = orc.init_symmetric(n, 4, wl.SYMMETRIC_ALL)
    _, rec, _ = orc.evolve(psi0, v, a, a * a / 4, 40000, 100, 1e-7, True, wl.SYMMETRIC_ALL, v_inf=1.0 / a)
    assert rec["converged"]
    assert rec["Eb"] == pytest.approx(gold["E0"], rel=0.05)
    assert rec["E"] == pytest.approx(rec["Eb"] + 1.0 / a, rel=1e-14)


# ----------------------------------------------------------------- symmetry

@pytest.mark.parametrize("n", [6, 7])
def test_parity_operators(orc, n):
    rng = np.random.default_rng(n)
    f = rng.standard_normal((n, n, n))
    for mask, sx, sy, sz in [(wl.ODD_X, -1, 0, 0), (wl.SYMMETRIC_ALL, 1, 1, 1), (wl.ODD_Z | 0b0100, 0, 1, -1)]:
        g = orc.impose_parity(f, mask)
        for axis, s in ((2, sx), (1, sy), (0, sz)):  # numpy axes: x=2, y=1, z=0
            if s:
                np.testing.assert_array_equal(np.flip(g, axis=axis), s * g)
        # the lower half along every masked axis is the source and is unchanged
        lo = tuple(slice(0, n // 2) if s else slice(None) for s in (sz, sy, sx))
        np.testing.assert_array_equal(g[lo], f[lo])
        np.testing.assert_array_equal(orc.impose_parity(g, mask), g)  # idempotent
        y = rng.standard_normal((n, n, n))
        assert np.sum(g * y) == pytest.approx(np.sum(f * orc.impose_parity_adjoint(y, mask)), rel=1e-12)
    with pytest.raises(ValueError):
        orc.impose_parity(f, 0b11)


def test_parity_is_kept_by_the_update(orc):
    n, L = 10, 5.0
    a = L / n
    v = wl.harmonic(n, L)
    f = orc.init_symmetric(n, 9, wl.ODD_Y)
    g = orc.steps(f, v, a, a * a / 4, 50)
    assert np.max(np.abs(np.flip(g, axis=1) + g)) <= 1e-15 * np.abs(g).max() * 50


# ----------------------------------------------------------------- renormalisation

def test_renormalisation_and_scale_invariance(orc):
    n, L = 12, 6.0
    a = L / n
    v = wl.harmonic(n, L)
    psi, rec, _ = orc.evolve(orc.init_random(n, 2), v, a, a * a / 4, 300, 100)
    assert np.sum(psi**2) * a**3 == pytest.approx(1.0, abs=1e-14)
    o1 = orc.observables(psi, v, a)
    o2 = orc.observables(7.25 * psi, v, a)
    assert o1["E"] == pytest.approx(o2["E"], rel=1e-14)
    assert o1["r2"] == pytest.approx(o2["r2"], rel=1e-14)


# ----------------------------------------------------------------- multi-resolution

def test_upsample_exact_on_affine_fields(orc):
    nc, L = 6, 3.0
    z, y, x = wl.grid(nc, L)
    f = 0.3 + 1.1 * x - 0.7 * y + 2.0 * z + 0 * (x + y + z)
    up = orc.upsample(f)
    zf, yf, xf = wl.grid(2 * nc, L)
    want = 0.3 + 1.1 * xf - 0.7 * yf + 2.0 * zf + 0 * (xf + yf + zf)
    inner = (slice(1, -1),) * 3  # sites whose 8 coarse neighbours are all interior
    np.testing.assert_allclose(up[inner], want[inner], atol=1e-13)


def test_upsample_matches_kronecker_interpolation(orc):
    nc = 5
    f = np.random.default_rng(0).standard_normal((nc, nc, nc))
    p = interpolation_1d(nc)
    want = (np.kron(np.kron(p, p), p) @ f.reshape(-1)).reshape((2 * nc,) * 3)
    np.testing.assert_allclose(orc.upsample(f), want, atol=1e-14)


def test_upsampled_ground_state_is_a_good_start(orc):
    L = 8.0
    nc = 16
    vc = wl.harmonic(nc, L)
    ac = L / nc
    pc, rc, _ = orc.evolve(orc.init_random(nc, 3), vc, ac, ac * ac / 4, 100000, 100, 1e-12)
    nf = 2 * nc
    af = L / nf
    vf = wl.harmonic(nf, L)
    start = orc.upsample(pc)
    assert orc.observables(start, vf, af)["E"] == pytest.approx(rc["E"], rel=2e-2)
    _, r_up, _ = orc.evolve(start, vf, af, af * af / 4, 100000, 100, 1e-9)
    _, r_rand, _ = orc.evolve(orc.init_random(nf, 3), vf, af, af * af / 4, 100000, 100, 1e-9)
    assert r_up["E"] == pytest.approx(r_rand["E"], abs=1e-7)
    assert r_up["steps"] < r_rand["steps"]


# ----------------------------------------------------------------- adjoint

def test_adjoint_step_is_the_transpose(orc):
    n, L = 6, 3.0
    a = L / n
    dtau = a * a / 4
    rng = np.random.default_rng(8)
    v = rng.uniform(-1, 3, (n, n, n))
    x, y = rng.standard_normal((2, n, n, n))
    lhs = np.sum(orc.step(x, v, a, dtau) * y)
    rhs = np.sum(x * orc.adjoint_step(y, v, a, dtau))
    assert lhs == pytest.approx(rhs, rel=1e-13)
    mt = update_matrix(v, a, dtau).T
    np.testing.assert_allclose(orc.adjoint_step(y, v, a, dtau).reshape(-1), mt @ y.reshape(-1), atol=1e-13)


def test_grad_v_accum_matches_finite_difference_of_one_step(orc):
    n, L = 5, 3.0
    a = L / n
    dtau = a * a / 4
    rng = np.random.default_rng(4)
    v = rng.uniform(-1, 3, (n, n, n))
    psi, lam = rng.standard_normal((2, n, n, n))
    g = orc.grad_v_accum(psi, lam, v, a, dtau)
    h = 1e-4
    for site in [(0, 0, 0), (2, 3, 1), (4, 4, 4)]:
        vp, vm = v.copy(), v.copy()
        vp[site] += h
        vm[site] -= h
        fd = (np.sum(orc.step(psi, vp, a, dtau) * lam) - np.sum(orc.step(psi, vm, a, dtau) * lam)) / (2 * h)
        assert g[site] == pytest.approx(fd, rel=1e-7, abs=1e-9)


@pytest.mark.parametrize("mask", [0, wl.ODD_X])
def test_backward_matches_central_differences(orc, mask):
    """Gradient of E + 0.3 <r^2> after T unrolled steps (renormalisation and
    symmetry re-imposition at checks) against central differences of the
    oracle's own forward evolution, h = 1e-4 (FP64)."""
    n, L, T, ce = 6, 4.0, 40, 15
    a = L / n
    dtau = a * a / 4
    v = wl.harmonic(n, L) + 0.2 * wl.grid(n, L)[2]
    psi0 = orc.init_symmetric(n, 12, mask)
    g, obs = orc.backward(psi0, v, a, dtau, T, ce, mask, 1.0, 0.3)

    def loss(vv):
        _, rec, _ = orc.evolve(psi0, vv, a, dtau, T, ce, 0.0, False, mask)
        return rec["E"] + 0.3 * rec["r2"]

    assert obs["loss"] == pytest.approx(loss(v), rel=1e-13)
    h = 1e-4
    for site in [(1, 2, 3), (3, 3, 0), (5, 0, 2)]:
        vp, vm = v.copy(), v.copy()
        vp[site] += h
        vm[site] -= h
        fd = (loss(vp) - loss(vm)) / (2 * h)
        assert g[site] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_hellmann_feynman_at_convergence(orc):
    """Near the fixed point dE/dtheta -> <psi|dV/dtheta|psi>/<psi|psi>, up to
    the O(dtau) offset between the FDTD fixed point and H's eigenvector."""
    n, L = 10, 6.0
    a = L / n
    dtau = a * a / 4
    g_basis, _ = wl.theta_basis(n, L, count=3)
    v = wl.harmonic(n, L) + 0.3 * g_basis[0]
    psi0 = orc.init_random(n, 5)
    gv, obs = orc.backward(psi0, v, a, dtau, 1500, 100, 0, 1.0, 0.0)
    psi, rec, _ = orc.evolve(psi0, v, a, dtau, 1500, 100)
    for k in range(3):
        adj = float(np.sum(gv * g_basis[k]))
        hf = float(np.sum(g_basis[k] * psi**2) / np.sum(psi**2))
        assert adj == pytest.approx(hf, rel=0.02, abs=2e-3)


# ----------------------------------------------------------------- snapshot projection

def test_projection_of_a_snapshot_gives_the_first_excited_level(orc):
    """Sec. III: a snapshot taken at tau_snap >> 1/(E2 - E1), with the
    converged ground state projected out, has the energy of the first
    excited level -- here the isotropic oscillator's p triplet, whose energy
    the A_x sector (Sec. IV) gives independently."""
    n, L = 16, 8.0
    a = L / n
    dtau = a * a / 4
    v = wl.harmonic(n, L)
    snap, _, _ = orc.evolve(orc.init_random(n, 9), v, a, dtau, int(6.0 / dtau), 100)
    ground, rec0, _ = orc.evolve(snap, v, a, dtau, 200000, 100, 1e-14)
    e1 = orc.observables(orc.project_out(snap, [ground], a), v, a)["E"]
    _, rec_odd, _ = orc.evolve(orc.init_symmetric(n, 9, wl.ODD_X), v, a, dtau, 200000, 100, 1e-14, False, wl.ODD_X)
    assert e1 == pytest.approx(rec_odd["E"], rel=1e-4)
    assert e1 > rec0["E"] + 0.9
    p = orc.project_out(snap, [ground], a)
    assert abs(np.sum(p * ground)) < 1e-10 * np.sqrt(np.sum(p * p) * np.sum(ground * ground))
    assert np.sum(p * p) * a**3 == pytest.approx(1.0, rel=1e-14)
    c = orc.combine([ground, p], [2.0, -1.0], a)
    assert np.sum(c * c) * a**3 == pytest.approx(1.0, rel=1e-14)
    assert np.sum(c * ground) / np.sum(c * p) * np.sum(p * p) / np.sum(ground * ground) == pytest.approx(-2.0, rel=1e-10)
