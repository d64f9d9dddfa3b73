"""Complex potentials on the GPU (FDTD_C64 / FDTD_C32 lattices) against the
complex oracle, through the C ABI.

Tolerances: C64 as the FP64 path (max |dpsi| / max |psi| <= 1e-12 after 100
steps with checks, energies to 1e-12 relative); C32 as the FP32 path (2e-5
on psi after 100 steps, converged energies to 1e-6)."""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_0904_0939_gb300 as fd

    return fd


def rel_max(got, ref):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def cap_potential(n, L):
    """oscillator + a bump, with an absorbing layer in the outer quarter"""
    return (wl.harmonic(n, L) + 0.3 * np.cos(wl.grid(n, L)[2])) - 1j * wl.absorbing_layer(n, L, 0.25 * L, 2.0)


@pytest.mark.parametrize("n,mask", [(20, 0), (13, wl.ODD_X), (33, wl.SYMMETRIC_ALL)])
def test_complex_evolution_matches_oracle(fd, orc, n, mask):
    """100 steps with a check every 50 from the seeded start (real part
    random, imaginary part zero), absorbing layer on: psi element by element
    and the complex energy of the last check."""
    L = 0.4 * n
    a = L / n
    v = cap_potential(n, L)
    start = orc.init_symmetric(n, 11, mask) + 0j
    ref, rec = orc.cevolve(start, v, a, a * a / 4, 100, 50, mask=mask)
    for prec, tol in ((fd.C64, 1e-12), (fd.C32, 2e-5)):
        s = fd.Solver(fd.Lattice(n, L, prec), fd.default_options(check_every=50, tol=0.0))
        s.set_potential(v if prec == fd.C64 else v.astype(np.complex64))
        s.init_symmetric(11, mask)
        s.evolve(100)
        got = s.get_psi()
        assert got.dtype == np.complex128
        assert rel_max(got, ref) <= tol, prec
        o = s.last_check()
        etol = 1e-12 if prec == fd.C64 else 1e-5
        assert abs(complex(o["energy"], o["energy_imag"]) - rec["E"]) <= etol * abs(rec["E"]), prec
        assert o["r2"] == pytest.approx(rec["r2"], rel=etol)
        s.close()


def test_complex_sums_of_a_given_field(fd, orc):
    """observables of an arbitrary complex field: E = <psi|H|psi>/<psi|psi>,
    <V>, <r^2> and the norm against the oracle."""
    n, L = 24, 7.0
    a = L / n
    rng = np.random.default_rng(2)
    v = cap_potential(n, L)
    psi = rng.standard_normal((n, n, n)) + 1j * rng.standard_normal((n, n, n))
    ref = orc.cobservables(psi, v, a)
    s = fd.Solver(fd.Lattice(n, L, fd.C64), fd.default_options(tol=0.0))
    s.set_potential(v)
    s.set_psi(psi)
    o = s.observables()
    assert complex(o["energy"], o["energy_imag"]) == pytest.approx(ref["E"], rel=1e-13)
    assert o["r2"] == pytest.approx(ref["r2"], rel=1e-13)
    assert o["v_expect"] == pytest.approx(ref["V"].real, rel=1e-13)
    assert o["norm"] == pytest.approx(ref["S0"] * a**3, rel=1e-13)
    s.close()


def test_complex_oscillator_ground_level(fd, orc):
    """V = w2 r^2 / 2 with w2 = 1 + 0.4i on 32^3, L = 8, converged from the
    Gaussian start: the level equals the oracle's converged level (C64 to
    1e-10, C32 to 1e-6) and lies within the lattice error of (3/2) sqrt(w2)."""
    n, L, w2 = 32, 8.0, 1.0 + 0.4j
    a = L / n
    v = wl.complex_oscillator(n, L, w2)
    start = np.exp(-0.5 * wl.radius2(n, L)) + 0j
    _, rec = orc.cevolve(start, v, a, a * a / 4, 200000, 100, 1e-12, True)
    for prec, tol in ((fd.C64, 1e-10), (fd.C32, 1e-6)):
        s = fd.Solver(fd.Lattice(n, L, prec),
                      fd.default_options(check_every=100, tol=1e-12 if prec == fd.C64 else 1e-8, tol_relative=1))
        s.set_potential(v)
        s.set_psi(start)
        steps, conv = s.evolve(200000)
        assert conv
        o = s.last_check()
        e = complex(o["energy"], o["energy_imag"])
        assert abs(e - rec["E"]) <= tol * abs(rec["E"]), (prec, e, rec["E"])
        assert abs(e - 1.5 * np.sqrt(w2)) < 0.1
        s.close()


def test_complex_transfer_and_graph_path(fd, orc):
    """The trilinear transfer of both parts (Sec. VI) 14^3 -> 28^3 with the
    renormalisation and the A_y mask, against the oracle's transfer; then the
    graph and stream forms of evolve give the same bits."""
    nc, L = 14, 6.0
    vc, vf = cap_potential(nc, L), cap_potential(2 * nc, L)
    c = fd.Solver(fd.Lattice(nc, L, fd.C64), fd.default_options(check_every=20, tol=0.0))
    c.set_potential(vc)
    c.init_symmetric(3, wl.ODD_Y)
    c.evolve(60)
    coarse = c.get_psi()
    out = {}
    for graphs in (0, 1):
        f = fd.Solver(fd.Lattice(2 * nc, L, fd.C64), fd.default_options(check_every=20, tol=0.0, graphs=graphs))
        f.set_potential(vf)
        f.upsample_from(c)
        up = f.get_psi()
        want = orc.cupsample(coarse)
        want = want / np.sqrt(np.sum(np.abs(want) ** 2) * (L / (2 * nc)) ** 3)
        assert rel_max(up, want) <= 1e-13
        f.evolve(90)
        out[graphs] = (f.get_psi(), f.last_check())
        f.close()
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1]["energy"] == out[1][1]["energy"] and out[0][1]["energy_imag"] == out[1][1]["energy_imag"]
    c.close()


def test_complex_lattice_refusals(fd):
    """Real fields into complex lattices (and complex into real ones), and the
    real-only calls, are refused with FDTD_ERR_INVALID_ARG."""
    n, L = 8, 4.0
    s = fd.Solver(fd.Lattice(n, L, fd.C32), fd.default_options(tol=0.0, backward_steps=10))
    s.set_potential(wl.harmonic(n, L))  # a real potential is allowed (V_I = 0)
    with pytest.raises(fd.FdtdError) as e:
        s.set_psi(np.zeros((n, n, n)))
    assert e.value.code == fd.ERR_INVALID_ARG
    s.set_psi(np.ones((n, n, n), dtype=np.complex64))
    with pytest.raises(fd.FdtdError):
        s.backward(5)
    with pytest.raises(fd.FdtdError):
        s.get_psi(dtype=np.float64)
    r = fd.Solver(fd.Lattice(n, L, fd.F64), fd.default_options(tol=0.0))
    with pytest.raises(fd.FdtdError):
        r.set_potential(wl.harmonic(n, L) + 0.1j)
    with pytest.raises(fd.FdtdError):
        fd.Solver(fd.Lattice(n, L, fd.C64), fd.default_options(boundary=1))
    s.close()
    r.close()
