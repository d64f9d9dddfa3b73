"""GPU checks at the sizes of the benchmark workloads and against the
numbers the paper prints (tests/golden/paper_values.json)."""
import json
import math
import os

import numpy as np
import pytest

import workloads as wl
from conftest import GOLDEN

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fd():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_0904_0939_gb300 as fd

    return fd


def paper(key):
    return json.load(open(os.path.join(GOLDEN, "paper_values.json")))[key]


# ------------------------------------------------------------------ gradients

def test_theta_gradients_128_finite_differences_and_hellmann_feynman(fd):
    """V_theta = r^2/2 + sum_{k<16} theta_k G_k on 128^3, L = 10, 4000
    unrolled steps from the oscillator Gaussian: the adjoint gradient of E
    and <r^2> w.r.t. theta (sqrt(T) checkpointing) against central
    differences of the FP64 forward (h = 1e-4), the FP32 adjoint against the
    FP64 one, and dE/dtheta against Hellmann-Feynman <G_k>; then the same
    gradient of E + 0.3 <r^2> through torch (EnergyFn) against the central
    differences."""
    n, L, T = 128, 10.0, 4000
    G, th = wl.config_theta(n, L)
    v = wl.v_theta(n, L, th, G)
    psi0 = np.exp(-0.5 * wl.radius2(n, L))

    def solver(prec, back):
        return fd.Solver(fd.Lattice(n, L, prec),
                         fd.default_options(check_every=100, tol=0.0, backward_steps=T if back else 0))

    grads = {}
    for prec in (fd.F64, fd.F32):
        s = solver(prec, True)
        s.set_potential(v)
        s.set_psi(psi0)
        g_e, obs = s.backward(T, 1.0, 0.0)
        psi_t = s.get_psi()
        s.set_psi(psi0)
        g_r, _ = s.backward(T, 0.0, 1.0)
        grads[prec] = (np.tensordot(G, g_e, axes=3), np.tensordot(G, g_r, axes=3), obs, psi_t)
        s.close()

    def forward(theta):
        s = solver(fd.F64, False)
        s.set_potential(wl.v_theta(n, L, theta, G))
        s.set_psi(psi0)
        s.evolve(T)
        o = s.last_check()
        s.close()
        return o["energy"], o["r2"]

    h = 1e-4
    fd_e, fd_r = np.zeros(16), np.zeros(16)
    for k in range(16):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        (ep, rp), (em, rm) = forward(tp), forward(tm)
        fd_e[k] = (ep - em) / (2 * h)
        fd_r[k] = (rp - rm) / (2 * h)
    ge64, gr64, obs64, psi_t = grads[fd.F64]
    ge32, gr32, _, _ = grads[fd.F32]
    np.testing.assert_allclose(ge64, fd_e, rtol=1e-5, atol=1e-7 * np.abs(fd_e).max())
    np.testing.assert_allclose(gr64, fd_r, rtol=1e-5, atol=1e-7 * np.abs(fd_r).max())
    assert np.max(np.abs(ge32 - ge64)) <= 1e-3 * np.max(np.abs(ge64))
    assert np.max(np.abs(gr32 - gr64)) <= 1e-3 * np.max(np.abs(gr64))
    # Hellmann-Feynman: <psi_T| dV/dtheta_k |psi_T> / <psi_T|psi_T>
    w = psi_t**2 / np.sum(psi_t**2)
    hf = np.tensordot(G, w, axes=3)
    assert np.max(np.abs(ge64 - hf)) <= 2e-2 * np.max(np.abs(hf))
    # the same gradients through torch: V_theta built from theta in torch,
    # EnergyFn over fdtd_backward, theta.grad by torch's chain rule
    import torch

    dev = torch.device("cuda")
    Gt = torch.from_numpy(G).to(dev)
    r2 = torch.from_numpy(wl.radius2(n, L)).to(dev)
    psi0_t = torch.from_numpy(psi0).to(dev)
    w_r = 0.3
    want = fd_e + w_r * fd_r
    through_torch = {}
    for prec in (fd.F64, fd.F32):
        theta = torch.tensor(th, dtype=torch.float64, device=dev, requires_grad=True)
        s = solver(prec, True)
        E, R = fd.energy_fn().apply(0.5 * r2 + torch.tensordot(theta, Gt, dims=1), s, T, psi0_t)
        (E + w_r * R).backward()
        through_torch[prec] = theta.grad.cpu().numpy()
        assert float(E) == pytest.approx(grads[prec][2]["energy"], rel=1e-12)
        s.close()
    np.testing.assert_allclose(through_torch[fd.F64], want, rtol=1e-5, atol=1e-7 * np.abs(want).max())
    assert np.max(np.abs(through_torch[fd.F32] - want)) <= 1e-3 * np.max(np.abs(want))


# ------------------------------------------------------------------ full-size sampled parity

def test_anisotropic_512_sampled_sites(fd, orc):
    """The 512^3, L = 16 anisotropic workload (oscillator + 32 Gaussians) in
    the FP32 launch configuration the benchmark uses: sampled sites after 6
    steps against the oracle on each site's cone of dependence."""
    n, L, steps = 512, 16.0, 6
    a = L / n
    v32 = wl.anisotropic(n, L).astype(np.float32)
    s = fd.Solver(fd.Lattice(n, L, fd.F32), fd.default_options(check_every=1000, tol=0.0))
    s.set_potential(v32)
    s.init_symmetric(23, 0)
    psi0 = s.get_psi(dtype=np.float32)
    s0 = float(np.sum(psi0.astype(np.float64) ** 2))
    s.evolve(steps)
    sT = s.last_check()["norm"] / a**3
    got = s.get_psi(dtype=np.float32)
    scale = 1.0 / math.sqrt(s0 * a**3) / math.sqrt(sT * a**3)
    rng = np.random.default_rng(1)
    sites = [tuple(int(c) for c in rng.integers(8, n - 8, size=3)) for _ in range(16)] + [(256, 255, 9), (500, 7, 250)]
    r = steps + 1
    peak = float(np.abs(got).max())
    for (z, y, x) in sites:
        sub = psi0[z - r:z + r + 1, y - r:y + r + 1, x - r:x + r + 1].astype(np.float64)
        vs = v32[z - r:z + r + 1, y - r:y + r + 1, x - r:x + r + 1].astype(np.float64)
        want = scale * orc.steps(sub, vs, a, a * a / 4, steps)[r, r, r]
        assert got[z, y, x] == pytest.approx(want, rel=2e-5, abs=2e-5 * peak)


def test_largest_lattice_2048_sampled_sites(fd, orc):
    """n = 2048, the largest lattice the library accepts: 8.6e9 sites, so
    every linear index past plane 512 is above 2^31, and 34 GB per field.
    FP32 in the tuned TMA configuration, V = r^2/2 built in FP32 on the
    device, sampled sites (near the first and the last planes, rows and
    columns) after 6 steps against the oracle on each site's cone of
    dependence, as at 512^3."""
    import torch

    if torch.cuda.get_device_properties(0).total_memory < 240 * 2**30:
        pytest.skip("needs about 210 GB of device memory")
    n, L, steps = 2048, 64.0, 6
    a = L / n
    r = steps + 1
    dev = torch.device("cuda")
    rng = np.random.default_rng(3)
    sites = [tuple(int(c) for c in rng.integers(8, n - 8, size=3)) for _ in range(10)]
    sites += [(2039, 2039, 2039), (2040, 8, 2031), (9, 2035, 8), (1024, 1023, 2040), (513, 1, 1)]
    ax2 = torch.as_tensor(wl.axis(n, L), dtype=torch.float32, device=dev) ** 2
    v = 0.5 * ((ax2[None, None, :] + ax2[None, :, None]) + ax2[:, None, None])
    s = fd.Solver(fd.Lattice(n, L, fd.F32), fd.default_options(check_every=1000, tol=0.0))
    try:
        s.set_potential(v)

        w = 2 * r + 1
        corner = [[min(max(c - r, 0), n - w) for c in site] for site in sites]

        def boxes(t):
            # a (2r+1)^3 box around each site's cone of dependence, moved
            # inside the lattice at its faces: a box face on a lattice face
            # is the Dirichlet wall (the oracle's zero padding), any other
            # face is at least r > steps sites from the site
            return [t[lo[0]:lo[0] + w, lo[1]:lo[1] + w, lo[2]:lo[2] + w].double().cpu().numpy() for lo in corner]

        vs = boxes(v)
        del v
        torch.cuda.empty_cache()
        s.init_symmetric(23, 0)
        buf = torch.empty((n, n, n), dtype=torch.float32, device=dev)
        s.get_psi(out=buf)
        subs = boxes(buf)
        s0 = sum(float(torch.sum(buf[z0:z0 + 128].double() ** 2)) for z0 in range(0, n, 128))
        s.evolve(steps)
        sT = s.last_check()["norm"] / a**3
        s.get_psi(out=buf)
        got = [float(buf[z, y, x]) for (z, y, x) in sites]
        peak = float(buf.abs().max())
        scale = 1.0 / math.sqrt(s0 * a**3) / math.sqrt(sT * a**3)
        for site, lo, g, sub, vsub in zip(sites, corner, got, subs, vs):
            cz, cy, cx = (c - o for c, o in zip(site, lo))
            want = scale * orc.steps(sub, vsub, a, a * a / 4, steps)[cz, cy, cx]
            assert g == pytest.approx(want, rel=2e-5, abs=2e-5 * peak)
        del buf
    finally:
        s.close()
        torch.cuda.empty_cache()


def test_batch_subset_matches_separate_runs(fd):
    """Eight lattices of the 64-lattice batch (sizes 48..160, oscillator or
    soft Coulomb, four sectors) in one persistent launch vs one by one from
    the same starting fields."""
    lats = wl.config_batch()[:8]
    opts = dict(check_every=100, tol=1e-6, tol_relative=1)
    b = fd.Solver([fd.Lattice(l.n, l.length, fd.F32) for l in lats], fd.default_options(batched=1, **opts))
    starts = []
    for i, l in enumerate(lats):
        b.set_potential(l.potential().astype(np.float32), lat=i)
        b.init_symmetric(l.seed, l.mask, lat=i)
        starts.append(b.get_psi(lat=i, dtype=np.float32))
    b.evolve(200_000)
    for i, l in enumerate(lats):
        s = fd.Solver(fd.Lattice(l.n, l.length, fd.F32), fd.default_options(**opts))
        s.set_potential(l.potential().astype(np.float32))
        s.set_psi(starts[i], mask=l.mask)
        s.evolve(200_000)
        ob, os_ = b.last_check(lat=i), s.last_check()
        assert ob["steps"] == os_["steps"] and ob["energy"] == os_["energy"], i
        np.testing.assert_array_equal(b.get_psi(lat=i, dtype=np.float32), s.get_psi(dtype=np.float32))
        s.close()


# ------------------------------------------------------------------ the paper's printed values

def test_paper_oscillator_512(fd):
    """Sec. VII.D: 512^3, a = 0.02, dtau = a^2/4 = 1e-4, L = 10.24 gives
    E0 = 1.49996 (multi-resolution 128^3 -> 256^3 -> 512^3, FP32)."""
    g = paper("ho_512")
    L = g["L"]
    opts = fd.default_options(check_every=100, tol=2e-8, tol_relative=1)
    levels = [fd.Lattice(n, L, fd.F32) for n in (128, 256, 512)]
    out = fd.multires(levels, [wl.harmonic(n, L).astype(np.float32) for n in (128, 256, 512)],
                      mask=wl.SYMMETRIC_ALL, options=opts)
    e = out[-1][1]["energy"]
    assert abs(levels[-1].tau_step - g["dtau"]) < 1e-15
    assert e == pytest.approx(g["E0"], abs=1e-5)


@pytest.mark.parametrize("printed", [False, True])
def test_paper_dodecahedron_128(fd, printed):
    """Sec. VII.E: V = -100 inside the dodecahedron, 128^3, a = 0.1,
    dtau = 0.001, m = 1: the paper prints E0 = -99.78.  Both the regular
    solid and the vertex list as printed give a ground state a few hundredths
    lower (a larger effective well); checked to 0.1 % of |E0|."""
    g = paper("dodecahedron_128")
    n, a = g["n"], g["a"]
    s = fd.Solver(fd.Lattice(n, n * a, fd.F32, dtau=g["dtau"]),
                  fd.default_options(check_every=100, tol=1e-7, tol_relative=1))
    s.set_potential(wl.dodecahedron(n, printed=printed).astype(np.float32))
    s.init_symmetric(3, 0)
    steps, conv = s.evolve(400_000)
    assert conv
    e = s.last_check()["energy"]
    print(f"dodecahedron 128^3 ({'printed' if printed else 'regular'} vertices): E0 = {e:.5f}")
    assert -100.0 < e < -99.5
    assert e == pytest.approx(g["E0"], rel=1e-3)


def test_dodecahedron_24_matches_oracle(fd, orc):
    """The dodecahedral well (Eq. dodecahedronpotential) at 24^3, a = 0.1,
    dtau = 0.001, m = 1: 100 steps from the seeded random start with a check
    every 50, element by element against the oracle: FP64 to 1e-12, FP32 to
    2e-5 (max-norm relative), energies to 1e-12 / 1e-6."""
    n, a, dtau = 24, 0.1, 1e-3
    v = wl.dodecahedron(n)
    psi0 = orc.init_symmetric(n, 7, 0)
    ref, rec, _ = orc.evolve(psi0, v, a, dtau, 100, 50, 0.0, False, 0)
    for prec, tol in ((fd.F64, 1e-12), (fd.F32, 2e-5)):
        s = fd.Solver(fd.Lattice(n, n * a, prec, dtau=dtau), fd.default_options(check_every=50, tol=0.0))
        s.set_potential(v.astype(np.float32) if prec == fd.F32 else v)
        s.set_psi(psi0)
        s.evolve(100)
        got = s.get_psi()
        assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref)), prec
        assert s.last_check()["energy"] == pytest.approx(rec["E"], rel=1e-12 if prec == fd.F64 else 1e-6)
        s.close()


def test_paper_dodecahedron_512_stopping_rule(fd):
    """Sec. VII.E: 512^3, a = 0.1, dtau = 0.001, m = 1, from a random start,
    stopped when the energy changes by less than a part in 10^6 between
    checks (100 steps): the paper prints E0 = -99.97.  The same procedure
    stops at -99.973 here.  The level itself lies lower (about -99.991,
    reached only after a few hundred thousand more steps, consistent with
    the 128^3 level and the 1/R^2 scaling of the kinetic energy): with the
    well this wide the gap to the next level is ~0.01, so the change per
    check falls below the tolerance long before the excited admixture has
    decayed, and the printed number is where the criterion stops."""
    g = paper("dodecahedron_512")
    n, a = g["n"], g["a"]
    s = fd.Solver(fd.Lattice(n, n * a, fd.F32, dtau=g["dtau"]),
                  fd.default_options(check_every=100, tol=1e-6, tol_relative=1))
    import torch

    v = torch.from_numpy(wl.dodecahedron(n).astype(np.float32)).cuda()
    s.set_potential(v)
    s.init_symmetric(3, 0)
    steps, conv = s.evolve(200_000)
    e = s.last_check()["energy"]
    print(f"dodecahedron 512^3, paper's stopping rule: E0 = {e:.5f} after {steps} steps")
    assert conv
    assert e == pytest.approx(g["E0"], abs=5e-3)
    # further steps keep lowering it: the stop was not the level
    more = fd.Solver(fd.Lattice(n, n * a, fd.F32, dtau=g["dtau"]), fd.default_options(check_every=100, tol=0.0))
    more.set_potential(v)
    psi = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    more.set_psi(s.get_psi(out=psi))
    s.close()
    more.evolve(20_000)
    assert more.last_check()["energy"] < e - 1e-3
    more.close()


def test_paper_antisymmetric_z_coulomb_256(fd):
    """Sec. VII.F: A_z initial condition on the Coulomb potential of
    Eq. coulombpot, 256^3, a = 0.2, dtau = 0.01: binding energy
    E1 = -0.12507 (V_inf = 1/a)."""
    g = paper("coulomb_antisym_z_256")
    n, a = g["n"], g["a"]
    s = fd.Solver(fd.Lattice(n, n * a, fd.F32, dtau=g["dtau"], v_inf=1.0 / a),
                  fd.default_options(check_every=100, tol=1e-7, tol_relative=1))
    s.set_potential(wl.coulomb_paper(n, n * a).astype(np.float32))
    s.init_symmetric(5, wl.ODD_Z)
    steps, conv = s.evolve(400_000)
    assert conv
    assert s.last_check()["binding_energy"] == pytest.approx(g["E1"], abs=2e-4)


def test_paper_antisymmetric_z_second_state_by_projection(fd):
    """Sec. VII.F: in the A_z run on 256^3, a = 0.2, dtau = 0.01, the next
    state antisymmetric about z follows from a snapshot with the first one
    projected out (Sec. III): E2 = -0.055360.  FP64, so that the projected
    part (~1e-6 of the snapshot) keeps its precision."""
    g = paper("coulomb_antisym_z_256")
    n, a = g["n"], g["a"]
    lat = fd.Lattice(n, n * a, fd.F64, dtau=g["dtau"], v_inf=1.0 / a)
    s = fd.Solver(lat, fd.default_options(check_every=100, tol=0.0, snapshots=2))
    s.set_potential(wl.coulomb_paper(n, n * a))
    s.init_symmetric(5, wl.ODD_Z)
    s.evolve(15000)               # tau = 150: the n = 4 states have decayed
    s.snapshot_save(0)
    s.evolve(10000)               # tau = 250: the 2p_z state
    s.snapshot_save(1)
    s.snapshot_load(0)
    s.project_out([1])
    e2 = s.observables()["binding_energy"]
    assert e2 == pytest.approx(g["E2"], abs=5e-4)


def _coulomb_multires(fd, sizes, length, mask, tol):
    """Multi-resolution bootstrap (Sec. VI) on the Coulomb potential of
    Eq. coulombpot, FP32, dtau = a^2/4 and V_inf = 1/a on every level."""
    import torch

    levels = [fd.Lattice(n, length, fd.F32, v_inf=n / length) for n in sizes]
    pots = [wl.coulomb_paper_device(n, length, "cuda", torch.float32) for n in sizes]
    opts = fd.default_options(check_every=100, tol=tol, tol_relative=1)
    out = fd.multires(levels, pots, mask=mask, options=opts, max_steps=400_000)
    for s, _ in out:
        s.close()
    return [o for _, o in out]


def test_paper_coulomb_512_ground_and_first_excited(fd):
    """Sec. VII.C: Coulomb potential of Eq. coulombpot on 512^3, a = 0.05,
    dtau = a^2/4 = 6.25e-4, m = 1: binding energies E0 = -0.499 (0.2 % from
    -1/2) and E1 = -0.122 (2.4 % from -1/8).  Reached here by the
    multi-resolution bootstrap from 128^3 -- the lattice eigenvalue does not
    depend on the start -- with the A_z sector (Sec. IV) for E1.  The A_z
    sector gives the lattice 2p level itself, much closer to -1/8 than the
    printed E1, which the text quotes as 2.4 % off (a snapshot estimate); E1
    is held to that accuracy bound and E0 to the printed digits."""
    g = paper("coulomb_512")
    length = g["n"] * g["a"]
    obs0 = _coulomb_multires(fd, (128, 256, 512), length, wl.SYMMETRIC_ALL, 1e-6)[-1]
    obs1 = _coulomb_multires(fd, (128, 256, 512), length, wl.ODD_Z, 1e-6)[-1]
    print(f"Coulomb 512^3 a=0.05: E0 = {obs0['binding_energy']:.6f}, E1 = {obs1['binding_energy']:.6f}")
    assert obs0["converged"] and obs1["converged"]
    assert obs0["binding_energy"] == pytest.approx(g["E0"], abs=1e-3)
    assert abs(obs1["binding_energy"] + 0.125) <= abs(g["E1"] + 0.125)


def test_paper_multires_coulomb_1024(fd):
    """Sec. VII.G: bootstrapping 128^3 -> 256^3 -> 512^3 -> 1024^3 at fixed
    L = 25.6 (final a = 0.025) gives E0 = -0.499632; each level stops when
    E_b changes by less than a part in 10^6 between checks, which leaves the
    fine level within ~5e-5 of its limit."""
    g = paper("multires_1024")
    obs = _coulomb_multires(fd, (128, 256, 512, 1024), g["L"], wl.SYMMETRIC_ALL, 1e-6)
    print("multires Coulomb: " + ", ".join(f"{n}^3 E = {o['binding_energy']:.6f} ({o['steps']} steps)"
                                           for n, o in zip((128, 256, 512, 1024), obs)))
    assert all(o["converged"] for o in obs)
    assert obs[-1]["binding_energy"] == pytest.approx(g["E0"], abs=1e-4)
    # the levels approach the continuum -1/2 from above as a shrinks
    e = [o["binding_energy"] for o in obs]
    assert e[0] > e[1] > e[2] > e[3] > -0.5


def test_paper_dodecahedron_first_excited_128(fd):
    """Sec. VII.E: ground and first excited levels of the dodecahedral well
    (128^3, a = 0.1, dtau = 0.001), the excited one from the A_x, A_y and
    A_z sectors (Sec. IV).  The paper prints E0 = -99.78 and E1 = -99.55;
    the regular solid the text specifies (circumradius sqrt(3)(N-1)/(2 phi)
    sites) puts both lower, as if the printed well were ~0.82 of its linear
    size, so this test checks what does not depend on the size: the ratio of
    the two levels above the well floor (printed: 0.45 / 0.22 = 2.05) and the
    threefold degeneracy of the p-like level that the solid's x -> y -> z
    symmetry gives."""
    g = paper("dodecahedron_128")
    n, a = g["n"], g["a"]
    v = wl.dodecahedron(n).astype(np.float32)
    e = {}
    for mask in (0, wl.ODD_X, wl.ODD_Y, wl.ODD_Z):
        s = fd.Solver(fd.Lattice(n, n * a, fd.F32, dtau=g["dtau"]),
                      fd.default_options(check_every=100, tol=1e-8, tol_relative=1))
        s.set_potential(v)
        s.init_symmetric(3, mask)
        steps, conv = s.evolve(400_000)
        assert conv
        e[mask] = s.last_check()["energy"]
        s.close()
    e0, e1 = e[0], e[wl.ODD_X]
    print(f"dodecahedron 128^3: E0 = {e0:.5f}, E1 = {e1:.5f} / {e[wl.ODD_Y]:.5f} / {e[wl.ODD_Z]:.5f} (A_x/A_y/A_z)")
    floor = -100.0
    assert (e1 - floor) / (e0 - floor) == pytest.approx((g["E1"] - floor) / (g["E0"] - floor), rel=0.03)
    assert e[wl.ODD_Y] == pytest.approx(e1, abs=2e-4) and e[wl.ODD_Z] == pytest.approx(e1, abs=2e-4)
