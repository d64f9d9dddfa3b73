"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (stated per test):
  * FP64 path: max |psi_gpu - psi_ref| / max |psi_ref| <= 1e-12 after 100
    steps with checks; energies and radii to 1e-12 relative.
  * FP32 path: the update rounds psi to 24 bits every step (relative error
    <= 6e-8 per step, growing at most linearly over the 100 steps of a
    check interval) -> 2e-5 on psi after 100 steps; converged energies to
    1e-6 relative (the energy is second order in the error of psi).
  * integer work (random start, symmetry copies) is bit-exact.
"""
import math

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


def solver(fd, n, L, prec, **opt):
    kw = dict(check_every=100, tol=0.0)
    kw.update(opt)
    return fd.Solver(fd.Lattice(n, L, prec), fd.default_options(**kw))


# ------------------------------------------------------------------ random start

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 33])
@pytest.mark.parametrize("dist", [0, 1])
def test_random_start_matches_oracle(fd, orc, n, dist):
    s = solver(fd, n, 4.0, fd.F64)
    s.init_symmetric(77, 0, lat=0, dist=dist)
    ref = orc.init_random(n, 77, 0, dist)
    got = s.get_psi()
    if dist == 0:
        np.testing.assert_array_equal(got, ref)  # integer hash + exact scaling
    else:
        np.testing.assert_allclose(got, ref, rtol=1e-14, atol=1e-14)  # libm vs CUDA log/cos


@pytest.mark.parametrize("n", [4, 7, 8])
@pytest.mark.parametrize("mask", [wl.ODD_X, wl.SYMMETRIC_ALL, wl.ODD_Z | 0b0100, wl.ODD_X | wl.ODD_Y | wl.ODD_Z])
def test_symmetric_start_bit_exact(fd, orc, n, mask):
    s = solver(fd, n, 4.0, fd.F64)
    s.init_symmetric(5, mask)
    np.testing.assert_array_equal(s.get_psi(), orc.init_symmetric(n, 5, mask))


def test_lattice_index_selects_the_stream(fd, orc):
    lats = [fd.Lattice(6, 4.0, fd.F64), fd.Lattice(6, 4.0, fd.F64)]
    s = fd.Solver(lats, fd.default_options(tol=0.0))
    s.init_symmetric(9, 0, lat=1)
    np.testing.assert_array_equal(s.get_psi(lat=1), orc.init_random(6, 9, 1, 0))


# ------------------------------------------------------------------ evolution, FP64

@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 8, 33, 48])
def test_fp64_100_steps_match_oracle(fd, orc, n):
    L = 0.75 * n if n > 3 else 3.0
    a = L / n
    rng = np.random.default_rng(n)
    v = wl.harmonic(n, L) + rng.uniform(-0.3, 0.3, (n, n, n))
    s = solver(fd, n, L, fd.F64, check_every=30)
    s.set_potential(v)
    s.init_symmetric(11, 0)
    steps, _ = s.evolve(100)
    ref, rec, _ = orc.evolve(orc.init_random(n, 11), v, a, a * a / 4, 100, 30)
    assert steps == 100
    assert rel_max(s.get_psi(), ref) <= 1e-12
    o = s.last_check()
    assert o["energy"] == pytest.approx(rec["E"], rel=1e-12, abs=1e-13)
    assert o["r2"] == pytest.approx(rec["r2"], rel=1e-12)
    assert o["norm"] == pytest.approx(rec["S0"] * a**3, rel=1e-12)


@pytest.mark.parametrize("graphs", [0, 1])
def test_check_history_matches_oracle(fd, orc, graphs):
    """The per-check records of an FP64 evolve (t, E, <r^2>, S0 before the
    renormalisation) against the oracle's check history, through the stream
    and through the evolve graph."""
    n, L = 12, 6.0
    a = L / n
    v = wl.harmonic(n, L)
    s = solver(fd, n, L, fd.F64, check_every=20, graphs=graphs)
    s.set_potential(v)
    s.init_symmetric(8, 0)
    s.evolve(270)
    h = s.history()
    _, rec, hist = orc.evolve(orc.init_random(n, 8), v, a, a * a / 4, 270, 20)
    assert h.shape == (len(hist), 8) == (15, 8)
    np.testing.assert_array_equal(h[:, 0], hist[:, 0])
    np.testing.assert_allclose(h[:, 1], hist[:, 1], rtol=1e-12)
    np.testing.assert_allclose(h[:, 4], hist[:, 2], rtol=1e-12)
    np.testing.assert_allclose(h[:, 7], hist[:, 3], rtol=1e-12)
    np.testing.assert_allclose(h[:, 3], hist[:, 3] * a**3, rtol=1e-12)
    assert h[0, 6] == -1.0 and np.all(h[1:, 6] >= 0.0)
    np.testing.assert_allclose(h[1:, 6], np.abs(np.diff(h[:, 2])), rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("mask", [wl.ODD_X, wl.ODD_Z | wl.ODD_Y, wl.SYMMETRIC_ALL])
@pytest.mark.parametrize("n", [9, 16])
def test_fp64_sector_evolution_matches_oracle(fd, orc, n, mask):
    L = 6.0
    a = L / n
    v = wl.harmonic(n, L)
    s = solver(fd, n, L, fd.F64, check_every=25)
    s.set_potential(v)
    s.init_symmetric(3, mask)
    s.evolve(100)
    ref, rec, _ = orc.evolve(orc.init_symmetric(n, 3, mask), v, a, a * a / 4, 100, 25, 0.0, False, mask)
    assert rel_max(s.get_psi(), ref) <= 1e-12
    assert s.last_check()["energy"] == pytest.approx(rec["E"], rel=1e-12)


def test_fp64_convergence_small_ho(fd, orc):
    """The 32^3, L = 10 oscillator run to |dE| < 1e-10 between checks."""
    lat = wl.config_small_ho()
    v = lat.potential()
    s = solver(fd, lat.n, lat.length, fd.F64, tol=1e-10, tol_relative=0)
    s.set_potential(v)
    s.init_symmetric(wl.BASE_SEED, 0)
    steps, conv = s.evolve(100000)
    _, rec, _ = orc.evolve(orc.init_random(lat.n, wl.BASE_SEED), v, lat.a, lat.dtau, 100000, 100, 1e-10)
    assert conv and steps == rec["steps"]
    o = s.last_check()
    assert o["energy"] == pytest.approx(rec["E"], rel=1e-12)
    assert o["r2"] == pytest.approx(rec["r2"], rel=1e-11)


# ------------------------------------------------------------------ evolution, FP32

@pytest.mark.parametrize("n", [3, 8, 33, 48])
def test_fp32_100_steps_close_to_oracle(fd, orc, n):
    L = 0.6 * n if n > 3 else 3.0
    a = L / n
    v = wl.harmonic(n, L)
    s = solver(fd, n, L, fd.F32, check_every=50)
    s.set_potential(v)
    s.init_symmetric(8, 0)
    s.evolve(100)
    ref, rec, _ = orc.evolve(orc.init_random(n, 8), v, a, a * a / 4, 100, 50)
    assert rel_max(s.get_psi(), ref) <= 2e-5


@pytest.mark.parametrize("mask", [0, wl.ODD_X])
def test_fp32_converged_energy_within_1e6(fd, orc, mask):
    lat = wl.config_small_ho()
    v = lat.potential()
    _, rec, _ = orc.evolve(orc.init_symmetric(lat.n, 2, mask), v, lat.a, lat.dtau, 200000, 100, 1e-13, False, mask)
    # FP32 evaluation of E fluctuates between checks at ~1e-9..1e-8 relative
    # once the iteration has converged, so the run stops at 1e-8
    s = solver(fd, lat.n, lat.length, fd.F32, tol=1e-8, tol_relative=1)
    s.set_potential(v)
    s.init_symmetric(2, mask)
    steps, conv = s.evolve(200000)
    o = s.last_check()
    assert conv
    assert o["energy"] == pytest.approx(rec["E"], rel=1e-6)
    assert o["r2"] == pytest.approx(rec["r2"], rel=1e-5)


def test_bf16_storage_runs_and_stays_close(fd, orc):
    n, L = 32, 10.0
    v = wl.harmonic(n, L)
    _, rec, _ = orc.evolve(orc.init_random(n, 2), v, L / n, (L / n) ** 2 / 4, 100000, 100, 1e-12)
    s = solver(fd, n, L, fd.BF16, tol=1e-4, tol_relative=1)
    s.set_potential(v)
    s.init_symmetric(2, 0)
    s.evolve(20000)
    assert s.last_check()["energy"] == pytest.approx(rec["E"], rel=2e-3)


# ------------------------------------------------------------------ sums and transfer

@pytest.mark.parametrize("prec,tol", [(0, 1e-13), (1, 1e-6)])
def test_observables_of_a_given_field(fd, orc, prec, tol):
    n, L = 20, 7.0
    rng = np.random.default_rng(1)
    v = wl.anisotropic(n, L)
    psi = np.exp(-wl.radius2(n, L)) * (1 + 0.1 * rng.standard_normal((n, n, n)))
    if prec == 1:
        psi = psi.astype(np.float32).astype(np.float64)
        v = v.astype(np.float32).astype(np.float64)
    s = solver(fd, n, L, prec)
    s.set_potential(v)
    s.set_psi(psi)
    o = s.observables()
    ref = orc.observables(psi, v, L / n)
    assert o["energy"] == pytest.approx(ref["E"], rel=tol)
    assert o["r2"] == pytest.approx(ref["r2"], rel=tol)
    assert o["v_expect"] == pytest.approx(ref["V"], rel=tol)
    assert o["norm"] == pytest.approx(ref["S0"] * (L / n) ** 3, rel=tol)


@pytest.mark.parametrize("prec,tol", [("F64", 1e-14), ("F32", 1e-6)])
@pytest.mark.parametrize("nc,mask", [(5, 0), (8, wl.ODD_Y), (12, wl.SYMMETRIC_ALL), (68, wl.ODD_Z)])
def test_upsample_matches_oracle(fd, orc, nc, mask, prec, tol):
    """Trilinear transfer Nc^3 -> (2 Nc)^3 (Sec. VI), renormalised and with
    the coarse field's symmetry: FP64 to rounding, FP32 (separable FP32
    interpolation, FP32 start field) to a few units of FP32 rounding."""
    L = 5.0
    p = getattr(fd, prec)
    coarse = solver(fd, nc, L, p)
    coarse.set_potential(wl.harmonic(nc, L))
    coarse.init_symmetric(4, mask)
    fine = solver(fd, 2 * nc, L, p)
    fine.set_potential(wl.harmonic(2 * nc, L))
    fine.upsample_from(coarse)
    up = orc.upsample(orc.init_symmetric(nc, 4, mask))
    af = L / (2 * nc)
    up = up / math.sqrt(np.sum(up**2) * af**3)
    up = orc.impose_parity(up, mask)
    assert rel_max(fine.get_psi(), up) <= tol


def test_upsample_shape_mismatch(fd):
    a = solver(fd, 8, 4.0, fd.F64)
    b = solver(fd, 12, 4.0, fd.F64)
    b.set_potential(np.zeros((12, 12, 12)))
    a.init_symmetric(1)
    with pytest.raises(fd.FdtdError) as e:
        b.upsample_from(a)
    assert e.value.code == fd.ERR_SHAPE


def test_multires_reaches_same_energy_in_fewer_fine_steps(fd, orc):
    L = 8.0
    opts = fd.default_options(tol=1e-9, tol_relative=1)
    levels = [fd.Lattice(16, L, fd.F64), fd.Lattice(32, L, fd.F64)]
    pots = [wl.harmonic(16, L), wl.harmonic(32, L)]
    out = fd.multires(levels, pots, options=opts)
    _, rec, _ = orc.evolve(orc.init_random(32, 904939), pots[1], L / 32, (L / 32) ** 2 / 4, 100000, 100, 1e-12)
    assert out[-1][1]["energy"] == pytest.approx(rec["E"], rel=1e-7)
    direct, o = fd.solve(pots[1], 32, L, fd.F64, options=opts)
    assert out[-1][1]["steps"] < o["steps"]


# ------------------------------------------------------------------ errors

@pytest.mark.parametrize("vdtype", [np.float64, np.float32])
def test_input_guards(fd, vdtype):
    """FP64 host input goes through the staging conversion, FP32 host input
    into an FP32 lattice is copied straight into place and checked there:
    both refuse non-finite values and 1 + dtau V / 2 <= 0."""
    s = solver(fd, 8, 4.0, fd.F32)
    v = np.zeros((8, 8, 8), dtype=vdtype)
    v[1, 2, 3] = np.nan
    with pytest.raises(fd.FdtdError) as e:
        s.set_potential(v)
    assert e.value.code == fd.ERR_NONFINITE
    v[1, 2, 3] = np.inf
    with pytest.raises(fd.FdtdError) as e:
        s.set_potential(v)
    assert e.value.code == fd.ERR_NONFINITE
    a = 4.0 / 8
    v = np.full((8, 8, 8), -2.5 / (a * a / 4), dtype=vdtype)  # 1 + dtau V / 2 < 0
    with pytest.raises(fd.FdtdError) as e:
        s.set_potential(v)
    assert e.value.code == fd.ERR_UNSTABLE_DT
    with pytest.raises(fd.FdtdError) as e:
        s.evolve(10)
    assert e.value.code == fd.ERR_STATE
    with pytest.raises(fd.FdtdError) as e:
        s.init_symmetric(1, 0b11)
    assert e.value.code == fd.ERR_INVALID_ARG


def test_pinned_host_input_is_read_before_the_call_returns(fd):
    """A host input is borrowed for the call only, also from pinned memory
    (where the copies are asynchronous): overwriting the buffer right after
    fdtd_set_potential / fdtd_set_psi returns changes nothing."""
    import torch

    n, L = 64, 19.2
    v = (wl.harmonic(n, L) + 0.1 * np.cos(wl.radius2(n, L))).astype(np.float32)
    psi = np.exp(-0.5 * wl.radius2(n, L)).astype(np.float32)
    out = []
    for pinned in (False, True):
        s = solver(fd, n, L, fd.F32, check_every=20)
        if pinned:
            vp, pp = torch.from_numpy(v.copy()).pin_memory(), torch.from_numpy(psi.copy()).pin_memory()
            s.set_potential(vp)
            vp.fill_(1.0e6)
            s.set_psi(pp)
            pp.fill_(-3.0)
        else:
            s.set_potential(torch.from_numpy(v).cuda())
            s.set_psi(torch.from_numpy(psi).cuda())
        s.evolve(60)
        out.append(s.get_psi(dtype=np.float32))
        s.close()
    np.testing.assert_array_equal(out[0], out[1])


def test_zero_field_reports_nonfinite(fd):
    s = solver(fd, 8, 4.0, fd.F64)
    s.set_potential(np.zeros((8, 8, 8)))
    s.set_psi(np.zeros((8, 8, 8)))
    with pytest.raises(fd.FdtdError) as e:
        s.evolve(10)
    assert e.value.code == fd.ERR_NONFINITE


# ------------------------------------------------------------------ full size, sampled

def _cone(orc, psi, v, a, dtau, steps, site):
    r = steps + 1
    z, y, x = site
    sub = psi[z - r:z + r + 1, y - r:y + r + 1, x - r:x + r + 1]
    vs = v[z - r:z + r + 1, y - r:y + r + 1, x - r:x + r + 1]
    out = orc.steps(sub, vs, a, dtau, steps)
    return out[r, r, r]


def test_full_size_256_sampled_sites(fd, orc):
    """Coulomb workload at 256^3, L = 40 (FP32, the benchmark launch shapes):
    sampled interior sites after 6 steps against the oracle applied to each
    site's cone of dependence."""
    n, L, steps = 256, 40.0, 6
    a = L / n
    v = wl.coulomb_soft(n, L)
    s = solver(fd, n, L, fd.F32, check_every=1000)
    s.set_potential(v)
    s.init_symmetric(21, 0)
    psi0 = s.get_psi()
    s0 = float(np.sum(psi0**2))
    s.evolve(steps)
    sT = s.last_check()["norm"] / a**3
    got = s.get_psi()
    scale = 1.0 / math.sqrt(s0 * a**3) / math.sqrt(sT * a**3)
    v32 = v.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(0)
    sites = [(int(rng.integers(8, n - 8)), int(rng.integers(8, n - 8)), int(rng.integers(8, n - 8)))
             for _ in range(24)] + [(128, 128, 128), (8, 8, 8), (247, 247, 247), (127, 128, 129)]
    for site in sites:
        want = scale * _cone(orc, psi0, v32, a, a * a / 4, steps, site)
        assert got[site] == pytest.approx(want, rel=2e-5, abs=2e-5 * np.abs(got).max())


# ------------------------------------------------------------------ temporal blocking

@pytest.mark.parametrize("n", [64, 96, 132, 256])
def test_blocked_kernels_bit_identical_to_single_steps(fd, n):
    """The TMA-streamed kernel at depth K reproduces K plain steps bit for
    bit (ragged x/y tiles and z-chunks at n = 132; check cadence not a
    multiple of K), also with short spans that run on into the next tile
    column or leave a ragged last chunk (down to one plane) and in the
    configuration the autotuner picks, the balanced and the columns-first
    partitions."""
    L = 0.3 * n
    rng = np.random.default_rng(n)
    v = (wl.harmonic(n, L) + rng.uniform(-0.5, 0.5, (n, n, n))).astype(np.float32)
    outs = {}
    variants = [("plain", dict(stencil_kernel=1)), ("direct", dict(stencil_kernel=2)), ("k1", dict(temporal_depth=1)),
                ("k2", dict(temporal_depth=2)), ("k3", dict(temporal_depth=3)),
                ("k1z2", dict(temporal_depth=1, zchunk=2)), ("k1z3", dict(temporal_depth=1, zchunk=3)),
                ("k2z9", dict(temporal_depth=2, zchunk=9)), ("k3z12", dict(temporal_depth=3, zchunk=12)),
                ("k2z1", dict(temporal_depth=2, zchunk=1)), ("k3z1", dict(temporal_depth=3, zchunk=1)),
                ("k3z200", dict(temporal_depth=3, zchunk=200)),
                ("k1bal", dict(temporal_depth=1, zchunk=-1)), ("k2bal", dict(temporal_depth=2, zchunk=-1)),
                ("k3bal", dict(temporal_depth=3, zchunk=-1)),
                ("k1col", dict(temporal_depth=1, zchunk=-2)), ("k2col", dict(temporal_depth=2, zchunk=-2)),
                ("k3col", dict(temporal_depth=3, zchunk=-2)),
                ("auto", dict(autotune=1))]
    for name, kw in variants:
        s = solver(fd, n, L, fd.F32, check_every=50, **kw)
        s.set_potential(v)
        s.init_symmetric(31, wl.ODD_Z)
        s.evolve(100)
        outs[name] = s.get_psi(dtype=np.float32)
        if name in ("plain", "direct"):
            assert s.tuned_kernel() == (0, 0)
        elif name.startswith("k"):
            assert s.tuned_kernel() == (128 if n > 64 else 64, 16), name
        s.close()
    for name, _ in variants[1:]:
        np.testing.assert_array_equal(outs[name], outs["plain"], err_msg=name)


@pytest.mark.parametrize("n", [32, 68, 136])
def test_bf16_kernels_match_zmarch(fd, n):
    """BF16 storage: the direct four-site kernel (stencil_kernel 2), the
    temporally blocked TMA kernel (n % 8 == 0: BF16 psi boxes, every level
    rounded to BF16 as a stored step is; depths 1-3, both tile widths,
    spans and partitions), the z-marching kernel (stencil_kernel 1) and the
    autotuner's choice give the same bits after 100 steps with checks."""
    L = 0.3 * n
    rng = np.random.default_rng(n + 1)
    v = (wl.harmonic(n, L) + rng.uniform(-0.5, 0.5, (n, n, n))).astype(np.float32)
    variants = [("plain", dict(stencil_kernel=1)), ("direct", dict(stencil_kernel=2)), ("auto", {})]
    if n % 8 == 0:
        variants += [(f"k{d}t{t}z{z}", dict(temporal_depth=d, tile_x=t, zchunk=z))
                     for d in (1, 2, 3) for t in (64, 128) for z in (0, -1, -2, 7)]
    outs = {}
    for name, kw in variants:
        s = solver(fd, n, L, fd.BF16, check_every=50, **kw)
        s.set_potential(v)
        s.init_symmetric(17, wl.ODD_Y)
        s.evolve(100)
        outs[name] = (s.get_psi(dtype=np.float32), s.last_check()["energy"])
        if name.startswith("k"):
            assert s.tuned_kernel()[0] == kw["tile_x"], name
        s.close()
    for name, _ in variants[1:]:
        np.testing.assert_array_equal(outs[name][0], outs["plain"][0], err_msg=name)
        assert outs[name][1] == outs["plain"][1], name


# ------------------------------------------------------------------ evolve graph

@pytest.mark.parametrize("prec,n,kw", [("F32", 64, {}), ("F32", 36, {}), ("F32", 48, dict(temporal_depth=3)),
                                       ("F64", 24, {}), ("BF16", 32, {})])
def test_evolve_graph_matches_stream(fd, prec, n, kw):
    """fdtd_evolve through the CUDA graph whose while loop the convergence
    check ends on the device gives the stream path's result bit for bit: a
    run the check stops, a run stopped by max_steps with a remainder after
    the last full pair of segments, and an evolve continuing from it."""
    L = 0.3 * n
    v = wl.harmonic(n, L) + 0.1 * np.cos(wl.radius2(n, L))
    runs = {}
    for g in (0, 1):
        res = []
        s = solver(fd, n, L, getattr(fd, prec), check_every=50, tol=1e-6, tol_relative=1, graphs=g, **kw)
        s.set_potential(v)
        s.init_symmetric(5, wl.ODD_X)
        res.append(s.evolve(100_000))
        res.append(s.last_check())
        res.append(s.get_psi())
        u = solver(fd, n, L, getattr(fd, prec), check_every=50, tol=0.0, graphs=g, **kw)
        u.set_potential(v)
        u.init_symmetric(6, 0)
        res.append(u.evolve(730))
        res.append(u.last_check())
        res.append(u.get_psi())
        res.append(u.evolve(250))
        res.append(u.last_check())
        res.append(u.get_psi())
        graphs = s.stats()["graph_launches"] + u.stats()["graph_launches"]
        assert (graphs >= 3) if g else (graphs == 0)
        runs[g] = res
    assert runs[0][0][1] and runs[0][0][0] < 100_000  # the first run converged
    for a, b in zip(runs[0], runs[1]):
        if isinstance(a, np.ndarray):
            np.testing.assert_array_equal(a, b)
        else:
            assert a == b


@pytest.mark.parametrize("profiling", [False, True])
def test_lattices_of_a_handle_evolve_concurrently_as_alone(fd, profiling):
    """The graph loops of a handle's lattices run at the same time on their
    own streams; every lattice ends bit-identical to the same lattice
    evolved alone: different sizes, masks and precisions, one that
    converges early, one stopped by max_steps, and a second evolve."""
    specs = [(64, fd.F32, wl.ODD_X, 11), (36, fd.F32, 0, 12), (24, fd.F64, wl.SYMMETRIC_ALL, 13),
             (48, fd.F32, wl.ODD_Z | wl.ODD_Y, 14)]
    opts = dict(check_every=50, tol=1e-6, tol_relative=1)

    def potential(i, n):
        # the 36^3 lattice is a free particle in the box: a small gap, slow to converge
        L = 0.3 * n
        return np.zeros((n, n, n)) if n == 36 else wl.harmonic(n, L) + 0.1 * np.cos(wl.radius2(n, L)) + 0.05 * i

    together = fd.Solver([fd.Lattice(n, 0.3 * n, p) for n, p, _, _ in specs], fd.default_options(**opts))
    together.set_profiling(profiling)
    psi0 = []
    for i, (n, _, mask, seed) in enumerate(specs):
        together.set_potential(potential(i, n), lat=i)
        together.init_symmetric(seed, mask, lat=i)  # the start hashes the lattice index too
        psi0.append(together.get_psi(lat=i))
    first = together.evolve(1900)
    res_t = [(together.last_check(lat=i), together.get_psi(lat=i)) for i in range(len(specs))]
    second = together.evolve(400)
    res_t2 = [(together.last_check(lat=i), together.get_psi(lat=i)) for i in range(len(specs))]
    assert together.stats()["graph_launches"] >= len(specs)
    together.close()
    for i, sp in enumerate(specs):
        alone = fd.Solver(fd.Lattice(sp[0], 0.3 * sp[0], sp[1]), fd.default_options(**opts))
        alone.set_profiling(profiling)
        alone.set_potential(potential(i, sp[0]))
        alone.set_psi(psi0[i], mask=sp[2])
        alone.evolve(1900)
        assert alone.last_check() == res_t[i][0], i
        np.testing.assert_array_equal(alone.get_psi(), res_t[i][1], err_msg=str(i))
        alone.evolve(400)
        assert alone.last_check() == res_t2[i][0], i
        np.testing.assert_array_equal(alone.get_psi(), res_t2[i][1], err_msg=str(i))
        alone.close()
    assert first[0] == max(r[0]["steps"] for r in res_t)
    assert any(r[0]["converged"] for r in res_t)


# ------------------------------------------------------------------ adjoint

@pytest.mark.parametrize("n,mask,T,ce", [(8, 0, 40, 15), (12, wl.ODD_X, 57, 10), (9, wl.SYMMETRIC_ALL, 30, 7)])
def test_backward_matches_oracle(fd, orc, n, mask, T, ce):
    """dL/dV of L = E + 0.3 <r^2> after T steps (sqrt(T) checkpoints,
    checks inside segments, symmetry projection) against the oracle's
    full-trajectory adjoint: FP64 to 1e-10, FP32 to 1e-4 (max-norm relative)."""
    L = 0.5 * n
    a = L / n
    v = wl.harmonic(n, L) + 0.1 * wl.grid(n, L)[2] ** 2
    psi0 = orc.init_symmetric(n, 4, mask)
    ref, obs = orc.backward(psi0, v, a, a * a / 4, T, ce, mask, 1.0, 0.3)
    for prec, tol in ((fd.F64, 1e-10), (fd.F32, 1e-4)):
        s = solver(fd, n, L, prec, check_every=ce, backward_steps=T)
        s.set_potential(v)
        s.set_psi(psi0, mask=mask)
        g, o = s.backward(T, 1.0, 0.3)
        assert rel_max(g, ref) <= tol, prec
        assert o["energy"] == pytest.approx(obs["E"], rel=1e-12 if prec == fd.F64 else 1e-6)


def test_backward_fp32_across_tiles_matches_oracle(fd, orc):
    """The FP32 adjoint at n = 132: the four-site adjoint pass and the
    blocked forward cover several 128-wide tiles with a ragged 4-site tail
    and many z-chunks.  dL/dV of L = E + 0.3 <r^2> after T = 24 steps with
    checks every 10 (A_x projection), element by element against the
    oracle's full-trajectory adjoint to 1e-4 (max-norm relative)."""
    n, L, T, ce, mask = 132, 10.0, 24, 10, wl.ODD_X
    a = L / n
    v = wl.anisotropic(n, L)
    psi0 = orc.init_symmetric(n, 5, mask)
    ref, obs = orc.backward(psi0, v, a, a * a / 4, T, ce, mask, 1.0, 0.3)
    s = solver(fd, n, L, fd.F32, check_every=ce, backward_steps=T)
    s.set_potential(v)
    s.set_psi(psi0, mask=mask)
    g, o = s.backward(T, 1.0, 0.3)
    assert rel_max(g, ref) <= 1e-4
    assert o["energy"] == pytest.approx(obs["E"], rel=1e-6)
    s.close()


# ------------------------------------------------------------------ snapshots

@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 2e-3)])
def test_snapshot_projection_matches_oracle(fd, orc, prec, tol):
    """Sec. III projection on the GPU (save, evolve, load, project) against
    the oracle's definition on the same fields, FP64 to 1e-9 (the projected
    part is ~1e-3 of the snapshot, so rounding is amplified), FP32 to 2e-3;
    and the Sec. VI combination."""
    n, L = 16, 8.0
    a = L / n
    dtau = a * a / 4
    v = wl.harmonic(n, L)
    s = solver(fd, n, L, prec, snapshots=2, tol=0.0)
    s.set_potential(v)
    s.init_symmetric(9, 0)
    s.evolve(int(6.0 / dtau) // 100 * 100)
    s.snapshot_save(0)
    snap = s.get_psi()
    s.evolve(20000)  # tau = 1250: the ground state
    s.snapshot_save(1)
    ground = s.get_psi()
    s.snapshot_load(0)
    s.project_out([1])
    want = orc.project_out(snap, [ground], a)
    assert rel_max(s.get_psi(), want) <= tol
    assert s.observables()["energy"] == pytest.approx(orc.observables(want, v, a)["E"], rel=tol)
    s.combine([0, 1], [0.5, -2.0])
    assert rel_max(s.get_psi(), orc.combine([snap, ground], [0.5, -2.0], a)) <= (1e-12 if prec == 0 else 1e-5)
