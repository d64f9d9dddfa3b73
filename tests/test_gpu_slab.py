"""The z-slab decomposition of Sec. V on one GPU: several slabs of one
lattice in one process (halos copied between their buffers, sums added),
each driven through the fdtd_slab_* C ABI, against the whole-lattice FP32
solver (same stencil arithmetic; psi to 1e-6 of max |psi| and E, <r^2> to
1e-7: the slab sums share the whole-lattice sums' FP32 per-site arithmetic
but cut the planes into other partial sums, so the energies and the
renormalisation factors may differ by a rounding) and the FP64 oracle (2e-5,
the FP32 tolerance).  The cases cover one slab (both lattice faces in one
buffer), two and three slabs, the thinnest slabs (nz_own = halo), passes of
depth 1, 2 and 3, partial passes before a check, and the x / y symmetry
masks."""
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


def _start(n, seed=5):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, (n, n, n))


@pytest.mark.parametrize("n,parts,halo,mask,steps,every", [
    (64, 1, 3, 0, 250, 100),
    (64, 2, 3, 0, 250, 100),
    (64, 3, 3, wl.ODD_X, 250, 100),
    (40, 3, 2, wl.ODD_Y, 131, 50),
    (12, 4, 3, 0, 120, 40),           # slabs of three planes: a neighbour's halo is all its own planes
    (36, 2, 1, wl.ODD_X | wl.ODD_Y, 90, 30),
])
def test_slabs_match_the_whole_lattice_and_the_oracle(fd, orc, n, parts, halo, mask, steps, every):
    from paper_0904_0939_gb300 import slab

    L = 0.3 * n
    a = L / n
    v = wl.anisotropic(n, L)
    start = _start(n)
    slabs = [slab.Slab(n, L, z0, k, halo) for z0, k in slab.partition(n, parts)]
    try:
        for s in slabs:
            s.load(v, which="v")
            s.load(start, 0)
        comm = slab.LocalComm(slabs)
        cur, rec, checks = slab.evolve(comm, n, L, steps, every, mask_xy=mask)
        got = slab.gather(slabs, cur)
    finally:
        for s in slabs:
            s.close()
    assert rec["steps"] == steps and checks == steps // every + 1 + (steps % every != 0)

    whole = fd.Solver(fd.Lattice(n, L, fd.F32), fd.default_options(check_every=every, tol=0.0))
    whole.set_potential(v)
    whole.set_psi(start, mask=mask)
    whole.evolve(steps)
    ref32 = whole.get_psi().astype(np.float64)
    o = whole.last_check()
    whole.close()
    assert rel_max(got, ref32) <= 1e-6
    assert rec["E"] == pytest.approx(o["energy"], rel=1e-7)
    assert rec["r2"] == pytest.approx(o["r2"], rel=1e-7)

    ref, orec, _ = orc.evolve(start, v, a, a * a / 4, steps, every, mask=mask)
    assert rel_max(got, ref) <= 2e-5
    assert rec["E"] == pytest.approx(orec["E"], rel=1e-5)


@pytest.mark.parametrize("parts,halo", [(2, 3), (3, 2)])
def test_inside_out_passes_match_plain_passes(fd, parts, halo):
    """The inside-out pass (both ends of every slab, their exchange, then the
    interior) gives the same bits as whole-slab passes, and as the whole
    lattice's stencil."""
    from paper_0904_0939_gb300 import slab

    n, L = 48, 12.0
    v = wl.anisotropic(n, L)
    start = _start(n, 3)
    out = {}
    for inside_out in (True, False):
        slabs = [slab.Slab(n, L, z0, k, halo) for z0, k in slab.partition(n, parts)]
        try:
            for s in slabs:
                s.load(v, which="v")
                s.load(start, 0)
            cur, rec, _ = slab.evolve(slab.LocalComm(slabs), n, L, 170, 50, inside_out=inside_out)
            out[inside_out] = (slab.gather(slabs, cur), rec["E"])
        finally:
            for s in slabs:
                s.close()
    np.testing.assert_array_equal(out[True][0], out[False][0])
    assert out[True][1] == out[False][1]


def test_two_slabs_at_512_match_the_whole_lattice(fd):
    """The benchmark's lattice size: 512^3 cut into two slabs (inside-out
    passes), 30 steps with a check every 10, against the whole-lattice solver
    on the same start, compared on the device: psi to 1e-6 of max |psi|, E to
    1e-7."""
    import torch

    from paper_0904_0939_gb300 import slab

    n, L = 512, 25.6
    dev = torch.device("cuda")
    v = wl.anisotropic_device(n, L, dev, dtype=torch.float32)
    g = torch.Generator(device=dev).manual_seed(5)
    start = torch.rand((n, n, n), generator=g, device=dev, dtype=torch.float32) * 2 - 1
    whole = fd.Solver(fd.Lattice(n, L, fd.F32), fd.default_options(check_every=10, tol=0.0))
    whole.set_potential(v)
    whole.set_psi(start)
    whole.evolve(30)
    ref = torch.empty_like(start)
    whole.get_psi(out=ref)
    e_ref = whole.last_check()["energy"]
    whole.close()
    slabs = [slab.Slab(n, L, z0, k, 3) for z0, k in slab.partition(n, 2)]
    try:
        for s in slabs:
            h, k = s.halo, s.nz_own
            lo, hi = max(0, s.z_first - h), min(n, s.z_first + k + h)
            b0 = lo - (s.z_first - h)
            s.v[b0:b0 + hi - lo].copy_(v[lo:hi])
            s.psi[0].zero_()
            s.psi[0][b0:b0 + hi - lo].copy_(start[lo:hi])
        cur, rec, _ = slab.evolve(slab.LocalComm(slabs), n, L, 30, 10, inside_out=True)
        got = torch.cat([s.own(cur) for s in slabs], dim=0)
        err = float((got - ref).abs().max() / ref.abs().max())
    finally:
        for s in slabs:
            s.close()
    assert err <= 1e-6
    assert rec["E"] == pytest.approx(e_ref, rel=1e-7)


def test_slab_sums_add_up_to_the_lattice_sums(fd, orc):
    """the partial sums of three slabs of a given field, added, give the oracle's
    E, <r^2>, <V> and norm of the same (FP32-rounded) field to 1e-6, the FP32
    tolerance of the whole-lattice sums, whose per-site arithmetic they share"""
    from paper_0904_0939_gb300 import slab

    n, L = 48, 9.0
    rng = np.random.default_rng(1)
    v = wl.anisotropic(n, L).astype(np.float32).astype(np.float64)
    psi = np.exp(-wl.radius2(n, L)) * (1 + 0.1 * rng.standard_normal((n, n, n)))
    psi = psi.astype(np.float32).astype(np.float64)
    slabs = [slab.Slab(n, L, z0, k, 3) for z0, k in slab.partition(n, 3)]
    try:
        for s in slabs:
            s.load(v, which="v")
            s.load(psi, 1)
        total = slab.LocalComm(slabs).allreduce([s.sums(1) for s in slabs])
    finally:
        for s in slabs:
            s.close()
    ref = orc.observables(psi, v, L / n)
    got = slab.check_values(total, L, n)
    assert got["E"] == pytest.approx(ref["E"], rel=1e-6)
    assert got["r2"] == pytest.approx(ref["r2"], rel=1e-6)
    assert got["V"] == pytest.approx(ref["V"], rel=1e-6)
    assert got["norm"] == pytest.approx(ref["S0"] * (L / n) ** 3, rel=1e-6)


def test_slab_create_refusals(fd):
    import torch

    from paper_0904_0939_gb300 import slab

    for args in ((30, 0, 30, 3),      # n % 4 != 0
                 (32, 0, 32, 4),      # halo above the deepest temporal block
                 (32, 0, 2, 3),       # halo thicker than the own planes
                 (32, 30, 4, 1)):     # slab beyond the lattice
        with pytest.raises(fd.FdtdError) as e:
            slab.Slab(args[0], 8.0, args[1], args[2], args[3])
        assert e.value.code == fd.ERR_INVALID_ARG
    with pytest.raises(fd.FdtdError) as e:
        slab.Slab(32, 8.0, 0, 16, 3, dtau=(8.0 / 32) ** 2 / 2)  # dtau above m a^2 / 3
    assert e.value.code == fd.ERR_UNSTABLE_DT
    s = slab.Slab(32, 8.0, 0, 16, 3)
    with pytest.raises(fd.FdtdError):
        s.steps(0, 4)  # deeper than the halo
    with pytest.raises(fd.FdtdError):
        s.steps(0, 3, 5, 4)  # an inverted plane range
    with pytest.raises(fd.FdtdError):
        s.steps(0, 3, 0, 17)  # beyond the own planes
    s.steps(0, 3, 4, 4)  # an empty range does nothing
    with pytest.raises(fd.FdtdError):
        s.scale(0, 1, 1.0, mask=0b110000)  # z symmetry needs the whole z axis
    with pytest.raises(fd.FdtdError):
        s.scale(1, 1, 1.0, mask=wl.ODD_X)  # mirrored in place
    s.scale(1, 1, 2.0)  # in place without a mask
    s.close()
    torch.cuda.synchronize()
