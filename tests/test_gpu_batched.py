"""Batched persistent driver (one cooperative launch for every lattice).

Every lattice of a batched handle must end bit-identical to a separate
fdtd_evolve of the same lattice (same update arithmetic, same reduction
order, same checks), and close to the oracle."""
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


def run_batch(fd, lats, pots, masks, seeds, batched, max_steps, **opt):
    kw = dict(check_every=100, tol=1e-6, tol_relative=1, batched=int(batched))
    kw.update(opt)
    if batched:
        s = fd.Solver([fd.Lattice(l.n, l.length, fd.F32) for l in lats], fd.default_options(**kw))
        for i, (v, m, sd) in enumerate(zip(pots, masks, seeds)):
            s.set_potential(v.astype(np.float32), lat=i)
            s.init_symmetric(sd, m, lat=i)
        s.evolve(max_steps)
        out = [(s.get_psi(lat=i, dtype=np.float32), s.last_check(lat=i)) for i in range(len(lats))]
        s.close()
        return out
    out = []
    for i, (l, v, m, sd) in enumerate(zip(lats, pots, masks, seeds)):
        # the random start depends on the lattice index, so give the separate
        # handle as many lattices and use the same index
        s = fd.Solver([fd.Lattice(l.n, l.length, fd.F32)] * (i + 1), fd.default_options(**kw))
        for j in range(i + 1):
            s.set_potential(v.astype(np.float32), lat=j)
            s.init_symmetric(sd, m, lat=j)
        s.evolve(max_steps)
        out.append((s.get_psi(lat=i, dtype=np.float32), s.last_check(lat=i)))
        s.close()
    return out


def small_batch():
    lats = [wl.Lattice(16, 7.0), wl.Lattice(24, 9.0), wl.Lattice(32, 10.0), wl.Lattice(48, 20.0),
            wl.Lattice(64, 24.0)]
    pots = [wl.harmonic(16, 7.0), wl.harmonic(24, 9.0, 1.3), wl.anisotropic(32, 10.0),
            wl.coulomb_soft(48, 20.0), wl.coulomb_soft(64, 24.0, 1.5)]
    masks = [0, wl.ODD_X, 0, wl.SYMMETRIC_ALL, wl.ODD_Z]
    seeds = [1, 2, 3, 4, 5]
    return lats, pots, masks, seeds


@pytest.mark.parametrize("depth,tile", [(1, (64, 16)), (2, (64, 16)), (3, (64, 16)), (1, (128, 16)), (2, (128, 16)),
                                        (3, (128, 16)), (1, (64, 32)), (2, (64, 32)), (3, (64, 32))])
def test_batched_bit_identical_to_separate_runs(fd, depth, tile):
    lats, pots, masks, seeds = small_batch()
    a = run_batch(fd, lats, pots, masks, seeds, True, 3000, temporal_depth=depth, tile_x=tile[0], tile_y=tile[1])
    b = run_batch(fd, lats, pots, masks, seeds, False, 3000, temporal_depth=depth)
    for (pa, oa), (pb, ob) in zip(a, b):
        assert oa["steps"] == ob["steps"] and oa["converged"] == ob["converged"]
        assert oa["energy"] == ob["energy"]
        np.testing.assert_array_equal(pa, pb)


def test_batched_autotuned_launch_matches_a_fixed_configuration(fd):
    """With autotuning the first batched evolve times its (depth, tile
    width) candidates on update passes into the spare fields, which leave
    the state where it was, and then runs the whole evolve in one launch:
    the result equals one launch at a fixed configuration bit for bit, and
    the second evolve of the same sizes launches once with the cached
    choice."""
    lats, pots, masks, seeds = small_batch()
    fixed = run_batch(fd, lats, pots, masks, seeds, True, 3000, temporal_depth=2, tile_x=64, check_every=50)
    kw = dict(check_every=50, tol=1e-6, tol_relative=1, batched=1)
    s = fd.Solver([fd.Lattice(l.n, l.length, fd.F32) for l in lats], fd.default_options(**kw))
    for rep in range(2):
        for i, (v, m, sd) in enumerate(zip(pots, masks, seeds)):
            s.set_potential(v.astype(np.float32), lat=i)
            s.init_symmetric(sd, m, lat=i)
        s.reset_stats()
        s.evolve(3000)
        launches = s.stats()["graph_launches"]
        # nine candidates, each launched untimed and timed, then the run; later: the run only
        assert launches == (1 if rep else 19), (rep, launches)
        for i, (pf, of) in enumerate(fixed):
            o = s.last_check(lat=i)
            assert o["steps"] == of["steps"] and o["energy"] == of["energy"], (rep, i)
            np.testing.assert_array_equal(s.get_psi(lat=i, dtype=np.float32), pf)
            h = s.history(lat=i)  # the check records of the persistent launch
            assert len(h) == o["checks"] and h[-1, 0] == o["steps"] and h[-1, 1] == o["energy"]
            assert np.all(np.diff(h[:, 0]) > 0)
    depth, zc = s.tuned_config()
    tx, ty = s.tuned_kernel()
    assert depth in (1, 2, 3) and zc == -1 and (tx, ty) in ((64, 16), (128, 16), (64, 32))
    s.close()


def test_batched_lattices_converging_at_different_steps(fd):
    """Lattices that converge early drop out of the cost line of the update
    passes, which is cut anew after every check: eight lattices of the C4
    mix's sizes with tolerances that retire them hundreds of steps apart end
    bit-identical to separate runs, with every tile shape."""
    lats = [wl.Lattice(n, 0.25 * n) for n in (48, 64, 96, 48, 128, 64, 160, 96)]
    pots = [wl.harmonic(l.n, l.length, w) for l, w in zip(lats, (1.0, 1.7, 0.6, 2.0, 0.8, 1.2, 1.0, 1.5))]
    masks = [0, wl.ODD_X, wl.SYMMETRIC_ALL, wl.ODD_Z, 0, wl.ODD_Y, 0, wl.ODD_X]
    seeds = list(range(8))
    b = run_batch(fd, lats, pots, masks, seeds, False, 1500, temporal_depth=3)
    steps = {o["steps"] for _, o in b}
    assert len(steps) > 1  # the lattices retire at different checks
    for tile in ((64, 16), (128, 16), (64, 32)):
        a = run_batch(fd, lats, pots, masks, seeds, True, 1500, temporal_depth=3, tile_x=tile[0], tile_y=tile[1])
        for (pa, oa), (pb, ob) in zip(a, b):
            assert oa["steps"] == ob["steps"] and oa["energy"] == ob["energy"], tile
            np.testing.assert_array_equal(pa, pb)


def test_batched_fixed_steps_match_oracle(fd, orc):
    lats = [wl.Lattice(8, 4.0), wl.Lattice(12, 5.0), wl.Lattice(20, 6.0)]
    pots = [wl.harmonic(8, 4.0), wl.anisotropic(12, 5.0), wl.harmonic(20, 6.0)]
    masks = [0, 0, wl.ODD_Y]
    s = fd.Solver([fd.Lattice(l.n, l.length, fd.F32) for l in lats],
                  fd.default_options(check_every=30, tol=0.0, batched=1))
    for i, (v, m) in enumerate(zip(pots, masks)):
        s.set_potential(v, lat=i)
        s.init_symmetric(7, m, lat=i)
    steps, _ = s.evolve(100)
    assert steps == 100
    for i, (l, v, m) in enumerate(zip(lats, pots, masks)):
        a = l.length / l.n
        ref, rec, _ = orc.evolve(orc.init_symmetric(l.n, 7, m, lat=i), v.astype(np.float32).astype(np.float64),
                                 a, a * a / 4, 100, 30, 0.0, False, m)
        got = s.get_psi(lat=i)
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 2e-5
        assert s.last_check(lat=i)["energy"] == pytest.approx(rec["E"], rel=1e-6)


def test_batched_rejects_unsupported_lattices(fd):
    s = fd.Solver([fd.Lattice(10, 4.0, fd.F32)], fd.default_options(batched=1))
    s.set_potential(np.zeros((10, 10, 10)))
    s.init_symmetric(1)
    with pytest.raises(fd.FdtdError) as e:
        s.evolve(10)
    assert e.value.code == fd.ERR_INVALID_ARG
