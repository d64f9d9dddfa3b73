"""Checkpoint files (fdtd_save_psi / fdtd_load_psi; Sec. VII.G: a saved
wavefunction starts a later run, at the same or a finer resolution).
Malformed files are made on the host and must be rejected before the
lattice is touched."""
import math
import os

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


def solver(fd, n, L, prec, **opt):
    kw = dict(check_every=50, tol=0.0)
    kw.update(opt)
    s = fd.Solver(fd.Lattice(n, L, prec), fd.default_options(**kw))
    s.set_potential(wl.harmonic(n, L))
    return s


@pytest.mark.parametrize("prec", ["F64", "F32", "BF16"])
def test_round_trip_resumes_bit_for_bit(fd, tmp_path, prec):
    """Save after 100 steps, load into a fresh handle, evolve both 150 more
    steps: identical fields and energies (the mask travels with the file)."""
    n, L = 24, 8.0
    p = getattr(fd, prec)
    a = solver(fd, n, L, p)
    a.init_symmetric(3, wl.ODD_Y)
    a.evolve(100)
    path = tmp_path / "psi.fdtd"
    a.save(path)
    b = solver(fd, n, L, p)
    b.load(path)
    np.testing.assert_array_equal(b.get_psi(), a.get_psi())
    a.evolve(150)
    b.evolve(150)
    np.testing.assert_array_equal(b.get_psi(), a.get_psi())
    assert b.last_check()["energy"] == a.last_check()["energy"]
    size = 64 + n**3 * (8 if prec == "F64" else 4)
    assert os.path.getsize(path) == size


@pytest.mark.parametrize("levels", [1, 2])
def test_load_at_a_finer_resolution_is_the_transfer(fd, tmp_path, levels):
    """A 12^3 file loaded into 24^3 equals fdtd_upsample of the same field
    bit for bit; into 48^3 it equals two transfers up to the intermediate
    renormalisation."""
    nc, L = 12, 6.0
    c = solver(fd, nc, L, fd.F64)
    c.init_symmetric(5, wl.SYMMETRIC_ALL)
    c.evolve(60)
    path = tmp_path / "coarse.fdtd"
    c.save(path)
    nf = nc << levels
    f = solver(fd, nf, L, fd.F64)
    f.load(path)
    ref, prev = None, c
    for k in range(levels):
        m = solver(fd, nc << (k + 1), L, fd.F64)
        m.upsample_from(prev)
        prev = m
    ref = prev.get_psi()
    got = f.get_psi()
    if levels == 1:
        np.testing.assert_array_equal(got, ref)
    else:
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.abs(ref).max())
    assert np.sum(got**2) * (L / nf) ** 3 == pytest.approx(1.0, rel=1e-13)
    f.evolve(50)  # and it evolves with the coarse run's symmetry
    assert f.last_check()["energy"] == pytest.approx(1.5, abs=0.2)


def test_malformed_files_are_rejected(fd, tmp_path):
    n, L = 16, 6.0
    a = solver(fd, n, L, fd.F32)
    a.init_symmetric(2, 0)
    good = tmp_path / "good.fdtd"
    a.save(good)
    raw = good.read_bytes()
    b = solver(fd, n, L, fd.F32)
    b.init_symmetric(9, 0)
    before = b.get_psi()
    cases = {
        "truncated": raw[:-4],
        "short header": raw[:40],
        "trailing": raw + b"\0",
        "bad magic": b"XDTDPSI1" + raw[8:],
        "flipped data byte": raw[:100] + bytes([raw[100] ^ 1]) + raw[101:],
    }
    for name, blob in cases.items():
        p = tmp_path / f"{name}.fdtd"
        p.write_bytes(blob)
        with pytest.raises(fd.FdtdError) as e:
            b.load(p)
        assert e.value.code == fd.ERR_IO, name
        np.testing.assert_array_equal(b.get_psi(), before)  # untouched
    with pytest.raises(fd.FdtdError) as e:
        b.load(tmp_path / "missing.fdtd")
    assert e.value.code == fd.ERR_IO
    # a box of another length, or a size that is no power-of-two multiple
    with pytest.raises(fd.FdtdError) as e:
        solver(fd, n, L + 1.0, fd.F32).load(good)
    assert e.value.code == fd.ERR_SHAPE
    with pytest.raises(fd.FdtdError) as e:
        solver(fd, 24, L, fd.F32).load(good)
    assert e.value.code == fd.ERR_SHAPE
