"""Periodic boundaries on the GPU (options.boundary = 1; the paper's remark
that other boundary conditions are easily implemented, Sec. III) against
the oracle in periodic mode: steps, checks, transfer, backward, and the
crystal ground state."""
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


@pytest.fixture()
def per(orc):
    orc.set_boundary(True)
    yield orc
    orc.set_boundary(False)


def rel_max(got, ref):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(ref)), 1e-300))


def solver(fd, n, L, prec, **opt):
    kw = dict(check_every=100, tol=0.0, boundary=1)
    kw.update(opt)
    return fd.Solver(fd.Lattice(n, L, prec), fd.default_options(**kw))


def crystal(n, L, v0=1.5):
    """A smooth periodic potential: cosines of the box period along x and y
    and a weaker one along z."""
    z, y, x = wl.grid(n, L)
    k = 2 * math.pi / L
    return np.ascontiguousarray(np.broadcast_to(v0 * (np.cos(k * x) + 0.6 * np.cos(k * y)) + 0.3 * np.sin(k * z),
                                                (n, n, n)))


@pytest.mark.parametrize("n", [2, 5, 8, 33, 40])
def test_periodic_fp64_steps_match_oracle(fd, per, n):
    """100 FP64 steps with checks every 30 (sizes with ragged 32 x 8 tiles
    and z-chunks, where the wrapped neighbours come from other blocks)."""
    L = 0.5 * n if n > 3 else 3.0
    a = L / n
    v = crystal(n, L) + np.random.default_rng(n).uniform(-0.2, 0.2, (n, n, n))
    s = solver(fd, n, L, fd.F64, check_every=30)
    s.set_potential(v)
    s.init_symmetric(11, 0)
    s.evolve(100)
    ref, rec, _ = per.evolve(per.init_random(n, 11), v, a, a * a / 4, 100, 30)
    assert rel_max(s.get_psi(), ref) <= 1e-12
    assert s.last_check()["energy"] == pytest.approx(rec["E"], rel=1e-12, abs=1e-13)


@pytest.mark.parametrize("prec", ["F32", "BF16"])
def test_periodic_fp32_steps_close_to_oracle(fd, per, prec):
    n, L = 24, 8.0
    a = L / n
    v = crystal(n, L)
    s = solver(fd, n, L, getattr(fd, prec), check_every=25)
    s.set_potential(v.astype(np.float32))
    s.init_symmetric(4, 0)
    s.evolve(100)
    ref, rec, _ = per.evolve(per.init_random(n, 4), v.astype(np.float32).astype(np.float64), a, a * a / 4, 100, 25)
    tol = 1e-5 if prec == "F32" else 2e-2
    assert rel_max(s.get_psi(), ref) <= tol
    assert s.last_check()["energy"] == pytest.approx(rec["E"], rel=tol)


@pytest.mark.parametrize("prec,tol", [("F64", 1e-10), ("F32", 1e-6)])
def test_periodic_crystal_ground_state_matches_oracle(fd, per, prec, tol):
    n, L = 16, 6.0
    a = L / n
    v = crystal(n, L)
    s = solver(fd, n, L, getattr(fd, prec), tol=1e-12 if prec == "F64" else 1e-8, tol_relative=1)
    s.set_potential(v)
    s.init_symmetric(2, 0)
    steps, conv = s.evolve(400_000)
    assert conv
    _, rec, _ = per.evolve(per.init_random(n, 2), v, a, a * a / 4, 400_000, 100, 1e-13, True)
    assert s.last_check()["energy"] == pytest.approx(rec["E"], rel=tol)


def test_periodic_zero_and_periodic_differ(fd):
    """The same start on the same crystal evolves differently with the zero
    shell: the wrap really reaches the kernels."""
    n, L = 16, 6.0
    out = []
    for b in (0, 1):
        s = solver(fd, n, L, fd.F64, boundary=b)
        s.set_potential(crystal(n, L))
        s.init_symmetric(7, 0)
        s.evolve(50)
        out.append(s.get_psi())
    assert rel_max(out[0], out[1]) > 1e-3


def test_periodic_upsample_matches_oracle(fd, per):
    nc, L = 10, 5.0
    coarse = solver(fd, nc, L, fd.F64)
    coarse.set_potential(crystal(nc, L))
    coarse.init_symmetric(4, 0)
    fine = solver(fd, 2 * nc, L, fd.F64)
    fine.set_potential(crystal(2 * nc, L))
    fine.upsample_from(coarse)
    up = per.upsample(per.init_random(nc, 4))
    up = up / math.sqrt(np.sum(up**2) * (L / (2 * nc)) ** 3)
    assert rel_max(fine.get_psi(), up) <= 1e-14


@pytest.mark.parametrize("n", [4, 12, 24])
def test_periodic_direct_kernel_bit_identical(fd, n):
    """The four-site one-step kernel with wrapped neighbours (stencil_kernel
    = 2) reproduces the periodic z-marching kernel bit for bit (n = 4: one
    float4 per row, both x-neighbours wrap), and so does the autotuner's
    choice between the two (stencil_kernel = 0)."""
    L = n / 3.0
    v = crystal(n, L).astype(np.float32)
    out = []
    for k in (1, 2, 0):
        s = solver(fd, n, L, fd.F32, check_every=25, stencil_kernel=k)
        s.set_potential(v)
        s.init_symmetric(9, 0)
        s.evolve(60)
        out.append(s.get_psi(dtype=np.float32))
        s.close()
    np.testing.assert_array_equal(out[0], out[1])
    np.testing.assert_array_equal(out[0], out[2])


@pytest.mark.parametrize("n", [10, 12])
@pytest.mark.parametrize("prec,tol", [("F64", 1e-10), ("F32", 1e-4)])
def test_periodic_backward_matches_oracle(fd, per, prec, tol, n):
    """n = 10: the fused z-marching FP32 adjoint step; n = 12: the split
    four-site one."""
    L, T, ce = n / 2.0, 40, 15
    a = L / n
    v = crystal(n, L)
    psi0 = per.init_random(n, 6)
    ref, obs = per.backward(psi0, v, a, a * a / 4, T, ce, 0, 1.0, 0.3)
    s = solver(fd, n, L, getattr(fd, prec), check_every=ce, backward_steps=T)
    s.set_potential(v)
    s.set_psi(psi0)
    g, o = s.backward(T, 1.0, 0.3)
    assert rel_max(g, ref) <= tol
    # psi_T is 40 steps from a random start: E is a difference of a kinetic
    # term several times |E| and the potential term, so FP32 storage
    # rounding (6e-8 per value) shows at a few parts in 10^6
    assert o["energy"] == pytest.approx(obs["E"], rel=1e-12 if prec == "F64" else 5e-6)


def test_periodic_option_checks(fd):
    with pytest.raises(fd.FdtdError):
        fd.Solver(fd.Lattice(8, 4.0, fd.F32), fd.default_options(boundary=2))
    with pytest.raises(fd.FdtdError):
        fd.Solver([fd.Lattice(8, 4.0, fd.F32)], fd.default_options(boundary=1, batched=1))
    a = solver(fd, 8, 4.0, fd.F64)
    a.init_symmetric(1)
    b = fd.Solver(fd.Lattice(16, 4.0, fd.F64), fd.default_options())
    b.set_potential(np.zeros((16, 16, 16)))
    with pytest.raises(fd.FdtdError) as e:
        b.upsample_from(a)
    assert e.value.code == fd.ERR_INVALID_ARG
