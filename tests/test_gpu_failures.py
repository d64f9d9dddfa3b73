"""Failure detection without faulting the GPU.

Every device-side wait (the TMA pipeline's mbarrier waits, the batched
kernel's grid barrier) is bounded; when a bound expires the kernel records
it, waits (bounded) for its own copies in flight and returns, and the host
reports FDTD_ERR_TIMEOUT.  These tests make real waits run out by giving
them no budget (options.wait_limit_us < 0), then check the status and that
the CUDA context stays usable.  Input faults are made on the host."""
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


def ho_solver(fd, n, **kw):
    opts = dict(check_every=50, tol=0.0, temporal_depth=2)
    opts.update(kw)
    s = fd.Solver(fd.Lattice(n, 8.0, fd.F32), fd.default_options(**opts))
    s.set_potential(wl.harmonic(n, 8.0))
    s.init_symmetric(3)
    return s


def test_expired_pipeline_wait_reports_timeout(fd):
    s = ho_solver(fd, 64, wait_limit_us=-1)
    with pytest.raises(fd.FdtdError) as e:
        s.evolve(100)
    assert e.value.code == fd.ERR_TIMEOUT
    with pytest.raises(fd.FdtdError) as e:  # stays reported, nothing hangs
        s.evolve(100)
    assert e.value.code == fd.ERR_TIMEOUT


def test_expired_grid_barrier_reports_timeout(fd):
    s = fd.Solver([fd.Lattice(32, 8.0, fd.F32), fd.Lattice(48, 8.0, fd.F32)],
                  fd.default_options(check_every=50, tol=0.0, batched=1, wait_limit_us=-1))
    for i, n in enumerate((32, 48)):
        s.set_potential(wl.harmonic(n, 8.0), lat=i)
        s.init_symmetric(3, lat=i)
    with pytest.raises(fd.FdtdError) as e:
        s.evolve(100)
    assert e.value.code == fd.ERR_TIMEOUT


def test_context_usable_after_timeouts(fd):
    bad = ho_solver(fd, 64, wait_limit_us=-1)
    with pytest.raises(fd.FdtdError):
        bad.evolve(50)
    good = ho_solver(fd, 64)
    ref = ho_solver(fd, 64, stencil_kernel=1)
    good.evolve(100)
    ref.evolve(100)
    np.testing.assert_array_equal(good.get_psi(dtype=np.float32), ref.get_psi(dtype=np.float32))


def test_host_side_input_faults(fd):
    s = fd.Solver(fd.Lattice(16, 8.0, fd.F64), fd.default_options(tol=0.0))
    v = wl.harmonic(16, 8.0)
    v[3, 4, 5] = np.inf
    with pytest.raises(fd.FdtdError) as e:
        s.set_potential(v)
    assert e.value.code == fd.ERR_NONFINITE
    s.set_potential(wl.harmonic(16, 8.0))
    psi = np.ones((16, 16, 16))
    psi[0, 0, 0] = np.nan
    s.set_psi(psi)
    with pytest.raises(fd.FdtdError) as e:
        s.evolve(10)
    assert e.value.code == fd.ERR_NONFINITE
    with pytest.raises(fd.FdtdError) as e:  # a short buffer never reaches the C ABI
        s.set_psi(np.ones(100))
    assert e.value.code == fd.ERR_SHAPE
