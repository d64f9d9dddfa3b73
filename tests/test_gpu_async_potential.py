"""fdtd_set_potential_async: the potential's copy and checks enqueued
without waiting.  The lattice it loads evolves to the same bits as one
loaded by fdtd_set_potential (host and device input); the checks' result
comes from the next call that uses V; several handles on their own streams
upload while another one computes, with unchanged results."""
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


def solver(fd, n, L, prec, stream=None, **opt):
    kw = dict(check_every=50, tol=0.0)
    kw.update(opt)
    return fd.Solver(fd.Lattice(n, L, prec), fd.default_options(**kw), stream=stream)


def potential(n, L):
    return (wl.harmonic(n, L) + 0.3 * np.cos(wl.radius2(n, L))).astype(np.float32)


@pytest.mark.parametrize("prec", ["F32", "BF16", "F64", "C64", "C32"])
@pytest.mark.parametrize("where", ["pinned", "device", "numpy"])
def test_async_equals_blocking(fd, prec, where):
    import torch

    n, L = 40, 12.0
    v = potential(n, L)
    if prec in ("C64", "C32"):  # a complex potential: an absorbing imaginary part
        v = (v - 0.05j * wl.radius2(n, L)).astype(np.complex64)
    src = {"pinned": lambda: torch.from_numpy(v.copy()).pin_memory(),
           "device": lambda: torch.from_numpy(v).cuda(), "numpy": lambda: v.copy()}[where]
    out = []
    for wait in (True, False):
        s = solver(fd, n, L, getattr(fd, prec))
        s.set_potential(src(), wait=wait)  # the binding keeps the temporary alive
        s.init_symmetric(5, 0)
        s.evolve(200)
        out.append((s.get_psi(), s.last_check()["energy"]))
        s.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


def test_async_checks_reported_by_the_next_call(fd):
    n, L = 16, 6.0
    s = solver(fd, n, L, fd.F32)
    v = potential(n, L)
    bad = v.copy()
    bad[3, 4, 5] = np.nan
    s.set_potential(bad, wait=False)  # returns before the checks ran
    s.init_symmetric(1, 0)
    with pytest.raises(fd.FdtdError) as e:
        s.evolve(10)
    assert e.value.code == fd.ERR_NONFINITE
    with pytest.raises(fd.FdtdError) as e:  # V stays unset
        s.evolve(10)
    assert e.value.code == fd.ERR_STATE
    a = L / n
    unstable = np.full((n, n, n), -2.5 / (a * a / 4), dtype=np.float32)
    s.set_potential(unstable, wait=False)
    with pytest.raises(fd.FdtdError) as e:
        s.observables()
    assert e.value.code == fd.ERR_UNSTABLE_DT
    s.set_potential(v, wait=False)
    steps, _ = s.evolve(10)
    assert steps == 10
    s.close()


def test_uploads_overlap_another_handles_evolve(fd):
    """Three handles on their own streams: the second and third potentials
    are enqueued before the first handle evolves, and every handle's result
    equals the one of a handle loaded and run on its own."""
    import torch

    sizes = (24, 48, 96)
    L = 10.0
    pots = [torch.from_numpy(potential(n, L)).pin_memory() for n in sizes]
    ref = []
    for n, v in zip(sizes, pots):
        s = solver(fd, n, L, fd.F32)
        s.set_potential(v)
        s.init_symmetric(9, 0)
        s.evolve(150)
        ref.append(s.get_psi())
        s.close()
    streams = [torch.cuda.Stream() for _ in sizes]
    ss = [solver(fd, n, L, fd.F32, stream=st) for n, st in zip(sizes, streams)]
    for s, v in zip(ss, pots):
        s.set_potential(v, wait=False)
    for s, r in zip(ss, ref):
        s.init_symmetric(9, 0)
        s.evolve(150)
        assert np.array_equal(s.get_psi(), r)
    for s in ss:
        s.close()
