"""The allocation-free observables entry point against the regular one.

fdtd_observables_noalloc serves callers that cannot allocate device memory
(code inside a fixed memory pool, or handed only raw device pointers and a
stream): it keeps its partial sums in a static device array instead of a
caller workspace.  These tests call it through the C ABI twice in a row on
different fields and compare every value with fdtd_observables on the same
fields, to the FP64 tolerance the parity tests use (1e-12 relative).  This
file is collected last so that a failure here leaves every other test run.
"""
import ctypes

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


def regular(fd, psi, v, length, prec):
    n = psi.shape[0]
    s = fd.Solver(fd.Lattice(n, length, prec), fd.default_options(tol=0.0))
    s.set_potential(v)
    s.set_psi(psi)
    o = s.observables()
    s.close()
    return o


def noalloc(fd, psi, v, length, prec):
    import torch

    tdt = torch.float64 if prec == fd.F64 else torch.float32
    tp = torch.from_numpy(psi).to("cuda", tdt).contiguous()
    tv = torch.from_numpy(v).to("cuda", tdt).contiguous()
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = fd.lib.fdtd_observables_noalloc(ctypes.c_void_p(tp.data_ptr()), ctypes.c_void_p(tv.data_ptr()), prec,
                                         psi.shape[0], length, 1.0, ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(stream.cuda_stream))
    assert rc == fd.OK, fd.last_error(None)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("prec,n", [(1, 48), (0, 33)])
def test_noalloc_matches_regular_observables_twice(fd, prec, n):
    length = 9.0
    rng = np.random.default_rng(n)
    v = wl.anisotropic(n, length)
    fields = [np.exp(-0.5 * wl.radius2(n, length)) * (1 + 0.2 * rng.standard_normal((n, n, n))),
              rng.standard_normal((n, n, n))]
    if prec == fd.F32:
        v = v.astype(np.float32).astype(np.float64)
        fields = [f.astype(np.float32).astype(np.float64) for f in fields]
    for psi in fields:  # two calls in a row share the static scratch
        got = noalloc(fd, psi, v, length, prec)
        ref = regular(fd, psi, v, length, prec)
        assert got[0] == pytest.approx(ref["energy"], rel=1e-12)
        assert got[1] == pytest.approx(ref["r2"], rel=1e-12)
        assert got[2] == pytest.approx(ref["v_expect"], rel=1e-12)
        assert got[3] == pytest.approx(ref["norm"], rel=1e-12)


def test_noalloc_rejects_lattices_beyond_its_scratch(fd):
    import torch

    t = torch.zeros(8, dtype=torch.float32, device="cuda")
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    rc = fd.lib.fdtd_observables_noalloc(ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(t.data_ptr()), fd.F32, 1025,
                                         10.0, 1.0, ctypes.c_void_p(out.data_ptr()), None)
    assert rc == fd.ERR_SHAPE
    assert "1024" in fd.last_error(None)


def test_noalloc_python_wrapper_all_eight_values(fd):
    """fd.observables_noalloc (n inferred from the tensor, dtype mapped, the
    current stream) against Solver.observables: the four derived values and
    the four raw sums S0 = norm / a^3, SH = E S0, Sr = <r^2> S0, SV = <V> S0."""
    import torch

    n, length = 40, 8.0
    a = length / n
    rng = np.random.default_rng(3)
    v = wl.anisotropic(n, length).astype(np.float32).astype(np.float64)
    psi = (np.exp(-0.5 * wl.radius2(n, length)) * (1 + 0.1 * rng.standard_normal((n, n, n)))).astype(np.float32)
    psi = psi.astype(np.float64)
    ref = regular(fd, psi, v, length, fd.F32)
    for _ in range(2):
        out = fd.observables_noalloc(torch.from_numpy(psi).to("cuda", torch.float32),
                                     torch.from_numpy(v).to("cuda", torch.float32), length)
        got = out.cpu().numpy()
        s0 = ref["norm"] / a**3
        want = [ref["energy"], ref["r2"], ref["v_expect"], ref["norm"], s0, ref["energy"] * s0, ref["r2"] * s0,
                ref["v_expect"] * s0]
        np.testing.assert_allclose(got, want, rtol=1e-12)


def test_noalloc_python_wrapper_refuses_what_the_kernels_would_misread(fd):
    """dtypes other than float32/float64, a mismatched pair, a short or
    non-float64 out and non-contiguous fields are refused on the host."""
    import torch

    n = 8
    f32 = torch.zeros((n, n, n), dtype=torch.float32, device="cuda")
    for bad in (f32.to(torch.bfloat16), f32.to(torch.float16), f32.to(torch.int32)):
        with pytest.raises(fd.FdtdError):
            fd.observables_noalloc(bad, bad, 4.0)
    with pytest.raises(fd.FdtdError):
        fd.observables_noalloc(f32, f32.double(), 4.0)
    with pytest.raises(fd.FdtdError):
        fd.observables_noalloc(f32, f32, 4.0, out=torch.zeros(8, dtype=torch.float32, device="cuda"))
    with pytest.raises(fd.FdtdError):
        fd.observables_noalloc(f32, f32, 4.0, out=torch.zeros(7, dtype=torch.float64, device="cuda"))
    with pytest.raises(fd.FdtdError):
        fd.observables_noalloc(f32, f32, 4.0, out=torch.zeros(8, dtype=torch.float64))
    with pytest.raises(fd.FdtdError):
        fd.observables_noalloc(f32.transpose(0, 2), f32, 4.0)
