"""Gradients through torch: EnergyFn (the torch.autograd.Function over
fdtd_backward) on a potential V_theta = r^2/2 + sum_k theta_k G_k built in
torch from parameters theta, against the oracle's full-trajectory adjoint
contracted with the basis G_k by hand.

Tolerances (max-norm relative over the 16 components of dL/dtheta): FP64
1e-10 (the adjoint is the exact transpose of the unrolled map; only the
order of the sums differs), FP32 1e-4 (24-bit rounding of psi and lambda
over T steps, the same bound the dV parity tests use).
"""
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


def theta_setup(n, L):
    g, th = wl.config_theta(n, L)
    return g, th


def torch_grad(fd, prec, n, L, T, ce, g, th, psi0, mask, seed, w_e, w_r, vdtype=None):
    """theta.grad of w_e E + w_r <r^2> through EnergyFn, V_theta built in torch."""
    import torch

    dev = torch.device("cuda")
    vdtype = vdtype or torch.float64
    G = torch.from_numpy(g).to(dev, vdtype)
    theta = torch.tensor(th, dtype=vdtype, device=dev, requires_grad=True)
    r2 = torch.from_numpy(wl.radius2(n, L)).to(dev, vdtype)
    v = 0.5 * r2 + torch.tensordot(theta, G, dims=1)
    s = fd.Solver(fd.Lattice(n, L, prec), fd.default_options(check_every=ce, tol=0.0, backward_steps=T))
    E, R = fd.energy_fn().apply(v, s, T, None if psi0 is None else torch.from_numpy(psi0).to(dev), seed, mask)
    loss = w_e * E + w_r * R
    loss.backward()
    out = theta.grad.detach().double().cpu().numpy(), float(E.detach()), float(R.detach())
    s.close()
    return out


@pytest.mark.parametrize("start", ["gaussian", "random_odd_x"])
def test_energy_fn_theta_gradient_matches_oracle(fd, orc, start):
    """n = 12, L = 6, T = 60 unrolled steps, checks every 10 (so the
    renormalisations and, for the odd start, the symmetry projection are
    inside the differentiated map): theta.grad from torch's chain rule
    through EnergyFn equals sum_s dL/dV(s) G_k(s) of the oracle's adjoint."""
    n, L, T, ce = 12, 6.0, 60, 10
    a = L / n
    g, th = theta_setup(n, L)
    v = wl.v_theta(n, L, th, g)
    if start == "gaussian":
        mask, seed = 0, 0
        psi0 = np.exp(-0.5 * wl.radius2(n, L))
        ref_start = psi0
    else:
        mask, seed = wl.ODD_X, 31
        psi0 = None
        ref_start = orc.init_symmetric(n, seed, mask)
    w_e, w_r = 1.0, 0.3
    gv, obs = orc.backward(ref_start, v, a, a * a / 4, T, ce, mask, w_e, w_r)
    want = np.tensordot(g, gv, axes=3)
    for prec, tol in ((fd.F64, 1e-10), (fd.F32, 1e-4)):
        got, e, r = torch_grad(fd, prec, n, L, T, ce, g, th, psi0, mask, seed, w_e, w_r)
        assert rel_max(got, want) <= tol, (prec, got, want)
        assert e == pytest.approx(obs["E"], rel=1e-12 if prec == fd.F64 else 1e-6)
        assert r == pytest.approx(obs["r2"], rel=1e-12 if prec == fd.F64 else 1e-6)


def test_energy_fn_weights_are_the_incoming_gradients(fd, orc):
    """Only <r^2> in the loss (E unused): the backward receives w_e = 0 and
    w_r = 1; an FP32 potential tensor gets an FP32 gradient."""
    import torch

    n, L, T, ce = 8, 4.0, 30, 7
    a = L / n
    g, th = theta_setup(n, L)
    v = wl.v_theta(n, L, th, g)
    psi0 = np.exp(-0.5 * wl.radius2(n, L))
    gv, _ = orc.backward(psi0, v, a, a * a / 4, T, ce, 0, 0.0, 1.0)
    got, _, _ = torch_grad(fd, fd.F64, n, L, T, ce, g, th, psi0, 0, 0, 0.0, 1.0)
    assert rel_max(got, np.tensordot(g, gv, axes=3)) <= 1e-10
    # an FP32 potential: the gradient comes back in the potential's dtype
    dev = torch.device("cuda")
    v32 = torch.from_numpy(v).to(dev, torch.float32).requires_grad_()
    s = fd.Solver(fd.Lattice(n, L, fd.F32), fd.default_options(check_every=ce, tol=0.0, backward_steps=T))
    E, R = fd.energy_fn().apply(v32, s, T, torch.from_numpy(psi0).to(dev))
    R.backward()
    assert v32.grad.dtype == torch.float32 and v32.grad.shape == v32.shape
    assert rel_max(v32.grad.double().cpu().numpy(), gv) <= 1e-4
    s.close()


def test_energy_fn_rejects_a_forward_that_could_stop_early(fd):
    """The forward must run exactly T steps: a solver with a tolerance, or
    without backward storage for T steps, is refused before any work."""
    import torch

    n, L = 8, 4.0
    v = torch.from_numpy(wl.harmonic(n, L)).cuda()
    EnergyFn = fd.energy_fn()
    with_tol = fd.Solver(fd.Lattice(n, L, fd.F64), fd.default_options(tol=1e-6, backward_steps=50))
    with pytest.raises(fd.FdtdError, match="tol"):
        EnergyFn.apply(v, with_tol, 50)
    short = fd.Solver(fd.Lattice(n, L, fd.F64), fd.default_options(tol=0.0, backward_steps=20))
    with pytest.raises(fd.FdtdError, match="backward_steps"):
        EnergyFn.apply(v, short, 50)
    with_tol.close()
    short.close()
