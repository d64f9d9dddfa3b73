"""z-slab decomposition of one lattice over several processes (Sec. V).

The paper splits the N^3 lattice into slabs along z, one per process; every
process updates its own planes, trades boundary planes with its two
neighbours, and at each check the processes reduce their partial sums, so
that every process applies the same renormalisation and sees the same
energy.  Here each process drives its slab on its GPU through the C ABI
(fdtd_slab_*: the temporally blocked stencil on the own planes, the partial
sums, the renormalisation, the check arithmetic), and a communicator moves
the halo planes and reduces the sums:

  * TorchComm -- one process per GPU, torch.distributed point-to-point
    send/recv of the halo planes and an all-reduce of four doubles (NCCL on
    GPUs, gloo on CPU tensors);
  * LocalComm -- several slabs in one process (one GPU), halos copied
    between their buffers.

A pass advances every slab by `halo` steps (the temporal block depth) and
is followed by one exchange of `halo` planes per side, so the update of a
pass never reads a plane another process has not yet sent.  The caller
passes the slab objects; the per-slab work itself runs in the library.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import F32, MEM_HOST, ERR_INVALID_ARG, FdtdError, _check, lib

_vp, _i32, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
lib.fdtd_slab_workspace_size.argtypes = [_i32, _i32, ctypes.POINTER(ctypes.c_size_t)]
lib.fdtd_slab_create.argtypes = [_i32, _i32, _i32, _i32, _d, _d, _d, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp,
                                 ctypes.POINTER(_vp)]
lib.fdtd_slab_destroy.argtypes = [_vp]
lib.fdtd_slab_steps.argtypes = [_vp, _i32, _i32]
lib.fdtd_slab_steps_range.argtypes = [_vp, _i32, _i32, _i32, _i32]
lib.fdtd_slab_sums.argtypes = [_vp, _i32, ctypes.POINTER(_d), _i32]
lib.fdtd_slab_scale.argtypes = [_vp, _i32, _i32, _d, _i32]
lib.fdtd_check_sums.argtypes = [ctypes.POINTER(_d), _d, _i32, _d, ctypes.POINTER(_d)]
for _f in ("fdtd_slab_workspace_size", "fdtd_slab_create", "fdtd_slab_destroy", "fdtd_slab_steps",
           "fdtd_slab_steps_range", "fdtd_slab_sums", "fdtd_slab_scale", "fdtd_check_sums"):
    getattr(lib, _f).restype = ctypes.c_int


def partition(n: int, parts: int):
    """(z_first, nz_own) of each of `parts` slabs: consecutive planes, the
    first n % parts slabs one plane thicker."""
    if not 1 <= parts <= n:
        raise FdtdError(ERR_INVALID_ARG, f"cannot cut {n} planes into {parts} slabs")
    base, extra = divmod(n, parts)
    out, z = [], 0
    for r in range(parts):
        k = base + (1 if r < extra else 0)
        out.append((z, k))
        z += k
    return out


def check_values(sums4, length: float, n: int, v_inf: float = 0.0) -> dict:
    """E, E_b, <r^2>, <V>, norm and the renormalisation factor from the
    lattice-wide sums (fdtd_check_sums)."""
    s = (ctypes.c_double * 4)(*[float(x) for x in sums4])
    out = (ctypes.c_double * 6)()
    _check(lib.fdtd_check_sums(s, float(length), int(n), float(v_inf), out))
    return {"E": out[0], "E_b": out[1], "r2": out[2], "V": out[3], "norm": out[4], "scale": out[5]}


class Slab:
    """One process's slab of an N^3 FP32 lattice on a CUDA device: own planes
    z_first .. z_first + nz_own - 1, `halo` planes on each side, two fields
    and the potential as torch tensors of shape (nz_own + 2 halo, n, n)."""

    def __init__(self, n: int, length: float, z_first: int, nz_own: int, halo: int = 3, mass: float = 1.0,
                 dtau: float = 0.0, device=None, stream=None):
        import torch

        self.n, self.length, self.z_first, self.nz_own, self.halo = n, float(length), z_first, nz_own, halo
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        nzb = nz_own + 2 * halo
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.psi = torch.zeros((2, nzb, n, n), dtype=torch.float32, device=self.device)
            self.v = torch.zeros((nzb, n, n), dtype=torch.float32, device=self.device)
            size = ctypes.c_size_t()
            _check(lib.fdtd_slab_workspace_size(n, nz_own, ctypes.byref(size)))
            self.ws = torch.empty(size.value, dtype=torch.uint8, device=self.device)
            h = ctypes.c_void_p()
            _check(lib.fdtd_slab_create(n, z_first, nz_own, halo, float(length), float(mass), float(dtau),
                                        ctypes.c_void_p(self.psi[0].data_ptr()), ctypes.c_void_p(self.psi[1].data_ptr()),
                                        ctypes.c_void_p(self.v.data_ptr()), ctypes.c_void_p(self.ws.data_ptr()),
                                        size.value, ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.handle = h

    # planes of the buffer that hold global planes [lo, hi) (clipped to the buffer)
    def _rows(self, lo: int, hi: int):
        b0 = self.z_first - self.halo
        return max(lo, b0) - b0, min(hi, b0 + self.nz_own + 2 * self.halo) - b0

    def load(self, field, buf: int = 0, which: str = "psi"):
        """Copy the planes of a whole-lattice field (n, n, n), [z][y][x], that
        fall in this slab's buffer (own and halo planes inside the lattice)."""
        import torch

        lo, hi = self._rows(0, self.n)
        g0 = self.z_first - self.halo
        src = torch.as_tensor(np.asarray(field)[g0 + lo:g0 + hi], dtype=torch.float32)
        dst = self.psi[buf] if which == "psi" else self.v
        if which == "psi":
            dst.zero_()  # halo planes beyond the lattice hold psi = 0
        dst[lo:hi].copy_(src.to(self.device))

    def own(self, buf: int):
        return self.psi[buf][self.halo:self.halo + self.nz_own]

    def steps(self, src: int, depth: int, z_begin: int = 0, z_end: int | None = None):
        """`depth` steps from field src into the other field's own planes
        z_begin .. z_end - 1 (default: all own planes)."""
        z_end = self.nz_own if z_end is None else z_end
        _check(lib.fdtd_slab_steps_range(self.handle, src, depth, z_begin, z_end))

    def sums(self, src: int) -> np.ndarray:
        out = (ctypes.c_double * 4)()
        _check(lib.fdtd_slab_sums(self.handle, src, out, MEM_HOST))
        return np.array(out[:])

    def scale(self, src: int, dst: int, factor: float, mask: int = 0):
        _check(lib.fdtd_slab_scale(self.handle, src, dst, float(factor), int(mask)))

    def close(self):
        if getattr(self, "handle", None):
            lib.fdtd_slab_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LocalComm:
    """Several slabs of one lattice in one process: halos copied between the
    slabs' buffers, sums added.  The copies run in stream order, so there is
    nothing for the inside-out pass order to overlap."""

    overlaps = False

    def __init__(self, slabs):
        self.slabs = list(slabs)

    def exchange(self, buf: int):
        for lower, upper in zip(self.slabs[:-1], self.slabs[1:]):
            h = lower.halo
            # the lower slab's top halo <- the upper slab's first own planes, and back
            lower.psi[buf][h + lower.nz_own:h + lower.nz_own + h].copy_(upper.psi[buf][h:2 * h])
            upper.psi[buf][0:h].copy_(lower.psi[buf][lower.nz_own:lower.nz_own + h])

    def exchange_start(self, buf: int):
        self.exchange(buf)  # copies on the slabs' stream, in order

    def exchange_wait(self):
        pass

    def allreduce(self, parts):
        return np.sum(np.asarray(parts), axis=0)


class TorchComm:
    """One slab per process: halos by torch.distributed send/recv with the
    neighbouring ranks, sums by an all-reduce (the process group's backend:
    NCCL for CUDA tensors, gloo for CPU tensors)."""

    overlaps = True

    def __init__(self, slab, rank: int, world: int, group=None):
        self.slabs = [slab]
        self.rank, self.world, self.group = rank, world, group

    def exchange_start(self, buf: int):
        """Post the sends of this slab's boundary planes of field `buf` and
        the receives into its halo planes; on NCCL they run on the
        communicator's stream after the work already queued on the current
        stream, so kernels queued afterwards overlap them."""
        import torch.distributed as dist

        s = self.slabs[0]
        h, k = s.halo, s.nz_own
        f = s.psi[buf]
        ops = []
        if self.rank > 0:  # below: send my first own planes, receive its last ones into my lower halo
            ops.append(dist.P2POp(dist.isend, f[h:2 * h], self.rank - 1, self.group))
            ops.append(dist.P2POp(dist.irecv, f[0:h], self.rank - 1, self.group))
        if self.rank < self.world - 1:
            ops.append(dist.P2POp(dist.isend, f[k:k + h], self.rank + 1, self.group))
            ops.append(dist.P2POp(dist.irecv, f[h + k:h + k + h], self.rank + 1, self.group))
        self._reqs = dist.batch_isend_irecv(ops) if ops else []

    def exchange_wait(self):
        for req in getattr(self, "_reqs", []):
            req.wait()
        self._reqs = []

    def exchange(self, buf: int):
        self.exchange_start(buf)
        self.exchange_wait()

    def allreduce(self, parts):
        import torch
        import torch.distributed as dist

        t = torch.tensor(np.sum(np.asarray(parts), axis=0), dtype=torch.float64, device=self.slabs[0].psi.device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t.cpu().numpy()


def evolve(comm, n: int, length: float, max_steps: int, check_every: int = 100, tol: float = 0.0,
           tol_relative: bool = True, mask_xy: int = 0, v_inf: float = 0.0, cur: int = 0,
           inside_out: bool | None = None):
    """The evolution of Secs. III-V over the slabs of `comm`, starting from
    field `cur` of every slab: a check at t = 0, check_every, ... and at
    max_steps (lattice-wide sums, renormalisation, the x/y symmetry mask,
    the convergence test on E_b); between checks, passes of `halo` steps
    each followed by a halo exchange.  With inside_out (and slabs of at
    least three halos) a pass is the paper's inside-out order: the `halo`
    planes at each end of every slab first, their exchange started, then
    the interior planes while it is in flight, then the wait; by default
    when the communicator's exchange can overlap the update (TorchComm).
    Returns (cur, record of the last check, number of checks)."""
    if inside_out is None:
        inside_out = getattr(comm, "overlaps", False)
    slabs = comm.slabs
    depth = min(s.halo for s in slabs)
    comm.exchange(cur)
    prev, checks, t = None, 0, 0
    rec = None
    while True:
        if t % check_every == 0 or t == max_steps:
            vals = check_values(comm.allreduce([s.sums(cur) for s in slabs]), length, n, v_inf)
            for s in slabs:
                s.scale(cur, 1 - cur, vals["scale"], mask_xy)
            cur = 1 - cur
            comm.exchange(cur)
            checks += 1
            delta = abs(vals["E_b"] - prev) if prev is not None else -1.0
            rec = dict(vals, t=t, delta_e=delta, converged=False)
            if prev is not None and tol > 0 and delta <= tol * (abs(vals["E_b"]) if tol_relative else 1.0):
                rec["converged"] = True
                break
            prev = vals["E_b"]
        if t == max_steps:
            break
        k = min(depth, max_steps - t, check_every - t % check_every)
        if inside_out and all(s.nz_own >= 3 * s.halo for s in slabs):
            for s in slabs:  # the planes the neighbours need
                s.steps(cur, k, 0, s.halo)
                s.steps(cur, k, s.nz_own - s.halo, s.nz_own)
            comm.exchange_start(1 - cur)
            for s in slabs:  # the interior, while the halos travel
                s.steps(cur, k, s.halo, s.nz_own - s.halo)
            comm.exchange_wait()
        else:
            for s in slabs:
                s.steps(cur, k)
            comm.exchange(1 - cur)
        cur = 1 - cur
        t += k
    rec["steps"] = t
    return cur, rec, checks


def gather(slabs, buf: int) -> np.ndarray:
    """The whole-lattice field (n, n, n) from the own planes of the slabs (in order)."""
    return np.concatenate([s.own(buf).float().cpu().numpy() for s in slabs], axis=0)
