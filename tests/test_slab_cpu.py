"""The z-slab decomposition's host side on CPU ranks (gloo, world size 2
and 3): partition, halo exchange by send/recv, all-reduce of the partial
sums, the check arithmetic of the library and the evolve loop of
paper_0904_0939_gb300.slab, with a plain numpy slab (Eq. updateeq on the own
and halo planes, FP64) standing in for the GPU slab.  The gathered field
after the run must equal the oracle's whole-lattice evolution element by
element (FP64, 1e-12), and the energy of the last check the oracle's.
"""
import socket

import numpy as np
import pytest

import workloads as wl


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class NumpySlab:
    """Test double of slab.Slab on the host: same buffers (2, nz_own + 2 halo,
    n, n), same calls, plain FP64 numpy arithmetic."""

    def __init__(self, n, length, z_first, nz_own, halo, v_full):
        import torch

        self.n, self.length, self.z_first, self.nz_own, self.halo = n, length, z_first, nz_own, halo
        nzb = nz_own + 2 * halo
        self.psi = torch.zeros((2, nzb, n, n), dtype=torch.float64)
        self.a = length / n
        self.dtau = self.a * self.a / 4
        g0 = z_first - halo
        self.inside = np.array([0 <= g0 + k < n for k in range(nzb)])
        self.v = np.zeros((nzb, n, n))
        for k in range(nzb):
            if self.inside[k]:
                self.v[k] = v_full[g0 + k]

    def load(self, field, buf=0):
        import torch

        g0 = self.z_first - self.halo
        self.psi[buf].zero_()
        for k in range(self.psi.shape[1]):
            if self.inside[k]:
                self.psi[buf][k] = torch.from_numpy(np.asarray(field[g0 + k], dtype=np.float64))

    def own(self, buf):
        return self.psi[buf][self.halo:self.halo + self.nz_own]

    def _step(self, f):
        c = self.dtau / (2 * self.a * self.a)
        p = np.pad(f, ((1, 1), (1, 1), (1, 1)))
        s = (p[1:-1, 1:-1, :-2] + p[1:-1, 1:-1, 2:]) + (p[1:-1, :-2, 1:-1] + p[1:-1, 2:, 1:-1]) + \
            (p[:-2, 1:-1, 1:-1] + p[2:, 1:-1, 1:-1])
        h = 0.5 * self.dtau * self.v
        out = (1 - h) / (1 + h) * f + c / (1 + h) * (s - 6 * f)
        out[~self.inside] = 0.0
        return out

    def steps(self, src, depth, z_begin=0, z_end=None):
        import torch

        z_end = self.nz_own if z_end is None else z_end
        f = self.psi[src].numpy().copy()
        for _ in range(depth):
            f = self._step(f)
        h = self.halo
        self.psi[1 - src][h + z_begin:h + z_end] = torch.from_numpy(f[h + z_begin:h + z_end])

    def sums(self, src):
        f = self.psi[src].numpy()
        h, n, a = self.halo, self.n, self.a
        p = np.pad(f, ((0, 0), (1, 1), (1, 1)))
        own = slice(h, h + self.nz_own)
        c = f[own]
        s = (p[own, 1:-1, :-2] + p[own, 1:-1, 2:]) + (p[own, :-2, 1:-1] + p[own, 2:, 1:-1]) + \
            (f[h - 1:h - 1 + self.nz_own] + f[h + 1:h + 1 + self.nz_own])
        lap = s - 6 * c
        ax = (np.arange(n) - 0.5 * (n - 1)) * a
        zs = (np.arange(self.z_first, self.z_first + self.nz_own) - 0.5 * (n - 1)) * a
        r2 = zs[:, None, None] ** 2 + ax[None, :, None] ** 2 + ax[None, None, :] ** 2
        v = self.v[own]
        return np.array([np.sum(c * c), np.sum(c * (-lap / (2 * a * a) + v * c)), np.sum(r2 * c * c),
                         np.sum(v * c * c)])

    def scale(self, src, dst, factor, mask=0):
        import torch

        h = self.halo
        c = self.psi[src][h:h + self.nz_own].numpy().copy()
        for ax, dim in ((0, 2), (1, 1)):
            mode = (mask >> (2 * ax)) & 3
            if mode:
                n = c.shape[dim]
                idx = [slice(None)] * 3
                for i in range(n):
                    m = n - 1 - i
                    if i > m:
                        sl, sm = list(idx), list(idx)
                        sl[dim], sm[dim] = i, m
                        c[tuple(sl)] = (-1.0 if mode == 2 else 1.0) * c[tuple(sm)]
                    elif i == m and mode == 2:
                        sl = list(idx)
                        sl[dim] = i
                        c[tuple(sl)] = 0.0
        self.psi[dst][h:h + self.nz_own] = torch.from_numpy(factor * c)


CASE = dict(n=20, length=8.0, steps=50, check_every=20, halo=3)


def _problem():
    n, L = CASE["n"], CASE["length"]
    return wl.anisotropic(n, L), np.random.default_rng(8).uniform(-1, 1, (n, n, n))


def _worker(rank, world, port, mask, inside_out, out):
    import torch.distributed as dist

    from paper_0904_0939_gb300 import slab

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    v, start = _problem()
    n, L = CASE["n"], CASE["length"]
    z_first, nz_own = slab.partition(n, world)[rank]
    s = NumpySlab(n, L, z_first, nz_own, CASE["halo"], v)
    s.load(start, 0)
    comm = slab.TorchComm(s, rank, world)
    cur, rec, checks = slab.evolve(comm, n, L, CASE["steps"], CASE["check_every"], mask_xy=mask,
                                   inside_out=inside_out)
    dist.barrier()
    dist.destroy_process_group()
    out[rank] = (z_first, s.own(cur).numpy().copy(), rec, checks)


@pytest.mark.parametrize("world,mask,inside_out", [(2, 0, True), (2, 0, False), (3, wl.ODD_X, False)])
def test_slab_evolution_over_gloo_ranks_matches_the_oracle(orc, world, mask, inside_out):
    """world 2: slabs of ten planes, so the inside-out order updates three
    planes at each end, exchanges them and updates the four interior planes
    while they travel; world 3: slabs of seven and six planes, too thin for
    it, so each pass is followed by its exchange"""
    import torch.multiprocessing as mp

    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, mask, inside_out, out), nprocs=world, join=True)
        res = dict(out)
    field = np.concatenate([res[r][1] for r in range(world)], axis=0)
    n, L = CASE["n"], CASE["length"]
    a = L / n
    v, start = _problem()
    ref, rec, _ = orc.evolve(start, v, a, a * a / 4, CASE["steps"], CASE["check_every"], mask=mask)
    assert np.max(np.abs(field - ref)) <= 1e-12 * np.max(np.abs(ref))
    for r in range(world):
        assert res[r][2]["E"] == pytest.approx(rec["E"], rel=1e-12)  # every rank sees the lattice-wide E
        assert res[r][3] == 4  # checks at t = 0, 20, 40, 50


def test_partition_and_check_values():
    from paper_0904_0939_gb300 import slab

    assert slab.partition(10, 3) == [(0, 4), (4, 3), (7, 3)]
    assert sum(k for _, k in slab.partition(512, 7)) == 512
    with pytest.raises(Exception):
        slab.partition(4, 5)
    vals = slab.check_values([2.0, 3.0, 4.0, 5.0], length=4.0, n=8, v_inf=0.5)
    a3 = 0.5**3
    assert vals["E"] == 1.5 and vals["E_b"] == 1.0 and vals["r2"] == 2.0 and vals["V"] == 2.5
    assert vals["norm"] == 2.0 * a3 and vals["scale"] == pytest.approx(1 / np.sqrt(2.0 * a3))
