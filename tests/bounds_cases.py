"""Run by tests/test_gpu_bounds.py with FDTD_LIB pointing at the
bounds-checking build: every TMA tile-pipeline configuration on small,
ragged lattices, then the total of out-of-allocation accesses as JSON."""
import json
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import paper_0904_0939_gb300 as fd  # noqa: E402
import workloads as wl  # noqa: E402

assert fd.LIB_PATH.endswith("libfdtd_checked.so"), fd.LIB_PATH
bad, cases = 0, 0


def run(s):
    global bad, cases
    bad += s.bounds_violations()
    cases += 1
    s.close()


for n in (8, 12, 20, 36, 44, 68, 132):
    L = 0.4 * n
    v = wl.harmonic(n, L).astype(np.float32)
    for depth in (1, 2, 3):
        for zc in (0, -1, -2, 1, 3, 9, n + 5):
            s = fd.Solver(fd.Lattice(n, L, fd.F32), fd.default_options(check_every=5, tol=0.0, temporal_depth=depth,
                                                                         zchunk=zc))
            s.set_potential(v)
            s.init_symmetric(1, wl.ODD_Y)
            s.evolve(13)
            s.observables()
            run(s)
    s = fd.Solver(fd.Lattice(n, L, fd.F32), fd.default_options(check_every=10, tol=1e-5, tol_relative=1))
    s.set_potential(v)
    s.init_symmetric(2, 0)
    s.evolve(60)  # autotuned: every candidate runs once
    run(s)
# BF16 storage: the TMA stencil with BF16 psi boxes (n % 8 == 0)
for n in (8, 16, 40, 72, 136):
    L = 0.4 * n
    v = wl.harmonic(n, L).astype(np.float32)
    for depth in (1, 2, 3):
        for tx in (64, 128):
            for zc in (0, -1, -2, 5):
                s = fd.Solver(fd.Lattice(n, L, fd.BF16),
                              fd.default_options(check_every=5, tol=0.0, temporal_depth=depth, tile_x=tx, zchunk=zc))
                s.set_potential(v)
                s.init_symmetric(1, wl.ODD_Y)
                s.evolve(13)
                run(s)
lats = [fd.Lattice(n, 0.4 * n, fd.F32) for n in (8, 12, 20, 36, 68)]
for kw in (dict(), dict(temporal_depth=3, tile_x=64), dict(temporal_depth=2, tile_x=128),
           dict(temporal_depth=3, tile_x=64, tile_y=32), dict(temporal_depth=1, tile_x=64, tile_y=32)):
    s = fd.Solver(lats, fd.default_options(check_every=10, tol=1e-4, tol_relative=1, batched=1, **kw))
    for i, l in enumerate(lats):
        s.set_potential(wl.harmonic(l.n, l.length).astype(np.float32), lat=i)
        s.init_symmetric(3, wl.ODD_X, lat=i)
    s.evolve(200)  # batched: with its timed tuning passes, then every tile shape in a whole run
    run(s)
# z-slabs: the slab stencil over own-plane ranges, the slab sums; a slab's
# count of accesses outside the allocation is the fourth word of its workspace
from paper_0904_0939_gb300 import slab  # noqa: E402

for n, parts, halo in ((36, 2, 3), (44, 3, 2), (20, 2, 1), (12, 4, 3)):
    L = 0.4 * n
    v = wl.anisotropic(n, L)
    start = np.random.default_rng(n).uniform(-1.0, 1.0, (n, n, n))
    for inside_out in (True, False):
        slabs = [slab.Slab(n, L, z0, k, halo) for z0, k in slab.partition(n, parts)]
        for sl in slabs:
            sl.load(v, which="v")
            sl.load(start, 0)
        slab.evolve(slab.LocalComm(slabs), n, L, 23, 10, inside_out=inside_out)
        for sl in slabs:
            bad += int(sl.ws.view(torch.int32)[3].item())
            sl.close()
        cases += 1
print(json.dumps({"violations": bad, "cases": cases}))
