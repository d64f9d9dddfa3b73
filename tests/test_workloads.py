"""Host checks of the seeded input generators (shared by the oracle tests
and the GPU path; they hold none of the method's arithmetic; no GPU).

The dodecahedral well of Sec. VII.E (Eq. dodecahedronpotential) is pinned to
closed forms that do not go through the generator's convex hull: the
regular dodecahedron whose vertices are the paper's list has circumradius
sqrt(3)/phi, edge 2/phi^2 and 12 pentagonal faces whose outward normals
point along the icosahedron's vertices (0, +-phi, +-1), (+-1, 0, +-phi),
(+-phi, +-1, 0); its inside is therefore the intersection of the 12
half-spaces |n_k . p| <= r_in with r_in = (e/2) sqrt((25 + 11 sqrt 5)/10).
"""
import math

import numpy as np
import pytest

import workloads as wl

PHI = (1 + math.sqrt(5)) / 2
EDGE = 2 / PHI**2
R_IN = EDGE / 2 * math.sqrt((25 + 11 * math.sqrt(5)) / 10)


def face_normals():
    out = []
    for s1 in (-1, 1):
        for s2 in (-1, 1):
            out += [(0, s1 * PHI, s2), (s2, 0, s1 * PHI), (s1 * PHI, s2, 0)]
    n = np.array(out, dtype=np.float64)
    return n / np.linalg.norm(n, axis=1, keepdims=True)


def test_dodecahedron_vertices_are_a_regular_solid():
    v = wl.dodecahedron_vertices()
    assert v.shape == (20, 3)
    assert len({tuple(np.round(p, 12)) for p in v}) == 20
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), math.sqrt(3) / PHI, rtol=1e-14)
    d = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=2)
    np.fill_diagonal(d, np.inf)
    # every vertex has exactly three neighbours at the edge length, none closer
    assert np.all(np.sum(np.isclose(d, EDGE, rtol=1e-12), axis=1) == 3)
    assert np.min(d) == pytest.approx(EDGE, rel=1e-12)
    # each of the 12 face planes holds five vertices at the inradius
    nrm = face_normals()
    proj = v @ nrm.T
    assert np.all(np.sum(np.isclose(proj, R_IN, rtol=1e-12), axis=0) == 5)
    assert np.max(proj) == pytest.approx(R_IN, rel=1e-12)


def test_printed_vertex_list_is_not_regular():
    """The third group as printed, (+-1/phi^2, 0, +-1), does not close a
    regular solid: some vertices sit closer together than an edge."""
    v = wl.dodecahedron_vertices(printed=True)
    d = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=2)
    np.fill_diagonal(d, np.inf)
    assert np.min(d) < 0.8 * EDGE


@pytest.mark.parametrize("n", [21, 40])
def test_dodecahedron_potential_is_the_half_space_intersection(n):
    """Site index 1 -> -1 and index N -> +1 on every axis; V = -100 exactly
    where all 12 half-spaces hold (sites within 1e-9 of a face plane are
    not compared), 0 elsewhere."""
    v = wl.dodecahedron(n)
    assert set(np.unique(v)) <= {0.0, -100.0}
    u = -1.0 + 2.0 * np.arange(n) / (n - 1)
    p = np.stack(np.meshgrid(u, u, u, indexing="ij")[::-1], axis=-1)  # [z][y][x] -> (x, y, z)
    m = p @ face_normals().T
    inside = np.all(m <= R_IN + 1e-9, axis=-1)
    clear = np.all(np.abs(m - R_IN) > 1e-9, axis=-1)
    np.testing.assert_array_equal((v == -100.0)[clear], inside[clear])
    # inside sites times the cell volume approach the solid's volume
    vol = (15 + 7 * math.sqrt(5)) / 4 * EDGE**3
    assert np.sum(v == -100.0) * (2.0 / (n - 1)) ** 3 == pytest.approx(vol, rel=0.02)


def test_dodecahedron_mapping_of_known_points():
    """n = 41: the centre site (index 21) is inside; the corners of the box
    are outside; the edge of the solid at x = +-1 (the segment between the
    vertices (+-1, 0, +-1/phi^2)) is reached by sites 1 and N on the x axis;
    the faces' tangent point along (0, phi, 1) lies inside, just beyond it
    outside."""
    n = 41
    v = wl.dodecahedron(n)
    c = n // 2
    assert v[c, c, c] == -100.0
    for z in (0, n - 1):
        for y in (0, n - 1):
            for x in (0, n - 1):
                assert v[z, y, x] == 0.0
    assert v[c, c, 0] == -100.0 and v[c, c, n - 1] == -100.0
    # y, z axes: along y the solid reaches +-1 too ((1/phi^2, +-1, 0) edge)
    assert v[c, 0, c] == -100.0 and v[0, c, c] == -100.0
    # sites just off the x-axis edge towards a corner are outside
    assert v[c + 3, c + 3, n - 1] == 0.0


def test_theta_basis_and_batch_recipes():
    """V_theta's basis: 16 unit-height Gaussians with seeded centres in
    [-L/4, L/4]^3 and widths in [0.5, 1.5]; the batch recipe: 64 lattices of
    the five sizes, both potential kinds, four sectors."""
    n, L = 16, 10.0
    g, th = wl.config_theta(n, L)
    assert g.shape == (16, n, n, n) and th.shape == (16,)
    assert np.all(np.abs(th) <= 1) and np.all(g > 0) and np.all(g <= 1)
    lats = wl.config_batch()
    assert len(lats) == 64
    assert {l.n for l in lats} <= {48, 64, 96, 128, 160}
    assert {l.kind for l in lats} == {"harmonic", "coulomb_soft"}
    assert {l.mask for l in lats} == {wl.SYMMETRIC_ALL, wl.ODD_X, wl.ODD_Y, wl.ODD_Z}


def test_device_generators_match_numpy():
    """The torch versions used for the large lattices (512^3, 1024^3) build
    the same fields as the numpy ones (evaluated here on the CPU)."""
    torch = pytest.importorskip("torch")
    n, L = 18, 25.6
    np.testing.assert_allclose(wl.coulomb_paper_device(n, L, "cpu").numpy(), wl.coulomb_paper(n, L),
                               rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(wl.anisotropic_device(n, 16.0, "cpu").numpy(), wl.anisotropic(n, 16.0),
                               rtol=1e-13, atol=1e-13)
    assert wl.coulomb_paper_device(n, L, "cpu", torch.float32).dtype == torch.float32


def test_coulomb_paper_is_flat_inside_one_spacing_and_continuous():
    """Eq. coulombpot: 0 for r < a, -1/r + 1/a for r >= a (continuous at a)."""
    n, L = 20, 10.0
    a = L / n
    v = wl.coulomb_paper(n, L)
    r = np.sqrt(wl.radius2(n, L))
    assert np.all(v[r < a] == 0.0)
    far = r >= a
    np.testing.assert_allclose(v[far], -1.0 / r[far] + 1.0 / a, rtol=1e-15)
    # shifted so that V -> V_inf = 1/a far away: 0 <= V < 1/a
    assert np.all(v >= 0.0) and np.all(v < 1.0 / a)
