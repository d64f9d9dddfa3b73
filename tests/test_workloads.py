"""Host checks of the seeded input generators (shared by the oracle tests
and the GPU path; they hold none of the method's arithmetic)."""
import numpy as np
import pytest

import workloads as wl


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
