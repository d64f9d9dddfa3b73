"""bench.py's ncu traffic tables name the sources they were captured from:
the committed figures must belong to the committed kernels, so a change to
the stencil or the batched driver without a new capture fails here (the
bench line itself would report its traffic as null)."""
import bench


def test_stencil_traffic_is_for_the_current_sources():
    digest = bench.stencil_digest()
    keys = [k for k in bench.TRAFFIC if k[0] == digest]
    assert keys, f"no traffic capture for stencil sources {digest}"
    # the benchmark's 512^3 depth-3 configuration, both partitions the tuner may pick
    for span in (-1, -2):
        assert (digest, 512, 3, span, 128, 16) in bench.TRAFFIC


def test_batched_traffic_is_for_the_current_sources():
    digest = bench.stencil_digest(bench.BATCHED_SOURCES)
    assert any(k[0] == digest for k in bench.BATCHED_TRAFFIC), f"no capture for batched sources {digest}"


def test_traffic_figures_are_plausible():
    # within a factor 2 above the algorithmic 12 B per site of a launch
    for (_, n, depth, span, tx, ty), t in bench.TRAFFIC.items():
        algo = 12.0 * n**3
        assert algo <= t <= 2 * algo
