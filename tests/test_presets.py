"""The named workloads: sizes as the paper-shaped configurations state them
(rows, unknowns, slices, noise), the geometry the library receives, and the
benchmark's workload table agreeing with them."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_2412_07631_b300 import presets  # noqa: E402


@pytest.mark.parametrize("name,n,m,rows,k", [
    ("plain_32", 1024, 2760, 2760, 1),
    ("plain_128", 16384, 32760, 49144, 64),
    ("mixed_256", 65536, 131040, 196576, 512),
    ("diff_128", 16384, 32760, 49144, 256),
    ("ooc_512", 262144, 525600, 787744, 1024),
])
def test_sizes(name, n, m, rows, k):
    w = presets.PRESETS[name]
    assert (w.n, w.m, w.rows, w.slices) == (n, m, rows, k)
    # the detector covers the image diagonal in every view
    assert w.n_bins >= 2 ** 0.5 * w.n_side


def test_geometry_struct():
    g = presets.geometry("mixed_256")
    assert (g.n_side, g.n_views, g.n_bins) == (256, 360, 364)
    assert g.sqrt_lambda == 0.05 and g.arc_deg == 180.0 and g.pixel_width == 1.0


@pytest.mark.parametrize("bench_name,preset", [("c1", "plain_32"), ("c2", "plain_128"),
                                               ("c3", "mixed_256"), ("c4", "diff_128")])
def test_bench_workloads_match_presets(bench_name, preset):
    ns, nv, nb, sl, k, i0, ne = bench.WORKLOADS[bench_name]
    w = presets.PRESETS[preset]
    assert (ns, nv, nb, sl, k, i0, ne) == (w.n_side, w.n_views, w.n_bins, w.sqrt_lambda, w.slices,
                                            w.i0, w.ellipses)
