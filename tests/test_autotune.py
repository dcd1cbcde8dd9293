"""Autotuner selection and cache logic (CPU, with a stand-in timer), and one
real tuning run on the GPU."""
import json

import pytest


def test_autotune_picks_fastest_and_caches(tmp_path):
    from paper_2412_07631_b300 import autotune, make_geometry
    g = make_geometry(24, 40, 36, 0.05)
    calls = []

    def timer(geom, prec, nb):
        calls.append(nb)
        return {1024: 9.0, 1536: 7.5, 2048: 8.0, 2560: 8.5}[nb]

    path = str(tmp_path / "tune.json")
    assert autotune.outer_block(g, "tf32", path=path, timer=timer) == 1536
    assert sorted(calls) == [1024, 1536, 2048, 2560]
    d = json.load(open(path))
    (entry,) = d.values()
    assert entry["nb_outer"] == 1536 and set(entry["ms"]) == {"1024", "1536", "2048", "2560"}
    # second call: from the cache, no timing
    calls.clear()
    assert autotune.outer_block(g, "tf32", path=path, timer=timer) == 1536
    assert calls == []
    # another precision or geometry is a different key
    assert autotune.outer_block(g, "bf16", path=path, timer=lambda *a: 1.0) == 1024
    assert len(json.load(open(path))) == 2


def test_autotune_tie_goes_to_narrower():
    from paper_2412_07631_b300 import autotune
    assert autotune.pick({1024: 5.0, 512: 5.0, 768: 6.0}) == 512


@pytest.mark.gpu
def test_autotune_real_run(tmp_path):
    from gpu_util import need_cuda
    need_cuda()
    import paper_2412_07631_b300 as ct
    from paper_2412_07631_b300 import autotune
    g = ct.make_geometry(32, 60, 46, 0.05)
    path = str(tmp_path / "tune.json")
    nb = autotune.outer_block(g, "tf32", candidates=(64, 128), path=path)
    assert nb in (64, 128)
    F = ct.System(g, "fp32").factor("tf32", nb_outer=nb)
    assert F.n == 32 * 32


def test_solve_plan_picks_fastest_and_caches(tmp_path):
    """The solve-plan tuner: the fastest (superblock rows, split depth) is
    chosen, set on the factor and cached per geometry, precision and batch."""
    from paper_2412_07631_b300 import autotune, make_geometry

    class _B:
        shape = (512, 100)

    class _F:
        precision = "bf16"
        solve_plan = (0, 0)

        class system:
            geom = make_geometry(24, 40, 36, 0.05)

    times = {(2048, 256): 9.0, (1024, 256): 9.5, (4096, 256): 8.0, (2048, 512): 8.5,
             (2048, 1024): 8.9, (4096, 1024): 7.9}
    calls = []

    def timer(f, b, plan):
        calls.append(tuple(plan))
        return times[tuple(plan)]

    path = str(tmp_path / "tune.json")
    f = _F()
    assert autotune.solve_plan(f, _B(), path=path, timer=timer) == (4096, 1024)
    assert f.solve_plan == (4096, 1024) and sorted(calls) == sorted(times)
    calls.clear()
    g = _F()
    assert autotune.solve_plan(g, _B(), path=path, timer=timer) == (4096, 1024) and calls == []
    assert g.solve_plan == (4096, 1024)
    class _B2:
        shape = (64, 100)
    assert autotune.solve_plan(_F(), _B2(), path=path, timer=lambda *a: 1.0) == (1024, 256)


@pytest.mark.gpu
def test_solve_plan_real_run(tmp_path):
    """The solve-plan tuner on the GPU: it times the candidates on the given
    factor and batch, leaves the factor at the choice, and the factor then
    solves with that plan."""
    from gpu_util import need_cuda
    torch = need_cuda()
    import paper_2412_07631_b300 as ct
    from paper_2412_07631_b300 import autotune
    g = ct.make_geometry(40, 70, 58, 0.05)
    sysg = ct.System(g, "fp32")
    F = sysg.factor("bf16")
    B = torch.ones((8, sysg.m), dtype=torch.float64, device="cuda")
    plan = autotune.solve_plan(F, B, candidates=((512, 256), (1024, 64)), path=str(tmp_path / "t.json"),
                               max_iter=10, tol=1e-8)
    assert plan in ((512, 256), (1024, 64)) and F.solve_plan == plan
    X = F.solve(B, max_iter=10, tol=1e-8)
    assert torch.isfinite(X).all() and F.last_info["stop_measure"] <= 1e-8
