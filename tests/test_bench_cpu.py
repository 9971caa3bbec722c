"""CPU checks of bench.py's workload recipes: the mixed batch has the stated size mix, seeds
and per-pair settings, drawn deterministically."""
import math
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


def test_mixed_batch_recipe():
    bench = _bench()
    specs = bench.c4_specs()
    assert len(specs) == 256
    counts = {n: sum(1 for s in specs if s["n"] == n) for n in (128, 256, 512)}
    assert counts == {128: 147, 256: 73, 512: 36}  # 4 : 2 : 1
    assert [s["seed"] for s in specs] == list(range(4000, 4256))
    assert {s["regnorm"] for s in specs} == {1, 2}
    assert {s["beta"] for s in specs} == {1e-2, 1e-3}
    assert {s["gamma"] for s in specs} == {0.0, 1e-3, math.inf}
    assert specs == bench.c4_specs()


def test_mixed_batch_velocities_keep_cfl_quarter_at_nt16():
    bench = _bench()
    for n, vmax in bench.C4_VMAX.items():
        cfl = vmax * n / (2 * math.pi * bench.C4_NT)
        assert abs(cfl - 0.25) < 0.01
