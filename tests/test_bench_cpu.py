"""CPU checks of bench.py's workload recipes (the mixed batch has the stated size mix, seeds
and per-pair settings, drawn deterministically) and of its matvec ceiling models."""
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


def test_matvec_flop_model_counts_the_transforms_of_each_rk2_stage():
    """The closed form against an explicit tally of the complex transforms one Hessian matvec
    performs in its 4 nt RK2 stages (5 n log2 n flop per transform of length n)."""
    bench = _bench()
    for n1, n2, nt in [(512, 512, 32), (1024, 1024, 32), (128, 256, 8), (256, 64, 4)]:
        fft = lambda n: 5 * n * math.log2(n)
        per_stage = (2 * (n2 // 2) * fft(n1)            # column transform pair over the spectrum columns
                     + n1 * fft(n2)                     # inverse row transforms (both derivatives / the flux)
                     + (n1 // 2) * fft(n2))             # forward row transforms, two real rows packed
        want = 2 * 2 * nt * per_stage                   # incremental state + adjoint, 2 stages per step
        m = bench.matvec_models(n1, n2, nt, 2.0, 6000.0, 80.0)
        assert abs(m["flops"]["flop"] - want) <= 1e-9 * want
        # rate x time gives back the count
        assert abs(m["flops"]["TFLOP/s"] * 1e12 * 2e-3 - want) <= 1e-9 * want


def test_matvec_byte_models():
    bench = _bench()
    m = bench.matvec_models(512, 512, 32, 1.0, 6780.4, 80.0)
    N = 512 * 512
    # streaming: history 2 (nt + 1) fields read, 2 nt states round-tripped (2 fields each), ~10 fields
    # of v, v~ and H v~ (4 bytes per node and field)
    assert abs(m["streaming"]["bytes"] - (2 * 33 + 2 * 32 * 2 + 10) * 4 * N) <= 8 * 4 * N  # within 8 fields
    assert m["streaming"]["bytes"] == (24 * 32 + 40) * N
    assert m["fft_pass"]["bytes"] == 280 * 32 * N
    for k in ("streaming", "fft_pass"):
        gbs = m[k]["bytes"] / 1e-3 / 1e9
        assert abs(m[k]["GB/s"] - gbs) <= 1e-9 * gbs
        assert abs(m[k]["frac_hbm"] - gbs / 6780.4) <= 1e-12
    assert bench.matvec_models(64, 64, 4, 1.0, 1.0, 0.0)["flops"]["frac_fp32"] is None
