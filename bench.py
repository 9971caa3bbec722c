"""Benchmark: registrations/s and Gauss-Newton Hessian matvecs/s at 512^2, nt=32.

Workload: synthetic "brain-like" nested smoothed ellipses (5 labels, random
contrasts), reference = template displaced by a divergence-free velocity with
modes |k| <= 16 (max |v| = 0.098, CFL 0.25 at nt = 32); H1 seminorm,
incompressible (div v = 0), beta_v = 1e-3, zero start, relative gradient 1e-2.
One step = one full Newton-Krylov registration (reg_solve: state, adjoint,
gradient, PCG with GN matvecs, Armijo, Newton) plus det F1 (reg_detgrad).

Arms:
  default            the CUDA library through the C ABI (device-resident inputs);
                     also e2e through reg_register_host with host buffers,
                     a matvec throughput loop, per-kernel-class timing for the
                     roofline and the FP64 oracle CPU baseline.
  --impl reference   the FP64 oracle on the host cores (bounded sample).
Multi-GPU (torchrun): independent replicas, one registration per rank
(pairs are independent), value = all ranks' registrations / max time.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "registrations/sec and Hessian matvecs/sec at 512² nt=32; warm-start vs plain"
PAIRS = 5  # independent 512^2 pairs per step (seeds 3000..3004), solved concurrently
N_GRID, NT, BETA, SEED, VMAX = 512, 32, 1e-3, 3000, 0.098
WORKLOAD = ("synthetic brain-like ellipses 512x512, nt=32, H1, beta_v=1e-3, incompressible, "
            "shear s=0, zero start, tol 1e-2; step = 5 independent pairs solved concurrently + det F1 each")
# PDE solves of one zero-start registration of this workload as counted by
# reg_solve on the GPU (stats n_pde: 5 Newton iterations, 38 matvecs, 5
# line-search evaluations); scales the oracle's per-PDE-solve time to a
# registration in the reference arm, which runs without a GPU.
PDE_PER_REG = 93


def rank_seeds(rank, pairs=None):
    """Seeds of the pairs one rank registers per step (disjoint across ranks)."""
    pairs = PAIRS if pairs is None else pairs
    return [SEED + rank * pairs + i for i in range(pairs)]


def aggregate_ms(ms_local, world, dist=None, device=None):
    """Max over ranks of a per-rank step time (replicas only; no data-path collective)."""
    if world == 1 or dist is None:
        return float(ms_local)
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(ms_step, world, pairs=None):
    """Registrations per second of the whole job: all ranks' pairs / max step time."""
    pairs = PAIRS if pairs is None else pairs
    return world * pairs * 1e3 / ms_step


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def matvec_models(n1, n2, nt, ms, hbm_gbs, fp32_tflops):
    """One Gauss-Newton Hessian matvec taking `ms` milliseconds on an n1 x n2 grid with nt
    time steps, against two byte models and an FFT flop model (N = n1 n2 nodes, FP32):
      streaming  (24 nt + 40) N bytes: a time step fully on chip, so that each of the two
                 sweeps reads the state history once and round-trips one state per step;
      fft_pass   280 nt N bytes: every 2-D FFT pass (about 15 real 2-D transforms per step,
                 16 N bytes each) and the pointwise work (about 40 N) through memory;
      flops      the transforms of the 4 nt RK2 stages (incremental state and adjoint, two
                 stages per step), 5 n log2 n flop per complex transform of length n: per
                 stage one column transform pair over n2/2 spectrum columns (5 N log2 n1)
                 and 1.5 row transforms' worth over the n1 rows (7.5 N log2 n2).
    Returns bytes or flops, the achieved rate and its fraction of the given ceiling."""
    N = n1 * n2
    sec = ms * 1e-3
    out = {"ms_per_matvec": ms}
    for name, byt in (("streaming", (24 * nt + 40) * N), ("fft_pass", 280 * nt * N)):
        gbs = byt / sec / 1e9
        out[name] = {"bytes": byt, "GB/s": gbs, "frac_hbm": gbs / hbm_gbs}
    fl = 4 * nt * (5 * math.log2(n1) + 7.5 * math.log2(n2)) * N
    tf = fl / sec / 1e12
    out["flops"] = {"flop": fl, "TFLOP/s": tf, "frac_fp32": (tf / fp32_tflops) if fp32_tflops else None}
    return out


def images(seed=SEED):
    from paper_1503_00757_gb300 import synth
    mT, mR, _ = synth.ellipses_pair(N_GRID, seed, vmax=VMAX)
    return mT.astype(np.float32), mR.astype(np.float32)


# DRAM bytes (read + write) per launch of the RK2 row-stage kernel at 512^2, nt=32: the mean over
# 8 incremental-state launches of one ncu capture (cold L2), profiles/traffic_row_stage_512_nt32.md.
ROW_STAGE_TRAFFIC_512 = 9.99e6

C4_SIZES = (128, 256, 512)
C4_COUNTS = (147, 73, 36)  # 4 : 2 : 1 over 256 pairs
C4_VMAX = {128: 0.196, 256: 0.098, 512: 0.049}  # CFL 0.25 at nt = 16
C4_NT = 16


def c4_specs():
    """The mixed batch: 256 pairs (seeds 4000-4255), grid sizes 128^2 : 256^2 : 512^2 = 4 : 2 : 1,
    per pair a seeded random seminorm (H1 / H2), beta_v in {1e-2, 1e-3} and beta_w in {0, 1e-3, inf}."""
    rng = np.random.default_rng(4000)
    sizes = [n for n, c in zip(C4_SIZES, C4_COUNTS) for _ in range(c)]
    specs = []
    for i, n in enumerate(sizes):
        specs.append(dict(n=n, seed=4000 + i, regnorm=int(rng.choice([1, 2])), beta=[1e-2, 1e-3][int(rng.integers(2))],
                          gamma=[0.0, 1e-3, math.inf][int(rng.integers(3))]))
    return specs


def run_batched_mixed(dev, stream, opts, nworkers=16):
    """The mixed-size batch through the executor (autotuned tiles, concurrent streams) against a
    sequential per-pair loop of the same library (one context per grid size, one pair at a time)."""
    import torch
    from paper_1503_00757_gb300 import synth
    from paper_1503_00757_gb300.binding import Context, Executor, autotune
    specs = c4_specs()
    t0 = time.perf_counter()
    imgs = synth.ellipses_images([(s["n"], s["seed"], C4_VMAX[s["n"]]) for s in specs],
                                 workers=max(1, min(16, os.cpu_count() or 1)))
    gen_s = time.perf_counter() - t0
    tiles = {}
    for n in C4_SIZES:
        R, C, P, D, ms = autotune(n, n, nt=8, concurrency=8, force=True)
        tiles[str(n)] = {"rows_per_cta": R, "cols_per_cta": C, "prefetch": P, "pdl": D}
    pairs = []
    for s, (a, b) in zip(specs, imgs):
        n = s["n"]
        pairs.append(dict(mT=torch.from_numpy(a).to(dev), mR=torch.from_numpy(b).to(dev),
                          v=torch.zeros(2, n, n, device=dev), nt=C4_NT, regnorm=s["regnorm"], beta=s["beta"],
                          gamma=s["gamma"], shear=0.0))
    ex = Executor(nworkers)

    def batched():
        for p in pairs:
            p["v"].zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        _, st = ex.solve(pairs, opts, check=False)
        return st, time.perf_counter() - t

    batched()  # warm-up: contexts, captured graphs
    st_b, sec_b = batched()
    ctxs = {n: Context(n, n, C4_NT, stream=stream) for n in C4_SIZES}

    def sequential(subset):
        for p in subset:
            p["v"].zero_()
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = []
        for p in subset:
            c = ctxs[p["mT"].shape[0]]
            c.set_params(C4_NT, regnorm=p["regnorm"], beta=p["beta"], gamma=p["gamma"])
            c.set_images(p["mT"], p["mR"])
            out.append(c.solve(p["v"], opts, check=False))
        stream.synchronize()
        return out, time.perf_counter() - t

    sequential([p for p in pairs if p["beta"] == 1e-2][:12])  # warm-up
    st_s, sec_s = sequential(pairs)
    for c in ctxs.values():
        c.close()
    ex.close()
    ok_b = sum(1 for s in st_b if s["rc"] == 0)
    ok_s = sum(1 for s in st_s if s["rc"] == 0)
    return {"workload": "mixed batch: 256 pairs, 128^2:256^2:512^2 = 147:73:36, nt=16, seeded random "
                        "H1/H2, beta_v in {1e-2,1e-3}, beta_w in {0,1e-3,inf}, zero start, tol 1e-2",
            "batched": {"pairs_per_s": len(pairs) / sec_b, "seconds": sec_b, "converged": ok_b, "workers": nworkers},
            "sequential": {"pairs_per_s": len(pairs) / sec_s, "seconds": sec_s, "converged": ok_s},
            "speedup": sec_s / sec_b, "tiles": tiles, "image_generation_s": gen_s,
            "matvecs_total": int(sum(s["n_mv"] for s in st_b))}


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    def __init__(self, index, directory):
        self.index = index
        self.proc = None
        self.path = os.path.join(directory, f"clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_pde_time(mT, mR):
    """Time one FP64 oracle state solve (one PDE solve) of this workload."""
    from oracle.transport import state_solve
    from paper_1503_00757_gb300 import synth
    v = 0.5 * synth.velocity(N_GRID, N_GRID, 16, VMAX, np.random.default_rng(SEED + 7))
    t0 = time.perf_counter()
    state_solve(mT.astype(np.float64), v, NT)
    return time.perf_counter() - t0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    mT, mR = images()
    pde_per_reg = PDE_PER_REG
    for _ in range(args.warmup):
        cpu_oracle_pde_time(mT, mR)  # untimed warm-up steps
    times = [cpu_oracle_pde_time(mT, mR) for _ in range(args.steps)]
    t = float(np.mean(times))
    value = 1.0 / (t * pde_per_reg)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "registrations/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": value, "unit": "registrations/s", "cores": 1, "kind": "oracle",
                         "sample": f"one FP64 oracle state solve (512^2, nt=32) per step, scaled by "
                                   f"{pde_per_reg} PDE solves per registration"},
        "e2e": {"value": value, "unit": "registrations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-dir", default=None,
                    help="where the nvidia-smi clock samples of the timed region are written (default: a temp dir)")
    ap.add_argument("--matvecs", type=int, default=200)
    ap.add_argument("--no-warm", dest="warm", action="store_false",
                    help="skip the warm-start comparison")
    ap.add_argument("--no-big", dest="big", action="store_false",
                    help="skip the 1024^2 matvec measurement")
    ap.add_argument("--no-shear", dest="shear", action="store_false",
                    help="skip the shear-control (nonlinear Stokes) solves")
    ap.add_argument("--no-batched", dest="batched", action="store_false",
                    help="skip the mixed-size batch (256 pairs) against the sequential loop")
    ap.add_argument("--profile", action="store_true",
                    help="run --warmup registrations then one registration and exit (for ncu launch lists)")
    ap.add_argument("--profile-net", action="store_true",
                    help="run 4 training steps of the warm-start network (256^2, batch 8) and exit (for ncu)")
    ap.add_argument("--profile-grid", type=int, default=0,
                    help="with --profile: instead run a gradient and 3 GN matvecs on this grid (nt=32)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile_net:
        import torch
        from paper_1503_00757_gb300 import warmstart as ws
        from paper_1503_00757_gb300.binding import Net, flatten_params
        x = torch.from_numpy(ws.make_images(256, range(ws.TRAIN_SEED, ws.TRAIN_SEED + 8))).cuda().contiguous()
        t = torch.zeros(8, 2, 256, 256, device="cuda")
        net = Net(256, 256, 8)
        net.set_params(torch.tensor(flatten_params(ws.he_init(1)), dtype=torch.float32, device="cuda"))
        losses = [net.train_step(x, t, 1e-3) for _ in range(4)]
        torch.cuda.synchronize()
        print(json.dumps({"profile_net": True, "losses": losses}))
        net.close()
        return

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1503_00757_gb300 import build as libbuild
    if not os.path.exists(libbuild.LIB_PATH):
        libbuild.build()
    from paper_1503_00757_gb300.binding import Context, default_opts

    from paper_1503_00757_gb300.binding import Executor, autotune

    # FFT tiles of the workload's grid, picked once by the autotuner before any context exists
    # (with --profile-grid: the tiles of that grid instead)
    tR, tC, tP, tD, _ = autotune(args.profile_grid or N_GRID, args.profile_grid or N_GRID, nt=8,
                                 concurrency=1 if args.profile_grid else PAIRS)

    # the step's batch: PAIRS independent registrations of this rank (seeds differ per rank)
    pairs_np = [images(s) for s in rank_seeds(rank)]
    mT_np, mR_np = pairs_np[0]
    pairs = [dict(mT=torch.from_numpy(a).to(dev), mR=torch.from_numpy(b).to(dev),
                  v=torch.zeros(2, N_GRID, N_GRID, device=dev), nt=NT, regnorm=1, beta=BETA,
                  gamma=math.inf, shear=0.0, detgrad=1) for a, b in pairs_np]
    mT, mR = pairs[0]["mT"], pairs[0]["mR"]
    stream = torch.cuda.Stream(device=dev)
    ctx = Context(N_GRID, N_GRID, NT, regnorm=1, beta=BETA, gamma=math.inf, shear=0.0, stream=stream)
    v = torch.zeros(2, N_GRID, N_GRID, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    opts = default_opts(tol=1e-2)
    ex = Executor(PAIRS)
    stats = {}

    def single():
        ctx.set_images(mT, mR)
        st = ctx.solve(v, opts)
        det = ctx.detgrad(v)
        return st, det

    def step():
        _, st = ex.solve(pairs, opts)
        return st

    def barrier():
        if world > 1:
            dist.barrier()

    if args.profile and args.profile_grid:
        nb = args.profile_grid
        from paper_1503_00757_gb300 import synth
        bT, bR, bv = synth.ellipses_pair(nb, SEED, vmax=VMAX * N_GRID / nb)
        cb = Context(nb, nb, NT, regnorm=1, beta=BETA, gamma=math.inf, shear=0.0, stream=stream)
        with torch.cuda.stream(stream):
            cb.set_images(torch.from_numpy(bT.astype(np.float32)).to(dev), torch.from_numpy(bR.astype(np.float32)).to(dev))
            vb = torch.from_numpy((0.5 * bv).astype(np.float32)).to(dev).contiguous()
            gb = torch.empty_like(vb)
            cb.gradient(vb, gb)
            vtb = torch.randn_like(vb)
            Hb = torch.empty_like(vb)
            for _ in range(3):
                cb.hessian_matvec(vtb, Hb)
            torch.cuda.synchronize()
        print(json.dumps({"profile": True, "grid": nb, "launches": cb.launch_count()}))
        cb.close()
        return

    if args.profile:
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                single()
            torch.cuda.synchronize()
            l0 = ctx.launch_count()
            st, _ = single()
            torch.cuda.synchronize()
        print(json.dumps({"profile": True, "launches_warmup": l0, "launches_step": ctx.launch_count() - l0,
                          "solve": {k: st[k] for k in ("n_newton", "n_mv", "n_pde", "n_ls")}}))
        ctx.close()
        return

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            bstats = step()
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        import tempfile
        clocks = Clocks(local, args.clocks_dir or tempfile.gettempdir())
        clocks.start()
        total_ms = 0.0
        wall = 0.0
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            t0 = time.perf_counter()
            e0.record(stream)
            bstats = step()  # synchronous: returns after every pair's work has finished
            e1.record(stream)
            e1.synchronize()
            wall += time.perf_counter() - t0
            total_ms += e0.elapsed_time(e1)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms_step = aggregate_ms(total_ms / args.steps, world, dist if world > 1 else None, dev)
        value = throughput(ms_step, world)

        # single-stream measurements (one registration alone, matvecs/s) with the tiles and launch mode
        # tuned for one solve at a time
        sR, sC, sP, sD, _ = autotune(N_GRID, N_GRID, nt=8, concurrency=1, force=True)
        ctx.set_tiles(sR, sC, sP)
        ctx.set_pdl(sD)
        # single-registration latency (one pair alone on one stream)
        for _ in range(2):
            stats, det = single()
        torch.cuda.synchronize()
        lat = 0.0
        nlat = 3
        l0 = ctx.launch_count()
        for _ in range(nlat):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            stats, det = single()
            e1.record(stream)
            e1.synchronize()
            lat += e0.elapsed_time(e1)
        launches_single = (ctx.launch_count() - l0) // nlat
        launches = launches_single * PAIRS
        lat /= nlat

        # e2e: the same batch from pinned host buffers (H2D of images, D2H of velocities and stats inside)
        hpairs = [(torch.from_numpy(a).pin_memory(), torch.from_numpy(b).pin_memory()) for a, b in pairs_np]
        hv = [torch.empty(2, N_GRID, N_GRID, dtype=torch.float32).pin_memory() for _ in range(PAIRS)]
        torch.cuda.synchronize()
        e2e_ms = 0.0
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for p, (a, b) in zip(pairs, hpairs):
                p["mT"].copy_(a, non_blocking=True)
                p["mR"].copy_(b, non_blocking=True)
            stream.synchronize()
            step()
            for p, h in zip(pairs, hv):
                h.copy_(p["v"], non_blocking=True)
            e1.record(stream)
            e1.synchronize()
            e2e_ms += e0.elapsed_time(e1)
        e2e_value = throughput(aggregate_ms(e2e_ms / args.steps, world, dist if world > 1 else None, dev), world)

        # Hessian matvec throughput at a fixed linearization point (the converged v)
        g = torch.empty_like(v)
        ctx.gradient(v, g)
        vt = torch.randn_like(v)
        Hv = torch.empty_like(v)
        for _ in range(5):
            ctx.hessian_matvec(vt, Hv)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.matvecs):
            ctx.hessian_matvec(vt, Hv)
        e1.record(stream)
        e1.synchronize()
        mv_ms = e0.elapsed_time(e1) / args.matvecs

        # roofline: per-kernel-class CUDA-event timing over one more registration
        ctx.kernel_timing(True)
        ctx.set_images(mT, mR)
        ctx.solve(v, opts)
        torch.cuda.synchronize()
        classes = {}
        names = ["column FFT + multiplier", "row FFT + RK2 stage", "row FFT (other)", "pointwise/reduction"]
        for kc in range(4):
            n, ms, byt = ctx.kernel_time(kc)
            classes[kc] = (n, ms, byt)
        ctx.kernel_timing(False)

        # HBM regime: 1024^2, nt=32 (history 132 MiB + 264 MiB > L2): matvec throughput and per-class roofline
        big = {}
        if args.big:
            nb = 1024
            from paper_1503_00757_gb300 import synth
            bT, bR, bv = synth.ellipses_pair(nb, SEED, vmax=0.049)
            autotune(nb, nb, nt=8, concurrency=1)
            ctxb = Context(nb, nb, NT, regnorm=1, beta=BETA, gamma=math.inf, shear=0.0, stream=stream)
            ctxb.set_images(torch.from_numpy(bT.astype(np.float32)).to(dev), torch.from_numpy(bR.astype(np.float32)).to(dev))
            vb = torch.from_numpy((0.5 * bv).astype(np.float32)).to(dev).contiguous()
            gb = torch.empty_like(vb)
            ctxb.gradient(vb, gb)
            vtb = torch.randn_like(vb)
            Hb = torch.empty_like(vb)
            for _ in range(3):
                ctxb.hessian_matvec(vtb, Hb)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            nmv = 20
            e0.record(stream)
            for _ in range(nmv):
                ctxb.hessian_matvec(vtb, Hb)
            e1.record(stream)
            e1.synchronize()
            big["ms_per_matvec"] = e0.elapsed_time(e1) / nmv
            ctxb.kernel_timing(True)
            for _ in range(3):
                ctxb.hessian_matvec(vtb, Hb)
            torch.cuda.synchronize()
            bcls = {kc: ctxb.kernel_time(kc) for kc in range(4)}
            ctxb.kernel_timing(False)
            ctxb.close()
            bd = max(bcls, key=lambda k: bcls[k][1])
            ach = bcls[bd][2] / (bcls[bd][1] * 1e-3) / 1e9 if bcls[bd][1] > 0 else 0.0
            big["roofline"] = {"kernel": ["column FFT + multiplier", "row FFT + RK2 stage", "row FFT (other)",
                                          "pointwise/reduction"][bd], "achieved": ach, "launches": bcls[bd][0]}
            big["kernel_classes"] = {str(k): {"launches": bcls[k][0], "ms": bcls[k][1], "GB": bcls[k][2] / 1e9}
                                     for k in bcls}
        # learned warm start vs plain zero start (256^2, nt=16, held-out pairs) with the committed weights
        warm = None
        wpath = os.path.join(ROOT, "paper_1503_00757_gb300", "weights", "warmstart_n256.npy")
        if args.warm and os.path.exists(wpath):
            from paper_1503_00757_gb300 import warmstart as ws
            from paper_1503_00757_gb300.binding import Net
            xw = ws.make_images(256, range(ws.TEST_SEED, ws.TEST_SEED + 16))
            exw = Executor(8)
            netw = Net(256, 256, 8)
            netw.set_params(torch.from_numpy(np.load(wpath).astype(np.float32)).to(dev))
            mpath = os.path.splitext(wpath)[0] + ".json"
            wscale = json.load(open(mpath))["output_scale"] if os.path.exists(mpath) else 1.0
            netw.set_output_scale(wscale)
            ws.solve_all(xw[:8], exw, opts)  # warm-up (contexts, graphs)
            _, st0, s0 = ws.solve_all(xw, exw, opts)
            t0 = time.perf_counter()
            vp = ws.predict(netw, xw, 8)
            sp = time.perf_counter() - t0
            _, st1, s1 = ws.solve_all(xw, exw, default_opts(tol=1e-2, warm_start=1), v0=vp)
            z, w_ = ws.summarize(st0, s0), ws.summarize(st1, s1 + sp)
            warm = {"workload": "learned warm start 256x256, nt=16, H1, beta_v=1e-3, incompressible, 16 held-out pairs, tol 1e-2",
                    "output_scale": wscale,
                    "plain": z, "warm": w_, "matvec_reduction": 1.0 - w_["matvec_mean"] / z["matvec_mean"],
                    "speedup": w_["registrations_per_s"] / z["registrations_per_s"]}
            netw.close()
            exw.close()
        # shear-control model (nonlinear Stokes, s = -1/2: shear thickening, +1/2: shear thinning) on the
        # first 512^2 pair: a full solve and Hessian matvecs/s at its solution (one context, single-stream tiles)
        shear = {}
        if args.shear:
            for s_ in (-0.5, 0.5):
                cs = Context(N_GRID, N_GRID, NT, regnorm=1, beta=BETA, gamma=math.inf, shear=s_, stream=stream)
                cs.set_images(mT, mR)
                vsh = torch.zeros(2, N_GRID, N_GRID, device=dev)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                sts = cs.solve(vsh, opts, check=False)
                torch.cuda.synchronize()
                tsol = time.perf_counter() - t0
                gs, Hs_, vts = torch.empty_like(vsh), torch.empty_like(vsh), torch.randn_like(vsh)
                cs.gradient(vsh, gs)
                for _ in range(3):
                    cs.hessian_matvec(vts, Hs_)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(50):
                    cs.hessian_matvec(vts, Hs_)
                e1.record(stream)
                e1.synchronize()
                shear[str(s_)] = {"nu": (1 + s_) / (1 - s_), "solve_ms": 1e3 * tsol,
                                  "solve": {k: sts[k] for k in ("rc", "n_newton", "n_mv", "gnorm_rel", "rnorm_rel_sq")},
                                  "matvec_per_s": 1e3 * 50 / e0.elapsed_time(e1)}
                cs.close()
        batched_mixed = run_batched_mixed(dev, stream, opts) if (args.batched and rank == 0) else None
    from paper_1503_00757_gb300.binding import fp32_peak
    fp32_tf, _ = fp32_peak()
    dom = max(classes, key=lambda k: classes[k][1])
    n_dom, ms_dom, bytes_dom = classes[dom]
    peak, peak_kind = peaks()
    achieved = (bytes_dom / (ms_dom * 1e-3)) / 1e9 if ms_dom > 0 else 0.0

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        t_pde = cpu_oracle_pde_time(mT_np, mR_np)
        n_pde = stats.get("n_pde", PDE_PER_REG)
        cpu = {"value": 1.0 / (t_pde * n_pde), "unit": "registrations/s", "cores": 1, "kind": "oracle",
               "sample": f"one FP64 oracle state solve (512^2, nt=32) = {t_pde:.1f} s, scaled by the "
                         f"{n_pde} PDE solves of the GPU registration"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "registrations/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [N_GRID, N_GRID], "nt": NT, "pairs_per_step": PAIRS,
                       "tiles": {"rows_per_cta": tR, "cols_per_cta": tC, "prefetch": tP, "pdl": tD,
                                 "tuned_for": f"{PAIRS} concurrent solves"},
                       "tiles_single_stream": {"rows_per_cta": sR, "cols_per_cta": sC, "prefetch": sP, "pdl": sD,
                                               "used_for": "latency_ms_single_registration, matvec_per_s"},
                       "l2": "flushed between steps", "parallelism": f"replicas x{world}, {PAIRS} concurrent streams",
                       "start": "zero (plain); warm start reported in warm_start_vs_plain"},
            "latency_ms_single_registration": lat,
            "warm_start_vs_plain": warm,
            "batched_mixed_vs_sequential": batched_mixed,
            "shear_control_512": shear or None,
            "matvec_per_s": 1e3 / mv_ms, "ms_per_matvec": mv_ms,
            "solve": {k: stats[k] for k in ("n_newton", "n_mv", "n_pde", "n_ls", "gnorm_rel", "rnorm_rel_sq", "status")},
            "solve_batch": [{k: b[k] for k in ("n_newton", "n_mv", "gnorm_rel", "rc")} for b in bstats],
            "detF": {"min": det[0], "mean": det[1], "max": det[2], "maxD": det[3]},
            "e2e": {"value": e2e_value, "unit": "registrations/s", "h2d_bytes_per_step": PAIRS * 2 * 4 * N_GRID * N_GRID,
                    "d2h_bytes_per_step": PAIRS * 2 * 4 * N_GRID * N_GRID},
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": ROW_STAGE_TRAFFIC_512 if dom == 1 else None, "kernel": names[dom],
                         "launches": n_dom, "ms": ms_dom, "peak_kind": peak_kind},
            "matvec_1024": ({"ms_per_matvec": big["ms_per_matvec"], "matvec_per_s": 1e3 / big["ms_per_matvec"],
                             "roofline": {"bound": "hbm", "kernel": big["roofline"]["kernel"],
                                          "achieved": big["roofline"]["achieved"], "peak": peak,
                                          "frac": big["roofline"]["achieved"] / peak, "unit": "GB/s"},
                             "kernel_classes": big["kernel_classes"]} if big else None),
            "ceilings": {"fp32_tflops_measured": fp32_tf, "hbm_gbs": peak,
                         "matvec_512": matvec_models(N_GRID, N_GRID, NT, mv_ms, peak, fp32_tf),
                         "matvec_1024": (matvec_models(1024, 1024, NT, big["ms_per_matvec"], peak, fp32_tf)
                                         if big else None)},
            "kernel_classes": {names[k]: {"launches": classes[k][0], "ms": classes[k][1],
                                          "GB": classes[k][2] / 1e9} for k in classes},
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    ctx.close()
    ex.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
