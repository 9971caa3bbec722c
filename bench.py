"""Benchmark: registrations/s and Gauss-Newton Hessian matvecs/s at 512^2, nt=32.

Workload: synthetic "brain-like" nested smoothed ellipses (5 labels, random
contrasts), reference = template displaced by a divergence-free velocity with
modes |k| <= 16 (max |v| = 0.098, CFL 0.25 at nt = 32); H1 seminorm,
incompressible (div v = 0), beta_v = 1e-3, zero start, relative gradient 1e-2.
One step = PAIRS independent full Newton-Krylov registrations (reg_solve:
state, adjoint, gradient, PCG with GN matvecs, Armijo, Newton) plus det F1
(reg_detgrad) of each, solved concurrently through the batch executor.

Arms:
  default            the CUDA library through the C ABI.  `value`: device-resident
                     inputs.  `e2e`: one reg_register_host call per pair from
                     pinned host buffers (images in, velocity out inside the call)
                     on PAIRS host threads, each pair's context on its own stream,
                     then det F1 from the velocity copied back in.  Also: matvec
                     throughput (one context, and PAIRS contexts at once), the
                     roofline of the matvec against the streaming byte model, and
                     the FP64 oracle timed on the host cores (cpu_baseline).
  --impl reference   the FP64 oracle on the host cores: every step, one 512^2
                     Gauss-Newton matvec per core (a process pool).
Multi-GPU (torchrun): independent replicas, PAIRS registrations per rank
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
# PDE solves of one zero-start registration of this workload's first pair as
# counted by reg_solve on the GPU (stats n_pde: 5 Newton iterations, 38 matvecs,
# 5 line-search evaluations): the matvec equivalents (n_pde / 2) that turn the
# oracle's measured matvecs/s into registrations/s in the reference arm, which
# runs without a GPU.
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


def stream_bytes(n1, n2, nt):
    """Algorithmic bytes of one Gauss-Newton matvec, the minimal streaming model (FP32): the
    two transport sweeps each read the state history once (2 (nt+1) fields), round-trip one
    state per step (2 nt x 2 fields), and v, v~ are read and H v~ written (about 10 fields):
    about (24 nt + 40) N bytes, N = n1 n2."""
    return (24 * nt + 40) * n1 * n2


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per Gauss-Newton matvec at 512^2,
# nt = 32, summed over its 260 launches from one ncu capture of the current kernels (ncu flushes
# the caches before each launch, so this is the cold-cache traffic; command in the profiles
# folder's matvec traffic summary).
MATVEC_TRAFFIC_512 = 1.2932e9


def roofline(bytes_per_matvec, conc, ms_single, peak, peak_kind):
    """The matvec against the HBM roofline: algorithmic bytes (streaming model) per matvec
    times the matvecs completed, over the CUDA-event time of the window, with PAIRS contexts
    issuing matvecs at once (the concurrency of the registration step); the same for one
    context alone."""
    ach = bytes_per_matvec * conc["matvec_per_s"] / 1e9
    ach1 = bytes_per_matvec / ms_single / 1e6
    return {"bound": "hbm", "unit": "GB/s", "kernel": "Gauss-Newton matvec (all its kernels)",
            "bytes_per_matvec": bytes_per_matvec, "achieved": ach, "peak": peak, "peak_kind": peak_kind,
            "frac": ach / peak, "mode": f"{conc['contexts']} contexts issuing matvecs concurrently",
            "single_context": {"achieved": ach1, "frac": ach1 / peak, "ms_per_matvec": ms_single},
            "traffic": MATVEC_TRAFFIC_512}


def matvec_concurrent(dev, pairs, opts, nmv):
    """Gauss-Newton matvecs/s with one context per pair (each linearized at its pair's current
    velocity, a random direction), all issuing matvecs on their own streams at once; timed
    with CUDA events between a fork and a join on the current stream."""
    import torch
    from paper_1503_00757_gb300.binding import Context
    torch.cuda.synchronize()
    K = len(pairs)
    streams = [torch.cuda.Stream(device=dev) for _ in range(K)]
    gen = torch.Generator(device=dev)
    gen.manual_seed(11)
    ctxs, vts, Hs = [], [], []
    for p, s in zip(pairs, streams):
        c = Context(N_GRID, N_GRID, NT, regnorm=1, beta=BETA, gamma=math.inf, shear=0.0, stream=s)
        vt = torch.randn(2, N_GRID, N_GRID, device=dev, generator=gen)
        H = torch.empty_like(vt)
        g = torch.empty_like(vt)
        torch.cuda.synchronize()
        c.set_images(p["mT"], p["mR"])
        c.gradient(p["v"], g)
        for _ in range(3):
            c.hessian_matvec(vt, H)
        ctxs.append(c)
        vts.append(vt)
        Hs.append(H)
    torch.cuda.synchronize()
    cur = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(cur)
    for s in streams:
        s.wait_event(e0)
    for _ in range(nmv):
        for c, vt, H in zip(ctxs, vts, Hs):
            c.hessian_matvec(vt, H)
    for s in streams:
        e = torch.cuda.Event()
        e.record(s)
        cur.wait_event(e)
    e1.record(cur)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    for c in ctxs:
        c.close()
    return {"contexts": K, "matvecs": K * nmv, "ms": ms, "matvec_per_s": K * nmv * 1e3 / ms,
            "ms_per_matvec": ms / (K * nmv)}


def images(seed=SEED):
    from paper_1503_00757_gb300 import synth
    mT, mR, _ = synth.ellipses_pair(N_GRID, seed, vmax=VMAX)
    return mT.astype(np.float32), mR.astype(np.float32)


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
        R, C, P, D, ms = autotune(n, n, nt=C4_NT, concurrency=8, force=True)
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
            "design": "multi-stream executor (host worker threads, one stream each), not a persistent launch",
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


# ---------------------------------------------------------------------------
# FP64 oracle timed on the host cores (cpu_baseline and the reference arm).
# Worker processes are started with "spawn" (a fork after the first CUDA call
# can hang) and run one thread each (BLAS / OpenMP pools pinned to 1).
# ---------------------------------------------------------------------------
_ORACLE = {}


def _oracle_init(seed):
    """Worker set-up (untimed): the 512^2 workload's pair `seed`, its linearization point
    v = v*/2 (the oracle's gradient: state solve, adjoint, grad m history) and a
    band-limited direction v~."""
    from oracle.registration import Registration
    from paper_1503_00757_gb300 import synth
    mT, mR, vs = synth.ellipses_pair(N_GRID, seed, vmax=VMAX)
    P = Registration(mT, mR, NT, regnorm=1, beta_v=BETA, beta_w=math.inf)
    P.gradient(0.5 * vs)
    _ORACLE["P"] = P
    _ORACLE["vt"] = synth.velocity(N_GRID, N_GRID, 16, 0.3, np.random.default_rng(seed + 7))


def _oracle_matvec(_):
    """One FP64 Gauss-Newton matvec (incremental state and adjoint solves, b~, K); seconds."""
    t0 = time.perf_counter()
    _ORACLE["P"].matvec(_ORACLE["vt"])
    return time.perf_counter() - t0


def _oracle_register(spec):
    """One full FP64 registration (Algorithm 1: gradient, PCG, Armijo, Newton) from zero;
    returns (seconds, Newton iterations, matvecs, status)."""
    from oracle.registration import Registration
    from paper_1503_00757_gb300 import synth
    kind, n, nt, seed, regnorm, beta, gamma, vmax, policy = spec
    if kind == "blobs":
        mT, mR, _ = synth.blobs_pair(n, seed)
    else:
        mT, mR, _ = synth.ellipses_pair(n, seed, vmax=vmax)
    t0 = time.perf_counter()
    _, st = Registration(mT, mR, nt, regnorm=regnorm, beta_v=beta, beta_w=gamma).solve(tol=1e-2, nt_policy=policy)
    return time.perf_counter() - t0, st["n_newton"], st["n_mv"], st["status"]


def _oracle_pool(workers, init_seed=None):
    import multiprocessing as mp
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        if init_seed is None:
            return ctx.Pool(workers)
        return ctx.Pool(workers, initializer=_oracle_init, initargs=(init_seed,))
    finally:
        for k, val in saved.items():
            if val is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = val


def c1_specs(count):
    """C1 plain FP64 problems: 64^2 Gaussian blobs, H1, div v = 0, beta_v = 1e-2 (seeds 1000+), nt
    adapted to CFL 0.25 from nt = 4 per outer iteration (at the literal nt = 4, CFL 1.27, some
    seeds do not converge within 50 Newton iterations)."""
    return [("blobs", 64, 4, 1000 + i, 1, 1e-2, math.inf, None, "cfl") for i in range(count)]


def c4_subset_specs(count):
    """The first `count` 128^2 pairs of the mixed batch (nt = 16, their seeded settings)."""
    out = []
    for s in c4_specs():
        if s["n"] == 128 and len(out) < count:
            out.append(("ellipses", 128, C4_NT, s["seed"], s["regnorm"], s["beta"], s["gamma"], C4_VMAX[128],
                        "fixed"))
    return out


def cpu_oracle_baseline(pde_per_reg):
    """The FP64 oracle as it stands, timed on this host's cores (a bounded sample, ~1 min):
    full C1 registrations (1 core, all cores), 512^2 nt=32 Gauss-Newton matvecs (1 core:
    3 matvecs; all cores: one per core), 16 full 128^2 registrations of the mixed batch
    (all cores).  512^2 registrations/s = matvecs/s on all cores / (pde_per_reg / 2), the
    matvec equivalents of one registration of the workload (a matvec is two PDE solves)."""
    nproc = os.cpu_count() or 1
    res = {"nproc": nproc}
    with _oracle_pool(1) as pool:
        ts = pool.map(_oracle_register, c1_specs(3))
    res["c1_64_registrations_per_s_1core"] = len(ts) / sum(t[0] for t in ts)
    with _oracle_pool(nproc) as pool:
        t0 = time.perf_counter()
        ts = pool.map(_oracle_register, c1_specs(2 * nproc), chunksize=1)
        res["c1_64_registrations_per_s_allcores"] = len(ts) / (time.perf_counter() - t0)
        t0 = time.perf_counter()
        ts = pool.map(_oracle_register, c4_subset_specs(16), chunksize=1)
        res["c4_128_subset_pairs_per_s_allcores"] = len(ts) / (time.perf_counter() - t0)
        res["c4_128_subset_converged"] = sum(1 for t in ts if t[3] == 0)
    with _oracle_pool(1, SEED) as pool:
        ts = pool.map(_oracle_matvec, range(3))
    res["matvec_512_per_s_1core"] = len(ts) / sum(ts)
    with _oracle_pool(nproc, SEED) as pool:
        pool.map(_oracle_matvec, range(nproc), chunksize=1)  # every worker has finished its set-up
        t0 = time.perf_counter()
        pool.map(_oracle_matvec, range(nproc), chunksize=1)
        res["matvec_512_per_s_allcores"] = nproc / (time.perf_counter() - t0)
    value = res["matvec_512_per_s_allcores"] / (pde_per_reg / 2.0)
    return {"value": value, "unit": "registrations/s", "cores": nproc, "kind": "oracle",
            "sample": (f"FP64 oracle on {nproc} host cores: {nproc} Gauss-Newton matvecs at 512^2 nt=32 (one per "
                       f"core) timed, registrations/s = matvecs/s / {pde_per_reg / 2:g} matvec equivalents per "
                       f"registration of this workload; also timed: full 64^2 (C1, CFL nt) registrations on 1 "
                       f"and {nproc} cores, 3 matvecs on 1 core, 16 full 128^2 mixed-batch registrations"),
            "measured": res}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    nproc = os.cpu_count() or 1
    with _oracle_pool(nproc, SEED) as pool:
        for _ in range(max(1, args.warmup)):  # untimed: the first one also waits for every worker's set-up
            pool.map(_oracle_matvec, range(nproc), chunksize=1)
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            pool.map(_oracle_matvec, range(nproc), chunksize=1)
            times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    mv_per_s = nproc / t
    value = mv_per_s / (PDE_PER_REG / 2.0)
    sample = (f"per step {nproc} FP64 oracle Gauss-Newton matvecs at 512^2 nt=32, one per host core (process "
              f"pool); registrations/s = matvecs/s / {PDE_PER_REG / 2:g} matvec equivalents per registration "
              f"({PDE_PER_REG} PDE solves, counted by the GPU solve of this workload)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "registrations/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "config": {"workload": WORKLOAD},
        "matvec_per_s": mv_per_s,
        "cpu_baseline": {"value": value, "unit": "registrations/s", "cores": nproc, "kind": "oracle",
                         "sample": sample},
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
    ap.add_argument("--no-vol", dest="vol", action="store_false",
                    help="skip the three-dimensional gradient and matvec measurement (128^3, nt=16)")
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
    ap.add_argument("--conv-kernel", default="tcgen05", choices=["tcgen05", "mma_sync"],
                    help="with --profile-net: the convolution kernel of the network")
    ap.add_argument("--profile-grid", type=int, default=0,
                    help="with --profile: instead run a gradient and 3 GN matvecs on this grid (nt=32)")
    ap.add_argument("--transport", default="auto", choices=["auto", "cluster", "two-kernel"],
                    help="with --profile-grid: the transport path of the profiled context (auto: the tuned one)")
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
        from paper_1503_00757_gb300.binding import REG_CONV_MMA_SYNC, REG_CONV_TCGEN05
        net = Net(256, 256, 8)
        net.set_conv_kernel(REG_CONV_TCGEN05 if args.conv_kernel == "tcgen05" else REG_CONV_MMA_SYNC)
        net.set_params(torch.tensor(flatten_params(ws.he_init(1)), dtype=torch.float32, device="cuda"))
        losses = [net.train_step(x, t, 1e-3) for _ in range(4)]
        # forward passes (8 convolutions + the output projection), timed with CUDA events
        v = torch.empty(8, 2, 256, 256, device="cuda")
        for _ in range(3):
            net.forward(x, v)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(20):
            net.forward(x, v)
        e1.record()
        torch.cuda.synchronize()
        fwd_ms = e0.elapsed_time(e1) / 20
        # training steps (forward, backward, Adam; each reads its loss back)
        e0.record()
        for _ in range(10):
            net.train_step(x, t, 1e-4)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"profile_net": True, "conv_kernel": args.conv_kernel, "losses": losses,
                          "forward_ms": fwd_ms, "train_step_ms": e0.elapsed_time(e1) / 10}))
        net.close()
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # the oracle on the host cores first, before this process touches the GPU (its worker
    # processes are spawned; measured on an otherwise idle host)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline and not (args.profile or args.profile_grid):
        cpu = cpu_oracle_baseline(PDE_PER_REG)

    import torch
    import torch.distributed as dist

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
    tR, tC, tP, tD, _ = autotune(args.profile_grid or N_GRID, args.profile_grid or N_GRID, nt=NT,
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
    transport_tuned = ctx.transport_config()  # (cluster kernel chosen, CTAs per cluster, clusters that fit)
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
        if args.transport != "auto":
            cb.set_transport(args.transport == "cluster")
        with torch.cuda.stream(stream):
            cb.set_images(torch.from_numpy(bT.astype(np.float32)).to(dev), torch.from_numpy(bR.astype(np.float32)).to(dev))
            vb = torch.from_numpy((0.5 * bv).astype(np.float32)).to(dev).contiguous()
            gb = torch.empty_like(vb)
            vtb = torch.randn_like(vb)
            Hb = torch.empty_like(vb)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push("profile")  # ncu --nvtx --nvtx-include profile/ captures this part only
            cb.gradient(vb, gb)
            for _ in range(3):
                cb.hessian_matvec(vtb, Hb)
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
        print(json.dumps({"profile": True, "grid": nb, "launches": cb.launch_count(),
                          "transport": "cluster" if cb.transport_config()[0] else "two-kernel"}))
        cb.close()
        return

    if args.profile:
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                single()
            torch.cuda.synchronize()
            l0 = ctx.launch_count()
            torch.cuda.nvtx.range_push("profile")  # ncu --nvtx --nvtx-include profile/ captures this part only
            st, _ = single()
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_pop()
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
        sR, sC, sP, sD, _ = autotune(N_GRID, N_GRID, nt=NT, concurrency=1, force=True)
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

        # e2e through the public host-buffer call: per pair one reg_register_host (H2D of the
        # pinned images, the solve, D2H of the velocity inside the call) on its own host thread,
        # context and stream, then det F1 of the velocity copied back to the device
        import threading
        hstreams = [torch.cuda.Stream(device=dev) for _ in range(PAIRS)]
        hctx = [Context(N_GRID, N_GRID, NT, regnorm=1, beta=BETA, gamma=math.inf, shear=0.0, stream=hs)
                for hs in hstreams]
        hpairs = [(torch.from_numpy(a).pin_memory(), torch.from_numpy(b).pin_memory()) for a, b in pairs_np]
        hv = [torch.empty(2, N_GRID, N_GRID, dtype=torch.float32).pin_memory() for _ in range(PAIRS)]
        vdev = [torch.empty(2, N_GRID, N_GRID, device=dev) for _ in range(PAIRS)]
        e2e_stats = [None] * PAIRS

        def e2e_pair(i):
            c, hs = hctx[i], hstreams[i]
            st = c.register_host(hpairs[i][0], hpairs[i][1], hv[i], opts)
            with torch.cuda.stream(hs):
                vdev[i].copy_(hv[i], non_blocking=True)
            e2e_stats[i] = (st, c.detgrad(vdev[i]))  # reads the statistics back: synchronizes hs

        def e2e_step():
            ths = [threading.Thread(target=e2e_pair, args=(i,)) for i in range(PAIRS)]
            for t in ths:
                t.start()
            for t in ths:
                t.join()

        e2e_step()  # warm-up: captured launch sequences of the new contexts
        torch.cuda.synchronize()
        e2e_ms = 0.0
        for _ in range(args.steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e2e_step()
            e2e_ms += 1e3 * (time.perf_counter() - t0)
        for c in hctx:
            c.close()
        e2e_value = throughput(aggregate_ms(e2e_ms / args.steps, world, dist if world > 1 else None, dev), world)
        e2e_ok = all(st["rc"] == 0 for st, _ in e2e_stats)

        # Hessian matvec throughput at a fixed linearization point (the converged v): one
        # context alone, and PAIRS contexts (one per pair, each at its own solution) at once
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
        mv_conc = matvec_concurrent(dev, pairs, opts, args.matvecs // 4)
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
            autotune(nb, nb, nt=NT, concurrency=1)
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
            big["kernel_classes"] = {str(k): {"launches": bcls[k][0], "ms": bcls[k][1], "GB": bcls[k][2] / 1e9}
                                     for k in bcls}
        # three-dimensional problem: gradient and Gauss-Newton matvecs at 128^3, nt=16 (H1, div v = 0)
        vol = None
        if args.vol:
            from paper_1503_00757_gb300.binding import Context3D
            n3, nt3 = 128, 16
            xs = 2.0 * np.pi * np.arange(n3) / n3
            X1, X2, X3 = np.meshgrid(xs, xs, xs, indexing="ij")
            bump = lambda a, b, c: np.exp(-4.0 * (np.sin((X1 - a) / 2) ** 2 + np.sin((X2 - b) / 2) ** 2 +
                                                  np.sin((X3 - c) / 2) ** 2))
            f3 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
            c3 = Context3D(n3, n3, n3, nt3, beta=1e-2, gamma=math.inf, stream=stream)
            # a displacement of ~0.1 rad keeps the solution within the fixed-nt explicit scheme's
            # stability at 128^3 (max|v| h_t k_max < 1; the 3-D solve has no CFL nt policy)
            c3.set_images(f3(bump(3.0, 3.1, 2.9)), f3(bump(3.07, 3.04, 2.96)))
            v3 = f3(0.2 * np.stack([np.sin(X2 + X3), np.cos(X1) * np.sin(X3), np.sin(X1 - X2)]))
            vt3 = f3(0.1 * np.stack([np.cos(X3), np.sin(X1 + X3), np.cos(X2)]))
            g3_, H3_ = torch.empty_like(v3), torch.empty_like(v3)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c3.gradient(v3, g3_)
            torch.cuda.synchronize()
            e0.record(stream)
            c3.gradient(v3, g3_)
            e1.record(stream)
            e1.synchronize()
            ms_g3 = e0.elapsed_time(e1)
            c3.hessian_matvec(vt3, H3_)
            torch.cuda.synchronize()
            nmv3 = 5
            e0.record(stream)
            for _ in range(nmv3):
                c3.hessian_matvec(vt3, H3_)
            e1.record(stream)
            e1.synchronize()
            ms_mv3 = e0.elapsed_time(e1) / nmv3
            # a whole 3-D registration (Algorithm 1 from v = 0, tol 1e-2)
            vs3 = torch.empty_like(v3)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st3 = c3.solve(vs3, tol=1e-2, check=False)
            torch.cuda.synchronize()
            solve3 = dict(st3, seconds=time.perf_counter() - t0)
            c3.close()
            # streaming model: the gradient history (3 floats per point and time level) read twice,
            # v and v~ read, H v~ and b~ written once
            b3 = (24 * (nt3 + 1) + 48) * n3 ** 3
            pk3, _ = peaks()
            vol = {"workload": "128^3 periodic box, nt=16, H1, beta_v=1e-2, div v = 0 (reg3_*)",
                   "ms_per_gradient": ms_g3, "ms_per_matvec": ms_mv3, "matvec_per_s": 1e3 / ms_mv3,
                   "solve": solve3,
                   "roofline_streaming": {"bytes_per_matvec": b3, "GB/s": b3 / ms_mv3 / 1e6,
                                          "frac_hbm": b3 / ms_mv3 / 1e6 / pk3}}
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
            # the network on this benchmark's own 512^2, nt=32 pairs: zero start against the prediction,
            # same stopping test, through the executor that times `value`; the prediction made at the
            # network's training resolution (images restricted to 256^2, velocity prolonged back,
            # reg_net_forward_fine) and, for comparison, by the fully convolutional network applied at 512^2
            xb = torch.stack([torch.stack([p_["mT"], p_["mR"]]) for p_ in pairs]).contiguous()

            def run512(v0, o):
                ps = [dict(p_, v=(torch.zeros(2, N_GRID, N_GRID, device=dev) if v0 is None else v0[i].clone()),
                           detgrad=0) for i, p_ in enumerate(pairs)]
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                _, st_ = ex.solve(ps, o, check=False)
                torch.cuda.synchronize()
                return st_, time.perf_counter() - t0

            st0b, s0b = run512(None, opts)
            zb = ws.summarize(st0b, s0b)
            warm["at_512"] = {"workload": WORKLOAD.split(";")[0] + f"; {PAIRS} pairs of this step, tol 1e-2",
                              "plain": zb}
            for tag, grid, fine in (("warm_restricted_256", N_GRID // 2, True), ("warm_direct_512", N_GRID, False)):
                netb = Net(grid, grid, PAIRS)
                netb.set_params(torch.from_numpy(np.load(wpath).astype(np.float32)).to(dev))
                netb.set_output_scale(wscale)
                vpb = torch.empty(PAIRS, 2, N_GRID, N_GRID, device=dev)
                (netb.forward_fine if fine else netb.forward)(xb, vpb)  # first call: allocation and set-up
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                (netb.forward_fine if fine else netb.forward)(xb, vpb)
                torch.cuda.synchronize()
                spb = time.perf_counter() - t0
                st1b, s1b = run512(vpb, default_opts(tol=1e-2, warm_start=1))
                wb = ws.summarize(st1b, s1b + spb)
                warm["at_512"][tag] = dict(wb, matvec_reduction=1.0 - wb["matvec_mean"] / zb["matvec_mean"],
                                           speedup=wb["registrations_per_s"] / zb["registrations_per_s"])
                netb.close()
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
    peak, peak_kind = peaks()

    if rank == 0:
        names = ["column FFT + multiplier", "row FFT + RK2 stage", "row FFT (other)", "pointwise/reduction"]
        sb512 = stream_bytes(N_GRID, N_GRID, NT)
        line = {
            "metric": METRIC, "value": value, "unit": "registrations/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": [N_GRID, N_GRID], "nt": NT, "pairs_per_step": PAIRS,
                       "tiles": {"rows_per_cta": tR, "cols_per_cta": tC, "prefetch": tP, "pdl": tD,
                                 "transport": "cluster-resident" if transport_tuned[0] else "row/column kernel pairs",
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
            "matvec_concurrent": mv_conc,
            "solve": {k: stats[k] for k in ("n_newton", "n_mv", "n_pde", "n_ls", "gnorm_rel", "rnorm_rel_sq", "status")},
            "solve_batch": [{k: b[k] for k in ("n_newton", "n_mv", "gnorm_rel", "rc")} for b in bstats],
            "detF": {"min": det[0], "mean": det[1], "max": det[2], "maxD": det[3]},
            "e2e": {"value": e2e_value, "unit": "registrations/s", "all_converged": e2e_ok,
                    "call": "reg_register_host per pair (pinned host buffers) + reg_detgrad, one host thread per pair",
                    "h2d_bytes_per_step": PAIRS * (1 + 1 + 2) * 4 * N_GRID * N_GRID,
                    "d2h_bytes_per_step": PAIRS * (2 * 4 * N_GRID * N_GRID + 5 * 8)},
            "gpu_launches": launches,
            "roofline": roofline(sb512, mv_conc, mv_ms, peak, peak_kind),
            "matvec_1024": ({"ms_per_matvec": big["ms_per_matvec"], "matvec_per_s": 1e3 / big["ms_per_matvec"],
                             "roofline_single_context": {
                                 "bound": "hbm", "unit": "GB/s", "bytes_per_matvec": stream_bytes(1024, 1024, NT),
                                 "achieved": stream_bytes(1024, 1024, NT) / big["ms_per_matvec"] / 1e6,
                                 "peak": peak,
                                 "frac": stream_bytes(1024, 1024, NT) / big["ms_per_matvec"] / 1e6 / peak},
                             "kernel_classes": big["kernel_classes"]} if big else None),
            "matvec_3d": vol,
            "ceilings": {"fp32_tflops_measured": fp32_tf, "hbm_gbs": peak,
                         "matvec_512": matvec_models(N_GRID, N_GRID, NT, mv_ms, peak, fp32_tf),
                         "matvec_512_concurrent": matvec_models(N_GRID, N_GRID, NT, mv_conc["ms_per_matvec"], peak,
                                                                fp32_tf),
                         "matvec_1024": (matvec_models(1024, 1024, NT, big["ms_per_matvec"], peak, fp32_tf)
                                         if big else None)},
            "kernel_classes": {names[k]: {"launches": classes[k][0], "ms": classes[k][1],
                                          "GB_library_tally": classes[k][2] / 1e9} for k in classes},
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
