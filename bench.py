"""Throughput of the laboratory-frame Glasma CPIC leapfrog step on GB300.

Workload (default): the SU(3) single event, N_L = 512 x 64^2 transverse,
dt = a/2, sigma_L = 8a, g^2 mu a = 0.1, m = 0.2/a, synthetic MV charges from
a fixed seed; FP32 links and fields, FP64 reductions.  One bench step = one
lattice time step of the whole event (CPIC hop on the scheduled steps,
E update, link update).  Metric: site-updates/s (sites x steps / time).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W]
                       [--impl ours|reference] [--precision fp32|fp64]
Under torchrun (N > 1) every rank evolves its own event (replicas, no data
exchange); value = all ranks' site-updates / max-over-ranks time.

The reference arm (--impl reference) times the FP64 CPU oracle, as it
stands, on the host cores: each step is one oracle step of a two-slice
64 x 64 slab of the same SU(3) workload (a bounded sample).

Fields of the JSON line beyond the metric:
  roofline      the step kernel (the only kernel of the timed region):
                achieved = compulsory bytes per launch (read and write 3
                links and 3 fields per site, plus the charge windows on hop
                steps) / its launch time from CUDA events, against the
                measured HBM copy bandwidth; traffic = DRAM bytes per launch
                from the committed ncu capture (null once the kernel sources
                differ from the captured ones, or for another kernel than
                the captured one); fma_pipe = the FFMA count of
                the same capture over the launch time, against 152 SMs x 128
                FP32 lanes x the maximum SM clock
  e2e           the same metric through the C ABI from host charges: the
                initial state, the workload's steps (at most 400; K if
                larger) and T^{mu nu} to the host, wall
                clock, with the bytes copied each way per step
  cpu_baseline  the FP64 oracle on a bounded slab of the workload, with the
                cores it used
  clocks        SM clocks and throttle reasons sampled during the timed
                region
  extras        (unless --no-extras) the FP64 path and the FP32 energy-
                density error against it, one T^{mu nu} sample, the improved
                scheme on its 2048 x 128^2 workload, the batched ensemble,
                the rest-frame analysis, the adjoint gradient, and the
                event split into z slabs with their halo exchange on one GPU
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import glasma_inputs as gi  # noqa: E402

WORKLOAD = "su3_512x64x64"
METRIC = "site-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--nz", type=int, default=0,
                    help="override the lattice length (profiling on a smaller case)")
    ap.add_argument("--kernel", default="auto",
                    choices=["auto", "staple", "staple_staged", "staple_pairs",
                             "plaquette", "plaquette_256"],
                    help="leapfrog step kernel (glasma_set_step_kernel)")
    ap.add_argument("--zlen", type=int, default=0,
                    help="z slices per block of the plaquette kernel (0 = automatic)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64 comparison, e2e and error check")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# bytes per site-update of the step kernel (compulsory HBM traffic)
# ---------------------------------------------------------------------------

def bytes_per_site(nc, rs):
    """Read and write the three links (SU(2): 4 reals, SU(3): 18 reals) and
    the three E fields (nc^2 - 1 reals) of one site once."""
    link = (4 if nc == 2 else 18) * rs
    field = (nc * nc - 1) * rs
    return 2 * 3 * (link + field)


def step_kernel_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2009_02044_gb300", "csrc")
    for f in ("k_step.cu", "step_link.cuh", "link_alg.cuh", "lattice.cuh",
              "su_n.cuh", "step_pair.cuh", "pair.cuh", "k_step_plaq.cu",
              "k_step_staged.cu"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def step_kernel_name(nc, precision, kernel, nx=64):
    """The CUDA kernel glasma_step launches for this choice (the library's
    automatic choice: plaquette kernel in FP64; in FP32 the staged staple
    kernel for SU(3) rows of 64 sites, else the one-site staple kernel)."""
    if kernel == "auto":
        kernel = ("plaquette" if precision == "fp64" else
                  "staple_staged" if (nc == 3 and nx == 64) else "staple")
    return {"staple": "k_step_leapfrog", "staple_pairs": "k_step_pair",
            "staple_staged": "k_step_staged",
            "plaquette": "k_step_plaq", "plaquette_256": "k_step_plaq"}[kernel]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def load_profile_entry(workload, precision, nz, kernel=None):
    """The committed ncu figures of the step kernel (per-launch DRAM bytes
    and FFMA count), valid only for the workload's own lattice, for the
    kernel they were taken on (`kernel`, a CUDA kernel name, if given) and
    if the kernel sources are unchanged since; else None."""
    path = os.path.join(ROOT, "profiles", "step_traffic.json")
    try:
        if nz != gi.CONFIGS[workload]["nz"]:
            return None
        d = json.load(open(path))
        e = d[workload + ":" + precision]
        if kernel is not None and not e.get("kernel", "").startswith(kernel):
            return None
        if e["kernel_hash"] == step_kernel_hash():
            return e
    except Exception:
        pass
    return None


def load_traffic(workload, precision, nz, kernel=None):
    e = load_profile_entry(workload, precision, nz, kernel)
    return e["dram_bytes_per_launch"] if e else None


# FP32 FMA lanes per SM and SMs of a GB300: the ALU peak is lanes x SMs x
# the maximum SM clock
FP32_LANES_PER_SM, GB300_SMS = 128, 152


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (baseline and reference arm)
# ---------------------------------------------------------------------------

def oracle_sample_state(cfg, nz, seed=0, charges=True):
    from oracle import glasma_oracle as O
    p = O.Params.from_dict(dict(cfg, nz=nz))
    rng = np.random.default_rng(seed)
    nc, na = p.nc, p.na
    U = gi.near_identity_su(nc, (3, nz, p.ny, p.nx), rng, 0.1)
    U[2][nz - 1] = np.eye(nc)
    E = 0.01 * rng.standard_normal((3, nz, p.ny, p.nx, na))
    E[2][nz - 1] = 0.0
    QA = np.zeros((nz, p.ny, p.nx, na))
    QB = np.zeros((nz, p.ny, p.nx, na))
    if charges:  # one slice of B charges, kept clear of the upper boundary
        QB[0] = 0.01 * rng.standard_normal(QB[0].shape)
    return O, O.State(p, U, E, QA, QB, 0)


def oracle_threads():
    try:
        from threadpoolctl import threadpool_info
        n = max([d.get("num_threads", 1) for d in threadpool_info()] + [1])
        return int(n)
    except Exception:
        return 1


def cpu_baseline(cfg, slices=16, steps=8):
    O, st = oracle_sample_state(cfg, slices)
    V = slices * cfg["nx"] * cfg["ny"]
    t = time.perf_counter()
    s = O.step(st, steps)
    dt = time.perf_counter() - t
    del s
    return {"value": V * steps / dt, "unit": METRIC, "cores": 1,
            "blas_threads": oracle_threads(), "kind": "oracle",
            "sample": "%d FP64 oracle steps of a %d-slice %dx%d slab of the "
                      "SU(3) workload (%d sites), %.1f s"
                      % (steps, slices, cfg["nx"], cfg["ny"], V, dt)}


def run_reference(args, cfg):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    slices = 2
    O, st = oracle_sample_state(cfg, slices, charges=False)
    V = slices * cfg["nx"] * cfg["ny"]
    for _ in range(args.warmup):
        st = O.step(st, 1)
    t = time.perf_counter()
    for _ in range(args.steps):
        st = O.step(st, 1)
    dt = time.perf_counter() - t
    v = V * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": METRIC,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded SU(3) links/fields)",
        "config": {"workload": args.workload, "sample": "%d-slice %dx%d slab"
                   % (slices, cfg["nx"], cfg["ny"])},
        "cpu_baseline": {"value": v, "unit": METRIC, "cores": 1,
                         "kind": "oracle",
                         "sample": "one FP64 oracle step of a %d-slice "
                                   "%dx%d slab (%d sites) per bench step"
                                   % (slices, cfg["nx"], cfg["ny"], V)},
        "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def aggregate(ms_local, sites_per_rank, steps, world):
    """Whole-job throughput of `world` replicas: every rank evolved its own
    event of `sites_per_rank` sites for `steps` steps; the job takes as long
    as the slowest rank (max over ranks of the device time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_local)], dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * sites_per_rank * steps / (ms_max * 1e-3)


def run_ours(args, cfg):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("gloo")
    from paper_2009_02044_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    from paper_2009_02044_gb300 import glasma as G

    cfg = dict(cfg, precision=args.precision, seed=cfg["seed"] + rank)
    stream = torch.cuda.Stream()
    nc = cfg["nc"]
    rs = 4 if args.precision == "fp32" else 8
    V = cfg["nz"] * cfg["nx"] * cfg["ny"]
    W, K = args.warmup, args.steps
    if W < 3:
        raise SystemExit("warmup must be >= 3")

    with torch.cuda.stream(stream):
        h = G.glasma_init_mv(cfg, None, stream=stream)
    G.glasma_set_step_kernel(h, args.kernel, args.zlen)
    G.glasma_step(h, W)
    info = G.glasma_get_info(h)
    state_bytes = info.state_device_bytes
    # count the hop launches in the timed window for the algorithmic bytes
    from fractions import Fraction
    r = Fraction(cfg["dt"]) / Fraction(cfg.get("a_z", 1.0))
    pp, qq = r.numerator, r.denominator
    hops = sum(1 for n in range(W, W + K)
               if (2 * (n + 1) * pp + qq) // (2 * qq) > (2 * n * pp + qq) // (2 * qq))
    na = nc * nc - 1
    qbytes = 2 * rs * na * (info.window_a[1] + info.window_b[1]) * cfg["nx"] * cfg["ny"]

    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        G.glasma_step(h, K)
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    launches = G.glasma_get_info(h).kernel_launches
    ms_max, value = aggregate(ms, V, K, world)

    # roofline of the step kernel (the only kernel in the timed region of a
    # leapfrog workload; implicit workloads report their sweep roofline in
    # the "improved" field)
    per_launch_ms = ms / launches
    alg = V * bytes_per_site(nc, rs) + (hops / K) * qbytes
    peak, peak_kind = load_peaks()
    achieved = alg / (per_launch_ms * 1e-3) / 1e9
    kname = step_kernel_name(nc, args.precision, args.kernel, cfg["nx"])
    prof = load_profile_entry(args.workload, args.precision, cfg["nz"], kname)
    traffic = prof["dram_bytes_per_launch"] if prof else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak,
            "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
            "kernel": kname,
            "peak_source": peak_kind,
            "alg_bytes_per_launch": alg}
    if prof and prof.get("ffma_per_launch"):
        # the FP32 FMA pipe next to HBM: the kernel's FFMA count (ncu) over
        # its live launch time, against lanes x SMs x the maximum SM clock
        mhz = clk.summary().get("sm_max_mhz") or 2070.0
        peak_fma = FP32_LANES_PER_SM * GB300_SMS * mhz * 1e6 / 1e12
        got_fma = prof["ffma_per_launch"] / (per_launch_ms * 1e-3) / 1e12
        roof["fma_pipe"] = {"achieved": got_fma, "peak": peak_fma, "unit": "TFMA/s",
                            "frac": got_fma / peak_fma,
                            "ffma_per_launch": prof["ffma_per_launch"],
                            "peak_source": "152 SMs x 128 FP32 lanes x max SM clock"}

    extras = {}
    if rank == 0 and not args.no_extras:
        extras = run_extras(G, torch, cfg, args, stream, value)
    gauss = G.glasma_gauss_residual(h)
    G.glasma_free(h)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": METRIC,
            "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_max / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else "f64",
            "data": "synthetic (MV charges, seeded Philox)",
            "config": {"workload": args.workload, "nc": nc,
                       "lattice": [cfg["nz"], cfg["ny"], cfg["nx"]],
                       "dt": cfg["dt"], "sigma_l": cfg["sigma_l"],
                       "g2mu": cfg["g2mu"], "m_ir": cfg["m_ir"],
                       "scheme": cfg.get("scheme", "leapfrog"), "precision": args.precision,
                       "reductions": "fp64",
                       "l2": "inputs larger than L2 (state %.2f GB)"
                             % (state_bytes / 1e9),
                       "parallelism": "replicas" if world > 1 else "1 gpu"},
            "roofline": roof,
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "gauss_after": {"max": gauss[0], "rms": gauss[1],
                            "rho_max": gauss[2]},
        }
        line.update(extras)
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(cfg)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_extras(G, torch, cfg, args, stream, value):
    """FP64 throughput, the FP32 energy-density error against the FP64 path
    (itself parity-checked against the oracle), and the end-to-end number
    through the C ABI from host buffers."""
    out = {}
    # end to end: host rho -> init -> the workload's steps (its own length,
    # up to 400, whatever a smaller --steps is, so that the initial state is
    # amortised as in a real run) -> T^{mu nu} table to host
    p = cfg
    rho = gi.mv_rho(p["seed"], p["nc"], p["nx"], p["ny"], p["g2mu"])
    rho_t = torch.from_numpy(rho).pin_memory()
    rho_pinned = rho_t.numpy()
    K = max(min(int(p["steps"]), 400), args.steps)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        h = G.glasma_init_mv(p, rho_pinned, stream=stream)
    G.glasma_step(h, K)
    tab, H = G.glasma_tmunu(h)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    G.glasma_free(h)
    V = p["nz"] * p["nx"] * p["ny"]
    out["e2e"] = {"value": V * K / (t1 - t0), "unit": METRIC,
                  "h2d_bytes_per_step": rho.nbytes / K,
                  "d2h_bytes_per_step": tab.nbytes / K,
                  "what": "glasma_init_mv from host rho + %d steps + "
                          "glasma_tmunu to host, wall clock" % K}
    # sampling cost, timed apart from the steps: one T^{mu nu}(z) table of
    # the state (FP64 sums) written to device memory
    with torch.cuda.stream(stream):
        hs = G.glasma_init_mv(p, rho_pinned, stream=stream)
        tab_dev = torch.empty((p["nz"], 4), dtype=torch.float64, device="cuda")
    G.glasma_step(hs, 3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(20):
        G.glasma_tmunu_device(hs, tab_dev.data_ptr())
    e1.record(stream)
    torch.cuda.synchronize()
    out["tmunu_sample"] = {"ms": e0.elapsed_time(e1) / 20,
                           "what": "one T^{mu nu}(z) sample of the state (k_tmunu, "
                                   "FP64 sums, device output), timed apart from the steps"}
    G.glasma_free(hs)
    # FP64 comparison run (same event) and energy-density error over the
    # workload's full step count, whatever --steps is (outside the timed
    # region)
    other = "fp64" if args.precision == "fp32" else "fp32"
    k64 = int(p["steps"])
    res = {}
    for prec in (args.precision, other):
        c = dict(p, precision=prec)
        with torch.cuda.stream(stream):
            hh = G.glasma_init_mv(c, rho_pinned, stream=stream)
        tabs = []
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        tot = 0.0
        for blk in range(k64 // 50 + (1 if k64 % 50 else 0)):
            n = min(50, k64 - 50 * blk)
            ev0.record(stream)
            G.glasma_step(hh, n)
            ev1.record(stream)
            torch.cuda.synchronize()
            tot += ev0.elapsed_time(ev1)
            tabs.append(G.glasma_tmunu(hh)[0][:, 0])
        res[prec] = (V * k64 / (tot * 1e-3), np.array(tabs))
        G.glasma_free(hh)
    e32 = res["fp32"][1]
    e64 = res["fp64"][1]
    err = float(np.max(np.abs(e32 - e64)) / np.max(np.abs(e64)))
    out["fp64"] = {"value": res["fp64"][0], "unit": METRIC, "steps": k64}
    out["fp32_over_fp64"] = res["fp32"][0] / res["fp64"][0]
    out["eps_error_fp32_vs_fp64"] = {
        "max_rel": err, "definition":
            "max over z and sampled t (every 50 steps) of |eps32 - eps64| / "
            "max eps64; FP64 path parity-checked against the oracle"}
    out["su2_fp32"] = run_su2(G, torch, stream)
    out["improved"] = run_improved(G, torch, stream)
    out["improved"]["fp32_error"] = run_improved_error(G, torch)
    out["ensemble"] = run_ensemble(G, torch, stream)
    out["slab"] = run_slab(G, torch, stream, cfg)
    out["observables"] = run_observables(G, torch, stream)
    out["adjoint"] = run_adjoint(G, torch)
    return out


def run_su2(G, torch, stream, steps=100, warm=5):
    """The same leapfrog kernel for SU(2) in FP32 on a 1024 x 128^2 event
    (2.8 GB of state per step): 168 compulsory bytes per site, a quarter of
    SU(3)'s, with far less arithmetic, reported next to the SU(3) figure to
    show the kernel where its arithmetic per byte is low."""
    cfg = dict(gi.CONFIGS["su2_1024x128x128"])
    V = cfg["nz"] * cfg["nx"] * cfg["ny"]
    with torch.cuda.stream(stream):
        h = G.glasma_init_mv(cfg, None, stream=stream)
    G.glasma_step(h, warm)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    G.glasma_step(h, steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = G.glasma_get_info(h).kernel_launches
    G.glasma_free(h)
    per_launch = ms / launches
    alg = V * bytes_per_site(2, 4)
    peak, kind = load_peaks()
    gbs = alg / (per_launch * 1e-3) / 1e9
    return {"workload": "su2_1024x128x128", "value": V * steps / (ms * 1e-3),
            "unit": METRIC, "ms_per_step": ms / steps, "steps_timed": steps,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak,
                         "unit": "GB/s", "frac": gbs / peak, "peak_source": kind,
                         "alg_bytes_per_launch": alg,
                         "note": "compulsory bytes only (the charge windows of "
                                 "hop steps are left out)"}}


def run_adjoint(G, torch, probes=4, h=1e-4):
    """The differentiated workload (SU(2) 256 x 32^2, 200 steps, FP64): one
    gradient of the mid-rapidity energy (|z - z_c| < 16a) w.r.t. the MV
    charges through the hand-written adjoint (checkpoint every 20 steps),
    timed against the forward alone, and its agreement with central
    differences at a few random entries."""
    cfg = dict(gi.CONFIGS["su2_256x32x32"], precision="fp64")
    n, hw = cfg["steps"], 16.0
    rho = gi.mv_rho(cfg["seed"], 2, cfg["nx"], cfg["ny"], cfg["g2mu"])
    G.glasma_adjoint_energy(cfg, rho, 2, hw)            # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    val, _ = G.glasma_adjoint_energy(cfg, rho, n, hw, grad=False)
    t1 = time.perf_counter()
    val2, g = G.glasma_adjoint_energy(cfg, rho, n, hw, checkpoint_every=20)
    t2 = time.perf_counter()
    rng = np.random.default_rng(1404)
    errs = []
    for _ in range(probes):
        idx = tuple(int(rng.integers(0, s)) for s in rho.shape)
        rp, rm = rho.copy(), rho.copy()
        rp[idx] += h
        rm[idx] -= h
        fd = (G.glasma_adjoint_energy(cfg, rp, n, hw, grad=False)[0]
              - G.glasma_adjoint_energy(cfg, rm, n, hw, grad=False)[0]) / (2 * h)
        errs.append(abs(g[idx] - fd) / abs(fd))
    # the workload's own precision: FP32 forward and checkpoints, FP64 reverse
    cfg32 = dict(gi.CONFIGS["su2_256x32x32"], precision="fp32")
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    v32, g32 = G.glasma_adjoint_energy(cfg32, rho, n, hw, checkpoint_every=20)
    t4 = time.perf_counter()
    return {"workload": "su2_256x32x32, 200 steps, |z - z_c| < 16",
            "observable": val, "forward_s": t1 - t0, "forward_and_gradient_s": t2 - t1,
            "gradient_over_forward": (t2 - t1) / (t1 - t0), "checkpoint_every": 20,
            "fd_probes": probes, "fd_h": h, "fd_max_rel_err": max(errs),
            "fp32_forward": {"forward_and_gradient_s": t4 - t3,
                             "observable_rel_diff": abs(v32 - val) / abs(val),
                             "grad_max_rel_diff_vs_fp64": float(np.max(np.abs(g32 - g)) / np.max(np.abs(g)))},
            "note": "wall clock through the C ABI from host rho; the 64-entry "
                    "check is tests/test_gpu_adjoint.py"}


def run_observables(G, torch, stream, ms=(0.1, 0.2, 0.4), events=8, every=8,
                    taus=(12.0, 16.0, 20.0), eta_max=1.2):
    """The Sec. 4 analysis chain in the regime of the paper's rapidity-
    profile study (glasma_inputs.thin_ensemble_configs: SU(2), sigma_L =
    a_T, g^2 mu a_T = 0.4, a_z = a_T/8).  For each IR regulator m, `events`
    events run through the collision as one batch and T^{mu nu}(z) of every
    event is sampled on the device every `every` steps; then the event
    mean, the local rest frame, eps_loc(tau, eta_s) on hyperbolae of
    constant tau, the Gaussian width sigma_eta (Fig. 4 quotes widths that
    shrink as m grows) and the free-streaming check tau eps_loc = const at
    eta_s = 0 (Eq. late_time_energy).  The <p_T>(t, z) map of Fig. 5 is
    sampled for the smallest m.  The points of the hyperbolae stay at
    t - z = tau exp(-|eta_s|) >= 3.6 a_T behind the receding nuclei, whose
    charge ends 4 sigma_L = 4 a_T behind their centres."""
    res = {"workload": "su2_768x64x64_thin: a_z = a_T/8, dt = a_z/2, sigma_L = a_T, g2mu = 0.4",
           "events_per_m": events, "every_steps": every, "taus": list(taus),
           "eta_range": [-eta_max, eta_max], "by_m": {}}
    analysis_ms = 0.0
    for m in ms:
        cfgs = gi.thin_ensemble_configs(m, events)
        c0 = cfgs[0]
        nz, dt, az = c0["nz"], c0["dt"], c0["a_z"]
        n_s = c0["steps"] // every + 1
        hs = []
        with torch.cuda.stream(stream):
            for c in cfgs:
                hs.append(G.glasma_init_mv(c, None, stream=stream))
            tabs = torch.zeros((len(cfgs), n_s, nz, 4), dtype=torch.float64,
                               device="cuda")
        b = G.glasma_batch_create(hs)
        for k in range(n_s):
            if k:
                G.glasma_batch_step(b, every)
            for e, h in enumerate(hs):
                G.glasma_tmunu_device(h, tabs[e, k].data_ptr())
        torch.cuda.synchronize()
        b.close()
        for h in hs:
            G.glasma_free(h)
        # collision origin: the nuclei start at z_c -/+ d and meet at t = d
        d = (math.ceil(4 * c0["sigma_l"] / az) + 2) * az
        t0, dts, z0 = -d, every * dt, -nz * az / 2.0
        with torch.cuda.stream(stream):
            rest = torch.empty((n_s * nz, 8), dtype=torch.float64, device="cuda")
            eta = torch.linspace(-eta_max, eta_max, 25, dtype=torch.float64,
                                 device="cuda")
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            G.glasma_rest_frame(tabs.data_ptr(), len(cfgs), n_s * nz,
                                rest.data_ptr(), stream)
            prof = {}
            for tau in taus:
                tt = torch.full_like(eta, tau)
                out = torch.empty_like(eta)
                G.glasma_sample_grid(rest.data_ptr(), n_s, nz, 8, 4, t0, dts, z0,
                                     az, tt.data_ptr(), eta.data_ptr(),
                                     eta.numel(), out.data_ptr(), coords="milne",
                                     stream=stream)
                prof[tau] = (out, tt)      # tt kept alive until the kernel ran
            ev1.record(stream)
            torch.cuda.synchronize()
        analysis_ms += ev0.elapsed_time(ev1)
        eta_h = eta.cpu().numpy()
        mid = len(eta_h) // 2
        r = {"valid_fraction": float(rest[:, 7].mean().item()), "sigma_eta": {},
             "mu_eta": {}}
        for tau in taus:
            f = prof[tau][0].cpu().numpy()
            try:
                _, mu, sig = G.glasma_fit_gaussian(eta_h, f, 0.1)
                r["sigma_eta"][str(tau)] = sig
                r["mu_eta"][str(tau)] = mu
            except G.GlasmaError as ex:
                r["sigma_eta"][str(tau)] = None
                r["fit_error"] = str(ex)
        last = prof[taus[-1]][0].cpu().numpy()
        r["eps_loc_tau%g" % taus[-1]] = [float("%.4g" % v) for v in last[::3]]
        r["eta"] = [float("%.3g" % v) for v in eta_h[::3]]
        te = [tau * float(prof[tau][0][mid].item()) for tau in taus]
        r["tau_eps_loc_eta0"] = dict(zip([str(t) for t in taus], te))
        r["free_streaming_spread"] = (max(te) - min(te)) / (sum(te) / len(te))
        if m == ms[0]:
            # <p_T>(t, z) / <p_T>(0, 0) (the Fig. 5 map) at a few (t, z) points
            tl = [0.0, 2.0, 2.0, 4.0, 4.0, 8.0, 8.0, 16.0, 16.0]
            zl = [0.0, 0.0, 1.0, 0.0, 2.0, 0.0, 4.0, 0.0, 8.0]
            with torch.cuda.stream(stream):
                tt_lab = torch.tensor(tl, dtype=torch.float64, device="cuda")
                zz_lab = torch.tensor(zl, dtype=torch.float64, device="cuda")
                pt_lab = torch.empty_like(tt_lab)
                G.glasma_sample_grid(rest.data_ptr(), n_s, nz, 8, 2, t0, dts, z0,
                                     az, tt_lab.data_ptr(), zz_lab.data_ptr(),
                                     len(tl), pt_lab.data_ptr(), coords="lab",
                                     stream=stream)
                torch.cuda.synchronize()
            ptl = pt_lab.cpu().numpy()
            res["pT_map_over_pT00"] = {
                "m": m, "t": tl, "z": zl,
                "value": [float("%.4g" % (v / ptl[0])) for v in ptl]}
        res["by_m"][str(m)] = r
    res["analysis_ms"] = analysis_ms
    return res


def run_ensemble(G, torch, stream, steps=40, warm=3):
    """The 24-event ensemble (SU(3), 256 x {32^2, 48^2, 64^2}, FP32): the
    events stepped one after another with glasma_step against one batched
    launch per step (glasma_batch_step, block shape from glasma_batch_tune),
    both from the same states, plus the ensemble mean of eps(z) after the
    run (the event average of the energy density)."""
    cfgs = gi.ensemble_configs()
    sites = sum(c["nz"] * c["nx"] * c["ny"] for c in cfgs)
    hs = []
    with torch.cuda.stream(stream):
        for c in cfgs:
            hs.append(G.glasma_init_mv(c, None, stream=stream))
    b = G.glasma_batch_create(hs)
    G.glasma_batch_step(b, warm)
    bx, mode = G.glasma_batch_tune(b, 10)
    blobs = [G.glasma_get_state(h) for h in hs]
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for h in hs:
        G.glasma_step(h, steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_seq = ev0.elapsed_time(ev1)
    seq_tabs = [G.glasma_tmunu(h)[0] for h in hs]
    for h, blob in zip(hs, blobs):
        G.glasma_set_state(h, blob)
    torch.cuda.synchronize()
    ev0.record(stream)
    G.glasma_batch_step(b, steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms_bat = ev0.elapsed_time(ev1)
    tabs = [G.glasma_tmunu(h)[0] for h in hs]
    same = all(np.array_equal(x, y) for x, y in zip(tabs, seq_tabs))
    eps = np.array([t[:, 0] for t in tabs])
    mean = eps.mean(axis=0)
    zpk = int(np.argmax(mean))
    b.close()
    for h in hs:
        G.glasma_free(h)
    return {"workload": "su3_ensemble_24x256x{32,48,64}^2", "events": len(cfgs),
            "value": sites * steps / (ms_bat * 1e-3), "unit": METRIC,
            "sequential": sites * steps / (ms_seq * 1e-3),
            "batched_over_sequential": ms_seq / ms_bat,
            "block_sites": bx, "mode": mode,
            "steps_timed": steps,
            "batched_equals_sequential": bool(same),
            "eps_mean_peak": {"z": zpk, "value": float(mean[zpk]),
                              "event_std": float(eps[:, zpk].std(ddof=1))}}


def run_slab(G, torch, stream, cfg, nranks=(2, 4), steps=100, warm=5):
    """The z-slab decomposition (glasma_slab_*) of the benchmark event on
    one GPU: P slab contexts (paper_2009_02044_gb300.slab) exchange their
    halo slices by device copies before every step (LocalTransport: pack,
    copy into the neighbour's buffer, unpack), the data path a multi-GPU run
    sends over NCCL.  Reported per P: ms per step of all slabs with their
    exchange against the whole lattice, the exchange alone, the halo bytes
    per step, and whether the owned slices' T^{mu nu} rows and H equal the
    whole lattice's bit for bit after the run."""
    from paper_2009_02044_gb300 import slab as SL
    V = cfg["nz"] * cfg["nx"] * cfg["ny"]
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)

    def timed(fn):
        torch.cuda.synchronize()
        ev0.record(stream)
        fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1)

    with torch.cuda.stream(stream):
        whole = G.glasma_init_mv(cfg, None, stream=stream)
    G.glasma_step(whole, warm)
    ms_whole = timed(lambda: G.glasma_step(whole, steps))
    tab_w, H_w = G.glasma_tmunu(whole)
    G.glasma_free(whole)
    out = {"workload": "%s (%d slices)" % ("su3_512x64x64", cfg["nz"]),
           "steps_timed": steps, "whole_ms_per_step": ms_whole / steps,
           "by_ranks": {},
           "note": "one GPU; the exchange is device copies between slab "
                   "contexts, not NCCL; multi-GPU unmeasured on hardware"}
    for P in nranks:
        with torch.cuda.stream(stream):
            ranks = [SL.SlabRank(cfg, r, P, stream=stream) for r in range(P)]
            T = SL.LocalTransport(ranks)
            T.setup()

            def run_steps(n):
                for _ in range(n):
                    T.step()

            def run_exchanges(n):
                for _ in range(n):
                    T.exchange()

            run_steps(warm)
            ms = timed(lambda: run_steps(steps))
            ms_x = timed(lambda: run_exchanges(steps))
            T.exchange()
            rows = T.gather_rows()
        halo = sum(r.buf[("send", d)].numel() for r in ranks for d in (+1, -1)
                   if r.has(d))
        out["by_ranks"][str(P)] = {
            "ms_per_step": ms / steps, "exchange_ms_per_step": ms_x / steps,
            "over_whole": (ms / steps) / (ms_whole / steps),
            "value": V * steps / (ms * 1e-3), "unit": METRIC,
            "halo_bytes_per_step": halo,
            "equals_whole_lattice": bool(np.array_equal(rows, tab_w)
                                         and SL.total_energy(cfg, rows) == H_w)}
        for r in ranks:
            G.glasma_free(r.h)
    out["improved"] = run_slab_improved(G, torch, stream)
    return out


def run_slab_improved(G, torch, stream, nt=32, P=2, steps=10, warm=3):
    """The improved-scheme workload (SU(3), 2048 slices, a_z = dt = a_T/4,
    FP32), cut to nt x nt transversally, on P slabs of one GPU driven sweep
    by sweep (glasma_implicit_*: each sweep's maxima read back and folded
    across the slabs before the stopping rule) against the whole lattice's
    glasma_step (every sweep queued at once): ms per step, sweeps per step,
    and whether rows and H agree bit for bit."""
    from paper_2009_02044_gb300 import slab as SL
    cfg = dict(gi.CONFIGS["su3_2048x128x128_improved"], nx=nt, ny=nt, precision="fp32")
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        whole = G.glasma_init_mv(cfg, None, stream=stream)
        G.glasma_step(whole, warm)
        torch.cuda.synchronize()
        ev0.record(stream)
        its_w = []
        for _ in range(steps):
            G.glasma_step(whole, 1)
            its_w.append(G.glasma_get_info(whole).implicit_iters)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_w = ev0.elapsed_time(ev1)
        tab_w, H_w = G.glasma_tmunu(whole)
        G.glasma_free(whole)
        ranks = [SL.SlabRank(cfg, r, P, stream=stream) for r in range(P)]
        T = SL.LocalTransport(ranks)
        T.setup()
        for _ in range(warm):
            T.step()
        torch.cuda.synchronize()
        ev0.record(stream)
        its_s = [T.step() for _ in range(steps)]
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_s = ev0.elapsed_time(ev1)
        T.exchange()
        rows = T.gather_rows()
    for r in ranks:
        G.glasma_free(r.h)
    return {"workload": "su3_2048x128x128_improved cut to %dx%d, FP32" % (nt, nt),
            "slabs": P, "steps_timed": steps,
            "whole_ms_per_step": ms_w / steps, "slabs_ms_per_step": ms_s / steps,
            "over_whole": ms_s / ms_w,
            "sweeps_per_step": sum(its_s) / steps,
            "same_sweeps": its_s == its_w,
            "equals_whole_lattice": bool(np.array_equal(rows, tab_w)
                                         and SL.total_energy(cfg, rows) == H_w)}


def run_improved_error(G, torch, nt=16, steps=1000, every=50):
    """The FP32 energy-density error of the improved scheme against its FP64
    path (parity-checked against the oracle), over the workload's 1000
    steps, on a transverse cut of the 2048-slice lattice (the FP64 path at
    the full 128^2 would take about 20 GPU-minutes): e_eps = max over z and
    over the samples (every 50 steps) of |eps32 - eps64| / max eps64, with
    the energy and Gauss-residual histories.  Two readings of the workload:
    the primary a_z = dt = a_T/4 (dispersion-free along z) and the literal
    isotropic a_z = a_T, dt = a_T/4."""
    res = {}
    for name, upd in (("primary_az_dt_0.25", {}), ("isotropic_az_1_dt_0.25", dict(a_z=1.0, dt=0.25))):
        runs = {}
        for prec in ("fp32", "fp64"):
            cfg = dict(gi.CONFIGS["su3_2048x128x128_improved"], nx=nt, ny=nt,
                       precision=prec, **upd)
            h = G.glasma_init_mv(cfg, None)
            tab, H0 = G.glasma_tmunu(h)
            eps, Hs, gs = [tab[:, 0].copy()], [H0], []
            for _ in range(steps // every):
                G.glasma_step(h, every)
                tab, H = G.glasma_tmunu(h)
                eps.append(tab[:, 0].copy())
                Hs.append(H)
                g = G.glasma_gauss_residual(h)
                gs.append(g[0] / g[2])
            G.glasma_free(h)
            runs[prec] = (np.array(eps), np.array(Hs), gs)
        e32, e64 = runs["fp32"][0], runs["fp64"][0]
        per = np.max(np.abs(e32 - e64), axis=1) / np.max(np.abs(e64), axis=1)
        res[name] = {
            "lattice": [cfg["nz"], nt, nt], "steps": steps,
            "e_eps": float(np.max(np.abs(e32 - e64)) / np.max(np.abs(e64))),
            "e_eps_at_step": {str(every * k): float("%.3g" % v) for k, v in enumerate(per)
                              if k in (1, 2, 4, 10, 20)},
            "energy_change_fp32": float(runs["fp32"][1][-1] / runs["fp32"][1][0] - 1),
            "energy_change_fp64": float(runs["fp64"][1][-1] / runs["fp64"][1][0] - 1),
            "gauss_rel_final_fp32": float(runs["fp32"][2][-1]),
            "gauss_rel_final_fp64": float(runs["fp64"][2][-1])}
    res["definition"] = ("max over z and over samples every 50 steps of |eps32(z,t) - eps64(z,t)| "
                         "/ max_z eps64(z,t); FP64 path parity-checked against the oracle")
    res["note"] = ("at dt = a_z every mode with k_z = pi / a_z has sin^2(w dt / 2) = 1, a double "
                   "root: FP32 rounding of the force and links forces that family and its "
                   "amplitude grows like (steps)^2 u, so e_eps exceeds 1e-5 after about 50 steps; "
                   "a second FP32 word for E changed nothing (measured), the isotropic reading has "
                   "no such family")
    return res


def run_improved(G, torch, stream, steps=20, warm=480):
    """The thin-nucleus workload with the semi-implicit scheme: SU(3)
    2048 x 128^2, a_z = dt = a_T/4, sigma_L = 2 a_T, FP32 state.  Times
    `steps` steps after `warm` untimed steps, a bounded sample from the
    middle of the 1000-step run (the nuclei have met, and the iteration
    needs more sweeps than before the collision), and reports the
    iterations per step, the bandwidth of the iteration kernel and the
    energy and Gauss-law behaviour."""
    cfg = dict(gi.CONFIGS["su3_2048x128x128_improved"], implicit_tol=1e-9,
               implicit_max_iter=40)
    V = cfg["nz"] * cfg["nx"] * cfg["ny"]
    with torch.cuda.stream(stream):
        h = G.glasma_init_mv(cfg, None, stream=stream)
    G.glasma_step(h, warm)
    H0 = G.glasma_tmunu(h)[1]
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    iters = []
    total = 0.0
    for _ in range(steps):
        ev0.record(stream)
        G.glasma_step(h, 1)
        ev1.record(stream)
        torch.cuda.synchronize()
        total += ev0.elapsed_time(ev1)
        iters.append(G.glasma_get_info(h).implicit_iters)
    H1 = G.glasma_tmunu(h)[1]
    g = G.glasma_gauss_residual(h)
    G.glasma_free(h)
    # per sweep: read U(n) and the iterate, the work field (E(n-1/2) + dt J
    # + the fixed-slot force) and E; write E and the next iterate
    # (FP32 SU(3): 2*216 + 3*96 + 216 bytes per site); U(n-1) is read once
    # per step by the prepare kernel
    sweep_bytes = V * (2 * 216 + 3 * 96 + 216)
    n_sweeps = sum(iters)
    peak, kind = load_peaks()
    gbs = sweep_bytes * n_sweeps / (total * 1e-3) / 1e9
    return {"workload": "su3_2048x128x128_improved", "value": V * steps / (total * 1e-3),
            "unit": METRIC, "steps_timed": steps, "ms_per_step": total / steps,
            "iterations_per_step": iters,
            "sweep_roofline": {"bound": "hbm", "achieved": gbs, "peak": peak,
                               "unit": "GB/s", "frac": gbs / peak,
                               "peak_source": kind,
                               "note": "includes the prep and skipped launches"},
            "energy_rel_change": (H1 - H0) / H0,
            "gauss_rel": g[0] / g[2]}


def main():
    args = parse()
    cfg = dict(gi.CONFIGS[args.workload])
    if args.nz:
        cfg["nz"] = args.nz
    if args.impl == "reference":
        run_reference(args, cfg)
    else:
        run_ours(args, cfg)


if __name__ == "__main__":
    main()
