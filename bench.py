"""Throughput of the order-5 anelastic clustered-LTS ADER-DG update on one GB300.

Workload: 96 x 96 x 38 hexes x 6 = 2,101,248 jittered graded tetrahedra (h = 250 m,
z spacing 125 -> 500 m), 8 random layers vs ~ U[500, 4000] m/s (vp = sqrt(3) vs,
rho = 2700, Qs = 50 vs[km/s], Qp = 2 Qs), 3 relaxation mechanisms over 0.1-5 Hz, order
5, 5 LTS clusters with the lambda search, CFL 0.5, a moment-tensor Ricker source and
64 surface receivers. One step = one macro step (16 finest steps: every cluster
completes its 2^(4-l) steps). The metric is element updates per second.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--fused F runs the fused-simulation workload instead: 64 x 64 x 40 hexes x 6 = 983,040
tetrahedra of the same generator, F simulations (a multiple of 4), each driven by its own
moment-tensor Ricker source (seeded random positions and orientations, f0 in [1, 4] Hz);
the metric is then simulation element updates per second.

--impl reference times the FP64 CPU oracle (the only reference there is) on the machine's
host cores on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "element-updates/s and % HBM roofline, order-5 anelastic LTS, 1 GB300 (vs plain FP32)"
UNIT = "element-updates/s"
ORDER, NMECH, NCLUSTERS, CFL = 5, 3, 5, 0.5
FULL = dict(nx=96, ny=96, nz=38, h=250.0, hz=125.0)
FUSED_FULL = dict(nx=64, ny=64, nz=40, h=250.0, hz=125.0)
# elastic order-5 workload: 64 x 64 x 32 hexes x 6 = 786,432 tets, three layers by depth
ELASTIC_FULL = dict(nx=64, ny=64, nz=32, h=250.0, hz=125.0)
ELASTIC_ORDER, ELASTIC_CLUSTERS = 5, 4


def make_elastic_workload(nx, ny, nz, h, hz):
    """Layers 0-1 km vs 1000, 1-3 km vs 2000, below vs 3500 m/s (vp = sqrt(3) vs, rho 2700),
    a 2 Hz Ricker moment-tensor source at the centre 2 km deep (t0 = 1.2 / f0), 64 surface
    receivers."""
    from paper_2202_10313_gb300 import synth
    mesh = synth.graded_box(nx, ny, nz, h, hz)
    mat = synth.layered(mesh, [1000.0, 3000.0], [1000.0, 2000.0, 3500.0])
    lx, ly, depth = nx * h, ny * h, mesh["depth"]
    src = dict(x=np.array([0.5 * lx + 17.0, 0.5 * ly - 23.0, -2000.0 if depth > 2500 else -0.4 * depth]),
               m6=np.array([0.0, 0.0, 0.0, 1.0, 0.0, 0.0]), f0=2.0, t0=0.6, m0=1e15)
    recs = synth.surface_receiver_grid(8, 8, (0.0, lx), (0.0, ly), depth=1.0)
    return mesh, mat, src, recs
SAMPLE = dict(nx=12, ny=12, nz=5, h=250.0, hz=125.0)   # bounded CPU sample of the same generator


def make_workload(nx, ny, nz, h, hz):
    from paper_2202_10313_gb300 import synth
    mesh = synth.graded_box(nx, ny, nz, h, hz)
    mat = synth.random_layers(mesh)
    lx, ly, depth = nx * h, ny * h, mesh["depth"]
    src = dict(x=np.array([0.5 * lx + 17.0, 0.5 * ly - 23.0, -2000.0 if depth > 2500 else -0.4 * depth]),
               m6=np.array([0.0, 0.0, 0.0, 1.0, 0.0, 0.0]), f0=2.0, t0=0.6, m0=1e15)
    recs = synth.surface_receiver_grid(8, 8, (0.0, lx), (0.0, ly), depth=1.0)
    return mesh, mat, src, recs


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6778.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region (read from a pipe)."""

    def __init__(self, index):
        self.proc = None
        self.index = index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (out or "").splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_hash():
    """Hash of the forward kernels' source without its // comments (the DRAM counters in
    profiles/traffic.json are valid only for the code they were taken on; a comment edit does
    not change the code)."""
    import re
    h = hashlib.sha256()
    for f in ("kernels.cuh", "kernels_sp.cuh", "gen_sparse.cpp"):
        src = open(os.path.join(ROOT, "paper_2202_10313_gb300", "csrc", f), encoding="utf-8").read()
        code = "\n".join(l.rstrip() for l in re.sub(r"//[^\n]*", "", src).split("\n") if l.strip())
        h.update(code.encode("utf-8"))
    return h.hexdigest()[:16]


def oracle_sample(seconds_cap=25.0, steps=None):
    """Element updates/s of the FP64 oracle on the bounded sample (one macro step each)."""
    import oracle  # noqa: F401  (test infrastructure: only this leg and --impl reference use it)
    from oracle.mesh import Mesh
    from oracle.scheme import Solver as Oracle
    mesh, mat, src, recs = make_workload(**SAMPLE)
    om = Mesh(mesh["xyz"], mesh["tet"], mesh["face_bc"])
    o = Oracle(ORDER, NMECH, om, mat["rho"], mat["vp"], mat["vs"], mat["qp"], mat["qs"])
    o.setup_clusters(NCLUSTERS, CFL)
    o.add_point_source(src["x"], src["m6"], src["f0"], src["t0"], src["m0"])
    period = 2 ** (NCLUSTERS - 1)
    per_macro = o.element_updates(period)
    times, cpu = [], []
    t_all = time.time()
    n = steps if steps is not None else 10 ** 9
    for _ in range(n):
        t0, c0 = time.perf_counter(), time.process_time()
        o.run_lts(period)
        times.append(time.perf_counter() - t0)
        cpu.append(time.process_time() - c0)
        if steps is None and time.time() - t_all > seconds_cap:
            break
    return per_macro, times, om.K, cpu


def _oracle_worker(args):
    """One independent oracle run of the bounded sample in a spawned process (one BLAS
    thread): returns the updates per macro step and the timed steps' durations."""
    warmup, steps = args
    per_macro, times, _, _ = oracle_sample(steps=warmup + steps)
    return per_macro, times[warmup:]


def oracle_all_cores(warmup, steps, procs=None):
    """The oracle on every host core: `procs` independent runs of the bounded sample in
    spawned processes, one per core (the elements of a phase are independent, so this is
    what a split of the phases over the cores would reach without its communication).
    Throughput = all processes' timed updates / the longest process's timed wall time."""
    import multiprocessing as mp
    procs = procs or os.cpu_count() or 1
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(_oracle_worker, [(warmup, steps)] * procs)
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    wall = max(sum(t) for _, t in res)
    updates = sum(pm * len(t) for pm, t in res)
    return updates / wall, procs


def threads_used(times, cpu):
    """Cores the oracle actually kept busy: process CPU time over wall time of the timed
    steps (the oracle's small products leave most of a BLAS thread pool idle)."""
    wall = sum(times)
    ratio = sum(cpu) / wall if wall > 0 else 1.0
    return max(1, int(round(ratio))), ratio


def run_reference(args, rank, world):
    if rank != 0:
        return
    per_macro, times, K, cpu = oracle_sample(steps=args.warmup + args.steps)
    timed = times[args.warmup:]
    cores, busy = threads_used(timed, cpu[args.warmup:])
    total = sum(timed)
    single = per_macro * len(timed) / total
    # every host core: independent sample runs, one per core, same step count
    value, procs = oracle_all_cores(args.warmup, args.steps)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / len(timed),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "anelastic O5 m3 LTS Nc=5, bounded sample %d tets of the same generator" % K,
                   "elements": K, "order": ORDER, "n_mech": NMECH, "clusters": NCLUSTERS},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "host_cores": os.cpu_count(), "kind": "oracle",
                         "single_core": {"value": single, "cores": cores, "cpu_time_over_wall": busy},
                         "sample": "%d-tet mesh (12x12x5 hexes) of the same generator, one macro step per step; "
                                   "value: %d independent runs in %d spawned processes (one per host core), all "
                                   "timed updates over the longest run's wall time" % (K, procs, procs)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2202_10313_gb300 import binding, build, perfmodel, synth
    torch.cuda.set_device(local_rank)
    build.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    F = max(1, args.fused)
    order, nmech, nclusters = (ELASTIC_ORDER, 0, ELASTIC_CLUSTERS) if args.elastic else (ORDER, NMECH, NCLUSTERS)
    cfg = ELASTIC_FULL if args.elastic else (FUSED_FULL if F > 1 else FULL)
    if args.small:
        cfg = dict(nx=24, ny=24, nz=10, h=250.0, hz=125.0)
    elif args.medium:
        cfg = dict(nx=48, ny=48, nz=19, h=250.0, hz=125.0)
    mesh, mat, src, recs = (make_elastic_workload if args.elastic else make_workload)(**cfg)
    K = mesh["tet"].shape[0]
    s = binding.Solver(order, nmech, device=local_rank, n_fused=F)
    s.set_mesh(mesh["xyz"], mesh["tet"], mesh["face_bc"])
    s.set_material(mat["rho"], mat["vp"], mat["vs"], mat.get("qp"), mat.get("qs"), 0.1, 5.0)
    if F == 1:
        s.add_point_source(src["x"], src["m6"], src["f0"], src["t0"], src["m0"])
    else:
        lx, ly, depth = cfg["nx"] * cfg["h"], cfg["ny"] * cfg["h"], mesh["depth"]
        pos, m6s, f0s = synth.random_sources(F, [0.1 * lx, 0.1 * ly, -0.6 * depth], [0.9 * lx, 0.9 * ly, -0.05 * depth],
                                             f0_range=(1.0, 4.0), seed=7)
        for f in range(F):
            s.add_point_source(pos[f], m6s[f], f0s[f], 1.2 / f0s[f], src["m0"], fused_idx=f)
    dt_rec = 0.01
    for r in recs:
        s.add_receiver(r, dt_rec)
    if args.partition <= 1:
        s.use_torch_memory(nclusters)
    if args.contraction != "auto":
        s.set_contraction(args.contraction)
        s.set_tile(args.tile)
    _, lam, speedup = s.setup_clusters(nclusters, CFL)
    pstats = None
    if args.partition > 1:
        part, pstats = s.partition(args.partition)
        s.set_partition(part, args.partition)
    tuned = None
    if args.contraction == "auto":
        tuned = s.autotune(allow_tf32=False, stream=torch.cuda.current_stream())
    info = s.info()
    period = 2 ** (nclusters - 1)
    per_macro = int(info["updates_per_macro"].sum()) * F      # simulation element updates
    stream = torch.cuda.current_stream()
    # warm-up
    s.advance_steps(period * args.warmup, stream)
    torch.cuda.synchronize()
    # timed region: device-resident state
    clocks = ClockSampler(local_rank)
    s.set_profiling(True)
    launches0 = s.info()["launches"]
    xb0 = s.exchange_bytes()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        s.advance_steps(period, stream)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    launches = s.info()["launches"] - launches0
    xbytes = (s.exchange_bytes() - xb0) / args.steps
    kst = s.kernel_stats()
    s.set_profiling(False)
    # end to end through the public API: advance + seismogram read-back every step
    h2d0, d2h0 = s.transfer_bytes()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        s.advance(s.info()["time"] + period * info["finest_dt"] * (1 + 1e-6), stream)
        for rid in range(len(recs)):
            for f in range(F):
                s.seismogram(rid, f)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    h2d1, d2h1 = s.transfer_bytes()
    ms_t = torch.tensor([ms, e2e_s * 1000.0], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
    ms, e2e_ms = float(ms_t[0]), float(ms_t[1])
    if rank != 0:
        return
    # FP32 and tf32 throughput probes of this GPU (after the timed region)
    try:
        pk = s.measure_peaks()
    except Exception as exc:   # reported, not fatal: the derived peak stays the denominator
        pk = {"error": str(exc)}
    total_updates = per_macro * args.steps * world
    value = total_updates / (ms / 1000.0)
    hbm_gbs, sm_max, peak_src = peaks()
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12     # TFLOP/s at the maximum SM clock
    # dominant kernel by device time
    kind = int(np.argmax(kst["ms"]))
    engine = tuned["contraction"] if tuned else args.contraction
    predict_name = "k_predict_sp" if engine == "sparse" else ("k_predict_tc" if engine.startswith("tf32")
                                                               else "k_predict_local")
    name = [predict_name, "k_neighbour_sp" if (engine == "sparse" and args.partition <= 1) else "k_neighbour"][kind]
    avg_ms = kst["ms"][kind] / max(kst["launches"][kind], 1)
    elems_per_launch = kst["elems"][kind] * F / max(kst["launches"][kind], 1)    # simulation elements
    # flops the dominant kernel's formulation needs per element: the sparse engine multiplies
    # only the operators' nonzero entries (its count is lower than the block count of the
    # dense kernels, given beside it)
    fl_block = perfmodel.flops_predict(order, nmech) if kind == 0 else perfmodel.flops_neighbour(order, nmech)
    fl = fl_block
    if engine == "sparse" and F == 1:
        fl = perfmodel.flops_predict_sparse(order, nmech) if kind == 0 else perfmodel.flops_neighbour_sparse(order, nmech)
    by = (perfmodel.bytes_predict(order, nmech, n_fused=F) if kind == 0
          else perfmodel.bytes_neighbour(order, nmech, n_fused=F))
    achieved_tf = fl * elems_per_launch / (avg_ms / 1000.0) / 1e12
    achieved_gbs = by * elems_per_launch / (avg_ms / 1000.0) / 1e9
    traffic = None
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tp):
        t = json.load(open(tp))
        ent = t.get(name)
        if F > 1:
            ent = t.get(name + "_fused%d" % F)
        # only for the kernel instantiation the counters were taken on
        if (ent and ent.get("kernel_hash") == kernel_hash() and ent.get("order") == order
                and ent.get("n_mech") == nmech):
            traffic = ent["dram_bytes_per_element"] * elems_per_launch
    metric, unit = METRIC, UNIT
    if args.elastic:
        metric = "element-updates/s, order-5 elastic LTS, 1 GB300"
    srcs = "1 moment-tensor source"
    if F > 1:
        metric = "simulation element-updates/s, order-5 anelastic LTS, %d fused sources, 1 GB300" % F
        unit = "sim-element-updates/s"
        srcs = "%d fused simulations, one random moment-tensor source each" % F
    dof_bytes = K * (9 + 6 * nmech) * perfmodel.nbasis(order) * 4 * F
    line = {
        "metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "contraction": tuned["contraction"] if tuned else args.contraction, "autotune": tuned,
        "config": {"workload": ("elastic O5" if args.elastic else "anelastic O5 m3") +
                               " LTS, %d jittered graded tets, Nc=%d, lambda=%.2f, CFL %.1f, "
                               "%s, 64 receivers; step = 1 macro step (%d finest steps)"
                               % (K, nclusters, lam, CFL, srcs, period),
                   "elements": K, "fused": F, "updates_per_step": per_macro,
                   "launch": dict(s.launch_config(), engine=engine, tile=(tuned["tile"] if tuned else args.tile)),
                   "cluster_elems": info["cluster_elems"].tolist(), "theoretical_lts_speedup": speedup,
                   "l2": ("inputs larger than L2 (DOFs %.1f GB)" if dof_bytes > 129e6 else
                          "inputs within L2 (DOFs %.2f GB): a quick-check size, not a timing case") % (dof_bytes / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "kernel": name, "achieved": achieved_tf, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved_tf / fp32_peak, "traffic": traffic,
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 x %.0f MHz (derived)" % sm_max,
                     "flops_per_element": fl, "elements_per_launch": elems_per_launch, "avg_launch_ms": avg_ms,
                     "flops_per_element_block": fl_block,
                     "frac_block": fl_block * elems_per_launch / (avg_ms / 1000.0) / 1e12 / fp32_peak,
                     # roofline time of one launch, max(bytes / HBM, flops / FP32 peak), over its duration
                     "roofline_time_attained": max(by * elems_per_launch / (hbm_gbs * 1e9),
                                                   fl * elems_per_launch / (fp32_peak * 1e12)) / (avg_ms / 1000.0),
                     "measured_peak": pk.get("fp32_tflops"),
                     "frac_of_measured": (achieved_tf / pk["fp32_tflops"]) if pk.get("fp32_tflops") else None},
        "peaks_measured": pk,
        "hbm": {"kernel": name, "achieved": achieved_gbs, "peak": hbm_gbs, "unit": "GB/s",
                "frac": achieved_gbs / hbm_gbs, "peak_source": peak_src, "bytes_per_element": by},
        "kernel_ms": {"k_predict_local": kst["ms"][0], "k_neighbour": kst["ms"][1],
                      "launches": kst["launches"].tolist(), "predict_kernel": predict_name},
        "gpu_launches": int(launches),
        "e2e": {"value": total_updates / (e2e_ms / 1000.0), "unit": unit,
                "h2d_bytes_per_step": (h2d1 - h2d0) / args.steps, "d2h_bytes_per_step": (d2h1 - d2h0) / args.steps},
        "clocks": ck,
    }
    if pstats is not None:
        B = order * (order + 1) * (order + 2) // 6
        line["partition"] = dict(parts=args.partition, face_local_bytes_per_step=xbytes,
                                 whole_buffer_bytes_per_step=pstats["buffer_msgs_per_macro"] * 9 * B * 4,
                                 **{k: v for k, v in pstats.items()})
    if not args.no_cpu_baseline and world == 1:
        per_m, times, Ks, cpu = oracle_sample(seconds_cap=12.0)
        v1 = per_m * len(times) / sum(times)
        cores, busy = threads_used(times, cpu)
        v, procs = oracle_all_cores(1, 3)
        line["cpu_baseline"] = {"value": v, "unit": unit, "cores": procs, "host_cores": os.cpu_count(),
                                "kind": "oracle",
                                "single_core": {"value": v1, "cores": cores, "cpu_time_over_wall": busy,
                                                "macro_steps": len(times)},
                                "sample": "a %d-tet mesh (12x12x5 hexes) of the same generator, one macro step per "
                                          "step; value: %d independent runs (1 untimed + 3 timed macro steps each) in "
                                          "%d spawned processes, one per host core, all timed updates over the "
                                          "longest run's wall time" % (Ks, procs, procs)}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--small", action="store_true", help="small mesh (quick check)")
    ap.add_argument("--medium", action="store_true", help="262k-tet mesh (profiling captures)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fused", type=int, default=1, help="fused simulations (multiple of 4; 1 = single)")
    ap.add_argument("--elastic", action="store_true",
                    help="elastic order-5 workload: 786,432 tets, 3 layers, 4 clusters (a parity config)")
    ap.add_argument("--partition", type=int, default=1,
                    help="emulated partitioned run: P weighted parts exchanging face-local messages")
    ap.add_argument("--tile", type=int, default=1, choices=[0, 1],
                    help="with an explicit --contraction sparse: the neighbour kernel's 8 (0) or 4 (1, the "
                         "library default) elements per CTA")
    ap.add_argument("--contraction", default="auto", choices=["auto", "fp32", "sparse", "tf32x3", "tf32"],
                    help="engine of the time/volume contractions: FP32 CUDA cores or tensor cores; auto runs "
                         "the autotuner over the FP32-accurate engines and the grid shapes")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
