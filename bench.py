"""Benchmark: H² matrix-vector product of the Galerkin single-layer matrix.

Workload (the paper's test surface, a polyhedral unit sphere): icosphere
level 7 (327,680 flat triangles = DoF), leaf size 32, eta = 2, tensor
Chebyshev order m = 4 (rank 64), coupling matrices stored, Sauter-Schwab
nearfield of order 3, a block of 16 seeded right-hand sides.  One step is one
product y = G~ x of the whole block (all phases: permute in, leaf forward,
upward transfer, coupling, downward transfer, leaf backward + nearfield,
permute out).  The solve leg times GMRES(30) to a relative residual of 1e-8
on the same matrix.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec f64|f32]
                    [--impl ours|reference] [--level L] [--no-solve]

Prints one JSON line.  With --impl reference the FP64 CPU oracle is timed
instead, on a bounded sample of the workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H2 matvec DoF/s & % HBM roofline; solves/s, p99 latency at 1e-8 residual"
UNIT = "DoF/s"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return {"hbm_gbs": float(p["hbm_gbs"]), "src": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "src": "fallback"}


# FP64 arithmetic peak: the nominal 1.25 TFLOP/s of the part (FP64 FMA pipe)
FP64_TFLOPS = 1.25
# FP32 non-tensor peak: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz
FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# double-float multiply-add = 12 FP32 instructions (TwoProduct with two cross
# terms, TwoSum, two adds, renormalisation), so its FP64-equivalent peak is
DD_TFLOPS = FP32_TFLOPS / 12


class Clocks:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
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

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = float(p[2])
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _algorithmic(stats, nrhs, esize):
    """Algorithmic bytes and flops of one product (full, not symmetry-halved representation)."""
    n, k, m = stats["n"], stats["rank"], stats["order"]
    nclu, nadm, nnear, ne = stats["clusters"], stats["adm_blocks"], stats["near_blocks"], stats["near_entries"]
    far_clusters = nclu - (2 ** stats["first_adm_level"] - 1)
    coupling_bytes = esize * (nadm * k * k + 2 * far_clusters * k * nrhs)
    coupling_flops = 2.0 * nadm * k * k * nrhs
    total_bytes = esize * (ne + n * k + (nclu - 1) * 3 * m * m + nadm * k * k + 4 * nclu * k * nrhs) \
        + 8 * 2 * n * nrhs
    total_flops = 2.0 * nrhs * (ne + 2 * n * k + nadm * k * k) + 2 * 2 * (nclu - 1) * 3 * m * k * nrhs
    return dict(coupling_bytes=coupling_bytes, coupling_flops=coupling_flops, total_bytes=total_bytes,
                total_flops=total_flops)


def run_ours(args):
    import torch
    import paper_2203_05665_gb300 as pkg
    from paper_2203_05665_gb300 import H2Matrix, colmajor, inputs

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    pkg.load()
    v, f = inputs.icosphere(args.level)
    n = f.shape[0]
    nrhs = args.nrhs
    x_np = inputs.uniform_rhs(n, nrhs, 1002)
    stream = torch.cuda.current_stream()
    t0 = time.time()
    h = H2Matrix(v, f, leaf_size=32, eta=2.0, order=args.order, prec=args.prec, device=local,
                 stream=stream.cuda_stream)
    build_s = time.time() - t0
    low = args.prec in ("f32", "bf16", "f16")
    dt = torch.float32 if low else torch.float64
    esize = 4 if low else 8
    x = colmajor(torch.from_numpy(x_np).to(device="cuda", dtype=dt))
    y = colmajor(torch.empty_like(x))

    for _ in range(args.warmup):
        h.matvec(x, y)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # timed region: K products, inputs resident (the stored representation,
    # > 10 GB in FP64, is far larger than the 126 MB L2)
    h.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            h.matvec(x, y)
        ev1.record(stream)
        barrier()
    ms_total = ev0.elapsed_time(ev1)
    phases, products = h.phase_times()
    h.profile(False)
    ms = ms_total / args.steps
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    launches = sum(v[1] for v in phases.values())

    st = h.stats
    alg = _algorithmic(st, nrhs, esize)
    peaks = _peaks()
    cpl_ms = phases["coupling"][0] / products
    if args.prec == "f64n":
        roof = {"bound": "alu", "achieved": alg["coupling_flops"] / (cpl_ms * 1e-3) / 1e12, "peak": FP64_TFLOPS,
                "unit": "TFLOP/s", "kernel": "k_blockrow (coupling, FP64 FMA pipe)"}
    elif args.prec == "f64" and st.get("tensor", 0):
        # tensor-core coupling: a stream of the stored slices; algorithmic bytes are
        # those of the FP64 coupling matrices (k^2 x 8 B per block) and coefficients
        # stored_stream_frac: the E4M3 digit planes of S alone (10 B per entry), the part
        # of the kernel's input that must come from DRAM on every product (the
        # coefficient tiles are read again by every block of their column and are
        # mostly L2 hits)
        roof = {"bound": "hbm", "achieved": alg["coupling_bytes"] / (cpl_ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "kernel": "k_coupling_tc (tcgen05 kind::f8f6f4, ten 5-bit E4M3 digits, exact FP32 sums)",
                "stored_bytes_per_entry": 10,
                "stored_stream_frac": (st["adm_blocks"] * 10 * st["rank"] ** 2 / (cpl_ms * 1e-3) / 1e9
                                       / peaks["hbm_gbs"])}
    elif args.prec == "f64":
        roof = {"bound": "alu", "achieved": alg["coupling_flops"] / (cpl_ms * 1e-3) / 1e12, "peak": DD_TFLOPS,
                "unit": "TFLOP/s", "kernel": "k_blockrow (coupling, double-float on the FP32 pipe)",
                "hbm_frac": alg["coupling_bytes"] / (cpl_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}
    elif args.prec in ("bf16", "f16"):
        # regenerated coupling: 2 k^2 nrhs multiply-adds plus one kernel evaluation
        # (about 10 FP32 instructions and one MUFU rsqrt) per entry of S
        k = st["rank"]
        flops = alg["coupling_flops"] + 10.0 * st["adm_blocks"] * k * k
        roof = {"bound": "alu", "achieved": flops / (cpl_ms * 1e-3) / 1e12, "peak": FP32_TFLOPS,
                "unit": "TFLOP/s", "kernel": "k_blockrow (coupling regenerated in FP32)"}
    else:
        roof = {"bound": "hbm", "achieved": alg["coupling_bytes"] / (cpl_ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "kernel": "k_blockrow (coupling, stored S stream)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # DRAM bytes (read + write) per coupling launch from the ncu capture of the
    # same kernel at level 5 (profiles/k_coupling_tc_icosphere_L5_m4_16rhs_f64.md,
    # profiles/k_blockrow_coupling_icosphere_L5_m4_16rhs_f64.md), scaled by
    # admissible blocks; None where no capture of the current kernel exists
    tc = args.prec == "f64" and st.get("tensor", 0)
    traffic_per_block = {"f64": 691.93e6 / 18876, "f64-tc": (794.690048e6 + 7.657472e6) / 18876}
    key = "f64-tc" if tc else args.prec
    roof["traffic"] = (traffic_per_block[key] * st["adm_blocks"]
                       if key in traffic_per_block and args.order == 4 and args.nrhs == 16 else None)
    roof["peak_source"] = {"f64n": "nominal FP64 rate",
                           "f64": (f"{peaks['src']} HBM copy bandwidth" if tc else
                                   "FP32 FMA rate (152 SMs x 128 lanes x 2.07 GHz) / 12 instructions per dd FMA"),
                           "f32": f"{peaks['src']} HBM copy bandwidth",
                           "bf16": "FP32 FMA rate (152 SMs x 128 lanes x 2 flop x 2.07 GHz)",
                           "f16": "FP32 FMA rate (152 SMs x 128 lanes x 2 flop x 2.07 GHz)"}[args.prec]
    roof["kernel_ms"] = cpl_ms
    roof["hbm_frac_whole_product"] = alg["total_bytes"] / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"]

    # end to end: host FP64 buffers through the C ABI, copies included.  A
    # stream of steps (h2_matvec_host_stream): every step copies its own input
    # block in and its result out, the copies of neighbouring steps overlapped
    # with each product; also the one-call form (h2_matvec_host) for reference
    xp = torch.from_numpy(np.asfortranarray(x_np)).pin_memory() if torch.cuda.is_available() else None
    xh = colmajor(xp)
    yh = colmajor(torch.empty_like(xp).pin_memory())
    for _ in range(2):
        h.matvec_host((xh, yh))
    e2e_times = []
    for _ in range(max(3, min(args.steps, 10))):
        t1 = time.perf_counter()
        h.matvec_host((xh, yh))
        e2e_times.append(time.perf_counter() - t1)
    e2e_single_s = statistics.median(e2e_times)
    ecount = max(4, min(args.steps, 12))
    xs = torch.empty((ecount, nrhs, n), dtype=torch.float64).pin_memory()
    ys = torch.empty((ecount, nrhs, n), dtype=torch.float64).pin_memory()
    xt = torch.from_numpy(np.ascontiguousarray(x_np.T))
    for i in range(ecount):
        xs[i] = xt
    h.matvec_host_stream(xs[:2], ys[:2])
    stream_runs = []
    for _ in range(3):
        t1 = time.perf_counter()
        h.matvec_host_stream(xs, ys)
        stream_runs.append((time.perf_counter() - t1) / ecount)
    e2e_s = statistics.median(stream_runs)
    e2e_equals_device = bool(torch.equal(ys[ecount - 1], y.t().cpu().to(torch.float64)))

    # the same product replayed from a CUDA graph: median of per-replay CUDA-event pairs
    g = h.graph(x, y)
    for _ in range(3):
        g.launch()
    torch.cuda.synchronize()
    gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(max(20, args.steps))]
    for a, b in gev:
        a.record(stream)
        g.launch()
        b.record(stream)
    torch.cuda.synchronize()
    gms = sorted(a.elapsed_time(b) for a, b in gev)
    graph = {"replays": len(gms), "median_ms": gms[len(gms) // 2], "min_ms": gms[0], "max_ms": gms[-1],
             "median_dof_per_s": n * nrhs / (gms[len(gms) // 2] * 1e-3)}
    g.close()

    # parity spot check of this very run against the stored oracle rows is
    # done by the tests; here only a sanity check that the output is finite
    finite = bool(torch.isfinite(y).all().item())

    solve = None
    if not args.no_solve and rank == 0:
        b = np.asfortranarray(x_np[:, :args.solve_nrhs])

        def timed(fn):
            lat, res = [], None
            for _ in range(args.solve_reps):
                t1 = time.perf_counter()
                res = fn()
                lat.append(time.perf_counter() - t1)
            lat_sorted = sorted(lat)
            z, it, rel, stt = res
            return {"solves_per_s": args.solve_nrhs / statistics.median(lat), "p50_s": statistics.median(lat),
                    "p99_s": lat_sorted[min(len(lat) - 1, int(0.99 * len(lat)))], "reps": len(lat),
                    "iters": [int(i) for i in it], "max_relres": float(max(rel)), "status": int(stt)}

        solve = {"rtol": 1e-8, "restart": 30, "nrhs": args.solve_nrhs,
                 "gmres": dict(timed(lambda: h.solve(b, rtol=1e-8, restart=30, maxit=5000)),
                               product=args.prec)}
        if args.prec in ("f64", "f64n"):
            lo = H2Matrix(v, f, leaf_size=32, eta=2.0, order=args.order, prec="f32", device=local,
                          stream=stream.cuda_stream)
            solve["gmres_ir"] = dict(timed(lambda: h.solve_ir(lo, b, rtol=1e-8, inner_rtol=1e-4, restart=30,
                                                              maxit_inner=5000, maxit_outer=50)),
                                     residual=args.prec, inner="f32 GMRES(30) to 1e-4")
            # the FP32 product of the same workload (FP64 vs FP32 on one matrix)
            xf = colmajor(x.float())
            yf = colmajor(torch.empty_like(xf))
            for _ in range(3):
                lo.matvec(xf, yf)
            lo.profile(True)
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for _ in range(10):
                lo.matvec(xf, yf)
            f1.record(stream)
            torch.cuda.synchronize()
            fph, fpr = lo.phase_times()
            lo.profile(False)
            fms = f0.elapsed_time(f1) / 10
            a32 = _algorithmic(lo.stats, nrhs, 4)
            fcpl = fph["coupling"][0] / fpr
            solve["fp32_product"] = {
                "ms": fms, "dof_per_s": n * nrhs / (fms * 1e-3),
                "rel_diff_vs_f64": float(torch.linalg.norm(yf.double() - y) / torch.linalg.norm(y)),
                "phases_ms": {k2: v2[0] / fpr for k2, v2 in fph.items()},
                "coupling_hbm_frac": a32["coupling_bytes"] / (fcpl * 1e-3) / 1e9 / peaks["hbm_gbs"],
                "kernel": ("k_coupling_tc (tcgen05 kind::f8f6f4, six 5-bit E4M3 digits, exact FP32 sums)"
                           if lo.stats.get("tensor", 0) else "k_blockrow (coupling, stored FP32 S)")}
            lo.close()

    small = None
    if rank == 0 and not args.no_small:
        small = run_small(args, local, stream)

    helm = None
    if rank == 0 and not args.no_helmholtz:
        helm = run_helmholtz(args, local, stream)

    gca = None
    if rank == 0 and not args.no_gca:
        gca = run_gca(args, local, stream)

    serve = None
    if rank == 0 and not args.no_serve:
        serve = run_serve(args, local, stream)

    mixed = None
    if rank == 0 and not args.no_mixed:
        mixed = run_mixed(args, local, stream)

    batch = None
    if not args.no_batch:
        batch = run_batch(args, local, stream, ws, rank)

    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(args)

    value = n * nrhs * ws / (ms * 1e-3)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"f64": "f32x2 (double-float) with exact e4m3 digit products on the tensor cores "
                                              "(FP64-accurate)", "f32": "f32",
                                       "f64n": "f64", "bf16": "bf16 storage, f32 arithmetic",
                                       "f16": "f16 storage, f32 arithmetic"}[args.prec], "data": "synthetic",
        "config": {"workload": f"icosphere L{args.level} ({n} triangles), m={args.order} (k={args.order ** 3}), "
                               f"leaf 32, eta 2, stored S, SS order 3, {nrhs} RHS",
                   "n": n, "nrhs": nrhs, "order": args.order, "leaf_size": 32, "eta": 2.0,
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "l2": "inputs larger than L2 (stored representation %.2f GB)" % (st["device_bytes"] / 1e9)},
        "roofline": roof,
        "phases_ms": {k: v[0] / products for k, v in phases.items()},
        "graph": graph,
        "gpu_launches": int(launches),
        "e2e": {"value": n * nrhs / e2e_s, "unit": UNIT, "api": "h2_matvec_host_stream", "steps": ecount,
                "equals_device_result": e2e_equals_device,
                "one_call_value": n * nrhs / e2e_single_s, "h2d_bytes_per_step": int(8 * n * nrhs),
                "d2h_bytes_per_step": int(8 * n * nrhs)},
        "clocks": clk.summary(),
        "build_s": build_s,
        "build_phases_ms": h.build_times(),
        "finite": finite,
        "solve": solve,
        "small": small,
        "helmholtz": helm,
        "gca": gca,
        "serve": serve,
        "mixed": mixed,
        "batch": batch,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(out))
    h.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


SERVE_GEOMS = {
    # name: (mesh factory, leaf)
    "icosphere L4": (lambda I: I.icosphere(4), 32),
    "icosphere L5": (lambda I: I.icosphere(5), 32),
    "icosphere L6": (lambda I: I.icosphere(6), 32),
    "icosphere L7": (lambda I: I.icosphere(7), 32),
    "icosphere L8": (lambda I: I.icosphere(8), 32),
    "ellipsoid L6 (1.5,1,0.7)": (lambda I: I.ellipsoid(6, (1.5, 1.0, 0.7)), 32),
    "ellipsoid L7 (2,1,0.5)": (lambda I: I.ellipsoid(7, (2.0, 1.0, 0.5)), 32),
    "cube s=100": (lambda I: I.cube(100), 32),
}
SERVE_SMALL = ["icosphere L4", "icosphere L5", "icosphere L6", "ellipsoid L6 (1.5,1,0.7)"]


def _serve_stream(srv, geoms, nreq, rate, seed):
    """Submit a seeded Poisson stream (mean rate requests/s; geometry, 1-32 RHS and
    rtol 1e-6 / 1e-8 drawn per request) and collect the results: latency of each
    request from its arrival time, solves/s over the whole span, peak HBM held by
    the engines."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, nreq)
    gsel = rng.integers(0, len(geoms), nreq)
    nr = rng.integers(1, 33, nreq)
    rt = np.where(rng.integers(0, 2, nreq) == 0, 1e-6, 1e-8)
    rhs = [np.asfortranarray(np.random.default_rng(seed * 10 + i).uniform(-1, 1, (geoms[gsel[i]][1], nr[i])))
           for i in range(nreq)]
    pending, lat, worst, peak = {}, [], 0.0, 0
    t0 = time.perf_counter()
    arrive = t0 + np.cumsum(gaps)
    i = 0
    while i < nreq or pending:
        now = time.perf_counter()
        while i < nreq and arrive[i] <= now:
            t, shape = srv.submit(geoms[gsel[i]][2], rhs[i], float(rt[i]))
            pending[t] = (shape, arrive[i])
            i += 1
        for t in list(pending):
            shape, ta = pending[t]
            res = srv.poll(t, shape)
            if res is not None:
                lat.append(time.perf_counter() - ta)
                worst = max(worst, float(np.max(res[2])))
                del pending[t]
        peak = max(peak, srv.stats()["engine_bytes"])
        time.sleep(0.0005)
    span = time.perf_counter() - t0
    steps = srv.stats()["steps"]
    lat.sort()
    return {"requests": nreq, "rate_per_s": rate, "solves_per_s": nreq / span,
            "columns_per_s": float(nr.sum()) / span, "p50_s": lat[len(lat) // 2],
            "p99_s": lat[min(len(lat) - 1, int(0.99 * len(lat)))], "wall_s": span, "engine_steps": steps,
            "max_relres_over_rtol": worst, "peak_engine_hbm_gb": peak / 1e9}


def run_serve(args, local, stream):
    """Serving (continuous batching) over resident geometries: every geometry has
    an FP64-accurate handle and an FP32 handle; plain engines run GMRES(30) with
    FP64-accurate products, IR engines GMRES-IR (FP32 inner cycles to 1e-4,
    FP64-accurate residuals).  Two regimes on seeded Poisson streams: the
    arrival rate of the configuration (200 requests/s, above what one GPU
    serves, so latency there is mostly queueing) and a sustainable rate (half
    the lower of the two measured capacities), where p50/p99 are service
    latencies."""
    from paper_2203_05665_gb300 import H2Matrix, Server, inputs
    names = SERVE_SMALL if args.serve_small else list(SERVE_GEOMS)
    geoms, builds = [], {}
    for name in names:
        make, leaf = SERVE_GEOMS[name]
        v, f = make(inputs)
        t = time.perf_counter()
        hi = H2Matrix(v, f, leaf_size=leaf, eta=2.0, order=3, prec="f64", device=local, stream=stream.cuda_stream)
        lo = H2Matrix(v, f, leaf_size=leaf, eta=2.0, order=3, prec="f32", device=local, stream=stream.cuda_stream)
        builds[name] = time.perf_counter() - t
        geoms.append((name, f.shape[0], hi, lo))
    out = {"geometries": {nm: int(n) for nm, n, _, _ in geoms}, "m": 3, "nrhs": "U{1..32}",
           "rtol": "1e-6 or 1e-8", "seeds": [1005, 1006], "slots": 32, "build_s": builds,
           "handles_hbm_gb": sum(hi.stats["device_bytes"] + lo.stats["device_bytes"] for _, _, hi, lo in geoms) / 1e9}

    def regime(nreq, rate, seed):
        res = {}
        for mode in ("plain", "ir"):
            srv = Server(device=local)
            for name, n, hi, lo in geoms:
                srv.register(hi, lo if mode == "ir" else None, slots=32, restart=30, maxit=20000, inner_rtol=1e-4)
            res[mode] = _serve_stream(srv, geoms, nreq, rate, seed)
            srv.close()
        return res

    out["at_rate"] = regime(args.serve_requests, args.serve_rate, 1005)
    cap = min(out["at_rate"]["plain"]["solves_per_s"], out["at_rate"]["ir"]["solves_per_s"])
    out["sustained"] = regime(args.serve_sustain_requests, 0.5 * cap, 1006)
    for name, n, hi, lo in geoms:
        hi.close()
        lo.close()
    return out


def run_helmholtz(args, local, stream):
    """The Helmholtz single-layer matrix (Section 1's kernel e^{i kappa r}/(4 pi r))
    on icosphere level 7, m = 4, kappa = 2, 8 complex right-hand sides, FP64-
    accurate (both real parts on the tensor-core path): complex DoF x RHS per
    second of the product, and GMRES(30) on the real form to 1e-8 on icosphere
    level 5 (4 complex right-hand sides)."""
    import torch
    from paper_2203_05665_gb300 import HelmholtzMatrix, colmajor, inputs
    kappa, nrhs = 2.0, 8
    v, f = inputs.icosphere(args.level)
    n = f.shape[0]
    t = time.perf_counter()
    h = HelmholtzMatrix(v, f, kappa, leaf_size=32, eta=2.0, order=4, prec="f64", device=local,
                        stream=stream.cuda_stream)
    build_s = time.perf_counter() - t
    x_np = inputs.uniform_rhs(n, nrhs, 1007) + 1j * inputs.uniform_rhs(n, nrhs, 1008)
    x = colmajor(torch.from_numpy(x_np).to(device="cuda"))
    y = colmajor(torch.empty_like(x))
    for _ in range(3):
        h.matvec(x, y)
    reps = max(10, args.steps // 3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        h.matvec(x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    # algorithmic bytes: two real products (G_c, G_s) of 2 nrhs real columns each
    peaks = _peaks()
    hb = 2 * _algorithmic(h.stats, 2 * nrhs, 8)["total_bytes"]
    out = {"workload": f"Helmholtz kappa={kappa}, icosphere L{args.level} ({n} triangles), m=4, leaf 32, eta 2, "
                       f"{nrhs} complex RHS, FP64-accurate (tensor-core coupling and nearfield in both parts)",
           "ms_per_product": ms, "complex_dof_per_s": n * nrhs / (ms * 1e-3), "build_s": build_s,
           "device_bytes": h.stats["device_bytes"], "tensor": h.stats["tensor"], "tensor_near": h.stats["tensor_near"],
           "hbm_frac_whole_product": hb / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
           "algorithmic_bytes": hb, "peak_source": f"{peaks['src']} HBM copy bandwidth"}
    h.close()
    v5, f5 = inputs.icosphere(5)
    h5 = HelmholtzMatrix(v5, f5, kappa, leaf_size=32, eta=2.0, order=4, prec="f64", device=local,
                         stream=stream.cuda_stream)
    b = inputs.uniform_rhs(f5.shape[0], 4, 1009) + 1j * inputs.uniform_rhs(f5.shape[0], 4, 1010)
    h5.solve(b[:, :1], rtol=1e-8, restart=30, maxit=5000)
    t = time.perf_counter()
    z, it, rel, st = h5.solve(b, rtol=1e-8, restart=30, maxit=5000)
    ts = time.perf_counter() - t
    out["gmres"] = {"workload": f"icosphere L5 ({f5.shape[0]} triangles), 4 complex RHS, rtol 1e-8, GMRES(30) on "
                                "the real form", "solve_s": ts, "solves_per_s": 4 / ts,
                    "iters": [int(i) for i in it], "max_relres": float(max(rel)), "status": int(st)}
    h5.close()
    return out


def run_gca(args, local, stream):
    """GCA-H^2 (Section 3's GCA-H^2 example; the paper runs it with quadrature
    order 4, eta = 2 and cross-approximation accuracy 1e-4) on the main
    workload's mesh (icosphere level 7, leaf 32, 16 right-hand sides):
    products in FP64-accurate double-float and in FP32, their phases and a
    coupling roofline, the build, and GMRES(30) / GMRES-IR to 1e-8."""
    import torch
    from paper_2203_05665_gb300 import GcaMatrix, colmajor, inputs
    v, f = inputs.icosphere(args.level)
    n, nrhs = f.shape[0], args.nrhs
    x_np = inputs.uniform_rhs(n, nrhs, 1002)
    peaks = _peaks()
    out = {"workload": f"GCA-H2 eps 1e-4, Green quadrature order 4, eta 2, icosphere L{args.level} ({n} triangles), "
                       f"leaf 32, {nrhs} RHS"}
    mats = {}
    for prec in (("f64", "f32") if args.gca_prec == "both" else (args.gca_prec,)):
        t = time.perf_counter()
        h = GcaMatrix(v, f, leaf_size=32, eta=2.0, eps=1e-4, prec=prec, device=local, stream=stream.cuda_stream)
        build_s = time.perf_counter() - t
        dt, es = (torch.float64, 8) if prec == "f64" else (torch.float32, 4)
        x = colmajor(torch.from_numpy(x_np).to(device="cuda", dtype=dt))
        y = colmajor(torch.empty_like(x))
        for _ in range(3):
            h.matvec(x, y)
        reps = max(10, args.steps // 3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            h.matvec(x, y)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        h.profile(True)
        for _ in range(5):
            h.matvec(x, y)
        phases, products = h.phase_times()
        h.profile(False)
        st = h.stats
        cpl_ms = phases["coupling"][0] / products
        s_bytes = st["coupling_entries"] * es
        flops = 2.0 * nrhs * st["coupling_entries"]
        if prec == "f64":
            roof = {"bound": "alu", "achieved": flops / (cpl_ms * 1e-3) / 1e12, "peak": DD_TFLOPS, "unit": "TFLOP/s",
                    "peak_source": "FP32 FMA rate / 12 instructions per double-float multiply-add",
                    "hbm_frac": s_bytes / (cpl_ms * 1e-3) / 1e9 / peaks["hbm_gbs"]}
        else:
            roof = {"bound": "hbm", "achieved": s_bytes / (cpl_ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "peak_source": f"{peaks['src']} HBM copy bandwidth",
                    "algorithmic_bytes": "the stored coupling matrices (padded per level)"}
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof["kernel_ms"] = cpl_ms
        # whole product: nearfield, leaf bases (padded rank of the leaf level), coupling, transfer
        # matrices (two copies, one per direction, at most rank^2 per cluster), vectors
        K = st["rank"]
        tot = es * (st["near_entries"] + n * K + st["coupling_entries"] + 2 * st["clusters"] * K * K) \
            + 8 * 2 * n * nrhs
        roof["hbm_frac_whole_product_upper_bound"] = tot / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"]
        out[prec] = {"ms_per_product": ms, "dof_per_s": n * nrhs / (ms * 1e-3), "build_s": build_s,
                     "build_phases_ms": h.build_times(), "max_padded_rank": st["rank"],
                     "coupling_entries": st["coupling_entries"], "device_bytes": st["device_bytes"],
                     "phases_ms": {k: v_[0] / products for k, v_ in phases.items()}, "coupling_roofline": roof}
        mats[prec] = h
    if len(mats) < 2 or args.gca_only:
        for h in mats.values():
            h.close()
        return out
    b = inputs.uniform_rhs(n, nrhs, 1003)
    t = time.perf_counter()
    z, it, rel, st_ = mats["f64"].solve(b, rtol=1e-8, restart=30, maxit=2000)
    ts = time.perf_counter() - t
    out["gmres"] = {"solve_s": ts, "solves_per_s": nrhs / ts, "iters_max": int(it.max()), "max_relres": float(rel.max()),
                    "status": int(st_)}
    t = time.perf_counter()
    z, it, rel, st_ = mats["f64"].solve_ir(mats["f32"], b, rtol=1e-8)
    ts = time.perf_counter() - t
    out["gmres_ir_f32_inner"] = {"solve_s": ts, "solves_per_s": nrhs / ts, "max_relres": float(rel.max()),
                                 "status": int(st_)}
    for h in mats.values():
        h.close()
    return out


def run_small(args, local, stream):
    """The 5,120-triangle configuration (icosphere L4, m = 3, leaf 32, eta 2,
    FP64-accurate): latency of one product with one right-hand side, launched
    kernel by kernel (h2_matvec) and replayed from a CUDA graph (h2_graph_*),
    each the median over per-product CUDA-event pairs; and GMRES(30) to 1e-8 on
    the seeded uniform right-hand side and on the constant density."""
    import torch
    from paper_2203_05665_gb300 import H2Matrix, colmajor, inputs
    v, f = inputs.icosphere(4)
    n = f.shape[0]
    h = H2Matrix(v, f, leaf_size=32, eta=2.0, order=3, prec="f64", device=local, stream=stream.cuda_stream)
    x = colmajor(torch.from_numpy(inputs.uniform_rhs(n, 1, 1001)).to(device="cuda"))
    y = colmajor(torch.empty_like(x))
    yg = colmajor(torch.empty_like(x))
    g = h.graph(x, yg)
    reps = max(30, args.steps // 2)

    def lat(fn):
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        wall = []
        for a, b in ev:
            t = time.perf_counter()
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            wall.append(time.perf_counter() - t)
        dev = sorted(a.elapsed_time(b) * 1e3 for a, b in ev)
        wall.sort()
        return {"median_us": dev[len(dev) // 2], "min_us": dev[0], "p99_us": dev[min(reps - 1, int(0.99 * reps))],
                "host_wall_median_us": wall[len(wall) // 2] * 1e6}

    out = {"workload": f"icosphere L4 ({n} triangles), m=3 (k=27), leaf 32, eta 2, stored S, SS order 3, "
                       "FP64-accurate (double-float)", "reps": reps,
           "direct": lat(lambda: h.matvec(x, y)), "graph": lat(g.launch)}
    torch.cuda.synchronize()
    out["graph_equals_direct"] = bool(torch.equal(y, yg))
    out["graph_speedup"] = out["direct"]["median_us"] / out["graph"]["median_us"]
    # the single-launch product (h2_options.fused): one cooperative kernel
    hf = H2Matrix(v, f, leaf_size=32, eta=2.0, order=3, prec="f64", device=local, stream=stream.cuda_stream,
                  fused=True)
    yf = colmajor(torch.empty_like(x))
    ygf = colmajor(torch.empty_like(x))
    gf = hf.graph(x, ygf)
    out["fused"] = {"direct": lat(lambda: hf.matvec(x, yf)), "graph": lat(gf.launch)}
    torch.cuda.synchronize()
    out["fused"]["rel_diff_vs_phase_product"] = float(torch.linalg.norm(yf - y) / torch.linalg.norm(y))
    out["fused"]["graph_equals_direct"] = bool(torch.equal(yf, ygf))
    bf = np.asfortranarray(inputs.uniform_rhs(n, 1, 1001))
    hf.solve(bf, rtol=1e-8, restart=30, maxit=2000)
    t = time.perf_counter()
    zf, itf, relf, stf = hf.solve(bf, rtol=1e-8, restart=30, maxit=2000)
    out["fused"]["gmres"] = {"solve_s": time.perf_counter() - t, "iters": [int(i) for i in itf],
                             "relres": [float(r) for r in relf], "status": int(stf)}
    gf.close()
    hf.close()
    # constant density f = 1: the Galerkin right-hand side b_i = integral of f over T_i = |T_i|
    area = 0.5 * np.linalg.norm(np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]]), axis=1)
    b = np.asfortranarray(np.stack([inputs.uniform_rhs(n, 1, 1001)[:, 0], area], axis=1))
    h.solve(b, rtol=1e-8, restart=30, maxit=2000)
    t = time.perf_counter()
    z, it, rel, st = h.solve(b, rtol=1e-8, restart=30, maxit=2000)
    out["gmres"] = {"rhs": ["uniform [-1,1] seed 1001", "constant density (b_i = area of T_i)"], "rtol": 1e-8, "restart": 30,
                    "solve_s": time.perf_counter() - t, "iters": [int(i) for i in it],
                    "relres": [float(r) for r in rel], "status": int(st)}
    g.close()
    h.close()
    return out


def run_mixed(args, local, stream):
    """Mixed precision on icosphere level 8 (m = 3, 4 RHS): V and nearfield in
    BF16 or FP16 with FP32 accumulation, coupling regenerated in FP32; product
    time and error against the FP64-accurate product, and GMRES-IR to 1e-8
    (inner GMRES(30) on the 16-bit handle to 1e-2, FP64-accurate residuals)."""
    import torch
    from paper_2203_05665_gb300 import H2Matrix, colmajor, inputs
    v, f = inputs.icosphere(args.mixed_level)
    n = f.shape[0]
    x_np = inputs.uniform_rhs(n, 4, 1003)
    hi = H2Matrix(v, f, leaf_size=32, eta=2.0, order=3, prec="f64", device=local, stream=stream.cuda_stream)
    xd = colmajor(torch.from_numpy(x_np).to(device="cuda", dtype=torch.float64))
    yref = colmajor(torch.empty_like(xd))
    hi.matvec(xd, yref)
    out = {"workload": f"icosphere L{args.mixed_level} ({n} triangles), m=3, leaf 32, eta 2, 4 RHS",
           "hi": "f64 (double-float), stored S"}
    for prec in ("bf16", "f16"):
        lo = H2Matrix(v, f, leaf_size=32, eta=2.0, order=3, prec=prec, device=local, stream=stream.cuda_stream)
        xf = colmajor(xd.float())
        yf = colmajor(torch.empty_like(xf))
        for _ in range(3):
            lo.matvec(xf, yf)
        lo.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        reps = 20
        for _ in range(reps):
            lo.matvec(xf, yf)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        ph, prods = lo.phase_times()
        lo.profile(False)
        err = float(torch.linalg.norm(yf.double() - yref) / torch.linalg.norm(yref))
        t = time.perf_counter()
        z, it, rel, st = hi.solve_ir(lo, x_np, rtol=1e-8, inner_rtol=1e-2, restart=30, maxit_inner=5000,
                                     maxit_outer=50)
        ts = time.perf_counter() - t
        out[prec] = {"matvec_ms": ms, "dof_per_s": n * 4 / (ms * 1e-3), "rel_err_vs_f64": err,
                     "basis_prec": {1: "f32", 3: "bf16", 4: "f16"}[lo.stats["basis_prec"]],
                     "phases_ms": {k: vv[0] / prods for k, vv in ph.items()},
                     "device_bytes": lo.stats["device_bytes"], "build_phases_ms": lo.build_times(),
                     "ir_solve_s": ts, "ir_solves_per_s": 4 / ts, "ir_inner_iters": [int(i) for i in it],
                     "ir_max_relres": float(max(rel)), "ir_status": int(st)}
        lo.close()
    # the byte cost of the FP32 leaf bases under bfloat16: the same matrix with bfloat16 V
    lo = H2Matrix(v, f, leaf_size=32, eta=2.0, order=3, prec="bf16", basis="bf16", device=local,
                  stream=stream.cuda_stream)
    xf = colmajor(xd.float())
    yf = colmajor(torch.empty_like(xf))
    lo.matvec(xf, yf)
    torch.cuda.synchronize()
    out["bf16_with_bf16_bases"] = {
        "rel_err_vs_f64": float(torch.linalg.norm(yf.double() - yref) / torch.linalg.norm(yref)),
        "device_bytes": lo.stats["device_bytes"]}
    lo.close()
    out["hi_device_bytes"] = hi.stats["device_bytes"]
    out["hi_build_phases_ms"] = hi.build_times()
    hi.close()
    return out


def run_batch(args, local, stream, ws=1, rank=0):
    """Uneven batch: independent FP32 problems (random ellipsoids and subdivided
    cubes of 20k-400k triangles, m = 3 or 4, 1-8 RHS; leaf sizes chosen by the
    measuring autotuner) multiplied together, one persistent launch per
    block-row phase, replayed from a CUDA graph.  Reports aggregate DoF/s, the
    coupling kernel's HBM roofline fraction and an end-to-end figure with the
    packed vectors copied from and to pinned host memory."""
    import torch
    from paper_2203_05665_gb300 import Batch, H2Matrix, inputs, shard, tune
    all_specs = inputs.batch_problems(args.batch_problems, 1004)
    # N GPUs: each rank takes its share of the independent problems (weak scaling, no collective on the data path)
    specs = shard.shard_problems(all_specs, ws)[rank]
    t0 = time.time()
    free, _ = torch.cuda.mem_get_info()
    notes = []
    if args.batch_leaf:
        leaf = {s["index"]: args.batch_leaf for s in specs}
        timings = {}
    else:
        leaf, timings = tune.choose_leaf(specs, budget_bytes=int(0.8 * free), log=notes.append)
    tune_s = time.time() - t0
    t0 = time.time()
    mats = []
    for s in specs:
        v, f = inputs.problem_mesh(s)
        mats.append(H2Matrix(v, f, leaf_size=leaf[s["index"]], eta=2.0, order=s["order"], prec="f32",
                             coupling="stored", device=local, stream=stream.cuda_stream))
    build_s = time.time() - t0
    b = Batch(mats, [s["nrhs"] for s in specs], stream=stream.cuda_stream)
    g = torch.Generator(device="cuda").manual_seed(1004)
    x = torch.empty(b.length, dtype=torch.float32, device="cuda").uniform_(-1.0, 1.0, generator=g)
    y = torch.empty_like(x)
    b.matvec(x, y)
    t0 = time.time()
    if args.batch_shapes:
        shapes = [int(c) for c in args.batch_shapes.split(",")]
        b.set_shapes(shapes)
    else:
        shapes = b.tune(5)
    shape_s = time.time() - t0
    for _ in range(args.warmup):
        b.matvec(x, y)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(args.steps, 5)
    barrier()
    e0.record(stream)
    for _ in range(reps):
        b.matvec(x, y)
    e1.record(stream)
    barrier()
    b.sync()
    ms_rank = e0.elapsed_time(e1) / reps
    ms, all_dofs = shard.combine(ms_rank, b.info()["dofs"])
    b.profile(True)
    for _ in range(5):
        b.matvec(x, y)
    ph, prods = b.phase_times()
    b.profile(False)
    info = b.info()
    # algorithmic bytes (FP32): the coupling stream of every problem
    cbytes, tbytes, nbytes = 0, 0, 0
    for s, m in zip(specs, mats):
        a = _algorithmic(m.stats, s["nrhs"], 4)
        cbytes += a["coupling_bytes"]
        # leaf backward + nearfield: V and the nearfield blocks, the leaf vectors read and written
        nbytes += 4 * (m.stats["near_entries"] + m.n * m.stats["rank"] + 3 * m.n * s["nrhs"])
        tbytes += a["total_bytes"] - 8 * 2 * m.n * s["nrhs"] + 4 * 2 * m.n * s["nrhs"]
    cpl_ms = ph["coupling"][0] / prods
    peaks = _peaks()
    # end to end: packed x from pinned host memory, product, y back to pinned host memory
    xh = x.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    lat = []
    for i in range(max(3, min(args.steps, 10)) + 2):
        t1 = time.perf_counter()
        x.copy_(xh, non_blocking=True)
        b.matvec(x, y)
        yh.copy_(y, non_blocking=True)
        torch.cuda.synchronize()
        if i >= 2:
            lat.append(time.perf_counter() - t1)
    e2e_ms, _ = shard.combine(statistics.median(lat) * 1e3, 0)
    e2e_s = e2e_ms * 1e-3
    leaves = [leaf[s["index"]] for s in specs]
    out = {"workload": f"{len(all_specs)} problems: ellipsoids (icosphere L5-L7, semi-axes U[0.5,2]) and cubes "
                       f"(s in 41..182), m in {{3,4}}, 1-8 RHS, FP32 stored S, eta 2",
           "problems": len(all_specs), "problems_rank0": len(specs), "n_gpus": ws, "scaling": "weak",
           "triangles": int(sum(s["n"] for s in all_specs)), "dofs_x_rhs": int(all_dofs),
           "leaf_counts": {str(lf): leaves.count(lf) for lf in sorted(set(leaves))},
           "leaf_tuning_ms": {str(k): v for k, v in timings.items()}, "tune_notes": notes,
           "shapes": shapes, "tune_s": tune_s, "shape_tune_s": shape_s, "build_s": build_s,
           "ms_per_product": ms, "dof_per_s": all_dofs / (ms * 1e-3),
           "phases_ms": {k: v[0] / prods for k, v in ph.items()}, "gpu_launches": info["launches"],
           "graph": True,
           "roofline": {"bound": "hbm", "kernel": "k_batch_rows (coupling)", "unit": "GB/s",
                        "achieved": cbytes / (cpl_ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"],
                        "frac": cbytes / (cpl_ms * 1e-3) / 1e9 / peaks["hbm_gbs"], "kernel_ms": cpl_ms,
                        "hbm_frac_whole_product": tbytes / (ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                        "hbm_frac_leaf_near": nbytes / (ph["leaf_near"][0] / prods * 1e-3) / 1e9 / peaks["hbm_gbs"]},
           "device_bytes": int(sum(m.stats["device_bytes"] for m in mats) + info["work_bytes"]),
           "e2e": {"value": all_dofs / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(4 * b.length),
                   "d2h_bytes_per_step": int(4 * b.length)},
           "l2": "inputs larger than L2"}
    b.close()
    for m in mats:
        m.close()
    return out


def _oracle_sample(level, order, nrhs):
    import oracle
    from paper_2203_05665_gb300 import inputs
    v, f = inputs.icosphere(level)
    o = oracle.Oracle(v, f, leaf_size=32, eta=2.0, order=order)
    x = inputs.uniform_rhs(f.shape[0], nrhs, 1002)
    return o, x, f.shape[0]


def cpu_baseline(args):
    """The FP64 oracle as it stands on the host cores: full products of the bench
    workload on all cores (median of 5), and on one core a bounded sample (median
    of 5 full products on icosphere L5: the oracle is O(n), so its DoF/s per core
    hardly depends on the size, and one level-7 product takes about a minute on
    one core)."""
    import oracle
    lvl = args.cpu_level if args.cpu_level else args.level
    t = time.perf_counter()
    o, x, n = _oracle_sample(lvl, args.order, args.nrhs)
    setup_s = time.perf_counter() - t

    def median_of(obj, xx, reps=5):
        times = []
        for _ in range(reps):
            t1 = time.perf_counter()
            obj.matvec(xx)
            times.append(time.perf_counter() - t1)
        return statistics.median(times)

    cores = oracle.oracle.threads()
    t_all = median_of(o, x)
    del o
    oracle.oracle.set_threads(1)
    try:
        o1, x1, n1 = _oracle_sample(5, args.order, args.nrhs)
        t_one = median_of(o1, x1)
        del o1
    finally:
        oracle.oracle.set_threads(cores)
    return {"value": n * args.nrhs / t_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 C oracle, full product on icosphere L{lvl} ({n} triangles), m={args.order}, leaf 32, "
                      f"eta 2, {args.nrhs} RHS, nearfield stored, S evaluated on the fly; median of 5 products "
                      f"(set-up {setup_s:.1f} s, not timed)",
            "one_core": {"value": n1 * args.nrhs / t_one, "unit": UNIT, "cores": 1,
                         "sample": f"median of 5 full products on icosphere L5 ({n1} triangles), same m, leaf, "
                                   f"eta and RHS"}}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    import oracle
    lvl = args.cpu_level if args.cpu_level else 6
    o, x, n = _oracle_sample(lvl, args.order, args.nrhs)
    for _ in range(args.warmup):
        o.matvec(x)
    t = time.perf_counter()
    for _ in range(args.steps):
        o.matvec(x)
    el = time.perf_counter() - t
    ms = el / args.steps * 1e3
    value = n * args.nrhs / (ms * 1e-3)
    sample = (f"FP64 C oracle on the host cores: one full product per step on icosphere L{lvl} "
              f"({n} triangles), m={args.order}, leaf 32, eta 2, {args.nrhs} RHS")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"icosphere L{lvl} ({n} triangles), m={args.order}, leaf 32, eta 2, "
                                  f"{args.nrhs} RHS (bounded sample of the level-{args.level} workload)"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.oracle.threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="f64", choices=["f64", "f32", "f64n", "bf16", "f16"],
                    help="f64: FP64-accurate double-float arithmetic; f32; f64n: native FP64; "
                         "bf16 / f16: 16-bit storage, FP32 accumulation, regenerated coupling")
    ap.add_argument("--level", type=int, default=7)
    ap.add_argument("--order", type=int, default=4)
    ap.add_argument("--nrhs", type=int, default=16)
    ap.add_argument("--cpu-level", type=int, default=0,
                    help="icosphere level of the oracle timings (0: the bench level for cpu_baseline, "
                         "6 for --impl reference)")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--solve-nrhs", type=int, default=16)
    ap.add_argument("--solve-reps", type=int, default=3)
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-small", action="store_true", help="skip the icosphere L4 latency leg")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-helmholtz", action="store_true")
    ap.add_argument("--no-gca", action="store_true")
    ap.add_argument("--gca-only", action="store_true",
                    help="run the GCA-H2 leg alone and print its result (for profiling; no benchmark line)")
    ap.add_argument("--gca-prec", default="both", choices=["both", "f64", "f32"])
    ap.add_argument("--mixed-level", type=int, default=8)
    ap.add_argument("--serve-small", action="store_true",
                    help="four small geometries (icosphere L4-L6, ellipsoid L6) instead of all eight")
    ap.add_argument("--serve-requests", type=int, default=32, help="requests of the stream at --serve-rate")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-sustain-requests", type=int, default=16,
                    help="requests of the stream at half the measured capacity")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-problems", type=int, default=64)
    ap.add_argument("--batch-leaf", type=int, default=0, help="fixed leaf size instead of the autotuner")
    ap.add_argument("--batch-shapes", default="", help="four launch-shape indices instead of the shape tuner")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.gca_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"gca": run_gca(args, 0, torch.cuda.current_stream())}))
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
