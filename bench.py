"""Benchmark of the GB300 ray-transport hot path.

One step = one pass of the whole path (source sampling, crystal entry, depth
walk, detector binning, tallies) over one batch of rays of the von Hamos HAPG
workload (R = 80 mm, 40 um, pseudo-Voigt mosaic 0.1 deg, Darwin-Prins IRC,
three lines on a 1/E continuum, 1024^2 detector), 1e8 rays per step, FP32
kernel, each step a fresh ray range (new Philox counters).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  --impl reference times the CPU oracle (plain
FP64 C, all host cores) on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rays/sec to detector and fraction of FP32/SFU roofline; p50/p99 job latency"
UNIT = "rays/s"
# Algorithmic work per unit in lane-instructions (one thread executing one instruction:
# an FP32 add / multiply / fused multiply-add, an SFU function, a 32 x 32 -> 64-bit
# multiply, a compare or select, a shared-memory load), counted operation by operation
# from the method's steps, item by item:
ALGO_PER_RAY = {                # every emitted ray
    "philox_block": 40,         # call 0: 10 rounds x (2 wide multiplies + 2 three-input XORs)
    "uniforms": 8,              # its 4 words -> (0, 1): convert + fused multiply-add
    "cone_direction": 22,       # 1 - cos(phi), sin(phi), sin / cos of the azimuth, k, k.N offset
    "gaussian_spot": 17,        # Box-Muller radius and angle, origin += spot
    "cylinder_entry": 23,       # |o_perp + t k_perp| = R, smallest t > 0, axial and azimuth tests
}
ALGO_PER_ENTERED = {            # every ray that enters the crystal
    "philox_block": 40,         # call 1: the energy's words, drawn for entered rays only
    "entry_anchor": 14,         # |k.N| at the entry minus the cone axis's, as small terms
    "energy_and_bragg": 50,     # component, Gaussian line or 1/E draw, sin(aB) offset, anchor, Q, mu0
}
ALGO_PER_SEGMENT = {            # every straight segment (entered rays and reflections)
    "exit_distance": 42,        # inner / outer cylinder, axial and azimuth planes, exit anchor
    "thinning_bounds": 50,      # Bragg distance, tilt bound and table word, arc bound, shares
    "band_b_bound": 24,         # band B: its first word and 1 / sin, M, width, rsqrt, mirror test, rates
    "majorant": 8,              # mu0 + lambda, its inverse, absorption share and word threshold
}
ALGO_PER_COLLISION = {          # every tentative collision
    "philox_block": 40,
    "free_path": 9,             # word -> ln u, times 1/mu, Kahan sum, exit compare
    "absorb_and_share": 5,      # raw-word absorption compare, conditional uniform
    "local_normal": 14,         # cylinder: k.N and k.t2 at the collision from the path length
    "candidate": 22,            # stream split, table word map, quantile lookup, tilt test, sin theta
    "azimuth_and_offset": 10,   # azimuth sine / cosine (or arc test), k.n - sin(aB + dM)
    "rocking_curve_bound": 8,   # R bound at |e|, accept compare
}
ALGO_PER_EXIT = {               # every ray leaving the crystal
    "detector": 30,             # line-plane intersection, (u, v), pixel, atomic
}
ALGO_PER_END = 3                # tallies of an ended ray (outcome, reflections, no-Bragg)
ISSUE_PER_SM_CLK = 4            # 4 sub-partitions, one warp instruction each per clock
SM_COUNT = 152
SM_MAX_MHZ = 2070.0


def algorithmic_instructions(t):
    """lane-instructions of a trace's algorithmic work, from its tallies"""
    entered = t["emitted"] - t["miss"]
    reflections = sum(h * c for h, c in enumerate(t["refl_hist"]))
    exits = t["exit_front"] + t["exit_back"] + t["exit_side"]
    return (sum(ALGO_PER_RAY.values()) * t["emitted"] + sum(ALGO_PER_ENTERED.values()) * entered +
            sum(ALGO_PER_SEGMENT.values()) * (entered + reflections) +
            sum(ALGO_PER_COLLISION.values()) * t["collisions"] + sum(ALGO_PER_EXIT.values()) * exits +
            ALGO_PER_END * entered)


def algorithmic_roofline(t, seconds, sm_mhz):
    """algorithmic lane-instructions per second against the SM issue rate (32 lanes x
    4 sub-partitions x SMs x clock): the path runs on the integer, FP32 and SFU pipes"""
    achieved = algorithmic_instructions(t) / seconds / 1e12
    peak = SM_COUNT * ISSUE_PER_SM_CLK * 32 * sm_mhz * 1e6 / 1e12
    return achieved, peak


# rays per chunk of the two-pass trace (the library's largest hit-queue chunk)
WAVE_CHUNK = 1 << 26
# Per emitted ray of the von Hamos workload, from ncu captures of the two-pass kernels
# (both passes summed): DRAM bytes read + written (the hit queue written and read back;
# one chunk of 2^24 rays, whose 0.66 GB queue, unlike a smaller one, does not stay in
# L2) and warp instructions issued per pipe (2^22 rays), both with the library's default
# launch shape (bench.py --no-tune); valid only for the kernel sources with the hash below.
TRAFFIC_BYTES_PER_RAY = (0.165120e6 + 617.240832e6 + 676.016384e6 + 0.512512e6) / (1 << 24)   # 2^24 rays
PIPE_INST_PER_RAY = {"alu": 10.9531, "fma": 13.2470, "fmaheavy": 5.3638, "fmalite": 8.5234, "xu": 1.7617,
                     "lsu": 1.2817, "adu": 1.5328, "cbu": 2.7325, "uniform": 0.6104, "fp64": 0.0168,
                     "total": 35.6005}
TRAFFIC_SOURCES = ("paper_2503_16955_gb300/csrc/heart_fp32.cu", "paper_2503_16955_gb300/csrc/heart_fp64.cuh",
                   "paper_2503_16955_gb300/csrc/heart_internal.h")
TRAFFIC_SOURCE_HASH = "12e422257558e818"


def sources_hash():
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(n_rays):
    """DRAM traffic of one step of n_rays, or None if the kernels changed since the capture"""
    if TRAFFIC_BYTES_PER_RAY is None or sources_hash() != TRAFFIC_SOURCE_HASH:
        return None
    return TRAFFIC_BYTES_PER_RAY * n_rays


def per_pipe_roofline(H, n_rays, seconds, sm_mhz):
    """Issued warp instructions per pipe (ncu capture, per ray) over the step's time,
    against each pipe's issue rate measured on this GPU by heart_pipe_peaks (per SM
    per clock) at the step's SM clock; None if the kernels changed since the capture."""
    if PIPE_INST_PER_RAY is None or sources_hash() != TRAFFIC_SOURCE_HASH:
        return None
    peaks = H.heart_pipe_peaks()
    clk = sm_mhz * 1e6
    # pipe <- the microbenchmarked instruction that runs on it
    per_clk = {"alu": peaks["lop3"][1], "fma": peaks["ffma"][1], "fmaheavy": peaks["imad"][1],
               "xu": peaks["mufu_lg2"][1], "issue": float(ISSUE_PER_SM_CLK)}
    out = {}
    for pipe, rate in per_clk.items():
        inst = PIPE_INST_PER_RAY["total" if pipe == "issue" else pipe] * n_rays
        achieved = inst / seconds
        peak = rate * SM_COUNT * clk
        out[pipe] = {"warp_inst_per_ray": PIPE_INST_PER_RAY["total" if pipe == "issue" else pipe],
                     "achieved": achieved, "peak": peak, "frac": achieved / peak}
    binding = max((p for p in out if p != "issue"), key=lambda p: out[p]["frac"])
    return {"pipes": out, "binding_pipe": binding, "frac": out[binding]["frac"], "unit": "warp inst/s",
            "peak_basis": "heart_pipe_peaks per SM per clock (alu: LOP3, fma: FFMA, fmaheavy: IMAD, xu: "
                          "MUFU.LG2) x %d SMs x the step's median SM clock (%.0f MHz); issue: 4 per SM per "
                          "clock" % (SM_COUNT, sm_mhz),
            "microbenchmark": {k: v for k, v in peaks.items() if k not in ("sms",)}}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--rays", type=float, default=1e8)
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--serving-jobs", type=int, default=10_000)
    p.add_argument("--no-extra", action="store_true", help="skip batched / serving / FP64 measurements")
    p.add_argument("--no-tune", action="store_true",
                   help="keep the library's default launch shape instead of heart_autotune's choice (profiling: "
                        "the tuner times its probes, and under a profiler those times say nothing)")
    return p.parse_args()


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None
        self.file = None

    def __enter__(self):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        for line in self.file.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)
        os.unlink(self.file.name)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            for n, v in zip(names, s[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def cpu_baseline(workload, seconds, threads=0):
    """Oracle (plain FP64 C) on host cores over a bounded sample of the workload."""
    from oracle import binding as ob
    nthreads = threads or (os.cpu_count() or 1)
    spec, src = workload["spec"], workload["source"]
    ob.trace(spec, src, 2000, 77, n_threads=nthreads)            # table build, warm
    n = 20_000 * nthreads
    t0 = time.perf_counter()
    ob.trace(spec, src, n, 78, n_threads=nthreads)
    dt = time.perf_counter() - t0
    n2 = int(min(5e8, max(n, n * seconds / max(dt, 1e-3))))
    t0 = time.perf_counter()
    _, tal, _ = ob.trace(spec, src, n2, 79, n_threads=nthreads)
    dt = time.perf_counter() - t0
    return {"value": n2 / dt, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": "%d rays of %s (seed 79), %.1f s on %d host threads" % (n2, workload["name"], dt, nthreads),
            "collisions_per_ray": tal["collisions"] / max(1, n2)}


def batched_measurement(H, W, torch, stream, sm_mhz):
    """64 spectrometers of uneven ray counts in one heart_trace_batch call (jobs
    of 2^18 rays or more as two-pass traces, the rest in one persistent launch)."""
    jobs = W.batched_64()
    specs = [H.heart_spectrometer_create(j["spec"]) for j in jobs]
    imgs = [torch.zeros(s.shape, dtype=torch.int32, device="cuda") for s in specs]
    args = ([j["source"] for j in jobs], [j["n_rays"] for j in jobs], [j["seed"] for j in jobs])
    # warm: the same kernels (two-pass for the large jobs, the hit queue at full size)
    small = [min(n, WAVE_CHUNK) if n >= 1 << 18 else max(1, n // 100) for n in args[1]]
    H.heart_trace_batch(specs, args[0], small, args[2], imgs, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tl = H.heart_trace_batch(specs, args[0], args[1], args[2], imgs, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    total = sum(args[1])
    # the same batch through the entry point that allocates nothing (every job on the persistent kernel)
    H.heart_trace_batch_static(specs, args[0], [max(1, n // 100) for n in args[1]], args[2], imgs, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    H.heart_trace_batch_static(specs, args[0], args[1], args[2], imgs, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    sec_static = e0.elapsed_time(e1) / 1e3
    for s in specs:
        s.close()
    summed = {k: sum(t[k] for t in tl) for k in ("emitted", "miss", "exit_front", "exit_back", "exit_side",
                                                  "collisions")}
    summed["refl_hist"] = [sum(t["refl_hist"][h] for t in tl) for h in range(16)]
    achieved, peak = algorithmic_roofline(summed, sec, sm_mhz)
    return {"jobs": len(jobs), "rays": total, "seconds": sec, "rays_per_s": total / sec,
            "collisions_per_ray": sum(t["collisions"] for t in tl) / total,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T lane-instr/s",
                         "frac": achieved / peak, "basis": "the headline's per-unit counts over the batch's "
                                                           "tallies, CUDA-event time of the call"},
            "static_rays_per_s": total / sec_static,
            "note": "one heart_trace_batch call: jobs of >= 2^18 rays as two-pass traces, the rest in one "
                    "persistent launch (includes tally read-back); static: heart_trace_batch_static on the same "
                    "jobs, one persistent launch over all of them, no device allocation"}


def serving_measurement(H, W, n_jobs, rate, rho=None, capacity=None):
    """Poisson stream of trace jobs through the request loop; latencies are
    measured by the server from submit to completion.  rate None: the rate that
    offers rho times `capacity` rays/s."""
    import threading as th
    pool = W.batched_64(seed=4, ray_range=(1e4, 1e8))
    specs = [H.heart_spectrometer_create(j["spec"]) for j in pool]
    if rate is None:
        mean_rays = sum(j["n_rays"] for j in W.serving_stream(n_jobs=n_jobs, rate_per_s=1.0)) / n_jobs
        rate = rho * capacity / mean_rays
    stream = W.serving_stream(n_jobs=n_jobs, rate_per_s=rate)
    srv = H.heart_server_create(40 << 30)
    ids = []
    lat = []
    done = th.Event()

    def reaper():
        i = 0
        while i < len(stream):
            while i >= len(ids):
                time.sleep(0.0005)
            st, t, _ = srv.poll(ids[i], timeout_ms=600_000)
            lat.append(srv.latency(ids[i]))
            srv.release(ids[i])
            i += 1
        done.set()

    r = th.Thread(target=reaper, daemon=True)
    r.start()
    t0 = time.perf_counter()
    rays = 0
    for k, job in enumerate(stream):
        delay = job["arrival_s"] - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        j = k % len(specs)
        ids.append(srv.submit(specs[j], pool[j]["source"], job["n_rays"], job["seed"]))
        rays += job["n_rays"]
    done.wait()
    wall = time.perf_counter() - t0
    srv.close()
    lat_ms = sorted(1e3 * x for x in lat)
    q = lambda v, p: v[min(len(v) - 1, int(p * len(v)))]
    offered = rays / stream[-1]["arrival_s"]
    # the same jobs as serial single-job launches (one heart_trace each, FP32, synchronised):
    # their service times, and the latencies of a first-come-first-served serial server fed
    # by the same arrivals
    import torch
    imgs = [torch.zeros(sp.shape, dtype=torch.int64 if j["spec"]["count_type"] == "i64" else torch.int32,
                        device="cuda") for sp, j in zip(specs, pool)]
    service = []
    for k, job in enumerate(stream):
        j = k % len(specs)
        torch.cuda.synchronize()
        c0 = time.perf_counter()
        H.heart_trace(specs[j], pool[j]["source"], job["n_rays"], job["seed"], 0, imgs[j], want_tally=False)
        torch.cuda.synchronize()
        service.append(time.perf_counter() - c0)
    for sp in specs:
        sp.close()
    finish, serial_lat = 0.0, []
    for job, sv in zip(stream, service):
        finish = max(job["arrival_s"], finish) + sv
        serial_lat.append(1e3 * (finish - job["arrival_s"]))
    serial_lat.sort()
    return {"jobs": n_jobs, "rate_per_s": rate, "p50_ms": q(lat_ms, 0.50), "p99_ms": q(lat_ms, 0.99),
            "max_ms": lat_ms[-1], "rays_per_s": rays / wall, "offered_rays_per_s": offered,
            "utilisation_rho": offered / (rays / sum(service)),
            "serial_fp32": {"rays_per_s": rays / sum(service), "p50_ms": q(serial_lat, 0.50),
                            "p99_ms": q(serial_lat, 0.99), "max_ms": serial_lat[-1],
                            "note": "the same jobs, one synchronised heart_trace each, queued first come first "
                                    "served at the same arrival times"},
            "note": "spectrometers drawn from a pool of 64 (seed 4); rays log-uniform 1e4-1e8"}


def fp64_measurement(H, W, torch, stream):
    """Plain FP64 single-configuration path on the flat HOPG workload (2e5 rays)."""
    w = W.flat_hopg_mono()
    s = H.heart_spectrometer_create(w["spec"])
    img = torch.zeros(s.shape, dtype=torch.int32, device="cuda")
    H.heart_trace(s, w["source"], w["n_rays"], w["seed"], 0, img, precision="fp64", stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record(stream)
    for i in range(reps):
        H.heart_trace(s, w["source"], w["n_rays"], w["seed"], (i + 1) * w["n_rays"], img, precision="fp64",
                      stream=stream, want_tally=False)
    e1.record(stream)
    torch.cuda.synchronize()
    fp64 = reps * w["n_rays"] / (e0.elapsed_time(e1) / 1e3)
    n32 = 100 * w["n_rays"]
    H.heart_trace(s, w["source"], n32, w["seed"], 0, img, precision="fp32", stream=stream, want_tally=False)
    e0.record(stream)
    H.heart_trace(s, w["source"], n32, w["seed"], n32, img, precision="fp32", stream=stream, want_tally=False)
    e1.record(stream)
    torch.cuda.synchronize()
    fp32 = n32 / (e0.elapsed_time(e1) / 1e3)
    s.close()
    return {"workload": w["name"], "fp64_rays_per_s": fp64, "fp32_rays_per_s": fp32, "fp32_speedup": fp32 / fp64}


def features_measurement(H, W, torch, stream):
    """Throughput of the path's options on the von Hamos workload (device-timed,
    inputs resident): energy image, polarised source, user-supplied rays, no
    rocking curve (FP32), and three reflection orders with an energy-dependent
    rocking curve (FP32 on the persistent kernel, and FP64)."""
    w = W.von_hamos_hapg()
    out = {}

    def timed(fn, n):
        fn(0)                                                 # warm (autotune-free path)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        t = fn(n)
        e1.record(stream)
        torch.cuda.synchronize()
        return n / (e0.elapsed_time(e1) / 1e3), t

    s = H.heart_spectrometer_create(w["spec"])
    img = torch.zeros(s.shape, dtype=torch.int32, device="cuda")
    eimg = torch.zeros(s.shape, dtype=torch.int64, device="cuda")
    n = 50_000_000
    r, _ = timed(lambda off: H.heart_trace_energy(s, w["source"], n, w["seed"], off, img, eimg,
                                                 qe=[(7.0, 0.8), (9.0, 0.6)], stream=stream), n)
    out["energy_image_rays_per_s"] = r
    pol = dict(w["source"], polarization=[0.0, 1.0, 0.0])
    r, _ = timed(lambda off: H.heart_trace(s, pol, n, w["seed"], off, img, stream=stream), n)
    out["polarised_rays_per_s"] = r
    nu = 10_000_000
    rays = W.user_rays(w, nu, seed=7, polarised=True)
    names = dict(ox="origin_x", oy="origin_y", oz="origin_z", kx="dir_x", ky="dir_y", kz="dir_z",
                 E="energy_keV", px="pol_x", py="pol_y", pz="pol_z")
    dev = {names[k]: torch.as_tensor(v, dtype=torch.float64, device="cuda").contiguous() for k, v in rays.items()}
    r, _ = timed(lambda off: H.heart_trace_rays(s, dev, w["seed"], off, img, stream=stream), nu)
    out["user_rays_polarised_rays_per_s"] = r
    s.close()
    s = H.heart_spectrometer_create(dict(w["spec"], irc="none"))
    nn = 10_000_000
    r, t = timed(lambda off: H.heart_trace(s, w["source"], nn, w["seed"], off, img, stream=stream), nn)
    out["irc_none_rays_per_s"] = r
    out["irc_none_collisions_per_ray"] = t["collisions"] / nn
    s.close()
    s = H.heart_spectrometer_create(dict(w["spec"], orders=[(1, 1.0, 1.0), (2, 0.45, 0.6), (3, 0.2, 0.4)],
                                         irc_energy=[(7.6, 0.8, -1e-5), (8.4, 1.4, 2e-5)]))
    n32 = 50_000_000
    r, _ = timed(lambda off: H.heart_trace(s, w["source"], n32, w["seed"], off, img, stream=stream), n32)
    out["orders3_energy_table_fp32_rays_per_s"] = r
    n64 = 1_000_000
    r, _ = timed(lambda off: H.heart_trace(s, w["source"], n64, w["seed"], off, img, precision="fp64",
                                           stream=stream), n64)
    out["orders3_energy_table_fp64_rays_per_s"] = r
    s.close()
    out["note"] = ("von_hamos_hapg; energy image with a 2-knot QE; polarised: source p0 = y; user rays: 1e7 "
                   "polarised arrays in HBM; irc none: FP32 cone candidates; orders: (002), (004), (006) with "
                   "an energy table, FP32 and FP64")
    return out


def large_measurement(H, W, torch, stream, sm_mhz):
    """The large single job: von Hamos R = 100 mm, Lorentzian mosaic, elastic +
    inelastic lines, 4096^2 int64 detector, 1e10 rays in one call (streamed by
    the library in chunks of 2^26 rays), FP32; device-timed."""
    w = W.von_hamos_large()
    s = H.heart_spectrometer_create(w["spec"])
    img = torch.zeros(s.shape, dtype=torch.int64, device="cuda")
    H.heart_trace(s, w["source"], 1 << 26, w["seed"], 0, img, stream=stream)          # warm (queue, tables)
    torch.cuda.synchronize()
    n = w["n_rays"]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t = H.heart_trace(s, w["source"], n, w["seed"], 1 << 26, img, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    s.close()
    achieved, peak = algorithmic_roofline(t, sec, sm_mhz)
    entered = n - t["miss"]
    return {"workload": w["name"], "rays": n, "seconds": sec, "rays_per_s": n / sec,
            "collisions_per_ray": t["collisions"] / n, "entered_per_ray": entered / n,
            "collisions_per_entered_ray": t["collisions"] / max(1, entered), "det_hits": t["det_hits"],
            "detector": "%dx%d int64" % (w["spec"]["det_ny"], w["spec"]["det_nx"]),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T lane-instr/s",
                         "frac": achieved / peak}}


def run_reference(args):
    import torch.distributed as dist  # noqa: F401
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2503_16955_gb300 import workloads as W
    w = W.von_hamos_hapg()
    steps, warm = args.steps, args.warmup
    base = cpu_baseline(w, min(args.cpu_seconds, 6.0))
    # each step: a bounded sample of the workload traced by the oracle
    from oracle import binding as ob
    nthreads = os.cpu_count() or 1
    n = int(max(10_000, base["value"] * 1.5))
    for i in range(warm):
        ob.trace(w["spec"], w["source"], max(1000, n // 10), 100 + i, n_threads=nthreads)
    t0 = time.perf_counter()
    for i in range(steps):
        ob.trace(w["spec"], w["source"], n, 200 + i, ray_offset=i * n, n_threads=nthreads)
    dt = time.perf_counter() - t0
    v = n * steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": warm, "ms_per_step": 1e3 * dt / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "rays_per_step": n, "sample_of": int(w["n_rays"]),
                       "l2": "oracle on host cores"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                             "sample": "%d rays per step x %d steps of %s" % (n, steps, w["name"])},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    import paper_2503_16955_gb300 as H
    from paper_2503_16955_gb300 import workloads as W

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    w = W.von_hamos_hapg()
    n = int(args.rays)
    spec = H.heart_spectrometer_create(w["spec"])
    stream = torch.cuda.Stream()
    img = torch.zeros(spec.shape, dtype=torch.int32, device="cuda")
    # rank r traces its own ray ranges: weak scaling, no data-path collective
    def offset(step):
        return (step * world + rank) * n

    def barrier():
        if world > 1:
            dist.barrier()

    tune = ("library default (refill 8 idle lanes, 6 blocks per SM)" if args.no_tune else
            H.heart_autotune(spec, w["source"], probe_rays=min(n, 1 << 24), stream=stream))
    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            H.heart_trace(spec, w["source"], n, w["seed"], offset(1000 + i), img, precision="fp32",
                          stream=stream, want_tally=False)
    stream.synchronize()
    # timed region: K steps, CUDA events on the launching stream
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    tallies = []
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        with torch.cuda.stream(stream):
            ev[0].record(stream)
            for i in range(args.steps):
                H.heart_trace(spec, w["source"], n, w["seed"], offset(i), img, precision="fp32", stream=stream,
                              want_tally=False)
                ev[i + 1].record(stream)
        stream.synchronize()
    torch.cuda.synchronize()
    barrier()
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_s = sum(step_ms) / 1e3
    t = torch.tensor([total_s], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    total_max = float(t.item())
    value = n * args.steps * world / total_max

    # one more step with tallies for the work count (outside the timed region)
    tal = H.heart_trace(spec, w["source"], n, w["seed"], offset(args.steps + 7), img, precision="fp32",
                        stream=stream)
    coll_per_ray = tal["collisions"] / n
    det_frac = tal["det_hits"] / n
    # straight segments: one per entered ray plus one per reflection
    seg_per_ray = ((n - tal["miss"]) + sum(h * c for h, c in enumerate(tal["refl_hist"]))) / n

    # end to end through the C ABI with host buffers (copies inside the call), the image in
    # pinned host memory
    h_img_t = torch.zeros(spec.shape, dtype=torch.int32, pin_memory=True)
    h_img = h_img_t.numpy()
    e2e_steps = max(1, min(args.steps, 5))
    H.heart_trace_host(spec, w["source"], n, w["seed"], offset(2000), h_img, precision="fp32")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        H.heart_trace_host(spec, w["source"], n, w["seed"], offset(3000 + i), h_img, precision="fp32")
    e2e_s = time.perf_counter() - t0
    e2e_value = n * e2e_steps * world / e2e_s
    img_bytes = h_img.nbytes

    # roofline: issue-bound (integer, FP32 and SFU instructions); algorithmic work from the
    # tallies of a step, over the step's mean duration, against the SM issue rate at the
    # step's median SM clock (the max clock if unsampled)
    clocks = clk.summary()
    sm_mhz = clocks.get("sm_mhz") or SM_MAX_MHZ
    mean_launch_s = total_max / args.steps
    tal_step = dict(tal)
    achieved, peak = algorithmic_roofline(tal_step, mean_launch_s, sm_mhz)
    pipes = per_pipe_roofline(H, n, mean_launch_s, sm_mhz) if rank == 0 else None
    cpu = cpu_baseline(w, args.cpu_seconds) if rank == 0 and world == 1 else None
    spec.close()
    extra = {}
    if rank == 0 and world == 1 and not args.no_extra:
        extra["batched"] = batched_measurement(H, W, torch, stream, sm_mhz)
        extra["fp64_plain"] = fp64_measurement(H, W, torch, stream)
        extra["serving"] = serving_measurement(H, W, args.serving_jobs, 200.0)
        extra["serving_high_rate"] = serving_measurement(H, W, args.serving_jobs, None, rho=0.9,
                                                         capacity=extra["serving"]["serial_fp32"]["rays_per_s"])
        extra["features"] = features_measurement(H, W, torch, stream)
        extra["large_job"] = large_measurement(H, W, torch, stream, sm_mhz)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["name"], "rays_per_step": n, "precision": "fp32",
                       "detector": "%dx%d int32" % (w["spec"]["det_ny"], w["spec"]["det_nx"]),
                       "launch": tune,
                       "sampler": "thinned",
                       "collisions_per_ray": coll_per_ray, "segments_per_ray": seg_per_ray,
                       "det_hits_per_ray": det_frac,
                       "detector_hits_per_s": value * det_frac,
                       "l2": "inputs are per-ray counters (no input data); the 4 MB image stays in L2"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "T lane-instr/s",
                         "frac": achieved / peak, "traffic": measured_traffic(n),
                         "traffic_note": "ncu dram__bytes_read+write of the step's launches, per step (hit "
                                         "queue written by the spawn pass and read by the walk pass; "
                                         "captured on one 2^24-ray chunk, scaled by rays)",
                         "kernel": "k_spawn32 + k_walk32 (two passes per chunk of up to 2^26 rays)",
                         "peak_basis": "152 SMs x 4 sub-partitions x 32 lanes x %.0f MHz (the step's median SM "
                                       "clock); algorithmic lane-instructions counted per ray %d, per entered "
                                       "ray %d, per segment %d, per collision %d, per exit %d (bench.py ALGO_*)"
                                       % (sm_mhz, sum(ALGO_PER_RAY.values()), sum(ALGO_PER_ENTERED.values()),
                                          sum(ALGO_PER_SEGMENT.values()), sum(ALGO_PER_COLLISION.values()),
                                          sum(ALGO_PER_EXIT.values())),
                         "per_pipe": pipes},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": img_bytes,
                    "d2h_bytes_per_step": img_bytes + 27 * 8,
                    "path": "heart_trace_host (pinned host image uploaded, traced, downloaded each step)"},
            "gpu_launches": args.steps * 2 * ((n + WAVE_CHUNK - 1) // WAVE_CHUNK),
            "clocks": clocks,
            "cpu_baseline": cpu,
            **extra,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
