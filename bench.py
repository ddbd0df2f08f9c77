"""Benchmark of the symbolic-phase sampling hot path on GB300.

One step = one call of sp_sample producing the measurement, detector and
observable records of 1,000,000 shots of the rotated surface-code Z memory
(d = 11, 11 rounds, circuit-level noise p = 1e-3): the Philox fault draw, the
GF(2) product and the record epilogue, with the sampler program already
built (the paper times initialization and sampling separately; the build
time is reported in the JSON line as build_ms).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) each rank samples its own shot range with no
collective (weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = {"name": "surface_code_d11_r11_p1e-3", "distance": 11, "rounds": 11, "p": 1e-3}
SHOTS = 1_000_000
METRIC = "shots_per_s"
UNIT = "shots/s"

# DRAM traffic of one launch of the fused sampling kernel on this workload:
# dram__bytes_read.sum + dram__bytes_write.sum from a one-pass ncu capture of
# the first timed 1,000,000-shot launch. The figure belongs to the kernel
# source it was taken on; when the hash of that source differs, it is dropped
# (reported as null) until a new capture replaces it.
FUSED_TRAFFIC = {"shots": 1_000_000, "bytes": 1_020_000 + 300_970_000,
                 "sources_sha256": "a8808867e4aabe5c74ebf48eec83518928132dec1dcf33584241907bd620ebb9"}
FUSED_SOURCES = ("paper_2311_03906_gb300/csrc/sp_fused.cu", "paper_2311_03906_gb300/csrc/sp_internal.h")


def _sources_sha256(paths=FUSED_SOURCES):
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _fused_traffic(shots_per_launch):
    """Measured DRAM bytes of one fused launch of shots_per_launch shots (the
    records written grow in proportion to the shots), or None when no capture
    matches the current kernel source."""
    t = FUSED_TRAFFIC
    if t["bytes"] is None or t["sources_sha256"] != _sources_sha256():
        return None
    return t["bytes"] * shots_per_launch / t["shots"]


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "sm_max_mhz": d.get("sm_max_mhz", 2070.0),
                "bf16_tflops": d.get("bf16_tflops", 1900.0), "source": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "bf16_tflops": 1900.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            os.makedirs(os.path.join(ROOT, "gpurun_out"), exist_ok=True)
            self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
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
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    from paper_2311_03906_gb300.dist import world
    return world()


def _cpu_baseline(circuit, budget_s: float = 12.0, seed: int = 1):
    """The oracle as it stands, single-threaded, on a bounded sample."""
    import oracle
    t0 = time.perf_counter()
    prog = oracle.Program(circuit)
    build_s = time.perf_counter() - t0
    done, batch = 0, 64
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        prog.sample(seed, done, batch)
        done += batch
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} shots of {WORKLOAD['name']} (shots 0..{done - 1}, seed {seed}), "
                      f"single-threaded plain C oracle, {dt:.1f} s; oracle build {build_s * 1e3:.0f} ms"}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return
    from workloads import surface_code
    import oracle
    circuit = surface_code(WORKLOAD["distance"], WORKLOAD["rounds"], WORKLOAD["p"])
    prog = oracle.Program(circuit)
    per_step = 2048
    for w in range(args.warmup):
        prog.sample(1, w * per_step, 64)
    times = []
    for k in range(args.steps):
        t0 = time.perf_counter()
        prog.sample(1, k * per_step, per_step)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = per_step * args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "shots_per_step": per_step,
                       "note": "bounded sample of the 1e6-shot step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} steps x {per_step} shots, single-threaded plain C oracle"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _batched_vs_plain(args):
    """64 uneven circuits (rotated surface codes d = 3..15, p in {5e-4, 1e-3,
    2e-3}, seeds 0..63), 1e5 shots each: one graph-captured batched enqueue
    vs 64 separate sp_sample calls, identical records."""
    import torch
    import paper_2311_03906_gb300 as sp
    from workloads import batch_suite
    suite = batch_suite(64)
    t0 = time.perf_counter()
    progs = [sp.build(c) for c, _ in suite]
    build_s = time.perf_counter() - t0
    seeds = [s for _, s in suite]
    shots = [args.batch_shots] * len(progs)
    outs = [p.alloc_outputs(n) for p, n in zip(progs, shots)]
    stream = torch.cuda.current_stream()

    def batched():
        sp.sample_batch(progs, seeds, shots, outs=outs)

    def plain():
        for p, s, n, o in zip(progs, seeds, shots, outs):
            p.sample(n, seed=s, out=o)

    res = {}
    for name, fn in (("batched", batched), ("plain", plain)):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reps = 3
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"ms": ms, "shots_per_s": sum(shots) / (ms / 1e3)}
    res["speedup"] = res["plain"]["ms"] / res["batched"]["ms"]
    res["config"] = {"workload": "64 rotated surface codes d=3+2*(i mod 7), p=(5e-4,1e-3,2e-3)[(i//7) mod 3], seed i",
                     "shots_per_circuit": args.batch_shots, "build_s": build_s,
                     "paths": {"fused": sum(p.info["path"] == 3 for p in progs),
                               "staged": sum(p.info["path"] == 1 for p in progs)}}
    for p in progs:
        p.close()
    return res


def _dense_paths(args):
    """A circuit whose coefficient rows are dense (mirror circuit: 512 qubits,
    16 random Clifford layers then their inverse, DEPOLARIZE1(p) after
    every layer, every qubit measured with one detector each; about 33k
    symbols, 1,024 record rows, ~40 % of the coefficients set): the same
    shots sampled with the product as the tcgen05 tensor-core contraction,
    the CUDA-core AND/popcount form and the sparse fused kernel, plus the
    build's own timed choice. The tensor kernel's roofline is its FP8 rate
    (measured bf16 peak x 2, the nominal FP8:BF16 ratio)."""
    import torch
    import paper_2311_03906_gb300 as sp
    from workloads import mirror_circuit
    peaks = _peaks()
    c = mirror_circuit(512, 16, p=args.dense_p, seed=1)
    t0 = time.perf_counter()
    prog = sp.build(c)
    build_s = time.perf_counter() - t0
    info = prog.info
    auto = info["path"]
    shots = args.dense_shots
    out = prog.alloc_outputs(shots)
    rows = info["num_measurements"] + info["num_detectors"] + info["num_observables"]
    flops = 2.0 * rows * (info["num_symbols"] + 1) * shots
    stream = torch.cuda.current_stream()
    names = {sp.PATH_TENSOR: "tensor", sp.PATH_DENSE: "dense", sp.PATH_FUSED: "fused", sp.PATH_SPARSE: "staged-sparse"}
    sparse_path = sp.PATH_FUSED if info["fused_tile_shots"] else sp.PATH_SPARSE
    res = {}
    for path in (sp.PATH_TENSOR, sp.PATH_DENSE, sparse_path):
        prog.set_path(path)
        prog.sample(shots, seed=1, out=out)
        torch.cuda.synchronize()
        prog.profile(True)
        prog.profile_read()
        reps = 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for r in range(reps):
            prog.sample(shots, seed=1, shot0=(r + 1) * shots, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        prof = prog.profile_read()
        prog.profile(False)
        kern = {k: {"ms_per_step": v[0] / reps, "launches_per_step": v[1] / reps} for k, v in prof.items() if v[1]}
        res[names[path]] = {"ms": ms, "shots_per_s": shots / (ms / 1e3), "kernels": kern}
    status = prog.device_status()
    t = res["tensor"]["kernels"].get("tensor")
    roof = None
    if t:
        achieved = flops / (t["ms_per_step"] / 1e3) / 1e12
        peak = 2.0 * peaks["bf16_tflops"]
        roof = {"kernel": "k_tc_product", "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "peak_source": f"MEASURED_PEAKS.json bf16_tflops x 2 (nominal FP8:BF16 ratio; {peaks['source']})"}
    prog.close()
    return {"config": {"workload": f"mirror_circuit(n=512, layers=16, p={args.dense_p:g}, seed=1)", "shots_per_step": shots,
                       "symbols": info["num_symbols"], "record_rows": rows, "density": info["density"],
                       "build_s": build_s, "auto_path": names.get(auto, str(auto)),
                       "build_probe_ms": {names[k]: v for k, v in enumerate(info["path_probe_ms"]) if v > 0 and k in names}},
            "paths": res, "tensor_roofline": roof, "device_status": status,
            "algorithmic_flops_per_shot": flops / shots}


def _build_times(args):
    """Time to initialize a sampler (the paper's second measure, Sec. 5): sp_build
    (GPU traversal, replay, detector rows, sampler program, autotuner) against
    the oracle's build on the random layered circuits of Fig. 3c (n qubits x n
    layers, floor(n/2) CX pairs and DEPOLARIZE1(0.01) on every qubit per layer,
    5% of the qubits measured per layer, all measured at the end). The oracle
    is timed only up to n = 300 (its cost grows about as n^4)."""
    import paper_2311_03906_gb300 as sp
    import oracle
    from workloads import random_layered
    out = []
    for n in args.build_sizes:
        c = random_layered(n, n, depolarize=0.01, seed=1)
        t0 = time.perf_counter()
        prog = sp.build(c)
        gpu_s = time.perf_counter() - t0
        row = {"n": n, "ops": len(c.ops), "symbols": prog.info["num_symbols"],
               "measurements": prog.info["num_measurements"], "gpu_build_s": gpu_s,
               "gpu_build_ms_library": prog.info["build_ms"]}
        prog.close()
        if n <= 300:
            t0 = time.perf_counter()
            oracle.Program(c)
            row["oracle_build_s"] = time.perf_counter() - t0
            row["oracle_over_gpu"] = row["oracle_build_s"] / gpu_s
        out.append(row)
    return {"workload": "random_layered(n, n, depolarize=0.01, seed=1)", "rows": out}


def _fit(args):
    """Config 5: d=11, 11 rounds, per-channel p_i ~ U(5e-4, 2e-3); 1e6 shots
    sampled at p' = p(1 + delta), delta ~ U(-0.2, 0.2); the per-channel
    probabilities are fitted to the sampled detector rates by Adam on
    sum_j (r_j(p) - r^_j)^2, r_j = (1 - E_j)/2, through the expectation's
    forward and hand-written backward kernels."""
    import torch
    import paper_2311_03906_gb300 as sp
    from workloads import channel_probabilities, perturbed_probabilities, surface_code, with_channel_probabilities
    base = surface_code(11, 11, 1e-3)
    p0 = channel_probabilities(base.num_fault_channels, seed=0)
    pt = perturbed_probabilities(p0, seed=1)
    prog_t = sp.build(with_channel_probabilities(base, pt))
    prog = sp.build(with_channel_probabilities(base, p0))
    shots = 1_000_000
    ndet = prog.num_detectors
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = prog_t.alloc_outputs(shots)
    prog_t.sample(shots, seed=11, out=out, meas=False, obs=False)
    torch.cuda.synchronize()
    e0.record()
    prog_t.sample(shots, seed=11, out=out, meas=False, obs=False)
    e1.record()
    torch.cuda.synchronize()
    sample_ms = e0.elapsed_time(e1)
    d = out[1]
    counts = torch.zeros(d.shape[1] * 64, dtype=torch.float64, device="cuda")
    shifts = torch.arange(64, device="cuda", dtype=torch.int64)
    for s0 in range(0, shots, 131072):
        counts += ((d[s0:s0 + 131072].unsqueeze(-1) >> shifts) & 1).sum(0).reshape(-1).double()
    r_hat = (counts[:ndet] / shots).float()
    _, kind, _ = prog.channels()
    fault = torch.as_tensor(kind != 3, device="cuda")
    base_p = torch.full((prog.num_channels,), 0.5, device="cuda")
    pt_t = torch.as_tensor(pt, dtype=torch.float32, device="cuda")

    def step(q, opt):
        p = base_p.clone()
        p[fault] = torch.exp(q)
        r = (1 - torch.exp(sp.expect(prog, p)[:ndet])) / 2
        loss = ((r - r_hat) ** 2).sum()
        opt.zero_grad()
        loss.backward()
        opt.step()
        return float(loss.detach())

    # untimed warm-up: PyTorch initializes its optimizer machinery on the first step
    qw = torch.log(torch.as_tensor(p0, dtype=torch.float32, device="cuda")).requires_grad_(True)
    step(qw, torch.optim.Adam([qw], lr=0.01))
    q = torch.log(torch.as_tensor(p0, dtype=torch.float32, device="cuda")).requires_grad_(True)
    opt = torch.optim.Adam([q], lr=0.01)
    losses, steps = [], 100
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        losses.append(step(q, opt))
    torch.cuda.synchronize()
    fit_s = time.perf_counter() - t0
    err0 = float((torch.as_tensor(p0, dtype=torch.float32, device="cuda") - pt_t).abs().mean())
    err1 = float((torch.exp(q.detach()) - pt_t).abs().mean())
    prog.close()
    prog_t.close()
    return {"workload": "d=11 r=11, p_i ~ U(5e-4, 2e-3) per channel, target p(1+U(-0.2, 0.2)), 1e6 shots",
            "channels": int(fault.sum()), "detectors": ndet, "sample_ms": sample_ms,
            "adam_steps": steps, "ms_per_step": 1e3 * fit_s / steps, "loss_first": losses[0],
            "loss_last": losses[-1], "mean_abs_p_error_first": err0, "mean_abs_p_error_last": err1}


def run_profile_case():
    """Small case for ncu: build the d=11 program, then sample 65536 shots
    once. The autotuner's timing launches of the fused kernel come first;
    their number is printed so a capture can skip them."""
    import torch
    import paper_2311_03906_gb300 as sp
    from workloads import surface_code
    prog = sp.build(surface_code(WORKLOAD["distance"], WORKLOAD["rounds"], WORKLOAD["p"]))
    i = prog.info
    shots = 65536
    out = prog.alloc_outputs(shots)
    prog.sample(shots, seed=1, out=out)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": WORKLOAD["name"], "shots": shots, "path": i["path"],
                      "fused_tile_shots": i["fused_tile_shots"], "fused_ctas_per_sm": i["fused_ctas_per_sm"],
                      "fused_variant": i["fused_variant"],
                      "autotune_fused_launches": i["autotune_launches"]}))


def run_ours(args):
    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    import paper_2311_03906_gb300 as sp
    from workloads import surface_code

    circuit = surface_code(WORKLOAD["distance"], WORKLOAD["rounds"], WORKLOAD["p"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prog = sp.build(circuit)
    torch.cuda.synchronize()
    build_ms = (time.perf_counter() - t0) * 1e3
    info = prog.info
    shots = args.shots
    out = prog.alloc_outputs(shots)
    stream = torch.cuda.current_stream()
    from paper_2311_03906_gb300.dist import max_over_ranks, shard_range
    steps_total = args.steps + args.warmup + 4

    def step(i):
        prog.sample(shots, seed=1, shot0=shard_range(rank, world, shots, i, steps_total)[0], out=out)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    prog.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
    ev1.record(stream)
    torch.cuda.synchronize()
    prof = prog.profile_read()
    prog.profile(False)
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    if world > 1:
        ms = max_over_ranks(ms, device="cuda")
        torch.distributed.barrier()

    # end to end through the public API with host buffers: D2H of every record
    hout = prog.alloc_outputs(shots, device="cpu", pin_memory=True)
    prog.sample_host(shots, seed=7, shot0=shard_range(rank, world, shots, 0, steps_total)[0], out=hout)  # warm
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for i in range(e2e_steps):
        prog.sample_host(shots, seed=7, shot0=shard_range(rank, world, shots, i, steps_total)[0], out=hout)
    e2e_s = (time.perf_counter() - t1) / e2e_steps
    d2h = sum(t.numel() * 8 for t in hout)

    if rank != 0:
        return
    nrec = info["num_measurements"] + info["num_detectors"] + info["num_observables"]
    value = shots * world * args.steps / (ms / 1e3)
    peaks = _peaks()
    # live per-kernel figures over the timed region
    kern = {}
    total_ms = sum(v[0] for v in prof.values()) or 1.0
    bytes_B = info["num_symbols"] * shots / 8.0
    bytes_rec = nrec * shots / 8.0
    nblocks = -(-info["num_channels"] // 4)
    # Philox4x32-10 per (shot, 4-channel block): 16 of its 20 32x32->64-bit
    # products depend on both the shot and the block (rounds 3-10); round 1's
    # two and round 2's M1 product depend on the shot or the block alone, and
    # round 2's M0 product on the block and the shot's high word (shared by a
    # whole tile). Each product costs two integer-multiply issues (low and
    # high word).
    mul_ops = nblocks * 32.0 * shots
    mul_peak = 152 * 64 * peaks["sm_max_mhz"] * 1e6 / 1e12  # T int32 multiplies/s at max SM clock
    for name, (kms, n) in prof.items():
        if n == 0:
            continue
        avg = kms / n
        d = {"launches": n, "ms_total": kms, "avg_ms": avg, "share": kms / total_ms}
        if name in ("draw", "fused"):
            achieved = mul_ops / (avg / 1e3) / 1e12
            d.update({"bound": "alu", "achieved": achieved, "peak": mul_peak, "unit": "Tmul/s",
                      "frac": achieved / mul_peak})
            if name == "draw":
                d["write_GBs"] = bytes_B / (avg / 1e3) / 1e9
        elif name == "product":
            achieved = (bytes_B + bytes_rec) / (avg / 1e3) / 1e9
            d.update({"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                      "frac": achieved / peaks["hbm_gbs"]})
        elif name == "emit":
            achieved = 2 * bytes_rec / (avg / 1e3) / 1e9
            d.update({"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                      "frac": achieved / peaks["hbm_gbs"]})
        kern[name] = d
    dom = max(kern, key=lambda k: kern[k]["ms_total"]) if kern else None
    roof = None
    if dom:
        k = kern[dom]
        traffic = None
        if dom == "fused":
            traffic = _fused_traffic(shots * args.steps / k["launches"])
        roof = {"kernel": dom, "bound": k.get("bound"), "achieved": k.get("achieved"), "peak": k.get("peak"),
                "unit": k.get("unit"), "frac": k.get("frac"), "traffic": traffic,
                "algorithmic_record_bytes": bytes_rec * args.steps / k["launches"],
                "peak_source": ("152 SMs x 64 int32 multiplies/clk x max SM clock (derived)" if k.get("bound") == "alu"
                                else f"MEASURED_PEAKS.json hbm_gbs ({peaks['source']})")}
    launches = sum(v[1] for v in prof.values())
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD["name"], "shots_per_step": shots, "qubits": info["num_qubits"],
                   "symbols": info["num_symbols"], "channels": info["num_channels"],
                   "measurements": info["num_measurements"], "detectors": info["num_detectors"],
                   "observables": info["num_observables"], "nnz_delta": info["nnz_delta"],
                   "path": {1: "staged-sparse", 2: "dense", 3: "fused", 4: "tensor"}.get(info["path"], "?"),
                   "fused_tile_shots": info["fused_tile_shots"],
                   "fused_variant": info["fused_variant"],
                   "chunk_shots": info["chunk_shots"],
                   "parallelism": f"shot-sharded x{world}" if world > 1 else "single GPU",
                   "l2": "outputs larger than L2: records %.2f GB per step (fault bits %.2f GB, in shared "
                         "memory on the fused path)" % (bytes_rec / 1e9, bytes_B / 1e9)},
        "record_gbit_s": value * nrec / 1e9,
        "build_ms": build_ms,
        "gpu_launches": launches,
        "kernels": kern,
        "roofline": roof,
        "clocks": clk,
        "e2e": {"value": shots * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": d2h},
    }
    if world == 1 and not args.no_batch:
        line["batched"] = _batched_vs_plain(args)
    if world == 1 and not args.no_dense:
        line["dense_rows"] = _dense_paths(args)
    if world == 1 and not args.no_build_times:
        line["build_times"] = _build_times(args)
    if world == 1 and not args.no_fit:
        line["fit"] = _fit(args)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(circuit, budget_s=args.cpu_seconds)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=150)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--shots", type=int, default=SHOTS)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-shots", type=int, default=100_000)
    ap.add_argument("--no-dense", action="store_true", help="skip the dense-row (mirror circuit) section")
    ap.add_argument("--dense-shots", type=int, default=262_144)
    ap.add_argument("--dense-p", type=float, default=0.01, help="noise rate of the dense-row workload")
    ap.add_argument("--no-build-times", action="store_true", help="skip the sampler-initialization timings")
    ap.add_argument("--no-fit", action="store_true", help="skip the noise-model fit (config 5)")
    ap.add_argument("--build-sizes", type=int, nargs="*", default=[100, 200, 300, 500])
    ap.add_argument("--profile", action="store_true",
                    help="build, then one 65536-shot sample only (the case captured by ncu)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.profile:
        run_profile_case()
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
