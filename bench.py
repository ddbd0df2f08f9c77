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
FUSED_TRAFFIC = {"shots": 1_000_000, "bytes": 625_920 + 301_106_944,
                 "sources_sha256": "775fc16de88f41fe111e3ad18a570e608b7c724374a92ddec592856b43a4bd69"}
FUSED_SOURCES = ("paper_2311_03906_gb300/csrc/sp_fused.cu", "paper_2311_03906_gb300/csrc/sp_fused_dev.cuh",
                 "paper_2311_03906_gb300/csrc/sp_internal.h")


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
    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, window=None):
        """Median SM clock and throttle reasons of the samples taken inside
        window = (t0, t1) (host wall-clock seconds), or of all samples."""
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        lines = open(self.path).read().splitlines()
        try:
            os.unlink(self.path)
        except OSError:
            pass
        import datetime
        rows = []
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        inside = [r for r in rows if window and window[0] - 0.02 <= r[0] <= window[1] + 0.02]
        use = inside if inside else rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in use for n, v in zip(names, r[3]) if v.lower() == "active"})
        sm = [r[1] for r in use]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(r[2] for r in use) if use else None,
                "reasons": reasons, "samples": len(sm),
                "scope": "timed region" if inside else "whole sampler run (no sample inside the timed region)"}


def _dist():
    from paper_2311_03906_gb300.dist import world
    return world()


def _oracle_rate(prog, budget_s: float, threads: int, seed: int = 1):
    """Shots/s of the oracle as it stands on `threads` host threads, each
    sampling its own contiguous shot ranges of 64 (the oracle's C calls run
    without the GIL), over about budget_s seconds."""
    import concurrent.futures as cf
    batch = 64

    def worker(t):
        done, k = 0, 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < budget_s:
            prog.sample(seed, (k * threads + t) * batch, batch)
            done += batch
            k += 1
        return done
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        done = sum(ex.map(worker, range(threads)))
    dt = time.perf_counter() - t0
    return done, dt


def _cpu_baseline_child(budget_s: float):
    """Runs in its own process (no CUDA library loaded): the oracle on one
    host thread, then on every host core."""
    import oracle
    from workloads import surface_code
    circuit = surface_code(WORKLOAD["distance"], WORKLOAD["rounds"], WORKLOAD["p"])
    t0 = time.perf_counter()
    prog = oracle.Program(circuit)
    build_s = time.perf_counter() - t0
    n1, dt1 = _oracle_rate(prog, budget_s, 1)
    cores = os.cpu_count() or 1
    nn, dtn = _oracle_rate(prog, max(2.0, budget_s / 2), cores)
    return {"value": n1 / dt1, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{n1} shots of {WORKLOAD['name']} (seed 1), single-threaded plain C oracle, {dt1:.1f} s; "
                      f"oracle build {build_s * 1e3:.0f} ms",
            "all_cores": {"value": nn / dtn, "unit": UNIT, "cores": cores, "kind": "oracle",
                          "sample": f"{nn} shots in 64-shot ranges on {cores} host threads (nproc), {dtn:.1f} s"}}


def _cpu_baseline(budget_s: float = 12.0):
    """The oracle timed in a child process, so that this process maps only
    the CUDA library."""
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-child",
                        "--cpu-seconds", str(budget_s)], capture_output=True, text=True, cwd=ROOT)
    if r.returncode != 0:
        return {"value": None, "unit": UNIT, "cores": 0, "kind": "oracle",
                "sample": "oracle child process failed: " + r.stderr.strip()[-200:]}
    return json.loads(r.stdout.strip().splitlines()[-1])


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


def _mul_roofline(info, shots, avg_ms):
    """Achieved integer multiplies of the fused kernel's Philox draw against
    the multiply pipe: 32 multiply issues per (shot, 4-channel block the draw
    evaluates; blocks whose channels change no record are skipped)."""
    peaks = _peaks()
    nblocks = info["live_blocks"]
    achieved = nblocks * 32.0 * shots / (avg_ms / 1e3) / 1e12
    peak = 152 * 64 * peaks["sm_max_mhz"] * 1e6 / 1e12
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tmul/s", "frac": achieved / peak,
            "peak_source": "152 SMs x 64 int32 multiplies/clk x max SM clock (derived)"}


def _config_section(name, gen, gen_args, shots, chunk, seed, steps):
    """Another configuration of the same step: build, warm up, then `steps`
    timed sp_sample calls of `shots` shots (in chunks of `chunk` shots when
    nonzero) with the per-kernel CUDA-event profile."""
    import torch
    import paper_2311_03906_gb300 as sp
    import workloads
    circuit = getattr(workloads, gen)(*gen_args)
    t0 = time.perf_counter()
    prog = sp.build(circuit)
    build_ms = (time.perf_counter() - t0) * 1e3
    if chunk:
        prog.set_chunk(chunk)
    info = prog.info
    out = prog.alloc_outputs(shots)
    stream = torch.cuda.current_stream()
    for w in range(3):
        prog.sample(shots, seed=seed, shot0=w * shots, out=out)
    torch.cuda.synchronize()
    prog.profile(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(steps):
        prog.sample(shots, seed=seed, shot0=(3 + k) * shots, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = prog.profile_read()
    prog.profile(False)
    ms = e0.elapsed_time(e1) / steps
    nrec = info["num_measurements"] + info["num_detectors"] + info["num_observables"]
    value = shots / (ms / 1e3)
    kern = {k: {"launches_per_step": v[1] / steps, "ms_per_step": v[0] / steps} for k, v in prof.items() if v[1]}
    roof = None
    if "fused" in prof and prof["fused"][1]:
        kms, n = prof["fused"]
        roof = dict(_mul_roofline(info, shots * steps / n, kms / n), kernel="fused")
    prog.close()
    return {"metric": METRIC, "value": value, "unit": UNIT, "ms_per_step": ms, "steps": steps, "warmup": 3,
            "record_gbit_s": value * nrec / 1e9, "build_ms": build_ms, "kernels": kern, "roofline": roof,
            "config": {"workload": name, "shots_per_step": shots, "chunk_shots": info["chunk_shots"],
                       "symbols": info["num_symbols"], "channels": info["num_channels"],
                       "measurements": info["num_measurements"], "detectors": info["num_detectors"],
                       "path": {1: "staged-sparse", 2: "dense", 3: "fused", 4: "tensor"}.get(info["path"], "?"),
                       "fused_tile_shots": info["fused_tile_shots"], "fused_variant": info["fused_variant"]}}


def _grouped_stream(args):
    """The opt-in grouped fault draw (stream 2: a group test per 32 channels,
    then a walk to the first fired channel) on the d=11 and d=17
    configurations: same records' distribution, other bits. Reported with
    its expected Philox blocks per shot (group quads + walks of the groups
    that fire + random-outcome blocks) against the multiply peak, and its
    record bytes against the HBM peak."""
    import torch
    import numpy as np
    import paper_2311_03906_gb300 as sp
    from workloads import surface_code
    peaks = _peaks()
    out = {}
    for name, d, p, shots, chunk in (("surface_code_d11_r11_p1e-3", 11, 1e-3, 1_000_000, 0),
                                     ("surface_code_d17_r17_p2e-3", 17, 2e-3, 1_000_000, 65536)):
        c = surface_code(d, d, p)
        prog = sp.build(c)
        if chunk:
            prog.set_chunk(chunk)
        prog.set_stream(2)
        info = prog.info
        o = prog.alloc_outputs(shots)
        stream = torch.cuda.current_stream()
        for w in range(3):
            prog.sample(shots, seed=1, shot0=w * shots, out=o)
        torch.cuda.synchronize()
        steps = 10
        prog.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(steps):
            prog.sample(shots, seed=1, shot0=(3 + k) * shots, out=o)
        e1.record(stream)
        torch.cuda.synchronize()
        prof = prog.profile_read()
        prog.profile(False)
        ms = e0.elapsed_time(e1) / steps
        kms, kn = prof["fused"]
        avg = kms / kn
        # expected Philox blocks per shot: from the channels' probabilities
        _, kind, _ = prog.channels()
        pf = np.array([op_p for op_p in _fault_probabilities(c)])
        ngrp = -(-len(pf) // 32)
        walks = 0.0
        for g in range(ngrp):
            pg = 1.0 - np.prod(1.0 - pf[32 * g:32 * g + 32])
            walks += pg * -(-len(pf[32 * g:32 * g + 32]) // 4)
        nrnd = int((kind == 3).sum())
        blocks = -(-ngrp // 4) + walks + -(-nrnd // 128)
        mul = blocks * 32.0 * shots * (steps / kn) / (avg / 1e3) / 1e12
        mul_peak = 152 * 64 * peaks["sm_max_mhz"] * 1e6 / 1e12
        nrec = info["num_measurements"] + info["num_detectors"] + info["num_observables"]
        rec_bytes = nrec / 8.0 * shots * (steps / kn)
        out[name] = {"value": shots / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
                     "record_gbit_s": shots / (ms / 1e3) * nrec / 1e9,
                     "philox_blocks_per_shot": blocks,
                     "roofline_multiply": {"achieved": mul, "peak": mul_peak, "unit": "Tmul/s", "frac": mul / mul_peak},
                     "roofline_hbm": {"achieved": rec_bytes / (avg / 1e3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                      "frac": rec_bytes / (avg / 1e3) / 1e9 / peaks["hbm_gbs"]},
                     "fused_tile_shots": info["fused_tile_shots"], "fused_variant": info["fused_variant"]}
        prog.close()
    return out


def _fault_probabilities(circuit):
    """Probability of each channel other than random outcomes, in channel
    order (one per target of a one-qubit noise op, one per pair of
    DEPOLARIZE2)."""
    ps = []
    for op in circuit.ops:
        if op.name in ("X_ERROR", "Y_ERROR", "Z_ERROR", "DEPOLARIZE1"):
            ps += [op.arg] * len(op.targets)
        elif op.name == "DEPOLARIZE2":
            ps += [op.arg] * (len(op.targets) // 2)
    return ps


def _batched_vs_plain(args):
    """64 uneven circuits (rotated surface codes d = 3..15, p in {5e-4, 1e-3,
    2e-3}, seeds 0..63) at several shot counts per circuit: one
    graph-captured batched enqueue vs 64 separate sp_sample calls, identical
    records.  The batch pays off where a single circuit's launch does not
    fill the GPU (few shots per circuit, small codes); at 1e5 shots each
    the separate calls already run several waves per launch."""
    import torch
    import paper_2311_03906_gb300 as sp
    from workloads import batch_suite
    suite = batch_suite(64)
    t0 = time.perf_counter()
    progs = [sp.build(c) for c, _ in suite]
    build_s = time.perf_counter() - t0
    seeds = [s for _, s in suite]
    stream = torch.cuda.current_stream()
    sweep = []
    for nshots in args.batch_shots:
        shots = [nshots] * len(progs)
        outs = [p.alloc_outputs(n) for p, n in zip(progs, shots)]
        outs_plain = [p.alloc_outputs(n) for p, n in zip(progs, shots)]

        def batched():
            sp.sample_batch(progs, seeds, shots, outs=outs)

        def plain():
            for p, s, n, o in zip(progs, seeds, shots, outs_plain):
                p.sample(n, seed=s, out=o)

        res = {"shots_per_circuit": nshots}
        for name, fn in (("batched", batched), ("plain", plain)):
            for _ in range(2):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            reps = 5
            for _ in range(reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            res[name] = {"ms": ms, "shots_per_s": sum(shots) / (ms / 1e3)}
        res["speedup"] = res["plain"]["ms"] / res["batched"]["ms"]
        res["identical"] = all(torch.equal(a, b) for oa, ob in zip(outs, outs_plain) for a, b in zip(oa, ob))
        sweep.append(res)
        del outs, outs_plain
    shapes = {}
    for p in progs:
        k = f"{p.info['fused_tile_shots']}-shot tiles, variant {p.info['fused_variant']}"
        shapes[k] = shapes.get(k, 0) + 1
    config = {"workload": "64 rotated surface codes d=3+2*(i mod 7), p=(5e-4,1e-3,2e-3)[(i//7) mod 3], seed i",
              "build_s": build_s,
              "paths": {"fused": sum(p.info["path"] == 3 for p in progs),
                        "staged": sum(p.info["path"] == 1 for p in progs)},
              "launch_shapes": shapes,
              "identical": "torch.equal of every record tensor, batched vs 64 separate sp_sample calls"}
    for p in progs:
        p.close()
    return {"sweep": sweep, "identical": all(r["identical"] for r in sweep), "config": config}


def _dense_paths(args):
    """A circuit whose coefficient rows are dense (mirror circuit: 512 qubits,
    16 random Clifford layers then their inverse, DEPOLARIZE1(p) after
    every layer, every qubit measured with one detector each; about 33k
    symbols, 1,024 record rows, ~11 % of the coefficients set), over noise
    rates p: the same shots sampled with the product as the tcgen05
    tensor-core contraction, the CUDA-core AND/popcount form and the sparse
    fused kernel, plus the build's own timed choice. The tensor kernel's
    roofline is its FP8 rate (measured bf16 peak x 2, the nominal FP8:BF16
    ratio), counted on the dense contraction (2 rows (n_s+1) FLOP per shot)
    and on the set coefficients only (2 nnz FLOP per shot)."""
    import torch
    import paper_2311_03906_gb300 as sp
    from workloads import mirror_circuit
    peaks = _peaks()
    names = {sp.PATH_TENSOR: "tensor", sp.PATH_DENSE: "dense", sp.PATH_FUSED: "fused", sp.PATH_SPARSE: "staged-sparse"}
    sweep = []
    for p in args.dense_p:
        c = mirror_circuit(512, 16, p=p, seed=1)
        t0 = time.perf_counter()
        prog = sp.build(c)
        build_s = time.perf_counter() - t0
        info = prog.info
        auto = info["path"]
        shots = args.dense_shots
        out = prog.alloc_outputs(shots)
        rows = info["num_measurements"] + info["num_detectors"] + info["num_observables"]
        flops = 2.0 * rows * (info["num_symbols"] + 1) * shots
        flops_set = 2.0 * info["nnz_rows"] * shots
        stream = torch.cuda.current_stream()
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
            sec = t["ms_per_step"] / 1e3
            peak = 2.0 * peaks["bf16_tflops"]
            roof = {"kernel": "k_tc_product", "bound": "tensor", "achieved": flops / sec / 1e12, "peak": peak,
                    "unit": "TFLOP/s", "frac": flops / sec / 1e12 / peak,
                    "achieved_set_coefficients": flops_set / sec / 1e12, "frac_set_coefficients": flops_set / sec / 1e12 / peak,
                    "traffic": None,
                    "peak_source": f"MEASURED_PEAKS.json bf16_tflops x 2 (nominal FP8:BF16 ratio; {peaks['source']})"}
        pp = res["dense"]["kernels"].get("product")
        popc = None
        if pp:
            # one LOP3 (acc ^= a & b) per (record row, 32-position word of b, shot)
            lops = rows * -(-(info["num_symbols"] + 1) // 32) * shots
            achieved = lops / (pp["ms_per_step"] / 1e3) / 1e12
            lpeak = 152 * 64 * peaks["sm_max_mhz"] * 1e6 / 1e12
            popc = {"kernel": "k_popc_product", "bound": "alu", "achieved": achieved, "peak": lpeak,
                    "unit": "T LOP3/s", "frac": achieved / lpeak,
                    "peak_source": "152 SMs x 64 int32 logic ops/clk x max SM clock (derived)"}
        fastest = min(res, key=lambda k: res[k]["ms"])
        sweep.append({"p": p, "symbols": info["num_symbols"], "record_rows": rows, "density": info["density"],
                      "build_s": build_s, "auto_path": names.get(auto, str(auto)), "fastest": fastest,
                      "build_probe_ms": {names[k]: v for k, v in enumerate(info["path_probe_ms"]) if v > 0 and k in names},
                      "paths": res, "tensor_roofline": roof, "popc_roofline": popc, "device_status": status})
        prog.close()
    return {"config": {"workload": "mirror_circuit(n=512, layers=16, p, seed=1)", "shots_per_step": args.dense_shots},
            "sweep": sweep}


def _layered_sampling(args):
    """The paper's first measure (Sec. 5, Fig. 3): the time to generate
    10,000 samples of the random layered circuits, n qubits x n layers, with
    the three noise and entangling settings of Fig. 3a-c (5 CX pairs per
    layer; floor(n/2) pairs; floor(n/2) pairs and DEPOLARIZE1(0.01) on every
    qubit per layer), 5 % of the qubits measured per layer and all at the
    end. Reported per circuit: the product form the build chose and the
    density that decided it, the build time, and the sampling time of 10,000
    shots into device buffers (best of three after a warm-up)."""
    import torch
    import paper_2311_03906_gb300 as sp
    from workloads import random_layered
    names = {sp.PATH_TENSOR: "tensor", sp.PATH_DENSE: "dense", sp.PATH_FUSED: "fused", sp.PATH_SPARSE: "staged-sparse"}
    shots = 10_000
    rows = []
    for panel, kw in (("3a", dict(cnot_pairs=5)), ("3b", dict()), ("3c", dict(depolarize=0.01))):
        for n in args.layered_sizes:
            c = random_layered(n, n, seed=1, **kw)
            t0 = time.perf_counter()
            prog = sp.build(c)
            build_s = time.perf_counter() - t0
            info = prog.info
            out = prog.alloc_outputs(shots)
            prog.sample(shots, seed=1, out=out)
            torch.cuda.synchronize()
            best = 1e30
            for r in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                prog.sample(shots, seed=1, shot0=(r + 1) * shots, out=out)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            nrec = info["num_measurements"] + info["num_detectors"] + info["num_observables"]
            rows.append({"panel": panel, "n": n, "symbols": info["num_symbols"], "measurements": info["num_measurements"],
                         "density": info["density"], "path": names.get(info["path"], str(info["path"])),
                         "build_s": build_s, "sample_ms": best, "shots_per_s": shots / (best / 1e3),
                         "record_gbit_s": nrec * shots / (best / 1e3) / 1e9})
            del out
            prog.close()
    return {"workload": "random_layered(n, n, seed=1): Fig. 3a (5 CX pairs/layer), 3b (floor(n/2) pairs), "
                        "3c (floor(n/2) pairs + DEPOLARIZE1(0.01)); 5 % of qubits measured per layer",
            "shots": shots, "rows": rows}


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


def run_profile_case(case="fused"):
    """Small cases for ncu, each one process:
    - fused: build the d=11 program, then sample 65536 shots once. The
      autotuner's timing launches of the fused kernel come first; their
      number is printed so a capture can skip them.
    - grouped: the same program switched to the grouped draw (stream 2),
      then 65536 shots once; the stream's own autotuner launches come first
      and are printed.
    - dense, tensor: the dense-row mirror circuit (512 qubits, 16 layers,
      p = 0.01), then 32768 shots once on that product form. The build's
      path probe runs each form three times first (draw and product of both
      record kinds per run)."""
    import torch
    import paper_2311_03906_gb300 as sp
    from workloads import mirror_circuit, surface_code
    if case in ("fused", "grouped"):
        prog = sp.build(surface_code(WORKLOAD["distance"], WORKLOAD["rounds"], WORKLOAD["p"]))
        a0 = 0
        if case == "grouped":
            # the grouped stream's autotuner runs at the switch: count only its launches
            a0 = prog.info["autotune_launches"]
            prog.set_stream(2)
        shots = 65536
        name = WORKLOAD["name"]
    else:
        prog = sp.build(mirror_circuit(512, 16, p=0.01, seed=1))
        a0 = 0
        prog.set_path(sp.PATH_DENSE if case == "dense" else sp.PATH_TENSOR)
        shots = 32768
        name = "mirror_circuit(512, 16, p=0.01, seed=1)"
    i = prog.refresh_info()
    out = prog.alloc_outputs(shots)
    prog.sample(shots, seed=1, out=out)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": name, "case": case, "shots": shots, "path": i["path"], "stream": i["stream"],
                      "fused_tile_shots": i["fused_tile_shots"], "fused_ctas_per_sm": i["fused_ctas_per_sm"],
                      "fused_variant": i["fused_variant"],
                      "autotune_fused_launches": i["autotune_launches"] - a0,
                      "device_status": prog.device_status()}))


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

    # the clock sampler starts first, so that it samples from the first timed step on
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    prog.profile(True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    wall0 = time.time()
    ev0.record(stream)
    for i in range(args.steps):
        step(args.warmup + i)
    ev1.record(stream)
    torch.cuda.synchronize()
    wall1 = time.time()
    prof = prog.profile_read()
    prog.profile(False)
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop(window=(wall0, wall1))
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
    nblocks = info["live_blocks"]   # the blocks the draw evaluates (see _mul_roofline)
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
                "d2h_bytes_per_step": d2h,
                "inputs": "a step's inputs are its seed and shot range (16 bytes), passed as kernel launch "
                          "parameters; the program is resident; every record is copied to pinned host memory"},
    }
    if world == 1 and not args.no_c1:
        line["c1"] = _config_section("repetition_code_d5_r5_p0.01", "repetition_code", (5, 5, 0.01), 10_000, 0,
                                     seed=1, steps=20)
    if world == 1 and not args.no_d17:
        line["d17"] = _config_section("surface_code_d17_r17_p2e-3", "surface_code", (17, 17, 2e-3), 1_000_000, 65536,
                                      seed=3, steps=3)
    if world == 1 and not args.no_grouped:
        line["grouped_stream"] = _grouped_stream(args)
    if world == 1 and not args.no_batch:
        line["batched"] = _batched_vs_plain(args)
    if world == 1 and not args.no_dense:
        line["dense_rows"] = _dense_paths(args)
    if world == 1 and not args.no_build_times:
        line["build_times"] = _build_times(args)
    if world == 1 and args.layered_sizes:
        line["layered_sampling"] = _layered_sampling(args)
    if world == 1 and not args.no_fit:
        line["fit"] = _fit(args)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(budget_s=args.cpu_seconds)
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
    ap.add_argument("--batch-shots", type=int, nargs="*", default=[10_000, 100_000])
    ap.add_argument("--no-dense", action="store_true", help="skip the dense-row (mirror circuit) section")
    ap.add_argument("--dense-shots", type=int, default=262_144)
    ap.add_argument("--dense-p", type=float, nargs="*", default=[1e-3, 1e-2, 3e-2, 1e-1],
                    help="noise rates of the dense-row workload")
    ap.add_argument("--no-build-times", action="store_true", help="skip the sampler-initialization timings")
    ap.add_argument("--no-fit", action="store_true", help="skip the noise-model fit (config 5)")
    ap.add_argument("--build-sizes", type=int, nargs="*", default=[100, 200, 300, 500])
    ap.add_argument("--layered-sizes", type=int, nargs="*", default=[100, 500, 1000],
                    help="n of the random layered circuits sampled for the paper's Fig. 3 measure (none: skip)")
    ap.add_argument("--cpu-baseline-child", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-d17", action="store_true", help="skip the d=17 configuration")
    ap.add_argument("--no-c1", action="store_true", help="skip the repetition-code configuration")
    ap.add_argument("--no-grouped", action="store_true", help="skip the grouped fault-draw stream")
    ap.add_argument("--profile", action="store_true",
                    help="build, then one small sample only (the case captured by ncu)")
    ap.add_argument("--profile-case", default="fused", choices=["fused", "grouped", "dense", "tensor"],
                    help="which small case --profile runs")
    args = ap.parse_args()
    if args.cpu_baseline_child:
        print(json.dumps(_cpu_baseline_child(args.cpu_seconds)), flush=True)
    elif args.impl == "reference":
        run_reference(args)
    elif args.profile:
        run_profile_case(args.profile_case)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
