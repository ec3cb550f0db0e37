#!/usr/bin/env python3
"""Benchmark: SHA3-256 over 2^24 messages of 64 bytes on one GB300 (Mhash/s).

One step = one call of keccak_batch_uniform (the fixed-stride batch mode of
the paper's Section 4: one thread per message, same-length messages) over
2^24 seeded random 64-byte messages already resident in HBM.  The inputs
(1 GiB) are larger than L2, so no flush is needed between steps.

Printed (rank 0, one JSON line): the headline Mhash/s, the ALU roofline of the
hashing kernel, an end-to-end figure through keccak_batch_uniform_host (host
buffers, copies inside the timed region), SM clocks sampled during the timed
region, and the CPU oracle timed on a bounded sample of the same messages.

``--impl reference`` times the CPU oracle alone on the same workload and
metric (there is no other implementation of the paper's method to run).

Multi-GPU (torchrun): every rank hashes its own 2^24 messages (weak scaling,
no collective on the data path); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
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

N_MSGS = 1 << 24
MSG_BYTES = 64
DIGEST = 32
VARIANT = 1  # SHA3-256
WORKLOAD = "sha3_256_2p24_msgs_x_64B"
METRIC = "SHA3-256 Mhash/s (64 B msgs)"

# Algorithmic 32-bit integer operations of one Keccak-f[1600] permutation in
# the bit-interleaved form: per round theta 20 (parities) + 5 (rotate) + 50
# (apply), rho 47, chi 50, plus iota's non-zero halves (derived below).
ROUND_OPS_NO_IOTA = 20 + 5 + 50 + 47 + 50

# SMs x 32-bit integer lanes per SM per clock x maximum SM clock: the ALU
# issue roofline.  LOP3 and SHF run on the ALU pipe, which takes one warp
# instruction per SM sub-partition every two cycles (ncu's pipe counters on
# the hashing kernel), i.e. 16 lanes per sub-partition and 64 per SM.
SM_COUNT_GB300 = 152
INT_LANES_PER_SM_CLK = 64
SM_MAX_MHZ = 2070.0


def _interleaved_nonzero_halves() -> int:
    """Number of non-zero 32-bit halves among the 24 round constants."""
    from paper_1902_05320_gb300 import binding

    total = 0
    for rc in binding.round_constants():
        e = sum(((rc >> (2 * k)) & 1) << k for k in range(32))
        o = sum(((rc >> (2 * k + 1)) & 1) << k for k in range(32))
        total += (e != 0) + (o != 0)
    return total


def ops_per_permutation() -> int:
    return 24 * ROUND_OPS_NO_IOTA + _interleaved_nonzero_halves()


# ---------------------------------------------------------------------------
# Replicas: every rank hashes its own messages (seeded by rank), the step time
# is the slowest rank's, and the value counts the messages of all ranks.
def rank_seed(base: int, rank: int) -> int:
    return base + rank


def max_over_ranks(ms: float, world: int) -> float:
    """The slowest rank's time (a collective on timing only, never on data)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mhash_s(n_per_rank: int, world: int, ms: float) -> float:
    return world * n_per_rank / (ms / 1e3) / 1e6


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.device_index = device_index
        self.samples = []
        self.proc = None
        self.marks = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.device_index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.monotonic(), line.strip()))

    def mark(self):
        self.marks.append(time.monotonic())

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        t0, t1 = (self.marks + [0, 0])[:2] if len(self.marks) >= 2 else (0, 1e30)
        inside = [s for t, s in self.samples if t0 - 0.15 <= t <= t1 + 0.15] or [s for _, s in self.samples]
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for s in inside:
            parts = [p.strip() for p in s.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(inside)}


# ---------------------------------------------------------------------------
def cpu_baseline(msgs: np.ndarray, seconds: float = 8.0) -> dict:
    """The CPU oracle, as it stands, on a bounded sample of the messages."""
    import oracle

    oracle.build()
    cores = len(os.sched_getaffinity(0))

    def run(k, threads):
        offs = np.arange(k, dtype=np.uint64) * np.uint64(MSG_BYTES)
        t = time.perf_counter()
        oracle.hash_batch(msgs[: k * MSG_BYTES], offs, np.full(k, MSG_BYTES, np.uint64),
                          np.full(k, VARIANT, np.uint8), np.full(k, DIGEST, np.uint32), threads)
        return time.perf_counter() - t

    k0 = 64 * cores
    dt0 = run(k0, cores)
    k = int(min(N_MSGS, max(k0, k0 * seconds / max(dt0, 1e-6))))
    dt = run(k, cores)
    # The same on one host thread, for a per-core figure (a shorter sample).
    k1 = max(64, k // (4 * cores))
    dt1 = run(k1, 1)
    return {"value": k / dt / 1e6, "unit": "Mhash/s", "cores": cores, "kind": "oracle",
            "sample": f"first {k} of the 2^24 64-byte messages, SHA3-256, {dt:.1f} s on {cores} host threads",
            "single_core_value": k1 / dt1 / 1e6,
            "single_core_sample": f"first {k1} of the same messages, {dt1:.1f} s on 1 host thread"}


def run_reference(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1902_05320_gb300 import workloads

    import oracle

    oracle.build()
    cores = len(os.sched_getaffinity(0))
    msgs = workloads.uniform_messages(N_MSGS, MSG_BYTES, seed=1)
    # Each step hashes a bounded sample sized so the whole run takes ~2 minutes.
    probe = 64 * cores
    offs = np.arange(probe, dtype=np.uint64) * np.uint64(MSG_BYTES)
    t = time.perf_counter()
    oracle.hash_batch(msgs[: probe * MSG_BYTES], offs, np.full(probe, MSG_BYTES, np.uint64),
                      np.full(probe, VARIANT, np.uint8), np.full(probe, DIGEST, np.uint32), cores)
    rate = probe / (time.perf_counter() - t)
    per_step = int(max(probe, min(N_MSGS, rate * 100.0 / max(1, args.steps + args.warmup))))
    offs = np.arange(per_step, dtype=np.uint64) * np.uint64(MSG_BYTES)
    lens = np.full(per_step, MSG_BYTES, np.uint64)
    var = np.full(per_step, VARIANT, np.uint8)
    ol = np.full(per_step, DIGEST, np.uint32)
    sample = msgs[: per_step * MSG_BYTES]
    for _ in range(args.warmup):
        oracle.hash_batch(sample, offs, lens, var, ol, cores)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.hash_batch(sample, offs, lens, var, ol, cores)
    dt = (time.perf_counter() - t) / max(1, args.steps)
    value = per_step / dt / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mhash/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_per_step": per_step,
                   "note": "CPU oracle (bit-level FIPS 202 restatement) on host cores; bounded sample per step"},
        "cpu_baseline": {"value": value, "unit": "Mhash/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {per_step} of the 2^24 64-byte messages per step"},
        "e2e": {"value": value, "unit": "Mhash/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--messages", type=int, default=N_MSGS,
                    help="messages per step (default 2^24; smaller only for profiling captures)")
    ap.add_argument("--serving-only", type=float, default=0.0, metavar="SECONDS",
                    help="only run the serving measurement for SECONDS of arrivals")
    ap.add_argument("--merkle-only", type=int, default=0, metavar="LEAVES",
                    help="only run the Merkle measurement on LEAVES 8 KiB leaves (profiling captures)")
    ap.add_argument("--ragged-only", type=int, default=0, metavar="N",
                    help="only run the ragged-batch measurement on N messages (profiling captures)")
    ap.add_argument("--keccak-p-only", default="", metavar="B,NR,N",
                    help="only time Keccak-p[B, NR] on N raw states (profiling captures)")
    ap.add_argument("--next-only", action="store_true",
                    help="only run the streaming, many-tree, message-tree and Keccak-p measurements")
    ap.add_argument("--config", type=int, default=0, choices=sorted(CONFIG_WORKLOADS),
                    help="only run the measurement of one workload: " +
                         "; ".join(f"{k}: {v}" for k, v in CONFIG_WORKLOADS.items()))
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
        return

    import torch
    import torch.distributed as dist

    from paper_1902_05320_gb300 import binding, build, workloads

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    binding.load()
    if args.serving_only:
        print(json.dumps(serving_measurements(workloads, torch, rank, seconds=args.serving_only)), flush=True)
        return
    if args.merkle_only:
        print(json.dumps(merkle_measurements(binding, workloads, torch, torch.cuda.current_stream(), rank,
                                             n_leaves=args.merkle_only)), flush=True)
        return
    if args.ragged_only:
        print(json.dumps(ragged_measurements(binding, workloads, torch, torch.cuda.current_stream(), rank,
                                             n=args.ragged_only, autotune=False)), flush=True)
        return
    if args.config:
        print(json.dumps(config_measurement(args.config, binding, workloads, torch, rank)), flush=True)
        return
    if args.keccak_p_only:
        print(json.dumps(keccak_p_measurement(binding, workloads, torch, rank, args.keccak_p_only)), flush=True)
        return
    if args.next_only:
        print(json.dumps(next_rows_measurements(binding, workloads, torch, torch.cuda.current_stream(), rank)),
              flush=True)
        return

    n_msgs = args.messages
    msgs_np = workloads.uniform_messages(n_msgs, MSG_BYTES, seed=rank_seed(1, rank))
    msgs = torch.from_numpy(msgs_np).cuda()
    digests = torch.empty(n_msgs * DIGEST, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        binding.keccak_batch_uniform(msgs, MSG_BYTES, MSG_BYTES, VARIANT, DIGEST, digests, n_msgs, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # Spot check before timing: a few digests against hashlib.
    got = digests[: 4 * DIGEST].cpu().numpy().reshape(4, DIGEST)
    for i in range(4):
        want = hashlib.sha3_256(msgs_np[i * MSG_BYTES:(i + 1) * MSG_BYTES].tobytes()).digest()
        if got[i].tobytes() != want:
            raise SystemExit(f"digest mismatch at message {i}")

    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    # One event between consecutive steps: the first and last bracket the
    # whole timed region, the others give each step's own time.
    marks = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    sampler.mark()
    marks[0].record(stream)
    for k in range(args.steps):
        step()
        marks[k + 1].record(stream)
    torch.cuda.synchronize()
    sampler.mark()
    if world > 1:
        dist.barrier()
    ms = marks[0].elapsed_time(marks[-1]) / args.steps
    per_step = sorted(marks[k].elapsed_time(marks[k + 1]) for k in range(args.steps))
    time.sleep(0.2)
    sampler.stop()
    ms = max_over_ranks(ms, world)
    clocks = sampler.summary()

    value = whole_job_mhash_s(n_msgs, world, ms)
    ops_perm = ops_per_permutation()
    achieved = n_msgs * ops_perm / (ms / 1e3) / 1e12
    peak = SM_COUNT_GB300 * INT_LANES_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12
    traffic = measured_traffic()

    # End to end through the host-buffer entry point (copies in the timed region).
    e2e = None
    if not args.no_e2e:
        e2e = e2e_measurements(binding, torch, stream, msgs_np, digests, n_msgs, world, args.steps)

    with_oracle = rank == 0 and not args.no_cpu_baseline
    extra = {} if args.no_extra else extra_measurements(binding, workloads, torch, stream, msgs, rank, with_oracle)
    del msgs, digests

    line = {
        "metric": METRIC, "value": value, "unit": "Mhash/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms,
        "ms_per_step_best": per_step[0], "ms_per_step_median": per_step[len(per_step) // 2],
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD if n_msgs == N_MSGS else f"sha3_256_{n_msgs}_msgs_x_64B",
                   "messages_per_gpu": n_msgs, "msg_bytes": MSG_BYTES,
                   "variant": "SHA3-256", "entry_point": "keccak_batch_uniform",
                   "l2": "inputs (1 GiB per step) larger than L2; no flush", "parallelism": f"replicas{world}"},
        "gb_per_s": world * n_msgs * MSG_BYTES / (ms / 1e3) / 1e9,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "ops_per_hash": ops_perm,
                     "peak_basis": f"{SM_COUNT_GB300} SMs x {INT_LANES_PER_SM_CLK} int32 lanes/clk x "
                                   f"{SM_MAX_MHZ:.0f} MHz max SM clock",
                     "kernel": "k_sha3_uniform64_tma<SHA3-256> (64-byte messages staged by bulk copies)"},
        "e2e": e2e,
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    if extra:
        line["extra"] = extra
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(msgs_np[: min(n_msgs, N_MSGS) * MSG_BYTES])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def extra_measurements(binding, workloads, torch, stream, msgs, rank, with_oracle=False) -> dict:
    """Secondary figures: the rest of the fixed-length family, then the other
    workloads (not the headline), each with the CPU oracle timed beside it on
    a bounded sample when with_oracle is set."""
    out = fixed_length_measurements(binding, workloads, torch, stream, msgs, rank, with_oracle)
    out["small_batches"] = small_batch_measurements(binding, workloads, torch, stream, rank, with_oracle)
    out["ragged_2p20_loguniform_0_64KiB"] = ragged_measurements(binding, workloads, torch, stream, rank,
                                                                with_oracle=with_oracle)
    out["serving_poisson_200k_rps_10s"] = serving_measurements(workloads, torch, rank, with_oracle=with_oracle)
    out["merkle_4GiB_8KiB_leaves"] = merkle_measurements(binding, workloads, torch, stream, rank,
                                                         with_oracle=with_oracle)
    out["next_rows"] = next_rows_measurements(binding, workloads, torch, stream, rank)
    try:
        out["int_lanes_per_sm_clk"] = {name: round(binding.int_issue_probe(op, 4096, stream), 2)
                                       for op, name in enumerate(("lop3_chi", "shf_reg", "prmt_reg", "iadd3"))}
    except Exception as e:  # diagnostic only
        out["int_lanes_per_sm_clk"] = f"probe failed: {e}"
    return out


# ---------------------------------------------------------------------------
def oracle_sample(oracle, msgs, offsets, lens, variants, out_lens, perms, seconds, seed, cores=None):
    """The CPU oracle on a seeded random sample of a batch, sized to about
    `seconds` of work on the host's cores: returns (sample size, its
    permutations, elapsed seconds, cores)."""
    cores = cores or len(os.sched_getaffinity(0))
    n = len(offsets)
    rng = np.random.default_rng(seed)
    order = rng.permutation(n)
    k = min(n, 64 * cores)
    while True:
        idx = np.sort(order[:k])
        t = time.perf_counter()
        oracle.hash_batch(msgs, offsets[idx], lens[idx], variants[idx], out_lens[idx], cores)
        dt = time.perf_counter() - t
        if dt >= 0.25 * seconds or k >= n:
            return k, int(perms[idx].sum()), dt, cores
        k = min(n, int(k * min(8.0, max(2.0, seconds / max(dt, 1e-3)))))


def oracle_entry(k, n, sample_perms, total_perms, dt, cores, what, unit_rate=None):
    """An oracle sub-entry: the sample's own rate, and the whole workload's
    time extrapolated by permutation count (stated as such)."""
    full_s = dt * total_perms / max(sample_perms, 1)
    e = {"kind": "oracle", "cores": cores, "sample": f"{k} of {n} {what} (seeded random), {dt:.2f} s",
         "mperm_s": sample_perms / dt / 1e6, "full_ms_extrapolated": full_s * 1e3,
         "extrapolation": "sample time x (workload permutations / sample permutations)"}
    if unit_rate is not None:
        e.update(unit_rate(k, dt))
    return e


def e2e_measurements(binding, torch, stream, msgs_np, digests, n_msgs, world, steps) -> dict:
    """The headline workload end to end through keccak_batch_uniform_host on
    page-locked buffers placed on the GPU's NUMA node, with the host link's
    copy rates, the buffers' NUMA node and this process's CPUs in the same
    run, so that the figure can be read against the link that bounds it."""
    h_in, h_out = binding.HostBuffer(n_msgs * MSG_BYTES), binding.HostBuffer(n_msgs * DIGEST)
    h_in.array[:] = msgs_np
    probe_dev = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    link = {}
    for mode, name in ((0, "copy_engine_h2d_gb_s"), (1, "copy_engine_d2h_gb_s"), (2, "copy_engine_both_ways_gb_s"),
                       (3, "sm_loads_h2d_gb_s")):
        try:
            link[name] = round(binding.host_link_probe(h_in, probe_dev, 256 << 20, mode, 8, stream), 1)
        except Exception as e:  # diagnostic only
            link[name] = f"probe failed: {e}"
    del probe_dev
    # Up to 40 calls per path (~0.25 s each): one slow call then moves the mean
    # by a few percent rather than by half.
    reps = max(10, min(2 * steps, 40))

    per_call = {}

    def timed(path, name):
        # Each call is synchronous (it returns with the digests in host
        # memory); the rate is the mean over the calls, and each call's time
        # is kept so that a stall of the host shows as itself.
        binding.keccak_tune_set(binding.KB_TUNE_HOST_PATH, path)
        try:
            binding.keccak_batch_uniform_host(h_in, MSG_BYTES, MSG_BYTES, VARIANT, DIGEST, h_out, n_msgs, stream)
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                t = time.perf_counter()
                binding.keccak_batch_uniform_host(h_in, MSG_BYTES, MSG_BYTES, VARIANT, DIGEST, h_out, n_msgs, stream)
                ts.append(time.perf_counter() - t)
            per_call[name] = {"min": round(min(ts) * 1e3, 3), "median": round(statistics.median(ts) * 1e3, 3),
                              "max": round(max(ts) * 1e3, 3), "calls": reps}
            return sum(ts) / reps
        finally:
            binding.keccak_tune_set(binding.KB_TUNE_HOST_PATH, binding.KB_HOST_PATH_AUTO)

    s_staged = timed(binding.KB_HOST_PATH_STAGED, "staged")
    s_in_place = timed(binding.KB_HOST_PATH_ZERO_COPY, "in_place")
    # The default: the first call of this size class decides by a trial.
    s_auto = timed(binding.KB_HOST_PATH_AUTO, "default")
    chosen = binding.keccak_host_path_for(n_msgs)
    if not np.array_equal(h_out.array[: 1 << 20], digests[: 1 << 20].cpu().numpy()):
        raise SystemExit("host-buffer path disagrees with the device path")
    nodes = numa_nodes_of_cpus(sorted(os.sched_getaffinity(0)))
    in_b, out_b = n_msgs * MSG_BYTES, n_msgs * DIGEST
    res = {"value": world * n_msgs / s_auto / 1e6, "unit": "Mhash/s", "h2d_bytes_per_step": in_b,
           "d2h_bytes_per_step": out_b,
           "entry_point": "keccak_batch_uniform_host (KB_HOST_PATH_AUTO; buffers from keccak_host_alloc)",
           "host_path_chosen": {binding.KB_HOST_PATH_STAGED: "staged", binding.KB_HOST_PATH_ZERO_COPY: "in_place"}.get(
               chosen, str(chosen)),
           "staged_mhash_s": n_msgs / s_staged / 1e6, "in_place_mhash_s": n_msgs / s_in_place / 1e6,
           "ms_per_call": per_call,
           "link": link,
           "link_bound_mhash_s": None,
           "buffers_numa_node": {"messages": h_in.numa_node(), "digests": h_out.numa_node()},
           "process_cpus": compact_ranges(sorted(os.sched_getaffinity(0))), "process_cpus_numa_nodes": nodes}
    # The link bound: every step moves in_b bytes in and out_b bytes out.
    # While both directions run they share the link (each at half the
    # measured two-way rate); the direction with more bytes then finishes
    # alone at its one-way rate.  No schedule of the copies is shorter.
    res["link_bound_mhash_s"] = link_bound_mhash_s(link, in_b, out_b, n_msgs)
    h_in.free()
    h_out.free()
    return res


def link_bound_mhash_s(link, in_b, out_b, n_msgs):
    """Hashes per second the host link allows when every step moves in_b bytes
    to the device and out_b bytes back (both directions overlapped as far as
    the link lets them), from the link rates measured in the same run."""
    both, h2d, d2h = (link.get(k) for k in ("copy_engine_both_ways_gb_s", "copy_engine_h2d_gb_s",
                                             "copy_engine_d2h_gb_s"))
    if not all(isinstance(x, float) and x > 0 for x in (both, h2d, d2h)):
        return None
    each = both / 2 * 1e9  # per direction while both run
    shared = min(in_b, out_b)
    rest_rate = (h2d if in_b >= out_b else d2h) * 1e9
    seconds = shared / each + (max(in_b, out_b) - shared) / rest_rate
    return n_msgs / seconds / 1e6


def compact_ranges(xs) -> str:
    out, start, prev = [], None, None
    for x in xs:
        if start is None:
            start = prev = x
        elif x == prev + 1:
            prev = x
        else:
            out.append(f"{start}-{prev}" if start != prev else str(start))
            start = prev = x
    if start is not None:
        out.append(f"{start}-{prev}" if start != prev else str(start))
    return ",".join(out)


def numa_nodes_of_cpus(cpus) -> list:
    nodes = set()
    base = "/sys/devices/system/node"
    try:
        for d in os.listdir(base):
            if not d.startswith("node"):
                continue
            with open(os.path.join(base, d, "cpulist")) as f:
                text = f.read().strip()
            mine = set()
            for part in text.split(","):
                if "-" in part:
                    a, b = part.split("-")
                    mine.update(range(int(a), int(b) + 1))
                elif part:
                    mine.add(int(part))
            if mine & set(cpus):
                nodes.add(int(d[4:]))
    except OSError:
        return []
    return sorted(nodes)


def alu_frac(perms, ms) -> float:
    """Fraction of the integer-ALU roofline: permutations x the algorithmic ops
    of one permutation, per second, over the ALU peak."""
    peak = SM_COUNT_GB300 * INT_LANES_PER_SM_CLK * SM_MAX_MHZ * 1e6
    return perms * ops_per_permutation() / (ms / 1e3) / peak


def uniform_oracle(torch, d_msgs, n, length, variant, out_len, seconds, seed, perms_per_msg):
    """The oracle on a seeded random sample of a fixed-length batch resident on
    the device (only the sampled messages are copied back)."""
    import oracle

    oracle.build()
    rng = np.random.default_rng(seed)
    cores = len(os.sched_getaffinity(0))
    k = 64 * cores
    while True:
        idx = np.sort(rng.choice(n, min(k, n), replace=False))
        sample = d_msgs.view(n, length)[torch.from_numpy(idx).cuda()].cpu().numpy().reshape(-1)
        offs = np.arange(idx.size, dtype=np.uint64) * np.uint64(length)
        t = time.perf_counter()
        oracle.hash_batch(sample, offs, np.full(idx.size, length, np.uint64), np.full(idx.size, variant, np.uint8),
                          np.full(idx.size, out_len, np.uint32), cores)
        dt = time.perf_counter() - t
        if dt >= 0.25 * seconds or idx.size >= n:
            break
        k = int(k * min(8.0, max(2.0, seconds / max(dt, 1e-3))))
    return {"kind": "oracle", "cores": cores, "mhash_s": idx.size / dt / 1e6,
            "sample": f"{idx.size} of {n} messages (seeded random), {dt:.2f} s on {cores} host threads",
            "full_ms_extrapolated": dt * n / idx.size * 1e3,
            "extrapolation": "sample time x (messages / sample messages)",
            "mperm_s": idx.size * perms_per_msg / dt / 1e6}


def fixed_length_measurements(binding, workloads, torch, stream, msgs, rank, with_oracle=False) -> dict:
    """2^24 x 64 B with the two state-layout and staging controls and with
    SHA3-512, and 2^22 x 1 KiB SHA3-256."""
    out = {}
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        a, b = ev(), ev()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    n = msgs.numel() // MSG_BYTES
    controls = {}
    # The bit-interleaved state layout, the measured control for the default.
    d32 = torch.empty(n * 32, dtype=torch.uint8, device="cuda")
    binding.keccak_tune_set(binding.KB_TUNE_REPRESENTATION, binding.KB_REP_INTERLEAVED)
    try:
        ms = timed(lambda: binding.keccak_batch_uniform(msgs, 64, 64, 1, 32, d32, n, stream))
    finally:
        binding.keccak_tune_set(binding.KB_TUNE_REPRESENTATION, binding.KB_REP_PLAIN)
    controls["interleaved_state_mhash_s"] = n / ms / 1e3
    # Each thread loading its own message, against the default bulk-copy staging.
    binding.keccak_tune_set(binding.KB_TUNE_STAGING, binding.KB_STAGING_DIRECT)
    try:
        ms = timed(lambda: binding.keccak_batch_uniform(msgs, 64, 64, 1, 32, d32, n, stream))
    finally:
        binding.keccak_tune_set(binding.KB_TUNE_STAGING, binding.KB_STAGING_TMA)
    controls["direct_load_mhash_s"] = n / ms / 1e3
    out["controls_sha3_256_2p24_x_64B"] = controls
    del d32
    d64 = torch.empty(n * 64, dtype=torch.uint8, device="cuda")
    ms = timed(lambda: binding.keccak_batch_uniform(msgs, 64, 64, 3, 64, d64, n, stream))
    out["sha3_512_2p24_x_64B"] = {"ms": ms, "mhash_s": n / ms / 1e3, "alu_frac": alu_frac(n, ms)}
    if with_oracle:
        out["sha3_512_2p24_x_64B"]["oracle"] = uniform_oracle(torch, msgs, n, 64, 3, 64, 3.0, 11, 1)
    del d64
    n2, l2 = 1 << 22, 1024
    m2 = torch.from_numpy(workloads.uniform_messages(n2, l2, seed=2 + rank)).cuda()
    d2 = torch.empty(n2 * 32, dtype=torch.uint8, device="cuda")
    ms = timed(lambda: binding.keccak_batch_uniform(m2, l2, l2, 1, 32, d2, n2, stream))
    perms2 = n2 * (l2 // 136 + 1)
    out["sha3_256_2p22_x_1KiB"] = {"ms": ms, "mhash_s": n2 / ms / 1e3, "gb_s": n2 * l2 / ms / 1e6,
                                   "alu_frac": alu_frac(perms2, ms)}
    if with_oracle:
        out["sha3_256_2p22_x_1KiB"]["oracle"] = uniform_oracle(torch, m2, n2, l2, 1, 32, 3.0, 12, l2 // 136 + 1)
    del m2, d2
    return out


CONFIG_WORKLOADS = {
    1: "4096 x 64 B SHA3-256, one launch (and 119,040 x 10 B, the paper's largest batch)",
    2: "2^24 x 64 B SHA3-256 and SHA3-512, 2^22 x 1 KiB SHA3-256",
    3: "2^20 ragged messages, lengths log-uniform 0..64 KiB, six functions mixed",
    4: "Merkle root of 4 GiB in 8 KiB leaves",
    5: "serving: Poisson arrivals at 200k requests/s for 10 s, 32 B..1 MiB, 2 GiB HBM budget",
}


def config_measurement(config, binding, workloads, torch, rank) -> dict:
    """One workload's measurement on its own (bench.py --config N)."""
    stream = torch.cuda.current_stream()
    if config == 1:
        res = small_batch_measurements(binding, workloads, torch, stream, rank)
    elif config == 2:
        msgs = torch.from_numpy(workloads.uniform_messages(N_MSGS, MSG_BYTES, seed=rank_seed(1, rank))).cuda()
        d = torch.empty(N_MSGS * DIGEST, dtype=torch.uint8, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(3):
            binding.keccak_batch_uniform(msgs, MSG_BYTES, MSG_BYTES, VARIANT, DIGEST, d, N_MSGS, stream)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(10):
            binding.keccak_batch_uniform(msgs, MSG_BYTES, MSG_BYTES, VARIANT, DIGEST, d, N_MSGS, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        del d
        res = {"sha3_256_2p24_x_64B_mhash_s": N_MSGS / (e0.elapsed_time(e1) / 10) / 1e3}
        res.update(fixed_length_measurements(binding, workloads, torch, stream, msgs, rank))
    elif config == 3:
        res = ragged_measurements(binding, workloads, torch, stream, rank)
    elif config == 4:
        res = merkle_measurements(binding, workloads, torch, stream, rank)
    else:
        res = serving_measurements(workloads, torch, rank)
    return {"config": config, "workload": CONFIG_WORKLOADS[config], "result": res}


RATES = (144, 136, 104, 72, 168, 136)


def ragged_measurements(binding, workloads, torch, stream, rank, n=1 << 20, autotune=True, with_oracle=False) -> dict:
    """The ragged, mixed-variant batch: 2^20 messages, lengths log-uniform over
    0..64 KiB, variants uniform over the six functions, SHAKE outputs 16..512 B.
    Input-order single launch vs the cost-bucketed persistent queue (graph
    replay), then the queue with the autotuned configuration."""
    b = workloads.ragged_batch(n, seed=3 + rank, max_len=65536)
    rates = np.array(RATES, dtype=np.uint64)[b.variants]
    perms = (b.lens // rates + 1 + np.where(b.out_lens > rates, (b.out_lens.astype(np.uint64) - 1) // rates, 0))
    total_perms = int(perms.sum())
    to_dev = lambda a: torch.from_numpy(a.view({8: np.int64, 4: np.int32, 1: np.uint8}[a.itemsize])).cuda()  # noqa
    d = [to_dev(x) for x in (b.msgs, b.offsets, b.lens, b.variants, b.out_lens)]
    out = torch.empty(b.total_out(), dtype=torch.uint8, device="cuda")
    msg_bytes = int(b.lens.sum())

    def timed(reps=3):
        binding.keccak_batch(*d, out, b.n, stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            binding.keccak_batch(*d, out, b.n, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    res = {"messages": b.n, "message_bytes": msg_bytes, "permutations": total_perms}
    saved = [binding.keccak_tune_get(k) for k in range(binding.KB_TUNE_KEYS)]
    try:
        binding.keccak_tune_set(binding.KB_TUNE_RAGGED_SCHEDULE, binding.KB_SCHEDULE_INPUT_ORDER)
        ms_in = timed()
        ref = out.clone()
        binding.keccak_tune_set(binding.KB_TUNE_RAGGED_SCHEDULE, binding.KB_SCHEDULE_PER_VARIANT)
        ms_pv = timed()
        same = bool(torch.equal(ref, out))
        binding.keccak_tune_set(binding.KB_TUNE_RAGGED_SCHEDULE, binding.KB_SCHEDULE_QUEUE)
        ms_q = timed()
        same = same and bool(torch.equal(ref, out))
        tuned, ms_t = None, None
        if autotune:
            tuned = binding.keccak_batch_autotune(*d, out, b.n, stream)
            ms_t = timed()
            same = same and bool(torch.equal(ref, out))
    finally:
        for k, v in enumerate(saved):
            binding.keccak_tune_set(k, v)
    for name, ms in (("input_order", ms_in), ("per_variant_launches", ms_pv), ("queue", ms_q),
                     ("queue_autotuned", ms_t)):
        if ms is None:
            continue
        res[name] = {"ms": ms, "mhash_s": b.n / ms / 1e3, "gb_s": msg_bytes / ms / 1e6,
                     "gperm_s": total_perms / ms / 1e6, "alu_frac": alu_frac(total_perms, ms)}
    res["autotuned_config"] = tuned
    res["schedules_agree_bytewise"] = same
    if with_oracle:
        import oracle

        oracle.build()
        k, kp, dt, cores = oracle_sample(oracle, b.msgs, b.offsets, b.lens, b.variants, b.out_lens, perms, 5.0, 31)
        res["oracle"] = oracle_entry(k, b.n, kp, total_perms, dt, cores, "messages")
    return res


def next_rows_measurements(binding, workloads, torch, stream, rank) -> dict:
    """The rows beyond the batch hash: streaming sponge states absorbing in
    pieces, many small Merkle trees, the tree of one long message, and the bare
    permutation Keccak-p[b, n_r] on raw states.  Each against the integer-ALU
    roofline where its work is whole Keccak-f[1600] permutations."""
    peak = SM_COUNT_GB300 * INT_LANES_PER_SM_CLK * SM_MAX_MHZ * 1e6 / 1e12
    ops = ops_per_permutation()

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def rates(ms, perms, data_bytes):
        return {"ms": ms, "gperm_s": perms / ms / 1e6, "gb_s": data_bytes / ms / 1e6,
                "alu_frac": perms * ops / (ms / 1e3) / 1e12 / peak}

    dev = lambda *shape, dtype=torch.uint8: torch.empty(*shape, dtype=dtype, device="cuda")  # noqa: E731
    res = {}
    # Streaming: 2^20 SHA3-256 states, init, four absorbs of 2 KiB (not a
    # multiple of the rate, so every call leaves pending bytes), final.
    n, piece, k = 1 << 20, 2048, 4
    buf = torch.from_numpy(workloads.random_bytes(n * piece, seed=rank_seed(20, rank))).cuda()
    offs = torch.arange(n, dtype=torch.int64, device="cuda") * piece
    lens = torch.full((n,), piece, dtype=torch.int64, device="cuda")
    states = dev(n * binding.KB_STATE_BYTES)
    variants = torch.full((n,), 1, dtype=torch.uint8, device="cuda")
    out_lens = torch.full((n,), 32, dtype=torch.int32, device="cuda")
    dig = dev(n * 32)

    def stream_run():
        # k pieces in k calls: the first fused with the initialisation, the
        # last with the padding and squeeze.
        binding.keccak_stream_init_absorb(states, variants, buf, offs, lens, n, stream)
        for _ in range(k - 2):
            binding.keccak_stream_absorb(states, buf, offs, lens, n, stream)
        binding.keccak_stream_absorb_final(states, buf, offs, lens, out_lens, dig, n, stream)

    def stream_run_separate():
        binding.keccak_stream_init(states, variants, n, stream)
        for _ in range(k):
            binding.keccak_stream_absorb(states, buf, offs, lens, n, stream)
        binding.keccak_stream_final(states, out_lens, dig, n, stream)

    ms = timed(stream_run)
    res["stream_2p20_states_4x2KiB_sha3_256"] = rates(ms, n * (k * piece // 136 + 1), n * k * piece)
    res["stream_2p20_states_4x2KiB_sha3_256"]["separate_init_final_ms"] = timed(stream_run_separate)
    # The same 8 KiB per message in one call, for comparison.
    one = dev(n * 8192)
    for j in range(k):
        one.view(n, 8192)[:, j * piece:(j + 1) * piece] = buf.view(n, piece)
    ms1 = timed(lambda: binding.keccak_batch_uniform(one, 8192, 8192, 1, 32, dig, n, stream))
    res["stream_2p20_states_4x2KiB_sha3_256"]["one_call_ms"] = ms1
    del buf, offs, lens, states, variants, out_lens, dig, one
    torch.cuda.empty_cache()
    # Many small trees: 2^18 trees of 16 leaves of 256 B (one thread per tree,
    # 3.4 waves of threads on the GPU).
    nt, lpt, lb = 1 << 18, 16, 256
    tb = torch.from_numpy(workloads.random_bytes(nt * lpt * lb, seed=rank_seed(21, rank))).cuda()
    roots = dev(nt * 32)
    ms = timed(lambda: binding.merkle_sha3_256_many(tb, nt, lpt, lb, roots, stream))
    perms = nt * (lpt * ((1 + lb) // 136 + 1) + (lpt - 1))
    res["merkle_many_2p18_trees_x16_x256B"] = rates(ms, perms, nt * lpt * lb)
    del tb, roots
    torch.cuda.empty_cache()
    # The tree of one 1 GiB message in 8 KiB chunks.
    length, chunk = 1 << 30, 8192
    mb = torch.from_numpy(workloads.random_bytes(length, seed=rank_seed(22, rank))).cuda()
    ms = timed(lambda: binding.merkle_sha3_256_message(mb, length, chunk, stream), reps=3)
    leaves = length // chunk
    res["merkle_message_1GiB_8KiB_chunks"] = rates(ms, leaves * ((1 + chunk) // 136 + 1) + leaves - 1, length)
    del mb
    torch.cuda.empty_cache()
    # The bare permutation on 2^24 raw 200-byte states.
    ns = 1 << 24
    st = torch.from_numpy(workloads.random_bytes(ns * 200, seed=rank_seed(23, rank))).cuda().view(torch.int64)
    for b, nr in ((1600, 24), (1600, 12), (200, 18)):
        ms = timed(lambda: binding.keccak_p_batch(st, b, nr, ns, stream))
        r = {"ms": ms, "gstates_s": ns / ms / 1e6, "hbm_gb_s": ns * 400 / ms / 1e6}
        if b == 1600 and nr == 24:
            r["alu_frac"] = ns * ops / (ms / 1e3) / 1e12 / peak
        res[f"keccak_p_{b}_{nr}_2p24_states"] = r
    del st
    torch.cuda.empty_cache()
    return res


def small_batch_measurements(binding, workloads, torch, stream, rank, with_oracle=False) -> dict:
    """Latency-bound single launches: 4096 x 64 B SHA3-256, and the paper's
    own workload shape (119,040 messages of 10 bytes, the largest point of its
    Table 3; the paper does not name the variant, SHA3-256 here).  The oracle
    hashes each whole batch."""
    res = {}
    for name, n, length in (("sha3_256_4096_x_64B", 4096, 64), ("sha3_256_119040_x_10B", 119040, 10)):
        m_np = workloads.uniform_messages(n, length, seed=10 + rank)
        m = torch.from_numpy(m_np).cuda()
        d = torch.empty(n * 32, dtype=torch.uint8, device="cuda")
        for _ in range(3):
            binding.keccak_batch_uniform(m, length, length, 1, 32, d, n, stream)
        torch.cuda.synchronize()
        reps = 50
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            binding.keccak_batch_uniform(m, length, length, 1, 32, d, n, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) / reps * 1e3
        res[name] = {"us_per_launch": us, "mhash_s": n / us, "gb_s": n * length / us / 1e3,
                     "alu_frac": alu_frac(n, us / 1e3)}
        if with_oracle:
            import oracle

            oracle.build()
            cores = len(os.sched_getaffinity(0))
            offs = np.arange(n, dtype=np.uint64) * np.uint64(length)
            t = time.perf_counter()
            oracle.hash_batch(m_np, offs, np.full(n, length, np.uint64), np.full(n, 1, np.uint8),
                              np.full(n, 32, np.uint32), cores)
            dt = time.perf_counter() - t
            res[name]["oracle"] = {"kind": "oracle", "cores": cores, "mhash_s": n / dt / 1e6,
                                   "us_per_batch": dt * 1e6, "sample": f"the whole batch of {n}, {dt:.2f} s"}
    return res


def merkle_measurements(binding, workloads, torch, stream, rank, n_leaves=1 << 19, leaf_bytes=8192,
                        with_oracle=False) -> dict:
    """Tree mode: 4 GiB of random bytes in 8 KiB leaves up to the root."""
    buf_np = workloads.merkle_buffer(n_leaves, leaf_bytes, seed=4 + rank)
    buf = torch.from_numpy(buf_np).cuda()
    nodes = torch.empty(32 * binding.merkle_node_count(n_leaves), dtype=torch.uint8, device="cuda")

    def run():
        binding.merkle_sha3_256_levels(buf, n_leaves, leaf_bytes, nodes, stream)

    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record(stream)
    for _ in range(reps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    leaf_perms = (leaf_bytes + 1) // 136 + 1
    perms = n_leaves * leaf_perms + (binding.merkle_node_count(n_leaves) - n_leaves)
    t = time.perf_counter()
    root = binding.merkle_sha3_256(buf, n_leaves, leaf_bytes, stream)
    root_ms = (time.perf_counter() - t) * 1e3
    hbm_bytes = n_leaves * leaf_bytes + 32 * binding.merkle_node_count(n_leaves) * 2
    res = {"leaves": n_leaves, "leaf_bytes": leaf_bytes, "ms": ms, "root_call_ms": root_ms,
           "gb_s": n_leaves * leaf_bytes / ms / 1e6, "gperm_s": perms / ms / 1e6,
           "alu_frac": alu_frac(perms, ms), "bound": "alu",
           "hbm_frac_of_measured": hbm_bytes / ms / 1e6 / measured_hbm_gbs(), "root": root.hex()}
    del buf, nodes
    torch.cuda.empty_cache()
    if with_oracle:
        import oracle

        oracle.build()
        # Leaf digests of a seeded sample of leaves (each leaf prefixed 0x00, as
        # the tree rules have it), the tree's time extrapolated by permutations.
        rng = np.random.default_rng(41)
        cores = len(os.sched_getaffinity(0))
        k = 16 * cores
        while True:
            idx = np.sort(rng.choice(n_leaves, min(k, n_leaves), replace=False))
            sample = np.zeros((idx.size, leaf_bytes + 1), np.uint8)
            sample[:, 1:] = buf_np.reshape(n_leaves, leaf_bytes)[idx]
            offs = np.arange(idx.size, dtype=np.uint64) * np.uint64(leaf_bytes + 1)
            t = time.perf_counter()
            oracle.hash_batch(sample.reshape(-1), offs, np.full(idx.size, leaf_bytes + 1, np.uint64),
                              np.full(idx.size, 1, np.uint8), np.full(idx.size, 32, np.uint32), cores)
            dt = time.perf_counter() - t
            if dt >= 1.0 or idx.size >= n_leaves:
                break
            k = int(k * min(8.0, max(2.0, 4.0 / max(dt, 1e-3))))
        res["oracle"] = oracle_entry(idx.size, n_leaves, idx.size * leaf_perms, perms, dt, cores,
                                     "leaves hashed (0x00 || leaf)")
    return res


def measured_hbm_gbs() -> float:
    """The measured copy bandwidth of this machine's GPUs when the driver's peaks
    file is present, else the figure measured on an earlier GB300 run."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6699.8


def serving_measurements(workloads, torch, rank, rate=200_000, seconds=10.0, with_oracle=False) -> dict:
    """The serving loop: Poisson arrivals at `rate` requests/s for `seconds`,
    messages log-uniform 32 B..1 MiB from a 4 GiB pinned pool, variants mixed,
    admitted against a 2 GiB device budget, 48 batches in flight per lane."""
    from paper_1902_05320_gb300.serve import Server

    from paper_1902_05320_gb300 import binding

    wl = workloads.serving_workload(rate, seconds, seed=5 + rank, pool_bytes=4 << 30)
    # The message pool and the outputs in page-locked memory on the GPU's NUMA
    # node (the gather kernel reads the pool over the host link).
    pool = binding.HostBuffer(wl.pool.size)
    pool.array[:] = wl.pool
    total = int(wl.out_lens.sum(dtype=np.uint64))
    outputs = binding.HostBuffer(max(total, 1))
    lat = np.zeros(wl.n, dtype=np.int64)
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    time.sleep(0.3)
    # 48 batches in flight per lane: a long-lane stream stays busy until the
    # slowest chain of its batch ends (measured p99: 16 per lane 31.7-108 ms,
    # 32 per lane 24.1-24.2 ms with one run in seven at 35.9 ms, 48 per lane
    # 23.6-23.7 ms in five runs out of five).
    with Server(hbm_budget_bytes=2 << 30, max_inflight=48, max_batch_requests=4096) as srv:
        sampler.mark()
        st = srv.replay(pool, wl.offsets, wl.lens, wl.variants, wl.out_lens, wl.arrival_ns, outputs, lat)
        sampler.mark()
    sampler.stop()
    pool_node, out_node = pool.numa_node(), outputs.numa_node()
    pool.free()
    outputs.free()
    offered_bytes = int(wl.lens.sum())
    big = wl.lens >= (512 << 10)
    res = {"requests": wl.n, "offered_rps": rate, "offered_gb_s": offered_bytes / seconds / 1e9,
           "throughput_rps": st["throughput_rps"], "throughput_gb_s": st["throughput_gbs"],
           "p50_us": st["lat_p50_us"], "p90_us": st["lat_p90_us"], "p99_us": st["lat_p99_us"],
           "p999_us": st["lat_p999_us"], "max_us": st["lat_max_us"], "mean_us": st["lat_mean_us"],
           "batches": st["batches"], "max_batch_requests_seen": st["max_batch_requests_seen"],
           "peak_arena_bytes": st["peak_arena_bytes"], "per_request_completion": bool(st["completion_ring"]),
           "p50_us_small_lt_4KiB": float(np.percentile(lat[wl.lens < 4096], 50) / 1e3),
           "p99_us_small_lt_4KiB": float(np.percentile(lat[wl.lens < 4096], 99) / 1e3),
           "p50_us_large_ge_512KiB": float(np.percentile(lat[big], 50) / 1e3) if big.any() else None,
           "latency_parts_us": {k: st[k] for k in ("submit_lag_p50_us", "submit_lag_p99_us", "queue_wait_p50_us",
                                                    "queue_wait_p99_us", "service_p50_us", "service_p99_us")},
           "pool_numa_node": pool_node, "outputs_numa_node": out_node, "clocks": sampler.summary()}
    if with_oracle:
        import oracle

        oracle.build()
        rates = np.array(RATES, dtype=np.uint64)[wl.variants]
        perms = (wl.lens // rates + 1 + np.where(wl.out_lens > rates, (wl.out_lens.astype(np.uint64) - 1) // rates, 0))
        k, kp, dt, cores = oracle_sample(oracle, wl.pool, wl.offsets, wl.lens, wl.variants, wl.out_lens, perms, 8.0, 51)
        e = oracle_entry(k, wl.n, kp, int(perms.sum()), dt, cores, "requests")
        # Requests per second the oracle sustains on this mix (by permutations).
        e["capacity_rps_extrapolated"] = wl.n / (e["full_ms_extrapolated"] / 1e3)
        res["oracle"] = e
    return res


def keccak_p_measurement(binding, workloads, torch, rank, spec: str) -> dict:
    """Keccak-p[b, n_r] in place on n random 200-byte states: the median of
    five launches after three warm-up launches."""
    b, nr, n = (int(x) for x in spec.split(","))
    st = torch.from_numpy(workloads.random_bytes(n * 200, seed=rank_seed(23, rank))).cuda().view(torch.int64)
    stream = torch.cuda.current_stream()
    for _ in range(3):
        binding.keccak_p_batch(st, b, nr, n, stream)
    ts = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        binding.keccak_p_batch(st, b, nr, n, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = statistics.median(ts)
    return {"b": b, "nr": nr, "states": n, "ms": ms, "gstates_s": n / ms / 1e6, "hbm_gb_s": n * 400 / ms / 1e6}


def measured_traffic():
    """DRAM bytes per launch of the hashing kernel from the committed ncu
    summary, or None when the kernel sources changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "k_sha3_uniform_sha3_256_64B.md")
    if not os.path.exists(path):
        return None
    fields = {}
    for ln in open(path):
        if ":" in ln and ln.startswith("- "):
            k, v = ln[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    try:
        bytes_per_launch = float(fields["dram_bytes_per_launch_full_size"])
        recorded = fields["csrc_sha256"]
    except (KeyError, ValueError):
        return None
    return bytes_per_launch if recorded == csrc_digest() else None


def csrc_digest() -> str:
    """Hash of the headline kernel's sources with comments and blank space
    removed, so that only changes to the code itself invalidate the profile."""
    import re

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1902_05320_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name in ("keccak_core.cuh", "keccak_interleaved.cuh", "sponge.cuh", "sha3_uniform.cu", "runtime.cuh",
                    "tma.cuh"):
            text = open(os.path.join(csrc, name), encoding="utf-8").read()
            text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
            text = re.sub(r"//[^\n]*", " ", text)
            h.update(name.encode())
            h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


if __name__ == "__main__":
    main()
