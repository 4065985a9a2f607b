#!/usr/bin/env python3
"""Benchmark of the PYRIT GB300 coding path.

Default workload (one JSON line): GF(2^10) (w=10, n=11, all-one modulus), Cauchy code k=10, m=4,
packets of 64 KiB (blocks of 640 KiB), 256 stripes of seeded uniform random bytes. One step =
encode every stripe, then decode every stripe with its own seeded random pattern of 1..4 erased
blocks (rebuilt in place), each as one persistent batched launch replayed from a CUDA graph.

  value    source GB/s (10^9 B/s): 2 x stripes x k x w x P bytes (encode + decode) per step time,
           inputs resident in HBM (2.19 GiB of stripes, larger than L2; no flush needed).
  e2e      the same metric with the data blocks uploaded from pinned host memory and the parity
           read back every step (chunked over streams so copies overlap the kernels).
  roofline for each timed kernel (the encode and the decode launch), its algorithmic bytes
           ((k+m)wP per encoded stripe, (k+e)wP per decoded stripe with e erasures) per launch over
           its event-timed duration, against the measured HBM copy bandwidth; the headline object
           is the kernel with the larger share of the step.
  served   (sub-object) a 2 s Poisson window at 20k requests/s of GF(2^12) k=16 m=4 requests
           (packets 4 KiB-1 MiB, half 4-erasure decodes): p50/p99/p99.9 latency and sustained GB/s
           with continuous batching, and the same arrivals served one request per launch (two
           passes per arm, alternating).
  mixed    (sub-object) 4096 uneven stripes in one batched launch per ring size against 4096
           per-stripe launches of the same kernel: GB/s, roofline fraction, speed-up.
  sweep32k (sub-object) the 32 KiB point of the GF(2^12) k=16 m=4 packet-size sweep (~8 GiB of
           source): encode and 4-erasure decode roofline fractions.

`--impl reference` times the CPU oracle (the plain log/antilog coder) on a bounded sample of the
same workload. Multi-GPU (torchrun): every rank codes its own 256 stripes (weak scaling, no
collective on the data path); the step time is the maximum over ranks.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

W, N, K, M, P, STRIPES = 10, 11, 10, 4, 64 * 1024, 256
CONFIG = {"workload": "GF(2^10) AOP ring n=11, Cauchy k=10 m=4, 64 KiB packets, 256 stripes; "
                      "encode + decode with 1-4 random erasures per stripe",
          "w": W, "n": N, "k": K, "m": M, "packet_bytes": P, "stripes": STRIPES,
          "l2": "inputs larger than L2 (2.19 GiB of stripes per GPU), no flush"}
METRIC = "encode+decode GB/s of source data"
FALLBACK_PEAK = 6800.0


def peak_hbm():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_PEAK, "fallback"


# Library sources that do not shape the batched coding kernels: the server, the allocation-free
# entry point, single calls and the synthetic-data fill.
NOT_KERNEL_SOURCES = ("server.cpp", "noalloc.cu", "capi.cu", "synth.cu")


def kernel_source_digest():
    """Digest of the sources that define the batched coding kernels, their generated networks and
    their launch shapes (the device code, the network generator, the planner's masks, the batch
    and launch logic and the tuner)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1709_00178_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h", ".inc", ".cpp")) and name not in NOT_KERNEL_SOURCES:
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(name.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "coding_kernels_config2_traffic.json")


def recorded_traffic():
    """DRAM bytes per launch of the timed encode and decode kernels ({"encode": B, "decode": B})
    from the committed ncu record, if the kernel sources have not changed since it was taken."""
    try:
        with open(TRAFFIC_RECORD) as f:
            rec = json.load(f)
    except Exception:
        return {}
    if rec.get("kernel_src_digest") != kernel_source_digest():
        return {}
    return rec.get("traffic_bytes_per_launch", {})


def kernel_name(shape):
    """Name of the kernel a batch group launches, as ncu lists it."""
    if shape["dispatch"] == 3:
        return "ring_staged_net (%s network, words %d, %d consumer warps)" % (
            ("syndrome-decode" if shape["mode"] in (1, 3) else "direct") +
            (", parity transform" if shape["mode"] in (2, 3) else ""), shape["words"], shape["nc"])
    return "ring_staged_kernel<%d, %d, %d, %d, %d, %d>" % (shape["n"], shape["words"], shape["mg"], shape["minb"],
                                                          shape["dispatch"], shape["nc"])


def make_plan(pyrit, generator, w, k, m, transform="embedding"):
    """The library plan of a code: the plain Cauchy generator, or the weight-optimised generalized
    Cauchy one (the oracle legs compute their own copy; a CPU test pins the two equal), under the
    embedding or the parity transform (Sec. 2.3)."""
    n = 9 if w == 6 else w + 1  # GF(2^6) from x^6 + x^3 + 1 lives in R_{2,9}; the others in R_{2,w+1}
    if generator == "weighted":
        G, _ = pyrit.pyrit_generator_weighted(w, n, k, m)
        plan = pyrit.pyrit_plan_create(w, n, k, m, G)
    else:
        plan = pyrit.pyrit_plan_create(w, n, k, m)
    if transform == "parity":
        pyrit.pyrit_plan_set_transform(plan, pyrit.PYRIT_TRANSFORM_PARITY)
    return plan


def oracle_codec(transform):
    """The oracle's (encode, decode) pair for a transform."""
    import oracle
    return (oracle.encode_pt, oracle.decode_pt) if transform == "parity" else (oracle.encode, oracle.decode)


def rank_shard(rank, stripe_bytes, stripes):
    """What rank `rank` codes (weak scaling, no data-path collective): its stripes' bytes are the
    synthetic stream's bytes [rank * S * B, (rank + 1) * S * B) and its erasure patterns come from
    their own seed. Returns (stream offset, pattern seed)."""
    from paper_1709_00178_gb300.synth import BASE_SEED
    return rank * stripes * stripe_bytes, BASE_SEED + 1 + 1000 * rank


def max_over_ranks(value, world, dist, device):
    """The maximum of a per-rank float over all ranks (the job is as slow as its slowest rank)."""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(world, src_bytes_per_rank_step, ms_per_step):
    """Whole-job throughput: every rank's source bytes per step over the slowest rank's step time."""
    return world * src_bytes_per_rank_step / (ms_per_step * 1e-3) / 1e9


def patterns(seed, stripes, k, m):
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(stripes):
        e = int(rng.integers(1, m + 1))
        out.append(sum(1 << int(x) for x in rng.choice(k + m, e, replace=False)))
    return out


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = "/tmp/pyrit_clocks_%d.csv" % os.getpid()

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def run_reference(args):
    """The CPU oracle timed as the reference arm, on a bounded sample of the workload."""
    import numpy as np
    import oracle
    from paper_1709_00178_gb300.synth import BASE_SEED, synth_bytes
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    sample = 4  # stripes encoded and decoded per step
    G = oracle.cauchy_weighted(W, K, M)[0] if args.generator == "weighted" else oracle.cauchy(W, K, M)
    pats = patterns(BASE_SEED + 1, STRIPES, K, M)
    blk = W * P
    # the same bytes as the GPU arm's first stripes: data blocks are contiguous in the stream
    data = [synth_bytes(BASE_SEED + 1, s * K * blk, K * blk).reshape(K, W, P) for s in range(sample)]

    o_enc, o_dec = oracle_codec(args.transform)
    CONFIG["generator"] = "plain Cauchy" if args.generator == "cauchy" else "weight-optimised generalized Cauchy"
    CONFIG["transform"] = "phi_E (embedding)" if args.transform == "embedding" else "phi_P (parity bit)"

    def step():
        for s in range(sample):
            par = o_enc(W, K, M, G, data[s], nthreads=cores)
            full = np.concatenate([data[s], par])
            o_dec(W, K, M, G, full, pats[s], nthreads=cores)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    gbs = 2 * sample * K * blk / dt / 1e9
    desc = "%d stripes of the workload encoded and decoded per step on %d threads" % (sample, cores)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic", "config": CONFIG,
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def main():
    global STRIPES
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--stripes", type=int, default=STRIPES,
                    help="stripes per GPU (default 256; smaller values make profiling cases)")
    ap.add_argument("--workload", default="coding", choices=["coding", "sweep", "mixed", "served", "gf16", "transforms", "paper", "fields"],
                    help="coding: the default line; sweep: GF(2^12) k=16 m=4 packet sweep 4 KiB-1 MiB; mixed: "
                         "4096 uneven stripes batched vs per-stripe launches; served: Poisson arrivals; gf16: "
                         "GF(16) k=4 m=2, one stripe, encode + every erasure pattern (L2-resident); transforms: "
                         "embedding vs parity transform on k >= m and k < m codes; paper: the paper's (12,8), (60,40) and "
                         "(60,20) use cases across block sizes; fields: GF(16) and GF(8) from other factors of x^n+1")
    ap.add_argument("--seconds", type=float, default=10.0, help="served: arrival window")
    ap.add_argument("--rate", type=float, default=20000.0, help="served: Poisson arrival rate (requests/s)")
    ap.add_argument("--slots", type=int, default=16, help="served: stream slots of the batching server")
    ap.add_argument("--packet", type=int, default=0,
                    help="sweep: one packet size in bytes instead of 4 KiB..1 MiB (with --stripes: a profiling case)")
    ap.add_argument("--generator", default="cauchy", choices=["cauchy", "weighted"],
                    help="cauchy: the plain Cauchy code of the configurations; weighted: the same code "
                         "family with weight-optimised row/column scalings (generalized Cauchy)")
    ap.add_argument("--transform", default="embedding", choices=["embedding", "parity"],
                    help="embedding: phi_E (the configurations' transform, k >= m); parity: phi_P, the "
                         "parity-bit transform (Sec. 2.3.1), a different code of the same parameters")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner: time the automatic shapes (profiling cases of a fixed kernel)")
    ap.add_argument("--no-extras", action="store_true",
                    help="default line without its served / mixed / sweep32k sub-objects (profiling runs)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "coding":
        return {"sweep": run_sweep, "mixed": run_mixed, "served": run_served, "gf16": run_gf16,
                "transforms": run_transforms, "paper": run_paper, "fields": run_fields}[args.workload](args)
    if args.stripes != STRIPES:
        STRIPES = max(8, args.stripes // 8 * 8)
        CONFIG["stripes"] = STRIPES
        CONFIG["workload"] = CONFIG["workload"].replace("256 stripes", "%d stripes" % STRIPES)
        CONFIG["l2"] = "%.2f GiB of stripes per GPU" % (STRIPES * (K + M) * W * P / 2 ** 30)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1709_00178_gb300 import pyrit
    from paper_1709_00178_gb300.synth import BASE_SEED

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)

    blk = W * P
    stripe_bytes = (K + M) * blk
    # Layout: every stripe's k data blocks contiguous in a data region, its m parity blocks in a
    # parity region, so host<->device transfers of a run of stripes are single copies.
    buf = torch.empty(STRIPES * stripe_bytes, dtype=torch.uint8, device=dev)
    shard_off, pat_seed = rank_shard(rank, stripe_bytes, STRIPES)
    pyrit.pyrit_synth_fill(buf.data_ptr(), buf.numel(), BASE_SEED + 1, shard_off)
    torch.cuda.synchronize(dev)
    base = buf.data_ptr()
    par0 = STRIPES * K * blk
    blocks = [[base + (s * K + j) * blk for j in range(K)] + [base + par0 + (s * M + i) * blk for i in range(M)]
              for s in range(STRIPES)]
    pats = patterns(pat_seed, STRIPES, K, M)
    plan = make_plan(pyrit, args.generator, W, K, M, args.transform)
    CONFIG["generator"] = "plain Cauchy" if args.generator == "cauchy" else "weight-optimised generalized Cauchy"
    CONFIG["transform"] = "phi_E (embedding)" if args.transform == "embedding" else "phi_P (parity bit)"
    enc = pyrit.pyrit_batch_create([(plan, pyrit.PYRIT_OP_ENCODE, 0, P, blocks[s]) for s in range(STRIPES)])
    dec = pyrit.pyrit_batch_create([(plan, pyrit.PYRIT_OP_DECODE, pats[s], P, blocks[s]) for s in range(STRIPES)])
    es, ds = pyrit.pyrit_batch_stats(enc), pyrit.pyrit_batch_stats(dec)
    launches_per_step = es["launches"] + ds["launches"]
    stream = torch.cuda.Stream(device=dev)
    # The library's autotuner times every kernel variant (and generated network shape) on these
    # batches and keeps the fastest.
    if not args.no_tune:
        pyrit.pyrit_batch_tune(enc, stream, 6)
        pyrit.pyrit_batch_tune(dec, stream, 6)

    def step(evs=None):
        if evs is not None:
            evs[0].record(stream)
        pyrit.pyrit_batch_run(enc, stream, graph=True)
        if evs is not None:
            evs[1].record(stream)
        pyrit.pyrit_batch_run(dec, stream, graph=True)
        if evs is not None:
            evs[2].record(stream)

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    nvtx = torch.cuda.nvtx
    code, where = pyrit.pyrit_device_status()
    if code != 0:
        raise RuntimeError("device status %d at site %d after warm-up" % (code, where))

    # ---- device-resident timed region ----
    # Clocks are sampled from one second before the timed steps (the GPU kept busy with untimed
    # steps meanwhile) until after them.
    clocks = Clocks(local)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    t_pre = time.perf_counter()
    while time.perf_counter() - t_pre < 1.0:
        for _ in range(20):
            step()
        torch.cuda.synchronize(dev)
    barrier()
    torch.cuda.synchronize(dev)
    nvtx.range_push("timed")
    t0.record(stream)
    for i in range(args.steps):
        step(evs[i])
    t1.record(stream)
    torch.cuda.synchronize(dev)
    nvtx.range_pop()
    clk = clocks.stop()
    barrier()
    ms = max_over_ranks(t0.elapsed_time(t1), world, dist, dev)
    ms_step = ms / args.steps
    src_per_step = es["src_bytes"] + ds["src_bytes"]
    value = whole_job_gbs(world, src_per_step, ms_step)
    enc_ms = sum(e[0].elapsed_time(e[1]) for e in evs) / args.steps
    dec_ms = sum(e[1].elapsed_time(e[2]) for e in evs) / args.steps
    peak, peak_kind = peak_hbm()
    traffic = recorded_traffic()
    kernels = []
    for role, batch, st_, kms in (("encode", enc, es, enc_ms), ("decode", dec, ds, dec_ms)):
        ach = st_["alg_bytes"] / (kms * 1e-3) / 1e9
        kernels.append({"role": role, "kernel": kernel_name(pyrit.pyrit_batch_shape(batch, 0)), "ms": kms,
                        "alg_bytes_per_launch": st_["alg_bytes"], "achieved": ach, "frac": ach / peak,
                        "traffic": traffic.get(role)})
    dominant = max(kernels, key=lambda kk: kk["ms"])
    code, where = pyrit.pyrit_device_status()
    if code != 0:
        raise RuntimeError("device status %d at site %d" % (code, where))

    # ---- end to end: data from pinned host memory, parity back, every step ----
    CH = 16  # chunks of stripes; chunk c's data and parity are each one contiguous copy
    per = STRIPES // CH
    host = torch.empty(STRIPES * K * blk, dtype=torch.uint8, pin_memory=True)
    host.copy_(buf[:par0])
    host_par = torch.empty(STRIPES * M * blk, dtype=torch.uint8, pin_memory=True)
    cenc = [pyrit.pyrit_batch_create([(plan, 0, 0, P, blocks[s]) for s in range(c * per, (c + 1) * per)])
            for c in range(CH)]
    # The blocks each decode rebuilds (its erased ones) go to one contiguous device buffer, in stripe
    # order (the decode writes each erased block wherever its pointer says), so that every chunk's
    # rebuilt blocks come back to pinned host memory in one copy.
    lost = [(s, e) for s in range(STRIPES) for e in range(K + M) if (pats[s] >> e) & 1]
    rebuilt_dev = torch.empty(len(lost) * blk, dtype=torch.uint8, device=dev)
    host_rebuilt = torch.empty(len(lost) * blk, dtype=torch.uint8, pin_memory=True)
    slot_of = {se: i for i, se in enumerate(lost)}
    dec_blocks = [[rebuilt_dev.data_ptr() + slot_of[(s, e)] * blk if (s, e) in slot_of else blocks[s][e]
                   for e in range(K + M)] for s in range(STRIPES)]
    cdec = [pyrit.pyrit_batch_create([(plan, 1, pats[s], P, dec_blocks[s]) for s in range(c * per, (c + 1) * per)])
            for c in range(CH)]
    chunk_lost = [(min((i for i, (s, e) in enumerate(lost) if s >= c * per), default=len(lost)),
                   min((i for i, (s, e) in enumerate(lost) if s >= (c + 1) * per), default=len(lost)))
                  for c in range(CH)]
    streams = [torch.cuda.Stream(device=dev) for _ in range(4)]
    dev_block = lambda s, e: buf[s * K * blk + e * blk:s * K * blk + (e + 1) * blk] if e < K else \
        buf[par0 + (s * M + e - K) * blk:par0 + (s * M + e - K + 1) * blk]

    def e2e_step():
        for c in range(CH):
            st = streams[c % len(streams)]
            d0, d1 = c * per * K * blk, (c + 1) * per * K * blk
            p0, p1 = c * per * M * blk, (c + 1) * per * M * blk
            with torch.cuda.stream(st):
                buf[d0:d1].copy_(host[d0:d1], non_blocking=True)
                pyrit.pyrit_batch_run(cenc[c], st, graph=True)
                pyrit.pyrit_batch_run(cdec[c], st, graph=True)
                host_par[p0:p1].copy_(buf[par0 + p0:par0 + p1], non_blocking=True)
                r0, r1 = chunk_lost[c][0] * blk, chunk_lost[c][1] * blk
                if r1 > r0:
                    host_rebuilt[r0:r1].copy_(rebuilt_dev[r0:r1], non_blocking=True)

    def e2e_timed(steps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        main = torch.cuda.current_stream(dev)
        a.record(main)
        for st in streams:
            st.wait_event(a)
        for _ in range(steps):
            e2e_step()
        for st in streams:
            main.wait_stream(st)
        b.record(main)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b)

    e2e_timed(2)
    barrier()
    nvtx.range_push("e2e")
    e2e_ms = e2e_timed(args.steps)
    nvtx.range_pop()
    e2e_ms = max_over_ranks(e2e_ms, world, dist, dev)
    e2e_val = whole_job_gbs(world, src_per_step, e2e_ms / args.steps)
    # every parity block read back must equal the device-resident result, and every rebuilt block
    # the block it rebuilt (still in place in the device-resident stripes)
    e2e_ok = bool(torch.equal(buf[par0:].cpu(), host_par))
    e2e_rebuilt_ok = all(bool(torch.equal(host_rebuilt[i * blk:(i + 1) * blk], dev_block(s, e).cpu()))
                         for i, (s, e) in enumerate(lost))

    out = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u8", "data": "synthetic (seeded SplitMix64 bytes)", "config": CONFIG,
        "e2e": {"value": e2e_val, "unit": "GB/s", "h2d_bytes_per_step": STRIPES * K * blk,
                "d2h_bytes_per_step": STRIPES * M * blk + len(lost) * blk, "parity_readback_matches": e2e_ok,
                "rebuilt_readback_matches": e2e_rebuilt_ok,
                "what": "per step: the data blocks uploaded from pinned host memory, encode, decode (the erased "
                        "blocks rebuilt into one device buffer per chunk), the parity blocks and every rebuilt "
                        "block read back to pinned host memory; 16 chunks over 4 streams"},
        "gpu_launches": launches_per_step * args.steps,
        "roofline": {"bound": "hbm", "achieved": dominant["achieved"], "peak": peak, "unit": "GB/s",
                     "frac": dominant["frac"], "traffic": dominant["traffic"],
                     "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind if peak_kind == "measured"
                     else "fallback 6800 GB/s",
                     "kernel": dominant["kernel"], "role": dominant["role"],
                     "alg_bytes_per_launch": dominant["alg_bytes_per_launch"], "kernels": kernels,
                     "step_frac": (es["alg_bytes"] + ds["alg_bytes"]) / ((enc_ms + dec_ms) * 1e-3) / 1e9 / peak},
        "clocks": clk,
    }

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(buf, blocks, pats, plan, pyrit, args.generator, args.transform)
    for b in [enc, dec] + cenc + cdec:
        pyrit.pyrit_batch_destroy(b)
    del buf, host, host_par, host_rebuilt, rebuilt_dev
    torch.cuda.empty_cache()
    if world == 1 and not args.no_extras:
        # The other configurations, compact: the served loop (a short Poisson window, both server
        # policies), the 4096-stripe mixed batch against per-stripe launches, and the 32 KiB point of
        # the GF(2^12) sweep.
        out["served"] = served_measure(torch, pyrit, dev, 20000.0, 2.0, args.slots)
        out["mixed"] = mixed_measure(torch, pyrit, dev, 5)
        plan12 = make_plan(pyrit, args.generator, 12, 16, 4)
        out["sweep32k"] = sweep_point(torch, pyrit, dev, plan12, 32768, 5, generator=args.generator)
        pyrit.pyrit_plan_destroy(plan12)
    if rank == 0:
        print(json.dumps(out))
    pyrit.pyrit_plan_destroy(plan)
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline(buf, blocks, pats, plan, pyrit, generator="cauchy", transform="embedding"):
    """The oracle, as it stands, on bounded samples of the same stripes and patterns: on all host
    cores (48 stripes, about 1 s of wall time there), and single-threaded (4 stripes); its parity
    is also compared with the GPU's for the sampled stripes."""
    import numpy as np
    import oracle
    cores = os.cpu_count() or 1
    blk = W * P
    G = oracle.cauchy_weighted(W, K, M)[0] if generator == "weighted" else oracle.cauchy(W, K, M)
    o_enc, o_dec = oracle_codec(transform)
    par0 = STRIPES * K * blk

    def timed(sample, nthreads):
        data = buf[:sample * K * blk].cpu().numpy().reshape(sample, K, W, P)
        gpar = buf[par0:par0 + sample * M * blk].cpu().numpy().reshape(sample, M, W, P)
        t0 = time.perf_counter()
        match = True
        for s in range(sample):
            par = o_enc(W, K, M, G, data[s], nthreads=nthreads)
            full = np.concatenate([data[s], par])
            rebuilt = o_dec(W, K, M, G, full, pats[s], nthreads=nthreads)
            match = match and np.array_equal(par, gpar[s]) and np.array_equal(rebuilt, full)
        dt = time.perf_counter() - t0
        return 2 * sample * K * blk / dt / 1e9, dt, match

    many = min(48, STRIPES)
    v_all, dt_all, ok_all = timed(many, cores)
    v_one, dt_one, ok_one = timed(4, 1)
    return {"value": v_all, "unit": "GB/s", "cores": cores, "kind": "oracle",
            "sample": "first %d of the %d stripes, encode + decode (same erasure patterns), %.1f s on %d threads" % (
                many, STRIPES, dt_all, cores),
            "single_thread": {"value": v_one, "unit": "GB/s", "cores": 1,
                              "sample": "first 4 stripes, encode + decode, %.1f s" % dt_one},
            "gpu_parity_on_sample": ok_all and ok_one}


# ---------------------------------------------------------------------------------------------
# Further measured workloads (one JSON line each; not the default line)
# ---------------------------------------------------------------------------------------------

def _setup_gpu():
    import torch
    from paper_1709_00178_gb300 import pyrit
    torch.cuda.set_device(0)
    return torch, pyrit, torch.device("cuda", 0)


def _time_batch(torch, pyrit, batch, stream, steps):
    for _ in range(3):
        pyrit.pyrit_batch_run(batch, stream, graph=True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        pyrit.pyrit_batch_run(batch, stream, graph=True)
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def sweep_point(torch, pyrit, dev, plan, P, steps, tune=True, stripes=0, generator="cauchy"):
    """One point of the GF(2^12) (n=13) Cauchy k=16 m=4 packet-size sweep: stripes filling ~8 GiB of
    source at packet size P (or `stripes` of them), an encode batch and a 4-erasure decode batch,
    tuned and timed (graph replay). A sampled stripe is checked against the oracle."""
    from paper_1709_00178_gb300.synth import BASE_SEED
    import numpy as np
    w, k, m = 12, 16, 4
    peak, _ = peak_hbm()
    e = P.bit_length() - 1
    S = stripes if stripes else (8 << 30) // (k * w * P)
    blk = w * P
    buf = torch.empty(S * (k + m) * blk, dtype=torch.uint8, device=dev)
    pyrit.pyrit_synth_fill(buf.data_ptr(), buf.numel(), BASE_SEED + 2, 0)
    torch.cuda.synchronize()
    base, par0 = buf.data_ptr(), S * k * blk
    blocks = [[base + (s * k + j) * blk for j in range(k)] + [base + par0 + (s * m + i) * blk for i in range(m)]
              for s in range(S)]
    rng = np.random.default_rng(BASE_SEED + 2 + e)
    pats = [sum(1 << int(x) for x in rng.choice(k + m, m, replace=False)) for _ in range(S)]
    enc = pyrit.pyrit_batch_create([(plan, 0, 0, P, blocks[s]) for s in range(S)])
    dec = pyrit.pyrit_batch_create([(plan, 1, pats[s], P, blocks[s]) for s in range(S)])
    stream = torch.cuda.Stream(device=dev)
    if tune:
        pyrit.pyrit_batch_tune(enc, stream, 2)
        pyrit.pyrit_batch_tune(dec, stream, 2)
    nvtx = torch.cuda.nvtx
    nvtx.range_push("timed")
    te = _time_batch(torch, pyrit, enc, stream, steps)
    td = _time_batch(torch, pyrit, dec, stream, steps)
    nvtx.range_pop()
    torch.cuda.synchronize()
    # the last runs encoded every stripe and then decoded it in place: stripe 0 is the oracle's codeword
    import oracle
    G = oracle.cauchy_weighted(w, k, m)[0] if generator == "weighted" else oracle.cauchy(w, k, m)
    cw = min(P, 4096)
    data0 = np.ascontiguousarray(buf[:k * blk].cpu().numpy().reshape(k, w, P)[:, :, :cw])
    par_got = buf[par0:par0 + m * blk].cpu().numpy().reshape(m, w, P)[:, :, :cw]
    ok = bool(np.array_equal(par_got, oracle.encode(w, k, m, G, data0, nthreads=os.cpu_count() or 1)))
    es, ds = pyrit.pyrit_batch_stats(enc), pyrit.pyrit_batch_stats(dec)
    ae, ad = es["alg_bytes"] / te / 1e6, ds["alg_bytes"] / td / 1e6
    out = {"workload": "GF(2^12) n=13 Cauchy k=16 m=4, %d KiB packets, %d stripes, 4-erasure decode" % (P // 1024, S),
           "packet_bytes": P, "stripes": S,
           "value": (es["src_bytes"] + ds["src_bytes"]) / (te + td) / 1e6, "unit": "GB/s",
           "encode_ms": te, "decode_ms": td, "encode_roofline_frac": ae / peak, "decode_roofline_frac": ad / peak,
           "encode_alg_gbs": ae, "decode_alg_gbs": ad,
           "encode_kernel": kernel_name(pyrit.pyrit_batch_shape(enc, 0)),
           "decode_kernel": kernel_name(pyrit.pyrit_batch_shape(dec, 0)), "oracle_parity_stripe0": ok}
    pyrit.pyrit_batch_destroy(enc)
    pyrit.pyrit_batch_destroy(dec)
    del buf
    torch.cuda.empty_cache()
    return out


def run_sweep(args):
    """GF(2^12) (n=13), Cauchy k=16 m=4: packet sizes 4 KiB..1 MiB, stripes filling ~8 GiB of
    source data; encode and 4-erasure decode per point, batched and autotuned (sweep_point)."""
    torch, pyrit, dev = _setup_gpu()
    plan = make_plan(pyrit, args.generator, 12, 16, 4)
    for e in range(12, 21):
        P = 1 << e
        if args.packet and P != args.packet:
            continue
        S = max(1, args.stripes) if (args.packet and args.stripes != STRIPES) else 0
        r = sweep_point(torch, pyrit, dev, plan, P, args.steps, tune=not args.no_tune, stripes=S,
                        generator=args.generator)
        out = {"metric": "encode+decode GB/s of source data", "workload": "sweep", "value": r.pop("value"),
               "unit": r.pop("unit"), "config": {"workload": r.pop("workload"), "packet_bytes": P, "stripes": r["stripes"],
                                                 "generator": args.generator}, "dtype": "u8", "data": "synthetic"}
        out.update(r)
        print(json.dumps(out), flush=True)
    pyrit.pyrit_plan_destroy(plan)


def run_transforms(args):
    """The two transforms of Sec. 2.3 on the same codes: GF(2^10) (n=11) Cauchy k=10 m=4 (k >= m,
    where the paper prefers the embedding) and k=4 m=8, GF(2^12) (n=13) k=2 m=6 (k < m, where it
    prefers the parity bit); 64 KiB packets, stripes filling ~2 GiB of source; encode and
    mixed-pattern (1..m erasures) decode batches, tuned, one JSON line per (code, transform). A
    sampled stripe of each is checked against the oracle's codec for that transform."""
    torch, pyrit, dev = _setup_gpu()
    from paper_1709_00178_gb300.synth import BASE_SEED
    import numpy as np
    import oracle
    peak, _ = peak_hbm()
    stream = torch.cuda.Stream(device=dev)
    P = 65536
    for (w, k, m) in [(10, 10, 4), (10, 4, 8), (12, 2, 6)]:
        blk = w * P
        S = (2 << 30) // (k * blk)
        buf = torch.empty(S * (k + m) * blk, dtype=torch.uint8, device=dev)
        rng = np.random.default_rng(BASE_SEED + 3 + k)
        pats = [sum(1 << int(x) for x in rng.choice(k + m, int(rng.integers(1, m + 1)), replace=False))
                for _ in range(S)]
        for transform in ("embedding", "parity"):
            pyrit.pyrit_synth_fill(buf.data_ptr(), buf.numel(), BASE_SEED + 3, 0)
            torch.cuda.synchronize()
            base, par0 = buf.data_ptr(), S * k * blk
            blocks = [[base + (s * k + j) * blk for j in range(k)] + [base + par0 + (s * m + i) * blk for i in range(m)]
                      for s in range(S)]
            plan = make_plan(pyrit, args.generator, w, k, m, transform)
            enc = pyrit.pyrit_batch_create([(plan, 0, 0, P, blocks[s]) for s in range(S)])
            dec = pyrit.pyrit_batch_create([(plan, 1, pats[s], P, blocks[s]) for s in range(S)])
            pyrit.pyrit_batch_tune(enc, stream, 2)
            pyrit.pyrit_batch_tune(dec, stream, 2)
            te = _time_batch(torch, pyrit, enc, stream, args.steps)
            td = _time_batch(torch, pyrit, dec, stream, args.steps)
            # the last runs decoded the encoded stripes in place: stripe 0 must be the oracle's codeword
            o_enc, _ = oracle_codec(transform)
            G = oracle.cauchy_weighted(w, k, m)[0] if args.generator == "weighted" else oracle.cauchy(w, k, m)
            torch.cuda.synchronize()
            data0 = buf[:k * blk].cpu().numpy().reshape(k, w, P)
            par_ok = bool(np.array_equal(buf[par0:par0 + m * blk].cpu().numpy().reshape(m, w, P),
                                         o_enc(w, k, m, G, data0, nthreads=os.cpu_count() or 1)))
            es, ds = pyrit.pyrit_batch_stats(enc), pyrit.pyrit_batch_stats(dec)
            ae, ad = es["alg_bytes"] / te / 1e6, ds["alg_bytes"] / td / 1e6
            print(json.dumps({
                "metric": "encode+decode GB/s of source data", "workload": "transforms",
                "value": (es["src_bytes"] + ds["src_bytes"]) / (te + td) / 1e6, "unit": "GB/s",
                "config": {"workload": "GF(2^%d) n=%d Cauchy k=%d m=%d, 64 KiB packets, %d stripes, 1-%d erasures"
                           % (w, w + 1, k, m, S, m), "transform": transform, "generator": args.generator},
                "encode_ms": te, "decode_ms": td, "encode_roofline_frac": ae / peak, "decode_roofline_frac": ad / peak,
                "encode_kernel": kernel_name(pyrit.pyrit_batch_shape(enc, 0)),
                "decode_kernel": kernel_name(pyrit.pyrit_batch_shape(dec, 0)),
                "oracle_parity_stripe0": par_ok, "dtype": "u8", "data": "synthetic"}), flush=True)
            pyrit.pyrit_batch_destroy(enc)
            pyrit.pyrit_batch_destroy(dec)
            pyrit.pyrit_plan_destroy(plan)
        del buf
        torch.cuda.empty_cache()


def run_paper(args):
    """The paper's three use cases (Sec. 5): (n, k) = (12, 8) over GF(2^4) with the embedding,
    (60, 40) over GF(2^6) with the embedding and (60, 20) over GF(2^6) with the parity transform
    (GF(2^6) from x^6 + x^3 + 1, Sec. 2.4), encode and decode across block sizes. Decoding rebuilds
    n - k lost blocks, the same ones in every stripe (failed devices). Stripes fill ~2 GiB of
    source per point (larger than L2); batches are tuned; a sampled stripe of each point is checked
    against the oracle's codec for its transform."""
    torch, pyrit, dev = _setup_gpu()
    from paper_1709_00178_gb300.synth import BASE_SEED
    import numpy as np
    import oracle
    peak, _ = peak_hbm()
    stream = torch.cuda.Stream(device=dev)
    cases = [("(12,8) GF(2^4) embedding", 4, 8, 4, "embedding"),
             ("(60,40) GF(2^6) embedding", 6, 40, 20, "embedding"),
             ("(60,20) GF(2^6) parity transform", 6, 20, 40, "parity")]
    for name, w, k, m, transform in cases:
        n = 9 if w == 6 else w + 1
        plan = make_plan(pyrit, args.generator, w, k, m, transform)
        G = oracle.cauchy_weighted(w, k, m)[0] if args.generator == "weighted" else oracle.cauchy(w, k, m)
        o_enc, o_dec = oracle_codec(transform)
        rng = np.random.default_rng(BASE_SEED + 5 + k)
        lost = sum(1 << int(x) for x in rng.choice(k + m, m, replace=False))
        for block_kib in (64, 256, 1024, 4096):
            P = block_kib * 1024 // w // 16 * 16
            blk = w * P
            S = max(8, (2 << 30) // (k * blk))
            buf = torch.empty(S * (k + m) * blk, dtype=torch.uint8, device=dev)
            pyrit.pyrit_synth_fill(buf.data_ptr(), buf.numel(), BASE_SEED + 5, 0)
            torch.cuda.synchronize()
            base, par0 = buf.data_ptr(), S * k * blk
            blocks = [[base + (s * k + j) * blk for j in range(k)] + [base + par0 + (s * m + i) * blk for i in range(m)]
                      for s in range(S)]
            enc = pyrit.pyrit_batch_create([(plan, 0, 0, P, blocks[s]) for s in range(S)])
            dec = pyrit.pyrit_batch_create([(plan, 1, lost, P, blocks[s]) for s in range(S)])
            pyrit.pyrit_batch_tune(enc, stream, 2)
            pyrit.pyrit_batch_tune(dec, stream, 2)
            te = _time_batch(torch, pyrit, enc, stream, args.steps)
            td = _time_batch(torch, pyrit, dec, stream, args.steps)
            torch.cuda.synchronize()
            # the last runs decoded the encoded stripes in place: stripe 0 must be the oracle's codeword
            # (checked on its first 2 KiB columns: every byte column is an independent codeword)
            cw = min(P, 2048)
            data0 = np.ascontiguousarray(buf[:k * blk].cpu().numpy().reshape(k, w, P)[:, :, :cw])
            want = o_enc(w, k, m, G, data0, nthreads=os.cpu_count() or 1)
            got = buf[par0:par0 + m * blk].cpu().numpy().reshape(m, w, P)[:, :, :cw]
            ok = bool(np.array_equal(got, want))
            es, ds = pyrit.pyrit_batch_stats(enc), pyrit.pyrit_batch_stats(dec)
            ae, ad = es["alg_bytes"] / te / 1e6, ds["alg_bytes"] / td / 1e6
            print(json.dumps({
                "metric": "encode / decode GB/s of source data", "workload": "paper",
                "config": {"workload": name, "w": w, "n": n, "k": k, "m": m, "block_bytes": blk, "packet_bytes": P,
                           "stripes": S, "lost_blocks": m, "transform": transform, "generator": args.generator},
                "encode_gbs": es["src_bytes"] / te / 1e6, "decode_gbs": ds["src_bytes"] / td / 1e6,
                "encode_ms": te, "decode_ms": td, "encode_roofline_frac": ae / peak, "decode_roofline_frac": ad / peak,
                "encode_kernel": kernel_name(pyrit.pyrit_batch_shape(enc, 0)),
                "decode_kernel": kernel_name(pyrit.pyrit_batch_shape(dec, 0)),
                "launches": [es["launches"], ds["launches"]], "oracle_parity_stripe0": ok,
                "dtype": "u8", "data": "synthetic"}), flush=True)
            pyrit.pyrit_batch_destroy(enc)
            pyrit.pyrit_batch_destroy(dec)
            del buf
            torch.cuda.empty_cache()
        pyrit.pyrit_plan_destroy(plan)


def run_fields(args):
    """Fields from other factors of x^n + 1 (Props. 1-2) beside a native one, same code shape:
    GF(16) from the AOP on R_{2,5} (native), GF(16) from x^4 + x + 1 on R_{2,15} (k=8 m=4), GF(8)
    from x^3 + x + 1 on R_{2,7} (k=5 m=3: k + m <= 8); 64 KiB packets, stripes filling ~2 GiB of
    source; encode and an m-erasure decode (one pattern for all stripes), tuned; a stripe checked
    against the oracle's codec over the plan's modulus."""
    torch, pyrit, dev = _setup_gpu()
    from paper_1709_00178_gb300.synth import BASE_SEED
    import numpy as np
    import oracle
    peak, _ = peak_hbm()
    stream = torch.cuda.Stream(device=dev)
    nvtx = torch.cuda.nvtx
    P = 65536
    for (w, n, k, m, name) in [(4, 5, 8, 4, "GF(2^4) from the AOP on R_{2,5} (native)"),
                               (4, 15, 8, 4, "GF(2^4) from x^4+x+1 on R_{2,15}"),
                               (3, 7, 5, 3, "GF(2^3) from x^3+x+1 on R_{2,7}")]:
        blk = w * P
        S = (2 << 30) // (k * blk)
        buf = torch.empty(S * (k + m) * blk, dtype=torch.uint8, device=dev)
        pyrit.pyrit_synth_fill(buf.data_ptr(), buf.numel(), BASE_SEED + 6, 0)
        torch.cuda.synchronize()
        base, par0 = buf.data_ptr(), S * k * blk
        blocks = [[base + (s * k + j) * blk for j in range(k)] + [base + par0 + (s * m + i) * blk for i in range(m)]
                  for s in range(S)]
        plan = pyrit.pyrit_plan_create(w, n, k, m)
        g, native = pyrit.pyrit_plan_modulus(plan)
        lost = (0b1011 | (1 << (k + 1))) if m == 4 else (0b101 | (1 << k))
        enc = pyrit.pyrit_batch_create([(plan, 0, 0, P, blocks[s]) for s in range(S)])
        dec = pyrit.pyrit_batch_create([(plan, 1, lost, P, blocks[s]) for s in range(S)])
        if not args.no_tune:
            pyrit.pyrit_batch_tune(enc, stream, 2)
            pyrit.pyrit_batch_tune(dec, stream, 2)
        nvtx.range_push("timed")
        te = _time_batch(torch, pyrit, enc, stream, args.steps)
        td = _time_batch(torch, pyrit, dec, stream, args.steps)
        nvtx.range_pop()
        torch.cuda.synchronize()
        cw = 4096
        data0 = np.ascontiguousarray(buf[:k * blk].cpu().numpy().reshape(k, w, P)[:, :, :cw])
        want = oracle.encode_mod(w, g, k, m, oracle.cauchy_mod(w, g, k, m), data0, nthreads=os.cpu_count() or 1)
        got = buf[par0:par0 + m * blk].cpu().numpy().reshape(m, w, P)[:, :, :cw]
        es, ds = pyrit.pyrit_batch_stats(enc), pyrit.pyrit_batch_stats(dec)
        ae, ad = es["alg_bytes"] / te / 1e6, ds["alg_bytes"] / td / 1e6
        print(json.dumps({
            "metric": "encode / decode GB/s of source data", "workload": "fields",
            "config": {"workload": name + ", k=%d m=%d, 64 KiB packets, %d stripes" % (k, m, S), "w": w, "n": n,
                       "modulus": hex(g), "native": native},
            "encode_gbs": es["src_bytes"] / te / 1e6, "decode_gbs": ds["src_bytes"] / td / 1e6,
            "encode_roofline_frac": ae / peak, "decode_roofline_frac": ad / peak,
            "encode_kernel": kernel_name(pyrit.pyrit_batch_shape(enc, 0)),
            "decode_kernel": kernel_name(pyrit.pyrit_batch_shape(dec, 0)),
            "oracle_parity_stripe0": bool(np.array_equal(got, want)), "dtype": "u8", "data": "synthetic"}), flush=True)
        pyrit.pyrit_batch_destroy(enc)
        pyrit.pyrit_batch_destroy(dec)
        pyrit.pyrit_plan_destroy(plan)
        del buf
        torch.cuda.empty_cache()


def run_gf16(args):
    """GF(16) (w=4, n=5), Cauchy k=4 m=2, one stripe of 4 x 256 KiB packets per block (4 MiB of
    source): encode, then every erasure pattern of one or two blocks (21) decoded, each on its own
    copy of the stripe, in one batch; every byte checked against the oracle. The stripe is
    L2-resident, so its GB/s is not an HBM figure."""
    torch, pyrit, dev = _setup_gpu()
    from itertools import combinations
    from paper_1709_00178_gb300.synth import BASE_SEED
    import numpy as np
    import oracle
    w, k, m, P = 4, 4, 2, 256 * 1024
    blk = w * P
    plan = make_plan(pyrit, args.generator, w, k, m)
    G = oracle.cauchy_weighted(w, k, m)[0] if args.generator == "weighted" else oracle.cauchy(w, k, m)
    pats = [sum(1 << b for b in c) for e in (1, 2) for c in combinations(range(k + m), e)]
    copies = 1 + len(pats)
    buf = torch.zeros(copies * (k + m) * blk, dtype=torch.uint8, device=dev)
    pyrit.pyrit_synth_fill(buf.data_ptr(), k * blk, BASE_SEED + 5, 0)
    base = buf.data_ptr()
    stripe = lambda c: [base + (c * (k + m) + e) * blk for e in range(k + m)]
    stream = torch.cuda.Stream(device=dev)
    enc = pyrit.pyrit_batch_create([(plan, 0, 0, P, stripe(0))])
    t_enc = _time_batch(torch, pyrit, enc, stream, args.steps)
    torch.cuda.synchronize()
    data = buf[:k * blk].cpu().numpy().reshape(k, w, P)
    full = np.concatenate([data, oracle.encode(w, k, m, G, data, nthreads=os.cpu_count() or 1)])
    enc_ok = bool(np.array_equal(buf[:(k + m) * blk].cpu().numpy().reshape(k + m, w, P), full))
    one = buf[:(k + m) * blk]

    def reset():
        for c in range(1, copies):
            view = buf[c * (k + m) * blk:(c + 1) * (k + m) * blk].view(k + m, blk)
            view.copy_(one.view(k + m, blk))
            for e in range(k + m):
                if (pats[c - 1] >> e) & 1:
                    view[e].fill_(0xE7)

    reset()
    dec = pyrit.pyrit_batch_create([(plan, 1, pats[c - 1], P, stripe(c)) for c in range(1, copies)])
    pyrit.pyrit_batch_run(dec, stream)
    torch.cuda.synchronize()
    dec_ok = all(bool(np.array_equal(buf[c * (k + m) * blk:(c + 1) * (k + m) * blk].cpu().numpy().reshape(k + m, w, P),
                                     full)) for c in range(1, copies))
    t_dec = _time_batch(torch, pyrit, dec, stream, args.steps)
    es, ds = pyrit.pyrit_batch_stats(enc), pyrit.pyrit_batch_stats(dec)
    print(json.dumps({
        "metric": "encode / decode GB/s of source data (L2-resident)", "workload": "gf16", "unit": "GB/s",
        "value": (es["src_bytes"] + ds["src_bytes"]) / (t_enc + t_dec) / 1e6,
        "encode_gbs": es["src_bytes"] / t_enc / 1e6, "decode_gbs": ds["src_bytes"] / t_dec / 1e6,
        "encode_ms": t_enc, "decode_ms_21_patterns": t_dec,
        "bit_exact_encode": enc_ok, "bit_exact_all_21_patterns": dec_ok,
        "config": {"workload": "GF(16) n=5 Cauchy k=4 m=2, 256 KiB packets, 1 stripe; encode + all 21 patterns of "
                               "1-2 erasures", "generator": args.generator},
        "dtype": "u8", "data": "synthetic"}), flush=True)
    pyrit.pyrit_batch_destroy(enc)
    pyrit.pyrit_batch_destroy(dec)
    pyrit.pyrit_plan_destroy(plan)


def mixed_measure(torch, pyrit, dev, steps, tune=True, per_stripe_reps=3, oracle_sample=6):
    """4096 uneven stripes (the mixed-batch workload of synth.mixed_batch_specs) coded by one
    batched persistent launch per ring size (default compilation policy, autotuned, replayed from
    a CUDA graph) against 4096 per-stripe launches of the same generic kernel (run-time compilation
    off for that arm only). Both must write the same bytes, and a seeded sample of stripes is
    compared with the oracle. Returns the measurement as a dict."""
    from paper_1709_00178_gb300.synth import BASE_SEED, mixed_batch_specs, stripe_offsets
    import numpy as np
    specs = mixed_batch_specs(BASE_SEED + 3, 4096)
    offs, total = stripe_offsets(specs)
    buf = torch.empty(total, dtype=torch.uint8, device=dev)
    pyrit.pyrit_synth_fill(buf.data_ptr(), total, BASE_SEED + 3, 0)
    torch.cuda.synchronize()
    plans = {}
    for (w, k, m, P, op, er) in specs:
        if (w, k, m) not in plans:
            plans[(w, k, m)] = pyrit.pyrit_plan_create(w, w + 1, k, m)
    base = buf.data_ptr()
    stripes = [(plans[(w, k, m)], op, er, P, [base + o + e * w * P for e in range(k + m)])
               for (w, k, m, P, op, er), o in zip(specs, offs)]
    stream = torch.cuda.Stream(device=dev)
    batch = pyrit.pyrit_batch_create(stripes)
    st = pyrit.pyrit_batch_stats(batch)
    if tune:
        pyrit.pyrit_batch_tune(batch, stream, 2)
    t_batch = _time_batch(torch, pyrit, batch, stream, steps)
    shapes = []
    for g in range(st["launches"]):
        try:
            shapes.append(kernel_name(pyrit.pyrit_batch_shape(batch, g)))
        except Exception:
            break
    after_batch = buf.clone()
    ks = [spec[1] for spec in specs]

    def per_stripe():
        for (plan, op, er, P, blocks), kk in zip(stripes, ks):
            if op == 0:
                pyrit.pyrit_encode(plan, blocks[:kk], blocks[kk:], P, stream)
            else:
                pyrit.pyrit_decode(plan, blocks, er, P, stream)

    mode = pyrit.pyrit_jit_mode(pyrit.PYRIT_JIT_OFF)
    try:
        per_stripe()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(per_stripe_reps):
            per_stripe()
        b.record(stream)
        torch.cuda.synchronize()
    finally:
        pyrit.pyrit_jit_mode(mode)
    t_per = a.elapsed_time(b) / per_stripe_reps
    same = bool(torch.equal(after_batch, buf))
    del after_batch
    oracle_ok = None
    if oracle_sample:
        import oracle
        rng = np.random.default_rng(BASE_SEED + 33)
        small = [i for i, sp in enumerate(specs) if sp[3] <= 16384]
        ok = True
        for i in rng.choice(small, oracle_sample, replace=False):
            w, k, m, P, op, er = specs[i]
            h = buf[offs[i]:offs[i] + (k + m) * w * P].cpu().numpy().reshape(k + m, w, P)
            G = oracle.cauchy(w, k, m)
            if op == 0:
                ok = ok and np.array_equal(h[k:], oracle.encode(w, k, m, G, h[:k], nthreads=os.cpu_count() or 1))
            else:
                ok = ok and np.array_equal(h, oracle.decode(w, k, m, G, h, er, nthreads=os.cpu_count() or 1))
        oracle_ok = bool(ok)
    peak, _ = peak_hbm()
    out = {"workload": "4096 uneven stripes, n in {5,11,13}, k 4-32, m 2-8, P 512 B-256 KiB, half decode",
           "value": st["src_bytes"] / t_batch / 1e6, "unit": "GB/s", "stripes": len(specs),
           "alg_bytes": st["alg_bytes"], "src_bytes": st["src_bytes"], "launches": st["launches"], "tiles": st["tiles"],
           "kernels": shapes, "batched_ms": t_batch, "per_stripe_ms": t_per, "speedup_vs_per_stripe": t_per / t_batch,
           "roofline_frac": st["alg_bytes"] / t_batch / 1e6 / peak, "same_bytes_as_per_stripe": same,
           "oracle_sample_ok": oracle_ok, "oracle_sample": oracle_sample}
    pyrit.pyrit_batch_destroy(batch)
    for p in plans.values():
        pyrit.pyrit_plan_destroy(p)
    del buf
    torch.cuda.empty_cache()
    return out


def run_mixed(args):
    """The mixed-batch workload as its own JSON line (mixed_measure)."""
    torch, pyrit, dev = _setup_gpu()
    r = mixed_measure(torch, pyrit, dev, args.steps, tune=not args.no_tune, per_stripe_reps=max(1, min(5, args.steps)))
    out = {"metric": "encode+decode GB/s of source data", "workload": "mixed", "unit": "GB/s", "value": r.pop("value"),
           "config": {"workload": r.pop("workload"), "stripes": r["stripes"]}, "dtype": "u8", "data": "synthetic"}
    out.update(r)
    print(json.dumps(out), flush=True)


def served_measure(torch, pyrit, dev, rate, seconds, slots, pool=512):
    """Poisson arrivals (seeded, `rate` requests/s for `seconds`) of GF(2^12) k=16 m=4 requests, P
    one of 4 KiB..1 MiB (powers of two, uniform), half encode and half 4-erasure decode, served with
    continuous batching under a 16 GiB budget; payloads pre-generated in device memory. Then the same
    arrivals through the same server with one request per launch. Returns the measurement."""
    from paper_1709_00178_gb300.synth import BASE_SEED
    import numpy as np
    w, k, m = 12, 16, 4
    rng = np.random.default_rng(BASE_SEED + 4)
    POOL = pool
    pool_P = [1 << int(e) for e in rng.integers(12, 21, POOL)]
    pool_pat = [sum(1 << int(x) for x in rng.choice(k + m, m, replace=False)) for _ in range(POOL)]
    offs, total = [], 0
    for P in pool_P:
        offs.append(total)
        total += (k + m) * w * P
    buf = torch.empty(total, dtype=torch.uint8, device=dev)
    pyrit.pyrit_synth_fill(buf.data_ptr(), total, BASE_SEED + 4, 0)
    torch.cuda.synchronize()
    plan = pyrit.pyrit_plan_create(w, w + 1, k, m)
    for pat in set(pool_pat):  # the plan caches every decoding matrix before the timed window
        pyrit.pyrit_plan_decode_masks(plan, pat)
    # the plan's generated networks (encode table, syndrome decode) are compiled before serving;
    # without this the server codes with the generic kernel until its background compiles finish
    pyrit.pyrit_plan_specialise(plan, pyrit.PYRIT_OP_ENCODE)
    pyrit.pyrit_plan_specialise(plan, pyrit.PYRIT_OP_DECODE_ANY)
    base = buf.data_ptr()
    nreq = int(rate * seconds)
    gaps = rng.exponential(1e9 / rate, nreq)
    arrivals = np.cumsum(gaps).astype(np.int64)
    ops = rng.integers(0, 2, nreq)
    reqs, src_bytes = [], 0
    for i in range(nreq):
        s = i % POOL
        P = pool_P[s]
        blocks = [base + offs[s] + e * w * P for e in range(k + m)]
        reqs.append((plan, int(ops[i]), pool_pat[s] if ops[i] else 0, P, blocks, i, 0))
        src_bytes += k * w * P
    arr, keep = pyrit.pyrit_requests_array(reqs)
    def serve(max_batch, slots):
        """One pass of the arrival stream through a server; latency and throughput statistics."""
        srv = pyrit.pyrit_server_create(16 << 30, max_batch=max_batch, slots=slots)
        # The clock sampler starts before anything is timed: its startup queries the driver, which
        # stalled the server's stream calls for tens of milliseconds when it coincided with the
        # first arrivals. Then a short unmeasured burst warms the launch shapes and the device.
        clocks = Clocks(0)
        clocks.start()
        pyrit.pyrit_server_submit_slice(srv, arr, 0, min(64, nreq))
        pyrit.pyrit_server_drain(srv, 60000)
        pyrit.pyrit_server_poll(srv, 1 << 20)
        time.sleep(0.5)
        # The arrival times are written first (200k ctypes fields take tens of milliseconds), with
        # the first arrival far enough ahead that submission starts before it: arrivals must not
        # pile up into a burst the load generator itself created.
        t0 = pyrit.pyrit_server_now_ns(srv) + 1000000000
        for i in range(nreq):
            arr[i].arrival_ns = int(t0 + arrivals[i])
        if pyrit.pyrit_server_now_ns(srv) >= t0:
            raise RuntimeError("load generator set-up ran past the first arrival")
        # The load generator is the library's native replay loop (this thread, outside Python):
        # each request is submitted, and validated, when its arrival time comes. A Python loop
        # submitted 5-8 us late at the 99th percentile and, about once in 10-30 passes, stalled
        # for 10-60 ms, which counted as service latency.
        pyrit.pyrit_server_replay(srv, arr, 0, nreq)
        pyrit.pyrit_server_drain(srv, 600000)
        clk = clocks.stop()
        done = pyrit.pyrit_server_poll(srv, nreq + 64)
        st = pyrit.pyrit_server_stats(srv)
        pyrit.pyrit_server_destroy(srv)
        done = [d for d in done if d[0] < nreq]
        t_first = min(d[2] for d in done)
        t_last = max(d[4] for d in done)
        return {"done": done, "all_ok": all(d[1] == 0 for d in done),
                "sustained_gbs": src_bytes / ((t_last - t_first) * 1e-9) / 1e9,
                "batches": st["batches"], "launches": st["launches"], "max_inflight_bytes": st["max_inflight"],
                "clocks": clk}

    def pooled(runs):
        """Latency statistics over the requests of several passes of the arrival stream."""
        done = [d for r in runs for d in r["done"]]
        lat = np.array([d[4] - d[2] for d in done], dtype=np.float64) / 1e3  # us
        wait = np.array([d[3] - d[2] for d in done], dtype=np.float64) / 1e3
        run = np.array([d[4] - d[3] for d in done], dtype=np.float64) / 1e3
        per_pass = [float(np.percentile(np.array([d[4] - d[2] for d in r["done"]], dtype=np.float64) / 1e3, 99))
                    for r in runs]
        return {"p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
                "p999_us": float(np.percentile(lat, 99.9)), "max_us": float(lat.max()), "requests": len(lat),
                "passes": len(runs), "p99_per_pass_us": per_pass,
                "arrival_to_launch_p50_us": float(np.percentile(wait, 50)),
                "arrival_to_launch_p99_us": float(np.percentile(wait, 99)),
                "launch_to_done_p50_us": float(np.percentile(run, 50)),
                "launch_to_done_p99_us": float(np.percentile(run, 99)),
                "all_ok": all(r["all_ok"] for r in runs),
                "sustained_gbs": min(r["sustained_gbs"] for r in runs),
                "batches": sum(r["batches"] for r in runs), "launches": sum(r["launches"] for r in runs),
                "max_inflight_bytes": max(r["max_inflight_bytes"] for r in runs)}

    # Continuous batching (up to 64 admitted requests per launch group, `slots` stream slots whose
    # launches overlap: a request that finds a slot free starts alone, requests that arrive while
    # every slot is busy share the next free one), and the same arrivals through the same server
    # and kernels with one request per launch: per-stripe launches as requests arrive, up to 16 in
    # flight on their own streams. The arms alternate (batching, per-request, per-request,
    # batching) so that neither always runs first; each arm's two passes are pooled.
    b1 = serve(64, slots)
    s1 = serve(1, 16)
    s2 = serve(1, 16)
    b2 = serve(64, slots)
    clk = b1["clocks"]
    batched = pooled([b1, b2])
    single = pooled([s1, s2])
    out = dict(batched)
    out.update({
        "offered_gbs": src_bytes / (arrivals[-1] * 1e-9) / 1e9,
        "per_request_launches": single,
        "workload": "Poisson %gk req/s for %g s, GF(2^12) k=16 m=4, P 4 KiB-1 MiB, half 4-erasure decode, 16 GiB "
                    "budget, %d stream slots, batches up to 64; per_request_launches: the same arrivals one request "
                    "per launch, 16 stream slots; two passes per arm, alternating" % (rate / 1000, seconds, slots),
        "clocks": clk})
    pyrit.pyrit_plan_destroy(plan)
    del buf, arr, keep
    torch.cuda.empty_cache()
    return out


def run_served(args):
    """The served workload as its own JSON line (served_measure)."""
    torch, pyrit, dev = _setup_gpu()
    r = served_measure(torch, pyrit, dev, args.rate, args.seconds, args.slots)
    out = {"metric": "served p50/p99 latency", "workload": "served", "unit": "us", "value": r["p99_us"]}
    out.update(r)
    out.update({"config": {"workload": r.pop("workload"), "seconds": args.seconds},
                "higher_is_better": False, "dtype": "u8", "data": "synthetic"})
    out.pop("workload", None)
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
