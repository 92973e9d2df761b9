#!/usr/bin/env python
"""Benchmark: decoded GB/s of canonical-Huffman decoding on GB300 through the
library's C ABI.

Headline (`value`): one step = one hd_decode of a 512^3 field of Lorenzo
quantization codes with its gap array (decode-table kernel, count kernel,
decode-and-write kernel), inputs resident in HBM, L2 flushed between steps.
Extra keys: the same field by self-synchronisation, end to end from pinned
host buffers (`e2e`), the batched workload (256 fields of uneven sizes, one
graph launch, autotuned shape) against one launch per field (`batched`), and
a served request trace (Poisson arrivals, continuous batching, p50/p99
latency) against one launch per request (`served`).  Prints one JSON line
(rank 0).  ``--impl reference`` times the CPU oracle instead (bounded samples
of the same workload on the host cores).

Multi-GPU (torchrun): every rank decodes its own field of the same shape
(replicas, no collective on the data path); value = all ranks' symbols / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "decoded GB/s & % HBM roofline; batched/served vs per-field; p50/p99 latency"
FALLBACK_HBM_GBS = 6800.0


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def ranks_max(vals, dist, device):
    """Element-wise maximum over ranks (the slowest rank's times); identity
    without a process group."""
    if not dist:
        return [float(v) for v in vals]
    import torch
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def ranks_min(vals, dist, device):
    """Element-wise minimum over ranks."""
    if not dist:
        return [float(v) for v in vals]
    import torch
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MIN)
    return [float(v) for v in t.tolist()]


def whole_job_gbps(codes_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Decoded GB/s of the whole job: every rank's uint16 output over the
    slowest rank's time (ranks decode equal-sized replicas)."""
    return 2.0 * codes_per_rank * steps * world / (max_ms * 1e-3) / 1e9


def workload_quantized(side: int, seed: int, keep_field: bool = False):
    import synth
    return synth.field3d_quantized(side, rel_eb=1e-4, noise=0.01, seed=seed,
                                   keep_field=keep_field)


def workload_codes(side: int, seed: int):
    return workload_quantized(side, seed)["codes"]


def workload_desc(side: int) -> str:
    return (f"{side}^3 float32 field (64 Fourier modes, 1/k^2 amplitude, +1% Gaussian noise), "
            f"3D Lorenzo, rel. error bound 1e-4, radius 512 -> {side**3} uint16 codes; "
            f"canonical Huffman (max 32 bits), MSB-first uint32 stream, S=128, uint8 gap array")


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# kernel sources behind each traffic record (profiles/traffic.json)
KERNEL_SOURCES = {
    "decode_gap": ("decode2.cu", "decode_common.cuh", "common.cuh"),
    "decode_gap_one_pass": ("decode_warp.cu", "decode_common.cuh", "common.cuh"),
}
# kernels between the library's timing events, per decoder (hd_config.decoder)
DECODER_KERNELS = {1: ("decode_gap", "k_count + k_scan + k_write"),
                   2: ("decode_gap_one_pass", "k_decode_warp")}


def roofline_of(nbytes: float, ms: float, peak: float, peak_kind: str) -> dict:
    """HBM roofline of a decode: algorithmic bytes over its time, against the
    measured copy bandwidth."""
    achieved = nbytes / (ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "peak_kind": peak_kind, "algorithmic_bytes": nbytes,
            "kernel_ms": ms}


def kernel_source_hash(kernel: str = "decode_gap") -> str:
    h = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_2201_09118_gb300", "csrc")
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(cs, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, n_codes: int, launch: dict):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source in the same launch shape (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d[kernel]
        if e.get("source_hash") != kernel_source_hash(kernel):
            return None
        # the DRAM bytes of a decode are the stream, gap array and output read
        # and written once, whatever the launch shape of the same kernel source
        return float(e["dram_bytes_per_launch"]) * n_codes / float(e["n_codes"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
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
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def cpu_baseline_one_thread(codes: np.ndarray, target_s: float = 12.0):
    """The oracle's sequential bit-by-bit decoder on a prefix sample of the
    same field (single host thread)."""
    import oracle
    n = min(codes.size, 1 << 24)
    x = codes[:n]
    c = oracle.compress(x, 1024, S=128)
    t0 = time.perf_counter()
    reps = 0
    while True:
        out = oracle.decode(c["words"], c["nbits"], c["codes"], c["lengths"], n_cap=n)
        reps += 1
        el = time.perf_counter() - t0
        if el >= target_s or reps >= 64:
            break
    assert np.array_equal(out, x)
    gbps = 2.0 * n * reps / el / 1e9
    return {"value": gbps, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"first {n} codes of the field ({c['nbits']} bits), decoded {reps}x "
                      f"sequentially by the oracle's bit-by-bit tree walk, 1 host thread",
            "seconds": el}


# --- the oracle on every host core: independent gap-array chunks -------------
_CPU = {}


def _cpu_init(words_path, codes_path, lengths, cw):
    _CPU["words"] = np.load(words_path, mmap_mode="r")
    _CPU["x"] = np.load(codes_path, mmap_mode="r")
    _CPU["lengths"] = lengths
    _CPU["cw"] = cw


def _cpu_chunk(task):
    """Decodes stream bits [b0, b1) (codeword boundaries from the gap array)
    with the oracle; with `verify`, compares them with codes [s0, s1)."""
    import oracle
    b0, b1, s0, s1, verify = task
    out = oracle.decode(_CPU["words"], b1, _CPU["cw"], _CPU["lengths"], n_cap=s1 - s0,
                        start_bit=b0)
    if verify:
        return out.size == s1 - s0 and bool(np.array_equal(out, _CPU["x"][s0:s1]))
    return out.size == s1 - s0


def oracle_all_cores(codes: np.ndarray, target_s: float = 10.0, steps: int = 0,
                     warmup: int = 1):
    """The oracle's bit-by-bit decoder on every host core: the field (or a
    prefix of 2^26 codes) is split at gap-array subsequence boundaries into
    chunks that decode independently (Sec. III-C), one process per core (a
    spawn pool, so it is safe after CUDA work).  Times `steps` whole-sample
    decodes, or as many as fit in target_s.  Returns (GB/s of uint16 output,
    info dict)."""
    import multiprocessing as mp
    import oracle
    n = min(codes.size, 1 << 26)
    x = np.ascontiguousarray(codes[:n])
    c = oracle.compress(x, 1024, S=128)
    S = 128
    nsub = c["gap"].size
    counts = oracle.subseq_counts(x, c["lengths"], S, c["nbits"]).astype(np.uint64)
    first = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint64)
    cores = os.cpu_count() or 1
    nchunk = min(nsub, 8 * cores)
    edges = np.linspace(0, nsub, nchunk + 1).astype(np.int64)
    tmp = tempfile.mkdtemp(prefix="oracle_cpu_")
    wp, xp = os.path.join(tmp, "words.npy"), os.path.join(tmp, "codes.npy")
    np.save(wp, c["words"])
    np.save(xp, x)

    def tasks(verify):
        out = []
        for k in range(nchunk):
            i0, i1 = int(edges[k]), int(edges[k + 1])
            if i0 == i1:
                continue
            b0 = i0 * S + int(c["gap"][i0])
            b1 = i1 * S + int(c["gap"][i1]) if i1 < nsub else int(c["nbits"])
            out.append((b0, b1, int(first[i0]), int(first[i1]), verify))
        return out

    pool = mp.get_context("spawn").Pool(cores, initializer=_cpu_init,
                                        initargs=(wp, xp, c["lengths"], c["codes"]))
    try:
        assert all(pool.map(_cpu_chunk, tasks(True), chunksize=1)), "oracle chunk mismatch"
        for _ in range(max(0, warmup - 1)):
            pool.map(_cpu_chunk, tasks(False), chunksize=1)
        times = []
        t_all = time.perf_counter()
        while True:
            t0 = time.perf_counter()
            ok = pool.map(_cpu_chunk, tasks(False), chunksize=1)
            times.append(time.perf_counter() - t0)
            assert all(ok)
            if steps and len(times) >= steps:
                break
            if not steps and (time.perf_counter() - t_all >= target_s or len(times) >= 200):
                break
    finally:
        pool.close()
        pool.join()
        for p in (wp, xp):
            os.unlink(p)
        os.rmdir(tmp)
    total = sum(times)
    gbps = 2.0 * n * len(times) / total / 1e9
    info = {"cores": cores, "sample": f"first {n} codes of the field ({c['nbits']} bits) split "
                                      f"at gap-array boundaries into {nchunk} chunks decoded by "
                                      f"the oracle's bit-by-bit tree walk on {cores} processes, "
                                      f"{len(times)} whole-sample passes",
            "seconds": total, "passes": len(times), "ms_per_pass": 1e3 * total / len(times)}
    return gbps, info


def cpu_baseline(codes: np.ndarray):
    """All host cores (the value) and one host thread, both the oracle."""
    one = cpu_baseline_one_thread(codes)
    gbps, info = oracle_all_cores(codes)
    return {"value": gbps, "unit": "GB/s", "cores": info["cores"], "kind": "oracle",
            "sample": info["sample"], "seconds": info["seconds"], "one_thread": one}


def run_reference(args):
    """CPU oracle arm: each step decodes a bounded sample of the workload."""
    import oracle
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    side = args.side
    codes = workload_codes(side, seed=1001)
    value, info = oracle_all_cores(codes, steps=args.steps, warmup=args.warmup)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": info["ms_per_pass"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u16", "data": "synthetic",
        "config": {"workload": workload_desc(side),
                   "parallelism": f"{info['cores']} host processes"},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": info["cores"],
                         "kind": "oracle", "sample": info["sample"] + " (one per step)"},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def make_batch_field(spec):
    """Pool worker: one field of the batched workload, encoded on the host
    (product encoder, own codebook).  Returns the stream and a CRC of the codes."""
    import zlib

    import synth
    from paper_2201_09118_gb300 import hd
    x = synth.smooth_codes_1d(spec.n, spec.rel_eb, alphabet=spec.alphabet, seed=spec.seed)
    lengths = hd.hd_build_codebook(x, spec.alphabet, 32)
    enc = hd.hd_encode(x, lengths, 128)
    return {"words": enc["words"], "gap": enc["gap"], "nbits": enc["nbits"],
            "nwords": enc["nwords"], "subseq_bits": 128, "lengths": lengths, "n": int(x.size),
            "alphabet": spec.alphabet, "rel_eb": spec.rel_eb, "crc": zlib.crc32(x.tobytes())}


def start_batch_generation(n_fields: int, procs: int):
    """Starts encoding the batched workload in a spawn pool (before any CUDA
    call in this process); returns (pool, async result)."""
    import multiprocessing as mp

    import synth
    specs = synth.batch_spec(n_fields, lo=1 << 16, hi=1 << 26, seed=1003)
    pool = mp.get_context("spawn").Pool(procs)
    # largest fields first so the pool finishes evenly
    order = sorted(range(len(specs)), key=lambda k: -specs[k].n)
    res = pool.map_async(make_batch_field, [specs[k] for k in order], chunksize=1)
    return pool, res, order


def run_encode(hd, torch, ctx, codes, lengths, enc, stream, flush, steps: int = 5):
    """The step before the decoder: GPU canonical-Huffman encode with gap
    array (hd_encode_device, synchronous: two kernels, a 16-byte read-back of
    the stream length, the write kernel) of the same field, checked against
    the host encoder's stream."""
    d_codes = torch.from_numpy(codes.view(np.int16)).to(f"cuda:{torch.cuda.current_device()}")
    e = ctx.encode(d_codes, lengths, 128, stream=stream)
    ok = (e["nbits"] == enc["nbits"]
          and np.array_equal(e["words"].cpu().numpy().view(np.uint32), enc["words"])
          and np.array_equal(e["gap"].cpu().numpy(), enc["gap"]))
    times = []
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.encode(d_codes, lengths, 128, stream=stream)
        times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    n = codes.size
    alg = 2 * n + (enc["nbits"] + 7) // 8 + enc["nsub"]
    peak, kind = measured_peak()
    return {"value": 2.0 * n / t / 1e9, "unit": "GB/s (uint16 codes in)", "ms": 1e3 * t,
            "algorithmic_bytes": alg, "hbm_frac": alg / t / 1e9 / peak, "peak_kind": kind,
            "matches_host_encoder": bool(ok),
            "timing": "wall clock around the synchronous call (incl. its length read-back)"}


def run_decompress(hd, torch, ctx, field, dec_codes, g, stream, flush, steps: int = 5):
    """The step after the decoder: Lorenzo reconstruction of the decoded codes
    into float32 (hd_reconstruct_device), and decode + reconstruction in one
    call (hd_decompress_device), on the same field; values checked against the
    original field's error bound."""
    side = round(dec_codes.numel() ** (1 / 3))
    dims = (side, side, side)
    dev = dec_codes.device
    idx = torch.from_numpy(g["out_idx"].view(np.int64)).to(dev)
    val = torch.from_numpy(g["out_val"]).to(dev)
    n = dec_codes.numel()
    fout = torch.empty(n, dtype=torch.float32, device=dev)

    def timed(fn):
        fn()
        ms = []
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    L = hd.lorenzo_params(dims, 512, g["eb"], idx, val)
    recon_ms = timed(lambda: ctx.reconstruct(dec_codes, L, fout, stream))
    ok = ctx.status(stream) == 0
    # the band path (groups of 64 slices, or all slices in one group) for comparison
    sweep = {}
    for zc in (64, side):
        Lz = hd.lorenzo_params(dims, 512, g["eb"], idx, val, zc)
        sweep[str(zc)] = timed(lambda: ctx.reconstruct(dec_codes, Lz, fout, stream))
    dec_ms = timed(lambda: ctx.decompress(field, L, fout, stream))
    ok = ok and ctx.status(stream) == 0
    f = g.get("field")
    bound_ok = None
    if f is not None:
        x = fout.cpu().numpy().astype(np.float64)
        fl = f.reshape(-1).astype(np.float64)
        bound_ok = bool(np.all(np.abs(x - fl) <= g["eb"] * (1 + 1e-6) + 2.0 ** -23 * np.abs(fl)))
    alg = 2 * n + 4 * n + 12 * int(g["out_idx"].size)
    peak, kind = measured_peak()
    return {"workload": f"{side}^3 codes of the decode workload -> float32, "
                        f"{g['out_idx'].size} outliers, abs. error bound {g['eb']:.6g}",
            "value": 4.0 * n / (dec_ms * 1e-3) / 1e9,
            "unit": "GB/s (float32 values out, decode + reconstruction)",
            "decompress_ms": dec_ms, "reconstruct_ms": recon_ms,
            "reconstruct_band_path_ms_by_slice_group": sweep,
            "reconstruct_roofline": {"bound": "hbm", "achieved": alg / (recon_ms * 1e-3) / 1e9,
                                     "peak": peak, "unit": "GB/s",
                                     "frac": alg / (recon_ms * 1e-3) / 1e9 / peak,
                                     "peak_kind": kind, "algorithmic_bytes": alg},
            "status_ok": bool(ok), "within_error_bound": bound_ok}


def run_decompress_1d(hd, torch, ctx_dev, stream, flush, steps: int = 5, n: int = 280_953_867):
    """Decode + reconstruction of a 1D field of the HACC particle count: the
    fused path (values straight from the decoder) against decode into codes
    then reconstruction, and the two halves alone."""
    import synth
    f1 = synth.fourier_field((n,), noise=1e-4, kmax=8, seed=1002)
    g = synth.lorenzo_quantize(f1, 1e-4, radius=512)
    del f1
    codes = g["codes"]
    lengths = hd.hd_build_codebook(codes, 1024, 32)
    enc = hd.hd_encode(codes, lengths, 128)
    dev = f"cuda:{ctx_dev}"
    f = hd.DeviceField.upload(enc, lengths, n, device=dev)
    idx = torch.from_numpy(g["out_idx"].view(np.int64)).to(dev)
    val = torch.from_numpy(g["out_val"]).to(dev)
    vals = torch.empty(n, dtype=torch.float32, device=dev)
    dec = torch.empty(n, dtype=torch.int16, device=dev)
    ctx = hd.Context(ctx_dev)
    launch = ctx.autotune([f], [dec], stream)

    def timed(fn):
        fn()
        ms = []
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    Lf = hd.lorenzo_params((n,), 512, g["eb"], idx, val)
    Ls = hd.lorenzo_params((n,), 512, g["eb"], idx, val, separate=True)
    fused = timed(lambda: ctx.decompress(f, Lf, vals, stream))
    ok = ctx.status(stream) == 0
    first = vals[:1 << 20].clone()
    separate = timed(lambda: ctx.decompress(f, Ls, vals, stream))
    ok = ok and ctx.status(stream) == 0 and bool(torch.equal(first, vals[:1 << 20]))
    decode = timed(lambda: ctx.decode(f, dec, stream))
    recon = timed(lambda: ctx.reconstruct(dec, Lf, vals, stream))
    ok = ok and ctx.status(stream) == 0
    ctx.close()
    return {"workload": f"{n} 1D codes (rel. error bound 1e-4, radius 512, "
                        f"{enc['nbits'] / n:.2f} bits/code, {g['out_idx'].size} outliers)",
            "value": 4.0 * n / (fused * 1e-3) / 1e9,
            "unit": "GB/s (float32 values out, fused decode + reconstruction)",
            "fused_ms": fused, "separate_ms": separate, "decode_ms": decode,
            "reconstruct_ms": recon, "launch": launch, "status_ok": bool(ok)}


def run_skew(hd, torch, ctx_dev, stream, flush, n: int = 1 << 26, steps: int = 5):
    """Decode throughput across compressibility: 1D fields (the same smooth
    generator, 8 Fourier modes to bound generation time) quantized at relative
    error bounds 1e-2 / 1e-4 / 1e-6 with alphabets 256 / 1024 / 4096, gap
    array (autotuned shape) and self-synchronisation."""
    import synth
    dev = f"cuda:{ctx_dev}"
    out = torch.empty(n, dtype=torch.int16, device=dev)
    peak, _ = measured_peak()
    res = []
    for rel_eb, alphabet in ((1e-2, 256), (1e-4, 1024), (1e-6, 4096)):
        f1 = synth.fourier_field((n,), noise=1e-4, kmax=8, seed=1002)
        codes, _, _ = synth.lorenzo_codes(f1, rel_eb, radius=alphabet // 2)
        del f1
        lengths = hd.hd_build_codebook(codes, alphabet, 32)
        enc = hd.hd_encode(codes, lengths, 128)
        f = hd.DeviceField.upload(enc, lengths, n, device=dev)
        fs = hd.DeviceField(f.words, f.nbits, None, 128, f.lengths, alphabet, n)
        ctx = hd.Context(ctx_dev)
        row = {"rel_eb": rel_eb, "alphabet": alphabet, "bits_per_code": enc["nbits"] / n}
        for name, field in (("gap", f), ("selfsync", fs)):
            ctx.reset_config()
            row[name + "_launch"] = ctx.autotune([field], [out], stream)
            ctx.decode(field, out, stream)
            ok = ctx.status(stream) == 0 and np.array_equal(out.cpu().numpy().view(np.uint16),
                                                              codes)
            ms = []
            for _ in range(steps):
                flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctx.decode(field, out, stream)
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            t = statistics.median(ms)
            row[name + "_ms"] = t
            row[name + "_gbps"] = 2.0 * n / (t * 1e-3) / 1e9
            # algorithmic bytes: stream in (+ one gap byte per 128 bits), codes out
            nb = (enc["nbits"] + 7) // 8 + 2 * n + (enc["nsub"] if name == "gap" else 0)
            row[name + "_hbm_frac"] = nb / (t * 1e-3) / 1e9 / peak
            row[name + "_ok"] = bool(ok and ctx.status(stream) == 0)
        ctx.close()
        res.append(row)
    return {"workload": f"{n} 1D codes per case, S=128 stream; GB/s of uint16 codes out",
            "cases": res}


def mixed_cr_workload(n_seg: int = 32, seg: int = 1 << 21, seed: int = 1005):
    """A 1D field whose compressibility changes along it (segments quantized at
    error bounds 1e-2 .. 1e-6), for the window-class ablation."""
    import synth
    ebs = [1e-2, 1e-6, 1e-3, 1e-5, 1e-2, 1e-4, 1e-6, 1e-2]
    return np.concatenate([synth.smooth_codes_1d(seg, ebs[k % 8], alphabet=1024, seed=seed + k)
                           for k in range(n_seg)])


def run_cr_ablation(hd, torch, ctx_dev, stream, flush, codes, steps: int = 5):
    """Algorithm 2 (per-tile compression-ratio window classes) against the
    autotuned single-window shape on a field of mixed compressibility."""
    n = codes.size
    lengths = hd.hd_build_codebook(codes, 1024, 32)
    enc = hd.hd_encode(codes, lengths, 128)
    f = hd.DeviceField.upload(enc, lengths, n, device=f"cuda:{ctx_dev}")
    out = torch.empty(n, dtype=torch.int16, device=f"cuda:{ctx_dev}")
    ctx = hd.Context(ctx_dev)
    best = ctx.autotune([f], [out], stream)

    def timed():
        ctx.decode(f, out, stream)
        assert ctx.status(stream) == 0
        assert np.array_equal(out.cpu().numpy().view(np.uint16), codes)
        ms = []
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.decode(f, out, stream)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    uniform = timed()
    res = {"workload": f"{n} 1D codes in 32 segments at rel. error bounds 1e-2..1e-6 "
                       f"({enc['nbits'] / n:.2f} bits/code overall), S=128 gap array",
           "autotuned": best, "uniform_ms": uniform}
    for classes in (4, 16):
        ctx.set_config(subseq_bits=best["subseq_bits"], threads=best["threads"],
                       lut_bits=best["lut_bits"], cr_classes=classes)
        res[f"cr_classes_{classes}_ms"] = timed()
    ctx.close()
    res["note"] = ("class launches include the host read-back of the class sizes "
                   "(a stream synchronisation) as Algorithm 2 does")
    return res


def run_batched(hd, torch, dev, stream, flush, fields_h, steps: int):
    """Config-3 leg: all fields in one graph launch (autotuned shape) against
    one hd_decode launch per field, same outputs."""
    import zlib
    fields = [hd.DeviceField.upload(f, f["lengths"], f["n"], device=f"cuda:{dev}")
              for f in fields_h]
    outs = [torch.empty(max(1, f["n"]), dtype=torch.int16, device=f"cuda:{dev}")
            for f in fields_h]
    total = sum(f["n"] for f in fields_h)
    ctx = hd.Context(dev)
    t0 = time.perf_counter()
    best = ctx.autotune(fields, outs, stream)
    tune_s = time.perf_counter() - t0
    bad = [k for k, (f, o) in enumerate(zip(fields_h, outs))
           if zlib.crc32(o[:f["n"]].cpu().numpy().tobytes()) != f["crc"]]

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    l0 = ctx.launch_count()
    ms_b = timed(lambda: ctx.decode_batch(fields, outs, stream))
    rc_b, _ = ctx.batch_status(len(fields), stream)
    launches_b = (ctx.launch_count() - l0) // (steps + 1)

    def per_field():
        for f, o in zip(fields, outs):
            ctx.decode(f, o, stream)
    ms_p = timed(per_field)
    st_p = ctx.status(stream)
    caps, cached = ctx.graph_stats()
    ctx.close()
    return {"value": 2.0 * total / (ms_b * 1e-3) / 1e9, "unit": "GB/s", "fields": len(fields_h),
            "codes": total, "ms_per_batch": ms_b, "kernels_per_batch": launches_b,
            "per_field": {"value": 2.0 * total / (ms_p * 1e-3) / 1e9, "unit": "GB/s",
                          "ms": ms_p, "status_last": st_p},
            "speedup_vs_per_field": ms_p / ms_b, "autotuned": best, "tune_s": tune_s,
            "graphs_captured": caps, "status": rc_b, "crc_mismatches": len(bad),
            "workload": "256 1D fields, codes log-uniform in [2^16, 2^26], alphabets "
                        "{256,1024,4096}, rel. error bound log-uniform in [1e-6, 1e-2], own "
                        "codebook each, S=128 gap arrays; L2 flushed between steps"}, fields


def serve_trace(hd, dev, fields, arrivals, ids, sizes, direct: bool, shape):
    """Replays one request trace through a server; returns throughput and
    latency percentiles (latency = submission to observed completion)."""
    srv = hd.Server(dev, budget_bytes=40 << 30, slots=1 if direct else 2,
                    max_batch=1 if direct else 64, direct=direct, shape=shape)
    fid = [srv.register(f) for f in fields]
    n_req = len(ids)
    lat = np.zeros(n_req)
    status_bad = 0
    tick_req = {}
    i = done = 0
    t0 = time.perf_counter()
    while done < n_req:
        now = time.perf_counter() - t0
        while i < n_req and arrivals[i] <= now:
            tick_req[srv.submit(fid[ids[i]])] = i
            i += 1
        for t in srv.completed():
            t = int(t)
            r = srv.poll(t)
            lat[tick_req.pop(t)] = r["latency_us"]
            status_bad += r["status"] != 0
            srv.release(t)
            done += 1
    span = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    out_bytes = 2.0 * float(np.sum(sizes[ids]))
    return {"throughput_gbps": out_bytes / span / 1e9, "requests_per_s": n_req / span,
            "p50_ms": float(np.percentile(lat, 50)) / 1e3,
            "p99_ms": float(np.percentile(lat, 99)) / 1e3, "span_s": span,
            "batches": st["batches"], "peak_budget_bytes": st["peak_bytes"],
            "bad_status": int(status_bad)}


def run_served(hd, dev, fields, batch_ms: float, n_req: int, shape):
    """Config-4 leg: Poisson arrivals at 0.8x the batched capacity over the
    resident pool, batched server vs one launch per request; both at
    saturation (all requests queued at once); and both at 0.8x the
    per-request server's capacity, a rate both sustain."""
    sizes = np.array([f.n for f in fields], dtype=np.float64)
    rng = np.random.default_rng(1004)
    ids = rng.integers(0, len(fields), size=n_req)
    capacity = len(fields) / (batch_ms * 1e-3)  # requests/s when decoding in full batches
    rate = 0.8 * capacity
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
    zero = np.zeros(n_req)
    out = {"requests": n_req, "arrival": "Poisson", "rate_rps": rate, "load": 0.8,
           "capacity_rps": capacity, "budget_bytes": 40 << 30,
           "pool": f"{len(fields)} resident fields of the batched workload"}
    out["batched"] = serve_trace(hd, dev, fields, arrivals, ids, sizes, False, shape)
    out["per_request"] = serve_trace(hd, dev, fields, arrivals, ids, sizes, True, None)
    out["saturated"] = {
        "batched": serve_trace(hd, dev, fields, zero, ids, sizes, False, shape),
        "per_request": serve_trace(hd, dev, fields, zero, ids, sizes, True, None)}
    # a load both servers sustain: 0.8x the per-request server's capacity
    # (measured at saturation), so both latencies are service, not queue growth
    cap_pr = out["saturated"]["per_request"]["requests_per_s"]
    rate_m = 0.8 * cap_pr
    arr_m = np.cumsum(np.random.default_rng(1014).exponential(1.0 / rate_m, size=n_req))
    out["matched_load"] = {
        "rate_rps": rate_m, "load": "0.8x per-request capacity", "per_request_capacity_rps": cap_pr,
        "batched": serve_trace(hd, dev, fields, arr_m, ids, sizes, False, shape),
        "per_request": serve_trace(hd, dev, fields, arr_m, ids, sizes, True, None)}
    m = out["matched_load"]
    m["p50_ratio_per_request_over_batched"] = m["per_request"]["p50_ms"] / max(
        1e-9, m["batched"]["p50_ms"])
    m["p99_ratio_per_request_over_batched"] = m["per_request"]["p99_ms"] / max(
        1e-9, m["batched"]["p99_ms"])
    out["value"] = out["batched"]["throughput_gbps"]
    out["unit"] = "GB/s"
    return out


def run_gpu(args):
    gen = None
    if not args.no_batch and _env_int("RANK", 0) == 0:
        gen = start_batch_generation(args.batch_fields, max(1, min(16, os.cpu_count() or 1)))
    import torch
    from paper_2201_09118_gb300 import hd

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    side = args.side
    quant = workload_quantized(side, seed=1001 + rank, keep_field=rank == 0)
    codes = quant["codes"]
    n = codes.size
    lengths = hd.hd_build_codebook(codes, 1024, 32)
    enc = hd.hd_encode(codes, lengths, 128)
    fields_h = None
    mixed_codes = mixed_cr_workload() if gen is not None else None
    if gen is not None:
        # the batched workload is encoded by the pool meanwhile; collect it
        # before anything is timed so that no host work overlaps a timing
        pool, res, order = gen
        got = res.get()
        pool.close()
        pool.join()
        fields_h = [None] * len(got)
        for k, f in zip(order, got):
            fields_h[k] = f
        del got
    field = hd.DeviceField.upload(enc, lengths, n, device=f"cuda:{dev}")
    field_ss = hd.DeviceField(field.words, field.nbits, None, 128, field.lengths, 1024, n)
    out = torch.empty(n, dtype=torch.int16, device=f"cuda:{dev}")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=f"cuda:{dev}")
    ctx = hd.Context(dev)
    if args.threads or args.window or args.lut_bits or args.subseq_bits or args.decoder:
        ctx.set_config(subseq_bits=args.subseq_bits, threads=args.threads, window=args.window,
                       lut_bits=args.lut_bits, decoder=args.decoder)
    stream = torch.cuda.current_stream()
    tuned = None
    if not (args.threads or args.window or args.lut_bits or args.subseq_bits or args.decoder):
        # launch shapes for this field's class, chosen by the library's autotuner
        t0 = time.perf_counter()
        tuned = {"gap": ctx.autotune([field], [out], stream),
                 "selfsync": ctx.autotune([field_ss], [out], stream)}
        tuned["seconds"] = time.perf_counter() - t0

    # correctness of the timed configuration (round trip against the codes)
    ctx.decode(field, out, stream)
    st = ctx.status(stream)
    ok = st == 0 and np.array_equal(out.cpu().numpy().view(np.uint16), codes)
    if not ok:
        print(json.dumps({"error": f"decode mismatch or status {st}"}), flush=True)
        return 1

    def timed(f, steps, warmup):
        for _ in range(warmup):
            ctx.decode(f, out, stream)
        torch.cuda.synchronize()
        ctx.profile(True)
        ctx.kernel_time()  # clear
        l0 = ctx.launch_count()
        evs = []
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for _ in range(steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ctx.decode(f, out, stream)
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        launches = ctx.launch_count() - l0
        kms, kl = ctx.kernel_time()
        ctx.profile(False)
        ms = sum(a.elapsed_time(b) for a, b in evs)
        st = ctx.status(stream)
        return ms, kms, kl, launches, st

    sampler = ClockSampler(dev)
    sampler.start()
    ms, kms, kl, launches, st = timed(field, args.steps, args.warmup)
    clocks = sampler.stop()
    launch_gap = ctx.get_config()
    if st != 0:
        print(json.dumps({"error": f"decode status {st} in timed region"}), flush=True)
        return 1
    ms_ss, kms_ss, kl_ss, _, st_ss = timed(field_ss, max(3, args.steps // 2), 2)
    launch_ss = ctx.get_config()
    encode_leg = run_encode(hd, torch, ctx, codes, lengths, enc, stream, flush)

    ms, ms_ss = ranks_max([ms, ms_ss], dist, f"cuda:{dev}")

    # end to end through the host-buffer entry point (pinned host memory)
    words_h = torch.from_numpy(enc["words"].view(np.int32)).pin_memory()
    gap_h = torch.from_numpy(enc["gap"]).pin_memory()
    len_h = torch.from_numpy(lengths).pin_memory()
    out_h = torch.empty(n, dtype=torch.int16).pin_memory()
    e2e_times = []
    e2e_steps = max(3, args.steps // 2)
    for k in range(2 + e2e_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc = ctx.decode_host_ptrs(words_h.data_ptr(), enc["nwords"], enc["nbits"],
                                  gap_h.data_ptr(), 128, len_h.data_ptr(), 1024, n,
                                  out_h.data_ptr(), stream)
        t1 = time.perf_counter()
        if rc != 0:
            print(json.dumps({"error": f"hd_decode_host status {rc}"}), flush=True)
            return 1
        if k >= 2:
            e2e_times.append(t1 - t0)
    assert np.array_equal(out_h.numpy().view(np.uint16), codes)
    e2e_gbps = ranks_min([2.0 * n / statistics.median(e2e_times) / 1e9], dist,
                         f"cuda:{dev}")[0] * world

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    extra = {}
    extra["decompress"] = run_decompress(hd, torch, ctx, field, out, quant, stream, flush)
    quant.pop("field", None)
    if fields_h is not None:
        extra["decompress_1d"] = run_decompress_1d(hd, torch, dev, stream, flush)
        extra["skew"] = run_skew(hd, torch, dev, stream, flush)
    if fields_h is not None:
        extra["cr_class_ablation"] = run_cr_ablation(hd, torch, dev, stream, flush, mixed_codes)
        batched, dev_fields = run_batched(hd, torch, dev, stream, flush, fields_h, 3)
        extra["batched"] = batched
        extra["served"] = run_served(hd, dev, dev_fields, batched["ms_per_batch"],
                                     args.requests, batched["autotuned"])

    nbytes_alg = (enc["nbits"] + 7) // 8 + enc["nsub"] + 2 * n
    traffic_key, kernel_label = DECODER_KERNELS[launch_gap.get("decoder", 1) or 1]
    kernel_ms = kms / max(1, kl)
    achieved = nbytes_alg / (kernel_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    value = whole_job_gbps(n, args.steps, world, ms)
    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u16", "data": "synthetic",
        "config": {"workload": workload_desc(side), "n_codes": n,
                   "bits_per_code": enc["nbits"] / n, "strategy": "gap array",
                   "l2": "flushed between steps (256 MiB write outside the timed events)",
                   "parallelism": f"replicas x{world}", "launch": launch_gap,
                   "autotuned": tuned},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": recorded_traffic(traffic_key, n, launch_gap),
                     "peak_kind": peak_kind, "kernel": kernel_label,
                     "kernel_ms": kernel_ms, "algorithmic_bytes": nbytes_alg},
        "e2e": {"value": e2e_gbps, "unit": "GB/s",
                "h2d_bytes_per_step": int(enc["nwords"] * 4 + enc["nsub"] + 1024),
                "d2h_bytes_per_step": int(2 * n)},
        "clocks": clocks,
        "gpu_launches": int(launches),
        "selfsync": {"value": whole_job_gbps(n, max(3, args.steps // 2), world, ms_ss),
                     "unit": "GB/s", "kernel_ms": kms_ss / max(1, kl_ss), "status": st_ss,
                     "launch": launch_ss,
                     # algorithmic bytes without a gap array: stream in, codes out
                     "roofline": roofline_of((enc["nbits"] + 7) // 8 + 2 * n,
                                             kms_ss / max(1, kl_ss), peak, peak_kind)},
    }
    line["encode"] = encode_leg
    line.update(extra)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(codes)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_profile_recon(args):
    """Reconstructs the workload's codes `steps` times after `warmup` (for
    profiler captures); prints one timing line, no bench line."""
    import torch
    from paper_2201_09118_gb300 import hd
    torch.cuda.set_device(0)
    g = workload_quantized(args.side, seed=1001)
    n = g["codes"].size
    codes = torch.from_numpy(g["codes"].view(np.int16)).cuda()
    idx = torch.from_numpy(g["out_idx"].view(np.int64)).cuda()
    val = torch.from_numpy(g["out_val"]).cuda()
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    ctx = hd.Context(0)
    side = args.side
    L = hd.lorenzo_params((side, side, side), 512, g["eb"], idx, val)
    for _ in range(args.warmup):
        ctx.reconstruct(codes, L, out)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        ctx.reconstruct(codes, L, out)
    b.record()
    b.synchronize()
    st = ctx.status()
    print(json.dumps({"profile_case": "recon", "n_codes": n,
                      "ms": a.elapsed_time(b) / max(1, args.steps), "ok": st == 0}), flush=True)
    return 0 if st == 0 else 1


def run_profile_fused1d(args, n: int = 280_953_867):
    """Fused decode + reconstruction of the 1D field of the decompress_1d leg,
    `steps` times after `warmup` (profiler captures); one timing line."""
    import synth
    import torch
    from paper_2201_09118_gb300 import hd
    torch.cuda.set_device(0)
    f1 = synth.fourier_field((n,), noise=1e-4, kmax=8, seed=1002)
    g = synth.lorenzo_quantize(f1, 1e-4, radius=512)
    del f1
    lengths = hd.hd_build_codebook(g["codes"], 1024, 32)
    enc = hd.hd_encode(g["codes"], lengths, 128)
    f = hd.DeviceField.upload(enc, lengths, n)
    idx = torch.from_numpy(g["out_idx"].view(np.int64)).cuda()
    val = torch.from_numpy(g["out_val"]).cuda()
    vals = torch.empty(n, dtype=torch.float32, device="cuda")
    ctx = hd.Context(0)
    if args.threads or args.window or args.lut_bits or args.subseq_bits:
        ctx.set_config(subseq_bits=args.subseq_bits, threads=args.threads, window=args.window,
                       lut_bits=args.lut_bits)
    L = hd.lorenzo_params((n,), 512, g["eb"], idx, val)
    for _ in range(args.warmup):
        ctx.decompress(f, L, vals)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        ctx.decompress(f, L, vals)
    b.record()
    b.synchronize()
    st = ctx.status()
    print(json.dumps({"profile_case": "fused1d", "n_codes": n,
                      "ms": a.elapsed_time(b) / max(1, args.steps), "ok": st == 0}), flush=True)
    return 0 if st == 0 else 1


def run_profile_case(args):
    """Decodes one strategy `steps` times after `warmup` (for profiler
    captures); prints one timing line, no bench line."""
    import torch
    from paper_2201_09118_gb300 import hd
    if args.profile_strategy == "recon":
        return run_profile_recon(args)
    if args.profile_strategy == "fused1d":
        return run_profile_fused1d(args)
    torch.cuda.set_device(0)
    codes = workload_codes(args.side, seed=1001)
    n = codes.size
    lengths = hd.hd_build_codebook(codes, 1024, 32)
    enc = hd.hd_encode(codes, lengths, 128)
    f = hd.DeviceField.upload(enc, lengths, n, with_gap=args.profile_strategy == "gap")
    out = torch.empty(n, dtype=torch.int16, device="cuda")
    ctx = hd.Context(0)
    if args.threads or args.window or args.lut_bits or args.subseq_bits or args.decoder:
        ctx.set_config(subseq_bits=args.subseq_bits, threads=args.threads, window=args.window,
                       lut_bits=args.lut_bits, decoder=args.decoder)
    for _ in range(args.warmup):
        ctx.decode(f, out)
    torch.cuda.synchronize()
    ctx.profile(True)
    ctx.kernel_time()
    for _ in range(args.steps):
        ctx.decode(f, out)
    ms, k = ctx.kernel_time()
    st = ctx.status()
    ok = st == 0 and np.array_equal(out.cpu().numpy().view(np.uint16), codes)
    print(json.dumps({"profile_case": args.profile_strategy, "n_codes": n,
                      "kernel_ms": ms / max(1, k), "ok": bool(ok)}), flush=True)
    return 0 if ok else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=512)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--window", type=int, default=0)
    ap.add_argument("--lut-bits", dest="lut_bits", type=int, default=0)
    ap.add_argument("--subseq-bits", dest="subseq_bits", type=int, default=0)
    ap.add_argument("--decoder", type=int, default=0,
                    help="gap-array decoder: 0 automatic, 1 two phases, 2 one pass")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched (256 fields) and served (request trace) legs")
    ap.add_argument("--batch-fields", dest="batch_fields", type=int, default=256)
    ap.add_argument("--requests", type=int, default=10000)
    ap.add_argument("--profile-strategy", choices=["gap", "selfsync", "recon", "fused1d"],
                    default=None,
                    help="decode one strategy (or reconstruct the decoded codes) only and "
                         "print its time (profiler runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_strategy:
        return run_profile_case(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
