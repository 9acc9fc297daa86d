"""Benchmark: TFHE gate bootstrapping throughput on GB300 (gate bootstraps/s).

Workload (one "step"): 65,536 independent NAND gate bootstraps, parameters n = 630,
N = 1024, k = 1, Bgbit = 10, lg = 3, basebit = 2, t = 8, keys from seed 0 and inputs
encrypting uniform bits under seed 1 -- the whole hot path per gate: pre-combination,
modulus switch, blind rotation (630 CMux external products), sample extraction, key
switch.  Keys and inputs are resident in HBM before the timed region; the inputs
(2 x 165 MB per step) exceed the 129 MB L2.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

COUNT = 65536
N_LWE, N_RING = 630, 1024
# Algorithmic 32-bit modular multiplications per blind-rotation step of one ciphertext:
# two NTT primes x (6 forward + 2 inverse length-1024 transforms x 5,120 butterflies +
# 12 x 1,024 pointwise products) = 2 x 53,248.
MODMUL_PER_STEP = 2 * ((6 + 2) * 5120 + 12 * 1024)
# Peak modmul rate from unit counts and clocks: 152 SMs x 2,070 MHz x 64 integer-multiply
# pipe slots per SM per clock / 4 slots per lazy Shoup product (y w and q p take one slot each,
# the multiply-high q = mulhi(y, w') two, as it runs at half rate).  The rate measured on GB300
# agrees: 16.0 Shoup products per SM per clock (bench_int_peaks.cu, `bench.py --int-peaks`).
SMS, MAX_MHZ, IMAD_PER_CLK_SM = 152, 2070.0, 64
SLOTS_PER_SHOUP = 4
PEAK_MODMUL_PER_S = SMS * MAX_MHZ * 1e6 * IMAD_PER_CLK_SM / SLOTS_PER_SHOUP
# Charging the multiply-high one slot only (3 per product) gives a higher, unreachable figure;
# reported as a labelled note.
PEAK_MODMUL_3_SLOT = SMS * MAX_MHZ * 1e6 * IMAD_PER_CLK_SM / 3
# Key switch (table gather-accumulate): algorithmic DRAM bytes per launch are the digit-pair
# table once plus the extracted inputs and the outputs; its own floor is shared-memory
# bandwidth, one 4-byte table read per output word and digit pair, 128 B/clock/SM.
KS_TABLE_BYTES = 1024 * 4 * 16 * 632 * 4
# Blind rotation: the transform-domain key once per launch (n x 2 primes x 6 rows x 2 x N
# words), plus per ciphertext its mod-switched inputs (632 u16) and its extracted sample
# (1028 u32).
BR_KEY_BYTES = N_LWE * 2 * 6 * 2 * N_RING * 4
BR_BYTES_PER_CT = 632 * 2 + 1028 * 4
BR_TRAFFIC_NOTE = ("dram__bytes_read.sum + dram__bytes_write.sum of one br_kernel launch on a small case "
                   "(profiles/traffic.json), scaled to this launch as key + per-ciphertext bytes x ciphertexts; "
                   "null once the kernel sources differ from the captured ones")
KS_SMEM_BYTES_PER_CT = 1024 * 4 * 632 * 4
SMEM_BYTES_PER_CLK_SM = 128


# Per-device cache of the autotuner's choices (lp_autotune_cached), beside the build outputs;
# --retune measures again whatever the cache holds (so every run launches the same kernels).
TUNING_CACHE = os.environ.get("LOCPIR_TUNING_CACHE", os.path.join(ROOT, "_build", "tuning.json"))
RETUNE = False


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dev(a):
    import torch
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a.view(np.int32) if a.dtype == np.uint32 else a).cuda()


def reduce_max(x: float, dist) -> float:
    """Maximum of x over all ranks (a time: the job takes as long as its slowest rank)."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, steps: int, max_seconds: float) -> float:
    """Whole-job units per second: every rank processes its own batch (weak scaling)."""
    return units_per_rank * world * steps / max_seconds


def rank_seed(rank: int) -> int:
    """Input seed of a rank's batch: seed 1 on rank 0 (the workload's own seed), distinct
    seeds on the others, so that ranks never duplicate work."""
    return 1 if rank == 0 else 1000 + rank


def setup_gpu(local: int, seed_keys: int = 0, seed_inputs: int = 1, count: int = COUNT):
    """Keys generated on the device from the seed-0 draws, inputs encrypted on the device."""
    import torch
    from paper_2407_19871_gb300 import build, locpir
    build.build()
    torch.cuda.set_device(local)
    p = locpir.params_default()
    d = synth.key_draws(seed_keys)
    bsk = torch.empty(p.n * 6 * 2 * p.N, dtype=torch.int32, device="cuda")
    ksk = torch.empty(p.N * 8 * 4 * (p.n + 1), dtype=torch.int32, device="cuda")
    s_dev, S_dev = _dev(d.s), _dev(d.S)
    locpir.lp_client_keygen_bsk(p, s_dev, S_dev, _dev(d.bsk_mask), _dev(d.bsk_noise), bsk)
    locpir.lp_client_keygen_ksk(p, s_dev, S_dev, _dev(d.ksk_mask), _dev(d.ksk_noise), ksk)
    ctx = locpir.Context(local)
    ctx.lp_load_bsk_device(bsk)
    ctx.lp_load_ksk_device(ksk)
    del bsk, ksk
    # launch policy measured on this GPU (or read from the per-device cache written by an earlier run)
    os.makedirs(os.path.dirname(TUNING_CACHE), exist_ok=True)
    ctx.tuning = ctx.lp_autotune_cached(TUNING_CACHE, force=RETUNE)
    ctx.split_max = ctx.tuning["split_max"]
    A, B = synth.nand_pairs(seed_inputs, count)
    cts = []
    for bits, off in ((A, 0), (B, count)):
        dr = synth.lwe_draws(seed_inputs, count, offset=off)
        out = torch.empty(count, p.n + 1, dtype=torch.int32, device="cuda")
        mu = np.where(bits == 1, 1 << 29, (1 << 32) - (1 << 29)).astype(np.uint32)
        locpir.lp_client_lwe_encrypt(p.n, s_dev, _dev(dr.mask), _dev(dr.noise), _dev(mu), out, count)
        cts.append(out)
    torch.cuda.synchronize()
    return ctx, p, s_dev, (A, B), cts


def locpir_throughput(ctx, p, s_dev, nq: int, seed: int = 2, executor: int = 0) -> dict:
    """LocPIR queries/s on the city-batch shape (l = 32 unsigned, one box, 256-bit service,
    half of the points inside): nq queries scheduled together and captured in a CUDA graph
    (lp_plan_locpir), with the per-level kernels (executor 0) or the persistent executor (1);
    one warm-up replay, one timed replay (CUDA events).  Every output is decrypted on the
    device and compared with the plaintext truth."""
    import torch
    from paper_2407_19871_gb300 import locpir
    ctx.lp_set_executor(executor)
    l, m = 32, 256
    qs = synth.city_batch(seed, nq, l, m)
    per_q = 2 * l + 4 * l + m
    bits = np.zeros(nq * per_q, np.uint8)
    for k, q in enumerate(qs):
        row = [synth.int_to_bits(q.x, l), synth.int_to_bits(q.y, l)] + \
              [synth.int_to_bits(v, l) for v in q.box] + [q.service]
        bits[k * per_q:(k + 1) * per_q] = np.concatenate(row)
    mu = np.where(bits == 1, 1 << 29, (1 << 32) - (1 << 29)).astype(np.uint32)
    W = p.n + 1
    ct = torch.empty(len(bits), W, dtype=torch.int32, device="cuda")
    step = 256 * per_q          # draws in slices of 256 queries bound the host memory
    for o in range(0, len(bits), step):
        e = min(o + step, len(bits))
        dr = synth.lwe_draws(seed, e - o, offset=o)
        locpir.lp_client_lwe_encrypt(p.n, s_dev, _dev(dr.mask), _dev(dr.noise), _dev(mu[o:e]), ct[o:e], e - o)
    out = torch.empty(nq * m, W, dtype=torch.int32, device="cuda")
    queries = []
    for k in range(nq):
        b = k * per_q
        queries.append(dict(l=l, is_signed=0, n_boxes=1, m=m, comb=locpir.LP_XOR_TREE, x=ct[b:b + l],
                            y=ct[b + l:b + 2 * l], boxes=ct[b + 2 * l:b + 6 * l], services=ct[b + 6 * l:b + per_q],
                            out_service=out[k * m:(k + 1) * m]))
    plan = ctx.lp_plan_locpir(queries)
    info = plan.lp_plan_info()
    st = torch.cuda.current_stream()
    plan.lp_plan_run(st)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    plan.lp_plan_run(st)
    e1.record(st)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) / 1e3
    ph = torch.empty(nq * m, dtype=torch.int32, device="cuda")
    locpir.lp_client_lwe_phase(p.n, s_dev, out, ph, nq * m)
    got = (ph.cpu().numpy() > 0).astype(np.uint8).reshape(nq, m)
    wrong = 0
    wrong_queries = []
    for k, q in enumerate(qs):
        x1, x2, y1, y2 = q.box
        inside = x1 <= q.x < x2 and y1 <= q.y < y2
        bad = int((got[k] != (q.service if inside else 0)).sum())
        wrong += bad
        if bad:
            wrong_queries.append(k)
    plan.lp_plan_destroy()
    ctx.lp_set_executor(locpir.LP_EXEC_LEVELS)
    # The comparators' chained MUX decides wrongly with probability ~1.9e-5 per decision, so a
    # batch of thousands of queries flips about one query's result now and then; the flipped
    # query is reported (tests/test_gpu_fullsize.py reproduces such a query with the oracle).
    return {"queries_per_s": nq / sec, "queries": nq, "seconds": sec,
            "executor": "persistent kernel" if executor else "per-level kernels",
            "blind_rotations_per_s": info["blind_rotations"] / sec, "blind_rotations": info["blind_rotations"],
            "kernels_per_run": info["kernels"], "wrong_bits": wrong, "wrong_queries": wrong_queries[:16],
            "shape": f"city batch: l=32 unsigned, 1 box, m=256, half the points inside (seed {seed}), "
                     "CUDA-graph plan"}


def single_query_latency(ctx, p, s_dev) -> dict:
    """The single-query workload: 16-bit unsigned fixed-point coordinates (Seoul's Table 1 box
    and a point inside it, shifted by +90 / +180 degrees, 7 fraction bits), one box, a 64-bit
    service holding 427, encrypted under the seed-0 keys with seed-0 draws.  Median time of
    lp_locpir_query over 3 runs after a warm-up; the decrypted service is checked."""
    import torch
    from paper_2407_19871_gb300 import locpir
    l, m = 16, 64
    enc = lambda deg: int(np.floor(deg * 128 + 0.5))
    box = (enc(37.4758 + 90), enc(37.6195 + 90), enc(126.8831 + 180), enc(127.1331 + 180))
    px, py = enc(37.55 + 90), enc(127.0 + 180)
    bits = np.concatenate([synth.int_to_bits(px, l), synth.int_to_bits(py, l)] +
                          [synth.int_to_bits(v, l) for v in box] + [synth.int_to_bits(427, m)])
    ct = _encrypt_bits(p, s_dev, bits, 0)
    out = torch.empty(m, p.n + 1, dtype=torch.int32, device="cuda")
    run = lambda: ctx.lp_locpir_query(l, 0, ct[:l], ct[l:2 * l], 1, ct[2 * l:6 * l], m, ct[6 * l:],
                                      locpir.LP_XOR_TREE, out)
    sec = _timed(run)
    ph = torch.empty(m, dtype=torch.int32, device="cuda")
    locpir.lp_client_lwe_phase(p.n, s_dev, out, ph, m)
    got = sum(int(b > 0) << j for j, b in enumerate(ph.cpu().numpy()))
    return {"ms_per_query": sec * 1e3, "blind_rotations": 12 * l + 3 + m, "result": got, "expected": 427,
            "shape": "1 query, l=16 unsigned, 1 box (Seoul), m=64, keys and draws seed 0"}


def known_bounds_throughput(ctx, p, s_dev, nq: int, seed: int = 5) -> dict:
    """City-shaped queries (l = 32 unsigned, one box, m = 256) evaluated twice through the
    batch entry points: with the box bounds encrypted (lp_locpir_batch) and known to the
    server (lp_locpir_known_batch).  Blind rotations counted from the circuits' gate counts
    as the library schedules them (MUX = 2); outputs decrypted and checked."""
    import torch
    from paper_2407_19871_gb300 import locpir
    l, m = 32, 256
    qs = synth.city_batch(seed, nq, l, m)
    per_q = 2 * l + 4 * l + m
    bits = np.concatenate([np.concatenate([synth.int_to_bits(q.x, l), synth.int_to_bits(q.y, l)] +
                                          [synth.int_to_bits(v, l) for v in q.box] + [q.service]) for q in qs])
    ct = _encrypt_bits(p, s_dev, bits, seed + 100)
    W = p.n + 1
    out_e = torch.empty(nq * m, W, dtype=torch.int32, device="cuda")
    out_k = torch.empty(nq * m, W, dtype=torch.int32, device="cuda")
    enc, known = [], []
    for k, q in enumerate(qs):
        b = k * per_q
        common = dict(l=l, is_signed=0, n_boxes=1, m=m, comb=locpir.LP_XOR_TREE, x=ct[b:b + l], y=ct[b + l:b + 2 * l],
                      services=ct[b + 6 * l:b + per_q])
        enc.append(dict(common, boxes=ct[b + 2 * l:b + 6 * l], out_service=out_e[k * m:(k + 1) * m]))
        known.append(dict(common, bounds=[q.box], out_service=out_k[k * m:(k + 1) * m]))
    t_enc = _timed(lambda: ctx.lp_locpir_batch(enc), reps=1)
    t_known = _timed(lambda: ctx.lp_locpir_known_batch(known), reps=1)
    wrong = 0
    for out in (out_e, out_k):
        ph = torch.empty(nq * m, dtype=torch.int32, device="cuda")
        locpir.lp_client_lwe_phase(p.n, s_dev, out, ph, nq * m)
        got = (ph.cpu().numpy() > 0).astype(np.uint8).reshape(nq, m)
        for k, q in enumerate(qs):
            x1, x2, y1, y2 = q.box
            wrong += int((got[k] != (q.service if (x1 <= q.x < x2 and y1 <= q.y < y2) else 0)).sum())

    def known_br(K: int) -> int:
        # comp_s_known: one gate per bit after the first set bit (unsigned)
        return 0 if K == 0 else l - 1 - (K & -K).bit_length() + 1

    br_known = sum(sum(known_br(v) for v in q.box) + 3 + m for q in qs)
    return {"experiment": "known_bounds", "queries": nq, "l": l, "m": m,
            "encrypted_bounds_queries_per_s": nq / t_enc, "known_bounds_queries_per_s": nq / t_known,
            "encrypted_bounds_blind_rotations": nq * (12 * l + 3 + m), "known_bounds_blind_rotations": br_known,
            "wrong_bits": wrong}


def engines_bench(count: int, ks_count: int) -> None:
    """Head-to-head of the product engines on NAND gates: the NTT blind rotation against the
    bf16 and int8 Toeplitz GEMM engines (count gates each), and the digit-pair table key switch
    against the int8 one-hot GEMM (ks_count gates).  Per engine: bootstraps/s from the library's
    CUDA events around its blind-rotation (or key-switch) work, the GEMM rate that implies, and
    the decrypted outputs checked.  Prints one JSON line per engine."""
    import torch
    from paper_2407_19871_gb300 import locpir
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    n = 630
    # GEMM operations per blind rotation: per CMux step 2 M (K + (W - 1) 2K), M = 2N, K = 6N.
    M, K = 2048, 6144
    gemm_ops = {1: 2 * M * (K + 5 * 2 * K) * n, 2: 2 * M * (K + 3 * 2 * K) * n}
    ctx, p, s_dev, (A, B), (a, b) = setup_gpu(0, count=max(count, ks_count))
    out = torch.empty_like(a)
    for br, name in ((0, "ntt"), (1, "tensor_bf16"), (2, "tensor_int8")):
        ctx.lp_set_engines(br, 0)
        ctx.lp_gate_batch(locpir.LP_NAND, a[:8], b[:8], None, out[:8], 8)   # warm-up (cuBLAS, scratch)
        ctx.lp_sync()
        ctx.lp_set_timing(True)
        ctx.lp_reset_timing()
        ctx.lp_gate_batch(locpir.LP_NAND, a[:count], b[:count], None, out[:count], count)
        ctx.lp_sync()
        ms, _ = ctx.lp_kernel_time("br")
        ctx.lp_set_timing(False)
        wrong = check_outputs(p, s_dev, out[:count], A[:count], B[:count])
        line = {"experiment": "engines", "stage": "blind_rotation", "engine": name, "gates": count,
                "ms": ms, "bootstraps_per_s": count / (ms / 1e3), "decrypt_errors": wrong}
        if br:
            ops = gemm_ops[br] * count / (ms / 1e3)
            line["gemm_rate"] = ops / 1e12
            line["gemm_unit"] = "TFLOP/s" if br == 1 else "TOPS"
            if br == 1 and "bf16_tflops" in peaks:
                line["frac_of_measured_bf16_peak"] = ops / 1e12 / peaks["bf16_tflops"]
        print(json.dumps(line), flush=True)
    for ks, name in ((0, "table"), (1, "tensor_int8_onehot")):
        ctx.lp_set_engines(0, ks)
        ctx.lp_gate_batch(locpir.LP_NAND, a[:8], b[:8], None, out[:8], 8)
        ctx.lp_sync()
        ctx.lp_set_timing(True)
        ctx.lp_reset_timing()
        ctx.lp_gate_batch(locpir.LP_NAND, a[:ks_count], b[:ks_count], None, out[:ks_count], ks_count)
        ctx.lp_sync()
        ms, _ = ctx.lp_kernel_time("ks")
        ctx.lp_set_timing(False)
        wrong = check_outputs(p, s_dev, out[:ks_count], A[:ks_count], B[:ks_count])
        line = {"experiment": "engines", "stage": "key_switch", "engine": name, "gates": ks_count, "ms": ms,
                "key_switches_per_s": ks_count / (ms / 1e3), "decrypt_errors": wrong}
        if ks:
            line["gemm_rate"] = 2 * 4 * 632 * 24576 * ks_count / (ms / 1e3) / 1e12
            line["gemm_unit"] = "TOPS"
        print(json.dumps(line), flush=True)
    ctx.lp_set_engines(0, 0)
    ctx.close()


def br_latency_bench() -> None:
    """Blind-rotation time per launch against the level width, for the batched kernel (4
    ciphertexts per CTA), the split kernel (one ciphertext per CTA over 12 warps), the paired
    kernel (one ciphertext per cluster of two CTAs, one per NTT prime) and the quad kernel (four
    CTAs: prime x ACC component): CUDA
    events around the library's blind-rotation launches, median of 3 after a warm-up, outputs
    decrypted.  One JSON line per (kernel, width)."""
    from paper_2407_19871_gb300 import locpir
    import torch
    widths = (1, 4, 16, 64, 152, 304, 608, 1216)
    ctx, p, s_dev, (A, B), (a, b) = setup_gpu(0, count=max(widths))
    out = torch.empty_like(a)
    for eng, name in ((locpir.LP_BR_NTT_BATCHED, "batched"), (locpir.LP_BR_NTT_SPLIT, "split"),
                      (locpir.LP_BR_NTT_PAIR, "pair"), (locpir.LP_BR_NTT_QUAD, "quad")):
        ctx.lp_set_engines(eng, 0)
        for w in widths:
            ctx.lp_gate_batch(locpir.LP_NAND, a[:w], b[:w], None, out[:w], w)
            ctx.lp_sync()
            ts, tk = [], []
            for _ in range(3):
                ctx.lp_set_timing(True)
                ctx.lp_reset_timing()
                ctx.lp_gate_batch(locpir.LP_NAND, a[:w], b[:w], None, out[:w], w)
                ctx.lp_sync()
                ts.append(ctx.lp_kernel_time("br")[0])
                tk.append(ctx.lp_kernel_time("ks")[0])
                ctx.lp_set_timing(False)
            ms = float(np.median(ts))
            wrong = check_outputs(p, s_dev, out[:w], A[:w], B[:w])
            print(json.dumps({"experiment": "br_latency", "kernel": name, "ciphertexts": w, "br_ms": ms,
                              "bootstraps_per_s": w / (ms / 1e3), "ks_ms": float(np.median(tk)),
                              "decrypt_errors": wrong}), flush=True)
    ctx.lp_set_engines(0, 0)
    ctx.close()


def int_peaks() -> int:
    """Build and run bench_int_peaks.cu, the integer-pipe throughput microbenchmark behind the
    "alu" roofline's peak: one JSON line of operations per SM per clock for each pattern."""
    from paper_2407_19871_gb300.build import ARCH, nvcc
    out_dir = os.path.join(ROOT, "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "bench_int_peaks")
    subprocess.check_call([nvcc(), os.path.join(ROOT, "bench_int_peaks.cu"), "-o", exe, "-O3"] + ARCH)
    return subprocess.call([exe])


def check_outputs(p, s_dev, out, A, B) -> int:
    import torch
    from paper_2407_19871_gb300 import locpir
    ph = torch.empty(out.shape[0], dtype=torch.int32, device="cuda")
    locpir.lp_client_lwe_phase(p.n, s_dev, out, ph, out.shape[0])
    bits = (ph.cpu().numpy() > 0).astype(np.uint8)
    return int((bits != (1 - (A & B))).sum())


def cpu_baseline(seconds_target: float = 15.0) -> dict:
    """The oracle as it stands, on all host cores, on the first S gates of the workload."""
    import oracle
    keys = oracle.keygen(synth.key_draws(0))
    cores = oracle.threads()
    A, B = synth.nand_pairs(1, COUNT)
    # calibrate with one gate per core, then size the sample to ~seconds_target
    S0 = cores
    a = oracle.encrypt(keys.s, A[:S0], synth.lwe_draws(1, S0))
    b = oracle.encrypt(keys.s, B[:S0], synth.lwe_draws(1, S0, offset=COUNT))
    t0 = time.perf_counter()
    oracle.gate_batch(keys, oracle.NAND, a, b, nthreads=cores)
    dt0 = time.perf_counter() - t0
    S = max(cores, min(COUNT, int(cores * max(1, round(seconds_target / max(dt0, 1e-3))))))
    a = oracle.encrypt(keys.s, A[:S], synth.lwe_draws(1, S))
    b = oracle.encrypt(keys.s, B[:S], synth.lwe_draws(1, S, offset=COUNT))
    t0 = time.perf_counter()
    oracle.gate_batch(keys, oracle.NAND, a, b, nthreads=cores)
    dt = time.perf_counter() - t0
    # the same oracle on one thread, on the first few gates
    S1 = 4
    t0 = time.perf_counter()
    oracle.gate_batch(keys, oracle.NAND, a[:S1], b[:S1], nthreads=1)
    dt1 = time.perf_counter() - t0
    return {"value": S / dt, "unit": "bootstraps/s", "cores": cores, "kind": "oracle",
            "sample": f"first {S} of the 65,536 NAND gates (OpenMP over gates, {cores} threads), {dt:.1f} s",
            "single_thread_value": S1 / dt1,
            "single_thread_sample": f"first {S1} gates on 1 thread, {dt1:.1f} s"}


def kernel_source_sha256(spec: list[str]) -> str:
    """SHA-256 of the sources a kernel is built from.  An entry "path#marker" takes the file's
    text before the first line that starts with marker (the kernel's part of a larger file)."""
    import hashlib
    h = hashlib.sha256()
    for entry in spec:
        path, _, marker = entry.partition("#")
        text = open(os.path.join(ROOT, path), "rb").read()
        if marker:
            cut = text.find(("\n" + marker).encode())
            text = text[:cut + 1] if cut >= 0 else text
        h.update(text)
    return h.hexdigest()


def br_traffic(count: int):
    """DRAM bytes of one blind-rotation launch over `count` ciphertexts, from the small-case
    ncu capture recorded in profiles/traffic.json: the key once, plus the capture's bytes per
    ciphertext beyond the key times `count`.  None once the kernel sources differ from the
    ones the counters were taken on."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f)
        if kernel_source_sha256(rec["source_files"]) != rec["source_sha256"]:
            return None
        small = rec["br_kernel"]["small_case"]
        per_ct = (small["dram_bytes"] - BR_KEY_BYTES) / small["ciphertexts"]
        return int(BR_KEY_BYTES + per_ct * count)
    except Exception:
        return None


def _measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ---------------------------------------------------------------------------------------
# Paper experiment shapes on the GPU (Table 2, Fig. 4(a), Fig. 5's parallel width).
# ---------------------------------------------------------------------------------------
def _fixed(deg: float, frac: int) -> int:
    """Section 4.1's fixed-point encoding: 9 integer bits, `frac` fraction bits, rounded half
    away from zero (two's complement in l = 9 + frac bits)."""
    v = deg * (1 << frac)
    return int(np.floor(abs(v) + 0.5)) * (1 if v >= 0 else -1)


def _encrypt_bits(p, s_dev, bits: np.ndarray, seed: int):
    import torch
    from paper_2407_19871_gb300 import locpir
    dr = synth.lwe_draws(seed, len(bits), synth.Params(n=p.n))
    mu = np.where(bits == 1, 1 << 29, (1 << 32) - (1 << 29)).astype(np.uint32)
    ct = torch.empty(len(bits), p.n + 1, dtype=torch.int32, device="cuda")
    locpir.lp_client_lwe_encrypt(p.n, s_dev, _dev(dr.mask), _dev(dr.noise), _dev(mu), ct, len(bits))
    return ct


def _keys_for(n: int):
    """Device keys for LWE dimension n (seed 0), loaded into a fresh context."""
    import torch
    from paper_2407_19871_gb300 import locpir
    p = locpir.params_default()
    p.n = n
    d = synth.key_draws(0, synth.Params(n=n))
    bsk = torch.empty(p.n * 6 * 2 * p.N, dtype=torch.int32, device="cuda")
    ksk = torch.empty(p.N * 8 * 4 * (p.n + 1), dtype=torch.int32, device="cuda")
    s_dev = _dev(d.s)
    locpir.lp_client_keygen_bsk(p, s_dev, _dev(d.S), _dev(d.bsk_mask), _dev(d.bsk_noise), bsk)
    locpir.lp_client_keygen_ksk(p, s_dev, _dev(d.S), _dev(d.ksk_mask), _dev(d.ksk_noise), ksk)
    ctx = locpir.Context(0, p)
    ctx.lp_load_bsk_device(bsk)
    ctx.lp_load_ksk_device(ksk)
    os.makedirs(os.path.dirname(TUNING_CACHE), exist_ok=True)
    ctx.tuning = ctx.lp_autotune_cached(TUNING_CACHE)
    ctx.split_max = ctx.tuning["split_max"]
    return ctx, p, s_dev


def _timed(fn, reps: int = 3) -> float:
    """Median seconds of `reps` runs of fn after one untimed run (which sizes the scratch)."""
    import torch
    fn()
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    return float(np.median(ts))


def _random_query_time(ctx, p, s_dev, l: int, nb: int, m: int, seed: int) -> tuple[float, int]:
    """One unsigned LocPIR query (XOR tree) with nb random boxes of l-bit bounds, a random point
    and m-bit services: median seconds of lp_locpir_query (after a warm-up run) and the number
    of service bits that decrypt wrongly against the plaintext truth."""
    import torch
    from paper_2407_19871_gb300 import locpir
    L = 1 << l
    d = synth.splitmix64(4, seed, 4 * nb + 2)
    boxes = []
    for b in range(nb):
        x1, x2 = sorted(int(v) % L for v in d[4 * b:4 * b + 2])
        y1, y2 = sorted(int(v) % L for v in d[4 * b + 2:4 * b + 4])
        boxes.append((x1, x2, y1, y2))
    px, py = int(d[4 * nb]) % L, int(d[4 * nb + 1]) % L
    svc = synth.bits(4, seed, nb * m).reshape(nb, m)
    bits = np.concatenate([synth.int_to_bits(px, l), synth.int_to_bits(py, l)] +
                          [synth.int_to_bits(v, l) for b in boxes for v in b] + [svc.reshape(-1)])
    ct = _encrypt_bits(p, s_dev, bits, seed + 1)
    W = p.n + 1
    out = torch.empty(m, W, dtype=torch.int32, device="cuda")
    run = lambda: ctx.lp_locpir_query(l, 0, ct[:l], ct[l:2 * l], nb, ct[2 * l:2 * l + 4 * l * nb], m,
                                      ct[2 * l + 4 * l * nb:], locpir.LP_XOR_TREE, out)
    sec = _timed(run)
    want = np.zeros(m, np.uint8)
    for (x1, x2, y1, y2), sv in zip(boxes, svc):
        if x1 <= px < x2 and y1 <= py < y2:
            want ^= sv
    ph = torch.empty(m, dtype=torch.int32, device="cuda")
    locpir.lp_client_lwe_phase(p.n, s_dev, out, ph, m)
    wrong = int(((ph.cpu().numpy() > 0).astype(np.uint8) != want).sum())
    return sec, wrong


def paper_shapes(table2_only: bool = False) -> None:
    import torch
    from paper_2407_19871_gb300 import locpir
    table = json.load(open(os.path.join(ROOT, "tests", "golden", "table1.json")))["rows"]
    m = 9
    # Table 2: m = B_x = 9 over Table 1's cities; l = 13 (4 fraction bits) and 16 (7 bits);
    # 80-bit (n = 540) and 128-bit (n = 630) LWE dimensions.  The point is Seoul's centre.
    for n in (540, 630):
        ctx, p, s_dev = _keys_for(n)
        W = p.n + 1
        for l in (13, 16):
            frac = l - 9
            enc = lambda v: synth.int_to_bits(v, l)
            boxes = [tuple(_fixed(r[k], frac) for k in ("lat1", "lat2", "lon1", "lon2")) for r in table]
            px = _fixed((table[0]["lat1"] + table[0]["lat2"]) / 2, frac)
            py = _fixed((table[0]["lon1"] + table[0]["lon2"]) / 2, frac)
            bits = np.concatenate([enc(px), enc(py)] + [enc(v) for b in boxes for v in b] +
                                  [synth.int_to_bits(r["service"], m) for r in table])
            ct = _encrypt_bits(p, s_dev, bits, 7)
            x, y = ct[:l], ct[l:2 * l]
            bx = ct[2 * l:2 * l + 36 * l]
            sv = ct[2 * l + 36 * l:]
            out = torch.empty(m, W, dtype=torch.int32, device="cuda")
            run = lambda: ctx.lp_locpir_query(l, 1, x, y, 9, bx, m, sv, locpir.LP_XOR_CHAIN, out)
            total = _timed(run)
            # Phases, each batch timed on its own, with the gate counts and depths of the query's own
            # phases: the 36 comparators (4 per box) as one batch (LT(a, b) = NOT LE(b, a), and NOT
            # costs no bootstrap), validation (3 ANDs per box, 2 levels), services (9 x 9 bitwise
            # AND) and the 9 levels of the XOR chain (Algorithm 4 starts from S = Enc(0)^m, so box 1's
            # services are XORed into the trivial zero too).
            cx1 = bx.view(9, 4, l, W)
            pt = torch.cat([x.expand(9, l, W), y.expand(9, l, W)]).reshape(-1, W)
            a_le = torch.cat([cx1[:, 0], cx1[:, 2], cx1[:, 1], cx1[:, 3]]).reshape(-1, W).contiguous()
            b_le = torch.cat([pt, pt]).contiguous()
            cmp_out = torch.empty(36, W, dtype=torch.int32, device="cuda")
            t_cmp = _timed(lambda: ctx.lp_compare_batch(locpir.LP_LE, 1, l, a_le, b_le, cmp_out, 36))
            # The phase inputs are real encryptions of random bits: a zero or garbage mask would
            # let the blind rotation skip its steps (abar_i = 0) and time too little work.
            g = _encrypt_bits(p, s_dev, synth.bits(9, 1, 27), 9)
            t_val = _timed(lambda: (ctx.lp_gate_batch(locpir.LP_AND, g[:18], g[9:27], None, g[:18].clone(), 18),
                                    ctx.lp_gate_batch(locpir.LP_AND, g[:9], g[9:18], None, g[18:27].clone(), 9)))
            svc = _encrypt_bits(p, s_dev, synth.bits(9, 2, 81), 10)
            t_svc = _timed(lambda: ctx.lp_gate_batch(locpir.LP_AND, svc, svc, None, svc.clone(), 81))
            t_xor = _timed(lambda: [ctx.lp_gate_batch(locpir.LP_XOR, svc[:9], svc[9:18], None, svc[18:27].clone(), 9)
                                    for _ in range(9)])
            ph = torch.empty(m, dtype=torch.int32, device="cuda")
            locpir.lp_client_lwe_phase(p.n, s_dev, out, ph, m)
            got = sum(int(b > 0) << j for j, b in enumerate(ph.cpu().numpy()))
            print(json.dumps({"experiment": "table2", "n": n, "l": l, "m": m, "boxes": 9, "seconds_total": total,
                              "seconds_comparison": t_cmp, "seconds_validation": t_val,
                              "seconds_service_and": t_svc, "seconds_addxor_chain": t_xor,
                              "result": got, "expected": table[0]["service"],
                              "paper_seconds_total": {(540, 13): 4.36, (630, 13): 4.88, (540, 16): 5.12,
                                                      (630, 16): 5.67}[(n, l)],
                              "paper_hardware": "Ryzen 5 3500X, TFHE library v1.1 (Table 2)"}), flush=True)
        if n == 630 and not table2_only:
            # Fig. 4(a): time against (B_x, l) at m = 9; the paper prints its B_x = 10 row.
            paper4a = {8: 3.256, 16: 6.139, 24: 8.764, 32: 11.670}
            for nb in (2, 4, 6, 8, 10, 16, 28):
                for l in (8, 16, 24, 32):
                    sec, wrong = _random_query_time(ctx, p, s_dev, l, nb, m, seed=100 * nb + l)
                    line = {"experiment": "fig4a", "l": l, "boxes": nb, "m": m, "seconds": sec, "wrong_bits": wrong}
                    if nb == 10:
                        line.update(paper_seconds=paper4a[l], paper_hardware="Ryzen 5 3500X, 6 threads (Section 6.2)")
                    print(json.dumps(line), flush=True)
            # Fig. 4(b): time against (m, B_x) at l = 16.
            for nb in (2, 10, 28):
                for mm in (9, 32, 64, 128):
                    sec, wrong = _random_query_time(ctx, p, s_dev, 16, nb, mm, seed=7000 + 100 * nb + mm)
                    print(json.dumps({"experiment": "fig4b", "l": 16, "boxes": nb, "m": mm, "seconds": sec,
                                      "wrong_bits": wrong}), flush=True)
            # One query with a single box: l = 16, m = 64.
            sec, wrong = _random_query_time(ctx, p, s_dev, 16, 1, 64, seed=9164)
            print(json.dumps({"experiment": "single_query", "l": 16, "boxes": 1, "m": 64, "seconds": sec,
                              "wrong_bits": wrong}), flush=True)
            # Server-known bounds (beyond the paper) against encrypted bounds, same city batch.
            for nq in (152, 608):
                print(json.dumps(known_bounds_throughput(ctx, p, s_dev, nq)), flush=True)
            # Fig. 5's parallel width on the GPU: queries per batch (city shape) -> queries/s.
            for nq in (1, 8, 64, 152, 304, 4096):
                r = locpir_throughput(ctx, p, s_dev, nq, seed=2)
                print(json.dumps({"experiment": "batch_width", "queries": nq, "queries_per_s": r["queries_per_s"],
                                  "seconds": r["seconds"], "wrong_bits": r["wrong_bits"],
                                  "wrong_queries": r["wrong_queries"]}), flush=True)
        ctx.close()


# ---------------------------------------------------------------------------------------
# The multi-box uneven batch: 1,024 queries, B_x ~ U{1..128}, l ~ U{16, 24, 32}, m = 512,
# per-box results combined by an encrypted OR tree, run in memory-budgeted waves.
# ---------------------------------------------------------------------------------------
def multibox_uneven(args) -> None:
    """Queries from synth.multibox_batch(3, nq) (m = 512).  Input ciphertexts are gathered on the
    device from a pool of 65,536 fresh encryptions of random bits (synth draws, seed 3): each
    input bit of a query takes a pool ciphertext of the same bit, so every blind rotation runs all
    of its steps on a real encryption.  Queries go to lp_locpir_batch_waves in chunks whose
    inputs are gathered before the chunk's timed region; each chunk runs in waves whose circuits
    fit the memory budget.  Every output bit is decrypted and checked against the plaintext
    truth (OR of the services of the boxes holding the point).  One JSON line."""
    import torch
    from paper_2407_19871_gb300 import locpir
    ctx, p, s_dev, _, _ = setup_gpu(0, count=1)
    W = p.n + 1
    nq, m = args.multibox_queries, 512
    qs = synth.multibox_batch(3, nq, m=m)
    P = 1 << 16
    pool_bits = synth.bits(3, 900, P)
    pool = _encrypt_bits(p, s_dev, pool_bits, 3)
    zeros, ones = np.flatnonzero(pool_bits == 0), np.flatnonzero(pool_bits == 1)
    total_br = sum(locpir.lp_circuit_info(q.l, 0, len(q.boxes), m, locpir.LP_OR_TREE)["blind_rotations"] for q in qs)
    budget = int(args.multibox_budget_gb * 2**30)
    ctx.lp_set_executor(locpir.LP_EXEC_PERSISTENT if args.multibox_executor == "persistent" else locpir.LP_EXEC_LEVELS)
    ctx.lp_reset_timing()
    ctx.lp_set_timing(True)
    seconds, waves, wrong_bits, wrong_queries, chunks = 0.0, 0, 0, [], 0
    k0 = 0
    while k0 < nq:
        # a chunk: queries whose gathered inputs fit the input budget
        k1, cnt = k0, 0
        while k1 < nq:
            q = qs[k1]
            c = 2 * q.l + len(q.boxes) * (4 * q.l + m)
            if k1 > k0 and (cnt + c) * W * 4 > args.multibox_input_gb * 2**30:
                break
            cnt += c
            k1 += 1
        bits = np.concatenate([np.concatenate([synth.int_to_bits(q.x, q.l), synth.int_to_bits(q.y, q.l)] +
                                              [synth.int_to_bits(v, q.l) for b in q.boxes for v in b] +
                                              [np.asarray(q.services, np.uint8).reshape(-1)]) for q in qs[k0:k1]])
        h = (np.arange(len(bits), dtype=np.uint64) * np.uint64(2654435761) + np.uint64(977 * k0)) % np.uint64(1 << 32)
        idx = np.where(bits == 1, ones[h % np.uint64(len(ones))], zeros[h % np.uint64(len(zeros))])
        ct = pool.index_select(0, torch.from_numpy(idx.astype(np.int64)).cuda())
        out = torch.empty((k1 - k0) * m, W, dtype=torch.int32, device="cuda")
        batch, off = [], 0
        for j, q in enumerate(qs[k0:k1]):
            l, nb = q.l, len(q.boxes)
            c = 2 * l + nb * (4 * l + m)
            d = ct[off:off + c]
            batch.append(dict(l=l, is_signed=0, n_boxes=nb, m=m, comb=locpir.LP_OR_TREE, x=d[:l], y=d[l:2 * l],
                              boxes=d[2 * l:2 * l + 4 * l * nb], services=d[2 * l + 4 * l * nb:],
                              out_service=out[j * m:(j + 1) * m]))
            off += c
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        waves += ctx.lp_locpir_batch_waves(batch, budget)
        torch.cuda.synchronize()
        seconds += time.perf_counter() - t0
        ph = torch.empty(out.shape[0], dtype=torch.int32, device="cuda")
        locpir.lp_client_lwe_phase(p.n, s_dev, out, ph, out.shape[0])
        got = (ph.cpu().numpy() > 0).astype(np.uint8).reshape(k1 - k0, m)
        for j, q in enumerate(qs[k0:k1]):
            want = np.zeros(m, np.uint8)
            for (x1, x2, y1, y2), sv in zip(q.boxes, np.asarray(q.services, np.uint8).reshape(-1, m)):
                if x1 <= q.x < x2 and y1 <= q.y < y2:
                    want |= sv
            bad = int((got[j] != want).sum())
            wrong_bits += bad
            if bad:
                wrong_queries.append(k0 + j)
        del ct, out, batch
        chunks += 1
        k0 = k1
    br_ms, _ = ctx.lp_kernel_time("br")
    ks_ms, _ = ctx.lp_kernel_time("ks")
    ex_ms, _ = ctx.lp_kernel_time("exec")
    ctx.lp_set_timing(False)
    hist = {}
    for q in qs:
        hist[q.l] = hist.get(q.l, 0) + 1
    print(json.dumps({"experiment": "multibox_uneven", "executor": args.multibox_executor, "queries": nq, "m": m,
                      "comb": "OR tree",
                      "boxes_mean": float(np.mean([len(q.boxes) for q in qs])), "widths": hist,
                      "blind_rotations": total_br, "seconds": seconds, "queries_per_s": nq / seconds,
                      "blind_rotations_per_s": total_br / seconds, "br_kernel_s": br_ms / 1e3, "ks_kernel_s": ks_ms / 1e3, "exec_kernel_s": ex_ms / 1e3,
                      "chunks": chunks, "waves": waves, "memory_budget_gb": args.multibox_budget_gb,
                      "wrong_bits": wrong_bits, "wrong_queries": len(wrong_queries),
                      "wrong_query_ids": wrong_queries[:32], "autotune": ctx.tuning}), flush=True)
    ctx.close()


# ---------------------------------------------------------------------------------------
# Serving: Poisson arrivals into the query server (continuous batching).
# ---------------------------------------------------------------------------------------
def serve(args) -> None:
    import torch
    from paper_2407_19871_gb300 import locpir
    ctx, p, s_dev, _, _ = setup_gpu(0, count=1)
    W = p.n + 1
    rng = np.random.default_rng(4)
    if args.serve_shape == "uneven":
        # uneven multi-box queries: B_x ~ U{1..128}, l ~ U{16, 24, 32}, m = 512
        protos = synth.multibox_batch(4, args.serve_distinct, m=512)
        specs = [(q.l, q.x, q.y, q.boxes, q.services) for q in protos]
    else:
        protos = synth.city_batch(4, args.serve_distinct, 32, 256)
        specs = [(32, q.x, q.y, [q.box], q.service[None, :]) for q in protos]
    queries, expect = [], []
    for k, (l, x, y, boxes, services) in enumerate(specs):
        bits = np.concatenate([synth.int_to_bits(x, l), synth.int_to_bits(y, l)] +
                              [synth.int_to_bits(v, l) for b in boxes for v in b] +
                              [np.asarray(services, np.uint8).reshape(-1)])
        ct = _encrypt_bits(p, s_dev, bits, 40 + k)
        nb, m = len(boxes), np.asarray(services).shape[-1]
        queries.append(dict(l=l, is_signed=0, n_boxes=nb, m=m, comb=locpir.LP_XOR_TREE, x=ct[:l], y=ct[l:2 * l],
                            boxes=ct[2 * l:2 * l + 4 * l * nb], services=ct[2 * l + 4 * l * nb:]))
        # plaintext truth: XOR of the services of the boxes holding the point (X1 <= x < X2, Y1 <= y < Y2)
        e = np.zeros(m, np.uint8)
        for (x1, x2, y1, y2), sv in zip(boxes, np.asarray(services, np.uint8).reshape(nb, m)):
            if x1 <= x < x2 and y1 <= y < y2:
                e ^= sv
        expect.append(e)
    torch.cuda.synchronize()
    policy = locpir.LP_SERVER_REJECT if args.serve_policy == "reject" else locpir.LP_SERVER_QUEUE
    ctx.lp_server_start(int(args.serve_budget_gb * 2**30), policy)
    tickets, t0 = [], time.perf_counter()
    next_t = t0
    offered, submit_s = 0, 0.0
    try:
        while True:
            now = time.perf_counter()
            if now - t0 >= args.serve_seconds:
                break
            if now >= next_t:
                k = offered % len(queries)
                offered += 1
                q = dict(queries[k])
                q["out_service"] = torch.empty(q["m"], W, dtype=torch.int32, device="cuda")
                ts = time.perf_counter()
                try:
                    tickets.append((ctx.lp_server_submit(q), k, q["out_service"]))
                except locpir.LocpirError:
                    pass
                submit_s += time.perf_counter() - ts
                next_t += rng.exponential(1.0 / args.serve_rate)
            else:
                time.sleep(min(next_t - now, 0.01))
        deadline = time.perf_counter() + args.serve_drain
        while time.perf_counter() < deadline and not all(ctx.lp_server_poll(t) for t, _, _ in tickets):
            time.sleep(0.05)
        st = ctx.lp_server_stats()
        done = [(k, o) for t, k, o in tickets if ctx.lp_server_poll(t)]
    finally:
        ctx.lp_server_stop()
    wrong = 0
    for k, o in done:
        ph = torch.empty(o.shape[0], dtype=torch.int32, device="cuda")
        locpir.lp_client_lwe_phase(p.n, s_dev, o, ph, o.shape[0])
        wrong += int(((ph.cpu().numpy() > 0).astype(np.uint8) != expect[k]).sum())
    print(json.dumps({"experiment": "serving", "shape": args.serve_shape, "arrival_rate_per_s": args.serve_rate,
                      "policy": args.serve_policy, "offered": offered,
                      "submit_ms_mean": 1e3 * submit_s / max(offered, 1),
                      "arrival_seconds": args.serve_seconds, "drain_seconds": args.serve_drain,
                      "memory_budget_gb": args.serve_budget_gb, "distinct_queries": len(queries),
                      "submitted": st["submitted"], "admitted": st["admitted"], "completed": st["completed"],
                      "rejected": st["rejected"], "still_waiting": st["waiting"], "still_active": st["active"],
                      "sustained_queries_per_s": st["queries_per_s"], "bootstraps": st["bootstraps"],
                      "bootstraps_per_s": st["bootstraps_per_s"], "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                      "mean_ms": st["mean_ms"], "ticks": st["ticks"], "checked_queries": len(done),
                      "wrong_bits": wrong}), flush=True)


def workload_config(world: int) -> dict:
    """The workload both arms report: one step is COUNT independent NAND bootstraps per rank."""
    return {"workload": f"NAND gate bootstrapping: {COUNT:,} independent gates per step (n=630, N=1024, k=1, "
                        "Bgbit=10, lg=3, basebit=2, t=8; keys seed 0, inputs seed 1)",
            "global_batch": COUNT * world, "parallelism": f"replicas x{world}" if world > 1 else "1 GPU",
            "l2": f"inputs larger than L2 (2 x {COUNT * (N_LWE + 1) * 4 / 1e6:.0f} MB per step)"}


def run_reference(args) -> None:
    rank, world, _ = _dist()
    if rank != 0:
        return
    import oracle
    keys = oracle.keygen(synth.key_draws(0))
    cores = oracle.threads()
    A, B = synth.nand_pairs(1, COUNT)
    S = 2 * cores
    a = oracle.encrypt(keys.s, A[:S], synth.lwe_draws(1, S))
    b = oracle.encrypt(keys.s, B[:S], synth.lwe_draws(1, S, offset=COUNT))
    for _ in range(args.warmup):
        oracle.gate_batch(keys, oracle.NAND, a[:cores], b[:cores], nthreads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.gate_batch(keys, oracle.NAND, a, b, nthreads=cores)
    dt = time.perf_counter() - t0
    value = S * args.steps / dt
    line = {"impl": "reference", "metric": "gate bootstraps/s", "value": value, "unit": "bootstraps/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": workload_config(args.gpus),
            "cpu_baseline": {"value": value, "unit": "bootstraps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{S} of the {COUNT:,} NAND gates per step (OpenMP, {cores} threads)"},
            "e2e": {"value": value, "unit": "bootstraps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args) -> None:
    import torch
    from paper_2407_19871_gb300 import locpir
    rank, world, local = _dist()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    ctx, p, s_dev, (A, B), (a, b) = setup_gpu(local, seed_inputs=rank_seed(rank), count=COUNT)
    out = torch.empty_like(a)
    st = torch.cuda.current_stream()

    def step():
        ctx.lp_gate_batch(locpir.LP_NAND, a, b, None, out, COUNT, st)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    wrong = check_outputs(p, s_dev, out, A, B)

    # ---- device-resident timed region
    clocks = Clocks(local)
    ctx.lp_reset_timing()
    ctx.lp_set_timing(True)
    launches0 = ctx.lp_launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = ctx.lp_launch_count() - launches0
    br_ms, br_n = ctx.lp_kernel_time("br")
    ks_ms, ks_n = ctx.lp_kernel_time("ks")
    ctx.lp_set_timing(False)
    ms = reduce_max(ms, dist)
    value = job_throughput(COUNT, world, args.steps, ms / 1e3)

    # ---- end to end through the host-pointer entry point (pinned host buffers)
    W = p.n + 1
    ha = torch.empty(COUNT, W, dtype=torch.int32, pin_memory=True)
    hb = torch.empty(COUNT, W, dtype=torch.int32, pin_memory=True)
    ho = torch.empty(COUNT, W, dtype=torch.int32, pin_memory=True)
    ha.copy_(a.cpu())
    hb.copy_(b.cpu())
    na, nb, no = ha.numpy().view(np.uint32), hb.numpy().view(np.uint32), ho.numpy().view(np.uint32)
    ctx.lp_gate_batch_host(locpir.LP_NAND, na, nb, None, no, COUNT)  # warm the staging buffers
    e2e_steps = max(1, min(args.steps, 3))
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ctx.lp_gate_batch_host(locpir.LP_NAND, na, nb, None, no, COUNT)
    e2e_s = time.perf_counter() - t0
    e2e_s = reduce_max(e2e_s, dist)
    e2e_value = job_throughput(COUNT, world, e2e_steps, e2e_s)

    # ---- per-gate path (same kernels, one gate per launch), on a sample
    per_gate = None
    if rank == 0 and args.per_gate > 0:
        k = args.per_gate
        torch.cuda.synchronize()
        g0 = time.perf_counter()
        for g in range(k):
            ctx.lp_gate_batch(locpir.LP_NAND, a[g:g + 1], b[g:g + 1], None, out[g:g + 1], 1, st)
            torch.cuda.synchronize()
        per_gate = k / (time.perf_counter() - g0)

    loc = single = None
    if rank == 0 and args.locpir_queries > 0:
        loc = locpir_throughput(ctx, p, s_dev, args.locpir_queries)
        pers = locpir_throughput(ctx, p, s_dev, args.locpir_queries, executor=locpir.LP_EXEC_PERSISTENT)
        loc["persistent_executor"] = {k: pers[k] for k in ("queries_per_s", "seconds", "kernels_per_run", "wrong_bits")}
        single = single_query_latency(ctx, p, s_dev)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    br_avg_ms = br_ms / max(br_n, 1)
    ks_avg_ms = ks_ms / max(ks_n, 1)
    achieved = COUNT * N_LWE * MODMUL_PER_STEP / (br_avg_ms / 1e3)
    traffic = br_traffic(COUNT)
    peaks = _measured_peaks()
    ks_bytes = KS_TABLE_BYTES + COUNT * (4 * 1028 + 4 * W)
    ks_gbs = ks_bytes / (ks_avg_ms / 1e3) / 1e9 if ks_avg_ms > 0 else None
    smem_floor_ms = COUNT * KS_SMEM_BYTES_PER_CT / (SMEM_BYTES_PER_CLK_SM * SMS * MAX_MHZ * 1e6) * 1e3
    line = {
        "metric": "gate bootstraps/s", "value": value, "unit": "bootstraps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload_config(world),
        "e2e": {"value": e2e_value, "unit": "bootstraps/s", "h2d_bytes_per_step": 2 * COUNT * W * 4,
                "d2h_bytes_per_step": COUNT * W * 4},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "kernel": "br_kernel (blind rotation + extraction)",
                     "achieved": achieved / 1e12, "peak": PEAK_MODMUL_PER_S / 1e12, "unit": "Tmodmul/s",
                     "frac": achieved / PEAK_MODMUL_PER_S, "traffic": traffic,
                     "algorithmic_bytes": BR_KEY_BYTES + COUNT * BR_BYTES_PER_CT,
                     "traffic_source": BR_TRAFFIC_NOTE,
                     "peak_source": "152 SMs x 2070 MHz x 64 multiply-pipe slots / 4 slots per lazy Shoup "
                                    "product; measured 16.0 Shoup products per SM per clock",
                     "peak_3_slot_note": PEAK_MODMUL_3_SLOT / 1e12,
                     "br_ms_per_launch": br_avg_ms, "ks_ms_per_launch": ks_avg_ms},
        "ks": {"kernel": "ks_kernel (digit-pair table gather-accumulate)", "ms_per_launch": ks_avg_ms,
               "algorithmic_bytes": ks_bytes, "achieved_gbs": ks_gbs, "hbm_peak_gbs": peaks.get("hbm_gbs"),
               "hbm_frac": (ks_gbs / peaks["hbm_gbs"]) if ks_gbs and peaks.get("hbm_gbs") else None,
               "smem_floor_ms": smem_floor_ms, "frac_of_smem_floor": smem_floor_ms / ks_avg_ms if ks_avg_ms else None},
        "clocks": clk,
        "per_gate_bootstraps_per_s": per_gate,
        "batched_speedup_vs_per_gate": (value / world / per_gate) if per_gate else None,
        "decrypt_errors": wrong,
        "locpir": loc,
        "single_query": single,
        "autotune": ctx.tuning,
    }
    if args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    global COUNT
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--per-gate", type=int, default=16, help="gates timed one per launch (0: skip)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--locpir-queries", type=int, default=152,
                    help="LocPIR queries of the city-batch shape timed for queries/s (0: skip)")
    ap.add_argument("--paper-shapes", action="store_true",
                    help="run the paper's experiment shapes (Table 2, Fig. 4(a), batch width); one JSON line each")
    ap.add_argument("--table2-only", action="store_true", help="with --paper-shapes: Table 2's four rows only")
    ap.add_argument("--serve", action="store_true", help="serving run: Poisson arrivals into the query server")
    ap.add_argument("--engines", action="store_true",
                    help="head-to-head of the NTT and tensor-core (GEMM) engines instead of the bench line")
    ap.add_argument("--engines-count", type=int, default=4096)
    ap.add_argument("--br-latency", action="store_true",
                    help="blind-rotation time against level width, batched and split kernels")
    ap.add_argument("--engines-ks-count", type=int, default=65536)
    ap.add_argument("--multibox", action="store_true",
                    help="the uneven multi-box batch (1,024 queries, B_x ~ U{1..128}, l ~ U{16,24,32}, m=512, OR tree)")
    ap.add_argument("--multibox-queries", type=int, default=1024)
    ap.add_argument("--multibox-budget-gb", type=float, default=96.0)
    ap.add_argument("--multibox-input-gb", type=float, default=32.0)
    ap.add_argument("--multibox-executor", default="levels", choices=["levels", "persistent"])
    ap.add_argument("--int-peaks", action="store_true",
                    help="integer-pipe throughput microbenchmark (the alu roofline's measured peak)")
    ap.add_argument("--serve-shape", default="uneven", choices=["uneven", "city"])
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-drain", type=float, default=30.0)
    ap.add_argument("--serve-budget-gb", type=float, default=4.0)
    ap.add_argument("--serve-distinct", type=int, default=4)
    ap.add_argument("--serve-policy", default="queue", choices=["queue", "reject"])
    ap.add_argument("--count", type=int, default=COUNT,
                    help="gates per step (default 65,536; smaller values are for profiling only)")
    ap.add_argument("--retune", action="store_true", help="measure the launch policy again instead of reading its cache")
    args = ap.parse_args()
    COUNT = args.count
    global RETUNE
    RETUNE = args.retune
    if args.int_peaks:
        sys.exit(int_peaks())
    if args.multibox:
        multibox_uneven(args)
    elif args.paper_shapes:
        paper_shapes(args.table2_only)
    elif args.serve:
        serve(args)
    elif args.engines:
        engines_bench(args.engines_count, args.engines_ks_count)
    elif args.br_latency:
        br_latency_bench()
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
