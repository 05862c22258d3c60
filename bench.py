#!/usr/bin/env python3
"""Benchmark of batched midsize integer addition and multiplication on GB300.

One step = one pass of the whole hot path over the size-sweep workload:
  * addition and schoolbook multiplication of 1K .. 256K-bit integers
    (u32 limbs), each size a batch holding 64 MiB of operand limbs per side;
  * transform multiplication (one 64-bit prime with 16-bit digits, two
    64-bit primes with 32-bit digits and CRT, three 32-bit primes) at
    16K .. 256K bits, same batches.
Each operation is one kernel launch through the library's C ABI (plans).

Printed on stdout: one compact JSON line (rank 0, at most about 3 KB).
`value` is multiplications completed per second over the step (inputs
resident in HBM); beside it the addition throughput, the roofline of the
dominant kernel, the clocks seen during the timed region, an end-to-end
figure through the host-buffer entry point, the CPU oracle timed on a bounded
sample, and summary figures of the off-step sections (roofline fractions of
the kernels at their key sizes, the transform/schoolbook crossover sizes, the
mixed-size batch against the plain per-class and per-item launches, the
serving loop's latencies).  The full detail (per-op breakdown and rooflines,
every product form timed alone at every size, the fused programs, the mixed
and serving runs) goes to the file named by --detail, else to stderr.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--detail PATH]
Under torchrun each rank runs the same per-rank workload (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time
from dataclasses import dataclass, field
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

from paper_2405_14642_gb300 import workloads  # noqa: E402

METRIC = "integer mults/s and add GB/s, 1K–256K bits; mixed-size batched vs plain"
UNIT = "mults/s"
NUM_SMS_NOMINAL = 152
SM_MAX_MHZ_NOMINAL = 2070.0


@dataclass
class Op:
    name: str          # add | quad | ntt64 | crt | ntt3
    bits: int
    na: int
    nb: int
    batch: int
    seed: int
    mults: int = 0     # multiplications per launch
    bytes: int = 0     # algorithmic HBM bytes per launch
    prods: int = 0     # algorithmic 32x32->64-bit word products per launch
    times_ms: list = field(default_factory=list)

    @property
    def nout(self):
        return self.na + 1 if self.name == "add" else self.na + self.nb

    @property
    def label(self):
        return f"{self.name}@{self.bits // 1024}K"


OPCODES = {"add": lambda bn: bn.BN_OP_ADD, "quad": lambda bn: bn.BN_OP_MUL_QUAD,
           "quadtc": lambda bn: bn.BN_OP_MUL_QUAD_TC,
           "ntt64": lambda bn: bn.BN_OP_MUL_NTT64, "crt": lambda bn: bn.BN_OP_MUL_NTT_CRT,
           "ntt3": lambda bn: bn.BN_OP_MUL_NTT3}

# The schoolbook product runs on the integer pipes below this size and on the
# tensor cores (byte digits, exact f32 sums) from it up, where that kernel is
# the faster schoolbook on GB300; both compute every word product.
TC_MIN_BITS = 16384
# fp16-equivalent FLOP of one 32x32-bit word product on the tensor cores:
# 16 byte products, 2 FLOP each.
TC_FLOP_PER_WORD_PRODUCT = 32


def ntt_lengths(n: int):
    """Transform lengths and 64-bit modular products per pair (per prime)."""
    n64 = 1 << math.ceil(math.log2(4 * n))      # 16-bit digits, 2n + 2n digits
    ncrt = 1 << math.ceil(math.log2(2 * n))     # 32-bit digits, n + n digits
    def modmuls(N):                              # 3 transforms + pointwise + scale
        return 3 * (N // 2) * int(math.log2(N)) + 2 * N
    return n64, ncrt, modmuls(n64), 2 * modmuls(ncrt)


def build_ops(quick: bool = False, integer_schoolbook: bool = False):
    pts = workloads.sweep_points()
    if quick:
        pts = [p for p in pts if p.bits in (1024, 32768, 262144)]
    ops = []
    for p in pts:
        n = p.limbs
        ops.append(Op("add", p.bits, n, n, p.batch, p.seed, mults=0,
                      bytes=4 * (3 * n + 1) * p.batch))
        tc = p.bits >= TC_MIN_BITS and not integer_schoolbook
        ops.append(Op("quadtc" if tc else "quad", p.bits, n, n, p.batch, p.seed,
                      mults=p.batch, bytes=4 * 4 * n * p.batch, prods=n * n * p.batch))
    for p in pts:
        if p.bits not in workloads.NTT_BITS:
            continue
        n = p.limbs
        _, _, mm64, mmcrt = ntt_lengths(n)
        # A 64x64-bit modular product needs at least the 4 word products of
        # its 128-bit product (the reduction's products are not counted).
        ops.append(Op("ntt64", p.bits, n, n, p.batch, p.seed, mults=p.batch,
                      bytes=16 * n * p.batch, prods=4 * mm64 * p.batch))
        ops.append(Op("crt", p.bits, n, n, p.batch, p.seed, mults=p.batch,
                      bytes=16 * n * p.batch, prods=4 * mmcrt * p.batch))
        # Three 32-bit primes at the CRT form's length: one word product per
        # modular product.
        ops.append(Op("ntt3", p.bits, n, n, p.batch, p.seed, mults=p.batch,
                      bytes=16 * n * p.batch, prods=3 * (mmcrt // 2) * p.batch))
    return ops


def workload_config(ops, world: int):
    bits = sorted({o.bits for o in ops})
    return {
        "workload": "size sweep 1K-256K bits: add + schoolbook mul at every size (integer-pipe "
                    "kernel below 16K bits, tensor-core kernel from 16K bits), NTT mul "
                    "(1x64-bit prime/16-bit digits, 2x64-bit primes CRT/32-bit digits, "
                    "3x32-bit primes/32-bit digits) at 16K-256K; 64 MiB of u32 operand limbs "
                    "per side per size",
        "sizes_bits": bits,
        "batch_per_size": {str(b): next(o.batch for o in ops if o.bits == b) for b in bits},
        "ops_per_step": len(ops),
        "cache": "inputs larger than L2 (>= 128 MiB of operands per launch), no flush",
        "per_rank": "each rank runs the full workload (weak scaling)",
        "ranks": world,
    }


# ---- clocks ---------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in Path(self.path).read_text().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        power = [num(r[3]) for r in rows if num(r[3])]
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(num(r[2]) or 0 for r in rows),
                "sm_mhz_min": min(sm) if sm else None,
                "power_w_max": max(power) if power else None,
                "reasons": reasons, "samples": len(rows)}


# ---- GPU arm ---------------------------------------------------------------

def imad_peak(torch, bn, dev):
    """Time the register-only multiply-add probe and derive the word-product
    ceiling: a 32x32->64 product needs one mad.lo and one mad.hi, so with
    per-clock rates lo and hi (snapped to powers of two) the ceiling is
    1 / (1/lo + 1/hi) products per clock per SM, times SMs and the max clock."""
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    out = torch.zeros(sms * 8, dtype=torch.int32, device=dev)
    res = {}
    for name, kind in (("mad_lo", 0), ("mad_hi", 1), ("mad_wide", 2), ("mac_chain", 3)):
        iters = 2048
        bn.bn_probe_int_throughput(kind, sms * 8, 256, 64, out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sampler = ClockSampler(dev.index or 0)
        sampler.start()
        best = None
        for _ in range(3):
            e0.record()
            ops = bn.bn_probe_int_throughput(kind, sms * 8, 256, iters, out)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        clk = sampler.stop()
        total = ops * sms * 8 * 256
        rate = total / (best * 1e-3)
        mhz = clk.get("sm_mhz") or SM_MAX_MHZ_NOMINAL
        res[name] = {"ops_per_s": rate, "per_clk_per_sm": rate / (sms * mhz * 1e6), "sm_mhz": mhz}

    def snap(x):
        return 2 ** round(math.log2(x)) if x > 0 else 0
    lo, hi = snap(res["mad_lo"]["per_clk_per_sm"]), snap(res["mad_hi"]["per_clk_per_sm"])
    per_clk = 1.0 / (1.0 / lo + 1.0 / hi) if lo and hi else 0.0
    peak = per_clk * sms * SM_MAX_MHZ_NOMINAL * 1e6
    return {"mad_lo_per_clk_per_sm": lo, "mad_hi_per_clk_per_sm": hi,
            "word_products_per_clk_per_sm": per_clk, "sms": sms, "peak_word_products_per_s": peak,
            "probe": res}


MMA_PROBE_CASES = ((32, 1, 1 << 30), (32, 2, 1 << 30), (32, 4, 1 << 30), (32, 8, 1 << 30), (32, 8, 8),
                   (64, 4, 8), (64, 8, 1 << 30), (128, 2, 8), (128, 4, 1 << 30), (256, 2, 1 << 30))


def mma_probe(torch, bn, dev):
    """SM clocks per tensor-core MMA (kind::f16, M = 128, K = 16, N = n, operands
    in shared memory at moving windows) for a number of independent
    accumulation chains, each restarted every chain_len of its MMAs; one CTA
    per SM issues them from one thread (bn_probe_mma_throughput)."""
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    out = []
    for n, chains, chain_len in MMA_PROBE_CASES:
        iters = 16384
        bn.bn_probe_mma_throughput(n, chains, chain_len, 64, sms, status)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        bn.bn_probe_mma_throughput(n, chains, chain_len, iters, sms, status)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out.append({"n": n, "chains": chains, "chain_len": chain_len if chain_len < (1 << 30) else None,
                    "clocks_per_mma": round(ms * 1e-3 * SM_MAX_MHZ_NOMINAL * 1e6 / iters, 1)})
    if int(status.item()):
        raise RuntimeError("the tensor-core probe's wait timed out")
    return out


def kernel_traffic(op_label: str):
    """DRAM bytes per launch from the committed ncu capture of this op, if none
    of the kernel's source files changed since the capture (else None)."""
    import hashlib
    p = ROOT / "profiles" / "traffic.json"
    if not p.exists():
        return None
    entry = json.loads(p.read_text()).get(op_label)
    if not entry:
        return None
    if not entry.get("sources"):
        return None
    for rel, digest in entry["sources"].items():
        src = ROOT / rel
        if not src.exists() or hashlib.sha256(src.read_bytes()).hexdigest() != digest:
            return None
    return entry["dram_bytes"]


def read_tensor_peak():
    """Dense bf16 TFLOP/s sustained over a long run (the figure for a kernel
    timed inside a long step); fp16 has the same nominal tensor rate."""
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        try:
            d = json.loads(p.read_text())
            return float(d["bf16_tflops_sustained"]), "measured (cuBLAS bf16, sustained)"
        except (ValueError, KeyError):
            pass
    return 1700.0, "fallback (sustained)"


def read_measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        try:
            d = json.loads(p.read_text())
            return float(d["hbm_gbs"]), "measured"
        except (ValueError, KeyError):
            pass
    return 6800.0, "fallback"


def run_gpu(args, rank, world, local_rank):
    import torch
    import paper_2405_14642_gb300 as bn

    dev = torch.device(f"cuda:{local_rank}")
    torch.cuda.set_device(dev)
    bn.load()
    ops = build_ops(args.quick, args.integer_schoolbook)
    if args.only:
        keep = set(args.only.split(","))
        ops = [o for o in ops if o.name in keep or o.label in keep]
    stream = torch.cuda.current_stream(dev)

    # Inputs: one seeded pair per size, shared by the ops at that size.
    inputs, hosts = {}, {}
    for o in ops:
        if o.bits in inputs:
            continue
        a, b = workloads.pair_batch(o.batch, o.na, o.nb, seed=o.seed + 7919 * rank, edges=False)
        ta = torch.from_numpy(a.view(np.int32)).to(dev)
        tb = torch.from_numpy(b.view(np.int32)).to(dev)
        inputs[o.bits] = (ta, tb)
        hosts[o.bits] = (a, b)
    outs = {}
    plans = {}
    skipped = []
    for o in list(ops):
        opcode = OPCODES[o.name](bn)
        try:
            plans[o.label] = bn.Plan(opcode, o.na, o.nb, o.batch)
        except bn.BnError as e:
            if e.status != 4:       # only "unsupported size" may be skipped, and is reported
                raise
            skipped.append(o.label)
            ops.remove(o)
            continue
        key = (o.bits, o.nout)
        if key not in outs:
            outs[key] = torch.empty((o.batch, o.nout), dtype=torch.int32, device=dev)

    def step(record=None):
        for i, o in enumerate(ops):
            ta, tb = inputs[o.bits]
            if record is not None:
                record[i][0].record(stream)
            plans[o.label].execute(ta, tb, out=outs[(o.bits, o.nout)], stream=stream)
            if record is not None:
                record[i][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    peak_info = imad_peak(torch, bn, dev) if rank == 0 else None
    mma_info = mma_probe(torch, bn, dev) if rank == 0 and not args.quick else None

    evs = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
            for _ in ops] for _ in range(args.steps)]
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    t0.record(stream)
    for k in range(args.steps):
        step(evs[k])
    t1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    elapsed_ms = t0.elapsed_time(t1)
    for i, o in enumerate(ops):
        o.times_ms = [evs[k][i][0].elapsed_time(evs[k][i][1]) for k in range(args.steps)]
    max_ms = allreduce_max(elapsed_ms, world, dev)
    mults_per_step = sum(o.mults for o in ops)
    value = aggregate_value(mults_per_step, args.steps, max_ms, world)
    ms_per_step = max_ms / args.steps
    gpu_launches = args.steps * len(ops)

    # End to end: host arrays in pinned memory through the host-buffer entry
    # point, on every rank (whole-job figure, like the step).
    e2e = None
    if args.e2e_steps > 0:
        e2e = run_e2e(args, torch, bn, ops, hosts, dev, world)
    if rank != 0:
        return None
    # Per-GPU sections, on rank 0 only.
    forms = (run_forms(args, torch, bn, ops, inputs, outs, stream, dev)
             if args.isolated_reps else None)
    fused = None
    if args.fused_reps > 0:
        fused = run_fused(args, torch, bn, dev, inputs, peak_info)
    mixed = None
    if args.mixed_items > 0:
        mixed = run_mixed(args, torch, bn, dev, rank)
    serving = None
    if args.serve_requests > 0:
        serving = run_serving(args, torch, bn, dev, rank)
    hbm_peak, hbm_kind = read_measured_peaks()
    tc_peak, tc_kind = read_tensor_peak()
    rows, rooflines = [], []
    for o in ops:
        ms = float(np.mean(o.times_ms))
        row = {"op": o.label, "ms": round(ms, 4), "batch": o.batch}
        rf = roofline_of(o, ms, hbm_peak, hbm_kind, tc_peak, tc_kind, peak_info)
        if o.name == "add":
            row.update(gbs=rf["achieved"], adds_per_s=o.batch / (ms * 1e-3))
        else:
            row.update(mults_per_s=o.batch / (ms * 1e-3), word_tprods=round(o.prods / (ms * 1e-3) / 1e12, 3))
        rooflines.append(rf)
        rows.append(row)
    total_ms = [sum(o.times_ms[k] for o in ops) for k in range(args.steps)]
    dom = max(range(len(ops)), key=lambda i: np.mean(ops[i].times_ms))
    roof = dict(rooflines[dom])
    roof["traffic"] = kernel_traffic(ops[dom].label)
    roof["kernel_share_of_step"] = round(float(np.mean(ops[dom].times_ms)) / float(np.mean(total_ms)), 4)
    roof["ms"] = round(float(np.mean(ops[dom].times_ms)), 4)
    add_ops = [o for o in ops if o.name == "add"]
    add_gbs = (sum(o.bytes for o in add_ops) / (sum(np.mean(o.times_ms) for o in add_ops) * 1e-3) / 1e9
               if add_ops else None)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(ops, budget_s=args.cpu_budget)
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload_config(ops, world),
        "add_gbs": round(add_gbs, 1) if add_gbs else None,
        "roofline": roof, "rooflines": rooflines, "breakdown": rows,
        "imad_probe": peak_info, "mma_probe": mma_info, "clocks": clocks, "gpu_launches": gpu_launches,
        "e2e": e2e, "cpu_baseline": cpu, "impl": "ours", "skipped_ops": skipped,
        "mixed": mixed, "serving": serving, "fused": fused, "forms": forms,
    }


def roofline_of(o, ms, hbm_peak, hbm_kind, tc_peak, tc_kind, peak_info):
    """Roofline entry of one op from its mean event time: algorithmic bytes
    (add) against measured HBM, fp16-equivalent FLOP (tensor-core schoolbook)
    against the measured sustained tensor peak, word products (integer-pipe
    products) against the derived word-product ceiling."""
    if o.name == "add":
        gbs = o.bytes / (ms * 1e-3) / 1e9
        return {"op": o.label, "bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak,
                "unit": "GB/s", "frac": round(gbs / hbm_peak, 4), "peak_kind": hbm_kind + " copy",
                "traffic": None}
    gp = o.prods / (ms * 1e-3) / 1e12
    if o.name == "quadtc":
        tf = TC_FLOP_PER_WORD_PRODUCT * gp
        return {"op": o.label, "bound": "tensor", "achieved": round(tf, 1), "peak": tc_peak,
                "unit": "TFLOP/s", "frac": round(tf / tc_peak, 4),
                "peak_kind": tc_kind + "; 32 fp16 FLOP per word product", "traffic": None}
    peak_t = peak_info["peak_word_products_per_s"] / 1e12
    return {"op": o.label, "bound": "alu", "achieved": round(gp, 3), "peak": round(peak_t, 3),
            "unit": "T word-products/s", "frac": round(gp / peak_t, 4),
            "peak_kind": "derived: 1/(1/%d+1/%d) word products/clk/SM x %d SMs x %.0f MHz"
                         % (peak_info["mad_lo_per_clk_per_sm"], peak_info["mad_hi_per_clk_per_sm"],
                            peak_info["sms"], SM_MAX_MHZ_NOMINAL),
            "traffic": None}


FORMS = ("quad", "quadtc", "ntt64", "crt", "ntt3")


def crossover_bits(table, form):
    """Smallest size from which `form` is faster than the better of the two
    schoolbook kernels at that size and at every larger size timed (None if
    it is not faster at the largest size)."""
    sizes = sorted(table)
    best = None
    for bits in reversed(sizes):
        row = table[bits]
        school = [row[f] for f in ("quad", "quadtc") if row.get(f)]
        if not row.get(form) or not school or row[form] >= min(school):
            break
        best = bits
    return best


def run_forms(args, torch, bn, ops, inputs, outs, stream, dev):
    """Every product form alone at every size of the sweep, on the step's
    operands: the integer-pipe and tensor-core schoolbooks and the three
    transform forms (plus the addition), each the median of the isolated
    repetitions, each launch after a read-only pass over 256 MiB so that L2
    holds no dirty lines from another kernel.  From this table, the
    transform/schoolbook crossover size of each transform form."""
    clean_buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    table, rows = {}, []
    for bits in sorted(inputs):
        ta, tb = inputs[bits]
        batch, n = ta.shape
        table[bits] = {}
        for name in ("add",) + FORMS:
            nout = n + 1 if name == "add" else 2 * n
            out = outs.get((bits, nout))
            if out is None:
                out = torch.empty((batch, nout), dtype=torch.int32, device=dev)
                outs[(bits, nout)] = out
            try:
                plan = bn.Plan(OPCODES[name](bn), n, n, batch)
            except bn.BnError as e:
                if e.status != 4:
                    raise
                continue
            with plan:
                plan.execute(ta, tb, out=out, stream=stream)
                ts = []
                for _ in range(args.isolated_reps):
                    clean_buf.sum(dtype=torch.int64)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    plan.execute(ta, tb, out=out, stream=stream)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ts.append(e0.elapsed_time(e1))
            ms = float(np.median(ts))
            table[bits][name] = ms
            rows.append({"op": f"{name}@{bits // 1024}K", "ms": round(ms, 4)})
    bn.bn_tc_check()
    cross = {f: crossover_bits(table, f) for f in ("ntt64", "crt", "ntt3")}
    return {"how": "each (form, size) alone, median of %d launches after a read-only pass over "
                   "256 MiB" % args.isolated_reps,
            "crossover_bits": cross, "ops": rows,
            "table_ms": {str(k): {f: round(v, 4) for f, v in r.items()} for k, r in table.items()}}


def run_fused(args, torch, bn, dev, inputs, peak_info):
    """Section 6's programs at each sweep size on the same operands, results
    kept at the operands' length n (mod 2^(32n)): 1-Add against 6-Add
    (bn_add6, six dependent additions in one kernel) in GB/s by the paper's
    count 3 * NumInsts * NumBits / 8, and 1-Mul (bn_mul_low, the low half of
    the product) against Poly (bn_poly, four products and three additions in
    one kernel) in word products per second (n(n+1)/2 per low product).  The
    paper's scalability measures are the time ratios 6-Add / 1-Add and
    Poly / 1-Mul."""
    stream = torch.cuda.current_stream(dev)
    peak_t = peak_info["peak_word_products_per_s"] / 1e12 if peak_info else None
    rows = []
    for bits in sorted(inputs):
        ta, tb = inputs[bits]
        batch, n = ta.shape
        o1 = torch.empty((batch, n + 1), dtype=torch.int32, device=dev)
        on = torch.empty((batch, n), dtype=torch.int32, device=dev)
        calls = {"add": lambda: bn.bn_add(ta, tb, out=o1, stream=stream),
                 "add6": lambda: bn.bn_add6(ta, tb, out=on, stream=stream),
                 "mul_low": lambda: bn.bn_mul_low(ta, tb, out=on, stream=stream),
                 "poly": lambda: bn.bn_poly(ta, tb, out=on, stream=stream)}
        ms = {}
        for name, fn in calls.items():
            fn()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(args.fused_reps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms[name] = e0.elapsed_time(e1) / args.fused_reps
        paper_bytes = 3 * batch * bits / 8
        prods = n * (n + 1) / 2 * batch
        row = {"bits": bits, "batch": batch, **{f"{k}_ms": round(v, 4) for k, v in ms.items()},
               "add6_gbs": round(paper_bytes / (ms["add6"] * 1e-3) / 1e9, 1),
               "add6_over_add": round(ms["add6"] / ms["add"], 3),
               "mul_low_tprods": round(prods / (ms["mul_low"] * 1e-3) / 1e12, 3),
               "poly_tprods": round(4 * prods / (ms["poly"] * 1e-3) / 1e12, 3),
               "poly_over_mul_low": round(ms["poly"] / ms["mul_low"], 3)}
        if peak_t:
            row["poly_frac_of_word_product_peak"] = round(row["poly_tprods"] / peak_t, 4)
        rows.append(row)
    return {"programs": "1-Add, 6-Add (x_{k+1} = x_k + x_{k-1}, result 8a + 13b), 1-Mul "
                        "(low half), Poly (a*a + b)*(b*b + b) + a*b, all mod 2^(32n)",
            "reps": args.fused_reps, "sizes": rows}


def run_mixed(args, torch, bn, dev, rank):
    """Mixed-size batch (200k operations by default, 70% products / 30% sums,
    limb counts log-uniform in 32..8192 for each operand, 5% edge cases):
    the batched graph (autotuned) against two plain baselines over the same
    items and kernel choices: per size class one padded ordinary launch
    (gather, launch, scatter; the paper's one-size-per-launch method) and one
    ordinary launch per item.  Results must be identical."""
    items, a, b, c_limbs = workloads.mixed_workload(args.mixed_items,
                                                    seed=workloads.seed_for(3, 0) + 7919 * rank)
    ta = torch.from_numpy(a.view(np.int32)).to(dev)
    tb = torch.from_numpy(b.view(np.int32)).to(dev)
    tc = torch.empty(c_limbs, dtype=torch.int32, device=dev)
    n_mul = int((items["op"] != 0).sum())
    stream = torch.cuda.current_stream(dev)
    out, results = {}, {}
    for name, flags, steps in (("batched", bn.BN_BATCH_AUTOTUNE, args.mixed_steps),
                               ("plain_class", bn.BN_BATCH_AUTOTUNE | bn.BN_BATCH_PLAIN_CLASSES,
                                args.mixed_steps),
                               ("plain_item", bn.BN_BATCH_AUTOTUNE | bn.BN_BATCH_PLAIN, 1)):
        t = time.perf_counter()
        batch = bn.Batch(items, flags)
        create_ms = (time.perf_counter() - t) * 1e3
        tc.fill_(-1)
        batch.execute(ta, tb, tc, stream=stream)
        torch.cuda.synchronize()
        results[name] = tc.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            batch.execute(ta, tb, tc, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        info = batch.info
        batch.close()
        out[name] = {"ms": round(ms, 3), "ops_per_s": len(items) / (ms * 1e-3),
                     "mults_per_s": n_mul / (ms * 1e-3), "launches": info["launches"],
                     "classes": info["classes"], "create_ms": round(create_ms, 1), "steps": steps,
                     "items_by_kernel": {k: info[k] for k in ("items_add", "items_quad",
                                                              "items_ntt64", "items_crt",
                                                              "items_ntt3")}}
    identical = bool(torch.equal(results["batched"], results["plain_class"])
                     and torch.equal(results["batched"], results["plain_item"]))
    del results
    # The graph's fixed cost: the same kind of batch at 1/10 and 1/100 of the
    # items (every class still present at 1/100 here); a straight line through
    # (items, ms) meets the axis at the cost of launching the per-class
    # persistent kernels with nothing to do, which is all that one kernel over
    # every class could save on the launch structure.
    scaling = [{"items": len(items), "ms": out["batched"]["ms"], "classes": out["batched"]["classes"]}]
    for every in (10, 100):
        sub = items[::every]
        batch = bn.Batch(sub, bn.BN_BATCH_AUTOTUNE)
        batch.execute(ta, tb, tc, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.mixed_steps):
            batch.execute(ta, tb, tc, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        scaling.append({"items": len(sub), "ms": round(e0.elapsed_time(e1) / args.mixed_steps, 3),
                        "classes": batch.info["classes"]})
        batch.close()
    xs = np.array([r["items"] for r in scaling], float)
    ys = np.array([r["ms"] for r in scaling], float)
    slope, icpt = np.polyfit(xs, ys, 1)
    return {"workload": f"{len(items)} ops, 70% mul (auto quad/NTT) / 30% add, limbs log-uniform "
                        "32..8192 per operand, 5% edge cases",
            "batched": out["batched"], "plain_class": out["plain_class"],
            "plain_item": out["plain_item"],
            "graph_scaling": scaling, "graph_fixed_ms": round(float(icpt), 4),
            "speedup_vs_class": round(out["plain_class"]["ms"] / out["batched"]["ms"], 2),
            "speedup_vs_item": round(out["plain_item"]["ms"] / out["batched"]["ms"], 2),
            "results_identical": identical}


def serve_trace(srv, bn, reqs, arrivals, poll_max=8192):
    """Replay requests at their arrival times (server clock, microseconds);
    returns per-request (arrival, done) in microseconds.  Arrival times are the
    scheduled ones, so any lateness of this driver loop counts as latency."""
    n = reqs.shape[0]
    done = np.zeros(n, np.float64)
    index = {}
    i, got = 0, 0
    t0 = srv.now_us()
    reqs = reqs.copy()
    reqs["arrival_us"] = arrivals + t0
    while got < n:
        now = srv.now_us()
        j = int(np.searchsorted(reqs["arrival_us"], now, side="right"))
        if j > i:
            for k, t in enumerate(srv.submit(reqs[i:j])):
                index[int(t)] = i + k
            i = j
        comps = srv.poll(poll_max)
        if comps.shape[0]:
            for c in comps:
                done[index.pop(int(c["ticket"]))] = c["done_us"]
            srv.release(comps["ticket"])
            got += comps.shape[0]
    return reqs["arrival_us"], done


def run_serving(args, torch, bn, dev, rank):
    """Poisson arrivals of products with limb counts log-uniform in 32..8192
    (each operand independently), operands resident in device memory, an
    8 GiB result pool; continuous batching vs one request at a time."""
    rng = np.random.Generator(np.random.PCG64(workloads.seed_for(5, 0) + 7919 * rank))
    pool_limbs = 32 << 20
    ops_buf = torch.from_numpy(workloads.uniform_limbs(1, pool_limbs, rng)[0].view(np.int32)).to(dev)
    base = ops_buf.data_ptr()

    def make(count):
        reqs = np.zeros(count, bn.REQUEST_DTYPE)
        reqs["op"] = bn.BN_OP_MUL_AUTO
        reqs["na"] = workloads.log_uniform_sizes(rng, count, 32, 8192)
        reqs["nb"] = workloads.log_uniform_sizes(rng, count, 32, 8192)
        for f, n in (("a", reqs["na"]), ("b", reqs["nb"])):
            off = rng.integers(0, (pool_limbs - n.astype(np.int64)) // 4) * 4
            reqs[f] = base + 4 * off.astype(np.uint64)
        return reqs

    out = {"workload": "products, limbs log-uniform 32..8192 per operand (1K-256K bits), "
                       "Poisson arrivals, operands device-resident, 8 GiB result pool",
           "runs": []}
    # The batched server at both ends of the offered range; the one-at-a-time
    # baseline at a rate below its capacity (about 15k requests/s), so that
    # its percentiles are latencies rather than a growing queue.
    plan = [("batched", rate, args.serve_requests if rate >= 100000 else args.serve_requests // 5)
            for rate in (50000, 500000)]
    plan.append(("sequential", args.seq_rate, max(200, args.serve_requests // 50)))
    for mode, rate, count in plan:
        reqs = make(count)
        arrivals = np.cumsum(rng.exponential(1e6 / rate, size=count)) + 2000.0
        with bn.Server(pool_bytes=8 << 30, sequential=(mode == "sequential")) as srv:
            warm = make(64)
            serve_trace(srv, bn, warm, np.zeros(64))            # first launches, plan warm-up
            arr, done = serve_trace(srv, bn, reqs, arrivals)
            st = srv.stats
        lat = done - arr
        span_s = (done.max() - arr.min()) * 1e-6
        out["runs"].append({"mode": mode, "offered_per_s": rate, "requests": count,
                            "throughput_per_s": round(count / span_s, 1),
                            "p50_us": round(float(np.percentile(lat, 50)), 1),
                            "p99_us": round(float(np.percentile(lat, 99)), 1),
                            "batches": st["batches"],
                            "max_inflight": st["max_inflight_seen"]})
    return out


def run_e2e(args, torch, bn, ops, hosts, dev, world=1):
    """Same metric through the host-buffer entry point with pinned host
    buffers: every op copies its operands in and its result out inside the
    timed region (bn_plan_execute_host_async), the ops spread round-robin over
    --e2e-streams streams so that copies of one op overlap kernels of another;
    the timed region ends when all streams are synchronised."""
    pinned_in, pinned_out, plans = {}, {}, {}
    for o in ops:
        if o.bits not in pinned_in:
            a, b = hosts[o.bits]
            pa = torch.from_numpy(a.view(np.int32)).pin_memory()
            pb = torch.from_numpy(b.view(np.int32)).pin_memory()
            pinned_in[o.bits] = (pa, pb)
        key = (o.bits, o.nout)
        if key not in pinned_out:
            pinned_out[key] = torch.empty((o.batch, o.nout), dtype=torch.int32).pin_memory()
        opcode = OPCODES[o.name](bn)
        plans[o.label] = bn.Plan(opcode, o.na, o.nb, o.batch)
    streams = [torch.cuda.Stream(dev) for _ in range(args.e2e_streams)]

    def step():
        for i, o in enumerate(ops):
            pa, pb = pinned_in[o.bits]
            plans[o.label].execute_host_async(pa, pb, pinned_out[(o.bits, o.nout)],
                                              stream=streams[i % len(streams)])

    for _ in range(2):  # the first allocates staging buffers; both warm the copy paths
        step()
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, args.e2e_steps))
    barrier(world)
    t = time.perf_counter()
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    el = time.perf_counter() - t
    barrier(world)
    el = allreduce_max(el, world, dev)
    for p in plans.values():
        p.close()
    mults = sum(o.mults for o in ops)
    h2d = sum(4 * (o.na + o.nb) * o.batch for o in ops)
    d2h = sum(4 * o.nout * o.batch for o in ops)
    return {"value": world * mults * steps / el, "unit": UNIT, "h2d_bytes_per_step": world * h2d,
            "d2h_bytes_per_step": world * d2h, "steps": steps, "ms_per_step": round(el / steps * 1e3, 3),
            "ranks": world, "streams": args.e2e_streams,
            "api": f"bn_plan_execute_host_async on {args.e2e_streams} streams (pinned host buffers, "
                   "copies inside the timed region)"}


# ---- CPU oracle ------------------------------------------------------------

_SAMPLES = {}


def _sample_inputs(o: Op, count: int):
    key = (o.label, count)
    if key not in _SAMPLES:
        _SAMPLES[key] = workloads.pair_batch(count, o.na, o.nb, seed=o.seed, edges=False)
    return _SAMPLES[key]


def oracle_time_op(o: Op, count: int, threads: int):
    """Seconds the oracle takes on `count` pairs of this op (inputs made beforehand)."""
    import oracle
    a, b = _sample_inputs(o, count)
    t = time.perf_counter()
    if o.name == "add":
        oracle.add(a, b, threads=threads)
    else:
        oracle.mul(a, b, threads=threads)
    return time.perf_counter() - t


def sample_counts(ops, budget_s: float, threads: int):
    """Pairs per op so the whole sample takes about budget_s on `threads` cores:
    the same fraction of every op's batch (at least one pair per thread).
    Each op's per-pair cost is calibrated on a small run of that op."""
    per_pair = {}
    for o in ops:
        words = (o.na * o.nb / 4) if o.name != "add" else o.na
        c0 = int(min(o.batch, max(threads, 2e6 / max(words, 1))))
        per_pair[o.label] = oracle_time_op(o, c0, threads) / c0
    full_s = sum(per_pair[o.label] * o.batch for o in ops)
    frac = min(1.0, budget_s / full_s) if full_s > 0 else 1.0
    return {o.label: int(min(o.batch, max(threads, round(o.batch * frac)))) for o in ops}, frac


def sample_text(ops, counts, frac):
    big = max(ops, key=lambda o: o.na * o.nb if o.mults else 0)
    return ("%.3g%% of every op's pairs (at least one per core), e.g. %s %d of %d; ops timed in "
            "turn, multiplications counted over the sample's measured time"
            % (100 * frac, big.label, counts[big.label], big.batch))


def oracle_sample_step(ops, counts, threads):
    """One sampled step of the oracle: every op on its sample, in turn.
    Returns (seconds measured over the whole sample, the same seconds
    extrapolated to every op's full batch)."""
    t0 = time.perf_counter()
    full = 0.0
    for o in ops:
        c = counts[o.label]
        full += oracle_time_op(o, c, threads) * (o.batch / c)
    return time.perf_counter() - t0, full


def cpu_baseline(ops, budget_s=15.0):
    """The oracle as it stands, on all host cores, over one bounded sample of
    the step's workload: value = multiplications in the sample / its time."""
    import oracle
    threads = oracle.default_threads()
    counts, frac = sample_counts(ops, budget_s, threads)
    wall, full = oracle_sample_step(ops, counts, threads)
    mults = sum(counts[o.label] for o in ops if o.mults)
    return {"value": mults / wall, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": sample_text(ops, counts, frac), "sample_s": round(wall, 3),
            "extrapolated_full_step_s": round(full, 3)}


def run_reference(args, rank, world):
    """The oracle, as it stands, on the host cores: each step one bounded
    sample of the step's workload (the same fraction of every op), timed as a
    whole; ms_per_step is that measured time and value the sample's
    multiplications over it."""
    if rank != 0:
        return None
    import oracle
    oracle.build()
    ops = build_ops(args.quick, getattr(args, "integer_schoolbook", False))
    threads = oracle.default_threads()
    counts, frac = sample_counts(ops, args.ref_step_budget, threads)
    for _ in range(args.warmup):
        oracle_sample_step(ops, counts, threads)
    walls, fulls = [], []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        w, f = oracle_sample_step(ops, counts, threads)
        walls.append(w)
        fulls.append(f)
    t_all = time.perf_counter() - t_all
    mults = sum(counts[o.label] for o in ops if o.mults)
    value = mults * args.steps / sum(walls)
    cpu = {"value": value, "unit": UNIT, "kind": "oracle", "cores": threads,
           "sample": sample_text(ops, counts, frac)}
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(float(np.mean(walls)) * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": workload_config(ops, world), "impl": "reference",
        "cpu_baseline": cpu,
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "timed_s": round(t_all, 4),
        "extrapolated_full_step_s": round(float(np.mean(fulls)), 3),
    }


# ---- the printed line ------------------------------------------------------

# Kernels whose roofline fractions the compact line carries (the targets the
# design tracks), by op label.
KEY_OPS = ("add@256K", "add@128K", "quad@1K", "quad@2K", "quadtc@32K", "quadtc@64K",
           "quadtc@256K", "ntt64@256K", "crt@256K", "ntt3@256K")


def compact(full: dict) -> dict:
    """The printed line: the contract's keys plus summary scalars of every
    section; the per-op detail stays in the full record."""
    keep = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
            "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "impl",
            "e2e", "cpu_baseline", "clocks", "gpu_launches", "add_gbs", "roofline", "timed_s",
            "extrapolated_full_step_s", "skipped_ops")
    out = {k: full[k] for k in keep if k in full}
    if isinstance(out.get("e2e"), dict) and "api" in out["e2e"]:
        out["e2e"] = dict(out["e2e"], api="bn_plan_execute_host_async, pinned host buffers, "
                                          "%d streams" % full["e2e"].get("streams", 8))
    if isinstance(out.get("roofline"), dict):
        out["roofline"] = dict(out["roofline"])
    if full.get("rooflines"):
        fr = {r["op"]: r["frac"] for r in full["rooflines"]}
        out["frac"] = {k: fr[k] for k in KEY_OPS if k in fr}
    if full.get("forms"):
        out["crossover_bits"] = full["forms"]["crossover_bits"]
    m = full.get("mixed")
    if m:
        out["mixed"] = {"batched_ms": m["batched"]["ms"], "plain_class_ms": m["plain_class"]["ms"],
                        "plain_item_ms": m["plain_item"]["ms"],
                        "speedup_vs_class": m["speedup_vs_class"],
                        "speedup_vs_item": m["speedup_vs_item"],
                        "graph_fixed_ms": m.get("graph_fixed_ms"),
                        "results_identical": m["results_identical"]}
    sv = full.get("serving")
    if sv:
        out["serving"] = {("%s@%dk" % (r["mode"], r["offered_per_s"] // 1000)):
                          [round(r["throughput_per_s"]), r["p50_us"], r["p99_us"]]
                          for r in sv["runs"]}
        out["serving"]["fields"] = "served/s, p50 us, p99 us"
    f = full.get("fused")
    if f and f.get("sizes"):
        last = f["sizes"][-1]
        out["fused_256K"] = {"add6_over_add": last["add6_over_add"],
                             "poly_over_mul_low": last["poly_over_mul_low"]}
    return out


def emit(full: dict, detail_path: str):
    """Full record to the detail file (or stderr), compact line to stdout."""
    text = json.dumps(full)
    if detail_path:
        Path(detail_path).parent.mkdir(parents=True, exist_ok=True)
        Path(detail_path).write_text(text + "\n")
    else:
        print(text, file=sys.stderr, flush=True)
    line = compact(full)
    if detail_path:
        line["detail"] = detail_path
    print(json.dumps(line), flush=True)


# ---- distributed plumbing --------------------------------------------------

def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        if dist.get_backend() == "nccl":
            import torch
            dist.barrier(device_ids=[torch.cuda.current_device()])
        else:
            dist.barrier()


def allreduce_max(x: float, world: int, dev):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=dev if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_value(units_per_rank_step: int, steps: int, max_ms: float, world: int) -> float:
    """Whole-job throughput: every rank processes the same per-rank work
    (weak scaling), timed by the slowest rank."""
    return world * units_per_rank_step * steps / (max_ms * 1e-3)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--quick", action="store_true", help="3 sizes only (smoke runs)")
    ap.add_argument("--only", default="", help="comma list of op names/labels to keep")
    ap.add_argument("--integer-schoolbook", action="store_true",
                    help="the integer-pipe schoolbook at every size (for profiling that kernel)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--e2e-streams", type=int, default=8,
                    help="streams the end-to-end pass spreads the ops over")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--ref-step-budget", type=float, default=4.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mixed-items", type=int, default=200000,
                    help="operations in the mixed-size batch comparison (0 = skip)")
    ap.add_argument("--mixed-steps", type=int, default=5)
    ap.add_argument("--isolated-reps", type=int, default=3,
                    help="launches per op in the isolated per-kernel pass (0 = skip)")
    ap.add_argument("--fused-reps", type=int, default=3,
                    help="timed repetitions of each fused program per size (0 = skip)")
    ap.add_argument("--serve-requests", type=int, default=50000,
                    help="requests per serving run at 500k/s (0 = skip the serving runs)")
    ap.add_argument("--seq-rate", type=int, default=5000,
                    help="offered rate (requests/s) of the one-at-a-time serving baseline")
    ap.add_argument("--detail", default="",
                    help="file for the full JSON record (default: stderr)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            if torch.cuda.is_available():
                torch.cuda.set_device(local_rank)  # before NCCL binds the rank to a device
            dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        res = run_gpu(args, rank, world, local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
    if res is not None:
        emit(res, args.detail)


if __name__ == "__main__":
    main()
