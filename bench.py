#!/usr/bin/env python3
"""Benchmark of the GB300 Cartesian FMM.

One step = one pass of the whole hot path over one batch: uniform-octree
build, P2M, M2M, M2L over all interaction lists (levels 2..6), L2L, L2P and
P2P, on 4,194,304 uniform particles with equal masses, a depth-6 octree
(262,144 leaves, 16 particles per leaf on average) and traceless tensors at
p = 8 (the precision-form workload).  Inputs are resident in HBM when the
timed region starts; L2 is flushed (a 256 MiB write) before every timed step.

Printed (rank 0, one JSON line): FMM particles/s of the chosen form, the
plain FP64 GPU form's particles/s and M2L pairs/s beside it, the relative
force error against an FP64 direct sum on sampled targets, the roofline of
the dominant kernel (M2L), the oracle timed on the host cores, an
end-to-end figure through fmm_evaluate_host, and SM clocks sampled during the
timed region.

  python bench.py [--gpus N --steps K --warmup W] [--form bf16x3|tf32x3|fp32|fp64]
  python bench.py --impl reference ...      # the FP64 CPU oracle
  python bench.py --workload m2l ...        # per-pair M2L micro-benchmark sweep
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMM particles/s at 1e-4 rel force err; M2L pairs/s vs plain FP64 GPU form"
N_PART, DEPTH, P, BASIS = 4194304, 6, 8, 1
TC_LEVEL = 5   # first level on the tensor cores (class grid of 16 cells per axis)
SEED = 3
WORKLOAD = "uniform cube, 4,194,304 particles, equal masses 1/N, depth-6 octree (262,144 leaves), traceless p=8"
L2_FLUSH_BYTES = 256 << 20
NOMINAL = {"sm_count": 152, "fp64_fma_per_clk_sm": 2, "fp32_fma_per_clk_sm": 128}
# DRAM bytes (read + write) of the dominant kernel per step, from one ncu
# capture of its level-6 launch (dram__bytes_read.sum + dram__bytes_write.sum)
# scaled by the cells of the levels it runs on, with the profile summary it
# comes from; a form is absent while its kernel has changed since its
# counters were taken (traffic is then reported as null).
# key: (form, tensor-core kernel, chunk width) -- (None, None) for the ALU forms
M2L_TRAFFIC = {
    # k_m2l_tc_slab<0, 4>, cw 48: 787.1 MB read + 155.9 MB written at level 6, x 9/8 for levels 5-6
    ("bf16x3", 0, 48): (1.0609e9, "ncu capture of the level-6 launch scaled by cells to levels 5-6 "
                                  "(profiles/m2l_tensorcore_bf16x3_level6_uniform4M_p8.md)"),
    # k_m2l_tc_t<32> (kernel 2): 722.5 MB read + 154.8 MB written at level 6, x 9/8 for levels 5-6
    ("bf16x3", 2, 256): (9.870e8, "ncu capture of the level-6 launch scaled by cells to levels 5-6 "
                                  "(profiles/m2l_tensorcore_swapped_bf16x3_level6_uniform4M_p8.md)"),
    # kernel 3, every launch of levels 6 and 5 (operand split, k_m2l_tc_t first K-part, column pack,
    # k_m2l_rest, level 5's group sum): 310.9 MB at level 6 + 33.3 MB at level 5, read + written
    ("bf16x3", 3, 256): (3.442e8, "ncu capture of every launch of the tensor-core levels 6 and 5 (operand split, "
                                   "tensor-core kernel, column pack, CUDA-core columns, group sum) "
                                   "(profiles/m2l_tensorcore_split_bf16x3_level6_uniform_p8.md)"),
    # m2l_grp_p8_b1_r0: 653.9 MB read + 154.4 MB written at level 6, x 299584/262144 for levels 2-6
    ("fp32", None, None): (9.237e8, "ncu capture of the level-6 launch scaled by cells to levels 2-6 "
                                    "(profiles/m2l_grouped_fp32_level6_uniform4M_p8.md)"),
}
# nominal dense tensor rates (PFLOP/s): a TF32 contraction takes the measured
# BF16 peak scaled by their ratio
NOMINAL_TENSOR = {"bf16": 2.25, "tf32": 1.1}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


def m2l_pairs_uniform(depth):
    """Number of M2L (target, source) pairs of the uniform interaction lists
    (per axis: sources j in [2p-2, 2p+3] inside the grid, p the parent of i)."""
    return sum(m2l_pairs_level(l) for l in range(2, depth + 1))


def max_over_ranks(v, world, dist, device):
    """Maximum of a per-rank value (a time) over the ranks: the job's time is
    its slowest rank's.  One rank: v itself."""
    if world <= 1:
        return float(v)
    import torch
    t = torch.tensor([float(v)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank holds its own independent set)."""
    return world * units_per_rank / seconds


def rank_seed(rank):
    """Input seed of a rank: every rank evaluates its own particle set."""
    return SEED + 1000 * rank


def m2l_pairs_level(l):
    """M2L pairs of uniform level l (sources in the parents' neighbours'
    children, minus the target's own neighbours), grid boundary included."""
    s = 1 << l
    i = np.arange(s)
    p = i >> 1
    cnt_all = np.minimum(2 * p + 3, s - 1) - np.maximum(2 * p - 2, 0) + 1
    cnt_adj = np.minimum(i + 1, s - 1) - np.maximum(i - 1, 0) + 1
    return int(np.einsum("i,j,k->", cnt_all, cnt_all, cnt_all) - np.einsum("i,j,k->", cnt_adj, cnt_adj, cnt_adj))


def m2l_fma_per_pair(p, basis):
    """FMAs of one M2L as the SIMT kernels execute it: symmetric -> C(p+6,6);
    traceless on the reduced representative -> sum_a (2a+1)(p-a+1)^2."""
    if basis == 0:
        from math import comb
        return comb(p + 6, 6)
    return sum((2 * a + 1) * (p - a + 1) ** 2 for a in range(p + 1))


def alu_peak_tflops(bits, mhz):
    """Nominal FP64 (bits 64) or FP32 (bits 32) FMA peak at the SM clock mhz,
    counting an FMA as two flops."""
    per = NOMINAL["fp64_fma_per_clk_sm"] if bits == 64 else NOMINAL["fp32_fma_per_clk_sm"]
    return NOMINAL["sm_count"] * per * 2 * mhz * 1e6 / 1e12


def m2l_alg_fma_per_pair(p, basis):
    """Algorithmic FMAs of one M2L (Eq. M2L with independent local outputs
    and full multipoles): symmetric C(p+6,6); traceless
    F_tl(p) = sum_n (2n+1) C(p-n+3,3) (2079 at p = 8)."""
    from math import comb
    if basis == 0:
        return comb(p + 6, 6)
    return sum((2 * n + 1) * comb(p - n + 3, 3) for n in range(p + 1))


def p2p_pairs_uniform(x, y, z, depth):
    """Particle pairs of the uniform near field: every particle against the
    particles of its own and its (up to 26) adjacent leaves, self excluded."""
    s = 1 << depth
    ix = [np.minimum((v * s).astype(np.int64), s - 1) for v in (x, y, z)]
    cnt = np.zeros((s, s, s), dtype=np.int64)
    np.add.at(cnt, (ix[2], ix[1], ix[0]), 1)
    pad = np.pad(cnt, 1)
    box = sum(pad[1 + a:1 + a + s, 1 + b:1 + b + s, 1 + c:1 + c + s]
              for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1))
    return int((cnt * box).sum() - len(x))


P2P_FLOP_PER_PAIR = 20   # 3 differences, |r|^2 (3), 1/|r| (1), 1/|r|^3 (2), q terms (2), pot and acc sums (4), 5 adds


def roofline_per_op(stage, form, nc, depth, n, npart_pairs, pk, mhz, fp_peak, alg_m2l_flop, tc_roof):
    """Roofline of each operator of the step.  HBM-bound operators take
    their algorithmic bytes (the inputs and outputs they must move in the
    library's storage formats, each once); P2P takes its FP32 (FP64) ALU
    work; M2L the tensor (ALU) work."""
    hbm = pk.get("hbm_gbs", 6800.0)
    leaves = 8 ** depth
    cells = lambda l: 8 ** l   # noqa: E731
    es = 8
    pos = 16 if form != "fp64" else 32        # float4 leaf-relative positions (FP32 forms) or x, y, z, q doubles
    out = {}

    def hb(name, bytes_, ms, what):
        ach = bytes_ / (ms * 1e-3) / 1e9
        out[name] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "ms": ms, "algorithmic_bytes": bytes_, "bytes_are": what}
    hb("p2m", n * pos + leaves * (4 + nc * es), stage["p2m"],
       "particles in, leaf ranges, leaf multipoles out (FP64)")
    m2m_b = sum(cells(l + 1) * nc * es + cells(l) * nc * es for l in range(2, depth))
    hb("m2m", m2m_b, stage["m2m"], "child multipoles in, parent multipoles out, levels 6 -> 2")
    l2l_b = sum(cells(l) * nc * es + 2 * cells(l + 1) * nc * es for l in range(2, depth))
    hb("l2l", l2l_b, stage["l2l"], "parent locals in, child locals read and written, levels 2 -> 6")
    hb("l2p", leaves * nc * es + n * (pos + 4 + 4 * 8), stage["l2p"],
       "leaf locals in, particles and permutation in, pot and acc out (FP64)")
    p2p_flop = npart_pairs * P2P_FLOP_PER_PAIR
    ach = p2p_flop / (stage["p2p"] * 1e-3) / 1e12
    out["p2p"] = {"bound": "alu", "achieved": ach, "peak": fp_peak, "unit": "TFLOP/s", "frac": ach / fp_peak,
                  "ms": stage["p2p"], "pairs": npart_pairs, "flop_per_pair": P2P_FLOP_PER_PAIR,
                  "pairs_per_s": npart_pairs / (stage["p2p"] * 1e-3)}
    if "l2p_p2p" in stage:
        # the fused pass: the near-field flops and the far-field evaluation
        # (2 (ns(p) + 3 ns(p - 1)) flop per particle)
        ns = lambda p: (p + 1) * (p + 2) * (p + 3) // 6   # noqa: E731
        pp = int(round((nc ** 0.5) - 1))
        l2p_flop = n * 2 * (ns(pp) + 3 * ns(pp - 1))
        fl = p2p_flop + l2p_flop
        ach = fl / (stage["l2p_p2p"] * 1e-3) / 1e12
        out["l2p_p2p"] = {"bound": "alu", "achieved": ach, "peak": fp_peak, "unit": "TFLOP/s", "frac": ach / fp_peak,
                          "ms": stage["l2p_p2p"], "flop": fl,
                          "flop_are": "near field (flop_per_pair of p2p) and far-field evaluation per particle",
                          "note": "one pass; the l2p and p2p entries time the two steps run separately"}
    m2l_ms = stage["m2l_2_4"] + stage["m2l_5_6"]
    ach = alg_m2l_flop / (m2l_ms * 1e-3) / 1e12
    out["m2l"] = {"bound": "alu" if tc_roof is None else "tensor", "achieved": ach,
                  "peak": fp_peak if tc_roof is None else tc_roof, "unit": "TFLOP/s",
                  "frac": ach / (fp_peak if tc_roof is None else tc_roof), "ms": m2l_ms,
                  "levels": "2..%d" % depth,
                  "flop_are": "algorithmic F_tl count" if tc_roof is not None else "executed (reduced representative)"}
    return out


class Clocks:
    """SM clock and clock-event reasons of the GPU during the timed region.

    Read through NVML (ctypes on libnvidia-ml, read-only queries) on a thread
    every 2 ms, so that a timed region of a few tens of milliseconds still
    gets samples; the thread is running before the region starts.  Without
    NVML, nvidia-smi every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # clock-event reason bits of the NVML API
    BITS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
            0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index, device=None):
        self.index = index
        self.device = device
        self.proc = None
        self.rows = []
        self.nvml = None

    def _nvml_open(self):
        import ctypes
        lib = ctypes.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None
        h = ctypes.c_void_p()
        ok = False
        try:
            import torch
            u = str(torch.cuda.get_device_properties(self.device if self.device is not None else 0).uuid)
            u = u if u.startswith("GPU-") else "GPU-" + u
            ok = lib.nvmlDeviceGetHandleByUUID(u.encode(), ctypes.byref(h)) == 0
        except Exception:
            ok = False
        if not ok and lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.index), ctypes.byref(h)) != 0:
            return None
        reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons
        mx = ctypes.c_uint()
        if lib.nvmlDeviceGetMaxClockInfo(h, ctypes.c_int(1), ctypes.byref(mx)) != 0:
            return None
        self.max_mhz = float(mx.value)
        return lib, h, reasons

    def _poll(self):
        import ctypes
        lib, h, reasons = self.nvml
        clk, rs = ctypes.c_uint(), ctypes.c_ulonglong()
        while True:
            a = lib.nvmlDeviceGetClockInfo(h, ctypes.c_int(1), ctypes.byref(clk))
            b = reasons(h, ctypes.byref(rs))
            if a == 0 and b == 0:
                self.rows.append((float(clk.value), int(rs.value)))
            if self.stop.wait(0.002):
                break

    def __enter__(self):
        import threading
        try:
            self.nvml = self._nvml_open()
        except Exception:
            self.nvml = None
        if self.nvml is not None:
            self.stop = threading.Event()
            self.thread = threading.Thread(target=self._poll, daemon=True)
            self.thread.start()
            t0 = time.time()
            while not self.rows and time.time() - t0 < 1.0:
                time.sleep(0.001)
            self.rows.clear()
            return self
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.nvml is not None:
            self.stop.set()
            self.thread.join(timeout=5)
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        if self.nvml is not None:
            if not self.rows:
                return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["no samples"], "samples": 0,
                        "sampler": "nvml, 2 ms"}
            reasons = sorted({n for _, r in self.rows for bit, n in self.BITS.items() if r & bit})
            return {"sm_mhz": float(np.median([c for c, _ in self.rows])), "sm_max_mhz": self.max_mhz,
                    "sm_min_mhz": min(c for c, _ in self.rows), "reasons": reasons, "samples": len(self.rows),
                    "sampler": "nvml, 2 ms"}
        rows = [r.split(", ") for r in getattr(self, "out", "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "sampler": "nvidia-smi, 200 ms"}


# ---------------------------------------------------------------------------
def cpu_reference(steps, warmup, emit=True):
    """The FP64 oracle on the host cores: a full FMM on a 262,144-particle
    uniform cube at the same leaf density (depth 4, 16 per leaf) and p."""
    import oracle
    from paper_1811_06332_gb300 import inputs
    n, depth = 262144, 4
    x, y, z = inputs.uniform_cube(n, SEED)
    q = inputs.masses_equal(n)
    times = []
    for k in range(warmup + steps):
        t0 = time.perf_counter()
        oracle.fmm_uniform(x, y, z, q, depth, P, BASIS)
        dt = time.perf_counter() - t0
        if k >= warmup:
            times.append(dt)
    v = n / float(np.mean(times))
    return {"value": v, "unit": "particles/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": "full oracle FMM on 262,144 uniform particles, depth 4 (16 per leaf), traceless p=8; "
                      "same leaf density and order as the GPU workload, mean of %d run(s)" % len(times),
            "seconds_per_run": float(np.mean(times))}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cb = cpu_reference(args.steps, args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "particles/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": cb["seconds_per_run"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": cb["sample"]},
            "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": cb["value"], "unit": "particles/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_1811_06332_gb300 import fmm as F
    from paper_1811_06332_gb300 import inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    forms = {"fp64": F.FP64, "fp32": F.FP32, "bf16x3": F.GEMM_BF16X3, "tf32x3": F.GEMM_TF32X3}
    form = args.form
    prec = forms[form]
    # each rank evaluates its own independent particle set (weak scaling)
    x, y, z = inputs.uniform_cube(N_PART, rank_seed(rank))
    q = inputs.masses_equal(N_PART)
    X = [torch.from_numpy(a).to(dev) for a in (x, y, z, q)]
    out = torch.empty((4, N_PART), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    tc_form = prec in (F.GEMM_BF16X3, F.GEMM_TF32X3)
    # use_graph: fmm_evaluate (the host entry point below) replays the whole
    # step from a CUDA graph; the per-operator calls of the timed region run
    # eagerly, so that each stage is timed on its own
    plan = F.Plan(p=P, basis=BASIS, prec=prec, depth=DEPTH, autotune=tc_form, use_graph=True)

    # M2L runs as two calls, levels 2..4 and 5..6 (the tensor-core levels of
    # the tensor-core forms), so that the dominant kernel is timed on its own;
    # the far and near field run as one call (fmm_l2p_p2p: one kernel in the
    # FP32 and tensor-core forms)
    stages = ["tree", "p2m", "m2m", "m2l_2_4", "m2l_5_6", "l2l", "l2p_p2p"]
    NST = len(stages)

    def step(ev):
        ev[0].record(stream)
        plan.fmm_build_tree(*X); ev[1].record(stream)
        plan.fmm_p2m(); ev[2].record(stream)
        plan.fmm_m2m(); ev[3].record(stream)
        plan.fmm_m2l_levels(2, TC_LEVEL - 1); ev[4].record(stream)
        plan.fmm_m2l_levels(TC_LEVEL, DEPTH); ev[5].record(stream)
        plan.fmm_l2l(); ev[6].record(stream)
        plan.fmm_l2p_p2p(out[0], out[1], out[2], out[3]); ev[7].record(stream)

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(NST + 1)] for _ in range(args.steps)]
    wev = [torch.cuda.Event(enable_timing=True) for _ in range(NST + 1)]
    for _ in range(args.warmup):
        flush.fill_(1.0)
        step(wev)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = F.kernel_launches()
    with Clocks(local, dev) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            step(evs[k])
        torch.cuda.synchronize()
    launches = F.kernel_launches() - launches0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    per_stage = np.array([[evs[k][i].elapsed_time(evs[k][i + 1]) for i in range(NST)] for k in range(args.steps)])
    step_ms = per_stage.sum(1)
    t_ms = max_over_ranks(float(step_ms.mean()), world, dist, dev)
    value = job_rate(N_PART, world, t_ms * 1e-3)

    # breakdown of the far and near field as separate steps (untimed for the
    # step; the second of two passes recorded), for the per-operator roofline
    for k in range(2):
        flush.fill_(3.0 + k)
        eb = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        eb[0].record(stream)
        plan.fmm_l2p(out[0], out[1], out[2], out[3]); eb[1].record(stream)
        plan.fmm_p2p(out[0], out[1], out[2], out[3]); eb[2].record(stream)
        torch.cuda.synchronize()
    sep = {"l2p": eb[0].elapsed_time(eb[1]), "p2p": eb[1].elapsed_time(eb[2])}

    # accuracy: relative force error against an FP64 direct sum on 4096 sampled targets
    torch.cuda.synchronize()
    tsel = torch.from_numpy(np.sort(np.unique((inputs.u01(SEED, 91, 4096) * N_PART).astype(np.int64)))).to(dev)
    ref = torch.empty((4, len(tsel)), dtype=torch.float64, device=dev)
    F.fmm_direct(X[0], X[1], X[2], X[3], ref[0], ref[1], ref[2], ref[3], targets=tsel)
    plan.fmm_evaluate(*X, out[0], out[1], out[2], out[3])
    torch.cuda.synchronize()
    acc = out[1:, tsel]
    rel_err = float(torch.sqrt(((acc - ref[1:]) ** 2).sum() / (ref[1:] ** 2).sum()).item())

    m2l_ms = float((per_stage[:, 3] + per_stage[:, 4]).mean())
    tc_ms = float(per_stage[:, 4].mean())
    npairs = m2l_pairs_uniform(DEPTH)
    tc_pairs = sum(m2l_pairs_level(l) for l in range(TC_LEVEL, DEPTH + 1))
    fma = m2l_fma_per_pair(P, BASIS)
    afma = m2l_alg_fma_per_pair(P, BASIS)
    pk, pk_kind = peaks()
    mhz = pk.get("sm_max_mhz", 2070.0)
    tc = None
    if prec in (F.GEMM_BF16X3, F.GEMM_TF32X3):
        # executed tensor-core work of levels 5..6: per tile of 128 targets and
        # offset, 3 passes; the local components run in N-chunks of cw rows,
        # chunk j (lowest rank a_j) over the (p - a_j + 1)^2 multipole columns
        # it needs, rounded up to K-steps of 16 (BF16) or 8 (TF32) columns
        # (the kernel's chunk rule)
        tuning = plan.tuning()
        cw = tuning["cw"]
        ks = 16 if prec == F.GEMM_BF16X3 else 8
        nc = (P + 1) ** 2
        rk = [a for a in range(P + 1) for _ in range(2 * a + 1)]   # rank of each traceless component
        cols = sum(cw * ks * (((P - rk[r0] + 1) ** 2 + ks - 1) // ks) for r0 in range(0, nc, cw))
        tiles = sum(8 ** (l - 1) // 128 * 8 for l in range(5, DEPTH + 1))
        # kernels 0 and 1 execute 3 cw columns per K-step and chunk (3 MMAs of N = cw, or the
        # stacked hi/lo MMA of N = 2 cw and the lo.hi MMA of N = cw) for 128 cells per offset
        ex = tiles * 189 * 3 * 2 * 128 * cols
        if tuning["kernel"] in (2, 3):
            # kernel 2: per tile of 8 x TY cells (N) and offset, two K-parts x 3 K-steps x 3
            # passes of M = 128 x N x 16; offsets of planes outside the grid are skipped;
            # kernel 3: the first K-part only (the columns >= 48 on the CUDA cores)
            nkp = 2 if tuning["kernel"] == 2 else 1
            ex = 0
            for l in range(5, DEPTH + 1):
                hs = 1 << (l - 1)
                ty = 32 if l >= 6 else 16
                for c in range(8):
                    cx, cy, cz = c & 1, (c >> 1) & 1, c >> 2
                    for tk in range(hs):
                        offs = 0
                        for sc in range(8):
                            sx, sy, sz = sc & 1, (sc >> 1) & 1, sc >> 2
                            for dz in (-1, 0, 1):
                                if not 0 <= tk + dz < hs:
                                    continue
                                oz = 2 * dz + sz - cz
                                offs += sum(1 for dy in (-1, 0, 1) for dx in (-1, 0, 1)
                                            if max(abs(2 * dx + sx - cx), abs(2 * dy + sy - cy), abs(oz)) > 1)
                        ex += (hs // 8) * (hs // ty) * offs * nkp * 9 * 2 * 128 * (8 * ty) * 16
        tc = {"executed_flop_per_step": ex, "shape": tuning}
    if prec == F.FP64:
        peak = NOMINAL["sm_count"] * NOMINAL["fp64_fma_per_clk_sm"] * 2 * mhz * 1e6 / 1e12
        peak_note = "FP64 ALU: 152 SMs x 2 FMA/clk x 2 flop x %.0f MHz (nominal units, max clock)" % mhz
    else:
        peak = NOMINAL["sm_count"] * NOMINAL["fp32_fma_per_clk_sm"] * 2 * mhz * 1e6 / 1e12
        peak_note = "FP32 ALU: 152 SMs x 128 FMA/clk x 2 flop x %.0f MHz (nominal units, max clock)" % mhz
    tkey = (form, tc["shape"]["kernel"], tc["shape"]["cw"]) if tc is not None else (form, None, None)
    traffic, traffic_src = M2L_TRAFFIC.get(tkey, (None, "no capture of this kernel and shape"))
    # ALU forms: the traceless kernels contract the reduced representative
    # (sum_a (2a+1)(p-a+1)^2 = 1365 FMA at p = 8), fewer than the
    # full-multipole count F_tl (2079); the fraction is taken on the work
    # executed, so it cannot pass 1, with the F_tl-count rate beside it
    achieved = npairs * fma * 2 / (m2l_ms * 1e-3) / 1e12
    a_tl = npairs * afma * 2 / (m2l_ms * 1e-3) / 1e12
    roof = {"bound": "alu", "kernel": "m2l (levels 2..6, %d pairs per step)" % npairs,
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_source": traffic_src, "peak_source": peak_note,
            "flops_per_pair": 2 * fma,
            "flops_per_pair_is": "executed: the operator as the kernels contract it (%d FMA at p = %d)" % (fma, P),
            "F_tl_count_tflops": a_tl, "frac_of_F_tl_count": a_tl / peak, "m2l_ms_per_step": m2l_ms}
    if tc is not None:
        bf = pk.get("bf16_tflops", 1900.0)
        src = "bf16_tflops of MEASURED_PEAKS.json (%s, burst)" % pk_kind
        if prec == F.GEMM_TF32X3:
            bf *= NOMINAL_TENSOR["tf32"] / NOMINAL_TENSOR["bf16"]
            src += " x nominal TF32/BF16 ratio 1.1/2.25"
        # algorithmic work: Eq. M2L with independent local outputs and full
        # multipoles, 2 F_tl(p) flop per pair (the method's work, one
        # product); the executed work adds the three split-precision
        # products and the padding of the dense MMA tiles
        alg = tc_pairs * 2 * afma
        ach = alg / (tc_ms * 1e-3) / 1e12
        ex = tc["executed_flop_per_step"] / (tc_ms * 1e-3) / 1e12
        roof = {"bound": "tensor",
                "kernel": "tensor-core M2L, levels %d..%d (%d pairs; operand split included)" % (TC_LEVEL, DEPTH,
                                                                                               tc_pairs),
                "achieved": ach, "peak": bf, "unit": "TFLOP/s", "frac": ach / bf, "traffic": traffic,
                "traffic_source": traffic_src, "peak_source": src, "kernel_ms_per_step": tc_ms,
                "flops_per_pair": 2 * afma,
                "flops_per_pair_is": "algorithmic, Eq. M2L with full multipoles (F_tl(8) = 2079 FMA)",
                "algorithmic_flop_per_step": alg, "executed_flop_per_step": tc["executed_flop_per_step"],
                "executed_tflops": ex, "executed_frac": ex / bf,
                "split_product_tflops": 3 * tc_pairs * 2 * fma / (tc_ms * 1e-3) / 1e12,
                "kernel_shape": tc["shape"],
                "m2l_all_levels_ms_per_step": m2l_ms}

    stage_mean = {st: float(per_stage[:, i].mean()) for i, st in enumerate(stages)}
    per_op = roofline_per_op(dict(stage_mean, **sep), form, (P + 1) ** 2, DEPTH, N_PART, p2p_pairs_uniform(x, y, z, DEPTH), pk,
                             mhz, peak if prec == F.FP64 else
                             NOMINAL["sm_count"] * NOMINAL["fp32_fma_per_clk_sm"] * 2 * mhz * 1e6 / 1e12,
                             npairs * 2 * (afma if tc is not None else fma), roof["peak"] if tc is not None else None)

    # plain FP64 GPU form beside it (same workload, fewer steps)
    fp64 = None
    if prec != F.FP64 and not args.no_fp64:
        p64 = F.Plan(p=P, basis=BASIS, prec=F.FP64, depth=DEPTH)
        p64.fmm_evaluate(*X, out[0], out[1], out[2], out[3])
        tot, m2l64 = [], []
        for k in range(args.fp64_steps):
            e0, e1, e2, e3 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
            flush.fill_(2.0 + k)
            e0.record(stream)
            p64.fmm_build_tree(*X); p64.fmm_p2m(); p64.fmm_m2m()
            e1.record(stream)
            p64.fmm_m2l()
            e2.record(stream)
            p64.fmm_l2l(); p64.fmm_l2p(out[0], out[1], out[2], out[3]); p64.fmm_p2p(out[0], out[1], out[2], out[3])
            e3.record(stream)
            torch.cuda.synchronize()
            tot.append(e0.elapsed_time(e3))
            m2l64.append(e1.elapsed_time(e2))
        ms, mm = float(np.mean(tot)), float(np.mean(m2l64))
        pk64 = NOMINAL["sm_count"] * NOMINAL["fp64_fma_per_clk_sm"] * 2 * mhz * 1e6 / 1e12
        a64 = npairs * 2 * afma / (mm * 1e-3) / 1e12
        fp64 = {"value": N_PART / (ms * 1e-3), "m2l_pairs_per_s": npairs / (mm * 1e-3), "ms_per_step": ms,
                "steps": len(tot), "m2l_ms": mm,
                "m2l_roofline": {"bound": "alu", "achieved": npairs * 2 * fma / (mm * 1e-3) / 1e12, "peak": pk64,
                                 "unit": "TFLOP/s", "frac": npairs * 2 * fma / (mm * 1e-3) / 1e12 / pk64,
                                 "flops_per_pair": 2 * fma,
                                 "flops_per_pair_is": "executed: the reduced traceless representative, "
                                                      "sum_a (2a+1)(p-a+1)^2 = 1365 FMA at p = 8",
                                 "frac_of_F_tl_count": a64 / pk64,
                                 "peak_source": "FP64 ALU: 152 SMs x 2 FMA/clk x 2 flop x %.0f MHz" % mhz}}
        p64.close()
    elif prec == F.FP64:
        fp64 = {"value": value / world, "m2l_pairs_per_s": npairs / (m2l_ms * 1e-3), "ms_per_step": t_ms}
    else:
        fp64 = None   # --no-fp64: not measured

    # the same step as one fmm_evaluate replayed from a CUDA graph (device
    # arrays, L2 flushed before each step): the per-operator sequence above
    # without its ~145 separate launches and the stage events
    gr = None
    gs = torch.cuda.Stream()   # a capturable (non-default) stream
    torch.cuda.synchronize()
    with torch.cuda.stream(gs):
        for _ in range(2):   # capture, then a first replay
            plan.fmm_evaluate(*X, out[0], out[1], out[2], out[3], stream=gs)
        gts = []
        for k in range(args.steps):
            flush.fill_(3.0 + k)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(gs)
            plan.fmm_evaluate(*X, out[0], out[1], out[2], out[3], stream=gs)
            e1.record(gs)
            torch.cuda.synchronize()
            gts.append(e0.elapsed_time(e1))
    plan.sync_status()
    gms = max_over_ranks(float(np.mean(gts)), world, dist, dev)
    gr = {"value": job_rate(N_PART, world, gms * 1e-3), "ms_per_step": gms, "graph": plan.stats().get("graph"),
          "api": "fmm_evaluate (use_graph plan)"}

    # end to end through the host entry point (pinned host buffers)
    e2e = None
    if not args.no_e2e:
        hx = [torch.from_numpy(a).pin_memory() for a in (x, y, z, q)]
        ho = torch.empty((4, N_PART), dtype=torch.float64).pin_memory()
        es = torch.cuda.Stream()
        for _ in range(2):   # the first call captures the step, the second replays it
            plan.fmm_evaluate_host(*hx, ho[0], ho[1], ho[2], ho[3], stream=es)
        tms = []
        for _ in range(max(1, min(args.steps, 5))):
            t0 = time.perf_counter()
            plan.fmm_evaluate_host(*hx, ho[0], ho[1], ho[2], ho[3], stream=es)
            tms.append(time.perf_counter() - t0)
        e2e = {"value": job_rate(N_PART, world, max_over_ranks(float(np.mean(tms)), world, dist, dev)),
               "unit": "particles/s",
               "h2d_bytes_per_step": 4 * 8 * N_PART, "d2h_bytes_per_step": 4 * 8 * N_PART,
               "host_api": "fmm_evaluate_host (pinned host arrays; the step replayed from a CUDA graph)",
               "graph": plan.stats().get("graph")}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cb = cpu_reference(1, 0)
        cpu = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}

    line = {
        "metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp64": "f64", "fp32": "f32 (P2M, M2L, L2P, P2P) + f64",
                  "bf16x3": "bf16x3 tensor-core M2L + f32 (P2M, L2P, P2P) + f64",
                  "tf32x3": "tf32x3 tensor-core M2L + f32 (P2M, L2P, P2P) + f64"}[form],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": form, "p": P, "basis": "traceless", "depth": DEPTH,
                   "particles_per_gpu": N_PART, "m2l_pairs": npairs, "l2": "flushed (256 MiB write) before each step"},
        "rel_force_err": rel_err,
        "stage_ms": dict({s: float(per_stage[:, i].mean()) for i, s in enumerate(stages)}, m2l=m2l_ms),
        "l2p_p2p_as_two_steps_ms": sep,
        "m2l_pairs_per_s": world * npairs / (m2l_ms * 1e-3),
        "fp64_form": fp64,
        "vs_fp64_form": value / world / fp64["value"] if fp64 else None,
        "roofline": roof,
        "roofline_per_op": per_op,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "graph_replay": gr,
        "clocks": clk.summary(),
        "peaks_source": pk_kind,
    }
    plan.close()
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
def run_m2l_sweep(args):
    """Per-pair M2L micro-benchmark: 2^20 independent side-1 cell pairs,
    offsets uniform over the 316 well-separated integer vectors, multipoles
    from P2M of 16 unit-mass particles per cell (GPU P2M), D on the fly."""
    import torch

    from paper_1811_06332_gb300 import fmm as F
    from paper_1811_06332_gb300 import inputs
    dev = torch.device("cuda", 0)
    n = 1 << 20
    r, src, q = inputs.m2l_pairs(n, 2)
    R = torch.from_numpy(r).to(dev)
    per = src.shape[1]
    start = torch.arange(0, (n + 1) * per, per, device=dev, dtype=torch.int64)
    xs = [torch.from_numpy(np.ascontiguousarray(src[d].T.reshape(-1))).to(dev) for d in range(3)]
    qs = torch.from_numpy(np.ascontiguousarray(q.T.reshape(-1))).to(dev)
    zero = torch.zeros((3, n), device=dev, dtype=torch.float64)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ps = [int(v) for v in args.orders.split(",")]
    pk, _ = peaks()
    mhz_max = float(pk.get("sm_max_mhz", 2070.0))
    for p in ps:
        for basis in (0, 1):
            nc = F.ncoef(p, basis)
            M = torch.empty((nc, n), device=dev, dtype=torch.float64)
            F.fmm_op_p2m(p, basis, start, xs[0], xs[1], xs[2], qs, zero, M)
            res = {}
            for prec, dt in ((F.FP64, torch.float64), (F.FP32, torch.float32)):
                Mi = M.to(dt)
                L = torch.empty((nc, n), device=dev, dtype=dt)
                for _ in range(args.warmup):
                    F.fmm_op_m2l(p, basis, prec, Mi, R, L)
                times = []
                for _ in range(args.steps):
                    flush.fill_(1.0)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    F.fmm_op_m2l(p, basis, prec, Mi, R, L)
                    e1.record()
                    torch.cuda.synchronize()
                    times.append(e0.elapsed_time(e1))
                ms = float(np.median(times))
                s = 8 if prec == F.FP64 else 4
                # algorithmic work of one pair: the Eq. M2L FMAs (full
                # multipoles, independent local outputs); bytes: M in, L out,
                # the offset r (3 doubles), each once
                gbs = n * (2 * nc * s + 24) / (ms * 1e-3) / 1e9
                fma = m2l_alg_fma_per_pair(p, basis)
                tfl = n * 2 * fma / (ms * 1e-3) / 1e12
                alu_peak = alu_peak_tflops(64 if prec == F.FP64 else 32, mhz_max)
                res["fp64" if prec == F.FP64 else "fp32"] = {
                    "pairs_per_s": n / (ms * 1e-3), "ms": ms, "GB_per_s": gbs,
                    "hbm_frac": gbs / pk.get("hbm_gbs", 6800.0), "alg_fma_per_pair": fma, "TFLOP_s": tfl,
                    "alu_frac": tfl / alu_peak, "alu_peak_tflops": alu_peak}
            if not args.no_cpu:
                # the FP64 oracle's per-pair M2L (D by Eq. Detracer3, the literal
                # double loop) on the host cores, on the first 2^12 offsets with
                # seeded coefficients (the time does not depend on their values)
                import oracle
                ns_ = 1 << 12
                Mh = inputs.u01(2, 40 + p, nc * ns_).reshape(nc, ns_)
                t0 = time.perf_counter()
                oracle.m2l_batch(p, basis, Mh, r[:, :ns_])
                dt = time.perf_counter() - t0
                res["oracle_cpu"] = {"pairs_per_s": ns_ / dt, "cores": oracle.num_threads(),
                                     "sample": "first 4096 pairs, FP64"}
            print(json.dumps({"workload": "m2l per-pair, 2^20 pairs", "p": p,
                              "basis": "sym" if basis == 0 else "traceless", **res,
                              "fp32_vs_fp64": res["fp32"]["pairs_per_s"] / res["fp64"]["pairs_per_s"]}))
    return 0


def run_adaptive(args):
    """Batching-form workload: 8,388,608 particles from a Plummer sphere
    (scale radius 1, radii beyond 20 redrawn, equal masses), adaptive octree
    with at most 64 particles per leaf, MAC theta = 0.6, symmetric tensors at
    p = 6 in FP32; list M2L and P2P run as persistent kernels and the
    operator sequence replays from a captured CUDA graph.  One step = tree
    build + traversal + all operators."""
    import torch

    from paper_1811_06332_gb300 import fmm as F
    from paper_1811_06332_gb300 import inputs
    dev = torch.device("cuda", 0)
    n, p, basis, ml, theta = 8388608, 6, 0, 64, 0.6
    x, y, z = inputs.plummer(n, 4)
    q = inputs.masses_equal(n)
    X = [torch.from_numpy(a).to(dev) for a in (x, y, z, q)]
    out = torch.empty((4, n), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream()
    res = {}
    for form, prec in (("fp32", F.FP32), ("fp64", F.FP64)):
        plan = F.Plan(p=p, basis=basis, prec=prec, adaptive=True, max_leaf=ml, theta=theta, use_graph=True)
        if form == "fp64" and args.no_fp64:
            continue
        steps = args.steps if form == "fp32" else 1
        times, tb = [], []
        with torch.cuda.stream(stream):
            def one(k):
                flush.fill_(float(k))
                e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
                e0.record(stream)
                plan.fmm_evaluate(*X, out[0], out[1], out[2], out[3], stream=stream)   # tree + operators
                e1.record(stream)
                stream.synchronize()
                return e0.elapsed_time(e1)
            for k in range(args.warmup):
                one(k)
            with Clocks(0, dev) as clk:
                for k in range(steps):
                    times.append(one(args.warmup + k))
            res.setdefault("clocks_" + form, clk.summary())
            # breakdown: the same sequence through the per-operator entry
            # points (no graph), twice, the second pass recorded
            names = ["tree", "p2m", "m2m", "m2l", "l2l", "l2p", "p2p"]
            for k in range(2):
                flush.fill_(float(k))
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
                ev[0].record(stream)
                plan.fmm_build_tree(*X, stream=stream); ev[1].record(stream)
                plan.fmm_p2m(stream=stream); ev[2].record(stream)
                plan.fmm_m2m(stream=stream); ev[3].record(stream)
                plan.fmm_m2l(stream=stream); ev[4].record(stream)
                plan.fmm_l2l(stream=stream); ev[5].record(stream)
                plan.fmm_l2p(out[0], out[1], out[2], out[3], stream=stream); ev[6].record(stream)
                plan.fmm_p2p(out[0], out[1], out[2], out[3], stream=stream); ev[7].record(stream)
                stream.synchronize()
                tb = {nm: ev[i].elapsed_time(ev[i + 1]) for i, nm in enumerate(names)}
        st = plan.stats()
        res[form] = {"ms_per_step": float(np.mean(times)), "tree_ms": tb["tree"], "stage_ms": tb, "stats": st}
        if form == "fp32":
            tsel = torch.from_numpy(np.sort(np.unique((inputs.u01(4, 95, 4096) * n).astype(np.int64)))).to(dev)
            ref = torch.empty((4, len(tsel)), dtype=torch.float64, device=dev)
            F.fmm_direct(X[0], X[1], X[2], X[3], ref[0], ref[1], ref[2], ref[3], targets=tsel)
            torch.cuda.synchronize()
            acc = out[1:, tsel]
            res[form]["rel_force_err"] = float(torch.sqrt(((acc - ref[1:]) ** 2).sum() / (ref[1:] ** 2).sum()).item())
        plan.close()
    v32 = n / (res["fp32"]["ms_per_step"] * 1e-3)
    v64 = n / (res["fp64"]["ms_per_step"] * 1e-3) if "fp64" in res else None
    line = {"metric": METRIC, "value": v32, "unit": "particles/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": res["fp32"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 operators, f64 tree geometry and storage",
            "data": "synthetic",
            "config": {"workload": "Plummer sphere, 8,388,608 particles, equal masses, adaptive octree "
                                   "<= 64 per leaf, MAC theta 0.6, symmetric p=6",
                       "form": "fp32 persistent list kernels + CUDA graph", "l2": "flushed before each step",
                       "step": "fmm_build_tree + fmm_evaluate (tree, traversal, operators)"},
            "rel_force_err": res["fp32"]["rel_force_err"], "tree_ms": res["fp32"]["tree_ms"],
            "stage_ms": res["fp32"]["stage_ms"],
            "tree": res["fp32"]["stats"],
            "fp64_form": {"value": v64, "ms_per_step": res["fp64"]["ms_per_step"]} if v64 else None,
            "vs_fp64_form": v32 / v64 if v64 else None, "clocks": res["clocks_fp32"]}
    print(json.dumps(line))
    return 0


def run_small(args):
    """Small uniform workload: 4,096 particles U[0,1)^3, masses 1 - U[0,1),
    uniform octree of depth 3, symmetric p = 4, FP64 (launch-bound).  Per
    step fmm_evaluate with the tree build, and the operators alone (P2M ..
    P2P after one build); both eager and replayed from a CUDA graph, the
    median of at least 20 warm replays; the FP64 oracle FMM and the direct
    sum on the host cores beside them; errors against the direct sum."""
    import torch

    import oracle
    from paper_1811_06332_gb300 import fmm as F
    from paper_1811_06332_gb300 import inputs
    dev = torch.device("cuda", 0)
    n, depth, p = 4096, 3, 4
    x, y, z = inputs.uniform_cube(n, 1)
    q = inputs.masses_open_unit(n, 1)
    X = [torch.from_numpy(a).to(dev) for a in (x, y, z, q)]
    out = torch.empty((4, n), dtype=torch.float64, device=dev)
    stream = torch.cuda.Stream()
    reps = max(20, args.steps)

    def median_ms(fn):
        ts = []
        with torch.cuda.stream(stream):
            for k in range(args.warmup + reps):
                e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
                e0.record(stream)
                fn()
                e1.record(stream)
                stream.synchronize()
                if k >= args.warmup:
                    ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    res = {}
    for name, graph in (("eager", False), ("graph", True)):
        plan = F.Plan(p=p, basis=F.BASIS_SYM, prec=F.FP64, depth=depth, use_graph=graph)
        ev = lambda: plan.fmm_evaluate(*X, out[0], out[1], out[2], out[3], stream=stream)   # noqa: E731

        def ops():
            plan.fmm_p2m(stream=stream); plan.fmm_m2m(stream=stream); plan.fmm_m2l(stream=stream)
            plan.fmm_l2l(stream=stream); plan.fmm_l2p_p2p(out[0], out[1], out[2], out[3], stream=stream)
        res[name] = {"with_tree_ms": median_ms(ev)}
        if not graph:
            res[name]["operators_only_ms"] = median_ms(ops)
        res[name]["graph_in_use"] = bool(plan.stats()["graph"])
        plan.close()
    torch.cuda.synchronize()
    pot, acc = out[0].cpu().numpy(), out[1:].cpu().numpy()
    t0 = time.perf_counter()
    pd, ad = oracle.direct(x, y, z, q)
    t_direct = time.perf_counter() - t0
    t0 = time.perf_counter()
    po, ao = oracle.fmm_uniform(x, y, z, q, depth, p, 0)
    t_fmm = time.perf_counter() - t0
    err = float(np.linalg.norm(acc - ad) / np.linalg.norm(ad))
    ms = res["graph"]["with_tree_ms"]
    line = {"metric": METRIC, "value": n / (ms * 1e-3), "unit": "particles/s", "n_gpus": 1, "steps": reps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "uniform cube, 4,096 particles, masses 1 - U[0,1), depth-3 octree, symmetric p=4",
                       "timing": "median of %d warm steps, not flushed (the working set is ~1 MB)" % reps,
                       "step": "fmm_evaluate with the tree build, replayed from a CUDA graph"},
            "rel_force_err": err,
            "vs_oracle_fmm_rel_err": float(np.linalg.norm(acc - ao) / np.linalg.norm(ao)),
            "forms": res,
            "cpu_baseline": {"value": n / t_fmm, "unit": "particles/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": "the whole workload: oracle FMM (FP64)",
                             "direct_sum_s": t_direct}}
    print(json.dumps(line))
    return 0


def stage_breakdown(F, plan, X, out, flush):
    """One pass of the plan's operator sequence through the per-operator
    entry points (after one untimed pass), with CUDA events between them."""
    import torch
    names = ["tree", "p2m", "m2m", "m2l", "l2l", "l2p", "p2p"]
    tb = {}
    for k in range(2):
        flush.fill_(float(k))
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
        ev[0].record()
        plan.fmm_build_tree(*X); ev[1].record()
        plan.fmm_p2m(); ev[2].record()
        plan.fmm_m2m(); ev[3].record()
        plan.fmm_m2l(); ev[4].record()
        plan.fmm_l2l(); ev[5].record()
        plan.fmm_l2p(out[0], out[1], out[2], out[3]); ev[6].record()
        plan.fmm_p2p(out[0], out[1], out[2], out[3]); ev[7].record()
        torch.cuda.synchronize()
        tb = {nm: ev[i].elapsed_time(ev[i + 1]) for i, nm in enumerate(names)}
    return tb


def run_tclevel(args):
    """One tensor-core M2L level alone, per kernel shape: a 262,144-particle
    uniform cube (the M2L work of a level does not depend on the particle
    count), traceless p = 8, BF16x3, an octree of --depth levels; each shape
    times fmm_m2l_levels(l, l) on the deepest level (median of --steps after
    --warmup calls).  For kernel-level profiling on a small device footprint."""
    import torch

    from paper_1811_06332_gb300 import fmm as F
    from paper_1811_06332_gb300 import inputs
    dev = torch.device("cuda", 0)
    n, depth = 262144, args.depth
    x, y, z = inputs.uniform_cube(n, SEED)
    q = inputs.masses_equal(n)
    X = [torch.from_numpy(a).to(dev) for a in (x, y, z, q)]
    plan = F.Plan(p=P, basis=BASIS, prec=F.GEMM_BF16X3, depth=depth)
    plan.fmm_build_tree(*X)
    plan.fmm_p2m()
    plan.fmm_m2m()
    res = {}
    for shape in args.tc_shapes.split(","):
        kern, cw = (int(v) for v in shape.split(":"))
        plan.set_tc_shape(kern, cw)
        ts = []
        for k in range(args.warmup + args.steps):
            e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
            e0.record()
            plan.fmm_m2l_levels(depth, depth)
            e1.record()
            torch.cuda.synchronize()
            if k >= args.warmup:
                ts.append(e0.elapsed_time(e1))
        res["%d:%d" % (kern, cw)] = float(np.median(ts))
    plan.sync_status()
    plan.close()
    print(json.dumps({"workload": "tensor-core M2L, level %d of a depth-%d uniform octree, traceless p=%d, bf16x3"
                      % (depth, depth, P), "ms_per_level_by_shape": res, "steps": args.steps,
                      "warmup": args.warmup}))
    return 0


def run_variant(args):
    """Sec. 3 and App. C variants on the batching-form workload (8,388,608
    Plummer particles, MAC theta 0.6, traceless p = 6, FP64): --workload ap:
    the AP variant (centre-of-mass centres, dipole 0, gradient only) on the
    adaptive octree with <= 64 particles per leaf; --workload binary: the
    binary median-split tree with shrink-wrapped cells, at leaf bounds 64, 32
    and 16 (a median split leaves 32..64 particles per leaf at bound 64,
    against 19 on average for the octree), the fastest reported.  Beside
    each, the same FP64 traceless FMM on the adaptive octree (<= 64 per leaf)
    about geometric centres.  One step = fmm_evaluate (tree, centres,
    traversal, operators)."""
    import torch

    from paper_1811_06332_gb300 import fmm as F
    from paper_1811_06332_gb300 import inputs
    dev = torch.device("cuda", 0)
    n, p, theta = 8388608, 6, 0.6
    x, y, z = inputs.plummer(n, 4)
    q = inputs.masses_equal(n)
    X = [torch.from_numpy(a).to(dev) for a in (x, y, z, q)]
    out = torch.empty((4, n), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    tsel = torch.from_numpy(np.sort(np.unique((inputs.u01(4, 95, 4096) * n).astype(np.int64)))).to(dev)
    ref = torch.empty((4, len(tsel)), dtype=torch.float64, device=dev)
    F.fmm_direct(X[0], X[1], X[2], X[3], ref[0], ref[1], ref[2], ref[3], targets=tsel)
    kind = args.workload
    runs = [("octree_geometric", 64, {})]
    if kind == "ap":
        runs.append(("ap", 64, dict(ap=True)))
    else:
        runs += [("binary_leaf%d" % ml, ml, dict(binary_tree=True)) for ml in (64, 32, 16)]
    res = {}
    for name, ml, kw in runs:
        plan = F.Plan(p=p, basis=F.BASIS_TRACELESS, prec=F.FP64, adaptive=True, max_leaf=ml, theta=theta, **kw)
        times = []
        for k in range(args.warmup + args.steps):
            flush.fill_(float(k))
            e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
            e0.record()
            plan.fmm_evaluate(*X, out[0], out[1], out[2], out[3])
            e1.record()
            torch.cuda.synchronize()
            if k >= args.warmup:
                times.append(e0.elapsed_time(e1))
        acc = out[1:, tsel]
        err = float(torch.sqrt(((acc - ref[1:]) ** 2).sum() / (ref[1:] ** 2).sum()).item())
        res[name] = {"max_leaf": ml, "ms_per_step": float(np.mean(times)), "rel_force_err": err,
                     "stage_ms": stage_breakdown(F, plan, X, out, flush), "stats": plan.stats()}
        plan.close()
    best = min((k for k in res if k != "octree_geometric"), key=lambda k: res[k]["ms_per_step"])
    ms = res[best]["ms_per_step"]
    form = {"ap": "AP variant (centre-of-mass centres, dipole 0, gradient only), FP64",
            "binary": "binary median-split tree, shrink-wrapped cells, FT, FP64"}[kind]
    tree = {"ap": "adaptive octree <= 64 per leaf",
            "binary": "binary median-split tree <= %d per leaf" % res[best]["max_leaf"]}[kind]
    line = {"metric": METRIC, "value": n / (ms * 1e-3), "unit": "particles/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "Plummer sphere, 8,388,608 particles, equal masses, %s, MAC theta 0.6, "
                                   "traceless p=6" % tree,
                       "form": form, "l2": "flushed before each step"},
            "rel_force_err": res[best]["rel_force_err"], "runs": res,
            "vs_octree_geometric_centres": res["octree_geometric"]["ms_per_step"] / ms}
    print(json.dumps(line))
    return 0


def run_learned(args):
    """Learned-order form: 16,777,216 particles, 32 Gaussian blobs (sigma
    U[0.005, 0.05], centres U[0,1)^3) plus a 10% uniform background, equal
    masses, adaptive octree with at most 64 particles per leaf, MAC theta
    0.6, target relative force error 1e-4.  The order model is trained on the
    GPU on a Plummer and a blob set (65,536 particles each, other seeds), its
    kappa calibrated per storage order on a third set (262,144 particles),
    then the full set is evaluated with the learned orders and with fixed
    orders (the lowest uniform p reaching 1e-4, 8 and 10).  One step =
    fmm_evaluate (tree, traversal, features, inference, operators)."""
    import torch

    from paper_1811_06332_gb300 import fmm as F
    from paper_1811_06332_gb300 import inputs, order_model
    dev = torch.device("cuda", 0)
    n, ml, theta, target = 1 << 24, 64, 0.6, 1e-4
    t0 = time.time()
    # ---- training and calibration (untimed)
    sets = []
    for gen, sd in ((inputs.plummer, 301), (inputs.blobs, 302)):
        x, y, z = gen(65536, sd)
        sets.append((x, y, z, inputs.masses_equal(65536)))
    feat, lab = order_model.pair_samples(sets, ml, theta)
    blob, losses = order_model.train(feat, lab, seed=303, epochs=20, batch=1024, lr=2e-3)
    xc, yc, zc = inputs.blobs(262144, 304)
    Xc = (xc, yc, zc, inputs.masses_equal(262144))
    cal = {}
    for P in (8, 6):
        cal[P] = order_model.calibrate(blob, Xc, P, ml, theta, target)
    t_train = time.time() - t0
    # ---- the full set
    x, y, z = inputs.blobs(n, 5)
    q = inputs.masses_equal(n)
    X = [torch.from_numpy(a).to(dev) for a in (x, y, z, q)]
    out = torch.empty((4, n), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream()

    def run(p, prec=F.FP32, blob_p=None, steps=args.steps, warmup=args.warmup):
        plan = F.Plan(p=p, basis=F.BASIS_SYM, prec=prec, adaptive=True, max_leaf=ml, theta=theta,
                      use_graph=True, learned_p=blob_p is not None, target_rel_err=target)
        if blob_p is not None:
            plan.set_mlp(blob_p)
        times = []
        with torch.cuda.stream(stream):
            for k in range(warmup + steps):
                flush.fill_(float(k))
                e0, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(2))
                e0.record(stream)
                plan.fmm_evaluate(*X, out[0], out[1], out[2], out[3], stream=stream)
                e1.record(stream)
                stream.synchronize()
                if k >= warmup:
                    times.append(e0.elapsed_time(e1))
        err = order_model.force_error(out[1:], X, 4096, 5)
        # stage breakdown through the per-operator entry points (no graph)
        names = ["tree", "p2m", "m2m", "m2l", "l2l", "l2p", "p2p"]
        with torch.cuda.stream(stream):
            flush.fill_(0.5)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(8)]
            ev[0].record(stream)
            plan.fmm_build_tree(*X, stream=stream); ev[1].record(stream)
            plan.fmm_p2m(stream=stream); ev[2].record(stream)
            plan.fmm_m2m(stream=stream); ev[3].record(stream)
            plan.fmm_m2l(stream=stream); ev[4].record(stream)
            plan.fmm_l2l(stream=stream); ev[5].record(stream)
            plan.fmm_l2p(out[0], out[1], out[2], out[3], stream=stream); ev[6].record(stream)
            plan.fmm_p2p(out[0], out[1], out[2], out[3], stream=stream); ev[7].record(stream)
            stream.synchronize()
        stages = {nm: round(ev[i].elapsed_time(ev[i + 1]), 3) for i, nm in enumerate(names)}
        st = plan.stats()
        plan.close()
        r = {"p": p, "ms_per_step": float(np.mean(times)), "rel_force_err": err,
             "particles_per_s": n / (np.mean(times) * 1e-3), "m2l_pairs": st["m2l_pairs"], "stage_ms": stages}
        if "pairs_per_order" in st:
            c = np.array(st["pairs_per_order"], dtype=np.float64)
            r["pairs_per_order"] = st["pairs_per_order"]
            r["mean_order"] = float((c * np.arange(len(c))).sum() / max(c.sum(), 1))
            # M2L FMAs of Eq. M2L, symmetric form: C(q+6, 6) per pair at order q
            from math import comb
            r["m2l_fma_vs_fixed"] = float((c * np.array([comb(k + 6, 6) for k in range(len(c))])).sum() /
                                          (c.sum() * comb(p + 6, 6)))
        return r

    res = {"learned_p8": run(8, blob_p=cal[8][0]), "learned_p6": run(6, blob_p=cal[6][0])}
    uni = {}
    for p in (4, 5, 6, 7, 8):
        uni[p] = run(p, steps=2, warmup=1)
        if uni[p]["rel_force_err"] <= target:
            break
    p_uni = min((p for p in uni if uni[p]["rel_force_err"] <= target), default=max(uni))
    fixed10 = run(10, steps=1, warmup=1)
    fp64 = run(p_uni, prec=F.FP64, steps=1, warmup=1)
    best = min((r for r in (res["learned_p8"], res["learned_p6"]) if r["rel_force_err"] <= target),
               key=lambda r: r["ms_per_step"], default=res["learned_p8"])
    line = {"metric": METRIC, "value": best["particles_per_s"], "unit": "particles/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 operators, bf16 MLP on tensor cores, f64 tree geometry and storage",
            "data": "synthetic",
            "config": {"workload": "32 Gaussian blobs + 10% uniform background, 16,777,216 particles, adaptive "
                                   "octree <= 64 per leaf, MAC theta 0.6, learned per-pair order, target 1e-4",
                       "l2": "flushed before each step", "step": "fmm_evaluate (tree, lists, features, "
                                                                 "inference, grouping, operators)"},
            "rel_force_err": best["rel_force_err"],
            "learned": res, "uniform": {str(k): v for k, v in uni.items()}, "lowest_uniform_p": p_uni,
            "fixed_p10": fixed10, "fp64_form_at_lowest_uniform_p": fp64,
            "vs_lowest_uniform": best["particles_per_s"] / uni[p_uni]["particles_per_s"],
            "vs_fixed_p10": best["particles_per_s"] / fixed10["particles_per_s"],
            "vs_fp64_form": best["particles_per_s"] / fp64["particles_per_s"],
            "training": {"pairs": int(feat.shape[0]), "epoch_loss_first_last": [float(losses[0]),
                                                                               float(losses[-1])],
                         "calibration": {str(P): cal[P][1] for P in cal}, "seconds": t_train}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="bf16x3", choices=["fp64", "fp32", "bf16x3", "tf32x3"])
    ap.add_argument("--workload", default="fmm",
                    choices=["fmm", "small", "m2l", "adaptive", "learned", "ap", "binary", "tclevel"])
    ap.add_argument("--tc-shapes", default="0:48,2:256,3:256", help="tclevel: kernel:cw list")
    ap.add_argument("--depth", type=int, default=6, help="tclevel: octree depth (the level timed)")
    ap.add_argument("--orders", default="2,3,4,5,6,7,8,9,10")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=5)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours" and args.workload == "fmm":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    import __graft_entry__ as g
    g.build()
    if args.workload == "m2l":
        return run_m2l_sweep(args)
    if args.workload == "small":
        return run_small(args)
    if args.workload == "adaptive":
        return run_adaptive(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload in ("ap", "binary"):
        return run_variant(args)
    if args.workload == "tclevel":
        return run_tclevel(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
