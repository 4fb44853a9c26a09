"""Benchmark of the accelerated hot path on GB300.

One step = one pass of every hot-path row over its synthetic workload, inputs resident in
HBM when the timed region starts:
  segreduce   4,096 int32 sequences (lengths U{0..256}, values U{-1000..1000}): ragged
              marshal -> fused map x*x+1 + int64 segmented sum -> int64 max; plus the loop
              body b = 2a over the flat data
  hmm_plain   FP32 log-space HMM forward, K=64, M=32, 512 sequences x 1000 steps
  hmm_bf16    BF16 tensor-core scaled forward, K=256, M=64, 4,096 sequences, lengths
              log-uniform in [50, 5000], one persistent launch
  hmm_adjoint forward + adjoint, K=256, M=64, 1,024 sequences, lengths U{200..2000}
  hmm_mstep   the re-estimation that follows: softmax-parameterised gradient and
              Baum-Welch M-step from the adjoint's expected counts
  allpairs    records {pos: float3, mass: float} -> SoA, all-pairs softened gravity, N=65,536

Metric: HMM state-steps per second (K x sum of lengths, counted once for every forward
pass and once for every adjoint pass) over the whole step; per-row times, the segmented
reduce's and the marshal's GB/s at HBM scale and every kernel's roofline fraction are
reported beside it.  ALU rooflines use the FP32 rate measured in the same run
(accel_alu_rate); the tensor and HBM ones the measured peaks.

The CPU leg (rank 0, N=1) times the float64 oracle on the host cores -- one worker and one
worker per allowed core, in each configuration's own unit -- and, from the oracle values it
computes, states every result's error against the oracle (`errors`).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
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

from paper_2211_00621_gb300 import synth  # noqa: E402

METRIC = "HMM fwd+adjoint state-steps/s & seg-reduce GB/s vs plain form, 1 GB300"
UNIT = "state-steps/s"
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
L2_FLUSH_BYTES = 256 << 20


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------ workloads
def hmm_inputs(cfg, torch, dev):
    p = synth.hmm_workload(cfg["seed"], cfg["K"], cfg["M"], cfg["S"], cfg["kind"], cfg["lo"], cfg["hi"])
    logs = synth.hmm_log_inputs_f32(p)
    d = {k: torch.from_numpy(v).to(dev) for k, v in logs.items()}
    d["obs"] = torch.from_numpy(p["obs"]).to(dev)
    d["offsets"] = torch.from_numpy(p["offsets"]).to(dev)
    d["host"] = {"obs": p["obs"], "offsets": p["offsets"], **logs}
    d["K"], d["S"], d["sumT"], d["maxT"] = cfg["K"], cfg["S"], int(p["lengths"].sum()), int(p["lengths"].max())
    d["M"] = cfg["M"]
    return d


class Workload:
    def __init__(self, torch, dev, with_adjoint: bool):
        from paper_2211_00621_gb300 import api
        self.torch, self.dev, self.api = torch, dev, api
        c = synth.CFG_SEGREDUCE
        seqs = synth.ragged_int32(c["seed"], c["S"], c["len_lo"], c["len_hi"], c["val_lo"], c["val_hi"])
        self.seq_host = seqs
        self.seq_dev = [torch.from_numpy(s).to(dev) for s in seqs]
        self.seg_N = int(sum(len(s) for s in seqs))
        self.seg_S = c["S"]
        self.table_dev = api.ragged_table(self.seq_dev)
        self.seq_pinned = [torch.from_numpy(s).pin_memory() for s in seqs]
        self.table_pinned = api.ragged_table(self.seq_pinned)
        self.plain = hmm_inputs(synth.CFG_HMM_PLAIN, torch, dev)
        self.bf16 = hmm_inputs(synth.CFG_HMM_BATCHED, torch, dev)
        self.adj = hmm_inputs(synth.CFG_HMM_ADJOINT, torch, dev) if with_adjoint else None
        b = synth.bodies(synth.CFG_ALLPAIRS["seed"], synth.CFG_ALLPAIRS["N"])
        self.aos_host = b["aos"]
        self.aos = torch.from_numpy(b["aos"]).to(dev)
        self.N = synth.CFG_ALLPAIRS["N"]
        self.eps = synth.CFG_ALLPAIRS["eps"]
        f32 = torch.float32
        self.fields = [(0, f32), (4, f32), (8, f32), (12, f32)]
        self.with_adjoint = with_adjoint
        self.bf16_graph = None
        self.bf16_out = None
        self.seg_graph = None
        self.tuned = None

    def tune_and_capture(self, tune_cache=None):
        """Autotune the batched BF16 forward's launch configuration on its inputs (or take it
        from the JSON-lines file `tune_cache`), then capture the call (preparation kernels + the
        one persistent launch) into a CUDA graph."""
        import ctypes as C
        api, torch = self.api, self.torch
        q = self.bf16
        ms, cfg = api.hmm_autotune(q["log_A"], q["log_B"], q["log_pi"], q["obs"], q["offsets"], cache_path=tune_cache)
        self.tuned = {"split": cfg[0], "rows": cfg[1], "pair": cfg[2], "units": cfg[3], "best_ms": ms}
        lib = api.L.load()
        m = api._model(q["log_A"], q["log_B"], q["log_pi"])
        nb = lib.hmm_forward_workspace_size(C.byref(m), q["S"], q["obs"].numel(), api.HMM_BF16_SCALED)
        self.bf16_ws = torch.empty(nb, dtype=torch.uint8, device=self.dev)
        self.bf16_out = torch.empty(q["S"], dtype=torch.float64, device=self.dev)
        side = torch.cuda.Stream()
        self.side = torch.cuda.Stream()     # the overlapped BF16 row of a step
        self.side2 = torch.cuda.Stream()    # ... and the adjoint's forward phase
        self.n_sms = torch.cuda.get_device_properties(self.dev).multi_processor_count
        torch.cuda.synchronize()
        g = api.Graph()
        g.capture(lambda: api.hmm_forward(q["log_A"], q["log_B"], q["log_pi"], q["obs"], q["offsets"],
                                          api.HMM_BF16_SCALED, out=self.bf16_out, ws=self.bf16_ws), stream=side)
        torch.cuda.synchronize()
        self.bf16_graph = g
        self.tuned["graph_nodes"] = g.nodes()
        self.capture_seg(side)

    def capture_seg(self, side):
        """The seg-reduce row (ragged marshal -> fused map + int64 segmented sum -> int64 max,
        and the loop b = 2a over the flat data, a parallel branch after the marshal) captured
        into one CUDA graph over buffers allocated once: the config-1 latency without a host
        round trip per call."""
        api, torch, dev = self.api, self.torch, self.dev
        lib = api.L.load()
        N, S = self.seg_N, self.seg_S
        b = {"flat": torch.empty(N, dtype=torch.int32, device=dev),
             "off": torch.empty(S + 1, dtype=torch.int64, device=dev),
             "ws_m": torch.empty(lib.accel_marshal_ragged_workspace_size(S), dtype=torch.uint8, device=dev),
             "seg": torch.empty(S, dtype=torch.int64, device=dev),
             "ws_s": torch.empty(lib.accel_segreduce_workspace_size(N, S), dtype=torch.uint8, device=dev),
             "max": torch.empty(1, dtype=torch.int64, device=dev),
             "ws_r": torch.empty(max(lib.accel_reduce_workspace_size(S, api.L.I64), 256), dtype=torch.uint8,
                                 device=dev),
             "twice": torch.empty(N, dtype=torch.int32, device=dev)}
        self.seg_bufs = b

        fork = torch.cuda.Stream()

        def body():
            cur = torch.cuda.current_stream()
            api.accel_marshal_ragged_table(self.table_dev, out=(b["flat"], b["off"]), ws=b["ws_m"])
            # the loop over the flat data does not depend on the reductions: a parallel branch
            e0 = torch.cuda.Event()
            e0.record(cur)
            fork.wait_event(e0)
            with torch.cuda.stream(fork):
                api.accel_loop(api.LOOP_SCALE, b["twice"], b["flat"], 2.0)
            api.accel_segreduce(api.RED_ADD, api.MAP_SQ_PLUS_ONE, b["flat"], b["off"], torch.int64, out=b["seg"],
                                ws=b["ws_s"])
            api.accel_reduce(api.RED_MAX, b["seg"], out=b["max"], ws=b["ws_r"])
            e1 = torch.cuda.Event()
            e1.record(fork)
            cur.wait_event(e1)
        torch.cuda.synchronize()
        g = api.Graph()
        n0 = lib.accel_launch_count()
        g.capture(body, stream=side)
        self.seg_kernels = int(lib.accel_launch_count() - n0)    # kernels in one replay
        torch.cuda.synchronize()
        self.seg_graph = g
        self.seg_graph_nodes = g.nodes()

    def state_steps(self):
        n = self.plain["K"] * self.plain["sumT"] + self.bf16["K"] * self.bf16["sumT"]
        if self.adj is not None:
            n += 2 * self.adj["K"] * self.adj["sumT"]
        return n

    # one step, device-resident inputs.  With `ev` (per-row (start, end) events) the rows run one
    # after another on the current stream, so each row's time is its own.  Without it the
    # step overlaps independent rows: the batched BF16 forward -- a latency-bound persistent
    # launch whose CTAs fill the register files of the SMs they hold and leave the others
    # idle -- runs on a second stream; the adjoint's forward phase runs on a third within the
    # SMs the BF16 launch leaves (accel_set_sm_budget), and the seg-reduce, plain FP32 and
    # all-pairs rows on the main stream take what is free; the adjoint's backward rounds and
    # the re-estimation, which want every SM, follow.
    def adj_budget(self):
        """SMs for the adjoint's forward phase in the step: those the BF16 forward's persistent
        clusters leave, less a tenth of the device for the rows that run beside them (measured
        at 152 SMs: budgets 94 / 86 / 78 / 70 gave steps of 19.70 / 19.60 / 19.45 / 19.67 ms)."""
        units = (self.tuned or {}).get("units", 0)
        nc = 2 if (self.tuned or {}).get("pair", 0) == 1 else 4 if (self.tuned or {}).get("pair", 0) == 2 else 1
        free = self.n_sms - units * nc - self.n_sms // 10
        return free if units > 0 and free > 0 else 0

    def adj_forward_side(self, cur, adj_inputs):
        """The adjoint's forward phase on the third stream within the free SMs; returns
        (logL, saved state, event)."""
        api, torch = self.api, self.torch
        a = adj_inputs
        e_in = torch.cuda.Event()
        e_in.record(cur)
        self.side2.wait_event(e_in)
        with torch.cuda.stream(self.side2):
            api.set_sm_budget(self.adj_budget())
            try:
                ll, saved = api.hmm_adjoint_forward(a["log_A"], a["log_B"], a["log_pi"], a["obs"], a["offsets"],
                                                    max_T=self.adj["maxT"])
            finally:
                api.set_sm_budget(0)
            e_af = torch.cuda.Event()
            e_af.record(self.side2)
        ll.record_stream(cur)
        saved.ws.record_stream(cur)
        return ll, saved, e_af

    def step(self, ev=None):
        api, torch = self.api, self.torch
        overlap = ev is None and self.bf16_graph is not None
        cur = torch.cuda.current_stream()
        if overlap:
            e_in = torch.cuda.Event()
            e_in.record(cur)
            self.side.wait_event(e_in)
            self.bf16_graph.launch(stream=self.side)
            e_bf16 = torch.cuda.Event()
            e_bf16.record(self.side)
            if self.adj is not None:
                adj_ll, adj_saved, e_af = self.adj_forward_side(cur, self.adj)

        def mark(name, fn):
            if ev is None:
                return fn()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            r = fn()
            b.record()
            ev.setdefault(name, []).append((a, b))
            return r

        def seg():
            if self.seg_graph is not None:
                self.seg_graph.launch()
                return self.seg_bufs["seg"], self.seg_bufs["max"]
            flat, off = api.accel_marshal_ragged_table(self.table_dev)
            s = api.accel_segreduce(api.RED_ADD, api.MAP_SQ_PLUS_ONE, flat, off, torch.int64)
            m = api.accel_reduce(api.RED_MAX, s)
            twice = torch.empty_like(flat)
            api.accel_loop(api.LOOP_SCALE, twice, flat, 2.0)
            return s, m

        out = {}
        out["seg"] = mark("segreduce", seg)
        p = self.plain
        out["plain"] = mark("hmm_plain", lambda: api.hmm_forward(p["log_A"], p["log_B"], p["log_pi"], p["obs"],
                                                                 p["offsets"], api.HMM_FP32_LOG))
        q = self.bf16
        if overlap:
            def allpairs_row():
                x, y, z, m = api.accel_marshal_records(self.aos, self.fields)
                return api.pairwise_mapreduce(x, y, z, m, self.eps)
            out["allpairs"] = allpairs_row()
            out["bf16"] = self.bf16_out         # joined at the end of the step
        elif self.bf16_graph is not None:
            def bf16():
                self.bf16_graph.launch()
                return self.bf16_out
            out["bf16"] = mark("hmm_bf16", bf16)
        else:
            out["bf16"] = mark("hmm_bf16", lambda: api.hmm_forward(q["log_A"], q["log_B"], q["log_pi"], q["obs"],
                                                                   q["offsets"], api.HMM_BF16_SCALED))
        if self.adj is not None:
            a = self.adj

            def adjoint():
                # one pass: the adjoint's checkpointed forward returns logL, then the backward
                return api.hmm_adjoint(a["log_A"], a["log_B"], a["log_pi"], a["obs"], a["offsets"],
                                       max_T=a["maxT"], want_loglik=True)
            if overlap:
                cur.wait_event(e_af)
                g3 = api.hmm_adjoint_backward(a["log_A"], a["log_B"], a["log_pi"], a["obs"], a["offsets"], adj_saved)
                out["adj"] = (*g3, adj_ll)
            else:
                out["adj"] = mark("hmm_adjoint", adjoint)
            g = out["adj"]
            # the re-estimation that follows the adjoint in a training step
            out["mstep"] = mark("hmm_mstep", lambda: api.hmm_mstep(a["log_A"], a["log_B"], a["log_pi"], g[0], g[1],
                                                                   g[2]))
        if overlap:
            # the adjoint's backward phase starts when its forward phase ends, on the SMs the
            # BF16 forward leaves until it finishes
            cur.wait_event(e_bf16)

        if not overlap:
            def allpairs():
                x, y, z, m = api.accel_marshal_records(self.aos, self.fields)
                return api.pairwise_mapreduce(x, y, z, m, self.eps)
            out["allpairs"] = mark("allpairs", allpairs)
        return out

    # end-to-end step: inputs copied from pinned host memory, results read back
    def e2e_step(self, host):
        api, torch, dev = self.api, self.torch, self.dev
        st = torch.cuda.current_stream()
        res = []
        # ragged pieces are read by the marshal kernel straight from pinned host memory
        flat, off = api.accel_marshal_ragged_table(self.table_pinned)
        s = api.accel_segreduce(api.RED_ADD, api.MAP_SQ_PLUS_ONE, flat, off, torch.int64)
        m = api.accel_reduce(api.RED_MAX, s)
        res += [s, m]
        # the BF16 row on the second stream, beside the rows that follow (as in step())
        e_in = torch.cuda.Event()
        e_in.record(st)
        self.side.wait_event(e_in)
        with torch.cuda.stream(self.side):
            h = host["bf16"]
            d = {k: v.to(dev, non_blocking=True) for k, v in h.items()}
            r_bf16 = api.hmm_forward(d["log_A"], d["log_B"], d["log_pi"], d["obs"], d["offsets"], api.HMM_BF16_SCALED)
            e_bf16 = torch.cuda.Event()
            e_bf16.record(self.side)
        if self.adj is not None:
            # the adjoint's inputs and forward phase on the third stream (as in step())
            self.side2.wait_event(e_in)
            with torch.cuda.stream(self.side2):
                dadj = {k: v.to(dev, non_blocking=True) for k, v in host["adj"].items()}
            adj_ll, adj_saved, e_af = self.adj_forward_side(st, dadj)
            for v in dadj.values():
                v.record_stream(st)
        h = host["plain"]
        d = {k: v.to(dev, non_blocking=True) for k, v in h.items()}
        res.append(api.hmm_forward(d["log_A"], d["log_B"], d["log_pi"], d["obs"], d["offsets"], api.HMM_FP32_LOG))
        aos = host["aos"].to(dev, non_blocking=True)
        x, y, z, mm = api.accel_marshal_records(aos, self.fields)
        res += list(api.pairwise_mapreduce(x, y, z, mm, self.eps))
        if self.adj is not None:
            st.wait_event(e_af)
            d = dadj
            gA, gB, gpi = api.hmm_adjoint_backward(d["log_A"], d["log_B"], d["log_pi"], d["obs"], d["offsets"],
                                                   adj_saved)
            th, nw = api.hmm_mstep(d["log_A"], d["log_B"], d["log_pi"], gA, gB, gpi)
            res += [gA, gB, gpi, adj_ll, *th, *nw]
        st.wait_event(e_bf16)
        r_bf16.record_stream(st)
        res.append(r_bf16)
        outs = [torch.empty(r.shape, dtype=r.dtype, pin_memory=True) for r in res]
        for o, r in zip(outs, res):
            o.copy_(r, non_blocking=True)
        st.synchronize()
        return sum(o.numel() * o.element_size() for o in outs)

    def host_inputs(self):
        torch = self.torch
        h = {}
        for name, d in (("plain", self.plain), ("bf16", self.bf16), ("adj", self.adj)):
            if d is None:
                continue
            h[name] = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in d["host"].items()}
        h["aos"] = torch.from_numpy(self.aos_host).pin_memory()
        nb = sum(t.numel() * t.element_size() for name in h if name != "aos" for t in h[name].values())
        nb += h["aos"].numel() * 4
        nb += 4 * self.seg_N + 16 * self.seg_S          # ragged pieces + pointer/length tables
        return h, nb


# ------------------------------------------------------------------------ rooflines
def source_hash(path):
    with open(path, "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()[:12]


def traffic_for(row: str):
    """DRAM bytes per launch of a row's call, from a committed ncu summary, if none of the
    row's kernel sources has changed since the capture (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(row)
    if not e:
        return None
    for name, sha in e.get("sources", {}).items():
        src = os.path.join(ROOT, "paper_2211_00621_gb300", "csrc", name)
        if not os.path.exists(src) or source_hash(src) != sha:
            return None
    return e.get("dram_bytes_per_launch")


def measure_alu(api):
    """Arithmetic rates measured on this GPU at its running clocks (best of three launches
    each): FP32 FMA and packed FMA (flop/s), MUFU rsqrt (op/s), FP64 FMA (flop/s)."""
    L = api.L
    r = {}
    for name, kind in (("ffma", L.PROBE_FFMA), ("ffma2", L.PROBE_FFMA2), ("rsqrt", L.PROBE_RSQRT),
                       ("dfma", L.PROBE_DFMA)):
        r[name] = max(api.alu_rate(kind, iters=2048 if name != "dfma" else 64) for _ in range(3))
    r["fp32_tflops"] = max(r["ffma"], r["ffma2"]) / 1e12
    return r


def rooflines(W, row_ms, peaks, fp32_peak):
    """Per-row roofline: algorithmic work / time against the bounding unit's peak
    (fp32_peak: the FP32 rate measured in this run, TFLOP/s)."""
    r = {}
    seg_bytes = 4 * W.seg_N * 3 + 8 * (W.seg_S + 1) * 3 + 8 * W.seg_S * 2 + 16 * W.seg_S
    r["segreduce"] = {"bound": "hbm", "achieved": seg_bytes / (row_ms["segreduce"] * 1e-3) / 1e9,
                      "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    p = W.plain
    r["hmm_plain"] = {"bound": "alu", "achieved": 2 * p["K"] ** 2 * p["sumT"] / (row_ms["hmm_plain"] * 1e-3) / 1e12,
                      "peak": fp32_peak, "unit": "TFLOP/s"}
    q = W.bf16
    r["hmm_bf16"] = {"bound": "tensor", "achieved": 2 * q["K"] ** 2 * q["sumT"] / (row_ms["hmm_bf16"] * 1e-3) / 1e12,
                     "peak": peaks["bf16_tflops_sustained"], "unit": "TFLOP/s"}
    if W.adj is not None and "hmm_mstep" in row_ms:
        a = W.adj
        nb = 16 * (a["K"] * a["K"] + a["K"] * a["M"] + a["K"])      # read log P and g, write two outputs
        r["hmm_mstep"] = {"bound": "hbm", "achieved": nb / (row_ms["hmm_mstep"] * 1e-3) / 1e9,
                          "peak": peaks["hbm_gbs"], "unit": "GB/s"}
    if W.adj is not None and "hmm_adjoint" in row_ms:
        a = W.adj
        # 8 K^2 flop per time step: the forward, the checkpoint recomputation, the backward
        # recursion and the xi accumulation, 2 K^2 each (6 K^2 without the recomputation)
        sec = row_ms["hmm_adjoint"] * 1e-3
        r["hmm_adjoint"] = {"bound": "alu", "achieved": 8 * a["K"] ** 2 * a["sumT"] / sec / 1e12,
                            "peak": fp32_peak, "unit": "TFLOP/s", "flop_per_step": "8 K^2",
                            "achieved_6K2": 6 * a["K"] ** 2 * a["sumT"] / sec / 1e12}
    r["allpairs"] = {"bound": "alu", "achieved": 20.0 * W.N * W.N / (row_ms["allpairs"] * 1e-3) / 1e12,
                     "peak": fp32_peak, "unit": "TFLOP/s"}
    for v in r.values():
        v["frac"] = v["achieved"] / v["peak"]
    return r


# ---------------------------------------------------------------------- CPU oracle
# The oracle as it stands, timed on the host cores: each worker process (spawned, so it never
# inherits a CUDA context) runs one kind of unit for `seconds` and returns (units, seconds).
#   hmm       random sequences of the three HMM configurations: the forward (K=64 plain and
#             K=256 batched) or the forward-backward (K=256 adjoint); unit = state-steps, K
#             per time step and pass (forward-backward counts two passes, as on the GPU)
#   segreduce the config-1 segmented sum of x*x+1 (the oracle's vectorised form); unit = bytes
#             of the algorithmic traffic 4 N + 16 S
#   allpairs  the acceleration of random bodies of the N = 65,536 set; unit = interactions
def _oracle_units(kind: str, seconds: float, seed: int):
    from oracle import hmm as ohmm
    from oracle import pairwise as opair
    from oracle import patterns as op
    g = synth.rng(seed)
    units, busy = 0, 0.0
    if kind == "hmm":
        cfgs = [(synth.CFG_HMM_PLAIN, False), (synth.CFG_HMM_BATCHED, False), (synth.CFG_HMM_ADJOINT, True)]
        work = []
        for c, fb in cfgs:
            p = synth.hmm_workload(c["seed"], c["K"], c["M"], c["S"], c["kind"], c["lo"], c["hi"])
            work.append((p, ohmm.params_from_f32_logs(synth.hmm_log_inputs_f32(p)), fb))
        t_end = time.perf_counter() + seconds
        while time.perf_counter() < t_end:
            for p, par, fb in work:
                sq = int(g.integers(0, p["S"]))
                t0 = time.perf_counter()
                if fb:
                    ohmm.gradients_batch(p, seqs=[sq], params=par)
                else:
                    ohmm.loglik_batch(p, seqs=[sq], params=par)
                busy += time.perf_counter() - t0
                units += (2 if fb else 1) * p["K"] * int(p["lengths"][sq])
    elif kind == "segreduce":
        c = synth.CFG_SEGREDUCE
        data, lengths = synth.ragged_flat_int32(c["seed"], c["S"], c["len_lo"], c["len_hi"], c["val_lo"], c["val_hi"])
        off = np.zeros(c["S"] + 1, np.int64)
        np.cumsum(lengths, out=off[1:])
        nbytes = 4 * len(data) + 16 * c["S"]
        t_end = time.perf_counter() + seconds
        while time.perf_counter() < t_end:
            t0 = time.perf_counter()
            op.segreduce_fast(op.RED_ADD, op.MAP_SQ_PLUS_ONE, data, off, np.int64)
            busy += time.perf_counter() - t0
            units += nbytes
    elif kind == "allpairs":
        b = synth.bodies(synth.CFG_ALLPAIRS["seed"], synth.CFG_ALLPAIRS["N"])
        pos, mass = b["aos"][:, :3].astype(np.float64), b["aos"][:, 3].astype(np.float64)
        t_end = time.perf_counter() + seconds
        while time.perf_counter() < t_end:
            i = int(g.integers(0, len(mass)))
            t0 = time.perf_counter()
            opair.accel(pos, mass, synth.CFG_ALLPAIRS["eps"], [i])
            busy += time.perf_counter() - t0
            units += len(mass)
    else:
        raise ValueError(kind)
    return units, busy


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def oracle_rate(kind: str, seconds: float, workers: int, seed: int = 0):
    """Units per second of `workers` oracle processes running side by side for `seconds`
    (the sum of the workers' units over the longest worker's busy time)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    old = os.environ.get("OPENBLAS_NUM_THREADS")
    os.environ["OPENBLAS_NUM_THREADS"] = "1"        # one core per worker (inherited at spawn)
    try:
        with ctx.Pool(workers) as pool:
            res = pool.starmap(_oracle_units, [(kind, seconds, seed + 7919 * k) for k in range(workers)])
    finally:
        if old is None:
            os.environ.pop("OPENBLAS_NUM_THREADS", None)
        else:
            os.environ["OPENBLAS_NUM_THREADS"] = old
    units = sum(u for u, _ in res)
    busy = max(b for _, b in res)
    return units / busy, units, busy


UNITS = {"hmm": "state-steps/s", "segreduce": "GB/s", "allpairs": "interactions/s"}
SAMPLES = {"hmm": "random sequences of the K=64 plain and K=256 batched configurations (forward) and of the "
                  "K=256 adjoint configuration (forward-backward), float64 numpy",
           "segreduce": "the 4,096-sequence segmented sum of x*x+1 (oracle.patterns.segreduce_fast, int64)",
           "allpairs": "single bodies of the N=65,536 set against all N (oracle.pairwise.accel, float64)"}


def cpu_baseline(seconds_each: float):
    """The oracle per configuration unit at one core and at every allowed core."""
    cores = host_cores()
    out = {}
    for kind in ("hmm", "segreduce", "allpairs"):
        r1, _, b1 = oracle_rate(kind, seconds_each, 1, seed=11)
        rn, _, bn = oracle_rate(kind, seconds_each, cores, seed=13)
        scale = 1e-9 if kind == "segreduce" else 1.0
        out[kind] = {"unit": UNITS[kind], "one_core": r1 * scale, "all_cores": rn * scale, "cores": cores,
                     "sample": SAMPLES[kind] + f", {seconds_each:.0f} s per worker"}
    return out


def _relstats(rel):
    rel = np.asarray(rel, dtype=np.float64)
    return {"max": float(rel.max()), "p99": float(np.percentile(rel, 99)), "median": float(np.median(rel)),
            "n": int(rel.size)}


def errors_leg(W, out, api, torch, dev, seed: int = 0):
    """Every result's error against the float64 oracle, from the outputs of the last timed
    step (and, for the adjoint, one more untimed call on a subset of sequences): this leg runs
    the oracle, so it belongs to the CPU leg.  Samples are stated; the tests compare every
    element."""
    from oracle import hmm as ohmm
    from oracle import pairwise as opair
    from oracle import patterns as op
    g = synth.rng(seed)
    e = {}
    # seg-reduce (config 1): int64, bit-exact
    c = synth.CFG_SEGREDUCE
    data, lengths = synth.ragged_flat_int32(c["seed"], c["S"], c["len_lo"], c["len_hi"], c["val_lo"], c["val_hi"])
    off = np.zeros(c["S"] + 1, np.int64)
    np.cumsum(lengths, out=off[1:])
    ref = op.segreduce_fast(op.RED_ADD, op.MAP_SQ_PLUS_ONE, data, off, np.int64)
    seg, mx = out["seg"]
    got = seg.cpu().numpy()
    e["segreduce"] = {"mismatches": int(np.count_nonzero(got != ref)), "max_equal": int(mx.item()) == int(ref.max()),
                      "n": int(ref.size), "criterion": "bit-exact int64"}
    # HMM FP32 log-space forward (config 2): every sequence, oracle on the float32-rounded logs
    cp = synth.CFG_HMM_PLAIN
    p = synth.hmm_workload(cp["seed"], cp["K"], cp["M"], cp["S"], cp["kind"], cp["lo"], cp["hi"])
    ref = ohmm.loglik_scaled_batch(p, params=ohmm.params_from_f32_logs(synth.hmm_log_inputs_f32(p)))
    e["hmm_fp32_logL"] = dict(_relstats(np.abs(out["plain"].cpu().numpy() - ref) / np.abs(ref)),
                              tolerance=1e-5, reading="relative per sequence; oracle on the float32-rounded logs")
    # HMM BF16 batched forward (config 3): a sample (the 16 longest + 496 random sequences)
    # under three readings of the reference parameters
    cb = synth.CFG_HMM_BATCHED
    p = synth.hmm_workload(cb["seed"], cb["K"], cb["M"], cb["S"], cb["kind"], cb["lo"], cb["hi"])
    logs = synth.hmm_log_inputs_f32(p)
    sample = np.unique(np.concatenate([np.argsort(p["lengths"])[-16:], g.choice(cb["S"], 496, replace=False)]))
    ll = out["bf16"].cpu().numpy()[sample]
    bf = {}
    for tag, par in (("original_params", None), ("fp32_rounded_params", ohmm.params_from_f32_logs(logs)),
                     ("bf16_rounded_params", ohmm.params_bf16_from_f32_logs(logs))):
        r = ohmm.loglik_scaled_batch(p, seqs=sample, params=par)
        bf[tag] = _relstats(np.abs(ll - r) / np.abs(r))
    bf.update(tolerance=1e-3, sample=f"{sample.size} sequences: the 16 longest and random ones",
              reading="original: total error incl. rounding the parameters; bf16: the BF16 arithmetic alone")
    e["hmm_bf16_logL"] = bf
    # adjoint (config 4): the gradient of a subset's summed logL (0/1 weights), entry by entry
    # against the oracle's expected counts, and against central differences of the oracle
    if W.adj is not None:
        ca = synth.CFG_HMM_ADJOINT
        a = W.adj
        p = synth.hmm_workload(ca["seed"], ca["K"], ca["M"], ca["S"], ca["kind"], ca["lo"], ca["hi"])
        par = ohmm.params_from_f32_logs(synth.hmm_log_inputs_f32(p))
        sub = sorted(set(g.choice(ca["S"], 7, replace=False).tolist() + [int(np.argmax(p["lengths"]))]))
        w = np.zeros(ca["S"])
        w[sub] = 1.0
        gA, gB, gpi, _ = api.hmm_adjoint(a["log_A"], a["log_B"], a["log_pi"], a["obs"], a["offsets"],
                                         weights=torch.from_numpy(w).to(dev), max_T=a["maxT"], want_loglik=False)
        _, rA, rB, rpi = ohmm.gradients_batch(p, seqs=sub, params=par)
        adj = {}
        for name, gg, rr in (("log_A", gA, rA), ("log_B", gB, rB), ("log_pi", gpi, rpi)):
            gg = gg.cpu().numpy().astype(np.float64)
            rel = np.abs(gg - rr) / np.maximum(np.abs(rr), 1e-300)
            big = rr > 1e-6 * rr.sum(axis=-1, keepdims=True)     # entries above the row-total floor
            adj[name] = {"max_entry_rel": float(rel[big].max()), "median_entry_rel": float(np.median(rel[big])),
                         "rel_frobenius": float(np.linalg.norm(gg - rr) / np.linalg.norm(rr))}
        # central differences (h = 1e-6) of sum_s logL_s over the subset, float64 oracle
        h = 1e-6
        fd_err = []
        gA_np = gA.cpu().numpy()
        top = np.argsort(rA, axis=None)[-rA.size // 100:]          # among the largest 1% of entries
        for q in g.choice(top, 4, replace=False):
            i, j = (int(x) for x in np.unravel_index(int(q), rA.shape))
            lo, hi = dict(par), dict(par)
            lo["A"], hi["A"] = par["A"].copy(), par["A"].copy()
            hi["A"][i, j] *= np.exp(h)
            lo["A"][i, j] *= np.exp(-h)
            fd = (ohmm.loglik_scaled_batch(p, seqs=sub, params=hi).sum()
                  - ohmm.loglik_scaled_batch(p, seqs=sub, params=lo).sum()) / (2 * h)
            fd_err.append(abs(gA_np[i, j] - fd) / max(abs(fd), 1e-12))
        adj["fd_log_A_max_rel"] = float(max(fd_err))
        adj.update(sample=f"{len(sub)} sequences (0/1 weights), all entries; central differences of 4 of the "
                          "largest 1% entries of log A",
                   tolerance="|g - r| <= 1e-4 |r| + 1e-6 row total")
        e["hmm_adjoint_grad"] = adj
    # all-pairs (config 5): 256 random bodies
    ca = synth.CFG_ALLPAIRS
    b = synth.bodies(ca["seed"], ca["N"])
    pos, mass = b["aos"][:, :3].astype(np.float64), b["aos"][:, 3].astype(np.float64)
    idx = np.sort(g.choice(ca["N"], 256, replace=False))
    ref = opair.accel(pos, mass, ca["eps"], idx)
    ax, ay, az = out["allpairs"]
    got = torch.stack([ax, ay, az], 1).cpu().numpy().astype(np.float64)[idx]
    err = np.linalg.norm(got - ref, axis=1)
    scale = np.maximum(np.linalg.norm(ref, axis=1), opair.term_scale(pos, mass, ca["eps"], idx))
    e["allpairs_accel"] = dict(_relstats(err / np.linalg.norm(ref, axis=1)),
                               criterion_max=float((err / scale).max()), tolerance=1e-4,
                               sample="256 random bodies", reading="per-body relative; criterion_max = "
                               "max |a - a_ref| / max(|a_ref|, sum_j |term_ij| / sqrt(N))")
    return e


# ------------------------------------------------------------- single-kernel cases
def sweep_inputs(torch, dev, S):
    data, lengths = synth.ragged_flat_int32(1, S)
    off = np.zeros(S + 1, np.int64)
    np.cumsum(lengths, out=off[1:])
    return torch.from_numpy(data).to(dev), torch.from_numpy(off).to(dev)


def segreduce_sweep(torch, dev, api, S=1 << 20, reps=10, plain=False):
    """Fused map + segmented int64 sum at HBM scale (L2 flushed before each rep).  With
    plain=True the same result is computed in the plain (unfused) form: the map writes an
    int64 array, then an identity segmented sum reads it; GB/s is then still the fused
    form's algorithmic bytes over the plain form's time."""
    d, o = sweep_inputs(torch, dev, S)
    out = torch.empty(S, dtype=torch.int64, device=dev)
    ws = torch.empty(api.L.load().accel_segreduce_workspace_size(d.numel(), S), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    if plain:
        def run():
            mapped = api.accel_map(api.MAP_SQ_PLUS_ONE, d, torch.int64)
            return api.accel_segreduce(api.RED_ADD, api.MAP_IDENTITY, mapped, o, torch.int64, out=out, ws=ws)
    else:
        run = lambda: api.accel_segreduce(api.RED_ADD, api.MAP_SQ_PLUS_ONE, d, o, torch.int64, out=out, ws=ws)
    for _ in range(3):
        run()
    ts = []
    for _ in range(reps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        run()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    ms = statistics.median(ts)
    nbytes = 4 * d.numel() + 16 * S + 8
    return {"S": S, "N": int(d.numel()), "ms": ms, "GB/s": nbytes / (ms * 1e-3) / 1e9, "bytes": nbytes}


def marshal_sweep(torch, dev, api, S, reps=10):
    """accel_marshal_ragged at HBM scale: S int32 sequences with lengths U{0..256} stored as
    separate pieces in device memory (placed in a shuffled order, so the gather reads
    scattered addresses) -> flat data + int64 offsets; L2 flushed before each rep.  The
    call's pointer and length tables (page-locked host memory, copied in stream order) are
    part of the timed call.  Algorithmic bytes: 8 per element (read + write) + 24 per
    sequence (the two 8-byte table entries read, one offset written)."""
    import ctypes as C
    lib = api.L.load()
    lengths = synth.ragged_lengths(1, S)
    N = int(lengths.sum())
    g = synth.rng(5)
    perm = g.permutation(S)                      # piece order in the source buffer
    start = np.zeros(S, np.int64)
    start[perm] = np.concatenate([[0], np.cumsum(lengths[perm])[:-1]])
    src = torch.randint(-1000, 1001, (N,), dtype=torch.int32, device=dev)
    ptrs = torch.from_numpy(src.data_ptr() + 4 * start).pin_memory()
    lens = torch.from_numpy(lengths.astype(np.int64)).pin_memory()
    flat = torch.empty(N, dtype=torch.int32, device=dev)
    offsets = torch.empty(S + 1, dtype=torch.int64, device=dev)
    ws = torch.empty(lib.accel_marshal_ragged_workspace_size(S), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def run():
        st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        api.L.check("accel_marshal_ragged", lib.accel_marshal_ragged(
            C.c_void_p(ptrs.data_ptr()), C.c_void_p(lens.data_ptr()), S, api.L.I32, C.c_void_p(flat.data_ptr()),
            C.c_void_p(offsets.data_ptr()), C.c_void_p(ws.data_ptr()), ws.numel(), st))
    for _ in range(3):
        run()
    ts = []
    for _ in range(reps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        run()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    ms = statistics.median(ts)
    nbytes = 8 * N + 24 * S
    return {"S": S, "N": N, "ms": ms, "GB/s": nbytes / (ms * 1e-3) / 1e9, "bytes": nbytes}


PROFILE_CASES = ("segreduce_sweep", "marshal_sweep", "step", "hmm_plain", "hmm_bf16", "hmm_bf16_small", "hmm_adjoint",
                 "hmm_adjoint_small", "allpairs", "hmm_long", "hmm_long_small", "pairhist", "pairhist_small")


def profile_case(name, reps, torch, dev, tune_cache=None):
    """Runs one kernel case `reps` times (for ncu captures of a single kernel).  The BF16 forward
    runs in its tuned launch configuration: taken from `tune_cache` when that file has an entry
    for the case's sizes (no timing launches), else tuned first (and appended to it)."""
    from paper_2211_00621_gb300 import api
    if name == "segreduce_sweep":
        d, o = sweep_inputs(torch, dev, 1 << 20)
        fn = lambda: api.accel_segreduce(api.RED_ADD, api.MAP_SQ_PLUS_ONE, d, o, torch.int64)
    elif name == "marshal_sweep":
        # 2^18 sequences (N ~ 33.5M elements): the marshal sweep's middle size, run `reps` times
        marshal_sweep(torch, dev, api, 1 << 18, reps=reps)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": name, "reps": reps, "ok": True}))
        return 0
    elif name == "step":
        W = Workload(torch, dev, True)
        W.tune_and_capture(tune_cache)
        fn = lambda: W.step()
    elif name in ("hmm_plain", "hmm_bf16", "hmm_bf16_small", "hmm_adjoint", "hmm_adjoint_small"):
        cfg = {"hmm_plain": synth.CFG_HMM_PLAIN, "hmm_bf16": synth.CFG_HMM_BATCHED,
               "hmm_bf16_small": dict(synth.CFG_HMM_BATCHED, S=1024, hi=1000),
               "hmm_adjoint": synth.CFG_HMM_ADJOINT,
               "hmm_adjoint_small": dict(synth.CFG_HMM_ADJOINT, S=256, lo=100, hi=400)}[name]
        h = hmm_inputs(cfg, torch, dev)
        if name.startswith("hmm_adjoint"):
            fn = lambda: api.hmm_adjoint(h["log_A"], h["log_B"], h["log_pi"], h["obs"], h["offsets"],
                                         max_T=h["maxT"], want_loglik=False)
        else:
            prec = api.HMM_FP32_LOG if name == "hmm_plain" else api.HMM_BF16_SCALED
            if prec == api.HMM_BF16_SCALED:
                api.hmm_autotune(h["log_A"], h["log_B"], h["log_pi"], h["obs"], h["offsets"], cache_path=tune_cache)
            fn = lambda: api.hmm_forward(h["log_A"], h["log_B"], h["log_pi"], h["obs"], h["offsets"], prec)
    elif name in ("hmm_long", "hmm_long_small"):
        cfg = synth.CFG_HMM_LONG if name == "hmm_long" else dict(synth.CFG_HMM_LONG, lo=20000, hi=20000)
        h = hmm_inputs(cfg, torch, dev)
        fn = lambda: api.hmm_forward_long(h["log_A"], h["log_B"], h["log_pi"], h["obs"], h["offsets"],
                                          max_T=h["maxT"])
    elif name in ("pairhist", "pairhist_small"):
        ch = synth.CFG_PAIRHIST
        n = ch["N"] if name == "pairhist" else 8192
        pts = torch.from_numpy(synth.sphere_points(ch["seed"], n)).to(dev)
        edges = synth.angle_edges(ch["nbins"], ch["amin"], ch["amax"])
        fn = lambda: api.accel_pair_histogram(pts, edges)
    elif name == "allpairs":
        b = synth.bodies(0, synth.CFG_ALLPAIRS["N"])
        aos = torch.from_numpy(b["aos"]).to(dev)
        f32 = torch.float32
        x, y, z, m = api.accel_marshal_records(aos, [(0, f32), (4, f32), (8, f32), (12, f32)])
        fn = lambda: api.pairwise_mapreduce(x, y, z, m, synth.CFG_ALLPAIRS["eps"])
    else:
        raise ValueError(name)
    for _ in range(reps):
        fn()
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": name, "reps": reps, "ok": True}))
    return 0


# ---------------------------------------------------------------------------- main
def aggregate_ranks(ms_local: float, work_per_rank: float, world: int, allreduce_max=None):
    """Whole-job timing of replicas: the slowest rank's step time bounds the job, and every
    rank processes `work_per_rank` units per step (weak scaling, no data exchange).
    Returns (ms, units per second for the whole job)."""
    ms = ms_local if world <= 1 else float(allreduce_max(ms_local))
    return ms, work_per_rank * world / (ms * 1e-3)


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    # the reference arm is the oracle, timed as it stands on the host cores (one worker per
    # allowed core), in the line's own unit: HMM state-steps per second
    cores = host_cores()
    for _ in range(args.warmup):
        oracle_rate("hmm", min(args.ref_step_seconds, 1.0), cores, seed=1000)
    units, secs = 0, 0.0
    for k in range(args.steps):
        _, u, b = oracle_rate("hmm", args.ref_step_seconds, cores, seed=k)
        units += u
        secs += b
    value = units / secs
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "HMM rows of the hot path (K=64 plain, K=256 batched, K=256 adjoint), bounded "
                                   "random sample of sequences per step, one oracle process per host core"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": SAMPLES["hmm"] + f"; {args.ref_step_seconds:.0f} s per step per worker, "
                                                        f"{args.steps} steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-step-seconds", type=float, default=4.0)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--profile-case", choices=PROFILE_CASES, default=None,
                    help="run one kernel case --reps times and exit (for ncu captures)")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--tune-cache", default=None,
                    help="JSON-lines file of BF16 launch configurations (read, and appended to when tuning)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    from paper_2211_00621_gb300 import _lib, api
    from paper_2211_00621_gb300 import build as _build

    if not torch.cuda.is_available():
        print(json.dumps({"metric": METRIC, "error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    if not _build.up_to_date():
        if rank == 0:
            _build.build()
        if world > 1:
            dist.barrier()
    lib = _lib.load()
    if args.profile_case:
        return profile_case(args.profile_case, args.reps, torch, dev, args.tune_cache)

    with_adj = not args.no_adjoint
    if with_adj:
        try:
            W0 = hmm_inputs(dict(seed=0, K=8, M=4, S=2, kind="fixed", lo=3, hi=3), torch, dev)
            api.hmm_adjoint(W0["log_A"], W0["log_B"], W0["log_pi"], W0["obs"], W0["offsets"])
        except _lib.AccelError:
            with_adj = False
    W = Workload(torch, dev, with_adj)
    W.tune_and_capture(args.tune_cache)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(max(args.warmup, 3) if args.warmup >= 3 else args.warmup):
        W.step()
    barrier()

    # ---------------- timed region: K steps, L2 flushed (untimed) before each
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ev = {}
    step_ms = []
    launches0 = lib.accel_launch_count()
    barrier()
    last = None
    for _ in range(args.steps):
        flush.zero_()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record()
        last = W.step()
        e.record()
        e.synchronize()
        step_ms.append(s.elapsed_time(e))
    barrier()
    launches = lib.accel_launch_count() - launches0
    if W.bf16_graph is not None:
        launches += 5 * args.steps      # kernels inside each replay of the captured BF16 call
    if W.seg_graph is not None:
        launches += W.seg_kernels * args.steps    # ... and of the captured seg-reduce row
    clk = clocks.stop()
    def allreduce_max(x):
        t = torch.tensor([x], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    # per-row times: the same step with its rows one after another (untimed by the step)
    for _ in range(3):
        flush.zero_()
        W.step(ev)
    torch.cuda.synchronize()
    row_ms = {k: statistics.median(a.elapsed_time(b) for a, b in v) for k, v in ev.items()}
    work = W.state_steps()
    ms, value = aggregate_ranks(sum(step_ms) / len(step_ms), work, world, allreduce_max)

    # ---------------- end to end through the public API with host buffers
    host, h2d = W.host_inputs()
    for _ in range(2):
        W.e2e_step(host)
    barrier()
    e2e_ms = []
    d2h = 0
    for _ in range(max(2, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d2h = W.e2e_step(host)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e, e2e_value = aggregate_ranks(statistics.median(e2e_ms), work, world, allreduce_max)

    # ---------------- seg-reduce and marshal at HBM scale (2^16, 2^18, 2^20 segments; the
    # seg-reduce's plain form at 2^20)
    sweeps = [segreduce_sweep(torch, dev, api, S=1 << e) for e in (16, 18, 20)]
    sweep = sweeps[-1]
    plain_form = segreduce_sweep(torch, dev, api, S=1 << 20, plain=True)
    msweeps = [marshal_sweep(torch, dev, api, S=1 << e) for e in (16, 18, 20)]

    # ---------------- measured ALU rates (the denominators of the "alu" rooflines)
    alu = measure_alu(api)

    # ---------------- reported comparisons (untimed by the step): BF16 vs FP32 forward on the
    # batched input, adjoint vs forward-only on the adjoint input, adjoint memory
    def timed_once(fn, reps=2):
        fn()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            best = min(best, a.elapsed_time(b))
        return best

    q = W.bf16
    fp32_on_bf16 = timed_once(lambda: api.hmm_forward(q["log_A"], q["log_B"], q["log_pi"], q["obs"], q["offsets"],
                                                      api.HMM_FP32_LOG), reps=1)
    compare = {"bf16_vs_fp32_forward_K256": {"fp32_ms": fp32_on_bf16, "bf16_ms": row_ms["hmm_bf16"],
                                             "speedup": fp32_on_bf16 / row_ms["hmm_bf16"]}}
    if W.adj is not None:
        import ctypes as C
        a = W.adj
        fwd_only = timed_once(lambda: api.hmm_forward(a["log_A"], a["log_B"], a["log_pi"], a["obs"], a["offsets"],
                                                      api.HMM_FP32_LOG))
        m = api._model(a["log_A"], a["log_B"], a["log_pi"])
        ws_bytes = lib.hmm_adjoint_workspace_size(C.byref(m), a["S"], a["obs"].numel(), a["maxT"])
        compare["adjoint_vs_forward_only"] = {"adjoint_ms": row_ms["hmm_adjoint"], "fp32_forward_ms": fwd_only,
                                              "ratio": row_ms["hmm_adjoint"] / fwd_only,
                                              "workspace_bytes": int(ws_bytes),
                                              "all_alphas_bytes": int(a["sumT"]) * a["K"] * 4}
    # parallel-in-T forward on few, very long sequences, against the sequential FP32 forward
    lg = hmm_inputs(synth.CFG_HMM_LONG, torch, dev)
    long_ms = timed_once(lambda: api.hmm_forward_long(lg["log_A"], lg["log_B"], lg["log_pi"], lg["obs"], lg["offsets"],
                                                      max_T=lg["maxT"]))
    seq_ms = timed_once(lambda: api.hmm_forward(lg["log_A"], lg["log_B"], lg["log_pi"], lg["obs"], lg["offsets"],
                                                api.HMM_FP32_LOG), reps=1)
    compare["hmm_long_parallel_in_T"] = {
        "workload": "K=64 M=32, 4 sequences x 250,000 steps", "ms": long_ms, "sequential_fp32_ms": seq_ms,
        "speedup": seq_ms / long_ms, "state_steps_per_s": lg["K"] * lg["sumT"] / (long_ms * 1e-3),
        # work of the method: one 64 x 64 x 64 product per step (2 K^3 flop)
        "TFLOP/s": 2 * lg["K"] ** 3 * lg["sumT"] / (long_ms * 1e-3) / 1e12}
    # all-pairs angular histogram (tpacf shape) on synthetic sphere points
    ch = synth.CFG_PAIRHIST
    pts = torch.from_numpy(synth.sphere_points(ch["seed"], ch["N"])).to(dev)
    edges = synth.angle_edges(ch["nbins"], ch["amin"], ch["amax"])
    hist_ms = timed_once(lambda: api.accel_pair_histogram(pts, edges))
    npairs = ch["N"] * (ch["N"] - 1) // 2
    compare["pair_histogram_tpacf"] = {"workload": f"N={ch['N']} points, {ch['nbins']} log-spaced bins "
                                                   f"({ch['amin']:g}-{ch['amax']:g} arcmin), self pairs",
                                       "ms": hist_ms, "pairs_per_s": npairs / (hist_ms * 1e-3)}
    compare["allpairs_interactions_per_s"] = W.N * W.N / (row_ms["allpairs"] * 1e-3)
    compare["segreduce_plain_form"] = {"ms": plain_form["ms"], "GB/s_equiv": plain_form["GB/s"],
                                       "fused_speedup": plain_form["ms"] / sweep["ms"]}

    # ---------------- rooflines
    peaks, peak_src = load_peaks()
    for sw in sweeps + msweeps:
        sw["frac"] = sw["GB/s"] / peaks["hbm_gbs"]
    rl = rooflines(W, row_ms, peaks, alu["fp32_tflops"])
    dom = max((k for k in rl), key=lambda k: row_ms.get(k, 0.0))
    roof = dict(rl[dom])
    roof["kernel"] = dom
    roof["traffic"] = traffic_for(dom)
    roof["peak_source"] = {"tensor": f"{peak_src} sustained bf16 (MEASURED_PEAKS.json)",
                           "hbm": f"{peak_src} HBM copy (MEASURED_PEAKS.json)",
                           "alu": "measured in this run: FP32 FMA rate (accel_alu_rate, best of FFMA and packed "
                                  "FFMA2)"}[roof["bound"]]

    rows = {k: {kk: v for kk, v in rl[k].items() if kk != "peak"} | {"ms": row_ms[k]} for k in rl}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16+fp32 (HMM), int64 (seg-reduce), fp32 (all-pairs)",
            "data": "synthetic",
            "config": {"workload": "all hot-path rows once per step: seg-reduce 4096 seqs; HMM plain K=64 S=512 T=1000;"
                                   " HMM batched BF16 K=256 S=4096 T log-U[50,5000]; HMM adjoint K=256 S=1024 "
                                   "T U[200,2000]" + ("" if with_adj else " (adjoint not built: skipped)") +
                                   "; all-pairs N=65536",
                       "l2": "flushed before every timed step (256 MiB write, untimed)",
                       "schedule": "three streams: the batched BF16 forward (a CUDA graph of its 5 kernels, "
                                   "its tuned persistent units) beside the adjoint's forward phase within the "
                                   "SMs it leaves less a tenth of the device (accel_set_sm_budget) and the "
                                   "seg-reduce, plain FP32 and all-pairs rows on the main stream; then, "
                                   "after those rows and the forward phase, the adjoint's backward phase "
                                   "(three streams of its own) and the re-estimation; the BF16 stream joins "
                                   "at the end; per-row times in `rows` come from the same step run row "
                                   "after row",
                       "parallelism": f"replicas x{world} (sequences shard with no exchange)"},
            "seg_reduce_gbs": sweep["GB/s"], "seg_reduce_sweep": sweeps, "marshal_sweep": msweeps,
            "compare": compare, "rows": rows, "roofline": roof,
            "alu_measured": {"ffma_tflops": alu["ffma"] / 1e12, "ffma2_tflops": alu["ffma2"] / 1e12,
                             "rsqrt_gops": alu["rsqrt"] / 1e9, "dfma_tflops": alu["dfma"] / 1e12,
                             "how": "accel_alu_rate: 4 CTAs x 512 threads per SM, 8 independent dependent "
                                    "chains per thread, CUDA events, running clocks, best of 3"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e},
            "gpu_launches": int(launches), "clocks": clk,
            "autotune": W.tuned}

    if rank == 0 and world == 1 and args.cpu_seconds > 0:
        # the CPU leg: the oracle timed on the host cores, and the errors against it
        per = cpu_baseline(args.cpu_seconds / 6)
        h = per["hmm"]
        line["cpu_baseline"] = {"value": h["all_cores"], "unit": UNIT, "cores": h["cores"], "kind": "oracle",
                                "one_core": h["one_core"], "sample": h["sample"], "per_config": per}
        line["errors"] = errors_leg(W, last, api, torch, dev)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
