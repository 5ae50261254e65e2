#!/usr/bin/env python3
"""Benchmark of the ConKer hot path on one GB300 per rank.

One step = one catalog end to end on the device: grid the randoms and the
data (mapping), FFT-convolve both fields with every shell kernel, the n-point
product sums for num and den, and xi (ck_set_randoms + ck_compute).  Inputs
are resident in HBM before timing; the timed region is exactly --steps steps
bracketed by a barrier and a device synchronisation, timed with CUDA events
on the launching stream; the max over ranks is taken.  Every step moves
far more than the 129 MB L2 (the 512^3 W bank alone is 8.6 GB per field), so
no explicit L2 flush is added between steps.

Also reported: `e2e` (the same step through the C ABI with host input
buffers and host outputs, copies inside the timed region), `roofline` for
the dominant kernel from the library's per-launch CUDA events, the FP64 CPU
oracle on a bounded sample (`cpu_baseline`), SM clocks sampled during the
timed region, and the number of library kernel launches.

`--impl reference` times the FP64 CPU oracle on the host cores (there is no
reference implementation to install: the paper's code is not part of it).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("ms/catalog for ξ_2..ξ_5 (mixed vs plain FP32, rel err ≤1e-5); FFT GB/s; TC util %")
FALLBACK_HBM_GBS = 6800.0


def _sources_sha(source):
    """First 16 hex digits of the SHA-256 of the named csrc files, concatenated in order."""
    names = [source] if isinstance(source, str) else list(source)
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2108_00015_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="survey512")
    ap.add_argument("--orders", default=None, help="e.g. 23 or 2345 (default: the workload's)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="split_tf32", choices=["split_tf32", "split_bf16", "split_fp16", "fp32"],
                    help="headline form: mixed split-TF32 tensor-core sums (fused pass), split-BF16 or "
                         "split-FP16 tensor-core sums (kind::f16, bank kept), or plain FP32")
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain FP32 form beside the headline")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes (ck_plan_autotune times the choices after warm-up)")
    ap.add_argument("--tuning", default=None,
                    help="fixed launch shapes instead of the autotuner: fwd_cols,zreg_cols,yinv_cols,ctas_per_sm"
                         "[,stack_cols[,thin_overlap[,z_direct]]] (8 or 16 columns per tile of the strided passes, 1..3 "
                         "contraction CTAs per SM, the widest stacked contraction tile, thin tiles on a second stream, "
                         "the z step by the shells' short filters)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the higher-order workloads timed beside the headline at N = 1 (stress256: xi_2..xi_5, "
                         "survey512_s32: xi_2..xi_4, in every contraction form)")
    ap.add_argument("--diagonal", action="store_true",
                    help="time ck_set_randoms_diagonal + ck_compute_diagonal (Eq. 14, the (s, .., s) entries "
                         "only) instead of ck_set_randoms + ck_compute; "
                         "no e2e, plain-form or CPU legs")
    ap.add_argument("--factorised", action="store_true",
                    help="build the randoms field with ck_set_randoms_factorised (Eq. 7) from a CMASS-like "
                         "selection (P_ang uniform on dec >= 30 deg, P_z uniform on 0.43 <= z < 0.70, the "
                         "survey mask's footprint) instead of gridding the random catalog; "
                         "no e2e or plain-form legs")
    ap.add_argument("--continuous", action="store_true",
                    help="time ck_compute_continuous (Eqs. 15-17) on line-intensity-like maps D, R of the "
                         "workload's grid (built at 1/4 resolution and repeated; device-resident) instead of "
                         "catalogs; no e2e or plain-form legs")
    return ap.parse_args()


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


# dense TF32 / BF16 tensor rate, NVIDIA's nominal figures (1.1 and 2.25 PFLOP/s)
TF32_PER_BF16 = 1.1 / 2.25
FALLBACK_BF16_SUSTAINED_TFLOPS = 1700.0


def _tensor_peak(precision):
    """Sustained dense tensor peak of the contraction's operand kind: the
    measured sustained BF16 GEMM rate (BF16 and FP16 operands run at the same
    dense rate), times the nominal TF32/BF16 ratio for TF32 operands (the
    contraction is timed inside a long step)."""
    ratio = TF32_PER_BF16 if precision == "split_tf32" else 1.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops_sustained"]) * ratio, "measured"
    except Exception:
        return FALLBACK_BF16_SUSTAINED_TFLOPS * ratio, "fallback"


def _tc_work(ns, orders):
    """Per cell, the multiply-adds of the blocked product the tensor-core
    contraction computes (live operand rows x the columns each 128-row tile
    needs, the library's tile rule; thin tiles of at most 16 columns and 256
    outputs run on the CUDA cores and are left out) and the useful ones (one
    per output multiset)."""
    rows, cols = [], []
    if 2 in orders:
        rows.append((-1, -1))
    if 3 in orders:
        rows += [(a, -1) for a in range(ns)]
    if 4 in orders or 5 in orders:
        rows += [(a, b) for b in range(ns) for a in range(b + 1)]
    if 2 in orders or 3 in orders or 4 in orders:
        cols += [(k, -1) for k in range(ns)]
    if 5 in orders:
        cols += [(k, l) for k in range(ns) for l in range(k, ns)]

    def canon(r, c):
        da, db = (r[0] >= 0) + (r[1] >= 0), (c[0] >= 0) + (c[1] >= 0)
        n = 0
        if da == 0 and db == 1:
            n = 2
        elif da == 1 and db == 1 and r[0] <= c[0]:
            n = 3
        elif da == 2 and db == 1 and r[1] <= c[0]:
            n = 4
        elif da == 2 and db == 2 and r[1] <= c[0]:
            n = 5
        return n in orders

    dense = 0
    for m0 in range(0, len(rows), 128):
        tile = rows[m0:m0 + 128]
        need = sum(1 for c in cols if any(canon(r, c) for r in tile))
        smem = (2 * (ns + 2) + len(tile) + 16) * 260 * 4 + (len(tile) + 16) * 8
        if need <= 16 and len(tile) * need <= 256 and smem <= 227 * 1024:
            continue  # a thin tile: the CUDA cores sum it
        dense += len(tile) * need
    useful = sum(math.comb(ns + n - 2, n - 1) for n in orders)
    return dense, useful


class Clocks:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", delete=False, suffix=".csv")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        self.f.close()
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for name, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(name)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def _smi_index(torch, local):
    """nvidia-smi's name for this rank's GPU (UUID when torch reports it)."""
    try:
        u = str(torch.cuda.get_device_properties(local).uuid)
        if u and u != "None":
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        return vis.split(",")[local]
    return str(local)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _orders(args, w):
    if args.orders:
        return tuple(int(c) for c in args.orders)
    return tuple(w["orders"])


# ---------------------------------------------------------------------------
# CPU oracle legs

def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def cpu_engine_catalog(w, orders):
    """One whole catalog through the oracle's FP64 C++/OpenMP engine on all
    host cores (gridding, forward FFT, every shell's convolution, the sums
    of every requested order): wall-clock ms, and the description."""
    from oracle import cpu_engine
    t0 = time.perf_counter()
    cpu_engine.correlate(w["grid"], w["shells"], w["width"], w["data"], w["randoms"], orders=orders, engine="fft")
    ms = (time.perf_counter() - t0) * 1000.0
    n = cpu_engine.threads()
    return ms, n, (f"the whole catalog ({w['data'].n} + {w['randoms'].n} points, {len(w['shells'])} shells, orders "
                   f"{list(orders)}) through the oracle's FP64 C++/OpenMP engine (FFT convolution) on {n} threads, "
                   f"{os.cpu_count()} host cores ({cpu_model()}); no scaling")


def cpu_oracle_sample(w, orders, point_frac=1 / 8, fields=2):
    """Time the FP64 oracle on a bounded sample of the workload and scale each
    stage to one catalog: gridding of `point_frac` of the points (x 1/frac),
    the density fields once, one shell's FFT convolution of one field
    (x N_s x fields), and the product sums of one multiset per order
    (x the number of multisets x fields)."""
    import numpy as np
    from oracle import conker_oracle as O

    g = w["grid"]
    d, r = w["data"], w["randoms"]
    nd, nr = max(1, int(d.n * point_frac)), max(1, int(r.n * point_frac))
    t0 = time.perf_counter()
    D, _ = O.grid_counts(d.x[:nd], d.y[:nd], d.z[:nd], g)
    R, _ = O.grid_counts(r.x[:nr], r.y[:nr], r.z[:nr], g)
    t_grid = (time.perf_counter() - t0) / point_frac
    t0 = time.perf_counter()
    alpha, N, Rt = O.density_fields(D, R)
    t_prep = time.perf_counter() - t0
    offs = O.shell_offsets(w["shells"][len(w["shells"]) // 2], w["width"], g.cell)
    t0 = time.perf_counter()
    W = O.convolve_fft(N, offs)
    t_conv = time.perf_counter() - t0
    ns = len(w["shells"])
    t_sum = 0.0
    for n in orders:
        t0 = time.perf_counter()
        O.product_sums(N, [W], n)  # exactly one multiset
        t_sum += (time.perf_counter() - t0) * math.comb(ns + n - 2, n - 1)
    total = t_grid + t_prep + fields * (t_conv * ns + t_sum)
    sample = (f"oracle (numpy FP64, single thread) on {nd + nr} of {d.n + r.n} points, one shell's FFT "
              f"convolution of one field and one multiset per order; stages scaled to the catalog "
              f"(gridding x{1 / point_frac:.0f}, convolution x{fields * ns}, sums x multisets x{fields})")
    return total * 1000.0, sample


def cpu_oracle_mode_sample(w, orders, mode, maps=None, selection=None, cells=2000):
    """The oracle for the --factorised and --continuous steps, on bounded
    samples scaled to one step:
    * factorised: Eq. 7 at `cells` sampled cells (x N_c / cells), the data
      catalog's gridding (1/8 of its points, x 8), and both fields'
      convolution and sums as in cpu_oracle_sample;
    * continuous: Eq. 15 on the whole maps, and one field's convolution and
      sums."""
    import numpy as np
    from oracle import conker_oracle as O

    g = w["grid"]
    nc = int(np.prod(g.n))
    ns = len(w["shells"])
    t0 = time.perf_counter()
    if mode == "factorised":
        rng = np.random.default_rng(5)
        pick = np.stack([rng.integers(0, n, cells) for n in g.n], axis=1)
        O.factorised_randoms_at(pick, g, **selection)
        t_field = (time.perf_counter() - t0) * nc / cells
        d = w["data"]
        nd = max(1, d.n // 8)
        t0 = time.perf_counter()
        D, _ = O.grid_counts(d.x[:nd], d.y[:nd], d.z[:nd], g)
        t_field += (time.perf_counter() - t0) * 8
        F = D.astype(np.float64)
        fields = 2
        what = (f"oracle (numpy FP64, single thread): Eq. 7 at {cells} sampled cells (x{nc // cells}), "
                f"gridding of 1/8 of the data (x8)")
    else:
        F = O.delta_field(maps[0], maps[1])
        t_field = time.perf_counter() - t0
        fields = 1
        what = "oracle (numpy FP64, single thread): Eq. 15 on the whole maps"
    offs = O.shell_offsets(w["shells"][ns // 2], w["width"], g.cell)
    t0 = time.perf_counter()
    W = O.convolve_fft(F, offs)
    t_conv = time.perf_counter() - t0
    t_sum = 0.0
    for n in orders:
        t0 = time.perf_counter()
        O.product_sums(F, [W], n)
        t_sum += (time.perf_counter() - t0) * math.comb(ns + n - 2, n - 1)
    total = t_field + fields * (t_conv * ns + t_sum)
    sample = what + (f", one shell's FFT convolution of one field and one multiset per order, scaled "
                     f"(convolution x{fields * ns}, sums x multisets x{fields})")
    return total * 1000.0, sample


# ---------------------------------------------------------------------------

def _summed_cells(w):
    """Cells the bank contractions visit: the planes between the lowest and
    the highest occupied z cell of the data and the randoms (the library
    sums only those planes; W_0 vanishes elsewhere)."""
    import numpy as np
    g = w["grid"]
    zs = []
    for c in (w["data"], w["randoms"]):
        k = np.floor((c.z.astype(np.float64) - g.origin[2]) / g.cell).astype(np.int64)
        k = np.mod(k, g.n[2]) if g.periodic else k[(k >= 0) & (k < g.n[2])]
        if k.size:
            zs += [int(k.min()), int(k.max())]
    planes = max(zs) - min(zs) + 1 if zs else 0
    return planes * g.n[0] * g.n[1]


def _time_extra(torch, w, orders, precision, steps, warmup):
    """One higher-order workload in one form: ck_set_randoms + ck_compute
    per step on device-resident catalogs, CUDA events around `steps` steps
    after `warmup`, the library's per-launch times for the roofline of the
    tensor-core contraction (or of the dominant stage), clocks sampled
    meanwhile."""
    import numpy as np
    from paper_2108_00015_gb300 import Plan
    g = w["grid"]
    ns = len(w["shells"])
    plan = Plan(g.n, g.origin, g.cell, g.periodic, w["shells"], w["width"], max_order=max(orders),
                precision=precision)
    d, r = w["data"], w["randoms"]
    dev = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
    dx, dy, dz, rx, ry, rz = (dev(a) for a in (d.x, d.y, d.z, r.x, r.y, r.z))
    outs = {k: {n: torch.empty((ns,) * (n - 1), dtype=torch.float64, device="cuda") for n in orders}
            for k in ("xi", "num", "den")}
    outs["dropped"] = torch.zeros(2, dtype=torch.int64, device="cuda")

    def step():
        plan.set_randoms(rx, ry, rz)
        return plan.compute(dx, dy, dz, orders=orders, out="device", outputs=outs)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    tuning = plan.autotune()
    step()
    torch.cuda.synchronize()
    if plan.status() != 0:
        raise RuntimeError(f"device status after warm-up ({precision})")
    stream = torch.cuda.current_stream()
    plan.profile(True)
    clocks = Clocks(_smi_index(torch, torch.cuda.current_device()))
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    t_ms = e0.elapsed_time(e1)
    stages = plan.profile_read()
    plan.profile(False)
    if plan.status() != 0:
        raise RuntimeError(f"device status in the timed region ({precision})")
    plan.close()
    out = {"ms_per_catalog": round(t_ms / steps, 3), "steps": steps, "clocks": clk, "tuning": tuning}
    dname, dv = max(stages.items(), key=lambda kv: kv[1]["ms"])
    t_launch = dv["ms"] / dv["launches"] * 1e-3
    out["dominant"] = {"stage": dname, "ms_per_step": round(dv["ms"] / steps, 3)}
    if "contract" in stages and precision.startswith("split_"):
        cv = stages["contract"]
        tc = cv["ms"] / cv["launches"] * 1e-3
        dense, useful = _tc_work(ns, orders)
        nc = _summed_cells(w)
        flops = 3 * 2 * dense * nc
        tpk, tkind = _tensor_peak(precision)
        out["roofline"] = {"bound": "tensor", "kernel": "contract", "achieved": round(flops / tc / 1e12, 1),
                           "cells_summed": nc,
                           "peak": round(tpk, 1), "unit": "TFLOP/s", "frac": round(flops / tc / 1e12 / tpk, 4),
                           "algorithmic_flops_per_launch": flops, "ms_per_launch": round(tc * 1e3, 3),
                           "useful_tflops": round(2 * useful * nc / tc / 1e12, 1),
                           "peak_source": f"{tkind} MEASURED_PEAKS.json bf16_tflops_sustained"
                                          + (f" x {TF32_PER_BF16:.3f} (nominal TF32/BF16)" if precision == "split_tf32"
                                             else " (dense BF16/FP16 rate)")}
    else:
        peak, _ = _peaks()
        gbs = dv["bytes"] / (dv["ms"] * 1e-3) / 1e9
        out["roofline"] = {"bound": "hbm", "kernel": dname, "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                           "frac": round(gbs / peak, 4)}
    return out


def run_extras(torch, steps, warmup):
    """The metric's higher orders beside the headline: xi_2..xi_5 on the
    256^3 stress catalog (20M + 40M points, 16 shells) and xi_2..xi_4 on the
    512^3 survey catalog with 32 shells, each in the mixed forms (split-TF32,
    split-BF16, split-FP16 tensor-core sums) and the plain FP32 form."""
    from synth import workload
    res = {}
    for name, orders, forms, plain_steps in (("stress256", (2, 3, 4, 5), ("split_tf32", "split_bf16", "split_fp16"), 3),
                                             ("survey512_s32", (2, 3, 4), ("split_tf32", "split_bf16", "split_fp16"), 1)):
        w = workload(name)
        ent = {"grid": list(w["grid"].n), "shells": len(w["shells"]), "orders": list(orders),
               "n_data": w["data"].n, "n_randoms": w["randoms"].n, "forms": {}}
        for prec in forms:
            ent["forms"][prec] = _time_extra(torch, w, orders, prec, steps, warmup)
        ent["forms"]["fp32"] = _time_extra(torch, w, orders, "fp32", plain_steps, 1)
        best = min(ent["forms"][p]["ms_per_catalog"] for p in forms)
        ent["mixed_speedup_over_plain"] = round(ent["forms"]["fp32"]["ms_per_catalog"] / best, 2)
        res[name] = ent
        del w
    return res


def run_gb300(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2108_00015_gb300 import Plan
    from synth import workload

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = workload(args.workload)
    orders = _orders(args, w)
    g = w["grid"]
    precision = args.precision
    plan = Plan(g.n, g.origin, g.cell, g.periodic, w["shells"], w["width"], max_order=max(orders),
                precision=precision)
    d, r = w["data"], w["randoms"]
    dev = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
    dx, dy, dz = dev(d.x), dev(d.y), dev(d.z)
    rx, ry, rz = dev(r.x), dev(r.y), dev(r.z)
    ns = len(w["shells"])
    outs = {k: {n: torch.empty((ns,) * (n - 1), dtype=torch.float64, device="cuda") for n in orders}
            for k in ("xi", "num", "den")}
    outs["dropped"] = torch.zeros(2, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()

    # the factorised selection: one-degree sky cells, 27 redshift bins
    sel_pa = np.zeros((180, 360))
    sel_pa[120:, :] = 1.0 / (2.0 * math.pi * (1.0 - math.sin(math.radians(30.0))))  # per sr over dec >= 30
    sel_pz = np.full(27, 1.0 / 0.27)

    if args.continuous:
        from synth import continuous_maps
        cs = tuple(max(1, v // 4) for v in (g.n[2], g.n[1], g.n[0]))
        D4, R4 = continuous_maps(12, cs, g.cell * 4)
        rep = lambda a: np.ascontiguousarray(a.repeat(4, 0).repeat(4, 1).repeat(4, 2)[:g.n[2], :g.n[1], :g.n[0]])  # noqa
        map_d, map_r = dev(rep(D4)), dev(rep(R4))

    def step():
        if args.continuous:
            return plan.compute_continuous(map_d, map_r, orders=orders, out="device")
        if args.factorised:
            plan.set_randoms_factorised(float(d.n), sel_pa, sel_pz, 0.43, 0.70, z_max=0.75)
            return plan.compute(dx, dy, dz, orders=orders, out="device", outputs=outs)
        if args.diagonal:
            plan.set_randoms_diagonal(rx, ry, rz)
            return plan.compute_diagonal(dx, dy, dz, orders=orders, out="device")
        plan.set_randoms(rx, ry, rz)
        return plan.compute(dx, dy, dz, orders=orders, out="device", outputs=outs)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    tuning = None
    if args.tuning:
        plan.set_tuning(*[int(v) for v in args.tuning.split(",")])
        tuning = plan.tuning()
        step()
        torch.cuda.synchronize()
    elif not args.no_autotune and not (args.continuous or args.diagonal):
        # launch-shape choices timed on the resident randoms (results unchanged)
        tuning = plan.autotune()
        step()
        torch.cuda.synchronize()
    st = plan.status()
    if st not in (0,):
        raise RuntimeError(f"device status {st} after warm-up")
    plan.profile(True)
    clocks = Clocks(_smi_index(torch, local))
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    t_ms = e0.elapsed_time(e1)
    if ws > 1:
        t = torch.tensor([t_ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
    stages = plan.profile_read()
    plan.profile(False)
    st = plan.status()
    if st != 0:
        raise RuntimeError(f"device status {st} in the timed region")

    peak, peak_kind = _peaks()
    launches = sum(v["launches"] for v in stages.values())
    stage_out = {}
    for name, v in stages.items():
        per = v["ms"] / v["launches"]
        gbs = v["bytes"] / (v["ms"] * 1e-3) / 1e9 if v["ms"] > 0 else None
        stage_out[name] = {"ms_per_step": round(v["ms"] / args.steps, 4), "launches_per_step": v["launches"] / args.steps,
                           "us_per_launch": round(per * 1e3, 2),
                           "achieved_gbs": round(gbs, 1) if gbs else None}
    dom = max(stages.items(), key=lambda kv: kv[1]["ms"])
    dname, dv = dom
    achieved = dv["bytes"] / (dv["ms"] * 1e-3) / 1e9
    traffic = None
    tr_path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr_path):
        try:
            tr = json.load(open(tr_path))
            ent = tr.get(args.workload, {}).get(dname)
            # counters of the same sources (the kernel's file and the headers
            # it includes, hashed in order) and, where recorded, the same tile width
            cols = {"fft_z_inv_mul": "zreg_cols", "fft_y_inv": "yinv_cols"}.get(dname)
            same_shape = ent is not None and ("cols" not in ent or (tuning or plan.tuning()).get(cols) == ent["cols"])
            if ent and same_shape and _sources_sha(ent["source"]) == ent["sha"]:
                traffic = ent["bytes_per_launch"]
        except Exception:
            traffic = None
    roofline = {"bound": "hbm", "kernel": dname, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "algorithmic_bytes_per_launch": dv["bytes"] / dv["launches"],
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback"}
    if dname == "contract" and args.precision.startswith("split_") and not plan.fused and not args.diagonal:
        # the tcgen05 blocked product: three split products per operand pair
        dense, useful = _tc_work(len(w["shells"]), orders)
        nc = _summed_cells(w)
        flops = 3 * 2 * dense * nc
        t_launch = dv["ms"] / dv["launches"] * 1e-3
        tpk, tkind = _tensor_peak(args.precision)
        roofline = {"bound": "tensor", "kernel": dname, "achieved": round(flops / t_launch / 1e12, 1),
                    "peak": round(tpk, 1), "unit": "TFLOP/s", "frac": round(flops / t_launch / 1e12 / tpk, 4),
                    "traffic": None, "algorithmic_flops_per_launch": flops,
                    "useful_tflops": round(2 * useful * nc / t_launch / 1e12, 1),
                    "peak_source": (f"{tkind}: MEASURED_PEAKS.json bf16_tflops_sustained x {TF32_PER_BF16:.3f} "
                                    "(nominal TF32/BF16 ratio)" if args.precision == "split_tf32" else
                                    f"{tkind}: MEASURED_PEAKS.json bf16_tflops_sustained (dense BF16/FP16 rate)")}
    fft_names = [k for k in stages if k.startswith("fft_") or k in ("x_c2r_contract", "z_conv")]
    fft_bytes = sum(stages[k]["bytes"] for k in fft_names)
    fft_ms = sum(stages[k]["ms"] for k in fft_names)

    e2e = None
    if not args.no_e2e:
        hx = [torch.from_numpy(a).pin_memory() for a in (d.x, d.y, d.z)]
        hr = [torch.from_numpy(a).pin_memory() for a in (r.x, r.y, r.z)]
        houts = {k: {n: torch.empty((ns,) * (n - 1), dtype=torch.float64).pin_memory() for n in orders}
                 for k in ("xi", "num", "den")}
        houts["dropped"] = torch.zeros(2, dtype=torch.int64).pin_memory()
        hx_np = [t.numpy() for t in hx]
        hr_np = [t.numpy() for t in hr]

        def step_host():
            plan.set_randoms(*hr_np)
            res = plan.compute(*hx_np, orders=orders, out="host", outputs=houts)
            return float(res["xi"][orders[0]].reshape(-1)[0])

        step_host()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            step_host()
        t_e2e = (time.perf_counter() - t0) * 1000.0
        if ws > 1:
            t = torch.tensor([t_e2e], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t_e2e = float(t.item())
        h2d = 12 * (d.n + r.n)
        d2h = sum(3 * 8 * ns ** (n - 1) for n in orders) + 16
        e2e = {"value": round(t_e2e / (args.e2e_steps * ws), 3), "unit": "ms/catalog", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": args.e2e_steps,
               "path": "ck_set_randoms + ck_compute with pinned host positions and host outputs"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        t0 = time.perf_counter()
        if args.factorised:
            sel = dict(n_tot=float(d.n), p_ang=sel_pa, p_z=sel_pz, z_lo=0.43, z_hi=0.70, z_max=0.75, h0=100.0,
                       omega_m=0.307, omega_k=0.0, omega_l=0.693, c=300000.0)
            ms, sample = cpu_oracle_mode_sample(w, orders, "factorised", selection=sel)
        elif args.continuous:
            ms, sample = cpu_oracle_mode_sample(w, orders, "continuous",
                                                maps=(map_d.cpu().numpy(), map_r.cpu().numpy()))
        else:
            ms, nth, sample = cpu_engine_catalog(w, orders)
        if args.factorised or args.continuous:
            cpu = {"value": round(ms, 1), "unit": "ms/catalog", "cores": 1, "kind": "oracle", "sample": sample,
                   "wall_s": round(time.perf_counter() - t0, 1)}
        else:
            cpu = {"value": round(ms, 1), "unit": "ms/catalog", "cores": nth, "kind": "oracle", "sample": sample,
                   "cpu_model": cpu_model(), "host_cores": os.cpu_count(),
                   "wall_s": round(time.perf_counter() - t0, 1)}

    plan.close()
    forms = {precision: {"ms_per_catalog": round(t_ms / (args.steps * ws), 4)}}
    if precision != "fp32" and not args.no_plain:
        # the plain FP32 form on the same catalog, timed the same way
        pplan = Plan(g.n, g.origin, g.cell, g.periodic, w["shells"], w["width"], max_order=max(orders),
                     precision="fp32")

        def pstep():
            pplan.set_randoms(rx, ry, rz)
            return pplan.compute(dx, dy, dz, orders=orders, out="device", outputs=outs)

        for _ in range(max(2, args.warmup)):
            pstep()
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        for _ in range(args.steps):
            pstep()
        p1.record(stream)
        torch.cuda.synchronize()
        tp = p0.elapsed_time(p1)
        if ws > 1:
            t = torch.tensor([tp], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            tp = float(t.item())
        if pplan.status() != 0:
            raise RuntimeError("device status in the plain FP32 form")
        pplan.close()
        forms["fp32"] = {"ms_per_catalog": round(tp / (args.steps * ws), 4)}
        forms["mixed_speedup_over_plain"] = round(tp / t_ms, 3)

    extras = None
    if ws == 1 and not args.no_extras and args.workload == "survey512" and not (
            args.diagonal or args.factorised or args.continuous):
        torch.cuda.empty_cache()
        extras = run_extras(torch, max(2, min(args.steps, 5)), 2)

    value = t_ms / (args.steps * ws)
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "ms/catalog", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_ms / args.steps, 4), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": f"f32 FFT, {precision.replace('_', '-')} sums" if precision != "fp32" else "f32",
        "data": "synthetic: seeded Neyman-Scott catalog with a lognormal-biased parent field in a survey-shell "
                "mask and uniform randoms (stand-in for SDSS DR12 CMASS + randoms)",
        "config": {"workload": args.workload, "grid": list(g.n), "cell": g.cell, "periodic": g.periodic,
                   "shells": ns, "width": w["width"], "orders": list(orders), "n_data": d.n, "n_randoms": r.n,
                   "precision": precision,
                   "step": ("ck_set_randoms + ck_compute_diagonal (both fields, every shell; Eq. 14 only)"
                            if args.diagonal else
                            "ck_set_randoms_factorised (Eq. 7, CMASS-like selection) + ck_compute"
                            if args.factorised else
                            "ck_compute_continuous (Eqs. 15-17: one delta field, every shell, no denominator)"
                            if args.continuous else "ck_set_randoms + ck_compute (both fields, every shell)"),
                   "l2": "no flush: inputs and intermediates far larger than L2 (16 scratch spectra, 8.7 GB)",
                   "tuning": tuning},
        "forms": forms,
        "roofline": roofline,
        "fft": {"gbs": round(fft_bytes / (fft_ms * 1e-3) / 1e9, 1), "frac": round(fft_bytes / (fft_ms * 1e-3) / 1e9 / peak, 4),
                "ms_per_step": round(fft_ms / args.steps, 3), "passes_per_transform": 3},
        "stages": stage_out,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
        "higher_orders": extras,
    }
    if ws > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))


def run_batch(args):
    """The batched form: 64 mocks over 8 grid classes; one step = each class's
    randoms once plus every mock through ck_batch_compute (captured CUDA
    graphs), timed against the same work as one ck_compute per mock."""
    import torch

    from paper_2108_00015_gb300 import Plan, batch_compute
    from synth import batch_workload

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    w = batch_workload()
    orders = tuple(int(c) for c in args.orders) if args.orders else w["orders"]
    dev = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
    plans, rnd = [], []
    for c in w["classes"]:
        g = c["grid"]
        plans.append(Plan(g.n, g.origin, g.cell, g.periodic, w["shells"], w["width"], max_order=max(orders),
                          precision=args.precision))
        r = c["randoms"]
        rnd.append((dev(r.x), dev(r.y), dev(r.z)))
    cats = [(dev(m.x), dev(m.y), dev(m.z), j) for j, m in w["mocks"]]
    stream = torch.cuda.current_stream()

    def step_batched():
        for p, r in zip(plans, rnd):
            p.set_randoms(*r)
        return batch_compute(plans, cats, orders=orders, out="device")

    def step_loop():
        for p, r in zip(plans, rnd):
            p.set_randoms(*r)
        return [plans[j].compute(x, y, z, orders=orders, out="device") for x, y, z, j in cats]

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    tunings = None
    if args.tuning:
        # fixed launch shapes for every grid class
        tunings = []
        for p in plans:
            p.set_tuning(*[int(v) for v in args.tuning.split(",")])
            tunings.append(p.tuning())
    elif not args.no_autotune:
        # each grid class's launch shapes, timed on its own randoms
        tunings = []
        for p, r in zip(plans, rnd):
            p.set_randoms(*r)
            tunings.append(p.autotune())
    clocks = Clocks(_smi_index(torch, local))
    clocks.start()
    t_b = timed(step_batched)
    clk = clocks.stop()
    for p in plans:
        if p.status() != 0:
            raise RuntimeError("device status in the batched form")
    t_l = timed(step_loop)
    ncat = len(cats)
    # the same batch in the plain FP32 form (CUDA-core sums), batched the same way
    t_p = None
    if args.precision != "fp32" and not args.no_plain:
        for p in plans:
            p.close()
        plans = [Plan(c["grid"].n, c["grid"].origin, c["grid"].cell, c["grid"].periodic, w["shells"], w["width"],
                      max_order=max(orders), precision="fp32") for c in w["classes"]]
        t_p = timed(step_batched)
        for p in plans:
            if p.status() != 0:
                raise RuntimeError("device status in the plain batched form")
    value = t_b / (args.steps * ncat)
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "ms/catalog", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(t_b / args.steps, 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": f"f32 FFT, {args.precision.replace('_', '-')} sums" if args.precision != "fp32" else "f32",
        "data": "synthetic: 64 seeded Neyman-Scott mocks in 8 periodic grid classes, one uniform random "
                "catalog of 10M per class",
        "config": {"workload": "batch64", "classes": [list(c["grid"].n[:1]) + [c["grid"].cell] for c in w["classes"]],
                   "mocks": ncat, "points": int(sum(m.n for _, m in w["mocks"])), "shells": len(w["shells"]),
                   "orders": list(orders), "precision": args.precision,
                   "step": "per class ck_set_randoms, then all mocks through ck_batch_compute",
                   "tuning": tunings},
        "forms": {"batched_graphs": {"ms_per_catalog": round(value, 4)},
                  **({"batched_graphs_plain_fp32": {"ms_per_catalog": round(t_p / (args.steps * ncat), 4)},
                      "mixed_speedup_over_plain": round(t_p / t_b, 3)} if t_p else {}),
                  "loop_ck_compute": {"ms_per_catalog": round(t_l / (args.steps * ncat), 4)},
                  "batched_speedup_over_loop": round(t_l / t_b, 3)},
        "clocks": clk,
    }
    for p in plans:
        p.close()
    if rank == 0:
        print(json.dumps(line))


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return
    from synth import workload
    w = workload(args.workload)
    orders = _orders(args, w)
    # each step: one whole catalog through the oracle's FP64 C++/OpenMP engine
    from oracle import cpu_engine
    cpu_engine.build()
    for _ in range(args.warmup):
        cpu_engine_catalog(w, orders)
    vals = []
    sample = None
    nth = cpu_engine.threads()
    t_run = time.perf_counter()
    for _ in range(args.steps):
        ms, nth, sample = cpu_engine_catalog(w, orders)
        vals.append(ms)
    wall = time.perf_counter() - t_run
    value = statistics.mean(vals)
    g = w["grid"]
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "ms/catalog", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(value, 1), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "grid": list(g.n), "shells": len(w["shells"]), "orders": list(orders)},
        "cpu_baseline": {"value": round(value, 1), "unit": "ms/catalog", "cores": nth, "kind": "oracle",
                         "sample": sample, "cpu_model": cpu_model(), "host_cores": os.cpu_count()},
        "e2e": {"value": round(value, 1), "unit": "ms/catalog", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "timed_wall_s": round(wall, 1),
    }
    print(json.dumps(line))


def main():
    args = _args()
    if args.diagonal:
        args.no_e2e = args.no_cpu_baseline = args.no_plain = True
    if args.factorised or args.continuous:
        args.no_e2e = args.no_plain = True
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
