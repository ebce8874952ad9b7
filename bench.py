"""Benchmark of the fused LBM stream-collide + Knudsen sensor step (one JSON line on rank 0).

Workload (default): D3Q19 BGK lid-driven cavity, 256^3 cells, FP32 populations in SoA layout,
Re = 1000 (lid u = 0.1, tau = 3 u N / Re + 1/2 = 0.5768), the sensor evaluated on every step and
reduced to 16^3 block maxima (4096 blocks), top-10 % block flags every step.  One bench step =
one fused step kernel (stream, bounce-back, moments, equilibrium, sensor, tile max, collision) +
the block-max / top-fraction flag kernels.  Data: synthetic (the cavity starts from rest).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

--impl reference times the FP64 CPU oracle on the host cores (the only CPU code this script runs,
besides the cpu_baseline sample of the default arm).  Under torchrun (N > 1) every rank runs an
independent replica of the workload on its own GPU (the path has no data-path collective here);
time is the max over ranks and the value is the total over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (lattice q, n, dtype name, re, steps of the paper-scale run, block, flag rule)
    "d3q19_256_fp32_re1000": dict(q=19, n=256, dtype="F32", re=1000.0, u=0.1, block=16,
                                  rule="top", param=0.1, sensor_every=1),
    "d2q9_128_fp64_re100": dict(q=9, n=128, dtype="F64", re=100.0, u=0.1, block=16,
                                rule="threshold", param=None, sensor_every=100),
    # mixed precision: populations stored as f - w_i in 16 bits, arithmetic in FP32
    "d3q19_512_f16s_re1000": dict(q=19, n=512, dtype="F16S", re=1000.0, u=0.1, block=16,
                                  rule="top", param=0.1, sensor_every=1),
    "d3q19_512_bf16s_re1000": dict(q=19, n=512, dtype="BF16S", re=1000.0, u=0.1, block=16,
                                   rule="top", param=0.1, sensor_every=1),
    "d3q19_512_fp32_re1000": dict(q=19, n=512, dtype="F32", re=1000.0, u=0.1, block=16,
                                  rule="top", param=0.1, sensor_every=1),
    # multi-level block mesh: 16^3 physical blocks of 32 finest cells (512^3 finest), 3 levels
    # (blocks of 8^3 / 16^3 / 32^3 cells), placement from the sensor of a seeded Re 2000 cavity
    "d3q19_blocks_512_3level": dict(q=19, n=512, dtype="F32", re=1000.0, u=0.1, block=32,
                                    rule="blocks", param=None, sensor_every=1, lmax=2,
                                    placement_re=2000.0, placement_steps=2000, seed=2000),
    # learned sensor predictor: D2Q9 1024^2 FP32 cavities, Re ~ U[100, 5000] per seed, 64 x 64
    # blocks of 16^2, a 3-layer 16-channel BF16 conv net predicting the block maxima 200 steps
    # ahead from the block-averaged (rho, u_x, u_y); regrid every 200 steps
    "d2q9_1024_learned": dict(q=9, n=1024, dtype="F32", re=None, u=0.1, block=16,
                              rule="learned", param=None, sensor_every=200, horizon=200,
                              re_range=(100.0, 5000.0), train_seeds=8, eval_seeds=2, warm=2000,
                              snapshots=60, epochs=40, batch=16, lr=2e-3, fallback_below=0.9),
    # regrid of the developed 256^3 cavity from its per-cell sensor (Sec. 5.2): tags on 4^3 tag
    # cells above the fixed threshold, one buffer layer, clustering at 80 % efficiency; plus the
    # fitted level map of the 16^3 block maxima
    "d3q19_256_regrid": dict(q=19, n=256, dtype="F32", re=1000.0, u=0.1, block=16,
                             rule="regrid", param=None, sensor_every=1, warm=2000, coarsen=4,
                             buffer=1, efficiency=0.8, min_width=2),
}
DEFAULT_WORKLOAD = "d3q19_256_fp32_re1000"
BYTES_PER_ELEM = {"F64": 8, "F32": 4, "F16S": 2, "BF16S": 2}
DTYPE_NAME = {"F64": "f64", "F32": "f32", "F16S": "f16(f-w)/f32", "BF16S": "bf16(f-w)/f32"}


def tau_of(w):
    # nu = u N / Re and nu = (tau - 1/2) / 3
    return 3.0 * w["u"] * w["n"] / w["re"] + 0.5


def threshold_of(w):
    # four times the Couette-level sensor value of the mean lid shear, (4/3) tau u / N
    return 4.0 * (4.0 / 3.0) * tau_of(w) * w["u"] / w["n"]


def cells_of(w):
    return w["n"] ** (3 if w["q"] == 19 else 2)


def algorithmic_bytes_per_cell(w):
    # read q populations + write q populations; the tile maxima are < 0.01 % of it
    return 2 * w["q"] * BYTES_PER_ELEM[w["dtype"]]


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            pk = json.load(fh)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def step_kernel_of(w, variant="auto"):
    """Name of the fused step kernel the library picks for the workload (LBM_KERNEL_AUTO: the
    two-cell packed kernel with an even nx and (q + 1) * cells < 2^32 for 16-bit storage and for
    FP32 storage on D2Q9 lattices of at least 2^17 cells; else the one-cell kernel) and the headers
    that define it."""
    cells = w["n"] ** (3 if w["q"] == 19 else 2)
    pair = ("fused_step_pair_kernel", ("lbm_step_pair.cuh", "lbm_step.cuh", "lbm_traits.cuh"))
    if variant == "pair":
        return pair
    if variant == "tma":
        return "fused_step_tma_kernel", ("lbm_step_tma.cuh", "lbm_step.cuh", "lbm_traits.cuh")
    if variant == "tma_pair":
        return "fused_step_tma_pair_kernel", ("lbm_step_tma_pair.cuh", "lbm_step_tma.cuh",
                                              "lbm_step_pair.cuh", "lbm_step.cuh", "lbm_traits.cuh")
    applicable = w["n"] % 2 == 0 and (w["q"] + 1) * cells < 1 << 32
    if variant == "auto" and applicable and (
            w["dtype"] in ("F16S", "BF16S") or (w["dtype"] == "F32" and w["q"] == 9
                                                 and cells >= 1 << 17)):
        return pair
    return "fused_step_kernel", ("lbm_step.cuh", "lbm_traits.cuh")


def kernel_source_hash(w, variant="auto"):
    h = hashlib.sha256()
    for fn in step_kernel_of(w, variant)[1]:
        with open(os.path.join(ROOT, "paper_1507_06767_gb300", "csrc", fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload, w, variant="auto"):
    """DRAM bytes per launch of the fused step from the committed ncu summary, if it was taken on
    the current kernel source at the lattice size run now, with the default kernel choice; else
    None."""
    if w["n"] != WORKLOADS[workload]["n"] or variant != "auto":
        return None
    path = os.path.join(ROOT, "profiles", f"fused_step_{workload}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m_src = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    m_tr = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not m_src or not m_tr or m_src.group(1) != kernel_source_hash(w, variant):
        return None
    return float(m_tr.group(1))


# sources of the multi-level cycle's kernels (steps, ghost fills, restrictions)
CYCLE_SOURCES = ("lbm_multilevel.cu", "lbm_step_pair.cuh", "lbm_step.cuh", "lbm_traits.cuh")


def cycle_source_hash():
    h = hashlib.sha256()
    for fn in CYCLE_SOURCES:
        with open(os.path.join(ROOT, "paper_1507_06767_gb300", "csrc", fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_cycle_traffic(workload, w, step_form="auto", fusion="auto", schedule="auto",
                           persistent=False):
    """DRAM bytes per level-0 cycle of the multi-level mesh (all kernels of the cycle's graph)
    from the committed ncu summary, if it was taken on the current sources, on the full mesh, with
    the automatic schedule and the graph form of the cycle; else None."""
    if (persistent or w["n"] != WORKLOADS[workload]["n"]
            or (step_form, fusion, schedule) != ("auto", "auto", "auto")):
        return None
    path = os.path.join(ROOT, "profiles", f"cycle_dram_{workload}.md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m_src = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    m_tr = re.search(r"dram_bytes_per_cycle:\s*([0-9.eE+]+)", txt)
    if not m_src or not m_tr or m_src.group(1) != cycle_source_hash():
        return None
    return float(m_tr.group(1))


def nvtx_push(name):
    """Open an NVTX range on the host thread (a no-op where NVTX is not available)."""
    try:
        import torch

        torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


def nvtx_pop():
    try:
        import torch

        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


class ClockSampler:
    """nvidia-smi clock / throttle samples of this process's GPU.  Each sample carries nvidia-smi's
    own timestamp, so samples can be assigned to the timed windows (``window``) even when the
    pipe delivers them late; the statistics cover the samples inside a window ("under load"), or
    every sample when no window was marked."""

    FIELDS = ("timestamp,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.lines = []
        self.windows = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def window(self, t0, t1):
        """Mark [t0, t1] (time.time() seconds) as a timed window."""
        self.windows.append((t0, t1))

    @staticmethod
    def _stamp(text):
        import datetime

        try:
            return datetime.datetime.strptime(text, "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def parse(self):
        """Samples of this GPU as (time, sm MHz, max MHz, power W, set of active reasons)."""
        out = []
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 10:
                continue
            if self.uuid and parts[1] != self.uuid:
                continue
            try:
                sm, mx = float(parts[2]), float(parts[3])
            except ValueError:
                continue
            try:
                pw = float(parts[4])
            except ValueError:
                pw = None
            reasons = {name for name, val in zip(self.REASONS, parts[6:10])
                       if val.lower() == "active"}
            out.append((self._stamp(parts[0]), sm, mx, pw, reasons))
        return out

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        samples = self.parse()
        if not samples:
            return None
        if self.windows:
            load = [sm for sm in samples if sm[0] is not None and
                    any(t0 <= sm[0] <= t1 for t0, t1 in self.windows)]
        else:
            load = samples
        use = load if load else samples
        bins = {}
        for sm in use:
            key = str(int(round(sm[1])))
            bins[key] = bins.get(key, 0) + 1
        reasons = set()
        for sm in use:
            reasons |= sm[4]
        powers = [sm[3] for sm in use if sm[3] is not None]
        return {"sm_mhz": statistics.median(sm[1] for sm in use),
                "sm_max_mhz": max(sm[2] for sm in samples), "samples": len(samples),
                "samples_under_load": len(load),
                "sm_mhz_bins": dict(sorted(bins.items(), key=lambda kv: -int(kv[0]))),
                "power_w_max": max(powers) if powers else None,
                "reasons": sorted(reasons)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(value, ws):
    if ws == 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


# --------------------------------------------------------------------- multi-level placement
def balance_levels(leaf):
    """Raise levels until touching blocks (26-neighbourhood) differ by at most one."""
    import numpy as np

    leaf = leaf.copy()
    while True:
        pad = np.pad(leaf, 1, mode="edge")
        nbmax = leaf.copy()
        nz, ny, nx = leaf.shape
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    nbmax = np.maximum(nbmax, pad[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny,
                                                  1 + dx:1 + dx + nx])
        new = np.maximum(leaf, nbmax - 1)
        if np.array_equal(new, leaf):
            return leaf
        leaf = new


def block_placement(w, L):
    """Leaf levels of the 16^3 blocks: the Knudsen sensor of a seeded D2Q9 128^2 cavity at
    Re = placement_re after placement_steps steps, reduced to 8x8-cell block maxima (16 x 16),
    mapped onto levels 0..lmax with the fitted level map (phi = log2 K normalised over the blocks),
    extruded along z and balanced 2:1."""
    import numpy as np

    n2 = 128
    tau2 = 3.0 * w["u"] * n2 / w["placement_re"] + 0.5
    lat = L.Lattice(L.LBM_D2Q9, n2, n2, 1, tau2, dtype=L.LBM_F64, lid=(w["u"], 0.0))
    f = lat.populations()
    g = np.random.default_rng(w["seed"])
    f = f * (1.0 + g.uniform(-1e-6, 1e-6, size=f.shape))  # the seeded perturbation of the start
    lat.set_populations(f)
    lat.step(w["placement_steps"])
    nb = w["n"] // w["block"]
    lev2 = lat.levels_fit(n2 // nb, 0, w["lmax"]).reshape(nb, nb)
    lat.close()
    leaf = np.repeat(lev2[None, :, :], nb, axis=0).astype(np.int8)
    return balance_levels(leaf)


def run_blocks(args, w, ws, rank, local):
    import numpy as np
    import torch

    import paper_1507_06767_gb300 as L

    torch.cuda.set_device(local)
    leaf = block_placement(w, L)
    tau = tau_of(w)
    form = getattr(L, "LBM_STEP_FORM_" + args.step_form.upper())
    fusion = getattr(L, "LBM_FUSION_" + args.fusion.upper())
    schedule = getattr(L, "LBM_SCHEDULE_" + args.schedule.upper())
    mesh = L.BlockMesh(leaf, w["block"], w["lmax"], tau, lid=(w["u"], 0.0), step_form=form,
                       fusion=fusion, schedule=schedule)
    persistent = mesh.cycle_form() == L.LBM_SCHEDULE_PERSISTENT
    info = [mesh.info(l) for l in range(w["lmax"] + 1)]
    updates = info[0][5]  # cell updates per cycle over all levels
    for _ in range(args.warmup):
        mesh.step(1)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(None)
    sampler.start()
    time.sleep(0.3)
    nvtx_push("timed")  # lets a profiler capture the timed loop alone (ncu --nvtx-include timed/)
    reps = timed_repeats(lambda: mesh.step(args.steps), stream, ws, sampler, args.min_time)
    nvtx_pop()
    clocks = sampler.stop()
    ms = reduce_max(statistics.median(reps), ws)  # one repeat of args.steps cycles
    value = updates * args.steps * ws / (ms / 1e3) / 1e6
    # N_eff (Sec. 5.2): cells weighted by their update frequency, sum_l n_l / 2^(L - l) over the
    # leaf cells
    leaf_cells = [int((leaf == l).sum()) * info[l][0] ** 3 for l in range(w["lmax"] + 1)]
    n_eff = sum(c / 2 ** (w["lmax"] - l) for l, c in enumerate(leaf_cells))
    peak, peak_kind = load_peaks()
    achieved = 152.0 * updates / (ms / args.steps / 1e3) / 1e9
    t0 = time.perf_counter()
    bm = mesh.step(1, block_max=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    out = {
        "metric": "multi-level fused stream-collide+sensor MLUPS (cell updates, all levels)",
        "value": round(value, 1), "unit": "MLUPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (lid-driven cavity from rest on a sensor-placed 3-level block mesh)",
        "config": {"workload": args.workload, "blocks": int(leaf.size), "block_edge": w["block"],
                   "levels": w["lmax"] + 1,
                   "blocks_per_leaf_level": [int((leaf == l).sum()) for l in range(w["lmax"] + 1)],
                   "cells_per_level": [info[l][2] * info[l][0] ** 3 for l in range(w["lmax"] + 1)],
                   "tau_per_level": [round(info[l][1], 6) for l in range(w["lmax"] + 1)],
                   "step_launch_shape": [[info[l][3], info[l][4]] for l in range(w["lmax"] + 1)],
                   "step_schedule": [dict(zip(("form", "planes", "fused_planes"),
                                              mesh.schedule(l))) for l in range(w["lmax"] + 1)],
                   "cell_updates_per_cycle": updates, "n_eff": n_eff,
                   "uniform_finest_cells": w["n"] ** 3,
                   "step": ("one level-0 cycle (one persistent launch, replayed as a graph)"
                            if persistent else "one level-0 cycle (graph of separate launches)"),
                   "timing": (f"{len(reps)} repeats of {args.steps} cycles (>= {args.min_time} s of "
                              "device time), median"),
                   "l2": "level buffers > 129 MB L2, no flush"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "traffic": recorded_cycle_traffic(args.workload, w, args.step_form,
                                                       args.fusion, args.schedule, persistent),
                     "traffic_unit": "DRAM bytes per cycle, all kernels (ncu)",
                     "algorithmic_bytes_per_cycle": 152 * updates, "peak_kind": peak_kind,
                     "kernel": "whole cycle (152 B per cell update; ghost and restriction work "
                               "not counted)"},
        "e2e": {"value": round(updates / e2e_s / 1e6, 1), "unit": "MLUPS",
                "h2d_bytes_per_step": int(leaf.size), "d2h_bytes_per_step": int(8 * bm.size)},
        "repeats": len(reps),
        # per cycle, graph form: level l takes 2^l steps, a finer one a ghost fill before every
        # pair of its steps (one launch fills the ghosts of both), and 2^l restrictions onto
        # level l unless the finer level's second sub-step does them (brick or tiled fused form);
        # persistent form: one launch per cycle
        "gpu_launches": len(reps) * args.steps if persistent else len(reps) * args.steps * sum(
            (1 << l) + ((1 << (l - 1)) if l > 0 else 0)
            + ((1 << l) if l < w["lmax"] and info[l + 1][2] > 0
               and mesh.schedule(l + 1)[2] == 0 else 0)
            for l in range(w["lmax"] + 1) if info[l][2] > 0),
        "clocks": clocks,
    }
    mesh.close()
    return out


def run_regrid(args, w, ws, rank, local):
    """Regrid workload: the developed cavity's per-cell sensor field is tagged, buffered and
    clustered into boxes (lbm_regrid), and its block maxima mapped to levels (lbm_levels_fit); one
    bench step is one such regrid.  lbm_regrid makes its cut decisions on the host between rounds
    of GPU signature passes, so a regrid is timed on the host clock around the synchronising
    call."""
    import numpy as np
    import torch

    import paper_1507_06767_gb300 as L

    torch.cuda.set_device(local)
    n = w["n"]
    tau = tau_of(w)
    lat = L.Lattice(19, n, n, n, tau, dtype=L.LBM_F32, lid=(w["u"], 0.0))
    L.lbm_set_sensor_every(lat.h, 0)
    L.lbm_set_sensor_field(lat.h, 1)
    lat.step(w["warm"])
    torch.cuda.synchronize()
    T = threshold_of(w)
    kw = dict(coarsen=w["coarsen"], buffer=w["buffer"], efficiency=w["efficiency"],
              min_width=w["min_width"])
    nb = L.lbm_nblocks(lat.h, w["block"])
    lev = np.empty(nb, dtype=np.int8)
    for _ in range(args.warmup):
        boxes, tags = lat.regrid(T, **kw)
    torch.cuda.synchronize()
    sampler = ClockSampler(None)
    sampler.start()
    time.sleep(0.3)
    barrier(ws)
    t_reg, t_lev = [], []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        boxes, tags = lat.regrid(T, **kw)
        t1 = time.perf_counter()
        L.lbm_levels_fit(lat.h, w["block"], 0, 2, L.LBM_SENSOR_LAST, lev)
        t2 = time.perf_counter()
        t_reg.append(t1 - t0)
        t_lev.append(t2 - t1)
    clocks = sampler.stop()
    ms = reduce_max(1e3 * statistics.median(t_reg), ws)
    cells = n ** 3
    field_bytes = 4 * cells  # the FP32 sensor field the tag pass reads
    covered = int(((boxes[:, 3:] - boxes[:, :3]).prod(axis=1)).sum()) if len(boxes) else 0
    peak, peak_kind = load_peaks()
    out = {
        "metric": "regrid of one level from the per-cell sensor (tags, buffer, clustering)",
        "value": round(ms, 3), "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 field, integer tags",
        "data": "synthetic (lid-driven cavity from rest, sensor field after the warm-up steps)",
        "config": {"workload": args.workload, "lattice": "D3Q19", "cells": cells,
                   "warm_steps": w["warm"], "threshold": T, "coarsen": w["coarsen"],
                   "buffer": w["buffer"], "efficiency": w["efficiency"],
                   "min_width": w["min_width"], "boxes": int(len(boxes)),
                   "tagged_tag_cells": int(tags.sum()), "tag_cells": int(tags.size),
                   "cells_in_boxes": covered, "level_map_ms": round(1e3 * statistics.median(t_lev), 3),
                   "timing": "host clock around the synchronising call, median over steps"},
        "roofline": {"bound": "hbm", "achieved": round(field_bytes / (ms / 1e3) / 1e9, 1),
                     "peak": peak, "unit": "GB/s",
                     "frac": round(field_bytes / (ms / 1e3) / 1e9 / peak, 4), "traffic": None,
                     "peak_kind": peak_kind,
                     "kernel": "whole regrid (sensor-field bytes over the call's time; the call "
                               "also waits on host decisions between signature rounds)"},
        "e2e": {"value": round(ms, 3), "unit": "ms", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": int(tags.size + 24 * len(boxes))},
        # per step: tag pass, three 1-D dilations, one signature pass per clustering round (the
        # rounds follow the data: 4 on this workload, profiles/launches_d3q19_256_regrid.md), and
        # the level map's two kernels
        "gpu_launches": args.steps * (1 + 3 + 4 + 2),
        "clocks": clocks,
    }
    lat.close()
    return out


def run_learned(args, w, ws, rank, local):
    """Learned-predictor workload: solver traces on seeded cavities, BF16 training, judging on
    held-out seeds, then the timed dynamic-refinement loop (solver steps; every `horizon` steps
    the block features, the network's forward pass, the predicted maxima and their flags)."""
    import numpy as np
    import torch

    import paper_1507_06767_gb300 as L
    from paper_1507_06767_gb300 import learned as LN

    torch.cuda.set_device(local)
    n, b, hz = w["n"], w["block"], w["horizon"]
    g = np.random.default_rng(np.random.SeedSequence([1024, 5000, rank]))
    res = g.uniform(w["re_range"][0], w["re_range"][1], size=w["train_seeds"] + w["eval_seeds"])
    t0 = time.perf_counter()
    # the residual predictor: block means and the log sensor maximum now in, the change of log10 K
    # over the horizon out
    traces = [LN.cavity_trace(n, float(re), w["u"], b, w["warm"], w["snapshots"], hz,
                              with_sensor=True) for re in res]
    trace_s = time.perf_counter() - t0
    Xs, Ts = zip(*[LN.pairs(f, k) for f, k, _ in traces[:w["train_seeds"]]])
    X, T = torch.cat(Xs), torch.cat(Ts)
    net = L.Net(4, 16)
    shift, scale = LN.normalisation(w["u"], with_sensor=True)
    net.set_normalisation(shift, scale)
    # He-uniform initial weights from a seeded generator, zero biases
    theta = []
    for cin in (4, 16, 16):
        cout = 1 if len(theta) == 4 else 16
        lim = math.sqrt(6.0 / (cin * 9))
        theta += [g.uniform(-lim, lim, cout * cin * 9), np.zeros(cout)]
    net.set_params(np.concatenate(theta))
    t0 = time.perf_counter()
    losses = LN.train(net, X, T, w["epochs"], w["batch"], w["lr"], seed=7)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    steps_trained = w["epochs"] * (X.shape[0] // w["batch"])
    judged = []
    for (f, k, tau) in traces[w["train_seeds"]:]:
        judged.append(LN.judge(net, f, k, LN.threshold(tau, w["u"], n), w["fallback_below"]))
    summary = {key: float(np.mean([j[key] for j in judged])) for key in judged[0]
               if key != "per_regrid"}

    # timed loop on a fresh cavity at the mean Reynolds number of the range
    re = 0.5 * (w["re_range"][0] + w["re_range"][1])
    tau = 3.0 * w["u"] * n / re + 0.5
    lat = L.Lattice(L.LBM_D2Q9, n, n, 1, tau, dtype=L.LBM_F32, lid=(w["u"], 0.0))
    L.lbm_set_kernel_variant(lat.h, getattr(L, "LBM_KERNEL_" + args.kernel.upper()))
    L.lbm_set_sensor_every(lat.h, hz)
    side = n // b
    feats = torch.empty((1, 4, side, side), dtype=torch.float32, device="cuda")
    y = torch.empty((1, 1, side, side), dtype=torch.float32, device="cuda")
    know = torch.empty(side * side, dtype=torch.float64, device="cuda")
    kpred = torch.empty(side * side, dtype=torch.float64, device="cuda")
    fl = torch.empty(side * side, dtype=torch.int8, device="cuda")
    T_thr = LN.threshold(tau, w["u"], n)
    stream = torch.cuda.current_stream()

    def predict():
        L.lbm_sensor_dev(lat.h, b, know)
        L.lbm_block_features(lat.h, b, feats)
        L.lbm_net_log_targets(know, know.numel(), LN.LOG_OFFSET, LN.FLOOR_K, feats[0, 3])
        net.forward(feats, out=y)
        L.lbm_net_to_maxima_residual(y, know, y.numel(), LN.FLOOR_K, kpred)
        L.lbm_flags_from_maxima(kpred, L.LBM_F64, kpred.numel(), L.LBM_FLAG_THRESHOLD, T_thr, fl,
                                stream.cuda_stream)

    def regrid_step():
        L.lbm_step(lat.h, hz)
        predict()

    for _ in range(args.warmup):
        regrid_step()
    torch.cuda.synchronize()
    nreg = max(1, args.steps // hz)
    # the fused kernel's duration, from the library's per-launch CUDA events over one pass of the
    # loop; the timed pass below runs without them (at 1024^2 a step is ~16 us, and two event
    # records per launch would show in the loop's time)
    L.lbm_set_profiling(lat.h, 1)
    for _ in range(nreg):
        regrid_step()
    k_ms, k_n = L.lbm_kernel_time(lat.h)
    L.lbm_set_profiling(lat.h, 0)
    sampler = ClockSampler(None)
    sampler.start()
    time.sleep(0.3)
    barrier(ws)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    nvtx_push("timed")  # lets a profiler capture the timed loop alone (ncu --nvtx-include timed/)
    ev0.record(stream)
    for _ in range(nreg):
        regrid_step()
    ev1.record(stream)
    nvtx_pop()
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    ms = reduce_max(ev0.elapsed_time(ev1), ws)
    steps = nreg * hz
    value = n * n * steps * ws / (ms / 1e3) / 1e6
    # the network's share: time the regrid-only calls alone
    ev2 = torch.cuda.Event(enable_timing=True)
    ev3 = torch.cuda.Event(enable_timing=True)
    ev2.record(stream)
    for _ in range(20):
        predict()
    ev3.record(stream)
    torch.cuda.synchronize()
    regrid_ms = ev2.elapsed_time(ev3) / 20
    # end to end: host features of each regrid come back with its flags
    host_fl = torch.empty(side * side, dtype=torch.int8, pin_memory=True)
    t0 = time.perf_counter()
    for _ in range(nreg):
        regrid_step()
        host_fl.copy_(fl)
    torch.cuda.synchronize()
    e2e_s = reduce_max(time.perf_counter() - t0, ws)
    peak, peak_kind = load_peaks()
    avg_kernel_ms = k_ms / max(k_n, 1)
    per_launch = 2 * 9 * 4 * n * n
    achieved = per_launch / (avg_kernel_ms / 1e3) / 1e9
    lat.close()
    net.close()
    return {
        "metric": "dynamic-refinement loop MLUPS with the learned sensor predictor",
        "value": round(value, 1), "unit": "MLUPS", "n_gpus": ws, "steps": steps,
        "warmup": args.warmup, "ms_per_step": round(ms / steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 solver, bf16 network",
        "data": "synthetic (seeded lid-driven cavities from rest, Re ~ U[100, 5000])",
        "config": {"workload": args.workload, "lattice": "D2Q9", "cells": n * n, "block": b,
                   "blocks": side * side, "horizon": hz, "train_cavities": w["train_seeds"],
                   "eval_cavities": w["eval_seeds"], "timed_re": re,
                   "l2": "population buffers 75 MB, below the 129 MB L2 (a launch-bound size)"},
        "predictor": {"form": "residual: block means and log10 K now in, change of log10 K out",
                      "train_samples": int(X.shape[0]), "epochs": w["epochs"],
                      "adam_steps": steps_trained, "trace_s": round(trace_s, 2),
                      "train_s": round(train_s, 2),
                      "train_ms_per_step": round(1e3 * train_s / max(steps_trained, 1), 3),
                      "loss_first_epoch": round(losses[0], 5), "loss_last_epoch": round(losses[-1], 5),
                      "regrid_ms": round(regrid_ms, 4), **{k: round(v, 4) for k, v in summary.items()}},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": None, "peak_kind": peak_kind,
                     "kernel": step_kernel_of(w, args.kernel)[0] + " (D2Q9 FP32, 72 B per cell)",
                     "kernel_ms": round(avg_kernel_ms, 5),
                     "note": "kernel_ms from a pass with per-launch events, which lengthen a "
                             "~12 us launch; the loop's own time per step bounds it from above",
                     "loop_gbs": round(per_launch / (ms / steps / 1e3) / 1e9, 1)},
        "e2e": {"value": round(n * n * steps * ws / e2e_s / 1e6, 1), "unit": "MLUPS",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": round(side * side / hz, 2)},
        # per regrid: block maxima (2), features, log channel, three convolutions, maxima, flags
        "gpu_launches": steps + nreg * 9,
        "clocks": clocks,
    }


# ----------------------------------------------------------------------------------- our arm
# Device time the timed region accumulates: the loop of --steps steps is repeated until at least
# this much device time has passed, and the per-step time is the median over the repeats.
MIN_TIMED_S = 1.5
# mixed-precision row: the 512^3 cavity in each storage type, and the error check at 128^3
MIXED_WORKLOADS = ("d3q19_512_fp32_re1000", "d3q19_512_f16s_re1000", "d3q19_512_bf16s_re1000")
MIXED_ERROR = dict(n=128, steps=5000, re=1000.0, u=0.1, block=16)


def timed_repeats(run_k, stream, ws, sampler, min_s=MIN_TIMED_S):
    """Run ``run_k()`` (one repeat of the timed steps) until ``min_s`` seconds of device time have
    accumulated.  The first repeat is timed alone to size the rest, which are queued back to back
    (an event pair around each, one synchronisation at the end) so the GPU never idles between
    them.  Returns the per-repeat milliseconds."""
    import torch

    barrier(ws)
    torch.cuda.synchronize()
    t_start = time.time()

    def pair():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    e0, e1 = pair()
    e0.record(stream)
    run_k()
    e1.record(stream)
    e1.synchronize()
    first = e0.elapsed_time(e1)
    reps = max(0, math.ceil(min_s * 1e3 / max(first, 1e-3)) - 1)
    evs = []
    for _ in range(reps):
        a, b = pair()
        a.record(stream)
        run_k()
        b.record(stream)
        evs.append((a, b))
    torch.cuda.synchronize()
    sampler.window(t_start, time.time())
    barrier(ws)
    return [first] + [a.elapsed_time(b) for a, b in evs]


def time_uniform(L, w, args, ws, sampler, kernel="auto", min_s=MIN_TIMED_S):
    """Time the uniform-lattice workload ``w``: one bench step = one fused step (sensor on its
    sensor steps) + the block-max / flag kernels.  Returns the open lattice, its flag closure and
    the timing record."""
    import torch

    q, n = w["q"], w["n"]
    nz = n if q == 19 else 1
    tau = tau_of(w)
    lat = L.Lattice(q, n, n, nz, tau, dtype=getattr(L, "LBM_" + w["dtype"]), lid=(w["u"], 0.0))
    h = lat.h
    L.lbm_set_kernel_variant(h, getattr(L, "LBM_KERNEL_" + kernel.upper()))
    L.lbm_set_sensor_every(h, w["sensor_every"])
    lat.block = w["block"]
    nb = L.lbm_nblocks(h, w["block"])
    flags_dev = torch.empty(nb, dtype=torch.int8, device="cuda")
    param = w["param"] if w["rule"] == "top" else threshold_of(w)
    flag_dev = L.lbm_flag_top_dev if w["rule"] == "top" else L.lbm_flag_dev

    def one_step():
        L.lbm_step(h, 1)
        if w["sensor_every"] == 1 or L.lbm_steps_done(h) % w["sensor_every"] == 0:
            flag_dev(h, param, flags_dev)

    def run_k():
        for _ in range(args.steps):
            one_step()

    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    L.lbm_set_profiling(h, 1)
    reps = timed_repeats(run_k, stream, ws, sampler, min_s)
    k_ms, k_n = L.lbm_kernel_time(h)
    L.lbm_set_profiling(h, 0)
    per_step = sorted(r / args.steps for r in reps)
    ms_step = reduce_max(statistics.median(per_step), ws)
    cells = cells_of(w)
    peak, peak_kind = load_peaks()
    per_launch_bytes = algorithmic_bytes_per_cell(w) * cells
    avg_kernel_ms = k_ms / max(k_n, 1)
    achieved = per_launch_bytes / (avg_kernel_ms / 1e3) / 1e9
    rec = {
        "value": cells * ws / (ms_step / 1e3) / 1e6, "ms_per_step": ms_step,
        "repeats": len(reps), "timed_steps": len(reps) * args.steps,
        "ms_per_step_min_max": [per_step[0], per_step[-1]],
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4),
                     "traffic": recorded_traffic(w["name"], w, kernel),
                     "peak_kind": peak_kind, "kernel": step_kernel_of(w, kernel)[0],
                     "kernel_ms": round(avg_kernel_ms, 5),
                     "algorithmic_bytes_per_launch": per_launch_bytes},
        "nbytes": L.lbm_population_bytes(h), "nb": nb, "param": param, "tau": tau,
        "n_sensor_per_repeat": args.steps // w["sensor_every"],
    }
    return lat, flag_dev, rec


def mixed_error_block(L):
    """Error of each storage type against the library's FP64 path (which the parity tests hold to
    the FP64 oracle within 1e-12) on the 128^3 Re 1000 cavity after 5000 steps, sensor on the last
    step: populations, density, velocity, per-cell sensor, 16^3 block maxima, flag agreement."""
    import numpy as np

    e = MIXED_ERROR
    n, u = e["n"], e["u"]
    tau = 3.0 * u * n / e["re"] + 0.5
    T = 4.0 * (4.0 / 3.0) * tau * u / n
    res = {}
    for name in ("F64", "F32", "F16S", "BF16S"):
        lat = L.Lattice(19, n, n, n, tau, dtype=getattr(L, "LBM_" + name), lid=(u, 0.0))
        L.lbm_set_sensor_field(lat.h, 1)
        lat.step(e["steps"])
        rho, uu = lat.moments()
        res[name] = dict(f=lat.populations(), rho=rho, u=uu, K=lat.sensor_field(),
                         bmax=lat.sensor(e["block"]), top=lat.flag_top(0.1, block=e["block"]),
                         thr=lat.flag(T, block=e["block"]))
        lat.close()
    ref = res["F64"]
    out = {"lattice": f"D3Q19 {n}^3 cavity", "re": e["re"], "tau": round(tau, 6),
           "steps": e["steps"], "against": "the library's FP64 storage path",
           "umax": float(np.abs(ref["u"]).max()), "Kmax": float(ref["K"].max())}
    for name in ("F32", "F16S", "BF16S"):
        g = res[name]
        out[name.lower()] = {
            "f_rel": float(np.abs(g["f"] - ref["f"]).max() / np.abs(ref["f"]).max()),
            "rho_abs": float(np.abs(g["rho"] - ref["rho"]).max()),
            "u_rel": float(np.abs(g["u"] - ref["u"]).max() / np.abs(ref["u"]).max()),
            "K_rel": float(np.abs(g["K"] - ref["K"]).max() / ref["K"].max()),
            "K_blockmax_rel": float(np.abs(g["bmax"] - ref["bmax"]).max() / ref["bmax"].max()),
            "top10_flags_agree": float((g["top"] == ref["top"]).mean()),
            "threshold_flags_agree": float((g["thr"] == ref["thr"]).mean()),
        }
    return out


def run_mixed(args, ws, uuid):
    """Mixed-precision half of the metric: the 512^3 D3Q19 Re 1000 cavity stored in FP32, FP16
    (f - w_i) and BF16 (f - w_i), each timed like the headline workload, plus the live error
    check of the storage types."""
    import torch

    import paper_1507_06767_gb300 as L

    out = {"workload": "d3q19_512_re1000", "cells": 512 ** 3}
    sampler = ClockSampler(uuid)
    sampler.start()
    time.sleep(0.3)
    fp32 = None
    for name in MIXED_WORKLOADS:
        w = dict(WORKLOADS[name], name=name)
        lat, _, rec = time_uniform(L, w, args, ws, sampler, min_s=min(1.0, args.min_time))
        lat.close()
        torch.cuda.synchronize()
        key = w["dtype"].lower()
        entry = {"value": round(rec["value"], 1), "unit": "MLUPS",
                 "ms_per_step": round(rec["ms_per_step"], 5), "repeats": rec["repeats"],
                 "dtype": DTYPE_NAME[w["dtype"]], "roofline": rec["roofline"]}
        if fp32 is None:
            fp32 = rec["value"]
        else:
            entry["ratio_to_fp32"] = round(rec["value"] / fp32, 4)
        out[key] = entry
    out["clocks"] = sampler.stop()
    out["error_vs_f64"] = mixed_error_block(L)
    return out


def run_ours(args, w, ws, rank, local):
    import torch

    import paper_1507_06767_gb300 as L

    torch.cuda.set_device(local)
    dev_props = torch.cuda.get_device_properties(local)
    uuid = getattr(dev_props, "uuid", None)
    uuid = f"GPU-{uuid}" if uuid is not None and not str(uuid).startswith("GPU-") else uuid
    w = dict(w, name=args.workload)
    q, n = w["q"], w["n"]
    cells = cells_of(w)

    # ---- device-resident timed region: repeats of --steps steps, >= MIN_TIMED_S of device time
    sampler = ClockSampler(uuid)
    sampler.start()
    time.sleep(0.3)
    lat, flag_dev, rec = time_uniform(L, w, args, ws, sampler, kernel=args.kernel,
                                      min_s=args.min_time)
    clocks = sampler.stop()
    h = lat.h
    nb, param, nbytes = rec["nb"], rec["param"], rec["nbytes"]
    stream = torch.cuda.current_stream()

    # ---- end to end through the C ABI with host buffers, one job of as many steps as the timed
    # region ran: the job's initial state goes up from pinned host memory, every sensor step's
    # flags come back to pinned host memory, the final state comes back.  The flags of a step are
    # copied while the next step runs (two flag buffers); the host waits for step k's flags after
    # launching step k + 1, as a driver that regrids from them would.
    host_state = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    L.lbm_get_raw(h, host_state.data_ptr(), nbytes)
    host_flags = [torch.empty(nb, dtype=torch.int8, pin_memory=True) for _ in range(2)]
    dev_flags = [torch.empty(nb, dtype=torch.int8, device="cuda") for _ in range(2)]
    flag_ready = [torch.cuda.Event() for _ in range(2)]
    e2e_steps = rec["timed_steps"]
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L.lbm_set_raw(h, host_state.data_ptr(), nbytes)
    t_up = time.perf_counter() - t0
    pending = None
    for k in range(e2e_steps):
        L.lbm_step(h, 1)
        if w["sensor_every"] == 1 or (k + 1) % w["sensor_every"] == 0:
            j = k & 1
            flag_dev(h, param, dev_flags[j])
            host_flags[j].copy_(dev_flags[j], non_blocking=True)
            flag_ready[j].record(stream)
            if pending is not None:
                flag_ready[pending].synchronize()  # the previous sensor step's flags are home
            pending = j
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    L.lbm_get_raw(h, host_state.data_ptr(), nbytes)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    t_down = t2 - t1
    e2e_s = reduce_max(t2 - t0, ws)
    barrier(ws)
    lat.close()
    del host_state
    torch.cuda.synchronize()
    n_flag_reads = e2e_steps // w["sensor_every"]
    e2e = {"value": round(cells * e2e_steps * ws / e2e_s / 1e6, 1), "unit": "MLUPS",
           "h2d_bytes_per_step": int(round(nbytes / e2e_steps)),
           "d2h_bytes_per_step": int(round((nbytes + n_flag_reads * nb) / e2e_steps)),
           "job_steps": e2e_steps,
           # host link rates seen by the state copies of this run (they vary with the host)
           "state_h2d_gbs": round(nbytes / t_up / 1e9, 1),
           "state_d2h_gbs": round(nbytes / t_down / 1e9, 1)}

    # launches of our kernels in the timed region: fused step every step, plus tile->block and
    # flag kernels on sensor steps
    gpu_launches = rec["timed_steps"] + 2 * rec["n_sensor_per_repeat"] * rec["repeats"]
    out = {
        "metric": "fused stream-collide+sensor MLUPS",
        "value": round(rec["value"], 1),
        "unit": "MLUPS",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(rec["ms_per_step"], 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": DTYPE_NAME[w["dtype"]],
        "data": "synthetic (lid-driven cavity from rest)",
        "config": {"workload": args.workload, "lattice": f"D{3 if q == 19 else 2}Q{q}",
                   "edge": n, "cells": cells, "re": w["re"], "tau": round(rec["tau"], 6),
                   "lid_u": w["u"], "sensor_every": w["sensor_every"], "block": w["block"],
                   "blocks": nb, "flag_rule": w["rule"], "flag_param": param,
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "timing": (f"{rec['repeats']} repeats of {args.steps} steps (>= {args.min_time} s "
                              "of device time), CUDA events per repeat, median per-step time"),
                   "l2": (f"population buffers {2 * nbytes / 1e9:.2f} GB > 129 MB L2, no flush"
                          if 2 * nbytes > 129e6 else "working set fits L2 (launch-bound case)")},
        "repeats": rec["repeats"],
        "ms_per_step_min_max": [round(x, 5) for x in rec["ms_per_step_min_max"]],
        "roofline": rec["roofline"],
        "e2e": e2e,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
    }
    if (ws == 1 and not args.no_mixed and args.workload == DEFAULT_WORKLOAD
            and args.edge is None and args.kernel == "auto"):
        out["mixed"] = run_mixed(args, ws, uuid)
    return out


# ------------------------------------------------------------------------------- oracle arm
def oracle_sample(w, n_edge, steps, rng_note=""):
    """Time `steps` oracle steps of the workload's cavity on an n_edge lattice (sensor + block max +
    flags every sensor step).  Returns (MLUPS, seconds, threads)."""
    import oracle as O

    q = w["q"]
    nz = n_edge if q == 19 else 1
    o = O.Oracle(q, n_edge, n_edge, nz, tau_of(w), lid=(w["u"], 0.0, 0.0))
    f = o.rest()
    t0 = time.perf_counter()
    for k in range(steps):
        sensor = (k + 1) % w["sensor_every"] == 0
        f, K, _, _ = o.step(f, sensor=sensor)
        if sensor:
            m = O.block_max(K, w["block"])
            if w["rule"] == "top":
                O.flags_top(m, w["param"])
            else:
                O.flags_threshold(m, threshold_of(w))
    dt = time.perf_counter() - t0
    cells = n_edge ** (3 if q == 19 else 2)
    return cells * steps / dt / 1e6, dt, O.threads()


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform

    return platform.machine()


def cpu_baseline_block(w):
    """The oracle on the host cores on a bounded sample of the full workload (all cores), plus a
    single-thread sample on a smaller cube of the same cavity."""
    import oracle as O

    n = w["n"]
    cells = cells_of(w)
    # calibrate on a couple of steps, then size the sample to ~15 s
    rate, _, _ = oracle_sample(w, min(n, 64 if w["q"] == 19 else 128), 2)
    steps = max(2, min(200, int(15.0 * rate * 1e6 / cells)))
    mlups, dt, threads = oracle_sample(w, n, steps)
    prev = O.set_threads(1)
    try:
        edge = min(n, 64 if w["q"] == 19 else 256)
        one, dt1, _ = oracle_sample(w, edge, 4)
    finally:
        O.set_threads(prev)
    dim = 3 if w["q"] == 19 else 2
    return {"value": round(mlups, 3), "unit": "MLUPS", "cores": threads, "kind": "oracle",
            "sample": f"{steps} steps of the full {n}^{dim} lattice from rest, "
                      f"FP64, sensor+block max+flags every sensor step ({dt:.1f} s)",
            "single_thread": {"value": round(one, 3), "unit": "MLUPS",
                              "sample": f"4 steps of a {edge}^{dim} cube ({dt1:.1f} s)"},
            "cpu": cpu_model()}


def run_reference(args, w):
    cells_full = cells_of(w)
    rate, _, _ = oracle_sample(w, 48 if w["q"] == 19 else 96, 2)
    budget_s = 90.0
    total_steps = args.steps + args.warmup
    target_cells = rate * 1e6 * budget_s / max(total_steps, 1)
    dim = 3 if w["q"] == 19 else 2
    edge = int(max(8, min(w["n"], target_cells ** (1.0 / dim))))
    if args.warmup:
        oracle_sample(w, edge, args.warmup)
    mlups, dt, threads = oracle_sample(w, edge, args.steps)
    sample = (f"each step: one FP64 oracle step of a {edge}^{dim} cavity with the workload's tau and "
              f"lid (full lattice {w['n']}^{dim} = {cells_full} cells), sensor + block max + flags")
    return {
        "metric": "fused stream-collide+sensor MLUPS", "value": round(mlups, 3), "unit": "MLUPS",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3 / max(args.steps, 1), 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample": sample},
        "impl": "reference",
        "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--min-time", type=float, default=MIN_TIMED_S,
                    help="device seconds the timed loop accumulates (repeats of --steps steps); "
                         "a shorter time is for profiling captures only")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the mixed-precision row (512^3 FP32 / FP16 / BF16 storage and the "
                         "error check) that the default workload's line carries")
    ap.add_argument("--kernel", default="auto", choices=["auto", "cell", "pair", "tma", "tma_pair"],
                    help="fused step kernel (default: the library's automatic choice)")
    ap.add_argument("--fusion", default="auto", choices=["auto", "separate", "fused", "brick"],
                    help="multi-level workload: the finest level's restriction as a separate "
                         "kernel or fused into its second sub-step (default: the library's)")
    ap.add_argument("--schedule", default="auto",
                    choices=["auto", "graph", "persistent", "persistent_brick", "persistent_lean"],
                    help="multi-level workload: a cycle as a graph of separate launches or one "
                         "persistent launch (default: timed at mesh build)")
    ap.add_argument("--step-form", default="auto",
                    choices=["auto", "flat", "tiled", "select", "pair"],
                    help="multi-level workload: force one form of the level step kernel on the "
                         "levels it applies to (default: timed per level at mesh build)")
    ap.add_argument("--edge", type=int, default=None,
                    help="run the workload on a lattice of this edge instead (small profiling "
                         "captures); the JSON line then names the edge in its config")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    w = dict(WORKLOADS[args.workload])
    if args.edge is not None:
        if args.edge < 8 or (w["rule"] == "blocks" and (args.edge % w["block"] or
                                                         128 % (args.edge // w["block"]))):
            ap.error("--edge must be >= 8 (multi-level: a multiple of the block edge whose block "
                     "count divides 128)")
        w["n"] = args.edge
    ws, rank, local = dist_env()

    if args.impl == "reference":
        if rank == 0:
            if w["rule"] in ("blocks", "learned", "regrid"):
                print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the "
                                  "uniform-lattice workloads only"}), flush=True)
            else:
                print(json.dumps(run_reference(args, w)), flush=True)
        return

    if ws > 1:
        import torch
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if w["rule"] in ("blocks", "learned", "regrid"):
        runner = {"blocks": run_blocks, "learned": run_learned, "regrid": run_regrid}[w["rule"]]
        out = runner(args, w, ws, rank, local)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    out = run_ours(args, w, ws, rank, local)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_block(w)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
