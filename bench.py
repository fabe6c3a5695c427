#!/usr/bin/env python3
"""Training throughput of the per-object NeRF step (RO-MAP Sec. V) on GB300.

One step = one forward + loss + backward + Adam pass of every object of the
workload (ray draw, box sampling, hash encoding, MLP, compositing, Eq. 7-11
losses, adjoints, hash-gradient scatter, Adam), run through the C ABI of
libromap.  The default workload is the uneven batched configuration: 32
objects whose rays per step are log-uniform in 256..16384, 128 candidate
samples per ray culled by a 64^3 occupancy bitgrid, hash grid L=16, F=2,
T=2^19, resolutions 16..512, each object seen in 3 frames of 640x480; the
batched mixed-precision step is timed against the plain per-object FP32
path, and the two are compared at the same final loss over several seeds
(the FP32 side in its bit-reproducible deterministic mode).

Prints one JSON line (rank 0).  Under torchrun the 32 objects are placed on
the ranks by LPT bin-packing (no collective on the data path).
--impl reference times the CPU oracle (plain FP64 C) on a bounded sample of
the same workload.
"""
import argparse
import ctypes as C
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2304_05735_gb300.sharding import max_over_ranks, sum_over_ranks  # noqa: E402

METRIC = "train samples/s (fwd+bwd+Adam), batched mixed vs plain fp32, at oracle-matched loss"
WORKLOAD_KEY = "multi8"  # the chosen workload's key (set in main)
WORKLOADS = {
    # 8 objects of equal batch size (weak scaling under torchrun: every rank trains 8 objects)
    "multi8": dict(
        name="multi-object training: 8 objects x 4096 rays x 64 samples per step, hash grid L=16 F=2 T=2^16 "
             "(16->512), MLP 32-64-16 / 18-64-64-3, 30 frames of 320x240 per object",
        objects=8, rays_per_object=4096, samples_per_ray=64, levels=16, features=2, log2_table=16,
        base_resolution=16, max_resolution=512, frames=30, width=320, height=240, focal=320.0, occupancy=None,
        seed0=1, scaling="weak",
        l2="inputs larger than L2: per step 219 MB of parameters, gradients and Adam moments plus 0.4 GB of ray "
           "pools (L2 129 MB)"),
    # uneven batches with occupancy culling (the objects are placed on ranks by LPT bin-packing: strong scaling)
    "uneven32": dict(
        name="uneven batched training: 32 objects, rays per object per step log-uniform in 256..16384 (seeded, "
             "fixed per object), 128 candidate samples per ray culled by a 64^3 occupancy bitgrid (shape dilated "
             "by 2 cells plus 5% random cells), hash grid L=16 F=2 T=2^19 (16->512), 3 frames of 640x480 per object",
        objects=32, rays_per_object=(256, 16384), samples_per_ray=128, levels=16, features=2, log2_table=19,
        base_resolution=16, max_resolution=512, frames=3, width=640, height=480, focal=640.0,
        occupancy=dict(dilate=2, p=0.05), seed0=40, scaling="strong",
        l2="inputs larger than L2: per step 6.1 GB of parameters, gradients, Adam moments and FP16 tables "
           "(L2 129 MB)"),
    # streaming mapping: objects appear along a camera path; per frame, Eq. 5 decides which observations extend a
    # pool (300 more iterations each), then a 40 ms budget of batched steps trains the objects that owe steps
    "stream96": dict(
        name="streaming mapping: 96 objects in a 24 m x 24 m room seen along a 600-frame figure-eight at 25 Hz "
             "(640x480, f=525); an object is created when its projected box first exceeds 16 px; Eq. 5 (25 deg) "
             "gates each observation's detection-box rays into its pool and grants 300 iterations; 40 ms budget "
             "of batched steps per frame; 4096 rays x 32 samples per object step; hash grid L=16 F=2 T=2^19",
        objects=96, frames=600, rate_hz=25.0, budget_ms=40.0, min_box_px=16, alpha_deg=25.0, iterations=300,
        rays_per_object=4096, samples_per_ray=32, levels=16, features=2, log2_table=19, base_resolution=16,
        max_resolution=512, width=640, height=480, focal=525.0, occupancy=None, seed0=1000, scaling="strong",
        l2="per step up to 190 MB of parameters, moments and tables per trained object (L2 129 MB)"),
    # Table 4 of the paper: iteration time of one object at 4096 rays x 32 samples as the hash table grows
    "table4": dict(
        name="per-object iteration time vs hash table size: 1 object, 4096 rays x 32 samples per step, L=16 F=2, "
             "resolutions 16->2048, T = 2^14, 2^16, 2^18, 2^20 (the paper's Table 4 sizes), 30 frames of 320x240",
        objects=1, rays_per_object=4096, samples_per_ray=32, levels=16, features=2, log2_table=16,
        log2_tables=(14, 16, 18, 20), base_resolution=16, max_resolution=2048, frames=30, width=320, height=240,
        focal=320.0, occupancy=None, seed0=1, scaling="weak",
        l2="per step 2 to 400 MB of parameters, moments and tables (L2 129 MB)",
        paper_ms={14: 0.658, 16: 0.706, 18: 0.921, 20: 1.495}, paper_layers_ms={2: 0.862, 3: 1.052}),
}
WORKLOAD = WORKLOADS["multi8"]
# FP32 SIMT peak of the GB300: 152 SMs x 128 FP32 lanes x 2 FLOP per FMA x 2070 MHz maximum SM clock.
FP32_SIMT_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# Algorithmic work per live sample (real multiply-adds of the five layers, no padding):
#   forward MLP 8512 MAC; backward input gradients 8320 MAC (the direction inputs need none);
#   weight gradients 8512 MAC; the backward kernel recomputes the forward.
MAC_FWD, MAC_DX, MAC_DW = 8512, 8320, 8512
PHASE_KERNEL = ("k_ray_setup + k_scan + k_write_samples", "k_tile_mlp<forward>", "k_composite<loss>",
                "k_tile_mlp<backward>", "k_adam + k_advance_step")
# the mixed-precision path: the tile plan, then one fused kernel for the forward, compositing and backward
PHASE_KERNEL_MIXED = ("k_ray_setup + k_plan_patterns + k_scan + k_plan_rays", "fused into k_tile_tc",
                      "fused into k_tile_tc", "k_tile_tc", "k_adam + k_advance_step")
TC_KERNEL = "k_tile_tc (fused: samples, FP16 gather, BF16 tcgen05 MLP fwd+bwd, Eq. 6-11, scatter)"
WS_KERNEL = "k_tile_ws (warp-specialized variant of the fused kernel)"
TC_TRAFFIC_KEY = "k_tile_tc"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--precision", choices=("fp32", "mixed", "fp8", "fp16"), default="mixed")
    ap.add_argument("--workload", choices=tuple(WORKLOADS), default="uneven32")
    ap.add_argument("--loss-steps", type=int, default=500)
    ap.add_argument("--loss-seeds", type=int, default=3,
                    help="training runs per precision for the loss comparison (object seeds shifted per run)")
    ap.add_argument("--objects", type=int, default=None,
                    help="train only the workload's first N objects (a smaller case of the same kind, e.g. for ncu)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    return ap.parse_args()


def config_keys(w):
    return {k: v for k, v in w.items() if k not in ("name", "scaling", "seed0")}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-i", str(gpu_index), "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.p = None

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [ln.strip().split(", ") for ln in self.f if ln.strip()]
        self.f.close()
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
DTYPES = {"mixed": "bf16 (MLP GEMM operands; FP16 table copy; FP32 accumulation, scan, loss, Adam)",
          "fp16": "fp16 (MLP GEMM operands, gradient operands scaled by the batch size; FP16 table copy; FP32 "
                  "accumulation, scan, loss, Adam)",
          "fp8": "fp8 e4m3 hidden 64x64 GEMM, bf16 other GEMMs (FP16 table copy; FP32 accumulation, scan, loss, "
                 "Adam)"}
KERNEL_SOURCES = {
    "fp32": ("kernels_tile.cu", "device_common.cuh", "romap_internal.cuh"),
    "mixed": ("tc_tile_kernel.cuh", "kernels_tc.cu", "kernels_tc1.cu", "tc_common.cuh", "device_common.cuh",
              "romap_internal.cuh"),
    "fp8": ("tc_tile_kernel.cuh", "kernels_tc.cu", "tc_common.cuh", "device_common.cuh", "romap_internal.cuh"),
    "fp16": ("tc_tile_kernel.cuh", "kernels_tc16.cu", "tc_common.cuh", "device_common.cuh", "romap_internal.cuh"),
}


def kernel_source_hash(precision):
    """Hash of the code (comments and blank lines left out) of the sources the dominant kernel of `precision` is
    built from (profiles/dram_traffic.json keys)."""
    h = hashlib.sha256()
    for name in KERNEL_SOURCES[precision]:
        with open(os.path.join(ROOT, "paper_2304_05735_gb300", "csrc", name), encoding="utf-8") as f:
            for line in f:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic(kernel, precision):
    """Per-launch DRAM bytes of `kernel` on this workload from the committed ncu summary, if the kernel source is
    unchanged."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        e = d.get(f"{kernel}|{precision}|{workload_id()}")
        if e and e.get("source_hash") == kernel_source_hash(precision):
            return e.get("bytes_per_launch_full_workload")
    except (OSError, ValueError):
        return None
    return None


class Item:
    """One object of the workload on this rank: its scene, rays per step and occupancy bitgrid (or None)."""

    def __init__(self, scene, rays, occ):
        self.scene, self.rays, self.occ = scene, rays, occ


def workload_rays(w):
    if isinstance(w["rays_per_object"], int):
        return [w["rays_per_object"]] * w["objects"]
    import numpy as np

    lo, hi = w["rays_per_object"]
    rng = np.random.default_rng(7)
    return [int(r) for r in np.exp(rng.uniform(np.log(lo), np.log(hi), w["objects"]))]


def build_items(w, rank, world):
    """This rank's objects.  Equal batches: every rank trains its own w["objects"] objects (seeds shifted by rank).
    Uneven batches: the w["objects"] objects are placed on the ranks by LPT bin-packing on rays x samples."""
    from paper_2304_05735_gb300 import synth
    from paper_2304_05735_gb300.sharding import lpt_partition

    rays = workload_rays(w)
    if w["scaling"] == "weak":
        seeds = [w["seed0"] + w["objects"] * rank + k for k in range(w["objects"])]
        mine = list(range(w["objects"]))
    else:
        mine = lpt_partition([r * w["samples_per_ray"] for r in rays], world)[rank]
        seeds = [w["seed0"] + k for k in mine]
    items = []
    for k, seed in zip(mine, seeds):
        sc = synth.multi_object_scene(1, seed0=seed, n_frames=w["frames"], W=w["width"], H=w["height"],
                                      f=w["focal"])[0]
        occ = None
        if w["occupancy"]:
            occ = synth.occupancy_bits(sc.shape, sc.half, dilate=w["occupancy"]["dilate"], p=w["occupancy"]["p"],
                                       seed=sc.seed)
        items.append(Item(sc, rays[k], occ))
    return items


def make_ctx(R, torch, precision, single_net=False, hidden_layers=1, deterministic=False, per_object=False):
    """A context for the current workload; single_net selects the position-only single-network model of Sec. V
    (hidden_layers hidden layers of 64, Table 4) instead of the density + colour nets; deterministic the
    bit-reproducible FP32 mode; per_object one launch sequence per object (the plain per-object path)."""
    w = WORKLOAD
    rc = R.make_config(n_levels=w["levels"], log2_table_size=w["log2_table"], base_resolution=w["base_resolution"],
                       growth=0.0, max_resolution=w["max_resolution"], n_samples=w["samples_per_ray"],
                       rays_per_step=4096, bg_random=True, single_net=single_net, dir_dims=0 if single_net else 3,
                       hidden_layers=hidden_layers,
                       precision={"mixed": R.ROMAP_PREC_MIXED_BF16, "fp8": R.ROMAP_PREC_MIXED_FP8,
                                  "fp16": R.ROMAP_PREC_MIXED_FP16}.get(
                           precision, R.ROMAP_PREC_FP32),
                       max_objects=2 * w["objects"], deterministic=deterministic, per_object=per_object)
    h = C.c_void_p()
    R.check(R.romap_init(C.byref(rc), C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(h)), "romap_init")
    return rc, h


def add_objects(R, h, items, seed_offset=0):
    """Creates the workload's objects; seed_offset shifts every object's random stream (initial parameters, ray
    draws, jitter, background colours) for repeated training runs on the same scenes."""
    import numpy as np

    ids = []
    for it in items:
        sc = it.scene
        oid = C.c_int32()
        d = R.object_desc(t=tuple(sc.t), yaw=sc.yaw, half_size=tuple(sc.half), seed=sc.seed + seed_offset,
                          rays_per_step=it.rays)
        R.check(R.romap_create_object(h, C.byref(d), C.byref(oid)), "romap_create_object")
        if it.occ is not None:
            bits = np.ascontiguousarray(it.occ)
            R.check(R.romap_set_occupancy(h, oid.value, bits.ctypes.data, 0), "romap_set_occupancy")
        p = sc.pool
        rays = R.romap_rays(p["origin"].ctypes.data, p["dir"].ctypes.data, p["rgb"].ctypes.data,
                            p["depth"].ctypes.data, p["cls"].ctypes.data)
        R.check(R.romap_add_rays(h, oid.value, C.byref(rays), p["cls"].size, 0), "romap_add_rays")
        ids.append(oid.value)
    return ids


def per_object_cmp(obj_final):
    """Per object and seed, the relative difference of the mixed run's final loss from the FP32 run's: median,
    quartiles and the fraction within 1e-3."""
    import numpy as np

    if not obj_final["fp32"] or not obj_final["mixed"]:
        return None
    f = np.concatenate(obj_final["fp32"]).astype(np.float64)
    m = np.concatenate(obj_final["mixed"]).astype(np.float64)
    d = (m - f) / f
    return {"pairs": int(d.size), "median": float(np.median(d)), "q25": float(np.quantile(d, 0.25)),
            "q75": float(np.quantile(d, 0.75)), "within_1e-3": float(np.mean(np.abs(d) <= 1e-3))}


def curve_steps(k):
    """Step indices of the reported loss curve: the first step, then every tenth of the run."""
    return sorted({0, *range(max(1, k // 10) - 1, k, max(1, k // 10))})


def psnr_rays(items, per_object=4096, seed=123):
    """A fixed sample of each object's training rays (object and background classes) for the PSNR of a trained model."""
    import numpy as np

    rng = np.random.default_rng(seed)
    out = []
    for it in items:
        p = it.scene.pool
        keep = np.nonzero(p["cls"] <= 1)[0]
        sel = np.sort(rng.choice(keep, min(per_object, keep.size), replace=False))
        out.append({k: np.ascontiguousarray(p[k][sel]) for k in ("origin", "dir", "rgb", "cls")})
    return out


def trained_psnr(R, h, ids, evalset, bg=(0.5, 0.5, 0.5)):
    """Training-view PSNR of each trained object: its rays rendered by romap_render (FP32 forward from the FP32
    parameters, midpoint samples) over a grey background, against the target colour (object rays) or that
    background (background rays)."""
    import numpy as np

    bgc = np.array(bg, np.float32)
    vals = []
    for oid, e in zip(ids, evalset):
        m = e["cls"].size
        col = np.zeros((m, 3), np.float32)
        R.check(R.romap_render(h, oid, e["origin"].ctypes.data, e["dir"].ctypes.data, m, bgc.ctypes.data,
                               col.ctypes.data, None, None, 0), "romap_render")
        tgt = np.where(e["cls"][:, None] == 0, e["rgb"], bgc[None, :])
        mse = float(((col.astype(np.float64) - tgt) ** 2).mean())
        vals.append(-10.0 * np.log10(max(mse, 1e-12)))
    return {"mean": float(np.mean(vals)), "median": float(np.median(vals)), "min": float(np.min(vals))}


def timed(torch, fn, world, dist):
    """Runs fn() between barrier + synchronize brackets; returns (device ms on the current stream, max over ranks)."""
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    fn()
    e.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = s.elapsed_time(e)
    return max_over_ranks(ms, dist if world > 1 else None, "cuda")


def allsum(torch, dist, world, x):
    return sum_over_ranks(x, dist if world > 1 else None, "cuda") if world > 1 else x


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_2304_05735_gb300 import romap as R
    from paper_2304_05735_gb300 import synth

    R.lib()
    w = WORKLOAD
    items = build_items(w, rank, world)
    n = len(items)
    main_prec = args.precision

    # ---- loss comparison (untimed): batched mixed vs plain FP32 at the same final loss ----------------------------
    # args.loss_seeds runs per precision, run k with every object's seed shifted by 1000 k (initial parameters, ray
    # draws, jitter, background colours); the FP32 side runs in the deterministic mode (fixed-point accumulation), so
    # a run is reproducible bit for bit and the spread between runs is the spread between seeds alone.  The final
    # loss of a run is its mean per-step loss over the last K/4 steps, averaged over the objects.
    runs = {"fp32": [], "mixed": []}
    obj_final = {"fp32": [], "mixed": []}  # per run: each object's mean loss over the last K/4 steps
    psnr = {}
    fp32_repeat_identical = None
    # control: seed 0 once more in FP32 with ordinary (order-dependent) atomic accumulation, against the
    # deterministic FP32 run of the same seed: how far training alone moves the final losses when only the rounding
    # order of the sums changes
    fp32_nondet = None
    if not args.no_plain:
        evalset = psnr_rays(items)
        for k in range(args.loss_seeds):
            for prec in ("fp32", "mixed") + (("fp32_repeat", "fp32_nondet") if k == 0 else ()):
                det = prec not in ("mixed", "fp32_nondet")
                rc, h = make_ctx(R, torch, main_prec if prec == "mixed" else "fp32", deterministic=det)
                ids = add_objects(R, h, items, seed_offset=1000 * k)
                idarr = (C.c_int32 * n)(*ids)
                ls = np.zeros((args.loss_steps, n), np.float32)
                for j in range(args.loss_steps):
                    R.check(R.romap_train_step(h, idarr, n, 1, ls[j].ctypes.data))
                if prec == "fp32_repeat":
                    fp32_repeat_identical = bool(np.array_equal(ls.mean(axis=1), runs["fp32"][0]))
                elif prec == "fp32_nondet":
                    tail_nd = max(1, args.loss_steps // 4)
                    fp32_nondet = {"run": ls.mean(axis=1), "obj": ls[-tail_nd:].mean(axis=0)}
                else:
                    runs[prec].append(ls.mean(axis=1))
                    obj_final[prec].append(ls[-max(1, args.loss_steps // 4):].mean(axis=0))
                    if k == 0:
                        psnr[prec] = trained_psnr(R, h, ids, evalset)
                R.check(R.romap_destroy(h))

    # ---- the timed batched step -------------------------------------------------------------------------------------
    rc, h = make_ctx(R, torch, main_prec)
    ids = add_objects(R, h, items)
    idarr = (C.c_int32 * len(ids))(*ids)
    R.check(R.romap_train_step(h, idarr, n, max(args.warmup, 3), None))
    torch.cuda.synchronize()
    R.check(R.romap_reset_stats(h))
    gpu_index = (os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[local]
                 if os.environ.get("CUDA_VISIBLE_DEVICES") else str(local))
    sampler = ClockSampler(gpu_index)
    time.sleep(0.3)

    def steps():  # one call of args.steps steps (as the comparison arms): the library replays captured CUDA graphs,
        # and each step's sampling overlaps the previous step's Adam update
        R.check(R.romap_train_step(h, idarr, n, args.steps, None))

    ms = timed(torch, steps, world, dist)
    clocks = sampler.stop()
    st = R.romap_stats()
    R.check(R.romap_get_stats(h, C.byref(st)))
    live = allsum(torch, dist, world, st.live_samples)
    value = live / (ms / 1e3)
    live_per_step = st.live_samples / args.steps  # this rank
    launches = st.kernel_launches
    autotune = None
    if main_prec != "fp32":
        chosen = C.c_int32()
        tms = (C.c_float * 16)()
        names = C.create_string_buffer(2048)
        R.check(R.romap_autotune_report(h, C.byref(chosen), tms, 16, names, 2048))
        cands = names.value.decode().split(";")
        autotune = {"chosen": cands[chosen.value] if chosen.value >= 0 else None,
                    "ms_per_launch": {c: float(tms[i]) for i, c in enumerate(cands)}}
    # per-phase device time: the same steps again with CUDA events around every phase (eager launches)
    k_prof = max(3, min(args.steps, 100))
    R.check(R.romap_reset_stats(h))
    R.check(R.romap_set_profiling(h, 1))
    R.check(R.romap_train_step(h, idarr, n, k_prof, None))
    phase_ms = (C.c_double * R.ROMAP_N_PHASES)()
    phase_n = (C.c_int64 * R.ROMAP_N_PHASES)()
    R.check(R.romap_phase_times(h, phase_ms, phase_n))
    R.check(R.romap_set_profiling(h, 0))
    for i in range(R.ROMAP_N_PHASES):
        phase_ms[i] *= args.steps / k_prof  # per-step averages below divide by args.steps

    # phases and the roofline of the dominant kernel
    phases = {}
    labels = PHASE_KERNEL if main_prec == "fp32" else PHASE_KERNEL_MIXED
    for i, name in enumerate(R.PHASES):
        phases[name] = {"kernel": labels[i], "ms_per_step": phase_ms[i] / max(1, args.steps),
                        "share": phase_ms[i] / max(1e-9, sum(phase_ms))}
    bwd_ms = phase_ms[3] / args.steps
    fwd_ms = phase_ms[1] / args.steps
    mixed = main_prec != "fp32"
    peaks = {}
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        peaks = json.load(open(peaks_path))
    flop_bwd = 2.0 * (MAC_FWD + MAC_DX + MAC_DW) * live_per_step
    flop_fwd = 2.0 * MAC_FWD * live_per_step
    if mixed:
        phases["mlp_backward_scatter"]["kernel"] = TC_KERNEL
    if bwd_ms > 0:
        phases["mlp_backward_scatter"]["achieved_tflops"] = flop_bwd / (bwd_ms / 1e3) / 1e12
    if fwd_ms > 0:
        phases["mlp_forward"]["achieved_tflops"] = flop_fwd / (fwd_ms / 1e3) / 1e12
    n_params = int(R.param_layout(rc).n_params)
    adam_bytes = (32.0 + (2.0 if mixed else 0.0)) * n_params * n
    hbm = peaks.get("hbm_gbs") or 6800.0
    if phase_ms[4] > 0:
        # dense-equivalent rate: Adam skips 256-parameter chunks that never received a gradient (their update is
        # exactly zero) and reads only their gradient, so this counts bytes a dense Adam would move
        phases["adam"]["achieved_gbs"] = adam_bytes / (phase_ms[4] / args.steps / 1e3) / 1e9
        phases["adam"]["frac_of_hbm"] = phases["adam"]["achieved_gbs"] / hbm
        phases["adam"]["note"] = ("dense-equivalent: 34 B per parameter of every object; never-touched chunks are "
                                  "skipped after a 4 B gradient read")
    dominant = max(range(R.ROMAP_N_PHASES), key=lambda i: phase_ms[i])
    if dominant == 3 and mixed:
        # the fused kernel's algorithmic traffic: per live sample the FP16 gather of 8 corners x L levels x F
        # features and the FP32 scatter-add of as many gradients; its MLP work is reported against the tensor peak
        # beside it
        lvl = w["levels"]
        bytes_per_sample = 8 * lvl * 2 * 2 + 8 * lvl * 2 * 4
        achieved = bytes_per_sample * live_per_step / (bwd_ms / 1e3) / 1e9
        tpeak = peaks.get("bf16_tflops_sustained") or 1700.0
        tach = flop_bwd / (bwd_ms / 1e3) / 1e12
        ws = bool(autotune and autotune["chosen"] and autotune["chosen"].startswith("warp-specialized"))
        kname = WS_KERNEL if ws else TC_KERNEL.replace("BF16", {"fp16": "FP16", "fp8": "FP8/BF16"}.get(main_prec,
                                                                                                        "BF16"))
        if autotune and autotune["chosen"]:
            kname += f"; autotuned: {autotune['chosen']}"
        # the roof that binds: the SMs' scattered-request rate into L2, measured live (romap_measure_request_rates:
        # one 4-byte load and one 8-byte reduction per step, every lane its own random address in L2-resident
        # buffers); per live sample the kernel needs 8 L gathers and 8 L scatter-adds, i.e. 8 L such pairs
        rates = (C.c_double * 3)()
        R.check(R.romap_measure_request_rates(C.c_void_p(torch.cuda.current_stream().cuda_stream), rates),
                "romap_measure_request_rates")
        pair_bytes = 2 * 2 + 2 * 4  # FP16 feature pair + FP32 gradient pair
        l2_peak = rates[2] * pair_bytes / 1e9
        roofline = {"bound": "l2", "kernel": kname, "achieved": achieved, "peak": l2_peak, "unit": "GB/s",
                    "frac": achieved / l2_peak,
                    "traffic": profiled_traffic(TC_TRAFFIC_KEY, main_prec) if not ws else None,
                    "peak_source": "measured live by romap_measure_request_rates: "
                                   f"{rates[2]:.4g} scattered load + red.global.add.v2.f32 pairs/s x {pair_bytes} B "
                                   f"(loads alone {rates[0]:.4g}/s, reductions alone {rates[1]:.4g}/s)",
                    "work_per_unit": f"{bytes_per_sample} B per live sample (FP16 gather {8 * lvl * 4} B + FP32 "
                                     f"scatter-add {8 * lvl * 8} B) = {8 * lvl} load/reduction pairs",
                    "units_per_launch": live_per_step, "ms_per_launch": bwd_ms,
                    "hbm": {"achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                            "note": "the same logical bytes against the HBM copy bandwidth; the tables stay in L2, "
                                    "see traffic for the DRAM bytes actually moved",
                            "peak_source": "measured HBM copy (MEASURED_PEAKS.json)" if peaks else "fallback"},
                    "tensor": {"achieved": tach, "peak": tpeak, "unit": "TFLOP/s", "frac": tach / tpeak,
                               "work_per_unit": f"{2 * (MAC_FWD + MAC_DX + MAC_DW)} FLOP per live sample (BF16 MMA)",
                               "peak_source": "measured bf16 dense, sustained (MEASURED_PEAKS.json)"}}
    elif dominant in (1, 3):
        flop = flop_bwd if dominant == 3 else flop_fwd
        kms = bwd_ms if dominant == 3 else fwd_ms
        achieved = flop / (kms / 1e3) / 1e12
        roofline = {"bound": "alu", "kernel": PHASE_KERNEL[dominant], "achieved": achieved,
                    "peak": FP32_SIMT_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_SIMT_TFLOPS,
                    "traffic": profiled_traffic(PHASE_KERNEL[dominant], main_prec),
                    "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz (FP32 SIMT FMA)",
                    "work_per_unit": f"{2 * (MAC_FWD + MAC_DX + MAC_DW) if dominant == 3 else 2 * MAC_FWD} "
                                     "FLOP per live sample",
                    "units_per_launch": live_per_step, "ms_per_launch": kms}
    else:
        ach = phases["adam"].get("achieved_gbs") if dominant == 4 else None
        roofline = {"bound": "hbm", "kernel": PHASE_KERNEL[dominant], "achieved": ach, "peak": hbm,
                    "unit": "GB/s", "frac": (ach / hbm) if ach else None, "traffic": None}

    # ---- end to end through the C ABI with host buffers ---------------------------------------------------------------
    # each step replaces every object's rays with a fresh batch of its rays per step from pinned host memory, trains,
    # and reads the losses back
    e2e = None
    if not args.no_e2e:
        rng = np.random.default_rng(100 + rank)
        k_e2e = max(3, min(args.steps, 50))
        # per step, every object's new rays in one page-locked structure of arrays (objects concatenated), handed
        # to the library by one romap_add_rays_multi call (one keyframe's observations of all objects)
        counts = (C.c_int64 * n)(*[it.rays for it in items])
        batches = []
        for _ in range(k_e2e + 2):
            arrs = {}
            sels = [rng.integers(0, it.scene.pool["cls"].size, it.rays) for it in items]
            for k in ("origin", "dir", "rgb", "depth", "cls"):
                a = np.concatenate([it.scene.pool[k][sel] for it, sel in zip(items, sels)])
                t = torch.empty(a.shape, dtype=torch.uint8 if k == "cls" else torch.float32, pin_memory=True)
                t.numpy()[...] = a
                arrs[k] = t
            batches.append(arrs)
        h2d = sum(t.numel() * t.element_size() for t in batches[0].values())
        # the step's losses come back asynchronously into one of two page-locked slots; the host reads step k - 1's
        # losses after it has enqueued step k, so the device never waits for the host between steps
        outs = [torch.zeros(n, dtype=torch.float32, pin_memory=True) for _ in range(2)]
        losses = []

        def e2e_step(arrs, out):
            rays = R.romap_rays(arrs["origin"].data_ptr(), arrs["dir"].data_ptr(), arrs["rgb"].data_ptr(),
                                arrs["depth"].data_ptr(), arrs["cls"].data_ptr())
            R.check(R.romap_add_rays_multi(h, idarr, counts, n, C.byref(rays), R.ROMAP_REPLACE | R.ROMAP_ASYNC_HOST),
                    "romap_add_rays_multi")
            R.check(R.romap_train_step_async(h, idarr, n, 1, C.c_void_p(out.data_ptr())), "romap_train_step_async")
            ev = torch.cuda.Event()
            ev.record()
            return ev

        def e2e_run(bs):
            prev = None
            for k, arrs in enumerate(bs):
                ev = e2e_step(arrs, outs[k % 2])
                if prev is not None:
                    prev.synchronize()
                    losses.append(outs[(k - 1) % 2].numpy().copy())
                prev = ev
            prev.synchronize()
            losses.append(outs[(len(bs) - 1) % 2].numpy().copy())

        e2e_run(batches[:2])
        R.check(R.romap_check_device_status(h), "romap_check_device_status")
        R.check(R.romap_reset_stats(h))
        losses.clear()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_run(batches[2:])
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        R.check(R.romap_check_device_status(h), "romap_check_device_status")
        assert len(losses) == k_e2e and all(np.isfinite(x).all() for x in losses)
        el = max_over_ranks(el, dist if world > 1 else None, "cuda")
        ste = R.romap_stats()
        R.check(R.romap_get_stats(h, C.byref(ste)))
        live_e = allsum(torch, dist, world, ste.live_samples)
        e2e = {"value": live_e / el, "unit": "samples/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(4 * n), "steps": k_e2e,
               "path": f"romap_add_rays_multi(REPLACE | ASYNC_HOST, pinned host, {n} objects) + "
                       f"romap_train_step_async (losses to pinned host, read one step later), wall clock"}

    # ---- mesh extraction of the trained objects (Table 3: marching cubes at 64^3) -----------------------------------
    mesh = None
    if rank == 0:
        iso = 5.0
        cap_v, cap_t = 1 << 21, 1 << 22
        dv = torch.empty((cap_v, 3), device="cuda")
        dtr = torch.empty((cap_t, 3), dtype=torch.int32, device="cuda")
        nv, nt = C.c_int64(), C.c_int64()
        for oid in ids[:1]:  # warm-up (case table upload, workspace)
            R.check(R.romap_extract_mesh(h, oid, iso, dv.data_ptr(), cap_v, dtr.data_ptr(), cap_t, C.byref(nv),
                                         C.byref(nt), R.ROMAP_DEVICE_PTR))
        torch.cuda.synchronize()
        tv, tt, times = [], [], []
        for oid in ids:
            t0 = time.perf_counter()
            R.check(R.romap_extract_mesh(h, oid, iso, dv.data_ptr(), cap_v, dtr.data_ptr(), cap_t, C.byref(nv),
                                         C.byref(nt), R.ROMAP_DEVICE_PTR))
            torch.cuda.synchronize()
            times.append((time.perf_counter() - t0) * 1e3)
            tv.append(nv.value)
            tt.append(nt.value)
        mesh = {"ms_per_object": float(np.mean(times)), "ms_max": float(np.max(times)), "iso_density": iso,
                "vertices_mean": float(np.mean(tv)), "triangles_mean": float(np.mean(tt)),
                "path": "romap_extract_mesh (64^3 cubes, device outputs), wall clock incl. its count read-back",
                "paper_ms_per_object": 2.84}
    R.check(R.romap_destroy(h))

    # ---- the comparison paths: batched FP32 and the plain per-object FP32 path -------------------------------------
    # the plain path trains each object with its own launch sequence (per_object: one CUDA graph per object, all
    # kept in the context's graph cache and replayed), and again with eager launches (no graphs)
    others = {}
    if not args.no_plain:
        k_cmp = max(5, min(args.steps, 100))
        for label, per_object, graphs, det in (("batched_fp32", False, True, False),
                                               ("plain_fp32_per_object", True, True, False),
                                               ("plain_fp32_per_object_eager", True, False, False),
                                               ("plain_fp32_per_object_deterministic", True, True, True)):
            rc2, h2 = make_ctx(R, torch, "fp32", per_object=per_object, deterministic=det)
            R.check(R.romap_set_graphs(h2, 1 if graphs else 0))
            ids2 = add_objects(R, h2, items)
            arr2 = (C.c_int32 * n)(*ids2)
            R.check(R.romap_train_step(h2, arr2, n, 3, None))
            R.check(R.romap_reset_stats(h2))

            def run_cmp():
                R.check(R.romap_train_step(h2, arr2, n, k_cmp, None))

            ms_c = timed(torch, run_cmp, world, dist)
            stc = R.romap_stats()
            R.check(R.romap_get_stats(h2, C.byref(stc)))
            live_c = allsum(torch, dist, world, stc.live_samples)
            others[label] = {"value": live_c / (ms_c / 1e3), "ms_per_step": ms_c / k_cmp, "steps": k_cmp,
                             "graph_captures": int(stc.graph_captures), "graph_replays": int(stc.graph_replays),
                             "path": ("one launch sequence per object" if per_object else "one batched launch sequence")
                                     + (", CUDA graphs replayed" if graphs else ", eager launches")
                                     + (", deterministic fixed-point accumulation" if det else "")}
            R.check(R.romap_destroy(h2))

    loss_cmp = None
    if runs["fp32"]:
        # "at oracle-matched loss", two-sided: the mean final loss of the mixed runs within 1e-3 (relative) of the mean
        # final loss of the deterministic FP32 runs over the same seeds; the paired per-seed differences and their
        # standard error say whether a gap is larger than the seed-to-seed spread
        tail = max(1, args.loss_steps // 4)
        fin = {p: np.array([float(c[-tail:].mean()) for c in runs[p]]) for p in runs}
        mf, mm = float(fin["fp32"].mean()), float(fin["mixed"].mean())
        paired = (fin["mixed"] - fin["fp32"]) / fin["fp32"]
        se = float(paired.std(ddof=1) / np.sqrt(paired.size)) if paired.size > 1 else None
        cf, cm = np.mean(runs["fp32"], axis=0), np.mean(runs["mixed"], axis=0)
        reach = np.nonzero(cm <= mf)[0]
        loss_cmp = {
            "steps": args.loss_steps, "seeds": args.loss_seeds, "mean_loss_last_steps": tail,
            "criterion": "two-sided: |mean mixed - mean FP32| <= 1e-3 x mean FP32, final loss = mean per-step loss of "
                         "the last K/4 steps; FP32 in the deterministic (bit-reproducible) mode; seeds shift every "
                         "object's random stream",
            "fp32": {"mean": mf, "std": float(fin["fp32"].std(ddof=1)) if paired.size > 1 else 0.0,
                     "runs": fin["fp32"].tolist()},
            "mixed": {"mean": mm, "std": float(fin["mixed"].std(ddof=1)) if paired.size > 1 else 0.0,
                      "runs": fin["mixed"].tolist()},
            "rel_diff": (mm - mf) / mf, "matched": bool(abs(mm - mf) <= 1e-3 * mf),
            "paired_rel_diff": paired.tolist(), "paired_rel_diff_se": se,
            # robust to the occasional seed whose mixed or FP32 run reaches a sharp loss drop many steps earlier
            "paired_rel_diff_median": float(np.median(paired)),
            # the same per object (every object of every seed): how a typical object's final loss compares
            "per_object": per_object_cmp(obj_final),
            "control_fp32_order": None if fp32_nondet is None else {
                "what": "seed 0: FP32 with order-dependent atomic sums vs the deterministic FP32 run (no precision "
                        "change, only the rounding order of the sums)",
                "rel_diff": float((fp32_nondet["run"][-tail:].mean() - runs["fp32"][0][-tail:].mean())
                                  / runs["fp32"][0][-tail:].mean()),
                "per_object": per_object_cmp({"fp32": [obj_final["fp32"][0]], "mixed": [fp32_nondet["obj"]]})},
            "within_two_se": bool(se is not None and abs(float(paired.mean())) <= 2.0 * se),
            "fp32_repeat_bit_identical": fp32_repeat_identical,
            "first_step_rel_diff": float(abs(cm[0] - cf[0]) / cf[0]),
            "mixed_steps_to_fp32_final_loss": int(reach[0] + 1) if reach.size else None,
            "curve": {"steps": [k + 1 for k in curve_steps(args.loss_steps)],
                      "fp32": [float(cf[k]) for k in curve_steps(args.loss_steps)],
                      "mixed": [float(cm[k]) for k in curve_steps(args.loss_steps)]},
            "psnr_db_after_k_steps": psnr}
        if mixed and others.get("plain_fp32_per_object") and reach.size:
            t_mixed = (reach[0] + 1) * ms / args.steps
            t_plain = args.loss_steps * others["plain_fp32_per_object"]["ms_per_step"]
            loss_cmp["time_to_fp32_final_loss_ms"] = {"mixed_batched": t_mixed, "plain_fp32_per_object": t_plain}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_all_cores(n_rays=4096)
        cpu["single_core"] = cpu_baseline(n_rays=4096, steps=1)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
               "scaling": w["scaling"], "vs_baseline": None,
               "dtype": DTYPES.get(main_prec, "f32"),
               "data": "synthetic (analytic shapes, seeded)",
               "config": {"workload": w["name"], **config_keys(w), "precision": main_prec, "path": "batched",
                          "objects_this_rank": n, "rays_per_step_this_rank": int(sum(it.rays for it in items)),
                          "parallelism": f"{world} rank(s), objects sharded, no collective"},
               "live_samples_per_step": live_per_step, "roofline": roofline, "phases": phases,
               "comparison": others, "loss_check": loss_cmp, "autotune": autotune, "e2e": e2e, "cpu_baseline": cpu,
               "mesh": mesh,
               "gpu_launches": int(launches), "clocks": clocks}
        if others.get("plain_fp32_per_object"):
            out["speedup_vs_plain_fp32_per_object"] = value / others["plain_fp32_per_object"]["value"]
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# the CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------
def _oracle_setup(n_rays, k=0):
    """Object k of the workload (seed seed0 + k, up to 4 frames, its occupancy bitgrid if the workload culls)."""
    import numpy as np

    from oracle import romap_oracle as O
    from paper_2304_05735_gb300 import synth

    w = WORKLOAD
    sc = synth.multi_object_scene(1, seed0=w["seed0"] + k, n_frames=min(4, w["frames"]), W=w["width"],
                                  H=w["height"], f=w["focal"])[0]
    occ = None
    if w["occupancy"]:
        occ = synth.occupancy_bits(sc.shape, sc.half, dilate=w["occupancy"]["dilate"], p=w["occupancy"]["p"],
                                   seed=sc.seed)
    oc = O.make_config(L=w["levels"], T=2 ** w["log2_table"], n_min=w["base_resolution"], growth=0.0,
                       n_max=w["max_resolution"], n_samples=w["samples_per_ray"], rays_per_step=n_rays,
                       bg_random=True)
    o, d = O.world_to_object(sc.pool["origin"], sc.pool["dir"], sc.t.astype(np.float32), sc.yaw)
    pool = dict(o=o, d=d, rgb=sc.pool["rgb"], depth=sc.pool["depth"], cls=sc.pool["cls"])
    p = O.init_params(oc, sc.seed)
    return O, oc, sc, pool, p, occ


def cpu_baseline(n_rays=4096, steps=1):
    import numpy as np

    O, oc, sc, pool, p, occ = _oracle_setup(n_rays)
    m, v = np.zeros_like(p), np.zeros_like(p)
    live = 0
    t0 = time.perf_counter()
    for s in range(1, steps + 1):
        r = O.train_step(oc, sc.half.astype(np.float32), sc.seed, s, pool, p, m, v, occ=occ, want_samples=True)
        p, m, v = r["params"], r["m"], r["v"]
        live += int(r["samples"][:, :, 5].sum())
    el = time.perf_counter() - t0
    return {"value": live / el, "unit": "samples/s", "cores": 1, "kind": "oracle",
            "sample": f"{steps} step(s) of 1 object x {n_rays} rays x {WORKLOAD['samples_per_ray']} samples at the "
                      f"workload's model size (FP64 C oracle, single thread), {live} live samples in {el:.1f} s"}


def _oracle_worker(workload, k, n_rays, barrier, queue):
    """One process of the all-cores baseline: one oracle step of object k, timed after every worker is ready."""
    global WORKLOAD
    import numpy as np

    WORKLOAD = WORKLOADS[workload]
    O, oc, sc, pool, p, occ = _oracle_setup(n_rays, k)
    m, v = np.zeros_like(p), np.zeros_like(p)
    barrier.wait(timeout=600)
    t0 = time.perf_counter()
    r = O.train_step(oc, sc.half.astype(np.float32), sc.seed, 1, pool, p, m, v, occ=occ, want_samples=True)
    t1 = time.perf_counter()
    queue.put((int(r["samples"][:, :, 5].sum()), t0, t1))


def cpu_baseline_all_cores(n_rays=4096, workers=None):
    """The oracle on every host core: one single-threaded process per core (started with spawn), each running one
    step of a different object of the workload; live samples of all processes / wall time from the first start to
    the last finish."""
    import multiprocessing as mp

    workers = workers or os.cpu_count() or 1
    name = WORKLOAD_KEY
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(workers), ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(name, k, n_rays, barrier, queue)) for k in range(workers)]
    for pr in procs:
        pr.start()
    res, deadline = [], time.time() + 900
    while len(res) < workers:  # a worker that dies ends the wait instead of leaving it blocked
        try:
            res.append(queue.get(timeout=5))
        except Exception:
            if time.time() > deadline or any(pr.exitcode not in (None, 0) for pr in procs):
                for pr in procs:
                    if pr.is_alive():
                        pr.terminate()
                raise RuntimeError("an oracle worker of the all-cores baseline failed")
    for pr in procs:
        pr.join()
    live = sum(r[0] for r in res)
    el = max(r[2] for r in res) - min(r[1] for r in res)
    return {"value": live / el, "unit": "samples/s", "cores": workers, "kind": "oracle",
            "sample": f"{workers} processes x 1 step of 1 object x {n_rays} rays x {WORKLOAD['samples_per_ray']} "
                      f"samples at the workload's model size (FP64 C oracle, one thread each, objects seed0 .. "
                      f"seed0 + {workers - 1}), {live} live samples in {el:.1f} s"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import numpy as np

    n_rays = 256
    O, oc, sc, pool, p, occ = _oracle_setup(n_rays)
    m, v = np.zeros_like(p), np.zeros_like(p)
    half = sc.half.astype(np.float32)
    step = 1
    for _ in range(args.warmup):
        r = O.train_step(oc, half, sc.seed, step, pool, p, m, v, occ=occ)
        p, m, v = r["params"], r["m"], r["v"]
        step += 1
    live = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = O.train_step(oc, half, sc.seed, step, pool, p, m, v, occ=occ, want_samples=True)
        p, m, v = r["params"], r["m"], r["v"]
        live += int(r["samples"][:, :, 5].sum())
        step += 1
    el = time.perf_counter() - t0
    value = live / el
    w = WORKLOAD
    sample = (f"each step: 1 object x {n_rays} rays x {w['samples_per_ray']} samples of the workload's model "
              f"(L={w['levels']}, T=2^{w['log2_table']}{', occupancy-culled' if occ is not None else ''}) incl. "
              f"dense Adam over all parameters; FP64 C oracle, one thread")
    out = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps, "higher_is_better": True,
           "scaling": w["scaling"], "vs_baseline": None, "dtype": "f64", "data": "synthetic (analytic shapes, seeded)",
           "config": {"workload": w["name"], **config_keys(w), "reference_sample_rays": n_rays},
           "impl": "reference",
           "cpu_baseline": {"value": value, "unit": "samples/s", "cores": 1, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def stream_inputs(w, R):
    """Input generation for the streaming workload (untimed): per frame the objects first seen there, and the
    observations that the Eq. 5 rule accepts (the decision uses the library's romap_view_angle), with their rays."""
    import numpy as np

    from paper_2304_05735_gb300 import synth

    sc = synth.streaming_scene(n_objects=w["objects"], n_frames=w["frames"], W=w["width"], H=w["height"],
                               f=w["focal"], rate_hz=w["rate_hz"], seed=w["seed0"])
    first = {}
    last_used = {}
    frames = []
    deg = C.c_double()
    for k in range(w["frames"]):
        new, obs = [], []
        for i, ob in enumerate(sc.objects):
            box = synth.detection_box(ob, sc.cam_pos[k], sc.cam_rot[k], sc.W, sc.H, sc.f)
            if box is None or max(box[2] - box[0], box[3] - box[1]) + 1 <= w["min_box_px"]:
                continue
            if i not in first:
                first[i] = k
                new.append(i)
            cam = np.ascontiguousarray(sc.cam_pos[k], np.float64)
            if i in last_used:
                R.check(R.romap_view_angle(last_used[i].ctypes.data, cam.ctypes.data,
                                           np.ascontiguousarray(ob.t, np.float64).ctypes.data, C.byref(deg)))
                if not deg.value > w["alpha_deg"]:
                    continue
            last_used[i] = cam
            rng = np.random.default_rng(ob.seed * 100003 + k)
            obs.append((i, cam, synth.frame_rays(ob, sc.cam_pos[k], sc.cam_rot[k], box, sc.f, sc.W, sc.H, rng,
                                                 stride=1)))
        frames.append((new, obs))
    return sc, frames


def run_stream(args):
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(0)
    from paper_2304_05735_gb300 import romap as R

    R.lib()
    w = WORKLOAD
    sc, frames = stream_inputs(w, R)
    n_obs = sum(len(o) for _, o in frames)
    rays_in = sum(len(r["cls"]) for _, o in frames for _, _, r in o)
    # pinned host copies of every observation (the timed loop copies them to the device through romap_observe)
    pinned = []
    for _, obs in frames:
        per = []
        for i, cam, r in obs:
            t = {k: torch.from_numpy(v).pin_memory() for k, v in r.items()}
            per.append((i, cam, t))
        pinned.append(per)
    rc, h = make_ctx(R, torch, args.precision)
    ids = {}
    steps_per_frame, ms_per_frame, wall_per_frame = [], [], []
    steps_c, ms_c = C.c_int32(), C.c_float()
    upd = C.c_int32()
    R.check(R.romap_reset_stats(h))
    sampler = ClockSampler("0")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k, ((new, _), obs) in enumerate(zip(frames, pinned)):
        tf = time.perf_counter()
        for i in new:
            ob = sc.objects[i]
            oid = C.c_int32()
            d = R.object_desc(t=tuple(ob.t), yaw=ob.yaw, half_size=tuple(ob.half), seed=ob.seed,
                              rays_per_step=w["rays_per_object"])
            R.check(R.romap_create_object(h, C.byref(d), C.byref(oid)), "romap_create_object")
            ids[i] = oid.value
        for i, cam, t in obs:
            rays = R.romap_rays(t["origin"].data_ptr(), t["dir"].data_ptr(), t["rgb"].data_ptr(),
                                t["depth"].data_ptr(), t["cls"].data_ptr())
            R.check(R.romap_observe(h, ids[i], cam.ctypes.data, w["alpha_deg"], C.byref(rays), t["cls"].numel(), 0,
                                    w["iterations"], C.byref(upd)), "romap_observe")
            assert upd.value == 1
        live = list(ids.values())
        arr = (C.c_int32 * len(live))(*live)
        R.check(R.romap_train_budget(h, arr, len(live), w["budget_ms"], 64, C.byref(steps_c), C.byref(ms_c), None))
        steps_per_frame.append(steps_c.value)
        ms_per_frame.append(ms_c.value)
        wall_per_frame.append((time.perf_counter() - tf) * 1e3)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    st = R.romap_stats()
    R.check(R.romap_get_stats(h, C.byref(st)))
    owed = C.c_int64()
    backlog = 0
    for oid in ids.values():
        R.check(R.romap_pending(h, oid, C.byref(owed)))
        backlog += owed.value
    # per-object quality: render each object's last accepted observation and compare on its object rays
    psnr, losses = [], []
    last_obs = {}
    for _, obs in frames:
        for i, cam, r in obs:
            last_obs[i] = r
    for i, r in last_obs.items():
        m = r["cls"] == 0
        if m.sum() < 16:
            continue
        n = int(m.sum())
        o, dd = np.ascontiguousarray(r["origin"][m]), np.ascontiguousarray(r["dir"][m])
        out = np.zeros((n, 3), np.float32)
        bg = (C.c_float * 3)(1.0, 1.0, 1.0)
        R.check(R.romap_render(h, ids[i], o.ctypes.data, dd.ctypes.data, n, bg, out.ctypes.data, None, None, 0))
        mse = float(np.mean((out - r["rgb"][m]) ** 2))
        losses.append(mse)
        psnr.append(-10.0 * np.log10(max(mse, 1e-12)))
    R.check(R.romap_destroy(h))
    train_ms = float(np.sum(ms_per_frame))
    steps = np.array(steps_per_frame)
    value = st.live_samples / (train_ms / 1e3) if train_ms > 0 else 0.0
    out = {"metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": 1, "steps": int(steps.sum()),
           "warmup": 0, "ms_per_step": train_ms / max(1, int(steps.sum())), "higher_is_better": True,
           "scaling": w["scaling"], "vs_baseline": None,
           "dtype": DTYPES.get(args.precision, "f32"),
           "data": "synthetic (analytic shapes, seeded)",
           "config": {"workload": w["name"], **config_keys(w), "precision": args.precision,
                      "observations_accepted": n_obs, "rays_observed": int(rays_in)},
           "stream": {"frames": len(frames), "objects_created": len(ids),
                      "iterations_per_frame": {"mean": float(steps.mean()), "min": int(steps.min()),
                                               "max": int(steps.max())},
                      "train_ms_per_frame": {"mean": float(np.mean(ms_per_frame)), "max": float(np.max(ms_per_frame))},
                      "wall_ms_per_frame": {"mean": float(np.mean(wall_per_frame)),
                                            "p95": float(np.percentile(wall_per_frame, 95))},
                      "frames_budget_used_90pct": float(np.mean(np.array(ms_per_frame) >= 0.9 * w["budget_ms"])),
                      "wall_s": wall, "object_steps": int(st.steps), "live_samples": int(st.live_samples),
                      "owed_steps_at_end": int(backlog),
                      "object_rgb_mse": {"mean": float(np.mean(losses)), "median": float(np.median(losses))},
                      "object_psnr_db": {"mean": float(np.mean(psnr)), "median": float(np.median(psnr)),
                                         "min": float(np.min(psnr))}},
           "gpu_launches": int(st.kernel_launches), "clocks": clocks, "e2e": {
               "value": st.live_samples / wall, "unit": "samples/s",
               "h2d_bytes_per_step": int(rays_in * 45 / max(1, int(steps.sum()))), "d2h_bytes_per_step": 0,
               "path": "create_object + romap_observe (pinned host rays) + romap_train_budget per frame, wall clock"}}
    print(json.dumps(out), flush=True)


def run_table4(args):
    """ms per training iteration of one object (CUDA events over graph-replayed steps) for each table size, in both
    precisions, for the two-net model and for the paper's single-network model, next to the paper's Table 4 (RTX
    4090, single-network model)."""
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(0)
    from paper_2304_05735_gb300 import romap as R

    R.lib()
    global WORKLOAD
    base = dict(WORKLOAD)
    items = build_items(base, 0, 1)
    rows = []
    cases = [(lt, 1, base["paper_ms"][lt], ((("mixed", False), ("fp32", False), ("mixed", True), ("fp32", True))))
             for lt in base["log2_tables"]]
    # Table 4's last two columns: the single network with 2 and 3 hidden layers at T = 2^16
    cases += [(16, k, ms, (("mixed", True), ("fp32", True))) for k, ms in base["paper_layers_ms"].items()]
    for lt, layers, paper_ms, arms in cases:
        row = {"log2_table": lt, "hidden_layers": layers, "paper_ms": paper_ms}
        for prec, single in arms:
            WORKLOAD = dict(base, log2_table=lt)
            rc, h = make_ctx(R, torch, prec, single_net=single, hidden_layers=layers)
            ids = add_objects(R, h, items)
            arr = (C.c_int32 * 1)(*ids)
            R.check(R.romap_train_step(h, arr, 1, max(args.warmup, 3), None))
            R.check(R.romap_reset_stats(h))
            k = args.steps
            ms = timed(torch, lambda: [R.check(R.romap_train_step(h, arr, 1, 1, None)) for _ in range(k)], 1, None)
            st = R.romap_stats()
            R.check(R.romap_get_stats(h, C.byref(st)))
            key = ("single_" if single else "") + prec
            row[f"{key}_ms"] = ms / k
            row[f"{key}_samples_per_s"] = st.live_samples / (ms / 1e3)
            row["params"] = int(R.param_layout(rc).n_params)
            R.check(R.romap_destroy(h))
        rows.append(row)
    WORKLOAD = base
    out = {"metric": METRIC, "value": rows[1]["mixed_samples_per_s"], "unit": "samples/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": rows[1]["mixed_ms"], "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16 (MLP GEMM operands; FP16 table copy; FP32 accumulation, scan, loss, Adam)",
           "data": "synthetic (analytic shapes, seeded)",
           "config": {"workload": base["name"],
                      **{k: v for k, v in config_keys(base).items() if k not in ("paper_ms", "paper_layers_ms")}},
           "sweep": rows,
           "note": "value and ms_per_step: T = 2^16, two-net model; single_* columns: the paper's single-network "
                   "model (position only; hidden_layers of 64), the model its Table 4 times on an RTX 4090 (context, "
                   "not a target)"}
    print(json.dumps(out), flush=True)


def workload_id():
    """The workload's key, with the object count when --objects shrank it (keys of profiles/dram_traffic.json)."""
    return WORKLOAD_KEY + (f":objects={WORKLOAD['objects']}" if WORKLOAD is not WORKLOADS[WORKLOAD_KEY] else "")


def main():
    global WORKLOAD, WORKLOAD_KEY
    args = parse()
    WORKLOAD_KEY = args.workload
    WORKLOAD = WORKLOADS[args.workload]
    if args.objects is not None and args.workload in ("multi8", "uneven32"):
        if not 1 <= args.objects <= WORKLOAD["objects"]:
            raise SystemExit(f"--objects must be in 1..{WORKLOAD['objects']}")
        WORKLOAD = dict(WORKLOAD, objects=args.objects,
                        name=WORKLOAD["name"] + f" (only the first {args.objects} objects)")
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "stream96":
        run_stream(args)
    elif args.workload == "table4":
        run_table4(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
