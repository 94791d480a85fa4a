"""Benchmark: keyframe de-/re-integrations per second on the Kinect-scale workload.

Workload (640x480 Kinect-class frames, 1 cm voxels, 4 cm truncation, 2^20 hash
buckets): 600 synthetic depth + colour frames of a 10x8x3 m multi-room scene,
fused 10 per keyframe into 60 keyframes, integrated at drifted poses, then one
pose-graph update re-integrates all 60 at their true poses.  The inputs are
seeded synthetic stand-ins for the paper's RGB-D sequences; all of them (737 MB of
depth, 737 MB of colour) are resident in HBM before the timed region, and they
exceed the 126 MB L2, so no flush is needed between steps.

One step = one pass of the whole hot path over that input:
  fuse 600 frames into 60 keyframes (Eq. 1), and beside it, on a second stream, reset
  the volume -> integrate the 60 keyframes (allocation + running average) -> ONE
  batched pose update (de-integrate
  all 60 at the drifted poses, re-integrate at the true poses) -> SDF loss at 1 M
  surface points + adjoint for all 60 keyframes, and beside them, on a second stream
  (it reads only the hash table), extract the block list.
value = 60 re-integrations / step time.  The JSON line also reports the update
alone, batched (one graph) vs plain (120 per-keyframe calls), the roofline of the
dominant kernel, the oracle on the host cores, clocks and the kernel count, and,
under "rows", the batching workload (2000 keyframes of 640x480 over a 30x20x3 m room
grid; 10 pose updates of 10-200 keyframes, each batched as one graph launch against
the plain per-keyframe path, with the net-delta kernel's HBM fraction), the batched
forward + backward of 256 of those keyframes against per-keyframe calls, colour
keyframe fusion of the 600 textured frames into the 60 keyframes (its CUDA-event
time, HBM roofline and the oracle beside it), Marching Cubes of the corrected
volume, the KF_OVRLP keyframe grouping of the 600 frames and one streamed pose
update of 10 keyframes (Eq. 3 vs the 10 most-moved), all measured outside the step.

--gpus N > 1 (under torchrun) runs N independent replicas (the path does not
shard across GPUs in this build); value sums the replicas' throughput.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "keyframe de+re-integrations/s @640x480,1cm; batched vs plain; HBM GB/s % peak"
UNIT = "re-integrations/s"
KAPPA = 10
DEPTH_UNITS_PER_M = 5000.0  # 16-bit sensor depth units (TUM RGB-D format)
KF_OVRLP_THR = 0.95  # overlap threshold of the measured KF_OVRLP grouping
# streamed update: m keyframes; resident sphere radius around the camera (m)
STREAM_M, STREAM_RADIUS = 10, 2.0
N_FRAMES = 600
N_POINTS = 1_000_000
LAMBDA = 0.1
IMG_BYTES = 640 * 480 * (4 + 4)  # keyframe depth f32 + RGBA8
VOXEL_BYTES_RW = 24             # D, W, RGBA8: 12 B read + 12 B written per voxel

# Instruction-issue roofline.  The step's largest kernels are bound by instruction
# issue (ncu: issue active 70-72 %, DRAM < 20 % of peak), so the roofline is the issue
# rate: 148 SMs x 4 schedulers x 1 warp instruction / cycle x 32 lanes x SM clock.
# Warp instructions per unit of work and DRAM bytes per unit come from the ncu capture
# of the 12-keyframe case (profiles/instructions_kinect_small.md); units are frames
# (fusion) and keyframe images (batched allocation).
SMS, SCHEDULERS, LANES = 148, 4, 32
WINST_PER_UNIT = {"fuse_kernel": 895077.4, "batch_alloc_kernel": 3241665.3}
DRAM_PER_UNIT = {"fuse_kernel": 1.5641e6, "batch_alloc_kernel": 1.2865e6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=60, help="keyframe re-integrations the oracle times per step")
    ap.add_argument("--profile-region", action="store_true",
                    help="run --steps steps between cudaProfilerStart/Stop and exit (for ncu "
                         "--profile-from-start off); prints only the timing")
    ap.add_argument("--profile-colour", action="store_true",
                    help="run colour fusion steps between cudaProfilerStart/Stop (for ncu) and exit")
    ap.add_argument("--profile-extra", choices=["mc", "kf", "overlap", "stream"], default=None,
                    help="run Marching Cubes / KF_OVRLP grouping / a stream-out + stream-in of the "
                         "step's volume between cudaProfilerStart/Stop (for ncu) and exit")
    ap.add_argument("--keyframes", type=int, default=60, help="keyframes of the workload (small ncu cases)")
    ap.add_argument("--max-blocks", type=int, default=1 << 21)
    ap.add_argument("--no-batching", action="store_true", help="skip the 2000-keyframe batching rows")
    ap.add_argument("--profile-batching", action="store_true",
                    help="batching workload cut to --keyframes keyframes: one pose update of its first update's "
                         "size (at most half the keyframes) between cudaProfilerStart/Stop (for ncu), then exit")
    ap.add_argument("--batching-reps", type=int, default=10, help="replays per pose update in the batching rows")
    ap.add_argument("--batch-config", default=None,
                    help="warps_per_cta,ctas_per_sm,blocks_per_grab of the net-delta launch instead of the autotuned "
                         "one (so that an ncu capture of a small case runs the full-size launch shape)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def _busy_wait(seconds):
    """Spin instead of sleeping: an idle host drops its clock and the next steps' host-side
    launch work runs several times slower until it ramps back up."""
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        pass


class Clocks:
    """nvidia-smi sampled every 50 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        _busy_wait(0.3)  # give the sampler time to start without letting the host idle
        return self

    def __exit__(self, *a):
        if self.proc:
            _busy_wait(0.3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
                for name, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        except Exception:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.remove(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


# --------------------------------------------------------------------------------------

def make_workload(device, keyframes=60):
    import torch
    from paper_1709_03763_b300 import synthetic
    w = synthetic.workload_kinect(device=device, n_frames=N_FRAMES, kappa=KAPPA, render_frames=keyframes * KAPPA,
                                  textured=True)
    # sensor-format depth: 16-bit in 1/5000 m units (the TUM RGB-D format); the frames
    # the step reads are exactly raw * float32(1/5000), as sc_depth_from_u16 makes them
    raw = torch.clamp(torch.round(w.frames_depth.double() * DEPTH_UNITS_PER_M), 0, 65535).to(torch.int32)
    w.extra["depth_raw"] = raw.to(torch.int16)  # the 16-bit pattern
    w.frames_depth = (raw.to(torch.float32) * torch.tensor(1.0 / DEPTH_UNITS_PER_M, dtype=torch.float32,
                                                           device=raw.device)).contiguous()
    w.kf_poses = w.kf_poses[:keyframes]
    w.new_poses = w.new_poses[:keyframes]
    w.kf_rgba = w.kf_rgba[:keyframes].contiguous()
    pts = synthetic.surface_points(w.scene, N_POINTS, 4, lo=np.array([0.0, 0.0, 0.0]),
                                   hi=np.array([10.0, 8.0, 3.0]))
    w.extra["points"] = torch.tensor(pts, dtype=torch.float32, device=device)
    return w


class Pipeline:
    """One step of the whole hot path (see module docstring)."""

    def __init__(self, w, vol):
        import torch
        self.w = w
        self.V = vol
        K = len(w.kf_poses)
        self.K = K
        dev = w.frames_depth.device
        self.kf_depth = torch.empty((K, w.intr.height, w.intr.width), dtype=torch.float32, device=dev)
        self.kf_weight = torch.empty_like(self.kf_depth)
        self.kf_rgba = w.kf_rgba
        self.ids = list(range(K))
        from paper_1709_03763_b300 import make_intrinsics, make_pose
        # ABI structs built once, outside the timed region
        self.intr = make_intrinsics(w.intr)
        self.frame_poses = [make_pose(T) for T in w.frame_poses]
        self.drift = [make_pose(T) for T in w.kf_poses]
        self.true = [make_pose(T) for T in w.new_poses]
        self.grad_D = vol.grad_buffer()
        # argument arrays of the per-step calls, built once
        from paper_1709_03763_b300 import prepare_fuse
        nf = K * KAPPA
        self.prep_fuse = prepare_fuse(self.frame_poses[:nf], [f // KAPPA for f in range(nf)], self.frame_poses[:nf:KAPPA])
        self.prep_int = vol.prepare_integrate_many(self.ids, self.kf_depth, self.kf_rgba, self.drift)
        self.prep_upd = vol.prepare_batch(self.ids, self.kf_depth, self.kf_rgba, self.drift, self.true)
        self.prep_adj = vol.prepare_adjoint(self.ids, self.kf_depth, self.true)
        from paper_1709_03763_b300 import prepare_colour
        self.prep_col = prepare_colour(self.frame_poses[:nf], [f // KAPPA for f in range(nf)],
                                       self.frame_poses[:nf:KAPPA], w.intr.width, w.intr.height, dev)
        self.kf_colour = torch.empty((K, w.intr.height, w.intr.width, 4), dtype=torch.uint8, device=dev)
        self.loss_out = torch.empty(5, dtype=torch.float64, device=dev)
        self.gx = torch.empty((K, 6), dtype=torch.float64, device=dev)
        self.gd = torch.empty((K, w.intr.height, w.intr.width), dtype=torch.float32, device=dev)
        self.side = torch.cuda.Stream(device=dev)  # the reset's and the extraction's stream (see step)
        self.ev_upd = torch.cuda.Event()
        self.ev_prev = torch.cuda.Event()
        self.ev_reset = torch.cuda.Event()

    def fuse(self):
        """Eq. 1 for all keyframes in one call (KF_CONST: frames k*10 .. k*10+9 -> keyframe k)."""
        from paper_1709_03763_b300 import fuse_keyframes
        nf = self.K * KAPPA
        fuse_keyframes(self.w.frames_depth[:nf], intr=self.intr, disc_rel=0.1, out_depth=self.kf_depth,
                       out_weight=self.kf_weight, prepared=self.prep_fuse)

    def colour(self):
        """Colour keyframe fusion of all 600 frames into the 60 keyframes (Section 3)."""
        from paper_1709_03763_b300 import fuse_colour_keyframes
        nf = self.K * KAPPA
        fuse_colour_keyframes(self.w.frames_rgba[:nf], self.w.frames_depth[:nf], self.kf_depth, intr=self.intr,
                              out_rgba=self.kf_colour, prepared=self.prep_col)

    def integrate(self):
        """Reset, then integrate every keyframe at its drifted pose (one graph launch)."""
        self.V.reset()
        self.V.integrate_many(intr=self.intr, prepared=self.prep_int)

    def integrate_plain(self):
        self.V.reset()
        for k in range(self.K):
            self.V.integrate(k, self.kf_depth[k], self.kf_rgba[k], self.intr, self.drift[k])

    def update_batched(self):
        self.V.reintegrate_batch(intr=self.intr, prepared=self.prep_upd)

    def update_plain(self):
        for k in self.ids:
            self.V.deintegrate(k, self.kf_depth[k], self.kf_rgba[k], self.intr, self.drift[k])
        for k in self.ids:
            self.V.integrate(k, self.kf_depth[k], self.kf_rgba[k], self.intr, self.true[k])

    def loss_adjoint(self):
        out, _ = self.V.sdf_loss(self.w.extra["points"], LAMBDA, grad_D=self.grad_D, out=self.loss_out)
        gx, gd = self.V.sdf_adjoint(intr=self.intr, grad_D=self.grad_D, prepared=self.prep_adj, out=(self.gx, self.gd))
        return out, gx, gd

    def extract(self):
        return self.V.extract(payload=False, capacity=self.capacity)

    def step(self):
        import torch
        # the reset touches only the volume, which the fusion leaves alone: it runs on a
        # second stream beside the fusion, once the previous step's adjoint is done
        self.ev_prev.record()
        self.side.wait_event(self.ev_prev)
        self.V.reset(stream=self.side)
        self.ev_reset.record(self.side)
        self.fuse()
        torch.cuda.current_stream().wait_event(self.ev_reset)
        self.V.integrate_many(intr=self.intr, prepared=self.prep_int)
        self.update_batched()
        # the block-list extraction reads only the hash table, which the loss and the
        # adjoint leave as it is: it runs on a second stream beside them, so its count
        # read-back waits for the extraction alone, and the next step's launches queue
        # behind the adjoint instead of following a drained device
        self.ev_upd.record()
        out, gx, gd = self.loss_adjoint()
        self.side.wait_event(self.ev_upd)
        ex = self.V.extract(payload=False, capacity=self.capacity, stream=self.side)
        return out, ex


def time_region(fn, steps, warmup, ws):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1) / steps
    return max_over_ranks(ms, ws)


def update_only_timing(P, steps, batched: bool):
    """Median time of one 60-keyframe pose update (the integrated state is re-built before
    each repetition, outside the timed part)."""
    import torch
    ts = []
    s = torch.cuda.current_stream()
    for _ in range(steps):
        P.integrate()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        (P.update_batched if batched else P.update_plain)()
        e1.record(s)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


# algorithmic bytes of colour fusion: its inputs and outputs -- per frame, the RGBA read
# and the depth read by the occlusion test; per keyframe, Z* read and C* written.  The
# unsharp texels are an intermediate that the library keeps in L2 (32-frame chunks).
def colour_bytes(n_frames, n_kf, H, W):
    px = H * W
    return n_frames * px * (4 + 4) + n_kf * px * (4 + 4)


def colour_timing(P, reps, warmup):
    """CUDA-event time of one colour fusion call over the whole workload (median)."""
    import torch
    for _ in range(warmup):
        P.colour()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        P.colour()
        e1.record(s)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts)


def oracle_mc(max_blocks=20000):
    """The oracle's Marching Cubes on (a bounded sample of) the oracle's own re-integrated
    volume from the CPU baseline: (blocks per second, blocks, triangles, seconds)."""
    import oracle
    O = getattr(oracle_reintegration, "last_volume", None)
    if O is None:
        return None
    ex = O.export()
    n = min(max_blocks, len(ex.coords))
    D, W = ex.D[:n].astype(np.float32), ex.W[:n].astype(np.float32)
    t0 = time.perf_counter()
    tri, _ = oracle.marching_cubes(ex.coords[:n], D, W, O.voxel_size)
    dt = time.perf_counter() - t0
    return n / dt, n, len(tri), dt


def streaming_protocol(P, V, store, strategy, m, radius):
    """One pose update of m keyframes under the streaming sphere (Section 4.3): from the
    state "only the sphere around the camera is resident", stream in the stored blocks
    the selected keyframes' block lists name and the stored blocks their updated poses'
    allocation reaches, re-integrate the m keyframes in one batch, stream back out
    around the camera.  strategy: "consecutive" (Eq. 3) or "topm" (the m most-moved,
    BundleFusion).  Returns (CUDA-event ms of the whole update, (blocks in for the
    lists, blocks in for the poses), blocks out, ids)."""
    import torch
    from paper_1709_03763_b300 import pose_distance, select_consecutive, select_topm
    w = P.w
    new_poses = w.extra["stream_new_poses"]
    dist = np.array([pose_distance(a, b) for a, b in zip(w.kf_poses, new_poses)])
    if strategy == "consecutive":
        j = select_consecutive(dist, m)
        ids = list(range(j, j + m))
    else:
        ids = sorted(int(i) for i in select_topm(dist, m))
    cam = np.asarray(w.frame_poses[P.K * KAPPA - 1], np.float32)[:, 3]
    depths = [P.kf_depth[k] for k in ids]
    P.integrate()
    V.stream_out(store, cam, radius)
    torch.cuda.synchronize()
    res = {}

    def update():
        res["lists"] = V.stream_in_keyframes(store, ids)
        res["poses"] = V.stream_in_poses(store, depths, new_poses[ids], P.intr)
        V.reintegrate_batch(ids, P.kf_depth[ids], P.kf_rgba[ids], w.kf_poses[ids], new_poses[ids], P.intr)
        res["out"] = V.stream_out(store, cam, radius)
    ms = _event_ms(update)
    V.stream_in(store, cam)  # leave the volume whole
    return ms, (res["lists"], res["poses"]), res["out"], ids


def oracle_kf(w, n):
    """The oracle's KF_OVRLP grouping of the first n frames: (frames per second, seconds)."""
    import oracle
    d = w.frames_depth[:n].cpu().numpy()
    t0 = time.perf_counter()
    oracle.segment(oracle.KF_OVRLP, (KF_OVRLP_THR,), w.frame_poses[:n], w.intr.as_tuple(), d)
    dt = time.perf_counter() - t0
    return n / dt, dt


def mc_timing(V, out, reps, warmup):
    """Median time of one sc_marching_cubes call (count read-back and status included) and
    the mean CUDA-event time of its kernel (the library's profile)."""
    import torch
    for _ in range(warmup):
        tri = V.marching_cubes(capacity=out.shape[0], out=out)
    torch.cuda.synchronize()
    ts = []
    V.set_profiling(True)
    for _ in range(reps):
        t0 = time.perf_counter()
        tri = V.marching_cubes(capacity=out.shape[0], out=out)
        ts.append((time.perf_counter() - t0) * 1e3)
    prof = V.profile()
    V.set_profiling(False)
    kernel_ms = prof["mc_ms"] / max(1, prof["mc_launches"])
    return statistics.median(ts), kernel_ms, int(tri.shape[0])


def oracle_colour(w, kf_depth, n_kf=3):
    """The oracle's colour fusion of the first n_kf keyframes (10 frames each) on the host
    cores: (keyframes per second, threads)."""
    import oracle
    oracle.build()
    it = w.intr.as_tuple()
    rgba = w.frames_rgba[:n_kf * KAPPA].cpu().numpy()
    depth = w.frames_depth[:n_kf * KAPPA].cpu().numpy()
    kd = kf_depth[:n_kf].cpu().numpy()
    t0 = time.perf_counter()
    for k in range(n_kf):
        sl = slice(k * KAPPA, (k + 1) * KAPPA)
        oracle.fuse_colour(rgba[sl], depth[sl], w.frame_poses[sl], kd[k], w.frame_poses[k * KAPPA], it)
    dt = time.perf_counter() - t0
    return n_kf / dt, oracle.get_threads(), dt


def oracle_reintegration(n_kf, steps=1, warmup=0, w=None):
    """The FP64 oracle, as it stands, re-integrating the first n_kf keyframes of this
    workload (de-integrate at the drifted pose + integrate at the true pose, allocation
    included) on the host cores.  Its keyframe depth is the oracle's own Eq. 1 fusion of
    the keyframe's 10 frames.  Returns (median seconds per step, threads used)."""
    import oracle
    from paper_1709_03763_b300 import synthetic
    oracle.build()
    if w is None:  # the same workload as the GPU arm (sensor-format depth, textured colour)
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        w = make_workload(torch.device(dev), n_kf)
    it = w.intr.as_tuple()
    frames = w.frames_depth[:n_kf * KAPPA].cpu()
    depth = []
    for k in range(n_kf):
        s = k * KAPPA
        Z, _, _ = oracle.fuse(frames[s:s + KAPPA], w.frame_poses[s:s + KAPPA], w.frame_poses[s], it)
        depth.append(Z.astype(np.float32))
    rgba = w.kf_rgba.cpu().numpy()
    times = []
    for step in range(warmup + steps):
        O = oracle.Volume(w.voxel_size, w.trunc, rgba8=True)
        for k in range(n_kf):
            O.integrate(k, depth[k], rgba[k], it, w.kf_poses[k])
        t0 = time.perf_counter()
        for k in range(n_kf):
            O.deintegrate(k, depth[k], rgba[k], it, w.kf_poses[k])
            O.integrate(k, depth[k], rgba[k], it, w.new_poses[k])
        if step >= warmup:
            times.append(time.perf_counter() - t0)
    oracle_reintegration.last_volume = O
    return statistics.median(times), oracle.get_threads()


def cpu_baseline(n_kf, w, reps=3):
    dt, cores = oracle_reintegration(n_kf, steps=reps, w=w)
    return {"value": n_kf / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n_kf} keyframe re-integrations (de-integrate at drifted pose + integrate at true pose, "
                      f"allocation included) of the 640x480 / 1 cm workload, RGBA8 colour, FP64; median of "
                      f"{reps} passes, {dt:.1f} s each"}


def fp32_peak():
    """Measured FP32 FMA rate of this GPU (lane FMAs per second, in T/s), or None."""
    import ctypes
    from paper_1709_03763_b300 import lib
    r, ms = ctypes.c_double(0), ctypes.c_double(0)
    rc = lib().sc_measure_fp32_rate(4096, ctypes.byref(r), ctypes.byref(ms), None)
    return (r.value / 1e12, ms.value) if rc == 0 else (None, None)


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def _event_ms(fn):
    """CUDA-event time of fn() on the current stream (host work inside fn included)."""
    import torch
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def batching_rows(dev, hbm_peak, peak_kind, reps, cpu_sample, ws):
    """The batching workload (2000 keyframes of 640x480 over a 30x20x3 m room grid, 1 cm
    voxels, 2^22 buckets, RGBA8) and its 10 pose updates of a seeded 10-200 keyframes
    chosen by largest pose change (Section 4.3): per update, the batched path (one graph
    launch, autotuned on the first update) against the plain path (n de-integrations then
    n integrations), each the median of `reps` replays that alternate the update and its
    reverse (the reverse is an update of the same keyframes back to their former poses,
    so every replay starts from a volume integrated at the poses it de-integrates);
    then 256 of those keyframes as one batched forward + backward (one integration graph,
    the loss at 1 M points, one adjoint launch) against 256 plain integrations, the loss
    and 256 per-keyframe adjoint calls."""
    import torch
    from paper_1709_03763_b300 import Volume, make_intrinsics, make_pose, pose_distance, select_topm, synthetic
    t0 = time.perf_counter()
    w = synthetic.workload_batching(device=dev)
    K = len(w.kf_poses)
    D, C = w.kf_depth, w.kf_rgba
    intr = make_intrinsics(w.intr)
    V = Volume(w.voxel_size, w.trunc, w.n_buckets, colour="rgba8", max_blocks=1 << 21, max_keyframes=K,
               max_blocks_per_keyframe=1 << 16, max_batch=256)
    for s0 in range(0, K, 256):
        ids = list(range(s0, min(K, s0 + 256)))
        V.integrate_many(ids, [D[k] for k in ids], [C[k] for k in ids], w.kf_poses[ids], intr)
    V.check()
    counts = np.array([V.keyframe_blocks(k).numel() for k in range(K)])
    setup_s = time.perf_counter() - t0
    cur = w.kf_poses.copy()
    ups, tuned = [], None
    for u, upd in enumerate(w.updates):
        tgt = upd["target_poses"]
        dist = np.array([pose_distance(cur[k], tgt[k]) for k in range(K)])
        ids = [int(i) for i in select_topm(dist, upd["n"])]
        n = len(ids)
        dl, cl = [D[k] for k in ids], [C[k] for k in ids]
        fwd = V.prepare_batch(ids, dl, cl, cur[ids], tgt[ids])
        rev = V.prepare_batch(ids, dl, cl, tgt[ids], cur[ids])
        if tuned is None:
            tuned, _ = V.autotune_batch(ids, dl, cl, cur[ids], tgt[ids], intr)
        for _ in range(2):
            V.reintegrate_batch(intr=intr, prepared=fwd)
            V.reintegrate_batch(intr=intr, prepared=rev)
        tb = [_event_ms(lambda r=r: V.reintegrate_batch(intr=intr, prepared=fwd if r % 2 == 0 else rev))
              for r in range(reps)]
        V.set_profiling(True)
        V.reintegrate_batch(intr=intr, prepared=fwd)
        pr = V.profile()
        V.set_profiling(False)
        V.reintegrate_batch(intr=intr, prepared=rev)
        po = {k: make_pose(cur[k]) for k in ids}
        pn = {k: make_pose(tgt[k]) for k in ids}
        n_old = sum(V.keyframe_blocks(k).numel() for k in ids)

        def plain(a, b):
            for k in ids:
                V.deintegrate(k, D[k], C[k], intr, a[k])
            for k in ids:
                V.integrate(k, D[k], C[k], intr, b[k])
        plain(po, pn)
        n_new = sum(V.keyframe_blocks(k).numel() for k in ids)
        plain(pn, po)
        tp = [_event_ms(lambda r=r: plain(po, pn) if r % 2 == 0 else plain(pn, po)) for r in range(reps)]
        # advance to the updated poses (batched)
        V.reintegrate_batch(intr=intr, prepared=fwd)
        V.check()
        cur[ids] = tgt[ids]
        U, P = pr["batch_union_blocks"], pr["batch_pairs"]
        net_bytes = U * 512 * VOXEL_BYTES_RW + n * IMG_BYTES + P * 4
        plain_bytes = (n_old + n_new) * 512 * VOXEL_BYTES_RW + 2 * n * IMG_BYTES + (n_old + n_new) * 32
        bm, pm = statistics.median(tb), statistics.median(tp)
        ups.append({"n": n, "union_blocks": U, "pairs": P, "batched_ms": bm, "plain_ms": pm,
                    "batched_reint_per_s": n / (bm / 1e3), "plain_reint_per_s": n / (pm / 1e3),
                    "speedup": pm / bm, "net_delta_ms": pr["batch_net_ms"], "alloc_ms": pr["batch_alloc_ms"],
                    "mark_ms": pr["batch_mark_ms"], "net_delta_bytes": net_bytes,
                    "net_delta_hbm_frac": net_bytes / (pr["batch_net_ms"] / 1e3) / 1e9 / hbm_peak,
                    "update_hbm_frac": net_bytes / (bm / 1e3) / 1e9 / hbm_peak,
                    "plain_hbm_frac": plain_bytes / (pm / 1e3) / 1e9 / hbm_peak})
    nsum = sum(x["n"] for x in ups)
    tb_sum = sum(x["batched_ms"] for x in ups)
    tp_sum = sum(x["plain_ms"] for x in ups)
    nd_bytes = sum(x["net_delta_bytes"] for x in ups)
    nd_ms = sum(x["net_delta_ms"] for x in ups)
    row = {"workload": "batching: 2000 keyframes 640x480 over a 30x20x3 m room grid, voxel 1 cm, trunc 4 cm, "
                       "2^22 buckets, RGBA8; 10 pose updates of 10-200 keyframes (largest pose change)",
           "allocated_blocks": V.info()["allocated_blocks"],
           "touched_blocks_per_keyframe": {"min": int(counts.min()), "median": int(np.median(counts)),
                                           "max": int(counts.max())},
           "batch_config": tuned, "replays": reps,
           "batched_reint_per_s": ws * nsum / (tb_sum / 1e3), "plain_reint_per_s": ws * nsum / (tp_sum / 1e3),
           "speedup": tp_sum / tb_sum,
           "net_delta_hbm": {"achieved": nd_bytes / (nd_ms / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                             "frac": nd_bytes / (nd_ms / 1e3) / 1e9 / hbm_peak, "peak_kind": peak_kind,
                             "min_frac": min(x["net_delta_hbm_frac"] for x in ups),
                             "max_frac": max(x["net_delta_hbm_frac"] for x in ups)},
           "update_hbm_frac": nd_bytes / (tb_sum / 1e3) / 1e9 / hbm_peak,
           "updates": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in x.items()
                        if k not in ("net_delta_bytes",)} for x in ups],
           "setup_s": setup_s}

    # ---- 256 keyframes: batched forward + backward vs per-keyframe
    nfb = 256
    ids = list(range(nfb))
    dl, cl = [D[k] for k in ids], [C[k] for k in ids]
    pts = torch.tensor(synthetic.surface_points(w.scene, N_POINTS, 5), dtype=torch.float32, device=dev)
    prep_i = V.prepare_integrate_many(ids, dl, cl, w.kf_poses[ids])
    prep_a = V.prepare_adjoint(ids, dl, w.kf_poses[ids])
    prep_a1 = [V.prepare_adjoint([k], [D[k]], w.kf_poses[k:k + 1]) for k in ids]
    pz = [make_pose(w.kf_poses[k]) for k in ids]
    gD = V.grad_buffer()
    lo = torch.empty(5, dtype=torch.float64, device=dev)
    gx = torch.empty((nfb, 6), dtype=torch.float64, device=dev)
    gd = torch.empty((nfb, w.intr.height, w.intr.width), dtype=torch.float32, device=dev)

    def fb_batched():
        V.reset()
        V.integrate_many(intr=intr, prepared=prep_i)
        V.sdf_loss(pts, LAMBDA, grad_D=gD, out=lo)
        V.sdf_adjoint(intr=intr, grad_D=gD, prepared=prep_a, out=(gx, gd))

    def fb_plain():
        V.reset()
        for k in ids:
            V.integrate(k, D[k], C[k], intr, pz[k])
        V.sdf_loss(pts, LAMBDA, grad_D=gD, out=lo)
        for k in ids:
            V.sdf_adjoint(intr=intr, grad_D=gD, prepared=prep_a1[k], out=(gx[k:k + 1], gd[k:k + 1]))
    fb_batched()
    fb_plain()
    tfb = statistics.median(_event_ms(fb_batched) for _ in range(3))
    tfp = statistics.median(_event_ms(fb_plain) for _ in range(3))
    fb_row = {"workload": "256 keyframes of the batching workload: integration + loss at 1 M surface points + "
                          "adjoint (pose and depth gradients)",
              "batched_ms": tfb, "plain_ms": tfp, "batched_keyframes_per_s": ws * nfb / (tfb / 1e3),
              "plain_keyframes_per_s": ws * nfb / (tfp / 1e3), "speedup": tfp / tfb,
              "batched": "one integration graph launch, one loss, one adjoint launch for all 256",
              "plain": "256 sc_integrate_keyframe calls, one loss, 256 sc_sdf_adjoint calls"}
    V.close()
    del w, D, C
    torch.cuda.empty_cache()
    return row, fb_row


def profile_batching(dev, n_kf, max_blocks, steps, warmup):
    """The batching workload with n_kf keyframes: integrate all, then replay one pose
    update (the first update's size, at most n_kf / 2 keyframes chosen by largest pose
    change) and its reverse; the timed replays run between cudaProfilerStart/Stop."""
    import torch
    from paper_1709_03763_b300 import Volume, make_intrinsics, pose_distance, select_topm, synthetic
    w = synthetic.workload_batching(device=dev, n_keyframes=n_kf, n_updates=1)
    D, C = w.kf_depth, w.kf_rgba
    intr = make_intrinsics(w.intr)
    V = Volume(w.voxel_size, w.trunc, w.n_buckets, colour="rgba8", max_blocks=max_blocks, max_keyframes=n_kf,
               max_blocks_per_keyframe=1 << 16, max_batch=256)
    for s0 in range(0, n_kf, 256):
        ids = list(range(s0, min(n_kf, s0 + 256)))
        V.integrate_many(ids, [D[k] for k in ids], [C[k] for k in ids], w.kf_poses[ids], intr)
    upd = w.updates[0]
    tgt = upd["target_poses"]
    dist = np.array([pose_distance(w.kf_poses[k], tgt[k]) for k in range(n_kf)])
    ids = [int(i) for i in select_topm(dist, min(upd["n"], n_kf // 2))]
    dl, cl = [D[k] for k in ids], [C[k] for k in ids]
    fwd = V.prepare_batch(ids, dl, cl, w.kf_poses[ids], tgt[ids])
    rev = V.prepare_batch(ids, dl, cl, tgt[ids], w.kf_poses[ids])
    V.autotune_batch(ids, dl, cl, w.kf_poses[ids], tgt[ids], intr)  # the launch shape the bench row uses
    for _ in range(warmup):
        V.reintegrate_batch(intr=intr, prepared=fwd)
        V.reintegrate_batch(intr=intr, prepared=rev)
    V.check()
    torch.cuda.synchronize()
    torch.cuda.profiler.start()
    for r in range(steps):
        V.reintegrate_batch(intr=intr, prepared=fwd if r % 2 == 0 else rev)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    V.set_profiling(True)
    V.reintegrate_batch(intr=intr, prepared=fwd)
    pr = V.profile()
    print(json.dumps({"profile_batching": len(ids), "keyframes": n_kf, "blocks": V.info()["allocated_blocks"],
                      "union_blocks": pr["batch_union_blocks"], "pairs": pr["batch_pairs"],
                      "net_delta_ms": pr["batch_net_ms"], "alloc_ms": pr["batch_alloc_ms"]}), flush=True)


def oracle_batching_sample(n_kf=2):
    """The oracle re-integrating n_kf keyframes of the batching workload's first update
    (FP64, host cores): (seconds per re-integration, threads)."""
    import oracle
    from paper_1709_03763_b300 import synthetic
    oracle.build()
    w = synthetic.workload_batching(device="cpu", n_keyframes=n_kf, n_updates=1)
    it = w.intr.as_tuple()
    O = oracle.Volume(w.voxel_size, w.trunc, rgba8=True)
    d, c = w.kf_depth.numpy(), w.kf_rgba.numpy()
    for k in range(n_kf):
        O.integrate(k, d[k], c[k], it, w.kf_poses[k])
    tgt = w.updates[0]["target_poses"]
    t0 = time.perf_counter()
    for k in range(n_kf):
        O.deintegrate(k, d[k], c[k], it, w.kf_poses[k])
        O.integrate(k, d[k], c[k], it, tgt[k])
    return (time.perf_counter() - t0) / n_kf, oracle.get_threads()


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores (rank 0 only)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_kf = max(1, args.cpu_sample)
    sec, cores = oracle_reintegration(n_kf, steps=args.steps, warmup=args.warmup)
    ms = sec * 1000.0
    value = n_kf / sec
    sample = (f"{n_kf} keyframe re-integrations per step (de-integrate at drifted pose + integrate at true "
              f"pose, allocation included), 640x480, 1 cm voxels, FP64")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "kinect-scale: 60 keyframes 640x480 fused from 600 frames, voxel 1 cm, "
                                   "trunc 4 cm, 2^20 buckets", "sample_keyframes": n_kf},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    ws, rank, local = dist_init()
    from paper_1709_03763_b300 import Volume, lib
    from paper_1709_03763_b300 import build as _build
    _build.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    if args.profile_batching:
        profile_batching(dev, args.keyframes, args.max_blocks, args.steps, args.warmup)
        return

    t_setup = time.perf_counter()
    w = make_workload(dev, args.keyframes)
    V = Volume(w.voxel_size, w.trunc, w.n_buckets, bucket_size=4, max_blocks=args.max_blocks, colour="rgba8",
               max_keyframes=64, max_blocks_per_keyframe=1 << 17, max_batch=64)
    P = Pipeline(w, V)
    P.capacity = args.max_blocks
    P.fuse()
    P.integrate()
    torch.cuda.synchronize()
    cfg, tune_ms = V.autotune_batch(P.ids, P.kf_depth, P.kf_rgba, P.drift, P.true, P.intr)
    if args.batch_config:
        wpc, cps, bpg = (int(x) for x in args.batch_config.split(","))
        V.set_batch_config(wpc, cps, bpg)
        cfg = V.batch_config()
    P.prep_upd = V.prepare_batch(P.ids, P.kf_depth, P.kf_rgba, P.drift, P.true)
    setup_s = time.perf_counter() - t_setup

    if args.profile_extra:
        from paper_1709_03763_b300 import KF_OVRLP, BlockStore, overlap_counts, segment_keyframes
        P.step()
        torch.cuda.synchronize()
        nfr = P.K * KAPPA
        cam = np.asarray(w.frame_poses[nfr - 1], np.float32)[:, 3]
        store = BlockStore(V.info()["allocated_blocks"] + 1024, "rgba8") if args.profile_extra == "stream" else None
        mc_out = torch.empty((4 << 20, 3, 3), dtype=torch.float32, device=dev) if args.profile_extra == "mc" else None

        def extra():
            if args.profile_extra == "mc":
                V.marching_cubes(capacity=mc_out.shape[0], out=mc_out)
            elif args.profile_extra == "kf":
                segment_keyframes(KF_OVRLP, (KF_OVRLP_THR,), w.frame_poses[:nfr], w.intr, w.frames_depth[:nfr])
            elif args.profile_extra == "overlap":  # the overlap counts of 32 frames against frame 0
                overlap_counts(w.frames_depth[:32], w.frame_poses[:32], w.frame_poses[0], w.intr)
            else:
                V.stream_out(store, cam, STREAM_RADIUS)
                V.stream_in(store, cam)
        for _ in range(args.warmup):
            extra()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        for _ in range(args.steps):
            extra()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile_extra": args.profile_extra, "steps": args.steps}), flush=True)
        return

    if args.profile_colour:
        for _ in range(args.warmup):
            P.colour()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        for _ in range(args.steps):
            P.colour()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile_colour_steps": args.steps, "keyframes": P.K}), flush=True)
        return

    if args.profile_region:
        for _ in range(args.warmup):
            P.step()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            P.step()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile_region_steps": args.steps, "keyframes": P.K,
                          "ms_per_step_host": (time.perf_counter() - t0) * 1000 / args.steps}), flush=True)
        return

    # ---- the timed whole-path step
    L0 = lib().sc_kernel_launches()
    with Clocks(local) as clk:
        ms = time_region(P.step, args.steps, args.warmup, ws)
    launches_per_step = (lib().sc_kernel_launches() - L0) / (args.steps + args.warmup)
    clocks = clk.summary()
    value = ws * P.K / (ms / 1000.0)

    # ---- end to end through the public API with host buffers: per step, the 600 depth
    # frames and the 60 keyframe colour images (the only colour the path reads: the
    # keyframe's colour is its own frame's) go host -> device from pinned memory, and
    # the loss and block count come back
    from paper_1709_03763_b300 import depth_from_u16, rgba_from_rgb
    h_depth = w.frames_depth.cpu().pin_memory()
    h_raw = w.extra["depth_raw"].cpu().pin_memory()
    h_rgba = P.kf_rgba.cpu().pin_memory()
    h_rgb = P.kf_rgba[..., :3].contiguous().cpu().pin_memory()  # the sensor's RGB8 (alpha is 255)
    h_out = torch.empty(6, dtype=torch.float64).pin_memory()
    d_depth, d_rgba = w.frames_depth, P.kf_rgba
    depth_scale = float(np.float32(1.0 / DEPTH_UNITS_PER_M))

    def e2e_step_serial():
        d_depth.copy_(h_depth, non_blocking=True)
        d_rgba.copy_(h_rgba, non_blocking=True)
        out, ex = P.step()
        h_out[:5].copy_(out, non_blocking=True)
        h_out[5] = ex["coords"].shape[0]
    e2e_serial_ms = time_region(e2e_step_serial, args.steps, args.warmup, ws)

    # pipelined, from the sensor formats: the 16-bit depth frames and the RGB8 keyframe
    # colour are double-buffered; while step k computes, a copy stream loads step k+1's
    # inputs into the other buffers, and step k ends only once they have arrived, so
    # every step's inputs still cross within the timed region; each step converts its
    # raw frames to metres (sc_depth_from_u16) and its colour to RGBA8
    # (sc_rgba_from_rgb) before it runs
    cur = torch.cuda.current_stream()
    copy_stream = torch.cuda.Stream()
    bufs = [torch.empty_like(w.extra["depth_raw"]), torch.empty_like(w.extra["depth_raw"])]
    rgb_bufs = [torch.empty(h_rgb.shape, dtype=torch.uint8, device=dev) for _ in range(2)]
    ev_copied = [torch.cuda.Event(), torch.cuda.Event()]
    ev_used = [torch.cuda.Event(), torch.cuda.Event()]
    for e in ev_used:
        e.record(cur)
    st = {"k": 0}

    def issue_copy(b):
        copy_stream.wait_event(ev_used[b])  # the step that read buffer b is done with it
        with torch.cuda.stream(copy_stream):
            bufs[b].copy_(h_raw, non_blocking=True)
            rgb_bufs[b].copy_(h_rgb, non_blocking=True)
        ev_copied[b].record(copy_stream)

    def e2e_step():
        k = st["k"]
        b = k % 2
        if k == 0:
            issue_copy(b)
        issue_copy(1 - b)  # the next step's frames, overlapped with this step
        cur.wait_event(ev_copied[b])
        rgba_from_rgb(rgb_bufs[b], out=d_rgba)
        depth_from_u16(bufs[b], depth_scale, out=d_depth)
        out, ex = P.step()
        ev_used[b].record(cur)
        h_out[:5].copy_(out, non_blocking=True)
        h_out[5] = ex["coords"].shape[0]
        cur.wait_event(ev_copied[1 - b])
        st["k"] = k + 1
    e2e_ms = time_region(e2e_step, args.steps, args.warmup, ws)
    torch.cuda.synchronize()
    del bufs, rgb_bufs
    h2d = h_raw.numel() * 2 + h_rgb.numel()
    h2d_serial = h_depth.numel() * 4 + h_rgba.numel()
    d2h = 5 * 8 + 8

    # ---- breakdown: the update alone, batched vs plain; per-kernel profile of one step
    upd_batched_ms = update_only_timing(P, 5, True)
    upd_plain_ms = update_only_timing(P, 5, False)
    # per-stage device time of one step (events, no profiling)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    ev[0].record(s)
    P.fuse()
    ev[1].record(s)
    P.integrate()
    ev[2].record(s)
    P.update_batched()
    ev[3].record(s)
    P.loss_adjoint()
    ev[4].record(s)
    P.extract()
    ev[5].record(s)
    torch.cuda.synchronize()
    stage = {n: ev[i].elapsed_time(ev[i + 1]) for i, n in enumerate(["fuse", "integrate", "batched_update",
                                                                      "loss_adjoint", "extract"])}
    # per-kernel profiles (library events; graph event nodes inside the batch graph)
    P.integrate()
    V.set_profiling(True)
    P.update_batched()
    prof_upd = V.profile()
    V.set_profiling(True)
    P.integrate()
    prof_int = V.profile()
    V.set_profiling(True)
    P.integrate_plain()
    prof_plain = V.profile()
    V.set_profiling(False)

    from paper_1709_03763_b300.volume import fusion_profile
    fusion_profile(1)
    P.fuse()
    fprof = fusion_profile(0)

    hbm_peak, peak_kind = peaks()
    sm_mhz = clocks.get("sm_mhz") or 2032.0

    # ---- colour keyframe fusion, measured on its own (the step integrates the keyframes'
    # own colour images, as the depth-only path defines it)
    nf = P.K * KAPPA
    col_ms = colour_timing(P, 10, 3)
    col_b = colour_bytes(nf, P.K, w.intr.height, w.intr.width)
    col_gbs = col_b / (col_ms / 1e3) / 1e9
    colour_row = {"ms_per_call": col_ms, "frames": nf, "keyframes": P.K,
                  "keyframes_per_s": ws * P.K / (col_ms / 1e3),
                  "roofline": {"bound": "hbm", "achieved": col_gbs, "peak": hbm_peak, "unit": "GB/s",
                               "frac": col_gbs / hbm_peak, "traffic": None, "peak_kind": peak_kind,
                               "algorithmic_bytes": col_b}}
    # ---- roofline of the dominant kernel: algorithmic bytes per launch / live CUDA-event
    # time per launch, against the measured HBM copy peak; the instruction-issue view
    # beside it uses the FP32 FMA rate measured here
    fma_tps, _ = fp32_peak()
    derived_issue = SMS * SCHEDULERS * LANES * sm_mhz * 1e6 / 1e12
    H, Wd = w.intr.height, w.intr.width
    f_launches = max(fprof["launches"], 1)
    f_frames = fprof["frames"] / f_launches
    n_img = P.K
    cand = {
        # per launch: (ms, launches per step, units per launch, algorithmic bytes per launch)
        # the scatter launches take the KAPPA - 1 frames of each group that are not at the
        # keyframe pose (the first initialises the sums): per launch, their depth read
        # and the sums of the keyframes they feed, written once
        "fuse_kernel": (fprof["ms"] / f_launches, fprof["launches"], f_frames,
                        f_frames * H * Wd * 4 + (f_frames / (KAPPA - 1)) * IMG_BYTES),
        "batch_alloc_kernel": (prof_int["batch_alloc_ms"], 2, n_img,
                               n_img * H * Wd * 4 + prof_int["batch_pairs"] * 20),
        "net_delta_kernel": (prof_upd["batch_net_ms"], 1, n_img,
                             prof_upd["batch_union_blocks"] * 512 * VOXEL_BYTES_RW + n_img * IMG_BYTES
                             + prof_upd["batch_pairs"] * 4),
    }
    dom = max(cand, key=lambda k: cand[k][0] * cand[k][1])
    t_ms, _, units, abytes = cand[dom]
    achieved = abytes / (t_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_kind": peak_kind,
                "traffic": (DRAM_PER_UNIT[dom] * units if dom in DRAM_PER_UNIT else None),
                "traffic_note": "ncu dram__bytes_read+write per unit of the 12-keyframe capture, scaled to the "
                                "launch's units",
                "algorithmic_bytes_per_launch": abytes, "ms_per_launch": t_ms, "units_per_launch": units,
                "kernels": {k: {"ms_per_launch": round(v[0], 5), "launches_per_step": v[1],
                                "GBps": round(v[3] / (v[0] / 1e3) / 1e9, 1),
                                "hbm_frac": round(v[3] / (v[0] / 1e3) / 1e9 / hbm_peak, 4)}
                            for k, v in cand.items()}}
    if dom in WINST_PER_UNIT:
        lane_inst = WINST_PER_UNIT[dom] * LANES * units
        ach_i = lane_inst / (t_ms / 1000.0) / 1e12
        roofline["issue_view"] = {"bound": "alu", "achieved": ach_i, "unit": "T lane instructions/s",
                                  "peak_measured_fp32_fma": fma_tps,
                                  "frac_of_measured": ach_i / fma_tps if fma_tps else None,
                                  "peak_derived": derived_issue, "frac_of_derived": ach_i / derived_issue,
                                  "note": "warp instructions per unit from ncu smsp__inst_executed of the "
                                          "12-keyframe capture; measured peak = sc_measure_fp32_rate"}
    # HBM view of the voxel-update kernels (algorithmic bytes / live time)
    hbm = {}
    if prof_plain["update_launches"]:
        nb = prof_plain["update_blocks"] / prof_plain["update_launches"]
        t = prof_plain["update_ms"] / prof_plain["update_launches"]
        b = nb * 512 * VOXEL_BYTES_RW + IMG_BYTES + nb * 32
        hbm["update_kernel (plain integrate)"] = {"frac": round(b / (t / 1e3) / 1e9 / hbm_peak, 4),
                                                  "ms_per_launch": round(t, 5)}
    for name, pr in (("net_delta_kernel (pose update)", prof_upd), ("net_delta_kernel (integration)", prof_int)):
        if pr["batch_launches"]:
            u = pr["batch_union_blocks"] / pr["batch_launches"]
            t = pr["batch_net_ms"] / pr["batch_launches"]
            b = u * 512 * VOXEL_BYTES_RW + P.K * IMG_BYTES + pr["batch_pairs"] * 4 / pr["batch_launches"]
            hbm[name] = {"frac": round(b / (t / 1e3) / 1e9 / hbm_peak, 4), "ms_per_launch": round(t, 5),
                         "union_blocks": u, "block_item_pairs": pr["batch_pairs"] / pr["batch_launches"]}
    # the whole fusion stage (init, scatter and normalisation launches): its inputs (the
    # 600 depth frames) and outputs (Z*, W* of the 60 keyframes)
    fb = P.K * KAPPA * H * Wd * 4 + P.K * IMG_BYTES
    hbm["fusion stage (600 frames -> 60 keyframes)"] = {"frac": round(fb / (stage["fuse"] / 1e3) / 1e9 / hbm_peak, 4),
                                                       "ms": round(stage["fuse"], 5)}
    roofline["hbm_view"] = hbm

    # ---- Marching Cubes of the corrected volume (after the step's pose update), measured
    # on its own: one call = the slot-count read-back, one kernel launch, count + status
    P.step()
    torch.cuda.synchronize()
    n_blocks = V.info()["allocated_blocks"]
    mc_out = torch.empty((8 << 20, 3, 3), dtype=torch.float32, device=dev)
    mc_ms, mc_kernel_ms, n_tri = mc_timing(V, mc_out, 10, 3)
    mc_b = n_blocks * 512 * 8 + n_tri * 36
    mc_gbs = mc_b / (mc_kernel_ms / 1e3) / 1e9
    mc_row = {"ms_per_call": mc_ms, "kernel_ms": mc_kernel_ms, "blocks": n_blocks, "triangles": n_tri,
              "blocks_per_s": ws * n_blocks / (mc_ms / 1e3),
              "roofline": {"bound": "hbm", "achieved": mc_gbs, "peak": hbm_peak, "unit": "GB/s",
                           "frac": mc_gbs / hbm_peak, "traffic": None, "peak_kind": peak_kind,
                           "algorithmic_bytes": mc_b,
                           "note": "mc_kernel's CUDA-event time (library profile); ms_per_call is the whole "
                                   "call with its two host round trips (slot count, triangle count + status)"}}
    del mc_out

    # ---- the streaming sphere (Section 3) with Eq. 3 vs the m most-moved (Section 4.3)
    from paper_1709_03763_b300 import BlockStore, synthetic
    # a pose-graph correction spread over the trajectory (as after a loop closure): each
    # keyframe moved by a seeded random amount, so the most-moved ones are scattered
    g = synthetic.rng(2, 91)
    w.extra["stream_new_poses"] = np.stack([
        synthetic.perturb_pose(T, math.radians(g.uniform(0.0, 1.0)), g.uniform(0.0, 0.02), g)
        for T in w.kf_poses]).astype(np.float32)
    store = BlockStore(V.info()["allocated_blocks"] + 4096, "rgba8")
    block_bytes = 512 * 12
    stream_row = {"m": STREAM_M, "radius_m": STREAM_RADIUS}
    # the two strategies alternate (one warm-up each, then 10 timed updates each), so
    # that a change of the host's clock during the row affects both alike
    strats = ("consecutive", "topm")
    for strat in strats:
        streaming_protocol(P, V, store, strat, STREAM_M, STREAM_RADIUS)  # warm-up
    runs = {strat: [] for strat in strats}
    for _ in range(10):
        for strat in strats:
            runs[strat].append(streaming_protocol(P, V, store, strat, STREAM_M, STREAM_RADIUS))
    for strat in strats:
        st_ms = statistics.median(r[0] for r in runs[strat])
        _, n_in, n_out, ids = runs[strat][-1]
        stream_row[strat] = {"ms": st_ms, "blocks_in_for_lists": n_in[0], "blocks_in_for_updated_poses": n_in[1],
                             "blocks_out": n_out, "bytes_moved": (sum(n_in) + n_out) * block_bytes,
                             "keyframes": ids}
    # the paper's point (Section 4.3, the 47 % of its results): consecutive keyframes need
    # fewer streamed blocks -- both the blocks their lists name and the blocks their
    # updated poses reach (neighbouring keyframes share most of both)
    cb = stream_row["consecutive"]["blocks_in_for_lists"] + stream_row["consecutive"]["blocks_in_for_updated_poses"]
    tb = stream_row["topm"]["blocks_in_for_lists"] + stream_row["topm"]["blocks_in_for_updated_poses"]
    stream_row["saving_blocks_for_lists"] = 1.0 - (stream_row["consecutive"]["blocks_in_for_lists"] /
                                                   max(1, stream_row["topm"]["blocks_in_for_lists"]))
    stream_row["saving_blocks_in"] = 1.0 - cb / max(1, tb)
    stream_row["saving_time"] = 1.0 - stream_row["consecutive"]["ms"] / stream_row["topm"]["ms"]
    # the bound is the host link: its rate measured here with a pinned 256 MB copy each way
    h_probe = torch.empty(256 << 20, dtype=torch.uint8).pin_memory()
    d_probe = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    for _ in range(2):
        d_probe.copy_(h_probe, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record()
    d_probe.copy_(h_probe, non_blocking=True)
    e1.record()
    h_probe.copy_(d_probe, non_blocking=True)
    e2.record()
    torch.cuda.synchronize()
    link = {"h2d_GBps": (256 << 20) / (e0.elapsed_time(e1) / 1e3) / 1e9,
            "d2h_GBps": (256 << 20) / (e1.elapsed_time(e2) / 1e3) / 1e9}
    del h_probe, d_probe
    cons = stream_row["consecutive"]
    moved_gbs = cons["bytes_moved"] / (cons["ms"] / 1e3) / 1e9
    link_peak = 0.5 * (link["h2d_GBps"] + link["d2h_GBps"])
    stream_row["roofline"] = {"bound": "host link", "achieved": moved_gbs, "peak": link_peak, "unit": "GB/s",
                              "frac": moved_gbs / link_peak, "traffic": None, "peak_kind": "measured here (pinned "
                              "256 MB copies, mean of H2D and D2H)", "link": link,
                              "note": "whole update (median of 10, CUDA events): stream-in of the listed and "
                                      "the newly reached blocks, batch re-integration and stream-out; the "
                                      "re-integration itself is not link traffic"}
    store.close()
    P.integrate()

    # ---- KF_OVRLP keyframe grouping of the 600 frames (Section 4.2), measured on its own
    from paper_1709_03763_b300 import KF_OVRLP, segment_keyframes
    nfr = P.K * KAPPA
    kf_poses_all = w.frame_poses[:nfr]
    for _ in range(2):
        segment_keyframes(KF_OVRLP, (KF_OVRLP_THR,), kf_poses_all, w.intr, w.frames_depth[:nfr])
    torch.cuda.synchronize()
    ts = []
    for _ in range(5):
        t0 = time.perf_counter()
        fk_ov, g_ov = segment_keyframes(KF_OVRLP, (KF_OVRLP_THR,), kf_poses_all, w.intr, w.frames_depth[:nfr])
        ts.append((time.perf_counter() - t0) * 1e3)
    ov_ms = statistics.median(ts)
    ov_b = nfr * w.intr.width * w.intr.height * 4
    kf_row = {"strategy": "KF_OVRLP", "threshold": KF_OVRLP_THR, "ms_per_call": ov_ms, "frames": nfr,
              "keyframes": int(g_ov), "frames_per_s": ws * nfr / (ov_ms / 1e3),
              "roofline": {"bound": "hbm", "achieved": ov_b / (ov_ms / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                           "frac": ov_b / (ov_ms / 1e3) / 1e9 / hbm_peak, "traffic": None, "peak_kind": peak_kind,
                           "algorithmic_bytes": ov_b,
                           "note": "each frame's depth read once; the sequential grouping loop runs on the "
                                   "device (one graph launch with a while node: per step an overlap launch of "
                                   "8-32 frames and a one-warp decision kernel), so it is bound by the steps' "
                                   "launch latency"}}

    # ---- the batching workload (2000 keyframes, 10 pose updates of 10-200 keyframes) and the
    # batched forward + backward of 256 of its keyframes, measured on their own
    batch_row = fb_row = None
    if not args.no_batching:
        torch.cuda.empty_cache()
        batch_row, fb_row = batching_rows(dev, hbm_peak, peak_kind, args.batching_reps, rank == 0, ws)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_sample, w)
        cpu["cpu_model"] = cpu_model()
        cpu["nproc"] = os.cpu_count()
        # the same oracle on one thread, over a smaller sample
        import oracle
        nt = oracle.get_threads()
        oracle.set_threads(1)
        n1 = 2
        last = oracle_reintegration.last_volume
        dt1, _ = oracle_reintegration(n1, steps=1, w=w)
        oracle_reintegration.last_volume = last
        oracle.set_threads(nt)
        cpu["single_thread"] = {"value": n1 / dt1, "unit": UNIT, "cores": 1,
                                "sample": f"{n1} keyframe re-integrations of the same workload, FP64, {dt1:.1f} s"}
        if batch_row is not None:
            spr, thr = oracle_batching_sample(2)
            batch_row["cpu_baseline"] = {"value": 1.0 / spr, "unit": "re-integrations/s", "cores": thr,
                                         "kind": "oracle", "sample": "2 keyframe re-integrations of the batching "
                                         f"workload's first update (640x480, 1 cm, RGBA8), FP64, {2 * spr:.1f} s"}
        kps, threads, dt = oracle_colour(w, P.kf_depth)
        colour_row["cpu_baseline"] = {"value": kps, "unit": "keyframes/s", "cores": threads, "kind": "oracle",
                                      "sample": f"colour fusion of 3 keyframes (10 frames each, 640x480), FP64, "
                                                f"{dt:.1f} s"}
        stream_row["cpu_baseline"] = {"value": cpu["value"] / STREAM_M, "unit": "updates/s", "cores": cpu["cores"],
                                      "kind": "oracle", "sample": f"the oracle's re-integration rate "
                                      f"({cpu['value']:.1f} keyframes/s, the main baseline) for {STREAM_M} "
                                      f"keyframes; the oracle has no streaming (streaming changes no voxel)"}
        ko = oracle_kf(w, 60)
        kf_row["cpu_baseline"] = {"value": ko[0], "unit": "frames/s", "cores": 1, "kind": "oracle",
                                  "sample": f"KF_OVRLP grouping of the first 60 frames, FP64, {ko[1]:.1f} s"}
        om = oracle_mc()
        if om:
            mc_row["cpu_baseline"] = {"value": om[0], "unit": "blocks/s", "cores": 1, "kind": "oracle",
                                      "sample": f"Marching Cubes of {om[1]} blocks of the oracle's re-integrated "
                                                f"volume ({om[2]} triangles), FP64, {om[3]:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "clocks": clocks,
            "config": {"workload": "kinect-scale: 600 frames 640x480 (16-bit sensor depth, 1/5000 m) fused 10 per "
                                   "keyframe into 60 keyframes, "
                                   "voxel 1 cm, trunc 4 cm, 2^20 buckets, one pose update of all 60, "
                                   "1M-point SDF loss + adjoint, block-list extraction",
                       "l2": "inputs (737 MB of depth frames, 74 MB of keyframe colour, 0.3 GB voxel state) exceed L2; no flush",
                       "parallelism": "replicas" if ws > 1 else "single",
                       "colour": "rgba8", "batch_config": cfg},
            "e2e": {"value": ws * P.K / (e2e_ms / 1000.0), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                    "inputs": "600 depth frames as 16-bit sensor depth (1/5000 m) converted on the device, "
                              "60 keyframe colour images as RGB8 expanded to RGBA8 on the device",
                    "pipelining": "raw depth and keyframe colour double-buffered: step k+1's inputs cross on "
                                  "a copy stream while step k computes; each step waits for them before it ends",
                    "serial_float_depth": {"ms_per_step": e2e_serial_ms, "h2d_bytes_per_step": h2d_serial}},
            "gpu_launches_per_step": launches_per_step,
            "update_only": {"batched_ms": upd_batched_ms, "plain_ms": upd_plain_ms,
                            "batched_reint_per_s": P.K / (upd_batched_ms / 1000.0),
                            "plain_reint_per_s": P.K / (upd_plain_ms / 1000.0),
                            "union_blocks": prof_upd["batch_union_blocks"], "pairs": prof_upd["batch_pairs"]},
            "stage_ms": {k: round(v, 4) for k, v in stage.items()},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "rows": {"batching": batch_row, "forward_backward_256": fb_row, "colour_fusion": colour_row,
                     "marching_cubes": mc_row, "keyframe_strategy": kf_row, "streaming": stream_row},
            "setup_s": setup_s,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
