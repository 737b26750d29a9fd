"""Benchmark of the dense-CRF hot path: Frank-Wolfe iterations/s at 500x375, L=21.

One step = one dcrf_qp_fw call of `--iters` Frank-Wolfe iterations over a batch
of `--batch` synthetic VOC-shaped images (500x375, 21 labels, 30 Voronoi
regions), lattices built beforehand (they are reused by every iteration), with
float16 lattice storage.  value = images x iterations / second over all ranks.

Also reported: the plain float32 single-image form, the end-to-end rate
through the C ABI's host-buffer call dcrf_qp_fw_host (uploads, features,
lattice builds, solver and download inside the timed region), the roofline of
the dominant kernel from CUDA events taken on the launching stream in a second
pass over the same steps (the first, un-instrumented pass gives `value`), the
oracle timed on one host core and on all of them, and SM clocks sampled during
the timed region.

Multi-GPU: one process per GPU (torchrun); every rank solves its own batch
(images are independent problems), so there is no data-path collective; only
the timing uses a max-reduction over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

# the oracle baseline is timed on one host thread: pin the BLAS pools before
# numpy loads them (threadpoolctl, when present, limits them again)
for _var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_var, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1608_06192_gb300 import synthetic as S  # noqa: E402

METRIC = "FW iters/s at 500x375, L=21 (batched FP16 vs plain FP32); % HBM roofline"
UNIT = "image-iterations/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--iters", type=int, default=100)
    ap.add_argument("--storage", default="f16", choices=["f16", "f32"])
    ap.add_argument("--width", type=int, default=500)
    ap.add_argument("--height", type=int, default=375)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-all-cores", action="store_true")
    ap.add_argument("--no-lp", action="store_true")
    ap.add_argument("--no-uneven", action="store_true", help="skip the uneven-size batch arm")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the batched other-storage and single-image FP16 arms")
    ap.add_argument("--no-dcneg", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the CCCP and reverse-mode timings")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_seeds(rank: int, batch: int) -> list[int]:
    """Seeds of the images one rank solves: disjoint across ranks (weak scaling)."""
    return [1000 * rank + i for i in range(batch)]


def max_over_ranks(ms: float, dist, world: int, device) -> float:
    """The job's time is the slowest rank's (a MAX all-reduce when world > 1)."""
    if world <= 1:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(world: int, batch: int, iters: int, ms_per_step: float) -> float:
    """Image-iterations per second of the whole job: every rank did batch x iters per step."""
    return world * batch * iters / (ms_per_step / 1000.0)


# ---------------------------------------------------------------------------
# oracle (CPU) timing: the reference arm and the cpu_baseline leg

def oracle_rate(iters: int, seed: int = 0):
    """Oracle Frank-Wolfe on one 500x375 image: (image-iterations/s, seconds, threads)."""
    try:
        from threadpoolctl import threadpool_limits
    except Exception:
        threadpool_limits = None
    if threadpool_limits is not None:
        with threadpool_limits(1):
            return _oracle_rate(iters, seed)
    return _oracle_rate(iters, seed)


def _oracle_rate(iters, seed):
    from oracle import crf, qp
    from oracle import permutohedral as P
    p = S.make_problem(500, 375, 30, 21, seed)
    fb, fs = crf.features(p.rgb, *p.thetas)
    k = P.LatticeGaussian([crf.to_fp32_features(fb), crf.to_fp32_features(fs)], p.weights)
    c = crf.DenseCRF(p.unaries, k)
    qp.frank_wolfe(c, p.y0, 1)                      # warm-up
    t0 = time.perf_counter()
    qp.frank_wolfe(c, p.y0, iters)
    dt = time.perf_counter() - t0
    return iters / dt, dt, 1


def _oracle_worker(seed, iters, barrier, out):
    """One process of the all-cores oracle timing: its own image, timed after a common start."""
    from oracle import crf, qp
    from oracle import permutohedral as P
    p = S.make_problem(500, 375, 30, 21, seed)
    fb, fs = crf.features(p.rgb, *p.thetas)
    k = P.LatticeGaussian([crf.to_fp32_features(fb), crf.to_fp32_features(fs)], p.weights)
    c = crf.DenseCRF(p.unaries, k)
    qp.frank_wolfe(c, p.y0, 1)                      # warm-up
    barrier.wait()
    t0 = time.perf_counter()
    qp.frank_wolfe(c, p.y0, iters)
    out.put(time.perf_counter() - t0)


def oracle_rate_all_cores(iters: int, workers: int):
    """The oracle on every host core at once: one single-threaded process per
    core, each on its own 500x375 image (the images are independent problems).
    Returns (image-iterations/s over all processes, slowest process's seconds)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")                  # never fork a process that holds a CUDA context
    barrier, out = ctx.Barrier(workers), ctx.SimpleQueue()
    procs = [ctx.Process(target=_oracle_worker, args=(100 + w, iters, barrier, out)) for w in range(workers)]
    for q in procs:
        q.start()
    for q in procs:
        q.join(timeout=600)
    if any(q.exitcode != 0 for q in procs):
        return None, None
    dts = [out.get() for _ in range(workers)]
    return workers * iters / max(dts), max(dts)


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def workload_config(B, W, H, T, storage):
    """The workload both arms report (the measured lattice sizes are added by ours)."""
    return {"workload": f"{B} x {W}x{H} synthetic VOC-shaped images per GPU, L=21, "
                        f"{storage} lattice storage, {T} Frank-Wolfe iterations per step",
            "images_per_gpu": B, "iters_per_step": T, "storage": storage, "pixels_per_gpu": B * W * H,
            "l2": "inputs larger than L2 (per-pixel state of the batch is several GB)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    per_step = 3
    oracle_rate(1)
    times = []
    for _ in range(args.warmup):
        oracle_rate(per_step)
    for _ in range(args.steps):
        r, dt, cores = oracle_rate(per_step)
        times.append(dt)
    total = sum(times)
    value = args.steps * per_step / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(args.batch, args.width, args.height, args.iters, args.storage),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "cpu_model": cpu_model(),
                         "sample": f"each step: {per_step} oracle FW iterations (FP64 numpy) on one "
                                   f"{args.width}x{args.height} image of the workload, scaled to image-iterations/s"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if sm:
            busy = [x for x in sm if x > 0.5 * max(sm)] or sm
            out.update(sm_mhz=statistics.median(busy), sm_max_mhz=max(smax), reasons=sorted(reasons),
                       samples=len(sm))
        return out


def measured_traffic(kind, n):
    """DRAM bytes per launch of the pixel kernel from the committed ncu capture
    (profiles/fw_pixel_traffic.json: a 1-pass capture of dram__bytes_read.sum +
    dram__bytes_write.sum on the benchmark's own batch), scaled by pixels when
    the batch differs; None when the kernel's source (csrc/fw_pixel.cuh)
    changed since the capture, or for other kernels."""
    if kind != "fw_pixel":
        return None
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "fw_pixel_traffic.json")))
        import hashlib
        src = open(os.path.join(ROOT, "paper_1608_06192_gb300", "csrc", "fw_pixel.cuh"), "rb").read()
        if hashlib.sha1(src).hexdigest() != rec["source_sha1"]:
            return None
        return int(rec["dram_bytes_per_launch"] * n / rec["pixels"])
    except (OSError, KeyError, ValueError):
        return None


def lp_algorithmic_bytes(n, L, levels, lat_d):
    """Bytes one LP subgradient must move at least (a lower bound: the blur of
    the tagged vertices is left out, their count depends on the level).

    Per label and level and lattice (d+1 corners per point): the tagged keys
    of the node lattices (16 B per incidence), the splat of the right child
    (vertex id + weight, 8 B per incidence), the slice at the left child
    (8 B per incidence) and the point's upper sum U (read + write, 8 B).  Per
    label once: the column sort (key + value read and written, 16 B per
    point) and G (y, phi read, G written: 12 B per point).
    """
    per_level = sum(n * ((d + 1) * 32 + 8) for d in lat_d)
    return L * (levels * per_level + 28 * n)


def algorithmic_bytes(kind, n, L, lat_m, lat_d, storage):
    """Bytes one Frank-Wolfe iteration must move for a kernel kind (all launches of it).

    Per pixel: y read+write and (phi - d) read (12 L), s read+write and c (6),
    vertex id + weight per simplex corner (8 (d+1) per lattice).  Per lattice
    vertex row of Lp labels: the one-hot splat S s in 32-bit fixed point (4),
    B S s and the sliced B S y in the storage type (esz), Ylat and BY in float32.
    The line-search kernel also brings Ylat up to date (the previous step's
    splat folded in); the lattice update then only advances BY.
    """
    Lp = 8 if L <= 8 else (24 if L <= 24 else 64)
    esz = 2 if storage == "f16" else 4
    half_copy = 2 if storage == "f16" else 0
    if kind == "fw_pixel":
        per_px = 12 * L + 6 + sum(8 * (d + 1) for d in lat_d)
        return n * per_px + sum(m * Lp * (esz + 4) for m in lat_m)
    if kind == "fw_blur":
        return sum(m * Lp * (4 + esz) + d * m * Lp * 2 * esz + (d + 1) * 8 * m for m, d in zip(lat_m, lat_d))
    if kind == "fw_latdot":
        # Ylat read and written (the deferred update), S s^{t-1} read and
        # cleared, S s^t read, B S s^t read, the vertex's image
        return sum(m * Lp * (20 + esz) + 4 * m for m in lat_m)
    if kind == "fw_latupd":
        # BY read and written, B S s read, the half copy of BY written
        return sum(m * Lp * (8 + esz + half_copy) + 4 * m for m in lat_m)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist
    from paper_1608_06192_gb300 import _abi as D, build
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    dev = torch.device("cuda", local)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    stream = torch.cuda.Stream(device=dev)
    B, T, W_, H_ = args.batch, args.iters, args.width, args.height
    probs = [S.make_problem(W_, H_, 30, 21, seed=sd) for sd in rank_seeds(rank, B)]
    L = 21
    n = sum(p.n_pixels for p in probs)
    rgb_h = torch.from_numpy(np.concatenate([p.rgb.reshape(-1, 3) for p in probs])).pin_memory()
    phi_h = torch.from_numpy(np.concatenate([p.unaries for p in probs])).pin_memory()
    y0_h = torch.from_numpy(np.concatenate([p.y0 for p in probs])).pin_memory()
    widths, heights = [p.width for p in probs], [p.height for p in probs]
    off = np.concatenate([[0], np.cumsum([p.n_pixels for p in probs])]).astype(np.int64)
    th, wts = probs[0].thetas, probs[0].weights

    with torch.cuda.stream(stream):
        rgb = rgb_h.to(dev, non_blocking=True)
        phi = phi_h.to(dev, non_blocking=True)
        y0 = y0_h.to(dev, non_blocking=True)
        fb, fs = D.dcrf_features(rgb, widths, heights, *th, stream=stream)
        t0 = time.perf_counter()
        lb = D.dcrf_lattice_build(fb, off, stream=stream)
        ls = D.dcrf_lattice_build(fs, off, stream=stream)
        stream.synchronize()
        build_s = time.perf_counter() - t0
        Y = torch.empty_like(y0)

        def step():
            Y.copy_(y0)
            D.dcrf_qp_fw(phi, [lb, ls], wts, Y, T, storage=args.storage, records=False, stream=stream)

        for _ in range(max(3, args.warmup)):
            step()
        stream.synchronize()
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(args.steps):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
        elapsed_ms = max_over_ranks(e0.elapsed_time(e1), dist, world, dev)
        # end to end through the C ABI's host-buffer entry point, timed right
        # after the device-resident steps (same batch, same state): every step
        # uploads the images, unaries and y0 from page-locked memory, builds
        # the features and both lattices, runs the solver and downloads y
        e2e = None
        if not args.no_e2e:
            Yh = torch.empty_like(y0_h).pin_memory()

            def e2e_step():
                D.dcrf_qp_fw_host(rgb_h, phi_h, y0_h, widths, heights, th, wts, T, Y=Yh, storage=args.storage,
                                  stream=stream)

            e2e_step()
            stream.synchronize()
            b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            k = max(1, args.steps)
            b0.record(stream)
            for _ in range(k):
                e2e_step()
            b1.record(stream)
            stream.synchronize()
            e2e_ms = max_over_ranks(b0.elapsed_time(b1) / k, dist, world, dev)
            e2e = {"value": aggregate_rate(world, B, T, e2e_ms), "unit": UNIT,
                   "h2d_bytes_per_step": int(rgb_h.numel() * 4 + phi_h.numel() * 4 + y0_h.numel() * 4),
                   "d2h_bytes_per_step": int(Yh.numel() * 4), "ms_per_step": round(e2e_ms, 3)}

        # per-kernel durations: the same steps again, every launch of the
        # library bracketed by CUDA events on its stream (launched one by one:
        # the hooks keep the solver from replaying its CUDA graph, so this
        # pass is not the one `value` comes from)
        D.profile_enable(True)
        torch.cuda.synchronize()
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0.record(stream)
        for _ in range(args.steps):
            step()
        k1.record(stream)
        torch.cuda.synchronize()
        prof = D.profile_read()
        D.profile_enable(False)
        hooked_ms = k0.elapsed_time(k1) / args.steps
        ms_step = elapsed_ms / args.steps
        value = aggregate_rate(world, B, T, ms_step)

        # roofline of the dominant kernel (CUDA events on the launching stream)
        lat_m, lat_d = [lb.m, ls.m], [5, 2]
        per_iter_launch = {"fw_pixel": 1, "fw_blur": max(lat_d) + 1, "fw_latdot": 1, "fw_latupd": 1}
        roof = None
        kinds = {}
        for kind, (cnt, ms) in prof.items():
            by = algorithmic_bytes(kind, n, L, lat_m, lat_d, args.storage)
            if by and cnt and kind in per_iter_launch:
                per_launch = by / per_iter_launch[kind]
                gbs = per_launch / (ms / cnt / 1000.0) / 1e9
                kinds[kind] = {"launches": cnt, "ms": round(ms, 3), "GB/s": round(gbs, 1),
                               "bytes_per_launch": int(per_launch), "us_per_launch": round(1000 * ms / cnt, 2)}
            else:
                kinds[kind] = {"launches": cnt, "ms": round(ms, 3)}
        dom = max((k for k in kinds if "GB/s" in kinds[k]), key=lambda k: kinds[k]["ms"], default=None)
        if dom is not None:
            ach = kinds[dom]["GB/s"]
            roof = {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(ach / hbm_peak, 4), "peak_source": peak_src,
                    "bytes_per_launch": kinds[dom]["bytes_per_launch"], "traffic": measured_traffic(dom, n)}
        launches = sum(c for c, _ in prof.values())
        kernel_pass = {"ms_per_step": round(hooked_ms, 3),
                       "note": "kernels and roofline: a second pass over the same steps with per-launch CUDA "
                               "events (launched one by one, no graph replay)"}

        # the precision effect at equal batching, and the uneven batch: each
        # arm timed like the headline (graph replay, CUDA events on the
        # stream), then one instrumented step for its pixel-pass roofline
        def arm(lats, phi_, y0_, storage, images, reps):
            Ya = torch.empty_like(y0_)

            def run():
                Ya.copy_(y0_)
                D.dcrf_qp_fw(phi_, lats, wts, Ya, T, storage=storage, records=False, stream=stream)

            for _ in range(2):
                run()
            stream.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(reps):
                run()
            a1.record(stream)
            stream.synchronize()
            ms = a0.elapsed_time(a1) / reps
            D.profile_enable(True)
            run()
            pr = D.profile_read()
            D.profile_enable(False)
            nn = y0_.shape[0]
            cnt, kms = pr.get("fw_pixel", (0, 0.0))
            out = {"value": images * T / (ms / 1000.0), "unit": UNIT, "ms_per_step": round(ms, 3),
                   "pixel_iterations_per_s": nn * T / (ms / 1000.0)}
            by = algorithmic_bytes("fw_pixel", nn, L, [lt.m for lt in lats], [lt.d for lt in lats], storage)
            if cnt:
                per_launch = by                    # one pixel launch per iteration
                gbs = per_launch / (kms / cnt / 1000.0) / 1e9
                out["roofline"] = {"kernel": "fw_pixel", "bound": "hbm", "achieved": round(gbs, 1),
                                   "peak": hbm_peak, "unit": "GB/s", "frac": round(gbs / hbm_peak, 4),
                                   "peak_source": peak_src, "bytes_per_launch": int(per_launch),
                                   "us_per_launch": round(1000 * kms / cnt, 2)}
            return out

        p1 = [probs[0]]
        n1 = p1[0].n_pixels
        l1b = D.dcrf_lattice_build(fb[:n1].contiguous(), [0, n1], stream=stream)
        l1s = D.dcrf_lattice_build(fs[:n1].contiguous(), [0, n1], stream=stream)
        single32 = arm([l1b, l1s], phi[:n1], y0[:n1], "f32", 1, 5)
        plain_fp32 = single32["value"]
        other = "f32" if args.storage == "f16" else "f16"
        precision = None
        if not args.no_precision:
            precision = {
                "note": "lattice storage at equal batching: the batched arms run the headline batch, the single "
                        "arms its first image alone",
                f"batched_{args.storage}": {"value": value, "unit": UNIT, "ms_per_step": round(ms_step, 3)},
                f"batched_{other}": arm([lb, ls], phi, y0, other, B, 3),
                "single_image_f32": single32,
                "single_image_f16": arm([l1b, l1s], phi[:n1], y0[:n1], "f16", 1, 5),
            }
        # the uneven batch: 32 images of W ~ U[240,500] x H ~ U[160,500]
        uneven = None
        if not args.no_uneven:
            pu = S.make_batch(B, 0)
            ou = np.concatenate([[0], np.cumsum([q.n_pixels for q in pu])]).astype(np.int64)
            rgu = torch.from_numpy(np.concatenate([q.rgb.reshape(-1, 3) for q in pu])).to(dev)
            fbu, fsu = D.dcrf_features(rgu, [q.width for q in pu], [q.height for q in pu], *th, stream=stream)
            lub, lus = D.dcrf_lattice_build(fbu, ou, stream=stream), D.dcrf_lattice_build(fsu, ou, stream=stream)
            phu = torch.from_numpy(np.concatenate([q.unaries for q in pu])).to(dev)
            yu = torch.from_numpy(np.concatenate([q.y0 for q in pu])).to(dev)
            uneven = dict(arm([lub, lus], phu, yu, args.storage, B, 3),
                          workload=f"{B} synthetic images, W ~ U[240,500] x H ~ U[160,500] (seed 0), L=21, "
                                   f"{args.storage} lattice storage, {T} Frank-Wolfe iterations per step",
                          pixels=int(ou[-1]), vertices={"bilateral": lub.m, "spatial": lus.m})
            del lub, lus

        # LP subgradient (sort + divide and conquer) on one 500x375 image, L=21
        lp = None
        if not args.no_lp:
            y_lp = torch.from_numpy(S.dirichlet_labels(n1, L, seed=5)).to(dev)
            D.dcrf_lp_subgrad(phi[:n1], y_lp, [l1b, l1s], wts, energy=False, stream=stream)
            stream.synchronize()
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            reps_lp = 2
            for _ in range(reps_lp):
                D.dcrf_lp_subgrad(phi[:n1], y_lp, [l1b, l1s], wts, energy=False, stream=stream)
            c1.record(stream)
            stream.synchronize()
            lp_ms = c0.elapsed_time(c1) / reps_lp
            nlev = int(np.ceil(np.log2(n1)))
            # the same image under a tree (r-HST) label metric (Appendix F):
            # one sorted column per subtree of a three-level tree
            members, c_t = S.hst_tree(L)
            D.dcrf_lp_subgrad_tree(phi[:n1], y_lp, [l1b, l1s], wts, members, c_t, energy=False, stream=stream)
            stream.synchronize()
            c0.record(stream)
            for _ in range(reps_lp):
                D.dcrf_lp_subgrad_tree(phi[:n1], y_lp, [l1b, l1s], wts, members, c_t, energy=False, stream=stream)
            c1.record(stream)
            stream.synchronize()
            tree_ms = c0.elapsed_time(c1) / reps_lp
            # Kleinberg-Tardos rounding of that point (700 phases label every
            # pixel but with probability ~1e-10)
            pl, pt = S.kt_phases(L, 700, seed=6)
            D.dcrf_round_kt(y_lp, pl, pt, count=False, stream=stream)
            stream.synchronize()
            c0.record(stream)
            for _ in range(reps_lp):
                D.dcrf_round_kt(y_lp, pl, pt, count=False, stream=stream)
            c1.record(stream)
            stream.synchronize()
            kt_ms = c0.elapsed_time(c1) / reps_lp
            # 200 projected-subgradient steps (Algorithm 3) from the same point
            Ys = y_lp.clone()
            c0.record(stream)
            D.dcrf_lp_solve(phi[:n1], [l1b, l1s], wts, Ys, 200, energies=False, stream=stream)
            c1.record(stream)
            stream.synchronize()
            solve_ms = c0.elapsed_time(c1)
            lp_bytes = lp_algorithmic_bytes(n1, L, nlev, [l1b.d, l1s.d])
            lp_gbs = lp_bytes / (lp_ms / 1000.0) / 1e9
            lp = {"workload": "one 500x375 image, L=21, y ~ Dirichlet(0.5), bilateral + spatial lattices",
                  "ms_per_subgradient": round(lp_ms, 3), "subgradients_per_s": round(1000.0 / lp_ms, 2),
                  "label_levels_per_s": round(L * nlev * 1000.0 / lp_ms, 1),
                  "effective_GBps": round(lp_gbs, 1), "bytes_per_subgradient": int(lp_bytes),
                  "roofline": {"bound": "hbm", "achieved": round(lp_gbs, 1), "peak": hbm_peak, "unit": "GB/s",
                               "frac": round(lp_gbs / hbm_peak, 4), "peak_source": peak_src},
                  "projected_subgradient_200_steps": {"ms": round(solve_ms, 1),
                                                      "ms_per_step": round(solve_ms / 200, 3)},
                  "tree_metric": {"tree": "r-HST, r=2: 2 halves, groups of 4, %d leaves (%d subtrees)"
                                          % (L, len(c_t)),
                                  "ms_per_subgradient": round(tree_ms, 3),
                                  "subtree_levels_per_s": round(len(c_t) * nlev * 1000.0 / tree_ms, 1)},
                  "kt_rounding": {"phases": 700, "ms": round(kt_ms, 4)}}

        # CCCP for negative semi-definite compatibilities (Section 5.2) on the
        # same batch: one filter (both blur directions) and one per-pixel
        # projection per outer step
        dcneg = None
        if not args.no_dcneg:
            outer = 10
            Yn = torch.empty_like(y0)
            Yn.copy_(y0)
            D.dcrf_dc_neg(phi, [lb, ls], wts, Yn, 2, 0, storage=args.storage, energies=False, stream=stream)
            stream.synchronize()
            d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            Yn.copy_(y0)
            d0.record(stream)
            D.dcrf_dc_neg(phi, [lb, ls], wts, Yn, outer, 0, storage=args.storage, energies=False, stream=stream)
            d1.record(stream)
            stream.synchronize()
            dn_ms = d0.elapsed_time(d1)
            dcneg = {"workload": f"same batch ({B} x {W_}x{H_}), L=21, Potts, {args.storage} lattice storage, "
                                 f"{outer} outer steps + the final energy",
                     "ms_per_outer_step": round(dn_ms / (outer + 1), 3),
                     "image_outer_steps_per_s": round(B * (outer + 1) / (dn_ms / 1000.0), 1)}

        # CCCP on the generic DC relaxation (Section 5.1) at 320x213, L=21, FP32,
        # 10 outer x 50 inner steps, and reverse mode through 10 unrolled
        # Frank-Wolfe iterations on 8 images of 320x213 (forward recompute +
        # backward), each a separate timed region
        cccp = backward = None
        if not args.no_extras:
            def small_batch(k, seed0):
                pr = [S.make_problem(320, 213, 30, 21, seed=seed0 + i) for i in range(k)]
                nn = [q.n_pixels for q in pr]
                of = np.concatenate([[0], np.cumsum(nn)]).astype(np.int64)
                rg = torch.from_numpy(np.concatenate([q.rgb.reshape(-1, 3) for q in pr])).to(dev)
                f_b, f_s = D.dcrf_features(rg, [q.width for q in pr], [q.height for q in pr], *th, stream=stream)
                return (pr, D.dcrf_lattice_build(f_b, of, stream=stream), D.dcrf_lattice_build(f_s, of, stream=stream),
                        torch.from_numpy(np.concatenate([q.unaries for q in pr])).to(dev),
                        torch.from_numpy(np.concatenate([q.y0 for q in pr])).to(dev))

            def timed(fn):
                fn()
                stream.synchronize()
                x0, x1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                x0.record(stream)
                fn()
                x1.record(stream)
                stream.synchronize()
                return x0.elapsed_time(x1)

            pc, cb, cs, cphi, cy0 = small_batch(1, 7000 + rank)
            Yc = torch.empty_like(cy0)

            def run_cccp():
                Yc.copy_(cy0)
                D.dcrf_qp_fw(cphi, [cb, cs], wts, Yc, 50, records=False, stream=stream)
                D.dcrf_dc_cccp(cphi, [cb, cs], wts, Yc, 10, 50, energies=False, stream=stream)

            c_ms = timed(run_cccp)
            cccp = {"workload": "one 320x213 image, L=21, FP32: 50 QP Frank-Wolfe iterations, then CCCP "
                                "10 outer x 50 inner", "ms": round(c_ms, 3),
                    "fw_iterations_per_s": round(550 / (c_ms / 1000.0), 1)}
            pg, gb, gs, gphi, gy0 = small_batch(8, 8000 + rank)
            ybar = torch.randn(gy0.shape, generator=torch.Generator().manual_seed(1)).to(dev)
            g_ms = timed(lambda: D.dcrf_qp_fw_backward(gphi, [gb, gs], wts, gy0, ybar, 10, stream=stream))
            backward = {"workload": "8 x 320x213, L=21: gradient of <ybar, y^10> in the unaries and the two "
                                    "kernel weights through 10 unrolled Frank-Wolfe iterations (forward recompute "
                                    "included)", "ms": round(g_ms, 3),
                        "images_per_s": round(8 / (g_ms / 1000.0), 1)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, dt, cores = oracle_rate(20)
        cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "20 oracle Frank-Wolfe iterations on one 500x375 image (FP64 numpy)",
               "seconds": round(dt, 2), "cpu_model": cpu_model(), "host_cores": os.cpu_count()}
        workers = os.cpu_count() or 1
        if workers > 1 and not args.no_cpu_all_cores:
            ra, dta = oracle_rate_all_cores(5, workers)
            if ra is not None:
                cpu["all_cores"] = {"value": ra, "unit": UNIT, "cores": workers,
                                    "sample": "%d processes, one per core, 5 oracle Frank-Wolfe iterations each on "
                                              "its own 500x375 image" % workers, "seconds": round(dta, 2)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": dict(workload_config(B, W_, H_, T, args.storage),
                           vertices={"bilateral": lb.m, "spatial": ls.m}, lattice_build_s=round(build_s, 4)),
            "plain_fp32_single_image": {"value": plain_fp32, "unit": UNIT},
            "precision": precision,
            "uneven_batch": uneven,
            "lp_subgrad": lp,
            "dc_neg": dcneg,
            "cccp": cccp,
            "backward": backward,
            "roofline": roof,
            "kernels": kinds,
            "kernel_pass": kernel_pass,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
