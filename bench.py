#!/usr/bin/env python
"""Throughput of the Tucker-FFT VIE operator product (Eq. 7-11) on GB300.

One step = one batched operator product y = Kop x over nb = 16 right-hand
sides (ports) of the 512 x 512 x 24 eSFQ-like multilayer block (seeded
synthetic structure shaped like the paper's eSFQ subsystem, Sec. III.C: four
metal layers, wiring, vias and a perforated ground plane, 0.5 um voxels,
P = 1024 x 1024 x 48): the Tucker restore of the kernel spectra (Eq. 10),
the zero-padded forward 3-D FFT of the five basis grids, the 5 x 5 block
multiply, the inverse FFT with truncation (Eq. 9), the two-fluid diagonal
(Eq. 3, 22-23) and the incidence A / A^T apply (Eq. 7). FP32 complex is the
headline; the FP64 product is timed on the same workload for comparison.

Metric: voxel-matvecs/s = (sum over the batch of Kx*Ky*Kz) * steps / time.
L2 is flushed (a 512 MB write) before every timed step; each step is timed
by CUDA events on the library's stream.

--impl reference times the CPU FP64 oracle (scipy.fft) on the same workload
(one right-hand side per step) on the host cores; it is the only arm that
runs the oracle besides the cpu_baseline block. The oracle's set-up (its
quadrature of the unit kernels, their circulant spectra and the 5 x 5 block
spectra, all independent of the right-hand side) runs once, untimed.

The whole-solve block times port solves of the 256 x 256 x 8 meander (by
default; --solve-workload) with the spectra resident and with the Tucker
restore in every product (Sec. II.B.2).

Multi-GPU (torchrun): replicas only -- every rank runs its own batch (weak
scaling); the ranks only exchange their timings.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "voxel-matvecs/s of Tucker-FFT VIE operator, FP32+refine vs FP64, % HBM peak"
UNIT = "voxel-matvecs/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="svh", choices=["svh", "reference"])
    p.add_argument("--nb", type=int, default=None,
                   help="right-hand sides per step (default: 16 for esfq512, 4 meander256, 2 pair128, 1 strip16)")
    p.add_argument("--workload", default="esfq512", choices=["meander256", "esfq512", "pair128", "strip16"])
    p.add_argument("--solve-workload", default="meander256",
                   choices=["meander256", "esfq512", "pair128", "strip16", "none"],
                   help="structure of the whole-solve timing block (none: skip it)")
    p.add_argument("--tucker-tol", type=float, default=1e-8)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--tiles", default=None,
                   help="comma-separated FFT tile choices (7 values, as svh_autotune reports) "
                        "instead of running the autotuner (e.g. for profiling)")
    p.add_argument("--with-tucker-sweep", action="store_true",
                   help="add CR / CO of the Tucker-compressed spectra vs tolerance on plates and cubes")
    p.add_argument("--no-batch", action="store_true",
                   help="skip the persistent batched product over the 64 cfg-3 structures")
    a = p.parse_args()
    if a.nb is None:
        a.nb = {"esfq512": 16, "meander256": 4, "pair128": 2, "strip16": 1}[a.workload]
    return a


def structure(name):
    import svh_synth as S
    if name == "meander256":
        return S.meander_cfg2(), "meander 256x256x8 over a holed ground plane (seed 202), 0.1 um voxels"
    if name == "esfq512":
        return S.esfq_cfg5(), "eSFQ-like 512x512x24 multilayer block (seed 505), 0.5 um voxels"
    if name == "pair128":
        return S.pair_cfg4(), "two overlapping meanders 128x128x16, log-normal lambda (seed 404), 0.1 um voxels"
    return S.strip_cfg1(), "strip 16x16x4 (1024 voxels), 0.1 um"


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as td
        td.init_process_group("gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as td
        td.barrier()


def allmax(ws, v):
    if ws == 1:
        return v
    import torch
    import torch.distributed as td
    t = torch.tensor([float(v)], dtype=torch.float64)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        self.proc.wait()
        self.f.flush()
        self.f.seek(0)
        rows = [l.strip().split(",") for l in self.f.read().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                for n, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


TF32_PER_BF16 = 1.1 / 2.25   # nominal dense tensor rates per GPU (TF32 / BF16)


def tensor_peak_tf32():
    """TF32 tensor peak: the measured cuBLAS bf16 burst rate x the nominal TF32/BF16 ratio."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]) * TF32_PER_BF16, "measured bf16 x nominal tf32/bf16"
    except Exception:
        return 1900.0 * TF32_PER_BF16, "fallback bf16 x nominal tf32/bf16"


def restore_flops(info, ranks):
    """Algorithmic FP32 flops of one restore of all 7 spectra (mode 3 folded into the core at
    load): stage 1 2 Hx Hz d2 d1, stage 2 2 Hz Hy Hx d2 per kernel. The tensor cores execute
    3x this in TF32 (hi/lo split)."""
    Hx, Hy, Hz = info["Hx"], info["Hy"], info["Hz"]
    return sum(2.0 * Hx * Hz * int(r[1]) * int(r[0]) + 2.0 * Hz * Hy * Hx * int(r[1]) for r in ranks)


def pass_bytes(info, nb, csz, fused=False, zk_planes=0):
    """Algorithmic HBM bytes of each pass for one batched call (compulsory reads + writes).
    fused: the y/z/y passes run as one kernel (reported under z_pass) that reads and
    writes only the active x-lines and reads the spectra. zk_planes > 0: the direct z pass,
    which reads 7 z-space kernels of zk_planes planes (FP32) instead of the octant spectra
    (made from them after each restore: read the spectra, write the kernels)."""
    K, M = info["K"], info["M"]
    nza, nrows = info["n_active_planes"], info["n_active_rows"]
    Kx, Px, Py = info["Kx"], info["Px"], info["Py"]
    Ht = info["Hx"] * info["Hy"] * info["Hz"]
    rows_line = 5 * nrows * Px * csz          # all active x-lines of one item, padded
    planes = 5 * nza * Py * Px * csz          # all active planes after the y transform
    vidx = 8 * nrows + 4 * K                  # per active row: first voxel and count; per voxel: x
    if fused:
        return {
            "tucker_rebuild": 7 * Ht * 4,
            "x_fwd": nb * (5 * K * csz + rows_line) + vidx,
            "y_fwd": 0,
            "z_pass": nb * 2 * rows_line + 7 * Ht * csz // 2 + 4 * nrows,
            "y_inv": 0,
            "x_inv_epilogue": nb * (rows_line + 5 * K * csz + 5 * K * csz + M * csz) + vidx + 40 * K,
            "node_rows": nb * (5 * K * csz + M * csz) + 9 * M,
        }
    zk = 7 * info["Hx"] * info["Hy"] * zk_planes * 4
    return {
        "tucker_rebuild": 7 * Ht * 4 + (7 * Ht * 4 + zk if zk_planes else 0),
        "x_fwd": nb * (5 * K * csz + rows_line) + vidx,
        "y_fwd": nb * (rows_line + planes),
        "z_pass": nb * 2 * planes + (zk if zk_planes else 7 * Ht * csz // 2),
        "y_inv": nb * (planes + rows_line),
        "x_inv_epilogue": nb * (rows_line + 5 * K * csz + 5 * K * csz + M * csz) + vidx + 40 * K,
        "node_rows": nb * (5 * K * csz + M * csz) + 9 * M,
    }


# FP32 peak of the CUDA cores: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.07 GHz (maximum SM clock)
FP32_ALU_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def fused_flops(info, nb):
    """Algorithmic FP32 flops of the fused y/z/y kernel for one batched call: complex FFTs
    counted as 5 N log2 N (the usual convention), the 5 x 5 block multiply as 17
    complex-by-real multiply-adds (68 flops) per (ky, kz) point."""
    import math
    Px, Py, Pz, nza = info["Px"], info["Py"], info["Pz"], info["n_active_planes"]
    fy = 5 * Py * math.log2(Py)
    fz = 5 * Pz * math.log2(Pz)
    per_kx = 2 * 5 * nza * fy + 5 * Py * 2 * fz + Py * Pz * 68
    return nb * Px * per_kx


def kernel_sources_sha():
    """Hash of every library source: ncu counters recorded for another version are not used."""
    import hashlib
    d = os.path.join(ROOT, "paper_2105_08627_gb300", "csrc")
    hsh = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        hsh.update(open(os.path.join(d, f), "rb").read())
    return hsh.hexdigest()[:16]


def traffic_from_profiles(kernel, workload):
    """DRAM bytes per launch recorded from ncu for this kernel and workload, if current."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"traffic_{workload}.txt")
    if not os.path.exists(path):
        return None
    sha = kernel_sources_sha()
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("csrc_sha256_16") != sha:
        return None
    v = vals.get(f"{kernel}_dram_bytes_per_launch")
    return float(v) if v else None


def oracle_setup(s):
    """The oracle's right-hand-side-independent set-up for a structure: grid, FFT sizes,
    the 7 circulant spectra and the 5 x 5 block spectra (kernels by the oracle's own
    quadrature, its z planes in worker processes)."""
    from oracle import geometry as G
    from oracle import greens as gr
    from oracle import operator as op
    g = G.build_grid(s)
    P = (op.fft_size(g.Kx), op.fft_size(g.Ky), op.fft_size(g.Kz))
    T = gr.toeplitz_octant(g.Kx, g.Ky, g.Kz, processes=os.cpu_count() or 1)
    S7 = op.spectra(gr.signed_from_octant(T), P)
    Zh = op.block_spectra(S7)
    return g, P, S7, Zh


def cpu_baseline(s, min_s=10.0, max_s=30.0):
    """The oracle's FP64 FFT product timed on the host cores (bounded sample)."""
    import svh_synth as S
    from oracle import operator as op
    t0 = time.perf_counter()
    g, P, S7, Zh = oracle_setup(s)
    t_setup = time.perf_counter() - t0
    cores = os.cpu_count()
    x = S.random_complex(7, g.N)
    om = 2 * np.pi * s.freqs[0]
    op.apply_K_fft(g, S7, x, om, P, workers=cores, Zh=Zh)     # warm-up
    n, t0 = 0, time.perf_counter()
    while True:
        op.apply_K_fft(g, S7, x, om, P, workers=cores, Zh=Zh)
        n += 1
        el = time.perf_counter() - t0
        if el >= min_s or el + el / n > max_s:
            break
    return {"value": g.Kx * g.Ky * g.Kz * n / el, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} single-vector FP64 products of the same structure (oracle: numpy + "
                      f"scipy.fft workers={cores}), {el:.1f} s; oracle set-up (kernel quadrature, "
                      f"circulant and block spectra) {t_setup:.0f} s untimed"}


def run_reference(args):
    ws, rank, _ = dist()
    if rank != 0:
        return 0
    import svh_synth as S
    from oracle import operator as op
    s, desc = structure(args.workload)
    t0 = time.perf_counter()
    g, P, S7, Zh = oracle_setup(s)
    t_setup = time.perf_counter() - t0
    cores = os.cpu_count()
    x = S.random_complex(7, g.N)
    om = 2 * np.pi * s.freqs[0]
    for _ in range(args.warmup):
        op.apply_K_fft(g, S7, x, om, P, workers=cores, Zh=Zh)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        op.apply_K_fft(g, S7, x, om, P, workers=cores, Zh=Zh)
    el = time.perf_counter() - t0
    Kt = g.Kx * g.Ky * g.Kz
    val = Kt * args.steps / el
    sample = (f"{args.steps} single-vector FP64 products (oracle: numpy + scipy.fft workers={cores}); "
              f"one right-hand side per step instead of {args.nb}; oracle set-up (kernel quadrature, "
              f"circulant and block spectra) {t_setup:.0f} s untimed")
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128 (fp64 complex)",
           "data": "synthetic",
           "config": {"workload": desc, "Kx": g.Kx, "Ky": g.Ky, "Kz": g.Kz, "K": g.K, "N": g.N, "nb": 1,
                      "precision": "fp64", "parallelism": f"replicas x{args.gpus}"},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def time_steps(h, torch, omega, x, y, steps, flush, profile=False):
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    if profile:
        h.profile_begin(steps)
    for k in range(steps):
        flush.fill_(k & 0xFF)
        evs[k][0].record()
        h.matvec(omega, x, y)
        evs[k][1].record()
    torch.cuda.synchronize()
    prof = h.profile_end() if profile else None
    return sum(a.elapsed_time(b) for a, b in evs), prof


def run_batch(torch, svh, S, args):
    """The 64 seeded cfg-3 structures (uneven grids 32..128 x 32..128 x 8..16, 4-8 ports each),
    every port at the three frequencies 1, 10, 50 GHz as its own right-hand side, all products
    in one persistent, graph-captured launch of the batch queue."""
    items = S.batch_cfg3()
    stream = torch.cuda.current_stream().cuda_stream
    hs, xs, ys, oms, kts = [], [], [], [], []
    t0 = time.perf_counter()
    for i, it in enumerate(items):
        h = svh.Handle(0, stream)
        h.setup_structure(it)
        h.generate_toeplitz()
        hs.append(h)
    setup = time.perf_counter() - t0
    b = svh.Batch(0)
    rhs = 0
    for i, (h, it) in enumerate(zip(hs, items)):
        b.add(h)
        info = h.info()
        nb = max(1, info["nports"]) * len(it.freqs)
        rhs += nb
        kts.append(nb * info["Kx"] * info["Ky"] * info["Kz"])
        xs.append(torch.from_numpy(S.random_complex(i, (nb, info["N"])).astype(np.complex64)).cuda())
        ys.append(torch.empty_like(xs[-1]))
        oms.append(2 * np.pi * np.tile(np.asarray(it.freqs, np.float64), nb // len(it.freqs)))
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    mode_ms = b.autotune(oms, xs, ys, svh.SVH_FP32)     # persistent queue vs per-structure chains
    for _ in range(max(3, args.warmup)):
        b.matvec(oms, xs, ys, svh.SVH_FP32)
    b.sync()
    bs = torch.cuda.ExternalStream(b.stream)
    tot = 0.0
    for k in range(args.steps):
        flush.fill_(k & 0xFF)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(bs)
        b.matvec(oms, xs, ys, svh.SVH_FP32)
        e1.record(bs)
        b.sync()
        tot += e0.elapsed_time(e1)
    vox = sum(kts)
    out = {"value": vox * args.steps / (tot / 1e3), "unit": UNIT, "ms_per_step": tot / args.steps,
           "structures": len(items), "right_hand_sides": rhs, "sum_nb_Kt": int(vox),
           "mode": ["persistent queue", "per-structure chains"][b.mode],
           "autotune_ms_per_launch": {"persistent queue (one kernel)": float(mode_ms[0]),
                                      "per-structure chains (one graph)": float(mode_ms[1])},
           "launch": "one CUDA graph per step: mode 0 = one persistent kernel (device work queue over "
                     "every pass of every structure), mode 1 = every structure's launch sequence on "
                     "16 forked streams", "setup_s": setup}
    b.close()
    for h in hs:
        h.close()
    return out


def tucker_compression_ratio(H, ranks):
    """CR of Sec. III.B: values of the 7 octant spectra (H = (Hx, Hy, Hz)) over the values of
    their Tucker cores and factor matrices (ranks[u] = (d1, d2, d3)); both stored in FP32."""
    full = 7 * H[0] * H[1] * H[2]
    comp = sum(int(d1 * d2 * d3 + H[0] * d1 + H[1] * d2 + H[2] * d3) for d1, d2, d3 in ranks)
    return full / comp


def run_tucker_sweep(torch, svh, S):
    """Compression ratio and restore overhead of the Tucker-compressed kernel
    spectra (Sec. III.B.1, Figs. 2-3) on fully occupied plates (4 voxels thick)
    and cubes with 1 um voxels, at tol 1e-4, 1e-6, 1e-8.
    CR = bytes of the 7 octant spectra / bytes of their Tucker cores and factors
    (both FP32); CO = time of the device restore of all 7 (svh_rebuild_spectra)
    / time of one product (one right-hand side, resident spectra)."""
    out = []
    cases = [("plate", n, n, 4) for n in (128, 256, 512)] + [("cube", n, n, n) for n in (32, 64, 96)]
    stream = torch.cuda.current_stream().cuda_stream
    for kind, Kx, Ky, Kz in cases:
        st = S.bar(Kx, Ky, Kz, 0, Kx - 1, 0, Ky - 1, 0, Kz - 1, dx=1e-6)   # inclusive bounds: the full box
        h = svh.Handle(0, stream)
        h.setup_structure(st)
        h.generate_toeplitz()
        info = h.info()
        H = (info["Hx"], info["Hy"], info["Hz"])
        x = torch.from_numpy(S.random_complex(1, (1, info["N"])).astype(np.complex64)).cuda()
        y = torch.empty_like(x)
        om = 2 * np.pi * 1e9

        def timed(fn, reps=5):
            fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        for tol in (1e-4, 1e-6, 1e-8):
            ranks = h.tucker_compress(tol)
            h.set_kernel_mode(svh.SVH_KERNELS_RESIDENT)
            t_restore = timed(h.rebuild_spectra)
            t_prod = timed(lambda: h.matvec(om, x, y))
            out.append({"structure": kind, "K": [Kx, Ky, Kz], "Kt": Kx * Ky * Kz, "tol": tol,
                        "ranks_G00": [int(v) for v in ranks[0]], "max_rank_G00": int(ranks[0].max()),
                        "max_rank_all": int(ranks.max()), "CR": tucker_compression_ratio(H, ranks),
                        "CO": t_restore / t_prod,
                        "restore_ms": t_restore, "product_ms": t_prod})
        h.close()
    return out


def run_solves(torch, svh, args, h_main, s_main, desc_main):
    if args.solve_workload == args.workload:
        hs, s, desc, own = h_main, s_main, desc_main, False
    else:
        s, desc = structure(args.solve_workload)
        hs = svh.Handle(h_main.device, torch.cuda.current_stream().cuda_stream)
        hs.setup_structure(s)
        hs.generate_toeplitz()
        hs.tucker_compress(args.tucker_tol)
        own = True
    out = {"workload": desc, "note": "GMRES(50), FP32 products in FP64 refinement (RRE 1e-8), "
                                      "Schur solves by AMG-CG on the device (1e-8)"}
    for mode, name in ((svh.SVH_KERNELS_RESIDENT, "resident"), (svh.SVH_KERNELS_TUCKER_REBUILD, "tucker_restore")):
        hs.set_kernel_mode(mode)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = hs.solve([s.freqs[0]])
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        st = res["stats"]
        out[name] = {"seconds": wall, "setup_s": st["setup_seconds"], "iterations": st["iterations"],
                     "refinements": st["refinements"], "final_rre": st["final_rre"],
                     "amg_avg_cg_iterations": st["amg_avg_iterations"],
                     "L_pH": float(res["L"][0, 0, 0] * 1e12)}
    hs.set_kernel_mode(svh.SVH_KERNELS_TUCKER_REBUILD)
    if own:
        hs.close()
    return out


def run_svh(args):
    ws, rank, local = dist()
    import torch

    import svh_synth as S
    from paper_2105_08627_gb300 import build, svh
    torch.cuda.set_device(local)
    build.build()
    s, desc = structure(args.workload)
    stream = torch.cuda.current_stream().cuda_stream
    h = svh.Handle(local, stream)
    h.setup_structure(s)
    t_setup = time.perf_counter()
    h.generate_toeplitz()
    ranks = h.tucker_compress(args.tucker_tol)
    h.set_kernel_mode(svh.SVH_KERNELS_TUCKER_REBUILD)
    t_setup = time.perf_counter() - t_setup
    info = h.info()
    N, nb = info["N"], args.nb
    if args.tiles:
        tiles = np.array([int(v) for v in args.tiles.split(",")], np.int32)
        for p_, v_ in enumerate(tiles):
            h.set_pass_variant(p_, int(v_))
    else:
        tiles, tile_ms = h.autotune(nb)     # FFT tile variants, timed once before the run
    Kt = info["Kx"] * info["Ky"] * info["Kz"]
    omega = 2 * np.pi * s.freqs[0]
    x = torch.from_numpy(S.random_complex(1000 + rank, (nb, N)).astype(np.complex64)).cuda()
    y = torch.empty_like(x)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        flush.fill_(1)
        h.matvec(omega, x, y)
    torch.cuda.synchronize()
    barrier(ws)
    clk = Clocks(local)
    clk.start()
    ms, _ = time_steps(h, torch, omega, x, y, args.steps, flush)
    clocks = clk.stop()
    ms = allmax(ws, ms)
    value = ws * nb * Kt * args.steps / (ms / 1e3)
    # per-pass durations (CUDA events on the library's stream) over a second identical region
    _, (pass_ms, ncalls) = time_steps(h, torch, omega, x, y, args.steps, flush, profile=True)
    cnt, cho = h.pass_variants()
    fused = bool(cnt[5] == 2 and cho[5] == 1)
    zdirect = not fused and int(cho[2]) == 3
    nb_launch = nb
    zact = np.nonzero(s.occ.reshape(s.occ.shape[0], -1).any(axis=1))[0]
    zspan = int(zact[-1] - zact[0] + 1) if len(zact) else 0
    pb = pass_bytes(info, nb_launch, 8, fused, zk_planes=zspan if zdirect else 0)
    dom = max((k for k in pass_ms if k != "tucker_rebuild"), key=lambda k: pass_ms[k])
    per_launch_ms = pass_ms[dom] / ncalls
    peak, peak_kind = peaks()
    achieved = pb[dom] / (per_launch_ms / 1e3) / 1e9
    traffic = traffic_from_profiles(dom, args.workload)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": peak_kind,
                "path": "fused y/z/y" if fused else ("separate passes, direct z" if zdirect else "separate passes"),
                "algorithmic_bytes_per_launch": pb[dom], "avg_launch_ms": per_launch_ms,
                "share_of_step": pass_ms[dom] / sum(pass_ms.values()),
                "pass_ms_per_step": {k: v / ncalls for k, v in pass_ms.items()},
                "step_model_bytes": sum(pass_bytes(info, nb, 8, fused, zk_planes=zspan if zdirect else 0).values()),
                "step_model_frac": sum(pass_bytes(info, nb, 8, fused, zk_planes=zspan if zdirect else 0).values())
                / (ms / args.steps / 1e3) / 1e9 / peak}
    # the restore (tensor cores): TF32 MMA flops (3 per algorithmic flop) over its event time
    rf = restore_flops(info, ranks)
    t_rb = pass_ms["tucker_rebuild"] / ncalls
    tpk, tpk_kind = tensor_peak_tf32()
    roofline["restore"] = {"bound": "tensor", "kernel": "k_tc_restore (2 launches)", "unit": "TFLOP/s",
                           "algorithmic_fp32_flops": rf, "tf32_mma_flops": 3 * rf, "avg_ms": t_rb,
                           "achieved": 3 * rf / (t_rb / 1e3) / 1e12, "peak": tpk, "peak_source": tpk_kind,
                           "frac": 3 * rf / (t_rb / 1e3) / 1e12 / tpk}
    if fused and dom == "z_pass":
        # the fused kernel keeps its grids in shared memory: its bound is the FP32 ALUs
        fl = fused_flops(info, nb)
        tf = fl / (per_launch_ms / 1e3) / 1e12
        roofline.update({"bound": "alu", "achieved": tf, "peak": FP32_ALU_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": tf / FP32_ALU_PEAK_TFLOPS, "peak_source": "derived: 152 SM x 128 FP32 x 2 x 2.07 GHz",
                         "algorithmic_flops_per_launch": fl,
                         "hbm_view": {"achieved_GBs": achieved, "frac": achieved / peak}})
    # FP64 product on the same workload
    fp64 = None
    if not args.no_fp64:
        x64 = x.to(torch.complex128)
        y64 = torch.empty_like(x64)
        for _ in range(2):
            h.matvec(omega, x64, y64)
        n64 = max(3, args.steps // 4)
        ms64, _ = time_steps(h, torch, omega, x64, y64, n64, flush)
        ms64 = allmax(ws, ms64)
        fp64 = {"value": ws * nb * Kt * n64 / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64 / n64,
                "steps": n64}
        del x64, y64
    # end to end through the host-memory entry point (pinned buffers, copies inside the timing)
    e2e = None
    if not args.no_e2e:
        xh = torch.empty((nb, N), dtype=torch.complex64, pin_memory=True)
        yh = torch.empty((nb, N), dtype=torch.complex64, pin_memory=True)
        xh.copy_(x.cpu())
        for _ in range(2):
            h._ck(svh.lib().svh_matvec_host(h._h, omega, nb, svh._P(xh.data_ptr()), svh._P(yh.data_ptr()),
                                            svh.SVH_FP32), "svh_matvec_host")
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            h._ck(svh.lib().svh_matvec_host(h._h, omega, nb, svh._P(xh.data_ptr()), svh._P(yh.data_ptr()),
                                            svh.SVH_FP32), "svh_matvec_host")
        el = allmax(ws, time.perf_counter() - t0)
        e2e = {"value": ws * nb * Kt * args.steps / el, "unit": UNIT,
               "h2d_bytes_per_step": nb * N * 8, "d2h_bytes_per_step": nb * N * 8,
               "entry_point": "svh_matvec_host (pinned host buffers)"}
    # whole port solves (FP32 products inside FP64 refinement, RRE 1e-8) of the solve structure,
    # with the spectra resident and with the Tucker restore in every product (Sec. II.B.2)
    solve = None
    if args.solve_workload != "none":
        solve = run_solves(torch, svh, args, h, s, desc)
    sweep = None
    if args.with_tucker_sweep and rank == 0:
        sweep = run_tucker_sweep(torch, svh, S)
    batch = None
    if not args.no_batch and rank == 0:
        batch = run_batch(torch, svh, S, args)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(s)
    # restore (2 tensor-core GEMM stages) + FFT passes (5 separate, or x / fused y-z-y / x) + node rows
    launches_per_step = 2 + (3 if fused else 5) + 1
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "c64 (fp32 complex)", "data": "synthetic",
               "config": {"workload": desc, "Kx": info["Kx"], "Ky": info["Ky"], "Kz": info["Kz"],
                          "P": [info["Px"], info["Py"], info["Pz"]], "K": info["K"], "M": info["M"],
                          "N": N, "nb": nb, "precision": "fp32", "kernel_spectra": "Tucker restore every step",
                          "tucker_tol": args.tucker_tol, "tucker_ranks_G00": ranks[0].tolist(),
                          "l2": "flushed before every step (512 MB write, outside the events)",
                          "parallelism": f"replicas x{ws}", "setup_s": t_setup,
                          "fft_tiles": {k: int(v) for k, v in zip(svh.Handle.FFT_PASSES, tiles)}},
               "fp64": fp64, "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "solve": solve,
               "batch_cfg3": batch, "tucker_sweep": sweep,
               "gpu_launches": launches_per_step * args.steps, "clocks": clocks}
        print(json.dumps(out), flush=True)
    h.close()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_svh(args)


if __name__ == "__main__":
    sys.exit(main())
