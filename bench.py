"""Benchmark of the grid-integration hot path on GB300.

One step = the per-SCF-iteration grid work on one structure: V_mu,nu(R) (gint_vlocal), the
backward pass rho(r) + Pulay force (gint_rho_force) and the FP64 checks Sum rho dV
(gint_charge) and Tr(rho_mu,nu V_mu,nu) (gint_block_dot).  The geometry set-up (block list,
batch lists) is done once per structure and is outside the timed region.  The headline runs the
FP16x3 split; the line also carries every other precision's time and error against the FP64
oracle (on a seeded sample of blocks, grid points and atoms), the multi-structure job and the
CPU oracle on the other configurations.

Default workload: the 512-atom Si precision case (4x4x4 diamond supercell, 6656 orbitals,
grid 192^3 = 7,077,888 points), synthetic seeded inputs.  Metric: grid points per second.

  python bench.py [--steps K] [--warmup W] [--prec tf32x3] [--workload si512]
  python bench.py --impl reference ...    # the FP64 CPU oracle on a bounded sample
Under torchrun (N > 1) every rank runs an independent replica (the path has no data
exchange across structures); value = points of all ranks / max time over ranks.
"""
from __future__ import annotations

import argparse
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

METRIC = "gint V_mu_nu + rho(r) grid points/s (split-precision vs FP64, at stated error)"
L2_FLUSH_BYTES = 512 << 20


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return m, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# DRAM bytes per launch of the tensor-core kernels (dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture), keyed by the SHA-256 prefix of the kernel sources
# the counters were taken on: once a kernel source changes, the bench reports traffic = null.
NCU_TRAFFIC = {
    # profiles/dram_k_vlocal_tc_k_rho_tc_si64_fp16x3.md (Si64 counters x 8)
    "e174c6cfea1317cc": {"si512/fp16x3/rho_force": 183.4e6, "si512/fp16x3/vlocal": 151.1e6},
}
TC_SOURCES = ("gint_tc.cu", "gint_device.cuh", "gint_tcgen05.cuh")


def _source_key():
    import hashlib
    h = hashlib.sha256()
    for name in TC_SOURCES:
        with open(os.path.join(ROOT, "paper_2501_08697_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(kernel, workload, prec):
    return NCU_TRAFFIC.get(_source_key(), {}).get(f"{workload}/{prec}/{kernel}")


def _tensor_peak(prec, peaks, sustained=True):
    """Dense peak (TFLOP/s) for the contraction dtype: measured bf16 x nominal dtype ratio."""
    bf16 = peaks.get("bf16_tflops_sustained" if sustained else "bf16_tflops", 1700.0)
    ratio = {"tf32x3": 1.1 / 2.25, "bf16x3": 1.0, "bf16x6": 1.0, "fp16x3": 1.0, "fp32": 1.1 / 2.25}.get(prec, 1.0)
    return bf16 * ratio


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, world, device=None):
    """Largest value of x over the ranks of the process group (x itself at N = 1): the slowest
    rank's time makes the job's time."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def workload_name(name, st):
    return f"{name}: {st.natoms} atoms, {st.nbasis} orbitals, grid {'x'.join(map(str, st.grid))}"


def build_inputs(name):
    from paper_2501_08697_gb300 import synth as S
    st = S.workload(name)
    V = S.local_potential(st)
    return st, V


# vlocal batch shape per precision: FP16x3's 16-deep MMA steps keep 128-point batches inside the
# 1e-6 accumulation-error budget, the other tensor-core schemes stay at 64 points
VBATCH = {"fp16x3": (4, 4, 8)}
PRECS = ("fp16x3", "tf32x3", "bf16x6", "bf16x3", "fp32")


def vbatch(prec):
    return VBATCH.get(prec, (4, 4, 4))


def oracle_samples(st, Vn, DMn, keys, offs, n_blocks=4096, n_pts=100000, n_atoms=64, seed=2501):
    """FP64 oracle values on a seeded sample of the workload: n_blocks blocks drawn from the whole
    pair list (each summed over its first atom's sphere), n_pts grid points of rho and the force
    on n_atoms atoms (each summed over its own sphere)."""
    from oracle import Oracle
    o = Oracle.from_structure(st)
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(len(keys), min(n_blocks, len(keys)), replace=False))
    idx = np.concatenate([np.arange(offs[b], offs[b + 1]) for b in sel])
    pts = np.sort(rng.choice(st.npts, min(n_pts, st.npts), replace=False))
    atoms = np.sort(rng.choice(st.natoms, min(n_atoms, st.natoms), replace=False))
    t0 = time.perf_counter()
    ref = dict(idx=idx, H=o.vlocal_blocks(Vn, sel), pts=pts, rho=o.rho(DMn, pts), atoms=atoms,
               F=-o.dLdtau_atoms(Vn, DMn, atoms))
    ref["oracle_s"] = time.perf_counter() - t0
    ref["desc"] = (f"{len(sel)} seeded blocks of the pair list, {len(pts)} seeded grid points, "
                   f"force on {len(atoms)} seeded atoms")
    return ref


def run_ours(args, rank, world):
    import torch
    from paper_2501_08697_gb300 import gint as G
    from paper_2501_08697_gb300 import synth as S

    dev = torch.device(f"cuda:{int(os.environ.get('LOCAL_RANK', 0))}")
    torch.cuda.set_device(dev)
    st, Vn = build_inputs(args.workload)
    prec = args.prec
    batch = tuple(args.batch) if args.batch else vbatch(prec)
    t0 = time.time()
    h = G.setup_structure(st, batch=batch, batch_rho=tuple(args.batch_rho))
    setup_s = time.time() - t0
    keys, offs = h.layout()
    DMn = S.density_matrix(keys, st.norb_atom, seed=st.seed)
    info = h.info
    V = torch.from_numpy(Vn.reshape(-1)).to(dev)
    DM = torch.from_numpy(DMn).to(dev)
    H = torch.empty(info["nvalues"], dtype=torch.float64, device=dev)
    rho = torch.empty(info["npts"], dtype=torch.float64, device=dev)
    F = torch.empty(3 * st.natoms, dtype=torch.float64, device=dev)
    chk = torch.zeros(2, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(hh, p, ev=None):
        if ev:
            ev[0].record(stream)
        G.gint_vlocal(hh, V, H, p)
        if ev:
            ev[1].record(stream)
        G.gint_rho_force(hh, V, DM, rho, F, p)
        if ev:
            ev[2].record(stream)
        G.gint_charge(hh, rho, chk[0:1])
        G.gint_block_dot(hh, DM, H, chk[1:2])
        if ev:
            ev[3].record(stream)

    def timed(hh, p, steps, warmup, all_ranks=True):
        for _ in range(warmup):
            step(hh, p)
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
        if all_ranks:
            barrier(world)
        torch.cuda.synchronize()
        for i in range(steps):
            flush.fill_(float(i))                       # evict L2 (512 MiB write) outside the events
            step(hh, p, evs[i])
        torch.cuda.synchronize()
        tot = sum(e[0].elapsed_time(e[3]) for e in evs) / 1e3
        tv = sum(e[0].elapsed_time(e[1]) for e in evs) / steps / 1e3
        tr = sum(e[1].elapsed_time(e[2]) for e in evs) / steps / 1e3
        tc = sum(e[2].elapsed_time(e[3]) for e in evs) / steps / 1e3
        return tot, tv, tr, tc

    with ClockSampler(dev.index) as clk:
        tot, tv, tr, tc = timed(h, prec, args.steps, args.warmup)
    clocks = clk.summary()
    assert G.gint_get_status(h) == 0
    tmax = max_over_ranks(tot, world, dev)
    npts = info["npts"]
    value = world * npts * args.steps / tmax
    ms = tmax / args.steps * 1e3
    extras = rank == 0 and world == 1 and not args.quick

    # errors of each precision against the FP64 oracle (seeded sample) and the FP64 GPU path
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    ref = oracle_samples(st, Vn, DMn, keys, offs) if extras else None

    def errors(p_):
        Hn, rn, Fn = H.cpu().numpy(), rho.cpu().numpy(), F.cpu().numpy().reshape(-1, 3)
        return {"H": rel(Hn[ref["idx"]], ref["H"]), "rho": rel(rn[ref["pts"]], ref["rho"]),
                "F": rel(Fn[ref["atoms"]], ref["F"])}

    err_oracle = None
    if extras:
        step(h, prec)
        torch.cuda.synchronize()
        err_oracle = errors(prec)

    # the FP64 GPU path on the same step, for the split-vs-FP64 comparison
    fp64 = None
    err = None
    if not args.skip_fp64 and rank == 0:
        f_tot, f_tv, f_tr, _ = timed(h, "fp64", 1, 1, all_ranks=False)   # rank 0 alone
        fp64 = {"pts_per_s": npts / f_tot, "ms_per_step": f_tot * 1e3, "vlocal_ms": f_tv * 1e3,
                "rho_force_ms": f_tr * 1e3,
                # algorithmic FP64 FLOP/s of the step's two contractions against the FP64 pipe
                # (2 DFMA per clock per SM sub-partition pair: 2 x 2 x 152 x 2.07 GHz = 1.26 TFLOP/s)
                "alg_tflops": 2 * info["flops_useful"] / f_tot / 1e12}
        fp64["frac_of_fp64_pipe"] = fp64["alg_tflops"] / (2 * 2 * 152 * 2.070e9 / 1e12)
        # the per-batch contractions as executed (nb x nb per point; vlocal forms the upper
        # triangle only), against the same pipe
        fp64["batch_tflops"] = (0.5 * info["flops_dense"] + info["flops_dense_rho"]) / f_tot / 1e12
        fp64["batch_frac_of_fp64_pipe"] = fp64["batch_tflops"] / (2 * 2 * 152 * 2.070e9 / 1e12)
        if extras:
            fp64["err_vs_oracle"] = errors("fp64")
        H64, rho64, F64 = H.clone(), rho.clone(), F.clone()
        step(h, prec)
        torch.cuda.synchronize()
        relt = lambda a, b: float(torch.linalg.norm(a - b) / torch.linalg.norm(b))
        err = {"H": relt(H, H64), "rho": relt(rho, rho64), "F": relt(F, F64)}

    # the other precisions on the same workload (each with its own vlocal batch shape)
    per_prec = {}
    if extras:
        for p_ in PRECS:
            if p_ == prec:
                per_prec[p_] = {"pts_per_s": npts / (tot / args.steps), "vlocal_ms": tv * 1e3, "rho_force_ms": tr * 1e3,
                                "batch_vlocal": list(batch), "err_vs_oracle": err_oracle}
                continue
            h2 = G.setup_structure(st, batch=vbatch(p_), batch_rho=tuple(args.batch_rho))
            n = 3 if p_ != "fp32" else 1
            t2, v2, r2, _ = timed(h2, p_, n, 2 if p_ != "fp32" else 1, all_ranks=False)
            assert G.gint_get_status(h2) == 0
            step(h2, p_)
            torch.cuda.synchronize()
            per_prec[p_] = {"pts_per_s": npts * n / t2, "vlocal_ms": v2 * 1e3, "rho_force_ms": r2 * 1e3,
                            "batch_vlocal": list(vbatch(p_)), "err_vs_oracle": errors(p_)}
            h2.close()

    # position updates (host lists and tables, re-upload of what changed): seeded N(0, 0.05 bohr)
    # moves of every atom, alternating between two moved geometries, on a handle of its own
    upd = None
    if extras:
        h3 = G.setup_structure(st, batch=batch, batch_rho=tuple(args.batch_rho))
        rng = np.random.default_rng(2501)
        taus = [st.tau + rng.normal(0.0, 0.05, st.tau.shape) for _ in range(2)]
        ts, refused = [], 0
        for i in range(8):
            t0 = time.perf_counter()
            try:
                G.gint_update_positions(h3, taus[i % 2])
            except G.GintError:
                refused += 1
                continue
            ts.append(time.perf_counter() - t0)
        h3.close()
        upd = {"sigma_bohr": 0.05, "median_ms": 1e3 * statistics.median(ts) if ts else None,
               "first_ms": 1e3 * ts[0] if ts else None, "updates": len(ts), "refused": refused}

    # end to end through the C ABI with host buffers (copies inside the timed region)
    pin = lambda n: torch.empty(n, dtype=torch.float64).pin_memory()
    Vh, DMh = pin(npts), pin(info["nvalues"])
    Vh.copy_(torch.from_numpy(Vn.reshape(-1)))
    DMh.copy_(torch.from_numpy(DMn))
    Hh, rhoh, Fh = pin(info["nvalues"]), pin(npts), pin(3 * st.natoms)
    G.gint_run_host(h, Vh, DMh, Hh, rhoh, Fh, prec)
    t0 = time.perf_counter()
    n_e2e = max(1, args.steps)
    for _ in range(n_e2e):
        G.gint_run_host(h, Vh, DMh, Hh, rhoh, Fh, prec)
    e2e_s = (time.perf_counter() - t0) / n_e2e
    e2e = {"value": world * npts / e2e_s, "unit": "grid points/s",
           "h2d_bytes_per_step": 8 * (npts + info["nvalues"]),
           "d2h_bytes_per_step": 8 * (info["nvalues"] + npts + 3 * st.natoms)}

    peaks, src = _peaks()
    dominant = ("rho_force", tr) if tr >= tv else ("vlocal", tv)
    alg_flops = info["flops_useful"]                       # 2 n(r)^2 summed over the grid
    exec_flops = {"tf32x3": 3, "bf16x3": 3, "bf16x6": 6, "fp16x3": 3}.get(prec, 1) * (
        info["flops_dense"] if dominant[0] == "vlocal" else info["flops_dense_rho"])
    tp = _tensor_peak(prec, peaks, sustained=True)
    achieved = alg_flops / dominant[1] / 1e12
    roofline = {"bound": "tensor", "kernel": dominant[0], "achieved": achieved, "peak": tp, "unit": "TFLOP/s",
                "frac": achieved / tp, "traffic": _traffic(dominant[0], args.workload, prec),
                "peak_source": f"{src} bf16 sustained x nominal {prec} ratio",
                "executed_tflops": exec_flops / dominant[1] / 1e12,
                "other_kernel": {"kernel": "vlocal" if dominant[0] == "rho_force" else "rho_force",
                                 "achieved": alg_flops / (tv if dominant[0] == "rho_force" else tr) / 1e12}}
    out = {
        "metric": METRIC, "value": value, "unit": "grid points/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": prec, "data": "synthetic (seeded Si diamond 4x4x4, plane-wave V, random DM)",
        "config": {"workload": workload_name(args.workload, st),
                   "prec": prec, "batch_vlocal": list(batch), "batch_rho": list(args.batch_rho),
                   "step": "vlocal + rho_force + charge + trace", "l2": "flushed between steps (512 MiB write)",
                   "parallelism": f"replicas x{world}", "setup_s": round(setup_s, 3),
                   "position_update": upd,
                   "nbatches": info["nbatches"], "nbatches_rho": info["nbatches_rho"]},
        "kernel_ms": {"vlocal": tv * 1e3, "rho_force": tr * 1e3, "checks": tc * 1e3},
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": args.steps * 10,
        "clocks": clocks,
        "fp64_gpu": fp64,
        "err_vs_fp64_gpu": err,
        "err_vs_oracle": err_oracle,
        "oracle_sample": ref["desc"] if ref else None,
        "speedup_vs_fp64_gpu": (value / world / fp64["pts_per_s"]) if fp64 else None,
        "precisions": per_prec or None,
    }
    if extras and not args.skip_batching:
        out["batching"] = run_batching(args, rank, world, quiet=True)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, st, Vn, keys, offs, DMn)
        if extras:
            out["cpu_baseline_configs"] = cpu_baseline_configs(args)
    h.close()
    return out


def _oracle_sample(st, DMn=None):
    """The FP64 CPU oracle of a structure and a function that runs vlocal + rho + dL/dtau on
    the first n grid points (a contiguous slab of i-planes)."""
    from oracle import Oracle
    from paper_2501_08697_gb300 import synth as S
    o = Oracle.from_structure(st)
    k2, o2 = o.pairs()
    if DMn is None:
        DMn = S.density_matrix(k2, st.norb_atom, seed=st.seed)

    def run(Vn, n):
        pts = np.arange(n, dtype=np.int64)
        o.vlocal(Vn, pts)
        o.rho(DMn, pts)
        o.dLdtau(Vn, DMn, pts)

    return run


def cpu_baseline(args, st, Vn, keys=None, offs=None, DMn=None, budget_pts=None):
    """The FP64 CPU oracle (as it stands) on a bounded sample of the same workload:
    vlocal + rho + dL/dtau contributions of a contiguous slab of grid points."""
    from oracle import Oracle
    run = _oracle_sample(st, DMn)
    n = budget_pts or args.cpu_points
    t0 = time.perf_counter()
    run(Vn, n)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "grid points/s", "cores": Oracle.threads(), "kind": "oracle",
            "sample": f"first {n} grid points (a slab of i-planes) of {args.workload}: vlocal + rho + force, "
                      f"{dt:.1f} s"}


def cpu_baseline_configs(args):
    """The FP64 CPU oracle (as it stands) on the other configurations: the forward pass (vlocal +
    rho) of the 8-atom Si cell (48^3) in full, and of the 64-atom Si cell (96^3) and the 64-water
    box (128^3) on their first 1e5 grid points (a slab of i-planes; whole-grid time = slab time
    x points / 1e5, as the cost per point is uniform to first order)."""
    from oracle import Oracle
    from paper_2501_08697_gb300 import synth as S
    out = {}
    for name, n in (("si8", None), ("si64", 100000), ("water64", 100000)):
        st = S.workload(name)
        Vn = S.local_potential(st)
        o = Oracle.from_structure(st)
        k2, _ = o.pairs()
        DMn = S.density_matrix(k2, st.norb_atom, seed=st.seed)
        pts = None if n is None else np.arange(n, dtype=np.int64)
        t0 = time.perf_counter()
        o.vlocal(Vn, pts)
        o.rho(DMn, pts)
        dt = time.perf_counter() - t0
        np_ = st.npts if n is None else n
        out[name] = {"value": np_ / dt, "unit": "grid points/s", "cores": Oracle.threads(),
                     "sample": "whole grid" if n is None else f"first {n} of {st.npts} grid points",
                     "forward_s": dt if n is None else dt * st.npts / n,
                     "forward_s_kind": "measured" if n is None else "extrapolated from the slab"}
    return out


def run_batching(args, rank, world, quiet=False):
    """The multi-structure case: 32 structures of uneven size (Si 8/16/64/216 atoms x 4 strains,
    water boxes of 8..32 molecules), forward (vlocal) + adjoint (rho) in one graph-replayed job
    with autotuned batch shapes, against sequential per-structure launches."""
    import torch
    from paper_2501_08697_gb300 import gint as G
    from paper_2501_08697_gb300 import synth as S
    dev = torch.device(f"cuda:{int(os.environ.get('LOCAL_RANK', 0))}")
    torch.cuda.set_device(dev)
    sts = S.batching_set()
    prec = args.prec
    # autotune once per structure class (largest member) and reuse the shapes
    shapes = {}
    for cls in ("si", "water"):
        rep = max((st for st in sts if st.name.startswith(cls)), key=lambda st: st.npts)
        bv, br, tv, tr = G.gint_autotune(rep, prec)
        shapes[cls] = (bv, br, tv, tr)
    hs, V, DM, H, rho = [], [], [], [], []
    for st in sts:
        bv, br = shapes["si" if st.name.startswith("si") else "water"][:2]
        h = G.setup_structure(st, batch=bv, batch_rho=br)
        keys, offs = h.layout()
        hs.append(h)
        V.append(torch.from_numpy(S.local_potential(st).reshape(-1)).to(dev))
        DM.append(torch.from_numpy(S.density_matrix(keys, st.norb_atom, seed=st.seed)).to(dev))
        H.append(torch.empty(h.info["nvalues"], dtype=torch.float64, device=dev))
        rho.append(torch.empty(h.info["npts"], dtype=torch.float64, device=dev))
    npts = sum(h.info["npts"] for h in hs)
    job = G.Batch(hs, V, H, DM, rho, prec)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def seq():
        for h, v, d, hh, r in zip(hs, V, DM, H, rho):
            G.gint_vlocal(h, v, hh, prec)
            G.gint_rho(h, d, r, prec)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        barrier(world)
        tot = 0.0
        for i in range(args.steps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b) / 1e3
        return tot

    with ClockSampler(dev.index) as clk:
        t_job = max_over_ranks(timed(job.launch), world, dev)
    t_seq = max_over_ranks(timed(seq), world, dev)
    value = world * npts * args.steps / t_job
    if quiet:
        return {"workload": f"batching: {len(sts)} structures, {npts} grid points", "prec": prec,
                "pts_per_s": value, "ms_per_job": t_job / args.steps * 1e3,
                "sequential_pts_per_s": npts * args.steps / t_seq, "speedup_vs_sequential": t_seq / t_job,
                "autotuned": {k: {"batch": v[0], "batch_rho": v[1], "vlocal_ms": v[2], "rho_ms": v[3]}
                              for k, v in shapes.items()}}
    return {"metric": METRIC + " [batched]", "value": value, "unit": "grid points/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_job / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": prec,
            "data": "synthetic (32 seeded structures)",
            "config": {"workload": f"batching: {len(sts)} structures, {npts} grid points", "prec": prec,
                       "step": "vlocal + rho of every structure", "l2": "flushed between steps (512 MiB write)",
                       "autotuned": {k: {"batch": v[0], "batch_rho": v[1], "vlocal_ms": v[2], "rho_ms": v[3]}
                                     for k, v in shapes.items()}},
            "sequential_pts_per_s": npts * args.steps / t_seq, "speedup_vs_sequential": t_seq / t_job,
            "clocks": clk.summary(), "gpu_launches": args.steps * (2 * len(sts) + 1 + len(sts) + 1)}


def run_kspace(args, rank, world):
    """The k-space transforms on the Si512 block store: gint_fold of H(R) to 4 dense k-point
    matrices (6656^2 complex each) and gint_unfold back; memory-bound, reported in GB/s of
    algorithmic traffic (block store read or written once, dense entries written or read once)."""
    import numpy as np
    import torch
    from paper_2501_08697_gb300 import gint as G
    from paper_2501_08697_gb300 import synth as S
    dev = torch.device(f"cuda:{int(os.environ.get('LOCAL_RANK', 0))}")
    torch.cuda.set_device(dev)
    st, Vn = build_inputs("si512")
    h = G.setup_structure(st)
    keys, offs = h.layout()
    info = h.info
    N, nv = info["nbasis"], info["nvalues"]
    X = torch.from_numpy(S.density_matrix(keys, st.norb_atom, seed=st.seed)).to(dev)
    rng = np.random.default_rng(S.BASE_SEED + 7)
    kap = np.vstack([[0.0, 0.0, 0.0], rng.uniform(-0.5, 0.5, (3, 3))])
    w = np.full(len(kap), 1.0 / len(kap))
    nk = len(kap)
    Xk = torch.empty((nk, N, N), dtype=torch.complex128, device=dev)
    Xb = torch.empty_like(X)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    # unique dense entries the unfold reads: the sub-blocks of atom pairs that have blocks
    pairs = {(int(k[0]), int(k[1])) for k in keys}
    nint = sum(int(st.norb_atom[i]) * int(st.norb_atom[j]) for i, j in pairs)
    bytes_fold = 8 * nv + 16 * N * N * nk
    bytes_unfold = 16 * nint * nk + 8 * nv

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        barrier(world)
        tot = 0.0
        for i in range(args.steps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b) / 1e3
        return tot / args.steps

    with ClockSampler(dev.index) as clk:
        tf = max_over_ranks(timed(lambda: G.gint_fold(h, X, kap, Xk)), world, dev)
        tu = max_over_ranks(timed(lambda: G.gint_unfold(h, Xk, kap, w, Xb)), world, dev)
    peaks, src = _peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    gf, gu = bytes_fold / tf / 1e9, bytes_unfold / tu / 1e9
    return {"metric": "k-space fold of the block store, GB/s of algorithmic traffic", "value": world * gf,
            "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tf * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (Si512 block-symmetric random store)",
            "config": {"workload": f"kspace: si512 store ({nv} values), {nk} k points, nbasis {N}",
                       "l2": "flushed between steps (512 MiB write)"},
            "roofline": {"bound": "hbm", "kernel": "k_fold", "achieved": gf, "peak": hbm, "unit": "GB/s",
                         "frac": gf / hbm, "traffic": None, "peak_source": src,
                         "bytes_per_launch": bytes_fold},
            "unfold": {"ms": tu * 1e3, "GB/s": gu, "frac": gu / hbm, "bytes_per_launch": bytes_unfold},
            "clocks": clk.summary(), "gpu_launches": args.steps * 4}


def run_dm(args, rank, world):
    """Density matrix from eigenvectors (Eq. density_matrix) for the Si512 Gamma-point supercell:
    C is nbasis x nbands (6656 x 1024, complex storage), rho(Gamma) = C diag(f) C^H, then added
    into the block store.  Both paths are timed: TF32x3 on the tensor cores (K = 2048 real terms in
    64-term TMEM segments) and FP64 on the CUDA cores; value = algorithmic FLOP/s of the complex
    product (8 per complex multiply-add; at Gamma only Re rho is formed, 4 per term) of the
    tensor-core path."""
    import numpy as np
    import torch
    from paper_2501_08697_gb300 import gint as G
    dev = torch.device(f"cuda:{int(os.environ.get('LOCAL_RANK', 0))}")
    torch.cuda.set_device(dev)
    st, Vn = build_inputs(args.dm_structure)
    h = G.setup_structure(st)
    N = h.info["nbasis"]
    nb = 4 * st.natoms // 2                       # Si: 4 valence electrons per atom, 2 per band
    gen = torch.Generator(device=dev).manual_seed(2501)
    C = torch.randn((1, N, nb), dtype=torch.complex128, device=dev, generator=gen) / N ** 0.5
    f = torch.full((1, nb), 2.0, dtype=torch.float64, device=dev)
    DM = torch.empty(h.info["nvalues"], dtype=torch.float64, device=dev)
    DM64 = torch.empty_like(DM)
    kap, w = np.zeros((1, 3)), [1.0]
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(prec, out, steps):
        for _ in range(args.warmup):
            G.gint_density_matrix(h, kap, w, C, f, out, prec)
        torch.cuda.synchronize()
        barrier(world)
        tot = 0.0
        for i in range(steps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            G.gint_density_matrix(h, kap, w, C, f, out, prec)
            b.record(stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b) / 1e3
        return tot / steps

    with ClockSampler(dev.index) as clk:
        t_tc = max_over_ranks(timed("tf32x3", DM, args.steps), world, dev)
    t_64 = timed("fp64", DM64, max(1, min(args.steps, 2)))
    err = float(torch.linalg.norm(DM - DM64) / torch.linalg.norm(DM64))
    alg = 4.0 * N * N * nb                       # Re part of the complex product at Gamma
    exe = 2.0 * N * N * (2 * nb) * 3             # one real GEMM, K = 2 nb, 3 TF32 products
    peaks, src = _peaks()
    tp = _tensor_peak("tf32x3", peaks, sustained=False)
    return {"metric": f"density matrix from eigenvectors ({args.dm_structure} Gamma), algorithmic TFLOP/s", "value": world * alg / t_tc / 1e12,
            "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_tc * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "tf32x3",
            "data": "synthetic (random complex C / sqrt(nbasis), f = 2)",
            "config": {"workload": f"dm: {args.dm_structure} Gamma, nbasis {N}, {nb} bands", "l2": "flushed between steps"},
            "roofline": {"bound": "tensor", "kernel": "k_rhok_tc", "achieved": exe / t_tc / 1e12, "peak": tp,
                         "unit": "TFLOP/s", "frac": exe / t_tc / 1e12 / tp, "traffic": None,
                         "peak_source": f"{src} bf16 burst x nominal tf32 ratio (executed tf32 flops)"},
            "fp64": {"ms": t_64 * 1e3, "executed_TFLOP/s": 8.0 * N * N * nb / t_64 / 1e12,
                     "frac_of_fp64_pipe": 8.0 * N * N * nb / t_64 / 1e12 / (2 * 2 * 152 * 2.070e9 / 1e12),
                     "note": "the FP64 kernel forms Re and Im of the complex product"},
            "err_vs_fp64": err, "speedup_vs_fp64": t_64 / t_tc,
            "clocks": clk.summary(), "gpu_launches": args.steps * 2}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    from oracle import Oracle
    st, Vn = build_inputs(args.workload)
    run = _oracle_sample(st)                    # oracle set-up (pair list, DM) outside the timing
    n = args.cpu_points
    for _ in range(args.warmup):
        run(Vn, n)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run(Vn, n)
    tot = time.perf_counter() - t0
    value = n * args.steps / tot
    res = {"cores": Oracle.threads(),
           "sample": f"first {n} grid points (a slab of i-planes) of {args.workload} per step: vlocal + rho + "
                     f"force, {tot / max(1, args.steps):.1f} s per step"}
    return {"metric": METRIC, "value": value, "unit": "grid points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": workload_name(args.workload, st), "prec": "fp64 (CPU oracle)",
                       "sample_points_per_step": args.cpu_points},
            "cpu_baseline": {"value": value, "unit": "grid points/s", "cores": res["cores"], "kind": "oracle",
                             "sample": res["sample"]},
            "e2e": {"value": value, "unit": "grid points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="si512")
    ap.add_argument("--prec", default="fp16x3")
    ap.add_argument("--batch", type=int, nargs=3, default=None, help="vlocal batch (default: per precision)")
    ap.add_argument("--batch-rho", type=int, nargs=3, default=[4, 4, 8])
    ap.add_argument("--cpu-points", type=int, default=100000)
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--skip-batching", action="store_true")
    ap.add_argument("--quick", action="store_true", help="headline line only (no per-precision, oracle or batching extras)")
    ap.add_argument("--dm-structure", default="si512", help="structure of --workload dm (si8, si64, si512)")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "ours":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        # the reference arm is the CPU oracle: its ranks meet over gloo
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.workload == "batching":
        out = run_batching(args, rank, world)
    elif args.workload == "kspace":
        out = run_kspace(args, rank, world)
    elif args.workload == "dm":
        out = run_dm(args, rank, world)
    else:
        out = run_ours(args, rank, world)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
