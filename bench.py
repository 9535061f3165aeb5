"""Benchmark: finite-element integration throughput on GB300.

A step is one pass of the whole hot path over one batch: the FP64 integration of
6,000,000 generic convection-diffusion-reaction tetrahedra (100^3 cubes x 6,
nodes jittered by +-0.2 h, 4-point rule, 20 coefficients per element, element-
contiguous order): edge vectors, Jacobian terms, global derivatives, coefficient
products, accumulation and stores, in double arithmetic (one kernel; the FP64
form flags elements but needs no fix-up pass). The paper's arithmetic is double
precision throughout (Sec. 5), so this is the line's value.

The same mesh is also timed in the mixed form (float bulk, double Jacobian for
poorly shaped elements: main kernel plus fix-up) and in the double-word form
(double accuracy from float pairs), each under a key of its own with its own
roofline; and the other workloads (the 48,000-element Poisson set as stated,
prisms, node tables, batches, serving) under further keys.

Prints one JSON line (rank 0). Under torchrun every rank integrates its own
seeded mesh of that size on its own GPU (weak scaling, no data-path
collective; the barrier and the max over ranks are timing only).

--impl reference times the FP64 CPU oracle (Algorithm 1 as written) on the host
cores instead, on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Melements/s & % of HBM roofline, FP32 vs FP64 form; served p50/p99 latency"
MESH = ("generic conv-diff-reaction tetrahedra: unit cube 100^3 x 6 Kuhn = 6,000,000 elements, "
        "jitter +-0.2h, TET4 rule, per-element coefficients (c^{ij} SPD eig U[0.1,10], c^{i0},c^{0i} "
        "U[-1,1]^3, c^{00} U[0,1], d U[-1,1]), element-contiguous (natural) input and output order")
WORKLOAD = MESH + ", FP64 arithmetic (results within 1e-12 of the FP64 oracle)"
MIXED_WORKLOAD = MESH + ", mixed FP32 with FP64 Jacobian for mean ratio < 0.1"
N_ELEM = 6_000_000
SEED = 1504010230 + 2
PRISM_WORKLOAD = ("generic conv-diff-reaction prisms: [0,1]^2 in 1000 x 1000 squares x 2 triangles, one layer "
                  "h = 1e-3 with z-jitter +-0.1h = 2,000,000 elements, PRISM6 rule (3 triangle x 2 line), 20 "
                  "coefficients per integration point, mixed FP32 with FP64 Jacobian for mean ratio < 0.1, "
                  "element-contiguous order")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--n-cubes", type=int, default=100,
                    help="cubes per axis of the tetrahedral mesh (6 n^3 elements); smaller only for profiling")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    ap.add_argument("--no-indexed", action="store_true")
    ap.add_argument("--no-prism", action="store_true")
    ap.add_argument("--workload", default="tet", choices=["tet", "prism"],
                    help="tet: the 6M generic tetrahedra (default); prism: the 2M generic prisms (profiling)")
    ap.add_argument("--form", default="fp64", choices=["fp64", "mixed", "dw"],
                    help="precision form of the timed step: fp64 (default, the line's value), mixed or dw "
                         "(double-word); other forms only for profiling")
    ap.add_argument("--only", action="store_true", help="time the step only (no other keys; profiling)")
    ap.add_argument("--kind", default="generic", choices=["generic", "poisson"],
                    help="generic (default) or the Laplace kind (tetrahedra: TET1, d^0 = 1; prisms: d^0 per "
                         "point); other kinds only for profiling")
    ap.add_argument("--shape", default=None, help="BLOCK,PERSISTENT[,THREADS_PER_ELEMENT]: pin the main kernel's "
                                                  "launch shape instead of autotuning it (profiling)")
    ap.add_argument("--n-slab", type=int, default=1000,
                    help="squares per axis of the prism slab (2 n^2 elements); smaller only for profiling")
    return ap.parse_args()


# ---------------------------------------------------------------------------
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(rank: int, n_cubes: int = 100):
    from paper_1504_01023_gb300 import meshgen
    mesh = meshgen.tet_cube_mesh(n_cubes, jitter=0.2, seed=SEED + 1000 * rank)
    coefs = meshgen.generic_coefs(len(mesh), 1, seed=SEED + 1000 * rank)
    return mesh, coefs


class ClockSampler:
    """nvidia-smi samples (200 ms) of the GPU's clocks and throttle reasons."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, which):
        if which == 0:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for t, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            rows.append((t, parts))
        inside = [r for r in rows if self.t0 is not None and self.t0 - 0.2 <= r[0] <= (self.t1 or 1e30) + 0.2]
        use = inside or rows[-3:]
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(p[1]) for _, p in use if p[1].replace(".", "").isdigit()]
        smax = [float(p[2]) for _, p in use if p[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, p in use for i in range(4) if p[5 + i].lower() == "active"})
        pw = [float(p[3]) for _, p in use if re.match(r"^[0-9.]+$", p[3])]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(use), "samples_in_region": len(inside),
                "power_w_max": max(pw) if pw else None}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def same_run_copy_gbs(dev, nbytes=2 << 30, reps=10):
    """A STREAM-style copy in this run (the paper reports STREAM beside its kernels,
    Sec. 4.5): device-to-device copy of a 2 GiB buffer, bytes read + written per
    second, CUDA events. Context for the roofline, whose denominator stays the
    measured peak; None if it cannot run."""
    import torch
    try:
        a = torch.empty(nbytes // 4, dtype=torch.float32, device=dev)
        b = torch.empty_like(a)
        a.fill_(1.0)
        for _ in range(3):
            b.copy_(a)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record()
        for _ in range(reps):
            b.copy_(a)
        e1.record()
        torch.cuda.synchronize(dev)
        gbs = 2.0 * nbytes * reps / (e0.elapsed_time(e1) * 1e-3) / 1e9
        del a, b
        torch.cuda.empty_cache()
        return gbs
    except Exception:
        return None


# The sources that determine the element kernels' code: every header, and the
# translation units that instantiate the single-set kernels (host runtime, batch,
# serving, study and self-test units are left out).
KERNEL_UNITS = ("fe_tet_", "fe_prism_", "fe_idx_", "fe_group_", "fe_entry_")


def code_only(text: str) -> str:
    """C++ source without its comments and blank lines (the sources carry no
    comment markers inside string literals), so that editing a comment keeps the
    hash of the code."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.rstrip() for line in text.splitlines() if line.strip())


def kernel_source_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1504_01023_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cuh", ".h")) or (name.endswith(".cu") and name.startswith(KERNEL_UNITS)):
            with open(os.path.join(csrc, name), encoding="utf-8") as f:
                h.update((name + code_only(f.read())).encode())
    return h.hexdigest()[:16]


# The paper's own measurements (Table 7, Sec. 5): best loop ordering, ns per
# element, double precision, OpenCL, on other hardware. Context only: its workloads
# are per-point d^0 (Laplace) and per-element coefficients (convection-diffusion),
# 4-point tetrahedra and 6-point prisms; mesh sizes are not given.
PAPER_TABLE7_NS = {
    "Tesla K20m": {"laplace_tet": 2.02, "cd_tet": 4.46, "laplace_prism": 12.80, "cd_prism": 15.58},
    "Xeon Phi 5110P": {"laplace_tet": 8.77, "cd_tet": 15.97, "laplace_prism": 25.09, "cd_prism": 33.29},
    "2x Xeon E5-2620": {"laplace_tet": 17.76, "cd_tet": 24.86, "laplace_prism": 49.74, "cd_prism": 64.27},
}


def paper_context():
    return {"source": "the paper's Table 7: best of its three loop orderings, ns per element, FP64 OpenCL, "
                      "on the hardware named; other machines, context only (not a target)",
            "melem_s": {hw: {case: round(1000.0 / ns, 1) for case, ns in cases.items()}
                        for hw, cases in PAPER_TABLE7_NS.items()}}


# GB300 HBM3e nominal bandwidth (GB/s), reported beside the measured copy ceiling
NOMINAL_HBM_GBS = 7900.0
# FP64 pipe: 2 instructions per clock per SM (the nominal 1.25 TFLOP/s of FMAs);
# instruction issue: one warp instruction per clock per SM sub-partition (4 per SM)
FP64_PIPE_PER_CLK_SM = 2
ISSUE_PER_CLK_SM = 4 * 32
NCU_RECORDS = os.path.join(ROOT, "profiles", "ncu_records.json")


def ncu_record(tag: str, field: str):
    """One figure of an ncu capture (DRAM bytes per launch, instructions per
    element), from the machine-readable record under profiles/, if that record was
    taken on the current kernel sources; otherwise None."""
    try:
        with open(NCU_RECORDS) as f:
            rec = json.load(f)["records"].get(tag)
    except (OSError, ValueError, KeyError):
        return None
    if not rec or rec.get("source_hash") != kernel_source_hash():
        return None
    v = rec.get(field)
    return float(v) if v is not None else None


def device_sms(dev) -> int:
    import torch
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def hbm_roofline(n, bpe, k_ms, peak, peak_kind, traffic=None):
    achieved = n * bpe / (k_ms * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_kind": peak_kind, "algorithmic_bytes_per_launch": n * bpe, "kernel_ms": k_ms,
            "frac_of_nominal": achieved / NOMINAL_HBM_GBS, "nominal_peak": NOMINAL_HBM_GBS}


def pipe_roofline(melem_s, inst_per_elem, sms, sm_mhz, per_clk_sm, what, tag):
    """Instruction-rate roofline: instructions per element from the ncu record of
    `tag` (null when the kernel changed since), peak = per_clk_sm x SMs x the median
    SM clock measured in this run."""
    peak = per_clk_sm * sms * sm_mhz * 1e6 / 1e12
    res = {"bound": "alu", "unit": f"T {what} instructions/s", "peak": peak,
           "peak_kind": f"{per_clk_sm} per clock per SM x {sms} SMs x {sm_mhz:.0f} MHz (median SM clock, this run)",
           "instructions_per_element": inst_per_elem, "ncu_record": tag}
    if inst_per_elem is None:
        res.update(achieved=None, frac=None, note="no ncu record on the current kernel sources")
    else:
        achieved = melem_s * 1e6 * inst_per_elem / 1e12
        res.update(achieved=achieved, frac=achieved / peak)
    return res


def shape_dict(shape):
    """A launch shape (elements per block, persistent[, threads per element]) as JSON."""
    return {"elements_per_block": shape[0], "persistent": shape[1],
            "threads_per_element": shape[2] if len(shape) > 2 else 1}


def kernel_ms(ctx, call, reps):
    """Average main-kernel time (ms) of `reps` calls, from the library's profiling
    events on the launching stream."""
    ctx.set_profiling(True)
    ctx.kernel_time(reset=True)
    for _ in range(reps):
        call()
    kms, kn = ctx.kernel_time(reset=True)
    ctx.set_profiling(False)
    return kms / max(kn, 1)


# ---------------------------------------------------------------------------
def cpu_baseline(mesh, coefs, target_s=10.0, gpu_out=None, tol=1e-12):
    """The FP64 oracle as it stands, on all host cores, over repeated passes of the
    workload's elements (a bounded sample of about target_s seconds of CPU work:
    whole passes while they fit, then a leading part of one more). With the GPU's
    results of the timed steps, the oracle's results of its first sample (the
    leading 50,000 elements) also give the error statistics of those elements.
    `coefs` are the values the GPU read (double for the FP64 form)."""
    import oracle
    cores = os.cpu_count() or 1
    c = np.asarray(coefs, dtype=np.float64)
    n = len(mesh)
    probe = min(n, 50_000)
    t = time.perf_counter()
    Ao, bo, _ = oracle.integrate(oracle.TET, oracle.GENERIC, oracle.Q_TET4, mesh[:probe], c[:probe], n_threads=cores)
    rate = probe / max(time.perf_counter() - t, 1e-6)
    errors = None
    if gpu_out is not None:
        A, b, f = gpu_out
        An = A[:probe].double().cpu().numpy().reshape(probe, 4, 4)
        bn = b[:probe].double().cpu().numpy().reshape(probe, 4)
        flagged = (f[:probe].cpu().numpy() & 1) != 0
        errors = {"elements": f"the leading {probe:,} elements of the timed steps' results",
                  "metric": f"relative Frobenius error per element against the FP64 oracle (tolerance {tol:g})",
                  "flagged": int(flagged.sum())}
        for name, e in (("A", oracle.rel_frobenius(An, Ao)), ("b", oracle.rel_frobenius(bn, bo))):
            for grp, sel in (("unflagged", ~flagged), ("flagged", flagged)):
                v = e[sel]
                errors[f"{name}_{grp}"] = ({"max": float(v.max()), "p99.9": float(np.quantile(v, 0.999))}
                                           if len(v) else None)
    total = int(min(max(probe, rate * target_s), 50 * n))
    done = 0
    t = time.perf_counter()
    while done < total:
        m = min(n, total - done)
        oracle.integrate(oracle.TET, oracle.GENERIC, oracle.Q_TET4, mesh[:m], c[:m], n_threads=cores)
        done += m
    dt = time.perf_counter() - t
    # one thread, on a sample of about a second
    m1 = int(min(n, max(1000, rate / cores * 1.0)))
    t1 = time.perf_counter()
    oracle.integrate(oracle.TET, oracle.GENERIC, oracle.Q_TET4, mesh[:m1], c[:m1], n_threads=1)
    one = m1 / (time.perf_counter() - t1) / 1e6
    res = {"value": done / dt / 1e6, "unit": "Melem/s", "cores": cores, "kind": "oracle",
           "sample": f"{done:,} element integrations ({done / n:.2f} passes over the {n:,}-element workload), FP64, "
                     f"OpenMP over elements", "seconds": dt,
           "single_thread": {"value": one, "unit": "Melem/s", "sample": f"first {m1:,} elements, one thread"},
           "cpu": cpu_model()}
    if errors is not None:
        res["gpu_error_vs_oracle"] = errors
    res["other_workloads"] = oracle_other_workloads(cores)
    return res


def oracle_other_workloads(cores):
    """The oracle on the other single-set workloads, all host cores and one core:
    the 48,000 Poisson tetrahedra as stated (TET1, d^0 = 1, FP64), and a 200,000-
    element subsample of the 2M generic prisms (PRISM6, 20 coefficients per point)."""
    import oracle
    from paper_1504_01023_gb300 import meshgen
    out = {}
    tm = meshgen.tet_cube_mesh(20, jitter=0.2, seed=meshgen.SEED_BASE + 1)
    pm = meshgen.prism_slab_mesh(1000, None, 0.1, seed=meshgen.SEED_BASE + 3, n_elem=200_000)
    pc = meshgen.generic_coefs(len(pm), 6, seed=meshgen.SEED_BASE + 3)
    cases = {"poisson_tet1_48k": (oracle.TET, oracle.POISSON, oracle.Q_TET1, tm, np.ones(len(tm)), False),
             "generic_prism_per_point_200k": (oracle.PRISM, oracle.GENERIC, oracle.Q_PRISM6, pm, pc, True)}
    for name, (et, kind, rule, m, c, cpq) in cases.items():
        rec = {"elements": len(m), "unit": "Melem/s"}
        for label, nt in (("all_cores", cores), ("one_core", 1)):
            t = time.perf_counter()
            oracle.integrate(et, kind, rule, m, c, coef_per_q=cpq, n_threads=nt)
            rec[label] = len(m) / (time.perf_counter() - t) / 1e6
        out[name] = rec
    return out


def cpu_model():
    """CPU name from /proc/cpuinfo ("model name" on x86; Arm cores give an
    implementer/part pair, named here for the parts of current servers)."""
    arm = {"0xd4f": "Arm Neoverse V2", "0xd40": "Arm Neoverse V1", "0xd0c": "Arm Neoverse N1",
           "0xd49": "Arm Neoverse N2", "0xd8e": "Arm Neoverse N3"}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":", 1)[0].strip().lower()
                if key == "model name":
                    return line.split(":", 1)[1].strip()
                if key == "cpu part":
                    part = line.split(":", 1)[1].strip()
                    return arm.get(part, "Arm part " + part)
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args):
    rank, world, _ = dist_env()
    if world > 1 and rank != 0:
        return
    import oracle
    mesh, coefs = workload(0)
    cores = os.cpu_count() or 1
    c = np.asarray(coefs, dtype=np.float64)
    # size each step for ~1.5 s, so that warmup + steps stay within a few minutes
    per_step = min(1.5, 150.0 / max(args.steps + args.warmup, 1))
    probe = 20_000
    t = time.perf_counter()
    oracle.integrate(oracle.TET, oracle.GENERIC, oracle.Q_TET4, mesh[:probe], c[:probe], n_threads=cores)
    rate = probe / max(time.perf_counter() - t, 1e-6)
    s = int(min(len(mesh), max(1000, rate * per_step)))
    rng = np.random.default_rng(7)
    for _ in range(args.warmup):
        o = int(rng.integers(0, len(mesh) - s + 1))
        oracle.integrate(oracle.TET, oracle.GENERIC, oracle.Q_TET4, mesh[o:o + s], c[o:o + s], n_threads=cores)
    t = time.perf_counter()
    for _ in range(args.steps):
        o = int(rng.integers(0, len(mesh) - s + 1))
        oracle.integrate(oracle.TET, oracle.GENERIC, oracle.Q_TET4, mesh[o:o + s], c[o:o + s], n_threads=cores)
    dt = time.perf_counter() - t
    value = s * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Melem/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_elem": N_ELEM, "step": f"{s:,} elements of the workload"},
            "cpu_baseline": {"value": value, "unit": "Melem/s", "cores": cores, "kind": "oracle",
                             "sample": f"{s:,}-element contiguous slices of the {N_ELEM:,}-element workload per step"},
            "e2e": {"value": value, "unit": "Melem/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def aggregate(ms_total, n_per_rank, steps, world, dist=None, device=None):
    """Max of the timed region over ranks (each rank did n_per_rank elements per
    step); returns (ms per step, whole-job Melem/s)."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([ms_total], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = float(t.item())
        dist.barrier()
    ms_step = ms_total / steps
    return ms_step, world * n_per_rank / (ms_step * 1e-3) / 1e6


# ---------------------------------------------------------------------------
FORMS = {"fp64": ("FP64", "f64"), "mixed": ("FP32_MIXED", "f32"), "dw": ("FP64_DW", "f32 double-word")}
PREC_TAG = {"fp64": "FP64", "mixed": "MIXED", "dw": "DWORD"}


def run_native(args):
    import torch
    import torch.distributed as dist
    from paper_1504_01023_gb300 import api

    rank, world, local = dist_env()
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    ctx = api.Context(dev.index)
    prec = getattr(api, FORMS[args.form][0])
    cdt = np.float32 if prec == api.FP32_MIXED else np.float64
    lap = args.kind == "poisson"
    if args.workload == "tet":
        et, mesh, coefs = api.TET, *workload(rank, args.n_cubes)
        if lap:
            coefs = np.ones((len(mesh), 1))
        kw = dict(kind=api.POISSON if lap else api.GENERIC, quad=api.QUAD_TET1 if lap else api.QUAD_TET4,
                  coef_mode=api.PER_ELEMENT, prec=prec, layout=api.AOS, out_layout=api.AOS)
        wl_name = {"fp64": WORKLOAD, "mixed": MIXED_WORKLOAD}.get(args.form, MESH + ", double-word form")
        if lap:
            wl_name = MESH.split(", TET4")[0] + ", Laplace operator, TET1, d^0 = 1, " + args.form + " form"
        kname = {"fp64": "elem_kernel_f64t", "dw": "elem_kernel_dwt"}.get(args.form, "elem_kernel")
        kernel_name = (f"{kname}<TET,{'POISSON' if lap else 'GENERIC'},{PREC_TAG[args.form]},"
                       f"{'TET1' if lap else 'TET4'},per-element,AOS,AOS>")
        tag = f"tet_{'poisson_tet1' if lap else 'generic'}_{args.form}_aos"
    else:
        et, mesh, coefs = api.PRISM, *prism_workload(rank, args.n_slab)
        if lap:
            from paper_1504_01023_gb300 import meshgen
            coefs = meshgen.poisson_coefs(len(mesh), 6, None, seed=meshgen.SEED_BASE + 3)
        kw = dict(kind=api.POISSON if lap else api.GENERIC, quad=api.QUAD_PRISM6, coef_mode=api.PER_QPOINT,
                  prec=prec, layout=api.AOS, out_layout=api.AOS)
        wl_name = PRISM_WORKLOAD
        kernel_name = f"elem_kernel<PRISM,{'POISSON' if lap else 'GENERIC'},{PREC_TAG[args.form]},PRISM6,per-point,AOS,AOS>"
        tag = f"prism_{'poisson' if lap else 'generic'}_{args.form}_aos"
    n = len(mesh)
    X = torch.from_numpy(np.ascontiguousarray(mesh)).to(dev)                       # [E,NS,3] f64
    C = torch.from_numpy(np.ascontiguousarray(coefs.reshape(n, -1).astype(cdt))).to(dev)
    out = api.alloc_out(et, n, prec, api.AOS, dev, with_flags=True)
    stream = torch.cuda.current_stream(dev)
    if args.shape:
        vals = [int(v) for v in args.shape.split(",")]
        blk, pers, tpe = vals[0], vals[1], vals[2] if len(vals) > 2 else 1
        ctx.set_shape(blk, pers, et, X, C, out=out, tpe=tpe, **kw)
        shape = (blk, pers, tpe)
    else:
        shape = ctx.tune(et, X, C, out=out, **kw)                                  # autotuner (untimed)
    step = lambda: ctx.integrate(et, X, C, out=out, **kw)
    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)
    bpe = api.bytes_per_element(et, kw["kind"], kw["quad"], kw["coef_mode"], prec)

    clocks = ClockSampler(dev.index)
    clocks.start()
    time.sleep(0.5)
    ctx.set_profiling(True)
    ctx.kernel_time(reset=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    l0 = api.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.mark(0)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks.mark(1)
    launches = api.launch_count() - l0
    ms_total = e0.elapsed_time(e1)
    kms, kn = ctx.kernel_time(reset=True)
    ctx.set_profiling(False)
    clocks.stop()
    ms_step, value = aggregate(ms_total, n, args.steps, world, dist if world > 1 else None, dev)
    k_ms = kms / max(kn, 1)
    peak, peak_kind = measured_peaks()
    clk = clocks.summary()
    sm_mhz = clk.get("sm_mhz") or 2070.0
    sms = device_sms(dev)
    hbm = hbm_roofline(n, bpe, k_ms, peak, f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                       ncu_record(tag, "dram_bytes"))
    hbm.update(kernel=kernel_name, same_run_copy_gbs=same_run_copy_gbs(dev) if rank == 0 else None)
    melem_k = n / k_ms / 1e3
    if args.form == "mixed":
        roofline = hbm
    else:
        # the double-precision forms are bound by an instruction rate, not by HBM:
        # the FP64 pipe (plain FP64) or instruction issue (double-word); the HBM
        # figures stay beside it
        pipe = (FP64_PIPE_PER_CLK_SM, "FP64-pipe", "fp64_pipe_inst_per_elem") if args.form == "fp64" else \
            (ISSUE_PER_CLK_SM, "thread", "inst_per_elem")
        roofline = pipe_roofline(melem_k, ncu_record(tag, pipe[2]), sms, sm_mhz, pipe[0], pipe[1], tag)
        roofline.update(kernel=kernel_name, kernel_ms=k_ms, traffic=hbm["traffic"],
                        hbm={k: hbm[k] for k in ("achieved", "peak", "unit", "frac", "peak_kind",
                                                 "algorithmic_bytes_per_launch", "frac_of_nominal",
                                                 "same_run_copy_gbs")})
        # the attainable rate: the lower of the HBM bound (peak / bytes per element)
        # and the pipe bound (peak / instructions per element)
        ipe = roofline["instructions_per_element"]
        hbm_bound = peak * 1e9 / bpe / 1e6
        pipe_bound = roofline["peak"] * 1e12 / ipe / 1e6 if ipe else None
        att = min(hbm_bound, pipe_bound) if pipe_bound else hbm_bound
        roofline["attainable"] = {"melem_s": att, "unit": "Melem/s", "hbm_bound_melem_s": hbm_bound,
                                  "pipe_bound_melem_s": pipe_bound, "frac": melem_k / att}

    result = {"metric": METRIC, "value": value, "unit": "Melem/s", "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": FORMS[args.form][1], "data": "synthetic",
              "config": {"workload": wl_name, "n_elem_per_gpu": n, "bytes_per_element": bpe,
                         "launch_shape": shape_dict(shape),
                         "l2": "inputs larger than L2: %.2f GB read+written per step per GPU" % (n * bpe / 1e9),
                         "parallelism": f"weak: {world} independent mesh(es), one per GPU"},
              "roofline": roofline, "gpu_launches": int(launches), "clocks": clk}
    if args.only:
        pass
    elif rank == 0 and world == 1 and args.workload == "tet" and not lap:
        if args.form == "fp64":
            # the GPU's FP64 results of the timed steps, for the error statistics
            gpu_out = tuple(t.clone() for t in out)
        del out
        torch.cuda.empty_cache()
        rates = dict(sms=sms, sm_mhz=sm_mhz)
        result["mixed_form"] = mixed_form(ctx, dev, api, X, coefs, args)
        if not args.no_fp64:
            result["double_word_form"], result["fp64_forms"] = double_forms(ctx, dev, api, X, coefs, args, rates)
            result["cfg1_stated"] = cfg1_stated(ctx, dev, api, args, rates)
            result["threads_per_element"] = tpe_study(ctx, dev, api, mesh, coefs, args)
        del X, C
        torch.cuda.empty_cache()
        if not args.no_e2e:
            result["e2e"] = e2e(ctx, api, mesh, coefs, args)
        if not args.no_prism:
            result["prism_form"] = prism_form(ctx, dev, api, args, rates)
            result["coef_function_form"] = coef_function_form(ctx, dev, api, args)
        if not args.no_fp64:
            result["packed_form"] = packed_form(ctx, dev, api, mesh, args)
            result["ordering_study"] = ordering_study(ctx, dev, api, mesh, coefs, args)
        if not args.no_indexed:
            result["indexed_form"] = indexed_form(ctx, dev, api, coefs, args)
            result["apply_form"] = apply_form(ctx, dev, api, coefs, args)
        if not args.no_batch:
            result["batched"] = bench_batch(api, dev, args)
        if not args.no_serve:
            result["serving"] = bench_serve(api, dev, args)
        if not args.no_cpu_baseline and args.form == "fp64":
            result["cpu_baseline"] = cpu_baseline(mesh, coefs, gpu_out=gpu_out, tol=1e-12)
        result["paper_context"] = paper_context()
    elif rank == 0:
        result["e2e"] = {"value": None, "unit": "Melem/s", "note": "measured at N=1 only"}
    if rank == 0:
        print(json.dumps(result), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


def mixed_form(ctx, dev, api, X, coefs, args):
    """The same mesh and coefficients in the mixed form (float bulk, double Jacobian
    for mean ratio < 0.1; main kernel plus fix-up per step): step time with CUDA
    events on the stream, main-kernel time from the library's profiling events,
    HBM roofline with the hash-gated ncu DRAM bytes."""
    import torch
    n = X.shape[0]
    C = torch.from_numpy(np.ascontiguousarray(coefs.reshape(n, -1).astype(np.float32))).to(dev)
    out = api.alloc_out(api.TET, n, api.FP32_MIXED, api.AOS, dev, with_flags=True)
    kw = dict(kind=api.GENERIC, quad=api.QUAD_TET4, coef_mode=api.PER_ELEMENT, prec=api.FP32_MIXED,
              layout=api.AOS, out_layout=api.AOS)
    shape = ctx.tune(api.TET, X, C, out=out, **kw)
    call = lambda: ctx.integrate(api.TET, X, C, out=out, **kw)
    for _ in range(5):
        call()
    torch.cuda.synchronize(dev)
    reps = max(20, min(400, args.steps // 5))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        call()
    e1.record()
    torch.cuda.synchronize(dev)
    step_ms = e0.elapsed_time(e1) / reps
    k_ms = kernel_ms(ctx, call, reps)
    bpe = api.bytes_per_element(api.TET, api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, api.FP32_MIXED)
    peak, peak_kind = measured_peaks()
    roof = hbm_roofline(n, bpe, k_ms, peak, f"{peak_kind} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                        ncu_record("tet_generic_mixed_aos", "dram_bytes"))
    roof["kernel"] = "elem_kernel<TET,GENERIC,MIXED,TET4,per-element,AOS,AOS>"
    flagged = int((out[2] & 1).sum().item())
    del C, out
    torch.cuda.empty_cache()
    return {"workload": MIXED_WORKLOAD, "value": n / step_ms / 1e3, "unit": "Melem/s", "ms_per_step": step_ms,
            "dtype": "f32 (FP64 Jacobian for flagged elements)", "tolerance": "2e-5 relative Frobenius per element",
            "launch_shape": shape_dict(shape), "flagged_to_fp64": flagged, "roofline": roof}


def prism_workload(rank: int, n_slab: int = 1000):
    from paper_1504_01023_gb300 import meshgen
    mesh = meshgen.prism_slab_mesh(n_slab, None, 0.1, seed=meshgen.SEED_BASE + 3 + 1000 * rank)
    coefs = meshgen.generic_coefs(len(mesh), 6, seed=meshgen.SEED_BASE + 3 + 1000 * rank)
    return mesh, coefs


def prism_form(ctx, dev, api, args, rates):
    """The 2,000,000 generic prisms (per-point coefficients), mixed form, timed
    with CUDA events around the main kernel."""
    import torch
    mesh, coefs = prism_workload(0, args.n_slab)
    n = len(mesh)
    X = torch.from_numpy(np.ascontiguousarray(mesh)).to(dev)
    C = torch.from_numpy(np.ascontiguousarray(coefs.reshape(n, -1).astype(np.float32))).to(dev)
    out = api.alloc_out(api.PRISM, n, api.FP32_MIXED, api.AOS, dev, with_flags=True)
    kw = dict(kind=api.GENERIC, quad=api.QUAD_PRISM6, coef_mode=api.PER_QPOINT, prec=api.FP32_MIXED,
              layout=api.AOS, out_layout=api.AOS)
    shape = ctx.tune(api.PRISM, X, C, out=out, **kw)
    for _ in range(3):
        ctx.integrate(api.PRISM, X, C, out=out, **kw)
    torch.cuda.synchronize(dev)
    reps = max(20, min(200, args.steps // 20))
    ctx.set_profiling(True)
    ctx.kernel_time(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        ctx.integrate(api.PRISM, X, C, out=out, **kw)
    e1.record()
    kms, kn = ctx.kernel_time(reset=True)
    ctx.set_profiling(False)
    step_ms = e0.elapsed_time(e1) / reps
    bpe = api.bytes_per_element(api.PRISM, api.GENERIC, api.QUAD_PRISM6, api.PER_QPOINT, api.FP32_MIXED)
    k_ms = kms / kn
    peak, _ = measured_peaks()
    gbs = n * bpe / (k_ms * 1e-3) / 1e9
    del out
    # the same prisms in the double-precision forms (tuned shapes, which may put
    # two threads on each element)
    gen = {"workload": "the same 2,000,000 prisms and coefficients, results within 1e-12 of the FP64 oracle"}
    C64 = C.double()
    del C
    for name, prec, tg in (("double_word", api.FP64_DW, "prism_generic_dw_aos"),
                           ("native_fp64", api.FP64, "prism_generic_fp64_aos")):
        gen[name] = _fp64_run(ctx, dev, api, X, C64, api.PRISM, api.GENERIC, api.QUAD_PRISM6, prec, args,
                              cm=api.PER_QPOINT, rates=rates, tag=tg)
    del C64
    torch.cuda.empty_cache()
    # the Laplace kind on the same prisms: d^0 per point, in the three precision forms
    from paper_1504_01023_gb300 import meshgen
    d0 = meshgen.poisson_coefs(n, 6, None, seed=meshgen.SEED_BASE + 3)
    lap = {"workload": "the same 2,000,000 prisms, Laplace operator, d^0 ~ U[-1,1] per integration point"}
    for name, prec in (("mixed", api.FP32_MIXED), ("double_word", api.FP64_DW), ("native_fp64", api.FP64)):
        Cd = torch.from_numpy(np.ascontiguousarray(d0.astype(np.float32 if prec == api.FP32_MIXED else np.float64))).to(dev)
        lap[name] = _fp64_run(ctx, dev, api, X, Cd, api.PRISM, api.POISSON, api.QUAD_PRISM6, prec, args,
                              cm=api.PER_QPOINT, rates=rates,
                              tag=None if prec == api.FP32_MIXED else f"prism_poisson_{'fp64' if prec == api.FP64 else 'dw'}_aos")
        del Cd
    del X
    torch.cuda.empty_cache()
    return {"workload": PRISM_WORKLOAD, "value": n / step_ms / 1e3, "unit": "Melem/s", "ms_per_step": step_ms,
            "kernel_ms": k_ms, "bytes_per_element": bpe, "achieved_gbs": gbs, "hbm_frac": gbs / peak,
            "launch_shape": {"elements_per_block": shape[0], "persistent": shape[1], "threads_per_element": shape[2]},
            "dtype": "f32", "double_precision_forms": gen, "laplace": lap}


def _indexed_run(ctx, dev, api, et, nodes, conn, coefs, kind, quad, cm, args):
    """Kernel time of one mixed-form set with a node table (tuned shape), and the
    algorithmic bytes: per element its node indices, coefficients and outputs,
    plus every node's coordinates once."""
    import torch
    n = len(conn)
    X = torch.from_numpy(nodes).to(dev)
    K = torch.from_numpy(conn).to(dev)
    C = torch.from_numpy(np.ascontiguousarray(coefs.reshape(n, -1).astype(np.float32))).to(dev)
    out = api.alloc_out(et, n, api.FP32_MIXED, api.AOS, dev, with_flags=True)
    kw = dict(kind=kind, quad=quad, coef_mode=cm, prec=api.FP32_MIXED, layout=api.INDEXED, out_layout=api.AOS,
              conn=K)
    shape = ctx.tune(et, X, C, out=out, **kw)
    for _ in range(3):
        ctx.integrate(et, X, C, out=out, **kw)
    torch.cuda.synchronize(dev)
    reps = max(20, min(200, args.steps // 10))
    ctx.set_profiling(True)
    ctx.kernel_time(reset=True)
    for _ in range(reps):
        ctx.integrate(et, X, C, out=out, **kw)
    kms, kn = ctx.kernel_time(reset=True)
    ctx.set_profiling(False)
    k_ms = kms / kn
    ns = api.NS[et]
    per = api.bytes_per_element(et, kind, quad, cm, api.FP32_MIXED) - 3 * ns * 8 + ns * 4
    total = n * per + len(nodes) * 24
    peak, _ = measured_peaks()
    gbs = total / (k_ms * 1e-3) / 1e9
    del X, K, C, out
    torch.cuda.empty_cache()
    return {"value": n / k_ms / 1e3, "unit": "Melem/s", "kernel_ms": k_ms, "nodes": len(nodes),
            "bytes_per_element": total / n, "bytes_per_element_element_contiguous":
                api.bytes_per_element(et, kind, quad, cm, api.FP32_MIXED),
            "achieved_gbs": gbs, "hbm_frac": gbs / peak, "launch_shape": shape_dict(shape)}


def indexed_form(ctx, dev, api, coefs, args):
    """The headline tetrahedra and the 2M generic prisms with connectivity-indexed
    geometry (a node array plus an int32 element -> node table) instead of
    per-element coordinates: the same elements, coefficients and results."""
    from paper_1504_01023_gb300 import meshgen
    nodes, conn = meshgen.tet_cube_indexed(args.n_cubes, 0.2, seed=SEED)
    tet = _indexed_run(ctx, dev, api, api.TET, nodes, conn, coefs, api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT, args)
    del nodes, conn
    nodes, conn = meshgen.prism_slab_indexed(args.n_slab, None, 0.1, seed=meshgen.SEED_BASE + 3)
    pc = meshgen.generic_coefs(len(conn), 6, seed=meshgen.SEED_BASE + 3)
    prism = _indexed_run(ctx, dev, api, api.PRISM, nodes, conn, pc, api.GENERIC, api.QUAD_PRISM6, api.PER_QPOINT,
                         args)
    return {"workload": "the headline generic tetrahedra (100^3 x 6, TET4, per-element coefficients) and the 2M "
                        "generic prisms (PRISM6, per-point coefficients), mixed form, node array + int32 "
                        "element -> node table, element-contiguous coefficients and outputs",
            "value": tet["value"], "unit": "Melem/s", "hbm_frac": tet["hbm_frac"], "tet": tet, "prism": prism}


def apply_form(ctx, dev, api, coefs, args):
    """Matrix-free y += sum_e P_e^T A^e P_e x and f += sum_e P_e^T b^e over the
    headline tetrahedra with a node table: the element matrices are consumed
    where they are computed and never written. Algorithmic bytes: per element its
    indices and coefficients, plus per node x read once and y, f read and
    written once."""
    import torch
    from paper_1504_01023_gb300 import meshgen
    nodes, conn = meshgen.tet_cube_indexed(args.n_cubes, 0.2, seed=SEED)
    n, m = len(conn), len(nodes)
    X = torch.from_numpy(nodes).to(dev)
    K = torch.from_numpy(conn).to(dev)
    C = torch.from_numpy(np.ascontiguousarray(coefs.reshape(n, -1).astype(np.float32))).to(dev)
    x = torch.from_numpy(np.random.default_rng(SEED).uniform(-1, 1, m).astype(np.float32)).to(dev)
    y = torch.zeros(m, dtype=torch.float32, device=dev)
    f = torch.zeros(m, dtype=torch.float32, device=dev)
    call = lambda: ctx.apply(api.TET, X, K, C, api.GENERIC, api.QUAD_TET4, x, y, f, api.PER_ELEMENT,
                             api.FP32_MIXED)
    for _ in range(3):
        call()
    torch.cuda.synchronize(dev)
    reps = max(20, min(200, args.steps // 10))
    ctx.set_profiling(True)
    ctx.kernel_time(reset=True)
    for _ in range(reps):
        call()
    kms, kn = ctx.kernel_time(reset=True)
    ctx.set_profiling(False)
    k_ms = kms / kn
    total = n * (4 * 4 + 20 * 4) + m * 4 * 5
    peak, _ = measured_peaks()
    gbs = total / (k_ms * 1e-3) / 1e9
    del X, K, C, x, y, f
    torch.cuda.empty_cache()
    return {"workload": "y += A x and f += b, matrix-free (element matrices never stored), the headline generic "
                        "tetrahedra (TET4, per-element coefficients) with a node table, mixed form, float atomics",
            "value": n / k_ms / 1e3, "unit": "Melem/s", "kernel_ms": k_ms, "bytes_per_element": total / n,
            "achieved_gbs": gbs, "hbm_frac": gbs / peak, "nodes": m}


def packed_form(ctx, dev, api, mesh, args):
    """The Laplace tetrahedra (TET1, d^0 = 1 per element) on the headline mesh with
    full and with packed (upper-triangle, 10 of 16 entries) A^e, in the mixed and
    the double-word forms; kernel times from the library's profiling events."""
    import torch
    n = len(mesh)
    X = torch.from_numpy(np.ascontiguousarray(mesh)).to(dev)
    peak, _ = measured_peaks()
    res = {"workload": "Laplace tetrahedra, 6,000,000 elements, TET1, d^0 = 1 per element, element-contiguous "
                       "order; A^e full (16 entries) or packed (upper triangle, 10 entries)"}
    for prec, name in ((api.FP32_MIXED, "mixed"), (api.FP64_DW, "double_word")):
        dt = torch.float32 if prec == api.FP32_MIXED else torch.float64
        C = torch.ones((n, 1), dtype=dt, device=dev)
        for packed in (False, True):
            out = api.alloc_out(api.TET, n, prec, api.AOS, dev, with_flags=True, packed=packed)
            kw = dict(kind=api.POISSON, quad=api.QUAD_TET1, coef_mode=api.PER_ELEMENT, prec=prec, layout=api.AOS,
                      out_layout=api.AOS, packed=packed)
            ctx.tune(api.TET, X, C, out=out, **kw)
            for _ in range(3):
                ctx.integrate(api.TET, X, C, out=out, **kw)
            torch.cuda.synchronize(dev)
            ctx.set_profiling(True)
            ctx.kernel_time(reset=True)
            for _ in range(max(20, min(200, args.steps // 10))):
                ctx.integrate(api.TET, X, C, out=out, **kw)
            kms, kn = ctx.kernel_time(reset=True)
            ctx.set_profiling(False)
            k_ms = kms / kn
            cs = 4 if prec == api.FP32_MIXED else 8
            bpe = 96 + cs + (10 if packed else 16) * cs + 4 * cs
            gbs = n * bpe / (k_ms * 1e-3) / 1e9
            res[f"{name}_{'packed' if packed else 'full'}"] = {"value": n / k_ms / 1e3, "unit": "Melem/s",
                                                              "bytes_per_element": bpe, "achieved_gbs": gbs,
                                                              "hbm_frac": gbs / peak}
            del out
        del C
    del X
    torch.cuda.empty_cache()
    res.update(value=res["mixed_packed"]["value"], unit="Melem/s", hbm_frac=res["mixed_packed"]["hbm_frac"])
    return res


def ordering_study(ctx, dev, api, mesh, coefs, args):
    """A counterpart of the paper's Table 7 (Sec. 5): nanoseconds per element of
    the QSS, SQS and SSQ loop orderings (Algorithms 2-7) for the four cases
    Poisson / convection-diffusion x tetrahedra / prisms, mixed form, element-
    contiguous order, tuned launch shape, 1,000,000 tetrahedra (a prefix of the
    headline mesh) and 500,000 prisms. Poisson: d^0 per point (TET4, PRISM6);
    convection-diffusion: 20 coefficients per element."""
    import torch
    from paper_1504_01023_gb300 import meshgen
    nt, npr = min(1_000_000, len(mesh)), 500_000
    pmesh = meshgen.prism_slab_mesh(1000, None, 0.1, seed=meshgen.SEED_BASE + 3, n_elem=npr)
    cases = {
        ("poisson", "tetra"): (api.TET, mesh[:nt], meshgen.poisson_coefs(nt, 4, None, seed=SEED), api.POISSON,
                               api.QUAD_TET4, api.PER_QPOINT),
        ("poisson", "prism"): (api.PRISM, pmesh, meshgen.poisson_coefs(npr, 6, None, seed=SEED), api.POISSON,
                               api.QUAD_PRISM6, api.PER_QPOINT),
        ("conv-diff", "tetra"): (api.TET, mesh[:nt], coefs[:nt], api.GENERIC, api.QUAD_TET4, api.PER_ELEMENT),
        ("conv-diff", "prism"): (api.PRISM, pmesh, meshgen.generic_coefs(npr, 1, seed=SEED), api.GENERIC,
                                 api.QUAD_PRISM6, api.PER_ELEMENT),
    }
    table = {}
    for (problem, elem), (et, m, c, kind, quad, cm) in cases.items():
        n = len(m)
        X = torch.from_numpy(np.ascontiguousarray(m)).to(dev)
        C = torch.from_numpy(np.ascontiguousarray(c.reshape(n, -1).astype(np.float32))).to(dev)
        out = api.alloc_out(et, n, api.FP32_MIXED, api.AOS, dev, with_flags=True)
        for name, order in (("QSS", api.QSS), ("SQS", api.SQS), ("SSQ", api.SSQ)):
            kw = dict(kind=kind, quad=quad, coef_mode=cm, prec=api.FP32_MIXED, layout=api.AOS, out_layout=api.AOS,
                      ordering=order)
            ctx.tune(et, X, C, out=out, **kw)
            ctx.integrate(et, X, C, out=out, **kw)
            torch.cuda.synchronize(dev)
            ctx.set_profiling(True)
            ctx.kernel_time(reset=True)
            for _ in range(10):
                ctx.integrate(et, X, C, out=out, **kw)
            kms, kn = ctx.kernel_time(reset=True)
            ctx.set_profiling(False)
            table.setdefault(name, {})[f"{problem} {elem}"] = kms / kn * 1e6 / n   # ns per element
        del X, C, out
    torch.cuda.empty_cache()
    return {"workload": "ns per element (lower is better) of the QSS, SQS and SSQ orderings, mixed form: 1,000,000 "
                        "tetrahedra and 500,000 prisms; Poisson with d^0 per point, convection-diffusion with "
                        "per-element coefficients", "unit": "ns/element", "table": table}


def coef_function_form(ctx, dev, api, args):
    """The 2M generic prisms with the coefficients at every point computed from a
    function of a nodal field (c_j(u_Q) = P0_j + P1_j u_Q + P2_j u_Q^2) instead of
    read as 120 per-point values: 24 instead of 480 coefficient bytes per element.
    Mixed form, element-contiguous order, tuned shape."""
    import torch
    mesh, _ = prism_workload(0, args.n_slab)
    n = len(mesh)
    x, y, z = mesh[..., 0], mesh[..., 1], mesh[..., 2]
    u = (np.sin(3.0 * x) + y * y - 0.5 * z).astype(np.float32)
    P = np.random.default_rng(SEED).uniform(-1.0, 1.0, (3, 20))
    for i in (5, 10, 15):
        P[0, i] += 4.0
    X = torch.from_numpy(np.ascontiguousarray(mesh)).to(dev)
    U = torch.from_numpy(np.ascontiguousarray(u)).to(dev)
    del mesh
    out = api.alloc_out(api.PRISM, n, api.FP32_MIXED, api.AOS, dev, with_flags=True)
    kw = dict(kind=api.GENERIC, quad=api.QUAD_PRISM6, coef_mode=api.COEF_FN_U, prec=api.FP32_MIXED, layout=api.AOS,
              out_layout=api.AOS, coef_fn=P)
    shape = ctx.tune(api.PRISM, X, U, out=out, **kw)
    for _ in range(3):
        ctx.integrate(api.PRISM, X, U, out=out, **kw)
    torch.cuda.synchronize(dev)
    ctx.set_profiling(True)
    ctx.kernel_time(reset=True)
    for _ in range(max(20, min(200, args.steps // 10))):
        ctx.integrate(api.PRISM, X, U, out=out, **kw)
    kms, kn = ctx.kernel_time(reset=True)
    ctx.set_profiling(False)
    k_ms = kms / kn
    bpe = api.bytes_per_element(api.PRISM, api.GENERIC, api.QUAD_PRISM6, api.COEF_FN_U, api.FP32_MIXED)
    peak, _ = measured_peaks()
    gbs = n * bpe / (k_ms * 1e-3) / 1e9
    del X, U, out
    torch.cuda.empty_cache()
    return {"workload": "2,000,000 generic prisms, PRISM6, coefficients at every point from c(u) of a nodal field "
                        "(quadratic in u), mixed form, element-contiguous order", "value": n / k_ms / 1e3,
            "unit": "Melem/s", "kernel_ms": k_ms, "bytes_per_element": bpe, "achieved_gbs": gbs,
            "hbm_frac": gbs / peak, "launch_shape": shape_dict(shape)}


def _fp64_run(ctx, dev, api, X, C, et, kind, quad, prec, args, cm=None, rates=None, tag=None):
    """Tuned shape, then the average kernel time (profiling events) of repeated
    calls; with `tag`, the instruction-rate roofline of the form (FP64 pipe for
    plain FP64, instruction issue for double-word) from that ncu record."""
    import torch
    n = X.shape[0]
    cm = api.PER_ELEMENT if cm is None else cm
    out = api.alloc_out(et, n, prec, api.AOS, dev, with_flags=True)
    kw = dict(kind=kind, quad=quad, coef_mode=cm, prec=prec, layout=api.AOS, out_layout=api.AOS)
    shape = ctx.tune(et, X, C, out=out, **kw)
    call = lambda: ctx.integrate(et, X, C, out=out, **kw)
    for _ in range(3):
        call()
    torch.cuda.synchronize(dev)
    k_ms = kernel_ms(ctx, call, max(20, min(200, args.steps // 10)))
    flagged = int((out[2] & 1).sum().item())
    del out
    bpe = api.bytes_per_element(et, kind, quad, cm, prec)
    peak, src = measured_peaks()
    gbs = n * bpe / (k_ms * 1e-3) / 1e9
    res = {"value": n / k_ms / 1e3, "unit": "Melem/s", "kernel_ms": k_ms, "bytes_per_element": bpe,
           "achieved_gbs": gbs, "hbm_frac": gbs / peak, "peak_source": src, "flagged_to_fp64": flagged,
           "launch_shape": shape_dict(shape)}
    if tag is not None and rates is not None:
        if prec == api.FP64:
            res["fp64_pipe"] = pipe_roofline(res["value"], ncu_record(tag, "fp64_pipe_inst_per_elem"), rates["sms"],
                                             rates["sm_mhz"], FP64_PIPE_PER_CLK_SM, "FP64-pipe", tag)
        else:
            res["issue"] = pipe_roofline(res["value"], ncu_record(tag, "inst_per_elem"), rates["sms"],
                                         rates["sm_mhz"], ISSUE_PER_CLK_SM, "thread", tag)
    return res


def double_forms(ctx, dev, api, X, coefs, args, rates):
    """The double-accuracy forms on the headline mesh (results within 1e-12 of the
    FP64 oracle): the double-word form (float pairs on the float pipes, edges in
    FP64, flagged elements in FP64) of the generic tetrahedra and of the Laplace
    tetrahedra (the 48,000-element Poisson workload scaled to 100^3 x 6: TET1,
    d^0 = 1); and the plain FP64 form of the Laplace tetrahedra."""
    import torch
    n = X.shape[0]
    wl = ("tetrahedra, 6,000,000 elements (100^3 x 6, jitter +-0.2h), element-contiguous order, tolerance 1e-12 "
          "relative Frobenius per element against the FP64 oracle")
    Cg = torch.from_numpy(np.ascontiguousarray(coefs.reshape(n, -1))).to(dev)
    dw_gen = _fp64_run(ctx, dev, api, X, Cg, api.TET, api.GENERIC, api.QUAD_TET4, api.FP64_DW, args, rates=rates,
                       tag="tet_generic_dw_aos")
    del Cg
    C1 = torch.ones((n, 1), dtype=torch.float64, device=dev)
    dw_lap = _fp64_run(ctx, dev, api, X, C1, api.TET, api.POISSON, api.QUAD_TET1, api.FP64_DW, args, rates=rates,
                       tag="tet_poisson_tet1_dw_aos")
    nat_lap = _fp64_run(ctx, dev, api, X, C1, api.TET, api.POISSON, api.QUAD_TET1, api.FP64, args, rates=rates,
                        tag="tet_poisson_tet1_fp64_aos")
    del C1
    torch.cuda.empty_cache()
    dword = {"workload": wl, "value": dw_gen["value"], "unit": "Melem/s", "hbm_frac": dw_gen["hbm_frac"],
             "dtype": "f32 double-word (float pairs), f64 edge vectors and f64 for flagged elements",
             "precision_enum": "FE_FP64_DW", "tolerance": "1e-12 relative Frobenius per element (the FP64 tolerance)",
             "roofline": dw_gen.get("issue"), "generic_tet4": dw_gen, "poisson_tet1": dw_lap}
    fp64 = {"workload": wl + "; Laplace operator, TET1, d^0 = 1 (the 48,000-element Poisson workload scaled)",
            "value": nat_lap["value"], "unit": "Melem/s", "hbm_frac": nat_lap["hbm_frac"], "dtype": "f64",
            "roofline": nat_lap.get("fp64_pipe"), "poisson_tet1": nat_lap}
    return dword, fp64


def cfg1_stated(ctx, dev, api, args, rates):
    """The 48,000-element Poisson workload as stated (unit cube 20^3 x 6, jitter
    +-0.2h, TET1, d^0 = 1, FP64 and double-word forms): kernel throughput, and the
    latency of one call through fe_integrate_tet (host clock from the call to the
    end of a stream synchronisation) and its device time, p50 and p99 over 1,000
    calls each. At 12.7 MB the set is L2-resident and launch-bound."""
    import torch
    from paper_1504_01023_gb300 import meshgen
    mesh = meshgen.tet_cube_mesh(20, jitter=0.2, seed=meshgen.SEED_BASE + 1)
    n = len(mesh)
    X = torch.from_numpy(np.ascontiguousarray(mesh)).to(dev)
    C = torch.ones((n, 1), dtype=torch.float64, device=dev)
    res = {"workload": "Poisson (c^{ij} = I, d^0 = 1) on linear tetrahedra: unit cube 20^3 x 6 = 48,000 elements, "
                       "jitter +-0.2h, TET1, element-contiguous order, outputs 4x4 A^e + 4-vector b^e"}
    stream = torch.cuda.current_stream(dev)
    for name, prec in (("native_fp64", api.FP64), ("double_word", api.FP64_DW)):
        out = api.alloc_out(api.TET, n, prec, api.AOS, dev, with_flags=True)
        kw = dict(kind=api.POISSON, quad=api.QUAD_TET1, coef_mode=api.PER_ELEMENT, prec=prec, layout=api.AOS,
                  out_layout=api.AOS)
        shape = ctx.tune(api.TET, X, C, out=out, **kw)
        call = lambda: ctx.integrate(api.TET, X, C, out=out, **kw)
        for _ in range(20):
            call()
        torch.cuda.synchronize(dev)
        k_ms = kernel_ms(ctx, call, 1000)
        lat, dev_ms = [], []
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(1000)]
        for a, b in evs:
            t0 = time.perf_counter()
            a.record(stream)
            call()
            b.record(stream)
            stream.synchronize()
            lat.append((time.perf_counter() - t0) * 1e3)
        dev_ms = [a.elapsed_time(b) for a, b in evs]
        bpe = api.bytes_per_element(api.TET, api.POISSON, api.QUAD_TET1, api.PER_ELEMENT, prec)
        peak, _ = measured_peaks()
        res[name] = {"value": n / k_ms / 1e3, "unit": "Melem/s", "kernel_ms": k_ms, "bytes_per_element": bpe,
                     "hbm_frac": n * bpe / (k_ms * 1e-3) / 1e9 / peak, "launch_shape": shape_dict(shape),
                     "call_latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                                         "calls": len(lat), "clock": "host, call to stream synchronised"},
                     "call_device_ms": {"p50": float(np.percentile(dev_ms, 50)),
                                        "p99": float(np.percentile(dev_ms, 99)),
                                        "clock": "CUDA events around the call on its stream"}}
        del out
    del X, C
    torch.cuda.empty_cache()
    return res


def tpe_study(ctx, dev, api, mesh, coefs, args):
    """Threads per element (the thread-per-element versus group-per-element
    variants): for the generic tetrahedra (TET4, per-element coefficients; 2,000,000
    of the headline mesh) and the generic prisms (PRISM6, per-point coefficients;
    1,000,000 of the prism workload), in each precision form, the best launch shape
    of every threads-per-element value (elements per block x persistent, timed
    like the autotuner), its Melem/s, and the shape the autotuner keeps."""
    import torch
    from paper_1504_01023_gb300 import meshgen
    nt, npr = min(2_000_000, len(mesh)), 1_000_000
    pm, pc = prism_workload(0, args.n_slab)
    cases = {"generic tetrahedra, TET4, per-element coefficients, 2,000,000 elements":
                 (api.TET, mesh[:nt], coefs[:nt], api.QUAD_TET4, api.PER_ELEMENT, (1, 4, 16)),
             "generic prisms, PRISM6, per-point coefficients, 1,000,000 elements":
                 (api.PRISM, pm[:npr], pc[:npr], api.QUAD_PRISM6, api.PER_QPOINT, (1, 2, 6))}
    res = {"unit": "Melem/s", "note": "best shape per threads-per-element value; main-kernel time from profiling "
                                      "events, 10 calls after one warm-up"}
    for name, (et, m, c, quad, cm, tpes) in cases.items():
        n = len(m)
        X = torch.from_numpy(np.ascontiguousarray(m)).to(dev)
        row = {}
        for fname, prec in (("fp64", api.FP64), ("mixed", api.FP32_MIXED), ("double_word", api.FP64_DW)):
            cdt = np.float32 if prec == api.FP32_MIXED else np.float64
            C = torch.from_numpy(np.ascontiguousarray(c.reshape(n, -1).astype(cdt))).to(dev)
            out = api.alloc_out(et, n, prec, api.AOS, dev, with_flags=True)
            kw = dict(kind=api.GENERIC, quad=quad, coef_mode=cm, prec=prec, layout=api.AOS, out_layout=api.AOS,
                      out=out)
            call = lambda: ctx.integrate(et, X, C, **kw)
            per = {}
            for tpe in tpes:
                epw = 32 // tpe
                lim = 512 if (tpe == 1 and et == api.TET and prec != api.FP64_DW) else 256
                best = None
                warps = 2
                while warps * 32 <= lim:
                    for pers in (0, 1):
                        try:
                            ctx.set_shape(warps * epw, pers, et, X, C, tpe=tpe, **kw)
                        except api.FeError:          # the tile's shared memory does not fit
                            continue
                        call()
                        ms = kernel_ms(ctx, call, 10)
                        if best is None or ms < best[0]:
                            best = (ms, warps * epw, pers)
                    warps *= 2
                if best is not None:
                    per[f"tpe{tpe}"] = {"value": n / best[0] / 1e3, "elements_per_block": best[1],
                                        "persistent": best[2]}
            tuned = ctx.tune(et, X, C, **kw)
            row[fname] = {"threads_per_element": per, "tuner_keeps": shape_dict(tuned)}
            del C, out
        res[name] = row
        del X
        torch.cuda.empty_cache()
    return res


def e2e(ctx, api, mesh, coefs, args):
    """Same metric through the C ABI with pinned HOST buffers (the FP64 form of the
    headline step): the inputs are read and the outputs written in host memory
    inside the timed call."""
    import torch
    n = len(mesh)
    Xh = torch.from_numpy(np.ascontiguousarray(mesh)).pin_memory()
    Ch = torch.from_numpy(np.ascontiguousarray(coefs.reshape(n, -1).astype(np.float64))).pin_memory()
    out = api.alloc_out(api.TET, n, api.FP64, api.AOS, "cpu", with_flags=True, pin=True)
    kw = dict(kind=api.GENERIC, quad=api.QUAD_TET4, coef_mode=api.PER_ELEMENT, prec=api.FP64,
              layout=api.AOS, out_layout=api.AOS)
    for _ in range(2):
        ctx.integrate(api.TET, Xh, Ch, out=out, **kw)
    reps = max(3, min(20, args.steps // 100))
    t = time.perf_counter()
    for _ in range(reps):
        ctx.integrate(api.TET, Xh, Ch, out=out, **kw)
    dt = (time.perf_counter() - t) / reps
    bi = Xh.numel() * 8 + Ch.numel() * 8
    bo = out[0].numel() * 8 + out[1].numel() * 8 + out[2].numel()
    return {"value": n / dt / 1e6, "unit": "Melem/s", "h2d_bytes_per_step": int(bi), "d2h_bytes_per_step": int(bo),
            "ms_per_step": dt * 1e3, "steps": reps, "dtype": "f64",
            "path": "pinned host buffers through fe_integrate_tet (FE_MEM_HOST), FP64 form: the kernels read the "
                    "inputs and write the outputs in host memory over the host link, no staging copies; the call "
                    "returns when the outputs are in host memory"}


# ---------------------------------------------------------------------------
# Many meshes: the batched persistent launch and the serving loop
# ---------------------------------------------------------------------------
class DevicePool:
    """The seeded MixPool on the device, and per-mesh inputs cut from it."""

    def __init__(self, max_elems, seed, dev):
        import torch
        from paper_1504_01023_gb300 import meshgen
        self.mp = meshgen.MixPool(max_elems, seed)
        self.dev = dev
        self.base = {0: torch.from_numpy(self.mp.tet).to(dev), 1: torch.from_numpy(self.mp.prism).to(dev)}
        self.generic = torch.from_numpy(self.mp.generic.astype(np.float32)).to(dev)
        self.poisson = torch.from_numpy(self.mp.poisson.astype(np.float32)).to(dev)

    def mesh(self, et, kind, n):
        import torch
        from paper_1504_01023_gb300 import meshgen
        quad, cpq = meshgen.mix_spec(et, kind)
        off = self.mp.window(et, n)
        X = self.base[et][off:off + n].clone()
        k = (6 if cpq else 1)
        idx = (self.mp.coef_offset() + torch.arange(n * k, device=self.dev)) % self.poisson.numel()
        if kind == 0:
            C = self.poisson[idx].reshape(n, k).contiguous()
        else:
            C = self.generic[idx].reshape(n, 20 * k).contiguous()
        return X, C, quad, cpq


def bench_batch(api, dev, args):
    """256 meshes, sizes log-uniform in [1e3, 2e6], 50/50 tetrahedra/prisms and
    Poisson/generic, mixed precision, one persistent launch from a captured graph
    per step (tile size chosen by the library's autotuner on first submission)."""
    import torch
    from paper_1504_01023_gb300 import meshgen
    specs = meshgen.batch_mix(256, 1e3, 2e6, seed=meshgen.SEED_BASE + 4)
    pool = DevicePool(2_000_000, meshgen.SEED_BASE + 40, dev)
    ctx = api.Context(dev.index, autotune=True)
    items, keep, total, total_bytes = [], [], 0, 0
    for n, et, kind in specs:
        X, C, quad, cpq = pool.mesh(et, kind, n)
        out = api.alloc_out(et, n, api.FP32_MIXED, api.AOS, dev, with_flags=True)
        cm = api.PER_QPOINT if cpq else api.PER_ELEMENT
        items.append((et, api.make_args(et, X, C, kind, quad, cm, api.FP32_MIXED, api.AOS), api.make_out(*out, api.AOS)))
        keep.append((X, C, out))
        total += n
        total_bytes += n * api.bytes_per_element(et, kind, quad, cm, api.FP32_MIXED)
    del pool
    torch.cuda.synchronize(dev)
    ctx.batch_submit(items)                      # plan + autotune + graph capture
    for _ in range(3):
        ctx.batch_submit(items)
    torch.cuda.synchronize(dev)
    steps = max(5, min(50, args.steps // 200))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = api.launch_count()
    e0.record()
    for _ in range(steps):
        ctx.batch_submit(items)
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    ctx.sync()
    peak, _ = measured_peaks()
    gbs = total_bytes / (ms * 1e-3) / 1e9
    res = {"workload": "256 meshes, sizes log-uniform [1e3, 2e6] (seeded), 50/50 tetrahedra/prisms and "
                       "Poisson/generic (tet Poisson TET1, tet generic TET4 per element, prism PRISM6 per point), "
                       "mixed FP32 with FP64 Jacobian fallback, one persistent kernel per step from a captured graph",
           "n_elem": total, "value": total / ms / 1e3, "unit": "Melem/s", "ms_per_step": ms,
           "algorithmic_gb_per_step": total_bytes / 1e9, "achieved_gbs": gbs, "hbm_frac": gbs / peak,
           "gpu_launches_per_step": (api.launch_count() - l0) / steps, "steps": steps}
    ctx.close()
    del items, keep
    torch.cuda.empty_cache()
    return res


def bench_serve(api, dev, args):
    """Poisson arrivals (2000 requests/s, seeded) of requests on a pool of 64
    resident meshes (sizes log-uniform [1e4, 4e6], the batched mix), served under a
    120 GB HBM budget by the continuous-batching loop; an arrival-rate sweep; the
    loop's capacity (closed loop); then the same arrival stream replayed against the
    plain one-request-at-a-time FP64 path (first 0.25 s)."""
    import torch
    from paper_1504_01023_gb300 import meshgen
    specs = meshgen.batch_mix(64, 1e4, 4e6, seed=meshgen.SEED_BASE + 5)
    pool = DevicePool(4_000_000, meshgen.SEED_BASE + 50, dev)
    ctx = api.Context(dev.index, hbm_budget=120_000_000_000, serve_slots=4)
    meshes = []
    for n, et, kind in specs:
        X, C, quad, cpq = pool.mesh(et, kind, n)
        mid = ctx.mesh_register(et, X, api.AOS)
        meshes.append(dict(id=mid, et=et, kind=kind, quad=quad, cm=api.PER_QPOINT if cpq else api.PER_ELEMENT, C=C,
                           X=X, n=n))
    del pool
    torch.cuda.synchronize(dev)
    # warm the serving path before the timed windows: every resident mesh, one at a
    # time and then all at once, twice (first launch of each combination, growth of
    # the output pool and of the slots' fix-up lists to the working set)
    for m in meshes:
        tk = ctx.serve_submit(m["id"], m["kind"], m["quad"], m["cm"], m["C"])
        while ctx.serve_poll(tk) is None:
            time.sleep(0.0005)
        ctx.serve_release(tk)
    for _ in range(2):
        tks = [ctx.serve_submit(m["id"], m["kind"], m["quad"], m["cm"], m["C"]) for m in meshes]
        for tk in tks:
            while ctx.serve_poll(tk) is None:
                time.sleep(0.0005)
        ctx.serve_release_many(tks)
    lam, T = 2000.0, args.serve_seconds
    served, arrivals, choice = serve_open_loop(ctx, meshes, lam, T, meshgen.SEED_BASE + 55)
    # arrival-rate sweep: 2000/s x {2, 4, 8, 16}, a shorter window each
    sweep = []
    for k in (2, 4, 8, 16):
        r, _, _ = serve_open_loop(ctx, meshes, lam * k, min(T, 1.5), meshgen.SEED_BASE + 55 + k)
        sweep.append({key: r[key] for key in ("arrival_rate_per_s", "seconds", "requests", "errors", "p50_ms",
                                               "p99_ms", "sustained_melem_s", "offered_melem_s")})
    # capacity: closed loops with 48 and 96 requests outstanding
    saturated = [serve_saturated(api, ctx, meshes, max(1.0, args.serve_seconds / 2), d) for d in (48, 96)]
    upload = serve_upload_inclusive(api, ctx, meshes, dev, meshgen.SEED_BASE + 56)
    ctx.close()

    # plain one-request-at-a-time FP64 path on the same arrivals (first 0.25 s)
    sel = arrivals < 0.25
    arr, ch = arrivals[sel], choice[sel]
    cp = api.Context(dev.index)
    lat64, elems64 = [], 0
    C64 = {}
    # warm-up outside the window: one call per kernel the window uses (module load,
    # shared-memory attributes), on the smallest mesh of each combination
    warm = {}
    for j in sorted(set(ch.tolist()), key=lambda j: meshes[j]["n"]):
        m = meshes[j]
        warm.setdefault((m["et"], m["kind"], m["quad"], m["cm"]), j)
    for j in warm.values():
        m = meshes[j]
        C64[j] = m["C"].double()
        cp.integrate(m["et"], m["X"], C64[j], m["kind"], m["quad"], m["cm"], api.FP64, api.AOS, api.AOS)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for t_arr, j in zip(arr, ch):
        dt = t_arr - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        m = meshes[j]
        if j not in C64:
            C64[j] = m["C"].double()
        cp.integrate(m["et"], m["X"], C64[j], m["kind"], m["quad"], m["cm"], api.FP64, api.AOS, api.AOS)
        torch.cuda.synchronize(dev)
        lat64.append((time.perf_counter() - t0) - t_arr)
        elems64 += m["n"]
    wall64 = time.perf_counter() - t0
    cp.close()
    l64 = np.array(lat64) * 1e3
    plain = {"path": "fe_integrate_* FP64, one request at a time, synchronous", "arrival_window_s": 0.25,
             "requests": int(len(lat64)), "p50_ms": float(np.percentile(l64, 50)),
             "p99_ms": float(np.percentile(l64, 99)), "sustained_melem_s": elems64 / wall64 / 1e6}
    for m in meshes:
        m.pop("C"), m.pop("X")
    torch.cuda.empty_cache()
    return {"workload": "Poisson arrivals 2000/s (seeded) on 64 resident meshes, sizes log-uniform [1e4, 4e6], "
                        "50/50 tetrahedra/prisms and Poisson/generic, mixed precision, 120 GB budget, 4 stream slots",
            "served": served, "arrival_sweep": sweep, "saturated": saturated, "upload_inclusive": upload,
            "plain_fp64": plain}


def serve_upload_inclusive(api, ctx, meshes, dev, seed, n_meshes=16, passes=3):
    """Latency with the upload included: requests on meshes that are not resident.
    For each request, one after another: register its geometry from pinned host
    memory (fe_mesh_register copies it to the device), copy its coefficients from
    pinned host memory, submit, wait for the completion, then release the request
    and the mesh. Latency = wall clock from the start of the upload to the
    completion; `upload_ms` is the part before the submission. A seeded draw of
    `n_meshes` of the pool's meshes, `passes` times each."""
    import torch
    rng = np.random.default_rng(seed)
    pick = rng.choice(len(meshes), size=n_meshes, replace=False)
    host = {int(j): (meshes[j]["X"].cpu().pin_memory(), meshes[j]["C"].cpu().pin_memory()) for j in pick}
    stream = torch.cuda.current_stream(dev)
    lat, up, elems = [], [], 0
    order = [int(j) for _ in range(passes) for j in rng.permutation(pick)]
    for i, j in enumerate(order):
        m, (Xh, Ch) = meshes[j], host[j]
        t0 = time.perf_counter()
        mid = ctx.mesh_register(m["et"], Xh, api.AOS)
        Cd = Ch.to(dev, non_blocking=True)
        stream.synchronize()
        t1 = time.perf_counter()
        tk = ctx.serve_submit(mid, m["kind"], m["quad"], m["cm"], Cd)
        while ctx.serve_poll(tk) is None:
            time.sleep(0.0001)
        t2 = time.perf_counter()
        ctx.serve_release(tk)
        ctx.mesh_release(mid)
        del Cd
        if i >= n_meshes // 2:          # the first requests warm the register path
            lat.append((t2 - t0) * 1e3)
            up.append((t1 - t0) * 1e3)
            elems += m["n"]
    lat, up = np.array(lat), np.array(up)
    return {"path": "fe_mesh_register from pinned host memory + coefficient copy + fe_serve_submit, one request "
                    "at a time, mesh released after each", "requests": int(len(lat)),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "upload_p50_ms": float(np.percentile(up, 50)), "upload_p99_ms": float(np.percentile(up, 99)),
            "mean_elements": elems / max(len(lat), 1), "sustained_melem_s": elems / (lat.sum() * 1e-3) / 1e6}


def serve_open_loop(ctx, meshes, lam, T, seed):
    """Open loop: seeded Poisson arrivals at `lam` requests/s for T seconds, each on a
    mesh drawn from the pool; completions taken from the completion queue by a
    second thread. Latency = library completion stamp - submission stamp."""
    import threading
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / lam, size=int(lam * T * 1.5) + 100)
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < T]
    choice = rng.integers(0, len(meshes), size=len(arrivals))
    sizes, lock, lat, done_elems, errors = {}, threading.Lock(), [], [0], []
    finished = threading.Event()
    submitted = [0]

    def collector():
        while True:
            with lock:
                pending = submitted[0] - len(lat)
            if pending == 0 and finished.is_set():
                return
            got = ctx.serve_wait_any(timeout_us=2000, max_results=64)
            for tk, r in got:
                if r.status != 0:
                    errors.append(r.status)
                with lock:
                    n = sizes.pop(tk)
                    lat.append((r.t_done_us - r.t_submit_us, r.t_done_us, r.t_submit_us))
                done_elems[0] += n
            ctx.serve_release_many([tk for tk, _ in got])

    th = threading.Thread(target=collector, daemon=True)
    th.start()
    t0 = time.perf_counter()
    for t_arr, j in zip(arrivals, choice):
        dt = t_arr - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        m = meshes[j]
        with lock:
            tk = ctx.serve_submit(m["id"], m["kind"], m["quad"], m["cm"], m["C"])
            sizes[tk] = m["n"]
            submitted[0] += 1
    finished.set()
    th.join(timeout=300)
    wall = time.perf_counter() - t0
    lat_ms = np.array([x[0] for x in lat]) / 1e3
    span_s = (max(x[1] for x in lat) - min(x[2] for x in lat)) / 1e6
    offered = float(sum(meshes[j]["n"] for j in choice)) / T / 1e6
    return ({"arrival_rate_per_s": lam, "seconds": T, "requests": int(len(lat)), "errors": len(errors),
             "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
             "mean_ms": float(lat_ms.mean()), "sustained_melem_s": done_elems[0] / span_s / 1e6,
             "offered_melem_s": offered, "wall_s": wall}, arrivals, choice)


def serve_saturated(api, ctx, meshes, seconds, depth):
    """Capacity of the serving loop: a closed loop keeps `depth` requests of the same
    mix outstanding (completions taken from the completion queue, released in one
    call and replaced one by one) for about `seconds`; throughput = elements completed / (last completion - first
    submission), with the library's own timestamps. HBM fraction from the
    algorithmic bytes of each request."""
    from paper_1504_01023_gb300 import meshgen
    rng = np.random.default_rng(meshgen.SEED_BASE + 56)
    bpe = {}
    for m in meshes:
        key = (m["et"], m["kind"], m["quad"], m["cm"])
        if key not in bpe:
            bpe[key] = api.bytes_per_element(m["et"], m["kind"], m["quad"], m["cm"], api.FP32_MIXED)
    out, lat, first, last, elems, nbytes, errors = {}, [], None, 0.0, 0, 0, 0
    t_end = time.perf_counter() + seconds

    def submit():
        m = meshes[int(rng.integers(0, len(meshes)))]
        out[ctx.serve_submit(m["id"], m["kind"], m["quad"], m["cm"], m["C"])] = m

    for _ in range(depth):
        submit()
    while out:
        got = ctx.serve_wait_any(timeout_us=100000, max_results=64)
        for tk, r in got:
            m = out.pop(tk)
            errors += r.status != 0
            first = r.t_submit_us if first is None else min(first, r.t_submit_us)
            last = max(last, r.t_done_us)
            lat.append((r.t_done_us - r.t_submit_us) / 1e3)
            elems += m["n"]
            nbytes += m["n"] * bpe[(m["et"], m["kind"], m["quad"], m["cm"])]
        # what finished is released in one call; each is replaced by a new request
        # submitted on its own (submitting the replacements as one group keeps
        # them together as a cohort, which measured slower at 48 outstanding)
        ctx.serve_release_many([tk for tk, _ in got])
        if time.perf_counter() < t_end:
            for _ in got:
                submit()
    span = (last - first) / 1e6
    peak, src = measured_peaks()
    gbs = nbytes / span / 1e9
    return {"loop": f"closed, {depth} requests outstanding", "requests": len(lat), "errors": int(errors),
            "seconds": span, "melem_s": elems / span / 1e6, "achieved_gbs": gbs, "hbm_frac": gbs / peak,
            "peak_source": src, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99))}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
