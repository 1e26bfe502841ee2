#!/usr/bin/env python
"""Benchmark: BSE force evaluations per second on one GB300 (or N independent replicas).

A step is one full force evaluation of the 63-atom diamond-vacancy Gaussian-well model
(72^3 grid, N_occ = 128, N_pdep = 256, FP64): new atomic positions -> local potential,
ground state, tau cache, Davidson for the lowest TDA-BSE root, U vector, Z-vector solve,
relaxed density and forces.  Inputs (the PDEP basis) are resident in HBM; every step
recomputes everything from the positions.  The working set (24.7 GB of tau) is far
larger than L2, so no L2 flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank solves its own replica (no collective on the data path; a
gloo group only reduces the timings), so scaling is weak.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BSE force evals/s (FP64, diamond-vacancy 63-atom model, 72^3, N_occ=128, N_pdep=256)"
UNIT = "force_evals/s"
DAVIDSON_TOL = 1e-8
MIXED_DAVIDSON_TOL = 1e-5
ZVEC_TOL = 1e-10
GS_TOL = 1e-10

# DRAM traffic per launch of the fused K1d/combine kernel from one ncu capture, valid
# only for the kernel source it was measured on (hash of kernels.cu).
# DRAM traffic of the timed kernels, from one ncu capture each of a smaller case of the same
# kernel (profiles/), keyed by a hash of the kernel's source text so that a changed kernel
# reports null.  tau_factor: DRAM bytes read per algorithmic tau byte; the traffic of a full
# launch is its algorithmic bytes with tau counted tau_factor times.
NCU_TRAFFIC = {
    # k1d_tma_kernel (column order, two-column register prefetch), N_occ = 64, 4-vector block:
    # 3.59 GB read + 0.37 GB written against 3.97 GB algorithmic (tau 3.11 GB read once);
    # profiles/k1d_tma_persistent_nocc64_mixed.md
    "baa5281222e96203": {"tau_factor": 1.0},
    # combine_tau_kernel (FP64), N_occ = 48, 2-vector block: 7.34 GB read + 0.28 GB written against
    # 4.24 GB algorithmic (tau 3.51 GB, read about twice: by the two output tiles of each pair);
    # profiles/combine_tau_nocc48_fp64.md
    "a5f5b8bfb34f34ad": {"tau_factor": 1.96},
}


def kernel_text(path, name):
    """Source text of the __global__ function `name` (with its template line)."""
    import re
    with open(path) as f:
        src = f.read()
    m = re.search(r"__global__[^;{]*?\b" + re.escape(name) + r"\s*\(", src)
    if not m:
        return ""
    start = src.rfind("\ntemplate", 0, m.start())
    start = start + 1 if start >= 0 and m.start() - start < 200 else m.start()
    return src[start:src.index("\n}\n", m.end()) + 3]


def kernel_source_hash(fname="kernels.cu", name="combine_tau_kernel"):
    txt = kernel_text(os.path.join(ROOT, "paper_2607_20728_gb300", "csrc", fname), name)
    return hashlib.sha256(txt.encode()).hexdigest()[:16]


def traffic_per_launch(key, alg_bytes_per_launch, tau_bytes):
    t = NCU_TRAFFIC.get(key)
    if not t:
        return None
    return alg_bytes_per_launch + (t["tau_factor"] - 1.0) * tau_bytes


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------------------
# oracle baseline (the reference arm and the cpu_baseline key)
def oracle_sample(spec, rows=1):
    """Time the oracle's own Liouville operator (oracle.liouville.Liouville: tau_{v'v} =
    W * (phi_v' phi_v) through its tau() method, the K1d accumulation and the K1e term of
    Eq. 2) for `rows` output rows of one apply on the full-size workload.  Each row needs N_occ
    screened convolutions on the 72^3 grid; the oracle's tau cache does not fit at this size
    (N_occ^2 grids), so every apply recomputes them.  The occupied orbitals are seeded random
    orthonormal functions standing in for the ground state (the oracle's dense eigensolve of the
    6859-function Hamiltonian alone exceeds the sample budget).  Returns (seconds per full
    apply, seconds measured)."""
    import types

    from oracle.basis import PWBasis
    from oracle.liouville import Liouville
    b = PWBasis(spec.lattice, spec.ecut, spec.grid)
    rng = np.random.default_rng(7)
    q, _ = np.linalg.qr(rng.standard_normal((b.npw, spec.n_occ)))
    phi = b.real_to_full(q.T)
    gs = types.SimpleNamespace(basis=b, phi=phi, phi_r=b.to_grid(phi), eps=np.zeros(spec.n_occ))
    op = Liouville(spec, gs=gs, tau_cache_bytes=0)
    t0 = time.perf_counter()
    A = op.Pc(b.real_to_full(rng.standard_normal((spec.n_occ, b.npw))))
    a_r = b.to_grid(A)
    drho = np.sum(np.conj(gs.phi_r) * a_r, axis=0)
    vH = b.coulomb(drho)
    for v in range(rows):
        acc = np.zeros(b.grid, dtype=np.complex128)
        for vp in range(spec.n_occ):
            acc += op.tau(vp, v) * a_r[vp]
        _ = b.from_grid(2.0 * vH * gs.phi_r[v] - acc)
    dt = time.perf_counter() - t0
    per_apply = dt / rows * spec.n_occ
    return per_apply, dt


def cpu_baseline(spec, applies_per_eval, rows=1):
    per_apply, dt = oracle_sample(spec, rows=rows)
    value = 1.0 / (per_apply * applies_per_eval)
    return {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "estimate": True,
            "sample": f"ESTIMATE: oracle (numpy FP64, oracle.liouville.Liouville.tau) time of {rows} of "
                      f"{spec.n_occ} output rows of one Liouville apply on the 72^3 workload ({dt:.1f} s), "
                      f"scaled to a full apply and multiplied by the {applies_per_eval} applies of one GPU "
                      f"force evaluation (ground state, U and Z-vector work not counted, so this overstates "
                      f"the oracle's speed); measured oracle force evaluations and applies on smaller cells "
                      f"are under oracle_plan"}


def workload_config(spec, world):
    return {"workload": "diamond-vacancy-63atom-72^3 (FP64 plain path)", "n_atoms": spec.n_atoms,
            "grid": list(spec.grid), "n_occ": spec.n_occ, "n_pdep": spec.n_pdep, "n_pw": spec.n_pw,
            "n_roots": 1, "davidson_tol": DAVIDSON_TOL, "zvector_tol": ZVEC_TOL, "gs_tol": GS_TOL,
            "l2": "working set (24.7 GB tau) larger than L2; no flush", "parallelism": f"replicas x{world}"}


def run_reference(args, rank, world):
    import bse_inputs
    if rank != 0:
        return
    spec = bse_inputs.diamond63()
    applies = 88  # trial vectors through the Liouville operator in one GPU FP64 force evaluation (measured)
    for _ in range(args.warmup):
        oracle_sample(spec, rows=1)
    vals = []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        per_apply, dt = oracle_sample(spec, rows=1)
        vals.append(1.0 / (per_apply * applies))
    wall = time.perf_counter() - t_all
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(spec, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "threads": thread_counts(), "estimate": True,
                             "sample": "1 of 128 output rows of one oracle Liouville apply per step "
                                       "(oracle.liouville.Liouville.tau, no tau cache at this size), scaled "
                                       f"by 128 rows and {applies} applies per force evaluation"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------
def max_over_ranks(x, dist=None):
    """Max of a host float over all ranks of a (gloo) process group; identity without one."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, t_max_s):
    """Units processed by all ranks divided by the slowest rank's time."""
    return world * units_per_rank / t_max_s


# ---------------------------------------------------------------------------------------
def measure_fp64_peak(n=8192, reps=3):
    """Dense FP64 rate of this GPU: torch.matmul (cuBLAS DGEMM) on n x n float64, best of reps,
    CUDA events on the current stream.  The denominator of the FP64 ALU roofline."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    c = a @ b
    stream = torch.cuda.current_stream()
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        torch.matmul(a, b, out=c)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b, c
    torch.cuda.empty_cache()
    return 2.0 * n ** 3 / (best / 1e3) / 1e12


def _event_ms(fn, reps=3):
    """Mean CUDA-event time of fn() on the current stream after one untimed call."""
    import torch
    stream = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def fft_comparator(pkg, sysm, n_rows):
    """The apply's wave-function transforms of n_rows real functions (n_rows / 2 packed complex
    grids) against cuFFT (torch.fft) on the same grids: the library's sphere-pruned transforms
    (bse_sphere_to_grid / bse_grid_to_sphere, scatter/gather included), its full-grid FFT
    (bse_fft3d, FP64 contexts only), and torch.fft.ifftn / fftn of n_rows / 2 and n_rows full
    grids.  Rates are counted as 5 N log2 N flops per complex grid."""
    import torch
    n1, n2, n3 = sysm.grid
    nr = n1 * n2 * n3
    nq = (n_rows + 1) // 2
    dt = torch.complex128 if sysm.precision == 0 else torch.complex64
    X = torch.randn(n_rows, sysm.n_pw, dtype=torch.float64, device="cuda")
    P = torch.empty((nq, n3, n2, n1), dtype=dt, device="cuda")
    Y = torch.empty(n_rows, sysm.n_pw, dtype=torch.float64, device="cuda")
    out = {"grids": [n1, n2, n3], "rows": n_rows, "packed_grids": nq, "dtype": str(dt).replace("torch.", "")}
    flops = 5.0 * nq * nr * np.log2(nr)
    out["sphere_inverse_ms"] = _event_ms(lambda: sysm.sphere_to_grid(X, out=P))

    def fwd():
        sysm.sphere_to_grid(X, out=P)
        sysm.grid_to_sphere(P, n_rows, out=Y)
    out["sphere_forward_ms"] = max(0.0, _event_ms(fwd) - out["sphere_inverse_ms"])
    if sysm.precision == 0:
        G = torch.randn((nq, n3, n2, n1), dtype=dt, device="cuda")
        out["full_grid_ms"] = _event_ms(lambda: pkg.bse_fft3d(G, +1))
        del G
    G = torch.randn((nq, n3, n2, n1), dtype=dt, device="cuda")
    out["cufft_ms"] = _event_ms(lambda: torch.fft.ifftn(G, dim=(1, 2, 3)))
    del G
    G = torch.randn((2 * nq, n3, n2, n1), dtype=dt, device="cuda")
    out["cufft_2x_batch_ms"] = _event_ms(lambda: torch.fft.ifftn(G, dim=(1, 2, 3)))
    del G, P, X, Y
    torch.cuda.empty_cache()
    for k in ("sphere_inverse_ms", "sphere_forward_ms", "full_grid_ms", "cufft_ms"):
        if k in out and out[k] > 0:
            out[k.replace("_ms", "_tflops_equiv")] = flops / (out[k] / 1e3) / 1e12
    out["sphere_inverse_vs_cufft"] = out["cufft_ms"] / out["sphere_inverse_ms"] if out["sphere_inverse_ms"] else None
    return out


PARITY_DAVIDSON_TOL = {0: 1e-10, 1: 1e-6}


def parity_gpu(pkg, spec):
    """GPU force evaluations of a parity cell, FP64 and mixed: omega, forces and the Eq. 5-6
    densities, compared later with the oracle's."""
    import torch
    out = {}
    for prec in (0, 1):
        s = pkg.BSESystem(spec, gs_tol=3e-13 if prec == 0 else 1e-10, precision=prec)
        w, _ = s.davidson(n_roots=1, tol=PARITY_DAVIDSON_TOL[prec], max_iter=500)
        s.zvector(0, tol=1e-11 if prec == 0 else ZVEC_TOL, max_iter=3000)
        F = s.forces(0)
        out[prec] = (float(w[0]), F, s.density(0), s.density(1))
        s.close()
        torch.cuda.synchronize()
    return out


def oracle_force_eval_by_phase(spec, tol=1e-10):
    """The oracle's own force pipeline (forces.bse_forces, step by step) with a timer per phase."""
    from oracle import forces, model
    t = {}
    t0 = time.perf_counter()
    gs = model.GroundState(spec, all_states=True)
    t["ground_state_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    w, A, op = forces.excitation(spec, gs=gs, tol=tol)
    t["tau_and_davidson_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    U = forces.u_vector(op, A[0])
    t["u_vector_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    Z = forces.zvector_cg(op, U)
    t["zvector_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    rx, rz = forces.densities(op, A[0], Z)
    F = -forces.force_contraction(op, (rx + rz).real)
    t["forces_s"] = time.perf_counter() - t0
    t["total_s"] = sum(t.values())
    return t, (float(w[0]), F, rx.real.transpose(2, 1, 0), rz.real.transpose(2, 1, 0)), op


def oracle_apply_rates(op, spec, nbs=(1, 2, 4, 8)):
    """The oracle's Liouville.apply (tau cached) on blocks of N_b trial vectors: vectors/s."""
    b = op.basis
    rng = np.random.default_rng(99)
    out = {}
    for nb in nbs:
        A = [op.Pc(b.real_to_full(rng.standard_normal((spec.n_occ, b.npw)))) for _ in range(nb)]
        t0 = time.perf_counter()
        for a in A:
            op.apply(a)
        out[f"nb{nb}"] = nb / (time.perf_counter() - t0)
    return out


def thread_counts():
    out = {"cpu_count": os.cpu_count(), "fft": "numpy pocketfft, 1 thread"}
    try:
        from threadpoolctl import threadpool_info
        out["blas"] = [{"api": i.get("internal_api"), "threads": i.get("num_threads")} for i in threadpool_info()]
    except ImportError:
        out["blas"] = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS")}
        out["blas_note"] = "threadpoolctl not installed; OpenBLAS defaults to one thread per core"
    return out


def oracle_plan(parity=None):
    """The oracle timed on the host cores: its force evaluation by phase on the tiny
    cell, on the N_occ = 48 parity cell and on the smallest system of the 48-system batch; its
    Liouville apply at N_b = 1, 2, 4, 8 on the tiny and N_occ = 48 cells; and, when GPU results
    of the parity cell are given, the per-result error of the GPU paths against it."""
    import bse_inputs
    res = {"threads": thread_counts()}
    tiny = bse_inputs.tiny()
    t, _, op = oracle_force_eval_by_phase(tiny, tol=1e-10)
    res["tiny"] = {"force_eval": t, "apply_vectors_per_s": oracle_apply_rates(op, tiny)}
    m48 = bse_inputs.mid48()
    t, ref, op = oracle_force_eval_by_phase(m48, tol=1e-11)
    res["mid48"] = {"force_eval": t, "apply_vectors_per_s": oracle_apply_rates(op, m48)}
    specs = bse_inputs.batch48()
    small = min(specs, key=lambda sp: np.prod(sp.grid) * sp.n_occ ** 2)
    t, _, _ = oracle_force_eval_by_phase(small, tol=1e-8)
    res["batch_smallest"] = {"system": small.name, "n_occ": small.n_occ, "force_eval": t}
    errors = None
    if parity is not None:
        errors = {"workload": "12 wells, 36^3, N_occ 48, N_pdep 96 (oracle Davidson residual 1e-11)"}
        wo, Fo, xo, zo = ref
        for prec, name in ((0, "fp64"), (1, "mixed")):
            w, F, rx, rz = parity[prec]
            dF = np.abs(F - Fo)
            errors[name] = {
                "omega_ha": w, "omega_oracle_ha": wo, "abs_domega_ha": abs(w - wo),
                "max_abs_dF_ha_per_bohr": float(dF.max()),
                "abs_dF_per_component": [float(x) for x in dF.ravel()],
                "rel_l2_drho_x": float(np.linalg.norm(rx - xo) / np.linalg.norm(xo)),
                "rel_l2_drho_z": float(np.linalg.norm(rz - zo) / np.linalg.norm(zo)),
                "davidson_tol": PARITY_DAVIDSON_TOL[prec]}
    return res, errors


# ---------------------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch

    import bse_inputs
    import paper_2607_20728_gb300 as pkg

    torch.cuda.set_device(local_rank)
    pkg.load_library()
    spec = bse_inputs.diamond63()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)

    def barrier():
        if dist is not None:
            dist.barrier()

    sysm = pkg.BSESystem(spec, gs_tol=GS_TOL)
    sysm_keep_alive = [sysm]
    rng = np.random.default_rng(1234 + rank)
    dirn = rng.standard_normal(spec.pos.shape)
    dirn /= np.abs(dirn).max()

    def step(k):
        sysm.set_positions(spec.pos + 1e-4 * (k % 7) * dirn)
        w, _ = sysm.davidson(n_roots=1, tol=DAVIDSON_TOL, max_iter=500)
        sysm.zvector(0, tol=ZVEC_TOL, max_iter=3000)
        F = sysm.forces(0)
        return w, F

    for k in range(args.warmup):
        step(k)
    fp64_peak = measure_fp64_peak()
    st_warm = sysm.stats()
    applies_per_eval = st_warm["n_applies"] // max(1, args.warmup + 0) if args.warmup else None

    clocks = ClockSampler(local_rank)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sysm.profile(True)
    n0 = pkg.bse_launch_count()
    a0 = sysm.stats()["n_applies"]
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0.record(stream)
    for k in range(args.steps):
        w, F = step(args.warmup + k)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    n_launch = pkg.bse_launch_count() - n0
    applies = sysm.stats()["n_applies"] - a0
    k1d = sysm.kernel_timing(pkg.KERNEL_K1D)
    fft = sysm.kernel_timing(pkg.KERNEL_FFT)
    sfft = sysm.kernel_timing(pkg.KERNEL_SPHERE_FFT)
    sysm.profile(False)
    t_ms = ev0.elapsed_time(ev1)
    t_max = max_over_ranks(t_ms, dist)
    value = whole_job_rate(world, args.steps, t_max / 1e3)
    stats = sysm.stats()

    # Liouville apply throughput (tau resident), trial vectors per second
    apply_rate = {}
    for nb in (1, 2, 4, 8):
        X = torch.randn(nb, sysm.n_occ, sysm.n_pw, dtype=torch.float64, device="cuda")
        sysm.apply(X)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            sysm.apply(X)
        e1.record(stream)
        torch.cuda.synchronize()
        apply_rate[f"nb{nb}"] = 3 * nb / (e0.elapsed_time(e1) / 1e3)
    fftcmp = {"fp64": fft_comparator(pkg, sysm, sysm.n_occ)}

    # end to end through the C ABI from host buffers: setup (PDEP basis and atoms copied
    # host->device), Davidson, Z-vector, forces copied device->host, destroy
    e2e_steps = 1
    h2d = spec.pdep_coef.nbytes + spec.pdep_lambda.nbytes + spec.pos.nbytes + spec.Z.nbytes + spec.sigma.nbytes
    d2h = 8 * (3 * spec.n_atoms + 1)
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(e2e_steps):
        ctx = pkg.bse_setup(spec.lattice, spec.grid, spec.ecut, spec.pos, spec.Z, spec.sigma, spec.n_occ,
                            spec.pdep_coef, spec.pdep_lambda, gs_tol=GS_TOL)
        pkg.bse_davidson(ctx, 1, DAVIDSON_TOL, 500)
        pkg.bse_zvector(ctx, 0, ZVEC_TOL, 3000)
        Fe = pkg.bse_forces(ctx, 0, spec.n_atoms)
        pkg.load_library().bse_destroy(ctx)
    torch.cuda.synchronize()
    e2e_val = whole_job_rate(world, e2e_steps, max_over_ranks(time.perf_counter() - te, dist))

    peaks, src = measured_peaks()
    launches = max(1, k1d["launches"])
    per_launch_ms = k1d["ms"] / launches
    achieved = (k1d["alg_flops"] / launches) / (per_launch_ms / 1e3) / 1e12 if per_launch_ms > 0 else 0.0
    traffic = traffic_per_launch(kernel_source_hash("kernels.cu", "combine_tau_kernel"), k1d["alg_bytes"] / launches,
                                 stats.get("bytes_tau", 0.0))
    roofline = {"kernel": "combine_tau_kernel (fused V a + 2 v_H phi - sum tau a, Eq. 2)", "bound": "alu",
                "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                "traffic": traffic, "peak_source": "measured: cuBLAS DGEMM (torch.matmul float64 8192^3, best of 3, "
                                                   "CUDA events) on this GPU before the timed region",
                "peak_nominal": 1.25,
                "launches": k1d["launches"], "ms_per_launch": per_launch_ms,
                "share_of_step": k1d["ms"] / t_ms if t_ms > 0 else None,
                "achieved_gbs": (k1d["alg_bytes"] / launches) / (per_launch_ms / 1e3) / 1e9 if per_launch_ms else 0.0,
                "hbm_peak_gbs": peaks.get("hbm_gbs"), "hbm_peak_source": src,
                "fft_ms_per_launch": fft["ms"] / max(1, fft["launches"]), "fft_launches": fft["launches"],
                "fft_share_of_step": fft["ms"] / t_ms if t_ms > 0 else None,
                "sphere_fft_ms_per_launch": sfft["ms"] / max(1, sfft["launches"]),
                "sphere_fft_launches": sfft["launches"],
                "sphere_fft_share_of_step": sfft["ms"] / t_ms if t_ms > 0 else None,
                "sphere_fft_tflops": (sfft["alg_flops"] / (sfft["ms"] / 1e3) / 1e12) if sfft["ms"] > 0 else None}

    # the mixed-precision form on the same workload and the same last geometry
    mixed = None
    if not args.fp64_only:
        del sysm_keep_alive[:]
        sysm.close()
        torch.cuda.synchronize()
        msys = pkg.BSESystem(spec, gs_tol=GS_TOL, precision=1)

        def mstep(k):
            msys.set_positions(spec.pos + 1e-4 * (k % 7) * dirn)
            wm, _ = msys.davidson(n_roots=1, tol=MIXED_DAVIDSON_TOL, max_iter=500)
            msys.zvector(0, tol=ZVEC_TOL, max_iter=3000)
            return wm, msys.forces(0)

        mstep(args.warmup + args.steps - 1)   # warm-up at the last FP64 geometry
        msys.profile(True)
        m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        m0.record(stream)
        for k in range(args.steps):
            wm, Fm = mstep(args.warmup + k)
        m1.record(stream)
        torch.cuda.synchronize()
        barrier()
        mk1d = msys.kernel_timing(pkg.KERNEL_K1D)
        msys.profile(False)
        tm_max = max_over_ranks(m0.elapsed_time(m1), dist)
        mst = msys.stats()
        mrate = {}
        for nb in (1, 2, 4, 8):
            X = torch.randn(nb, msys.n_occ, msys.n_pw, dtype=torch.float64, device="cuda")
            msys.apply(X)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                msys.apply(X)
            e1.record(stream)
            torch.cuda.synchronize()
            mrate[f"nb{nb}"] = 3 * nb / (e0.elapsed_time(e1) / 1e3)
        fftcmp["fp32"] = fft_comparator(pkg, msys, msys.n_occ)
        ml = max(1, mk1d["launches"])
        mms = mk1d["ms"] / ml
        mixed = {
            "value": whole_job_rate(world, args.steps, tm_max / 1e3), "unit": UNIT, "ms_per_step": tm_max / args.steps,
            "dtype": "fp32 grids/FFT/tau + FP64 subspace, refinement, forces",
            "applies_per_s": mrate,
            "omega_ha": float(wm[0]),
            "abs_domega_vs_fp64_ha": abs(float(wm[0]) - float(w[0])),
            "max_abs_dF_vs_fp64_ha_per_bohr": float(np.abs(Fm - F).max()),
            "davidson_tol": MIXED_DAVIDSON_TOL,
            "per_step": {"davidson_iterations": mst["davidson_iterations"], "zvector_iterations": mst["zvector_iterations"],
                         "ms_ground_state": mst["ms_ground_state"], "ms_tau": mst["ms_tau"],
                         "ms_davidson": mst["ms_davidson"], "ms_uvec": mst["ms_uvec"], "ms_zvector": mst["ms_zvector"],
                         "ms_forces": mst["ms_forces"]},
            "k1d_roofline": {"bound": "hbm", "achieved": (mk1d["alg_bytes"] / ml) / (mms / 1e3) / 1e9 if mms else 0.0,
                             "traffic": traffic_per_launch(kernel_source_hash("k1d_tma.cu", "k1d_tma_kernel"),
                                                           mk1d["alg_bytes"] / ml, mst.get("bytes_tau", 0.0)),
                             "peak": peaks.get("hbm_gbs"), "unit": "GB/s",
                             "frac": ((mk1d["alg_bytes"] / ml) / (mms / 1e3) / 1e9) / peaks.get("hbm_gbs") if mms else 0.0,
                             "ms_per_launch": mms, "launches": mk1d["launches"]},
        }
        msys.close()

    # relaxation-style sequence: each step seeded with the previous geometry's states and roots
    warm = None
    if world == 1 and not args.no_warm:
        warm = run_warm(pkg, spec, dirn, args)

    # the Hartree-SCF ground-state model of the same cell
    hartree = None
    if world == 1 and not args.no_hartree:
        hartree = run_hartree(pkg, bse_inputs, args)

    # the BSE beyond the TDA (coupling block) on the same cell's Hartree model
    full_bse = None
    if world == 1 and not args.no_full_bse:
        full_bse = run_full_bse(pkg, bse_inputs, args)

    # an excited-state relaxation driven by the forces
    relax = None
    if world == 1 and not args.no_relax:
        relax = run_relax(pkg, bse_inputs, args)

    # Wannier pair pruning of K1d (an approximation, with its error against the exact path)
    wannier = None
    if world == 1 and not args.no_wannier:
        wannier = run_wannier(pkg, bse_inputs, args)

    # the batched form: 48 independent systems of uneven size, set up and solved concurrently
    batched = None
    if world == 1 and not args.no_batched:
        batched = run_batched(pkg, bse_inputs)

    # GPU force evaluations of the N_occ = 48 parity cell (compared with the oracle below)
    parity = None
    if world == 1 and not args.no_parity:
        parity = parity_gpu(pkg, bse_inputs.mid48())

    # where the GPU waits within one force evaluation (torch.profiler kernel records)
    busy = None
    if world == 1 and not args.no_busy:
        try:
            busy = measure_gpu_busy()
        except Exception as e:  # the profiler is a measurement aid: report, do not fail the line
            busy = {"unavailable": f"{type(e).__name__}: {e}"[:200]}

    if rank != 0:
        return
    cpu = None
    errors = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(spec, applies_per_eval=max(1, applies // max(1, args.steps)), rows=4)
        cpu["oracle_plan"], errors = oracle_plan(parity)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(spec, world),
        "applies_per_s": apply_rate,
        "omega_ha": float(w[0]),
        "per_step": {"applies": applies / args.steps, "davidson_iterations": stats["davidson_iterations"],
                     "zvector_iterations": stats["zvector_iterations"], "gs_iterations": stats["gs_iterations"],
                     "ms_ground_state": stats["ms_ground_state"], "ms_tau": stats["ms_tau"],
                     "ms_davidson": stats["ms_davidson"], "ms_uvec": stats["ms_uvec"],
                     "ms_zvector": stats["ms_zvector"], "ms_forces": stats["ms_forces"]},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(n_launch),
        "roofline": roofline,
        "fft_comparator": fftcmp,
        "parity_vs_oracle": errors,
        "clocks": clk,
        "cpu_baseline": cpu,
        "mixed": mixed,
        "batched": batched,
        "warm_start": warm,
        "hartree_scf": hartree,
        "full_bse": full_bse,
        "relaxation": relax,
        "wannier_pruning": wannier,
        "gpu_busy": busy,
    }
    print(json.dumps(line), flush=True)


def run_warm(pkg, spec, dirn, args):
    """Force evaluations along the same geometry sequence with BSE_FLAG_WARM_START (the previous
    geometry's ground-state block and excitation vectors as starting vectors): the rate of a
    relaxation or dynamics step, FP64 and mixed."""
    import torch
    out = {"note": "steps of 1e-4..6e-4 bohr along a fixed direction, each seeded with the previous "
                   "geometry's states and roots; same tolerances as the cold evaluations"}
    for prec, name, dtol in ((0, "fp64", DAVIDSON_TOL), (1, "mixed", MIXED_DAVIDSON_TOL)):
        s = pkg.BSESystem(spec, gs_tol=GS_TOL, precision=prec, flags=pkg.FLAG_WARM_START)

        def wstep(k):
            s.set_positions(spec.pos + 1e-4 * (k % 7) * dirn)
            w, _ = s.davidson(n_roots=1, tol=dtol, max_iter=500)
            s.zvector(0, tol=ZVEC_TOL, max_iter=3000)
            return s.forces(0)

        s.davidson(n_roots=1, tol=dtol, max_iter=500)
        wstep(args.warmup)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(args.steps):
            wstep(args.warmup + 1 + k)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        st = s.stats()
        out[name] = {"value": args.steps / dt, "unit": UNIT, "ms_per_step": dt / args.steps * 1e3,
                     "gs_iterations": st["gs_iterations"], "davidson_iterations": st["davidson_iterations"],
                     "ms_ground_state": st["ms_ground_state"], "ms_davidson": st["ms_davidson"]}
        s.close()
        torch.cuda.synchronize()
    return out


def run_hartree(pkg, bse_inputs, args):
    """Force evaluations of the Hartree-SCF model of the 63-atom cell (one doubly occupied orbital
    and a Gaussian ionic charge 2 per site, N_occ = 63): each step moves the atoms and runs the SCF
    ground state from scratch, tau, Davidson, U, the coupled Z-vector and the forces; FP64 and
    mixed, timed with CUDA events on the library's stream."""
    import torch
    spec = bse_inputs.hartree_model(bse_inputs.diamond63())
    rng = np.random.default_rng(4321)
    dirn = rng.standard_normal(spec.pos.shape)
    dirn /= np.abs(dirn).max()
    out = {"workload": "diamond-vacancy 63 wells, 72^3, 30 Ry, N_occ 63, N_pdep 256, Hartree-SCF ground state "
                       "(q_ion = 2 per site), cold SCF at every step"}
    res = {}
    for prec, name, dtol in ((0, "fp64", DAVIDSON_TOL), (1, "mixed", MIXED_DAVIDSON_TOL)):
        s = pkg.BSESystem(spec, gs_tol=GS_TOL, precision=prec)
        stream = torch.cuda.current_stream()

        def hstep(k):
            s.set_positions(spec.pos + 1e-4 * (k % 7) * dirn)
            w, _ = s.davidson(n_roots=1, tol=dtol, max_iter=500)
            s.zvector(0, tol=ZVEC_TOL, max_iter=3000)
            return w, s.forces(0)

        hstep(1)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k in range(args.steps):
            w, F = hstep(2 + k)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        st = s.stats()
        res[name] = (w, F)
        out[name] = {"value": 1e3 / ms, "unit": UNIT, "ms_per_step": ms, "omega_ha": float(w[0]),
                     "scf_iterations": st["scf_iterations"], "scf_residual": st["scf_residual"],
                     "gs_iterations": st["gs_iterations"], "homo_lumo_gap_ha": st["homo_lumo_gap"],
                     "ms_ground_state": st["ms_ground_state"], "ms_tau": st["ms_tau"],
                     "ms_davidson": st["ms_davidson"], "ms_uvec": st["ms_uvec"], "ms_zvector": st["ms_zvector"],
                     "ms_forces": st["ms_forces"], "davidson_iterations": st["davidson_iterations"],
                     "zvector_iterations": st["zvector_iterations"]}
        s.close()
        torch.cuda.synchronize()
    out["abs_domega_mixed_vs_fp64_ha"] = abs(float(res["mixed"][0][0]) - float(res["fp64"][0][0]))
    out["max_abs_dF_mixed_vs_fp64_ha_per_bohr"] = float(np.abs(res["mixed"][1] - res["fp64"][1]).max())
    return out


def run_full_bse(pkg, bse_inputs, args):
    """The BSE beyond the TDA on the Hartree-SCF model of the 63-atom cell (whose TDA root is
    positive, so the full BSE has a real spectrum; the non-SCF cell's is not): throughput of the
    coupling block B (N_occ^2 = 3969 pair densities through W per vector) and the full-BSE
    Davidson for the lowest root, FP64 and mixed, timed with CUDA events."""
    import torch
    spec = bse_inputs.hartree_model(bse_inputs.diamond63())
    out = {"workload": "diamond-vacancy 63 wells, Hartree-SCF ground state, N_occ 63, N_pdep 256, lowest root"}
    for prec, name, dtol in ((0, "fp64", DAVIDSON_TOL), (1, "mixed", MIXED_DAVIDSON_TOL)):
        s = pkg.BSESystem(spec, gs_tol=GS_TOL, precision=prec)
        stream = torch.cuda.current_stream()
        X = torch.randn(1, s.n_occ, s.n_pw, dtype=torch.float64, device="cuda")
        s.apply(X, op=3)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            s.apply(X, op=3)
        e1.record(stream)
        torch.cuda.synchronize()
        b_rate = 3 / (e0.elapsed_time(e1) / 1e3)
        wt, _ = s.davidson(n_roots=1, tol=dtol, max_iter=500)
        torch.cuda.synchronize()
        e0.record(stream)
        wf, _, _ = s.davidson_full(n_roots=1, tol=dtol, max_iter=300)
        e1.record(stream)
        torch.cuda.synchronize()
        st = s.stats()
        out[name] = {"b_applies_per_s": b_rate, "full_bse_ms": e0.elapsed_time(e1),
                     "full_bse_iterations": st["davidson_iterations"], "omega_full_ha": float(wf[0]),
                     "omega_tda_ha": float(wt[0]), "davidson_tol": dtol}
        s.close()
        torch.cuda.synchronize()
    return out


def run_relax(pkg, bse_inputs, args):
    """Excited-state relaxation of the Hartree-SCF model of the 63-atom cell in mixed precision on
    E = E_gs + omega, E_gs a harmonic well 1/2 k |R - R0|^2 (k = 0.2 Ha/bohr^2) standing in for the
    ground-state surface, to the paper's threshold max |F| < 0.03 eV/A: with the inexact
    (force-proportional) tolerances and with the tight ones throughout."""
    import torch
    spec = bse_inputs.hartree_model(bse_inputs.diamond63())
    k = 0.2
    fmax = 0.03 / 51.42208619083232          # eV/A -> Ha/bohr

    def gs(pos):
        d = pos - spec.pos
        return 0.5 * k * float(np.sum(d * d)), -k * d

    out = {"workload": "diamond-vacancy 63 wells, Hartree-SCF, mixed precision, harmonic ground-state well "
                       "k = 0.2 Ha/bohr^2, FIRE to max |F| < 0.03 eV/A", "fmax_ha_per_bohr": fmax}
    for inexact in (True, False):
        s = pkg.BSESystem(spec, gs_tol=GS_TOL, precision=1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pos, E, w, evals = s.relax(gs, fmax=fmax, max_steps=300, inexact=inexact,
                                   davidson_tol=MIXED_DAVIDSON_TOL, zvector_tol=ZVEC_TOL)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out["inexact" if inexact else "exact"] = {
            "seconds": dt, "force_evaluations": evals, "s_per_evaluation": dt / max(1, evals),
            "omega_ha": w, "energy_ha": E, "max_displacement_bohr": float(np.abs(pos - spec.pos).max())}
        s.close()
        torch.cuda.synchronize()
    return out


def run_wannier(pkg, bse_inputs, args):
    """Wannier pair pruning of K1d on the Hartree-SCF model of the 63-atom cell (localised
    orbitals): for each cutoff the kept pairs, the cached tau bytes, the force evaluation's time
    and its omega / force error against the unpruned (canonical) path, FP64 and mixed."""
    import torch
    spec = bse_inputs.hartree_model(bse_inputs.diamond63())
    out = {"workload": "diamond-vacancy 63 wells, Hartree-SCF, N_occ 63 (2016 pairs), force evaluation"}
    for prec, name, dtol in ((0, "fp64", DAVIDSON_TOL), (1, "mixed", MIXED_DAVIDSON_TOL)):
        rows = []
        ref = None
        for cutoff in (None, 9.0, 6.0, 4.0):
            s = pkg.BSESystem(spec, gs_tol=GS_TOL, precision=prec, pair_cutoff=cutoff)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.set_positions(spec.pos)
            w, _ = s.davidson(n_roots=1, tol=dtol, max_iter=500)
            s.zvector(0, tol=ZVEC_TOL, max_iter=3000)
            F = s.forces(0)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            st = s.stats()
            row = {"cutoff_bohr": cutoff, "pairs": st["wannier_pairs"] if cutoff else spec.n_occ * (spec.n_occ + 1) // 2,
                   "tau_bytes": st["bytes_tau"], "force_eval_s": dt, "ms_davidson": st["ms_davidson"],
                   "omega_ha": float(w[0])}
            if ref is None:
                ref = (float(w[0]), F)
            else:
                row["abs_domega_ha"] = abs(float(w[0]) - ref[0])
                row["max_abs_dF_ha_per_bohr"] = float(np.abs(F - ref[1]).max())
            rows.append(row)
            s.close()
            torch.cuda.synchronize()
        out[name] = rows
    return out


def run_batched(pkg, bse_inputs, workers=8):
    """Setup (ground state, tau) and solve (Davidson, Z-vector, forces) of the 48-system batch in
    mixed precision, timed end to end on the host through bse_setup_batch / bse_solve_batch."""
    import torch
    specs = bse_inputs.batch48()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = pkg.BSEBatch(specs, n_workers=workers, precision=1, gs_tol=GS_TOL)
    t1 = time.perf_counter()
    w, F, st = b.solve(davidson_tol=MIXED_DAVIDSON_TOL, zvector_tol=ZVEC_TOL)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    ok = sum(1 for i in range(len(specs)) if b.status(i) == 0)
    setup_ms, solve_ms = b.timing()
    choices = {}
    graphed = 0
    for i in range(len(specs)):
        st = b.system_stats(i)
        if st is None:
            continue
        key = (f"fft={'full' if st['tuned_full_grid_fft'] else 'sphere'} k1d_nb={st['tuned_k1d_nb']} "
               f"xy_threads={st['tuned_xy_threads'] or 512} gemm_split={st['tuned_gemm_split_pct']}%")
        choices[key] = choices.get(key, 0) + 1
        graphed += st["zvector_graphed"]
    b.close()
    return {"workload": "48 seeded Gaussian-well models: 8-64 atoms, 36^3-64^3 grids, N_occ 16-128, "
                        "N_pdep 64-256, one root each, mixed precision",
            "systems": len(specs), "ok": ok, "workers": workers,
            "setup_device_ms": setup_ms, "solve_device_ms": solve_ms,
            "value": ok / ((setup_ms + solve_ms) / 1e3), "unit": "force_evals/s",
            "timing": "CUDA events on the worker streams (first start to last end), setup and solve separately",
            "host_setup_s": t1 - t0, "host_solve_s": t2 - t1,
            "autotuned_choices": choices, "zvector_solves_as_one_graph": graphed}


def run_hbn(args):
    """Config 4, the 8 x 8 honeycomb slab (96 x 96 x 160 grid, 20 bohr vacuum), on its own line:
      hbn128          non-SCF model, N_occ 256, N_pdep 512, 4 roots, mixed precision (its FP64 tau,
                      388 GB, does not fit one GPU): force evaluation time by phase, tau bytes;
      hbn128-hartree  the Hartree-SCF variant (N_occ 128): FP64 and mixed force evaluations, their
                      difference, the Wannier-pruned FP64 evaluation at a 9 bohr cutoff, and the
                      FP64 analytic force on one dimer atom against Richardson finite differences
                      (h = 2e-3, 1e-3 bohr) of the library's own omega(R)."""
    import torch

    import bse_inputs
    import paper_2607_20728_gb300 as pkg
    pkg.load_library()
    base = bse_inputs.hbn128()
    hartree = args.config == "hbn128-hartree"
    spec = bse_inputs.hartree_model(base) if hartree else base
    stream = torch.cuda.current_stream()
    out = {"config": {"workload": spec.name, "grid": list(spec.grid), "n_atoms": spec.n_atoms,
                      "n_occ": spec.n_occ, "n_pdep": spec.n_pdep, "n_roots": spec.n_roots, "n_pw": spec.n_pw},
           "metric": "force evaluations/s", "data": "synthetic"}

    def evaluate(s, dtol, pos=None):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        s.set_positions(spec.pos if pos is None else pos)
        w, _ = s.davidson(n_roots=spec.n_roots, tol=dtol, max_iter=600)
        s.zvector(0, tol=ZVEC_TOL, max_iter=3000)
        F = s.forces(0)
        e1.record(stream)
        torch.cuda.synchronize()
        st = s.stats()
        return w, F, {"seconds": e0.elapsed_time(e1) / 1e3, "omega_ha": [float(x) for x in w],
                      "tau_bytes": st["bytes_tau"], "homo_lumo_gap_ha": st["homo_lumo_gap"],
                      **{k: st[k] for k in ("ms_ground_state", "ms_tau", "ms_davidson", "ms_uvec", "ms_zvector",
                                            "ms_forces", "davidson_iterations", "zvector_iterations",
                                            "gs_iterations", "scf_iterations")}}

    precs = ((0, "fp64", DAVIDSON_TOL), (1, "mixed", MIXED_DAVIDSON_TOL)) if hartree else \
        ((1, "mixed", MIXED_DAVIDSON_TOL),)
    res = {}
    for prec, name, dtol in precs:
        s = pkg.BSESystem(spec, gs_tol=GS_TOL, precision=prec)
        w, F, rec = evaluate(s, dtol)
        res[name] = (w, F)
        out[name] = rec
        if hartree and prec == 0:
            # the dimer atom's out-of-plane force against Richardson finite differences of omega(R)
            atom, alpha = int(base.extra["dimer"][0]), 2

            def omega_at(dx):
                p = spec.pos.copy()
                p[atom, alpha] += dx
                s.set_positions(p)
                ww, _ = s.davidson(n_roots=spec.n_roots, tol=1e-10, max_iter=600)
                return float(ww[0])
            d = {}
            for h in (2e-3, 1e-3):
                d[h] = (omega_at(h) - omega_at(-h)) / (2 * h)
            fd = (4 * d[1e-3] - d[2e-3]) / 3
            out["fd_check"] = {"atom": atom, "component": alpha, "analytic_F": float(F[atom, alpha]),
                               "richardson_F": -fd, "abs_diff_ha_per_bohr": abs(float(F[atom, alpha]) + fd),
                               "steps_bohr": [2e-3, 1e-3]}
        s.close()
        torch.cuda.synchronize()
        out[name]["value"] = 1.0 / out[name]["seconds"]
    if hartree:
        out["abs_domega_mixed_vs_fp64_ha"] = float(np.abs(res["mixed"][0] - res["fp64"][0]).max())
        out["max_abs_dF_mixed_vs_fp64_ha_per_bohr"] = float(np.abs(res["mixed"][1] - res["fp64"][1]).max())
        s = pkg.BSESystem(spec, gs_tol=GS_TOL, precision=0, pair_cutoff=9.0)
        w, F, rec = evaluate(s, DAVIDSON_TOL)
        st = s.stats()
        s.close()
        rec.update({"cutoff_bohr": 9.0, "pairs": st["wannier_pairs"],
                    "abs_domega_ha": float(abs(w[0] - res["fp64"][0][0])),
                    "max_abs_dF_ha_per_bohr": float(np.abs(F - res["fp64"][1]).max())})
        out["wannier_fp64"] = rec
    else:
        out["note"] = ("FP64 tau (388 GB) does not fit one GPU; the non-SCF slab's HOMO-LUMO gap is 2.4e-5 Ha, "
                       "so this line is a throughput measurement, validated only through the Hartree variant")
    print(json.dumps(out), flush=True)


def profile_run(args):
    import dataclasses

    import torch

    import bse_inputs
    import paper_2607_20728_gb300 as pkg
    spec = bse_inputs.diamond63()
    if args.profile_small:
        no = args.profile_nocc
        spec = dataclasses.replace(spec, n_occ=no, n_pdep=2 * no, pdep_coef=spec.pdep_coef[:2 * no],
                                   pdep_lambda=spec.pdep_lambda[:2 * no])
    sysm = pkg.BSESystem(spec, gs_tol=GS_TOL, precision=args.precision)
    torch.cuda.synchronize()
    n_setup = pkg.bse_launch_count()
    if args.profile_small:
        X = torch.randn(4, sysm.n_occ, sysm.n_pw, dtype=torch.float64, device="cuda")
        for nb in (1, 2, 3, 4):
            sysm.apply(X[:nb].contiguous())
    else:
        sysm.set_positions(spec.pos)
        sysm.davidson(n_roots=1, tol=DAVIDSON_TOL if args.precision == 0 else MIXED_DAVIDSON_TOL, max_iter=500)
        sysm.zvector(0, tol=ZVEC_TOL, max_iter=3000)
        sysm.forces(0)
    torch.cuda.synchronize()
    if not args.profile_small:
        st = sysm.stats()
        st["setup_launches"] = n_setup
        st["step_launches"] = pkg.bse_launch_count() - n_setup
        print(json.dumps(st), flush=True)
    sysm.close()


def gpu_busy_run(args):
    print(json.dumps(measure_gpu_busy()), flush=True)


def measure_gpu_busy():
    """Where the GPU waits in one force evaluation of the 63-atom cell, per phase and precision:
    the union of the kernel (and copy) intervals that torch.profiler records, against the wall
    time of each phase.  Kernels inside the Z-vector's conditional graph node may not be
    recorded, so that phase can read low by the loop's duration; the total is also given with
    that phase counted as busy."""
    import torch
    from torch.profiler import profile, ProfilerActivity, record_function
    import bse_inputs
    import paper_2607_20728_gb300 as pkg
    pkg.load_library()
    spec = bse_inputs.diamond63()
    rng = np.random.default_rng(1234)
    dirn = rng.standard_normal(spec.pos.shape)
    dirn /= np.abs(dirn).max()
    out = {"metric": "GPU busy fraction per phase of one cold force evaluation (torch.profiler kernel records)",
           "workload": "diamond-vacancy-63atom-72^3"}
    phases = ("set_positions", "davidson", "zvector", "forces")
    for prec, tol in ((0, DAVIDSON_TOL), (1, MIXED_DAVIDSON_TOL)):
        s = pkg.BSESystem(spec, gs_tol=GS_TOL, precision=prec)
        for k in range(2):
            s.set_positions(spec.pos + 1e-4 * k * dirn)
            s.davidson(1, tol=tol, max_iter=500)
            s.zvector(0, tol=ZVEC_TOL, max_iter=3000)
            s.forces(0)
        torch.cuda.synchronize()
        with profile(activities=[ProfilerActivity.CPU, ProfilerActivity.CUDA]):
            s.forces(0)  # the profiler's first session warms up its kernel tracing
            torch.cuda.synchronize()
        with profile(activities=[ProfilerActivity.CPU, ProfilerActivity.CUDA]) as p:
            calls = {"set_positions": lambda: s.set_positions(spec.pos + 3e-4 * dirn),
                     "davidson": lambda: s.davidson(1, tol=tol, max_iter=500),
                     "zvector": lambda: s.zvector(0, tol=ZVEC_TOL, max_iter=3000),
                     "forces": lambda: s.forces(0)}
            for ph in phases:
                with record_function("phase_" + ph):
                    calls[ph]()
                    torch.cuda.synchronize()
        st = s.stats()
        s.close()
        ev = p.events()
        dev = torch.autograd.DeviceType.CUDA
        kern = sorted((e.time_range.start, e.time_range.end) for e in ev
                      if e.device_type == dev and not e.name.startswith("phase_"))
        res = {}
        for ph in phases:
            rng_ = [(e.time_range.start, e.time_range.end) for e in ev
                    if e.name == "phase_" + ph and e.device_type == torch.autograd.DeviceType.CPU]
            a, b = rng_[0]
            busy, cur = 0.0, None
            for x, y in kern:
                if y <= a or x >= b:
                    continue
                x, y = max(x, a), min(y, b)
                if cur is None or x > cur[1]:
                    if cur is not None:
                        busy += cur[1] - cur[0]
                    cur = [x, y]
                else:
                    cur[1] = max(cur[1], y)
            if cur is not None:
                busy += cur[1] - cur[0]
            res[ph] = {"wall_ms": round((b - a) / 1e3, 2), "busy_ms": round(busy / 1e3, 2),
                       "busy_frac": round(busy / max(1.0, b - a), 3)}
        wall = sum(v["wall_ms"] for v in res.values())
        busy = sum(v["busy_ms"] for v in res.values())
        out["fp64" if prec == 0 else "mixed"] = {
            "phases": res, "busy_frac": round(busy / wall, 3),
            "busy_frac_zvector_loop_counted": round((busy + res["zvector"]["wall_ms"] - res["zvector"]["busy_ms"]) / wall, 3),
            "ms_host_eig": round(st["ms_host_eig"], 1), "gs_iterations": st["gs_iterations"],
            "davidson_iterations": st["davidson_iterations"]}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-only", action="store_true", help="skip the mixed-precision measurement")
    ap.add_argument("--profile-once", action="store_true",
                    help="setup plus one force evaluation of the timed workload, no output (ncu launch list)")
    ap.add_argument("--profile-small", action="store_true",
                    help="63-atom cell with N_occ = --profile-nocc, N_pdep = 2 N_occ: setup and 4 applies (ncu capture)")
    ap.add_argument("--no-batched", action="store_true", help="skip the 48-system batched line")
    ap.add_argument("--no-warm", action="store_true", help="skip the warm-started (relaxation step) line")
    ap.add_argument("--no-hartree", action="store_true", help="skip the Hartree-SCF model line")
    ap.add_argument("--no-full-bse", action="store_true", help="skip the beyond-TDA (coupling block) line")
    ap.add_argument("--no-relax", action="store_true", help="skip the excited-state relaxation line")
    ap.add_argument("--no-wannier", action="store_true", help="skip the Wannier pair-pruning line")
    ap.add_argument("--no-parity", action="store_true",
                    help="skip the GPU-vs-oracle errors on the N_occ = 48 parity cell")
    ap.add_argument("--profile-nocc", type=int, default=32,
                    help="N_occ of the --profile-small case (N_pdep = 2 N_occ)")
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1],
                    help="precision of the --profile-* runs: 0 FP64, 1 mixed")
    ap.add_argument("--no-busy", action="store_true", help="skip the per-phase GPU busy fractions")
    ap.add_argument("--gpu-busy", action="store_true",
                    help="per-phase GPU busy fractions of one force evaluation (torch.profiler), FP64 and mixed")
    ap.add_argument("--config", choices=["diamond63", "hbn128", "hbn128-hartree"], default="diamond63",
                    help="diamond63: the benchmark line; hbn128 / hbn128-hartree: the 2D slab on its own line")
    args = ap.parse_args()
    if args.config != "diamond63":
        run_hbn(args)
        return
    if args.profile_once or args.profile_small:
        profile_run(args)
        return
    if args.gpu_busy:
        gpu_busy_run(args)
        return
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus if args.gpus else 1)))
    if "WORLD_SIZE" not in os.environ:
        world = 1
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
