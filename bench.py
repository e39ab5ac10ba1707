#!/usr/bin/env python3
"""Walker-step throughput of the k-point phaseless AFQMC hot path on GB300.

One step = one hybrid propagation of every walker (Green's function, force
bias, vHS, 6-term Taylor exp(V) with both one-body halves, weight update, a
re-orthonormalisation every 5th step) followed by the local energy (E1 +
Coulomb + exchange) of every walker, for the 3x3x3 diamond-sized synthetic
system (M = 26 orbitals per k, 4 occupied per k per spin, 208 Cholesky vectors
per Q, 64 walkers per GPU, walkers seeded near the trial).  The K timed steps
are taken in five windows that each restart from the seeded walkers; the
headline is the median window.  The line is marked invalid (and the exit code
is 1) if the library's sticky device flags report a fault, a bounded wait that
gave up or a vHS entry out of range, or if no walker is alive afterwards.
Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
  python bench.py --impl reference ...   # the FP64 CPU oracle on a bounded sample

Multi-GPU runs (torchrun, one process per GPU) are independent walker
replicas: no collective on the data path, only the timing max over ranks.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402

METRIC = "walker-steps/s (propagate+E_L) mixed vs FP64 at stated error; % roofline"
UNIT = "walker-steps/s"
QR_PERIOD = 5
PAPER_BLOCK_STEPS = 20      # a block: 20 propagation steps, one energy, one orthogonalisation (Sec. 3.1)
BLOCK_SEED = 0x2003094680000001
WINDOWS = 5                 # timed windows of `steps` steps each; the headline is their median
DRIFT_STEPS = 10            # trajectory length of the drift report (QR every QR_PERIOD)
FP64_STEPS = 3              # timed steps of the FP64 comparison arm
STATUS_NAMES = {0: "ok", 1: "invalid", 2: "oom", 3: "cuda", 4: "singular", 5: "timeout", 6: "vhs-range"}
# the task's bars for the mixed path (per call on the same inputs)
BARS_MIXED = {"E_L_ha_per_cell": 1e-5, "force_bias_rel": 1e-6, "phi_rel": 1e-6, "weight_rel": 1e-5,
              "logdet_abs": 1e-5}
WORKLOADS = {
    "diamond-3x3x3": gen.DIAMOND_3x3x3,
    "small-2x2x2": gen.SMALL_2x2x2,
    "diamond-4x4x4": gen.DIAMOND_4x4x4,
}
LARGE_NK = 64               # from this k-point count on: sampled oracle legs, no FP64 arm
EX_SAMPLE_Q = 2             # momentum transfers in the sampled oracle exchange of a large workload


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------
# algorithmic work (complex multiply-add = 8 real flops)
# ---------------------------------------------------------------------------
def canonical_triples(spec) -> int:
    """Number of (Q, k, k') terms kept after pairing (Q, k, k') with (-Q, k'-Q, k)."""
    g = np.array(spec.grid)
    kp = gen.kpoints(spec.grid)
    lin = lambda v: int((v[0] * g[1] + v[1]) * g[2] + v[2])
    minus = [lin((-kp[q]) % g) for q in range(spec.nk)]
    t = 0
    for Q in range(spec.nk):
        for k in range(spec.nk):
            for kx in range(spec.nk):
                if Q < minus[Q] or (Q == minus[Q] and k <= kx):
                    t += 1
    return t


def exchange_flops(spec) -> float:
    """Direct exchange (Sec. 3.2 steps 2a-2c) for all walkers and both spins: every
    T^Q_g = LH^{Qg} Gh^T element once (N x N per (Q, g), M complex MACs each) plus the
    pairing products.  This is what the FP64 kernel executes."""
    nk, G, N, M = spec.nk, spec.nchol, spec.N, spec.M
    return spec.nwalkers * 2 * 8.0 * nk * G * N * N * (M + 0.5)


def exchange_precontracted_flops(spec) -> float:
    """Exchange through the precontracted tensor: one (nM x nM) x WS complex GEMM per
    canonical triple, 8 real flops per complex MAC."""
    nM = spec.nocc * spec.M
    return 8.0 * canonical_triples(spec) * nM * nM * 2 * spec.nwalkers


def adjoint_exchange_flops(spec) -> float:
    """Exchange adjoint through the precontracted tensor: for every block and every Q one
    (nM x nM) x WS complex GEMM, i.e. all Nk^3 triples, 8 real flops per complex MAC."""
    nM = spec.nocc * spec.M
    return 8.0 * spec.nk ** 3 * nM * nM * 2 * spec.nwalkers


def taylor_flops(spec, order=6) -> float:
    return 8.0 * order * spec.nwalkers * spec.NM * spec.NM * 2 * spec.N


def taylor_term_flops(spec) -> float:
    """One Taylor term, V u for every walker: (2N x NM) x (NM x NM) complex, 8 flops per MAC."""
    return 8.0 * spec.nwalkers * spec.NM * spec.NM * 2 * spec.N


def vhs_bytes(spec) -> float:
    """Cholesky tensor read once and V written once, both as four fp16 planes (8 bytes per
    complex element), which is the form the kernel reads and writes."""
    return 8.0 * spec.nk * spec.nk * spec.nchol * spec.M * spec.M + 8.0 * spec.nwalkers * spec.NM * spec.NM


FF_OPS_PER_CMAC = 48.0   # FP32 instructions per complex double-float multiply-add (unnormalised accumulate)


def step_roofline_model(spec, qr_period: int, tensor_tfs: float, hbm_gbs: float, sm_mhz: float, sms: int = 152):
    """Ideal time of each stage of one mixed-path step, each kernel at its own bound
    (algorithmic flops at the tensor peak, algorithmic bytes at the HBM copy rate, double-float
    operations at the FP32 issue rate of sms x 128 lanes x clock), summed over the stage's
    kernels; QR amortised over qr_period steps.  Returns {stage: (bound, ideal_ms)}."""
    W, nk, M, n, G = spec.nwalkers, spec.nk, spec.M, spec.nocc, spec.nchol
    WS, NM, N, nM = 2 * W, spec.NM, spec.N, spec.nocc * spec.M
    Mp = -(-M // 32) * 32
    nMp = n * Mp
    T = tensor_tfs * 1e12
    B = hbm_gbs * 1e9
    F = sms * 128 * sm_mhz * 1e6
    ms = lambda x: 1e3 * x
    out = {}
    # Green's function of the propagated walkers: double-float overlap and projection, the
    # double-float inverse, the tensor-core GEMM S^-T phi_perp^T (+ its operands and outputs)
    ov = max(2.0 * WS * nk * M * n * N * FF_OPS_PER_CMAC / F, 16.0 * WS * NM * N / B)
    gj = WS * float(N) ** 3 * FF_OPS_PER_CMAC / F
    gg = max(8.0 * WS * N * NM * N / T, (8.0 * WS * NM * N + 16.0 * nk * nk * WS * nMp) / B)
    out["green"] = ("ff + tensor", ms(ov + gj + gg))
    # Cholesky trace X of the new Green's function (spin-summed rows) and the force bias
    out["force_bias"] = ("hbm", ms(max(8.0 * W * nk * nk * G * nM / T, 8.0 * nk * nk * G * nMp / B)))
    out["vhs"] = ("hbm", ms(max(8.0 * W * nk * nk * G * M * M / T, vhs_bytes(spec) / B)))
    out["taylor"] = ("tensor", ms(6 * taylor_term_flops(spec) / T))
    # the one-body halves: phi read twice and written once in FP64, the fp32 iterate and the
    # corrections written and read
    out["onebody"] = ("hbm", ms(80.0 * WS * NM * N / B))
    # exchange: the precontracted tensor streams once per step
    t = canonical_triples(spec)
    out["exchange"] = ("hbm", ms(max(exchange_precontracted_flops(spec) / T, 8.0 * t * nMp * nMp / B)))
    # Cholesky-QR2 every qr_period steps: two Gram and two apply GEMMs
    qr = 2 * (8.0 * WS * N * N * NM * 2) / T
    out["qr"] = ("tensor", ms(qr / qr_period))
    return out


# ---------------------------------------------------------------------------
# measured DRAM traffic of a kernel, from its committed ncu summary
# ---------------------------------------------------------------------------
KERNEL_POLICY = {"taylor": "TaylorP", "exchange": "ExchangeP", "vhs": "VhsP", "adjoint": "AdjointP"}
CSRC = os.path.join(ROOT, "paper_2003_09468_gb300", "csrc")


def kernel_fingerprint(stage: str, read=None):
    """sha256 (12 hex digits) of the device code of the stage's GEMM kernel: tc.cuh and
    split.cuh, the device part of tc_gemm.cuh (from its namespace to the host-side
    section) and the text of the policy struct in mixed.cu.  `read(name)` returns a
    source file's text (default: the working tree)."""
    import hashlib
    pol = KERNEL_POLICY.get(stage)
    if pol is None:
        return None
    if read is None:
        def read(name):
            with open(os.path.join(CSRC, name)) as fh:
                return fh.read()
    h = hashlib.sha256()
    try:
        for f in ("tc.cuh", "split.cuh"):
            h.update(read(f).encode())
        g = read("tc_gemm.cuh")
        h.update(g[g.index("namespace tcg {"):g.index("// ---------------------------------------------------------------- host side")].encode())
        src = read("mixed.cu")
        a = src.index(f"struct {pol} {{")
        h.update(src[a:src.index("\n};\n", a)].encode())
    except (OSError, ValueError):
        return None
    return h.hexdigest()[:12]


def measured_traffic(stage: str, workload: str):
    """(bytes per launch, file) from profiles/<stage>_gemm_<workload>.md when the
    fingerprint recorded there matches the current sources, else (None, reason)."""
    path = os.path.join(ROOT, "profiles", f"{stage}_gemm_{workload}.md")
    try:
        with open(path) as f:
            text = f.read()
    except OSError:
        return None, "no ncu summary"
    vals = {}
    for line in text.splitlines():
        for key in ("traffic_bytes_per_launch:", "source_fingerprint:"):
            if line.strip().startswith(key):
                vals[key] = line.split(":", 1)[1].strip()
    fp = kernel_fingerprint(stage)
    if fp is None or vals.get("source_fingerprint:") != fp:
        return None, "kernel changed since the ncu capture"
    try:
        return float(vals["traffic_bytes_per_launch:"]), os.path.relpath(path, ROOT)
    except (KeyError, ValueError):
        return None, "no traffic line"


# ---------------------------------------------------------------------------
# clocks sampling during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.file.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# CPU oracle timing (test infrastructure; used only for cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
class OracleStepper:
    """The FP64 CPU oracle, built once for a workload; times single walker-steps and follows
    sampled walkers through the same steps the GPU takes."""

    def __init__(self, spec, L=None):
        from oracle import afqmc_kp as ok
        self.ok = ok
        self.spec = spec
        L = gen.cholesky(spec) if L is None else L      # the GPU arm passes its own copy of the inputs
        self.osys = ok.System(spec.grid, L, gen.one_body(spec), gen.trial(spec), spec.dt)

    def walker(self, walker_index: int = 0):
        return gen.near_trial_walkers(self.spec, 1, first=walker_index)[0]

    def seconds(self, walker_index: int = 0, step: int = 0) -> float:
        return self.run(walker_index, step)[0]

    def run(self, walker_index: int = 0, step: int = 0):
        """(seconds, propagated walker, weight for w = 1, (E1, EC, EX)) of one walker-step."""
        spec, ok = self.spec, self.ok
        phi = self.walker(walker_index)
        x = gen.fields(spec, step, 1, first=walker_index)[0]
        t0 = time.perf_counter()
        phi_new, w_new, _, _, _ = ok.propagate_walker(self.osys, phi, x, 1.0)
        e = ok.local_energy(self.osys, phi_new)
        return time.perf_counter() - t0, phi_new, w_new, np.array(e)

    def seeded(self, walker_index: int = 0):
        """(E1, EC, EX) and the force bias of a seeded walker as generated (untimed)."""
        ok = self.ok
        phi = self.walker(walker_index)
        Ghs = [ok.green_half(self.osys, phi[s])[0] for s in range(2)]
        return np.array(ok.local_energy(self.osys, phi)), ok.force_bias(self.osys, ok.cholesky_trace(self.osys, Ghs))

    def trajectory(self, walker_index: int, nsteps: int, qr_period: int, keep=()):
        """{step: (walker, weight, log det per spin, (E1, EC, EX))} after the steps listed in
        `keep` (1-based), for the seeded walker with the fields of steps 0 .. nsteps-1 and a QR
        after every qr_period-th step (untimed)."""
        ok, spec = self.ok, self.spec
        phi, w = self.walker(walker_index), 1.0
        out = {}
        for s in range(nsteps):
            x = gen.fields(spec, s, 1, first=walker_index)[0]
            phi, w, _, _, _ = ok.propagate_walker(self.osys, phi, x, w)
            if (s + 1) % qr_period == 0:
                phi = np.stack([ok.orthonormalise(phi[sp]) for sp in range(2)])
            if s + 1 in keep:
                ld = np.array([ok.log_det(ok.overlap(self.osys, phi[sp])) for sp in range(2)])
                out[s + 1] = (phi.copy(), w, ld, np.array(ok.local_energy(self.osys, phi)))
        return out

    def sampled_seconds(self, walker_index: int = 0, step: int = 0, nq: int = EX_SAMPLE_Q):
        """(seconds scaled to one walker-step, propagated walker, weight, description): the
        propagation, E1 and E_C of one walker timed in full and the exchange timed over the
        first nq momentum transfers and scaled by Nk / nq (every Q costs the same)."""
        spec, ok = self.spec, self.ok
        phi = self.walker(walker_index)
        x = gen.fields(spec, step, 1, first=walker_index)[0]
        t0 = time.perf_counter()
        phi_new, w_new, _, _, _ = ok.propagate_walker(self.osys, phi, x, 1.0)
        Ghs = [ok.green_half(self.osys, phi_new[s])[0] for s in range(2)]
        ok.one_body_energy(self.osys, Ghs)
        ok.coulomb_energy(self.osys, ok.cholesky_trace(self.osys, Ghs))
        t1 = time.perf_counter()
        ok.exchange_energy(self.osys, Ghs, Qs=range(nq))
        t2 = time.perf_counter()
        total = (t1 - t0) + (t2 - t1) * spec.nk / nq
        desc = (f"1 walker x 1 step of the workload: propagation, E1 and E_C timed in full ({t1 - t0:.1f} s), "
                f"the exchange timed over {nq} of {spec.nk} momentum transfers ({t2 - t1:.1f} s) and scaled "
                f"by {spec.nk // nq}: {total:.0f} s per walker-step (extrapolated), FP64 NumPy")
        return total, phi_new, w_new, desc

    def energy_parts(self, phi, pool_workers: int = 0):
        """(E1, EC, EX) of a walker; with pool_workers > 1 the exchange sum over Q is split over
        that many spawned processes (each sums the oracle's own exchange over its Q's)."""
        ok = self.ok
        Ghs = [ok.green_half(self.osys, phi[s])[0] for s in range(2)]
        e1 = ok.one_body_energy(self.osys, Ghs)
        ec = ok.coulomb_energy(self.osys, ok.cholesky_trace(self.osys, Ghs))
        if pool_workers <= 1:
            return np.array([e1, ec, ok.exchange_energy(self.osys, Ghs)])
        return np.array([e1, ec, exchange_in_pool(self.osys, Ghs, pool_workers)])

    def log_det_of(self, phi):
        ok = self.ok
        return np.array([ok.log_det(ok.overlap(self.osys, phi[s])) for s in range(2)])

    def force_bias_of(self, phi):
        ok = self.ok
        Ghs = [ok.green_half(self.osys, phi[s])[0] for s in range(2)]
        return ok.force_bias(self.osys, ok.cholesky_trace(self.osys, Ghs))


def cpu_cores() -> int:
    return os.cpu_count() or 1


class _ExchangeView:
    """What the oracle's exchange_energy reads from a System: the momentum tables, the block
    slices and LH, here holding only the momentum transfers one worker sums and their
    partners (the rest of the array is never touched, so it is never backed by memory)."""

    def __init__(self, grid, n, M, lh_parts):
        from oracle import afqmc_kp as ok
        self.kminus, self.minus = ok.kgrid_tables(grid)
        self.nk, self.n, self.M = len(self.minus), n, M
        shape = next(iter(lh_parts.values())).shape
        self.LH = np.zeros((self.nk,) + shape, dtype=np.complex128)
        for Q, v in lh_parts.items():
            self.LH[Q] = v

    def rows(self, k):
        return slice(k * self.n, (k + 1) * self.n)

    def cols(self, k):
        return slice(k * self.M, (k + 1) * self.M)


def _exchange_worker(args):
    from oracle import afqmc_kp as ok
    grid, n, M, lh_parts, Ghs, Qs = args
    return ok.exchange_energy(_ExchangeView(grid, n, M, lh_parts), Ghs, Qs=Qs)


def _gamma_worker(args):
    from oracle import afqmc_kp as ok
    grid, n, M, lh_parts, Gh, X, c2, c3, Qs = args
    return ok.gamma_two_body(_ExchangeView(grid, n, M, lh_parts), Gh, X, c2, c3, np.zeros_like(Gh), Qs=Qs)


def gamma_in_pool(workers):
    """A two_body for the oracle's local_energy_grad that splits its sum over Q across `workers`
    spawned processes (each runs the oracle's own gamma_two_body on its momentum transfers) and
    adds the partial blocks in Q-chunk order."""
    import multiprocessing as mp

    def two_body(osys, Gh, X, c2, c3, Gam):
        chunks = [c for c in (list(range(osys.nk))[i::workers] for i in range(workers)) if c]
        jobs = []
        for c in chunks:
            need = set(c) | {int(osys.minus[Q]) for Q in c}
            jobs.append((osys.grid, osys.n, osys.M, {Q: osys.LH[Q] for Q in need}, Gh, X, c2, c3, c))
        with mp.get_context("spawn").Pool(len(jobs)) as pool:
            for part in pool.map(_gamma_worker, jobs):
                Gam += part
        return Gam
    return two_body


def exchange_in_pool(osys, Ghs, workers):
    """The oracle's exchange energy with its sum over Q split across `workers` spawned
    processes (spawn: safe after the GPU has been used); the partial sums are added in Q order."""
    import multiprocessing as mp
    chunks = [list(range(osys.nk))[i::workers] for i in range(workers)]
    chunks = [c for c in chunks if c]
    jobs = []
    for c in chunks:
        need = set(c) | {int(osys.minus[Q]) for Q in c}
        jobs.append((osys.grid, osys.n, osys.M, {Q: osys.LH[Q] for Q in need}, Ghs, c))
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        parts = pool.map(_exchange_worker, jobs)
    return complex(sum(parts))


def workload_config(spec, workload, precision, world):
    """The `config` object of a k-point workload's line (the same for both arms)."""
    return {"workload": workload, "grid": list(spec.grid), "M": spec.M, "nocc": spec.nocc,
            "nchol": spec.nchol, "walkers_per_gpu": spec.nwalkers, "taylor_order": 6,
            "qr_period": QR_PERIOD, "precision": precision, "parallelism": f"replicas x{world}",
            "walkers": "near-trial: orthonormalised trial + 0.1 relative complex-normal noise per column",
            "l2": "inputs larger than L2 (Cholesky tensor alone exceeds 129 MB)"}


def parity_report_large(stepper, gpu_seeded, gpu_track, oracle_step, precision):
    """Walker 0 of a large workload against the oracle at the task's bars: the seeded walker's
    E_L parts and force bias, and after the first fused step the walker, weight, log det and
    E_L parts (the oracle's exchange summed in a process pool); no drift trajectory."""
    nk = stepper.spec.nk
    bars = BARS_MIXED if precision == "mixed" else {k: 1e-10 for k in BARS_MIXED}
    workers = cpu_cores()
    e_seed = stepper.energy_parts(stepper.walker(0), workers)
    xb_seed = stepper.force_bias_of(stepper.walker(0))
    es_g, xbs_g = gpu_seeded
    seeded_err = [float(abs(es_g[j] - e_seed[j]) / nk) for j in range(3)]
    xb_err = float(np.linalg.norm(xbs_g - xb_seed) / np.linalg.norm(xb_seed))
    seeded = {"E_L_err_ha_per_cell": seeded_err, "E_L_ha_per_cell": [float(e_seed[j].real / nk) for j in range(3)],
              "force_bias_rel_err": xb_err,
              "pass": bool(max(seeded_err) < bars["E_L_ha_per_cell"] and xb_err < bars["force_bias_rel"])}
    phi_r, w_r = oracle_step
    phi_g, w_g, e_g, ld_g = gpu_track[1]
    e_r = stepper.energy_parts(phi_r, workers)
    ld_own = stepper.log_det_of(phi_g)
    step1 = {"phi_rel_err": float(np.linalg.norm(phi_g - phi_r) / np.linalg.norm(phi_r)), "weight": w_g,
             "weight_rel_err": float(abs(w_g - w_r) / abs(w_r)) if w_r else None,
             "logdet_abs_err": float(np.max(np.abs(ld_g.real - ld_own.real))),
             "E_L_err_ha_per_cell": [float(abs(e_g[j] - e_r[j]) / nk) for j in range(3)],
             "E_L_ha_per_cell": [float(e_r[j].real / nk) for j in range(3)]}
    step1["pass"] = bool(w_r > 0 and step1["phi_rel_err"] < bars["phi_rel"]
                         and step1["weight_rel_err"] < bars["weight_rel"]
                         and step1["logdet_abs_err"] < bars["logdet_abs"]
                         and max(step1["E_L_err_ha_per_cell"]) < bars["E_L_ha_per_cell"])
    return {"walker": 0, "walkers": "near-trial (seeded)", "bars": bars, "seeded": seeded, "step_1": step1,
            "drift": None, "oracle_exchange": f"summed over Q in {workers} spawned processes",
            "device_flags_of_the_parity_run": STATUS_NAMES.get(gpu_track.get("status", 0), "?"),
            "pass": bool(seeded["pass"] and step1["pass"])}


def parity_report(stepper, gpu_seeded, gpu_track, oracle_step, precision):
    """Walker 0 of the GPU run against the oracle, at the task's bars.

    seeded   E_L and force bias of the seeded walker (per call, identical inputs);
    step_1   the walker, weight, log det and E_L after the first fused step, against the
             oracle's step from the same walker with the same fields;
    drift    the same after DRIFT_STEPS steps (QR every QR_PERIOD) against the oracle's own
             trajectory, and the force bias of the GPU's final walker against the oracle
             evaluated on that walker."""
    nk = stepper.spec.nk
    mixed = precision == "mixed"
    bars = BARS_MIXED if mixed else {k: 1e-10 for k in BARS_MIXED}
    e_seed, xb_seed = stepper.seeded(0)
    es_g, xbs_g = gpu_seeded
    seeded_err = [float(abs(es_g[j] - e_seed[j]) / nk) for j in range(3)]
    xb_err = float(np.linalg.norm(xbs_g - xb_seed) / np.linalg.norm(xb_seed))
    e_bar = [bars["E_L_ha_per_cell"] if mixed else bars["E_L_ha_per_cell"] * abs(e_seed[j]) / nk
             for j in range(3)]
    seeded = {"E_L_err_ha_per_cell": seeded_err, "E_L_ha_per_cell": [float(e_seed[j].real / nk) for j in range(3)],
              "force_bias_rel_err": xb_err,
              "pass": bool(all(seeded_err[j] < e_bar[j] for j in range(3)) and xb_err < bars["force_bias_rel"])}

    def compare(gpu, ref):
        phi_g, w_g, e_g, ld_g = gpu
        phi_r, w_r, ld_r, e_r = ref
        # the returned log det against the oracle's log det of the walker it belongs to (the
        # GPU's); against the oracle's trajectory it also carries the trajectories' difference
        ld_own = stepper.log_det_of(phi_g)
        row = {"phi_rel_err": float(np.linalg.norm(phi_g - phi_r) / np.linalg.norm(phi_r)),
               "weight": w_g, "weight_rel_err": float(abs(w_g - w_r) / abs(w_r)) if w_r else None,
               "logdet_abs_err": float(np.max(np.abs(ld_g.real - ld_own.real))),
               "logdet_abs_diff_vs_oracle_trajectory": float(np.max(np.abs(ld_g.real - ld_r.real))),
               "E_L_err_ha_per_cell": [float(abs(e_g[j] - e_r[j]) / nk) for j in range(3)],
               "E_L_ha_per_cell": [float(e_r[j].real / nk) for j in range(3)]}
        eb = [bars["E_L_ha_per_cell"] if mixed else bars["E_L_ha_per_cell"] * abs(e_r[j]) / nk for j in range(3)]
        row["pass"] = bool(w_r > 0 and row["phi_rel_err"] < bars["phi_rel"]
                           and row["weight_rel_err"] < bars["weight_rel"]
                           and row["logdet_abs_err"] < bars["logdet_abs"]
                           and all(row["E_L_err_ha_per_cell"][j] < eb[j] for j in range(3)))
        return row

    traj = stepper.trajectory(0, DRIFT_STEPS, QR_PERIOD, keep=(1, DRIFT_STEPS))
    step1 = compare(gpu_track[1], traj[1])
    drift = compare(gpu_track[DRIFT_STEPS], traj[DRIFT_STEPS])
    xb_ref = stepper.force_bias_of(gpu_track[DRIFT_STEPS][0])
    drift["force_bias_rel_err_on_gpu_walker"] = float(np.linalg.norm(gpu_track["xbar_end"] - xb_ref)
                                                      / np.linalg.norm(xb_ref))
    drift["pass"] = bool(drift["pass"] and drift["force_bias_rel_err_on_gpu_walker"] < bars["force_bias_rel"])
    drift["steps"] = DRIFT_STEPS
    phi_ref, w_ref, e_ref = oracle_step
    return {"walker": 0, "walkers": "near-trial (seeded)", "bars": bars, "seeded": seeded, "step_1": step1,
            "drift": drift, "device_flags_of_the_parity_run": STATUS_NAMES.get(gpu_track.get("status", 0), "?"),
            "pass": bool(seeded["pass"] and step1["pass"] and drift["pass"])}


def run_reference(args, spec, wl_name):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    times = []
    stepper = OracleStepper(spec)
    for i in range(args.warmup + args.steps):
        t = stepper.seconds(walker_index=i % spec.nwalkers, step=i)
        if i >= args.warmup:
            times.append(t)
    mean_s = sum(times) / len(times)
    value = 1.0 / mean_s
    cb = {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
          "sample": f"1 walker x 1 step (propagate + E_L) of {wl_name} per timed step, FP64 NumPy"}
    config = workload_config(spec, wl_name, "mixed" if args.precision in ("auto", "mixed") else "fp64", args.gpus)
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean_s * 1e3,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                      "data": "synthetic", "config": config,
                      "cpu_baseline": cb,
                      "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
GROUP_WORKLOAD = "batched-uneven-8"
DENSE_WORKLOAD = "dense-1x1x2"


def dense_oracle_seconds(nwalk, step):
    """Seconds per walker-step (propagate + E_L) of the standard-representation oracle on the
    dense workload, over nwalk walkers of one step."""
    from oracle import standard as so
    ds = gen.DENSE_1x1x2
    osys = so.StandardSystem(gen.dense_cholesky(ds), gen.dense_one_body(ds), gen.dense_trial(ds), ds.dt)
    phis, xo = gen.dense_near_trial_walkers(ds, nwalk), gen.dense_fields(ds, step, nwalk)
    t0 = time.perf_counter()
    for i in range(nwalk):
        pn, _, _, _ = so.propagate_walker(osys, phis[i], xo[i], 1.0)
        so.local_energy(osys, pn)
    return (time.perf_counter() - t0) / nwalk


def run_dense_reference(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    times = [dense_oracle_seconds(4, i) for i in range(args.warmup + args.steps)][args.warmup:]
    t = sum(times) / len(times)
    v = 1.0 / t
    sample = f"4 walkers x 1 step per timed step of {DENSE_WORKLOAD}, FP64 NumPy standard representation"
    print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": DENSE_WORKLOAD},
                      "cpu_baseline": {"value": v, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                                       "sample": sample},
                      "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def run_dense(args):
    """The standard (dense) representation of a two-cell Gamma-point supercell (M = 52, N = 8,
    416 real vectors, 64 walkers) against the same cells in the k-point representation
    (1x1x2 grid, M = 26, n = 4, 208 vectors per Q), the comparison of Sec. 3.1 on one GPU."""
    if int(os.environ.get("RANK", "0")) != 0:
        return   # one GPU's comparison: the other ranks of a multi-GPU launch have no work
    import torch
    from paper_2003_09468_gb300 import DenseAFQMC, KPointAFQMC

    def handle_fields(x):
        # real symmetric vectors: the + fields drive the handle's vectors; plane 1 has no effect
        out = np.zeros((x.shape[0], 2, 1, x.shape[2]))
        out[:, 0, 0, :] = x[:, 0]
        return out

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    ds, ks = gen.DENSE_1x1x2, gen.KPOINT_1x1x2
    nsteps = args.warmup + args.steps
    stream = torch.cuda.current_stream()

    def timed_steps(sys_, phi0, xs):
        phi = phi0.clone()
        w = torch.ones(phi.shape[0], dtype=torch.float64, device=dev)
        el = torch.empty((phi.shape[0], 3), dtype=torch.complex128, device=dev)
        for i in range(args.warmup):
            sys_.step(phi, xs[i], w, el, do_qr=((i + 1) % QR_PERIOD == 0), reuse=i > 0)
        torch.cuda.synchronize()
        sys_.profile(True)
        sys_.stage_times()
        launches = 0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(args.warmup, nsteps):
            sys_.step(phi, xs[i], w, el, do_qr=((i + 1) % QR_PERIOD == 0))
            launches += sys_.launch_count()
        e1.record(stream)
        torch.cuda.synchronize()
        st = sys_.stage_times()
        sys_.profile(False)
        return e0.elapsed_time(e1) / args.steps, launches, st, bool(torch.isfinite(el).all())

    dsys = DenseAFQMC(gen.dense_cholesky(ds), gen.dense_one_body(ds), gen.dense_trial(ds), ds.nwalkers, ds.dt,
                      precision="mixed", hermitian=True)
    dphi = torch.from_numpy(gen.dense_near_trial_walkers(ds)).to(dev)
    dxs = [torch.from_numpy(handle_fields(gen.dense_fields(ds, i))).to(dev) for i in range(nsteps)]
    clocks = Clocks(0)
    clocks.start()
    ms_d, launches_d, st_d, fin_d = timed_steps(dsys, dphi, dxs)
    clk = clocks.stop()
    dsys.close()
    ksys = KPointAFQMC(ks.grid, gen.cholesky(ks), gen.one_body(ks), gen.trial(ks), ks.nwalkers, ks.dt,
                       precision="mixed")
    kphi = torch.from_numpy(gen.near_trial_walkers(ks)).to(dev)
    kxs = [torch.from_numpy(gen.fields(ks, i)).to(dev) for i in range(nsteps)]
    ms_k, _, st_k, fin_k = timed_steps(ksys, kphi, kxs)
    ksys.close()
    cpu = None
    if not args.no_cpu_baseline:
        t = dense_oracle_seconds(4, 0)
        cpu = {"value": 1.0 / t, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": f"4 walkers x 1 step (propagate + E_L) of {DENSE_WORKLOAD}, FP64 NumPy standard "
                         f"representation, {t:.3f} s per walker-step"}
    out = {
        "metric": METRIC, "value": ds.nwalkers / (ms_d * 1e-3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_d, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f16x2-split/f32-acc + f64", "data": "synthetic",
        "config": {"workload": DENSE_WORKLOAD, "representation": "standard (dense), Gamma-point supercell",
                   "M": ds.M, "nocc": ds.nocc, "nchol": ds.nchol, "walkers_per_gpu": ds.nwalkers, "taylor_order": 6,
                   "qr_period": QR_PERIOD, "precision": "mixed", "parallelism": "replicas x1"},
        "kpoint_same_cells": {"grid": list(ks.grid), "M": ks.M, "nocc": ks.nocc, "nchol": ks.nchol,
                              "value": ks.nwalkers / (ms_k * 1e-3), "ms_per_step": ms_k,
                              "stages_ms": {k: round(v[0] / args.steps, 3) for k, v in st_k.items() if v[1]},
                              "finite": fin_k},
        "kpoint_over_dense": ms_d / ms_k,
        "stages_ms": {k: round(v[0] / args.steps, 3) for k, v in st_d.items() if v[1]},
        "roofline": None, "cpu_baseline": cpu, "e2e": None, "gpu_launches": launches_d, "clocks": clk,
        "finite": fin_d,
    }
    print(json.dumps(out))


def run_group(args):
    """Eight uneven systems (1024 walkers) advanced as one group, in each of the group's modes:
    the Taylor-term GEMMs shared (one persistent launch per term over all members' tiles, the
    rest of each member's step on its own stream; the default), every GEMM kind shared, and
    every member on its own launches.  Each mode is timed as a captured graph of two group
    steps (the headline is the default mode's) and as eager group steps; the members stepped
    one after another on one stream are what the group is measured against."""
    import torch
    import torch.distributed as dist
    from paper_2003_09468_gb300 import KPointAFQMC, KPointGroup

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    specs = gen.BATCHED_UNEVEN
    systems = [KPointAFQMC(s.grid, gen.cholesky(s), gen.one_body(s), gen.trial(s), s.nwalkers, s.dt,
                           precision="mixed") for s in specs]
    grp = KPointGroup(systems)
    shared_default = grp.shared
    tunings = [s_.gemm_tuning() for s_ in systems]
    nw = sum(s.nwalkers for s in specs)
    nsteps = args.warmup + args.steps
    xs = [[torch.from_numpy(gen.fields(s, i, s.nwalkers, first=rank * s.nwalkers)).to(dev) for s in specs]
          for i in range(nsteps)]
    phi0 = [torch.from_numpy(gen.near_trial_walkers(s, s.nwalkers, first=rank * s.nwalkers)).to(dev) for s in specs]
    phis = [p.clone() for p in phi0]
    ws = [torch.ones(s.nwalkers, dtype=torch.float64, device=dev) for s in specs]
    els = [torch.empty((s.nwalkers, 3), dtype=torch.complex128, device=dev) for s in specs]
    stream = torch.cuda.current_stream()

    def restart():
        for p, q, w in zip(phis, phi0, ws):
            p.copy_(q)
            w.fill_(1.0)

    def timed(fn):
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        if world > 1:
            t = torch.tensor([ms], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms

    def group_steps(lo, hi, launches=None):
        for i in range(lo, hi):
            grp.step(phis, xs[i], ws, els, do_qr=((i + 1) % QR_PERIOD == 0), reuse=i > 0)
            if launches is not None:
                launches[0] += grp.launch_count()

    def eager(mode, name):
        grp.shared = mode
        restart()
        group_steps(0, args.warmup)
        launches = [0]
        # an NVTX range names the timed steps for a profiler's launch filter
        torch.cuda.nvtx.range_push("eager_" + name)
        ms = timed(lambda: group_steps(args.warmup, nsteps, launches))
        torch.cuda.nvtx.range_pop()
        return ms, launches[0], all(bool(torch.isfinite(e).all()) for e in els)

    pairs = max(1, args.steps // 2)

    def graph(mode):
        """A captured graph of two group steps, replayed with each step's fields copied in."""
        grp.shared = mode
        restart()
        group_steps(0, 1)
        xa = [torch.empty_like(x) for x in xs[0]]
        xb = [torch.empty_like(x) for x in xs[0]]
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            grp.step(phis, xa, ws, els, do_qr=False)
            grp.step(phis, xb, ws, els, do_qr=True)

        def replays():
            for r in range(pairs):
                i = args.warmup + 2 * r
                for a, b, x0, x1 in zip(xa, xb, xs[i % nsteps], xs[(i + 1) % nsteps]):
                    a.copy_(x0)
                    b.copy_(x1)
                g.replay()

        replays()
        ms = timed(replays)
        del g
        return ms

    modes = {"shared_taylor": KPointGroup.SHARED_TAYLOR, "shared_all": KPointGroup.SHARED_ALL,
             "per_member": KPointGroup.PER_MEMBER}
    default = next(k for k, v in modes.items() if v == shared_default)
    order = [default] + [k for k in modes if k != default]
    clocks = Clocks(local)
    clocks.start()
    measured, finite = {}, True
    for name in order:
        ms_e, launches, fin = eager(modes[name], name)
        ms_g = graph(modes[name])
        finite = finite and fin
        measured[name] = {"graph": {"value": world * nw * 2 * pairs / (ms_g * 1e-3), "ms_per_step": ms_g / (2 * pairs)},
                          "eager": {"value": world * nw * args.steps / (ms_e * 1e-3),
                                    "ms_per_step": ms_e / args.steps, "gpu_launches": launches}}
        if name == default:
            clk = clocks.stop()

    # the same steps, members one after another on one stream
    restart()

    def seq_steps(lo, hi):
        for i in range(lo, hi):
            for j, s_ in enumerate(systems):
                s_.step(phis[j], xs[i][j], ws[j], els[j], do_qr=((i + 1) % QR_PERIOD == 0), reuse=i > 0)

    seq_steps(0, args.warmup)
    ms_seq = timed(lambda: seq_steps(args.warmup, nsteps))
    grp.close()
    for s_ in systems:
        s_.close()
    if rank == 0:
        per_graph = measured[default]["graph"]["ms_per_step"]
        seq = ms_seq / args.steps
        out = {
            "metric": METRIC, "value": measured[default]["graph"]["value"], "unit": UNIT, "n_gpus": world,
            "steps": 2 * pairs, "warmup": args.warmup, "ms_per_step": per_graph, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16x2-split/f32-acc + f64", "data": "synthetic",
            "config": {"workload": GROUP_WORKLOAD, "systems": [
                {"grid": list(s.grid), "M": s.M, "nocc": s.nocc, "nchol": s.nchol, "walkers": s.nwalkers}
                for s in specs], "walkers_per_gpu": nw, "taylor_order": 6, "qr_period": QR_PERIOD,
                "precision": "mixed", "parallelism": f"replicas x{world}", "group_mode": default,
                "timing": "CUDA graph of two group steps, replayed; fields copied in before each replay"},
            "modes": measured,
            "sequential_members": {"value": world * nw * args.steps / (ms_seq * 1e-3), "ms_per_step": seq},
            "speedup_graph_over_sequential": {k: seq / v["graph"]["ms_per_step"] for k, v in measured.items()},
            "roofline": None, "cpu_baseline": None, "e2e": None,
            "gpu_launches": measured[default]["eager"]["gpu_launches"],
            "clocks": clk, "finite": finite,
            "autotune": {"ring_depth_per_member": [{k: v["ring_depth"] for k, v in t.items()} for t in tunings]},
        }
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["auto", "mixed", "fp64"], default="auto")
    ap.add_argument("--workload", choices=list(WORKLOADS) + [GROUP_WORKLOAD, DENSE_WORKLOAD], default="diamond-3x3x3")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-block", action="store_true", help="skip the graph-captured paper block")
    ap.add_argument("--no-adjoint", action="store_true", help="skip timing the local-energy adjoint")
    ap.add_argument("--compare-fp64", type=int, default=1, help="also time one step of the FP64 path (N=1)")
    ap.add_argument("--windows", type=int, default=WINDOWS, help="timed windows of --steps steps (median)")
    ap.add_argument("--taylor-form", choices=["auto", "single", "pair"], default="auto",
                    help="the Taylor GEMM's tile form: the autotuner's choice, 128-row tiles, or CTA pairs")
    args = ap.parse_args()
    if args.workload == DENSE_WORKLOAD:
        if args.impl == "reference":
            return run_dense_reference(args)
        return run_dense(args)
    if args.workload == GROUP_WORKLOAD:
        if args.impl == "reference":
            # the oracle on one walker-step of the smallest member, as for the other workloads
            return run_reference(args, gen.BATCHED_UNEVEN[0], GROUP_WORKLOAD)
        return run_group(args)
    spec = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, spec, args.workload)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2003_09468_gb300 import KPointAFQMC, AfqmcError

    L, h1, A = gen.cholesky(spec), gen.one_body(spec), gen.trial(spec)
    precision = args.precision
    sys_ = None
    if precision in ("auto", "mixed"):
        try:
            sys_ = KPointAFQMC(spec.grid, L, h1, A, spec.nwalkers, spec.dt, precision="mixed")
            precision = "mixed"
        except AfqmcError as e:
            if args.precision == "mixed":
                raise
            if e.status != 6:
                raise
    if sys_ is None:
        precision = "fp64"
        sys_ = KPointAFQMC(spec.grid, L, h1, A, spec.nwalkers, spec.dt, precision="fp64")
    # TMA ring depth per GEMM and the Taylor GEMM's form, picked at create by the library's
    # autotuner (timed per launch); --taylor-form overrides the form
    if precision == "mixed" and args.taylor_form != "auto":
        sys_.set_gemm_form("taylor", args.taylor_form == "pair")
    autotune = sys_.gemm_tuning() if precision == "mixed" else None

    # walkers and fields: independent replicas per rank (disjoint walker indices); the walkers
    # start near the trial, as a projection does (Sec. 2.1)
    first = rank * spec.nwalkers
    phi0 = gen.near_trial_walkers(spec, spec.nwalkers, first=first)
    nsteps = args.warmup + args.steps
    nfields = max(nsteps, DRIFT_STEPS)
    xs = [torch.from_numpy(gen.fields(spec, i, spec.nwalkers, first=first)).to(dev) for i in range(nfields)]
    # the seeded walkers stay on the host (pinned) for the largest workload, whose handle takes
    # most of the device
    phi0_d = torch.from_numpy(phi0).pin_memory() if spec.nk >= LARGE_NK else torch.from_numpy(phi0).to(dev)
    phi = phi0_d.to(dev, copy=True)
    w = torch.ones(spec.nwalkers, dtype=torch.float64, device=dev)
    eloc = torch.empty((spec.nwalkers, 3), dtype=torch.complex128, device=dev)
    stream = torch.cuda.current_stream()

    launches = [0]

    def step(i, x, count=False):
        # one fused call: propagate, then the local energy of the new walkers; the Green's
        # function formed at the end of a step serves the next step's force bias (the first
        # step after a restart forms it afresh)
        sys_.step(phi, x, w, eloc, do_qr=((i + 1) % QR_PERIOD == 0), reuse=i > 0)
        if count:
            launches[0] += sys_.launch_count()

    def restart():
        phi.copy_(phi0_d)
        w.fill_(1.0)

    # Timed windows: each restarts from the seeded walkers, takes the W warm-up steps untimed
    # and then times exactly K steps (the same work in every window); the headline is the
    # median window.
    clocks = Clocks(local)
    window_ms = []
    stages = None
    gpu_launches = 0
    clocks.start()
    for r in range(args.windows):
        restart()
        for i in range(args.warmup):
            step(i, xs[i])
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        profile = r == args.windows - 1     # stage times from the last window
        if profile:
            sys_.profile(True)
            sys_.stage_times()
        launches[0] = 0
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for i in range(args.warmup, nsteps):
            step(i, xs[i], count=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_r = ev0.elapsed_time(ev1)
        if world > 1:
            t = torch.tensor([ms_r], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_r = float(t.item())
            dist.barrier()
        window_ms.append(ms_r)
        if profile:
            stages = sys_.stage_times()
            sys_.profile(False)
            gpu_launches = launches[0]
    clk = clocks.stop()
    torch.cuda.synchronize()
    ms = statistics.median(window_ms)
    value = world * spec.nwalkers * args.steps / (ms * 1e-3)
    windows = {"count": args.windows, "ms": [round(v, 4) for v in window_ms],
               "walker_steps_per_s": [world * spec.nwalkers * args.steps / (v * 1e-3) for v in window_ms],
               "headline": "median window; each window restarts from the seeded walkers, takes the warm-up "
                           "steps untimed and times exactly `steps` steps"}

    # validity of the timed steps: the library's sticky device flags (CUDA fault, a bounded
    # wait that gave up, a vHS entry beyond the split format, singular walkers) and a live
    # population with a finite mixed energy estimate
    status, n_sing = sys_.last_error()
    eloc_h = eloc.cpu().numpy()
    w_h = w.cpu().numpy()
    finite = bool(np.all(np.isfinite(eloc_h)))
    from paper_2003_09468_gb300.replicas import block_energy
    e_blk, w_blk = block_energy(eloc, w)
    e_cell = e_blk.real / spec.nk
    block = {"E_mixed_ha_per_cell": e_cell, "weight_sum": w_blk, "ranks": world,
             "live_walkers": int(np.sum(w_h > 0)), "walkers": int(w_h.size),
             "log10_weight_range": [float(np.log10(w_h[w_h > 0].min())), float(np.log10(w_h.max()))]
             if np.any(w_h > 0) else None}
    flags = {"status": int(status), "status_name": STATUS_NAMES.get(int(status), "?"), "singular_walkers": int(n_sing)}
    invalid = []
    if status in (3, 5, 6):
        invalid.append(f"device flag: {flags['status_name']}")
    if not (np.isfinite(w_blk) and w_blk > 0):
        invalid.append("no live walker after the timed steps")
    if not np.isfinite(e_cell):
        invalid.append("mixed energy estimate not finite")
    if not finite:
        invalid.append("non-finite local energies")

    # end-to-end through the public API with pinned host buffers: each step's fields copied in
    # from the host, each step's energies and weights copied back
    e2e = None
    if not args.no_e2e:
        xs_host = [x.cpu().pin_memory() for x in xs]
        e_host = torch.empty((spec.nwalkers, 3), dtype=torch.complex128).pin_memory()
        w_host = torch.empty(spec.nwalkers, dtype=torch.float64).pin_memory()
        xdev = torch.empty_like(xs[0])
        restart()
        for i in range(args.warmup):
            step(i, xs[i])
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for i in range(args.warmup, nsteps):
            xdev.copy_(xs_host[i], non_blocking=True)
            sys_.step(phi, xdev, w, eloc, do_qr=((i + 1) % QR_PERIOD == 0), reuse=True)
            e_host.copy_(eloc, non_blocking=True)
            w_host.copy_(w, non_blocking=True)
            stream.synchronize()
        t_e2e = time.perf_counter() - t0
        if world > 1:
            t = torch.tensor([t_e2e], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            t_e2e = float(t.item())
        e2e = {"value": world * spec.nwalkers * args.steps / t_e2e, "unit": UNIT,
               "h2d_bytes_per_step": int(xs[0].numel() * 8),
               "d2h_bytes_per_step": int(e_host.numel() * 16 + w_host.numel() * 8)}

    # the paper's block (20 propagation steps, then one energy evaluation and one walker
    # orthogonalisation, Sec. 3.1), fields drawn on the device and the comb at the end, all in
    # one captured CUDA graph; reported beside the step metric, untimed by the step clock
    paper_block = None
    if not args.no_block:
        nb = PAPER_BLOCK_STEPS
        xb = torch.empty_like(xs[0])
        ehb = torch.empty((1, spec.nwalkers, 3), dtype=torch.complex128, device=dev)
        counter = torch.tensor([1 << 20], dtype=torch.int64, device=dev)
        restart()

        def blk():
            sys_.block(phi, w, xb, ehb, counter, BLOCK_SEED + rank, nsteps=nb, qr_period=nb, energy_period=nb,
                       comb=True)

        blk()                      # eager: one-time kernel attributes, and the launch count
        blk_launches = sys_.launch_count()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            blk()
        g.replay()
        torch.cuda.synchronize()
        reps = 5 if spec.nk < LARGE_NK else 1
        b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        b0.record(stream)
        for _ in range(reps):
            g.replay()
        b1.record(stream)
        torch.cuda.synchronize()
        ms_blk = b0.elapsed_time(b1) / reps
        if world > 1:
            t = torch.tensor([ms_blk], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_blk = float(t.item())
        eb = ehb[0].cpu().numpy()
        wb = w.cpu().numpy()
        bst, _ = sys_.last_error()
        paper_block = {"ms_per_block": ms_blk, "walker_steps_per_s": world * spec.nwalkers * nb / (ms_blk * 1e-3),
                       "unit": UNIT, "steps_per_block": nb, "energy_evaluations": 1, "qr": 1, "comb": True,
                       "fields": "Philox4x32-10 + Box-Muller on the device", "cuda_graph": True,
                       "replays_timed": reps, "gpu_launches_per_block": blk_launches,
                       "finite": bool(np.all(np.isfinite(eb))), "weight_after_comb": float(wb[0]),
                       "device_flags": STATUS_NAMES.get(int(bst), "?")}
        del g

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # GPU walker 0 after one step and after DRIFT_STEPS steps (QR every QR_PERIOD), from the
    # seeded walkers with the fields of steps 0, 1, ...: the parity report's GPU side (untimed)
    gpu_track = {}
    gpu_seeded = None
    if not args.no_cpu_baseline and world == 1:
        restart()
        e_s = sys_.local_energy(phi)
        xb_s = sys_.force_bias(phi)
        torch.cuda.synchronize()
        gpu_seeded = (e_s[0].cpu().numpy(), xb_s[0].cpu().numpy())
        ld = torch.empty((spec.nwalkers, 2), dtype=torch.complex128, device=dev)
        for i in range(1 if spec.nk >= LARGE_NK else DRIFT_STEPS):
            sys_.step(phi, xs[i], w, eloc, logdet=ld, do_qr=((i + 1) % QR_PERIOD == 0), reuse=i > 0)
            if i + 1 in (1, DRIFT_STEPS):
                torch.cuda.synchronize()
                gpu_track[i + 1] = (phi[0].cpu().numpy(), float(w[0].item()), eloc[0].cpu().numpy(),
                                    ld[0].cpu().numpy())
        xb_end = sys_.force_bias(phi)
        torch.cuda.synchronize()
        gpu_track["xbar_end"] = xb_end[0].cpu().numpy()
        tst, _ = sys_.last_error()
        gpu_track["status"] = int(tst)

    # derived rates from the per-stage times: propagation (with the Green's function that the
    # fused step forms for the next step) and the local energy
    steps_t = max(args.steps, 1)
    prop_ms = sum(stages[k][0] for k in ("green", "force_bias", "vhs", "taylor", "onebody", "weight", "qr")) / steps_t
    en_ms = sum(stages[k][0] for k in ("energy", "exchange")) / steps_t
    rates = {"propagate_only": spec.nwalkers * world / (prop_ms * 1e-3) if prop_ms > 0 else None,
             "local_energy_only": spec.nwalkers * world / (en_ms * 1e-3) if en_ms > 0 else None,
             "unit": UNIT, "source": "per-stage CUDA-event times of the last timed window"}

    peaks, peaks_kind = load_peaks()
    rooflines = {}
    tensor_peak = peaks.get("bf16_tflops_sustained", 1700.0)

    def put(stage, bound, work, peak, unit, note):
        """Per-launch roofline of the kernel a stage times: the library records one
        interval per launch for the Taylor GEMM and the exchange GEMM."""
        ms_s, n_s = stages[stage]
        if not n_s:
            return
        per = ms_s / n_s
        scale = 1e12 if unit == "TFLOP/s" else 1e9
        ach = work / (per * 1e-3) / scale
        traffic, src = measured_traffic(stage, args.workload) if precision == "mixed" else (None, None)
        rooflines[stage] = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                            "traffic": traffic, "traffic_source": src, "kernel": stage, "launches": n_s,
                            "launch_ms": per, "algorithmic_per_launch": work, "peak_source": note}

    if precision == "fp64":
        dtype = "f64"
        put("exchange", "alu", exchange_flops(spec), 1.25, "TFLOP/s",
            "FP64 nominal 1.25 TFLOP/s (GB300 FP64 pipe); a DFMA probe measured 1.20")
    else:
        dtype = "f16x2-split/f32-acc + f64"
        note = f"dense f16/bf16 tensor, sustained (kernel timed inside the step), {peaks_kind}"
        put("taylor", "tensor", taylor_term_flops(spec), tensor_peak, "TFLOP/s",
            note + "; one Taylor-term GEMM per launch, algorithmic flops (the 3-product fp16 split "
                   "issues up to 3x as many)")
        put("exchange", "tensor", exchange_precontracted_flops(spec), tensor_peak, "TFLOP/s",
            note + "; algorithmic flops")
        put("vhs", "hbm", vhs_bytes(spec), peaks.get("hbm_gbs", 6800.0), "GB/s",
            f"HBM copy, {peaks_kind}; stage = operand split + one GEMM launch")
    # dominant kernel: the largest total time in the timed region
    dom = max(rooflines, key=lambda k: stages[k][0]) if rooflines else None
    # whole step: every stage at its own bound against the live stage times
    step_roofline = None
    if precision == "mixed":
        model = step_roofline_model(spec, QR_PERIOD, tensor_peak, peaks.get("hbm_gbs", 6800.0),
                                    (clk or {}).get("sm_max_mhz") or 2070.0)
        per = {}
        for k, (bound, ideal) in model.items():
            live = stages[k][0] / steps_t if stages.get(k) and stages[k][1] else None
            per[k] = {"bound": bound, "ideal_ms": round(ideal, 4), "live_ms": round(live, 4) if live else None,
                      "frac": round(ideal / live, 3) if live else None}
        ideal_total = sum(v[1] for v in model.values())
        step_roofline = {"ideal_ms": ideal_total, "measured_ms": ms / args.steps,
                         "frac": ideal_total / (ms / args.steps), "stages": per,
                         "model": "each stage's kernels at their own bound: algorithmic flops at the sustained "
                                  "tensor peak, algorithmic bytes at the HBM copy rate, double-float work at "
                                  f"{FF_OPS_PER_CMAC:.0f} FP32 instructions per complex multiply-add at the FP32 "
                                  "issue rate; E1/E_C, weights and reductions omitted (small)"}
    roofline = rooflines.get(dom)

    # the adjoint (dE/dphi and dE/dh for every walker; configs of the adjoint study use the
    # same system), timed with CUDA events after one warm-up call
    adjoint = None
    g_up = torch.from_numpy(gen.upstream(spec)).to(dev)
    restart()

    def time_backward(s_, reps, profile=False):
        s_.local_energy_backward(phi, g_up)
        torch.cuda.synchronize()
        if profile:
            s_.profile(True)
            s_.stage_times()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(reps):
            s_.local_energy_backward(phi, g_up)
        a1.record(stream)
        torch.cuda.synchronize()
        st_ = None
        if profile:
            st_ = s_.stage_times()
            s_.profile(False)
        return a0.elapsed_time(a1) / reps, s_.launch_count(), st_

    if not args.no_adjoint:
        ms_adj, adj_launches, adj_stages = time_backward(sys_, 3, profile=True)
        adjoint = {"ms_per_call": ms_adj, "walker_gradients_per_s": world * spec.nwalkers / (ms_adj * 1e-3),
                   "precision": precision, "gpu_launches_per_call": adj_launches,
                   "stages_ms_per_call": {k: round(v[0] / 3, 3) for k, v in adj_stages.items() if v[1]},
                   "outputs": "dE/dphi [W][2][NM][N] and dE/dh [Nk][M][M] for upstream g[W][3]"}
        if precision == "mixed":
            ms_s, n_s = adj_stages["adjoint_gemm"]
            if n_s:
                per = ms_s / n_s
                work = adjoint_exchange_flops(spec)
                ach = work / (per * 1e-3) / 1e12
                traffic, src = measured_traffic("adjoint", args.workload)
                rooflines["adjoint_gemm"] = {
                    "bound": "tensor", "achieved": ach, "peak": tensor_peak, "unit": "TFLOP/s",
                    "frac": ach / tensor_peak, "traffic": traffic, "traffic_source": src, "kernel": "adjoint_gemm",
                    "launches": n_s, "launch_ms": per, "algorithmic_per_launch": work,
                    "peak_source": f"dense f16/bf16 tensor, sustained, {peaks_kind}; algorithmic flops of the "
                                   "exchange adjoint over all Nk^3 triples (outside the step)"}

    fp64_cmp = None
    large = spec.nk >= LARGE_NK
    if large:
        fp64_cmp = {"skipped": "FP64 handle at this size: ~150 GB of device buffers and a direct exchange of "
                               "~375 TFLOP per step on the 1.2 TFLOP/s FP64 pipe (minutes per step)"}
    if precision == "mixed" and args.compare_fp64 and world == 1 and not large:
        del sys_
        torch.cuda.synchronize()
        s64 = KPointAFQMC(spec.grid, L, h1, A, spec.nwalkers, spec.dt, precision="fp64")
        restart()
        step_fn = lambda i, x: s64.step(phi, x, w, eloc, do_qr=((i + 1) % QR_PERIOD == 0), reuse=i > 0)
        step_fn(0, xs[0])
        torch.cuda.synchronize()
        n64 = max(FP64_STEPS, 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(1, 1 + n64):
            step_fn(i, xs[i % nfields])
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1) / n64
        fp64_cmp = {"value": spec.nwalkers / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64, "steps": n64,
                    "speedup_mixed_over_fp64": value / (spec.nwalkers / (ms64 * 1e-3))}
        if adjoint is not None:
            restart()
            ms_adj64, _, _ = time_backward(s64, 1)
            adjoint["fp64_ms_per_call"] = ms_adj64
            adjoint["speedup_mixed_over_fp64"] = ms_adj64 / adjoint["ms_per_call"]
        s64.close()
        sys_ = None

    cpu_baseline = None
    parity = None
    if not args.no_cpu_baseline and world == 1:
        stepper = OracleStepper(spec, L)
        if large:
            t, phi_ref, w_ref, desc = stepper.sampled_seconds(0, 0)
            cpu_baseline = {"value": 1.0 / t, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
                            "extrapolated": True}
            if gpu_track:
                parity = parity_report_large(stepper, gpu_seeded, gpu_track, (phi_ref, w_ref), precision)
        else:
            t, phi_ref, w_ref, e_ref = stepper.run(0, 0)
            cpu_baseline = {"value": 1.0 / t, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                            "sample": f"1 walker x 1 step (propagate + E_L) of {args.workload}, FP64 NumPy, "
                                      f"{t:.1f} s"}
            if gpu_track:
                parity = parity_report(stepper, gpu_seeded, gpu_track, (phi_ref, w_ref, e_ref), precision)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": workload_config(spec, args.workload, precision, world),
        "roofline": roofline,
        "rooflines": rooflines,
        "step_roofline": step_roofline,
        "windows": windows,
        "autotune": autotune,
        "fp64_path": fp64_cmp,
        "cpu_baseline": cpu_baseline,
        "parity": parity,
        "block_energy": block,
        "device_flags": flags,
        "valid": not invalid,
        "invalid_reasons": invalid,
        "rates": rates,
        "paper_block": paper_block,
        "adjoint": adjoint,
        "e2e": e2e,
        "gpu_launches": gpu_launches,
        "clocks": clk,
        "stages_ms": {k: round(v[0], 3) for k, v in stages.items() if v[1]},
        "finite": finite,
    }
    print(json.dumps(out))
    if sys_ is not None:
        sys_.close()
    if world > 1:
        dist.destroy_process_group()
    if invalid:
        sys.exit(1)


if __name__ == "__main__":
    main()
