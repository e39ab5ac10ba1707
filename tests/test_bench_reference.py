"""The benchmark's reference arm (the FP64 oracle on the host cores) keeps its JSON contract:
one line with impl = reference, the metric and unit of the GPU arm, a positive rate, the CPU
baseline it measured and an end-to-end entry with no host/device copies.  CPU only."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("workload", ["small-2x2x2", "dense-1x1x2", "batched-uneven-8"])
def test_reference_arm_line(workload):
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", workload,
                        "--steps", "1", "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"].startswith("walker-steps/s") and d["unit"] == "walker-steps/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]


def test_parity_report_gates_at_the_task_bars():
    """The benchmark's parity block, fed the oracle's own values for the GPU side, passes with
    zero errors; a walker moved by 1e-5 (ten times the phi bar) fails it."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import gen
    spec = gen.SMALL_2x2x2
    st = bench.OracleStepper(spec)
    e0, xb0 = st.seeded(0)
    traj = st.trajectory(0, bench.DRIFT_STEPS, bench.QR_PERIOD, keep=(1, bench.DRIFT_STEPS))
    track = {n: (traj[n][0], traj[n][1], traj[n][3], traj[n][2]) for n in (1, bench.DRIFT_STEPS)}
    track["xbar_end"] = st.force_bias_of(traj[bench.DRIFT_STEPS][0])
    _, phi1, w1, e1 = st.run(0, 0)
    rep = bench.parity_report(st, (e0, xb0), track, (phi1, w1, e1), "mixed")
    assert rep["pass"], rep
    assert rep["step_1"]["phi_rel_err"] == 0.0 and max(rep["drift"]["E_L_err_ha_per_cell"]) == 0.0
    assert rep["step_1"]["weight"] > 0 and rep["drift"]["weight"] > 0
    bad = dict(track)
    p, w, e, ld = track[bench.DRIFT_STEPS]
    bad[bench.DRIFT_STEPS] = (p * (1 + 1e-5), w, e, ld)
    rep = bench.parity_report(st, (e0, xb0), bad, (phi1, w1, e1), "mixed")
    assert not rep["drift"]["pass"] and not rep["pass"] and rep["step_1"]["pass"]


def test_pooled_oracle_sums_equal_the_oracle():
    """The benchmark's process-pool forms of the oracle's exchange energy and of its two-body
    gradient blocks (the sum over Q split across spawned processes) give the oracle's values."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    import gen
    from oracle import afqmc_kp as ok
    spec = gen.SystemSpec(grid=(2, 2, 1), M=5, nocc=2, nchol=6, nwalkers=1, random_trial=True, seed=3)
    osys = ok.System(spec.grid, gen.cholesky(spec), gen.one_body(spec), gen.trial(spec), spec.dt)
    phi = gen.near_trial_walkers(spec)[0]
    Ghs = [ok.green_half(osys, phi[s])[0] for s in range(2)]
    ex = ok.exchange_energy(osys, Ghs)
    assert abs(bench.exchange_in_pool(osys, Ghs, 3) - ex) < 1e-12 * abs(ex)
    g = gen.upstream(spec)[0]
    a = ok.local_energy_vjp(osys, phi, g)
    b = ok.local_energy_vjp(osys, phi, g, two_body=bench.gamma_in_pool(3))
    assert np.abs(a[0] - b[0]).max() < 1e-12 * np.abs(a[0]).max()
    assert np.abs(a[1] - b[1]).max() == 0.0
