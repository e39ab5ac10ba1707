"""Groups of uneven systems (afqmc_kp_group_*) against the members run alone and the oracle.

Each member of a group computes what the same call on the member alone computes, bit for
bit: the group only places the members' kernels on concurrent streams.  That holds for
eager group calls, for a group step captured in a CUDA graph and for the group block.  The
energy each member returns inside the group is also checked against the oracle on the
walker the GPU propagated, at the per-path bars of test_gpu_step.
"""
import numpy as np
import pytest

import gen
from oracle import afqmc_kp as ok

torch = pytest.importorskip("torch")
from gpu_util import dev, host, make  # noqa: E402

pytestmark = pytest.mark.gpu

# uneven sizes, walker counts and precisions in one group (ragged tiles in every member)
MEMBERS = [
    (gen.SystemSpec(grid=(2, 2, 1), M=6, nocc=2, nchol=24, nwalkers=8, random_trial=True, seed=21), "mixed"),
    (gen.SystemSpec(grid=(1, 2, 3), M=8, nocc=3, nchol=32, nwalkers=12, random_trial=True, seed=22), "mixed"),
    (gen.SystemSpec(grid=(2, 2, 2), M=8, nocc=2, nchol=48, nwalkers=16, random_trial=True, seed=23), "fp64"),
    (gen.SystemSpec(grid=(1, 1, 1), M=5, nocc=2, nchol=4, nwalkers=3, random_trial=True, seed=24), "mixed"),
]
# walkers near the trial: the task's absolute energy bar on the mixed path
BARS = {"fp64": dict(e_cell=1e-10, e_rel=1e-10), "mixed": dict(e_cell=1e-5, e_rel=0.0)}


def state(spec):
    return dev(gen.near_trial_walkers(spec)), dev(np.linspace(0.8, 1.2, spec.nwalkers))


def run_steps(mode, nsteps=3):
    """(phi, w, eloc) per member after nsteps steps: 'alone', 'group' or 'graph'."""
    from paper_2003_09468_gb300 import KPointGroup
    sys_ = [make(spec, prec)[0] for spec, prec in MEMBERS]
    st = [state(spec) for spec, _ in MEMBERS]
    el = [torch.empty((spec.nwalkers, 3), dtype=torch.complex128, device="cuda") for spec, _ in MEMBERS]
    xs = [[dev(gen.fields(spec, s)) for s in range(nsteps)] for spec, _ in MEMBERS]
    if mode == "alone":
        for i, s_ in enumerate(sys_):
            for s in range(nsteps):
                s_.step(st[i][0], xs[i][s], st[i][1], el[i], do_qr=(s == 1), reuse=s > 0)
    else:
        grp = KPointGroup(sys_)
        phis, ws = [p for p, _ in st], [w for _, w in st]
        grp.step(phis, [x[0] for x in xs], ws, el, reuse=False)
        if mode == "group":
            for s in range(1, nsteps):
                grp.step(phis, [x[s] for x in xs], ws, el, do_qr=(s == 1))
        else:
            xa = [torch.empty_like(x[0]) for x in xs]
            xb = [torch.empty_like(x[0]) for x in xs]
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                grp.step(phis, xa, ws, el, do_qr=True)
                grp.step(phis, xb, ws, el, do_qr=False)
            for a, b, x in zip(xa, xb, xs):
                a.copy_(x[1])
                b.copy_(x[2])
            g.replay()
        assert grp.launch_count() > 0
        grp.close()
    torch.cuda.synchronize()
    out = [(host(p), host(w), host(e), s_.last_error()) for (p, w), e, s_ in zip(st, el, sys_)]
    for s_ in sys_:
        s_.close()
    return out


def test_group_steps_equal_members_alone_and_graph():
    alone = run_steps("alone")
    group = run_steps("group")
    graph = run_steps("graph")
    for a, g, c in zip(alone, group, graph):
        for j in range(3):
            assert np.array_equal(a[j], g[j])
            assert np.array_equal(a[j], c[j])
        assert a[3] == g[3] == c[3] == (0, 0)
        assert np.all(np.isfinite(a[2]))


def test_group_energies_match_oracle():
    from paper_2003_09468_gb300 import KPointGroup
    made = [make(spec, prec) for spec, prec in MEMBERS]
    sys_ = [m[0] for m in made]
    st = [state(spec) for spec, _ in MEMBERS]
    grp = KPointGroup(sys_)
    el = [torch.empty((spec.nwalkers, 3), dtype=torch.complex128, device="cuda") for spec, _ in MEMBERS]
    grp.step([p for p, _ in st], [dev(gen.fields(spec, 0)) for spec, _ in MEMBERS], [w for _, w in st], el,
             reuse=False)
    for (spec, prec), (_, osys), (p, _), e in zip(MEMBERS, made, st, el):
        got_phi, got_e = host(p), host(e)
        for i in (0, spec.nwalkers - 1):
            ref = np.array(ok.local_energy(osys, got_phi[i]))
            err = np.abs(got_e[i] - ref) / spec.nk
            allowed = np.maximum(BARS[prec]["e_cell"], BARS[prec]["e_rel"] * np.abs(ref) / spec.nk)
            assert np.all(err < allowed), (spec.grid, prec, i, err, allowed)
    grp.close()
    for s_ in sys_:
        s_.close()


def test_group_block_equals_member_blocks():
    from paper_2003_09468_gb300 import KPointGroup
    nsteps, seed = 4, 99

    def run(grouped):
        sys_ = [make(spec, prec)[0] for spec, prec in MEMBERS]
        st = [state(spec) for spec, _ in MEMBERS]
        xs = [torch.empty(s_.field_shape, dtype=torch.float64, device="cuda") for s_ in sys_]
        eh = [torch.empty((2, spec.nwalkers, 3), dtype=torch.complex128, device="cuda") for spec, _ in MEMBERS]
        cs = [torch.tensor([7 * i], dtype=torch.int64, device="cuda") for i in range(len(MEMBERS))]
        if grouped:
            grp = KPointGroup(sys_)
            grp.block([p for p, _ in st], [w for _, w in st], xs, eh, cs, seed, nsteps, qr_period=2,
                      energy_period=2)
            grp.close()
        else:
            for i, s_ in enumerate(sys_):
                s_.block(st[i][0], st[i][1], xs[i], eh[i], cs[i], seed, nsteps=nsteps, qr_period=2, energy_period=2)
        torch.cuda.synchronize()
        out = [(host(p), host(w), host(e), int(host(c)[0])) for (p, w), e, c in zip(st, eh, cs)]
        for s_ in sys_:
            s_.close()
        return out

    a, g = run(False), run(True)
    for x, y in zip(a, g):
        for j in range(3):
            assert np.array_equal(x[j], y[j])
        assert x[3] == y[3]


def test_group_rejects_bad_arguments():
    from paper_2003_09468_gb300 import KPointGroup, AfqmcError
    spec, prec = MEMBERS[0]
    s_ = make(spec, prec)[0]
    with pytest.raises(AfqmcError):
        KPointGroup([s_, s_])               # a handle may appear once
    grp = KPointGroup([s_])
    p, w = state(spec)
    with pytest.raises(ValueError):
        grp.step([p, p], [dev(gen.fields(spec, 0))], [w])
    grp.close()
    s_.close()
