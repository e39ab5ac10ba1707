"""Groups of uneven systems (afqmc_kp_group_*) against the members run alone and the oracle.

Each member of a group computes what the same call on the member alone computes, bit for
bit, whether the group places the members' kernels on concurrent streams or (all members
mixed) launches the Taylor-term GEMMs, or every GEMM kind, once over the tiles of every member.  That holds for eager
group calls, for a group step captured in a CUDA graph and for the group block.  The energy
each member returns inside the group is also checked against the oracle on the walker the
GPU propagated, at the per-path bars of test_gpu_step.
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
# all mixed: the GEMMs are shared launches.  Uneven grids, orbital and vector counts, walker
# counts; the last member has more than 128 walker-spin rows (two row tiles in the exchange).
MIXED = [
    (gen.SystemSpec(grid=(2, 2, 1), M=6, nocc=2, nchol=24, nwalkers=8, random_trial=True, seed=31), "mixed"),
    (gen.SystemSpec(grid=(1, 2, 3), M=8, nocc=3, nchol=32, nwalkers=12, random_trial=True, seed=32), "mixed"),
    (gen.SystemSpec(grid=(2, 2, 2), M=8, nocc=2, nchol=48, nwalkers=16, random_trial=True, seed=33), "mixed"),
    (gen.SystemSpec(grid=(1, 1, 1), M=5, nocc=2, nchol=4, nwalkers=3, random_trial=True, seed=34), "mixed"),
    (gen.SystemSpec(grid=(1, 1, 2), M=6, nocc=2, nchol=12, nwalkers=70, random_trial=True, seed=35), "mixed"),
]
# walkers near the trial: the task's absolute energy bar on the mixed path
BARS = {"fp64": dict(e_cell=1e-10, e_rel=1e-10), "mixed": dict(e_cell=1e-5, e_rel=0.0)}


def state(spec):
    return dev(gen.near_trial_walkers(spec)), dev(np.linspace(0.8, 1.2, spec.nwalkers))


def run_steps(mode, members=MEMBERS, shared=None, nsteps=3):
    """(phi, w, eloc, logdet, last_error) per member after nsteps steps: 'alone', 'group' or
    'graph'.  Member 1 skips its energy on the last step; the do_qr step returns log dets."""
    from paper_2003_09468_gb300 import KPointGroup
    sys_ = [make(spec, prec)[0] for spec, prec in members]
    st = [state(spec) for spec, _ in members]
    el = [torch.zeros((spec.nwalkers, 3), dtype=torch.complex128, device="cuda") for spec, _ in members]
    ld = [torch.zeros((spec.nwalkers, 2), dtype=torch.complex128, device="cuda") for spec, _ in members]
    xs = [[dev(gen.fields(spec, s)) for s in range(nsteps)] for spec, _ in members]

    def elocs(s):
        return [None if (i == 1 and s == nsteps - 1) else e for i, e in enumerate(el)]

    if mode == "alone":
        for i, s_ in enumerate(sys_):
            for s in range(nsteps):
                e = elocs(s)[i]
                s_.step(st[i][0], xs[i][s], st[i][1], e, logdet=ld[i] if s == 1 else None, do_qr=(s == 1),
                        reuse=s > 0, energy=e is not None)
    else:
        grp = KPointGroup(sys_)
        if shared is not None:
            grp.shared = shared
        phis, ws = [p for p, _ in st], [w for _, w in st]
        grp.step(phis, [x[0] for x in xs], ws, elocs(0), reuse=False)
        if mode == "group":
            for s in range(1, nsteps):
                grp.step(phis, [x[s] for x in xs], ws, elocs(s), logdets=ld if s == 1 else None, do_qr=(s == 1))
        else:
            xa = [torch.empty_like(x[0]) for x in xs]
            xb = [torch.empty_like(x[0]) for x in xs]
            torch.cuda.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                grp.step(phis, xa, ws, elocs(1), logdets=ld, do_qr=True)
                grp.step(phis, xb, ws, elocs(2), do_qr=False)
            for a, b, x in zip(xa, xb, xs):
                a.copy_(x[1])
                b.copy_(x[2])
            g.replay()
        assert grp.launch_count() > 0
        grp.close()
    torch.cuda.synchronize()
    out = [(host(p), host(w), host(e), host(d), s_.last_error()) for (p, w), e, d, s_ in zip(st, el, ld, sys_)]
    for s_ in sys_:
        s_.close()
    return out


def check_equal(runs):
    first = runs[0]
    for other in runs[1:]:
        for a, b in zip(first, other):
            for j in range(4):
                assert np.array_equal(a[j], b[j])
            assert a[4] == b[4] == (0, 0)
    for a in first:
        assert np.all(np.isfinite(a[2]))


def test_group_steps_equal_members_alone_and_graph():
    check_equal([run_steps("alone"), run_steps("group"), run_steps("graph")])


def test_shared_gemm_group_steps_equal_members_alone_and_graph():
    from paper_2003_09468_gb300 import KPointGroup as G
    alone = run_steps("alone", MIXED)
    check_equal([alone, run_steps("group", MIXED), run_steps("graph", MIXED),
                 run_steps("group", MIXED, shared=G.SHARED_ALL), run_steps("graph", MIXED, shared=G.SHARED_ALL),
                 run_steps("group", MIXED, shared=G.PER_MEMBER)])


def test_shared_gemms_only_for_mixed_groups_of_one_order():
    from paper_2003_09468_gb300 import KPointGroup, AfqmcError
    sys_ = [make(spec, prec)[0] for spec, prec in MEMBERS]
    grp = KPointGroup(sys_)               # an FP64 member: per-member streams
    assert grp.shared == KPointGroup.PER_MEMBER
    for mode in (KPointGroup.SHARED_ALL, KPointGroup.SHARED_TAYLOR):
        with pytest.raises(AfqmcError):
            grp.shared = mode
    with pytest.raises(AfqmcError):
        grp.shared = 3
    grp.close()
    mixed = [s_ for s_, (_, prec) in zip(sys_, MEMBERS) if prec == "mixed"]
    grp = KPointGroup(mixed)
    assert grp.shared == KPointGroup.SHARED_TAYLOR
    for mode in (KPointGroup.PER_MEMBER, KPointGroup.SHARED_ALL, KPointGroup.SHARED_TAYLOR):
        grp.shared = mode
        assert grp.shared == mode
    grp.close()
    other = make(MIXED[3][0], "mixed", taylor_order=4)[0]
    grp = KPointGroup(mixed + [other])    # two Taylor orders
    assert grp.shared == KPointGroup.PER_MEMBER
    grp.close()
    for s_ in sys_ + [other]:
        s_.close()


@pytest.mark.parametrize("members", [MEMBERS, MIXED], ids=["streams", "shared"])
def test_group_energies_match_oracle(members):
    from paper_2003_09468_gb300 import KPointGroup
    made = [make(spec, prec) for spec, prec in members]
    sys_ = [m[0] for m in made]
    st = [state(spec) for spec, _ in members]
    grp = KPointGroup(sys_)
    el = [torch.empty((spec.nwalkers, 3), dtype=torch.complex128, device="cuda") for spec, _ in members]
    grp.step([p for p, _ in st], [dev(gen.fields(spec, 0)) for spec, _ in members], [w for _, w in st], el,
             reuse=False)
    for (spec, prec), (_, osys), (p, _), e in zip(members, made, st, el):
        got_phi, got_e = host(p), host(e)
        for i in (0, spec.nwalkers - 1):
            ref = np.array(ok.local_energy(osys, got_phi[i]))
            err = np.abs(got_e[i] - ref) / spec.nk
            allowed = np.maximum(BARS[prec]["e_cell"], BARS[prec]["e_rel"] * np.abs(ref) / spec.nk)
            assert np.all(err < allowed), (spec.grid, prec, i, err, allowed)
    grp.close()
    for s_ in sys_:
        s_.close()


@pytest.mark.parametrize("members,shared", [(MEMBERS, 0), (MIXED, 2), (MIXED, 1)],
                         ids=["streams", "shared_taylor", "shared_all"])
def test_group_block_equals_member_blocks(members, shared):
    from paper_2003_09468_gb300 import KPointGroup
    nsteps, seed = 4, 99

    def run(grouped):
        sys_ = [make(spec, prec)[0] for spec, prec in members]
        st = [state(spec) for spec, _ in members]
        xs = [torch.empty(s_.field_shape, dtype=torch.float64, device="cuda") for s_ in sys_]
        eh = [torch.empty((2, spec.nwalkers, 3), dtype=torch.complex128, device="cuda") for spec, _ in members]
        cs = [torch.tensor([7 * i], dtype=torch.int64, device="cuda") for i in range(len(members))]
        if grouped:
            grp = KPointGroup(sys_)
            grp.shared = shared
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
