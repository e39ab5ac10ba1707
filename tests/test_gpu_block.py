"""Device field generator, comb and block driver against the CPU restatement.

* Philox4x32-10 words bit for bit (known answers and random counters).
* Fields within the Box-Muller error bound of fp32 logf / sqrtf / sincospif:
  every intrinsic is within 1 ulp (sqrtf exact), so |z_gpu - z_cpu| <= 4 ulp of r.
* The comb's indices, weights and walkers bit for bit (fp64 running sums on both
  sides in walker order, the same fp64 expression for the comb points).
* One block (afqmc_kp_block) bit for bit against the same calls made one by one, and
  a captured CUDA graph of a block bit for bit against eager blocks.
"""
import os

import numpy as np
import pytest

import gen
from oracle import rng

torch = pytest.importorskip("torch")
from gpu_util import dev, host, make  # noqa: E402

pytestmark = pytest.mark.gpu

SPEC = gen.SystemSpec(grid=(2, 2, 2), M=8, nocc=2, nchol=48, nwalkers=16, random_trial=True, seed=4)
SEED = 0x5EED_1234_ABCD_0001


def binding():
    from paper_2003_09468_gb300 import binding as b
    return b


def u32_to_i32(a):
    return np.asarray(a, dtype=np.uint64).astype(np.uint32).view(np.int32)


def test_philox_known_answers_on_device():
    golden = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    for line in open(golden):
        if line.startswith("#") or not line.strip():
            continue
        left, right = line.split("|")
        a = [int(v, 16) for v in left.split()]
        want = [int(v, 16) for v in right.split()]
        seed = a[4] | (a[5] << 32)
        out = host(binding().philox4x32_10(dev(u32_to_i32(np.array([a[:4]]))), seed))
        assert [int(v) for v in out.view(np.uint32)[0]] == want


def test_philox_words_match_oracle_bitwise():
    g = np.random.default_rng(3)
    ctr = g.integers(0, 2 ** 32, (5000, 4), dtype=np.uint64)
    seed = int(g.integers(0, 2 ** 63))
    out = host(binding().philox4x32_10(dev(u32_to_i32(ctr)), seed)).view(np.uint32)
    assert np.array_equal(out, rng.philox4x32_10(ctr, rng.key_of(seed)))
    empty = binding().philox4x32_10(torch.empty((0, 4), dtype=torch.int32, device="cuda"), seed)
    assert empty.shape == (0, 4)


@pytest.mark.parametrize("G", [48, 45])       # a field count that is not a multiple of four
def test_fields_match_oracle_and_advance_counter(G):
    spec = gen.SystemSpec(grid=(2, 2, 1), M=6, nocc=2, nchol=G, nwalkers=7, random_trial=True, seed=2)
    sys_, _ = make(spec, "mixed")
    counter = torch.tensor([41], dtype=torch.int64, device="cuda")
    x = sys_.fields(counter, SEED)
    x2 = sys_.fields(counter, SEED)
    got, got2, c = host(x), host(x2), int(host(counter)[0])
    assert c == 43
    shape = sys_.field_shape
    for val, cnt in ((got, 41), (got2, 42)):
        want = rng.fields(SEED, cnt, shape)
        F = int(np.prod(shape[1:]))
        w = rng.field_words(SEED, cnt, shape[0], F)
        r = np.concatenate([np.repeat(rng.box_muller(w[..., 0], w[..., 1])[2][..., None], 2, -1),
                            np.repeat(rng.box_muller(w[..., 2], w[..., 3])[2][..., None], 2, -1)],
                           axis=-1).reshape(shape[0], -1)[:, :F].reshape(shape)
        assert np.all(np.abs(val - want) <= 4 * 2.0 ** -23 * np.maximum(r, 1.0))
        assert np.all(val.astype(np.float32).astype(np.float64) == val)   # fp32 values
    assert not np.array_equal(got, got2)
    sys_.close()


def comb_case(weights, precision="mixed"):
    sys_, _ = make(SPEC, precision)
    phi0 = gen.walkers(SPEC)
    phi, w = dev(phi0), dev(np.asarray(weights, dtype=np.float64))
    counter = torch.tensor([9], dtype=torch.int64, device="cuda")
    idx = sys_.comb(phi, w, counter, SEED)
    out = host(phi), host(w), host(idx), sys_.last_error(), int(host(counter)[0])
    sys_.close()
    return phi0, out


@pytest.mark.parametrize("kind", ["exponential", "sparse", "equal"])
def test_comb_matches_oracle_bitwise(kind):
    g = np.random.default_rng(8)
    W = SPEC.nwalkers
    w = {"exponential": g.exponential(size=W), "sparse": g.exponential(size=W) * (g.random(W) < 0.3),
         "equal": np.full(W, 0.37)}[kind]
    if w.sum() == 0:
        w[3] = 1.0
    phi0, (phi, wn, idx, err, c) = comb_case(w)
    ophi, ow, oidx = rng.comb(phi0, w, SEED, 9)
    assert np.array_equal(idx, oidx)
    assert np.array_equal(wn, ow)
    assert np.array_equal(phi, ophi)
    assert err == (0, 0) and c == 9          # the comb does not advance the counter


@pytest.mark.parametrize("bad", ["zero", "nan"])
def test_comb_rejects_unusable_total(bad):
    w = np.zeros(SPEC.nwalkers) if bad == "zero" else np.r_[np.nan, np.ones(SPEC.nwalkers - 1)]
    phi0, (phi, wn, idx, err, _) = comb_case(w)
    assert np.array_equal(phi, phi0)
    assert np.array_equal(wn, w, equal_nan=True)
    assert list(idx) == list(range(SPEC.nwalkers))
    assert err[0] == 1                        # AFQMC_ERR_INVALID from the sticky flags


def run_block(precision, how, nsteps=4, qr_period=2, blocks=2, energy_period=1):
    """Final (phi, weight, eloc history, weight history, counter) of `blocks` blocks."""
    nmeas = -(-nsteps // energy_period)
    sys_, _ = make(SPEC, precision)
    phi = dev(gen.walkers(SPEC))
    w = torch.ones(SPEC.nwalkers, dtype=torch.float64, device="cuda")
    x = torch.empty(sys_.field_shape, dtype=torch.float64, device="cuda")
    eh = torch.zeros((nmeas, SPEC.nwalkers, 3), dtype=torch.complex128, device="cuda")
    wh = torch.zeros((nsteps, SPEC.nwalkers), dtype=torch.float64, device="cuda")
    counter = torch.tensor([100], dtype=torch.int64, device="cuda")
    hist = []
    if how == "calls":
        for _ in range(blocks):
            for s in range(nsteps):
                sys_.fields(counter, SEED, x)
                measure = (s + 1) % energy_period == 0 or s == nsteps - 1
                sys_.step(phi, x, w, eh[s // energy_period] if measure else None,
                          do_qr=((s + 1) % qr_period == 0 or s == nsteps - 1), reuse=s > 0, energy=measure)
                wh[s].copy_(w)
            sys_.comb(phi, w, counter, SEED)
            hist.append((host(eh).copy(), host(wh).copy()))
    elif how == "block":
        for _ in range(blocks):
            sys_.block(phi, w, x, eh, counter, SEED, nsteps=nsteps, qr_period=qr_period,
                       energy_period=energy_period, weight_hist=wh)
            hist.append((host(eh).copy(), host(wh).copy()))
    else:
        # one eager block on a throwaway handle sets the kernels' one-time attributes first
        warm, _ = make(SPEC, precision)
        warm.block(phi.clone(), w.clone(), torch.empty_like(x), torch.empty_like(eh), counter.clone(), SEED,
                   nsteps=nsteps, qr_period=qr_period, energy_period=energy_period)
        torch.cuda.synchronize()
        warm.close()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            sys_.block(phi, w, x, eh, counter, SEED, nsteps=nsteps, qr_period=qr_period,
                       energy_period=energy_period, weight_hist=wh)
        for _ in range(blocks):
            g.replay()
            hist.append((host(eh).copy(), host(wh).copy()))
    out = host(phi), host(w), hist, int(host(counter)[0]), sys_.last_error()
    sys_.close()
    return out


@pytest.mark.parametrize("precision,energy_period", [("mixed", 1), ("fp64", 1), ("mixed", 3)])
def test_block_equals_calls_and_graph_replay(precision, energy_period):
    calls = run_block(precision, "calls", energy_period=energy_period)
    block = run_block(precision, "block", energy_period=energy_period)
    graph = run_block(precision, "graph", energy_period=energy_period)
    for other in (block, graph):
        assert np.array_equal(calls[0], other[0])
        assert np.array_equal(calls[1], other[1])
        for (ea, wa), (eb, wb) in zip(calls[2], other[2]):
            assert np.array_equal(ea, eb) and np.array_equal(wa, wb)
        assert other[3] == calls[3] == 100 + 2 * 4
        assert other[4] == (0, 0)
    # after the comb every weight equals the block's mean weight
    assert np.all(calls[1] == calls[1][0])
    assert calls[1][0] == pytest.approx(calls[2][-1][1][-1].mean(), rel=1e-14)
    assert np.all(np.isfinite(calls[2][-1][0]))
    # the two blocks drew different fields
    assert not np.array_equal(calls[2][0][0], calls[2][1][0])
