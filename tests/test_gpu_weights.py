"""GPU parity of the superparticle weights w_i of Eq. PIC (Sec. III.A).

Deterministic build: with an importance-sampled source (birth cell and bin
drawn from biased distributions, weight p/q per carrier, inherited by the
secondaries) the weighted densities, weighted fluxes, summed source weight,
per-slot weights, records and ledger are bit-identical to the oracle's, with
compaction, capacity drops, a running (unfinished) moment window, graph
replay and loaded carriers with a common weight.
"""
import numpy as np
import pytest

from oracle.oracle import OracleSim, REC_DTYPE, pack
from paper_1807_04733_gb300 import pic
from paper_1807_04733_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FLAGS = W.FLAG_DETERMINISTIC | W.FLAG_WEIGHTS


def biased(wl):
    for st in wl.stacks:
        z = np.arange(st.n_cells, dtype=np.float64)
        st.cell_bias = np.exp(z / 15.0)
        st.e_bias = np.arange(1, wl.n_e + 1, dtype=np.float64) ** 2
    return wl


def compare(wl, checkpoints, use_graph=False, set_recs=None, weights=None):
    ctx = pic.Context(wl, use_graph=use_graph)
    ref = OracleSim(wl)
    if set_recs is not None:
        recs, nid = set_recs
        ctx.set_records(recs, nid)
        ref.set_records(recs, nid)
        if weights is not None:
            ctx.set_weights(weights)
            ref.set_weights(weights)
    done = 0
    for cp in checkpoints:
        ctx.step(cp - done)
        assert ref.step(cp - done) == 0
        done = cp
        n, J, led = ctx.moments(0)
        rn, rJ, rled = ref.moments()
        assert led == rled, cp
        assert np.array_equal(n.cpu().numpy().view(np.uint32), rn), cp
        assert np.array_equal(J.cpu().numpy(), rJ), cp
        nw, Jw, wi = ctx.weighted_moments(0)
        rnw, rJw, rwi = ref.weighted_moments()
        assert wi == rwi, cp
        assert np.array_equal(nw.cpu().numpy().view(np.uint64), rnw), cp
        assert np.array_equal(Jw.cpu().numpy(), rJw), cp
        a, b = ctx.records(0), ref.records()
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), cp
        assert np.array_equal(ctx.weights(0), ref.weights()), cp
    ctx.close()
    return rled, rnw


def test_weights_bitexact_biased_source_through_capacity():
    wl = biased(W.config(0, scale=0.02, flags=FLAGS).replace(n_steps=260))
    led, nw = compare(wl, [1, 77, 150, 260])
    assert led["spawn_dropped"] > 0              # capacity was reached
    assert len(np.unique(nw[nw > 0] % (1 << 20))) > 10   # weights are not all whole


def test_weights_bitexact_spin_valve_running_window_and_graph():
    wl = biased(W.spin_valve(True, n0=20_000, capacity=90_000, n_steps=300, flags=FLAGS,
                             moment_every=3, compact_every=7))
    wl.stacks[0].excite_mask = 0b101
    compare(wl, [3, 100, 151, 300])              # 100 and 151 end inside a window
    compare(wl, [150, 300], use_graph=True)


def test_weights_loaded_carriers_keep_a_common_weight():
    """Loaded carriers all of weight 3: secondaries inherit it, so every
    weighted moment is three times the count (and equal to the oracle's)."""
    N = 30_000
    wl = W.bilayer(n0=0, capacity=120_000, n_steps=40, flags=FLAGS, compact_every=9)
    wl.stacks[0].tau_in *= 0.2
    rng = np.random.default_rng(8)
    r = np.zeros(N, REC_DTYPE)
    r["z"] = rng.uniform(0, 115, N).astype(np.float32)
    r["mu"] = rng.uniform(-1, 1, N).astype(np.float32)
    r["id"] = np.arange(N, dtype=np.uint32)
    r["packed"] = pack(rng.integers(2, 31, N), rng.integers(0, 2, N),
                       (r["z"] >= 15).astype(np.uint32), 1)
    w = np.full(N, 3 << 20, np.uint32)
    led, nw = compare(wl, [13, 40], set_recs=(r, N), weights=w)
    assert led["spawned"] > 1000


def test_weighted_moments_need_the_flag():
    wl = W.config(0, scale=0.01, flags=W.FLAG_DETERMINISTIC).replace(n_steps=10)
    ctx = pic.Context(wl)
    ctx.step(5)
    with pytest.raises(pic.PicError) as e:
        ctx.weighted_moments(0)
    assert e.value.status == 1
    ctx.close()
