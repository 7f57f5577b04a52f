"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle.

Deterministic build (PIC_F_DETERMINISTIC): particle records, integer
densities, integer fluxes, the generation map (Figs. 5(b), 7) and the ledger
must be bit-identical to the oracle's on the same seeded inputs.  Sizes span many tiles, several blocks
per look-back chain and ragged tails; edge cases cover empty inputs, a
single carrier, a full buffer, strict capacity and batched stacks.
"""
import math

import numpy as np
import pytest

from oracle.oracle import OracleSim, REC_DTYPE, pack, unpack
from paper_1807_04733_gb300 import pic
from paper_1807_04733_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DET = W.FLAG_DETERMINISTIC


def same_records(a, b):
    return len(a) == len(b) and np.array_equal(a.view(np.uint32), b.view(np.uint32))


def compare_run(wl, checkpoints, hist_mode=0, stacks=None, set_recs=None, dep_warps=None,
                event_pass=0):
    """Step the GPU context and the oracle to each checkpoint and compare.
    A single-stack context runs its ordinary steps with the general step
    inside the streaming pass unless event_pass is 1."""
    ctx = pic.Context(wl, hist_mode=hist_mode, event_pass=event_pass)
    fused = ctx.launch_config()["grid_step_fused"]
    assert (fused > 0) == (len(wl.stacks) == 1 and event_pass == 0)
    if dep_warps is not None:
        assert ctx.launch_config()["warps_step_moments"] == dep_warps
    idx = range(len(wl.stacks)) if stacks is None else stacks
    refs = {s: OracleSim(wl, stack=s) for s in idx}
    if set_recs is not None:
        for s, (recs, nid) in set_recs.items():
            ctx.set_records(recs, nid, stack=s)
            refs[s].set_records(recs, nid)
    done = 0
    for cp in checkpoints:
        ctx.step(cp - done)
        for s, ref in refs.items():
            assert ref.step(cp - done) == 0
        done = cp
        for s, ref in refs.items():
            n, J, led = ctx.moments(s)
            rn, rJ, rled = ref.moments()
            assert led == rled, (cp, s, led, rled)
            assert np.array_equal(n.cpu().numpy().view(np.uint32), rn), (cp, s)
            assert np.array_equal(J.cpu().numpy(), rJ), (cp, s)
            assert np.array_equal(ctx.gen_moments(s).cpu().numpy().view(np.uint64),
                                  ref.gen_moments()), (cp, s)
            assert same_records(ctx.records(s), ref.records()), (cp, s)
    ctx.close()
    return led


@pytest.mark.parametrize("rep,event_pass", [(0, 0), (1, 0), (2, 0), (0, 1)])
def test_det_bitexact_bilayer_through_capacity(rep, event_pass):
    wl = W.config(0, scale=0.02, flags=DET).replace(n_steps=300)
    led = compare_run(wl, [1, 40, 99, 100, 101, 180, 300], event_pass=event_pass)
    assert led["spawn_dropped"] > 0          # capacity was reached
    assert led["injected"] == 2000


@pytest.mark.parametrize("flags", [W.FLAG_NO_SECONDARIES, W.FLAG_TRANSPARENT,
                                   W.FLAG_LOWEST_BIN_ANY])
def test_det_bitexact_variants(flags):
    wl = W.config(0, scale=0.01, flags=DET | flags).replace(n_steps=200)
    compare_run(wl, [50, 200])


def test_det_bitexact_excitation_variant():
    """The excitation of Sec. III / Sec. V.A: homogeneous over the excited
    layers (abs_len = 0, both Fe layers of the spin valve), fixed energy per
    spin (e_mode = 1: majority 1.5 eV, minority 1.0 eV)."""
    wl = W.spin_valve(False, n0=20_000, capacity=90_000, n_steps=300, flags=DET)
    st = wl.stacks[0]
    st.abs_len = 0.0
    st.e_mode = W.E_MONO
    st.k_mono = (30, 20)
    st.excite_mask = 0b101
    compare_run(wl, [60, 150, 300])


@pytest.mark.parametrize("ap", [False, True])
def test_det_bitexact_spin_valve(ap):
    wl = W.spin_valve(ap, n0=20_000, capacity=90_000, n_steps=400, flags=DET,
                      moment_every=3, compact_every=7)
    compare_run(wl, [3, 151, 400])


def test_det_bitexact_warp_aggregated_histogram():
    wl = W.config(0, scale=0.02, flags=DET).replace(n_steps=150)
    compare_run(wl, [150], hist_mode=1)


@pytest.mark.parametrize("hist_mode", [0, 1])
def test_det_bitexact_large_histograms(hist_mode):
    """The large workload's grid (315 cells, 60 energy bins: 151 KB of
    density histogram) leaves room for one density-step block per SM, which
    then runs two groups of eight consumer warps sharing the histograms;
    densities every other step."""
    wl = W.config(4, scale=1e-4, flags=DET).replace(n_steps=120, moment_every=2,
                                                     compact_every=25)
    compare_run(wl, [2, 61, 120], hist_mode=hist_mode, dep_warps=16)


@pytest.mark.parametrize("rep", range(2))
def test_det_bitexact_batched_stacks(rep):
    wl = W.batched(n_stacks=6, scale=2e-3, n_steps=200, flags=DET)
    compare_run(wl, [1, 77, 200])


@pytest.mark.parametrize("event_pass", [0, 1])
def test_det_bitexact_many_tiles_and_blocks(event_pass):
    """1.2M carriers (hundreds of tiles, every block a multi-tile chunk) with
    fast scattering so that every tile spawns; ragged count (not a multiple
    of the 4-wide vectors or of the tile).  Every other step is ordinary (the
    general step inside the streaming pass, or in its own pass)."""
    N = 1_200_003
    wl = W.bilayer(n0=0, capacity=3_000_000, n_steps=12, flags=DET, compact_every=5,
                   moment_every=2)
    st = wl.stacks[0]
    st.tau_in *= 0.2
    rng = np.random.default_rng(21)
    r = np.zeros(N, REC_DTYPE)
    r["z"] = rng.uniform(0, 115, N).astype(np.float32)
    r["mu"] = rng.uniform(-1, 1, N).astype(np.float32)
    r["id"] = np.arange(N, dtype=np.uint32)
    k = rng.integers(1, 31, N)
    r["packed"] = pack(k, rng.integers(0, 2, N), (r["z"] >= 15).astype(np.uint32), 1)
    compare_run(wl, [1, 5, 12], set_recs={0: (r, N)}, event_pass=event_pass)


def test_edge_empty_and_single():
    wl = W.bilayer(n0=0, capacity=16, n_steps=20, flags=DET)
    ctx = pic.Context(wl)
    ctx.step(10)
    n, J, led = ctx.moments(0)
    assert int(n.abs().sum()) == 0 and int(J.abs().sum()) == 0
    assert led["particle_steps"] == 0 and len(ctx.records(0)) == 0
    one = np.zeros(1, REC_DTYPE)
    one["z"] = 14.9; one["mu"] = 0.7; one["packed"] = pack(30, 0, 0, 1)
    ref = OracleSim(wl)
    ref.set_step(0)
    ctx.close()
    compare_run(wl, [3, 20], set_recs={0: (one, 1)})


def test_edge_full_buffer_drops_every_secondary():
    N = 5000
    wl = W.bilayer(n0=0, capacity=N, n_steps=30, flags=DET)
    wl.stacks[0].tau_in *= 0.1
    rng = np.random.default_rng(2)
    r = np.zeros(N, REC_DTYPE)
    r["z"] = rng.uniform(0, 115, N).astype(np.float32)
    r["mu"] = rng.uniform(-1, 1, N).astype(np.float32)
    r["id"] = np.arange(N, dtype=np.uint32)
    r["packed"] = pack(rng.integers(2, 31, N), 0, (r["z"] >= 15).astype(np.uint32), 1)
    led = compare_run(wl, [30], set_recs={0: (r, N)})
    assert led["spawned"] == 0 and led["spawn_dropped"] > 0


def test_edge_strict_capacity_reports_error():
    wl = W.config(0, scale=0.01, flags=DET | W.FLAG_STRICT_CAPACITY).replace(n_steps=300)
    ctx = pic.Context(wl)
    ctx.step(300)
    with pytest.raises(pic.PicError) as e:
        ctx.moments(0)
    assert e.value.status == 3
    ctx.close()


def test_fast_build_conserves_exactly():
    """The default (fused multiply-add) build: exact conservation laws."""
    wl = W.config(0, scale=0.05).replace(n_steps=200)
    ctx = pic.Context(wl)
    for _ in range(4):
        ctx.step(50)
        n, J, led = ctx.moments(0)
        r = ctx.records(0)
        k = unpack(r["packed"])["k"]
        assert led["injected"] + led["spawned"] == (k > 0).sum() + led["absorbed"]
        assert led["q_injected"] == int(k.sum()) + led["q_bath"] + led["q_dropped"]
        t = ctx.shape(0)[2] - 1
        assert int(n[t].sum()) == int((k > 0).sum())
        # the generation map at the last instant is the live carriers' labels
        gen = unpack(r["packed"])["gen"]
        assert int(ctx.gen_moments(0)[t].sum()) == int(gen[k > 0].sum())
    ctx.close()


def test_det_bitexact_stack_base_shard():
    """A context holding stacks 2..4 of a batched workload with stack_base = 2
    (one rank's shard) reproduces those stacks of the oracle, which keys its
    random streams by the global stack index."""
    wl = W.batched(n_stacks=5, scale=2e-3, n_steps=120, flags=DET)
    part = wl.replace(stacks=list(wl.stacks[2:]))
    ctx = pic.Context(part, stack_base=2)
    ctx.step(120)
    for j in range(3):
        ref = OracleSim(wl, stack=2 + j)
        assert ref.step(120) == 0
        n, J, led = ctx.moments(j)
        rn, rJ, rled = ref.moments()
        assert led == rled
        assert np.array_equal(n.cpu().numpy().view(np.uint32), rn)
        assert np.array_equal(J.cpu().numpy(), rJ)
        assert np.array_equal(ctx.gen_moments(j).cpu().numpy().view(np.uint64), ref.gen_moments())
        assert same_records(ctx.records(j), ref.records())
    ctx.close()
