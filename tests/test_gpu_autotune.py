"""The autotuner (pic_autotune) times launch configurations on the running
simulation; results must not depend on the configuration, so a tuned run is
bit-identical to an untuned one (deterministic build), and the kept
configuration is the fastest trial."""
import numpy as np
import pytest

from paper_1807_04733_gb300 import pic
from paper_1807_04733_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DET = W.FLAG_DETERMINISTIC


def test_autotune_keeps_results_and_picks_fastest():
    wl = W.spin_valve(False, n0=30_000, capacity=90_000, n_steps=1300, flags=DET,
                      moment_every=3, compact_every=7)
    plain = pic.Context(wl)
    tuned = pic.Context(wl, use_graph=True)
    plain.step(100)
    tuned.step(100)
    trials = tuned.autotune(6)
    assert len(trials) >= 4
    assert sum(t["chosen"] for t in trials) == 1
    # both shapes of the streaming pass were timed: 8 consumer warps with 4
    # slots per thread and 4 with 8
    assert {t["consumer_warps"] for t in trials} == {4, 8}
    # and the general step inside the streaming pass or in a pass of its own
    assert {t["event_pass"] for t in trials} == {0, 1}
    assert all(t["blocks_per_sm"] <= 3 for t in trials if t["event_pass"] == 0)
    best = min(trials, key=lambda t: t["ns_per_particle_step"])
    assert best["chosen"] == 1
    info = tuned.launch_config()
    assert info["ring_step"] == best["ring_stages"]
    assert info["warps_step"] == best["consumer_warps"]
    assert (info["grid_step_fused"] > 0) == (best["event_pass"] == 0)
    done = tuned.shape(0)[2]
    end = max(900, done)
    plain.step(done - 100)
    plain.step(end - done)
    tuned.step(end - done)
    n1, J1, l1 = plain.moments(0)
    n2, J2, l2 = tuned.moments(0)
    assert l1 == l2
    assert torch.equal(n1, n2) and torch.equal(J1, J2)
    r1, r2 = plain.records(0), tuned.records(0)
    assert np.array_equal(r1.view(np.uint32), r2.view(np.uint32))
    plain.close()
    tuned.close()


def test_autotune_refuses_without_steps_left():
    wl = W.config(0, scale=0.01, flags=DET).replace(n_steps=50)
    ctx = pic.Context(wl)
    with pytest.raises(pic.PicError) as e:
        ctx.autotune(10)
    assert e.value.status == 1
    ctx.close()
