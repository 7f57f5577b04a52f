"""GPU parity of the velocity moment behind the spin current (Eq. spincurrent).

The sums are integers (2^-32 nm/fs per carrier, truncated), so the
deterministic build must reproduce the oracle's bit for bit, with single
launches and with graph-replayed periods, for one stack and for several.
"""
import numpy as np
import pytest

from oracle.oracle import OracleSim
from paper_1807_04733_gb300 import pic
from paper_1807_04733_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FLAGS = W.FLAG_DETERMINISTIC | W.FLAG_VELOCITY


@pytest.mark.parametrize("graph", [False, True])
def test_velocity_moment_bitexact_bilayer(graph):
    wl = W.config(0, scale=0.05, flags=FLAGS).replace(n_steps=150, moment_every=5)
    ctx = pic.Context(wl, use_graph=graph)
    ref = OracleSim(wl)
    done = 0
    for cp in (50, 150):
        ctx.step(cp - done)
        assert ref.step(cp - done) == 0
        done = cp
        v = ctx.vel_moments(0).cpu().numpy()
        rv = ref.vel_moments()
        assert np.any(rv != 0)
        assert np.array_equal(v, rv), cp
        n, _, _ = ctx.moments(0)
        rn, _, _ = ref.moments()
        assert np.array_equal(n.cpu().numpy().view(np.uint32), rn)
    ctx.close()


def test_velocity_moment_bitexact_batched():
    wl = W.batched(n_stacks=3, scale=2e-3, n_steps=60, flags=FLAGS)
    ctx = pic.Context(wl)
    ctx.step(60)
    for s in range(3):
        ref = OracleSim(wl, stack=s)
        assert ref.step(60) == 0
        assert np.array_equal(ctx.vel_moments(s).cpu().numpy(), ref.vel_moments()), s
    ctx.close()


def test_velocity_moment_needs_the_flag():
    wl = W.config(0, scale=0.02, flags=W.FLAG_DETERMINISTIC).replace(n_steps=10)
    ctx = pic.Context(wl)
    ctx.step(10)
    with pytest.raises(pic.PicError):
        ctx.vel_moments(0)
    ctx.close()
