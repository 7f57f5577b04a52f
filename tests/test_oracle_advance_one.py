"""or_advance_one (the oracle's single-carrier step used for sampled parity at
full size) reproduces the oracle's own full step carrier by carrier."""
import numpy as np

from oracle.oracle import OracleSim, unpack
from paper_1807_04733_gb300 import workloads as W


def test_advance_one_equals_full_step():
    wl = W.config(0, scale=0.05, flags=W.FLAG_DETERMINISTIC).replace(n_steps=200)
    sim = OracleSim(wl)
    sim.step(160)                       # past the pulse; no compaction at step 160
    before = sim.records()
    nid0 = sim.next_id
    sim.step(1)
    after = sim.records()
    one = OracleSim(wl, capacity=4)
    one.set_step(160)
    secs = []
    room = len(before) < wl.stacks[0].capacity
    for i, r in enumerate(before):
        out, sec = one.advance_one(r, i, room)
        assert out.tobytes() == after[i].tobytes(), i
        if sec is not None:
            secs.append(sec)
    new = after[len(before):]
    assert len(new) == len(secs) and len(secs) > 0
    mask = np.uint32(0x1FFFFF)          # k, spin, layer, gen
    for s, g in zip(secs, new):         # appended in parent slot order
        assert s["z"] == g["z"] and s["mu"] == g["mu"]
        assert (s["packed"] & mask) == (g["packed"] & mask)
    assert (unpack(new["packed"])["gen"] >= 2).all() and new["id"][0] == nid0 & 0xFFFFFFFF
