"""The allocation-free compaction entry point against the library's own.

pic_compact_static serves callers that cannot call cudaMalloc (an
application whose device memory belongs to its own allocator, or a loop
that must not allocate).  Its output must equal, bit for bit, the
compaction that pic_step performs inside a context on the same slots, on
two calls in a row (the second call runs on the scratch the first one left
behind).  This file
is collected last so that a failure here leaves every other test run.
"""
import numpy as np
import pytest

from oracle.oracle import REC_DTYPE, pack
from paper_1807_04733_gb300 import pic
from paper_1807_04733_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def soa_on_device(recs):
    n = len(recs)
    pad = (n + 3) // 4 * 4             # inputs are read in 4-wide vectors
    out = []
    for f, dt in (("z", torch.float32), ("mu", torch.float32), ("id", torch.int32),
                  ("packed", torch.int32)):
        host = np.zeros(pad, recs.dtype[f])
        host[:n] = recs[f]
        out.append(torch.from_numpy(host.view(np.int32) if dt == torch.int32 else host).cuda())
    return out


def compact_static(recs):
    n = len(recs)
    src = soa_on_device(recs)
    dst = [torch.empty_like(t) for t in src]
    torch.cuda.synchronize()
    alive = pic.pic_compact_static(*(t.data_ptr() for t in src), n,
                                   *(t.data_ptr() for t in dst),
                                   stream=torch.cuda.current_stream().cuda_stream)
    out = np.zeros(alive, REC_DTYPE)
    for t, f in zip(dst, ("z", "mu", "id", "packed")):
        out[f] = t[:alive].cpu().numpy().view(REC_DTYPE[f])
    return out


def library_compaction(wl, recs, next_id):
    """pic_step's own compaction of `recs`: a context whose step changes no
    carrier (no scattering, velocity 1e-30 nm/fs so z + v mu dt/2 rounds to
    z in float32) and that compacts after every step."""
    frozen = wl.replace(compact_every=1)
    st = frozen.stacks[0]
    st.tau_in[:] = np.inf
    st.tau_el[:] = np.inf
    st.v[:] = np.float32(1e-30)
    ctx = pic.Context(frozen)
    ctx.set_records(recs, next_id)
    ctx.step(1)
    out = ctx.records(0)
    ctx.close()
    return out


def test_compact_static_matches_pic_step_compaction_twice():
    N = 300_001
    wl = W.bilayer(n0=0, capacity=2_000_000, n_steps=4, flags=W.FLAG_DETERMINISTIC)
    st = wl.stacks[0]
    st.tau_in *= 0.1                   # many removals and secondaries per step
    rng = np.random.default_rng(31)
    r = np.zeros(N, REC_DTYPE)
    r["z"] = rng.uniform(0.5, 114.5, N).astype(np.float32)
    r["mu"] = rng.uniform(-1, 1, N).astype(np.float32)
    r["id"] = np.arange(N, dtype=np.uint32)
    k = rng.integers(1, 6, N)
    k[rng.random(N) < 0.2] = 0         # dead slots scattered through the input
    r["packed"] = pack(k, rng.integers(0, 2, N), (r["z"] >= 15).astype(np.uint32), 1)
    keeping = pic.Context(wl.replace(compact_every=1000))
    keeping.set_records(r, N)
    for call in range(2):
        keeping.step(1)               # a real step: removals, secondaries, moves
        raw = keeping.records(0)
        assert (raw["packed"] & 0xFF == 0).sum() > 1000     # there is work to do
        expect = library_compaction(wl, raw, 10 ** 7)
        got = compact_static(raw)
        assert len(got) == len(expect), call
        assert np.array_equal(got.view(np.uint32), expect.view(np.uint32)), call
    keeping.close()


def test_compact_static_rejects_sizes_beyond_its_scratch():
    with pytest.raises(pic.PicError) as e:
        pic.pic_compact_static(0, 0, 0, 0, 1 << 30, 0, 0, 0, 0)
    assert e.value.status == 1
