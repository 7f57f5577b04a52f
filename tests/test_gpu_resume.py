"""Checkpoint and resume (pic_save / pic_load): stepping on from a restored
state gives the uninterrupted run bit for bit (deterministic build), for the
pulse-driven bilayer (single launches and graph-replayed periods), batched
stacks with superparticle weights and velocity moments, and the adjoint
replayed after a resume equals the uninterrupted run's.  A checkpoint is
refused by a context with other parameters or excitation."""
import numpy as np
import pytest

from paper_1807_04733_gb300 import pic
from paper_1807_04733_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DET = W.FLAG_DETERMINISTIC


def state(ctx, wl):
    out = []
    for s in range(len(wl.stacks)):
        n, J, led = ctx.moments(s)
        out += [n.cpu().numpy(), J.cpu().numpy(), led, ctx.records(s).view(np.uint32),
                ctx.gen_moments(s).cpu().numpy()]
        if wl.flags & W.FLAG_WEIGHTS:
            nw, Jw, wi = ctx.weighted_moments(s)
            out += [nw.cpu().numpy(), Jw.cpu().numpy(), wi, ctx.weights(s)]
        if wl.flags & W.FLAG_VELOCITY:
            out.append(ctx.vel_moments(s).cpu().numpy())
    return out


def same(a, b):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        if isinstance(x, np.ndarray):
            assert np.array_equal(x, y)
        else:
            assert x == y


def resume_equals_straight(wl, total, cut, **kw):
    straight = pic.Context(wl, **kw)
    straight.step(total)
    ref = state(straight, wl)
    first = pic.Context(wl, **kw)
    first.step(cut)
    blob = first.save()
    first.close()
    second = pic.Context(wl, **kw)
    second.load(blob)
    assert second.shape(0)[2] == cut
    second.step(total - cut)
    same(state(second, wl), ref)
    return straight, second


@pytest.mark.parametrize("graph", [False, True])
def test_resume_bilayer_through_the_pulse(graph):
    wl = W.config(0, scale=0.02, flags=DET).replace(n_steps=200)
    a, b = resume_equals_straight(wl, 200, 73, use_graph=graph)   # mid-pulse, mid-period
    a.close()
    b.close()


def test_resume_batched_weights_velocity():
    wl = W.batched(n_stacks=4, scale=2e-3, n_steps=150,
                   flags=DET | W.FLAG_WEIGHTS | W.FLAG_VELOCITY).replace(moment_every=4, compact_every=9)
    for st in wl.stacks:
        st.e_bias = np.arange(1, wl.n_e + 1, dtype=np.float64)
    a, b = resume_equals_straight(wl, 150, 61)
    a.close()
    b.close()


def test_adjoint_after_resume():
    wl = W.config(0, scale=0.01, flags=DET).replace(n_steps=120)
    a, b = resume_equals_straight(wl, 120, 50)
    nc, no, _ = a.shape(0)
    gn = torch.zeros((1, no, 2, wl.n_e, nc), dtype=torch.float32, device="cuda")
    gJ = torch.zeros((1, no, 2, nc + 1), dtype=torch.float32, device="cuda")
    gn[0, :, 0, :, 90:100] = 1.0
    gJ[0, :, 1, 15] = -1.0
    ga = [g.cpu().numpy() for g in a.grad(gn, gJ)]
    gb = [g.cpu().numpy() for g in b.grad(gn, gJ)]
    for x, y in zip(ga, gb):
        assert np.allclose(x, y, rtol=1e-12, atol=1e-12)
    a.close()
    b.close()


def test_load_refuses_another_run():
    wl = W.config(0, scale=0.01, flags=DET).replace(n_steps=40)
    a = pic.Context(wl)
    a.step(10)
    blob = a.save()
    other = pic.Context(wl.replace(dt=0.5))
    with pytest.raises(pic.PicError) as e:
        other.load(blob)
    assert e.value.status == 1
    wl2 = W.config(0, scale=0.01, flags=DET).replace(n_steps=40)
    wl2.stacks[0].n0 += 1                    # another excitation
    c = pic.Context(wl2)
    with pytest.raises(pic.PicError):
        c.load(blob)
    with pytest.raises(pic.PicError):
        a.load(blob[:-8])                    # truncated
    for x in (a, other, c):
        x.close()
