"""Pins of the oracle's adjoint (score-function gradient) to closed forms.

The gradient of E[O], O = sum gn * n + sum gJ * J, with respect to the
inelastic lifetimes and the interface transmittances is estimated by the
oracle's two-pass replay (or_grad).  Each test below checks it against a
result that does not come from the oracle:

* exact identities that the estimator must satisfy sample by sample in
  settings where every score and every reward-to-go is known in closed form
  (survival: P1'; single interface, both as a density and as a flux: P3';
  one inelastic generation with secondaries: lineage totals);
* expectations in closed form within 4 standard errors (survival,
  elastic/inelastic channel choice, transmission);
* the exact cascade recurrence of an infinite medium (Fig. 3's setting)
  differentiated with torch float64 autograd (P7');
* central finite differences with common random numbers on a Fe/Au bilayer.
"""
import copy
import math
import os

import numpy as np
import pytest

from oracle.oracle import OracleSim, REC_DTYPE, pack, unpack
from paper_1807_04733_gb300 import workloads as W

from .test_oracle_pins import cascade_matrix, initial, slab

INF = math.inf


def zero_weights(s, wl):
    gn = np.zeros((s.n_out, 2, wl.n_e, s.n_cells), np.float32)
    gJ = np.zeros((s.n_out, 2, s.n_cells + 1), np.float32)
    return gn, gJ


# ---------------------------------------------------------------------------
# P1': survival under a constant lifetime.  With k = 1, tau_el = inf and O =
# N_live(n), a carrier alive at step n contributes n no-scattering scores
# dt/tau^2 times reward 1, a removed one nothing: grad = n dt/tau^2 N_live
# exactly, and E[grad] = N0 n (dt/tau^2) e^{-n dt/tau}.
# ---------------------------------------------------------------------------
def test_p1prime_survival_gradient():
    N, tau, n, dt = 200_000, 30.0, 20, 1.0
    wl = slab(tau_in=tau, tau_el=INF, n_steps=n, dt=dt)
    s = OracleSim(wl)
    s.set_records(initial(N, 5000.0, 1), N)
    s.step(n)
    dens, _, _ = s.moments()
    alive = int(dens[n - 1].sum())
    gn, gJ = zero_weights(s, wl)
    gn[n - 1] = 1.0
    g_tau, g_T, _, _ = s.grad(gn, gJ)
    m = W.MAT_AU
    c = dt / tau ** 2
    assert g_tau[m, 0, 0] == pytest.approx(n * c * alive, rel=1e-10)
    g_tau[m, 0, 0] = 0.0
    assert not g_tau.any() and not g_T.any()
    p = 1.0 - math.exp(-dt / tau)
    surv = (1.0 - p) ** n
    se = n * c * math.sqrt(N * surv * (1 - surv))
    assert abs(n * c * alive - N * n * c * math.exp(-n * dt / tau)) <= 4 * se


# ---------------------------------------------------------------------------
# Elastic/inelastic channel: k = 1 carriers with both channels and removal on
# an inelastic event survive a step with probability 1 - p q, p = 1 -
# e^{-dt (r_in + r_el)}, q = r_in / (r_in + r_el):
#   dE[N_n]/dtau_in = N0 n (1-pq)^{n-1} r_in^2 (dt e^{-dt r} q + p r_el / r^2)
# ---------------------------------------------------------------------------
def test_channel_scores_survival_gradient():
    N, n, R = 20_000, 10, 16
    ti, te, dt = 15.0, 10.0, 1.0
    wl = slab(n_e=3, tau_in=ti, tau_el=te, n_steps=n, mat=W.MAT_FE)
    est = []
    for rep in range(R):
        s = OracleSim(wl, seed=50 + rep)
        s.set_records(initial(N, 5000.0, 1, seed=rep), N)
        s.step(n)
        gn, gJ = zero_weights(s, wl)
        gn[n - 1] = 1.0
        g, _, _, _ = s.grad(gn, gJ)
        est.append(g[W.MAT_FE, 0, 0])
    est = np.array(est)
    ri, re_ = 1 / ti, 1 / te
    r = ri + re_
    p, q = -math.expm1(-dt * r), ri / r
    expect = N * n * (1 - p * q) ** (n - 1) * ri ** 2 * (dt * math.exp(-dt * r) * q + p * re_ / r ** 2)
    se = est.std(ddof=1) / math.sqrt(R)
    assert abs(est.mean() - expect) <= 4 * se, (est.mean(), expect, se)


# ---------------------------------------------------------------------------
# P3': one interface, no scattering.  Carriers just below the Fe/Au interface
# moving up are transmitted with probability T[0][up][spin][k].  For O = the
# carriers in Au after one step (or the flux through the interface face) a
# transmitted carrier contributes 1/T and a reflected one nothing:
# grad_T = N_trans / T entry by entry, zero elsewhere; E[grad_T] = N.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("up", [True, False])
def test_p3prime_interface_gradient(up):
    wl = W.bilayer(n0=0, capacity=100_000, n_steps=5, moment_every=1)
    st = wl.stacks[0]
    st.tau_in[:] = INF
    st.tau_el[:] = INF
    nc0 = st.layer_cells[0]
    zi = float(nc0) * wl.dz
    N = 50_000
    rng = np.random.default_rng(3 if up else 4)
    r = np.zeros(N, REC_DTYPE)
    r["z"] = np.float32(zi - 0.01 if up else zi + 0.01)
    mu = rng.uniform(0.5, 1.0, N).astype(np.float32)
    r["mu"] = mu if up else -mu
    r["id"] = np.arange(N, dtype=np.uint32)
    k = rng.integers(1, wl.n_e + 1, N)
    sp = rng.integers(0, 2, N)
    r["packed"] = pack(k, sp, 0 if up else 1, 1)
    s = OracleSim(wl)
    s.set_records(r, N)
    s.step(1)
    u = unpack(s.records()["packed"])
    dest = 1 if up else 0
    d = 0 if up else 1
    moved = u["layer"] == dest
    ntr = np.zeros((2, wl.n_e))
    np.add.at(ntr, (u["spin"][moved], u["k"][moved] - 1), 1)
    T = st.T[0, d]
    for kind in ("density", "flux"):
        gn, gJ = zero_weights(s, wl)
        if kind == "density":
            if up:
                gn[0, :, :, nc0:] = 1.0
            else:
                gn[0, :, :, :nc0] = 1.0
        else:
            gJ[0, :, nc0] = 1.0 if up else -1.0
        g_tau, g_T, _, _ = s.grad(gn, gJ)
        assert np.allclose(g_T[0, d], ntr / T, rtol=1e-12, atol=1e-9), kind
        assert not g_T[0, 1 - d].any() and not g_tau.any()
    cnt = np.zeros((2, wl.n_e))
    np.add.at(cnt, (sp, k - 1), 1)
    se = math.sqrt((cnt * (1 - T) / T).sum())
    assert abs(g_T[0, d].sum() - N) <= 4 * se


# ---------------------------------------------------------------------------
# Lineage totals: k = 2 carriers, inelastic scattering only, one step.  A
# scattered carrier ends in k = 1 with a k = 1 secondary, so for O = N after
# the step its decision is weighted by 2 (its own count and its
# secondary's): grad = N_scat 2 s_scat + (N - N_scat) s_noscat exactly, with
# s_scat = -dt r^2 e^{-dt r} / p and s_noscat = dt r^2; E[grad] = N dp/dtau.
# ---------------------------------------------------------------------------
def test_secondary_lineage_gradient():
    N, tau, dt = 100_000, 3.0, 1.0
    wl = slab(n_e=4, tau_in=tau, tau_el=INF, n_steps=3, mat=W.MAT_FE)
    s = OracleSim(wl)
    s.set_records(initial(N, 5000.0, 2), N)
    s.step(1)
    _, _, led = s.moments()
    gn, gJ = zero_weights(s, wl)
    gn[0] = 1.0
    g_tau, _, _, _ = s.grad(gn, gJ)
    nsc = led["spawned"]
    a = dt / tau
    p = -math.expm1(-a)
    s_scat = -dt / tau ** 2 * math.exp(-a) / p
    s_no = dt / tau ** 2
    assert g_tau[W.MAT_FE, 0, 1] == pytest.approx(nsc * 2 * s_scat + (N - nsc) * s_no, rel=1e-10)
    g_tau[W.MAT_FE, 0, 1] = 0.0
    assert not g_tau.any()
    # E: N dp/dtau = -N dt/tau^2 e^{-a}; per-carrier variance p(1-p)(2 s_scat - s_no)^2
    se = math.sqrt(N * p * (1 - p)) * abs(2 * s_scat - s_no)
    assert abs(nsc * 2 * s_scat + (N - nsc) * s_no + N * dt / tau ** 2 * math.exp(-a)) <= 4 * se


# ---------------------------------------------------------------------------
# P7': the cascade recurrence E[N_{n+1}] = A(tau) E[N_n] of an infinite
# medium, with p and q as smooth functions of tau_in, differentiated by torch
# float64 autograd; the oracle's gradient averaged over 16 seeds agrees
# entry by entry within 4 SE.
# ---------------------------------------------------------------------------
def test_p7prime_cascade_gradient_autograd():
    torch = pytest.importorskip("torch")
    n_e, n, N, R = 8, 12, 3000, 16
    wl = slab(cells=4000, n_e=n_e, dt=1.0, n_steps=n, mat=W.MAT_FE, capacity=200_000)
    st = wl.stacks[0]
    e = 0.125 * np.arange(1, n_e + 1)
    st.tau_in[W.MAT_FE, 0] = 20.0 / e ** 2 * 0.05
    st.tau_in[W.MAT_FE, 1] = 5.0 / e ** 2 * 0.05
    st.tau_el[:] = 30.0
    wts = np.random.default_rng(7).uniform(-1, 1, (2, n_e))
    G = []
    for rep in range(R):
        s = OracleSim(wl, seed=100 + rep)
        k0 = np.full(N, n_e)
        sp0 = (np.arange(N) % 3 == 2).astype(np.uint32)
        s.set_records(initial(N, 2000.0, k0, spin=sp0, seed=rep), N)
        s.step(n)
        gn, gJ = zero_weights(s, wl)
        gn[n - 1] = wts[:, :, None]
        g, _, _, _ = s.grad(gn, gJ)
        G.append(g[W.MAT_FE])
    G = np.array(G)

    # the transfer matrix with the exact energy-split weights of the integer
    # map k' = 1 + floor(x (k-1) / 2^32) and the secondary spin threshold
    P0t = s.tables()["P0_thr"][W.MAT_FE]
    split = cascade_matrix(np.full((2, n_e), 2 ** 32), np.full((2, n_e), 2 ** 32), P0t, n_e)
    S = 2 * n_e
    # with p = q = 1 the diagonal is 1 - pq = 0 and the columns hold the split
    move = split.copy()
    np.fill_diagonal(move, 0.0)
    tau = torch.tensor(st.tau_in[W.MAT_FE], dtype=torch.float64, requires_grad=True)
    rin = 1.0 / tau
    rr = rin + 1.0 / 30.0
    pq = (-torch.expm1(-1.0 * rr) * (rin / rr)).reshape(-1)       # event rate per (spin, k)
    A = torch.eye(S, dtype=torch.float64) * (1 - pq)[None, :] + torch.tensor(move) * pq[None, :]
    v = torch.zeros(S, dtype=torch.float64)
    v[n_e - 1] = float((np.arange(N) % 3 != 2).sum())
    v[2 * n_e - 1] = float((np.arange(N) % 3 == 2).sum())
    for _ in range(n):
        v = A @ v
    (torch.tensor(wts.reshape(-1)) * v).sum().backward()
    expect = tau.grad.numpy()
    mean, se = G.mean(0), G.std(0, ddof=1) / math.sqrt(R)
    assert (np.abs(mean - expect) <= 4 * se + 1e-9).all(), (mean, expect, se)
    assert np.abs(expect).max() > 50        # the observable really depends on tau


# ---------------------------------------------------------------------------
# Central finite differences with common random numbers (same seed, so the
# same Philox words) on a Fe/Au bilayer with the pulse source: directional
# derivatives along tau_in and along T, for a spin-density window in Au and
# the spin flux through the interface face.
# ---------------------------------------------------------------------------
def test_finite_differences_common_random_numbers():
    R, h = 24, 0.1
    base = W.config(0, scale=0.02).replace(n_steps=150)
    st0 = base.stacks[0]

    def run(wl, seed):
        s = OracleSim(wl, seed=seed)
        s.step(wl.n_steps)
        n, J, _ = s.moments()
        return s, n, J

    d_tau, d_T = [], []
    for rep in range(R):
        s, n, J = run(base, rep)
        gn, gJ = zero_weights(s, base)
        gn[:, 0, :, 90:100] = 1.0
        gn[:, 1, :, 90:100] = -1.0
        gJ[:, 0, 15] = 1.0
        gJ[:, 1, 15] = -1.0
        g_tau, g_T, _, _ = s.grad(gn, gJ)

        def O(wl):
            _, n2, J2 = run(wl, rep)
            return float((gn * n2).sum() + (gJ * J2).sum())

        vals = []
        for f in (1 + h, 1 - h):
            wl = copy.deepcopy(base)
            wl.stacks[0].tau_in = st0.tau_in * f
            vals.append(O(wl))
        d_tau.append((vals[0] - vals[1]) / (2 * h) - (g_tau * st0.tau_in).sum())
        vals = []
        for f in (1 + h, 1 - h):
            wl = copy.deepcopy(base)
            wl.stacks[0].T = np.clip(st0.T * f, 0.0, 1.0)
            vals.append(O(wl))
        d_T.append((vals[0] - vals[1]) / (2 * h) - (g_T * st0.T).sum())
    for d in (np.array(d_tau), np.array(d_T)):
        assert abs(d.mean()) <= 3 * d.std(ddof=1) / math.sqrt(R), d


# ---------------------------------------------------------------------------
# The adjoint against central finite differences at a relative step of 1e-3
# with common random numbers, 2 SE over 16 seeds, compaction on (every 50
# steps).  With the random words keyed by slot, as in the library, a flipped
# decision that creates or removes a carrier renumbers every later slot, so
# at this step the two perturbed runs share almost no words (measured: the
# spread of the estimate is that of independent runs, sqrt(2) sd(O) / 2h,
# some 200 times the gradient).  The oracle's lineage keys (a carrier's words
# keyed by its birth, not its slot) keep every other carrier's words common.
# The direction perturbs every entry by 1e-3 of itself with the sign of the
# gradient of an independent pilot run, so that a few flips carry a signal;
# the test then can tell a wrong sign (the adjoint mean lies >= 2 SE from 0).
# ---------------------------------------------------------------------------
def _fd_seed(args):
    import copy as _copy
    import numpy as _np
    from oracle.oracle import OracleSim as _Sim
    rep, base, d_tau, d_T, gn, gJ, h = args
    st0 = base.stacks[0]

    def O(wl):
        s = _Sim(wl, seed=rep)
        s.step(wl.n_steps)
        n, J, _ = s.moments()
        return float((gn * n).sum() + (gJ * J).sum())

    s = _Sim(base, seed=rep)
    s.step(base.n_steps)
    g_tau, g_T, _, _ = s.grad(gn, gJ)
    out = []
    for d, field in ((d_tau, "tau_in"), (d_T, "T")):
        v = []
        for f in (h, -h):
            wl = _copy.deepcopy(base)
            setattr(wl.stacks[0], field, getattr(st0, field) + f * d)
            v.append(O(wl))
        g = g_tau if field == "tau_in" else g_T
        out.append(((v[0] - v[1]) / (2 * h), float((g * d).sum())))
    return out


def test_finite_differences_step_1e3_lineage_crn_with_compaction():
    import multiprocessing as mp
    R, h = 16, 1e-3
    base = W.config(3, scale=0.004, flags=W.FLAG_LINEAGE_KEYS).replace(n_steps=150,
                                                                        compact_every=50)
    st0 = base.stacks[0]
    st0.capacity = 40 * st0.n0             # nothing is dropped: no coupling through the slots
    pilot = OracleSim(base, seed=10_000)
    pilot.step(base.n_steps)
    gn, gJ = zero_weights(pilot, base)
    gn[:, 0, :, 90:100] = 1.0
    gn[:, 1, :, 90:100] = -1.0
    gJ[:, 0, 15] = 1.0
    gJ[:, 1, 15] = -1.0
    pt, pT, _, _ = pilot.grad(gn, gJ)
    d_tau = np.sign(pt) * st0.tau_in
    d_T = np.sign(pT) * st0.T
    args = [(rep, base, d_tau, d_T, gn, gJ, h) for rep in range(R)]
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        rows = pool.map(_fd_seed, args)
    for j in range(2):
        fd = np.array([r[j][0] for r in rows])
        ad = np.array([r[j][1] for r in rows])
        d = fd - ad
        se = d.std(ddof=1) / math.sqrt(R)
        assert abs(d.mean()) <= 2 * se, (j, d.mean(), se)
        assert ad.mean() >= 2 * se, (j, ad.mean(), se)      # a flipped sign would fail
    # an independent check of the run: no carrier was dropped
    assert pilot.moments()[2]["spawn_dropped"] == 0
