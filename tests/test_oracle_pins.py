"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Each test targets a step of the method (Sec. III of arXiv:1807.04733) with a
result that does not come from the oracle itself: closed forms (survival,
ballistic flight, diffusion and the alpha(t) of Sec. IV), exact binomial laws
(interface transmission), an exact branching recurrence (the energy cascade
of Fig. 3's setting), exact conservation laws, scipy's normal CDF for the
pulse, and an independent brute-force tracer on a few particles.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle.oracle import OracleSim, REC_DTYPE, pack, unpack
from paper_1807_04733_gb300 import workloads as W

from .brute_tracer import Tracer

INF = math.inf


def slab(cells=10_000, n_e=30, dt=1.0, tau_in=INF, tau_el=INF, v=None, capacity=2_000_000,
         n_steps=100, moment_every=1, compact_every=1000, seed=0, flags=0, mat=W.MAT_AU):
    wl = W.infinite_slab(n_e=n_e, dt=dt, cells=cells, capacity=capacity, n_steps=n_steps,
                         moment_every=moment_every, compact_every=compact_every,
                         seed=seed, flags=flags, mat=mat)
    st = wl.stacks[0]
    st.tau_in[:] = tau_in
    st.tau_el[:] = tau_el
    if v is not None:
        st.v[:] = np.float32(v)
    return wl


def initial(n, z0, k, spin=0, layer=0, seed=1, mu=None):
    rng = np.random.default_rng(seed)
    r = np.zeros(n, REC_DTYPE)
    r["z"] = np.float32(z0)
    r["mu"] = rng.uniform(-1, 1, n).astype(np.float32) if mu is None else np.float32(mu)
    r["id"] = np.arange(n, dtype=np.uint32)
    r["packed"] = pack(k, spin, layer, 1)
    return r


def thr(p):
    if not p > 0:
        return 0
    return 0xFFFFFFFF if p >= 1 else min(int(math.floor(p * 2 ** 32)), 0xFFFFFFFF)


# ---------------------------------------------------------------------------
# P1: survival under a constant lifetime, exp(-t/tau) (scattering test, Sec. III)
# ---------------------------------------------------------------------------
def test_p1_survival_exponential():
    N, tau, n = 1_000_000, 30.0, 60
    wl = slab(tau_in=tau, tau_el=INF, n_steps=n)
    s = OracleSim(wl)
    s.set_records(initial(N, 5000.0, 1), N)
    assert s.step(n) == 0
    dens, _, led = s.moments()
    live = dens.sum(axis=(1, 2, 3)).astype(np.float64)
    t = np.arange(1, n + 1) * wl.dt
    surv = np.exp(-t / tau)                     # closed form, Sec. III scattering test
    se = np.sqrt(N * surv * (1 - surv))
    assert np.all(np.abs(live - N * surv) <= 4 * se + 1), np.max(np.abs(live - N * surv) / se)
    # the plausible slip p = dt/tau instead of 1 - exp(-dt/tau) would sit >10 SE away
    wrong = N * (1 - wl.dt / tau) ** np.arange(1, n + 1)
    assert abs(live[-1] - wrong[-1]) > 8 * se[-1]
    assert led["absorbed"] == N - live[-1] and led["q_bath"] == led["absorbed"]


# ---------------------------------------------------------------------------
# P2: ballistic flight with vacuum reflection and a transparent interface
# ---------------------------------------------------------------------------
def ballistic_reference(z, mu, t_total, edges, vel):
    """Event-driven flight in double precision: velocity vel[layer] * mu,
    mirror reflection at the two outer surfaces, transmission at interfaces."""
    lay = int(np.searchsorted(edges, z, side="right") - 1)
    lay = min(max(lay, 0), len(vel) - 1)
    t = t_total
    while t > 0:
        w = vel[lay] * mu
        zn = z + w * t
        if mu > 0 and zn > edges[lay + 1]:
            t -= (edges[lay + 1] - z) / w
            z = edges[lay + 1]
            if lay == len(vel) - 1:
                mu = -mu
            else:
                lay += 1
        elif mu < 0 and zn < edges[lay]:
            t -= (edges[lay] - z) / w
            z = edges[lay]
            if lay == 0:
                mu = -mu
            else:
                lay -= 1
        else:
            return zn, mu, lay
    return z, mu, lay


def test_p2_ballistic_front_and_reflection():
    n_steps = 120
    wl = W.bilayer(fe_nm=15, au_nm=35, n0=0, capacity=1000, n_steps=n_steps,
                   flags=W.FLAG_TRANSPARENT)
    st = wl.stacks[0]
    st.tau_in[:] = INF
    st.tau_el[:] = INF
    st.v[W.MAT_FE] = np.float32(0.9)
    st.v[W.MAT_AU] = np.float32(1.3)
    rng = np.random.default_rng(3)
    N = 400
    r = initial(N, 0, 5, seed=4)
    r["z"] = rng.uniform(0, 50, N).astype(np.float32)
    layers = (r["z"] >= 15).astype(np.uint32)
    r["packed"] = pack(5, 0, layers, 1)
    s = OracleSim(wl)
    s.set_records(r, N)
    assert s.step(n_steps) == 0
    out = s.records()
    edges = np.array([0.0, 15.0, 50.0])
    vel = [0.9, 1.3]
    ref = np.array([ballistic_reference(float(z), float(m), n_steps * wl.dt, edges, vel)
                    for z, m in zip(r["z"], r["mu"])])
    # float32 flight: a few ulps of 50 nm per half step at most
    tol = 2 * n_steps * 2 * np.spacing(np.float32(50.0))
    assert np.max(np.abs(out["z"] - ref[:, 0])) < tol
    assert np.all(np.sign(out["mu"]) == np.sign(ref[:, 1]))
    assert np.all(unpack(out["packed"])["layer"] == ref[:, 2])
    # front before the first reflection: max z = max z0 + v t for mu = 1
    wl2 = slab(cells=1000, v=1.0, n_steps=10)
    s2 = OracleSim(wl2)
    r2 = initial(3, 100.0, 3, mu=[0.5, 0.25, -0.5])
    r2["mu"] = np.array([0.5, 0.25, -0.5], np.float32)
    s2.set_records(r2, 3)
    s2.step(10)
    z = s2.records()["z"]
    assert np.allclose(z, [105.0, 102.5, 95.0], atol=1e-5)


# ---------------------------------------------------------------------------
# P3: transmitted fraction at a single interface ~ Binomial(N, T)
# ---------------------------------------------------------------------------
def test_p3_single_interface_binomial():
    n_e = 4
    wl = W.bilayer(fe_nm=20, au_nm=20, n0=0, capacity=200_000, n_e=n_e, n_steps=2)
    st = wl.stacks[0]
    st.tau_in[:] = INF
    st.tau_el[:] = INF
    st.v[:] = np.float32(0.5)
    # a distinct transmittance for every (direction, spin, energy): an index
    # slip in the table lookup changes the expected fraction
    for d in range(2):
        for sp in range(2):
            for k in range(n_e):
                st.T[0, d, sp, k] = 0.05 + 0.4 * d + 0.2 * sp + 0.08 * k
    groups, recs = [], []
    per = 6000
    nid = 0
    for d in range(2):
        for sp in range(2):
            for k in range(1, n_e + 1):
                r = initial(per, 0, k, spin=sp, seed=nid + 7)
                if d == 0:
                    r["z"] = np.float32(19.9); r["mu"] = np.float32(0.9)
                    r["packed"] = pack(k, sp, 0, 1)
                else:
                    r["z"] = np.float32(20.1); r["mu"] = np.float32(-0.9)
                    r["packed"] = pack(k, sp, 1, 1)
                r["id"] = np.arange(nid, nid + per, dtype=np.uint32)
                nid += per
                recs.append(r)
                groups.append((d, sp, k))
    recs = np.concatenate(recs)
    s = OracleSim(wl)
    s.set_records(recs, nid)
    assert s.step(1) == 0
    out = s.records()
    lay = unpack(out["packed"])["layer"]
    for g, (d, sp, k) in enumerate(groups):
        sl = slice(g * per, (g + 1) * per)
        crossed = (lay[sl] == 1) if d == 0 else (lay[sl] == 0)
        T = st.T[0, d, sp, k - 1]
        se = math.sqrt(per * T * (1 - T))
        assert abs(crossed.sum() - per * T) <= 4 * se, (d, sp, k, crossed.sum(), per * T)
    _, _, led = s.moments()
    assert led["iface_hits"] == len(recs)


# ---------------------------------------------------------------------------
# P4: diffusion: exact discrete MSD, and alpha(t) of Sec. IV (Fig. 2)
# ---------------------------------------------------------------------------
def exact_msd(n_steps, p, seg):
    """E[(z_n - z_0)^2] for half-step segments of length seg*mu_j where mu
    is redrawn (isotropically) with probability p at each mid-step point;
    Corr(mu_a, mu_b) = (1/3)(1-p)^(number of mid-step points between)."""
    m = 2 * n_steps
    a = np.arange(m)
    # mid-step point of step s sits between segments 2s and 2s+1
    nmid = (a + 1) // 2                      # mid points before segment a
    d = np.abs(nmid[:, None] - nmid[None, :])
    return seg * seg / 3.0 * np.sum((1.0 - p) ** d)


def test_p4_diffusion_msd_and_alpha():
    tau, v, dt, n = 30.0, 1.0, 0.5, 400
    N = 60_000
    wl = slab(cells=2000, dt=dt, tau_in=INF, tau_el=tau, v=v, n_steps=n, n_e=1)
    s = OracleSim(wl)
    z0 = 1000.0
    s.set_records(initial(N, z0, 1, seed=11), N)
    p = thr(-math.expm1(-dt / tau)) / 2 ** 32
    msd, msd_se, ts = [], [], []
    for chunk in range(8):
        s.step(n // 8)
        dz2 = (s.records()["z"].astype(np.float64) - z0) ** 2
        msd.append(dz2.mean()); msd_se.append(dz2.std() / math.sqrt(N))
        ts.append(s.step_index)
    for t, m, se in zip(ts, msd, msd_se):
        ex = exact_msd(t, p, v * dt / 2)
        assert abs(m - ex) <= 4 * se, (t, m, ex, se)
    # continuum limit: 2 v^2 tau^2/3 (t/tau - 1 + e^{-t/tau}), i.e. D = v^2 tau/3
    for t in ts:
        ex = exact_msd(t, p, v * dt / 2)
        T = t * dt
        cont = 2 * v * v * tau * tau / 3 * (T / tau - 1 + math.exp(-T / tau))
        assert abs(ex - cont) / cont < 0.03
    # alpha(t) from the oracle's MSD vs the closed form of Sec. IV (Weiss)
    T = np.array(ts) * dt
    lm, lt = np.log(msd), np.log(T)
    alpha_num = np.gradient(lm, lt)
    alpha_ref = T * (1 - np.exp(-T / tau)) / (T - tau * (1 - np.exp(-T / tau)))
    assert np.all(np.abs(alpha_num[1:-1] - alpha_ref[1:-1]) < 0.08), (alpha_num, alpha_ref)
    assert alpha_ref[0] > 1.6 and alpha_ref[-1] < 1.3   # ballistic -> diffusive


# ---------------------------------------------------------------------------
# P5: exact conservation of carriers and energy quanta, with capacity drops
# ---------------------------------------------------------------------------
def test_p5_conservation_with_drops():
    wl = W.config(0, scale=0.02)   # 2000 carriers, capacity 8000 -> drops happen
    wl = wl.replace(n_steps=260)
    s = OracleSim(wl)
    for _ in range(13):
        s.step(20)
        r = s.records()
        k = unpack(r["packed"])["k"]
        _, _, led = s.moments()
        assert led["injected"] + led["spawned"] == (k > 0).sum() + led["absorbed"]
        assert led["q_injected"] == int(k.sum()) + led["q_bath"] + led["q_dropped"]
    assert led["spawn_dropped"] > 0 and led["injected"] == 2000
    # elastic-only: sum of k never changes
    wl2 = slab(tau_in=INF, tau_el=5.0, n_steps=30)
    s2 = OracleSim(wl2)
    r0 = initial(5000, 5000.0, np.arange(5000) % 30 + 1)
    s2.set_records(r0, 5000)
    s2.step(30)
    assert unpack(s2.records()["packed"])["k"].sum() == unpack(r0["packed"])["k"].sum()


# ---------------------------------------------------------------------------
# P7: branching recurrence E[N_{n+1}] = A E[N_n] in an infinite medium
# ---------------------------------------------------------------------------
def cascade_matrix(P, Q, P0t, n_e):
    """Expected one-step transfer between (spin, k) states for exact integer
    thresholds: no event / elastic keep the state, inelastic at k=1 removes,
    inelastic at k>=2 sends the carrier to k' = 1 + floor(x (k-1) / 2^32) and
    creates a secondary at k - k' with spin up iff y < P0t."""
    S = 2 * n_e
    A = np.zeros((S, S))
    two32 = 2.0 ** 32
    pu = P0t / two32
    for s in range(2):
        for k in range(1, n_e + 1):
            src = s * n_e + k - 1
            p, q = P[s, k - 1] / two32, Q[s, k - 1] / two32
            A[src, src] += 1 - p * q
            if k == 1:
                continue
            for kp in range(1, k):
                # exact count of words x with floor(x (k-1) / 2^32) == kp - 1
                lo = -(-(kp - 1) * 2 ** 32 // (k - 1))
                hi = -(-kp * 2 ** 32 // (k - 1))
                w = (hi - lo) / two32
                A[s * n_e + kp - 1, src] += p * q * w
                ks = k - kp
                A[0 * n_e + ks - 1, src] += p * q * w * pu
                A[1 * n_e + ks - 1, src] += p * q * w * (1 - pu)
    return A


def test_p7_branching_recurrence():
    n_e, n, N, R = 12, 25, 3000, 16
    wl = slab(cells=4000, n_e=n_e, dt=1.0, n_steps=n, mat=W.MAT_FE, capacity=200_000)
    st = wl.stacks[0]
    e = 0.125 * np.arange(1, n_e + 1)
    st.tau_in[W.MAT_FE, 0] = 20.0 / e ** 2 * 0.05
    st.tau_in[W.MAT_FE, 1] = 5.0 / e ** 2 * 0.05
    st.tau_el[:] = 30.0
    counts = []
    for rep in range(R):
        s = OracleSim(wl, seed=100 + rep)
        k0 = np.full(N, n_e); sp0 = (np.arange(N) % 3 == 2).astype(np.uint32)
        r = initial(N, 2000.0, k0, spin=sp0, seed=rep)
        s.set_records(r, N)
        s.step(n)
        dens, _, _ = s.moments()
        counts.append(dens[-1].sum(axis=2).reshape(-1).astype(np.float64))
    tabs = s.tables()
    A = cascade_matrix(tabs["P_thr"][W.MAT_FE], tabs["Q_thr"][W.MAT_FE],
                       tabs["P0_thr"][W.MAT_FE], n_e)
    N0 = np.zeros(2 * n_e)
    N0[n_e - 1] = (np.arange(N) % 3 != 2).sum()
    N0[2 * n_e - 1] = (np.arange(N) % 3 == 2).sum()
    expect = np.linalg.matrix_power(A, n) @ N0
    counts = np.array(counts)
    # a bin with a few carriers per run is a rare-event count (Poisson in the
    # limit): over 16 runs its sample variance can fall far below that, so the
    # SE is floored at the Poisson value of the expected count
    var = np.maximum(counts.var(0, ddof=1), expect)
    mean, se = counts.mean(0), np.sqrt(var / R)
    ok = np.abs(mean - expect) <= 4 * se + 0.5
    assert ok.all(), (mean, expect, se)
    assert expect.sum() > 2 * N          # the cascade really multiplied carriers


# ---------------------------------------------------------------------------
# Source term: pulse schedule (scipy normal CDF), depth profile, spin, energy
# ---------------------------------------------------------------------------
def test_source_pulse_profile_and_draws():
    wl = W.bilayer(n0=200_000, capacity=400_000, n_steps=160)
    wl.stacks[0].tau_in[:] = INF
    wl.stacks[0].tau_el[:] = INF
    s = OracleSim(wl)
    inj = s.tables()["inj"]
    st = wl.stacks[0]
    assert inj.sum() == st.n0 and inj.min() >= 0
    sd = st.fwhm / (2 * math.sqrt(2 * math.log(2)))
    dist = stats.norm(st.t0, sd)
    t = np.arange(len(inj) + 1) * wl.dt / 2
    Fr = np.clip((dist.cdf(t) - dist.cdf(0)) / (dist.cdf(2 * st.t0) - dist.cdf(0)), 0, 1)
    assert np.all(np.abs(inj - st.n0 * np.diff(Fr)) <= 1.0 + 1e-6)
    # draws: run the pulse out with no scattering and look at the carriers' birth state
    s.step(1)            # one step: births in half steps 0 and 1
    s2 = OracleSim(wl)
    s2.step(160)
    r = s2.records()
    u = unpack(r["packed"])
    assert len(r) == st.n0 and np.all(u["gen"] == 1) and np.all(u["layer"] <= 1)
    N = len(r)
    up = (u["spin"] == 0).sum()
    assert abs(up - N * 2 / 3) <= 4 * math.sqrt(N * 2 / 9)
    kc = np.bincount(u["k"], minlength=31)[1:]
    assert stats.chisquare(kc).pvalue > 1e-4
    ids = np.sort(r["id"])
    assert np.array_equal(ids, np.arange(N, dtype=np.uint32))


def test_source_depth_profile():
    """Births follow exp(-z/15 nm) over the Fe cells only (absorption profile)."""
    wl = W.bilayer(n0=300_000, capacity=300_000, n_steps=1)
    st = wl.stacks[0]
    st.t0 = 0.5; st.fwhm = 0.2        # the whole pulse inside the first step
    st.tau_in[:] = INF; st.tau_el[:] = INF
    st.v[:] = np.float32(1e-9)        # carriers stay where they are born
    s = OracleSim(wl)
    s.step(1)
    z = s.records()["z"]
    assert z.max() <= 15.0 and z.min() >= 0.0
    edges = np.arange(16.0)
    cnt, _ = np.histogram(z, edges)
    lam = st.abs_len
    mass = np.exp(-edges[:-1] / lam) - np.exp(-edges[1:] / lam)
    exp_cnt = len(z) * mass / mass.sum()
    assert stats.chisquare(cnt, exp_cnt).pvalue > 1e-4


# ---------------------------------------------------------------------------
# Moments: density = histogram of live carriers, flux = net face crossings
# ---------------------------------------------------------------------------
def test_moments_density_and_flux_from_records():
    wl = W.bilayer(fe_nm=15, au_nm=40, n0=0, capacity=20_000, n_steps=40)
    st = wl.stacks[0]
    st.tau_in[:] = INF                # no secondaries, no removal: ids persist
    st.tau_el[:] = 8.0
    rng = np.random.default_rng(5)
    N = 5000
    r = initial(N, 0, rng.integers(1, 31, N), spin=rng.integers(0, 2, N), seed=6)
    r["z"] = rng.uniform(0, 55, N).astype(np.float32)
    r["packed"] = pack(unpack(r["packed"])["k"], unpack(r["packed"])["spin"],
                       (r["z"] >= 15).astype(np.uint32), 1)
    s = OracleSim(wl)
    s.set_records(r, N)
    prev = r.copy()
    for step in range(6):
        s.step(1)
        cur = s.records()
        dens, J, _ = s.moments()
        cell = lambda z: np.clip(np.floor(z).astype(int), 0, 54)
        u = unpack(cur["packed"])
        h = np.zeros((2, 30, 55), np.int64)
        np.add.at(h, (u["spin"], u["k"] - 1, cell(cur["z"])), 1)
        assert np.array_equal(dens[step], h)
        jj = np.zeros((2, 56), np.int64)
        a, b = cell(prev["z"]), cell(cur["z"])
        for sp, x, y in zip(u["spin"], a, b):
            if y > x: jj[sp, x + 1:y + 1] += 1
            if y < x: jj[sp, y + 1:x + 1] -= 1
        assert np.array_equal(J[step], jj)
        assert np.all(J[step][:, 0] == 0) and np.all(J[step][:, -1] == 0)
        prev = cur


# ---------------------------------------------------------------------------
# P6: brute force, a few particles traced by an independent implementation
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("flags", [0, W.FLAG_NO_SECONDARIES, W.FLAG_TRANSPARENT,
                                   W.FLAG_LOWEST_BIN_ANY])
def test_p6_brute_force_tracer(flags):
    wl = W.spin_valve(antiparallel=True, fe_nm=3, au_nm=4, n0=0, capacity=40,
                      n_steps=30, compact_every=7, flags=flags, seed=77)
    st = wl.stacks[0]
    st.tau_in *= 0.05                 # many inelastic events
    st.tau_el[:] = 6.0
    rng = np.random.default_rng(8)
    N = 8
    r = initial(N, 0, rng.integers(1, 31, N), spin=rng.integers(0, 2, N), seed=9)
    r["z"] = rng.uniform(0, 10, N).astype(np.float32)
    lay = np.searchsorted([3.0, 7.0], r["z"], side="right").astype(np.uint32)
    r["packed"] = pack(unpack(r["packed"])["k"], unpack(r["packed"])["spin"], lay, 1)
    r["packed"][0] = pack(1, 0, int(lay[0]), 1)
    s = OracleSim(wl)
    s.set_records(r, N)
    tr = Tracer(wl)
    tr.load(r, N)
    for step in range(30):
        s.step(1)
        tr.step()
        a, b = s.records(), tr.records()
        assert len(a) == len(b), step
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), step
    dens, J, led = s.moments()
    for (t, sp, k, c), v in tr.dens.items():
        assert dens[t, sp, k - 1, c] == v
    assert dens.sum() == sum(tr.dens.values())
    for (t, sp, f), v in tr.flux.items():
        assert J[t, sp, f] == v
    assert np.abs(J).sum() == sum(abs(v) for v in tr.flux.values())
    # generation map (Figs. 5(b), 7): the labels of the traced carriers
    g = s.gen_moments()
    for (t, c), v in tr.gens.items():
        assert g[t, c] == v
    assert int(g.sum()) == sum(tr.gens.values())
    if flags & W.FLAG_NO_SECONDARIES:
        assert np.array_equal(g, dens.sum(axis=(1, 2)).astype(np.uint64))
    assert led["absorbed"] == tr.counts["absorbed"]
    assert led["spawned"] == tr.counts["spawned"]
    assert led["iface_hits"] == tr.counts["iface"]
    if not flags & (W.FLAG_NO_SECONDARIES):
        assert led["spawned"] > 0


# ---------------------------------------------------------------------------
# Generation map (Figs. 5(b), 7(b),(d)): label sums against the densities
# ---------------------------------------------------------------------------
def test_generation_map_primaries_only_equals_density():
    """Without secondaries every carrier is a primary (label 1): the label sum
    of every (output time, cell) equals the carrier count there."""
    wl = W.config(0, scale=0.05, flags=W.FLAG_NO_SECONDARIES).replace(n_steps=120)
    s = OracleSim(wl)
    assert s.step(wl.n_steps) == 0
    dens, _, _ = s.moments()
    g = s.gen_moments()
    assert dens.sum() > 0
    assert np.array_equal(g, dens.sum(axis=(1, 2)).astype(np.uint64))


def test_generation_map_counts_secondaries():
    """With the cascade on, a secondary carries its parent's label + 1, so the
    label sum exceeds the count by at least the live secondaries, and the mean
    label rises over time as the cascade develops (Fig. 5(b))."""
    wl = W.config(0, scale=0.05).replace(n_steps=200)
    s = OracleSim(wl)
    assert s.step(wl.n_steps) == 0
    dens, _, _ = s.moments()
    g = s.gen_moments().astype(np.int64)
    n = dens.sum(axis=(1, 2)).astype(np.int64)
    recs = s.records()
    gen = (recs["packed"] >> 13) & 0xFF
    live = (recs["packed"] & 0xFF) > 0
    last = wl.n_steps // wl.moment_every - 1
    assert g[last].sum() == int(gen[live].sum())            # the final instant
    assert np.all(g >= n)
    assert g.sum() - n.sum() >= int(((gen >= 2) & live).sum())
    occupied = n.sum(axis=1) > 0                             # after the pulse starts
    mean = g.sum(axis=1)[occupied] / n.sum(axis=1)[occupied]
    assert mean[-1] > mean[0] >= 1.0


# ---------------------------------------------------------------------------
# Velocity moment behind the spin current (Eq. spincurrent, Sec. V)
# ---------------------------------------------------------------------------
def _ballistic_slab(n, seed):
    """Carriers in the middle of a 2 um slab with no scattering: no wall and
    no event within a few steps."""
    wl = W.infinite_slab(cells=2000, capacity=n, n_steps=4, moment_every=1,
                         flags=W.FLAG_VELOCITY, dt=0.5)
    st = wl.stacks[0]
    st.tau_in[:] = np.inf
    st.tau_el[:] = np.inf
    rng = np.random.default_rng(seed)
    r = initial(n, 0.0, rng.integers(1, wl.n_e + 1, n), spin=rng.integers(0, 2, n), seed=seed)
    r["z"] = rng.uniform(900.0, 1100.0, n).astype(np.float32)
    return wl, r


def test_velocity_moment_is_the_rate_of_the_first_moment():
    """d/dt sum z = sum v mu for free flights: the summed velocity moment at
    the end of step 0 times dt equals the summed displacement over step 1."""
    wl, r = _ballistic_slab(4000, 21)
    s = OracleSim(wl)
    s.set_records(r, len(r))
    assert s.step(1) == 0
    z0 = s.records()["z"].astype(np.float64)
    assert s.step(1) == 0
    z1 = s.records()["z"].astype(np.float64)
    v = s.vel_moments()
    rate = v[0].sum() / 2.0 ** 32                        # nm/fs, both spins
    disp = (z1 - z0).sum()
    scale = np.abs(z1 - z0).sum()
    assert scale > 100.0
    assert abs(disp - wl.dt * rate) <= 1e-4 * scale
    # each spin separately
    spin = (s.records()["packed"] >> 8) & 1
    for sg in (0, 1):
        d = (z1 - z0)[spin == sg].sum()
        assert abs(d - wl.dt * v[0, sg].sum() / 2.0 ** 32) <= 1e-4 * scale


def test_velocity_moment_mirror_symmetry():
    """Mirroring every direction cosine negates the velocity moment of each
    spin exactly (summed over cells: the carriers move the other way)."""
    wl, r = _ballistic_slab(3000, 22)
    a = OracleSim(wl)
    a.set_records(r, len(r))
    assert a.step(2) == 0
    m = r.copy()
    m["mu"] = -m["mu"]
    b = OracleSim(wl)
    b.set_records(m, len(m))
    assert b.step(2) == 0
    va, vb = a.vel_moments(), b.vel_moments()
    assert np.any(va[:2] != 0)
    assert np.array_equal(va[:2].sum(axis=2), -vb[:2].sum(axis=2))


def test_velocity_moment_off_without_the_flag():
    wl = W.config(0, scale=0.02).replace(n_steps=40)
    s = OracleSim(wl)
    assert s.step(40) == 0
    assert not s.vel_moments().any()


# ---------------------------------------------------------------------------
# Excitation variant of Sec. III ("Number of Particles") and Sec. V.A: carriers
# created homogeneously over the excited layers, at a fixed energy per spin
# (majority 1.5 eV, minority 1.0 eV above E_F)
# ---------------------------------------------------------------------------
def _mono_homogeneous_run(excite_mask, k_mono, n0=120_000):
    wl = W.spin_valve(False, fe_nm=10, au_nm=20, n0=n0, capacity=n0, n_steps=1)
    st = wl.stacks[0]
    st.t0 = 0.25; st.fwhm = 0.1          # the whole pulse inside the first 0.5 fs step
    st.tau_in[:] = INF; st.tau_el[:] = INF
    st.v[:] = np.float32(1e-9)           # carriers stay where they are born
    st.abs_len = 0.0                     # homogeneous in the excited layers
    st.e_mode = W.E_MONO
    st.k_mono = k_mono
    st.excite_mask = excite_mask
    s = OracleSim(wl)
    assert s.step(1) == 0
    return wl, s.records()


def test_excitation_homogeneous_fixed_energy_per_spin():
    # distinct bins per spin, so that a swapped index cannot pass: 1.5 eV
    # (k = 30) for the majority and 1.0 eV (k = 20) for the minority channel
    wl, r = _mono_homogeneous_run(0b101, (30, 20))
    st = wl.stacks[0]
    u = unpack(r["packed"])
    N = len(r)
    assert N == st.n0 and np.all(u["gen"] == 1)
    assert np.all(u["k"][u["spin"] == 0] == 30) and np.all(u["k"][u["spin"] == 1] == 20)
    up = int((u["spin"] == 0).sum())
    assert abs(up - N * 2 / 3) <= 4 * math.sqrt(N * 2 / 9)
    # births only in the two excited Fe layers (cells 0..9 and 30..39), each
    # cell equally likely; none in the Au spacer
    z = r["z"]
    assert np.all((z < 10.0) | (z >= 30.0)) and z.min() >= 0.0 and z.max() <= 40.0
    assert np.array_equal(u["layer"], np.where(z < 10.0, 0, 2).astype(np.uint32))
    cnt, _ = np.histogram(z, np.arange(41.0))
    assert np.all(cnt[10:30] == 0)
    exc = np.concatenate([cnt[:10], cnt[30:]])
    assert stats.chisquare(exc).pvalue > 1e-4
    # an exp(-z/15 nm) profile over the same cells would be rejected outright
    lam = 15.0
    zc = np.concatenate([np.arange(10.0), np.arange(30.0, 40.0)])
    m = np.exp(-zc / lam) - np.exp(-(zc + 1) / lam)
    assert stats.chisquare(exc, N * m / m.sum()).pvalue < 1e-12
    # the position inside a cell is uniform
    assert stats.kstest(z - np.floor(z), "uniform").pvalue > 1e-4


def test_excitation_variant_single_layer_and_equal_bins():
    # one excited layer (the collector only) and the same bin for both spins
    wl, r = _mono_homogeneous_run(0b100, (7, 7), n0=30_000)
    u = unpack(r["packed"])
    assert np.all(u["k"] == 7) and np.all(u["layer"] == 2)
    cnt, _ = np.histogram(r["z"], np.arange(30.0, 41.0))
    assert cnt.sum() == len(r) and stats.chisquare(cnt).pvalue > 1e-4
