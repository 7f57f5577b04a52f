"""Pins of the superparticle weights w_i of Eq. PIC (Sec. III.A) in the oracle.

The paper represents the distribution as C * sum_i w_i delta(...) and adjusts
the weights "to improve the representation of less likely events"; the
reading built here is importance sampling of the source: a carrier is born
in cell i and bin k with the sampling probability q = q_cell(i) q_bin(k),
q proportional to p * bias, and carries w = p/q (in units of 2^-20), which a
secondary inherits from its parent.  Weighted moments count every carrier w
times.  The pins: unit weights give the counts times 2^20 exactly; a common
weight W on every carrier gives W times the counts (secondaries inherit);
each birth weight equals p/q computed here from the profile; the weighted
moments of the biased source have the expectation of the unbiased run
(with room for every carrier: a secondary dropped at capacity would bias
any estimator, weighted or not).
"""
import math

import numpy as np
from scipy import stats

from oracle.oracle import OracleSim, REC_DTYPE, pack, unpack
from paper_1807_04733_gb300 import workloads as W

UNIT = 1 << 20


def bilayer(n0=20_000, n_steps=150, flags=W.FLAG_WEIGHTS, seed=0, cap=None):
    wl = W.config(0, scale=n0 / 1e5, seed=seed, flags=flags).replace(n_steps=n_steps)
    if cap is not None:
        wl.stacks[0].capacity = cap
    return wl


def biased(wl):
    st = wl.stacks[0]
    z = np.arange(st.n_cells, dtype=np.float64)
    st.cell_bias = np.exp(z / 15.0)              # deep emitter cells over-sampled
    st.e_bias = np.arange(1, wl.n_e + 1, dtype=np.float64) ** 2   # high energies over-sampled
    return wl


def test_unit_weights_reproduce_counts():
    wl = bilayer()
    a = OracleSim(wl)
    b = OracleSim(wl, flags=0)
    assert a.step(wl.n_steps) == 0 and b.step(wl.n_steps) == 0
    assert np.array_equal(a.records().view(np.uint32), b.records().view(np.uint32))
    n, J, led = a.moments()
    nw, Jw, wi = a.weighted_moments()
    assert np.array_equal(nw, n.astype(np.uint64) * UNIT)
    assert np.array_equal(Jw, J.astype(np.int64) * UNIT)
    assert wi == led["injected"] * UNIT
    assert np.all(a.weights() == UNIT)


def test_secondaries_inherit_the_parent_weight():
    """Every loaded carrier weighs 3; with a strong cascade every secondary
    (and its secondaries) must weigh 3 as well."""
    wl = bilayer(n0=0, n_steps=60, cap=200_000)
    st = wl.stacks[0]
    st.tau_in *= 0.1
    rng = np.random.default_rng(4)
    N = 20_000
    r = np.zeros(N, REC_DTYPE)
    r["z"] = rng.uniform(0, 115, N).astype(np.float32)
    r["mu"] = rng.uniform(-1, 1, N).astype(np.float32)
    r["id"] = np.arange(N, dtype=np.uint32)
    r["packed"] = pack(rng.integers(2, 31, N), rng.integers(0, 2, N),
                       (r["z"] >= 15).astype(np.uint32), 1)
    s = OracleSim(wl)
    s.set_records(r, N)
    s.set_weights(np.full(N, 3 * UNIT, np.uint32))
    assert s.step(wl.n_steps) == 0
    n, J, led = s.moments()
    nw, Jw, _ = s.weighted_moments()
    assert led["spawned"] > 10_000
    assert np.array_equal(nw, n.astype(np.uint64) * 3 * UNIT)
    assert np.array_equal(Jw, J.astype(np.int64) * 3 * UNIT)
    assert np.all(s.weights()[unpack(s.records()["packed"])["k"] > 0] == 3 * UNIT)


def birth_weight_tables(wl):
    """p/q of the birth cell and bin, from the absorption profile exp(-z/l)
    over the excited cells and the uniform energy distribution."""
    st = wl.stacks[0]
    cells = np.arange(st.layer_cells[0])            # the excited Fe layer
    m = st.abs_len * (np.exp(-cells / st.abs_len) - np.exp(-(cells + 1) / st.abs_len))
    p_c = m / m.sum()
    q_c = m * st.cell_bias[cells] / (m * st.cell_bias[cells]).sum()
    p_k = np.full(wl.n_e, 1.0 / wl.n_e)
    q_k = st.e_bias / st.e_bias.sum()
    return p_c / q_c, p_k / q_k, q_c, q_k


def test_birth_weights_are_p_over_q():
    wl = biased(bilayer(n0=60_000, n_steps=1, cap=60_000))
    st = wl.stacks[0]
    st.t0, st.fwhm = 0.5, 0.2                      # the whole pulse in the first step
    st.tau_in[:] = math.inf
    st.tau_el[:] = math.inf
    st.v[:] = np.float32(1e-9)                     # carriers stay where they are born
    s = OracleSim(wl)
    assert s.step(1) == 0
    r, w = s.records(), s.weights()
    u = unpack(r["packed"])
    cell = np.floor(r["z"]).astype(int)
    wc, wk, q_c, q_k = birth_weight_tables(wl)
    expect = wc[cell] * wk[u["k"] - 1] * UNIT
    assert np.all(np.abs(w.astype(np.float64) - expect) <= 0.5 + 1e-6 * expect)
    # the draws follow q: cells and bins chi-square against the biased law
    N = len(r)
    assert stats.chisquare(np.bincount(cell, minlength=15), N * q_c).pvalue > 1e-4
    assert stats.chisquare(np.bincount(u["k"] - 1, minlength=wl.n_e), N * q_k).pvalue > 1e-4
    # the summed weight estimates the number of physical carriers created:
    # E_q[w] = 1, Var_q[w] = sum p^2/q - 1 (cells and bins independent)
    e2 = ((wc ** 2) * q_c).sum() * ((wk ** 2) * q_k).sum()
    _, _, wi = s.weighted_moments()
    assert abs(wi / UNIT - N) <= 4 * math.sqrt(N * (e2 - 1))


def test_importance_sampled_source_is_unbiased():
    """16 seeds of the biased source against 16 other seeds of the physical
    one: the weighted spin densities per layer and window and the weighted
    interface flux have the same expectation (Welch statistic within 4 SE);
    the unweighted counts of the biased run do not (the weights matter)."""
    R = 16

    def summary(wl, seed):
        wl.stacks[0].capacity = 40 * wl.stacks[0].n0     # nothing is dropped
        s = OracleSim(wl, seed=seed)
        assert s.step(wl.n_steps) == 0
        assert s.moments()[2]["spawn_dropped"] == 0
        nw, Jw, _ = s.weighted_moments()
        n, J, _ = s.moments()
        t = slice(9, None, 10)                       # every 10th window
        out = []
        for arr in (nw.astype(np.float64) / UNIT, n.astype(np.float64)):
            fe = arr[t, 0, :, :15].sum(axis=(1, 2)) - arr[t, 1, :, :15].sum(axis=(1, 2))
            au = arr[t, :, :, 15:].sum(axis=(1, 2, 3))
            out.append(np.concatenate([fe, au]))
        out.append(np.cumsum((Jw[:, 0, 15] - Jw[:, 1, 15]).astype(np.float64) / UNIT)[t])
        return out

    plain = [summary(bilayer(), 100 + i) for i in range(R)]
    tilt = [summary(biased(bilayer()), 200 + i) for i in range(R)]
    def welch(a, b):
        a, b = np.array(a), np.array(b)
        se = np.sqrt(a.var(0, ddof=1) / R + b.var(0, ddof=1) / R)
        return (a.mean(0) - b.mean(0)) / np.maximum(se, 1e-9)
    zw = welch([p[0] for p in plain], [q[0] for q in tilt])
    zf = welch([p[2] for p in plain], [q[2] for q in tilt])
    assert np.all(np.abs(zw) <= 4.0), zw
    assert np.all(np.abs(zf) <= 4.0), zf
    # without the weights the tilted run's counts are far off
    zc = welch([p[1] for p in plain], [q[1] for q in tilt])
    assert np.abs(zc).max() > 8.0, zc
