"""The host-side space-time maps (Sec. V) against the carriers themselves.

At an output instant the oracle's records are the carriers the densities
and label sums were taken from: counting them per cell by spin, and summing
their labels, must give P_hot (Eq. hot_carrier_polarization) and the mean
generation (Figs. 5(b), 7) exactly.
"""
import numpy as np

from oracle.oracle import OracleSim
from paper_1807_04733_gb300 import analysis
from paper_1807_04733_gb300 import workloads as W


def _run(flags=0, n_steps=150):
    wl = W.config(0, scale=0.05, flags=flags).replace(n_steps=n_steps)
    s = OracleSim(wl)
    assert s.step(wl.n_steps) == 0
    return wl, s


def _per_cell(wl, s):
    r = s.records()
    k = r["packed"] & 0xFF
    live = k > 0
    spin = (r["packed"] >> 8) & 1
    gen = (r["packed"] >> 13) & 0xFF
    nc = s.n_cells
    cell = np.minimum(np.floor(r["z"].astype(np.float32) / np.float32(wl.dz)).astype(np.int64), nc - 1)
    up = np.bincount(cell[live & (spin == 0)], minlength=nc).astype(np.float64)
    dn = np.bincount(cell[live & (spin == 1)], minlength=nc).astype(np.float64)
    gs = np.bincount(cell[live], weights=gen[live].astype(np.float64), minlength=nc)
    return up, dn, gs


def test_p_hot_last_instant_from_records():
    wl, s = _run()
    n, _, _ = s.moments()
    t = wl.n_steps // wl.moment_every - 1
    up, dn, _ = _per_cell(wl, s)
    tot = up + dn
    ph = analysis.p_hot(n)
    assert ph.shape == (s.n_out, s.n_cells)
    occ = tot > 0
    assert occ.any()
    assert np.array_equal(ph[t][occ], (up - dn)[occ] / tot[occ])
    assert np.all(np.isnan(ph[t][~occ]))
    assert np.all((ph[t][occ] >= -1) & (ph[t][occ] <= 1))


def test_mean_generation_last_instant_from_records():
    wl, s = _run()
    n, _, _ = s.moments()
    g = s.gen_moments()
    t = wl.n_steps // wl.moment_every - 1
    up, dn, gs = _per_cell(wl, s)
    occ = (up + dn) > 0
    mg = analysis.mean_generation(g, n)
    assert np.array_equal(mg[t][occ], gs[occ] / (up + dn)[occ])
    assert np.all(mg[t][occ] >= 1.0)


def test_mean_generation_is_one_without_secondaries():
    wl, s = _run(flags=W.FLAG_NO_SECONDARIES)
    n, _, _ = s.moments()
    mg = analysis.mean_generation(s.gen_moments(), n)
    occ = ~np.isnan(mg)
    assert occ.any() and np.all(mg[occ] == 1.0)


def test_spin_current_from_records():
    """With the velocity moment on, the spin current at an output instant
    equals (sum v mu of up carriers - of down carriers) / dz per cell,
    counted from the records with the velocity table (float64 sums)."""
    wl, s = _run(flags=W.FLAG_VELOCITY)
    t = wl.n_steps // wl.moment_every - 1
    js = analysis.spin_current(s.vel_moments(), wl.dz)
    r = s.records()
    k = (r["packed"] & 0xFF).astype(np.int64)
    live = k > 0
    spin = ((r["packed"] >> 8) & 1).astype(np.int64)
    layer = ((r["packed"] >> 9) & 0xF).astype(np.int64)
    st = wl.stacks[0]
    mat = np.asarray(st.layer_mat)[layer]
    v = st.v[mat, spin, np.maximum(k, 1) - 1].astype(np.float32)
    w = (v * r["mu"].astype(np.float32)).astype(np.float64)
    nc = s.n_cells
    cell = np.minimum(np.floor(r["z"].astype(np.float32) / np.float32(wl.dz)).astype(np.int64), nc - 1)
    sign = np.where(spin == 0, 1.0, -1.0)
    ref = np.bincount(cell[live], weights=(sign * w)[live], minlength=nc) / wl.dz
    # each carrier's term was truncated to 2^-32 nm/fs
    assert np.abs(js[t] - ref).max() <= live.sum() * 2.0 ** -32 / wl.dz + 1e-12
    assert np.abs(ref).max() > 1e-3
