"""Fast (fused multiply-add) build against the oracle, statistically.

The fast build rounds the flight differently from the scalar float32 oracle,
which flips rare threshold and face decisions, so trajectories diverge and
the two are compared as distributions (the reading of the 4-SE criterion
over 16 seeds for ~10^6 bins): 16 independent seeds per side (disjoint seed
sets), on the Fe(15 nm)/Au(100 nm) bilayer with the pump pulse.

* coarse bins (spin, 5-nm slab, 10 time windows, all energies) of the
  density, and the spin flux through the interface and a few depth faces in
  the same windows: each bin's Welch t (SE from both sides' spreads) turned
  into a normal quantile with its Welch-Satterthwaite degrees of freedom;
  none beyond 5 and at most one of the ~540 beyond 4 (the 4-SE criterion
  with its multiplicity: under the null, P(two beyond 4) ~ 1e-3);
* the sum of squares of those quantiles against its permutation distribution
  (the 32 runs relabelled at random), which accounts for the correlation
  between bins of one run: p > 1e-3;
* fine (t, spin, k, cell) bins with mean count >= 30: at most 1e-3 of them
  outside 4 SE;
* a fine snapshot bin that is zero in all 16 runs of one side has at most 20
  carriers over the 16 runs of the other (structural zeros: energies above
  the pulse, depths not yet reached; with a Poisson mean m per run, "all 16
  zero" and "sum >= 21" have joint probability below e^-21, ~1e-4 over the
  ~7e4 bins);
* conservation laws hold exactly in every GPU run.
"""
import numpy as np
import pytest
from scipy import stats

from oracle.oracle import OracleSim
from paper_1807_04733_gb300 import pic
from paper_1807_04733_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R = 16
STEPS = 500
WIN = 50          # time steps per coarse window
SLAB = 5          # cells (nm) per coarse slab
FACES = (5, 10, 15, 20, 30, 60, 110)


def workload(seed):
    return W.config(0, scale=0.2, seed=seed).replace(n_steps=STEPS)


def reduce(n, J):
    """n [T][2][n_e][cells], J [T][2][cells+1] -> coarse and fine arrays."""
    T, _, ne, nc = n.shape
    nt = T // WIN
    dens = n.reshape(nt, WIN, 2, ne, nc).sum(axis=(1, 3)).astype(np.float64)
    dens = dens.reshape(nt, 2, nc // SLAB, SLAB).sum(axis=3)
    flux = J.reshape(nt, WIN, 2, nc + 1).sum(axis=1)[:, :, list(FACES)].astype(np.float64)
    fine = n[WIN - 1::WIN].astype(np.float64)           # one snapshot per window
    return dens, flux, fine


def calibrated_z(a, b):
    """Per column: Welch t of the two samples' means, as a normal quantile
    (same tail probability under Student t with the Welch-Satterthwaite
    degrees of freedom); 0 where both samples are constant."""
    ra, rb = a.shape[0], b.shape[0]
    va, vb = a.var(0, ddof=1) / ra, b.var(0, ddof=1) / rb
    v = va + vb
    live = v > 0
    t = (a.mean(0) - b.mean(0))[live] / np.sqrt(v[live])
    nu = v[live] ** 2 / (va[live] ** 2 / (ra - 1) + vb[live] ** 2 / (rb - 1))
    z = np.zeros(v.shape)
    z[live] = stats.norm.isf(stats.t.sf(np.abs(t), nu)) * np.sign(t)
    return z


def test_fast_build_matches_oracle_in_distribution():
    o_d, o_f, o_n, g_d, g_f, g_n = [], [], [], [], [], []
    for r in range(R):
        wl = workload(r)
        ref = OracleSim(wl)
        assert ref.step(STEPS) == 0
        n, J, _ = ref.moments()
        d, f, fn = reduce(n, J)
        o_d.append(d); o_f.append(f); o_n.append(fn)
    for r in range(R):
        wl = workload(1000 + r)
        ctx = pic.Context(wl)
        ctx.step(STEPS)
        n, J, led = ctx.moments(0)
        rec = ctx.records(0)
        k = rec["packed"] & 0xFF
        assert led["injected"] + led["spawned"] == (k > 0).sum() + led["absorbed"]
        assert led["q_injected"] == int(k.sum()) + led["q_bath"] + led["q_dropped"]
        d, f, fn = reduce(n.cpu().numpy().view(np.uint32), J.cpu().numpy())
        g_d.append(d); g_f.append(f); g_n.append(fn)
        ctx.close()

    og = np.concatenate([np.array(o_d).reshape(R, -1), np.array(o_f).reshape(R, -1)], axis=1)
    gg = np.concatenate([np.array(g_d).reshape(R, -1), np.array(g_f).reshape(R, -1)], axis=1)
    z = calibrated_z(og, gg)
    assert (np.abs(z) > 0).sum() > 300
    assert np.abs(z).max() <= 5 and (np.abs(z) > 4).sum() <= 1, np.sort(np.abs(z))[-5:]
    chi2 = float((z ** 2).sum())
    pool = np.concatenate([og, gg])
    rng = np.random.default_rng(0)
    n_perm, above = 2000, 0
    for _ in range(n_perm):
        i = rng.permutation(2 * R)
        above += float((calibrated_z(pool[i[:R]], pool[i[R:]]) ** 2).sum()) >= chi2
    assert (above + 1) / (n_perm + 1) > 1e-3, (chi2, above)

    a, b = np.array(o_n), np.array(g_n)
    for zero_side, other in ((a, b), (b, a)):
        only = (zero_side == 0).all(0)
        assert other.sum(0)[only].max(initial=0) <= 20
    ma, mb = a.mean(0), b.mean(0)
    se = np.sqrt(a.var(0, ddof=1) / R + b.var(0, ddof=1) / R)
    big = (ma >= 30) & (se > 0)
    frac = (np.abs(ma - mb)[big] > 4 * se[big]).mean()
    assert big.sum() > 1000 and frac <= 1e-3, (big.sum(), frac)
