"""Space-time maps derived from the moments on the host (Sec. V).

Post-processing of what ``pic_moments`` and ``pic_gen_moments`` return, as the
paper plots it; nothing here is part of the time step.

* ``p_hot``: the hot-carrier polarisation of Eq. hot_carrier_polarization,
  (n_up - n_down) / (n_up + n_down) per (output time, cell), the densities
  summed over the energy bins (every simulated carrier is a hot one: the
  grid starts at one bin above the Fermi level).
* ``mean_generation``: the mean generation label per (output time, cell) of
  Figs. 5(b) and 7(b),(d), the label sums divided by the carrier counts.
* ``spin_current``: the spin-current density of Eq. spincurrent per
  (output time, cell), (sum of v mu over up carriers - over down carriers)
  / dz, in carriers nm/fs per nm (the paper's factor -e and its units are
  left out), from the velocity moment of ``pic_vel_moments``.

Cells without carriers are NaN (the white regions of Figs. 5 and 7).
"""
from __future__ import annotations

import numpy as np


def _np(x):
    if hasattr(x, "detach"):                       # a torch tensor
        x = x.detach().cpu().numpy()
    return np.asarray(x)


def p_hot(n) -> np.ndarray:
    """n: densities [n_out][2][n_e][n_cells] (spin 0 = up); returns float64
    [n_out][n_cells]."""
    n = _np(n).astype(np.float64)
    up = n[:, 0].sum(axis=1)
    dn = n[:, 1].sum(axis=1)
    tot = up + dn
    out = np.full(tot.shape, np.nan)
    np.divide(up - dn, tot, out=out, where=tot > 0)
    return out


def mean_generation(g, n) -> np.ndarray:
    """g: label sums [n_out][n_cells]; n: densities [n_out][2][n_e][n_cells];
    returns float64 [n_out][n_cells]."""
    g = _np(g)
    if g.dtype == np.int64:                        # uint64 sums carried as int64
        g = g.view(np.uint64)
    g = g.astype(np.float64)
    cnt = _np(n).astype(np.float64).sum(axis=(1, 2))
    out = np.full(cnt.shape, np.nan)
    np.divide(g, cnt, out=out, where=cnt > 0)
    return out


def spin_current(v, dz: float) -> np.ndarray:
    """v: velocity sums [n_out][2][n_cells] in units of 2^-32 nm/fs; returns
    float64 [n_out][n_cells]."""
    v = _np(v).astype(np.float64)
    return (v[:, 0] - v[:, 1]) / (4294967296.0 * dz)
