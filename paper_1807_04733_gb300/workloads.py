"""Seeded synthetic inputs for the hot-electron superparticle step.

This module only *generates inputs*: layer stacks, physical material tables
(velocity v, inelastic lifetime tau_in, elastic lifetime tau_el, interface
transmittance T, equilibrium polarisation P0) and excitation-pulse parameters.
It holds none of the method's arithmetic: it derives no scattering
probability, threshold, injection count or particle update.  Both the CUDA
path (through the C-ABI) and the CPU oracle consume exactly what is built
here, so the two sides always see identical inputs.

The paper's ab-initio tables (its Fig. 1: velocities, lifetimes and Fe/Au
transmittances) are not available, so synthetic tables with the same shape
stand in for them:

* energy grid E_k = k * dE above E_F, k = 1..N_E;
* v(E) rising linearly from 0.2 to 1.4 nm/fs over the grid (Sec. V gives
  0.5-1 nm/fs for Fe majority carriers around 1-1.5 eV);
* Fermi-liquid lifetimes tau_in = tau0 / (E - E_F)^2 with tau0 = 20 (Fe
  majority), 5 (Fe minority) and 50 (Au) fs eV^2;
* tau_el = 30 fs in Fe and Au (Sec. II, elastic scattering);
* T_up = 0.7 + 0.2 x, T_dn = 0.4 + 0.2 x with x = (k-1)/(N_E-1): the majority
  channel transmits better (Sec. V.A);
* P0 = +1/3 in Fe (2:1 majority excitation), 0 in Au (Eq. eq_pol, Sec. III).

An antiparallel (AP) Fe layer is the material ``FE_AP`` whose spin-resolved
tables are the Fe tables with the spin index swapped.
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

MAT_FE, MAT_AU, MAT_FE_AP = 0, 1, 2
N_MAT = 3
MAT_NAMES = ("Fe", "Au", "Fe_AP")

# Flags shared by the C-ABI (pic_params.flags) and the oracle.
FLAG_DETERMINISTIC = 1      # CUDA path: no fused multiply-add in the flight
FLAG_NO_SECONDARIES = 2     # Sec. V.A variant (3): no secondary generation
FLAG_TRANSPARENT = 4        # Sec. V.A variant (2): T == 1 at every interface
FLAG_LOWEST_BIN_ANY = 8     # remove a lowest-bin carrier on ANY scattering event
FLAG_STRICT_CAPACITY = 16   # capacity overflow is an error instead of drop-and-count
FLAG_VELOCITY = 32          # also sum the velocities v*mu per (time, spin, cell)
FLAG_WEIGHTS = 64           # superparticle weights w_i (importance-sampled source)
# oracle only: random words keyed by lineage instead of slot (common random
# numbers for finite differences); the library keys by slot
FLAG_LINEAGE_KEYS = 128

E_UNIFORM = 0               # injected energy uniform over the N_E bins
E_MONO = 1                  # injected energy fixed per spin (k_mono[spin])

TAU0_FS_EV2 = {             # tau_in = tau0 / E^2
    (MAT_FE, 0): 20.0, (MAT_FE, 1): 5.0,
    (MAT_AU, 0): 50.0, (MAT_AU, 1): 50.0,
    (MAT_FE_AP, 0): 5.0, (MAT_FE_AP, 1): 20.0,
}
TAU_EL_FS = 30.0
P0 = (1.0 / 3.0, 0.0, -1.0 / 3.0)


@dataclass
class Stack:
    """One laterally homogeneous layer stack with its own tables and pulse."""
    layer_cells: list           # thickness of each layer in grid cells (dz each)
    layer_mat: list             # material id of each layer
    v: np.ndarray               # float32 [N_MAT][2][N_E]  nm/fs
    tau_in: np.ndarray          # float64 [N_MAT][2][N_E]  fs (inf = none)
    tau_el: np.ndarray          # float64 [N_MAT]          fs (inf = none)
    T: np.ndarray               # float64 [n_layers-1][2 dir][2 spin][N_E]
    p0: np.ndarray              # float64 [N_MAT]
    capacity: int               # particle slots
    n0: int = 0                 # carriers injected by the pulse
    fwhm: float = 30.0          # fs
    t0: float = 75.0            # pulse centre, fs
    abs_len: float = 15.0       # nm, exp(-z/abs_len) absorption; 0 = homogeneous
    excite_mask: int = 1        # bit l set: layer l is excited
    up_frac: float = 2.0 / 3.0  # fraction of injected carriers with spin up
    e_mode: int = E_UNIFORM
    k_mono: tuple = (1, 1)      # bins for E_MONO (spin up, spin down)
    # importance sampling of the source (FLAG_WEIGHTS): relative sampling
    # densities of the birth cell (float64 [n_cells]) and of the birth bin
    # (float64 [n_e], E_UNIFORM only); None = sample the physical profile
    cell_bias: np.ndarray = None
    e_bias: np.ndarray = None

    @property
    def n_cells(self) -> int:
        return int(sum(self.layer_cells))


@dataclass
class Workload:
    name: str
    n_e: int
    de: float                   # eV per bin
    dt: float                   # fs
    dz: float                   # nm per cell
    n_steps: int
    moment_every: int
    compact_every: int
    seed: int
    flags: int
    stacks: list = field(default_factory=list)

    def replace(self, **kw) -> "Workload":
        return dataclasses.replace(self, **kw)


def energy_grid(n_e: int, de: float) -> np.ndarray:
    return de * np.arange(1, n_e + 1, dtype=np.float64)


def base_tables(n_e: int, de: float):
    """Synthetic v, tau_in, tau_el, P0 for (Fe, Au, Fe_AP)."""
    e = energy_grid(n_e, de)
    x = np.linspace(0.0, 1.0, n_e) if n_e > 1 else np.zeros(1)
    v = np.empty((N_MAT, 2, n_e), np.float32)
    v[:] = (0.2 + 1.2 * x).astype(np.float32)
    tau_in = np.empty((N_MAT, 2, n_e), np.float64)
    for (m, s), t0 in TAU0_FS_EV2.items():
        tau_in[m, s] = t0 / (e * e)
    tau_el = np.full(N_MAT, TAU_EL_FS)
    p0 = np.array(P0, np.float64)
    return v, tau_in, tau_el, p0


def interface_T(mat_a: int, mat_b: int, n_e: int) -> np.ndarray:
    """T[dir][spin][k] for the interface between materials a (left) and b."""
    x = np.linspace(0.0, 1.0, n_e) if n_e > 1 else np.zeros(1)
    t_up, t_dn = 0.7 + 0.2 * x, 0.4 + 0.2 * x
    out = np.empty((2, 2, n_e))
    swap = (mat_a == MAT_FE_AP) or (mat_b == MAT_FE_AP)
    out[:, 0] = t_dn if swap else t_up
    out[:, 1] = t_up if swap else t_dn
    return out


def make_stack(layer_cells, layer_mat, n_e, de, capacity, n0, **pulse) -> Stack:
    v, tau_in, tau_el, p0 = base_tables(n_e, de)
    nl = len(layer_cells)
    T = np.stack([interface_T(layer_mat[i], layer_mat[i + 1], n_e)
                  for i in range(nl - 1)]) if nl > 1 else np.zeros((0, 2, 2, n_e))
    return Stack(list(map(int, layer_cells)), list(map(int, layer_mat)), v, tau_in,
                 tau_el, T, p0, int(capacity), int(n0), **pulse)


def perturb(stack: Stack, rng: np.random.Generator, rel: float = 0.2) -> Stack:
    """Independent factor U[1-rel, 1+rel] on every tau_in and T entry."""
    tau_in = stack.tau_in * rng.uniform(1 - rel, 1 + rel, stack.tau_in.shape)
    T = np.clip(stack.T * rng.uniform(1 - rel, 1 + rel, stack.T.shape), 0.0, 1.0)
    return dataclasses.replace(stack, tau_in=tau_in, T=T)


# --------------------------------------------------------------------------
# The five workloads: bilayer, spin valve, batched stacks, adjoint, large.
# `scale` shrinks particle counts and capacities (for tests and CPU runs).
# --------------------------------------------------------------------------

def bilayer(fe_nm=15, au_nm=100, n0=100_000, capacity=400_000, n_e=30, de=0.05,
            dt=1.0, n_steps=500, moment_every=1, compact_every=50, seed=0,
            flags=0, name="fe15_au100_bilayer") -> Workload:
    st = make_stack([fe_nm, au_nm], [MAT_FE, MAT_AU], n_e, de, capacity, n0)
    return Workload(name, n_e, de, dt, 1.0, n_steps, moment_every, compact_every,
                    seed, flags, [st])


def spin_valve(antiparallel=False, fe_nm=10, au_nm=50, n0=10_000_000,
               capacity=50_000_000, n_e=30, de=0.05, dt=0.5, n_steps=2000,
               moment_every=1, compact_every=50, seed=0, flags=0) -> Workload:
    mats = [MAT_FE, MAT_AU, MAT_FE_AP if antiparallel else MAT_FE]
    st = make_stack([fe_nm, au_nm, fe_nm], mats, n_e, de, capacity, n0)
    name = "fe10_au50_fe10_%s" % ("ap" if antiparallel else "p")
    return Workload(name, n_e, de, dt, 1.0, n_steps, moment_every, compact_every,
                    seed, flags, [st])


def batched(n_stacks=64, scale=1.0, n_e=30, de=0.05, dt=1.0, n_steps=1000,
            moment_every=1, compact_every=50, seed=0, flags=0,
            table_seed=12345) -> Workload:
    """Fe(15)/Au(d) stacks, d ~ round(U[20,200]) nm, P/AP alternating (the
    second half of each pair has an AP Fe emitter, i.e. spin tables swapped),
    N ~ logU[1e5, 1e7], capacity 4N, tables perturbed +-20 % per stack."""
    rng = np.random.default_rng(table_seed)
    stacks = []
    for i in range(n_stacks):
        d = int(round(rng.uniform(20.0, 200.0)))
        n = int(round(math.exp(rng.uniform(math.log(1e5), math.log(1e7))) * scale))
        n = max(n, 1)
        emitter = MAT_FE if i % 2 == 0 else MAT_FE_AP
        st = make_stack([15, d], [emitter, MAT_AU], n_e, de, 4 * n, n)
        stacks.append(perturb(st, rng))
    return Workload("batched_%dx_fe15_au20-200" % n_stacks, n_e, de, dt, 1.0,
                    n_steps, moment_every, compact_every, seed, flags, stacks)


def config(i: int, scale: float = 1.0, seed: int = 0, flags: int = 0) -> Workload:
    """The five standard workloads (particle counts multiplied by `scale`)."""
    s = lambda x: max(1, int(round(x * scale)))
    if i == 0:
        return bilayer(n0=s(1e5), capacity=s(4e5), seed=seed, flags=flags)
    if i == 1:
        return spin_valve(False, n0=s(1e7), capacity=s(5e7), seed=seed, flags=flags)
    if i == 2:
        return batched(scale=scale, seed=seed, flags=flags)
    if i == 3:
        return bilayer(n0=s(1e7), capacity=s(5e7), n_steps=800, seed=seed,
                       flags=flags, name="fe15_au100_adjoint")
    if i == 4:
        return bilayer(au_nm=300, n0=s(2e8), capacity=s(4e8), n_e=60, de=0.025,
                       dt=0.5, n_steps=10000, moment_every=50, compact_every=50,
                       seed=seed, flags=flags, name="fe15_au300_large")
    raise ValueError(i)


def infinite_slab(n_e=30, de=0.05, dt=1.0, cells=100_000, capacity=100_000,
                  n_steps=100, moment_every=1, compact_every=50, seed=0, flags=0,
                  mat=MAT_AU) -> Workload:
    """One very thick layer: walls are never reached (Sec. IV test settings)."""
    st = make_stack([cells], [mat], n_e, de, capacity, 0)
    return Workload("infinite_slab", n_e, de, dt, 1.0, n_steps, moment_every,
                    compact_every, seed, flags, [st])
