"""ctypes wrapper around the C oracle (``pic_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``.  The product path (the package
and its C-ABI library) never imports this module.

``OracleSim(workload, stack=0)`` runs the plain scalar CPU implementation of
the per-step superparticle update (Sec. III of the paper) for one stack.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liboracle.so")

REC_DTYPE = np.dtype([("z", "<f4"), ("mu", "<f4"), ("id", "<u4"), ("packed", "<u4")])
MAX_LAYERS = 16


def build(force: bool = False) -> str:
    """Compile the oracle with no floating-point contraction."""
    src = os.path.join(HERE, "pic_oracle.c")
    if not force and os.path.exists(LIB_PATH) and \
            os.path.getmtime(LIB_PATH) >= max(os.path.getmtime(src),
                                               os.path.getmtime(os.path.join(HERE, "pic_oracle.h"))):
        return LIB_PATH
    os.makedirs(os.path.dirname(LIB_PATH), exist_ok=True)
    tmp = LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fexcess-precision=standard", "-shared", "-fPIC", "-o", tmp, src, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class _Config(C.Structure):
    _fields_ = [
        ("n_e", C.c_int32), ("dt", C.c_float), ("dz", C.c_float),
        ("seed", C.c_uint64), ("stack_index", C.c_uint32), ("flags", C.c_uint32),
        ("capacity", C.c_int64), ("compact_every", C.c_int32),
        ("moment_every", C.c_int32), ("n_steps_max", C.c_int32),
        ("n_layers", C.c_int32), ("layer_cells", C.c_int32 * MAX_LAYERS),
        ("layer_mat", C.c_int32 * MAX_LAYERS), ("n_mat", C.c_int32),
        ("v", C.POINTER(C.c_float)), ("tau_in", C.POINTER(C.c_double)),
        ("tau_el", C.POINTER(C.c_double)), ("T", C.POINTER(C.c_double)),
        ("p0", C.POINTER(C.c_double)),
        ("n0", C.c_int64), ("fwhm", C.c_double), ("t0", C.c_double),
        ("abs_len", C.c_double), ("excite_mask", C.c_uint32), ("up_frac", C.c_double),
        ("e_mode", C.c_int32), ("k_mono", C.c_int32 * 2),
        ("cell_bias", C.POINTER(C.c_double)), ("e_bias", C.POINTER(C.c_double)),
    ]


class Ledger(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in (
        "injected", "inject_dropped", "spawned", "spawn_dropped", "absorbed",
        "q_injected", "q_bath", "q_dropped", "iface_hits", "iface_transmit",
        "truncated", "particle_steps", "changed", "eventful")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.c_void_p
        L.or_create.argtypes = [C.POINTER(_Config), C.POINTER(P)]
        L.or_destroy.argtypes = [P]
        L.or_step.argtypes = [P, C.c_int]
        L.or_n_slots.argtypes = [P]; L.or_n_slots.restype = C.c_int64
        L.or_records.argtypes = [P, P]
        L.or_set_records.argtypes = [P, P, C.c_int64, C.c_uint64]
        L.or_moments.argtypes = [P, P, P, C.POINTER(Ledger)]
        L.or_gen_moments.argtypes = [P, P]
        L.or_vel_moments.argtypes = [P, P]
        L.or_weighted_moments.argtypes = [P, P, P, P]
        L.or_weights.argtypes = [P, P]
        L.or_set_weights.argtypes = [P, P, C.c_int64]
        L.or_n_cells.argtypes = [P]; L.or_n_cells.restype = C.c_int32
        L.or_n_out.argtypes = [P]; L.or_n_out.restype = C.c_int32
        L.or_step_index.argtypes = [P]; L.or_step_index.restype = C.c_int32
        L.or_set_step.argtypes = [P, C.c_int32]
        L.or_next_id.argtypes = [P]; L.or_next_id.restype = C.c_uint64
        L.or_tables.argtypes = [P, P, P, P, P, P, P]
        L.or_philox4x32_10.argtypes = [P, P, P]
        L.or_grad.argtypes = [C.POINTER(_Config), P, C.c_int64, C.c_uint64, C.c_int,
                              P, P, P, P, P, P]
        L.or_advance_one.argtypes = [P, P, C.c_int64, C.c_int, P, P]
        _lib = L
    return _lib


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, np.uint32).copy()
    k = np.asarray(key, np.uint32).copy()
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def _ptr(a, t):
    return a.ctypes.data_as(C.POINTER(t))


class OracleSim:
    """One stack of a workload, stepped by the scalar CPU oracle."""

    def __init__(self, wl, stack: int = 0, n_steps_max: int | None = None,
                 capacity: int | None = None, seed: int | None = None,
                 flags: int | None = None):
        st = wl.stacks[stack]
        self.wl, self.st = wl, st
        self._keep = [np.ascontiguousarray(st.v, np.float32),
                      np.ascontiguousarray(st.tau_in, np.float64),
                      np.ascontiguousarray(st.tau_el, np.float64),
                      np.ascontiguousarray(st.T, np.float64).reshape(-1).copy()
                      if st.T.size else np.zeros(1),
                      np.ascontiguousarray(st.p0, np.float64)]
        v, ti, te, T, p0 = self._keep
        cfg = _Config()
        cfg.n_e = wl.n_e; cfg.dt = wl.dt; cfg.dz = wl.dz
        cfg.seed = wl.seed if seed is None else seed
        cfg.stack_index = stack
        cfg.flags = wl.flags if flags is None else flags
        cfg.capacity = st.capacity if capacity is None else capacity
        cfg.compact_every = wl.compact_every; cfg.moment_every = wl.moment_every
        cfg.n_steps_max = wl.n_steps if n_steps_max is None else n_steps_max
        cfg.n_layers = len(st.layer_cells)
        for i, (c, m) in enumerate(zip(st.layer_cells, st.layer_mat)):
            cfg.layer_cells[i] = c; cfg.layer_mat[i] = m
        cfg.n_mat = v.shape[0]
        cfg.v = _ptr(v, C.c_float); cfg.tau_in = _ptr(ti, C.c_double)
        cfg.tau_el = _ptr(te, C.c_double); cfg.T = _ptr(T, C.c_double)
        cfg.p0 = _ptr(p0, C.c_double)
        cfg.n0 = st.n0; cfg.fwhm = st.fwhm; cfg.t0 = st.t0; cfg.abs_len = st.abs_len
        cfg.excite_mask = st.excite_mask; cfg.up_frac = st.up_frac
        cfg.e_mode = st.e_mode; cfg.k_mono[0] = st.k_mono[0]; cfg.k_mono[1] = st.k_mono[1]
        if getattr(st, "cell_bias", None) is not None:
            cb = np.ascontiguousarray(st.cell_bias, np.float64)
            assert cb.shape == (st.n_cells,)
            self._keep.append(cb)
            cfg.cell_bias = _ptr(cb, C.c_double)
        if getattr(st, "e_bias", None) is not None:
            eb = np.ascontiguousarray(st.e_bias, np.float64)
            assert eb.shape == (wl.n_e,)
            self._keep.append(eb)
            cfg.e_bias = _ptr(eb, C.c_double)
        self.cfg = cfg
        h = C.c_void_p()
        rc = lib().or_create(C.byref(cfg), C.byref(h))
        if rc != 0:
            raise ValueError("or_create failed with code %d" % rc)
        self.h = h
        self.n_cells = lib().or_n_cells(h)
        self.n_out = lib().or_n_out(h)
        # initial state the adjoint replays from (records loaded at step 0)
        self._init = np.zeros(0, REC_DTYPE)
        self._init_next_id = 0

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and h.value:
            lib().or_destroy(h)
            self.h = None

    def step(self, n: int = 1) -> int:
        return lib().or_step(self.h, n)

    def records(self) -> np.ndarray:
        n = lib().or_n_slots(self.h)
        out = np.zeros(n, REC_DTYPE)
        if n:
            lib().or_records(self.h, out.ctypes.data)
        return out

    def set_records(self, recs: np.ndarray, next_id: int):
        recs = np.ascontiguousarray(recs, REC_DTYPE)
        rc = lib().or_set_records(self.h, recs.ctypes.data, len(recs), next_id)
        if rc:
            raise ValueError("set_records failed")
        if self.step_index == 0:
            self._init = recs.copy()
            self._init_next_id = int(next_id)
        else:
            self._init = None                # the run can no longer be replayed

    def moments(self):
        ne, nc = self.wl.n_e, self.n_cells
        n = np.zeros((self.n_out, 2, ne, nc), np.uint32)
        J = np.zeros((self.n_out, 2, nc + 1), np.int32)
        led = Ledger()
        lib().or_moments(self.h, n.ctypes.data, J.ctypes.data, C.byref(led))
        return n, J, led.as_dict()

    def vel_moments(self) -> np.ndarray:
        """Velocities v*mu summed per [output time][spin][cell] in units of
        2^-32 nm/fs (requires FLAG_VELOCITY; Eq. spincurrent)."""
        v = np.zeros((self.n_out, 2, self.n_cells), np.int64)
        lib().or_vel_moments(self.h, v.ctypes.data)
        return v

    def weighted_moments(self):
        """Superparticle weights (FLAG_WEIGHTS; Eq. PIC): the densities
        [n_out][2][n_e][n_cells] (uint64) and fluxes [n_out][2][n_cells+1]
        (int64) with every carrier counted with its weight, in units of
        2^-20, and the summed weight of the carriers the source created."""
        nw = np.zeros((self.n_out, 2, self.wl.n_e, self.n_cells), np.uint64)
        Jw = np.zeros((self.n_out, 2, self.n_cells + 1), np.int64)
        wi = np.zeros(1, np.uint64)
        lib().or_weighted_moments(self.h, nw.ctypes.data, Jw.ctypes.data, wi.ctypes.data)
        return nw, Jw, int(wi[0])

    def weights(self) -> np.ndarray:
        n = lib().or_n_slots(self.h)
        w = np.zeros(n, np.uint32)
        if n:
            lib().or_weights(self.h, w.ctypes.data)
        return w

    def set_weights(self, w):
        w = np.ascontiguousarray(w, np.uint32)
        if lib().or_set_weights(self.h, w.ctypes.data, len(w)):
            raise ValueError("set_weights: one weight per slot, each > 0")

    def gen_moments(self) -> np.ndarray:
        """Generation labels summed per [output time][cell] at the density
        instants (the numerator of the mean-generation maps, Figs. 5(b), 7)."""
        g = np.zeros((self.n_out, self.n_cells), np.uint64)
        lib().or_gen_moments(self.h, g.ctypes.data)
        return g

    def grad(self, gn, gJ, n_steps: int | None = None):
        """Score-function gradient of sum(gn * n) + sum(gJ * J) with respect to
        tau_in [n_mat][2][n_e] and T [n_if][2][2][n_e], over the first n_steps
        steps (default: the steps run so far) from the initial state.

        Returns (g_tau, g_T, mag_tau, mag_T); mag_* sum |score| (|total| +
        |earned|) per entry, the scale of rounding differences."""
        if self._init is None:
            raise ValueError("records were replaced after step 0: nothing to replay")
        n_steps = self.step_index if n_steps is None else n_steps
        ne, nc = self.wl.n_e, self.n_cells
        gn = np.ascontiguousarray(np.broadcast_to(np.asarray(gn, np.float32),
                                                  (self.n_out, 2, ne, nc)))
        gJ = np.ascontiguousarray(np.broadcast_to(np.asarray(gJ, np.float32),
                                                  (self.n_out, 2, nc + 1)))
        nm, nif = self.cfg.n_mat, len(self.st.layer_cells) - 1
        g_tau = np.zeros((nm, 2, ne)); m_tau = np.zeros_like(g_tau)
        g_T = np.zeros((max(nif, 0), 2, 2, ne)); m_T = np.zeros_like(g_T)
        init = np.ascontiguousarray(self._init, REC_DTYPE)
        rc = lib().or_grad(C.byref(self.cfg), init.ctypes.data if len(init) else None,
                           len(init), self._init_next_id, n_steps, gn.ctypes.data,
                           gJ.ctypes.data, g_tau.ctypes.data,
                           g_T.ctypes.data if g_T.size else None, m_tau.ctypes.data,
                           m_T.ctypes.data if m_T.size else None)
        if rc:
            raise ValueError("or_grad failed with code %d" % rc)
        return g_tau, g_T, m_tau, m_T

    def advance_one(self, rec, slot: int, room: bool = True):
        """One carrier (a REC_DTYPE record) in slot `slot` advanced by one step
        at the current step index: (record after the step, secondary or None)."""
        inp = np.ascontiguousarray(np.asarray(rec, REC_DTYPE).reshape(1))
        out = np.zeros(1, REC_DTYPE)
        sec = np.zeros(1, REC_DTYPE)
        made = lib().or_advance_one(self.h, inp.ctypes.data, slot, 1 if room else 0,
                                    out.ctypes.data, sec.ctypes.data)
        return out[0], (sec[0] if made else None)

    def set_step(self, step: int):
        lib().or_set_step(self.h, step)

    @property
    def step_index(self) -> int:
        return lib().or_step_index(self.h)

    @property
    def next_id(self) -> int:
        return int(lib().or_next_id(self.h))

    def tables(self):
        wl, st = self.wl, self.st
        ne, nm, nif = wl.n_e, self.cfg.n_mat, len(st.layer_cells) - 1
        P = np.zeros((nm, 2, ne), np.uint32); Q = np.zeros_like(P)
        T = np.zeros((max(nif, 0), 2, 2, ne), np.uint32)
        P0 = np.zeros(nm, np.uint32); up = np.zeros(1, np.uint32)
        inj = np.zeros(2 * self.cfg.n_steps_max, np.int64)
        lib().or_tables(self.h, P.ctypes.data, Q.ctypes.data, T.ctypes.data,
                        P0.ctypes.data, up.ctypes.data, inj.ctypes.data)
        return dict(P_thr=P, Q_thr=Q, T_thr=T, P0_thr=P0, up_thr=int(up[0]), inj=inj)


# ---- helpers for reading packed words (the record layout of the method) ----
def unpack(packed: np.ndarray):
    packed = np.asarray(packed, np.uint32)
    return dict(k=packed & 0xFF, spin=(packed >> 8) & 1, layer=(packed >> 9) & 0xF,
                gen=(packed >> 13) & 0xFF, id_hi=packed >> 21)


def pack(k, spin, layer, gen, id_hi=0):
    return (np.asarray(k, np.uint32) | (np.asarray(spin, np.uint32) << 8)
            | (np.asarray(layer, np.uint32) << 9) | (np.asarray(gen, np.uint32) << 13)
            | (np.asarray(id_hi, np.uint32) << 21)).astype(np.uint32)


if __name__ == "__main__":
    build(force="--force" in sys.argv)
    print(LIB_PATH)
