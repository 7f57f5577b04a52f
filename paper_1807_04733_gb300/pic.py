"""Thin Python binding of the C-ABI in ``include/pic.h`` (ctypes).

Argument marshalling only: every step of the hot path runs in the CUDA
kernels of ``libpic.so``.  The functions carry the C names (``pic_init``,
``pic_excite``, ``pic_step``, ``pic_moments``, ``pic_grad`` ...).  Device
buffers are torch tensors passed by ``data_ptr()``; streams are torch
streams passed by their ``cuda_stream`` handle.

There is no CPU fallback: if the library was not built, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libpic.so")

MAX_LAYERS = 16
MAX_MAT = 8
LEDGER_FIELDS = ("injected", "inject_dropped", "spawned", "spawn_dropped", "absorbed",
                 "q_injected", "q_bath", "q_dropped", "iface_hits", "iface_transmit",
                 "truncated", "particle_steps", "changed", "eventful")
STATUS = {0: "PIC_OK", 1: "PIC_ERR_ARG", 2: "PIC_ERR_ALLOC", 3: "PIC_ERR_CAPACITY",
          4: "PIC_ERR_TIMEOUT", 5: "PIC_ERR_CUDA", 6: "PIC_ERR_STATE"}
REC_DTYPE = np.dtype([("z", "<f4"), ("mu", "<f4"), ("id", "<u4"), ("packed", "<u4")])

# symbols declared in include/pic.h
EXPORTS = ("pic_init", "pic_excite", "pic_step", "pic_moments", "pic_moment_window",
           "pic_gen_moments",
           "pic_vel_moments", "pic_weighted_moments", "pic_weights", "pic_set_weights", "pic_grad",
           "pic_records",
           "pic_set_records", "pic_save", "pic_load", "pic_sync", "pic_derive_tables", "pic_shape", "pic_profile",
           "pic_profile_read", "pic_compact_static", "pic_launch_config", "pic_launch_count",
           "pic_destroy", "pic_last_error", "pic_status_string", "pic_autotune")
KERNEL_KINDS = ("inject", "step", "step_moments", "compact", "step_events", "adjoint_step",
                "adjoint_events", "adjoint_other", "flux", "weights")


class pic_params(C.Structure):
    _fields_ = [("n_e", C.c_int32), ("dt", C.c_float), ("dz", C.c_float),
                ("seed", C.c_uint64), ("flags", C.c_uint32), ("compact_every", C.c_int32),
                ("moment_every", C.c_int32), ("n_steps_max", C.c_int32),
                ("blocks_per_sm", C.c_int32), ("hist_mode", C.c_int32),
                ("ring_stages", C.c_int32), ("use_graph", C.c_int32),
                ("stack_base", C.c_int32), ("consumer_warps", C.c_int32),
                ("event_pass", C.c_int32)]


class pic_stack_desc(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("layer_cells", C.c_int32 * MAX_LAYERS),
                ("layer_mat", C.c_int32 * MAX_LAYERS), ("capacity", C.c_int64)]


class pic_tables(C.Structure):
    _fields_ = [("n_mat", C.c_int32), ("v", C.POINTER(C.c_float)),
                ("tau_in", C.POINTER(C.c_double)), ("tau_el", C.POINTER(C.c_double)),
                ("T", C.POINTER(C.c_double)), ("p0", C.POINTER(C.c_double))]


class pic_pulse(C.Structure):
    _fields_ = [("n0", C.c_int64), ("fwhm", C.c_double), ("t0", C.c_double),
                ("abs_len", C.c_double), ("excite_mask", C.c_uint32), ("up_frac", C.c_double),
                ("e_mode", C.c_int32), ("k_mono", C.c_int32 * 2),
                ("cell_bias", C.POINTER(C.c_double)), ("e_bias", C.POINTER(C.c_double))]


class pic_ledger(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in LEDGER_FIELDS]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n in LEDGER_FIELDS}


class pic_launch_info(C.Structure):
    _fields_ = [("grid_step", C.c_int32), ("grid_step_moments", C.c_int32),
                ("grid_slow", C.c_int32), ("grid_slow_moments", C.c_int32),
                ("grid_compact", C.c_int32), ("grid_inject", C.c_int32),
                ("ring_step", C.c_int32), ("ring_step_moments", C.c_int32),
                ("smem_step", C.c_int64), ("smem_step_moments", C.c_int64),
                ("warps_step", C.c_int32), ("warps_step_moments", C.c_int32),
                ("grid_adj_step", C.c_int32 * 2), ("ring_adj_step", C.c_int32 * 2),
                ("smem_adj_step", C.c_int64 * 2),
                ("grid_step_fused", C.c_int32), ("ring_step_fused", C.c_int32),
                ("smem_step_fused", C.c_int64)]

    def as_dict(self):
        out = {}
        for n, t in self._fields_:
            v = getattr(self, n)
            out[n] = [int(x) for x in v] if hasattr(t, "_length_") else int(v)
        return out


class pic_tune_entry(C.Structure):
    _fields_ = [("blocks_per_sm", C.c_int32), ("ring_stages", C.c_int32),
                ("hist_mode", C.c_int32), ("chosen", C.c_int32),
                ("ns_per_particle_step", C.c_double), ("consumer_warps", C.c_int32),
                ("event_pass", C.c_int32)]

    def as_dict(self):
        return {n: (float(getattr(self, n)) if n.startswith("ns") else int(getattr(self, n)))
                for n, _ in self._fields_}


class pic_kernel_times(C.Structure):
    _fields_ = [("launches", C.c_int64 * len(KERNEL_KINDS)), ("ms", C.c_double * len(KERNEL_KINDS))]


class PicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


_lib = None


def lib():
    """Load the in-tree library; fails loudly when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libpic.so is missing (%s): run __graft_entry__.build() first"
                               % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.pic_init.argtypes = [C.POINTER(P), C.POINTER(pic_params), C.POINTER(pic_stack_desc),
                               C.c_int, C.POINTER(pic_tables), P]
        L.pic_excite.argtypes = [P, C.c_int, C.POINTER(pic_pulse)]
        L.pic_step.argtypes = [P, C.c_int]
        L.pic_moments.argtypes = [P, C.c_int, P, P, C.POINTER(pic_ledger)]
        L.pic_moment_window.argtypes = [P, C.c_int, C.c_int, P, P, C.POINTER(pic_ledger)]
        L.pic_gen_moments.argtypes = [P, C.c_int, P]
        L.pic_vel_moments.argtypes = [P, C.c_int, P]
        L.pic_weighted_moments.argtypes = [P, C.c_int, P, P, C.POINTER(C.c_uint64)]
        L.pic_weights.argtypes = [P, C.c_int, P, C.POINTER(C.c_int64)]
        L.pic_set_weights.argtypes = [P, C.c_int, P, C.c_int64]
        L.pic_save.argtypes = [P, P, C.POINTER(C.c_size_t)]
        L.pic_load.argtypes = [P, P, C.c_size_t]
        L.pic_grad.argtypes = [P, P, P, P, P]
        L.pic_records.argtypes = [P, C.c_int, P, C.POINTER(C.c_int64)]
        L.pic_set_records.argtypes = [P, C.c_int, P, C.c_int64, C.c_uint64]
        L.pic_sync.argtypes = [P]
        L.pic_derive_tables.argtypes = [C.POINTER(pic_params), C.POINTER(pic_stack_desc),
                                        C.POINTER(pic_tables), C.POINTER(pic_pulse),
                                        P, P, P, P, P, P]
        L.pic_shape.argtypes = [P, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                C.POINTER(C.c_int32)]
        L.pic_profile.argtypes = [P, C.c_int]
        L.pic_profile_read.argtypes = [P, C.POINTER(pic_kernel_times)]
        L.pic_compact_static.argtypes = [P, P, P, P, C.c_int64, P, P, P, P,
                                         C.POINTER(C.c_int64), P]
        L.pic_launch_config.argtypes = [P, C.POINTER(pic_launch_info)]
        L.pic_autotune.argtypes = [P, C.c_int, C.POINTER(pic_tune_entry), C.c_int,
                                   C.POINTER(C.c_int)]
        L.pic_launch_count.argtypes = [P]
        L.pic_launch_count.restype = C.c_int64
        L.pic_destroy.argtypes = [P]
        L.pic_destroy.restype = None
        L.pic_last_error.argtypes = [P]
        L.pic_last_error.restype = C.c_char_p
        L.pic_status_string.argtypes = [C.c_int]
        L.pic_status_string.restype = C.c_char_p
        for name in EXPORTS:
            if name not in ("pic_launch_count", "pic_destroy", "pic_last_error",
                            "pic_status_string"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(status, ctx=None):
    if status != 0:
        raise PicError(status, lib().pic_last_error(ctx).decode())


# ---------------------------------------------------------------------------
# marshalling of the workload description
# ---------------------------------------------------------------------------
def make_params(wl, n_steps_max=None, flags=None, seed=None, blocks_per_sm=0, hist_mode=0,
                ring_stages=0, use_graph=0, stack_base=0, consumer_warps=0, event_pass=0):
    p = pic_params()
    p.n_e = wl.n_e; p.dt = wl.dt; p.dz = wl.dz
    p.seed = wl.seed if seed is None else seed
    p.flags = wl.flags if flags is None else flags
    p.compact_every = wl.compact_every; p.moment_every = wl.moment_every
    p.n_steps_max = wl.n_steps if n_steps_max is None else n_steps_max
    p.blocks_per_sm = blocks_per_sm; p.hist_mode = hist_mode; p.ring_stages = ring_stages
    # True/1: graph-replayed periods; 2 or "persistent": one persistent launch per period
    p.use_graph = 2 if use_graph in (2, "persistent") else (1 if use_graph else 0)
    p.stack_base = stack_base
    p.consumer_warps = consumer_warps
    p.event_pass = event_pass
    return p


def make_stack(st, capacity=None):
    d = pic_stack_desc()
    d.n_layers = len(st.layer_cells)
    for i, (c, m) in enumerate(zip(st.layer_cells, st.layer_mat)):
        d.layer_cells[i] = c; d.layer_mat[i] = m
    d.capacity = st.capacity if capacity is None else capacity
    return d


class _Tables:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, st):
        self.v = np.ascontiguousarray(st.v, np.float32)
        self.tau_in = np.ascontiguousarray(st.tau_in, np.float64)
        self.tau_el = np.ascontiguousarray(st.tau_el, np.float64)
        self.T = np.ascontiguousarray(st.T, np.float64).reshape(-1).copy() \
            if st.T.size else np.zeros(1)
        self.p0 = np.ascontiguousarray(st.p0, np.float64)
        t = pic_tables()
        t.n_mat = self.v.shape[0]
        t.v = self.v.ctypes.data_as(C.POINTER(C.c_float))
        t.tau_in = self.tau_in.ctypes.data_as(C.POINTER(C.c_double))
        t.tau_el = self.tau_el.ctypes.data_as(C.POINTER(C.c_double))
        t.T = self.T.ctypes.data_as(C.POINTER(C.c_double))
        t.p0 = self.p0.ctypes.data_as(C.POINTER(C.c_double))
        self.c = t


def make_pulse(st):
    """The pulse of a stack; the bias arrays (if any) are kept on the returned
    structure (attribute _keep) while it is alive."""
    u = pic_pulse()
    u.n0 = st.n0; u.fwhm = st.fwhm; u.t0 = st.t0; u.abs_len = st.abs_len
    u.excite_mask = st.excite_mask; u.up_frac = st.up_frac; u.e_mode = st.e_mode
    u.k_mono[0] = st.k_mono[0]; u.k_mono[1] = st.k_mono[1]
    keep = []
    if getattr(st, "cell_bias", None) is not None:
        cb = np.ascontiguousarray(st.cell_bias, np.float64)
        keep.append(cb)
        u.cell_bias = cb.ctypes.data_as(C.POINTER(C.c_double))
    if getattr(st, "e_bias", None) is not None:
        eb = np.ascontiguousarray(st.e_bias, np.float64)
        keep.append(eb)
        u.e_bias = eb.ctypes.data_as(C.POINTER(C.c_double))
    u._keep = keep
    return u


# ---------------------------------------------------------------------------
# C-named entry points
# ---------------------------------------------------------------------------
def pic_init(params, stacks, tables, stream=None):
    n = len(stacks)
    sarr = (pic_stack_desc * n)(*stacks)
    tarr = (pic_tables * n)(*tables)
    h = C.c_void_p()
    st = lib().pic_init(C.byref(h), C.byref(params), sarr, n, tarr,
                        C.c_void_p(stream) if stream else None)
    _check(st)
    return h


def pic_excite(ctx, stack, pulse):
    _check(lib().pic_excite(ctx, stack, C.byref(pulse)), ctx)


def pic_step(ctx, n_steps):
    _check(lib().pic_step(ctx, n_steps), ctx)


def pic_moments(ctx, stack, n_dev_ptr, J_dev_ptr):
    led = pic_ledger()
    _check(lib().pic_moments(ctx, stack, C.c_void_p(n_dev_ptr or 0) if n_dev_ptr else None,
                             C.c_void_p(J_dev_ptr) if J_dev_ptr else None, C.byref(led)), ctx)
    return led.as_dict()


def pic_moment_window(ctx, stack, window, n_ptr, J_ptr):
    """One moment window into host or device buffers (addresses); the ledger."""
    led = pic_ledger()
    _check(lib().pic_moment_window(ctx, stack, window, C.c_void_p(n_ptr) if n_ptr else None,
                                   C.c_void_p(J_ptr) if J_ptr else None, C.byref(led)), ctx)
    return led.as_dict()


def pic_weighted_moments(ctx, stack, nw_dev_ptr, Jw_dev_ptr):
    wi = C.c_uint64(0)
    _check(lib().pic_weighted_moments(ctx, stack, C.c_void_p(nw_dev_ptr) if nw_dev_ptr else None,
                                      C.c_void_p(Jw_dev_ptr) if Jw_dev_ptr else None,
                                      C.byref(wi)), ctx)
    return wi.value


def pic_weights(ctx, stack):
    n = C.c_int64(0)
    _check(lib().pic_weights(ctx, stack, None, C.byref(n)), ctx)
    out = np.zeros(n.value, np.uint32)
    if n.value:
        _check(lib().pic_weights(ctx, stack, out.ctypes.data, C.byref(n)), ctx)
    return out


def pic_set_weights(ctx, stack, w):
    w = np.ascontiguousarray(w, np.uint32)
    _check(lib().pic_set_weights(ctx, stack, w.ctypes.data if len(w) else None, len(w)), ctx)


def pic_save(ctx):
    """The context's checkpoint as bytes."""
    n = C.c_size_t(0)
    _check(lib().pic_save(ctx, None, C.byref(n)), ctx)
    buf = (C.c_ubyte * n.value)()
    _check(lib().pic_save(ctx, buf, C.byref(n)), ctx)
    return bytes(buf)


def pic_load(ctx, data):
    buf = (C.c_ubyte * len(data)).from_buffer_copy(data)
    _check(lib().pic_load(ctx, buf, len(data)), ctx)


def pic_gen_moments(ctx, stack, g_dev_ptr):
    _check(lib().pic_gen_moments(ctx, stack, C.c_void_p(g_dev_ptr)), ctx)


def pic_vel_moments(ctx, stack, v_dev_ptr):
    _check(lib().pic_vel_moments(ctx, stack, C.c_void_p(v_dev_ptr)), ctx)


def pic_grad(ctx, grad_n_ptr, grad_J_ptr, grad_tau_ptr, grad_T_ptr):
    _check(lib().pic_grad(ctx, C.c_void_p(grad_n_ptr) if grad_n_ptr else None,
                          C.c_void_p(grad_J_ptr) if grad_J_ptr else None,
                          C.c_void_p(grad_tau_ptr), C.c_void_p(grad_T_ptr)), ctx)


def pic_records(ctx, stack):
    n = C.c_int64(0)
    _check(lib().pic_records(ctx, stack, None, C.byref(n)), ctx)
    out = np.zeros(n.value, REC_DTYPE)
    if n.value:
        _check(lib().pic_records(ctx, stack, C.c_void_p(out.ctypes.data), C.byref(n)), ctx)
    return out[: n.value]


def pic_set_records(ctx, stack, recs, next_id):
    recs = np.ascontiguousarray(recs, REC_DTYPE)
    _check(lib().pic_set_records(ctx, stack, C.c_void_p(recs.ctypes.data) if len(recs) else None,
                                 len(recs), next_id), ctx)


def pic_sync(ctx):
    _check(lib().pic_sync(ctx), ctx)


def pic_shape(ctx, stack):
    nc, no, sp = C.c_int32(), C.c_int32(), C.c_int32()
    _check(lib().pic_shape(ctx, stack, C.byref(nc), C.byref(no), C.byref(sp)), ctx)
    return nc.value, no.value, sp.value


def pic_profile(ctx, enable):
    _check(lib().pic_profile(ctx, 1 if enable else 0), ctx)


def pic_profile_read(ctx):
    t = pic_kernel_times()
    _check(lib().pic_profile_read(ctx, C.byref(t)), ctx)
    return {k: (int(t.launches[i]), float(t.ms[i])) for i, k in enumerate(KERNEL_KINDS)}


def pic_compact_static(z, mu, id_, packed, n, z_out, mu_out, id_out, packed_out, stream=None):
    """Allocation-free stable compaction of caller-owned device arrays (data
    pointers); returns the number of live slots written to the outputs."""
    alive = C.c_int64(0)
    _check(lib().pic_compact_static(z, mu, id_, packed, n, z_out, mu_out, id_out, packed_out,
                                    C.byref(alive), C.c_void_p(stream) if stream else None))
    return alive.value


def pic_launch_config(ctx):
    info = pic_launch_info()
    _check(lib().pic_launch_config(ctx, C.byref(info)), ctx)
    return info.as_dict()


def pic_autotune(ctx, trial_steps, max_entries=256):
    buf = (pic_tune_entry * max_entries)()
    n = C.c_int(0)
    _check(lib().pic_autotune(ctx, trial_steps, buf, max_entries, C.byref(n)), ctx)
    return [buf[i].as_dict() for i in range(min(n.value, max_entries))]


def pic_launch_count(ctx):
    return int(lib().pic_launch_count(ctx))


def pic_destroy(ctx):
    if ctx is not None and ctx.value:
        lib().pic_destroy(ctx)


def pic_derive_tables(params, stack, tables, pulse, n_mat, n_e, n_steps_max):
    nl = stack.n_layers
    P = np.zeros((n_mat, 2, n_e), np.uint32); Q = np.zeros_like(P)
    T = np.zeros((max(nl - 1, 0), 2, 2, n_e), np.uint32)
    P0 = np.zeros(n_mat, np.uint32); up = np.zeros(1, np.uint32)
    inj = np.zeros(2 * n_steps_max, np.int64)
    _check(lib().pic_derive_tables(C.byref(params), C.byref(stack), C.byref(tables),
                                   C.byref(pulse) if pulse is not None else None,
                                   P.ctypes.data, Q.ctypes.data,
                                   T.ctypes.data if T.size else None, P0.ctypes.data,
                                   up.ctypes.data, inj.ctypes.data))
    return dict(P_thr=P, Q_thr=Q, T_thr=T, P0_thr=P0, up_thr=int(up[0]), inj=inj)


# ---------------------------------------------------------------------------
# convenience wrapper: a context for a workload, torch tensors as device memory
# ---------------------------------------------------------------------------
class Context:
    """All stacks of a workload in one context on the current CUDA device."""

    def __init__(self, wl, n_steps_max=None, flags=None, seed=None, blocks_per_sm=0,
                 hist_mode=0, stream=None, excite=True, capacity=None, ring_stages=0,
                 use_graph=False, stack_base=0, consumer_warps=0, event_pass=0):
        import torch
        self.wl = wl
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.params = make_params(wl, n_steps_max, flags, seed, blocks_per_sm, hist_mode,
                                  ring_stages, use_graph, stack_base, consumer_warps, event_pass)
        self._tabs = [_Tables(st) for st in wl.stacks]
        self.stacks = [make_stack(st, capacity) for st in wl.stacks]
        self.ctx = pic_init(self.params, self.stacks, [t.c for t in self._tabs],
                            self.stream.cuda_stream)
        if excite:
            for i, st in enumerate(wl.stacks):
                if st.n0 > 0:
                    pic_excite(self.ctx, i, make_pulse(st))

    def close(self):
        if getattr(self, "ctx", None) is not None:
            pic_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        pic_step(self.ctx, n)

    def shape(self, stack=0):
        return pic_shape(self.ctx, stack)

    def moments(self, stack=0):
        torch = self.torch
        nc, no, _ = self.shape(stack)
        dev = torch.device("cuda", torch.cuda.current_device())
        n = torch.empty((no, 2, self.wl.n_e, nc), dtype=torch.int32, device=dev)
        J = torch.empty((no, 2, nc + 1), dtype=torch.int32, device=dev)
        led = pic_moments(self.ctx, stack, n.data_ptr(), J.data_ptr())
        return n, J, led

    def gen_moments(self, stack=0):
        """Generation labels summed per [n_out][n_cells] (uint64 on the device,
        returned as int64), the numerator of the mean-generation map."""
        torch = self.torch
        nc, no, _ = self.shape(stack)
        dev = torch.device("cuda", torch.cuda.current_device())
        g = torch.empty((no, nc), dtype=torch.int64, device=dev)
        pic_gen_moments(self.ctx, stack, g.data_ptr())
        return g

    def vel_moments(self, stack=0):
        """Velocities v*mu summed per [n_out][2][n_cells] in units of 2^-32
        nm/fs (int64 on the device); needs FLAG_VELOCITY."""
        torch = self.torch
        nc, no, _ = self.shape(stack)
        dev = torch.device("cuda", torch.cuda.current_device())
        v = torch.empty((no, 2, nc), dtype=torch.int64, device=dev)
        pic_vel_moments(self.ctx, stack, v.data_ptr())
        return v

    def weighted_moments(self, stack=0):
        """Densities [n_out][2][n_e][n_cells] (uint64 as int64 on the device)
        and fluxes [n_out][2][n_cells+1] (int64) with every carrier counted
        with its weight (2^-20 units), and the summed weight the source
        created (PIC_F_WEIGHTS; Eq. PIC)."""
        torch = self.torch
        nc, no, _ = self.shape(stack)
        dev = torch.device("cuda", torch.cuda.current_device())
        nw = torch.empty((no, 2, self.wl.n_e, nc), dtype=torch.int64, device=dev)
        Jw = torch.empty((no, 2, nc + 1), dtype=torch.int64, device=dev)
        wi = pic_weighted_moments(self.ctx, stack, nw.data_ptr(), Jw.data_ptr())
        return nw, Jw, wi

    def save(self):
        """Checkpoint of the evolving state (pic_save), as bytes."""
        return pic_save(self.ctx)

    def load(self, data):
        """Restore a checkpoint of a context with the same workload (pic_load)."""
        pic_load(self.ctx, data)

    def weights(self, stack=0):
        return pic_weights(self.ctx, stack)

    def set_weights(self, w, stack=0):
        pic_set_weights(self.ctx, stack, w)

    def ledger(self, stack=0):
        return pic_moments(self.ctx, stack, None, None)

    def records(self, stack=0):
        return pic_records(self.ctx, stack)

    def set_records(self, recs, next_id, stack=0):
        pic_set_records(self.ctx, stack, recs, next_id)

    def sync(self):
        pic_sync(self.ctx)

    def launch_config(self):
        return pic_launch_config(self.ctx)

    @property
    def launches(self):
        return pic_launch_count(self.ctx)

    def autotune(self, trial_steps):
        """Time candidate launch configurations on the next steps of the run
        and keep the fastest; returns the trials (pic_autotune)."""
        return pic_autotune(self.ctx, trial_steps)

    # ---- adjoint ----
    @property
    def n_mat_max(self):
        return max(t.c.n_mat for t in self._tabs)

    @property
    def n_cells_max(self):
        return max(self.shape(s)[0] for s in range(len(self.wl.stacks)))

    def grad(self, grad_n=None, grad_J=None):
        """Score-function gradient of sum(grad_n * n) + sum(grad_J * J) over the
        steps run so far, with respect to tau_in [stack][mat][spin][k] and T
        [stack][interface][dir][spin][k] (float64 tensors on the device).

        grad_n: float [stacks][n_out][2][n_e][n_cells_max]; grad_J: float
        [stacks][n_out][2][n_cells_max+1] (device tensors, None = zero)."""
        torch = self.torch
        S, ne = len(self.wl.stacks), self.wl.n_e
        _, n_out, _ = self.shape(0)
        ncm = self.n_cells_max
        dev = torch.device("cuda", torch.cuda.current_device())
        if grad_n is not None:
            grad_n = grad_n.to(dev, torch.float32).contiguous()
            assert grad_n.shape == (S, n_out, 2, ne, ncm), grad_n.shape
        if grad_J is not None:
            grad_J = grad_J.to(dev, torch.float32).contiguous()
            assert grad_J.shape == (S, n_out, 2, ncm + 1), grad_J.shape
        g_tau = torch.empty((S, self.n_mat_max, 2, ne), dtype=torch.float64, device=dev)
        g_T = torch.empty((S, MAX_LAYERS - 1, 2, 2, ne), dtype=torch.float64, device=dev)
        pic_grad(self.ctx, grad_n.data_ptr() if grad_n is not None else None,
                 grad_J.data_ptr() if grad_J is not None else None,
                 g_tau.data_ptr(), g_T.data_ptr())
        return g_tau, g_T

    def moments_all(self):
        """Densities and fluxes of every stack, padded to the widest stack:
        n [stacks][n_out][2][n_e][n_cells_max], J [stacks][n_out][2][n_cells_max+1]
        (float32), the layouts grad() takes."""
        torch = self.torch
        S, ne = len(self.wl.stacks), self.wl.n_e
        ncm = self.n_cells_max
        _, n_out, _ = self.shape(0)
        dev = torch.device("cuda", torch.cuda.current_device())
        n_all = torch.zeros((S, n_out, 2, ne, ncm), dtype=torch.float32, device=dev)
        J_all = torch.zeros((S, n_out, 2, ncm + 1), dtype=torch.float32, device=dev)
        for s in range(S):
            n, J, _ = self.moments(s)
            nc = n.shape[-1]
            n_all[s, ..., :nc] = n.to(torch.float32)
            J_all[s, ..., : nc + 1] = J.to(torch.float32)
        return n_all, J_all


class PicTransport:
    """The PIC run as a differentiable function of the tables (torch autograd).

    ``PicTransport.apply(tau_in, T, wl, n_steps)`` builds a context for the
    workload with these lifetime ([stack][mat][2][n_e]) and transmittance
    ([stack][n_layers-1][2][2][n_e]) tables, runs n_steps and returns the
    densities and fluxes (padded layouts of Context.moments_all).  The
    backward pass is the library's adjoint (pic_grad): a score-function
    estimate of d E[moments] / d tables, contracted with the incoming
    gradients."""

    _fn = None

    @classmethod
    def apply(cls, tau_in, T, wl, n_steps, **ctx_kw):
        if cls._fn is None:
            import torch

            class _Fn(torch.autograd.Function):
                @staticmethod
                def forward(fctx, tau_in, T, wl, n_steps, ctx_kw):
                    import copy
                    w = copy.deepcopy(wl)
                    ti = tau_in.detach().cpu().numpy()
                    Tt = T.detach().cpu().numpy()
                    for s, st in enumerate(w.stacks):
                        st.tau_in = ti[s, : st.tau_in.shape[0]].copy()
                        nif = len(st.layer_cells) - 1
                        st.T = Tt[s, :nif].copy()
                    c = Context(w, **ctx_kw)
                    c.step(n_steps)
                    n_all, J_all = c.moments_all()
                    fctx.pic = c
                    fctx.shapes = (tau_in.shape, T.shape)
                    fctx.devs = (tau_in.device, T.device)
                    return n_all, J_all

                @staticmethod
                def backward(fctx, g_n, g_J):
                    c = fctx.pic
                    g_tau, g_T = c.grad(g_n, g_J)
                    sh_tau, sh_T = fctx.shapes
                    gt = torch.zeros(sh_tau, dtype=torch.float64, device=g_tau.device)
                    gt[:, : g_tau.shape[1]] = g_tau[:, : sh_tau[1]]
                    gT = torch.zeros(sh_T, dtype=torch.float64, device=g_T.device)
                    gT[:, : sh_T[1]] = g_T[:, : sh_T[1]]
                    c.close()
                    return gt.to(fctx.devs[0]), gT.to(fctx.devs[1]), None, None, None

            cls._fn = _Fn
        return cls._fn.apply(tau_in, T, wl, n_steps, ctx_kw)
