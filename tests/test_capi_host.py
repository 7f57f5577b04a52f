"""C-ABI checks that need no GPU: the library builds, loads and exports every
symbol declared in include/pic.h, and its host-side table derivation (the
integer thresholds and the source schedule) equals the oracle's bit-for-bit.
"""
import math
import os
import re

import numpy as np
import pytest

from oracle.oracle import OracleSim
from paper_1807_04733_gb300 import build as B
from paper_1807_04733_gb300 import pic
from paper_1807_04733_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("pic_init", "pic_excite", "pic_step", "pic_moments", "pic_grad",
                     "pic_destroy", "pic_last_error", "pic_records"):
        assert required in names
    assert set(names) == set(pic.EXPORTS)


def test_library_exports_every_declared_symbol():
    L = pic.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert L.pic_status_string(3) == b"PIC_ERR_CAPACITY"
    assert L.pic_last_error(None) == b"no context"


def test_init_rejects_bad_arguments_without_a_device():
    wl = W.config(0, scale=0.01)
    p = pic.make_params(wl)
    p.n_e = 0
    tabs = pic._Tables(wl.stacks[0])
    with pytest.raises(pic.PicError) as e:
        pic.pic_init(p, [pic.make_stack(wl.stacks[0])], [tabs.c])
    assert e.value.status == 1


@pytest.mark.parametrize("field,value", [("event_pass", 2), ("event_pass", -1),
                                         ("consumer_warps", 6), ("hist_mode", 3)])
def test_init_rejects_bad_launch_options_without_a_device(field, value):
    wl = W.config(0, scale=0.01)
    p = pic.make_params(wl)
    setattr(p, field, value)
    tabs = pic._Tables(wl.stacks[0])
    with pytest.raises(pic.PicError) as e:
        pic.pic_init(p, [pic.make_stack(wl.stacks[0])], [tabs.c])
    assert e.value.status == 1


def test_compact_static_rejects_misaligned_inputs_without_a_device():
    # the compaction reads its inputs in 16-byte vectors: any input array
    # off a 16-byte boundary is an argument error, found before any device
    # work (the addresses are never dereferenced)
    good = 1 << 20
    for bad in range(4):
        ptrs = [good] * 4
        ptrs[bad] = good + 4
        with pytest.raises(pic.PicError) as e:
            pic.pic_compact_static(*ptrs, 1000, good, good, good, good)
        assert e.value.status == 1


WORKLOADS = [
    W.config(0, scale=0.01),
    W.spin_valve(True, n0=1000, capacity=4000, n_steps=300),
    W.batched(n_stacks=3, scale=1e-3, n_steps=160),
    W.config(4, scale=1e-4).replace(n_steps=400),
]


@pytest.mark.parametrize("wl", WORKLOADS, ids=lambda w: w.name)
def test_derived_tables_match_oracle(wl):
    for s, st in enumerate(wl.stacks):
        ref = OracleSim(wl, stack=s).tables()
        tabs = pic._Tables(st)
        got = pic.pic_derive_tables(pic.make_params(wl), pic.make_stack(st), tabs.c,
                                    pic.make_pulse(st), st.v.shape[0], wl.n_e, wl.n_steps)
        for key in ("P_thr", "Q_thr", "T_thr", "P0_thr"):
            assert np.array_equal(got[key], ref[key]), key
        assert got["up_thr"] == ref["up_thr"]
        assert np.array_equal(got["inj"], ref["inj"])
        assert got["inj"].sum() == st.n0


def test_threshold_edge_cases_match_oracle():
    wl = W.config(0, scale=0.01)
    st = wl.stacks[0]
    st.tau_in[0, 0, :5] = math.inf          # no inelastic channel
    st.tau_el[1] = math.inf                 # no elastic channel in Au
    st.tau_in[1, 1, :3] = 1e-12             # certain scattering
    st.T[0, 0, 0, :4] = [0.0, 1.0, 1e-12, 1 - 1e-16]
    ref = OracleSim(wl).tables()
    tabs = pic._Tables(st)
    got = pic.pic_derive_tables(pic.make_params(wl), pic.make_stack(st), tabs.c,
                                pic.make_pulse(st), 3, wl.n_e, wl.n_steps)
    for key in ("P_thr", "Q_thr", "T_thr", "P0_thr"):
        assert np.array_equal(got[key], ref[key]), key
    assert got["P_thr"][1, 1, 0] == 0xFFFFFFFF
    assert got["T_thr"][0, 0, 0, 0] == 0 and got["T_thr"][0, 0, 0, 1] == 0xFFFFFFFF
