"""pic_moment_window: one moment window into host or device memory.

The window read must equal the same window of pic_moments, whether the
caller's buffers are pinned host memory, pageable host memory (numpy) or
device memory, for a finished window and for the running one (whose fluxes
are the crossings so far); a window outside [0, n_out) is an argument error.
"""
import numpy as np
import pytest

from paper_1807_04733_gb300 import pic
from paper_1807_04733_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_moment_window_matches_pic_moments():
    wl = W.config(0, scale=0.02, flags=W.FLAG_DETERMINISTIC).replace(n_steps=120,
                                                                      moment_every=10)
    ctx = pic.Context(wl)
    ctx.step(75)                          # 7 windows done, the 8th running
    n_all, J_all, led = ctx.moments(0)
    n_all, J_all = n_all.cpu().numpy(), J_all.cpu().numpy()
    nc, no, _ = ctx.shape(0)
    for w in (0, 3, 6, 7, no - 1):
        # pinned host
        n_p = torch.zeros((2, wl.n_e, nc), dtype=torch.int32, pin_memory=True)
        J_p = torch.zeros((2, nc + 1), dtype=torch.int32, pin_memory=True)
        led_w = pic.pic_moment_window(ctx.ctx, 0, w, n_p.data_ptr(), J_p.data_ptr())
        assert led_w == led
        assert np.array_equal(n_p.numpy(), n_all[w].view(np.int32))
        assert np.array_equal(J_p.numpy(), J_all[w])
        # pageable host
        n_h = np.zeros((2, wl.n_e, nc), np.uint32)
        J_h = np.zeros((2, nc + 1), np.int32)
        pic.pic_moment_window(ctx.ctx, 0, w, n_h.ctypes.data, J_h.ctypes.data)
        assert np.array_equal(n_h, n_all[w].view(np.uint32))
        assert np.array_equal(J_h, J_all[w])
        # device, densities only
        n_d = torch.zeros((2, wl.n_e, nc), dtype=torch.int32, device="cuda")
        pic.pic_moment_window(ctx.ctx, 0, w, n_d.data_ptr(), None)
        assert np.array_equal(n_d.cpu().numpy(), n_all[w].view(np.int32))
    for bad in (-1, no):
        with pytest.raises(pic.PicError):
            pic.pic_moment_window(ctx.ctx, 0, bad, None, None)
    ctx.close()
