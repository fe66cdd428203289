"""lb_observables_static: observables without any device allocation by the library.

Callers that cannot allocate device memory (a plug-in inside an application that owns every
allocation, a real-time loop that must not take cudaMalloc's device-wide synchronisation) pass
their own device copy of the state and get the observables back; the library's scratch is a fixed
device array.  This file is collected last so that a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_2109_12565_gb300 import build as B
from paper_2109_12565_gb300 import inputs as I
from paper_2109_12565_gb300 import lb

pytestmark = pytest.mark.gpu


def _call(cp, d_state, d_mask, stream):
    L = lb.lib()
    L.lb_observables_static.argtypes = [ctypes.POINTER(lb.LbParams), ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.POINTER(lb.LbObs), ctypes.c_void_p]
    L.lb_observables_static.restype = ctypes.c_int
    o = lb.LbObs()
    rc = L.lb_observables_static(ctypes.byref(cp), ctypes.c_void_p(d_state), ctypes.c_void_p(d_mask),
                                 ctypes.byref(o), ctypes.c_void_p(stream))
    return rc, o


def _check_same(o, ref):
    np.testing.assert_allclose(np.array(o.mass[:]), ref["mass"], rtol=1e-13)
    np.testing.assert_allclose(np.array(o.mom[:]), ref["mom"], rtol=0, atol=1e-11)
    assert abs(o.Nu - ref["Nu"]) <= 1e-10 and abs(o.E - ref["E"]) <= 1e-14
    np.testing.assert_allclose(np.array(o.wall_fx[:]), ref["wall_fx"], rtol=0, atol=1e-12)
    assert o.n_fluid == ref["n_fluid"] and o.n_bad == 0 and o.status == lb.LB_OK


def _workloads():
    w = I.emulsion_small()
    yield "64x64 walls + posts", w, I.posts_mask(64, 64, 3, 4, 16)
    # widths that are not a multiple of the handle's 16-double row padding: the caller's unpadded
    # layout differs from the handle's
    w = I.emulsion_small(nx=50, ny=40, n_drops=2, R=6.0)
    yield "50x40 walls", w, None
    w = I.emulsion_small(nx=48, ny=36, n_drops=2, R=6.0)
    w.params = dict(w.params, periodic_y=1)
    yield "48x36 periodic y", w, None


@pytest.mark.parametrize("case", [0, 1, 2])
def test_static_scratch_observables_match_workspace_path(case):
    import torch

    B.build()
    name, w, mask = list(_workloads())[case]
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, mask=mask, precision=lb.LB_FP64)
    d_mask = torch.from_numpy(mask).cuda() if mask is not None else None
    mp = d_mask.data_ptr() if d_mask is not None else 0
    stream = torch.cuda.current_stream().cuda_stream
    for k, n in enumerate((25, 40)):  # two calls in a row on different states share the scratch array
        g.step(n)
        ref = g.observables()
        d_state = torch.from_numpy(g.get_state()).cuda()
        torch.cuda.synchronize()
        if k == 0:
            rc, o = _call(g.cp, d_state.data_ptr(), mp, stream)
        else:
            # every tensor of this call exists already: the library's call must not change free memory
            free0 = torch.cuda.mem_get_info()[0]
            rc, o = _call(g.cp, d_state.data_ptr(), mp, stream)
            assert torch.cuda.mem_get_info()[0] == free0, name
        assert rc == lb.LB_OK, name
        _check_same(o, ref)
    g.close()


def test_static_scratch_rejects_oversized_lattice_and_misaligned_state():
    import torch

    B.build()
    p = dict(I.emulsion_small().params, nx=8192, ny=4096)
    d = torch.zeros(4, dtype=torch.float64, device="cuda")  # never read: the checks come first
    stream = torch.cuda.current_stream().cuda_stream
    rc, _ = _call(lb.make_params(p), d.data_ptr(), 0, stream)
    assert rc == lb.LB_EINVAL
    small = lb.make_params(I.emulsion_small().params)
    rc, _ = _call(small, d.data_ptr() + 4, 0, stream)  # not 8-byte aligned
    assert rc == lb.LB_EINVAL
