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


def test_static_scratch_observables_match_workspace_path():
    import torch

    B.build()
    w = I.emulsion_small()
    mask = I.posts_mask(64, 64, 3, 4, 16)
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, mask=mask, precision=lb.LB_FP64)
    d_mask = torch.from_numpy(mask).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for n in (25, 40):  # two calls in a row on different states share the scratch array
        g.step(n)
        ref = g.observables()
        d_state = torch.from_numpy(g.get_state()).cuda()
        torch.cuda.synchronize()
        rc, o = _call(g.cp, d_state.data_ptr(), d_mask.data_ptr(), stream)
        assert rc == lb.LB_OK
        np.testing.assert_allclose(np.array(o.mass[:]), ref["mass"], rtol=1e-13)
        np.testing.assert_allclose(np.array(o.mom[:]), ref["mom"], rtol=0, atol=1e-11)
        assert abs(o.Nu - ref["Nu"]) <= 1e-10 and abs(o.E - ref["E"]) <= 1e-14
        assert o.n_fluid == ref["n_fluid"] and o.n_bad == 0 and o.status == lb.LB_OK


def test_static_scratch_rejects_oversized_lattice():
    import torch

    B.build()
    p = dict(I.emulsion_small().params, nx=8192, ny=4096)
    d = torch.zeros(1, dtype=torch.float64, device="cuda")  # never read: the size check comes first
    rc, _ = _call(lb.make_params(p), d.data_ptr(), 0, torch.cuda.current_stream().cuda_stream)
    assert rc == lb.LB_EINVAL
