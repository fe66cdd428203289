"""The C-ABI library loads and exports every symbol include/tlb.h declares; host-side
parameter checks and workspace sizing (no GPU needed for any of these)."""
import math
import os
import re

import pytest

from paper_2109_12565_gb300 import build as B
from paper_2109_12565_gb300 import inputs as I
from paper_2109_12565_gb300 import lb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return lb.lib()


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:[A-Za-z_][\w ]*[\s*]+)(lb_\w+)\s*\(", txt, re.M))
    return names


def test_every_declared_symbol_is_exported(L):
    names = _declared_symbols()
    assert {"lb_init", "lb_step", "lb_observables", "lb_workspace_size"} <= names
    for n in names:
        assert hasattr(L, n), n
    assert set(lb.EXPORTS) <= names


def test_version_and_error_text(L):
    assert b"sm_103a" in L.lb_version()
    assert L.lb_last_error(None) is not None


def test_workspace_size_layout():
    w = I.emulsion_small()
    n64 = lb.workspace_size(w.params, False, lb.LB_FP64)
    n32 = lb.workspace_size(w.params, False, lb.LB_FP32_SHIFTED)
    # two buffers of 27 planes; FP64 rows padded to 16 doubles, FP32 rows to 32 floats
    assert n64 >= 2 * 27 * 64 * 64 * 8 and n32 >= 2 * 27 * 64 * 64 * 4
    assert n32 < n64
    assert lb.workspace_size(w.params, True, lb.LB_FP64) > n64
    big = I.emulsion_1024x512()
    assert lb.workspace_size(big.params, False, lb.LB_FP64) < 2 * 27 * 1024 * 512 * 8 * 1.01
    # FP32 fluid + FP16 thermal: 18 * 4 + 9 * 2 = 90 bytes per node and buffer
    # double-float pairs take the FP64 footprint
    assert lb.workspace_size(big.params, False, lb.LB_DF64) == lb.workspace_size(big.params, False, lb.LB_FP64)
    n16 = lb.workspace_size(big.params, False, lb.LB_FP32_FP16T)
    assert 2 * 90 * 1024 * 512 <= n16 < 2 * 90 * 1024 * 512 * 1.01
    assert n16 < lb.workspace_size(big.params, False, lb.LB_FP32_SHIFTED)


@pytest.mark.parametrize("bad", [dict(tau=0.5), dict(tau_g=0.4), dict(rho0=0.0), dict(nx=0), dict(ny=2),
                                 dict(precision=7), dict(G12=math.inf), dict(rho_wall=(0.0, 0.5)),
                                 dict(nx=32, ny=65536), dict(nx=16384, ny=4864)])
def test_invalid_parameters_rejected(bad):
    p = dict(I.emulsion_small().params)
    p.update(bad)
    with pytest.raises(lb.LbError) as e:
        lb.workspace_size(p, False, p.get("precision", lb.LB_FP64))
    assert e.value.code == lb.LB_EINVAL
