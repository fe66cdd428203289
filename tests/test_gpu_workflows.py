"""Workflows on top of the step, on the GPU.

- Appendix B phase-separation sweep as a GPU regression: every printed G12 row of the table runs
  as one replica of a batched ensemble (FP64, 128 x 2, fully periodic, two-layer start, 5e4 steps)
  and must reproduce the printed bulk densities of component 1.
- Preparation -> convection restart (Sec. 3.2.3): the emulsion relaxes without buoyancy
  (alpha_g = 0, linear temperature between the walls), its populations are read back with
  lb_get_state and loaded into a lattice with the convection parameters (alpha_g > 0) with
  lb_set_state; the continued run equals the oracle doing the same restart.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_2109_12565_gb300 import build as B
from paper_2109_12565_gb300 import inputs as I
from paper_2109_12565_gb300 import lb

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()


def _appB_table(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "appB_phase_separation.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                g, a, b = (float(v) for v in line.split())
                rows.append((g, a, b))
    return rows


def test_appendix_b_sweep_as_gpu_ensemble(golden_dir):
    """All 18 printed rows in one batched launch sequence.  The printed "0.40" row was run at the
    production coupling G12 = 0.405 (Appendix A).  Rows at or below 0.20 are mixed states whose
    printed max and min differ by a residue of the slow initial relaxation; rows 0.25 and 0.30 sit
    next to the critical coupling and relax slowly.  Tolerances as for the oracle pin, plus the
    same mass check."""
    table = _appB_table(golden_dir)
    ws = [I.layered(G12=0.405 if abs(g - 0.40) < 1e-9 else g) for g, _, _ in table]
    b = lb.Batch([w.params for w in ws], [w.rho1 for w in ws], [w.rho2 for w in ws], [w.T0 for w in ws],
                 precision=lb.LB_FP64)
    b.step(50000)
    for r, (g, want_max, want_min) in enumerate(table):
        r1 = b.fields(r)["rho1"]
        tol = 5e-5 if round(g, 2) in (0.25, 0.30) else 2e-6
        assert abs(r1.max() - want_max) <= tol, (g, r1.max(), want_max)
        assert abs(r1.min() - want_min) <= tol, (g, r1.min(), want_min)
        assert abs(r1.mean() - (65 * 1.4 + 63 * 0.1) / 128) < 5e-11
    b.close()


def test_preparation_then_convection_restart_matches_oracle():
    w = I.emulsion_small(nx=96, ny=48, n_drops=6, R=6.0)
    prep = dict(w.params, alpha_g=0.0)
    y = np.arange(w.params["ny"])[:, None] * np.ones((1, w.params["nx"]))
    H = w.params["ny"] - 2
    T_lin = w.params["T_down"] + (w.params["T_up"] - w.params["T_down"]) * (y - 0.5) / H
    g = lb.Lattice(prep, w.rho1, w.rho2, T_lin)
    o = O.Oracle(prep, w.rho1, w.rho2, T_lin)
    g.step(300)
    o.step(300)
    state = g.get_state()
    assert np.abs(state - o.state).max() <= 1e-12
    conv = dict(w.params, alpha_g=4.0 * w.params["alpha_g"])
    g2 = lb.Lattice.from_state(conv, state)
    o2 = O.Oracle.from_state(conv, o.state)
    assert g2.observables()["step"] == 0
    g2.step(400)
    o2.step(400)
    assert np.abs(g2.get_state() - o2.state).max() <= 1e-11
    og, oo = g2.observables(), o2.observables()
    assert abs(og["Nu"] - oo["Nu"]) <= 1e-10
    # the restart continued the prepared emulsion instead of starting over
    fresh = O.Oracle(conv, w.rho1, w.rho2, T_lin)
    fresh.step(400)
    assert np.abs(fresh.state - o2.state).max() > 1e-3
