"""GPU total shear stress (lb_stress, lb_batch_stress; Sec. 2.1 after Eq. NS, Sec. 3.2.1) against the
FP64 oracle (orc_stress) on the same state, element by element.

Tolerances: FP64 storage, max |GPU - oracle| <= 1e-10 max |sigma_xy| (both compute the same FP64
formula in a different order; the central differences of u^(H) cancel about two digits).  FP32
storage: the state itself is rounded to FP32 deviations (relative 6e-8 of w_i rho, about 1e-8 in
rho and u^(H)); the interaction terms multiply density errors by couplings |G| psi' ~ 10 and the
stress is about 1e-4, so the bound is 1e-3 max |sigma_xy| (FP32 + FP16 thermal: the same, T enters
only through the buoyancy).  Physics on the GPU path: steady Couette flow gives rho nu gamma-dot at
every node; a sheared emulsion's averaged stress balances its wall stress within 2%.
"""
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

    assert torch.cuda.is_available()
    B.build()


def _cases():
    w = I.emulsion_small()
    yield "64x64 moving walls + posts", dict(w.params, u_wall=(-0.01, 0.015)), w, I.posts_mask(64, 64, 3, 4, 16)
    w = I.emulsion_small(nx=70, ny=36, n_drops=2, R=6.0)
    yield "70x36 ragged, walls", dict(w.params, u_wall=(0.0, 0.02)), w, None
    w = I.emulsion_small(nx=48, ny=48, n_drops=3, R=6.0)
    yield "48x48 periodic y", dict(w.params, periodic_y=1), w, None


def _compare(g, p, state, mask, tol):
    s_o = O.stress(p, state, mask=mask)
    s_g = g.stress()
    scale = np.abs(s_o["sxy"]).max()
    assert scale > 0
    err = np.abs(s_g["sxy"] - s_o["sxy"]).max()
    assert err <= tol * scale, (err, scale)
    np.testing.assert_allclose(s_g["row"], s_o["row"], rtol=0, atol=tol * scale)
    for k in ("Sigma", "visc", "pint", "pforce"):
        assert abs(s_g[k] - s_o[k]) <= tol * scale, (k, s_g[k], s_o[k])
    return err / scale


@pytest.mark.parametrize("case", [0, 1, 2])
@pytest.mark.parametrize("precision,tol", [(lb.LB_FP64, 1e-10), (lb.LB_DF64, 1e-10), (lb.LB_FP32_SHIFTED, 1e-3),
                                           (lb.LB_FP32_FP16T, 1e-3)])
def test_stress_matches_oracle(case, precision, tol):
    name, p, w, mask = list(_cases())[case]
    o = O.Oracle(p, w.rho1, w.rho2, w.T0, mask=mask)
    o.step(150)
    g = lb.Lattice(p, w.rho1, w.rho2, w.T0, mask=mask, precision=precision)
    g.set_state(o.state)
    rel = _compare(g, p, o.state, mask, tol)
    print(name, precision, f"{rel:.2e}")
    # the stress pass leaves the state alone
    g2 = lb.Lattice(p, w.rho1, w.rho2, w.T0, mask=mask, precision=precision)
    g2.set_state(o.state)
    g.step(3)
    g2.step(3)
    assert np.array_equal(g.get_state(), g2.get_state())
    g.close()
    g2.close()


def test_stress_full_size_1024x512():
    """The benchmark lattice in the benchmark's storage (FP32-shifted), at a state the oracle made."""
    w = I.emulsion_1024x512()
    o = O.Oracle(w.params, w.rho1, w.rho2, w.T0, omp=True)
    o.step(10)
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, precision=lb.LB_FP32_SHIFTED)
    g.set_state(o.state)
    _compare(g, w.params, o.state, None, 1e-3)
    g64 = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, precision=lb.LB_FP64)
    g64.set_state(o.state)
    _compare(g64, w.params, o.state, None, 1e-10)


def test_batch_stress_equals_single_lattice():
    w = I.emulsion_small(nx=96, ny=40, n_drops=3, R=6.0)
    w2 = I.emulsion_small(nx=64, ny=64)
    ps = [dict(w.params, u_wall=(-0.01, 0.01)), dict(w2.params, u_wall=(0.0, 0.02))]
    ws = [w, w2]
    b = lb.Batch(ps, [x.rho1 for x in ws], [x.rho2 for x in ws], [x.T0 for x in ws], precision=lb.LB_FP32_SHIFTED)
    b.step(40)
    for r in range(2):
        g = lb.Lattice(ps[r], ws[r].rho1, ws[r].rho2, ws[r].T0, precision=lb.LB_FP32_SHIFTED)
        g.step(40)
        sb, sg = b.stress(r), g.stress()
        assert np.array_equal(sb["sxy"], sg["sxy"]) and np.array_equal(sb["row"], sg["row"])
        assert sb["Sigma"] == sg["Sigma"]
        g.close()
    b.close()


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_couette_stress_on_the_gpu(tau):
    nx, ny, ud, uu = 32, 18, -0.02, 0.03
    p = dict(I.EMULSION_PARAMS, nx=nx, ny=ny, periodic_y=0, tau=tau, G12=0.0, Ga=(0.0, 0.0), Gr=(0.0, 0.0),
             rho_wall=(0.5, 0.5), T_down=0.0, T_up=0.0, alpha_g=0.0, u_wall=(ud, uu))
    g = lb.Lattice(p, 0.6, 0.4, 0.0)
    g.step(6000)
    s = g.stress()
    want = 1.0 * (tau - 0.5) / 3.0 * (uu - ud) / (ny - 2)
    np.testing.assert_allclose(s["sxy"][1:-1], want, rtol=1e-9)
    wf = g.observables()["wall_fx"]
    assert abs(s["Sigma"] + wf[1] / nx) <= 1e-9 * want


def test_sheared_emulsion_stress_balance_on_the_gpu():
    """The oracle pin's momentum balance, run on the GPU path (FP64 storage)."""
    nx, ny = 48, 34
    w = I.emulsion_small(nx=nx, ny=ny, n_drops=2, R=6.0, Ra=0.0)
    p = dict(w.params, alpha_g=0.0, u_wall=(-0.01, 0.01), T_down=0.0, T_up=0.0)
    g = lb.Lattice(p, w.rho1, w.rho2, 0.0)
    g.step(6000)
    S, W = [], []
    for _ in range(200):
        g.step(10)
        S.append(g.stress(field=False)["Sigma"])
        wf = g.observables()["wall_fx"]
        W.append((wf[0] - wf[1]) / (2 * nx))
    S, W = np.mean(S), np.mean(W)
    assert abs(S - W) <= 2e-2 * W, (S, W)
