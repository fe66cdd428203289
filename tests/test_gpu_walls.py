"""Moving flat walls (Couette, Sec. 2.2 and 3.2.1) and the wall momentum exchange on the GPU.

- FP64: an emulsion sheared between walls moving at -u and +u (posts at rest) equals the oracle
  to 1e-12 on every population after 400 steps, and the x momentum handed to each wall per step
  (lb_obs.wall_fx) equals the oracle's to 1e-12 relative;
- FP32-shifted: the steady Couette profile of an ideal mixture is linear between the half-way walls
  and the wall force equals the viscous stress rho nu (u_up - u_down) / H times nx, within the FP32
  bound (1e-4 relative);
- a batched replica with moving walls equals the separate lattice bitwise; the adjoint refuses
  moving walls.
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

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()


def test_sheared_emulsion_fp64_matches_oracle():
    w = I.emulsion_small(nx=96, ny=48, n_drops=5, R=6.0)
    params = dict(w.params, u_wall=(-0.02, 0.02))
    mask = I.rough_wall_mask(96, 48, 3, 4, 24, alpha=0.4, asymmetric=True, up=False)
    g = lb.Lattice(params, w.rho1, w.rho2, w.T0, mask=mask)
    o = O.Oracle(params, w.rho1, w.rho2, w.T0, mask=mask)
    for n in (1, 399):
        g.step(n)
        o.step(n)
        assert np.abs(g.get_state() - o.state).max() <= 1e-12
    og, oo = g.observables(), o.observables()
    np.testing.assert_allclose(og["wall_fx"], oo["wall_fx"], rtol=1e-12, atol=1e-15)
    assert abs(oo["wall_fx"][1]) > 1e-4  # the moving top wall feels the fluid
    np.testing.assert_allclose(og["mass"], oo["mass"], rtol=1e-13)


@pytest.mark.parametrize("precision", [lb.LB_FP32_SHIFTED, lb.LB_FP64])
def test_couette_profile_and_wall_stress(precision):
    nx, ny, ud, uu, tau = 64, 34, -0.02, 0.03, 0.8
    p = dict(nx=nx, ny=ny, periodic_y=0, tau=tau, tau_g=1.0, rho0=0.83, G12=0.0, Ga=(0.0, 0.0), Gr=(0.0, 0.0),
             rho_wall=(0.5, 0.5), T_down=0.0, T_up=0.0, alpha_g=0.0, body_fx=0.0, u_wall=(ud, uu))
    g = lb.Lattice(p, 0.6, 0.4, 0.0, precision=precision)
    g.step(20000)
    ux = g.fields()["ux"]
    H = ny - 2
    y = np.arange(1, ny - 1)
    want = ud + (uu - ud) * (y - 0.5) / H
    tol = 1e-9 if precision == lb.LB_FP64 else 1e-5
    np.testing.assert_allclose(ux[1:-1, :], want[:, None] * np.ones((1, nx)), rtol=0, atol=tol)
    stress = (tau - 0.5) / 3.0 * (uu - ud) / H  # rho = 1
    wf = g.observables()["wall_fx"]
    np.testing.assert_allclose(wf, [stress * nx, -stress * nx], rtol=1e-8 if precision == lb.LB_FP64 else 1e-4)


def test_batched_replica_with_moving_walls_equals_separate_lattice():
    w = I.emulsion_small(nx=64, ny=40, n_drops=3, R=5.0)
    params = dict(w.params, u_wall=(0.0, 0.015))
    b = lb.Batch([params, w.params], [w.rho1] * 2, [w.rho2] * 2, [w.T0] * 2, precision=lb.LB_FP32_SHIFTED)
    b.step(60)
    g = lb.Lattice(params, w.rho1, w.rho2, w.T0, precision=lb.LB_FP32_SHIFTED)
    g.step(60)
    np.testing.assert_array_equal(b.get_state(0), g.get_state())
    np.testing.assert_array_equal(b.observables(0)["wall_fx"], g.observables()["wall_fx"])
    b.close()


def test_adjoint_refuses_moving_walls():
    w = I.emulsion_small(nx=32, ny=16, n_drops=1, R=4.0)
    g = lb.Lattice(dict(w.params, u_wall=(0.0, 0.01)), w.rho1, w.rho2, w.T0)
    with pytest.raises(lb.LbError) as e:
        g.adjoint(4)
    assert e.value.code == lb.LB_EINVAL
