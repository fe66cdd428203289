"""Pins of the moving-wall (Couette) boundary and the wall momentum exchange of the oracle, and of the
trapezoidal rough-wall generator (Sec. 2.2 flat moving walls, Sec. 3.2.1 rheology, Sec. 5 roughness).

- Couette: between flat walls moving at u_down and u_up, the steady velocity of the half-way
  bounce-back lattice is exactly linear between the half-way walls (y = 1/2, ny - 3/2), for any tau;
- the steady x momentum handed to each wall per step is the viscous stress rho nu du/dy times nx:
  +rho nu (u_up - u_down) / H on the bottom wall and its opposite on the top wall;
- the moving-wall bounce-back conserves the mass of each component (the links crossing a flat
  wall have sum_i w_i c_ix = 0), also with droplets and interaction forces;
- alpha = 0 roughness is the rectangular post mask; symmetric obstacles are mirror-symmetric and
  hold height * width + tan(alpha) height^2 nodes up to rasterisation.
"""
import numpy as np
import pytest

import oracle as O
from paper_2109_12565_gb300 import inputs as I


def _couette(nx, ny, tau, ud, uu):
    return dict(nx=nx, ny=ny, periodic_y=0, tau=tau, tau_g=1.0, rho0=0.83, G12=0.0, Ga=(0.0, 0.0),
                Gr=(0.0, 0.0), rho_wall=(0.5, 0.5), T_down=0.0, T_up=0.0, alpha_g=0.0, body_fx=0.0,
                u_wall=(ud, uu))


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_couette_profile_is_linear_and_wall_force_is_the_viscous_stress(tau):
    nx, ny, ud, uu = 4, 18, -0.02, 0.03
    p = _couette(nx, ny, tau, ud, uu)
    o = O.Oracle(p, 0.6, 0.4, 0.0)
    o.step(6000)
    f = o.fields()
    H = ny - 2
    y = np.arange(1, ny - 1)
    want = ud + (uu - ud) * (y - 0.5) / H
    np.testing.assert_allclose(f["ux"][1:-1, :], want[:, None] * np.ones((1, nx)), rtol=0, atol=1e-12)
    np.testing.assert_allclose(f["uy"][1:-1, :], 0.0, atol=1e-13)
    nu = (tau - 0.5) / 3.0
    stress = 1.0 * nu * (uu - ud) / H
    wf = o.observables()["wall_fx"]
    np.testing.assert_allclose(wf, [stress * nx, -stress * nx], rtol=1e-10, atol=1e-14)


def test_resting_walls_are_unchanged_and_moving_walls_conserve_mass():
    w = I.emulsion_small()
    rest = O.Oracle(w.params, w.rho1, w.rho2, w.T0)
    rest0 = O.Oracle(dict(w.params, u_wall=(0.0, 0.0)), w.rho1, w.rho2, w.T0)
    rest.step(20)
    rest0.step(20)
    assert np.array_equal(rest.state, rest0.state)
    mov = O.Oracle(dict(w.params, u_wall=(-0.01, 0.02)), w.rho1, w.rho2, w.T0, mask=I.posts_mask(64, 64, 3, 4, 16))
    m0 = mov.observables()["mass"]
    mov.step(1000)
    np.testing.assert_allclose(mov.observables()["mass"], m0, rtol=1e-12)
    # the walls drive a shear: the mean x momentum near the top exceeds that near the bottom
    ux = mov.fields()["ux"]
    assert ux[50:62].mean() > ux[2:14].mean() + 1e-3


def test_rough_wall_masks():
    assert np.array_equal(I.rough_wall_mask(96, 40, 8, 8, 32), I.posts_mask(96, 40, 8, 8, 32))
    h, wdt, lam, a = 12, 10, 150, 0.25
    sym = I.rough_wall_mask(600, 60, h, wdt, lam, alpha=a, asymmetric=False, up=False, x0=40)
    asym = I.rough_wall_mask(600, 60, h, wdt, lam, alpha=a, asymmetric=True, up=False, x0=40)
    per = lam  # one obstacle per period
    n_sym = sym.sum() / (600 / per)
    n_asym = asym.sum() / (600 / per)
    t = np.tan(a)
    assert abs(n_sym - (h * wdt + t * h * h)) <= h  # rasterisation: at most one node per row
    assert abs(n_asym - (h * wdt + t * h * h / 2)) <= h
    # a symmetric obstacle is mirror-symmetric about its centre column
    ob = sym[1:1 + h, 0:per * 2][:, 40 - 6:40 + wdt + 6]
    assert np.array_equal(ob, ob[:, ::-1])
    # the asymmetric one keeps a vertical trailing side: column x0 + width is free in every row
    assert not asym[1:1 + h, 40 + wdt].any() and asym[1:1 + h, 40 + wdt - 1].all()
    # top-wall obstacles mirror the bottom ones
    both = I.rough_wall_mask(600, 60, h, wdt, lam, alpha=a)
    assert np.array_equal(both[1:1 + h], both[58 - h + 1:59][::-1])
