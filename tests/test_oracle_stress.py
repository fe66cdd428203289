"""Pins of the oracle's total shear stress (Sec. 2.1, text after Eq. NS; Sec. 3.2.1 rheology):
sigma_xy = eta_0 (d_x u^(H)_y + d_y u^(H)_x) - P^int_xy - P^F_xy with eta_0 = rho (tau - 1/2) / 3
(Eq. VISCO), P^int_xy the virial form of the interaction forces and P^F_xy = tau^2 sum_l F_lx F_ly /
rho_l - F_x F_y / (4 rho) the momentum flux of the forcing of Eq. shift.

- Virial theorem: for pair forces f_{a<-b} = -G W psi_a psi_b (x_b - x_a), the sum over nodes of
  y F_x equals the sum over pairs of G W psi_a psi_b c_x c_y, which is the sum over nodes of P^int_xy
  (half of each pair at each end).  With flat walls (x periodic, y not) it holds exactly for any
  density field: the wall rows add no x force and no xy virial, their pseudo-potential being uniform
  along x.  This pins P^int against the independently pinned forces of Eqs. FAB, FintAttrattive,
  FintRepulsive: a wrong weight, link, sign or component pairing, or c_x^2 in place of c_x c_y,
  breaks it.
- Closed form of the viscous part: with no interaction, a state whose momentum is rho u with
  u_x = u_down + b (y - 1/2) (linear between the moving half-way walls) and u_y = c sin(k x) has
  sigma_xy = rho (tau - 1/2) / 3 (b + c sin(k) cos(k x)) at every fluid node, exactly (the central
  difference of sin(k x) is sin(k) cos(k x); the mirror rule continues the linear profile).
- Steady Couette flow: sigma_xy = rho nu gamma-dot at every fluid node, and the mean stress equals the
  x momentum the top wall receives per step and unit length, -wall_fx[top] / nx.
- Sheared emulsion: the space-time averaged stress balances the wall stress (momentum balance), which
  pins P^F: without it a quarter of the stress is missing.
"""
import numpy as np
import pytest

import oracle as O
from paper_2109_12565_gb300 import inputs as I


def _walled(nx, ny, **kw):
    p = dict(I.EMULSION_PARAMS, nx=nx, ny=ny, periodic_y=0, T_down=1.0, T_up=0.0, alpha_g=0.0, body_fx=0.0,
             u_wall=(0.0, 0.0))
    p.update(kw)
    return p


def _random_densities(nx, ny, seed):
    u = I.uniform(seed, 2 * nx * ny).reshape(2, ny, nx)
    return 0.1 + 1.3 * u[0], 0.1 + 1.3 * u[1]


@pytest.mark.parametrize("G12,rho_wall", [(0.405, (0.612, 0.612)), (0.9, (1.3, 0.2))])
def test_interaction_stress_obeys_the_virial_theorem(G12, rho_wall):
    nx, ny = 40, 30
    p = _walled(nx, ny, G12=G12, rho_wall=rho_wall)
    r1, r2 = _random_densities(nx, ny, 11)
    o = O.Oracle(p, r1, r2, 0.5)
    st = O.stress(p, o.state)
    solid = o.solid().astype(bool)
    F = O.forces(p, r1, r2, 0.5)
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    virial = float(np.sum((y * (F[0, 0] + F[1, 0]))[~solid]))
    psum = float(np.sum(st["pint_field"][~solid]))
    scale = float(np.sum(np.abs(y * (F[0, 0] + F[1, 0]))[~solid]))
    assert scale > 1.0
    assert abs(psum - virial) <= 1e-12 * scale, (psum, virial)
    assert abs(st["pint"] * (~solid).sum() - psum) <= 1e-12 * scale
    # the same holds with the origin of y moved: the interaction forces carry no net momentum
    assert abs(float(np.sum(((y + 7.0) * (F[0, 0] + F[1, 0]))[~solid])) - virial) <= 1e-12 * scale


def test_uniform_state_has_no_shear_stress():
    p = _walled(24, 20)
    o = O.Oracle(p, 1.1, 0.3, 0.5)
    st = O.stress(p, o.state)
    assert np.abs(st["sxy"]).max() <= 1e-15 and abs(st["Sigma"]) <= 1e-15


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_viscous_stress_closed_form(tau):
    nx, ny = 32, 22
    H = ny - 2
    ud, uu, c = -0.015, 0.025, 0.004
    b = (uu - ud) / H
    p = _walled(nx, ny, tau=tau, G12=0.0, Ga=(0.0, 0.0), Gr=(0.0, 0.0), u_wall=(ud, uu))
    r1, r2 = _random_densities(nx, ny, 5)
    o = O.Oracle(p, r1, r2, 0.5)
    k = 2.0 * np.pi / nx
    x = np.arange(nx)[None, :] * np.ones((ny, 1))
    yy = np.arange(ny)[:, None] * np.ones((1, nx))
    ux = ud + b * (yy - 0.5)
    uy = c * np.sin(k * x)
    st = o.state
    solid = o.solid().astype(bool)
    # give every fluid node the momentum rho u without changing its densities: move rho_l u_x / 2 from
    # the -x to the +x link and rho_l u_y / 2 from the -y to the +y link of each component
    for l, r in ((0, r1), (1, r2)):
        st[9 * l + 1] += 0.5 * r * ux
        st[9 * l + 3] -= 0.5 * r * ux
        st[9 * l + 2] += 0.5 * r * uy
        st[9 * l + 4] -= 0.5 * r * uy
    st[:, solid] = 0.0
    s = O.stress(p, st)
    want = (r1 + r2) * (tau - 0.5) / 3.0 * (b + c * np.sin(k) * np.cos(k * x))
    err = np.abs(s["sxy"] - want)[~solid].max()
    assert err <= 1e-14 * np.abs(want).max() * 10, err
    assert np.abs(s["pint_field"]).max() == 0.0
    np.testing.assert_allclose(s["row"][1:-1], want[1:-1].mean(axis=1), rtol=1e-12)


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_couette_stress_is_the_wall_stress(tau):
    nx, ny, ud, uu = 4, 18, -0.02, 0.03
    p = _walled(nx, ny, tau=tau, G12=0.0, Ga=(0.0, 0.0), Gr=(0.0, 0.0), rho_wall=(0.5, 0.5), u_wall=(ud, uu),
                T_down=0.0, T_up=0.0)
    o = O.Oracle(p, 0.6, 0.4, 0.0)
    o.step(6000)
    s = O.stress(p, o.state)
    H = ny - 2
    want = 1.0 * (tau - 0.5) / 3.0 * (uu - ud) / H
    np.testing.assert_allclose(s["sxy"][1:-1], want, rtol=1e-10)
    wf = o.observables()["wall_fx"]
    assert abs(s["Sigma"] - (-wf[1] / nx)) <= 1e-10 * want
    assert abs(s["Sigma"] - wf[0] / nx) <= 1e-10 * want


def test_sheared_emulsion_stress_balances_the_wall_stress():
    """Momentum balance of a sheared emulsion (Couette walls at -+0.01, tau = 1, two droplets of
    radius 6 in 48 x 34): once the shear has developed, the space-time average of sigma_xy equals the
    x momentum the walls take per step and unit length, (wall_fx[bottom] - wall_fx[top]) / (2 nx).
    Measured agreement: 1e-4 to 1e-2 depending on the averaging window; the residual is the
    discretisation of the viscous stress across the density layers at the walls.  The forcing part
    P^F carries about a quarter of the stress here: without it the balance misses by more than 20%."""
    nx, ny = 48, 34
    w = I.emulsion_small(nx=nx, ny=ny, n_drops=2, R=6.0, Ra=0.0)
    p = dict(w.params, alpha_g=0.0, u_wall=(-0.01, 0.01), T_down=0.0, T_up=0.0)
    o = O.Oracle(p, w.rho1, w.rho2, 0.0)
    o.step(6000)
    S, Pf, W = [], [], []
    for _ in range(200):
        o.step(10)
        s = O.stress(p, o.state)
        wf = o.observables()["wall_fx"]
        S.append(s["Sigma"])
        Pf.append(s["pforce"])
        W.append((wf[0] - wf[1]) / (2 * nx))
    S, Pf, W = np.mean(S), np.mean(Pf), np.mean(W)
    assert W > 1e-4
    assert abs(S - W) <= 2e-2 * W, (S, W)
    assert abs((S + Pf) - W) > 0.2 * W
