"""Physics pins of the FP64 CPU oracle: results the paper or textbook hydrodynamics fix.

- Appendix B phase-separation table (the paper's only printed simulation
  output), at 128 x 2 after 5e4 steps;
- shear-wave and temperature-mode decay at nu k^2 and kappa k^2 (Eqs. VISCO, K),
  also in a moving frame (Galilean invariance of the second-order equilibrium);
- Poiseuille flow under a body force between half-way bounce-back walls,
  second-order convergent;
- Laplace law for a single droplet (pressure jump linear in 1/R);
- Rayleigh-Benard onset at the rigid-rigid critical Rayleigh number 1708
  (pins the sign and size of the buoyancy of Eq. alphaG and the coupling
  through u^(H)).
"""
import math
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle as O
from paper_2109_12565_gb300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _ideal(nx, ny, periodic_y, **kw):
    p = dict(nx=nx, ny=ny, periodic_y=periodic_y, tau=1.0, tau_g=1.0, rho0=0.83, G12=0.0, Ga=(0.0, 0.0),
             Gr=(0.0, 0.0), rho_wall=(0.5, 0.5), T_down=0.0, T_up=0.0, alpha_g=0.0, body_fx=0.0)
    p.update(kw)
    return p


def _eq_state(r1, r2, T, ux, uy):
    """Initial populations at a prescribed velocity (second-order Maxwellian); initial condition only."""
    c = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)], float)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    out = []
    for a in (r1, r2, T):
        for i in range(9):
            cu = c[i, 0] * ux + c[i, 1] * uy
            out.append(w[i] * a * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy)))
    return np.array(out)


# ---------------------------------------------------------------- P10: Appendix B


def _appB_row(G12):
    w = I.layered(G12=G12)
    o = O.Oracle(w.params, w.rho1, w.rho2, w.T0)
    o.step(50000)
    r1 = o.fields()["rho1"]
    return G12, float(r1.max()), float(r1.min()), float(r1.mean())


def _load_appB(golden_dir):
    rows = {}
    with open(os.path.join(golden_dir, "appB_phase_separation.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                g, a, b = (float(v) for v in line.split())
                rows[round(g, 2)] = (a, b)
    return rows


def test_appendix_b_phase_separation_table(golden_dir):
    """Appendix B: rho_max / rho_min of component 1 after 5e4 steps from the two-layer start.
    The printed "0.40" row was run at the production value G12 = 0.405 (Appendix A table), which
    reproduces it to all printed digits; rows 0.25 and 0.30 sit next to the critical coupling and
    relax slowly, so they get the looser bound."""
    table = _load_appB(golden_dir)
    cases = [0.10, 0.20, 0.25, 0.30, 0.35, 0.405, 0.50, 0.90]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(cases), max(1, O.available_cores()))) as pool:
        got = pool.map(_appB_row, cases)
    for G12, rmax, rmin, rmean in got:
        want = table[0.40 if G12 == 0.405 else round(G12, 2)]
        tol = 5e-5 if G12 in (0.25, 0.30) else 2e-6
        assert abs(rmax - want[0]) <= tol, (G12, rmax, want)
        assert abs(rmin - want[1]) <= tol, (G12, rmin, want)
        # mass of component 1 is conserved: 65 columns at 1.4 and 63 at 0.1 out of 128
        assert abs(rmean - (65 * 1.4 + 63 * 0.1) / 128) < 5e-11  # 5e4 steps of FP64 round-off


# ---------------------------------------------------------------- P7: wave decay


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_shear_wave_and_temperature_mode_decay(tau):
    """Eq. (VISCO) and Eq. (K): a shear wave u_x = U sin(k y) decays at nu k^2, nu = (tau - 1/2)/3, and
    a temperature mode at kappa k^2; k = 2 pi / 64, relative error <= 1e-3."""
    nx, ny = 4, 64
    p = _ideal(nx, ny, 1, tau=tau, tau_g=tau)
    k = 2 * math.pi / ny
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    ux = 1e-3 * np.sin(k * y)
    T = 0.1 * np.sin(k * y)
    o = O.Oracle.from_state(p, _eq_state(0.5 + 0 * ux, 0.5 + 0 * ux, T, ux, 0 * ux))
    obs0 = o.observables()
    assert obs0["E"] == pytest.approx(np.mean(ux * ux), rel=1e-12)
    amp = []
    for n in (100, 500):
        o.step(n)
        f = o.fields()
        s = np.sin(k * y[:, 0])
        amp.append(((f["ux"][:, 0] * s).sum(), (f["T"][:, 0] * s).sum()))
    nu = (tau - 0.5) / 3.0
    rate_u = -math.log(amp[1][0] / amp[0][0]) / 500
    rate_T = -math.log(amp[1][1] / amp[0][1]) / 500
    assert rate_u == pytest.approx(nu * k * k, rel=1e-3)
    assert rate_T == pytest.approx(nu * k * k, rel=1e-3)


def test_advected_shear_wave_galilean_invariance():
    """A shear wave u_y = A sin(k x) carried by a uniform flow U0 along x moves at U0 and decays at
    nu k^2: this needs the quadratic terms of the equilibrium (Sec. 2.1)."""
    nx, ny = 64, 2
    U0, A = 0.05, 1e-3
    p = _ideal(nx, ny, 1)
    k = 2 * math.pi / nx
    x = np.ones((ny, 1)) * np.arange(nx)[None, :]
    o = O.Oracle.from_state(p, _eq_state(0.5 + 0 * x, 0.5 + 0 * x, 0 * x, U0 + 0 * x, A * np.sin(k * x)))
    z = []
    for n in (200, 300):
        o.step(n)
        uy = o.fields()["uy"][0]
        z.append((uy * np.exp(-1j * k * np.arange(nx))).sum())
    dt = 300  # phase advance k U0 dt = 1.5 rad stays below pi
    rate = -math.log(abs(z[1]) / abs(z[0])) / dt
    phase_speed = -np.angle(z[1] / z[0]) / (k * dt)
    nu = 1.0 / 6.0
    assert rate == pytest.approx(nu * k * k, rel=1e-2)
    assert phase_speed == pytest.approx(U0, rel=1e-2)


# ---------------------------------------------------------------- P8: Poiseuille


def _poiseuille_err(ny, tau, steps):
    g = 1e-6
    H = ny - 2
    o = O.Oracle(_ideal(2, ny, 0, tau=tau, body_fx=g), 0.5, 0.5, 0.0)
    o.step(steps)
    f = o.fields()
    y = np.arange(1, ny - 1) - 0.5
    nu = (tau - 0.5) / 3.0
    exact = g / (2 * nu) * y * (H - y)
    assert np.abs(f["uy"]).max() < 1e-12
    return np.abs(f["ux"][1:-1, 0] - exact).max() / exact.max()


@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_poiseuille_profile_second_order(tau):
    """Body force between half-way bounce-back walls (Sec. 2.2, u_w = 0): parabolic u^(H)_x with walls
    at y = 1/2 and y = ny - 3/2; error <= 2.1e-3 at H = 16 and falls ~4x when H doubles."""
    e16 = _poiseuille_err(18, tau, 8000)
    e32 = _poiseuille_err(34, tau, 30000)
    assert e16 < 2.1e-3
    assert 3.5 < e16 / e32 < 4.5


# ---------------------------------------------------------------- P9: Laplace law


def _bulk_pressure(p, r1, r2):
    """Bulk pressure of the model (Eq. Pbulk completed with rho0 and the self-interaction terms; both
    force stencils have second moment c_s^2)."""
    cs2, rho0 = 1.0 / 3.0, p["rho0"]
    pe = lambda r: rho0 * (1 - np.exp(-r / rho0))  # noqa: E731
    return (cs2 * (r1 + r2) + cs2 * p["G12"] * (r1 / rho0) * (r2 / rho0)
            + cs2 / 2 * ((p["Ga"][0] + p["Gr"][0]) * pe(r1) ** 2 + (p["Ga"][1] + p["Gr"][1]) * pe(r2) ** 2))


def _laplace_case(R):
    n = 64
    p = _ideal(n, n, 1, G12=0.405, Ga=(-9.0, -8.0), Gr=(8.1, 7.1))
    y, x = np.mgrid[0:n, 0:n].astype(float)
    inside = (x - n / 2 + 0.5) ** 2 + (y - n / 2 + 0.5) ** 2 <= R * R
    r1 = np.where(inside, 1.4, 0.1)
    o = O.Oracle(p, r1, 1.5 - r1, 0.0)
    o.step(4000)
    f = o.fields()
    P = _bulk_pressure(p, f["rho1"], f["rho2"])
    rin, rout = f["rho1"][n // 2, n // 2], f["rho1"][0, 0]
    Reff = math.sqrt(((f["rho1"] - rout).sum() / (rin - rout)) / math.pi)
    return Reff, P[n // 2, n // 2] - P[0, 0]


def test_laplace_law_single_droplet():
    """Single droplet of component 1 with the paper's interaction set: P_in - P_out = sigma / R + c
    (R measured from the excess mass) with R^2 >= 0.99, sigma > 0 and |c| small against sigma / 8."""
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(4, max(1, O.available_cores()))) as pool:
        res = np.array(pool.map(_laplace_case, [8, 10, 12, 16]))
    A = np.vstack([1 / res[:, 0], np.ones(len(res))]).T
    (sigma, c), *_ = np.linalg.lstsq(A, res[:, 1], rcond=None)
    pred = A @ np.array([sigma, c])
    r2 = 1 - ((res[:, 1] - pred) ** 2).sum() / ((res[:, 1] - res[:, 1].mean()) ** 2).sum()
    assert sigma > 0
    assert r2 >= 0.99
    assert abs(c) < 0.25 * sigma / 8


# ---------------------------------------------------------------- P11: onset of convection


def _mode_amplitude(fac, H=16, steps=(1500, 4500)):
    ny, nx = H + 2, 2 * H
    p = _ideal(nx, ny, 0, T_down=0.5, T_up=-0.5, alpha_g=I.rayleigh_alpha_g(fac * 1708.0, 1.0, H))
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    T0 = I.linear_T(nx, ny, 0.5, -0.5) + 1e-3 * np.sin(2 * np.pi * x / nx) * np.sin(np.pi * (y - 0.5) / H)
    o = O.Oracle(p, 0.5, 0.5, T0)
    amps, t = [], 0
    for s in steps:
        o.step(s - t)
        t = s
        uy = o.fields()["uy"][1:-1]
        amps.append(abs((uy * np.exp(-2j * np.pi * x[1:-1] / nx)).sum()))
    return amps[1] / amps[0], o.observables()["Nu"]


def test_rayleigh_benard_onset_at_1708():
    """Rigid-rigid Rayleigh-Benard: the convective mode (aspect 2, H = 16) decays at Ra = 0.9 x 1708
    and grows at Ra = 1.1 x 1708 (hot bottom wall, Eq. alphaG pushes warm fluid up)."""
    g_below, nu_below = _mode_amplitude(0.9)
    g_above, nu_above = _mode_amplitude(1.1)
    assert g_below < 0.5
    assert g_above > 2.0
    assert abs(nu_below - 1.0) < 1e-3
