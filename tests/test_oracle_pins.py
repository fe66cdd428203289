"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: the expected values are
closed forms of the stencil sums (derived by hand from Fig. 1b), exact
rational identities of the printed weight table, brute-force sums written
as offset loops over the 5x5 box, conservation laws of the lattice
Boltzmann map, and exact steady states.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2109_12565_gb300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _fig1b(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "fig1b_weights.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                r2, n, wn, wd, pn, pd = (int(v) for v in line.split())
                rows.append((r2, n, Fraction(wn, wd), Fraction(pn, pd)))
    return rows


def _weights_by_r2(golden_dir):
    rows = _fig1b(golden_dir)
    return {r2: (w, p) for r2, _, w, p in rows}


# ---------------------------------------------------------------- P2: weight table


def test_fig1b_table_identities(golden_dir):
    """Fig. 1b: sum w = sum p = 1; second moments c_s^2 = 1/3; p is 4th-order isotropic
    (sum p c_x^4 = 4/7 = 3 sum p c_x^2 c_y^2)."""
    wb = _weights_by_r2(golden_dir)
    links = [(dx, dy) for dx in range(-2, 3) for dy in range(-2, 3)]
    sw = sum(wb[dx * dx + dy * dy][0] for dx, dy in links)
    sp = sum(wb[dx * dx + dy * dy][1] for dx, dy in links)
    assert sw == 1 and sp == 1
    assert sum(wb[dx * dx + dy * dy][0] * dx * dx for dx, dy in links) == Fraction(1, 3)
    assert sum(wb[dx * dx + dy * dy][1] * dx * dx for dx, dy in links) == Fraction(1, 3)
    assert sum(wb[dx * dx + dy * dy][1] * dx ** 4 for dx, dy in links) == Fraction(4, 7)
    assert sum(wb[dx * dx + dy * dy][1] * dx * dx * dy * dy for dx, dy in links) == Fraction(4, 21)
    # link counts per shell
    for r2, n, _, _ in _fig1b(golden_dir):
        assert sum(1 for dx, dy in links if dx * dx + dy * dy == r2) == n


def test_oracle_tables_match_fig1b(golden_dir):
    wb = _weights_by_r2(golden_dir)
    c, w, p = O.tables()
    seen = set()
    for i in range(25):
        r2 = int(c[i, 0] ** 2 + c[i, 1] ** 2)
        seen.add((int(c[i, 0]), int(c[i, 1])))
        assert p[i] == pytest.approx(float(wb[r2][1]), abs=1e-17)
        if i < 9:
            assert w[i] == pytest.approx(float(wb[r2][0]), abs=1e-17)
            assert r2 <= 2
    assert len(seen) == 25  # all 25 offsets of the 5x5 box, each once
    # D2Q9 opposite pairs within 1..8 and the i=0 rest link
    assert tuple(c[0]) == (0, 0)


# ---------------------------------------------------------------- P1: forces, closed forms


def _S_w(kx, ky):
    """sum_i w_i sin(k.c_i) c_i over the D2Q9 links, by hand from Fig. 1b."""
    return np.array([math.sin(kx) / 9.0 * (2.0 + math.cos(ky)), math.sin(ky) / 9.0 * (2.0 + math.cos(kx))])


def _S_p(kx, ky):
    """sum_i p_i sin(k.c_i) c_i over the 24 links of both belts, by hand from Fig. 1b."""
    a, q, b, d, e = 4 / 63, 4 / 135, 1 / 180, 2 / 945, 1 / 15120

    def comp(k1, k2):
        return (2 * a * math.sin(k1) + 4 * q * math.sin(k1) * math.cos(k2) + 4 * b * math.sin(2 * k1)
                + 4 * d * math.sin(k1) * math.cos(2 * k2) + 8 * d * math.sin(2 * k1) * math.cos(k2)
                + 8 * e * math.sin(2 * k1) * math.cos(2 * k2))

    return np.array([comp(kx, ky), comp(ky, kx)])


def _periodic_params(nx, ny, **kw):
    p = dict(nx=nx, ny=ny, periodic_y=1, tau=1.0, tau_g=1.0, rho0=0.83, G12=0.0, Ga=(0.0, 0.0),
             Gr=(0.0, 0.0), rho_wall=(0.612, 0.612), T_down=0.0, T_up=0.0, alpha_g=0.0, body_fx=0.0)
    p.update(kw)
    return p


@pytest.mark.parametrize("m,n", [(1, 0), (0, 1), (3, 2), (5, 3), (2, 5)])
@pytest.mark.parametrize("comp", [0, 1])
def test_force_plane_wave_closed_forms(m, n, comp):
    """Eqs. (FAB), (FintAttrattive), (FintRepulsive) on plane waves psi = A + B sin(k.x): each stencil
    sum equals B cos(k.x) S(k) with S(k) the closed forms above; one coupling at a time."""
    nx, ny = 16, 12
    rho0 = 0.83
    kx, ky = 2 * math.pi * m / nx, 2 * math.pi * n / ny
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    th = kx * x + ky * y
    A, B = 0.4, 0.15
    psi = A + B * np.sin(th)
    other = comp ^ 1
    rnd = 0.3 + I.uniform(7 + m + 10 * n, nx * ny).reshape(ny, nx)  # arbitrary positive field
    # F^x: psi~ of the OTHER component is the plane wave; this component's rho is arbitrary
    rho = [None, None]
    rho[other] = rho0 * psi
    rho[comp] = rnd
    G12 = 0.37
    F = O.forces(_periodic_params(nx, ny, G12=G12), rho[0], rho[1], 0.0)
    want = -G12 * (rho[comp] / rho0)[None] * B * np.cos(th)[None] * _S_w(kx, ky)[:, None, None]
    np.testing.assert_allclose(F[comp], want, rtol=0, atol=1e-14)
    # F^a and F^r: psi_l = rho0 (1 - exp(-rho_l/rho0)) of THIS component is the plane wave
    rho = [rnd, rnd.copy()]
    rho[comp] = -rho0 * np.log(1.0 - psi / rho0)
    G = [0.0, 0.0]
    G[comp] = -2.3
    F = O.forces(_periodic_params(nx, ny, Ga=tuple(G)), rho[0], rho[1], 0.0)
    want = -G[comp] * psi[None] * B * np.cos(th)[None] * _S_w(kx, ky)[:, None, None]
    np.testing.assert_allclose(F[comp], want, rtol=0, atol=1e-14)
    G[comp] = 1.9
    F = O.forces(_periodic_params(nx, ny, Gr=tuple(G)), rho[0], rho[1], 0.0)
    want = -G[comp] * psi[None] * B * np.cos(th)[None] * _S_p(kx, ky)[:, None, None]
    np.testing.assert_allclose(F[comp], want, rtol=0, atol=1e-14)


def test_force_buoyancy_and_body_force():
    """Eq. (alphaG): F^ext_l = rho_l alpha g T e_y (plus the constant x acceleration), no interaction."""
    nx, ny = 6, 5
    r1 = 0.2 + I.uniform(11, nx * ny).reshape(ny, nx)
    r2 = 0.2 + I.uniform(12, nx * ny).reshape(ny, nx)
    T = I.uniform(13, nx * ny).reshape(ny, nx) - 0.5
    F = O.forces(_periodic_params(nx, ny, alpha_g=0.01, body_fx=2e-5), r1, r2, T)
    for l, r in enumerate((r1, r2)):
        np.testing.assert_allclose(F[l, 1], r * 0.01 * T, rtol=1e-15, atol=0)
        np.testing.assert_allclose(F[l, 0], r * 2e-5, rtol=1e-15, atol=0)


def test_force_brute_force_8x8_with_walls_and_obstacles(golden_dir):
    """P1: the full interaction force on an 8x8 random field with wall rows and obstacle nodes,
    against an offset loop over the 5x5 box with weights looked up from Fig. 1b by |c|^2."""
    wb = _weights_by_r2(golden_dir)
    nx, ny = 8, 8
    prm = dict(nx=nx, ny=ny, periodic_y=0, tau=1.0, tau_g=1.0, rho0=0.83, G12=0.405, Ga=(-9.0, -8.0),
               Gr=(8.1, 7.1), rho_wall=(0.9, 0.2), T_down=0.0, T_up=0.0, alpha_g=0.0, body_fx=0.0)
    mask = np.zeros((ny, nx), np.uint8)
    mask[3, 2] = mask[4, 6] = 1
    r1 = 0.1 + 1.3 * I.uniform(21, nx * ny).reshape(ny, nx)
    r2 = 0.1 + 1.3 * I.uniform(22, nx * ny).reshape(ny, nx)
    F = O.forces(prm, r1, r2, 0.0, mask=mask)

    solid = mask.astype(bool).copy()
    solid[0, :] = solid[ny - 1, :] = True
    rho = (r1, r2)
    rho0 = prm["rho0"]

    def val(l, x, y, kind):
        x %= nx
        if y < 0 or y >= ny or solid[y, x]:
            r = prm["rho_wall"][l]
        else:
            r = rho[l][y, x]
        return r / rho0 if kind == "lin" else rho0 * (1 - math.exp(-r / rho0))

    want = np.zeros_like(F)
    for y in range(ny):
        for x in range(nx):
            if solid[y, x]:
                continue
            for l in range(2):
                m = 1 - l
                acc = np.zeros(2)
                for dx in range(-2, 3):
                    for dy in range(-2, 3):
                        r2_ = dx * dx + dy * dy
                        w, p = float(wb[r2_][0]), float(wb[r2_][1])
                        cvec = np.array([dx, dy], float)
                        acc += -prm["G12"] * val(l, x, y, "lin") * w * val(m, x + dx, y + dy, "lin") * cvec
                        acc += -prm["Ga"][l] * val(l, x, y, "exp") * w * val(l, x + dx, y + dy, "exp") * cvec
                        acc += -prm["Gr"][l] * val(l, x, y, "exp") * p * val(l, x + dx, y + dy, "exp") * cvec
                want[l, :, y, x] = acc
    np.testing.assert_allclose(F, want, rtol=0, atol=1e-13)


def test_force_at_flat_walls_closed_form():
    """Sec. 2.2.1: wall rows and the ghost rows beyond them carry rho_w.  For a uniform fluid the
    force is then a closed form on the first two rows next to each wall and zero further in."""
    nx, ny = 6, 12
    rho0 = 0.83
    prm = dict(nx=nx, ny=ny, periodic_y=0, tau=1.0, tau_g=1.0, rho0=rho0, G12=0.3, Ga=(-2.0, -1.0),
               Gr=(1.5, 1.1), rho_wall=(0.9, 0.15), T_down=0.0, T_up=0.0, alpha_g=0.0, body_fx=0.0)
    rf = (0.7, 0.5)
    F = O.forces(prm, np.full((ny, nx), rf[0]), np.full((ny, nx), rf[1]), 0.0)
    lin = lambda r: r / rho0  # noqa: E731
    ex = lambda r: rho0 * (1 - math.exp(-r / rho0))  # noqa: E731
    s_w1 = -(1 / 9 + 2 / 36)                        # sum over c_y = -1 of w_i c_iy
    s_p1 = -(4 / 63 + 2 * 4 / 135 + 2 * 2 / 945)     # sum over c_y = -1 of p_i c_iy
    s_p2 = -2 * (1 / 180 + 2 * 2 / 945 + 2 / 15120)  # sum over c_y = -2 of p_i c_iy
    for l in range(2):
        m = 1 - l
        dl = lin(prm["rho_wall"][m]) - lin(rf[m])
        de = ex(prm["rho_wall"][l]) - ex(rf[l])
        row1 = (-prm["G12"] * lin(rf[l]) * dl * s_w1 - prm["Ga"][l] * ex(rf[l]) * de * s_w1
                - prm["Gr"][l] * ex(rf[l]) * de * (s_p1 + s_p2))
        row2 = -prm["Gr"][l] * ex(rf[l]) * de * s_p2
        np.testing.assert_allclose(F[l, 1, 1], row1, rtol=1e-13)
        np.testing.assert_allclose(F[l, 1, 2], row2, rtol=1e-13)
        np.testing.assert_allclose(F[l, 1, ny - 2], -row1, rtol=1e-13)
        np.testing.assert_allclose(F[l, 1, ny - 3], -row2, rtol=1e-13)
        np.testing.assert_allclose(F[l, 1, 3:ny - 3], 0.0, atol=1e-15)
        np.testing.assert_allclose(F[l, 0], 0.0, atol=1e-15)


# ---------------------------------------------------------------- P3-P6, P12: invariants


def test_uniform_state_is_fixed_point():
    """P3: a uniform periodic mixture at rest has F = 0 and f = w_i rho is a fixed point."""
    nx, ny = 8, 6
    prm = _periodic_params(nx, ny, G12=0.405, Ga=(-9.0, -8.0), Gr=(8.1, 7.1))
    o = O.Oracle(prm, 0.7, 0.6, 0.3)
    s0 = o.state.copy()
    o.step(50)
    np.testing.assert_allclose(o.state, s0, rtol=0, atol=1e-15)


def test_mass_conservation_walls_and_posts():
    """P4: per-component mass is conserved by BGK + streaming + half-way bounce-back (1000 steps,
    emulsion with buoyancy, flat walls and rectangular posts)."""
    w = I.emulsion_small()
    mask = I.posts_mask(64, 64, 4, 4, 16)
    o = O.Oracle(w.params, w.rho1, w.rho2, w.T0, mask=mask)
    m0 = o.observables()["mass"]
    o.step(1000)
    obs = o.observables()
    assert obs["n_bad"] == 0
    np.testing.assert_allclose(obs["mass"], m0, rtol=1e-12)


def _equilibrium_state(rho1, rho2, T, ux, uy):
    """Populations at a given velocity (initial condition only): second-order Maxwellian."""
    c = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)], float)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    st = []
    for a in (rho1, rho2, T):
        for i in range(9):
            cu = c[i, 0] * ux + c[i, 1] * uy
            st.append(w[i] * a * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy)))
    return np.array(st)


def test_momentum_conservation_periodic():
    """P5: with no external force the pair terms of F^int cancel over a periodic lattice, so the
    total momentum sum rho u^(H) is conserved (200 steps of a phase-separating emulsion)."""
    nx, ny = 24, 20
    prm = _periodic_params(nx, ny, G12=0.405, Ga=(-9.0, -8.0), Gr=(8.1, 7.1))
    r1 = 0.1 + 1.3 * (I.uniform(31, nx * ny).reshape(ny, nx) > 0.5)
    r2 = 1.5 - r1
    ux = 0.02 * (I.uniform(32, nx * ny).reshape(ny, nx) - 0.5)
    uy = 0.02 * (I.uniform(33, nx * ny).reshape(ny, nx) - 0.5)
    o = O.Oracle.from_state(prm, _equilibrium_state(r1, r2, np.zeros_like(r1), ux, uy))
    p0 = o.observables()["mom"]
    assert np.abs(p0).max() > 1e-2
    o.step(200)
    np.testing.assert_allclose(o.observables()["mom"], p0, rtol=0, atol=1e-11)


@pytest.mark.parametrize("tau_g", [1.0, 0.8, 1.7])
def test_pure_conduction_linear_profile_and_unit_nusselt(tau_g):
    """P6: with no flow the anti-bounce-back thermal walls keep the linear conduction profile
    exactly (walls half-way), and Eq. (NuTime) gives Nu = 1."""
    nx, ny = 8, 34
    prm = dict(nx=nx, ny=ny, periodic_y=0, tau=1.0, tau_g=tau_g, rho0=0.83, G12=0.0, Ga=(0.0, 0.0),
               Gr=(0.0, 0.0), rho_wall=(0.5, 0.5), T_down=0.5, T_up=-0.5, alpha_g=0.0, body_fx=0.0)
    T0 = I.linear_T(nx, ny, 0.5, -0.5)
    o = O.Oracle(prm, 0.5, 0.5, T0)
    o.step(300)
    f = o.fields()
    np.testing.assert_allclose(f["T"][1:-1], T0[1:-1], rtol=0, atol=1e-13)
    obs = o.observables()
    assert abs(obs["Nu"] - 1.0) < 1e-12
    assert obs["E"] < 1e-28


def test_conduction_relaxes_to_linear_profile():
    """P6 from a uniform start: T relaxes to the linear profile between T_down and T_up."""
    nx, ny = 4, 18
    prm = dict(nx=nx, ny=ny, periodic_y=0, tau=1.0, tau_g=1.0, rho0=0.83, G12=0.0, Ga=(0.0, 0.0),
               Gr=(0.0, 0.0), rho_wall=(0.5, 0.5), T_down=1.0, T_up=0.0, alpha_g=0.0, body_fx=0.0)
    o = O.Oracle(prm, 0.5, 0.5, 0.5)
    o.step(6000)
    np.testing.assert_allclose(o.fields()["T"][1:-1], I.linear_T(nx, ny, 1.0, 0.0)[1:-1], atol=1e-9)
    assert abs(o.observables()["Nu"] - 1.0) < 1e-8


def test_mirror_symmetry_in_x():
    """P12: a state symmetric under x -> -x stays symmetric (rho, T even; u_x odd)."""
    w = I.emulsion_small(nx=32, ny=32, n_drops=2, R=5.0)
    r1 = 0.5 * (w.rho1 + w.rho1[:, ::-1])
    r2 = 1.5 - r1
    T = w.T0 + 0.01 * np.cos(2 * np.pi * (np.arange(32) + 0.5) / 32)[None, :]
    T = 0.5 * (T + T[:, ::-1])
    # mirror axis x -> 31 - x keeps both fields invariant
    np.testing.assert_array_equal(r1, r1[:, ::-1])
    np.testing.assert_array_equal(T, T[:, ::-1])
    o = O.Oracle(w.params, r1, r2, T)
    o.step(200)
    f = o.fields()
    for k in ("rho1", "rho2", "T", "uy"):
        np.testing.assert_allclose(f[k], f[k][:, ::-1], rtol=0, atol=1e-12)
    np.testing.assert_allclose(f["ux"], -f["ux"][:, ::-1], rtol=0, atol=1e-12)
    assert np.abs(f["ux"]).max() > 1e-6  # the check is not vacuous
