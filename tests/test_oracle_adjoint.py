"""Pins of the oracle's discrete adjoint against central finite differences of the (separately
pinned) forward oracle: the reverse step is the transpose of the step's Jacobian (dot-product test),
the Nusselt seed is the gradient of Eq. NuTime, and the full reverse sweep gives dJ/dT0 and dJ/dT_down
of J = (1/N) sum_{t=1..N} Nu(S_t)."""
import numpy as np
import pytest

import oracle as O
from paper_2109_12565_gb300 import inputs as I

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _case(nx=20, ny=18, steps=8, posts=False, **over):
    w = I.emulsion_small(nx=nx, ny=ny, n_drops=1, R=4.0, Ra=2.5e3)
    params = dict(w.params, **over)
    mask = I.posts_mask(nx, ny, 2, 3, 7) if posts else None
    o = O.Oracle(params, w.rho1, w.rho2, w.T0, mask=mask)
    o.step(steps)  # a state with flow, interfaces and buoyancy
    return params, mask, o.state.copy(), o.solid()


def _step(params, mask, S):
    o = O.Oracle.from_state(params, S, mask=mask)
    o.step(1)
    return o.state


def _nu(params, mask, S):
    return O.Oracle.from_state(params, S, mask=mask).observables()["Nu"]


def _rand_like(seed, S, solid):
    v = I.uniform(seed, S.size).reshape(S.shape) - 0.5
    v[:, solid.astype(bool)] = 0.0
    return v


@pytest.mark.parametrize("posts", [False, True])
def test_adjoint_step_is_transpose_of_step_jacobian(posts):
    params, mask, S, solid = _case(posts=posts)
    v = 1e-2 * _rand_like(101, S, solid)
    lam = _rand_like(102, S, solid)
    eps = 1e-6
    jv = (_step(params, mask, S + eps * v) - _step(params, mask, S - eps * v)) / (2 * eps)
    lam_in, _ = O.adjoint_step(params, S, lam, 0.0, mask=mask)
    lhs, rhs = float(np.sum(lam * jv)), float(np.sum(lam_in * v))
    assert abs(lhs - rhs) <= 1e-7 * max(abs(lhs), 1e-12), (lhs, rhs)


@pytest.mark.parametrize("tau,tau_g", [(0.8, 1.0), (1.0, 0.7), (0.75, 0.9)])
def test_adjoint_step_with_relaxation_is_transpose(tau, tau_g):
    """With tau or tau_g away from 1 the BGK relaxation keeps (1 - 1/tau) f of the population (Eqs. BGK,
    LBMg): the reverse step carries those terms, checked like the tau = 1 case."""
    params, mask, S, solid = _case(posts=True, tau=tau, tau_g=tau_g)
    v = 1e-2 * _rand_like(111, S, solid)
    lam = _rand_like(112, S, solid)
    eps = 1e-6
    jv = (_step(params, mask, S + eps * v) - _step(params, mask, S - eps * v)) / (2 * eps)
    lam_in, _ = O.adjoint_step(params, S, lam, 0.0, mask=mask)
    lhs, rhs = float(np.sum(lam * jv)), float(np.sum(lam_in * v))
    assert abs(lhs - rhs) <= 1e-7 * max(abs(lhs), 1e-12), (lhs, rhs)


def test_adjoint_nusselt_seed_is_gradient_of_nu():
    params, mask, S, solid = _case(steps=30)
    v = 1e-2 * _rand_like(103, S, solid)
    eps = 1e-6
    fd = (_nu(params, mask, S + eps * v) - _nu(params, mask, S - eps * v)) / (2 * eps)
    g, _ = O.adjoint_step(params, S, None, 1.0, mask=mask)
    ad = float(np.sum(g * v))
    assert abs(fd) > 1e-6
    assert abs(ad - fd) <= 1e-6 * abs(fd), (ad, fd)


def test_adjoint_T_down_terms():
    """dT_down enters through the thermal anti-bounce-back of the step and through Eq. NuTime
    (dT in the normalisation and the mirror rule at the bottom wall)."""
    params, mask, S, solid = _case(posts=True)
    lam = _rand_like(104, S, solid)
    eps = 1e-6
    pp, pm = dict(params, T_down=params["T_down"] + eps), dict(params, T_down=params["T_down"] - eps)
    fd_step = float(np.sum(lam * (_step(pp, mask, S) - _step(pm, mask, S)))) / (2 * eps)
    _, d_step = O.adjoint_step(params, S, lam, 0.0, mask=mask)
    assert abs(d_step - fd_step) <= 1e-7 * abs(fd_step)
    fd_nu = (_nu(pp, mask, S) - _nu(pm, mask, S)) / (2 * eps)
    _, d_nu = O.adjoint_step(params, S, None, 1.0, mask=mask)
    assert abs(d_nu - fd_nu) <= 1e-6 * abs(fd_nu), (d_nu, fd_nu)


def test_adjoint_run_gradient_matches_finite_differences():
    """Full reverse sweep: dJ/dT0 along random directions and dJ/dT_down against central differences
    of J (eps = 1e-6, relative error <= 1e-5)."""
    nx, ny, N = 24, 20, 40
    w = I.emulsion_small(nx=nx, ny=ny, n_drops=1, R=4.0, Ra=2.5e3)
    mask = I.posts_mask(nx, ny, 2, 3, 8)
    J, gT0, gTd = O.adjoint_run(w.params, w.rho1, w.rho2, w.T0, N, mask=mask)

    def J_of(T0, params=w.params):
        return O.adjoint_run(params, w.rho1, w.rho2, T0, N, mask=mask)[0]

    eps = 1e-6
    solid = O.Oracle(w.params, w.rho1, w.rho2, w.T0, mask=mask).solid().astype(bool)
    for k in range(3):
        d = I.uniform(200 + k, nx * ny).reshape(ny, nx) - 0.5
        d[solid] = 0.0
        fd = (J_of(w.T0 + eps * d) - J_of(w.T0 - eps * d)) / (2 * eps)
        ad = float(np.sum(gT0 * d))
        assert abs(ad - fd) <= 1e-5 * max(abs(fd), 1e-8), (k, ad, fd)
    pp, pm = dict(w.params, T_down=w.params["T_down"] + eps), dict(w.params, T_down=w.params["T_down"] - eps)
    fd = (J_of(w.T0, pp) - J_of(w.T0, pm)) / (2 * eps)
    assert abs(gTd - fd) <= 1e-5 * abs(fd), (gTd, fd)
    assert np.all(gT0[solid] == 0.0)
