"""The GPU discrete adjoint (lb_adjoint_step / lb_adjoint) against the oracle's adjoint and against
central finite differences.

Tolerances: one reverse step and a full short gradient match the FP64 oracle adjoint to rounding
(<= 1e-10 relative); the 512 x 256, 2000-step gradient with sqrt(N) checkpoints matches central
differences (eps = 1e-6) within 1e-3 relative: of the GPU FP64 forward in 32 random directions of T0
and for T_down, and, in FP64 and in FP32-shifted storage, of the FP64 oracle in the 8 directions
stored in tests/golden/adjoint_fd_emulsion_512x256.txt and for T_down."""
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

    assert torch.cuda.is_available()
    B.build()


def _small(nx=37, ny=21, posts=True, Ra=2.5e3):
    w = I.emulsion_small(nx=nx, ny=ny, n_drops=1, R=4.0, Ra=Ra)
    mask = I.posts_mask(nx, ny, 2, 3, 9) if posts else None
    return w, mask


@pytest.mark.parametrize("cJ,with_lam", [(0.0, True), (0.37, True), (1.0, False)])
def test_adjoint_step_matches_oracle(cJ, with_lam):
    w, mask = _small()
    o = O.Oracle(w.params, w.rho1, w.rho2, w.T0, mask=mask)
    o.step(20)
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, mask=mask)
    g.set_state(o.state)
    solid = o.solid().astype(bool)
    lam_next = None
    if with_lam:
        lam_next = I.uniform(77, o.state.size).reshape(o.state.shape) - 0.5
        lam_next[:, solid] = 0.0
    want, want_d = O.adjoint_step(w.params, o.state, lam_next, cJ, mask=mask)
    lam_dev, got_d = g.adjoint_step(None if lam_next is None else g.to_device_vector(lam_next), cJ)
    got = g.from_device_vector(lam_dev)
    scale = np.abs(want).max()
    assert scale > 0
    assert np.abs(got - want).max() <= 1e-10 * scale, np.abs(got - want).max() / scale
    assert abs(got_d - want_d) <= 1e-10 * max(abs(want_d), 1e-12)


@pytest.mark.parametrize("tau,tau_g", [(0.8, 1.0), (0.75, 0.9)])
def test_adjoint_step_with_relaxation_matches_oracle(tau, tau_g):
    """tau or tau_g away from 1 selects the reverse-step kernel that carries the relaxation terms."""
    w, mask = _small()
    params = dict(w.params, tau=tau, tau_g=tau_g)
    o = O.Oracle(params, w.rho1, w.rho2, w.T0, mask=mask)
    o.step(20)
    g = lb.Lattice(params, w.rho1, w.rho2, w.T0, mask=mask)
    g.set_state(o.state)
    solid = o.solid().astype(bool)
    lam_next = I.uniform(78, o.state.size).reshape(o.state.shape) - 0.5
    lam_next[:, solid] = 0.0
    want, want_d = O.adjoint_step(params, o.state, lam_next, 0.37, mask=mask)
    lam_dev, got_d = g.adjoint_step(g.to_device_vector(lam_next), 0.37)
    got = g.from_device_vector(lam_dev)
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-10 * scale, np.abs(got - want).max() / scale
    assert abs(got_d - want_d) <= 1e-10 * max(abs(want_d), 1e-12)


def test_adjoint_gradient_matches_oracle_gradient():
    w, mask = _small(nx=40, ny=24)
    N = 60
    J0, gT0_o, gTd_o = O.adjoint_run(w.params, w.rho1, w.rho2, w.T0, N, mask=mask)
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, mask=mask)
    J, gT0, gTd = g.adjoint(N, ckpt_every=7)  # checkpoint spacing that does not divide N
    assert abs(J - J0) <= 1e-11 * abs(J0)
    assert np.abs(gT0 - gT0_o).max() <= 1e-9 * np.abs(gT0_o).max()
    assert abs(gTd - gTd_o) <= 1e-9 * abs(gTd_o)
    assert g.observables()["step"] == N


def _J_of(w, T0, n, params=None, precision=lb.LB_FP64):
    g = lb.Lattice(params or w.params, w.rho1, w.rho2, T0, mask=w.mask, precision=precision)
    J, _, _ = g.adjoint(n, gradient=False)
    g.close()
    return J


def test_adjoint_512x256_2000_steps_matches_finite_differences():
    """The adjoint workload: 512 x 256 emulsion (phi = 0.7), J over 2000 steps, sqrt(N) = 45
    checkpoints; central differences of the GPU FP64 forward with eps = 1e-6 in 32 random
    directions of T0 and for T_down."""
    w = I.emulsion_512x256()
    N = 2000
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, mask=w.mask)
    J, gT0, gTd = g.adjoint(N, ckpt_every=45)
    g.close()
    eps = 1e-6
    solid = np.zeros_like(w.T0, dtype=bool)
    solid[0, :] = solid[-1, :] = True
    errs = []
    for k in range(32):
        d = I.uniform(500 + k, w.T0.size).reshape(w.T0.shape) - 0.5
        d[solid] = 0.0
        fd = (_J_of(w, w.T0 + eps * d, N) - _J_of(w, w.T0 - eps * d, N)) / (2 * eps)
        ad = float(np.sum(gT0 * d))
        errs.append(abs(ad - fd) / abs(fd))
    assert max(errs) <= 1e-3, errs
    pp = dict(w.params, T_down=w.params["T_down"] + eps)
    pm = dict(w.params, T_down=w.params["T_down"] - eps)
    fd = (_J_of(w, w.T0, N, pp) - _J_of(w, w.T0, N, pm)) / (2 * eps)
    assert abs(gTd - fd) <= 1e-3 * abs(fd), (gTd, fd)


def _golden_fd(golden_dir):
    """Oracle central differences of J on the 512 x 256 workload (tests/golden/make_adjoint_fd.py)."""
    vals = {}
    with open(os.path.join(golden_dir, "adjoint_fd_emulsion_512x256.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = float(v)
    return vals


def _direction(w, seed):
    d = I.uniform(seed, w.T0.size).reshape(w.T0.shape) - 0.5
    d[0, :] = d[-1, :] = 0.0
    return d


@pytest.mark.parametrize("precision", [lb.LB_FP64, lb.LB_FP32_SHIFTED])
def test_adjoint_512x256_matches_oracle_finite_differences(precision, golden_dir):
    """The adjoint workload in both precisions against central differences (eps = 1e-6) of the FP64
    oracle's J over 2000 steps, in the 8 stored directions of T0 and for T_down; the FP32-shifted
    gradient is the gradient of its own FP32 trajectory, held to the same 1e-3 relative bound, and its
    J to 1e-3 of the oracle's (the FP32 bound on the time-averaged Nusselt number)."""
    gold = _golden_fd(golden_dir)
    w = I.emulsion_512x256()
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, mask=w.mask, precision=precision)
    J, gT0, gTd = g.adjoint(2000, ckpt_every=45)
    g.close()
    tolJ = 1e-11 if precision == lb.LB_FP64 else 1e-3
    assert abs(J - gold["J0"]) <= tolJ * abs(gold["J0"]), (J, gold["J0"])
    errs = {}
    for k, fd in gold.items():
        if k.startswith("dir"):
            ad = float(np.sum(gT0 * _direction(w, int(k[3:]))))
            errs[k] = abs(ad - fd) / abs(fd)
    errs["T_down"] = abs(gTd - gold["T_down"]) / abs(gold["T_down"])
    assert len(errs) == 9
    print(f"precision {precision}: max relative error {max(errs.values()):.3e}", errs)
    assert max(errs.values()) <= 1e-3, errs


def test_fp32_adjoint_with_posts_matches_oracle_gradient():
    """FP32-shifted adjoint on a lattice with posts against the FP64 oracle's adjoint gradient:
    J within 1e-3 and the directional derivatives dJ/dT0 . d (8 seeded directions) and dJ/dT_down
    within 1e-3 relative."""
    w, mask = _small(nx=64, ny=40)
    N = 200
    Jo, gT0_o, gTd_o = O.adjoint_run(w.params, w.rho1, w.rho2, w.T0, N, mask=mask)
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, mask=mask, precision=lb.LB_FP32_SHIFTED)
    J, gT0, gTd = g.adjoint(N)
    g.close()
    assert abs(J - Jo) <= 1e-3 * abs(Jo)
    solid = np.zeros_like(w.T0, dtype=bool)
    solid[0, :] = solid[-1, :] = True
    solid |= mask.astype(bool)
    errs = []
    for k in range(8):
        d = I.uniform(900 + k, w.T0.size).reshape(w.T0.shape) - 0.5
        d[solid] = 0.0
        ref = float(np.sum(gT0_o * d))
        errs.append(abs(float(np.sum(gT0 * d)) - ref) / abs(ref))
    errs.append(abs(gTd - gTd_o) / abs(gTd_o))
    assert max(errs) <= 1e-3, errs


def test_autograd_function_gives_the_adjoint_gradient():
    import torch

    w, mask = _small(nx=32, ny=20)
    N = 40
    T0 = torch.tensor(w.T0, dtype=torch.float64, requires_grad=True)
    Td = torch.tensor(w.params["T_down"], dtype=torch.float64, requires_grad=True)
    J = lb.nusselt_mean(T0, Td, w.params, w.rho1, w.rho2, N, mask=mask)
    J.backward()
    Jo, gT0, gTd = O.adjoint_run(w.params, w.rho1, w.rho2, w.T0, N, mask=mask)
    assert abs(J.item() - Jo) <= 1e-11 * abs(Jo)
    np.testing.assert_allclose(T0.grad.numpy(), gT0, rtol=0, atol=1e-9 * np.abs(gT0).max())
    assert abs(Td.grad.item() - gTd) <= 1e-9 * abs(gTd)
