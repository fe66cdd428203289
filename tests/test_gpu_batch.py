"""Batched ensembles through the lb_batch_* C ABI: every replica must evolve exactly as a separate
lattice handle (same fused step, so bit-identical), under both schedules (per-step graph launches and
the persistent kernel with neighbour-tile step counters), and the persistent kernel's bounded waits
must turn a withheld counter into LB_ETIMEOUT instead of a hang."""
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


def _replicas():
    w0 = I.emulsion_hex(96, 40, 3, 1, 0.5, 3e4, seed=11)
    m0 = I.posts_mask(96, 40, 3, 4, 12)
    nx, ny = 130, 70
    y, x = np.mgrid[0:ny, 0:nx]
    r1 = np.where(((x - 60) ** 2 + (y - 30) ** 2) < 20 ** 2, 1.4, 0.1)
    p1 = dict(I.EMULSION_PARAMS, nx=nx, ny=ny, periodic_y=1, T_down=0.0, T_up=0.0, alpha_g=2e-4)
    w2 = I.emulsion_small(seed=3)
    w2.params = dict(w2.params, alpha_g=5e-4)
    return ([w0.params, p1, w2.params], [w0.rho1, r1, w2.rho1], [w0.rho2, 1.5 - r1, w2.rho2],
            [w0.T0, 0.05 * np.sin(2 * np.pi * x / nx), w2.T0], [m0, None, None])


def _singles(params, r1, r2, T0, masks, precision, steps):
    out = []
    for r in range(len(params)):
        g = lb.Lattice(params[r], r1[r], r2[r], T0[r], mask=masks[r], precision=precision)
        g.step(steps)
        out.append(g.get_state())
        g.close()
    return out


@pytest.mark.parametrize("precision", [lb.LB_FP64, lb.LB_FP32_SHIFTED])
@pytest.mark.parametrize("schedule,spl", [(0, 64), (1, 4), (1, 10)])
def test_batch_equals_separate_lattices(precision, schedule, spl):
    params, r1, r2, T0, masks = _replicas()
    b = lb.Batch(params, r1, r2, T0, masks=masks, precision=precision)
    nc = b.info()["tile_candidates"]
    ref = _singles(params, r1, r2, T0, masks, precision, 37)
    for tile in range(nc):
        b2 = lb.Batch(params, r1, r2, T0, masks=masks, precision=precision)
        b2.configure(schedule, tile, spl)
        b2.step(37)
        assert b2.sync() == lb.LB_OK
        for r in range(len(params)):
            np.testing.assert_array_equal(b2.get_state(r), ref[r], err_msg=f"tile {tile} replica {r}")
        assert b2.observables(0)["step"] == 37
        b2.close()
    b.close()


def test_batch_replica_matches_oracle():
    params, r1, r2, T0, masks = _replicas()
    b = lb.Batch(params, r1, r2, T0, masks=masks, precision=lb.LB_FP64)
    b.configure(1, 0, 8)
    b.step(50)
    for r in (0, 1):
        o = O.Oracle(params[r], r1[r], r2[r], T0[r], mask=masks[r])
        o.step(50)
        assert np.abs(b.get_state(r) - o.state).max() <= 1e-12
        ob, oo = b.observables(r), o.observables()
        np.testing.assert_allclose(ob["mass"], oo["mass"], rtol=1e-13)
        assert abs(ob["Nu"] - oo["Nu"]) <= 1e-10


def test_batch_autotune_advances_consistently():
    params, r1, r2, T0, masks = _replicas()
    b = lb.Batch(params, r1, r2, T0, masks=masks, precision=lb.LB_FP32_SHIFTED)
    res = b.autotune(trial_steps=4)
    assert res["steps_taken"] == 2 * 4 * 2 * b.info()["tile_candidates"]
    assert res["schedule"] in (0, 1)
    b.step(6)
    ref = _singles(params, r1, r2, T0, masks, lb.LB_FP32_SHIFTED, res["steps_taken"] + 6)
    for r in range(len(params)):
        np.testing.assert_array_equal(b.get_state(r), ref[r])


def test_persistent_wait_timeout_is_reported_not_hung():
    """Failure detection: CTA 0 of the persistent kernel leaves before the first step barrier; the other
    CTAs' waits there run out after ~1e6 SM cycles, the kernel ends and the host sees LB_ETIMEOUT."""
    params, r1, r2, T0, masks = _replicas()
    b = lb.Batch(params, r1, r2, T0, masks=masks, precision=lb.LB_FP32_SHIFTED)
    b.configure(1, 0, 4)
    b.set_wait_budget(1_000_000, withhold_item=0)
    b.step(4)
    assert b.sync() == lb.LB_ETIMEOUT
    with pytest.raises(lb.LbError) as e:
        b.observables(0)
    assert e.value.code == lb.LB_ETIMEOUT
    b.close()
    # the context stays usable
    g = lb.Lattice(params[2], r1[2], r2[2], T0[2])
    g.step(3)
    assert g.observables()["n_bad"] == 0


def test_full_ensemble_64_replicas_against_oracle():
    """The 64-replica ensemble (16.5 M nodes, uneven sizes) in the launch configuration the benchmark
    times (schedule x tile picked by the autotuner), FP32-shifted; three replicas of different sizes
    checked node by node against the FP64 oracle (OpenMP build) within the FP32 bound."""
    ens = I.ensemble()
    b = lb.Batch([w.params for w in ens], [w.rho1 for w in ens], [w.rho2 for w in ens], [w.T0 for w in ens],
                 precision=lb.LB_FP32_SHIFTED)
    tune = b.autotune(trial_steps=2)
    b.step(4)
    steps = tune["steps_taken"] + 4
    sizes = [w.params["nx"] * w.params["ny"] for w in ens]
    picks = sorted({0, int(np.argmin(sizes)), int(np.argmax(sizes))})
    for r in picks:
        w = ens[r]
        o = O.Oracle(w.params, w.rho1, w.rho2, w.T0, omp=True)
        o.step(steps)
        fb, fo = b.fields(r), o.fields()
        for k in ("rho1", "rho2", "T"):
            rel = np.abs(fb[k] - fo[k]).max() / np.abs(fo[k]).max()
            assert rel <= 1e-4, (r, k, rel)
        np.testing.assert_allclose(b.observables(r)["mass"], o.observables()["mass"], rtol=1e-6)
    b.close()
