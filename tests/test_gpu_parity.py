"""GPU parity: the CUDA library (through its C ABI) against the FP64 CPU oracle, element by element.

Tolerances (stated per result):
  FP64 GPU vs oracle: max abs <= 1e-11 on every population and field after 1000 steps of the
  64 x 64 emulsion; the two differ only by rounding order (fused multiply-adds, pair-difference
  stencils, reciprocal multiplies) and exp ulps.
  FP32-shifted vs FP64: norm-relative max|d| / max|ref| <= 1e-4 on rho and T after 200 steps,
  <= 1e-3 on the time-averaged Nusselt number.
"""
import numpy as np
import pytest

import oracle as O
from paper_2109_12565_gb300 import build as B
from paper_2109_12565_gb300 import inputs as I
from paper_2109_12565_gb300 import lb

pytestmark = pytest.mark.gpu

# FP32 fluid + FP16 thermal: tolerances on T (norm-relative, 200 steps) and on the time-averaged Nu
FP16T_T_TOL = 3e-3
FP16T_NU_TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()


def _pair(params, r1, r2, T0, mask=None, precision=lb.LB_FP64, omp=False):
    g = lb.Lattice(params, r1, r2, T0, mask=mask, precision=precision)
    o = O.Oracle(params, r1, r2, T0, mask=mask, omp=omp)
    return g, o


def _max_field_diff(fg, fo, keys=("rho1", "rho2", "T", "ux", "uy")):
    return {k: float(np.abs(fg[k] - fo[k]).max()) for k in keys}


@pytest.mark.parametrize("precision", [lb.LB_FP64, lb.LB_DF64])
def test_fp64_emulsion_64x64_1000_steps_matches_oracle(precision):
    """FP64 storage, and double-float storage and arithmetic (LB_DF64), against the FP64 oracle: both
    held to the FP64 bound of 1e-11 after 1000 steps."""
    w = I.emulsion_small()
    g, o = _pair(w.params, w.rho1, w.rho2, w.T0, precision=precision)
    g.step(1000)
    o.step(1000)
    d_state = np.abs(g.get_state() - o.state).max()
    d = _max_field_diff(g.fields(), o.fields())
    print(f"precision {precision}: max |GPU - oracle| state {d_state:.3e}")
    assert d_state <= 1e-11, d_state
    assert max(d.values()) <= 1e-11, d
    og, oo = g.observables(), o.observables()
    np.testing.assert_allclose(og["mass"], oo["mass"], rtol=1e-13)
    np.testing.assert_allclose(og["mom"], oo["mom"], rtol=0, atol=1e-11)
    assert abs(og["Nu"] - oo["Nu"]) <= 1e-10
    assert abs(og["E"] - oo["E"]) <= 1e-14
    assert og["n_fluid"] == oo["n_fluid"] == 64 * 62 and og["n_bad"] == 0
    # the check is not vacuous: the emulsion moves
    assert oo["E"] > 1e-10 and abs(oo["Nu"] - 1.0) > 1e-4


@pytest.mark.parametrize("precision", [lb.LB_FP64, lb.LB_DF64])
@pytest.mark.parametrize("nx,ny,periodic,posts", [
    (37, 21, 0, True),    # ragged in x and y against the 32x16 / 64x16 tiles, posts on both walls
    (70, 35, 1, False),   # periodic, several tiles with ragged tails
    (16, 8, 1, False),
    (8, 8, 0, False),
    (5, 7, 0, False),     # narrower than the 5-wide stencil: x wraps onto itself
    (129, 40, 0, True),
])
def test_fp64_small_and_ragged_lattices(precision, nx, ny, periodic, posts):
    """FP64 within 1e-12 of the oracle after 200 steps; LB_DF64 (48-bit significand) within the FP64
    form's bound, 1e-11."""
    tol = 1e-12 if precision == lb.LB_FP64 else 1e-11
    R = min(nx, ny) / 5.0
    w = I.emulsion_small(nx=nx, ny=ny, n_drops=1, R=max(R, 1.5)) if not periodic else None
    if periodic:
        y, x = np.mgrid[0:ny, 0:nx]
        r1 = np.where((x - nx / 2) ** 2 + (y - ny / 2) ** 2 < (min(nx, ny) / 4) ** 2, 1.4, 0.1)
        r1 = r1 + 1e-3 * (I.uniform(5, nx * ny).reshape(ny, nx) - 0.5)
        params = dict(I.EMULSION_PARAMS, nx=nx, ny=ny, periodic_y=1, T_down=0.0, T_up=0.0, alpha_g=1e-4)
        T0 = 0.1 * np.sin(2 * np.pi * x / nx)
        r2 = 1.5 - r1
        mask = None
    else:
        params, r1, r2, T0 = w.params, w.rho1, w.rho2, w.T0
        params = dict(params, alpha_g=1e-3)
        mask = I.posts_mask(nx, ny, 2, 3, 7) if posts else None
    g, o = _pair(params, r1, r2, T0, mask=mask, precision=precision)
    for n in (1, 16, 183):
        g.step(n)
        o.step(n)
        d_state = np.abs(g.get_state() - o.state).max()
        assert d_state <= tol, (n, d_state)
    d = _max_field_diff(g.fields(), o.fields())
    assert max(d.values()) <= tol, d
    og, oo = g.observables(), o.observables()
    np.testing.assert_allclose(og["mass"], oo["mass"], rtol=1e-13)
    assert abs(og["Nu"] - oo["Nu"]) <= 1e-10
    assert og["n_fluid"] == oo["n_fluid"]


@pytest.mark.parametrize("precision", [lb.LB_FP32_SHIFTED, lb.LB_FP32_FP16T])
@pytest.mark.parametrize("nx,ny,periodic,posts", [(37, 21, 0, True), (5, 7, 0, False), (33, 12, 1, False),
                                                  (129, 40, 0, True)])
def test_fp32_forms_small_odd_and_ragged_lattices(precision, nx, ny, periodic, posts):
    """FP32 storage on lattices narrower than a tile and of odd width (periodic wraps that split a
    pair of region nodes, posts on both walls): rho and T stay within the FP32 (FP16 thermal) bound
    of the FP64 oracle and mass is conserved."""
    if periodic:
        y, x = np.mgrid[0:ny, 0:nx]
        r1 = np.where((x - nx / 2) ** 2 + (y - ny / 2) ** 2 < (min(nx, ny) / 4) ** 2, 1.4, 0.1)
        params = dict(I.EMULSION_PARAMS, nx=nx, ny=ny, periodic_y=1, T_down=0.0, T_up=0.0, alpha_g=1e-4)
        T0 = 0.1 * np.sin(2 * np.pi * x / nx)
        r2, mask = 1.5 - r1, None
    else:
        w = I.emulsion_small(nx=nx, ny=ny, n_drops=1, R=max(min(nx, ny) / 5.0, 1.5))
        params, r1, r2, T0 = dict(w.params, alpha_g=1e-3), w.rho1, w.rho2, w.T0
        mask = I.posts_mask(nx, ny, 2, 3, 7) if posts else None
    g, o = _pair(params, r1, r2, T0, mask=mask, precision=precision)
    g.step(60)
    o.step(60)
    fg, fo = g.fields(), o.fields()
    for k in ("rho1", "rho2"):
        assert _norm_rel(fg[k], fo[k]) <= 1e-4, (k, _norm_rel(fg[k], fo[k]))
    tolT = 1e-4 if precision == lb.LB_FP32_SHIFTED else FP16T_T_TOL
    assert np.abs(fg["T"] - fo["T"]).max() <= tolT * max(np.abs(fo["T"]).max(), 0.5)
    np.testing.assert_allclose(g.observables()["mass"], o.observables()["mass"], rtol=1e-6)


def test_graph_replay_equals_single_launches_bitwise():
    """lb_step(n) replays 16-step CUDA graphs plus single launches; the result is bit-identical
    whatever the split (the kernel is deterministic)."""
    w = I.emulsion_small()
    a = lb.Lattice(w.params, w.rho1, w.rho2, w.T0)
    b = lb.Lattice(w.params, w.rho1, w.rho2, w.T0)
    a.step(37)
    for _ in range(37):
        b.step(1)
    np.testing.assert_array_equal(a.get_state(), b.get_state())
    a.step(0)
    np.testing.assert_array_equal(a.get_state(), b.get_state())
    assert a.observables()["step"] == 37


def test_state_roundtrip_and_restart():
    """lb_set_state / lb_get_state move the exact FP64 populations; a restart from the oracle's state
    continues in step with the oracle."""
    w = I.emulsion_small()
    o = O.Oracle(w.params, w.rho1, w.rho2, w.T0)
    o.step(50)
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0)
    g.set_state(o.state)
    np.testing.assert_array_equal(g.get_state(), o.state)
    g.step(50)
    o.step(50)
    assert np.abs(g.get_state() - o.state).max() <= 1e-12


def test_observables_over_time_match_oracle():
    w = I.emulsion_small()
    g, o = _pair(w.params, w.rho1, w.rho2, w.T0)
    for _ in range(4):
        og, oo = g.observables(), o.observables()
        for k in ("Nu", "E"):
            assert abs(og[k] - oo[k]) <= 1e-10 * max(1.0, abs(oo[k])), (k, og[k], oo[k])
        np.testing.assert_allclose(og["mass"], oo["mass"], rtol=1e-13)
        g.step(100)
        o.step(100)


def _norm_rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def test_fp32_shifted_against_fp64_oracle_200_steps():
    """Precision form: rho and T within 1e-4 (norm-relative) of the FP64 oracle after 200 steps, and
    the Nusselt number averaged over the 200 post-step states within 1e-3."""
    w = I.emulsion_small()
    g, o = _pair(w.params, w.rho1, w.rho2, w.T0, precision=lb.LB_FP32_SHIFTED)
    nu_g, nu_o = [], []
    for _ in range(200):
        g.step(1)
        o.step(1)
        nu_g.append(g.observables()["Nu"])
        nu_o.append(o.observables()["Nu"])
    fg, fo = g.fields(), o.fields()
    for k in ("rho1", "rho2", "T"):
        assert _norm_rel(fg[k], fo[k]) <= 1e-4, (k, _norm_rel(fg[k], fo[k]))
    assert abs(np.mean(nu_g) - np.mean(nu_o)) <= 1e-3 * abs(np.mean(nu_o))
    np.testing.assert_allclose(g.observables()["mass"], o.observables()["mass"], rtol=1e-6)


def test_fp16_thermal_against_fp64_oracle_200_steps():
    """FP32 fluid + FP16 thermal storage: every step rounds the thermal deviations g_i - w_i T_bar to
    FP16 (relative half-ulp 2^-11), so T carries a rounding noise of at most 2^-11 sum_i |g_i - w_i T_bar|
    <= 2^-11 |T - T_bar| ~ 2.4e-4 per step at |T - T_bar| <= 1/2, which diffusion damps; rho sees T
    only through the buoyancy alpha_g T and keeps the FP32 bound."""
    w = I.emulsion_small()
    g, o = _pair(w.params, w.rho1, w.rho2, w.T0, precision=lb.LB_FP32_FP16T)
    nu_g, nu_o = [], []
    for _ in range(200):
        g.step(1)
        o.step(1)
        nu_g.append(g.observables()["Nu"])
        nu_o.append(o.observables()["Nu"])
    fg, fo = g.fields(), o.fields()
    for k in ("rho1", "rho2"):
        assert _norm_rel(fg[k], fo[k]) <= 1e-4, (k, _norm_rel(fg[k], fo[k]))
    assert _norm_rel(fg["T"], fo["T"]) <= FP16T_T_TOL, _norm_rel(fg["T"], fo["T"])
    assert abs(np.mean(nu_g) - np.mean(nu_o)) <= FP16T_NU_TOL * abs(np.mean(nu_o))
    np.testing.assert_allclose(g.observables()["mass"], o.observables()["mass"], rtol=1e-6)


def test_fp16_thermal_state_roundtrip():
    """Set/get of the state rounds g_i - w_i T_bar to FP16 once (relative half-ulp 2^-11) and keeps the
    fluid planes at FP32."""
    w = I.emulsion_small()
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, precision=lb.LB_FP32_FP16T)
    o = O.Oracle(w.params, w.rho1, w.rho2, w.T0)
    wts = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    T_bar = 0.5 * (w.params["T_down"] + w.params["T_up"])
    solid = o.solid().astype(bool)
    dev = o.state[18:] - wts[:, None, None] * T_bar
    dev[:, solid] = 0.0
    bound = 2.0 ** -11 * np.abs(dev) + 1e-12
    for st in (g.get_state(), None):
        if st is None:
            g.set_state(o.state)
            st = g.get_state()
        assert np.abs(st[:18] - o.state[:18]).max() <= 1e-7
        assert np.all(np.abs(st[18:] - o.state[18:]) <= bound)


def test_fp16_thermal_rejected_by_batch_and_adjoint():
    w = I.emulsion_small(nx=32, ny=16, n_drops=1, R=4.0)
    with pytest.raises(lb.LbError) as e:
        lb.batch_workspace_size([w.params], precision=lb.LB_FP32_FP16T)
    assert e.value.code == lb.LB_EINVAL
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, precision=lb.LB_FP32_FP16T)
    with pytest.raises(lb.LbError) as e:
        g.adjoint(4)
    assert e.value.code == lb.LB_EINVAL


def test_fp32_shifted_state_roundtrip():
    w = I.emulsion_small()
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, precision=lb.LB_FP32_SHIFTED)
    o = O.Oracle(w.params, w.rho1, w.rho2, w.T0)
    st = g.get_state()
    assert np.abs(st - o.state).max() <= 1e-7
    g.set_state(o.state)
    assert np.abs(g.get_state() - o.state).max() <= 1e-7


@pytest.mark.parametrize("precision,steps,tol", [(lb.LB_FP64, 12, 1e-12), (lb.LB_FP32_SHIFTED, 12, 1e-4),
                                                 (lb.LB_FP32_FP16T, 12, FP16T_T_TOL), (lb.LB_DF64, 12, 1e-12)])
def test_full_size_1024x512_against_oracle(precision, steps, tol):
    """The 1024 x 512 concentrated emulsion in the launch configuration the benchmark times, checked
    against the oracle on every node (the OpenMP oracle finishes this in seconds)."""
    w = I.emulsion_1024x512()
    g, o = _pair(w.params, w.rho1, w.rho2, w.T0, precision=precision, omp=True)
    import torch

    scratch = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    g.autotune(launches=3, scratch=scratch)  # the benchmark times the tile picked with L2 flushed
    del scratch
    g.step(steps)
    o.step(steps)
    fg, fo = g.fields(), o.fields()
    if precision in (lb.LB_FP64, lb.LB_DF64):
        d = _max_field_diff(fg, fo)
        assert max(d.values()) <= tol, d
        assert np.abs(g.get_state() - o.state).max() <= tol
    else:
        for k in ("rho1", "rho2", "T"):
            assert _norm_rel(fg[k], fo[k]) <= tol, k


def test_rough_channel_4096x2048_full_size_against_oracle():
    """The 4096 x 2048 rough channel (8.4 M nodes, posts on both walls) in the launch configuration
    the benchmark times (cold-L2 autotuned tile), FP32-shifted, against the FP64 oracle (OpenMP)."""
    import torch

    w = I.rough_channel_4096x2048()
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, mask=w.mask, precision=lb.LB_FP32_SHIFTED)
    scratch = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    g.autotune(launches=2, scratch=scratch)
    del scratch
    o = O.Oracle(w.params, w.rho1, w.rho2, w.T0, mask=w.mask, omp=True)
    g.step(5)
    o.step(5)
    fg, fo = g.fields(), o.fields()
    for k in ("rho1", "rho2", "T"):
        assert _norm_rel(fg[k], fo[k]) <= 1e-4, k
    np.testing.assert_allclose(g.observables()["mass"], o.observables()["mass"], rtol=1e-6)


def test_unstable_state_is_reported():
    w = I.emulsion_small(nx=16, ny=16, n_drops=1, R=3.0)
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0)
    st = g.get_state()
    st[0, 5, 5] = -10.0  # f_{1,0} at a fluid node: rho_1 < 0
    g.set_state(st)
    obs = g.observables(check=False)
    assert obs["status"] == lb.LB_EUNSTABLE and obs["n_bad"] == 1
    with pytest.raises(lb.LbError) as e:
        g.observables()
    assert e.value.code == lb.LB_EUNSTABLE


def test_init_errors():
    import ctypes

    import torch

    w = I.emulsion_small(nx=16, ny=16, n_drops=1, R=3.0)
    cp = lb.make_params(w.params)
    need = lb.workspace_size(w.params)
    small = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
    h = ctypes.c_void_p()
    r = [np.ascontiguousarray(a, dtype=np.float64) for a in (w.rho1, w.rho2, w.T0)]
    dp = [a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) for a in r]
    rc = lb.lib().lb_init(ctypes.byref(h), ctypes.byref(cp), None, *dp, ctypes.c_void_p(small.data_ptr()),
                          small.numel(), None)
    assert rc == lb.LB_ENOSPACE
    assert b"workspace" in lb.lib().lb_last_error(None)
    with pytest.raises(lb.LbError) as e:
        lb.Lattice(dict(w.params, periodic_y=1), w.rho1, w.rho2, w.T0, mask=np.ones((16, 16), np.uint8))
    assert e.value.code == lb.LB_EINVAL
    bad = w.rho1.copy()
    bad[4, 4] = 0.0
    with pytest.raises(lb.LbError) as e:
        lb.Lattice(w.params, bad, w.rho2, w.T0)
    assert e.value.code == lb.LB_EINVAL


@pytest.mark.parametrize("precision", [lb.LB_FP64, lb.LB_FP32_SHIFTED, lb.LB_FP32_FP16T, lb.LB_DF64])
@pytest.mark.parametrize("periodic", [0, 1])
@pytest.mark.parametrize("nx,ny", [(300, 130), (277, 45)])
def test_every_tile_candidate_gives_identical_results(precision, periodic, nx, ny):
    """Tile shapes only change which CTA computes a node and how its inputs reach shared memory, never
    the arithmetic of a node: every autotuner candidate must give bit-identical populations (fast
    interior path, general path, ragged and odd-width tiles, periodic wrap)."""
    if periodic:
        y, x = np.mgrid[0:ny, 0:nx]
        r1 = np.where(((x - nx // 2) ** 2 + (y - ny // 2) ** 2) < (ny // 3) ** 2, 1.4, 0.1)
        # tau != 1 also runs the relaxation branch (populations read back in phase B)
        params = dict(I.EMULSION_PARAMS, nx=nx, ny=ny, periodic_y=1, T_down=0.0, T_up=0.0, alpha_g=1e-4,
                      tau=0.8, tau_g=0.9)
        T0 = 0.1 * np.sin(2 * np.pi * x / nx)
        mask = None
    else:
        w = I.emulsion_hex(nx, ny, 6, 2, 0.6, 3e4, seed=9)
        params, r1, T0 = w.params, w.rho1, w.T0
        mask = I.posts_mask(nx, ny, 4, 5, 25)
    ref = None
    n_cand = None
    for k in range(64):
        g = lb.Lattice(params, r1, 1.5 - r1, T0, mask=mask, precision=precision)
        n_cand = g.tile_info(0)["candidates"]
        if k >= n_cand:
            break
        g.set_tile(k)
        g.step(21)
        st = g.get_state()
        if ref is None:
            ref = st
        else:
            np.testing.assert_array_equal(st, ref, err_msg=f"candidate {k}")
    assert n_cand >= 2


def test_autotune_keeps_state_and_picks_a_candidate():
    w = I.emulsion_small()
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, precision=lb.LB_FP32_SHIFTED)
    g.step(3)
    before = g.get_state()
    k, ms = g.autotune(launches=3)
    assert 0 <= k < len(ms) and all(m > 0 for m in ms)
    assert ms[k] == min(ms)
    np.testing.assert_array_equal(g.get_state(), before)
    assert g.observables()["step"] == 3
    g.step(5)
    h = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, precision=lb.LB_FP32_SHIFTED)
    h.step(8)
    np.testing.assert_array_equal(g.get_state(), h.get_state())


def test_cold_autotune_keeps_state_and_needs_scratch():
    import ctypes

    import torch

    w = I.emulsion_small()
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, precision=lb.LB_FP32_SHIFTED)
    g.step(4)
    before = g.get_state()
    scratch = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    k, ms = g.autotune(launches=2, scratch=scratch)
    assert 0 <= k < len(ms) and ms[k] == min(ms) and all(m > 0 for m in ms)
    np.testing.assert_array_equal(g.get_state(), before)
    assert g.tile_info()["tx"] == g.tile_info(k)["tx"]
    chosen = ctypes.c_int()
    rc = lb.lib().lb_autotune_cold(g._h, 2, None, 0, ctypes.byref(chosen), None, 0)
    assert rc == lb.LB_EINVAL


def test_fresh_handle_reports_no_error_on_reused_memory():
    """The workspace's error word starts at zero even when the caller's memory held other data."""
    import torch

    w = I.emulsion_small(nx=16, ny=16, n_drops=1, R=3.0)
    junk = torch.full((lb.workspace_size(w.params) // 4 + 64,), -1, dtype=torch.int32, device="cuda")
    del junk  # the caching allocator hands this memory to the next workspace
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0)
    g.step(2)
    g.sync()
    assert g.observables()["status"] == lb.LB_OK


def test_df64_state_roundtrip_and_rejections():
    """LB_DF64: lb_set_state splits each FP64 population into a double-float pair and lb_get_state
    adds the pair back, so a round trip loses at most 2^-48 relative; batches and the adjoint, which
    exist for FP64 and FP32-shifted storage, reject the form."""
    w = I.emulsion_small()
    o = O.Oracle(w.params, w.rho1, w.rho2, w.T0)
    o.step(30)
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, precision=lb.LB_DF64)
    g.set_state(o.state)
    back = g.get_state()
    assert np.abs(back - o.state).max() <= 2.0 ** -48 * np.abs(o.state).max()
    g.step(40)
    o.step(40)
    assert np.abs(g.get_state() - o.state).max() <= 1e-11
    with pytest.raises(lb.LbError) as e:
        g.adjoint(4)
    assert e.value.code == lb.LB_EINVAL
    with pytest.raises(lb.LbError) as e:
        lb.Batch([w.params], [w.rho1], [w.rho2], [w.T0], precision=lb.LB_DF64)
    assert e.value.code == lb.LB_EINVAL
