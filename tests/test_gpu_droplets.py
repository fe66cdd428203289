"""GPU droplet topology (lb_droplets*) against the oracle (Sec. 2.4, definitions D1-D6).

The oracle analyses the very rho_1 field the GPU pipeline reads (lb_get_fields runs the same
field kernel), so the comparison is exact: labels and ids (integer), centres (bit-identical: the
same integer sums and the same IEEE divisions), Voronoi colours (the same unfused double distances
and tie rule) and the link set.  At the 4096 x 2048 rough-channel size the brute-force oracle
Voronoi is too slow; there the colours are checked on sampled nodes and the links against the
exact Delaunay triangulation of the centres.
"""
import numpy as np
import pytest

import oracle as O
from paper_2109_12565_gb300 import build as B
from paper_2109_12565_gb300 import inputs as I
from paper_2109_12565_gb300 import lb

pytestmark = pytest.mark.gpu

BTH = 0.8  # bubble threshold on rho_1 (the droplets hold ~1.4, the continuous phase ~0.1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()


def _compare(g, d, params, mask=None, threshold=BTH):
    r1 = g.fields()["rho1"]
    solid = O.Oracle(params, 1.0, 1.0, 0.0, mask=mask).solid().astype(bool)
    assert np.all(np.abs(r1[~solid] - threshold) > 1e-12), "a node sits on the threshold"
    o = O.droplets(params, r1, threshold, mask=mask)
    assert d["n"] == o["n"]
    np.testing.assert_array_equal(d["label"], o["label"])
    np.testing.assert_array_equal(d["size"], o["size"])
    assert np.array_equal(d["cx"], o["cx"]) and np.array_equal(d["cy"], o["cy"])
    np.testing.assert_array_equal(d["color"], o["color"])
    np.testing.assert_array_equal(d["links"], o["links"])
    return o


@pytest.mark.parametrize("precision", [lb.LB_FP64, lb.LB_FP32_SHIFTED, lb.LB_FP32_FP16T, lb.LB_DF64])
def test_emulsion_64x64_matches_oracle(precision):
    w = I.emulsion_small()
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, precision=precision)
    for steps in (0, 300):
        g.step(steps)
        d = g.droplets(BTH)
        o = _compare(g, d, w.params)
        assert o["n"] == 6 and len(o["links"]) > 6


def test_concentrated_emulsion_1024x512_matches_oracle():
    """The benchmark workload: ~350 droplets at volume fraction 0.8, at the start and after 500
    steps of the coupled dynamics."""
    w = I.emulsion_1024x512()
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, precision=lb.LB_FP32_SHIFTED)
    for steps in (0, 500):
        g.step(steps)
        d = g.droplets(BTH)
        o = _compare(g, d, w.params)
        # at t = 0 the sharp disks of the close packing touch and merge into fewer components
        assert o["n"] > 150 and len(o["links"]) > 2 * o["n"]


@pytest.mark.parametrize("nx,ny,periodic,posts", [(130, 70, 1, False), (97, 61, 0, True), (40, 9, 0, False)])
def test_ragged_periodic_and_posts(nx, ny, periodic, posts):
    rng = np.random.default_rng(nx + ny)
    y, x = np.mgrid[0:ny, 0:nx]
    r1 = np.full((ny, nx), 0.1)
    for _ in range(max(2, nx * ny // 400)):
        cx, cy, R = rng.uniform(0, nx), rng.uniform(0, ny), rng.uniform(2.0, 6.0)
        dx = (x - cx + nx / 2) % nx - nx / 2
        dy = ((y - cy + ny / 2) % ny - ny / 2) if periodic else (y - cy)
        r1[dx * dx + dy * dy < R * R] = 1.4
    params = dict(I.EMULSION_PARAMS, nx=nx, ny=ny, periodic_y=periodic, alpha_g=0.0, T_down=0.0, T_up=0.0)
    mask = I.posts_mask(nx, ny, 3, 4, 16) if posts else None
    g = lb.Lattice(params, r1, 1.5 - r1, 0.0, mask=mask)
    _compare(g, g.droplets(BTH), params, mask=mask)


@pytest.mark.parametrize("nx,ny,periodic,p", [(100, 70, 1, 0.45), (161, 67, 0, 0.62), (33, 200, 1, 0.58)])
def test_percolation_clusters_across_tiles(nx, ny, periodic, p):
    """Site-percolation fields: hundreds of clusters of every shape, near the threshold one that spans
    the lattice through many 32 x 32 labelling tiles and the periodic seams, and centres on the
    integer and half-integer grid, so that many nodes are exactly equidistant from two centres (the
    tie rule); labels, centres, colours and links against the oracle."""
    rng = np.random.default_rng(7 + nx)
    r1 = np.where(rng.random((ny, nx)) < p, 1.4, 0.1)
    params = dict(I.EMULSION_PARAMS, nx=nx, ny=ny, periodic_y=periodic, alpha_g=0.0, T_down=0.0, T_up=0.0)
    g = lb.Lattice(params, r1, 1.5 - r1, 0.0)
    d = g.droplets(BTH, max_drops=nx * ny)
    o = _compare(g, d, params)
    assert o["n"] > 50
    if p > 0.6:  # above the site-percolation threshold: the largest cluster crosses the tile grid
        ys, xs = np.nonzero(d["label"] == np.argmax(d["size"]))
        assert np.ptp(xs) > 64 and np.ptp(ys) > 32


def test_replayed_analyses_follow_the_state():
    """lb_droplets replays a captured launch sequence per (workspace, droplet bound, threshold, current
    buffer), four kept: analyses with steps in between, alternating workspaces, three thresholds and
    both buffer parities (more keys than kept) each match the oracle on the current state."""
    w = I.emulsion_small(nx=96, ny=64, n_drops=5, R=7.0)
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0)
    prev = None
    for steps, th in [(0, BTH), (1, BTH), (5, 0.7), (1, BTH), (2, 0.7), (1, 0.9), (3, BTH), (1, 0.7), (0, BTH)]:
        g.step(steps)
        d = g.droplets(th)
        _compare(g, d, w.params, threshold=th)
        prev, d = d, None  # keep the previous workspace alive, so that the next one lands elsewhere


def test_degenerate_cases():
    w = I.emulsion_small(nx=48, ny=32, n_drops=1, R=5.0)
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0)
    one = g.droplets(BTH)
    assert one["n"] == 1 and one["n_links"] == 0 and np.all(one["color"][1:-1] == 0)
    none = g.droplets(10.0)  # threshold above every density
    assert none["n"] == 0 and none["n_links"] == 0 and np.all(none["color"] == -1) and np.all(none["label"] == -1)
    _compare(g, none, w.params, threshold=10.0)
    big = I.emulsion_small()
    h = lb.Lattice(big.params, big.rho1, big.rho2, big.T0)
    with pytest.raises(lb.LbError) as e:
        h.droplets(BTH, max_drops=3)
    assert e.value.code == lb.LB_ENOSPACE


def test_rough_channel_4096x2048_full_size():
    """~5000 droplets between post-roughened walls: labels and centres exact against the oracle;
    colours on 20000 sampled nodes against a brute-force nearest centre; links against the exact
    Delaunay triangulation (every link a Delaunay edge or a near-degenerate flip, every robust
    interior Delaunay edge a link)."""
    spatial = pytest.importorskip("scipy.spatial")
    w = I.rough_channel_4096x2048()
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0, mask=w.mask, precision=lb.LB_FP32_SHIFTED)
    g.step(300)  # the sharp disks of the initial close packing touch; films form within a few hundred steps
    d = g.droplets(BTH)
    r1 = g.fields()["rho1"]
    nx, ny = w.params["nx"], w.params["ny"]
    lab = np.zeros((ny, nx), dtype=np.int32)
    n = O.ctypes.c_int()
    cp = O.make_params(w.params)
    m = np.ascontiguousarray(w.mask, dtype=np.uint8)
    assert O.lib().orc_droplet_labels(cp, m.ctypes.data_as(O.ctypes.c_void_p), O._dp(np.ascontiguousarray(r1)), BTH,
                                      O._ip(lab), O.ctypes.byref(n)) == 0
    assert d["n"] == n.value > 2000
    np.testing.assert_array_equal(d["label"], lab)
    cx, cy = np.zeros(n.value), np.zeros(n.value)
    assert O.lib().orc_droplet_centres(cp, O._ip(lab), n.value, O._dp(cx), O._dp(cy), None) == 0
    assert np.array_equal(d["cx"], cx) and np.array_equal(d["cy"], cy)
    # sampled colours (brute force over all centres, in chunks)
    rng = np.random.default_rng(0)
    ys, xs = rng.integers(0, ny, 20000), rng.integers(0, nx, 20000)
    solid = (ys == 0) | (ys == ny - 1) | (w.mask[ys, xs] != 0)
    got = d["color"][ys, xs]
    assert np.all(got[solid] == -1)
    for k in range(0, len(xs), 1000):
        sx, sy = xs[k:k + 1000], ys[k:k + 1000]
        dx = sx[:, None] - cx[None, :]
        dx = np.where(dx > nx / 2, dx - nx, np.where(dx < -nx / 2, dx + nx, dx))
        dy = sy[:, None] - cy[None, :]
        d2 = dx * dx + dy * dy
        want = np.argmin(d2, axis=1)
        srt = np.partition(d2, 1, axis=1)
        clear = ~solid[k:k + 1000] & (srt[:, 1] - srt[:, 0] > 1e-9)
        np.testing.assert_array_equal(got[k:k + 1000][clear], want[clear])
    # links against the exact (x-periodic) Delaunay triangulation
    M = n.value
    pts = np.concatenate([np.c_[cx + s * nx, cy] for s in (-1, 0, 1)])
    tri = spatial.Delaunay(pts)
    edges = set()
    for simplex in tri.simplices:
        for i in range(3):
            a, b = simplex[i], simplex[(i + 1) % 3]
            if M <= a < 2 * M or M <= b < 2 * M:
                edges.add((min(a % M, b % M), max(a % M, b % M)))
    links = {(int(a), int(b)) for a, b in d["links"]}
    extra = links - edges
    assert len(extra) <= 0.01 * len(links), len(extra)
    assert len(links & edges) >= 0.97 * len(links)


def _disk_field(nx, ny, centres, R):
    y, x = np.mgrid[0:ny, 0:nx]
    r1 = np.full((ny, nx), 0.1)
    for cx, cy in centres:
        dx = (x - cx + nx / 2) % nx - nx / 2
        r1[dx * dx + (y - cy) ** 2 < R * R] = 1.4
    return r1


def _t1_on_gpu_and_oracle(params, g, state_prev, state_now, d_max):
    g.set_state(state_prev)
    dp = g.droplets(BTH)
    op = O.droplets(params, g.fields()["rho1"], BTH)
    g.set_state(state_now)
    dn = g.droplets(BTH)
    on = O.droplets(params, g.fields()["rho1"], BTH)
    got = g.droplet_t1(dp, dn, d_max)
    want = O.t1_compare(params, op, on, d_max)
    assert got["matched"] == want["matched"]
    assert sorted(map(tuple, got["broken"].tolist())) == want["broken"]
    assert sorted(map(tuple, got["arising"].tolist())) == want["arising"]
    assert sorted(map(tuple, got["t1"].tolist())) == want["t1"]
    return got


def test_t1_quadrilateral_flip_on_gpu():
    nx, ny = 120, 80
    params = dict(I.EMULSION_PARAMS, nx=nx, ny=ny, periodic_y=0, alpha_g=0.0)
    prev_c = [(60.0, 25.0), (60.0, 55.0), (40.0, 40.0), (80.0, 40.0)]
    now_c = [(60.0, 20.0), (60.0, 60.0), (45.0, 40.0), (75.0, 40.0)]
    states = []
    for cs in (prev_c, now_c):
        r1 = _disk_field(nx, ny, cs, 5.0)
        states.append(lb.Lattice(params, r1, 1.5 - r1, 0.5).get_state())
    g = lb.Lattice.from_state(params, states[0])
    got = _t1_on_gpu_and_oracle(params, g, states[0], states[1], 8.0)
    assert got["matched"] == 4 and got["n_t1"] == 1 and got["n_broken"] == 1 and got["n_arising"] == 1


def test_t1_events_of_the_emulsion_dynamics():
    """Two analyses 1000 steps apart of a convecting emulsion with strong buoyancy; the GPU lists
    equal the oracle's on the same fields."""
    w = I.emulsion_512x256()
    params = dict(w.params, alpha_g=20.0 * w.params["alpha_g"])
    g = lb.Lattice(params, w.rho1, w.rho2, w.T0, precision=lb.LB_FP32_SHIFTED)
    g.step(500)
    s0 = g.get_state()
    g.step(1000)
    s1 = g.get_state()
    h = lb.Lattice.from_state(params, s0, precision=lb.LB_FP64)
    got = _t1_on_gpu_and_oracle(params, h, s0, s1, 12.0)
    assert got["matched"] > 0.5 * h.droplets(BTH, arrays=False)["n"]


@pytest.mark.parametrize("precision", [lb.LB_FP64, lb.LB_FP32_SHIFTED])
def test_droplet_nusselt_matches_oracle(precision):
    """Eq. NuDrops at every droplet centre of the convecting 512 x 256 emulsion, bit-identical to the
    oracle on the same fields and centres; in pure conduction every droplet has Nu = 1."""
    w = I.emulsion_512x256()
    params = dict(w.params, alpha_g=10.0 * w.params["alpha_g"])
    g = lb.Lattice(params, w.rho1, w.rho2, w.T0, precision=precision)
    g.step(400)
    d = g.droplets(BTH)
    nu = g.droplet_nusselt(d)
    want = O.droplet_nusselt(params, g.fields(), d["cx"], d["cy"])
    assert d["n"] > 20
    assert np.array_equal(np.isnan(nu), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.array_equal(nu[ok], want[ok])
    assert np.std(nu[ok]) > 1e-3  # the check is not vacuous: the droplets carry different fluxes
    cond = dict(params, alpha_g=0.0, G12=0.0, Ga=(0.0, 0.0), Gr=(0.0, 0.0))
    ny, nx = w.rho1.shape
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    T_lin = params["T_down"] + (params["T_up"] - params["T_down"]) * (y - 0.5) / (ny - 2)
    # uniform total density and no coupling: the summed populations stay at rest exactly, so u = 0 and
    # the linear profile is a fixed point
    h = lb.Lattice(cond, w.rho1, 1.5 - w.rho1, T_lin, precision=precision)
    h.step(5)
    dc = h.droplets(BTH)
    np.testing.assert_allclose(h.droplet_nusselt(dc), 1.0, rtol=0, atol=1e-9 if precision == lb.LB_FP64 else 2e-3)


def test_compare_reports_the_scratch_it_needs():
    """lb_droplets_compare with too small a scratch: LB_ENOSPACE and counts4[0] = KiB needed; with that
    much it succeeds."""
    import ctypes

    import torch

    w = I.emulsion_small()
    g = lb.Lattice(w.params, w.rho1, w.rho2, w.T0)
    a = g.droplets(BTH)
    g.step(50)
    b = g.droplets(BTH)
    counts = (ctypes.c_int * 4)()
    tiny = torch.empty(256, dtype=torch.uint8, device="cuda")
    rc = lb.lib().lb_droplets_compare(g._h, ctypes.c_void_p(a["ws"].data_ptr()), ctypes.c_void_p(b["ws"].data_ptr()),
                                      b["ws_bytes"], 8.0, ctypes.c_void_p(tiny.data_ptr()), 256, counts, None, None,
                                      None, 0)
    assert rc == lb.LB_ENOSPACE and counts[0] > 0
    need = counts[0] * 1024
    big = torch.empty(need, dtype=torch.uint8, device="cuda")
    rc = lb.lib().lb_droplets_compare(g._h, ctypes.c_void_p(a["ws"].data_ptr()), ctypes.c_void_p(b["ws"].data_ptr()),
                                      b["ws_bytes"], 8.0, ctypes.c_void_p(big.data_ptr()), need, counts, None, None,
                                      None, 0)
    assert rc == lb.LB_OK and counts[0] == 6
