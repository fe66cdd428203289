"""Pins of the droplet-topology oracle (Sec. 2.4; definitions D1-D6 in oracle/tlb_droplets.c).

Each step is pinned to something other than itself:
- labels: scipy.ndimage.label with 4-connectivity on fields that do not touch the periodic seam
  (both number components in raster order of their first node), plus hand-made periodic cases;
- centres: rasterised disks symmetric about a known centre (exact mean), also across the seam;
- digital Voronoi: a periodic k-d tree nearest-neighbour query (scipy.spatial.cKDTree, boxsize);
- links: the exact Delaunay triangulation of the centres (scipy.spatial.Delaunay on the points
  tiled across the periodic seam): every digital link is a Delaunay edge, and every Delaunay edge
  whose dual Voronoi edge is long and inside the lattice is found;
- T1 detection: a hand-built quadrilateral whose diagonal flips between two frames.
"""
import numpy as np
import pytest

import oracle as O

scipy = pytest.importorskip("scipy")
from scipy import ndimage, spatial  # noqa: E402


def _params(nx, ny, periodic_y=0):
    return dict(nx=nx, ny=ny, periodic_y=periodic_y, tau=1.0, tau_g=1.0, rho0=0.83, G12=0.0, Ga=(0.0, 0.0),
                Gr=(0.0, 0.0), rho_wall=(0.6, 0.6), T_down=0.0, T_up=0.0, alpha_g=0.0, body_fx=0.0)


def _disks(nx, ny, centres, R, periodic_y=False, hi=1.4, lo=0.1):
    y, x = np.mgrid[0:ny, 0:nx]
    rho = np.full((ny, nx), lo)
    for cx, cy in centres:
        dx = (x - cx + nx / 2) % nx - nx / 2
        dy = ((y - cy + ny / 2) % ny - ny / 2) if periodic_y else (y - cy)
        rho[dx * dx + dy * dy < R * R] = hi
    return rho


def test_labels_match_scipy_on_fields_away_from_the_seam():
    rng = np.random.default_rng(3)
    nx, ny = 97, 61
    p = _params(nx, ny)
    rho = np.where(rng.random((ny, nx)) < 0.45, 1.2, 0.3)
    rho[:, 0] = 0.3  # no component crosses the periodic x seam
    d = O.droplets(p, rho, 0.8)
    fg = rho > 0.8
    fg[0, :] = fg[-1, :] = False  # wall rows are solid
    ref, n_ref = ndimage.label(fg, structure=[[0, 1, 0], [1, 1, 1], [0, 1, 0]])
    assert d["n"] == n_ref > 50
    np.testing.assert_array_equal(d["label"] + 1, ref)
    np.testing.assert_array_equal(d["size"], np.bincount(ref.ravel())[1:])


def test_periodic_seams_join_components():
    nx, ny = 40, 30
    p = _params(nx, ny, periodic_y=1)
    rho = np.full((ny, nx), 0.1)
    rho[10:14, 0:3] = 1.4
    rho[10:14, 37:40] = 1.4  # one droplet across x = 0
    rho[0:2, 20:24] = 1.4
    rho[28:30, 20:24] = 1.4  # one droplet across y = 0 (periodic y)
    d = O.droplets(p, rho, 0.8)
    assert d["n"] == 2
    # ids follow the smallest node index: the y-seam droplet starts in row 0
    assert d["label"][0, 20] == 0 and d["label"][10, 0] == 1
    assert d["label"][29, 23] == 0 and d["label"][13, 39] == 1
    np.testing.assert_allclose([d["cx"][1], d["cy"][1]], [39.5, 11.5], atol=0)
    np.testing.assert_allclose([d["cx"][0], d["cy"][0]], [21.5, 29.5], atol=0)
    # with walls the y-seam droplet splits: rows 0 and 29 are solid, rows 1 and 28 stay apart
    w = O.droplets(_params(nx, ny, 0), rho, 0.8)
    assert w["n"] == 3


@pytest.mark.parametrize("cx,cy", [(20.0, 15.0), (20.5, 15.5), (0.5, 15.0), (63.5, 30.0)])
def test_centres_of_symmetric_disks_are_exact(cx, cy):
    nx, ny = 64, 48
    p = _params(nx, ny)
    rho = _disks(nx, ny, [(cx, cy)], 6.3)
    d = O.droplets(p, rho, 0.8)
    assert d["n"] == 1
    assert d["cx"][0] == cx and d["cy"][0] == cy


def test_digital_voronoi_is_the_periodic_nearest_centre():
    rng = np.random.default_rng(11)
    nx, ny = 128, 72
    p = _params(nx, ny)
    cx = rng.uniform(0, nx, 40)
    cy = rng.uniform(1, ny - 1, 40)
    label = -np.ones((ny, nx), dtype=np.int32)
    # droplets of one node each at the rounded centres are not needed: call the Voronoi step directly
    col = np.zeros((ny, nx), dtype=np.int32)
    cp = O.make_params(p)
    rc = O.lib().orc_digital_voronoi(cp, None, O._dp(np.ascontiguousarray(cx)), O._dp(np.ascontiguousarray(cy)),
                                     40, O._ip(col))
    assert rc == 0
    tree = spatial.cKDTree(np.c_[cx, cy], boxsize=[nx, 10 * ny])
    y, x = np.mgrid[0:ny, 0:nx]
    dist, idx = tree.query(np.c_[x.ravel(), y.ravel()], k=2)
    clear = (dist[:, 1] - dist[:, 0]) > 1e-9
    got = col.ravel()
    fluid = (y.ravel() > 0) & (y.ravel() < ny - 1)
    assert np.all(got[~fluid] == -1)
    sel = fluid & clear
    np.testing.assert_array_equal(got[sel], idx[sel, 0])
    assert sel.sum() > 0.99 * fluid.sum()
    del label


def _periodic_delaunay(cx, cy, nx):
    """Exact Delaunay edges and Voronoi ridges of points periodic in x (tiled at x - nx, x, x + nx)."""
    n = len(cx)
    pts = np.concatenate([np.c_[cx + s * nx, cy] for s in (-1, 0, 1)])
    tri = spatial.Delaunay(pts)
    edges = set()
    for simplex in tri.simplices:
        for i in range(3):
            a, b = simplex[i], simplex[(i + 1) % 3]
            if n <= a < 2 * n or n <= b < 2 * n:  # one end in the central copy
                edges.add((min(a % n, b % n), max(a % n, b % n)))
    vor = spatial.Voronoi(pts)
    ridges = {}
    for (a, b), rv in zip(vor.ridge_points, vor.ridge_vertices):
        if not (n <= a < 2 * n or n <= b < 2 * n) or -1 in rv:
            continue
        v0, v1 = vor.vertices[rv[0]], vor.vertices[rv[1]]
        key = (min(a % n, b % n), max(a % n, b % n))
        ridges[key] = (v0, v1)
    return edges, ridges


def test_links_are_the_delaunay_edges():
    rng = np.random.default_rng(5)
    nx, ny = 256, 160
    p = _params(nx, ny)
    # well-separated random centres (minimum distance 14) as disks of radius 4
    pts = []
    while len(pts) < 120:
        c = (rng.uniform(0, nx), rng.uniform(8, ny - 8))
        if all(((c[0] - q[0] + nx / 2) % nx - nx / 2) ** 2 + (c[1] - q[1]) ** 2 > 14.0 ** 2 for q in pts):
            pts.append(c)
    rho = _disks(nx, ny, pts, 4.0)
    d = O.droplets(p, rho, 0.8)
    assert d["n"] == len(pts)
    edges, ridges = _periodic_delaunay(d["cx"], d["cy"], nx)
    links = {(int(a), int(b)) for a, b in d["links"]}
    # a digital link that is not a Delaunay edge must be the other diagonal of a nearly co-circular
    # quadrilateral: it crosses a Delaunay edge whose Voronoi ridge is shorter than the lattice
    # spacing can resolve (< 2 nodes)
    for a, b in links - edges:
        na = {e[0] + e[1] - a for e in edges if a in e}
        nb = {e[0] + e[1] - b for e in edges if b in e}
        common = sorted(na & nb)
        short = [(c, e) for i, c in enumerate(common) for e in common[i + 1:]
                 if (c, e) in ridges and np.hypot(*(ridges[(c, e)][1] - ridges[(c, e)][0])) < 2.0]
        assert short, (a, b)
    assert len(links - edges) <= 3
    robust = set()
    for e, (v0, v1) in ridges.items():
        inside = 1.5 < min(v0[1], v1[1]) and max(v0[1], v1[1]) < ny - 2.5
        if e in edges and inside and np.hypot(*(v1 - v0)) > 3.0:
            robust.add(e)
    assert len(robust) > 200
    assert robust <= links, sorted(robust - links)


def test_t1_flip_of_a_quadrilateral_diagonal():
    nx, ny = 120, 80
    p = _params(nx, ny)
    # a, b on the short diagonal first; then the quadrilateral is stretched the other way
    prev_c = [(60.0, 25.0), (60.0, 55.0), (40.0, 40.0), (80.0, 40.0)]
    now_c = [(60.0, 20.0), (60.0, 60.0), (45.0, 40.0), (75.0, 40.0)]
    prev = O.droplets(p, _disks(nx, ny, prev_c, 5.0), 0.8)
    now = O.droplets(p, _disks(nx, ny, now_c, 5.0), 0.8)
    assert prev["n"] == now["n"] == 4
    res = O.t1_compare(p, prev, now, d_max=8.0)
    assert res["matched"] == 4
    ids = lambda d, c: int(d["label"][int(c[1]), int(c[0])])  # noqa: E731
    a, b, c, dd = (ids(prev, q) for q in prev_c)
    assert res["broken"] == [tuple(sorted((a, b)))]
    assert res["arising"] == [tuple(sorted((c, dd)))]
    assert len(res["t1"]) == 1
    # nothing happens when the frame is compared with itself
    same = O.t1_compare(p, prev, prev, d_max=8.0)
    assert same["broken"] == same["arising"] == same["t1"] == []


def test_droplet_nusselt_closed_forms():
    """Eq. NuDrops: in pure conduction (u = 0, T linear between the half-way walls) every droplet has
    Nu = 1, also next to the walls where the mirror rule enters; a uniform u_y U at uniform T0 gives
    U T0 / (kappa Delta T / H)."""
    nx, ny = 80, 40
    p = dict(_params(nx, ny), T_down=1.0, T_up=0.0, tau_g=0.8)
    H = ny - 2
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    T_lin = 1.0 - (y - 0.5) / H
    fields = {"T": T_lin, "uy": np.zeros((ny, nx))}
    cx = np.array([3.2, 40.0, 79.6, 10.0, 20.0])
    cy = np.array([1.2, 20.4, 38.3, 37.9, 0.6])
    nu = O.droplet_nusselt(p, fields, cx, cy)
    np.testing.assert_allclose(nu, 1.0, rtol=0, atol=1e-12)
    kappa = (0.8 - 0.5) / 3.0
    fields = {"T": np.full((ny, nx), 0.3), "uy": np.full((ny, nx), 2e-3)}
    nu = O.droplet_nusselt(p, fields, np.array([40.0]), np.array([20.0]))
    assert abs(nu[0] - 2e-3 * 0.3 / (kappa * 1.0 / H)) < 1e-12
    # periodic y or no temperature difference: 0 by convention
    assert O.droplet_nusselt(dict(p, periodic_y=1), fields, cx, cy).tolist() == [0.0] * 5
