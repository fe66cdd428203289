"""Seeded synthetic inputs for the thermal emulsion lattice Boltzmann step.

This module only draws random numbers and lays out initial fields and
obstacle masks; it holds none of the lattice Boltzmann arithmetic.  Both the
CUDA path and the FP64 CPU oracle consume its numpy output, so the two sides
always start from bit-identical inputs.

Random numbers come from a counter-based SplitMix64 generator (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
value k of stream ``seed`` is ``mix64(seed + (k + 1) * 0x9E3779B97F4A7C15)``.

Workloads follow the paper's emulsion set-up (Sec. 3, Appendix A tables):
droplets of component 1 (rho1 = rhoMax = 1.4, rho2 = rhoMin = 0.1 inside,
swapped outside), a linear temperature profile between a hot bottom and a
cold top wall (temperature initialisation 2), tau = tau_g = 1, rho0 = 0.83,
G12 = 0.405, G^a = -9 / -8, G^r = +8.1 / +7.1, rho_w = 0.612 / 0.612.  The
buoyancy coefficient alpha*g is set from a Rayleigh number
Ra = alpha g dT H^3 / (nu kappa), nu = (tau - 1/2)/3, kappa = (tau_g - 1/2)/3.
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

RHO_MAX, RHO_MIN = 1.4, 0.1

# Interaction parameters of the paper's preparation run (Appendix A, Table "Input preparation parameters");
# G^r taken positive as stated in Sec. 2.1.
EMULSION_PARAMS = dict(tau=1.0, tau_g=1.0, rho0=0.83, G12=0.405, Ga=(-9.0, -8.0), Gr=(8.1, 7.1),
                       rho_wall=(0.612, 0.612), body_fx=0.0)


def splitmix64(seed, counters):
    """Counter-based SplitMix64: uint64 outputs for the given counters of stream ``seed``."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (np.asarray(counters, dtype=np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed, n, offset=0):
    """n doubles in [0, 1) from stream ``seed`` starting at counter ``offset`` (53-bit mantissa)."""
    z = splitmix64(seed, np.arange(offset, offset + n, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def rayleigh_alpha_g(Ra, dT, H, tau=1.0, tau_g=1.0):
    """alpha*g giving Rayleigh number Ra for wall-to-wall height H and temperature jump dT."""
    nu = (tau - 0.5) / 3.0
    kappa = (tau_g - 0.5) / 3.0
    return Ra * nu * kappa / (dT * H ** 3)


def linear_T(nx, ny, T_down, T_up):
    """Conduction profile between the half-way walls y = 1/2 and y = ny - 3/2."""
    H = ny - 2
    y = np.arange(ny, dtype=np.float64)
    T = T_down + (T_up - T_down) * (y - 0.5) / H
    return np.repeat(T[:, None], nx, axis=1)


def posts_mask(nx, ny, height, width, period):
    """Rectangular posts (obstacles) of the given height/width every ``period`` columns on both walls."""
    m = np.zeros((ny, nx), dtype=np.uint8)
    cols = (np.arange(nx) % period) < width
    m[1:1 + height, :] |= cols[None, :].astype(np.uint8)
    m[ny - 1 - height:ny - 1, :] |= cols[None, :].astype(np.uint8)
    return m


def rough_wall_mask(nx, ny, height, width, lam, alpha=0.0, asymmetric=False, down=True, up=True, x0=0):
    """Trapezoidal roughness on the walls (Sec. 5, Fig. roughness a): an obstacle every ``lam``
    columns starting at column x0, ``height`` rows tall above the wall row (below it on the top wall),
    ``width`` columns wide at its top; its sides lean outwards by tan(alpha) columns per row towards
    the wall (alpha in radians from the vertical), the trailing (right) side stays vertical when
    ``asymmetric``.  alpha = 0 gives rectangular posts.  A node is solid when its column centre lies
    inside the trapezoid at the row's mid-height.  The top-wall obstacles are the mirror images of
    the bottom ones in y."""
    m = np.zeros((ny, nx), dtype=np.uint8)
    t = float(np.tan(alpha))
    x = np.arange(nx, dtype=np.float64) + 0.5
    for k in range(height):
        # row k above the wall: its mid-height is height - k - 0.5 below the obstacle top
        spread = t * (height - k - 0.5)
        rel = (x - x0) % lam
        left = rel >= lam - spread  # the leaning left side spills into the end of the previous period
        body = rel < width
        right = (rel >= width) & (rel < width + (0.0 if asymmetric else spread))
        row = (left | body | right).astype(np.uint8)
        if down:
            m[1 + k, :] |= row
        if up:
            m[ny - 2 - k, :] |= row
    return m


def _disk_fields(nx, ny, centres, R):
    """rho1, rho2 with sharp disks of component 1 (x periodic); node (x, y) is inside a disk when
    dx^2 + dy^2 <= R^2 with dx the periodic x distance."""
    inside = np.zeros((ny, nx), dtype=bool)
    r = int(np.ceil(R)) + 1
    for cx, cy in centres:
        ys = np.arange(max(0, int(np.floor(cy)) - r), min(ny, int(np.floor(cy)) + r + 2))
        xs = np.arange(int(np.floor(cx)) - r, int(np.floor(cx)) + r + 2)
        dx = np.abs(xs - cx)
        dx = np.minimum(dx, nx - dx)
        hit = dx[None, :] ** 2 + (ys[:, None] - cy) ** 2 <= R * R
        inside[np.ix_(ys, xs % nx)] |= hit
    rho1 = np.where(inside, RHO_MAX, RHO_MIN)
    rho2 = np.where(inside, RHO_MIN, RHO_MAX)
    return rho1, rho2


def random_disks(nx, ny, n, R, seed, ylo, yhi, min_dist, max_tries=100000):
    """n disk centres drawn uniformly with rejection (periodic-x distance >= min_dist)."""
    centres = []
    k = 0
    while len(centres) < n:
        if k >= max_tries:
            raise RuntimeError("random_disks: could not place all disks")
        u = uniform(seed, 2, offset=2 * k)
        k += 1
        cx = u[0] * nx
        cy = ylo + u[1] * (yhi - ylo)
        ok = True
        for (ax, ay) in centres:
            dx = abs(cx - ax)
            dx = min(dx, nx - dx)
            if dx * dx + (cy - ay) ** 2 < min_dist * min_dist:
                ok = False
                break
        if ok:
            centres.append((cx, cy))
    return centres


def hex_disks(nx, ylo, yhi, ndx, ndy, jitter, seed):
    """ndx * ndy centres on a hexagonal (honeycomb) arrangement between rows ylo..yhi, jittered."""
    ax = nx / ndx
    ay = (yhi - ylo) / ndy
    u = uniform(seed, 2 * ndx * ndy) * 2.0 - 1.0
    centres = []
    for j in range(ndy):
        for i in range(ndx):
            k = j * ndx + i
            cx = (i + 0.5 + 0.5 * (j % 2)) * ax + jitter * u[2 * k]
            cy = ylo + (j + 0.5) * ay + jitter * u[2 * k + 1]
            centres.append((cx % nx, cy))
    return centres


@dataclass
class Workload:
    """One lattice: parameters (a dict in the C-ABI's field names) and initial host fields."""
    name: str
    params: dict
    rho1: np.ndarray
    rho2: np.ndarray
    T0: np.ndarray
    mask: Optional[np.ndarray] = None
    nsteps: int = 0
    extra: dict = field(default_factory=dict)


def _base_params(nx, ny, T_down, T_up, alpha_g, periodic_y=0):
    p = dict(EMULSION_PARAMS)
    p.update(nx=nx, ny=ny, periodic_y=periodic_y, T_down=T_down, T_up=T_up, alpha_g=alpha_g)
    return p


def emulsion_small(nx=64, ny=64, seed=1, n_drops=6, R=8.0, Ra=2.0e3, T_down=1.0, T_up=0.0):
    """Small emulsion: walls at y = 0 and y = ny-1 (hot bottom), 6 disks of radius 8 placed with
    rejection at distance >= 2R + 2, kept >= 2 rows away from the walls; Ra ~ 2e3."""
    H = ny - 2
    centres = random_disks(nx, ny, n_drops, R, seed, ylo=1 + R + 2, yhi=ny - 2 - R - 2, min_dist=2 * R + 2)
    rho1, rho2 = _disk_fields(nx, ny, centres, R)
    ag = rayleigh_alpha_g(Ra, T_down - T_up, H)
    return Workload("emulsion_64x64", _base_params(nx, ny, T_down, T_up, ag), rho1, rho2,
                    linear_T(nx, ny, T_down, T_up), None, 1000, dict(centres=centres, R=R))


def emulsion_hex(nx, ny, ndx, ndy, phi, Ra, seed, noise=1e-3, T_down=0.5, T_up=-0.5, mask=None, post_h=0,
                 name=None):
    """Concentrated emulsion: ndx*ndy droplets on a jittered honeycomb at area fraction phi of the
    fluid slab, +-noise uniform density noise on rho1 and rho2, linear T, Ra just above onset."""
    H = ny - 2
    ylo, yhi = 1.0 + post_h, ny - 1.0 - post_h
    area = nx * (yhi - ylo)
    R = float(np.sqrt(phi * area / (ndx * ndy) / np.pi))
    centres = hex_disks(nx, ylo, yhi, ndx, ndy, jitter=0.5, seed=seed)
    rho1, rho2 = _disk_fields(nx, ny, centres, R)
    if noise:
        u = uniform(seed + 1000003, 2 * nx * ny).reshape(2, ny, nx) * 2.0 - 1.0
        rho1 = rho1 + noise * u[0]
        rho2 = rho2 + noise * u[1]
    ag = rayleigh_alpha_g(Ra, T_down - T_up, H)
    return Workload(name or f"emulsion_{nx}x{ny}", _base_params(nx, ny, T_down, T_up, ag), rho1, rho2,
                    linear_T(nx, ny, T_down, T_up), mask, 0, dict(R=R, n_drops=ndx * ndy, phi=phi, Ra=Ra))


def emulsion_1024x512(seed=2):
    """Concentrated emulsion 1024 x 512: 25 x 14 = 350 droplets at phi = 0.8 (diameter ~39),
    Ra = 3.6e4 (just above onset), +-1e-3 density noise; 20000 steps, observables every 500."""
    w = emulsion_hex(1024, 512, 25, 14, 0.8, 3.6e4, seed, name="emulsion_1024x512")
    w.nsteps = 20000
    return w


def emulsion_512x256(seed=4):
    """Adjoint workload: 512 x 256 emulsion at phi = 0.7 (14 x 7 droplets)."""
    w = emulsion_hex(512, 256, 14, 7, 0.7, 3.6e4, seed, name="emulsion_512x256")
    w.nsteps = 2000
    return w


def rough_channel_4096x2048(seed=5):
    """Large rough channel: 4096 x 2048, posts 8 x 8 every 32 columns on both walls, ~5000 droplets
    (94 x 53 = 4982 on a near-isotropic honeycomb: x spacing 43.6, row spacing 38.3) at phi = 0.8 of
    the slab between the post tops, so d = 41.2 and neighbouring disks start ~2.4 nodes apart."""
    mask = posts_mask(4096, 2048, 8, 8, 32)
    w = emulsion_hex(4096, 2048, 94, 53, 0.8, 3.6e4, seed, mask=mask, post_h=8, name="rough_channel_4096x2048")
    w.nsteps = 50000
    return w


def ensemble(n_replicas=64, seed=3, base_ra=3.6e4):
    """Batched ensemble: nx = 256 + 64 k, k ~ U{0..12}, ny = nx/2, phi ~ U[0.5, 0.85],
    Ra ~ U[1.1, 2] x 3.6e4; 5000 steps each."""
    u = uniform(seed, 3 * n_replicas).reshape(n_replicas, 3)
    out = []
    for r in range(n_replicas):
        k = int(u[r, 0] * 13)
        nx = 256 + 64 * k
        ny = nx // 2
        phi = 0.5 + 0.35 * u[r, 1]
        Ra = (1.1 + 0.9 * u[r, 2]) * base_ra
        ndx = max(2, int(round(nx / 41.0)))
        ndy = max(2, int(round((ny - 2) / 36.0)))
        w = emulsion_hex(nx, ny, ndx, ndy, phi, Ra, seed * 1000 + r, name=f"replica{r}_{nx}x{ny}")
        w.nsteps = 5000
        out.append(w)
    return out


def layered(nx=128, ny=2, width=65, G12=0.405):
    """Two-layer initialisation (droplet initialisation 3, Appendix B): component 1 at rhoMax on the
    first ``width`` columns, rhoMin elsewhere; fully periodic, no thermal coupling."""
    rho1 = np.where(np.arange(nx)[None, :] < width, RHO_MAX, RHO_MIN) * np.ones((ny, nx))
    rho2 = (RHO_MAX + RHO_MIN) - rho1
    p = dict(EMULSION_PARAMS)
    p.update(nx=nx, ny=ny, periodic_y=1, G12=G12, T_down=0.0, T_up=0.0, alpha_g=0.0)
    return Workload(f"layered_{nx}x{ny}", p, rho1, rho2, np.zeros((ny, nx)), None, 50000)
