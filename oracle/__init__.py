"""ctypes wrapper of the FP64 CPU oracle (``oracle/tlb_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the CUDA library never does.  It
takes plain numpy arrays and shares no code with the GPU path.

State layout: ``state[27, ny, nx]`` float64, planes 0-8 component 1, 9-17
component 2, 18-26 thermal, holding the pre-collision populations S_t.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIBS = {}


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int),
        ("ny", ctypes.c_int),
        ("periodic_y", ctypes.c_int),
        ("_pad", ctypes.c_int),
        ("tau", ctypes.c_double),
        ("tau_g", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("G12", ctypes.c_double),
        ("Ga", ctypes.c_double * 2),
        ("Gr", ctypes.c_double * 2),
        ("rho_wall", ctypes.c_double * 2),
        ("T_down", ctypes.c_double),
        ("T_up", ctypes.c_double),
        ("alpha_g", ctypes.c_double),
        ("body_fx", ctypes.c_double),
        ("u_wall", ctypes.c_double * 2),
    ]


_PARAM_KEYS = ("nx", "ny", "periodic_y", "tau", "tau_g", "rho0", "G12", "Ga", "Gr", "rho_wall",
               "T_down", "T_up", "alpha_g", "body_fx", "u_wall")


def lib(omp=False):
    key = bool(omp)
    if key not in _LIBS:
        _build.build()
        L = ctypes.CDLL(_build.lib_path(omp))
        dp = ctypes.POINTER(ctypes.c_double)
        u8 = ctypes.c_void_p
        P = ctypes.POINTER(OrcParams)
        L.orc_tables.argtypes = [ctypes.POINTER(ctypes.c_int), dp, dp]
        L.orc_solid_map.argtypes = [P, u8, u8]
        L.orc_init.argtypes = [P, u8, dp, dp, dp, dp]
        L.orc_forces.argtypes = [P, u8, dp, dp, dp, dp]
        L.orc_step.argtypes = [P, u8, dp, dp]
        L.orc_run.argtypes = [P, u8, dp, dp, ctypes.c_long]
        L.orc_fields.argtypes = [P, u8, dp, dp, dp, dp, dp, dp]
        L.orc_observables.argtypes = [P, u8, dp, dp]
        L.orc_wall_force.argtypes = [P, u8, dp, dp]
        L.orc_stress.argtypes = [P, u8, dp, dp, dp, dp, dp]
        L.orc_adjoint_step.argtypes = [P, u8, dp, dp, ctypes.c_double, dp, dp]
        L.orc_adjoint_run.argtypes = [P, u8, dp, dp, dp, ctypes.c_long, dp, dp, dp]
        ip = ctypes.POINTER(ctypes.c_int)
        L.orc_droplet_labels.argtypes = [P, u8, dp, ctypes.c_double, ip, ip]
        L.orc_droplet_centres.argtypes = [P, ip, ctypes.c_int, dp, dp, ctypes.POINTER(ctypes.c_longlong)]
        L.orc_digital_voronoi.argtypes = [P, u8, dp, dp, ctypes.c_int, ip]
        L.orc_voronoi_links.argtypes = [P, ip, ip, ctypes.c_long, ctypes.POINTER(ctypes.c_long)]
        for f in ("orc_solid_map", "orc_init", "orc_forces", "orc_step", "orc_run", "orc_fields",
                  "orc_observables", "orc_wall_force", "orc_stress", "orc_adjoint_step", "orc_adjoint_run", "orc_droplet_labels",
                  "orc_droplet_centres", "orc_digital_voronoi", "orc_voronoi_links"):
            getattr(L, f).restype = ctypes.c_int
        _LIBS[key] = L
    return _LIBS[key]


def make_params(p):
    """Build the C struct from a dict with the keys of ``_PARAM_KEYS`` (missing ones default to 0)."""
    s = OrcParams()
    for k in _PARAM_KEYS:
        if k not in p:
            continue
        v = p[k]
        if k in ("Ga", "Gr", "rho_wall", "u_wall"):
            getattr(s, k)[0] = float(v[0])
            getattr(s, k)[1] = float(v[1])
        elif k in ("nx", "ny", "periodic_y"):
            setattr(s, k, int(v))
        else:
            setattr(s, k, float(v))
    return s


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _mask(mask):
    if mask is None:
        return None, None
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    return m, m.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed (rc={rc})")


def tables():
    c = (ctypes.c_int * 50)()
    w = np.zeros(9)
    p = np.zeros(25)
    lib().orc_tables(c, _dp(w), _dp(p))
    return np.array(list(c), dtype=np.int64).reshape(25, 2), w, p


class Oracle:
    """One lattice: parameters, obstacle mask and the FP64 state S_t."""

    def __init__(self, params, rho1, rho2, T0, mask=None, omp=False):
        self.p = dict(params)
        self.cp = make_params(self.p)
        self.nx, self.ny = int(self.p["nx"]), int(self.p["ny"])
        self._mask_arr, self._mask_ptr = _mask(mask)
        self.L = lib(omp)
        shape = (self.ny, self.nx)
        r1 = np.ascontiguousarray(np.broadcast_to(rho1, shape), dtype=np.float64)
        r2 = np.ascontiguousarray(np.broadcast_to(rho2, shape), dtype=np.float64)
        t0 = np.ascontiguousarray(np.broadcast_to(T0, shape), dtype=np.float64)
        self.state = np.zeros((27, self.ny, self.nx))
        self.work = np.zeros_like(self.state)
        _check(self.L.orc_init(ctypes.byref(self.cp), self._mask_ptr, _dp(r1), _dp(r2), _dp(t0), _dp(self.state)),
               "init")
        self.step_count = 0

    @classmethod
    def from_state(cls, params, state, mask=None, omp=False):
        o = cls.__new__(cls)
        o.p = dict(params)
        o.cp = make_params(o.p)
        o.nx, o.ny = int(o.p["nx"]), int(o.p["ny"])
        o._mask_arr, o._mask_ptr = _mask(mask)
        o.L = lib(omp)
        o.state = np.ascontiguousarray(state, dtype=np.float64).copy()
        o.work = np.zeros_like(o.state)
        o.step_count = 0
        return o

    def step(self, n=1):
        _check(self.L.orc_run(ctypes.byref(self.cp), self._mask_ptr, _dp(self.state), _dp(self.work), int(n)), "run")
        self.step_count += n
        return self

    def fields(self):
        N = (self.ny, self.nx)
        r1, r2, T, ux, uy = (np.zeros(N) for _ in range(5))
        _check(self.L.orc_fields(ctypes.byref(self.cp), self._mask_ptr, _dp(self.state), _dp(r1), _dp(r2), _dp(T),
                                 _dp(ux), _dp(uy)), "fields")
        return {"rho1": r1, "rho2": r2, "T": T, "ux": ux, "uy": uy}

    def observables(self):
        out = np.zeros(8)
        _check(self.L.orc_observables(ctypes.byref(self.cp), self._mask_ptr, _dp(self.state), _dp(out)),
               "observables")
        wf = np.zeros(2)
        _check(self.L.orc_wall_force(ctypes.byref(self.cp), self._mask_ptr, _dp(self.state), _dp(wf)), "wall_force")
        return {"mass": out[0:2].copy(), "mom": out[2:4].copy(), "Nu": out[4], "E": out[5], "n_bad": int(out[6]),
                "n_fluid": int(out[7]), "wall_fx": wf}

    def solid(self):
        s = np.zeros((self.ny, self.nx), dtype=np.uint8)
        _check(self.L.orc_solid_map(ctypes.byref(self.cp), self._mask_ptr, s.ctypes.data_as(ctypes.c_void_p)),
               "solid_map")
        return s


def forces(params, rho1, rho2, T, mask=None):
    """F[l, xy, ny, nx] of Eqs. (FAB)+(FintAttrattive)+(FintRepulsive)+(alphaG) for given fields."""
    cp = make_params(params)
    ny, nx = int(params["ny"]), int(params["nx"])
    r1 = np.ascontiguousarray(rho1, dtype=np.float64)
    r2 = np.ascontiguousarray(rho2, dtype=np.float64)
    t = np.ascontiguousarray(np.broadcast_to(T, (ny, nx)), dtype=np.float64)
    F = np.zeros((2, 2, ny, nx))
    m, mp = _mask(mask)
    _check(lib().orc_forces(ctypes.byref(cp), mp, _dp(r1), _dp(r2), _dp(t), _dp(F)), "forces")
    return F


def available_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def adjoint_step(params, state, lam_out, cJ, mask=None):
    """(lam_in, dJ/dT_down increment) of one reverse step at state S_t (see orc_adjoint_step)."""
    cp = make_params(params)
    st = np.ascontiguousarray(state, dtype=np.float64)
    lo = None if lam_out is None else np.ascontiguousarray(lam_out, dtype=np.float64)
    lam_in = np.zeros_like(st)
    d = ctypes.c_double(0.0)
    m, mp = _mask(mask)
    _check(lib().orc_adjoint_step(ctypes.byref(cp), mp, _dp(st), None if lo is None else _dp(lo), float(cJ),
                                  _dp(lam_in), ctypes.byref(d)), "adjoint_step")
    return lam_in, d.value


def adjoint_run(params, rho1, rho2, T0, nsteps, mask=None):
    """(J, dJ/dT0 [ny, nx], dJ/dT_down) for J = time-averaged Nu over nsteps steps."""
    cp = make_params(params)
    ny, nx = int(params["ny"]), int(params["nx"])
    r1 = np.ascontiguousarray(np.broadcast_to(rho1, (ny, nx)), dtype=np.float64)
    r2 = np.ascontiguousarray(np.broadcast_to(rho2, (ny, nx)), dtype=np.float64)
    t0 = np.ascontiguousarray(np.broadcast_to(T0, (ny, nx)), dtype=np.float64)
    J = ctypes.c_double()
    dT0 = np.zeros((ny, nx))
    dTd = ctypes.c_double()
    m, mp = _mask(mask)
    _check(lib().orc_adjoint_run(ctypes.byref(cp), mp, _dp(r1), _dp(r2), _dp(t0), int(nsteps), ctypes.byref(J),
                                 _dp(dT0), ctypes.byref(dTd)), "adjoint_run")
    return J.value, dT0, dTd.value


def stress(params, state, mask=None):
    """Total shear stress of the state S_t (see orc_stress): dict with the means over fluid nodes of
    sigma_xy ("Sigma"), of the viscous part ("visc"), of the interaction pressure tensor P^int_xy
    ("pint") and of the forcing part P^F_xy ("pforce"), the per-row means "row" [ny], and the fields
    "sxy", "pint_field" [ny, nx]."""
    cp = make_params(params)
    ny, nx = int(params["ny"]), int(params["nx"])
    st = np.ascontiguousarray(state, dtype=np.float64)
    sxy, pint, row, out = np.zeros((ny, nx)), np.zeros((ny, nx)), np.zeros(ny), np.zeros(4)
    m, mp = _mask(mask)
    _check(lib().orc_stress(ctypes.byref(cp), mp, _dp(st), _dp(sxy), _dp(pint), _dp(row), _dp(out)), "stress")
    return {"Sigma": out[0], "visc": out[1], "pint": out[2], "pforce": out[3], "row": row, "sxy": sxy,
            "pint_field": pint}


def nusselt_mean(params, rho1, rho2, T0, nsteps, mask=None, omp=False):
    """J = (1/N) sum_{t=1..N} Nu(S_t) (Eq. NuTime) from the rest-equilibrium start of (rho1, rho2, T0):
    the forward half of ``adjoint_run`` alone (one step, then the observables of the new state, N
    times), without storing the states."""
    o = Oracle(params, rho1, rho2, T0, mask=mask, omp=omp)
    out = np.zeros(8)
    s = 0.0
    for _ in range(int(nsteps)):
        o.step(1)
        _check(o.L.orc_observables(ctypes.byref(o.cp), o._mask_ptr, _dp(o.state), _dp(out)), "observables")
        s += out[4]
    return s / float(nsteps)


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def droplets(params, rho1, threshold, mask=None):
    """Droplet topology of a density field (Sec. 2.4, definitions D1-D6 of tlb_droplets.c):
    label [ny, nx] (droplet id or -1), centres cx, cy, sizes, Voronoi colours [ny, nx] and the
    sorted link pairs [n_links, 2]."""
    cp = make_params(params)
    ny, nx = int(params["ny"]), int(params["nx"])
    r1 = np.ascontiguousarray(rho1, dtype=np.float64)
    m, mp = _mask(mask)
    label = np.zeros((ny, nx), dtype=np.int32)
    n = ctypes.c_int()
    L = lib()
    _check(L.orc_droplet_labels(ctypes.byref(cp), mp, _dp(r1), float(threshold), _ip(label), ctypes.byref(n)),
           "droplet_labels")
    M = n.value
    cx, cy = np.zeros(max(M, 1)), np.zeros(max(M, 1))
    size = np.zeros(max(M, 1), dtype=np.int64)
    _check(L.orc_droplet_centres(ctypes.byref(cp), _ip(label), M, _dp(cx), _dp(cy),
                                 size.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong))), "droplet_centres")
    color = np.zeros((ny, nx), dtype=np.int32)
    _check(L.orc_digital_voronoi(ctypes.byref(cp), mp, _dp(cx), _dp(cy), M, _ip(color)), "digital_voronoi")
    nl = ctypes.c_long()
    _check(L.orc_voronoi_links(ctypes.byref(cp), _ip(color), None, 0, ctypes.byref(nl)), "voronoi_links")
    links = np.zeros((max(nl.value, 1), 2), dtype=np.int32)
    _check(L.orc_voronoi_links(ctypes.byref(cp), _ip(color), _ip(links), nl.value, ctypes.byref(nl)),
           "voronoi_links")
    return {"label": label, "n": M, "cx": cx[:M].copy(), "cy": cy[:M].copy(), "size": size[:M].copy(),
            "color": color, "links": links[:nl.value].copy()}


def _min_image(d, n):
    if d > 0.5 * n:
        d -= n
    elif d < -0.5 * n:
        d += n
    return d


def t1_compare(params, prev, now, d_max):
    """Plastic (T1) events between two droplet analyses (Sec. 2.4, Fig. delaunayVoronoi b).

    A droplet of ``now`` is matched to one of ``prev`` when each is the other's nearest centre
    (minimum image, ties to the smaller id) and they lie within d_max.  Broken links: links of prev
    whose two matched droplets are no longer linked; arising links: links of now (in prev ids)
    absent from prev.  A T1 event is a broken link (a, b) and an arising link (c, d) with c and d
    each linked to both a and b in prev: the diagonal of the quadrilateral a c b d flipped.
    Returns sorted lists of pairs (prev ids) and of (a, b, c, d) quadruples."""
    nx, ny, per_y = int(params["nx"]), int(params["ny"]), bool(params.get("periodic_y", 0))

    def dist2(x0, y0, x1, y1):
        dx = _min_image(x0 - x1, nx)
        dy = _min_image(y0 - y1, ny) if per_y else y0 - y1
        return dx * dx + dy * dy

    def nearest(x, y, cx, cy):
        best, bid = None, -1
        for k in range(len(cx)):
            d2 = dist2(x, y, cx[k], cy[k])
            if bid < 0 or d2 < best:
                best, bid = d2, k
        return bid, best

    n2p = {}
    for j in range(now["n"]):
        i, d2 = nearest(now["cx"][j], now["cy"][j], prev["cx"], prev["cy"])
        if i < 0 or d2 > d_max * d_max:
            continue
        jj, _ = nearest(prev["cx"][i], prev["cy"][i], now["cx"], now["cy"])
        if jj == j:
            n2p[j] = i
    p2n = {i: j for j, i in n2p.items()}
    prev_links = {(int(a), int(b)) for a, b in prev["links"]}
    now_links = {(int(a), int(b)) for a, b in now["links"]}
    now_in_prev = set()
    for c, d in now_links:
        if c in n2p and d in n2p:
            a, b = n2p[c], n2p[d]
            now_in_prev.add((min(a, b), max(a, b)))
    broken = sorted((a, b) for a, b in prev_links if a in p2n and b in p2n and (a, b) not in now_in_prev)
    arising = sorted(e for e in now_in_prev if e not in prev_links)

    def linked(a, b):
        return (min(a, b), max(a, b)) in prev_links

    t1 = sorted((a, b, c, d) for a, b in broken for c, d in arising
                if linked(a, c) and linked(a, d) and linked(b, c) and linked(b, d))
    return {"matched": len(n2p), "broken": broken, "arising": arising, "t1": t1}


def droplet_nusselt(params, fields, cx, cy, mask=None):
    """Droplet Nusselt number of Eq. NuDrops for every droplet centre (cx[i], cy[i]).

    u_y = u^(H)_y, T and dT/dy are taken at the lattice node nearest to the centre (x rounded half
    up, periodic; y rounded half up): dT/dy = (T(y+1) - T(y-1)) / 2 with the mirror 2 T_w - T(y) at a
    solid neighbour (the same rule as Eq. NuTime), kappa = (tau_g - 1/2) / 3, "ny" of the formula the
    wall-to-wall height H = ny - 2, Delta T = T_down - T_up.  0 when periodic in y or Delta T = 0; NaN
    when the nearest node is solid."""
    nx, ny = int(params["nx"]), int(params["ny"])
    per_y = bool(params.get("periodic_y", 0))
    Td, Tu = float(params["T_down"]), float(params["T_up"])
    dT = Td - Tu
    kappa = (float(params["tau_g"]) - 0.5) / 3.0
    H = float(ny - 2)
    solid = np.zeros((ny, nx), dtype=bool)
    if not per_y:
        solid[0, :] = solid[-1, :] = True
    if mask is not None:
        solid |= np.asarray(mask) != 0
    T, uy = fields["T"], fields["uy"]
    out = np.zeros(len(cx))
    if per_y or dT == 0.0:
        return out
    den = kappa * (dT / H)
    for i in range(len(cx)):
        x = int(np.floor(cx[i] + 0.5)) % nx
        y = min(max(int(np.floor(cy[i] + 0.5)), 0), ny - 1)
        if solid[y, x]:
            out[i] = np.nan
            continue
        t = T[y, x]

        def neighbour(yy):
            if solid[yy, x]:
                tw = Td if 2 * yy < ny else Tu
                return 2.0 * tw - t
            return T[yy, x]

        dTdy = 0.5 * (neighbour(y + 1) - neighbour(y - 1))
        out[i] = (uy[y, x] * t - kappa * dTdy) / den
    return out
