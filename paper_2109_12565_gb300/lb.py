"""Thin ctypes binding of the C ABI in ``include/tlb.h`` (argument marshalling only).

Device memory comes from PyTorch (one uint8 workspace tensor per lattice) and
the CUDA stream is PyTorch's current stream; every step of the method runs
in the library's kernels.  The binding raises if the CUDA library has not
been built: there is no CPU fallback.
"""
import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtlbgb300.so")

LB_OK, LB_EINVAL, LB_ENOSPACE, LB_ECUDA, LB_ETIMEOUT, LB_EUNSTABLE = 0, -1, -2, -3, -4, -5
LB_FP64, LB_FP32_SHIFTED, LB_FP32_FP16T, LB_DF64 = 0, 1, 2, 3
_NAMES = {0: "LB_OK", -1: "LB_EINVAL", -2: "LB_ENOSPACE", -3: "LB_ECUDA", -4: "LB_ETIMEOUT", -5: "LB_EUNSTABLE"}

# every symbol include/tlb.h declares
EXPORTS = ("lb_workspace_size", "lb_init", "lb_step", "lb_observables", "lb_get_fields", "lb_get_state",
           "lb_set_state", "lb_sync", "lb_destroy", "lb_last_error", "lb_version", "lb_autotune", "lb_autotune_cold",
           "lb_set_tile", "lb_tile_info", "lb_batch_workspace_size", "lb_batch_init", "lb_batch_step", "lb_batch_configure",
           "lb_batch_autotune", "lb_batch_info", "lb_batch_observables", "lb_batch_get_fields", "lb_batch_get_state",
           "lb_batch_sync", "lb_batch_set_wait_budget", "lb_batch_destroy", "lb_batch_last_error",
           "lb_state_layout", "lb_adjoint_workspace_size", "lb_adjoint_step", "lb_adjoint", "lb_adjoint_timing",
           "lb_droplets_workspace_size", "lb_droplets", "lb_droplets_get", "lb_droplets_nusselt",
           "lb_droplets_compare", "lb_stress", "lb_batch_stress")


class LbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class LbParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("periodic_y", ctypes.c_int), ("precision", ctypes.c_int),
        ("tau", ctypes.c_double), ("tau_g", ctypes.c_double), ("rho0", ctypes.c_double), ("G12", ctypes.c_double),
        ("Ga", ctypes.c_double * 2), ("Gr", ctypes.c_double * 2), ("rho_wall", ctypes.c_double * 2),
        ("T_down", ctypes.c_double), ("T_up", ctypes.c_double), ("alpha_g", ctypes.c_double),
        ("body_fx", ctypes.c_double), ("shift_rho", ctypes.c_double * 2), ("shift_T", ctypes.c_double),
        ("u_wall", ctypes.c_double * 2),
    ]


class LbObs(ctypes.Structure):
    _fields_ = [
        ("mass", ctypes.c_double * 2), ("mom", ctypes.c_double * 2), ("Nu", ctypes.c_double), ("E", ctypes.c_double),
        ("step", ctypes.c_longlong), ("n_fluid", ctypes.c_longlong), ("n_bad", ctypes.c_longlong),
        ("status", ctypes.c_int), ("_pad", ctypes.c_int), ("wall_fx", ctypes.c_double * 2),
    ]


_LIB = None


def lib():
    """Load the library (raises if it was not built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built ({LIB_PATH} missing): run paper_2109_12565_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, dp, i, sz = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_size_t
        P = ctypes.POINTER(LbParams)
        L.lb_workspace_size.argtypes = [P, i, ctypes.POINTER(sz)]
        L.lb_init.argtypes = [ctypes.POINTER(vp), P, vp, dp, dp, dp, vp, sz, vp]
        L.lb_step.argtypes = [vp, i]
        L.lb_observables.argtypes = [vp, ctypes.POINTER(LbObs)]
        L.lb_get_fields.argtypes = [vp, dp, dp, dp, dp, dp]
        L.lb_get_state.argtypes = [vp, dp, sz]
        L.lb_set_state.argtypes = [vp, dp, sz]
        L.lb_sync.argtypes = [vp]
        L.lb_destroy.argtypes = [vp]
        L.lb_destroy.restype = None
        L.lb_last_error.argtypes = [vp]
        L.lb_last_error.restype = ctypes.c_char_p
        L.lb_autotune.argtypes = [vp, i, ctypes.POINTER(i), dp, i]
        L.lb_autotune_cold.argtypes = [vp, i, vp, sz, ctypes.POINTER(i), dp, i]
        L.lb_set_tile.argtypes = [vp, i]
        L.lb_tile_info.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i)]
        ip, ll = ctypes.POINTER(ctypes.c_int), ctypes.c_longlong
        pp = ctypes.POINTER(ctypes.c_void_p)
        L.lb_batch_workspace_size.argtypes = [P, i, ip, ctypes.POINTER(sz)]
        L.lb_batch_init.argtypes = [ctypes.POINTER(vp), P, i, pp, pp, pp, pp, vp, sz, vp]
        L.lb_batch_step.argtypes = [vp, i]
        L.lb_batch_configure.argtypes = [vp, i, i, i]
        L.lb_batch_autotune.argtypes = [vp, i, ip, ip, ctypes.POINTER(ll), dp, i]
        L.lb_batch_info.argtypes = [vp, ip, ip, ip, ip, ip]
        L.lb_batch_observables.argtypes = [vp, i, ctypes.POINTER(LbObs)]
        L.lb_batch_get_fields.argtypes = [vp, i, dp, dp, dp, dp, dp]
        L.lb_batch_get_state.argtypes = [vp, i, dp, sz]
        L.lb_batch_sync.argtypes = [vp]
        L.lb_batch_set_wait_budget.argtypes = [vp, ll, i]
        L.lb_batch_destroy.argtypes = [vp]
        L.lb_batch_destroy.restype = None
        L.lb_batch_last_error.argtypes = [vp]
        L.lb_batch_last_error.restype = ctypes.c_char_p
        for f in ("lb_batch_workspace_size", "lb_batch_init", "lb_batch_step", "lb_batch_configure",
                  "lb_batch_autotune", "lb_batch_info", "lb_batch_observables", "lb_batch_get_fields",
                  "lb_batch_get_state", "lb_batch_sync", "lb_batch_set_wait_budget"):
            getattr(L, f).restype = ctypes.c_int
        L.lb_state_layout.argtypes = [vp, ip, ctypes.POINTER(sz), ip]
        L.lb_adjoint_workspace_size.argtypes = [vp, i, i, ctypes.POINTER(sz)]
        L.lb_adjoint_step.argtypes = [vp, vp, vp, ctypes.c_double, vp, sz, dp]
        L.lb_adjoint.argtypes = [vp, i, i, vp, sz, dp, dp, dp]
        L.lb_adjoint_timing.argtypes = [dp]
        for f in ("lb_state_layout", "lb_adjoint_workspace_size", "lb_adjoint_step", "lb_adjoint", "lb_adjoint_timing"):
            getattr(L, f).restype = ctypes.c_int
        L.lb_droplets_workspace_size.argtypes = [vp, i, ctypes.POINTER(sz)]
        L.lb_droplets.argtypes = [vp, ctypes.c_double, i, vp, sz, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.lb_droplets_get.argtypes = [vp, vp, sz, dp, dp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(i),
                                      ctypes.POINTER(i), ctypes.POINTER(i)]
        L.lb_droplets_compare.argtypes = [vp, vp, vp, sz, ctypes.c_double, vp, sz, ctypes.POINTER(i),
                                          ctypes.POINTER(i), ctypes.POINTER(i), ctypes.POINTER(i), i]
        L.lb_droplets_nusselt.argtypes = [vp, vp, sz, dp]
        for f in ("lb_droplets_workspace_size", "lb_droplets", "lb_droplets_get", "lb_droplets_nusselt",
                  "lb_droplets_compare", "lb_stress", "lb_batch_stress"):
            getattr(L, f).restype = ctypes.c_int
        L.lb_stress.argtypes = [vp, dp, dp, dp]
        L.lb_stress.restype = ctypes.c_int
        L.lb_batch_stress.argtypes = [vp, i, dp, dp, dp]
        L.lb_batch_stress.restype = ctypes.c_int
        L.lb_version.argtypes = []
        L.lb_version.restype = ctypes.c_char_p
        for f in ("lb_workspace_size", "lb_init", "lb_step", "lb_observables", "lb_get_fields", "lb_get_state",
                  "lb_set_state", "lb_sync", "lb_autotune", "lb_autotune_cold", "lb_set_tile", "lb_tile_info"):
            getattr(L, f).restype = ctypes.c_int
        _LIB = L
    return _LIB


def make_params(p, precision=LB_FP64):
    """C struct from a parameter dict (keys as in the C struct; shift_* default to NaN = automatic)."""
    s = LbParams()
    s.nx, s.ny = int(p["nx"]), int(p["ny"])
    s.periodic_y = int(p.get("periodic_y", 0))
    s.precision = int(p.get("precision", precision))
    for k in ("tau", "tau_g", "rho0", "G12", "T_down", "T_up", "alpha_g", "body_fx"):
        setattr(s, k, float(p.get(k, 0.0)))
    for k in ("Ga", "Gr", "rho_wall", "u_wall"):
        v = p.get(k, (0.0, 0.0))
        getattr(s, k)[0], getattr(s, k)[1] = float(v[0]), float(v[1])
    sr = p.get("shift_rho", (math.nan, math.nan))
    s.shift_rho[0], s.shift_rho[1] = float(sr[0]), float(sr[1])
    s.shift_T = float(p.get("shift_T", math.nan))
    return s


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc, h=None):
    if rc != LB_OK:
        raise LbError(rc, lib().lb_last_error(h).decode())
    return rc


def workspace_size(params, has_mask=False, precision=LB_FP64):
    n = ctypes.c_size_t()
    _check(lib().lb_workspace_size(ctypes.byref(make_params(params, precision)), int(bool(has_mask)), ctypes.byref(n)))
    return n.value


class Lattice:
    """One lattice on the current CUDA device: workspace tensor + library handle."""

    def __init__(self, params, rho1, rho2, T0, mask=None, precision=LB_FP64, device=None, stream=None):
        import torch

        self.params = dict(params)
        self.cp = make_params(self.params, precision)
        self.nx, self.ny = self.cp.nx, self.cp.ny
        shape = (self.ny, self.nx)
        self._r1 = np.ascontiguousarray(np.broadcast_to(rho1, shape), dtype=np.float64)
        self._r2 = np.ascontiguousarray(np.broadcast_to(rho2, shape), dtype=np.float64)
        self._t0 = np.ascontiguousarray(np.broadcast_to(T0, shape), dtype=np.float64)
        self._mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.device = dev
        nbytes = workspace_size(self.params, self._mask is not None, self.cp.precision)
        with torch.cuda.device(dev):
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self._h = ctypes.c_void_p()
        mptr = None if self._mask is None else self._mask.ctypes.data_as(ctypes.c_void_p)
        _check(lib().lb_init(ctypes.byref(self._h), ctypes.byref(self.cp), mptr, _dp(self._r1), _dp(self._r2),
                             _dp(self._t0), ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                             ctypes.c_void_p(self.stream.cuda_stream)))

    @classmethod
    def from_state(cls, params, state, mask=None, precision=LB_FP64, device=None, stream=None):
        """A lattice whose S_0 is a given state (27 planes of ny x nx doubles): the restart of a run
        under new parameters, e.g. a prepared emulsion continued with buoyancy.  The lattice is
        created from the state's own moments (which also fix the FP32 shifts) and then loaded with
        lb_set_state; the step counter starts at 0."""
        st = np.ascontiguousarray(state, dtype=np.float64)
        rho1, rho2, T = st[0:9].sum(axis=0), st[9:18].sum(axis=0), st[18:27].sum(axis=0)
        # solid nodes hold 0; any positive density will do there (lb_init ignores them)
        rho1 = np.where(rho1 > 0.0, rho1, 1.0)
        rho2 = np.where(rho2 > 0.0, rho2, 1.0)
        g = cls(params, rho1, rho2, T, mask=mask, precision=precision, device=device, stream=stream)
        g.set_state(st)
        return g

    # -- C-ABI calls
    def step(self, n=1):
        _check(lib().lb_step(self._h, int(n)), self._h)
        return self

    def observables(self, check=True):
        o = LbObs()
        rc = lib().lb_observables(self._h, ctypes.byref(o))
        if rc not in (LB_OK, LB_EUNSTABLE) or (check and rc != LB_OK):
            _check(rc, self._h)
        return {"mass": np.array(o.mass[:]), "mom": np.array(o.mom[:]), "Nu": o.Nu, "E": o.E, "step": o.step,
                "wall_fx": np.array(o.wall_fx[:]),
                "n_fluid": o.n_fluid, "n_bad": o.n_bad, "status": o.status}

    def fields(self):
        out = {k: np.zeros((self.ny, self.nx)) for k in ("rho1", "rho2", "T", "ux", "uy")}
        _check(lib().lb_get_fields(self._h, *(_dp(out[k]) for k in ("rho1", "rho2", "T", "ux", "uy"))), self._h)
        return out

    def get_state(self):
        st = np.zeros((27, self.ny, self.nx))
        _check(lib().lb_get_state(self._h, _dp(st), st.nbytes), self._h)
        return st

    def stress(self, field=True):
        """Total shear stress (lb_stress): means of sigma_xy ("Sigma"), of its viscous part ("visc"), of
        the interaction pressure tensor ("pint") and of the forcing part ("pforce"), the per-row means
        "row" [ny] and, with field=True, sigma_xy "sxy" [ny, nx]."""
        out, row = np.zeros(4), np.zeros(self.ny)
        f = np.zeros((self.ny, self.nx)) if field else None
        _check(lib().lb_stress(self._h, _dp(out), _dp(row), _dp(f)), self._h)
        return {"Sigma": out[0], "visc": out[1], "pint": out[2], "pforce": out[3], "row": row, "sxy": f}

    def set_state(self, state):
        st = np.ascontiguousarray(state, dtype=np.float64)
        if st.shape != (27, self.ny, self.nx):
            raise ValueError("state must have shape (27, ny, nx)")
        _check(lib().lb_set_state(self._h, _dp(st), st.nbytes), self._h)

    def tile_info(self, candidate=-1):
        tx, ty, th = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        n = lib().lb_tile_info(self._h, int(candidate), ctypes.byref(tx), ctypes.byref(ty), ctypes.byref(th))
        if n < 0:
            _check(n, self._h)
        return {"tx": tx.value, "ty": ty.value, "threads": th.value, "candidates": n}

    def autotune(self, launches=20, scratch=None):
        """Time every tile candidate (state unchanged) and keep the fastest; returns (index, ms list).

        With ``scratch`` (a device tensor larger than L2, overwritten) every timed launch starts with
        the state evicted from L2 (lb_autotune_cold); without it the launches run back to back."""
        n = self.tile_info(0)["candidates"]
        ms = np.zeros(n)
        chosen = ctypes.c_int()
        if scratch is None:
            _check(lib().lb_autotune(self._h, int(launches), ctypes.byref(chosen), _dp(ms), n), self._h)
        else:
            nbytes = scratch.numel() * scratch.element_size()
            _check(lib().lb_autotune_cold(self._h, int(launches), ctypes.c_void_p(scratch.data_ptr()), nbytes,
                                          ctypes.byref(chosen), _dp(ms), n), self._h)
        return chosen.value, ms.tolist()

    # -- droplet topology (lb_droplets*)
    def droplets(self, threshold=0.8, max_drops=None, arrays=True):
        """Droplet analysis of the current state (labels, centres, digital Voronoi, links).  Returns a
        dict with the counts and, with arrays=True, the host copies; the device workspace is kept
        in the dict ("ws") for droplet_t1."""
        import torch

        if max_drops is None:
            max_drops = max(16, self.nx * self.ny // 64)
        n = ctypes.c_size_t()
        _check(lib().lb_droplets_workspace_size(self._h, int(max_drops), ctypes.byref(n)), self._h)
        ws = torch.empty(n.value, dtype=torch.uint8, device=self.workspace.device)
        M, K = ctypes.c_int(), ctypes.c_int()
        _check(lib().lb_droplets(self._h, float(threshold), int(max_drops), ctypes.c_void_p(ws.data_ptr()), n.value,
                                 ctypes.byref(M), ctypes.byref(K)), self._h)
        out = {"n": M.value, "n_links": K.value, "ws": ws, "ws_bytes": n.value}
        if arrays:
            m, k = max(M.value, 1), max(K.value, 1)
            cx, cy = np.zeros(m), np.zeros(m)
            size = np.zeros(m, dtype=np.int64)
            links = np.zeros((k, 2), dtype=np.int32)
            label = np.zeros((self.ny, self.nx), dtype=np.int32)
            color = np.zeros((self.ny, self.nx), dtype=np.int32)
            ip = ctypes.POINTER(ctypes.c_int)
            _check(lib().lb_droplets_get(self._h, ctypes.c_void_p(ws.data_ptr()), n.value, _dp(cx), _dp(cy),
                                         size.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)),
                                         links.ctypes.data_as(ip), label.ctypes.data_as(ip),
                                         color.ctypes.data_as(ip)), self._h)
            out.update(cx=cx[:M.value], cy=cy[:M.value], size=size[:M.value], links=links[:K.value], label=label,
                       color=color)
        return out

    def droplet_nusselt(self, res):
        """Eq. NuDrops for every droplet of a droplets() result taken on the current state."""
        nu = np.zeros(max(res["n"], 1))
        _check(lib().lb_droplets_nusselt(self._h, ctypes.c_void_p(res["ws"].data_ptr()), res["ws_bytes"], _dp(nu)),
               self._h)
        return nu[:res["n"]]

    def droplet_t1(self, prev, now, d_max, cap=None):
        """T1 events between two results of droplets() (lb_droplets_compare)."""
        import torch

        if prev["ws_bytes"] != now["ws_bytes"]:
            raise ValueError("both analyses need the same max_drops")
        cap = int(cap if cap is not None else 16 * max(prev["n"], now["n"], 1))
        counts = (ctypes.c_int * 4)()
        ip = ctypes.POINTER(ctypes.c_int)
        scratch_bytes = 1 << 20
        for _ in range(2):
            scratch = torch.empty(scratch_bytes, dtype=torch.uint8, device=self.workspace.device)
            broken = np.zeros((max(cap, 1), 2), dtype=np.int32)
            arising = np.zeros((max(cap, 1), 2), dtype=np.int32)
            t1 = np.zeros((max(cap, 1), 4), dtype=np.int32)
            rc = lib().lb_droplets_compare(self._h, ctypes.c_void_p(prev["ws"].data_ptr()),
                                           ctypes.c_void_p(now["ws"].data_ptr()), now["ws_bytes"], float(d_max),
                                           ctypes.c_void_p(scratch.data_ptr()), scratch_bytes, counts,
                                           broken.ctypes.data_as(ip), arising.ctypes.data_as(ip),
                                           t1.ctypes.data_as(ip), cap)
            if rc == LB_ENOSPACE:
                scratch_bytes = int(counts[0]) * 1024 + 4096
                continue
            _check(rc, self._h)
            break
        nb_, na_, nt_ = (min(int(counts[k]), cap) for k in (1, 2, 3))
        return {"matched": int(counts[0]), "n_broken": int(counts[1]), "n_arising": int(counts[2]),
                "n_t1": int(counts[3]), "broken": broken[:nb_], "arising": arising[:na_], "t1": t1[:nt_]}

    def set_tile(self, candidate):
        _check(lib().lb_set_tile(self._h, int(candidate)), self._h)

    def sync(self):
        _check(lib().lb_sync(self._h), self._h)

    # -- adjoint
    def state_layout(self):
        pitch, plane, elem = ctypes.c_int(), ctypes.c_size_t(), ctypes.c_int()
        _check(lib().lb_state_layout(self._h, ctypes.byref(pitch), ctypes.byref(plane), ctypes.byref(elem)), self._h)
        return pitch.value, plane.value, elem.value

    def to_device_vector(self, arr):
        """[27, ny, nx] host array -> device tensor in the storage layout (for lb_adjoint_step)."""
        import torch

        pitch, _, elem = self.state_layout()
        dt = torch.float64 if elem == 8 else torch.float32
        t = torch.zeros((27, self.ny, pitch), dtype=dt, device=self.workspace.device)
        t[:, :, :self.nx] = torch.from_numpy(np.ascontiguousarray(arr, dtype=np.float64)).to(dt)
        return t

    def from_device_vector(self, t):
        return t[:, :, :self.nx].double().cpu().numpy()

    def _adj_ws(self, n_steps, ckpt_every):
        import torch

        n = ctypes.c_size_t()
        _check(lib().lb_adjoint_workspace_size(self._h, int(n_steps), int(ckpt_every), ctypes.byref(n)), self._h)
        return torch.empty(n.value, dtype=torch.uint8, device=self.workspace.device), n.value

    def adjoint_step(self, lam_next, cJ):
        """lam_t (device tensor) and the dJ/dT_down increment of one reverse step at the current state;
        lam_next: device tensor in the storage layout, or None."""
        import torch

        ws, nb = self._adj_ws(1, 1)
        pitch, _, elem = self.state_layout()
        dt = torch.float64 if elem == 8 else torch.float32
        lam = torch.zeros((27, self.ny, pitch), dtype=dt, device=self.workspace.device)
        d = ctypes.c_double()
        nxt = None if lam_next is None else ctypes.c_void_p(lam_next.data_ptr())
        _check(lib().lb_adjoint_step(self._h, nxt, ctypes.c_void_p(lam.data_ptr()), float(cJ),
                                     ctypes.c_void_p(ws.data_ptr()), nb, ctypes.byref(d)), self._h)
        return lam, d.value

    def adjoint(self, n_steps, ckpt_every=None, gradient=True):
        """(J, dJ/dT0 [ny, nx], dJ/dT_down) of J = time-averaged Nu over n_steps steps from the current
        state, with sqrt-N checkpointing; with gradient=False only J (the other two are None)."""
        ckpt = int(ckpt_every or max(1, round(n_steps ** 0.5)))
        ws, nb = self._adj_ws(n_steps, ckpt)
        J = ctypes.c_double()
        g = np.zeros((self.ny, self.nx)) if gradient else None
        d = ctypes.c_double()
        _check(lib().lb_adjoint(self._h, int(n_steps), ckpt, ctypes.c_void_p(ws.data_ptr()), nb, ctypes.byref(J),
                                _dp(g), ctypes.byref(d) if gradient else None), self._h)
        return J.value, g, (d.value if gradient else None)

    @staticmethod
    def adjoint_timing():
        """Phase times of the last adjoint(): forward ms, recompute ms, reverse ms, adjoint steps."""
        out = np.zeros(4)
        lib().lb_adjoint_timing(_dp(out))
        return {"forward_ms": out[0], "recompute_ms": out[1], "reverse_ms": out[2], "adjoint_steps": int(out[3])}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().lb_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _bcheck(rc, b=None):
    if rc != LB_OK:
        raise LbError(rc, lib().lb_batch_last_error(b).decode())
    return rc


def batch_workspace_size(params_list, masks=None, precision=LB_FP32_SHIFTED):
    n = len(params_list)
    arr = (LbParams * n)(*[make_params(p, precision) for p in params_list])
    hm = (ctypes.c_int * n)(*[int(masks is not None and masks[r] is not None) for r in range(n)])
    out = ctypes.c_size_t()
    _bcheck(lib().lb_batch_workspace_size(arr, n, hm, ctypes.byref(out)))
    return out.value


class Batch:
    """An ensemble of independent lattices advanced together (lb_batch_* C ABI)."""

    def __init__(self, params_list, rho1s, rho2s, T0s, masks=None, precision=LB_FP32_SHIFTED, device=None):
        import torch

        n = len(params_list)
        self.n = n
        self.params = [dict(p) for p in params_list]
        self._cps = (LbParams * n)(*[make_params(p, precision) for p in params_list])
        self.shapes = [(int(p["ny"]), int(p["nx"])) for p in params_list]
        self._keep = []

        def arr(a, shape):
            x = np.ascontiguousarray(np.broadcast_to(a, shape), dtype=np.float64)
            self._keep.append(x)
            return x.ctypes.data_as(ctypes.c_void_p)

        r1 = (ctypes.c_void_p * n)(*[arr(rho1s[r], self.shapes[r]) for r in range(n)])
        r2 = (ctypes.c_void_p * n)(*[arr(rho2s[r], self.shapes[r]) for r in range(n)])
        t0 = (ctypes.c_void_p * n)(*[arr(T0s[r], self.shapes[r]) for r in range(n)])
        mk = (ctypes.c_void_p * n)()
        for r in range(n):
            if masks is not None and masks[r] is not None:
                m = np.ascontiguousarray(masks[r], dtype=np.uint8)
                self._keep.append(m)
                mk[r] = m.ctypes.data_as(ctypes.c_void_p)
        nbytes = batch_workspace_size(params_list, masks, precision)
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        with torch.cuda.device(dev):
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
            self.stream = torch.cuda.current_stream(dev)
        self._b = ctypes.c_void_p()
        _bcheck(lib().lb_batch_init(ctypes.byref(self._b), self._cps, n, mk, r1, r2, t0,
                                    ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                    ctypes.c_void_p(self.stream.cuda_stream)))

    def step(self, n=1):
        _bcheck(lib().lb_batch_step(self._b, int(n)), self._b)
        return self

    def configure(self, schedule, tile=0, steps_per_launch=64):
        _bcheck(lib().lb_batch_configure(self._b, int(schedule), int(tile), int(steps_per_launch)), self._b)

    def info(self):
        v = [ctypes.c_int() for _ in range(5)]
        nc = lib().lb_batch_info(self._b, *(ctypes.byref(x) for x in v))
        if nc < 0:
            _bcheck(nc, self._b)
        return {"items": v[0].value, "grid": v[1].value, "schedule": v[2].value, "tile": v[3].value,
                "graphs": v[4].value, "tile_candidates": nc}

    def autotune(self, trial_steps=16):
        nc = self.info()["tile_candidates"]
        ms = np.zeros(2 * nc)
        sch, tile, taken = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
        _bcheck(lib().lb_batch_autotune(self._b, int(trial_steps), ctypes.byref(sch), ctypes.byref(tile),
                                        ctypes.byref(taken), _dp(ms), 2 * nc), self._b)
        return {"schedule": sch.value, "tile": tile.value, "steps_taken": taken.value,
                "ms_per_step": ms.reshape(2, nc).tolist()}

    def observables(self, r, check=True):
        o = LbObs()
        rc = lib().lb_batch_observables(self._b, int(r), ctypes.byref(o))
        if rc not in (LB_OK, LB_EUNSTABLE) or (check and rc != LB_OK):
            _bcheck(rc, self._b)
        return {"mass": np.array(o.mass[:]), "mom": np.array(o.mom[:]), "Nu": o.Nu, "E": o.E, "step": o.step,
                "wall_fx": np.array(o.wall_fx[:]),
                "n_fluid": o.n_fluid, "n_bad": o.n_bad, "status": o.status}

    def fields(self, r):
        ny, nx = self.shapes[r]
        out = {k: np.zeros((ny, nx)) for k in ("rho1", "rho2", "T", "ux", "uy")}
        _bcheck(lib().lb_batch_get_fields(self._b, int(r), *(_dp(out[k]) for k in ("rho1", "rho2", "T", "ux", "uy"))),
                self._b)
        return out

    def get_state(self, r):
        ny, nx = self.shapes[r]
        st = np.zeros((27, ny, nx))
        _bcheck(lib().lb_batch_get_state(self._b, int(r), _dp(st), st.nbytes), self._b)
        return st

    def stress(self, r, field=True):
        """lb_batch_stress of replica r (see Lattice.stress)."""
        ny, nx = self.shapes[r]
        out, row = np.zeros(4), np.zeros(ny)
        f = np.zeros((ny, nx)) if field else None
        _bcheck(lib().lb_batch_stress(self._b, int(r), _dp(out), _dp(row), _dp(f)), self._b)
        return {"Sigma": out[0], "visc": out[1], "pint": out[2], "pforce": out[3], "row": row, "sxy": f}

    def sync(self):
        return lib().lb_batch_sync(self._b)

    def set_wait_budget(self, cycles, withhold_item=-1):
        _bcheck(lib().lb_batch_set_wait_budget(self._b, int(cycles), int(withhold_item)), self._b)

    def close(self):
        if getattr(self, "_b", None) and self._b.value:
            lib().lb_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nusselt_mean(T0, T_down, params, rho1, rho2, n_steps, mask=None, precision=LB_FP64, ckpt_every=None):
    """Differentiable J = time-averaged Nusselt number over n_steps steps started from the rest
    equilibrium with temperature field T0 (torch tensor [ny, nx], float64) and bottom-wall
    temperature T_down (0-d torch tensor); backward gives dJ/dT0 and dJ/dT_down from the library's
    discrete adjoint (lb_adjoint)."""
    import torch

    class _NusseltMean(torch.autograd.Function):
        @staticmethod
        def forward(ctx, t0, td):
            p = dict(params, T_down=float(td))
            g = Lattice(p, rho1, rho2, t0.detach().cpu().double().numpy(), mask=mask, precision=precision)
            J, dT0, dTd = g.adjoint(n_steps, ckpt_every)
            g.close()
            ctx.save_for_backward(torch.from_numpy(dT0).to(t0.dtype).to(t0.device),
                                  torch.tensor(dTd, dtype=td.dtype, device=td.device))
            return torch.tensor(J, dtype=t0.dtype, device=t0.device)

        @staticmethod
        def backward(ctx, grad_out):
            dT0, dTd = ctx.saved_tensors
            return grad_out * dT0, grad_out * dTd

    return _NusseltMean.apply(T0, T_down)
