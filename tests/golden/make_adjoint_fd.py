"""Write ``adjoint_fd_emulsion_512x256.txt``: central finite differences of the FP64 oracle's
time-averaged Nusselt number on the adjoint workload.

J = (1/N) sum_{t=1..N} Nu(S_t) (Eq. NuTime) over N = 2000 steps of the 512 x 256 emulsion
(phi = 0.7, ``inputs.emulsion_512x256``), started from the rest equilibrium of its initial fields.
For each seeded direction d_k (``inputs.uniform(500 + k)`` - 1/2 on fluid nodes, 0 on the wall
rows) the file holds (J(T0 + eps d_k) - J(T0 - eps d_k)) / (2 eps), and for T_down
(J(T_down + eps) - J(T_down - eps)) / (2 eps), with eps = 1e-6.  Only ``oracle/`` computes
anything here; ``inputs`` only draws the seeded fields and directions.

Run from the repository root: ``python tests/golden/make_adjoint_fd.py`` (about half an hour on
8 cores with the OpenMP oracle).
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2109_12565_gb300 import inputs as I  # noqa: E402

N_STEPS = 2000
EPS = 1e-6
N_DIRS = 8
OUT = os.path.join(HERE, "adjoint_fd_emulsion_512x256.txt")


def direction(w, k):
    d = I.uniform(500 + k, w.T0.size).reshape(w.T0.shape) - 0.5
    d[0, :] = d[-1, :] = 0.0
    return d


def main():
    w = I.emulsion_512x256()
    J = lambda p, T0: float(O.nusselt_mean(p, w.rho1, w.rho2, T0, N_STEPS, mask=w.mask, omp=True))  # noqa: E731
    t0 = time.time()
    rows = []
    J0 = J(w.params, w.T0)
    print(f"J0 = {J0!r} ({time.time() - t0:.0f} s)", flush=True)
    for k in range(N_DIRS):
        d = direction(w, k)
        fd = (J(w.params, w.T0 + EPS * d) - J(w.params, w.T0 - EPS * d)) / (2 * EPS)
        rows.append((f"dir{500 + k}", float(fd)))
        print(f"direction {500 + k}: {fd!r} ({time.time() - t0:.0f} s)", flush=True)
    pp = dict(w.params, T_down=w.params["T_down"] + EPS)
    pm = dict(w.params, T_down=w.params["T_down"] - EPS)
    fd = (J(pp, w.T0) - J(pm, w.T0)) / (2 * EPS)
    rows.append(("T_down", float(fd)))
    print(f"T_down: {fd!r} ({time.time() - t0:.0f} s)", flush=True)
    with open(OUT + ".tmp", "w") as fh:
        fh.write("# Central differences (eps = 1e-6) of J = (1/N) sum_{t=1..N} Nu(S_t), Eq. NuTime, N = 2000,\n")
        fh.write("# on the 512 x 256 emulsion (phi = 0.7, inputs.emulsion_512x256), computed by the FP64 C oracle\n")
        fh.write("# (OpenMP build) with tests/golden/make_adjoint_fd.py.  dir<s>: direction uniform(s) - 1/2 of T0\n")
        fh.write("# on fluid nodes (0 on the wall rows); T_down: the bottom-wall temperature.\n")
        fh.write(f"J0 {J0!r}\n")
        for name, v in rows:
            fh.write(f"{name} {v!r}\n")
    os.replace(OUT + ".tmp", OUT)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
