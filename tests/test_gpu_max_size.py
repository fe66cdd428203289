"""Near the largest lattice the library accepts: 27 * pitch * ny must stay below 2^31 population slots
per buffer, and 16384 x 4608 nodes (75.5 M, 2.04e9 slots) is 95% of that.

The lattice is made of 16 x 9 copies of one fully periodic 1024 x 512 emulsion.  Every node's update
depends only on its 5 x 5 neighbourhood, so on a periodic lattice each copy must evolve exactly like
the single 1024 x 512 lattice: all 144 copies are bit-identical to each other (the kernels' arithmetic
does not depend on where a node sits), and copy (0, 0) equals the FP64 oracle of the single lattice
within the form's tolerance (FP64 and double-float: max abs <= 1e-12 after 4 steps; FP32-shifted:
norm-relative <= 1e-4).  The droplet analysis of the whole lattice finds 144 times the droplets and
links the oracle finds on copy (0, 0)'s own density field, with the same sizes.  This exercises the
31-bit index arithmetic of the step, of the field read-back and of the droplet analysis at full scale.
"""
import numpy as np
import pytest

import oracle as O
from paper_2109_12565_gb300 import build as B
from paper_2109_12565_gb300 import inputs as I
from paper_2109_12565_gb300 import lb

pytestmark = pytest.mark.gpu

CX, CY = 16, 9  # copies along x and y
STEPS = 4


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    B.build()


@pytest.fixture(scope="module")
def small():
    """The periodic 1024 x 512 emulsion, its oracle fields after STEPS steps, and its tiled inputs."""
    w = I.emulsion_1024x512()
    p = dict(w.params)
    p["periodic_y"] = 1
    ny, nx = int(p["ny"]), int(p["nx"])
    T0 = np.broadcast_to(0.5 * np.cos(2 * np.pi * (np.arange(ny) + 0.5) / ny)[:, None], (ny, nx)).copy()
    o = O.Oracle(p, w.rho1, w.rho2, T0, omp=True)
    o.step(STEPS)
    big = dict(p)
    big["nx"], big["ny"] = CX * nx, CY * ny
    tiled = [np.tile(a, (CY, CX)) for a in (w.rho1, w.rho2, T0)]
    return p, o.fields(), big, tiled


@pytest.mark.parametrize("precision", [lb.LB_FP64, lb.LB_FP32_SHIFTED, lb.LB_DF64])
def test_near_maximum_lattice_copies_match_oracle(small, precision):
    p, fo, big, tiled = small
    ny, nx = int(p["ny"]), int(p["nx"])
    assert 27 * big["nx"] * big["ny"] < 2 ** 31 <= 27 * big["nx"] * (big["ny"] + 256)
    g = lb.Lattice(big, *tiled, precision=precision)
    g.step(STEPS)
    fg = g.fields()
    for k in ("rho1", "rho2", "T", "ux", "uy"):
        v = fg[k].reshape(CY, ny, CX, nx)
        first = v[0, :, 0, :]
        assert np.array_equal(v, np.broadcast_to(first[None, :, None, :], v.shape)), k
        if precision == lb.LB_FP32_SHIFTED:
            if k in ("rho1", "rho2", "T"):
                assert np.abs(first - fo[k]).max() / np.abs(fo[k]).max() <= 1e-4, k
        else:
            assert np.abs(first - fo[k]).max() <= 1e-12, k
    r1 = fg["rho1"][:ny, :nx].copy()
    del fg
    d = g.droplets(0.8, arrays=False)
    od = O.droplets(p, r1, 0.8)
    assert od["n"] > 300
    assert d["n"] == CX * CY * od["n"] and d["n_links"] == CX * CY * len(od["links"])
    g.close()
