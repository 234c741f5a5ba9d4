"""The allocation-free diagnostics entry point.

gamer_hydro_diagnose_noalloc serves callers that cannot call cudaMalloc
(a thread that must not synchronise the device, code inside a memory arena
that owns the whole GPU): it takes no handle and keeps its scratch in a
fixed array inside the library.  Its results must match the handle-based
gamer_hydro_diagnose on two calls in a row (the second call on a changed
state, so stale scratch from the first call would show), and sizes above
its fixed limit must be refused.

This file is named to run last, so that a run stopping at the first
failure has already run every other test; it also passes alone.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_0907_3390_gb300 import binding as B  # noqa: E402
from paper_0907_3390_gb300 import hierarchy as hm  # noqa: E402
from paper_0907_3390_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


def _amr():
    def score(level, centres):
        x, y, z = (centres[a][:, 0, 0, 0] for a in range(3))
        r = np.sqrt((x - 0.45) ** 2 + (y - 0.55) ** 2 + (z - 0.5) ** 2)
        return 0.3 - r if level == 0 else 0.17 - r
    H = hm.build_hierarchy((3, 3, 3), score, 3)

    def prim(x, y, z, dh):
        rho = 1.0 + 0.3 * np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
        return rho, 0.3 * np.cos(2 * np.pi * y), 0.2 * np.sin(2 * np.pi * z), -0.25 * np.cos(2 * np.pi * x), \
            0.8 + 0.1 * np.cos(2 * np.pi * (x + y))
    return H, wl.level_fields(H, prim)


@pytest.mark.parametrize("prec", [(B.GAMER_FP32, torch.float32), (B.GAMER_FP64, torch.float64)])
@pytest.mark.parametrize("case", ["uniform", "amr"])
def test_noalloc_matches_handle_diagnose_twice(prec, case):
    if case == "uniform":
        u, npg = wl.smooth_grf(64, seed=9)
        H, st = wl.single_level(u, npg)
    else:
        H, st = _amr()
    S = B.Solver(G, 0, prec[0])
    # the no-handle call returns the shared-time-step dt of Eq. CFL: compare
    # with a handle in that mode (individual time steps scale level l by 2^l)
    B.gamer_hydro_set_time_steps(S.h, 0)
    D = B.DeviceHierarchy(H, st, prec[1])
    for call in range(2):
        torch.cuda.synchronize()
        ref_dt, ref_sums, ref_nb = B.gamer_hydro_diagnose(S.h, D, 0.5)
        dt, sums, nb = B.gamer_hydro_diagnose_noalloc(G, prec[0], D, 0.5)
        assert dt == ref_dt or (np.isnan(dt) and np.isnan(ref_dt))   # NaN once a bad cell is planted
        assert nb == ref_nb == call
        assert np.allclose(sums, ref_sums, rtol=1e-13, atol=1e-13 * np.abs(ref_sums).max())
        if call == 0:
            # change the state (one step, and a planted bad cell) for the second call
            S.step(D, 0.3 * dt)
            D.u[0][0, 5, 1, 2, 3] = -1.0
    S.close()


def test_noalloc_rejects_sizes_above_its_limit():
    H = wl.uniform_hierarchy((1, 1, 1))
    D = B.DeviceHierarchy(H, [np.ones((5, 8, 8, 8))], torch.float32)
    D._levels[0].n_groups = 65537          # more groups than the fixed scratch holds
    with pytest.raises(B.GamerError) as e:
        B.gamer_hydro_diagnose_noalloc(G, B.GAMER_FP32, D, 0.5)
    assert e.value.code == B.GAMER_ERR_ARG
    assert "65536" in B.gamer_hydro_last_error(None)
