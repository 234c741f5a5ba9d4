"""Regression of the CUDA path against the paper's accuracy tests (Sec. 4),
at sizes beyond the CPU pins:

* Sod shock tube (Sec. 4.2) on 512 x 16 x 16 cells, FP32, along x, y, z:
  against the exact Riemann solution (shock and contact within 2 cells, the
  shock at most 4 cells wide, rarefaction error under 3 %);
* acoustic wave (Sec. 4.1), FP64 (as in the paper), N x N x 16 cells with
  N = 64, 128, 256: L1 order close to 2 (paper: N^-1.9);
* Sedov-Taylor blast (Sec. 4.3), FP32, 128^3: shock radius within 2.5 cells
  of 1.15 (E t^2 / rho)^(1/5), compression below 4 and above the coarse
  oracle runs.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import riemann  # noqa: E402
from paper_0907_3390_gb300 import binding as B  # noqa: E402
from paper_0907_3390_gb300 import hierarchy as hm  # noqa: E402
from paper_0907_3390_gb300 import workloads as wl  # noqa: E402

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def run_to(S, D, t_end, cfl=0.5):
    """Sweep sets up to t_end with dt from Eq. CFL before each xyz set (held
    for the zyx set), the last dt clipped to land on t_end."""
    t, dt = 0.0, None
    while t < t_end - 1e-12:
        if B.gamer_hydro_get_parity(S.h, 0) == 0 or dt is None:
            dt = B.gamer_hydro_cfl_dt(S.h, D, cfl)
        step = min(dt, t_end - t)
        S.step(D, step)
        t += step
    torch.cuda.synchronize()
    return t


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_sod_fp32_against_exact(axis):
    u, npg, bc = wl.sod(axis, 512, 16)
    H, st = wl.single_level(u, npg, bc=bc)
    S = B.Solver(G, B.GAMER_LIMITER_VANLEER, B.GAMER_FP32)
    D = B.DeviceHierarchy(H, st, torch.float32)
    N = 512
    dx = H.levels[0].dh
    t = run_to(S, D, 0.2 * N * dx)
    d = hm.patches_to_domain(D.u[0].double().cpu().numpy(), npg)
    d = np.moveaxis(d, 3 - axis, 3)[:, 5, 9, :]
    r = d[0]
    v = d[1 + axis] / r
    P = (G - 1) * (d[4] - 0.5 * r * v * v)
    x = (np.arange(N) + 0.5) * dx
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    w = riemann.wave_positions(L, R, G)
    x0 = 0.5 * N * dx
    xi = (x - x0) / t
    re, ve, pe = riemann.sample(L, R, G, xi)
    rs = re[np.searchsorted(xi, w["shock"]) - 1]
    cross = lambda f, lev: x[np.nonzero((f[:-1] - lev) * (f[1:] - lev) <= 0)[0]]
    assert np.min(np.abs(cross(r, 0.5 * (rs + 0.125)) - (x0 + w["shock"] * t))) < 2 * dx
    rl = re[np.searchsorted(xi, w["contact"]) - 1]
    assert np.min(np.abs(cross(r, 0.5 * (rl + rs)) - (x0 + w["contact"] * t))) < 2 * dx
    lo, hi = 0.125 + 0.1 * (rs - 0.125), 0.125 + 0.9 * (rs - 0.125)
    assert np.sum((r > lo) & (r < hi) & (x > x0 + w["contact"] * t + 0.05 * N * dx)) <= 4
    fan = (x > x0 + w["rare_head"] * t + 4 * dx) & (x < x0 + w["rare_tail"] * t - 4 * dx)
    assert np.max(np.abs(r[fan] - re[fan]) / re[fan]) < GOLD["sod_max_rarefaction_error"]["value"]
    assert np.mean(np.abs(r - re)) < 5e-3
    S.close()


def test_acoustic_fp64_second_order():
    errs, Ns = [], [64, 128, 256]
    for N in Ns:
        u, k, npg = wl.acoustic_wave(N, amp=1e-6, n_z=16)
        H, st = wl.single_level(u, npg)
        S = B.Solver(G, B.GAMER_LIMITER_VANLEER, B.GAMER_FP64)
        D = B.DeviceHierarchy(H, st, torch.float64)
        period = 2 * np.pi / np.linalg.norm(k)
        dx = H.levels[0].dh
        n_calls = 2 * int(np.ceil(period / (0.5 * dx) / 2))
        dt = period / n_calls
        for _ in range(n_calls):
            S.step(D, dt)
        torch.cuda.synchronize()
        rho = hm.patches_to_domain(D.u[0].cpu().numpy(), npg)[0]
        z, y, x = np.meshgrid((np.arange(16) + 0.5) * dx, (np.arange(N) + 0.5) * dx, (np.arange(N) + 0.5) * dx,
                              indexing="ij")
        exact = 1.0 + 1e-6 * np.sin(k[0] * x + k[1] * y) * np.cos(np.linalg.norm(k) * n_calls * dt)
        errs.append(np.mean(np.abs(rho - exact)) / 1e-6)
        S.close()
    slope = np.polyfit(np.log(Ns), np.log(errs), 1)[0]
    assert -2.3 < slope < -1.7, (errs, slope)


def test_sedov_fp32_128():
    N = 128
    s = (N, N, N)
    zr = np.zeros(s)
    u = wl.prim_to_cons(np.ones(s), zr, zr, zr, np.full(s, 1e-5))
    dh = 1.0 / N
    c = N // 2
    u[4, c - 1:c + 1, c - 1:c + 1, c - 1:c + 1] += 1.0 / (8 * dh ** 3)
    H, st = wl.single_level(u, (N // 16,) * 3)
    S = B.Solver(G, B.GAMER_LIMITER_VANLEER, B.GAMER_FP32)
    D = B.DeviceHierarchy(H, st, torch.float32)
    beta = GOLD["sedov_beta"]["value"]
    t = run_to(S, D, (0.3 / beta) ** 2.5)
    rs = beta * (t * t) ** 0.2
    rho = hm.patches_to_domain(D.u[0].double().cpu().numpy(), (N // 16,) * 3)[0]
    cc = (np.arange(N) + 0.5) * dh - 0.5
    zz, yy, xx = np.meshgrid(cc, cc, cc, indexing="ij")
    rr = np.sqrt(xx * xx + yy * yy + zz * zz).ravel()
    bins = np.arange(0, 0.5, dh)
    idx = np.digitize(rr, bins)
    cnt = np.bincount(idx, minlength=len(bins) + 1)[1:len(bins)]
    prof = np.bincount(idx, weights=rho.ravel(), minlength=len(bins) + 1)[1:len(bins)] / np.maximum(cnt, 1)
    rc = 0.5 * (bins[1:] + bins[:-1])
    assert abs(rc[np.argmax(prof)] - rs) < 2.5 * dh
    assert rho.max() < GOLD["sedov_strong_shock_compression"]["value"]
    assert prof.max() > 2.5                      # sharper than the 32^3 / 48^3 oracle runs
    sums, nb = B.gamer_hydro_check(S.h, D)
    assert nb == 0
    assert sums[0] == pytest.approx(1.0, rel=1e-6)
    assert sums[4] == pytest.approx(1.0 + 1.5e-5, rel=1e-6)
    S.close()
