"""Convergence studies of the CUDA path at scale: regression benches of the
paper's accuracy tests (Sec. 4), run through the benchmark's call,
gamer_hydro_step_pair (an xyz and a zyx sweep set per call, dt from
Eq. CFL on the device, CFL 0.5), and compared with the exact solutions at
the time actually reached:

* Sod shock tube (Sec. 4.2), FP32, N = 256 ... 2048 cells along x (x 16 x
  16, outflow ends), t ~ 0.2: L1(rho) against the exact Riemann solution
  falls with N at order 0.6 to 1.2 (first order at the discontinuities),
  shock and contact within 2 cells at every N;
* standing acoustic wave (Sec. 4.1), FP64, N = 64 ... 512 (x 16), one
  period: L1(rho) falls at order 1.7 to 2.3 (the paper reports N^-1.9);
* Sedov-Taylor blast (Sec. 4.3), FP32, N = 64, 128, 256: shock radius
  within 2.5 cells of 1.15 (E t^2 / rho)^(1/5), the peak of the radial
  density profile rising with N and below the strong-shock limit 4.

Each test prints its table (pytest -s).
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


def run_pairs(S, D, t_end, cfl=0.5):
    """Pairs of sweep sets until t_end is reached; returns the time reached."""
    t = 0.0
    while t < t_end:
        B.gamer_hydro_step_pair(S.h, D, cfl)
        dt, _, _, nb = B.gamer_hydro_step_result(S.h)
        assert nb == 0
        t += 2.0 * dt
    torch.cuda.synchronize()
    return t


def order(ns, errs):
    return -np.polyfit(np.log(ns), np.log(errs), 1)[0]


def test_sod_convergence_fp32():
    Ns, errs = [256, 512, 1024, 2048], []
    L, R = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)
    w = riemann.wave_positions(L, R, G)
    for N in Ns:
        u, npg, bc = wl.sod(0, N, 16)
        H, st = wl.single_level(u, npg, bc=bc)
        S = B.Solver(G, B.GAMER_LIMITER_VANLEER, B.GAMER_FP32)
        D = B.DeviceHierarchy(H, st, torch.float32)
        dx = H.levels[0].dh
        t = run_pairs(S, D, 0.2 * N * dx)
        d = hm.patches_to_domain(D.u[0].double().cpu().numpy(), npg)[:, 5, 9, :]
        r = d[0]
        x = (np.arange(N) + 0.5) * dx
        x0 = 0.5 * N * dx
        xi = (x - x0) / t
        re = riemann.sample(L, R, G, xi)[0]
        errs.append(float(np.mean(np.abs(r - re))))
        rs = re[np.searchsorted(xi, w["shock"]) - 1]
        cross = lambda f, lev: x[np.nonzero((f[:-1] - lev) * (f[1:] - lev) <= 0)[0]]
        assert np.min(np.abs(cross(r, 0.5 * (rs + 0.125)) - (x0 + w["shock"] * t))) < 2 * dx, N
        rl = re[np.searchsorted(xi, w["contact"]) - 1]
        assert np.min(np.abs(cross(r, 0.5 * (rl + rs)) - (x0 + w["contact"] * t))) < 2 * dx, N
        S.close()
    p = order(Ns, errs)
    print("\nSod FP32 L1(rho):", dict(zip(Ns, [f"{e:.3e}" for e in errs])), f"order {p:.2f}")
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert 0.6 < p < 1.2, (errs, p)


def test_acoustic_convergence_fp64():
    Ns, errs = [64, 128, 256, 512], []
    amp = 1e-6
    for N in Ns:
        u, k, npg = wl.acoustic_wave(N, amp=amp, n_z=16)
        H, st = wl.single_level(u, npg)
        S = B.Solver(G, B.GAMER_LIMITER_VANLEER, B.GAMER_FP64)
        D = B.DeviceHierarchy(H, st, torch.float64)
        kk = float(np.linalg.norm(k))
        t = run_pairs(S, D, 2 * np.pi / kk)
        dx = H.levels[0].dh
        rho = hm.patches_to_domain(D.u[0].cpu().numpy(), npg)[0]
        z, y, x = np.meshgrid((np.arange(16) + 0.5) * dx, (np.arange(N) + 0.5) * dx, (np.arange(N) + 0.5) * dx,
                              indexing="ij")
        exact = 1.0 + amp * np.sin(k[0] * x + k[1] * y) * np.cos(kk * t)
        errs.append(float(np.mean(np.abs(rho - exact)) / amp))
        S.close()
    p = order(Ns, errs)
    print("\nacoustic FP64 L1(rho)/amp:", dict(zip(Ns, [f"{e:.3e}" for e in errs])), f"order {p:.2f}")
    assert all(a > b for a, b in zip(errs, errs[1:])), errs
    assert 1.7 < p < 2.3, (errs, p)


def test_sedov_convergence_fp32():
    beta = GOLD["sedov_beta"]["value"]
    rows = []
    peaks = []
    for N in (64, 128, 256):
        s = (N, N, N)
        zr = np.zeros(s)
        u = wl.prim_to_cons(np.ones(s), zr, zr, zr, np.full(s, 1e-5))
        dh = 1.0 / N
        c = N // 2
        u[4, c - 1:c + 1, c - 1:c + 1, c - 1:c + 1] += 1.0 / (8 * dh ** 3)
        H, st = wl.single_level(u, (N // 16,) * 3)
        S = B.Solver(G, B.GAMER_LIMITER_VANLEER, B.GAMER_FP32)
        D = B.DeviceHierarchy(H, st, torch.float32)
        t = run_pairs(S, D, (0.3 / beta) ** 2.5)
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
        r_peak = rc[np.argmax(prof)]
        rows.append((N, t, rs, r_peak, prof.max(), rho.max()))
        peaks.append(prof.max())
        assert abs(r_peak - rs) < 2.5 * dh, (N, r_peak, rs)
        assert rho.max() < GOLD["sedov_strong_shock_compression"]["value"], N
        S.close()
    print("\nSedov FP32 (N, t, r_s exact, r_peak, profile peak, max rho):")
    for r in rows:
        print("   ", " ".join(f"{v:.4g}" for v in r))
    assert peaks[0] < peaks[1] < peaks[2], peaks
