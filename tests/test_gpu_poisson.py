"""The red-black SOR Poisson solver on the GPU (gamer_poisson_sor) against
the oracle (Sec. 2.3; reading R24):

* FP64, a fixed number of iterations (tol = 0): bit for bit on every group
  (the updates are independent within a colour and follow the oracle's
  order of operations);
* FP32: within 1e-5 of the FP64 oracle relative to the potential's scale
  after 25 iterations (single rounding per update, no accumulation beyond a
  few ulps per iteration at this contraction rate);
* converged with a tolerance: the exact discrete solution, and iteration
  counts within one of the oracle's (the residual norms are summed in a
  different order, so the last iteration can fall either side).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_0907_3390_gb300 import binding as B  # noqa: E402

pytestmark = pytest.mark.gpu
P, N = 18, 16
G_AMMA = 5.0 / 3.0


def data(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, P, P, P)), rng.standard_normal((n, N, N, N))


def test_sor_fp64_bitwise():
    phi, rho = data(6, 1)
    dphi = torch.tensor(phi, device="cuda")
    it = torch.zeros(6, dtype=torch.int32, device="cuda")
    B.gamer_poisson_sor(B.GAMER_FP64, torch.tensor(rho, device="cuda"), dphi, 0.7, 1.7, 25, 0.0, it)
    got = dphi.cpu().numpy()
    assert np.all(it.cpu().numpy() == 25)
    for g in range(6):
        want, n_it, _ = oracle.sor_group(phi[g], rho[g], 0.7, 1.7, 25, 0.0)
        assert n_it == 25
        assert np.array_equal(got[g], want), g


def test_sor_fp32_tolerance():
    phi, rho = data(4, 2)
    phi32, rho32 = phi.astype(np.float32), rho.astype(np.float32)
    dphi = torch.tensor(phi32, device="cuda")
    B.gamer_poisson_sor(B.GAMER_FP32, torch.tensor(rho32, device="cuda"), dphi, 0.7, 1.7, 25, 0.0)
    got = dphi.cpu().numpy().astype(np.float64)
    for g in range(4):
        want, _, _ = oracle.sor_group(phi32[g].astype(np.float64), rho32[g].astype(np.float64), 0.7, 1.7, 25, 0.0)
        assert np.abs(got[g] - want).max() / np.abs(want).max() <= 1e-5, g


def lap(phi):
    return (((((phi[1:-1, 1:-1, 2:] + phi[1:-1, 2:, 1:-1]) + phi[2:, 1:-1, 1:-1]) + phi[1:-1, 1:-1, :-2]) +
             phi[1:-1, :-2, 1:-1]) + phi[:-2, 1:-1, 1:-1]) - 6.0 * phi[1:-1, 1:-1, 1:-1]


def test_sor_converged_exact_solution_and_counts():
    rng = np.random.default_rng(3)
    n = 5
    exact = rng.standard_normal((n, P, P, P))
    coef = 0.5
    rho = np.stack([lap(e) / coef for e in exact])
    start = exact.copy()
    start[:, 1:-1, 1:-1, 1:-1] = 0.0
    omega = 2.0 / (1.0 + np.sin(np.pi / (N + 1)))
    dphi = torch.tensor(start, device="cuda")
    it = torch.zeros(n, dtype=torch.int32, device="cuda")
    B.gamer_poisson_sor(B.GAMER_FP64, torch.tensor(rho, device="cuda"), dphi, coef, omega, 5000, 1e-13, it)
    got = dphi.cpu().numpy()
    its = it.cpu().numpy()
    for g in range(n):
        _, n_it, _ = oracle.sor_group(start[g], rho[g], coef, omega, 5000, 1e-13)
        assert abs(int(its[g]) - n_it) <= 1 and its[g] < 5000, (g, its[g], n_it)
        assert np.allclose(got[g], exact[g], rtol=0, atol=1e-10), g


def _hierarchy():
    from paper_0907_3390_gb300 import hierarchy as hm

    def score(level, centres):
        x, y, z = (centres[a][:, 0, 0, 0] for a in range(3))
        r = np.sqrt((x - 0.45) ** 2 + (y - 0.55) ** 2 + (z - 0.5) ** 2)
        return 0.3 - r if level == 0 else 0.17 - r
    return hm.build_hierarchy((3, 3, 3), score, 3)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_prepare_sor_gravity_chain_matches_oracle(prec):
    """The refined levels' Poisson path and the gravity operator on a
    3-level hierarchy: SOR inputs from the coarser level's potential
    (gamer_poisson_prepare), SOR iterations, then G with the solved
    potential; FP64 bit for bit against the oracle's chain, FP32 within
    1e-5 of it (inputs rounded to float first)."""
    from paper_0907_3390_gb300 import workloads as wl
    p, tdt, npdt = {"f32": (B.GAMER_FP32, torch.float32, np.float32),
                    "f64": (B.GAMER_FP64, torch.float64, np.float64)}[prec]
    H = _hierarchy()
    st = wl.level_fields(H, lambda x, y, z, dh: (1.0 + 0.4 * np.sin(6 * x) * np.cos(4 * y) + 0.3 * z,
                                                0.2 * np.cos(5 * z), 0 * x, -0.1 + 0 * x, 1.0 + 0 * x))
    st = [np.asarray(s).astype(npdt).astype(np.float64) for s in st]
    rng = np.random.default_rng(41)
    S = B.Solver(G_AMMA, B.GAMER_LIMITER_VANLEER, p)
    D = B.DeviceHierarchy(H, st, tdt)
    O = oracle.OracleLevels(H, st)
    coef, omega, iters, dt = 0.3, 1.6, 12, 0.002
    for l in range(1, H.n_levels):
        c = H.cell_centres(l - 1)
        phi_c = (np.sin(3 * c[0]) * np.cos(2 * c[1]) + 0.5 * c[2] + 0.05 * rng.standard_normal(c[0].shape))
        phi_c = phi_c.astype(npdt).astype(np.float64)
        n = H.levels[l].n_groups
        want_phi, want_rho = O.poisson_prepare(l, phi_c)
        dphi = torch.empty((n, 18, 18, 18), dtype=tdt, device="cuda")
        drho = torch.empty((n, 16, 16, 16), dtype=tdt, device="cuda")
        B.gamer_poisson_prepare(S.h, D, l, torch.tensor(phi_c, dtype=tdt, device="cuda"), dphi, drho)
        torch.cuda.synchronize()
        assert np.array_equal(drho.double().cpu().numpy(), want_rho)
        got = dphi.double().cpu().numpy()
        if prec == "f64":
            assert np.array_equal(got, want_phi)
        else:
            assert np.abs(got - want_phi).max() <= 1e-6 * np.abs(want_phi).max()
        # SOR on the prepared blocks, then G on the level
        B.gamer_poisson_sor(p, drho, dphi, coef, omega, iters, 0.0)
        solved = np.stack([oracle.sor_group(want_phi[g], want_rho[g], coef, omega, iters, 0.0)[0]
                           for g in range(n)])
        B.gamer_gravity_update(p, D.u[l], dphi, H.levels[l].dh, dt)
        O.gravity(l, solved, dt)
        torch.cuda.synchronize()
        got_phi = dphi.double().cpu().numpy()
        got_u = D.u[l].double().cpu().numpy()
        if prec == "f64":
            assert np.array_equal(got_phi, solved)
            assert np.array_equal(got_u, O.u[l])
        else:
            assert np.abs(got_phi - solved).max() <= 1e-5 * np.abs(solved).max()
            scale = np.abs(O.u[l]).reshape(5, -1).max(1)[:, None]
            assert (np.abs(got_u - O.u[l]).reshape(5, -1) / scale).max() <= 1e-5
    S.close()


def test_prepare_rejects_level_zero():
    H = _hierarchy()
    from paper_0907_3390_gb300 import workloads as wl
    st = wl.level_fields(H, lambda x, y, z, dh: (1.0 + 0 * x, 0 * x, 0 * x, 0 * x, 1.0 + 0 * x))
    S = B.Solver(G_AMMA, B.GAMER_LIMITER_VANLEER, B.GAMER_FP64)
    D = B.DeviceHierarchy(H, st, torch.float64)
    t = torch.zeros((8, 8, 8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(B.GamerError) as e:
        B.gamer_poisson_prepare(S.h, D, 0, t, t, t)
    assert e.value.code == B.GAMER_ERR_ARG
    S.close()
