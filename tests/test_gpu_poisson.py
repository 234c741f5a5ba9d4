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
