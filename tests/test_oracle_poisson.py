"""Pins of the oracle's red-black SOR Poisson solver of one patch group
(Sec. 2.3, Eqs. DiscretePoisson, Residual, SOR; reading R24):

* one iteration equals an independent numpy statement of the even and odd
  half-steps, bit for bit;
* converged, it reproduces an exact discrete solution (density built from
  the discrete Laplacian of a random potential) and the quadratic
  potential whose discrete Laplacian is exactly 6;
* converged, it agrees with a direct sparse solve of the same 16^3 system
  with random Dirichlet values and density;
* the stopping rule: a huge tol stops after one iteration, a tighter tol takes
  more iterations and leaves a smaller residual.
"""
import numpy as np
import pytest

import oracle

P, N = 18, 16


def lap(phi):
    c = phi[1:-1, 1:-1, 1:-1]
    return (((((phi[1:-1, 1:-1, 2:] + phi[1:-1, 2:, 1:-1]) + phi[2:, 1:-1, 1:-1]) + phi[1:-1, 1:-1, :-2]) +
             phi[1:-1, :-2, 1:-1]) + phi[:-2, 1:-1, 1:-1]) - 6.0 * c


def numpy_iteration(phi, rho, coef, omega):
    phi = phi.copy()
    k, j, i = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    w6 = omega / 6.0
    for color in (0, 1):
        R = lap(phi) - coef * rho
        sel = ((i + j + k) & 1) == color
        inner = phi[1:-1, 1:-1, 1:-1]
        inner[sel] = inner[sel] + w6 * R[sel]
    return phi


def test_one_iteration_bitwise():
    rng = np.random.default_rng(3)
    phi = rng.standard_normal((P, P, P))
    rho = rng.standard_normal((N, N, N))
    got, it, _ = oracle.sor_group(phi, rho, 0.37, 1.6, 1, 0.0)
    assert it == 1
    # the numpy statement updates colour by colour with whole-array residuals;
    # cells of one colour only read the other colour, so this is the same update
    assert np.array_equal(got, numpy_iteration(phi, rho, 0.37, 1.6))


def omega_opt():
    return 2.0 / (1.0 + np.sin(np.pi / (N + 1)))


def test_exact_discrete_solution():
    rng = np.random.default_rng(4)
    exact = rng.standard_normal((P, P, P))
    coef = 0.5
    rho = lap(exact) / coef
    start = exact.copy()
    start[1:-1, 1:-1, 1:-1] = 0.0
    got, it, res = oracle.sor_group(start, rho, coef, omega_opt(), 5000, 1e-15)
    assert it < 5000
    assert np.allclose(got, exact, rtol=0, atol=1e-11)
    # the ghost layer is kept
    assert np.array_equal(got[0], exact[0]) and np.array_equal(got[:, :, -1], exact[:, :, -1])


def test_quadratic_potential():
    z, y, x = np.meshgrid(np.arange(P) - 8.5, np.arange(P) - 8.5, np.arange(P) - 8.5, indexing="ij")
    exact = x * x + y * y + z * z
    assert np.all(lap(exact) == 6.0)
    coef = 2.0
    rho = np.full((N, N, N), 6.0 / coef)
    start = exact.copy()
    start[1:-1, 1:-1, 1:-1] = 0.0
    got, it, res = oracle.sor_group(start, rho, coef, omega_opt(), 5000, 1e-15)
    assert np.allclose(got, exact, rtol=1e-13, atol=1e-11)


def test_against_direct_sparse_solve():
    sp = pytest.importorskip("scipy.sparse")
    spl = pytest.importorskip("scipy.sparse.linalg")
    rng = np.random.default_rng(5)
    phi = rng.standard_normal((P, P, P))
    rho = rng.standard_normal((N, N, N))
    coef = 0.8
    # A x = b with x the interior: 6 x - sum of interior neighbours = boundary terms - coef rho
    n = N ** 3
    idx = np.arange(n).reshape(N, N, N)
    rows, cols, vals = [idx.ravel()], [idx.ravel()], [np.full(n, 6.0)]
    b = -coef * rho.copy()
    for ax in range(3):
        for sd in (-1, 1):
            src = np.roll(idx, -sd, axis=ax)
            inside = np.ones((N, N, N), dtype=bool)
            sl = [slice(None)] * 3
            sl[ax] = N - 1 if sd == 1 else 0
            inside[tuple(sl)] = False
            rows.append(idx[inside]); cols.append(src[inside]); vals.append(np.full(inside.sum(), -1.0))
            # boundary neighbours go to the right-hand side
            ghost = phi.copy()[1:-1, 1:-1, 1:-1] * 0
            shifted = np.roll(np.arange(P), -sd)[1:-1]
            sl_full = [slice(1, -1)] * 3
            sl_full[ax] = shifted
            nb = phi[tuple(sl_full)]
            b[~inside] += nb[~inside]
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    direct = spl.spsolve(A, b.ravel()).reshape(N, N, N)
    got, it, res = oracle.sor_group(phi, rho, coef, omega_opt(), 5000, 1e-15)
    assert np.allclose(got[1:-1, 1:-1, 1:-1], direct, rtol=0, atol=1e-10)


def test_stopping_rule():
    rng = np.random.default_rng(6)
    phi = rng.standard_normal((P, P, P))
    rho = rng.standard_normal((N, N, N))
    _, it1, _ = oracle.sor_group(phi, rho, 1.0, 1.5, 100, 1e6)
    assert it1 == 1
    _, ita, ra = oracle.sor_group(phi, rho, 1.0, 1.5, 1000, 1e-6)
    _, itb, rb = oracle.sor_group(phi, rho, 1.0, 1.5, 1000, 1e-10)
    assert 1 < ita < itb < 1000 and rb < ra


# ------------------------------------------ SOR inputs of a refined level

def _two_level_central():
    from paper_0907_3390_gb300 import hierarchy as hm

    def score(level, centres):
        x, y, z = (centres[a][:, 0, 0, 0] for a in range(3))
        return 0.2 - np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
    return hm.build_hierarchy((4, 4, 4), score, 2)


def _states(H):
    from paper_0907_3390_gb300 import workloads as wl
    return wl.level_fields(H, lambda x, y, z, dh: (1.0 + 0.5 * np.sin(7 * x) * np.cos(5 * y) + 0.2 * z,
                                                  0 * x, 0 * x, 0 * x, 1.0 + 0 * x))


def test_prepare_linear_potential_exact():
    """Min-Mod interpolation (R8) is exact on linear data, so a linear coarse
    potential gives the same linear function at every fine cell and ghost
    cell of every group (reading R26; the refined region lies far from the
    periodic boundary, so no stencil wraps)."""
    H = _two_level_central()
    st = _states(H)
    a = (0.3, 1.7, -0.6, 0.9)
    c0 = H.cell_centres(0)
    phi_c = a[0] + a[1] * c0[0] + a[2] * c0[1] + a[3] * c0[2]
    O = oracle.OracleLevels(H, st)
    phi, _ = O.poisson_prepare(1, phi_c)
    L1 = H.levels[1]
    i = np.arange(P) - 1 + 0.5
    for g in range(L1.n_groups):
        gx, gy, gz = (16 * L1.coords[g] + 0.0)
        z, y, x = np.meshgrid((gz + i) * L1.dh, (gy + i) * L1.dh, (gx + i) * L1.dh, indexing="ij")
        want = a[0] + a[1] * x + a[2] * y + a[3] * z
        assert np.allclose(phi[g], want, rtol=0, atol=1e-12), g


def test_prepare_density_blocks():
    """The density blocks are the level's density, rearranged from the patch
    layout to one x-fastest 16^3 block per group."""
    H = _two_level_central()
    st = _states(H)
    c0 = H.cell_centres(0)
    O = oracle.OracleLevels(H, st)
    _, rho = O.poisson_prepare(1, np.zeros_like(c0[0]))
    n = H.levels[1].n_groups
    u0 = np.asarray(st[1][0]).reshape(n, 2, 2, 2, 8, 8, 8)          # g, pz, py, px, z, y, x
    want = u0.transpose(0, 1, 4, 2, 5, 3, 6).reshape(n, 16, 16, 16)
    assert np.array_equal(rho, want)


def test_prepare_rejects_level_zero():
    H = _two_level_central()
    O = oracle.OracleLevels(H, _states(H))
    with pytest.raises(ValueError):
        O.poisson_prepare(0, np.zeros(1))


@pytest.mark.parametrize("omega", [1.0, 1.5])
def test_asymptotic_convergence_factor(omega):
    """The red-black iteration on the 16^3 Dirichlet problem contracts the
    error, asymptotically, by the spectral radius the theory of SOR gives
    for consistently ordered matrices: with the Jacobi radius
    mu = cos(pi / 17) of the 7-point Laplacian on 16 interior cells per
    axis, lambda solves (lambda + omega - 1)^2 = lambda omega^2 mu^2, the
    largest root being ((omega mu + sqrt(omega^2 mu^2 - 4 (omega - 1))) / 2)^2
    below the optimal omega (mu^2 for Gauss-Seidel, omega = 1).  A wrong
    colouring, weight or neighbour sum changes the rate."""
    rng = np.random.default_rng(9)
    phi = np.zeros((P, P, P))
    phi[1:-1, 1:-1, 1:-1] = rng.standard_normal((N, N, N))
    rho = np.zeros((N, N, N))
    mu = np.cos(np.pi / (N + 1))
    lam = ((omega * mu + np.sqrt(omega ** 2 * mu ** 2 - 4 * (omega - 1))) / 2) ** 2
    k1, k2 = 150, 350
    _, _, r1 = oracle.sor_group(phi, rho, 1.0, omega, k1, 0.0)
    _, _, r2 = oracle.sor_group(phi, rho, 1.0, omega, k2, 0.0)
    rate = (r2 / r1) ** (1.0 / (k2 - k1))
    assert abs(rate - lam) < 1e-6, (rate, lam)
