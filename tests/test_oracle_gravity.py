"""Pins of the oracle's gravity operator G and of the xyzGGzyx coupling
(Sec. 2.3: Eqs. MomConserve and EnergyConserve with the flux terms dropped,
the 3-point central difference for the acceleration, the operator order
xyzGGzyx with GG taken as one G of twice the step; reading R25):

* a constant potential changes nothing, bit for bit;
* a linear potential gives the constant acceleration -grad(phi): the
  momentum change is rho g dt, density and thermal energy are unchanged;
* a quadratic potential: the central difference is exact, so the
  acceleration at every cell centre is the analytic -k (x - x0);
* the thermal energy e - |m|^2 / (2 rho) is invariant for any state and
  potential (G changes the kinetic energy only);
* two G of dt equal one G of 2 dt (the combination the paper uses for GG);
* free fall through xyzGGzyx: a uniform gas in a linear potential keeps
  its density and pressure and its velocity grows as g t.
"""
import numpy as np
import pytest

import oracle
from paper_0907_3390_gb300 import workloads as W
from paper_0907_3390_gb300.hierarchy import domain_to_patches

G = 5.0 / 3.0


def state(n=32, seed=5):
    u, npg = W.lognormal_cells(n, seed=seed, sigma=0.5)
    H, st = W.single_level(u, npg)
    return H, st[0], npg


def thermal(u):
    return u[4] - 0.5 * (u[1] ** 2 + u[2] ** 2 + u[3] ** 2) / u[0]


def test_constant_potential_changes_nothing():
    H, u, npg = state()
    phi = np.full((u.shape[1] // 8, 18, 18, 18), 3.25)
    out = oracle.gravity_level(u, phi, H.levels[0].dh, 0.01)
    assert np.array_equal(out, u)


def test_linear_potential_constant_acceleration():
    H, u, npg = state()
    dh, dt = H.levels[0].dh, 0.004
    a = np.array([0.7, -1.3, 0.45])
    phi = W.potential_blocks(lambda x, y, z: a[0] * x + a[1] * y + a[2] * z, npg, dh)
    out = oracle.gravity_level(u, phi, dh, dt)
    assert np.array_equal(out[0], u[0])
    for k in range(3):
        want = u[1 + k] - u[0] * a[k] * dt
        assert np.allclose(out[1 + k], want, rtol=0, atol=1e-12 * np.abs(u[1 + k]).max())
    assert np.allclose(thermal(out), thermal(u), rtol=1e-11, atol=0)


def test_quadratic_potential_exact_gradient():
    H, u, npg = state()
    dh, dt, k = H.levels[0].dh, 0.003, 2.5
    x0 = np.array([0.41, 0.53, 0.47])
    phi = W.potential_blocks(lambda x, y, z: 0.5 * k * ((x - x0[0]) ** 2 + (y - x0[1]) ** 2 + (z - x0[2]) ** 2),
                             npg, dh)
    out = oracle.gravity_level(u, phi, dh, dt)
    # analytic acceleration at the cell centres, in the patch layout
    n = 32
    c = (np.arange(n) + 0.5) * dh
    zz, yy, xx = np.meshgrid(c, c, c, indexing="ij")
    gdom = np.stack([-k * (xx - x0[0]), -k * (yy - x0[1]), -k * (zz - x0[2])])
    g = domain_to_patches(gdom, npg)
    for a in range(3):
        want = u[1 + a] + u[0] * g[a] * dt
        assert np.allclose(out[1 + a], want, rtol=0, atol=1e-11 * np.abs(u[1 + a]).max())


def test_thermal_energy_invariant():
    H, u, npg = state(seed=9)
    rng = np.random.default_rng(11)
    phi = W.periodic_potential_blocks(rng.standard_normal((32, 32, 32)), npg)
    out = oracle.gravity_level(u, phi, H.levels[0].dh, 0.002)
    assert not np.array_equal(out[1], u[1])
    assert np.array_equal(out[0], u[0])
    assert np.allclose(thermal(out), thermal(u), rtol=1e-10, atol=0)


def test_two_steps_equal_one_double_step():
    H, u, npg = state(seed=13)
    rng = np.random.default_rng(17)
    phi = W.periodic_potential_blocks(rng.standard_normal((32, 32, 32)), npg)
    dh, dt = H.levels[0].dh, 0.0025
    twice = oracle.gravity_level(oracle.gravity_level(u, phi, dh, dt), phi, dh, dt)
    once = oracle.gravity_level(u, phi, dh, 2 * dt)
    for v in range(5):
        assert np.allclose(twice[v], once[v], rtol=0, atol=1e-12 * np.abs(once[v]).max()), v


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_free_fall_through_xyzGGzyx(axis):
    n = 32
    u, npg = W.uniform_flow(n, rho=1.0, v=(0.0, 0.0, 0.0), P=1.0)
    H, st = W.single_level(u, npg)
    dh = H.levels[0].dh              # 2^-5
    a = 0.5                          # powers of two: every difference is exact
    phi = W.potential_blocks(lambda x, y, z: a * (x, y, z)[axis], npg, dh)
    O = oracle.OracleLevels(H, st)
    dt = 2.0 ** -8
    steps = 6
    for _ in range(steps):
        O.step(G, dt, 0)                                   # xyz
        O.gravity(0, phi, 2 * dt)                          # GG
        O.step(G, dt, 1)                                   # zyx
    out = O.u[0]
    t = 2 * dt * steps
    assert np.all(out[0] == 1.0)
    for k in range(3):
        want = -a * t if k == axis else 0.0
        assert np.all(out[1 + k] == want), (k, np.unique(out[1 + k])[:4])
    assert np.allclose(thermal(out), 1.0 / (G - 1.0), rtol=1e-14, atol=0)
