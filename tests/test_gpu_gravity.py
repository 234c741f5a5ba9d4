"""The gravity operator G on the GPU (gamer_gravity_update) and the
xyzGGzyx coupling of Sec. 2.3 (reading R25) against the oracle:

* FP64: bit for bit on a random state and potential, for a group count
  that is not a multiple of anything (37 groups);
* FP32: within 1e-6 of the FP64 oracle, relative to each field's scale,
  from the same single-precision inputs (a handful of roundings per cell);
* xyzGGzyx through the C ABI (hydro set, G of twice the step, hydro set):
  FP64 bit for bit against the oracle's sequence on a lognormal state in a
  smooth periodic potential; FP32 within 1e-4;
* free fall: a uniform gas in a linear potential keeps its density and
  pressure and gains exactly -grad(phi) t of velocity, in both precisions
  (every difference is a power of two).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_0907_3390_gb300 import binding as B  # noqa: E402
from paper_0907_3390_gb300 import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0
PREC = {"f32": (B.GAMER_FP32, torch.float32, np.float32), "f64": (B.GAMER_FP64, torch.float64, np.float64)}


def random_level(n, seed):
    rng = np.random.default_rng(seed)
    s = (8 * n, 8, 8, 8)
    rho = np.exp(0.5 * rng.standard_normal(s))
    v = 0.5 * rng.standard_normal((3,) + s)
    P = 1.0 + 0.1 * rng.random(s)
    u = W.prim_to_cons(rho, v[0], v[1], v[2], P, G)
    phi = rng.standard_normal((n, 18, 18, 18))
    return u, phi


def test_gravity_fp64_bitwise():
    u, phi = random_level(37, 1)
    du = torch.tensor(u, device="cuda")
    B.gamer_gravity_update(B.GAMER_FP64, du, torch.tensor(phi, device="cuda"), 1.0 / 48, 0.0031)
    want = oracle.gravity_level(u, phi, 1.0 / 48, 0.0031)
    assert np.array_equal(du.cpu().numpy(), want)


def test_gravity_fp32_tolerance():
    u, phi = random_level(37, 2)
    u32, phi32 = u.astype(np.float32), phi.astype(np.float32)
    du = torch.tensor(u32, device="cuda")
    B.gamer_gravity_update(B.GAMER_FP32, du, torch.tensor(phi32, device="cuda"), 1.0 / 48, 0.0031)
    want = oracle.gravity_level(u32.astype(np.float64), phi32.astype(np.float64), 1.0 / 48, 0.0031)
    got = du.cpu().numpy().astype(np.float64)
    assert np.array_equal(got[0], want[0])
    for v in range(1, 5):
        err = np.abs(got[v] - want[v]).max() / np.abs(want[v]).max()
        assert err <= 1e-6, (v, err)


def test_gravity_zero_groups_is_a_no_op():
    u = torch.zeros((5, 0, 8, 8, 8), device="cuda")
    phi = torch.zeros((0, 18, 18, 18), device="cuda")
    B.gamer_gravity_update(B.GAMER_FP32, u, phi, 0.1, 0.01)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_xyzGGzyx_matches_oracle(prec):
    p, tdt, npdt = PREC[prec]
    u, npg = W.lognormal_cells(32, seed=31, sigma=0.5)
    H, st = W.single_level(u, npg)
    st = [np.asarray(s).astype(npdt).astype(np.float64) for s in st]
    rng = np.random.default_rng(33)
    field = W.smoothed(rng.standard_normal((32, 32, 32)), 3.0)
    field = 0.05 * field / np.abs(field).max()
    phi = W.periodic_potential_blocks(field, npg).astype(npdt).astype(np.float64)
    dh = H.levels[0].dh
    O = oracle.OracleLevels(H, st)
    dt = 0.5 * O.cfl_dt(G, 0.5)
    S = B.Solver(G, B.GAMER_LIMITER_VANLEER, p)
    D = B.DeviceHierarchy(H, st, tdt)
    dphi = torch.tensor(phi, device="cuda", dtype=tdt)
    for _ in range(2):
        O.step(G, dt, 0)
        O.gravity(0, phi, 2 * dt)
        O.step(G, dt, 1)
        S.step(D, dt)                                            # xyz
        B.gamer_gravity_update(p, D.u[0], dphi, dh, 2 * dt)      # GG
        S.step(D, dt)                                            # zyx
    torch.cuda.synchronize()
    got = D.u[0].double().cpu().numpy()
    want = O.u[0]
    if prec == "f64":
        assert np.array_equal(got, want)
    else:
        scale = np.abs(want).reshape(5, -1).max(1)[:, None]
        err = (np.abs(got - want).reshape(5, -1) / scale).max()
        assert err <= 1e-4, err
    S.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("axis", [0, 2])
def test_free_fall(prec, axis):
    p, tdt, npdt = PREC[prec]
    u, npg = W.uniform_flow(32, rho=1.0, v=(0.0, 0.0, 0.0), P=1.0)
    H, st = W.single_level(u, npg)
    dh, a, dt, steps = H.levels[0].dh, 0.5, 2.0 ** -8, 6
    phi = torch.tensor(W.potential_blocks(lambda x, y, z: a * (x, y, z)[axis], npg, dh), device="cuda", dtype=tdt)
    S = B.Solver(G, B.GAMER_LIMITER_VANLEER, p)
    D = B.DeviceHierarchy(H, st, tdt)
    for _ in range(steps):
        S.step(D, dt)
        B.gamer_gravity_update(p, D.u[0], phi, dh, 2 * dt)
        S.step(D, dt)
    out = D.u[0].double().cpu().numpy()
    t = 2 * dt * steps
    assert np.all(out[0] == 1.0)
    for k in range(3):
        assert np.all(out[1 + k] == (-a * t if k == axis else 0.0)), k
    thermal = out[4] - 0.5 * (out[1] ** 2 + out[2] ** 2 + out[3] ** 2) / out[0]
    assert np.allclose(thermal, 1.0 / (G - 1.0), rtol=1e-6 if prec == "f32" else 1e-14, atol=0)
    S.close()
