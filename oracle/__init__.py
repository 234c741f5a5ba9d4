"""Plain FP64 CPU oracle of the relaxing-TVD patch-group hydro path and of
the pieces around it: individual time steps, the refinement-map rebuild,
the red-black SOR Poisson solver and the gravity operator of the xyzGGzyx
splitting.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package; the product
path never does.  It shares no code with the CUDA library.

The arithmetic lives in ``hydro_oracle.c`` (compiled here with gcc,
``-O2 -ffp-contract=off -fopenmp``); this module only marshals numpy arrays
through ctypes and composes the per-level calls into one step of the level
evolution of Sec. 2.1 (update every level, then correct the coarser levels
from the finer ones, finest first).

Parity status: every function is pinned by tests under ``tests/`` against
closed forms, invariants, brute force or the exact Riemann solution, except
the FP32-path comparison tolerances, which are measured, not pinned.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hydro_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libhydro_oracle.so")
_lock = threading.Lock()
_lib = None

VANLEER, MINMOD = 0, 1


class _Level(C.Structure):
    _fields_ = [("n_groups", C.c_int32), ("pad_", C.c_int32), ("dh", C.c_double),
                ("u", C.c_void_p), ("u_out", C.c_void_p), ("nbr", C.c_void_p),
                ("parent", C.c_void_p), ("child", C.c_void_p), ("face_flux", C.c_void_p),
                ("u_new", C.c_void_p), ("coarse_w", C.c_double), ("face_flux2", C.c_void_p)]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int32)
            L.orc_phi_vanleer.restype = C.c_double
            L.orc_phi_vanleer.argtypes = [C.c_double, C.c_double]
            L.orc_phi_minmod.restype = C.c_double
            L.orc_phi_minmod.argtypes = [C.c_double, C.c_double]
            L.orc_pressure.restype = C.c_double
            L.orc_pressure.argtypes = [dp, C.c_double]
            L.orc_tvd_column.argtypes = [dp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, dp]
            L.orc_domain_sweepset.argtypes = [dp, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int),
                                              C.c_double, C.c_int, C.c_double, C.c_double, C.c_int]
            L.orc_minmod_children.argtypes = [dp, dp]
            L.orc_level_advance.argtypes = [C.POINTER(_Level), C.c_int, C.c_int, C.c_double, C.c_int,
                                            C.c_double, C.c_int, ip, C.c_int]
            L.orc_level_fixup.argtypes = [C.POINTER(_Level), C.c_int, C.c_int, C.c_double]
            L.orc_level_max_speed.restype = C.c_double
            L.orc_level_max_speed.argtypes = [C.POINTER(_Level), C.c_double]
            L.orc_cfl_dt.restype = C.c_double
            L.orc_cfl_dt.argtypes = [C.POINTER(_Level), C.c_int, C.c_double, C.c_double]
            L.orc_flag_level.argtypes = [C.POINTER(_Level), C.c_int, C.c_int, C.c_double, C.c_int, C.c_double,
                                         C.c_int, C.c_double, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                         C.POINTER(C.c_int64)]
            L.orc_flag_criterion.argtypes = [C.POINTER(_Level), C.c_int, C.c_int, C.c_double, C.c_int,
                                             C.c_double, dp, dp]
            L.orc_refine_fill.argtypes = [C.POINTER(_Level), C.c_int, C.c_int, C.POINTER(C.c_int32),
                                          C.POINTER(C.c_int32), dp, C.c_int, dp]
            L.orc_gravity_level.argtypes = [dp, C.c_int, dp, C.c_double, C.c_double]
            L.orc_poisson_prepare.argtypes = [C.POINTER(_Level), C.c_int, C.c_int, dp, dp, dp]
            L.orc_sor_group.restype = C.c_int
            L.orc_sor_group.argtypes = [dp, dp, C.c_double, C.c_double, C.c_int, C.c_double, dp]
            L.orc_cfl_dt_steps.restype = C.c_double
            L.orc_cfl_dt_steps.argtypes = [C.POINTER(_Level), C.c_int, C.c_double, C.c_double, C.c_int]
            L.orc_gather_block.argtypes = [C.POINTER(_Level), C.c_int, C.c_int, C.c_int, dp]
            L.orc_check.argtypes = [C.POINTER(_Level), C.c_int, C.c_double, dp, C.POINTER(C.c_int64)]
            _lib = L
    return _lib


def set_threads(n: int) -> None:
    """OpenMP thread count of the oracle's parallel loops."""
    C.CDLL(None)
    try:
        gomp = C.CDLL("libgomp.so.1")
        gomp.omp_set_num_threads(C.c_int(int(n)))
    except OSError:
        pass


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ----------------------------------------------------------- point functions

def phi_vanleer(a: float, b: float) -> float:
    return lib().orc_phi_vanleer(a, b)


def phi_minmod(a: float, b: float) -> float:
    return lib().orc_phi_minmod(a, b)


def pressure(u, gamma: float) -> float:
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().orc_pressure(_dp(u), gamma)


def tvd_column(q: np.ndarray, d: int, lam: float, gamma: float, limiter: int = VANLEER) -> np.ndarray:
    """One 1-D relaxing-TVD step of column q[L][5]; cells 3..L-4 updated."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    out = np.empty_like(q)
    r = lib().orc_tvd_column(_dp(q), q.shape[0], d, lam, gamma, limiter, _dp(out))
    if r != 0:
        raise ValueError(f"orc_tvd_column: {r}")
    return out


def sor_group(phi: np.ndarray, rho: np.ndarray, coef: float, omega: float, max_iter: int, tol: float):
    """Red-black SOR of one patch group (orc_sor_group): returns (phi [18]^3
    after the iterations, iterations done, last residual one-norm)."""
    ph = np.array(phi, dtype=np.float64, order="C", copy=True).reshape(18, 18, 18)
    rh = np.ascontiguousarray(rho, dtype=np.float64).reshape(16, 16, 16)
    res = C.c_double(0.0)
    it = lib().orc_sor_group(_dp(ph), _dp(rh), coef, omega, max_iter, tol, C.byref(res))
    return ph, int(it), float(res.value)


def gravity_level(u: np.ndarray, phi: np.ndarray, dh: float, dt: float) -> np.ndarray:
    """The gravity operator G over dt (orc_gravity_level) on one level's
    state u [5][8 n][8][8][8] with the groups' potentials phi [n][18][18][18];
    returns the new state."""
    out = np.array(u, dtype=np.float64, order="C", copy=True)
    n = out.shape[1] // 8
    ph = np.ascontiguousarray(phi, dtype=np.float64).reshape(n, 18, 18, 18)
    lib().orc_gravity_level(_dp(out), n, _dp(ph), dh, dt)
    return out


def minmod_children(block: np.ndarray) -> np.ndarray:
    """Children [5][2][2][2] of the centre of a coarse block [5][3][3][3]."""
    b = np.ascontiguousarray(block, dtype=np.float64)
    out = np.empty((5, 2, 2, 2))
    lib().orc_minmod_children(_dp(b), _dp(out))
    return out


# ------------------------------------------------------------- whole domain

BC = {"periodic": 0, "outflow": 1}


def domain_sweepset(u: np.ndarray, gamma: float, dt: float, dh: float, order: int,
                    limiter: int = VANLEER, bc=("periodic",) * 3) -> np.ndarray:
    """One sweep set (xyz if order == 0 else zyx) of a whole single-level
    domain u[5][nz][ny][nx]; returns the new state."""
    out = np.array(u, dtype=np.float64, order="C", copy=True)
    nz, ny, nx = out.shape[1:]
    b = (C.c_int * 3)(*[BC[x] for x in bc])
    r = lib().orc_domain_sweepset(_dp(out), nx, ny, nz, b, gamma, limiter, dt, dh, order)
    if r != 0:
        raise ValueError(f"orc_domain_sweepset: {r}")
    return out


# ------------------------------------------------------------ hierarchy form

class OracleLevels:
    """Host copies of a hierarchy's maps and per-level FP64 states."""

    def __init__(self, H, states, with_flux: bool | None = None):
        self.H = H
        self.n = H.n_levels
        if with_flux is None:
            with_flux = self.n > 1
        # private copies: step() ping-pongs between u and u_out and must not
        # write into the caller's arrays
        self.u = [np.array(s, dtype=np.float64, order="C", copy=True) for s in states]
        self.u_out = [np.empty_like(s) for s in self.u]
        self.nbr = [np.ascontiguousarray(lv.nbr, dtype=np.int32) for lv in H.levels]
        self.parent = [None if lv.parent is None else np.ascontiguousarray(lv.parent, dtype=np.int32)
                       for lv in H.levels]
        self.child = [None if lv.child is None else np.ascontiguousarray(lv.child, dtype=np.int32)
                      for lv in H.levels]
        self.flux = [np.zeros((lv.n_groups, 3, 3, 5, 16, 16)) if with_flux else None for lv in H.levels]
        # individual time steps: per level the face fluxes of its two steps
        # within a coarser step, the weight of its coarse ghosts' time
        # interpolation, and which of the two flux arrays its sweeps write
        self.flux2 = None
        self._cw = [0.0] * self.n
        self._slot = [0] * self.n
        self._arr = (_Level * max(self.n, 1))()
        self._refresh()

    def _refresh(self):
        for l, lv in enumerate(self.H.levels):
            s = self._arr[l]
            s.n_groups = lv.n_groups
            s.dh = lv.dh
            s.u = self.u[l].ctypes.data
            s.u_out = self.u_out[l].ctypes.data
            s.nbr = self.nbr[l].ctypes.data
            s.parent = None if self.parent[l] is None else self.parent[l].ctypes.data
            s.child = None if self.child[l] is None else self.child[l].ctypes.data
            s.face_flux = None if self.flux[l] is None else self.flux[l].ctypes.data
            s.u_new = None
            s.coarse_w = 0.0
            s.face_flux2 = None
            if self.flux2 is not None:
                s.face_flux = self.flux2[l][self._slot[l]].ctypes.data
                s.u_new = self.u_out[l].ctypes.data
                s.coarse_w = self._cw[l]

    def advance_level(self, l: int, gamma: float, dt: float, order: int, limiter: int = VANLEER,
                      groups=None) -> None:
        """Sweep set of level l (all groups, or the listed ones) into u_out."""
        self._refresh()
        if groups is None:
            lst, n = None, 0
        else:
            arr = np.ascontiguousarray(groups, dtype=np.int32)
            lst, n = arr.ctypes.data_as(C.POINTER(C.c_int32)), len(arr)
        r = lib().orc_level_advance(self._arr, self.n, l, gamma, limiter, dt, order, lst, n)
        if r != 0:
            raise ValueError(f"orc_level_advance: {r}")

    def gather_block(self, l: int, g: int) -> np.ndarray:
        """Padded block [5][22][22][22] of group g of level l (pre-step state)."""
        self._refresh()
        out = np.empty((5, 22, 22, 22))
        r = lib().orc_gather_block(self._arr, self.n, l, g, _dp(out))
        if r != 0:
            raise ValueError(f"orc_gather_block: {r}")
        return out

    def poisson_prepare(self, l: int, phi_c: np.ndarray):
        """SOR inputs of level l >= 1 (orc_poisson_prepare): (phi blocks
        [n][18][18][18] interpolated from the coarser level's potential phi_c
        [8 n_c][8][8][8], density blocks [n][16][16][16])."""
        self._refresh()
        n = self.H.levels[l].n_groups
        pc = np.ascontiguousarray(phi_c, dtype=np.float64)
        phi = np.empty((n, 18, 18, 18))
        rho = np.empty((n, 16, 16, 16))
        r = lib().orc_poisson_prepare(self._arr, self.n, l, _dp(pc), _dp(phi), _dp(rho))
        if r != 0:
            raise ValueError(f"orc_poisson_prepare: {r}")
        return phi, rho

    def gravity(self, l: int, phi: np.ndarray, dt: float) -> None:
        """The gravity operator G over dt on level l's state, in place
        (orc_gravity_level; phi [n_groups][18][18][18])."""
        self.u[l][...] = gravity_level(self.u[l], phi, self.H.levels[l].dh, dt)

    def fixup_level(self, l: int, dt: float) -> None:
        self._refresh()
        r = lib().orc_level_fixup(self._arr, self.n, l, dt)
        if r != 0:
            raise ValueError(f"orc_level_fixup: {r}")

    def step(self, gamma: float, dt: float, order: int, limiter: int = VANLEER) -> None:
        """One step of the level evolution with a uniform dt (reading R9):
        every level advanced from the pre-step state, then levels n-2..0
        corrected by restriction and flux correction; then u <- u_out."""
        for l in range(self.n):
            self.advance_level(l, gamma, dt, order, limiter)
        for l in range(self.n - 2, -1, -1):
            self.fixup_level(l, dt)
        self.u, self.u_out = self.u_out, self.u
        self._refresh()

    def cfl_dt(self, gamma: float, cfl: float, individual: bool = False) -> float:
        """Eq. CFL; with individual time steps the dt of level 0."""
        self._refresh()
        return lib().orc_cfl_dt_steps(self._arr, self.n, gamma, cfl, 1 if individual else 0)

    def cycle_individual(self, gamma: float, dt0: float, limiter: int = VANLEER) -> None:
        """Individual time steps (Sec. 2.1, readings R18-R20): two steps of
        level 0 with dt0 (an xyz and a zyx set with one dt, reading R1), so
        2^(l+1) steps of level l with dt0 / 2^l.  A step of level l is its
        sweep set from u into u_out (sweep order alternating per level; its
        coarse ghosts interpolated in time between the coarser level's state
        before and after that level's sweep set, weight 0 in the first and
        1/2 in the second of its two steps), then the two steps of the finer
        level, then the fix-up of level l from the finer level (restriction
        of the finer state; flux correction with this step's fluxes and the
        finer fluxes averaged over its two steps), then u <- u_out.  Every
        level ends in u."""
        if self.flux2 is None:
            self.flux2 = [[np.zeros((lv.n_groups, 3, 3, 5, 16, 16)) for _ in range(2)] for lv in self.H.levels]
        self._level_steps(0, gamma, dt0, limiter)

    def _level_steps(self, l: int, gamma: float, dt: float, limiter: int) -> None:
        for k in range(2):
            self._cw[l] = 0.5 * k if l > 0 else 0.0
            self._slot[l] = k
            self._refresh()
            r = lib().orc_level_advance(self._arr, self.n, l, gamma, limiter, dt, k, None, 0)
            if r != 0:
                raise ValueError(f"orc_level_advance: {r}")
            if l + 1 < self.n:
                self._level_steps(l + 1, gamma, 0.5 * dt, limiter)
                # fix-up of level l: this step's fluxes against the finer
                # level's two steps; the finer state is in its u
                self._slot[l] = k
                self._refresh()
                F = self._arr[l + 1]
                F.u_out = self.u[l + 1].ctypes.data
                F.face_flux = self.flux2[l + 1][0].ctypes.data
                F.face_flux2 = self.flux2[l + 1][1].ctypes.data
                r = lib().orc_level_fixup(self._arr, self.n, l, dt)
                if r != 0:
                    raise ValueError(f"orc_level_fixup: {r}")
            self.u[l], self.u_out[l] = self.u_out[l], self.u[l]
        self._cw[l] = 0.0
        self._slot[l] = 0
        self._refresh()

    def max_speed(self, l: int, gamma: float) -> float:
        self._refresh()
        return lib().orc_level_max_speed(C.byref(self._arr[l]), gamma)

    def flag_level(self, l: int, gamma: float, criterion: int, threshold: float, n_buffer: int) -> np.ndarray:
        """Per-patch flag-buffer masks of level l (orc_flag_level), the
        criterion decided in double precision."""
        return self.flag_level_bounds(l, gamma, criterion, threshold, n_buffer, 0.0)[0]

    def flag_level_bounds(self, l: int, gamma: float, criterion: int, threshold: float, n_buffer: int,
                          u_eval: float):
        """(masks of the cells flagged whatever the rounding, masks of the
        cells that may be flagged, number of cells that may go either way)
        when the criterion is evaluated in a format of unit roundoff u_eval
        (orc_flag_level); u_eval = 0 gives the double decision twice."""
        self._refresh()
        n = 8 * self.H.levels[l].n_groups
        sure = np.zeros(n, dtype=np.uint32)
        maybe = np.zeros(n, dtype=np.uint32)
        near = C.c_int64(0)
        r = lib().orc_flag_level(self._arr, self.n, l, gamma, criterion, threshold, n_buffer, float(u_eval),
                                 sure.ctypes.data_as(C.POINTER(C.c_uint32)),
                                 maybe.ctypes.data_as(C.POINTER(C.c_uint32)), C.byref(near))
        if r != 0:
            raise ValueError(f"orc_flag_level: {r}")
        return sure, maybe, int(near.value)

    def flag_criterion(self, l: int, gamma: float, criterion: int, u_eval: float = 0.0):
        """Per cell of level l ([8 n_groups][8][8][8]) the criterion value in
        double precision and the bound on its error when evaluated at unit
        roundoff u_eval (orc_flag_criterion)."""
        self._refresh()
        n = 8 * self.H.levels[l].n_groups
        val = np.empty((n, 8, 8, 8))
        bound = np.empty((n, 8, 8, 8))
        r = lib().orc_flag_criterion(self._arr, self.n, l, gamma, criterion, float(u_eval), _dp(val), _dp(bound))
        if r != 0:
            raise ValueError(f"orc_flag_criterion: {r}")
        return val, bound

    def refine_fill(self, l: int, parent_new, inherit, u_old) -> np.ndarray:
        """Data of a rebuilt level l+1 (orc_refine_fill) from this level's u."""
        self._refresh()
        pn = np.ascontiguousarray(parent_new, dtype=np.int32)
        ih = np.ascontiguousarray(inherit, dtype=np.int32)
        n_new = len(pn)
        uo = np.ascontiguousarray(u_old if u_old is not None else np.zeros((5, 8, 512)), dtype=np.float64)
        n_old = uo.shape[1] // 8
        out = np.empty((5, 8 * n_new, 8, 8, 8))
        r = lib().orc_refine_fill(self._arr, l, n_new, pn.ctypes.data_as(C.POINTER(C.c_int32)),
                                  ih.ctypes.data_as(C.POINTER(C.c_int32)), _dp(uo), n_old, _dp(out))
        if r != 0:
            raise ValueError(f"orc_refine_fill: {r}")
        return out

    def check(self, gamma: float):
        self._refresh()
        sums = np.zeros(5)
        nb = C.c_int64(0)
        lib().orc_check(self._arr, self.n, gamma, _dp(sums), C.byref(nb))
        return sums, int(nb.value)


def run(O: OracleLevels, gamma: float, cfl: float, n_calls: int, limiter: int = VANLEER,
        order0: int = 0):
    """n_calls sweep sets alternating xyz / zyx (reading R1); dt from Eq. CFL
    before every xyz call and held for the following zyx call.  Returns the
    list of dt used."""
    dts = []
    dt = None
    for c in range(n_calls):
        order = (order0 + c) % 2
        if order == 0 or dt is None:
            dt = O.cfl_dt(gamma, cfl)
        O.step(gamma, dt, order, limiter)
        dts.append(dt)
    return dts
