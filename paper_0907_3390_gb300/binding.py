"""Thin Python binding of ``libgamer_hydro.so`` (declared in
``include/gamer_hydro.h``).

The functions below carry the C names and only marshal arguments; every
step of the computation runs in the library's CUDA kernels.  PyTorch is
used for device memory and streams only.  Loading fails loudly (raises)
when the library is missing or cannot be built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

GAMER_OK, GAMER_ERR_ARG, GAMER_ERR_CUDA, GAMER_ERR_MAP = 0, -1, -2, -3
GAMER_ERR_TIMEOUT, GAMER_ERR_UNSUPPORTED, GAMER_ERR_STATE = -4, -5, -6
GAMER_TIME_STEPS_UNIFORM, GAMER_TIME_STEPS_INDIVIDUAL = 0, 1
GAMER_FLAG_DENSITY_GRADIENT, GAMER_FLAG_PRESSURE_GRADIENT, GAMER_FLAG_DENSITY = 0, 1, 2
GAMER_LIMITER_VANLEER, GAMER_LIMITER_MINMOD = 0, 1
GAMER_FP32, GAMER_FP64 = 0, 1

EXPORTS = [
    "gamer_hydro_create", "gamer_hydro_destroy", "gamer_hydro_set_stream",
    "gamer_hydro_set_parity", "gamer_hydro_get_parity", "gamer_hydro_cfl_dt",
    "gamer_hydro_advance", "gamer_hydro_fixup", "gamer_hydro_advance_all",
    "gamer_hydro_check", "gamer_hydro_diagnose", "gamer_hydro_step", "gamer_hydro_step_pair",
    "gamer_hydro_set_time_steps", "gamer_hydro_set_launch_groups", "gamer_hydro_flag", "gamer_hydro_refine_fill", "gamer_poisson_sor",
    "gamer_gravity_update", "gamer_hydro_test_withhold", "gamer_poisson_prepare",
    "gamer_hydro_step_result",
    "gamer_hydro_diagnose_noalloc", "gamer_hydro_tune", "gamer_hydro_get_config",
    "gamer_hydro_set_profiling", "gamer_hydro_last_error",
]


class gamer_level_t(C.Structure):
    _fields_ = [("n_groups", C.c_int32), ("reserved", C.c_int32), ("dh", C.c_double),
                ("u", C.c_void_p), ("u_out", C.c_void_p), ("nbr", C.c_void_p),
                ("parent", C.c_void_p), ("child", C.c_void_p), ("face_flux", C.c_void_p)]


class gamer_hierarchy_t(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("reserved", C.c_int32),
                ("levels", C.POINTER(gamer_level_t)), ("version", C.c_uint64)]


class GamerError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_needed: bool = True) -> C.CDLL:
    """Load the CUDA library (building it first when sources are newer)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_needed else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libgamer_hydro.so not found at {path}; run __graft_entry__.build()")
        L = C.CDLL(path)
        H, vp, dp, ip = C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
        hp = C.POINTER(gamer_hierarchy_t)
        L.gamer_hydro_create.argtypes = [C.c_double, C.c_int, C.c_int, C.c_int, C.POINTER(H)]
        L.gamer_hydro_destroy.argtypes = [H]
        L.gamer_hydro_set_stream.argtypes = [H, vp]
        L.gamer_hydro_set_parity.argtypes = [H, C.c_int, C.c_int]
        L.gamer_hydro_get_parity.argtypes = [H, C.c_int, ip]
        L.gamer_hydro_cfl_dt.argtypes = [H, hp, C.c_double, dp]
        L.gamer_hydro_advance.argtypes = [H, hp, C.c_int, C.c_double]
        L.gamer_hydro_fixup.argtypes = [H, hp, C.c_int, C.c_double]
        L.gamer_hydro_advance_all.argtypes = [H, hp, C.c_double]
        L.gamer_hydro_check.argtypes = [H, hp, dp, C.POINTER(C.c_int64)]
        L.gamer_hydro_diagnose.argtypes = [H, hp, C.c_double, dp, dp, C.POINTER(C.c_int64)]
        L.gamer_hydro_step.argtypes = [H, hp, C.c_double]
        L.gamer_hydro_step_pair.argtypes = [H, hp, C.c_double]
        L.gamer_hydro_set_time_steps.argtypes = [H, C.c_int]
        L.gamer_hydro_set_launch_groups.argtypes = [H, C.c_int]
        L.gamer_hydro_flag.argtypes = [H, hp, C.c_int, C.c_int, C.c_double, C.c_int, vp]
        L.gamer_hydro_refine_fill.argtypes = [H, hp, C.c_int, C.c_int, vp, vp, vp, C.c_int, vp]
        L.gamer_poisson_sor.argtypes = [C.c_int, C.c_int, vp, vp, C.c_double, C.c_double, C.c_int, C.c_double,
                                        vp, vp]
        L.gamer_gravity_update.argtypes = [C.c_int, C.c_int, vp, vp, C.c_double, C.c_double, vp]
        L.gamer_hydro_test_withhold.argtypes = [H, C.c_int]
        L.gamer_poisson_prepare.argtypes = [H, hp, C.c_int, vp, vp, vp]
        L.gamer_hydro_step_result.argtypes = [H, dp, dp, dp, C.POINTER(C.c_int64)]
        L.gamer_hydro_diagnose_noalloc.argtypes = [C.c_double, C.c_int, hp, C.c_double, vp, dp, dp,
                                                   C.POINTER(C.c_int64)]
        L.gamer_hydro_tune.argtypes = [H, hp, C.c_char_p]
        L.gamer_hydro_get_config.argtypes = [H, C.c_char_p, C.c_int]
        L.gamer_hydro_set_profiling.argtypes = [H, vp, vp]
        L.gamer_hydro_last_error.argtypes = [H]
        L.gamer_hydro_last_error.restype = C.c_char_p
        for name in EXPORTS:
            if name != "gamer_hydro_last_error":
                getattr(L, name).restype = C.c_int
        _lib = L
        return L


def _check(h, code):
    if code != GAMER_OK:
        msg = load().gamer_hydro_last_error(h).decode()
        raise GamerError(code, msg)


# ------------------------------------------------ C functions, same names

def gamer_hydro_create(gamma: float, limiter: int = GAMER_LIMITER_VANLEER, ghost_width: int = 3,
                       precision: int = GAMER_FP32):
    h = C.c_void_p()
    _check(None, load().gamer_hydro_create(gamma, limiter, ghost_width, precision, C.byref(h)))
    return h


def gamer_hydro_destroy(h) -> None:
    load().gamer_hydro_destroy(h)


def gamer_hydro_set_stream(h, stream) -> None:
    """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
    raw = None if stream is None else getattr(stream, "cuda_stream", stream)
    _check(h, load().gamer_hydro_set_stream(h, C.c_void_p(raw) if raw else None))


def gamer_hydro_set_parity(h, level: int, parity: int) -> None:
    _check(h, load().gamer_hydro_set_parity(h, level, parity))


def gamer_hydro_get_parity(h, level: int) -> int:
    p = C.c_int()
    _check(h, load().gamer_hydro_get_parity(h, level, C.byref(p)))
    return p.value


def gamer_hydro_cfl_dt(h, H, cfl: float) -> float:
    dt = C.c_double()
    _check(h, load().gamer_hydro_cfl_dt(h, H.struct(), cfl, C.byref(dt)))
    return dt.value


def gamer_hydro_advance(h, H, level: int, dt: float) -> None:
    _check(h, load().gamer_hydro_advance(h, H.struct(), level, dt))


def gamer_hydro_fixup(h, H, level: int, dt: float) -> None:
    _check(h, load().gamer_hydro_fixup(h, H.struct(), level, dt))


def gamer_hydro_advance_all(h, H, dt: float) -> None:
    _check(h, load().gamer_hydro_advance_all(h, H.struct(), dt))


def gamer_hydro_check(h, H):
    sums = (C.c_double * 5)()
    nb = C.c_int64()
    _check(h, load().gamer_hydro_check(h, H.struct(), sums, C.byref(nb)))
    return np.array(sums[:]), int(nb.value)


def gamer_hydro_diagnose(h, H, cfl: float):
    dt = C.c_double()
    sums = (C.c_double * 5)()
    nb = C.c_int64()
    _check(h, load().gamer_hydro_diagnose(h, H.struct(), cfl, C.byref(dt), sums, C.byref(nb)))
    return dt.value, np.array(sums[:]), int(nb.value)


def gamer_hydro_step(h, H, cfl: float) -> None:
    _check(h, load().gamer_hydro_step(h, H.struct(), cfl))


def gamer_hydro_set_time_steps(h, mode: int) -> None:
    _check(h, load().gamer_hydro_set_time_steps(h, mode))


def gamer_hydro_set_launch_groups(h, n: int) -> None:
    _check(h, load().gamer_hydro_set_launch_groups(h, int(n)))


def gamer_hydro_flag(h, H, level: int, criterion: int, threshold: float, n_buffer: int, masks) -> None:
    """masks: device uint32 tensor [8 n_groups] of the level (written)."""
    _check(h, load().gamer_hydro_flag(h, H.struct(), level, criterion, threshold, n_buffer, masks.data_ptr()))


def gamer_hydro_refine_fill(h, H, level: int, parent_new, inherit, u_old, u_new) -> None:
    """parent_new, inherit: device int32 tensors [n_new]; u_old: device state
    of the previous level l+1 or None; u_new: device state [5, 8 n_new, 8, 8, 8]."""
    n_new = int(parent_new.numel())
    n_old = 0 if u_old is None else int(u_old.shape[1]) // 8
    _check(h, load().gamer_hydro_refine_fill(h, H.struct(), level, n_new, parent_new.data_ptr(), inherit.data_ptr(),
                                              None if u_old is None else u_old.data_ptr(), n_old, u_new.data_ptr()))


def gamer_poisson_sor(precision: int, rho, phi, coef: float, omega: float, max_iter: int, tol: float,
                      iters=None, stream=None) -> None:
    """rho: device tensor [n, 16, 16, 16]; phi: device tensor [n, 18, 18, 18]
    (updated in place); iters: device int32 tensor [n] or None."""
    n = int(rho.shape[0])
    st = None if stream is None else getattr(stream, "cuda_stream", stream)
    _check(None, load().gamer_poisson_sor(precision, n, rho.data_ptr(), phi.data_ptr(), coef, omega, max_iter, tol,
                                          None if iters is None else iters.data_ptr(), st))


def gamer_poisson_prepare(h, H, level: int, phi_c, phi_blocks, rho_blocks) -> None:
    """phi_c: device tensor [8 n_c, 8, 8, 8] (level-1 potential); phi_blocks
    [n, 18, 18, 18] and rho_blocks [n, 16, 16, 16] are filled."""
    _check(h, load().gamer_poisson_prepare(h, H.struct(), level, phi_c.data_ptr(), phi_blocks.data_ptr(),
                                           rho_blocks.data_ptr()))


def gamer_hydro_test_withhold(h, group: int) -> None:
    """The next fused pair launch withholds group `group`'s xyz mark (-1: none)."""
    _check(h, load().gamer_hydro_test_withhold(h, group))


def gamer_gravity_update(precision: int, u, phi, dh: float, dt: float, stream=None) -> None:
    """u: one level's device state [5, 8 n, 8, 8, 8] (updated in place);
    phi: device tensor [n, 18, 18, 18] of the same dtype."""
    n = int(phi.shape[0])
    if int(u.shape[1]) != 8 * n:
        raise ValueError("u holds 8 patches per potential block")
    st = None if stream is None else getattr(stream, "cuda_stream", stream)
    _check(None, load().gamer_gravity_update(precision, n, u.data_ptr(), phi.data_ptr(), dh, dt, st))


def gamer_hydro_step_pair(h, H, cfl: float) -> None:
    """xyz + zyx sweep sets with one dt; the result is back in H.u (no swap)."""
    _check(h, load().gamer_hydro_step_pair(h, H.struct(), cfl))


def gamer_hydro_step_result(h):
    """(dt_used, dt_next, sums[5], n_bad) of the last gamer_hydro_step."""
    du, dn = C.c_double(), C.c_double()
    sums = (C.c_double * 5)()
    nb = C.c_int64()
    _check(h, load().gamer_hydro_step_result(h, C.byref(du), C.byref(dn), sums, C.byref(nb)))
    return du.value, dn.value, np.array(sums[:]), int(nb.value)


def gamer_hydro_diagnose_noalloc(gamma: float, precision: int, H, cfl: float, stream=None):
    """(dt, sums[5], n_bad) without a handle or any device allocation."""
    raw = None if stream is None else getattr(stream, "cuda_stream", stream)
    dt = C.c_double()
    sums = (C.c_double * 5)()
    nb = C.c_int64()
    _check(None, load().gamer_hydro_diagnose_noalloc(gamma, precision, H.struct(), cfl,
                                                     C.c_void_p(raw) if raw else None, C.byref(dt), sums,
                                                     C.byref(nb)))
    return dt.value, np.array(sums[:]), int(nb.value)


def gamer_hydro_tune(h, H, cache_path=None) -> None:
    _check(h, load().gamer_hydro_tune(h, H.struct(), None if cache_path is None else str(cache_path).encode()))


def gamer_hydro_get_config(h) -> str:
    buf = C.create_string_buffer(256)
    _check(h, load().gamer_hydro_get_config(h, buf, 256))
    return buf.value.decode()


def gamer_hydro_set_profiling(h, ev_before, ev_after) -> None:
    """ev_*: torch.cuda.Event(enable_timing=True) or raw cudaEvent_t, or None."""
    raw = [None if e is None else getattr(e, "cuda_event", e) for e in (ev_before, ev_after)]
    _check(h, load().gamer_hydro_set_profiling(h, *[C.c_void_p(r) if r else None for r in raw]))


def gamer_hydro_last_error(h) -> str:
    return load().gamer_hydro_last_error(h).decode()


# ------------------------------------------------ device-side hierarchy

_version_counter = [0]


class DeviceHierarchy:
    """A hierarchy snapshot on the device: maps as int32 tensors, per-level
    state tensors u / u_out ([5, 8n, 8, 8, 8], float32 or float64), and the
    C structs that point at them.  ``swap()`` exchanges u and u_out.  The
    output buffers (u_out and the face fluxes) start filled with NaN, so a
    cell that a call fails to write never holds a plausible value;
    ``poison()`` refills them."""

    def __init__(self, H, states, dtype, device="cuda", with_flux=False):
        import torch
        self.torch = torch
        self.H = H
        self.dtype = dtype
        self.device = torch.device(device)
        n = H.n_levels
        # states: host arrays, or device tensors of this dtype that are used as they are
        self.u = [s if (torch.is_tensor(s) and s.is_cuda and s.dtype == dtype and s.is_contiguous())
                  else torch.as_tensor(np.ascontiguousarray(s), dtype=dtype).to(self.device) for s in states]
        self.u_out = [torch.full_like(x, float("nan")) for x in self.u]
        self.nbr = [torch.as_tensor(np.ascontiguousarray(lv.nbr, dtype=np.int32)).to(self.device)
                    for lv in H.levels]
        self.parent = [None if lv.parent is None else
                       torch.as_tensor(np.ascontiguousarray(lv.parent, dtype=np.int32)).to(self.device)
                       for lv in H.levels]
        self.child = [None if lv.child is None else
                      torch.as_tensor(np.ascontiguousarray(lv.child, dtype=np.int32)).to(self.device)
                      for lv in H.levels]
        self.flux = [torch.full((lv.n_groups, 3, 3, 5, 16, 16), float("nan"), dtype=dtype, device=self.device)
                     if (with_flux and n > 1) else None for lv in H.levels]
        _version_counter[0] += 1
        self.version = _version_counter[0]
        self._levels = (gamer_level_t * n)()
        self._hier = gamer_hierarchy_t()
        self._refresh()

    @staticmethod
    def _ptr(t):
        return None if t is None or t.numel() == 0 else t.data_ptr()

    def _refresh(self):
        for l, lv in enumerate(self.H.levels):
            s = self._levels[l]
            s.n_groups = lv.n_groups
            s.dh = lv.dh
            s.u = self._ptr(self.u[l])
            s.u_out = self._ptr(self.u_out[l])
            s.nbr = self._ptr(self.nbr[l])
            s.parent = self._ptr(self.parent[l]) if l > 0 else None
            s.child = self._ptr(self.child[l]) if l + 1 < self.H.n_levels else None
            s.face_flux = self._ptr(self.flux[l])
        self._hier.n_levels = self.H.n_levels
        self._hier.levels = self._levels
        self._hier.version = self.version

    def struct(self):
        return C.byref(self._hier)

    def swap(self):
        self.u, self.u_out = self.u_out, self.u
        self._refresh()

    def poison(self):
        """Fill the output buffers (u_out, caller-owned face fluxes) with NaN."""
        for t in self.u_out + [f for f in self.flux if f is not None]:
            t.fill_(float("nan"))

    def states(self):
        return [x.detach().double().cpu().numpy() for x in self.u]


class Solver:
    """Convenience wrapper: one handle + the calls of one step."""

    def __init__(self, gamma=5.0 / 3.0, limiter=GAMER_LIMITER_VANLEER, precision=GAMER_FP32, stream=None):
        self.h = gamer_hydro_create(gamma, limiter, 3, precision)
        if stream is not None:
            gamer_hydro_set_stream(self.h, stream)

    def close(self):
        if self.h:
            gamer_hydro_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, D: DeviceHierarchy, dt: float):
        """advance_all + swap."""
        gamer_hydro_advance_all(self.h, D, dt)
        D.swap()

    def run(self, D: DeviceHierarchy, cfl: float, n_calls: int):
        """n_calls sweep sets; dt from Eq. CFL before each xyz call, held for
        the following zyx call.  Returns the dt list."""
        dts, dt = [], None
        for c in range(n_calls):
            if gamer_hydro_get_parity(self.h, 0) == 0 or dt is None:
                dt = gamer_hydro_cfl_dt(self.h, D, cfl)
            self.step(D, dt)
            dts.append(dt)
        return dts
