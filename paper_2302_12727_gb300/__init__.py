"""GB300 photon-transport library (FVPM radiative transfer of GEAR-RT, arXiv 2302.12727).

The compute path is the CUDA library ``_lib/librt_gb300.so`` behind the C interface of
``include/rt.h``.  This module is its thin binding: the functions below carry the C names
and only marshal arguments (torch tensors or raw device pointers) before calling the
library.  There is no CPU fallback: if the library is missing, loading fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os

from .build_ext import LIB as _LIB_PATH

RT_FP64 = 0
RT_FP32_MIXED = 1

RT_OK = 0
_STATUS = {0: "RT_OK", 1: "RT_ERR_INVALID", 2: "RT_ERR_CUDA", 3: "RT_ERR_OOM", 4: "RT_ERR_NOCONV",
           5: "RT_ERR_GEOMETRY", 6: "RT_ERR_TIMEOUT", 7: "RT_ERR_STATE"}

EXPORTED = ["rt_create", "rt_set_stream", "rt_neighbours", "rt_neighbours_given_h", "rt_neighbours_given_fields",
            "rt_source_fields", "rt_source_norms",
            "rt_set_owned", "rt_gradients", "rt_transport_step", "rt_inject", "rt_transport_step_given_gradients",
            "rt_set_fields", "rt_subcycle",
            "rt_drift", "rt_set_time_bins", "rt_get_time_bins", "rt_step_bins", "rt_set_absorbers", "rt_cross_section", "rt_blackbody_groups",
            "rt_photon_number_to_luminosity",
            "rt_adjoint", "rt_energy", "rt_particle_fields", "rt_pairs", "rt_diagnostics", "rt_set_profiling",
            "rt_kernel_times", "rt_set_tuning", "rt_get_tuning", "rt_autotune", "rt_wave_table",
            "rt_energy_static", "rt_wait_selftest", "rt_last_error", "rt_destroy"]

RT_ENERGY_STATIC_MAX_GROUPS = 16

RT_KERNEL_INJECT, RT_KERNEL_GRADIENT, RT_KERNEL_FLUX, RT_KERNEL_FLUX_GATHER, RT_KERNEL_KINDS = 0, 1, 2, 3, 4
RT_RIEMANN_GLF, RT_RIEMANN_HLL = 0, 1
RT_WAVE_NF, RT_WAVE_NTH = 101, 101
RT_TUNE_CANDIDATES = 18


class rt_config(C.Structure):
    _fields_ = [("n_groups", C.c_int32), ("c_red", C.c_double), ("eta_res", C.c_double),
                ("eta_res_star", C.c_double), ("box", C.c_double * 3), ("periodic", C.c_int32),
                ("precision", C.c_int32), ("clamp_negative", C.c_int32), ("limiter_variant", C.c_int32),
                ("h_tol", C.c_double), ("h_max_iter", C.c_int32), ("device_wait_budget_cycles", C.c_uint64),
                ("riemann_solver", C.c_int32)]


class rt_diag(C.Structure):
    _fields_ = [("n_pairs", C.c_int64), ("n_directed", C.c_int64), ("n_injection", C.c_int64),
                ("n_ill_conditioned", C.c_int64), ("cond_max", C.c_double), ("h_min", C.c_double),
                ("h_max", C.c_double), ("dx_min", C.c_double), ("clamp_events", C.c_int64),
                ("grid", C.c_int32 * 3), ("threads_per_particle", C.c_int32), ("kernel_launches", C.c_int64),
                ("pair_build", C.c_int32), ("wait_timeouts", C.c_int32), ("h_refined", C.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["grid"] = list(self.grid)
        return d


class rt_tuning(C.Structure):
    _fields_ = [("flux_variant", C.c_int32), ("gather_variant", C.c_int32), ("gradient_variant", C.c_int32),
                ("cell_eighths", C.c_int32), ("gradient_block", C.c_int32), ("gather_block", C.c_int32),
                ("pair_warps", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


TUNING_KEYS = tuple(k for k, _ in rt_tuning._fields_)


class RTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def library_path() -> str:
    return _LIB_PATH


def load_library():
    """Load librt_gb300.so (built by ``build_ext.build()``); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: build it with paper_2302_12727_gb300.build_ext.build()")
    lib = C.CDLL(_LIB_PATH)
    vp, dp, i64 = C.c_void_p, C.c_void_p, C.c_int64
    lib.rt_create.argtypes = [C.POINTER(rt_config), i64, i64, vp, C.POINTER(vp)]
    lib.rt_set_stream.argtypes = [vp, vp]
    lib.rt_neighbours.argtypes = [vp, dp, dp, dp, dp]
    lib.rt_neighbours_given_h.argtypes = [vp, dp, dp, dp, dp, dp]
    lib.rt_source_fields.argtypes = [vp, dp]
    lib.rt_neighbours_given_fields.argtypes = [vp, dp, dp, dp, dp, dp, dp, dp]
    lib.rt_source_norms.argtypes = [vp, dp, dp]
    lib.rt_set_owned.argtypes = [vp, i64]
    lib.rt_gradients.argtypes = [vp, dp, dp]
    lib.rt_transport_step.argtypes = [vp, C.c_double, dp, dp, dp]
    lib.rt_inject.argtypes = [vp, C.c_double, dp, dp]
    lib.rt_transport_step_given_gradients.argtypes = [vp, C.c_double, dp, dp, dp]
    lib.rt_set_fields.argtypes = [vp, i64, i64, dp, dp]
    lib.rt_subcycle.argtypes = [vp, C.c_int32, C.c_double, dp, dp, dp]
    lib.rt_adjoint.argtypes = [vp, C.c_int32, C.c_double, C.c_int32, dp, dp, dp, dp, dp, dp]
    lib.rt_energy.argtypes = [vp, dp, C.POINTER(C.c_double)]
    lib.rt_drift.argtypes = [vp, dp, dp, C.c_double]
    lib.rt_set_time_bins.argtypes = [vp, vp, C.c_double, C.c_double, C.c_int32, C.c_int32]
    lib.rt_get_time_bins.argtypes = [vp, vp, C.POINTER(C.c_int32)]
    lib.rt_step_bins.argtypes = [vp, dp, dp, dp]
    lib.rt_set_absorbers.argtypes = [vp, C.c_int32, dp, dp]
    lib.rt_cross_section.argtypes = [C.c_int32, C.c_double, dp]
    lib.rt_blackbody_groups.argtypes = [C.c_double, C.c_int32, dp, dp, dp, dp]
    lib.rt_photon_number_to_luminosity.argtypes = [C.c_double, C.c_double, C.c_int32, dp, dp]
    lib.rt_particle_fields.argtypes = [vp, dp, dp, dp, dp]
    lib.rt_pairs.argtypes = [vp, dp, dp]
    lib.rt_diagnostics.argtypes = [vp, C.POINTER(rt_diag)]
    lib.rt_set_profiling.argtypes = [vp, C.c_int32]
    lib.rt_kernel_times.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64)]
    lib.rt_wave_table.argtypes = [dp, dp]
    lib.rt_set_tuning.argtypes = [vp, C.POINTER(rt_tuning)]
    lib.rt_wait_selftest.argtypes = [vp, C.c_uint64]
    lib.rt_get_tuning.argtypes = [vp, C.POINTER(rt_tuning)]
    lib.rt_autotune.argtypes = [vp, dp, C.c_double, C.c_int32, dp, dp, C.c_int32, C.POINTER(rt_tuning),
                                C.POINTER(C.c_double)]
    lib.rt_energy_static.argtypes = [vp, vp, i64, C.c_int32, C.c_int32, vp, vp]
    lib.rt_last_error.argtypes = [vp]
    lib.rt_last_error.restype = C.c_char_p
    lib.rt_destroy.argtypes = [vp]
    lib.rt_destroy.restype = None
    for name in EXPORTED:
        if name not in ("rt_last_error", "rt_destroy"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


# ----------------------------------------------------------------------------------------
# argument marshalling
def _ptr(t):
    """Device pointer of a CUDA tensor (or an int pointer, or None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _check(ctx, status):
    if status != RT_OK:
        msg = load_library().rt_last_error(ctx)
        raise RTError(status, msg.decode() if msg else "")


def make_config(n_groups=1, c_red=1.0, eta_res=1.2348, eta_res_star=1.2348, box=(1.0, 1.0, 1.0), periodic=True,
                precision=RT_FP32_MIXED, clamp_negative=False, h_tol=1e-6, h_max_iter=100,
                riemann="glf") -> rt_config:
    if riemann not in ("glf", "hll"):
        raise ValueError("riemann must be 'glf' or 'hll'")
    return rt_config(n_groups, c_red, eta_res, eta_res_star, (C.c_double * 3)(*box), int(periodic), precision,
                     int(clamp_negative), 0, h_tol, h_max_iter, 0,
                     RT_RIEMANN_HLL if riemann == "hll" else RT_RIEMANN_GLF)


def rt_create(cfg: rt_config, n: int, n_src: int, stream=None):
    """Returns the context handle (an int)."""
    lib = load_library()
    out = C.c_void_p()
    s = lib.rt_create(C.byref(cfg), int(n), int(n_src), stream, C.byref(out))
    if s != RT_OK:
        msg = lib.rt_last_error(out) if out.value else b"allocation failed"
        if out.value:
            lib.rt_destroy(out)
        raise RTError(s, msg.decode())
    return out.value


def rt_set_stream(ctx, stream):
    _check(ctx, load_library().rt_set_stream(ctx, stream))


def rt_neighbours(ctx, x, m=None, xsrc=None, h_out=None):
    _check(ctx, load_library().rt_neighbours(ctx, _ptr(x), _ptr(m), _ptr(xsrc), _ptr(h_out)))


def rt_neighbours_given_h(ctx, x, m, xsrc, h, hs):
    _check(ctx, load_library().rt_neighbours_given_h(ctx, _ptr(x), _ptr(m), _ptr(xsrc), _ptr(h), _ptr(hs)))


def rt_neighbours_given_fields(ctx, x, m, xsrc, h, hs, omegas, octw):
    _check(ctx, load_library().rt_neighbours_given_fields(ctx, _ptr(x), _ptr(m), _ptr(xsrc), _ptr(h), _ptr(hs),
                                                          _ptr(omegas), _ptr(octw)))


def rt_source_fields(ctx, hs_out):
    _check(ctx, load_library().rt_source_fields(ctx, _ptr(hs_out)))


def rt_source_norms(ctx, omegas_out, octw_out):
    _check(ctx, load_library().rt_source_norms(ctx, _ptr(omegas_out), _ptr(octw_out)))


def rt_set_owned(ctx, n_owned):
    _check(ctx, load_library().rt_set_owned(ctx, int(n_owned)))


def rt_gradients(ctx, U, gradU):
    _check(ctx, load_library().rt_gradients(ctx, _ptr(U), _ptr(gradU)))


def rt_transport_step(ctx, dt, U, Lsrc=None, alpha=None):
    _check(ctx, load_library().rt_transport_step(ctx, float(dt), _ptr(U), _ptr(Lsrc), _ptr(alpha)))


def rt_inject(ctx, dt, U, Lsrc=None):
    _check(ctx, load_library().rt_inject(ctx, float(dt), _ptr(U), _ptr(Lsrc)))


def rt_transport_step_given_gradients(ctx, dt, U, gradU, alpha=None):
    _check(ctx, load_library().rt_transport_step_given_gradients(ctx, float(dt), _ptr(U), _ptr(gradU), _ptr(alpha)))


def rt_set_fields(ctx, first, count, omega, B):
    _check(ctx, load_library().rt_set_fields(ctx, int(first), int(count), _ptr(omega), _ptr(B)))


def rt_subcycle(ctx, n_sub, dt, U, Lsrc=None, alpha=None):
    _check(ctx, load_library().rt_subcycle(ctx, int(n_sub), float(dt), _ptr(U), _ptr(Lsrc), _ptr(alpha)))


def rt_adjoint(ctx, n_sub, dt, ckpt_every, U0, Lsrc, alpha, dLdU_final, dLdU0, dLdLsrc=None):
    _check(ctx, load_library().rt_adjoint(ctx, int(n_sub), float(dt), int(ckpt_every), _ptr(U0), _ptr(Lsrc),
                                          _ptr(alpha), _ptr(dLdU_final), _ptr(dLdU0), _ptr(dLdLsrc)))


def rt_energy(ctx, U, n_groups):
    out = (C.c_double * n_groups)()
    _check(ctx, load_library().rt_energy(ctx, _ptr(U), out))
    return list(out)


def rt_particle_fields(ctx, h=None, omega=None, V=None, B=None):
    _check(ctx, load_library().rt_particle_fields(ctx, _ptr(h), _ptr(omega), _ptr(V), _ptr(B)))


def rt_pairs(ctx, offsets, cols):
    _check(ctx, load_library().rt_pairs(ctx, _ptr(offsets), _ptr(cols)))


def rt_diagnostics(ctx) -> dict:
    d = rt_diag()
    _check(ctx, load_library().rt_diagnostics(ctx, C.byref(d)))
    return d.as_dict()


def rt_drift(ctx, U, v, dt_drift):
    """U += grad U . (v dt_drift) in place (Sec. "Dealing With Particle Drifts")."""
    _check(ctx, load_library().rt_drift(ctx, _ptr(U), _ptr(v), float(dt_drift)))


def rt_set_absorbers(ctx, n_species, sigma):
    """Photo-ionisation sink per group: n_species [J, N] device densities (or None to clear),
    sigma [G, J] cross sections (host)."""
    import numpy as np
    if n_species is None:
        _check(ctx, load_library().rt_set_absorbers(ctx, 0, None, None))
        return
    sig = np.ascontiguousarray(sigma, dtype=np.float64)
    _check(ctx, load_library().rt_set_absorbers(ctx, int(sig.shape[1]), _ptr(n_species), sig.ctypes.data))


def rt_cross_section(species: int, E_eV: float) -> float:
    out = C.c_double()
    if load_library().rt_cross_section(int(species), float(E_eV), C.addressof(out)) != RT_OK:
        raise RTError(1, "rt_cross_section: species must be 0, 1 or 2")
    return out.value


def rt_blackbody_groups(T_bb: float, nu_edges):
    """(eps_mean [G] erg, sigma_N [G, 3], sigma_E [G, 3] cm^2) for a blackbody spectrum."""
    import numpy as np
    e = np.ascontiguousarray(nu_edges, dtype=np.float64)
    G = e.size - 1
    eps, sN, sE = np.empty(G), np.empty((G, 3)), np.empty((G, 3))
    st = load_library().rt_blackbody_groups(float(T_bb), G, e.ctypes.data, eps.ctypes.data, sN.ctypes.data,
                                            sE.ctypes.data)
    if st != RT_OK:
        raise RTError(st, "rt_blackbody_groups")
    return eps, sN, sE


def rt_photon_number_to_luminosity(T_bb: float, Ndot: float, nu_edges):
    import numpy as np
    e = np.ascontiguousarray(nu_edges, dtype=np.float64)
    L = np.empty(e.size - 1)
    st = load_library().rt_photon_number_to_luminosity(float(T_bb), float(Ndot), e.size - 1, e.ctypes.data,
                                                       L.ctypes.data)
    if st != RT_OK:
        raise RTError(st, "rt_photon_number_to_luminosity")
    return L


def rt_set_time_bins(ctx, bins=None, dt_min=1.0, cfl=0.0, max_bin=20, limit=True):
    """Time bins from `bins` (device int32 [N]) or from the CFL step (bins None)."""
    _check(ctx, load_library().rt_set_time_bins(ctx, _ptr(bins), float(dt_min), float(cfl), int(max_bin),
                                                1 if limit else 0))


def rt_get_time_bins(ctx, bins_out=None) -> int:
    """Writes the bins in use into bins_out (device int32 [N], optional); returns B."""
    mx = C.c_int32(0)
    _check(ctx, load_library().rt_get_time_bins(ctx, _ptr(bins_out), C.byref(mx)))
    return mx.value


def rt_step_bins(ctx, U, Lsrc=None, alpha=None):
    _check(ctx, load_library().rt_step_bins(ctx, _ptr(U), _ptr(Lsrc), _ptr(alpha)))


def rt_set_profiling(ctx, on):
    """on: False / 0 off, True / 1 every kernel of the step, k >= 2 the pair-flux launches
    only, one in every k - 1 of a call."""
    _check(ctx, load_library().rt_set_profiling(ctx, int(on)))


def rt_kernel_times(ctx):
    """{kind: (ms, launches)} of the most recent profiled step or sub-cycle call."""
    ms = (C.c_double * RT_KERNEL_KINDS)()
    nl = (C.c_int64 * RT_KERNEL_KINDS)()
    _check(ctx, load_library().rt_kernel_times(ctx, ms, nl))
    names = ("inject", "gradient", "flux", "flux_gather")
    return {names[k]: (ms[k], nl[k]) for k in range(RT_KERNEL_KINDS)}


def rt_set_tuning(ctx, flux_variant: int = 2, gather_variant: int = 1, gradient_variant: int = 2,
                  cell_eighths: int = 0, gradient_block: int = 0, gather_block: int = 0, pair_warps: int = 0):
    """Launch variants and shapes of the float pair kernels and the cell size of the neighbour
    search (see rt.h; 0 keeps the cell size and takes the default shapes)."""
    t = rt_tuning(int(flux_variant), int(gather_variant), int(gradient_variant), int(cell_eighths),
                  int(gradient_block), int(gather_block), int(pair_warps))
    _check(ctx, load_library().rt_set_tuning(ctx, C.byref(t)))


def rt_wait_selftest(ctx, budget_cycles: int) -> bool:
    """True when the bounded device wait on a barrier that nothing completes ran out after
    budget_cycles SM cycles (the expected outcome, status RT_ERR_TIMEOUT); other errors raise."""
    s = load_library().rt_wait_selftest(ctx, int(budget_cycles))
    if s == 6:
        return True
    _check(ctx, s)
    return False


def rt_get_tuning(ctx) -> dict:
    t = rt_tuning()
    _check(ctx, load_library().rt_get_tuning(ctx, C.byref(t)))
    return t.as_dict()


def rt_autotune(ctx, U, dt, n_sub, Lsrc=None, alpha=None, repeats=3):
    """Times every launch-variant candidate on U and adopts the fastest:
    returns ({flux_variant, gather_variant, gradient_variant}, [ms per candidate])."""
    t = rt_tuning()
    ms = (C.c_double * RT_TUNE_CANDIDATES)()
    _check(ctx, load_library().rt_autotune(ctx, _ptr(U), float(dt), int(n_sub), _ptr(Lsrc), _ptr(alpha),
                                           int(repeats), C.byref(t), ms))
    return t.as_dict(), list(ms)


def rt_wave_table():
    """The library's HLL wave-speed table (lmax, lmin), [RT_WAVE_NF, RT_WAVE_NTH] in units of c
    (host computation, no context or GPU)."""
    import numpy as np
    lmax = np.empty((RT_WAVE_NF, RT_WAVE_NTH))
    lmin = np.empty((RT_WAVE_NF, RT_WAVE_NTH))
    st = load_library().rt_wave_table(lmax.ctypes.data, lmin.ctypes.data)
    if st != RT_OK:
        raise RTError(st, "rt_wave_table")
    return lmax, lmin


def rt_energy_static(U, V, n, n_groups, precision, E_out, stream=None):
    """Energy per group into the device array E_out without any allocation (no context)."""
    st = load_library().rt_energy_static(_ptr(U), _ptr(V), int(n), int(n_groups), int(precision), stream,
                                         _ptr(E_out))
    if st != RT_OK:
        raise RTError(st, "rt_energy_static rejected the call")


def rt_last_error(ctx) -> str:
    m = load_library().rt_last_error(ctx)
    return m.decode() if m else ""


def rt_destroy(ctx):
    if ctx:
        load_library().rt_destroy(ctx)


from .transport import Transport, SubcycleFunction  # noqa: E402  (torch-facing wrapper)
