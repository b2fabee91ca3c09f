"""ctypes binding of the FP64 CPU oracle (``rt_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it to check and time the CUDA library.  The library never
imports this package.

Array layouts follow the C interface of the library: positions [3, N], state
[G, 4, N] (E, Fx, Fy, Fz), luminosities [S, G], gradients [4G, 3, N].
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

from . import m1_eigen

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rt_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")

H_OVER_h = 1.825742


def build(force: bool = False) -> str:
    """Compile the oracle (plain g++, no contraction of multiply-adds, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c++17",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Cfg(C.Structure):
    _fields_ = [("n_groups", C.c_int32), ("c_red", C.c_double), ("eta_res", C.c_double),
                ("eta_res_star", C.c_double), ("box", C.c_double * 3), ("periodic", C.c_int32),
                ("clamp_negative", C.c_int32), ("h_tol", C.c_double), ("h_max_iter", C.c_int32),
                ("brute_force", C.c_int32), ("riemann", C.c_int32)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        vp, dp, lp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_long), C.POINTER(C.c_int32)
        lib.orc_create.restype = vp
        lib.orc_create.argtypes = [C.POINTER(_Cfg), C.c_long, dp, dp, C.c_long, dp, C.POINTER(C.c_int)]
        lib.orc_destroy.argtypes = [vp]
        lib.orc_create_given_h.restype = vp
        lib.orc_create_given_h.argtypes = [C.POINTER(_Cfg), C.c_long, dp, dp, C.c_long, dp, dp, dp, dp, dp,
                                           C.POINTER(C.c_int)]
        lib.orc_num_directed_pairs.restype = C.c_long
        lib.orc_num_directed_pairs.argtypes = [vp]
        lib.orc_get_pairs.argtypes = [vp, lp, ip]
        lib.orc_get_particles.argtypes = [vp, dp, dp, dp, dp, dp]
        lib.orc_get_surfaces.argtypes = [vp, dp]
        lib.orc_get_psitilde.argtypes = [vp, dp]
        lib.orc_num_injection_entries.restype = C.c_long
        lib.orc_num_injection_entries.argtypes = [vp]
        lib.orc_get_sources.argtypes = [vp, dp, dp, dp, ip, ip, dp]
        lib.orc_geometry_stats.argtypes = [vp, lp, dp]
        lib.orc_gradients.argtypes = [vp, dp, dp]
        lib.orc_run.restype = C.c_long
        lib.orc_run.argtypes = [vp, C.c_int, C.c_double, dp, dp, dp]
        lib.orc_inject.argtypes = [vp, C.c_double, dp, dp]
        lib.orc_transport_given_gradients.restype = C.c_long
        lib.orc_transport_given_gradients.argtypes = [vp, C.c_double, dp, dp, dp]
        lib.orc_set_fields.argtypes = [vp, C.c_long, C.c_long, dp, dp]
        lib.orc_jvp.argtypes = [vp, C.c_int, C.c_double, dp, dp, dp, dp, dp, dp, dp]
        lib.orc_jvp_kinks.restype = C.c_long
        lib.orc_jvp_kinks.argtypes = [vp, C.c_int, C.c_double, dp, dp, dp, dp, dp, C.c_double]
        lib.orc_energy.argtypes = [vp, dp, dp]
        lib.orc_dt_positivity.restype = C.c_double
        lib.orc_dt_positivity.argtypes = [vp]
        lib.orc_m1_flux.argtypes = [dp, dp, C.c_double, dp]
        lib.orc_kernel_W.restype = C.c_double
        lib.orc_kernel_W.argtypes = [C.c_double, C.c_double]
        lib.orc_minmod.restype = C.c_double
        lib.orc_minmod.argtypes = [C.c_double, C.c_double]
        lib.orc_num_threads.restype = C.c_int
        lib.orc_face_states.argtypes = [dp, dp, dp, dp, dp, C.c_double, C.c_double, dp, dp]
        lib.orc_glf_flux.argtypes = [dp, dp, dp, C.c_double, dp]
        lib.orc_get_psi.argtypes = [vp, dp, dp]
        lib.orc_set_wave_table.argtypes = [vp, dp, dp, C.c_int, C.c_int]
        lib.orc_drift.argtypes = [vp, dp, dp, C.c_double, dp]
        lib.orc_step_bins.restype = C.c_long
        lib.orc_step_bins.argtypes = [vp, C.c_double, ip, C.c_int, dp, dp, dp]
        lib.orc_cfl_bins.argtypes = [vp, C.c_double, C.c_double, C.c_int, ip]
        lib.orc_run_groups.restype = C.c_long
        lib.orc_run_groups.argtypes = [vp, C.c_int, C.c_double, dp, dp, dp]
        lib.orc_hll_flux.argtypes = [vp, dp, dp, dp, dp]
        lib.orc_wave_speeds.argtypes = [vp, dp, dp, dp, dp]
        lib.orc_pair_flops.argtypes = [vp, dp]
        _lib = lib
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    pass


@dataclass
class Sources:
    hs: np.ndarray
    omegas: np.ndarray
    octw: np.ndarray      # [S, 8]
    e_src: np.ndarray
    e_gas: np.ndarray
    e_xi: np.ndarray


class Oracle:
    """One particle set with its neighbour geometry, built by the oracle."""

    def __init__(self, x, m, xsrc=None, *, n_groups=1, c_red=1.0, eta_res=1.2348, eta_res_star=1.2348,
                 box=(1.0, 1.0, 1.0), periodic=True, clamp_negative=False, h_tol=1e-15, h_max_iter=200,
                 brute_force=False, riemann="glf", wave_table=None, h=None, hs=None, omegas=None,
                 octw=None):
        """riemann: "glf" (Eq. riemann-GLF) or "hll" (Eq. riemann-HLL); for HLL the wave-speed
        table (lmax, lmin) over (f, theta) defaults to m1_eigen.default_table().  h [N] and hs
        [S]: smoothing lengths given instead of solved (omega is then evaluated at them);
        with them, omegas [S] and octw [S, 8]: the sources' omega_s and octant sums given
        instead of formed from this set's gas."""
        lib = _load()
        self.lib = lib
        self.x = _c(x)
        self.m = _c(m)
        self.n = self.x.shape[1]
        self.xsrc = _c(np.zeros((3, 0)) if xsrc is None else xsrc)
        self.n_src = self.xsrc.shape[1]
        self.G = n_groups
        self.c_red = c_red
        if riemann not in ("glf", "hll"):
            raise ValueError("riemann must be 'glf' or 'hll'")
        cfg = _Cfg(n_groups, c_red, eta_res, eta_res_star, (C.c_double * 3)(*box), int(periodic),
                   int(clamp_negative), h_tol, h_max_iter, int(brute_force), int(riemann == "hll"))
        st = C.c_int(0)
        if h is None:
            self._p = lib.orc_create(C.byref(cfg), self.n, _dp(self.x), _dp(self.m), self.n_src,
                                     _dp(self.xsrc) if self.n_src else _dp(np.zeros(3)), C.byref(st))
        else:
            hh = _c(h)
            hsa = _c(hs if hs is not None and self.n_src else np.zeros(1))
            oms = None if omegas is None or not self.n_src else _c(omegas)
            ow = None if octw is None or not self.n_src else _c(octw).reshape(self.n_src, 8)
            self._p = lib.orc_create_given_h(C.byref(cfg), self.n, _dp(self.x), _dp(self.m), self.n_src,
                                             _dp(self.xsrc) if self.n_src else _dp(np.zeros(3)), _dp(hh),
                                             _dp(hsa), None if oms is None else _dp(oms),
                                             None if ow is None else _dp(ow), C.byref(st))
        if st.value != 0:
            lib.orc_destroy(self._p)
            self._p = None
            raise OracleError(f"oracle build failed with status {st.value}")
        self._cache = {}
        if riemann == "hll" or wave_table is not None:
            self.set_wave_table(*(wave_table if wave_table is not None else m1_eigen.default_table()))

    def set_wave_table(self, lmax, lmin):
        lmax, lmin = _c(lmax), _c(lmin)
        self._wt = (lmax, lmin)
        self.lib.orc_set_wave_table(self._p, _dp(lmax), _dp(lmin), lmax.shape[0], lmax.shape[1])

    def hll_flux(self, uL, uR, A):
        phi = np.empty(4)
        self.lib.orc_hll_flux(self._p, _dp(_c(uL)), _dp(_c(uR)), _dp(_c(A)), _dp(phi))
        return phi

    def wave_speeds(self, u, A):
        a, b = C.c_double(0), C.c_double(0)
        self.lib.orc_wave_speeds(self._p, _dp(_c(u)), _dp(_c(A)), C.byref(a), C.byref(b))
        return a.value, b.value

    def __del__(self):
        if getattr(self, "_p", None):
            self.lib.orc_destroy(self._p)
            self._p = None

    # -- geometry --------------------------------------------------------------------
    def particles(self):
        if "part" not in self._cache:
            n = self.n
            h, om, V, B, cond = (np.empty(n), np.empty(n), np.empty(n), np.empty(9 * n), np.empty(n))
            self.lib.orc_get_particles(self._p, _dp(h), _dp(om), _dp(V), _dp(B), _dp(cond))
            self._cache["part"] = dict(h=h, omega=om, V=V, B=B.reshape(n, 3, 3), cond=cond)
        return self._cache["part"]

    @property
    def h(self):
        return self.particles()["h"]

    @property
    def omega(self):
        return self.particles()["omega"]

    @property
    def V(self):
        return self.particles()["V"]

    def pairs(self):
        if "pairs" not in self._cache:
            P2 = self.lib.orc_num_directed_pairs(self._p)
            off = np.empty(self.n + 1, dtype=np.int64)
            cols = np.empty(P2, dtype=np.int32)
            self.lib.orc_get_pairs(self._p, off.ctypes.data_as(C.POINTER(C.c_long)),
                                   cols.ctypes.data_as(C.POINTER(C.c_int32)))
            self._cache["pairs"] = (off, cols)
        return self._cache["pairs"]

    def surfaces(self):
        P2 = self.lib.orc_num_directed_pairs(self._p)
        A = np.empty(3 * P2)
        self.lib.orc_get_surfaces(self._p, _dp(A))
        return A.reshape(3, P2)

    def psitilde(self):
        P2 = self.lib.orc_num_directed_pairs(self._p)
        A = np.empty(3 * P2)
        self.lib.orc_get_psitilde(self._p, _dp(A))
        return A.reshape(3, P2)

    def psi(self):
        """(psi_j(x_i) per directed pair entry, psi_i(x_i) per particle)."""
        P2 = self.lib.orc_num_directed_pairs(self._p)
        ps, self_ = np.empty(P2), np.empty(self.n)
        self.lib.orc_get_psi(self._p, _dp(ps), _dp(self_))
        return ps, self_

    def sources(self) -> Sources:
        S = self.n_src
        ne = self.lib.orc_num_injection_entries(self._p)
        hs, om, octw = np.empty(max(S, 1)), np.empty(max(S, 1)), np.empty(8 * max(S, 1))
        es, eg, ex = np.empty(max(ne, 1), np.int32), np.empty(max(ne, 1), np.int32), np.empty(max(ne, 1))
        ip = C.POINTER(C.c_int32)
        self.lib.orc_get_sources(self._p, _dp(hs), _dp(om), _dp(octw), es.ctypes.data_as(ip),
                                 eg.ctypes.data_as(ip), _dp(ex))
        return Sources(hs[:S], om[:S], octw[:8 * S].reshape(S, 8), es[:ne], eg[:ne], ex[:ne])

    def geometry_stats(self):
        n_ill = C.c_long(0)
        cmax = C.c_double(0)
        self.lib.orc_geometry_stats(self._p, C.byref(n_ill), C.byref(cmax))
        return n_ill.value, cmax.value

    def dt_positivity(self) -> float:
        return self.lib.orc_dt_positivity(self._p)

    # -- transport -----------------------------------------------------------------------
    def gradients(self, U):
        U = _c(U).reshape(4 * self.G, self.n)
        g = np.empty((4 * self.G, 3, self.n))
        self.lib.orc_gradients(self._p, _dp(U), _dp(g))
        return g

    def run(self, U0, n_sub, dt, L=None, alpha=None, alpha_groups=None):
        """n_sub steps (inject -> transport -> sink); returns (U, clamp_count).  alpha [N] is a
        grey absorption; alpha_groups [G, N] one per group (photo-ionisation sink)."""
        U = _c(U0).copy().reshape(self.G, 4, self.n)
        L = _c(np.zeros((self.n_src, self.G)) if L is None else L).reshape(self.n_src, self.G)
        if alpha_groups is not None:
            ag = _c(alpha_groups).reshape(self.G, self.n)
            nclamp = self.lib.orc_run_groups(self._p, int(n_sub), float(dt), _dp(U),
                                             _dp(L) if L.size else _dp(np.zeros(1)), _dp(ag))
            return U, nclamp
        a = None if alpha is None else _c(alpha)
        nclamp = self.lib.orc_run(self._p, int(n_sub), float(dt), _dp(U), _dp(L) if L.size else _dp(np.zeros(1)),
                                  _dp(a))
        return U, nclamp

    def inject(self, U0, dt, L):
        """The injection stage of one step alone (E_g += xi_sg L_s dt / V_g); returns U."""
        U = _c(U0).copy().reshape(self.G, 4, self.n)
        L = _c(np.zeros((self.n_src, self.G)) if L is None else L).reshape(self.n_src, self.G)
        self.lib.orc_inject(self._p, float(dt), _dp(U), _dp(L) if L.size else _dp(np.zeros(1)))
        return U

    def transport_given_gradients(self, U0, grad, dt, alpha=None):
        """The transport and sink of one step with the gradients grad [G, 4, 3, N] given (no
        injection); returns (U, clamp_count)."""
        U = _c(U0).copy().reshape(self.G, 4, self.n)
        g = _c(grad).reshape(self.G, 4, 3, self.n)
        a = None if alpha is None else _c(alpha)
        nclamp = self.lib.orc_transport_given_gradients(self._p, float(dt), _dp(U), _dp(g), _dp(a))
        return U, nclamp

    def set_fields(self, first, omega, B):
        """Give omega (V = 1 / omega) and B [k, 3, 3] of particles first, first + 1, ..."""
        om = _c(omega).reshape(-1)
        b = _c(B).reshape(len(om), 3, 3)
        self.lib.orc_set_fields(self._p, int(first), len(om), _dp(om), _dp(b))
        self._cache.clear()

    def jvp(self, U0, dU0, n_sub, dt, L, dL, alpha=None):
        U0 = _c(U0).reshape(self.G, 4, self.n)
        dU0 = _c(dU0).reshape(self.G, 4, self.n)
        L = _c(L).reshape(self.n_src, self.G)
        dL = _c(dL).reshape(self.n_src, self.G)
        U = np.empty_like(U0)
        dU = np.empty_like(U0)
        a = None if alpha is None else _c(alpha)
        z = _dp(np.zeros(1))
        self.lib.orc_jvp(self._p, int(n_sub), float(dt), _dp(U0), _dp(dU0), _dp(L) if L.size else z,
                         _dp(dL) if dL.size else z, _dp(a), _dp(U), _dp(dU))
        return U, dU

    def jvp_kinks(self, U0, dU0, n_sub, dt, L, dL, alpha=None, eps=1e-6):
        """Branch points of the limiter and the closure within eps along (dU0, dL) over n_sub
        steps (first order): 0 means central differences of step eps see a smooth map."""
        U0 = _c(U0).reshape(self.G, 4, self.n)
        dU0 = _c(dU0).reshape(self.G, 4, self.n)
        L = _c(L).reshape(self.n_src, self.G)
        dL = _c(dL).reshape(self.n_src, self.G)
        a = None if alpha is None else _c(alpha)
        z = _dp(np.zeros(1))
        return int(self.lib.orc_jvp_kinks(self._p, int(n_sub), float(dt), _dp(U0), _dp(dU0),
                                          _dp(L) if L.size else z, _dp(dL) if dL.size else z, _dp(a), float(eps)))

    def step_bins(self, U0, dt_min, bins, L=None, alpha=None, limit=True):
        """One hydro step with individual time bins (see rt_oracle.cpp): returns
        (U, bins after the limiter, clamp count)."""
        U = _c(U0).copy().reshape(self.G, 4, self.n)
        L = _c(np.zeros((self.n_src, self.G)) if L is None else L).reshape(self.n_src, self.G)
        b = np.ascontiguousarray(bins, dtype=np.int32).copy()
        a = None if alpha is None else _c(alpha)
        ip = C.POINTER(C.c_int32)
        nclamp = self.lib.orc_step_bins(self._p, float(dt_min), b.ctypes.data_as(ip), int(limit), _dp(U),
                                        _dp(L) if L.size else _dp(np.zeros(1)), _dp(a))
        return U, b, nclamp

    def cfl_bins(self, cfl, dt_min, max_bin):
        b = np.empty(self.n, dtype=np.int32)
        self.lib.orc_cfl_bins(self._p, float(cfl), float(dt_min), int(max_bin), b.ctypes.data_as(C.POINTER(C.c_int32)))
        return b

    def drift(self, U, v, dt_drift):
        """Drift-corrected state U + grad U . (v dt_drift) (Sec. "Dealing With Particle Drifts");
        v is [3, N]; the gradients are those of this (old) particle set."""
        U = _c(U).reshape(self.G, 4, self.n)
        out = np.empty_like(U)
        self.lib.orc_drift(self._p, _dp(U), _dp(_c(v)), float(dt_drift), _dp(out))
        return out

    def pair_flops(self):
        """Floating-point operations of one pair evaluation, counted on the oracle's own pair
        arithmetic (add, sub, mul, div, sqrt one each): dict with flux_geometry (per
        unordered pair, averaged over this particle set's pairs), flux_per_group (per pair
        and group, general branch), accumulate_per_group (both particles' sums),
        gradient_geometry (per directed entry, averaged) and gradient_per_group (per
        directed entry and group)."""
        out = np.zeros(5)
        self.lib.orc_pair_flops(self._p, _dp(out))
        keys = ("flux_geometry", "flux_per_group", "accumulate_per_group", "gradient_geometry",
                "gradient_per_group")
        return dict(zip(keys, out.tolist()))

    def energy(self, U):
        U = _c(U)
        E = np.empty(self.G)
        self.lib.orc_energy(self._p, _dp(U), _dp(E))
        return E


def kernel_W(r: float, h: float) -> float:
    return _load().orc_kernel_W(float(r), float(h))


def minmod(a: float, b: float) -> float:
    return _load().orc_minmod(float(a), float(b))


def m1_flux(u4, A, c: float):
    u4 = _c(u4)
    A = _c(A)
    out = np.empty(4)
    _load().orc_m1_flux(_dp(u4), _dp(A), float(c), _dp(out))
    return out


def face_states(uk, ul, gk, gl, d, hk, hl):
    """Limited interface states of one pair and group; g* are [4, 3] gradients."""
    uL, uR = np.empty(4), np.empty(4)
    _load().orc_face_states(_dp(_c(uk)), _dp(_c(ul)), _dp(_c(gk).ravel()), _dp(_c(gl).ravel()), _dp(_c(d)),
                            float(hk), float(hl), _dp(uL), _dp(uR))
    return uL, uR


def glf_flux(uL, uR, A, c: float):
    phi = np.empty(4)
    _load().orc_glf_flux(_dp(_c(uL)), _dp(_c(uR)), _dp(_c(A)), float(c), _dp(phi))
    return phi


def num_threads() -> int:
    return _load().orc_num_threads()
