"""Torch-facing wrapper of the C interface.

``Transport`` owns one library context for one particle set: it moves the inputs to the
device, calls ``rt_neighbours`` once, and exposes the transport calls on torch tensors.
``SubcycleFunction`` makes ``rt_subcycle`` differentiable through the library's
hand-written adjoint (``rt_adjoint``).  PyTorch only provides device memory and the
current stream here; all arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import (RT_FP32_MIXED, RT_FP64, make_config, rt_adjoint, rt_create, rt_destroy, rt_diagnostics, rt_drift,
               rt_energy, rt_get_tuning, rt_gradients, rt_neighbours, rt_neighbours_given_h, rt_pairs,
               rt_inject, rt_neighbours_given_fields, rt_particle_fields, rt_set_fields, rt_set_owned,
               rt_set_stream, rt_set_tuning, rt_source_fields, rt_source_norms, rt_subcycle, rt_transport_step,
               rt_transport_step_given_gradients)


def _dev(a, dtype, device):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        a = torch.from_numpy(np.ascontiguousarray(a))
    return a.to(device=device, dtype=dtype).contiguous()


class Transport:
    """One particle configuration with its neighbour lists and geometry on the GPU.

    x [3, N] and m [N] (float64), xsrc [3, S].  ``precision`` is "fp32" (mixed: float
    fluxes and gradients, double geometry and energy sums) or "fp64".
    """

    def __init__(self, x, m=None, xsrc=None, *, n_groups=1, c_red=1.0, eta_res=1.2348, eta_res_star=None,
                 box=(1.0, 1.0, 1.0), periodic=True, precision="fp32", clamp_negative=False, h_tol=1e-6,
                 h_max_iter=100, device="cuda:0", riemann="glf", h=None, hs=None, omegas=None, octw=None):
        self.device = torch.device(device)
        self.x = _dev(x, torch.float64, self.device)
        self.n = int(self.x.shape[1])
        self.m = _dev(m if m is not None else np.full(self.n, 1.0 / self.n), torch.float64, self.device)
        xs = np.zeros((3, 0)) if xsrc is None else xsrc
        self.xsrc = _dev(xs, torch.float64, self.device)
        self.n_src = int(self.xsrc.shape[1])
        self.G = int(n_groups)
        self.precision = precision
        self.riemann = riemann
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.cfg = make_config(self.G, c_red, eta_res, eta_res if eta_res_star is None else eta_res_star, box,
                               periodic, RT_FP64 if precision == "fp64" else RT_FP32_MIXED, clamp_negative, h_tol,
                               h_max_iter, riemann)
        self.c_red = c_red
        self.ctx = None
        with torch.cuda.device(self.device):
            self.ctx = rt_create(self.cfg, self.n, self.n_src, self._stream())
            self.h = torch.empty(self.n, dtype=torch.float64, device=self.device)
            if h is None:
                rt_neighbours(self.ctx, self.x, self.m, self.xsrc if self.n_src else None, self.h)
            else:
                self.rebuild_given_h(h, hs, omegas=omegas, octw=octw)

    def rebuild_given_h(self, h, hs=None, x=None, omegas=None, octw=None):
        """Neighbour search with given smoothing lengths h [N] and source lengths hs [S]
        (rt_neighbours_given_h), and with omegas [S] and octw [S, 8] also the sources'
        normalisations (rt_neighbours_given_fields)."""
        if x is not None:
            self.x = _dev(x, torch.float64, self.device)
        self._sync_stream()
        hd = _dev(h, torch.float64, self.device)
        hsd = _dev(hs, torch.float64, self.device) if self.n_src else None
        xs = self.xsrc if self.n_src else None
        if omegas is not None and self.n_src:
            rt_neighbours_given_fields(self.ctx, self.x, self.m, xs, hd, hsd, _dev(omegas, torch.float64, self.device),
                                       _dev(octw, torch.float64, self.device))
        else:
            rt_neighbours_given_h(self.ctx, self.x, self.m, xs, hd, hsd)
        self.h = hd.clone()

    def source_norms(self):
        """The sources' omega_s [S] and octant sums [S, 8] (device tensors)."""
        self._sync_stream()
        om = torch.zeros(self.n_src, dtype=torch.float64, device=self.device)
        ow = torch.zeros((self.n_src, 8), dtype=torch.float64, device=self.device)
        if self.n_src:
            rt_source_norms(self.ctx, om, ow)
        return om, ow

    def source_h(self):
        """Smoothing lengths of the sources [S] (device tensor)."""
        self._sync_stream()
        out = torch.zeros(self.n_src, dtype=torch.float64, device=self.device)
        if self.n_src:
            rt_source_fields(self.ctx, out)
        return out

    def set_owned(self, n_owned):
        """Particles [0, n_owned) are owned; rt_energy sums those only (rt_set_owned)."""
        rt_set_owned(self.ctx, n_owned)

    def _stream(self):
        return torch.cuda.current_stream(self.device).cuda_stream

    def _sync_stream(self):
        rt_set_stream(self.ctx, self._stream())

    def rebuild(self, x=None):
        """Neighbour search again (after the particles moved)."""
        if x is not None:
            self.x = _dev(x, torch.float64, self.device)
        self._sync_stream()
        rt_neighbours(self.ctx, self.x, self.m, self.xsrc if self.n_src else None, self.h)

    # -- state helpers ----------------------------------------------------------------
    def state(self, U0):
        """U0 [G, 4, N] (numpy or tensor) -> device tensor in the working precision."""
        return _dev(U0, self.dtype, self.device)

    def luminosities(self, L):
        return None if (L is None or self.n_src == 0) else _dev(L, torch.float64, self.device)

    def alpha(self, a):
        return None if a is None else _dev(a, torch.float64, self.device)

    # -- calls --------------------------------------------------------------------------
    def gradients(self, U):
        self._sync_stream()
        g = torch.empty((self.G, 4, 3, self.n), dtype=self.dtype, device=self.device)
        rt_gradients(self.ctx, U, g)
        return g

    def step(self, U, dt, L=None, alpha=None):
        self._sync_stream()
        rt_transport_step(self.ctx, dt, U, L, alpha)
        return U

    def step_given_gradients(self, U, gradU, dt, alpha=None):
        """Transport and sink of one step with the gradients gradU [G, 4, 3, N] given, in place
        (no injection; rt_transport_step_given_gradients)."""
        self._sync_stream()
        rt_transport_step_given_gradients(self.ctx, dt, U, gradU.contiguous(), alpha)
        return U

    def set_fields(self, first, omega, B):
        """Give omega [k] and B [k, 3, 3] (float64) of particles first, first + 1, ...
        (rt_set_fields)."""
        self._sync_stream()
        om = _dev(omega, torch.float64, self.device)
        b = _dev(B, torch.float64, self.device)
        rt_set_fields(self.ctx, first, om.numel(), om, b)

    def inject(self, U, dt, L=None):
        """The injection stage of one step alone, in place (rt_inject)."""
        self._sync_stream()
        rt_inject(self.ctx, dt, U, L)
        return U

    def subcycle(self, U, n_sub, dt, L=None, alpha=None):
        self._sync_stream()
        rt_subcycle(self.ctx, n_sub, dt, U, L, alpha)
        return U

    def adjoint(self, U0, n_sub, dt, lam_final, L=None, alpha=None, ckpt_every=4):
        """(dLoss/dU0 [G,4,N], dLoss/dL [S,G] or None) for dLoss/dU(final) = lam_final."""
        self._sync_stream()
        lam0 = torch.empty_like(U0)
        dL = torch.empty((self.n_src, self.G), dtype=torch.float64, device=self.device) if (
            L is not None and self.n_src) else None
        rt_adjoint(self.ctx, n_sub, dt, ckpt_every, U0, L, alpha, lam_final, lam0, dL)
        return lam0, dL

    def set_time_bins(self, bins=None, dt_min=1.0, cfl=0.0, max_bin=20, limit=True):
        """Individual time bins (rt_set_time_bins); returns the bins in use [N] (int32 tensor)
        and B.  bins: int array [N] or None for the CFL rule."""
        from . import rt_get_time_bins, rt_set_time_bins
        self._sync_stream()
        b = None if bins is None else _dev(bins, torch.int32, self.device)
        rt_set_time_bins(self.ctx, b, dt_min, cfl, max_bin, limit)
        out = torch.empty(self.n, dtype=torch.int32, device=self.device)
        B = rt_get_time_bins(self.ctx, out)
        return out, B

    def step_bins(self, U, L=None, alpha=None):
        """One hydro step with individual time bins, in place."""
        from . import rt_step_bins
        self._sync_stream()
        rt_step_bins(self.ctx, U, L, alpha)

    def set_absorbers(self, n_species, sigma):
        """Photo-ionisation sink per group (rt_set_absorbers): n_species [J, N] float64
        number densities, sigma [G, J] cross sections; None clears."""
        from . import rt_set_absorbers
        self._sync_stream()
        nd = None if n_species is None else _dev(n_species, torch.float64, self.device)
        rt_set_absorbers(self.ctx, nd, sigma)

    def drift(self, U, v, dt_drift):
        """In place: U += grad U . (v dt_drift) on the current particle set (then call
        rebuild with the moved positions).  v: [3, N] float64 (numpy or tensor)."""
        self._sync_stream()
        rt_drift(self.ctx, U, _dev(v, torch.float64, self.device), dt_drift)

    def energy(self, U):
        self._sync_stream()
        return rt_energy(self.ctx, U, self.G)

    def fields(self):
        self._sync_stream()
        f = {k: torch.empty(self.n, dtype=torch.float64, device=self.device) for k in ("h", "omega", "V")}
        f["B"] = torch.empty((self.n, 3, 3), dtype=torch.float64, device=self.device)
        rt_particle_fields(self.ctx, f["h"], f["omega"], f["V"], f["B"])
        return f

    def pairs(self):
        self._sync_stream()
        d = rt_diagnostics(self.ctx)
        off = torch.empty(self.n + 1, dtype=torch.int64, device=self.device)
        cols = torch.empty(max(d["n_directed"], 1), dtype=torch.int32, device=self.device)
        rt_pairs(self.ctx, off, cols)
        return off, cols[:d["n_directed"]]

    def diagnostics(self):
        self._sync_stream()
        return rt_diagnostics(self.ctx)

    def set_tuning(self, flux_variant=2, gather_variant=1, gradient_variant=2, cell_eighths=0, gradient_block=0,
                   gather_block=0, pair_warps=0):
        rt_set_tuning(self.ctx, flux_variant, gather_variant, gradient_variant, cell_eighths, gradient_block,
                      gather_block, pair_warps)

    def tuning(self):
        return rt_get_tuning(self.ctx)

    def close(self):
        if self.ctx:
            rt_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SubcycleFunction(torch.autograd.Function):
    """U_final = subcycle(U0, L) with gradients w.r.t. U0 and L from the library adjoint."""

    @staticmethod
    def forward(ctx, U0, L, transport: Transport, n_sub: int, dt: float, alpha=None, ckpt_every: int = 4):
        U = U0.detach().clone().contiguous()
        Ld = None if L is None else L.detach().contiguous()
        transport.subcycle(U, n_sub, dt, Ld, alpha)
        ctx.transport = transport
        ctx.args = (n_sub, dt, alpha, ckpt_every)
        ctx.save_for_backward(U0.detach().clone(), Ld if Ld is not None else torch.empty(0))
        ctx.has_L = L is not None
        return U

    @staticmethod
    def backward(ctx, gout):
        U0, L = ctx.saved_tensors
        n_sub, dt, alpha, ckpt_every = ctx.args
        lam0, dL = ctx.transport.adjoint(U0, n_sub, dt, gout.contiguous(), L if ctx.has_L else None, alpha,
                                         ckpt_every)
        return lam0, (dL if ctx.has_L else None), None, None, None, None, None
