"""Photo-ionisation sink per photon group (rt_set_absorbers; Eqs. dEdt-group, dFdt-group)
against the oracle: absorption alpha_g = sum_j sigma^N_gj n_j from blackbody-averaged cross
sections of the thesis's fits, on the benchmark's shape (Poisson sine density, 3 groups split at the H0, He0 and He+
thresholds, source and collimated beam)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import photo  # noqa: E402
from paper_2302_12727_gb300 import RTError, Transport, workloads as W  # noqa: E402

from test_gpu_parity import cfl_dt, fp64_close, rel_l1  # noqa: E402

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def absorbers(w, o):
    """Species densities (code units) tracing the density with an ionised fraction that
    varies along x, and the three groups' sigma^N scaled so that H0 in group 1 gives
    alpha = 0.1 rho (the grey kappa of the benchmark workload)."""
    rho = w.m * o.omega
    xi = 0.5 * (1 + np.sin(2 * np.pi * w.x[0]))
    n = np.stack([rho * (1 - xi), 0.08 * rho * (1 - xi), 0.08 * rho * xi])
    edges = [photo.E_ION[s] * photo.EV / photo.H_PLANCK for s in photo.SPECIES] + [math.inf]
    _, sN, _ = photo.group_averages(1e5, edges)
    sig = 0.1 * sN / sN[0, 0]
    return n, sig


def test_group_sink_against_oracle():
    _need_gpu()
    w = W.poisson_sine_beam(24)
    o = oracle.Oracle(w.x, w.m, w.xsrc, n_groups=w.n_groups, c_red=w.c_red)
    dt = cfl_dt(o)
    n, sig = absorbers(w, o)
    ag = photo.absorption(n, sig)
    ref, _ = o.run(w.U0, 5, dt, w.Lsrc, alpha_groups=ag)
    for prec in ("fp64", "fp32"):
        t = Transport(w.x, w.m, w.xsrc, n_groups=w.n_groups, precision=prec, c_red=w.c_red)
        t.set_absorbers(n, sig)
        L = t.luminosities(w.Lsrc)
        if prec == "fp64":
            Uo = w.U0.copy()
            for k in range(5):
                U = t.state(Uo)
                t.step(U, dt, L)
                Uo, _ = o.run(Uo, 1, dt, w.Lsrc, alpha_groups=ag)
                nbad, rmax = fp64_close(U.cpu().numpy(), Uo)
                assert nbad == 0, (k, rmax)
        else:
            U = t.state(w.U0)
            t.subcycle(U, 5, dt, L)
            # five steps of the per-step FP32 bar (1e-5 each)
            assert rel_l1(U.cpu().numpy().astype(np.float64), ref).max() <= 5e-5
        # the adjoint covers the grey sink only
        with pytest.raises(RTError):
            t.adjoint(t.state(w.U0), 2, dt, t.state(w.U0))
        t.close()


def test_equal_group_absorption_is_the_grey_sink_and_clearing_restores_none():
    """alpha_g equal in every group gives bitwise the grey run; a grey alpha given to the
    call overrides the absorbers; clearing them removes the sink."""
    _need_gpu()
    w = W.poisson_sine_beam(16)
    o = oracle.Oracle(w.x, w.m, w.xsrc, n_groups=w.n_groups, c_red=w.c_red)
    dt = cfl_dt(o)
    a = w.kappa * w.m * o.omega
    t = Transport(w.x, w.m, w.xsrc, n_groups=w.n_groups, precision="fp32", c_red=w.c_red)
    L = t.luminosities(w.Lsrc)
    grey = t.state(w.U0)
    t.subcycle(grey, 4, dt, L, t.alpha(a))
    none = t.state(w.U0)
    t.subcycle(none, 4, dt, L)
    t.set_absorbers(a[None, :], np.ones((w.n_groups, 1)))
    grp = t.state(w.U0)
    t.subcycle(grp, 4, dt, L)
    assert torch.equal(grp, grey)
    over = t.state(w.U0)
    t.subcycle(over, 4, dt, L, t.alpha(0.5 * a))
    ref_half = t.state(w.U0)
    t.set_absorbers(None, None)
    t.subcycle(ref_half, 4, dt, L, t.alpha(0.5 * a))
    assert torch.equal(over, ref_half)
    cleared = t.state(w.U0)
    t.subcycle(cleared, 4, dt, L)
    assert torch.equal(cleared, none)
    t.close()
