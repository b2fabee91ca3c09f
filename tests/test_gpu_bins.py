"""Individual time bins (rt_set_time_bins, rt_step_bins; Part II Sec. "Individual
Timstepping", Eq. transport-update-explicit with min(dt_k, dt_l)) against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2302_12727_gb300 import RTError, Transport, workloads as W  # noqa: E402

from test_gpu_parity import fp64_close, rel_l1  # noqa: E402

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def setup(n_side=12, G=2, seed=91):
    rng = np.random.default_rng(seed)
    x = W.jittered_lattice(n_side, 0.25, rng)
    n = x.shape[1]
    xs = np.array([[0.5], [0.5], [0.5]])
    U0 = np.zeros((G, 4, n))
    U0[:, 0] = rng.uniform(0.5, 2.0, size=(G, n))
    U0[:, 1:] = 0.4 * U0[:, :1] * rng.uniform(-1, 1, size=(G, 3, n)) / np.sqrt(3)
    o = oracle.Oracle(x, np.full(n, 1.0 / n), xs, n_groups=G)
    dt = 0.3 * ((o.V / (4 * np.pi / 3)) ** (1 / 3)).min()
    L = rng.uniform(0.5, 1.5, size=(1, G))
    alpha = rng.uniform(0.0, 2.0, size=n)
    return rng, x, xs, U0, o, dt, L, alpha


def test_uniform_bins_equal_uniform_steps():
    """Every bin 0 is one rt_transport_step of dt_min; every bin 1 with dt_min = dt / 2 is one
    step of dt (each exchange is 2 Phi dt_min) -- bitwise, in both precisions."""
    _need_gpu()
    rng, x, xs, U0, o, dt, Ls, a = setup()
    n = x.shape[1]
    for prec in ("fp64", "fp32"):
        t = Transport(x, None, xs, n_groups=2, precision=prec)
        L, al = t.luminosities(Ls), t.alpha(a)
        ref = t.state(U0)
        t.step(ref, dt, L, al)
        b, B = t.set_time_bins(np.zeros(n, np.int32), dt_min=dt)
        assert B == 0 and int(b.max()) == 0
        U = t.state(U0)
        t.step_bins(U, L, al)
        assert torch.equal(U, ref)
        b, B = t.set_time_bins(np.ones(n, np.int32), dt_min=dt / 2)
        assert B == 1
        U = t.state(U0)
        t.step_bins(U, L, al)
        assert torch.equal(U, ref)
        t.close()


def test_mixed_bins_against_oracle():
    """Random bins 0..3, limited to a factor 4 between neighbours: the same bins as the
    oracle's limiter; FP64 state per element and FP32 in relative L1 after one hydro step."""
    _need_gpu()
    rng, x, xs, U0, o, dt, Ls, a = setup()
    n = x.shape[1]
    b0 = rng.integers(0, 4, size=n).astype(np.int32)
    dt_min = dt / 4
    ref, bo, _ = o.step_bins(U0, dt_min, b0, Ls, a)
    assert bo.max() >= 2
    for prec in ("fp64", "fp32"):
        t = Transport(x, None, xs, n_groups=2, precision=prec)
        b, B = t.set_time_bins(b0, dt_min=dt_min)
        np.testing.assert_array_equal(b.cpu().numpy(), bo)
        assert B == int(bo.max())
        U = t.state(U0)
        t.step_bins(U, t.luminosities(Ls), t.alpha(a))
        Ug = U.cpu().numpy().astype(np.float64)
        if prec == "fp64":
            nbad, rmax = fp64_close(Ug, ref)
            assert nbad == 0, rmax
        else:
            assert rel_l1(Ug, ref).max() <= 1e-5
        t.close()


def test_mixed_bins_conserve_energy_and_cfl_bins():
    """Without sources and sinks the min(dt_k, dt_l) exchange keeps sum_i V_i E_i; bins from
    each particle's CFL step (Eq. rt-cfl) equal the oracle's rule followed by its limiter."""
    _need_gpu()
    rng, x, xs, U0, o, dt, Ls, a = setup(seed=92)
    n = x.shape[1]
    b0 = rng.integers(0, 4, size=n).astype(np.int32)
    for prec, tol in (("fp64", 1e-13), ("fp32", 1e-6)):
        t = Transport(x, None, None, n_groups=2, precision=prec)
        t.set_time_bins(b0, dt_min=dt / 4)
        U = t.state(U0)
        E0 = np.array(t.energy(U))
        t.step_bins(U)
        assert np.all(np.abs(np.array(t.energy(U)) - E0) <= tol * E0)
        t.close()
    dx = (o.V / (4 * np.pi / 3)) ** (1 / 3)
    dt_min = 0.9 * dx.min() / 2.7
    ob = o.cfl_bins(0.9, dt_min, 3)
    _, ob_lim, _ = o.step_bins(U0, dt_min, ob, limit=True)
    t = Transport(x, None, xs, n_groups=2, precision="fp32")
    b, B = t.set_time_bins(None, dt_min=dt_min, cfl=0.9, max_bin=3)
    np.testing.assert_array_equal(b.cpu().numpy(), ob_lim)
    t.rebuild()
    with pytest.raises(RTError):
        t.step_bins(t.state(U0))      # rt_neighbours discards the bins
    t.close()


def test_bins_with_hll_and_group_sink():
    """Time bins with the HLL flux against the oracle (FP64 per element); with absorbers of
    equal alpha in every group, bitwise the grey sink's run."""
    _need_gpu()
    rng, x, xs, U0, o, dt, Ls, a = setup(seed=93)
    n = x.shape[1]
    b0 = rng.integers(0, 3, size=n).astype(np.int32)
    oh = oracle.Oracle(x, np.full(n, 1.0 / n), xs, n_groups=2, riemann="hll")
    ref, bo, _ = oh.step_bins(U0, dt / 4, b0, Ls, a)
    t = Transport(x, None, xs, n_groups=2, precision="fp64", riemann="hll")
    t.set_time_bins(b0, dt_min=dt / 4)
    U = t.state(U0)
    t.step_bins(U, t.luminosities(Ls), t.alpha(a))
    nbad, rmax = fp64_close(U.cpu().numpy(), ref)
    assert nbad == 0, rmax
    t.close()
    t = Transport(x, None, xs, n_groups=2, precision="fp32")
    L = t.luminosities(Ls)
    t.set_time_bins(b0, dt_min=dt / 4)
    grey = t.state(U0)
    t.step_bins(grey, L, t.alpha(a))
    t.set_absorbers(a[None, :], np.ones((2, 1)))
    grp = t.state(U0)
    t.step_bins(grp, L)
    assert torch.equal(grp, grey)
    t.close()
