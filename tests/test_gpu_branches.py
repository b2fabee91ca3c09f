"""The non-default branches of the pair flux and the update against the FP64 oracle.

Eq. eddington-group defines the closure for E > 0 and |F| <= cE only.  The readings the
library and the oracle share: the reduced flux is clipped to 1
when |F| > cE, a state with E <= 0 carries no pressure (its energy flux F . A stays), and
the fix-up of the thesis's Riemann-solver and limiter tests (Part III, "Testing Riemann
Solvers and Limiters") sets E < 0 to 0 after the sink and counts the events.  These tests
drive states into every one of those branches on purpose:
  - FP64: every element after three steps within the FP64 bar, and the fix-up count equal
    to the oracle's, with the GLF and the HLL flux;
  - FP32: each step from the oracle's state within relative L1 1e-5 per component and
    group, and the fix-up count equal to the oracle's apart from states whose pre-fix-up E
    lies within float rounding of zero.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2302_12727_gb300 import Transport, workloads as W  # noqa: E402

from test_gpu_parity import cfl_dt, fp64_close, rel_l1  # noqa: E402

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def branch_state(n, G, c, rng):
    """[G, 4, N] with a quarter of the states in each branch: ordinary (f < 1), |F| > cE
    (f from 1.05 to 2), E = 0 with a non-zero flux, E < 0 with a flux."""
    kind = rng.integers(0, 4, size=(G, n))
    E = rng.uniform(0.2, 2.0, size=(G, n))
    E[kind == 2] = 0.0
    E[kind == 3] = -rng.uniform(0.05, 0.5, size=int((kind == 3).sum()))
    f = rng.uniform(0.0, 0.9, size=(G, n))
    f[kind == 1] = rng.uniform(1.05, 2.0, size=int((kind == 1).sum()))
    mag = f * c * np.abs(E)
    mag[kind >= 2] = c * rng.uniform(0.1, 1.0, size=int((kind >= 2).sum()))
    d = rng.normal(size=(G, 3, n))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    U = np.empty((G, 4, n))
    U[:, 0] = E
    U[:, 1:] = mag[:, None, :] * d
    return U, kind


@pytest.fixture(scope="module")
def setup():
    _need_gpu()
    rng = np.random.default_rng(4242)
    x = W.jittered_lattice(12, 0.2, rng)
    n = x.shape[1]
    G, c = 2, 1.0
    U0, kind = branch_state(n, G, c, rng)
    assert all((kind == k).sum() > 100 for k in range(4))
    xs = np.array([[0.3], [0.55], [0.7]])
    Ls = np.array([[0.5, 1.5]])
    alpha = rng.uniform(0.0, 0.5, size=n)
    return x, U0, xs, Ls, alpha, G, c


@pytest.mark.parametrize("riemann", ["glf", "hll"])
def test_closure_and_fixup_branches_fp64(setup, riemann):
    x, U0, xs, Ls, alpha, G, c = setup
    n = x.shape[1]
    o = oracle.Oracle(x, np.full(n, 1.0 / n), xs, n_groups=G, c_red=c, clamp_negative=True, riemann=riemann)
    dt = cfl_dt(o, 0.6)
    t = Transport(x, None, xs, n_groups=G, c_red=c, precision="fp64", clamp_negative=True, riemann=riemann)
    L, al = t.luminosities(Ls), t.alpha(alpha)
    # step by step from the same state: the fix-up count of every step
    Uo = U0.copy()
    Ug = t.state(U0)
    total = 0
    for k in range(3):
        before = t.diagnostics()["clamp_events"]
        t.step(Ug, dt, L, al)
        Uo, nclamp = o.run(Uo, 1, dt, Ls, alpha)
        got = t.diagnostics()["clamp_events"] - before
        assert got == nclamp, (k, got, nclamp)
        total += nclamp
        nbad, rmax = fp64_close(Ug.cpu().numpy(), Uo)
        assert nbad == 0, (k, rmax)
    assert total > 20            # the fix-up branch did run
    # the three steps as one graph-replayed call: same state and count
    V = t.state(U0)
    before = t.diagnostics()["clamp_events"]
    t.subcycle(V, 3, dt, L, al)
    assert t.diagnostics()["clamp_events"] - before == total
    nbad, rmax = fp64_close(V.cpu().numpy(), Uo)
    assert nbad == 0, rmax
    t.close()


def test_closure_branches_without_fixup_fp64(setup):
    """Without the fix-up, negative energies stay and keep feeding the zero-pressure branch;
    the transport still conserves sum V E exactly (no sources, no sink)."""
    x, U0, xs, Ls, alpha, G, c = setup
    n = x.shape[1]
    o = oracle.Oracle(x, np.full(n, 1.0 / n), None, n_groups=G, c_red=c)
    dt = cfl_dt(o, 0.6)
    ref, nclamp = o.run(U0, 3, dt)
    assert nclamp == 0
    t = Transport(x, None, None, n_groups=G, c_red=c, precision="fp64")
    U = t.state(U0)
    t.subcycle(U, 3, dt)
    nbad, rmax = fp64_close(U.cpu().numpy(), ref)
    assert nbad == 0, rmax
    e0, e1 = o.energy(U0), t.energy(U)
    np.testing.assert_allclose(e1, e0, rtol=1e-13, atol=1e-13 * np.abs(U0[:, 0]).sum() / n)
    assert t.diagnostics()["clamp_events"] == 0
    t.close()


def test_closure_and_fixup_branches_fp32(setup):
    x, U0, xs, Ls, alpha, G, c = setup
    n = x.shape[1]
    o = oracle.Oracle(x, np.full(n, 1.0 / n), xs, n_groups=G, c_red=c, clamp_negative=True)
    o_free = oracle.Oracle(x, np.full(n, 1.0 / n), xs, n_groups=G, c_red=c)
    dt = cfl_dt(o, 0.6)
    t = Transport(x, None, xs, n_groups=G, c_red=c, precision="fp32", clamp_negative=True)
    L, al = t.luminosities(Ls), t.alpha(alpha)
    Uo = U0.copy()
    total = 0
    for k in range(3):
        Ug = t.state(Uo)
        before = t.diagnostics()["clamp_events"]
        t.step(Ug, dt, L, al)
        got = t.diagnostics()["clamp_events"] - before
        pre, _ = o_free.run(Uo, 1, dt, Ls, alpha)       # E before the fix-up
        Uo, nclamp = o.run(Uo, 1, dt, Ls, alpha)
        err = rel_l1(Ug.cpu().numpy().astype(np.float64), Uo)
        nz = np.abs(Uo.reshape(-1, n)).sum(1) > 0
        assert err[nz].max() <= 1e-5, (k, err)
        # states whose E before the fix-up is within float rounding of zero may go either way
        scale = np.abs(pre[:, 0]).max(axis=1, keepdims=True)
        ambiguous = int((np.abs(pre[:, 0]) < 1e-6 * scale).sum())
        assert abs(got - nclamp) <= ambiguous, (k, got, nclamp, ambiguous)
        total += nclamp
    assert total > 20
    t.close()
