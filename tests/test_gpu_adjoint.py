"""Hand-written adjoint (rt_adjoint) against the oracle's exact directional derivatives
(forward-mode dual numbers), finite differences, and the degree-1 homogeneity of the step.

Loss (the reading for the multi-source lattice): L = sum over groups and over particles within 0.15 of the box
centre of E, so dL/dU(final) is that indicator on the E rows.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2302_12727_gb300 import SubcycleFunction, Transport, workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def loss_weights(w):
    d = w.x - 0.5
    d -= np.rint(d)
    inside = np.sqrt((d ** 2).sum(0)) < 0.15
    wt = np.zeros((w.n_groups, 4, w.n))
    wt[:, 0, inside] = 1.0
    return wt


def setup(n_side=16, alpha=True):
    w = W.lattice_sources(n_side)
    o = oracle.Oracle(w.x, w.m, w.xsrc, n_groups=w.n_groups, c_red=w.c_red)
    dt = 0.6 * ((o.V / (4 * np.pi / 3)) ** (1 / 3)).min() / w.c_red
    a = 0.3 * w.m * o.omega if alpha else None    # grey alpha = kappa rho, rho = m omega ~ 1
    return w, o, dt, a


def gpu_adjoint(w, dt, a, n_sub, ckpt, precision="fp64", U0=None):
    t = Transport(w.x, w.m, w.xsrc, n_groups=w.n_groups, precision=precision, c_red=w.c_red)
    U0 = t.state(w.U0 if U0 is None else U0)
    L = t.luminosities(w.Lsrc)
    al = t.alpha(a)
    lam = t.state(loss_weights(w))
    dU0, dL = t.adjoint(U0, n_sub, dt, lam, L, al, ckpt)
    Uf = U0.clone()
    t.subcycle(Uf, n_sub, dt, L, al)
    out = dU0.double().cpu().numpy(), dL.cpu().numpy(), Uf.double().cpu().numpy()
    t.close()
    return out


def test_adjoint_matches_exact_directional_derivative():
    """<dL/dU0, v> + <dL/dLsrc, vL> equals the oracle's dual-number JVP along (v, vL)."""
    _need_gpu()
    w, o, dt, a = setup(16)
    n_sub = 6
    dU0, dL, _ = gpu_adjoint(w, dt, a, n_sub, 4)
    rng = np.random.default_rng(5)
    wt = loss_weights(w)
    for _ in range(3):
        v = rng.normal(size=w.U0.shape) * np.abs(w.U0).max()
        vL = rng.normal(size=w.Lsrc.shape)
        _, dUf = o.jvp(w.U0, v, n_sub, dt, w.Lsrc, vL, a)
        exact = (wt * dUf).sum()
        adj = (dU0 * v).sum() + (dL * vL).sum()
        assert adj == pytest.approx(exact, rel=1e-9, abs=1e-12 * abs(exact))


def test_adjoint_homogeneity():
    """Without the fix-up the final state is degree-1 homogeneous in (U0, L):
    sum_s L_s dL/dL_s + <U0, dL/dU0> = L(final)."""
    _need_gpu()
    w, o, dt, a = setup(16)
    n_sub = 5
    dU0, dL, Uf = gpu_adjoint(w, dt, a, n_sub, 2)
    lhs = (dU0 * w.U0).sum() + (dL * w.Lsrc).sum()
    loss = (loss_weights(w) * Uf).sum()
    assert lhs == pytest.approx(loss, rel=1e-10)


def test_checkpoint_interval_does_not_change_the_result():
    _need_gpu()
    w, o, dt, a = setup(12)
    r1 = gpu_adjoint(w, dt, a, 7, 1)
    r3 = gpu_adjoint(w, dt, a, 7, 3)
    r7 = gpu_adjoint(w, dt, a, 7, 7)
    for x, y in ((r1, r3), (r1, r7)):
        np.testing.assert_array_equal(x[0], y[0])
        np.testing.assert_array_equal(x[1], y[1])


def test_lattice_sources_finite_differences_and_fp32():
    """The multi-source lattice (32^3, 2 groups, 8 sources, 16 sub-cycles, checkpoint every
    4): central differences with a 1e-6 relative step on the FP64 path, and the FP32
    adjoint.  The initial state is the workload's scaled by 1e10 (E0 of order one, same pattern), so that a
    1e-6 relative step of U0 moves the loss well above double-precision resolution."""
    _need_gpu()
    w, o, dt, _ = setup(32, alpha=False)
    n_sub, ck = w.n_steps, w.ckpt_every
    U0 = w.U0 * 1e10
    dU0, dL, _ = gpu_adjoint(w, dt, None, n_sub, ck, U0=U0)
    wt = loss_weights(w)
    rng = np.random.default_rng(9)
    t = Transport(w.x, w.m, w.xsrc, n_groups=w.n_groups, precision="fp64", c_red=w.c_red)
    L0 = w.Lsrc
    for kind in ("L", "U"):
        if kind == "L":
            vU, vL = np.zeros_like(U0), rng.normal(size=L0.shape) * L0
        else:
            vU, vL = rng.normal(size=U0.shape) * U0, np.zeros_like(L0)
        adj = (dU0 * vU).sum() + (dL * vL).sum()
        errs = {}
        for eps in (1e-6, 1e-7, 1e-8):
            vals = []
            for sgn in (1, -1):
                U = t.state(U0 + sgn * eps * vU)
                t.subcycle(U, n_sub, dt, t.luminosities(L0 + sgn * eps * vL))
                vals.append((wt * U.cpu().numpy()).sum())
            fd = (vals[0] - vals[1]) / (2 * eps)
            errs[eps] = abs(adj - fd) / abs(fd)
        print(kind, errs)
        # ~1e8 minmod evaluations: a 1e-6 stencil crosses some of their kinks, so the
        # agreement improves as the stencil shrinks until rounding takes over
        assert errs[1e-6] <= 2e-3, (kind, errs)
        assert min(errs.values()) <= 2e-6, (kind, errs)
    t.close()
    dU32, dL32, _ = gpu_adjoint(w, dt, None, n_sub, ck, precision="fp32", U0=U0)
    assert np.linalg.norm(dL32 - dL) <= 1e-4 * np.linalg.norm(dL)
    assert np.linalg.norm(dU32 - dU0) <= 1e-4 * np.linalg.norm(dU0)


def test_autograd_function_uses_the_adjoint():
    _need_gpu()
    w, o, dt, a = setup(12)
    t = Transport(w.x, w.m, w.xsrc, n_groups=w.n_groups, precision="fp64", c_red=w.c_red)
    U0 = t.state(w.U0).requires_grad_(True)
    L = t.luminosities(w.Lsrc).requires_grad_(True)
    al = t.alpha(a)
    wt = t.state(loss_weights(w))
    Uf = SubcycleFunction.apply(U0, L, t, 4, dt, al, 2)
    (wt * Uf).sum().backward()
    dU0, dL = t.adjoint(U0.detach(), 4, dt, wt, L.detach(), al, 2)
    assert torch.equal(U0.grad, dU0) and torch.equal(L.grad, dL)
    t.close()
