"""The spatial domain decomposition with the library as every rank's engine.

Two processes share the one GPU, each with its own context, and exchange their ghosts'
states through gloo on the host between steps (no kernel waits on another process).  The
decomposed run equals a single context's run of the whole set: FP64 to 1e-12 per element
and the energy to 1e-13; FP32 within the FP32 bar against the oracle (relative L1 1e-5 per
component and group after the steps)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_2302_12727_gb300 import Transport, domain  # noqa: E402

from test_domain import _case, _free_port  # noqa: E402
from test_gpu_parity import rel_l1  # noqa: E402

pytestmark = pytest.mark.gpu


def _rank_main(rank, ws, port, name, precision, dt, out_path, exchange="state"):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        torch.cuda.set_device(0)
        x, m, xsrc, U0, Ls, alpha, G, c, nsteps = _case(name)
        eng = domain.CudaEngine(G, c, precision=precision, device=torch.device("cuda", 0))
        D = domain.DistributedTransport(x, m, xsrc, eng, nb=32, exchange=exchange)
        U = D.local_state(U0)
        D.subcycle(U, nsteps, dt, D.local_luminosities(Ls), D.local_alpha(alpha))
        full = D.gather(U)
        E = D.energy(U)
        n_local = D._all_sum(np.eye(ws)[rank] * len(D.plan.local))
        if rank == 0:
            np.savez(out_path, U=full, E=E, n_local=n_local)
        D.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("precision, name, exchange", [("fp64", "lattice-48", "state"),
                                                       ("fp32", "lattice-48", "state"),
                                                       ("fp64", "lattice-48-dark", "gradients"),
                                                       ("fp64", "lattice-48-edge", "gradients"),
                                                       ("fp32", "lattice-48-dark", "gradients")])
def test_decomposed_library_run_equals_single_context(tmp_path, precision, name, exchange):
    """Both exchange modes; the gradient-exchange case has no sources, so its halo is one
    support radius deep and the ghosts' fields and gradients must come from their owners."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    ws = 2
    x, m, xsrc, U0, Ls, alpha, G, c, nsteps = _case(name)
    xs = xsrc if xsrc.shape[1] else None
    o = oracle.Oracle(x, m, xs, n_groups=G, c_red=c)
    dt = 0.6 * ((o.V / (4 * np.pi / 3)) ** (1 / 3)).min() / c
    out = str(tmp_path / "dd")
    mp.start_processes(_rank_main, args=(ws, _free_port(), name, precision, dt, out, exchange), nprocs=ws,
                       start_method="spawn")
    r = np.load(out + ".npz")
    assert r["n_local"].max() < x.shape[1]
    if precision == "fp64":
        t = Transport(x, m, xs, n_groups=G, c_red=c, precision="fp64")
        U = t.state(U0)
        for _ in range(nsteps):
            t.step(U, dt, None if Ls is None else t.luminosities(Ls), t.alpha(alpha))
        ref = U.cpu().numpy()
        E_ref = t.energy(U)
        t.close()
        scale = np.abs(ref).reshape(G, -1).max(axis=1)[:, None, None]
        err = np.abs(r["U"] - ref) / (1e-12 * np.abs(ref) + 1e-14 * scale)
        assert err.max() <= 1.0, err.max()
        np.testing.assert_allclose(r["E"], E_ref, rtol=1e-13)
    else:
        ref, _ = o.run(U0, nsteps, dt, Ls, alpha)
        assert rel_l1(r["U"], ref).max() <= 1e-5
        np.testing.assert_allclose(r["E"], o.energy(ref), rtol=1e-6)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_inject_then_sourceless_step_equals_step(precision):
    """rt_inject, the injection stage alone, against the oracle's (Sec. "Weights For
    Distribution Of Energy Density"), adding L dt per group; followed by rt_transport_step
    without sources it is bitwise rt_transport_step with them (the decomposition exchanges
    ghosts between the two)."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2302_12727_gb300 import RTError
    x, m, xsrc, U0, Ls, alpha, G, c, _ = _case("lattice-48")
    t = Transport(x, m, xsrc, n_groups=G, c_red=c, precision=precision)
    dt = 0.5 * t.diagnostics()["dx_min"] / c
    L, al = t.luminosities(Ls), t.alpha(alpha)
    U1 = t.state(U0)
    t.step(U1, dt, L, al)
    U2 = t.state(U0)
    t.inject(U2, dt, L)
    t.step(U2, dt, None, al)
    assert torch.equal(U1, U2)
    U3 = t.state(U0)
    E0 = np.asarray(t.energy(U3))
    t.inject(U3, dt, L)
    fp64 = precision == "fp64"
    np.testing.assert_allclose(np.asarray(t.energy(U3)) - E0, dt * Ls.sum(0), rtol=1e-12 if fp64 else 1e-5)
    o = oracle.Oracle(x, m, xsrc, n_groups=G, c_red=c)
    ref = o.inject(U0, dt, Ls)
    got = U3.cpu().numpy().astype(np.float64)
    if fp64:
        scale = np.abs(ref).reshape(G, -1).max(axis=1)[:, None, None]
        assert (np.abs(got - ref) <= 1e-12 * np.abs(ref) + 1e-14 * scale).all()
    else:
        assert rel_l1(got, ref).max() <= 1e-6
    U4 = t.state(U0)
    t.inject(U4, dt, None)                 # no luminosities: nothing changes
    assert torch.equal(U4, t.state(U0))
    with pytest.raises(RTError):
        t.inject(U4, -dt, L)
    t.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_step_given_gradients_and_fields(precision):
    """rt_transport_step_given_gradients with rt_gradients' own output is bitwise
    rt_transport_step without sources; rt_set_fields with the context's own omega and B
    changes nothing, and with another omega it changes V to 1 / omega."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2302_12727_gb300 import RTError
    x, m, xsrc, U0, Ls, alpha, G, c, _ = _case("lattice-48")
    t = Transport(x, m, xsrc, n_groups=G, c_red=c, precision=precision)
    dt = 0.5 * t.diagnostics()["dx_min"] / c
    al = t.alpha(alpha)
    U1 = t.state(U0)
    t.step(U1, dt, None, al)
    U2 = t.state(U0)
    t.step_given_gradients(U2, t.gradients(U2), dt, al)
    assert torch.equal(U1, U2)
    f = t.fields()
    n = t.n
    t.set_fields(n // 3, f["omega"][n // 3:], f["B"][n // 3:])
    U3 = t.state(U0)
    t.step(U3, dt, None, al)
    assert torch.equal(U1, U3)
    t.set_fields(5, 2.0 * f["omega"][5:6], f["B"][5:6])
    g = t.fields()
    assert float(g["V"][5]) == 1.0 / (2.0 * float(f["omega"][5]))
    with pytest.raises(RTError):
        t.set_fields(n - 1, f["omega"][:2], f["B"][:2])
    t.close()


def test_given_source_norms_reproduce_the_build():
    """rt_neighbours_given_fields with the normalisations (rt_source_norms) that a build with
    the same given h and h_s forms itself gives bitwise that build's step with sources; the
    normalisations of a build that solved its h are within rounding of them."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    x, m, xsrc, U0, Ls, alpha, G, c, _ = _case("lattice-48")
    for precision in ("fp64", "fp32"):
        a = Transport(x, m, xsrc, n_groups=G, c_red=c, precision=precision)
        h, hs = a.h.clone(), a.source_h()
        b = Transport(x, m, xsrc, n_groups=G, c_red=c, precision=precision, h=h, hs=hs)
        om, ow = b.source_norms()
        assert om.shape == (2,) and ow.shape == (2, 8) and bool((om > 0).all())
        oma, owa = a.source_norms()
        np.testing.assert_allclose(oma.cpu().numpy(), om.cpu().numpy(), rtol=1e-12)
        np.testing.assert_allclose(owa.cpu().numpy(), ow.cpu().numpy(), rtol=1e-12, atol=1e-15)
        d = Transport(x, m, xsrc, n_groups=G, c_red=c, precision=precision, h=h, hs=hs, omegas=om, octw=ow)
        dt = 0.5 * b.diagnostics()["dx_min"] / c
        Ub, Ud = b.state(U0), d.state(U0)
        b.step(Ub, dt, b.luminosities(Ls), b.alpha(alpha))
        d.step(Ud, dt, d.luminosities(Ls), d.alpha(alpha))
        assert torch.equal(Ub, Ud), precision
        for t in (a, b, d):
            t.close()


@pytest.mark.parametrize("exchange", ["state", "gradients"])
def test_bench_decomposed_mode_runs(exchange):
    """bench.py --decompose under torchrun: two ranks split one particle set (gloo backend,
    sharing the one GPU) and print one JSON line whose pair count is the whole set's."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), os.path.join(root, "bench.py"), "--gpus", "2",
           "--decompose", "--backend", "gloo", "--workload", "lattice-sources", "--steps", "2", "--warmup", "1",
           "--exchange", exchange]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=600, cwd=root)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1]
    d = json.loads(line)
    from paper_2302_12727_gb300 import workloads as W
    w = W.lattice_sources()
    o = oracle.Oracle(w.x, w.m, w.xsrc, n_groups=w.n_groups, c_red=w.c_red)
    assert d["config"]["pairs"] == int(o.pairs()[0][-1]) // 2
    assert d["n_gpus"] == 2 and d["value"] > 0 and d["scaling"] == "strong"
    assert d["config"]["exchange"] == exchange and d["config"]["particles_held_over_owned"] >= 1.0
