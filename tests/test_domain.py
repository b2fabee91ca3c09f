"""Spatial domain decomposition (paper_2302_12727_gb300.domain) on CPU ranks.

World-size 2 and 4 gloo process groups run the decomposition with the FP64 oracle as every
rank's engine (the library itself needs a GPU; tests/test_gpu_domain.py runs it there).  The
decomposed run must reproduce the single-rank oracle run on every particle to 1e-12 (the
ranks sum each neighbour loop over the same neighbours, possibly in another order) and its
energy to 1e-13: owners solve h with complete neighbourhoods, every rank builds with the
owners' h, and the ghosts (two support radii deep) are refreshed before every step
(Part II, "Distributed Memory Parallelism: Domain Decomposition and MPI")."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_2302_12727_gb300 import domain, workloads as W  # noqa: E402


class OracleEngine:
    """One rank's transport computed by the oracle (test stand-in for the library)."""

    def __init__(self, n_groups, c_red, box=(1.0, 1.0, 1.0), periodic=True):
        self.G, self.c_red, self.box, self.periodic = n_groups, c_red, box, periodic
        self.o = None

    def solve(self, x, m, xsrc):
        o = oracle.Oracle(x, m, xsrc if xsrc.shape[1] else None, n_groups=self.G, c_red=self.c_red, box=self.box,
                          periodic=self.periodic)
        if not xsrc.shape[1]:
            return o.h.copy(), np.zeros(0), np.zeros(0), np.zeros((0, 8))
        s = o.sources()
        return o.h.copy(), s.hs.copy(), s.omegas.copy(), s.octw.copy()

    def build(self, x, m, xsrc, h, hs, n_owned, omegas=None, octw=None):
        self.o = oracle.Oracle(x, m, xsrc if xsrc.shape[1] else None, n_groups=self.G, c_red=self.c_red,
                               box=self.box, periodic=self.periodic, h=h, hs=hs, omegas=omegas, octw=octw)
        self.n_owned = n_owned
        self.ns = xsrc.shape[1]

    def state(self, U):
        return torch.from_numpy(np.array(U, dtype=np.float64))

    def alpha(self, a):
        return None if a is None else np.asarray(a, dtype=np.float64)

    def luminosities(self, L):
        return None if L is None else np.asarray(L, dtype=np.float64)

    def inject(self, U, dt, L):
        if self.ns:
            U.copy_(torch.from_numpy(self.o.inject(U.numpy(), dt, L)))

    def fields(self):
        p = self.o.particles()
        return torch.from_numpy(p["omega"].copy()), torch.from_numpy(p["B"].copy())

    def set_fields(self, first, omega, B):
        self.o.set_fields(first, np.asarray(omega), np.asarray(B))

    def gradients(self, U):
        return torch.from_numpy(self.o.gradients(U.numpy()).reshape(self.G, 4, 3, -1).copy())

    def step_given_gradients(self, U, g, dt, alpha):
        Un, _ = self.o.transport_given_gradients(U.numpy(), g.numpy(), dt, alpha)
        U.copy_(torch.from_numpy(Un))

    def step(self, U, dt, L, alpha):
        Un, _ = self.o.run(U.numpy(), 1, dt, L if self.ns else None, alpha)
        U.copy_(torch.from_numpy(Un))

    def energy(self, U):
        k = self.n_owned
        return (self.o.V[:k] * U.numpy()[:, 0, :k]).sum(axis=1)

    def close(self):
        self.o = None


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case(name):
    if name == "lattice-40-walls":
        # non-periodic unit box (walls: truncated supports), two groups, one source
        rng = np.random.default_rng(77)
        x = W.jittered_lattice(40, 0.2, rng)
        n = x.shape[1]
        G = 2
        U0 = np.zeros((G, 4, n))
        U0[:, 0] = 1e-3 * (1 + 0.2 * rng.uniform(-1, 1, size=(G, n)))
        U0[:, 1:] = 0.3 * U0[:, :1] * rng.normal(size=(G, 3, n)) / np.sqrt(3)
        return x, np.full(n, 1.0 / n), np.array([[0.3], [0.6], [0.5]]), U0, np.array([[1.0, 2.0]]), None, G, 1.0, 3
    if name == "lattice-point-source":
        w = W.lattice_point_source()
        return w.x, w.m, w.xsrc, w.U0, w.Lsrc, None, w.n_groups, w.c_red, 4
    if name == "lattice-48-edge":
        # sources just inside one half of the box each: their supports cross the cut between
        # two ranks and reach past the other rank's one-radius halo (the weights of the other
        # rank's targets come from the owners' normalisations)
        x, m, _, U0, Ls, alpha, G, c, nsteps = _case("lattice-48")
        return x, m, np.array([[0.3, 0.7], [0.45, 0.6], [0.53, 0.47]]), U0, Ls, alpha, G, c, nsteps
    if name == "lattice-48-dark":
        # no sources: the gradient-exchange halo is one support radius deep, so the ghosts'
        # own neighbourhoods are cut and their fields and gradients must be their owners'
        x, m, _, U0, _, alpha, G, c, nsteps = _case("lattice-48")
        return x, m, np.zeros((3, 0)), U0, None, alpha, G, c, nsteps
    rng = np.random.default_rng(512)
    x = W.jittered_lattice(48, 0.2, rng)
    n = x.shape[1]
    G = 2
    U0 = np.zeros((G, 4, n))
    U0[:, 0] = 1e-3 * (1 + 0.2 * rng.uniform(-1, 1, size=(G, n)))
    U0[:, 1:] = 0.3 * U0[:, :1] * rng.normal(size=(G, 3, n)) / np.sqrt(3)
    xsrc = np.array([[0.3, 0.8], [0.45, 0.2], [0.5, 0.66]])
    Ls = np.array([[1.0, 0.5], [0.7, 2.0]])
    alpha = rng.uniform(0.0, 2.0, size=n)
    return x, np.full(n, 1.0 / n), xsrc, U0, Ls, alpha, G, 1.0, 3


def _rank_main(rank, ws, port, name, out_path, exchange="state"):
    os.environ["OMP_NUM_THREADS"] = str(max(1, (os.cpu_count() or 2) // ws))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        x, m, xsrc, U0, Ls, alpha, G, c, nsteps = _case(name)
        periodic = name != "lattice-40-walls"
        eng = OracleEngine(G, c, periodic=periodic)
        dt_ = 0.6 * float(np.load(out_path + ".dt.npy"))
        D = domain.DistributedTransport(x, m, xsrc, eng, nb=16 if name == "lattice-point-source" else 32,
                                        periodic=periodic, exchange=exchange)
        U = D.local_state(U0)
        D.subcycle(U, nsteps, dt_, D.local_luminosities(Ls), D.local_alpha(alpha))
        full = D.gather(U)
        E = D.energy(U)
        n_local = len(D.plan.local)
        counts = D._all_sum(np.eye(ws)[rank] * n_local)
        owned = D._all_sum(np.eye(ws)[rank] * D.plan.n_owned)
        if rank == 0:
            np.savez(out_path, U=full, E=E, n_local=counts, owned=owned, reach=D.reach)
        D.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name, ws, exchange", [("lattice-point-source", 2, "state"), ("lattice-48", 2, "state"),
                                                ("lattice-48", 4, "state"), ("lattice-40-walls", 3, "state"),
                                                ("lattice-48", 2, "gradients"), ("lattice-48-dark", 2, "gradients"),
                                                ("lattice-48-edge", 2, "gradients"),
                                                ("lattice-48-dark", 4, "gradients"),
                                                ("lattice-40-walls", 3, "gradients")])
def test_decomposed_oracle_run_equals_single_rank(tmp_path, name, ws, exchange):
    """Both exchange modes: the ghosts' states only (deep halo), or states and gradients
    with the ghosts' omega and B from their owners (the thesis's pattern, shallow halo)."""
    x, m, xsrc, U0, Ls, alpha, G, c, nsteps = _case(name)
    o = oracle.Oracle(x, m, xsrc if xsrc.shape[1] else None, n_groups=G, c_red=c, periodic=name != "lattice-40-walls")
    dxm = ((o.V / (4 * np.pi / 3)) ** (1 / 3)).min()
    out = str(tmp_path / "dd")
    np.save(out + ".dt.npy", np.array(dxm / c))
    ref, _ = o.run(U0, nsteps, 0.6 * dxm / c, Ls, alpha)
    E_ref = o.energy(ref)
    mp.start_processes(_rank_main, args=(ws, _free_port(), name, out, exchange), nprocs=ws, start_method="spawn")
    r = np.load(out + ".npz")
    n = x.shape[1]
    assert r["owned"].sum() == n                       # every particle has exactly one owner
    if name != "lattice-point-source":
        assert r["n_local"].max() < n                  # the halos are proper subsets
    if name == "lattice-48-dark":                      # one support radius of halo, not two
        H = oracle.H_OVER_h * o.h.max()
        assert int(r["reach"]) < domain.reach_blocks(2.0 * H, (1.0, 1.0, 1.0), 32)
    scale = np.abs(ref).reshape(G, -1).max(axis=1)[:, None, None]
    err = np.abs(r["U"] - ref) / (1e-12 * np.abs(ref) + 1e-14 * scale)
    assert err.max() <= 1.0, err.max()
    np.testing.assert_allclose(r["E"], E_ref, rtol=1e-13)


def test_partition_balances_work_and_plans_match():
    """Morton partition: contiguous runs of equal work; the send list of rank r to q equals
    the receive list of q from r (same global particles, same order)."""
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, size=(3, 20000))
    x[0] = x[0] ** 2                                   # uneven density along x
    ws, nb = 4, 8
    owner = domain.partition(x, (1, 1, 1), nb, ws)
    bc = domain.block_of(x, (1, 1, 1), nb)
    pown = owner[(bc[2] * nb + bc[1]) * nb + bc[0]]
    counts = np.bincount(pown, minlength=ws)
    assert counts.max() - counts.min() <= 0.05 * counts.mean() + 1.5 * np.bincount(
        (bc[2] * nb + bc[1]) * nb + bc[0]).max()
    plans = [domain.make_plan(x, (1, 1, 1), True, nb, owner, r, 2) for r in range(ws)]
    for r in range(ws):
        for q, idx in plans[r].send.items():
            g_send = plans[r].local[idx]
            g_recv = plans[q].local[plans[q].recv[r]]
            assert np.array_equal(g_send, g_recv)
        # ghosts are exactly the non-owned particles of the dilated blocks
        assert len(np.intersect1d(plans[r].owned, plans[r].ghosts)) == 0
    assert sum(p.n_owned for p in plans) == x.shape[1]
