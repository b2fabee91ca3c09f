"""Spatial domain decomposition of the transport path over ranks (one GPU per rank).

The thesis distributes SWIFT's cells over MPI ranks by the work they hold and refreshes the
"foreign" cells (copies of cells another rank owns) by send/recv tasks before every
interaction loop that reads them (Part II, Sec. "Distributed Memory Parallelism: Domain
Decomposition and MPI"; Part III, Sec. "Implementation in SWIFT", the RT send/recv tasks).
Here a rank runs the library on its own particles plus ghost copies of the particles around
its domain, and only the ghosts' data crosses ranks:

  partition   the box is cut into nb^3 blocks, the blocks are ordered along a Morton curve,
              and the curve is cut into one contiguous piece of equal work per rank (work per
              particle: its pair count when known, else 1);
  halo        a rank's ghosts are the particles of every block within `reach` blocks (per
              axis) of one of its own blocks;
  hydro step  (once per particle configuration)
              1. each rank solves h for its own particles, and h_s, omega_s and the octant
                 sums for the sources inside its blocks, with ghosts out to the largest
                 support radius;
              2. the owners send h to the ranks holding the particles as ghosts, and every
                 rank learns every source's h_s, omega_s and octant sums (sums over ranks);
              3. each rank builds its lists, geometry and injection weights with all of them
                 given (rt_neighbours_given_fields), on ghosts out to D = 2 H_max, with the
                 sources within H_s,max of its blocks;
  sub-cycle   every rank injects its sources' energy (rt_inject), the owners send the
              ghosts' injected states (U), then every rank runs the rest of the step
              (rt_transport_step without sources: gradients, fluxes, update, sink) on its own
              particles and ghosts; the energy is summed over owned particles in double and
              over ranks by an all-reduce.

Why D = 2 H_max reproduces the single-rank result on every owned particle.  Injection: an
owned particle receives energy from sources within H_s,max, whose weights depend on their
gas only through omega_s and the octant sums, which come from the sources' owners; the
target's volume is its own.  Transport: an owned particle's pairs reach at most H_max, so its partners j lie
within H_max of the domain; the flux of (i, j) needs grad U_j and B_j, i.e. j's own pair list
and the states of j's neighbours, all within 2 H_max, and those states are the owners'
injected states, refreshed after the injection.  Every h is the owner's, so every rank
decides each pair with the same two smoothing lengths.  The ghosts' own results are
discarded: the next refresh overwrites them.  Unlike the thesis's scheme, gradients are not
exchanged: the ghosts within H_max of the domain compute them (the halo is one H_max deeper),
so a sub-cycle has one exchange instead of two.

exchange="gradients" follows the thesis's pattern instead: the ghosts are only H_max deep,
their omega and B come from their
owners once per build (rt_set_fields), and each sub-cycle exchanges U, then the gradients
(rt_gradients on every rank, the ghosts' rows replaced by their owners'), then runs the
transport with those gradients (rt_transport_step_given_gradients).  An owned particle's
pairs, its partners' states, gradients, omega, V, B and h are then all the owners' values.

The exchanges are grouped point-to-point sends and receives (torch.distributed: NCCL between
GPUs, gloo between CPU ranks); the energy all-reduce is in float64.  A rank's engine is the
library (``CudaEngine``); the tests drive the same decomposition with the FP64 oracle as the
engine on CPU ranks.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

H_OVER_h = 1.825742


# ---------------------------------------------------------------------------------------
# partition and halo (pure numpy: every rank computes the same plan from the same inputs)
def _spread3(v: np.ndarray) -> np.ndarray:
    """Interleave the bits of v (< 2^21) with two zero bits each."""
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def morton_keys(ix, iy, iz) -> np.ndarray:
    return _spread3(ix) | (_spread3(iy) << np.uint64(1)) | (_spread3(iz) << np.uint64(2))


def block_of(x: np.ndarray, box, nb: int) -> np.ndarray:
    """[3, N] block coordinates of the particles (blocks of box/nb per axis)."""
    b = np.floor(x / np.asarray(box, dtype=np.float64)[:, None] * nb).astype(np.int64)
    return np.clip(b, 0, nb - 1)


def partition(x: np.ndarray, box, nb: int, n_ranks: int, work: np.ndarray | None = None) -> np.ndarray:
    """Owner rank of every block ([nb^3], flat index (bz * nb + by) * nb + bx): the blocks in
    Morton order, cut into n_ranks contiguous runs of equal work."""
    bc = block_of(x, box, nb)
    flat = (bc[2] * nb + bc[1]) * nb + bc[0]
    w = np.ones(x.shape[1]) if work is None else np.asarray(work, dtype=np.float64)
    bwork = np.bincount(flat, weights=w, minlength=nb ** 3)
    g = np.arange(nb)
    bz, by, bx = np.meshgrid(g, g, g, indexing="ij")
    keys = morton_keys(bx.ravel(), by.ravel(), bz.ravel())
    order = np.argsort(keys, kind="stable")
    cum = np.cumsum(bwork[order])
    total = cum[-1] if len(cum) else 0.0
    # block k of the curve goes to the rank whose share contains the middle of its work
    mid = cum - 0.5 * bwork[order]
    rank_of_curve = np.minimum((mid / max(total, 1e-300) * n_ranks).astype(np.int64), n_ranks - 1)
    owner = np.empty(nb ** 3, dtype=np.int64)
    owner[order] = rank_of_curve
    return owner


def dilate(mask: np.ndarray, nb: int, reach: int, periodic: bool) -> np.ndarray:
    """Blocks within `reach` blocks per axis of a block of mask ([nb^3] bool)."""
    m = mask.reshape(nb, nb, nb)
    out = m.copy()
    r = min(reach, nb)
    for axis in range(3):
        cur = out.copy()
        for s in range(1, r + 1):
            if periodic:
                cur |= np.roll(out, s, axis) | np.roll(out, -s, axis)
            else:
                lo = [slice(None)] * 3
                hi = [slice(None)] * 3
                lo[axis], hi[axis] = slice(s, None), slice(None, -s)
                sh = np.zeros_like(out)
                sh[tuple(lo)] = out[tuple(hi)]
                cur |= sh
                sh = np.zeros_like(out)
                sh[tuple(hi)] = out[tuple(lo)]
                cur |= sh
        out = cur
    return out.ravel()


@dataclass
class Plan:
    """Which particles a rank holds and what it exchanges.  Local order: owned particles
    (ascending global index), then ghosts (ascending global index)."""
    rank: int
    n_ranks: int
    owned: np.ndarray                     # global indices
    ghosts: np.ndarray                    # global indices
    send: dict = field(default_factory=dict)   # q -> local indices of owned particles that q holds as ghosts
    recv: dict = field(default_factory=dict)   # q -> local indices of ghosts that q owns

    @property
    def local(self) -> np.ndarray:
        return np.concatenate([self.owned, self.ghosts])

    @property
    def n_owned(self) -> int:
        return len(self.owned)


def make_plan(x: np.ndarray, box, periodic: bool, nb: int, block_owner: np.ndarray, rank: int, reach: int) -> Plan:
    """The holdings and exchange lists of `rank` (and implicitly of every other rank: all
    ranks derive the same lists from the same inputs, so no lists are communicated)."""
    n_ranks = int(block_owner.max()) + 1 if len(block_owner) else 1
    bc = block_of(x, box, nb)
    flat = (bc[2] * nb + bc[1]) * nb + bc[0]
    pown = block_owner[flat]

    def ghost_mask(r):
        held = dilate(block_owner == r, nb, reach, periodic)
        return held[flat] & (pown != r)

    owned = np.flatnonzero(pown == rank)
    gm = ghost_mask(rank)
    ghosts = np.flatnonzero(gm)
    local = np.concatenate([owned, ghosts])
    loc = np.full(x.shape[1], -1, dtype=np.int64)
    loc[local] = np.arange(len(local))
    plan = Plan(rank, n_ranks, owned, ghosts)
    for q in range(n_ranks):
        if q == rank:
            continue
        gq = ghost_mask(q)
        s = np.flatnonzero(gq & (pown == rank))      # mine, held by q
        r = np.flatnonzero(gm & (pown == q))         # q's, held by me
        if len(s):
            plan.send[q] = loc[s]
        if len(r):
            plan.recv[q] = loc[r]
    return plan


def reach_blocks(dist: float, box, nb: int) -> int:
    return int(math.ceil(dist / (min(box) / nb) - 1e-12))


def source_mask(xsrc: np.ndarray, box, periodic: bool, nb: int, block_owner: np.ndarray, rank: int,
                reach: int) -> np.ndarray:
    """Sources whose block lies within `reach` blocks of one of rank's blocks."""
    if xsrc.shape[1] == 0:
        return np.zeros(0, dtype=bool)
    near = dilate(block_owner == rank, nb, reach, periodic)
    bc = block_of(xsrc, box, nb)
    return near[(bc[2] * nb + bc[1]) * nb + bc[0]]


# ---------------------------------------------------------------------------------------
# exchange
def exchange(t, plan: Plan, group=None):
    """Ghost refresh of t [..., n_local] (torch tensor, last axis = local particle): the
    owners' values of plan.send go out, plan.recv's come in, as one group of point-to-point
    operations."""
    import torch
    import torch.distributed as dist
    if t.is_cuda and dist.get_backend(group) == "gloo":
        # gloo moves host memory only: stage the device tensor through the host
        h = t.cpu()
        exchange(h, plan, group)
        t.copy_(h)
        return t
    ops, bufs = [], []
    for q, idx in sorted(plan.send.items()):
        buf = t.index_select(-1, torch.as_tensor(idx, device=t.device)).contiguous()
        ops.append(dist.P2POp(dist.isend, buf, q, group))
    for q, idx in sorted(plan.recv.items()):
        buf = torch.empty(t.shape[:-1] + (len(idx),), dtype=t.dtype, device=t.device)
        bufs.append((idx, buf))
        ops.append(dist.P2POp(dist.irecv, buf, q, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for idx, buf in bufs:
        t[..., torch.as_tensor(idx, device=t.device)] = buf
    return t


# ---------------------------------------------------------------------------------------
# engines: one rank's transport
class CudaEngine:
    """The library on one rank (a Transport per particle configuration)."""

    def __init__(self, n_groups, c_red, precision="fp64", device=None, riemann="glf", box=(1.0, 1.0, 1.0),
                 periodic=True):
        import torch
        self.G, self.c_red, self.precision, self.riemann = n_groups, c_red, precision, riemann
        self.box, self.periodic = tuple(box), periodic
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.t = None

    def _new(self, x, m, xsrc, h=None, hs=None, omegas=None, octw=None):
        from .transport import Transport
        if self.t is not None:
            self.t.close()
        self.t = Transport(x, m, xsrc if xsrc.shape[1] else None, n_groups=self.G, c_red=self.c_red,
                           precision=self.precision, device=self.device, riemann=self.riemann, box=self.box,
                           periodic=self.periodic, h=h, hs=hs, omegas=omegas, octw=octw)

    def solve(self, x, m, xsrc):
        """Solve h (and h_s); returns h [N], hs [S] and the sources' omega_s [S] and octant
        sums [S, 8] as float64 numpy arrays."""
        self._new(x, m, xsrc)
        om, ow = self.t.source_norms()
        return self.t.h.cpu().numpy(), self.t.source_h().cpu().numpy(), om.cpu().numpy(), ow.cpu().numpy()

    def build(self, x, m, xsrc, h, hs, n_owned, omegas=None, octw=None):
        self._new(x, m, xsrc, h=h, hs=hs, omegas=omegas, octw=octw)
        self.t.set_owned(n_owned)

    def state(self, U):
        return self.t.state(U)

    def alpha(self, a):
        return None if a is None else self.t.alpha(a)

    def luminosities(self, L):
        return self.t.luminosities(L)

    def inject(self, U, dt, L):
        self.t.inject(U, dt, L)

    def fields(self):
        f = self.t.fields()
        return f["omega"], f["B"]

    def set_fields(self, first, omega, B):
        self.t.set_fields(first, omega, B)

    def gradients(self, U):
        return self.t.gradients(U)

    def step_given_gradients(self, U, g, dt, alpha):
        self.t.step_given_gradients(U, g, dt, alpha)

    def step(self, U, dt, L, alpha):
        self.t.step(U, dt, L, alpha)

    def energy(self, U):
        return np.asarray(self.t.energy(U), dtype=np.float64)

    def pair_counts(self):
        off, _ = self.t.pairs()
        return np.diff(off.cpu().numpy())

    def close(self):
        if self.t is not None:
            self.t.close()
            self.t = None


# ---------------------------------------------------------------------------------------
class DistributedTransport:
    """The transport of one particle set decomposed over the ranks of a process group.

    x [3, N], m [N], xsrc [3, S] are the whole set on every rank (a rank keeps what its plan
    holds).  ``engine`` runs one rank's share; ``nb`` is the number of partition blocks per
    axis (a power of two).  ``exchange`` chooses what crosses ranks in a sub-cycle: "state"
    (the ghosts' U only, with ghosts 2 H_max deep) or "gradients" (U, then the
    ghosts' gradients, with ghosts H_max deep and their omega and B taken
    from their owners once per build)."""

    def __init__(self, x, m, xsrc, engine, *, box=(1.0, 1.0, 1.0), periodic=True, nb=32, group=None,
                 work=None, eta_res=1.2348, exchange="state"):
        if exchange not in ("state", "gradients"):
            raise ValueError("exchange must be 'state' or 'gradients'")
        self.exchange_mode = exchange
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.n_ranks = dist.get_world_size(group)
        self.x = np.ascontiguousarray(x, dtype=np.float64)
        self.m = np.ascontiguousarray(m, dtype=np.float64)
        self.xsrc = np.zeros((3, 0)) if xsrc is None else np.ascontiguousarray(xsrc, dtype=np.float64)
        self.box, self.periodic, self.nb = tuple(box), periodic, nb
        self.engine = engine
        n = self.x.shape[1]
        self.block_owner = partition(self.x, box, nb, self.n_ranks, work)
        bc = block_of(self.x, box, nb)
        self.p_owner = self.block_owner[(bc[2] * nb + bc[1]) * nb + bc[0]]
        # 1. h of the owned particles and h_s of the sources in owned blocks, with ghosts out
        #    to the largest support radius (grown until it covers every owned support)
        vol = box[0] * box[1] * box[2]
        depth = 2.0 * H_OVER_h * eta_res * (vol / n) ** (1.0 / 3.0)
        s_own = source_mask(self.xsrc, box, periodic, nb, self.block_owner, self.rank, 0)
        while True:
            reach = reach_blocks(depth, box, nb)
            plan = make_plan(self.x, box, periodic, nb, self.block_owner, self.rank, reach)
            loc = plan.local
            h, hs, oms, octw = engine.solve(self.x[:, loc], self.m[loc], self.xsrc[:, s_own])
            H_need = H_OVER_h * max(h[:plan.n_owned].max(initial=0.0), hs.max(initial=0.0))
            ok = self._all_min(float(H_need <= reach * min(box) / nb))
            if ok > 0.5 or reach >= nb:
                break
            depth = 1.5 * max(depth, self._all_max(H_need))
        self.h = np.zeros(n)
        self.h[plan.owned] = h[:plan.n_owned]
        S = self.xsrc.shape[1]
        self.hs = np.zeros(S)
        self.hs[s_own] = hs
        self.hs = self._all_sum(self.hs)
        # each source's normalisation (omega_s, octant sums) from its owner, whose gas
        # neighbourhood is complete: no rank needs a gas halo for the injection
        self.oms = np.zeros(S)
        self.oms[s_own] = oms
        self.oms = self._all_sum(self.oms)
        self.octw = np.zeros((S, 8))
        self.octw[s_own] = np.asarray(octw).reshape(-1, 8)
        self.octw = self._all_sum(self.octw.reshape(-1)).reshape(S, 8)
        self.H_max = H_OVER_h * self._all_max(float(self.h[plan.owned].max(initial=0.0)))
        self.Hs_max = H_OVER_h * float(self.hs.max(initial=0.0))
        # 2.-3. the halo of the transport and the build with every h given: the transport
        #    needs 2 H_max (H_max when the ghosts' gradients and fields come from their
        #    owners); the injection into owned particles needs the sources within H_s,max,
        #    with their owners' normalisations, and no gas beyond the owned particles
        self.depth = self.H_max if exchange == "gradients" else 2.0 * self.H_max
        reach_src = reach_blocks(self.Hs_max, box, nb)
        reach = reach_blocks(self.depth, box, nb)
        self.plan = make_plan(self.x, box, periodic, nb, self.block_owner, self.rank, reach)
        self.reach = reach
        self._exchange_owned_h()
        self.src_mask = source_mask(self.xsrc, box, periodic, nb, self.block_owner, self.rank, reach_src)
        loc = self.plan.local
        engine.build(self.x[:, loc], self.m[loc], self.xsrc[:, self.src_mask], self.h[loc],
                     self.hs[self.src_mask], self.plan.n_owned, self.oms[self.src_mask], self.octw[self.src_mask])
        if exchange == "gradients":
            self._exchange_fields()

    # collectives on host scalars / arrays (float64)
    def _tensor(self, v):
        import torch
        dev = "cpu" if self.dist.get_backend(self.group) == "gloo" else getattr(self.engine, "device", "cpu")
        return torch.as_tensor(np.asarray(v, dtype=np.float64), device=dev).clone()

    def _all(self, v, op):
        t = self._tensor(v)
        self.dist.all_reduce(t, op=op, group=self.group)
        return t.cpu().numpy()

    def _all_sum(self, v):
        return self._all(v, self.dist.ReduceOp.SUM)

    def _all_max(self, v):
        return float(self._all([v], self.dist.ReduceOp.MAX)[0])

    def _all_min(self, v):
        return float(self._all([v], self.dist.ReduceOp.MIN)[0])

    def _exchange_owned_h(self):
        """Owners send h; every rank then holds h for all its local particles."""
        import torch
        loc = self.plan.local
        hl = torch.as_tensor(np.where(np.arange(len(loc)) < self.plan.n_owned, self.h[loc], 0.0))
        hl = hl.to(self._tensor(0.0).device)
        exchange(hl, self.plan, self.group)
        self.h[loc] = hl.cpu().numpy()

    def _exchange_fields(self):
        """Owners send omega and B; the ghosts take them (their own neighbourhoods are cut
        by the halo)."""
        import torch
        om, B = self.engine.fields()
        k = self.plan.n_owned
        fb = torch.cat([om.reshape(1, -1), B.reshape(-1, 9).T], dim=0).to(torch.float64).contiguous()
        if self.dist.get_backend(self.group) == "gloo" and fb.is_cuda:
            fb = fb.cpu()
        exchange(fb, self.plan, self.group)
        n_loc = fb.shape[1]
        if n_loc > k:
            self.engine.set_fields(k, fb[0, k:].contiguous(), fb[1:, k:].T.reshape(-1, 3, 3).contiguous())

    # ----- state
    def local_state(self, U_global):
        """This rank's [G, 4, n_local] share of a global [G, 4, N] state, in the engine's type."""
        return self.engine.state(np.ascontiguousarray(U_global[..., self.plan.local]))

    def local_alpha(self, alpha_global):
        return None if alpha_global is None else self.engine.alpha(alpha_global[self.plan.local])

    def local_luminosities(self, L_global):
        if L_global is None or self.xsrc.shape[1] == 0 or not self.src_mask.any():
            return None
        return self.engine.luminosities(np.ascontiguousarray(np.asarray(L_global)[self.src_mask]))

    def subcycle(self, U, n_sub, dt, L=None, alpha=None):
        """n_sub transport steps of the local state U (in place): the injection, the ghost
        refresh (carrying the owners' injected states), then the rest of the step; with
        exchange="gradients" the ghosts' gradients are refreshed from their owners before the
        transport, as the thesis's RT gradient send/recv tasks do."""
        for _ in range(n_sub):
            if L is not None:
                self.engine.inject(U, dt, L)
            exchange(U, self.plan, self.group)
            if self.exchange_mode == "gradients":
                g = self.engine.gradients(U)
                exchange(g, self.plan, self.group)
                self.engine.step_given_gradients(U, g, dt, alpha)
            else:
                self.engine.step(U, dt, None, alpha)
        return U

    def energy(self, U):
        """sum_i V_i E_i,g over all owned particles of all ranks (float64)."""
        return self._all_sum(self.engine.energy(U))

    def gather(self, U):
        """The global [G, 4, N] state assembled from every rank's owned particles (float64)."""
        own = U[..., :self.plan.n_owned]
        own = own.detach().cpu().numpy() if hasattr(own, "detach") else np.asarray(own)
        full = np.zeros(U.shape[:-1] + (self.x.shape[1],))
        full[..., self.plan.owned] = own
        return self._all_sum(full)

    def close(self):
        self.engine.close()
