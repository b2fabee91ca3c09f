"""Seeded synthetic particle sets for the photon-transport step.

This module only draws random inputs: particle positions and masses, source
positions and luminosities, initial radiation states.  It holds none of the
transport method's arithmetic, so that the CUDA path and the CPU oracle can be
fed the very same arrays.

The shapes stand in for the test set-ups of the thesis (uniform and glass-like
particle sets of 128^3 particles, about 48 neighbours, a few photon groups,
point sources, reduced speed of light; Part III, Iliev tests).  None of the
thesis's initial-condition files are used: everything is drawn from
``numpy.random.default_rng(12727 + seed_id)``, one seed offset per workload.

Arrays are in the layouts of the C interface:
  x      float64 [3, N]      positions, component-major (SoA)
  m      float64 [N]         particle masses
  xsrc   float64 [3, S]      source positions
  Lsrc   float64 [S, G]      source luminosity per photon group
  U0     float64 [G, 4, N]   (E, Fx, Fy, Fz) per group, component-major
"""
from __future__ import annotations

from dataclasses import dataclass, field
import numpy as np

SEED_BASE = 12727


@dataclass
class Workload:
    name: str
    seed_id: int
    x: np.ndarray
    m: np.ndarray
    xsrc: np.ndarray
    Lsrc: np.ndarray
    U0: np.ndarray
    n_groups: int
    n_steps: int
    c_red: float = 1.0
    box: tuple = (1.0, 1.0, 1.0)
    periodic: bool = True
    kappa: float = 0.0          # grey opacity: alpha_i = kappa * rho_i, rho_i = m_i * omega_i
    ckpt_every: int = 0
    dt_factor: float = 0.9      # dt = dt_factor * min(h) / c_red
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.x.shape[1]

    @property
    def n_src(self) -> int:
        return self.xsrc.shape[1]


def _rng(seed_id: int) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + seed_id)


def jittered_lattice(n_side: int, jitter: float, rng: np.random.Generator) -> np.ndarray:
    """Cubic lattice (i + 1/2)/n_side with a uniform jitter of +-jitter spacing per axis,
    wrapped into the periodic unit box."""
    i = np.arange(n_side, dtype=np.float64)
    gx, gy, gz = np.meshgrid(i, i, i, indexing="ij")
    pts = np.stack([gx.ravel(), gy.ravel(), gz.ravel()])  # [3, N]
    pts = (pts + 0.5 + rng.uniform(-jitter, jitter, size=pts.shape)) / n_side
    return np.mod(pts, 1.0)


def perfect_lattice(n_side: int) -> np.ndarray:
    i = (np.arange(n_side, dtype=np.float64) + 0.5) / n_side
    gx, gy, gz = np.meshgrid(i, i, i, indexing="ij")
    return np.stack([gx.ravel(), gy.ravel(), gz.ravel()])


def poisson_sine_density(n: int, rng: np.random.Generator) -> np.ndarray:
    """Rejection sampling of rho(x) = 1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z)
    (accept with probability rho / 1.5) until exactly n points are kept."""
    out = np.empty((3, 0))
    while out.shape[1] < n:
        need = n - out.shape[1]
        cand = rng.uniform(0.0, 1.0, size=(3, int(need * 1.6) + 1024))
        rho = 1.0 + 0.5 * np.sin(2 * np.pi * cand[0]) * np.sin(2 * np.pi * cand[1]) * np.sin(2 * np.pi * cand[2])
        keep = rng.uniform(0.0, 1.5, size=cand.shape[1]) < rho
        out = np.concatenate([out, cand[:, keep]], axis=1)
    return np.ascontiguousarray(out[:, :n])


def lognormal_field_particles(n: int, grid: int, sigma_ln: float, rng: np.random.Generator) -> np.ndarray:
    """Particles drawn from a lognormal density rho = exp(delta - sigma^2/2), delta a Gaussian
    random field on a grid^3 mesh with P(k) ~ k^-2 (k = 0 mode removed), rescaled to
    standard deviation sigma_ln.  Multinomial counts per mesh cell, uniform within a cell."""
    kf = np.fft.fftfreq(grid) * grid
    kz = np.fft.rfftfreq(grid) * grid
    k2 = kf[:, None, None] ** 2 + kf[None, :, None] ** 2 + kz[None, None, :] ** 2
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (-0.5)          # sqrt(P(k)) with P ~ k^-2
    noise = rng.standard_normal(k2.shape) + 1j * rng.standard_normal(k2.shape)
    delta = np.fft.irfftn(noise * amp, s=(grid, grid, grid), axes=(0, 1, 2))
    delta *= sigma_ln / delta.std()
    rho = np.exp(delta - 0.5 * sigma_ln ** 2).ravel()
    counts = rng.multinomial(n, rho / rho.sum())
    cell = np.repeat(np.arange(grid ** 3), counts)
    cz = cell % grid
    cy = (cell // grid) % grid
    cx = cell // (grid * grid)
    pts = np.stack([cx, cy, cz]).astype(np.float64)
    pts += rng.uniform(0.0, 1.0, size=pts.shape)
    return np.ascontiguousarray(pts / grid)


def random_unit_vectors(n: int, rng: np.random.Generator) -> np.ndarray:
    v = rng.standard_normal((3, n))
    return v / np.linalg.norm(v, axis=0, keepdims=True)


def lattice_point_source() -> Workload:
    """16^3 jittered lattice, 1 group, one source of luminosity 1 at the centre, 10 steps."""
    rng = _rng(1)
    x = jittered_lattice(16, 0.2, rng)
    n = x.shape[1]
    G = 1
    U0 = np.zeros((G, 4, n))
    U0[:, 0, :] = 1e-10
    return Workload("jittered-lattice-16^3-G1", 1, x, np.full(n, 1.0 / n),
                    np.array([[0.5], [0.5], [0.5]]), np.ones((1, G)), U0, G, 10)


def poisson_sine_beam(n_side: int = 64) -> Workload:
    """64^3 Poisson-sampled sine density, 3 groups, central source plus a collimated beam,
    grey opacity kappa = 0.1, 50 steps."""
    rng = _rng(2)
    n = n_side ** 3
    x = poisson_sine_density(n, rng)
    G = 3
    c = 1.0
    U0 = np.zeros((G, 4, n))
    U0[:, 0, :] = 1e-10
    ryz = np.hypot(x[1] - 0.5, x[2] - 0.5)
    beam = (ryz < 0.05) & (x[0] >= 0.1) & (x[0] <= 0.2)
    U0[:, 0, beam] = 1.0
    U0[:, 1, beam] = c * 1.0
    return Workload(f"poisson-sine-{n_side}^3-G3", 2, x, np.full(n, 1.0 / n),
                    np.array([[0.5], [0.5], [0.5]]), np.ones((1, G)), U0, G, 50,
                    c_red=c, kappa=0.1, extra={"beam_particles": int(beam.sum())})


def lattice_sources(n_side: int = 32) -> Workload:
    """32^3 jittered lattice, 2 groups, 8 sources with lognormal(0,1) luminosities,
    16 sub-cycles with a checkpoint every 4."""
    rng = _rng(3)
    x = jittered_lattice(n_side, 0.2, rng)
    n = x.shape[1]
    G = 2
    c = 1.0
    S = 8
    xsrc = rng.uniform(0.0, 1.0, size=(3, S))
    Lsrc = rng.lognormal(0.0, 1.0, size=(S, G))
    E0 = 1e-10 * (1.0 + 0.1 * rng.uniform(-1.0, 1.0, size=(G, n)))
    dirs = np.stack([random_unit_vectors(n, rng) for _ in range(G)])  # [G, 3, N]
    U0 = np.zeros((G, 4, n))
    U0[:, 0, :] = E0
    U0[:, 1:, :] = 0.05 * c * E0[:, None, :] * dirs
    return Workload(f"jittered-lattice-{n_side}^3-G2-S8", 3, x, np.full(n, 1.0 / n), xsrc, Lsrc, U0,
                    G, 16, c_red=c, ckpt_every=4)


def lognormal_sources(n_side: int = 128, grid: int = 256, sigma_ln: float = 1.0, G: int = 4, S: int = 64,
                      n_sub: int = 32, seed_id: int = 4, sigma_L: float = 1.0, kappa: float = 0.0) -> Workload:
    """Lognormal clustered particle set (P(k) ~ k^-2), G groups, S sources with lognormal
    luminosities, n_sub sub-cycles."""
    rng = _rng(seed_id)
    n = n_side ** 3
    x = lognormal_field_particles(n, grid, sigma_ln, rng)
    xsrc = rng.uniform(0.0, 1.0, size=(3, S))
    Lsrc = rng.lognormal(0.0, sigma_L, size=(S, G))
    U0 = np.zeros((G, 4, n))
    U0[:, 0, :] = 1e-10
    return Workload(f"lognormal-{n_side}^3-sigma{sigma_ln:g}-G{G}-S{S}", seed_id, x, np.full(n, 1.0 / n),
                    xsrc, Lsrc, U0, G, n_sub, kappa=kappa)


def lognormal_sources_large() -> Workload:
    """256^3 lognormal set (sigma_ln = 2, P(k) ~ k^-2), 4 groups, 1000 sources with
    lognormal(0, 2) luminosities, grey kappa = 0.1, 64 sub-cycles."""
    return lognormal_sources(256, 512, 2.0, 4, 1000, 64, seed_id=5, sigma_L=2.0, kappa=0.1)


def plane_wave(n_side: int, width: float, shape: str = "gaussian", c: float = 1.0) -> Workload:
    """Perfect lattice with E a function of x only and F = c E along +x (free streaming)."""
    x = perfect_lattice(n_side)
    n = x.shape[1]
    U0 = np.zeros((1, 4, n))
    if shape == "gaussian":
        E = np.exp(-0.5 * ((x[0] - 0.3) / width) ** 2)
    else:
        E = np.where(np.abs(x[0] - 0.3) < width, 1.0, 0.0)
    U0[0, 0] = E
    U0[0, 1] = c * E
    return Workload(f"plane-wave-{shape}-{n_side}^3", 0, x, np.full(n, 1.0 / n),
                    np.zeros((3, 0)), np.zeros((0, 1)), U0, 1, 0, c_red=c)


# bench.py's --workload names
WORKLOADS = {"lattice-point-source": lattice_point_source, "poisson-sine-beam": poisson_sine_beam,
             "lattice-sources": lattice_sources, "lognormal-sources": lognormal_sources,
             "lognormal-sources-large": lognormal_sources_large}
