"""The oracle's per-pair operation counter against counts derived by hand, and the benchmark's
flop constants against the counter.

The counter (oracle.Oracle.pair_flops) runs the oracle's own pair arithmetic on a scalar that
counts add, subtract, multiply, divide and square root (one each).  Its figures are pinned
here to a count written out from the formulas the oracle implements:

  cubic spline W(r, h) (Eq. cubic-spline-kernel): q = r / H (1); for q <= 1/2 the two cubes
    (1-q)^3 (3 subtractions, 2 multiplications) and 4 (1/2-q)^3 (3 + 3) and their difference
    (1), times sigma / H^3 (1): K = 14; for 1/2 < q < 1: 1 + 5 + 1 = 7; for q >= 1: 2.
  psitilde_j(x_i) = B_i d W / omega_i (Eq. psitilde): W (K) / omega (1), B d (9 mul + 6 add),
    times psi (3): K + 19.
  separation 3, |d| = sqrt(d.d) 6.
  flux geometry per pair: 3 + 6 + psitilde both ways (2 x 19 + K_i + K_j) + A_ij = V_i p_i -
    V_j p_j (9) + |A| (6) + c/2 |A| (1) = 63 + K_i + K_j.
  gradient geometry per directed entry: 3 + 6 + 19 + K_i = 28 + K_i.
  face states (Eq. rt-riemann-problem) per group: weights h_k/(h_k+h_l), h_l/(..) (3), per
    component two 3-term dot products (12), minmod (comparisons only), two updates (4): 67.
  M1 flux F(U).A in the general branch (Eq. eddington-group): F.A 5, |F|^2 5, sqrt 1,
    f = |F|/(cE) 2, f^2 1, chi 8, n = F/|F| 3, n.A 5, (1-chi)/2 2, (3chi-1)/2 3, the three
    flux rows c^2 E (a_iso A + a_dir (n.A) n) 3 x 6: 53.
  GLF (Eq. riemann-GLF) per component 1/2 (fL + fR) - diss (uR - uL): 5, x 4 = 20.
  flux per pair and group: 67 + 2 x 53 + 20 = 193.
  gradient per directed entry and group: four components x (1 difference + 3 products +
    3 sums) = 28; accumulation into both particles: 2 x 4 = 8.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2302_12727_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
H_h = oracle.H_OVER_h


def _K(q):
    return np.where(q <= 0.5, 14, np.where(q < 1.0, 7, 2))


def _hand_geometry(w, o):
    off, cols = o.pairs()
    n = w.n
    rows = np.repeat(np.arange(n), np.diff(off))
    d = w.x[:, cols] - w.x[:, rows]
    d -= np.rint(d)
    r = np.sqrt((d * d).sum(0))
    Ki = _K(r / (H_h * o.h[rows]))
    Kj = _K(r / (H_h * o.h[cols]))
    up = cols > rows
    return float(np.mean(63 + Ki[up] + Kj[up])), float(np.mean(28 + Ki))


def test_counter_equals_the_hand_count():
    w = W.poisson_sine_beam(16)
    o = oracle.Oracle(w.x, w.m, w.xsrc, n_groups=w.n_groups, c_red=w.c_red)
    f = o.pair_flops()
    assert f["flux_per_group"] == 193
    assert f["gradient_per_group"] == 28
    assert f["accumulate_per_group"] == 8
    geo, ggeo = _hand_geometry(w, o)
    assert f["flux_geometry"] == pytest.approx(geo, rel=1e-12)
    assert f["gradient_geometry"] == pytest.approx(ggeo, rel=1e-12)


def _bench_constants():
    src = open(os.path.join(ROOT, "bench.py")).read()
    ns = {}
    block = src[src.index("PAIR_FLOPS = {"):src.index("def pair_flops(")]
    exec(block, ns)
    return ns


@pytest.mark.parametrize("name", ["poisson-sine-beam", "lognormal-sources"])
def test_bench_constants_match_the_counter(name):
    """bench.py's roofline uses these per-pair counts on the full 262,144- and
    2,097,152-particle sets."""
    c = _bench_constants()
    w = W.WORKLOADS[name]()
    o = oracle.Oracle(w.x, w.m, w.xsrc, n_groups=w.n_groups, c_red=w.c_red)
    f = o.pair_flops()
    assert f["flux_per_group"] == c["FLUX_PER_GROUP"]
    assert f["gradient_per_group"] == c["GRAD_PER_GROUP"]
    assert f["accumulate_per_group"] == c["ACC_PER_GROUP"]
    assert f["flux_geometry"] == pytest.approx(c["PAIR_FLOPS"][name]["flux_geometry"], abs=0.006)
    assert f["gradient_geometry"] == pytest.approx(c["PAIR_FLOPS"][name]["gradient_geometry"], abs=0.006)
