"""The float arctangent of the HLL wave speeds (angle_0_pi in csrc/rt_pair.cuh).

Its coefficients must be those that csrc/fit_atan.py fits, the fit's largest error in float32
must stay within 2e-7 rad of atan on [0, 1], and the octant and half-plane folds must give
numpy's arctan2 for y >= 0 (the HLL table's theta = atan2(|F x A|, F . A) lies in [0, pi]).
The GPU HLL parity tests check its use against the FP64 oracle."""
import importlib.util
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2302_12727_gb300", "csrc")


def _fit_module():
    spec = importlib.util.spec_from_file_location("fit_atan", os.path.join(CSRC, "fit_atan.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _kernel_coefficients():
    src = open(os.path.join(CSRC, "rt_pair.cuh")).read()
    body = src[src.index("__device__ __forceinline__ float angle_0_pi"):]
    body = body[:body.index("float r = a * q;")]
    lits = [float(v) for v in re.findall(r"(-?\d+\.\d+(?:e-?\d+)?)f", body)]
    return lits[::-1]          # the kernel's Horner order is c7 first


def _angle_f32(c, y, x):
    y = np.asarray(y, dtype=np.float32)
    x = np.asarray(x, dtype=np.float32)
    ax = np.abs(x)
    mx, mn = np.maximum(ax, y), np.minimum(ax, y)
    with np.errstate(divide="ignore", invalid="ignore"):
        a = np.where(mx > 0, mn / np.where(mx > 0, mx, 1), 0).astype(np.float32)
    m = _fit_module()
    r = m.horner_f32(c, a)
    r = np.where(y > ax, np.float32(1.57079637) - r, r)
    return np.where(x < 0, np.float32(3.14159274) - r, r).astype(np.float32)


def test_kernel_coefficients_are_the_fit():
    m = _fit_module()
    c = m.fit()
    k = _kernel_coefficients()
    assert len(k) == m.DEGREE + 1
    np.testing.assert_allclose(k, c, rtol=2e-8, atol=1e-9)


def test_fit_error_in_float32():
    m = _fit_module()
    c = np.array(_kernel_coefficients())
    a = np.linspace(0.0, 1.0, 1_000_001)
    err = np.abs(m.horner_f32(c, a).astype(np.float64) - np.arctan(a.astype(np.float32).astype(np.float64)))
    assert err.max() < 2e-7


def test_folds_give_arctan2_on_the_upper_half_plane():
    c = np.array(_kernel_coefficients())
    rng = np.random.default_rng(5)
    x = rng.normal(size=200_000) * 10.0 ** rng.uniform(-12, 3, size=200_000)
    y = np.abs(rng.normal(size=200_000)) * 10.0 ** rng.uniform(-12, 3, size=200_000)
    x[:100], y[:100] = 0.0, 0.0                      # F = 0
    y[100:200] = 0.0                                 # F parallel or antiparallel to A
    x[200:300] = 0.0                                 # F perpendicular to A
    got = _angle_f32(c, y, x).astype(np.float64)
    ref = np.arctan2(y.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64))
    ref[:100] = 0.0                                  # the fold's reading of (0, 0)
    assert np.abs(got - ref).max() < 5e-7
    assert got.min() >= 0.0 and got.max() <= np.float32(3.14159274)
