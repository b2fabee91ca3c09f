"""Coefficients of the float arctangent in rt_pair.cuh (angle_0_pi).

atan(a) on a in [0, 1] is written a * q(a^2) with q a polynomial of degree 7, fitted by
iteratively reweighted least squares towards the smallest largest error on 4001
Chebyshev-spaced values of a^2.  Run this file to print the coefficients c0 ... c7 and the
largest error of the fit evaluated in float32 by Horner's rule (about 1.3e-7 rad).
"""
import numpy as np

DEGREE = 7


def fit(degree: int = DEGREE) -> np.ndarray:
    t = np.cos(np.linspace(0.0, np.pi, 4001)) * 0.5 + 0.5      # a^2 in [0, 1]
    a = np.sqrt(t)
    basis = np.stack([a * t**k for k in range(degree + 1)], axis=1)
    y = np.arctan(a)
    w = np.ones_like(t)
    c = None
    for _ in range(60):
        c, *_ = np.linalg.lstsq(basis * w[:, None], y * w, rcond=None)
        err = basis @ c - y
        w = w * (np.abs(err) / np.abs(err).max() + 1e-3) ** 0.5
        w /= w.max()
    return c


def horner_f32(c: np.ndarray, a: np.ndarray) -> np.ndarray:
    """a * q(a^2) in float32, the way the kernel evaluates it."""
    c32 = np.asarray(c, dtype=np.float32)
    a = np.asarray(a, dtype=np.float32)
    t = (a * a).astype(np.float32)
    q = np.full_like(a, c32[-1])
    for k in range(len(c32) - 2, -1, -1):
        q = (q * t + c32[k]).astype(np.float32)
    return (a * q).astype(np.float32)


if __name__ == "__main__":
    c = fit()
    a = np.linspace(0.0, 1.0, 2_000_001)
    e = np.abs(horner_f32(c, a).astype(np.float64) - np.arctan(a.astype(np.float32).astype(np.float64)))
    print("coefficients:", ", ".join("%.9g" % v for v in c))
    print("largest error in float32: %.3g rad" % e.max())
