"""CPU check of the culling pass's arctangent (fast_atan2 in grca_kernels.cu).

The coefficients are read from the CUDA source and the function is evaluated
in float32 with the same operation order; its error against the FP64
arctangent must stay below the padding the culling pass adds (2e-6 rad).
"""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2605_10457_gb300", "csrc",
                   "grca_kernels.cu")


def coefficients():
    src = open(SRC).read()
    c = {int(k): np.float32(float(v)) for k, v in re.findall(r"ATAN_C(\d) = (-?[0-9.e-]+)f", src)}
    pad = float(re.search(r"FAST_ATAN_PAD = ([0-9.e-]+)f", src).group(1))
    return [c[k] for k in range(7)], pad


def fast_atan2(y, x, c):
    y = y.astype(np.float32)
    x = x.astype(np.float32)
    ax, ay = np.abs(x), np.abs(y)
    mx, mn = np.maximum(ax, ay), np.minimum(ax, ay)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = np.where(mx > 0, mn / mx, np.float32(0)).astype(np.float32)
    t2 = (t * t).astype(np.float32)
    r = np.float32(c[6]) * t2 + c[5]
    for k in (4, 3, 2, 1, 0):
        r = (t2 * r + c[k]).astype(np.float32)
    r = (r * t).astype(np.float32)
    r = np.where(ay > ax, np.float32(1.5707963) - r, r).astype(np.float32)
    r = np.where(x < 0, np.float32(3.1415927) - r, r).astype(np.float32)
    return np.copysign(r, y)


def test_fast_atan2_error_below_padding():
    c, pad = coefficients()
    rng = np.random.default_rng(0)
    ang = np.concatenate([rng.uniform(-np.pi, np.pi, 2_000_000), np.linspace(-np.pi, np.pi, 200_001)])
    rad = np.exp(rng.uniform(np.log(1e-3), np.log(1e3), ang.size))
    x, y = (rad * np.cos(ang)).astype(np.float32), (rad * np.sin(ang)).astype(np.float32)
    got = fast_atan2(y, x, c).astype(np.float64)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    err = np.abs(np.angle(np.exp(1j * (got - ref))))
    assert err.max() < 0.5 * pad, err.max()
    # axes and diagonals
    for yy, xx in [(0.0, 1.0), (1.0, 0.0), (0.0, -1.0), (-1.0, 0.0), (1.0, 1.0), (-1.0, -1.0), (1e-30, 1.0)]:
        g = float(fast_atan2(np.array([yy]), np.array([xx]), c)[0])
        assert abs(np.angle(np.exp(1j * (g - np.arctan2(yy, xx))))) < 0.5 * pad
