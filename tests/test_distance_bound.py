"""CPU checks of the distance lower bound that the FP32 pass uses to drop
occluded pairs and to raise the lower bound of queued re-test entries:
t_lb = min_k |p_k| (1 - 4e-6) - max_k |p_k1 - p_k| (1 + 4e-6), with p the
triangle's vertices relative to the sensor origin.  Every point of a
triangle lies within its longest edge of each vertex, so the distance from
the origin to any point of the triangle, and hence to any ray hit on it, is
at least t_lb.  The bound is computed here in FP32 (the kernel's precision,
explicitly rounded) and checked against the exact closest-point distance in
FP64, over random and adversarial triangles."""
import numpy as np


SQRT_ERR = 2.0 ** -22   # relative error bound of the hardware's approximate square root


def t_lb_fp32(p, adverse_sqrt=True):
    """The bound in FP32 arithmetic, the kernel's operation order; the square
    roots take their worst-case approximation error in the direction that
    loosens the bound the least (smaller nearest distance, longer edge)."""
    p = np.asarray(p, np.float32)
    f = np.float32
    r2 = [f(f(p[k, 0] * p[k, 0]) + f(p[k, 1] * p[k, 1])) + f(p[k, 2] * p[k, 2]) for k in range(3)]
    e = [p[1] - p[0], p[2] - p[1], p[0] - p[2]]
    ee = [f(f(v[0] * v[0]) + f(v[1] * v[1])) + f(v[2] * v[2]) for v in e]
    lo, hi = (f(1 - SQRT_ERR), f(1 + SQRT_ERR)) if adverse_sqrt else (f(1), f(1))
    r = f(np.sqrt(f(min(r2))) * lo)
    l = f(np.sqrt(f(max(ee))) * hi)
    lb = f(f(r * f(1 - 4e-6)) - f(l * f(1 + 4e-6)))
    return float(lb) if lb > 0 else 0.0


def emitter_frame_fp32(v, origin, basis):
    """The kernel's path from world vertices to emitter-frame vertices in
    FP32: w = (v - o_hi) - o_lo with the origin split into FP32 high and low
    parts, then p = B w with the FP32 rows of an orthonormal basis."""
    o_hi = np.asarray(origin, np.float64).astype(np.float32)
    o_lo = (np.asarray(origin, np.float64) - o_hi.astype(np.float64)).astype(np.float32)
    w = (np.asarray(v, np.float32) - o_hi) - o_lo
    B = np.asarray(basis, np.float64).astype(np.float32)
    f = np.float32
    return np.array([[f(f(f(B[i, 0] * wk[0]) + f(B[i, 1] * wk[1])) + f(B[i, 2] * wk[2])) for i in range(3)] for wk in w],
                    np.float32)


def closest_distance(p):
    """Exact (FP64) distance from the origin to the closed triangle p: the
    plane projection if it falls inside, else the nearest point of an edge."""
    a, b, c = (np.asarray(v, np.float64) for v in p)
    n = np.cross(b - a, c - a)
    nn = n @ n
    if nn > 0:
        q = (a @ n) / nn * n                      # projection of the origin on the plane
        w = [np.cross(b - a, q - a) @ n, np.cross(c - b, q - b) @ n, np.cross(a - c, q - c) @ n]
        if min(w) >= 0:
            return float(np.linalg.norm(q))
    best = np.inf
    for u, v in ((a, b), (b, c), (c, a)):
        e = v - u
        s = 0.0 if e @ e == 0 else min(max(-(u @ e) / (e @ e), 0.0), 1.0)
        best = min(best, float(np.linalg.norm(u + s * e)))
    return best


def test_bound_never_exceeds_the_closest_point_distance():
    """World triangles of size 10^U(-3, 1) m at 10^U(-1, 2.5) m from a sensor
    whose origin sits up to 3 km from the world origin (so that its FP32 low
    part matters) and whose frame is a random rotation: the bound from the
    FP32 emitter-frame vertices never exceeds the exact FP64 distance from the
    FP64 origin to the FP32 triangle."""
    rng = np.random.default_rng(7)
    checked = 0
    for it in range(3000):
        origin = rng.normal(size=3) * (3000.0 if it % 2 else 2.0)
        basis, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        centre = rng.normal(size=3)
        centre *= 10 ** rng.uniform(-1, 2.5) / np.linalg.norm(centre)
        v = (origin + centre + rng.normal(size=(3, 3)) * 10 ** rng.uniform(-3, 1)).astype(np.float32)
        lb = t_lb_fp32(emitter_frame_fp32(v, origin, basis))
        d = closest_distance(v.astype(np.float64) - origin)
        assert lb <= d, (v, origin, lb, d)
        checked += lb > 0
    assert checked > 1000   # the bound is informative for most small, far triangles


def test_bound_is_tight_for_small_far_triangles():
    # a 5 cm triangle 40 m away: the bound lies within the triangle's size of the distance
    p = np.array([[40.0, 0.0, 0.0], [40.0, 0.05, 0.0], [40.0, 0.0, 0.05]], np.float32)
    lb = t_lb_fp32(p)
    d = closest_distance(p)
    assert abs(d - 40.0) < 1e-9
    assert 40.0 - 0.0708 - 1e-3 < lb <= d


def test_bound_is_zero_where_it_says_nothing():
    # a triangle around the origin, a huge triangle, and a non-finite vertex
    assert t_lb_fp32([[1, -1, -1], [1, 1, -1], [-2, 0, 2]]) == 0.0
    assert t_lb_fp32([[5, 0, 0], [5, 100, 0], [5, 0, 100]]) == 0.0
    assert t_lb_fp32([[np.inf, 0, 0], [5, 1, 0], [5, 0, 1]]) == 0.0
    assert t_lb_fp32([[np.nan, 0, 0], [5, 1, 0], [5, 0, 1]]) == 0.0


def test_bound_holds_at_grazing_and_degenerate_shapes():
    rng = np.random.default_rng(11)
    for _ in range(2000):
        # slivers (aspect up to 1e4) and triangles seen edge-on, near and far
        r = 10 ** rng.uniform(-0.5, 2)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        t = np.cross(d, rng.normal(size=3))
        t /= np.linalg.norm(t)
        long_ = 10 ** rng.uniform(-2, 1)
        short = long_ * 10 ** rng.uniform(-4, 0)
        base = r * d
        p = np.array([base, base + long_ * t, base + short * np.cross(d, t) + 0.5 * long_ * t], np.float32)
        assert t_lb_fp32(p) <= closest_distance(p.astype(np.float64))


def test_bound_holds_for_large_triangles_facing_the_sensor():
    # an equilateral triangle of side L centred on the foot of the perpendicular
    # at distance D: its nearest vertex is about 0.58 L away, its plane only D;
    # a bound that took less than L / sqrt(3) off the nearest vertex would
    # exceed D once L is large against D
    rng = np.random.default_rng(3)
    for _ in range(500):
        D = 10 ** rng.uniform(-1, 1.5)
        L = D * 10 ** rng.uniform(0, 2)
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        u = np.cross(n, rng.normal(size=3))
        u /= np.linalg.norm(u)
        w = np.cross(n, u)
        ang = rng.uniform(0, 2 * np.pi) + np.array([0, 2 * np.pi / 3, 4 * np.pi / 3])
        p = np.array([D * n + L / np.sqrt(3) * (np.cos(a) * u + np.sin(a) * w) for a in ang], np.float32)
        assert t_lb_fp32(p) <= closest_distance(p.astype(np.float64))
