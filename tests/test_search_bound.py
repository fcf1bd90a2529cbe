"""The segment search's pruning bound against binary32 rounding (no GPU).

The rollout kernel skips a bound box (the level-2 and chunk boxes, and the prefix/suffix boxes of
the vertices) when the box's computed squared distance from the point exceeds prune_lim(best): the
search's result is then the brute-force minimum key only if no segment inside a skipped box has a
computed squared distance at or below the best one.  The bound rests on a rounding argument (the
errors of seg_dist2 and box_dist2 are relative to the differences they form, and a segment's far end
lies within 2^-24 |e| of its vertex).  This test restates the kernel's binary32 arithmetic in numpy
(each operation rounded to binary32, a fused multiply-add as one rounding of the exact result) and
checks the claim on adversarial geometry: segments from a millimetre to ten metres long, coordinates
up to 10 km from the frame's origin, points from a micrometre to tens of metres off the lane, near
vertices and on segment extensions.  The square root of the best distance is taken 2^-22 low (the
hardware reciprocal square root is within a few ulp), which only makes the bound tighter.  A relative
slack alone (1/1024 or 2^-20 of the squared distance) or the bound without its length term fails
this test on these geometries.
"""
import numpy as np
import pytest

F = np.float32
TWO_M20 = F(2.0 ** -20)


def fma(a, b, c):
    """binary32 fused multiply-add: the exact a*b (representable in binary64) plus c, rounded once
    to binary64 and then to binary32 (the double rounding changes at most the last bit in rare ties,
    far below the margins tested here)."""
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(F)


def seg_records(vx, vy):
    """The kernel's segment records from binary32 vertices: e = b - a rounded, and e / |e|^2."""
    ex = (vx[1:] - vx[:-1]).astype(F)
    ey = (vy[1:] - vy[:-1]).astype(F)
    l2 = fma(ex, ex, (ey * ey).astype(F))
    inv = np.where(l2 > 0, (F(1.0) / np.where(l2 > 0, l2, F(1.0))).astype(F), F(0.0)).astype(F)
    return ex, ey, (ex * inv).astype(F), (ey * inv).astype(F)


def seg_dist2(px, py, ax, ay, ex, ey, sz, sw):
    dax = (px - ax).astype(F)
    day = (py - ay).astype(F)
    tau = np.clip(fma(dax, sz, (day * sw).astype(F)), F(0.0), F(1.0)).astype(F)
    dx = fma(-tau, ex, dax)
    dy = fma(-tau, ey, day)
    return fma(dx, dx, (dy * dy).astype(F))


def box_dist2(px, py, x0, y0, x1, y1):
    dx = np.maximum(np.maximum((x0 - px).astype(F), (px - x1).astype(F)), F(0.0))
    dy = np.maximum(np.maximum((y0 - py).astype(F), (py - y1).astype(F)), F(0.0))
    return fma(dx, dx, (dy * dy).astype(F))


def prune_lim(best2, lfac):
    d = (np.sqrt(best2.astype(np.float64)) * (1.0 - 2.0 ** -22)).astype(F)
    e = (TWO_M20 * fma(F(2.0), d, lfac)).astype(F)
    r = fma(d, TWO_M20, (d + e).astype(F))
    return (r * r).astype(F)


def lane(rng, kind, n, origin):
    """A polyline in binary64 world coordinates, its vertices rounded to binary32 in a frame centred
    on `origin` as scene preparation does."""
    lengths = np.exp(rng.uniform(np.log(1e-3), np.log(10.0), n - 1))
    if kind == "straight":
        ang = np.full(n - 1, rng.uniform(-np.pi, np.pi))
    elif kind == "zigzag":
        ang = rng.uniform(-np.pi, np.pi) + np.where(np.arange(n - 1) % 2 == 0, 1.2, -1.2)
    else:
        ang = np.cumsum(rng.normal(0.0, 0.6, n - 1))
    world = np.zeros((n, 2))
    world[0] = origin + rng.uniform(-50.0, 50.0, 2)
    world[1:] = world[0] + np.cumsum(np.stack([lengths * np.cos(ang), lengths * np.sin(ang)], 1), 0)
    return (world[:, 0] - origin[0]).astype(F), (world[:, 1] - origin[1]).astype(F)


def points_near(rng, vx, vy, m):
    """Points at distances from 1e-6 m to 30 m of the lane: off segment interiors, off vertices and
    on the extensions of segments."""
    n = vx.shape[0]
    i = rng.integers(0, n - 1, m)
    t = rng.choice([0.0, 1.0, -0.3, 1.3, 0.5], m) * rng.uniform(0.0, 1.0, m) ** rng.choice([0.0, 1.0], m)
    ax, ay = vx[i].astype(np.float64), vy[i].astype(np.float64)
    bx, by = vx[i + 1].astype(np.float64), vy[i + 1].astype(np.float64)
    qx, qy = ax + t * (bx - ax), ay + t * (by - ay)
    off = np.exp(rng.uniform(np.log(1e-6), np.log(30.0), m))
    ang = rng.uniform(-np.pi, np.pi, m)
    return (qx + off * np.cos(ang)).astype(F), (qy + off * np.sin(ang)).astype(F)


def points_past_ends(rng, vx, vy, m):
    """Points just past a vertex along the segment that ends there (1e-7 m to 1e-2 m beyond it):
    where the rounded segment's far end a + e may lie outside the box of the vertices."""
    n = vx.shape[0]
    i = rng.integers(0, n - 1, m)
    forward = rng.integers(0, 2, m).astype(bool)
    ax, ay = vx[i].astype(np.float64), vy[i].astype(np.float64)
    bx, by = vx[i + 1].astype(np.float64), vy[i + 1].astype(np.float64)
    ux, uy = bx - ax, by - ay
    ln = np.hypot(ux, uy)
    ln = np.where(ln > 0, ln, 1.0)
    ux, uy = ux / ln, uy / ln
    d = np.exp(rng.uniform(np.log(1e-7), np.log(1e-2), m))
    sx, sy = np.where(forward, bx, ax), np.where(forward, by, ay)
    sgn = np.where(forward, 1.0, -1.0)
    return (sx + sgn * d * ux).astype(F), (sy + sgn * d * uy).astype(F)


@pytest.mark.parametrize("kind", ["straight", "zigzag", "walk"])
@pytest.mark.parametrize("scale", [0.0, 3e2, 1e4])
def test_no_box_can_be_skipped_against_its_own_closest_segment(kind, scale):
    """For every point and every prefix range (segments 0 .. i-1, the box of the vertices 0 .. i)
    and suffix range (segments i .., the vertices i .. n-1) — the boxes the search tests around its
    window and in its side walks — and every chunk and level-2 range (the boxes of its range
    search), the box's computed squared distance is at most prune_lim of the
    smallest computed squared distance of a segment inside it.  Then no best distance can let the
    search skip a box that holds a segment at or below it (were the box skipped against best, its
    own closest segment would be above best)."""
    rng = np.random.default_rng(1000 * ["straight", "zigzag", "walk"].index(kind) + int(scale))
    n = 257
    for rep in range(6):
        origin = rng.uniform(-scale, scale, 2)
        vx, vy = lane(rng, kind, n, origin)
        ex, ey, sz, sw = seg_records(vx, vy)
        lmax = np.sqrt(fma(ex, ex, (ey * ey).astype(F)).astype(np.float64)).astype(F).max()
        lfac = F(4.0 * lmax)
        qx, qy = points_near(rng, vx, vy, 300)
        rx, ry = points_past_ends(rng, vx, vy, 300)
        px, py = np.concatenate([qx, rx]), np.concatenate([qy, ry])
        # every segment's computed squared distance from every point: [points, segments]
        d2 = seg_dist2(px[:, None], py[:, None], vx[None, :-1], vy[None, :-1], ex[None], ey[None], sz[None], sw[None])
        pre_x0 = np.minimum.accumulate(vx); pre_x1 = np.maximum.accumulate(vx)
        pre_y0 = np.minimum.accumulate(vy); pre_y1 = np.maximum.accumulate(vy)
        suf_x0 = np.minimum.accumulate(vx[::-1])[::-1]; suf_x1 = np.maximum.accumulate(vx[::-1])[::-1]
        suf_y0 = np.minimum.accumulate(vy[::-1])[::-1]; suf_y1 = np.maximum.accumulate(vy[::-1])[::-1]
        seg_lo = np.minimum.accumulate(d2, axis=1)                      # min over segments 0 .. i
        seg_hi = np.minimum.accumulate(d2[:, ::-1], axis=1)[:, ::-1]     # min over segments i .. n-2
        for i in range(1, n - 1):
            bp = box_dist2(px, py, pre_x0[i], pre_y0[i], pre_x1[i], pre_y1[i])
            assert np.all(bp <= prune_lim(seg_lo[:, i - 1], lfac)), (kind, scale, "prefix", i)
            bs = box_dist2(px, py, suf_x0[i], suf_y0[i], suf_x1[i], suf_y1[i])
            assert np.all(bs <= prune_lim(seg_hi[:, i], lfac)), (kind, scale, "suffix", i)
        # the chunk boxes (4 segments: vertices 4c .. 4c + 4) and level-2 boxes (16 chunks)
        for width in (4, 64):
            for c0 in range(0, n - 1, width):
                c1 = min(c0 + width, n - 1)
                b = box_dist2(px, py, vx[c0:c1 + 1].min(), vy[c0:c1 + 1].min(), vx[c0:c1 + 1].max(),
                              vy[c0:c1 + 1].max())
                assert np.all(b <= prune_lim(d2[:, c0:c1].min(1), lfac)), (kind, scale, width, c0)


@pytest.mark.parametrize("scale", [0.0, 1e4])
def test_vertex_mode_boxes(scale):
    """The closest-vertex reading (ref_mode 1) prunes its chunk and level-2 boxes with prune_lim and
    no length term: a box of vertices holds no vertex whose computed squared distance is below
    prune_lim's argument when the box is skipped."""
    rng = np.random.default_rng(7 + int(scale))
    for kind in ("straight", "zigzag", "walk"):
        origin = rng.uniform(-scale, scale, 2)
        vx, vy = lane(rng, kind, 257, origin)
        px, py = points_near(rng, vx, vy, 400)
        dx = (px[:, None] - vx[None, :]).astype(F)
        dy = (py[:, None] - vy[None, :]).astype(F)
        d2 = fma(dx, dx, (dy * dy).astype(F))
        for width in (5, 65):                     # a chunk covers its 4 segments' 5 vertices
            for c0 in range(0, 256, width - 1):
                c1 = min(c0 + width, 257)
                b = box_dist2(px, py, vx[c0:c1].min(), vy[c0:c1].min(), vx[c0:c1].max(), vy[c0:c1].max())
                assert np.all(b <= prune_lim(d2[:, c0:c1].min(1), F(0.0))), (kind, scale, width, c0)


def test_bound_is_close_to_the_best_distance():
    """On a 2000-point lane of 0.1 m segments a point 2 m off the lane may skip every box more than
    about 1.3 cm farther than its best segment (the bound adds 2^-20 (2d + 4 l) to d, and 2^-20 d)."""
    best = F(4.0)
    lim = prune_lim(np.array([best]), F(0.4))[0]
    assert best < lim < best * (1.0 + 3e-5)
    along = np.sqrt(float(lim) - float(best))
    assert along < 0.013
