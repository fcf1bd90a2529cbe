"""mppi_box_to_circles: an oriented rectangle covered by circles (Sec. III-C, Fig. 3).

Host code of the library; no GPU.  Checked against the geometry it claims: the circles
cover every point of the rectangle, each circle is the smallest one through the corners of
its slice (a smaller radius leaves the slice's corners out), centres on the centre line, and
the object's velocity carried to every circle.
"""
import math

import numpy as np
import pytest

import paper_2308_01654_gb300 as mp


def rect_points(x, y, yaw, length, width, n=41):
    u = np.linspace(-0.5, 0.5, n)
    a, b = np.meshgrid(u * length, u * width)
    a, b = a.ravel(), b.ravel()
    c, s = math.cos(yaw), math.sin(yaw)
    return np.stack([x + a * c - b * s, y + a * s + b * c], axis=1)


def covered(circ, pts, slack=1e-9):
    d = np.hypot(pts[:, None, 0] - circ[None, :, 0], pts[:, None, 1] - circ[None, :, 1])
    return (d <= circ[None, :, 2] + slack).any(axis=1)


@pytest.mark.parametrize("x,y,yaw,length,width,n", [(0, 0, 0, 4.5, 1.8, 3), (12.5, -3, 0.7, 4.5, 1.8, 0),
                                                    (-2, 7, -2.9, 12.0, 2.5, 0), (1, 1, 1.2, 1.0, 3.0, 0),
                                                    (5, 5, 0.3, 4.0, 2.0, 1)])
def test_circles_cover_the_rectangle(x, y, yaw, length, width, n):
    circ = mp.box_to_circles(x, y, yaw, length, width, 1.5, -0.5, n)
    k = n if n else max(1, math.ceil(length / width))
    assert circ.shape == (k, 5)
    assert covered(circ, rect_points(x, y, yaw, length, width)).all()
    # radius of the circle through the corners of a length/k x width slice
    np.testing.assert_allclose(circ[:, 2], math.hypot(length / (2 * k), width / 2), rtol=1e-15)
    # centres on the centre line, spaced length/k, symmetric about (x, y)
    c, s = math.cos(yaw), math.sin(yaw)
    along = (circ[:, 0] - x) * c + (circ[:, 1] - y) * s
    across = -(circ[:, 0] - x) * s + (circ[:, 1] - y) * c
    np.testing.assert_allclose(across, 0, atol=1e-12)
    np.testing.assert_allclose(along, (np.arange(k) + 0.5) * length / k - length / 2, atol=1e-12)
    np.testing.assert_array_equal(circ[:, 3:], np.tile([1.5, -0.5], (k, 1)))


def test_smaller_circles_leave_the_corners_out():
    circ = mp.box_to_circles(0, 0, 0.4, 4.5, 1.8, n=3)
    shrunk = circ.copy()
    shrunk[:, 2] *= 1 - 1e-6
    assert not covered(shrunk, rect_points(0, 0, 0.4, 4.5, 1.8), slack=0).all()


def test_the_paper_figure_three_circle_car():
    # a car-sized object in three circles, as drawn in Fig. 3
    circ = mp.box_to_circles(20.0, 0.0, 0.0, 4.5, 1.8, n=3)
    np.testing.assert_allclose(circ[:, 0], [18.5, 20.0, 21.5])
    assert circ[0, 2] == pytest.approx(math.hypot(0.75, 0.9))


@pytest.mark.parametrize("args", [(0, 0, 0, 0.0, 1.0, 0), (0, 0, 0, 1.0, -1.0, 0), (math.nan, 0, 0, 1, 1, 0),
                                  (0, 0, math.inf, 1, 1, 0), (0, 0, 0, 1, 1, -2)])
def test_invalid_arguments(args):
    x, y, yaw, length, width, n = args
    with pytest.raises(mp.MppiError) as e:
        mp.box_to_circles(x, y, yaw, length, width, n=n)
    assert e.value.status == -1


def test_capacity():
    import ctypes as C
    out = (mp.MppiCircle * 2)() if hasattr(mp, "MppiCircle") else (C.c_double * 10)()
    rc = mp.lib().mppi_box_to_circles(0.0, 0.0, 0.0, 9.0, 1.0, 0.0, 0.0, 0, C.cast(out, C.c_void_p), 2)
    assert rc == -6
