// mppi_shapes.cu - host helper: an oriented rectangular object covered by circles, the form
// the obstacle term takes its obstacles in (arXiv 2308.01654, Sec. III-C, Fig. 3; Algorithm 1,
// ApproximateObstacles).  Host code only: it runs once per object before a plan.
#include <math.h>

#include "mppi.h"

extern "C" int32_t mppi_box_to_circles(double x, double y, double yaw, double length, double width, double vx,
                                       double vy, int32_t n, mppi_circle* out, int32_t max_out) {
    const double v[] = {x, y, yaw, length, width, vx, vy};
    for (double a : v)
        if (!isfinite(a)) return MPPI_ERR_ARG;
    if (!(length > 0.0) || !(width > 0.0) || n < 0 || max_out < 0 || (max_out > 0 && !out)) return MPPI_ERR_ARG;
    if (n == 0) {
        const double q = ceil(length / width - 1e-12);   // slices about as long as the object is wide
        n = q < 1.0 ? 1 : (q > 1e6 ? 1000000 : (int32_t)q);
    }
    if (n > max_out) return MPPI_ERR_CAPACITY;
    // n equal slices along the heading; each slice (length/n x width) lies inside the circle
    // through its four corners, centred on the centre line
    const double c = cos(yaw), s = sin(yaw);
    const double h = 0.5 * length / n;
    const double r = sqrt(h * h + 0.25 * width * width);
    for (int32_t i = 0; i < n; ++i) {
        const double o = (2.0 * i + 1.0) * h - 0.5 * length;   // slice centre along the heading
        out[i].x = x + o * c;
        out[i].y = y + o * s;
        out[i].r = r;
        out[i].vx = vx;
        out[i].vy = vy;
    }
    return n;
}
