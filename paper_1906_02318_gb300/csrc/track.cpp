// Track preprocessing for the race car's safety test (Sec. V-C.1: the car is
// unsafe once it leaves the road).
//
// Safe iff the distance from the position to the closed centre-line polyline is
// below w (half width minus inflation).  The device must answer that for every
// candidate at every step, so the plane around the track is covered by a uniform
// grid whose cells are classified once, here, in float64:
//   inside    every point of the cell is within w - e of the centre line;
//   outside   every point of the cell is farther than w + e;
//   boundary  anything else; the cell keeps the list of segments within
//             w + r + e of its centre (r = half diagonal), nearest first.
// For a point p in a boundary cell the segment nearest to p is within
// w + r of the cell centre whenever p is safe, so the minimum over the list
// decides "< w" exactly as the minimum over all segments would.  The margin e
// also covers float32 rounding that puts a point into a neighbouring cell.
#include <math.h>

#include <algorithm>
#include <string>
#include <utility>
#include <vector>

#include "internal.h"

namespace mpmi {

static double seg_dist(double px, double py, double ax, double ay, double dx, double dy,
                       double inv) {
  const double rx = px - ax, ry = py - ay;
  double t = (rx * dx + ry * dy) * inv;
  t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
  const double ex = rx - t * dx, ey = ry - t * dy;
  return sqrt(ex * ex + ey * ey);
}

int build_track_grid(const double* xy, int n, double w, TrackGrid* g, std::string* err) {
  if (n < 3) {
    *err = "set_safety_set: a track needs at least 3 vertices";
    return MPMI_E_INVALID_ARG;
  }
  if (!(w > 0.0)) {
    *err = "set_safety_set: track half width minus inflation must be > 0";
    return MPMI_E_INVALID_ARG;
  }
  std::vector<double> ax(n), ay(n), dx(n), dy(n), inv(n);
  double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY, cmax = 0;
  for (int i = 0; i < n; ++i) {
    const double x0 = xy[2 * i], y0 = xy[2 * i + 1];
    const double x1 = xy[2 * ((i + 1) % n)], y1 = xy[2 * ((i + 1) % n) + 1];
    if (!isfinite(x0) || !isfinite(y0)) {
      *err = "set_safety_set: non-finite track vertex";
      return MPMI_E_NONFINITE;
    }
    ax[i] = x0; ay[i] = y0; dx[i] = x1 - x0; dy[i] = y1 - y0;
    const double l2 = dx[i] * dx[i] + dy[i] * dy[i];
    inv[i] = l2 > 0 ? 1.0 / l2 : 0.0;
    xmin = fmin(xmin, x0); xmax = fmax(xmax, x0);
    ymin = fmin(ymin, y0); ymax = fmax(ymax, y0);
    cmax = fmax(cmax, fmax(fabs(x0), fabs(y0)));
  }
  const double pad = w + 1.0;
  xmin -= pad; ymin -= pad; xmax += pad; ymax += pad;
  const double extent = fmax(xmax - xmin, ymax - ymin);
  double h = w / 2.0;
  if (extent / h > 1024.0) h = extent / 1024.0;
  const int gnx = (int)ceil((xmax - xmin) / h), gny = (int)ceil((ymax - ymin) / h);
  const double r = h * sqrt(2.0) / 2.0;
  const double e = 1e-3 + 2e-5 * (cmax + pad);
  g->gx0 = xmin; g->gy0 = ymin; g->h = h; g->gnx = gnx; g->gny = gny;
  g->cells.assign((size_t)gnx * gny, 0);
  g->list.clear();
  std::vector<std::pair<double, int>> near;
  for (int cy = 0; cy < gny; ++cy) {
    for (int cx = 0; cx < gnx; ++cx) {
      const double px = xmin + (cx + 0.5) * h, py = ymin + (cy + 0.5) * h;
      near.clear();
      double dmin = INFINITY;
      for (int i = 0; i < n; ++i) {
        const double d = seg_dist(px, py, ax[i], ay[i], dx[i], dy[i], inv[i]);
        dmin = fmin(dmin, d);
        if (d < w + r + e) near.emplace_back(d, i);
      }
      uint32_t word;
      if (dmin + r < w - e) {
        word = kCellInside;
      } else if (dmin - r > w + e) {
        word = kCellOutside;
      } else {
        std::sort(near.begin(), near.end());
        if (near.size() > 255 || g->list.size() + near.size() >= (1u << 22)) {
          *err = "set_safety_set: track too dense for the grid (segment list overflow)";
          return MPMI_E_UNSUPPORTED;
        }
        word = kCellBoundary | ((uint32_t)g->list.size() << 2) |
               ((uint32_t)near.size() << 24);
        for (auto& pr : near) g->list.push_back((uint16_t)pr.second);
      }
      g->cells[(size_t)cy * gnx + cx] = word;
    }
  }
  g->seg.resize(4 * (size_t)n);
  g->seg_inv.resize(n);
  for (int i = 0; i < n; ++i) {
    g->seg[4 * i + 0] = (float)ax[i];
    g->seg[4 * i + 1] = (float)ay[i];
    g->seg[4 * i + 2] = (float)dx[i];
    g->seg[4 * i + 3] = (float)dy[i];
    g->seg_inv[i] = (float)inv[i];
  }
  if (g->list.empty()) g->list.push_back(0);
  return MPMI_OK;
}

}  // namespace mpmi
