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
// The grid is packed into one blob that every block stages in shared memory;
// the cell size grows until the blob fits kMaxTrackBytes.
#include <math.h>
#include <string.h>

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

static size_t up16(size_t b) { return (b + 15) & ~(size_t)15; }

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
  const double e = 1e-3 + 2e-5 * (cmax + pad);
  std::vector<std::pair<double, int>> near;
  for (int attempt = 0; attempt < 12; ++attempt, h *= 1.25) {
    const int gnx = (int)ceil((xmax - xmin) / h), gny = (int)ceil((ymax - ymin) / h);
    const double r = h * sqrt(2.0) / 2.0;
    if (up16(4 * (size_t)gnx * gny) > (size_t)kMaxTrackBytes) continue;
    g->gx0 = xmin; g->gy0 = ymin; g->h = h; g->gnx = gnx; g->gny = gny;
    g->cells.assign((size_t)gnx * gny, 0);
    g->list.clear();
    bool overflow = false;
    for (int cy = 0; cy < gny && !overflow; ++cy) {
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
            overflow = true;
            break;
          }
          word = kCellBoundary | ((uint32_t)g->list.size() << 2) |
                 ((uint32_t)near.size() << 24);
          for (auto& pr : near) g->list.push_back((uint16_t)pr.second);
        }
        g->cells[(size_t)cy * gnx + cx] = word;
      }
    }
    if (overflow) continue;
    if (g->list.empty()) g->list.push_back(0);
    const size_t b_cells = up16(4 * g->cells.size());
    const size_t b_list = up16(2 * g->list.size());
    const size_t b_seg = 16 * (size_t)n, b_inv = up16(4 * (size_t)n);
    const size_t total = b_cells + b_list + b_seg + b_inv;
    if (total > (size_t)kMaxTrackBytes) continue;
    g->off_list = (int)b_cells;
    g->off_seg = (int)(b_cells + b_list);
    g->off_inv = (int)(b_cells + b_list + b_seg);
    g->blob.assign(total, 0);
    memcpy(g->blob.data(), g->cells.data(), 4 * g->cells.size());
    memcpy(g->blob.data() + g->off_list, g->list.data(), 2 * g->list.size());
    for (int i = 0; i < n; ++i) {
      const float sg[4] = {(float)ax[i], (float)ay[i], (float)dx[i], (float)dy[i]};
      memcpy(g->blob.data() + g->off_seg + 16 * (size_t)i, sg, 16);
      const float iv = (float)inv[i];
      memcpy(g->blob.data() + g->off_inv + 4 * (size_t)i, &iv, 4);
    }
    return MPMI_OK;
  }
  *err = "set_safety_set: track grid does not fit the shared-memory budget";
  return MPMI_E_UNSUPPORTED;
}

// Host mirror of the device's track test over a packed grid (the cell lookup
// and the listed-segment test, in float32), for checking the grid builder on
// machines without a GPU: on_road[i] = 1 iff point i is within the half width.
int track_query_host(const double* xy, int n, double half_width, const float* pts, int64_t np,
                     uint8_t* on_road, std::string* err) {
  TrackGrid g;
  const int rc = build_track_grid(xy, n, half_width, &g, err);
  if (rc != MPMI_OK) return rc;
  const uint8_t* base = g.blob.data();
  const uint32_t* cells = reinterpret_cast<const uint32_t*>(base);
  const uint16_t* list = reinterpret_cast<const uint16_t*>(base + g.off_list);
  const float* seg = reinterpret_cast<const float*>(base + g.off_seg);
  const float* inv = reinterpret_cast<const float*>(base + g.off_inv);
  const float gx0 = (float)g.gx0, gy0 = (float)g.gy0, inv_h = (float)(1.0 / g.h);
  const float w2 = (float)(half_width * half_width);
  for (int64_t i = 0; i < np; ++i) {
    const float px = pts[2 * i], py = pts[2 * i + 1];
    bool ok = false;
    const float fx = (px - gx0) * inv_h, fy = (py - gy0) * inv_h;
    if (fx >= 0.f && fx < (float)g.gnx && fy >= 0.f && fy < (float)g.gny) {
      const uint32_t c = cells[(int)fy * g.gnx + (int)fx];
      const uint32_t cls = c & 3u;
      if (cls == kCellInside) {
        ok = true;
      } else if (cls == kCellBoundary) {
        const int off = (int)((c >> 2) & 0x3FFFFFu), cnt = (int)(c >> 24);
        for (int k = 0; k < cnt && !ok; ++k) {
          const int s = list[off + k];
          const float* sg = seg + 4 * s;
          const float rx = px - sg[0], ry = py - sg[1];
          float t = (rx * sg[2] + ry * sg[3]) * inv[s];
          t = t < 0.f ? 0.f : (t > 1.f ? 1.f : t);
          const float ex = rx - t * sg[2], ey = ry - t * sg[3];
          ok = ex * ex + ey * ey < w2;
        }
      }
    }
    on_road[i] = ok ? 1 : 0;
  }
  return MPMI_OK;
}

}  // namespace mpmi
