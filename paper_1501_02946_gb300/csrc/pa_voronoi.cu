// pa_voronoi.cu -- detector weights h_m from the sensor positions (the
// areas h_m of eq:disc_rec, Sec. 2: sum h_m = X^(d-1)) as Voronoi cells of
// the periodic sensor set, and their derivatives for the chain rule.
//
// The sums of eq:disc_rec are X- and Y-periodic, so the tessellation is the
// one of the torus X x Y (the periodic images of every sensor take part):
//   3-D plans: h_m = area of the cell of (x_m, y_m); one thread per sensor
//     clips the rectangle [-X/2, X/2] x [-Y/2, Y/2] around it (the bisectors
//     with its own images) by the bisectors with the other sensors' images,
//     taken ring by ring over the plan's oversampled binning cells, until the
//     ring is farther than twice the polygon's farthest vertex (no bisector
//     beyond can cut it).  FP64 relative coordinates.
//   2-D plans: h_m = (right neighbour - left neighbour) / 2 on the circle X.
// Gradient: with edge (m, k) of length l at distance d = |x_k - x_m| and
// midpoint p, dA_m/dx_k = (l/d)(x_k - p) and dA_m/dx_m = sum_k (l/d)(p - x_m);
// gathered per sensor over its own edges:
//   dL/dx_m += sum_k (l/d)(p - x_m) (grad_h[m] - grad_h[k]).
// In 2-D: dL/dx_m += (grad_h[left] - grad_h[right]) / 2.
// Every loop is bounded (rings by the grid size, vertices by kVorMaxV, with
// kStatusVoronoi set when a cell outgrows the vertex buffer).
#include "pa_device.cuh"

namespace pa {

namespace {

constexpr int kVorThreads = 128;
constexpr int kVorMaxV = 48;

struct VorArgs {
  int M, Mx, My;
  double X, Y;
  const double2 *pos;      // [M] caller order, reduced into [-X/2, X/2) x [-Y/2, Y/2)
  const int *perm, *sbx, *sby, *cell_start;
  float *h;                // [M] output (weights) or null
  const float *grad_h;     // [M] input (gradient) or null
  float *grad_xy;          // [M][2] accumulated (gradient) or null
  int *status;
};

// Cell of sensor m (sorted index i) clipped in place; returns the vertex
// count (0 when the buffer overflowed).  vx, vy relative to pos[m]; lab[e] =
// caller index of the sensor whose bisector carries edge e (from vertex e to
// e + 1), or -1 for the sensor's own images.
__device__ int voronoi_cell(const VorArgs &a, int i, double *vx, double *vy, int *lab) {
  const int m = __ldg(a.perm + i);
  const double2 x0 = a.pos[m];
  const double hX = 0.5 * a.X, hY = 0.5 * a.Y;
  int nv = 4;
  vx[0] = -hX, vy[0] = -hY, vx[1] = hX, vy[1] = -hY, vx[2] = hX, vy[2] = hY, vx[3] = -hX, vy[3] = hY;
  lab[0] = lab[1] = lab[2] = lab[3] = -1;
  double r2 = hX * hX + hY * hY;
  const double csx = a.X / a.Mx, csy = a.Y / a.My, cs = fmin(csx, csy);
  const int bx = __ldg(a.sbx + i), by = __ldg(a.sby + i);
  const int rmax = (max(a.Mx, a.My) + 1) / 2 + 1;
  double tx[kVorMaxV], ty[kVorMaxV];
  int tl[kVorMaxV];
  for (int r = 0; r <= rmax; ++r) {
    if (r >= 2 && double(r - 1) * cs > 2.0 * sqrt(r2)) break;
    for (int dy = -r; dy <= r; ++dy) {
      const int step = (dy == -r || dy == r) ? 1 : 2 * r;  // the ring's cells only
      for (int dx = -r; dx <= r; dx += (step > 0 ? step : 1)) {
        const int cx = wrap(bx + dx, a.Mx), cy = wrap(by + dy, a.My);
        const int c = cx * a.My + cy;
        const int k1 = __ldg(a.cell_start + c + 1);
        for (int j = __ldg(a.cell_start + c); j < k1; ++j) {
          const int k = __ldg(a.perm + j);
          const double2 xk = a.pos[k];
          // the image of k that sits near the cell offset (dx, dy)
          double px = xk.x - x0.x, py = xk.y - x0.y;
          px -= a.X * floor((px - (dx * csx)) / a.X + 0.5);
          py -= a.Y * floor((py - (dy * csy)) / a.Y + 0.5);
          const double d2 = px * px + py * py;
          if (d2 == 0.0) continue;  // the sensor itself (or a coincident one)
          if (d2 > 4.0 * r2) continue;
          // keep q with q . p <= |p|^2 / 2 (Sutherland-Hodgman on one half-plane)
          const double lim = 0.5 * d2;
          int nt = 0;
          bool over = false;
          for (int e = 0; e < nv; ++e) {
            const int f = e + 1 == nv ? 0 : e + 1;
            const double se = vx[e] * px + vy[e] * py - lim, sf = vx[f] * px + vy[f] * py - lim;
            if (se <= 0.0) {
              if (nt >= kVorMaxV) { over = true; break; }
              tx[nt] = vx[e], ty[nt] = vy[e], tl[nt] = lab[e];
              ++nt;
            }
            if ((se <= 0.0) != (sf <= 0.0)) {
              const double t = se / (se - sf);
              if (nt >= kVorMaxV) { over = true; break; }
              tx[nt] = vx[e] + t * (vx[f] - vx[e]);
              ty[nt] = vy[e] + t * (vy[f] - vy[e]);
              // the edge leaving a vertex that enters the half-plane lies on the bisector
              tl[nt] = se <= 0.0 ? k : lab[e];
              ++nt;
            }
          }
          if (over) {
            atomicOr(a.status, kStatusVoronoi);
            return 0;
          }
          nv = nt;
          r2 = 0.0;
          for (int e = 0; e < nv; ++e) {
            vx[e] = tx[e], vy[e] = ty[e], lab[e] = tl[e];
            r2 = fmax(r2, vx[e] * vx[e] + vy[e] * vy[e]);
          }
        }
      }
    }
  }
  return nv;
}

__global__ void __launch_bounds__(kVorThreads) k_voronoi_2d(VorArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.M) return;
  double vx[kVorMaxV], vy[kVorMaxV];
  int lab[kVorMaxV];
  const int nv = voronoi_cell(a, i, vx, vy, lab);
  const int m = __ldg(a.perm + i);
  if (nv == 0) return;
  if (a.h) {
    double s = 0.0;
    for (int e = 0; e < nv; ++e) {
      const int f = e + 1 == nv ? 0 : e + 1;
      s += vx[e] * vy[f] - vx[f] * vy[e];
    }
    a.h[m] = float(0.5 * s);
  }
  if (a.grad_h) {
    const double gm = __ldg(a.grad_h + m);
    double gx = 0.0, gy = 0.0;
    for (int e = 0; e < nv; ++e) {
      const int k = lab[e];
      if (k < 0) continue;
      const int f = e + 1 == nv ? 0 : e + 1;
      const double ex = vx[f] - vx[e], ey = vy[f] - vy[e];
      const double l = sqrt(ex * ex + ey * ey);
      const double mx = 0.5 * (vx[e] + vx[f]), my = 0.5 * (vy[e] + vy[f]);
      // the neighbour's image sits at twice the foot of the perpendicular:
      // d = 2 |projection of the midpoint on the edge normal|
      const double nx = ey, ny = -ex;  // a normal of the edge
      const double nn = sqrt(nx * nx + ny * ny);
      const double d = nn > 0.0 ? 2.0 * fabs(mx * nx + my * ny) / nn : 0.0;
      if (!(d > 0.0)) continue;
      const double w = (l / d) * (gm - double(__ldg(a.grad_h + k)));
      gx += w * mx;
      gy += w * my;
    }
    a.grad_xy[2 * m] += float(gx);
    a.grad_xy[2 * m + 1] += float(gy);
  }
}

// 2-D plans: neighbours on the circle X (positions (x_m, 0), My = 1).
__global__ void __launch_bounds__(kVorThreads) k_voronoi_1d(VorArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.M) return;
  const int m = __ldg(a.perm + i);
  const double x0 = a.pos[m].x;
  // nearest on each side (ties broken by caller index); full scan of the
  // binning cells outward until both sides are found (bounded by Mx cells)
  double dl = a.X, dr = a.X;
  int kl = m, kr = m;
  const int bx = __ldg(a.sbx + i);
  const double cs = a.X / a.Mx;
  for (int r = 0; r <= a.Mx / 2 + 1; ++r) {
    if (double(r - 1) * cs > fmax(dl, dr) && r >= 2) break;
    for (int s = -1; s <= 1; s += 2) {
      if (r == 0 && s == 1) continue;
      const int c = wrap(bx + s * r, a.Mx);
      const int k1 = __ldg(a.cell_start + c + 1);
      for (int j = __ldg(a.cell_start + c); j < k1; ++j) {
        const int k = __ldg(a.perm + j);
        if (k == m) continue;
        double p = a.pos[k].x - x0;
        p -= a.X * floor(p / a.X + 0.5);  // nearest image, in [-X/2, X/2)
        const bool right = p > 0.0 || (p == 0.0 && k > m);
        const double q = fabs(p);
        if (right) {
          if (q < dr || (q == dr && k < kr)) dr = q, kr = k;
        } else {
          if (q < dl || (q == dl && k < kl)) dl = q, kl = k;
        }
      }
    }
  }
  if (a.h) a.h[m] = float(0.5 * (dl + dr));
  if (a.grad_h) {
    // h_m = (x_right - x_left)/2: dh_left/dx_m = 1/2 (m is its right
    // neighbour), dh_right/dx_m = -1/2
    a.grad_xy[2 * m] += float(0.5 * (double(__ldg(a.grad_h + kl)) - double(__ldg(a.grad_h + kr))));
  }
}

}  // namespace

cudaError_t launch_voronoi(const VoronoiLaunch &v, cudaStream_t s) {
  VorArgs a{};
  a.M = v.M;
  a.Mx = v.Mx;
  a.My = v.My;
  a.X = v.X;
  a.Y = v.Y;
  a.pos = v.pos;
  a.perm = v.perm;
  a.sbx = v.sbx;
  a.sby = v.sby;
  a.cell_start = v.cell_start;
  a.h = v.h;
  a.grad_h = v.grad_h;
  a.grad_xy = v.grad_xy;
  a.status = v.status;
  const int blocks = (v.M + kVorThreads - 1) / kVorThreads;
  if (v.line) {
    k_voronoi_1d<<<blocks, kVorThreads, 0, s>>>(a);
  } else {
    k_voronoi_2d<<<blocks, kVorThreads, 0, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace pa
