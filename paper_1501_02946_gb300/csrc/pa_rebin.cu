// pa_rebin.cu -- plan setup for new sensor positions on the device: the
// positions reduced modulo (X, Y) and split into oversampled base cells and
// fractions in FP64, the counting sort of the sensors by cell, the window
// taps and their derivatives, and the spread entry lists per (strip, column)
// -- the same tables the host builds at plan creation, in the same order.
//
// Order: within a cell the sensors keep their caller order; within an entry
// list the sensors follow the host's walk (bin row of the strip's candidate
// rows, then sorted sensor index).  Atomic placement is followed by a sort of
// each (short) cell or list, so the result does not depend on scheduling.
#include "pa_device.cuh"

namespace pa {

namespace {

constexpr int kRebinThreads = 256;

// Modified Bessel functions by their power series (all terms positive).
__device__ double d_bessel_i0(double z) {
  const double q = 0.25 * z * z;
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 500; ++k) {
    term *= q / (double(k) * double(k));
    sum += term;
    if (term < 1e-17 * sum) break;
  }
  return sum;
}
__device__ double d_bessel_i1(double z) {
  const double q = 0.25 * z * z;
  double term = 0.5 * z, sum = term;
  for (int k = 1; k < 500; ++k) {
    term *= q / (double(k) * double(k + 1));
    sum += term;
    if (fabs(term) < 1e-17 * fabs(sum)) break;
  }
  return sum;
}
// Kaiser-Bessel window of w taps with phi(0) = 1, and its derivative.
__device__ double d_kb_phi(double x, int w, double beta, double phi0) {
  const double t = 1.0 - (2.0 * x / w) * (2.0 * x / w);
  if (t < 0.0) return 0.0;
  return d_bessel_i0(beta * sqrt(t)) / phi0;
}
__device__ double d_kb_dphi(double x, int w, double beta, double phi0) {
  const double t = 1.0 - (2.0 * x / w) * (2.0 * x / w);
  if (t <= 0.0) return 0.0;
  const double s = sqrt(t);
  return d_bessel_i1(beta * s) * beta * (-4.0 * x / (double(w) * w)) / s / phi0;
}

__global__ void k_rb_coords(RebinArgs a) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= a.M) return;
  double x = a.xy[2 * m], y = a.xy[2 * m + 1];
  if (!isfinite(x) || !isfinite(y)) {
    atomicOr(a.status, kStatusBadPositions);
    x = 0.0;
    y = 0.0;
  }
  double ux = x / a.X, uy = y / a.Y;
  ux -= floor(ux + 0.5);
  uy -= floor(uy + 0.5);
  a.pos[m] = make_double2(ux * a.X, uy * a.Y);
  const double Ux = a.Mx * ux, Uy = a.My * uy;
  const double fbx = floor(Ux), fby = floor(Uy);
  a.frx[m] = Ux - fbx;
  a.fry[m] = Uy - fby;
  const int bx = ((int(fbx) % a.Mx) + a.Mx) % a.Mx, by = ((int(fby) % a.My) + a.My) % a.My;
  a.bx[m] = bx;
  a.by[m] = by;
  atomicAdd(a.cell_start + (size_t)bx * a.My + by + 1, 1);
}

// In-place inclusive scan of v[0..n) by one block (v[0] = 0 on entry makes it
// the exclusive offsets of the counts in v[1..n)).
__global__ void k_rb_scan(int *v, int n) {
  __shared__ int part[kRebinThreads];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int chunk = (n + nthr - 1) / nthr;
  const int lo = min(n, tid * chunk), hi = min(n, lo + chunk);
  int s = 0;
  for (int i = lo; i < hi; ++i) s += v[i];
  part[tid] = s;
  __syncthreads();
  if (tid == 0)
    for (int i = 1; i < nthr; ++i) part[i] += part[i - 1];
  __syncthreads();
  int run = tid == 0 ? 0 : part[tid - 1];
  for (int i = lo; i < hi; ++i) {
    run += v[i];
    v[i] = run;
  }
}

__global__ void k_rb_scatter(RebinArgs a) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= a.M) return;
  const size_t cell = (size_t)a.bx[m] * a.My + a.by[m];
  a.perm[a.cell_start[cell] + atomicAdd(a.fill + cell, 1)] = m;
}

// Sensors of a cell in caller order (insertion sort of a short run).
__global__ void k_rb_sort_cells(RebinArgs a, int ncell) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int lo = a.cell_start[c], hi = a.cell_start[c + 1];
  for (int i = lo + 1; i < hi; ++i) {
    const int v = a.perm[i];
    int j = i - 1;
    while (j >= lo && a.perm[j] > v) {
      a.perm[j + 1] = a.perm[j];
      --j;
    }
    a.perm[j + 1] = v;
  }
}

__global__ void k_rb_taps(RebinArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.M) return;
  const int m = a.perm[i];
  const int w = a.w;
  a.sbx[i] = a.bx[m];
  a.sby[i] = a.by[m];
  const double amp = a.weights[m] * a.ax;
  for (int t = 0; t < w; ++t) {
    const double ddx = a.frx[m] + 0.5 * w - 1.0 - t;
    const double ddy = a.fry[m] + 0.5 * w - 1.0 - t;
    a.wx[(size_t)i * w + t] = float(d_kb_phi(ddx, w, a.beta, a.phi0));
    a.wy[(size_t)i * w + t] = float(amp * d_kb_phi(ddy, w, a.beta, a.phi0));
    a.dwx[(size_t)i * w + t] = float(d_kb_dphi(ddx, w, a.beta, a.phi0) * a.Mx / a.X);
    a.dwy[(size_t)i * w + t] = float(amp * d_kb_dphi(ddy, w, a.beta, a.phi0) * a.My / a.Y);
  }
}

// Visit the spread entries of sorted sensor i: for every strip its w-row
// footprint meets, the tap products of the strip's rows and each of its w
// columns.  fn(strip, column, key, products) with key the host's walk order.
template <typename Fn>
__device__ __forceinline__ void for_each_entry(const RebinArgs &a, int i, Fn fn) {
  const int w = a.w, Mx = a.Mx, My = a.My, P = kSpreadP;
  const int bx = a.sbx[i], by = a.sby[i];
  const float *wxi = a.wx + (size_t)i * w;
  const float *wyi = a.wy + (size_t)i * w;
  const int nrows = min(P + w - 1, Mx);
  for (int st = 0; st < a.nstrips; ++st) {
    const int p0 = st * P;
    // the strip takes this sensor when its base row is one of the strip's
    // candidate rows p0 - w/2 + dr, dr < nrows (mod Mx)
    const int dr = ((bx - (p0 - w / 2)) % Mx + Mx) % Mx;
    if (dr >= nrows) continue;
    float wxr[P];
    bool any = false;
    for (int r = 0; r < P; ++r) {
      const int p = p0 + r;
      const int tx = ((p - bx + w / 2 - 1) % Mx + Mx) % Mx;
      const bool in = tx < w && p < Mx;
      wxr[r] = in ? wxi[tx] : 0.f;
      any = any || in;
    }
    if (!any) continue;
    const long long key = (long long)dr * a.M + i;
    const int q0 = by - w / 2 + 1;
    for (int t = 0; t < w; ++t) {
      const int q = ((q0 + t) % My + My) % My;
      const float wyq = wyi[t];
      fn(st, q, key, make_float4(wyq * wxr[0], wyq * wxr[1], wyq * wxr[2], wyq * wxr[3]));
    }
  }
}

__global__ void k_rb_entry_count(RebinArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.M) return;
  for_each_entry(a, i, [&](int st, int q, long long, float4) {
    atomicAdd(a.sp_cnt + (size_t)st * a.My + q + 1, 1);
  });
}

__global__ void k_rb_entry_fill(RebinArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.M) return;
  const int m = a.perm[i];
  for_each_entry(a, i, [&](int st, int q, long long key, float4 pw) {
    const size_t k = (size_t)st * a.My + q;
    const int e = a.sp_cnt[k] + atomicAdd(a.fill + k, 1);
    a.sp_m[e] = m;
    a.sp_w[e] = pw;
    a.sp_key[e] = key;
  });
}

// Each entry list in the host's order (insertion sort of a short run).
__global__ void k_rb_sort_entries(RebinArgs a, int nkeys) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nkeys) return;
  const int lo = a.sp_cnt[k], hi = a.sp_cnt[k + 1];
  for (int i = lo + 1; i < hi; ++i) {
    const long long key = a.sp_key[i];
    const int m = a.sp_m[i];
    const float4 pw = a.sp_w[i];
    int j = i - 1;
    while (j >= lo && a.sp_key[j] > key) {
      a.sp_key[j + 1] = a.sp_key[j];
      a.sp_m[j + 1] = a.sp_m[j];
      a.sp_w[j + 1] = a.sp_w[j];
      --j;
    }
    a.sp_key[j + 1] = key;
    a.sp_m[j + 1] = m;
    a.sp_w[j + 1] = pw;
  }
}

int nblk(long long n) { return int((n + kRebinThreads - 1) / kRebinThreads); }

}  // namespace

cudaError_t rebin_sensors(const RebinArgs &a, cudaStream_t s) {
  const int ncell = a.Mx * a.My;
  cudaError_t e;
  if ((e = cudaMemsetAsync(a.cell_start, 0, sizeof(int) * (size_t(ncell) + 1), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.fill, 0, sizeof(int) * size_t(ncell), s)) != cudaSuccess) return e;
  k_rb_coords<<<nblk(a.M), kRebinThreads, 0, s>>>(a);
  k_rb_scan<<<1, kRebinThreads, 0, s>>>(a.cell_start, ncell + 1);
  k_rb_scatter<<<nblk(a.M), kRebinThreads, 0, s>>>(a);
  k_rb_sort_cells<<<nblk(ncell), kRebinThreads, 0, s>>>(a, ncell);
  k_rb_taps<<<nblk(a.M), kRebinThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t rebin_count_entries(const RebinArgs &a, cudaStream_t s) {
  const int nkeys = a.nstrips * a.My;
  cudaError_t e;
  if ((e = cudaMemsetAsync(a.sp_cnt, 0, sizeof(int) * (size_t(nkeys) + 1), s)) != cudaSuccess) return e;
  k_rb_entry_count<<<nblk(a.M), kRebinThreads, 0, s>>>(a);
  k_rb_scan<<<1, kRebinThreads, 0, s>>>(a.sp_cnt, nkeys + 1);
  return cudaGetLastError();
}

cudaError_t rebin_fill_entries(const RebinArgs &a, cudaStream_t s) {
  const int nkeys = a.nstrips * a.My;
  cudaError_t e;
  if ((e = cudaMemsetAsync(a.fill, 0, sizeof(int) * size_t(nkeys), s)) != cudaSuccess) return e;
  k_rb_entry_fill<<<nblk(a.M), kRebinThreads, 0, s>>>(a);
  k_rb_sort_entries<<<nblk(nkeys), kRebinThreads, 0, s>>>(a, nkeys);
  return cudaGetLastError();
}

}  // namespace pa
