// pa_d2.cu -- the spatial step of the d = 2 operator (Sec. 2 with d - 1 = 1:
// sensors on the line z = 0 at x_m, images f[x][z]).
//
// A 2-D plan is the 3-D plan with Ny = 1 and no oversampling or window in y
// (My = 1, jy = 0 only): the column FFT over x, the NER stage and the inverse
// x DFT run unchanged on the single jy column.  These kernels replace the
// stages that involve y:
//   k_spread_x  T[p][0][n] = (sum_m a_m wx_m(p) g[m][n], 0)   1-D window spread
//               (gather form: a warp owns a strip of 4 grid rows and 128
//               samples and walks the sensors whose base row is within reach)
//   k_interp_x  g'[m][n] = a_m sum_t wx_m(t) Re T[bx_m - w/2 + 1 + t][0][n]
//               (its transpose), with the window-derivative partials of the
//               position gradient (d/dx_m only)
//   k_real_out  f[x][z] = Re U[x][0][z]      (the real inverse DFT over the
//               single jy = 0 bin)
//   k_real_in   U[x][0][z] = (f[x][z], 0)    (its transpose)
// a_m = h_m/dx is kept in tap 0 of the plan's wy table.
#include "pa_device.cuh"

namespace pa {

namespace {

constexpr int kD2Rows = 4;      // grid rows per spread strip
constexpr int kD2Samples = 4;   // samples per lane in the spread
constexpr int kD2Threads = 256;

__global__ void __launch_bounds__(kD2Threads) k_spread_x(const InstDesc *__restrict__ descs, IoPtrs io) {
  griddep_enter();  // the previous kernel of the stream has completed
  const InstDesc &d = descs[0];
  const int Mx = d.Mx, Nt = d.Nt, w = d.w;
  const int nstrips = (Mx + kD2Rows - 1) / kD2Rows;
  constexpr int CH = 32 * kD2Samples;
  const int nch = (Nt + CH - 1) / CH;
  const int gw = int((blockIdx.x * size_t(blockDim.x) + threadIdx.x) >> 5);
  if (gw >= nstrips * nch) return;  // whole warps leave; no block barrier
  const int st = gw % nstrips, c = gw / nstrips;
  const int lane = threadIdx.x & 31;
  const int p0 = st * kD2Rows, n = c * CH + lane * kD2Samples;
  const float *__restrict__ g = io.g_in;
  const bool vec = (Nt & 3) == 0 && (reinterpret_cast<uintptr_t>(g) & 15u) == 0 && n + kD2Samples <= Nt;
  float acc[kD2Rows][kD2Samples];
#pragma unroll
  for (int r = 0; r < kD2Rows; ++r)
#pragma unroll
    for (int u = 0; u < kD2Samples; ++u) acc[r][u] = 0.f;
  // a sensor with base row b covers rows b - w/2 + 1 .. b + w/2 (mod Mx): the
  // strip's rows p0 .. p0 + 3 are reached from b in [p0 - w/2, p0 + 3 + w/2 - 1]
  for (int b = p0 - w / 2; b <= p0 + kD2Rows - 1 + w / 2 - 1; ++b) {
    const int row = wrap(b, Mx);
    const int i1 = __ldg(d.cell_start + row + 1);
    for (int i = __ldg(d.cell_start + row); i < i1; ++i) {
      const int m = __ldg(d.perm + i);
      const float a = __ldg(d.wy + (size_t)i * w);
      float wr[kD2Rows];
#pragma unroll
      for (int r = 0; r < kD2Rows; ++r) {
        const int t = p0 + r - (b - w / 2 + 1);
        wr[r] = (t >= 0 && t < w && p0 + r < Mx) ? a * __ldg(d.wx + (size_t)i * w + t) : 0.f;
      }
      float v[kD2Samples];
      const float *row_g = g + (size_t)m * Nt + n;
      if (vec) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(row_g));
        v[0] = q.x;
        v[1] = q.y;
        v[2] = q.z;
        v[3] = q.w;
      } else {
#pragma unroll
        for (int u = 0; u < kD2Samples; ++u) v[u] = n + u < Nt ? __ldg(row_g + u) : 0.f;
      }
#pragma unroll
      for (int r = 0; r < kD2Rows; ++r)
#pragma unroll
        for (int u = 0; u < kD2Samples; ++u) acc[r][u] = fmaf(wr[r], v[u], acc[r][u]);
    }
  }
#pragma unroll
  for (int r = 0; r < kD2Rows; ++r) {
    const int p = p0 + r;
    if (p >= Mx) break;
    float2 *dst = d.T + (size_t)p * Nt + n;  // nY1 = 1
#pragma unroll
    for (int u = 0; u < kD2Samples; ++u)
      if (n + u < Nt) dst[u] = make_float2(acc[r][u], 0.f);
  }
}

// One warp per (sorted sensor i, 32 samples), lane = sample.
template <bool GRAD>
__global__ void __launch_bounds__(kD2Threads) k_interp_x(const InstDesc *__restrict__ descs, IoPtrs io) {
  griddep_enter();  // the previous kernel of the stream has completed
  const InstDesc &d = descs[0];
  const int Mx = d.Mx, Nt = d.Nt, w = d.w, M = d.M;
  const int nch = (Nt + 31) / 32;
  const int gw = int((blockIdx.x * size_t(blockDim.x) + threadIdx.x) >> 5);
  if (gw >= M * nch) return;
  const int i = gw / nch, c = gw % nch;
  const int lane = threadIdx.x & 31, n = c * 32 + lane;
  const int m = __ldg(d.perm + i), bx = __ldg(d.sbx + i);
  const float a = __ldg(d.wy + (size_t)i * w);
  float s = 0.f, sd = 0.f;
  if (n < Nt) {
    for (int t = 0; t < w; ++t) {
      const float v = d.T[(size_t)wrap(bx - w / 2 + 1 + t, Mx) * Nt + n].x;
      s = fmaf(__ldg(d.wx + (size_t)i * w + t), v, s);
      if (GRAD) sd = fmaf(__ldg(d.dwx + (size_t)i * w + t), v, sd);
    }
    if (io.g_out) io.g_out[(size_t)m * Nt + n] = a * s;
  }
  if (GRAD) {
    float px = n < Nt ? a * sd * __ldg(io.g_in + (size_t)m * Nt + n) : 0.f;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) px += __shfl_xor_sync(0xffffffffu, px, off);
    if (lane == 0) d.grad_part[(size_t)c * M + i] = make_float2(px, 0.f);
  }
}

__global__ void k_real_out(const InstDesc *__restrict__ descs, IoPtrs io) {
  griddep_enter();  // the previous kernel of the stream has completed
  const InstDesc &d = descs[0];
  const size_t n = size_t(d.Nx) * d.Nz;
  for (size_t k = blockIdx.x * size_t(blockDim.x) + threadIdx.x; k < n; k += size_t(gridDim.x) * blockDim.x)
    io.f_out[k] = d.U[k].x;  // U[x][0][z], nY1 = 1
}

__global__ void k_real_in(const InstDesc *__restrict__ descs, IoPtrs io) {
  griddep_enter();  // the previous kernel of the stream has completed
  const InstDesc &d = descs[0];
  const size_t n = size_t(d.Nx) * d.Nz;
  for (size_t k = blockIdx.x * size_t(blockDim.x) + threadIdx.x; k < n; k += size_t(gridDim.x) * blockDim.x)
    d.U[k] = make_float2(io.f_in[k], 0.f);
}

int grid_of(size_t threads) {
  const size_t b = (threads + kD2Threads - 1) / kD2Threads;
  return int(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}

}  // namespace

cudaError_t launch_spread_x(const Launch &L, const InstDesc &h) {
  const size_t warps = size_t((h.Mx + kD2Rows - 1) / kD2Rows) * ((h.Nt + 32 * kD2Samples - 1) / (32 * kD2Samples));
  return launch_pdl(k_spread_x, int((warps * 32 + kD2Threads - 1) / kD2Threads), kD2Threads, 0, L.stream, L.descs, L.io);
}

cudaError_t launch_interp_x(const Launch &L, const InstDesc &h, bool grad) {
  const size_t warps = size_t(h.M) * ((h.Nt + 31) / 32);
  const int blocks = int((warps * 32 + kD2Threads - 1) / kD2Threads);
  return grad ? launch_pdl(k_interp_x<true>, blocks, kD2Threads, 0, L.stream, L.descs, L.io)
              : launch_pdl(k_interp_x<false>, blocks, kD2Threads, 0, L.stream, L.descs, L.io);
}

cudaError_t launch_real_out(const Launch &L, const InstDesc &h) {
  return launch_pdl(k_real_out, grid_of(size_t(h.Nx) * h.Nz), kD2Threads, 0, L.stream, L.descs, L.io);
}

cudaError_t launch_real_in(const Launch &L, const InstDesc &h) {
  return launch_pdl(k_real_in, grid_of(size_t(h.Nx) * h.Nz), kD2Threads, 0, L.stream, L.descs, L.io);
}

}  // namespace pa
