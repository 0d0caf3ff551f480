// pa_metrics.cu -- the image quality measures of the paper's appendix on the
// device: the correlation coefficient rho(U1, U2) = Cov / sqrt(Var Var)
// (eq:corrcoeff; population moments, two passes: means, then centred sums)
// and the Tenenbaum sharpness F = sum (g * U)^2 + (g^T * U)^2 / N with g the
// 3x3 Sobel operator, over the pixels where the stencil lies inside each
// image of a stack U[n0][n1][n2] (images over the first two axes).
//
// Every sum accumulates in FP64: per thread, then per block (warp shuffles),
// then over the blocks' partials in block order by one block, so results do
// not depend on scheduling.  Scratch comes from the stream-ordered allocator.
#include <cmath>

#include "pa_device.cuh"
#include "pa_nufft.h"

namespace pa {

namespace {

constexpr int kMetricThreads = 256;
constexpr int kMetricBlocks = 1024;
constexpr int kSums = 3;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Block sums of the kSums values into part[blockIdx.x * kSums + k].
__device__ __forceinline__ void block_sums(double (&v)[kSums], double *part) {
  __shared__ double red[kMetricThreads / 32][kSums];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kSums; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < kSums; ++k) red[warp][k] = v[k];
  __syncthreads();
  if (threadIdx.x < kSums) {
    double s = 0.0;
    for (int w = 0; w < kMetricThreads / 32; ++w) s += red[w][threadIdx.x];
    part[blockIdx.x * kSums + threadIdx.x] = s;
  }
}

// pass 1 (centre = null): sums of a and b; pass 2: sums of (a - ma)(b - mb),
// (a - ma)^2, (b - mb)^2 with the means from pass 1's totals.
__global__ void __launch_bounds__(kMetricThreads) k_corr(const float *__restrict__ a, const float *__restrict__ b,
                                                         long long n, const double *__restrict__ totals,
                                                         double *part) {
  double v[kSums] = {0.0, 0.0, 0.0};
  const double ma = totals ? totals[0] / double(n) : 0.0, mb = totals ? totals[1] / double(n) : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double x = __ldg(a + i), y = __ldg(b + i);
    if (!totals) {
      v[0] += x;
      v[1] += y;
    } else {
      const double dx = x - ma, dy = y - mb;
      v[0] += dx * dy;
      v[1] += dx * dx;
      v[2] += dy * dy;
    }
  }
  block_sums(v, part);
}

__global__ void __launch_bounds__(kMetricThreads) k_tenenbaum(const float *__restrict__ u, long long n0, long long n1,
                                                              long long n2, double *part) {
  double v[kSums] = {0.0, 0.0, 0.0};
  const long long m1 = n1 - 2, total = (n0 - 2) * m1 * n2;
  const long long s0 = n1 * n2, s1 = n2;  // strides of the first two axes
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long k = t % n2, ij = t / n2;
    const long long i = 1 + ij / m1, j = 1 + ij % m1;
    const float *c = u + i * s0 + j * s1 + k;
    auto at = [&](int di, int dj) { return double(__ldg(c + di * s0 + dj * s1)); };
    const double gx = (at(-1, 1) - at(-1, -1)) + 2.0 * (at(0, 1) - at(0, -1)) + (at(1, 1) - at(1, -1));
    const double gy = (at(1, -1) - at(-1, -1)) + 2.0 * (at(1, 0) - at(-1, 0)) + (at(1, 1) - at(-1, 1));
    v[0] += gx * gx + gy * gy;
  }
  block_sums(v, part);
}

// totals[k] = sum over the blocks' partials, in block order.
__global__ void k_total(const double *__restrict__ part, int nblocks, double *totals) {
  if (threadIdx.x < kSums) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[b * kSums + threadIdx.x];
    totals[threadIdx.x] = s;
  }
}

int blocks_for(long long n) {
  const long long b = (n + kMetricThreads - 1) / kMetricThreads;
  return int(b < 1 ? 1 : (b > kMetricBlocks ? kMetricBlocks : b));
}

// One warp per sensor: grad_h[m] = inv_h[m] sum_n g[m][n] gb[m][n].
__global__ void k_weight_grad(const float *__restrict__ g, const float *__restrict__ gb,
                              const float *__restrict__ inv_h, int M, int Nt, float *grad_h) {
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= M) return;
  const float *a = g + w * Nt, *b = gb + w * Nt;
  double s = 0.0;
  for (int n = lane; n < Nt; n += 32) s += double(__ldg(a + n)) * double(__ldg(b + n));
  s = warp_sum(s);
  if (lane == 0) grad_h[w] = float(s * double(__ldg(inv_h + w)));
}

__global__ void k_ratio(WeightRescale r) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= r.M) return;
  const float hn = __ldg(r.h_new + m);
  r.ratio[m] = hn * r.inv_h[m];
  r.inv_h[m] = 1.f / hn;
  if (r.lat_amp) r.lat_amp[m] *= r.ratio[m];
}

__global__ void k_scale_sorted(WeightRescale r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= r.M) return;
  const float q = r.ratio[__ldg(r.perm + i)];
  for (int t = 0; t < r.w; ++t) {
    r.wy[(size_t)i * r.w + t] *= q;
    r.dwy[(size_t)i * r.w + t] *= q;
  }
}

__global__ void k_scale_entries(WeightRescale r) {
  for (size_t e = blockIdx.x * size_t(blockDim.x) + threadIdx.x; e < r.n_entries; e += size_t(gridDim.x) * blockDim.x) {
    const float q = r.ratio[__ldg(r.sp_m + e)];
    float4 v = r.sp_w[e];
    v.x *= q;
    v.y *= q;
    v.z *= q;
    v.w *= q;
    r.sp_w[e] = v;
  }
}

}  // namespace

cudaError_t rescale_weights(const WeightRescale &r, cudaStream_t s) {
  const int b = (r.M + 255) / 256;
  k_ratio<<<b, 256, 0, s>>>(r);
  k_scale_sorted<<<b, 256, 0, s>>>(r);
  if (r.n_entries) {
    const size_t be = (r.n_entries + 255) / 256;
    k_scale_entries<<<int(be < 4096 ? be : 4096), 256, 0, s>>>(r);
  }
  return cudaGetLastError();
}

cudaError_t launch_weight_grad(const float *g, const float *gb, const float *inv_h, int M, int Nt, float *grad_h,
                               cudaStream_t s) {
  const long long threads = (long long)M * 32;
  k_weight_grad<<<int((threads + kMetricThreads - 1) / kMetricThreads), kMetricThreads, 0, s>>>(g, gb, inv_h, M, Nt,
                                                                                               grad_h);
  return cudaGetLastError();
}

}  // namespace pa

namespace {
int metric_fail(int code, const char *msg) { return pa::set_error(code, msg); }

// scratch: partials of up to kMetricBlocks blocks, then two totals vectors
struct MetricScratch {
  double *p = nullptr;
  cudaStream_t s = nullptr;
  ~MetricScratch() {
    if (p) cudaFreeAsync(p, s);
  }
};
}  // namespace

extern "C" int pa_correlation(const float *a_dev, const float *b_dev, int64_t n, double *rho, void *stream) {
  pa::set_error(PA_OK, "");
  if (!a_dev || !b_dev || !rho || n < 2) return metric_fail(PA_ERR_INVALID_ARG, "pa_correlation: bad arguments");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  MetricScratch sc;
  sc.s = s;
  const size_t nd = size_t(pa::kMetricBlocks) * pa::kSums + 2 * pa::kSums;
  if (cudaMallocAsync(reinterpret_cast<void **>(&sc.p), nd * sizeof(double), s) != cudaSuccess)
    return metric_fail(PA_ERR_OOM, "pa_correlation: scratch allocation failed");
  double *part = sc.p, *t1 = sc.p + size_t(pa::kMetricBlocks) * pa::kSums, *t2 = t1 + pa::kSums;
  const int nb = pa::blocks_for(n);
  pa::k_corr<<<nb, pa::kMetricThreads, 0, s>>>(a_dev, b_dev, n, nullptr, part);
  pa::k_total<<<1, 32, 0, s>>>(part, nb, t1);
  pa::k_corr<<<nb, pa::kMetricThreads, 0, s>>>(a_dev, b_dev, n, t1, part);
  pa::k_total<<<1, 32, 0, s>>>(part, nb, t2);
  double h[pa::kSums];
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, t2, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return metric_fail(PA_ERR_CUDA, cudaGetErrorString(e));
  *rho = h[0] / std::sqrt(h[1] * h[2]);
  return PA_OK;
}

extern "C" int pa_tenenbaum(const float *u_dev, int64_t n0, int64_t n1, int64_t n2, double *value, void *stream) {
  pa::set_error(PA_OK, "");
  if (!u_dev || !value || n0 < 3 || n1 < 3 || n2 < 1)
    return metric_fail(PA_ERR_INVALID_ARG, "pa_tenenbaum: bad arguments (images need n0, n1 >= 3)");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  MetricScratch sc;
  sc.s = s;
  const size_t nd = size_t(pa::kMetricBlocks) * pa::kSums + pa::kSums;
  if (cudaMallocAsync(reinterpret_cast<void **>(&sc.p), nd * sizeof(double), s) != cudaSuccess)
    return metric_fail(PA_ERR_OOM, "pa_tenenbaum: scratch allocation failed");
  double *part = sc.p, *tot = sc.p + size_t(pa::kMetricBlocks) * pa::kSums;
  const int nb = pa::blocks_for((n0 - 2) * (n1 - 2) * n2);
  pa::k_tenenbaum<<<nb, pa::kMetricThreads, 0, s>>>(u_dev, n0, n1, n2, part);
  pa::k_total<<<1, 32, 0, s>>>(part, nb, tot);
  double h[pa::kSums];
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, tot, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return metric_fail(PA_ERR_CUDA, cudaGetErrorString(e));
  *value = h[0] / (double(n0) * double(n1) * double(n2));
  return PA_OK;
}
