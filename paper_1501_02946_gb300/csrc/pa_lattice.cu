// pa_lattice.cu -- the spatial step for sensors exactly on the output lattice
// (x_m = (i - floor(nx/2)) dx, y_m = (k - floor(ny/2)) dy, one sensor per
// node).  There the non-uniform sum of the NED step is a plain DFT over the
// lattice (Sec. 2, the equispaced case the NER-only reconstruction uses), so
// no window spreading or deconvolution is needed: the data are placed on an
// nx x ny grid at p = i - floor(nx/2) (mod nx), q likewise, scaled by
// h_m/(dx dy), and transformed by the row and column FFT kernels at
// sigma = 1.  The adjoint gathers the grid back to the sensors.
//
// With sigma = 1 the spatial frequencies +nx/2 and -nx/2 of an even nx are
// the same DFT bin: the forward copies that bin's row of the half spectrum
// into the row of +nx/2 (which the Hermitian Nyquist handling reads), and
// the adjoint adds the cotangent of that row into the shared bin.
#include "pa_device.cuh"

namespace pa {

namespace {

constexpr int kThreadsLattice = 256;

// G0[pq[m]][n] = a[m] g[m][n]
__global__ void k_lattice_scatter(float *__restrict__ G0, const int *__restrict__ pq, const float *__restrict__ a,
                                  const float *__restrict__ g, int M, int Nt) {
  griddep_enter();  // the previous kernel of the stream has completed
  const size_t total = size_t(M) * Nt;
  const bool vec = (Nt & 3) == 0 && ((reinterpret_cast<uintptr_t>(g) & 15u) == 0);
  if (vec) {
    const int n4 = Nt >> 2;
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total / 4; i += size_t(gridDim.x) * blockDim.x) {
      const int m = int(i / n4), k = int(i - size_t(m) * n4);
      const float s = __ldg(a + m);
      const float4 v = __ldg(reinterpret_cast<const float4 *>(g) + i);
      reinterpret_cast<float4 *>(G0 + size_t(__ldg(pq + m)) * Nt)[k] = make_float4(s * v.x, s * v.y, s * v.z, s * v.w);
    }
  } else {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total; i += size_t(gridDim.x) * blockDim.x) {
      const int m = int(i / Nt), n = int(i - size_t(m) * Nt);
      G0[size_t(__ldg(pq + m)) * Nt + n] = __ldg(a + m) * __ldg(g + i);
    }
  }
}

// g[m][n] = a[m] G0b[pq[m]][n]
__global__ void k_lattice_gather(float *__restrict__ g, const float *__restrict__ G0, const int *__restrict__ pq,
                                 const float *__restrict__ a, int M, int Nt) {
  griddep_enter();  // the previous kernel of the stream has completed
  const size_t total = size_t(M) * Nt;
  const bool vec = (Nt & 3) == 0 && ((reinterpret_cast<uintptr_t>(g) & 15u) == 0);
  if (vec) {
    const int n4 = Nt >> 2;
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total / 4; i += size_t(gridDim.x) * blockDim.x) {
      const int m = int(i / n4), k = int(i - size_t(m) * n4);
      const float s = __ldg(a + m);
      const float4 v = __ldg(reinterpret_cast<const float4 *>(G0 + size_t(__ldg(pq + m)) * Nt) + k);
      reinterpret_cast<float4 *>(g)[i] = make_float4(s * v.x, s * v.y, s * v.z, s * v.w);
    }
  } else {
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < total; i += size_t(gridDim.x) * blockDim.x) {
      const int m = int(i / Nt), n = int(i - size_t(m) * Nt);
      g[i] = __ldg(a + m) * G0[size_t(__ldg(pq + m)) * Nt + n];
    }
  }
}

// Rows jx = -hx (index 0) and jx = +hx (index 2 hx) of the half spectrum
// G1[jx + hx][jy][n] are one bin at sigma = 1.  dir 0: copy 0 -> 2hx;
// dir 1: add the cotangent of 2hx into 0.
__global__ void k_lattice_alias(float2 *G1, int nY1, int Nt, int hx, int dir) {
  griddep_enter();  // the previous kernel of the stream has completed
  const size_t row = size_t(nY1) * Nt;
  float2 *r0 = G1, *r1 = G1 + size_t(2 * hx) * row;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < row; i += size_t(gridDim.x) * blockDim.x) {
    if (dir == 0) {
      r1[i] = r0[i];
    } else {
      r0[i] = cadd(r0[i], r1[i]);
    }
  }
}

int grid_for(size_t n) {
  const size_t b = (n + kThreadsLattice - 1) / kThreadsLattice;
  return int(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

}  // namespace

cudaError_t launch_lattice_scatter(float *G0, const int *pq, const float *a, const float *g, int M, int Nt,
                                   cudaStream_t s) {
  return launch_pdl(k_lattice_scatter, grid_for(size_t(M) * Nt / 4), kThreadsLattice, 0, s, G0, pq, a, g, M, Nt);
}

cudaError_t launch_lattice_gather(float *g, const float *G0, const int *pq, const float *a, int M, int Nt,
                                  cudaStream_t s) {
  return launch_pdl(k_lattice_gather, grid_for(size_t(M) * Nt / 4), kThreadsLattice, 0, s, g, G0, pq, a, M, Nt);
}

cudaError_t launch_lattice_alias(float2 *G1, int nY1, int Nt, int hx, int dir, cudaStream_t s) {
  return launch_pdl(k_lattice_alias, grid_for(size_t(nY1) * Nt), kThreadsLattice, 0, s, G1, nY1, Nt, hx, dir);
}

}  // namespace pa
