// pa_image.cu -- third step of the NEDNER-NUFFT (Sec. 3): the uniform
// inverse DFT in x and y that turns the half spectrum Fz[jx][jy][z] (already
// inverse-transformed over depth) into the real image f[x][y][z], and its
// exact transpose.
//
//   k_imgx  inverse DFT over jx (complex), x_p = (p - hx) dx as an index shift.
//   k_imgy  real inverse DFT over jy from the half spectrum jy = 0..hy; two
//           depth samples share one complex transform (one in the real, one in
//           the imaginary part).  Interior bins count twice, jy = 0 and the
//           even-length Nyquist bin once, each through its real part.
// Both keep depth innermost, so every global access is a contiguous run.
#include "pa_device.cuh"

namespace pa {

namespace {

constexpr int kThreadsImg = 256;

__device__ __forceinline__ IoPtrs io_of_img(const IoPtrs &io, const IoPtrs *table, int inst) {
  return table ? table[inst] : io;
}

// Forward: Fz[ix][iy][z] -> U[x][iy][z] = sum_jx Fz[jx + hx] e^{2 pi i jx (x - hx)/Nx}.
// Adjoint: U[x][iy][z] -> Fz[ix][iy][z] = sum_x U[x] e^{-2 pi i jx (x - hx)/Nx}.
template <bool ADJ>
__global__ void __launch_bounds__(kThreadsImg) k_imgx(const InstDesc *__restrict__ descs,
                                                      const int2 *__restrict__ work) {
  extern __shared__ float4 smem_f4[];
  float2 *buf = reinterpret_cast<float2 *>(smem_f4);
  int inst, tile;
  block_work(work, inst, tile);
  const InstDesc &d = descs[inst];
  const int Nx = d.Nx, Nz = d.Nz, nY1 = d.nY1, hx = d.hx;
  constexpr int ZC = kImgZC;
  const int nzc = (Nz + ZC - 1) / ZC;
  if (tile >= nY1 * nzc) return;
  const int iy = tile / nzc;
  const int z0 = (tile % nzc) * ZC;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const float2 *src = ADJ ? d.U : d.Fz;
  float2 *dst = ADJ ? d.Fz : d.U;
  copy_unrolled<8, float2>(
      Nx * ZC, tid, nthr,
      [&](int idx) {
        const int zz = idx % ZC, a = idx / ZC;
        const int z = z0 + zz;
        return z < Nz ? src[((size_t)a * nY1 + iy) * Nz + z] : make_float2(0.f, 0.f);
      },
      [&](int idx, float2 v) {
        const int zz = idx % ZC, a = idx / ZC;
        buf[wrap(a - hx, Nx) * ZC + zz] = v;
      });
  __syncthreads();
  if (ADJ) {
    fft_smem<-1>(buf, ZC, ZC, d.fNx, d.tw, tid, nthr);
  } else {
    fft_smem<+1>(buf, ZC, ZC, d.fNx, d.tw, tid, nthr);
  }
  for (int idx = tid; idx < Nx * ZC; idx += nthr) {
    const int zz = idx % ZC, a = idx / ZC;
    const int z = z0 + zz;
    const int m = wrap(a - hx, Nx);
    if (z < Nz) dst[((size_t)a * nY1 + iy) * Nz + z] = buf[m * ZC + zz];
  }
}

// Forward: U[x][jy][z] -> f[x][y][z] = sum_{jy=0}^{hy} c_jy Re(U e^{2 pi i jy (y-hy)/Ny}).
// Adjoint: f[x][y][z] -> U[x][jy][z] = c_jy sum_y f e^{-2 pi i jy (y-hy)/Ny}.
template <bool ADJ>
__global__ void __launch_bounds__(kThreadsImg) k_imgy(const InstDesc *__restrict__ descs,
                                                      const int2 *__restrict__ work, IoPtrs io0,
                                                      const IoPtrs *__restrict__ io_table) {
  extern __shared__ float4 smem_f4[];
  float2 *buf = reinterpret_cast<float2 *>(smem_f4);
  int inst, tile;
  block_work(work, inst, tile);
  const InstDesc &d = descs[inst];
  const int Nx = d.Nx, Ny = d.Ny, Nz = d.Nz, nY1 = d.nY1, hy = d.hy;
  constexpr int ZP = kImgZP;
  const int nzc = (Nz + 2 * ZP - 1) / (2 * ZP);
  if (tile >= Nx * nzc) return;
  const int x = tile / nzc;
  const int z0 = (tile % nzc) * 2 * ZP;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const IoPtrs io = io_of_img(io0, io_table, inst);
  const bool ny_even = (Ny & 1) == 0;
  if (!ADJ) {
    // one (jy, depth pair) item reads two samples and fills bins jy and Ny - jy
    copy_unrolled<8, float4>(
        nY1 * ZP, tid, nthr,
        [&](int idx) {
          const int zp = idx % ZP, jy = idx / ZP;
          const int za = z0 + 2 * zp, zb = za + 1;
          const float2 *col = d.U + ((size_t)x * nY1 + jy) * Nz;
          const float2 Ya = za < Nz ? col[za] : make_float2(0.f, 0.f);
          const float2 Yb = zb < Nz ? col[zb] : make_float2(0.f, 0.f);
          return make_float4(Ya.x, Ya.y, Yb.x, Yb.y);
        },
        [&](int idx, float4 ab) {
          const int zp = idx % ZP, jy = idx / ZP;
          if (jy == 0 || (ny_even && jy == hy)) {
            buf[jy * ZP + zp] = make_float2(ab.x, ab.z);
          } else {
            buf[jy * ZP + zp] = make_float2(ab.x - ab.w, ab.y + ab.z);
            buf[(Ny - jy) * ZP + zp] = make_float2(ab.x + ab.w, ab.z - ab.y);
          }
        });
    __syncthreads();
    fft_smem<+1>(buf, ZP, ZP, d.fNy, d.tw, tid, nthr);
    for (int idx = tid; idx < Ny * 2 * ZP; idx += nthr) {
      const int zz = idx % (2 * ZP), y = idx / (2 * ZP);
      const int z = z0 + zz;
      const int m = wrap(y - hy, Ny);
      const float2 v = buf[m * ZP + (zz >> 1)];
      if (z < Nz) io.f_out[((size_t)x * Ny + y) * Nz + z] = (zz & 1) ? v.y : v.x;
    }
  } else {
    copy_unrolled<8, float2>(
        Ny * ZP, tid, nthr,
        [&](int idx) {
          const int zp = idx % ZP, y = idx / ZP;
          const int za = z0 + 2 * zp, zb = za + 1;
          const float *row = io.f_in + ((size_t)x * Ny + y) * Nz;
          return make_float2(za < Nz ? row[za] : 0.f, zb < Nz ? row[zb] : 0.f);
        },
        [&](int idx, float2 v) {
          const int zp = idx % ZP, y = idx / ZP;
          buf[wrap(y - hy, Ny) * ZP + zp] = v;
        });
    __syncthreads();
    fft_smem<-1>(buf, ZP, ZP, d.fNy, d.tw, tid, nthr);
    for (int idx = tid; idx < nY1 * 2 * ZP; idx += nthr) {
      const int zz = idx % (2 * ZP), jy = idx / (2 * ZP);
      const int z = z0 + zz;
      if (z >= Nz) continue;
      const int zp = zz >> 1;
      const float2 Z = buf[jy * ZP + zp];
      const float2 Zm = buf[(jy == 0 ? 0 : Ny - jy) * ZP + zp];
      const float cj = (jy == 0 || (ny_even && jy == hy)) ? 1.f : 2.f;
      float2 v;
      if ((zz & 1) == 0) {
        v = make_float2(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));
      } else {
        v = make_float2(0.5f * (Z.y + Zm.y), -0.5f * (Z.x - Zm.x));
      }
      d.U[((size_t)x * nY1 + jy) * Nz + z] = cscale(v, cj);
    }
  }
}

}  // namespace

int blocks_imgx(const InstDesc &d) { return d.nY1 * ((d.Nz + kImgZC - 1) / kImgZC); }
size_t smem_imgx(const InstDesc &d) { return (size_t)d.Nx * kImgZC * sizeof(float2); }
int blocks_imgy(const InstDesc &d) { return d.Nx * ((d.Nz + 2 * kImgZP - 1) / (2 * kImgZP)); }
size_t smem_imgy(const InstDesc &d) { return (size_t)d.Ny * kImgZP * sizeof(float2); }

template <typename K>
static cudaError_t set_smem_img(K kernel, size_t smem) {
  if (smem > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

cudaError_t launch_imgx(const Launch &L, bool adjoint) {
  cudaError_t e;
  if (adjoint) {
    e = set_smem_img(k_imgx<true>, L.smem);
    if (e != cudaSuccess) return e;
    k_imgx<true><<<L.nblocks, kThreadsImg, L.smem, L.stream>>>(L.descs, L.work);
  } else {
    e = set_smem_img(k_imgx<false>, L.smem);
    if (e != cudaSuccess) return e;
    k_imgx<false><<<L.nblocks, kThreadsImg, L.smem, L.stream>>>(L.descs, L.work);
  }
  return cudaGetLastError();
}

cudaError_t launch_imgy(const Launch &L, bool adjoint) {
  cudaError_t e;
  if (adjoint) {
    e = set_smem_img(k_imgy<true>, L.smem);
    if (e != cudaSuccess) return e;
    k_imgy<true><<<L.nblocks, kThreadsImg, L.smem, L.stream>>>(L.descs, L.work, L.io, L.io_table);
  } else {
    e = set_smem_img(k_imgy<false>, L.smem);
    if (e != cudaSuccess) return e;
    k_imgy<false><<<L.nblocks, kThreadsImg, L.smem, L.stream>>>(L.descs, L.work, L.io, L.io_table);
  }
  return cudaGetLastError();
}

}  // namespace pa
