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
#include "pa_tmap.h"

namespace pa {

namespace {

constexpr int kThreadsImg = 256;
// Blocks per SM the persistent image transforms budget registers for (with
// a budget for one, ptxas gives them about 160 registers and one block per
// SM: 57 -> 73 us at 256x256x512).
#ifndef PA_IMG_MINB
#define PA_IMG_MINB 2
#endif

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

// Persistent, double-buffered k_imgx for Nx = 2^LGL and even Nz (one plan):
// the rows of the next tile arrive by bulk copies (TMA engine) while the
// current tile is transformed.
// With use_map, a tile arrives as two boxes of the 3-D tensor map over the
// source (floats; dims 2 Nz, nY1, Nx; box 32 x 1 x Nx/2): rows a >= hx to
// buffer rows 0.., rows a < hx to buffer rows Nx - hx.. (hx = Nx/2).
template <bool ADJ, int LGL>
__global__ void __launch_bounds__(kThreadsImg, PA_IMG_MINB) k_imgx_pipe(const InstDesc *__restrict__ descs, int nwork,
                                                           const __grid_constant__ CUtensorMap map, int use_map) {
  griddep_enter();  // the previous kernel of the stream has completed
  extern __shared__ __align__(128) float4 smem_a128[];  // box destinations 128-byte aligned
  __shared__ __align__(8) uint64_t bars[2];
  constexpr int L = 1 << LGL, ZC = kImgZC, LGZC = 4;
  static_assert(ZC == 1 << LGZC, "tile width");
  float2 *buf0 = reinterpret_cast<float2 *>(smem_a128);
  float2 *buf1 = buf0 + L * ZC;
  const InstDesc &d = descs[0];
  if (!smem_aligned_128(smem_a128, d.status)) return;
  const int Nz = d.Nz, nY1 = d.nY1, hx = d.hx;
  const int nzc = (Nz + ZC - 1) / ZC;
  const int tid = threadIdx.x, nthr = blockDim.x, lgT = ilog2_pow2(nthr);
  const float2 *tw = d.tw + d.fNx.tw;
  const float2 *src = ADJ ? d.U : d.Fz;
  float2 *dst = ADJ ? d.Fz : d.U;
  auto issue = [&](int w, float2 *buf, uint64_t *bar) {
    const int iy = w / nzc, z0 = (w - iy * nzc) * ZC;
    if (use_map) {
      if (tid == 0) {
        mbar_arrive_expect_tx(bar, uint32_t(L * ZC * sizeof(float2)));
        tma_load_3d(buf, &map, 2 * z0, iy, L / 2, bar);
        tma_load_3d(buf + (L / 2) * ZC, &map, 2 * z0, iy, 0, bar);
      }
      return;
    }
    const uint32_t rb = uint32_t(min(ZC, Nz - z0)) * sizeof(float2);
    if (tid == 0) mbar_arrive_expect_tx(bar, rb * L);
    for (int a = tid; a < L; a += nthr)
      bulk_g2s(buf + ((a - hx) & (L - 1)) * ZC, src + ((size_t)a * nY1 + iy) * Nz + z0, rb, bar);
  };
  auto compute = [&](int w, float2 *buf) {
    const int iy = w / nzc, z0 = (w - iy * nzc) * ZC;
    fft_fixed<LGL, ADJ ? -1 : +1>(buf, ZC, LGZC, lgT, tw, tid);
    for (int idx = tid; idx < L * ZC; idx += nthr) {
      const int zz = idx & (ZC - 1), a = idx >> LGZC;
      const int z = z0 + zz;
      if (z < Nz) dst[((size_t)a * nY1 + iy) * Nz + z] = buf[((a - hx) & (L - 1)) * ZC + zz];
    }
  };
  tile_pipeline(nwork, buf0, buf1, bars, d.status, issue, compute);
}

// Persistent, double-buffered k_imgy for Ny = 2^LGL and Nz % 4 == 0 (one
// plan).  Forward: the half-spectrum rows U[x][jy] land in a staging buffer;
// adjoint: the image rows f[x][y] land directly as depth pairs.
// With use_map, forward staging rows arrive as one box of the 2-D map over U
// (floats; dims 2 Nz, Nx nY1; box 64 x nY1), adjoint image rows as two boxes
// of the 2-D map over f_in (dims Nz, Nx Ny; box 32 x Ny/2), rows y >= hy to
// buffer rows 0.., rows y < hy to buffer rows Ny - hy.. (hy = Ny/2).
template <bool ADJ, int LGL>
__global__ void __launch_bounds__(kThreadsImg, PA_IMG_MINB) k_imgy_pipe(const InstDesc *__restrict__ descs, int nwork, IoPtrs io,
                                                           const __grid_constant__ CUtensorMap map, int use_map) {
  griddep_enter();  // the previous kernel of the stream has completed
  extern __shared__ __align__(128) float4 smem_a128[];  // box destinations 128-byte aligned
  __shared__ __align__(8) uint64_t bars[2];
  constexpr int L = 1 << LGL, ZP = kImgZP, LGZP = 4;
  static_assert(ZP == 1 << LGZP, "tile width");
  const InstDesc &d = descs[0];
  if (!smem_aligned_128(smem_a128, d.status)) return;
  const int Nz = d.Nz, nY1 = d.nY1, hy = d.hy;
  const bool ny_even = (L & 1) == 0;
  const int nzc = (Nz + 2 * ZP - 1) / (2 * ZP);
  const int tid = threadIdx.x, nthr = blockDim.x, lgT = ilog2_pow2(nthr);
  const float2 *tw = d.tw + d.fNy.tw;
  float2 *B = reinterpret_cast<float2 *>(smem_a128);
  // [Ny][ZP] depth pairs; forward: two staging buffers [nY1][2 ZP] (rounded
  // to 128 bytes); adjoint: two tile buffers [Ny][ZP]
  const int stage = (nY1 * 2 * ZP + 15) & ~15;
  float2 *b0 = ADJ ? B : B + L * ZP;
  float2 *b1 = ADJ ? B + L * ZP : b0 + stage;
  auto issue = [&](int w, float2 *buf, uint64_t *bar) {
    const int x = w / nzc, z0 = (w - x * nzc) * 2 * ZP;
    const int nz = min(2 * ZP, Nz - z0);
    if (use_map) {
      if (tid == 0) {
        if (!ADJ) {
          mbar_arrive_expect_tx(bar, uint32_t(nY1 * 2 * ZP * sizeof(float2)));
          tma_load_2d(buf, &map, 2 * z0, x * nY1, bar);
        } else {
          mbar_arrive_expect_tx(bar, uint32_t(L * ZP * sizeof(float2)));
          tma_load_2d(buf, &map, z0, x * L + L / 2, bar);
          tma_load_2d(buf + (L / 2) * ZP, &map, z0, x * L, bar);
        }
      }
      return;
    }
    if (!ADJ) {
      const uint32_t rb = uint32_t(nz) * sizeof(float2);
      if (tid == 0) mbar_arrive_expect_tx(bar, rb * nY1);
      const float2 *Ur = d.U + (size_t)x * nY1 * Nz + z0;
      for (int jy = tid; jy < nY1; jy += nthr) bulk_g2s(buf + jy * 2 * ZP, Ur + (size_t)jy * Nz, rb, bar);
    } else {
      const uint32_t rb = uint32_t(nz) * sizeof(float);
      if (tid == 0) mbar_arrive_expect_tx(bar, rb * L);
      const float *fr = io.f_in + (size_t)x * L * Nz + z0;
      for (int y = tid; y < L; y += nthr) bulk_g2s(buf + ((y - hy) & (L - 1)) * ZP, fr + (size_t)y * Nz, rb, bar);
    }
  };
  auto compute = [&](int w, float2 *buf) {
    const int x = w / nzc, z0 = (w - x * nzc) * 2 * ZP;
    const int nz = min(2 * ZP, Nz - z0);
    if (!ADJ) {
      // interior bins jy and Ny - jy from (U[z], U[z+1]); jy = 0 and the
      // even-length Nyquist bin through their real parts
      for (int idx = tid; idx < L * ZP; idx += nthr) {
        const int q = idx >> LGZP, zp = idx & (ZP - 1);
        const int jy = q <= L / 2 ? q : L - q;
        const bool in = 2 * zp < nz;
        const float2 Ya = in ? buf[jy * 2 * ZP + 2 * zp] : make_float2(0.f, 0.f);
        const float2 Yb = in ? buf[jy * 2 * ZP + 2 * zp + 1] : make_float2(0.f, 0.f);
        float2 v;
        if (jy == 0 || (ny_even && jy == hy)) {
          v = make_float2(Ya.x, Yb.x);
        } else if (q == jy) {
          v = make_float2(Ya.x - Yb.y, Ya.y + Yb.x);
        } else {
          v = make_float2(Ya.x + Yb.y, Yb.x - Ya.y);
        }
        B[idx] = v;
      }
      __syncthreads();
      fft_fixed<LGL, +1>(B, ZP, LGZP, lgT, tw, tid);
      float *fo = io.f_out + (size_t)x * L * Nz + z0;
      const int nv4 = nz >> 2;
      if (nv4 == ZP / 2) {  // full chunk: index splits by shifts
        for (int idx = tid; idx < L * (ZP / 2); idx += nthr) {
          const int y = idx >> (LGZP - 1), k2 = idx & (ZP / 2 - 1);
          *reinterpret_cast<float4 *>(fo + (size_t)y * Nz + 4 * k2) =
              reinterpret_cast<const float4 *>(B + ((y - hy) & (L - 1)) * ZP)[k2];
        }
      } else {
        for (int idx = tid; idx < L * nv4; idx += nthr) {
          const int y = idx / nv4, k2 = idx - y * nv4;
          *reinterpret_cast<float4 *>(fo + (size_t)y * Nz + 4 * k2) =
              reinterpret_cast<const float4 *>(B + ((y - hy) & (L - 1)) * ZP)[k2];
        }
      }
    } else {
      fft_fixed<LGL, -1>(buf, ZP, LGZP, lgT, tw, tid);
      float2 *Ur = d.U + (size_t)x * nY1 * Nz + z0;
      for (int idx = tid; idx < nY1 * ZP; idx += nthr) {
        const int jy = idx >> LGZP, zp = idx & (ZP - 1);
        if (2 * zp >= nz) continue;
        const float2 Z = buf[jy * ZP + zp];
        const float2 Zm = buf[(jy == 0 ? 0 : L - jy) * ZP + zp];
        const float cj = (jy == 0 || (ny_even && jy == hy)) ? 0.5f : 1.f;
        const float2 va = make_float2(cj * (Z.x + Zm.x), cj * (Z.y - Zm.y));
        const float2 vb = make_float2(cj * (Z.y + Zm.y), -cj * (Z.x - Zm.x));
        *reinterpret_cast<float4 *>(Ur + (size_t)jy * Nz + 2 * zp) = make_float4(va.x, va.y, vb.x, vb.y);
      }
    }
  };
  tile_pipeline(nwork, b0, b1, bars, d.status, issue, compute);
}

}  // namespace

int blocks_imgx(const InstDesc &d) { return d.nY1 * ((d.Nz + kImgZC - 1) / kImgZC); }
size_t smem_imgx(const InstDesc &d) { return (size_t)d.Nx * kImgZC * sizeof(float2); }
int blocks_imgy(const InstDesc &d) { return d.Nx * ((d.Nz + 2 * kImgZP - 1) / (2 * kImgZP)); }
size_t smem_imgy(const InstDesc &d) { return (size_t)d.Ny * kImgZP * sizeof(float2); }

template <typename K>
static cudaError_t set_smem_img(K kernel, size_t smem) {
  if (smem > 40 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

cudaError_t launch_imgx(const Launch &L, bool adjoint) {
  if (L.host && !L.work && (L.host->Nz % 2) == 0) {
    const InstDesc &h = *L.host;
    const int nwork = h.nY1 * ((h.Nz + kImgZC - 1) / kImgZC);
    const size_t smem = 2 * size_t(h.Nx) * kImgZC * sizeof(float2);
    CUtensorMap map;
    const int use_map = h.Nx / 2 <= 256 && encode_3d(adjoint ? (const void *)h.U : (const void *)h.Fz,
                                                     2 * uint64_t(h.Nz), uint64_t(h.nY1), uint64_t(h.Nx),
                                                     uint64_t(h.Nz) * sizeof(float2),
                                                     uint64_t(h.nY1) * h.Nz * sizeof(float2), 32u, 1u,
                                                     uint32_t(h.Nx / 2), &map);
    switch (pow2_log(h.Nx)) {
#define PA_IMGX_CASE(G)                                                                                    \
  case G:                                                                                                  \
    return adjoint ? launch_persistent_map(k_imgx_pipe<true, G>, L, kThreadsImg, smem, nwork, map, use_map)  \
                   : launch_persistent_map(k_imgx_pipe<false, G>, L, kThreadsImg, smem, nwork, map, use_map);
      PA_IMGX_CASE(5) PA_IMGX_CASE(6) PA_IMGX_CASE(7) PA_IMGX_CASE(8) PA_IMGX_CASE(9)
#undef PA_IMGX_CASE
      default: break;
    }
  }
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

template <typename K>
static cudaError_t launch_persistent_io(K kernel, const Launch &L, size_t smem, int nwork, const CUtensorMap &map,
                                        int use_map) {
  if (smem > 40 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  const int grid = persistent_grid(kernel, kThreadsImg, smem, nwork);
  return launch_pdl(kernel, grid, kThreadsImg, smem, L.stream, L.descs, nwork, L.io, map, use_map);
}

cudaError_t launch_imgy(const Launch &L, bool adjoint) {
  if (L.host && !L.work && (L.host->Nz % 4) == 0) {
    const InstDesc &h = *L.host;
    const int nwork = h.Nx * ((h.Nz + 2 * kImgZP - 1) / (2 * kImgZP));
    const size_t stage = size_t((h.nY1 * 2 * kImgZP + 15) & ~15);
    const size_t smem = (adjoint ? 2 * size_t(h.Ny) * kImgZP : size_t(h.Ny) * kImgZP + 2 * stage) * sizeof(float2);
    CUtensorMap map;
    int use_map = 0;
    if (!adjoint) {
      use_map = h.nY1 <= 256 && encode_2d(h.U, 2 * uint64_t(h.Nz), uint64_t(h.Nx) * h.nY1,
                                          uint64_t(h.Nz) * sizeof(float2), 2u * 2 * kImgZP, uint32_t(h.nY1), &map);
    } else {
      use_map = h.Ny / 2 <= 256 && L.io.f_in &&
                encode_2d(L.io.f_in, uint64_t(h.Nz), uint64_t(h.Nx) * h.Ny, uint64_t(h.Nz) * sizeof(float),
                          2u * kImgZP, uint32_t(h.Ny / 2), &map);
    }
    switch (pow2_log(h.Ny)) {
#define PA_IMGY_CASE(G)                                                                       \
  case G:                                                                                     \
    return adjoint ? launch_persistent_io(k_imgy_pipe<true, G>, L, smem, nwork, map, use_map) \
                   : launch_persistent_io(k_imgy_pipe<false, G>, L, smem, nwork, map, use_map);
      PA_IMGY_CASE(5) PA_IMGY_CASE(6) PA_IMGY_CASE(7) PA_IMGY_CASE(8) PA_IMGY_CASE(9)
#undef PA_IMGY_CASE
      default: break;
    }
  }
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
