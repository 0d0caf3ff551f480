// pa_ned.cu -- NED-NUFFT stage (eq:NED_NUFFT, Sec. 3) on sm_103a.
//
// Forward:  g[m][n] --spread--> G0[p][q][n] (real, oversampled sigma*nx x
// sigma*ny grid) --FFT over q, keep jy = 0..hy--> T[p][jy][n] --FFT over p,
// keep jx = -hx..hx, divide by phihat--> G1[jx][jy][n].
//   k_spread_rowfft  spreads one strip of P grid rows x (2*NCP) samples in
//                    registers (no atomics: each warp owns cells and gathers
//                    the sensors that touch them), then runs the row FFT of
//                    the strip in shared memory; G0 never reaches HBM.
//   k_colfft         column FFT + truncation + deconvolution (and its adjoint).
// Adjoint:  the exact transposes, fused into k_rowifft_interp, which rebuilds
// the G0 cotangent rows a sensor strip needs (with a halo of w-1 rows) by an
// inverse row FFT in shared memory and interpolates at the sensors, and
// optionally accumulates the sensor-position gradient through the window
// derivative.
#include "pa_device.cuh"

namespace pa {

namespace {

constexpr int kThreadsCol = 256;
constexpr int kThreadsInterp = 256;

__device__ __forceinline__ IoPtrs io_of(const IoPtrs &io, const IoPtrs *table, int inst) {
  return table ? table[inst] : io;
}

// ------------------------------------------------------------------ spread
// Shared memory of one strip:
//   strip  float2 [My][P][NCP]   sample pairs (n even, n odd) as (re, im)
//   sg     float2 [SMAX][NCP]    staged data of the sensors of one grid row
//   sprod  float  [SMAX][w][P]   tap products wy[t] * wx[row r]
//   sby    int    [SMAX]
//   scs    int    [My + 1]       row-relative cell offsets
template <int P, int NCP, int GPW>
__global__ void __launch_bounds__(512, 1) k_spread_rowfft(const InstDesc *__restrict__ descs,
                                                        const int2 *__restrict__ work, IoPtrs io0,
                                                        const IoPtrs *__restrict__ io_table) {
  constexpr int QG = 32 / NCP;  // q columns per lane group
  extern __shared__ float4 smem_f4[];
  int inst, tile;
  block_work(work, inst, tile);
  const InstDesc &d = descs[inst];
  const int Mx = d.Mx, My = d.My, Nt = d.Nt, w = d.w, M = d.M;
  const int nstrips = (Mx + P - 1) / P;
  const int nchunks = (Nt + 2 * NCP - 1) / (2 * NCP);
  if (tile >= nstrips * nchunks) return;
  const int s = tile % nstrips;
  const int c = tile / nstrips;
  const int p0 = s * P;
  const int n0 = c * 2 * NCP;
  const IoPtrs io = io_of(io0, io_table, inst);
  const float *__restrict__ g = io.g_in;

  float2 *strip = reinterpret_cast<float2 *>(smem_f4);
  float2 *sg = strip + (size_t)My * P * NCP;
  float *sprod = reinterpret_cast<float *>(sg + kSpreadSMax * NCP);
  int *sby = reinterpret_cast<int *>(sprod + kSpreadSMax * w * P);
  int *scs = sby + kSpreadSMax;

  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int qi = lane / NCP, k = lane % NCP;

  float2 acc[GPW][P];
#pragma unroll
  for (int gi = 0; gi < GPW; ++gi)
#pragma unroll
    for (int r = 0; r < P; ++r) acc[gi][r] = make_float2(0.f, 0.f);

  const int nrows = min(P + w - 1, Mx);
  const bool pair_load = ((Nt & 1) == 0);
  for (int dr = 0; dr < nrows; ++dr) {
    const int bx = wrap(p0 - w / 2 + dr, Mx);
    const int row_lo = __ldg(d.cell_start + (size_t)bx * My);
    const int row_hi = __ldg(d.cell_start + (size_t)bx * My + My);
    if (row_hi == row_lo) continue;  // uniform across the block
    __syncthreads();
    for (int q = tid; q <= My; q += nthr) scs[q] = __ldg(d.cell_start + (size_t)bx * My + q) - row_lo;
    for (int i0 = row_lo; i0 < row_hi; i0 += kSpreadSMax) {
      const int cnt = min(kSpreadSMax, row_hi - i0);
      __syncthreads();
      // stage data pairs
      for (int idx = tid; idx < cnt * NCP; idx += nthr) {
        const int si = idx / NCP, kk = idx % NCP;
        const int m = __ldg(d.perm + i0 + si);
        const int n = n0 + 2 * kk;
        const float *row = g + (size_t)m * Nt;
        float2 v;
        if (pair_load && n + 1 < Nt) {
          v = __ldg(reinterpret_cast<const float2 *>(row + n));
        } else {
          v.x = n < Nt ? __ldg(row + n) : 0.f;
          v.y = n + 1 < Nt ? __ldg(row + n + 1) : 0.f;
        }
        sg[si * NCP + kk] = v;
      }
      // stage tap products for the P rows of the strip
      for (int idx = tid; idx < cnt * w; idx += nthr) {
        const int si = idx / w, t = idx % w;
        const int i = i0 + si;
        const float wyv = __ldg(d.wy + (size_t)i * w + t);
#pragma unroll
        for (int r = 0; r < P; ++r) {
          const int tx = wrap(p0 + r - bx + w / 2 - 1, Mx);
          const float wxv = (tx < w && p0 + r < Mx) ? __ldg(d.wx + (size_t)i * w + tx) : 0.f;
          sprod[(si * w + t) * P + r] = wyv * wxv;
        }
      }
      for (int si = tid; si < cnt; si += nthr) sby[si] = __ldg(d.sby + i0 + si);
      __syncthreads();
      // gather: warp owns q-groups; lane owns (q, sample pair)
      const int lo_win = i0 - row_lo, hi_win = lo_win + cnt;
#pragma unroll
      for (int gi = 0; gi < GPW; ++gi) {
        const int qg = (warp * GPW + gi) * QG;
        if (qg < My) {
          const int q = qg + qi;
          const int blo = qg - w / 2, bhi = qg + QG - 2 + w / 2;  // bins, inclusive
          int ra0, ra1, rb0, rb1;
          if (blo < 0) {
            ra0 = scs[My + blo]; ra1 = scs[My];
            rb0 = scs[0]; rb1 = scs[min(bhi + 1, My)];
          } else if (bhi >= My) {
            ra0 = scs[blo]; ra1 = scs[My];
            rb0 = scs[0]; rb1 = scs[bhi - My + 1];
          } else {
            ra0 = scs[blo]; ra1 = scs[bhi + 1];
            rb0 = 0; rb1 = 0;
          }
#pragma unroll
          for (int part = 0; part < 2; ++part) {
            int a0 = part ? rb0 : ra0, a1 = part ? rb1 : ra1;
            a0 = max(a0, lo_win);
            a1 = min(a1, hi_win);
            for (int li = a0; li < a1; ++li) {
              const int si = li - lo_win;
              int tq = q - sby[si] + w / 2 - 1;
              if (tq < 0) tq += My;
              if (tq >= My) tq -= My;
              float pr[P];
              if (tq < w && q < My) {
#pragma unroll
                for (int r = 0; r < P; ++r) pr[r] = sprod[(si * w + tq) * P + r];
              } else {
#pragma unroll
                for (int r = 0; r < P; ++r) pr[r] = 0.f;
              }
              const float2 gv = sg[si * NCP + k];
#pragma unroll
              for (int r = 0; r < P; ++r) {
                acc[gi][r].x = fmaf(pr[r], gv.x, acc[gi][r].x);
                acc[gi][r].y = fmaf(pr[r], gv.y, acc[gi][r].y);
              }
            }
          }
        }
      }
    }
  }
  __syncthreads();
  // the strip rows in shared memory, layout [q][r][k]
  for (int idx = tid; idx < My * P * NCP; idx += nthr) strip[idx] = make_float2(0.f, 0.f);
  __syncthreads();
#pragma unroll
  for (int gi = 0; gi < GPW; ++gi) {
    const int q = (warp * GPW + gi) * QG + qi;
    if (q < My) {
#pragma unroll
      for (int r = 0; r < P; ++r) strip[(q * P + r) * NCP + k] = acc[gi][r];
    }
  }
  __syncthreads();
  // FFT along q of the P*NCP packed sequences (element stride P*NCP)
  fft_smem<-1>(strip, P * NCP, P * NCP, d.fMy, d.tw, tid, nthr);
  // unpack the two real transforms, deconvolve in y, write T[p][jy][n]
  const int nY1 = d.nY1;
  const int total = P * nY1 * NCP * 2;
  for (int idx = tid; idx < total; idx += nthr) {
    const int par = idx & 1;
    const int kk = (idx >> 1) % NCP;
    const int rest = (idx >> 1) / NCP;
    const int jy = rest % nY1;
    const int r = rest / nY1;
    const int p = p0 + r;
    const int n = n0 + 2 * kk + par;
    if (p < Mx && n < Nt) {
      const float2 Z = strip[(jy * P + r) * NCP + kk];
      const int jm = jy == 0 ? 0 : My - jy;
      const float2 Zm = strip[(jm * P + r) * NCP + kk];
      float2 v;
      if (par == 0) {
        v = make_float2(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));
      } else {
        v = make_float2(0.5f * (Z.y + Zm.y), -0.5f * (Z.x - Zm.x));
      }
      const float sc = __ldg(d.invphy + jy);
      d.T[((size_t)p * nY1 + jy) * Nt + n] = cscale(v, sc);
    }
  }
  (void)M;
}

// ------------------------------------------------------------- column FFT
// Forward: T[p][jy][n] (p = 0..Mx-1) -> FFT over p -> keep jx in [-hx, hx],
// times 1/phihat_x -> G1[jx + hx][jy][n].
// Adjoint: G1b[jx + hx][jy][n] times 1/phihat_x placed at bins jx mod Mx,
// inverse FFT over p -> Tb[p][jy][n].
template <bool ADJ>
__global__ void __launch_bounds__(kThreadsCol) k_colfft(const InstDesc *__restrict__ descs,
                                                        const int2 *__restrict__ work) {
  extern __shared__ float4 smem_f4[];
  float2 *buf = reinterpret_cast<float2 *>(smem_f4);
  int inst, tile;
  block_work(work, inst, tile);
  const InstDesc &d = descs[inst];
  const int Mx = d.Mx, Nt = d.Nt, nY1 = d.nY1, nX1 = d.nX1, hx = d.hx;
  constexpr int NC = kColNC;
  const int nchunks = (Nt + NC - 1) / NC;
  if (tile >= nY1 * nchunks) return;
  const int jy = tile % nY1;
  const int n0 = (tile / nY1) * NC;
  const int tid = threadIdx.x, nthr = blockDim.x;
  if (!ADJ) {
    for (int idx = tid; idx < Mx * NC; idx += nthr) {
      const int kk = idx % NC, p = idx / NC;
      const int n = n0 + kk;
      buf[idx] = n < Nt ? d.T[((size_t)p * nY1 + jy) * Nt + n] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft_smem<-1>(buf, NC, NC, d.fMx, d.tw, tid, nthr);
    for (int idx = tid; idx < nX1 * NC; idx += nthr) {
      const int kk = idx % NC, ix = idx / NC;
      const int n = n0 + kk;
      if (n < Nt) {
        const int b = wrap(ix - hx, Mx);
        d.G1[((size_t)ix * nY1 + jy) * Nt + n] = cscale(buf[b * NC + kk], __ldg(d.invphx + ix));
      }
    }
  } else {
    for (int idx = tid; idx < Mx * NC; idx += nthr) buf[idx] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int idx = tid; idx < nX1 * NC; idx += nthr) {
      const int kk = idx % NC, ix = idx / NC;
      const int n = n0 + kk;
      const int b = wrap(ix - hx, Mx);
      buf[b * NC + kk] = n < Nt ? cscale(d.G1[((size_t)ix * nY1 + jy) * Nt + n], __ldg(d.invphx + ix))
                                : make_float2(0.f, 0.f);
    }
    __syncthreads();
    fft_smem<+1>(buf, NC, NC, d.fMx, d.tw, tid, nthr);
    for (int idx = tid; idx < Mx * NC; idx += nthr) {
      const int kk = idx % NC, p = idx / NC;
      const int n = n0 + kk;
      if (n < Nt) d.T[((size_t)p * nY1 + jy) * Nt + n] = buf[idx];
    }
  }
}

// ------------------------------------------------- adjoint row FFT + interp
// One tile owns the sensors whose base row bx lies in [p0, p0 + Po) and the
// sample pairs [n0, n0 + 2 NCP).  It rebuilds the R = Po + w - 1 cotangent
// rows p = p0 - w/2 + 1 + r of the oversampled grid from Tb by the transpose
// of (row FFT, unpack, deconvolution), then interpolates them at its sensors.
// Shared memory: G [My][R][NCP] float2.
template <int W, int Po, int NCP, bool GRAD>
__global__ void __launch_bounds__(kThreadsInterp) k_rowifft_interp(const InstDesc *__restrict__ descs,
                                                                   const int2 *__restrict__ work, IoPtrs io0,
                                                                   const IoPtrs *__restrict__ io_table) {
  extern __shared__ float4 smem_f4[];
  float2 *G = reinterpret_cast<float2 *>(smem_f4);
  int inst, tile;
  block_work(work, inst, tile);
  const InstDesc &d = descs[inst];
  const int Mx = d.Mx, My = d.My, Nt = d.Nt, hy = d.hy, nY1 = d.nY1, M = d.M;
  const int nstrips = (Mx + Po - 1) / Po;
  const int nchunks = (Nt + 2 * NCP - 1) / (2 * NCP);
  if (tile >= nstrips * nchunks) return;
  const int s = tile % nstrips;
  const int c = tile / nstrips;
  const int p0 = s * Po;
  const int n0 = c * 2 * NCP;
  constexpr int R = Po + W - 1;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const IoPtrs io = io_of(io0, io_table, inst);

  // owned sensors
  const int i_lo = __ldg(d.cell_start + (size_t)p0 * My);
  const int i_hi = __ldg(d.cell_start + (size_t)min(p0 + Po, Mx) * My);

  // packed Hermitian spectra of the R rows
  for (int idx = tid; idx < My * R * NCP; idx += nthr) {
    const int kk = idx % NCP;
    const int r = (idx / NCP) % R;
    const int q = idx / (NCP * R);
    const int p = wrap(p0 - W / 2 + 1 + r, Mx);
    float2 S = make_float2(0.f, 0.f);
    int jy = -1;
    bool lower = true;
    if (q <= hy) {
      jy = q;
    } else if (q >= My - hy) {
      jy = My - q;
      lower = false;
    }
    if (jy >= 0) {
      const int n = n0 + 2 * kk;
      const float2 *Trow = d.T + ((size_t)p * nY1 + jy) * Nt;
      const float sc = __ldg(d.invphy + jy);
      const float2 a = n < Nt ? cscale(Trow[n], sc) : make_float2(0.f, 0.f);
      const float2 b = n + 1 < Nt ? cscale(Trow[n + 1], sc) : make_float2(0.f, 0.f);
      if (jy == 0) {
        S = make_float2(a.x, b.x);
      } else if (lower) {
        S = make_float2(0.5f * (a.x - b.y), 0.5f * (a.y + b.x));
      } else {
        S = make_float2(0.5f * (a.x + b.y), 0.5f * (b.x - a.y));
      }
    }
    G[idx] = S;
  }
  __syncthreads();
  fft_smem<+1>(G, R * NCP, R * NCP, d.fMy, d.tw, tid, nthr);

  // interpolation: warp per sensor, lane = (ty, kk)
  const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
  constexpr int TYS = 32 / NCP;
  const int kk = lane % NCP, ty0 = lane / NCP;
  for (int i = i_lo + warp; i < i_hi; i += nwarp) {
    const int bx = __ldg(d.sbx + i), by = __ldg(d.sby + i);
    const int rb = bx - p0;  // 0 .. Po-1
    if (rb < 0 || rb >= Po) {
      if (lane == 0) atomicExch(d.status, 1);
      continue;
    }
    float wxr[W], dwxr[W];
#pragma unroll
    for (int t = 0; t < W; ++t) {
      wxr[t] = __ldg(d.wx + (size_t)i * W + t);
      if (GRAD) dwxr[t] = __ldg(d.dwx + (size_t)i * W + t);
    }
    float2 a0 = make_float2(0.f, 0.f), ax = a0, ay = a0;
#pragma unroll
    for (int tyb = 0; tyb < W; tyb += TYS) {
      const int ty = tyb + ty0;
      if (ty < W) {
        const int q = wrap(by - W / 2 + 1 + ty, My);
        const float2 *Gq = G + ((size_t)q * R + rb) * NCP + kk;
        float2 rs = make_float2(0.f, 0.f), rsx = rs;
#pragma unroll
        for (int tx = 0; tx < W; ++tx) {
          const float2 v = Gq[tx * NCP];
          rs.x = fmaf(wxr[tx], v.x, rs.x);
          rs.y = fmaf(wxr[tx], v.y, rs.y);
          if (GRAD) {
            rsx.x = fmaf(dwxr[tx], v.x, rsx.x);
            rsx.y = fmaf(dwxr[tx], v.y, rsx.y);
          }
        }
        const float wyv = __ldg(d.wy + (size_t)i * W + ty);
        a0.x = fmaf(wyv, rs.x, a0.x);
        a0.y = fmaf(wyv, rs.y, a0.y);
        if (GRAD) {
          const float dwyv = __ldg(d.dwy + (size_t)i * W + ty);
          ax.x = fmaf(wyv, rsx.x, ax.x);
          ax.y = fmaf(wyv, rsx.y, ax.y);
          ay.x = fmaf(dwyv, rs.x, ay.x);
          ay.y = fmaf(dwyv, rs.y, ay.y);
        }
      }
    }
#pragma unroll
    for (int off = NCP; off < 32; off <<= 1) {
      a0.x += __shfl_xor_sync(0xffffffffu, a0.x, off);
      a0.y += __shfl_xor_sync(0xffffffffu, a0.y, off);
      if (GRAD) {
        ax.x += __shfl_xor_sync(0xffffffffu, ax.x, off);
        ax.y += __shfl_xor_sync(0xffffffffu, ax.y, off);
        ay.x += __shfl_xor_sync(0xffffffffu, ay.x, off);
        ay.y += __shfl_xor_sync(0xffffffffu, ay.y, off);
      }
    }
    const int m = __ldg(d.perm + i);
    const int n = n0 + 2 * kk;
    float px = 0.f, py = 0.f;
    if (lane < NCP) {
      if (io.g_out) {
        float *orow = io.g_out + (size_t)m * Nt;
        if (n < Nt) orow[n] = a0.x;
        if (n + 1 < Nt) orow[n + 1] = a0.y;
      }
      if (GRAD) {
        const float *grow = io.g_in + (size_t)m * Nt;
        const float g0 = n < Nt ? __ldg(grow + n) : 0.f;
        const float g1 = n + 1 < Nt ? __ldg(grow + n + 1) : 0.f;
        px = ax.x * g0 + ax.y * g1;
        py = ay.x * g0 + ay.y * g1;
      }
    }
    if (GRAD) {
#pragma unroll
      for (int off = 1; off < NCP; off <<= 1) {
        px += __shfl_xor_sync(0xffffffffu, px, off);
        py += __shfl_xor_sync(0xffffffffu, py, off);
      }
      if (lane == 0) d.grad_part[(size_t)c * M + i] = make_float2(px, py);
    }
  }
}

// Sum the per-chunk gradient partials and scatter to the caller's order.
__global__ void k_grad_reduce(const InstDesc *__restrict__ descs, IoPtrs io0, const IoPtrs *__restrict__ io_table,
                              int inst_count) {
  for (int inst = 0; inst < inst_count; ++inst) {
    const InstDesc &d = descs[inst];
    const IoPtrs io = io_of(io0, io_table, inst);
    if (!io.grad_xy) continue;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.M; i += gridDim.x * blockDim.x) {
      float sx = 0.f, sy = 0.f;
      for (int c = 0; c < d.nchunk_adj; ++c) {
        const float2 v = d.grad_part[(size_t)c * d.M + i];
        sx += v.x;
        sy += v.y;
      }
      const int m = d.perm[i];
      io.grad_xy[2 * m] = sx;
      io.grad_xy[2 * m + 1] = sy;
    }
  }
}

}  // namespace

// ------------------------------------------------------------------ host side
int threads_spread(const InstDesc &d) {
  constexpr int QG = 32 / kSpreadNCP;
  int warps = (d.My + QG * kSpreadGPW - 1) / (QG * kSpreadGPW);
  if (warps < 8) warps = 8;
  return warps * 32;
}
int blocks_spread(const InstDesc &d) {
  return ((d.Mx + kSpreadP - 1) / kSpreadP) * ((d.Nt + 2 * kSpreadNCP - 1) / (2 * kSpreadNCP));
}
size_t smem_spread(const InstDesc &d) {
  return (size_t)d.My * kSpreadP * kSpreadNCP * sizeof(float2) + kSpreadSMax * kSpreadNCP * sizeof(float2) +
         (size_t)kSpreadSMax * d.w * kSpreadP * sizeof(float) + kSpreadSMax * sizeof(int) +
         (size_t)(d.My + 1) * sizeof(int);
}
int blocks_colfft(const InstDesc &d) { return d.nY1 * ((d.Nt + kColNC - 1) / kColNC); }
size_t smem_colfft(const InstDesc &d) { return (size_t)d.Mx * kColNC * sizeof(float2); }
int blocks_interp(const InstDesc &d) {
  return ((d.Mx + kAdjPo - 1) / kAdjPo) * ((d.Nt + 2 * kAdjNCP - 1) / (2 * kAdjNCP));
}
size_t smem_interp(const InstDesc &d) {
  return (size_t)d.My * (kAdjPo + d.w - 1) * kAdjNCP * sizeof(float2);
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t smem) {
  if (smem > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

cudaError_t launch_spread(const Launch &L, int threads) {
  auto kern = k_spread_rowfft<kSpreadP, kSpreadNCP, kSpreadGPW>;
  cudaError_t e = set_smem(kern, L.smem);
  if (e != cudaSuccess) return e;
  kern<<<L.nblocks, threads, L.smem, L.stream>>>(L.descs, L.work, L.io, L.io_table);
  return cudaGetLastError();
}

cudaError_t launch_colfft(const Launch &L, bool adjoint) {
  cudaError_t e;
  if (adjoint) {
    e = set_smem(k_colfft<true>, L.smem);
    if (e != cudaSuccess) return e;
    k_colfft<true><<<L.nblocks, kThreadsCol, L.smem, L.stream>>>(L.descs, L.work);
  } else {
    e = set_smem(k_colfft<false>, L.smem);
    if (e != cudaSuccess) return e;
    k_colfft<false><<<L.nblocks, kThreadsCol, L.smem, L.stream>>>(L.descs, L.work);
  }
  return cudaGetLastError();
}

template <int W, bool GRAD>
static cudaError_t launch_interp_w(const Launch &L) {
  auto kern = k_rowifft_interp<W, kAdjPo, kAdjNCP, GRAD>;
  cudaError_t e = set_smem(kern, L.smem);
  if (e != cudaSuccess) return e;
  kern<<<L.nblocks, kThreadsInterp, L.smem, L.stream>>>(L.descs, L.work, L.io, L.io_table);
  return cudaGetLastError();
}

cudaError_t launch_interp_width(const Launch &L, int width, bool grad) {
  switch (width) {
    case 6: return grad ? launch_interp_w<6, true>(L) : launch_interp_w<6, false>(L);
    case 8: return grad ? launch_interp_w<8, true>(L) : launch_interp_w<8, false>(L);
    case 12: return grad ? launch_interp_w<12, true>(L) : launch_interp_w<12, false>(L);
    case 16: return grad ? launch_interp_w<16, true>(L) : launch_interp_w<16, false>(L);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_grad_reduce(const Launch &L, int n_inst) {
  k_grad_reduce<<<L.nblocks, 256, 0, L.stream>>>(L.descs, L.io, L.io_table, n_inst);
  return cudaGetLastError();
}

}  // namespace pa
