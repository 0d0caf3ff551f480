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
#include <cooperative_groups.h>

#include "pa_device.cuh"

namespace cg = cooperative_groups;

namespace pa {

namespace {

constexpr int kThreadsCol = 256;
constexpr int kThreadsInterp = 256;

__device__ __forceinline__ IoPtrs io_of(const IoPtrs &io, const IoPtrs *table, int inst) {
  return table ? table[inst] : io;
}

// ------------------------------------------------------------------ spread
// One tile: a strip of P oversampled grid rows x 2*NCP samples.  Warp w owns
// the q-groups w*GPW .. w*GPW+GPW-1 (QG columns each); lane (qi, k) owns
// column qi of the group and the sample pair k for all P rows, in registers.
// It streams the group's visits (precomputed by the plan: caller index of the
// sensor and the tap products for its QG columns x P rows) and reads the
// sample pair straight from g (L2-resident), so the accumulation needs no
// shared memory and no barrier.  The strip is then FFT'd over q in shared
// memory (float2 [My][P][NCP], element stride P*NCP) and written as T.
template <int P, int NCP, int GPW>
__global__ void __launch_bounds__(512, 1) k_spread_rowfft(const InstDesc *__restrict__ descs,
                                                        const int2 *__restrict__ work, IoPtrs io0,
                                                        const IoPtrs *__restrict__ io_table) {
  constexpr int QG = 32 / NCP;  // q columns per lane group
  static_assert(P == 4, "visit products hold four rows");
  extern __shared__ float4 smem_f4[];
  int inst, tile;
  block_work(work, inst, tile);
  const InstDesc &d = descs[inst];
  const int Mx = d.Mx, My = d.My, Nt = d.Nt;
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

  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int qi = lane / NCP, k = lane % NCP;
  const int n = n0 + 2 * k;
  const bool pair_ok = ((Nt & 1) == 0) && (n + 1 < Nt);
  const int NG = (My + QG - 1) / QG;
  const int *__restrict__ vstart = d.visit_start + (size_t)s * NG;
  const int *__restrict__ vm = d.vm;
  const float4 *__restrict__ vprod = d.vprod;

  float2 acc[GPW][P];
#pragma unroll
  for (int gi = 0; gi < GPW; ++gi)
#pragma unroll
    for (int r = 0; r < P; ++r) acc[gi][r] = make_float2(0.f, 0.f);

#pragma unroll
  for (int gi = 0; gi < GPW; ++gi) {
    const int grp = warp * GPW + gi;
    if (grp < NG) {
      const int v0 = __ldg(vstart + grp), v1 = __ldg(vstart + grp + 1);
#pragma unroll 4
      for (int v = v0; v < v1; ++v) {
        const int m = __ldg(vm + v);
        const float4 pr = __ldg(vprod + (size_t)v * QG + qi);
        const float *row = g + (size_t)m * Nt;
        float2 gv;
        if (pair_ok) {
          gv = __ldg(reinterpret_cast<const float2 *>(row + n));
        } else {
          gv.x = n < Nt ? __ldg(row + n) : 0.f;
          gv.y = n + 1 < Nt ? __ldg(row + n + 1) : 0.f;
        }
        acc[gi][0].x = fmaf(pr.x, gv.x, acc[gi][0].x);
        acc[gi][0].y = fmaf(pr.x, gv.y, acc[gi][0].y);
        acc[gi][1].x = fmaf(pr.y, gv.x, acc[gi][1].x);
        acc[gi][1].y = fmaf(pr.y, gv.y, acc[gi][1].y);
        acc[gi][2].x = fmaf(pr.z, gv.x, acc[gi][2].x);
        acc[gi][2].y = fmaf(pr.z, gv.y, acc[gi][2].y);
        acc[gi][3].x = fmaf(pr.w, gv.x, acc[gi][3].x);
        acc[gi][3].y = fmaf(pr.w, gv.y, acc[gi][3].y);
      }
    }
  }
  // the strip rows in shared memory, layout [q][r][k]; every q < My is
  // owned by exactly one lane group
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
    const int nn = n0 + 2 * kk + par;
    if (p < Mx && nn < Nt) {
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
      d.T[((size_t)p * nY1 + jy) * Nt + nn] = cscale(v, sc);
    }
  }
}

// ---------------------------------------------------------- cluster spread
// A cluster of two blocks owns one strip (P grid rows) and 2*NCP samples; the
// block of rank h owns the columns [h*My/2, (h+1)*My/2).  Each block stages
// the sensors whose footprint meets its rows and columns (taps and sample
// pairs) in shared memory once, then every warp accumulates its q-groups in
// registers from those staged values (lane = (column qi, sample pair k)).
// The length-My FFT over q then starts with one radix-2 decimation-in-
// frequency step across the pair through distributed shared memory
//   y_h[q] = x[q] + x[q + My/2]               (h = 0)
//   y_h[q] = (x[q] - x[q + My/2]) W_My^q      (h = 1),
// after which block h holds, by a local length-My/2 FFT, the bins jy = 2k+h.
// Bins jy and My - jy have the same parity, so the real-pair unpack and the
// deconvolution stay local.
template <int P, int NCP, int GPW, int W>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(512, 1)
    k_spread_cl(const InstDesc *__restrict__ descs, const int2 *__restrict__ work, IoPtrs io0,
                const IoPtrs *__restrict__ io_table) {
  constexpr int QG = 32 / NCP;
  static_assert(P == 4, "staged x taps hold four rows");
  extern __shared__ float4 smem_f4[];
  cg::cluster_group cluster = cg::this_cluster();
  const int h = int(cluster.block_rank());
  int inst, tile;
  if (work) {
    const int2 wv = work[blockIdx.x >> 1];
    inst = wv.x;
    tile = wv.y;
  } else {
    inst = 0;
    tile = blockIdx.x >> 1;
  }
  const InstDesc &d = descs[inst];
  const int Mx = d.Mx, My = d.My, Nt = d.Nt;
  const int H = My / 2;
  const int nstrips = (Mx + P - 1) / P;
  const int nchunks = (Nt + 2 * NCP - 1) / (2 * NCP);
  if (tile >= nstrips * nchunks) return;  // both blocks of the cluster leave together
  const int s = tile % nstrips;
  const int c = tile / nstrips;
  const int p0 = s * P;
  const int n0 = c * 2 * NCP;
  const IoPtrs io = io_of(io0, io_table, inst);
  const float *__restrict__ g = io.g_in;
  const int key = s * 2 + h;
  const int NGH = (H + QG - 1) / QG;
  const int smax = d.cl_smax;

  float2 *strip = reinterpret_cast<float2 *>(smem_f4);          // [H][P][NCP]
  float4 *s_wx = reinterpret_cast<float4 *>(strip + (size_t)H * P * NCP);
  float2 *s_g = reinterpret_cast<float2 *>(s_wx + smax);        // [smax][NCP]
  int2 *s_meta = reinterpret_cast<int2 *>(s_g + (size_t)smax * NCP);
  float *s_wy = reinterpret_cast<float *>(s_meta + smax);       // [smax][W]

  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const int qi = lane / NCP, k = lane % NCP;

  // stage the slots of this (strip, half)
  const int sbase = __ldg(d.cl_slot_start + key);
  const int ns = __ldg(d.cl_slot_start + key + 1) - sbase;
  copy_unrolled<4, int2>(
      ns, tid, nthr, [&](int i) { return d.cl_meta[sbase + i]; }, [&](int i, int2 v) { s_meta[i] = v; });
  copy_unrolled<4, float4>(
      ns, tid, nthr, [&](int i) { return __ldg(d.cl_wx + sbase + i); }, [&](int i, float4 v) { s_wx[i] = v; });
  copy_unrolled<8, float>(
      ns * W, tid, nthr, [&](int i) { return __ldg(d.cl_wy + (size_t)sbase * W + i); },
      [&](int i, float v) { s_wy[i] = v; });
  __syncthreads();
  const bool pair_ok = (Nt & 1) == 0;
  copy_unrolled<8, float2>(
      ns * NCP, tid, nthr,
      [&](int i) {
        const int slot = i / NCP, kk = i % NCP;
        const int n = n0 + 2 * kk;
        const float *row = g + (size_t)s_meta[slot].x * Nt;
        float2 v;
        if (pair_ok && n + 1 < Nt) {
          v = __ldg(reinterpret_cast<const float2 *>(row + n));
        } else {
          v.x = n < Nt ? __ldg(row + n) : 0.f;
          v.y = n + 1 < Nt ? __ldg(row + n + 1) : 0.f;
        }
        return v;
      },
      [&](int i, float2 v) { s_g[i] = v; });
  __syncthreads();

  float2 acc[GPW][P];
#pragma unroll
  for (int gi = 0; gi < GPW; ++gi)
#pragma unroll
    for (int r = 0; r < P; ++r) acc[gi][r] = make_float2(0.f, 0.f);
  const int *__restrict__ vst = d.cl_vstart + (size_t)key * NGH;
#pragma unroll
  for (int gi = 0; gi < GPW; ++gi) {
    const int grp = warp * GPW + gi;
    if (grp < NGH) {
      const int ql = grp * QG + qi;       // column within the half
      const int q = h * H + ql;
      const bool qok = ql < H;
      const int v0 = __ldg(vst + grp), v1 = __ldg(vst + grp + 1);
      for (int vb = v0; vb < v1; vb += 32) {
        const int mine = vb + lane < v1 ? __ldg(d.cl_vslot + vb + lane) : 0;
        const int cnt = min(32, v1 - vb);
#pragma unroll 2
        for (int j = 0; j < cnt; ++j) {
          const int slot = __shfl_sync(0xffffffffu, mine, j);
          int tq = q - s_meta[slot].y + W / 2 - 1;
          if (tq < 0) tq += My;
          if (tq >= My) tq -= My;
          const float wyq = (qok && tq < W) ? s_wy[slot * W + tq] : 0.f;
          const float4 wx4 = s_wx[slot];
          const float2 gv = s_g[slot * NCP + k];
          const float p0w = wyq * wx4.x, p1w = wyq * wx4.y, p2w = wyq * wx4.z, p3w = wyq * wx4.w;
          acc[gi][0].x = fmaf(p0w, gv.x, acc[gi][0].x);
          acc[gi][0].y = fmaf(p0w, gv.y, acc[gi][0].y);
          acc[gi][1].x = fmaf(p1w, gv.x, acc[gi][1].x);
          acc[gi][1].y = fmaf(p1w, gv.y, acc[gi][1].y);
          acc[gi][2].x = fmaf(p2w, gv.x, acc[gi][2].x);
          acc[gi][2].y = fmaf(p2w, gv.y, acc[gi][2].y);
          acc[gi][3].x = fmaf(p3w, gv.x, acc[gi][3].x);
          acc[gi][3].y = fmaf(p3w, gv.y, acc[gi][3].y);
        }
      }
    }
  }
#pragma unroll
  for (int gi = 0; gi < GPW; ++gi) {
    const int ql = (warp * GPW + gi) * QG + qi;
    if (ql < H) {
#pragma unroll
      for (int r = 0; r < P; ++r) strip[(ql * P + r) * NCP + k] = acc[gi][r];
    }
  }
  // radix-2 decimation in frequency across the pair
  cluster.sync();
  float2 *peer = cluster.map_shared_rank(strip, 1 - h);
  const float2 *tw = d.tw + d.fMy.tw;
  constexpr int PER = 16;  // values per thread per round (H*P*NCP / nthr for My = 256)
  const int total = H * P * NCP;
  for (int base = 0; base < total; base += nthr * PER) {
    float2 y[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int idx = base + j * nthr + tid;
      if (idx < total) {
        const float2 mine = strip[idx], other = peer[idx];
        const float2 a = h == 0 ? mine : other, b = h == 0 ? other : mine;  // x[q], x[q + H]
        if (h == 0) {
          y[j] = cadd(a, b);
        } else {
          const int ql = idx / (P * NCP);
          y[j] = cmul(csub(a, b), __ldg(tw + ql));
        }
      }
    }
    cluster.sync();  // the peer has read this block's values
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int idx = base + j * nthr + tid;
      if (idx < total) strip[idx] = y[j];
    }
    cluster.sync();  // next round reads values untouched by this round's writes
  }
  __syncthreads();
  fft_smem<-1>(strip, P * NCP, P * NCP, d.fMyh, d.tw, tid, nthr);
  // unpack (bins jy = 2k + h and My - jy live in this block), deconvolve, write
  const int nY1 = d.nY1;
  const int nk = (d.hy - h) / 2 + 1;  // jy = 2k + h <= hy
  const int tot = P * nk * NCP * 2;
  for (int idx = tid; idx < tot; idx += nthr) {
    const int par = idx & 1;
    const int kk = (idx >> 1) % NCP;
    const int rest = (idx >> 1) / NCP;
    const int kb = rest % nk;
    const int r = rest / nk;
    const int jy = 2 * kb + h;
    const int p = p0 + r;
    const int nn = n0 + 2 * kk + par;
    if (p < Mx && nn < Nt && jy <= d.hy) {
      const float2 Z = strip[(kb * P + r) * NCP + kk];
      const int km = h == 0 ? (kb == 0 ? 0 : H - kb) : H - kb - 1;
      const float2 Zm = strip[(km * P + r) * NCP + kk];
      float2 v;
      if (par == 0) {
        v = make_float2(0.5f * (Z.x + Zm.x), 0.5f * (Z.y - Zm.y));
      } else {
        v = make_float2(0.5f * (Z.y + Zm.y), -0.5f * (Z.x - Zm.x));
      }
      d.T[((size_t)p * nY1 + jy) * Nt + nn] = cscale(v, __ldg(d.invphy + jy));
    }
  }
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
    const float2 *Tsrc = d.T + (size_t)jy * Nt + n0;
    const size_t pstride = (size_t)nY1 * Nt;
    copy_unrolled<8, float2>(
        Mx * NC, tid, nthr,
        [&](int idx) {
          const int kk = idx % NC, p = idx / NC;
          return n0 + kk < Nt ? Tsrc[p * pstride + kk] : make_float2(0.f, 0.f);
        },
        [&](int idx, float2 v) { buf[idx] = v; });
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
    copy_unrolled<8, float2>(
        nX1 * NC, tid, nthr,
        [&](int idx) {
          const int kk = idx % NC, ix = idx / NC;
          const int n = n0 + kk;
          return n < Nt ? cscale(d.G1[((size_t)ix * nY1 + jy) * Nt + n], __ldg(d.invphx + ix))
                        : make_float2(0.f, 0.f);
        },
        [&](int idx, float2 v) {
          const int kk = idx % NC, ix = idx / NC;
          buf[wrap(ix - hx, Mx) * NC + kk] = v;
        });
    __syncthreads();
    fft_smem<+1>(buf, NC, NC, d.fMx, d.tw, tid, nthr);
    for (int idx = tid; idx < Mx * NC; idx += nthr) {
      const int kk = idx % NC, p = idx / NC;
      const int n = n0 + kk;
      if (n < Nt) d.T[((size_t)p * nY1 + jy) * Nt + n] = buf[idx];
    }
  }
}

// ------------------------------------------------------- adjoint row FFT
// Transpose of (spread-strip row FFT, unpack, deconvolution in y): for one
// grid row p and the sample pairs [n0, n0 + 2 NCP):
//   G0b[p][q][n] = Re sum_{jy=0}^{hy} (1/phihat_y(jy)) Tb[p][jy][n] exp(+2 pi i jy q / My)
// evaluated for two samples at once as one inverse FFT of the packed
// Hermitian spectrum S(jy) = (a + i b)/2, S(-jy) = (conj a + i conj b)/2,
// S(0) = Re a + i Re b, whose real and imaginary parts are the two results.
template <int NCP>
__global__ void __launch_bounds__(kThreadsCol) k_rowifft(const InstDesc *__restrict__ descs,
                                                         const int2 *__restrict__ work) {
  extern __shared__ float4 smem_f4[];
  float2 *S = reinterpret_cast<float2 *>(smem_f4);  // [My][NCP]
  int inst, tile;
  block_work(work, inst, tile);
  const InstDesc &d = descs[inst];
  const int Mx = d.Mx, My = d.My, Nt = d.Nt, hy = d.hy, nY1 = d.nY1;
  const int nchunks = (Nt + 2 * NCP - 1) / (2 * NCP);
  if (tile >= Mx * nchunks) return;
  const int p = tile % Mx;
  const int n0 = (tile / Mx) * 2 * NCP;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const float2 *Trow = d.T + (size_t)p * nY1 * Nt;
  for (int idx = tid; idx < My * NCP; idx += nthr) S[idx] = make_float2(0.f, 0.f);
  __syncthreads();
  // one (jy, pair) item reads two samples and fills bins jy and My - jy
  copy_unrolled<8, float4>(
      nY1 * NCP, tid, nthr,
      [&](int idx) {
        const int kk = idx % NCP, jy = idx / NCP;
        const int n = n0 + 2 * kk;
        const float sc = __ldg(d.invphy + jy);
        const float2 *src = Trow + (size_t)jy * Nt;
        const float2 a = n < Nt ? cscale(src[n], sc) : make_float2(0.f, 0.f);
        const float2 b = n + 1 < Nt ? cscale(src[n + 1], sc) : make_float2(0.f, 0.f);
        return make_float4(a.x, a.y, b.x, b.y);
      },
      [&](int idx, float4 ab) {
        const int kk = idx % NCP, jy = idx / NCP;
        if (jy == 0) {
          S[kk] = make_float2(ab.x, ab.z);
        } else {
          S[jy * NCP + kk] = make_float2(0.5f * (ab.x - ab.w), 0.5f * (ab.y + ab.z));
          S[(My - jy) * NCP + kk] = make_float2(0.5f * (ab.x + ab.w), 0.5f * (ab.z - ab.y));
        }
      });
  __syncthreads();
  fft_smem<+1>(S, NCP, NCP, d.fMy, d.tw, tid, nthr);
  float *G0 = d.G0 + (size_t)p * My * Nt;
  for (int idx = tid; idx < My * 2 * NCP; idx += nthr) {
    const int j = idx % (2 * NCP), q = idx / (2 * NCP);
    const int n = n0 + j;
    if (n < Nt) {
      const float2 v = S[q * NCP + (j >> 1)];
      G0[(size_t)q * Nt + n] = (j & 1) ? v.y : v.x;
    }
  }
}

// ---------------------------------------------------- adjoint interpolation
// g'[m][n] = sum_{r,t} wx[r] wy[t] G0b[bx - w/2 + 1 + r][by - w/2 + 1 + t][n]
// (wy carries a_m), the transpose of the spread.  One tile: the sensors whose
// base cell lies in a TX x TY block of the oversampled grid and 32 samples;
// the block loads the G0b cells of the tile plus the w-1 halo (periodic) into
// shared memory once, then each warp interpolates one sensor at a time with
// lane = sample.  GRAD also accumulates the window-derivative sums and the
// per-(chunk, sensor) position-gradient partials  sum_n g[m][n] (...).
template <int W, int TX, int TY, bool GRAD>
__global__ void __launch_bounds__(kThreadsInterp) k_interp(const InstDesc *__restrict__ descs,
                                                           const int2 *__restrict__ work, IoPtrs io0,
                                                           const IoPtrs *__restrict__ io_table) {
  constexpr int HX = TX + W - 1, HY = TY + W - 1, NC = 32;
  extern __shared__ float4 smem_f4[];
  float *Gs = reinterpret_cast<float *>(smem_f4);  // [HX][HY][NC]
  __shared__ int row_lo[TX], row_pref[TX + 1];
  int inst, tile;
  block_work(work, inst, tile);
  const InstDesc &d = descs[inst];
  const int Mx = d.Mx, My = d.My, Nt = d.Nt, M = d.M;
  const int ntx = (Mx + TX - 1) / TX, nty = (My + TY - 1) / TY;
  const int nchunks = (Nt + NC - 1) / NC;
  if (tile >= ntx * nty * nchunks) return;
  const int tx = tile % ntx;
  const int ty = (tile / ntx) % nty;
  const int c = tile / (ntx * nty);
  const int p0 = tx * TX, q0 = ty * TY, n0 = c * NC;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
  const IoPtrs io = io_of(io0, io_table, inst);

  // sensors of the tile: TX contiguous ranges of the sorted order
  if (tid == 0) {
    int acc = 0;
    for (int r = 0; r < TX; ++r) {
      const int p = p0 + r;
      int lo = 0, hi = 0;
      if (p < Mx) {
        lo = __ldg(d.cell_start + (size_t)p * My + q0);
        hi = __ldg(d.cell_start + (size_t)p * My + min(q0 + TY, My));
      }
      row_lo[r] = lo;
      row_pref[r] = acc;
      acc += hi - lo;
    }
    row_pref[TX] = acc;
  }
  // G0b tile with halo, 128-byte rows of 32 samples
  const float *G0 = d.G0;
  const bool vec4 = (Nt & 3) == 0;
  copy_unrolled<8, float4>(
      HX * HY * (NC / 4), tid, nthr,
      [&](int idx) {
        const int v4 = idx % (NC / 4), cell = idx / (NC / 4);
        const int hr = cell / HY, hc = cell % HY;
        const int p = wrap(p0 - W / 2 + 1 + hr, Mx), q = wrap(q0 - W / 2 + 1 + hc, My);
        const int n = n0 + 4 * v4;
        const float *src = G0 + ((size_t)p * My + q) * Nt + n;
        float4 v;
        if (vec4 && n + 3 < Nt) {
          v = __ldg(reinterpret_cast<const float4 *>(src));
        } else {
          v.x = n < Nt ? __ldg(src) : 0.f;
          v.y = n + 1 < Nt ? __ldg(src + 1) : 0.f;
          v.z = n + 2 < Nt ? __ldg(src + 2) : 0.f;
          v.w = n + 3 < Nt ? __ldg(src + 3) : 0.f;
        }
        return v;
      },
      [&](int idx, float4 v) { reinterpret_cast<float4 *>(Gs)[idx] = v; });
  __syncthreads();
  const int ns = row_pref[TX];
  const int n = n0 + lane;
  for (int u = warp; u < ns; u += nwarp) {
    int r = 0;
    while (r + 1 < TX && row_pref[r + 1] <= u) ++r;
    const int i = row_lo[r] + (u - row_pref[r]);
    const int bx = __ldg(d.sbx + i), by = __ldg(d.sby + i);
    const int hr0 = bx - p0, hc0 = by - q0;  // footprint starts at halo row hr0, column hc0
    float wxr[W], wyr[W], dwxr[W], dwyr[W];
#pragma unroll
    for (int t = 0; t < W; ++t) {
      wxr[t] = __ldg(d.wx + (size_t)i * W + t);
      wyr[t] = __ldg(d.wy + (size_t)i * W + t);
      if (GRAD) {
        dwxr[t] = __ldg(d.dwx + (size_t)i * W + t);
        dwyr[t] = __ldg(d.dwy + (size_t)i * W + t);
      }
    }
    float a0 = 0.f, ax = 0.f, ay = 0.f;
#pragma unroll
    for (int rr = 0; rr < W; ++rr) {
      const float *row = Gs + ((size_t)(hr0 + rr) * HY + hc0) * NC + lane;
      float rs = 0.f, rsy = 0.f;
#pragma unroll
      for (int t = 0; t < W; ++t) {
        const float v = row[t * NC];
        rs = fmaf(wyr[t], v, rs);
        if (GRAD) rsy = fmaf(dwyr[t], v, rsy);
      }
      a0 = fmaf(wxr[rr], rs, a0);
      if (GRAD) {
        ax = fmaf(dwxr[rr], rs, ax);
        ay = fmaf(wxr[rr], rsy, ay);
      }
    }
    const int m = __ldg(d.perm + i);
    if (io.g_out && n < Nt) io.g_out[(size_t)m * Nt + n] = a0;
    if (GRAD) {
      const float gv = n < Nt ? __ldg(io.g_in + (size_t)m * Nt + n) : 0.f;
      float px = ax * gv, py = ay * gv;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
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
size_t smem_spread(const InstDesc &d) { return (size_t)d.My * kSpreadP * kSpreadNCP * sizeof(float2); }
constexpr int kClGPW = 4;
int threads_spread_cluster(const InstDesc &d) {
  const int ngh = (d.My / 2 + kSpreadQG - 1) / kSpreadQG;
  int warps = (ngh + kClGPW - 1) / kClGPW;
  if (warps < 8) warps = 8;
  return warps * 32;
}
size_t smem_spread_cluster(const InstDesc &d) {
  const size_t smax = (size_t)d.cl_smax;
  return (size_t)(d.My / 2) * kSpreadP * kSpreadNCP * sizeof(float2) + smax * sizeof(float4) +
         smax * kSpreadNCP * sizeof(float2) + smax * sizeof(int2) + smax * d.w * sizeof(float);
}
int blocks_colfft(const InstDesc &d) { return d.nY1 * ((d.Nt + kColNC - 1) / kColNC); }
size_t smem_colfft(const InstDesc &d) { return (size_t)d.Mx * kColNC * sizeof(float2); }
constexpr int kRowIfftNCP = 16;
constexpr int kInterpTX = 8, kInterpTY = 32;
int interp_ty(const InstDesc &d) { return d.w <= 8 ? kInterpTY : 16; }
int blocks_rowifft(const InstDesc &d) { return d.Mx * ((d.Nt + 2 * kRowIfftNCP - 1) / (2 * kRowIfftNCP)); }
size_t smem_rowifft(const InstDesc &d) { return (size_t)d.My * kRowIfftNCP * sizeof(float2); }
int blocks_interp(const InstDesc &d) {
  const int ty = interp_ty(d);
  return ((d.Mx + kInterpTX - 1) / kInterpTX) * ((d.My + ty - 1) / ty) * ((d.Nt + 31) / 32);
}
size_t smem_interp(const InstDesc &d) {
  return (size_t)(kInterpTX + d.w - 1) * (interp_ty(d) + d.w - 1) * 32 * sizeof(float);
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

template <int W>
static cudaError_t launch_spread_cl_w(const Launch &L, int threads) {
  auto kern = k_spread_cl<kSpreadP, kSpreadNCP, kClGPW, W>;
  cudaError_t e = set_smem(kern, L.smem);
  if (e != cudaSuccess) return e;
  kern<<<L.nblocks, threads, L.smem, L.stream>>>(L.descs, L.work, L.io, L.io_table);
  return cudaGetLastError();
}

cudaError_t launch_spread_cluster(const Launch &L, int threads, int width) {
  switch (width) {
    case 6: return launch_spread_cl_w<6>(L, threads);
    case 8: return launch_spread_cl_w<8>(L, threads);
    case 12: return launch_spread_cl_w<12>(L, threads);
    case 16: return launch_spread_cl_w<16>(L, threads);
    default: return cudaErrorInvalidValue;
  }
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

template <int W, int TY, bool GRAD>
static cudaError_t launch_interp_w(const Launch &L) {
  auto kern = k_interp<W, kInterpTX, TY, GRAD>;
  cudaError_t e = set_smem(kern, L.smem);
  if (e != cudaSuccess) return e;
  kern<<<L.nblocks, kThreadsInterp, L.smem, L.stream>>>(L.descs, L.work, L.io, L.io_table);
  return cudaGetLastError();
}

cudaError_t launch_interp_width(const Launch &L, int width, bool grad) {
  switch (width) {
    case 6: return grad ? launch_interp_w<6, kInterpTY, true>(L) : launch_interp_w<6, kInterpTY, false>(L);
    case 8: return grad ? launch_interp_w<8, kInterpTY, true>(L) : launch_interp_w<8, kInterpTY, false>(L);
    case 12: return grad ? launch_interp_w<12, 16, true>(L) : launch_interp_w<12, 16, false>(L);
    case 16: return grad ? launch_interp_w<16, 16, true>(L) : launch_interp_w<16, 16, false>(L);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_rowifft(const Launch &L) {
  auto kern = k_rowifft<kRowIfftNCP>;
  cudaError_t e = set_smem(kern, L.smem);
  if (e != cudaSuccess) return e;
  kern<<<L.nblocks, kThreadsCol, L.smem, L.stream>>>(L.descs, L.work);
  return cudaGetLastError();
}

cudaError_t launch_grad_reduce(const Launch &L, int n_inst) {
  k_grad_reduce<<<L.nblocks, 256, 0, L.stream>>>(L.descs, L.io, L.io_table, n_inst);
  return cudaGetLastError();
}

}  // namespace pa
