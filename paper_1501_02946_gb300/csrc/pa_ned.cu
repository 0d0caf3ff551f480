// pa_ned.cu -- NED-NUFFT stage (the spatial type-1 NUFFT of Sec. 3) on sm_103a.
//
// Forward:  g[m][n] --spread--> G0[p][q][n] (real, oversampled sigma*nx x
// sigma*ny grid) --FFT over q, keep jy = 0..hy--> T[p][jy][n] --FFT over p,
// keep jx = -hx..hx, divide by phihat--> G1[jx][jy][n].
//   k_spread    gather-form spread (sparse x dense), sums in registers.
//   k_rowfft    row FFT over q of two samples at once, deconvolution in y.
//   k_colfft    column FFT + truncation + deconvolution (and its adjoint).
// Adjoint:  the exact transposes: k_colfft<true>, k_rowifft (inverse row
// FFT back to the G0 cotangent) and k_interp (interpolation at the sensors,
// optionally with the sensor-position gradient through the window
// derivative).
#include <cstring>

#include "pa_device.cuh"
#include "pa_tmap.h"

// Blocks per SM the pipelined interpolation's register budget is set for
// (its two 54 KB stages allow two).
#ifndef PA_INTERP_MINB
#define PA_INTERP_MINB 2
#endif
#ifndef PA_INTERP_THREADS
#define PA_INTERP_THREADS 256
#endif
// Spread: entries whose g rows load together, and the blocks per SM its
// register budget is set for.
#ifndef PA_SPREAD_B
#define PA_SPREAD_B 4
#endif
#ifndef PA_SPREAD_MINB
#define PA_SPREAD_MINB 2
#endif
// 1: the row FFT's unpacked rows leave shared memory by TMA stores
#ifndef PA_ROWFFT_TMA_STORE
#define PA_ROWFFT_TMA_STORE 1
#endif
#ifndef PA_ROWFFT_STORE_MIN_MY
#define PA_ROWFFT_STORE_MIN_MY 0
#endif
// 1: the column FFT's tiles leave shared memory by TMA stores
#ifndef PA_COLFFT_TMA_STORE
#define PA_COLFFT_TMA_STORE 1
#endif
// 1: the inverse row FFT's tiles leave shared memory by TMA stores
#ifndef PA_ROWIFFT_TMA_STORE
#define PA_ROWIFFT_TMA_STORE 1
#endif
// blocks per SM the staged spread's register budget is set for
#ifndef PA_SPREAD_TILE_MINB
#define PA_SPREAD_TILE_MINB 4
#endif
#ifndef PA_SPREAD_TILE4_MINB
#define PA_SPREAD_TILE4_MINB 4
#endif
// 1: single-plan spreads stage their g rows in shared memory (k_spread_tile)
#ifndef PA_SPREAD_TILE
#define PA_SPREAD_TILE 1
#endif

namespace pa {

namespace {

constexpr int kThreadsCol = 256;
// Tiles of the persistent transform pipelines of length 2^LGL: nc sample
// pairs (row transforms) or complex samples (column transform) per tile,
// threads per block, and the blocks per SM their registers are budgeted for.
// Below length 512: 16 per tile, 256 threads.  From length 512 on, PA_FFT9_NCP
// per tile, PA_FFT9_THREADS threads and PA_FFT9_MINB blocks per SM: 8, 256
// and 2 (two tile buffers of 32 KB; two blocks per SM hide each other's
// barrier waits between the transform passes), or 16, 512 and 1.
#ifndef PA_FFT9_NCP
#define PA_FFT9_NCP 8
#endif
// Blocks per SM the shorter pipelines budget registers for (with a budget
// for one, ptxas gives them 131-183 registers and one 256-thread block per
// SM: at 128x128x256 the inverse row FFT took 64 us instead of 50).
#ifndef PA_FFT_MINB
#define PA_FFT_MINB 2
#endif
#ifndef PA_FFT9_THREADS
#define PA_FFT9_THREADS 256
#endif
#ifndef PA_FFT9_MINB
#define PA_FFT9_MINB 2
#endif
static_assert(PA_FFT9_NCP == 16 || PA_FFT9_NCP == 8 || PA_FFT9_NCP == 4, "length-512 tile width");
// 1: the 512-point inverse row FFT reads its unfilled bins nY1 .. L - nY1 as
// zeros instead of clearing them (skipping truncated bins on output in the
// forward transforms, or the dropped bins on input of the adjoint column
// transform, was slower: 357 -> 431, 195 -> 234, 221 -> 235 us).
#ifndef PA_FFT9_BAND
#define PA_FFT9_BAND 1
#endif
__host__ __device__ constexpr int pipe_nc(int lgl) { return lgl >= 9 ? PA_FFT9_NCP : 16; }
template <int LGL>
struct PipeTile {
  static constexpr int threads = LGL >= 9 ? PA_FFT9_THREADS : 256;
  static constexpr int minb = LGL >= 9 ? PA_FFT9_MINB : PA_FFT_MINB;
  static constexpr int nc = pipe_nc(LGL);
  static constexpr int lgnc = nc == 16 ? 4 : (nc == 8 ? 3 : 2);
  static constexpr bool band = LGL == 9 && PA_FFT9_BAND;
};
constexpr int kThreadsSpread = 256;  // 8 warps = 8 grid columns of one strip
constexpr int kThreadsInterp = 256;

__device__ __forceinline__ IoPtrs io_of(const IoPtrs &io, const IoPtrs *table, int inst) {
  return table ? table[inst] : io;
}

// ------------------------------------------------------------------ spread
// Gather form of the forward spread, a sparse-times-dense product:
//   G0[p][q][n] = sum_e sp_w[e][p - p0] * g[sp_m[e]][n]
// over the entries e of (strip p0 / P, column q), where sp_w holds the tap
// products wy(q) wx(p) of the sensor for the strip's P rows.  A warp owns one
// column of one strip and lane l the S consecutive samples n0 + l*S ..; an
// entry costs two warp-uniform loads (caller index, four products) and S/4
// vector loads of g for 4*S FMAs, and the P x S sums stay in registers (no
// shared memory, no atomics, no barrier).  The warps of a block own
// neighbouring columns of the same strip, which walk nearly the same sensors
// in the same order, so their reads of g mostly hit in L1.
template <int S>
__device__ __forceinline__ void load_samples(const float *__restrict__ row, int n, int Nt, bool vec, float (&v)[S]) {
  if (vec) {
#pragma unroll
    for (int u = 0; u < S / 4; ++u) {
      const float4 t = __ldg(reinterpret_cast<const float4 *>(row + n) + u);
      v[4 * u] = t.x;
      v[4 * u + 1] = t.y;
      v[4 * u + 2] = t.z;
      v[4 * u + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int u = 0; u < S; ++u) v[u] = n + u < Nt ? __ldg(row + n + u) : 0.f;
  }
}

// acc += w * v on four components as two packed two-wide FMAs
__device__ __forceinline__ void fma4(float w, const float4 &v, float4 &acc) {
  const float2 ww = make_float2(w, w);
  const float2 lo = __ffma2_rn(ww, make_float2(v.x, v.y), make_float2(acc.x, acc.y));
  const float2 hi = __ffma2_rn(ww, make_float2(v.z, v.w), make_float2(acc.z, acc.w));
  acc = make_float4(lo.x, lo.y, hi.x, hi.y);
}

template <int S>
__device__ __forceinline__ void fma_entry(float (&acc)[kSpreadP][S], const float4 &w, const float (&v)[S]) {
  // packed two-wide FMAs over sample pairs (each component rounds as fmaf)
#pragma unroll
  for (int u = 0; u < S; u += 2) {
    const float2 vv = make_float2(v[u], v[u + 1]);
    float2 a;
    a = __ffma2_rn(make_float2(w.x, w.x), vv, make_float2(acc[0][u], acc[0][u + 1]));
    acc[0][u] = a.x;
    acc[0][u + 1] = a.y;
    a = __ffma2_rn(make_float2(w.y, w.y), vv, make_float2(acc[1][u], acc[1][u + 1]));
    acc[1][u] = a.x;
    acc[1][u + 1] = a.y;
    a = __ffma2_rn(make_float2(w.z, w.z), vv, make_float2(acc[2][u], acc[2][u + 1]));
    acc[2][u] = a.x;
    acc[2][u + 1] = a.y;
    a = __ffma2_rn(make_float2(w.w, w.w), vv, make_float2(acc[3][u], acc[3][u + 1]));
    acc[3][u] = a.x;
    acc[3][u + 1] = a.y;
  }
}

template <int S>
__global__ void __launch_bounds__(kThreadsSpread, PA_SPREAD_MINB) k_spread(const InstDesc *__restrict__ descs,
                                                              const int2 *__restrict__ work, IoPtrs io0,
                                                              const IoPtrs *__restrict__ io_table) {
  griddep_enter();  // the previous kernel of the stream has completed
  constexpr int P = kSpreadP, QC = kThreadsSpread / 32, CH = 32 * S;
  static_assert(P == 4, "tap products hold four rows");
  static_assert(S % 4 == 0, "samples per lane load as float4");
  int inst, tile;
  block_work(work, inst, tile);
  const InstDesc &d = descs[inst];
  const int Mx = d.Mx, My = d.My, Nt = d.Nt;
  const int nstrips = (Mx + P - 1) / P, ncb = (My + QC - 1) / QC, nch = (Nt + CH - 1) / CH;
  if (tile >= nstrips * ncb * nch) return;
  const int st = tile % nstrips;
  const int cb = (tile / nstrips) % ncb;
  const int c = tile / (nstrips * ncb);
  const int q = cb * QC + (threadIdx.x >> 5);
  if (q >= My) return;  // whole warps leave; the kernel has no block barrier
  const int lane = threadIdx.x & 31;
  const int p0 = st * P;
  const int n = c * CH + lane * S;
  const IoPtrs io = io_of(io0, io_table, inst);
  const float *__restrict__ g = io.g_in;
  const bool rows16 = (Nt & 3) == 0;
  const bool vec = rows16 && ((reinterpret_cast<uintptr_t>(g) & 15u) == 0) && (n + S <= Nt);
  const int *__restrict__ em = d.sp_m;
  const float4 *__restrict__ ew = d.sp_w;
  const int e0 = __ldg(d.sp_start + (size_t)st * My + q), e1 = __ldg(d.sp_start + (size_t)st * My + q + 1);

  float acc[P][S];
#pragma unroll
  for (int r = 0; r < P; ++r)
#pragma unroll
    for (int u = 0; u < S; ++u) acc[r][u] = 0.f;

  // Entries in windows of 32: lane j loads entry j's caller index and tap
  // products (one coalesced load each), entry b reaches every lane by a
  // shuffle.  Within a window the g rows of batch k + 1 (B entries) load
  // while batch k is summed, so only the g loads remain on the path.
  constexpr int B = PA_SPREAD_B;
  for (int e = e0; e < e1; e += 32) {
    const int cnt = min(32, e1 - e);
    int mj = 0;
    float4 wj = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lane < cnt) {
      mj = __ldg(em + e + lane);
      wj = __ldg(ew + e + lane);
    }
    const int nb = (cnt + B - 1) / B;
    float va[B][S], vb[B][S];
    auto load_batch = [&](int k, float (&v)[B][S]) {
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int j = k * B + b;
        const int m = __shfl_sync(0xffffffffu, mj, j & 31);
        if (j < cnt) {
          load_samples<S>(g + (size_t)m * Nt, n, Nt, vec, v[b]);
        } else {
#pragma unroll
          for (int u = 0; u < S; ++u) v[b][u] = 0.f;
        }
      }
    };
    auto sum_batch = [&](int k, const float (&v)[B][S]) {
#pragma unroll
      for (int b = 0; b < B; ++b) {
        const int j = (k * B + b) & 31;
        const float4 w = make_float4(__shfl_sync(0xffffffffu, wj.x, j), __shfl_sync(0xffffffffu, wj.y, j),
                                     __shfl_sync(0xffffffffu, wj.z, j), __shfl_sync(0xffffffffu, wj.w, j));
        fma_entry<S>(acc, w, v[b]);  // entries past cnt carry zero products and samples
      }
    };
    load_batch(0, va);
#pragma unroll 1
    for (int k = 0; k < nb; k += 2) {
      if (k + 1 < nb) load_batch(k + 1, vb);
      sum_batch(k, va);
      if (k + 1 >= nb) break;
      if (k + 2 < nb) load_batch(k + 2, va);
      sum_batch(k + 1, vb);
    }
  }
  if (n >= Nt) return;
  const bool vst = rows16 && (n + S <= Nt);
#pragma unroll
  for (int r = 0; r < P; ++r) {
    const int p = p0 + r;
    if (p >= Mx) break;
    float *dst = d.G0 + ((size_t)p * My + q) * Nt + n;
    if (vst) {
#pragma unroll
      for (int u = 0; u < S / 4; ++u)
        reinterpret_cast<float4 *>(dst)[u] =
            make_float4(acc[r][4 * u], acc[r][4 * u + 1], acc[r][4 * u + 2], acc[r][4 * u + 3]);
    } else {
#pragma unroll
      for (int u = 0; u < S; ++u)
        if (n + u < Nt) dst[u] = acc[r][u];
    }
  }
}

// The spread with the block's g rows staged in shared memory.  A block
// (8 warps = the 8 columns q0 .. q0 + 7 of one strip, one chunk of CH = 32 S
// samples) first copies into shared memory, with bulk copies (TMA engine):
// the chunk of every g row its entries use -- its union of sensors, most
// used first, one copy per row -- and its entries (tap products and union
// slots: the 8 lists of its columns are one contiguous range).  It then sums
// exactly as k_spread does (same entries, same order, so the same results),
// reading only shared memory: broadcast loads for the entries, and lane l
// holds the samples n0 + 4 l + 128 k (k < S / 4) of each row (16-byte,
// bank-conflict-free loads).  Union rows past the buffer's sp_urows rows (the
// least used; the buffer is sized so that four blocks share an SM) are read
// from global memory.
template <int S>
struct SpreadTile {
  static constexpr int CH = 32 * S;
  // floats: g rows, then the entries' products (4 floats each), then their
  // slots (+ 8 for the 16-byte rounding of the copy)
  __host__ __device__ static size_t floats(int urows, int emax) {
    return size_t(urows) * CH + 4 * size_t(emax) + size_t(emax) + 8;
  }
};

template <int S>
__global__ void __launch_bounds__(kThreadsSpread, S == 4 ? PA_SPREAD_TILE4_MINB : PA_SPREAD_TILE_MINB) k_spread_tile(const InstDesc *__restrict__ descs, IoPtrs io) {
  griddep_enter();  // the previous kernel of the stream has completed
  constexpr int P = kSpreadP, QC = kSpreadQC, CH = SpreadTile<S>::CH, K4 = S / 4;
  static_assert(P == 4 && QC * 32 == kThreadsSpread, "tile shape");
  static_assert(S % 4 == 0, "samples per lane load as float4");
  extern __shared__ __align__(128) float4 smem_a128[];
  float *Gs = reinterpret_cast<float *>(smem_a128);  // [sp_urows][CH]
  __shared__ __align__(8) uint64_t bar;
  const InstDesc &d = descs[0];
  const int Mx = d.Mx, My = d.My, Nt = d.Nt;
  const int nstrips = (Mx + P - 1) / P, ncb = (My + QC - 1) / QC, nch = (Nt + CH - 1) / CH;
  const int tile = blockIdx.x;
  if (tile >= nstrips * ncb * nch) return;
  const int st = tile % nstrips;
  const int cb = (tile / nstrips) % ncb;
  const int c = tile / (nstrips * ncb);
  const int n0 = c * CH;
  const int nv = min(CH, Nt - n0);  // samples of the chunk (a multiple of 4)
  const float *__restrict__ g = io.g_in;
  const int blk = st * ncb + cb;
  const int u0 = __ldg(d.sp_ustart + blk), nu = __ldg(d.sp_ustart + blk + 1) - u0;
  const int ur = min(nu, d.sp_urows);
  const int2 er = __ldg(d.sp_erange + blk);
  const int ne = er.y - er.x, ea_al = er.x & ~3, eb_al = (er.y + 3) & ~3;
  float4 *W = reinterpret_cast<float4 *>(Gs + (size_t)d.sp_urows * CH);  // [sp_emax] tap products
  int *SL = reinterpret_cast<int *>(W + d.sp_emax);                      // slots from entry ea_al on
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0)
    mbar_arrive_expect_tx(&bar, uint32_t(ur) * uint32_t(nv) * 4u + uint32_t(ne) * 16u + uint32_t(eb_al - ea_al) * 4u);
  for (int u = tid; u < ur; u += kThreadsSpread)
    bulk_g2s(Gs + (size_t)u * CH, g + (size_t)__ldg(d.sp_um + u0 + u) * Nt + n0, uint32_t(nv) * 4u, &bar);
  if (tid == kThreadsSpread - 32 && ne > 0) bulk_g2s(W, d.sp_w + er.x, uint32_t(ne) * 16u, &bar);
  if (tid == kThreadsSpread - 31 && eb_al > ea_al) bulk_g2s(SL, d.sp_slot + ea_al, uint32_t(eb_al - ea_al) * 4u, &bar);
  // the warp's list bounds load while the copies are in flight
  const int q = cb * QC + (tid >> 5);
  int e0 = 0, e1 = 0;
  if (q < My) {
    e0 = __ldg(d.sp_start + (size_t)st * My + q) - er.x;
    e1 = __ldg(d.sp_start + (size_t)st * My + q + 1) - er.x;
  }
  if (__syncthreads_or(!mbar_wait(&bar, 0))) {
    if (tid == 0) atomicOr(d.status, kStatusWaitTimeout);
    mbar_wait(&bar, 0);  // one more bounded wait for the copies in flight
    return;
  }
  if (q >= My) return;  // whole warps leave; no block barrier follows
  const int p0 = st * P;
  const int *SLe = SL + (er.x - ea_al);  // slot of block entry e at SLe[e]
  float4 acc[P][K4];
#pragma unroll
  for (int r = 0; r < P; ++r)
#pragma unroll
    for (int k = 0; k < K4; ++k) acc[r][k] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
  for (int e = e0; e < e1; ++e) {
    const int slot = SLe[e];
    const float4 w = W[e];
    float4 v[K4];
    if (slot < ur) {
      const float4 *row = reinterpret_cast<const float4 *>(Gs + (size_t)slot * CH) + lane;
#pragma unroll
      for (int k = 0; k < K4; ++k) v[k] = row[32 * k];
    } else {
      const float *row = g + (size_t)__ldg(d.sp_um + u0 + slot) * Nt + n0 + 4 * lane;
#pragma unroll
      for (int k = 0; k < K4; ++k)
        v[k] = 4 * lane + 128 * k < nv ? __ldg(reinterpret_cast<const float4 *>(row + 128 * k))
                                       : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < K4; ++k) {
      fma4(w.x, v[k], acc[0][k]);
      fma4(w.y, v[k], acc[1][k]);
      fma4(w.z, v[k], acc[2][k]);
      fma4(w.w, v[k], acc[3][k]);
    }
  }
#pragma unroll
  for (int r = 0; r < P; ++r) {
    const int p = p0 + r;
    if (p >= Mx) break;
    float *dst = d.G0 + ((size_t)p * My + q) * Nt + n0 + 4 * lane;
#pragma unroll
    for (int k = 0; k < K4; ++k)
      if (4 * lane + 128 * k < nv) *reinterpret_cast<float4 *>(dst + 128 * k) = acc[r][k];
  }
}

// Row transform of the spread grid, the transpose of k_rowifft:
//   T[p][jy][n] = (1/phihat_y(jy)) sum_q G0[p][q][n] exp(-2 pi i jy q / My),  jy = 0..hy,
// two real samples per complex FFT (n in the real part, n + 1 in the
// imaginary part), separated afterwards through the Hermitian symmetry.
template <int NCP>
__global__ void __launch_bounds__(kThreadsCol) k_rowfft(const InstDesc *__restrict__ descs,
                                                        const int2 *__restrict__ work) {
  extern __shared__ float4 smem_f4[];
  float2 *S = reinterpret_cast<float2 *>(smem_f4);  // [My][NCP]
  static_assert(NCP % 2 == 0, "pairs load as float4");
  int inst, tile;
  block_work(work, inst, tile);
  const InstDesc &d = descs[inst];
  const int Mx = d.Mx, My = d.My, Nt = d.Nt, nY1 = d.nY1;
  const int nchunks = (Nt + 2 * NCP - 1) / (2 * NCP);
  if (tile >= Mx * nchunks) return;
  // chunk fastest: blocks that run together cover contiguous runs of each row
  const int p = tile / nchunks;
  const int n0 = (tile % nchunks) * 2 * NCP;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const float *G0 = d.G0 + (size_t)p * My * Nt;
  const bool vec4 = (Nt & 3) == 0;
  constexpr int K2 = NCP / 2;
  copy_unrolled<8, float4>(
      My * K2, tid, nthr,
      [&](int idx) {
        const int k2 = idx % K2, q = idx / K2;
        const int n = n0 + 4 * k2;
        const float *src = G0 + (size_t)q * Nt + n;
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
      [&](int idx, float4 v) { reinterpret_cast<float4 *>(S)[idx] = v; });
  __syncthreads();
  fft_smem<-1>(S, NCP, NCP, d.fMy, d.tw, tid, nthr);
  float2 *Trow = d.T + (size_t)p * nY1 * Nt;
  const bool vst = (Nt & 1) == 0;
  for (int idx = tid; idx < nY1 * NCP; idx += nthr) {
    const int k = idx % NCP, jy = idx / NCP;
    const int n = n0 + 2 * k;
    if (n >= Nt) continue;
    const float2 Z = S[jy * NCP + k];
    const float2 Zm = S[(jy == 0 ? 0 : My - jy) * NCP + k];
    const float sc = 0.5f * __ldg(d.invphy + jy);
    const float2 a = make_float2(sc * (Z.x + Zm.x), sc * (Z.y - Zm.y));
    const float2 b = make_float2(sc * (Z.y + Zm.y), -sc * (Z.x - Zm.x));
    float2 *dst = Trow + (size_t)jy * Nt + n;
    if (vst) {
      *reinterpret_cast<float4 *>(dst) = make_float4(a.x, a.y, b.x, b.y);
    } else {
      dst[0] = a;
      if (n + 1 < Nt) dst[1] = b;
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
  const int jy = tile / nchunks;
  const int n0 = (tile % nchunks) * NC;
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

// Persistent, double-buffered column FFT for Mx = 2^LGL and even Nt (one
// plan): the rows of the next tile arrive by bulk copies (TMA engine) while
// the current tile is transformed.  Same arithmetic as k_colfft.
// With use_map the rows arrive as boxes of a 3-D tensor map (floats): over T
// (dims 2 Nt, nY1, Mx; box 2 NC x 1 x min(Mx, 256)) forward, over G1 (dims
// 2 Nt, nY1, nX1; box 2 NC x 1 x (hx + kb), kb = use_map, 1 to 4) for the
// adjoint, whose two boxes start at rows hx and -kb (rows outside the grid
// read as zeros and land on bins that are cleared anyway); kb makes the
// second box's destination, bin L - hx - kb, 128-byte aligned.
// With use_omap (adjoint), the transformed tile leaves shared memory as boxes
// of the 3-D tensor map omap over T (the forward's input map) stored by the
// TMA engine; the buffer is refilled only after the stores have read it.
// In the forward, with use_omap the scaled bins leave as two boxes of the
// 3-D maps over G1 (box heights hx + 1 for rows hx .. 2 hx, from bins
// 0 .. hx, in omap; hx for rows 0 .. hx - 1, from bins L - hx .. L - 1, in
// omap2).
template <bool ADJ, int LGL>
__global__ void __launch_bounds__(PipeTile<LGL>::threads, PipeTile<LGL>::minb) k_colfft_pipe(const InstDesc *__restrict__ descs, int nwork,
                                                             const __grid_constant__ CUtensorMap map, int use_map,
                                                             const __grid_constant__ CUtensorMap omap, int use_omap,
                                                             const __grid_constant__ CUtensorMap omap2) {
  griddep_enter();  // the previous kernel of the stream has completed
  extern __shared__ __align__(128) float4 smem_a128[];  // box destinations 128-byte aligned
  __shared__ __align__(8) uint64_t bars[2];
  constexpr int L = 1 << LGL, NC = PipeTile<LGL>::nc, LGNC = PipeTile<LGL>::lgnc, BOX = L < 256 ? L : 256;
  static_assert(NC == 1 << LGNC, "tile width");
  float2 *buf0 = reinterpret_cast<float2 *>(smem_a128);
  float2 *buf1 = buf0 + L * NC;
  const InstDesc &d = descs[0];
  if (!smem_aligned_128(smem_a128, d.status)) return;
  const int Nt = d.Nt, nY1 = d.nY1, nX1 = d.nX1, hx = d.hx;
  const int nchunks = (Nt + NC - 1) / NC;
  const int tid = threadIdx.x, nthr = blockDim.x, lgT = ilog2_pow2(nthr);
  const float2 *tw = d.tw + d.fMx.tw;
  auto issue = [&](int w, float2 *buf, uint64_t *bar) {
    const int jy = w / nchunks, n0 = (w - jy * nchunks) * NC;
    if (use_map) {
      if (tid == 0) {
        if (!ADJ) {
          if (use_omap) bulk_wait_read<0>();  // this buffer's last tile has been stored
          mbar_arrive_expect_tx(bar, uint32_t(L * NC * sizeof(float2)));
          for (int b = 0; b < L; b += BOX) tma_load_3d(buf + b * NC, &map, 2 * n0, jy, b, bar);
        } else {
          if (use_omap) bulk_wait_read<0>();  // this buffer's last tile has been stored
          const int kb = use_map;
          mbar_arrive_expect_tx(bar, uint32_t(2 * (hx + kb) * NC * sizeof(float2)));
          tma_load_3d(buf, &map, 2 * n0, jy, hx, bar);                          // ix = hx .. 2 hx (+ zeros)
          tma_load_3d(buf + (L - hx - kb) * NC, &map, 2 * n0, jy, -kb, bar);  // ix = -kb .. hx - 1
        }
      }
      return;
    }
    const uint32_t rb = uint32_t(min(NC, Nt - n0)) * sizeof(float2);
    if (!ADJ) {
      if (tid == 0) mbar_arrive_expect_tx(bar, rb * L);
      for (int p = tid; p < L; p += nthr) bulk_g2s(buf + p * NC, d.T + ((size_t)p * nY1 + jy) * Nt + n0, rb, bar);
    } else {
      if (tid == 0) mbar_arrive_expect_tx(bar, rb * nX1);
      for (int ix = tid; ix < nX1; ix += nthr)
        bulk_g2s(buf + ((ix - hx) & (L - 1)) * NC, d.G1 + ((size_t)ix * nY1 + jy) * Nt + n0, rb, bar);
    }
  };
  auto compute = [&](int w, float2 *buf) {
    const int jy = w / nchunks, n0 = (w - jy * nchunks) * NC;
    if (!ADJ) {
      fft_fixed<LGL, -1>(buf, NC, LGNC, lgT, tw, tid);
      if (use_omap) {
        // scale the kept bins in place (bin (ix - hx) mod L holds row ix)
        for (int idx = tid; idx < nX1 * NC; idx += nthr) {
          const int kk = idx & (NC - 1), ix = idx >> LGNC;
          float2 *q = buf + ((ix - hx) & (L - 1)) * NC + kk;
          *q = cscale(*q, __ldg(d.invphx + ix));
        }
        fence_proxy_async_smem();  // the writes precede the stores' reads
        __syncthreads();
        if (tid == 0) {
          tma_store_3d(&omap, 2 * n0, jy, hx, buf);
          if (hx > 0) tma_store_3d(&omap2, 2 * n0, jy, 0, buf + (L - hx) * NC);
          bulk_commit();
        }
        return;
      }
      for (int idx = tid; idx < nX1 * NC; idx += nthr) {
        const int kk = idx & (NC - 1), ix = idx >> LGNC;
        const int n = n0 + kk;
        if (n < Nt)
          d.G1[((size_t)ix * nY1 + jy) * Nt + n] = cscale(buf[((ix - hx) & (L - 1)) * NC + kk], __ldg(d.invphx + ix));
      }
    } else {
      // bins jx mod Mx hold G1 row jx + hx; scale them, clear the others
      for (int idx = tid; idx < L * NC; idx += nthr) {
        const int r = idx >> LGNC;
        const int ix = (r + hx) & (L - 1);
        buf[idx] = ix < nX1 ? cscale(buf[idx], __ldg(d.invphx + ix)) : make_float2(0.f, 0.f);
      }
      __syncthreads();
      fft_fixed<LGL, +1>(buf, NC, LGNC, lgT, tw, tid);
      if (use_omap) {
        fence_proxy_async_smem();  // the transform's writes precede the stores' reads
        __syncthreads();
        if (tid == 0) {
          for (int b = 0; b < L; b += BOX) tma_store_3d(&omap, 2 * n0, jy, b, buf + b * NC);
          bulk_commit();
        }
        return;
      }
      for (int idx = tid; idx < L * NC; idx += nthr) {
        const int kk = idx & (NC - 1), p = idx >> LGNC;
        const int n = n0 + kk;
        if (n < Nt) d.T[((size_t)p * nY1 + jy) * Nt + n] = buf[idx];
      }
    }
  };
  tile_pipeline(nwork, buf0, buf1, bars, d.status, issue, compute);
  if (use_omap && tid == 0) bulk_wait<0>();  // every store complete before the block exits
}

// Persistent, double-buffered row FFT (k_rowfft) for My = 2^LGL and
// Nt % 4 == 0 (one plan).
// With use_map, a tile arrives as boxes of the 2-D tensor map over G0
// (dims Nt, Mx My; box 32 x min(My, 256)) instead of one copy per row q.
// With use_omap = hb > 0 (and use_map), the unpacked rows are staged in a
// third buffer [nY1][32 complex] and leave as boxes of the 2-D map omap over
// T (floats; dims 2 Nt, Mx nY1; box 64 x hb): one box when hb = nY1, else
// two (rows [0, hb) and [nY1 - hb, nY1)).
template <int LGL>
__global__ void __launch_bounds__(PipeTile<LGL>::threads, PipeTile<LGL>::minb) k_rowfft_pipe(const InstDesc *__restrict__ descs, int nwork,
                                                             const __grid_constant__ CUtensorMap map, int use_map,
                                                             const __grid_constant__ CUtensorMap omap, int use_omap) {
  griddep_enter();  // the previous kernel of the stream has completed
  extern __shared__ __align__(128) float4 smem_a128[];  // box destinations 128-byte aligned
  __shared__ __align__(8) uint64_t bars[2];
  constexpr int L = 1 << LGL, NCP = PipeTile<LGL>::nc, LGNCP = PipeTile<LGL>::lgnc, BOX = L < 256 ? L : 256;
  float2 *buf0 = reinterpret_cast<float2 *>(smem_a128);  // [My][NCP] sample pairs
  float2 *buf1 = buf0 + L * NCP;
  const InstDesc &d = descs[0];
  if (!smem_aligned_128(smem_a128, d.status)) return;
  const int Nt = d.Nt, nY1 = d.nY1;
  const int nchunks = (Nt + 2 * NCP - 1) / (2 * NCP);
  const int tid = threadIdx.x, nthr = blockDim.x, lgT = ilog2_pow2(nthr);
  const float2 *tw = d.tw + d.fMy.tw;
  auto issue = [&](int w, float2 *buf, uint64_t *bar) {
    const int p = w / nchunks, n0 = (w - p * nchunks) * 2 * NCP;
    if (use_map) {
      if (tid == 0) {
        mbar_arrive_expect_tx(bar, uint32_t(L * 2 * NCP * sizeof(float)));
        for (int b = 0; b < L; b += BOX) tma_load_2d(buf + b * NCP, &map, n0, p * L + b, bar);
      }
      return;
    }
    const uint32_t rb = uint32_t(min(2 * NCP, Nt - n0)) * sizeof(float);
    if (tid == 0) mbar_arrive_expect_tx(bar, rb * L);
    const float *G0 = d.G0 + (size_t)p * L * Nt + n0;
    for (int q = tid; q < L; q += nthr) bulk_g2s(buf + q * NCP, G0 + (size_t)q * Nt, rb, bar);
  };
  float4 *O = reinterpret_cast<float4 *>(buf1 + L * NCP);  // [nY1][NCP] staged (a, b) pairs
  auto compute = [&](int w, float2 *buf) {
    const int p = w / nchunks, n0 = (w - p * nchunks) * 2 * NCP;
    fft_fixed<LGL, -1>(buf, NCP, LGNCP, lgT, tw, tid);
    if (use_omap) {
      if (tid == 0) bulk_wait_read<0>();  // the previous tile's stores have read O
      __syncthreads();
      for (int idx = tid; idx < nY1 * NCP; idx += nthr) {
        const int k = idx & (NCP - 1), jy = idx >> LGNCP;
        const float2 Z = buf[jy * NCP + k];
        const float2 Zm = buf[((L - jy) & (L - 1)) * NCP + k];
        const float sc = 0.5f * __ldg(d.invphy + jy);
        O[idx] = make_float4(sc * (Z.x + Zm.x), sc * (Z.y - Zm.y), sc * (Z.y + Zm.y), -sc * (Z.x - Zm.x));
      }
      fence_proxy_async_smem();  // the writes precede the stores' reads
      __syncthreads();
      if (tid == 0) {
        const int hb = use_omap;
        tma_store_2d(&omap, 2 * n0, p * nY1, O);
        if (hb < nY1) tma_store_2d(&omap, 2 * n0, p * nY1 + nY1 - hb, O + (nY1 - hb) * NCP);
        bulk_commit();
      }
      return;
    }
    float2 *Trow = d.T + (size_t)p * nY1 * Nt;
    for (int idx = tid; idx < nY1 * NCP; idx += nthr) {
      const int k = idx & (NCP - 1), jy = idx >> LGNCP;
      const int n = n0 + 2 * k;
      if (n >= Nt) continue;
      const float2 Z = buf[jy * NCP + k];
      const float2 Zm = buf[((L - jy) & (L - 1)) * NCP + k];
      const float sc = 0.5f * __ldg(d.invphy + jy);
      const float2 a = make_float2(sc * (Z.x + Zm.x), sc * (Z.y - Zm.y));
      const float2 b = make_float2(sc * (Z.y + Zm.y), -sc * (Z.x - Zm.x));
      *reinterpret_cast<float4 *>(Trow + (size_t)jy * Nt + n) = make_float4(a.x, a.y, b.x, b.y);
    }
  };
  tile_pipeline(nwork, buf0, buf1, bars, d.status, issue, compute);
  if (use_omap && tid == 0) bulk_wait<0>();  // every store complete before the block exits
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
  const int Mx = d.Mx, My = d.My, Nt = d.Nt, nY1 = d.nY1;
  const int nchunks = (Nt + 2 * NCP - 1) / (2 * NCP);
  if (tile >= Mx * nchunks) return;
  // chunk fastest: blocks that run together cover contiguous runs of each row
  const int p = tile / nchunks;
  const int n0 = (tile % nchunks) * 2 * NCP;
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
        if (jy == 0 || 2 * jy == My) {  // bins that are their own mirror
          S[jy * NCP + kk] = make_float2(ab.x, ab.z);
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

// Persistent, double-buffered k_rowifft for My = 2^LGL and Nt % 4 == 0 (one
// plan): the T rows of the next tile land in a staging buffer by bulk copies
// while the current spectrum is built, transformed and written.
// With use_map = hb > 0, the staged rows arrive as boxes of the 2-D tensor
// map over T (floats; dims 2 Nt, Mx nY1; box 64 x hb): one box when
// hb = nY1 (<= 256), else two (rows [0, hb) and [nY1 - hb, nY1), the row
// they share written twice with the same values).
// With use_omap, the transformed tile leaves shared memory as boxes of the
// 2-D tensor map omap over G0 (floats; dims Nt, Mx My; box 32 x min(My, 256))
// stored by the TMA engine; the next tile's spectrum is built in the same
// buffer only after the stores have read it.
template <int LGL>
__global__ void __launch_bounds__(PipeTile<LGL>::threads, PipeTile<LGL>::minb) k_rowifft_pipe(const InstDesc *__restrict__ descs, int nwork,
                                                              const __grid_constant__ CUtensorMap map, int use_map,
                                                              const __grid_constant__ CUtensorMap omap, int use_omap) {
  griddep_enter();  // the previous kernel of the stream has completed
  extern __shared__ __align__(128) float4 smem_a128[];  // box destinations 128-byte aligned
  __shared__ __align__(8) uint64_t bars[2];
  constexpr int L = 1 << LGL, NCP = PipeTile<LGL>::nc, LGNCP = PipeTile<LGL>::lgnc;
  const InstDesc &d = descs[0];
  if (!smem_aligned_128(smem_a128, d.status)) return;
  const int Nt = d.Nt, nY1 = d.nY1;
  // staging buffers first
  float2 *st0 = reinterpret_cast<float2 *>(smem_a128);
  float2 *st1 = st0 + ((nY1 * 2 * NCP + 15) & ~15);  // [nY1][2 NCP] staged T rows
  float2 *S = st1 + ((nY1 * 2 * NCP + 15) & ~15);    // [My][NCP] packed spectrum
  const int nchunks = (Nt + 2 * NCP - 1) / (2 * NCP);
  const int tid = threadIdx.x, nthr = blockDim.x, lgT = ilog2_pow2(nthr);
  const float2 *tw = d.tw + d.fMy.tw;
  auto issue = [&](int w, float2 *stg, uint64_t *bar) {
    const int p = w / nchunks, n0 = (w - p * nchunks) * 2 * NCP;
    if (use_map) {
      if (tid == 0) {
        const int hb = use_map, nb = hb < nY1 ? 2 : 1;
        mbar_arrive_expect_tx(bar, uint32_t(nb * hb * 2 * NCP * sizeof(float2)));
        tma_load_2d(stg, &map, 2 * n0, p * nY1, bar);
        if (nb == 2) tma_load_2d(stg + (nY1 - hb) * 2 * NCP, &map, 2 * n0, p * nY1 + nY1 - hb, bar);
      }
      return;
    }
    const uint32_t rb = uint32_t(min(2 * NCP, Nt - n0)) * sizeof(float2);
    if (tid == 0) mbar_arrive_expect_tx(bar, rb * nY1);
    const float2 *Trow = d.T + (size_t)p * nY1 * Nt + n0;
    for (int jy = tid; jy < nY1; jy += nthr) bulk_g2s(stg + jy * 2 * NCP, Trow + (size_t)jy * Nt, rb, bar);
  };
  auto compute = [&](int w, float2 *stg) {
    const int p = w / nchunks, n0 = (w - p * nchunks) * 2 * NCP;
    if (use_omap) {  // the previous tile's stores have read S
      if (tid == 0) bulk_wait_read<0>();
      __syncthreads();
    }
    // bins jy and My - jy from the staged rows (one item reads a sample pair
    // and fills both); the bins nY1 .. My - nY1, which no jy reaches, are zero
    for (int idx = tid; idx < nY1 * NCP; idx += nthr) {
      const int jy = idx >> LGNCP, kk = idx & (NCP - 1);
      const int n = n0 + 2 * kk;
      const float sc = __ldg(d.invphy + jy);
      const float4 ab = *reinterpret_cast<const float4 *>(stg + jy * 2 * NCP + 2 * kk);
      const float2 a = n < Nt ? make_float2(sc * ab.x, sc * ab.y) : make_float2(0.f, 0.f);
      const float2 b = n + 1 < Nt ? make_float2(sc * ab.z, sc * ab.w) : make_float2(0.f, 0.f);
      if (jy == 0 || 2 * jy == L) {  // bins that are their own mirror
        S[jy * NCP + kk] = make_float2(a.x, b.x);
      } else {
        S[jy * NCP + kk] = make_float2(0.5f * (a.x - b.y), 0.5f * (a.y + b.x));
        S[(L - jy) * NCP + kk] = make_float2(0.5f * (a.x + b.y), 0.5f * (b.x - a.y));
      }
    }
    // (with the band, the transform reads those bins as zeros)
    constexpr bool BAND = PipeTile<LGL>::band;
    if (!BAND)
      for (int idx = tid; idx < (L - 2 * nY1 + 1) * (NCP / 2); idx += nthr)
        reinterpret_cast<float4 *>(S + nY1 * NCP)[idx] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    fft_fixed<LGL, +1, 0, BAND>(S, NCP, LGNCP, lgT, tw, tid, 0, nY1, L - nY1 + 1);
    if (use_omap) {
      fence_proxy_async_smem();  // the transform's writes precede the stores' reads
      __syncthreads();
      if (tid == 0) {
        constexpr int OB = L < 256 ? L : 256;
        for (int b = 0; b < L; b += OB) tma_store_2d(&omap, n0, p * L + b, S + b * NCP);
        bulk_commit();
      }
      return;
    }
    float *G0 = d.G0 + (size_t)p * L * Nt + n0;
    const int nv4 = (min(2 * NCP, Nt - n0)) >> 2;
    if (nv4 == NCP / 2) {  // full chunk: index splits by shifts
      for (int idx = tid; idx < L * (NCP / 2); idx += nthr) {
        const int q = idx >> (LGNCP - 1), k2 = idx & (NCP / 2 - 1);
        *reinterpret_cast<float4 *>(G0 + (size_t)q * Nt + 4 * k2) = reinterpret_cast<const float4 *>(S + q * NCP)[k2];
      }
    } else {
      for (int idx = tid; idx < L * nv4; idx += nthr) {
        const int q = idx / nv4, k2 = idx - q * nv4;
        *reinterpret_cast<float4 *>(G0 + (size_t)q * Nt + 4 * k2) = reinterpret_cast<const float4 *>(S + q * NCP)[k2];
      }
    }
  };
  tile_pipeline(nwork, st0, st1, bars, d.status, issue, compute);
  if (use_omap && tid == 0) bulk_wait<0>();  // every store complete before the block exits
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
  const int c = tile % nchunks;
  const int tx = (tile / nchunks) % ntx;
  const int ty = tile / (nchunks * ntx);
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
  // G0b tile with halo, 128-byte rows of 32 samples: one bulk copy (TMA
  // engine) per cell when rows are 16-byte aligned, else plain loads
  const float *G0 = d.G0;
  const bool vec4 = (Nt & 3) == 0;
  __shared__ __align__(8) uint64_t bar;
  if (vec4) {
    if (tid == 0) {
      mbar_init(&bar, 1);
      mbar_fence_init();
    }
    __syncthreads();
    const uint32_t rb = uint32_t(min(NC, Nt - n0)) * sizeof(float);
    if (tid == 0) mbar_arrive_expect_tx(&bar, rb * HX * HY);
    for (int cell = tid; cell < HX * HY; cell += nthr) {
      const int hr = cell / HY, hc = cell - hr * HY;
      const int p = wrap(p0 - W / 2 + 1 + hr, Mx), q = wrap(q0 - W / 2 + 1 + hc, My);
      bulk_g2s(Gs + cell * NC, G0 + ((size_t)p * My + q) * Nt + n0, rb, &bar);
    }
    if (__syncthreads_or(!mbar_wait(&bar, 0))) {
      if (tid == 0) atomicOr(d.status, kStatusWaitTimeout);
      mbar_wait(&bar, 0);  // one more bounded wait for the copies in flight
      return;
    }
  } else {
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
  }
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
      // samples past Nt hold stale tile values: keep them out of the sums
      const float gv = n < Nt ? __ldg(io.g_in + (size_t)m * Nt + n) : 0.f;
      float px = n < Nt ? ax * gv : 0.f, py = n < Nt ? ay * gv : 0.f;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        px += __shfl_xor_sync(0xffffffffu, px, off);
        py += __shfl_xor_sync(0xffffffffu, py, off);
      }
      if (lane == 0) d.grad_part[(size_t)c * M + i] = make_float2(px, py);
    }
  }
}

// The same interpolation as a persistent kernel for single-plan launches with
// Nt % 4 == 0: tiles w = blockIdx.x, blockIdx.x + gridDim.x, ... through two
// shared-memory buffers, the copies of tile w + 1 in flight while tile w is
// computed.  A tile whose halo lies inside the grid arrives as one 3-D box of
// the tensor map g0map (dims Nt, My, Mx; box 32 x HY x HX) when use_map is
// set; tiles at the periodic edges take one bulk copy per cell.  With the
// grid, the packs (taps, column, caller index) of the tile's first SMAX
// sensors arrive by bulk copies of the rows' contiguous sorted ranges, so
// the interpolation reads only shared memory.  A group of 8 lanes takes one
// sensor at a time, lane l8 the 4 samples n0 + 4 l8 .. + 3 (16-byte shared
// loads, 128-byte output rows): a warp interpolates 4 sensors at once.
template <int W, int TY, bool GRAD, int NSTAGE>
struct InterpPipe {
  static constexpr int TX = 8, NC = 32;
  static constexpr int HX = TX + W - 1, HY = TY + W - 1, CELLS = HX * HY;
  static constexpr int SMAX = TX * TY;  // packed sensors per tile
  static constexpr int PW = ipack_words(W), PD = GRAD ? ipackd_words(W) : 0;
  // floats per buffer, rounded to 128 bytes
  static constexpr int BUF = ((CELLS * NC + SMAX * (PW + PD)) + 31) / 32 * 32;
  static constexpr int NS = NSTAGE;      // pipeline stages (buffers)
  static constexpr int THREADS = PA_INTERP_THREADS;
  static constexpr size_t smem = size_t(NS * BUF) * sizeof(float);
};

template <int W, int TY, bool GRAD, int NS>
__global__ void __launch_bounds__(InterpPipe<W, TY, GRAD, NS>::THREADS, PA_INTERP_MINB) k_interp_pipe(const InstDesc *__restrict__ descs, IoPtrs io,
                                                                int nwork, const __grid_constant__ CUtensorMap g0map,
                                                                int use_map) {
  griddep_enter();  // the previous kernel of the stream has completed
  using S = InterpPipe<W, TY, GRAD, NS>;
  constexpr int TX = S::TX, HX = S::HX, HY = S::HY, NC = S::NC, CELLS = S::CELLS, SMAX = S::SMAX;
  constexpr int PW = S::PW, PD = S::PD;
  extern __shared__ __align__(128) float4 smem_a128[];  // box destinations 128-byte aligned
  float *base = reinterpret_cast<float *>(smem_a128);
  float2 *buf0 = reinterpret_cast<float2 *>(base);
  __shared__ __align__(8) uint64_t bars[S::NS];
  __shared__ int rlo[S::NS][TX], rpre[S::NS][TX + 1];
  const InstDesc &d = descs[0];
  if (!smem_aligned_128(smem_a128, d.status)) return;
  const int Mx = d.Mx, My = d.My, Nt = d.Nt, M = d.M;
  const int ntx = (Mx + TX - 1) / TX;
  const int nchunks = (Nt + NC - 1) / NC;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, l8 = tid & 7, grp = tid >> 3, ngrp = nthr >> 3;
  const unsigned gmask = 0xffu << (lane & 24);
  const float *G0 = d.G0;
  auto decode = [&](int w, int &p0, int &q0, int &n0) {
    p0 = ((w / nchunks) % ntx) * TX;
    q0 = (w / (nchunks * ntx)) * TY;
    n0 = (w % nchunks) * NC;
  };
  // sorted range of row `lane` of tile w (warp 0, lanes < TX); the ranges of
  // the tile issued next are loaded one issue ahead, so their latency hides
  // behind a compute phase
  auto row_range = [&](int w, int &lo, int &hi) {
    lo = hi = 0;
    if (w < nwork && lane < TX) {
      int p0, q0, n0;
      decode(w, p0, q0, n0);
      if (p0 + lane < Mx) {
        const size_t row = (size_t)(p0 + lane) * My;
        lo = __ldg(d.cell_start + row + q0);
        hi = __ldg(d.cell_start + row + min(q0 + TY, My));
      }
    }
  };
  int pf_w = -1, pf_lo = 0, pf_hi = 0;
  auto issue = [&](int w, float2 *buf, uint64_t *bar) {
    int p0, q0, n0;
    decode(w, p0, q0, n0);
    const int par = int((reinterpret_cast<float *>(buf) - base) / S::BUF);
    float *Gs = reinterpret_cast<float *>(buf);
    float *packs = Gs + CELLS * NC, *packd = packs + SMAX * PW;
    const int ps = p0 - W / 2 + 1, qs = q0 - W / 2 + 1;
    const bool box = use_map && ps >= 0 && ps + HX <= Mx && qs >= 0 && qs + HY <= My;
    // test hook: this item's byte count is posted and none of its copies is
    // issued, so its waits run out (nothing is left in flight)
    const bool drop = d.test_fault == w + 1;
    uint32_t pack_bytes = 0;
    if (tid < 32) {
      // rows r < TX of the tile: sorted ranges, their prefix, and the packs
      int lo, hi;
      if (pf_w == w) {
        lo = pf_lo;
        hi = pf_hi;
      } else {
        row_range(w, lo, hi);
      }
      pf_w = w + gridDim.x;
      row_range(pf_w, pf_lo, pf_hi);
      const int cnt = hi - lo;
      int inc = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += v;
      }
      const int pre = inc - cnt, total = __shfl_sync(0xffffffffu, inc, TX - 1);
      if (lane < TX) {
        rlo[par][lane] = lo;
        rpre[par][lane] = pre;
        const int k = min(cnt, SMAX - pre);
        if (k > 0 && !drop) {
          bulk_g2s(packs + pre * PW, d.ipack + (size_t)lo * (PW / 4), uint32_t(k * PW * 4), bar);
          if (GRAD) bulk_g2s(packd + pre * PD, d.ipack_d + (size_t)lo * (PD / 4), uint32_t(k * PD * 4), bar);
        }
      }
      if (lane == 0) rpre[par][TX] = total;
      pack_bytes = uint32_t(min(total, SMAX) * (PW + PD) * 4);
    }
    if (drop) {
      if (tid == 0) mbar_arrive_expect_tx(bar, uint32_t(CELLS * NC * sizeof(float)));
      return;
    }
    if (box) {
      if (tid == 0) {
        mbar_arrive_expect_tx(bar, uint32_t(CELLS * NC * sizeof(float)) + pack_bytes);
        tma_load_3d(Gs, &g0map, n0, qs, ps, bar);
      }
      return;
    }
    const uint32_t rb = uint32_t(min(NC, Nt - n0)) * sizeof(float);
    if (tid == 0) mbar_arrive_expect_tx(bar, rb * CELLS + pack_bytes);
    for (int cell = tid; cell < CELLS; cell += nthr) {
      const int hr = cell / HY, hc = cell - hr * HY;
      const int p = wrap(ps + hr, Mx), q = wrap(qs + hc, My);
      bulk_g2s(Gs + cell * NC, G0 + ((size_t)p * My + q) * Nt + n0, rb, bar);
    }
  };
  auto compute = [&](int w, float2 *buf) {
    int p0, q0, n0;
    decode(w, p0, q0, n0);
    const int par = int((reinterpret_cast<float *>(buf) - base) / S::BUF);
    const float *Gs = reinterpret_cast<const float *>(buf);
    const float *packs = Gs + CELLS * NC, *packd = packs + SMAX * PW;
    const int total = rpre[par][TX];
    const int n = n0 + 4 * l8;
    const int c = n0 / NC;
#pragma unroll 1
    for (int u = grp; u < total; u += ngrp) {
      int r = 0;
      while (r + 1 < TX && rpre[par][r + 1] <= u) ++r;
      const int i = rlo[par][r] + (u - rpre[par][r]);
      float pk[PW], pkd[PD > 0 ? PD : 1];
      // shared-memory packs, or (past SMAX sensors) the global ones: two
      // separate loops keep the shared loads in the shared address space
      auto unpack = [](float *dst, float4 v) {
        dst[0] = v.x;
        dst[1] = v.y;
        dst[2] = v.z;
        dst[3] = v.w;
      };
      if (u < SMAX) {
#pragma unroll
        for (int k = 0; k < PW / 4; ++k) unpack(pk + 4 * k, reinterpret_cast<const float4 *>(packs + u * PW)[k]);
        if (GRAD) {
#pragma unroll
          for (int k = 0; k < PD / 4; ++k) unpack(pkd + 4 * k, reinterpret_cast<const float4 *>(packd + u * PD)[k]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < PW / 4; ++k) unpack(pk + 4 * k, __ldg(d.ipack + (size_t)i * (PW / 4) + k));
        if (GRAD) {
#pragma unroll
          for (int k = 0; k < PD / 4; ++k) unpack(pkd + 4 * k, __ldg(d.ipack_d + (size_t)i * (PD / 4) + k));
        }
      }
      const int hr0 = r, hc0 = __float_as_int(pk[2 * W]) - q0;
      const int m = __float_as_int(pk[2 * W + 1]);
      float4 gv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (GRAD && n < Nt) gv = __ldg(reinterpret_cast<const float4 *>(io.g_in + (size_t)m * Nt + n));
      float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), ax = a0, ay = a0;
#pragma unroll
      for (int rr = 0; rr < W; ++rr) {
        const float4 *row = reinterpret_cast<const float4 *>(Gs + ((size_t)(hr0 + rr) * HY + hc0) * NC) + l8;
        float4 rs = make_float4(0.f, 0.f, 0.f, 0.f), rsy = rs;
#pragma unroll
        for (int t = 0; t < W; ++t) {
          const float4 v = row[t * (NC / 4)];
          const float wy = pk[W + t];
          fma4(wy, v, rs);
          if (GRAD) {
            const float dwy = pkd[W + t];
            rsy.x = fmaf(dwy, v.x, rsy.x);
            rsy.y = fmaf(dwy, v.y, rsy.y);
            rsy.z = fmaf(dwy, v.z, rsy.z);
            rsy.w = fmaf(dwy, v.w, rsy.w);
          }
        }
        const float wx = pk[rr];
        fma4(wx, rs, a0);
        if (GRAD) {
          const float dwx = pkd[rr];
          ax.x = fmaf(dwx, rs.x, ax.x);
          ax.y = fmaf(dwx, rs.y, ax.y);
          ax.z = fmaf(dwx, rs.z, ax.z);
          ax.w = fmaf(dwx, rs.w, ax.w);
          ay.x = fmaf(wx, rsy.x, ay.x);
          ay.y = fmaf(wx, rsy.y, ay.y);
          ay.z = fmaf(wx, rsy.z, ay.z);
          ay.w = fmaf(wx, rsy.w, ay.w);
        }
      }
      // Nt % 4 == 0: the 4 samples of a lane are all below Nt or all past it
      if (io.g_out && n < Nt) *reinterpret_cast<float4 *>(io.g_out + (size_t)m * Nt + n) = a0;
      if (GRAD) {
        float px = 0.f, py = 0.f;
        if (n < Nt) {
          px = ax.x * gv.x + ax.y * gv.y + ax.z * gv.z + ax.w * gv.w;
          py = ay.x * gv.x + ay.y * gv.y + ay.z * gv.z + ay.w * gv.w;
        }
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) {
          px += __shfl_xor_sync(gmask, px, off);
          py += __shfl_xor_sync(gmask, py, off);
        }
        if (l8 == 0) d.grad_part[(size_t)c * M + i] = make_float2(px, py);
      }
    }
  };
  tile_pipeline_n<S::NS>(nwork, buf0, S::BUF / 2, bars, d.status, issue, compute,
                         d.wait_polls > 0 ? d.wait_polls : kMbarPolls);
}

// ipack[i] = (wx[i][0..w), wy[i][0..w), sby[i], perm[i]); ipack_d[i] = (dwx, dwy)
__global__ void k_build_ipack(const InstDesc *__restrict__ dummy, int M, int w, const int *__restrict__ perm,
                              const int *__restrict__ sby, const float *__restrict__ wx, const float *__restrict__ wy,
                              const float *__restrict__ dwx, const float *__restrict__ dwy, float *pk, float *pkd) {
  (void)dummy;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const int PW = ipack_words(w), PD = ipackd_words(w);
  float *o = pk + (size_t)i * PW, *od = pkd + (size_t)i * PD;
  for (int t = 0; t < w; ++t) {
    o[t] = wx[(size_t)i * w + t];
    o[w + t] = wy[(size_t)i * w + t];
    od[t] = dwx[(size_t)i * w + t];
    od[w + t] = dwy[(size_t)i * w + t];
  }
  o[2 * w] = __int_as_float(sby[i]);
  o[2 * w + 1] = __int_as_float(perm[i]);
  for (int k = 2 * w + 2; k < PW; ++k) o[k] = 0.f;
  for (int k = 2 * w; k < PD; ++k) od[k] = 0.f;
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
int spread_spl(const InstDesc &d) { return d.spread_spl; }
int blocks_spread(const InstDesc &d, int spl) {
  constexpr int QC = kThreadsSpread / 32;
  const int ch = 32 * spl;
  return ((d.Mx + kSpreadP - 1) / kSpreadP) * ((d.My + QC - 1) / QC) * ((d.Nt + ch - 1) / ch);
}
constexpr int kRowFftNCP = 16;
int blocks_rowfft(const InstDesc &d) { return d.Mx * ((d.Nt + 2 * kRowFftNCP - 1) / (2 * kRowFftNCP)); }
size_t smem_rowfft(const InstDesc &d) { return (size_t)d.My * kRowFftNCP * sizeof(float2); }
int blocks_colfft(const InstDesc &d) { return d.nY1 * ((d.Nt + kColNC - 1) / kColNC); }
size_t smem_colfft(const InstDesc &d) { return (size_t)d.Mx * kColNC * sizeof(float2); }
constexpr int kRowIfftNCP = 16;
constexpr int kInterpTX = 8;
int interp_ty(const InstDesc &d) { return d.interp_ty; }
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
  if (smem > 40 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

// The staged spread for single-plan launches with 16-byte sample rows (g
// 16-byte aligned, Nt % 4 == 0) whose union lists were built.
template <int S>
static cudaError_t launch_spread_tile(const Launch &L) {
  const InstDesc &h = *L.host;
  const size_t smem = SpreadTile<S>::floats(h.sp_urows, h.sp_emax) * sizeof(float);
  auto kern = k_spread_tile<S>;
  cudaError_t e = set_smem(kern, smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(kern, blocks_spread(h, S), kThreadsSpread, smem, L.stream, L.descs, L.io);
}

cudaError_t launch_spread(const Launch &L, int spl) {
  if (L.host && !L.work && L.host->sp_slot && (L.host->Nt % 4) == 0 &&
      (reinterpret_cast<uintptr_t>(L.io.g_in) & 15u) == 0 && PA_SPREAD_TILE &&
      SpreadTile<8>::floats(L.host->sp_urows, L.host->sp_emax) * sizeof(float) <= smem_optin_limit()) {
    if (spl == 8) return launch_spread_tile<8>(L);
    if (spl == 4) return launch_spread_tile<4>(L);
  }
  if (spl == 8) return launch_pdl(k_spread<8>, L.nblocks, kThreadsSpread, 0, L.stream, L.descs, L.work, L.io, L.io_table);
  if (spl == 4) return launch_pdl(k_spread<4>, L.nblocks, kThreadsSpread, 0, L.stream, L.descs, L.work, L.io, L.io_table);
  return cudaErrorInvalidValue;
}

// The persistent kernels are instantiated for lengths 2^5 .. 2^9 (two tile
// buffers of at most 128 KB).

// Tensor map of the real grid G0 [Mx][My][Nt] (float) with box
// 32 x hy x hx (samples, columns, rows) for the interpolation tiles, through
// the driver's encoder (looked up once).  False (with the map zeroed) if the
// encoder or the layout is not available.
static bool encode_g0_box(const InstDesc &h, int hx, int hy, CUtensorMap *map) {
  std::memset(map, 0, sizeof(*map));
  PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
  if (!encode || (h.Nt % 4) != 0 || hx > 256 || hy > 256 || (reinterpret_cast<uintptr_t>(h.G0) & 15u)) return false;
  const cuuint64_t dims[3] = {cuuint64_t(h.Nt), cuuint64_t(h.My), cuuint64_t(h.Mx)};
  const cuuint64_t strides[2] = {cuuint64_t(h.Nt) * sizeof(float), cuuint64_t(h.My) * h.Nt * sizeof(float)};
  const cuuint32_t box[3] = {32u, cuuint32_t(hy), cuuint32_t(hx)};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, h.G0, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    std::memset(map, 0, sizeof(*map));
    return false;
  }
  return true;
}

cudaError_t launch_rowfft(const Launch &L) {
  if (L.host && !L.work && (L.host->Nt % 4) == 0) {
    const InstDesc &h = *L.host;
    const int lg = pow2_log(h.My), ncp = pipe_nc(lg);
    const int nwork = h.Mx * ((h.Nt + 2 * ncp - 1) / (2 * ncp));
    size_t smem = 2 * size_t(h.My) * ncp * sizeof(float2);
    CUtensorMap map, omap;
    const int use_map = encode_2d(h.G0, uint64_t(h.Nt), uint64_t(h.Mx) * h.My, uint64_t(h.Nt) * sizeof(float),
                                  uint32_t(2 * ncp), uint32_t(h.My < 256 ? h.My : 256), &map) ? 1 : 0;
    // TMA stores of the output from a third buffer of nY1 rows (measured
    // faster at My = 256 and 512 although it lowers the blocks per SM)
    const int hb = h.nY1 <= 256 ? h.nY1 : (h.nY1 + 1) / 2;
    const size_t osmem = size_t(h.nY1) * ncp * sizeof(float4);
    int use_omap = 0;
    if (use_map && PA_ROWFFT_TMA_STORE && h.My >= PA_ROWFFT_STORE_MIN_MY && hb <= 256 && smem + osmem <= smem_optin_limit())
      use_omap = encode_2d(h.T, 2 * uint64_t(h.Nt), uint64_t(h.Mx) * h.nY1, uint64_t(h.Nt) * sizeof(float2),
                           uint32_t(4 * ncp), uint32_t(hb), &omap) ? hb : 0;
    if (use_omap) smem += osmem;
    else std::memset(&omap, 0, sizeof(omap));
    switch (lg) {
#define PA_ROWFFT_CASE(G)                                                                                 \
  case G: {                                                                                               \
    auto kern = k_rowfft_pipe<G>;                                                                         \
    const cudaError_t e = set_smem(kern, smem);                                                           \
    if (e != cudaSuccess) return e;                                                                       \
    const int grid = persistent_grid(kern, PipeTile<G>::threads, smem, nwork);                               \
    return launch_pdl(kern, grid, PipeTile<G>::threads, smem, L.stream, L.descs, nwork, map, use_map, omap,  \
                      use_omap);                                                                          \
  }
      PA_ROWFFT_CASE(5) PA_ROWFFT_CASE(6) PA_ROWFFT_CASE(7) PA_ROWFFT_CASE(8) PA_ROWFFT_CASE(9)
#undef PA_ROWFFT_CASE
      default: break;
    }
  }
  auto kern = k_rowfft<kRowFftNCP>;
  cudaError_t e = set_smem(kern, L.smem);
  if (e != cudaSuccess) return e;
  kern<<<L.nblocks, kThreadsCol, L.smem, L.stream>>>(L.descs, L.work);
  return cudaGetLastError();
}

template <typename K>
static cudaError_t launch_colfft_pipe(K kernel, const Launch &L, int threads, size_t smem, int nwork,
                                      const CUtensorMap &map, int use_map, const CUtensorMap &omap, int use_omap,
                                      const CUtensorMap &omap2) {
  const cudaError_t e = set_smem(kernel, smem);
  if (e != cudaSuccess) return e;
  const int grid = persistent_grid(kernel, threads, smem, nwork);
  return launch_pdl(kernel, grid, threads, smem, L.stream, L.descs, nwork, map, use_map, omap, use_omap, omap2);
}

cudaError_t launch_colfft(const Launch &L, bool adjoint) {
  if (L.host && !L.work && (L.host->Nt % 2) == 0) {
    const InstDesc &h = *L.host;
    const int lg = pow2_log(h.Mx), nc = pipe_nc(lg);
    const int nwork = h.nY1 * ((h.Nt + nc - 1) / nc);
    const size_t smem = 2 * size_t(h.Mx) * nc * sizeof(float2);
    CUtensorMap map;
    int use_map = 0;
    if (!adjoint) {
      use_map = encode_3d(h.T, 2 * uint64_t(h.Nt), uint64_t(h.nY1), uint64_t(h.Mx), uint64_t(h.Nt) * sizeof(float2),
                          uint64_t(h.nY1) * h.Nt * sizeof(float2), uint32_t(2 * nc), 1u,
                          uint32_t(h.Mx < 256 ? h.Mx : 256), &map);
    } else {
      // boxes of hx + kb rows, kb >= 1 the least that puts the second on a
      // 128-byte aligned bin Mx - hx - kb; both fit the Mx bins
      int kb = 1;
      while (kb < 4 && (size_t(h.Mx - h.hx - kb) * nc * sizeof(float2)) % 128 != 0) ++kb;
      if (h.hx + kb <= 256 && 2 * (h.hx + kb) <= h.Mx &&
          (size_t(h.Mx - h.hx - kb) * nc * sizeof(float2)) % 128 == 0 &&
          encode_3d(h.G1, 2 * uint64_t(h.Nt), uint64_t(h.nY1), uint64_t(h.nX1), uint64_t(h.Nt) * sizeof(float2),
                    uint64_t(h.nY1) * h.Nt * sizeof(float2), uint32_t(2 * nc), 1u, uint32_t(h.hx + kb), &map))
        use_map = kb;
    }
    if (!use_map) {
      std::memset(&map, 0, sizeof(map));
    }
    // outputs by TMA stores (issued by the thread that issues the loads, so
    // only with the load map): the adjoint's T through the forward's input
    // map, the forward's G1 through two maps of box heights hx + 1 and hx
    CUtensorMap omap, omap2;
    std::memset(&omap2, 0, sizeof(omap2));
    int use_omap = 0;
    if (use_map && PA_COLFFT_TMA_STORE) {
      if (adjoint) {
        use_omap = encode_3d(h.T, 2 * uint64_t(h.Nt), uint64_t(h.nY1), uint64_t(h.Mx), uint64_t(h.Nt) * sizeof(float2),
                             uint64_t(h.nY1) * h.Nt * sizeof(float2), uint32_t(2 * nc), 1u,
                             uint32_t(h.Mx < 256 ? h.Mx : 256), &omap) ? 1 : 0;
      } else if (h.hx >= 1 && h.hx + 1 <= 256 && 2 * h.hx + 1 <= h.Mx &&
                 (size_t(h.Mx - h.hx) * nc * sizeof(float2)) % 128 == 0) {
        // (the second box leaves from bin Mx - hx, which must be 128-byte aligned)
        use_omap = encode_3d(h.G1, 2 * uint64_t(h.Nt), uint64_t(h.nY1), uint64_t(h.nX1),
                             uint64_t(h.Nt) * sizeof(float2), uint64_t(h.nY1) * h.Nt * sizeof(float2),
                             uint32_t(2 * nc), 1u, uint32_t(h.hx + 1), &omap) &&
                   encode_3d(h.G1, 2 * uint64_t(h.Nt), uint64_t(h.nY1), uint64_t(h.nX1),
                             uint64_t(h.Nt) * sizeof(float2), uint64_t(h.nY1) * h.Nt * sizeof(float2),
                             uint32_t(2 * nc), 1u, uint32_t(h.hx), &omap2) ? 1 : 0;
      }
    }
    if (!use_omap) std::memset(&omap, 0, sizeof(omap));
    switch (lg) {
#define PA_COLFFT_CASE(G)                                                                                        \
  case G:                                                                                                        \
    return adjoint ? launch_colfft_pipe(k_colfft_pipe<true, G>, L, PipeTile<G>::threads, smem, nwork, map, use_map, \
                                        omap, use_omap, omap2)                                                   \
                   : launch_colfft_pipe(k_colfft_pipe<false, G>, L, PipeTile<G>::threads, smem, nwork, map, use_map, \
                                        omap, use_omap, omap2);
      PA_COLFFT_CASE(5) PA_COLFFT_CASE(6) PA_COLFFT_CASE(7) PA_COLFFT_CASE(8) PA_COLFFT_CASE(9)
#undef PA_COLFFT_CASE
      default: break;
    }
  }
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

// The pipelined kernel with NS stages, if its buffers fit (else false).
template <int W, int TY, bool GRAD, int NS>
static bool launch_interp_pipe(const Launch &L, cudaError_t &err) {
  using IP = InterpPipe<W, TY, GRAD, NS>;
  if (IP::smem > smem_optin_limit()) return false;
  const InstDesc &h = *L.host;
  auto kp = k_interp_pipe<W, TY, GRAD, NS>;
  err = set_smem(kp, IP::smem);
  if (err != cudaSuccess) return true;
  CUtensorMap map;
  const int use_map = encode_g0_box(h, IP::HX, IP::HY, &map) ? 1 : 0;
  const int nwork = blocks_interp(h);
  const int grid = persistent_grid(kp, IP::THREADS, IP::smem, nwork);
  err = launch_pdl(kp, grid, IP::THREADS, IP::smem, L.stream, L.descs, L.io, nwork, map, use_map);
  return true;
}

template <int W, int TY, bool GRAD>
static cudaError_t launch_interp_w(const Launch &L) {
  // single-plan launches with 16-byte sample rows take the pipelined kernel
  // (two stages, two blocks per SM measured fastest; wider windows keep the
  // per-cell kernel: their unrolled tap loops would not stay in registers)
  if constexpr (W <= 8) {
    if (L.host && !L.work && (L.host->Nt % 4) == 0) {
      cudaError_t e = cudaSuccess;
      if (launch_interp_pipe<W, TY, GRAD, 2>(L, e)) return e;
    }
  }
  auto kern = k_interp<W, kInterpTX, TY, GRAD>;
  cudaError_t e = set_smem(kern, L.smem);
  if (e != cudaSuccess) return e;
  kern<<<L.nblocks, kThreadsInterp, L.smem, L.stream>>>(L.descs, L.work, L.io, L.io_table);
  return cudaGetLastError();
}

cudaError_t launch_interp_width(const Launch &L, int width, bool grad, int ty) {
#define PA_INTERP_W(W)                                                                                  \
  case W:                                                                                               \
    if (ty == 32) return grad ? launch_interp_w<W, 32, true>(L) : launch_interp_w<W, 32, false>(L);     \
    if (ty == 16) return grad ? launch_interp_w<W, 16, true>(L) : launch_interp_w<W, 16, false>(L);     \
    if (ty == 8) return grad ? launch_interp_w<W, 8, true>(L) : launch_interp_w<W, 8, false>(L);        \
    return cudaErrorInvalidValue;
  switch (width) {
    PA_INTERP_W(6)
    PA_INTERP_W(8)
    PA_INTERP_W(12)
    PA_INTERP_W(16)
    default: return cudaErrorInvalidValue;
  }
#undef PA_INTERP_W
}

cudaError_t launch_rowifft(const Launch &L) {
  if (L.host && !L.work && (L.host->Nt % 4) == 0) {
    const InstDesc &h = *L.host;
    const int lg = pow2_log(h.My), ncp = pipe_nc(lg);
    const int nwork = h.Mx * ((h.Nt + 2 * ncp - 1) / (2 * ncp));
    const size_t stage = size_t((h.nY1 * 2 * ncp + 15) & ~15);
    const size_t smem = (size_t(h.My) * ncp + 2 * stage) * sizeof(float2);
    CUtensorMap map;
    // the staging rows hold exactly nY1 rows: one box of nY1 rows, or two
    // boxes of ceil(nY1 / 2) rows (boxes are at most 256 high)
    const int hb = h.nY1 <= 256 ? h.nY1 : (h.nY1 + 1) / 2;
    const int use_map = hb <= 256 && encode_2d(h.T, 2 * uint64_t(h.Nt), uint64_t(h.Mx) * h.nY1,
                                               uint64_t(h.Nt) * sizeof(float2), uint32_t(4 * ncp), uint32_t(hb), &map)
                            ? hb : 0;
    CUtensorMap omap;
    const int use_omap = PA_ROWIFFT_TMA_STORE &&
                         encode_2d(h.G0, uint64_t(h.Nt), uint64_t(h.Mx) * h.My, uint64_t(h.Nt) * sizeof(float),
                                   uint32_t(2 * ncp), uint32_t(h.My < 256 ? h.My : 256), &omap) ? 1 : 0;
    switch (lg) {
#define PA_ROWIFFT_CASE(G)                                                                               \
  case G: {                                                                                              \
    auto kern = k_rowifft_pipe<G>;                                                                       \
    const cudaError_t e = set_smem(kern, smem);                                                          \
    if (e != cudaSuccess) return e;                                                                      \
    const int grid = persistent_grid(kern, PipeTile<G>::threads, smem, nwork);                              \
    return launch_pdl(kern, grid, PipeTile<G>::threads, smem, L.stream, L.descs, nwork, map, use_map, omap, \
                      use_omap);                                                                         \
  }
      PA_ROWIFFT_CASE(5) PA_ROWIFFT_CASE(6) PA_ROWIFFT_CASE(7) PA_ROWIFFT_CASE(8) PA_ROWIFFT_CASE(9)
#undef PA_ROWIFFT_CASE
      default: break;
    }
  }
  auto kern = k_rowifft<kRowIfftNCP>;
  cudaError_t e = set_smem(kern, L.smem);
  if (e != cudaSuccess) return e;
  kern<<<L.nblocks, kThreadsCol, L.smem, L.stream>>>(L.descs, L.work);
  return cudaGetLastError();
}

cudaError_t build_interp_pack(const InstDesc &h, cudaStream_t s) {
  if (h.M <= 0) return cudaSuccess;
  k_build_ipack<<<(h.M + 255) / 256, 256, 0, s>>>(nullptr, h.M, h.w, h.perm, h.sby, h.wx, h.wy, h.dwx, h.dwy,
                                                  reinterpret_cast<float *>(const_cast<float4 *>(h.ipack)),
                                                  reinterpret_cast<float *>(const_cast<float4 *>(h.ipack_d)));
  return cudaGetLastError();
}

cudaError_t launch_grad_reduce(const Launch &L, int n_inst) {
  k_grad_reduce<<<L.nblocks, 256, 0, L.stream>>>(L.descs, L.io, L.io_table, n_inst);
  return cudaGetLastError();
}

}  // namespace pa
