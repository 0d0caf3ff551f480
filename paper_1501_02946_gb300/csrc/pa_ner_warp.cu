// pa_ner_warp.cu -- the NER stage (Sec. 3) with one warp per column of the
// half spectrum, for sigma = 2 and power-of-two lengths Nt, Nz in [256, 1024].
//
// The block kernels of pa_ner.cu share every transform among the threads of
// a block (CB columns, block barriers between radix passes, runtime
// lengths).  Here a warp owns a whole column: the transforms are compile-time
// four-step FFTs held in registers (two in-register DFT passes around one
// transpose through shared memory), so a column needs no block barrier, and
// the index arithmetic folds to constants.
//
// The oversampled time transform uses the zero padding of Sec. 3: with
// Mt = 2 Nt and the centred samples x(n') nonzero for n' in [-Nt/2, Nt/2),
//   X(2k)     = sum_n' x(n') exp(-2 pi i n' k / Nt),
//   X(2k + 1) = sum_n' [x(n') exp(-2 pi i n' / Mt)] exp(-2 pi i n' k / Nt),
// two Nt-point transforms of the (cyclically placed) samples instead of one
// Mt-point transform of which half the input is zero.  The even and odd
// halves of the oversampled spectrum stay in two arrays He(k) = X(2k),
// Ho(k) = X(2k + 1), each followed by w/2 wrapped copies so that the w taps
// of a window never need a modulo.  The adjoint is the exact transpose.
#include "pa_ner_common.cuh"

// Resident blocks per SM the register allocation is held to (forward kernels
// with Nt <= 512 and adjoint kernels; larger forward transforms keep their
// registers).
#ifndef PA_NER_FWD_MINB
#define PA_NER_FWD_MINB 4
#endif
// 1: the adjoint's sliding windows add the points they leave without atomics
// where no two lanes can reach the same entry.
#ifndef PA_NER_PLAIN_FLUSH
#define PA_NER_PLAIN_FLUSH 1
#endif
#ifndef PA_NER_ADJ_MINB
#define PA_NER_ADJ_MINB 4
#endif

namespace pa {

namespace {

// Scratch entries of a 2^lg point warp transform: E = 2^lg / 32 rows of 32
// values, padded to a bank-conflict-free stride.
__host__ __device__ constexpr int warp_scratch(int lg) {
  return (32 + ((1 << (lg - 5)) == 8 ? 2 : 1)) * (1 << (lg - 5));
}

// Four-step layout of an N = 32 E point transform held by one warp.
template <int LGN>
struct WShape {
  static constexpr int N = 1 << LGN;
  static constexpr int LGE = LGN - 5;
  static constexpr int E = N / 32;                 // elements per lane
  static constexpr int A = 32 / E;                 // lanes per second-pass row (1, 2 or 4)
  static constexpr int RS = 32 + (E == 8 ? 2 : 1); // scratch row stride (bank-conflict free)
  static constexpr int SCR = RS * E;               // scratch entries
  static_assert(SCR == warp_scratch(LGN), "scratch layout");
};

// y(k) = sum_n x(n) exp(DIR 2 pi i n k / N) by one warp (all 32 lanes call
// it with the same arguments), n = n1 + 32 n2 (lane n1 holds n2 < E) and
// k = k2 + E k1:
//  (1) E-point DFTs over n2 in registers, then the twiddle
//      exp(DIR 2 pi i n1 k2 / N) from the table twT[k2][n1];
//  (2) the 32-point DFTs over n1, after a transpose through scr[k2][n1]:
//      lane k2 + E a takes n1 = a + A b (b < E), an E-point DFT over b, the
//      twiddle exp(DIR 2 pi i a c / 32), and an A-point DFT across its A
//      lanes, keeping output k1 = c + E a.
// ld(n) returns x(n); st(k, y) receives y(k).  Every input is loaded before
// the first scratch write and every scratch read precedes the first store,
// so scr may alias the memory that ld reads and st writes.
template <int LGN, int DIR, typename Ld, typename St>
__device__ __forceinline__ void warp_fft(float2 *scr, const float2 *__restrict__ twT, int lane, Ld ld, St st) {
  using S = WShape<LGN>;
  constexpr int E = S::E, A = S::A, RS = S::RS;
  float2 v[E];
#pragma unroll
  for (int n2 = 0; n2 < E; ++n2) v[n2] = ld(lane + 32 * n2);
  Dft<E, DIR>::run(v);
#pragma unroll
  for (int k2 = 1; k2 < E; ++k2) {
    float2 w = __ldg(twT + k2 * 32 + lane);
    if (DIR > 0) w.y = -w.y;
    v[k2] = cmul(v[k2], w);
  }
  __syncwarp();
#pragma unroll
  for (int k2 = 0; k2 < E; ++k2) scr[k2 * RS + lane] = v[k2];
  __syncwarp();
  const int k2 = lane & (E - 1), a = lane >> S::LGE;
#pragma unroll
  for (int b = 0; b < E; ++b) v[b] = scr[k2 * RS + a + A * b];
  __syncwarp();
  Dft<E, DIR>::run(v);
  if constexpr (A == 2) {
    // lanes k2 (a = 0) and k2 + 16 (a = 1): outputs c and c + 16
#pragma unroll
    for (int c = 0; c < E; ++c) {
      if (a && c > 0) v[c] = cmul(v[c], make_float2(Tw32::c(c), DIR * Tw32::s(c)));
      const float2 o = make_float2(__shfl_xor_sync(0xffffffffu, v[c].x, 16), __shfl_xor_sync(0xffffffffu, v[c].y, 16));
      v[c] = a ? csub(o, v[c]) : cadd(v[c], o);
    }
  } else if constexpr (A == 4) {
    // lanes k2 + 8 a, a < 4: Z(d) = Q0(d mod 2) + exp(DIR 2 pi i d / 4) Q1(d mod 2)
    // with Qa1(e) = T(a1) + (-1)^e T(a1 + 2); lane a keeps d = a
    const bool odd = a & 1, low = a < 2;
#pragma unroll
    for (int c = 0; c < E; ++c) {
      float2 t = v[c];
      if (c > 0) {  // exp(DIR 2 pi i a c / 32): a picks one of three constants
        const float wc = a == 1 ? Tw32::c(c) : (a == 2 ? Tw32::c(2 * c) : Tw32::c(3 * c));
        const float ws = a == 1 ? Tw32::s(c) : (a == 2 ? Tw32::s(2 * c) : Tw32::s(3 * c));
        if (a != 0) t = cmul(t, make_float2(wc, DIR * ws));
      }
      const float2 other = make_float2(__shfl_xor_sync(0xffffffffu, t.x, 16), __shfl_xor_sync(0xffffffffu, t.y, 16));
      const float2 lo = low ? t : other, hi = low ? other : t;
      const float2 q0 = cadd(lo, hi), q1 = csub(lo, hi);
      const float2 mine = odd ? q1 : q0, send = odd ? q0 : q1;
      const float2 recv = make_float2(__shfl_xor_sync(0xffffffffu, send.x, 8), __shfl_xor_sync(0xffffffffu, send.y, 8));
      const float2 Q0 = odd ? recv : mine, Q1 = odd ? mine : recv;
      const float2 r = (a == 0 || a == 2) ? Q1 : mul_i<DIR>(Q1);
      v[c] = a < 2 ? cadd(Q0, r) : csub(Q0, r);
    }
  }
#pragma unroll
  for (int c = 0; c < E; ++c) st(k2 + E * (c + E * a), v[c]);
}

template <int LGT, int W>
struct NerWarpShape {
  static constexpr int Nt = 1 << LGT;
  // half-spectrum array: Nt entries and W/2 wrapped copies, or the scratch
  static constexpr int HH = WShape<LGT>::SCR > Nt + W / 2 ? WShape<LGT>::SCR : Nt + W / 2;
};
template <int LGZ>
struct NerWarpFs {
  static constexpr int FS = WShape<LGZ>::SCR;  // >= Nz
};

// W taps of the oversampled spectrum X at the grid points p0 .. p0 + W - 1
// (p0 in [0, Mt)): p even at He(p / 2), p odd at Ho(p / 2).  Even taps t
// read ba[t / 2], odd taps bb[t / 2].
__device__ __forceinline__ void tap_bases(float2 *He, float2 *Ho, int p0, float2 *&ba, float2 *&bb) {
  const int h = p0 >> 1;
  if (p0 & 1) {
    ba = Ho + h;
    bb = He + h + 1;
  } else {
    ba = He + h;
    bb = Ho + h;
  }
}

template <int W>
__device__ __forceinline__ float2 interp_split(float2 *He, float2 *Ho, ff tau, const InstDesc &d,
                                               const HornerTable &ht) {
  int p0;
  float fr;
  footprint(tau, 2, d.Mt, W / 2, p0, fr);
  float wt[W];
  window_taps<W>(fr, ht, wt);
  float2 *ba, *bb;
  tap_bases(He, Ho, p0, ba, bb);
  float2 acc = make_float2(0.f, 0.f);
#pragma unroll
  for (int t = 0; t < W; ++t) {
    const float2 h = (t & 1) ? bb[t >> 1] : ba[t >> 1];
    acc = __ffma2_rn(make_float2(wt[t], wt[t]), h, acc);
  }
  return cmul(acc, centring_phase(d, tau));
}

// The window sum over the W grid points p0 .. p0 + W - 1 with taps wt[t],
// or (REV) with taps wt[W - 1 - t].
template <int W, bool REV>
__device__ __forceinline__ float2 window_sum(float2 *He, float2 *Ho, int p0, const float (&wt)[W]) {
  float2 *ba, *bb;
  tap_bases(He, Ho, p0, ba, bb);
  float2 acc = make_float2(0.f, 0.f);
#pragma unroll
  for (int t = 0; t < W; ++t) {
    const float2 h = (t & 1) ? bb[t >> 1] : ba[t >> 1];
    const float w = REV ? wt[W - 1 - t] : wt[t];
    acc = __ffma2_rn(make_float2(w, w), h, acc);
  }
  return acc;
}

// The points u = 2 tau and -u share their window taps: with u's footprint
// starting at the (unwrapped) point pu and taps wt[t] = phi(fr + W/2 - 1 - t),
// the footprint of -u starts at -pu - (W - 1) with taps wt[W - 1 - t] (the
// window is even), and the centring phase of -tau is the conjugate of that
// of tau.  pm_interp returns the interpolated values at tau and at -tau.
template <int W>
__device__ __forceinline__ void pm_interp(float2 *He, float2 *Ho, ff tau, const InstDesc &d, const HornerTable &ht,
                                          float2 &vp, float2 &vn) {
  int pu;
  float fr;
  footprint_unwrapped(tau, 2, W / 2, pu, fr);
  float wt[W];
  window_taps<W>(fr, ht, wt);
  const float2 ph = centring_phase(d, tau);
  vp = cmul(window_sum<W, false>(He, Ho, wrap(pu, d.Mt), wt), ph);
  vn = cmul(window_sum<W, true>(He, Ho, wrap(-pu - (W - 1), d.Mt), wt), cconj(ph));
}

template <int W>
__device__ __forceinline__ void spread_split(float2 *He, float2 *Ho, ff tau, float2 v, const InstDesc &d,
                                             const HornerTable &ht) {
  int p0;
  float fr;
  footprint(tau, 2, d.Mt, W / 2, p0, fr);
  float wt[W];
  window_taps<W>(fr, ht, wt);
  const float2 vv = cmul(v, cconj(centring_phase(d, tau)));
  float2 *ba, *bb;
  tap_bases(He, Ho, p0, ba, bb);
#pragma unroll
  for (int t = 0; t < W; ++t) {
    float2 *q = (t & 1) ? bb + (t >> 1) : ba + (t >> 1);
    atomicAdd(&q->x, wt[t] * vv.x);
    atomicAdd(&q->y, wt[t] * vv.y);
  }
}

// Adds v into the half-spectrum entry of grid point pu mod Mt (zeros
// skipped): atomically, or (plain) by a read-modify-write where no other lane
// can add to the same entry at the same time.
__device__ __forceinline__ void flush_point(float2 *He, float2 *Ho, int pu, int Mt, float2 v, bool plain = false) {
  if (v.x == 0.f && v.y == 0.f) return;
  const int p = wrap(pu, Mt);
  float2 *q = ((p & 1) ? Ho : He) + (p >> 1);
  if (plain) {
    *q = cadd(*q, v);
  } else {
    atomicAdd(&q->x, v.x);
    atomicAdd(&q->y, v.y);
  }
}

// Number of lanes i with P[i] <= x, for P[0..31] non-decreasing.
__device__ __forceinline__ int count_le(const int *P, int x) {
  int c = 0;
#pragma unroll
  for (int st = 16; st > 0; st >>= 1)
    if (P[c + st - 1] <= x) c += st;
  if (c < 32 && P[c] <= x) ++c;
  return c;
}

// Adds the warp's last sliding windows into the half spectrum: lane i's
// window acc[t] belongs to the grid point sgn (P[i] + t), t < W, with P
// non-decreasing in i (lanes without a window hold a P above every point).
// Neighbouring lanes' windows overlap, often with equal P where tau varies
// slowly, so instead of one atomic add per lane and point (serialised on the
// shared addresses) each lane parks its window in F[i][t], and the warp then
// takes the points P[0] .. pmax + W - 1 one per lane, summing the windows
// that reach each (lanes count_le(p - W) .. count_le(p) - 1) and adding the
// sum with a plain read-modify-write: every point is written by one lane.
// If the points span more than Mt (two could wrap onto one entry) the sums
// are added atomically.
template <int W>
__device__ __forceinline__ void flush_windows(float2 *He, float2 *Ho, float2 *F, const int *P, const float2 (&acc)[W],
                                              int lane, int pmax, int sgn, int Mt) {
#pragma unroll
  for (int t = 0; t < W; ++t) F[lane * W + t] = acc[t];
  __syncwarp();
  const int p0 = P[0], npts = pmax + W - p0;
  const bool plain = npts <= Mt;
  for (int q0 = 0; q0 < npts; q0 += 32) {
    const int p = p0 + q0 + lane;
    if (q0 + lane < npts) {
      const int hi = count_le(P, p);
      float2 v = make_float2(0.f, 0.f);
      for (int i = count_le(P, p - W); i < hi; ++i) v = cadd(v, F[i * W + (p - P[i])]);
      if (v.x != 0.f || v.y != 0.f) {
        const int e = wrap(sgn * p, Mt);
        float2 *q = ((e & 1) ? Ho : He) + (e >> 1);
        if (plain) {
          *q = cadd(*q, v);
        } else {
          atomicAdd(&q->x, v.x);
          atomicAdd(&q->y, v.y);
        }
      }
    }
  }
  __syncwarp();
}

// Forward NER, warp v of the grid on slot v: the slot's column (both sources
// of a two-source column, which lead at slot v with kind 2) is transformed in
// t, interpolated at tau(j, l), weighted and transformed back over depth.
template <int LGT, int LGZ, int W>
__global__ void __launch_bounds__(128, LGT <= 9 ? PA_NER_FWD_MINB : 1) k_ner_warp(const InstDesc *__restrict__ descs,
                                                  const __grid_constant__ HornerTable ht) {
  griddep_enter();  // the previous kernel of the stream has completed
  extern __shared__ float4 smem_f4[];
  constexpr int Nt = 1 << LGT, Nz = 1 << LGZ;
  constexpr int HH = NerWarpShape<LGT, W>::HH, FS = NerWarpFs<LGZ>::FS;
  const InstDesc &d = descs[0];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int v = blockIdx.x * (blockDim.x >> 5) + wib;
  if (v >= ner_fwd_slots(d)) return;
  const NerSlot lead = fwd_slot(d, v);
  if (lead.kind != 1 && lead.kind != 2) return;
  float2 *He = reinterpret_cast<float2 *>(smem_f4) + (size_t)wib * (2 * HH + FS);
  float2 *Ho = He + HH;
  float2 *Fs = Ho + HH;
  const float2 *twT = d.tw + d.wtw + wtw_T(LGT);
  const float2 *twZ = d.tw + d.wtw + wtw_T(LGZ);
  const float2 *twF = d.tw + d.wtw + wtw_F(LGT + 1);
  const ColInfo ci = col_info(d, lead.jx, lead.iy);
  const int hz = d.hz, nsrc = lead.kind == 2 ? 2 : 1;
  for (int s = 0; s < nsrc; ++s) {
    const NerSlot sl = s == 0 ? lead : fwd_slot(d, v + 1);
    const float2 *src = d.G1 + ((size_t)(sl.src == 0 ? ci.rowA : ci.rowB) * d.nY1 + sl.iy) * Nt;
    const bool cj = sl.src == 0 && ci.ynyq;
    // sample n of the row, deconvolved, at n' = n - Nt/2 (m = n' mod Nt)
    auto xt = [&](int m) {
      const int n = m ^ (Nt / 2);
      float2 x = __ldg(src + n);
      if (cj) x.y = -x.y;
      return cscale(x, __ldg(d.invpht + n));
    };
    warp_fft<LGT, -1>(He, twT, lane, xt, [&](int k, float2 y) { He[k] = y; });
    warp_fft<LGT, -1>(
        Ho, twT, lane, [&](int m) { return cmul(xt(m), __ldg(twF + (m < Nt / 2 ? m : m + Nt))); },
        [&](int k, float2 y) { Ho[k] = y; });
    __syncwarp();
    if (lane < W / 2) {
      He[Nt + lane] = He[lane];
      Ho[Nt + lane] = Ho[lane];
    }
    __syncwarp();
    const bool nyq = sl.kind >= 2;
    const ff tb = tau_base(d, ci.jx, ci.jy);
    // depths l and -l (l = 1 .. hz - 1) share tau, the weight, the window
    // taps and the centring phase; l = 0 and the unpaired l = -hz (Nz is even)
    // are taken alone
    auto put = [&](int z, float2 F) { Fs[z] = s == 0 ? F : cadd(Fs[z], F); };
#pragma unroll 1
    for (int l = 1 + lane; l < hz; l += 32) {
      const ff tau = tau_at(d, tb, l);
      const float wgt = weight_of(d, tau, l) * d.scale * (nyq ? 0.5f : 1.f);
      float2 vp, vn;
      pm_interp<W>(He, Ho, tau, d, ht, vp, vn);
      put(l, cscale(vp, wgt));
      put(Nz - l, cscale(vn, wgt));
    }
    if (lane == 0) {
      float2 F = make_float2(0.f, 0.f);
      if (ci.jx == 0 && ci.jy == 0) {
        const ff tau = tau_at(d, tb, 0);
        F = cscale(interp_split<W>(He, Ho, tau, d, ht), weight_of(d, tau, 0) * d.scale * (nyq ? 0.5f : 1.f));
      }
      put(0, F);
    } else if (lane == 1) {
      const int l = -hz;
      const ff tau = tau_at(d, tb, l);
      const float wgt = weight_of(d, tau, l) * d.scale;
      float2 val;
      if (nyq) {
        val = interp_split<W>(He, Ho, sl.src == 1 ? ff_neg(tau) : tau, d, ht);
      } else {
        float2 vp, vn;
        pm_interp<W>(He, Ho, tau, d, ht, vp, vn);
        val = cadd(vp, vn);
      }
      put(hz, cscale(val, 0.5f * wgt));
    }
    __syncwarp();
  }
  float2 *dst = d.Fz + ((size_t)(lead.jx + d.hx) * d.nY1 + lead.iy) * Nz;
  warp_fft<LGZ, +1>(Fs, twZ, lane, [&](int z) { return Fs[z]; }, [&](int k, float2 y) { dst[k] = y; });
}

// Adjoint NER: depth DFT of the cotangent column, transposed weight and
// window (spread into He/Ho), the two inverse Nt-point transforms, their
// combination into the Nt centred samples, 1/phihat, into the G1 row of the
// slot (summed over a two-source group).
template <int LGT, int LGZ, int W>
__global__ void __launch_bounds__(128, PA_NER_ADJ_MINB) k_ner_warp_adj(const InstDesc *__restrict__ descs,
                                                      const __grid_constant__ HornerTable ht) {
  griddep_enter();  // the previous kernel of the stream has completed
  extern __shared__ float4 smem_f4[];
  constexpr int Nt = 1 << LGT, Nz = 1 << LGZ;
  constexpr int HH = NerWarpShape<LGT, W>::HH, FS = NerWarpFs<LGZ>::FS;
  const InstDesc &d = descs[0];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int v = blockIdx.x * (blockDim.x >> 5) + wib;
  if (v >= ner_adj_slots(d)) return;
  const NerSlot lead = adj_slot(d, v);
  if (lead.kind != 1 && lead.kind != 2) return;
  float2 *He = reinterpret_cast<float2 *>(smem_f4) + (size_t)wib * (2 * HH + FS);
  float2 *Ho = He + HH;
  float2 *Fs = Ho + HH;
  static_assert(FS >= 32 * W, "window park in the depth scratch");
  __shared__ int s_last[4][32];  // last window start of each lane (<= 4 warps per block)
  int *P = s_last[wib];
  const float2 *twT = d.tw + d.wtw + wtw_T(LGT);
  const float2 *twZ = d.tw + d.wtw + wtw_T(LGZ);
  const float2 *twF = d.tw + d.wtw + wtw_F(LGT + 1);
  const int hz = d.hz, hx = d.hx, nY1 = d.nY1, nsrc = lead.kind == 2 ? 2 : 1;
  const ColInfo cl = col_info(d, lead.jx, lead.iy);
  float2 *dst = d.G1 + ((size_t)(lead.src == 0 ? cl.rowA : cl.rowB) * nY1 + lead.iy) * Nt;
  for (int s = 0; s < nsrc; ++s) {
    const NerSlot sl = s == 0 ? lead : adj_slot(d, v + 1);
    const ColInfo ci = col_info(d, sl.jx, sl.iy);
    const float2 *srcz = d.Fz + ((size_t)(sl.jx + hx) * nY1 + sl.iy) * Nz;
    warp_fft<LGZ, -1>(Fs, twZ, lane, [&](int z) { return __ldg(srcz + z); }, [&](int k, float2 y) { Fs[k] = y; });
    for (int i = lane; i < 2 * HH; i += 32) He[i] = make_float2(0.f, 0.f);
    __syncwarp();
    const bool nyq = ci.xnyq || ci.ynyq;
    const ff tb = tau_base(d, ci.jx, ci.jy);
    const float half = nyq ? 0.5f : 1.f;
    // Depths l and -l (l = 1 .. hz - 1) share tau, the weight, the window
    // taps and the centring phase (see pm_interp).  The points u(l) = 2 tau(j, l)
    // increase with l, so the taps of a lane's consecutive l overlap: they
    // accumulate in register windows acc[t] (grid points base + t, for +tau)
    // and accn[t] (points -(base + t), for -tau), which slide forward
    // together (adding the points they leave into shared memory) as the first
    // tap advances.  Only the points a window leaves, and its last W, reach
    // shared memory.  l = 0 and the unpaired l = -hz are spread on their own.
    constexpr int C2 = Nz / 64;  // pairs per lane: l = 1 + lane C2 .. (l < hz)
    // Points a window leaves inside the loop: lane i's are base values in
    // [first base, last base) of its own depths, ranges that do not overlap
    // from lane to lane (u increases with l), so lanes never add to the same
    // +tau point, nor to the same -tau point.  A +tau point and a -tau point
    // (of two lanes) can be one entry only near 0 (the +tau points start at
    // 1 - W/2, the -tau points end at W/2 - 1) or, if the points reach Nt,
    // across the period; elsewhere the loop adds without atomics.
    const bool far_seam = 2.f * tau_at(d, tb, hz - 1).hi + float(W + 2) < float(Nt);
    float2 acc[W], accn[W];
#pragma unroll
    for (int t = 0; t < W; ++t) acc[t] = accn[t] = make_float2(0.f, 0.f);
    int base = 0;
    bool open = false;
#pragma unroll 1
    for (int j = 0; j < C2; ++j) {
      const int l = 1 + lane * C2 + j;
      if (l >= hz) break;
      const ff tau = tau_at(d, tb, l);
      const float wgt = weight_of(d, tau, l) * d.scale * half;
      int pu;
      float fr;
      footprint_unwrapped(tau, 2, W / 2, pu, fr);
      float wt[W];
      window_taps<W>(fr, ht, wt);
      const float2 ph = centring_phase(d, tau);
      const float2 vp = cmul(cscale(Fs[l], wgt), cconj(ph));
      const float2 vn = cmul(cscale(Fs[Nz - l], wgt), ph);
      if (!open) {
        base = pu;
        open = true;
      }
      int adv = pu - base;
      if (adv < 0 || adv >= W) {
        const bool plain = PA_NER_PLAIN_FLUSH && far_seam && base > W;
#pragma unroll
        for (int t = 0; t < W; ++t) {
          flush_point(He, Ho, base + t, 2 * Nt, acc[t], plain);
          flush_point(He, Ho, -(base + t), 2 * Nt, accn[t], plain);
          acc[t] = accn[t] = make_float2(0.f, 0.f);
        }
        base = pu;
      } else {
        for (; adv > 0; --adv) {
          const bool plain = PA_NER_PLAIN_FLUSH && far_seam && base > W;
          flush_point(He, Ho, base, 2 * Nt, acc[0], plain);
          flush_point(He, Ho, -base, 2 * Nt, accn[0], plain);
#pragma unroll
          for (int t = 0; t + 1 < W; ++t) {
            acc[t] = acc[t + 1];
            accn[t] = accn[t + 1];
          }
          acc[W - 1] = accn[W - 1] = make_float2(0.f, 0.f);
          ++base;
        }
      }
#pragma unroll
      for (int t = 0; t < W; ++t) {
        acc[t] = __ffma2_rn(make_float2(wt[t], wt[t]), vp, acc[t]);
        accn[t] = __ffma2_rn(make_float2(wt[t], wt[t]), vn, accn[t]);
      }
    }
    // the last windows (points base + t and -(base + t)); base does not
    // decrease from lane to lane, and the lanes without any depth are last
    const float2 fs1 = Fs[lane == 0 ? 0 : hz];  // read before Fs takes the windows
    P[lane] = open ? base : (1 << 29);
    const int pmax = __reduce_max_sync(0xffffffffu, open ? base : -(1 << 29));
    __syncwarp();  // every lane's loop (its reads of Fs and its flushes) is done
    flush_windows<W>(He, Ho, Fs, P, acc, lane, pmax, 1, 2 * Nt);
    flush_windows<W>(He, Ho, Fs, P, accn, lane, pmax, -1, 2 * Nt);
    if (lane == 0 && ci.jx == 0 && ci.jy == 0) {  // l = 0 (W(j != 0, 0) = 0)
      const ff tau = tau_at(d, tb, 0);
      spread_split<W>(He, Ho, tau, cscale(fs1, weight_of(d, tau, 0) * d.scale * half), d, ht);
    } else if (lane == 1) {  // the depth Nyquist l = -hz also reaches -tau
      const int l = -hz;
      const ff tau = tau_at(d, tb, l);
      const float2 hv = cscale(fs1, 0.5f * weight_of(d, tau, l) * d.scale);
      if (!nyq) {
        spread_split<W>(He, Ho, tau, hv, d, ht);
        spread_split<W>(He, Ho, ff_neg(tau), hv, d, ht);
      } else {
        spread_split<W>(He, Ho, sl.src == 1 ? ff_neg(tau) : tau, hv, d, ht);
      }
    }
    __syncwarp();
    if (lane < W / 2) {
      He[lane] = cadd(He[lane], He[Nt + lane]);
      Ho[lane] = cadd(Ho[lane], Ho[Nt + lane]);
    }
    __syncwarp();
    warp_fft<LGT, +1>(Ho, twT, lane, [&](int m) { return Ho[m]; }, [&](int k, float2 y) { Ho[k] = y; });
    __syncwarp();
    warp_fft<LGT, +1>(He, twT, lane, [&](int m) { return He[m]; }, [&](int k, float2 y) { He[k] = y; });
    __syncwarp();
    // y(n') = Ae(m) + exp(2 pi i n' / Mt) Ao(m) at n' = n - Nt/2, m = n' mod Nt
    const bool cj = sl.src == 0 && ci.ynyq;
#pragma unroll 4
    for (int n = lane; n < Nt; n += 32) {
      const int m = n ^ (Nt / 2);
      float2 w = __ldg(twF + (m < Nt / 2 ? m : m + Nt));
      w.y = -w.y;
      float2 y = cscale(cadd(He[m], cmul(w, Ho[m])), __ldg(d.invpht + n));
      if (cj) y.y = -y.y;
      dst[n] = s == 0 ? y : cadd(dst[n], y);
    }
    __syncwarp();
  }
  if (lead.zero_row0) {
    float2 *z0 = d.G1 + (size_t)lead.iy * Nt;
    for (int n = lane; n < Nt; n += 32) z0[n] = make_float2(0.f, 0.f);
  }
}

// Shared memory of one warp: He and Ho (Nt + W/2 entries each, or the
// scratch of an Nt-point transform), then Fs (the scratch of an Nz-point
// transform, >= Nz entries).
size_t smem_per_warp(const InstDesc &d) {
  const int scr_t = warp_scratch(pow2_log(d.Nt));
  const int hh = scr_t > d.Nt + d.w / 2 ? scr_t : d.Nt + d.w / 2;
  return size_t(2 * hh + warp_scratch(pow2_log(d.Nz))) * sizeof(float2);
}

template <typename K>
cudaError_t launch_warp_kernel(K kernel, const Launch &L, const InstDesc &h, int nslots, const HornerTable &ht) {
  const int nw = ner_warp_block_warps(h);
  const size_t smem = smem_ner_warp(h);
  if (smem > 40 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  const int nblocks = (nslots + nw - 1) / nw;
  return launch_pdl(kernel, nblocks, nw * 32, smem, L.stream, L.descs, ht);
}

template <int LGT, int LGZ>
cudaError_t launch_tz(const Launch &L, const InstDesc &h, const HornerTable &ht, int which) {
  if (which == 1) return launch_warp_kernel(k_ner_warp_adj<LGT, LGZ, 8>, L, h, ner_adj_slots(h), ht);
  return launch_warp_kernel(k_ner_warp<LGT, LGZ, 8>, L, h, ner_fwd_slots(h), ht);
}

template <int LGT>
cudaError_t launch_t(const Launch &L, const InstDesc &h, const HornerTable &ht, int which) {
  switch (pow2_log(h.Nz)) {
    case 8: return launch_tz<LGT, 8>(L, h, ht, which);
    case 9: return launch_tz<LGT, 9>(L, h, ht, which);
    case 10: return launch_tz<LGT, 10>(L, h, ht, which);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool ner_warp_eligible(const InstDesc &d) {
  const int lt = pow2_log(d.Nt), lz = pow2_log(d.Nz);
  return d.sigma == 2 && d.w == 8 && lt >= 8 && lt <= 10 && lz >= 8 && lz <= 10 && d.Mt == 2 * d.Nt;
}

size_t smem_ner_warp(const InstDesc &d) { return size_t(ner_warp_block_warps(d)) * smem_per_warp(d); }

int ner_warp_block_warps(const InstDesc &d) { return smem_per_warp(d) <= 12 * 1024 ? 4 : 2; }

cudaError_t launch_ner_warp(const Launch &L, const HornerTable &ht, int which) {
  if (!L.host || !ner_warp_eligible(*L.host)) return cudaErrorInvalidValue;
  const InstDesc &h = *L.host;
  switch (pow2_log(h.Nt)) {
    case 8: return launch_t<8>(L, h, ht, which);
    case 9: return launch_t<9>(L, h, ht, which);
    case 10: return launch_t<10>(L, h, ht, which);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pa
