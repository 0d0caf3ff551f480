// pa_ner.cu -- NER-NUFFT stage (the temporal type-2 NUFFT of Sec. 3), the
// weight W(j, l) of the exact reconstruction formula and the inverse DFT over
// depth, on sm_103a.
//
// A block owns CB columns j = (jx, jy) of the half spectrum and transforms
// them together (batched in-place FFTs in shared memory, element n of slot b
// at [prow(n)*CB + b], prow adding a pad row per 16).  Forward, per column:
//   load G1(j, n) / phihat((n - nc)/Mt) at n' = n - nc (the paper's centred
//   theta = 2 pi n / N - pi), zero-pad to Mt = sigma Nt, FFT, evaluate at the
//   nz non-integer frequencies tau(j, l) = omega Nt dt / (2 pi) with w window
//   taps (Horner polynomials, tau in double-float) times the centring phase
//   exp(-2 pi i tau nc / Nt), multiply by (dt/dz) W(j, l), and take the
//   inverse DFT over l, all without leaving shared memory.
// Columns and depths on the unpaired Nyquist index of an even length are
// replaced by the Hermitian part F_sym(k) = (F(k) + conj F(-k mod N)) / 2,
// which makes the half-spectrum real inverse DFT equal to the real part of the
// full inverse DFT; it needs the spectrum at +N/2 as well, which G1 holds.
// Such columns take two passes (one per source); the work items are ordered
// so that one-pass columns fill most blocks.
// The adjoint kernel is the exact transpose (spread <-> interpolate).
#include "pa_device.cuh"

namespace pa {

namespace {

constexpr int kNerMaxCB = 4;  // most columns per block
constexpr int kNerPad = 4;    // one pad row per 16 rows of the [n][CB] buffers
__device__ __forceinline__ int prow(int e) { return pad_row<kNerPad>(e); }


template <int W>
struct HornerDeg {
  static constexpr int v = W <= 6 ? 7 : (W <= 8 ? 8 : (W <= 12 ? 10 : 14));
};

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

// tau(j, l) = sign(l) sqrt(ax jx^2 + ay jy^2 + az l^2) in double-float.
__device__ __forceinline__ ff tau_of(const InstDesc &d, int jx, int jy, int l) {
  const float jx2 = float(jx * jx), jy2 = float(jy * jy), l2 = float(l * l);
  ff t2 = ff_add(ff_add(ff_mul_f({d.ax_hi, d.ax_lo}, jx2), ff_mul_f({d.ay_hi, d.ay_lo}, jy2)),
                 ff_mul_f({d.az_hi, d.az_lo}, l2));
  ff t = ff_sqrt(t2);
  return l < 0 ? ff_neg(t) : t;
}

// W(j, l) = 2 c |kz| / |K| with W(0, 0) = 2c and W(j != 0, 0) = 0.
__device__ __forceinline__ float weight_of(const InstDesc &d, ff tau, int l) {
  if (l == 0) return tau.hi == 0.f ? d.two_c : 0.f;
  return d.two_c * d.sqrt_az * fabsf(float(l)) / fabsf(tau.hi);
}

// exp(-2 pi i tau nc / Nt) with the argument reduced in double-float.
__device__ __forceinline__ float2 centring_phase(const InstDesc &d, ff tau) {
  ff turns = ff_mul(tau, {d.ph_hi, d.ph_lo});
  const float ti = rintf(turns.hi);
  const float tr = (turns.hi - ti) + turns.lo;
  float sn, cs;
  sincospif(-2.f * tr, &sn, &cs);
  return make_float2(cs, sn);
}

// First tap index (mod L) and fraction of the point u = scale * tau.
__device__ __forceinline__ void footprint(ff tau, int scale, int L, int half, int &p0, float &fr) {
  const float uh = tau.hi * float(scale), ul = tau.lo * float(scale);
  float fb = floorf(uh);
  fr = (uh - fb) + ul;
  if (fr < 0.f) {
    fr += 1.f;
    fb -= 1.f;
  } else if (fr >= 1.f) {
    fr -= 1.f;
    fb += 1.f;
  }
  p0 = wrap(int(fb) - half + 1, L);
}

template <int W>
__device__ __forceinline__ void window_taps(float fr, const HornerTable &ht, float *wt) {
  constexpr int D = HornerDeg<W>::v;
  const float s = 2.f * fr - 1.f;
#pragma unroll
  for (int t = 0; t < W; ++t) {
    float a = ht.c[t][D];
#pragma unroll
    for (int k = D - 1; k >= 0; --k) a = fmaf(a, s, ht.c[t][k]);
    wt[t] = a;
  }
}

// H: element k of the transformed column at H[prow(k) * CB] (slot-offset pointer).
template <int W>
__device__ __forceinline__ float2 ner_interp(const float2 *H, int CB, ff tau, const InstDesc &d,
                                             const HornerTable &ht) {
  int p0;
  float fr;
  footprint(tau, d.sigma, d.Mt, W / 2, p0, fr);
  float wt[W];
  window_taps<W>(fr, ht, wt);
  float2 acc = make_float2(0.f, 0.f);
  int idx = p0;
  const int Mt = d.Mt;
#pragma unroll
  for (int t = 0; t < W; ++t) {
    const float2 h = H[prow(idx) * CB];
    acc.x = fmaf(wt[t], h.x, acc.x);
    acc.y = fmaf(wt[t], h.y, acc.y);
    idx = (idx + 1 == Mt) ? 0 : idx + 1;
  }
  return cmul(acc, centring_phase(d, tau));
}

// Transpose of ner_interp: H[p_t] += phi_t conj(phase) v.
template <int W>
__device__ __forceinline__ void ner_spread(float2 *H, int CB, ff tau, float2 v, const InstDesc &d,
                                           const HornerTable &ht) {
  int p0;
  float fr;
  footprint(tau, d.sigma, d.Mt, W / 2, p0, fr);
  float wt[W];
  window_taps<W>(fr, ht, wt);
  const float2 vv = cmul(v, cconj(centring_phase(d, tau)));
  int idx = p0;
  const int Mt = d.Mt;
#pragma unroll
  for (int t = 0; t < W; ++t) {
    atomicAdd(&H[prow(idx) * CB].x, wt[t] * vv.x);
    atomicAdd(&H[prow(idx) * CB].y, wt[t] * vv.y);
    idx = (idx + 1 == Mt) ? 0 : idx + 1;
  }
}

// 4-tap cubic Lagrange interpolation of the uniform Nt-point spectrum at tau
// (the polynomial-interpolation baseline of Sec. 2).
__device__ __forceinline__ float2 cubic_interp(const float2 *H, int CB, ff tau, int Nt) {
  int p0;
  float fr;
  footprint(tau, 1, Nt, 2, p0, fr);  // taps base-1 .. base+2
  const float a = fr + 1.f, b = fr, c = fr - 1.f, e = fr - 2.f;
  const float w0 = -(b * c * e) / 6.f;
  const float w1 = 0.5f * (a * c * e);
  const float w2 = -0.5f * (a * b * e);
  const float w3 = (a * b * c) / 6.f;
  const float wt[4] = {w0, w1, w2, w3};
  float2 acc = make_float2(0.f, 0.f);
  int idx = p0;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    const float2 h = H[prow(idx) * CB];
    acc.x = fmaf(wt[t], h.x, acc.x);
    acc.y = fmaf(wt[t], h.y, acc.y);
    idx = (idx + 1 == Nt) ? 0 : idx + 1;
  }
  return acc;
}

struct ColInfo {
  int jx, jy;
  bool xnyq, ynyq;
  int rowA, rowB;  // G1 rows of the two sources (B = the flipped frequency)
};

__device__ __forceinline__ ColInfo col_info(const InstDesc &d, int jx, int jy) {
  ColInfo c;
  c.jx = jx;
  c.jy = jy;
  c.xnyq = ((d.Nx & 1) == 0) && (jx == -d.hx);
  c.ynyq = ((d.Ny & 1) == 0) && (jy == d.hy);
  c.rowA = (c.ynyq ? -jx : jx) + d.hx;  // conj source when ynyq
  c.rowB = (c.xnyq ? d.hx : jx) + d.hx;
  return c;
}

// Slot of a NER block: one (column, source) transform.  A column on an
// unpaired Nyquist index has two sources (A, B); transforms whose results add
// into one output take two adjacent slots, the first (even) one leading.
struct NerSlot {
  int kind;   // 0 empty, 1 alone, 2 leads a group of two, 3 second of a group
  int jx, iy;
  int src;    // 0: source A, 1: source B
  int zero_row0;  // adjoint: G1 row jx = -hx of the y-Nyquist row is read by no column
};

// Forward slots: the one-source columns, (padding to an even count), then the
// two sources of every Nyquist column (x-Nyquist row ix = 0 for even Nx,
// y-Nyquist row iy = hy for even Ny).
__host__ __device__ __forceinline__ int ner_fwd_slots(const InstDesc &d) {
  const int xe = (d.Nx & 1) == 0, ye = (d.Ny & 1) == 0;
  const int R = (d.Nx - xe) * (d.nY1 - ye);
  return R + (R & 1) + 2 * (xe * d.nY1 + ye * (d.Nx - xe));
}
__device__ __forceinline__ NerSlot fwd_slot(const InstDesc &d, int v) {
  NerSlot sl{};
  const int xe = (d.Nx & 1) == 0, ye = (d.Ny & 1) == 0;
  const int ry = d.nY1 - ye;
  const int R = (d.Nx - xe) * ry;
  if (v < R) {
    sl.kind = 1;
    sl.jx = xe + v / ry - d.hx;
    sl.iy = v % ry;
    return sl;
  }
  const int O1 = R + (R & 1);
  if (v < O1) return sl;
  const int k = v - O1;
  int q = k >> 1;
  sl.src = k & 1;
  if (xe) {
    if (q < d.nY1) {
      sl.kind = 2 + sl.src;
      sl.jx = -d.hx;
      sl.iy = q;
      return sl;
    }
    q -= d.nY1;
  }
  if (ye && q < d.Nx - xe) {
    sl.kind = 2 + sl.src;
    sl.jx = xe + q - d.hx;
    sl.iy = d.hy;
  }
  return sl;
}

// Adjoint slots: the one-source columns, (padding), the two sources of the
// x-Nyquist columns (even Nx, jy < hy; they feed two different G1 rows), then
// for even Ny the y-Nyquist row, whose G1 rows each take two transforms:
// row hx from both sources of jx = 0, row 2hx from both sources of the corner
// jx = -hx (even Nx), and for each g > 0 of a pair {g, -g} row hx - g from
// (g, A) + (-g, B) and row hx + g from (g, B) + (-g, A).
__host__ __device__ __forceinline__ int ner_adj_slots(const InstDesc &d) {
  const int xe = (d.Nx & 1) == 0, ye = (d.Ny & 1) == 0;
  const int ry = d.nY1 - ye;
  const int R = (d.Nx - xe) * ry;
  const int npairs = xe ? d.hx - 1 : d.hx;
  return R + (R & 1) + 2 * xe * ry + ye * (2 + 2 * xe + 4 * (npairs > 0 ? npairs : 0));
}
__device__ __forceinline__ NerSlot adj_slot(const InstDesc &d, int v) {
  NerSlot sl{};
  const int xe = (d.Nx & 1) == 0, ye = (d.Ny & 1) == 0;
  const int ry = d.nY1 - ye, hx = d.hx;
  const int R = (d.Nx - xe) * ry;
  if (v < R) {
    sl.kind = 1;
    sl.jx = xe + v / ry - hx;
    sl.iy = v % ry;
    return sl;
  }
  int k = v - (R + (R & 1));
  if (k < 0) return sl;
  if (xe) {
    if (k < 2 * ry) {
      sl.kind = 1;
      sl.jx = -hx;
      sl.iy = k >> 1;
      sl.src = k & 1;
      return sl;
    }
    k -= 2 * ry;
  }
  if (!ye) return sl;
  sl.iy = d.hy;
  if (k < 2) {
    sl.kind = 2 + k;
    sl.jx = 0;
    sl.src = k;
    return sl;
  }
  k -= 2;
  if (xe) {
    if (k < 2) {
      sl.kind = 2 + k;
      sl.jx = -hx;
      sl.src = k;
      sl.zero_row0 = k == 0;
      return sl;
    }
    k -= 2;
  }
  const int npairs = xe ? hx - 1 : hx;
  const int p = k >> 2, r = k & 3;
  if (p >= npairs) return NerSlot{};
  const int g = 1 + p;
  sl.kind = 2 + (r & 1);
  sl.jx = (r == 0 || r == 2) ? g : -g;
  sl.src = (r == 0 || r == 3) ? 0 : 1;
  return sl;
}

// Forward NER: slot b of the block transforms slot tile*CB + b.
template <int W, bool CUBIC>
__global__ void __launch_bounds__(256, 2) k_ner(const InstDesc *__restrict__ descs,
                                                const int2 *__restrict__ work,
                                                const __grid_constant__ HornerTable ht) {
  extern __shared__ float4 smem_f4[];
  __shared__ NerSlot slots[kNerMaxCB];
  int inst, tile;
  block_work(work, inst, tile);
  const InstDesc &d = descs[inst];
  const int CB = d.ner_cb;
  const int Nt = d.Nt, Mt = d.Mt, Nz = d.Nz, nY1 = d.nY1, nc = d.nc, hz = d.hz, hx = d.hx;
  const int nslots = ner_fwd_slots(d);
  if (tile * CB >= nslots) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int L = CUBIC ? Nt : Mt;
  float2 *H = reinterpret_cast<float2 *>(smem_f4);     // [prow(L)][CB]
  float2 *Fs = H + (size_t)padded_rows<kNerPad>(Mt) * CB;  // [prow(Nz)][CB]
  if (tid < CB) {
    const int v = tile * CB + tid;
    slots[tid] = v < nslots ? fwd_slot(d, v) : NerSlot{};
  }
  __syncthreads();
  // slot b's source row, at n' = n - nc (mod Mt) after 1/phihat; an empty
  // slot keeps stale values (transformed, never stored).  All slots' rows
  // are read in one loop, so their loads are in flight together.
  {
    const float2 *src[kNerMaxCB];
    bool cj[kNerMaxCB];
#pragma unroll
    for (int b = 0; b < kNerMaxCB; ++b) {
      src[b] = nullptr;
      cj[b] = false;
      if (b < CB && slots[b].kind != 0) {
        const NerSlot sl = slots[b];
        const ColInfo ci = col_info(d, sl.jx, sl.iy);
        src[b] = d.G1 + ((size_t)(sl.src == 0 ? ci.rowA : ci.rowB) * nY1 + sl.iy) * Nt;
        cj[b] = sl.src == 0 && ci.ynyq;
      }
    }
#pragma unroll 2
    for (int n = tid; n < Nt; n += nthr) {
      float2 a[kNerMaxCB];
#pragma unroll
      for (int b = 0; b < kNerMaxCB; ++b)
        if (src[b]) a[b] = src[b][n];
      const float sc = CUBIC ? 1.f : __ldg(d.invpht + n);
      const int r = prow(CUBIC ? n : (n < nc ? n - nc + Mt : n - nc));
#pragma unroll
      for (int b = 0; b < kNerMaxCB; ++b)
        if (src[b]) {
          float2 v = a[b];
          if (cj[b]) v.y = -v.y;
          H[r * CB + b] = cscale(v, sc);
        }
    }
    if (!CUBIC)
      for (int u = tid; u < Mt - Nt; u += nthr)
#pragma unroll
        for (int b = 0; b < kNerMaxCB; ++b)
          if (b < CB) H[prow(Nt - nc + u) * CB + b] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  if (CUBIC) {
    fft_smem<-1, kNerPad>(H, CB, CB, d.fNt, d.tw, tid, nthr);
  } else {
    fft_smem<-1, kNerPad>(H, CB, CB, d.fMt, d.tw, tid, nthr);
  }
  const int lgcb = ilog2_pow2(CB);
#pragma unroll 1
  for (int idx = tid; idx < Nz * CB; idx += nthr) {
    const int il = idx >> lgcb, b = idx & (CB - 1);
    const NerSlot sl = slots[b];
    if (sl.kind == 0) continue;
    const ColInfo ci = col_info(d, sl.jx, sl.iy);
    const bool nyq = sl.kind >= 2;
    const int l = il - hz;
    float2 F = make_float2(0.f, 0.f);
    if (!(l == 0 && (ci.jx != 0 || ci.jy != 0))) {
      const ff tau = tau_of(d, ci.jx, ci.jy, l);
      const float wgt = weight_of(d, tau, l) * d.scale;
      const bool lnyq = ((Nz & 1) == 0) && (l == -hz);
      // the second evaluation point: -tau on the depth Nyquist (one source),
      // or -tau for the B source of a Nyquist column there
      const bool two = !nyq && lnyq;
      const ff tp = (nyq && sl.src == 1 && lnyq) ? ff_neg(tau) : tau;
      const float2 *Hb = H + b;
      float2 v = CUBIC ? cubic_interp(Hb, CB, tp, Nt) : ner_interp<W>(Hb, CB, tp, d, ht);
      if (two) {
        const ff tb = ff_neg(tau);
        const float2 vb = CUBIC ? cubic_interp(Hb, CB, tb, Nt) : ner_interp<W>(Hb, CB, tb, d, ht);
        v = cadd(v, vb);
      }
      F = cscale(v, (nyq || two) ? 0.5f * wgt : wgt);
    }
    Fs[prow(l < 0 ? l + Nz : l) * CB + b] = F;
  }
  __syncthreads();
  // a two-source column: the leading slot takes the sum
  for (int b = 0; b < CB; b += 2) {
    if (slots[b].kind != 2) continue;
    for (int z = tid; z < Nz; z += nthr) Fs[prow(z) * CB + b] = cadd(Fs[prow(z) * CB + b], Fs[prow(z) * CB + b + 1]);
  }
  __syncthreads();
  fft_smem<+1, kNerPad>(Fs, CB, CB, d.fNz, d.tw, tid, nthr);
  for (int b = 0; b < CB; ++b) {
    const NerSlot sl = slots[b];
    if (sl.kind != 1 && sl.kind != 2) continue;
    float2 *dst = d.Fz + ((size_t)(sl.jx + hx) * nY1 + sl.iy) * Nz;
    for (int z = tid; z < Nz; z += nthr) dst[z] = Fs[prow(z) * CB + b];
  }
}

// Adjoint NER: Fz cotangent -> DFT over depth -> transposed weight and
// window (spread in shared memory) -> inverse FFT -> un-centre, 1/phihat ->
// G1 row (the sum of a group's two slots).
template <int W>
__global__ void __launch_bounds__(256, 2) k_ner_adj(const InstDesc *__restrict__ descs,
                                                    const int2 *__restrict__ work,
                                                    const __grid_constant__ HornerTable ht) {
  extern __shared__ float4 smem_f4[];
  __shared__ NerSlot slots[kNerMaxCB];
  int inst, tile;
  block_work(work, inst, tile);
  const InstDesc &d = descs[inst];
  const int CB = d.ner_cb;
  const int Nt = d.Nt, Mt = d.Mt, Nz = d.Nz, nY1 = d.nY1, nc = d.nc, hz = d.hz, hx = d.hx;
  const int nslots = ner_adj_slots(d);
  if (tile * CB >= nslots) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  float2 *H = reinterpret_cast<float2 *>(smem_f4);     // [prow(Mt)][CB]
  float2 *Fs = H + (size_t)padded_rows<kNerPad>(Mt) * CB;  // [prow(Nz)][CB]
  if (tid < CB) {
    const int v = tile * CB + tid;
    slots[tid] = v < nslots ? adj_slot(d, v) : NerSlot{};
  }
  __syncthreads();
  {
    // all slots' columns in one loop (empty slots keep stale values:
    // transformed, never stored)
    const float2 *src[kNerMaxCB];
#pragma unroll
    for (int b = 0; b < kNerMaxCB; ++b) {
      src[b] = nullptr;
      if (b < CB && slots[b].kind != 0) src[b] = d.Fz + ((size_t)(slots[b].jx + hx) * nY1 + slots[b].iy) * Nz;
    }
#pragma unroll 2
    for (int z = tid; z < Nz; z += nthr) {
      float2 v[kNerMaxCB];
#pragma unroll
      for (int b = 0; b < kNerMaxCB; ++b)
        if (src[b]) v[b] = src[b][z];
#pragma unroll
      for (int b = 0; b < kNerMaxCB; ++b)
        if (src[b]) Fs[prow(z) * CB + b] = v[b];
    }
  }
  for (int idx = tid; idx < padded_rows<kNerPad>(Mt) * CB; idx += nthr) H[idx] = make_float2(0.f, 0.f);
  __syncthreads();
  fft_smem<-1, kNerPad>(Fs, CB, CB, d.fNz, d.tw, tid, nthr);
  // depth samples in the order il = (i * K) mod Nz (K prime to Nz, about
  // Nz / (samples per warp)): the lanes of a warp spread to distant grid
  // points, so their shared-memory atomics do not collide
  const int lgcb = ilog2_pow2(CB);
  const int K = d.ner_lperm;
#pragma unroll 1
  for (int idx = tid; idx < Nz * CB; idx += nthr) {
    const int il = int(((long long)(idx >> lgcb) * K) % Nz), b = idx & (CB - 1);
    const NerSlot sl = slots[b];
    if (sl.kind == 0) continue;
    const ColInfo ci = col_info(d, sl.jx, sl.iy);
    const bool nyq = ci.xnyq || ci.ynyq;
    const int l = il - hz;
    if (l == 0 && (ci.jx != 0 || ci.jy != 0)) continue;
    const ff tau = tau_of(d, ci.jx, ci.jy, l);
    const float wgt = weight_of(d, tau, l) * d.scale;
    const bool lnyq = ((Nz & 1) == 0) && (l == -hz);
    const float2 v = cscale(Fs[prow(l < 0 ? l + Nz : l) * CB + b], wgt);
    float2 *Hb = H + b;
    if (!nyq) {
      if (!lnyq) {
        ner_spread<W>(Hb, CB, tau, v, d, ht);
      } else {
        const float2 hv = cscale(v, 0.5f);
        ner_spread<W>(Hb, CB, tau, hv, d, ht);
        ner_spread<W>(Hb, CB, ff_neg(tau), hv, d, ht);
      }
    } else {
      ner_spread<W>(Hb, CB, (sl.src == 1 && lnyq) ? ff_neg(tau) : tau, cscale(v, 0.5f), d, ht);
    }
  }
  __syncthreads();
  fft_smem<+1, kNerPad>(H, CB, CB, d.fMt, d.tw, tid, nthr);
  for (int b = 0; b < CB; ++b) {
    const NerSlot sl = slots[b];
    if (sl.kind != 1 && sl.kind != 2) continue;
    // the A source of a y-Nyquist column is the conjugate of its G1 row
    const ColInfo ci = col_info(d, sl.jx, sl.iy);
    const bool cj = sl.src == 0 && ci.ynyq;
    bool cj2 = false;
    if (sl.kind == 2) {
      const NerSlot s2 = slots[b + 1];
      cj2 = s2.src == 0 && col_info(d, s2.jx, s2.iy).ynyq;
    }
    const int row = sl.src == 0 ? ci.rowA : ci.rowB;
    float2 *dst = d.G1 + ((size_t)row * nY1 + sl.iy) * Nt;
    float2 *dst0 = sl.zero_row0 ? d.G1 + ((size_t)0 * nY1 + sl.iy) * Nt : nullptr;
    for (int n = tid; n < Nt; n += nthr) {
      const int p = prow(n < nc ? n - nc + Mt : n - nc);
      const float sc = __ldg(d.invpht + n);
      float2 v = cscale(H[p * CB + b], sc);
      if (cj) v.y = -v.y;
      if (sl.kind == 2) {
        float2 v2 = cscale(H[p * CB + b + 1], sc);
        if (cj2) v2.y = -v2.y;
        v = cadd(v, v2);
      }
      dst[n] = v;
      if (dst0) dst0[n] = make_float2(0.f, 0.f);
    }
  }
}

}  // namespace

int blocks_ner(const InstDesc &d) { return (ner_fwd_slots(d) + d.ner_cb - 1) / d.ner_cb; }
int blocks_ner_adj(const InstDesc &d) { return (ner_adj_slots(d) + d.ner_cb - 1) / d.ner_cb; }
size_t smem_ner(const InstDesc &d) {
  return (size_t)(padded_rows<kNerPad>(d.Mt) + padded_rows<kNerPad>(d.Nz)) * d.ner_cb * sizeof(float2);
}

template <typename K>
static cudaError_t set_smem_ner(K kernel, size_t smem) {
  if (smem > 40 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

template <int W>
static cudaError_t launch_ner_w(const Launch &L, const HornerTable &ht, int which) {
  cudaError_t e;
  if (which == 1) {
    e = set_smem_ner(k_ner_adj<W>, L.smem);
    if (e != cudaSuccess) return e;
    k_ner_adj<W><<<L.nblocks, L.threads, L.smem, L.stream>>>(L.descs, L.work, ht);
  } else {
    e = set_smem_ner(k_ner<W, false>, L.smem);
    if (e != cudaSuccess) return e;
    k_ner<W, false><<<L.nblocks, L.threads, L.smem, L.stream>>>(L.descs, L.work, ht);
  }
  return cudaGetLastError();
}

cudaError_t launch_ner(const Launch &L, int width, const HornerTable &ht, bool adjoint) {
  return launch_ner_stage(L, width, ht, adjoint ? 1 : 0);
}

cudaError_t launch_ner_stage(const Launch &L, int width, const HornerTable &ht, int which) {
  switch (width) {
    case 6: return launch_ner_w<6>(L, ht, which);
    case 8: return launch_ner_w<8>(L, ht, which);
    case 12: return launch_ner_w<12>(L, ht, which);
    case 16: return launch_ner_w<16>(L, ht, which);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_cubic(const Launch &L) {
  HornerTable ht{};
  cudaError_t e = set_smem_ner(k_ner<8, true>, L.smem);
  if (e != cudaSuccess) return e;
  k_ner<8, true><<<L.nblocks, L.threads, L.smem, L.stream>>>(L.descs, L.work, ht);
  return cudaGetLastError();
}

}  // namespace pa
