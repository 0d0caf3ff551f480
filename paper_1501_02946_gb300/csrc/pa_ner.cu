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
#include "pa_ner_common.cuh"

namespace pa {

namespace {

constexpr int kNerMaxCB = 4;  // most columns per block
constexpr int kNerPad = 4;    // one pad row per 16 rows of the [n][CB] buffers
__device__ __forceinline__ int prow(int e) { return pad_row<kNerPad>(e); }


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
    acc = __ffma2_rn(make_float2(wt[t], wt[t]), h, acc);
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
    acc = __ffma2_rn(make_float2(wt[t], wt[t]), h, acc);
    idx = (idx + 1 == Nt) ? 0 : idx + 1;
  }
  return acc;
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
  if (L.host && L.host->ner_warp) return launch_ner_warp(L, ht, which);
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
