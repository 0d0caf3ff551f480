// pa_ner.cu -- NER-NUFFT stage (eq:NER_NUFFT, Sec. 3), the weight of
// eq:exact and the inverse DFT over depth, on sm_103a.
//
// One block owns one column j = (jx, jy) of the half spectrum.  Forward:
//   load G1(j, n) / phihat((n - nc)/Mt) at n' = n - nc (the paper's centred
//   theta = 2 pi n / N - pi), zero-pad to Mt = sigma Nt, FFT in shared memory,
//   evaluate at the nz non-integer frequencies tau(j, l) = omega Nt dt / (2 pi)
//   with w window taps (Horner polynomials, tau in double-float) times the
//   centring phase exp(-2 pi i tau nc / Nt), multiply by (dt/dz) W(j, l), and
//   take the inverse DFT over l, all without leaving shared memory.
// Columns and depths on the unpaired Nyquist index of an even length are
// replaced by the Hermitian part F_sym(k) = (F(k) + conj F(-k mod N)) / 2,
// which makes the half-spectrum real inverse DFT equal to the real part of the
// full inverse DFT; it needs the spectrum at +N/2 as well, which G1 holds.
// The adjoint kernel is the exact transpose (spread <-> interpolate).
#include "pa_device.cuh"

namespace pa {

namespace {

constexpr int kThreadsNer = 256;

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

template <int W>
__device__ __forceinline__ float2 ner_interp(const float2 *H, ff tau, const InstDesc &d, const HornerTable &ht) {
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
    const float2 h = H[pad32(idx)];
    acc.x = fmaf(wt[t], h.x, acc.x);
    acc.y = fmaf(wt[t], h.y, acc.y);
    idx = (idx + 1 == Mt) ? 0 : idx + 1;
  }
  return cmul(acc, centring_phase(d, tau));
}

// Transpose of ner_interp: H[p_t] += phi_t conj(phase) v.
template <int W>
__device__ __forceinline__ void ner_spread(float2 *H, ff tau, float2 v, const InstDesc &d, const HornerTable &ht) {
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
    atomicAdd(&H[pad32(idx)].x, wt[t] * vv.x);
    atomicAdd(&H[pad32(idx)].y, wt[t] * vv.y);
    idx = (idx + 1 == Mt) ? 0 : idx + 1;
  }
}

// 4-tap cubic Lagrange interpolation of the uniform Nt-point spectrum at tau
// (the polynomial-interpolation baseline of Sec. 2).
__device__ __forceinline__ float2 cubic_interp(const float2 *H, ff tau, int Nt) {
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
    const float2 h = H[pad32(idx)];
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

// Threads that share one column: the smallest group for which every stage
// of the column transforms fits one round (host-side check mirrors this).
__device__ __forceinline__ int ner_group(const InstDesc &d) { return d.ner_group; }
// Length of each of the two ping-pong buffers of a column.
__host__ __device__ __forceinline__ int ner_buf_len(const InstDesc &d) {
  int L = d.Mt > d.Nt ? d.Mt : d.Nt;
  return padded_len(L > d.Nz ? L : d.Nz);
}

// Forward NER: a group of G threads (G = 64/128/256, named barrier 1 + group
// index) owns one column of the half spectrum and two ping-pong buffers for
// out-of-place FFTs.  Columns on an unpaired Nyquist index (x or y) read two
// sources (A, B) that are transformed one after the other.  CUBIC selects
// the baseline (plain Nt-point FFT, 4-tap Lagrange interpolation, no window).
template <int W, bool CUBIC>
__global__ void __launch_bounds__(kThreadsNer, 3) k_ner(const InstDesc *__restrict__ descs,
                                                        const int2 *__restrict__ work,
                                                        const __grid_constant__ HornerTable ht) {
  extern __shared__ float4 smem_f4[];
  int inst, tile;
  block_work(work, inst, tile);
  const InstDesc &d = descs[inst];
  const int G = ner_group(d);
  const int ngrp = blockDim.x / G;
  const int grp = threadIdx.x / G, t = threadIdx.x % G, bar = 1 + grp;
  const int Nt = d.Nt, Mt = d.Mt, Nz = d.Nz, nY1 = d.nY1, nc = d.nc, hz = d.hz;
  const int ncols = d.Nx * nY1;
  const int col = tile * ngrp + grp;
  if (col >= ncols) return;  // the whole group leaves together
  const int ix = col / nY1, iy = col % nY1;
  const ColInfo ci = col_info(d, ix - d.hx, iy);
  const bool nyq = ci.xnyq || ci.ynyq;
  const int LB = ner_buf_len(d);
  const int LZ = padded_len(Nz);
  float2 *bufA = reinterpret_cast<float2 *>(smem_f4) + (size_t)grp * (2 * LB + LZ);
  float2 *bufB = bufA + LB;
  float2 *Fs = bufB + LB;
  const float scale = d.scale;

  for (int pass = 0; pass < (nyq ? 2 : 1); ++pass) {
    const float2 *src = d.G1 + ((size_t)(pass == 0 ? ci.rowA : ci.rowB) * nY1 + iy) * Nt;
    const bool cj = (pass == 0) && ci.ynyq;
    copy_unrolled<4, float2>(
        Nt, t, G,
        [&](int n) {
          float2 a = src[n];
          if (cj) a.y = -a.y;
          return CUBIC ? a : cscale(a, __ldg(d.invpht + n));
        },
        [&](int n, float2 a) { bufA[pad32(CUBIC ? n : wrap(n - nc, Mt))] = a; });
    if (!CUBIC)
      for (int u = t; u < Mt - Nt; u += G) bufA[pad32(Nt - nc + u)] = make_float2(0.f, 0.f);
    group_sync(bar, G);
    const float2 *H = fft_pingpong<-1>(bufA, bufB, CUBIC ? d.fNt : d.fMt, d.tw, t, G, bar);
#pragma unroll 1
    for (int il = t; il < Nz; il += G) {
      const int l = il - hz;
      float2 F = make_float2(0.f, 0.f);
      if (!(l == 0 && (ci.jx != 0 || ci.jy != 0))) {
        const ff tau = tau_of(d, ci.jx, ci.jy, l);
        const float wgt = weight_of(d, tau, l) * scale;
        const bool lnyq = ((Nz & 1) == 0) && (l == -hz);
        // the second evaluation point: -tau on the depth Nyquist (single
        // source), or the same tau for the B source of a Nyquist column
        const bool two = !nyq && lnyq;
        const ff tp = (nyq && pass == 1 && lnyq) ? ff_neg(tau) : tau;
        float2 v = CUBIC ? cubic_interp(H, tp, Nt) : ner_interp<W>(H, tp, d, ht);
        if (two) {
          const ff tb = ff_neg(tau);
          const float2 vb = CUBIC ? cubic_interp(H, tb, Nt) : ner_interp<W>(H, tb, d, ht);
          v = cadd(v, vb);
        }
        F = cscale(v, (nyq || two) ? 0.5f * wgt : wgt);
      }
      const int pos = pad32(wrap(l, Nz));
      Fs[pos] = pass == 0 ? F : cadd(Fs[pos], F);
    }
    group_sync(bar, G);
  }
  const float2 *R = fft_pingpong<+1>(Fs, bufA, d.fNz, d.tw, t, G, bar);
  float2 *dst = d.Fz + ((size_t)ix * nY1 + iy) * Nz;
  for (int z = t; z < Nz; z += G) dst[z] = R[pad32(z)];
}

// Cotangent sample n of a transformed column (un-centre, 1/phihat).
__device__ __forceinline__ float2 adj_sample(const InstDesc &d, const float2 *H, int n) {
  return cscale(H[pad32(wrap(n - d.nc, d.Mt))], __ldg(d.invpht + n));
}

// Adjoint NER: Fz cotangent -> DFT over depth -> transposed weight and
// window (spread in shared memory) -> inverse FFT -> un-centre, 1/phihat ->
// G1.  Work items: every column off the y-Nyquist row jy = hy (all rows when
// Ny is odd), then for even Ny the Nyquist row in pairs {g, -g}: both columns
// of a pair read the same two G1 sources, so one group computes the four
// contributions in turn and stores, then adds, into the two G1 rows.
template <int W>
__global__ void __launch_bounds__(kThreadsNer, 3) k_ner_adj(const InstDesc *__restrict__ descs,
                                                            const int2 *__restrict__ work,
                                                            const __grid_constant__ HornerTable ht) {
  extern __shared__ float4 smem_f4[];
  int inst, tile;
  block_work(work, inst, tile);
  const InstDesc &d = descs[inst];
  const int G = ner_group(d);
  const int ngrp = blockDim.x / G;
  const int grp = threadIdx.x / G, t = threadIdx.x % G, bar = 1 + grp;
  const int Nt = d.Nt, Mt = d.Mt, Nz = d.Nz, nY1 = d.nY1, hz = d.hz, hx = d.hx, hy = d.hy;
  const bool ny_even = (d.Ny & 1) == 0;
  const int reg_rows = ny_even ? nY1 - 1 : nY1;
  const int nreg = d.Nx * reg_rows;
  const int npair = ny_even ? hx + 1 : 0;
  // the y-Nyquist pairs take four passes each: schedule them first
  const int slot = tile * ngrp + grp;
  if (slot >= nreg + npair) return;
  const int item = slot < npair ? nreg + slot : slot - npair;
  const int LB = ner_buf_len(d);
  const int LZ = padded_len(Nz);
  float2 *bufA = reinterpret_cast<float2 *>(smem_f4) + (size_t)grp * (2 * LB + LZ);
  float2 *bufB = bufA + LB;
  float2 *Fs = bufB + LB;
  const float scale = d.scale;

  // columns handled by this item (one, or a pair on the y-Nyquist row)
  int jxs[2], ncol, iy;
  bool zero_row0 = false;
  if (item < nreg) {
    jxs[0] = item / reg_rows - hx;
    iy = item % reg_rows;
    ncol = 1;
  } else {
    const int g = item - nreg;
    iy = hy;
    if (g == 0) {
      jxs[0] = 0;
      ncol = 1;
    } else if ((d.Nx & 1) == 0 && g == hx) {
      jxs[0] = -hx;
      ncol = 1;
      zero_row0 = true;  // G1 row jx = -hx is read by no column of this row
    } else {
      jxs[0] = g;
      jxs[1] = -g;
      ncol = 2;
    }
  }
  // rows written so far by this item (to store first, then accumulate)
  int written[4];
  int nwritten = 0;
  for (int c = 0; c < ncol; ++c) {
    const ColInfo ci = col_info(d, jxs[c], iy);
    const bool nyq = ci.xnyq || ci.ynyq;
    const float2 *src = d.Fz + ((size_t)(jxs[c] + hx) * nY1 + iy) * Nz;
    copy_unrolled<4, float2>(
        Nz, t, G, [&](int z) { return src[z]; }, [&](int z, float2 v) { Fs[pad32(z)] = v; });
    group_sync(bar, G);
    const float2 *Fr = fft_pingpong<-1>(Fs, bufB, d.fNz, d.tw, t, G, bar);
    if (Fr != Fs) {  // keep the depth spectrum in Fs: both H buffers are needed below
      for (int z = t; z < Nz; z += G) Fs[pad32(z)] = Fr[pad32(z)];
      group_sync(bar, G);
    }
    for (int pass = 0; pass < (nyq ? 2 : 1); ++pass) {
      for (int p = t; p < padded_len(Mt); p += G) bufA[p] = make_float2(0.f, 0.f);
      group_sync(bar, G);
#pragma unroll 1
      for (int il = t; il < Nz; il += G) {
        const int l = il - hz;
        if (l == 0 && (ci.jx != 0 || ci.jy != 0)) continue;
        const ff tau = tau_of(d, ci.jx, ci.jy, l);
        const float wgt = weight_of(d, tau, l) * scale;
        const bool lnyq = ((Nz & 1) == 0) && (l == -hz);
        const float2 v = cscale(Fs[pad32(wrap(l, Nz))], wgt);
        if (!nyq) {
          if (!lnyq) {
            ner_spread<W>(bufA, tau, v, d, ht);
          } else {
            const float2 hv = cscale(v, 0.5f);
            ner_spread<W>(bufA, tau, hv, d, ht);
            ner_spread<W>(bufA, ff_neg(tau), hv, d, ht);
          }
        } else {
          ner_spread<W>(bufA, (pass == 1 && lnyq) ? ff_neg(tau) : tau, cscale(v, 0.5f), d, ht);
        }
      }
      group_sync(bar, G);
      const float2 *H = fft_pingpong<+1>(bufA, bufB, d.fMt, d.tw, t, G, bar);
      // the A source of a y-Nyquist column is the conjugate of its G1 row
      const int row = pass == 0 ? ci.rowA : ci.rowB;
      const bool cj = (pass == 0) && ci.ynyq;
      bool first = true;
      for (int k = 0; k < nwritten; ++k) first = first && (written[k] != row);
      float2 *dst = d.G1 + ((size_t)row * nY1 + iy) * Nt;
      for (int n = t; n < Nt; n += G) {
        float2 v = adj_sample(d, H, n);
        if (cj) v.y = -v.y;
        dst[n] = first ? v : cadd(dst[n], v);
      }
      if (first) written[nwritten++] = row;
      group_sync(bar, G);
    }
  }
  if (zero_row0) {
    float2 *dst = d.G1 + ((size_t)0 * nY1 + iy) * Nt;
    for (int n = t; n < Nt; n += G) dst[n] = make_float2(0.f, 0.f);
  }
}

}  // namespace

int blocks_ner(const InstDesc &d) {
  const int ngrp = kThreadsNer / d.ner_group;
  return (d.Nx * d.nY1 + ngrp - 1) / ngrp;
}
size_t smem_ner(const InstDesc &d) {
  return (size_t)(kThreadsNer / d.ner_group) * (2 * ner_buf_len(d) + padded_len(d.Nz)) * sizeof(float2);
}
int blocks_ner_adj(const InstDesc &d) {
  const int ngrp = kThreadsNer / d.ner_group;
  const bool ny_even = (d.Ny & 1) == 0;
  const int items = d.Nx * (ny_even ? d.nY1 - 1 : d.nY1) + (ny_even ? d.hx + 1 : 0);
  return (items + ngrp - 1) / ngrp;
}
size_t smem_ner_adj(const InstDesc &d) {
  return (size_t)(kThreadsNer / d.ner_group) * (2 * ner_buf_len(d) + padded_len(d.Nz)) * sizeof(float2);
}

template <typename K>
static cudaError_t set_smem_ner(K kernel, size_t smem) {
  if (smem > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

template <int W>
static cudaError_t launch_ner_w(const Launch &L, const HornerTable &ht, int which) {
  cudaError_t e;
  if (which == 1) {
    e = set_smem_ner(k_ner_adj<W>, L.smem);
    if (e != cudaSuccess) return e;
    k_ner_adj<W><<<L.nblocks, kThreadsNer, L.smem, L.stream>>>(L.descs, L.work, ht);
  } else {
    e = set_smem_ner(k_ner<W, false>, L.smem);
    if (e != cudaSuccess) return e;
    k_ner<W, false><<<L.nblocks, kThreadsNer, L.smem, L.stream>>>(L.descs, L.work, ht);
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
  k_ner<8, true><<<L.nblocks, kThreadsNer, L.smem, L.stream>>>(L.descs, L.work, ht);
  return cudaGetLastError();
}

}  // namespace pa
