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
    const float2 h = H[idx];
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
    atomicAdd(&H[idx].x, wt[t] * vv.x);
    atomicAdd(&H[idx].y, wt[t] * vv.y);
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
    const float2 h = H[idx];
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

// Forward NER of one column into Fz.  CUBIC selects the baseline.
template <int W, bool CUBIC>
__global__ void __launch_bounds__(kThreadsNer) k_ner(const InstDesc *__restrict__ descs, const int2 *__restrict__ work,
                                                     const __grid_constant__ HornerTable ht) {
  extern __shared__ float4 smem_f4[];
  int inst, tile;
  block_work(work, inst, tile);
  const InstDesc &d = descs[inst];
  const int Nt = d.Nt, Mt = d.Mt, Nz = d.Nz, nY1 = d.nY1, nc = d.nc, hz = d.hz;
  if (tile >= d.Nx * nY1) return;
  const int ix = tile / nY1, iy = tile % nY1;
  const ColInfo ci = col_info(d, ix - d.hx, iy);
  const bool nyq = ci.xnyq || ci.ynyq;
  const int L = CUBIC ? Nt : Mt;
  float2 *HA = reinterpret_cast<float2 *>(smem_f4);
  float2 *HB = HA + L;
  float2 *Fs = HB + L;
  const int tid = threadIdx.x, nthr = blockDim.x;

  const float2 *srcA = d.G1 + ((size_t)ci.rowA * nY1 + iy) * Nt;
  const float2 *srcB = d.G1 + ((size_t)ci.rowB * nY1 + iy) * Nt;
  for (int n = tid; n < Nt; n += nthr) {
    float2 a = srcA[n];
    if (ci.ynyq) a.y = -a.y;
    float2 b = nyq ? srcB[n] : make_float2(0.f, 0.f);
    if (CUBIC) {
      HA[n] = a;
      HB[n] = b;
    } else {
      const float sc = __ldg(d.invpht + n);
      const int pos = wrap(n - nc, Mt);
      HA[pos] = cscale(a, sc);
      HB[pos] = cscale(b, sc);
    }
  }
  if (!CUBIC) {
    for (int u = tid; u < Mt - Nt; u += nthr) {
      HA[Nt - nc + u] = make_float2(0.f, 0.f);
      HB[Nt - nc + u] = make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  const FftPlan &fp = CUBIC ? d.fNt : d.fMt;
  fft_smem<-1>(HA, 1, 1, fp, d.tw, tid, nthr);
  if (nyq) fft_smem<-1>(HB, 1, 1, fp, d.tw, tid, nthr);

  const float scale = d.scale;
  for (int il = tid; il < Nz; il += nthr) {
    const int l = il - hz;
    float2 F = make_float2(0.f, 0.f);
    if (!(l == 0 && (ci.jx != 0 || ci.jy != 0))) {
      const ff tau = tau_of(d, ci.jx, ci.jy, l);
      const float wgt = weight_of(d, tau, l) * scale;
      const bool lnyq = ((Nz & 1) == 0) && (l == -hz);
      float2 val = CUBIC ? cubic_interp(HA, tau, Nt) : ner_interp<W>(HA, tau, d, ht);
      if (nyq || lnyq) {
        const ff tb = lnyq ? ff_neg(tau) : tau;
        const float2 *Hb = nyq ? HB : HA;
        const float2 vb = CUBIC ? cubic_interp(Hb, tb, Nt) : ner_interp<W>(Hb, tb, d, ht);
        val = make_float2(0.5f * (val.x + vb.x), 0.5f * (val.y + vb.y));
      }
      F = cscale(val, wgt);
    }
    Fs[wrap(l, Nz)] = F;
  }
  __syncthreads();
  fft_smem<+1>(Fs, 1, 1, d.fNz, d.tw, tid, nthr);
  float2 *dst = d.Fz + ((size_t)ix * nY1 + iy) * Nz;
  for (int z = tid; z < Nz; z += nthr) dst[z] = Fs[z];
}

// Adjoint of one column: Fz cotangent -> A' (in HA) and B' (in HB), the
// cotangents of the two G1 sources of the column, before the final
// 1/phihat and un-centring (done by the caller).
template <int W>
__device__ void ner_adj_column(const InstDesc &d, const HornerTable &ht, const ColInfo &ci, int ix, int iy,
                               float2 *HA, float2 *HB, float2 *Fs, int tid, int nthr) {
  const int Mt = d.Mt, Nz = d.Nz, nY1 = d.nY1, hz = d.hz;
  const bool nyq = ci.xnyq || ci.ynyq;
  const float2 *src = d.Fz + ((size_t)ix * nY1 + iy) * Nz;
  for (int z = tid; z < Nz; z += nthr) Fs[z] = src[z];
  for (int p = tid; p < Mt; p += nthr) {
    HA[p] = make_float2(0.f, 0.f);
    HB[p] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  fft_smem<-1>(Fs, 1, 1, d.fNz, d.tw, tid, nthr);
  const float scale = d.scale;
  for (int il = tid; il < Nz; il += nthr) {
    const int l = il - hz;
    if (l == 0 && (ci.jx != 0 || ci.jy != 0)) continue;
    const ff tau = tau_of(d, ci.jx, ci.jy, l);
    const float wgt = weight_of(d, tau, l) * scale;
    const bool lnyq = ((Nz & 1) == 0) && (l == -hz);
    const float2 v = cscale(Fs[wrap(l, Nz)], wgt);
    if (!nyq && !lnyq) {
      ner_spread<W>(HA, tau, v, d, ht);
    } else {
      const float2 hv = cscale(v, 0.5f);
      ner_spread<W>(HA, tau, hv, d, ht);
      ner_spread<W>(nyq ? HB : HA, lnyq ? ff_neg(tau) : tau, hv, d, ht);
    }
  }
  __syncthreads();
  fft_smem<+1>(HA, 1, 1, d.fMt, d.tw, tid, nthr);
  if (nyq) fft_smem<+1>(HB, 1, 1, d.fMt, d.tw, tid, nthr);
}

// Cotangent sample n of a transformed column (un-centre, 1/phihat).
__device__ __forceinline__ float2 adj_sample(const InstDesc &d, const float2 *H, int n) {
  return cscale(H[wrap(n - d.nc, d.Mt)], __ldg(d.invpht + n));
}

// Work items: every column of the rows jy < hy (all rows when Ny is odd) on
// its own, then, for even Ny, the Nyquist row jy = hy in pairs {g, -g}
// because both columns of a pair read the same two G1 sources.
template <int W>
__global__ void __launch_bounds__(kThreadsNer) k_ner_adj(const InstDesc *__restrict__ descs,
                                                         const int2 *__restrict__ work,
                                                         const __grid_constant__ HornerTable ht) {
  extern __shared__ float4 smem_f4[];
  int inst, tile;
  block_work(work, inst, tile);
  const InstDesc &d = descs[inst];
  const int Nt = d.Nt, Mt = d.Mt, Nz = d.Nz, nY1 = d.nY1, hx = d.hx, hy = d.hy;
  const bool ny_even = (d.Ny & 1) == 0;
  const int reg_rows = ny_even ? nY1 - 1 : nY1;
  const int nreg = d.Nx * reg_rows;
  const int npair = ny_even ? hx + 1 : 0;
  if (tile >= nreg + npair) return;
  float2 *H = reinterpret_cast<float2 *>(smem_f4);  // 4 arrays of Mt, then Fs
  float2 *Fs = H + 4 * (size_t)Mt;
  const int tid = threadIdx.x, nthr = blockDim.x;
  float2 *G1 = d.G1;

  if (tile < nreg) {
    const int ix = tile / reg_rows, iy = tile % reg_rows;
    const ColInfo ci = col_info(d, ix - hx, iy);
    ner_adj_column<W>(d, ht, ci, ix, iy, H, H + Mt, Fs, tid, nthr);
    float2 *dA = G1 + ((size_t)ci.rowA * nY1 + iy) * Nt;
    float2 *dB = G1 + ((size_t)ci.rowB * nY1 + iy) * Nt;
    for (int n = tid; n < Nt; n += nthr) {
      dA[n] = adj_sample(d, H, n);
      if (ci.xnyq) dB[n] = adj_sample(d, H + Mt, n);
    }
    return;
  }
  // Nyquist row, pair {g, -g}
  const int g = tile - nreg;
  const int iy = hy;
  const bool x_even = (d.Nx & 1) == 0;
  const bool single_zero = (g == 0);
  const bool single_nyq = x_even && (g == hx);
  // first column: jx = g (or -hx for the even-Nx end), second: jx = -g
  const int jx0 = single_nyq ? -hx : g;
  {
    const ColInfo ci = col_info(d, jx0, iy);
    ner_adj_column<W>(d, ht, ci, jx0 + hx, iy, H, H + Mt, Fs, tid, nthr);
  }
  if (!single_zero && !single_nyq) {
    const ColInfo ci = col_info(d, -g, iy);
    ner_adj_column<W>(d, ht, ci, -g + hx, iy, H + 2 * Mt, H + 3 * Mt, Fs, tid, nthr);
  }
  // A' of column jx goes (conjugated) to row -jx, B' to row flip(jx).
  for (int n = tid; n < Nt; n += nthr) {
    const float2 A0 = adj_sample(d, H, n), B0 = adj_sample(d, H + Mt, n);
    if (single_zero) {
      G1[((size_t)hx * nY1 + iy) * Nt + n] = cadd(cconj(A0), B0);
    } else if (single_nyq) {
      G1[((size_t)(2 * hx) * nY1 + iy) * Nt + n] = cadd(cconj(A0), B0);
      G1[((size_t)0 * nY1 + iy) * Nt + n] = make_float2(0.f, 0.f);
    } else {
      const float2 A1 = adj_sample(d, H + 2 * Mt, n), B1 = adj_sample(d, H + 3 * Mt, n);
      // column g: A0 -> row -g, B0 -> row g; column -g: A1 -> row g, B1 -> row -g
      G1[((size_t)(g + hx) * nY1 + iy) * Nt + n] = cadd(cconj(A1), B0);
      G1[((size_t)(-g + hx) * nY1 + iy) * Nt + n] = cadd(cconj(A0), B1);
    }
  }
  (void)Nz;
}

}  // namespace

int blocks_ner(const InstDesc &d) { return d.Nx * d.nY1; }
size_t smem_ner(const InstDesc &d) {
  const int L = d.Mt > d.Nt ? d.Mt : d.Nt;
  return (2 * (size_t)L + d.Nz) * sizeof(float2);
}
int blocks_ner_adj(const InstDesc &d) {
  const bool ny_even = (d.Ny & 1) == 0;
  return d.Nx * (ny_even ? d.nY1 - 1 : d.nY1) + (ny_even ? d.hx + 1 : 0);
}
size_t smem_ner_adj(const InstDesc &d) { return (4 * (size_t)d.Mt + d.Nz) * sizeof(float2); }

template <typename K>
static cudaError_t set_smem_ner(K kernel, size_t smem) {
  if (smem > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaSuccess;
}

template <int W>
static cudaError_t launch_ner_w(const Launch &L, const HornerTable &ht, bool adjoint) {
  cudaError_t e;
  if (adjoint) {
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
  switch (width) {
    case 6: return launch_ner_w<6>(L, ht, adjoint);
    case 8: return launch_ner_w<8>(L, ht, adjoint);
    case 12: return launch_ner_w<12>(L, ht, adjoint);
    case 16: return launch_ner_w<16>(L, ht, adjoint);
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
