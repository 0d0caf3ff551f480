// pa_ner_common.cuh -- pieces of the NER stage (Sec. 3) shared by the block
// kernels (pa_ner.cu) and the warp-per-column kernels (pa_ner_warp.cu): the
// evaluation points tau(j, l), the weight W(j, l), the centring phase, the
// window taps of the oversampled time-frequency grid, and the slot lists
// that order the (column, source) transforms of the half spectrum.
#pragma once
#include "pa_device.cuh"

namespace pa {

namespace {

template <int W>
struct HornerDeg {
  static constexpr int v = W <= 6 ? 7 : (W <= 8 ? 8 : (W <= 12 ? 10 : 14));
};

__device__ __forceinline__ ff ff_neg(ff a) { return {-a.hi, -a.lo}; }

// tau(j, l) = sign(l) sqrt(ax jx^2 + ay jy^2 + az l^2) in double-float; the
// column's part ax jx^2 + ay jy^2 is tau_base(d, jx, jy).
__device__ __forceinline__ ff tau_base(const InstDesc &d, int jx, int jy) {
  return ff_add(ff_mul_f({d.ax_hi, d.ax_lo}, float(jx * jx)), ff_mul_f({d.ay_hi, d.ay_lo}, float(jy * jy)));
}
__device__ __forceinline__ ff tau_at(const InstDesc &d, ff base, int l) {
  ff t = ff_sqrt(ff_add(base, ff_mul_f({d.az_hi, d.az_lo}, float(l * l))));
  return l < 0 ? ff_neg(t) : t;
}
__device__ __forceinline__ ff tau_of(const InstDesc &d, int jx, int jy, int l) {
  return tau_at(d, tau_base(d, jx, jy), l);
}

// W(j, l) = 2 c |kz| / |K| with W(0, 0) = 2c and W(j != 0, 0) = 0.
__device__ __forceinline__ float weight_of(const InstDesc &d, ff tau, int l) {
  if (l == 0) return tau.hi == 0.f ? d.two_c : 0.f;
  return __fdividef(d.two_c * d.sqrt_az * fabsf(float(l)), fabsf(tau.hi));
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
// First tap (not reduced mod L; monotone in tau) and fraction of u = scale * tau.
__device__ __forceinline__ void footprint_unwrapped(ff tau, int scale, int half, int &pu, float &fr) {
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
  pu = int(fb) - half + 1;
}
__device__ __forceinline__ void footprint(ff tau, int scale, int L, int half, int &p0, float &fr) {
  int pu;
  footprint_unwrapped(tau, scale, half, pu, fr);
  p0 = wrap(pu, L);
}

template <int W>
__device__ __forceinline__ void window_taps(float fr, const HornerTable &ht, float *wt) {
  constexpr int D = HornerDeg<W>::v, KE = D / 2 + 1;
  const float s = 2.f * fr - 1.f, u = s * s;
  const float2 uu = make_float2(u, u), sm = make_float2(s, -s);
#pragma unroll
  for (int i = 0; i < W / 2; ++i) {  // taps i and W - 1 - i: E(u) +- s O(u)
    float2 a = ht.eo[i][KE - 1];
#pragma unroll
    for (int k = KE - 2; k >= 0; --k) a = __ffma2_rn(a, uu, ht.eo[i][k]);
    const float2 t = __ffma2_rn(sm, make_float2(a.y, a.y), make_float2(a.x, a.x));
    wt[i] = t.x;
    wt[W - 1 - i] = t.y;
  }
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

}  // namespace

}  // namespace pa
