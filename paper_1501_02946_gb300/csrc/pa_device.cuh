// pa_device.cuh -- device helpers of the NEDNER-NUFFT kernels: complex
// arithmetic, double-float arithmetic for the time-frequency arguments, and a
// batched mixed-radix Stockham FFT that runs in shared memory.
#pragma once

#include <cstdint>
#include <utility>

#include <cuda.h>
#include "pa_internal.h"

// Programmatic dependent launch of the single-plan pipeline kernels (0: the
// same kernels launched the ordinary way).
#ifndef PA_PDL
#define PA_PDL 1
#endif

namespace pa {

// Programmatic dependent launch.  A kernel started by launch_pdl may be
// scheduled while the previous kernel of its stream drains.  Its first
// statement is griddep_enter(): griddepcontrol.wait returns once that kernel
// has completed and its memory operations are visible (at once for a kernel
// launched the ordinary way), and griddepcontrol.launch_dependents then lets
// the next kernel of the stream be scheduled early in the same way.  The
// previous kernel never waits for its dependents, so no wait can cycle.
__device__ __forceinline__ void griddep_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ---------------------------------------------------------------- complex
// Complex sums as packed two-wide FP32 adds (sm_100+; each component rounds
// exactly as a scalar add).
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// multiply by DIR * i (DIR = -1: by -i, DIR = +1: by +i)
template <int DIR>
__device__ __forceinline__ float2 mul_i(float2 a) {
  return DIR > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ---------------------------------------------------------- double-float
// Error-free transformations (Knuth two-sum, FMA two-product) and the
// resulting ~48-bit arithmetic on (hi, lo) pairs of floats.
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff quick_two_sum(float a, float b) {
  float s = a + b;
  float e = b - (s - a);
  return {s, e};
}
__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ ff two_prod(float a, float b) {
  float p = a * b;
  float e = fmaf(a, b, -p);
  return {p, e};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  ff p = two_prod(a.hi, b);
  p.lo = fmaf(a.lo, b, p.lo);
  return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  ff p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  return quick_two_sum(p.hi, p.lo);
}
// square root with one Newton correction: s + (a - s^2) / (2 s)
__device__ __forceinline__ ff ff_sqrt(ff a) {
  if (!(a.hi > 0.f)) return {0.f, 0.f};
  float s = sqrtf(a.hi);
  ff s2 = two_prod(s, s);
  // the correction is ~1e-8 of s: a two-ulp quotient is exact enough
  float r = __fdividef((a.hi - s2.hi) - s2.lo + a.lo, 2.f * s);
  return quick_two_sum(s, r);
}

// -------------------------------------------------------------- FFT
// Exact values of cos(2 pi m / R) and sin(2 pi m / R) for R = 16, 3, 5, 7
// (indices are compile-time constants after unrolling, so these fold).
struct Tw16 {
  __device__ __forceinline__ static constexpr float c(int m) {
    return m == 0 ? 1.0f : m == 1 ? 0.92387953251128674f : m == 2 ? 0.70710678118654752f
         : m == 3 ? 0.38268343236508977f : m == 4 ? 0.0f : m == 5 ? -0.38268343236508977f
         : m == 6 ? -0.70710678118654752f : m == 7 ? -0.92387953251128674f : m == 8 ? -1.0f
         : m == 9 ? -0.92387953251128674f : m == 10 ? -0.70710678118654752f
         : m == 11 ? -0.38268343236508977f : m == 12 ? 0.0f : m == 13 ? 0.38268343236508977f
         : m == 14 ? 0.70710678118654752f : 0.92387953251128674f;
  }
  __device__ __forceinline__ static constexpr float s(int m) { return c((m + 12) & 15); }
};
// cos and sin of 2 pi m / 32 from the first octant by symmetry.
struct Tw32 {
  __device__ __forceinline__ static constexpr float oct(int m) {  // cos(2 pi m / 32), 0 <= m <= 8
    return m == 0 ? 1.0f : m == 1 ? 0.98078528040323043f : m == 2 ? 0.92387953251128674f
         : m == 3 ? 0.83146961230254524f : m == 4 ? 0.70710678118654752f : m == 5 ? 0.55557023301960218f
         : m == 6 ? 0.38268343236508977f : m == 7 ? 0.19509032201612826f : 0.0f;
  }
  __device__ __forceinline__ static constexpr float c(int m) {
    return m <= 8 ? oct(m) : m <= 16 ? -oct(16 - m) : m <= 24 ? -oct(m - 16) : oct(32 - m);
  }
  __device__ __forceinline__ static constexpr float s(int m) { return c((m + 24) & 31); }
};
struct Tw3 {
  __device__ __forceinline__ static constexpr float c(int m) { return m == 0 ? 1.0f : -0.5f; }
  __device__ __forceinline__ static constexpr float s(int m) {
    return m == 0 ? 0.0f : m == 1 ? 0.86602540378443865f : -0.86602540378443865f;
  }
};
struct Tw5 {
  __device__ __forceinline__ static constexpr float c(int m) {
    return m == 0 ? 1.0f : (m == 1 || m == 4) ? 0.30901699437494742f : -0.80901699437494742f;
  }
  __device__ __forceinline__ static constexpr float s(int m) {
    return m == 0 ? 0.0f : m == 1 ? 0.95105651629515357f : m == 2 ? 0.58778525229247313f
         : m == 3 ? -0.58778525229247313f : -0.95105651629515357f;
  }
};
struct Tw7 {
  __device__ __forceinline__ static constexpr float c(int m) {
    return m == 0 ? 1.0f : (m == 1 || m == 6) ? 0.62348980185873353f
         : (m == 2 || m == 5) ? -0.22252093395631440f : -0.90096886790241913f;
  }
  __device__ __forceinline__ static constexpr float s(int m) {
    return m == 0 ? 0.0f : m == 1 ? 0.78183148246802981f : m == 2 ? 0.97492791218182361f
         : m == 3 ? 0.43388373911755812f : m == 4 ? -0.43388373911755812f
         : m == 5 ? -0.97492791218182361f : -0.78183148246802981f;
  }
};

// In-register DFT of size R: v[k] <- sum_n v[n] exp(DIR 2 pi i n k / R).
template <int R, int DIR>
struct Dft;

template <int DIR>
struct Dft<2, DIR> {
  __device__ __forceinline__ static void run(float2 *v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <int DIR>
struct Dft<4, DIR> {
  __device__ __forceinline__ static void run(float2 *v) {
    float2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
    float2 s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
    float2 t = mul_i<DIR>(d13);
    v[0] = cadd(s02, s13);
    v[2] = csub(s02, s13);
    v[1] = cadd(d02, t);
    v[3] = csub(d02, t);
  }
};

template <typename TW, int R, int DIR>
struct DftNaive {
  __device__ __forceinline__ static void run(float2 *v) {
    float2 out[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
      float2 acc = v[0];
#pragma unroll
      for (int n = 1; n < R; ++n) {
        const int e = (n * k) % R;
        if (e == 0) {
          acc = cadd(acc, v[n]);
        } else {
          const float c = TW::c(e), s = DIR * TW::s(e);
          acc.x += v[n].x * c - v[n].y * s;
          acc.y += v[n].x * s + v[n].y * c;
        }
      }
      out[k] = acc;
    }
#pragma unroll
    for (int k = 0; k < R; ++k) v[k] = out[k];
  }
};
template <int DIR>
struct Dft<3, DIR> : DftNaive<Tw3, 3, DIR> {};
template <int DIR>
struct Dft<5, DIR> : DftNaive<Tw5, 5, DIR> {};
template <int DIR>
struct Dft<7, DIR> : DftNaive<Tw7, 7, DIR> {};

// Cooley-Tukey composition N = N1 N2 (N divides the size TWN of the table
// TW): n = N2 n1 + n2, k = k1 + N1 k2, inner twiddle exp(DIR 2 pi i n2 k1 / N).
template <int N1, int N2, int DIR, typename TW = Tw16, int TWN = 16>
struct DftComp {
  __device__ __forceinline__ static void run(float2 *v) {
    constexpr int N = N1 * N2;
    float2 y[N2][N1];
#pragma unroll
    for (int n2 = 0; n2 < N2; ++n2) {
      float2 t[N1];
#pragma unroll
      for (int n1 = 0; n1 < N1; ++n1) t[n1] = v[N2 * n1 + n2];
      Dft<N1, DIR>::run(t);
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) {
        const int e = ((n2 * k1) * (TWN / N)) % TWN;
        if (e == 0) {
          y[n2][k1] = t[k1];
        } else {
          const float c = TW::c(e), s = DIR * TW::s(e);
          y[n2][k1] = make_float2(t[k1].x * c - t[k1].y * s, t[k1].x * s + t[k1].y * c);
        }
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
      float2 t[N2];
#pragma unroll
      for (int n2 = 0; n2 < N2; ++n2) t[n2] = y[n2][k1];
      Dft<N2, DIR>::run(t);
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) v[k1 + N1 * k2] = t[k2];
    }
  }
};
template <int DIR>
struct Dft<8, DIR> : DftComp<2, 4, DIR> {};
template <int DIR>
struct Dft<16, DIR> : DftComp<4, 4, DIR> {};
template <int DIR>
struct Dft<32, DIR> : DftComp<2, 16, DIR, Tw32, 32> {};

// Items (butterflies) a thread holds per round, by radix.
template <int R>
struct Ipt {
  static constexpr int v = R >= 16 ? 1 : (R >= 5 ? 2 : 4);
};

// One Stockham stage (Govindaraju et al., "High performance discrete Fourier
// transforms on graphics processors", SC 2008) applied in place: every item
// j < L/R reads x[j + t L/R] (t < R), multiplies by exp(DIR 2 pi i t k / (Ns R))
// with k = j mod Ns, takes an R-point DFT and writes position
// (j / Ns) Ns R + k + t Ns.  Sequences b < nb are interleaved with stride 1
// (element i of sequence b at buf[i * estride + b]).  Reads of a round finish
// (barrier) before its writes; rounds cover whole sequences.
// Barrier of the threads that share one transform: the whole block
// (bar_id = 0), one whole warp (nthr = 32; the group must be warp-aligned) or
// a named barrier over `nthr` threads (bar_id >= 1).
__device__ __forceinline__ void group_sync(int bar_id, int nthr) {
  if (bar_id == 0) {
    __syncthreads();
  } else if (nthr == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(nthr) : "memory");
  }
}

// Element row e of a transform buffer, with one pad row after every 2^PADSH
// rows when PADSH > 0 (spreads strided accesses of narrow batches over the
// shared-memory banks).
template <int PADSH>
__host__ __device__ __forceinline__ int pad_row(int e) {
  return PADSH > 0 ? e + (e >> PADSH) : e;
}
template <int PADSH>
__host__ __device__ __forceinline__ int padded_rows(int L) {
  return PADSH > 0 ? L + (L >> PADSH) + 1 : L;
}

template <int R, int DIR, int PADSH>
__device__ __forceinline__ void fft_stage(float2 *buf, int estride, int nb, int L, int Ns,
                                          const float2 *__restrict__ tw, int tid, int nthr, int bar_id = 0) {
  constexpr int IPT = Ipt<R>::v;
  const int nj = L / R;
  const int twstep = L / (Ns * R);
  int spr = (nthr * IPT) / nj;
  if (spr < 1) spr = 1;
  for (int b0 = 0; b0 < nb; b0 += spr) {
    const int nbr = min(spr, nb - b0);
    const int items = nj * nbr;
    float2 v[IPT][R];
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
      const int item = tid + it * nthr;
      if (item < items) {
        const int b = b0 + item % nbr;
        const int j = item / nbr;
        const int k = j % Ns;
#pragma unroll
        for (int t = 0; t < R; ++t) {
          float2 x = buf[pad_row<PADSH>(j + t * nj) * estride + b];
          if (t > 0 && k > 0) {
            float2 w = __ldg(tw + t * k * twstep);
            if (DIR > 0) w.y = -w.y;
            x = cmul(x, w);
          }
          v[it][t] = x;
        }
      }
    }
    group_sync(bar_id, nthr);
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
      const int item = tid + it * nthr;
      if (item < items) {
        const int b = b0 + item % nbr;
        const int j = item / nbr;
        const int k = j % Ns;
        Dft<R, DIR>::run(v[it]);
        const int o = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int t = 0; t < R; ++t) buf[pad_row<PADSH>(o + t * Ns) * estride + b] = v[it][t];
      }
    }
    group_sync(bar_id, nthr);
  }
}

// The same stage when the length, the sequence count and the thread count are
// powers of two: every index split is a shift or a mask, and a thread keeps
// one sequence (b) for all its items of a round.
__device__ __forceinline__ int ilog2_pow2(int x) { return __ffs(x) - 1; }

// BAND: input rows zlo .. zhi - 1 are read as zeros (not loaded).
template <int R, int DIR, int PADSH, bool BAND = false>
__device__ __forceinline__ void fft_stage_p2(float2 *buf, int estride, int lgnb, int lgL, int lgNs,
                                             const float2 *__restrict__ tw, int tid, int lgT, int bar_id,
                                             int zlo = 0, int zhi = 0) {
  constexpr int IPT = Ipt<R>::v;
  constexpr int LGR = R == 32 ? 5 : (R == 16 ? 4 : (R == 8 ? 3 : (R == 4 ? 2 : 1)));
  constexpr int LGIPT = IPT == 1 ? 0 : (IPT == 2 ? 1 : 2);
  const int lgnj = lgL - LGR;
  const int nj = 1 << lgnj;
  int lgnbr = lgT + LGIPT - lgnj;  // sequences per round (the plan keeps it >= 0)
  if (lgnbr > lgnb) lgnbr = lgnb;
  if (lgnbr > lgT) lgnbr = lgT;
  if (lgnbr < 0) lgnbr = 0;
  const int nbr = 1 << lgnbr;
  const int j0 = tid >> lgnbr, jstep = 1 << (lgT - lgnbr);
  const int kmask = (1 << lgNs) - 1;
  const int lgtw = lgL - lgNs - LGR;
  for (int b0 = 0; b0 < (1 << lgnb); b0 += nbr) {
    const int b = b0 + (tid & (nbr - 1));
    float2 v[IPT][R];
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
      const int j = j0 + it * jstep;
      if (j < nj) {
        const int k = j & kmask;
#pragma unroll
        for (int t = 0; t < R; ++t) {
          const int row = j + (t << lgnj);
          float2 x = (BAND && row >= zlo && row < zhi) ? make_float2(0.f, 0.f) : buf[pad_row<PADSH>(row) * estride + b];
          if (t > 0) {  // tw[0] = 1 leaves x unchanged
            float2 w = __ldg(tw + ((t * k) << lgtw));
            if (DIR > 0) w.y = -w.y;
            x = cmul(x, w);
          }
          v[it][t] = x;
        }
      }
    }
    group_sync(bar_id, 1 << lgT);
#pragma unroll
    for (int it = 0; it < IPT; ++it) {
      const int j = j0 + it * jstep;
      if (j < nj) {
        const int k = j & kmask;
        Dft<R, DIR>::run(v[it]);
        const int o = ((j >> lgNs) << (lgNs + LGR)) + k;
#pragma unroll
        for (int t = 0; t < R; ++t) buf[pad_row<PADSH>(o + (t << lgNs)) * estride + b] = v[it][t];
      }
    }
    group_sync(bar_id, 1 << lgT);
  }
}

// Transform of compile-time length 2^LGL (radix-16 stages, then one radix-8,
// -4 or -2 stage): every index split folds to constants, so the transform can
// sit inside a loop without its address arithmetic being kept live across
// iterations.  Sequences and threads as in fft_stage_p2.
// BAND (length 512 only): input rows zlo .. zhi - 1 are zeros and are not
// read (the first pass takes them as zeros; it writes every row).
template <int LGL, int DIR, int PADSH = 0, bool BAND = false>
__device__ __forceinline__ void fft_fixed(float2 *buf, int estride, int lgnb, int lgT, const float2 *__restrict__ tw,
                                          int tid, int bar_id = 0, int zlo = 0, int zhi = 0) {
  static_assert(!BAND || LGL == 9, "a zero band for the 512-point schedule only");
  if constexpr (LGL == 9) {  // 16 x 32: two passes through shared memory instead of three
    fft_stage_p2<16, DIR, PADSH, BAND>(buf, estride, lgnb, LGL, 0, tw, tid, lgT, bar_id, zlo, zhi);
    fft_stage_p2<32, DIR, PADSH>(buf, estride, lgnb, LGL, 4, tw, tid, lgT, bar_id);
    return;
  }
  constexpr int n16 = LGL / 4, rem = LGL % 4;
#pragma unroll
  for (int st = 0; st < n16; ++st) fft_stage_p2<16, DIR, PADSH>(buf, estride, lgnb, LGL, 4 * st, tw, tid, lgT, bar_id);
  if (rem == 3) fft_stage_p2<8, DIR, PADSH>(buf, estride, lgnb, LGL, 4 * n16, tw, tid, lgT, bar_id);
  if (rem == 2) fft_stage_p2<4, DIR, PADSH>(buf, estride, lgnb, LGL, 4 * n16, tw, tid, lgT, bar_id);
  if (rem == 1) fft_stage_p2<2, DIR, PADSH>(buf, estride, lgnb, LGL, 4 * n16, tw, tid, lgT, bar_id);
}

// Whole transform y[k] = sum_i x[i] exp(DIR 2 pi i i k / L), unnormalised,
// in place in shared memory (element i of sequence b at
// buf[pad_row<PADSH>(i) * estride + b]).  All threads of the block must call it.
template <int DIR, int PADSH = 0>
__device__ void fft_smem(float2 *buf, int estride, int nb, const FftPlan &fp, const float2 *__restrict__ twbase,
                         int tid, int nthr, int bar_id = 0) {
  const float2 *tw = twbase + fp.tw;
  const int L = fp.L;
  const int nst = fp.nst;
  int Ns = 1, s = 0;
  if (((L & (L - 1)) | (nb & (nb - 1)) | (nthr & (nthr - 1))) == 0) {
    // power-of-two schedule: radices 16, 8, 4, 2 in that order
    const int lgL = ilog2_pow2(L), lgnb = ilog2_pow2(nb), lgT = ilog2_pow2(nthr);
    int lgNs = 0;
#define PA_FFT_RUN_P2(R, LGR)                                                    \
  while (s < nst && fp.radix[s] == R) {                                          \
    fft_stage_p2<R, DIR, PADSH>(buf, estride, lgnb, lgL, lgNs, tw, tid, lgT, bar_id);  \
    lgNs += LGR;                                                                 \
    ++s;                                                                         \
  }
    PA_FFT_RUN_P2(16, 4)
    PA_FFT_RUN_P2(8, 3)
    PA_FFT_RUN_P2(4, 2)
    PA_FFT_RUN_P2(2, 1)
#undef PA_FFT_RUN_P2
    return;
  }
  // The schedule lists radices in the order 16, 8, 4, 2, 3, 5, 7; one loop per
  // radix keeps the register allocation of each radix separate.
#define PA_FFT_RUN(R)                                                   \
  while (s < nst && fp.radix[s] == R) {                                 \
    fft_stage<R, DIR, PADSH>(buf, estride, nb, L, Ns, tw, tid, nthr, bar_id);  \
    Ns *= R;                                                            \
    ++s;                                                                \
  }
  PA_FFT_RUN(16)
  PA_FFT_RUN(8)
  PA_FFT_RUN(4)
  PA_FFT_RUN(2)
  PA_FFT_RUN(3)
  PA_FFT_RUN(5)
  PA_FFT_RUN(7)
#undef PA_FFT_RUN
}


// n items moved by the block with U loads in flight per thread: every thread
// first issues up to U independent loads ld(i), then stores them st(i, v).
template <int U, typename T, typename LoadF, typename StoreF>
__device__ __forceinline__ void copy_unrolled(int n, int tid, int nthr, LoadF ld, StoreF st) {
  for (int base = tid; base < n; base += nthr * U) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = base + u * nthr;
      if (i < n) v[u] = ld(i);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = base + u * nthr;
      if (i < n) st(i, v[u]);
    }
  }
}

// Instance and tile of this block.
// ------------------------------------------------ asynchronous tile copies
// Bulk copies global -> shared through the TMA engine (cp.async.bulk), each
// completing on an mbarrier of the block with a byte count (complete_tx).
// Every wait is bounded: after kMbarPolls unsuccessful polls it gives up and
// reports failure, which the kernel records in the plan's status word.
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// dst, src 16-byte aligned; bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// Tiled bulk copy of the 3-D box at element coordinates (x, y, z) of a tensor
// map (a __grid_constant__ kernel parameter) into shared memory, completing
// on `bar` with the box's full byte count (elements outside the tensor are
// filled with zeros).  dst 128-byte aligned; x * element size a multiple of 16.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}
// 2-D form: the box at (x, y).
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}
// Tiled bulk store of the 2-D box at element coordinates (x, y) of a tensor
// map from shared memory (128-byte aligned; x * element size a multiple of
// 16, x, y >= 0; elements outside the tensor are not written), in the
// calling thread's bulk group; commit, then wait until the sources of all
// but the last N groups have been read (wait_read) or written (wait).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, const void *src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(smem_addr(src))
               : "memory");
}
// 3-D form: the box at (x, y, z).
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, int x, int y, int z, const void *src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(x), "r"(y), "r"(z), "r"(smem_addr(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
template <int N>
__device__ __forceinline__ void bulk_wait() {
  asm volatile("cp.async.bulk.wait_group %0;" ::"n"(N) : "memory");
}
// Orders this thread's (and, after a block barrier, the block's) earlier
// shared-memory accesses before later bulk copies into the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
constexpr int kMbarPolls = 1 << 20;  // each poll suspends for a hardware-defined interval
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int polls = kMbarPolls) {
  for (int i = 0; i < polls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// Status-word bit recorded by a kernel whose bounded wait ran out.
constexpr int kStatusWaitTimeout = 1;
// Status-word bit: a kernel found its dynamic shared memory less than
// 128-byte aligned (what its tensor copies need) and did no work.
constexpr int kStatusSmemAlign = 4;
__device__ __forceinline__ bool smem_aligned_128(const void *p, int *status) {
  if ((smem_addr(p) & 127u) == 0) return true;
  if (threadIdx.x == 0) atomicOr(status, kStatusSmemAlign);
  return false;
}

// Persistent loop over the work items w = blockIdx.x, blockIdx.x + gridDim.x,
// ... with two tile buffers: while item i is computed in one buffer, the bulk
// copies of item i+1 fill the other.  issue(w, buf, bar) starts the copies of
// item w (all threads call it; one thread posts the expected byte count);
// compute(w, buf) runs on a landed tile and must leave `buf` free for reuse
// after the block barrier that follows it.  Returns false if a wait ran out
// (the status word then holds kStatusWaitTimeout).
template <typename Issue, typename Compute>
__device__ __forceinline__ bool tile_pipeline(int nwork, float2 *buf0, float2 *buf1, uint64_t *bars, int *status,
                                              Issue issue, Compute compute) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t parity = 0;  // bit s: parity of the next phase of barrier s
  int w = blockIdx.x;
  if (w < nwork) issue(w, buf0, &bars[0]);
  for (int i = 0; w < nwork; ++i, w += gridDim.x) {
    const int s = i & 1;
    float2 *cur = s ? buf1 : buf0;
    float2 *nxt = s ? buf0 : buf1;
    const int wn = w + gridDim.x;
    if (wn < nwork) {
      fence_proxy_async_smem();  // the other buffer's last reads precede its refill
      issue(wn, nxt, &bars[s ^ 1]);
    }
    const uint32_t par = (parity >> s) & 1u;
    const bool ok = mbar_wait(&bars[s], par);
    parity ^= 1u << s;
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicOr(status, kStatusWaitTimeout);
      // give the copies still in flight one more bounded wait before leaving
      mbar_wait(&bars[s], par);
      if (wn < nwork) mbar_wait(&bars[s ^ 1], (parity >> (s ^ 1)) & 1u);
      return false;
    }
    compute(w, cur);
    __syncthreads();
  }
  return true;
}

// The same loop with NS buffers: the copies of the next NS - 1 items are in
// flight while item i is computed in buffer i mod NS (buffer b at
// buf + b * stride floats2; barrier b at bars[b]).  One block barrier per
// item: a warp computes as soon as its own wait on the item's mbarrier has
// returned (the landed bytes are then visible to it), so the warps need not
// wait for the thread that issues the next copies.  What issue() writes to
// shared memory for item w is read by compute(w) only after the barrier that
// ends the previous item (or the one after the first issues).  compute() may
// not contain block barriers.  Each wait gives up after `polls` polls.
template <int NS, typename Issue, typename Compute>
__device__ __forceinline__ bool tile_pipeline_n(int nwork, float2 *buf, size_t stride, uint64_t *bars, int *status,
                                                Issue issue, Compute compute, int polls = kMbarPolls) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    for (int b = 0; b < NS; ++b) mbar_init(&bars[b], 1);
    mbar_fence_init();
  }
  __syncthreads();
#pragma unroll 1
  for (int k = 0; k < NS - 1; ++k) {
    const int w = blockIdx.x + k * gridDim.x;
    if (w < nwork) issue(w, buf + k * stride, &bars[k]);
  }
  __syncthreads();  // what the first issues wrote to shared memory
#pragma unroll 1
  for (int i = 0;; ++i) {
    const int w = blockIdx.x + i * gridDim.x;
    if (w >= nwork) break;
    const int s = i % NS;
    const int wn = w + (NS - 1) * gridDim.x;
    if (wn < nwork) {
      const int sn = (i + NS - 1) % NS;
      fence_proxy_async_smem();  // that buffer's last reads precede its refill
      issue(wn, buf + sn * stride, &bars[sn]);
    }
    const uint32_t par = uint32_t(i / NS) & 1u;
    // warp-uniform, so that compute() keeps its shuffles whole
    const bool ok = __all_sync(0xffffffffu, mbar_wait(&bars[s], par, polls));
    if (ok) compute(w, buf + s * stride);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) atomicOr(status, kStatusWaitTimeout);
      // one more bounded wait for every copy still in flight
      for (int k = 0; k < NS; ++k) {
        const int wk = w + k * gridDim.x;
        if (wk < nwork) mbar_wait(&bars[(i + k) % NS], uint32_t((i + k) / NS) & 1u, polls);
      }
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void block_work(const int2 *__restrict__ work, int &inst, int &tile) {
  if (work) {
    int2 w = work[blockIdx.x];
    inst = w.x;
    tile = w.y;
  } else {
    inst = 0;
    tile = blockIdx.x;
  }
}

__device__ __forceinline__ int wrap(int i, int n) {
  // one conditional add or subtract in the usual case -n <= i < 2n
  if (i >= n) {
    i -= n;
    if (i >= n) i %= n;
  } else if (i < 0) {
    i += n;
    if (i < 0) {
      i %= n;
      if (i < 0) i += n;
    }
  }
  return i;
}

// ------------------------------------------------------------ host side
// Blocks of a persistent launch: as many as fit on the device at once, at
// most one per work item.
template <typename K>
static int persistent_grid(K kernel, int threads, size_t smem, int nwork) {
  int dev = 0, nsm = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
  const long long g = (long long)(per < 1 ? 1 : per) * (nsm < 1 ? 1 : nsm);
  return int(g < nwork ? g : nwork);
}

template <typename K>
static cudaError_t launch_persistent(K kernel, const Launch &L, int threads, size_t smem, int nwork) {
  if (smem > 40 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  const int grid = persistent_grid(kernel, threads, smem, nwork);
  kernel<<<grid, threads, smem, L.stream>>>(L.descs, nwork);
  return cudaGetLastError();
}

// Launch with the programmatic-stream-serialization attribute (the kernel
// must begin with griddep_enter()); an ordinary launch while the stream is
// being captured into a graph.
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int threads, size_t smem, cudaStream_t s,
                              Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(grid));
  cfg.blockDim = dim3(unsigned(threads));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 0;
  if (PA_PDL) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusActive;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess)
      (void)cudaGetLastError();  // the query's own error: launch the ordinary way
    else if (cs == cudaStreamCaptureStatusNone)
      cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Opt-in shared memory per block of the current device (read once).
static inline size_t smem_optin_limit() {
  static int v = -1;
  if (v < 0) {
    int dev = 0, x = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&x, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    v = x;
  }
  return size_t(v);
}

// launch_persistent for kernels that also take a tensor map and its flag.
template <typename K>
static cudaError_t launch_persistent_map(K kernel, const Launch &L, int threads, size_t smem, int nwork,
                                         const CUtensorMap &map, int use_map) {
  if (smem > 40 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
  }
  const int grid = persistent_grid(kernel, threads, smem, nwork);
  return launch_pdl(kernel, grid, threads, smem, L.stream, L.descs, nwork, map, use_map);
}

static inline int pow2_log(int n) {
  if (n <= 0 || (n & (n - 1))) return -1;
  int lg = 0;
  while ((1 << lg) < n) ++lg;
  return lg;
}

}  // namespace pa
