// pa_plan.cu -- host side of the NEDNER-NUFFT library: plan construction
// (Sec. 3 set-up: grid coordinates of the sensors, their window taps and
// binning, deconvolution tables, FFT schedules, time-frequency constants),
// the C ABI of include/pa_nufft.h and the batched CUDA-graph path.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <string>
#include <numeric>
#include <vector>

#include "pa_internal.h"
#include "pa_nufft.h"

using pa::FftPlan;
using pa::HornerTable;
using pa::InstDesc;
using pa::IoPtrs;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string &msg) {
  g_err = msg;
  return code;
}

#define PA_CUDA(expr)                                                                 \
  do {                                                                                \
    cudaError_t e_ = (expr);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      if (e_ == cudaErrorMemoryAllocation)                                            \
        return fail(PA_ERR_OOM, std::string(#expr) + ": " + cudaGetErrorString(e_));  \
      return fail(PA_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));   \
    }                                                                                 \
  } while (0)

constexpr double kPi = 3.14159265358979323846;

// Modified Bessel functions by their power series (all terms positive).
double bessel_i0(double z) {
  const double q = 0.25 * z * z;
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 500; ++k) {
    term *= q / (double(k) * double(k));
    sum += term;
    if (term < 1e-17 * sum) break;
  }
  return sum;
}
double bessel_i1(double z) {
  const double q = 0.25 * z * z;
  double term = 0.5 * z, sum = term;
  for (int k = 1; k < 500; ++k) {
    term *= q / (double(k) * double(k + 1));
    sum += term;
    if (std::fabs(term) < 1e-17 * std::fabs(sum)) break;
  }
  return sum;
}

// Kaiser-Bessel window of w taps for oversampling sigma, normalised so that
// phi(0) = 1; phihat is its continuous Fourier transform (same normalisation).
struct Kb {
  int w;
  double beta, phi0;
  Kb(int w_, int sigma) : w(w_) {
    const double a = double(w_) / sigma * (sigma - 0.5);
    beta = kPi * std::sqrt(a * a - 0.8);
    phi0 = bessel_i0(beta);
  }
  double phi(double x) const {
    const double t = 1.0 - (2.0 * x / w) * (2.0 * x / w);
    if (t < 0.0) return 0.0;
    return bessel_i0(beta * std::sqrt(t)) / phi0;
  }
  double dphi(double x) const {
    const double t = 1.0 - (2.0 * x / w) * (2.0 * x / w);
    if (t <= 0.0) return 0.0;
    const double s = std::sqrt(t);
    return bessel_i1(beta * s) * beta * (-4.0 * x / (double(w) * w)) / s / phi0;
  }
  double phihat(double xi) const {
    const double a = kPi * w * xi;
    const double s = beta * beta - a * a;
    const double r = std::sqrt(std::fabs(s));
    double v;
    if (s > 1e-300)
      v = w * std::sinh(r) / r;
    else if (s < -1e-300)
      v = w * std::sin(r) / r;
    else
      v = w;
    return v / phi0;
  }
};

// Depth-order stride of the adjoint NER spread: near Nz / (samples per
// warp) and prime to Nz.
int ner_lperm_for(int Nz, int cb) {
  int K = std::max(1, Nz / (32 / cb) + 1);
  while (std::gcd(K, Nz) != 1) ++K;
  return K % Nz == 0 ? 1 : K;
}

bool smooth7(long n) {
  if (n < 1) return false;
  for (int p : {2, 3, 5, 7})
    while (n % p == 0) n /= p;
  return n == 1;
}

int ipt_of(int r) { return r >= 16 ? 1 : (r >= 5 ? 2 : 4); }

// Radix schedule of an in-place Stockham FFT; every stage must fit in one
// round per sequence for `nthr` threads.
bool make_fft_plan(int L, int nthr, FftPlan &fp) {
  std::memset(&fp, 0, sizeof(fp));
  fp.L = L;
  int rem = L;
  const int order[] = {16, 8, 4, 2, 3, 5, 7};
  while (rem > 1) {
    bool found = false;
    for (int r : order) {
      if (rem % r == 0) {
        if (fp.nst >= pa::kMaxStages) return false;
        fp.radix[fp.nst++] = r;
        rem /= r;
        found = true;
        break;
      }
    }
    if (!found) return false;
  }
  for (int s = 0; s < fp.nst; ++s)
    if (L / fp.radix[s] > nthr * ipt_of(fp.radix[s])) return false;
  return true;
}

void split_ff(double v, float &hi, float &lo) {
  hi = float(v);
  lo = float(v - double(hi));
}

int horner_degree(int w) { return w <= 6 ? 7 : (w <= 8 ? 8 : (w <= 12 ? 10 : 14)); }

// Monomial coefficients in s = 2 fr - 1 of the Chebyshev interpolant of
// degree D of phi(fr + w/2 - 1 - t), fr in [0, 1], for the taps t < w/2
// (the others follow from the window's symmetry, see HornerTable).
void fit_horner(const Kb &kb, int D, HornerTable &ht) {
  std::memset(&ht, 0, sizeof(ht));
  const int w = kb.w;
  std::vector<double> nodes(D + 1), vals(D + 1);
  for (int t = 0; t < w / 2; ++t) {
    for (int k = 0; k <= D; ++k) {
      nodes[k] = std::cos(kPi * (k + 0.5) / (D + 1));
      const double fr = 0.5 * (nodes[k] + 1.0);
      vals[k] = kb.phi(fr + 0.5 * w - 1.0 - t);
    }
    // Chebyshev coefficients a_j
    std::vector<double> a(D + 1, 0.0);
    for (int j = 0; j <= D; ++j) {
      double s = 0.0;
      for (int k = 0; k <= D; ++k) s += vals[k] * std::cos(j * kPi * (k + 0.5) / (D + 1));
      a[j] = 2.0 * s / (D + 1);
    }
    a[0] *= 0.5;
    // sum_j a_j T_j(s) -> monomials, with T_{j+1} = 2 s T_j - T_{j-1}
    std::vector<double> Tm(D + 1, 0.0), T0(D + 1, 0.0), T1(D + 1, 0.0), out(D + 1, 0.0);
    T0[0] = 1.0;
    if (D >= 1) T1[1] = 1.0;
    for (int k = 0; k <= D; ++k) out[k] += a[0] * T0[k];
    if (D >= 1)
      for (int k = 0; k <= D; ++k) out[k] += a[1] * T1[k];
    for (int j = 2; j <= D; ++j) {
      std::vector<double> T2(D + 1, 0.0);
      for (int k = 0; k <= D; ++k) {
        if (k >= 1) T2[k] += 2.0 * T1[k - 1];
        T2[k] -= T0[k];
      }
      for (int k = 0; k <= D; ++k) out[k] += a[j] * T2[k];
      T0 = T1;
      T1 = T2;
    }
    for (int k = 0; k <= D; ++k) ht.set(t, k, float(out[k]));
  }
}

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

struct pa_plan {
  int device = 0;
  int64_t M = 0, Nt = 0;
  double dt = 0, c = 0;
  pa_grid grid{};
  int sigma = 2, w = 8;
  InstDesc h{};
  InstDesc *d_desc = nullptr;
  HornerTable ht{};
  char *d_static = nullptr;
  char *d_work = nullptr;
  size_t static_bytes = 0, work_bytes = 0;
  std::vector<double> weights;  // h_m
  size_t smem_limit = 0;
  // forward-spread entry lists (device), reallocated when they outgrow it
  char *d_entries = nullptr;
  size_t entries_bytes = 0;
  // device re-binning scratch (first pa_plan_update_positions_device call)
  char *d_rebin = nullptr;
  size_t rebin_bytes = 0;
  // d = 2 operator (pa_plan_create_2d): Ny = 1, My = 1, sensors at (x_m, 0)
  bool d2 = false;
  float *d_invh = nullptr;        // [M] 1/h_m in the caller's order (static buffer)
  size_t n_entries = 0;           // spread entries (sp_m / sp_w)
  // lattice path: sensors on the output lattice (see pa_plan_is_lattice)
  bool lattice_allowed = true;
  bool lattice = false;
  InstDesc hl{};                  // spatial-step descriptor at sigma = 1
  InstDesc *d_desc_lat = nullptr;
  char *d_lattice = nullptr;      // node of each sensor | h_m/(dx dy) | ones
  const int *lat_pq = nullptr;
  const float *lat_amp = nullptr;
  // optional per-stage event timing
  uint32_t profile_mask = 0;  // stages whose launches are bracketed by events
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
};

struct pa_batch {
  std::vector<pa_plan *> plans;
  InstDesc *d_descs = nullptr;
  IoPtrs *d_io = nullptr;
  int2 *d_work = nullptr;
  struct Stage {
    size_t off = 0;
    int nblocks = 0;
    size_t smem = 0;
  } st_spread, st_rowfft, st_col, st_ner, st_imgx, st_imgy;
  int spread_spl = 4;
  int ner_threads = 0;
  HornerTable ht{};
  int width = 8;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  // mode 0: every instance's own single-plan launches, as concurrent branches
  // of one CUDA graph; mode 1: one launch per stage over all instances
  int mode = 0;
  std::vector<const float *> cap_g;  // caller buffers the graph was captured with
  std::vector<float *> cap_f;
  std::vector<cudaStream_t> side;    // branch streams (mode 0)
  std::vector<cudaEvent_t> ev;       // fork + one join per branch
};

namespace {

// Sensor geometry: grid coordinates, window taps, binning; uploads into the
// plan's static buffers.
int upload_sensors(pa_plan *P, const double *xy, cudaStream_t stream) {
  const int M = int(P->M), w = P->w;
  const int Mx = P->h.Mx, My = P->h.My;
  const double X = P->grid.nx * P->grid.dx, Y = P->grid.ny * P->grid.dy;
  const Kb kb(w, P->sigma);
  std::vector<int> bx(M), by(M);
  std::vector<double> frx(M), fry(M);
  std::vector<double2> pos(M);
  for (int m = 0; m < M; ++m) {
    const double x = xy[2 * m], y = xy[2 * m + 1];
    if (!std::isfinite(x) || !std::isfinite(y)) return fail(PA_ERR_INVALID_ARG, "non-finite sensor position");
    double ux = x / X, uy = y / Y;
    ux -= std::floor(ux + 0.5);
    uy -= std::floor(uy + 0.5);
    pos[m] = make_double2(ux * X, uy * Y);
    const double Ux = Mx * ux, Uy = My * uy;
    const double fbx = std::floor(Ux), fby = std::floor(Uy);
    frx[m] = Ux - fbx;
    fry[m] = Uy - fby;
    bx[m] = ((int(fbx) % Mx) + Mx) % Mx;
    by[m] = ((int(fby) % My) + My) % My;
  }
  // counting sort by cell
  const size_t ncell = size_t(Mx) * My;
  std::vector<int> cs(ncell + 1, 0), perm(M);
  for (int m = 0; m < M; ++m) cs[size_t(bx[m]) * My + by[m] + 1]++;
  for (size_t k = 0; k < ncell; ++k) cs[k + 1] += cs[k];
  {
    std::vector<int> fill(cs.begin(), cs.end() - 1);
    for (int m = 0; m < M; ++m) perm[fill[size_t(bx[m]) * My + by[m]]++] = m;
  }
  std::vector<int> sbx(M), sby(M);
  std::vector<float> wx(size_t(M) * w), wy(size_t(M) * w), dwx(size_t(M) * w), dwy(size_t(M) * w);
  const double ax = 1.0 / (P->grid.dx * P->grid.dy);
  for (int i = 0; i < M; ++i) {
    const int m = perm[i];
    sbx[i] = bx[m];
    sby[i] = by[m];
    const double a = P->weights[m] * ax;
    for (int t = 0; t < w; ++t) {
      const double ddx = frx[m] + 0.5 * w - 1.0 - t;
      const double ddy = fry[m] + 0.5 * w - 1.0 - t;
      wx[size_t(i) * w + t] = float(kb.phi(ddx));
      dwx[size_t(i) * w + t] = float(kb.dphi(ddx) * Mx / X);
      if (P->d2) {  // no window in y: a_m in tap 0
        wy[size_t(i) * w + t] = t == 0 ? float(a) : 0.f;
        dwy[size_t(i) * w + t] = 0.f;
      } else {
        wy[size_t(i) * w + t] = float(a * kb.phi(ddy));
        dwy[size_t(i) * w + t] = float(a * kb.dphi(ddy) * My / Y);
      }
    }
  }
  PA_CUDA(cudaMemcpyAsync((void *)P->h.pos, pos.data(), sizeof(double2) * M, cudaMemcpyHostToDevice, stream));
  PA_CUDA(cudaMemcpyAsync((void *)P->h.perm, perm.data(), sizeof(int) * M, cudaMemcpyHostToDevice, stream));
  PA_CUDA(cudaMemcpyAsync((void *)P->h.sbx, sbx.data(), sizeof(int) * M, cudaMemcpyHostToDevice, stream));
  PA_CUDA(cudaMemcpyAsync((void *)P->h.sby, sby.data(), sizeof(int) * M, cudaMemcpyHostToDevice, stream));
  PA_CUDA(cudaMemcpyAsync((void *)P->h.wx, wx.data(), sizeof(float) * wx.size(), cudaMemcpyHostToDevice, stream));
  PA_CUDA(cudaMemcpyAsync((void *)P->h.wy, wy.data(), sizeof(float) * wy.size(), cudaMemcpyHostToDevice, stream));
  PA_CUDA(cudaMemcpyAsync((void *)P->h.dwx, dwx.data(), sizeof(float) * dwx.size(), cudaMemcpyHostToDevice, stream));
  PA_CUDA(cudaMemcpyAsync((void *)P->h.dwy, dwy.data(), sizeof(float) * dwy.size(), cudaMemcpyHostToDevice, stream));
  PA_CUDA(cudaMemcpyAsync((void *)P->h.cell_start, cs.data(), sizeof(int) * cs.size(), cudaMemcpyHostToDevice,
                          stream));
  PA_CUDA(pa::build_interp_pack(P->h, stream));

  // Forward-spread entries.  Strip st covers grid rows p0 = st*P .. p0+P-1;
  // a sensor contributes to (st, q) for each column q of its w-column
  // footprint when its w-row footprint meets the strip, with the tap
  // products of the strip's rows.  Candidates are the sensors whose base row
  // lies within P + w - 1 rows of the strip, taken in sorted (cell) order,
  // so every list follows the same sensor order.
  constexpr int P_ = pa::kSpreadP;
  const int nstrips = (Mx + P_ - 1) / P_;
  const int nrows = std::min(P_ + w - 1, Mx);
  auto for_each_entry = [&](auto &&fn) {
    for (int st = 0; st < nstrips; ++st) {
      const int p0 = st * P_;
      for (int dr = 0; dr < nrows; ++dr) {
        const int row = ((p0 - w / 2 + dr) % Mx + Mx) % Mx;
        for (int i = cs[size_t(row) * My]; i < cs[size_t(row) * My + My]; ++i) {
          float wxr[P_];
          bool any = false;
          for (int r = 0; r < P_; ++r) {
            const int p = p0 + r;
            const int tx = ((p - sbx[i] + w / 2 - 1) % Mx + Mx) % Mx;
            wxr[r] = (tx < w && p < Mx) ? wx[size_t(i) * w + tx] : 0.f;
            any = any || (tx < w && p < Mx);
          }
          if (!any) continue;
          const int q0 = sby[i] - w / 2 + 1;
          for (int t = 0; t < w; ++t) {
            const int q = ((q0 + t) % My + My) % My;
            fn(st, q, i, wy[size_t(i) * w + t], wxr);
          }
        }
      }
    }
  };
  std::vector<int> sp_start(size_t(nstrips) * My + 1, 0);
  for_each_entry([&](int st, int q, int, float, const float *) { sp_start[size_t(st) * My + q + 1]++; });
  for (size_t k = 0; k + 1 < sp_start.size(); ++k) sp_start[k + 1] += sp_start[k];
  const size_t nent = size_t(sp_start.back());
  P->n_entries = nent;
  std::vector<int> sp_m(nent), sp_i(nent);
  std::vector<float4> sp_w(nent);
  {
    std::vector<int> fill(sp_start.begin(), sp_start.end() - 1);
    for_each_entry([&](int st, int q, int i, float wyq, const float *wxr) {
      const size_t e = size_t(fill[size_t(st) * My + q]++);
      sp_m[e] = perm[i];
      sp_i[e] = i;
      sp_w[e] = make_float4(wyq * wxr[0], wyq * wxr[1], wyq * wxr[2], wyq * wxr[3]);
    });
  }
  // Union lists of the staged spread: per block of kSpreadQC columns of a
  // strip, the sensors of its entries in sorted order, and each entry's
  // position in its block's union.
  const int QC = pa::kSpreadQC, ncb = (My + QC - 1) / QC;
  // (sp_slot is padded so that a block's slots copy as whole 16-byte words)
  std::vector<int> sp_slot(nent + 8, 0), sp_ustart(size_t(nstrips) * ncb + 1, 0), sp_um;
  std::vector<int2> sp_erange(size_t(nstrips) * ncb);
  sp_um.reserve(nent / 4 + 16);
  // A block's union is ordered by the number of its entries that use each
  // sensor (most used first), so that when the union is longer than the rows
  // the kernel stages, the rows it reads from global memory instead serve the
  // fewest entries.  The sums run in entry order whatever the slots are.
  int umax = 0, emax = 0;
  {
    std::vector<int> uni;
    std::vector<std::pair<int, int>> cnt;  // (-uses, sensor)
    std::vector<int> slot_of(size_t(M), 0);
    for (int st = 0; st < nstrips; ++st) {
      for (int cb = 0; cb < ncb; ++cb) {
        const size_t blk = size_t(st) * ncb + cb;
        const int qa = cb * QC, qb = std::min(My, qa + QC);
        const size_t ea = size_t(sp_start[size_t(st) * My + qa]), eb = size_t(sp_start[size_t(st) * My + qb]);
        uni.assign(sp_i.begin() + ea, sp_i.begin() + eb);
        std::sort(uni.begin(), uni.end());
        cnt.clear();
        for (size_t k = 0; k < uni.size();) {
          size_t k1 = k;
          while (k1 < uni.size() && uni[k1] == uni[k]) ++k1;
          cnt.emplace_back(-int(k1 - k), uni[k]);
          k = k1;
        }
        std::sort(cnt.begin(), cnt.end());
        for (size_t k = 0; k < cnt.size(); ++k) slot_of[size_t(cnt[k].second)] = int(k);
        for (size_t e = ea; e < eb; ++e) sp_slot[e] = slot_of[size_t(sp_i[e])];
        sp_ustart[blk] = int(sp_um.size());
        sp_erange[blk] = make_int2(int(ea), int(eb));
        for (const auto &c : cnt) sp_um.push_back(perm[c.second]);
        umax = std::max(umax, int(cnt.size()));
        emax = std::max(emax, int(eb - ea));
      }
    }
    sp_ustart.back() = int(sp_um.size());
  }
  // Staged rows: every block reserves the same shared memory, so the longest
  // union would set it for all.  The rows are held to what lets
  // kSpreadTileBlocks blocks of 8-sample lanes (1 KB per row) share an SM
  // (rows past it are read from global memory), unless that leaves fewer
  // than kSpreadUrowsMin.
  {
    // (1 KB of each block's shared memory is reserved by the system)
    int dev = 0, sm_smem = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) sm_smem = 0;
    const long budget = long(sm_smem) / pa::kSpreadTileBlocks - 1024 -
                        4L * long(pa::SpreadTileEntryFloats(emax));
    const int fit = int(std::max(0L, budget) / (32 * 8 * 4));
    int cap = std::min(umax, pa::kSpreadUrowsMax);
    if (fit >= pa::kSpreadUrowsMin) cap = std::min(cap, fit);
    P->h.sp_urows = cap;
  }
  P->h.sp_emax = emax;
  size_t off = 0;
  auto place = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + std::max<size_t>(bytes, 16));
    return o;
  };
  const size_t o_ss = place(sizeof(int) * sp_start.size());
  const size_t o_sm = place(sizeof(int) * nent);
  const size_t o_sw = place(sizeof(float4) * nent);
  const size_t o_sl = place(sizeof(int) * sp_slot.size());
  const size_t o_us = place(sizeof(int) * sp_ustart.size());
  const size_t o_um = place(sizeof(int) * sp_um.size());
  const size_t o_er = place(sizeof(int2) * sp_erange.size());
  const size_t need = off;
  if (need > P->entries_bytes) {
    if (P->d_entries) {
      PA_CUDA(cudaStreamSynchronize(stream));
      cudaFree(P->d_entries);
      P->d_entries = nullptr;
      P->entries_bytes = 0;
    }
    PA_CUDA(cudaMalloc(&P->d_entries, need));
    P->entries_bytes = need;
  }
  char *V = P->d_entries;
  P->h.sp_start = reinterpret_cast<const int *>(V + o_ss);
  P->h.sp_m = reinterpret_cast<const int *>(V + o_sm);
  P->h.sp_w = reinterpret_cast<const float4 *>(V + o_sw);
  P->h.sp_slot = reinterpret_cast<const int *>(V + o_sl);
  P->h.sp_ustart = reinterpret_cast<const int *>(V + o_us);
  P->h.sp_um = reinterpret_cast<const int *>(V + o_um);
  P->h.sp_erange = reinterpret_cast<const int2 *>(V + o_er);
  auto upv = [&](const void *dst, const void *src, size_t bytes) {
    return bytes ? cudaMemcpyAsync(const_cast<void *>(dst), src, bytes, cudaMemcpyHostToDevice, stream)
                 : cudaSuccess;
  };
  PA_CUDA(upv(P->h.sp_start, sp_start.data(), sizeof(int) * sp_start.size()));
  PA_CUDA(upv(P->h.sp_m, sp_m.data(), sizeof(int) * nent));
  PA_CUDA(upv(P->h.sp_w, sp_w.data(), sizeof(float4) * nent));
  PA_CUDA(upv(P->h.sp_slot, sp_slot.data(), sizeof(int) * sp_slot.size()));
  PA_CUDA(upv(P->h.sp_ustart, sp_ustart.data(), sizeof(int) * sp_ustart.size()));
  PA_CUDA(upv(P->h.sp_um, sp_um.data(), sizeof(int) * sp_um.size()));
  PA_CUDA(upv(P->h.sp_erange, sp_erange.data(), sizeof(int2) * sp_erange.size()));
  // pageable sources: the copies above are complete when they return
  return PA_OK;
}

void free_plan(pa_plan *P) {
  if (!P) return;
  for (auto &u : P->ev_used) {
    cudaEventDestroy(u.second.first);
    cudaEventDestroy(u.second.second);
  }
  for (auto e : P->ev_pool) cudaEventDestroy(e);
  cudaFree(P->d_desc);
  cudaFree(P->d_static);
  cudaFree(P->d_work);
  cudaFree(P->d_entries);
  cudaFree(P->d_rebin);
  cudaFree(P->d_lattice);
  cudaFree(P->d_desc_lat);
  delete P;
}

pa::Launch make_launch(const pa_plan *P, cudaStream_t s) {
  pa::Launch L{};
  L.descs = P->d_desc;
  L.work = nullptr;
  L.io_table = nullptr;
  L.stream = s;
  L.host = &P->h;
  return L;
}

int check_launch(cudaError_t e, const char *what) {
  if (e != cudaSuccess) return fail(PA_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return PA_OK;
}

const char *const kStageNames[PA_PROFILE_STAGES] = {
    "ned_spread", "ned_colfft", "ner_fused", "image_x", "image_y_c2r", "image_y_adj",
    "image_x_adj", "ner_adj", "ned_colfft_adj", "ned_interp", "grad_reduce", "cubic_baseline", "ned_rowifft",
    "ned_rowfft", "lattice_scatter", "lattice_gather", "lattice_alias"};

cudaEvent_t take_event(pa_plan *P) {
  if (!P->ev_pool.empty()) {
    cudaEvent_t e = P->ev_pool.back();
    P->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Launch `fn` on stream s; with profiling on for the stage, bracket it with
// events.
template <typename Fn>
int timed(pa_plan *P, int stage, cudaStream_t s, Fn fn, const char *what) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const bool prof = (P->profile_mask >> stage) & 1u;
  if (prof) {
    e0 = take_event(P);
    e1 = take_event(P);
    if (e0) cudaEventRecord(e0, s);
  }
  int rc = check_launch(fn(), what);
  if (prof && e0 && e1) {
    cudaEventRecord(e1, s);
    P->ev_used.push_back({stage, {e0, e1}});
  }
  return rc;
}

int run_forward(pa_plan *P, const IoPtrs &io, cudaStream_t s, bool cubic) {
  pa::Launch L = make_launch(P, s);
  L.io = io;
  const InstDesc &h = P->h;
  int rc;
  if (P->d2) {
    // d = 2: 1-D spread into T, then the column FFT, NER and inverse x DFT of
    // the 3-D path on the one jy column, then the real part
    if ((rc = timed(P, 0, s, [&] { return pa::launch_spread_x(L, h); }, "spread_x")) != PA_OK) return rc;
    L.nblocks = pa::blocks_colfft(h);
    L.smem = pa::smem_colfft(h);
    if ((rc = timed(P, 1, s, [&] { return pa::launch_colfft(L, false); }, "colfft")) != PA_OK) return rc;
    L.threads = h.ner_threads;
    L.nblocks = pa::blocks_ner(h);
    L.smem = pa::smem_ner(h);
    if (cubic) {
      if ((rc = timed(P, 11, s, [&] { return pa::launch_cubic(L); }, "cubic")) != PA_OK) return rc;
    } else {
      if ((rc = timed(P, 2, s, [&] { return pa::launch_ner(L, P->w, P->ht, false); }, "ner")) != PA_OK) return rc;
    }
    L.nblocks = pa::blocks_imgx(h);
    L.smem = pa::smem_imgx(h);
    if ((rc = timed(P, 3, s, [&] { return pa::launch_imgx(L, false); }, "imgx")) != PA_OK) return rc;
    return timed(P, 4, s, [&] { return pa::launch_real_out(L, h); }, "real_out");
  }
  if (P->lattice) {
    // sensors on the lattice: place, then DFT over the lattice (sigma = 1)
    const InstDesc &hl = P->hl;
    if ((rc = timed(P, 14, s, [&] {
           return pa::launch_lattice_scatter(h.G0, P->lat_pq, P->lat_amp, io.g_in, int(P->M), h.Nt, s);
         }, "lattice_scatter")) != PA_OK)
      return rc;
    pa::Launch Ll = L;
    Ll.descs = P->d_desc_lat;
    Ll.host = &hl;
    Ll.nblocks = pa::blocks_rowfft(hl);
    Ll.smem = pa::smem_rowfft(hl);
    if ((rc = timed(P, 13, s, [&] { return pa::launch_rowfft(Ll); }, "rowfft")) != PA_OK) return rc;
    Ll.nblocks = pa::blocks_colfft(hl);
    Ll.smem = pa::smem_colfft(hl);
    if ((rc = timed(P, 1, s, [&] { return pa::launch_colfft(Ll, false); }, "colfft")) != PA_OK) return rc;
    if ((h.Nx & 1) == 0 &&
        (rc = timed(P, 16, s, [&] { return pa::launch_lattice_alias(h.G1, h.nY1, h.Nt, h.hx, 0, s); },
                    "lattice_alias")) != PA_OK)
      return rc;
  } else {
    L.nblocks = pa::blocks_spread(h, pa::spread_spl(h));
    L.smem = 0;
    if ((rc = timed(P, 0, s, [&] { return pa::launch_spread(L, pa::spread_spl(h)); }, "spread")) != PA_OK) return rc;
    L.nblocks = pa::blocks_rowfft(h);
    L.smem = pa::smem_rowfft(h);
    if ((rc = timed(P, 13, s, [&] { return pa::launch_rowfft(L); }, "rowfft")) != PA_OK) return rc;
    L.nblocks = pa::blocks_colfft(h);
    L.smem = pa::smem_colfft(h);
    if ((rc = timed(P, 1, s, [&] { return pa::launch_colfft(L, false); }, "colfft")) != PA_OK) return rc;
  }
  L.threads = h.ner_threads;
  L.nblocks = pa::blocks_ner(h);
  L.smem = pa::smem_ner(h);
  if (cubic) {
    if ((rc = timed(P, 11, s, [&] { return pa::launch_cubic(L); }, "cubic")) != PA_OK) return rc;
  } else {
    if ((rc = timed(P, 2, s, [&] { return pa::launch_ner(L, P->w, P->ht, false); }, "ner")) != PA_OK) return rc;
  }
  L.nblocks = pa::blocks_imgx(h);
  L.smem = pa::smem_imgx(h);
  if ((rc = timed(P, 3, s, [&] { return pa::launch_imgx(L, false); }, "imgx")) != PA_OK) return rc;
  L.nblocks = pa::blocks_imgy(h);
  L.smem = pa::smem_imgy(h);
  if ((rc = timed(P, 4, s, [&] { return pa::launch_imgy(L, false); }, "imgy")) != PA_OK) return rc;
  return PA_OK;
}

int run_adjoint(pa_plan *P, const IoPtrs &io, cudaStream_t s, bool grad) {
  pa::Launch L = make_launch(P, s);
  L.io = io;
  const InstDesc &h = P->h;
  int rc;
  if (P->d2) {
    if ((rc = timed(P, 5, s, [&] { return pa::launch_real_in(L, h); }, "real_in")) != PA_OK) return rc;
    L.nblocks = pa::blocks_imgx(h);
    L.smem = pa::smem_imgx(h);
    if ((rc = timed(P, 6, s, [&] { return pa::launch_imgx(L, true); }, "imgx_adj")) != PA_OK) return rc;
    L.threads = h.ner_threads;
    L.nblocks = pa::blocks_ner_adj(h);
    L.smem = pa::smem_ner(h);
    if ((rc = timed(P, 7, s, [&] { return pa::launch_ner_stage(L, P->w, P->ht, 1); }, "ner_adj")) != PA_OK) return rc;
    L.nblocks = pa::blocks_colfft(h);
    L.smem = pa::smem_colfft(h);
    if ((rc = timed(P, 8, s, [&] { return pa::launch_colfft(L, true); }, "colfft_adj")) != PA_OK) return rc;
    if ((rc = timed(P, 9, s, [&] { return pa::launch_interp_x(L, h, grad); }, "interp_x")) != PA_OK) return rc;
    if (grad) {
      L.nblocks = std::min(1024, int((P->M + 255) / 256));
      if ((rc = timed(P, 10, s, [&] { return pa::launch_grad_reduce(L, 1); }, "grad_reduce")) != PA_OK) return rc;
    }
    return PA_OK;
  }
  L.nblocks = pa::blocks_imgy(h);
  L.smem = pa::smem_imgy(h);
  if ((rc = timed(P, 5, s, [&] { return pa::launch_imgy(L, true); }, "imgy_adj")) != PA_OK) return rc;
  L.nblocks = pa::blocks_imgx(h);
  L.smem = pa::smem_imgx(h);
  if ((rc = timed(P, 6, s, [&] { return pa::launch_imgx(L, true); }, "imgx_adj")) != PA_OK) return rc;
  L.threads = h.ner_threads;
  L.nblocks = pa::blocks_ner_adj(h);
  L.smem = pa::smem_ner(h);
  if ((rc = timed(P, 7, s, [&] { return pa::launch_ner_stage(L, P->w, P->ht, 1); }, "ner_adj")) != PA_OK) return rc;

  if (P->lattice && !grad) {
    const InstDesc &hl = P->hl;
    if ((h.Nx & 1) == 0 &&
        (rc = timed(P, 16, s, [&] { return pa::launch_lattice_alias(h.G1, h.nY1, h.Nt, h.hx, 1, s); },
                    "lattice_alias")) != PA_OK)
      return rc;
    pa::Launch Ll = L;
    Ll.descs = P->d_desc_lat;
    Ll.host = &hl;
    Ll.nblocks = pa::blocks_colfft(hl);
    Ll.smem = pa::smem_colfft(hl);
    if ((rc = timed(P, 8, s, [&] { return pa::launch_colfft(Ll, true); }, "colfft_adj")) != PA_OK) return rc;
    Ll.nblocks = pa::blocks_rowifft(hl);
    Ll.smem = pa::smem_rowifft(hl);
    if ((rc = timed(P, 12, s, [&] { return pa::launch_rowifft(Ll); }, "rowifft")) != PA_OK) return rc;
    return timed(P, 15, s, [&] {
      return pa::launch_lattice_gather(io.g_out, h.G0, P->lat_pq, P->lat_amp, int(P->M), h.Nt, s);
    }, "lattice_gather");
  }

  L.nblocks = pa::blocks_colfft(h);
  L.smem = pa::smem_colfft(h);
  if ((rc = timed(P, 8, s, [&] { return pa::launch_colfft(L, true); }, "colfft_adj")) != PA_OK) return rc;
  L.nblocks = pa::blocks_rowifft(h);
  L.smem = pa::smem_rowifft(h);
  if ((rc = timed(P, 12, s, [&] { return pa::launch_rowifft(L); }, "rowifft")) != PA_OK) return rc;
  L.nblocks = pa::blocks_interp(h);
  L.smem = pa::smem_interp(h);
  if ((rc = timed(P, 9, s, [&] { return pa::launch_interp_width(L, P->w, grad, h.interp_ty); }, "interp")) != PA_OK)
    return rc;
  if (grad) {
    L.nblocks = std::min(1024, int((P->M + 255) / 256));
    if ((rc = timed(P, 10, s, [&] { return pa::launch_grad_reduce(L, 1); }, "grad_reduce")) != PA_OK) return rc;
  }
  return PA_OK;
}

}  // namespace

namespace pa {
int plan_view(const pa_plan *P, PlanView *v) {
  if (!P || !v) return PA_ERR_INVALID_ARG;
  v->h = &P->h;
  v->width = P->w;
  v->ht = &P->ht;
  v->device = P->device;
  v->n_sensors = P->M;
  v->dims = P->d2 ? 2 : 3;
  return PA_OK;
}
int set_error(int code, const char *msg) { return fail(code, msg ? msg : ""); }
}  // namespace pa

namespace {
// Deterministic values in [-1, 1) for the autotuner's input.
__global__ void k_fill_pattern(float *x, size_t n, uint32_t seed) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    uint32_t v = uint32_t(i) * 2654435761u ^ seed;
    v ^= v >> 16;
    v *= 2246822519u;
    v ^= v >> 13;
    x[i] = float(v & 0xffffffu) * (2.0f / 16777216.0f) - 1.0f;
  }
}

// Median device time of `reps` calls of fn (after two untimed calls).
template <typename Fn>
int median_ms(cudaStream_t s, int reps, Fn fn, float *ms) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PA_CUDA(cudaEventCreate(&e0));
  PA_CUDA(cudaEventCreate(&e1));
  std::vector<float> t;
  int rc = PA_OK;
  for (int k = 0; k < reps + 2 && rc == PA_OK; ++k) {
    cudaEventRecord(e0, s);
    rc = fn();
    cudaEventRecord(e1, s);
    if (rc == PA_OK && cudaEventSynchronize(e1) == cudaSuccess && k >= 2) {
      float v = 0.f;
      cudaEventElapsedTime(&v, e0, e1);
      t.push_back(v);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != PA_OK) return rc;
  std::sort(t.begin(), t.end());
  *ms = t.empty() ? 0.f : t[t.size() / 2];
  return PA_OK;
}
}  // namespace

namespace {
// Sensors exactly on the output lattice, one per node: node index p*ny + q
// of each sensor on the sigma = 1 grid (p = i - floor(nx/2) mod nx for
// x = (i - floor(nx/2)) dx after the reduction modulo X; q likewise).
bool lattice_nodes(const pa_plan *P, const double *xy, std::vector<int> &pq) {
  const int nx = P->grid.nx, ny = P->grid.ny;
  if (P->M != int64_t(nx) * ny) return false;
  const double X = nx * P->grid.dx, Y = ny * P->grid.dy;
  std::vector<char> seen(size_t(P->M), 0);
  pq.assign(size_t(P->M), 0);
  for (int64_t m = 0; m < P->M; ++m) {
    double ux = xy[2 * m] / X, uy = xy[2 * m + 1] / Y;
    ux -= std::floor(ux + 0.5);
    uy -= std::floor(uy + 0.5);
    const double fi = ux * nx, fk = uy * ny;
    const double ri = std::nearbyint(fi), rk = std::nearbyint(fk);
    if (std::fabs(fi - ri) > 1e-9 || std::fabs(fk - rk) > 1e-9) return false;
    const int p = ((int(ri) % nx) + nx) % nx, q = ((int(rk) % ny) + ny) % ny;
    const size_t k = size_t(p) * ny + q;
    if (seen[k]) return false;
    seen[k] = 1;
    pq[size_t(m)] = int(k);
  }
  return true;
}

// Decide and set up the lattice path for host positions xy.
int setup_lattice(pa_plan *P, const double *xy, cudaStream_t s) {
  std::vector<int> pq;
  P->lattice = P->lattice_allowed && lattice_nodes(P, xy, pq);
  if (!P->lattice) return PA_OK;
  const InstDesc &h = P->h;
  const size_t M = size_t(P->M), nones = size_t(std::max(h.nX1, h.nY1));
  const size_t o_pq = 0, o_amp = align_up(sizeof(int) * M), o_one = o_amp + align_up(sizeof(float) * M);
  if (!P->d_lattice) PA_CUDA(cudaMalloc(&P->d_lattice, o_one + sizeof(float) * nones));
  if (!P->d_desc_lat) PA_CUDA(cudaMalloc(&P->d_desc_lat, sizeof(InstDesc)));
  std::vector<float> amp(M), ones(nones, 1.0f);
  const double ax = 1.0 / (P->grid.dx * P->grid.dy);
  for (size_t m = 0; m < M; ++m) amp[m] = float(P->weights[m] * ax);
  char *D = P->d_lattice;
  PA_CUDA(cudaMemcpyAsync(D + o_pq, pq.data(), sizeof(int) * M, cudaMemcpyHostToDevice, s));
  PA_CUDA(cudaMemcpyAsync(D + o_amp, amp.data(), sizeof(float) * M, cudaMemcpyHostToDevice, s));
  PA_CUDA(cudaMemcpyAsync(D + o_one, ones.data(), sizeof(float) * nones, cudaMemcpyHostToDevice, s));
  P->lat_pq = reinterpret_cast<const int *>(D + o_pq);
  P->lat_amp = reinterpret_cast<const float *>(D + o_amp);
  const float *one = reinterpret_cast<const float *>(D + o_one);
  InstDesc &hl = P->hl;
  hl = h;
  hl.Mx = h.Nx;
  hl.My = h.Ny;
  hl.fMx = h.fNx;
  hl.fMy = h.fNy;
  hl.invphx = one;
  hl.invphy = one;
  hl.nX1 = h.Nx;  // the row of +nx/2 (even nx) is the bin of -nx/2: see launch_lattice_alias
  // pageable source: consumed when the call returns
  PA_CUDA(cudaMemcpyAsync(P->d_desc_lat, &hl, sizeof(InstDesc), cudaMemcpyHostToDevice, s));
  return PA_OK;
}
}  // namespace

extern "C" {

const char *pa_last_error(void) { return g_err.c_str(); }

const char *pa_version(void) { return "pa_nufft 0.1 (sm_103a)"; }

namespace {
// Plan creation for d = 3 and (d2: Ny = 1, no oversampling or window in y,
// sensors at (x_m, 0)) for d = 2.
int create_plan(pa_plan **out, int64_t n_sensors, const double *sensor_xy, const double *weights, int64_t n_t,
                double dt, double c, const pa_grid *grid, int sigma, int width, int flags, void *stream, bool d2) {
  if (!out) return fail(PA_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!sensor_xy || !grid) return fail(PA_ERR_INVALID_ARG, "sensor_xy or grid is NULL");
  if (n_sensors < 1 || n_sensors > (int64_t(1) << 30)) return fail(PA_ERR_INVALID_ARG, "n_sensors out of range");
  if (n_t < 2 || n_t > 4096) return fail(PA_ERR_INVALID_ARG, "n_t out of range [2, 4096]");
  if (!(dt > 0) || !std::isfinite(dt)) return fail(PA_ERR_INVALID_ARG, "dt must be finite and > 0");
  if (!(c > 0) || !std::isfinite(c)) return fail(PA_ERR_INVALID_ARG, "c must be finite and > 0");
  if (grid->nx < 2 || (!d2 && grid->ny < 2) || grid->nz < 2) return fail(PA_ERR_INVALID_ARG, "grid sizes must be >= 2");
  if (!(grid->dx > 0) || !(grid->dy > 0) || !(grid->dz > 0) || !std::isfinite(grid->dx) ||
      !std::isfinite(grid->dy) || !std::isfinite(grid->dz))
    return fail(PA_ERR_INVALID_ARG, "grid spacings must be finite and > 0");
  if (sigma < 2 || sigma > 4) return fail(PA_ERR_INVALID_ARG, "sigma must be 2, 3 or 4");
  if (!(width == 6 || width == 8 || width == 12 || width == 16))
    return fail(PA_ERR_INVALID_ARG, "width must be 6, 8, 12 or 16");
  if ((flags & ~(PA_FLAG_NO_LATTICE | PA_FLAG_BLOCK_NER)) != 0) return fail(PA_ERR_INVALID_ARG, "unknown flags");
  for (int64_t m = 0; m < 2 * n_sensors; ++m)
    if (!std::isfinite(sensor_xy[m])) return fail(PA_ERR_INVALID_ARG, "non-finite sensor position");
  const double X = grid->nx * grid->dx, Y = grid->ny * grid->dy;
  if (weights) {
    for (int64_t m = 0; m < n_sensors; ++m)
      if (!(weights[m] > 0) || !std::isfinite(weights[m]))
        return fail(PA_ERR_INVALID_ARG, "weights must be finite and > 0");
  }
  const long Nx = grid->nx, Ny = grid->ny, Nz = grid->nz, Nt = n_t;
  const long Mx = sigma * Nx, My = d2 ? 1 : sigma * Ny, Mt = sigma * Nt;
  for (long L : {Nx, Ny, Nz, Nt, Mx, My, Mt})
    if (!smooth7(L)) return fail(PA_ERR_UNSUPPORTED_SIZE, "a transform length is not a product of 2, 3, 5, 7");
  if (Mx > 4096 || My > 512 || Nz > 4096 || Nx > 4096 || Ny > 4096 || Mt > 4096)
    return fail(PA_ERR_UNSUPPORTED_SIZE, "a transform length exceeds the supported maximum");
  if (Mx < 2 * width || (!d2 && My < 2 * width))
    return fail(PA_ERR_UNSUPPORTED_SIZE, "sigma*nx and sigma*ny must be >= 2*width");

  pa_plan *P = new pa_plan();
  P->d2 = d2;
  P->M = n_sensors;
  P->Nt = n_t;
  P->dt = dt;
  P->c = c;
  P->grid = *grid;
  P->sigma = sigma;
  P->w = width;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t ce = cudaGetDevice(&P->device);
  if (ce != cudaSuccess) {
    delete P;
    return fail(PA_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ce));
  }
  int smem_optin = 0;
  cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device);
  P->smem_limit = size_t(smem_optin);
  P->weights.resize(n_sensors);
  for (int64_t m = 0; m < n_sensors; ++m) P->weights[m] = weights ? weights[m] : X * Y / double(n_sensors);

  InstDesc &h = P->h;
  std::memset(&h, 0, sizeof(h));
  h.M = int(n_sensors);
  h.Nt = int(Nt);
  h.Nx = int(Nx);
  h.Ny = int(Ny);
  h.Nz = int(Nz);
  h.Mx = int(Mx);
  h.My = int(My);
  h.Mt = int(Mt);
  h.w = width;
  h.hx = int(Nx / 2);
  h.hy = int(Ny / 2);
  h.hz = int(Nz / 2);
  h.nc = int(Nt / 2);
  h.nX1 = 2 * h.hx + 1;
  h.nY1 = h.hy + 1;
  h.nchunk_adj = int((Nt + pa::kInterpNC - 1) / pa::kInterpNC);
  h.sigma = sigma;

  // NER block size: the smallest for which the column transforms have an
  // in-place schedule
  h.ner_threads = 0;
  for (int nt : {128, 256}) {
    FftPlan a, b, c;
    if (make_fft_plan(int(Mt), nt, a) && make_fft_plan(int(Nz), nt, b) && make_fft_plan(int(Nt), nt, c)) {
      h.ner_threads = nt;
      break;
    }
  }
  if (h.ner_threads == 0) {
    delete P;
    return fail(PA_ERR_UNSUPPORTED_SIZE, "time or depth transform too long for one block");
  }

  // FFT schedules and twiddles
  struct Len {
    FftPlan *fp;
    int L;
    int nthr;
  } lens[] = {{&h.fMy, int(My), 256},
              {&h.fMx, int(Mx), 256},
              {&h.fMt, int(Mt), h.ner_threads},
              {&h.fNz, int(Nz), h.ner_threads},
              {&h.fNx, int(Nx), 256},
              {&h.fNy, int(Ny), 256},
              {&h.fNt, int(Nt), h.ner_threads}};
  std::vector<float2> tw;
  for (auto &ln : lens) {
    if (!make_fft_plan(ln.L, ln.nthr, *ln.fp)) {
      delete P;
      return fail(PA_ERR_UNSUPPORTED_SIZE, "no in-place FFT schedule for length " + std::to_string(ln.L));
    }
    ln.fp->tw = int(tw.size());
    for (int m = 0; m < ln.L; ++m) {
      const double a = -2.0 * kPi * double(m) / ln.L;
      tw.push_back(make_float2(float(std::cos(a)), float(std::sin(a))));
    }
  }
  // warp-transform twiddles (FP64, rounded once)
  h.wtw = int(tw.size());
  for (int lgn = 8; lgn <= 10; ++lgn) {
    const int N = 1 << lgn;
    for (int k2 = 0; k2 < N / 32; ++k2)
      for (int n1 = 0; n1 < 32; ++n1) {
        const double a = -2.0 * kPi * double(n1 * k2) / N;
        tw.push_back(make_float2(float(std::cos(a)), float(std::sin(a))));
      }
  }
  for (int lgm = 9; lgm <= 11; ++lgm) {
    const int M = 1 << lgm;
    for (int j = 0; j < M; ++j) {
      const double a = -2.0 * kPi * double(j) / M;
      tw.push_back(make_float2(float(std::cos(a)), float(std::sin(a))));
    }
  }
  // NER blocks: ner_cb (column, source) transforms side by side, at least
  // two (the two transforms of a Nyquist column share a block); four when
  // their buffers stay within 48 KB
  h.ner_cb = 4;
  if (pa::smem_ner(h) > 48 * 1024) h.ner_cb = 2;
  // launch shapes before any tuning (pa_plan_autotune measures the others)
  h.spread_spl = Nt > 128 ? 8 : 4;
  h.interp_ty = 16;  // measured fastest at 128x128x256 and 256x256x512 (pa_plan_autotune may change it)
  h.ner_lperm = ner_lperm_for(h.Nz, h.ner_cb);

  // deconvolution tables and time-frequency constants
  const Kb kb(width, sigma);
  std::vector<float> ipx(h.nX1), ipy(h.nY1), ipt(Nt);
  for (int ix = 0; ix < h.nX1; ++ix) ipx[ix] = float(1.0 / kb.phihat(double(ix - h.hx) / Mx));
  for (int iy = 0; iy < h.nY1; ++iy) ipy[iy] = d2 ? 1.f : float(1.0 / kb.phihat(double(iy) / My));
  for (long n = 0; n < Nt; ++n) ipt[n] = float(1.0 / kb.phihat(double(n - h.nc) / Mt));
  const double Z = Nz * grid->dz;
  const double cT = c * Nt * dt;
  split_ff((cT / X) * (cT / X), h.ax_hi, h.ax_lo);
  split_ff((cT / Y) * (cT / Y), h.ay_hi, h.ay_lo);
  split_ff((cT / Z) * (cT / Z), h.az_hi, h.az_lo);
  split_ff(double(h.nc) / double(Nt), h.ph_hi, h.ph_lo);
  h.sqrt_az = float(cT / Z);
  h.two_c = float(2.0 * c);
  h.scale = float(dt / (grid->dz * double(Nx) * double(Ny) * double(Nz)));
  fit_horner(kb, horner_degree(width), P->ht);

  h.ner_warp = (flags & PA_FLAG_BLOCK_NER) == 0 && pa::ner_warp_eligible(h) &&
               pa::smem_ner_warp(h) <= P->smem_limit ? 1 : 0;

  // shared-memory limits
  const size_t smems[] = {pa::smem_rowfft(h), pa::smem_colfft(h), pa::smem_ner(h),
                          pa::smem_rowifft(h), pa::smem_imgx(h), pa::smem_imgy(h), pa::smem_interp(h)};
  for (size_t sm : smems)
    if (sm > P->smem_limit) {
      delete P;
      return fail(PA_ERR_UNSUPPORTED_SIZE, "problem needs more shared memory per block than the device has");
    }

  // static device memory
  const size_t M = size_t(n_sensors), W = size_t(width);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  const size_t o_perm = take(sizeof(int) * M), o_sbx = take(sizeof(int) * M), o_sby = take(sizeof(int) * M);
  const size_t o_wx = take(sizeof(float) * M * W), o_wy = take(sizeof(float) * M * W);
  const size_t o_dwx = take(sizeof(float) * M * W), o_dwy = take(sizeof(float) * M * W);
  const size_t o_cs = take(sizeof(int) * (size_t(Mx) * My + 1));
  const size_t o_invh = take(sizeof(float) * M);
  const size_t o_pos = take(sizeof(double2) * M);
  const size_t o_ipk = take(sizeof(float) * M * pa::ipack_words(width));
  const size_t o_ipkd = take(sizeof(float) * M * pa::ipackd_words(width));
  const size_t o_ipx = take(sizeof(float) * ipx.size()), o_ipy = take(sizeof(float) * ipy.size());
  const size_t o_ipt = take(sizeof(float) * ipt.size());
  const size_t o_tw = take(sizeof(float2) * tw.size());
  const size_t o_status = take(sizeof(int));
  P->static_bytes = off;
  // workspace
  off = 0;
  const size_t nG1 = size_t(h.nX1) * h.nY1 * Nt;
  const size_t nT = size_t(Mx) * h.nY1 * Nt;
  const size_t nF = size_t(Nx) * h.nY1 * Nz;
  const size_t o_G1 = take(sizeof(float2) * nG1);
  const size_t o_reg = take(sizeof(float2) * std::max(nT, 2 * nF));
  const size_t o_gp = take(sizeof(float2) * size_t(h.nchunk_adj) * M);
  const size_t o_G0 = take(sizeof(float) * size_t(Mx) * My * Nt);
  P->work_bytes = off;

  ce = cudaMalloc(&P->d_static, P->static_bytes);
  if (ce == cudaSuccess) ce = cudaMalloc(&P->d_work, P->work_bytes);
  if (ce == cudaSuccess) ce = cudaMalloc(&P->d_desc, sizeof(InstDesc));
  if (ce != cudaSuccess) {
    free_plan(P);
    return fail(ce == cudaErrorMemoryAllocation ? PA_ERR_OOM : PA_ERR_CUDA,
                std::string("cudaMalloc: ") + cudaGetErrorString(ce));
  }
  char *S = P->d_static;
  char *Wk = P->d_work;
  h.perm = reinterpret_cast<const int *>(S + o_perm);
  h.sbx = reinterpret_cast<const int *>(S + o_sbx);
  h.sby = reinterpret_cast<const int *>(S + o_sby);
  h.wx = reinterpret_cast<const float *>(S + o_wx);
  h.wy = reinterpret_cast<const float *>(S + o_wy);
  h.dwx = reinterpret_cast<const float *>(S + o_dwx);
  h.dwy = reinterpret_cast<const float *>(S + o_dwy);
  h.cell_start = reinterpret_cast<const int *>(S + o_cs);
  P->d_invh = reinterpret_cast<float *>(S + o_invh);
  h.pos = reinterpret_cast<const double2 *>(S + o_pos);
  h.ipack = reinterpret_cast<const float4 *>(S + o_ipk);
  h.ipack_d = reinterpret_cast<const float4 *>(S + o_ipkd);
  h.invphx = reinterpret_cast<const float *>(S + o_ipx);
  h.invphy = reinterpret_cast<const float *>(S + o_ipy);
  h.invpht = reinterpret_cast<const float *>(S + o_ipt);
  h.tw = reinterpret_cast<const float2 *>(S + o_tw);
  h.status = reinterpret_cast<int *>(S + o_status);
  h.G1 = reinterpret_cast<float2 *>(Wk + o_G1);
  h.T = reinterpret_cast<float2 *>(Wk + o_reg);
  h.Fz = reinterpret_cast<float2 *>(Wk + o_reg);
  h.U = h.Fz + nF;
  h.grad_part = reinterpret_cast<float2 *>(Wk + o_gp);
  h.G0 = reinterpret_cast<float *>(Wk + o_G0);

  int rc = upload_sensors(P, sensor_xy, s);
  if (rc == PA_OK) {
    P->lattice_allowed = !d2 && (flags & PA_FLAG_NO_LATTICE) == 0;
    rc = setup_lattice(P, sensor_xy, s);
  }
  if (rc != PA_OK) {
    free_plan(P);
    return rc;
  }
  auto up = [&](const void *dst, const void *src, size_t bytes) {
    return cudaMemcpyAsync(const_cast<void *>(dst), src, bytes, cudaMemcpyHostToDevice, s);
  };
  std::vector<float> invh(static_cast<size_t>(n_sensors));
  for (int64_t m = 0; m < n_sensors; ++m) invh[size_t(m)] = float(1.0 / P->weights[size_t(m)]);
  ce = up(P->d_invh, invh.data(), sizeof(float) * invh.size());
  if (ce == cudaSuccess) ce = up(h.invphx, ipx.data(), sizeof(float) * ipx.size());
  if (ce == cudaSuccess) ce = up(h.invphy, ipy.data(), sizeof(float) * ipy.size());
  if (ce == cudaSuccess) ce = up(h.invpht, ipt.data(), sizeof(float) * ipt.size());
  if (ce == cudaSuccess) ce = up(h.tw, tw.data(), sizeof(float2) * tw.size());
  if (ce == cudaSuccess) ce = cudaMemsetAsync(h.status, 0, sizeof(int), s);
  if (ce == cudaSuccess) ce = up(P->d_desc, &h, sizeof(InstDesc));
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) {
    free_plan(P);
    return fail(PA_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(ce));
  }
  *out = P;
  return PA_OK;
}
}  // namespace

int pa_plan_create(pa_plan **out, int64_t n_sensors, const double *sensor_xy, const double *weights, int64_t n_t,
                   double dt, double c, const pa_grid *grid, int sigma, int width, int flags, void *stream) {
  g_err.clear();
  return create_plan(out, n_sensors, sensor_xy, weights, n_t, dt, c, grid, sigma, width, flags, stream, false);
}

int pa_plan_create_2d(pa_plan **out, int64_t n_sensors, const double *sensor_x, const double *weights, int64_t n_t,
                      double dt, double c, const pa_grid2 *grid, int sigma, int width, int flags, void *stream) {
  g_err.clear();
  if (out) *out = nullptr;
  if (!sensor_x || !grid) return fail(PA_ERR_INVALID_ARG, "sensor_x or grid is NULL");
  if (n_sensors < 1 || n_sensors > (int64_t(1) << 30)) return fail(PA_ERR_INVALID_ARG, "n_sensors out of range");
  if ((flags & PA_FLAG_NO_LATTICE) != 0) return fail(PA_ERR_INVALID_ARG, "unknown flags");
  // the 3-D plan with one y row of unit spacing: h_m/(dx dy) = h_m/dx and
  // 1/(nx ny nz) = 1/(nx nz)
  std::vector<double> xy(size_t(2 * n_sensors));
  for (int64_t m = 0; m < n_sensors; ++m) {
    xy[size_t(2 * m)] = sensor_x[m];
    xy[size_t(2 * m + 1)] = 0.0;
  }
  const pa_grid g3{grid->nx, 1, grid->nz, grid->dx, 1.0, grid->dz};
  return create_plan(out, n_sensors, xy.data(), weights, n_t, dt, c, &g3, sigma, width, flags, stream, true);
}

int pa_plan_dims(const pa_plan *plan, int *d) {
  g_err.clear();
  if (!plan || !d) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  *d = plan->d2 ? 2 : 3;
  return PA_OK;
}

int pa_plan_update_positions(pa_plan *plan, const double *sensor_xy, void *stream) {
  g_err.clear();
  if (!plan || !sensor_xy) return fail(PA_ERR_INVALID_ARG, "plan or sensor_xy is NULL");
  if (plan->d2) return fail(PA_ERR_INVALID_ARG, "not supported for 2-D plans");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int rc = upload_sensors(plan, sensor_xy, s);
  if (rc != PA_OK) return rc;
  // the spread entry lists may have moved: refresh the device descriptor
  PA_CUDA(cudaMemcpyAsync(plan->d_desc, &plan->h, sizeof(InstDesc), cudaMemcpyHostToDevice, s));
  return setup_lattice(plan, sensor_xy, s);
}

int pa_plan_update_positions_device(pa_plan *plan, const float *xy_dev, void *stream) {
  g_err.clear();
  if (!plan || !xy_dev) return fail(PA_ERR_INVALID_ARG, "plan or xy_dev is NULL");
  if (plan->d2) return fail(PA_ERR_INVALID_ARG, "not supported for 2-D plans");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  pa_plan *P = plan;
  P->lattice = false;  // positions on the device are not tested for the lattice
  InstDesc &h = P->h;
  const int M = int(P->M), Mx = h.Mx, My = h.My, w = P->w;
  const int nstrips = (Mx + pa::kSpreadP - 1) / pa::kSpreadP;
  const size_t ncell = size_t(Mx) * My, nkeys = size_t(nstrips) * My;
  // scratch: weights, bx, by, frx, fry, counters, entry counts
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + std::max<size_t>(bytes, 16));
    return o;
  };
  const size_t o_w = take(sizeof(double) * M), o_bx = take(sizeof(int) * M), o_by = take(sizeof(int) * M);
  const size_t o_fx = take(sizeof(double) * M), o_fy = take(sizeof(double) * M);
  const size_t o_fill = take(sizeof(int) * std::max(ncell, nkeys)), o_cnt = take(sizeof(int) * (nkeys + 1));
  if (!P->d_rebin) {
    PA_CUDA(cudaMalloc(&P->d_rebin, off));
    P->rebin_bytes = off;
    PA_CUDA(cudaMemcpyAsync(P->d_rebin + o_w, P->weights.data(), sizeof(double) * M, cudaMemcpyHostToDevice, s));
  }
  char *R = P->d_rebin;
  const Kb kb(w, P->sigma);
  pa::RebinArgs a{};
  a.M = M;
  a.Mx = Mx;
  a.My = My;
  a.w = w;
  a.nstrips = nstrips;
  a.X = P->grid.nx * P->grid.dx;
  a.Y = P->grid.ny * P->grid.dy;
  a.ax = 1.0 / (P->grid.dx * P->grid.dy);
  a.beta = kb.beta;
  a.phi0 = kb.phi0;
  a.xy = xy_dev;
  a.pos = const_cast<double2 *>(h.pos);
  a.weights = reinterpret_cast<const double *>(R + o_w);
  a.status = h.status;
  a.perm = const_cast<int *>(h.perm);
  a.sbx = const_cast<int *>(h.sbx);
  a.sby = const_cast<int *>(h.sby);
  a.cell_start = const_cast<int *>(h.cell_start);
  a.wx = const_cast<float *>(h.wx);
  a.wy = const_cast<float *>(h.wy);
  a.dwx = const_cast<float *>(h.dwx);
  a.dwy = const_cast<float *>(h.dwy);
  a.bx = reinterpret_cast<int *>(R + o_bx);
  a.by = reinterpret_cast<int *>(R + o_by);
  a.frx = reinterpret_cast<double *>(R + o_fx);
  a.fry = reinterpret_cast<double *>(R + o_fy);
  a.fill = reinterpret_cast<int *>(R + o_fill);
  a.sp_cnt = reinterpret_cast<int *>(R + o_cnt);
  int st0 = 0;
  PA_CUDA(cudaMemcpyAsync(&st0, h.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  PA_CUDA(pa::rebin_sensors(a, s));
  PA_CUDA(pa::build_interp_pack(h, s));
  PA_CUDA(pa::rebin_count_entries(a, s));
  int nent = 0, st1 = 0;
  PA_CUDA(cudaMemcpyAsync(&nent, a.sp_cnt + nkeys, sizeof(int), cudaMemcpyDeviceToHost, s));
  PA_CUDA(cudaMemcpyAsync(&st1, h.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  PA_CUDA(cudaStreamSynchronize(s));
  if ((st1 & pa::kStatusBadPositions) && !(st0 & pa::kStatusBadPositions)) {
    int clear = st0;
    PA_CUDA(cudaMemcpy(h.status, &clear, sizeof(int), cudaMemcpyHostToDevice));
    return fail(PA_ERR_INVALID_ARG, "non-finite sensor position");
  }
  P->n_entries = size_t(nent);
  // entry lists: [sp_start | sp_m | sp_w | order keys]
  size_t eo = 0;
  auto place = [&](size_t bytes) {
    const size_t o = eo;
    eo = align_up(eo + std::max<size_t>(bytes, 16));
    return o;
  };
  const size_t o_ss = place(sizeof(int) * (nkeys + 1)), o_sm = place(sizeof(int) * size_t(nent));
  const size_t o_sw = place(sizeof(float4) * size_t(nent)), o_sk = place(sizeof(long long) * size_t(nent));
  if (eo > P->entries_bytes) {
    cudaFree(P->d_entries);
    P->d_entries = nullptr;
    P->entries_bytes = 0;
    PA_CUDA(cudaMalloc(&P->d_entries, eo));
    P->entries_bytes = eo;
  }
  char *V = P->d_entries;
  a.sp_m = reinterpret_cast<int *>(V + o_sm);
  a.sp_w = reinterpret_cast<float4 *>(V + o_sw);
  a.sp_key = reinterpret_cast<long long *>(V + o_sk);
  PA_CUDA(pa::rebin_fill_entries(a, s));
  PA_CUDA(cudaMemcpyAsync(V + o_ss, a.sp_cnt, sizeof(int) * (nkeys + 1), cudaMemcpyDeviceToDevice, s));
  h.sp_start = reinterpret_cast<const int *>(V + o_ss);
  h.sp_m = a.sp_m;
  h.sp_w = a.sp_w;
  // the staged spread's union lists are built on the host only
  h.sp_slot = h.sp_ustart = h.sp_um = nullptr;
  h.sp_erange = nullptr;
  h.sp_urows = h.sp_emax = 0;
  // pageable source: the copy has consumed the descriptor when it returns
  PA_CUDA(cudaMemcpyAsync(P->d_desc, &h, sizeof(InstDesc), cudaMemcpyHostToDevice, s));
  return PA_OK;
}

int pa_plan_autotune(pa_plan *plan, void *stream, int *choice) {
  g_err.clear();
  if (!plan) return fail(PA_ERR_INVALID_ARG, "plan is NULL");
  if (plan->d2) return fail(PA_ERR_INVALID_ARG, "not supported for 2-D plans");
  pa_plan *P = plan;
  InstDesc &h = P->h;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t ng = size_t(P->M) * size_t(P->Nt), nf = size_t(h.Nx) * h.Ny * h.Nz;
  float *g = nullptr, *f = nullptr;
  if (cudaMalloc(&g, sizeof(float) * ng) != cudaSuccess || cudaMalloc(&f, sizeof(float) * nf) != cudaSuccess) {
    cudaFree(g);
    return fail(PA_ERR_OOM, "autotune: no room for the test input");
  }
  int rc = PA_OK;
  const int ner_threads_min = h.ner_threads;
  auto upload = [&]() { return check_launch(cudaMemcpyAsync(P->d_desc, &h, sizeof(InstDesc), cudaMemcpyHostToDevice, s), "descriptor"); };
  IoPtrs io{};
  io.g_in = g;
  io.f_out = f;
  io.f_in = f;
  io.g_out = g;
  do {
    k_fill_pattern<<<1024, 256, 0, s>>>(g, ng, 1501u);
    k_fill_pattern<<<1024, 256, 0, s>>>(f, nf, 2u);
    if ((rc = check_launch(cudaGetLastError(), "autotune fill")) != PA_OK) break;
    // one forward + adjoint so that every intermediate holds realistic values
    IoPtrs fw{};
    fw.g_in = g;
    fw.f_out = f;
    if ((rc = run_forward(P, fw, s, false)) != PA_OK) break;
    if ((rc = run_adjoint(P, io, s, false)) != PA_OK) break;

    pa::Launch L = make_launch(P, s);
    L.io = io;
    // spread: samples per lane
    {
      float best = 1e30f;
      int pick = h.spread_spl;
      for (int spl : {4, 8}) {
        float ms = 0.f;
        L.nblocks = pa::blocks_spread(h, spl);
        L.smem = 0;
        if ((rc = median_ms(s, 5, [&] { return check_launch(pa::launch_spread(L, spl), "spread"); }, &ms)) != PA_OK) break;
        if (ms < best) {
          best = ms;
          pick = spl;
        }
      }
      if (rc != PA_OK) break;
      h.spread_spl = pick;
    }
    // NER: columns per block and block size (forward + adjoint) of the
    // block kernels; the warp-per-column kernels have one shape
    if (!h.ner_warp) {
      float best = 1e30f;
      int pick_cb = h.ner_cb, pick_t = h.ner_threads;
      for (int cb : {2, 4})
        for (int thr : {128, 256}) {
          if (thr < ner_threads_min) continue;
          h.ner_cb = cb;
          h.ner_threads = thr;
          h.ner_lperm = ner_lperm_for(h.Nz, cb);
          if (pa::smem_ner(h) > P->smem_limit) continue;
          if ((rc = upload()) != PA_OK) break;
          // forward repetitions first (G1 fixed), then adjoint ones (Fz fixed)
          float ms_f = 0.f, ms_a = 0.f;
          L.threads = thr;
          L.smem = pa::smem_ner(h);
          L.nblocks = pa::blocks_ner(h);
          rc = median_ms(s, 5, [&] { return check_launch(pa::launch_ner_stage(L, P->w, P->ht, 0), "ner"); }, &ms_f);
          if (rc != PA_OK) break;
          L.nblocks = pa::blocks_ner_adj(h);
          rc = median_ms(s, 5, [&] { return check_launch(pa::launch_ner_stage(L, P->w, P->ht, 1), "ner_adj"); },
                         &ms_a);
          if (rc != PA_OK) break;
          const float ms = ms_f + ms_a;
          if (ms < best) {
            best = ms;
            pick_cb = cb;
            pick_t = thr;
          }
        }
      if (rc != PA_OK) break;
      h.ner_cb = pick_cb;
      h.ner_threads = pick_t;
      h.ner_lperm = ner_lperm_for(h.Nz, pick_cb);
      if ((rc = upload()) != PA_OK) break;
    }
    // interpolation: tile height
    {
      float best = 1e30f;
      int pick = h.interp_ty;
      for (int ty : {8, 16, 32}) {
        h.interp_ty = ty;
        if (pa::smem_interp(h) > P->smem_limit) continue;
        if ((rc = upload()) != PA_OK) break;
        float ms = 0.f;
        L.nblocks = pa::blocks_interp(h);
        L.smem = pa::smem_interp(h);
        if ((rc = median_ms(s, 5, [&] { return check_launch(pa::launch_interp_width(L, P->w, false, ty), "interp"); },
                            &ms)) != PA_OK)
          break;
        if (ms < best) {
          best = ms;
          pick = ty;
        }
      }
      if (rc != PA_OK) break;
      h.interp_ty = pick;
    }
    rc = upload();
  } while (false);
  cudaStreamSynchronize(s);
  cudaFree(g);
  cudaFree(f);
  if (rc == PA_OK && choice) {
    choice[0] = h.spread_spl;
    choice[1] = h.ner_cb;
    choice[2] = h.ner_threads;
    choice[3] = h.interp_ty;
  }
  return rc;
}

int pa_reconstruct(pa_plan *plan, const float *g_dev, float *f_dev, void *stream) {
  g_err.clear();
  if (!plan || !g_dev || !f_dev) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  IoPtrs io{};
  io.g_in = g_dev;
  io.f_out = f_dev;
  return run_forward(plan, io, reinterpret_cast<cudaStream_t>(stream), false);
}

int pa_reconstruct_cubic(pa_plan *plan, const float *g_dev, float *f_dev, void *stream) {
  g_err.clear();
  if (!plan || !g_dev || !f_dev) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  IoPtrs io{};
  io.g_in = g_dev;
  io.f_out = f_dev;
  return run_forward(plan, io, reinterpret_cast<cudaStream_t>(stream), true);
}

int pa_reconstruct_adjoint(pa_plan *plan, const float *f_dev, float *g_dev, void *stream) {
  g_err.clear();
  if (!plan || !g_dev || !f_dev) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  IoPtrs io{};
  io.f_in = f_dev;
  io.g_out = g_dev;
  return run_adjoint(plan, io, reinterpret_cast<cudaStream_t>(stream), false);
}

int pa_position_grad(pa_plan *plan, const float *g_dev, const float *grad_f_dev, float *grad_g_dev,
                     float *grad_xy_dev, void *stream) {
  g_err.clear();
  if (!plan || !g_dev || !grad_f_dev || !grad_xy_dev) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  IoPtrs io{};
  io.g_in = g_dev;
  io.f_in = grad_f_dev;
  io.g_out = grad_g_dev;
  io.grad_xy = grad_xy_dev;
  return run_adjoint(plan, io, reinterpret_cast<cudaStream_t>(stream), true);
}

int pa_plan_set_weights_device(pa_plan *plan, const float *h_dev, void *stream) {
  g_err.clear();
  if (!plan || !h_dev) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  pa_plan *P = plan;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int M = int(P->M);
  std::vector<float> hh(static_cast<size_t>(M));
  PA_CUDA(cudaMemcpyAsync(hh.data(), h_dev, sizeof(float) * hh.size(), cudaMemcpyDeviceToHost, s));
  PA_CUDA(cudaStreamSynchronize(s));
  for (int m = 0; m < M; ++m)
    if (!(hh[size_t(m)] > 0.f) || !std::isfinite(hh[size_t(m)]))
      return fail(PA_ERR_INVALID_ARG, "weights must be finite and > 0");
  float *ratio = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void **>(&ratio), sizeof(float) * size_t(M), s) != cudaSuccess)
    return fail(PA_ERR_OOM, "pa_plan_set_weights_device: scratch allocation failed");
  pa::WeightRescale r{};
  r.M = M;
  r.w = P->w;
  r.h_new = h_dev;
  r.inv_h = P->d_invh;
  r.ratio = ratio;
  r.perm = P->h.perm;
  r.wy = const_cast<float *>(P->h.wy);
  r.dwy = const_cast<float *>(P->h.dwy);
  r.n_entries = P->n_entries;
  r.sp_m = P->h.sp_m;
  r.sp_w = const_cast<float4 *>(P->h.sp_w);
  r.lat_amp = const_cast<float *>(P->lat_amp);
  cudaError_t e = pa::rescale_weights(r, s);
  if (e == cudaSuccess) e = pa::build_interp_pack(P->h, s);
  cudaFreeAsync(ratio, s);
  if (e != cudaSuccess) return fail(PA_ERR_CUDA, std::string("set weights: ") + cudaGetErrorString(e));
  for (int m = 0; m < M; ++m) P->weights[size_t(m)] = double(hh[size_t(m)]);
  return PA_OK;
}

int pa_weight_grad(pa_plan *plan, const float *g_dev, const float *grad_f_dev, float *grad_h_dev, void *stream) {
  g_err.clear();
  if (!plan || !g_dev || !grad_f_dev || !grad_h_dev) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  float *gb = nullptr;
  const size_t n = size_t(plan->M) * size_t(plan->Nt);
  if (cudaMallocAsync(reinterpret_cast<void **>(&gb), sizeof(float) * n, s) != cudaSuccess)
    return fail(PA_ERR_OOM, "pa_weight_grad: scratch allocation failed");
  IoPtrs io{};
  io.f_in = grad_f_dev;
  io.g_out = gb;
  int rc = run_adjoint(plan, io, s, false);
  if (rc == PA_OK) {
    const cudaError_t e = pa::launch_weight_grad(g_dev, gb, plan->d_invh, int(plan->M), int(plan->Nt), grad_h_dev, s);
    if (e != cudaSuccess) rc = fail(PA_ERR_CUDA, std::string("weight_grad: ") + cudaGetErrorString(e));
  }
  cudaFreeAsync(gb, s);
  return rc;
}

namespace {
pa::VoronoiLaunch voronoi_launch(pa_plan *P) {
  pa::VoronoiLaunch v{};
  const InstDesc &h = P->h;
  v.M = int(P->M);
  v.Mx = h.Mx;
  v.My = h.My;
  v.X = P->grid.nx * P->grid.dx;
  v.Y = P->grid.ny * P->grid.dy;
  v.line = P->d2 ? 1 : 0;
  v.pos = h.pos;
  v.perm = h.perm;
  v.sbx = h.sbx;
  v.sby = h.sby;
  v.cell_start = h.cell_start;
  v.status = h.status;
  return v;
}
}  // namespace

int pa_voronoi_weights(pa_plan *plan, float *h_dev, void *stream) {
  g_err.clear();
  if (!plan || !h_dev) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  pa::VoronoiLaunch v = voronoi_launch(plan);
  v.h = h_dev;
  PA_CUDA(pa::launch_voronoi(v, reinterpret_cast<cudaStream_t>(stream)));
  return PA_OK;
}

int pa_voronoi_grad(pa_plan *plan, const float *grad_h_dev, float *grad_xy_dev, void *stream) {
  g_err.clear();
  if (!plan || !grad_h_dev || !grad_xy_dev) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  pa::VoronoiLaunch v = voronoi_launch(plan);
  v.grad_h = grad_h_dev;
  v.grad_xy = grad_xy_dev;
  PA_CUDA(pa::launch_voronoi(v, reinterpret_cast<cudaStream_t>(stream)));
  return PA_OK;
}

int pa_profile_enable(pa_plan *plan, int enable) {
  g_err.clear();
  if (!plan) return fail(PA_ERR_INVALID_ARG, "plan is NULL");
  plan->profile_mask = enable ? (1u << PA_PROFILE_STAGES) - 1u : 0u;
  return PA_OK;
}

int pa_profile_select(pa_plan *plan, uint32_t stage_mask) {
  g_err.clear();
  if (!plan) return fail(PA_ERR_INVALID_ARG, "plan is NULL");
  plan->profile_mask = stage_mask & ((1u << PA_PROFILE_STAGES) - 1u);
  return PA_OK;
}

int pa_profile_read(pa_plan *plan, double *ms_total, int64_t *launches) {
  g_err.clear();
  if (!plan || !ms_total || !launches) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  for (int k = 0; k < PA_PROFILE_STAGES; ++k) {
    ms_total[k] = 0.0;
    launches[k] = 0;
  }
  for (auto &u : plan->ev_used) {
    PA_CUDA(cudaEventSynchronize(u.second.second));
    float ms = 0.f;
    PA_CUDA(cudaEventElapsedTime(&ms, u.second.first, u.second.second));
    ms_total[u.first] += ms;
    launches[u.first] += 1;
    plan->ev_pool.push_back(u.second.first);
    plan->ev_pool.push_back(u.second.second);
  }
  plan->ev_used.clear();
  return PA_OK;
}

const char *pa_profile_stage_name(int stage) {
  if (stage < 0 || stage >= PA_PROFILE_STAGES) return "";
  return kStageNames[stage];
}

int pa_plan_destroy(pa_plan *plan) {
  g_err.clear();
  if (!plan) return PA_OK;
  cudaDeviceSynchronize();
  free_plan(plan);
  return PA_OK;
}

int pa_status(pa_plan *plan, int *device_status, void *stream) {
  g_err.clear();
  if (!plan || !device_status) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int v = 0;
  PA_CUDA(cudaMemcpyAsync(&v, plan->h.status, sizeof(int), cudaMemcpyDeviceToHost, s));
  PA_CUDA(cudaStreamSynchronize(s));
  PA_CUDA(cudaMemsetAsync(plan->h.status, 0, sizeof(int), s));
  *device_status = v;
  return v ? fail(PA_ERR_DEVICE, "a kernel recorded an error") : PA_OK;
}

int pa_plan_test_wait_fault(pa_plan *plan, int item, int polls, void *stream) {
  g_err.clear();
  if (!plan) return fail(PA_ERR_INVALID_ARG, "plan is NULL");
  if (plan->d2) return fail(PA_ERR_INVALID_ARG, "not supported for 2-D plans");
  plan->h.test_fault = item >= 0 ? item + 1 : 0;
  plan->h.wait_polls = item >= 0 && polls > 0 ? polls : 0;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  PA_CUDA(cudaMemcpyAsync(plan->d_desc, &plan->h, sizeof(InstDesc), cudaMemcpyHostToDevice, s));
  PA_CUDA(cudaStreamSynchronize(s));
  return PA_OK;
}

int pa_plan_is_lattice(const pa_plan *plan, int *is_lattice) {
  g_err.clear();
  if (!plan || !is_lattice) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  *is_lattice = plan->lattice ? 1 : 0;
  return PA_OK;
}

int pa_plan_uses_warp_ner(const pa_plan *plan, int *warp) {
  g_err.clear();
  if (!plan || !warp) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  *warp = plan->h.ner_warp ? 1 : 0;
  return PA_OK;
}

int pa_plan_info(const pa_plan *plan, int64_t *n_sensors, int64_t *n_t, int64_t *workspace_bytes) {
  g_err.clear();
  if (!plan) return fail(PA_ERR_INVALID_ARG, "plan is NULL");
  if (n_sensors) *n_sensors = plan->M;
  if (n_t) *n_t = plan->Nt;
  if (workspace_bytes) *workspace_bytes = int64_t(plan->work_bytes + plan->static_bytes);
  return PA_OK;
}

int pa_plan_buffer(const pa_plan *plan, int which, void *dst_dev, int64_t capacity_bytes, int64_t *bytes,
                   void *stream) {
  g_err.clear();
  if (!plan || !bytes) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  const InstDesc &h = plan->h;
  const void *src;
  int64_t n;
  if (which == 0) {
    src = h.G1;
    n = int64_t(sizeof(float2)) * h.nX1 * h.nY1 * h.Nt;
  } else if (which == 1) {
    src = h.Fz;
    n = int64_t(sizeof(float2)) * h.Nx * h.nY1 * h.Nz;
  } else {
    return fail(PA_ERR_INVALID_ARG, "unknown buffer");
  }
  *bytes = n;
  if (!dst_dev) return PA_OK;
  if (capacity_bytes < n) return fail(PA_ERR_INVALID_ARG, "destination buffer too small");
  PA_CUDA(cudaMemcpyAsync(dst_dev, src, size_t(n), cudaMemcpyDeviceToDevice, reinterpret_cast<cudaStream_t>(stream)));
  return PA_OK;
}

// ------------------------------------------------------------------ batch
int pa_batch_create(pa_batch **out, int n, pa_plan *const *plans, void *stream) {
  g_err.clear();
  if (!out || !plans || n < 1) return fail(PA_ERR_INVALID_ARG, "bad batch arguments");
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!plans[i]) return fail(PA_ERR_INVALID_ARG, "NULL plan in batch");
    if (plans[i]->d2) return fail(PA_ERR_INVALID_ARG, "2-D plans cannot be batched");
    if (plans[i]->w != plans[0]->w || plans[i]->sigma != plans[0]->sigma)
      return fail(PA_ERR_INVALID_ARG, "all plans of a batch need the same sigma and width");
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  pa_batch *B = new pa_batch();
  B->plans.assign(plans, plans + n);
  B->width = plans[0]->w;
  B->ht = plans[0]->ht;
  std::vector<InstDesc> descs(n);
  for (int i = 0; i < n; ++i) descs[i] = plans[i]->h;
  std::vector<int2> work;
  auto add_stage = [&](pa_batch::Stage &st, int (*nb)(const InstDesc &), size_t (*sm)(const InstDesc &)) {
    st.off = work.size();
    st.smem = 0;
    for (int i = 0; i < n; ++i) {
      const int cnt = nb(descs[i]);
      for (int t = 0; t < cnt; ++t) work.push_back(make_int2(i, t));
      st.smem = std::max(st.smem, sm(descs[i]));
    }
    st.nblocks = int(work.size() - st.off);
  };
  // one spread instantiation (samples per lane) serves the whole batch
  for (int i = 0; i < n; ++i) B->spread_spl = std::max(B->spread_spl, pa::spread_spl(descs[i]));
  B->st_spread.off = work.size();
  for (int i = 0; i < n; ++i) {
    const int cnt = pa::blocks_spread(descs[i], B->spread_spl);
    for (int t = 0; t < cnt; ++t) work.push_back(make_int2(i, t));
  }
  B->st_spread.nblocks = int(work.size() - B->st_spread.off);
  add_stage(B->st_rowfft, pa::blocks_rowfft, pa::smem_rowfft);
  add_stage(B->st_col, pa::blocks_colfft, pa::smem_colfft);
  // one NER block size for the whole batch (the largest any instance needs)
  for (int i = 0; i < n; ++i) B->ner_threads = std::max(B->ner_threads, descs[i].ner_threads);
  add_stage(B->st_ner, pa::blocks_ner, pa::smem_ner);
  add_stage(B->st_imgx, pa::blocks_imgx, pa::smem_imgx);
  add_stage(B->st_imgy, pa::blocks_imgy, pa::smem_imgy);
  cudaError_t ce = cudaMalloc(&B->d_descs, sizeof(InstDesc) * n);
  if (ce == cudaSuccess) ce = cudaMalloc(&B->d_io, sizeof(IoPtrs) * n);
  if (ce == cudaSuccess) ce = cudaMalloc(&B->d_work, sizeof(int2) * work.size());
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(B->d_descs, descs.data(), sizeof(InstDesc) * n, cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(B->d_work, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice, s);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
  if (ce != cudaSuccess) {
    cudaFree(B->d_descs);
    cudaFree(B->d_io);
    cudaFree(B->d_work);
    delete B;
    return fail(ce == cudaErrorMemoryAllocation ? PA_ERR_OOM : PA_ERR_CUDA,
                std::string("batch setup: ") + cudaGetErrorString(ce));
  }
  *out = B;
  return PA_OK;
}

static int batch_launches(pa_batch *B, cudaStream_t s) {
  pa::Launch L{};
  L.descs = B->d_descs;
  L.io_table = B->d_io;
  L.stream = s;
  int rc;
  L.work = B->d_work + B->st_spread.off;
  L.nblocks = B->st_spread.nblocks;
  L.smem = 0;
  if ((rc = check_launch(pa::launch_spread(L, B->spread_spl), "batch spread")) != PA_OK) return rc;
  L.work = B->d_work + B->st_rowfft.off;
  L.nblocks = B->st_rowfft.nblocks;
  L.smem = B->st_rowfft.smem;
  if ((rc = check_launch(pa::launch_rowfft(L), "batch rowfft")) != PA_OK) return rc;
  L.work = B->d_work + B->st_col.off;
  L.nblocks = B->st_col.nblocks;
  L.smem = B->st_col.smem;
  if ((rc = check_launch(pa::launch_colfft(L, false), "batch colfft")) != PA_OK) return rc;
  L.work = B->d_work + B->st_ner.off;
  L.nblocks = B->st_ner.nblocks;
  L.smem = B->st_ner.smem;
  L.threads = B->ner_threads;
  if ((rc = check_launch(pa::launch_ner(L, B->width, B->ht, false), "batch ner")) != PA_OK) return rc;
  L.work = B->d_work + B->st_imgx.off;
  L.nblocks = B->st_imgx.nblocks;
  L.smem = B->st_imgx.smem;
  if ((rc = check_launch(pa::launch_imgx(L, false), "batch imgx")) != PA_OK) return rc;
  L.work = B->d_work + B->st_imgy.off;
  L.nblocks = B->st_imgy.nblocks;
  L.smem = B->st_imgy.smem;
  if ((rc = check_launch(pa::launch_imgy(L, false), "batch imgy")) != PA_OK) return rc;
  return PA_OK;
}

static void batch_drop_graph(pa_batch *B) {
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  B->exec = nullptr;
  B->graph = nullptr;
}

// Mode 0: the instances' single-plan forward launches (the fastest kernels
// each size has: warp NER, tensor-map pipelines) as kBranches concurrent
// branches of one graph, largest instances first, each branch taking the
// next instance when it has the least estimated work.
constexpr int kBranches = 4;

static int batch_run_branches(pa_batch *B, const float *const *g_dev, float *const *f_dev, cudaStream_t s) {
  const int n = int(B->plans.size());
  bool same = B->exec != nullptr && int(B->cap_g.size()) == n;
  for (int i = 0; same && i < n; ++i) same = B->cap_g[i] == g_dev[i] && B->cap_f[i] == f_dev[i];
  if (same) {
    PA_CUDA(cudaGraphLaunch(B->exec, s));
    return PA_OK;
  }
  batch_drop_graph(B);
  auto io_of = [&](int i) {
    IoPtrs io{};
    io.g_in = g_dev[i];
    io.f_out = f_dev[i];
    return io;
  };
  // this call: the launches directly (also sets the kernels' attributes
  // outside the capture); later calls with the same buffers replay the graph
  for (int i = 0; i < n; ++i) {
    const int rc = run_forward(B->plans[i], io_of(i), s, false);
    if (rc != PA_OK) return rc;
  }
  if (B->side.empty()) {
    B->side.resize(kBranches);
    B->ev.resize(kBranches + 1);
    for (auto &st : B->side) PA_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    for (auto &e : B->ev) PA_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  auto cost = [&](int i) {
    const InstDesc &h = B->plans[i]->h;
    return double(h.Mx) * h.My * h.Nt + double(h.Nx) * h.Ny * h.Nz;
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  cudaStream_t cap;
  PA_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  int rc = PA_OK;
  cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (ce == cudaSuccess) {
    ce = cudaEventRecord(B->ev[0], cap);
    for (int k = 0; ce == cudaSuccess && k < kBranches; ++k) ce = cudaStreamWaitEvent(B->side[k], B->ev[0], 0);
    double load[kBranches] = {0.0};
    for (int j = 0; ce == cudaSuccess && rc == PA_OK && j < n; ++j) {
      const int i = order[j];
      int k = 0;
      for (int q = 1; q < kBranches; ++q)
        if (load[q] < load[k]) k = q;
      load[k] += cost(i);
      rc = run_forward(B->plans[i], io_of(i), B->side[k], false);
    }
    for (int k = 0; ce == cudaSuccess && k < kBranches; ++k) {
      ce = cudaEventRecord(B->ev[k + 1], B->side[k]);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cap, B->ev[k + 1], 0);
    }
    const cudaError_t ce2 = cudaStreamEndCapture(cap, &B->graph);
    if (ce == cudaSuccess) ce = ce2;
  }
  cudaStreamDestroy(cap);
  if (ce != cudaSuccess || rc != PA_OK) {
    batch_drop_graph(B);
    return rc != PA_OK ? rc : fail(PA_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  }
  PA_CUDA(cudaGraphInstantiate(&B->exec, B->graph, 0));
  B->cap_g.assign(g_dev, g_dev + n);
  B->cap_f.assign(f_dev, f_dev + n);
  return PA_OK;
}

int pa_batch_set_mode(pa_batch *B, int mode) {
  g_err.clear();
  if (!B || (mode != 0 && mode != 1)) return fail(PA_ERR_INVALID_ARG, "bad batch mode");
  if (mode != B->mode) {
    batch_drop_graph(B);
    B->cap_g.clear();
    B->cap_f.clear();
    B->mode = mode;
  }
  return PA_OK;
}

int pa_batch_run(pa_batch *B, const float *const *g_dev, float *const *f_dev, void *stream) {
  g_err.clear();
  if (!B || !g_dev || !f_dev) return fail(PA_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n = int(B->plans.size());
  std::vector<IoPtrs> io(n);
  for (int i = 0; i < n; ++i) {
    if (!g_dev[i] || !f_dev[i]) return fail(PA_ERR_INVALID_ARG, "NULL buffer in batch");
    io[i] = IoPtrs{};
    io[i].g_in = g_dev[i];
    io[i].f_out = f_dev[i];
  }
  if (B->mode == 0) return batch_run_branches(B, g_dev, f_dev, s);
  // pageable source: the copy has consumed `io` when the call returns
  PA_CUDA(cudaMemcpyAsync(B->d_io, io.data(), sizeof(IoPtrs) * n, cudaMemcpyHostToDevice, s));
  if (!B->exec) {
    // kernel attributes are set outside the capture by a first direct run
    int rc = batch_launches(B, s);
    if (rc != PA_OK) return rc;
    cudaStream_t cap;
    PA_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
      rc = batch_launches(B, cap);
      ce = cudaStreamEndCapture(cap, &B->graph);
    }
    cudaStreamDestroy(cap);
    if (ce != cudaSuccess || rc != PA_OK)
      return rc != PA_OK ? rc : fail(PA_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    PA_CUDA(cudaGraphInstantiate(&B->exec, B->graph, 0));
    return PA_OK;
  }
  PA_CUDA(cudaGraphLaunch(B->exec, s));
  return PA_OK;
}

int pa_batch_destroy(pa_batch *B) {
  g_err.clear();
  if (!B) return PA_OK;
  cudaDeviceSynchronize();
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  for (auto st : B->side) cudaStreamDestroy(st);
  for (auto e : B->ev) cudaEventDestroy(e);
  cudaFree(B->d_descs);
  cudaFree(B->d_io);
  cudaFree(B->d_work);
  delete B;
  return PA_OK;
}

}  // extern "C"
