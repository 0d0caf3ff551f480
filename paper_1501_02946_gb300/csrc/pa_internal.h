// pa_internal.h -- data structures shared by the host plan code and the
// sm_103a kernels of the NEDNER-NUFFT library.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

struct pa_plan;

namespace pa {

constexpr int kMaxStages = 12;
constexpr int kMaxFft = 4096;
constexpr int kMaxWidth = 16;
constexpr int kMaxDeg = 15;

// Mixed-radix Stockham schedule for one transform length L: the radices in
// the order they are applied and the offset of the length-L twiddle table
// exp(-2 pi i m / L), m = 0..L-1, inside the plan's twiddle array.
struct FftPlan {
  int L;
  int nst;
  int radix[kMaxStages];
  int tw;
};

// Horner coefficients of the window taps used by the NER interpolation:
// tap t (0..w-1) at fraction fr in [0,1) of the oversampled time-frequency
// grid is phi(fr + w/2 - 1 - t) = P_t(s) = sum_d c[t][d] s^d with
// s = 2 fr - 1, where phi is the Kaiser-Bessel window normalised to
// phi(0) = 1.  The window is even, so P_{w-1-t}(s) = P_t(-s): with
// P_t(s) = E_t(s^2) + s O_t(s^2) (the even and odd powers), taps t and
// w - 1 - t are E_t(u) +- s O_t(u), u = s^2.  The table holds the first w/2
// taps' coefficient pairs (c[t][2k], c[t][2k + 1]), so that E and O
// evaluate together as packed two-wide Horner steps in u.
struct HornerTable {
  float2 eo[kMaxWidth / 2][kMaxDeg / 2 + 1];
  __host__ void set(int t, int d, float v) {
    if (d & 1) {
      eo[t][d >> 1].y = v;
    } else {
      eo[t][d >> 1].x = v;
    }
  }
};

// One reconstruction instance as the kernels see it.  Every kernel reads
// only this struct (plus its own tile index), so a batch is an array of them.
struct InstDesc {
  // problem sizes
  int M, Nt, Nx, Ny, Nz;
  int Mx, My, Mt;       // oversampled lengths sigma*Nx, sigma*Ny, sigma*Nt
  int w;                // window taps
  int hx, hy, hz, nc;   // floor(N/2) of x, y, z, t
  int nX1, nY1;         // rows of the spatial spectrum: 2*hx+1 (jx) and hy+1 (jy)
  int nchunk_adj;       // n-chunks of the adjoint NED kernel (gradient partials)
  int ner_cb;           // columns per block of the NER kernels (1, 2 or 4)
  int ner_threads;      // block size of the NER kernels (128 or 256)
  int ner_lperm;        // adjoint NER depth order il = (i * ner_lperm) mod Nz
  int spread_spl;       // samples per lane of the spread (4 or 8)
  int interp_ty;        // grid columns per interpolation tile (8, 16 or 32)
  int ner_warp;         // 1: the NER stage runs the warp-per-column kernels
  int wtw;              // offset of the warp-transform twiddle tables in tw

  FftPlan fMy, fMx, fMt, fNz, fNx, fNy, fNt;
  const float2 *tw;

  // sensors sorted by (bx, by); taps t = 0..w-1 cover cells base - w/2 + 1 + t
  const int *perm;      // sorted -> caller's sensor index
  const int *sbx, *sby; // base cells, wrapped into [0, Mx) and [0, My)
  const float *wx, *wy; // [M][w]; wy carries a_m = h_m/(dx dy)
  const float *dwx, *dwy;  // [M][w] derivative taps d/dx_m and d/dy_m
  const int *cell_start;   // [Mx*My + 1] CSR offsets of the sorted sensors per cell
  const double2 *pos;      // [M] positions reduced into [-X/2, X/2) x [-Y/2, Y/2), caller order
  // per sorted sensor, for the interpolation tiles: ipack[i] holds
  // wx[0..w), wy[0..w), by, m (as int bits) in ipack_words(w) floats;
  // ipack_d[i] holds dwx[0..w), dwy[0..w) in ipackd_words(w) floats
  const float4 *ipack;
  const float4 *ipack_d;
  // forward spread entries: strip s (kSpreadP grid rows p0 = s*kSpreadP ..)
  // and column q own the entries sp_start[s*My + q] .. sp_start[s*My + q + 1]-1;
  // entry e is a sensor (caller index sp_m[e]) with its tap products
  // sp_w[e] = wy(q) * (wx(p0), wx(p0+1), wx(p0+2), wx(p0+3)), zero off the
  // footprint.  Within a list the sensors follow the sorted (cell) order.
  const int *sp_start;
  const int *sp_m;
  const float4 *sp_w;
  // the same entries for the staged spread: block b = strip * ceil(My / 8)
  // + (q / 8) stages the g rows of its union of sensors (caller indices
  // sp_um[sp_ustart[b] ..  sp_ustart[b + 1]), most used first) in shared
  // memory, and entry e names its sensor by the position sp_slot[e] in that
  // union; sp_urows is the number of rows the staging buffer holds (rows past
  // it are read from global memory).  Null when not built (then the spread
  // reads g through sp_m).
  const int *sp_slot;
  const int *sp_ustart;
  const int *sp_um;
  int sp_urows;
  // per spread block: its entries [x, y) (the 8 lists of its columns are one
  // contiguous range), and the most entries any block has
  const int2 *sp_erange;
  int sp_emax;
  // deconvolution factors 1/phihat (window normalised to phi(0) = 1)
  const float *invphx;  // [nX1], jx = ix - hx, at jx / Mx
  const float *invphy;  // [nY1], jy, at jy / My
  const float *invpht;  // [Nt], at (n - nc) / Mt

  // time-frequency constants, each as a double-float pair (hi, lo):
  // tau(j,l)^2 = ax jx^2 + ay jy^2 + az l^2, tau = omega Nt dt / (2 pi),
  // phase turns of the centring exp(-2 pi i tau nc / Nt) = tau * ph.
  float ax_hi, ax_lo, ay_hi, ay_lo, az_hi, az_lo;
  float ph_hi, ph_lo;
  float sqrt_az;        // c Nt dt / Z, for W(j,l) = 2c sqrt_az |l| / |tau|
  float two_c;          // 2 c
  float scale;          // dt / (dz Nx Ny Nz)
  int sigma;

  // workspace (device)
  float2 *T;            // [Mx][nY1][Nt]   after the row transform (aliases Fz/U)
  float2 *G1;           // [nX1][nY1][Nt]  spatial spectrum
  float2 *Fz;           // [Nx][nY1][Nz]   after NER and the inverse depth DFT
  float2 *U;            // [Nx][nY1][Nz]   after the inverse x DFT
  float2 *grad_part;    // [nchunk_adj][M] per-chunk position-gradient partials
  float *G0;            // [Mx][My][Nt] real oversampled grid (forward) or its cotangent (adjoint)
  int *status;
  // test hook of the pipelined interpolation (zero: off): work item
  // test_fault - 1 has its byte count posted but none of its copies issued,
  // and its waits give up after wait_polls polls (zero: kMbarPolls)
  int test_fault;
  int wait_polls;
};

// Twiddle tables of the warp-per-column NER kernels, appended to the plan's
// twiddle array at InstDesc::wtw: for N = 2^lgn, lgn = 8, 9, 10, the rows
// [k2][n1] = exp(-2 pi i n1 k2 / N) (k2 < N/32, n1 < 32) at wtw_T(lgn), then
// for M = 2^lgm, lgm = 9, 10, 11, the circle exp(-2 pi i j / M), j < M, at
// wtw_F(lgm).
__host__ __device__ constexpr int wtw_T(int lgn) { return lgn == 8 ? 0 : (lgn == 9 ? 256 : 768); }
__host__ __device__ constexpr int wtw_F(int lgm) { return lgm == 9 ? 1792 : (lgm == 10 ? 2304 : 3328); }
constexpr int kWtwSize = 5376;

// Floats per sensor of the interpolation packs (multiples of 4: 16-byte rows).
__host__ __device__ constexpr int ipack_words(int w) { return ((2 * w + 2 + 3) / 4) * 4; }
__host__ __device__ constexpr int ipackd_words(int w) { return ((2 * w + 3) / 4) * 4; }

// Caller buffers of one call (device pointers).  Single-plan launches pass
// them by value; batched launches pass a device table indexed by instance.
struct IoPtrs {
  const float *g_in;    // [M][Nt]
  float *f_out;         // [Nx][Ny][Nz]
  const float *f_in;    // [Nx][Ny][Nz]
  float *g_out;         // [M][Nt] or null
  float *grad_xy;       // [M][2] or null
};

// Tile shapes (chosen on the host; kernels are templated on them).
constexpr int kSpreadP = 4;      // oversampled rows per forward spread strip
constexpr int kSpreadQC = 8;     // columns per spread block (one warp each)
constexpr int kSpreadUrowsMax = 128;  // g rows the staged spread holds in shared memory
constexpr int kSpreadUrowsMin = 32;   // ... at least, when held down for more blocks per SM
constexpr int kSpreadTileBlocks = 4;  // staged-spread blocks per SM its shared memory is sized for
// floats of a staged-spread block after its g rows: the entries' tap products
// (4 each), their slots, and 8 for the 16-byte rounding of the slot copy
inline long SpreadTileEntryFloats(int emax) { return 5L * emax + 8; }
constexpr int kColNC = 16;       // samples per column-FFT tile
constexpr int kInterpNC = 32;    // samples per adjoint interpolation tile
constexpr int kImgZC = 16;       // depth samples per inverse-x tile
constexpr int kImgZP = 16;       // depth pairs per y-C2R tile

// Launch helpers implemented in the .cu files.  `work` lists (instance, tile)
// pairs for batched launches; null means instance 0 and tile = blockIdx.x.
struct Launch {
  const InstDesc *descs;  // device array
  const int2 *work;       // device array or null
  IoPtrs io;              // caller buffers (single plan)
  const IoPtrs *io_table; // device array (batch) or null
  int nblocks;
  size_t smem;
  cudaStream_t stream;
  int threads;            // block size, for kernels that take it from the host
  const InstDesc *host;   // host copy of the descriptor of a single-plan launch (else null)
};

// Block counts and shared-memory sizes per stage for one instance.
int spread_spl(const InstDesc &d);  // samples per lane of the spread (4 or 8)
int blocks_spread(const InstDesc &d, int spl);
int blocks_rowfft(const InstDesc &d);
size_t smem_rowfft(const InstDesc &d);
int blocks_colfft(const InstDesc &d);
size_t smem_colfft(const InstDesc &d);
int blocks_ner(const InstDesc &d);
int blocks_ner_adj(const InstDesc &d);
size_t smem_ner(const InstDesc &d);  // forward and adjoint
int blocks_imgx(const InstDesc &d);
size_t smem_imgx(const InstDesc &d);
int blocks_imgy(const InstDesc &d);
size_t smem_imgy(const InstDesc &d);
int blocks_interp(const InstDesc &d);
size_t smem_interp(const InstDesc &d);
int blocks_rowifft(const InstDesc &d);
size_t smem_rowifft(const InstDesc &d);

cudaError_t launch_spread(const Launch &L, int spl);
cudaError_t launch_rowfft(const Launch &L);
cudaError_t launch_colfft(const Launch &L, bool adjoint);
cudaError_t launch_ner(const Launch &L, int width, const HornerTable &ht, bool adjoint);
// which: 0 forward, 1 adjoint
cudaError_t launch_ner_stage(const Launch &L, int width, const HornerTable &ht, int which);
cudaError_t launch_cubic(const Launch &L);
// Warp-per-column NER kernels (pa_ner_warp.cu): sigma = 2, width 8, Nt and
// Nz powers of two in [256, 1024]; single-plan launches (L.host set).
bool ner_warp_eligible(const InstDesc &d);
size_t smem_ner_warp(const InstDesc &d);
int ner_warp_block_warps(const InstDesc &d);
cudaError_t launch_ner_warp(const Launch &L, const HornerTable &ht, int which);
cudaError_t launch_imgx(const Launch &L, bool adjoint);
cudaError_t launch_imgy(const Launch &L, bool adjoint);
cudaError_t launch_interp_width(const Launch &L, int width, bool grad, int ty);
cudaError_t launch_rowifft(const Launch &L);
cudaError_t launch_grad_reduce(const Launch &L, int M);
// The d = 2 operator's own stages (pa_d2.cu): 1-D spread into T, its
// transpose from T (with the position-gradient partials when grad), and the
// real part of the single jy column and its transpose.
cudaError_t launch_spread_x(const Launch &L, const InstDesc &h);
cudaError_t launch_interp_x(const Launch &L, const InstDesc &h, bool grad);
cudaError_t launch_real_out(const Launch &L, const InstDesc &h);
cudaError_t launch_real_in(const Launch &L, const InstDesc &h);
// grad_h[m] = inv_h[m] * sum_n g[m][n] gb[m][n] (pa_metrics.cu): the
// gradient with respect to the weights h_m, given gb = A^T grad_f.
cudaError_t launch_weight_grad(const float *g, const float *gb, const float *inv_h, int M, int Nt, float *grad_h,
                               cudaStream_t s);
// New detector weights h_new for a plan (pa_metrics.cu): ratio = h_new /
// h_old per sensor, the tables that carry h_m scaled by it (wy, dwy in
// sorted order, the spread entries' tap products, the lattice amplitudes),
// and inv_h rewritten.
struct WeightRescale {
  int M, w;
  const float *h_new;
  float *inv_h;            // [M] 1/h (in: old, out: new)
  float *ratio;            // [M] scratch
  const int *perm;
  float *wy, *dwy;         // [M][w], sorted order
  size_t n_entries;
  const int *sp_m;
  float4 *sp_w;
  float *lat_amp;          // [M] caller order, or null
};
cudaError_t rescale_weights(const WeightRescale &r, cudaStream_t s);
// Periodic Voronoi weights and their chain-rule gradient (pa_voronoi.cu).
struct VoronoiLaunch {
  int M, Mx, My;
  double X, Y;
  int line;                 // 1: 2-D plan (sensors on the circle X)
  const double2 *pos;       // [M] reduced positions, caller order
  const int *perm, *sbx, *sby, *cell_start;
  float *h;                 // [M] weights out, or null
  const float *grad_h;      // [M] gradient in, or null
  float *grad_xy;           // [M][2] accumulated, or null
  int *status;
};
cudaError_t launch_voronoi(const VoronoiLaunch &v, cudaStream_t s);
// Status-word bit: a Voronoi cell outgrew its vertex buffer (its weight and
// gradient were not written).
constexpr int kStatusVoronoi = 8;
// Rewrite ipack / ipack_d from perm, sby, wx, wy, dwx, dwy (after a sensor upload).
cudaError_t build_interp_pack(const InstDesc &h, cudaStream_t s);

// Device re-binning of new sensor positions (pa_rebin.cu): inputs, the plan
// tables it rewrites and its scratch.
struct RebinArgs {
  int M, Mx, My, w, nstrips;
  double X, Y, ax;         // period lengths and 1/(dx dy)
  double beta, phi0;       // Kaiser-Bessel window of the plan
  const float *xy;         // [M][2] new positions (caller's device buffer)
  double2 *pos;            // [M] reduced positions (plan table, output)
  const double *weights;   // [M] detector areas h_m
  int *status;             // plan status word (non-finite positions)
  // plan tables (outputs)
  int *perm, *sbx, *sby, *cell_start;
  float *wx, *wy, *dwx, *dwy;
  // scratch
  int *bx, *by;
  double *frx, *fry;
  int *fill;               // max(cells, entry lists) counters
  int *sp_cnt;             // [nstrips*My + 1] entry counts, then offsets
  int *sp_m;               // entry lists (outputs, sized by the count)
  float4 *sp_w;
  long long *sp_key;       // order keys of the entries
};
cudaError_t rebin_sensors(const RebinArgs &a, cudaStream_t s);
cudaError_t rebin_count_entries(const RebinArgs &a, cudaStream_t s);
cudaError_t rebin_fill_entries(const RebinArgs &a, cudaStream_t s);
// Status-word bit: non-finite sensor positions met by the device re-binning.
constexpr int kStatusBadPositions = 2;

// Lattice spatial step (pa_lattice.cu).
cudaError_t launch_lattice_scatter(float *G0, const int *pq, const float *a, const float *g, int M, int Nt,
                                   cudaStream_t s);
cudaError_t launch_lattice_gather(float *g, const float *G0, const int *pq, const float *a, int M, int Nt,
                                  cudaStream_t s);
cudaError_t launch_lattice_alias(float2 *G1, int nY1, int Nt, int hx, int dir, cudaStream_t s);

// Read-only view of a plan for the other translation units of the library.
struct PlanView {
  const InstDesc *h;        // host copy of the descriptor (device pointers inside)
  int width;
  const HornerTable *ht;
  int device;
  long long n_sensors;
  int dims;                 // 3, or 2 for a plan of pa_plan_create_2d
};
int plan_view(const pa_plan *P, PlanView *v);
// Record an error message for pa_last_error() and return `code`.
int set_error(int code, const char *msg);

}  // namespace pa
