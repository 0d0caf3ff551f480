// pa_noalloc.cu -- pa_position_grad_noalloc: the sensor-position gradient
// with its scratch (the per-chunk gradient partial sums) in a file-scope
// static device array instead of the plan's workspace, so that the call
// itself allocates no device memory.
//
// The array below is part of the library image: every GPU that loads the
// library holds it (16 MiB plus one descriptor) until the process exits.
// In host code its name is only a host-side stand-in for the device symbol,
// so its device address is looked up with that device current
// (cudaGetSymbolAddress) and passed to the kernels.  The lookup is made once
// per device and context: a new primary context (after cudaDeviceReset, say)
// may load the library's module at another address, so it is looked up again.
#include <mutex>
#include <string>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "pa_internal.h"
#include "pa_nufft.h"

namespace {

constexpr size_t kPartials = size_t(1) << 21;  // float2 entries (16 MiB)
constexpr int kMaxDevices = 64;

__device__ __align__(256) float2 pa_noalloc_partials[kPartials];
__device__ __align__(256) pa::InstDesc pa_noalloc_desc;

// The call's descriptor reaches the device as a kernel argument (copied at
// launch) and is stored into the static descriptor by one thread; no host
// buffer is read after the launch returns.
__global__ void k_store_desc(const __grid_constant__ pa::InstDesc d) { pa_noalloc_desc = d; }

std::mutex g_mu;
CUcontext g_ctx[kMaxDevices] = {};
bool g_ready[kMaxDevices] = {};
float2 *g_partials[kMaxDevices] = {};
pa::InstDesc *g_desc[kMaxDevices] = {};

// The current context through the runtime's driver entry-point query (null
// if unavailable; the lookup is then made on every call).
CUcontext current_context() {
  static PFN_cuCtxGetCurrent_v4000 get = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
  }
  CUcontext c = nullptr;
  if (get && get(&c) != CUDA_SUCCESS) c = nullptr;
  return c;
}

// Device addresses of the static arrays on the current device (looked up on
// the first call made on that device, and again when its context changed).
int static_addresses(int dev, float2 **partials, pa::InstDesc **desc) {
  std::lock_guard<std::mutex> lock(g_mu);
  const CUcontext ctx = current_context();
  if (!g_ready[dev] || !ctx || ctx != g_ctx[dev]) {
    void *p = nullptr, *q = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, pa_noalloc_partials);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, pa_noalloc_desc);
    if (e != cudaSuccess)
      return pa::set_error(PA_ERR_CUDA, (std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)).c_str());
    g_partials[dev] = static_cast<float2 *>(p);
    g_desc[dev] = static_cast<pa::InstDesc *>(q);
    g_ctx[dev] = ctx;
    g_ready[dev] = true;
  }
  *partials = g_partials[dev];
  *desc = g_desc[dev];
  return PA_OK;
}

int launched(cudaError_t e, const char *what) {
  if (e != cudaSuccess)
    return pa::set_error(PA_ERR_CUDA, (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
  return PA_OK;
}

}  // namespace

extern "C" int pa_position_grad_noalloc(pa_plan *plan, const float *g_dev, const float *grad_f_dev,
                                        float *grad_g_dev, float *grad_xy_dev, void *stream) {
  pa::set_error(PA_OK, "");
  pa::PlanView v{};
  if (!plan || !g_dev || !grad_f_dev || !grad_xy_dev || pa::plan_view(plan, &v) != PA_OK)
    return pa::set_error(PA_ERR_INVALID_ARG, "NULL argument");
  if (v.dims != 3) return pa::set_error(PA_ERR_INVALID_ARG, "pa_position_grad_noalloc: not supported for 2-D plans");
  const pa::InstDesc &h = *v.h;
  const size_t need = size_t(h.nchunk_adj) * size_t(h.M);
  if (need > kPartials)
    return pa::set_error(PA_ERR_UNSUPPORTED_SIZE,
                         ("pa_position_grad_noalloc: needs " + std::to_string(need) +
                          " gradient partials (ceil(n_t/32) * n_sensors), the static limit is " +
                          std::to_string(kPartials))
                             .c_str());
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return launched(e, "cudaGetDevice");
  if (dev != v.device) return pa::set_error(PA_ERR_INVALID_ARG, "the plan's device is not the current device");
  if (dev < 0 || dev >= kMaxDevices) return pa::set_error(PA_ERR_INVALID_ARG, "device index out of range");
  float2 *partials = nullptr;
  pa::InstDesc *ddesc = nullptr;
  int rc = static_addresses(dev, &partials, &ddesc);
  if (rc != PA_OK) return rc;

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // the plan's descriptor with the partial sums redirected to the static array
  pa::InstDesc d = h;
  d.grad_part = partials;
  k_store_desc<<<1, 1, 0, s>>>(d);
  if ((rc = launched(cudaGetLastError(), "descriptor store")) != PA_OK) return rc;

  pa::Launch L{};
  L.descs = ddesc;
  L.host = &d;
  L.stream = s;
  L.io.g_in = g_dev;
  L.io.f_in = grad_f_dev;
  L.io.g_out = grad_g_dev;
  L.io.grad_xy = grad_xy_dev;
  L.nblocks = pa::blocks_imgy(h);
  L.smem = pa::smem_imgy(h);
  if ((rc = launched(pa::launch_imgy(L, true), "imgy_adj")) != PA_OK) return rc;
  L.nblocks = pa::blocks_imgx(h);
  L.smem = pa::smem_imgx(h);
  if ((rc = launched(pa::launch_imgx(L, true), "imgx_adj")) != PA_OK) return rc;
  L.threads = h.ner_threads;
  L.nblocks = pa::blocks_ner_adj(h);
  L.smem = pa::smem_ner(h);
  if ((rc = launched(pa::launch_ner_stage(L, v.width, *v.ht, 1), "ner_adj")) != PA_OK) return rc;

  L.nblocks = pa::blocks_colfft(h);
  L.smem = pa::smem_colfft(h);
  if ((rc = launched(pa::launch_colfft(L, true), "colfft_adj")) != PA_OK) return rc;
  L.nblocks = pa::blocks_rowifft(h);
  L.smem = pa::smem_rowifft(h);
  if ((rc = launched(pa::launch_rowifft(L), "rowifft")) != PA_OK) return rc;
  L.nblocks = pa::blocks_interp(h);
  L.smem = pa::smem_interp(h);
  if ((rc = launched(pa::launch_interp_width(L, v.width, true, h.interp_ty), "interp")) != PA_OK) return rc;
  L.nblocks = int((h.M + 255) / 256) < 1024 ? int((h.M + 255) / 256) : 1024;
  if ((rc = launched(pa::launch_grad_reduce(L, 1), "grad_reduce")) != PA_OK) return rc;
  return PA_OK;
}
