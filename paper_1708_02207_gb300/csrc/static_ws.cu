// hdd_evaluate_static: the likelihood path with its workspace in a static device
// array, for callers that cannot allocate device memory at evaluation time.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "plan.h"

namespace hdd {
hdd_status set_error(hdd_status status, const std::string& msg);
}

namespace {

// The one workspace shared by every call on a device (held until process exit).
__device__ __align__(256) unsigned char g_static_workspace[HDD_STATIC_WORKSPACE_BYTES];

std::mutex g_static_mutex;
void* g_static_ptr[64] = {};

// Device address of g_static_workspace on `dev`, looked up once per device with
// that device current (a host-side use of the symbol is not a device address).
cudaError_t static_workspace(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_static_mutex);
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!g_static_ptr[dev]) {
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e == cudaSuccess && prev != dev) e = cudaSetDevice(dev);
    void* ptr = nullptr;
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&ptr, g_static_workspace);
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = ptr;
  }
  *out = g_static_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" hdd_status hdd_evaluate_static(hdd_plan_t plan, int32_t batch, const double* Z, const double* y,
                                          int32_t y_per_sample, double* loglik, double* u_obs,
                                          int32_t* sample_status, void* stream) {
  if (!plan) return hdd::set_error(HDD_EINVAL, "plan is NULL");
  if (!Z || !y || !loglik) return hdd::set_error(HDD_EINVAL, "Z, y or loglik is NULL");
  if (plan->p.device < 0) return hdd::set_error(HDD_ESTATE, "host-only plan");
  size_t need = 0;
  hdd_status s = hdd_workspace_size(plan, batch, &need);
  if (s != HDD_OK) return s;
  if (need > HDD_STATIC_WORKSPACE_BYTES)
    return hdd::set_error(HDD_EINVAL, "batch workspace of " + std::to_string(need) +
                                          " bytes exceeds HDD_STATIC_WORKSPACE_BYTES");
  void* ws = nullptr;
  const cudaError_t e = static_workspace(plan->p.device, &ws);
  if (e != cudaSuccess) return hdd::set_error(HDD_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  double* uo = u_obs ? u_obs
                     : reinterpret_cast<double*>(static_cast<char*>(ws) + hdd::layout(plan->p, batch).uobs);
  if ((s = hdd_assemble(plan, Z, batch, ws, stream)) != HDD_OK) return s;
  if ((s = hdd_upsweep(plan, batch, ws, stream)) != HDD_OK) return s;
  if ((s = hdd_point_solve(plan, batch, ws, uo, stream)) != HDD_OK) return s;
  return hdd_loglik(plan, batch, ws, uo, y, y_per_sample, loglik, sample_status, stream);
}
