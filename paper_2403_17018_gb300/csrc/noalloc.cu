// henry_residual_jacobian_noalloc: the residual/Jacobian evaluation of
// henry_residual_jacobian with its scratch memory in a file-scope device
// array, so that the call never allocates device memory (see henry.h).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/henry.h"
#include "solver.h"

namespace henry {
cudaError_t launch_residual_jacobian(const Phys& P, const Geom& G, double tau, int B,
                                     const double* phi, const double* K, const double* qin,
                                     const double* p, const double* c, const double* c_old,
                                     double* R, double* J, double* scratch, cudaStream_t s);
}  // namespace henry

namespace {

// 5 doubles per cell and sample: face constants tx, dx, ty, dy and the
// reduced pressure. 2^20 doubles = 8 MiB, held by every GPU that loads the
// library until the process exits.
constexpr size_t kNoAllocScratchDoubles = size_t(1) << 20;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

// Device address of g_noalloc_scratch per device, looked up once per device
// with that device current. In host code the symbol itself is only a
// host-side stand-in and must never be passed to a kernel.
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double* g_scratch_addr[kMaxDevices] = {};

int scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      henry::set_last_error(std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
      return HENRY_E_CUDA;
    }
    g_scratch_addr[dev] = (double*)p;
  }
  *out = g_scratch_addr[dev];
  return HENRY_OK;
}

int fail(int code, const std::string& msg) {
  henry::set_last_error(msg);
  return code;
}

}  // namespace

extern "C" int henry_residual_jacobian_noalloc(const henry_config* cfg, int nx, int ny, double tau,
                                               int B, const double* phi, const double* K,
                                               const double* qin, const double* p,
                                               const double* c, const double* c_old, double* R,
                                               double* J, void* stream) {
  if (!cfg) return fail(HENRY_E_INVALID, "config is NULL");
  if (nx < 2 || ny < 1 || B < 0 || B > HENRY_MAX_BATCH || !(tau > 0))
    return fail(HENRY_E_INVALID, "bad sizes (nx >= 2, ny >= 1, 0 <= B <= 65535, tau > 0)");
  if (B == 0) return HENRY_OK;
  if (!phi || !K || !qin || !p || !c || !c_old || !R) return fail(HENRY_E_INVALID, "NULL argument");
  const size_t need = (size_t)5 * (size_t)B * (size_t)nx * (size_t)ny;
  if (need > kNoAllocScratchDoubles)
    return fail(HENRY_E_INVALID,
                "henry_residual_jacobian_noalloc: B*nx*ny = " +
                    std::to_string((size_t)B * nx * ny) + " exceeds the maximum of " +
                    std::to_string(kNoAllocScratchDoubles / 5) + " cells");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(HENRY_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(HENRY_E_INVALID, "device index above 63");
  double* scratch = nullptr;
  const int rc = scratch_address(dev, &scratch);
  if (rc) return rc;
  henry::Phys P{cfg->rho0, cfg->rho1 - cfg->rho0, cfg->mu, cfg->g, cfg->D, cfg->K0, cfg->phi0,
                cfg->q0, cfg->Lx, cfg->Ly};
  henry::Geom G{nx, ny, cfg->Lx / nx, cfg->Ly / ny};
  e = henry::launch_residual_jacobian(P, G, tau, B, phi, K, qin, p, c, c_old, R, J, scratch,
                                      (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(HENRY_E_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return HENRY_OK;
}
