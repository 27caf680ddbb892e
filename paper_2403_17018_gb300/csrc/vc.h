// Host driver of the vertex-centred variant of the solve (see vc.cu).
#pragma once

#include <cuda_runtime.h>

#include "../../include/henry.h"
#include "henry_device.cuh"

namespace henry {

void set_last_error(const std::string& msg);

// Batched solves of one level with the vertex-centred discretisation:
// nodal unknowns on an nx x (ny + 1) node grid, BiCGStab preconditioned by
// red-black block Gauss-Seidel inside FP64 defect correction, host-side
// Newton loop. Outputs as henry_solve, with c_out / p_out of shape
// [B][ny + 1][nx] (the unknown nodes).
class VcSolver {
 public:
  VcSolver(const henry_config& cfg, int nx, int ny, int nt);
  ~VcSolver();
  VcSolver(const VcSolver&) = delete;
  VcSolver& operator=(const VcSolver&) = delete;
  int run(const double* xi, int B, double* q, double* c_out, double* p_out, int* status,
          int* iters, int status_or, cudaStream_t s);
  unsigned long long launches() const;

 private:
  int ensure(int B);
  void enqueue_linear(int B, cudaStream_t s);

  henry_config cfg_;
  Phys phys_;
  Geom G_;            // node grid: nx x (ny + 1)
  int nt_;
  double tau_;
  int kry_, sweeps_;  // BiCGStab iterations per correction, Gauss-Seidel sweeps per application
  int cap_ = 0, nchunk_ = 1, kry_nchunk_ = 1;
  void* arena_ = nullptr;
  int* host_ = nullptr;   // pinned: active count
  double *vphi_ = nullptr, *vol_ = nullptr, *tx_ = nullptr, *dx_ = nullptr, *ty_ = nullptr,
         *dy_ = nullptr, *qin_ = nullptr, *qin0_ = nullptr, *vphi_r_ = nullptr;
  double *p_ = nullptr, *c_ = nullptr, *c_old_ = nullptr, *p_prev_ = nullptr, *J_ = nullptr,
         *b_ = nullptr, *x_ = nullptr, *kv_[6] = {}, *kS_ = nullptr, *kpart_ = nullptr,
         *partial_ = nullptr, *res0_ = nullptr, *res_last_ = nullptr;
  int *active_ = nullptr, *it_step_ = nullptr, *status_w_ = nullptr, *iters_w_ = nullptr,
      *n_active_ = nullptr, *step_ = nullptr;
  unsigned int* acc_ = nullptr;
  unsigned long long* counter_ = nullptr;
};

// Context-free residual (and Jacobian) of the vertex-centred scheme for B
// states (henry_residual_jacobian_vc); scratch: 7 n + 2 rows doubles, n =
// B nx (ny + 1), rows = B (ny + 1).
cudaError_t launch_vc_residual_jacobian(const Phys& P, int nx, int ny, int model, int n_xi,
                                        double tau, int B, const double* xi, const double* p,
                                        const double* c, const double* c_old, double* R,
                                        double* J, double* scratch, cudaStream_t s);

}  // namespace henry
