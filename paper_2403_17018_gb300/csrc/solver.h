// Host-side solver of one grid level of the Henry problem (one "role" of an
// MLMC level pair). Owns the device workspace of its batch and issues the
// kernels of the time loop: per implicit Euler step, Newton defect
// correction with geometric-multigrid V-cycles (arxiv 2403.17018, section
// 2.3).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/henry.h"
#include "common.cuh"
#include "henry_device.cuh"

namespace henry {

struct MGLevel {
  Geom g;
  void* J = nullptr;     // T [B][20][ncell], colour-split planes
  void* b = nullptr;     // T [B][2][ncell]
  void* x = nullptr;     // T [B][2][ncell]
  void* x2 = nullptr;    // T [B][2][ncell], the other copy for temporally blocked legs
  double* p = nullptr;   // state at this level (finest: the solver's p)
  double* c = nullptr;
  double* phi = nullptr;
  double* K = nullptr;
  double* tx = nullptr;  // face constants
  double* dx = nullptr;
  double* ty = nullptr;
  double* dy = nullptr;
  double* qx = nullptr;  // face fluxes of the linearisation point (east / right side)
  double* qy = nullptr;  // (north faces)
};

// Build the multigrid hierarchy of an nx x ny grid: halve while nx is a
// multiple of 4, ny is even and the coarse grid keeps at least 8 cells.
// Returns false if the coarsest grid has more than 32 cells or an odd nx.
bool build_hierarchy(int nx, int ny, double Lx, double Ly, std::vector<Geom>& out);

class Solver;

// The body graph of one step's conditional while node, captured after the
// capture of the enclosing graph has ended.
struct StepBody {
  Solver* solver;
  cudaGraph_t body;
  unsigned long long cond;   // cudaGraphConditionalHandle of the node
};

class Solver {
 public:
  Solver(const henry_config& cfg, int nx, int ny, int nt);
  ~Solver();
  Solver(const Solver&) = delete;
  Solver& operator=(const Solver&) = delete;

  // Batched solve; see henry_solve in henry.h. status_or != 0 ORs the
  // per-sample status into `status` instead of overwriting it.
  int run(const double* xi, const double* logk, int B, double* q, double* c_out, double* p_out,
          int* status, int* iters, int status_or, cudaStream_t s);
  // run() that also stores the QoIs after steps every, 2 every, ...:
  // series [B][nt / every][kNQ]
  int run_series(const double* xi, const double* logk, int B, int every, double* series,
                 double* q, int* status, cudaStream_t s);
  // Discrete adjoint of QoI `qoi` (0 Q_S, 2 toe); see henry_adjoint.
  int adjoint(const double* xi, const double* logk, int B, int qoi, int ckpt_every, double* q,
              double* dq_dxi, double* dq_dlogk, int* status, cudaStream_t s);
  // A solve split for callers that drive the time steps themselves (one
  // graph for the steps of several solvers): begin() evaluates the fields
  // and the initial state, capture_steps() records `nsteps` implicit steps
  // on a stream that is capturing into graph g (bodies to be captured with
  // capture_body() after that capture ends), finish() computes the QoIs and
  // copies (or ORs) the status.
  int begin(const double* xi, const double* logk, int B, cudaStream_t s);
  int capture_steps(cudaGraph_t g, cudaStream_t cs, int B, int nsteps,
                    std::vector<StepBody>& bodies);
  int capture_body(const StepBody& sb, int B, cudaStream_t bs);
  int finish(int B, double* q, double* c_out, double* p_out, int* status, int* iters,
             int status_or, cudaStream_t s);
  // Fields only (henry_fields).
  int fields(const double* xi, const double* logk, int B, double* phi, double* K, double* qin,
             cudaStream_t s);

  const Geom& fine() const { return levels_.back().g; }
  int nt() const { return nt_; }
  int n_mg() const { return (int)levels_.size(); }
  unsigned long long launches() const;
  // Time one kernel of the finest level (see henry_time_kernel).
  int time_kernel(int which, int reps, cudaStream_t s, void* flush, int64_t flush_bytes,
                  double* avg_ms, double* bytes, double* flops);
  int batch() const { return last_B_; }
  // Incremented whenever the workspace is reallocated (graphs recorded on
  // the old workspace must be rebuilt).
  unsigned long long generation() const { return generation_; }
  // Scheduling priority given to the kernel nodes of graphs this solver
  // captures (the stream-priority scale; 0 leaves them unset), and the
  // helper that applies it to every kernel node of a captured graph.
  void set_priority(int p) { prio_ = p; }
  int priority() const { return prio_; }
  const unsigned long long* launch_counter() const { return counter_; }
  static cudaError_t set_node_priority(cudaGraphNode_t node, int p);
  // Copy an internal array (see henry_debug_copy); returns HENRY_* code.
  int debug_copy(int mg_level, int what, void* dst, int64_t bytes) const;

 private:
  template <typename T> int run_t(const double* xi, const double* logk, int B, double* q,
                                  double* c_out, double* p_out, int* status, int* iters,
                                  int status_or, cudaStream_t s);
  template <typename T> int setup_t(const double* xi, const double* logk, int B, cudaStream_t s);
  template <typename T> int step_t(int B, cudaStream_t s);
  template <typename T> void enqueue_coarse_ops(int B, cudaStream_t s, const int* refresh);
  template <typename T> void enqueue_coarse_inv(int B, cudaStream_t s, const int* refresh);
  template <typename T> void enqueue_vcycles(int B, cudaStream_t s);
  template <typename T> void enqueue_precond(int B, cudaStream_t s);
  template <typename T> void enqueue_bicgstab(int B, cudaStream_t s);
  template <typename T> void enqueue_iteration(int B, cudaStream_t s);
  template <typename T> void enqueue_rebuild(int B, cudaStream_t s);
  template <typename T> void enqueue_solve_update(int B, cudaStream_t s);
  template <typename T> void enqueue_vcycle(int k, int B, cudaStream_t s);
  template <typename T> void enqueue_resjac_check(int B, cudaStream_t s, bool set_cond,
                                                  unsigned long long cond = 0);
  template <typename T> int capture_step_t(cudaGraph_t g, cudaStream_t cs, int B,
                                           std::vector<StepBody>& bodies);
  template <typename T> int capture_body_t(const StepBody& sb, int B, cudaStream_t bs);
  template <typename T> int step_graph(int B, cudaStream_t s);
  template <typename T> void launch_timed(int which, int B, cudaStream_t s);
  template <typename T> void launch_small(int B, int ncycles, cudaStream_t s);
  template <typename T> void launch_cluster(int B, int ncycles, cudaStream_t s);
  int ensure(int B, cudaStream_t s);
  int ensure_adjoint(int B, int nckpt, int seglen);
  template <typename T> int adjoint_t(const double* xi, const double* logk, int B, int qoi, int kc,
                                      double* q, double* dq_dxi, double* dq_dlogk, int* status,
                                      cudaStream_t s);
  void free_all();

  henry_config cfg_;
  Phys phys_;
  int nt_;
  double tau_;
  size_t tsize_;              // sizeof(T) of the multigrid arrays
  std::vector<Geom> geoms_;   // 0 = coarsest
  std::vector<MGLevel> levels_;
  int cap_ = 0;               // allocated batch capacity
  unsigned long long generation_ = 0;
  int last_B_ = 0;            // batch of the last solve
  void* arena_ = nullptr;
  // finest-level / per-sample arrays
  double* c_old_ = nullptr;
  double* p_prev_ = nullptr;    // p of the previous step (initial-guess extrapolation)
  GuessHist hx_ = {};           // u^(n-2), ... for guesses of order >= 2
  // previous states the Newton guess reads beyond u^(n-1)
  void launch_begin_step(int B, cudaStream_t s);
  int guess_depth() const {
    const int d = cfg_.guess_extrapolation - 1;
    return d < 0 ? 0 : (d > kMaxGuessHist ? kMaxGuessHist : d);
  }
  // state components per adjoint checkpoint: u, u^(n-1) and the older
  // states of the guess
  size_t ckpt_width() const { return 4 + 2 * (size_t)guess_depth(); }
  double* mo_ = nullptr;        // old-time storage terms of the step (k_resid)
  double* so_ = nullptr;
  double* vt_ = nullptr;        // V phi / tau per cell (k_resid)
  int* step_ = nullptr;         // completed steps of the current solve (device)
  double* qin_ = nullptr;
  double* qin0_ = nullptr;     // inflow base of the paper field model (time factor per step)
  double* partial_ = nullptr;
  double* res0_ = nullptr;
  double* res_last_ = nullptr;
  char* cinv_ = nullptr;      // transposed inverse of the coarsest operator (multigrid type)
  int* active_ = nullptr;
  int* refresh_ = nullptr;      // per sample: rebuild operators next iteration (jac_lag)
  int* it_step_ = nullptr;
  int* status_w_ = nullptr;
  int* iters_w_ = nullptr;
  int* n_active_ = nullptr;     // device: active samples, samples rebuilding operators
  void* kry_v_[6] = {};           // BiCGStab vectors r, rh, p, v, t, xk (krylov_iters > 0)
  double* kry_S_ = nullptr;       // per-sample BiCGStab scalars [B][kKryS]
  double* kry_part_ = nullptr;    // dot-product partials [2][B][kry_nchunk_]
  int kry_nchunk_ = 1;
  double* series_ = nullptr;      // QoI time series output of run_series (else NULL)
  int series_every_ = 0;
  unsigned int* check_acc_ = nullptr;  // k_check's block count / active count (2 words)
  int* n_active_host_ = nullptr;  // pinned
  unsigned long long* counter_ = nullptr;  // device launch counter
  int prio_ = 0;
  int* keep_ = nullptr;       // device flag: operators kept across steps (k_check)
  int nchunk_ = 0;            // residual blocks per sample
  ResTile tile_{};            // tiling of the residual kernel
  int ks_ = 0;                // top multigrid level handled by k_vcycle_small
  int kc_ = 0;                // top multigrid level handled by k_vcycle_cluster
  int cl_ = 1;                // blocks per cluster (one cluster per sample)
  std::vector<char> tb_;      // per multigrid level: legs temporally blocked
  std::vector<TbTile> tbd_, tbu_;   // tiles of the down (halo 2 nu1 + 1) and up legs
  // CUDA graph of one time step (HENRY_LOOP_GRAPH), rebuilt when B changes
  cudaGraphExec_t step_exec_ = nullptr;
  cudaGraph_t step_graph_ = nullptr;
  int graph_B_ = -1;
  // adjoint workspace (allocated on the first henry_adjoint call)
  void* adj_arena_ = nullptr;
  int adj_B_ = 0, adj_nckpt_ = 0, adj_seg_ = 0, adj_nchunk_ = 0;
  double *ckpt_ = nullptr, *seg_ = nullptr, *J64_ = nullptr, *lam_ = nullptr, *rhs_ = nullptr;
  double *res_ = nullptr, *gK_ = nullptr, *gphi_ = nullptr, *gq_ = nullptr, *qtmp_ = nullptr;
  double* partial2_ = nullptr;
  std::vector<void*> JT_;     // transposed operators per multigrid level
};

void set_last_error(const std::string& msg);
const char* last_error_cstr();

}  // namespace henry
