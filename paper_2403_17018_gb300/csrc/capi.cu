// C ABI of libhenry (declarations and documentation in include/henry.h).
#include <cuda_runtime.h>

#include <cmath>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "../../include/henry.h"
#include "solver.h"
#include "vc.h"

namespace henry {
cudaError_t launch_level_stats(unsigned long long* ctr, int B, const double* qf, const double* qc,
                               const int* status, double* out, cudaStream_t s);
cudaError_t launch_field_exceed(unsigned long long* ctr, int ncell, int B, const double* c,
                                const int* status, double threshold, int64_t* count,
                                cudaStream_t s);
cudaError_t launch_field_stats(unsigned long long* ctr, int nx, int ny, int B, const double* cf,
                               const double* cc, const int* status, int64_t* n, double* mean_f,
                               double* m2_f, double* mean_d, double* m2_d, cudaStream_t s);
cudaError_t launch_residual_jacobian(const Phys& P, const Geom& G, double tau, int B,
                                     const double* phi, const double* K, const double* qin,
                                     const double* p, const double* c, const double* c_old,
                                     double* R, double* J, double* scratch, cudaStream_t s);
int or_status(const int* src, int* dst, int B, unsigned long long* ctr, cudaStream_t s);
constexpr int kProbeThreads = 152 * 8 * 256;
cudaError_t probe_fp64(int reps, double* out, cudaStream_t s, double* tflops);
}  // namespace henry

using henry::Solver;

struct henry_ctx {
  henry_config cfg;
  // per MLMC level l: the context's config with level l's schedule
  // (henry_set_schedule); used by the fine solver of level l and by the
  // coarse half (level l-1) of the pairs of level l
  std::vector<henry_config> level_cfg;
  int device = 0;
  // solvers per level: [0] fine role, [1] coarse role (level l-1 of a pair)
  std::vector<std::unique_ptr<Solver>> role[2];
  std::vector<std::unique_ptr<henry::VcSolver>> vc_role[2];   // discretisation = vertex
  // per level: stream, events and status buffer of the concurrently run
  // coarse half of a pair (created on first use)
  std::vector<cudaStream_t> pair_stream;
  std::vector<cudaEvent_t> pair_fork, pair_join;
  std::vector<int> pair_prio;        // priority each pair_stream was created with
  std::vector<int*> pair_status;
  std::vector<int> pair_status_cap;
  double* stats_dev = nullptr;         // 1 + 4*NQ doubles
  double* stats_host = nullptr;        // pinned
  unsigned long long* ctr = nullptr;   // launches outside the solvers
  // henry_sample_levels: the graph of one coarse time step (every solver's
  // chain of implicit steps as a parallel branch), its key (solvers,
  // batches, steps, workspace generations) and the capture streams/events
  cudaGraph_t multi_graph = nullptr;
  cudaGraphExec_t multi_exec = nullptr;
  std::vector<long long> multi_key;
  std::vector<cudaStream_t> multi_streams;
  std::vector<cudaEvent_t> multi_events;
};

namespace {

int fail(int code, const std::string& msg) {
  henry::set_last_error(msg);
  return code;
}

#define CKR(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(e_ == cudaErrorMemoryAllocation ? HENRY_E_NOMEM : HENRY_E_CUDA,   \
                  std::string(#call) + ": " + cudaGetErrorString(e_));              \
  } while (0)

int level_dims(const henry_config& c, int level, int* nx, int* ny, int* nt) {
  if (level < 0 || level >= c.nlevels) return HENRY_E_INVALID;
  *nx = c.nx0 << level;
  *ny = c.ny0 << level;
  *nt = c.nt0 << level;
  return HENRY_OK;
}

Solver* get_solver(henry_ctx* ctx, int level, int role) {
  auto& v = ctx->role[role];
  if (!v[level]) {
    int nx, ny, nt;
    level_dims(ctx->cfg, level, &nx, &ny, &nt);
    // role 1 solves level l-1 for the pairs of level l: that level's schedule
    const henry_config& c = ctx->level_cfg[role == 0 ? level : level + 1];
    v[level].reset(new Solver(c, nx, ny, nt));
  }
  return v[level].get();
}

henry::VcSolver* get_vc_solver(henry_ctx* ctx, int level, int role) {
  auto& v = ctx->vc_role[role];
  if (!v[level]) {
    int nx, ny, nt;
    level_dims(ctx->cfg, level, &nx, &ny, &nt);
    const henry_config& c = ctx->level_cfg[role == 0 ? level : level + 1];
    v[level].reset(new henry::VcSolver(c, nx, ny, nt));
  }
  return v[level].get();
}

bool is_vertex(const henry_ctx* ctx) { return ctx->cfg.discretisation == HENRY_DISC_VERTEX; }

void drop_multi_graph(henry_ctx* ctx) {
  if (ctx->multi_exec) cudaGraphExecDestroy(ctx->multi_exec);
  if (ctx->multi_graph) cudaGraphDestroy(ctx->multi_graph);
  ctx->multi_exec = nullptr;
  ctx->multi_graph = nullptr;
  ctx->multi_key.clear();
}

int validate(const henry_config* c) {
  if (!c) return fail(HENRY_E_INVALID, "config is NULL");
  if (c->nlevels < 1 || c->nlevels > 12) return fail(HENRY_E_INVALID, "nlevels must be in 1..12");
  if (c->nx0 < 2 || c->ny0 < 2 || c->nt0 < 1) return fail(HENRY_E_INVALID, "bad level-0 grid");
  if (c->n_xi != 3 && c->n_xi != 6) return fail(HENRY_E_INVALID, "n_xi must be 3 or 6");
  if (c->precision != HENRY_PREC_FP64 && c->precision != HENRY_PREC_FP32_MG)
    return fail(HENRY_E_INVALID, "bad precision");
  if (c->loop_mode != HENRY_LOOP_HOST && c->loop_mode != HENRY_LOOP_GRAPH)
    return fail(HENRY_E_INVALID, "bad loop_mode");
  if (!(c->T > 0) || !(c->Lx > 0) || !(c->Ly > 0) || !(c->mu > 0) || !(c->K0 > 0) ||
      !(c->phi0 > 0) || !(c->D >= 0))
    return fail(HENRY_E_INVALID, "non-positive physical parameter");
  if (c->newton_maxit < 0 || c->nu1 < 0 || c->nu2 < 0 || c->vcycles < 1 || c->mg_cluster_cells < 0 ||
      c->mg_small_cells < 0 || c->mg_small_cells > 512 || c->jac_lag < 0 ||
      c->field_model < 0 || c->field_model > 1 || (c->field_model == 1 && c->n_xi != 3) ||
      c->krylov_iters < 0 || c->krylov_iters > 64)
    return fail(HENRY_E_INVALID, "bad solver parameter");
  if (c->krylov_iters == 1)
    return fail(HENRY_E_INVALID, "krylov_iters = 1 is rejected (BiCGStab breakdown); use 0 or >= 2");
  if (!(c->adjoint_rtol > 0.0) || !(c->adjoint_rtol < 1e-3))
    return fail(HENRY_E_INVALID, "adjoint_rtol must be in (0, 1e-3)");
  if (c->res_rows < 0 || c->res_rows > 64) return fail(HENRY_E_INVALID, "res_rows must be in 0..64");
  if (c->mg_tb_cells < 0) return fail(HENRY_E_INVALID, "mg_tb_cells must be >= 0");
  if (c->jac_keep != 0 && c->jac_keep != 1) return fail(HENRY_E_INVALID, "jac_keep must be 0 or 1");
  if (c->guess_extrapolation < 0 || c->guess_extrapolation > 1 + henry::kMaxGuessHist)
    return fail(HENRY_E_INVALID, "guess_extrapolation must be in 0..6");
  if (c->discretisation != HENRY_DISC_CELL && c->discretisation != HENRY_DISC_VERTEX)
    return fail(HENRY_E_INVALID, "discretisation must be HENRY_DISC_CELL or HENRY_DISC_VERTEX");
  if (c->discretisation == HENRY_DISC_VERTEX && (c->nx0 % 2 || c->ny0 < 1))
    return fail(HENRY_E_INVALID, "the vertex-centred variant needs an even nx0");
  for (int l = 0; l < c->nlevels; ++l) {
    std::vector<henry::Geom> g;
    if (!henry::build_hierarchy(c->nx0 << l, c->ny0 << l, c->Lx, c->Ly, g))
      return fail(HENRY_E_UNSUPPORTED, "level " + std::to_string(l) +
                                           " does not coarsen to <= 32 cells with even nx");
  }
  return HENRY_OK;
}

}  // namespace

extern "C" {

int henry_default_config(henry_config* c) {
  if (!c) return fail(HENRY_E_INVALID, "config is NULL");
  *c = henry_config{};
  c->rho0 = 1000.0;
  c->rho1 = 1024.99;
  c->mu = 1e-3;
  c->g = 9.8;
  c->D = 18.8571e-6;
  c->K0 = 1.020408e-9;
  c->phi0 = 0.35;
  c->q0 = 6.6e-5;
  c->Lx = 2.0;
  c->Ly = 1.0;
  c->T = 43200.0;
  c->nx0 = 32;
  c->ny0 = 16;
  c->nt0 = 24;
  c->nlevels = 2;
  c->n_xi = 3;
  c->precision = HENRY_PREC_FP64;
  c->loop_mode = HENRY_LOOP_GRAPH;
  c->newton_rtol = 1e-10;
  c->newton_atol = 1e-11;
  c->newton_maxit = 30;
  c->nu1 = 2;
  c->nu2 = 2;
  c->vcycles = 3;
  c->guess_extrapolation = 4;
  c->newton_stag_tol = 1e-9;
  c->mg_fusion = 1;
  c->mg_cluster_cells = 0;
  c->mg_small_cells = 512;
  c->jac_lag = 0;
  c->field_model = 0;
  c->krylov_iters = 0;
  c->adjoint_rtol = 1e-14;
  c->mg_tb_cells = 0;
  c->jac_keep = 0;
  return HENRY_OK;
}

int henry_create_levels(const henry_config* cfg, henry_ctx** out) {
  if (!out) return fail(HENRY_E_INVALID, "out is NULL");
  *out = nullptr;
  int rc = validate(cfg);
  if (rc) return rc;
  henry_ctx* ctx = new (std::nothrow) henry_ctx;
  if (!ctx) return fail(HENRY_E_NOMEM, "host allocation failed");
  ctx->cfg = *cfg;
  ctx->level_cfg.assign(cfg->nlevels, *cfg);
  ctx->role[0].resize(cfg->nlevels);
  ctx->role[1].resize(cfg->nlevels);
  ctx->vc_role[0].resize(cfg->nlevels);
  ctx->vc_role[1].resize(cfg->nlevels);
  ctx->pair_stream.assign(cfg->nlevels, nullptr);
  ctx->pair_fork.assign(cfg->nlevels, nullptr);
  ctx->pair_join.assign(cfg->nlevels, nullptr);
  ctx->pair_prio.assign(cfg->nlevels, 0);
  ctx->pair_status.assign(cfg->nlevels, nullptr);
  ctx->pair_status_cap.assign(cfg->nlevels, 0);
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->stats_dev, sizeof(double) * (1 + 4 * HENRY_NQ) + 64);
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&ctx->stats_host, sizeof(double) * (1 + 4 * HENRY_NQ), 0);
  if (e == cudaSuccess) {
    ctx->ctr = (unsigned long long*)((char*)ctx->stats_dev + sizeof(double) * (1 + 4 * HENRY_NQ) + 32);
    e = cudaMemset(ctx->ctr, 0, sizeof(unsigned long long));
  }
  if (e != cudaSuccess) {
    henry_destroy(ctx);
    return fail(HENRY_E_CUDA, std::string("context set-up: ") + cudaGetErrorString(e));
  }
  *out = ctx;
  return HENRY_OK;
}

void henry_destroy(henry_ctx* ctx) {
  if (!ctx) return;
  cudaDeviceSynchronize();
  drop_multi_graph(ctx);
  for (cudaStream_t st : ctx->multi_streams) cudaStreamDestroy(st);
  for (cudaEvent_t ev : ctx->multi_events) cudaEventDestroy(ev);
  for (auto& v : ctx->role) v.clear();
  for (auto& v : ctx->vc_role) v.clear();
  for (size_t l = 0; l < ctx->pair_stream.size(); ++l) {
    if (ctx->pair_stream[l]) cudaStreamDestroy(ctx->pair_stream[l]);
    if (ctx->pair_fork[l]) cudaEventDestroy(ctx->pair_fork[l]);
    if (ctx->pair_join[l]) cudaEventDestroy(ctx->pair_join[l]);
    if (ctx->pair_status[l]) cudaFree(ctx->pair_status[l]);
  }
  if (ctx->stats_dev) cudaFree(ctx->stats_dev);
  if (ctx->stats_host) cudaFreeHost(ctx->stats_host);
  delete ctx;
}

int henry_level_info(const henry_ctx* ctx, int level, int* nx, int* ny, int* nt, int* n_mg) {
  if (!ctx || !nx || !ny || !nt || !n_mg) return fail(HENRY_E_INVALID, "NULL argument");
  if (level_dims(ctx->cfg, level, nx, ny, nt)) return fail(HENRY_E_INVALID, "bad level");
  std::vector<henry::Geom> g;
  henry::build_hierarchy(*nx, *ny, ctx->cfg.Lx, ctx->cfg.Ly, g);
  *n_mg = (int)g.size();
  return HENRY_OK;
}

int henry_solve(henry_ctx* ctx, int level, const double* xi, const double* logk, int B, double* q,
                double* c_out, double* p_out, int* status, int* iters, void* stream) {
  if (!ctx) return fail(HENRY_E_INVALID, "ctx is NULL");
  if (level < 0 || level >= ctx->cfg.nlevels) return fail(HENRY_E_INVALID, "bad level");
  if (B < 0 || B > HENRY_MAX_BATCH) return fail(HENRY_E_INVALID, "B must be in 0..65535");
  if (B == 0) return HENRY_OK;
  if (!xi || !q || !status) return fail(HENRY_E_INVALID, "xi, q and status are required");
  CKR(cudaSetDevice(ctx->device));
  if (is_vertex(ctx)) {
    if (logk) return fail(HENRY_E_UNSUPPORTED, "the vertex-centred variant takes no log-K field");
    return get_vc_solver(ctx, level, 0)->run(xi, B, q, c_out, p_out, status, iters, 0,
                                             (cudaStream_t)stream);
  }
  return get_solver(ctx, level, 0)->run(xi, logk, B, q, c_out, p_out, status, iters, 0,
                                        (cudaStream_t)stream);
}

int henry_solve_series(henry_ctx* ctx, int level, const double* xi, const double* logk, int B,
                       int every, double* q_series, double* q, int* status, void* stream) {
  if (!ctx) return fail(HENRY_E_INVALID, "ctx is NULL");
  if (level < 0 || level >= ctx->cfg.nlevels) return fail(HENRY_E_INVALID, "bad level");
  if (B < 0 || B > HENRY_MAX_BATCH) return fail(HENRY_E_INVALID, "B must be in 0..65535");
  if (every < 1) return fail(HENRY_E_INVALID, "every must be >= 1");
  if (B == 0) return HENRY_OK;
  if (!xi || !q_series || !q || !status)
    return fail(HENRY_E_INVALID, "xi, q_series, q and status are required");
  if (is_vertex(ctx)) return fail(HENRY_E_UNSUPPORTED, "no QoI series for the vertex-centred variant");
  CKR(cudaSetDevice(ctx->device));
  return get_solver(ctx, level, 0)->run_series(xi, logk, B, every, q_series, q, status,
                                               (cudaStream_t)stream);
}

int henry_sample_pairs(henry_ctx* ctx, int level, const double* xi, int B, double* q_fine,
                       double* q_coarse, double* c_fine, double* c_coarse, int* status,
                       void* stream) {
  if (!ctx) return fail(HENRY_E_INVALID, "ctx is NULL");
  if (level < 0 || level >= ctx->cfg.nlevels) return fail(HENRY_E_INVALID, "bad level");
  if (B < 0 || B > HENRY_MAX_BATCH) return fail(HENRY_E_INVALID, "B must be in 0..65535");
  if (level == 0 && (q_coarse || c_coarse))
    return fail(HENRY_E_INVALID, "level 0 has no coarse solve: q_coarse and c_coarse must be NULL");
  if (level > 0 && !q_coarse) return fail(HENRY_E_INVALID, "q_coarse is required for level > 0");
  if (B == 0) return HENRY_OK;
  if (!xi || !q_fine || !status) return fail(HENRY_E_INVALID, "xi, q_fine and status are required");
  CKR(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (is_vertex(ctx)) {   // the two halves one after the other on `stream`
    int rc = get_vc_solver(ctx, level, 0)->run(xi, B, q_fine, c_fine, nullptr, status, nullptr, 0, s);
    if (rc || level == 0) return rc;
    return get_vc_solver(ctx, level - 1, 1)->run(xi, B, q_coarse, c_coarse, nullptr, status,
                                                 nullptr, 1, s);
  }
  if (level == 0)
    return get_solver(ctx, 0, 0)->run(xi, nullptr, B, q_fine, c_fine, nullptr, status, nullptr, 0, s);
  // the coarse half runs concurrently on a stream forked from the caller's,
  // with the caller's stream priority
  int prio = 0;
  CKR(cudaStreamGetPriority(s, &prio));
  if (ctx->pair_stream[level] && ctx->pair_prio[level] != prio) {
    CKR(cudaStreamSynchronize(ctx->pair_stream[level]));
    CKR(cudaStreamDestroy(ctx->pair_stream[level]));
    ctx->pair_stream[level] = nullptr;
  }
  if (!ctx->pair_stream[level]) {
    CKR(cudaStreamCreateWithPriority(&ctx->pair_stream[level], cudaStreamNonBlocking, prio));
    ctx->pair_prio[level] = prio;
    if (!ctx->pair_fork[level]) {
      CKR(cudaEventCreateWithFlags(&ctx->pair_fork[level], cudaEventDisableTiming));
      CKR(cudaEventCreateWithFlags(&ctx->pair_join[level], cudaEventDisableTiming));
    }
  }
  if (ctx->pair_status_cap[level] < B) {
    CKR(cudaStreamSynchronize(ctx->pair_stream[level]));
    if (ctx->pair_status[level]) CKR(cudaFree(ctx->pair_status[level]));
    ctx->pair_status[level] = nullptr;
    CKR(cudaMalloc(&ctx->pair_status[level], sizeof(int) * B));
    ctx->pair_status_cap[level] = B;
  }
  cudaStream_t sc = ctx->pair_stream[level];
  CKR(cudaEventRecord(ctx->pair_fork[level], s));
  CKR(cudaStreamWaitEvent(sc, ctx->pair_fork[level], 0));
  int rc = get_solver(ctx, level - 1, 1)->run(xi, nullptr, B, q_coarse, c_coarse, nullptr,
                                              ctx->pair_status[level], nullptr, 0, sc);
  if (rc) return rc;
  CKR(cudaEventRecord(ctx->pair_join[level], sc));
  rc = get_solver(ctx, level, 0)->run(xi, nullptr, B, q_fine, c_fine, nullptr, status, nullptr, 0, s);
  if (rc) return rc;
  CKR(cudaStreamWaitEvent(s, ctx->pair_join[level], 0));
  return henry::or_status(ctx->pair_status[level], status, B, ctx->ctr, s);
}

int henry_set_schedule(henry_ctx* ctx, int level, const henry_schedule* sc) {
  if (!ctx || !sc) return fail(HENRY_E_INVALID, "NULL argument");
  if (level < 0 || level >= ctx->cfg.nlevels) return fail(HENRY_E_INVALID, "bad level");
  henry_config c = ctx->cfg;
  c.vcycles = sc->vcycles;
  c.nu1 = sc->nu1;
  c.nu2 = sc->nu2;
  c.mg_small_cells = sc->mg_small_cells;
  c.jac_lag = sc->jac_lag;
  c.res_rows = sc->res_rows;
  c.mg_tb_cells = sc->mg_tb_cells;
  c.jac_keep = sc->jac_keep;
  const int rc = validate(&c);
  if (rc) return rc;
  CKR(cudaSetDevice(ctx->device));
  CKR(cudaDeviceSynchronize());
  drop_multi_graph(ctx);
  ctx->level_cfg[level] = c;
  ctx->role[0][level].reset();
  if (level > 0) ctx->role[1][level - 1].reset();
  return HENRY_OK;
}

int henry_sample_levels(henry_ctx* ctx, const henry_level_batch* batches, int n, void* stream) {
  if (!ctx || !batches) return fail(HENRY_E_INVALID, "NULL argument");
  if (n < 1 || n > ctx->cfg.nlevels) return fail(HENRY_E_INVALID, "n must be in 1..nlevels");
  std::vector<int> seen(ctx->cfg.nlevels, 0);
  for (int i = 0; i < n; ++i) {
    const henry_level_batch& b = batches[i];
    if (b.level < 0 || b.level >= ctx->cfg.nlevels) return fail(HENRY_E_INVALID, "bad level");
    if (seen[b.level]++) return fail(HENRY_E_INVALID, "a level appears twice");
    if (b.B < 0 || b.B > HENRY_MAX_BATCH) return fail(HENRY_E_INVALID, "B must be in 0..65535");
    if (b.B == 0) continue;
    if (!b.xi || !b.q_fine || !b.status) return fail(HENRY_E_INVALID, "xi, q_fine and status are required");
    if (b.level == 0 && (b.q_coarse || b.c_coarse))
      return fail(HENRY_E_INVALID, "level 0 has no coarse solve: q_coarse and c_coarse must be NULL");
    if (b.level > 0 && !b.q_coarse) return fail(HENRY_E_INVALID, "q_coarse is required for level > 0");
  }
  CKR(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (ctx->cfg.loop_mode == HENRY_LOOP_HOST || is_vertex(ctx)) {
    // host-side Newton loops: the pairs one level after another
    for (int i = 0; i < n; ++i) {
      const henry_level_batch& b = batches[i];
      const int rc = henry_sample_pairs(ctx, b.level, b.xi, b.B, b.q_fine, b.q_coarse, b.c_fine,
                                        b.c_coarse, b.status, stream);
      if (rc) return rc;
    }
    return HENRY_OK;
  }
  // the chains of implicit steps: per coarse step, level l advances 2^l steps
  struct Chain { Solver* sv; int B; int steps; };
  std::vector<Chain> chains;
  // scheduling priorities: the finest level's chain is the critical path of
  // a coarse step (the most dependent steps, the smallest batch), so its
  // kernels go first and the coarser levels' fill the SMs it leaves idle
  int least = 0, greatest = 0;
  CKR(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  int lmax = 0;
  for (int i = 0; i < n; ++i)
    if (batches[i].B > 0 && batches[i].level > lmax) lmax = batches[i].level;
  auto prio = [&](int level) {
    const int p = greatest + (lmax - level);   // greatest is the numerically lowest
    return p > least ? least : p;
  };
  for (int i = 0; i < n; ++i) {
    const henry_level_batch& b = batches[i];
    if (b.B == 0) continue;
    chains.push_back({get_solver(ctx, b.level, 0), b.B, 1 << b.level});
    chains.back().sv->set_priority(prio(b.level));
    if (b.level > 0) {
      chains.push_back({get_solver(ctx, b.level - 1, 1), b.B, 1 << (b.level - 1)});
      chains.back().sv->set_priority(prio(b.level));
    }
  }
  if (chains.empty()) return HENRY_OK;
  // fields and initial states (these may grow workspaces)
  for (int i = 0, k = 0; i < n; ++i) {
    const henry_level_batch& b = batches[i];
    if (b.B == 0) continue;
    int rc = chains[k++].sv->begin(b.xi, nullptr, b.B, s);
    if (!rc && b.level > 0) rc = chains[k++].sv->begin(b.xi, nullptr, b.B, s);
    if (rc) return rc;
  }
  std::vector<long long> key;
  for (const Chain& c : chains) {
    key.push_back((long long)(intptr_t)c.sv);
    key.push_back(c.B);
    key.push_back(c.steps);
    key.push_back((long long)c.sv->generation());
  }
  if (key != ctx->multi_key) {
    drop_multi_graph(ctx);
    while (ctx->multi_streams.size() < chains.size() + 2) {
      cudaStream_t st;
      CKR(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
      ctx->multi_streams.push_back(st);
    }
    while (ctx->multi_events.size() < chains.size() + 1) {
      cudaEvent_t ev;
      CKR(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
      ctx->multi_events.push_back(ev);
    }
    cudaStream_t cs = ctx->multi_streams[0], bs = ctx->multi_streams[1];
    cudaGraph_t g;
    CKR(cudaGraphCreate(&g, 0));
    std::vector<henry::StepBody> bodies;
    int rc = HENRY_OK;
    cudaError_t e = cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      e = cudaEventRecord(ctx->multi_events[0], cs);
      for (size_t i = 0; i < chains.size() && e == cudaSuccess && !rc; ++i) {
        cudaStream_t si = ctx->multi_streams[i + 2];
        e = cudaStreamWaitEvent(si, ctx->multi_events[0], 0);
        if (e == cudaSuccess) rc = chains[i].sv->capture_steps(g, si, chains[i].B, chains[i].steps, bodies);
        if (e == cudaSuccess && !rc) e = cudaEventRecord(ctx->multi_events[i + 1], si);
        if (e == cudaSuccess && !rc) e = cudaStreamWaitEvent(cs, ctx->multi_events[i + 1], 0);
      }
      cudaGraph_t gout = g;
      const cudaError_t e2 = cudaStreamEndCapture(cs, &gout);
      if (e == cudaSuccess) e = e2;
    }
    // the step nodes of the top graph: each kernel's first argument is the
    // launch counter of the solver that launched it
    if (e == cudaSuccess && !rc) {
      size_t nn = 0;
      e = cudaGraphGetNodes(g, nullptr, &nn);
      std::vector<cudaGraphNode_t> nodes(nn);
      if (e == cudaSuccess && nn) e = cudaGraphGetNodes(g, nodes.data(), &nn);
      for (size_t k = 0; k < nn && e == cudaSuccess; ++k) {
        cudaGraphNodeType t;
        e = cudaGraphNodeGetType(nodes[k], &t);
        if (e != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp = {};
        e = cudaGraphKernelNodeGetParams(nodes[k], &kp);
        if (e != cudaSuccess || !kp.kernelParams) continue;
        const unsigned long long* ctr = *(unsigned long long* const*)kp.kernelParams[0];
        for (const Chain& c : chains)
          if (c.sv->launch_counter() == ctr) {
            e = Solver::set_node_priority(nodes[k], c.sv->priority());
            break;
          }
      }
    }
    for (size_t k = 0; k < bodies.size() && e == cudaSuccess && !rc; ++k) {
      int B = 0;
      for (const Chain& c : chains)
        if (c.sv == bodies[k].solver) B = c.B;
      rc = bodies[k].solver->capture_body(bodies[k], B, bs);
    }
    if (e == cudaSuccess && !rc) {
      e = cudaGraphInstantiate(&ctx->multi_exec, g, cudaGraphInstantiateFlagUseNodePriority);
      if (e != cudaSuccess) {   // priorities are a scheduling hint: run without them
        cudaGetLastError();
        e = cudaGraphInstantiate(&ctx->multi_exec, g, 0);
      }
    }
    if (e != cudaSuccess || rc) {
      cudaGraphDestroy(g);
      ctx->multi_exec = nullptr;
      if (rc) return rc;
      return fail(HENRY_E_CUDA, std::string("henry_sample_levels graph: ") + cudaGetErrorString(e));
    }
    ctx->multi_graph = g;
    ctx->multi_key = key;
  }
  for (int k = 0; k < ctx->cfg.nt0; ++k) CKR(cudaGraphLaunch(ctx->multi_exec, s));
  for (int i = 0, k = 0; i < n; ++i) {
    const henry_level_batch& b = batches[i];
    if (b.B == 0) continue;
    int rc = chains[k++].sv->finish(b.B, b.q_fine, b.c_fine, nullptr, b.status, nullptr, 0, s);
    if (!rc && b.level > 0)
      rc = chains[k++].sv->finish(b.B, b.q_coarse, b.c_coarse, nullptr, b.status, nullptr, 1, s);
    if (rc) return rc;
  }
  return HENRY_OK;
}

int henry_adjoint(henry_ctx* ctx, int level, const double* xi, const double* logk, int B,
                  int qoi_id, int ckpt_every, double* q, double* dq_dxi, double* dq_dlogk,
                  int* status, void* stream) {
  if (!ctx) return fail(HENRY_E_INVALID, "ctx is NULL");
  if (level < 0 || level >= ctx->cfg.nlevels) return fail(HENRY_E_INVALID, "bad level");
  if (B < 0 || B > HENRY_MAX_BATCH) return fail(HENRY_E_INVALID, "B must be in 0..65535");
  if (qoi_id != 0 && qoi_id != 2) return fail(HENRY_E_INVALID, "qoi_id must be 0 (Q_S) or 2 (toe)");
  if (B == 0) return HENRY_OK;
  if (!xi || !q || !dq_dxi || !status) return fail(HENRY_E_INVALID, "xi, q, dq_dxi, status required");
  if (is_vertex(ctx)) return fail(HENRY_E_UNSUPPORTED, "no adjoint for the vertex-centred variant");
  CKR(cudaSetDevice(ctx->device));
  return get_solver(ctx, level, 0)->adjoint(xi, logk, B, qoi_id, ckpt_every, q, dq_dxi, dq_dlogk,
                                            status, (cudaStream_t)stream);
}

int henry_fields(henry_ctx* ctx, int level, const double* xi, const double* logk, int B,
                 double* phi, double* K, double* qin, void* stream) {
  if (!ctx) return fail(HENRY_E_INVALID, "ctx is NULL");
  if (level < 0 || level >= ctx->cfg.nlevels) return fail(HENRY_E_INVALID, "bad level");
  if (B < 0 || B > HENRY_MAX_BATCH) return fail(HENRY_E_INVALID, "B must be in 0..65535");
  if (B == 0) return HENRY_OK;
  if (!xi || !phi || !K || !qin) return fail(HENRY_E_INVALID, "NULL argument");
  if (is_vertex(ctx)) return fail(HENRY_E_UNSUPPORTED, "cell fields only (cell-centred variant)");
  CKR(cudaSetDevice(ctx->device));
  return get_solver(ctx, level, 0)->fields(xi, logk, B, phi, K, qin, (cudaStream_t)stream);
}

int mlmc_level_stats(henry_ctx* ctx, int level, const double* q_fine, const double* q_coarse,
                     int B, const int* status, henry_level_stats* inout, void* stream) {
  if (!ctx || !inout) return fail(HENRY_E_INVALID, "NULL argument");
  if (level < 0 || level >= ctx->cfg.nlevels) return fail(HENRY_E_INVALID, "bad level");
  if (B < 0) return fail(HENRY_E_INVALID, "B < 0");
  if (B == 0) return HENRY_OK;
  if (!q_fine) return fail(HENRY_E_INVALID, "q_fine is NULL");
  if (level == 0 && q_coarse) return fail(HENRY_E_INVALID, "level 0 takes no q_coarse");
  CKR(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  CKR(henry::launch_level_stats(ctx->ctr, B, q_fine, q_coarse, status, ctx->stats_dev, s));
  CKR(cudaMemcpyAsync(ctx->stats_host, ctx->stats_dev, sizeof(double) * (1 + 4 * HENRY_NQ),
                      cudaMemcpyDeviceToHost, s));
  CKR(cudaStreamSynchronize(s));
  const double* o = ctx->stats_host;
  const double nb = o[0];
  if (nb == 0.0) return HENRY_OK;
  const double na = (double)inout->n;
  const double n = na + nb;
  for (int k = 0; k < HENRY_NQ; ++k) {
    double d = o[1 + k] - inout->mean_f[k];
    inout->mean_f[k] += d * (nb / n);
    inout->m2_f[k] += o[1 + HENRY_NQ + k] + d * d * (na * nb / n);
    d = o[1 + 2 * HENRY_NQ + k] - inout->mean_d[k];
    inout->mean_d[k] += d * (nb / n);
    inout->m2_d[k] += o[1 + 3 * HENRY_NQ + k] + d * d * (na * nb / n);
  }
  inout->n += (int64_t)nb;
  return HENRY_OK;
}

int mlmc_field_stats(henry_ctx* ctx, int level, const double* c_fine, const double* c_coarse, int B,
                     const int* status, int64_t* n, double* mean_f, double* m2_f, double* mean_d,
                     double* m2_d, void* stream) {
  if (!ctx) return fail(HENRY_E_INVALID, "ctx is NULL");
  if (level < 0 || level >= ctx->cfg.nlevels) return fail(HENRY_E_INVALID, "bad level");
  if (B < 0) return fail(HENRY_E_INVALID, "B < 0");
  if (level == 0 && c_coarse) return fail(HENRY_E_INVALID, "level 0 takes no c_coarse");
  if (B == 0) return HENRY_OK;
  if (!c_fine || !n || !mean_f || !m2_f || !mean_d || !m2_d)
    return fail(HENRY_E_INVALID, "NULL argument");
  CKR(cudaSetDevice(ctx->device));
  const int nx = ctx->cfg.nx0 << level, ny = ctx->cfg.ny0 << level;
  CKR(henry::launch_field_stats(ctx->ctr, nx, ny, B, c_fine, c_coarse, status, n, mean_f, m2_f,
                                mean_d, m2_d, (cudaStream_t)stream));
  return HENRY_OK;
}

int mlmc_field_exceedance(henry_ctx* ctx, int level, const double* c, int B, const int* status,
                          double threshold, int64_t* count, void* stream) {
  if (!ctx) return fail(HENRY_E_INVALID, "ctx is NULL");
  if (level < 0 || level >= ctx->cfg.nlevels) return fail(HENRY_E_INVALID, "bad level");
  if (B < 0) return fail(HENRY_E_INVALID, "B < 0");
  if (!(threshold == threshold)) return fail(HENRY_E_INVALID, "threshold is NaN");
  if (B == 0) return HENRY_OK;
  if (!c || !count) return fail(HENRY_E_INVALID, "NULL argument");
  CKR(cudaSetDevice(ctx->device));
  const int ncell = (ctx->cfg.nx0 << level) * (ctx->cfg.ny0 << level);
  CKR(henry::launch_field_exceed(ctx->ctr, ncell, B, c, status, threshold, count,
                                 (cudaStream_t)stream));
  return HENRY_OK;
}

int henry_residual_jacobian(const henry_config* cfg, int nx, int ny, double tau, int B,
                            const double* phi, const double* K, const double* qin, const double* p,
                            const double* c, const double* c_old, double* R, double* J,
                            void* stream) {
  if (!cfg) return fail(HENRY_E_INVALID, "config is NULL");
  if (nx < 2 || ny < 1 || B < 0 || B > HENRY_MAX_BATCH || !(tau > 0))
    return fail(HENRY_E_INVALID, "bad sizes (nx >= 2, ny >= 1, 0 <= B <= 65535, tau > 0)");
  if (B == 0) return HENRY_OK;
  if (!phi || !K || !qin || !p || !c || !c_old || !R) return fail(HENRY_E_INVALID, "NULL argument");
  henry::Phys P{cfg->rho0, cfg->rho1 - cfg->rho0, cfg->mu, cfg->g, cfg->D, cfg->K0, cfg->phi0,
                cfg->q0, cfg->Lx, cfg->Ly};
  henry::Geom G{nx, ny, cfg->Lx / nx, cfg->Ly / ny};
  cudaStream_t s = (cudaStream_t)stream;
  double* scratch = nullptr;
  CKR(cudaMallocAsync((void**)&scratch, sizeof(double) * 5 * (size_t)B * nx * ny, s));
  cudaError_t e = henry::launch_residual_jacobian(P, G, tau, B, phi, K, qin, p, c, c_old, R, J,
                                                  scratch, s);
  cudaError_t e2 = cudaFreeAsync(scratch, s);
  CKR(e);
  CKR(e2);
  return HENRY_OK;
}

int henry_residual_jacobian_vc(const henry_config* cfg, int nx, int ny, double tau, int B,
                               const double* xi, const double* p, const double* c,
                               const double* c_old, double* R, double* J, void* stream) {
  if (!cfg) return fail(HENRY_E_INVALID, "config is NULL");
  if (nx < 2 || nx % 2 || ny < 1 || B < 0 || B > HENRY_MAX_BATCH || !(tau > 0))
    return fail(HENRY_E_INVALID, "bad sizes (even nx >= 2, ny >= 1, 0 <= B <= 65535, tau > 0)");
  if (cfg->n_xi != 3 && cfg->n_xi != 6) return fail(HENRY_E_INVALID, "n_xi must be 3 or 6");
  if (B == 0) return HENRY_OK;
  if (!xi || !p || !c || !c_old || !R) return fail(HENRY_E_INVALID, "NULL argument");
  henry::Phys P{cfg->rho0, cfg->rho1 - cfg->rho0, cfg->mu, cfg->g, cfg->D, cfg->K0, cfg->phi0,
                cfg->q0, cfg->Lx, cfg->Ly};
  cudaStream_t s = (cudaStream_t)stream;
  const size_t n = (size_t)B * nx * (ny + 1), rows = (size_t)B * (ny + 1);
  double* scratch = nullptr;
  CKR(cudaMallocAsync((void**)&scratch, sizeof(double) * (7 * n + 2 * rows), s));
  cudaError_t e = henry::launch_vc_residual_jacobian(P, nx, ny, cfg->field_model, cfg->n_xi, tau, B,
                                                     xi, p, c, c_old, R, J, scratch, s);
  cudaError_t e2 = cudaFreeAsync(scratch, s);
  CKR(e);
  CKR(e2);
  return HENRY_OK;
}

int henry_debug_copy(henry_ctx* ctx, int level, int role, int mg_level, int what, void* dst,
                     int64_t bytes) {
  if (!ctx || level < 0 || level >= ctx->cfg.nlevels || role < 0 || role > 1)
    return fail(HENRY_E_INVALID, "bad context, level or role");
  const auto& s = ctx->role[role][level];
  if (!s) return fail(HENRY_E_INVALID, "no solver has run for this level and role");
  CKR(cudaSetDevice(ctx->device));
  int rc = s->debug_copy(mg_level, what, dst, bytes);
  if (rc) return fail(rc, "debug_copy: bad index, empty workspace or copy failure");
  return HENRY_OK;
}

int henry_time_kernel(henry_ctx* ctx, int level, int role, int which, int reps, void* flush,
                      int64_t flush_bytes, void* stream, double* avg_ms, double* bytes,
                      double* flops) {
  if (!ctx || level < 0 || level >= ctx->cfg.nlevels || role < 0 || role > 1 || !avg_ms ||
      !bytes || !flops)
    return fail(HENRY_E_INVALID, "bad argument");
  if (is_vertex(ctx)) return fail(HENRY_E_UNSUPPORTED, "kernel timing of the cell-centred solver only");
  const auto& s = ctx->role[role][level];
  if (!s) return fail(HENRY_E_INVALID, "no solver has run for this level and role");
  CKR(cudaSetDevice(ctx->device));
  int rc = s->time_kernel(which, reps, (cudaStream_t)stream, flush, flush_bytes, avg_ms, bytes,
                          flops);
  if (rc) return fail(rc, "time_kernel failed (which, reps, flush buffer or no previous solve)");
  return HENRY_OK;
}

int henry_probe_fp64(int reps, void* stream, double* tflops) {
  if (reps < 1 || reps > 1000 || !tflops) return fail(HENRY_E_INVALID, "bad argument");
  double* out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  CKR(cudaMallocAsync((void**)&out, sizeof(double) * henry::kProbeThreads, s));
  const cudaError_t e = henry::probe_fp64(reps, out, s, tflops);
  const cudaError_t e2 = cudaFreeAsync(out, s);
  CKR(e);
  CKR(e2);
  return HENRY_OK;
}

int64_t henry_launch_count(const henry_ctx* ctx) {
  if (!ctx) return -1;
  unsigned long long total = 0, v = 0;
  cudaDeviceSynchronize();
  if (ctx->ctr && cudaMemcpy(&v, ctx->ctr, sizeof(v), cudaMemcpyDeviceToHost) == cudaSuccess) total += v;
  for (const auto& r : ctx->role)
    for (const auto& s : r)
      if (s) total += s->launches();
  for (const auto& r : ctx->vc_role)
    for (const auto& s : r)
      if (s) total += s->launches();
  return (int64_t)total;
}

const char* henry_strerror(int code) {
  switch (code) {
    case HENRY_OK: return "ok";
    case HENRY_E_INVALID: return "invalid argument";
    case HENRY_E_CUDA: return "CUDA error";
    case HENRY_E_NOMEM: return "out of device memory";
    case HENRY_E_UNSUPPORTED: return "unsupported grid";
    default: return "unknown error";
  }
}

const char* henry_last_error(void) { return henry::last_error_cstr(); }

}  // extern "C"
