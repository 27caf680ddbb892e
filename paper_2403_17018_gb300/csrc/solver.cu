// Host orchestration of the batched Henry solve (see solver.h).
#include "solver.h"

#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "kernels.cuh"
#include "tb.cuh"

namespace henry {

namespace {
thread_local std::string g_last_error;

inline int grid1(int64_t n) { return (int)((n + kBlock - 1) / kBlock); }

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

// Check a CUDA call; on failure record the message and return HENRY_E_CUDA.
#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      set_last_error(std::string(#call) + ": " + cudaGetErrorString(e_));          \
      return e_ == cudaErrorMemoryAllocation ? HENRY_E_NOMEM : HENRY_E_CUDA;      \
    }                                                                              \
  } while (0)

__global__ void k_activate(unsigned long long* ctr, int B, const int* __restrict__ status,
                           int* __restrict__ active, int* __restrict__ it_step) {
  HENRY_COUNT_LAUNCH(ctr);
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < B) {
    active[b] = (status[b] & (kStatusNonfinite | kStatusBadInput | kStatusStall)) ? 0 : 1;
    it_step[b] = 0;
  }
}

__global__ void k_set_int(unsigned long long* ctr, int* __restrict__ dst, int v) {
  HENRY_COUNT_LAUNCH(ctr);
  if (threadIdx.x == 0) *dst = v;
}

__global__ void k_copy_int(unsigned long long* ctr, int n, const int* __restrict__ src,
                           int* __restrict__ dst, int do_or) {
  HENRY_COUNT_LAUNCH(ctr);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = do_or ? (dst[i] | src[i]) : src[i];
}
}  // namespace

void set_last_error(const std::string& msg) { g_last_error = msg; }
const char* last_error_cstr() { return g_last_error.c_str(); }

bool build_hierarchy(int nx, int ny, double Lx, double Ly, std::vector<Geom>& out) {
  std::vector<Geom> fine_to_coarse;
  int x = nx, y = ny;
  fine_to_coarse.push_back(Geom{x, y, Lx / x, Ly / y});
  while (x % 4 == 0 && y % 2 == 0 && (x / 2) * (y / 2) >= 8) {
    x /= 2;
    y /= 2;
    fine_to_coarse.push_back(Geom{x, y, Lx / x, Ly / y});
  }
  if (x % 2 != 0 || x * y > 32) return false;
  out.assign(fine_to_coarse.rbegin(), fine_to_coarse.rend());
  return true;
}

Solver::Solver(const henry_config& cfg, int nx, int ny, int nt) : cfg_(cfg), nt_(nt) {
  phys_ = Phys{cfg.rho0, cfg.rho1 - cfg.rho0, cfg.mu, cfg.g, cfg.D, cfg.K0, cfg.phi0, cfg.q0,
               cfg.Lx, cfg.Ly};
  tau_ = cfg.T / nt;
  tsize_ = cfg.precision == HENRY_PREC_FP32_MG ? sizeof(float) : sizeof(double);
  build_hierarchy(nx, ny, cfg.Lx, cfg.Ly, geoms_);
  levels_.resize(geoms_.size());
  for (size_t k = 0; k < geoms_.size(); ++k) levels_[k].g = geoms_[k];
  tile_ = make_res_tile(geoms_.back().nx, geoms_.back().ny, cfg.res_rows);
  nchunk_ = tile_.ntx * tile_.nty;
  ks_ = 0;
  kc_ = 0;
  for (size_t k = 0; k < geoms_.size(); ++k) {
    if (geoms_[k].ncell() <= cfg_.mg_small_cells) ks_ = (int)k;
    if (geoms_[k].ncell() <= cfg_.mg_cluster_cells) kc_ = (int)k;
  }
  const int per = geoms_[kc_].ncell() / 1024;
  cl_ = per < 1 ? 1 : (per > kMaxCluster ? kMaxCluster : per);
  if (!cfg_.mg_fusion) ks_ = kc_ = 0;
  // temporally blocked legs: batched levels (above the fused kernels) of at
  // most mg_tb_cells cells, tiles of at most 64 x 32 cells
  tb_.assign(geoms_.size(), 0);
  tbd_.resize(geoms_.size());
  tbu_.resize(geoms_.size());
  for (size_t k = 1; k < geoms_.size(); ++k) {
    const bool fused = (int)k <= ks_ || ((int)k <= kc_ && kc_ > ks_);
    if (fused || cfg_.nu1 < 1 || cfg_.nu2 < 1 || geoms_[k].ncell() > cfg_.mg_tb_cells) continue;
    tb_[k] = 1;
    tbd_[k] = make_tb_tile(geoms_[k], cfg_.nu1, 1, kTbTileX, kTbTileY, 20, tsize_);
    tbu_[k] = make_tb_tile(geoms_[k], cfg_.nu2, 0, kTbTileX, kTbTileY, 16, tsize_);
  }
}

Solver::~Solver() { free_all(); }

void Solver::free_all() {
  if (step_exec_) cudaGraphExecDestroy(step_exec_);
  if (step_graph_) cudaGraphDestroy(step_graph_);
  step_exec_ = nullptr;
  step_graph_ = nullptr;
  graph_B_ = -1;
  if (arena_) cudaFree(arena_);
  if (adj_arena_) cudaFree(adj_arena_);
  adj_arena_ = nullptr;
  adj_B_ = adj_nckpt_ = adj_seg_ = 0;
  if (n_active_host_) cudaFreeHost(n_active_host_);
  arena_ = nullptr;
  n_active_host_ = nullptr;
  cap_ = 0;
}

unsigned long long Solver::launches() const {
  unsigned long long v = 0;
  if (counter_) cudaMemcpy(&v, counter_, sizeof(v), cudaMemcpyDeviceToHost);
  return v;
}

int Solver::debug_copy(int mg_level, int what, void* dst, int64_t bytes) const {
  if (mg_level < 0 || mg_level >= (int)levels_.size() || what < 0 || what > 13 || !dst || bytes < 0)
    return HENRY_E_INVALID;
  if (cap_ == 0) return HENRY_E_INVALID;
  if (what == 13) {   // per-sample BiCGStab scalars [cap][8] (krylov_iters > 0)
    if (!cfg_.krylov_iters) return HENRY_E_INVALID;
    const size_t nb = (size_t)bytes < (size_t)cap_ * kKryS * 8 ? (size_t)bytes : (size_t)cap_ * kKryS * 8;
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(dst, kry_S_, nb, cudaMemcpyDefault));
    return HENRY_OK;
  }
  const MGLevel& L = levels_[mg_level];
  const size_t n = (size_t)L.g.ncell() * cap_;
  const void* src[13] = {L.J, L.b, L.x, L.p, L.c, L.phi, L.K, L.tx, L.dx, L.ty, L.dy, L.qx, L.qy};
  const size_t size[13] = {kJP * n * tsize_, 2 * n * tsize_, 2 * n * tsize_, n * 8, n * 8,
                           n * 8, n * 8, n * 8, n * 8, n * 8, n * 8, n * 8, n * 8};
  const size_t nb = (size_t)bytes < size[what] ? (size_t)bytes : size[what];
  CK(cudaDeviceSynchronize());
  CK(cudaMemcpy(dst, src[what], nb, cudaMemcpyDefault));
  return HENRY_OK;
}

// The dynamic shared-memory limit of a kernel is an attribute of the
// function in the device's context, shared by every solver of the process:
// it is only ever raised, to the largest size any solver needs, and outside
// stream capture (from ensure()), so that no solver's graph capture can meet
// a limit lowered by another solver.
static cudaError_t raise_smem_limit(const void* fn, size_t smem) {
  static std::mutex mu;
  static std::map<const void*, size_t> cur;
  std::lock_guard<std::mutex> lock(mu);
  size_t& c = cur[fn];
  if (smem <= c || smem <= 48 * 1024) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) c = smem;
  return e;
}

int Solver::ensure(int B, cudaStream_t s) {
  if (ks_ > 0) {
    SmallMG<float> Mf;
    SmallMG<double> Md;
    Mf.ks = Md.ks = ks_;
    for (int k = 0; k <= ks_; ++k) Mf.g[k] = Md.g[k] = geoms_[k];
    if (tsize_ == sizeof(float))
      CK(raise_smem_limit((const void*)k_vcycle_small<float>, small_smem_bytes(Mf)));
    else
      CK(raise_smem_limit((const void*)k_vcycle_small<double>, small_smem_bytes(Md)));
  }
  for (size_t k = 1; k < levels_.size(); ++k) {
    if (!tb_[k]) continue;
    const bool f32 = tsize_ == sizeof(float);
    const TbTile& d = tbd_[k];
    const TbTile& u = tbu_[k];
    const void* fd =
        d.cl ? (f32 ? (const void*)k_tbc_down<float> : (const void*)k_tbc_down<double>)
        : f32 ? (d.staged ? (const void*)k_tb_down<float, true> : (const void*)k_tb_down<float, false>)
              : (d.staged ? (const void*)k_tb_down<double, true> : (const void*)k_tb_down<double, false>);
    const void* fu =
        u.cl ? (f32 ? (const void*)k_tbc_up<float> : (const void*)k_tbc_up<double>)
        : f32 ? (u.staged ? (const void*)k_tb_up<float, true> : (const void*)k_tb_up<float, false>)
              : (u.staged ? (const void*)k_tb_up<double, true> : (const void*)k_tb_up<double, false>);
    CK(raise_smem_limit(fd, d.smem));
    CK(raise_smem_limit(fu, u.smem));
    // a cluster shape that cannot be resident on this GPU: one launch per
    // operation on this level instead
    for (const TbTile* t : {&d, &u}) {
      if (!t->cl) continue;
      cudaLaunchConfig_t lc = {};
      lc.gridDim = dim3((unsigned)t->cl);
      lc.blockDim = dim3(kTbBlock);
      lc.dynamicSmemBytes = t->smem;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = t->cl;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      lc.attrs = at;
      lc.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, t == &d ? fd : fu, &lc) != cudaSuccess ||
          nclusters < 1) {
        cudaGetLastError();
        tb_[k] = 0;
      }
    }
  }
  if (B <= cap_) return HENRY_OK;
  unsigned long long count = 0;
  if (counter_) CK(cudaMemcpy(&count, counter_, sizeof(count), cudaMemcpyDeviceToHost));
  CK(cudaDeviceSynchronize());
  free_all();
  const size_t Bz = (size_t)B;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  struct Off { size_t J, b, x, x2, p, c, phi, K, tx, dx, ty, dy, qx, qy; };
  std::vector<Off> lo(levels_.size());
  for (size_t k = 0; k < levels_.size(); ++k) {
    const size_t n = (size_t)levels_[k].g.ncell() * Bz;
    lo[k].J = take(kJP * n * tsize_);
    lo[k].b = take(2 * n * tsize_);
    lo[k].x = take(2 * n * tsize_);
    lo[k].x2 = take(tb_[k] ? 2 * n * tsize_ : 0);
    lo[k].p = take(n * 8);
    lo[k].c = take(n * 8);
    lo[k].phi = take(n * 8);
    lo[k].K = take(n * 8);
    lo[k].tx = take(n * 8);
    lo[k].dx = take(n * 8);
    lo[k].ty = take(n * 8);
    lo[k].dy = take(n * 8);
    lo[k].qx = take(n * 8);
    lo[k].qy = take(n * 8);
  }
  const Geom& F = levels_.back().g;
  const size_t o_cold = take((size_t)F.ncell() * Bz * 8);
  const size_t o_pprev = take((size_t)F.ncell() * Bz * 8);
  size_t o_hist[2 * kMaxGuessHist];
  for (int k = 0; k < 2 * kMaxGuessHist; ++k)
    o_hist[k] = take(k / 2 < guess_depth() ? (size_t)F.ncell() * Bz * 8 : 0);
  const size_t o_mo = take((size_t)F.ncell() * Bz * 8);
  const size_t o_so = take((size_t)F.ncell() * Bz * 8);
  const size_t o_vt = take((size_t)F.ncell() * Bz * 8);
  const size_t o_step = take(8);
  const size_t o_qin = take((size_t)F.ny * Bz * 8);
  const size_t o_qin0 = take((size_t)F.ny * Bz * 8);
  const size_t o_part = take((size_t)nchunk_ * Bz * 8);
  const size_t o_res0 = take(Bz * 8);
  const size_t o_resl = take(Bz * 8);
  const size_t o_cinv = take(Bz * kMaxCoarseUnknowns * kMaxCoarseUnknowns * 8);
  const size_t o_act = take(Bz * 4);
  const size_t o_ref = take(Bz * 4);
  const size_t o_its = take(Bz * 4);
  const size_t o_st = take(Bz * 4);
  const size_t o_it = take(Bz * 4);
  const size_t o_na = take(8);     // active count, rebuild count
  const size_t o_keep = take(8);   // operators kept across steps in this solve (k_check)
  const size_t o_acc = take(16);   // k_check's accumulators
  // BiCGStab vectors r, rh, p, v, t, xk ([B][2][ncell] of the finest level),
  // per-sample scalars and dot partials (only with krylov_iters > 0)
  const size_t n2 = (size_t)2 * F.ncell();
  const size_t kvec = cfg_.krylov_iters ? n2 * Bz * tsize_ : 0;
  size_t o_kv[6];
  for (int k = 0; k < 6; ++k) o_kv[k] = take(kvec);
  kry_nchunk_ = (int)((n2 + kBlock * 4 - 1) / (kBlock * 4));
  const size_t o_ks = take(cfg_.krylov_iters ? Bz * kKryS * 8 : 0);
  const size_t o_kp = take(cfg_.krylov_iters ? 2 * Bz * kry_nchunk_ * 8 : 0);
  const size_t o_ctr = take(8);
  CK(cudaMalloc(&arena_, off));
  CK(cudaHostAlloc((void**)&n_active_host_, 2 * sizeof(int), cudaHostAllocDefault));
  char* a = (char*)arena_;
  for (size_t k = 0; k < levels_.size(); ++k) {
    MGLevel& L = levels_[k];
    L.J = a + lo[k].J;
    L.b = a + lo[k].b;
    L.x = a + lo[k].x;
    L.x2 = tb_[k] ? a + lo[k].x2 : nullptr;
    L.p = (double*)(a + lo[k].p);
    L.c = (double*)(a + lo[k].c);
    L.phi = (double*)(a + lo[k].phi);
    L.K = (double*)(a + lo[k].K);
    L.tx = (double*)(a + lo[k].tx);
    L.dx = (double*)(a + lo[k].dx);
    L.ty = (double*)(a + lo[k].ty);
    L.dy = (double*)(a + lo[k].dy);
    L.qx = (double*)(a + lo[k].qx);
    L.qy = (double*)(a + lo[k].qy);
  }
  c_old_ = (double*)(a + o_cold);
  p_prev_ = (double*)(a + o_pprev);
  hx_ = {};
  hx_.depth = guess_depth();
  for (int k = 0; k < hx_.depth; ++k) {
    hx_.p[k] = (double*)(a + o_hist[2 * k]);
    hx_.c[k] = (double*)(a + o_hist[2 * k + 1]);
  }
  mo_ = (double*)(a + o_mo);
  so_ = (double*)(a + o_so);
  vt_ = (double*)(a + o_vt);
  step_ = (int*)(a + o_step);
  qin_ = (double*)(a + o_qin);
  qin0_ = (double*)(a + o_qin0);
  partial_ = (double*)(a + o_part);
  res0_ = (double*)(a + o_res0);
  res_last_ = (double*)(a + o_resl);
  cinv_ = a + o_cinv;
  active_ = (int*)(a + o_act);
  refresh_ = (int*)(a + o_ref);
  it_step_ = (int*)(a + o_its);
  status_w_ = (int*)(a + o_st);
  iters_w_ = (int*)(a + o_it);
  n_active_ = (int*)(a + o_na);
  keep_ = (int*)(a + o_keep);
  check_acc_ = (unsigned int*)(a + o_acc);
  for (int k = 0; k < 6; ++k) kry_v_[k] = a + o_kv[k];
  kry_S_ = (double*)(a + o_ks);
  kry_part_ = (double*)(a + o_kp);
  counter_ = (unsigned long long*)(a + o_ctr);
  CK(cudaMemset(arena_, 0, off));
  CK(cudaMemcpy(counter_, &count, sizeof(count), cudaMemcpyHostToDevice));
  cap_ = B;
  ++generation_;
  (void)s;
  return HENRY_OK;
}

template <typename T>
void Solver::launch_small(int B, int ncycles, cudaStream_t s) {
  SmallMG<T> M;
  M.ks = ks_;
  for (int k = 0; k <= ks_; ++k) {
    M.g[k] = levels_[k].g;
    M.J[k] = (T*)levels_[k].J;
    M.b[k] = (T*)levels_[k].b;
    M.x[k] = (T*)levels_[k].x;
  }
  const size_t smem = small_smem_bytes(M);
  k_vcycle_small<T><<<B, kBlock, smem, s>>>(counter_, M, B, active_, (const T*)cinv_, cfg_.nu1, cfg_.nu2,
                                            ncycles, status_w_);
}

template <typename T>
void Solver::launch_cluster(int B, int ncycles, cudaStream_t s) {
  SmallMG<T> M;
  M.ks = kc_;
  for (int k = 0; k <= kc_; ++k) {
    M.g[k] = levels_[k].g;
    M.J[k] = (T*)levels_[k].J;
    M.b[k] = (T*)levels_[k].b;
    M.x[k] = (T*)levels_[k].x;
  }
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)(B * cl_));
  lc.blockDim = dim3(kBlock);
  lc.dynamicSmemBytes = 0;
  lc.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl_;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  cudaLaunchKernelEx(&lc, k_vcycle_cluster<T>, counter_, M, B, (const int*)active_,
                     (const T*)cinv_, cfg_.nu1, cfg_.nu2, ncycles, cl_);
}

// Whole hierarchy fits the shared-memory kernel, or the cluster kernel, or
// neither (then the top levels are launched one kernel at a time).
template <typename T>
void Solver::enqueue_vcycle(int k, int B, cudaStream_t s) {
  MGLevel& L = levels_[k];
  const Geom& G = L.g;
  if (k == kc_ && kc_ > ks_ && k > 0) {
    launch_cluster<T>(B, 1, s);
    return;
  }
  if (k == ks_ && k > 0) {
    launch_small<T>(B, 1, s);
    return;
  }
  if (k == 0) {
    k_coarse_solve<T><<<(B + 7) / 8, kBlock, 0, s>>>(counter_, G, B, active_, (const T*)cinv_,
                                                     (const T*)L.b, (T*)L.x);
    return;
  }
  MGLevel& C = levels_[k - 1];
  if (tb_[k]) {
    // two launches: pre-sweeps + restriction (x -> x2), then the coarse
    // levels, then prolongation + post-sweeps (x2 -> x)
    const TbTile& td = tbd_[k];
    const TbTile& tu = tbu_[k];
    auto cluster_cfg = [&](const TbTile& t, cudaLaunchConfig_t& lc, cudaLaunchAttribute* at) {
      lc = {};
      lc.gridDim = dim3((unsigned)(B * t.cl));
      lc.blockDim = dim3(kTbBlock);
      lc.dynamicSmemBytes = t.smem;
      lc.stream = s;
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = t.cl;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      lc.attrs = at;
      lc.numAttrs = 1;
    };
    cudaLaunchConfig_t lc;
    cudaLaunchAttribute at[1];
    if (td.cl) {
      cluster_cfg(td, lc, at);
      cudaLaunchKernelEx(&lc, k_tbc_down<T>, counter_, G, C.g, B, (const int*)active_, cfg_.nu1,
                         td.cl, (const T*)L.J, (const T*)L.b, (const T*)L.x, (T*)L.x2,
                         (const T*)C.J, (T*)C.b, (T*)C.x, status_w_);
    } else {
      auto down = td.staged ? k_tb_down<T, true> : k_tb_down<T, false>;
      down<<<dim3(td.ntx * td.nty, B), kTbBlock, td.smem, s>>>(
          counter_, G, C.g, B, active_, td, cfg_.nu1, (const T*)L.J, (const T*)L.b,
          (const T*)L.x, (T*)L.x2, (const T*)C.J, (T*)C.b, (T*)C.x, status_w_);
    }
    enqueue_vcycle<T>(k - 1, B, s);
    if (tu.cl) {
      cluster_cfg(tu, lc, at);
      cudaLaunchKernelEx(&lc, k_tbc_up<T>, counter_, C.g, G, B, (const int*)active_, cfg_.nu2,
                         tu.cl, (const T*)C.x, (const T*)L.J, (const T*)L.b, (const T*)L.x2,
                         (T*)L.x, status_w_);
    } else {
      auto up = tu.staged ? k_tb_up<T, true> : k_tb_up<T, false>;
      up<<<dim3(tu.ntx * tu.nty, B), kTbBlock, tu.smem, s>>>(
          counter_, C.g, G, B, active_, tu, cfg_.nu2, (const T*)C.x, (const T*)L.J, (const T*)L.b,
          (const T*)L.x2, (T*)L.x, status_w_);
    }
    return;
  }
  const int gs = grid1((int64_t)B * G.half());
  for (int sw = 0; sw < cfg_.nu1; ++sw)
    for (int col = 0; col < 2; ++col)
      k_smooth<T><<<gs, kBlock, 0, s>>>(counter_, G, B, col, active_, (const T*)L.J,
                                       (const T*)L.b, (T*)L.x);
  k_resid_restrict<T><<<grid1((int64_t)B * C.g.ncell()), kBlock, 0, s>>>(
      counter_, G, C.g, B, active_, (const T*)L.J, (const T*)L.b, (const T*)L.x,
      (const T*)C.J, (T*)C.b, (T*)C.x, cfg_.nu1 > 0);
  enqueue_vcycle<T>(k - 1, B, s);
  const int black_only = cfg_.nu2 > 0;
  k_prolong<T><<<grid1((int64_t)B * (black_only ? G.half() : G.ncell())), kBlock, 0, s>>>(
      counter_, C.g, G, B, active_, (const T*)C.x, (T*)L.x, black_only);
  for (int sw = 0; sw < cfg_.nu2; ++sw)
    for (int col = 0; col < 2; ++col)
      k_smooth<T><<<gs, kBlock, 0, s>>>(counter_, G, B, col, active_, (const T*)L.J,
                                       (const T*)L.b, (T*)L.x);
}

// Coarse multigrid operators at the current iterate (linearised about the
// restricted face fluxes).
template <typename T>
void Solver::enqueue_coarse_ops(int B, cudaStream_t s, const int* refresh) {
  const int nl = (int)levels_.size();
  for (int k = nl - 1; k >= 1; --k) {
    MGLevel& F = levels_[k];
    MGLevel& C = levels_[k - 1];
    k_restrict_state<<<grid1((int64_t)B * C.g.ncell()), kBlock, 0, s>>>(
        counter_, F.g, C.g, B, active_, F.c, F.qx, F.qy, C.c, C.qx, C.qy, refresh);
    k_jac<T><<<grid1((int64_t)B * C.g.ncell()), kBlock, 0, s>>>(
        counter_, phys_, C.g, C.g.hx * C.g.hy / tau_, B, active_, C.p, C.c, C.phi, C.K, C.tx, C.dx, C.ty, C.dy,
        C.qx, C.qy, (T*)C.J, refresh);
  }
}

template <typename T>
void Solver::enqueue_coarse_inv(int B, cudaStream_t s, const int* refresh) {
  {
    const int n = 2 * levels_[0].g.ncell();
    k_coarse_inv<T><<<B, kBlock, coarse_inv_smem_bytes<T>(n), s>>>(
        counter_, levels_[0].g, B, active_, (const T*)levels_[0].J, (T*)cinv_, refresh);
  }
}

template <typename T>
void Solver::enqueue_vcycles(int B, cudaStream_t s) {
  const int nl = (int)levels_.size();
  if (ks_ == nl - 1 && nl > 1)
    launch_small<T>(B, cfg_.vcycles, s);
  else if (kc_ == nl - 1 && nl > 1)
    launch_cluster<T>(B, cfg_.vcycles, s);
  else
    for (int v = 0; v < cfg_.vcycles; ++v) enqueue_vcycle<T>(nl - 1, B, s);
}

// One V-cycle on the finest level's b and x (the BiCGStab preconditioner).
template <typename T>
void Solver::enqueue_precond(int B, cudaStream_t s) {
  const int nl = (int)levels_.size();
  if (ks_ == nl - 1 && nl > 1)
    launch_small<T>(B, 1, s);
  else if (kc_ == nl - 1 && nl > 1)
    launch_cluster<T>(B, 1, s);
  else
    enqueue_vcycle<T>(nl - 1, B, s);
}

// krylov_iters iterations of BiCGStab on At x = bt (finest level), each
// with two preconditioner applications; leaves the correction in x.
template <typename T>
void Solver::enqueue_bicgstab(int B, cudaStream_t s) {
  MGLevel& F = levels_.back();
  const Geom& G = F.g;
  const int n2 = 2 * G.ncell();
  const int gv = grid1((int64_t)B * n2);
  T* r = (T*)kry_v_[0];
  T* rh = (T*)kry_v_[1];
  T* p = (T*)kry_v_[2];
  T* v = (T*)kry_v_[3];
  T* t = (T*)kry_v_[4];
  T* xk = (T*)kry_v_[5];
  T* b = (T*)F.b;
  T* x = (T*)F.x;
  const dim3 gd(kry_nchunk_, B);
  const int gs = (B + kBlock - 1) / kBlock;
  auto upd = [&](int op) {
    k_kry_update<T><<<gv, kBlock, 0, s>>>(counter_, n2, B, op, active_, kry_S_, r, rh, p, v, t,
                                          xk, b, x);
  };
  upd(0);
  for (int it = 0; it < cfg_.krylov_iters; ++it) {
    k_kry_dot<T><<<gd, kBlock, 0, s>>>(counter_, n2, B, active_, rh, r, (const T*)nullptr,
                                       (const T*)nullptr, kry_part_);
    k_kry_scalars<<<gs, kBlock, 0, s>>>(counter_, B, kry_nchunk_, 0, active_, kry_part_, kry_S_);
    upd(1);                                            // p; b = p, x = 0
    enqueue_precond<T>(B, s);                          // y = M p in x
    k_kry_matvec<T><<<grid1((int64_t)B * G.ncell()), kBlock, 0, s>>>(
        counter_, G, B, active_, (const T*)F.J, (const T*)x, v);
    k_kry_dot<T><<<gd, kBlock, 0, s>>>(counter_, n2, B, active_, rh, v, (const T*)nullptr,
                                       (const T*)nullptr, kry_part_);
    k_kry_scalars<<<gs, kBlock, 0, s>>>(counter_, B, kry_nchunk_, 1, active_, kry_part_, kry_S_);
    upd(2);                                            // xk += alpha y; s = r - alpha v
    enqueue_precond<T>(B, s);                          // z = M s in x
    k_kry_matvec<T><<<grid1((int64_t)B * G.ncell()), kBlock, 0, s>>>(
        counter_, G, B, active_, (const T*)F.J, (const T*)x, t);
    k_kry_dot<T><<<gd, kBlock, 0, s>>>(counter_, n2, B, active_, t, r, t, t, kry_part_);
    k_kry_scalars<<<gs, kBlock, 0, s>>>(counter_, B, kry_nchunk_, 2, active_, kry_part_, kry_S_);
    upd(3);                                            // xk += omega z; r -= omega t
  }
  upd(4);                                              // x = xk
}

// Multigrid operators at the current iterate, for the samples that asked
// for them (all samples without operator reuse).
template <typename T>
void Solver::enqueue_rebuild(int B, cudaStream_t s) {
  const int* refresh = cfg_.jac_lag ? refresh_ : nullptr;
  if (refresh) {
    MGLevel& F = levels_.back();
    k_resjac<T, false><<<dim3(nchunk_, B), kBlock, 0, s>>>(
        counter_, phys_, F.g, F.g.hx * F.g.hy / tau_, B, tile_, F.p, F.c, c_old_, F.phi, F.K, F.tx,
        F.dx, F.ty, F.dy, qin_, active_, (T*)F.J, (T*)F.b, (T*)F.x, partial_, F.qx, F.qy, refresh);
  }
  enqueue_coarse_ops<T>(B, s, refresh);
  enqueue_coarse_inv<T>(B, s, refresh);
}

// Linear solve of the defect correction (V-cycles or BiCGStab) and the
// state update.
template <typename T>
void Solver::enqueue_solve_update(int B, cudaStream_t s) {
  if (cfg_.krylov_iters)
    enqueue_bicgstab<T>(B, s);
  else
    enqueue_vcycles<T>(B, s);
  MGLevel& F = levels_.back();
  k_update<T><<<grid1((int64_t)B * F.g.ncell()), kBlock, 0, s>>>(counter_, F.g, B, active_,
                                                                 (const T*)F.x, F.p, F.c);
}

template <typename T>
void Solver::enqueue_iteration(int B, cudaStream_t s) {
  enqueue_rebuild<T>(B, s);
  enqueue_solve_update<T>(B, s);
}

template <typename T>
void Solver::enqueue_resjac_check(int B, cudaStream_t s, bool set_cond,
                                  unsigned long long cond) {
  MGLevel& F = levels_.back();
  const Geom& G = F.g;
  if (cfg_.jac_lag)   // residual only; the next iteration rebuilds operators where needed
    k_resid<T><<<dim3(nchunk_, B), kBlock, 0, s>>>(
        counter_, phys_, G, B, tile_, F.p, F.c, vt_, mo_, so_, F.phi, F.tx, F.dx, F.ty, F.dy,
        qin_, active_, (const T*)F.J, (T*)F.b, (T*)F.x, partial_, F.qx, F.qy);
  else
    k_resjac<T, false><<<dim3(nchunk_, B), kBlock, 0, s>>>(
        counter_, phys_, G, G.hx * G.hy / tau_, B, tile_, F.p, F.c, c_old_, F.phi, F.K, F.tx, F.dx,
        F.ty, F.dy, qin_, active_, (T*)F.J, (T*)F.b, (T*)F.x, partial_, F.qx, F.qy, nullptr);
  int* refresh = cfg_.jac_lag ? refresh_ : nullptr;
  // residual scaled to units of c per step: RMS(R) * tau / (V phi0 rho0)
  const double scale = tau_ / (G.hx * G.hy * cfg_.phi0 * cfg_.rho0);
  const int gb = (B + 7) / 8;
  const double stag_tol = cfg_.newton_stag_tol;
  if (set_cond)
    k_check<true><<<gb, kBlock, 0, s>>>(counter_, B, nchunk_, G.ncell(), partial_, scale,
                                        cfg_.newton_rtol, cfg_.newton_atol, cfg_.newton_maxit,
                                        active_, it_step_, res0_, res_last_, status_w_, iters_w_,
                                        n_active_, check_acc_, stag_tol,
                                        (cudaGraphConditionalHandle)cond, refresh,
                                        cfg_.jac_lag, 0.0, keep_);
  else
    k_check<false><<<gb, kBlock, 0, s>>>(counter_, B, nchunk_, G.ncell(), partial_, scale,
                                         cfg_.newton_rtol, cfg_.newton_atol, cfg_.newton_maxit,
                                         active_, it_step_, res0_, res_last_, status_w_, iters_w_,
                                         n_active_, check_acc_, stag_tol, 0, refresh,
                                         cfg_.jac_lag, 0.0, keep_);
}

// The nodes of one implicit Euler step on stream cs, which is capturing into
// graph g: begin step, FP64 residual + convergence check, a conditional
// while node whose body (one defect-correction iteration and the next
// check) is recorded in `bodies` and captured by capture_body() once the
// capture of g has ended, then the end of the step. Each step has its own
// conditional handle, set by its own checks.
template <typename T>
int Solver::capture_step_t(cudaGraph_t g, cudaStream_t cs, int B, std::vector<StepBody>& bodies) {
  cudaGraphConditionalHandle h;
  CK(cudaGraphConditionalHandleCreate(&h, g, 0, 0));
  MGLevel& F = levels_.back();
  launch_begin_step(B, cs);
  enqueue_resjac_check<T>(B, cs, true, (unsigned long long)h);
  cudaStreamCaptureStatus st;
  cudaGraph_t cg;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(cs, &st, nullptr, &cg, &deps, nullptr, &nd));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t wn;
  CK(cudaGraphAddNode(&wn, cg, deps, nullptr, nd, &cp));
  bodies.push_back(StepBody{this, cp.conditional.phGraph_out[0], (unsigned long long)h});
  CK(cudaStreamUpdateCaptureDependencies(cs, &wn, nullptr, 1, cudaStreamSetCaptureDependencies));
  k_end_step<<<1, 32, 0, cs>>>(counter_, step_);
  CK(cudaGetLastError());
  return HENRY_OK;
}

cudaError_t Solver::set_node_priority(cudaGraphNode_t node, int p) {
  cudaLaunchAttributeValue v = {};
  v.priority = p;
  return cudaGraphKernelNodeSetAttribute(node, cudaLaunchAttributePriority, &v);
}

// Give every kernel node of g (not descending into conditional nodes, whose
// bodies are captured and prioritised on their own) the priority p.
static cudaError_t prioritise_kernels(cudaGraph_t g, int p) {
  size_t n = 0;
  cudaError_t e = cudaGraphGetNodes(g, nullptr, &n);
  if (e != cudaSuccess || n == 0) return e;
  std::vector<cudaGraphNode_t> nodes(n);
  e = cudaGraphGetNodes(g, nodes.data(), &n);
  for (size_t k = 0; k < n && e == cudaSuccess; ++k) {
    cudaGraphNodeType t;
    e = cudaGraphNodeGetType(nodes[k], &t);
    if (e == cudaSuccess && t == cudaGraphNodeTypeKernel) e = Solver::set_node_priority(nodes[k], p);
  }
  return e;
}

// The body of a step's while node: one defect-correction iteration and the
// next check. With operator reuse the rebuild kernels sit in a conditional
// IF node (captured after the body) set by k_set_rebuild, so iterations in
// which no sample rebuilds its operators launch none of them.
template <typename T>
int Solver::capture_body_t(const StepBody& sb, int B, cudaStream_t bs) {
  cudaGraph_t body = sb.body;
  CK(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaGraph_t rebuild = nullptr;
  if (cfg_.jac_lag) {
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, body, 0, 0);
    if (e == cudaSuccess) {
      k_set_rebuild<<<1, 32, 0, bs>>>(counter_, n_active_ + 1, h);
      cudaStreamCaptureStatus st;
      cudaGraph_t cg;
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      e = cudaStreamGetCaptureInfo(bs, &st, nullptr, &cg, &deps, nullptr, &nd);
      cudaGraphNodeParams cp = {};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeIf;
      cp.conditional.size = 1;
      cudaGraphNode_t in;
      if (e == cudaSuccess) e = cudaGraphAddNode(&in, cg, deps, nullptr, nd, &cp);
      if (e == cudaSuccess) {
        rebuild = cp.conditional.phGraph_out[0];
        e = cudaStreamUpdateCaptureDependencies(bs, &in, nullptr, 1, cudaStreamSetCaptureDependencies);
      }
    }
    if (e != cudaSuccess) {
      cudaStreamEndCapture(bs, &body);
      set_last_error(std::string("rebuild condition: ") + cudaGetErrorString(e));
      return HENRY_E_CUDA;
    }
  } else {
    enqueue_rebuild<T>(B, bs);
  }
  enqueue_solve_update<T>(B, bs);
  enqueue_resjac_check<T>(B, bs, true, sb.cond);
  CK(cudaStreamEndCapture(bs, &body));
  if (prio_) CK(prioritise_kernels(body, prio_));
  if (rebuild) {
    CK(cudaStreamBeginCaptureToGraph(bs, rebuild, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    enqueue_rebuild<T>(B, bs);
    CK(cudaStreamEndCapture(bs, &rebuild));
    if (prio_) CK(prioritise_kernels(rebuild, prio_));
  }
  return HENRY_OK;
}

int Solver::capture_steps(cudaGraph_t g, cudaStream_t cs, int B, int nsteps,
                          std::vector<StepBody>& bodies) {
  for (int k = 0; k < nsteps; ++k) {
    const int rc = tsize_ == sizeof(float) ? capture_step_t<float>(g, cs, B, bodies)
                                           : capture_step_t<double>(g, cs, B, bodies);
    if (rc) return rc;
  }
  return HENRY_OK;
}

int Solver::capture_body(const StepBody& sb, int B, cudaStream_t bs) {
  return tsize_ == sizeof(float) ? capture_body_t<float>(sb, B, bs)
                                 : capture_body_t<double>(sb, B, bs);
}

// One implicit Euler step as a CUDA graph (capture_step + its body),
// rebuilt when B changes: one graph launch per step, no host
// synchronisation.
template <typename T>
int Solver::step_graph(int B, cudaStream_t s) {
  if (graph_B_ != B) {
    if (step_exec_) cudaGraphExecDestroy(step_exec_);
    if (step_graph_) cudaGraphDestroy(step_graph_);
    step_exec_ = nullptr;
    step_graph_ = nullptr;
    cudaStream_t cs, bs;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
    cudaGraph_t g;
    CK(cudaGraphCreate(&g, 0));
    std::vector<StepBody> bodies;
    CK(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    int rc = capture_step_t<T>(g, cs, B, bodies);
    cudaGraph_t gout = g;
    const cudaError_t ee = cudaStreamEndCapture(cs, &gout);
    if (rc) return rc;
    CK(ee);
    for (const StepBody& sb : bodies)
      if ((rc = capture_body_t<T>(sb, B, bs))) return rc;
    CK(cudaGraphInstantiate(&step_exec_, g, 0));
    step_graph_ = g;
    graph_B_ = B;
    cudaStreamDestroy(cs);
    cudaStreamDestroy(bs);
  }
  CK(cudaGraphLaunch(step_exec_, s));
  return HENRY_OK;
}

int Solver::fields(const double* xi, const double* logk, int B, double* phi, double* K,
                   double* qin, cudaStream_t s) {
  if (B == 0) return HENRY_OK;
  int rc = ensure(B, s);
  if (rc) return rc;
  const Geom& G = levels_.back().g;
  k_fields<<<grid1((int64_t)B * G.ncell()), kBlock, 0, s>>>(
      counter_, phys_, G, B, cfg_.n_xi, cfg_.field_model, xi, logk, phi, K, qin, status_w_);
  CK(cudaGetLastError());
  return HENRY_OK;
}

template <typename T>
int Solver::setup_t(const double* xi, const double* logk, int B, cudaStream_t s) {
  const int nl = (int)levels_.size();
  MGLevel& F = levels_.back();
  const Geom& G = F.g;
  // the paper's field model has a time-dependent inflow: its base goes to
  // qin0_ and k_begin_step forms each step's inflow in qin_
  k_fields<<<grid1((int64_t)B * G.ncell()), kBlock, 0, s>>>(
      counter_, phys_, G, B, cfg_.n_xi, cfg_.field_model, xi, logk, F.phi, F.K,
      cfg_.field_model == 1 ? qin0_ : qin_, status_w_);
  for (int k = nl - 1; k >= 1; --k)
    k_coarsen_fields<<<grid1((int64_t)B * levels_[k - 1].g.ncell()), kBlock, 0, s>>>(
        counter_, levels_[k].g, levels_[k - 1].g, B, levels_[k].phi, levels_[k].K,
        levels_[k - 1].phi, levels_[k - 1].K);
  for (int k = 0; k < nl; ++k) {
    MGLevel& L = levels_[k];
    k_face_consts<<<grid1((int64_t)B * L.g.ncell()), kBlock, 0, s>>>(
        counter_, phys_, L.g, B, L.phi, L.K, L.tx, L.dx, L.ty, L.dy);
  }
  k_init_state<<<grid1((int64_t)B * G.ncell()), kBlock, 0, s>>>(counter_, phys_, G, B, F.p, F.c,
                                                                iters_w_, step_);
  k_set_int<<<1, 32, 0, s>>>(counter_, keep_, cfg_.jac_keep);
  CK(cudaGetLastError());
  return HENRY_OK;
}

// Begin every sample's step (k_begin_step, instantiated for the depth of
// the Newton guess's history).
void Solver::launch_begin_step(int B, cudaStream_t s) {
  MGLevel& F = levels_.back();
  const Geom& G = F.g;
  auto go = [&](auto kern) {
    kern<<<grid1((int64_t)B * G.ncell()), kBlock, 0, s>>>(
        counter_, G, B, F.p, F.c, p_prev_, c_old_, status_w_, active_, it_step_, step_,
        cfg_.guess_extrapolation, cfg_.field_model == 1 ? qin0_ : nullptr, qin_, tau_, F.phi,
        G.hx * G.hy / tau_, phys_.rho0, phys_.drho, mo_, so_, vt_, hx_);
  };
  switch (hx_.depth) {
    case 0: go(k_begin_step<0>); break;
    case 1: go(k_begin_step<1>); break;
    case 2: go(k_begin_step<2>); break;
    case 3: go(k_begin_step<3>); break;
    case 4: go(k_begin_step<4>); break;
    default: go(k_begin_step<5>); break;
  }
}

// One implicit Euler step of every sample (Newton defect correction).
template <typename T>
int Solver::step_t(int B, cudaStream_t s) {
  if (cfg_.loop_mode == HENRY_LOOP_GRAPH) return step_graph<T>(B, s);
  MGLevel& F = levels_.back();
  const Geom& G = F.g;
  launch_begin_step(B, s);
  for (;;) {
    enqueue_resjac_check<T>(B, s, false);
    CK(cudaMemcpyAsync(n_active_host_, n_active_, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (n_active_host_[0] == 0) break;
    // with operator reuse, the rebuild is skipped when no sample asked for it
    if (!cfg_.jac_lag || n_active_host_[1] > 0) enqueue_rebuild<T>(B, s);
    enqueue_solve_update<T>(B, s);
  }
  k_end_step<<<1, 32, 0, s>>>(counter_, step_);
  return HENRY_OK;
}

template <typename T>
int Solver::run_t(const double* xi, const double* logk, int B, double* q, double* c_out,
                  double* p_out, int* status, int* iters, int status_or, cudaStream_t s) {
  int rc = setup_t<T>(xi, logk, B, s);
  if (rc) return rc;
  const int nout = series_every_ > 0 ? nt_ / series_every_ : 0;
  for (int n = 0; n < nt_; ++n) {
    rc = step_t<T>(B, s);
    if (rc) return rc;
    if (series_ && (n + 1) % series_every_ == 0) {
      MGLevel& F = levels_.back();
      const int k = (n + 1) / series_every_ - 1;
      k_qoi<<<B, kBlock, 0, s>>>(counter_, phys_, F.g, B, F.p, F.c, F.phi, series_ + k * kNQ,
                                 nullptr, nullptr, nout * kNQ);
    }
  }
  return finish(B, q, c_out, p_out, status, iters, status_or, s);
}

int Solver::begin(const double* xi, const double* logk, int B, cudaStream_t s) {
  if (B == 0) return HENRY_OK;
  int rc = ensure(B, s);
  if (rc) return rc;
  last_B_ = B;
  return tsize_ == sizeof(float) ? setup_t<float>(xi, logk, B, s) : setup_t<double>(xi, logk, B, s);
}

int Solver::finish(int B, double* q, double* c_out, double* p_out, int* status, int* iters,
                   int status_or, cudaStream_t s) {
  MGLevel& F = levels_.back();
  const Geom& G = F.g;
  k_qoi<<<B, kBlock, 0, s>>>(counter_, phys_, G, B, F.p, F.c, F.phi, q, c_out, p_out, kNQ);
  k_copy_int<<<grid1(B), kBlock, 0, s>>>(counter_, B, status_w_, status, status_or);
  if (iters) k_copy_int<<<grid1(B), kBlock, 0, s>>>(counter_, B, iters_w_, iters, 0);
  CK(cudaGetLastError());
  return HENRY_OK;
}

template <typename T>
void Solver::launch_timed(int which, int B, cudaStream_t s) {
  MGLevel& F = levels_.back();
  if (which == 0) {
    k_smooth<T><<<grid1((int64_t)B * F.g.half()), kBlock, 0, s>>>(
        counter_, F.g, B, 0, active_, (const T*)F.J, (const T*)F.b, (T*)F.x);
  } else if (which == 2) {
    k_resid<T><<<dim3(nchunk_, B), kBlock, 0, s>>>(
        counter_, phys_, F.g, B, tile_, F.p, F.c, vt_, mo_, so_, F.phi, F.tx, F.dx, F.ty, F.dy,
        qin_, active_, (const T*)F.J, (T*)F.b, (T*)F.x, partial_, F.qx, F.qy);
  } else {
    k_resjac<T, false><<<dim3(nchunk_, B), kBlock, 0, s>>>(
        counter_, phys_, F.g, F.g.hx * F.g.hy / tau_, B, tile_, F.p, F.c, c_old_, F.phi, F.K, F.tx, F.dx, F.ty, F.dy,
        qin_, active_, (T*)F.J, (T*)F.b, (T*)F.x, partial_, F.qx, F.qy, nullptr);
  }
}

// Algorithmic counts per launch, the per-cell figures of the method's byte
// model (every array read or written once per launch, neighbour values
// reused on chip):
//  smoother half-sweep, per updated cell: operator A (20 values), b (2),
//    x read (2, the other colour) and written (2) = 26 values of type T
//    (104 B FP32, 208 B FP64). The row-scaled storage reads 16 operator
//    values instead of 20, so the kernel moves 22 values: the figure above
//    credits it with the unscaled operator's bytes. FP ops: 16 FMA per
//    update (32 FLOP).
//  residual only (which = 2): 56 B per cell, 46 FP64 operations.
//  residual + Jacobian, per cell: p, c, c_old, phi, K read (40 B), R written
//    (16 B), J written (20 values of type T): 136 B (FP32 J) or 216 B. FP
//    ops counted from the face-based code: 2 faces x 15 (flux) + 16
//    (accumulation, sums, norm) = 46 FP64 operations, plus the Jacobian,
//    2 faces x 30 + 24 = 84 operations in the multigrid type; the figure
//    reported is the FP64 count: 46 + (116 if T = double).
// flush (optional): before every timed launch `flush_bytes` bytes of
// `flush` are overwritten (cudaMemsetAsync), so that each launch starts
// with cold caches when flush_bytes exceeds the L2; every launch is then
// timed by its own event pair and the flush is not counted.
int Solver::time_kernel(int which, int reps, cudaStream_t s, void* flush, int64_t flush_bytes,
                        double* avg_ms, double* bytes, double* flops) {
  if (which < 0 || which > 2 || reps < 1 || reps > 100000 || last_B_ < 1 || flush_bytes < 0 ||
      (flush_bytes > 0 && !flush))
    return HENRY_E_INVALID;
  const int B = last_B_;
  // all samples active for the replay
  std::vector<int> ones(B, 1);
  CK(cudaMemcpyAsync(active_, ones.data(), sizeof(int) * B, cudaMemcpyHostToDevice, s));
  auto launch = [&]() {
    if (tsize_ == sizeof(float)) launch_timed<float>(which, B, s);
    else launch_timed<double>(which, B, s);
  };
  launch();
  const int nev = flush_bytes > 0 ? reps : 1;
  std::vector<cudaEvent_t> e0(nev, nullptr), e1(nev, nullptr);
  int rc = HENRY_OK;
  for (int r = 0; r < nev && rc == HENRY_OK; ++r) {
    if (cudaEventCreate(&e0[r]) != cudaSuccess || cudaEventCreate(&e1[r]) != cudaSuccess)
      rc = HENRY_E_CUDA;
  }
  float ms = 0.f;
  if (rc == HENRY_OK) {
    if (flush_bytes > 0) {
      for (int r = 0; r < reps; ++r) {
        cudaMemsetAsync(flush, r & 0xff, (size_t)flush_bytes, s);
        cudaEventRecord(e0[r], s);
        launch();
        cudaEventRecord(e1[r], s);
      }
    } else {
      cudaEventRecord(e0[0], s);
      for (int r = 0; r < reps; ++r) launch();
      cudaEventRecord(e1[0], s);
    }
    if (cudaEventSynchronize(e1[nev - 1]) != cudaSuccess) rc = HENRY_E_CUDA;
    for (int r = 0; r < nev && rc == HENRY_OK; ++r) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, e0[r], e1[r]) != cudaSuccess) rc = HENRY_E_CUDA;
      ms += t;
    }
  }
  for (int r = 0; r < nev; ++r) {
    if (e0[r]) cudaEventDestroy(e0[r]);
    if (e1[r]) cudaEventDestroy(e1[r]);
  }
  if (rc != HENRY_OK) {
    set_last_error(std::string("time_kernel: ") + cudaGetErrorString(cudaGetLastError()));
    return rc;
  }
  const Geom& G = levels_.back().g;
  const double T = (double)tsize_;
  if (which == 0) {
    const double cells = (double)B * G.half();
    *bytes = cells * 26.0 * T;
    *flops = cells * 32.0;
  } else if (which == 2) {   // residual only: 40 B read, R written (16 B)
    const double cells = (double)B * G.ncell();
    *bytes = cells * 56.0;
    *flops = cells * 46.0;
  } else {
    const double cells = (double)B * G.ncell();
    *bytes = cells * (40.0 + 16.0 + 20.0 * T);
    *flops = cells * (46.0 + (tsize_ == sizeof(double) ? 116.0 : 0.0));
  }
  *avg_ms = ms / reps;
  return HENRY_OK;
}

int Solver::run_series(const double* xi, const double* logk, int B, int every, double* series,
                       double* q, int* status, cudaStream_t s) {
  series_ = series;
  series_every_ = every;
  const int rc = run(xi, logk, B, q, nullptr, nullptr, status, nullptr, 0, s);
  series_ = nullptr;
  series_every_ = 0;
  return rc;
}

int Solver::run(const double* xi, const double* logk, int B, double* q, double* c_out,
                double* p_out, int* status, int* iters, int status_or, cudaStream_t s) {
  if (B == 0) return HENRY_OK;
  int rc = ensure(B, s);
  if (rc) return rc;
  last_B_ = B;
  if (tsize_ == sizeof(float))
    return run_t<float>(xi, logk, B, q, c_out, p_out, status, iters, status_or, s);
  return run_t<double>(xi, logk, B, q, c_out, p_out, status, iters, status_or, s);
}

// ---------------------------------------------------------------------------
// discrete adjoint (see henry_adjoint)
// ---------------------------------------------------------------------------
int Solver::ensure_adjoint(int B, int nckpt, int seglen) {
  if (adj_arena_ && B <= adj_B_ && nckpt <= adj_nckpt_ && seglen <= adj_seg_) return HENRY_OK;
  CK(cudaDeviceSynchronize());
  if (adj_arena_) cudaFree(adj_arena_);
  adj_arena_ = nullptr;
  const Geom& F = levels_.back().g;
  const size_t n = (size_t)F.ncell() * B;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  const size_t o_ck = take((size_t)nckpt * ckpt_width() * n * 8);
  const size_t o_sg = take((size_t)(seglen + 1) * 2 * n * 8);
  const size_t o_j64 = take(20 * n * 8);
  const size_t o_lam = take(2 * n * 8);
  const size_t o_rhs = take(2 * n * 8);
  const size_t o_res = take(2 * n * 8);
  const size_t o_gk = take(n * 8);
  const size_t o_gp = take(n * 8);
  const size_t o_gq = take((size_t)F.ny * B * 8);
  const size_t o_qt = take((size_t)B * kNQ * 8);
  adj_nchunk_ = (F.ncell() + kBlock - 1) / kBlock;
  const size_t o_p2 = take((size_t)adj_nchunk_ * B * 8);
  std::vector<size_t> o_jt(levels_.size());
  for (size_t k = 0; k < levels_.size(); ++k)
    o_jt[k] = take(kJP * (size_t)levels_[k].g.ncell() * B * tsize_);
  CK(cudaMalloc(&adj_arena_, off));
  char* a = (char*)adj_arena_;
  ckpt_ = (double*)(a + o_ck);
  seg_ = (double*)(a + o_sg);
  J64_ = (double*)(a + o_j64);
  lam_ = (double*)(a + o_lam);
  rhs_ = (double*)(a + o_rhs);
  res_ = (double*)(a + o_res);
  gK_ = (double*)(a + o_gk);
  gphi_ = (double*)(a + o_gp);
  gq_ = (double*)(a + o_gq);
  qtmp_ = (double*)(a + o_qt);
  partial2_ = (double*)(a + o_p2);
  JT_.resize(levels_.size());
  for (size_t k = 0; k < levels_.size(); ++k) JT_[k] = a + o_jt[k];
  adj_B_ = B;
  adj_nckpt_ = nckpt;
  adj_seg_ = seglen;
  return HENRY_OK;
}

template <typename T>
int Solver::adjoint_t(const double* xi, const double* logk, int B, int qoi, int kc, double* q,
                      double* dq_dxi, double* dq_dlogk, int* status, cudaStream_t s) {
  MGLevel& F = levels_.back();
  const Geom& G = F.g;
  const size_t n = (size_t)G.ncell() * B;   // doubles per state component
  const int nfull = nt_ / kc;
  const int nck = nfull + 1 + (nt_ % kc ? 1 : 0);
  auto slot_step = [&](int m) { return m <= nfull ? m * kc : nt_; };
  int rc = ensure_adjoint(B, nck, kc);
  if (rc) return rc;
  // a checkpoint holds u^m and the previous states that feed the
  // extrapolated Newton guess of the next step (u^{m-1}, and u^{m-2} ...
  // for guesses of higher order), so recomputed steps are bitwise the
  // forward's;
  // segment states keep u^n only
  auto save = [&](double* dst, bool full) -> int {
    CK(cudaMemcpyAsync(dst, F.p, n * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(dst + n, F.c, n * 8, cudaMemcpyDeviceToDevice, s));
    if (full) {
      CK(cudaMemcpyAsync(dst + 2 * n, p_prev_, n * 8, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(dst + 3 * n, c_old_, n * 8, cudaMemcpyDeviceToDevice, s));
      for (int k = 0; k < hx_.depth; ++k) {
        CK(cudaMemcpyAsync(dst + (4 + 2 * k) * n, hx_.p[k], n * 8, cudaMemcpyDeviceToDevice, s));
        CK(cudaMemcpyAsync(dst + (5 + 2 * k) * n, hx_.c[k], n * 8, cudaMemcpyDeviceToDevice, s));
      }
    }
    return HENRY_OK;
  };
  auto ck = [&](int m) { return ckpt_ + (size_t)m * ckpt_width() * n; };
  // forward with checkpoints
  rc = setup_t<T>(xi, logk, B, s);
  if (rc) return rc;
  // steps recomputed from a checkpoint must be bitwise the forward's, so
  // every step of the adjoint's forward builds its own operators
  k_set_int<<<1, 32, 0, s>>>(counter_, keep_, 0);
  if ((rc = save(ck(0), true))) return rc;
  for (int st = 1; st <= nt_; ++st) {
    if ((rc = step_t<T>(B, s))) return rc;
    if (st % kc == 0) { if ((rc = save(ck(st / kc), true))) return rc; }
    else if (st == nt_) { if ((rc = save(ck(nck - 1), true))) return rc; }
  }
  k_qoi<<<B, kBlock, 0, s>>>(counter_, phys_, G, B, F.p, F.c, F.phi, qtmp_, nullptr, nullptr, kNQ);
  CK(cudaMemcpy2DAsync(q, sizeof(double), qtmp_ + qoi, kNQ * sizeof(double), sizeof(double), B,
                       cudaMemcpyDeviceToDevice, s));
  // seed and zero the sensitivities
  k_adj_seed<<<grid1((int64_t)n), kBlock, 0, s>>>(counter_, phys_, G, B, qoi, F.c, rhs_, lam_);
  CK(cudaMemsetAsync(gK_, 0, n * 8, s));
  CK(cudaMemsetAsync(gphi_, 0, n * 8, s));
  CK(cudaMemsetAsync(gq_, 0, (size_t)G.ny * B * 8, s));
  // transposed solves: relative tolerance, and the rounding-floor stop once
  // the residual is within 1e3 of it (see adjoint_rtol in henry.h)
  const double adj_rtol = cfg_.adjoint_rtol;
  const double adj_stag = 1e3 * cfg_.adjoint_rtol;
  for (int m = nck - 2; m >= 0; --m) {
    const int n0 = slot_step(m), n1 = slot_step(m + 1);
    // recompute the segment's states from its checkpoint (bitwise the forward's)
    CK(cudaMemcpyAsync(F.p, ck(m), n * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(F.c, ck(m) + n, n * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(p_prev_, ck(m) + 2 * n, n * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c_old_, ck(m) + 3 * n, n * 8, cudaMemcpyDeviceToDevice, s));
    for (int k = 0; k < hx_.depth; ++k) {
      CK(cudaMemcpyAsync(hx_.p[k], ck(m) + (4 + 2 * k) * n, n * 8, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(hx_.c[k], ck(m) + (5 + 2 * k) * n, n * 8, cudaMemcpyDeviceToDevice, s));
    }
    k_set_int<<<1, 32, 0, s>>>(counter_, step_, n0);
    if ((rc = save(seg_, false))) return rc;
    for (int st = n0 + 1; st <= n1; ++st) {
      if ((rc = step_t<T>(B, s))) return rc;
      if ((rc = save(seg_ + (size_t)(st - n0) * 2 * n, false))) return rc;
    }
    for (int st = n1; st > n0; --st) {
      const double* u = seg_ + (size_t)(st - n0) * 2 * n;
      const double* uprev = seg_ + (size_t)(st - n0 - 1) * 2 * n;
      CK(cudaMemcpyAsync(F.p, u, n * 8, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(F.c, u + n, n * 8, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(c_old_, uprev + n, n * 8, cudaMemcpyDeviceToDevice, s));
      k_activate<<<grid1(B), kBlock, 0, s>>>(counter_, B, status_w_, active_, it_step_);
      // operators of step st: J (multigrid type, every level) and exact FP64 J
      k_resjac<T, false><<<dim3(nchunk_, B), kBlock, 0, s>>>(
          counter_, phys_, G, G.hx * G.hy / tau_, B, tile_, F.p, F.c, c_old_, F.phi, F.K, F.tx, F.dx, F.ty, F.dy,
          qin_, active_, (T*)F.J, (T*)F.b, (T*)F.x, partial_, F.qx, F.qy, nullptr);
      k_resjac<double, true><<<dim3(nchunk_, B), kBlock, 0, s>>>(
          counter_, phys_, G, G.hx * G.hy / tau_, B, tile_, F.p, F.c, c_old_, F.phi, F.K, F.tx, F.dx, F.ty, F.dy,
          qin_, active_, J64_, res_, nullptr, nullptr, nullptr, nullptr, nullptr);
      enqueue_coarse_ops<T>(B, s, nullptr);
      for (size_t k = 0; k < levels_.size(); ++k)
        k_transpose<T><<<grid1((int64_t)B * levels_[k].g.ncell()), kBlock, 0, s>>>(
            counter_, levels_[k].g, B, active_, (const T*)levels_[k].J, (T*)JT_[k]);
      // the multigrid cycles below read the transposed operators
      for (size_t k = 0; k < levels_.size(); ++k) std::swap(levels_[k].J, JT_[k]);
      enqueue_coarse_inv<T>(B, s, nullptr);
      CK(cudaMemsetAsync(lam_, 0, 2 * n * 8, s));
      for (;;) {
        k_adj_residual<T><<<dim3(adj_nchunk_, B), kBlock, 0, s>>>(
            counter_, G, B, active_, J64_, rhs_, lam_, res_, (const T*)F.J, (T*)F.b, (T*)F.x,
            partial2_);
        k_check<false><<<(B + 7) / 8, kBlock, 0, s>>>(
            counter_, B, adj_nchunk_, G.ncell(), partial2_, 1.0, adj_rtol, 0.0, cfg_.newton_maxit,
            active_, it_step_, res0_, res_last_, status_w_, iters_w_, n_active_, check_acc_, 0.0, 0,
            nullptr, 0, adj_stag);
        CK(cudaMemcpyAsync(n_active_host_, n_active_, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (*n_active_host_ == 0) break;
        enqueue_vcycles<T>(B, s);
        k_adj_update<T><<<grid1((int64_t)n), kBlock, 0, s>>>(counter_, G, B, active_,
                                                             (const T*)F.x, lam_);
      }
      for (size_t k = 0; k < levels_.size(); ++k) std::swap(levels_[k].J, JT_[k]);
      // Eq. e_recharge_of_param: the inflow of step st carries (1 + sin(pi t / 40)), t = st tau
      const double qfac =
          cfg_.field_model == 1 ? 1.0 + sin(3.14159265358979323846 * st * tau_ / 40.0) : 1.0;
      k_adj_sens<<<grid1((int64_t)n), kBlock, 0, s>>>(counter_, phys_, G, tau_, qfac, B, F.p, F.c,
                                                      c_old_,
                                                      F.phi, F.K, F.tx, F.dx, F.ty, F.dy, lam_, gK_,
                                                      gphi_, gq_);
      if (st > 1)
        k_adj_prev_rhs<<<grid1((int64_t)n), kBlock, 0, s>>>(counter_, phys_, G, tau_, B, F.phi,
                                                            c_old_, lam_, rhs_);
    }
  }
  k_adj_contract<<<B, kBlock, 0, s>>>(counter_, phys_, G, B, cfg_.n_xi, cfg_.field_model, xi, gK_,
                                      gphi_, gq_, dq_dxi);
  if (dq_dlogk) CK(cudaMemcpyAsync(dq_dlogk, gK_, n * 8, cudaMemcpyDeviceToDevice, s));
  k_copy_int<<<grid1(B), kBlock, 0, s>>>(counter_, B, status_w_, status, 0);
  CK(cudaGetLastError());
  return HENRY_OK;
}

int Solver::adjoint(const double* xi, const double* logk, int B, int qoi, int ckpt_every,
                    double* q, double* dq_dxi, double* dq_dlogk, int* status, cudaStream_t s) {
  if (B == 0) return HENRY_OK;
  int rc = ensure(B, s);
  if (rc) return rc;
  last_B_ = B;
  const int kc = ckpt_every < 1 ? 1 : (ckpt_every > nt_ ? nt_ : ckpt_every);
  if (tsize_ == sizeof(float))
    return adjoint_t<float>(xi, logk, B, qoi, kc, q, dq_dxi, dq_dlogk, status, s);
  return adjoint_t<double>(xi, logk, B, qoi, kc, q, dq_dxi, dq_dlogk, status, s);
}

// dst[b] |= src[b] on stream s (status of the coarse half of a pair).
int or_status(const int* src, int* dst, int B, unsigned long long* ctr, cudaStream_t s) {
  if (B == 0) return HENRY_OK;
  k_copy_int<<<grid1(B), kBlock, 0, s>>>(ctr, B, src, dst, 1);
  CK(cudaGetLastError());
  return HENRY_OK;
}

cudaError_t launch_residual_jacobian(const Phys& P, const Geom& G, double tau, int B,
                                     const double* phi, const double* K, const double* qin,
                                     const double* p, const double* c, const double* c_old,
                                     double* R, double* J, double* scratch, cudaStream_t s) {
  const int64_t n = (int64_t)B * G.ncell();
  const int grid = (int)((n + kBlock - 1) / kBlock);
  double* tx = scratch;
  double* dx = scratch + n;
  double* ty = scratch + 2 * n;
  double* dy = scratch + 3 * n;
  double* pr = scratch + 4 * n;
  k_face_consts<<<grid, kBlock, 0, s>>>(nullptr, P, G, B, phi, K, tx, dx, ty, dy);
  k_reduce_pressure<<<grid, kBlock, 0, s>>>(P, G, B, p, pr);
  const ResTile tl = make_res_tile(G.nx, G.ny);
  k_resjac<double, true><<<dim3(tl.ntx * tl.nty, B), kBlock, 0, s>>>(
      nullptr, P, G, G.hx * G.hy / tau, B, tl, pr, c, c_old, phi, K, tx, dx, ty, dy, qin, nullptr, J, R, nullptr,
      nullptr, nullptr, nullptr, nullptr);
  return cudaGetLastError();
}

}  // namespace henry
