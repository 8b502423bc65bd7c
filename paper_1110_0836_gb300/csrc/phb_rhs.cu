// Entry points phb_mls_derivs and phb_mhd_rhs: gather the caller's arrays
// into cell (slot) order, run the fused fit, scatter results back.
#include "phb_internal.cuh"

namespace phb {
namespace {

constexpr int kThreads = 256;

__global__ void k_gather_all(Grid g, const int32_t* __restrict__ perm, const double* __restrict__ pos,
                             const double* __restrict__ lam, const double* __restrict__ U,
                             double* __restrict__ spos, double* __restrict__ slam,
                             double* __restrict__ sU, float* __restrict__ rec,
                             int32_t* status_word, double* __restrict__ y0) {
  const int n = g.n;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int i = perm[s];
  double x[3], u[8];
  bool finite = true;
  for (int a = 0; a < 3; ++a) {
    x[a] = pos[a * static_cast<int64_t>(n) + i];
    spos[a * static_cast<int64_t>(n) + s] = x[a];
    if (y0) y0[a * static_cast<int64_t>(n) + s] = x[a];
    finite &= finite64(x[a]);
  }
  const double l = lam[i];
  slam[s] = l;
  if (!lambda_in_range(g, l)) raise_flag(status_word, PHB_FLAG_LAMBDA_RANGE);
  for (int f = 0; f < 8; ++f) {
    u[f] = U ? U[f * static_cast<int64_t>(n) + i] : 0.0;
    sU[f * static_cast<int64_t>(n) + s] = u[f];
    if (y0) y0[(3 + f) * static_cast<int64_t>(n) + s] = u[f];
    finite &= finite64(u[f]);
  }
  if (!finite) raise_flag(status_word, PHB_FLAG_NONFINITE);
  write_record(rec, s, x, u);
}

// Active subset: mark the slots of the listed caller indices, then list the
// marked slots in ascending order from the exclusive scan of the marks.
__global__ void k_mark_active(int n, int64_t m, const int32_t* __restrict__ active,
                              const int32_t* __restrict__ inv, int32_t* __restrict__ mark,
                              int32_t* status_word) {
  const int64_t k = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const int32_t i = active[k];
  if (i < 0 || i >= n) {
    raise_flag(status_word, PHB_FLAG_BAD_INDEX);
    return;
  }
  mark[inv[i]] = 1;
}

__global__ void k_list_active(int n, const int32_t* __restrict__ scan, int32_t* __restrict__ list,
                              int32_t* __restrict__ list_len) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s > n) return;
  if (s == n) {
    *list_len = scan[n];
    return;
  }
  if (scan[s + 1] != scan[s]) list[scan[s]] = s;
}

}  // namespace

cudaError_t run_fit_marked(const phb_plan* plan, const phb_params* prm, void* ws, double* dudt,
                           int32_t* fit_status, int32_t* status_word, cudaStream_t st) {
  const int n = static_cast<int>(plan->n);
  int32_t* mark = region<int32_t>(plan, ws, R_AFLAG);
  int32_t* list = region<int32_t>(plan, ws, R_ALIST);
  int32_t* list_len = region<int32_t>(plan, ws, R_MISC) + 4;
  cudaError_t e = scan_exclusive_i32(mark, n + 1, region<int64_t>(plan, ws, R_SCAN), st);
  if (e) return e;
  k_list_active<<<static_cast<unsigned>((n + 1 + kThreads - 1) / kThreads), kThreads, 0, st>>>(
      n, mark, list, list_len);
  note_launch();
  return run_fit(plan, prm, ws, FitMode::kRHS, region<int32_t>(plan, ws, R_PERM), dudt, nullptr,
                 nullptr, fit_status, status_word, st, list, list_len, n);
}

cudaError_t gather_sorted(const phb_plan* p, const Grid& g, const double* pos, const double* lam,
                          const double* U, void* ws, int32_t* status_word, cudaStream_t st,
                          double* y0) {
  k_gather_all<<<static_cast<unsigned>((g.n + kThreads - 1) / kThreads), kThreads, 0, st>>>(
      g, region<int32_t>(p, ws, R_PERM), pos, lam, U, region<double>(p, ws, R_SPOS),
      region<double>(p, ws, R_SLAM), region<double>(p, ws, R_SU), region<float>(p, ws, R_REC),
      status_word, y0);
  note_launch();
  return cudaGetLastError();
}

FitArgs fit_args(const phb_plan* plan, const phb_params* prm, void* ws, const int32_t* perm_out,
                 double* dudt, double* grad, double* hess, int32_t* fit_status,
                 int32_t* status_word) {
  FitArgs a;
  a.g = make_grid(plan);
  a.n = static_cast<int32_t>(plan->n);
  a.perm_in = region<int32_t>(plan, ws, R_PERM);
  a.perm_out = perm_out;
  a.spos = region<double>(plan, ws, R_SPOS);
  a.slam = region<double>(plan, ws, R_SLAM);
  a.sU = region<double>(plan, ws, R_SU);
  a.rec = region<float>(plan, ws, R_REC);
  a.off = region<int64_t>(plan, ws, R_OFF);
  a.idx = region<int32_t>(plan, ws, R_IDX);
  a.gamma = prm->gamma;
  a.weight_kind = prm->weight_kind;
  a.cond_threshold = static_cast<float>(prm->cond_threshold > 0 ? prm->cond_threshold : 3e4);
  a.zeta = prm->zeta;
  a.eta = prm->eta;
  a.c_zeta_l = prm->c_zeta_l;
  a.c_zeta_a = prm->c_zeta_a;
  a.c_eta = prm->c_eta;
  a.dudt = dudt;
  a.grad = grad;
  a.hess = hess;
  a.fit_status = fit_status;
  a.queue = region<int32_t>(plan, ws, R_QUEUE);
  a.queue_len = region<int32_t>(plan, ws, R_MISC);
  a.status_word = status_word;
  a.refine_mode = prm->refine < 0 ? -1 : (prm->refine > 0 ? 1 : 0);
  a.refine_kappa = static_cast<float>(prm->refine_kappa > 0 ? prm->refine_kappa : 500.0);
  // by size: the queue where the records fit in L2 and lambda varies (sets
  // of one resolution, lattices above all, rarely refine: they skip the
  // queue's launch and refine inside the tile when they do)
  a.refine_queued = prm->refine_schedule == 1 ||
                    (prm->refine_schedule != 2 && static_cast<size_t>(plan->n) * 96 <= l2_bytes() &&
                     plan->lambda_max > 1.01 * plan->lambda_min);
  a.rqueue = region<int32_t>(plan, ws, R_RQUEUE);
  a.rq_len = a.queue_len + 6;
  a.rstash = region<float>(plan, ws, R_RSTASH);
  a.refined_tiles = a.queue_len + 5;
  a.u_host = nullptr;
  a.pc_y0 = nullptr;
  a.pc_f0 = nullptr;
  a.pc_perm = nullptr;
  a.pc_frozen = nullptr;
  a.pc_done = nullptr;
  a.pc_h = 0.0;
  return a;
}

cudaError_t run_fit(const phb_plan* plan, const phb_params* prm, void* ws, FitMode mode,
                    const int32_t* perm_out, double* dudt, double* grad, double* hess,
                    int32_t* fit_status, int32_t* status_word, cudaStream_t st,
                    const int32_t* list, const int32_t* list_len, int64_t list_cap,
                    const HostU* hu) {
  FitArgs a = fit_args(plan, prm, ws, perm_out, dudt, grad, hess, fit_status, status_word);
  if (hu && mode == FitMode::kRHS && !list && !perm_out && prm->precision != PHB_FP64) {
    a.u_host = hu->u_host;
    a.pc_y0 = hu->y0;
    a.pc_f0 = hu->f0;
    a.pc_perm = hu->perm;
    a.pc_frozen = hu->frozen;
    a.pc_done = hu->done;
    a.pc_h = hu->h;
  }
  cudaError_t e;
  if (prm->precision == PHB_FP64) return launch_fit_fp64(a, mode, list, list_len, st);
  if ((e = cudaMemsetAsync(a.queue_len, 0, sizeof(int32_t), st))) return e;
  if ((e = cudaMemsetAsync(a.queue_len + 2, 0, sizeof(int32_t), st))) return e;
  if ((e = cudaMemsetAsync(a.refined_tiles, 0, 2 * sizeof(int32_t), st))) return e;  // and rq_len
  if ((e = launch_fit_mixed(a, mode, region<int2>(plan, ws, R_TPLAN), region<int32_t>(plan, ws, R_TSLOT),
                            region<uint16_t>(plan, ws, R_LSELF), region<uint8_t>(plan, ws, R_TMAP),
                            region<uint16_t>(plan, ws, R_LIDX),
                            a.queue_len + 2,
                            region<int32_t>(plan, ws, R_TORDER), list, list_len, list_cap, st)))
    return e;
  return launch_fit_fp64(a, mode, a.queue, a.queue_len, st, true);
}

}  // namespace phb

using namespace phb;

namespace {

phb_status fit_entry(const phb_plan* plan, const phb_params* prm, const double* pos,
                     const double* lambda, const double* U, void* ws, size_t ws_bytes, FitMode mode,
                     double* dudt, double* grad, double* hess, int32_t* fit_status,
                     int32_t* status_word, phb_stream_t stream) {
  phb_status s = check_common(plan, ws, ws_bytes, plan ? plan->ws_off[R_END_COMMON] : 0);
  if (s != PHB_OK) return s;
  if (!prm || !pos || !lambda || !U) return PHB_ERR_INVALID_ARG;
  if (prm->precision != PHB_FP64 && prm->precision != PHB_FP32_MIXED) return PHB_ERR_INVALID_ARG;
  if (prm->weight_kind != 0 && prm->weight_kind != 1) return PHB_ERR_INVALID_ARG;
  if (!(prm->gamma > 1.0)) return PHB_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Grid g = make_grid(plan);
  cudaError_t e = gather_sorted(plan, g, pos, lambda, U, ws, status_word, st);
  if (e == cudaSuccess)
    e = run_fit(plan, prm, ws, mode, region<int32_t>(plan, ws, R_PERM), dudt, grad, hess,
                fit_status, status_word, st);
  return launch_status(e);
}

}  // namespace

extern "C" phb_status phb_mls_derivs(const phb_plan* plan, const phb_params* params,
                                     const double* pos, const double* lambda, const double* U,
                                     void* ws, size_t ws_bytes, double* grad, double* hess,
                                     int32_t* fit_status, int32_t* status_word,
                                     phb_stream_t stream) {
  if (!grad) return PHB_ERR_INVALID_ARG;
  return fit_entry(plan, params, pos, lambda, U, ws, ws_bytes, FitMode::kDerivs, nullptr, grad,
                   hess, fit_status, status_word, stream);
}

extern "C" phb_status phb_mhd_rhs_active(const phb_plan* plan, const phb_params* prm,
                                         const double* pos, const double* lambda, const double* U,
                                         const int32_t* active, int64_t n_active, void* ws,
                                         size_t ws_bytes, double* dudt, int32_t* fit_status,
                                         int32_t* status_word, phb_stream_t stream) {
  phb_status s = check_common(plan, ws, ws_bytes, plan ? plan->ws_off[R_END_COMMON] : 0);
  if (s != PHB_OK) return s;
  if (!prm || !pos || !lambda || !U || !dudt || n_active < 0 || (n_active > 0 && !active))
    return PHB_ERR_INVALID_ARG;
  if (prm->precision != PHB_FP64 && prm->precision != PHB_FP32_MIXED) return PHB_ERR_INVALID_ARG;
  if (prm->weight_kind != 0 && prm->weight_kind != 1) return PHB_ERR_INVALID_ARG;
  if (!(prm->gamma > 1.0)) return PHB_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Grid g = make_grid(plan);
  const int n = g.n;
  int32_t* mark = region<int32_t>(plan, ws, R_AFLAG);
  int32_t* list = region<int32_t>(plan, ws, R_ALIST);
  int32_t* list_len = region<int32_t>(plan, ws, R_MISC) + 4;
  cudaError_t e = gather_sorted(plan, g, pos, lambda, U, ws, status_word, st);
  if (e) return launch_status(e);
  if ((e = cudaMemsetAsync(mark, 0, (size_t(n) + 1) * sizeof(int32_t), st))) return launch_status(e);
  if (n_active > 0) {
    k_mark_active<<<static_cast<unsigned>((n_active + kThreads - 1) / kThreads), kThreads, 0, st>>>(
        n, n_active, active, region<int32_t>(plan, ws, R_INV), mark, status_word);
    note_launch();
  }
  if ((e = scan_exclusive_i32(mark, n + 1, region<int64_t>(plan, ws, R_SCAN), st))) return launch_status(e);
  k_list_active<<<static_cast<unsigned>((n + 1 + kThreads - 1) / kThreads), kThreads, 0, st>>>(
      n, mark, list, list_len);
  note_launch();
  const int64_t cap = n_active < n ? n_active : n;
  e = run_fit(plan, prm, ws, FitMode::kRHS, region<int32_t>(plan, ws, R_PERM), dudt, nullptr,
              nullptr, fit_status, status_word, st, list, list_len, cap);
  return launch_status(e);
}

extern "C" int phb_fit_tc_experiment(const phb_plan* plan, const phb_params* prm, const double* pos,
                                     const double* lambda, const double* U, void* ws,
                                     size_t ws_bytes, float* gram, size_t gram_bytes, double* dudt,
                                     int32_t* status_word, phb_stream_t stream) {
  phb_status s = check_common(plan, ws, ws_bytes, plan ? plan->ws_off[R_END_COMMON] : 0);
  if (s != PHB_OK) return s;
  if (!prm || !pos || !lambda || !U || !dudt || !gram || plan->tile != 128 ||
      prm->precision != PHB_FP32_MIXED || (prm->weight_kind != 0 && prm->weight_kind != 1) ||
      !(prm->gamma > 1.0) || gram_bytes < size_t(80 + 7 * 19 + 1) * 4 * size_t(plan->n))
    return PHB_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Grid g = make_grid(plan);
  cudaError_t e = gather_sorted(plan, g, pos, lambda, U, ws, status_word, st);
  if (e) return launch_status(e);
  const FitArgs a = fit_args(plan, prm, ws, region<int32_t>(plan, ws, R_PERM), dudt, nullptr,
                             nullptr, nullptr, status_word);
  e = launch_fit_tc(a, region<int2>(plan, ws, R_TPLAN), region<int32_t>(plan, ws, R_TSLOT),
                    region<uint16_t>(plan, ws, R_LSELF), region<uint8_t>(plan, ws, R_TMAP),
                    region<uint16_t>(plan, ws, R_LIDX), gram, st);
  return launch_status(e);
}

extern "C" phb_status phb_mhd_rhs(const phb_plan* plan, const phb_params* params, const double* pos,
                                  const double* lambda, const double* U, void* ws, size_t ws_bytes,
                                  double* dudt, int32_t* fit_status, int32_t* status_word,
                                  phb_stream_t stream) {
  if (!dudt) return PHB_ERR_INVALID_ARG;
  return fit_entry(plan, params, pos, lambda, U, ws, ws_bytes, FitMode::kRHS, dudt, nullptr,
                   nullptr, fit_status, status_word, stream);
}
