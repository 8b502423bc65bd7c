// Individual power-of-two time steps (Paper II Sec. 2: every particle has its
// own step; Sec. 2.1: steps rounded down to powers of two, organised as
// GADGET's binary blocks), each particle advanced by the second-order
// predictor-corrector read as Heun.  Readings where the paper defers to
// GADGET's scheme:
//   * a synchronised step of dt_max is cut into 2^max_level substeps of
//     delta; a particle of level L takes steps of m = 2^(max_level - L)
//     substeps, all starting together;
//   * each particle keeps an anchor - its state (x0, U0) and dU/dt at the
//     start of its current step - and its current state at substep time t is
//     the prediction (x0, U0) + (t - t0) (V0, dU0/dt);
//   * at substep time t the particles whose step ends there are corrected,
//     x = x0 + (Delta/2)(V0 + V), U = U0 + (Delta/2)(dU0/dt + F), F the
//     right-hand side at the current states of all particles, Delta = m delta;
//     the right-hand side at the corrected states (the others still at their
//     predictions) is the derivative of their new anchor.
// With every particle on one level this is the plain Heun step.  Neighbour
// sets are rebuilt at the positions of each evaluation.
#include "phb_internal.cuh"

namespace phb {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int level_of(const int32_t* levels, int i, int max_level,
                                        int32_t* status_word) {
  int L = levels[i];
  if (L < 0 || L > max_level) {
    raise_flag(status_word, PHB_FLAG_BAD_INDEX);
    L = L < 0 ? 0 : max_level;
  }
  return L;
}

// Current states at t_{k+1} from the anchors: (x, U) = (x0, U0) + tau (V0, F0),
// tau = (k + 1 - s) delta, s the substep at which the particle's step began.
__global__ void k_block_drift(int n, const int32_t* __restrict__ levels, int k, int max_level,
                              double delta, const double* __restrict__ anc, double* __restrict__ pos,
                              double* __restrict__ U, int32_t* status_word) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t N = n;
  const int L = level_of(levels, i, max_level, status_word);
  const int m = 1 << (max_level - L);
  const int s = (k / m) * m;
  const double tau = static_cast<double>(k + 1 - s) * delta;
  for (int a = 0; a < 3; ++a) pos[a * N + i] = anc[a * N + i] + tau * anc[(3 + 1 + a) * N + i];
  for (int f = 0; f < 8; ++f) U[f * N + i] = anc[(3 + f) * N + i] + tau * anc[(11 + f) * N + i];
}

// Mark (slot order) the particles whose step ends at t_{k+1}.
__global__ void k_block_mark(int n, const int32_t* __restrict__ perm,
                             const int32_t* __restrict__ levels, int k, int max_level,
                             int32_t* __restrict__ mark) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s > n) return;
  if (s == n) {
    mark[n] = 0;
    return;
  }
  int L = levels[perm[s]];
  L = L < 0 ? 0 : (L > max_level ? max_level : L);
  mark[s] = (k + 1) % (1 << (max_level - L)) == 0 ? 1 : 0;
}

// Corrector of the particles whose step ends at t_{k+1}; their anchors' states
// become the corrected ones.
__global__ void k_block_correct(int n, const int32_t* __restrict__ levels, int k, int max_level,
                                double delta, const double* __restrict__ F, double* __restrict__ anc,
                                double* __restrict__ pos, double* __restrict__ U) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t N = n;
  int L = levels[i];
  L = L < 0 ? 0 : (L > max_level ? max_level : L);
  const int m = 1 << (max_level - L);
  if ((k + 1) % m != 0) return;
  const double half = 0.5 * (static_cast<double>(m) * delta);
  for (int a = 0; a < 3; ++a) {
    const double x = anc[a * N + i] + half * (anc[(3 + 1 + a) * N + i] + U[(1 + a) * N + i]);
    pos[a * N + i] = x;
    anc[a * N + i] = x;
  }
  for (int f = 0; f < 8; ++f) {
    const double u = anc[(3 + f) * N + i] + half * (anc[(11 + f) * N + i] + F[f * N + i]);
    U[f * N + i] = u;
    anc[(3 + f) * N + i] = u;
  }
}

// New anchor derivatives of the particles whose step ended at t_{k+1} (k < 0:
// all particles, with their states as the anchor states).
__global__ void k_block_anchor(int n, const int32_t* __restrict__ levels, int k, int max_level,
                               const double* __restrict__ F, const double* __restrict__ pos,
                               const double* __restrict__ U, double* __restrict__ anc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t N = n;
  if (k >= 0) {
    int L = levels[i];
    L = L < 0 ? 0 : (L > max_level ? max_level : L);
    if ((k + 1) % (1 << (max_level - L)) != 0) return;
  } else {
    for (int a = 0; a < 3; ++a) anc[a * N + i] = pos[a * N + i];
    for (int f = 0; f < 8; ++f) anc[(3 + f) * N + i] = U[f * N + i];
  }
  for (int f = 0; f < 8; ++f) anc[(11 + f) * N + i] = F[f * N + i];
}

// Right-hand side at (pos, U) of the particles whose step ends at t_{k+1}, or
// of all particles when levels is null: neighbour lists at pos, gather into
// slot order, mark, fit; F in caller order at the evaluated ones.
cudaError_t marked_rhs(const phb_plan* plan, const phb_params* prm, const double* pos,
                       const double* lam, const double* U, const int32_t* levels, int k,
                       int max_level, void* ws, double* F, int32_t* status_word, cudaStream_t st) {
  cudaError_t e = build_neighbors_impl(plan, pos, lam, ws, status_word, st);
  if (e) return e;
  const Grid g = make_grid(plan);
  if ((e = gather_sorted(plan, g, pos, lam, U, ws, status_word, st))) return e;
  if (!levels)
    return run_fit(plan, prm, ws, FitMode::kRHS, region<int32_t>(plan, ws, R_PERM), F, nullptr,
                   nullptr, nullptr, status_word, st);
  const int n = g.n;
  k_block_mark<<<static_cast<unsigned>((n + 1 + kThreads - 1) / kThreads), kThreads, 0, st>>>(
      n, region<int32_t>(plan, ws, R_PERM), levels, k, max_level, region<int32_t>(plan, ws, R_AFLAG));
  note_launch();
  return run_fit_marked(plan, prm, ws, F, nullptr, status_word, st);
}

phb_status check_block(const phb_plan* plan, const phb_params* prm, void* ws, size_t ws_bytes) {
  size_t need = plan ? plan->ws_off[R_PC_F0] + size_t(8) * 8 * plan->n : 0;
  phb_status s = check_common(plan, ws, ws_bytes, need);
  if (s != PHB_OK) return s;
  if (!prm || (prm->precision != PHB_FP64 && prm->precision != PHB_FP32_MIXED) ||
      (prm->weight_kind != 0 && prm->weight_kind != 1) || !(prm->gamma > 1.0))
    return PHB_ERR_INVALID_ARG;
  return PHB_OK;
}

}  // namespace
}  // namespace phb

using namespace phb;

extern "C" phb_status phb_block_begin(const phb_plan* plan, const phb_params* prm, const double* pos,
                                      const double* lambda, const double* U, double* anchor,
                                      void* ws, size_t ws_bytes, int32_t* status_word,
                                      phb_stream_t stream) {
  phb_status s = check_block(plan, prm, ws, ws_bytes);
  if (s != PHB_OK) return s;
  if (!pos || !lambda || !U || !anchor) return PHB_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int n = static_cast<int>(plan->n);
  double* F = region<double>(plan, ws, R_PC_F0);
  cudaError_t e = marked_rhs(plan, prm, pos, lambda, U, nullptr, -1, 0, ws, F, status_word, st);
  if (e) return launch_status(e);
  k_block_anchor<<<static_cast<unsigned>((n + kThreads - 1) / kThreads), kThreads, 0, st>>>(
      n, nullptr, -1, 0, F, pos, U, anchor);
  note_launch();
  return launch_status(cudaSuccess);
}

extern "C" phb_status phb_block_substep(const phb_plan* plan, const phb_params* prm, double* pos,
                                        const double* lambda, double* U, double* anchor,
                                        const int32_t* levels, int32_t k, int32_t max_level,
                                        double dt_max, void* ws, size_t ws_bytes,
                                        int32_t* status_word, phb_stream_t stream) {
  phb_status s = check_block(plan, prm, ws, ws_bytes);
  if (s != PHB_OK) return s;
  if (!pos || !lambda || !U || !anchor || !levels) return PHB_ERR_INVALID_ARG;
  if (max_level < 0 || max_level > 30 || k < 0 || k >= (1 << max_level) || !(dt_max > 0.0))
    return PHB_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int n = static_cast<int>(plan->n);
  const unsigned nb = static_cast<unsigned>((n + kThreads - 1) / kThreads);
  const double delta = dt_max / static_cast<double>(1 << max_level);
  double* F = region<double>(plan, ws, R_PC_F0);
  k_block_drift<<<nb, kThreads, 0, st>>>(n, levels, k, max_level, delta, anchor, pos, U, status_word);
  note_launch();
  cudaError_t e = marked_rhs(plan, prm, pos, lambda, U, levels, k, max_level, ws, F, status_word, st);
  if (e) return launch_status(e);
  k_block_correct<<<nb, kThreads, 0, st>>>(n, levels, k, max_level, delta, F, anchor, pos, U);
  note_launch();
  if ((e = marked_rhs(plan, prm, pos, lambda, U, levels, k, max_level, ws, F, status_word, st)))
    return launch_status(e);
  k_block_anchor<<<nb, kThreads, 0, st>>>(n, levels, k, max_level, F, pos, U, anchor);
  note_launch();
  return launch_status(cudaSuccess);
}
