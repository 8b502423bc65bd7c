// Individual power-of-two time-step levels with the spatial limiter
// (Paper II Sec. 2: each particle has its own step, independent of the bulk
// velocity, with its spatial variation limited; Sec. 2.1: steps rounded down
// to powers of two, the restriction sent from a particle to the neighbours of
// that particle).  The step is the Courant step on the fast magnetosonic
// bound; every floating-point operation that decides a level is a single
// IEEE-rounded FP64 operation (no contraction), so levels are exact integers
// of the definition.
#include "phb_internal.cuh"

namespace phb {
namespace {

constexpr int kThreads = 256;

// Unlimited level of every slot: the smallest L in [0, max_level] with
// dt_max / 2^L <= dt_i, dt_i = cfl lambda_i / sqrt((gamma P + |B|^2) / rho).
__global__ void k_levels0(Grid g, const double* __restrict__ slam, const double* __restrict__ sU,
                          double gamma, double cfl, double dt_max, int max_level,
                          int32_t* __restrict__ L0, int32_t* status_word) {
  const int n = g.n;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int64_t N = n;
  const double rho = sU[s], sig = sU[7 * N + s];
  const double bx = sU[4 * N + s], by = sU[5 * N + s], bz = sU[6 * N + s];
  const double P = __dmul_rn(__dsub_rn(gamma, 1.0), sig);
  const double B2 = __dadd_rn(__dadd_rn(__dmul_rn(bx, bx), __dmul_rn(by, by)), __dmul_rn(bz, bz));
  const double c2 = __ddiv_rn(__dadd_rn(__dmul_rn(gamma, P), B2), rho);
  if (!(rho > 0.0) || !(c2 > 0.0)) raise_flag(status_word, PHB_FLAG_NONFINITE);
  const double dt = __ddiv_rn(__dmul_rn(cfl, slam[s]), __dsqrt_rn(c2));
  int L = 0;
  while (L < max_level && ldexp(dt_max, -L) > dt) ++L;
  L0[s] = L;
}

// Limiter: every particle lifts its neighbours (exactly within r_f) to at
// least its own unlimited level minus one.  A max is order-independent, so
// the result does not depend on thread scheduling.
__global__ void k_levels_limit(Grid g, const double* __restrict__ spos, const double* __restrict__ slam,
                               const int64_t* __restrict__ off, const int32_t* __restrict__ idx,
                               const int32_t* __restrict__ L0, int32_t* __restrict__ L) {
  const int n = g.n;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int send = L0[s] - 1;
  if (send <= 0) return;  // levels are >= 0 already
  const double r = __dmul_rn(g.rf_factor, slam[s]);
  const double r2 = __dmul_rn(r, r);
  const int64_t e1 = off[s + 1] < g.capacity ? off[s + 1] : g.capacity;
  for (int64_t e = off[s]; e < e1; ++e) {
    const int t = idx[e];
    // only a neighbour below the level sent can change; the exact r_f test
    // (FP64) decides the rest
    if (send > L0[t] && dist2_exact(g, spos, n, s, t) < r2) atomicMax(&L[t], send);
  }
}

__global__ void k_levels_out(int n, const int32_t* __restrict__ perm, const int32_t* __restrict__ L,
                             int32_t* __restrict__ levels) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) levels[perm[s]] = L[s];
}

}  // namespace
}  // namespace phb

using namespace phb;

extern "C" phb_status phb_timestep_levels(const phb_plan* plan, const phb_params* prm,
                                          const double* pos, const double* lambda, const double* U,
                                          double cfl, double dt_max, int32_t max_level, void* ws,
                                          size_t ws_bytes, int32_t* levels, int32_t* status_word,
                                          phb_stream_t stream) {
  phb_status s = check_common(plan, ws, ws_bytes, plan ? plan->ws_off[R_END_COMMON] : 0);
  if (s != PHB_OK) return s;
  if (!prm || !pos || !lambda || !U || !levels) return PHB_ERR_INVALID_ARG;
  if (!(cfl > 0.0) || !(dt_max > 0.0) || max_level < 0 || max_level > 30) return PHB_ERR_INVALID_ARG;
  if (!(prm->gamma > 1.0)) return PHB_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Grid g = make_grid(plan);
  const int n = g.n;
  cudaError_t e = gather_sorted(plan, g, pos, lambda, U, ws, status_word, st);
  if (e) return launch_status(e);
  int32_t* L0 = region<int32_t>(plan, ws, R_AFLAG);
  int32_t* L = region<int32_t>(plan, ws, R_ALIST);
  const unsigned nb = static_cast<unsigned>((n + kThreads - 1) / kThreads);
  k_levels0<<<nb, kThreads, 0, st>>>(g, region<double>(plan, ws, R_SLAM), region<double>(plan, ws, R_SU),
                                     prm->gamma, cfl, dt_max, max_level, L0, status_word);
  note_launch();
  if ((e = cudaMemcpyAsync(L, L0, size_t(n) * sizeof(int32_t), cudaMemcpyDeviceToDevice, st)))
    return launch_status(e);
  k_levels_limit<<<nb, kThreads, 0, st>>>(g, region<double>(plan, ws, R_SPOS),
                                          region<double>(plan, ws, R_SLAM),
                                          region<int64_t>(plan, ws, R_OFF),
                                          region<int32_t>(plan, ws, R_IDX), L0, L);
  note_launch();
  k_levels_out<<<nb, kThreads, 0, st>>>(n, region<int32_t>(plan, ws, R_PERM), L, levels);
  note_launch();
  return launch_status(cudaSuccess);
}
