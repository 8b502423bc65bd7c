// Kelvin-Helmholtz mode amplitude by a discrete convolution over the
// particles (Paper II Sec. 3.4): with e_i = exp(-k |y~_i - y0|), y~ = y below
// ly / 2 and ly - y above it (the layer and its mirror image),
//   s = sum Vy_i sin(k x_i) e_i,  c = sum Vy_i cos(k x_i) e_i,  d = sum e_i^2,
//   M = 2 [ (s / d)^2 + (c / d)^2 ]^(1/2).
// FP64.  The sums are formed by a fixed grid of blocks, each over a fixed
// stride of particles, and the block partials are added in block order by one
// block, so the result does not depend on scheduling.
#include "phb_internal.cuh"

namespace phb {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void block_sum3(double (&v)[3], double* sm) {
  // tree reduction over the block in a fixed order
  const int t = threadIdx.x;
  for (int k = 0; k < 3; ++k) sm[k * kThreads + t] = v[k];
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (t < w)
      for (int k = 0; k < 3; ++k) sm[k * kThreads + t] += sm[k * kThreads + t + w];
    __syncthreads();
  }
  for (int k = 0; k < 3; ++k) v[k] = sm[k * kThreads];
}

__global__ void __launch_bounds__(kThreads) k_kh_partial(int64_t n, const double* __restrict__ pos,
                                                         const double* __restrict__ U, double k,
                                                         double y0, double ly,
                                                         double* __restrict__ part) {
  __shared__ double sm[3 * kThreads];
  double v[3] = {0.0, 0.0, 0.0};
  const double half = 0.5 * ly;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * kThreads) {
    const double x = pos[i], y = pos[n + i], vy = U[2 * n + i];
    const double yt = y < half ? y : ly - y;
    const double e = exp(-k * fabs(yt - y0));
    double sn, cs;
    sincos(k * x, &sn, &cs);
    v[0] += vy * sn * e;
    v[1] += vy * cs * e;
    v[2] += e * e;
  }
  block_sum3(v, sm);
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) part[q * gridDim.x + blockIdx.x] = v[q];
}

__global__ void __launch_bounds__(kThreads) k_kh_final(int nb, const double* __restrict__ part,
                                                       double* __restrict__ out) {
  __shared__ double sm[3 * kThreads];
  double v[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += kThreads)
    for (int q = 0; q < 3; ++q) v[q] += part[q * nb + b];
  block_sum3(v, sm);
  if (threadIdx.x == 0) {
    out[0] = v[0];
    out[1] = v[1];
    out[2] = v[2];
    const double a = v[0] / v[2], b = v[1] / v[2];
    out[3] = 2.0 * sqrt(a * a + b * b);
  }
}

}  // namespace
}  // namespace phb

using namespace phb;

extern "C" phb_status phb_kh_mode_amplitude(const phb_plan* plan, const double* pos, const double* U,
                                            double k, double y0, double ly, void* ws,
                                            size_t ws_bytes, double* out, phb_stream_t stream) {
  phb_status s = check_common(plan, ws, ws_bytes, plan ? plan->ws_off[R_END_COMMON] : 0);
  if (s != PHB_OK) return s;
  if (!pos || !U || !out || !(k > 0.0) || !(ly > 0.0) || !isfinite(k) || !isfinite(ly) ||
      !isfinite(y0))
    return PHB_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double* part = region<double>(plan, ws, R_DIAG);
  k_kh_partial<<<kDiagBlocks, kThreads, 0, st>>>(plan->n, pos, U, k, y0, ly, part);
  note_launch();
  k_kh_final<<<1, kThreads, 0, st>>>(kDiagBlocks, part, out);
  note_launch();
  return launch_status(cudaSuccess);
}
