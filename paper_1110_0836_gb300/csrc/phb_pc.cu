// Second-order predictor-corrector step (Paper II Sec. 2; Sec. 4.2 "explicit
// Hermitian time integration"), read as Heun's method on Y = (x, U):
//   Y^p = Y^n + dt F(Y^n),   Y^{n+1} = Y^n + dt/2 (F(Y^n) + F(Y^p)),
// with dx/dt = V and lambda unchanged.  One neighbour build per step at x^n
// with radius r_f + skin; both right-hand-side evaluations filter the lists
// at r_f with their own positions.  The whole step is a fixed sequence of
// launches on one stream (no host synchronisation), so it can be captured
// in a CUDA graph.  Particles marked in params->frozen keep x and U.
#include <cmath>
#include <mutex>

#include "phb_internal.cuh"

namespace phb {
namespace {

constexpr int kThreads = 256;

// Y^p = Y^n + dt F(Y^n) in slot order; refresh the FP32 records; flag a
// displacement above half the skin (the lists would then miss pairs).  A
// frozen particle (mask in caller order) keeps Y^n.
__global__ void k_predict(Grid g, double dt, const double* __restrict__ y0,
                          const double* __restrict__ f0, const int32_t* __restrict__ perm,
                          const uint8_t* __restrict__ frozen, double* __restrict__ spos,
                          double* __restrict__ sU, float* __restrict__ rec, int32_t* status_word) {
  const int n = g.n;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int64_t N = n;
  const double h = (frozen && frozen[perm[s]]) ? 0.0 : dt;
  double x[3], u[8];
  double disp2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double d = h * y0[(3 + 1 + a) * N + s];  // dt * V^n
    x[a] = y0[a * N + s] + d;
    spos[a * N + s] = x[a];
    disp2 += d * d;
  }
  for (int f = 0; f < 8; ++f) {
    u[f] = y0[(3 + f) * N + s] + h * f0[f * N + s];
    sU[f * N + s] = u[f];
  }
  if (4.0 * disp2 > g.skin * g.skin) raise_flag(status_word, PHB_FLAG_SKIN);
  write_record(rec, s, x, u);
}

// Y^{n+1} = Y^n + dt/2 (F(Y^n) + F(Y^p)), written to the caller's arrays;
// a frozen particle's entries are left as they are.  parts: 1 = positions
// (they need only V^n and V^p, so they can be written before F(Y^p) is
// known), 2 = fields (f1 = F(Y^p)), 3 = both.
__global__ void k_correct(int n, double dt, const int32_t* __restrict__ perm,
                          const uint8_t* __restrict__ frozen, const double* __restrict__ y0,
                          const double* __restrict__ sU_p, const double* __restrict__ f0,
                          const double* __restrict__ f1, double* __restrict__ pos,
                          double* __restrict__ U, int parts, const uint8_t* __restrict__ done) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int64_t N = n;
  const int i = perm[s];
  if (frozen && frozen[i]) return;
  const double h = 0.5 * dt;
  // x^n + h (V^n + V^p), U^n + h (F(Y^n) + F(Y^p)): one rounding of the sum,
  // one fused multiply-add (the corrector's fit writes U^{n+1} the same way)
  if (parts & 1)
    for (int a = 0; a < 3; ++a)
      pos[a * N + i] = __fma_rn(h, __dadd_rn(y0[(3 + 1 + a) * N + s], sU_p[(1 + a) * N + s]), y0[a * N + s]);
  if ((parts & 2) && !(done && done[s]))  // (done: already on the host)
    for (int f = 0; f < 8; ++f)
      U[f * N + i] = __fma_rn(h, __dadd_rn(f0[f * N + s], f1[f * N + s]), y0[(3 + f) * N + s]);
}

// Host-buffer step: U^{n+1} of the particles the corrector's fit did not
// write to the host (routed or queued fits, frozen particles, warps of
// scattered caller indices), in caller order, to the mapped host array.
__global__ void k_download_rest(int n, const int32_t* __restrict__ inv, const uint8_t* __restrict__ done,
                                const double* __restrict__ U, double* __restrict__ U_host) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || done[inv[i]]) return;
  const int64_t N = n;
  for (int f = 0; f < 8; ++f) U_host[f * N + i] = U[f * N + i];
}

// Side work of the host-buffer step: the upload of U to wait for before U is
// first read, and the download of x^{n+1} started on a side stream as soon as
// the positions are corrected (before the second fit).
struct PcOverlap {
  cudaEvent_t wait_U = nullptr;
  cudaStream_t side = nullptr;
  cudaEvent_t pos_ready = nullptr, pos_copied = nullptr;
  double* pos_out = nullptr;
  double* U_host = nullptr;  // mapped U_out: U^{n+1} written by the corrector (else copied after)
};

// The step on device arrays, with the overlaps of `ov` if given.
phb_status pc_step_impl(const phb_plan* plan, const phb_params* prm, double* pos,
                        const double* lambda, double* U, double dt, void* ws, int32_t* status_word,
                        cudaStream_t st, const PcOverlap* ov) {
  const Grid g = make_grid(plan);
  const int n = g.n;
  double* y0 = region<double>(plan, ws, R_PC_Y0);
  double* f0 = region<double>(plan, ws, R_PC_F0);
  double* f1 = region<double>(plan, ws, R_PC_F1);
  double* spos = region<double>(plan, ws, R_SPOS);
  double* sU = region<double>(plan, ws, R_SU);
  const unsigned blocks = static_cast<unsigned>((n + kThreads - 1) / kThreads);
  cudaError_t e;
  if ((e = build_neighbors_impl(plan, pos, lambda, ws, status_word, st))) return launch_status(e);
  if (ov && (e = cudaStreamWaitEvent(st, ov->wait_U, 0))) return launch_status(e);
  if ((e = gather_sorted(plan, g, pos, lambda, U, ws, status_word, st, y0)))
    return launch_status(e);
  if ((e = run_fit(plan, prm, ws, FitMode::kRHS, nullptr, f0, nullptr, nullptr, nullptr,
                   status_word, st)))
    return launch_status(e);
  const int32_t* perm = region<int32_t>(plan, ws, R_PERM);
  k_predict<<<blocks, kThreads, 0, st>>>(g, dt, y0, f0, perm, prm->frozen, spos, sU,
                                         region<float>(plan, ws, R_REC), status_word);
  note_launch();
  if (ov) {
    // x^{n+1} now, and its download beside the second fit
    k_correct<<<blocks, kThreads, 0, st>>>(n, dt, perm, prm->frozen, y0, sU, f0, nullptr, pos, U, 1,
                                           nullptr);
    note_launch();
    if ((e = cudaEventRecord(ov->pos_ready, st)) ||
        (e = cudaStreamWaitEvent(ov->side, ov->pos_ready, 0)) ||
        (e = cudaMemcpyAsync(ov->pos_out, pos, 3 * size_t(n) * sizeof(double),
                             cudaMemcpyDeviceToHost, ov->side)) ||
        (e = cudaEventRecord(ov->pos_copied, ov->side)))
      return launch_status(e);
  }
  // the corrector; on the host-buffer step with a mapped U_out its fit writes
  // U^{n+1} of most particles straight to the host, the rest follows
  const bool direct = ov && ov->U_host && prm->precision == PHB_FP32_MIXED;
  uint8_t* done = direct ? region<uint8_t>(plan, ws, R_PC_DONE) : nullptr;
  HostU hu{ov ? ov->U_host : nullptr, y0, f0, perm, prm->frozen, done, 0.5 * dt};
  if ((e = run_fit(plan, prm, ws, FitMode::kRHS, nullptr, f1, nullptr, nullptr, nullptr,
                   status_word, st, nullptr, nullptr, 0, direct ? &hu : nullptr)))
    return launch_status(e);
  k_correct<<<blocks, kThreads, 0, st>>>(n, dt, perm, prm->frozen, y0, sU, f0, f1, pos, U,
                                         ov ? 2 : 3, done);
  note_launch();
  if (direct) {
    k_download_rest<<<blocks, kThreads, 0, st>>>(n, region<int32_t>(plan, ws, R_INV), done, U,
                                                 ov->U_host);
    note_launch();
  }
  if (ov && (e = cudaStreamWaitEvent(st, ov->pos_copied, 0))) return launch_status(e);
  return launch_status(cudaSuccess);
}

phb_status pc_args(const phb_plan* plan, const phb_params* prm, const void* pos, const void* lambda,
                   const void* U, double dt, void* ws, size_t ws_bytes) {
  phb_status s = check_common(plan, ws, ws_bytes, plan ? plan->ws_off[R_END_PC] : 0);
  if (s != PHB_OK) return s;
  if (!prm || !pos || !lambda || !U || !std::isfinite(dt)) return PHB_ERR_INVALID_ARG;
  if (prm->precision != PHB_FP64 && prm->precision != PHB_FP32_MIXED) return PHB_ERR_INVALID_ARG;
  return PHB_OK;
}

// A side stream and two events per device for the host-buffer step, made on
// first use and kept for the process.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr, pos_ready = nullptr, pos_copied = nullptr;
};
std::mutex g_side_mu;
SideStream g_side[64];

cudaError_t side_stream(SideStream*& out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_side_mu);
  SideStream& ss = g_side[dev];
  if (!ss.s) {
    if ((e = cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking))) return e;
    if ((e = cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming))) return e;
    if ((e = cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming))) return e;
    if ((e = cudaEventCreateWithFlags(&ss.pos_ready, cudaEventDisableTiming))) return e;
    if ((e = cudaEventCreateWithFlags(&ss.pos_copied, cudaEventDisableTiming))) return e;
  }
  out = &ss;
  return cudaSuccess;
}

}  // namespace
}  // namespace phb

using namespace phb;

extern "C" phb_status phb_pc_step(const phb_plan* plan, const phb_params* prm, double* pos,
                                  const double* lambda, double* U, double dt, void* ws,
                                  size_t ws_bytes, int32_t* status_word, phb_stream_t stream) {
  const phb_status s = pc_args(plan, prm, pos, lambda, U, dt, ws, ws_bytes);
  if (s != PHB_OK) return s;
  return pc_step_impl(plan, prm, pos, lambda, U, dt, ws, status_word,
                      reinterpret_cast<cudaStream_t>(stream), nullptr);
}

extern "C" phb_status phb_pc_step_host(const phb_plan* plan, const phb_params* prm,
                                       const double* pos_in, const double* lambda_in,
                                       const double* U_in, double* pos_out, double* U_out,
                                       double dt, void* ws, size_t ws_bytes,
                                       int32_t* status_word, phb_stream_t stream) {
  phb_status s = pc_args(plan, prm, pos_in, lambda_in, U_in, dt, ws, ws_bytes);
  if (s != PHB_OK) return s;
  if (!pos_out || !U_out) return PHB_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t n = static_cast<size_t>(plan->n);
  double* dpos = region<double>(plan, ws, R_PC_IO);
  double* dlam = dpos + 3 * n;
  double* dU = dpos + 4 * n;
  SideStream* ss = nullptr;
  cudaError_t e;
  if ((e = side_stream(ss))) return launch_status(e);
  // positions and lambda first: the neighbour build needs only them; the
  // fields follow on the side stream while the build runs
  if ((e = cudaMemcpyAsync(dpos, pos_in, 3 * n * sizeof(double), cudaMemcpyHostToDevice, st)) ||
      (e = cudaMemcpyAsync(dlam, lambda_in, n * sizeof(double), cudaMemcpyHostToDevice, st)) ||
      (e = cudaEventRecord(ss->fork, st)) || (e = cudaStreamWaitEvent(ss->s, ss->fork, 0)) ||
      (e = cudaMemcpyAsync(dU, U_in, 8 * n * sizeof(double), cudaMemcpyHostToDevice, ss->s)) ||
      (e = cudaEventRecord(ss->join, ss->s)))
    return launch_status(e);
  PcOverlap ov;
  ov.wait_U = ss->join;
  ov.side = ss->s;
  ov.pos_ready = ss->pos_ready;
  ov.pos_copied = ss->pos_copied;
  ov.pos_out = pos_out;
  // a page-locked, mapped U_out takes U^{n+1} from the kernels themselves
  // (the corrector's fit for most particles); otherwise one copy after the step
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, U_out) == cudaSuccess) {
    if (pa.type == cudaMemoryTypeHost && pa.devicePointer != nullptr)
      ov.U_host = static_cast<double*>(pa.devicePointer);
  } else {
    cudaGetLastError();  // an unregistered pointer: clear the error, copy instead
  }
  if ((s = pc_step_impl(plan, prm, dpos, dlam, dU, dt, ws, status_word, st, &ov)) != PHB_OK)
    return s;
  if (!(ov.U_host && prm->precision == PHB_FP32_MIXED) &&
      (e = cudaMemcpyAsync(U_out, dU, 8 * n * sizeof(double), cudaMemcpyDeviceToHost, st)))
    return launch_status(e);
  return PHB_OK;
}
