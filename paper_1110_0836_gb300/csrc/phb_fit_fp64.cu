// FP64 fused MLS fit + MHD right-hand side (Paper II Sec. 2), the plain
// double-precision GPU form.  It serves every particle when the precision is
// PHB_FP64, and the particles that the FP32-mixed kernel routed to FP64.
//
// One thread per particle.  The 80 moments and 8 x 19 right-hand sides are
// accumulated in a thread-private shared-memory region (FP64 registers would
// not hold them), the normal matrix is assembled and factorised in place by
// the same unrolled Cholesky as the mixed kernel, and only the linear and
// quadratic coefficients are back-substituted.  Fits whose Jacobi-scaled
// conditioning estimate exceeds 1e4 take one corrected semi-normal-equations
// step (Bjorck): residuals r_j = (U_j - U_i) - p(q_j).c are recomputed from the
// data, A^T W r is accumulated again and solved with the same factor, so the
// error follows cond(A) rather than cond(A^T W A) = cond(A)^2.
#include "phb_internal.cuh"
#include "mls_gen.cuh"
#include "phb_mhd.cuh"

namespace phb {
namespace {

constexpr int kT = 64;
constexpr int kStride = kNM + kNT + kNF * kNB + 1;  // doubles per thread; odd stride avoids bank conflicts
static_assert(4 * kNB <= kNM, "the refinement accumulates four fields in the moments' region");

// Route queues (fits the FP32-mixed kernel handed over) up to this length
// are fitted by a warp per particle (neighbours split over the lanes, partial
// sums reduced in shared memory, the solve on lane 0): a handful of routed
// fits then takes tens of microseconds instead of one thread's serial FP64
// work.  Longer queues and the full FP64 path use one thread per particle
// (throughput).
constexpr int kWarpQueueMax = 4096;

template <FitMode MODE>
__global__ void __launch_bounds__(kT, 1) k_fit_fp64(const FitArgs a, int routed, const int32_t* list,
                                                 const int32_t* list_len) {
  extern __shared__ double sm[];
  const int n = a.n;
  const int total = list ? *list_len : n;
  // uniform over the launch; an active subset in FP64 keeps one thread per
  // particle so that its results are bit-identical to the full evaluation
  const int lanes = (routed && list && total <= kWarpQueueMax) ? 32 : 1;
  // fits routed from the FP32-mixed path need ~1e-5: FP64 normal equations
  // meet that up to cond(M) ~ 1e9; the FP64 path itself targets ~1e-12
  const double refine_above = routed ? 1e9 : 1e4;
  const int lane = threadIdx.x % lanes;
  const int groups = kT / lanes;
  const int grp = threadIdx.x / lanes;
  // a block without work (an empty or short routed queue) leaves before any
  // FP64 set-up
  if (static_cast<int64_t>(blockIdx.x) * groups >= total) return;
  double* my = sm + threadIdx.x * kStride;
  double* head = sm + grp * lanes * kStride;  // the group's lane 0 region: totals, factor, c
  double(&mom)[kNM] = *reinterpret_cast<double(*)[kNM]>(my);
  double(&M)[kNT] = *reinterpret_cast<double(*)[kNT]>(head + kNM);
  double* bs = my + kNM + kNT;
  double* hmom = head;
  double* hbs = head + kNM + kNT;
  constexpr int f0 = MODE == FitMode::kRHS ? 1 : 0;  // the RHS never needs the density fit
  // fields fitted, in U order without rho for the RHS
  double len[3], inv_len[3];
  for (int c = 0; c < 3; ++c) {
    len[c] = a.g.len[c];
    inv_len[c] = a.g.periodic[c] ? 1.0 / a.g.len[c] : 0.0;
  }
  // sum the lanes' partial accumulators [0, count) of the regions starting at
  // `at` into the group's lane 0 region (no-op for one lane per particle)
  auto reduce = [&](int at, int count) {
    if (lanes == 1) return;
    __syncwarp();
    for (int k = lane; k < count; k += lanes) {
      double t = 0.0;
      for (int l = 0; l < lanes; ++l) t += head[l * kStride + at + k];
      head[at + k] = t;
    }
    __syncwarp();
  };
  for (int w = blockIdx.x * groups + grp; w < total; w += gridDim.x * groups) {
    const int s = list ? list[w] : w;
    const double xs = a.spos[s], ys = a.spos[n + s], zs = a.spos[2 * n + s];
    double u[8];
#pragma unroll
    for (int f = 0; f < 8; ++f) u[f] = a.sU[f * static_cast<int64_t>(n) + s];
    const double lam = a.slam[s];
    const double rf = a.g.rf_factor * lam;
    const double inv_rf2 = 1.0 / (rf * rf);
    const double inv_l = 1.0 / lam;
    const int64_t beg = a.off[s];
    const int64_t end = a.off[s + 1] < a.g.capacity ? a.off[s + 1] : a.g.capacity;
    for (int k = 0; k < kNM; ++k) mom[k] = 0.0;
    for (int k = 0; k < kNF * kNB; ++k) bs[k] = 0.0;
    int cnt = 0;
    for (int64_t e = beg + lane; e < end; e += lanes) {
      const int t = a.idx[e];
      double dx = a.spos[t] - xs, dy = a.spos[n + t] - ys, dz = a.spos[2 * n + t] - zs;
      dx -= len[0] * rint(dx * inv_len[0]);
      dy -= len[1] * rint(dy * inv_len[1]);
      dz -= len[2] * rint(dz * inv_len[2]);
      const double s2 = (dx * dx + dy * dy + dz * dz) * inv_rf2;
      const bool inside = s2 < 1.0;
      if (!inside) continue;
      ++cnt;
      const double sw = 1.0 - s2;
      const double wt = a.weight_kind == 1 ? 1.0 : sw * sw;
      double qg[kNB], wq[kNB + 1];
      mls_monomials(dx * inv_l, dy * inv_l, dz * inv_l, wt, qg, wq);
      mls_accum_moments(qg, wq, mom);
#pragma unroll
      for (int f = f0; f < kNF; ++f) {
        const double du = a.sU[f * static_cast<int64_t>(n) + t] - u[f];
        mls_accum_rhs(wq, du, *reinterpret_cast<double(*)[kNB]>(bs + f * kNB));
      }
    }
    if (lanes > 1) cnt = __reduce_add_sync(0xffffffffu, cnt);
    reduce(0, kNM);                      // moments
    reduce(kNM + kNT, kNF * kNB);        // right-hand sides
    bool singular = cnt < kNB;
    bool refine = false;
    double invd[kNB];
    if (lane == 0 && !singular) {
      mls_assemble(*reinterpret_cast<double(*)[kNM]>(hmom), M);
      const double minpiv = mls_cholesky<double>(M, invd);
      double rmin = 1e300;
#pragma unroll
      for (int k = 0; k < kNB; ++k) {
        const double r = 1.0 / (invd[k] * invd[k] * M[k * (k + 1) / 2 + k]);
        rmin = r < rmin ? r : rmin;
      }
      // a Jacobi-scaled pivot below 1e-12 (cond(M) above ~1e12) is treated as singular
      singular = !(minpiv > 0.0) || !(rmin > 1e-12);
      // normal equations lose cond(M) * eps: above an estimate of refine_above
      // (n_b times the greedy ||M_s^-1||_inf estimate) take one corrected
      // semi-normal-equations step (residuals recomputed from the data)
      refine = !singular && kNB * mls_inv_norm_est<double>(M, invd) > refine_above;
      if (lanes > 1)
        for (int k = 0; k < kNB; ++k) head[kStride + k] = invd[k];  // lane 1's region is free here
    }
    if (lanes > 1) {
      singular = __shfl_sync(0xffffffffu, singular, 0);
      refine = __shfl_sync(0xffffffffu, refine, 0);
      __syncwarp();
      if (lane > 0 && lane < kNF - f0 && !singular)
        for (int k = 0; k < kNB; ++k) invd[k] = head[kStride + k];
      __syncwarp();
    }
    // coefficients of every field: the linear and quadratic ones, or all 19
    // when the fit is refined; kept in the right-hand-side region.  One lane
    // per field with a warp per particle, all fields in turn otherwise.
    const int fstep = lanes > 1 ? kNF : 1;
    if (!singular) {
      for (int f = f0 + (lanes > 1 ? lane : 0); f < kNF; f += fstep) {
        double b[kNB];
#pragma unroll
        for (int j = 0; j < kNB; ++j) b[j] = hbs[f * kNB + j];
        mls_forward(M, invd, b);
        if (refine) mls_back19(M, invd, b);
        else mls_back9(M, invd, b);
#pragma unroll
        for (int j = 0; j < kNB; ++j) hbs[f * kNB + j] = b[j];
      }
    }
    if (lanes > 1) __syncwarp();
    const int dst = a.perm_out ? a.perm_out[s] : s;
    if (refine) {
      // corrected semi-normal equations: one pass over the neighbours per
      // group of up to four fields accumulates A^T W r with the residuals
      // r = (U_j - U_i) - p(q_j).c recomputed from the data; the moments'
      // region (dead after the assembly) holds the four accumulators
      for (int g0 = f0; g0 < kNF; g0 += 4) {
        const int g1 = g0 + 4 < kNF ? g0 + 4 : kNF;
        for (int k = 0; k < 4 * kNB; ++k) mom[k] = 0.0;
        for (int64_t e = beg + lane; e < end; e += lanes) {
          const int t = a.idx[e];
          double dx = a.spos[t] - xs, dy = a.spos[n + t] - ys, dz = a.spos[2 * n + t] - zs;
          dx -= len[0] * rint(dx * inv_len[0]);
          dy -= len[1] * rint(dy * inv_len[1]);
          dz -= len[2] * rint(dz * inv_len[2]);
          const double s2 = (dx * dx + dy * dy + dz * dz) * inv_rf2;
          if (!(s2 < 1.0)) continue;
          const double sw = 1.0 - s2;
          const double wt = a.weight_kind == 1 ? 1.0 : sw * sw;
          double qg[kNB], wq[kNB + 1];
          mls_monomials(dx * inv_l, dy * inv_l, dz * inv_l, wt, qg, wq);
          for (int f = g0; f < g1; ++f) {
            double r = a.sU[f * static_cast<int64_t>(n) + t] - u[f];
#pragma unroll
            for (int k = 0; k < kNB; ++k) r = fma(-qg[k], hbs[f * kNB + k], r);
            mls_accum_rhs(wq, r, *reinterpret_cast<double(*)[kNB]>(mom + (f - g0) * kNB));
          }
        }
        reduce(0, 4 * kNB);
        for (int f = g0 + (lanes > 1 ? lane : 0); f < g1; f += fstep) {
          double acc[kNB];
#pragma unroll
          for (int k = 0; k < kNB; ++k) acc[k] = hmom[(f - g0) * kNB + k];
          mls_forward(M, invd, acc);
          mls_back9(M, invd, acc);
#pragma unroll
          for (int k = kQuad0; k < kNB; ++k) hbs[f * kNB + k] += acc[k];
        }
        if (lanes > 1) __syncwarp();
      }
    }
    if (lane == 0) {
      if (a.fit_status) a.fit_status[dst] = singular ? 1 : (routed ? 2 : 0);
      if (singular) raise_flag(a.status_word, PHB_FLAG_FIT_SINGULAR);
      const double il = inv_l, il2 = inv_l * inv_l;
      MhdDerivs<double> D;
      mhd_zero(D);
      for (int f = f0; f < kNF; ++f) {
        double g[3] = {0, 0, 0}, h[6] = {0, 0, 0, 0, 0, 0};
        if (!singular) {
          const double* b = hbs + f * kNB;
          g[0] = b[kLin0] * il; g[1] = b[kLin0 + 1] * il; g[2] = b[kLin0 + 2] * il;
          h[0] = 2.0 * b[kQuad0] * il2; h[1] = b[kQuad0 + 1] * il2; h[2] = b[kQuad0 + 2] * il2;
          h[3] = 2.0 * b[kQuad0 + 3] * il2; h[4] = b[kQuad0 + 4] * il2; h[5] = 2.0 * b[kQuad0 + 5] * il2;
        }
        if (MODE == FitMode::kDerivs) {
          for (int c = 0; c < 3; ++c) a.grad[(f * 3 + c) * static_cast<int64_t>(n) + dst] = g[c];
          if (a.hess)
            for (int c = 0; c < 6; ++c) a.hess[(f * 6 + c) * static_cast<int64_t>(n) + dst] = h[c];
        } else {
          mhd_collect(D, f, g, h);
        }
      }
      if (MODE == FitMode::kRHS) {
        const int src = a.perm_in ? a.perm_in[s] : s;
        double zeta = a.zeta ? a.zeta[src] : 0.0;
        double eta = a.eta ? a.eta[src] : 0.0;
        if (a.c_zeta_l != 0.0 || a.c_zeta_a != 0.0 || a.c_eta != 0.0)
          mhd_laws(u, D, a.gamma, lam, a.c_zeta_l, a.c_zeta_a, a.c_eta, zeta, eta);
        double out[8];
        mhd_rhs(u, D, a.gamma, zeta, eta, out);
        bool finite = true;
        for (int f = 0; f < 8; ++f) {
          finite &= isfinite(out[f]);
          a.dudt[f * static_cast<int64_t>(n) + dst] = out[f];
        }
        if (!finite) raise_flag(a.status_word, PHB_FLAG_NONFINITE);
      }
    }
    if (lanes > 1) __syncwarp();  // the group's regions are reused by the next particle
  }
}

}  // namespace

cudaError_t launch_fit_fp64(const FitArgs& a, FitMode mode, const int32_t* list,
                            const int32_t* list_len, cudaStream_t st, bool routed) {
  const size_t smem = size_t(kStride) * kT * sizeof(double);
  unsigned blocks = list ? static_cast<unsigned>(num_sms() * 2)
                         : static_cast<unsigned>((a.n + kT - 1) / kT);
  if (mode == FitMode::kDerivs) {
    cudaFuncSetAttribute(k_fit_fp64<FitMode::kDerivs>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    const int tr = trace_begin(list ? 3 : 2, st);
    k_fit_fp64<FitMode::kDerivs><<<blocks, kT, smem, st>>>(a, routed, list, list_len);
    note_launch();
    trace_end(tr, st);
  } else {
    cudaFuncSetAttribute(k_fit_fp64<FitMode::kRHS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    const int tr = trace_begin(list ? 3 : 2, st);
    k_fit_fp64<FitMode::kRHS><<<blocks, kT, smem, st>>>(a, routed, list, list_len);
    note_launch();
    trace_end(tr, st);
  }
  return cudaGetLastError();
}

}  // namespace phb
