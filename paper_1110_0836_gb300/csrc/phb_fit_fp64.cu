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

template <FitMode MODE>
__global__ void __launch_bounds__(kT) k_fit_fp64(const FitArgs a, int routed, const int32_t* list,
                                                 const int32_t* list_len) {
  extern __shared__ double sm[];
  double* my = sm + threadIdx.x * kStride;
  double(&mom)[kNM] = *reinterpret_cast<double(*)[kNM]>(my);
  double(&M)[kNT] = *reinterpret_cast<double(*)[kNT]>(my + kNM);
  double* bs = my + kNM + kNT;
  const int n = a.n;
  const int total = list ? *list_len : n;
  constexpr int f0 = MODE == FitMode::kRHS ? 1 : 0;  // the RHS never needs the density fit
  // fields fitted, in U order without rho for the RHS
  double len[3], inv_len[3];
  for (int c = 0; c < 3; ++c) {
    len[c] = a.g.len[c];
    inv_len[c] = a.g.periodic[c] ? 1.0 / a.g.len[c] : 0.0;
  }
  for (int w = blockIdx.x * kT + threadIdx.x; w < total; w += gridDim.x * kT) {
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
    for (int64_t e = beg; e < end; ++e) {
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
    bool singular = cnt < kNB;
    bool refine = false;
    double invd[kNB];
    if (!singular) {
      mls_assemble(mom, M);
      const double minpiv = mls_cholesky<double>(M, invd);
      double rmin = 1e300, rmax = 0.0;
#pragma unroll
      for (int k = 0; k < kNB; ++k) {
        const double r = 1.0 / (invd[k] * invd[k] * M[k * (k + 1) / 2 + k]);
        rmin = r < rmin ? r : rmin;
        rmax = r > rmax ? r : rmax;
      }
      // a Jacobi-scaled pivot below 1e-12 (cond(M) above ~1e12) is treated as singular
      singular = !(minpiv > 0.0) || !(rmin > 1e-12);
      // normal equations lose cond(M) * eps: above 1e4 take one corrected
      // semi-normal-equations step (residuals recomputed from the data)
      refine = !singular && rmax > 1e4 * rmin;
    }
    const int dst = a.perm_out ? a.perm_out[s] : s;
    if (a.fit_status) a.fit_status[dst] = singular ? 1 : (routed ? 2 : 0);
    if (singular) raise_flag(a.status_word, PHB_FLAG_FIT_SINGULAR);
    const double il = inv_l, il2 = inv_l * inv_l;
    MhdDerivs<double> D;
    mhd_zero(D);
    for (int f = f0; f < kNF; ++f) {
      double b[kNB];
#pragma unroll
      for (int j = 0; j < kNB; ++j) b[j] = bs[f * kNB + j];
      double g[3] = {0, 0, 0}, h[6] = {0, 0, 0, 0, 0, 0};
      if (!singular) {
        mls_forward(M, invd, b);
        if (!refine) {
          mls_back9(M, invd, b);
        } else {
          mls_back19(M, invd, b);  // b now holds all 19 coefficients c
          double acc[kNB];
#pragma unroll
          for (int k = 0; k < kNB; ++k) acc[k] = 0.0;
          for (int64_t e = beg; e < end; ++e) {
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
            double r = a.sU[f * static_cast<int64_t>(n) + t] - u[f];
#pragma unroll
            for (int k = 0; k < kNB; ++k) r = fma(-qg[k], b[k], r);
            mls_accum_rhs(wq, r, acc);
          }
          mls_forward(M, invd, acc);
          mls_back9(M, invd, acc);
#pragma unroll
          for (int k = kQuad0; k < kNB; ++k) b[k] += acc[k];
        }
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
      const double zeta = a.zeta ? a.zeta[src] : 0.0;
      const double eta = a.eta ? a.eta[src] : 0.0;
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
