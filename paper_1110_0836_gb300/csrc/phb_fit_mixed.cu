// FP32-mixed fused MLS fit + MHD right-hand side (Paper II Sec. 2).
//
// One thread per particle, in cell (slot) order.  Offsets and field
// differences come from FP32 hi/lo splits of the FP64 values, centred on the
// particle (q = d / lambda_i and U_j - U_i), so a 1e-6 perturbation on an O(1)
// background keeps ~7 significant digits.  The 80 distinct moments of the
// normal matrix and the right-hand sides of the fitted fields are accumulated
// in FP32 registers in two passes over the neighbour list (moments + first
// field group, then the second group), the 19x19 normal matrix is factorised
// by an unrolled in-register Cholesky, and only the linear and quadratic
// coefficients are back-substituted.  Fits whose Jacobi-scaled conditioning
// estimate (max L_kk / min L_kk)^2 exceeds the threshold, or whose
// factorisation fails, are pushed to a queue that the FP64 kernel redoes.
#include "phb_internal.cuh"
#include "mls_gen.cuh"
#include "phb_mhd.cuh"

namespace phb {
namespace {

constexpr int kT = 128;

struct Per32 {
  float len_h[3], len_l[3], inv_len[3];
};

__device__ __forceinline__ float hl(float ah, float al, float bh, float bl) {
  return (ah - bh) + (al - bl);
}

// Field groups.  Pass A: (rho), sigma, Vx, Vy.  Pass B: Vz, Bx, By, Bz.
// The RHS never uses the density fit (Drho/Dt needs only rho_i and div V),
// so the RHS mode skips it.
template <FitMode M>
struct Groups {
  static constexpr int NA = M == FitMode::kDerivs ? 4 : 3;
  static constexpr int NF = NA + 4;
  __host__ __device__ static constexpr int field(int k) {
    // slot k of the parked right-hand sides -> field index in U
    return M == FitMode::kDerivs ? (k == 0 ? 0 : k == 1 ? 7 : k == 2 ? 1 : k == 3 ? 2 : k - 1)
                                 : (k == 0 ? 7 : k == 1 ? 1 : k == 2 ? 2 : k);
  }
};

template <FitMode MODE>
__global__ void __launch_bounds__(kT, 1) k_fit_mixed(const FitArgs a, const Per32 P) {
  using G = Groups<MODE>;
  // park[slot][kT]: the fields' right-hand sides (G::NF x 19 slots) followed by
  // the 80 moments; after the solve each field's first 9 slots hold its
  // gradient and packed Hessian.
  extern __shared__ float park[];
  constexpr int kMom0 = G::NF * kNB;
  const int n = a.n;
  const int s = blockIdx.x * kT + threadIdx.x;
  if (s >= n) return;
  const int tid = threadIdx.x;
  const float4* rec = reinterpret_cast<const float4*>(a.rec);
  const float4 o0 = rec[6 * s + 0], o1 = rec[6 * s + 1];
  const double lam = a.slam[s];
  const double rf = a.g.rf_factor * lam;
  const float inv_l = static_cast<float>(1.0 / lam);
  const float inv_rf2 = static_cast<float>(1.0 / (rf * rf));
  const int64_t beg = a.off[s];
  const int64_t end = a.off[s + 1] < a.g.capacity ? a.off[s + 1] : a.g.capacity;
  const bool unweighted = a.weight_kind == 1;

  int cnt = 0;
  {
    const float4 o2 = rec[6 * s + 2], o3 = rec[6 * s + 3];
    float m[kNM];
#pragma unroll
    for (int k = 0; k < kNM; ++k) m[k] = 0.f;
    float bA[G::NA][kNB];
#pragma unroll
    for (int f = 0; f < G::NA; ++f)
#pragma unroll
      for (int k = 0; k < kNB; ++k) bA[f][k] = 0.f;
    for (int64_t e = beg; e < end; ++e) {
      const int t = a.idx[e];
      const float4 p0 = rec[6 * t + 0], p1 = rec[6 * t + 1];
      const float4 fh = rec[6 * t + 2], fl = rec[6 * t + 3];
      const float dx = mi_diff32(p0.x, p1.x, o0.x, o1.x, P.len_h[0], P.len_l[0], P.inv_len[0]);
      const float dy = mi_diff32(p0.y, p1.y, o0.y, o1.y, P.len_h[1], P.len_l[1], P.inv_len[1]);
      const float dz = mi_diff32(p0.z, p1.z, o0.z, o1.z, P.len_h[2], P.len_l[2], P.inv_len[2]);
      const float s2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * inv_rf2;
      const bool inside = s2 < 1.f;
      const float sw = 1.f - s2;
      const float wt = inside ? (unweighted ? 1.f : sw * sw) : 0.f;
      cnt += inside ? 1 : 0;
      float qg[kNB], wq[kNB + 1];
      mls_monomials(dx * inv_l, dy * inv_l, dz * inv_l, wt, qg, wq);
      mls_accum_moments(qg, wq, m);
      if (MODE == FitMode::kDerivs) mls_accum_rhs(wq, hl(fh.x, fl.x, o2.x, o3.x), bA[0]);
      mls_accum_rhs(wq, hl(fh.y, fl.y, o2.y, o3.y), bA[G::NA - 3]);
      mls_accum_rhs(wq, hl(fh.z, fl.z, o2.z, o3.z), bA[G::NA - 2]);
      mls_accum_rhs(wq, hl(fh.w, fl.w, o2.w, o3.w), bA[G::NA - 1]);
    }
#pragma unroll
    for (int f = 0; f < G::NA; ++f)
#pragma unroll
      for (int k = 0; k < kNB; ++k) park[(f * kNB + k) * kT + tid] = bA[f][k];
#pragma unroll
    for (int k = 0; k < kNM; ++k) park[(kMom0 + k) * kT + tid] = m[k];
  }
  {
    const float4 o4 = rec[6 * s + 4], o5 = rec[6 * s + 5];
    float bB[4][kNB];
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int k = 0; k < kNB; ++k) bB[f][k] = 0.f;
    for (int64_t e = beg; e < end; ++e) {
      const int t = a.idx[e];
      const float4 p0 = rec[6 * t + 0], p1 = rec[6 * t + 1];
      const float4 gh = rec[6 * t + 4], gl = rec[6 * t + 5];
      const float dx = mi_diff32(p0.x, p1.x, o0.x, o1.x, P.len_h[0], P.len_l[0], P.inv_len[0]);
      const float dy = mi_diff32(p0.y, p1.y, o0.y, o1.y, P.len_h[1], P.len_l[1], P.inv_len[1]);
      const float dz = mi_diff32(p0.z, p1.z, o0.z, o1.z, P.len_h[2], P.len_l[2], P.inv_len[2]);
      const float s2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * inv_rf2;
      const float sw = 1.f - s2;
      const float wt = s2 < 1.f ? (unweighted ? 1.f : sw * sw) : 0.f;
      float qg[kNB], wq[kNB + 1];
      mls_monomials(dx * inv_l, dy * inv_l, dz * inv_l, wt, qg, wq);
      mls_accum_rhs(wq, hl(gh.x, gl.x, o4.x, o5.x), bB[0]);
      mls_accum_rhs(wq, hl(gh.y, gl.y, o4.y, o5.y), bB[1]);
      mls_accum_rhs(wq, hl(gh.z, gl.z, o4.z, o5.z), bB[2]);
      mls_accum_rhs(wq, hl(gh.w, gl.w, o4.w, o5.w), bB[3]);
    }
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int k = 0; k < kNB; ++k) park[((G::NA + f) * kNB + k) * kT + tid] = bB[f][k];
  }

  const int dst = a.perm_out ? a.perm_out[s] : s;
  const bool singular = cnt < kNB;
  if (!singular) {
    float M[kNT], invd[kNB];
    {
      float m[kNM];
#pragma unroll
      for (int k = 0; k < kNM; ++k) m[k] = park[(kMom0 + k) * kT + tid];
      mls_assemble(m, M);
    }
    const float minpiv = mls_cholesky(M, invd);
    // Jacobi-scaled pivots L~_kk^2 = L_kk^2 / M_kk = 1 / (invd_k^2 M_kk)
    float rmin = 3.4e38f, rmax = 0.f;
#pragma unroll
    for (int k = 0; k < kNB; ++k) {
      const float r = 1.f / (invd[k] * invd[k] * M[k * (k + 1) / 2 + k]);
      rmin = fminf(rmin, r);
      rmax = fmaxf(rmax, r);
    }
    if (!(minpiv > 0.f) || !(rmax <= a.cond_threshold * rmin)) {
      const int q = atomicAdd(a.queue_len, 1);
      a.queue[q] = s;
      return;
    }
    const float il = inv_l, il2 = inv_l * inv_l;
#pragma unroll 1
    for (int k = 0; k < G::NF; ++k) {
      float b[kNB];
#pragma unroll
      for (int j = 0; j < kNB; ++j) b[j] = park[(k * kNB + j) * kT + tid];
      mls_forward(M, invd, b);
      mls_back9(M, invd, b);
      float* d = park + (k * kNB) * kT + tid;
      d[0 * kT] = b[kLin0] * il;
      d[1 * kT] = b[kLin0 + 1] * il;
      d[2 * kT] = b[kLin0 + 2] * il;
      d[3 * kT] = 2.f * b[kQuad0] * il2;
      d[4 * kT] = b[kQuad0 + 1] * il2;
      d[5 * kT] = b[kQuad0 + 2] * il2;
      d[6 * kT] = 2.f * b[kQuad0 + 3] * il2;
      d[7 * kT] = b[kQuad0 + 4] * il2;
      d[8 * kT] = 2.f * b[kQuad0 + 5] * il2;
    }
  } else {
#pragma unroll 1
    for (int k = 0; k < G::NF; ++k)
      for (int j = 0; j < 9; ++j) park[(k * kNB + j) * kT + tid] = 0.f;
  }
  if (a.fit_status) a.fit_status[dst] = singular ? 1 : 0;
  if (singular) raise_flag(a.status_word, PHB_FLAG_FIT_SINGULAR);
  if (MODE == FitMode::kDerivs) {
#pragma unroll 1
    for (int k = 0; k < G::NF; ++k) {
      const int f = G::field(k);
      const float* d = park + (k * kNB) * kT + tid;
      for (int c = 0; c < 3; ++c) a.grad[(f * 3 + c) * static_cast<int64_t>(n) + dst] = d[c * kT];
      if (a.hess)
        for (int c = 0; c < 6; ++c)
          a.hess[(f * 6 + c) * static_cast<int64_t>(n) + dst] = d[(3 + c) * kT];
    }
  } else {
    MhdDerivs<float> D;
    mhd_zero(D);
#pragma unroll
    for (int k = 0; k < G::NF; ++k) {
      const float* d = park + (k * kNB) * kT + tid;
      const float g[3] = {d[0], d[kT], d[2 * kT]};
      const float h[6] = {d[3 * kT], d[4 * kT], d[5 * kT], d[6 * kT], d[7 * kT], d[8 * kT]};
      mhd_collect(D, G::field(k), g, h);
    }
    const float4 o2 = rec[6 * s + 2], o3 = rec[6 * s + 3], o4 = rec[6 * s + 4], o5 = rec[6 * s + 5];
    const float u[8] = {o2.x + o3.x, o2.z + o3.z, o2.w + o3.w, o4.x + o5.x,
                        o4.y + o5.y, o4.z + o5.z, o4.w + o5.w, o2.y + o3.y};
    const int src = a.perm_in ? a.perm_in[s] : s;
    const float zeta = a.zeta ? static_cast<float>(a.zeta[src]) : 0.f;
    const float eta = a.eta ? static_cast<float>(a.eta[src]) : 0.f;
    float out[8];
    mhd_rhs(u, D, static_cast<float>(a.gamma), zeta, eta, out);
    bool finite = true;
#pragma unroll
    for (int f = 0; f < 8; ++f) {
      finite &= isfinite(out[f]);
      a.dudt[f * static_cast<int64_t>(n) + dst] = out[f];
    }
    if (!finite) raise_flag(a.status_word, PHB_FLAG_NONFINITE);
  }
}

Per32 make_per32(const Grid& g) {
  Per32 P;
  for (int a = 0; a < 3; ++a) {
    const float h = static_cast<float>(g.len[a]);
    P.len_h[a] = g.periodic[a] ? h : 0.f;
    P.len_l[a] = g.periodic[a] ? static_cast<float>(g.len[a] - static_cast<double>(h)) : 0.f;
    P.inv_len[a] = g.periodic[a] ? static_cast<float>(1.0 / g.len[a]) : 0.f;
  }
  return P;
}

}  // namespace

cudaError_t launch_fit_mixed(const FitArgs& a, FitMode mode, cudaStream_t st) {
  const Per32 P = make_per32(a.g);
  const unsigned blocks = static_cast<unsigned>((a.n + kT - 1) / kT);
  if (mode == FitMode::kDerivs) {
    const size_t smem = size_t(Groups<FitMode::kDerivs>::NF * kNB + kNM) * kT * sizeof(float);
    cudaFuncSetAttribute(k_fit_mixed<FitMode::kDerivs>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    const int tr = trace_begin(1, st);
    k_fit_mixed<FitMode::kDerivs><<<blocks, kT, smem, st>>>(a, P);
    note_launch();
    trace_end(tr, st);
  } else {
    const size_t smem = size_t(Groups<FitMode::kRHS>::NF * kNB + kNM) * kT * sizeof(float);
    cudaFuncSetAttribute(k_fit_mixed<FitMode::kRHS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    const int tr = trace_begin(1, st);
    k_fit_mixed<FitMode::kRHS><<<blocks, kT, smem, st>>>(a, P);
    note_launch();
    trace_end(tr, st);
  }
  return cudaGetLastError();
}

}  // namespace phb
