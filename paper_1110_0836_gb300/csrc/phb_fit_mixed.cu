// FP32-mixed fused MLS fit + MHD right-hand side (Paper II Sec. 2).
//
// One CTA per tile of consecutive particles (cell order), one thread per
// particle.  The tile's neighbourhood is staged in shared memory as 48-byte
// records: position and the 8 fields relative to the tile's middle particle,
// computed from FP32 hi/lo splits of the FP64 values (offsets with minimum
// image), so differences between neighbours keep ~7 significant digits even
// for a 1e-6 perturbation on an O(1) background.  Each thread accumulates the
// 80 distinct moments of the normal matrix and the right-hand sides of the
// fitted fields in FP32 registers in two passes over its neighbour list
// (moments + first field group, then the second group), factorises the
// 19x19 normal matrix by an unrolled in-register Cholesky and back-substitutes
// only the linear and quadratic coefficients.  Fits whose conditioning
// estimate (19 x a greedy estimate of ||M_s^-1||_inf of the Jacobi-scaled
// matrix M_s) exceeds the routing threshold, or whose factorisation fails,
// are queued for the FP64 kernel.  Tiles whose neighbourhood exceeds the
// staging capacity read neighbours from global memory (FP32 hi/lo records)
// through the same code.
//
// Corrected semi-normal equations (Bjorck).  FP32 normal equations lose about
// cond(M_s) x 2^-24 of the coefficient vector, and on density-sampled sets the
// odd and even blocks of M_s couple, so the large linear coefficients of a
// steep front leak into the quadratic ones (Hessian errors of 4e-4 of their
// scale at the shear layer).  A tile whose largest estimate exceeds
// refine_kappa (or every tile, by choice) therefore takes one corrected step
// after the first solve: with all 19 coefficients c0 of every field, one more
// pass over the neighbours accumulates P^T W r with the residuals
// r_j = (U_j - U_i) - p(q_j).c0 recomputed from the records, and the same
// factor (re-formed from the kept moments) solves for the correction.  The
// error then follows cond(A) = cond(M_s)^(1/2) instead of cond(M_s).  The
// decision is per tile (a per-fit rule leaves fits above the bar).  Where the
// set's FP32 records fit in L2, a refined tile queues its fits with their
// moments and c0 for k_fit_refine, which streams through the queue without
// the tile's barriers; larger sets take the step inside the tile, while its
// neighbourhood is still in L2.
#include "phb_internal.cuh"
#include "mls_gen.cuh"
#include "phb_mhd.cuh"

namespace phb {
namespace {

struct Per32 {
  float len_h[3], len_l[3], inv_len[3], len[3];
};

__device__ __forceinline__ float hl(float ah, float al, float bh, float bl) {
  return (ah - bh) + (al - bl);
}

// Column k (0..18) of paired accumulators (basis indices 2j, 2j+1 in pair j).
__device__ __forceinline__ float pair_at(const float2 (&v)[kNB2], int k) {
  return (k & 1) ? v[k >> 1].y : v[k >> 1].x;
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

// Neighbour data from the FP32 hi/lo records in global memory.
// du (pass A) = (rho, sigma, Vx, Vy) differences; (pass B) = (Vz, Bx, By, Bz).
// fetch_* issues a neighbour's loads, decode_* turns them into offsets and
// field differences, so that the loop can fetch one neighbour ahead.
struct GlobalSrc {
  static constexpr bool kPrefetch = true;  // accumulate: records loaded a neighbour ahead
  const float4* rec;
  const int32_t* idx;
  float4 o[6];
  Per32 P;
  struct Raw {
    float4 p0, p1, h, l;
  };
  using RawA = Raw;
  using RawB = Raw;
  __device__ __forceinline__ int index(int64_t e) const { return idx[e]; }
  __device__ __forceinline__ Raw fetch_a(int t) const {
    return Raw{rec[6 * t], rec[6 * t + 1], rec[6 * t + 2], rec[6 * t + 3]};
  }
  __device__ __forceinline__ Raw fetch_b(int t) const {
    return Raw{rec[6 * t], rec[6 * t + 1], rec[6 * t + 4], rec[6 * t + 5]};
  }
  __device__ __forceinline__ void offs(const Raw& r, float& dx, float& dy, float& dz) const {
    dx = mi_diff32(r.p0.x, r.p1.x, o[0].x, o[1].x, P.len_h[0], P.len_l[0], P.inv_len[0]);
    dy = mi_diff32(r.p0.y, r.p1.y, o[0].y, o[1].y, P.len_h[1], P.len_l[1], P.inv_len[1]);
    dz = mi_diff32(r.p0.z, r.p1.z, o[0].z, o[1].z, P.len_h[2], P.len_l[2], P.inv_len[2]);
  }
  __device__ __forceinline__ void decode_a(const Raw& r, float& dx, float& dy, float& dz,
                                           float (&du)[4]) const {
    offs(r, dx, dy, dz);
    du[0] = hl(r.h.x, r.l.x, o[2].x, o[3].x);
    du[1] = hl(r.h.y, r.l.y, o[2].y, o[3].y);
    du[2] = hl(r.h.z, r.l.z, o[2].z, o[3].z);
    du[3] = hl(r.h.w, r.l.w, o[2].w, o[3].w);
  }
  __device__ __forceinline__ void decode_b(const Raw& r, float& dx, float& dy, float& dz,
                                           float (&du)[4]) const {
    offs(r, dx, dy, dz);
    du[0] = hl(r.h.x, r.l.x, o[4].x, o[5].x);
    du[1] = hl(r.h.y, r.l.y, o[4].y, o[5].y);
    du[2] = hl(r.h.z, r.l.z, o[4].z, o[5].z);
    du[3] = hl(r.h.w, r.l.w, o[4].w, o[5].w);
  }
};

// Neighbour data from the staged records in shared memory:
// r0 = (x, y, z, sigma), r1 = (Vx, Vy, Vz, rho), r2 = (Bx, By, Bz, 0).
// Wrap = false for a tile whose staged offsets all lie within a quarter box
// length of its middle particle on every periodic axis: differences of two
// such offsets are minimum images already.
template <bool Wrap>
struct StagedSrc {
  static constexpr bool kPrefetch = false;
  const float4* stage;
  const uint16_t* lidx;
  float4 me0, me1, me2;
  float len[3], inv_len[3];
  struct RawA {
    float4 r0, r1;
  };
  struct RawB {
    float4 r0, r1, r2;
  };
  __device__ __forceinline__ void offs(float4 r0, float& dx, float& dy, float& dz) const {
    // relative offsets are minimum images of size <= len/2; one more wrap
    // keeps the difference a minimum image too (exact when no wrap occurs)
    const float ax = r0.x - me0.x, ay = r0.y - me0.y, az = r0.z - me0.z;
    if (Wrap) {
      dx = fmaf(-len[0], rintf(ax * inv_len[0]), ax);
      dy = fmaf(-len[1], rintf(ay * inv_len[1]), ay);
      dz = fmaf(-len[2], rintf(az * inv_len[2]), az);
    } else {
      dx = ax;
      dy = ay;
      dz = az;
    }
  }
  __device__ __forceinline__ int index(int64_t e) const { return lidx[e]; }
  __device__ __forceinline__ RawA fetch_a(int l) const { return RawA{stage[3 * l], stage[3 * l + 1]}; }
  __device__ __forceinline__ RawB fetch_b(int l) const {
    return RawB{stage[3 * l], stage[3 * l + 1], stage[3 * l + 2]};
  }
  __device__ __forceinline__ void decode_a(const RawA& r, float& dx, float& dy, float& dz,
                                           float (&du)[4]) const {
    offs(r.r0, dx, dy, dz);
    du[0] = r.r1.w - me1.w;
    du[1] = r.r0.w - me0.w;
    du[2] = r.r1.x - me1.x;
    du[3] = r.r1.y - me1.y;
  }
  __device__ __forceinline__ void decode_b(const RawB& r, float& dx, float& dy, float& dz,
                                           float (&du)[4]) const {
    offs(r.r0, dx, dy, dz);
    du[0] = r.r1.z - me1.z;
    du[1] = r.r2.x - me2.x;
    du[2] = r.r2.y - me2.y;
    du[3] = r.r2.z - me2.z;
  }
};

// Both accumulation passes of one particle.  Pass A's right-hand sides are
// parked in shared memory column `col` ([slot][T] layout); the moments and
// pass B's right-hand sides are returned in registers.  List indices are
// loaded four neighbours ahead (fetching the neighbours' data ahead as well
// measured slower: the extra registers cost more than the hidden
// shared-memory latency).  Both passes fold the weight into the field
// difference for the right-hand sides, so only the eight weighted basis
// pairs the moments need are formed (the moments, in the packed pair layout,
// are complete after pass A).
template <FitMode MODE, int T, class Src>
__device__ __forceinline__ int accumulate(const Src& src, int64_t beg, int64_t end, float inv_l,
                                          float inv_rf2, bool unweighted, float* park, int col,
                                          float2 (&m2)[kNM2], float2 (&bB)[4][kNB2]) {
  using G = Groups<MODE>;
  int cnt = 0;
#pragma unroll
  for (int k = 0; k < kNM2; ++k) m2[k] = make_float2(0.f, 0.f);
  {
    float2 bA[G::NA][kNB2];
#pragma unroll
    for (int f = 0; f < G::NA; ++f)
#pragma unroll
      for (int j = 0; j < kNB2; ++j) bA[f][j] = make_float2(0.f, 0.f);
    int n1 = beg < end ? src.index(beg) : 0;
    int n2 = beg + 1 < end ? src.index(beg + 1) : 0;
    int n3 = beg + 2 < end ? src.index(beg + 2) : 0;
    int n4 = beg + 3 < end ? src.index(beg + 3) : 0;
    typename Src::RawA ra;
    if (Src::kPrefetch && beg < end) {
      ra = src.fetch_a(n1);
      n1 = n2; n2 = n3; n3 = n4;
      if (beg + 4 < end) n4 = src.index(beg + 4);
    }
    for (int64_t e = beg; e < end; ++e) {
      typename Src::RawA cur;
      if constexpr (Src::kPrefetch) {
        cur = ra;
        if (e + 1 < end) ra = src.fetch_a(n1);
      } else {
        cur = src.fetch_a(n1);
      }
      n1 = n2; n2 = n3; n3 = n4;
      if (e + (Src::kPrefetch ? 5 : 4) < end) n4 = src.index(e + (Src::kPrefetch ? 5 : 4));
      float dx, dy, dz, du[4];
      src.decode_a(cur, dx, dy, dz, du);
      const float s2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * inv_rf2;
      const bool inside = s2 < 1.f;
      const float sw = 1.f - s2;
      const float wt = inside ? (unweighted ? 1.f : sw * sw) : 0.f;
      cnt += inside ? 1 : 0;
      float2 qg2[kNB2], wp[kNWP];
      mls_basis2(dx * inv_l, dy * inv_l, dz * inv_l, qg2);
      mls_weight_pairs(qg2, wt, wp);
      mls_accum_moments_p2(qg2, wp, m2);
      if (MODE == FitMode::kDerivs) mls_accum_rhs_basis2(qg2, wt * du[0], bA[0]);
      mls_accum_rhs_basis2(qg2, wt * du[1], bA[G::NA - 3]);
      mls_accum_rhs_basis2(qg2, wt * du[2], bA[G::NA - 2]);
      mls_accum_rhs_basis2(qg2, wt * du[3], bA[G::NA - 1]);
    }
#pragma unroll
    for (int f = 0; f < G::NA; ++f)
#pragma unroll
      for (int k = 0; k < kNB; ++k) park[(f * kNB + k) * T + col] = pair_at(bA[f], k);
  }
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int j = 0; j < kNB2; ++j) bB[f][j] = make_float2(0.f, 0.f);
  int n1 = beg < end ? src.index(beg) : 0;
  int n2 = beg + 1 < end ? src.index(beg + 1) : 0;
  int n3 = beg + 2 < end ? src.index(beg + 2) : 0;
  int n4 = beg + 3 < end ? src.index(beg + 3) : 0;
  typename Src::RawB rb;
  if (Src::kPrefetch && beg < end) {
    rb = src.fetch_b(n1);
    n1 = n2; n2 = n3; n3 = n4;
    if (beg + 4 < end) n4 = src.index(beg + 4);
  }
  for (int64_t e = beg; e < end; ++e) {
    typename Src::RawB cur;
    if constexpr (Src::kPrefetch) {
      cur = rb;
      if (e + 1 < end) rb = src.fetch_b(n1);
    } else {
      cur = src.fetch_b(n1);
    }
    n1 = n2; n2 = n3; n3 = n4;
    if (e + (Src::kPrefetch ? 5 : 4) < end) n4 = src.index(e + (Src::kPrefetch ? 5 : 4));
    float dx, dy, dz, du[4];
    src.decode_b(cur, dx, dy, dz, du);
    const float s2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * inv_rf2;
    const float sw = 1.f - s2;
    const float wt = s2 < 1.f ? (unweighted ? 1.f : sw * sw) : 0.f;
    float2 qg2[kNB2];
    mls_basis2(dx * inv_l, dy * inv_l, dz * inv_l, qg2);
#pragma unroll
    for (int f = 0; f < 4; ++f) mls_accum_rhs_basis2(qg2, wt * du[f], bB[f]);
  }
  return cnt;
}

// One corrected semi-normal-equations pass for the fields of slots
// [k0, k0 + NFG): c0 (all 19 coefficients of each, from the fit's column cg
// of the stash, stride cs) in registers, residuals r_j = du_j - p(q_j).c0
// recomputed from the global records (RawA = RawB there),
// acc_k = sum_j w_j p(q_j) r_j.  B selects the record half (false: rho,
// sigma, Vx, Vy; true: Vz, Bx, By, Bz); du0 is the first du component used.
template <int NFG, bool B, class Src>
__device__ __forceinline__ void csne_pass(const Src& src, int64_t beg, int64_t end, float inv_l,
                                          float inv_rf2, bool unweighted, const float* cg,
                                          int64_t cs, int k0, int du0, float2 (&acc)[NFG][kNB2]) {
  float2 c[NFG][kNB2];
#pragma unroll
  for (int f = 0; f < NFG; ++f)
#pragma unroll
    for (int j = 0; j < kNB2; ++j) {
      const float lo = cg[((k0 + f) * kNB + 2 * j) * cs];
      const float hi = 2 * j + 1 < kNB ? cg[((k0 + f) * kNB + 2 * j + 1) * cs] : 0.f;
      c[f][j] = make_float2(lo, hi);
      acc[f][j] = make_float2(0.f, 0.f);
    }
  // the next neighbour's record is loaded while this one is used, from an
  // index loaded two neighbours before that (so that the record's load does
  // not wait on its index's)
  typename Src::RawB nxt;
  int i2 = beg + 1 < end ? src.index(beg + 1) : 0;
  int i3 = beg + 2 < end ? src.index(beg + 2) : 0;
  if (beg < end) nxt = B ? src.fetch_b(src.index(beg)) : src.fetch_a(src.index(beg));
  for (int64_t e = beg; e < end; ++e) {
    const typename Src::RawB cur = nxt;
    if (e + 1 < end) nxt = B ? src.fetch_b(i2) : src.fetch_a(i2);
    i2 = i3;
    if (e + 3 < end) i3 = src.index(e + 3);
    float dx, dy, dz, du[4];
    if (B) src.decode_b(cur, dx, dy, dz, du);
    else src.decode_a(cur, dx, dy, dz, du);
    const float s2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * inv_rf2;
    const float sw = 1.f - s2;
    const float wt = s2 < 1.f ? (unweighted ? 1.f : sw * sw) : 0.f;
    float2 qg2[kNB2];
    mls_basis2(dx * inv_l, dy * inv_l, dz * inv_l, qg2);
#pragma unroll
    for (int f = 0; f < NFG; ++f) {
      const float r = du[du0 + f] - mls_dot2(qg2, c[f]);
      mls_accum_rhs_basis2(qg2, wt * r, acc[f]);
    }
  }
}


// Linear and quadratic coefficients b[10..18] -> derivatives in the first
// nine rows of the parked column (gradient, then the packed Hessian).
template <int T>
__device__ __forceinline__ void park_derivs(float* d, const float (&b)[kNB], float il, float il2) {
  d[0 * T] = b[kLin0] * il;
  d[1 * T] = b[kLin0 + 1] * il;
  d[2 * T] = b[kLin0 + 2] * il;
  d[3 * T] = 2.f * b[kQuad0] * il2;
  d[4 * T] = b[kQuad0 + 1] * il2;
  d[5 * T] = b[kQuad0 + 2] * il2;
  d[6 * T] = 2.f * b[kQuad0 + 3] * il2;
  d[7 * T] = b[kQuad0 + 4] * il2;
  d[8 * T] = 2.f * b[kQuad0 + 5] * il2;
}

// Solves of NF fields with one factor: with Pair two fields at a time (packed
// FMAs with the factor's entries broadcast; the last one alone when NF is
// odd), else one at a time.  load(k, j) gives row j of field k's right-hand
// side; use(k, b) takes its solution, all 19 coefficients (Full) or the
// linear and quadratic ones.  (The full solves stay one field at a time: a
// pair keeps the whole factor and 38 right-hand sides live and spills.)
template <int NF, bool Full, bool Pair, class Load, class Use>
__device__ __forceinline__ void solve_fields(const float (&M)[kNT], const float (&invd)[kNB], Load load,
                                             Use use) {
  constexpr int NP = Pair ? NF / 2 : 0;
#pragma unroll 1
  for (int k = 0; k < 2 * NP; k += 2) {
    float2 b2[kNB];
#pragma unroll
    for (int j = 0; j < kNB; ++j) b2[j] = make_float2(load(k, j), load(k + 1, j));
    mls_forward2(M, invd, b2);
    if constexpr (Full) {
      mls_back19_2(M, invd, b2);
    } else {
      mls_back9_2(M, invd, b2);
    }
    float b0[kNB], b1[kNB];
#pragma unroll
    for (int j = 0; j < kNB; ++j) {
      b0[j] = b2[j].x;
      b1[j] = b2[j].y;
    }
    use(k, b0);
    use(k + 1, b1);
  }
#pragma unroll 1
  for (int k = 2 * NP; k < NF; ++k) {
    float b[kNB];
#pragma unroll
    for (int j = 0; j < kNB; ++j) b[j] = load(k, j);
    mls_forward(M, invd, b);
    if constexpr (Full) {
      mls_back19(M, invd, b);
    } else {
      mls_back9(M, invd, b);
    }
    use(k, b);
  }
}

// Outputs of one fitted slot from its parked derivative rows: fit status
// and gradients / Hessians (derivative mode) or the MHD time derivatives.
// Singular fits (too few neighbours) report zero derivatives.  No barrier.
template <FitMode MODE, int T>
__device__ __forceinline__ void write_outputs(const FitArgs& a, int s, bool singular, float* park,
                                              int tid) {
  using G = Groups<MODE>;
  const int64_t n = a.n;
  const float4* rec = reinterpret_cast<const float4*>(a.rec);
  if (singular) {
#pragma unroll 1
    for (int k = 0; k < G::NF; ++k)
      for (int j = 0; j < 9; ++j) park[(k * kNB + j) * T + tid] = 0.f;
  }
  const int dst = a.perm_out ? a.perm_out[s] : s;
  if (a.fit_status) a.fit_status[dst] = singular ? 1 : 0;
  if (singular) raise_flag(a.status_word, PHB_FLAG_FIT_SINGULAR);
  if (MODE == FitMode::kDerivs) {
#pragma unroll 1
    for (int k = 0; k < G::NF; ++k) {
      const int f = G::field(k);
      const float* d = park + (k * kNB) * T + tid;
      for (int c = 0; c < 3; ++c) a.grad[(f * 3 + c) * n + dst] = d[c * T];
      if (a.hess)
        for (int c = 0; c < 6; ++c) a.hess[(f * 6 + c) * n + dst] = d[(3 + c) * T];
    }
  } else {
    MhdDerivs<float> D;
    mhd_zero(D);
#pragma unroll
    for (int k = 0; k < G::NF; ++k) {
      const float* d = park + (k * kNB) * T + tid;
      const float g[3] = {d[0], d[T], d[2 * T]};
      const float h[6] = {d[3 * T], d[4 * T], d[5 * T], d[6 * T], d[7 * T], d[8 * T]};
      mhd_collect(D, G::field(k), g, h);
    }
    const float4 o2 = rec[6 * s + 2], o3 = rec[6 * s + 3], o4 = rec[6 * s + 4], o5 = rec[6 * s + 5];
    const float u[8] = {o2.x + o3.x, o2.z + o3.z, o2.w + o3.w, o4.x + o5.x,
                        o4.y + o5.y, o4.z + o5.z, o4.w + o5.w, o2.y + o3.y};
    const int src = a.perm_in ? a.perm_in[s] : s;
    float zeta = a.zeta ? static_cast<float>(a.zeta[src]) : 0.f;
    float eta = a.eta ? static_cast<float>(a.eta[src]) : 0.f;
    if (a.c_zeta_l != 0.0 || a.c_zeta_a != 0.0 || a.c_eta != 0.0)
      mhd_laws(u, D, static_cast<float>(a.gamma), static_cast<float>(a.slam[s]),
               static_cast<float>(a.c_zeta_l), static_cast<float>(a.c_zeta_a),
               static_cast<float>(a.c_eta), zeta, eta);
    float out[8];
    mhd_rhs(u, D, static_cast<float>(a.gamma), zeta, eta, out);
    bool finite = true;
#pragma unroll
    for (int f = 0; f < 8; ++f) {
      finite &= isfinite(out[f]);
      a.dudt[f * n + dst] = out[f];
    }
    if (!finite) raise_flag(a.status_word, PHB_FLAG_NONFINITE);
  }
}

struct TileArgs {
  const int2* tplan;      // per tile: (staged particles, 1 = not staged)
  const int32_t* tslot;   // per tile: slot of every staged index (stage_cap stride)
  const uint16_t* lself;  // per slot: its own staged index
  const uint8_t* tmap;    // per tile: thread -> tile particle (longest list first)
  const uint16_t* lidx;
  int32_t* fallback_count;
  const int32_t* order;   // tile of each CTA in descending cost (schedule 1), or null
  int32_t ntiles;
  const int32_t* list;      // active subset: slots (ascending), or null for all particles
  const int32_t* list_len;  // device count of the active subset
};

// Shared memory of one CTA besides the dynamic park/staging region.
template <int T>
struct FitShared {
  int wfar[T / 32];  // per warp: staged an offset at or beyond a quarter box length
  uint8_t fin[T];   // host-buffer corrector: the tile particle's fit is final here
};

// Stage a tile's neighbourhood (count records, slots from the plan) in shared
// memory: offsets and field differences relative to the tile's middle slot
// sr, from the FP32 hi/lo records.  All T threads call it; no barrier inside.
// Returns whether this thread staged an offset of a quarter box length or
// more on a periodic axis (the tile's differences then need the wrap).
template <int T>
__device__ __forceinline__ bool stage_tile(const FitArgs& a, const Per32& P, const TileArgs& ta,
                                           int tile, int sr, int count, float4* stage, int tid) {
  bool far = false;
  const float4* rec = reinterpret_cast<const float4*>(a.rec);
  // records relative to the tile's middle particle: the staged FP32 offsets
  // and field differences round to at most half the tile's extent
  const float4 rh = rec[6 * sr], rl = rec[6 * sr + 1];
  const float4 fh = rec[6 * sr + 2], fl = rec[6 * sr + 3], gh = rec[6 * sr + 4], gl = rec[6 * sr + 5];
  const int32_t* slots = ta.tslot + static_cast<int64_t>(tile) * a.g.stage_cap;
  // eight records per thread in flight: slots first, then all their loads
  constexpr int kB = 8;
  for (int l0 = tid; l0 < count; l0 += kB * T) {
    int sl[kB];
#pragma unroll
    for (int u = 0; u < kB; ++u) sl[u] = l0 + u * T < count ? slots[l0 + u * T] : -1;
    float4 v[kB][6];
#pragma unroll
    for (int u = 0; u < kB; ++u)
      if (sl[u] >= 0)
#pragma unroll
        for (int k = 0; k < 6; ++k) v[u][k] = rec[6 * sl[u] + k];
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      if (sl[u] < 0) continue;
      const float4 p0 = v[u][0], p1 = v[u][1], f0 = v[u][2], f1 = v[u][3], g0 = v[u][4], g1 = v[u][5];
      float4* d = stage + 3 * (l0 + u * T);
      const float ox = mi_diff32(p0.x, p1.x, rh.x, rl.x, P.len_h[0], P.len_l[0], P.inv_len[0]);
      const float oy = mi_diff32(p0.y, p1.y, rh.y, rl.y, P.len_h[1], P.len_l[1], P.inv_len[1]);
      const float oz = mi_diff32(p0.z, p1.z, rh.z, rl.z, P.len_h[2], P.len_l[2], P.inv_len[2]);
      far |= fabsf(ox) * P.inv_len[0] >= 0.25f || fabsf(oy) * P.inv_len[1] >= 0.25f ||
             fabsf(oz) * P.inv_len[2] >= 0.25f;
      d[0] = make_float4(ox, oy, oz, hl(f0.y, f1.y, fh.y, fl.y));
      d[1] = make_float4(hl(f0.z, f1.z, fh.z, fl.z), hl(f0.w, f1.w, fh.w, fl.w),
                         hl(g0.x, g1.x, gh.x, gl.x), hl(f0.x, f1.x, fh.x, fl.x));
      d[2] = make_float4(hl(g0.y, g1.y, gh.y, gl.y), hl(g0.z, g1.z, gh.z, gl.z),
                         hl(g0.w, g1.w, gh.w, gl.w), 0.f);
    }
  }
  return far;
}

// Host-buffer step, corrector evaluation: thread t takes the tile's slot
// s0 + t (slot order) and, where its fit is final (not routed to FP64, not
// queued for the corrected step, not frozen) and the caller indices of its
// warp's slots lie within 64 of each other (so that the warp's host writes
// stay on a few lines), writes U^{n+1} = Y^n + h (F(Y^n) + F(Y^p)) - the
// corrector's arithmetic, with F(Y^p) read back from this tile's dudt - to
// the caller's row of the mapped host array; pc_done marks the slots
// written.  Called by all T threads after a barrier that follows the
// tile's output writes.
template <int T>
__device__ __forceinline__ void host_u_tile(const FitArgs& a, int s0, int cnt, const FitShared<T>& sh,
                                            int tid) {
  const int64_t n = a.n;
  const bool ok = tid < cnt;
  const int s = s0 + tid;
  const int i = ok ? a.pc_perm[s] : 0;
  const int lo = __reduce_min_sync(0xffffffffu, ok ? i : 0x7fffffff);
  const int hi = __reduce_max_sync(0xffffffffu, ok ? i : -1);
  const bool near = hi >= lo && hi - lo < 64;
  const bool w = ok && near && sh.fin[tid] != 0 && !(a.pc_frozen && a.pc_frozen[i]);
  if (w) {
#pragma unroll
    for (int f = 0; f < 8; ++f)
      a.u_host[f * n + i] =
          __fma_rn(a.pc_h, __dadd_rn(a.pc_f0[f * n + s], a.dudt[f * n + s]), a.pc_y0[(3 + f) * n + s]);
  }
  if (ok) a.pc_done[s] = w ? 1 : 0;
}

// One tile: stage its neighbourhood, accumulate, solve, write outputs.  All
// T threads call it (it contains block barriers).  Threads are assigned to
// the tile's particles in descending list length (map recorded by the
// neighbour build) so that the lanes of a warp run loops of similar length.
template <FitMode MODE, int T>
__device__ __forceinline__ void fit_tile(const FitArgs& a, const Per32& P, const TileArgs& ta,
                                         int tile, float* park, float4* stage, FitShared<T>& sh) {
  using G = Groups<MODE>;
  const int n = a.n;
  const int tid = threadIdx.x;
  const float4* rec = reinterpret_cast<const float4*>(a.rec);
  // an active subset runs in chunks of T listed slots through the unstaged path
  const bool listed = ta.list != nullptr;
  const int s0 = tile * T;
  const int cnt_tile = min(T, (listed ? *ta.list_len : n) - s0);
  const int mine = listed ? tid : ta.tmap[static_cast<int64_t>(tile) * T + tid];
  const bool active = mine < cnt_tile;
  const int s = listed ? (active ? ta.list[s0 + mine] : 0) : s0 + mine;

  // the neighbourhood planned by the neighbour build: one gather per staged record
  const int2 tp = listed ? make_int2(0, 1) : ta.tplan[tile];
  const bool fb = tp.y != 0;
  if (!fb) {
    const bool far = stage_tile<T>(a, P, ta, tile, s0 + (cnt_tile >> 1), tp.x, stage, tid);
    const bool wfar = __any_sync(0xffffffffu, far);
    if ((tid & 31) == 0) sh.wfar[tid >> 5] = wfar ? 1 : 0;
  } else if (tid == 0 && !listed) {
    atomicAdd(ta.fallback_count, 1);
  }
  __syncthreads();

  float2 m2[kNM2];
  float2 bB[4][kNB2];
  int cnt = 0;
  float inv_l = 1.f, inv_rf2 = 0.f;
  int64_t beg = 0, end = 0;
  const bool unweighted = a.weight_kind == 1;
  if (active) {
    // the scales in FP32: two FP64 divisions per particle would queue on
    // GB300's narrow FP64 pipe whenever a CTA's threads start together
    const float lamf = static_cast<float>(a.slam[s]);
    const float rff = static_cast<float>(a.g.rf_factor) * lamf;
    inv_l = 1.f / lamf;
    inv_rf2 = 1.f / (rff * rff);
    beg = a.off[s];
    end = a.off[s + 1] < a.g.capacity ? a.off[s + 1] : a.g.capacity;
    if (fb) {
      GlobalSrc src;
      src.rec = rec;
      src.idx = a.idx;
      for (int k = 0; k < 6; ++k) src.o[k] = rec[6 * s + k];
      src.P = P;
      cnt = accumulate<MODE, T>(src, beg, end, inv_l, inv_rf2, unweighted, park, tid, m2, bB);
    } else {
      auto run = [&](auto src) {
        src.stage = stage;
        src.lidx = ta.lidx;
        const int ls = ta.lself[s];
        src.me0 = stage[3 * ls];
        src.me1 = stage[3 * ls + 1];
        src.me2 = stage[3 * ls + 2];
        for (int c = 0; c < 3; ++c) {
          src.len[c] = P.len[c];
          src.inv_len[c] = P.inv_len[c];
        }
        return accumulate<MODE, T>(src, beg, end, inv_l, inv_rf2, unweighted, park, tid, m2, bB);
      };
      bool wrap = false;
      for (int w = 0; w < T / 32; ++w) wrap |= sh.wfar[w] != 0;
      cnt = wrap ? run(StagedSrc<true>{}) : run(StagedSrc<false>{});
    }
  }
  __syncthreads();  // the staged records are dead from here on
  // moments kept for the corrected step, after the parked right-hand sides
  float* mstash = park + G::NF * kNB * T;
  const bool may_refine = a.refine_mode >= 0;
  const bool singular = !active || cnt < kNB;
  bool routed = false, need = false;
  float M[kNT], invd[kNB];
  if (active) {
#pragma unroll
    for (int f = 0; f < 4; ++f)
#pragma unroll
      for (int k = 0; k < kNB; ++k) park[((G::NA + f) * kNB + k) * T + tid] = pair_at(bB[f], k);
    if (!singular) {
      if (may_refine)
#pragma unroll
        for (int k = 0; k < kNM2; ++k) {
          mstash[(2 * k) * T + tid] = m2[k].x;
          mstash[(2 * k + 1) * T + tid] = m2[k].y;
        }
      mls_assemble_p2(m2, M);
      const float minpiv = mls_cholesky<float>(M, invd);
      // conditioning estimate of the Jacobi-scaled matrix: n_b times the
      // greedy estimate of ||M_s^-1||_inf (|M_s,rc| <= 1, so ||M_s||_inf <= n_b)
      const float kappa = static_cast<float>(kNB) * mls_inv_norm_est<float>(M, invd);
      if (!(minpiv > 0.f) || !(kappa <= a.cond_threshold)) {
        const int q = atomicAdd(a.queue_len, 1);
        a.queue[q] = s;
        routed = true;
      } else {
        need = a.refine_mode == 1 || kappa > a.refine_kappa;
      }
    }
  }
  // one decision per tile keeps the CTA's control flow uniform
  const bool refine = may_refine && __syncthreads_or(need);
  if (refine && tid == 0) atomicAdd(a.refined_tiles, 1);
  const bool solve = !singular && !routed;
  const float il = inv_l, il2 = inv_l * inv_l;
  if (solve && !refine) {
    solve_fields<G::NF, false, true>(
        M, invd, [&](int k, int j) { return park[(k * kNB + j) * T + tid]; },
        [&](int k, const float(&b)[kNB]) { park_derivs<T>(park + (k * kNB) * T + tid, b, il, il2); });
  }
  // A refined tile of a set whose records fit in L2 hands its solved fits to
  // k_fit_refine: one queue position per fit (one atomic per warp), its
  // moments and the first solve's 19 coefficients of every field into the
  // queue's stash.  (Before the in-tile step below, so that the factor is
  // dead during that step's residual passes.)
  const bool deferred = refine && solve && a.refine_queued;
  const unsigned dmask = __ballot_sync(0xffffffffu, deferred);
  if (dmask != 0u) {
    const int lane = tid & 31;
    const int leader = __ffs(dmask) - 1;
    int qbase = 0;
    if (lane == leader) qbase = atomicAdd(a.rq_len, __popc(dmask));
    qbase = __shfl_sync(0xffffffffu, qbase, leader);
    if (deferred) {
      const int64_t q = qbase + __popc(dmask & ((1u << lane) - 1u));
      a.rqueue[q] = s;
      float* st = a.rstash + q;
#pragma unroll 4
      for (int k = 0; k < kNM; ++k) st[k * static_cast<int64_t>(n)] = mstash[k * T + tid];
      solve_fields<G::NF, true, false>(
          M, invd, [&](int k, int j) { return park[(k * kNB + j) * T + tid]; },
          [&](int k, const float(&b)[kNB]) {
#pragma unroll
            for (int j = 0; j < kNB; ++j) st[(kNM + k * kNB + j) * static_cast<int64_t>(n)] = b[j];
          });
    }
  }
  if (solve && refine && !a.refine_queued) {
    // Otherwise the corrected step here, while the tile's neighbourhood is
    // still in L2 (sets whose records exceed L2).  First solve: all 19 coefficients of
    // every field in place of its parked right-hand side, and the nine linear
    // and quadratic ones (which the correction is added to) in the slot's
    // column of the stash
    float* cq = a.rstash + s;
    solve_fields<G::NF, true, false>(
        M, invd, [&](int k, int j) { return park[(k * kNB + j) * T + tid]; },
        [&](int k, const float(&b)[kNB]) {
#pragma unroll
          for (int j = 0; j < kNB; ++j) park[(k * kNB + j) * T + tid] = b[j];
#pragma unroll
          for (int j = kQuad0; j < kNB; ++j) cq[(kNM + k * kNB + j) * static_cast<int64_t>(n)] = b[j];
        });
    // residual passes over the neighbours from the global records (see
    // k_fit_refine)
    GlobalSrc src;
    src.rec = rec;
    src.idx = a.idx;
    for (int k = 0; k < 6; ++k) src.o[k] = rec[6 * s + k];
    src.P = P;
    {
      float2 acc[G::NA][kNB2];
      csne_pass<G::NA, false>(src, beg, end, inv_l, inv_rf2, unweighted, park + tid, T, 0,
                              4 - G::NA, acc);
#pragma unroll
      for (int f = 0; f < G::NA; ++f)
#pragma unroll
        for (int k = 0; k < kNB; ++k) park[(f * kNB + k) * T + tid] = pair_at(acc[f], k);
    }
    {
      float2 acc[4][kNB2];
      csne_pass<4, true>(src, beg, end, inv_l, inv_rf2, unweighted, park + tid, T, G::NA, 0, acc);
#pragma unroll
      for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int k = 0; k < kNB; ++k) park[((G::NA + f) * kNB + k) * T + tid] = pair_at(acc[f], k);
    }
    // the same factor again from the kept moments; correction of the linear
    // and quadratic coefficients
    float2 mm[kNM2];
#pragma unroll
    for (int k = 0; k < kNM2; ++k)
      mm[k] = make_float2(mstash[(2 * k) * T + tid], mstash[(2 * k + 1) * T + tid]);
    float M2[kNT], invd2[kNB];
    mls_assemble_p2(mm, M2);
    mls_cholesky<float>(M2, invd2);
    // one field at a time, as k_fit_refine solves it: the two schedules then
    // round alike (the last scaling contracts with the added c0 into one FMA)
    solve_fields<G::NF, false, false>(
        M2, invd2, [&](int k, int j) { return park[(k * kNB + j) * T + tid]; },
        [&](int k, float(&b)[kNB]) {
#pragma unroll
          for (int j = kQuad0; j < kNB; ++j) b[j] += cq[(kNM + k * kNB + j) * static_cast<int64_t>(n)];
          park_derivs<T>(park + (k * kNB) * T + tid, b, il, il2);
        });
  }
  if (active && !routed && !deferred) write_outputs<MODE, T>(a, s, singular, park, tid);
  if (MODE == FitMode::kRHS && a.u_host != nullptr && !listed) {
    if (active) sh.fin[mine] = (!routed && !deferred) ? 1 : 0;
    __syncthreads();  // the tile's outputs and marks are written
    host_u_tile<T>(a, s0, cnt_tile, sh, tid);
  }
}

template <FitMode MODE, int T>
__global__ void __launch_bounds__(T, 256 / T) k_fit_mixed(const FitArgs a, const Per32 P, const TileArgs ta) {
  using G = Groups<MODE>;
  // dynamic shared memory: [park A: NA*19 slots x T][staged records: stage_cap x 3 float4];
  // after the accumulation the whole region holds the NF*19 parked slots.
  extern __shared__ float4 smem4[];
  __shared__ FitShared<T> sh;
  float* park = reinterpret_cast<float*>(smem4);
  float4* stage = smem4 + (G::NA * kNB * T) / 4;
  // schedule 1: the block scheduler's dispatch order runs the tiles in
  // descending cost (longest first), without a loop over tiles in the kernel
  fit_tile<MODE, T>(a, P, ta, ta.order ? ta.order[blockIdx.x] : static_cast<int>(blockIdx.x), park,
                    stage, sh);
}

// The corrected step of the fits of refined tiles (queued by k_fit_mixed with
// their moments and first solves): one thread per queued fit, grid-stride
// over the queue, no barrier, so that warps stream through the queue instead
// of waiting at a tile's barriers for its longest lists.  Two residual passes
// over the neighbours from the global records (offsets and field differences
// straight from the hi/lo splits of the particle and the neighbour round to
// ~2^-24 of the difference itself, while the staged ones, relative to a
// tile's middle particle, round to 2^-24 of the change across the tile - too
// coarse a floor for the corrected solution) accumulate P^T W (du - P c0);
// the factor re-formed from the moments gives the correction of the linear
// and quadratic coefficients, added to c0's, and the outputs follow.
template <FitMode MODE, int T>
__global__ void __launch_bounds__(T, 256 / T) k_fit_refine(const FitArgs a, const Per32 P) {
  using G = Groups<MODE>;
  extern __shared__ float4 smem4[];
  float* park = reinterpret_cast<float*>(smem4);  // [NF * 19][T]: one column per thread
  const int tid = threadIdx.x;
  const int64_t n = a.n;
  // launched as a programmatic dependent of k_fit_mixed: wait until it has
  // completed and its queue and stash are visible
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const int64_t len = *a.rq_len;
  const float4* rec = reinterpret_cast<const float4*>(a.rec);
  const bool unweighted = a.weight_kind == 1;
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * T + tid; q < len;
       q += static_cast<int64_t>(gridDim.x) * T) {
    const int s = a.rqueue[q];
    const float* st = a.rstash + q;
    const float lamf = static_cast<float>(a.slam[s]);
    const float rff = static_cast<float>(a.g.rf_factor) * lamf;
    const float inv_l = 1.f / lamf;
    const float inv_rf2 = 1.f / (rff * rff);
    const int64_t beg = a.off[s];
    const int64_t end = a.off[s + 1] < a.g.capacity ? a.off[s + 1] : a.g.capacity;
    GlobalSrc src;
    src.rec = rec;
    src.idx = a.idx;
    // the particle's own record: positions and the first field group now,
    // the second group before its pass (fewer registers live in the first)
    for (int k = 0; k < 4; ++k) src.o[k] = rec[6 * s + k];
    src.P = P;
    {
      float2 acc[G::NA][kNB2];
      csne_pass<G::NA, false>(src, beg, end, inv_l, inv_rf2, unweighted, st + kNM * n, n, 0,
                              4 - G::NA, acc);
#pragma unroll
      for (int f = 0; f < G::NA; ++f)
#pragma unroll
        for (int k = 0; k < kNB; ++k) park[(f * kNB + k) * T + tid] = pair_at(acc[f], k);
    }
    {
      src.o[4] = rec[6 * s + 4];
      src.o[5] = rec[6 * s + 5];
      float2 acc[4][kNB2];
      csne_pass<4, true>(src, beg, end, inv_l, inv_rf2, unweighted, st + kNM * n, n, G::NA, 0, acc);
#pragma unroll
      for (int f = 0; f < 4; ++f)
#pragma unroll
        for (int k = 0; k < kNB; ++k) park[((G::NA + f) * kNB + k) * T + tid] = pair_at(acc[f], k);
    }
    float2 mm[kNM2];
#pragma unroll
    for (int k = 0; k < kNM2; ++k) mm[k] = make_float2(st[(2 * k) * n], st[(2 * k + 1) * n]);
    float M[kNT], invd[kNB];
    mls_assemble_p2(mm, M);
    mls_cholesky<float>(M, invd);
    const float il = inv_l, il2 = inv_l * inv_l;
    solve_fields<G::NF, false, false>(
        M, invd, [&](int k, int j) { return park[(k * kNB + j) * T + tid]; },
        [&](int k, float(&b)[kNB]) {
#pragma unroll
          for (int j = kQuad0; j < kNB; ++j) b[j] += st[(kNM + k * kNB + j) * n];
          park_derivs<T>(park + (k * kNB) * T + tid, b, il, il2);
        });
    write_outputs<MODE, T>(a, s, false, park, tid);
  }
}

// ------------------------------------------------------------------------
// Tensor-core form of the accumulation (a measured experiment, reachable only
// through phb_fit_tc_experiment).  Per particle the moments and right-hand
// sides are the Gram matrix G = A^T W A of the rows a_j = [p(q_j) (19 basis
// monomials) | du_j (7 fitted fields) | 0 (6)], W = diag(w_j): a dense
// contraction over the neighbours.  One warp forms the Grams of its 32
// particles in turn: the lanes build 32 neighbour rows at a time in shared
// memory, then mma.sync m16n8k8 (TF32 inputs, FP32 accumulation) takes them
// eight rows per step, with each operand split into TF32 hi + lo parts and
// the three products hi*hi + hi*lo + lo*hi (3xTF32) for FP32-level products.
// Only the five 16x8 output tiles that hold the lower triangle's moments and
// right-hand sides are formed.  A second kernel reads them back and runs the
// same solve and right-hand side as k_fit_mixed (no FP64 routing and no
// corrected step: the experiment compares the accumulation alone).

constexpr int kTcRow = 33;                    // floats per staged row (32 + 1 pad)
constexpr int kTcWarpFloats = 32 * kTcRow + 32 + 26 * 26;  // rows, weights, Gram
constexpr int kTcWords = kNM + 7 * kNB + 1;   // moments, right-hand sides, count

__device__ __forceinline__ uint32_t tf32_of(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_of(x);
  lo = tf32_of(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One neighbour row: basis monomials, then the fitted fields' differences in
// the RHS mode's parked order (sigma, Vx, Vy, Vz, Bx, By, Bz); weight w.
template <class Src>
__device__ __forceinline__ void tc_row(const Src& src, int nb, float inv_l, float inv_rf2,
                                       bool unweighted, float* row, float& w) {
  float dx, dy, dz, ua[4], ub[4];
  src.decode_a(src.fetch_a(nb), dx, dy, dz, ua);
  src.decode_b(src.fetch_b(nb), dx, dy, dz, ub);
  const float s2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) * inv_rf2;
  const float sw = 1.f - s2;
  w = s2 < 1.f ? (unweighted ? 1.f : sw * sw) : 0.f;
  float qg[kNB];
  mls_basis(dx * inv_l, dy * inv_l, dz * inv_l, qg);
#pragma unroll
  for (int k = 0; k < kNB; ++k) row[k] = qg[k];
  row[19] = ua[1];
  row[20] = ua[2];
  row[21] = ua[3];
#pragma unroll
  for (int f = 0; f < 4; ++f) row[22 + f] = ub[f];
#pragma unroll
  for (int k = 26; k < 32; ++k) row[k] = 0.f;
}

template <int T>
__global__ void __launch_bounds__(T, 2) k_gram_tc(const FitArgs a, const Per32 P, const TileArgs ta,
                                                  float* __restrict__ gram) {
  extern __shared__ float4 smem4[];
  float4* stage = smem4;
  float* wbuf = reinterpret_cast<float*>(stage + 3 * a.g.stage_cap);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  float* rows = wbuf + warp * kTcWarpFloats;
  float* wts = rows + 32 * kTcRow;
  float* G = wts + 32;
  const int n = a.n, tile = blockIdx.x, s0 = tile * T;
  const int cnt_tile = min(T, n - s0);
  const int mine = ta.tmap[static_cast<int64_t>(tile) * T + tid];
  const bool active = mine < cnt_tile;
  const int s_own = s0 + mine;
  const float4* rec = reinterpret_cast<const float4*>(a.rec);
  const int2 tp = ta.tplan[tile];
  const bool fb = tp.y != 0;
  if (!fb) stage_tile<T>(a, P, ta, tile, s0 + (cnt_tile >> 1), tp.x, stage, tid);
  __syncthreads();
  const bool unweighted = a.weight_kind == 1;
  for (int p = 0; p < 32; ++p) {
    if (!__shfl_sync(0xffffffffu, active, p)) continue;
    const int s = __shfl_sync(0xffffffffu, s_own, p);
    const double lam = a.slam[s];
    const double rf = a.g.rf_factor * lam;
    const float inv_l = static_cast<float>(1.0 / lam);
    const float inv_rf2 = static_cast<float>(1.0 / (rf * rf));
    const int64_t beg = a.off[s];
    const int64_t end = a.off[s + 1] < a.g.capacity ? a.off[s + 1] : a.g.capacity;
    StagedSrc<true> ssrc;  // the experiment keeps the wrap everywhere
    GlobalSrc gsrc;
    if (fb) {
      gsrc.rec = rec;
      gsrc.idx = a.idx;
      for (int k = 0; k < 6; ++k) gsrc.o[k] = rec[6 * s + k];
      gsrc.P = P;
    } else {
      ssrc.stage = stage;
      ssrc.lidx = ta.lidx;
      const int ls = ta.lself[s];
      ssrc.me0 = stage[3 * ls];
      ssrc.me1 = stage[3 * ls + 1];
      ssrc.me2 = stage[3 * ls + 2];
      for (int c = 0; c < 3; ++c) {
        ssrc.len[c] = P.len[c];
        ssrc.inv_len[c] = P.inv_len[c];
      }
    }
    float acc[5][4];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][q] = 0.f;
    int inside = 0;
    for (int64_t c0 = beg; c0 < end; c0 += 32) {
      const int64_t e = c0 + lane;
      float w = 0.f;
      float* row = rows + lane * kTcRow;
      if (e < end) {
        if (fb) tc_row(gsrc, gsrc.index(e), inv_l, inv_rf2, unweighted, row, w);
        else tc_row(ssrc, ssrc.index(e), inv_l, inv_rf2, unweighted, row, w);
      } else {
        for (int k = 0; k < 32; ++k) row[k] = 0.f;
      }
      wts[lane] = w;
      inside += __popc(__ballot_sync(0xffffffffu, w > 0.f));
      __syncwarp();
      const int nrows = static_cast<int>(end - c0 < 32 ? end - c0 : 32);
      for (int ks = 0; ks * 8 < nrows; ++ks) {
        const int r0 = ks * 8 + t, r1 = r0 + 4;
        const float w0 = wts[r0], w1 = wts[r1];
        uint32_t ahi[2][4], alo[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          const int f = mt * 16 + g;
          split_tf32(rows[r0 * kTcRow + f], ahi[mt][0], alo[mt][0]);
          split_tf32(rows[r0 * kTcRow + f + 8], ahi[mt][1], alo[mt][1]);
          split_tf32(rows[r1 * kTcRow + f], ahi[mt][2], alo[mt][2]);
          split_tf32(rows[r1 * kTcRow + f + 8], ahi[mt][3], alo[mt][3]);
        }
        uint32_t bhi[3][2], blo[3][2];
#pragma unroll
        for (int nt = 0; nt < 3; ++nt) {
          const int f = nt * 8 + g;
          split_tf32(w0 * rows[r0 * kTcRow + f], bhi[nt][0], blo[nt][0]);
          split_tf32(w1 * rows[r1 * kTcRow + f], bhi[nt][1], blo[nt][1]);
        }
        // tiles (m, n): (0,0) (0,1) (1,0) (1,1) (1,2)
        constexpr int tm[5] = {0, 0, 1, 1, 1}, tn[5] = {0, 1, 0, 1, 2};
#pragma unroll
        for (int i = 0; i < 5; ++i) {
          mma_tf32(acc[i], ahi[tm[i]], bhi[tn[i]][0], bhi[tn[i]][1]);
          mma_tf32(acc[i], ahi[tm[i]], blo[tn[i]][0], blo[tn[i]][1]);
          mma_tf32(acc[i], alo[tm[i]], bhi[tn[i]][0], bhi[tn[i]][1]);
        }
      }
      __syncwarp();
    }
    // lower triangle of G from the accumulator fragments
    {
      constexpr int tm[5] = {0, 0, 1, 1, 1}, tn[5] = {0, 1, 0, 1, 2};
#pragma unroll
      for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = tm[i] * 16 + g + 8 * (q >> 1), c = tn[i] * 8 + 2 * t + (q & 1);
          if (r < 26 && c <= r) G[r * 26 + c] = acc[i][q];
        }
    }
    __syncwarp();
    for (int k = lane; k < kTcWords; k += 32) {
      float v;
      if (k < kNM) {
        int r, c;
        mls_moment_pair(k, r, c);
        v = G[r * 26 + c];
      } else if (k < kTcWords - 1) {
        const int f = (k - kNM) / kNB, j = (k - kNM) % kNB;
        v = G[(19 + f) * 26 + j];
      } else {
        v = static_cast<float>(inside);
      }
      gram[static_cast<int64_t>(k) * n + s] = v;
    }
    __syncwarp();
  }
}

// Solve and right-hand side from the Gram words (thread per slot).
__global__ void __launch_bounds__(128) k_solve_gram(const FitArgs a, const float* __restrict__ gram) {
  using G = Groups<FitMode::kRHS>;
  const int n = a.n;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int64_t N = n;
  const int dst = a.perm_out ? a.perm_out[s] : s;
  const float inv_l = static_cast<float>(1.0 / a.slam[s]);
  const float il = inv_l, il2 = inv_l * inv_l;
  MhdDerivs<float> D;
  mhd_zero(D);
  bool singular = gram[(kTcWords - 1) * N + s] < static_cast<float>(kNB);
  if (!singular) {
    float m[kNM], M[kNT], invd[kNB];
#pragma unroll
    for (int k = 0; k < kNM; ++k) m[k] = gram[k * N + s];
    mls_assemble(m, M);
    singular = !(mls_cholesky<float>(M, invd) > 0.f);
    if (!singular) {
#pragma unroll 1
      for (int k = 0; k < G::NF; ++k) {
        float b[kNB];
#pragma unroll
        for (int j = 0; j < kNB; ++j) b[j] = gram[(kNM + k * kNB + j) * N + s];
        mls_forward(M, invd, b);
        mls_back9(M, invd, b);
        const float gr[3] = {b[kLin0] * il, b[kLin0 + 1] * il, b[kLin0 + 2] * il};
        const float h[6] = {2.f * b[kQuad0] * il2, b[kQuad0 + 1] * il2, b[kQuad0 + 2] * il2,
                            2.f * b[kQuad0 + 3] * il2, b[kQuad0 + 4] * il2, 2.f * b[kQuad0 + 5] * il2};
        mhd_collect(D, G::field(k), gr, h);
      }
    }
  }
  if (a.fit_status) a.fit_status[dst] = singular ? 1 : 0;
  if (singular) {
    mhd_zero(D);
    raise_flag(a.status_word, PHB_FLAG_FIT_SINGULAR);
  }
  const float4* rec = reinterpret_cast<const float4*>(a.rec);
  const float4 o2 = rec[6 * s + 2], o3 = rec[6 * s + 3], o4 = rec[6 * s + 4], o5 = rec[6 * s + 5];
  const float u[8] = {o2.x + o3.x, o2.z + o3.z, o2.w + o3.w, o4.x + o5.x,
                      o4.y + o5.y, o4.z + o5.z, o4.w + o5.w, o2.y + o3.y};
  const int src = a.perm_in ? a.perm_in[s] : s;
  const float zeta = a.zeta ? static_cast<float>(a.zeta[src]) : 0.f;
  const float eta = a.eta ? static_cast<float>(a.eta[src]) : 0.f;
  float out[8];
  mhd_rhs(u, D, static_cast<float>(a.gamma), zeta, eta, out);
  for (int f = 0; f < 8; ++f) a.dudt[f * N + dst] = out[f];
}

Per32 make_per32(const Grid& g) {
  Per32 P;
  for (int a = 0; a < 3; ++a) {
    const float h = static_cast<float>(g.len[a]);
    P.len_h[a] = g.periodic[a] ? h : 0.f;
    P.len_l[a] = g.periodic[a] ? static_cast<float>(g.len[a] - static_cast<double>(h)) : 0.f;
    P.inv_len[a] = g.periodic[a] ? static_cast<float>(1.0 / g.len[a]) : 0.f;
    P.len[a] = h;
  }
  return P;
}

template <FitMode MODE, int T>
cudaError_t launch_t(const FitArgs& a, const Per32& P, const TileArgs& ta, int64_t list_cap,
                     cudaStream_t st) {
  using G = Groups<MODE>;
  const size_t park_a = size_t(G::NA) * kNB * T * sizeof(float);
  const size_t staged = size_t(a.g.stage_cap) * 3 * sizeof(float4);
  // after the accumulation: the parked columns of all fields, and the
  // moments kept for the corrected step
  const size_t park_all = size_t(G::NF * kNB + (a.refine_mode >= 0 ? kNM : 0)) * T * sizeof(float);
  const size_t smem = park_a + staged > park_all ? park_a + staged : park_all;
  const int64_t units = ta.list ? list_cap : a.n;
  const unsigned tiles = static_cast<unsigned>((units + T - 1) / T);
  cudaError_t e;
  if (units == 0) return cudaGetLastError();
  {
    cudaFuncSetAttribute(k_fit_mixed<MODE, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    const int tr = trace_begin(1, st);
    k_fit_mixed<MODE, T><<<tiles, T, smem, st>>>(a, P, ta);
    note_launch();
    trace_end(tr, st);
  }
  if ((e = cudaGetLastError())) return e;
  if (a.refine_mode >= 0 && a.refine_queued) {
    // the corrected step of the queued fits: a grid that keeps every SM busy
    const size_t rsmem = size_t(G::NF) * kNB * T * sizeof(float);
    cudaFuncSetAttribute(k_fit_refine<MODE, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(rsmem));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fit_refine<MODE, T>, T, rsmem);
    if (per_sm < 1) per_sm = 1;
    unsigned grid = static_cast<unsigned>(num_sms() * per_sm);
    if (grid > tiles) grid = tiles;
    // a programmatic dependent launch: its set-up overlaps the fused fit's
    // tail, and the kernel waits for the fit's completion before it reads the
    // queue (an empty queue then costs little more than that wait)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(T);
    cfg.dynamicSmemBytes = rsmem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int tr = trace_begin(8, st);
    if ((e = cudaLaunchKernelEx(&cfg, k_fit_refine<MODE, T>, a, P))) return e;
    note_launch();
    trace_end(tr, st);
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fit_mixed(const FitArgs& a, FitMode mode, const int2* tplan, const int32_t* tslot,
                             const uint16_t* lself, const uint8_t* tmap, const uint16_t* lidx,
                             int32_t* fallback_count, const int32_t* order,
                             const int32_t* list, const int32_t* list_len, int64_t list_cap,
                             cudaStream_t st) {
  const Per32 P = make_per32(a.g);
  const TileArgs ta{tplan, tslot, lself, tmap, lidx, fallback_count,
                    (a.g.schedule == 1 && !list) ? order : nullptr,
                    static_cast<int32_t>((a.n + a.g.tile - 1) / a.g.tile), list, list_len};
  if (mode == FitMode::kDerivs)
    return a.g.tile == 64 ? launch_t<FitMode::kDerivs, 64>(a, P, ta, list_cap, st)
                          : launch_t<FitMode::kDerivs, 128>(a, P, ta, list_cap, st);
  return a.g.tile == 64 ? launch_t<FitMode::kRHS, 64>(a, P, ta, list_cap, st)
                        : launch_t<FitMode::kRHS, 128>(a, P, ta, list_cap, st);
}

cudaError_t launch_fit_tc(const FitArgs& a, const int2* tplan, const int32_t* tslot,
                          const uint16_t* lself, const uint8_t* tmap, const uint16_t* lidx,
                          float* gram, cudaStream_t st) {
  if (a.g.tile != 128) return cudaErrorInvalidValue;
  const Per32 P = make_per32(a.g);
  const TileArgs ta{tplan, tslot, lself, tmap, lidx, nullptr, nullptr,
                    static_cast<int32_t>((a.n + 127) / 128), nullptr, nullptr};
  const size_t smem = size_t(a.g.stage_cap) * 3 * sizeof(float4) + 4 * kTcWarpFloats * sizeof(float);
  cudaFuncSetAttribute(k_gram_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       static_cast<int>(smem));
  const unsigned tiles = static_cast<unsigned>((a.n + 127) / 128);
  int tr = trace_begin(6, st);
  k_gram_tc<128><<<tiles, 128, smem, st>>>(a, P, ta, gram);
  note_launch();
  trace_end(tr, st);
  tr = trace_begin(7, st);
  k_solve_gram<<<static_cast<unsigned>((a.n + 127) / 128), 128, 0, st>>>(a, gram);
  note_launch();
  trace_end(tr, st);
  return cudaGetLastError();
}

}  // namespace phb
