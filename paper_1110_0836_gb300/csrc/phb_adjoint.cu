// Reverse-mode adjoint of the fused MLS fit + MHD right-hand side, FP64.
// (The paper has no adjoint; this differentiates the forward map of
// phb_mhd_rhs: Sec. 2 fit and App. A right-hand side, neighbour sets fixed,
// lambda constant.)
//
// Per particle i, with fitted fields f (V, B, sigma) and neighbours j:
//   forward   m_a = sum_j w_j q_j^a,  b_f = sum_j w_j p_j dU_fj,  M c_f = b_f,
//             derivatives from c_f, right-hand side from derivatives and U_i;
//   backward  cbar_f from the right-hand side's adjoint, bbar_f = M^-1 cbar_f,
//             Mbar = -sum_f bbar_f c_f^T folded onto the moments (mbar),
//             then per neighbour
//               dUbar_fj = w_j (p_j . bbar_f)
//               wbar_j   = sum_a mbar_a q_j^a + sum_f dU_fj (p_j . bbar_f)
//               qbar_j   = w_j grad_q[ sum_a mbar_a q^a + sum_f dU_fj p(q) . bbar_f ]
//               dbar_j   = qbar_j / lambda_i + wbar_j dw/dd,
//             whose negatives are particle i's own terms (U_i, x_i).
// The first kernel keeps, per particle, only its adjoint seeds bbar_f and
// mbar (213 doubles) and its own terms; a second kernel gathers, for every
// particle j, the contributions of each i that lists j - through a reverse
// neighbour list in ascending order of i, recomputing q, w, p(q) and dw/dd
// of the entry from the positions - so the result does not depend on thread
// scheduling and no per-entry buffer is needed.  By default the factorisation is
// recomputed here (nothing is stored by the forward call); the stored variant
// records, per particle, the Cholesky factor, its Jacobi scaling and the
// fitted coefficients once (kRecord) and the adjoint then starts from that
// record (kStored) instead of re-accumulating the moments and right-hand sides.
#include "phb_internal.cuh"
#include "mls_gen.cuh"
#include "phb_mhd.cuh"

namespace phb {
namespace {

constexpr int kT = 64;
constexpr int kThreads = 256;
constexpr int kNFit = 7;                 // fitted fields: U indices 1..7 (V, B, sigma)
constexpr int kSm = kNM + kNFit * kNB;   // 213 doubles per thread (the 190-entry M overlays it)
// per-particle scratch record (contiguous per particle, read by the gather):
// bbar_f (7 x 19), then the coefficients c_f (7 x 19) of the recomputing
// form, whose first 80 words take mbar once c_f is no longer needed
constexpr int kScrBbar = 0, kScrC = kNFit * kNB, kScrMbar = kScrC, kScr = 2 * kNFit * kNB;
static_assert(kSm >= kNT, "shared region must hold the normal matrix");
// record of one particle's forward fit, [k][n] layout: factor (190), Jacobi
// scaling invd (19), coefficients c_f (7 x 19), then 1 = singular / 0 = regular
constexpr int kRecFac = 0, kRecInvd = kNT, kRecCoef = kNT + kNB, kRecFlag = kRecCoef + kNFit * kNB;
constexpr int kRecWords = kRecFlag + 1;
enum AdjMode { kRecompute = 0, kRecord = 1, kStored = 2 };

// Column view of thread-private shared memory ([k][kT] layout, no bank conflicts).
struct SCol {
  double* p;
  __device__ __forceinline__ double& operator[](int k) const { return p[k * kT]; }
};
// Column view of a per-particle array in global scratch ([k][n] layout, coalesced).
struct GCol {
  double* p;
  int64_t n;
  __device__ __forceinline__ double& operator[](int k) const { return p[k * n]; }
};

struct AdjArgs {
  Grid g;
  int32_t n;
  const int32_t* perm;   // slot -> caller index
  const double* spos;
  const double* slam;
  const double* sU;
  const int64_t* off;
  const int32_t* idx;
  const double* gbar;    // caller order [8][n]
  double gamma;
  int32_t weight_kind;
  const double* zeta;    // caller order or null
  const double* eta;
  double c_zeta_l, c_zeta_a, c_eta;  // coefficient laws (phb_params), 0 = off
  double* scr;           // [n][kScr] slot order: bbar_f, then c_f / mbar
  double* self;          // [11][n] slot order
  double* rec;           // [kRecWords][n] slot order (stored variant) or null
  int32_t* status_word;
};

struct Geo {
  double dx, dy, dz, s2;
};

__device__ __forceinline__ Geo geometry(const AdjArgs& a, int t, double xs, double ys, double zs,
                                        const double (&len)[3], const double (&ilen)[3],
                                        double inv_rf2) {
  const int64_t N = a.n;
  Geo q;
  q.dx = a.spos[t] - xs;
  q.dy = a.spos[N + t] - ys;
  q.dz = a.spos[2 * N + t] - zs;
  q.dx -= len[0] * rint(q.dx * ilen[0]);
  q.dy -= len[1] * rint(q.dy * ilen[1]);
  q.dz -= len[2] * rint(q.dz * ilen[2]);
  q.s2 = (q.dx * q.dx + q.dy * q.dy + q.dz * q.dz) * inv_rf2;
  return q;
}

// Adjoint of the right-hand side at one particle.  In: point values u, the
// derivatives D, the input coefficients zeta / eta and the coefficient laws
// (lam, cl, ca, ce as in mhd_laws), output adjoint o.  Out: ubar (point
// values) and the adjoints of each fitted field's gradient gb[f][3] and
// packed Hessian hb[f][6] (f = 0..6 for U indices 1..7).
__device__ void rhs_adjoint_point(const double (&u)[8], const MhdDerivs<double>& D, double gamma,
                                  double zeta, double eta, double lam, double cl, double ca,
                                  double ce, const double (&o)[8], double (&ubar)[8],
                                  double (&gb)[kNFit][3], double (&hb)[kNFit][6]) {
  const double rho = u[0], sig = u[7];
  const double B[3] = {u[4], u[5], u[6]};
  const double divV = D.gV[0][0] + D.gV[1][1] + D.gV[2][2];
  // the laws' totals (forward as mhd_laws): c = sqrt(q), q = (gamma P + |B|^2) / rho
  const bool laws = cl != 0.0 || ca != 0.0 || ce != 0.0;
  double q = 0.0, c = 0.0;
  if (laws) {
    q = (gamma * ((gamma - 1.0) * sig) + B[0] * B[0] + B[1] * B[1] + B[2] * B[2]) / rho;
    c = sqrt(q);
    zeta += cl * lam * c;
    if (divV < 0.0) zeta -= ca * lam * lam * divV;
    eta += ce * lam * c;
  }
  const double J[3] = {D.gB[2][1] - D.gB[1][2], D.gB[0][2] - D.gB[2][0], D.gB[1][0] - D.gB[0][1]};
  const double F[3] = {J[1] * B[2] - J[2] * B[1], J[2] * B[0] - J[0] * B[2], J[0] * B[1] - J[1] * B[0]};
  for (int k = 0; k < 8; ++k) ubar[k] = 0.0;
  for (int f = 0; f < kNFit; ++f) {
    for (int c = 0; c < 3; ++c) gb[f][c] = 0.0;
    for (int c = 0; c < 6; ++c) hb[f][c] = 0.0;
  }
  const double irho = 1.0 / rho;
  // out[1+a] = (F_a - (gamma-1) gs_a) / rho + zeta gdivV_a
  double Fb[3], divVb = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double ob = o[1 + a];
    Fb[a] = ob * irho;
    gb[6][a] += -ob * (gamma - 1.0) * irho;                       // sigma gradient
    ubar[0] += -ob * (F[a] - (gamma - 1.0) * D.gs[a]) * irho * irho;
    // gdivV_a = sum_c h_{V_c}[a, c]
    for (int c = 0; c < 3; ++c) hb[c][hpack(a, c)] += ob * zeta;
  }
  // out[0] = -rho divV
  ubar[0] += -o[0] * divV;
  divVb += -o[0] * rho;
  // out[4+a] = sum_b B_b gV[a][b] - B_a divV + eta gdivB_a
  for (int a = 0; a < 3; ++a) {
    const double ob = o[4 + a];
    for (int b = 0; b < 3; ++b) {
      gb[a][b] += ob * B[b];                 // gV[a][b]
      ubar[4 + b] += ob * D.gV[a][b];
    }
    ubar[4 + a] += -ob * divV;
    divVb += -ob * B[a];
    for (int c = 0; c < 3; ++c) hb[3 + c][hpack(a, c)] += ob * eta;
  }
  // out[7] = -gamma sigma divV + rho zeta divV^2
  ubar[7] += -o[7] * gamma * divV;
  ubar[0] += o[7] * zeta * divV * divV;
  divVb += o[7] * (-gamma * sig + 2.0 * rho * zeta * divV);
  if (laws) {
    // zeta_bar and eta_bar, then through zeta = .. + cl lam c + ca lam^2
    // max(0, -div V) and eta = .. + ce lam c
    double zb = o[7] * rho * divV * divV, eb = 0.0;
    for (int a = 0; a < 3; ++a) {
      zb += o[1 + a] * D.gdivV[a];
      eb += o[4 + a] * D.gdivB[a];
    }
    if (divV < 0.0) divVb += -zb * ca * lam * lam;
    const double cb = (zb * cl + eb * ce) * lam;
    if (c > 0.0) {
      const double qb = cb / (2.0 * c);
      ubar[7] += qb * gamma * (gamma - 1.0) / rho;
      for (int b = 0; b < 3; ++b) ubar[4 + b] += qb * 2.0 * B[b] / rho;
      ubar[0] += -qb * q / rho;
    }
  }
  for (int a = 0; a < 3; ++a) gb[a][a] += divVb;
  // F = J x B:  Bbar += Fbar x J,  Jbar = B x Fbar
  ubar[4] += Fb[1] * J[2] - Fb[2] * J[1];
  ubar[5] += Fb[2] * J[0] - Fb[0] * J[2];
  ubar[6] += Fb[0] * J[1] - Fb[1] * J[0];
  const double Jb[3] = {B[1] * Fb[2] - B[2] * Fb[1], B[2] * Fb[0] - B[0] * Fb[2], B[0] * Fb[1] - B[1] * Fb[0]};
  // J = (gB[2][1] - gB[1][2], gB[0][2] - gB[2][0], gB[1][0] - gB[0][1]); B_c is field 3 + c
  gb[3 + 2][1] += Jb[0];
  gb[3 + 1][2] -= Jb[0];
  gb[3 + 0][2] += Jb[1];
  gb[3 + 2][0] -= Jb[1];
  gb[3 + 1][0] += Jb[2];
  gb[3 + 0][1] -= Jb[2];
}

// Adjoint contribution of one list entry (particle i at xs with fields u,
// neighbour t) to the neighbour: ub[f] to U_t (fitted fields 1..7) and xb to
// x_t, from i's seeds bbar_f (stride bs) and mbar (stride ms).  The entry's
// offset, weight, monomials and dw/dd are recomputed from the positions.
// Returns false (nothing written) for an entry beyond r_f,i (skin).
__device__ __forceinline__ bool entry_adjoint(const AdjArgs& a, int t, double xs, double ys,
                                              double zs, const double (&u)[8], double inv_rf2,
                                              double inv_l, const double (&len)[3],
                                              const double (&ilen)[3], const double* bb, int bs,
                                              const double* mbar, int ms, double (&ub)[kNFit],
                                              double (&xb)[3]) {
  const int64_t N = a.n;
  const Geo q = geometry(a, t, xs, ys, zs, len, ilen, inv_rf2);
  if (!(q.s2 < 1.0)) return false;
  const double sw = 1.0 - q.s2;
  const double wt = a.weight_kind == 1 ? 1.0 : sw * sw;
  double mono[kNMono];
  mls_monos6(q.dx * inv_l, q.dy * inv_l, q.dz * inv_l, mono);
  double p[kNB];
  mls_basis_from_monos(mono, p);
  double Bt[kNB];
  for (int k = 0; k < kNB; ++k) Bt[k] = 0.0;
  for (int fi = 0; fi < kNFit; ++fi) {
    const double du = a.sU[(fi + 1) * N + t] - u[fi + 1];
    double pb = 0.0;
    for (int k = 0; k < kNB; ++k) {
      const double bk = bb[(fi * kNB + k) * bs];
      pb = fma(p[k], bk, pb);
      Bt[k] = fma(du, bk, Bt[k]);
    }
    ub[fi] = wt * pb;
  }
  struct Strided {
    const double* p;
    int st;
    __device__ __forceinline__ double operator[](int k) const { return p[k * st]; }
  };
  double V, Vx, Vy, Vz, P, Px, Py, Pz;
  mls_eval_basis_poly(mono, Bt, V, Vx, Vy, Vz);
  mls_eval_moment_poly(mono, Strided{mbar, ms}, P, Px, Py, Pz);
  const double wbar = P + V;
  const double dwd_c = a.weight_kind == 1 ? 0.0 : -4.0 * inv_rf2;
  const double dw = wbar * dwd_c * sw;  // d w / d d = -4 (1 - s^2) d / r_f^2
  xb[0] = wt * (Px + Vx) * inv_l + dw * q.dx;
  xb[1] = wt * (Py + Vy) * inv_l + dw * q.dy;
  xb[2] = wt * (Pz + Vz) * inv_l + dw * q.dz;
  return true;
}

template <int MODE>
__global__ void __launch_bounds__(kT, 1) k_adjoint(const AdjArgs a) {
  extern __shared__ double sm[];
  const int s = blockIdx.x * kT + threadIdx.x;
  if (s >= a.n) return;
  double* my = sm + threadIdx.x;
  const SCol M{my};                 // normal matrix / factor (190), later mbar (80) + bbar (133)
  const SCol MB{my};                // mbar [80]
  const int64_t N = a.n;
  // c_f, f = 0..6: [f * 19 + k] (in the record for the stored variant)
  double* my_scr = a.scr + static_cast<int64_t>(s) * kScr;
  const GCol cf{MODE == kRecompute ? my_scr + kScrC : a.rec + kRecCoef * N + s,
                MODE == kRecompute ? 1 : N};
  const GCol bbar{my_scr + kScrBbar, 1};          // bbar_f
  double len[3], ilen[3];
  for (int c = 0; c < 3; ++c) {
    len[c] = a.g.len[c];
    ilen[c] = a.g.periodic[c] ? 1.0 / a.g.len[c] : 0.0;
  }
  const double xs = a.spos[s], ys = a.spos[N + s], zs = a.spos[2 * N + s];
  double u[8];
  for (int f = 0; f < 8; ++f) u[f] = a.sU[f * N + s];
  const double lam = a.slam[s];
  const double rf = a.g.rf_factor * lam;
  const double inv_rf2 = 1.0 / (rf * rf);
  const double inv_l = 1.0 / lam;
  const int64_t beg = a.off[s];
  const int64_t end = a.off[s + 1] < a.g.capacity ? a.off[s + 1] : a.g.capacity;
  const int src = a.perm[s];
  const double zeta = a.zeta ? a.zeta[src] : 0.0;
  const double eta = a.eta ? a.eta[src] : 0.0;

  // ---- forward: moments
  int cnt = 0;
  double invd[kNB];
  bool singular;
  if (MODE == kStored) {
    singular = a.rec[kRecFlag * N + s] != 0.0;
    if (!singular) {
      for (int k = 0; k < kNT; ++k) M[k] = a.rec[(kRecFac + k) * N + s];
      for (int k = 0; k < kNB; ++k) invd[k] = a.rec[(kRecInvd + k) * N + s];
    }
  } else {
    double m[kNM];
#pragma unroll
    for (int k = 0; k < kNM; ++k) m[k] = 0.0;
    for (int64_t e = beg; e < end; ++e) {
      const Geo q = geometry(a, a.idx[e], xs, ys, zs, len, ilen, inv_rf2);
      if (!(q.s2 < 1.0)) continue;
      ++cnt;
      const double sw = 1.0 - q.s2;
      const double wt = a.weight_kind == 1 ? 1.0 : sw * sw;
      double qg[kNB], wq[kNB + 1];
      mls_monomials(q.dx * inv_l, q.dy * inv_l, q.dz * inv_l, wt, qg, wq);
      mls_accum_moments(qg, wq, m);
    }
    singular = cnt < kNB;
    if (!singular) mls_assemble(m, M);
  }
  if (MODE != kStored && !singular) {
    const double minpiv = mls_cholesky<double>(M, invd);
    double rmin = 1e300;
    for (int k = 0; k < kNB; ++k) {
      const double r = 1.0 / (invd[k] * invd[k] * M[k * (k + 1) / 2 + k]);
      rmin = r < rmin ? r : rmin;
    }
    singular = !(minpiv > 0.0) || !(rmin > 1e-12);
  }
  if (MODE == kRecord) {
    a.rec[kRecFlag * N + s] = singular ? 1.0 : 0.0;
    if (singular) {
      raise_flag(a.status_word, PHB_FLAG_FIT_SINGULAR);
      return;
    }
    for (int k = 0; k < kNT; ++k) a.rec[(kRecFac + k) * N + s] = M[k];
    for (int k = 0; k < kNB; ++k) a.rec[(kRecInvd + k) * N + s] = invd[k];
  }
  double selfu[8], selfx[3] = {0.0, 0.0, 0.0};
  if (singular) {
    // the forward right-hand side is zero and does not depend on the inputs:
    // no own terms and zero seeds for the gather
    for (int k = 0; k < kNFit * kNB; ++k) my_scr[kScrBbar + k] = 0.0;
    for (int k = 0; k < kNM; ++k) my_scr[kScrMbar + k] = 0.0;
    for (int k = 0; k < 11; ++k) a.self[k * N + s] = 0.0;
    raise_flag(a.status_word, PHB_FLAG_FIT_SINGULAR);
    return;
  }
  // ---- forward: right-hand sides in two groups, full coefficients c_f
  for (int grp = 0; grp < (MODE == kStored ? 0 : 2); ++grp) {
    const int nf = grp == 0 ? 4 : 3;  // fields 1..4 (Vx, Vy, Vz, Bx) then 5..7 (By, Bz, sigma)
    double b[4][kNB];
    for (int f = 0; f < 4; ++f)
      for (int k = 0; k < kNB; ++k) b[f][k] = 0.0;
    for (int64_t e = beg; e < end; ++e) {
      const int t = a.idx[e];
      const Geo q = geometry(a, t, xs, ys, zs, len, ilen, inv_rf2);
      if (!(q.s2 < 1.0)) continue;
      const double sw = 1.0 - q.s2;
      const double wt = a.weight_kind == 1 ? 1.0 : sw * sw;
      double qg[kNB], wq[kNB + 1];
      mls_monomials(q.dx * inv_l, q.dy * inv_l, q.dz * inv_l, wt, qg, wq);
      for (int f = 0; f < nf; ++f) {
        const int uf = 1 + grp * 4 + f;
        mls_accum_rhs(wq, a.sU[uf * N + t] - u[uf], b[f]);
      }
    }
    for (int f = 0; f < nf; ++f) {
      mls_forward(M, invd, b[f]);
      mls_back19(M, invd, b[f]);
      const int fi = grp * 4 + f;  // 0..6 <-> U index 1..7
      for (int k = 0; k < kNB; ++k) cf[fi * kNB + k] = b[f][k];
    }
  }
  if (MODE == kRecord) return;
  double o[8];
  for (int f = 0; f < 8; ++f) o[f] = a.gbar[f * N + src];
  // ---- derivatives, right-hand-side adjoint, cbar -> bbar = M^-1 cbar
  const double il = inv_l, il2 = inv_l * inv_l;
  {
    MhdDerivs<double> D;
    mhd_zero(D);
    for (int fi = 0; fi < kNFit; ++fi) {
      const double g[3] = {cf[fi * kNB + kLin0] * il, cf[fi * kNB + kLin0 + 1] * il,
                           cf[fi * kNB + kLin0 + 2] * il};
      const double h[6] = {2.0 * cf[fi * kNB + kQuad0] * il2, cf[fi * kNB + kQuad0 + 1] * il2,
                           cf[fi * kNB + kQuad0 + 2] * il2, 2.0 * cf[fi * kNB + kQuad0 + 3] * il2,
                           cf[fi * kNB + kQuad0 + 4] * il2, 2.0 * cf[fi * kNB + kQuad0 + 5] * il2};
      mhd_collect(D, fi + 1, g, h);
    }
    double gb[kNFit][3], hb[kNFit][6];
    rhs_adjoint_point(u, D, a.gamma, zeta, eta, lam, a.c_zeta_l, a.c_zeta_a, a.c_eta, o, selfu,
                      gb, hb);
    for (int fi = 0; fi < kNFit; ++fi) {
      double cb[kNB];
      for (int k = 0; k < kQuad0; ++k) cb[k] = 0.0;
      cb[kQuad0] = 2.0 * hb[fi][0] * il2;
      cb[kQuad0 + 1] = hb[fi][1] * il2;
      cb[kQuad0 + 2] = hb[fi][2] * il2;
      cb[kQuad0 + 3] = 2.0 * hb[fi][3] * il2;
      cb[kQuad0 + 4] = hb[fi][4] * il2;
      cb[kQuad0 + 5] = 2.0 * hb[fi][5] * il2;
      cb[kLin0] = gb[fi][0] * il;
      cb[kLin0 + 1] = gb[fi][1] * il;
      cb[kLin0 + 2] = gb[fi][2] * il;
      mls_forward(M, invd, cb);
      mls_back19(M, invd, cb);
      for (int k = 0; k < kNB; ++k) bbar[fi * kNB + k] = cb[k];
    }
  }
  // ---- mbar = fold of -sum_f bbar_f c_f^T onto the moments; stage mbar, bbar
  // in shared memory and keep mbar in the scratch record (over c_f) for the gather
  {
    double mb[kNM];
#pragma unroll
    for (int k = 0; k < kNM; ++k) mb[k] = 0.0;
    for (int fi = 0; fi < kNFit; ++fi) {
      double bb[kNB], cc[kNB];
      for (int k = 0; k < kNB; ++k) {
        bb[k] = bbar[fi * kNB + k];
        cc[k] = cf[fi * kNB + k];
      }
      mls_accum_mbar(bb, cc, mb);
    }
#pragma unroll
    for (int k = 0; k < kNM; ++k) {
      MB[k] = mb[k];
      my_scr[kScrMbar + k] = mb[k];
    }
    for (int k = 0; k < kNFit * kNB; ++k) M[kNM + k] = bbar[k];  // M is dead now
  }
  // ---- backward pass over the neighbours: particle i's own terms
  for (int64_t e = beg; e < end; ++e) {
    const int t = a.idx[e];
    double ub[kNFit], xb[3];
    if (!entry_adjoint(a, t, xs, ys, zs, u, inv_rf2, inv_l, len, ilen, M.p + kNM * kT, kT,
                       MB.p, kT, ub, xb))
      continue;
    for (int fi = 0; fi < kNFit; ++fi) selfu[fi + 1] -= ub[fi];
    for (int c = 0; c < 3; ++c) selfx[c] -= xb[c];
  }
  for (int k = 0; k < 8; ++k) a.self[k * N + s] = selfu[k];
  for (int c = 0; c < 3; ++c) a.self[(8 + c) * N + s] = selfx[c];
}

// ---- reverse neighbour lists: for every particle t, the particles i whose
// list names t, in ascending order of i
__global__ void k_rev_count(int n, int64_t cap, const int64_t* __restrict__ off,
                            const int32_t* __restrict__ idx, int32_t* __restrict__ rcnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t end = off[i + 1] < cap ? off[i + 1] : cap;
  for (int64_t e = off[i]; e < end; ++e) atomicAdd(&rcnt[idx[e]], 1);
}

__global__ void k_rev_fill(int n, int64_t cap, const int64_t* __restrict__ off,
                           const int32_t* __restrict__ idx, const int64_t* __restrict__ roff,
                           int32_t* __restrict__ rcur, int32_t* __restrict__ rsrc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t end = off[i + 1] < cap ? off[i + 1] : cap;
  for (int64_t e = off[i]; e < end; ++e) {
    const int t = idx[e];
    rsrc[roff[t] + atomicAdd(&rcur[t], 1)] = i;
  }
}

__global__ void k_rev_sort(int n, const int64_t* __restrict__ roff, int32_t* __restrict__ rsrc) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int32_t* v = rsrc + roff[t];
  const int m = static_cast<int>(roff[t + 1] - roff[t]);
  for (int i = 1; i < m; ++i) {
    const int32_t x = v[i];
    int j = i - 1;
    while (j >= 0 && v[j] > x) {
      v[j + 1] = v[j];
      --j;
    }
    v[j + 1] = x;
  }
}

// Own terms plus the contribution of every particle i whose list names t,
// recomputed from i's seeds in ascending order of i; caller order out.
__global__ void __launch_bounds__(128) k_adj_gather(const AdjArgs a, const int64_t* __restrict__ roff,
                                                    const int32_t* __restrict__ rsrc,
                                                    double* __restrict__ Ubar,
                                                    double* __restrict__ xbar) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.n) return;
  const int64_t N = a.n;
  double len[3], ilen[3];
  for (int c = 0; c < 3; ++c) {
    len[c] = a.g.len[c];
    ilen[c] = a.g.periodic[c] ? 1.0 / a.g.len[c] : 0.0;
  }
  double acc[11];
  for (int k = 0; k < 11; ++k) acc[k] = a.self[k * N + t];
  for (int64_t r = roff[t]; r < roff[t + 1]; ++r) {
    const int i = rsrc[r];
    double u[8];
    for (int f = 0; f < 8; ++f) u[f] = a.sU[f * N + i];
    const double lam = a.slam[i];
    const double rf = a.g.rf_factor * lam;
    const double* bb = a.scr + static_cast<int64_t>(i) * kScr;
    double ub[kNFit], xb[3];
    if (!entry_adjoint(a, t, a.spos[i], a.spos[N + i], a.spos[2 * N + i], u, 1.0 / (rf * rf),
                       1.0 / lam, len, ilen, bb + kScrBbar, 1, bb + kScrMbar, 1, ub, xb))
      continue;
    for (int k = 0; k < kNFit; ++k) acc[1 + k] += ub[k];
    for (int c = 0; c < 3; ++c) acc[8 + c] += xb[c];
  }
  const int i = a.perm[t];
  for (int k = 0; k < 8; ++k) Ubar[k * N + i] = acc[k];
  for (int c = 0; c < 3; ++c) xbar[c * N + i] = acc[8 + c];
}

}  // namespace
}  // namespace phb

using namespace phb;

namespace {

phb_status adjoint_impl(int mode, const phb_plan* plan, const phb_params* prm, const double* pos,
                        const double* lambda, const double* U, const double* gbar, void* ws,
                        size_t ws_bytes, double* rec, size_t rec_bytes, double* Ubar, double* xbar,
                        int32_t* status_word, cudaStream_t st) {
  phb_status s = check_common(plan, ws, ws_bytes, plan ? plan->ws_off[R_END_ADJ] : 0);
  if (s != PHB_OK) return s;
  if (!prm || !pos || !lambda || !U) return PHB_ERR_INVALID_ARG;
  if (mode != kRecord && (!gbar || !Ubar || !xbar)) return PHB_ERR_INVALID_ARG;
  if (mode != kRecompute && (!rec || rec_bytes < size_t(kRecWords) * 8 * size_t(plan->n)))
    return PHB_ERR_INVALID_ARG;
  if (prm->weight_kind != 0 && prm->weight_kind != 1) return PHB_ERR_INVALID_ARG;
  if (!(prm->gamma > 1.0)) return PHB_ERR_INVALID_ARG;
  const Grid g = make_grid(plan);
  const int n = g.n;
  cudaError_t e = gather_sorted(plan, g, pos, lambda, U, ws, status_word, st);
  if (e) return launch_status(e);
  AdjArgs a;
  a.g = g;
  a.n = n;
  a.perm = region<int32_t>(plan, ws, R_PERM);
  a.spos = region<double>(plan, ws, R_SPOS);
  a.slam = region<double>(plan, ws, R_SLAM);
  a.sU = region<double>(plan, ws, R_SU);
  a.off = region<int64_t>(plan, ws, R_OFF);
  a.idx = region<int32_t>(plan, ws, R_IDX);
  a.gbar = gbar;
  a.gamma = prm->gamma;
  a.weight_kind = prm->weight_kind;
  a.zeta = prm->zeta;
  a.eta = prm->eta;
  a.c_zeta_l = prm->c_zeta_l;
  a.c_zeta_a = prm->c_zeta_a;
  a.c_eta = prm->c_eta;
  a.scr = region<double>(plan, ws, R_ADJ_SCR);
  a.self = region<double>(plan, ws, R_ADJ_SELF);
  a.rec = rec;
  a.status_word = status_word;
  const size_t smem = size_t(kSm) * kT * sizeof(double);
  const unsigned grid = static_cast<unsigned>((n + kT - 1) / kT);
  if (mode == kRecompute) {
    cudaFuncSetAttribute(k_adjoint<kRecompute>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    k_adjoint<kRecompute><<<grid, kT, smem, st>>>(a);
  } else if (mode == kRecord) {
    cudaFuncSetAttribute(k_adjoint<kRecord>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    k_adjoint<kRecord><<<grid, kT, smem, st>>>(a);
    note_launch();
    return launch_status(cudaSuccess);
  } else {
    cudaFuncSetAttribute(k_adjoint<kStored>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         static_cast<int>(smem));
    k_adjoint<kStored><<<grid, kT, smem, st>>>(a);
  }
  note_launch();
  int32_t* rcnt = region<int32_t>(plan, ws, R_ADJ_RCNT);
  int64_t* roff = region<int64_t>(plan, ws, R_ADJ_ROFF);
  int32_t* rsrc = region<int32_t>(plan, ws, R_ADJ_RSRC);
  int64_t* bsum = region<int64_t>(plan, ws, R_SCAN);
  const int64_t cap = plan->nbr_capacity;
  const unsigned nb = static_cast<unsigned>((n + kThreads - 1) / kThreads);
  if ((e = cudaMemsetAsync(rcnt, 0, (n + 1) * sizeof(int32_t), st))) return launch_status(e);
  k_rev_count<<<nb, kThreads, 0, st>>>(n, cap, a.off, a.idx, rcnt);
  note_launch();
  if ((e = scan_exclusive_i32_to_i64(rcnt, roff, n + 1, bsum, st))) return launch_status(e);
  if ((e = cudaMemsetAsync(rcnt, 0, (n + 1) * sizeof(int32_t), st))) return launch_status(e);
  k_rev_fill<<<nb, kThreads, 0, st>>>(n, cap, a.off, a.idx, roff, rcnt, rsrc);
  note_launch();
  k_rev_sort<<<nb, kThreads, 0, st>>>(n, roff, rsrc);
  note_launch();
  k_adj_gather<<<static_cast<unsigned>((n + 127) / 128), 128, 0, st>>>(a, roff, rsrc, Ubar, xbar);
  note_launch();
  return launch_status(cudaSuccess);
}

}  // namespace

extern "C" phb_status phb_rhs_adjoint(const phb_plan* plan, const phb_params* prm, const double* pos,
                                      const double* lambda, const double* U, const double* gbar,
                                      void* ws, size_t ws_bytes, double* Ubar, double* xbar,
                                      int32_t* status_word, phb_stream_t stream) {
  return adjoint_impl(kRecompute, plan, prm, pos, lambda, U, gbar, ws, ws_bytes, nullptr, 0, Ubar,
                      xbar, status_word, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" size_t phb_adjoint_record_bytes(const phb_plan* plan) {
  return plan && plan->n > 0 ? size_t(kRecWords) * 8 * size_t(plan->n) : 0;
}

extern "C" phb_status phb_adjoint_record(const phb_plan* plan, const phb_params* prm,
                                         const double* pos, const double* lambda, const double* U,
                                         void* ws, size_t ws_bytes, double* record,
                                         size_t record_bytes, int32_t* status_word,
                                         phb_stream_t stream) {
  return adjoint_impl(kRecord, plan, prm, pos, lambda, U, nullptr, ws, ws_bytes, record,
                      record_bytes, nullptr, nullptr, status_word,
                      reinterpret_cast<cudaStream_t>(stream));
}

extern "C" phb_status phb_rhs_adjoint_stored(const phb_plan* plan, const phb_params* prm,
                                             const double* pos, const double* lambda,
                                             const double* U, const double* gbar, void* ws,
                                             size_t ws_bytes, const double* record,
                                             size_t record_bytes, double* Ubar, double* xbar,
                                             int32_t* status_word, phb_stream_t stream) {
  return adjoint_impl(kStored, plan, prm, pos, lambda, U, gbar, ws, ws_bytes,
                      const_cast<double*>(record), record_bytes, Ubar, xbar, status_word,
                      reinterpret_cast<cudaStream_t>(stream));
}
