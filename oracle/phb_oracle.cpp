// Phurbas particle right-hand side: plain FP64 CPU oracle.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
// restatement of the method that the CUDA library is checked against.  Only
// tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference arm
// may load it.  It shares no code, header or table with the CUDA library.
//
// What it computes (Phurbas Paper II, Sec. 2 summary of the Paper I method):
//   * neighbours: strict fixed-radius set N(i) = { j != i : |x_j - x_i| < r_f,i },
//     r_f,i = 2.3 lambda_i, radius of the gathering particle, not mutual
//     (Sec. 2 and Sec. 2.1, "strict radius-based neighbor search");
//     brute force over all particles, FP64 in one fixed order, no FMA;
//   * fit: local third-order polynomial moving-least-squares fit, interpolating
//     (constant term pinned to particle i's own value, Acknowledgements), to
//     rho, V, B, sigma, solved as a weighted linear least-squares problem by
//     Householder QR of diag(sqrt w) P (textbook; no normal equations);
//   * derivatives from the fitted coefficients;
//   * ideal-MHD Lagrangian time derivatives with bulk viscosity and a
//     diffusive div B term (Sec. 2; App. A equations of motion);
//   * the second-order predictor-corrector read as Heun's method (Sec. 2,
//     Sec. 4.2 "explicit Hermitian time integration");
//   * a forward-mode (dual number) derivative of the right-hand side with the
//     neighbour sets frozen, used to pin the hand-written reverse-mode adjoint;
//   * individual power-of-two time-step levels with the spatial limiter
//     (Sec. 2: steps independent of the bulk velocity, spatial variation
//     limited; Sec. 2.1: rounded down to powers of two, information flows
//     from a particle to its neighbours);
//   * the particle adaptivity scan: voids found on a 9^3 grid of test points
//     around each particle and clumps of too-close particles (Sec. 2,
//     Sec. 2.1), with thresholds that are readings.
//
// Readings where the paper defers to Paper I:
//   weight w = (1 - s^2)^2 with s = |d| / r_f,i (or w = 1);
//   basis = the 19 monomials of total degree 1..3 in q = d / lambda_i,
//   graded-lexicographic order x y z xx xy xz yy yz zz xxx xxy xxz xyy xyz xzz
//   yyy yyz yzz zzz;
//   P = (gamma - 1) sigma;  mu_0 = 1 units (V_A^2 = B^2 / rho, App. A);
//   bulk viscosity zeta and div B diffusivity eta are per-particle inputs,
//   plus optional coefficient laws for the two bulk-viscosity fields and the
//   div B diffusivity (Sec. 2 states only what they do; Paper I's forms are
//   not available): with the fast-speed bound c = sqrt((gamma P + |B|^2)/rho)
//     zeta = zeta_in + C_l lambda c + C_a lambda^2 max(0, -div V)
//     eta  = eta_in  + C_eta lambda c
//   (C_l: damping at the resolution scale at the signal speed; C_a: damping
//   that grows with compression, as at shocks; C_eta: div B diffusion at the
//   resolution scale).
//
// Build: g++ -O2 -std=c++17 -fopenmp -ffp-contract=off -fPIC -shared.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>

namespace {

constexpr int NB = 19;  // basis size of the interpolating cubic fit
constexpr int NF = 8;   // fields rho, Vx, Vy, Vz, Bx, By, Bz, sigma

struct Box {
  double lo[3];
  double len[3];
  int32_t periodic[3];
};

struct Params {
  double gamma;
  double rf_factor;     // r_f = rf_factor * lambda (2.3 in the paper)
  int32_t weight_kind;  // 0: (1 - s^2)^2, 1: unweighted
  int32_t pad;
  const double* zeta;   // [n] or null (0)
  const double* eta;    // [n] or null (0)
  const uint8_t* frozen;  // [n] or null: nonzero = no time evolution (pc_step only)
  double c_zeta_l;        // coefficient laws (0 = off), see the header
  double c_zeta_a;
  double c_eta;
};

// ---------------------------------------------------------------- dual numbers
struct Dual {
  double v, d;
  Dual() : v(0), d(0) {}
  Dual(double a) : v(a), d(0) {}
  Dual(double a, double b) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) {
  double q = a.v / b.v;
  return Dual(q, (a.d - q * b.d) / b.v);
}
inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
inline Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
inline Dual sqrt(Dual a) {
  double r = std::sqrt(a.v);
  return Dual(r, r > 0 ? a.d / (2 * r) : 0.0);
}
inline double val(double a) { return a; }
inline double val(Dual a) { return a.v; }
inline double fabs_val(double a) { return std::fabs(a); }
inline double fabs_val(Dual a) { return std::fabs(a.v); }
// x with its value replaced by v (its tangent, if any, kept)
inline double with_value(double, double v) { return v; }
inline Dual with_value(Dual x, double v) { return Dual(v, x.d); }
using std::sqrt;

// ---------------------------------------------------------------- geometry
// Minimum-image offset on a periodic axis: d - len * nearbyint(d / len).
inline double min_image(double d, double len, int periodic) {
  if (periodic) d = d - len * std::nearbyint(d / len);
  return d;
}

// Exact FP64 membership test, evaluated in exactly this order:
//   ((dx*dx + dy*dy) + dz*dz) < r*r   (strict), r = rf_factor*lambda_i + skin.
inline bool is_neighbor(const Box& box, const double* pos, int64_t n, int64_t i, int64_t j,
                        double r) {
  double dx = min_image(pos[0 * n + j] - pos[0 * n + i], box.len[0], box.periodic[0]);
  double dy = min_image(pos[1 * n + j] - pos[1 * n + i], box.len[1], box.periodic[1]);
  double dz = min_image(pos[2 * n + j] - pos[2 * n + i], box.len[2], box.periodic[2]);
  double d2 = (dx * dx + dy * dy) + dz * dz;
  return d2 < r * r;
}

// The 19 basis monomials of total degree 1..3 at q (graded-lex order).
template <class T>
void basis(const T q[3], T p[NB]) {
  const T x = q[0], y = q[1], z = q[2];
  p[0] = x; p[1] = y; p[2] = z;
  p[3] = x * x; p[4] = x * y; p[5] = x * z; p[6] = y * y; p[7] = y * z; p[8] = z * z;
  p[9] = x * x * x; p[10] = x * x * y; p[11] = x * x * z; p[12] = x * y * y;
  p[13] = x * y * z; p[14] = x * z * z; p[15] = y * y * y; p[16] = y * y * z;
  p[17] = y * z * z; p[18] = z * z * z;
}

// Weighted least squares  min_c sum_j w_j (p_j . c - r_j)^2  for NF right-hand
// sides at once, by Householder QR of A = diag(sqrt w) P (rows j, n x 19) and
// the same reflections applied to Bm = diag(sqrt w) R (n x 8).  Returns false
// (singular) when n < 19 or some |R_kk| <= 1e-13 max_k |R_kk|.
template <class T>
bool wls_qr(int n, std::vector<T>& A, std::vector<T>& Bm, T C[NB * NF]) {
  for (int k = 0; k < NB * NF; ++k) C[k] = T(0.0);
  if (n < NB) return false;
  for (int k = 0; k < NB; ++k) {
    T norm2 = T(0.0);
    for (int r = k; r < n; ++r) norm2 += A[r * NB + k] * A[r * NB + k];
    T norm = sqrt(norm2);
    if (val(norm) == 0.0) continue;
    T alpha = val(A[k * NB + k]) > 0 ? -norm : norm;
    // v = a_k - alpha e_k  (stored in place below the diagonal, v_k separately)
    T vk = A[k * NB + k] - alpha;
    T vnorm2 = vk * vk;
    for (int r = k + 1; r < n; ++r) vnorm2 += A[r * NB + k] * A[r * NB + k];
    if (val(vnorm2) == 0.0) { A[k * NB + k] = alpha; continue; }
    auto reflect = [&](std::vector<T>& M, int ncol, int col) {
      T dot = vk * M[k * ncol + col];
      for (int r = k + 1; r < n; ++r) dot += A[r * NB + k] * M[r * ncol + col];
      T f = (dot + dot) / vnorm2;
      M[k * ncol + col] -= f * vk;
      for (int r = k + 1; r < n; ++r) M[r * ncol + col] -= f * A[r * NB + k];
    };
    for (int c = k + 1; c < NB; ++c) reflect(A, NB, c);
    for (int c = 0; c < NF; ++c) reflect(Bm, NF, c);
    A[k * NB + k] = alpha;
  }
  double rmax = 0.0;
  for (int k = 0; k < NB; ++k) rmax = std::max(rmax, fabs_val(A[k * NB + k]));
  for (int k = 0; k < NB; ++k)
    if (!(fabs_val(A[k * NB + k]) > 1e-13 * rmax)) return false;
  // back substitution R c = (Q^T Bm)[0:19]
  for (int f = 0; f < NF; ++f) {
    for (int k = NB - 1; k >= 0; --k) {
      T s = Bm[k * NF + f];
      for (int c = k + 1; c < NB; ++c) s -= A[k * NB + c] * C[c * NF + f];
      C[k * NF + f] = s / A[k * NB + k];
    }
  }
  return true;
}

// Fit all 8 fields at particle i and return gradients [8][3] and Hessians
// [8][6] (xx, xy, xz, yy, yz, zz).  pos, U carry tangents when T = Dual.
template <class T>
int fit_particle(const Box& box, int64_t n, const T* pos, const double* lam, const T* U,
                 const Params& prm, int64_t i, const int64_t* nb, int64_t nn, T grad[NF][3],
                 T hess[NF][6]) {
  const double li = lam[i];
  const double rf = prm.rf_factor * li;
  std::vector<T> A(std::max<int64_t>(nn, 1) * NB), Bm(std::max<int64_t>(nn, 1) * NF);
  for (int64_t a = 0; a < nn; ++a) {
    const int64_t j = nb[a];
    T d[3];
    for (int ax = 0; ax < 3; ++ax) {
      T diff = pos[ax * n + j] - pos[ax * n + i];
      // the image shift is a constant multiple of the box length
      d[ax] = with_value(diff, min_image(val(diff), box.len[ax], box.periodic[ax]));
    }
    T r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
    T s2 = r2 / T(rf * rf);
    T sw = prm.weight_kind == 1 ? T(1.0) : (T(1.0) - s2);  // sqrt of (1 - s^2)^2
    T q[3] = {d[0] / T(li), d[1] / T(li), d[2] / T(li)};
    T p[NB];
    basis(q, p);
    for (int c = 0; c < NB; ++c) A[a * NB + c] = sw * p[c];
    for (int f = 0; f < NF; ++f) Bm[a * NF + f] = sw * (U[f * n + j] - U[f * n + i]);
  }
  T C[NB * NF];
  bool ok = wls_qr<T>(static_cast<int>(nn), A, Bm, C);
  const T il = T(1.0 / li), il2 = T(1.0 / (li * li));
  for (int f = 0; f < NF; ++f) {
    grad[f][0] = C[0 * NF + f] * il;
    grad[f][1] = C[1 * NF + f] * il;
    grad[f][2] = C[2 * NF + f] * il;
    hess[f][0] = T(2.0) * C[3 * NF + f] * il2;
    hess[f][1] = C[4 * NF + f] * il2;
    hess[f][2] = C[5 * NF + f] * il2;
    hess[f][3] = T(2.0) * C[6 * NF + f] * il2;
    hess[f][4] = C[7 * NF + f] * il2;
    hess[f][5] = T(2.0) * C[8 * NF + f] * il2;
  }
  return ok ? 0 : 1;
}

// Hessian entry (a, b) from the packed [xx, xy, xz, yy, yz, zz] layout.
inline int hidx(int a, int b) {
  static const int t[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  return t[a][b];
}

// Ideal-MHD Lagrangian time derivatives at one particle from its point values
// and fitted derivatives (Sec. 2; App. A with the readings listed above):
//   Drho/Dt   = -rho div V
//   DV/Dt     = [-(gamma-1) grad sigma + (curl B) x B] / rho + zeta grad(div V)
//   DB/Dt     = (B . grad) V - B div V + eta grad(div B)
//   Dsigma/Dt = -gamma sigma div V + rho zeta (div V)^2
template <class T>
void mhd_rhs_point(const T u[NF], const T g[NF][3], const T h[NF][6], double gamma, T zeta,
                   T eta, T out[NF]) {
  const T rho = u[0], sig = u[7];
  const T B[3] = {u[4], u[5], u[6]};
  T divV = g[1][0] + g[2][1] + g[3][2];
  T gdivV[3], gdivB[3];
  for (int a = 0; a < 3; ++a) {
    gdivV[a] = h[1][hidx(a, 0)] + h[2][hidx(a, 1)] + h[3][hidx(a, 2)];
    gdivB[a] = h[4][hidx(a, 0)] + h[5][hidx(a, 1)] + h[6][hidx(a, 2)];
  }
  // J = curl B ;  g[4+c][b] = d B_c / d x_b
  T J[3] = {g[6][1] - g[5][2], g[4][2] - g[6][0], g[5][0] - g[4][1]};
  T F[3] = {J[1] * B[2] - J[2] * B[1], J[2] * B[0] - J[0] * B[2], J[0] * B[1] - J[1] * B[0]};
  out[0] = -rho * divV;
  for (int a = 0; a < 3; ++a) {
    out[1 + a] = (T(-(gamma - 1.0)) * g[7][a] + F[a]) / rho + zeta * gdivV[a];
    T adv = B[0] * g[1 + a][0] + B[1] * g[1 + a][1] + B[2] * g[1 + a][2];
    out[4 + a] = adv - B[a] * divV + eta * gdivB[a];
  }
  out[7] = T(-gamma) * sig * divV + rho * zeta * divV * divV;
}

template <class T>
int rhs_particle(const Box& box, int64_t n, const T* pos, const double* lam, const T* U,
                 const Params& prm, int64_t i, const int64_t* nb, int64_t nn, T out[NF]) {
  T g[NF][3], h[NF][6], u[NF];
  int st = fit_particle<T>(box, n, pos, lam, U, prm, i, nb, nn, g, h);
  for (int f = 0; f < NF; ++f) u[f] = U[f * n + i];
  T zeta = T(prm.zeta ? prm.zeta[i] : 0.0);
  T eta = T(prm.eta ? prm.eta[i] : 0.0);
  if (prm.c_zeta_l != 0.0 || prm.c_zeta_a != 0.0 || prm.c_eta != 0.0) {
    // coefficient laws (see the header): fast-speed bound and compression
    const T P = T(prm.gamma - 1.0) * u[7];
    const T c = sqrt((T(prm.gamma) * P + u[4] * u[4] + u[5] * u[5] + u[6] * u[6]) / u[0]);
    const T divV = g[1][0] + g[2][1] + g[3][2];
    const T l = T(lam[i]);
    zeta = zeta + T(prm.c_zeta_l) * l * c;
    if (val(divV) < 0.0) zeta = zeta - T(prm.c_zeta_a) * l * l * divV;
    eta = eta + T(prm.c_eta) * l * c;
  }
  mhd_rhs_point<T>(u, g, h, prm.gamma, zeta, eta, out);
  return st;
}

}  // namespace

extern "C" {

int orc_version() { return 1; }

// Brute-force neighbour lists for the query particles qidx[0..nq): for each,
// every j != i with ((dx*dx+dy*dy)+dz*dz) < r*r, r = rf_factor*lambda_i + skin,
// in increasing j.  CSR output off[nq+1], idx[cap].  Returns 0, or -1 when
// cap is too small (off is complete in that case, idx is not).
int orc_neighbors(const Box* box, int64_t n, const double* pos, const double* lam,
                  double rf_factor, double skin, int64_t nq, const int64_t* qidx, int64_t* off,
                  int64_t* idx, int64_t cap) {
  std::vector<int64_t> cnt(nq);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t a = 0; a < nq; ++a) {
    const int64_t i = qidx[a];
    const double r = rf_factor * lam[i] + skin;
    int64_t c = 0;
    for (int64_t j = 0; j < n; ++j)
      if (j != i && is_neighbor(*box, pos, n, i, j, r)) ++c;
    cnt[a] = c;
  }
  off[0] = 0;
  for (int64_t a = 0; a < nq; ++a) off[a + 1] = off[a] + cnt[a];
  if (off[nq] > cap) return -1;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t a = 0; a < nq; ++a) {
    const int64_t i = qidx[a];
    const double r = rf_factor * lam[i] + skin;
    int64_t c = off[a];
    for (int64_t j = 0; j < n; ++j)
      if (j != i && is_neighbor(*box, pos, n, i, j, r)) idx[c++] = j;
  }
  return 0;
}

// MLS derivatives of all 8 fields for the query particles, with given
// neighbour lists (CSR over the query list).  grad [8][3][nq], hess [8][6][nq]
// (may be null), status [nq]: 0 ok, 1 singular (derivatives set to 0).
int orc_mls_derivs(const Box* box, int64_t n, const double* pos, const double* lam,
                   const double* U, const Params* prm, int64_t nq, const int64_t* qidx,
                   const int64_t* off, const int64_t* idx, double* grad, double* hess,
                   int32_t* status) {
  int64_t nsing = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : nsing)
  for (int64_t a = 0; a < nq; ++a) {
    double g[NF][3], h[NF][6];
    int st = fit_particle<double>(*box, n, pos, lam, U, *prm, qidx[a], idx + off[a],
                                  off[a + 1] - off[a], g, h);
    for (int f = 0; f < NF; ++f) {
      for (int c = 0; c < 3; ++c) grad[(f * 3 + c) * nq + a] = g[f][c];
      if (hess)
        for (int c = 0; c < 6; ++c) hess[(f * 6 + c) * nq + a] = h[f][c];
    }
    if (status) status[a] = st;
    nsing += st;
  }
  return static_cast<int>(nsing > 0);
}

// Time derivatives dudt [8][nq] for the query particles (fit + RHS).
int orc_mhd_rhs(const Box* box, int64_t n, const double* pos, const double* lam, const double* U,
                const Params* prm, int64_t nq, const int64_t* qidx, const int64_t* off,
                const int64_t* idx, double* dudt, int32_t* status) {
  int64_t nsing = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : nsing)
  for (int64_t a = 0; a < nq; ++a) {
    double out[NF];
    int st = rhs_particle<double>(*box, n, pos, lam, U, *prm, qidx[a], idx + off[a],
                                  off[a + 1] - off[a], out);
    for (int f = 0; f < NF; ++f) dudt[f * nq + a] = out[f];
    if (status) status[a] = st;
    nsing += st;
  }
  return static_cast<int>(nsing > 0);
}

// Forward-mode derivative of the time derivatives along (dpos, dU) with the
// neighbour sets frozen: dudt [8][nq] and its directional derivative
// ddudt [8][nq].
int orc_rhs_jvp(const Box* box, int64_t n, const double* pos, const double* lam, const double* U,
                const double* dpos, const double* dU, const Params* prm, int64_t nq,
                const int64_t* qidx, const int64_t* off, const int64_t* idx, double* dudt,
                double* ddudt) {
  std::vector<Dual> P(3 * n), V(NF * n);
  for (int64_t k = 0; k < 3 * n; ++k) P[k] = Dual(pos[k], dpos ? dpos[k] : 0.0);
  for (int64_t k = 0; k < NF * n; ++k) V[k] = Dual(U[k], dU ? dU[k] : 0.0);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t a = 0; a < nq; ++a) {
    Dual out[NF];
    rhs_particle<Dual>(*box, n, P.data(), lam, V.data(), *prm, qidx[a], idx + off[a],
                       off[a + 1] - off[a], out);
    for (int f = 0; f < NF; ++f) {
      dudt[f * nq + a] = out[f].v;
      ddudt[f * nq + a] = out[f].d;
    }
  }
  return 0;
}

// One Heun (second-order predictor-corrector) step of all n particles, in
// place, with brute-force neighbour sets at x^n and again at x^p:
//   Y^p = Y^n + dt F(Y^n);   Y^{n+1} = Y^n + dt/2 (F(Y^n) + F(Y^p)),
// Y = (x, U), dx/dt = V, lambda unchanged; particles marked frozen keep their
// Y (the fixed-value boundaries of the Sec. 3 annulus test).  O(n^2): small n
// only.  Returns the number of singular fits seen in either stage.
int orc_pc_step(const Box* box, int64_t n, double* pos, const double* lam, double* U, double dt,
                const Params* prm) {
  std::vector<int64_t> all(n);
  for (int64_t i = 0; i < n; ++i) all[i] = i;
  auto eval = [&](const double* x, const double* u, double* F, int64_t& nsing) {
    std::vector<int64_t> off(n + 1);
    // count, then fill
    std::vector<int64_t> dummy(1);
    orc_neighbors(box, n, x, lam, prm->rf_factor, 0.0, n, all.data(), off.data(), dummy.data(), 0);
    std::vector<int64_t> idx(std::max<int64_t>(off[n], 1));
    orc_neighbors(box, n, x, lam, prm->rf_factor, 0.0, n, all.data(), off.data(), idx.data(),
                  off[n]);
    std::vector<int32_t> st(n);
    orc_mhd_rhs(box, n, x, lam, u, prm, n, all.data(), off.data(), idx.data(), F, st.data());
    for (int64_t i = 0; i < n; ++i) nsing += st[i];
  };
  int64_t nsing = 0;
  // frozen particles (fixed-value boundaries) keep x and U through both stages
  auto moving = [&](int64_t i) { return !(prm->frozen && prm->frozen[i]); };
  std::vector<double> F0(NF * n), F1(NF * n), xp(3 * n), up(NF * n);
  eval(pos, U, F0.data(), nsing);
  for (int ax = 0; ax < 3; ++ax)
    for (int64_t i = 0; i < n; ++i)
      xp[ax * n + i] = pos[ax * n + i] + (moving(i) ? dt * U[(1 + ax) * n + i] : 0.0);
  for (int f = 0; f < NF; ++f)
    for (int64_t i = 0; i < n; ++i)
      up[f * n + i] = U[f * n + i] + (moving(i) ? dt * F0[f * n + i] : 0.0);
  eval(xp.data(), up.data(), F1.data(), nsing);
  for (int ax = 0; ax < 3; ++ax)
    for (int64_t i = 0; i < n; ++i)
      if (moving(i)) pos[ax * n + i] += 0.5 * dt * (U[(1 + ax) * n + i] + up[(1 + ax) * n + i]);
  for (int f = 0; f < NF; ++f)
    for (int64_t i = 0; i < n; ++i)
      if (moving(i)) U[f * n + i] += 0.5 * dt * (F0[f * n + i] + F1[f * n + i]);
  return static_cast<int>(nsing);
}

// Individual time-step levels (Sec. 2, Sec. 2.1).  Readings: the Courant
// step of particle i is dt_i = cfl lambda_i / c_i with the fast magnetosonic
// bound c_i = sqrt((gamma P_i + |B_i|^2) / rho_i) (no bulk velocity, mu_0 = 1),
// evaluated as  B2 = (Bx*Bx + By*By) + Bz*Bz,  c2 = (gamma*P + B2) / rho,
// dt = (cfl*lambda) / sqrt(c2)  in FP64 without contraction.  Its level is
// the smallest L >= 0 with dt_max / 2^L <= dt_i (the step rounded down to a
// power of two of dt_max), capped at max_level.  The limiter then sends each
// particle's level to its neighbours: for every i and every j in N(i),
// L_j >= L_i - 1, applied once from the unlimited levels:
//   L_j = max(L0_j, max_{i : j in N(i)} (L0_i - 1)).
// Lists are CSR over all particles (nq = n, query i = i).  levels [n].
// Returns 0, or 1 for a non-positive dt_max / cfl or a non-physical state.
int orc_timestep_levels(int64_t n, const double* lam, const double* U, double gamma, double cfl,
                        double dt_max, int32_t max_level, const int64_t* off, const int64_t* idx,
                        int32_t* levels) {
  if (!(dt_max > 0.0) || !(cfl > 0.0) || max_level < 0) return 1;
  std::vector<int32_t> L0(n);
  int bad = 0;
  for (int64_t i = 0; i < n; ++i) {
    const double rho = U[i], sig = U[7 * n + i];
    const double bx = U[4 * n + i], by = U[5 * n + i], bz = U[6 * n + i];
    const double P = (gamma - 1.0) * sig;
    const double B2 = (bx * bx + by * by) + bz * bz;
    const double c2 = (gamma * P + B2) / rho;
    if (!(rho > 0.0) || !(c2 > 0.0)) bad = 1;
    const double dt = (cfl * lam[i]) / std::sqrt(c2);
    int32_t L = 0;
    while (L < max_level && std::ldexp(dt_max, -L) > dt) ++L;
    L0[i] = L;
  }
  for (int64_t j = 0; j < n; ++j) levels[j] = L0[j];
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = off[i]; e < off[i + 1]; ++e) {
      const int64_t j = idx[e];
      if (L0[i] - 1 > levels[j]) levels[j] = L0[i] - 1;
    }
  return bad;
}

// Particle adaptivity scan (Sec. 2: particles are added in voids and deleted
// in clumps so that every sphere of radius r_f stays well sampled; Sec. 2.1:
// the void search measures distances from the points of a 9^3 grid to the
// neighbour particles and drops every point found close to one; the
// thresholds are Paper I's and are readings here).  For every particle i
// with lists N(i) of the strict r_f sets (CSR over all particles):
//   grid: o_k = h (kx, ky, kz), kx, ky, kz in -4..4, h = (rf_factor lambda_i) / 4,
//     grid index k = ((kx + 4) * 9 + (ky + 4)) * 9 + (kz + 4);
//   test points: those with |o_k|^2 < (r_f - d_v)^2, d_v = void_factor
//     lambda_i, so that every particle within d_v of a test point is i or in
//     N(i) (triangle inequality);
//   a test point is covered when some j in {i} + N(i) has
//     |(x_j - x_i) - o_k|^2 < d_v^2  (minimum image, FP64, this order);
//   void_count[i] = number of uncovered test points; best[i] = the uncovered
//     point whose smallest squared distance to {i} + N(i) is largest (lowest
//     k on ties), -1 when none; cand[3][n] = x_i + o_best (unwrapped);
//   clump[i] = 1 when some j in N(i) with j < i has |x_j - x_i|^2 <
//     (clump_factor lambda_i)^2: of two particles closer than that the one
//     with the larger index is marked for deletion.
// For the query particles q[0..nq) with their lists at off[a]..off[a+1];
// outputs indexed by a (cand [3][nq]).  Returns the number with a void.
int64_t orc_adapt_scan(const Box* box, int64_t n, const double* pos, const double* lam,
                       double rf_factor, double void_factor, double clump_factor, int64_t nq,
                       const int64_t* q, const int64_t* off, const int64_t* idx,
                       int32_t* void_count, int32_t* best, double* cand, int32_t* clump) {
  int64_t with_void = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : with_void)
  for (int64_t a = 0; a < nq; ++a) {
    const int64_t i = q[a];
    const double r = rf_factor * lam[i];
    const double h = r * 0.25;
    const double dv = void_factor * lam[i];
    const double dv2 = dv * dv;
    const double rin = r - dv;
    const double dc = clump_factor * lam[i];
    // offsets of the particle itself and its neighbours
    std::vector<double> d;
    d.reserve(3 * (off[a + 1] - off[a] + 1));
    d.push_back(0.0); d.push_back(0.0); d.push_back(0.0);
    int32_t cl = 0;
    for (int64_t e = off[a]; e < off[a + 1]; ++e) {
      const int64_t j = idx[e];
      double o[3];
      for (int a = 0; a < 3; ++a)
        o[a] = min_image(pos[a * n + j] - pos[a * n + i], box->len[a], box->periodic[a]);
      for (int a = 0; a < 3; ++a) d.push_back(o[a]);
      const double dd = (o[0] * o[0] + o[1] * o[1]) + o[2] * o[2];
      if (j < i && dd < dc * dc) cl = 1;
    }
    const int64_t m = static_cast<int64_t>(d.size() / 3);
    int32_t cnt = 0, bk = -1;
    double bclear = -1.0;
    for (int kx = -4; kx <= 4; ++kx)
      for (int ky = -4; ky <= 4; ++ky)
        for (int kz = -4; kz <= 4; ++kz) {
          const double ox = kx * h, oy = ky * h, oz = kz * h;
          if (!((ox * ox + oy * oy) + oz * oz < rin * rin)) continue;
          double mind = 1e300;
          for (int64_t t = 0; t < m; ++t) {
            const double ex = d[3 * t] - ox, ey = d[3 * t + 1] - oy, ez = d[3 * t + 2] - oz;
            const double e2 = (ex * ex + ey * ey) + ez * ez;
            if (e2 < mind) mind = e2;
          }
          if (mind < dv2) continue;
          ++cnt;
          const int32_t k = ((kx + 4) * 9 + (ky + 4)) * 9 + (kz + 4);
          if (mind > bclear) {
            bclear = mind;
            bk = k;
          }
        }
    void_count[a] = cnt;
    best[a] = bk;
    clump[a] = cl;
    if (bk >= 0) {
      const int kx = bk / 81 - 4, ky = (bk / 9) % 9 - 4, kz = bk % 9 - 4;
      cand[a] = pos[i] + kx * h;
      cand[nq + a] = pos[n + i] + ky * h;
      cand[2 * nq + a] = pos[2 * n + i] + kz * h;
      ++with_void;
    } else {
      cand[a] = cand[nq + a] = cand[2 * nq + a] = 0.0;
    }
  }
  return with_void;
}

}  // extern "C"
