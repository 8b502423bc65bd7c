// Ideal-MHD Lagrangian time derivatives at one particle from its point values
// and MLS derivatives (Paper II Sec. 2; App. A equations of motion), mu_0 = 1:
//   Drho/Dt   = -rho div V
//   DV/Dt     = [-(gamma - 1) grad sigma + (curl B) x B] / rho + zeta grad(div V)
//   DB/Dt     = (B . grad) V - B div V + eta grad(div B)
//   Dsigma/Dt = -gamma sigma div V + rho zeta (div V)^2
// (bulk viscosity of Sec. 2 with a per-particle coefficient zeta, taken
// locally constant; diffusive div B correction with coefficient eta; the
// heating term makes the viscous force conserve total energy).
#pragma once

namespace phb {

// Derivatives the right-hand side needs, gathered from the per-field fits.
template <typename T>
struct MhdDerivs {
  T gs[3];      // grad sigma
  T gV[3][3];   // gV[a][b] = d V_a / d x_b
  T gB[3][3];   // gB[a][b] = d B_a / d x_b
  T gdivV[3];   // d/dx_a (div V) = sum_b d^2 V_b / dx_a dx_b
  T gdivB[3];
};

// Hessian packing (xx, xy, xz, yy, yz, zz) -> (a, b)
__host__ __device__ __forceinline__ int hpack(int a, int b) {
  return a == b ? (a == 0 ? 0 : (a == 1 ? 3 : 5)) : (a + b == 1 ? 1 : (a + b == 2 ? 2 : 4));
}

// Record the derivatives of field f (0..7) given its gradient g[3] and packed
// Hessian h[6].
template <typename T>
__device__ __forceinline__ void mhd_collect(MhdDerivs<T>& D, int f, const T (&g)[3], const T (&h)[6]) {
  if (f == 7) {
    D.gs[0] = g[0]; D.gs[1] = g[1]; D.gs[2] = g[2];
  } else if (f >= 1 && f <= 3) {
    const int c = f - 1;  // V component
    D.gV[c][0] = g[0]; D.gV[c][1] = g[1]; D.gV[c][2] = g[2];
    // contribution of d^2 V_c / dx_a dx_c to d/dx_a (div V)
    D.gdivV[0] += h[hpack(0, c)];
    D.gdivV[1] += h[hpack(1, c)];
    D.gdivV[2] += h[hpack(2, c)];
  } else if (f >= 4 && f <= 6) {
    const int c = f - 4;
    D.gB[c][0] = g[0]; D.gB[c][1] = g[1]; D.gB[c][2] = g[2];
    D.gdivB[0] += h[hpack(0, c)];
    D.gdivB[1] += h[hpack(1, c)];
    D.gdivB[2] += h[hpack(2, c)];
  }
}

template <typename T>
__device__ __forceinline__ void mhd_zero(MhdDerivs<T>& D) {
  for (int a = 0; a < 3; ++a) {
    D.gs[a] = T(0); D.gdivV[a] = T(0); D.gdivB[a] = T(0);
    for (int b = 0; b < 3; ++b) { D.gV[a][b] = T(0); D.gB[a][b] = T(0); }
  }
}

// Coefficient laws (readings of Sec. 2; see phb_params): with the fast-speed
// bound c = sqrt((gamma P + |B|^2) / rho), P = (gamma - 1) sigma,
//   zeta += cl lambda c + ca lambda^2 max(0, -div V),   eta += ce lambda c.
template <typename T>
__device__ __forceinline__ void mhd_laws(const T (&u)[8], const MhdDerivs<T>& D, T gamma, T lam,
                                         T cl, T ca, T ce, T& zeta, T& eta) {
  const T P = (gamma - T(1)) * u[7];
  const T c = sqrt((gamma * P + u[4] * u[4] + u[5] * u[5] + u[6] * u[6]) / u[0]);
  const T divV = D.gV[0][0] + D.gV[1][1] + D.gV[2][2];
  zeta += cl * lam * c;
  if (divV < T(0)) zeta -= ca * lam * lam * divV;
  eta += ce * lam * c;
}

// u: point values (rho, Vx, Vy, Vz, Bx, By, Bz, sigma); out: time derivatives.
template <typename T>
__device__ __forceinline__ void mhd_rhs(const T (&u)[8], const MhdDerivs<T>& D, T gamma, T zeta,
                                        T eta, T (&out)[8]) {
  const T rho = u[0], sig = u[7];
  const T Bx = u[4], By = u[5], Bz = u[6];
  const T divV = D.gV[0][0] + D.gV[1][1] + D.gV[2][2];
  // current J = curl B
  const T Jx = D.gB[2][1] - D.gB[1][2];
  const T Jy = D.gB[0][2] - D.gB[2][0];
  const T Jz = D.gB[1][0] - D.gB[0][1];
  // Lorentz force J x B
  const T Fx = Jy * Bz - Jz * By;
  const T Fy = Jz * Bx - Jx * Bz;
  const T Fz = Jx * By - Jy * Bx;
  const T inv_rho = T(1) / rho;
  const T pg = gamma - T(1);
  out[0] = -rho * divV;
  out[1] = (Fx - pg * D.gs[0]) * inv_rho + zeta * D.gdivV[0];
  out[2] = (Fy - pg * D.gs[1]) * inv_rho + zeta * D.gdivV[1];
  out[3] = (Fz - pg * D.gs[2]) * inv_rho + zeta * D.gdivV[2];
  for (int a = 0; a < 3; ++a) {
    const T adv = Bx * D.gV[a][0] + By * D.gV[a][1] + Bz * D.gV[a][2];
    out[4 + a] = adv - u[4 + a] * divV + eta * D.gdivB[a];
  }
  out[7] = -gamma * sig * divV + rho * zeta * divV * divV;
}

}  // namespace phb
