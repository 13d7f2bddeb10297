// Spin-projected Wilson hopping term (Sec. 2, the equation for D_xy(U)).
//
// Chiral basis: gamma_mu = [[0, B_mu], [C_mu, 0]] with C_mu = B_mu^dag and B_mu C_mu = 1:
//   B_x = -i sigma_1, B_y = -i sigma_2, B_z = -i sigma_3, B_t = 1.
// Upper spins (0, 1) have gamma_5 = +1, lower spins (2, 3) gamma_5 = -1.
//   (1 - gamma_mu) psi = [h, -C h],  h = psi_up - B psi_lo   (forward hop)
//   (1 + gamma_mu) psi = [h,  C h],  h = psi_up + B psi_lo   (backward hop)
// so each hop multiplies only a 2-spin x 3-colour half spinor by the link.
// Each B_mu, C_mu has one non-zero per row: row j reads column spin_B_col(mu, j) times a
// unit phase (0: 1, 1: i, 2: -1, 3: -i).
#pragma once
#include "wmg_common.cuh"

__host__ __device__ constexpr int spin_B_col(int mu, int j) { return (mu == 0 || mu == 1) ? 1 - j : j; }
__host__ __device__ constexpr int spin_B_ph(int mu, int j) {
  // B_x = [[0,-i],[-i,0]], B_y = [[0,-1],[1,0]], B_z = [[-i,0],[0,i]], B_t = 1
  return mu == 0 ? 3 : mu == 1 ? (j == 0 ? 2 : 0) : mu == 2 ? (j == 0 ? 3 : 1) : 0;
}
__host__ __device__ constexpr int spin_C_ph(int mu, int j) {
  // C = B^dag: C_x = [[0,i],[i,0]], C_y = [[0,1],[-1,0]], C_z = [[i,0],[0,-i]], C_t = 1
  return mu == 0 ? 1 : mu == 1 ? (j == 0 ? 0 : 2) : mu == 2 ? (j == 0 ? 1 : 3) : 0;
}

// half spinor h[3*j + a] for a hop in direction mu; SIGN = +1 forward (1 - gamma), -1 backward
template <int SIGN, typename R>
WMG_D void spin_project(int mu, const cpx<R> s[12], cpx<R> h[6]) {
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int col = spin_B_col(mu, j), ph = spin_B_ph(mu, j);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cpx<R> b = mul_phase(s[3 * (2 + col) + a], ph);
      h[3 * j + a] = (SIGN > 0) ? s[3 * j + a] - b : s[3 * j + a] + b;
    }
  }
}

// acc += [h, -C h] (forward) or [h, C h] (backward)
template <int SIGN, typename R>
WMG_D void spin_reconstruct_add(int mu, const cpx<R> h[6], cpx<R> acc[12]) {
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int col = spin_B_col(mu, j), ph = spin_C_ph(mu, j);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      acc[3 * j + a] += h[3 * j + a];
      cpx<R> c = mul_phase(h[3 * col + a], ph);
      if (SIGN > 0) acc[3 * (2 + j) + a] -= c;
      else acc[3 * (2 + j) + a] += c;
    }
  }
}

// out = U h (each spin row of h is a colour vector)
template <typename R>
WMG_D void link_mul(const cpx<R> u[9], const cpx<R> h[6], cpx<R> out[6]) {
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cpx<R> t = u[3 * a] * h[3 * j];
      cfma(t, u[3 * a + 1], h[3 * j + 1]);
      cfma(t, u[3 * a + 2], h[3 * j + 2]);
      out[3 * j + a] = t;
    }
}
// out = U^dag h
template <typename R>
WMG_D void link_mul_dag(const cpx<R> u[9], const cpx<R> h[6], cpx<R> out[6]) {
#pragma unroll
  for (int j = 0; j < 2; ++j)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      cpx<R> t = cmulc(u[a], h[3 * j]);
      cfmac(t, u[3 + a], h[3 * j + 1]);
      cfmac(t, u[6 + a], h[3 * j + 2]);
      out[3 * j + a] = t;
    }
}

// One hopping term accumulated WITHOUT the -1/2 factor:
//   SIGN = +1: acc += (1 - gamma_mu) U_mu(x) psi(x + mu)            (u = U_mu(x))
//   SIGN = -1: acc += (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu)   (u = U_mu(x - mu))
template <int SIGN, typename R>
WMG_D void hop_accumulate(int mu, const cpx<R> u[9], const cpx<R> nb[12], cpx<R> acc[12]) {
  cpx<R> h[6], uh[6];
  spin_project<SIGN>(mu, nb, h);
  if (SIGN > 0) link_mul(u, h, uh);
  else link_mul_dag(u, h, uh);
  spin_reconstruct_add<SIGN>(mu, uh, acc);
}

// The same hop with the neighbour spinor held as s * nb (FP16 storage with the per-site scale
// s): the scale is applied in the accumulation, acc += s * [h', -/+ C h'].
template <int SIGN>
WMG_D void hop_accumulate_scaled(int mu, const cpx<float> u[9], const cpx<float> nb[12], float sc, cpx<float> acc[12]) {
  cpx<float> h[6], uh[6];
  spin_project<SIGN>(mu, nb, h);
  if (SIGN > 0) link_mul(u, h, uh);
  else link_mul_dag(u, h, uh);
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int col = spin_B_col(mu, j), ph = spin_C_ph(mu, j);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const cpx<float> t = uh[3 * j + a];
      acc[3 * j + a].re = fmaf(sc, t.re, acc[3 * j + a].re);
      acc[3 * j + a].im = fmaf(sc, t.im, acc[3 * j + a].im);
      const cpx<float> c = mul_phase(uh[3 * col + a], ph);
      const float g = SIGN > 0 ? -sc : sc;
      acc[3 * (2 + j) + a].re = fmaf(g, c.re, acc[3 * (2 + j) + a].re);
      acc[3 * (2 + j) + a].im = fmaf(g, c.im, acc[3 * (2 + j) + a].im);
    }
  }
}
