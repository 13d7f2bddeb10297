/*
 * Plain FP64 Wilson-Dirac operator for the CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Restates Sec. 2's operator (read with the backward link at x - mu):
 *   (D psi)(x) = (4 + m) psi(x)
 *                - 1/2 sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
 *                             + (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu) ]
 * with full 4x4 gamma matrices (chiral basis, gamma_5 = diag(1, 1, -1, -1)) and periodic
 * boundaries; no spin projection, no compression.  A site loop parallelised with OpenMP.
 *
 * Layouts (lexicographic site index x + X*(y + Y*(z + Z*t))):
 *   U   : [V][4][3][3] complex double
 *   psi : [V][4][3]    complex double (spin, colour)
 */
#include <complex.h>
#include <string.h>

typedef double complex cplx;

/* gamma_k = [[0, -i sigma_k], [i sigma_k, 0]] (k = x, y, z), gamma_t = [[0, 1], [1, 0]] */
static void gamma_matrix(int mu, cplx g[4][4]) {
  cplx s[2][2];
  memset(s, 0, sizeof(s));
  if (mu == 0) { s[0][1] = 1; s[1][0] = 1; }
  if (mu == 1) { s[0][1] = -I; s[1][0] = I; }
  if (mu == 2) { s[0][0] = 1; s[1][1] = -1; }
  memset(g, 0, sizeof(cplx) * 16);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      if (mu < 3) {
        g[a][2 + b] = -I * s[a][b];
        g[2 + a][b] = I * s[a][b];
      } else {
        g[a][2 + b] = (a == b);
        g[2 + a][b] = (a == b);
      }
    }
}

static long lex(const int c[4], const int L[4]) { return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3])); }

/* out(x) = [accumulate ? out(x) : 0] + one hopping term reading x + sign*mu (see above) */
void dirac_ref_hop(const cplx* U, const cplx* psi, cplx* out, const int* L, int mu, int sign, int accumulate) {
  const long V = (long)L[0] * L[1] * L[2] * L[3];
  cplx g[4][4], P[4][4];
  gamma_matrix(mu, g);
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b) P[a][b] = -0.5 * ((a == b) - sign * g[a][b]);
#pragma omp parallel for schedule(static)
  for (long v = 0; v < V; ++v) {
    int c[4];
    long t = v;
    for (int i = 0; i < 4; ++i) { c[i] = (int)(t % L[i]); t /= L[i]; }
    int n[4] = {c[0], c[1], c[2], c[3]};
    n[mu] = (c[mu] + sign + L[mu]) % L[mu];
    const long y = lex(n, L);
    /* link: U_mu(x) forward, U_mu(x - mu)^dag backward */
    const cplx* u = U + ((sign > 0 ? v : y) * 4 + mu) * 9;
    cplx w[4][3];
    for (int s = 0; s < 4; ++s)
      for (int a = 0; a < 3; ++a) {
        cplx acc = 0;
        for (int b = 0; b < 3; ++b)
          acc += (sign > 0 ? u[a * 3 + b] : conj(u[b * 3 + a])) * psi[y * 12 + s * 3 + b];
        w[s][a] = acc;
      }
    for (int s = 0; s < 4; ++s)
      for (int a = 0; a < 3; ++a) {
        cplx acc = accumulate ? out[v * 12 + s * 3 + a] : 0;
        for (int r = 0; r < 4; ++r) acc += P[s][r] * w[r][a];
        out[v * 12 + s * 3 + a] = acc;
      }
  }
}

void dirac_ref_apply(const cplx* U, const cplx* psi, cplx* out, const int* L, double m) {
  const long V = (long)L[0] * L[1] * L[2] * L[3];
#pragma omp parallel for schedule(static)
  for (long i = 0; i < V * 12; ++i) out[i] = (4.0 + m) * psi[i];
  for (int mu = 0; mu < 4; ++mu) {
    dirac_ref_hop(U, psi, out, L, mu, +1, 1);
    dirac_ref_hop(U, psi, out, L, mu, -1, 1);
  }
}
