// Even-odd (red/black) form of the fine Wilson operator (Sec. 3: red/black preconditioning
// combined with multigrid).  D = d + H with d = 4 + m and H the hopping term (every hop joins
// sites of opposite parity (x + y + z + t) mod 2).  The solve runs on the even-site Schur
// complement S = d - H_eo H_oe / d; with the raw hop sum h(psi) = sum_mu [(1 - gamma_mu) U
// psi(x + mu) + (1 + gamma_mu) U^dag psi(x - mu)] (so H = -h / 2):
//   t_o  = h_oe(x_e)                       (mode HOP)
//   S x_e = d x_e - h_eo(t_o) / (4 d)       (mode SCHUR, optionally b - S x_e and |.|^2)
//   b^_e = b_e + h_eo(b_o) / (2 d)          (mode PREP:  b_e - H_eo b_o / d)
//   x_o  = (b_o + h_oe(x_e) / 2) / d        (mode RECON: (b_o - H_oe x_e) / d)
// Half-lattice fields: [rhs][6][V/2] chunks of two complex numbers; site v (either parity) sits
// at half index v >> 1 (the x extent is even, so sites 2k and 2k + 1 have opposite parities).
#include "kernels.h"
#include "wilson.cuh"

namespace wmg {

namespace {

struct EoDiv {
  FastDiv dx, dy, dz;
};

}  // namespace

// One thread per (half-lattice site k of parity p_out, rhs); the rhs index runs fastest over CTAs.
template <typename R, int RED, int GC>
__global__ void __launch_bounds__(128) k_dslash_eo(void* __restrict__ out, const void* __restrict__ in,
                                                   const void* __restrict__ self, const void* __restrict__ b,
                                                   const void* __restrict__ gauge, Geom g, EoDiv dv, int p_out,
                                                   int mode, const double* __restrict__ mass,
                                                   const int* __restrict__ active, int nrhs, int nblk,
                                                   RedBuf rb) {
  const int rhs = blockIdx.x % nrhs;
  const int sb = blockIdx.x / nrhs;
  if (active && !active[rhs]) return;  // whole CTA exits together (uniform per CTA)
  const int Vh = g.V / 2;
  const int k = sb * blockDim.x + threadIdx.x;
  const size_t fb = spinor_field_bytes<R>(Vh);
  const char* inr = reinterpret_cast<const char*>(in) + fb * rhs;
  R red = 0;
  if (k < Vh) {
    // coordinates of site 2k, then the site of parity p_out among 2k, 2k + 1
    const uint32_t v0 = 2u * (uint32_t)k;
    const uint32_t q0 = fdiv(v0, dv.dx), q1 = fdiv(q0, dv.dy), q2 = fdiv(q1, dv.dz);
    int c[4] = {(int)(v0 - q0 * g.L[0]), (int)(q0 - q1 * g.L[1]), (int)(q1 - q2 * g.L[2]), (int)q2};
    const int odd0 = (c[0] + c[1] + c[2] + c[3]) & 1;
    const int v = (int)v0 + (odd0 != p_out);
    c[0] += (odd0 != p_out);
    cpx<R> acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = cpx<R>{R(0), R(0)};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      cpx<R> u[9], nb[12];
      const int vf = neighbour(g, v, c, mu, +1);
      load_link_gc<R, GC>(gauge, g.V, mu, v, u);
      load_spinor<R>(inr, Vh, vf >> 1, nb);
      hop_accumulate<+1>(mu, u, nb, acc);
      const int vb = neighbour(g, v, c, mu, -1);
      load_link_gc<R, GC>(gauge, g.V, mu, vb, u);
      load_spinor<R>(inr, Vh, vb >> 1, nb);
      hop_accumulate<-1>(mu, u, nb, acc);
    }
    const R d = R(4.0 + mass[rhs]);
    cpx<R> sf[12];
    if (mode != 0) load_spinor<R>(reinterpret_cast<const char*>(self) + fb * rhs, Vh, k, sf);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      if (mode == 1) acc[i] = d * sf[i] - (R(0.25) / d) * acc[i];  // S x_e
      else if (mode == 2) acc[i] = sf[i] + (R(0.5) / d) * acc[i];  // b^_e
      else if (mode == 3) acc[i] = (R(1) / d) * (sf[i] + R(0.5) * acc[i]);  // x_o
    }
    if (b) {
      cpx<R> bb[12];
      load_spinor<R>(reinterpret_cast<const char*>(b) + fb * rhs, Vh, k, bb);
#pragma unroll
      for (int i = 0; i < 12; ++i) acc[i] = bb[i] - acc[i];
    }
    store_spinor<R>(reinterpret_cast<char*>(out) + fb * rhs, Vh, k, acc);
    if (RED) {
      R nn = 0;
#pragma unroll
      for (int i = 0; i < 12; ++i) norm2_acc(nn, acc[i]);
      red = nn;
    }
  }
  if (RED) {
    __shared__ double sm[32];
    double vals[1];
    R rv[1] = {red};
    cta_reduce_mixed<R, 1>(rv, vals, sm);
    grid_finish<1>(rb, rhs, sb, nblk, vals);
  }
}

// half <-> whole-lattice native fields: embed writes the even sites from half_e and the odd ones
// from half_o (zeros where a half field is null)
template <typename R>
__global__ void k_eo_embed(void* __restrict__ full, const void* __restrict__ half_e, const void* __restrict__ half_o,
                           Geom g, int nrhs) {
  const int rhs = blockIdx.y;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= g.V) return;
  int c[4];
  site_coords(g, v, c);
  const void* half = ((c[0] + c[1] + c[2] + c[3]) & 1) ? half_o : half_e;
  const int Vh = g.V / 2;
  char* f = reinterpret_cast<char*>(full) + spinor_field_bytes<R>(g.V) * rhs;
  const char* h = half ? reinterpret_cast<const char*>(half) + spinor_field_bytes<R>(Vh) * rhs : nullptr;
#pragma unroll
  for (int ch = 0; ch < 6; ++ch) {
    cpx<R> a{R(0), R(0)}, bb{R(0), R(0)};
    if (h) Chunk2<R>::load_cg(h, (size_t)ch * Vh + (v >> 1), a, bb);
    Chunk2<R>::store(f, (size_t)ch * g.V + v, a, bb);
  }
}

template <typename R>
__global__ void k_eo_extract(void* __restrict__ half, const void* __restrict__ full, Geom g, int p, int nrhs) {
  const int rhs = blockIdx.y;
  const int Vh = g.V / 2;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Vh) return;
  const int v = parity_site(g, k, p);
  const char* f = reinterpret_cast<const char*>(full) + spinor_field_bytes<R>(g.V) * rhs;
  char* h = reinterpret_cast<char*>(half) + spinor_field_bytes<R>(Vh) * rhs;
#pragma unroll
  for (int ch = 0; ch < 6; ++ch) {
    cpx<R> a, bb;
    Chunk2<R>::load_cg(f, (size_t)ch * g.V + v, a, bb);
    Chunk2<R>::store(h, (size_t)ch * Vh + k, a, bb);
  }
}

// The last MR step of the red/black solve's cycle, restricted to what the outer solve uses:
// out_e = x_e + alpha r_e at the even sites (alpha = red[0..1] / red[2] per rhs), written as
// half-lattice fields; x, r whole-lattice.  One thread per (even site k, rhs).
template <typename R>
__global__ void k_mr_update_even(const void* __restrict__ x, const void* __restrict__ r, void* __restrict__ out,
                                 Geom g, EoDiv dv, const double* __restrict__ red, const int* __restrict__ active) {
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const double qq = red[rhs * 3 + 2];
  R sc[2];
  cta_scalars<R, 2>(sc, [&](double* v) {
    v[0] = qq > 0.0 ? red[rhs * 3 + 0] / qq : 0.0;
    v[1] = qq > 0.0 ? red[rhs * 3 + 1] / qq : 0.0;
  });
  const cpx<R> al{sc[0], sc[1]};
  const int Vh = g.V / 2;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Vh) return;
  const uint32_t v0 = 2u * (uint32_t)k;
  const uint32_t q0 = fdiv(v0, dv.dx), q1 = fdiv(q0, dv.dy), q2 = fdiv(q1, dv.dz);
  const int odd0 = ((int)(v0 - q0 * g.L[0]) + (int)(q0 - q1 * g.L[1]) + (int)(q1 - q2 * g.L[2]) + (int)q2) & 1;
  const int v = (int)v0 + odd0;  // the even one of the sites 2k, 2k + 1
  const char* xr = reinterpret_cast<const char*>(x) + spinor_field_bytes<R>(g.V) * rhs;
  const char* rr = reinterpret_cast<const char*>(r) + spinor_field_bytes<R>(g.V) * rhs;
  char* o = reinterpret_cast<char*>(out) + spinor_field_bytes<R>(Vh) * rhs;
#pragma unroll
  for (int ch = 0; ch < 6; ++ch) {
    cpx<R> a, b, ra, rb2;
    Chunk2<R>::load(xr, (size_t)ch * g.V + v, a, b);
    Chunk2<R>::load(rr, (size_t)ch * g.V + v, ra, rb2);
    cfma(a, al, ra);
    cfma(b, al, rb2);
    Chunk2<R>::store(o, (size_t)ch * Vh + k, a, b);
  }
}

// The red/black cycle's MR smoother with its solution updates deferred: after steps 1..nsteps the
// result at the even sites is out_e = x_e + alpha_1 r_1 + ... + alpha_n r_n (the residual of step
// i in r.p[i], alpha_i = red[i][0..1] / red[i][2] per rhs, red[i] = red0 + i * rstride), formed
// with the same FMA sequence as step-by-step updates of x; half-lattice output.
template <typename R>
__global__ void k_mr_combine_even(const void* __restrict__ x, MrSteps rs, void* __restrict__ out, Geom g, EoDiv dv,
                                  const double* __restrict__ red0, int rstride, const int* __restrict__ active) {
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  R sc[2 * kMrMaxSteps];
  cta_scalars<R, 2 * kMrMaxSteps>(sc, [&](double* v) {
    for (int i = 0; i < kMrMaxSteps; ++i) {
      const double* rd = red0 + (size_t)i * rstride + rhs * 3;
      const bool ok = i < rs.n && rd[2] > 0.0;
      v[2 * i] = ok ? rd[0] / rd[2] : 0.0;
      v[2 * i + 1] = ok ? rd[1] / rd[2] : 0.0;
    }
  });
  const int Vh = g.V / 2;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Vh) return;
  const uint32_t v0 = 2u * (uint32_t)k;
  const uint32_t q0 = fdiv(v0, dv.dx), q1 = fdiv(q0, dv.dy), q2 = fdiv(q1, dv.dz);
  const int odd0 = ((int)(v0 - q0 * g.L[0]) + (int)(q0 - q1 * g.L[1]) + (int)(q1 - q2 * g.L[2]) + (int)q2) & 1;
  const int v = (int)v0 + odd0;  // the even one of the sites 2k, 2k + 1
  const size_t fb = spinor_field_bytes<R>(g.V);
  const char* xr = reinterpret_cast<const char*>(x) + fb * rhs;
  char* o = reinterpret_cast<char*>(out) + spinor_field_bytes<R>(Vh) * rhs;
#pragma unroll
  for (int ch = 0; ch < 6; ++ch) {
    cpx<R> a, b;
    Chunk2<R>::load(xr, (size_t)ch * g.V + v, a, b);
    for (int i = 0; i < rs.n; ++i) {
      cpx<R> ra, rb2;
      Chunk2<R>::load(reinterpret_cast<const char*>(rs.p[i]) + fb * rhs, (size_t)ch * g.V + v, ra, rb2);
      const cpx<R> al{sc[2 * i], sc[2 * i + 1]};
      cfma(a, al, ra);
      cfma(b, al, rb2);
    }
    Chunk2<R>::store(o, (size_t)ch * Vh + k, a, b);
  }
}

int dslash_eo_blocks(int V) { return (V / 2 + kDslashThreads - 1) / kDslashThreads; }

void mr_combine_even(int prec, const void* x, const MrSteps& rs, void* out_half, const Geom& g, int nrhs,
                     const double* red0, int rstride, const int* active, cudaStream_t s) {
  count_launch();
  const dim3 grid((g.V / 2 + 255) / 256, nrhs);
  const EoDiv dv{make_fastdiv(g.L[0]), make_fastdiv(g.L[1]), make_fastdiv(g.L[2])};
  if (prec == WMG_PREC_DOUBLE)
    k_mr_combine_even<double><<<grid, 256, 0, s>>>(x, rs, out_half, g, dv, red0, rstride, active);
  else
    k_mr_combine_even<float><<<grid, 256, 0, s>>>(x, rs, out_half, g, dv, red0, rstride, active);
}

void mr_update_even(int prec, const void* x, const void* r, void* out_half, const Geom& g, int nrhs,
                    const double* red, const int* active, cudaStream_t s) {
  count_launch();
  const dim3 grid((g.V / 2 + 255) / 256, nrhs);
  const EoDiv dv{make_fastdiv(g.L[0]), make_fastdiv(g.L[1]), make_fastdiv(g.L[2])};
  if (prec == WMG_PREC_DOUBLE) k_mr_update_even<double><<<grid, 256, 0, s>>>(x, r, out_half, g, dv, red, active);
  else k_mr_update_even<float><<<grid, 256, 0, s>>>(x, r, out_half, g, dv, red, active);
}

void dslash_eo(int prec, int mode, int p_out, void* out, const void* in, const void* self, const void* b,
               const void* gauge, int gc, const Geom& g, const double* mass_dev, const int* active, int nrhs,
               const RedBuf* rb, cudaStream_t s) {
  count_launch();
  const int nb = dslash_eo_blocks(g.V);
  const unsigned grid = (unsigned)nb * nrhs;
  const EoDiv dv{make_fastdiv(g.L[0]), make_fastdiv(g.L[1]), make_fastdiv(g.L[2])};
  RedBuf r = rb ? *rb : RedBuf{nullptr, nullptr, nullptr};
#define WMG_EO(R, RED, GC)                                                                                  \
  k_dslash_eo<R, RED, GC><<<grid, kDslashThreads, 0, s>>>(out, in, self, b, gauge, g, dv, p_out, mode, mass_dev, \
                                                          active, nrhs, nb, r)
  if (prec == WMG_PREC_DOUBLE) {
    if (rb) WMG_EO(double, 1, 12);
    else WMG_EO(double, 0, 12);
  } else if (gc == 8) {
    if (rb) WMG_EO(float, 1, 8);
    else WMG_EO(float, 0, 8);
  } else if (gc == 18) {
    if (rb) WMG_EO(float, 1, 18);
    else WMG_EO(float, 0, 18);
  } else {
    if (rb) WMG_EO(float, 1, 12);
    else WMG_EO(float, 0, 12);
  }
#undef WMG_EO
}

void eo_embed(int prec, void* full, const void* half_e, const void* half_o, const Geom& g, int nrhs, cudaStream_t s) {
  count_launch();
  const dim3 grid((g.V + 255) / 256, nrhs);
  if (prec == WMG_PREC_DOUBLE) k_eo_embed<double><<<grid, 256, 0, s>>>(full, half_e, half_o, g, nrhs);
  else k_eo_embed<float><<<grid, 256, 0, s>>>(full, half_e, half_o, g, nrhs);
}

void eo_extract(int prec, void* half, const void* full, const Geom& g, int p, int nrhs, cudaStream_t s) {
  count_launch();
  const dim3 grid((g.V / 2 + 255) / 256, nrhs);
  if (prec == WMG_PREC_DOUBLE) k_eo_extract<double><<<grid, 256, 0, s>>>(half, full, g, p, nrhs);
  else k_eo_extract<float><<<grid, 256, 0, s>>>(half, full, g, p, nrhs);
}

}  // namespace wmg
