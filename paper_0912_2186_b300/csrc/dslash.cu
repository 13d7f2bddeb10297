// Fine-lattice kernels: gauge 12-real packing (Table 2's "12 floats"), spinor layout
// conversion and the spin-projected Wilson operator (Sec. 2, eq. for D_xy(U)).
#include "kernels.h"
#include "wilson.cuh"

namespace wmg {

// ------------------------------------------------------------------------------------
// packing
// ------------------------------------------------------------------------------------
// canonical U [V][4][3][3] complex double -> native [mu][3][V] chunks (rows 0, 1)
template <typename R>
__global__ void k_pack_gauge(const double2* __restrict__ canon, void* __restrict__ out, int V) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  for (int mu = 0; mu < 4; ++mu) {
    const double2* u = canon + ((size_t)v * 4 + mu) * 9;
    for (int c = 0; c < 3; ++c) {
      double2 a = u[2 * c], b = u[2 * c + 1];
      Chunk2<R>::store(out, (size_t)(mu * 3 + c) * V + v, cpx<R>{R(a.x), R(a.y)}, cpx<R>{R(b.x), R(b.y)});
    }
  }
}

// native FP64 12-real links -> 8-real FP32 (see load_link8): row 2 rebuilt in FP64, then
// (a1, a2), (b0, arg a0, arg c0)
__global__ void k_pack_gauge8(const void* __restrict__ g64, float4* __restrict__ out, int V, int* degenerate) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  for (int mu = 0; mu < 4; ++mu) {
    cd u[9];
    load_link<double>(g64, V, mu, v, u);
    // the 8-real form divides by |a1|^2 + |a2|^2: links where it (nearly) vanishes are flagged
    if (norm2(u[1]) + norm2(u[2]) < 1e-6) atomicExch(degenerate, 1);
    out[(size_t)(mu * 2) * V + v] = make_float4((float)u[1].re, (float)u[1].im, (float)u[2].re, (float)u[2].im);
    out[(size_t)(mu * 2 + 1) * V + v] =
        make_float4((float)u[3].re, (float)u[3].im, (float)atan2(u[0].im, u[0].re), (float)atan2(u[6].im, u[6].re));
  }
}

// native FP64 12-real links -> 18-real FP32 (see load_link18), row 2 rebuilt in FP64
__global__ void k_pack_gauge18(const void* __restrict__ g64, float4* __restrict__ out, int V) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  float2* o8 = reinterpret_cast<float2*>(out + (size_t)16 * V);
  for (int mu = 0; mu < 4; ++mu) {
    cd u[9];
    load_link<double>(g64, V, mu, v, u);
    for (int c = 0; c < 4; ++c)
      out[(size_t)(mu * 4 + c) * V + v] = make_float4((float)u[2 * c].re, (float)u[2 * c].im,
                                                      (float)u[2 * c + 1].re, (float)u[2 * c + 1].im);
    o8[(size_t)mu * V + v] = make_float2((float)u[8].re, (float)u[8].im);
  }
}

// canonical [rhs][V][12] <-> native [rhs][6][V][2]
template <typename R>
__global__ void k_pack_spinor(const double2* __restrict__ canon, void* __restrict__ out, int V, int nrhs) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)V * nrhs) return;
  int r = (int)(i / V), v = (int)(i % V);
  const double2* s = canon + i * 12;
  char* o = reinterpret_cast<char*>(out) + spinor_field_bytes<R>(V) * r;
  for (int c = 0; c < 6; ++c) {
    double2 a = s[2 * c], b = s[2 * c + 1];
    Chunk2<R>::store(o, (size_t)c * V + v, cpx<R>{R(a.x), R(a.y)}, cpx<R>{R(b.x), R(b.y)});
  }
}
template <typename R>
__global__ void k_unpack_spinor(const void* __restrict__ in, double2* __restrict__ canon, int V, int nrhs) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)V * nrhs) return;
  int r = (int)(i / V), v = (int)(i % V);
  const char* p = reinterpret_cast<const char*>(in) + spinor_field_bytes<R>(V) * r;
  double2* s = canon + i * 12;
  for (int c = 0; c < 6; ++c) {
    cpx<R> a, b;
    Chunk2<R>::load(p, (size_t)c * V + v, a, b);
    s[2 * c] = make_double2(a.re, a.im);
    s[2 * c + 1] = make_double2(b.re, b.im);
  }
}

// ------------------------------------------------------------------------------------
// Wilson operator.  One thread per (site, rhs); the rhs index runs fastest over CTAs so
// that CTAs working on the same sites for different right-hand sides share the links in
// L2.  out = (4 + m_r) in - 1/2 sum_mu hops       (b == nullptr)
//      out = b - D in                               (b != nullptr, residual form)
// Optional fused reductions per rhs: red0 = {<out, in>, |out|^2} (MR smoother) or
// {|out|^2} alone.
// ------------------------------------------------------------------------------------
// Site coordinates by multiply-shift division (the lattice extents are runtime values).
struct DslashDiv {
  FastDiv dx, dy, dz;
};
WMG_D void site_coords_fast(const Geom& g, const DslashDiv& d, int v, int c[4]) {
  const uint32_t q0 = fdiv((uint32_t)v, d.dx), q1 = fdiv(q0, d.dy), q2 = fdiv(q1, d.dz);
  c[0] = v - (int)q0 * g.L[0];
  c[1] = (int)q0 - (int)q1 * g.L[1];
  c[2] = (int)q1 - (int)q2 * g.L[2];
  c[3] = (int)q2;
}

// With RED > 0 an FP32 CTA takes SPB consecutive site blocks of one rhs (its per-site sums
// added in that order), so that the CTAs publishing partial sums (a fence and an atomic each)
// are SPB times fewer; the partition depends on the volume only.  (The FP64 kernel runs one
// CTA per SM and keeps one block per CTA.)
template <typename R, int RED> constexpr int dslash_spb() { return RED > 0 && sizeof(R) == 4 ? 4 : 1; }

template <typename R, int RED, int GC>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 5 : 1) k_dslash(void* __restrict__ out,
                                                                        const void* __restrict__ in,
                                                                        const void* __restrict__ b,
                                                                        const void* __restrict__ gauge, Geom g,
                                                                        DslashDiv dv, const double* __restrict__ mass,
                                                                        const int* __restrict__ active, int nrhs,
                                                                        int nblk_site, RedBuf rb, int b_half) {
  constexpr int SPB = dslash_spb<R, RED>();
  const int rhs = blockIdx.x % nrhs;
  const int sbe = blockIdx.x / nrhs;
  if (active && !active[rhs]) return;  // whole CTA exits together (uniform per CTA)
  const size_t fb = spinor_field_bytes<R>(g.V);
  const char* inr = reinterpret_cast<const char*>(in) + fb * rhs;
  R red[3] = {R(0), R(0), R(0)};
#pragma unroll 1
  for (int j = 0; j < SPB; ++j) {
  const int v = (sbe * SPB + j) * blockDim.x + threadIdx.x;
  cpx<R> acc[12];
  if (v < g.V) {
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = cpx<R>{R(0), R(0)};
    int c[4];
    site_coords_fast(g, dv, v, c);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      cpx<R> u[9], nb[12];
      const int vf = neighbour(g, v, c, mu, +1);
      load_link_gc<R, GC>(gauge, g.V, mu, v, u);
      load_spinor<R>(inr, g.V, vf, nb);
      hop_accumulate<+1>(mu, u, nb, acc);
      const int vb = neighbour(g, v, c, mu, -1);
      load_link_gc<R, GC>(gauge, g.V, mu, vb, u);
      load_spinor<R>(inr, g.V, vb, nb);
      hop_accumulate<-1>(mu, u, nb, acc);
    }
    cpx<R> self[12];
    load_spinor<R>(inr, g.V, v, self);
    const R diag = R(4.0 + mass[rhs]);
    const R half = R(-0.5);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      cpx<R> o{diag * self[i].re + half * acc[i].re, diag * self[i].im + half * acc[i].im};
      acc[i] = o;
    }
    if (b) {
      // b_half: b holds the even sites only (half-lattice fields, site v at v >> 1), zero elsewhere
      cpx<R> bb[12];
      if (!b_half) {
        load_spinor<R>(reinterpret_cast<const char*>(b) + fb * rhs, g.V, v, bb);
      } else if (((c[0] + c[1] + c[2] + c[3]) & 1) == 0) {
        load_spinor<R>(reinterpret_cast<const char*>(b) + spinor_field_bytes<R>(g.V / 2) * rhs, g.V / 2, v >> 1, bb);
      } else {
#pragma unroll
        for (int i = 0; i < 12; ++i) bb[i] = cpx<R>{R(0), R(0)};
      }
#pragma unroll
      for (int i = 0; i < 12; ++i) acc[i] = bb[i] - acc[i];
    }
    store_spinor<R>(reinterpret_cast<char*>(out) + fb * rhs, g.V, v, acc);
    // per-site sums and the thread's and warp's sums in the field's precision; FP64 across the
    // warps and CTAs
    if (RED == 2) {
      R a0 = 0, a1 = 0;
#pragma unroll
      for (int i = 0; i < 12; ++i) {
        cdot_acc(a0, a1, acc[i], self[i]);
      }
      red[0] += a0;
      red[1] += a1;
    }
    if (RED >= 1) {
      R nn = 0;
#pragma unroll
      for (int i = 0; i < 12; ++i) norm2_acc(nn, acc[i]);
      red[RED == 2 ? 2 : 0] += nn;
    }
  }
  }
  if (RED > 0) {
    constexpr int NV = RED == 2 ? 3 : 1;
    __shared__ double sm[32 * 3];
    double vals[NV];
    cta_reduce_mixed<R, NV>(red, vals, sm);
    grid_finish<NV>(rb, rhs, sbe, nblk_site, vals);
  }
}

// ------------------------------------------------------------------------------------
// One MR step with the previous step's update fused in (the smoother of Sec. 3): with r, q =
// D r and alpha = <q, r> / |q|^2 of the previous step (red_prev, per rhs; 0 when |q| = 0),
//   r' = r - alpha q  (own site written to r_out; at the neighbours formed on the fly),
//   x += alpha r      (own site),
//   q' = D r'         with the sums {Re, Im <q', r'>, |q'|^2} into rb,
// so that the update costs no pass of its own.  r_out and out must not alias r or q (other CTAs
// read them at their neighbours); rb.result must not be red_prev.  Same partition of sites into
// CTAs as k_dslash<R, 2> (the order of the per-rhs sums depends on the volume only).
// ------------------------------------------------------------------------------------
template <typename R, int GC>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? 4 : 1) k_dslash_mr(void* __restrict__ out,
                                                                           const void* __restrict__ in,
                                                                           const void* __restrict__ qin,
                                                                           void* __restrict__ rout,
                                                                           void* __restrict__ x,
                                                                           const double* __restrict__ red_prev,
                                                                           const void* __restrict__ gauge, Geom g,
                                                                           DslashDiv dv,
                                                                           const double* __restrict__ mass,
                                                                           const int* __restrict__ active, int nrhs,
                                                                           int nblk_site, RedBuf rb) {
  constexpr int SPB = dslash_spb<R, 2>();
  const int rhs = blockIdx.x % nrhs;
  const int sbe = blockIdx.x / nrhs;
  if (active && !active[rhs]) return;  // whole CTA exits together (uniform per CTA)
  const size_t fb = spinor_field_bytes<R>(g.V);
  const char* inr = reinterpret_cast<const char*>(in) + fb * rhs;
  const char* qr = reinterpret_cast<const char*>(qin) + fb * rhs;
  const double qq = red_prev[rhs * 3 + 2];
  R sc[2];
  cta_scalars<R, 2>(sc, [&](double* v) {
    v[0] = qq > 0.0 ? red_prev[rhs * 3 + 0] / qq : 0.0;
    v[1] = qq > 0.0 ? red_prev[rhs * 3 + 1] / qq : 0.0;
  });
  const cpx<R> al{sc[0], sc[1]};
  R red[3] = {R(0), R(0), R(0)};
#pragma unroll 1
  for (int j = 0; j < SPB; ++j) {
    const int v = (sbe * SPB + j) * blockDim.x + threadIdx.x;
    if (v >= g.V) continue;
    cpx<R> acc[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = cpx<R>{R(0), R(0)};
    int c[4];
    site_coords_fast(g, dv, v, c);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      cpx<R> u[9], nb[12], nq[12];
      const int vf = neighbour(g, v, c, mu, +1);
      load_link_gc<R, GC>(gauge, g.V, mu, v, u);
      load_spinor<R>(inr, g.V, vf, nb);
      load_spinor<R>(qr, g.V, vf, nq);
#pragma unroll
      for (int i = 0; i < 12; ++i) nb[i] = nb[i] - al * nq[i];
      hop_accumulate<+1>(mu, u, nb, acc);
      const int vb = neighbour(g, v, c, mu, -1);
      load_link_gc<R, GC>(gauge, g.V, mu, vb, u);
      load_spinor<R>(inr, g.V, vb, nb);
      load_spinor<R>(qr, g.V, vb, nq);
#pragma unroll
      for (int i = 0; i < 12; ++i) nb[i] = nb[i] - al * nq[i];
      hop_accumulate<-1>(mu, u, nb, acc);
    }
    cpx<R> self[12], qs[12], xs[12];
    load_spinor<R>(inr, g.V, v, self);
    load_spinor<R>(qr, g.V, v, qs);
    char* xr = reinterpret_cast<char*>(x) + fb * rhs;
    load_spinor<R>(xr, g.V, v, xs);
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      cfma(xs[i], al, self[i]);       // x += alpha r
      self[i] = self[i] - al * qs[i];  // r' = r - alpha q
    }
    store_spinor<R>(xr, g.V, v, xs);
    store_spinor<R>(reinterpret_cast<char*>(rout) + fb * rhs, g.V, v, self);
    const R diag = R(4.0 + mass[rhs]);
    const R half = R(-0.5);
#pragma unroll
    for (int i = 0; i < 12; ++i)
      acc[i] = cpx<R>{diag * self[i].re + half * acc[i].re, diag * self[i].im + half * acc[i].im};
    store_spinor<R>(reinterpret_cast<char*>(out) + fb * rhs, g.V, v, acc);
    R a0 = 0, a1 = 0, nn = 0;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      cdot_acc(a0, a1, acc[i], self[i]);
      norm2_acc(nn, acc[i]);
    }
    red[0] += a0;
    red[1] += a1;
    red[2] += nn;
  }
  __shared__ double sm[32 * 3];
  double vals[3];
  cta_reduce_mixed<R, 3>(red, vals, sm);
  grid_finish<3>(rb, rhs, sbe, nblk_site, vals);
}

// ------------------------------------------------------------------------------------
// The smoother's FP16 storage (FP32 arithmetic).  out16 (+ per-site norms) = [b -] D in, with
// in FP32 native (IN16 = 0) or FP16 with norms (IN16 = 1) and b FP32 native; the scale of an
// FP16 neighbour enters the accumulation of its hop.  RED = 2: per rhs {<out, in>, |out|^2}
// from the FP32 values before rounding.
// ------------------------------------------------------------------------------------
template <int IN16, int RED, int GC>
__global__ void __launch_bounds__(128) k_dslash_h(void* __restrict__ out16, float* __restrict__ out_norm,
                                                  const void* __restrict__ in, const float* __restrict__ in_norm,
                                                  const void* __restrict__ b, const void* __restrict__ gauge, Geom g,
                                                  const double* __restrict__ mass, const int* __restrict__ active,
                                                  int nrhs, int nblk_site, RedBuf rb) {
  const int rhs = blockIdx.x % nrhs;
  const int sb = blockIdx.x / nrhs;
  if (active && !active[rhs]) return;  // whole CTA exits together (uniform per CTA)
  const int v = sb * blockDim.x + threadIdx.x;
  const size_t fbi = IN16 ? spinor_h_bytes(g.V) : spinor_field_bytes<float>(g.V);
  const char* inr = reinterpret_cast<const char*>(in) + fbi * rhs;
  const float* inn = IN16 ? in_norm + (size_t)g.V * rhs : nullptr;
  cpx<float> acc[12];
  float red[3] = {0.f, 0.f, 0.f};
  if (v < g.V) {
#pragma unroll
    for (int i = 0; i < 12; ++i) acc[i] = cpx<float>{0.f, 0.f};
    int c[4];
    site_coords(g, v, c);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      cpx<float> u[9], nb[12];
      const int vf = neighbour(g, v, c, mu, +1);
      load_link_gc<float, GC>(gauge, g.V, mu, v, u);
      if (IN16) {
        load_spinor_h(inr, g.V, vf, nb);
        hop_accumulate_scaled<+1>(mu, u, nb, __ldg(inn + vf), acc);
      } else {
        load_spinor<float>(inr, g.V, vf, nb);
        hop_accumulate<+1>(mu, u, nb, acc);
      }
      const int vb = neighbour(g, v, c, mu, -1);
      load_link_gc<float, GC>(gauge, g.V, mu, vb, u);
      if (IN16) {
        load_spinor_h(inr, g.V, vb, nb);
        hop_accumulate_scaled<-1>(mu, u, nb, __ldg(inn + vb), acc);
      } else {
        load_spinor<float>(inr, g.V, vb, nb);
        hop_accumulate<-1>(mu, u, nb, acc);
      }
    }
    cpx<float> self[12];
    if (IN16) {
      load_spinor_h(inr, g.V, v, self);
      const float sc = __ldg(inn + v);
#pragma unroll
      for (int i = 0; i < 12; ++i) self[i] = sc * self[i];
    } else {
      load_spinor<float>(inr, g.V, v, self);
    }
    const float diag = float(4.0 + mass[rhs]);
#pragma unroll
    for (int i = 0; i < 12; ++i)
      acc[i] = cpx<float>{fmaf(diag, self[i].re, -0.5f * acc[i].re), fmaf(diag, self[i].im, -0.5f * acc[i].im)};
    if (b) {
      cpx<float> bb[12];
      load_spinor<float>(reinterpret_cast<const char*>(b) + spinor_field_bytes<float>(g.V) * rhs, g.V, v, bb);
#pragma unroll
      for (int i = 0; i < 12; ++i) acc[i] = bb[i] - acc[i];
    }
    store_spinor_h(reinterpret_cast<char*>(out16) + spinor_h_bytes(g.V) * rhs, out_norm + (size_t)g.V * rhs, g.V, v,
                   acc);
    if (RED == 2) {
      float a0 = 0.f, a1 = 0.f, nn = 0.f;
#pragma unroll
      for (int i = 0; i < 12; ++i) {
        cdot_acc(a0, a1, acc[i], self[i]);
        norm2_acc(nn, acc[i]);
      }
      red[0] = a0;
      red[1] = a1;
      red[2] = nn;
    }
  }
  if constexpr (RED == 2) {
    __shared__ double sm[32 * 3];
    double vals[3];
    cta_reduce_mixed<float, 3>(red, vals, sm);
    grid_finish<3>(rb, rhs, sb, nblk_site, vals);
  }
}

// x += alpha r and (update_r) r -= alpha q, alpha = red[0..1] / red[2] per rhs; x FP32 native,
// r and q FP16 with per-site norms.  Thread per (site, rhs).
__global__ void k_mr_update_h(void* __restrict__ x, void* __restrict__ r16, float* __restrict__ rn,
                              const void* __restrict__ q16, const float* __restrict__ qn, int V,
                              const double* __restrict__ red, const int* __restrict__ active, int update_r) {
  const int rhs = blockIdx.y;
  if (active && !active[rhs]) return;
  const double qq = red[rhs * 3 + 2];
  if (!(qq > 0.0)) return;
  float sc[2];
  cta_scalars<float, 2>(sc, [&](double* v) {
    v[0] = red[rhs * 3 + 0] / qq;
    v[1] = red[rhs * 3 + 1] / qq;
  });
  const cpx<float> al{sc[0], sc[1]};
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  const size_t fh = spinor_h_bytes(V), ff = spinor_field_bytes<float>(V);
  char* rr = reinterpret_cast<char*>(r16) + fh * rhs;
  char* xr = reinterpret_cast<char*>(x) + ff * rhs;
  cpx<float> rv[12], xv[12];
  load_spinor_h(rr, V, v, rv);
  const float rs = rn[(size_t)V * rhs + v];
  load_spinor<float>(xr, V, v, xv);
#pragma unroll
  for (int i = 0; i < 12; ++i) {
    rv[i] = rs * rv[i];
    cfma(xv[i], al, rv[i]);
  }
  store_spinor<float>(xr, V, v, xv);
  if (!update_r) return;
  cpx<float> qv[12];
  load_spinor_h(reinterpret_cast<const char*>(q16) + fh * rhs, V, v, qv);
  const float qs = qn[(size_t)V * rhs + v];
#pragma unroll
  for (int i = 0; i < 12; ++i) rv[i] = rv[i] - (qs * al) * qv[i];
  store_spinor_h(rr, rn + (size_t)V * rhs, V, v, rv);
}

// native FP32 <-> FP16 with per-site norms (test entry point)
__global__ void k_spinor_to_h(const void* __restrict__ in, void* __restrict__ out16, float* __restrict__ norm, int V) {
  const int rhs = blockIdx.y, v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  cpx<float> t[12];
  load_spinor<float>(reinterpret_cast<const char*>(in) + spinor_field_bytes<float>(V) * rhs, V, v, t);
  store_spinor_h(reinterpret_cast<char*>(out16) + spinor_h_bytes(V) * rhs, norm + (size_t)V * rhs, V, v, t);
}
__global__ void k_spinor_from_h(const void* __restrict__ in16, const float* __restrict__ norm, void* __restrict__ out,
                                int V) {
  const int rhs = blockIdx.y, v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= V) return;
  cpx<float> t[12];
  load_spinor_h(reinterpret_cast<const char*>(in16) + spinor_h_bytes(V) * rhs, V, v, t);
  const float sc = norm[(size_t)V * rhs + v];
#pragma unroll
  for (int i = 0; i < 12; ++i) t[i] = sc * t[i];
  store_spinor<float>(reinterpret_cast<char*>(out) + spinor_field_bytes<float>(V) * rhs, V, v, t);
}

// ------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------
void pack_gauge(int prec, const double* canon, void* out, int V, cudaStream_t s) {
  count_launch();
  const int T = 256, B = (V + T - 1) / T;
  if (prec == WMG_PREC_DOUBLE) k_pack_gauge<double><<<B, T, 0, s>>>((const double2*)canon, out, V);
  else k_pack_gauge<float><<<B, T, 0, s>>>((const double2*)canon, out, V);
}

void pack_gauge8(const void* g64, void* out, int V, int* degenerate, cudaStream_t s) {
  count_launch();
  const int T = 256, B = (V + T - 1) / T;
  k_pack_gauge8<<<B, T, 0, s>>>(g64, (float4*)out, V, degenerate);
}

void pack_gauge18(const void* g64, void* out, int V, cudaStream_t s) {
  count_launch();
  const int T = 256, B = (V + T - 1) / T;
  k_pack_gauge18<<<B, T, 0, s>>>(g64, (float4*)out, V);
}

void pack_spinor(int prec, const double* canon, void* out, int V, int nrhs, cudaStream_t s) {
  count_launch();
  const size_t n = (size_t)V * nrhs;
  const int T = 256;
  const unsigned B = (unsigned)((n + T - 1) / T);
  if (prec == WMG_PREC_DOUBLE) k_pack_spinor<double><<<B, T, 0, s>>>((const double2*)canon, out, V, nrhs);
  else k_pack_spinor<float><<<B, T, 0, s>>>((const double2*)canon, out, V, nrhs);
}

void unpack_spinor(int prec, const void* in, double* canon, int V, int nrhs, cudaStream_t s) {
  count_launch();
  const size_t n = (size_t)V * nrhs;
  const int T = 256;
  const unsigned B = (unsigned)((n + T - 1) / T);
  if (prec == WMG_PREC_DOUBLE) k_unpack_spinor<double><<<B, T, 0, s>>>(in, (double2*)canon, V, nrhs);
  else k_unpack_spinor<float><<<B, T, 0, s>>>(in, (double2*)canon, V, nrhs);
}

int dslash_blocks(int V) { return (V + kDslashThreads - 1) / kDslashThreads; }

void dslash(int prec, void* out, const void* in, const void* b, const void* gauge, const Geom& g,
            const double* mass_dev, const int* active, int nrhs, int red, const RedBuf* rb, cudaStream_t s,
            int gc, int b_half) {
  count_launch();
  const int nb = dslash_blocks(g.V);
  const int spb = prec == WMG_PREC_DOUBLE ? dslash_spb<double, 1>() : dslash_spb<float, 1>();
  const int nbr = (nb + spb - 1) / spb;  // CTAs per rhs with RED > 0
  const unsigned grid = (unsigned)nb * nrhs, gridr = (unsigned)nbr * nrhs;
  RedBuf r = rb ? *rb : RedBuf{nullptr, nullptr, nullptr};
  const DslashDiv dv{make_fastdiv(g.L[0]), make_fastdiv(g.L[1]), make_fastdiv(g.L[2])};
#define WMG_DS(R, GC)                                                                                         \
  do {                                                                                                        \
    if (red == 0) k_dslash<R, 0, GC><<<grid, kDslashThreads, 0, s>>>(out, in, b, gauge, g, dv, mass_dev, active, nrhs, nb, r, b_half); \
    else if (red == 1) k_dslash<R, 1, GC><<<gridr, kDslashThreads, 0, s>>>(out, in, b, gauge, g, dv, mass_dev, active, nrhs, nbr, r, b_half); \
    else k_dslash<R, 2, GC><<<gridr, kDslashThreads, 0, s>>>(out, in, b, gauge, g, dv, mass_dev, active, nrhs, nbr, r, b_half); \
  } while (0)
  if (prec == WMG_PREC_DOUBLE) WMG_DS(double, 12);
  else if (gc == 8) WMG_DS(float, 8);
  else if (gc == 18) WMG_DS(float, 18);
  else WMG_DS(float, 12);
#undef WMG_DS
}

void dslash_mr(int prec, void* out, const void* r, const void* q, void* r_out, void* x, const double* red_prev,
               const void* gauge, const Geom& g, const double* mass_dev, const int* active, int nrhs,
               const RedBuf& rb, cudaStream_t s, int gc) {
  count_launch();
  const int nb = dslash_blocks(g.V);
  const int spb = prec == WMG_PREC_DOUBLE ? dslash_spb<double, 2>() : dslash_spb<float, 2>();
  const int nbr = (nb + spb - 1) / spb;
  const unsigned grid = (unsigned)nbr * nrhs;
  const DslashDiv dv{make_fastdiv(g.L[0]), make_fastdiv(g.L[1]), make_fastdiv(g.L[2])};
  if (prec == WMG_PREC_DOUBLE)
    k_dslash_mr<double, 12><<<grid, kDslashThreads, 0, s>>>(out, r, q, r_out, x, red_prev, gauge, g, dv, mass_dev,
                                                             active, nrhs, nbr, rb);
  else if (gc == 8)
    k_dslash_mr<float, 8><<<grid, kDslashThreads, 0, s>>>(out, r, q, r_out, x, red_prev, gauge, g, dv, mass_dev,
                                                           active, nrhs, nbr, rb);
  else if (gc == 18)
    k_dslash_mr<float, 18><<<grid, kDslashThreads, 0, s>>>(out, r, q, r_out, x, red_prev, gauge, g, dv, mass_dev,
                                                            active, nrhs, nbr, rb);
  else
    k_dslash_mr<float, 12><<<grid, kDslashThreads, 0, s>>>(out, r, q, r_out, x, red_prev, gauge, g, dv, mass_dev,
                                                            active, nrhs, nbr, rb);
}

template <int GC>
static void launch_dslash_h(int in16, void* out16, float* out_norm, const void* in, const float* in_norm,
                            const void* b, const void* gauge, const Geom& g, const double* mass_dev,
                            const int* active, int nrhs, int red, const RedBuf& r, cudaStream_t s) {
  const int nb = dslash_blocks(g.V);
  const unsigned grid = (unsigned)nb * nrhs;
  if (in16) {
    if (red == 2) k_dslash_h<1, 2, GC><<<grid, kDslashThreads, 0, s>>>(out16, out_norm, in, in_norm, b, gauge, g, mass_dev, active, nrhs, nb, r);
    else k_dslash_h<1, 0, GC><<<grid, kDslashThreads, 0, s>>>(out16, out_norm, in, in_norm, b, gauge, g, mass_dev, active, nrhs, nb, r);
  } else {
    if (red == 2) k_dslash_h<0, 2, GC><<<grid, kDslashThreads, 0, s>>>(out16, out_norm, in, in_norm, b, gauge, g, mass_dev, active, nrhs, nb, r);
    else k_dslash_h<0, 0, GC><<<grid, kDslashThreads, 0, s>>>(out16, out_norm, in, in_norm, b, gauge, g, mass_dev, active, nrhs, nb, r);
  }
}

void dslash_h(int in16, void* out16, float* out_norm, const void* in, const float* in_norm, const void* b,
              const void* gauge, const Geom& g, const double* mass_dev, const int* active, int nrhs, int red,
              const RedBuf* rb, cudaStream_t s, int gc) {
  count_launch();
  RedBuf r = rb ? *rb : RedBuf{nullptr, nullptr, nullptr};
  if (gc == 8) launch_dslash_h<8>(in16, out16, out_norm, in, in_norm, b, gauge, g, mass_dev, active, nrhs, red, r, s);
  else if (gc == 18)
    launch_dslash_h<18>(in16, out16, out_norm, in, in_norm, b, gauge, g, mass_dev, active, nrhs, red, r, s);
  else launch_dslash_h<12>(in16, out16, out_norm, in, in_norm, b, gauge, g, mass_dev, active, nrhs, red, r, s);
}

void mr_update_h(void* x, void* r16, float* rn, const void* q16, const float* qn, int V, int nrhs, const double* red,
                 const int* active, bool update_r, cudaStream_t s) {
  count_launch();
  dim3 grid((V + 127) / 128, nrhs);
  k_mr_update_h<<<grid, 128, 0, s>>>(x, r16, rn, q16, qn, V, red, active, update_r ? 1 : 0);
}

void spinor_to_h(const void* in, void* out16, float* norm, int V, int nrhs, cudaStream_t s) {
  count_launch();
  dim3 grid((V + 127) / 128, nrhs);
  k_spinor_to_h<<<grid, 128, 0, s>>>(in, out16, norm, V);
}

void spinor_from_h(const void* in16, const float* norm, void* out, int V, int nrhs, cudaStream_t s) {
  count_launch();
  dim3 grid((V + 127) / 128, nrhs);
  k_spinor_from_h<<<grid, 128, 0, s>>>(in16, norm, out, V);
}

}  // namespace wmg
