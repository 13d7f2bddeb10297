// Common device/host helpers of libwmg: complex arithmetic, lattice geometry,
// native field layouts and the deterministic reduction scheme.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cstdint>
#include <cstddef>

#include "wmg.h"

#define WMG_HD __host__ __device__ __forceinline__
#define WMG_D __device__ __forceinline__

// ---------------------------------------------------------------------------------
// complex numbers
// ---------------------------------------------------------------------------------
template <typename R>
struct cpx {
  R re, im;
};
using cd = cpx<double>;
using cf = cpx<float>;

template <typename R> WMG_HD cpx<R> operator+(cpx<R> a, cpx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> WMG_HD cpx<R> operator-(cpx<R> a, cpx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> WMG_HD cpx<R> operator-(cpx<R> a) { return {-a.re, -a.im}; }
template <typename R> WMG_HD cpx<R> operator*(cpx<R> a, cpx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> WMG_HD cpx<R> operator*(R s, cpx<R> a) { return {s * a.re, s * a.im}; }
template <typename R> WMG_HD cpx<R>& operator+=(cpx<R>& a, cpx<R> b) {
  a.re += b.re;
  a.im += b.im;
  return a;
}
template <typename R> WMG_HD cpx<R>& operator-=(cpx<R>& a, cpx<R> b) {
  a.re -= b.re;
  a.im -= b.im;
  return a;
}
template <typename R> WMG_HD cpx<R> conj(cpx<R> a) { return {a.re, -a.im}; }
// conj(a) * b
template <typename R> WMG_HD cpx<R> cmulc(cpx<R> a, cpx<R> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// acc += a * b
template <typename R> WMG_HD void cfma(cpx<R>& acc, cpx<R> a, cpx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc += conj(a) * b
template <typename R> WMG_HD void cfmac(cpx<R>& acc, cpx<R> a, cpx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}
// acc -= c * b
template <typename R> WMG_HD void cfms(cpx<R>& acc, cpx<R> c, cpx<R> b) {
  acc.re = fma(-c.re, b.re, acc.re);
  acc.re = fma(c.im, b.im, acc.re);
  acc.im = fma(-c.re, b.im, acc.im);
  acc.im = fma(-c.im, b.re, acc.im);
}
template <typename R> WMG_HD R norm2(cpx<R> a) { return a.re * a.re + a.im * a.im; }
// re += Re(conj(a) b), im += Im(conj(a) b) as FMA chains (4 operations instead of 6)
template <typename R> WMG_HD void cdot_acc(R& re, R& im, cpx<R> a, cpx<R> b) {
  re = fma(a.re, b.re, re);
  re = fma(a.im, b.im, re);
  im = fma(a.re, b.im, im);
  im = fma(-a.im, b.re, im);
}
// t += |a|^2 as two FMAs (a.re * a.re + a.im * a.im, then the add, is three operations)
template <typename R> WMG_HD void norm2_acc(R& t, cpx<R> a) {
  t = fma(a.re, a.re, t);
  t = fma(a.im, a.im, t);
}
template <typename T, typename R> WMG_HD cpx<T> ccast(cpx<R> a) { return {T(a.re), T(a.im)}; }

// multiply by a unit phase: ph = 0 -> 1, 1 -> i, 2 -> -1, 3 -> -i
template <typename R> WMG_HD cpx<R> mul_phase(cpx<R> a, int ph) {
  switch (ph & 3) {
    case 0: return a;
    case 1: return {-a.im, a.re};
    case 2: return {-a.re, -a.im};
    default: return {a.im, -a.re};
  }
}

// ---------------------------------------------------------------------------------
// lattice geometry
// ---------------------------------------------------------------------------------
struct Geom {
  int L[4];  // X, Y, Z, T
  int V;
};

// n / d for 0 <= n < 2^31 by multiply-high and shift (Granlund & Montgomery 1994, the
// round-up multiplier with the extra add): l = ceil(log2 d), m = floor(2^32 (2^l - d) / d) + 1,
// q = (mulhi(n, m) + n) >> l.
struct FastDiv {
  uint32_t d, m, l;
};
inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  f.l = 0;
  while ((1ull << f.l) < d) ++f.l;
  f.m = (uint32_t)((((1ull << 32) * ((1ull << f.l) - d)) / d) + 1);
  return f;
}
WMG_D uint32_t fdiv(uint32_t n, const FastDiv& f) { return (__umulhi(n, f.m) + n) >> f.l; }

inline Geom make_geom(const int d[4]) {
  Geom g;
  for (int i = 0; i < 4; ++i) g.L[i] = d[i];
  g.V = d[0] * d[1] * d[2] * d[3];
  return g;
}

WMG_HD void site_coords(const Geom& g, int v, int c[4]) {
  c[0] = v % g.L[0];
  v /= g.L[0];
  c[1] = v % g.L[1];
  v /= g.L[1];
  c[2] = v % g.L[2];
  c[3] = v / g.L[2];
}
// the k-th site (lexicographic order) of parity p = (x + y + z + t) mod 2; L[0] even, so the
// sites 2k and 2k + 1 share y, z, t and exactly one of them has parity p
WMG_HD int parity_site(const Geom& g, int k, int p) {
  int c[4];
  site_coords(g, 2 * k, c);
  return 2 * k + ((p + c[0] + c[1] + c[2] + c[3]) & 1);
}
WMG_HD int site_index(const Geom& g, const int c[4]) {
  return c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
}
WMG_HD int dir_stride(const Geom& g, int mu) {
  int s = 1;
  for (int i = 0; i < mu; ++i) s *= g.L[i];
  return s;
}
// neighbour of site v (coordinates c) in direction mu, sign +1/-1, periodic
WMG_HD int neighbour(const Geom& g, int v, const int c[4], int mu, int sign) {
  const int stride = dir_stride(g, mu);
  const int x = c[mu];
  if (sign > 0) return (x + 1 == g.L[mu]) ? v - (g.L[mu] - 1) * stride : v + stride;
  return (x == 0) ? v + (g.L[mu] - 1) * stride : v - stride;
}

// ---------------------------------------------------------------------------------
// native fine spinor layout: [rhs][6][V] chunks of two complex numbers.
// chunk c of site v holds the components k = 2c, 2c+1 (k = 3*spin + colour).
// ---------------------------------------------------------------------------------
template <typename R> struct Chunk2;
template <> struct Chunk2<float> {
  WMG_D static void load(const void* base, size_t idx, cf& a, cf& b) {
    float4 t = __ldg(reinterpret_cast<const float4*>(base) + idx);
    a = {t.x, t.y};
    b = {t.z, t.w};
  }
  WMG_D static void load_cg(const void* base, size_t idx, cf& a, cf& b) {  // no read-only path
    float4 t = reinterpret_cast<const float4*>(base)[idx];
    a = {t.x, t.y};
    b = {t.z, t.w};
  }
  WMG_D static void store(void* base, size_t idx, cf a, cf b) {
    reinterpret_cast<float4*>(base)[idx] = make_float4(a.re, a.im, b.re, b.im);
  }
};
template <> struct Chunk2<double> {
  WMG_D static void load(const void* base, size_t idx, cd& a, cd& b) {
    const double2* p = reinterpret_cast<const double2*>(base) + 2 * idx;
    double2 t0 = __ldg(p), t1 = __ldg(p + 1);
    a = {t0.x, t0.y};
    b = {t1.x, t1.y};
  }
  WMG_D static void load_cg(const void* base, size_t idx, cd& a, cd& b) {
    const double2* p = reinterpret_cast<const double2*>(base) + 2 * idx;
    double2 t0 = p[0], t1 = p[1];
    a = {t0.x, t0.y};
    b = {t1.x, t1.y};
  }
  WMG_D static void store(void* base, size_t idx, cd a, cd b) {
    double2* p = reinterpret_cast<double2*>(base) + 2 * idx;
    p[0] = make_double2(a.re, a.im);
    p[1] = make_double2(b.re, b.im);
  }
};

template <typename R>
WMG_D void load_spinor(const void* base, int V, int v, cpx<R> s[12]) {
#pragma unroll
  for (int c = 0; c < 6; ++c) Chunk2<R>::load(base, (size_t)c * V + v, s[2 * c], s[2 * c + 1]);
}
template <typename R>
WMG_D void store_spinor(void* base, int V, int v, const cpx<R> s[12]) {
#pragma unroll
  for (int c = 0; c < 6; ++c) Chunk2<R>::store(base, (size_t)c * V + v, s[2 * c], s[2 * c + 1]);
}
// byte offset of right-hand side r of a native fine field
template <typename R> WMG_HD size_t spinor_field_bytes(int V) { return (size_t)V * 12 * 2 * sizeof(R); }

// FP16 fine spinor with a per-site scale (the smoother's storage): [rhs][6][V] chunks of two
// complex numbers as __half2 (re, im) pairs (8 bytes) plus norm[rhs][V] = max |Re|, |Im| of the
// site's 24 reals; stored values are the components divided by the norm.
WMG_HD size_t spinor_h_bytes(int V) { return (size_t)V * 6 * 8; }
WMG_D void load_spinor_h(const void* base, int V, int v, cpx<float> s[12]) {
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const uint2 t = __ldg(reinterpret_cast<const uint2*>(base) + (size_t)c * V + v);
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&t.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&t.y));
    s[2 * c] = {a.x, a.y};
    s[2 * c + 1] = {b.x, b.y};
  }
}
// s / norm rounded to FP16; returns the norm written
WMG_D float store_spinor_h(void* base, float* norm, int V, int v, const cpx<float> s[12]) {
  float m = 0.f;
#pragma unroll
  for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf(s[k].re), fabsf(s[k].im)));
  const float inv = m > 0.f ? 1.f / m : 0.f;
#pragma unroll
  for (int c = 0; c < 6; ++c) {
    const __half2 a = __floats2half2_rn(s[2 * c].re * inv, s[2 * c].im * inv);
    const __half2 b = __floats2half2_rn(s[2 * c + 1].re * inv, s[2 * c + 1].im * inv);
    uint2 t;
    t.x = *reinterpret_cast<const unsigned*>(&a);
    t.y = *reinterpret_cast<const unsigned*>(&b);
    reinterpret_cast<uint2*>(base)[(size_t)c * V + v] = t;
  }
  norm[v] = m;
  return m;
}

// native gauge layout: [mu][3][V] chunks (rows 0 and 1 of U_mu(x), element e = 3*row + col,
// chunk c holds e = 2c, 2c+1); row 2 = conj(row0 x row1) is rebuilt on load.
template <typename R>
WMG_D void load_link(const void* base, int V, int mu, int v, cpx<R> u[9]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) Chunk2<R>::load(base, (size_t)(mu * 3 + c) * V + v, u[2 * c], u[2 * c + 1]);
  u[6] = conj(u[1] * u[5] - u[2] * u[4]);
  u[7] = conj(u[2] * u[3] - u[0] * u[5]);
  u[8] = conj(u[0] * u[4] - u[1] * u[3]);
}

// 8-real FP32 links (the "8 floats" gauge storage): [mu][2][V] float4, chunk 0 = (a1, a2) =
// elements (0,1), (0,2); chunk 1 = (b0, theta_a0, theta_c0) = element (1,0) and the phases of
// elements (0,0) and (2,0).  Rebuilt from unitarity with det U = 1: |a0|^2 = 1 - |a1|^2 - |a2|^2,
// |c0|^2 = 1 - |a0|^2 - |b0|^2 (column 0), and, with n = |a1|^2 + |a2|^2, the 2 x 2 systems of
// row 1 (resp. row 2) orthogonal to row 0 and the cofactor relations conj(c0) = a1 b2 - a2 b1,
// conj(b0) = a2 c1 - a1 c2 (U^-1 = U^dag = adj U), solved by Cramer's rule:
//   b1 = -(a1 b0 conj(a0) + conj(a2) conj(c0)) / n,  b2 = (conj(a1) conj(c0) - a2 b0 conj(a0)) / n,
//   c1 = (conj(a2) conj(b0) - a1 c0 conj(a0)) / n,   c2 = -(a2 c0 conj(a0) + conj(a1) conj(b0)) / n.
WMG_HD size_t gauge8_bytes(int V) { return (size_t)V * 4 * 2 * sizeof(float4); }
WMG_D void load_link8(const void* base, int V, int mu, int v, cpx<float> u[9]) {
  const float4 t0 = __ldg(reinterpret_cast<const float4*>(base) + (size_t)(mu * 2) * V + v);
  const float4 t1 = __ldg(reinterpret_cast<const float4*>(base) + (size_t)(mu * 2 + 1) * V + v);
  const cpx<float> a1{t0.x, t0.y}, a2{t0.z, t0.w}, b0{t1.x, t1.y};
  const float n = a1.re * a1.re + a1.im * a1.im + a2.re * a2.re + a2.im * a2.im;
  const float ra = sqrtf(fmaxf(1.f - n, 0.f));
  const float rc = sqrtf(fmaxf(n - (b0.re * b0.re + b0.im * b0.im), 0.f));  // 1 - |a0|^2 - |b0|^2
  float sa, ca, sc, cc;
  __sincosf(t1.z, &sa, &ca);
  __sincosf(t1.w, &sc, &cc);
  const cpx<float> a0{ra * ca, ra * sa}, c0{rc * cc, rc * sc};
  const float in = 1.f / n;
  const cpx<float> b0a0 = b0 * conj(a0), c0a0 = c0 * conj(a0);
  const cpx<float> b1 = -in * (a1 * b0a0 + conj(a2) * conj(c0));
  const cpx<float> b2 = in * (conj(a1) * conj(c0) - a2 * b0a0);
  const cpx<float> c1 = in * (conj(a2) * conj(b0) - a1 * c0a0);
  const cpx<float> c2 = -in * (a2 * c0a0 + conj(a1) * conj(b0));
  u[0] = a0, u[1] = a1, u[2] = a2;
  u[3] = b0, u[4] = b1, u[5] = b2;
  u[6] = c0, u[7] = c1, u[8] = c2;
}
// 18-real FP32 links (all nine elements stored; row 2 rebuilt once, in FP64, when packed):
// [mu][4][V] float4 chunks of elements (0, 1), (2, 3), (4, 5), (6, 7), then [mu][V] float2 of
// element 8 after the 16 V chunks.  Loading costs no arithmetic.
WMG_HD size_t gauge18_bytes(int V) { return (size_t)V * 4 * (4 * sizeof(float4) + sizeof(float2)); }
WMG_D void load_link18(const void* base, int V, int mu, int v, cpx<float> u[9]) {
  const float4* q = reinterpret_cast<const float4*>(base);
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float4 t = __ldg(q + (size_t)(mu * 4 + c) * V + v);
    u[2 * c] = {t.x, t.y};
    u[2 * c + 1] = {t.z, t.w};
  }
  const float2 t8 = __ldg(reinterpret_cast<const float2*>(q + (size_t)16 * V) + (size_t)mu * V + v);
  u[8] = {t8.x, t8.y};
}
// the link loader of a dslash kernel: 12-real in the kernel's precision, or FP32 8-real (GC = 8)
// or 18-real (GC = 18)
template <typename R, int GC>
WMG_D void load_link_gc(const void* base, int V, int mu, int v, cpx<R> u[9]) {
  if constexpr (GC == 8) load_link8(base, V, mu, v, u);
  else if constexpr (GC == 18) load_link18(base, V, mu, v, u);
  else load_link<R>(base, V, mu, v, u);
}

// ---------------------------------------------------------------------------------
// deterministic reductions: each CTA writes its partial sums (double) for its rhs;
// the last CTA of that rhs (counter) sums the partials in index order.
// ---------------------------------------------------------------------------------
struct RedBuf {
  double* partial;    // [nrhs][nblk][nval]
  unsigned* counter;  // [nrhs], zero between uses
  double* result;     // [nrhs][nval]
};

// Sum of NVAL values over a warp by recursive halving (NVAL <= 32, padded with zeros to P = 2^M):
// at each of the first M levels a lane keeps the half of its values that the lane bit selects and
// adds its partner's copy of that half, so the warp needs P - 1 + 5 - M additions and as many
// shuffles per lane instead of 5 NVAL.  On return s is the warp's sum of value idx, held by the
// 32 / P lanes with idx = lane >> (5 - M).  The order of the additions is fixed, and a + b = b + a,
// so both partners hold identical sums.
template <int NVAL>
constexpr int warp_reduce_levels() {
  return NVAL <= 1 ? 0 : NVAL <= 2 ? 1 : NVAL <= 4 ? 2 : NVAL <= 8 ? 3 : NVAL <= 16 ? 4 : 5;
}
template <typename T, int NVAL>
WMG_D void warp_reduce_multi(const T v[NVAL], T& s, int& idx) {
  constexpr int M = warp_reduce_levels<NVAL>();
  constexpr int P = 1 << M;
  static_assert(NVAL >= 1 && NVAL <= 32, "warp_reduce_multi: 1 <= NVAL <= 32");
  const int lane = threadIdx.x & 31;
  T w[P];
#pragma unroll
  for (int i = 0; i < P; ++i) w[i] = i < NVAL ? v[i] : T(0);
#pragma unroll
  for (int lev = 0; lev < 5; ++lev) {
    const int o = 16 >> lev;
    if (lev < M) {
      const int h = P >> (lev + 1);
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int i = 0; i < h; ++i) {
        const T send = up ? w[i] : w[i + h];
        const T keep = up ? w[i + h] : w[i];
        w[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    } else {
      w[0] += __shfl_xor_sync(0xffffffffu, w[0], o);
    }
  }
  s = w[0];
  idx = (lane >> (5 - M)) & (P - 1);
}

// Reduce NVAL doubles across the CTA (blockDim.x a multiple of 32, <= 1024); the result is
// valid in thread 0.  Fixed summation order: warp_reduce_multi within each warp, then the warps in
// index order (thread i combines value i).
template <int NVAL>
WMG_D void cta_reduce(double v[NVAL], double* smem /* >= 32*NVAL */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double ws;
  int idx;
  warp_reduce_multi<double, NVAL>(v, ws, idx);
  if (idx < NVAL && lane == (idx << (5 - warp_reduce_levels<NVAL>())))
    smem[warp * NVAL + idx] = ws;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x < NVAL) {
    for (int w = 0; w < nw; ++w) tot += smem[w * NVAL + threadIdx.x];
  }
  __syncthreads();
  if (threadIdx.x < NVAL) smem[threadIdx.x] = tot;
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int i = 0; i < NVAL; ++i) v[i] = smem[i];
  __syncthreads();
}

// As cta_reduce, for per-thread values in the kernel's own precision T: the sums within each warp
// run in T, the warps' results are summed in FP64 in index order (the same fixed shape), result
// in out[] of thread 0.  An FP32 kernel so keeps its reductions off the FP64 pipe (1/64 of the
// FP32 rate on B300) except for one sum per warp; for T = double it is cta_reduce.
template <typename T, int NVAL>
WMG_D void cta_reduce_mixed(T v[NVAL], double out[NVAL], double* smem /* >= 32*NVAL */) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T ws;
  int idx;
  warp_reduce_multi<T, NVAL>(v, ws, idx);
  if (idx < NVAL && lane == (idx << (5 - warp_reduce_levels<NVAL>())))
    smem[warp * NVAL + idx] = double(ws);
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x < NVAL) {
    for (int w = 0; w < nw; ++w) tot += smem[w * NVAL + threadIdx.x];
  }
  __syncthreads();
  if (threadIdx.x < NVAL) smem[threadIdx.x] = tot;
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int i = 0; i < NVAL; ++i) out[i] = smem[i];
  __syncthreads();
}

// NS per-rhs scalars of a vector kernel (f fills them in FP64), formed once per CTA by thread 0
// and read by every thread from shared memory.  FP64 division and square root cost tens of
// FP64-pipe operations on B300, which every thread would otherwise repeat.  The values are those
// each thread would have formed itself.  Call once per kernel, from every thread of the CTA.
template <typename R, int NS, typename F>
WMG_D void cta_scalars(R out[NS], F f) {
  __shared__ R sv[NS];
  if (threadIdx.x == 0) {
    double v[NS];
    f(v);
#pragma unroll
    for (int i = 0; i < NS; ++i) sv[i] = R(v[i]);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NS; ++i) out[i] = sv[i];
}

// Sum p[b * stride], b < count, over the whole CTA in a fixed order (thread t takes
// b = t, t + blockDim, ...; then the fixed-shape tree of cta_reduce).  Valid in thread 0.
WMG_D double cta_sum_strided(const volatile double* p, int count, int stride, double* smem /* >= 32 */) {
  double s[1] = {0.0};
  for (int b = threadIdx.x; b < count; b += blockDim.x) s[0] += p[(size_t)b * stride];
  cta_reduce<1>(s, smem);
  return s[0];
}

// Sums of nval rows of partials at once: value i is sum_b p[i * istride + b * bstride], b < count.
// Warp w takes values w, w + nwarps, ...; lane l adds b = l, l + 32, ... in order, then a fixed
// xor-shuffle tree; lane 0 hands (i, sum) to `store`.  The order depends on count only.  The
// partials come from other CTAs (written before their counter increment): they are read from
// L2 (ld.global.cg), eight per lane in flight before the additions, in the same order.
constexpr int kSumBatch = 8;
template <typename F>
WMG_D void cta_multi_sum(const volatile double* pv, int nval, size_t istride, int count, size_t bstride, F store) {
  const double* p = const_cast<const double*>(pv);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < nval; i += nw) {
    double s = 0.0;
    const double* row = p + i * istride;
    for (int b0 = lane; b0 < count; b0 += 32 * kSumBatch) {
      double t[kSumBatch];
#pragma unroll
      for (int u = 0; u < kSumBatch; ++u) {
        const int b = b0 + 32 * u;
        t[u] = b < count ? __ldcg(row + (size_t)b * bstride) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kSumBatch; ++u)
        if (b0 + 32 * u < count) s += t[u];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) store(i, s);
  }
}

// After cta_reduce (thread 0 holds v): writes the CTA's partials; the last CTA for `rhs`
// sums all partials (fixed order, whole CTA, all values in parallel) into rb.result.
// nblk = CTAs per rhs.  May be called several times in a row by one CTA.
// Returns true in the CTA that completed the sums (whose threads then see rb.result after a
// barrier).
template <int NVAL>
WMG_D bool grid_finish(const RedBuf& rb, int rhs, int blk, int nblk, const double v[NVAL]) {
  __shared__ bool last;
  __syncthreads();  // `last` of a previous call has been read by every thread
  if (threadIdx.x == 0) {
    double* p = rb.partial + ((size_t)rhs * nblk + blk) * NVAL;
#pragma unroll
    for (int i = 0; i < NVAL; ++i) p[i] = v[i];
    __threadfence();
    unsigned prev = atomicAdd(rb.counter + rhs, 1u);
    last = (prev == (unsigned)nblk - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    const volatile double* p = rb.partial + (size_t)rhs * nblk * NVAL;
    double* res = rb.result + (size_t)rhs * NVAL;
    cta_multi_sum(p, NVAL, 1, nblk, NVAL, [&](int i, double s) { res[i] = s; });
    if (threadIdx.x == 0) rb.counter[rhs] = 0u;
  }
  return last;
}

#define WMG_CUDA_TRY(expr)                                      \
  do {                                                          \
    cudaError_t e_ = (expr);                                    \
    if (e_ != cudaSuccess) return ::wmg_cuda_fail(e_, #expr);   \
  } while (0)

wmg_status wmg_cuda_fail(cudaError_t e, const char* what);
