// Transfer operators between lattice levels (Sec. 2): restriction R = P^dag, prolongation P,
// and the block orthonormalisation that defines P from the near-null vectors, with the
// chirality split sigma_3 P = P gamma_5 of Sec. 3.
//
// On every level the first half of a site's dof has chirality +1 (fine: spins 0, 1 =
// components 0..5; coarse: dof 0..N-1) and the second half chirality -1.  P is stored as N
// fields of the finer lattice (P_alpha, both chiralities in one field); the coarse dof of
// column (s, alpha) is s*N + alpha.
#include <cuda_fp16.h>

#include "kernels.h"

namespace wmg {

// 16-byte asynchronous global -> shared copies (Ampere-style cp.async; completion per group)
WMG_D void cp_async16(void* dst_smem, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
               "l"(src)
               : "memory");
}
WMG_D void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> WMG_D void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }
// two consecutive complex numbers from shared memory (16-byte aligned for float)
WMG_D void lds2(const cpx<float>* p, cpx<float>& a, cpx<float>& b) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  a = {t.x, t.y};
  b = {t.z, t.w};
}
WMG_D void lds2(const cpx<double>* p, cpx<double>& a, cpx<double>& b) {
  a = p[0];
  b = p[1];
}
WMG_D void cp_async8(void* dst_smem, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
               "l"(src)
               : "memory");
}

// Storage of the null vectors P for the transfers: complex in the vectors' precision, or FP16
// (__half2 = re, im) read into FP32.  One component pair (the unit of the native layout) is
// kPair bytes; copy() moves it global -> shared asynchronously, ld2() reads it back widened.
template <typename PT> struct PSt;
template <> struct PSt<cpx<float>> {
  static constexpr int kPair = 16;
  WMG_D static void copy(void* dst, const void* src) { cp_async16(dst, src); }
  WMG_D static void ld2(const cpx<float>* p, cf& a, cf& b) { lds2(p, a, b); }
  WMG_D static cpx<float> zero() { return cf{0.f, 0.f}; }
};
template <> struct PSt<cpx<double>> {
  static constexpr int kPair = 32;
  WMG_D static void copy(void* dst, const void* src) {
    cp_async16(dst, src);
    cp_async16((char*)dst + 16, (const char*)src + 16);
  }
  WMG_D static void ld2(const cpx<double>* p, cd& a, cd& b) { lds2(p, a, b); }
  WMG_D static cpx<double> zero() { return cd{0.0, 0.0}; }
};
template <> struct PSt<__half2> {
  static constexpr int kPair = 8;
  WMG_D static void copy(void* dst, const void* src) { cp_async8(dst, src); }
  WMG_D static void ld2(const __half2* p, cf& a, cf& b) {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    const float2 x = __half22float2(*reinterpret_cast<const __half2*>(&t.x));
    const float2 y = __half22float2(*reinterpret_cast<const __half2*>(&t.y));
    a = {x.x, x.y};
    b = {y.x, y.y};
  }
  WMG_D static __half2 zero() { return __floats2half2_rn(0.f, 0.f); }
};

WMG_D int block_site(const Blocking& bk, int xc, int e) {
  int c[4];
  site_coords(bk.coarse, xc, c);
  int o[4];
  o[0] = e % bk.b[0];
  int t = e / bk.b[0];
  o[1] = t % bk.b[1];
  t /= bk.b[1];
  o[2] = t % bk.b[2];
  o[3] = t / bk.b[2];
  int f[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) f[i] = c[i] * bk.b[i] + o[i];
  return site_index(bk.fine, f);
}

// The e-th even site of block xc, e < bs / 2.  The block's x extent is even, so its sites 2e and
// 2e + 1 are neighbours in x and exactly one of them is even.
WMG_D int even_block_site(const Blocking& bk, int xc, int e) {
  int c[4];
  site_coords(bk.coarse, xc, c);
  const int e2 = 2 * e;
  int o[4];
  o[0] = e2 % bk.b[0];
  int t = e2 / bk.b[0];
  o[1] = t % bk.b[1];
  t /= bk.b[1];
  o[2] = t % bk.b[2];
  o[3] = t / bk.b[2];
  int f[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) f[i] = c[i] * bk.b[i] + o[i];
  const int v = site_index(bk.fine, f);
  return ((f[0] + f[1] + f[2] + f[3]) & 1) ? v + 1 : v;
}

// fine field element (site v, component k) inside one native field
template <typename R>
WMG_D cpx<R>* fine_elem(void* f, int V, int v, int k) {
  return reinterpret_cast<cpx<R>*>(f) + ((size_t)(k >> 1) * V + v) * 2 + (k & 1);
}

// ------------------------------------------------------------------------------------
// restrict, fine level.  CTA per (coarse site, chunk of RC rhs).  The block's spinors are
// staged in shared memory as [r][k][site]; each warp takes a subset of the vectors alpha,
// its lanes stride over the block's sites, and a warp-shuffle reduction gives the two
// chirality components <P_alpha, psi>_s.
// ------------------------------------------------------------------------------------
template <typename R, int RC>
__global__ void k_restrict_fine(const void* __restrict__ P, Blocking bk, const void* __restrict__ in,
                                void* __restrict__ out, int nrhs, const int* __restrict__ active) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<R>* sm = reinterpret_cast<cpx<R>*>(smraw);  // [RC][12][bs]
  const int xc = blockIdx.x, r0 = blockIdx.y * RC;
  const int bs = bk.bs, V = bk.fine.V;
  const size_t fb = spinor_field_bytes<R>(V);
  for (int e = threadIdx.x; e < bs; e += blockDim.x) {
    const int v = block_site(bk, xc, e);
    for (int rr = 0; rr < RC; ++rr) {
      const int r = r0 + rr;
      cpx<R> s[12];
      if (r < nrhs && (!active || active[r])) load_spinor<R>((const char*)in + fb * r, V, v, s);
      else
        for (int k = 0; k < 12; ++k) s[k] = cpx<R>{R(0), R(0)};
      for (int k = 0; k < 12; ++k) sm[((size_t)rr * 12 + k) * bs + e] = s[k];
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int N = bk.N;
  for (int a = warp; a < N; a += nw) {
    const char* Pa = (const char*)P + fb * a;
    cpx<R> acc[RC][2];
#pragma unroll
    for (int rr = 0; rr < RC; ++rr) acc[rr][0] = acc[rr][1] = cpx<R>{R(0), R(0)};
    for (int e = lane; e < bs; e += 32) {
      const int v = block_site(bk, xc, e);
      cpx<R> p[12];
      load_spinor<R>(Pa, V, v, p);
#pragma unroll
      for (int rr = 0; rr < RC; ++rr)
#pragma unroll
        for (int k = 0; k < 12; ++k) cfmac(acc[rr][k / 6], p[k], sm[((size_t)rr * 12 + k) * bs + e]);
    }
#pragma unroll
    for (int rr = 0; rr < RC; ++rr)
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          acc[rr][s].re += __shfl_xor_sync(0xffffffffu, acc[rr][s].re, o);
          acc[rr][s].im += __shfl_xor_sync(0xffffffffu, acc[rr][s].im, o);
        }
    if (lane == 0) {
      for (int rr = 0; rr < RC; ++rr) {
        const int r = r0 + rr;
        if (r >= nrhs || (active && !active[r])) continue;
        cpx<R>* o = reinterpret_cast<cpx<R>*>(out) + ((size_t)r * bk.coarse.V + xc) * 2 * N;
        o[a] = acc[rr][0];
        o[N + a] = acc[rr][1];
      }
    }
  }
}

// prolong, fine level: CTA per (coarse site, chunk of RC rhs), thread per fine site.
template <typename R, int RC>
__global__ void k_prolong_fine(const void* __restrict__ P, Blocking bk, const void* __restrict__ in,
                               void* __restrict__ out, int nrhs, const int* __restrict__ active) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<R>* phi = reinterpret_cast<cpx<R>*>(smraw);  // [RC][2N]
  const int xc = blockIdx.x, r0 = blockIdx.y * RC;
  const int N = bk.N, V = bk.fine.V;
  const size_t fb = spinor_field_bytes<R>(V);
  for (int i = threadIdx.x; i < RC * 2 * N; i += blockDim.x) {
    const int rr = i / (2 * N), d = i % (2 * N), r = r0 + rr;
    phi[i] = (r < nrhs) ? reinterpret_cast<const cpx<R>*>(in)[((size_t)r * bk.coarse.V + xc) * 2 * N + d]
                        : cpx<R>{R(0), R(0)};
  }
  __syncthreads();
  for (int e = threadIdx.x; e < bk.bs; e += blockDim.x) {
    const int v = block_site(bk, xc, e);
    cpx<R> acc[RC][12];
#pragma unroll
    for (int rr = 0; rr < RC; ++rr)
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[rr][k] = cpx<R>{R(0), R(0)};
    for (int a = 0; a < N; ++a) {
      cpx<R> p[12];
      load_spinor<R>((const char*)P + fb * a, V, v, p);
#pragma unroll
      for (int rr = 0; rr < RC; ++rr) {
        const cpx<R> cp = phi[rr * 2 * N + a], cm = phi[rr * 2 * N + N + a];
#pragma unroll
        for (int k = 0; k < 12; ++k) cfma(acc[rr][k], p[k], k < 6 ? cp : cm);
      }
    }
#pragma unroll
    for (int rr = 0; rr < RC; ++rr) {
      const int r = r0 + rr;
      if (r < nrhs && (!active || active[r])) store_spinor<R>((char*)out + fb * r, V, v, acc[rr]);
    }
  }
}

// ------------------------------------------------------------------------------------
// Fine-level transfer, one thread per (block site, component pair c): all RC right-hand sides
// of the launch chunk are held in registers, so P is read once per launch with one
// coalesced 2-complex load per vector alpha.
//   prolong: CTA per (coarse site, pair c); psi_r(x)[2c..2c+1] = sum_alpha P_alpha(x)[..] phi_r
//   restrict: CTA per (coarse site, chirality s) covering the 3 pairs of s; per (pair, alpha)
//            the products are summed by warp shuffles and accumulated per warp in shared
//            memory, then over warps in order (fixed summation order).
// ------------------------------------------------------------------------------------
// Prolong: CTA per (coarse site, component pair c), thread per block site holding all RC
// right-hand sides; the thread's P entries stream through a kPSt-deep cp.async ring in shared
// memory (each thread reads back only its own copies, so no block barrier is needed).
constexpr int kPSt = 6;
template <typename R, typename PT, int RC>
__global__ void __launch_bounds__(256) k_prolong_fine3(const void* __restrict__ P, Blocking bk,
                                                       const void* __restrict__ in, void* __restrict__ out, int nrhs,
                                                       const int* __restrict__ active) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int CB = PSt<PT>::kPair;  // bytes of one component pair of P
  const int xc = blockIdx.x, c = blockIdx.y, r0 = blockIdx.z * RC;
  const int N = bk.N, V = bk.fine.V, s = c / 3, T = blockDim.x;
  cpx<R>* phi = reinterpret_cast<cpx<R>*>(smraw);  // [N][RC]
  unsigned char* ring = smraw + (((size_t)N * RC * sizeof(cpx<R>) + 15) / 16) * 16;  // [kPSt][T][CB]
  const size_t fb = spinor_field_bytes<R>(V), fbp = (size_t)V * 6 * CB;  // vector / P field bytes
  const int e = threadIdx.x;
  const bool live = e < bk.bs;
  const int v = live ? block_site(bk, xc, e) : 0;
  const char* src = (const char*)P + ((size_t)c * V + v) * CB;
  auto issue = [&](int a) {
    if (live && a < N)
      PSt<PT>::copy(ring + ((size_t)(a % kPSt) * T + e) * CB, src + fbp * a);
    cp_async_commit();
  };
#pragma unroll
  for (int a = 0; a < kPSt - 1; ++a) issue(a);
  for (int i = threadIdx.x; i < RC * N; i += T) {
    const int a = i / RC, rr = i - a * RC, r = r0 + rr;
    phi[i] = (r < nrhs) ? reinterpret_cast<const cpx<R>*>(in)[((size_t)r * bk.coarse.V + xc) * 2 * N + s * N + a]
                        : cpx<R>{R(0), R(0)};
  }
  __syncthreads();
  cpx<R> acc[RC][2];
#pragma unroll
  for (int rr = 0; rr < RC; ++rr) acc[rr][0] = acc[rr][1] = cpx<R>{R(0), R(0)};
  for (int a = 0; a < N; ++a) {
    cp_async_wait<kPSt - 2>();
    cpx<R> p0, p1;
    PSt<PT>::ld2(reinterpret_cast<const PT*>(ring + ((size_t)(a % kPSt) * T + e) * CB), p0, p1);
    issue(a + kPSt - 1);
#pragma unroll
    for (int rr = 0; rr < RC; rr += 2) {
      cpx<R> f0, f1;
      lds2(phi + (size_t)a * RC + rr, f0, f1);
      cfma(acc[rr][0], p0, f0);
      cfma(acc[rr][1], p1, f0);
      cfma(acc[rr + 1][0], p0, f1);
      cfma(acc[rr + 1][1], p1, f1);
    }
  }
  cp_async_wait<0>();
  if (!live) return;
#pragma unroll
  for (int rr = 0; rr < RC; ++rr) {
    const int r = r0 + rr;
    if (r < nrhs && (!active || active[r])) Chunk2<R>::store((char*)out + fb * r, (size_t)c * V + v, acc[rr][0], acc[rr][1]);
  }
}

// Restrict as a per-block complex GEMM  out[alpha][r] = sum_k conj(P[k][alpha]) x[k][r], k running
// over the block's sites x the 6 components of chirality s.  The block is streamed in chunks
// of S sites through a double-buffered cp.async stage in shared memory (P rows and x rows with
// k contiguous); warp w owns a fixed slice of every chunk's k range, lane (ag, rg) =
// (lane / 4, lane % 4) owns the TA x TR output tile alpha = ag*TA + i, r = rg*TR + j.  Warp
// partials are summed in warp order at the end, so the result for one right-hand side does not
// depend on the others or on TR.
constexpr int kRWarps = 8;  // warps of the restrict CTA
template <typename R, typename PT, int TA, int TR, int S>
__global__ void __launch_bounds__(kRWarps * 32) k_restrict_fine3(const void* __restrict__ P, Blocking bk,
                                                                 const void* __restrict__ in, void* __restrict__ out,
                                                                 int nrhs, const int* __restrict__ active, int half) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int NA = 8 * TA, RC = 4 * TR;
  constexpr int CB = 2 * sizeof(cpx<R>), CBP = PSt<PT>::kPair;  // bytes of a component pair: x, P
  constexpr int K = 6 * S, Kp = K + 2;            // complex k per chunk, padded row length
  constexpr int KW = ((K / 2 + kRWarps - 1) / kRWarps) * 2;  // even k slice per warp
  constexpr int NT = kRWarps * 32, CE = 3 * S;    // threads; (component pair, site) items per row
  constexpr int RSTEP = NT / CE;                  // rows staged per pass of the CTA
  // stage buffer q: P rows [NA][Kp] (PT), then x rows [RC][Kp] (complex R), 16-byte aligned
  constexpr size_t pbytes = (((size_t)NA * Kp * sizeof(PT) + 15) / 16) * 16;
  constexpr size_t stage = pbytes + (size_t)RC * Kp * sizeof(cpx<R>);
  const int xc = blockIdx.x, s = blockIdx.y, r0 = blockIdx.z * RC;
  const int N = bk.N, V = bk.fine.V, bs = bk.bs;
  // half: `in` holds the even sites only (half-lattice fields, site v at v >> 1; zero on the odd
  // sites), so only the block's bs / 2 even sites are read, of the vectors and of P
  const int bsx = half ? bs / 2 : bs;
  auto Pbuf = [&](int q) { return reinterpret_cast<PT*>(smraw + (size_t)q * stage); };
  auto Xbuf = [&](int q) { return reinterpret_cast<cpx<R>*>(smraw + (size_t)q * stage + pbytes); };
  int* vsite = reinterpret_cast<int*>(smraw + 2 * stage);  // [bs] fine site of each block site
  const size_t fb = spinor_field_bytes<R>(half ? V / 2 : V), fbp = (size_t)V * 6 * CBP;  // vector / P field bytes
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, ag = lane >> 2, rg = lane & 3;
  const int kb = warp * KW, ke = min(K, kb + KW);
  unsigned rmask = 0;  // right-hand sides of this chunk that are present and active
  for (int j = 0; j < RC; ++j)
    if (r0 + j < nrhs && (!active || active[r0 + j])) rmask |= 1u << j;
  for (int e = threadIdx.x; e < bsx; e += NT) vsite[e] = half ? even_block_site(bk, xc, e) : block_site(bk, xc, e);
  // P rows alpha >= N stay zero in both buffers
  for (int i = threadIdx.x; i < (NA - N) * Kp; i += NT) {
    Pbuf(0)[(size_t)N * Kp + i] = PSt<PT>::zero();
    Pbuf(1)[(size_t)N * Kp + i] = PSt<PT>::zero();
  }
  __syncthreads();
  // this thread stages item (cc, e) of rows row0, row0 + RSTEP, ...
  const int item = threadIdx.x % CE, row0 = threadIdx.x / CE, cc = item / S, e = item % S;
  const size_t coff = (size_t)(3 * s + cc) * V, xoff = half ? (size_t)(3 * s + cc) * (V / 2) : coff;
  const int nchunks = (bsx + S - 1) / S;
  auto issue = [&](int q) {
    if (q < nchunks && row0 < RSTEP) {
      const bool in_blk = q * S + e < bsx;
      const int vs = in_blk ? vsite[q * S + e] : 0;
      const size_t site = coff + vs, xsite = xoff + (half ? vs >> 1 : vs);
      for (int row = row0; row < N + RC; row += RSTEP) {
        if (row < N) {
          PT* dst = Pbuf(q & 1) + (size_t)row * Kp + (cc * S + e) * 2;
          if (in_blk) PSt<PT>::copy(dst, (const char*)P + fbp * row + site * CBP);
          else dst[0] = dst[1] = PSt<PT>::zero();
        } else {
          cpx<R>* dst = Xbuf(q & 1) + (size_t)(row - N) * Kp + (cc * S + e) * 2;
          if (in_blk && ((rmask >> (row - N)) & 1u)) {
            const char* src = (const char*)in + fb * (r0 + row - N) + xsite * CB;
#pragma unroll
            for (int h = 0; h < CB / 16; ++h) cp_async16((char*)dst + 16 * h, src + 16 * h);
          } else {
            dst[0] = dst[1] = cpx<R>{R(0), R(0)};
          }
        }
      }
    }
    cp_async_commit();
  };
  cpx<R> acc[TA][TR];
#pragma unroll
  for (int i = 0; i < TA; ++i)
#pragma unroll
    for (int j = 0; j < TR; ++j) acc[i][j] = cpx<R>{R(0), R(0)};
  issue(0);
  for (int q = 0; q < nchunks; ++q) {
    issue(q + 1);
    cp_async_wait<1>();
    __syncthreads();
    const PT* Ps = Pbuf(q & 1);
    const cpx<R>* Xs = Xbuf(q & 1);
#pragma unroll 2
    for (int k = kb; k < ke; k += 2) {
      cpx<R> p[TA][2], x[TR][2];
#pragma unroll
      for (int i = 0; i < TA; ++i) PSt<PT>::ld2(Ps + (size_t)(ag * TA + i) * Kp + k, p[i][0], p[i][1]);
#pragma unroll
      for (int j = 0; j < TR; ++j) lds2(Xs + (size_t)(rg * TR + j) * Kp + k, x[j][0], x[j][1]);
#pragma unroll
      for (int i = 0; i < TA; ++i)
#pragma unroll
        for (int j = 0; j < TR; ++j) {
          cfmac(acc[i][j], p[i][0], x[j][0]);
          cfmac(acc[i][j], p[i][1], x[j][1]);
        }
    }
    __syncthreads();
  }
  cp_async_wait<0>();
  cpx<R>* red = reinterpret_cast<cpx<R>*>(smraw);  // [warp][NA][RC]
#pragma unroll
  for (int i = 0; i < TA; ++i)
#pragma unroll
    for (int j = 0; j < TR; ++j) red[((size_t)warp * NA + ag * TA + i) * RC + rg * TR + j] = acc[i][j];
  __syncthreads();
  for (int i = threadIdx.x; i < N * RC; i += NT) {
    const int a = i / RC, j = i - a * RC;
    if (!((rmask >> j) & 1u)) continue;
    cpx<R> t = red[(size_t)a * RC + j];
    for (int w = 1; w < kRWarps; ++w) t += red[((size_t)w * NA + a) * RC + j];
    reinterpret_cast<cpx<R>*>(out)[((size_t)(r0 + j) * bk.coarse.V + xc) * 2 * N + s * N + a] = t;
  }
}

template <typename R, typename PT, int TA, int TR, int S>
static size_t restrict3_smem(int bs) {
  constexpr int NA = 8 * TA, RC = 4 * TR, Kp = 6 * S + 2;
  const size_t pbytes = (((size_t)NA * Kp * sizeof(PT) + 15) / 16) * 16;
  const size_t stage = 2 * (pbytes + (size_t)RC * Kp * sizeof(cpx<R>)) + (size_t)bs * sizeof(int);
  const size_t redb = (size_t)kRWarps * NA * RC * sizeof(cpx<R>);
  return stage > redb ? stage : redb;
}

template <typename R, typename PT, int TA, int TR, int S>
static void launch_restrict_fine3s(const void* P, const Blocking& bk, const void* in, void* out, int nrhs,
                                   const int* active, cudaStream_t s, int half) {
  constexpr int RC = 4 * TR;
  static const cudaError_t attr = cudaFuncSetAttribute(k_restrict_fine3<R, PT, TA, TR, S>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  (void)attr;
  dim3 g(bk.coarse.V, 2, (nrhs + RC - 1) / RC);
  k_restrict_fine3<R, PT, TA, TR, S><<<g, kRWarps * 32, restrict3_smem<R, PT, TA, TR, S>(bk.bs), s>>>(P, bk, in, out,
                                                                                                      nrhs, active, half);
}

// sites per staged chunk: 16, or 8 when two 16-site stages would not fit in shared memory
template <typename R, typename PT, int TA, int TR>
static void launch_restrict_fine3(const void* P, const Blocking& bk, const void* in, void* out, int nrhs,
                                  const int* active, cudaStream_t s, int half) {
  if (restrict3_smem<R, PT, TA, TR, 16>(bk.bs) <= 200 * 1024)
    launch_restrict_fine3s<R, PT, TA, TR, 16>(P, bk, in, out, nrhs, active, s, half);
  else
    launch_restrict_fine3s<R, PT, TA, TR, 8>(P, bk, in, out, nrhs, active, s, half);
}

template <typename R, typename PT, int TA>
static void restrict_fine3_tr(const void* P, const Blocking& bk, const void* in, void* out, int nrhs,
                              const int* active, cudaStream_t s, int half) {
  if (nrhs <= 4) launch_restrict_fine3<R, PT, TA, 1>(P, bk, in, out, nrhs, active, s, half);
  else if (nrhs <= 8) launch_restrict_fine3<R, PT, TA, 2>(P, bk, in, out, nrhs, active, s, half);
  else launch_restrict_fine3<R, PT, TA, 3>(P, bk, in, out, nrhs, active, s, half);
}

template <typename R, typename PT>
static void restrict_fine3(const void* P, const Blocking& bk, const void* in, void* out, int nrhs,
                           const int* active, cudaStream_t s, int half = 0) {
  const int ta = (bk.N + 7) / 8;
  if (ta <= 1) restrict_fine3_tr<R, PT, 1>(P, bk, in, out, nrhs, active, s, half);
  else if (ta <= 2) restrict_fine3_tr<R, PT, 2>(P, bk, in, out, nrhs, active, s, half);
  else if (ta <= 3) restrict_fine3_tr<R, PT, 3>(P, bk, in, out, nrhs, active, s, half);
  else if (ta <= 4) restrict_fine3_tr<R, PT, 4>(P, bk, in, out, nrhs, active, s, half);
  else if (ta <= 6) restrict_fine3_tr<R, PT, 6>(P, bk, in, out, nrhs, active, s, half);
  else restrict_fine3_tr<R, PT, 8>(P, bk, in, out, nrhs, active, s, half);
}

template <typename R, typename PT, int RC>
static void launch_prolong_fine3(const void* P, const Blocking& bk, const void* in, void* out, int nrhs,
                                 const int* active, cudaStream_t s) {
  dim3 g(bk.coarse.V, 6, (nrhs + RC - 1) / RC);
  const int T = ((bk.bs + 31) / 32) * 32;
  const size_t smem =
      (((size_t)bk.N * RC * sizeof(cpx<R>) + 15) / 16) * 16 + (size_t)kPSt * T * PSt<PT>::kPair;
  static const cudaError_t attr = cudaFuncSetAttribute(k_prolong_fine3<R, PT, RC>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  (void)attr;
  k_prolong_fine3<R, PT, RC><<<g, T, smem, s>>>(P, bk, in, out, nrhs, active);
}

template <typename R, typename PT>
static void prolong_fine3(const void* P, const Blocking& bk, const void* in, void* out, int nrhs,
                          const int* active, cudaStream_t s) {
  if (nrhs <= 2) launch_prolong_fine3<R, PT, 2>(P, bk, in, out, nrhs, active, s);
  else if (nrhs <= 4) launch_prolong_fine3<R, PT, 4>(P, bk, in, out, nrhs, active, s);
  else if (sizeof(R) == 8) launch_prolong_fine3<R, PT, 4>(P, bk, in, out, nrhs, active, s);
  else if (nrhs <= 8) launch_prolong_fine3<R, PT, 8>(P, bk, in, out, nrhs, active, s);
  else launch_prolong_fine3<R, PT, 12>(P, bk, in, out, nrhs, active, s);
}

// ------------------------------------------------------------------------------------
// restrict / prolong between coarse levels: fields [rhs][Vf][nf] -> [rhs][Vc][2N]
// ------------------------------------------------------------------------------------
template <typename R, int RC>
__global__ void k_restrict_coarse(const void* __restrict__ P, Blocking bk, const void* __restrict__ in,
                                  void* __restrict__ out, int nrhs, const int* __restrict__ active) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<R>* sm = reinterpret_cast<cpx<R>*>(smraw);  // [RC][bs*nf]
  const int xc = blockIdx.x, r0 = blockIdx.y * RC;
  const int nf = bk.nf, h = nf / 2, E = bk.bs * nf, Vf = bk.fine.V, N = bk.N;
  for (int i = threadIdx.x; i < RC * E; i += blockDim.x) {
    const int rr = i / E, e = i % E, r = r0 + rr;
    const int v = block_site(bk, xc, e / nf);
    sm[i] = (r < nrhs) ? reinterpret_cast<const cpx<R>*>(in)[((size_t)r * Vf + v) * nf + e % nf]
                       : cpx<R>{R(0), R(0)};
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int a = warp; a < N; a += nw) {
    const cpx<R>* Pa = reinterpret_cast<const cpx<R>*>(P) + (size_t)a * Vf * nf;
    cpx<R> acc[RC][2];
#pragma unroll
    for (int rr = 0; rr < RC; ++rr) acc[rr][0] = acc[rr][1] = cpx<R>{R(0), R(0)};
    for (int e = lane; e < E; e += 32) {
      const int v = block_site(bk, xc, e / nf), d = e % nf;
      const cpx<R> p = Pa[(size_t)v * nf + d];
      const int s = d >= h;
#pragma unroll
      for (int rr = 0; rr < RC; ++rr) cfmac(acc[rr][s], p, sm[rr * E + e]);
    }
#pragma unroll
    for (int rr = 0; rr < RC; ++rr)
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          acc[rr][s].re += __shfl_xor_sync(0xffffffffu, acc[rr][s].re, o);
          acc[rr][s].im += __shfl_xor_sync(0xffffffffu, acc[rr][s].im, o);
        }
    if (lane == 0)
      for (int rr = 0; rr < RC; ++rr) {
        const int r = r0 + rr;
        if (r >= nrhs || (active && !active[r])) continue;
        cpx<R>* o = reinterpret_cast<cpx<R>*>(out) + ((size_t)r * bk.coarse.V + xc) * 2 * N;
        o[a] = acc[rr][0];
        o[N + a] = acc[rr][1];
      }
  }
}

template <typename R, int RC>
__global__ void k_prolong_coarse(const void* __restrict__ P, Blocking bk, const void* __restrict__ in,
                                 void* __restrict__ out, int nrhs, const int* __restrict__ active) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<R>* phi = reinterpret_cast<cpx<R>*>(smraw);  // [RC][2N]
  const int xc = blockIdx.x, r0 = blockIdx.y * RC;
  const int N = bk.N, nf = bk.nf, h = nf / 2, E = bk.bs * nf, Vf = bk.fine.V;
  for (int i = threadIdx.x; i < RC * 2 * N; i += blockDim.x) {
    const int rr = i / (2 * N), d = i % (2 * N), r = r0 + rr;
    phi[i] = (r < nrhs) ? reinterpret_cast<const cpx<R>*>(in)[((size_t)r * bk.coarse.V + xc) * 2 * N + d]
                        : cpx<R>{R(0), R(0)};
  }
  __syncthreads();
  for (int e = threadIdx.x; e < E; e += blockDim.x) {
    const int v = block_site(bk, xc, e / nf), d = e % nf, s = d >= h;
    cpx<R> acc[RC];
#pragma unroll
    for (int rr = 0; rr < RC; ++rr) acc[rr] = cpx<R>{R(0), R(0)};
    for (int a = 0; a < N; ++a) {
      const cpx<R> p = reinterpret_cast<const cpx<R>*>(P)[((size_t)a * Vf + v) * nf + d];
#pragma unroll
      for (int rr = 0; rr < RC; ++rr) cfma(acc[rr], p, phi[rr * 2 * N + s * N + a]);
    }
#pragma unroll
    for (int rr = 0; rr < RC; ++rr) {
      const int r = r0 + rr;
      if (r < nrhs && (!active || active[r])) reinterpret_cast<cpx<R>*>(out)[((size_t)r * Vf + v) * nf + d] = acc[rr];
    }
  }
}

// ------------------------------------------------------------------------------------
// block Gram-Schmidt, FP64.  CTA per (coarse site, chirality s): the N vectors restricted to
// the block and to the s half of the dof are orthonormalised in order alpha = 0..N-1.  Each
// vector is projected against the previous ones by classical Gram-Schmidt, the k projections
// of a pass being reduced together, and projected a second time when the first pass lost more
// than half of its norm ("twice is enough"; the result is the basis of modified Gram-Schmidt
// to rounding); then it is normalised.  A vector whose norm after projection is
// below 1e-10 of its norm before sets *rank_flag.
// ------------------------------------------------------------------------------------
constexpr int kGsThreads = 256;
constexpr int kGsMaxPerThread = 8;
constexpr int kGsChunk = 8;  // projections reduced per CTA reduction

struct GsLayout {
  bool fine;
  Blocking bk;
  size_t field_stride;  // complex numbers per vector
};

// offset (in complex numbers) of element e of block xc, chirality s, inside vector 0
WMG_D size_t gs_offset(const GsLayout& L, int xc, int s, int e) {
  if (L.fine) {
    const int v = block_site(L.bk, xc, e / 6);
    const int k = s * 6 + e % 6;
    return ((size_t)(k >> 1) * L.bk.fine.V + v) * 2 + (k & 1);
  }
  const int h = L.bk.nf / 2;
  const int v = block_site(L.bk, xc, e / h);
  return (size_t)v * L.bk.nf + s * h + e % h;
}

__global__ void __launch_bounds__(kGsThreads) k_block_gs(void* vecs, GsLayout L, int* rank_flag) {
  __shared__ double sm[32 * 2 * kGsChunk];
  __shared__ double coef[2 * 128];
  const int xc = blockIdx.x, s = blockIdx.y;
  const int E = L.fine ? L.bk.bs * 6 : L.bk.bs * (L.bk.nf / 2);
  const int N = L.bk.N;
  cd* base = reinterpret_cast<cd*>(vecs);
  const size_t fs = L.field_stride;
  size_t off[kGsMaxPerThread];
  int ne = 0;
  for (int e = threadIdx.x; e < E && ne < kGsMaxPerThread; e += blockDim.x) off[ne++] = gs_offset(L, xc, s, e);
  for (int k = 0; k < N; ++k) {
    cd vk[kGsMaxPerThread];
    for (int i = 0; i < ne; ++i) vk[i] = base[fs * k + off[i]];
    double n0 = 0;
    {
      double t[1] = {0};
      for (int i = 0; i < ne; ++i) norm2_acc(t[0], vk[i]);
      cta_reduce<1>(t, sm);
      if (threadIdx.x == 0) coef[0] = t[0];
      __syncthreads();
      n0 = coef[0];
      __syncthreads();
    }
    for (int pass = 0; pass < 2 && k > 0; ++pass) {
      if (pass == 1) {
        // second projection only if the first one cancelled more than half of the norm
        // (Kahan-Parlett criterion: otherwise one classical pass is already orthogonal to
        // working precision)
        double t[1] = {0};
        for (int i = 0; i < ne; ++i) norm2_acc(t[0], vk[i]);
        cta_reduce<1>(t, sm);
        if (threadIdx.x == 0) coef[0] = t[0];
        __syncthreads();
        const double n_mid = coef[0];
        __syncthreads();
        if (n_mid > 0.5 * n0) break;
      }
      // c_j = <v_j, v_k> for all j < k, kGsChunk at a time
      for (int j0 = 0; j0 < k; j0 += kGsChunk) {
        double t[2 * kGsChunk];
#pragma unroll
        for (int q = 0; q < 2 * kGsChunk; ++q) t[q] = 0.0;
#pragma unroll
        for (int q = 0; q < kGsChunk; ++q) {
          const int j = j0 + q;
          if (j < k)
            for (int i = 0; i < ne; ++i) {
              // <v_j, v_k> as FMA chains: 4 FP64 operations per complex term instead of 6
              const cd a = base[fs * j + off[i]];
              t[2 * q] = fma(a.re, vk[i].re, t[2 * q]);
              t[2 * q] = fma(a.im, vk[i].im, t[2 * q]);
              t[2 * q + 1] = fma(a.re, vk[i].im, t[2 * q + 1]);
              t[2 * q + 1] = fma(-a.im, vk[i].re, t[2 * q + 1]);
            }
        }
        cta_reduce<2 * kGsChunk>(t, sm);
        if (threadIdx.x == 0)
          for (int q = 0; q < 2 * kGsChunk && 2 * j0 + q < 2 * 128; ++q) coef[2 * j0 + q] = t[q];
        __syncthreads();
      }
      for (int j = 0; j < k; ++j) {
        const cd cj{coef[2 * j], coef[2 * j + 1]};
        for (int i = 0; i < ne; ++i) cfms(vk[i], cj, base[fs * j + off[i]]);
      }
      __syncthreads();
    }
    double n1;
    {
      double t[1] = {0};
      for (int i = 0; i < ne; ++i) norm2_acc(t[0], vk[i]);
      cta_reduce<1>(t, sm);
      if (threadIdx.x == 0) coef[0] = t[0];
      __syncthreads();
      n1 = coef[0];
      __syncthreads();
    }
    if (!(n1 > 1e-20 * n0) || !(n0 > 0.0)) {
      if (threadIdx.x == 0) atomicExch(rank_flag, 1);
      n1 = 1.0;
    }
    const double inv = 1.0 / sqrt(n1);
    for (int i = 0; i < ne; ++i) base[fs * k + off[i]] = inv * vk[i];
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------
template <typename R, int RC>
static void launch_restrict_fine(const void* P, const Blocking& bk, const void* in, void* out, int nrhs,
                                 const int* active, cudaStream_t s) {
  const size_t smem = (size_t)RC * 12 * bk.bs * sizeof(cpx<R>);
  static const bool attr = [] {
    cudaFuncSetAttribute(k_restrict_fine<R, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    return true;
  }();
  (void)attr;
  dim3 g(bk.coarse.V, (nrhs + RC - 1) / RC);
  k_restrict_fine<R, RC><<<g, 128, smem, s>>>(P, bk, in, out, nrhs, active);
}

// FP32 vectors with FP16 null vectors (the native layout with __half2 elements); false when the
// blocking is outside what the staged kernels handle (the caller then uses the FP32 copy).
bool restrict_fine_h(const void* P16, const Blocking& bk, const void* in, void* out, int nrhs, const int* active,
                     cudaStream_t s, int half) {
  if (bk.N > 64) return false;
  count_launch();
  restrict_fine3<float, __half2>(P16, bk, in, out, nrhs, active, s, half);
  return true;
}
bool prolong_fine_h(const void* P16, const Blocking& bk, const void* in, void* out, int nrhs, const int* active,
                    cudaStream_t s) {
  if (bk.bs > 256 || bk.N > 64) return false;
  count_launch();
  prolong_fine3<float, __half2>(P16, bk, in, out, nrhs, active, s);
  return true;
}

__global__ void k_to_half2(const cd* __restrict__ src, __half2* __restrict__ dst, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = __floats2half2_rn((float)src[i].re, (float)src[i].im);
}
void convert_to_half2(const void* src64, void* dst16, size_t n, cudaStream_t s) {
  count_launch();
  size_t b = (n + 255) / 256;
  if (b > 148 * 16) b = 148 * 16;
  k_to_half2<<<(unsigned)b, 256, 0, s>>>((const cd*)src64, (__half2*)dst16, n);
}

void restrict_fine(int prec, const void* P, const Blocking& bk, const void* in, void* out, int nrhs,
                   const int* active, cudaStream_t s, int half) {
  count_launch();
  if (bk.N <= 64) {
    if (prec == WMG_PREC_DOUBLE) restrict_fine3<double, cpx<double>>(P, bk, in, out, nrhs, active, s, half);
    else restrict_fine3<float, cpx<float>>(P, bk, in, out, nrhs, active, s, half);
    return;
  }
  if (prec == WMG_PREC_DOUBLE) {
    if (nrhs == 1) launch_restrict_fine<double, 1>(P, bk, in, out, nrhs, active, s);
    else launch_restrict_fine<double, 2>(P, bk, in, out, nrhs, active, s);
  } else {
    if (nrhs == 1) launch_restrict_fine<float, 1>(P, bk, in, out, nrhs, active, s);
    else if (nrhs == 2) launch_restrict_fine<float, 2>(P, bk, in, out, nrhs, active, s);
    else launch_restrict_fine<float, 4>(P, bk, in, out, nrhs, active, s);
  }
}

template <typename R, int RC>
static void launch_prolong_fine(const void* P, const Blocking& bk, const void* in, void* out, int nrhs,
                                const int* active, cudaStream_t s) {
  const size_t smem = (size_t)RC * 2 * bk.N * sizeof(cpx<R>);
  dim3 g(bk.coarse.V, (nrhs + RC - 1) / RC);
  const int T = bk.bs < 256 ? ((bk.bs + 31) / 32) * 32 : 256;
  k_prolong_fine<R, RC><<<g, T, smem, s>>>(P, bk, in, out, nrhs, active);
}

void prolong_fine(int prec, const void* P, const Blocking& bk, const void* in, void* out, int nrhs,
                  const int* active, cudaStream_t s) {
  count_launch();
  if (bk.bs <= 256 && bk.N <= 64) {
    if (prec == WMG_PREC_DOUBLE) prolong_fine3<double, cpx<double>>(P, bk, in, out, nrhs, active, s);
    else prolong_fine3<float, cpx<float>>(P, bk, in, out, nrhs, active, s);
    return;
  }
  if (prec == WMG_PREC_DOUBLE) {
    if (nrhs == 1) launch_prolong_fine<double, 1>(P, bk, in, out, nrhs, active, s);
    else launch_prolong_fine<double, 2>(P, bk, in, out, nrhs, active, s);
  } else {
    if (nrhs == 1) launch_prolong_fine<float, 1>(P, bk, in, out, nrhs, active, s);
    else if (nrhs == 2) launch_prolong_fine<float, 2>(P, bk, in, out, nrhs, active, s);
    else launch_prolong_fine<float, 4>(P, bk, in, out, nrhs, active, s);
  }
}

template <typename R, int RC>
static void launch_restrict_coarse(const void* P, const Blocking& bk, const void* in, void* out, int nrhs,
                                   const int* active, cudaStream_t s) {
  const size_t smem = (size_t)RC * bk.bs * bk.nf * sizeof(cpx<R>);
  static const bool attr = [] {
    cudaFuncSetAttribute(k_restrict_coarse<R, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    return true;
  }();
  (void)attr;
  dim3 g(bk.coarse.V, (nrhs + RC - 1) / RC);
  k_restrict_coarse<R, RC><<<g, 128, smem, s>>>(P, bk, in, out, nrhs, active);
}

void restrict_coarse(int prec, const void* P, const Blocking& bk, const void* in, void* out, int nrhs,
                     const int* active, cudaStream_t s) {
  count_launch();
  if (prec == WMG_PREC_DOUBLE) {
    if (nrhs == 1) launch_restrict_coarse<double, 1>(P, bk, in, out, nrhs, active, s);
    else launch_restrict_coarse<double, 4>(P, bk, in, out, nrhs, active, s);
  } else {
    if (nrhs == 1) launch_restrict_coarse<float, 1>(P, bk, in, out, nrhs, active, s);
    else launch_restrict_coarse<float, 4>(P, bk, in, out, nrhs, active, s);
  }
}

template <typename R, int RC>
static void launch_prolong_coarse(const void* P, const Blocking& bk, const void* in, void* out, int nrhs,
                                  const int* active, cudaStream_t s) {
  const size_t smem = (size_t)RC * 2 * bk.N * sizeof(cpx<R>);
  dim3 g(bk.coarse.V, (nrhs + RC - 1) / RC);
  k_prolong_coarse<R, RC><<<g, 256, smem, s>>>(P, bk, in, out, nrhs, active);
}

void prolong_coarse(int prec, const void* P, const Blocking& bk, const void* in, void* out, int nrhs,
                    const int* active, cudaStream_t s) {
  count_launch();
  if (prec == WMG_PREC_DOUBLE) {
    if (nrhs == 1) launch_prolong_coarse<double, 1>(P, bk, in, out, nrhs, active, s);
    else launch_prolong_coarse<double, 4>(P, bk, in, out, nrhs, active, s);
  } else {
    if (nrhs == 1) launch_prolong_coarse<float, 1>(P, bk, in, out, nrhs, active, s);
    else launch_prolong_coarse<float, 4>(P, bk, in, out, nrhs, active, s);
  }
}

void block_gs(bool fine_level, void* vecs, const Blocking& bk, int* rank_flag, cudaStream_t s) {
  count_launch();
  GsLayout L;
  L.fine = fine_level;
  L.bk = bk;
  L.field_stride = fine_level ? (size_t)bk.fine.V * 12 : (size_t)bk.fine.V * bk.nf;
  dim3 g(bk.coarse.V, 2);
  k_block_gs<<<g, kGsThreads, 0, s>>>(vecs, L, rank_flag);
}

}  // namespace wmg
