// Transfer operators between lattice levels (Sec. 2): restriction R = P^dag, prolongation P,
// and the block orthonormalisation that defines P from the near-null vectors, with the
// chirality split sigma_3 P = P gamma_5 of Sec. 3.
//
// On every level the first half of a site's dof has chirality +1 (fine: spins 0, 1 =
// components 0..5; coarse: dof 0..N-1) and the second half chirality -1.  P is stored as N
// fields of the finer lattice (P_alpha, both chiralities in one field); the coarse dof of
// column (s, alpha) is s*N + alpha.
#include "kernels.h"

namespace wmg {

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
      for (int i = 0; i < ne; ++i) t[0] += norm2(vk[i]);
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
        for (int i = 0; i < ne; ++i) t[0] += norm2(vk[i]);
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
              const cd a = base[fs * j + off[i]];
              t[2 * q] += a.re * vk[i].re + a.im * vk[i].im;
              t[2 * q + 1] += a.re * vk[i].im - a.im * vk[i].re;
            }
        }
        cta_reduce<2 * kGsChunk>(t, sm);
        if (threadIdx.x == 0)
          for (int q = 0; q < 2 * kGsChunk && 2 * j0 + q < 2 * 128; ++q) coef[2 * j0 + q] = t[q];
        __syncthreads();
      }
      for (int j = 0; j < k; ++j) {
        const cd cj{coef[2 * j], coef[2 * j + 1]};
        for (int i = 0; i < ne; ++i) vk[i] = vk[i] - cj * base[fs * j + off[i]];
      }
      __syncthreads();
    }
    double n1;
    {
      double t[1] = {0};
      for (int i = 0; i < ne; ++i) t[0] += norm2(vk[i]);
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

void restrict_fine(int prec, const void* P, const Blocking& bk, const void* in, void* out, int nrhs,
                   const int* active, cudaStream_t s) {
  count_launch();
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
