// Galerkin coarse operator D^ = P^dag D P (Sec. 2) as a 9-point stencil of n x n complex
// blocks (n = 2N, chirality-split, Sec. 3) and its application.
//
// Storage: A[site][slot][col][row] complex (column-major blocks, so that the threads of a
// site, one per row, read consecutive addresses).  Slot 0 is the self coupling, slot
// 1 + 2 mu + (0: +mu, 1: -mu) multiplies phi(xhat +/- mu):
//   (D^ phi)(xhat) = sum_k A[xhat][k] phi(xhat + k).
// The adjoint is sigma_3 D^ sigma_3 (gamma_5-hermiticity carried to the coarse level, Sec. 3).
#include "kernels.h"
#include "wilson.cuh"

namespace wmg {

WMG_D int stencil_neighbour(const Geom& g, int v, const int c[4], int slot) {
  if (slot == 0) return v;
  const int mu = (slot - 1) >> 1, sign = ((slot - 1) & 1) ? -1 : +1;
  return neighbour(g, v, c, mu, sign);
}

// the neighbour in direction (mu, sign) of a site with coordinate x lies in the same block
WMG_HD bool same_block(int x, int L, int b, int sign) {
  int y = x + sign;
  if (y < 0) y += L;
  if (y >= L) y -= L;
  return (x / b) == (y / b);
}

// ------------------------------------------------------------------------------------
// apply: one CTA per coarse site and chunk of NR right-hand sides.  The nine neighbour
// vectors of the chunk are staged in shared memory (sigma_3 applied on load for the
// adjoint); thread (row, ks) accumulates the products of its row of the 9 n x n blocks over
// the columns kk = ks, ks + KS, ... for all NR right-hand sides in registers; the KS partial
// sums of a row are added in shared memory.  Optional per-rhs |out|^2 (deterministic order).
// ------------------------------------------------------------------------------------
constexpr int kCoarseKS = 4;

template <typename R, int NR>
__global__ void __launch_bounds__(256) k_coarse_apply(const void* __restrict__ A_, Geom g, int n,
                                                      const void* __restrict__ in_, void* __restrict__ out_, int nrhs,
                                                      const double* __restrict__ shift, int dagger,
                                                      const int* __restrict__ active, RedBuf rb, int want_norm) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<R>* xs = reinterpret_cast<cpx<R>*>(smraw);          // [9 n][NR]
  cpx<R>* red = xs + (size_t)9 * n * NR;                   // [KS][n][NR]
  const int v = blockIdx.x;
  const int r0 = blockIdx.y * NR;
  const int N = n / 2;
  const cpx<R>* A = reinterpret_cast<const cpx<R>*>(A_) + (size_t)v * 9 * n * n;
  const cpx<R>* in = reinterpret_cast<const cpx<R>*>(in_);
  cpx<R>* out = reinterpret_cast<cpx<R>*>(out_);
  __shared__ int nbs[9];
  if (threadIdx.x < 9) {
    int c[4];
    site_coords(g, v, c);
    nbs[threadIdx.x] = stencil_neighbour(g, v, c, threadIdx.x);
  }
  __syncthreads();
  for (int k = 0; k < 9; ++k)
    for (int i = threadIdx.x; i < n * NR; i += blockDim.x) {
      const int j = i / NR, rr = i % NR, r = r0 + rr;
      cpx<R> x{R(0), R(0)};
      if (r < nrhs) {
        x = in[((size_t)r * g.V + nbs[k]) * n + j];
        if (dagger && j >= N) x = -x;
      }
      xs[(size_t)(k * n + j) * NR + rr] = x;
    }
  __syncthreads();
  const int row = threadIdx.x % n, ks = threadIdx.x / n;
  cpx<R> acc[NR];
#pragma unroll
  for (int rr = 0; rr < NR; ++rr) acc[rr] = cpx<R>{R(0), R(0)};
  if (ks < kCoarseKS) {
    const int K = 9 * n;
#pragma unroll 4
    for (int kk = ks; kk < K; kk += kCoarseKS) {
      const cpx<R> a = A[(size_t)kk * n + row];
      const cpx<R>* xr = xs + (size_t)kk * NR;
#pragma unroll
      for (int rr = 0; rr < NR; ++rr) cfma(acc[rr], a, xr[rr]);
    }
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) red[((size_t)ks * n + row) * NR + rr] = acc[rr];
  }
  __syncthreads();
  double nv[NR];
#pragma unroll
  for (int rr = 0; rr < NR; ++rr) nv[rr] = 0.0;
  if (ks == 0) {
    const bool oneg = dagger && row >= N;
#pragma unroll
    for (int rr = 0; rr < NR; ++rr) {
      cpx<R> o = red[(size_t)row * NR + rr];
      for (int q = 1; q < kCoarseKS; ++q) o += red[((size_t)q * n + row) * NR + rr];
      const int r = r0 + rr;
      if (r >= nrhs) continue;
      if (oneg) o = -o;
      if (shift) o += R(shift[r]) * in[((size_t)r * g.V + v) * n + row];
      if (!active || active[r]) out[((size_t)r * g.V + v) * n + row] = o;
      nv[rr] = double(o.re) * o.re + double(o.im) * o.im;
    }
  }
  if (want_norm) {
    __shared__ double sm[32 * NR];
    cta_reduce<NR>(nv, sm);
    __shared__ bool last;
    const int nblk = gridDim.x;
    if (threadIdx.x == 0) {
      for (int rr = 0; rr < NR; ++rr)
        if (r0 + rr < nrhs) rb.partial[(size_t)(r0 + rr) * nblk + blockIdx.x] = nv[rr];
      __threadfence();
      const unsigned prev = atomicAdd(rb.counter + blockIdx.y, 1u);
      last = prev == (unsigned)nblk - 1;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      const int nvals = min(NR, nrhs - r0);
      cta_multi_sum(rb.partial + (size_t)r0 * nblk, nvals, (size_t)nblk, nblk, 1,
                    [&](int i, double s) { rb.result[r0 + i] = s; });
      if (threadIdx.x == 0) rb.counter[blockIdx.y] = 0u;
    }
  }
}

template <typename R, int NR>
static void launch_coarse_apply(const void* A, const Geom& g, int n, const void* in, void* out, int nrhs,
                                const double* shift, bool dagger, const int* active, const RedBuf* rb, cudaStream_t s) {
  const int T = ((n * kCoarseKS + 31) / 32) * 32;
  const size_t smem = ((size_t)9 * n * NR + (size_t)kCoarseKS * n * NR) * sizeof(cpx<R>);
  static const bool attr = [] {
    cudaFuncSetAttribute(k_coarse_apply<R, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    return true;
  }();
  (void)attr;
  dim3 grid(g.V, (nrhs + NR - 1) / NR);
  RedBuf r = rb ? *rb : RedBuf{nullptr, nullptr, nullptr};
  k_coarse_apply<R, NR><<<grid, T, smem, s>>>(A, g, n, in, out, nrhs, shift, dagger ? 1 : 0, active, r, rb ? 1 : 0);
}

void coarse_apply(int prec, const void* A, const Geom& g, int n, const void* in, void* out, int nrhs,
                  const double* shift, bool dagger, const int* active, const RedBuf* rb, cudaStream_t s) {
  count_launch();
  if (prec == WMG_PREC_DOUBLE) {
    if (nrhs == 1) launch_coarse_apply<double, 1>(A, g, n, in, out, nrhs, shift, dagger, active, rb, s);
    else if (nrhs <= 4) launch_coarse_apply<double, 4>(A, g, n, in, out, nrhs, shift, dagger, active, rb, s);
    else launch_coarse_apply<double, 8>(A, g, n, in, out, nrhs, shift, dagger, active, rb, s);
  } else {
    if (nrhs == 1) launch_coarse_apply<float, 1>(A, g, n, in, out, nrhs, shift, dagger, active, rb, s);
    else if (nrhs <= 4) launch_coarse_apply<float, 4>(A, g, n, in, out, nrhs, shift, dagger, active, rb, s);
    else if (nrhs <= 8) launch_coarse_apply<float, 8>(A, g, n, in, out, nrhs, shift, dagger, active, rb, s);
    else launch_coarse_apply<float, 12>(A, g, n, in, out, nrhs, shift, dagger, active, rb, s);
  }
}

// ------------------------------------------------------------------------------------
// Galerkin build, fine level.  For column c = (s, alpha) the field g_c holds P_alpha
// restricted to chirality s in every block.  Each hop term of D g_c at site x goes to the
// self field if its neighbour lies in the block of x, else to the field of its slot; the
// diagonal (4 + m) g_c goes to the self field.  Output: [cc][9] native fine fields.
// ------------------------------------------------------------------------------------
template <typename R>
__global__ void k_hop_split_fine(const void* __restrict__ gauge, const void* __restrict__ P, Blocking bk, R diag,
                                 int col0, void* __restrict__ out9) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int cc = blockIdx.y;
  const Geom& g = bk.fine;
  if (v >= g.V) return;
  const int col = col0 + cc, s = col / bk.N, a = col % bk.N;
  const size_t fb = spinor_field_bytes<R>(g.V);
  const char* Pa = (const char*)P + fb * a;
  char* o = (char*)out9 + fb * (size_t)cc * 9;
  int c[4];
  site_coords(g, v, c);
  cpx<R> self[12], t[12];
  load_spinor<R>(Pa, g.V, v, self);
#pragma unroll
  for (int k = 0; k < 12; ++k) self[k] = ((k < 6) == (s == 0)) ? diag * self[k] : cpx<R>{R(0), R(0)};
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
    for (int sg = 0; sg < 2; ++sg) {
      const int sign = sg ? -1 : +1;
      const int slot = 1 + 2 * mu + sg;
      const int nb = neighbour(g, v, c, mu, sign);
      cpx<R> u[9], x[12];
      load_spinor<R>(Pa, g.V, nb, x);
#pragma unroll
      for (int k = 0; k < 12; ++k)
        if ((k < 6) != (s == 0)) x[k] = cpx<R>{R(0), R(0)};
#pragma unroll
      for (int k = 0; k < 12; ++k) t[k] = cpx<R>{R(0), R(0)};
      if (sg == 0) {
        load_link<R>(gauge, g.V, mu, v, u);
        hop_accumulate<+1>(mu, u, x, t);
      } else {
        load_link<R>(gauge, g.V, mu, nb, u);
        hop_accumulate<-1>(mu, u, x, t);
      }
#pragma unroll
      for (int k = 0; k < 12; ++k) t[k] = R(-0.5) * t[k];
      const bool inb = same_block(c[mu], g.L[mu], bk.b[mu], sign);
      if (inb) {
#pragma unroll
        for (int k = 0; k < 12; ++k) self[k] += t[k];
#pragma unroll
        for (int k = 0; k < 12; ++k) t[k] = cpx<R>{R(0), R(0)};
      }
      store_spinor<R>(o + fb * slot, g.V, v, t);
    }
  }
  store_spinor<R>(o, g.V, v, self);
}

void hop_split_fine(int prec, const void* gauge, const void* P, const Blocking& bk, double mass, int col0, int ncol,
                    void* out9, cudaStream_t s) {
  count_launch();
  dim3 grid((bk.fine.V + 127) / 128, ncol);
  if (prec == WMG_PREC_DOUBLE)
    k_hop_split_fine<double><<<grid, 128, 0, s>>>(gauge, P, bk, 4.0 + mass, col0, out9);
  else
    k_hop_split_fine<float><<<grid, 128, 0, s>>>(gauge, P, bk, float(4.0 + mass), col0, out9);
}

// Fused Galerkin construction on the fine level: CTA per (column c, coarse block) with the
// columns of one block adjacent in the grid, so that the block's vectors P are shared in L2;
// one thread per block site (bs <= 256, every block extent >= 2).  Thread x computes the terms
// of D g_c at x (g_c = P_alpha restricted to chirality s in every block): the diagonal and the
// hops whose neighbour lies in the block go to the self slot, each hop leaving the block to the
// slot of its direction (at most one per direction).  For every row (s', alpha') the products
// <P_alpha'(x)|_s', term> are summed over the block by warp shuffles, per-warp partials in
// shared memory, and a final fixed-order sum; the CTA writes column c of all 9 blocks.
template <typename R>
__global__ void __launch_bounds__(256) k_galerkin_fine(const void* __restrict__ gauge, const void* __restrict__ P,
                                                       Blocking bk, R diag, void* __restrict__ Aout) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = bk.N, n = 2 * N;
  const int c = blockIdx.x % n, xc = blockIdx.x / n;
  const int s = c / N, a = c % N;
  const int e = threadIdx.x;
  const int nw = blockDim.x >> 5, warp = e >> 5, lane = e & 31;
  R* red = reinterpret_cast<R*>(smraw);  // [nw][N][9][2 chir][2 re/im]
  const Geom& g = bk.fine;
  const size_t fb = spinor_field_bytes<R>(g.V);
  const char* Pa = (const char*)P + fb * a;
  cpx<R> self[12], face[4][12];
  int fslot[4];
  const bool live = e < bk.bs;
  int v = 0;
  if (live) {
    // block site e -> fine site
    int cc[4];
    site_coords(bk.coarse, xc, cc);
    int o[4];
    o[0] = e % bk.b[0];
    int t = e / bk.b[0];
    o[1] = t % bk.b[1];
    t /= bk.b[1];
    o[2] = t % bk.b[2];
    o[3] = t / bk.b[2];
    int f[4];
    for (int i = 0; i < 4; ++i) f[i] = cc[i] * bk.b[i] + o[i];
    v = site_index(g, f);
    int crd[4];
    site_coords(g, v, crd);
    load_spinor<R>(Pa, g.V, v, self);
#pragma unroll
    for (int k = 0; k < 12; ++k) self[k] = ((k < 6) == (s == 0)) ? diag * self[k] : cpx<R>{R(0), R(0)};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      fslot[mu] = -1;
#pragma unroll
      for (int k = 0; k < 12; ++k) face[mu][k] = cpx<R>{R(0), R(0)};
#pragma unroll
      for (int sg = 0; sg < 2; ++sg) {
        const int sign = sg ? -1 : +1;
        const int nb = neighbour(g, v, crd, mu, sign);
        cpx<R> u[9], xg[12], tt[12];
        load_spinor<R>(Pa, g.V, nb, xg);
#pragma unroll
        for (int k = 0; k < 12; ++k)
          if ((k < 6) != (s == 0)) xg[k] = cpx<R>{R(0), R(0)};
#pragma unroll
        for (int k = 0; k < 12; ++k) tt[k] = cpx<R>{R(0), R(0)};
        if (sg == 0) {
          load_link<R>(gauge, g.V, mu, v, u);
          hop_accumulate<+1>(mu, u, xg, tt);
        } else {
          load_link<R>(gauge, g.V, mu, nb, u);
          hop_accumulate<-1>(mu, u, xg, tt);
        }
        const bool inb = same_block(crd[mu], g.L[mu], bk.b[mu], sign);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          const cpx<R> h = R(-0.5) * tt[k];
          if (inb) self[k] += h;
          else face[mu][k] = h;
        }
        if (!inb) fslot[mu] = 1 + 2 * mu + sg;
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) self[k] = cpx<R>{R(0), R(0)};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      fslot[mu] = -1;
#pragma unroll
      for (int k = 0; k < 12; ++k) face[mu][k] = cpx<R>{R(0), R(0)};
    }
  }
  for (int ap = 0; ap < N; ++ap) {
    cpx<R> p[12];
    if (live) load_spinor<R>((const char*)P + fb * ap, g.V, v, p);
    else
#pragma unroll
      for (int k = 0; k < 12; ++k) p[k] = cpx<R>{R(0), R(0)};
    R acc[9][4];
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q][0] = acc[q][1] = acc[q][2] = acc[q][3] = R(0);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const int ch = k < 6 ? 0 : 2;
      cpx<R> d = cmulc(p[k], self[k]);
      acc[0][ch] += d.re;
      acc[0][ch + 1] += d.im;
    }
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      cpx<R> d0{R(0), R(0)}, d1{R(0), R(0)};
#pragma unroll
      for (int k = 0; k < 6; ++k) cfmac(d0, p[k], face[mu][k]);
#pragma unroll
      for (int k = 6; k < 12; ++k) cfmac(d1, p[k], face[mu][k]);
      // the thread's face term of direction mu belongs to slot 1 + 2 mu (+) or 2 + 2 mu (-)
      const bool minus = fslot[mu] == 2 + 2 * mu;
#pragma unroll
      for (int sg = 0; sg < 2; ++sg) {
        const bool mine = (sg == 1) == minus;
        acc[1 + 2 * mu + sg][0] += mine ? d0.re : R(0);
        acc[1 + 2 * mu + sg][1] += mine ? d0.im : R(0);
        acc[1 + 2 * mu + sg][2] += mine ? d1.re : R(0);
        acc[1 + 2 * mu + sg][3] += mine ? d1.im : R(0);
      }
    }
#pragma unroll
    for (int q = 0; q < 9; ++q)
#pragma unroll
      for (int w = 0; w < 4; ++w)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[q][w] += __shfl_xor_sync(0xffffffffu, acc[q][w], o);
    if (lane == 0)
#pragma unroll
      for (int q = 0; q < 9; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) red[(((size_t)warp * N + ap) * 9 + q) * 4 + w] = acc[q][w];
  }
  __syncthreads();
  // column c of the 9 blocks: rows s'*N + alpha', summed over warps in order
  cpx<R>* A = reinterpret_cast<cpx<R>*>(Aout);
  for (int i = threadIdx.x; i < 9 * n; i += blockDim.x) {
    const int q = i / n, row = i % n, sp = row / N, ap = row % N;
    R re = 0, im = 0;
    for (int w = 0; w < nw; ++w) {
      re += red[(((size_t)w * N + ap) * 9 + q) * 4 + 2 * sp];
      im += red[(((size_t)w * N + ap) * 9 + q) * 4 + 2 * sp + 1];
    }
    A[(((size_t)xc * 9 + q) * n + c) * n + row] = cpx<R>{re, im};
  }
}

bool galerkin_fine_fused(int prec, const void* gauge, const void* P, const Blocking& bk, double mass, void* A,
                         cudaStream_t s) {
  if (bk.bs > 256) return false;
  for (int i = 0; i < 4; ++i)
    if (bk.b[i] < 2) return false;
  count_launch();
  const int T = ((bk.bs + 31) / 32) * 32;
  const size_t smem = (size_t)(T / 32) * bk.N * 9 * 4 * (prec == WMG_PREC_DOUBLE ? 8 : 4);
  dim3 grid((unsigned)(2 * bk.N) * bk.coarse.V);
  if (prec == WMG_PREC_DOUBLE) {
    static const bool attr = [] {
      cudaFuncSetAttribute(k_galerkin_fine<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      return true;
    }();
    (void)attr;
    k_galerkin_fine<double><<<grid, T, smem, s>>>(gauge, P, bk, 4.0 + mass, A);
  } else {
    static const bool attr = [] {
      cudaFuncSetAttribute(k_galerkin_fine<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      return true;
    }();
    (void)attr;
    k_galerkin_fine<float><<<grid, T, smem, s>>>(gauge, P, bk, float(4.0 + mass), A);
  }
  return true;
}

// Galerkin build, coarse level: the same split for the stencil A of the finer coarse lattice.
// Thread per (site of bk.fine, row).  Output: [cc][9] coarse fields [Vf][nf].
template <typename R>
__global__ void k_hop_split_coarse(const void* __restrict__ A_, const void* __restrict__ P_, Blocking bk, int col0,
                                   void* __restrict__ out9) {
  const int nf = bk.nf, h = nf / 2;
  const int spc = blockDim.x / nf;
  const int ls = threadIdx.x / nf, row = threadIdx.x % nf;
  const int v = blockIdx.x * spc + ls;
  const Geom& g = bk.fine;
  if (ls >= spc || v >= g.V) return;
  const int cc = blockIdx.y, col = col0 + cc, s = col / bk.N, a = col % bk.N;
  const cpx<R>* A = reinterpret_cast<const cpx<R>*>(A_);
  const cpx<R>* P = reinterpret_cast<const cpx<R>*>(P_) + (size_t)a * g.V * nf;
  cpx<R>* o = reinterpret_cast<cpx<R>*>(out9) + (size_t)cc * 9 * g.V * nf;
  int c[4];
  site_coords(g, v, c);
  cpx<R> self{R(0), R(0)};
  for (int k = 0; k < 9; ++k) {
    const int nb = stencil_neighbour(g, v, c, k);
    const cpx<R>* Ak = A + ((size_t)v * 9 + k) * nf * nf + row;
    cpx<R> t{R(0), R(0)};
    for (int j = s * h; j < (s + 1) * h; ++j) cfma(t, Ak[(size_t)j * nf], P[(size_t)nb * nf + j]);
    bool inb = true;
    if (k > 0) {
      const int mu = (k - 1) >> 1, sign = ((k - 1) & 1) ? -1 : +1;
      inb = same_block(c[mu], g.L[mu], bk.b[mu], sign);
    }
    if (inb) {
      self += t;
      if (k > 0) o[((size_t)k * g.V + v) * nf + row] = cpx<R>{R(0), R(0)};
    } else {
      o[((size_t)k * g.V + v) * nf + row] = t;
    }
  }
  o[(size_t)v * nf + row] = self;
}

void hop_split_coarse(int prec, const void* A, const void* P, const Blocking& bk, int col0, int ncol, void* out9,
                      cudaStream_t s) {
  count_launch();
  int spc = 256 / bk.nf;
  if (spc < 1) spc = 1;
  const int T = ((spc * bk.nf + 31) / 32) * 32;
  dim3 grid((bk.fine.V + spc - 1) / spc, ncol);
  if (prec == WMG_PREC_DOUBLE) k_hop_split_coarse<double><<<grid, T, 0, s>>>(A, P, bk, col0, out9);
  else k_hop_split_coarse<float><<<grid, T, 0, s>>>(A, P, bk, col0, out9);
}

// rs: [cc][9][Vc][n] restricted slot fields -> A[site][slot][col0 + cc][row]
template <typename R>
__global__ void k_stencil_scatter(const cpx<R>* __restrict__ rs, cpx<R>* __restrict__ A, int Vc, int n, int col0,
                                  int ncol) {
  const size_t tot = (size_t)ncol * 9 * Vc * n;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(i % n);
    size_t t = i / n;
    const int site = (int)(t % Vc);
    t /= Vc;
    const int slot = (int)(t % 9);
    const int cc = (int)(t / 9);
    A[(((size_t)site * 9 + slot) * n + (col0 + cc)) * n + row] = rs[i];
  }
}

void stencil_scatter(int prec, const void* rs, void* A, int Vc, int n, int col0, int ncol, cudaStream_t s) {
  count_launch();
  const size_t tot = (size_t)ncol * 9 * Vc * n;
  int B = (int)((tot + 255) / 256);
  if (B > 148 * 16) B = 148 * 16;
  if (prec == WMG_PREC_DOUBLE)
    k_stencil_scatter<double><<<B, 256, 0, s>>>((const cd*)rs, (cd*)A, Vc, n, col0, ncol);
  else
    k_stencil_scatter<float><<<B, 256, 0, s>>>((const cf*)rs, (cf*)A, Vc, n, col0, ncol);
}

template <typename Rd, typename Rs>
__global__ void k_stencil_convert(cpx<Rd>* d, const cpx<Rs>* s, size_t count) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
    d[i] = ccast<Rd>(s[i]);
}

void stencil_convert(int pd, void* dst, int ps, const void* src, size_t count, cudaStream_t s) {
  count_launch();
  int B = (int)((count + 255) / 256);
  if (B > 148 * 16) B = 148 * 16;
  if (pd == WMG_PREC_DOUBLE && ps == WMG_PREC_DOUBLE) k_stencil_convert<double, double><<<B, 256, 0, s>>>((cd*)dst, (const cd*)src, count);
  else if (pd == WMG_PREC_DOUBLE) k_stencil_convert<double, float><<<B, 256, 0, s>>>((cd*)dst, (const cf*)src, count);
  else if (ps == WMG_PREC_DOUBLE) k_stencil_convert<float, double><<<B, 256, 0, s>>>((cf*)dst, (const cd*)src, count);
  else k_stencil_convert<float, float><<<B, 256, 0, s>>>((cf*)dst, (const cf*)src, count);
}

}  // namespace wmg
