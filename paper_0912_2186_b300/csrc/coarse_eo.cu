// Even-odd form of the coarsest-level CG solve (Sec. 3: CG on the normal equations on the
// coarsest lattice).  Every hop of the coarse stencil joins sites of opposite parity, so with
// the even sites first A = [[A_ee, A_eo], [A_oe, A_oo]] and A_oo is block diagonal: the odd
// sites' own n x n blocks.  The solve runs CG on the normal equations of the Schur complement
// S = A_ee - A_eo A_oo^-1 A_oe and recovers x_o = A_oo^-1 (b_o - A_oe x_e).  S keeps the
// coarse operator's sigma_3-hermiticity (sigma_3 is site-local and commutes with the split),
// so S^dag = sigma_3 S sigma_3.
//
// This file holds the two kernels of the block-diagonal part: the inversion of
// A_oo + shift I per odd site and table entry (one entry per distinct mass shift of the
// right-hand sides in flight), and the per-right-hand-side application of those inverses.
// The stencil passes themselves are the coarse-stencil kernels with their parity options.
#include "kernels.h"

namespace wmg {

namespace {

constexpr int kInvThreads = 256;
constexpr int kInvApplyRhs = 4;  // right-hand sides per CTA of the inverse application

WMG_D cd crecip(cd a) {
  const double d = a.re * a.re + a.im * a.im;
  return cd{a.re / d, -a.im / d};
}

}  // namespace

// One CTA per (odd site k, table entry).  [M | W] = [A_kk + shift I | I] in FP64 in shared
// memory (row-major); Gauss-Jordan elimination column by column with partial pivoting (the
// largest |M_ij| of the rows i >= j, first on ties) leaves W = M^-1.
template <typename R>
__global__ void __launch_bounds__(kInvThreads) k_eo_invert(const cpx<R>* __restrict__ A, Geom g, int n,
                                                           const double* __restrict__ shifts,
                                                           cpx<R>* __restrict__ inv, int* __restrict__ singular) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cd* M = reinterpret_cast<cd*>(smraw);  // [n][n]
  cd* W = M + (size_t)n * n;             // [n][n]
  cd* f = W + (size_t)n * n;             // [n] column j of M before its elimination
  __shared__ int piv;
  __shared__ cd pivinv;
  const int k = blockIdx.x, Vh = g.V / 2;
  const int v = parity_site(g, k, 1);
  const cpx<R>* a = A + (size_t)v * 9 * n * n;  // slot 0, [col][row]
  const double sh = shifts[blockIdx.y];
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int col = i / n, row = i - col * n;
    const cpx<R> x = a[i];
    M[row * n + col] = cd{double(x.re) + (row == col ? sh : 0.0), double(x.im)};
    W[row * n + col] = cd{row == col ? 1.0 : 0.0, 0.0};
  }
  __syncthreads();
  const int w2 = 2 * n;
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = j;
      for (int i = j + (int)threadIdx.x; i < n; i += 32) {
        const cd x = M[i * n + j];
        const double m2 = x.re * x.re + x.im * x.im;
        if (m2 > best) {
          best = m2;
          bi = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (threadIdx.x == 0) {
        piv = bi;
        if (!(best > 0.0)) atomicExch(singular, 1);
      }
    }
    __syncthreads();
    const int p = piv;
    if (p != j)
      for (int c = threadIdx.x; c < w2; c += blockDim.x) {
        cd* B = c < n ? M : W;
        const int cc = c < n ? c : c - n;
        const cd t = B[j * n + cc];
        B[j * n + cc] = B[p * n + cc];
        B[p * n + cc] = t;
      }
    __syncthreads();
    if (threadIdx.x == 0) pivinv = crecip(M[j * n + j]);
    __syncthreads();
    const cd s = pivinv;
    for (int c = threadIdx.x; c < w2; c += blockDim.x) {
      cd* B = c < n ? M : W;
      const int cc = c < n ? c : c - n;
      B[j * n + cc] = s * B[j * n + cc];
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) f[i] = M[i * n + j];
    __syncthreads();
    for (int t = threadIdx.x; t < n * w2; t += blockDim.x) {
      const int i = t / w2, c = t - i * w2;
      if (i == j) continue;
      cd* B = c < n ? M : W;
      const int cc = c < n ? c : c - n;
      B[i * n + cc] -= f[i] * B[j * n + cc];
    }
    __syncthreads();
  }
  cpx<R>* o = inv + ((size_t)blockIdx.y * Vh + k) * n * n;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int col = i / n, row = i - col * n;
    const cd x = W[row * n + col];
    o[i] = cpx<R>{R(x.re), R(x.im)};
  }
}

// One CTA per (odd site, chunk of kInvApplyRhs right-hand sides), thread (row, rhs): the input
// column bc b + hc h of the site is staged in shared memory (sigma_3 applied for the adjoint),
// then row . input with the inverse read column by column (consecutive rows: consecutive
// addresses).  Every load precedes every store, so out may alias h.
template <typename R>
__global__ void k_eo_inv_apply(const cpx<R>* __restrict__ inv, const int* __restrict__ idx, Geom g, int n,
                               const cpx<R>* b, R bc, const cpx<R>* h, R hc, cpx<R>* out, int nrhs, int dagger,
                               const int* __restrict__ active) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<R>* xs = reinterpret_cast<cpx<R>*>(smraw);  // [kInvApplyRhs][n]
  const int k = blockIdx.x, Vh = g.V / 2, N = n / 2;
  const int v = parity_site(g, k, 1);
  const int row = threadIdx.x % n, rr = threadIdx.x / n, r = blockIdx.y * kInvApplyRhs + rr;
  const bool ok = rr < kInvApplyRhs && r < nrhs;
  const size_t at = ((size_t)(ok ? r : 0) * g.V + v) * n + row;
  if (ok) {
    cpx<R> x{R(0), R(0)};
    if (b) x += bc * b[at];
    if (h) x += hc * h[at];
    if (dagger && row >= N) x = -x;
    xs[rr * n + row] = x;
  }
  __syncthreads();
  if (!ok) return;
  const cpx<R>* m = inv + ((size_t)idx[r] * Vh + k) * n * n + row;
  const cpx<R>* x = xs + rr * n;
  cpx<R> acc{R(0), R(0)};
  for (int col = 0; col < n; ++col) cfma(acc, m[(size_t)col * n], x[col]);
  if (dagger && row >= N) acc = -acc;
  if (!active || active[r]) out[at] = acc;
}

// The odd-site pass of S as a plain hop stencil: for odd site k (grid.x) and hop slot
// 1 + blockIdx.y, B_slot = -M A_slot with M = (A_kk + shift I)^-1 (FP32 table entry, [col][row])
// and A_slot the site's hop block; written in the stencil layout [k][9][col][row] (slot 0 left
// as it is: the hop-only pass never reads it).  Both factors are staged in shared memory;
// thread (row, col) forms the n-term row-by-column product.
__global__ void __launch_bounds__(256) k_eo_hop_inverse(const cf* __restrict__ A, const cf* __restrict__ inv,
                                                        Geom g, int n, cf* __restrict__ B) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cf* Ms = reinterpret_cast<cf*>(smraw);  // [col][row]
  cf* As = Ms + (size_t)n * n;            // [col][row]
  const int k = blockIdx.x, slot = 1 + blockIdx.y, nn = n * n;
  const int v = parity_site(g, k, 1);
  const cf* a = A + ((size_t)v * 9 + slot) * nn;
  const cf* m = inv + (size_t)k * nn;
  for (int i = threadIdx.x; i < nn; i += blockDim.x) {
    Ms[i] = m[i];
    As[i] = a[i];
  }
  __syncthreads();
  cf* o = B + ((size_t)k * 9 + slot) * nn;
  for (int i = threadIdx.x; i < nn; i += blockDim.x) {
    const int col = i / n, row = i - col * n;
    cf acc{0.f, 0.f};
    for (int j = 0; j < n; ++j) cfma(acc, Ms[(size_t)j * n + row], As[(size_t)col * n + j]);
    o[i] = cf{-acc.re, -acc.im};
  }
}

void eo_hop_inverse(const void* A, const void* inv_entry, const Geom& g, int n, void* B, cudaStream_t s) {
  count_launch();
  const size_t smem = (size_t)2 * n * n * sizeof(cf);
  static const bool attr = [] {
    cudaFuncSetAttribute(k_eo_hop_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    return true;
  }();
  (void)attr;
  k_eo_hop_inverse<<<dim3(g.V / 2, 8), 256, smem, s>>>((const cf*)A, (const cf*)inv_entry, g, n, (cf*)B);
}

size_t eo_inverse_bytes(int prec, const Geom& g, int n) {
  return (size_t)(g.V / 2) * n * n * 2 * prec_real_bytes(prec);
}

void eo_invert(int prec, const void* A, const Geom& g, int n, const double* shifts, int e0, int ne, void* inv,
               int* singular, cudaStream_t s) {
  if (ne <= 0) return;
  count_launch();
  const size_t smem = ((size_t)2 * n * n + n) * sizeof(cd);
  static const bool attr = [] {
    cudaFuncSetAttribute(k_eo_invert<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_eo_invert<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    return true;
  }();
  (void)attr;
  const dim3 grid(g.V / 2, ne);
  const size_t off = (size_t)e0 * eo_inverse_bytes(prec, g, n);
  if (prec == WMG_PREC_DOUBLE)
    k_eo_invert<double><<<grid, kInvThreads, smem, s>>>((const cd*)A, g, n, shifts, (cd*)((char*)inv + off),
                                                        singular);
  else
    k_eo_invert<float><<<grid, kInvThreads, smem, s>>>((const cf*)A, g, n, shifts, (cf*)((char*)inv + off),
                                                       singular);
}

void eo_inv_apply(int prec, const void* inv, const int* idx, const Geom& g, int n, const void* b, double bc,
                  const void* h, double hc, void* out, int nrhs, bool dagger, const int* active, cudaStream_t s) {
  count_launch();
  const dim3 grid(g.V / 2, (nrhs + kInvApplyRhs - 1) / kInvApplyRhs);
  const int T = ((n * kInvApplyRhs + 31) / 32) * 32;
  const size_t smem = (size_t)kInvApplyRhs * n * 2 * prec_real_bytes(prec);
  if (prec == WMG_PREC_DOUBLE)
    k_eo_inv_apply<double><<<grid, T, smem, s>>>((const cd*)inv, idx, g, n, (const cd*)b, bc, (const cd*)h, hc,
                                                 (cd*)out, nrhs, dagger ? 1 : 0, active);
  else
    k_eo_inv_apply<float><<<grid, T, smem, s>>>((const cf*)inv, idx, g, n, (const cf*)b, (float)bc, (const cf*)h,
                                                (float)hc, (cf*)out, nrhs, dagger ? 1 : 0, active);
}

}  // namespace wmg
