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

template <typename R>
WMG_D cpx<R> crecip(cpx<R> a) {
  const R d = a.re * a.re + a.im * a.im;
  return cpx<R>{a.re / d, -a.im / d};
}

}  // namespace

// In-place inversion of the n x n matrix M (precision R, row-major, shared memory) by Gauss-Jordan
// elimination on [M | W] with W = I on entry: column by column, partial pivoting (the largest |M_ij|
// of the rows i >= j, first on ties); W = M^-1 on exit.  f: n scratch; *singular set on a zero pivot.
// Called by the whole CTA.
template <typename R>
WMG_D void gauss_jordan(cpx<R>* M, cpx<R>* W, cpx<R>* f, int n, int* singular) {
  using C = cpx<R>;
  __shared__ int piv;
  __shared__ C pivinv;
  const int w2 = 2 * n;
  for (int j = 0; j < n; ++j) {
    if (threadIdx.x < 32) {
      R best = R(-1);
      int bi = j;
      for (int i = j + (int)threadIdx.x; i < n; i += 32) {
        const C x = M[i * n + j];
        const R m2 = x.re * x.re + x.im * x.im;
        if (m2 > best) {
          best = m2;
          bi = i;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const R ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) {
          best = ob;
          bi = oi;
        }
      }
      if (threadIdx.x == 0) {
        piv = bi;
        if (!(best > R(0))) atomicExch(singular, 1);
      }
    }
    __syncthreads();
    const int p = piv;
    if (p != j)
      for (int c = threadIdx.x; c < w2; c += blockDim.x) {
        C* B = c < n ? M : W;
        const int cc = c < n ? c : c - n;
        const C t = B[j * n + cc];
        B[j * n + cc] = B[p * n + cc];
        B[p * n + cc] = t;
      }
    __syncthreads();
    if (threadIdx.x == 0) pivinv = crecip(M[j * n + j]);
    __syncthreads();
    const C s = pivinv;
    for (int c = threadIdx.x; c < w2; c += blockDim.x) {
      C* B = c < n ? M : W;
      const int cc = c < n ? c : c - n;
      B[j * n + cc] = s * B[j * n + cc];
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) f[i] = M[i * n + j];
    __syncthreads();
    for (int t = threadIdx.x; t < n * w2; t += blockDim.x) {
      const int i = t / w2, c = t - i * w2;
      if (i == j) continue;
      C* B = c < n ? M : W;
      const int cc = c < n ? c : c - n;
      B[i * n + cc] -= f[i] * B[j * n + cc];
    }
    __syncthreads();
  }
}

// One CTA per (odd site k, table entry): W = (A_kk + shift I)^-1 in shared memory, in the table's
// precision R (FP64 for the FP64 coarsest solve; FP32 for the tables of the FP32 and FP16 passes).
template <typename R>
__global__ void __launch_bounds__(kInvThreads) k_eo_invert(const cpx<R>* __restrict__ A, Geom g, int n,
                                                           const double* __restrict__ shifts,
                                                           cpx<R>* __restrict__ inv, int* __restrict__ singular) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<R>* M = reinterpret_cast<cpx<R>*>(smraw);  // [n][n]
  cpx<R>* W = M + (size_t)n * n;                 // [n][n]
  cpx<R>* f = W + (size_t)n * n;                 // [n] column j of M before its elimination
  const int k = blockIdx.x, Vh = g.V / 2;
  const int v = parity_site(g, k, 1);
  const cpx<R>* a = A + (size_t)v * 9 * n * n;  // slot 0, [col][row]
  const double sh = shifts[blockIdx.y];
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int col = i / n, row = i - col * n;
    const cpx<R> x = a[i];
    M[row * n + col] = cpx<R>{x.re + (row == col ? R(sh) : R(0)), x.im};
    W[row * n + col] = cpx<R>{row == col ? R(1) : R(0), R(0)};
  }
  __syncthreads();
  gauss_jordan<R>(M, W, f, n, singular);
  cpx<R>* o = inv + ((size_t)blockIdx.y * Vh + k) * n * n;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    const int col = i / n, row = i - col * n;
    o[i] = W[row * n + col];
  }
}

// One CTA per (odd site, chunk of kInvApplyRhs right-hand sides), thread (row, rhs): the input
// column bc b + hc h of the site is staged in shared memory (sigma_3 applied for the adjoint),
// then row . input with the inverse read column by column (consecutive rows: consecutive
// addresses).  Every load precedes every store, so out may alias h.
template <typename R>
__global__ void k_eo_inv_apply(const cpx<R>* __restrict__ inv, const int* __restrict__ idx, Geom g, int n,
                               const cpx<R>* b, R bc, const cpx<R>* h, R hc, cpx<R>* out, int nrhs, int dagger,
                               const int* __restrict__ active, int par) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<R>* xs = reinterpret_cast<cpx<R>*>(smraw);  // [kInvApplyRhs][n]
  const int k = blockIdx.x, Vh = g.V / 2, N = n / 2;
  const int v = parity_site(g, k, par);
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

// ---- right block-Jacobi preconditioning of the Schur complement: CG on T = S M, x_e = M y ----
// M_x = (S_xx)^-1 at even site x (grid.x = its parity-site number) for one shift:
//   S_xx = A_xx + shift I - sum over the two-hop paths x -> y = x + k1 -> x (every slot k2 of y that
//          points back at x: both slots on an extent of 2) of A(x, k1) (A_yy + shift I)^-1 A(y, k2),
// in FP32 (A: the FP32 stencil; the odd inverses: the shift's FP32 table entry, indexed by the odd
// parity-site number y >> 1), then inverted by Gauss-Jordan in FP32: the block-Jacobi preconditioner
// of the FP32 / FP16 coarsest CG.  Out: FP32 [k][col][row].
__global__ void __launch_bounds__(kInvThreads) k_eo_schur_self_inv(const cf* __restrict__ A, const cf* __restrict__ inv,
                                                                   Geom g, int n, double shift, cf* __restrict__ M,
                                                                   int* __restrict__ singular) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cf* S = reinterpret_cast<cf*>(smraw);  // [n][n] row-major
  cf* W = S + (size_t)n * n;
  cf* Pm = W + (size_t)n * n;            // A(x, k1) (A_yy + shift)^-1, row-major
  cf* f = Pm + (size_t)n * n;
  const float shf = (float)shift;
  const int k = blockIdx.x, nn = n * n;
  const int x = parity_site(g, k, 0);
  int cx[4];
  site_coords(g, x, cx);
  const cf* Ax = A + (size_t)x * 9 * nn;
  for (int i = threadIdx.x; i < nn; i += blockDim.x) {
    const int col = i / n, row = i - col * n;
    const cf a = Ax[i];
    S[row * n + col] = cf{a.re + (row == col ? shf : 0.f), a.im};
    W[row * n + col] = cf{row == col ? 1.f : 0.f, 0.f};
  }
  __syncthreads();
  for (int k1 = 1; k1 < 9; ++k1) {
    const int y = neighbour(g, x, cx, (k1 - 1) >> 1, ((k1 - 1) & 1) ? -1 : +1);
    const cf* iy = inv + (size_t)(y >> 1) * nn;  // [col][row]
    for (int i = threadIdx.x; i < nn; i += blockDim.x) {
      const int row = i / n, col = i - row * n;
      cf acc{0.f, 0.f};
      for (int j = 0; j < n; ++j) cfma(acc, Ax[((size_t)k1 * n + j) * n + row], iy[(size_t)col * n + j]);
      Pm[row * n + col] = acc;
    }
    __syncthreads();
    int cy[4];
    site_coords(g, y, cy);
    const cf* Ay = A + (size_t)y * 9 * nn;
    for (int k2 = 1; k2 < 9; ++k2) {
      if (neighbour(g, y, cy, (k2 - 1) >> 1, ((k2 - 1) & 1) ? -1 : +1) != x) continue;
      for (int i = threadIdx.x; i < nn; i += blockDim.x) {
        const int row = i / n, col = i - row * n;
        cf acc{0.f, 0.f};
        for (int j = 0; j < n; ++j) cfma(acc, Pm[row * n + j], Ay[((size_t)k2 * n + col) * n + j]);
        S[row * n + col] -= acc;
      }
    }
    __syncthreads();
  }
  gauss_jordan<float>(S, W, f, n, singular);
  cf* o = M + (size_t)k * nn;
  for (int i = threadIdx.x; i < nn; i += blockDim.x) {
    const int col = i / n, row = i - col * n;
    o[i] = W[row * n + col];
  }
}

// Tables of the preconditioned passes, FP32 in the stencil layout [parity site][9][col][row]:
//   mode 0 (odd site k, slot s = 1 + blockIdx.y): out = B[k][s] M(x + s), x odd, x + s even
//   mode 1 (even site k, slot s = blockIdx.y): s = 0: (A_xx + shift I) M_x; s > 0: A(x, s)
//   mode 2 (even site k, slot s = blockIdx.y): M_x X_s with X_0 = A_xx + shift I, X_s = A(x, s)
// Both factors staged in shared memory; thread (row, col) forms the n-term product.
__global__ void __launch_bounds__(256) k_eo_bj_table(int mode, const cf* __restrict__ A, const cf* __restrict__ B,
                                                     const cf* __restrict__ M, Geom g, int n, float shift,
                                                     cf* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cf* Ls = reinterpret_cast<cf*>(smraw);  // [col][row]
  cf* Rs = Ls + (size_t)n * n;
  const int k = blockIdx.x, nn = n * n;
  const int s = mode == 0 ? 1 + (int)blockIdx.y : (int)blockIdx.y;
  const int x = parity_site(g, k, mode == 0 ? 1 : 0);
  const cf* Ax = A + ((size_t)x * 9 + s) * nn;
  cf* o = out + ((size_t)k * 9 + s) * nn;
  if (mode == 1 && s > 0) {
    for (int i = threadIdx.x; i < nn; i += blockDim.x) o[i] = Ax[i];
    return;
  }
  const cf* L;
  const cf* R;
  bool shiftL = false, shiftR = false;
  if (mode == 0) {
    int c[4];
    site_coords(g, x, c);
    const int y = neighbour(g, x, c, (s - 1) >> 1, ((s - 1) & 1) ? -1 : +1);
    L = B + ((size_t)k * 9 + s) * nn;
    R = M + (size_t)(y >> 1) * nn;
  } else if (mode == 1) {
    L = Ax;
    R = M + (size_t)k * nn;
    shiftL = true;
  } else {
    L = M + (size_t)k * nn;
    R = Ax;
    shiftR = s == 0;
  }
  for (int i = threadIdx.x; i < nn; i += blockDim.x) {
    const int col = i / n, row = i - col * n;
    cf l = L[i], r = R[i];
    if (shiftL && row == col) l.re += shift;
    if (shiftR && row == col) r.re += shift;
    Ls[i] = l;
    Rs[i] = r;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nn; i += blockDim.x) {
    const int col = i / n, row = i - col * n;
    cf acc{0.f, 0.f};
    for (int j = 0; j < n; ++j) cfma(acc, Ls[(size_t)j * n + row], Rs[(size_t)col * n + j]);
    o[i] = acc;
  }
}

void eo_schur_self_inv(const void* A32, const void* inv_entry, const Geom& g, int n, double shift, void* M,
                       int* singular, cudaStream_t s) {
  count_launch();
  const size_t smem = ((size_t)3 * n * n + n) * sizeof(cf);
  static const bool attr = [] {
    cudaFuncSetAttribute(k_eo_schur_self_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    return true;
  }();
  (void)attr;
  k_eo_schur_self_inv<<<g.V / 2, kInvThreads, smem, s>>>((const cf*)A32, (const cf*)inv_entry, g, n, shift, (cf*)M,
                                                          singular);
}

void eo_bj_table(int mode, const void* A32, const void* B, const void* M, const Geom& g, int n, double shift,
                 void* out, cudaStream_t s) {
  count_launch();
  const size_t smem = (size_t)2 * n * n * sizeof(cf);
  static const bool attr = [] {
    cudaFuncSetAttribute(k_eo_bj_table, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    return true;
  }();
  (void)attr;
  k_eo_bj_table<<<dim3(g.V / 2, mode == 0 ? 8 : 9), 256, smem, s>>>(mode, (const cf*)A32, (const cf*)B, (const cf*)M,
                                                                   g, n, (float)shift, (cf*)out);
}

size_t eo_inverse_bytes(int prec, const Geom& g, int n) {
  return (size_t)(g.V / 2) * n * n * 2 * prec_real_bytes(prec);
}

void eo_invert(int prec, const void* A, const Geom& g, int n, const double* shifts, int e0, int ne, void* inv,
               int* singular, cudaStream_t s) {
  if (ne <= 0) return;
  count_launch();
  const size_t smem = ((size_t)2 * n * n + n) * 2 * prec_real_bytes(prec);
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
                  const void* h, double hc, void* out, int nrhs, bool dagger, const int* active, cudaStream_t s,
                  int par) {
  count_launch();
  const dim3 grid(g.V / 2, (nrhs + kInvApplyRhs - 1) / kInvApplyRhs);
  const int T = ((n * kInvApplyRhs + 31) / 32) * 32;
  const size_t smem = (size_t)kInvApplyRhs * n * 2 * prec_real_bytes(prec);
  if (prec == WMG_PREC_DOUBLE)
    k_eo_inv_apply<double><<<grid, T, smem, s>>>((const cd*)inv, idx, g, n, (const cd*)b, bc, (const cd*)h, hc,
                                                 (cd*)out, nrhs, dagger ? 1 : 0, active, par);
  else
    k_eo_inv_apply<float><<<grid, T, smem, s>>>((const cf*)inv, idx, g, n, (const cf*)b, (float)bc, (const cf*)h,
                                                (float)hc, (cf*)out, nrhs, dagger ? 1 : 0, active, par);
}

}  // namespace wmg
