// Level-1 vector kernels of the smoother, the coarsest CGNR and the outer GCR.  Vectors are
// flat arrays of n complex numbers per right-hand side (any field layout: operands of one
// call share it).  Every scalar is per right-hand side and lives on the device; reductions
// are deterministic (fixed-order two-stage sums in double precision).
#include "kernels.h"
#include "ptx.cuh"

namespace wmg {

constexpr int kBlasMaxBlocks = 148 * 2;
constexpr int kBlasPerThread = 4;

// CTAs per right-hand side: a function of the vector length only (so that every right-hand
// side is reduced in the same order whatever the batch): 4 elements per thread for short
// (coarse-level) vectors, at most 2 CTAs per SM per right-hand side for long ones
int blas_blocks(size_t n) {
  size_t b = (n + (size_t)kBlasThreads * kBlasPerThread - 1) / ((size_t)kBlasThreads * kBlasPerThread);
  if (b > (size_t)kBlasMaxBlocks) b = kBlasMaxBlocks;
  return b < 1 ? 1 : (int)b;
}

#define WMG_GRID_LOOP(i) \
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)

template <typename R>
WMG_D cpx<R>* vec(void* p, size_t n, int r) { return reinterpret_cast<cpx<R>*>(p) + n * r; }
template <typename R>
WMG_D const cpx<R>* vec(const void* p, size_t n, int r) { return reinterpret_cast<const cpx<R>*>(p) + n * r; }

template <typename R>
__global__ void k_zero(void* x, size_t n) {
  cpx<R>* a = vec<R>(x, n, blockIdx.y);
  WMG_GRID_LOOP(i) a[i] = cpx<R>{R(0), R(0)};
}

template <typename Rd, typename Rs>
__global__ void k_convert(void* dst, const void* src, size_t n, const int* mask) {
  const int r = blockIdx.y;
  if (mask && !mask[r]) return;
  cpx<Rd>* d = vec<Rd>(dst, n, r);
  const cpx<Rs>* s = vec<Rs>(src, n, r);
  WMG_GRID_LOOP(i) d[i] = ccast<Rd>(s[i]);
}

template <typename R>
__global__ void k_xmy(const void* x, void* y, size_t n) {
  const int r = blockIdx.y;
  const cpx<R>* a = vec<R>(x, n, r);
  cpx<R>* b = vec<R>(y, n, r);
  WMG_GRID_LOOP(i) b[i] = a[i] - b[i];
}

template <typename R>
__global__ void k_xpy(const void* x, void* y, size_t n) {
  const int r = blockIdx.y;
  const cpx<R>* a = vec<R>(x, n, r);
  cpx<R>* b = vec<R>(y, n, r);
  WMG_GRID_LOOP(i) b[i] = a[i] + b[i];
}

template <typename R>
__global__ void k_dot_norm(const void* a_, const void* b_, size_t n, RedBuf rb) {
  const int r = blockIdx.y;
  const cpx<R>* a = vec<R>(a_, n, r);
  const cpx<R>* b = vec<R>(b_, n, r);
  R t[3] = {0, 0, 0};  // per-thread sums in the vectors' precision, FP64 across threads
  WMG_GRID_LOOP(i) {
    cpx<R> x = a[i], y = b[i];
    cdot_acc(t[0], t[1], x, y);
    norm2_acc(t[2], x);
  }
  double v[3];
  __shared__ double sm[32 * 3];
  cta_reduce_mixed<R, 3>(t, v, sm);
  grid_finish<3>(rb, r, blockIdx.x, gridDim.x, v);
}

template <typename R>
__global__ void k_norm2(const void* a_, size_t n, RedBuf rb) {
  const int r = blockIdx.y;
  const cpx<R>* a = vec<R>(a_, n, r);
  R t = 0;
  WMG_GRID_LOOP(i) {
    cpx<R> x = a[i];
    norm2_acc(t, x);
  }
  double v[1];
  __shared__ double sm[32];
  R tv[1] = {t};
  cta_reduce_mixed<R, 1>(tv, v, sm);
  grid_finish<1>(rb, r, blockIdx.x, gridDim.x, v);
}

template <typename R>
__global__ void k_scale_inv_sqrt(void* x, size_t n, const double* nrm2, int stride) {
  const int r = blockIdx.y;
  const double q = nrm2[(size_t)r * stride];
  if (!(q > 0.0)) return;
  R sc[1];
  cta_scalars<R, 1>(sc, [&](double* v) { v[0] = 1.0 / sqrt(q); });
  const R s = sc[0];
  cpx<R>* a = vec<R>(x, n, r);
  WMG_GRID_LOOP(i) a[i] = s * a[i];
}

// y = gamma_5 x on native fine spinors: the components of spins 2 and 3 (chunks 3..5, the second
// half of each right-hand side's n complex numbers) change sign
template <typename R>
__global__ void k_gamma5(const void* x_, void* y_, size_t n) {
  const int r = blockIdx.y;
  const cpx<R>* x = vec<R>(x_, n, r);
  cpx<R>* y = vec<R>(y_, n, r);
  WMG_GRID_LOOP(i) y[i] = i < n / 2 ? x[i] : -x[i];
}

// x += alpha r and (update_r) r -= alpha q, alpha = red[0..1] / red[2] per rhs
template <typename R>
__global__ void k_mr_update(void* x_, void* r_, const void* q_, size_t n, const double* red, const int* active,
                            int update_r) {
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const double qq = red[r * 3 + 2];
  if (!(qq > 0.0)) return;
  R sc[2];
  cta_scalars<R, 2>(sc, [&](double* v) {
    v[0] = red[r * 3 + 0] / qq;
    v[1] = red[r * 3 + 1] / qq;
  });
  const cpx<R> al{sc[0], sc[1]};
  cpx<R>* x = vec<R>(x_, n, r);
  cpx<R>* rr = vec<R>(r_, n, r);
  const cpx<R>* q = vec<R>(q_, n, r);
  if (!update_r) {
    WMG_GRID_LOOP(i) cfma(x[i], al, rr[i]);
    return;
  }
  WMG_GRID_LOOP(i) {
    cpx<R> ri = rr[i];
    cfma(x[i], al, ri);
    cpx<R> t = al * q[i];
    rr[i] = ri - t;
  }
}

// x += alpha p, r -= alpha q with alpha = zz[parity]/qq; |r|^2 reduced; the CTA that completes
// the sum marks convergence (|r|^2 <= tol2 |b|^2) and counts the iteration (every other CTA of
// the right-hand side has read done[r] by then).  A thread takes kBlasPerThread elements per
// round, i0 + j blockDim (j < kBlasPerThread), and issues every load of the round before the
// arithmetic (one memory round trip per round; the coarsest solve's vectors take one round).
template <typename R>
// (In the kernels launched with programmatic serialisation the vectors written by the previous
// kernel are read through plain pointers: a const __restrict__ load may be taken as invariant over
// the kernel and issued before griddepcontrol.wait, i.e. before the previous kernel has finished.)
__global__ void k_cg_update(void* x_, void* r_, const void* p_, const void* q_, size_t n, CgScalars cg, int parity,
                            int nrhs, RedBuf rb) {
  constexpr int E = kBlasPerThread;
  const int r = blockIdx.y;
  griddep_wait();  // everything below reads the previous kernel's results
  const int done = cg.done[r];
  const double qq = cg.qq[r], zz = cg.zz[parity * nrhs + r];
  const bool on = !done && qq > 0.0;
  R sc[1];
  cta_scalars<R, 1>(sc, [&](double* v) { v[0] = on ? zz / qq : 0.0; });
  const R al = sc[0];
  cpx<R>* x = vec<R>(x_, n, r);
  cpx<R>* rr = vec<R>(r_, n, r);
  const cpx<R>* p = vec<R>(p_, n, r);
  const cpx<R>* q = vec<R>(q_, n, r);
  R t = 0;
  for (size_t i0 = (size_t)blockIdx.x * blockDim.x * E + threadIdx.x; i0 < n; i0 += (size_t)gridDim.x * blockDim.x * E) {
    cpx<R> rv[E], xv[E], pv[E], qv[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const size_t i = i0 + (size_t)j * blockDim.x;
      if (i < n) {
        rv[j] = rr[i];
        if (on) xv[j] = x[i], pv[j] = p[i], qv[j] = q[i];
      }
    }
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const size_t i = i0 + (size_t)j * blockDim.x;
      if (i < n) {
        if (on) {
          xv[j] += al * pv[j];
          rv[j] = rv[j] - al * qv[j];
          x[i] = xv[j];
          rr[i] = rv[j];
        }
        norm2_acc(t, rv[j]);
      }
    }
  }
  griddep_launch_dependents();
  double v[1];
  __shared__ double sm[32];
  R tv[1] = {t};
  cta_reduce_mixed<R, 1>(tv, v, sm);
  const bool last = grid_finish<1>(rb, r, blockIdx.x, gridDim.x, v);
  if (last) {
    __syncthreads();
    if (threadIdx.x == 0 && !cg.done[r]) {
      cg.iters[r] += 1;
      if (cg.rr[r] <= cg.tol2 * cg.bb[r]) cg.done[r] = 1;
    }
  }
}

// p = z + beta p, beta = zz[1-parity]/zz[parity] (loads of a round issued first, as above)
template <typename R>
__global__ void k_cg_xpay(void* p_, const void* z_, size_t n, CgScalars cg, int parity, int nrhs) {
  constexpr int E = kBlasPerThread;
  const int r = blockIdx.y;
  griddep_wait();  // everything below reads the previous kernel's results
  const int done = cg.done[r];
  const double zo = cg.zz[parity * nrhs + r], zn = cg.zz[(1 - parity) * nrhs + r];
  if (done) return;
  R sc[1];
  cta_scalars<R, 1>(sc, [&](double* v) { v[0] = zo > 0.0 ? zn / zo : 0.0; });
  const R be = sc[0];
  cpx<R>* p = vec<R>(p_, n, r);
  const cpx<R>* z = vec<R>(z_, n, r);
  for (size_t i0 = (size_t)blockIdx.x * blockDim.x * E + threadIdx.x; i0 < n; i0 += (size_t)gridDim.x * blockDim.x * E) {
    cpx<R> pv[E], zv[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const size_t i = i0 + (size_t)j * blockDim.x;
      if (i < n) pv[j] = p[i], zv[j] = z[i];
    }
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const size_t i = i0 + (size_t)j * blockDim.x;
      if (i < n) p[i] = zv[j] + be * pv[j];
    }
  }
  griddep_launch_dependents();
}

// coef_j = <W_j, w> for j = j0 .. j0+J-1 (j < kmax)
template <typename R, int J>
__global__ void k_multidot(const void* W, size_t slot_stride, int j0, int kmax, const void* w_, size_t n,
                           const int* active, RedBuf rb) {
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const cpx<R>* w = vec<R>(w_, n, r);
  R t[2 * J];
#pragma unroll
  for (int j = 0; j < 2 * J; ++j) t[j] = 0;
  WMG_GRID_LOOP(i) {
    const cpx<R> b = w[i];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      if (j0 + j < kmax) {
        const cpx<R> a = vec<R>((const char*)W + (j0 + j) * slot_stride, n, r)[i];
        cdot_acc(t[2 * j], t[2 * j + 1], a, b);
      }
    }
  }
  double v[2 * J];
  __shared__ double sm[32 * 2 * J];
  cta_reduce_mixed<R, 2 * J>(t, v, sm);
  grid_finish<2 * J>(rb, r, blockIdx.x, gridDim.x, v);
}


// w -= sum_{j<k} c_j W_j ; z -= sum c_j Z_j ; red = {|w|^2, Re<w,r>, Im<w,r>}
template <typename R>
__global__ void k_gcr_orth(const void* W, const void* Z, size_t slot_stride, int k, void* w_, void* z_,
                           const void* r_, const double* coef, int nrhs, size_t n, const int* active, RedBuf rb) {
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  __shared__ cpx<R> c[kMaxKrylov];
  if (threadIdx.x < k) {
    const int j = threadIdx.x;
    const double* cc = coef + ((size_t)(j / kDotChunk) * nrhs + r) * (2 * kDotChunk) + 2 * (j % kDotChunk);
    c[j] = cpx<R>{R(cc[0]), R(cc[1])};
  }
  __syncthreads();
  cpx<R>* w = vec<R>(w_, n, r);
  cpx<R>* z = Z ? vec<R>(z_, n, r) : nullptr;  // Z = nullptr: w only
  const cpx<R>* rv = vec<R>(r_, n, r);
  R t[3] = {0, 0, 0};
  WMG_GRID_LOOP(i) {
    cpx<R> wi = w[i];
    for (int j = 0; j < k; ++j) wi = wi - c[j] * vec<R>((const char*)W + j * slot_stride, n, r)[i];
    w[i] = wi;
    if (z) {
      cpx<R> zi = z[i];
      for (int j = 0; j < k; ++j) zi = zi - c[j] * vec<R>((const char*)Z + j * slot_stride, n, r)[i];
      z[i] = zi;
    }
    const cpx<R> ri = rv[i];
    norm2_acc(t[0], wi);
    cdot_acc(t[1], t[2], wi, ri);
  }
  double v[3];
  __shared__ double sm[32 * 3];
  cta_reduce_mixed<R, 3>(t, v, sm);
  grid_finish<3>(rb, r, blockIdx.x, gridDim.x, v);
}

// alpha = <w,r>/|w|^2; x += alpha z; r -= alpha w; w, z scaled by 1/|w|; red = |r|^2.  x is the
// iterate in the sloppy precision since the last reliable update.
template <typename R>
__global__ void k_gcr_update(void* x_, void* r_, void* w_, void* z_, const double* wred, size_t n,
                             const int* active, RedBuf rb) {
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const double ww = wred[r * 3 + 0];
  const bool ok = ww > 0.0;
  R sc[3];
  cta_scalars<R, 3>(sc, [&](double* v) {
    v[0] = ok ? 1.0 / sqrt(ww) : 0.0;
    v[1] = ok ? wred[r * 3 + 1] / ww : 0.0;
    v[2] = ok ? wred[r * 3 + 2] / ww : 0.0;
  });
  const R inv = sc[0];
  const cpx<R> al{sc[1], sc[2]};
  cpx<R>* x = vec<R>(x_, n, r);
  cpx<R>* rv = vec<R>(r_, n, r);
  cpx<R>* w = vec<R>(w_, n, r);
  cpx<R>* z = vec<R>(z_, n, r);
  R t = 0;
  WMG_GRID_LOOP(i) {
    const cpx<R> zi = z[i], wi = w[i];
    cpx<R> xi = x[i];
    cfma(xi, al, zi);
    x[i] = xi;
    const cpx<R> ri = rv[i] - al * wi;
    rv[i] = ri;
    w[i] = inv * wi;
    z[i] = inv * zi;
    norm2_acc(t, ri);
  }
  double v[1];
  __shared__ double sm[32];
  R tv[1] = {t};
  cta_reduce_mixed<R, 1>(tv, v, sm);
  grid_finish<1>(rb, r, blockIdx.x, gridDim.x, v);
}

// r_out = r - alpha q (an MR step whose solution update is deferred)
template <typename R>
__global__ void k_mr_rnext(void* __restrict__ ro_, const void* __restrict__ r_, const void* __restrict__ q_, size_t n,
                           const double* __restrict__ red, const int* __restrict__ active) {
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const double qq = red[r * 3 + 2];
  R sc[2];
  cta_scalars<R, 2>(sc, [&](double* v) {
    v[0] = qq > 0.0 ? red[r * 3 + 0] / qq : 0.0;
    v[1] = qq > 0.0 ? red[r * 3 + 1] / qq : 0.0;
  });
  const cpx<R> al{sc[0], sc[1]};
  cpx<R>* ro = vec<R>(ro_, n, r);
  const cpx<R>* rv = vec<R>(r_, n, r);
  const cpx<R>* q = vec<R>(q_, n, r);
  WMG_GRID_LOOP(i) ro[i] = rv[i] - al * q[i];
}

// alpha = <w,r>/|w|^2, r -= alpha w, w /= |w|; red = |r|^2 (the solution update is deferred)
template <typename R>
__global__ void k_gcr_update_r(void* r_, void* w_, const double* wred, size_t n, const int* active, RedBuf rb) {
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  const double ww = wred[r * 3 + 0];
  const bool ok = ww > 0.0;
  R sc[3];
  cta_scalars<R, 3>(sc, [&](double* v) {
    v[0] = ok ? 1.0 / sqrt(ww) : 0.0;
    v[1] = ok ? wred[r * 3 + 1] / ww : 0.0;
    v[2] = ok ? wred[r * 3 + 2] / ww : 0.0;
  });
  const R inv = sc[0];
  const cpx<R> al{sc[1], sc[2]};
  cpx<R>* rv = vec<R>(r_, n, r);
  cpx<R>* w = vec<R>(w_, n, r);
  R t = 0;
  WMG_GRID_LOOP(i) {
    const cpx<R> wi = w[i];
    const cpx<R> ri = rv[i] - al * wi;
    rv[i] = ri;
    w[i] = inv * wi;
    norm2_acc(t, ri);
  }
  double v[1];
  __shared__ double sm[32];
  R tv[1] = {t};
  cta_reduce_mixed<R, 1>(tv, v, sm);
  grid_finish<1>(rb, r, blockIdx.x, gridDim.x, v);
}

// x += sum_{j < K} xi[r][j] Z_j for the masked right-hand sides (xi: complex FP64, kMaxKrylov
// per rhs); the deferred solution update of the flexible GCR
template <typename R>
__global__ void k_gcr_xupdate(const void* Z, size_t slot_stride, int K, void* x_, const double* xi, size_t n,
                              const int* mask) {
  const int r = blockIdx.y;
  if (mask && !mask[r]) return;
  __shared__ cpx<R> c[kMaxKrylov];
  if (threadIdx.x < K) c[threadIdx.x] = cpx<R>{R(xi[((size_t)r * kMaxKrylov + threadIdx.x) * 2]),
                                                R(xi[((size_t)r * kMaxKrylov + threadIdx.x) * 2 + 1])};
  __syncthreads();
  cpx<R>* x = vec<R>(x_, n, r);
  WMG_GRID_LOOP(i) {
    cpx<R> xv = x[i];
    for (int j = 0; j < K; ++j) cfma(xv, c[j], vec<R>((const char*)Z + j * slot_stride, n, r)[i]);
    x[i] = xv;
  }
}

// Back-substitution of the deferred GCR update (see kernels.h): CTA r stages beta_jq (j < q < K),
// gamma_q and alpha_q in shared memory; lane j of warp 0 holds the running right-hand side of
// row j, and for q = K-1 .. 0 lane q divides by gamma_q and broadcasts xi_q, which rows j < q
// subtract (column-oriented back-substitution).
__global__ void __launch_bounds__(128) k_gcr_backsolve(const double* __restrict__ hist, size_t hstride, size_t kcoef,
                                                       int K, int nslots, const int* __restrict__ ints,
                                                       double* __restrict__ xi) {
  const int r = blockIdx.x;
  if (!ints[r]) return;
  const int from = ints[nslots + r];
  __shared__ cd beta[kMaxKrylov][kMaxKrylov];  // beta[q][j] = <W_j, w_q>, j < q
  __shared__ double gam[kMaxKrylov];
  __shared__ cd alpha[kMaxKrylov];
  for (int t = threadIdx.x; t < K * K; t += blockDim.x) {
    const int q = t / K, j = t % K;
    if (j < q) {
      const double* b = hist + (size_t)q * hstride + ((size_t)(j / kDotChunk) * nslots + r) * 2 * kDotChunk +
                        2 * (j % kDotChunk);
      beta[q][j] = cd{b[0], b[1]};
    }
  }
  if (threadIdx.x < K) {
    const int q = threadIdx.x;
    const double* hw = hist + (size_t)q * hstride + kcoef + 3 * (size_t)r;
    const double g = hw[0] > 0.0 ? sqrt(hw[0]) : 0.0;
    gam[q] = g;
    alpha[q] = (q >= from && g > 0.0) ? cd{hw[1] / g, hw[2] / g} : cd{0.0, 0.0};
  }
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int j = threadIdx.x;
  cd acc = j < K ? alpha[j] : cd{0.0, 0.0}, mine{0.0, 0.0};
  for (int q = K - 1; q >= 0; --q) {
    cd x{0.0, 0.0};
    if (j == q && gam[q] > 0.0) x = cd{acc.re / gam[q], acc.im / gam[q]};
    x.re = __shfl_sync(0xffffffffu, x.re, q);
    x.im = __shfl_sync(0xffffffffu, x.im, q);
    if (j == q) mine = x;
    if (j < q) acc -= beta[q][j] * x;
  }
  if (j < K) {
    xi[((size_t)r * kMaxKrylov + j) * 2] = mine.re;
    xi[((size_t)r * kMaxKrylov + j) * 2 + 1] = mine.im;
  }
}

// x64 += x (sloppy), x = 0, for the masked right-hand sides (reliable update)
template <typename R>
__global__ void k_fold(double* x64, void* x_, size_t n, const int* mask) {
  const int r = blockIdx.y;
  if (mask && !mask[r]) return;
  cd* X = reinterpret_cast<cd*>(x64) + n * r;
  cpx<R>* x = vec<R>(x_, n, r);
  WMG_GRID_LOOP(i) {
    const cpx<R> a = x[i];
    X[i] += cd{double(a.re), double(a.im)};
    x[i] = cpx<R>{R(0), R(0)};
  }
}

// ------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------
#define WMG_BY_PREC(prec, KER, ...)          \
  do {                                       \
    if ((prec) == WMG_PREC_DOUBLE) KER<double>__VA_ARGS__; \
    else KER<float>__VA_ARGS__;              \
  } while (0)

void blas_zero(int prec, void* x, size_t n, int nrhs, cudaStream_t s) {
  count_launch();
  dim3 g(blas_blocks(n), nrhs);
  WMG_BY_PREC(prec, k_zero, <<<g, kBlasThreads, 0, s>>>(x, n));
}

void blas_convert(int pd, void* dst, int ps, const void* src, size_t n, int nrhs, const int* mask, cudaStream_t s) {
  count_launch();
  dim3 g(blas_blocks(n), nrhs);
  if (pd == WMG_PREC_DOUBLE && ps == WMG_PREC_DOUBLE) k_convert<double, double><<<g, kBlasThreads, 0, s>>>(dst, src, n, mask);
  else if (pd == WMG_PREC_DOUBLE) k_convert<double, float><<<g, kBlasThreads, 0, s>>>(dst, src, n, mask);
  else if (ps == WMG_PREC_DOUBLE) k_convert<float, double><<<g, kBlasThreads, 0, s>>>(dst, src, n, mask);
  else k_convert<float, float><<<g, kBlasThreads, 0, s>>>(dst, src, n, mask);
}

void blas_xmy(int prec, const void* x, void* y, size_t n, int nrhs, cudaStream_t s) {
  count_launch();
  dim3 g(blas_blocks(n), nrhs);
  WMG_BY_PREC(prec, k_xmy, <<<g, kBlasThreads, 0, s>>>(x, y, n));
}

void blas_xpy(int prec, const void* x, void* y, size_t n, int nrhs, cudaStream_t s) {
  count_launch();
  dim3 g(blas_blocks(n), nrhs);
  WMG_BY_PREC(prec, k_xpy, <<<g, kBlasThreads, 0, s>>>(x, y, n));
}

void blas_dot_norm(int prec, const void* a, const void* b, size_t n, int nrhs, const RedBuf& rb, cudaStream_t s) {
  count_launch();
  dim3 g(blas_blocks(n), nrhs);
  WMG_BY_PREC(prec, k_dot_norm, <<<g, kBlasThreads, 0, s>>>(a, b, n, rb));
}

void blas_norm2(int prec, const void* a, size_t n, int nrhs, const RedBuf& rb, cudaStream_t s) {
  count_launch();
  dim3 g(blas_blocks(n), nrhs);
  WMG_BY_PREC(prec, k_norm2, <<<g, kBlasThreads, 0, s>>>(a, n, rb));
}

void blas_gamma5(int prec, const void* x, void* y, size_t n, int nrhs, cudaStream_t s) {
  count_launch();
  dim3 g(blas_blocks(n), nrhs);
  WMG_BY_PREC(prec, k_gamma5, <<<g, kBlasThreads, 0, s>>>(x, y, n));
}

void blas_scale_inv_sqrt(int prec, void* x, size_t n, int nrhs, const double* nrm2, int stride, cudaStream_t s) {
  count_launch();
  dim3 g(blas_blocks(n), nrhs);
  WMG_BY_PREC(prec, k_scale_inv_sqrt, <<<g, kBlasThreads, 0, s>>>(x, n, nrm2, stride));
}

void blas_mr_update(int prec, void* x, void* r, const void* q, size_t n, int nrhs, const double* red, bool update_r,
                    const int* active, cudaStream_t s) {
  count_launch();
  dim3 g(blas_blocks(n), nrhs);
  WMG_BY_PREC(prec, k_mr_update, <<<g, kBlasThreads, 0, s>>>(x, r, q, n, red, active, update_r ? 1 : 0));
}

void blas_mr_rnext(int prec, void* r_out, const void* r, const void* q, size_t n, int nrhs, const double* red,
                   const int* active, cudaStream_t s) {
  count_launch();
  dim3 g(blas_blocks(n), nrhs);
  WMG_BY_PREC(prec, k_mr_rnext, <<<g, kBlasThreads, 0, s>>>(r_out, r, q, n, red, active));
}

void cg_update(int prec, void* x, void* r, const void* p, const void* q, size_t n, int nrhs, const CgScalars& cg,
               int parity, const RedBuf& rb_rr, cudaStream_t s) {
  count_launch();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blas_blocks(n), nrhs);
  cfg.blockDim = dim3(kBlasThreads);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_launches() ? 1 : 0;
  if (prec == WMG_PREC_DOUBLE) cudaLaunchKernelEx(&cfg, k_cg_update<double>, x, r, p, q, n, cg, parity, nrhs, rb_rr);
  else cudaLaunchKernelEx(&cfg, k_cg_update<float>, x, r, p, q, n, cg, parity, nrhs, rb_rr);
}

void cg_xpay(int prec, void* p, const void* z, size_t n, int nrhs, const CgScalars& cg, int parity, cudaStream_t s) {
  count_launch();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blas_blocks(n), nrhs);
  cfg.blockDim = dim3(kBlasThreads);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_launches() ? 1 : 0;
  if (prec == WMG_PREC_DOUBLE) cudaLaunchKernelEx(&cfg, k_cg_xpay<double>, p, z, n, cg, parity, nrhs);
  else cudaLaunchKernelEx(&cfg, k_cg_xpay<float>, p, z, n, cg, parity, nrhs);
}

void gcr_multidot(int prec, const void* W, size_t slot_stride, int kmax, const void* w, size_t n, int nrhs,
                  const int* active, const RedBuf& rb, cudaStream_t s) {
  count_launch((kmax + kDotChunk - 1) / kDotChunk);
  dim3 g(blas_blocks(n), nrhs);
  for (int j0 = 0; j0 < kmax; j0 += kDotChunk) {
    RedBuf r = rb;
    r.result = rb.result + (size_t)(j0 / kDotChunk) * nrhs * 2 * kDotChunk;
    if (prec == WMG_PREC_DOUBLE)
      k_multidot<double, kDotChunk><<<g, kBlasThreads, 0, s>>>(W, slot_stride, j0, kmax, w, n, active, r);
    else
      k_multidot<float, kDotChunk><<<g, kBlasThreads, 0, s>>>(W, slot_stride, j0, kmax, w, n, active, r);
  }
}

void gcr_orth(int prec, const void* W, const void* Z, size_t slot_stride, int k, void* w, void* z, const void* r,
              const double* coef, int kmax, size_t n, int nrhs, const int* active, const RedBuf& rb, cudaStream_t s) {
  count_launch();
  (void)kmax;
  dim3 g(blas_blocks(n), nrhs);
  WMG_BY_PREC(prec, k_gcr_orth, <<<g, kBlasThreads, 0, s>>>(W, Z, slot_stride, k, w, z, r, coef, nrhs, n, active, rb));
}

void gcr_update(int prec, void* x, void* r, void* w, void* z, const double* wred, size_t n, int nrhs,
                const int* active, const RedBuf& rb, cudaStream_t s) {
  count_launch();
  dim3 g(blas_blocks(n), nrhs);
  WMG_BY_PREC(prec, k_gcr_update, <<<g, kBlasThreads, 0, s>>>(x, r, w, z, wred, n, active, rb));
}

void gcr_update_r(int prec, void* r, void* w, const double* wred, size_t n, int nrhs, const int* active,
                  const RedBuf& rb, cudaStream_t s) {
  count_launch();
  dim3 g(blas_blocks(n), nrhs);
  WMG_BY_PREC(prec, k_gcr_update_r, <<<g, kBlasThreads, 0, s>>>(r, w, wred, n, active, rb));
}

void gcr_xupdate(int prec, const void* Z, size_t slot_stride, int K, void* x, const double* xi, size_t n, int nrhs,
                 const int* mask, cudaStream_t s) {
  count_launch();
  dim3 g(blas_blocks(n), nrhs);
  WMG_BY_PREC(prec, k_gcr_xupdate, <<<g, kBlasThreads, 0, s>>>(Z, slot_stride, K, x, xi, n, mask));
}

void gcr_backsolve(const double* hist, size_t hstride, size_t kcoef, int K, int nslots, const int* ints, double* xi,
                   cudaStream_t s) {
  count_launch();
  k_gcr_backsolve<<<nslots, 128, 0, s>>>(hist, hstride, kcoef, K, nslots, ints, xi);
}

void blas_fold(int prec, double* x64, void* x, size_t n, int nrhs, const int* mask, cudaStream_t s) {
  count_launch();
  dim3 g(blas_blocks(n), nrhs);
  WMG_BY_PREC(prec, k_fold, <<<g, kBlasThreads, 0, s>>>(x64, x, n, mask));
}

}  // namespace wmg
