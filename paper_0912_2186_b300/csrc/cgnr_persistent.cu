// The coarsest-level solve (CG on the normal equations, Sec. 3) as one persistent cooperative
// kernel for up to 16 right-hand sides: one CTA per SM keeps its coarse sites for the whole
// solve, applies the FP16 tensor-core stencil to them (the site's operator fragments staged by
// bulk asynchronous copies, mma.sync m16n8k16 with FP32 accumulation, D^dag = sigma_3 D sigma_3),
// and performs the vector updates of its own sites; grid barriers separate the phases that read
// neighbour values or global sums.  Per iteration:
//     q = A p, |q|^2 | alpha = zz / qq; x += alpha p; r -= alpha q; |r|^2 | convergence;
//     z = A^dag r, |z|^2 | beta = zz' / zz; p = z + beta p |
// Every per-rhs sum is formed per CTA in a fixed order, stored as [phase][rhs][CTA] partials,
// and summed over the CTAs in a fixed order by every CTA, so all CTAs take the same decisions
// and a right-hand side's arithmetic does not depend on the others.  Every wait (grid barrier,
// mbarrier) is bounded; on expiry the kernel records an error, which the solve reports.
#include <cuda_fp16.h>

#include <cstdio>
#include <cstdlib>

#include "kernels.h"
#include "mma_sync.cuh"
#include "ptx.cuh"

namespace wmg {
namespace {

constexpr int kPThreads = 256;
constexpr int kPR = 16;                  // right-hand sides of the kernel (one 16-column chunk)
constexpr int kPWarps = kPThreads / 32;
constexpr long long kPSpin = 1LL << 22;  // polls of a wait before it gives up

struct PcgArgs {
  const uint4* A16;
  const float* sA;
  Geom g;
  const double* shift;  // per-rhs diagonal shift of this level's stencil
  const cf* b;
  cf *x, *r, *p, *q, *z;
  int nrhs;
  double tol2;
  int maxit;
  const int* active;
  double* part;   // [4][kPR][gridDim.x] per-CTA partial sums
  unsigned* bar;  // [0] arrivals, [1] generation (zero at launch)
  int* err;       // sticky error flag of the solve
  int* done_out;  // [kPR]
  int* iters_out; // [kPR]
};

// Grid-wide barrier (all CTAs are co-resident: cooperative launch) with a bounded wait.
WMG_D bool grid_barrier(const PcgArgs& a) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = a.bar + 1;
    volatile int* err = a.err;
    const unsigned my = *gen;
    __threadfence();
    int good = 1;
    if (atomicAdd(a.bar, 1u) == gridDim.x - 1) {
      atomicExch(a.bar, 0u);
      __threadfence();
      atomicAdd(a.bar + 1, 1u);
    } else {
      long long i = 0;
      while (*gen == my) {
        if (++i > kPSpin || *err) {
          good = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    if (!good) atomicExch(a.err, 1);
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

template <int NDOF>
struct Smem {
  static constexpr int n = NDOF, K = 9 * n, KP = K + kKPad, MT = n / 16, KS = K / 16, COLS = 2 * kPR;
  static constexpr uint32_t kTileBytes = (uint32_t)KS * 32 * 16;
  static constexpr size_t kA = (size_t)2 * MT * kTileBytes;  // one site's fragments
  static constexpr size_t kX = (size_t)COLS * KP * sizeof(__half);
  // fragment buffers: two (the next visit's copy overlaps the current one) when they fit
  static constexpr int NBUF = 2 * kA + kX <= 200 * 1024 ? 2 : 1;
  static constexpr size_t bytes() { return NBUF * kA + kX; }
};

// Per-CTA state, identical in every CTA (derived from the same global sums).
struct PcgState {
  double bb[kPR], zz[kPR], red[kPR];
  int done[kPR], iters[kPR];
  float xmax[kPR];
  double npart[kPWarps][32][2];
  int nbs[9];
  unsigned long long mbar[2];  // one per fragment buffer
};

// The CTA's own sites v = blockIdx.x + k gridDim.x are visited in the same cyclic order by every
// stencil application; the fragments of visit c + 1 are requested while visit c is computed
// (buffer c & 1, mbarrier phase (c >> 1) & 1), across applications too.
template <int NDOF>
WMG_D void request_fragments(const PcgArgs& a, PcgState& st, unsigned char* smraw, unsigned c) {
  using S = Smem<NDOF>;
  constexpr int MT = S::MT, KS = S::KS;
  const int nown = (a.g.V - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  if (threadIdx.x != 0 || nown <= 0) return;
  const int v = blockIdx.x + (int)(c % (unsigned)nown) * gridDim.x;
  const unsigned buf = S::NBUF == 2 ? (c & 1u) : 0u;
  uint4* As = reinterpret_cast<uint4*>(smraw + buf * S::kA);
  const uint32_t bar = smem_addr(&st.mbar[buf]);
  // order earlier generic-proxy reads of this buffer before the async-proxy writes
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  mbar_arrive_expect_tx(bar, (uint32_t)S::kA);
  for (int t = 0; t < MT; ++t)
    for (int pl = 0; pl < 2; ++pl)
      bulk_g2s(smem_addr(As + (size_t)(pl * MT + t) * KS * 32), a.A16 + (((size_t)v * 2 + pl) * MT + t) * KS * 32,
               S::kTileBytes, bar);
}

// out(v) = A in (v) [+ shift in(v)], sigma_3-conjugated if dagger; the thread's two norm sums
// (its right-hand sides blk * 8 + 2 q + {0, 1}) grow by |out|^2.
template <int NDOF>
WMG_D void site_apply(const PcgArgs& a, PcgState& st, unsigned char* smraw, int v, const cf* in, cf* out,
                      bool dagger, unsigned& visit, double nacc[2]) {
  using S = Smem<NDOF>;
  constexpr int n = S::n, N = n / 2, K = S::K, KP = S::KP, MT = S::MT, KS = S::KS;
  constexpr int EPL = (K + 31) / 32, RPW = kPR / kPWarps;
  const unsigned buf = S::NBUF == 2 ? (visit & 1u) : 0u;
  uint4* As = reinterpret_cast<uint4*>(smraw + buf * S::kA);
  __half* xb = reinterpret_cast<__half*>(smraw + S::NBUF * S::kA);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Geom& g = a.g;
  const uint32_t bar = smem_addr(&st.mbar[buf]);
  const unsigned mphase = S::NBUF == 2 ? ((visit >> 1) & 1u) : (visit & 1u);
  // two buffers: request the next visit (its buffer was freed by the last sync); one: this visit
  request_fragments<NDOF>(a, st, smraw, S::NBUF == 2 ? visit + 1 : visit);
  if (threadIdx.x < 9) {
    int c[4];
    site_coords(g, v, c);
    const int k = threadIdx.x;
    st.nbs[k] = k == 0 ? v : neighbour(g, v, c, (k - 1) >> 1, ((k - 1) & 1) ? -1 : +1);
  }
  __syncthreads();
  int offs[EPL];
  unsigned neg = 0;
#pragma unroll
  for (int i = 0; i < EPL; ++i) {
    const int e = lane + 32 * i;
    offs[i] = -1;
    if (e < K) {
      const int k = e / n, j = e - k * n;
      offs[i] = st.nbs[k] * n + j;
      if (dagger && j >= N) neg |= 1u << i;
    }
  }
  // gather (bypassing L1: other CTAs wrote these values since the last barrier)
  cf xv[RPW][EPL];
#pragma unroll
  for (int h = 0; h < RPW; ++h) {
    const int rr = warp + kPWarps * h;
    const bool ok = rr < a.nrhs;
    const cf* src = in + (size_t)(ok ? rr : 0) * g.V * n;
#pragma unroll
    for (int i = 0; i < EPL; ++i) {
      cf t{0.f, 0.f};
      if (ok && offs[i] >= 0) {
        const float2 u = __ldcg(reinterpret_cast<const float2*>(src + offs[i]));
        t = {u.x, u.y};
      }
      xv[h][i] = t;
    }
  }
#pragma unroll
  for (int h = 0; h < RPW; ++h) {
    const int rr = warp + kPWarps * h;
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < EPL; ++i) mx = fmaxf(mx, fmaxf(fabsf(xv[h][i].re), fabsf(xv[h][i].im)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) st.xmax[rr] = mx;
    const float inv = mx > 0.f ? 1.f / mx : 0.f;
    __half* colr = xb + (size_t)((rr >> 3) * 16 + (rr & 7)) * KP;
    __half* coli = colr + (size_t)8 * KP;
#pragma unroll
    for (int i = 0; i < EPL; ++i) {
      const int e = lane + 32 * i;
      if (e < K) {
        const float sg = ((neg >> i) & 1u) ? -inv : inv;
        colr[e] = __float2half_rn(xv[h][i].re * sg);
        coli[e] = __float2half_rn(xv[h][i].im * sg);
      }
    }
  }
  __syncthreads();
  const bool mma_warp = warp < MT * 2;
  const int m = warp % MT, blk = warp / MT, gq = lane >> 2, q = lane & 3;
  float acc[2][2][4];
#pragma unroll
  for (int pl = 0; pl < 2; ++pl)
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[pl][t][e] = 0.f;
  bool ready = true;
  if (mma_warp) {
    ready = mbar_wait_bounded(bar, mphase, kPSpin);
    if (!ready && lane == 0) atomicExch(a.err, 1);
  }
  if (mma_warp && ready) {
    const uint4* Ar = As + (size_t)(0 * MT + m) * KS * 32 + lane;
    const uint4* Ai = As + (size_t)(1 * MT + m) * KS * 32 + lane;
    const __half* colbase = xb + (size_t)(blk * 16 + gq) * KP + 2 * q;
#pragma unroll 9
    for (int k = 0; k < KS; ++k) {
      const uint4 a0 = Ar[(size_t)k * 32], a1 = Ai[(size_t)k * 32];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const __half* col = colbase + (size_t)t * 8 * KP + 16 * k;
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(col);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(col + 8);
        mma16816(acc[0][t], a0, b0, b1);
        mma16816(acc[1][t], a1, b0, b1);
      }
    }
    const float s_a = a.sA[v];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int row = 16 * m + gq + (e >= 2 ? 8 : 0);
      const int rr = blk * 8 + 2 * q + (e & 1);
      if (rr >= a.nrhs) continue;
      const float yr = acc[0][0][e] - acc[1][1][e];
      const float yi = acc[0][1][e] + acc[1][0][e];
      const float sc = s_a * st.xmax[rr] * ((dagger && row >= N) ? -1.f : 1.f);
      cf o{yr * sc, yi * sc};
      const size_t idx = ((size_t)rr * g.V + v) * n + row;
      if (a.shift) {
        const float2 u = __ldcg(reinterpret_cast<const float2*>(in + idx));
        o += (float)a.shift[rr] * cf{u.x, u.y};
      }
      out[idx] = o;
      nacc[e & 1] += double(o.re) * o.re + double(o.im) * o.im;
    }
  }
  if (mma_warp && !ready) mbar_wait_bounded(bar, mphase, kPSpin);  // let the copies land (bounded)
  ++visit;
  __syncthreads();  // this visit's buffers are free again
}

// The CTA's norm sums of one phase (per rhs, fixed order) -> part[ph][rhs][cta]
template <int NDOF>
WMG_D void store_norm_part(const PcgArgs& a, PcgState& st, int ph, double nacc[2]) {
  constexpr int MT = NDOF / 16;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  st.npart[warp][lane][0] = nacc[0];
  st.npart[warp][lane][1] = nacc[1];
  nacc[0] = nacc[1] = 0.0;
  __syncthreads();
  if (threadIdx.x < kPR) {
    const int rr = threadIdx.x, b = rr >> 3, qq = (rr & 7) >> 1, ee = rr & 1;
    double t = 0.0;
    for (int mm = 0; mm < MT; ++mm)
      for (int gg = 0; gg < 8; ++gg) t += st.npart[b * MT + mm][gg * 4 + qq][ee];
    a.part[((size_t)ph * kPR + rr) * gridDim.x + blockIdx.x] = t;
  }
}

// sum over the CTAs of part[ph][rhs][*] into st.red[rhs] (fixed order, the same in every CTA)
WMG_D void reduce_part(const PcgArgs& a, PcgState& st, int ph) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int rr = warp; rr < kPR; rr += kPWarps) {
    double t = 0.0;
    const double* p = a.part + ((size_t)ph * kPR + rr) * gridDim.x;
    for (int c = lane; c < (int)gridDim.x; c += 32) t += __ldcg(p + c);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (lane == 0) st.red[rr] = t;
  }
  __syncthreads();
}

// A per-site vector pass over the CTA's sites: warp w takes right-hand sides w, w + 8 and its
// lanes the site's components; f(rhs, index) returns the value whose |.|^2 enters the CTA's
// sum of phase ph for that rhs (ph < 0: none).
template <typename F>
WMG_D void site_pass(const PcgArgs& a, PcgState& st, int n, int ph, F f) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double s[kPR / kPWarps] = {};
  for (int v = blockIdx.x; v < a.g.V; v += gridDim.x)
#pragma unroll
    for (int h = 0; h < kPR / kPWarps; ++h) {
      const int rr = warp + kPWarps * h;
      if (rr >= a.nrhs) continue;
      for (int j = lane; j < n; j += 32) {
        const cf o = f(rr, ((size_t)rr * a.g.V + v) * n + j);
        s[h] += double(o.re) * o.re + double(o.im) * o.im;
      }
    }
  if (ph < 0) return;
#pragma unroll
  for (int h = 0; h < kPR / kPWarps; ++h) {
    double t = s[h];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    const int rr = warp + kPWarps * h;
    if (lane == 0 && rr < kPR) a.part[((size_t)ph * kPR + rr) * gridDim.x + blockIdx.x] = t;
  }
}

WMG_D cf ldcg(const cf* p) {
  const float2 u = __ldcg(reinterpret_cast<const float2*>(p));
  return cf{u.x, u.y};
}

// Element e of right-hand side rr in the CTA's sites (e = site visit * n + component).
WMG_D size_t own_index(const PcgArgs& a, int rr, int e, int n) {
  const int k = e / n, j = e - k * n;
  return ((size_t)rr * a.g.V + blockIdx.x + (size_t)k * gridDim.x) * n + j;
}

constexpr int kPCh = 4;  // elements per lane whose loads are issued together

// x += alpha p, r -= alpha q for the CTA's sites (rhs not done and qq > 0; alpha = zz / qq with
// qq in st.red); |r|^2 -> part[ph].  Warp w takes rhs w, w + 8; lanes stride the elements.
WMG_D void pass_xr(const PcgArgs& a, PcgState& st, int n, int ph) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nown = (a.g.V - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int ne = nown * n;
#pragma unroll
  for (int h = 0; h < kPR / kPWarps; ++h) {
    const int rr = warp + kPWarps * h;
    double s = 0.0;
    if (rr < a.nrhs) {
      const double qq = st.red[rr];
      const bool upd = !st.done[rr] && qq > 0.0;
      const float al = upd ? float(st.zz[rr] / qq) : 0.f;
      for (int e0 = lane; e0 < ne; e0 += 32 * kPCh) {
        cf rv[kPCh], pv[kPCh], qv[kPCh], xv[kPCh];
        size_t id[kPCh];
#pragma unroll
        for (int u = 0; u < kPCh; ++u) {
          const int e = e0 + 32 * u;
          id[u] = e < ne ? own_index(a, rr, e, n) : 0;
          if (e < ne) {
            rv[u] = ldcg(a.r + id[u]);
            if (upd) {
              pv[u] = ldcg(a.p + id[u]);
              qv[u] = ldcg(a.q + id[u]);
              xv[u] = ldcg(a.x + id[u]);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < kPCh; ++u) {
          if (e0 + 32 * u >= ne) continue;
          if (upd) {
            xv[u] += al * pv[u];
            rv[u] = rv[u] - al * qv[u];
            a.x[id[u]] = xv[u];
            a.r[id[u]] = rv[u];
          }
          s += double(rv[u].re) * rv[u].re + double(rv[u].im) * rv[u].im;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0 && rr < kPR) a.part[((size_t)ph * kPR + rr) * gridDim.x + blockIdx.x] = s;
  }
}

// p = z + beta p for the CTA's sites (rhs not done and zz > 0; beta = zz' / zz, zz' in st.red)
WMG_D void pass_p(const PcgArgs& a, PcgState& st, int n) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nown = (a.g.V - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const int ne = nown * n;
#pragma unroll
  for (int h = 0; h < kPR / kPWarps; ++h) {
    const int rr = warp + kPWarps * h;
    if (rr >= a.nrhs || st.done[rr] || !(st.zz[rr] > 0.0)) continue;
    const float be = float(st.red[rr] / st.zz[rr]);
    for (int e0 = lane; e0 < ne; e0 += 32 * kPCh) {
      cf zv[kPCh], pv[kPCh];
      size_t id[kPCh];
#pragma unroll
      for (int u = 0; u < kPCh; ++u) {
        const int e = e0 + 32 * u;
        id[u] = e < ne ? own_index(a, rr, e, n) : 0;
        if (e < ne) {
          zv[u] = ldcg(a.z + id[u]);
          pv[u] = ldcg(a.p + id[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < kPCh; ++u)
        if (e0 + 32 * u < ne) a.p[id[u]] = zv[u] + be * pv[u];
    }
  }
}

template <int NDOF>
__global__ void __launch_bounds__(kPThreads, 1) k_cgnr_persistent(PcgArgs a) {
  extern __shared__ __align__(128) unsigned char smraw[];
  __shared__ PcgState st;
  constexpr int n = NDOF;
  const int V = a.g.V;
  unsigned visit = 0;
  double nacc[2] = {0.0, 0.0};
  // before the CTA ends: the fragment request of the next visit must have landed (bounded)
  auto drain = [&]() {
    if (Smem<NDOF>::NBUF == 2 && threadIdx.x == 0 && V > (int)blockIdx.x)
      mbar_wait_bounded(smem_addr(&st.mbar[visit & 1u]), (visit >> 1) & 1u, kPSpin);
  };
  if (threadIdx.x == 0) {
    mbar_init(smem_addr(&st.mbar[0]), 1);
    mbar_init(smem_addr(&st.mbar[1]), 1);
    mbar_fence_init();
  }
  if (threadIdx.x < kPR) {
    const int r = threadIdx.x;
    st.done[r] = r >= a.nrhs || (a.active && !a.active[r]);
    st.iters[r] = 0;
  }
  __syncthreads();
  if (Smem<NDOF>::NBUF == 2) request_fragments<NDOF>(a, st, smraw, 0);  // during the first passes
  // x = 0, r = b (zero for inactive slots), z = p = 0; |b|^2 -> phase 0
  site_pass(a, st, n, 0, [&](int rr, size_t i) {
    const cf bv = st.done[rr] ? cf{0.f, 0.f} : ldcg(a.b + i);
    a.r[i] = bv;
    a.x[i] = a.p[i] = a.z[i] = cf{0.f, 0.f};
    return bv;
  });
  if (!grid_barrier(a)) return drain();
  reduce_part(a, st, 0);
  if (threadIdx.x < kPR) {
    st.bb[threadIdx.x] = st.red[threadIdx.x];
    if (!(st.red[threadIdx.x] > 0.0)) st.done[threadIdx.x] = 1;
  }
  __syncthreads();
  // z = A^dag r, |z|^2 -> phase 1
  for (int v = blockIdx.x; v < V; v += gridDim.x) site_apply<NDOF>(a, st, smraw, v, a.r, a.z, true, visit, nacc);
  store_norm_part<NDOF>(a, st, 1, nacc);
  if (!grid_barrier(a)) return drain();
  reduce_part(a, st, 1);
  if (threadIdx.x < kPR) st.zz[threadIdx.x] = st.red[threadIdx.x];
  __syncthreads();
  site_pass(a, st, n, -1, [&](int rr, size_t i) {
    a.p[i] = ldcg(a.z + i);
    return cf{0.f, 0.f};
  });
  if (!grid_barrier(a)) return drain();
  for (int it = 0; it < a.maxit; ++it) {
    bool all = true;
    for (int r = 0; r < kPR; ++r) all = all && st.done[r];
    if (all) break;
    // q = A p, |q|^2 -> phase 2
    for (int v = blockIdx.x; v < V; v += gridDim.x) site_apply<NDOF>(a, st, smraw, v, a.p, a.q, false, visit, nacc);
    store_norm_part<NDOF>(a, st, 2, nacc);
    if (!grid_barrier(a)) return drain();
    reduce_part(a, st, 2);
    // x += alpha p, r -= alpha q; |r|^2 -> phase 3
    pass_xr(a, st, n, 3);
    if (!grid_barrier(a)) return drain();
    reduce_part(a, st, 3);
    if (threadIdx.x < kPR) {
      const int r = threadIdx.x;
      if (!st.done[r]) {
        st.iters[r] += 1;
        if (st.red[r] <= a.tol2 * st.bb[r]) st.done[r] = 1;
      }
    }
    __syncthreads();
    all = true;
    for (int r = 0; r < kPR; ++r) all = all && st.done[r];
    if (all || it + 1 == a.maxit) break;
    // z = A^dag r, |z|^2 -> phase 1
    for (int v = blockIdx.x; v < V; v += gridDim.x) site_apply<NDOF>(a, st, smraw, v, a.r, a.z, true, visit, nacc);
    store_norm_part<NDOF>(a, st, 1, nacc);
    if (!grid_barrier(a)) return drain();
    reduce_part(a, st, 1);
    // p = z + beta p
    pass_p(a, st, n);
    __syncthreads();
    if (threadIdx.x < kPR && !st.done[threadIdx.x]) st.zz[threadIdx.x] = st.red[threadIdx.x];
    if (!grid_barrier(a)) return drain();
  }
  if (blockIdx.x == 0 && threadIdx.x < kPR) {
    a.done_out[threadIdx.x] = st.done[threadIdx.x];
    a.iters_out[threadIdx.x] = st.iters[threadIdx.x];
  }
  drain();
}

template <int NDOF>
bool launch_persistent(PcgArgs& a, cudaStream_t s) {
  static int grid = -1;
  const size_t smem = Smem<NDOF>::bytes();
  if (grid < 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_cgnr_persistent<NDOF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cgnr_persistent<NDOF>, kPThreads, smem);
    grid = per >= 1 ? sms : 0;
    if (std::getenv("WMG_DEBUG")) std::fprintf(stderr, "persistent CGNR (2N = %d): %d per SM, grid %d, smem %zu\n", NDOF, per, grid, smem);
  }
  if (grid == 0 || grid > kPersistentMaxGrid) return false;
  void* args[] = {&a};
  const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_cgnr_persistent<NDOF>, dim3(grid), dim3(kPThreads),
                                                    args, smem, s);
  if (e != cudaSuccess && std::getenv("WMG_DEBUG"))
    std::fprintf(stderr, "persistent CGNR (2N = %d): %s\n", NDOF, cudaGetErrorString(e));
  return e == cudaSuccess;
}

}  // namespace

bool cgnr_persistent(const void* A16, const float* sA, const Geom& g, int n, const double* shift, const void* b,
                     void* x, void* r, void* p, void* q, void* z, int nrhs, double tol2, int maxit, const int* active,
                     double* part, unsigned* bar, int* err, int* done_out, int* iters_out, cudaStream_t s) {
  if (nrhs < 1 || nrhs > kPR) return false;
  PcgArgs a{(const uint4*)A16, sA, g, shift, (const cf*)b, (cf*)x, (cf*)r, (cf*)p, (cf*)q, (cf*)z,
            nrhs, tol2, maxit, active, part, bar, err, done_out, iters_out};
  if (cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s) != cudaSuccess) return false;
  bool ok = false;
  switch (n) {
    case 16: ok = launch_persistent<16>(a, s); break;
    case 32: ok = launch_persistent<32>(a, s); break;
    case 48: ok = launch_persistent<48>(a, s); break;
    case 64: ok = launch_persistent<64>(a, s); break;
    default: return false;
  }
  if (ok) count_launch(2);
  return ok;
}

}  // namespace wmg
