// The coarsest-level solve (CG on the normal equations, Sec. 3) as one persistent cooperative
// kernel for up to 16 right-hand sides.  Each CTA owns fixed coarse sites v = blockIdx.x + k G and
// performs, for them, the tensor-core stencil applications and the vector updates; grid barriers
// separate the phases that read neighbour values or global sums.  Per iteration:
//     q = A p, |q|^2 | alpha = zz / qq; x += alpha p; r -= alpha q; |r|^2 | convergence;
//     z = A^dag r, |z|^2 | beta = zz' / zz; p = z + beta p |
// The vector passes also write FP16 copies of p and sigma_3 r in the B-fragment order of
// mma.sync m16n8k16, scaled per (site, rhs) by the largest |Re|, |Im| of the site's values.  A
// stencil application is a set of independent warp units (site, 16-row tile, 8-rhs block): per
// neighbour slot the unit multiplies the site's FP16 operator fragments by the neighbour's vector
// fragments (both read from L2, no staging), then rescales that slot's partial sums by the
// neighbour's scales (D^dag = sigma_3 D sigma_3: sigma_3 of the input is in r's copy, that of the
// output in the epilogue).  Per-rhs sums are formed per CTA in a fixed order, stored as
// [phase][rhs][CTA] partials and summed over the CTAs in a fixed order by every CTA, so all CTAs
// take the same decisions and a right-hand side's arithmetic does not depend on the others.
// Every grid-barrier wait is bounded; on expiry the kernel records an error, which the solve
// reports.
#include <cuda_fp16.h>

#include <cstdio>
#include <cstdlib>

#include "kernels.h"
#include "mma_sync.cuh"

namespace wmg {
namespace {

constexpr int kPThreads = 256;
constexpr int kPR = 16;                  // right-hand sides of the kernel
constexpr int kPNT = 2;                  // 8-rhs column blocks
constexpr int kPWarps = kPThreads / 32;
constexpr long long kPSpin = 1LL << 22;  // polls of a barrier wait before it gives up

struct PcgArgs {
  const uint4* A16;
  const float* sA;
  Geom g;
  const double* shift;  // per-rhs diagonal shift of this level's stencil
  const cf* b;
  cf *x, *r, *p, *q, *z;
  __half *r16, *p16;    // fragment-order FP16 copies of sigma_3 r and of p: [site][blk][kstep][lane][8]
  float *rsc, *psc;     // their scales [site][kPR]
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

// Per-CTA state, identical in every CTA (derived from the same global sums).
struct PcgState {
  double bb[kPR], zz[kPR], red[kPR];
  int done[kPR], iters[kPR];
  double wsum[kPWarps][kPR];  // per-warp norm sums of the current application
};

WMG_D cf ldcg(const cf* p) {
  const float2 u = __ldcg(reinterpret_cast<const float2*>(p));
  return cf{u.x, u.y};
}

WMG_D int own_sites(const PcgArgs& a) { return (a.g.V - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x; }

// Index (in halves) of component j, part t (0 Re, 1 Im), of right-hand side rr of site v in a
// fragment-order copy: B fragment of lane gq*4 + q holds k = 2q, 2q+1 (word 0) and 2q+8, 2q+9
// (word 1) of column gq; a lane's 16 bytes are {Re word 0, Re word 1, Im word 0, Im word 1}.
WMG_D size_t frag_half(int v, int rr, int j, int t, int n) {
  const int blk = rr >> 3, gq = rr & 7, kk = j >> 4, jj = j & 15;
  const int q = (jj & 7) >> 1, hi = jj >> 3, lane = gq * 4 + q;
  return ((((size_t)v * kPNT + blk) * (n / 16) + kk) * 32 + lane) * 8 + (t * 2 + hi) * 2 + (jj & 1);
}

// The warp's values val[u] (components j = lane + 32 u) of rhs rr at site v into a copy: scale
// = max |Re|, |Im| over the site (warp shuffles); sigma_3 flips the lower half if sg3.
template <int NE>
WMG_D void write_frag(__half* dst, float* sc, int v, int rr, int n, const cf val[NE], bool sg3) {
  const int lane = threadIdx.x & 31, N = n / 2;
  float mx = 0.f;
#pragma unroll
  for (int u = 0; u < NE; ++u)
    if (lane + 32 * u < n) mx = fmaxf(mx, fmaxf(fabsf(val[u].re), fabsf(val[u].im)));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const float inv = mx > 0.f ? 1.f / mx : 0.f;
#pragma unroll
  for (int u = 0; u < NE; ++u) {
    const int j = lane + 32 * u;
    if (j >= n) continue;
    const float s = (sg3 && j >= N) ? -inv : inv;
    dst[frag_half(v, rr, j, 0, n)] = __float2half_rn(val[u].re * s);
    dst[frag_half(v, rr, j, 1, n)] = __float2half_rn(val[u].im * s);
  }
  if (lane == 0) sc[(size_t)v * kPR + rr] = mx;
}

// One stencil application to the CTA's sites: out = A in (dagger: sigma_3 A sigma_3) + shift in,
// from the FP16 copy (in16, insc) of the input; |out|^2 per rhs into st.wsum.
template <int NDOF>
WMG_D void apply_units(const PcgArgs& a, PcgState& st, const __half* in16, const float* insc, const cf* in32, cf* out,
                       bool dagger) {
  constexpr int n = NDOF, N = n / 2, MT = n / 16, KPS = n / 16, KS = 9 * KPS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, gq = lane >> 2, q = lane & 3;
  const int nt = a.nrhs > 8 ? 2 : 1;
  const int units = own_sites(a) * MT * nt;
  const Geom& g = a.g;
  const uint4* X = reinterpret_cast<const uint4*>(in16);
  for (int u = warp; u < units; u += kPWarps) {
    const int k = u / (MT * nt), rem = u - k * (MT * nt), m = rem % MT, blk = rem / MT;
    const int v = blockIdx.x + k * gridDim.x;
    int c[4];
    site_coords(g, v, c);
    const uint4* Ar = a.A16 + ((size_t)v * 2 * MT + m) * KS * 32 + lane;
    const uint4* Ai = a.A16 + ((size_t)(v * 2 + 1) * MT + m) * KS * 32 + lane;
    float acc[2][2][4];
#pragma unroll
    for (int pl = 0; pl < 2; ++pl)
#pragma unroll
      for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[pl][t][e] = 0.f;
    // the fragments of slot s + 1 are requested before slot s is multiplied
    uint4 fa[2][KPS], fi[2][KPS], fb[2][KPS];
    float sc0[2], sc1[2];
    auto fetch = [&](int s, int bsel) {
      const int nb = s == 0 ? v : neighbour(g, v, c, (s - 1) >> 1, ((s - 1) & 1) ? -1 : +1);
#pragma unroll
      for (int kk = 0; kk < KPS; ++kk) {
        fa[bsel][kk] = __ldg(Ar + (size_t)(s * KPS + kk) * 32);
        fi[bsel][kk] = __ldg(Ai + (size_t)(s * KPS + kk) * 32);
        fb[bsel][kk] = __ldcg(X + (((size_t)nb * kPNT + blk) * KPS + kk) * 32 + lane);
      }
      sc0[bsel] = __ldcg(insc + (size_t)nb * kPR + blk * 8 + 2 * q);
      sc1[bsel] = __ldcg(insc + (size_t)nb * kPR + blk * 8 + 2 * q + 1);
    };
    fetch(0, 0);
#pragma unroll
    for (int s = 0; s < 9; ++s) {
      const int cur = s & 1;
      if (s + 1 < 9) fetch(s + 1, cur ^ 1);
      float t[2][2][4];
#pragma unroll
      for (int pl = 0; pl < 2; ++pl)
#pragma unroll
        for (int tt = 0; tt < 2; ++tt)
#pragma unroll
          for (int e = 0; e < 4; ++e) t[pl][tt][e] = 0.f;
#pragma unroll
      for (int kk = 0; kk < KPS; ++kk) {
        mma16816(t[0][0], fa[cur][kk], fb[cur][kk].x, fb[cur][kk].y);
        mma16816(t[1][0], fi[cur][kk], fb[cur][kk].x, fb[cur][kk].y);
        mma16816(t[0][1], fa[cur][kk], fb[cur][kk].z, fb[cur][kk].w);
        mma16816(t[1][1], fi[cur][kk], fb[cur][kk].z, fb[cur][kk].w);
      }
#pragma unroll
      for (int pl = 0; pl < 2; ++pl)
#pragma unroll
        for (int tt = 0; tt < 2; ++tt)
#pragma unroll
          for (int e = 0; e < 4; ++e)
            acc[pl][tt][e] = fmaf(t[pl][tt][e], (e & 1) ? sc1[cur] : sc0[cur], acc[pl][tt][e]);
    }
    // epilogue: rows 16 m + gq (+8), right-hand sides blk*8 + 2q + (e & 1)
    const float s_a = a.sA[v];
    double nv[2] = {0.0, 0.0};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int row = 16 * m + gq + (e >= 2 ? 8 : 0);
      const int rr = blk * 8 + 2 * q + (e & 1);
      if (rr >= a.nrhs) continue;
      const float yr = acc[0][0][e] - acc[1][1][e];
      const float yi = acc[0][1][e] + acc[1][0][e];
      const float sc = s_a * ((dagger && row >= N) ? -1.f : 1.f);
      cf o{yr * sc, yi * sc};
      const size_t idx = ((size_t)rr * g.V + v) * n + row;
      if (a.shift) o += (float)a.shift[rr] * ldcg(in32 + idx);
      out[idx] = o;
      nv[e & 1] += double(o.re) * o.re + double(o.im) * o.im;
    }
    // sum over the 8 row groups (lanes with the same q), then one lane per column adds in
#pragma unroll
    for (int cc = 0; cc < 2; ++cc)
#pragma unroll
      for (int o = 4; o < 32; o <<= 1) nv[cc] += __shfl_xor_sync(0xffffffffu, nv[cc], o);
    if (gq == 0)
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) st.wsum[warp][blk * 8 + 2 * q + cc] += nv[cc];
  }
}

// the CTA's application sums (warps in order) -> part[ph][rhs][cta]; clears the warp sums
WMG_D void store_apply_part(const PcgArgs& a, PcgState& st, int ph) {
  __syncthreads();
  if (threadIdx.x < kPR) {
    double t = 0.0;
    for (int w = 0; w < kPWarps; ++w) {
      t += st.wsum[w][threadIdx.x];
      st.wsum[w][threadIdx.x] = 0.0;
    }
    a.part[((size_t)ph * kPR + threadIdx.x) * gridDim.x + blockIdx.x] = t;
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

// Per-site vector pass over the CTA's sites: warp w takes right-hand sides w and w + 8 (also the
// padding ones up to 16, whose copies stay zero), lanes the components j = lane + 32 u.  f(rr, idx,
// val) fills the NE values of the site (idx[u] = index of component lane + 32 u, valid if < n);
// with dst they also go into a copy (scales sc, sigma_3 if sg3); |val|^2 enters part[ph] unless
// ph < 0.
template <int NE, typename F>
WMG_D void site_pass(const PcgArgs& a, int n, int ph, __half* dst, float* sc, bool sg3, F f) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nown = own_sites(a);
#pragma unroll
  for (int h = 0; h < kPR / kPWarps; ++h) {
    const int rr = warp + kPWarps * h;
    double s = 0.0;
    for (int k = 0; k < nown; ++k) {
      const int v = blockIdx.x + k * gridDim.x;
      cf val[NE];
      size_t idx[NE];
#pragma unroll
      for (int u = 0; u < NE; ++u) {
        idx[u] = ((size_t)rr * a.g.V + v) * n + lane + 32 * u;
        val[u] = cf{0.f, 0.f};
      }
      if (rr < a.nrhs) f(rr, idx, val);
#pragma unroll
      for (int u = 0; u < NE; ++u)
        if (lane + 32 * u < n) s += double(val[u].re) * val[u].re + double(val[u].im) * val[u].im;
      if (dst) write_frag<NE>(dst, sc, v, rr, n, val, sg3);
    }
    if (ph >= 0) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) a.part[((size_t)ph * kPR + rr) * gridDim.x + blockIdx.x] = s;
    }
  }
}

template <int NDOF>
__global__ void __launch_bounds__(kPThreads) k_cgnr_persistent(PcgArgs a) {
  __shared__ PcgState st;
  constexpr int n = NDOF, NE = (n + 31) / 32;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x < kPR) {
    const int r = threadIdx.x;
    st.done[r] = r >= a.nrhs || (a.active && !a.active[r]);
    st.iters[r] = 0;
    for (int w = 0; w < kPWarps; ++w) st.wsum[w][r] = 0.0;
  }
  __syncthreads();
  // x = 0, r = b (zero for inactive slots), z = p = 0; sigma_3 r -> copy; |b|^2 -> phase 0
  site_pass<NE>(a, n, 0, a.r16, a.rsc, true, [&](int rr, const size_t* idx, cf* val) {
#pragma unroll
    for (int u = 0; u < NE; ++u) {
      if (lane + 32 * u >= n) continue;
      const cf bv = st.done[rr] ? cf{0.f, 0.f} : ldcg(a.b + idx[u]);
      a.r[idx[u]] = bv;
      a.x[idx[u]] = a.p[idx[u]] = a.z[idx[u]] = cf{0.f, 0.f};
      val[u] = bv;
    }
  });
  if (!grid_barrier(a)) return;
  reduce_part(a, st, 0);
  if (threadIdx.x < kPR) {
    st.bb[threadIdx.x] = st.red[threadIdx.x];
    if (!(st.red[threadIdx.x] > 0.0)) st.done[threadIdx.x] = 1;
  }
  __syncthreads();
  // z = A^dag r, |z|^2 -> phase 1
  apply_units<NDOF>(a, st, a.r16, a.rsc, a.r, a.z, true);
  store_apply_part(a, st, 1);
  if (!grid_barrier(a)) return;
  reduce_part(a, st, 1);
  if (threadIdx.x < kPR) st.zz[threadIdx.x] = st.red[threadIdx.x];
  __syncthreads();
  // p = z -> copy
  site_pass<NE>(a, n, -1, a.p16, a.psc, false, [&](int rr, const size_t* idx, cf* val) {
#pragma unroll
    for (int u = 0; u < NE; ++u) {
      if (lane + 32 * u >= n) continue;
      val[u] = ldcg(a.z + idx[u]);
      a.p[idx[u]] = val[u];
    }
  });
  if (!grid_barrier(a)) return;
  for (int it = 0; it < a.maxit; ++it) {
    bool all = true;
    for (int r = 0; r < kPR; ++r) all = all && st.done[r];
    if (all) break;
    // q = A p, |q|^2 -> phase 2
    apply_units<NDOF>(a, st, a.p16, a.psc, a.p, a.q, false);
    store_apply_part(a, st, 2);
    if (!grid_barrier(a)) return;
    reduce_part(a, st, 2);
    // x += alpha p, r -= alpha q (rhs not done); sigma_3 r -> copy; |r|^2 -> phase 3
    site_pass<NE>(a, n, 3, a.r16, a.rsc, true, [&](int rr, const size_t* idx, cf* val) {
      const double qq = st.red[rr];
      const bool upd = !st.done[rr] && qq > 0.0;
      const float al = upd ? float(st.zz[rr] / qq) : 0.f;
      cf pv[NE], qv[NE], xv[NE];
#pragma unroll
      for (int u = 0; u < NE; ++u) {
        if (lane + 32 * u >= n) continue;
        val[u] = ldcg(a.r + idx[u]);
        if (upd) {
          pv[u] = ldcg(a.p + idx[u]);
          qv[u] = ldcg(a.q + idx[u]);
          xv[u] = ldcg(a.x + idx[u]);
        }
      }
      if (!upd) return;
#pragma unroll
      for (int u = 0; u < NE; ++u) {
        if (lane + 32 * u >= n) continue;
        xv[u] += al * pv[u];
        val[u] = val[u] - al * qv[u];
        a.x[idx[u]] = xv[u];
        a.r[idx[u]] = val[u];
      }
    });
    if (!grid_barrier(a)) return;
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
    apply_units<NDOF>(a, st, a.r16, a.rsc, a.r, a.z, true);
    store_apply_part(a, st, 1);
    if (!grid_barrier(a)) return;
    reduce_part(a, st, 1);
    // p = z + beta p (rhs not done) -> copy
    site_pass<NE>(a, n, -1, a.p16, a.psc, false, [&](int rr, const size_t* idx, cf* val) {
      const bool upd = !st.done[rr] && st.zz[rr] > 0.0;
      const float be = upd ? float(st.red[rr] / st.zz[rr]) : 0.f;
      cf zv[NE];
#pragma unroll
      for (int u = 0; u < NE; ++u) {
        if (lane + 32 * u >= n) continue;
        val[u] = ldcg(a.p + idx[u]);
        if (upd) zv[u] = ldcg(a.z + idx[u]);
      }
      if (!upd) return;
#pragma unroll
      for (int u = 0; u < NE; ++u) {
        if (lane + 32 * u >= n) continue;
        val[u] = zv[u] + be * val[u];
        a.p[idx[u]] = val[u];
      }
    });
    __syncthreads();
    if (threadIdx.x < kPR && !st.done[threadIdx.x]) st.zz[threadIdx.x] = st.red[threadIdx.x];
    if (!grid_barrier(a)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x < kPR) {
    a.done_out[threadIdx.x] = st.done[threadIdx.x];
    a.iters_out[threadIdx.x] = st.iters[threadIdx.x];
  }
}

template <int NDOF>
bool launch_persistent(PcgArgs& a, cudaStream_t s) {
  static int grid = -1;
  if (grid < 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cgnr_persistent<NDOF>, kPThreads, 0);
    grid = sms * (per >= 2 ? 2 : per);
    if (std::getenv("WMG_DEBUG")) std::fprintf(stderr, "persistent CGNR (2N = %d): %d per SM, grid %d\n", NDOF, per, grid);
  }
  if (grid <= 0 || grid > kPersistentMaxGrid) return false;
  void* args[] = {&a};
  const cudaError_t e =
      cudaLaunchCooperativeKernel((const void*)k_cgnr_persistent<NDOF>, dim3(grid), dim3(kPThreads), args, 0, s);
  if (e != cudaSuccess && std::getenv("WMG_DEBUG"))
    std::fprintf(stderr, "persistent CGNR (2N = %d): %s\n", NDOF, cudaGetErrorString(e));
  return e == cudaSuccess;
}

}  // namespace

size_t cgnr_persistent_copy_bytes(int Vc, int n) { return (size_t)Vc * kPNT * (n / 16) * 32 * 16; }

bool cgnr_persistent(const void* A16, const float* sA, const Geom& g, int n, const double* shift, const void* b,
                     void* x, void* r, void* p, void* q, void* z, void* r16, void* p16, float* rsc, float* psc,
                     int nrhs, double tol2, int maxit, const int* active, double* part, unsigned* bar, int* err,
                     int* done_out, int* iters_out, cudaStream_t s) {
  if (nrhs < 1 || nrhs > kPR) return false;
  PcgArgs a{(const uint4*)A16, sA, g, shift, (const cf*)b, (cf*)x, (cf*)r, (cf*)p, (cf*)q, (cf*)z,
            (__half*)r16, (__half*)p16, rsc, psc, nrhs, tol2, maxit, active, part, bar, err, done_out, iters_out};
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
