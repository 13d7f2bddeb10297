// Tensor-core application of the coarse stencil (Sec. 2 Galerkin operator) to many
// right-hand sides: per coarse site the 9 n x n complex blocks form one n x 9n complex matrix
// A that multiplies the 9n x R matrix X of gathered neighbour values.  In real arithmetic,
//     [Ar; Ai] (2n x 9n)  x  [Xr | Xi] (9n x 2R)  =  [[Ar Xr, Ar Xi], [Ai Xr, Ai Xi]],
// and Yr = Ar Xr - Ai Xi, Yi = Ar Xi + Ai Xr.  One warp owns the row tile of Ar and the
// same row tile of Ai, and the right-hand sides are laid out as column tiles
// [Xr 0..7 | Xi 0..7 | Xr 8..15 | Xi 8..15], so every thread holds all four products of its
// output elements in its own accumulators.
//
// Operands are FP16 with FP32 accumulation (mma.sync m16n8k16): A is stored once per
// setup in FP16 scaled by a per-site factor s_A (max |Re|, |Im| of the site's blocks) and
// pre-arranged in fragment order, so each lane reads one 16-byte word per 16 x 16 tile.  The
// site's fragments (both planes of one row tile are contiguous) arrive in shared memory by
// bulk asynchronous copies issued at kernel start, one per (plane, row tile), completing on
// one mbarrier per row tile (bounded wait); meanwhile the CTA gathers X and converts it in
// shared memory with a per-(site, rhs) factor s_X.  The result is
// rescaled by s_A s_X.  Relative error is about 1e-3 (FP16 operands), enough for the coarse
// solve of a preconditioner.
#include <cstdlib>

#include <cuda_fp16.h>

#include "kernels.h"
#include "ptx.cuh"
#include "mma_sync.cuh"

namespace wmg {

namespace {

constexpr long long kMmaSpinLimit = 1LL << 22;

__device__ int g_mma_error = 0;

}  // namespace

// Per-site scale: max over the site's 9 n x n blocks of |Re| and |Im|.
template <typename R>
__global__ void k_stencil_site_scale(const cpx<R>* __restrict__ A, int n, float* __restrict__ scale) {
  const int v = blockIdx.x;
  const size_t cnt = (size_t)9 * n * n;
  float m = 0.f;
  for (size_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    const cpx<R> a = A[(size_t)v * cnt + i];
    m = fmaxf(m, fmaxf(fabsf((float)a.re), fabsf((float)a.im)));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, sm[w]);
    scale[v] = t > 0.f ? t : 1.f;
  }
}

// Fragment-order FP16 copy of the stencil: [site][plane][mtile][kstep][lane] uint4, where
// plane 0 = Re, 1 = Im, and the 16 x 16 tile (rows 16 mtile.., k 16 kstep..) of the real
// n x 9n matrix of that plane is held as the m16n8k16 A fragment of each lane.
template <typename R>
__global__ void k_stencil_to_mma(const cpx<R>* __restrict__ A, int n, const float* __restrict__ scale,
                                 uint4* __restrict__ out, int Vc) {
  const int mt = n / 16, ks = 9 * n / 16;
  const size_t per_site = (size_t)2 * mt * ks * 32;
  const size_t total = per_site * Vc;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int lane = (int)(idx % 32);
    size_t t = idx / 32;
    const int kk = (int)(t % ks);
    t /= ks;
    const int m = (int)(t % mt);
    t /= mt;
    const int plane = (int)(t % 2);
    const int v = (int)(t / 2);
    const float inv = 1.f / scale[v];
    const int g = lane >> 2, q = lane & 3;
    auto val = [&](int row, int k) -> float {  // row of the n x 9n block matrix, k = slot * n + col
      const cpx<R> a = A[(((size_t)v * 9 + k / n) * n + (k % n)) * n + row];
      return (float)(plane == 0 ? a.re : a.im) * inv;
    };
    const int r0 = 16 * m + g, r1 = r0 + 8, c0 = 16 * kk + 2 * q, c1 = c0 + 8;
    uint4 w;
    w.x = pack_half2(val(r0, c0), val(r0, c0 + 1));
    w.y = pack_half2(val(r1, c0), val(r1, c0 + 1));
    w.z = pack_half2(val(r0, c1), val(r0, c1 + 1));
    w.w = pack_half2(val(r1, c1), val(r1, c1 + 1));
    out[idx] = w;
  }
}

// y = A x (+ shift x), optionally sigma_3 A sigma_3 x, for a chunk of up to 8 NT right-hand
// sides per CTA (grid.y chunks), n = NDOF coarse dof.  One CTA of 8 warps per coarse site.
// Every warp gathers X for R / 8 right-hand sides (all loads of the warp in flight together)
// and converts it to FP16 in shared memory; warp w < MT NT owns row tile m = w % MT and the
// column block of right-hand sides 8 (w / MT) .. + 7 (its Xr and Xi tiles).
constexpr int kMmaThreads = 256;
template <int NDOF, int NT>
__global__ void __launch_bounds__(kMmaThreads, 2) k_coarse_apply_mma(const uint4* __restrict__ A16,
                                                                     const float* __restrict__ sA, Geom g,
                                                                     const cf* in, cf* out,
                                                                     int nrhs, const double* __restrict__ shift,
                                                                     int dagger, const int* __restrict__ active,
                                                                     RedBuf rb, int want_norm, StencilEo eo,
                                                                     int* __restrict__ err) {
  constexpr int n = NDOF, N = n / 2, K = 9 * n, KP = K + kKPad;
  constexpr int MT = n / 16, KS = K / 16;
  constexpr int R = 8 * NT, COLS = 2 * R;
  constexpr int NW = kMmaThreads / 32, RPW = (R + NW - 1) / NW;  // right-hand sides per warp
  constexpr int EPL = (K + 31) / 32;                              // gathered values per lane
  constexpr uint32_t kTileBytes = (uint32_t)KS * 32 * 16;         // one plane of one row tile
  extern __shared__ __align__(128) unsigned char smraw[];
  uint4* As = reinterpret_cast<uint4*>(smraw);                                        // [2][MT][KS][32]
  __half* xb = reinterpret_cast<__half*>(smraw + (size_t)2 * MT * kTileBytes);        // [COLS][KP]
  float* xmax = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(xb) + (size_t)COLS * KP * sizeof(__half));
  __shared__ __align__(8) unsigned long long mbar[MT];
  __shared__ int nbs[9];
  __shared__ double npart[NW][32][2];  // per-lane norm partials of the MMA warps
  const int v = eo.parity < 0 ? (int)blockIdx.x : parity_site(g, blockIdx.x, eo.parity);
  // the operator (and its scale) of this site: the level's, or the precomputed odd-site pass
  const uint4* Aop = eo.opB ? reinterpret_cast<const uint4*>(eo.opB) : A16;
  const int vop = eo.opB ? (int)blockIdx.x : v;
  const float s_site = eo.opB ? eo.sB[blockIdx.x] : sA[v];
  const int r0 = blockIdx.y * R;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool mma_warp = warp < MT * NT;
  const int m = warp % MT, blk = warp / MT;
  if (threadIdx.x == 0) {
    for (int t = 0; t < MT; ++t) mbar_init(smem_addr(&mbar[t]), 1);
    mbar_fence_init();
    for (int t = 0; t < MT; ++t) {
      const uint32_t bar = smem_addr(&mbar[t]);
      mbar_arrive_expect_tx(bar, 2 * kTileBytes);
      for (int p = 0; p < 2; ++p)
        bulk_g2s(smem_addr(As + (size_t)(p * MT + t) * KS * 32), Aop + (((size_t)vop * 2 + p) * MT + t) * KS * 32,
                 kTileBytes, bar);
    }
  }
  if (threadIdx.x < 9) {
    int c[4];
    site_coords(g, v, c);
    const int k = threadIdx.x;
    nbs[k] = k == 0 ? v : neighbour(g, v, c, (k - 1) >> 1, ((k - 1) & 1) ? -1 : +1);
  }
  __syncthreads();
  // lane-owned elements e = lane + 32 i of the 9n gathered values (same for every rhs)
  int offs[EPL];
  unsigned neg = 0;   // bit i: sigma_3 sign flip of element i (adjoint, lower half of the dof)
  unsigned hopm = 0;  // bit i: element i is a neighbour value read from eo.hop_in
#pragma unroll
  for (int i = 0; i < EPL; ++i) {
    const int e = lane + 32 * i;
    offs[i] = -1;
    if (e < K) {
      const int k = e / n, j = e - k * n;
      if (!(k == 0 && eo.hop_only)) offs[i] = nbs[k] * n + j;
      if (dagger && j >= N) neg |= 1u << i;
      if (k > 0 && eo.hop_in) hopm |= 1u << i;
    }
  }
  const cf* hin = eo.hop_in ? reinterpret_cast<const cf*>(eo.hop_in) : in;
  // everything above reads only the operator tables and the geometry: with a programmatic launch
  // it overlaps the end of the previous kernel, whose results are read from here on (`in`, `out`
  // and the vectors of eo are plain pointers, so that no load of them is taken as invariant and
  // issued before the wait)
  griddep_wait();
  // gather this warp's right-hand sides (all loads first), then per rhs the max |Re|, |Im| by
  // shuffles and the scaled FP16 copy in column layout [Xr 0..7 | Xi 0..7 | Xr 8..15 | Xi 8..15]
  cf xv[RPW][EPL];
#pragma unroll
  for (int h = 0; h < RPW; ++h) {
    const int rr = warp + NW * h, r = r0 + rr;
    const bool ok = rr < R && r < nrhs;
    const size_t rb0 = (size_t)(ok ? r : 0) * g.V * n;
    const cf* src = in + rb0;
    const cf* hsrc = hin + rb0;
#pragma unroll
    for (int i = 0; i < EPL; ++i)
      xv[h][i] = (ok && offs[i] >= 0) ? (((hopm >> i) & 1u) ? hsrc : src)[offs[i]] : cf{0.f, 0.f};
  }
#pragma unroll
  for (int h = 0; h < RPW; ++h) {
    const int rr = warp + NW * h;
    if (rr >= R) continue;
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < EPL; ++i) mx = fmaxf(mx, fmaxf(fabsf(xv[h][i].re), fabsf(xv[h][i].im)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) xmax[rr] = mx;
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
  const int gq = lane >> 2, q = lane & 3;
  float acc[2][2][4];  // [plane Ar / Ai][tile Xr / Xi][fragment]
#pragma unroll
  for (int p = 0; p < 2; ++p)
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[p][t][e] = 0.f;
  bool ready = true;
  if (mma_warp) {
    ready = mbar_wait_bounded(smem_addr(&mbar[m]), 0, kMmaSpinLimit);
    if (!ready && lane == 0) atomicExch(err ? err : &g_mma_error, 1);
  }
  if (mma_warp && ready) {
    const uint4* Ar = As + (size_t)(0 * MT + m) * KS * 32 + lane;
    const uint4* Ai = As + (size_t)(1 * MT + m) * KS * 32 + lane;
    const __half* colbase = xb + (size_t)(blk * 16 + gq) * KP + 2 * q;
    const int k0 = eo.hop_only ? n / 16 : 0;  // the site's own block fills the first n / 16 k-steps
#pragma unroll 9
    for (int k = k0; k < KS; ++k) {
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
  }
  griddep_launch_dependents();  // the next kernel may start its own table-only prologue
  // a tile whose wait expired: give its copies a second bounded chance to land before exit
  if (mma_warp && !ready) mbar_wait_bounded(smem_addr(&mbar[m]), 0, kMmaSpinLimit);
  if (eo.inv) {
    // odd-site pass of the Schur complement: u = -M_r h with h = A_oe x (this CTA's result,
    // before the adjoint's output sigma_3) and M_r = A_oo^-1 of the rhs's table entry; for the
    // adjoint -sigma_3 M_r h (= -sigma_3 M_r sigma_3 of the sigma_3-flipped result).  h goes
    // through shared memory (the FP16 staging area, free once every warp is past its MMAs);
    // thread (row, rhs) forms the row's dot product, the inverse read by columns.
    __syncthreads();
    cf* hs = reinterpret_cast<cf*>(xb);  // [R][n]
    if (mma_warp) {
      const float s_a = s_site;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int row = 16 * m + gq + (e >= 2 ? 8 : 0);
        const int rr = blk * 8 + 2 * q + (e & 1);
        const float sc = s_a * xmax[rr];
        hs[rr * n + row] = cf{(acc[0][0][e] - acc[1][1][e]) * sc, (acc[0][1][e] + acc[1][0][e]) * sc};
      }
    }
    __syncthreads();
    const cf* inv = reinterpret_cast<const cf*>(eo.inv);
    for (int t = threadIdx.x; t < n * R; t += kMmaThreads) {
      const int rr = t / n, row = t - rr * n, r = r0 + rr;
      if (r >= nrhs) continue;
      const float2* mcol =
          reinterpret_cast<const float2*>(inv + ((size_t)eo.inv_idx[r] * (g.V / 2) + blockIdx.x) * n * n + row);
      const cf* h = hs + rr * n;
      cf u{0.f, 0.f};
#pragma unroll 8
      for (int col = 0; col < n; ++col) {
        const float2 a = __ldg(mcol + (size_t)col * n);
        cfma(u, cf{a.x, a.y}, h[col]);
      }
      const float sg = (dagger && row >= N) ? 1.f : -1.f;
      if (!active || active[r]) out[((size_t)r * g.V + v) * n + row] = cf{sg * u.re, sg * u.im};
    }
    return;
  }
  // epilogue: thread holds rows 16 m + gq (+8) and right-hand sides 8 blk + 2q + (e & 1)
  float nv2[2] = {0.f, 0.f};  // the thread's sums in FP32, FP64 across lanes, warps and CTAs
  if (mma_warp) {
    const float s_a = s_site;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int row = 16 * m + gq + (e >= 2 ? 8 : 0);
      const int rr = blk * 8 + 2 * q + (e & 1);
      const int r = r0 + rr;
      if (r >= nrhs) continue;
      // tile 0 = Xr, 1 = Xi; plane 0 = Ar, 1 = Ai
      const float yr = acc[0][0][e] - acc[1][1][e];
      const float yi = acc[0][1][e] + acc[1][0][e];
      const float sc = s_a * xmax[rr] * ((dagger && row >= N) ? -1.f : 1.f);
      cf o{yr * sc, yi * sc};
      if (shift && !eo.hop_only && !eo.opB) o += (float)shift[r] * in[((size_t)r * g.V + v) * n + row];
      if (eo.add) o += reinterpret_cast<const cf*>(eo.add)[((size_t)r * g.V + v) * n + row];
      if (!active || active[r]) out[((size_t)r * g.V + v) * n + row] = o;
      nv2[e & 1] += o.re * o.re + o.im * o.im;
    }
  }
  if (want_norm) {
    if (mma_warp) {
      npart[warp][lane][0] = nv2[0];
      npart[warp][lane][1] = nv2[1];
    }
    __syncthreads();
    __shared__ bool last;
    const int nblk = gridDim.x;
    if (threadIdx.x < R && r0 + (int)threadIdx.x < nrhs) {
      // fixed order: row tiles, then the 8 row groups of the fragment
      const int rr = threadIdx.x, b = rr >> 3, qq = (rr & 7) >> 1, ee = rr & 1;
      double t = 0.0;
      for (int mm = 0; mm < MT; ++mm)
        for (int gg = 0; gg < 8; ++gg) t += npart[b * MT + mm][gg * 4 + qq][ee];
      rb.partial[(size_t)(r0 + rr) * nblk + blockIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(rb.counter + blockIdx.y, 1u) == (unsigned)nblk - 1;
    __syncthreads();
    if (last) {
      __threadfence();
      const int nvals = min(R, nrhs - r0);
      cta_multi_sum(rb.partial + (size_t)r0 * nblk, nvals, (size_t)nblk, nblk, 1, [&](int i, double s) {
        if (!active || active[r0 + i]) rb.result[r0 + i] = s;  // a masked launch leaves the others' sums
      });
      if (threadIdx.x == 0) rb.counter[blockIdx.y] = 0u;
    }
  }
}

int coarse_mma_error() {
  int e = 0;
  cudaMemcpyFromSymbol(&e, g_mma_error, sizeof(int));
  return e;
}

size_t stencil_mma_words(int Vc, int n) { return (size_t)Vc * 2 * (n / 16) * (9 * n / 16) * 32; }

void stencil_to_mma(int prec, const void* A, int Vc, int n, float* scale, void* out, cudaStream_t s) {
  count_launch(2);
  if (prec == WMG_PREC_DOUBLE) k_stencil_site_scale<double><<<Vc, 256, 0, s>>>((const cd*)A, n, scale);
  else k_stencil_site_scale<float><<<Vc, 256, 0, s>>>((const cf*)A, n, scale);
  const size_t tot = stencil_mma_words(Vc, n);
  int B = (int)((tot + 255) / 256);
  if (B > 148 * 32) B = 148 * 32;
  if (prec == WMG_PREC_DOUBLE) k_stencil_to_mma<double><<<B, 256, 0, s>>>((const cd*)A, n, scale, (uint4*)out, Vc);
  else k_stencil_to_mma<float><<<B, 256, 0, s>>>((const cf*)A, n, scale, (uint4*)out, Vc);
}

template <int NDOF, int NT>
static void launch_mma(const void* A16, const float* sA, const Geom& g, const void* in, void* out, int nrhs,
                       const double* shift, bool dagger, const int* active, const RedBuf* rb, cudaStream_t s,
                       const StencilEo& eo, int* err) {
  constexpr int R = 8 * NT;
  const size_t smem = (size_t)2 * (NDOF / 16) * (9 * NDOF / 16) * 512 +
                      (size_t)2 * R * (9 * NDOF + kKPad) * sizeof(__half) + R * sizeof(float);
  static const bool attr = [] {
    cudaFuncSetAttribute(k_coarse_apply_mma<NDOF, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    return true;
  }();
  (void)attr;
  dim3 grid(eo.parity < 0 ? g.V : g.V / 2, (nrhs + R - 1) / R);
  RedBuf r = rb ? *rb : RedBuf{nullptr, nullptr, nullptr};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kMmaThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_launches() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k_coarse_apply_mma<NDOF, NT>, (const uint4*)A16, sA, g, (const cf*)in, (cf*)out, nrhs,
                     shift, dagger ? 1 : 0, active, r, rb ? 1 : 0, eo, err);
}

template <int NDOF>
static void launch_mma_n(const void* A16, const float* sA, const Geom& g, const void* in, void* out, int nrhs,
                         const double* shift, bool dagger, const int* active, const RedBuf* rb, cudaStream_t s,
                         const StencilEo& eo, int* err) {
  static const int nt_max = [] {
    const char* e = std::getenv("WMG_MMA_NT");
    return (e && e[0] == '1') ? 1 : 2;
  }();
  if (nrhs <= 8 || nt_max == 1) launch_mma<NDOF, 1>(A16, sA, g, in, out, nrhs, shift, dagger, active, rb, s, eo, err);
  else launch_mma<NDOF, 2>(A16, sA, g, in, out, nrhs, shift, dagger, active, rb, s, eo, err);
}

// n = 2N in {16, 32, 48, 64} (the tensor-core copy exists only for those)
void coarse_apply_mma(const void* A16, const float* sA, const Geom& g, int n, const void* in, void* out, int nrhs,
                      const double* shift, bool dagger, const int* active, const RedBuf* rb, cudaStream_t s,
                      const StencilEo* eo_opt, int* err) {
  count_launch();
  const StencilEo eo = eo_opt ? *eo_opt : StencilEo{};
  switch (n) {
    case 16: launch_mma_n<16>(A16, sA, g, in, out, nrhs, shift, dagger, active, rb, s, eo, err); break;
    case 32: launch_mma_n<32>(A16, sA, g, in, out, nrhs, shift, dagger, active, rb, s, eo, err); break;
    case 48: launch_mma_n<48>(A16, sA, g, in, out, nrhs, shift, dagger, active, rb, s, eo, err); break;
    default: launch_mma_n<64>(A16, sA, g, in, out, nrhs, shift, dagger, active, rb, s, eo, err); break;
  }
}

}  // namespace wmg
