// Coarse stencil on many right-hand sides with Blackwell tcgen05 tensor cores.
//
// Per coarse site v the 9 n x n complex blocks form the n x 9n matrix A; with X the 9n x R
// gathered neighbour values (R = 16 right-hand sides per chunk),
//     D (128 x 32) = [Ar; Ai; 0] (128 x 9n)  x  [Xr | Xi]^T  (32 x 9n)^T,
// Yr = Ar Xr - Ai Xi = D[r][c] - D[n + r][16 + c],   Yi = Ar Xi + Ai Xr = D[r][16 + c] + D[n + r][c].
// One tcgen05.mma (kind::f16, M = 128, N = 32, K = 16, FP32 accumulation in tensor memory) per
// 16 columns of 9n; operands are FP16 in shared memory in the K-major, no-swizzle canonical layout
// (8-row x 16-byte core matrices; the core matrices of one row group follow each other along K,
// 128 bytes apart; row groups are 9n/8 core matrices apart).  A is stored per site in exactly that
// layout (scaled by the site's max |Re|, |Im|), so it is copied verbatim; X is gathered and scaled
// per right-hand side.  One CTA of 4 warps per (site, chunk): warp 0 owns the TMEM allocation, thread
// 0 issues the MMAs and commits them to an mbarrier, every warp reads its 32 TMEM lanes back.  All
// mbarrier waits are bounded; on expiry the kernel records an error, waits once more (bounded) for
// the MMAs it issued, frees its TMEM and returns.
#include <cuda_fp16.h>

#include "kernels.h"

namespace wmg {

namespace {

constexpr int kTcRhs = 16;        // right-hand sides per chunk
constexpr int kTcN = 2 * kTcRhs;  // MMA N (Xr, Xi columns)
constexpr int kTcM = 128;         // MMA M (rows 2n padded)
constexpr int kTcCols = 32;       // TMEM columns (FP32 accumulator N = 32)
constexpr long long kSpinLimit = 1LL << 22;

__device__ int g_tc05_error = 0;

WMG_D uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle
WMG_D uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for sm_100-class parts
  // base offset 0, lbo mode 0, layout type 0 (no swizzle)
  return d;
}

// instruction descriptor, kind::f16: FP16 A and B (K-major), FP32 accumulator, M = 128, N = 32
constexpr uint32_t kIdesc = (1u << 4)                      // D format F32
                            | (0u << 7) | (0u << 10)       // A, B format F16
                            | ((uint32_t)(kTcN >> 3) << 17) // N >> 3
                            | ((uint32_t)(kTcM >> 4) << 24);// M >> 4

WMG_D bool mbar_wait(uint32_t bar, uint32_t phase) {
  for (long long i = 0; i < kSpinLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

}  // namespace

// FP16 copy of a stencil in the per-site canonical layout: [site][row group (2n/8)][k group (9n/8)]
// [8 rows][8 halves]; rows 0..n-1 Re, n..2n-1 Im of the n x 9n block matrix, scaled by 1/scale[v].
template <typename R>
__global__ void k_stencil_to_tc05(const cpx<R>* __restrict__ A, int n, const float* __restrict__ scale,
                                  __half* __restrict__ out, int Vc) {
  const int K = 9 * n, KG = K / 8, RG = 2 * n / 8;
  const size_t per_site = (size_t)RG * KG * 64;
  const size_t total = per_site * Vc;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (size_t)gridDim.x * blockDim.x) {
    const int h = (int)(idx % 8);
    size_t t = idx / 8;
    const int rr = (int)(t % 8);
    t /= 8;
    const int kg = (int)(t % KG);
    t /= KG;
    const int rg = (int)(t % RG);
    const int v = (int)(t / RG);
    const int row = rg * 8 + rr, k = kg * 8 + h;
    const int plane = row >= n, r = row - plane * n;
    const cpx<R> a = A[(((size_t)v * 9 + k / n) * n + (k % n)) * n + r];
    out[idx] = __float2half_rn((float)(plane ? a.im : a.re) / scale[v]);
  }
}

__global__ void __launch_bounds__(128) k_coarse_apply_tc05(const uint4* __restrict__ A16, const float* __restrict__ sA,
                                                           Geom g, int n, const cf* __restrict__ in,
                                                           cf* __restrict__ out, int nrhs,
                                                           const double* __restrict__ shift, int dagger,
                                                           const int* __restrict__ active, RedBuf rb, int want_norm,
                                                           int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  const int K = 9 * n, KG = K / 8;
  const uint32_t SBO = (uint32_t)KG * 128;  // bytes between row groups
  unsigned char* As = smraw;                                   // 16 row groups
  unsigned char* Bs = As + (size_t)(kTcM / 8) * SBO;           // 4 row groups
  float* Ds = reinterpret_cast<float*>(Bs + (size_t)(kTcN / 8) * SBO);  // [128][33]
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int nbs[9];
  __shared__ float xmax[kTcRhs];
  const int v = blockIdx.x, r0 = blockIdx.y * kTcRhs;
  const int N = n / 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  if (threadIdx.x < 9) {
    int c[4];
    site_coords(g, v, c);
    const int k = threadIdx.x;
    nbs[k] = k == 0 ? v : neighbour(g, v, c, (k - 1) >> 1, ((k - 1) & 1) ? -1 : +1);
  }
  // A: rows 0..2n-1 copied verbatim, the padding row groups zeroed
  {
    const size_t words = (size_t)(2 * n / 8) * SBO / 16;
    const uint4* src = A16 + (size_t)v * words;
    uint4* dst = reinterpret_cast<uint4*>(As);
    for (size_t i = threadIdx.x; i < words; i += blockDim.x) dst[i] = __ldg(src + i);
    const size_t total = (size_t)(kTcM / 8) * SBO / 16;
    for (size_t i = words + threadIdx.x; i < total; i += blockDim.x) dst[i] = make_uint4(0, 0, 0, 0);
  }
  __syncthreads();
  // B: one warp per right-hand side, [Xr | Xi] rows, scaled by the rhs's max |Re|, |Im|
  for (int rr = warp; rr < kTcRhs; rr += 4) {
    const int r = r0 + rr;
    float m = 0.f;
    const cf* src = in + (size_t)(r < nrhs ? r : 0) * g.V * n;
    for (int e = lane; e < K; e += 32) {
      if (r >= nrhs) break;
      const int k = e / n, j = e - k * n;
      const cf x = src[(size_t)nbs[k] * n + j];
      m = fmaxf(m, fmaxf(fabsf(x.re), fabsf(x.im)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) xmax[rr] = m;
    const float inv = m > 0.f ? 1.f / m : 0.f;
    for (int e = lane; e < K; e += 32) {
      const int k = e / n, j = e - k * n;
      float xr = 0.f, xi = 0.f;
      if (r < nrhs) {
        const cf x = src[(size_t)nbs[k] * n + j];
        const float sg = (dagger && j >= N) ? -inv : inv;
        xr = x.re * sg;
        xi = x.im * sg;
      }
      // element (row c, k = e) of B at (c/8)*SBO + (e/8)*128 + (c%8)*16 + (e%8)*2
      const int cr = rr, ci = kTcRhs + rr;
      __half* br = reinterpret_cast<__half*>(Bs + (size_t)(cr >> 3) * SBO + (size_t)(e >> 3) * 128 + (cr & 7) * 16) + (e & 7);
      __half* bi = reinterpret_cast<__half*>(Bs + (size_t)(ci >> 3) * SBO + (size_t)(e >> 3) * 128 + (ci & 7) * 16) + (e & 7);
      *br = __float2half_rn(xr);
      *bi = __float2half_rn(xi);
    }
  }
  // generic-proxy shared-memory writes must be visible to the tensor core (async proxy)
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base;
  if (threadIdx.x == 0) {
    const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
    for (int kk = 0; kk < K / 16; ++kk) {
      const uint64_t da = make_desc(a0 + kk * 256, 128, SBO);
      const uint64_t db = make_desc(b0 + kk * 256, 128, SBO);
      const uint32_t acc = kk > 0 ? 1u : 0u;
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
          "l"(da), "l"(db), "r"(kIdesc), "r"(acc));
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
        smem_u32(&mbar)));
  }
  bool ok = mbar_wait(smem_u32(&mbar), 0);
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err ? err : &g_tc05_error, 1);
    mbar_wait(smem_u32(&mbar), 0);  // give the issued MMAs a second bounded chance to drain
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  // TMEM -> registers: warp w reads lanes 32w..32w+31 (rows), 32 FP32 columns
  uint32_t d[32];
  if (ok) {
    const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(d[0]), "=r"(d[1]), "=r"(d[2]), "=r"(d[3]), "=r"(d[4]), "=r"(d[5]), "=r"(d[6]), "=r"(d[7]),
          "=r"(d[8]), "=r"(d[9]), "=r"(d[10]), "=r"(d[11]), "=r"(d[12]), "=r"(d[13]), "=r"(d[14]), "=r"(d[15]),
          "=r"(d[16]), "=r"(d[17]), "=r"(d[18]), "=r"(d[19]), "=r"(d[20]), "=r"(d[21]), "=r"(d[22]), "=r"(d[23]),
          "=r"(d[24]), "=r"(d[25]), "=r"(d[26]), "=r"(d[27]), "=r"(d[28]), "=r"(d[29]), "=r"(d[30]), "=r"(d[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
  } else {
#pragma unroll
    for (int i = 0; i < 32; ++i) d[i] = 0u;
  }
  const int row = threadIdx.x;
#pragma unroll
  for (int i = 0; i < 32; ++i) Ds[row * 33 + i] = __uint_as_float(d[i]);
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTcCols));
  // epilogue: thread -> (row, rhs) pairs
  double vals[kTcRhs];
#pragma unroll
  for (int rr = 0; rr < kTcRhs; ++rr) vals[rr] = 0.0;
  const float s_a = sA[v];
  for (int i = threadIdx.x; i < n * kTcRhs; i += blockDim.x) {
    const int rw = i % n, rr = i / n, r = r0 + rr;
    if (r >= nrhs || !ok) continue;
    const float yr = Ds[rw * 33 + rr] - Ds[(n + rw) * 33 + kTcRhs + rr];
    const float yi = Ds[rw * 33 + kTcRhs + rr] + Ds[(n + rw) * 33 + rr];
    const float sc = s_a * xmax[rr] * ((dagger && rw >= N) ? -1.f : 1.f);
    cf o{yr * sc, yi * sc};
    if (shift) o += (float)shift[r] * in[((size_t)r * g.V + v) * n + rw];
    if (!active || active[r]) out[((size_t)r * g.V + v) * n + rw] = o;
#pragma unroll
    for (int q = 0; q < kTcRhs; ++q)
      if (q == rr) vals[q] += double(o.re) * o.re + double(o.im) * o.im;
  }
  if (want_norm) {
    // |out|^2 per rhs, then the fixed-order grid reduction
    __shared__ double sm[32 * kTcRhs];
    cta_reduce<kTcRhs>(vals, sm);
    __shared__ bool last;
    const int nblk = gridDim.x;
    if (threadIdx.x == 0) {
      for (int rr = 0; rr < kTcRhs; ++rr)
        if (r0 + rr < nrhs) rb.partial[(size_t)(r0 + rr) * nblk + blockIdx.x] = vals[rr];
      __threadfence();
      last = atomicAdd(rb.counter + blockIdx.y, 1u) == (unsigned)nblk - 1;
    }
    __syncthreads();
    if (last) {
      __threadfence();
      const int nvals = min(kTcRhs, nrhs - r0);
      cta_multi_sum(rb.partial + (size_t)r0 * nblk, nvals, (size_t)nblk, nblk, 1,
                    [&](int i, double s) { rb.result[r0 + i] = s; });
      if (threadIdx.x == 0) rb.counter[blockIdx.y] = 0u;
    }
  }
}

size_t stencil_tc05_halves(int Vc, int n) { return (size_t)Vc * (2 * n / 8) * (9 * n / 8) * 64; }

void stencil_to_tc05(int prec, const void* A, int Vc, int n, const float* scale, void* out, cudaStream_t s) {
  count_launch();
  const size_t tot = stencil_tc05_halves(Vc, n);
  int B = (int)((tot + 255) / 256);
  if (B > 148 * 32) B = 148 * 32;
  if (prec == WMG_PREC_DOUBLE) k_stencil_to_tc05<double><<<B, 256, 0, s>>>((const cd*)A, n, scale, (__half*)out, Vc);
  else k_stencil_to_tc05<float><<<B, 256, 0, s>>>((const cf*)A, n, scale, (__half*)out, Vc);
}

bool coarse_tc05_supported(int n) { return n == 48 || n == 64 || n == 32 || n == 16; }

void coarse_apply_tc05(const void* A16, const float* sA, const Geom& g, int n, const void* in, void* out, int nrhs,
                       const double* shift, bool dagger, const int* active, const RedBuf* rb, cudaStream_t s,
                       int* err) {
  count_launch();
  const size_t SBO = (size_t)(9 * n / 8) * 128;
  const size_t smem = (size_t)(kTcM / 8) * SBO + (size_t)(kTcN / 8) * SBO + (size_t)kTcM * 33 * sizeof(float) + 1024;
  static const bool attr = [] {
    cudaFuncSetAttribute(k_coarse_apply_tc05, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    return true;
  }();
  (void)attr;
  dim3 grid(g.V, (nrhs + kTcRhs - 1) / kTcRhs);
  RedBuf r = rb ? *rb : RedBuf{nullptr, nullptr, nullptr};
  k_coarse_apply_tc05<<<grid, 128, smem, s>>>((const uint4*)A16, sA, g, n, (const cf*)in, (cf*)out, nrhs, shift,
                                              dagger ? 1 : 0, active, r, rb ? 1 : 0, err);
}

int coarse_tc05_error() {
  int e = 0;
  cudaMemcpyFromSymbol(&e, g_tc05_error, sizeof(int));
  return e;
}

}  // namespace wmg
