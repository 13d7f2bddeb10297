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
                                                      const int* __restrict__ active, RedBuf rb, int want_norm,
                                                      StencilEo eo) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<R>* xs = reinterpret_cast<cpx<R>*>(smraw);          // [9 n][NR]
  cpx<R>* red = xs + (size_t)9 * n * NR;                   // [KS][n][NR]
  const int v = eo.parity < 0 ? (int)blockIdx.x : parity_site(g, blockIdx.x, eo.parity);
  const int r0 = blockIdx.y * NR;
  const int N = n / 2;
  const cpx<R>* A = reinterpret_cast<const cpx<R>*>(A_) + (size_t)v * 9 * n * n;
  const cpx<R>* in = reinterpret_cast<const cpx<R>*>(in_);
  const cpx<R>* hin = eo.hop_in ? reinterpret_cast<const cpx<R>*>(eo.hop_in) : in;
  const cpx<R>* add = reinterpret_cast<const cpx<R>*>(eo.add);
  cpx<R>* out = reinterpret_cast<cpx<R>*>(out_);
  __shared__ int nbs[9];
  if (threadIdx.x < 9) {
    int c[4];
    site_coords(g, v, c);
    nbs[threadIdx.x] = stencil_neighbour(g, v, c, threadIdx.x);
  }
  __syncthreads();
  for (int k = 0; k < 9; ++k) {
    const cpx<R>* src = k == 0 ? in : hin;
    const bool skip = k == 0 && eo.hop_only;
    for (int i = threadIdx.x; i < n * NR; i += blockDim.x) {
      const int j = i / NR, rr = i % NR, r = r0 + rr;
      cpx<R> x{R(0), R(0)};
      if (r < nrhs && !skip) {
        x = src[((size_t)r * g.V + nbs[k]) * n + j];
        if (dagger && j >= N) x = -x;
      }
      xs[(size_t)(k * n + j) * NR + rr] = x;
    }
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
      if (shift && !eo.hop_only) o += R(shift[r]) * in[((size_t)r * g.V + v) * n + row];
      if (add) o += add[((size_t)r * g.V + v) * n + row];
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
                                const double* shift, bool dagger, const int* active, const RedBuf* rb, cudaStream_t s,
                                const StencilEo& eo) {
  const int T = ((n * kCoarseKS + 31) / 32) * 32;
  const size_t smem = ((size_t)9 * n * NR + (size_t)kCoarseKS * n * NR) * sizeof(cpx<R>);
  static const bool attr = [] {
    cudaFuncSetAttribute(k_coarse_apply<R, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    return true;
  }();
  (void)attr;
  dim3 grid(eo.parity < 0 ? g.V : g.V / 2, (nrhs + NR - 1) / NR);
  RedBuf r = rb ? *rb : RedBuf{nullptr, nullptr, nullptr};
  k_coarse_apply<R, NR><<<grid, T, smem, s>>>(A, g, n, in, out, nrhs, shift, dagger ? 1 : 0, active, r, rb ? 1 : 0,
                                              eo);
}

void coarse_apply(int prec, const void* A, const Geom& g, int n, const void* in, void* out, int nrhs,
                  const double* shift, bool dagger, const int* active, const RedBuf* rb, cudaStream_t s,
                  const StencilEo* eo_opt) {
  count_launch();
  const StencilEo eo = eo_opt ? *eo_opt : StencilEo{};
  if (prec == WMG_PREC_DOUBLE) {
    if (nrhs == 1) launch_coarse_apply<double, 1>(A, g, n, in, out, nrhs, shift, dagger, active, rb, s, eo);
    else if (nrhs <= 4) launch_coarse_apply<double, 4>(A, g, n, in, out, nrhs, shift, dagger, active, rb, s, eo);
    else launch_coarse_apply<double, 8>(A, g, n, in, out, nrhs, shift, dagger, active, rb, s, eo);
  } else {
    if (nrhs == 1) launch_coarse_apply<float, 1>(A, g, n, in, out, nrhs, shift, dagger, active, rb, s, eo);
    else if (nrhs <= 4) launch_coarse_apply<float, 4>(A, g, n, in, out, nrhs, shift, dagger, active, rb, s, eo);
    else if (nrhs <= 8) launch_coarse_apply<float, 8>(A, g, n, in, out, nrhs, shift, dagger, active, rb, s, eo);
    else launch_coarse_apply<float, 12>(A, g, n, in, out, nrhs, shift, dagger, active, rb, s, eo);
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

// Fused Galerkin construction on the fine level, as per-block complex GEMMs.  For coarse site
// xc and stencil slot q (0 = self, 1 + 2 mu + sg = the block across the face of direction mu,
// sg = 0 forward / 1 backward):
//     A_q[(s', alpha')][(s, a)] = sum_{x, k in s'} conj(P_alpha'(x)[k]) T_q,(s,a)(x)[k]
// where T_0 = (4 + m) g + the hops of D g that stay in the block and T_q (q > 0) is the hop of
// D g from across face q, g = P_a restricted to chirality s (every block).  One CTA of 256
// threads per coarse site takes the slots in turn and the contributing sites (all block sites
// for the self slot, the face sites for a face slot) in chunks of kGc sites: thread (j, a)
// stages P_a(x_j) (both chiralities) in shared memory as the GEMM's row operand and computes the
// 2N term columns (s, a) of its site; then thread (s', ta, tj) accumulates rows (s', ta + 8 i)
// x columns tj + 16 i over the chunk's components of chirality s'.  Fixed summation order; the
// CTA writes the 9 blocks [site][9][col][row].
constexpr int kGc = 8;           // sites per chunk
constexpr int kGThreads = 256;
template <typename R, int RT>    // RT = ceil(N / 8): rows (and columns) per thread
__global__ void __launch_bounds__(kGThreads, sizeof(R) == 4 ? 2 : 1) k_galerkin_fine(const void* __restrict__ gauge, const void* __restrict__ P,
                                                             Blocking bk, R diag, void* __restrict__ Aout) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int N = bk.N, n = 2 * N, xc = blockIdx.x;
  const int PW = N + 1, MW = n + 1;  // padded row widths (complex)
  cpx<R>* Ps = reinterpret_cast<cpx<R>*>(smraw);    // [kGc * 12][PW]: P_alpha(x_j)[k]
  cpx<R>* Ms = Ps + (size_t)kGc * 12 * PW;          // [kGc * 12][MW]: T column (s, a) at (x_j, k)
  const Geom& g = bk.fine;
  const size_t fb = spinor_field_bytes<R>(g.V);
  const int t = threadIdx.x;
  // producer role: site j of the chunk, vector a
  const int pj = t / N, pa = t % N;
  const bool producer = t < kGc * N;
  // GEMM role: row chirality ts, rows ta + 8 i, columns tj + 16 i
  const int tj = t & 15, ta = (t >> 4) & 7, ts = t >> 7;
  int cc[4];
  site_coords(bk.coarse, xc, cc);
  for (int q = 0; q < 9; ++q) {
    const int mu = (q - 1) >> 1, sg = (q - 1) & 1;
    // sites of this slot: all bs block sites (self) or the bs / b_mu on face q
    const int nsite = q == 0 ? bk.bs : bk.bs / bk.b[mu];
    cpx<R> acc[RT][RT];
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
      for (int k = 0; k < RT; ++k) acc[i][k] = cpx<R>{R(0), R(0)};
    for (int j0 = 0; j0 < nsite; j0 += kGc) {
      if (producer) {
        const int j = j0 + pj;
        cpx<R>* prow = Ps + (size_t)(pj * 12) * PW + pa;       // column a of the chunk's P rows
        cpx<R>* m0 = Ms + (size_t)(pj * 12) * MW + pa;         // term column (s = 0, a)
        cpx<R>* m1 = m0 + N;                                   // term column (s = 1, a)
        if (j < nsite) {
          // block offsets of site j of this slot's list
          int o[4];
          if (q == 0) {
            int e = j;
            o[0] = e % bk.b[0];
            e /= bk.b[0];
            o[1] = e % bk.b[1];
            e /= bk.b[1];
            o[2] = e % bk.b[2];
            o[3] = e / bk.b[2];
          } else {
            int e = j;
#pragma unroll
            for (int d = 0; d < 4; ++d) {
              if (d == mu) {
                o[d] = sg == 0 ? bk.b[d] - 1 : 0;
              } else {
                o[d] = e % bk.b[d];
                e /= bk.b[d];
              }
            }
          }
          int f[4];
#pragma unroll
          for (int d = 0; d < 4; ++d) f[d] = cc[d] * bk.b[d] + o[d];
          const int v = site_index(g, f);
          const char* Pa = (const char*)P + fb * pa;
          {
            cpx<R> self[12];
            load_spinor<R>(Pa, g.V, v, self);
#pragma unroll
            for (int k = 0; k < 12; ++k) {
              prow[(size_t)k * PW] = self[k];
              const bool up = k < 6;
              m0[(size_t)k * MW] = (q == 0 && up) ? diag * self[k] : cpx<R>{R(0), R(0)};
              m1[(size_t)k * MW] = (q == 0 && !up) ? diag * self[k] : cpx<R>{R(0), R(0)};
            }
          }
#pragma unroll
          for (int m2 = 0; m2 < 4; ++m2)
#pragma unroll
            for (int s2 = 0; s2 < 2; ++s2) {
              const int sign = s2 ? -1 : +1;
              const bool inb = same_block(f[m2], g.L[m2], bk.b[m2], sign);
              // self slot: the in-block hops; face slot q: its own hop when it leaves the block
              const bool take = q == 0 ? inb : (m2 == mu && s2 == sg && !inb);
              if (!take) continue;
              const int nb = neighbour(g, v, f, m2, sign);
              cpx<R> u[9], x[12];
              load_spinor<R>(Pa, g.V, nb, x);
#pragma unroll
              for (int k = 0; k < 12; ++k) x[k] = R(-0.5) * x[k];
              if (s2 == 0) load_link<R>(gauge, g.V, m2, v, u);
              else load_link<R>(gauge, g.V, m2, nb, u);
#pragma unroll
              for (int sc = 0; sc < 2; ++sc) {  // the hop of the chirality-sc part of P_a
                cpx<R> h[12], t[12];
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                  h[k] = ((k < 6) == (sc == 0)) ? x[k] : cpx<R>{R(0), R(0)};
                  t[k] = cpx<R>{R(0), R(0)};
                }
                if (s2 == 0) hop_accumulate<+1>(m2, u, h, t);
                else hop_accumulate<-1>(m2, u, h, t);
                cpx<R>* mc = sc == 0 ? m0 : m1;
#pragma unroll
                for (int k = 0; k < 12; ++k) mc[(size_t)k * MW] += t[k];
              }
            }
        } else {
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            prow[(size_t)k * PW] = cpx<R>{R(0), R(0)};
            m0[(size_t)k * MW] = m1[(size_t)k * MW] = cpx<R>{R(0), R(0)};
          }
        }
      }
      __syncthreads();
      // GEMM: rows (ts, ta + 8 i), columns tj + 16 i, over the chunk's components of chirality ts
      const int jn = min(kGc, nsite - j0);
      for (int j = 0; j < jn; ++j)
#pragma unroll 2
        for (int kk = 0; kk < 6; ++kk) {
          const int k = j * 12 + 6 * ts + kk;
          cpx<R> pv[RT], mv[RT];
#pragma unroll
          for (int i = 0; i < RT; ++i) {
            const int al = ta + 8 * i, col = tj + 16 * i;
            pv[i] = al < N ? Ps[(size_t)k * PW + al] : cpx<R>{R(0), R(0)};
            mv[i] = col < n ? Ms[(size_t)k * MW + col] : cpx<R>{R(0), R(0)};
          }
#pragma unroll
          for (int i = 0; i < RT; ++i)
#pragma unroll
            for (int i2 = 0; i2 < RT; ++i2) cfmac(acc[i][i2], pv[i], mv[i2]);
        }
      __syncthreads();
    }
    cpx<R>* A = reinterpret_cast<cpx<R>*>(Aout);
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
      for (int i2 = 0; i2 < RT; ++i2) {
        const int al = ta + 8 * i, col = tj + 16 * i2;
        if (al < N && col < n) A[(((size_t)xc * 9 + q) * n + col) * n + ts * N + al] = acc[i][i2];
      }
  }
}

template <typename R, int RT>
static void launch_galerkin_fine(const void* gauge, const void* P, const Blocking& bk, R diag, void* A, cudaStream_t s) {
  const size_t smem = (size_t)kGc * 12 * ((bk.N + 1) + (2 * bk.N + 1)) * sizeof(cpx<R>);
  static const cudaError_t attr =
      cudaFuncSetAttribute(k_galerkin_fine<R, RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  (void)attr;
  k_galerkin_fine<R, RT><<<bk.coarse.V, kGThreads, smem, s>>>(gauge, P, bk, diag, A);
}

template <typename R>
static void galerkin_fine_rt(const void* gauge, const void* P, const Blocking& bk, R diag, void* A, cudaStream_t s) {
  const int rt = (bk.N + 7) / 8;
  if (rt <= 1) launch_galerkin_fine<R, 1>(gauge, P, bk, diag, A, s);
  else if (rt == 2) launch_galerkin_fine<R, 2>(gauge, P, bk, diag, A, s);
  else if (rt == 3) launch_galerkin_fine<R, 3>(gauge, P, bk, diag, A, s);
  else launch_galerkin_fine<R, 4>(gauge, P, bk, diag, A, s);
}

bool galerkin_fine_fused(int prec, const void* gauge, const void* P, const Blocking& bk, double mass, void* A,
                         cudaStream_t s) {
  if (bk.N > 32 || kGc * bk.N > kGThreads) return false;
  count_launch();
  if (prec == WMG_PREC_DOUBLE) galerkin_fine_rt<double>(gauge, P, bk, 4.0 + mass, A, s);
  else galerkin_fine_rt<float>(gauge, P, bk, float(4.0 + mass), A, s);
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
