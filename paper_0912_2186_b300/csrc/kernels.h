// Internal launch interface of the libwmg kernels (host side, not part of the C ABI).
#pragma once
#include "wmg_common.cuh"

namespace wmg {

constexpr int kDslashThreads = 128;
// whether the coarsest CG's kernels are launched with programmatic stream serialisation (each may
// start while its predecessor finishes): inside pdl_scope(true) ... pdl_scope(false) only, and not
// with WMG_PDL=0
bool pdl_launches();
void pdl_scope(bool on);
constexpr int kBlasThreads = 256;
constexpr int kMaxRhs = 64;          // right-hand sides per batched launch
constexpr int kMaxKrylov = 32;       // outer GCR restart length limit

inline size_t prec_real_bytes(int prec) { return prec == WMG_PREC_DOUBLE ? 8 : 4; }

// number of kernel launches issued by this library (all contexts)
long long launch_count();
long long graph_launch_count();  // kernels launched inside device-side graph loops (synchronises)
void count_launch(int n = 1);

// N(0,1) reals from the counter-based generator (rng.cu): out[i] depends only on (seed, i)
void gaussian_fill(double* out, size_t n, uint64_t seed, size_t first, cudaStream_t s);  // first % 4 == 0

// ---- fine lattice (dslash.cu) ----
void pack_gauge(int prec, const double* canon, void* out, int V, cudaStream_t s);
void pack_spinor(int prec, const double* canon, void* out, int V, int nrhs, cudaStream_t s);
void unpack_spinor(int prec, const void* in, double* canon, int V, int nrhs, cudaStream_t s);
int dslash_blocks(int V);
// out = D in, or out = b - D in when b != nullptr.  mass_dev[nrhs]: per-rhs Wilson mass.
// red = 0: none; 1: |out|^2 per rhs into rb->result[rhs]; 2: {Re, Im <out,in>, |out|^2}.
// gc = 8 / 18: FP32 only, `gauge` holds 8-real (pack_gauge8) or 18-real (pack_gauge18) links.
// b_half = 1: b holds the even sites only, as half-lattice fields (zero on the odd sites).
void dslash(int prec, void* out, const void* in, const void* b, const void* gauge, const Geom& g,
            const double* mass_dev, const int* active, int nrhs, int red, const RedBuf* rb, cudaStream_t s,
            int gc = 12, int b_half = 0);
// one MR step with the previous update fused in: r_out = r - alpha q, x += alpha r, out = D r_out
// with the sums {Re, Im <out, r_out>, |out|^2} per rhs into rb (alpha from red_prev[3 r ..]);
// out and r_out must not alias r, q; rb.result must not alias red_prev
void dslash_mr(int prec, void* out, const void* r, const void* q, void* r_out, void* x, const double* red_prev,
               const void* gauge, const Geom& g, const double* mass_dev, const int* active, int nrhs,
               const RedBuf& rb, cudaStream_t s, int gc = 12);
// 8-real FP32 links from the native FP64 12-real links; *degenerate (device int) set to 1 if a
// link has |U_01|^2 + |U_02|^2 < 1e-6 (the 8-real form cannot represent it accurately)
void pack_gauge8(const void* g64, void* out, int V, int* degenerate, cudaStream_t s);
void pack_gauge18(const void* g64, void* out, int V, cudaStream_t s);
// the smoother's FP16 storage (per-site norms, FP32 arithmetic): out16 = [b -] D in with in
// FP32 native (in16 = 0) or FP16 (in16 = 1); red = 2 adds per-rhs {<out, in>, |out|^2}
void dslash_h(int in16, void* out16, float* out_norm, const void* in, const float* in_norm, const void* b,
              const void* gauge, const Geom& g, const double* mass_dev, const int* active, int nrhs, int red,
              const RedBuf* rb, cudaStream_t s, int gc = 12);
// x += alpha r, r -= alpha q (update_r) with x FP32 native and r, q FP16
void mr_update_h(void* x, void* r16, float* rn, const void* q16, const float* qn, int V, int nrhs, const double* red,
                 const int* active, bool update_r, cudaStream_t s);
void spinor_to_h(const void* in, void* out16, float* norm, int V, int nrhs, cudaStream_t s);
void spinor_from_h(const void* in16, const float* norm, void* out, int V, int nrhs, cudaStream_t s);

// ---- even-odd fine operator (dslash_eo.cu): half-lattice fields [rhs][6][V/2], site v at v >> 1 ----
// h = the raw hop sum onto the parity-p_out sites from the opposite-parity half field `in` (H = -h/2);
// mode 0: out = h;  1: out = d self - h / (4 d);  2: out = self + h / (2 d);  3: out = (self + h / 2) / d,
// d = 4 + m_r; with b: out = b - out; with rb: |out|^2 per rhs.  gc = 8 / 18: 8- or 18-real FP32 links.
void dslash_eo(int prec, int mode, int p_out, void* out, const void* in, const void* self, const void* b,
               const void* gauge, int gc, const Geom& g, const double* mass_dev, const int* active, int nrhs,
               const RedBuf* rb, cudaStream_t s);
int dslash_eo_blocks(int V);
// whole-lattice native field <- even sites from half_e, odd sites from half_o (zeros for a null
// one); and the half field of parity p from a whole-lattice one
// the residuals r_1 .. r_n of the MR steps whose solution updates are deferred (n <= kMrMaxSteps)
constexpr int kMrMaxSteps = 5;
struct MrSteps {
  const void* p[kMrMaxSteps];
  int n;
};
// out_e = x_e + sum_i alpha_i r_i at the even sites as half-lattice fields (alpha_i =
// red0[i * rstride + 3 r ..] per rhs, the sums {Re, Im <q_i, r_i>, |q_i|^2}; x, r_i whole-lattice)
void mr_combine_even(int prec, const void* x, const MrSteps& rs, void* out_half, const Geom& g, int nrhs,
                     const double* red0, int rstride, const int* active, cudaStream_t s);
// r_out = r - alpha q, alpha = red[0..1] / red[2] per rhs (r_out may not alias r or q)
void blas_mr_rnext(int prec, void* r_out, const void* r, const void* q, size_t n, int nrhs, const double* red,
                   const int* active, cudaStream_t s);
// out_e = x_e + alpha r_e at the even sites as half-lattice fields (alpha = red[0..1] / red[2] per
// rhs; x, r whole-lattice native fields): the last MR step of the red/black solve's cycle
void mr_update_even(int prec, const void* x, const void* r, void* out_half, const Geom& g, int nrhs,
                    const double* red, const int* active, cudaStream_t s);
void eo_embed(int prec, void* full, const void* half_e, const void* half_o, const Geom& g, int nrhs, cudaStream_t s);
void eo_extract(int prec, void* half, const void* full, const Geom& g, int p, int nrhs, cudaStream_t s);

// ---- BLAS on flat complex vectors: n complex numbers per rhs, rhs stride n (blas.cu) ----
int blas_blocks(size_t n);
void blas_zero(int prec, void* x, size_t n, int nrhs, cudaStream_t s);
// dst (prec_d) = src (prec_s) for rhs with mask==nullptr or mask[r] != 0
void blas_convert(int prec_d, void* dst, int prec_s, const void* src, size_t n, int nrhs, const int* mask,
                  cudaStream_t s);
// result[r] = {Re <a,b>, Im <a,b>, |a|^2}
void blas_dot_norm(int prec, const void* a, const void* b, size_t n, int nrhs, const RedBuf& rb, cudaStream_t s);
// result[r] = {|a|^2}
void blas_norm2(int prec, const void* a, size_t n, int nrhs, const RedBuf& rb, cudaStream_t s);
// x[r] *= scale[r] (scale double, per rhs; skip where scale pointer entry is not finite)
void blas_scale_inv_sqrt(int prec, void* x, size_t n, int nrhs, const double* norm2, int stride, cudaStream_t s);
// y = gamma_5 x for native fine spinors (n = 12 V complex per rhs; y may alias x)
void blas_gamma5(int prec, const void* x, void* y, size_t n, int nrhs, cudaStream_t s);
// y = x - y  (y := x - y)
void blas_xmy(int prec, const void* x, void* y, size_t n, int nrhs, cudaStream_t s);
// y = x + y
void blas_xpy(int prec, const void* x, void* y, size_t n, int nrhs, cudaStream_t s);
// MR update: alpha = qr/qq from red[r*3 + {0,1,2}]; x += alpha r; r -= alpha q
void blas_mr_update(int prec, void* x, void* r, const void* q, size_t n, int nrhs, const double* red, bool update_r,
                    const int* active, cudaStream_t s);
// CG (normal equations) helpers, scalars per rhs in `cg` (see blas.cu)
struct CgScalars {
  double* zz;       // [2][nrhs]  |z|^2, double-buffered by iteration parity
  double* rr;       // [nrhs] (RedBuf result of the update kernel)
  double* qq;       // [nrhs]
  double* bb;       // [nrhs]
  int* done;        // [nrhs]
  int* iters;       // [nrhs]
  double tol2;
};
void cg_update(int prec, void* x, void* r, const void* p, const void* q, size_t n, int nrhs, const CgScalars& cg,
               int parity, const RedBuf& rb_rr, cudaStream_t s);
void cg_xpay(int prec, void* p, const void* z, size_t n, int nrhs, const CgScalars& cg, int parity, cudaStream_t s);
// GCR
// <W_j, w> for j < kmax (W_j at W + j*slot_stride), in chunks of kDotChunk: the value for (j, r)
// is at coef + ((j / kDotChunk) * nrhs + r) * 2 kDotChunk + 2 (j % kDotChunk) (re, im)
constexpr int kDotChunk = 8;
void gcr_multidot(int prec, const void* W, size_t slot_stride, int kmax, const void* w, size_t n, int nrhs,
                  const int* active, const RedBuf& rb, cudaStream_t s);
// w -= sum_j c_j W_j (and z -= sum_j c_j Z_j unless Z is null), then red = {|w|^2, Re<w,r>, Im<w,r>}
void gcr_orth(int prec, const void* W, const void* Z, size_t slot_stride, int k, void* w, void* z, const void* r,
              const double* coef, int kmax, size_t n, int nrhs, const int* active, const RedBuf& rb, cudaStream_t s);
// alpha = <w,r>/|w|^2, x += alpha z, r -= alpha w, w /= |w|, z /= |w|; red = |r|^2 (x sloppy)
void gcr_update(int prec, void* x, void* r, void* w, void* z, const double* wred, size_t n, int nrhs,
                const int* active, const RedBuf& rb, cudaStream_t s);
// alpha = <w,r>/|w|^2, r -= alpha w, w /= |w|; red = |r|^2 (solution update deferred)
void gcr_update_r(int prec, void* r, void* w, const double* wred, size_t n, int nrhs, const int* active,
                  const RedBuf& rb, cudaStream_t s);
// Deferred solution update of the flexible GCR: for each right-hand side r with ints[r] != 0,
// solve Gamma xi = alpha by back-substitution (Gamma upper triangular: gamma_q = |w_q| before
// normalisation on the diagonal, beta_jq = <W_j, w_q> above it; alpha_q = <W_q, r_q> for q >=
// ints[nslots + r], 0 below) from the per-iteration history hist + q hstride = {multidot
// coefficients as gcr_multidot writes them (kcoef doubles), then |w|^2, Re, Im <w, r> per rhs};
// xi: complex FP64, kMaxKrylov per rhs.  One warp per right-hand side.
void gcr_backsolve(const double* hist, size_t hstride, size_t kcoef, int K, int nslots, const int* ints, double* xi,
                   cudaStream_t s);
// x += sum_{j<K} xi[r][j] Z_j (xi complex FP64, kMaxKrylov per rhs) for masked right-hand sides
void gcr_xupdate(int prec, const void* Z, size_t slot_stride, int K, void* x, const double* xi, size_t n, int nrhs,
                 const int* mask, cudaStream_t s);
// reliable update of the solution: x64 += x, x = 0 for masked right-hand sides
void blas_fold(int prec, double* x64, void* x, size_t n, int nrhs, const int* mask, cudaStream_t s);

// ---- transfer (transfer.cu) ----
struct Blocking {
  Geom fine, coarse;
  int b[4];      // block extents
  int bs;        // sites per block
  int N;         // vectors
  int nf;        // complex dof per fine site (12 on the fine lattice, 2N' on a coarse one)
};
// fine level: fine spinors (native) <-> coarse vectors; P = N native fine fields.  half = 1 (N <= 64,
// even block x extent): `in` holds the even sites only as half-lattice fields (zero on the odd
// sites), and only the even sites' rows of P are read.
void restrict_fine(int prec, const void* P, const Blocking& bk, const void* in, void* out, int nrhs,
                   const int* active, cudaStream_t s, int half = 0);
void prolong_fine(int prec, const void* P, const Blocking& bk, const void* in, void* out, int nrhs,
                  const int* active, cudaStream_t s);
// FP32 vectors, FP16 null vectors (false: blocking not handled, use the FP32 copy)
bool restrict_fine_h(const void* P16, const Blocking& bk, const void* in, void* out, int nrhs, const int* active,
                     cudaStream_t s, int half = 0);
bool prolong_fine_h(const void* P16, const Blocking& bk, const void* in, void* out, int nrhs, const int* active,
                    cudaStream_t s);
void convert_to_half2(const void* src64, void* dst16, size_t n, cudaStream_t s);  // complex FP64 -> (re, im) FP16
// coarse level: coarse vectors [rhs][Vf][nf] <-> [rhs][Vc][2N]; P = N coarse fields
void restrict_coarse(int prec, const void* P, const Blocking& bk, const void* in, void* out, int nrhs,
                     const int* active, cudaStream_t s);
void prolong_coarse(int prec, const void* P, const Blocking& bk, const void* in, void* out, int nrhs,
                    const int* active, cudaStream_t s);
// block Gram-Schmidt (FP64, in place) on N vectors; fine: native FP64 fields, coarse: coarse
// FP64 fields.  rank_flag: device int set to 1 on rank deficiency.
void block_gs(bool fine_level, void* vecs, const Blocking& bk, int* rank_flag, cudaStream_t s);

// ---- coarse operator (coarse.cu) ----
// stencil layout [site][9][col][row] complex (col-major blocks), n = 2N rows
// Options of a stencil application for the even-odd form of the coarsest solve: with
// parity >= 0 only the sites of that parity are computed and written (grid over V / 2 sites,
// every extent even); hop_only leaves out the site's own block and the shift; hop_in supplies
// the neighbour values (slots 1..8) instead of `in`; add is added to the result.
// The tensor-core stencil also takes the odd-site block inverses (inv, inv_idx as for
// eo_inv_apply; parity 1 and hop_only): it then writes -M_r (its result) instead of the result.
// With opB (tensor-core stencil, parity 1, hop_only) the operator is not the level's but opB
// with scales sB, both indexed by the parity-site number: the precomputed odd-site pass
// B_k = -A_oo^-1 A_oe,k of one mass shift (eo_hop_inverse).
struct StencilEo {
  int parity = -1;
  int hop_only = 0;
  const void* hop_in = nullptr;
  const void* add = nullptr;
  const void* inv = nullptr;
  const int* inv_idx = nullptr;
  const void* opB = nullptr;
  const float* sB = nullptr;
};
// out = A in (+ shift[r] in), or sigma_3 A sigma_3 in for dagger; optional |out|^2 per rhs
void coarse_apply(int prec, const void* A, const Geom& g, int n, const void* in, void* out, int nrhs,
                  const double* shift, bool dagger, const int* active, const RedBuf* rb_norm, cudaStream_t s,
                  const StencilEo* eo = nullptr);
// A_oo^-1 for the even-odd coarsest solve (coarse_eo.cu): for table entries e0 + j, j < ne,
// inv[e0 + j][k] = (A[odd site k][0] + shifts[j] I)^-1, Gauss-Jordan with partial pivoting in
// precision prec (A in that precision), stored [e][k][col][row]; *singular set to 1 on a zero pivot.
void eo_invert(int prec, const void* A, const Geom& g, int n, const double* shifts, int e0, int ne, void* inv,
               int* singular, cudaStream_t s);
size_t eo_inverse_bytes(int prec, const Geom& g, int n);  // one table entry
// B[k][slot][col][row] = -(inv_entry[k]) A[odd site k][slot] for the hop slots 1..8 (FP32; A in
// the stencil layout, inv_entry one FP32 table entry of eo_invert)
void eo_hop_inverse(const void* A, const void* inv_entry, const Geom& g, int n, void* B, cudaStream_t s);
// out_o[r] = M_r (bc b_o[r] + hc h_o[r]) at the odd sites, M_r = inv[idx[r]] or, for dagger,
// sigma_3 inv[idx[r]] sigma_3; b or h may be null; out may alias h (not b)
void eo_inv_apply(int prec, const void* inv, const int* idx, const Geom& g, int n, const void* b, double bc,
                  const void* h, double hc, void* out, int nrhs, bool dagger, const int* active, cudaStream_t s,
                  int par = 1);  // par = 0: the same at the even sites with a table of even-site blocks
// right block-Jacobi preconditioning of the Schur complement (coarse_eo.cu): M = (S_xx)^-1 per even
// site for one shift, formed and inverted in FP32 (FP32 [even site][col][row]; A32 the FP32
// stencil, inv_entry the shift's FP32 odd-inverse table entry), and the FP32 tables of the preconditioned passes (stencil layout
// [parity site][9][col][row]): mode 0 B M(x + s) (odd sites, B from eo_hop_inverse), mode 1 the
// even pass of S M, mode 2 M times the even pass (for M S)
void eo_schur_self_inv(const void* A32, const void* inv_entry, const Geom& g, int n, double shift, void* M,
                       int* singular, cudaStream_t s);
void eo_bj_table(int mode, const void* A32, const void* B, const void* M, const Geom& g, int n, double shift,
                 void* out, cudaStream_t s);
// Galerkin build helpers: split the operator applied to column vectors into 9 slot fields
// fine level: g = column (s, alpha) of P, written for ncol columns starting at col0
void hop_split_fine(int prec, const void* gauge, const void* P, const Blocking& bk, double mass, int col0,
                    int ncol, void* out9, cudaStream_t s);
// fused fine-level Galerkin construction straight into the stencil (false if the blocking is
// not supported: more than 256 sites per block or an extent of 1)
bool galerkin_fine_fused(int prec, const void* gauge, const void* P, const Blocking& bk, double mass, void* A,
                         cudaStream_t s);
void hop_split_coarse(int prec, const void* A, const void* P, const Blocking& bk, int col0, int ncol, void* out9,
                      cudaStream_t s);
// scatter restricted slot fields [ncol][9][Vc][n] into the stencil at columns col0..
void stencil_scatter(int prec, const void* rs, void* A, int Vc, int n, int col0, int ncol, cudaStream_t s);
// tensor-core (FP16 mma.sync) copy of a stencil and its application (coarse_mma.cu)
size_t stencil_mma_words(int Vc, int n);  // uint4 words of the fragment-order copy
void stencil_to_mma(int prec, const void* A, int Vc, int n, float* scale, void* out, cudaStream_t s);
void coarse_apply_mma(const void* A16, const float* sA, const Geom& g, int n, const void* in, void* out, int nrhs,
                      const double* shift, bool dagger, const int* active, const RedBuf* rb, cudaStream_t s,
                      const StencilEo* eo = nullptr, int* err = nullptr);
// tcgen05 tensor-core copy of a stencil and its application (coarse_tc05.cu)
size_t stencil_tc05_halves(int Vc, int n);
bool coarse_tc05_supported(int n);
void stencil_to_tc05(int prec, const void* A, int Vc, int n, const float* scale, void* out, cudaStream_t s);
void coarse_apply_tc05(const void* A16, const float* sA, const Geom& g, int n, const void* in, void* out, int nrhs,
                       const double* shift, bool dagger, const int* active, const RedBuf* rb, cudaStream_t s,
                       int* err = nullptr);
// Coarsest CGNR for nrhs <= 16 as one persistent cooperative kernel (FP16 tensor-core stencil
// with 2N in {16, 32, 48, 64}, FP32 vectors [rhs][site][2N]); false if it cannot run (the caller
// then uses the multi-kernel CGNR).  r16, p16: cgnr_persistent_copy_bytes each (FP16 copies);
// rsc, psc: 16 floats per site; part: 4 * 16 * kPersistentMaxGrid doubles; bar: 2 unsigned;
// err: sticky error flag (bounded waits expired); done_out, iters_out: 16 ints.
constexpr int kPersistentMaxGrid = 1024;
size_t cgnr_persistent_copy_bytes(int Vc, int n);
bool cgnr_persistent(const void* A16, const float* sA, const Geom& g, int n, const double* shift, const void* b,
                     void* x, void* r, void* p, void* q, void* z, void* r16, void* p16, float* rsc, float* psc,
                     int nrhs, double tol2, int maxit, const int* active, double* part, unsigned* bar, int* err,
                     int* done_out, int* iters_out, cudaStream_t s);
// err (per context) is set to 1 when a bounded wait of a tensor-core stencil expires; without one
// (err = nullptr) the kernels set a process-wide flag read by these (synchronises)
int coarse_mma_error();
int coarse_tc05_error();
// convert a stencil between precisions
void stencil_convert(int prec_d, void* dst, int prec_s, const void* src, size_t count, cudaStream_t s);

}  // namespace wmg
