// Host-side driver of libwmg: the multigrid cycle with post-smoothing (Sec. 3), the MR
// smoother, CG on the normal equations on the coarsest level, flexible GCR on the fine level
// with FP64 reliable updates, the adaptive setup (Sec. 2) and the Galerkin construction
// D^ = P^dag D P (Sec. 2).  Every arithmetic step runs in the kernels of this library; the
// host only sequences launches and reads per-rhs residual norms.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <random>

#include "ctx.h"
#include "solver.h"

using namespace wmg;

namespace wmg {
static std::atomic<long long> g_launches{0};
long long launch_count() { return g_launches.load(); }
void count_launch(int n) { g_launches += n; }
// Programmatic launches are used only inside the coarsest CG's loop (pdl_scope), where the
// operator tables and masks that a pass reads before its griddep_wait are final.
static thread_local bool t_pdl_scope = false;
void pdl_scope(bool on) { t_pdl_scope = on; }
bool pdl_launches() {
  static const bool on = [] {
    const char* e = getenv("WMG_PDL");
    return !(e && e[0] == '0');
  }();
  return on && t_pdl_scope;
}
}  // namespace wmg

wmg_status wmg_cuda_fail(cudaError_t e, const char* what) {
  (void)what;
  return e == cudaErrorMemoryAllocation ? WMG_ENOMEM : WMG_ECUDA;
}

namespace wmg {

static size_t csize(int prec) { return prec == WMG_PREC_DOUBLE ? sizeof(cd) : sizeof(cf); }

wmg_status fail(wmg_ctx* c, cudaError_t e, const char* what) {
  c->err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? WMG_ENOMEM : WMG_ECUDA;
}

wmg_status check(wmg_ctx* c, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, e, what);
  return WMG_OK;
}

#define TRY(x)                              \
  do {                                      \
    wmg_status st_ = (x);                   \
    if (st_ != WMG_OK) return st_;          \
  } while (0)
#define CU(c, x)                                      \
  do {                                                \
    cudaError_t e_ = (x);                             \
    if (e_ != cudaSuccess) return fail((c), e_, #x);  \
  } while (0)

wmg_status clear_graphs(wmg_ctx* c);

wmg_status ws_get(wmg_ctx* c, const std::string& name, size_t bytes, void** out) {
  auto it = c->ws.find(name);
  if (it != c->ws.end() && it->second.second >= bytes) {
    *out = it->second.first;
    return WMG_OK;
  }
  if (it != c->ws.end()) {
    CU(c, cudaStreamSynchronize(c->stream));
    cudaFree(it->second.first);
    c->ws.erase(it);
    clear_graphs(c);  // captured graphs may refer to the old buffer
  }
  void* p = nullptr;
  CU(c, cudaMalloc(&p, bytes > 0 ? bytes : 16));
  c->ws[name] = {p, bytes};
  *out = p;
  return WMG_OK;
}

// vector workspace of level l: nrhs fields of V_l * ndof_l complex numbers
wmg_status vec_ws(wmg_ctx* c, int l, const char* tag, int prec, int nrhs, void** out) {
  const size_t n = c->L[l].nvec_elems();
  return ws_get(c, "v" + std::to_string(l) + tag + (prec == WMG_PREC_DOUBLE ? "d" : "s"), n * nrhs * csize(prec),
                out);
}

static double* res_slot(wmg_ctx* c, int slot) { return c->res + (size_t)slot * kMaxRhs * 16; }
enum { RES_MR = 0, RES_NORM, RES_WRED, RES_RN, RES_R64, RES_BB, RES_CGQQ, RES_CGRR, RES_CGBB, RES_CGZZ,
       RES_SETUP, RES_MR2, RES_COEF = 16, RES_SLOTS = 24 };

RedBuf redbuf(wmg_ctx* c, int slot) { return RedBuf{c->red_partial, c->red_counter, res_slot(c, slot)}; }

wmg_status ensure_partials(wmg_ctx* c, size_t need) {
  if (need <= c->red_partial_n) return WMG_OK;
  CU(c, cudaStreamSynchronize(c->stream));
  if (c->red_partial) cudaFree(c->red_partial);
  c->red_partial = nullptr;
  clear_graphs(c);
  CU(c, cudaMalloc(&c->red_partial, need * sizeof(double)));
  c->red_partial_n = need;
  return WMG_OK;
}

wmg_status ensure_reductions(wmg_ctx* c, int nrhs) {
  // dslash: nrhs * blocks * 3; blas: nrhs * 1184 * 16; coarse apply: nrhs * blocks
  size_t need = (size_t)nrhs * (size_t)dslash_blocks(c->fine.V) * 3;
  need = std::max(need, (size_t)nrhs * 148 * 8 * 16);
  for (int l = 1; l < c->nlev; ++l) need = std::max(need, (size_t)nrhs * (size_t)c->L[l].g.V);
  return ensure_partials(c, need);
}

// Small asynchronous host-to-device copy through the context's pinned ring (no host
// synchronisation; the slot is reused only once the copy that last read it has completed).
wmg_status ring_upload(wmg_ctx* c, void* dst, const void* src, size_t bytes) {
  if (bytes > kRingInts * sizeof(int)) {
    c->err = "internal: upload larger than a ring slot";
    return WMG_EINVAL;
  }
  const int k = c->ring_pos;
  c->ring_pos = (k + 1) % kRingSlots;
  CU(c, cudaEventSynchronize(c->ring_ev[k]));
  int* slot = c->h_ring + (size_t)k * kRingInts;
  std::memcpy(slot, src, bytes);
  CU(c, cudaMemcpyAsync(dst, slot, bytes, cudaMemcpyHostToDevice, c->stream));
  CU(c, cudaEventRecord(c->ring_ev[k], c->stream));
  return WMG_OK;
}

// Per-rhs Wilson masses (d_mass) and coarse diagonal shifts m_r - m_setup (d_shift[l]); a set
// equal to the one last uploaded is not uploaded again.
wmg_status set_rhs_scalars(wmg_ctx* c, const double* masses, int nrhs) {
  double m[kMaxRhs], sh[kMaxRhs];
  bool same = true;
  for (int r = 0; r < nrhs; ++r) {
    m[r] = masses ? masses[r] : c->mass;
    same = same && m[r] == c->mass_up[r];
  }
  if (!same) {
    TRY(ring_upload(c, c->d_mass, m, nrhs * sizeof(double)));
    for (int r = 0; r < nrhs; ++r) c->mass_up[r] = m[r];
  }
  for (int l = 1; l < c->nlev; ++l) {
    same = true;
    for (int r = 0; r < nrhs; ++r) {
      sh[r] = c->h_shift[r] = m[r] - c->mass_setup;
      same = same && sh[r] == c->shift_up[l][r];
    }
    if (!same) {
      TRY(ring_upload(c, c->d_shift[l], sh, nrhs * sizeof(double)));
      for (int r = 0; r < nrhs; ++r) c->shift_up[l][r] = sh[r];
    }
  }
  return WMG_OK;
}

wmg_status upload_ints(wmg_ctx* c, int* dst, const std::vector<int>& v) {
  return ring_upload(c, dst, v.data(), v.size() * sizeof(int));
}

wmg_status download(wmg_ctx* c, const double* src, size_t n, std::vector<double>& out) {
  CU(c, cudaMemcpyAsync(c->h_pin, src, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaStreamSynchronize(c->stream));
  out.assign(c->h_pin, c->h_pin + n);
  return WMG_OK;
}

// ------------------------------------------------------------------------------------
// optional CUDA-event instrumentation: every timed launch (or launch group) is bracketed by
// two events on the context's stream; elapsed times are collected at wmg_profile_get.
// ------------------------------------------------------------------------------------
static cudaEvent_t ev_get(wmg_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void prof_flush(wmg_ctx* c) {
  for (auto& r : c->prof_pending) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    c->prof_ms[r.cls] += ms;
    c->prof_bytes[r.cls] += r.bytes;
    c->prof_units[r.cls] += r.units;
    c->prof_n[r.cls] += 1;
    c->ev_pool.push_back(r.a);
    c->ev_pool.push_back(r.b);
  }
  c->prof_pending.clear();
}

struct ProfScope {
  wmg_ctx* c;
  int cls;
  double bytes, units;
  cudaEvent_t a = nullptr;
  ProfScope(wmg_ctx* c_, int cls_, double bytes_, double units_ = 0)
      : c(c_), cls(cls_), bytes(bytes_), units(units_) {
    if (c->prof_on) {
      a = ev_get(c);
      cudaEventRecord(a, c->stream);
    }
  }
  ~ProfScope() {
    if (!c->prof_on || !a) return;
    cudaEvent_t b = ev_get(c);
    cudaEventRecord(b, c->stream);
    c->prof_pending.push_back({a, b, cls, bytes, units});
    if (c->prof_pending.size() > 8192) prof_flush(c);
  }
};

// algorithmic (compulsory) bytes of one launch
static double rb_(int prec) { return prec == WMG_PREC_DOUBLE ? 8.0 : 4.0; }
double dslash_bytes(const wmg_ctx* c, int prec, int nact, bool resid) {
  const double s = rb_(prec), V = c->fine.V;
  int gc;
  links(c, prec, &gc);
  return V * (4.0 * gc * s) + (double)nact * V * 24.0 * s * (resid ? 3.0 : 2.0);
}
// the links of the fine operator in precision prec: 12-real, or the 8- or 18-real FP32 links
const void* links(const wmg_ctx* c, int prec, int* gc) {
  if (prec == WMG_PREC_SINGLE && c->gauge_compress == 8 && c->gauge8 && c->gauge8_ok) {
    *gc = 8;
    return c->gauge8;
  }
  if (prec == WMG_PREC_SINGLE && c->gauge_compress == 18 && c->gauge18) {
    *gc = 18;
    return c->gauge18;
  }
  *gc = 12;
  return c->gauge[prec];
}
double coarse_bytes(const wmg_ctx* c, int l, int prec, int nact) {
  const double s = rb_(prec), V = c->L[l].g.V, n = c->L[l].ndof;
  const double sa = (prec == WMG_PREC_SINGLE && c->L[l].A16) ? 2.0 : s;  // FP16 tensor-core copy
  return V * 9.0 * n * n * 2.0 * sa + V * 4.0 + (double)nact * V * n * 2.0 * s * 2.0;
}
// one application of the even-odd Schur complement: the odd-site pass (8 blocks per site and the
// site's block inverse, in the vectors' precision) and the even-site pass (9 blocks per site)
// (with precomputed odd-site tables the odd pass reads its 8 table blocks instead of the 8 hop
// blocks and the inverse)
double coarse_bytes_eo(const wmg_ctx* c, int l, int prec, int nact, bool tables = false) {
  const double s = rb_(prec), V = c->L[l].g.V, n = c->L[l].ndof;
  const double sa = (prec == WMG_PREC_SINGLE && c->L[l].A16) ? 2.0 : s;
  const double inv = tables ? 0.0 : V / 2 * n * n * 2.0 * s;
  return V / 2 * 17.0 * n * n * 2.0 * sa + inv + V * 4.0 + (double)nact * V * n * 2.0 * s * 2.0;
}
double transfer_bytes(const wmg_ctx* c, int l, int prec, int nact, bool half = false) {
  const LevelData& L = c->L[l];
  const double s = rb_(prec), nf = (double)L.g.V * L.ndof * (half ? 0.5 : 1.0),
               nc = (double)L.bk.coarse.V * 2.0 * L.bk.N;
  return (double)L.bk.N * nf * 2.0 * s + (double)nact * (nf + nc) * 2.0 * s;
}
static int nact_of(const wmg_ctx* c, const int* active, int nrhs) { return active ? c->n_active : nrhs; }
// `passes` full reads or writes of nact vectors of level l (vector kernels)
static double vec_bytes(const wmg_ctx* c, int l, int prec, int nact, double passes) {
  return passes * (double)nact * (double)c->L[l].nvec_elems() * (prec == WMG_PREC_DOUBLE ? 16.0 : 8.0);
}
static int blas_cls(int l) { return l == 0 ? PROF_BLAS : PROF_BLAS_COARSE; }

// ------------------------------------------------------------------------------------
// operators of a level
// ------------------------------------------------------------------------------------
// coarse stencil of level l in precision prec (FP16 tensor-core copy when it exists and prec is SINGLE)
void coarse_op(wmg_ctx* c, int l, int prec, const void* in, void* out, int nrhs, bool dagger, const int* active,
               const RedBuf* rb) {
  const LevelData& L = c->L[l];
  int impl = 0;
  if (prec == WMG_PREC_SINGLE) impl = L.impl >= 0 ? L.impl : (L.A05 ? 2 : (L.A16 ? 1 : 0));
  if (impl == 2)
    coarse_apply_tc05(L.A05, L.sA, L.g, L.ndof, in, out, nrhs, c->d_shift[l], dagger, active, rb, c->stream,
                      c->d_err);
  else if (impl == 1)
    coarse_apply_mma(L.A16, L.sA, L.g, L.ndof, in, out, nrhs, c->d_shift[l], dagger, active, rb, c->stream,
                     nullptr, c->d_err);
  else
    coarse_apply(prec, L.A[prec], L.g, L.ndof, in, out, nrhs, c->d_shift[l], dagger, active, rb, c->stream);
}

// The autotuner of the FP32 cycle's coarse stencil (coarse_tc = 3): each implementation that
// exists for this level is timed on 12 right-hand sides (3 warm-up and 10 timed launches, CUDA
// events on the context's stream) and the fastest is kept until the next setup, so that a
// right-hand side's arithmetic never depends on the batch it is solved in.
static wmg_status tune_coarse(wmg_ctx* c, int l) {
  LevelData& L = c->L[l];
  const int nr = 12;
  void *in, *out;
  TRY(vec_ws(c, l, "tune_in", WMG_PREC_SINGLE, nr, &in));
  TRY(vec_ws(c, l, "tune_out", WMG_PREC_SINGLE, nr, &out));
  CU(c, cudaMemsetAsync(in, 0, L.nvec_elems() * nr * sizeof(cf), c->stream));
  cudaEvent_t e0, e1;
  CU(c, cudaEventCreate(&e0));
  CU(c, cudaEventCreate(&e1));
  float best = 0.f;
  int pick = 0;
  for (int impl = 0; impl <= 2; ++impl) {
    if ((impl == 1 && !L.A16) || (impl == 2 && !L.A05)) continue;
    L.impl = impl;
    for (int i = 0; i < 3; ++i) coarse_op(c, l, WMG_PREC_SINGLE, in, out, nr, false, nullptr, nullptr);
    CU(c, cudaEventRecord(e0, c->stream));
    for (int i = 0; i < 10; ++i) coarse_op(c, l, WMG_PREC_SINGLE, in, out, nr, false, nullptr, nullptr);
    CU(c, cudaEventRecord(e1, c->stream));
    CU(c, cudaEventSynchronize(e1));
    float ms = 0.f;
    CU(c, cudaEventElapsedTime(&ms, e0, e1));
    c->tune_ms[l][impl] = ms / 10.f;
    if (impl == 0 || ms < best) best = ms, pick = impl;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  L.impl = pick;
  return check(c, "coarse autotune");
}

// out = A_l in   (l = 0: Wilson D; l >= 1: coarse stencil with the per-rhs shift)
void level_apply(wmg_ctx* c, int l, int prec, const void* in, void* out, int nrhs, const int* active, int red,
                 const RedBuf* rb) {
  const int na = nact_of(c, active, nrhs);
  if (l == 0) {
    ProfScope ps(c, prec == WMG_PREC_DOUBLE ? PROF_DSLASH_64 : PROF_DSLASH_LO, dslash_bytes(c, prec, na, false), na);
    int gc;
    const void* U = links(c, prec, &gc);
    dslash(prec, out, in, nullptr, U, c->fine, c->d_mass, active, nrhs, red, rb, c->stream, gc);
  } else {
    ProfScope ps(c, PROF_COARSE, coarse_bytes(c, l, prec, na), na);
    coarse_op(c, l, prec, in, out, nrhs, false, active, red == 1 ? rb : nullptr);
  }
}

// MR smoother on the fine level with FP16 storage of r and q (per-site norms); x, b FP32
static wmg_status mr_half(wmg_ctx* c, void* x, const void* b, int nrhs, int nu, const int* active) {
  const int V = c->fine.V;
  void *r, *q, *rn, *qn;
  TRY(ws_get(c, "mr_r16", spinor_h_bytes(V) * nrhs, &r));
  TRY(ws_get(c, "mr_q16", spinor_h_bytes(V) * nrhs, &q));
  TRY(ws_get(c, "mr_rn", (size_t)V * nrhs * sizeof(float), &rn));
  TRY(ws_get(c, "mr_qn", (size_t)V * nrhs * sizeof(float), &qn));
  RedBuf rb = redbuf(c, RES_MR);
  const int na = nact_of(c, active, nrhs);
  int gc;
  const void* U = links(c, WMG_PREC_SINGLE, &gc);
  const double lb = 4.0 * gc * 4.0;  // links per site, FP32
  const double hb = (double)V * lb + (double)na * V * (96.0 + 52.0);  // gauge, x + b in, r out
  {
    ProfScope ps(c, PROF_DSLASH_LO, hb + (double)na * V * 96.0, na);
    dslash_h(0, r, (float*)rn, x, nullptr, b, U, c->fine, c->d_mass, active, nrhs, 0, nullptr, c->stream, gc);
  }
  for (int i = 0; i < nu; ++i) {
    {
      ProfScope ps(c, PROF_DSLASH_LO, (double)V * lb + (double)na * V * 104.0, na);
      dslash_h(1, q, (float*)qn, r, (const float*)rn, nullptr, U, c->fine, c->d_mass, active, nrhs, 2, &rb,
               c->stream, gc);
    }
    // x read + written (FP32), r16 read (+ written), q16 read when r is updated
    const double ub = (double)na * V * (192.0 + (i + 1 < nu ? 3.0 * 52.0 : 52.0));
    ProfScope ps(c, PROF_BLAS, ub, na);
    mr_update_h(x, r, (float*)rn, q, (const float*)qn, V, nrhs, rb.result, active, i + 1 < nu, c->stream);
  }
  return check(c, "mr (FP16 storage)");
}

// MR smoother (nu steps) on level l: x is the initial guess and the result, b the rhs
wmg_status mr(wmg_ctx* c, int l, int prec, void* x, const void* b, int nrhs, int nu, const int* active) {
  if (l == 0 && prec == WMG_PREC_SINGLE && c->prm.prec_smoother == WMG_PREC_HALF && nu > 0)
    return mr_half(c, x, b, nrhs, nu, active);
  void *r, *q;
  TRY(vec_ws(c, l, "mr_r", prec, nrhs, &r));
  TRY(vec_ws(c, l, "mr_q", prec, nrhs, &q));
  const size_t n = c->L[l].nvec_elems();
  RedBuf rb = redbuf(c, RES_MR);
  const int na = nact_of(c, active, nrhs);
  const int dcls = prec == WMG_PREC_DOUBLE ? PROF_DSLASH_64 : PROF_DSLASH_LO;
  int gc;
  const void* U = links(c, prec, &gc);
  // deferred solution updates keep the step residuals: used while they fit in kMrDeferBytes
  constexpr double kMrDeferBytes = 4.0e9;
  const double rbytes = (double)nrhs * (double)n * (prec == WMG_PREC_DOUBLE ? 16.0 : 8.0);
  if (l == 0 && c->cyc_out_half && !c->use_mr_fuse && nu >= 1 && nu <= kMrMaxSteps &&
      (nu - 1) * rbytes <= kMrDeferBytes) {
    // the red/black cycle's smoother with its solution updates deferred: the residuals of the
    // steps are kept (r_1 .. r_nu, each step r_{i+1} = r_i - alpha_i q_i) and the even sites of
    // x + sum_i alpha_i r_i are formed once at the end, in the order of step-by-step updates
    MrSteps rs{};
    rs.n = nu;
    void* rbuf[kMrMaxSteps];
    rbuf[0] = r;
    for (int i = 1; i < nu; ++i) {
      char tag[16];
      std::snprintf(tag, sizeof tag, "mr_rs%d", i);
      TRY(vec_ws(c, l, tag, prec, nrhs, &rbuf[i]));
    }
    for (int i = 0; i < nu; ++i) rs.p[i] = rbuf[i];
    {
      ProfScope ps(c, dcls, dslash_bytes(c, prec, na, true), na);
      dslash(prec, r, x, b, U, c->fine, c->d_mass, active, nrhs, 0, nullptr, c->stream, gc, c->cyc_b_half ? 1 : 0);
    }
    double* red0 = res_slot(c, RES_MR);  // step i's sums at red0 + i * 3 kMaxRhs (the slot holds 16 kMaxRhs)
    const int rstride = 3 * kMaxRhs;
    for (int i = 0; i < nu; ++i) {
      RedBuf rbi{c->red_partial, c->red_counter, red0 + (size_t)i * rstride};
      {
        ProfScope ps(c, dcls, dslash_bytes(c, prec, na, false), na);
        dslash(prec, q, rbuf[i], nullptr, U, c->fine, c->d_mass, active, nrhs, 2, &rbi, c->stream, gc);
      }
      if (i + 1 < nu) {
        ProfScope ps(c, PROF_BLAS, vec_bytes(c, l, prec, na, 3), na);  // r_i, q read; r_{i+1} written
        blas_mr_rnext(prec, rbuf[i + 1], rbuf[i], q, n, nrhs, rbi.result, active, c->stream);
      }
    }
    ProfScope ps(c, PROF_BLAS, vec_bytes(c, l, prec, na, 0.5 * (nu + 2)), na);  // even halves: x, r_i in, out
    mr_combine_even(prec, x, rs, c->cyc_out_half, c->fine, nrhs, red0, rstride, active, c->stream);
    return check(c, "mr (deferred updates)");
  }
  if (l == 0 && c->use_mr_fuse && nu > 0) {
    // r = b - D x; q = D r with the step's sums; then each later step fused with the previous
    // step's update (r and q ping-pong between two buffers, the sums between two result slots);
    // the last update (x += alpha r) on its own
    void *r2, *q2;
    TRY(vec_ws(c, l, "mr_r2", prec, nrhs, &r2));
    TRY(vec_ws(c, l, "mr_q2", prec, nrhs, &q2));
    RedBuf ra = rb, rbb = redbuf(c, RES_MR2);
    {
      ProfScope ps(c, dcls, dslash_bytes(c, prec, na, true), na);
      dslash(prec, r, x, b, U, c->fine, c->d_mass, active, nrhs, 0, nullptr, c->stream, gc, c->cyc_b_half ? 1 : 0);
    }
    {
      ProfScope ps(c, dcls, dslash_bytes(c, prec, na, false), na);
      dslash(prec, q, r, nullptr, U, c->fine, c->d_mass, active, nrhs, 2, &ra, c->stream, gc);
    }
    // fused step: links + (x, r, q read; x, r', q' written) per rhs
    const double fb = dslash_bytes(c, prec, na, false) + 4.0 * (double)na * c->fine.V * 24.0 * rb_(prec);
    for (int i = 1; i < nu; ++i) {
      {
        ProfScope ps(c, dcls, fb, na);
        dslash_mr(prec, q2, r, q, r2, x, ra.result, U, c->fine, c->d_mass, active, nrhs, rbb, c->stream, gc);
      }
      std::swap(r, r2);
      std::swap(q, q2);
      std::swap(ra, rbb);
    }
    ProfScope ps(c, PROF_BLAS, vec_bytes(c, l, prec, na, 3), na);
    blas_mr_update(prec, x, r, q, n, nrhs, ra.result, false, active, c->stream);
    return check(c, "mr (fused steps)");
  }
  if (l == 0) {
    ProfScope ps(c, dcls, dslash_bytes(c, prec, na, true), na);
    dslash(prec, r, x, b, U, c->fine, c->d_mass, active, nrhs, 0, nullptr, c->stream, gc, c->cyc_b_half ? 1 : 0);
  } else {
    level_apply(c, l, prec, x, r, nrhs, active, 0, nullptr);
    ProfScope ps(c, blas_cls(l), vec_bytes(c, l, prec, na, 3), na);
    blas_xmy(prec, b, r, n, nrhs, c->stream);
  }
  for (int i = 0; i < nu; ++i) {
    if (l == 0) {
      ProfScope ps(c, dcls, dslash_bytes(c, prec, na, false), na);
      dslash(prec, q, r, nullptr, U, c->fine, c->d_mass, active, nrhs, 2, &rb, c->stream, gc);
    } else {
      level_apply(c, l, prec, r, q, nrhs, active, 0, nullptr);
      ProfScope ps(c, blas_cls(l), vec_bytes(c, l, prec, na, 2), na);
      blas_dot_norm(prec, q, r, n, nrhs, rb, c->stream);
    }
    if (l == 0 && c->cyc_out_half && i + 1 == nu) {
      // the red/black solve uses only the even sites of the result: written as half-lattice fields
      ProfScope ps(c, PROF_BLAS, vec_bytes(c, l, prec, na, 1.5), na);
      mr_update_even(prec, x, r, c->cyc_out_half, c->fine, nrhs, rb.result, active, c->stream);
      continue;
    }
    // x read + written, r read (+ written), q read when r is updated
    ProfScope ps(c, blas_cls(l), vec_bytes(c, l, prec, na, i + 1 < nu ? 5 : 3), na);
    blas_mr_update(prec, x, r, q, n, nrhs, rb.result, i + 1 < nu, active, c->stream);  // last r unused
  }
  return check(c, "mr");
}

__global__ void k_cg_init(int* done, int* iters, const double* bb, const int* active, int nrhs, int* loop_it) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r == 0) *loop_it = 0;
  if (r >= nrhs) return;
  iters[r] = 0;
  done[r] = (active && !active[r]) || !(bb[r] > 0.0);
}

// kernels launched from inside device-side graph loops (added to the host launch count)
__device__ unsigned long long g_graph_launches = 0;

// end of one captured chunk of CGNR iterations: keep looping while some right-hand side is
// not converged and the iteration cap is not reached (the loop always terminates)
__global__ void k_cg_check(const int* done, int* loop_it, int nrhs, int chunk, int maxit, int kernels_per_body,
                           cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0) return;
  bool all = true;
  for (int r = 0; r < nrhs; ++r) all = all && done[r];
  const int it = *loop_it + chunk;
  *loop_it = it;
  g_graph_launches += (unsigned long long)kernels_per_body;
  cudaGraphSetConditional(h, (!all && it < maxit) ? 1u : 0u);
}

long long graph_launch_count() {
  unsigned long long v = 0;
  cudaMemcpyFromSymbol(&v, g_graph_launches, sizeof(v));
  return (long long)v;
}

wmg_status clear_graphs(wmg_ctx* c) {
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second.first);
  c->graphs.clear();
  return WMG_OK;
}

// ---- even-odd form of the coarsest solve ----
// CG on the normal equations of S = A_ee - A_eo A_oo^-1 A_oe (every hop of the coarse stencil
// changes the parity, so A_oo is block diagonal), then x_o = A_oo^-1 (b_o - A_oe x_e).  The
// vectors keep the whole-lattice layout with zero odd sites, so the CG vector kernels and
// their per-rhs sums are those of the plain CGNR; the stopping test |r_e| <= tol |b| is the
// whole system's (its residual vanishes at the odd sites).
static bool eo_possible(const LevelData& L) {
  if (L.ndof > 64 || !L.A[0]) return false;
  for (int i = 0; i < 4; ++i)
    if (L.g.L[i] % 2) return false;
  return true;
}
static bool eo_usable(const wmg_ctx* c, int l) { return c->prm.coarse_eo && eo_possible(c->L[l]); }

struct EoTable {
  const void* inv;
  const int* idx;
  int nB = 0;                   // entries of the precomputed odd-site pass in use (0: none)
  const char* B16 = nullptr;    // entry e at B16 + e * Bstride
  size_t Bstride = 0;
  const float* sB = nullptr;    // entry e at sB + e * V / 2
  // right block-Jacobi preconditioning (CG on T = S M): the odd pass of S M (Bp), the even passes
  // of S M (E) and of M S (F, for T^dag = sigma_3 M S sigma_3), M itself and the per-rhs entry
  bool bj = false;
  const char *Bp16 = nullptr, *E16 = nullptr, *F16 = nullptr;
  const float *sBp = nullptr, *sE = nullptr, *sF = nullptr;
  const void* M32 = nullptr;    // entry e at M32 + e * V / 2 * n^2 complex FP32
  const int* bj_idx = nullptr;  // [kMaxRhs] table entry of each right-hand side
  const int* Bmask = nullptr;   // launch i's right-hand sides: Bmask[i * kMaxRhs + r] (null for one launch)
  std::vector<int> order;       // launch i uses table entry order[i]
};

// the table entries for the shifts of right-hand sides 0 .. nrhs-1 (computed for shifts not
// yet in the table; each entry depends only on the operator and its shift) and the per-rhs
// entry index on the device
static wmg_status ensure_eo(wmg_ctx* c, int l, int prec, int nrhs, EoTable* tb) {
  LevelData& L = c->L[l];
  const std::string tag = std::to_string(l) + (prec == WMG_PREC_DOUBLE ? "d" : "s");
  std::vector<double>& tab = L.eo_shift[prec];
  if (L.eo_version[prec] != L.op_version) tab.clear();
  std::vector<double> need;
  for (int r = 0; r < nrhs; ++r)
    if (std::find(need.begin(), need.end(), c->h_shift[r]) == need.end()) need.push_back(c->h_shift[r]);
  std::vector<double> missing;
  for (double v : need)
    if (std::find(tab.begin(), tab.end(), v) == tab.end()) missing.push_back(v);
  const size_t eb = eo_inverse_bytes(prec, L.g, L.ndof);
  void* inv = nullptr;
  auto it = c->ws.find("eo_inv" + tag);
  const size_t cap = it == c->ws.end() ? 0 : it->second.second / eb;
  if (tab.size() + missing.size() > cap) {
    tab.clear();
    missing = need;
  }
  TRY(ws_get(c, "eo_inv" + tag, std::max(cap, tab.size() + missing.size()) * eb, &inv));
  if (inv != L.eo_inv_ptr[prec] && !tab.empty()) {
    tab.clear();  // the buffer moved (workspaces released): recompute what this call needs
    missing = need;
  }
  L.eo_inv_ptr[prec] = inv;
  L.eo_version[prec] = L.op_version;
  if (!missing.empty()) {
    double* sh;
    TRY(ws_get(c, "eo_sh" + tag, kMaxRhs * sizeof(double), (void**)&sh));
    for (size_t i = 0; i < missing.size(); ++i) c->h_pin[i] = missing[i];
    CU(c, cudaMemcpyAsync(sh, c->h_pin, missing.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CU(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
    {
      ProfScope ps(c, PROF_CGNR, 0);
      eo_invert(prec, L.A[prec], L.g, L.ndof, sh, (int)tab.size(), (int)missing.size(), inv, c->d_flag, c->stream);
    }
    CU(c, cudaMemcpyAsync(c->h_pin_i, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CU(c, cudaStreamSynchronize(c->stream));
    if (c->h_pin_i[0]) {
      tab.clear();
      c->err = "even-odd coarsest solve: singular site block at level " + std::to_string(l);
      return WMG_ERANK;
    }
    tab.insert(tab.end(), missing.begin(), missing.end());
  }
  std::vector<int> idx(nrhs);
  for (int r = 0; r < nrhs; ++r)
    idx[r] = (int)(std::find(tab.begin(), tab.end(), c->h_shift[r]) - tab.begin());
  int* didx;
  TRY(ws_get(c, "eo_idx" + tag, kMaxRhs * sizeof(int), (void**)&didx));
  if (didx != L.eo_idx_ptr[prec] || L.eo_idx_up[prec] != idx) {
    TRY(upload_ints(c, didx, idx));
    L.eo_idx_up[prec] = idx;
    L.eo_idx_ptr[prec] = didx;
  }
  tb->inv = inv;
  tb->idx = didx;
  return WMG_OK;
}

// the parity-restricted stencil passes use the mma.sync FP16 stencil where its copy exists and
// the level's choice is a tensor-core one, else the CUDA-core stencil of precision prec
static bool eo_mma(const wmg_ctx* c, int l, int prec) {
  const LevelData& L = c->L[l];
  const int impl = prec == WMG_PREC_SINGLE ? (L.impl >= 0 ? L.impl : (L.A16 ? 1 : 0)) : 0;
  return impl >= 1 && L.A16;
}
static void eo_stencil(wmg_ctx* c, int l, int prec, const void* in, void* out, int nrhs, bool dagger,
                       const StencilEo& eo, const RedBuf* rb) {
  const LevelData& L = c->L[l];
  if (eo_mma(c, l, prec))
    coarse_apply_mma(L.A16, L.sA, L.g, L.ndof, in, out, nrhs, c->d_shift[l], dagger, nullptr, rb, c->stream, &eo,
                     c->d_err);
  else
    coarse_apply(prec, L.A[prec], L.g, L.ndof, in, out, nrhs, c->d_shift[l], dagger, nullptr, rb, c->stream, &eo);
}

// When the parity passes run on the tensor-core stencil, the odd-site pass t_o = -A_oo^-1 A_oe x_e
// is a plain hop stencil with the blocks B_k = -A_oo^-1 A_oe,k of the right-hand side's mass
// shift: one table entry per distinct shift of the call (FP32 product of the shift's inverse and
// the hop blocks, then the FP16 fragment copy), built once per operator and shift, and one launch
// per entry over the right-hand sides with that shift (a mask), so that a right-hand side's
// arithmetic does not depend on the other shifts in its batch.
static wmg_status ensure_eoB(wmg_ctx* c, int l, int prec, int nrhs, EoTable* tb) {
  tb->nB = 0;
  tb->bj = false;
  if (!c->use_eoB || !eo_mma(c, l, prec)) return WMG_OK;
  LevelData& L = c->L[l];
  const int n = L.ndof, Vh = L.g.V / 2;
  const bool bj = c->use_eobj && !L.eo_bj_singular;
  const std::string tag = std::to_string(l);
  std::vector<double> need;
  for (int r = 0; r < nrhs; ++r)
    if (std::find(need.begin(), need.end(), c->h_shift[r]) == need.end()) need.push_back(c->h_shift[r]);
  const size_t eb = stencil_mma_words(Vh, n) * 16, mb = (size_t)Vh * n * n * sizeof(cf);
  std::vector<double>& tab = L.eoB_shift;
  if (L.eoB_version != L.op_version || L.eoB_bj != bj) tab.clear();
  std::vector<double> missing;
  for (double v : need)
    if (std::find(tab.begin(), tab.end(), v) == tab.end()) missing.push_back(v);
  auto it = c->ws.find("eoB16_" + tag);
  const size_t cap = it == c->ws.end() ? 0 : it->second.second / eb;
  if (tab.size() + missing.size() > cap) {
    tab.clear();
    missing = need;
  }
  const size_t want = std::max(cap, tab.size() + missing.size());
  // the tables: FP16 fragment copies with per-site scales, one entry per shift
  const char* names[4] = {"eoB16_", "eoBp16_", "eoE16_", "eoF16_"};
  void* t16[4] = {nullptr, nullptr, nullptr, nullptr};
  void* tsc[4] = {nullptr, nullptr, nullptr, nullptr};
  void* M32 = nullptr;
  for (int t = 0; t < (bj ? 4 : 1); ++t) {
    TRY(ws_get(c, names[t] + tag, want * eb, &t16[t]));
    TRY(ws_get(c, std::string(names[t]) + "s" + tag, want * Vh * sizeof(float), &tsc[t]));
  }
  if (bj) TRY(ws_get(c, "eoM_" + tag, want * mb, &M32));
  std::vector<const void*> ptrs{t16[0], t16[1], t16[2], t16[3], tsc[0], tsc[1], tsc[2], tsc[3], M32};
  if (ptrs != L.eoB_ptrs && !tab.empty()) {  // a buffer moved: rebuild what this call needs
    tab.clear();
    missing = need;
  }
  if (!missing.empty()) {
    void *Bt, *Bt2;
    TRY(ws_get(c, "eoBt_" + tag, (size_t)Vh * 9 * n * n * sizeof(cf), &Bt));
    if (bj) TRY(ws_get(c, "eoBt2_" + tag, (size_t)Vh * 9 * n * n * sizeof(cf), &Bt2));
    const std::vector<double>& inv_tab = L.eo_shift[prec];
    ProfScope ps(c, PROF_CGNR, 0);
    // slot 0 of the odd-site tables is never read by the hop-only pass; zero it so that it does not
    // enter the per-site scales
    CU(c, cudaMemsetAsync(Bt, 0, (size_t)Vh * 9 * n * n * sizeof(cf), c->stream));
    if (bj) CU(c, cudaMemsetAsync(c->d_flag + 3, 0, sizeof(int), c->stream));
    for (double sh : missing) {
      const size_t ei = (size_t)(std::find(inv_tab.begin(), inv_tab.end(), sh) - inv_tab.begin());
      const void* inv_e = (const char*)tb->inv + ei * eo_inverse_bytes(prec, L.g, n);
      const size_t e = tab.size();
      eo_hop_inverse(L.A[WMG_PREC_SINGLE], inv_e, L.g, n, Bt, c->stream);
      stencil_to_mma(WMG_PREC_SINGLE, Bt, Vh, n, (float*)tsc[0] + e * Vh, (char*)t16[0] + e * eb, c->stream);
      if (bj) {
        void* Me = (char*)M32 + e * mb;
        eo_schur_self_inv(L.A[WMG_PREC_SINGLE], inv_e, L.g, n, sh, Me, c->d_flag + 3, c->stream);
        // slot 0 of the odd-site table must be zero for every entry (the even-site tables written
        // before it fill slot 0): it enters the per-site scale of the FP16 copy
        CU(c, cudaMemsetAsync(Bt2, 0, (size_t)Vh * 9 * n * n * sizeof(cf), c->stream));
        for (int mode = 0; mode < 3; ++mode) {
          eo_bj_table(mode, L.A[WMG_PREC_SINGLE], Bt, Me, L.g, n, sh, Bt2, c->stream);
          stencil_to_mma(WMG_PREC_SINGLE, Bt2, Vh, n, (float*)tsc[1 + mode] + e * Vh, (char*)t16[1 + mode] + e * eb,
                         c->stream);
        }
      }
      tab.push_back(sh);
    }
    if (bj) {
      CU(c, cudaMemcpyAsync(c->h_pin_i, c->d_flag + 3, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
      CU(c, cudaStreamSynchronize(c->stream));
      if (c->h_pin_i[0]) {  // a singular diagonal block of S: this operator runs without the preconditioner
        L.eo_bj_singular = true;
        L.eoB_shift.clear();
        return ensure_eoB(c, l, prec, nrhs, tb);
      }
    }
  }
  TRY(check(c, "even-odd odd-site operator"));
  L.eoB_version = L.op_version;
  L.eoB_bj = bj;
  L.eoB_ptrs = ptrs;
  // the entries in the order of `need`, their right-hand-side masks and each rhs's entry
  std::vector<int> order(need.size());
  for (size_t i = 0; i < need.size(); ++i)
    order[i] = (int)(std::find(tab.begin(), tab.end(), need[i]) - tab.begin());
  tb->nB = (int)need.size();
  tb->B16 = (const char*)t16[0];
  tb->Bstride = eb;
  tb->sB = (const float*)tsc[0];
  tb->Bmask = nullptr;
  tb->order = order;
  if (need.size() > 1) {
    std::vector<int> mask((size_t)kMaxRhs * need.size(), 0);
    for (size_t i = 0; i < need.size(); ++i)
      for (int r = 0; r < nrhs; ++r) mask[i * kMaxRhs + r] = c->h_shift[r] == need[i];
    int* dm;
    TRY(ws_get(c, "eoBm_" + tag, (size_t)kMaxRhs * kMaxRhs * sizeof(int), (void**)&dm));
    if (mask != L.eoB_mask_up || dm != L.eoB_mask_ptr) {
      for (size_t off = 0; off < mask.size(); off += kRingInts) {
        const size_t cnt = std::min(mask.size() - off, (size_t)kRingInts);
        TRY(ring_upload(c, dm + off, mask.data() + off, cnt * sizeof(int)));
      }
      L.eoB_mask_up = mask;
      L.eoB_mask_ptr = dm;
    }
    tb->Bmask = dm;
  }
  if (bj) {
    tb->bj = true;
    tb->Bp16 = (const char*)t16[1];
    tb->E16 = (const char*)t16[2];
    tb->F16 = (const char*)t16[3];
    tb->sBp = (const float*)tsc[1];
    tb->sE = (const float*)tsc[2];
    tb->sF = (const float*)tsc[3];
    tb->M32 = M32;
    std::vector<int> idx(kMaxRhs, 0);
    for (int r = 0; r < nrhs; ++r) idx[r] = (int)(std::find(tab.begin(), tab.end(), c->h_shift[r]) - tab.begin());
    int* di;
    TRY(ws_get(c, "eoBidx_" + tag, (size_t)kMaxRhs * sizeof(int), (void**)&di));
    if (idx != L.eoB_idx_up || di != L.eoB_idx_ptr) {
      TRY(upload_ints(c, di, idx));
      L.eoB_idx_up = idx;
      L.eoB_idx_ptr = di;
    }
    tb->bj_idx = di;
  }
  return WMG_OK;
}

// out_e = S in_e (or S^dag = sigma_3 S sigma_3 in_e), odd sites of out untouched; t: scratch
static void schur_op(wmg_ctx* c, int l, int prec, const EoTable& tb, const void* in, void* out, void* t, int nrhs,
                     bool dagger, const RedBuf* rb) {
  const LevelData& L = c->L[l];
  StencilEo hop;  // t_o = -A_oo^-1 A_oe in_e
  hop.parity = 1;
  hop.hop_only = 1;
  if (eo_mma(c, l, prec) && tb.nB > 0) {
    // -A_oo^-1 A_oe precomputed per shift: one launch per shift of the call.  With the block-Jacobi
    // preconditioner the operator is T = S M (odd pass B M, even pass E = [(A_xx + s) M_x | A_eo])
    // and its adjoint sigma_3 (M S) sigma_3 (odd pass B, even pass F = M_x [A_xx + s | A_eo]).
    const int Vh = L.g.V / 2;
    const bool pre = tb.bj && !dagger;
    for (int i = 0; i < tb.nB; ++i) {
      const size_t e = (size_t)tb.order[i];
      hop.opB = (pre ? tb.Bp16 : tb.B16) + e * tb.Bstride;
      hop.sB = (pre ? tb.sBp : tb.sB) + e * Vh;
      coarse_apply_mma(L.A16, L.sA, L.g, L.ndof, in, t, nrhs, c->d_shift[l], dagger,
                       tb.Bmask ? tb.Bmask + (size_t)i * kMaxRhs : nullptr, nullptr, c->stream, &hop, c->d_err);
    }
    if (tb.bj) {
      StencilEo ev;
      ev.parity = 0;
      ev.hop_in = t;
      for (int i = 0; i < tb.nB; ++i) {
        const size_t e = (size_t)tb.order[i];
        ev.opB = (dagger ? tb.F16 : tb.E16) + e * tb.Bstride;
        ev.sB = (dagger ? tb.sF : tb.sE) + e * Vh;
        coarse_apply_mma(L.A16, L.sA, L.g, L.ndof, in, out, nrhs, nullptr, dagger,
                         tb.Bmask ? tb.Bmask + (size_t)i * kMaxRhs : nullptr, rb, c->stream, &ev, c->d_err);
      }
      return;
    }
  } else if (eo_mma(c, l, prec)) {
    hop.inv = tb.inv;  // the tensor-core pass applies the block inverses in its epilogue
    hop.inv_idx = tb.idx;
    eo_stencil(c, l, prec, in, t, nrhs, dagger, hop, nullptr);
  } else {
    eo_stencil(c, l, prec, in, t, nrhs, dagger, hop, nullptr);
    eo_inv_apply(prec, tb.inv, tb.idx, L.g, L.ndof, nullptr, 0.0, t, -1.0, t, nrhs, dagger, nullptr, c->stream);
  }
  StencilEo ev;  // out_e = (A_ee + shift) in_e + A_eo t_o
  ev.parity = 0;
  ev.hop_in = t;
  eo_stencil(c, l, prec, in, out, nrhs, dagger, ev, rb);
}

wmg_status schur_apply(wmg_ctx* c, int l, int prec, const void* in, void* out, int nrhs, bool dagger) {
  if (!eo_possible(c->L[l])) return WMG_EINVAL;
  EoTable tb;
  TRY(ensure_eo(c, l, prec, nrhs, &tb));
  TRY(ensure_eoB(c, l, prec, nrhs, &tb));
  tb.bj = false;  // this entry point applies S itself
  void* t;
  TRY(vec_ws(c, l, "eo_t", prec, nrhs, &t));
  blas_zero(prec, out, c->L[l].nvec_elems(), nrhs, c->stream);
  schur_op(c, l, prec, tb, in, out, t, nrhs, dagger, nullptr);
  return check(c, "schur_apply");
}

// CG on the normal equations on level l (coarse): x = A^-1 b approximately
wmg_status cgnr(wmg_ctx* c, int l, int prec, const void* b, void* x, int nrhs, const int* active) {
  const LevelData& L = c->L[l];
  const size_t n = L.nvec_elems();
  void *r, *p, *q, *z;
  TRY(vec_ws(c, l, "cg_r", prec, nrhs, &r));
  TRY(vec_ws(c, l, "cg_p", prec, nrhs, &p));
  TRY(vec_ws(c, l, "cg_q", prec, nrhs, &q));
  TRY(vec_ws(c, l, "cg_z", prec, nrhs, &z));
  const int impl = prec == WMG_PREC_SINGLE ? (L.impl >= 0 ? L.impl : (L.A05 ? 2 : (L.A16 ? 1 : 0))) : 0;
  const bool eo = eo_usable(c, l);
  if (!eo) {
    if (c->prm.coarse_persistent && impl == 1 && nrhs <= 16) {
      // the whole solve in one cooperative kernel (FP16 tensor-core stencil, fused updates)
      void *part, *bar, *r16, *p16, *rsc, *psc;
      TRY(ws_get(c, "pcg_part", (size_t)4 * 16 * kPersistentMaxGrid * sizeof(double), &part));
      TRY(ws_get(c, "pcg_bar", 4 * sizeof(unsigned), &bar));
      TRY(ws_get(c, "pcg_r16_" + std::to_string(l), cgnr_persistent_copy_bytes(L.g.V, L.ndof), &r16));
      TRY(ws_get(c, "pcg_p16_" + std::to_string(l), cgnr_persistent_copy_bytes(L.g.V, L.ndof), &p16));
      TRY(ws_get(c, "pcg_rsc_" + std::to_string(l), (size_t)L.g.V * 16 * sizeof(float), &rsc));
      TRY(ws_get(c, "pcg_psc_" + std::to_string(l), (size_t)L.g.V * 16 * sizeof(float), &psc));
      if (!c->d_pcg_err) {
        TRY(ws_get(c, "pcg_err", sizeof(int), (void**)&c->d_pcg_err));
        CU(c, cudaMemsetAsync(c->d_pcg_err, 0, sizeof(int), c->stream));
      }
      bool ran;
      {
        ProfScope ps(c, PROF_CGNR, 0, nact_of(c, active, nrhs));
        ran = cgnr_persistent(L.A16, L.sA, L.g, L.ndof, c->d_shift[l], b, x, r, p, q, z, r16, p16, (float*)rsc,
                              (float*)psc, nrhs,
                              c->prm.coarse_tol * c->prm.coarse_tol, c->prm.coarse_maxit, active, (double*)part,
                              (unsigned*)bar, c->d_pcg_err, c->d_cgint, c->d_cgint + kMaxRhs, c->stream);
      }
      if (ran) {
        if (c->prof_on) {
          // instrumentation: the stencil applications the kernel made (2 per iteration + 1 per rhs)
          // and the operator bytes they read, from its iteration counts
          CU(c, cudaMemcpyAsync(c->h_pin_i, c->d_cgint, 2 * kMaxRhs * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
          CU(c, cudaStreamSynchronize(c->stream));
          int maxit = 0;
          double applies = 0;
          for (int i = 0; i < nrhs; ++i) {
            const int it = c->h_pin_i[kMaxRhs + i];
            if (it > 0) applies += 2.0 * it + 1.0;
            maxit = std::max(maxit, it);
          }
          c->prof_units[PROF_COARSE] += applies;
          c->prof_bytes[PROF_CGNR] += (2.0 * maxit + 1.0) * coarse_bytes(c, l, prec, nact_of(c, active, nrhs));
        }
        return check(c, "cgnr (persistent kernel)");
      }
      (void)cudaGetLastError();  // not launchable here: the multi-kernel path below
    }
  }
  EoTable tb{nullptr, nullptr};
  void* t = nullptr;
  if (eo) {
    TRY(ensure_eo(c, l, prec, nrhs, &tb));
    TRY(vec_ws(c, l, "eo_t", prec, nrhs, &t));
    TRY(ensure_eoB(c, l, prec, nrhs, &tb));
  }
  // the operator of the CG: A, or the Schur complement S on the even sites
  auto op = [&](const void* in, void* out, bool dagger, const RedBuf* rb) {
    if (eo) schur_op(c, l, prec, tb, in, out, t, nrhs, dagger, rb);
    else coarse_op(c, l, prec, in, out, nrhs, dagger, nullptr, rb);
  };
  CgScalars cg;
  cg.zz = res_slot(c, RES_CGZZ);
  cg.rr = res_slot(c, RES_CGRR);
  cg.qq = res_slot(c, RES_CGQQ);
  cg.bb = res_slot(c, RES_CGBB);
  cg.done = c->d_cgint;
  cg.iters = c->d_cgint + kMaxRhs;
  cg.tol2 = c->prm.coarse_tol * c->prm.coarse_tol;
  cudaStream_t s = c->stream;
  blas_zero(prec, x, n, nrhs, s);
  blas_norm2(prec, b, n, nrhs, redbuf(c, RES_CGBB), s);
  if (eo) {
    // r_e = b_e - A_eo A_oo^-1 b_o; q, z keep zero odd sites (their passes write even sites only)
    blas_zero(prec, r, n, nrhs, s);
    blas_zero(prec, q, n, nrhs, s);
    blas_zero(prec, z, n, nrhs, s);
    eo_inv_apply(prec, tb.inv, tb.idx, L.g, L.ndof, b, -1.0, nullptr, 0.0, t, nrhs, false, nullptr, s);
    StencilEo pre;
    pre.parity = 0;
    pre.hop_only = 1;
    pre.add = b;
    eo_stencil(c, l, prec, t, r, nrhs, false, pre, nullptr);
  } else {
    blas_convert(prec, r, prec, b, n, nrhs, nullptr, s);
  }
  RedBuf rzz0{c->red_partial, c->red_counter, cg.zz};
  op(r, z, true, &rzz0);
  blas_convert(prec, p, prec, z, n, nrhs, nullptr, s);
  k_cg_init<<<1, 64, 0, s>>>(cg.done, cg.iters, cg.bb, active, nrhs, c->d_flag + 1);
  count_launch();
  RedBuf rqq{c->red_partial, c->red_counter, cg.qq};
  RedBuf rrr{c->red_partial, c->red_counter, cg.rr};
  const double cb = eo ? coarse_bytes_eo(c, l, prec, nrhs, tb.nB > 0) : coarse_bytes(c, l, prec, nrhs);
  // one CGNR iteration: q = A p (|q|^2), x += alpha p, r -= alpha q (|r|^2, convergence flags),
  // z = A^dag r (|z|^2), p = z + beta p
  auto body = [&](int parity) {
    {
      ProfScope ps(c, PROF_COARSE, cb, nrhs);
      op(p, q, false, &rqq);
    }
    {
      ProfScope ps(c, PROF_BLAS_COARSE, vec_bytes(c, l, prec, nrhs, 6), nrhs);  // x, r read + written; p, q read
      cg_update(prec, x, r, p, q, n, nrhs, cg, parity, rrr, s);
    }
    RedBuf rzz{c->red_partial, c->red_counter, cg.zz + (1 - parity) * nrhs};
    {
      ProfScope ps(c, PROF_COARSE, cb, nrhs);
      op(r, z, true, &rzz);
    }
    {
      ProfScope ps(c, PROF_BLAS_COARSE, vec_bytes(c, l, prec, nrhs, 3), nrhs);  // p read + written, z read
      cg_xpay(prec, p, z, n, nrhs, cg, parity, s);
    }
  };
  auto all_done = [&](bool* all) -> wmg_status {
    CU(c, cudaMemcpyAsync(c->h_pin_i, cg.done, nrhs * sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(c, cudaStreamSynchronize(s));
    *all = true;
    for (int i = 0; i < nrhs; ++i) *all = *all && c->h_pin_i[i];
    return WMG_OK;
  };
  const int chunk = c->cg_chunk;  // even: every chunk starts at parity 0
  if (!c->prof_on && c->use_graphs) {
    // The CGNR loop runs on the device: a graph whose WHILE node repeats a captured chunk of
    // iterations followed by a check kernel that clears the loop condition once every
    // right-hand side has converged or coarse_maxit is reached.  Built once per argument set.
    char key[512];
    std::snprintf(key, sizeof key, "cg%d/%d/%d/%p/%p/%p/%p/%p/%p/%p/%p/%p/%p/%.17g/%d/%d/%p/%p/%p/%p/%p", l, prec,
                  nrhs, L.A[prec], (void*)L.A16, x, r, p, q, z, (void*)c->d_shift[l], (void*)c->red_partial,
                  (void*)c->res, cg.tol2, c->prm.coarse_maxit * 64 + chunk, eo ? 1 : 0, tb.inv, (const void*)tb.idx,
                  t, (const void*)tb.B16, (const void*)(size_t)(tb.nB * 1000 + (tb.Bmask ? 1 : 0)));
    std::string gkey(key);
    for (int e : tb.order) gkey += "/" + std::to_string(e);  // the odd-site launches' table entries
    if (tb.bj) gkey += "/bj";
    auto it = c->graphs.find(gkey);
    if (it == c->graphs.end()) {
      if (c->graphs.size() > 64) TRY(clear_graphs(c));
      cudaGraph_t parent;
      CU(c, cudaGraphCreate(&parent, 0));
      cudaGraphConditionalHandle h;
      cudaError_t e = cudaGraphConditionalHandleCreate(&h, parent, 1u, cudaGraphCondAssignDefault);
      cudaGraphNodeParams np = {};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      cudaGraphNode_t node;
      if (e == cudaSuccess) e = cudaGraphAddNode(&node, parent, nullptr, nullptr, 0, &np);
      if (e != cudaSuccess) {
        cudaGraphDestroy(parent);
        return fail(c, e, "cgnr graph");
      }
      cudaGraph_t bodyg = np.conditional.phGraph_out[0];
      const long long l0 = launch_count();
      e = cudaStreamBeginCaptureToGraph(s, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        pdl_scope(true);
        for (int i = 0; i < chunk; ++i) body(i & 1);
        pdl_scope(false);
        const int per = (int)(launch_count() - l0) + 1;
        k_cg_check<<<1, 32, 0, s>>>(cg.done, c->d_flag + 1, nrhs, chunk, c->prm.coarse_maxit, per, h);
        e = cudaStreamEndCapture(s, &bodyg);
      }
      count_launch((int)-(launch_count() - l0));  // captured, not launched
      cudaGraphExec_t ge = nullptr;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, parent, 0);
      cudaGraphDestroy(parent);
      if (e != cudaSuccess) return fail(c, e, "cgnr graph capture");
      it = c->graphs.emplace(gkey, std::make_pair(ge, 0LL)).first;
    }
    CU(c, cudaGraphLaunch(it->second.first, s));
  } else {
    for (int itr = 0; itr < c->prm.coarse_maxit; itr += chunk) {
      pdl_scope(true);
      for (int i = 0; i < chunk; ++i) body(i & 1);
      pdl_scope(false);
      bool all;
      TRY(all_done(&all));
      if (all) break;
    }
  }
  if (eo && tb.bj)  // the CG ran on T = S M: x_e = M y
    eo_inv_apply(prec, tb.M32, tb.bj_idx, L.g, L.ndof, nullptr, 0.0, x, 1.0, x, nrhs, false, nullptr, s, 0);
  if (eo) {
    // x_o = A_oo^-1 (b_o - A_oe x_e)
    StencilEo hop;
    hop.parity = 1;
    hop.hop_only = 1;
    eo_stencil(c, l, prec, x, t, nrhs, false, hop, nullptr);
    eo_inv_apply(prec, tb.inv, tb.idx, L.g, L.ndof, b, 1.0, t, -1.0, x, nrhs, false, active, s);
  }
  return check(c, "cgnr");
}

// One application of the multigrid preconditioner of level l: e = K_l(r); the coarsest
// level used is `last` (CGNR there).
wmg_status cycle(wmg_ctx* c, int l, int last, int prec, const void* r, void* e, int nrhs, const int* active) {
  if (l == last) return cgnr(c, l, prec, r, e, nrhs, active);
  const LevelData& L = c->L[l];
  const size_t n = L.nvec_elems();
  const int lc = l + 1;
  void *rc, *ec, *t;
  TRY(vec_ws(c, lc, "in", prec, nrhs, &rc));
  TRY(vec_ws(c, lc, "out", prec, nrhs, &ec));
  const int reps = (l == 0) ? 1 : std::max(1, c->prm.cycle_gamma);  // W-cycle: gamma at middle levels
  for (int rep = 0; rep < reps; ++rep) {
    const void* rin = r;
    if (rep > 0) {
      TRY(vec_ws(c, l, "cyc_t", prec, nrhs, &t));
      level_apply(c, l, prec, e, t, nrhs, active, 0, nullptr);
      blas_xmy(prec, r, t, n, nrhs, c->stream);
      rin = t;
    }
    {
      const int half = l == 0 && c->cyc_b_half ? 1 : 0;  // r: the even sites as half-lattice fields
      ProfScope ps(c, PROF_RESTRICT, transfer_bytes(c, l, prec, nact_of(c, active, nrhs), half != 0),
                   nact_of(c, active, nrhs));
      if (l == 0) {
        if (!(prec == WMG_PREC_SINGLE && L.P16 &&
              restrict_fine_h(L.P16, L.bk, rin, rc, nrhs, active, c->stream, half)))
          restrict_fine(prec, L.P[prec], L.bk, rin, rc, nrhs, active, c->stream, half);
      }
      else restrict_coarse(prec, L.P[prec], L.bk, rin, rc, nrhs, active, c->stream);
    }
    TRY(cycle(c, lc, last, prec, rc, ec, nrhs, active));
    void* dst = e;
    if (rep > 0) TRY(vec_ws(c, l, "cyc_p", prec, nrhs, &dst));
    {
      ProfScope ps(c, PROF_PROLONG, transfer_bytes(c, l, prec, nact_of(c, active, nrhs)), nact_of(c, active, nrhs));
      if (l == 0) {
        if (!(prec == WMG_PREC_SINGLE && L.P16 && prolong_fine_h(L.P16, L.bk, ec, dst, nrhs, active, c->stream)))
          prolong_fine(prec, L.P[prec], L.bk, ec, dst, nrhs, active, c->stream);
      }
      else prolong_coarse(prec, L.P[prec], L.bk, ec, dst, nrhs, active, c->stream);
    }
    if (rep > 0) blas_xpy(prec, dst, e, n, nrhs, c->stream);
    TRY(mr(c, l, prec, e, r, nrhs, c->prm.nu_post, active));
  }
  return check(c, "cycle");
}

// ------------------------------------------------------------------------------------
// Galerkin construction of A_{l+1} = P_l^dag A_l P_l (Sec. 2), in precision prec, into
// L[l+1].A[prec]; the other precision is converted from it.
// ------------------------------------------------------------------------------------
wmg_status galerkin(wmg_ctx* c, int l, int prec) {
  LevelData& L = c->L[l];
  LevelData& C = c->L[l + 1];
  const Blocking& bk = L.bk;
  const int n = 2 * bk.N;
  const size_t fb = L.nvec_elems() * csize(prec);
  const size_t budget = (size_t)3 << 30;
  int ncol = (int)std::max<size_t>(1, budget / (9 * fb));
  ncol = std::min(ncol, n);
  void *out9 = nullptr, *rs = nullptr;
  const bool fused = l == 0 && c->use_fused_galerkin && L.bk.N <= 32;
  if (!fused) {
    TRY(ws_get(c, "gal_out9", (size_t)ncol * 9 * fb, &out9));
    TRY(ws_get(c, "gal_rs", (size_t)ncol * 9 * C.g.V * n * csize(prec), &rs));
  }
  const size_t count = (size_t)C.g.V * 9 * n * n;
  for (int p = 0; p < 2; ++p)
    if (!C.A[p]) CU(c, cudaMalloc(&C.A[p], count * csize(p)));
  ProfScope ps(c, PROF_SETUP, 0);
  if (l == 0 && c->use_fused_galerkin &&
      galerkin_fine_fused(prec, c->gauge[prec], L.P[prec], bk, c->mass_setup, C.A[prec], c->stream))
    ncol = 0;  // done by the fused kernel
  for (int col0 = 0; ncol > 0 && col0 < n; col0 += ncol) {
    const int nc = std::min(ncol, n - col0);
    if (l == 0) {
      hop_split_fine(prec, c->gauge[prec], L.P[prec], bk, c->mass_setup, col0, nc, out9, c->stream);
      restrict_fine(prec, L.P[prec], bk, out9, rs, 9 * nc, nullptr, c->stream);
    } else {
      hop_split_coarse(prec, L.A[prec], L.P[prec], bk, col0, nc, out9, c->stream);
      restrict_coarse(prec, L.P[prec], bk, out9, rs, 9 * nc, nullptr, c->stream);
    }
    stencil_scatter(prec, rs, C.A[prec], C.g.V, n, col0, nc, c->stream);
  }
  stencil_convert(1 - prec, C.A[1 - prec], prec, C.A[prec], count, c->stream);
  C.impl = -1;
  if (c->prm.coarse_tc && c->prm.prec_sloppy == WMG_PREC_SINGLE && n % 16 == 0 && n <= 64) {
    if (!C.A16) CU(c, cudaMalloc(&C.A16, stencil_mma_words(C.g.V, n) * 16));
    if (!C.sA) CU(c, cudaMalloc((void**)&C.sA, C.g.V * sizeof(float)));
    stencil_to_mma(WMG_PREC_SINGLE, C.A[1], C.g.V, n, C.sA, C.A16, c->stream);
    if ((c->prm.coarse_tc == 2 || c->prm.coarse_tc == 3) && coarse_tc05_supported(n)) {
      if (!C.A05) CU(c, cudaMalloc(&C.A05, stencil_tc05_halves(C.g.V, n) * 2));
      stencil_to_tc05(WMG_PREC_SINGLE, C.A[1], C.g.V, n, C.sA, C.A05, c->stream);
    }
  }
  ++C.op_version;
  C.eo_bj_singular = false;
  if (c->prm.coarse_tc == 3 && c->prm.prec_sloppy == WMG_PREC_SINGLE) TRY(tune_coarse(c, l + 1));
  return check(c, "galerkin");
}

// block-orthonormalise the FP64 vectors of level l in place (they become P_l) and derive the
// other precision
wmg_status orthonormalise(wmg_ctx* c, int l) {
  LevelData& L = c->L[l];
  CU(c, cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream));
  {
    ProfScope ps(c, PROF_SETUP, 0);
    block_gs(l == 0, L.P[0], L.bk, c->d_flag, c->stream);
  }
  blas_convert(WMG_PREC_SINGLE, L.P[1], WMG_PREC_DOUBLE, L.P[0], L.nvec_elems(), L.bk.N, nullptr, c->stream);
  if (L.P16) convert_to_half2(L.P[0], L.P16, L.nvec_elems() * L.bk.N, c->stream);
  CU(c, cudaMemcpyAsync(c->h_pin_i, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaStreamSynchronize(c->stream));
  if (c->h_pin_i[0]) {
    c->err = "block Gram-Schmidt: rank-deficient block at level " + std::to_string(l);
    return WMG_ERANK;
  }
  return check(c, "block_gs");
}

// vecs (precision prec, N fields of level l) -> P_l (both precisions) -> A_{l+1}
wmg_status build_from_vectors(wmg_ctx* c, int l, int prec, const void* vecs) {
  LevelData& L = c->L[l];
  blas_convert(WMG_PREC_DOUBLE, L.P[0], prec, vecs, L.nvec_elems(), L.bk.N, nullptr, c->stream);
  TRY(orthonormalise(c, l));
  return galerkin(c, l, c->prm.prec_sloppy);
}

wmg_status normalise(wmg_ctx* c, int l, int prec, void* v, int nrhs) {
  const size_t n = c->L[l].nvec_elems();
  RedBuf rb = redbuf(c, RES_SETUP);
  blas_norm2(prec, v, n, nrhs, rb, c->stream);
  blas_scale_inv_sqrt(prec, v, n, nrhs, rb.result, 1, c->stream);
  return check(c, "normalise");
}

// Adaptive setup of level l (Sec. 2): vecs (precision prec, N fields) hold the starts.
wmg_status setup_level(wmg_ctx* c, int l, void* vecs) {
  const int prec = c->prm.prec_sloppy;
  const int N = c->L[l].bk.N;
  void* zero;
  TRY(vec_ws(c, l, "zero", prec, N, &zero));
  blas_zero(prec, zero, c->L[l].nvec_elems(), N, c->stream);
  TRY(ensure_reductions(c, N));
  std::vector<double> m(N, c->mass_setup);
  TRY(set_rhs_scalars(c, m.data(), N));
  // pass 1: relax A psi = 0 from the starts
  TRY(mr(c, l, prec, vecs, zero, N, c->prm.setup_relax, nullptr));
  TRY(normalise(c, l, prec, vecs, N));
  TRY(build_from_vectors(c, l, prec, vecs));
  // later passes: one cycle of the trial hierarchy as an approximate solve of A psi' = psi
  return improve_level(c, l, vecs, c->prm.setup_passes - 1);
}

// `passes` improvement passes of level l's vectors (precision prec_sloppy, N fields): psi_k <-
// K(psi_k) with the two-level cycle of the current hierarchy (coarse solve on level l + 1),
// normalised; P and the coarse operator are rebuilt after each pass.
wmg_status improve_level(wmg_ctx* c, int l, void* vecs, int passes) {
  const int prec = c->prm.prec_sloppy;
  const int N = c->L[l].bk.N;
  TRY(ensure_reductions(c, N));
  std::vector<double> m(N, c->mass_setup);
  TRY(set_rhs_scalars(c, m.data(), N));
  c->n_active = N;
  void* out;
  TRY(vec_ws(c, l, "setup_out", prec, N, &out));
  for (int pass = 0; pass < passes; ++pass) {
    TRY(cycle(c, l, l + 1, prec, vecs, out, N, nullptr));
    blas_convert(prec, vecs, prec, out, c->L[l].nvec_elems(), N, nullptr, c->stream);
    TRY(normalise(c, l, prec, vecs, N));
    TRY(build_from_vectors(c, l, prec, vecs));
  }
  return check(c, "improve_level");
}

// ------------------------------------------------------------------------------------
// Outer flexible GCR (Sec. 3) with FP64 reliable updates, run as a slot engine: each
// right-hand side occupies one slot with its own mass, Krylov scalars, reliable-update
// reference and convergence state; kernels run over all slots and skip inactive ones.  New
// right-hand sides are admitted into free slots at restart boundaries (k = 0), so a solve
// can take in work while others are in flight (continuous batching).  The arithmetic of a
// slot never depends on the other slots: its result is the same alone and in a batch.
// ------------------------------------------------------------------------------------
wmg_status fgcr_engine(wmg_ctx* c, int nslots, SlotSource& src, bool use_mg) {
  const int lo = use_mg ? c->prm.prec_sloppy : WMG_PREC_DOUBLE;
  // red/black: the Krylov vectors live on the even sites (half-lattice fields)
  const bool eo = use_mg && c->prm.fine_eo && c->fine.L[0] % 2 == 0;
  const size_t nfull = (size_t)c->fine.V * 12;
  const size_t n = eo ? nfull / 2 : nfull;
  const int m = std::min(std::max(c->prm.gcr_restart, 1), kMaxKrylov);
  cudaStream_t s = c->stream;
  if (nslots < 1 || nslots > kMaxRhs) return WMG_EINVAL;
  TRY(ensure_reductions(c, nslots));
  void *b64, *x64, *r64, *rlo, *Z, *W;
  TRY(vec_ws(c, 0, "gcr_b64", WMG_PREC_DOUBLE, nslots, &b64));
  TRY(vec_ws(c, 0, "gcr_x64", WMG_PREC_DOUBLE, nslots, &x64));
  TRY(vec_ws(c, 0, "gcr_r64", WMG_PREC_DOUBLE, nslots, &r64));
  TRY(vec_ws(c, 0, "gcr_rlo", lo, nslots, &rlo));
  void* xlo;
  TRY(vec_ws(c, 0, "gcr_xlo", lo, nslots, &xlo));
  const size_t slot = n * nslots * csize(lo);
  TRY(ws_get(c, std::string("gcr_Z") + (lo ? "s" : "d"), slot * m, &Z));
  TRY(ws_get(c, std::string("gcr_W") + (lo ? "s" : "d"), slot * m, &W));
  const size_t f64 = n * sizeof(cd), flo = n * csize(lo);
  auto at = [](void* base, size_t bytes, int r) { return (void*)((char*)base + bytes * r); };
  // red/black workspaces: the whole-lattice b (for the odd-site reconstruction), the halves of b,
  // the odd-site intermediate of S in both precisions, the cycle's whole-lattice in / out, and
  // the reconstructed whole-lattice solution of one slot
  void *bfull = nullptr, *beh = nullptr, *boh = nullptr, *t64 = nullptr, *tlo = nullptr, *rfl = nullptr,
       *zfl = nullptr, *xfull = nullptr, *xo = nullptr;
  const size_t ffull = nfull * sizeof(cd);
  if (eo) {
    TRY(vec_ws(c, 0, "eo_bfull", WMG_PREC_DOUBLE, nslots, &bfull));
    TRY(vec_ws(c, 0, "eo_beh", WMG_PREC_DOUBLE, nslots, &beh));
    TRY(vec_ws(c, 0, "eo_boh", WMG_PREC_DOUBLE, nslots, &boh));
    TRY(vec_ws(c, 0, "eo_t64", WMG_PREC_DOUBLE, nslots, &t64));
    TRY(vec_ws(c, 0, "eo_tlo", lo, nslots, &tlo));
    TRY(vec_ws(c, 0, "eo_rfl", lo, nslots, &rfl));
    TRY(vec_ws(c, 0, "eo_zfl", lo, nslots, &zfl));
    TRY(vec_ws(c, 0, "eo_xfull", WMG_PREC_DOUBLE, nslots, &xfull));
    TRY(vec_ws(c, 0, "eo_xo", WMG_PREC_DOUBLE, nslots, &xo));
  }
  const Geom& fg = c->fine;
  // the system's operator in the sloppy precision: D, or S = d - H_eo H_oe / d on half fields
  auto sys_op = [&](const void* in, void* out) {
    int gc;
    const void* U = links(c, lo, &gc);
    if (!eo) {
      ProfScope ps(c, lo == WMG_PREC_DOUBLE ? PROF_DSLASH_64 : PROF_DSLASH_LO, dslash_bytes(c, lo, c->n_active, false),
                   c->n_active);
      dslash(lo, out, in, nullptr, U, fg, c->d_mass, c->d_active, nslots, 0, nullptr, s, gc);
      return;
    }
    // two half-lattice passes: links once each, half fields in / out (+ the self term)
    const double hb = 0.5 * dslash_bytes(c, lo, c->n_active, false) + 0.5 * dslash_bytes(c, lo, c->n_active, true);
    ProfScope ps(c, lo == WMG_PREC_DOUBLE ? PROF_DSLASH_64 : PROF_DSLASH_LO, hb, c->n_active);
    dslash_eo(lo, 0, 1, tlo, in, nullptr, nullptr, U, gc, fg, c->d_mass, c->d_active, nslots, nullptr, s);
    dslash_eo(lo, 1, 0, out, tlo, in, nullptr, U, gc, fg, c->d_mass, c->d_active, nslots, nullptr, s);
  };
  const double tol = c->prm.tol;
  const double delta = (lo == WMG_PREC_DOUBLE) ? 0.0 : c->prm.reliable_delta;
  std::vector<int> active(nslots, 0), rel(nslots, 0), iters(nslots, 0), relups(nslots, 0);
  std::vector<double> bnorm(nslots, 0.0), ref(nslots, 0.0), tres(nslots, 0.0), mass(nslots, c->mass);
  std::vector<std::chrono::steady_clock::time_point> t0(nslots);
  std::vector<double> rn2, t;
  RedBuf rb_coef = redbuf(c, RES_COEF), rb_w = redbuf(c, RES_WRED), rb_rn = redbuf(c, RES_RN),
         rb_r64 = redbuf(c, RES_R64), rb_bb = redbuf(c, RES_BB);
  // The solution update is deferred: the preconditioned directions Z_j are kept as they are, and
  // with A Z_k = sum_{j<k} beta_jk W_j + gamma_k W_k (W orthonormal) and alpha_k = <W_k, r>, the
  // increment x += sum_k xi_k Z_k solves Gamma xi = alpha (Gamma upper triangular, diagonal
  // gamma_k, above it beta_jk).  The coefficients of every iteration of the cycle are copied on
  // the device into a history; at a reliable update, a restart or the end, a kernel solves for
  // xi over the iterations not yet folded in (alpha of earlier ones set to 0) and the directions
  // are combined into the iterate, all on the device.
  const size_t kcoef = (size_t)((kMaxKrylov + kDotChunk - 1) / kDotChunk) * nslots * 2 * kDotChunk;
  const size_t hstride = kcoef + 3 * (size_t)nslots;
  void *hist, *xi_dev, *xmask_dev;
  TRY(ws_get(c, "gcr_hist", hstride * m * sizeof(double), &hist));
  TRY(ws_get(c, "gcr_xi", (size_t)nslots * kMaxKrylov * 2 * sizeof(double), &xi_dev));
  TRY(ws_get(c, "gcr_xmask", (size_t)2 * nslots * sizeof(int), &xmask_dev));
  std::vector<int> fold_from(nslots, 0);
  auto xupdate = [&](const std::vector<int>& sel, int K) -> wmg_status {
    std::vector<int> up(2 * (size_t)nslots, 0);  // mask, then the first iteration to fold per rhs
    bool any = false;
    for (int r = 0; r < nslots; ++r) {
      if (sel[r] && fold_from[r] < K) up[r] = 1, any = true;
      up[nslots + r] = fold_from[r];
    }
    if (!any || K == 0) return WMG_OK;
    TRY(upload_ints(c, (int*)xmask_dev, up));
    {
      ProfScope ps(c, PROF_BLAS, 0);
      gcr_backsolve((const double*)hist, hstride, kcoef, K, nslots, (const int*)xmask_dev, (double*)xi_dev, s);
    }
    int nup = 0;
    for (int r = 0; r < nslots; ++r) nup += up[r];
    {
      ProfScope ps(c, PROF_BLAS, vec_bytes(c, 0, lo, nup, K + 2), nup);  // Z_0..Z_{K-1} read, x read + written
      gcr_xupdate(lo, Z, slot, K, xlo, (const double*)xi_dev, n, nslots, (const int*)xmask_dev, s);
    }
    for (int r = 0; r < nslots; ++r)
      if (up[r]) fold_from[r] = K;
    return check(c, "gcr solution update");
  };
  auto count_active = [&]() {
    c->n_active = 0;
    for (int r = 0; r < nslots; ++r) c->n_active += active[r];
  };
  // hand the finished slots (slot, converged) to the source; red/black: x_o = (b_o - H_oe x_e) / d
  // for all of them in one launch, then each whole-lattice solution
  auto finish_many = [&](const std::vector<std::pair<int, bool>>& fl) -> wmg_status {
    if (fl.empty()) return WMG_OK;
    if (eo) {
      std::vector<int> m(nslots, 0);
      for (const auto& f : fl) m[f.first] = 1;
      TRY(upload_ints(c, c->d_mask, m));
      dslash_eo(WMG_PREC_DOUBLE, 3, 1, xo, x64, boh, nullptr, c->gauge[0], 12, fg, c->d_mass, c->d_mask, nslots,
                nullptr, s);
    }
    for (const auto& f : fl) {
      const int r = f.first;
      wmg_info info{};
      info.iters = iters[r];
      info.reliable_updates = relups[r];
      info.converged = f.second;
      info.true_resid = tres[r];
      info.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0[r]).count();
      active[r] = 0;
      if (!eo) {
        TRY(src.finish(c, r, at(x64, f64, r), info));
      } else {
        eo_embed(WMG_PREC_DOUBLE, at(xfull, ffull, r), at(x64, f64, r), at(xo, f64, r), fg, 1, s);
        TRY(src.finish(c, r, at(xfull, ffull, r), info));
      }
    }
    return WMG_OK;
  };
  TRY(set_rhs_scalars(c, mass.data(), nslots));
  CU(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), s));
  int k = 0;
  while (true) {
    if (k == 0) {
      // admission into free slots
      std::vector<int> free_slots;
      for (int r = 0; r < nslots; ++r)
        if (!active[r]) free_slots.push_back(r);
      std::vector<Admission> adm;
      if (!free_slots.empty()) src.admit(c, free_slots, adm);
      if (!adm.empty()) {
        std::vector<int> mask(nslots, 0);
        for (const Admission& a : adm) {
          mass[a.slot] = a.mass;
          mask[a.slot] = 1;
          iters[a.slot] = relups[a.slot] = 0;
          t0[a.slot] = std::chrono::steady_clock::now();
        }
        TRY(set_rhs_scalars(c, mass.data(), nslots));
        for (const Admission& a : adm)
          pack_spinor(WMG_PREC_DOUBLE, a.b_canon_dev, eo ? at(bfull, ffull, a.slot) : at(b64, f64, a.slot), fg.V, 1, s);
        if (eo) {
          // b^_e = b_e - H_eo b_o / d for the admitted slots in one launch (the halves of every slot's
          // b are rewritten from its unchanged whole-lattice b)
          TRY(upload_ints(c, c->d_mask, mask));
          eo_extract(WMG_PREC_DOUBLE, beh, bfull, fg, 0, nslots, s);
          eo_extract(WMG_PREC_DOUBLE, boh, bfull, fg, 1, nslots, s);
          dslash_eo(WMG_PREC_DOUBLE, 2, 0, b64, boh, beh, nullptr, c->gauge[0], 12, fg, c->d_mass, c->d_mask, nslots,
                    nullptr, s);
        }
        for (const Admission& a : adm) {
          blas_zero(WMG_PREC_DOUBLE, at(x64, f64, a.slot), n, 1, s);
          blas_zero(lo, at(xlo, flo, a.slot), n, 1, s);
          blas_convert(WMG_PREC_DOUBLE, at(r64, f64, a.slot), WMG_PREC_DOUBLE, at(b64, f64, a.slot), n, 1, nullptr, s);
        }
        // |b| of the whole system: the stopping test is |b - D x| <= tol |b| in both forms
        blas_norm2(WMG_PREC_DOUBLE, eo ? bfull : b64, eo ? nfull : n, nslots, rb_bb, s);
        std::vector<double> bb;
        TRY(download(c, rb_bb.result, nslots, bb));
        TRY(upload_ints(c, c->d_mask, mask));
        blas_convert(lo, rlo, WMG_PREC_DOUBLE, r64, n, nslots, c->d_mask, s);
        for (const Admission& a : adm) {
          const int r = a.slot;
          bnorm[r] = ref[r] = std::sqrt(bb[r]);
          tres[r] = 0.0;
          if (bb[r] > 0.0) active[r] = 1;
          else TRY(finish_many({{r, true}}));  // b = 0: x = 0 exactly
        }
        TRY(upload_ints(c, c->d_active, active));
        count_active();
      }
      bool any = false;
      for (int r = 0; r < nslots; ++r) any = any || active[r];
      if (!any) break;
    }
    void* zk = (char*)Z + slot * k;
    void* wk = (char*)W + slot * k;
    if (use_mg && eo) {
      // the whole-lattice cycle on (r_e, 0); its even part preconditions S.  Where the fine-level
      // kernels that read the cycle's right-hand side (the restriction and the smoother's first
      // residual) take the even sites as a half-lattice field, r_e goes in as it is; otherwise
      // through its whole-lattice embedding
      const LevelData& L0 = c->L[0];
      const bool half = lo == WMG_PREC_SINGLE && c->prm.prec_smoother != WMG_PREC_HALF && L0.bk.N <= 64 &&
                        L0.bk.b[0] % 2 == 0;
      // ... and, when the cycle ends with FP32 MR steps of its own, its last step writes the even
      // sites of the result straight into z_k
      const bool out_half = half && c->prm.nu_post > 0 && !c->use_mr_fuse;
      if (half) {
        c->cyc_b_half = true;
        c->cyc_out_half = out_half ? zk : nullptr;
        const wmg_status st = cycle(c, 0, c->nlev - 1, lo, rlo, zfl, nslots, c->d_active);
        c->cyc_b_half = false;
        c->cyc_out_half = nullptr;
        TRY(st);
      } else {
        eo_embed(lo, rfl, rlo, nullptr, fg, nslots, s);
        TRY(cycle(c, 0, c->nlev - 1, lo, rfl, zfl, nslots, c->d_active));
      }
      if (!out_half) eo_extract(lo, zk, zfl, fg, 0, nslots, s);
    } else if (use_mg) {
      TRY(cycle(c, 0, c->nlev - 1, lo, rlo, zk, nslots, c->d_active));
    } else {
      blas_convert(lo, zk, lo, rlo, n, nslots, c->d_active, s);
    }
    sys_op(zk, wk);
    {
      // multidot: W_0..W_{k-1} and w read; orth: W_0..W_{k-1}, r read, w read + written;
      // update: r, w read + written
      ProfScope ps(c, PROF_BLAS, vec_bytes(c, 0, lo, c->n_active, (k > 0 ? k + 1 : 0) + (k + 3) + 4), c->n_active);
      if (k > 0) gcr_multidot(lo, W, slot, k, wk, n, nslots, c->d_active, rb_coef, s);
      gcr_orth(lo, W, nullptr, slot, k, wk, nullptr, rlo, rb_coef.result, k, n, nslots, c->d_active, rb_w, s);
      gcr_update_r(lo, rlo, wk, rb_w.result, n, nslots, c->d_active, rb_rn, s);
      double* hk = (double*)hist + (size_t)k * hstride;
      if (k > 0) CU(c, cudaMemcpyAsync(hk, rb_coef.result, kcoef * sizeof(double), cudaMemcpyDeviceToDevice, s));
      CU(c, cudaMemcpyAsync(hk + kcoef, rb_w.result, 3 * (size_t)nslots * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    TRY(check(c, "gcr iteration"));
    TRY(download(c, rb_rn.result, nslots, rn2));
    ++k;
    bool anyrel = false;
    for (int r = 0; r < nslots; ++r) {
      rel[r] = 0;
      if (!active[r]) continue;
      ++iters[r];
      const double rn = std::sqrt(std::max(rn2[r], 0.0));
      // reliable update: residual dropped by delta, apparent convergence, iteration cap, or (FP64
      // outer solver only, as in the plain restarted method) the end of a restart cycle
      const bool restart_check = (k == m) && lo == WMG_PREC_DOUBLE;
      if (rn <= tol * bnorm[r] || rn < delta * ref[r] || restart_check || iters[r] >= c->prm.max_iter || !(rn == rn))
        rel[r] = 1;
      anyrel = anyrel || rel[r];
    }
    if (anyrel) {
      // fold the sloppy iterate into the FP64 solution, then the FP64 true residual
      // r64 = b - D x64 for the active slots; applied where rel is set
      // (the FP64 operator runs only on the slots that take the update)
      TRY(xupdate(rel, k));
      TRY(upload_ints(c, c->d_mask, rel));
      blas_fold(lo, (double*)x64, xlo, n, nslots, c->d_mask, s);
      int nrel = 0;
      for (int r = 0; r < nslots; ++r) nrel += rel[r];
      {
        ProfScope ps(c, PROF_DSLASH_64, dslash_bytes(c, WMG_PREC_DOUBLE, nrel, true), nrel);
        if (!eo) {
          dslash(WMG_PREC_DOUBLE, r64, x64, b64, c->gauge[0], fg, c->d_mass, c->d_mask, nslots, 1, &rb_r64, s);
        } else {  // r^_e = b^_e - S x_e (= the whole system's residual, zero on the odd sites)
          dslash_eo(WMG_PREC_DOUBLE, 0, 1, t64, x64, nullptr, nullptr, c->gauge[0], 12, fg, c->d_mass, c->d_mask,
                    nslots, nullptr, s);
          dslash_eo(WMG_PREC_DOUBLE, 1, 0, r64, t64, x64, b64, c->gauge[0], 12, fg, c->d_mass, c->d_mask, nslots,
                    &rb_r64, s);
        }
      }
      TRY(download(c, rb_r64.result, nslots, t));
      blas_convert(lo, rlo, WMG_PREC_DOUBLE, r64, n, nslots, c->d_mask, s);
      std::vector<std::pair<int, bool>> fin;
      for (int r = 0; r < nslots; ++r) {
        if (!rel[r]) continue;
        const double tr = std::sqrt(std::max(t[r], 0.0));
        tres[r] = tr / bnorm[r];
        ref[r] = tr;
        relups[r] += 1;
        if (tr <= tol * bnorm[r]) fin.push_back({r, true});
        else if (iters[r] >= c->prm.max_iter || !(tr == tr)) fin.push_back({r, false});
      }
      TRY(finish_many(fin));
      const bool changed = !fin.empty();
      if (changed) {
        TRY(upload_ints(c, c->d_active, active));
        count_active();
      }
    }
    if (k == m) {
      TRY(xupdate(active, k));  // restart: fold the cycle's remaining increments into x
      k = 0;
    }
    if (k != 0) {
      bool any = false;
      for (int r = 0; r < nslots; ++r) any = any || active[r];
      if (!any) k = 0;  // everything finished mid-cycle: go back to admission
    }
    if (k == 0) std::fill(fold_from.begin(), fold_from.end(), 0);
  }
  CU(c, cudaStreamSynchronize(s));
  if (use_mg && c->prm.coarse_tc) {
    int e = 0;
    CU(c, cudaMemcpy(&e, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
      c->err = "a bounded wait of the tensor-core coarse stencil expired";
      return WMG_ETIMEOUT;
    }
  }
  if (use_mg && c->d_pcg_err) {
    int e = 0;
    CU(c, cudaMemcpy(&e, c->d_pcg_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) {
      CU(c, cudaMemset(c->d_pcg_err, 0, sizeof(int)));
      c->err = "a bounded wait of the persistent coarsest solve expired";
      return WMG_ETIMEOUT;
    }
  }
  return WMG_OK;
}

// ------------------------------------------------------------------------------------
// Unpreconditioned baseline (Sec. 3 compares MG with CG): CG on the normal equations of the fine
// operator in FP64, the CGLS form of the coarsest solve applied to D with D^dag = gamma_5 D gamma_5:
// x = 0, r = b, z = D^dag r, p = z; per iteration q = D p, alpha = |z|^2 / |q|^2, x += alpha p,
// r -= alpha q, z = D^dag r, beta = |z'|^2 / |z|^2, p = z + beta p, until |r| <= tol |b| per
// right-hand side.  Then the true residual b - D x; a right-hand side above tol restarts from its
// x (the others keep theirs) while the iteration cap allows.  Every right-hand side is iterated
// independently.  info.iters counts CG iterations (two operator applications each) and
// info.reliable_updates the true-residual evaluations.
// ------------------------------------------------------------------------------------
wmg_status cgnr_fine(wmg_ctx* c, const double* b_canon, double* x_canon, int nrhs, int maxit, wmg_info* info) {
  const int prec = WMG_PREC_DOUBLE;
  const int V = c->fine.V;
  const size_t n = (size_t)V * 12;
  cudaStream_t s = c->stream;
  auto t_start = std::chrono::steady_clock::now();
  TRY(ensure_reductions(c, nrhs));
  TRY(set_rhs_scalars(c, nullptr, nrhs));
  void *b, *x, *r, *p, *q, *z, *t;
  TRY(vec_ws(c, 0, "cgf_b", prec, nrhs, &b));
  TRY(vec_ws(c, 0, "cgf_x", prec, nrhs, &x));
  TRY(vec_ws(c, 0, "cgf_r", prec, nrhs, &r));
  TRY(vec_ws(c, 0, "cgf_p", prec, nrhs, &p));
  TRY(vec_ws(c, 0, "cgf_q", prec, nrhs, &q));
  TRY(vec_ws(c, 0, "cgf_z", prec, nrhs, &z));
  TRY(vec_ws(c, 0, "cgf_t", prec, nrhs, &t));
  CgScalars cg;
  cg.zz = res_slot(c, RES_CGZZ);
  cg.rr = res_slot(c, RES_CGRR);
  cg.qq = res_slot(c, RES_CGQQ);
  cg.bb = res_slot(c, RES_CGBB);
  cg.done = c->d_cgint;
  cg.iters = c->d_cgint + kMaxRhs;
  cg.tol2 = c->prm.tol * c->prm.tol;
  pack_spinor(prec, b_canon, b, V, nrhs, s);
  blas_zero(prec, x, n, nrhs, s);
  blas_norm2(prec, b, n, nrhs, redbuf(c, RES_CGBB), s);
  std::vector<double> bb, tr;
  TRY(download(c, cg.bb, nrhs, bb));
  // out = D^dag in = gamma_5 D gamma_5 in, |out|^2 per rhs (gamma_5 is unitary)
  auto dag = [&](const void* in, void* out, const RedBuf* rb) {
    blas_gamma5(prec, in, t, n, nrhs, s);
    {
      ProfScope ps(c, PROF_DSLASH_64, dslash_bytes(c, prec, nrhs, false), nrhs);
      dslash(prec, out, t, nullptr, c->gauge[prec], c->fine, c->d_mass, nullptr, nrhs, 1, rb, s);
    }
    blas_gamma5(prec, out, out, n, nrhs, s);
  };
  RedBuf rqq{c->red_partial, c->red_counter, cg.qq}, rrr{c->red_partial, c->red_counter, cg.rr};
  RedBuf rtr = redbuf(c, RES_R64);
  std::vector<int> run(nrhs, 0), its(nrhs, 0), evals(nrhs, 0), conv(nrhs, 0);
  for (int i = 0; i < nrhs; ++i) run[i] = bb[i] > 0.0, conv[i] = !(bb[i] > 0.0);
  int total = 0;
  while (true) {
    bool any = false;
    for (int i = 0; i < nrhs; ++i) any = any || run[i];
    if (!any || total >= maxit) break;
    // (re)start the running right-hand sides from x: r = b - D x, z = D^dag r, p = z
    TRY(upload_ints(c, c->d_mask, run));
    dslash(prec, r, x, b, c->gauge[prec], c->fine, c->d_mass, nullptr, nrhs, 0, nullptr, s);
    RedBuf rzz0{c->red_partial, c->red_counter, cg.zz};
    dag(r, z, &rzz0);
    blas_convert(prec, p, prec, z, n, nrhs, nullptr, s);
    k_cg_init<<<1, 64, 0, s>>>(cg.done, cg.iters, cg.bb, c->d_mask, nrhs, c->d_flag + 1);
    count_launch();
    const int chunk = 16;
    bool all = false;
    while (!all && total < maxit) {
      for (int i = 0; i < chunk; ++i) {
        const int parity = i & 1;
        {
          ProfScope ps(c, PROF_DSLASH_64, dslash_bytes(c, prec, nrhs, false), nrhs);
          dslash(prec, q, p, nullptr, c->gauge[prec], c->fine, c->d_mass, nullptr, nrhs, 1, &rqq, s);
        }
        {
          ProfScope ps(c, PROF_BLAS, vec_bytes(c, 0, prec, nrhs, 6), nrhs);
          cg_update(prec, x, r, p, q, n, nrhs, cg, parity, rrr, s);
        }
        RedBuf rzz{c->red_partial, c->red_counter, cg.zz + (1 - parity) * nrhs};
        dag(r, z, &rzz);
        {
          ProfScope ps(c, PROF_BLAS, vec_bytes(c, 0, prec, nrhs, 3), nrhs);
          cg_xpay(prec, p, z, n, nrhs, cg, parity, s);
        }
      }
      total += chunk;
      CU(c, cudaMemcpyAsync(c->h_pin_i, cg.done, nrhs * sizeof(int), cudaMemcpyDeviceToHost, s));
      CU(c, cudaStreamSynchronize(s));
      all = true;
      for (int i = 0; i < nrhs; ++i) all = all && c->h_pin_i[i];
      TRY(check(c, "fine cgnr"));
    }
    CU(c, cudaMemcpyAsync(c->h_pin_i, cg.iters, nrhs * sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(c, cudaStreamSynchronize(s));
    for (int i = 0; i < nrhs; ++i)
      if (run[i]) its[i] += c->h_pin_i[i];
    // true residuals of the running right-hand sides
    {
      ProfScope ps(c, PROF_DSLASH_64, dslash_bytes(c, prec, nrhs, true), nrhs);
      dslash(prec, r, x, b, c->gauge[prec], c->fine, c->d_mass, nullptr, nrhs, 1, &rtr, s);
    }
    TRY(download(c, rtr.result, nrhs, tr));
    for (int i = 0; i < nrhs; ++i) {
      if (!run[i]) continue;
      evals[i] += 1;
      if (tr[i] <= cg.tol2 * bb[i]) run[i] = 0, conv[i] = 1;
    }
  }
  unpack_spinor(prec, x, x_canon, V, nrhs, s);
  CU(c, cudaStreamSynchronize(s));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  bool allc = true;
  for (int i = 0; i < nrhs; ++i) {
    if (info) {
      info[i] = wmg_info{};
      info[i].iters = its[i];
      info[i].reliable_updates = evals[i];
      info[i].converged = conv[i];
      info[i].true_resid = bb[i] > 0.0 ? std::sqrt(std::max(tr.empty() ? 0.0 : tr[i], 0.0) / bb[i]) : 0.0;
      info[i].seconds = secs;
    }
    allc = allc && conv[i];
  }
  TRY(check(c, "fine cgnr"));
  return allc ? WMG_OK : WMG_ENOCONV;
}

// All right-hand sides of one call, admitted at once; results unpacked into x (canonical).
namespace {
struct BatchSource : SlotSource {
  const double* b;  // canonical device
  double* x;        // canonical device
  const double* masses;
  int nrhs;
  bool given = false;
  wmg_info* info;
  bool allconv = true;
  void admit(wmg_ctx* c, const std::vector<int>& free_slots, std::vector<Admission>& out) override {
    if (given) return;
    given = true;
    for (int r = 0; r < nrhs; ++r)
      out.push_back({free_slots[r], b + (size_t)c->fine.V * 24 * r, masses ? masses[r] : c->mass});
  }
  wmg_status finish(wmg_ctx* c, int slot, const void* x64, const wmg_info& inf) override {
    unpack_spinor(WMG_PREC_DOUBLE, x64, x + (size_t)c->fine.V * 24 * slot, c->fine.V, 1, c->stream);
    if (info) info[slot] = inf;
    allconv = allconv && inf.converged;
    return check(c, "unpack");
  }
};
}  // namespace

wmg_status fgcr(wmg_ctx* c, const double* b_canon, double* x_canon, int nrhs, const double* masses, wmg_info* info,
                bool use_mg) {
  auto t0 = std::chrono::steady_clock::now();
  if (info) std::memset(info, 0, sizeof(wmg_info) * nrhs);
  BatchSource src;
  src.b = b_canon;
  src.x = x_canon;
  src.masses = masses;
  src.nrhs = nrhs;
  src.info = info;
  TRY(fgcr_engine(c, nrhs, src, use_mg));
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (info)
    for (int r = 0; r < nrhs; ++r) info[r].seconds = secs;
  return src.allconv ? WMG_OK : WMG_ENOCONV;
}

}  // namespace wmg
