// The C ABI of libwmg (include/wmg.h): argument checking, memory ownership and sequencing
// of the driver in solver.cu.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>

#include "ctx.h"
#include "solver.h"

using namespace wmg;

#define TRY(x)                     \
  do {                             \
    wmg_status st_ = (x);          \
    if (st_ != WMG_OK) return st_; \
  } while (0)
#define CU(c, x)                                     \
  do {                                               \
    cudaError_t e_ = (x);                            \
    if (e_ != cudaSuccess) return fail((c), e_, #x); \
  } while (0)

namespace {

size_t csize(int prec) { return prec == WMG_PREC_DOUBLE ? sizeof(cd) : sizeof(cf); }
bool prec_ok(int p) { return p == WMG_PREC_DOUBLE || p == WMG_PREC_SINGLE; }

void free_hierarchy(wmg_ctx* c) {
  cudaStreamSynchronize(c->stream);
  clear_graphs(c);
  for (int l = 0; l < WMG_MAX_LEVELS; ++l)
    for (int p = 0; p < 2; ++p) {
      if (c->L[l].A[p]) cudaFree(c->L[l].A[p]);
      if (p == 0 && c->L[l].A16) cudaFree(c->L[l].A16), c->L[l].A16 = nullptr;
      if (p == 0 && c->L[l].sA) cudaFree(c->L[l].sA), c->L[l].sA = nullptr;
      if (p == 0 && c->L[l].A05) cudaFree(c->L[l].A05), c->L[l].A05 = nullptr;
      if (c->L[l].P[p]) cudaFree(c->L[l].P[p]);
      if (p == 0 && c->L[l].P16) cudaFree(c->L[l].P16), c->L[l].P16 = nullptr;
      c->L[l].A[p] = c->L[l].P[p] = nullptr;
    }
  c->have_hier = false;
}

}  // namespace

namespace wmg {
// device bytes the context holds now: links, transfer operators, coarse operators (all copies),
// workspaces and reduction buffers
size_t context_device_bytes(const wmg_ctx* c) {
  size_t b = 0;
  const size_t V = c->fine.V;
  if (c->gauge[0]) b += V * 4 * 6 * sizeof(cd);
  if (c->gauge[1]) b += V * 4 * 6 * sizeof(cf);
  if (c->gauge8) b += gauge8_bytes((int)V);
  if (c->gauge18) b += gauge18_bytes((int)V);
  for (int l = 0; l < WMG_MAX_LEVELS; ++l) {
    const LevelData& L = c->L[l];
    const size_t pe = L.P[0] ? L.nvec_elems() * L.bk.N : 0;
    if (L.P[0]) b += pe * sizeof(cd);
    if (L.P[1]) b += pe * sizeof(cf);
    if (L.P16) b += pe * 4;
    const size_t ae = (size_t)L.g.V * 9 * L.ndof * L.ndof;
    if (L.A[0]) b += ae * sizeof(cd);
    if (L.A[1]) b += ae * sizeof(cf);
    if (L.A16) b += stencil_mma_words(L.g.V, L.ndof) * 16;
    if (L.sA) b += (size_t)L.g.V * sizeof(float);
    if (L.A05) b += stencil_tc05_halves(L.g.V, L.ndof) * 2;
  }
  for (const auto& kv : c->ws) b += kv.second.second;
  b += c->red_partial_n * sizeof(double);
  return b;
}
}  // namespace wmg

namespace {

wmg_status bad(wmg_ctx* c, const std::string& what) {
  if (c) c->err = what;
  return WMG_EINVAL;
}

// validate parameters and lay out (allocate) the hierarchy's transfer operators
wmg_status alloc_hierarchy(wmg_ctx* c, const wmg_params* p) {
  if (p->nlevels < 2 || p->nlevels > WMG_MAX_LEVELS) return bad(c, "nlevels must be 2 or 3");
  if (!prec_ok(p->prec_sloppy)) return bad(c, "prec_sloppy");
  if (p->gcr_restart < 1 || p->gcr_restart > kMaxKrylov) return bad(c, "gcr_restart must be in 1..32");
  if (p->setup_passes < 1 || p->nu_post < 0 || p->setup_relax < 0 || p->max_iter < 1 || p->coarse_maxit < 1)
    return bad(c, "iteration counts");
  if (!(p->tol > 0) || !(p->coarse_tol > 0)) return bad(c, "tolerances must be positive");
  if (p->coarse_tc < 0 || p->coarse_tc > 3) return bad(c, "coarse_tc must be 0..3");
  const bool half_ok = p->prec_sloppy == WMG_PREC_SINGLE;
  if (p->prec_nullvec != WMG_PREC_SINGLE && !(p->prec_nullvec == WMG_PREC_HALF && half_ok))
    return bad(c, "prec_nullvec must be SINGLE, or HALF with prec_sloppy SINGLE");
  if (p->prec_smoother != WMG_PREC_SINGLE && !(p->prec_smoother == WMG_PREC_HALF && half_ok))
    return bad(c, "prec_smoother must be SINGLE, or HALF with prec_sloppy SINGLE");
  if (p->coarse_persistent != 0 && p->coarse_persistent != 1) return bad(c, "coarse_persistent must be 0 or 1");
  if (p->coarse_eo != 0 && p->coarse_eo != 1) return bad(c, "coarse_eo must be 0 or 1");
  if (p->fine_eo != 0 && p->fine_eo != 1) return bad(c, "fine_eo must be 0 or 1");
  if (p->fine_eo && c->fine.L[0] % 2) return bad(c, "fine_eo needs an even x extent");
  free_hierarchy(c);
  c->prm = *p;
  c->nlev = p->nlevels;
  c->L[0].g = c->fine;
  c->L[0].ndof = 12;
  for (int l = 0; l + 1 < c->nlev; ++l) {
    LevelData& L = c->L[l];
    Blocking& bk = L.bk;
    bk.fine = L.g;
    int cd4[4];
    bk.bs = 1;
    for (int i = 0; i < 4; ++i) {
      const int b = p->block[l][i];
      if (b < 1 || L.g.L[i] % b) return bad(c, "block extents must divide the lattice");
      bk.b[i] = b;
      bk.bs *= b;
      cd4[i] = L.g.L[i] / b;
    }
    bk.coarse = make_geom(cd4);
    bk.N = p->nvec[l];
    bk.nf = L.ndof;
    if (bk.N < 1 || bk.N > 32) return bad(c, "nvec must be in 1..32");
    const int E = l == 0 ? bk.bs * 6 : bk.bs * (L.ndof / 2);
    if (E > 256 * 8) return bad(c, "block too large for the Gram-Schmidt kernel (sites x dof per chirality > 2048)");
    if (l == 0 && (size_t)4 * 12 * bk.bs * sizeof(cf) > 200 * 1024) return bad(c, "fine block too large");
    if (l > 0 && (size_t)4 * bk.bs * bk.nf * sizeof(cd) > 200 * 1024) return bad(c, "coarse block too large");
    if (E < bk.N) return bad(c, "more vectors than dof per block and chirality");
    c->L[l + 1].g = bk.coarse;
    c->L[l + 1].ndof = 2 * bk.N;
    for (int pr = 0; pr < 2; ++pr) CU(c, cudaMalloc(&L.P[pr], L.nvec_elems() * bk.N * csize(pr)));
    if (l == 0 && p->prec_nullvec == WMG_PREC_HALF)
      CU(c, cudaMalloc(&L.P16, L.nvec_elems() * bk.N * 4 /* __half2 */));
  }
  return WMG_OK;
}

// After a setup: with FP16 null vectors in the cycle (and a blocking their kernels take), the
// fine level keeps only the FP16 copy of P; when the setup's workspaces (sized for N vectors at
// once) hold more than a tenth of the device, or free memory is short, they are released and
// regrow for the solve.
wmg_status trim_after_setup(wmg_ctx* c) {
  LevelData& L = c->L[0];
  if (c->prm.prec_nullvec == WMG_PREC_HALF && L.P16 && L.bk.bs <= 256) {
    for (int p = 0; p < 2; ++p)
      if (L.P[p]) cudaFree(L.P[p]), L.P[p] = nullptr;
  }
  size_t free_b = 0, total_b = 0;
  CU(c, cudaMemGetInfo(&free_b, &total_b));
  size_t ws_total = 0;
  for (const auto& kv : c->ws) ws_total += kv.second.second;
  if (ws_total > total_b / 10 || free_b < total_b * 2 / 5) {
    clear_graphs(c);
    for (auto& kv : c->ws) cudaFree(kv.second.first);
    c->ws.clear();
  }
  return WMG_OK;
}

// 8-real links of the loaded field, and whether every link is representable (else the FP32
// operator keeps the 12-real links for this field)
wmg_status make_gauge8(wmg_ctx* c) {
  CU(c, cudaMemsetAsync(c->d_flag + 2, 0, sizeof(int), c->stream));
  pack_gauge8(c->gauge[0], c->gauge8, c->fine.V, c->d_flag + 2, c->stream);
  CU(c, cudaMemcpyAsync(c->h_pin_i, c->d_flag + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaStreamSynchronize(c->stream));
  c->gauge8_ok = c->h_pin_i[0] == 0;
  return check(c, "pack_gauge8");
}

// the FP32 links of the loaded field in the compressed (8-real) or uncompressed (18-real) form
// that the context keeps
wmg_status make_gauge_forms(wmg_ctx* c) {
  if (c->gauge8) TRY(make_gauge8(c));
  if (c->gauge18) pack_gauge18(c->gauge[0], c->gauge18, c->fine.V, c->stream);
  return check(c, "pack_gauge18");
}

}  // namespace

extern "C" {

void wmg_default_params(wmg_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->nlevels = 2;
  for (int l = 0; l < WMG_MAX_LEVELS - 1; ++l)
    for (int i = 0; i < 4; ++i) p->block[l][i] = l == 0 ? 4 : 2;
  p->nvec[0] = 24;
  p->nvec[1] = 32;
  p->setup_passes = 5;
  p->setup_relax = 100;
  p->nu_post = 4;
  p->gcr_restart = 16;
  p->cycle_gamma = 1;
  p->tol = 1e-10;
  p->coarse_tol = 0.1;
  p->coarse_maxit = 2000;
  p->max_iter = 1000;
  p->prec_sloppy = WMG_PREC_SINGLE;
  p->coarse_tc = 1;
  p->reliable_delta = 1e-4;
  p->seed = 20091212ULL;
  p->prec_nullvec = WMG_PREC_SINGLE;
  p->prec_smoother = WMG_PREC_SINGLE;
  p->coarse_persistent = 0;
  p->coarse_eo = 1;
  p->fine_eo = 0;
}

const char* wmg_strerror(wmg_status s) {
  switch (s) {
    case WMG_OK: return "ok";
    case WMG_EINVAL: return "invalid argument";
    case WMG_ENOMEM: return "out of memory";
    case WMG_ECUDA: return "CUDA error";
    case WMG_ENOCONV: return "solver did not converge";
    case WMG_ERANK: return "rank-deficient block in Gram-Schmidt";
    case WMG_ETIMEOUT: return "bounded device wait expired";
    case WMG_ESTATE: return "call order";
  }
  return "unknown status";
}

const char* wmg_last_error(const wmg_ctx* c) { return c ? c->err.c_str() : ""; }

wmg_status wmg_create(wmg_ctx** out, const int dims[4], void* stream) {
  if (!out || !dims) return WMG_EINVAL;
  *out = nullptr;
  for (int i = 0; i < 4; ++i)
    if (dims[i] < 2) return WMG_EINVAL;
  if ((long long)dims[0] * dims[1] * dims[2] * dims[3] > (1LL << 30)) return WMG_EINVAL;
  wmg_ctx* c = new wmg_ctx();
  c->fine = make_geom(dims);
  c->stream = (cudaStream_t)stream;
  cudaGetDevice(&c->device);
  if (!stream) {
    // a stream of our own (ordered with the legacy default stream) so that work can be captured
    if (cudaStreamCreate(&c->own_stream) != cudaSuccess) {
      delete c;
      return WMG_ECUDA;
    }
    c->stream = c->own_stream;
  }
  if (const char* g = std::getenv("WMG_NO_GRAPHS")) c->use_graphs = !(g[0] == '1');
  if (const char* g = std::getenv("WMG_CG_CHUNK")) {
    const int v = std::atoi(g);
    if (v >= 2 && v <= 32 && v % 2 == 0) c->cg_chunk = v;
  }
  if (const char* g = std::getenv("WMG_UNFUSED_GALERKIN")) c->use_fused_galerkin = !(g[0] == '1');
  if (const char* g = std::getenv("WMG_NO_EOB")) c->use_eoB = !(g[0] == '1');
  if (const char* g = std::getenv("WMG_NO_BJ")) c->use_eobj = !(g[0] == '1');
  if (const char* g = std::getenv("WMG_MR_FUSE")) c->use_mr_fuse = g[0] == '1';
  c->L[0].g = c->fine;
  c->L[0].ndof = 12;
  cudaError_t e = cudaSuccess;
  auto al = [&](void** p, size_t b) {
    if (e == cudaSuccess) e = cudaMalloc(p, b);
  };
  al((void**)&c->d_mass, kMaxRhs * sizeof(double));
  for (int l = 1; l < WMG_MAX_LEVELS; ++l) al((void**)&c->d_shift[l], kMaxRhs * sizeof(double));
  al((void**)&c->d_active, kMaxRhs * sizeof(int));
  al((void**)&c->d_mask, kMaxRhs * sizeof(int));
  al((void**)&c->d_flag, 4 * sizeof(int));
  al((void**)&c->d_cgint, 2 * kMaxRhs * sizeof(int));
  al((void**)&c->d_err, sizeof(int));
  al((void**)&c->red_counter, 4 * kMaxRhs * sizeof(unsigned));
  al((void**)&c->res, (size_t)24 * kMaxRhs * 16 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(c->red_counter, 0, 4 * kMaxRhs * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(c->d_shift[1], 0, kMaxRhs * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(c->d_shift[2], 0, kMaxRhs * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_pin, 4096 * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_pin_i, 4096 * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_ring, (size_t)kRingSlots * kRingInts * sizeof(int));
  for (int k = 0; k < kRingSlots && e == cudaSuccess; ++k)
    e = cudaEventCreateWithFlags(&c->ring_ev[k], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
  for (int r = 0; r < kMaxRhs; ++r) {
    c->mass_up[r] = std::nan("");
    for (int l = 0; l < WMG_MAX_LEVELS; ++l) c->shift_up[l][r] = std::nan("");
  }
  if (e == cudaSuccess) e = cudaMalloc(&c->gauge[0], (size_t)c->fine.V * 4 * 6 * sizeof(cd));
  if (e == cudaSuccess) e = cudaMalloc(&c->gauge[1], (size_t)c->fine.V * 4 * 6 * sizeof(cf));
  if (e != cudaSuccess) {
    wmg_destroy(c);
    return e == cudaErrorMemoryAllocation ? WMG_ENOMEM : WMG_ECUDA;
  }
  wmg_default_params(&c->prm);
  *out = c;
  return WMG_OK;
}

wmg_status wmg_destroy(wmg_ctx* c) {
  if (!c) return WMG_EINVAL;
  cudaStreamSynchronize(c->stream);
  prof_flush(c);
  clear_graphs(c);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  free_hierarchy(c);
  for (auto& kv : c->ws) cudaFree(kv.second.first);
  c->ws.clear();
  void* ptrs[] = {c->d_mass, c->d_shift[1], c->d_shift[2], c->d_active, c->d_mask, c->d_flag, c->d_cgint,
                  c->red_counter, c->res, c->red_partial, c->gauge[0], c->gauge[1], c->d_err, c->gauge8, c->gauge18};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->h_pin) cudaFreeHost(c->h_pin);
  if (c->h_pin_i) cudaFreeHost(c->h_pin_i);
  if (c->h_ring) cudaFreeHost(c->h_ring);
  for (int k = 0; k < kRingSlots; ++k)
    if (c->ring_ev[k]) cudaEventDestroy(c->ring_ev[k]);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  delete c;
  return WMG_OK;
}

wmg_status wmg_load_gauge_dev(wmg_ctx* c, const double* U) {
  if (!c || !U) return WMG_EINVAL;
  free_hierarchy(c);
  pack_gauge(WMG_PREC_DOUBLE, U, c->gauge[0], c->fine.V, c->stream);
  pack_gauge(WMG_PREC_SINGLE, U, c->gauge[1], c->fine.V, c->stream);
  TRY(make_gauge_forms(c));
  TRY(check(c, "pack_gauge"));
  c->have_gauge = true;
  return WMG_OK;
}

wmg_status wmg_load_gauge(wmg_ctx* c, const double* U_host) {
  if (!c || !U_host) return WMG_EINVAL;
  void* st;
  const size_t bytes = (size_t)c->fine.V * 4 * 9 * sizeof(cd);
  TRY(ws_get(c, "stage", bytes, &st));
  CU(c, cudaMemcpyAsync(st, U_host, bytes, cudaMemcpyHostToDevice, c->stream));
  TRY(wmg_load_gauge_dev(c, (const double*)st));
  CU(c, cudaStreamSynchronize(c->stream));
  return WMG_OK;
}

wmg_status wmg_set_gauge_compression(wmg_ctx* c, int reals) {
  if (!c || (reals != 12 && reals != 8 && reals != 18)) return WMG_EINVAL;
  if (reals != 8 && c->gauge8) {
    CU(c, cudaStreamSynchronize(c->stream));
    cudaFree(c->gauge8);
    c->gauge8 = nullptr;
  }
  if (reals != 18 && c->gauge18) {
    CU(c, cudaStreamSynchronize(c->stream));
    cudaFree(c->gauge18);
    c->gauge18 = nullptr;
  }
  if (reals == 8 && !c->gauge8) {
    CU(c, cudaMalloc(&c->gauge8, gauge8_bytes(c->fine.V)));
    c->gauge8_ok = false;
    if (c->have_gauge) TRY(make_gauge8(c));
  }
  if (reals == 18 && !c->gauge18) {
    CU(c, cudaMalloc(&c->gauge18, gauge18_bytes(c->fine.V)));
    if (c->have_gauge) {
      pack_gauge18(c->gauge[0], c->gauge18, c->fine.V, c->stream);
      TRY(check(c, "pack_gauge18"));
    }
  }
  c->gauge_compress = reals;
  clear_graphs(c);
  return WMG_OK;
}

wmg_status wmg_set_mass(wmg_ctx* c, double m) {
  if (!c || !(m == m)) return WMG_EINVAL;
  c->mass = m;
  return WMG_OK;
}

wmg_status wmg_setup(wmg_ctx* c, const wmg_params* p, const double* starts_host) {
  if (!c || !p) return WMG_EINVAL;
  if (!c->have_gauge) return WMG_ESTATE;
  TRY(alloc_hierarchy(c, p));
  c->mass_setup = c->mass;
  const int prec = p->prec_sloppy;
  // level 0 starts
  const int N0 = p->nvec[0];
  const size_t V = c->fine.V;
  void *canon, *vecs;
  // the starts go through a canonical FP64 stage one vector at a time (the stage of all N would be
  // 49 GB on a 48^3x96 lattice); the device stream of a vector is its slice of the seed's stream
  TRY(ws_get(c, "stage", V * 12 * sizeof(cd), &canon));
  TRY(vec_ws(c, 0, "setup_vecs", prec, N0, &vecs));
  const size_t fbp = V * 12 * (prec == WMG_PREC_DOUBLE ? sizeof(cd) : sizeof(cf));
  for (int a = 0; a < N0; ++a) {
    if (starts_host) {
      CU(c, cudaMemcpyAsync(canon, starts_host + V * 24 * a, V * 12 * sizeof(cd), cudaMemcpyHostToDevice, c->stream));
    } else {
      gaussian_fill((double*)canon, V * 24, p->seed, V * 24 * a, c->stream);
    }
    pack_spinor(prec, (const double*)canon, (char*)vecs + fbp * a, c->fine.V, 1, c->stream);
  }
  CU(c, cudaStreamSynchronize(c->stream));
  TRY(setup_level(c, 0, vecs));
  if (c->nlev == 3) {
    const int N1 = p->nvec[1];
    const size_t n1 = c->L[1].nvec_elems();
    void *stage1, *vecs1;
    TRY(ws_get(c, "stage1", n1 * N1 * sizeof(cd), &stage1));
    TRY(vec_ws(c, 1, "setup_vecs", prec, N1, &vecs1));
    gaussian_fill((double*)stage1, n1 * 2 * N1, p->seed + 1, 0, c->stream);
    blas_convert(prec, vecs1, WMG_PREC_DOUBLE, stage1, n1, N1, nullptr, c->stream);
    TRY(setup_level(c, 1, vecs1));
  }
  CU(c, cudaStreamSynchronize(c->stream));
  c->have_hier = true;
  TRY(trim_after_setup(c));
  return WMG_OK;
}

wmg_status wmg_update_gauge_dev(wmg_ctx* c, const double* U) {
  if (!c || !U) return WMG_EINVAL;
  if (!c->have_hier) return WMG_ESTATE;
  for (int l = 0; l + 1 < c->nlev; ++l)
    if (!c->L[l].P[c->prm.prec_sloppy] || !c->L[l].P[0]) {
      c->err = "update_gauge: the hierarchy keeps only FP16 fine null vectors (set up again instead)";
      return WMG_ESTATE;
    }
  CU(c, cudaStreamSynchronize(c->stream));
  pack_gauge(WMG_PREC_DOUBLE, U, c->gauge[0], c->fine.V, c->stream);
  pack_gauge(WMG_PREC_SINGLE, U, c->gauge[1], c->fine.V, c->stream);
  TRY(make_gauge_forms(c));
  TRY(check(c, "pack_gauge"));
  // the kept near-null subspace, the coarse operators of the new field
  for (int l = 0; l + 1 < c->nlev; ++l) TRY(galerkin(c, l, c->prm.prec_sloppy));
  CU(c, cudaStreamSynchronize(c->stream));
  return WMG_OK;
}

wmg_status wmg_update_gauge(wmg_ctx* c, const double* U_host) {
  if (!c || !U_host) return WMG_EINVAL;
  if (!c->have_hier) return WMG_ESTATE;
  void* st;
  const size_t bytes = (size_t)c->fine.V * 4 * 9 * sizeof(cd);
  TRY(ws_get(c, "stage", bytes, &st));
  CU(c, cudaMemcpyAsync(st, U_host, bytes, cudaMemcpyHostToDevice, c->stream));
  return wmg_update_gauge_dev(c, (const double*)st);
}

wmg_status wmg_refresh_setup(wmg_ctx* c, int passes) {
  if (!c || passes < 0) return WMG_EINVAL;
  if (!c->have_hier) return WMG_ESTATE;
  const int prec = c->prm.prec_sloppy;
  for (int l = 0; l + 1 < c->nlev; ++l) {
    LevelData& L = c->L[l];
    if (!L.P[prec] || !L.P[0]) {
      c->err = "refresh_setup: the hierarchy keeps only FP16 fine null vectors (set up again instead)";
      return WMG_ESTATE;
    }
    // the starting vectors: the N fields of P (field k holds basis vector k of every block)
    void* vecs;
    TRY(vec_ws(c, l, "setup_vecs", prec, L.bk.N, &vecs));
    blas_convert(prec, vecs, WMG_PREC_DOUBLE, L.P[0], L.nvec_elems(), L.bk.N, nullptr, c->stream);
    if (l > 0) TRY(galerkin(c, l, prec));  // the level's operator follows the refreshed level above
    TRY(improve_level(c, l, vecs, passes));
  }
  CU(c, cudaStreamSynchronize(c->stream));
  return WMG_OK;
}

wmg_status wmg_import_nullvecs(wmg_ctx* c, const wmg_params* p, int level, const double* host) {
  if (!c || !host) return WMG_EINVAL;
  if (!c->have_gauge) return WMG_ESTATE;
  if (p) {
    if (level == 0 || !c->L[0].P[0]) {
      TRY(alloc_hierarchy(c, p));
      c->mass_setup = c->mass;
    }
  } else if (!c->L[0].P[0]) {
    return WMG_ESTATE;
  }
  if (level < 0 || level >= c->nlev - 1) return bad(c, "level");
  if (level == 1 && !c->L[1].A[0]) return WMG_ESTATE;
  LevelData& L = c->L[level];
  const size_t n = L.nvec_elems();
  const int N = L.bk.N;
  TRY(ensure_reductions(c, N));
  std::vector<double> m(N, c->mass_setup);
  TRY(set_rhs_scalars(c, m.data(), N));
  if (level == 0) {
    void* canon;
    TRY(ws_get(c, "stage", n * N * sizeof(cd), &canon));
    CU(c, cudaMemcpy(canon, host, n * N * sizeof(cd), cudaMemcpyHostToDevice));
    pack_spinor(WMG_PREC_DOUBLE, (const double*)canon, L.P[0], c->fine.V, N, c->stream);
  } else {
    CU(c, cudaMemcpy(L.P[0], host, n * N * sizeof(cd), cudaMemcpyHostToDevice));
  }
  TRY(orthonormalise(c, level));
  TRY(galerkin(c, level, c->prm.prec_sloppy));
  for (int l = level + 1; l + 1 < c->nlev; ++l)
    if (c->L[l].P[0] && c->L[l].A[0] && level == 0 && c->have_hier) TRY(galerkin(c, l, c->prm.prec_sloppy));
  CU(c, cudaStreamSynchronize(c->stream));
  c->have_hier = (c->nlev == 2) || (level == 1) || c->have_hier;
  return WMG_OK;
}

wmg_status wmg_export_nullvecs(wmg_ctx* c, int level, double* host) {
  if (!c || !host) return WMG_EINVAL;
  if (level < 0 || level >= c->nlev - 1 || !c->L[level].P[0]) return WMG_ESTATE;
  LevelData& L = c->L[level];
  const size_t n = L.nvec_elems();
  const int N = L.bk.N;
  if (level == 0) {
    void* canon;
    TRY(ws_get(c, "stage", n * N * sizeof(cd), &canon));
    unpack_spinor(WMG_PREC_DOUBLE, L.P[0], (double*)canon, c->fine.V, N, c->stream);
    CU(c, cudaMemcpyAsync(host, canon, n * N * sizeof(cd), cudaMemcpyDeviceToHost, c->stream));
  } else {
    CU(c, cudaMemcpyAsync(host, L.P[0], n * N * sizeof(cd), cudaMemcpyDeviceToHost, c->stream));
  }
  CU(c, cudaStreamSynchronize(c->stream));
  return WMG_OK;
}

wmg_status wmg_export_coarse(wmg_ctx* c, int level, double* host) {
  if (!c || !host) return WMG_EINVAL;
  if (level < 0 || level + 1 >= c->nlev || !c->L[level + 1].A[0]) return WMG_ESTATE;
  const LevelData& C = c->L[level + 1];
  const int n = C.ndof;
  const size_t count = (size_t)C.g.V * 9 * n * n;
  std::vector<cd> tmp(count);
  CU(c, cudaMemcpyAsync(tmp.data(), C.A[0], count * sizeof(cd), cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaStreamSynchronize(c->stream));
  cd* out = reinterpret_cast<cd*>(host);
  for (size_t sk = 0; sk < (size_t)C.g.V * 9; ++sk)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) out[(sk * n + i) * n + j] = tmp[(sk * n + j) * n + i];
  return WMG_OK;
}

wmg_status wmg_coarse_impl(const wmg_ctx* c, int level, int* impl, float ms[3]) {
  if (!c || !impl || level < 1 || level >= WMG_MAX_LEVELS) return WMG_EINVAL;
  if (!c->have_hier || level >= c->nlev) return WMG_ESTATE;
  const LevelData& L = c->L[level];
  *impl = L.impl >= 0 ? L.impl : (L.A05 ? 2 : (L.A16 ? 1 : 0));
  if (ms)
    for (int i = 0; i < 3; ++i) ms[i] = c->tune_ms[level][i];
  return WMG_OK;
}

wmg_status wmg_device_bytes(const wmg_ctx* c, size_t* bytes) {
  if (!c || !bytes) return WMG_EINVAL;
  *bytes = context_device_bytes(c);
  return WMG_OK;
}

wmg_status wmg_level_info(const wmg_ctx* c, int level, int* nsites, int* ndof) {
  if (!c || level < 0 || level >= WMG_MAX_LEVELS) return WMG_EINVAL;
  if (level > 0 && level >= c->nlev) return WMG_ESTATE;
  if (nsites) *nsites = c->L[level].g.V;
  if (ndof) *ndof = c->L[level].ndof;
  return WMG_OK;
}

static wmg_status solve_dev_impl(wmg_ctx* c, const double* b, double* x, int nrhs, wmg_info* info, bool mg) {
  if (!c || !b || !x || nrhs < 1) return WMG_EINVAL;
  if (!c->have_gauge || (mg && !c->have_hier)) return WMG_ESTATE;
  const size_t V = c->fine.V;
  wmg_status worst = WMG_OK;
  for (int r0 = 0; r0 < nrhs; r0 += kMaxRhs) {
    const int nr = std::min(kMaxRhs, nrhs - r0);
    wmg_status st = fgcr(c, b + V * 24 * r0, x + V * 24 * r0, nr, nullptr, info ? info + r0 : nullptr, mg);
    if (st != WMG_OK && st != WMG_ENOCONV) return st;
    if (st != WMG_OK) worst = st;
  }
  CU(c, cudaStreamSynchronize(c->stream));
  TRY(check(c, "solve"));
  return worst;
}

wmg_status wmg_solve_dev(wmg_ctx* c, const double* b, double* x, int nrhs, wmg_info* info) {
  return solve_dev_impl(c, b, x, nrhs, info, true);
}

wmg_status wmg_solve_plain_dev(wmg_ctx* c, const double* b, double* x, int nrhs, wmg_info* info) {
  return solve_dev_impl(c, b, x, nrhs, info, false);
}

wmg_status wmg_solve_cgnr_dev(wmg_ctx* c, const double* b, double* x, int nrhs, int maxit, wmg_info* info) {
  if (!c || !b || !x || nrhs < 1 || maxit < 1) return WMG_EINVAL;
  if (!c->have_gauge) return WMG_ESTATE;
  const size_t V = c->fine.V;
  wmg_status worst = WMG_OK;
  for (int r0 = 0; r0 < nrhs; r0 += kMaxRhs) {
    const int nr = std::min(kMaxRhs, nrhs - r0);
    const wmg_status st = cgnr_fine(c, b + V * 24 * r0, x + V * 24 * r0, nr, maxit, info ? info + r0 : nullptr);
    if (st != WMG_OK && st != WMG_ENOCONV) return st;
    if (st != WMG_OK) worst = st;
  }
  return worst;
}

wmg_status wmg_solve(wmg_ctx* c, const double* b_host, double* x_host, int nrhs, wmg_info* info) {
  if (!c || !b_host || !x_host || nrhs < 1) return WMG_EINVAL;
  const size_t bytes = (size_t)c->fine.V * 12 * sizeof(cd) * nrhs;
  void *bd, *xd;
  TRY(ws_get(c, "host_b", bytes, &bd));
  TRY(ws_get(c, "host_x", bytes, &xd));
  CU(c, cudaMemcpyAsync(bd, b_host, bytes, cudaMemcpyHostToDevice, c->stream));
  wmg_status st = solve_dev_impl(c, (const double*)bd, (double*)xd, nrhs, info, true);
  if (st != WMG_OK && st != WMG_ENOCONV) return st;
  CU(c, cudaMemcpyAsync(x_host, xd, bytes, cudaMemcpyDeviceToHost, c->stream));
  CU(c, cudaStreamSynchronize(c->stream));
  return st;
}

wmg_status wmg_pack_spinor(wmg_ctx* c, int prec, const double* canon, void* native, int nrhs) {
  if (!c || !canon || !native || nrhs < 1 || !prec_ok(prec)) return WMG_EINVAL;
  pack_spinor(prec, canon, native, c->fine.V, nrhs, c->stream);
  return check(c, "pack_spinor");
}

wmg_status wmg_unpack_spinor(wmg_ctx* c, int prec, const void* native, double* canon, int nrhs) {
  if (!c || !canon || !native || nrhs < 1 || !prec_ok(prec)) return WMG_EINVAL;
  unpack_spinor(prec, native, canon, c->fine.V, nrhs, c->stream);
  return check(c, "unpack_spinor");
}

wmg_status wmg_apply_D(wmg_ctx* c, int prec, const void* in, void* out, int nrhs) {
  if (!c || !in || !out || nrhs < 1 || nrhs > kMaxRhs || in == out) return WMG_EINVAL;
  if (!(prec_ok(prec) || prec == WMG_PREC_HALF)) return WMG_EINVAL;
  if (!c->have_gauge) return WMG_ESTATE;
  TRY(set_rhs_scalars(c, nullptr, nrhs));
  if (prec == WMG_PREC_HALF) {
    // the smoother's FP16 storage: FP32 in -> FP16 (per-site norms) -> D -> FP16 -> FP32 out
    const int V = c->fine.V;
    void *h_in, *h_out, *n_in, *n_out;
    TRY(ws_get(c, "aD_h_in", spinor_h_bytes(V) * nrhs, &h_in));
    TRY(ws_get(c, "aD_h_out", spinor_h_bytes(V) * nrhs, &h_out));
    TRY(ws_get(c, "aD_n_in", (size_t)V * nrhs * sizeof(float), &n_in));
    TRY(ws_get(c, "aD_n_out", (size_t)V * nrhs * sizeof(float), &n_out));
    spinor_to_h(in, h_in, (float*)n_in, V, nrhs, c->stream);
    int gc;
    const void* U = links(c, WMG_PREC_SINGLE, &gc);
    dslash_h(1, h_out, (float*)n_out, h_in, (const float*)n_in, nullptr, U, c->fine, c->d_mass, nullptr, nrhs, 0,
             nullptr, c->stream, gc);
    spinor_from_h(h_out, (const float*)n_out, out, V, nrhs, c->stream);
    return check(c, "apply_D (FP16 storage)");
  }
  int gc;
  const void* U = links(c, prec, &gc);
  dslash(prec, out, in, nullptr, U, c->fine, c->d_mass, nullptr, nrhs, 0, nullptr, c->stream, gc);
  return check(c, "apply_D");
}

wmg_status wmg_apply_D_eo(wmg_ctx* c, int prec, const void* in, void* out, int nrhs) {
  if (!c || !in || !out || nrhs < 1 || nrhs > kMaxRhs || in == out || !prec_ok(prec)) return WMG_EINVAL;
  if (!c->have_gauge) return WMG_ESTATE;
  if (c->fine.L[0] % 2) return bad(c, "apply_D_eo: the x extent must be even");
  TRY(set_rhs_scalars(c, nullptr, nrhs));
  void *he, *ht, *hs;
  TRY(vec_ws(c, 0, "aDeo_e", prec, nrhs, &he));
  TRY(vec_ws(c, 0, "aDeo_t", prec, nrhs, &ht));
  TRY(vec_ws(c, 0, "aDeo_s", prec, nrhs, &hs));
  int gc;
  const void* U = links(c, prec, &gc);
  eo_extract(prec, he, in, c->fine, 0, nrhs, c->stream);
  dslash_eo(prec, 0, 1, ht, he, nullptr, nullptr, U, gc, c->fine, c->d_mass, nullptr, nrhs, nullptr, c->stream);
  dslash_eo(prec, 1, 0, hs, ht, he, nullptr, U, gc, c->fine, c->d_mass, nullptr, nrhs, nullptr, c->stream);
  eo_embed(prec, out, hs, nullptr, c->fine, nrhs, c->stream);
  return check(c, "apply_D_eo");
}

wmg_status wmg_apply_cycle(wmg_ctx* c, int prec, const void* in, void* out, int nrhs) {
  if (!c || !in || !out || nrhs < 1 || nrhs > kMaxRhs || in == out || !prec_ok(prec)) return WMG_EINVAL;
  if (!c->have_hier) return WMG_ESTATE;
  if (!c->L[0].P[prec]) {
    c->err = "apply_cycle: the hierarchy keeps only FP16 null vectors on the fine level";
    return WMG_ESTATE;
  }
  TRY(ensure_reductions(c, nrhs));
  TRY(set_rhs_scalars(c, nullptr, nrhs));
  c->n_active = nrhs;
  CU(c, cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
  TRY(cycle(c, 0, c->nlev - 1, prec, in, out, nrhs, nullptr));
  return check(c, "apply_cycle");
}

wmg_status wmg_smooth(wmg_ctx* c, int prec, const void* b, void* x, int nrhs, int nu) {
  if (!c || !b || !x || nrhs < 1 || nrhs > kMaxRhs || b == x || nu < 0 || !prec_ok(prec)) return WMG_EINVAL;
  if (!c->have_gauge) return WMG_ESTATE;
  TRY(ensure_reductions(c, nrhs));
  TRY(set_rhs_scalars(c, nullptr, nrhs));
  c->n_active = nrhs;
  TRY(mr(c, 0, prec, x, b, nrhs, nu, nullptr));
  return check(c, "smooth");
}

wmg_status wmg_restrict(wmg_ctx* c, int level, int prec, const void* fine, void* coarse, int nrhs) {
  if (!c || !fine || !coarse || nrhs < 1 || !(prec_ok(prec) || prec == WMG_PREC_HALF)) return WMG_EINVAL;
  if (level < 0 || level + 1 >= c->nlev || !c->L[level + 1].A[0]) return WMG_ESTATE;
  const LevelData& L = c->L[level];
  if (prec == WMG_PREC_HALF) {  // FP16 null vectors, FP32 buffers
    if (level != 0 || !L.P16) return WMG_ESTATE;
    if (!restrict_fine_h(L.P16, L.bk, fine, coarse, nrhs, nullptr, c->stream)) return WMG_EINVAL;
    return check(c, "restrict");
  }
  if (!L.P[prec]) {
    c->err = "restrict: the hierarchy keeps only FP16 null vectors (use WMG_PREC_HALF)";
    return WMG_ESTATE;
  }
  if (level == 0) restrict_fine(prec, L.P[prec], L.bk, fine, coarse, nrhs, nullptr, c->stream);
  else restrict_coarse(prec, L.P[prec], L.bk, fine, coarse, nrhs, nullptr, c->stream);
  return check(c, "restrict");
}

wmg_status wmg_prolong(wmg_ctx* c, int level, int prec, const void* coarse, void* fine, int nrhs) {
  if (!c || !fine || !coarse || nrhs < 1 || !(prec_ok(prec) || prec == WMG_PREC_HALF)) return WMG_EINVAL;
  if (level < 0 || level + 1 >= c->nlev || !c->L[level + 1].A[0]) return WMG_ESTATE;
  const LevelData& L = c->L[level];
  if (prec == WMG_PREC_HALF) {  // FP16 null vectors, FP32 buffers
    if (level != 0 || !L.P16) return WMG_ESTATE;
    if (!prolong_fine_h(L.P16, L.bk, coarse, fine, nrhs, nullptr, c->stream)) return WMG_EINVAL;
    return check(c, "prolong");
  }
  if (!L.P[prec]) {
    c->err = "prolong: the hierarchy keeps only FP16 null vectors (use WMG_PREC_HALF)";
    return WMG_ESTATE;
  }
  if (level == 0) prolong_fine(prec, L.P[prec], L.bk, coarse, fine, nrhs, nullptr, c->stream);
  else prolong_coarse(prec, L.P[prec], L.bk, coarse, fine, nrhs, nullptr, c->stream);
  return check(c, "prolong");
}

wmg_status wmg_apply_coarse(wmg_ctx* c, int level, int prec, int dagger, const void* in, void* out, int nrhs) {
  if (!c || !in || !out || nrhs < 1 || nrhs > kMaxRhs || in == out) return WMG_EINVAL;
  if (!prec_ok(prec) && prec != WMG_PREC_HALF) return WMG_EINVAL;
  if (level < 1 || level >= c->nlev || !c->L[level].A[0]) return WMG_ESTATE;
  if (prec == WMG_PREC_HALF && !c->L[level].A16) return WMG_ESTATE;
  TRY(set_rhs_scalars(c, nullptr, nrhs));
  const LevelData& L = c->L[level];
  if (prec == WMG_PREC_HALF && L.A05)
    coarse_apply_tc05(L.A05, L.sA, L.g, L.ndof, in, out, nrhs, c->d_shift[level], dagger != 0, nullptr, nullptr,
                      c->stream, c->d_err);
  else if (prec == WMG_PREC_HALF)
    coarse_apply_mma(L.A16, L.sA, L.g, L.ndof, in, out, nrhs, c->d_shift[level], dagger != 0, nullptr, nullptr,
                     c->stream, nullptr, c->d_err);
  else
    coarse_apply(prec, L.A[prec], L.g, L.ndof, in, out, nrhs, c->d_shift[level], dagger != 0, nullptr, nullptr,
                 c->stream);
  return check(c, "apply_coarse");
}

wmg_status wmg_apply_coarse_schur(wmg_ctx* c, int level, int prec, int dagger, const void* in, void* out, int nrhs) {
  if (!c || !in || !out || nrhs < 1 || nrhs > kMaxRhs || in == out) return WMG_EINVAL;
  if (!prec_ok(prec) && prec != WMG_PREC_HALF) return WMG_EINVAL;
  if (level < 1 || level >= c->nlev || !c->L[level].A[0]) return WMG_ESTATE;
  if (prec == WMG_PREC_HALF && !c->L[level].A16) return WMG_ESTATE;
  TRY(set_rhs_scalars(c, nullptr, nrhs));
  LevelData& L = c->L[level];
  const int keep = L.impl;
  L.impl = prec == WMG_PREC_HALF ? 1 : 0;  // the stencil copy the caller asked for
  const wmg_status st = schur_apply(c, level, prec == WMG_PREC_HALF ? WMG_PREC_SINGLE : prec, in, out, nrhs,
                                    dagger != 0);
  L.impl = keep;
  return st;
}

wmg_status wmg_profile_enable(wmg_ctx* c, int on) {
  if (!c) return WMG_EINVAL;
  prof_flush(c);
  c->prof_on = on != 0;
  for (int i = 0; i < PROF_NCLASS; ++i) {
    c->prof_ms[i] = c->prof_bytes[i] = c->prof_units[i] = 0.0;
    c->prof_n[i] = 0;
  }
  return WMG_OK;
}

wmg_status wmg_launch_count(long long* n) {
  if (!n) return WMG_EINVAL;
  *n = launch_count() + graph_launch_count();
  return WMG_OK;
}

wmg_status wmg_profile_get(wmg_ctx* c, int cls, double* ms, long long* launches, double* bytes, double* units) {
  if (!c || cls < 0 || cls >= PROF_NCLASS) return WMG_EINVAL;
  prof_flush(c);
  if (ms) *ms = c->prof_ms[cls];
  if (launches) *launches = c->prof_n[cls];
  if (bytes) *bytes = c->prof_bytes[cls];
  if (units) *units = c->prof_units[cls];
  return WMG_OK;
}

}  // extern "C"
