// Internal state of a libwmg context.
#pragma once
#include <string>
#include <vector>
#include <map>

#include "kernels.h"

namespace wmg {

// kernel classes timed by the optional CUDA-event instrumentation (wmg_profile_*)
enum { PROF_DSLASH_LO = 0, PROF_DSLASH_64, PROF_COARSE, PROF_RESTRICT, PROF_PROLONG, PROF_BLAS, PROF_SETUP,
       PROF_CGNR, PROF_BLAS_COARSE, PROF_NCLASS };

// pinned staging ring for small asynchronous host-to-device uploads (flags, masks): a slot is
// reused only after the copy that last read it has completed (one event per slot)
constexpr int kRingSlots = 8;
constexpr int kRingInts = 256;

struct ProfRec {
  cudaEvent_t a, b;
  int cls;
  double bytes;
  double units;  // right-hand sides (vector applications) processed
};

struct LevelData {
  Geom g;            // lattice of this level
  int ndof = 12;     // complex dof per site (12 fine, 2N coarse)
  // coarse operator of this level (levels >= 1): [site][9][col][row], per precision
  void* A[2] = {nullptr, nullptr};
  void* A16 = nullptr;     // FP16 fragment-order copy for the tensor-core apply (or null)
  float* sA = nullptr;     // its per-site scale
  void* A05 = nullptr;     // FP16 canonical-layout copy for the tcgen05 apply (or null)
  int impl = -1;           // FP32-cycle stencil implementation picked by the autotuner (coarse_tc 3):
                           // 0 CUDA cores FP32, 1 mma.sync FP16, 2 tcgen05 FP16; -1 by availability
  // transfer to the next level (levels < nlev - 1)
  Blocking bk{};
  void* P[2] = {nullptr, nullptr};  // N fields of this level, per precision (P[0] = FP64)
  void* P16 = nullptr;     // FP16 (__half2) copy of the fine-level P for the cycle (prec_nullvec HALF)
  long long op_version = 0;  // bumped whenever the coarse operator of this level is rebuilt
  // even-odd coarsest solve, per precision: table of (A_oo + shift I)^-1 entries, one per
  // distinct shift (in a workspace buffer), and the per-rhs entry index last uploaded
  std::vector<double> eo_shift[2];
  const void* eo_inv_ptr[2] = {nullptr, nullptr};
  long long eo_version[2] = {-1, -1};
  std::vector<int> eo_idx_up[2];
  const void* eo_idx_ptr[2] = {nullptr, nullptr};
  // precomputed odd-site pass -A_oo^-1 A_oe (FP16 tensor-core copies), one entry per mass shift
  std::vector<double> eoB_shift;
  long long eoB_version = -1;
  bool eoB_bj = false;               // the entries include the block-Jacobi tables
  bool eo_bj_singular = false;       // a diagonal block of S was singular: no block-Jacobi
  std::vector<const void*> eoB_ptrs;
  std::vector<int> eoB_idx_up;
  const void* eoB_idx_ptr = nullptr;
  std::vector<int> eoB_mask_up;  // per-entry right-hand-side masks last uploaded
  const void* eoB_mask_ptr = nullptr;
  size_t nvec_elems() const { return (size_t)g.V * ndof; }  // complex numbers per field
};

}  // namespace wmg

struct wmg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  Geom fine{};
  void* gauge[2] = {nullptr, nullptr};  // native 12-real links, FP64 and FP32
  int gauge_compress = 12;               // links of the FP32 sloppy operator: 18, 12 or 8 reals
  void* gauge8 = nullptr;                // 8-real FP32 links (with gauge_compress 8)
  void* gauge18 = nullptr;               // 18-real FP32 links (with gauge_compress 18)
  bool gauge8_ok = false;                // the loaded field is representable with 8 reals
  bool have_gauge = false;
  double mass = 0.0, mass_setup = 0.0;
  wmg_params prm{};
  bool have_hier = false;
  int nlev = 1;
  wmg::LevelData L[WMG_MAX_LEVELS];
  std::string err;
  // allocations
  std::vector<void*> owned;
  std::map<std::string, std::pair<void*, size_t>> ws;  // named grow-only workspaces
  // reductions (shared partials and counters, distinct result arrays)
  double* red_partial = nullptr;
  size_t red_partial_n = 0;
  unsigned* red_counter = nullptr;
  double* res = nullptr;  // result arena [kResSlots][kMaxRhs * 16]
  double* d_mass = nullptr;                    // [kMaxRhs] Wilson mass per rhs
  double* d_shift[WMG_MAX_LEVELS] = {nullptr, nullptr, nullptr};  // coarse shift per rhs
  double h_shift[wmg::kMaxRhs] = {};                                // its host copy
  int* d_active = nullptr;                     // [kMaxRhs]
  int* d_mask = nullptr;                       // [kMaxRhs]
  int* d_flag = nullptr;                       // misc device flag
  int* d_cgint = nullptr;                      // [2][kMaxRhs] cg done / iters
  cudaStream_t own_stream = nullptr;          // created when the caller passes no stream
  bool use_graphs = true;                      // capture the coarsest CGNR iterations
  int cg_chunk = 2;                            // CGNR iterations between convergence checks (even)
  bool cyc_b_half = false;  // the fine-level cycle's right-hand side is an even half-lattice field
  void* cyc_out_half = nullptr;  // non-null: the fine-level cycle's result goes here (even sites,
                                 // half-lattice), from its last MR step
  bool use_fused_galerkin = true;              // fused fine-level Galerkin kernel
  bool use_eoB = true;                         // precomputed odd-site pass of the coarse Schur complement
  bool use_eobj = true;                        // block-Jacobi preconditioned coarsest CG (with use_eoB)
  bool use_mr_fuse = false;                    // fine MR steps fused with the previous step's update
                                               // (WMG_MR_FUSE=1; measured no faster on the 16^3x32 job)
  int* d_pcg_err = nullptr;                    // sticky error flag of the persistent CGNR (per solve)
  int* d_err = nullptr;                        // error word of the tensor-core stencils' bounded waits
                                               // (cleared at the start of each solve)
  // values last uploaded to d_mass / d_shift (NaN = unknown), so that an unchanged set is not
  // uploaded again
  double mass_up[wmg::kMaxRhs];
  double shift_up[WMG_MAX_LEVELS][wmg::kMaxRhs];
  int* h_ring = nullptr;                       // pinned [kRingSlots][kRingInts]
  cudaEvent_t ring_ev[wmg::kRingSlots] = {};
  int ring_pos = 0;
  std::map<std::string, std::pair<cudaGraphExec_t, long long>> graphs;  // + launches per replay
  int n_active = 0;                            // active right-hand sides of the current solve
  float tune_ms[WMG_MAX_LEVELS][3] = {};       // autotuner: ms per 12-rhs launch of each stencil impl
  // instrumentation
  bool prof_on = false;
  std::vector<wmg::ProfRec> prof_pending;
  std::vector<cudaEvent_t> ev_pool;
  double prof_ms[wmg::PROF_NCLASS] = {};
  double prof_bytes[wmg::PROF_NCLASS] = {};
  double prof_units[wmg::PROF_NCLASS] = {};
  long long prof_n[wmg::PROF_NCLASS] = {};
  double* h_pin = nullptr;                     // pinned host scratch [4096]
  int* h_pin_i = nullptr;                      // pinned host scratch [4096]
};
