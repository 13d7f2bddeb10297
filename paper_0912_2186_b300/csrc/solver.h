// Internal host driver interface (solver.cu) used by the C ABI (api.cu).
#pragma once
#include <string>
#include <vector>

#include "ctx.h"

namespace wmg {

wmg_status fail(wmg_ctx* c, cudaError_t e, const char* what);
wmg_status check(wmg_ctx* c, const char* what);
wmg_status ws_get(wmg_ctx* c, const std::string& name, size_t bytes, void** out);
wmg_status vec_ws(wmg_ctx* c, int l, const char* tag, int prec, int nrhs, void** out);
wmg_status ensure_reductions(wmg_ctx* c, int nrhs);
wmg_status set_rhs_scalars(wmg_ctx* c, const double* masses, int nrhs);
// the links of the fine operator in precision prec and their form (gc: 12, or 8 / 18 for the
// FP32 compressed or uncompressed links selected by wmg_set_gauge_compression)
const void* links(const wmg_ctx* c, int prec, int* gc);
void level_apply(wmg_ctx* c, int l, int prec, const void* in, void* out, int nrhs, const int* active, int red,
                 const RedBuf* rb);
wmg_status mr(wmg_ctx* c, int l, int prec, void* x, const void* b, int nrhs, int nu, const int* active);
wmg_status cgnr(wmg_ctx* c, int l, int prec, const void* b, void* x, int nrhs, const int* active);
// out_e = S in_e (S^dag for dagger) with S the even-odd Schur complement of level l's operator
wmg_status schur_apply(wmg_ctx* c, int l, int prec, const void* in, void* out, int nrhs, bool dagger);
wmg_status cycle(wmg_ctx* c, int l, int last, int prec, const void* r, void* e, int nrhs, const int* active);
wmg_status galerkin(wmg_ctx* c, int l, int prec);
wmg_status orthonormalise(wmg_ctx* c, int l);
wmg_status build_from_vectors(wmg_ctx* c, int l, int prec, const void* vecs);
wmg_status setup_level(wmg_ctx* c, int l, void* vecs);
wmg_status improve_level(wmg_ctx* c, int l, void* vecs, int passes);
void prof_flush(wmg_ctx* c);
size_t context_device_bytes(const wmg_ctx* c);  // api.cu
wmg_status clear_graphs(wmg_ctx* c);
// a source of right-hand sides for the outer-solver slot engine
struct Admission {
  int slot;
  const double* b_canon_dev;  // one canonical fine spinor on the device
  double mass;
};
struct SlotSource {
  virtual ~SlotSource() {}
  // fill some of the free slots (called at restart boundaries)
  virtual void admit(wmg_ctx* c, const std::vector<int>& free_slots, std::vector<Admission>& out) = 0;
  // slot finished: its FP64 native solution and its info
  virtual wmg_status finish(wmg_ctx* c, int slot, const void* x64_native, const wmg_info& info) = 0;
};
wmg_status fgcr_engine(wmg_ctx* c, int nslots, SlotSource& src, bool use_mg);
// b_canon, x_canon: canonical device spinors, nrhs <= 64
// unpreconditioned CG on the fine normal equations (FP64 baseline); maxit caps CG iterations
wmg_status cgnr_fine(wmg_ctx* c, const double* b_canon, double* x_canon, int nrhs, int maxit, wmg_info* info);
wmg_status fgcr(wmg_ctx* c, const double* b_canon, double* x_canon, int nrhs, const double* masses, wmg_info* info,
                bool use_mg);

}  // namespace wmg
