// Internal host driver interface (solver.cu) used by the C ABI (api.cu).
#pragma once
#include <string>

#include "ctx.h"

namespace wmg {

wmg_status fail(wmg_ctx* c, cudaError_t e, const char* what);
wmg_status check(wmg_ctx* c, const char* what);
wmg_status ws_get(wmg_ctx* c, const std::string& name, size_t bytes, void** out);
wmg_status vec_ws(wmg_ctx* c, int l, const char* tag, int prec, int nrhs, void** out);
wmg_status ensure_reductions(wmg_ctx* c, int nrhs);
wmg_status set_rhs_scalars(wmg_ctx* c, const double* masses, int nrhs);
void level_apply(wmg_ctx* c, int l, int prec, const void* in, void* out, int nrhs, const int* active, int red,
                 const RedBuf* rb);
wmg_status mr(wmg_ctx* c, int l, int prec, void* x, const void* b, int nrhs, int nu, const int* active);
wmg_status cgnr(wmg_ctx* c, int l, int prec, const void* b, void* x, int nrhs, const int* active);
wmg_status cycle(wmg_ctx* c, int l, int last, int prec, const void* r, void* e, int nrhs, const int* active);
wmg_status galerkin(wmg_ctx* c, int l, int prec);
wmg_status orthonormalise(wmg_ctx* c, int l);
wmg_status build_from_vectors(wmg_ctx* c, int l, int prec, const void* vecs);
wmg_status setup_level(wmg_ctx* c, int l, void* vecs);
void prof_flush(wmg_ctx* c);
wmg_status clear_graphs(wmg_ctx* c);
wmg_status fgcr(wmg_ctx* c, const void* b64, void* x64, int nrhs, const double* masses, wmg_info* info, bool use_mg);

}  // namespace wmg
