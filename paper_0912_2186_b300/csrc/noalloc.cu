// Allocation-free variant of the residual computation r = b - D x with |r|^2 per
// right-hand side.
//
// Why it exists: some callers must not allocate device memory during a call -- code that
// has handed all device memory to its own arena, code running where a cudaMalloc /
// cudaFree (which can synchronise the whole device) would stall other work, or code that
// wants a call whose memory footprint is fixed once the library is loaded.  Every other
// entry point here may grow the context's workspaces on demand; this one never does.
//
// Its only scratch (the per-CTA partial sums of the norms, their completion counters and
// the per-rhs mass) lives in file-scope device arrays of a fixed size, which every GPU
// that loads the library holds until the process exits.  Because all calls share those
// arrays, calls that overlap on the GPU (two streams, or two host threads) race and give
// wrong norms; issue them one after another on a stream.
#include <cstdio>
#include <mutex>

#include "ctx.h"
#include "solver.h"

namespace wmg {
namespace {

constexpr size_t kNoallocPartials = 1u << 17;  // 131072 doubles = 1 MiB of partial sums
constexpr int kNoallocMaxRhs = 64;
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_partials[kNoallocPartials];
static __device__ __align__(256) unsigned g_noalloc_counters[kNoallocMaxRhs];
static __device__ __align__(256) double g_noalloc_mass[kNoallocMaxRhs];

struct NoallocPtrs {
  double* partials = nullptr;
  unsigned* counters = nullptr;
  double* mass = nullptr;
  bool ready = false;
};
NoallocPtrs g_ptrs[kNoallocMaxDevices];
std::mutex g_ptrs_mutex;

// Device addresses of the static arrays on the context's device.  In host code the array
// names are host-side stand-ins, so the addresses are looked up once per device, with that
// device current; a call from a thread whose current device is not the context's is refused
// (the lookup and the launch would otherwise use different devices).
wmg_status noalloc_ptrs(wmg_ctx* c, NoallocPtrs* out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(c, e, "cudaGetDevice");
  if (dev != c->device) {
    c->err = "wmg_residual_noalloc: the calling thread's current device is not the context's device";
    return WMG_EINVAL;
  }
  if (dev < 0 || dev >= kNoallocMaxDevices) {
    c->err = "wmg_residual_noalloc: device index out of range";
    return WMG_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_ptrs_mutex);
  NoallocPtrs& p = g_ptrs[dev];
  if (!p.ready) {
    void* a = nullptr;
    if ((e = cudaGetSymbolAddress(&a, g_noalloc_partials)) != cudaSuccess) return fail(c, e, "cudaGetSymbolAddress");
    p.partials = (double*)a;
    if ((e = cudaGetSymbolAddress(&a, g_noalloc_counters)) != cudaSuccess) return fail(c, e, "cudaGetSymbolAddress");
    p.counters = (unsigned*)a;
    if ((e = cudaGetSymbolAddress(&a, g_noalloc_mass)) != cudaSuccess) return fail(c, e, "cudaGetSymbolAddress");
    p.mass = (double*)a;
    p.ready = true;
  }
  *out = p;
  return WMG_OK;
}

__global__ void k_noalloc_prepare(double* mass, unsigned* counters, double m, int nrhs) {
  const int i = threadIdx.x;
  if (i < kNoallocMaxRhs) counters[i] = 0u;
  if (i < nrhs) mass[i] = m;
}

}  // namespace
}  // namespace wmg

using namespace wmg;

extern "C" wmg_status wmg_residual_noalloc(wmg_ctx* c, int prec, const void* b, const void* x, void* r,
                                           double* norm2, int nrhs) {
  if (!c || !b || !x || !r || !norm2 || nrhs < 1) return WMG_EINVAL;
  if (prec != WMG_PREC_DOUBLE && prec != WMG_PREC_SINGLE) return WMG_EINVAL;
  if (!c->have_gauge) return WMG_ESTATE;
  if (r == x) {
    c->err = "wmg_residual_noalloc: r must not alias x";
    return WMG_EINVAL;
  }
  const size_t need = (size_t)nrhs * (size_t)dslash_blocks(c->fine.V);
  if (nrhs > kNoallocMaxRhs || need > kNoallocPartials) {
    char msg[256];
    std::snprintf(msg, sizeof msg,
                  "wmg_residual_noalloc: nrhs = %d needs %zu partial sums (nrhs x ceil(V/128)); the static "
                  "scratch holds %zu and at most %d right-hand sides",
                  nrhs, need, kNoallocPartials, kNoallocMaxRhs);
    c->err = msg;
    return WMG_EINVAL;
  }
  NoallocPtrs p;
  wmg_status st = noalloc_ptrs(c, &p);
  if (st != WMG_OK) return st;
  k_noalloc_prepare<<<1, kNoallocMaxRhs, 0, c->stream>>>(p.mass, p.counters, c->mass, nrhs);
  count_launch();
  RedBuf rb{p.partials, p.counters, norm2};
  dslash(prec, r, x, b, c->gauge[prec], c->fine, p.mass, nullptr, nrhs, 1, &rb, c->stream);
  return check(c, "wmg_residual_noalloc");
}
