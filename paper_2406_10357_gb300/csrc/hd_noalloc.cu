// Nearest-triangle queries that allocate nothing.
//
// hd_nearest takes its per-point work records and counters from cudaMallocAsync.  Some
// callers cannot let a library allocate device memory while they run: programs that hand all
// device memory to their own allocator up front (a library allocation would fail, or take
// memory their allocator counts on), services that must keep within a fixed device-memory
// budget, and latency-critical loops that must not wait in the driver for an allocation.  This
// variant keeps its scratch in a fixed array that lives in the library's device image instead,
// so a call only issues a memset and kernel launches on the caller's stream.
//
// The array is a file-scope __device__ variable: every GPU that loads the library holds it
// (kNoAllocBytes) until the process exits.  All calls share it and it keeps the last call's
// contents; the counters are cleared at the start of every call, and the per-point records
// are fully written before they are read.  Calls whose work overlaps on the GPU (different
// streams, or different host threads, without ordering between them) race on the array and
// must be serialised by the caller.
#include <mutex>

#include "hd_bnb.cuh"
#include "hd_mixed.cuh"

namespace hd {
namespace {

constexpr int64_t kNoAllocMaxPoints = HD_NOALLOC_MAX_POINTS;
static_assert(sizeof(VtxM) == 64 && sizeof(VtxD) == 64, "one 64-byte record per point");
constexpr size_t kNoAllocTail = 512;  // the counters (RunState), after the per-point records
static_assert(sizeof(RunState) <= kNoAllocTail, "counters fit the reserved tail");
// per point: a 64-byte record and a slot of the long-query list; then the counters
constexpr size_t kNoAllocBytes = kNoAllocMaxPoints * (64 + 4) + kNoAllocTail;

static __device__ __align__(256) unsigned char g_scratch[kNoAllocBytes];

// Device address of g_scratch, per device.  In host code the name g_scratch is only a
// host-side stand-in for the symbol, not a device address, so it is looked up once per device
// with that device current.  The address is kept for the life of the process: it belongs to
// the device's primary context, so a cudaDeviceReset (which destroys that context and the
// module's copy of the array) makes it stale, and the entry point must not be used on a device
// after such a reset.
std::mutex g_mu;
void* g_addr[64] = {};

int scratch_address(void** out) {
  int dev = 0;
  HD_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return HD_ERR_INVALID;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    HD_TRY(cudaGetSymbolAddress(&p, g_scratch));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return HD_OK;
}

template <class P>
int run(const hd_bvh* B, const void* Pts, int ptype, int64_t n, cudaStream_t s, double* dist, int32_t* idx,
        double* foot, double* dlo) {
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != HD_OK) return rc;
  typename P::Vtx* rec = (typename P::Vtx*)base;
  RunState* st = (RunState*)((unsigned char*)base + kNoAllocMaxPoints * 64);
  int* list = (int*)((unsigned char*)base + kNoAllocMaxPoints * 64 + kNoAllocTail);
  HD_TRY(cudaMemsetAsync(st, 0, sizeof(RunState), s));  // counters start at zero every call
  if (ptype == HD_F64)
    k_points_in<P, double><<<blocks_for(n, 256), 256, 0, s>>>((const double*)Pts, n, rec);
  else
    k_points_in<P, float><<<blocks_for(n, 256), 256, 0, s>>>((const float*)Pts, n, rec);
  query_points<P>(bvh_dev(B), rec, n, st, list, s);
  k_points_out<P><<<blocks_for(n, 256), 256, 0, s>>>(rec, n, B->tri_vid, dist, idx, foot, dlo);
  HD_TRY_LAUNCH();
  return HD_OK;
}

}  // namespace
}  // namespace hd

extern "C" int hd_nearest_noalloc(const hd_bvh* B, const void* P, int32_t ptype, int64_t n, int32_t precision,
                                  void* stream, double* dist, int32_t* idx, double* foot, double* dist_lo) {
  using namespace hd;
  if (!B || n < 0 || n > kNoAllocMaxPoints) return HD_ERR_INVALID;
  if (n > 0 && (!P || !dist || !idx || !foot)) return HD_ERR_INVALID;
  if ((ptype != HD_F32 && ptype != HD_F64) || (precision != HD_FP64 && precision != HD_MIXED)) return HD_ERR_INVALID;
  int dev = -1;
  HD_TRY(cudaGetDevice(&dev));
  if (dev != B->device) return HD_ERR_INVALID;
  if (n == 0) return HD_OK;
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == HD_FP64) return run<PolicyD>(B, P, ptype, n, s, dist, idx, foot, dist_lo);
  return run<PolicyM>(B, P, ptype, n, s, dist, idx, foot, dist_lo);
}
