// The C ABI of include/hd.h: options, validation, dispatch to the FP64 or certified FP32
// branch-and-bound, and the step-level entry points used for parity checks.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "hd_batch.cuh"
#include "hd_bnb.cuh"
#include "hd_fp64.cuh"

namespace hd {

static thread_local char g_err[512] = "";

int set_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_err, sizeof g_err, "%s: %s (%s:%d)", cudaGetErrorString(e), what, file, line);
  return HD_ERR_CUDA;
}

// ----------------------------------------------------------------------------- kernel trace

namespace {
struct Pending {
  int kind;
  cudaEvent_t a, b;
};
struct Trace {
  std::mutex m;
  bool on = false;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> free_events;
  int64_t launches[8] = {};
  double ms[8] = {};
  cudaEvent_t get() {
    if (!free_events.empty()) {
      cudaEvent_t e = free_events.back();
      free_events.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void resolve() {  // caller holds m
    for (auto& p : pending) {
      float t = 0.f;
      if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
        launches[p.kind] += 1;
        ms[p.kind] += t;
      }
      free_events.push_back(p.a);
      free_events.push_back(p.b);
    }
    pending.clear();
  }
};
Trace& trace() {
  static Trace* t = new Trace();  // never destroyed: events may outlive static destruction order
  return *t;
}
}  // namespace

TraceScope::TraceScope(int k, cudaStream_t st) : kind(k), s(st) {
  Trace& t = trace();
  std::lock_guard<std::mutex> g(t.m);
  if (!t.on) return;
  a = t.get();
  b = t.get();
  if (a) cudaEventRecord(a, s);
}

TraceScope::~TraceScope() {
  if (!a || !b) return;
  Trace& t = trace();
  std::lock_guard<std::mutex> g(t.m);
  cudaEventRecord(b, s);
  t.pending.push_back({kind, a, b});
  if (t.pending.size() > 4096) t.resolve();
}

int resolve_options(const hd_options* in, Opts* o) {
  hd_options d;
  hd_options_default(&d);
  const hd_options& x = in ? *in : d;
  o->tol_mode = x.tol_mode;
  o->precision = x.precision;
  o->max_face_factor = x.max_face_factor;
  o->frontier_chunk = x.frontier_chunk;
  o->leaf_size = x.leaf_size;
  o->block_size = x.block_size;
  o->n_bounds = x.n_bounds;
  o->max_rounds = x.max_rounds;
  o->max_frontier_bytes = x.max_frontier_bytes;
  memcpy(o->order, x.bound_order, 4);
  o->flags = x.flags;
  if (x.reserved != 0 || (o->flags & ~(int)(HD_FLAG_NO_PARENT_CLAMP | HD_FLAG_ASYNC_BUILD | HD_FLAG_SHARE_MIDPOINTS | HD_FLAG_WELD_B |
                                      HD_FLAG_NO_SMALL_ROUNDS | HD_FLAG_BATCH_STREAMS | HD_FLAG_EXACT_QUERIES))) return HD_ERR_INVALID;
  if (o->tol_mode != HD_TOL_ABS && o->tol_mode != HD_TOL_REL) return HD_ERR_INVALID;
  if (o->precision != HD_FP64 && o->precision != HD_MIXED) return HD_ERR_INVALID;
  if (!(o->max_face_factor >= 1.0)) return HD_ERR_INVALID;
  if (o->leaf_size < 1 || o->leaf_size > 16) return HD_ERR_INVALID;
  if (o->block_size < 32 || o->block_size > 1024 || o->block_size % 32) return HD_ERR_INVALID;
  if (o->n_bounds < 1 || o->n_bounds > 4) return HD_ERR_INVALID;
  for (int k = 0; k < o->n_bounds; ++k)
    if (o->order[k] < 1 || o->order[k] > 4) return HD_ERR_INVALID;
  if (o->max_rounds < 1 || o->frontier_chunk < 0 || o->max_frontier_bytes < 0) return HD_ERR_INVALID;
  return HD_OK;
}

static int check_mesh(const hd_mesh* m) {
  if (!m || !m->V || !m->F || m->nV <= 0 || m->nF <= 0) return HD_ERR_INVALID;
  if (m->vtype != HD_F32 && m->vtype != HD_F64) return HD_ERR_INVALID;
  if (m->nV > INT32_MAX / 2 || m->nF > INT32_MAX / 4) return HD_ERR_INVALID;
  return HD_OK;
}

// The default stream-ordered pool keeps freed blocks, so the per-call work buffers are not
// returned to the driver between calls.
static void keep_pool_memory() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  static bool done[64] = {};
  if (dev < 64 && !done[dev]) {
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done[dev] = true;
  }
}

int run_fp64(const RunIO& io) { return run_bnb<PolicyD>(io); }
int run_mixed(const RunIO& io);
int run_batch_mixed(const hd_bvh* const* Bs, const hd_mesh* As, int64_t npairs, double tol, const Opts& o,
                    cudaStream_t s, hd_result* outs, std::vector<int64_t>* redo);

int nearest_points_fp64(const hd_bvh* B, const void* Pts, int ptype, int64_t n, cudaStream_t s, double* dist,
                        int32_t* idx, double* foot, double* dlo) {
  return nearest_points<PolicyD>(B, Pts, ptype, n, s, dist, idx, foot, dlo);
}
int nearest_points_mixed(const hd_bvh* B, const void* Pts, int ptype, int64_t n, cudaStream_t s, double* dist,
                         int32_t* idx, double* foot, double* dlo);
int upper_bounds_mixed(const hd_bvh* B, const double* T, const double* Td, const int32_t* TI, const double* Tq,
                       int64_t n, double l, const RunParams& rp, cudaStream_t s, double* U, int32_t* code);

__global__ void k_upper_bounds(BvhDev B, const int* inv, const double* T, const double* Td, const int32_t* TI,
                               const double* Tq, int64_t n, double l, RunParams rp, double* U, int32_t* code) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  VI t[3];
  for (int k = 0; k < 3; ++k) {
    const double* v = T + 9 * i + 3 * k;
    const double* q = Tq + 9 * i + 3 * k;
    int I = TI[3 * i + k];
    if (I < 0 || I >= B.nF) {  // not a triangle of B: no bound
      U[i] = NAN;
      code[i] = -1;
      return;
    }
    t[k] = {{v[0], v[1], v[2]}, Td[3 * i + k], inv[I], {q[0], q[1], q[2]}};
  }
  unsigned ev = 0;
  int c;
  U[i] = upper_bound_d(B, t, l, rp.order, rp.n_bounds, c, ev);
  code[i] = c;
}

}  // namespace hd

using namespace hd;

// The stream and event that host arrays of A go up with, one pair per host thread and device
// (created once, kept for the process): the copy then overlaps what the caller queued before
// the call (B's asynchronous build, say), and the caller's stream waits for the event.
static int upload_stream(int dev, cudaStream_t* up, cudaEvent_t* ev) {
  static thread_local cudaStream_t st[64] = {};
  static thread_local cudaEvent_t evs[64] = {};
  if (dev < 0 || dev >= 64) return HD_ERR_INVALID;
  if (!st[dev]) HD_TRY(cudaStreamCreateWithFlags(&st[dev], cudaStreamNonBlocking));
  if (!evs[dev]) HD_TRY(cudaEventCreateWithFlags(&evs[dev], cudaEventDisableTiming));
  *up = st[dev];
  *ev = evs[dev];
  return HD_OK;
}

// One-sided h(A, B) with l starting at l0 (a known lower bound of the quantity bracketed).
static int hausdorff_one(const hd_bvh* B, const hd_mesh* A, double tol, const hd_options* opt, void* stream,
                         hd_result* out, double l0) {
  if (!out) return HD_ERR_INVALID;
  memset(out, 0, sizeof *out);
  out->status = HD_ERR_INVALID;
  Opts o;
  if (!B || !(tol > 0.0) || !(l0 >= 0.0) || resolve_options(opt, &o) != HD_OK || check_mesh(A) != HD_OK)
    return HD_ERR_INVALID;
  int dev = -1;
  HD_TRY(cudaGetDevice(&dev));
  if (dev != B->device) return HD_ERR_INVALID;
  keep_pool_memory();
  cudaStream_t s = (cudaStream_t)stream;
  const size_t vbytes = (size_t)A->nV * 3 * (A->vtype == HD_F64 ? 8 : 4);
  const void* VA = A->V;
  const int32_t* FA = A->F;
  void* Vtmp = nullptr;
  int32_t* Ftmp = nullptr;
  if (!A->on_device) {
    // on the upload stream (the stream-ordered frees below, on s, follow the wait)
    cudaStream_t up = s;
    cudaEvent_t ev = nullptr;
    if (upload_stream(dev, &up, &ev) != HD_OK) {
      up = s;
      ev = nullptr;
    }
    HD_TRY(cudaMallocAsync(&Vtmp, vbytes, up));
    HD_TRY(cudaMallocAsync((void**)&Ftmp, (size_t)A->nF * 12, up));
    HD_TRY(cudaMemcpyAsync(Vtmp, A->V, vbytes, cudaMemcpyHostToDevice, up));
    HD_TRY(cudaMemcpyAsync(Ftmp, A->F, (size_t)A->nF * 12, cudaMemcpyHostToDevice, up));
    if (ev) {
      HD_TRY(cudaEventRecord(ev, up));
      HD_TRY(cudaStreamWaitEvent(s, ev, 0));
    }
    VA = Vtmp;
    FA = Ftmp;
  }
  RunIO io{B, VA, A->vtype, A->nV, FA, A->nF, tol, &o, s, out, l0};
  int rc = o.precision == HD_FP64 ? run_fp64(io) : run_mixed(io);
  if (Vtmp) cudaFreeAsync(Vtmp, s);
  if (Ftmp) cudaFreeAsync(Ftmp, s);
  if (rc != HD_OK) {
    out->status = rc;
    return rc;
  }
  return HD_OK;
}

// Pairs `todo` as independent single runs.  Pairs are independent: host threads, each with
// its own non-blocking stream, take pairs in turn, so that the kernels of several small pairs
// share the GPU (two threads per host core, 8 to 64: each thread spends much of a pair
// waiting for its stream).  The streams start after the work queued so far on the caller's
// stream; every pair is complete when the call returns.
static int streams_batch(const hd_bvh* const* Bs, const hd_mesh* As, const std::vector<int64_t>& todo, double tol,
                         const hd_options* opt, void* stream, hd_result* outs, int dev) {
  const int64_t npairs = (int64_t)todo.size();
  const unsigned cores = std::max(1u, std::thread::hardware_concurrency());
  const int streams = (int)std::min(64u, std::max(8u, 2 * cores));
  const int nw = (int)std::min<int64_t>(npairs, streams);
  cudaEvent_t start;
  HD_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  cudaError_t e = cudaEventRecord(start, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    cudaEventDestroy(start);
    return set_cuda_error(e, "cudaEventRecord", __FILE__, __LINE__);
  }
  std::atomic<int64_t> next{0};
  std::atomic<int> fail{HD_OK};
  std::mutex em;
  std::string first_err;
  auto work = [&]() {
    cudaStream_t s = nullptr;
    cudaError_t err = cudaSetDevice(dev);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(s, start, 0);
    if (err != cudaSuccess) {
      set_cuda_error(err, "batch stream set-up", __FILE__, __LINE__);
      int ok = HD_OK;
      if (fail.compare_exchange_strong(ok, HD_ERR_CUDA)) {
        std::lock_guard<std::mutex> g(em);
        first_err = g_err;
      }
    }
    while (err == cudaSuccess && fail.load() == HD_OK) {
      const int64_t k = next.fetch_add(1);
      if (k >= npairs) break;
      const int64_t i = todo[k];
      int rc = hausdorff_one(Bs[i], &As[i], tol, opt, s, &outs[i], 0.0);
      if (rc == HD_ERR_INVALID || rc == HD_ERR_CUDA) {
        int ok = HD_OK;
        if (fail.compare_exchange_strong(ok, rc)) {
          std::lock_guard<std::mutex> g(em);
          first_err = g_err;
        }
      }
    }
    if (s) {
      cudaStreamSynchronize(s);
      cudaStreamDestroy(s);
    }
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < nw; ++w) pool.emplace_back(work);
  work();
  for (auto& t : pool) t.join();
  cudaEventDestroy(start);
  if (fail.load() != HD_OK) {
    snprintf(g_err, sizeof g_err, "%s", first_err.c_str());
    return fail.load();
  }
  return HD_OK;
}


extern "C" {

void hd_options_default(hd_options* o) {
  if (!o) return;
  memset(o, 0, sizeof *o);
  o->tol_mode = HD_TOL_ABS;
  o->precision = HD_FP64;
  o->max_face_factor = 1e7;
  o->frontier_chunk = 0;
  o->leaf_size = 1;
  o->block_size = 64;
  o->bound_order[0] = 1;
  o->bound_order[1] = 2;
  o->bound_order[2] = 3;
  o->bound_order[3] = 4;
  o->n_bounds = 4;
  o->max_rounds = 1000000;
  o->max_frontier_bytes = 0;
}

const char* hd_status_str(int s) {
  switch (s) {
    case HD_OK: return "HD_OK";
    case HD_ERR_INVALID: return "HD_ERR_INVALID";
    case HD_ERR_CAPACITY: return "HD_ERR_CAPACITY";
    case HD_ERR_NUMERIC: return "HD_ERR_NUMERIC";
    case HD_ERR_TIMEOUT: return "HD_ERR_TIMEOUT";
    case HD_ERR_CUDA: return "HD_ERR_CUDA";
    default: return "HD_UNKNOWN";
  }
}

const char* hd_last_error(void) { return g_err; }

void hd_trace_enable(int on) {
  Trace& t = trace();
  std::lock_guard<std::mutex> g(t.m);
  t.on = on != 0;
}

int hd_trace_read(hd_trace* out, int reset) {
  if (!out) return HD_ERR_INVALID;
  Trace& t = trace();
  std::lock_guard<std::mutex> g(t.m);
  t.resolve();
  for (int k = 0; k < 8; ++k) {
    out->launches[k] = t.launches[k];
    out->ms[k] = t.ms[k];
  }
  if (reset) {
    memset(t.launches, 0, sizeof t.launches);
    memset(t.ms, 0, sizeof t.ms);
  }
  return HD_OK;
}

int hd_build_B(const hd_mesh* B, const hd_options* opt, void* stream, hd_bvh** out) {
  if (!out) return HD_ERR_INVALID;
  *out = nullptr;
  Opts o;
  if (resolve_options(opt, &o) != HD_OK || check_mesh(B) != HD_OK) return HD_ERR_INVALID;
  if (B->nF >= (int64_t)1 << 27) return HD_ERR_INVALID;  // traversal stack entries pack 27-bit indices
  keep_pool_memory();
  return build_bvh(B, o, (cudaStream_t)stream, out);
}

void hd_free_B(hd_bvh* b) {
  if (!b) return;
  if (b->block) {
    // stream-ordered release on the legacy default stream of the BVH's device: it follows
    // all earlier work on blocking streams; the block returns to the pool, not the driver
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != b->device) cudaSetDevice(b->device);
    cudaFreeAsync(b->block, 0);
    if (cur >= 0 && cur != b->device) cudaSetDevice(cur);
  }
  delete b;
}

int64_t hd_bvh_num_faces(const hd_bvh* b) { return b ? b->nF : 0; }

int hd_hausdorff(const hd_bvh* B, const hd_mesh* A, double tol, const hd_options* opt, void* stream,
                 hd_result* out) {
  return hausdorff_one(B, A, tol, opt, stream, out, 0.0);
}

int hd_hausdorff_from(const hd_bvh* B, const hd_mesh* A, double tol, double l0, const hd_options* opt,
                      void* stream, hd_result* out) {
  return hausdorff_one(B, A, tol, opt, stream, out, l0);
}

int hd_hausdorff_sym(const hd_bvh* bvhB, const hd_mesh* A, const hd_bvh* bvhA, const hd_mesh* B, double tol,
                     const hd_options* opt, void* stream, hd_result* out, hd_result* ab, hd_result* ba) {
  if (!out) return HD_ERR_INVALID;
  memset(out, 0, sizeof *out);
  out->status = HD_ERR_INVALID;
  hd_result rab, rba;
  int rc = hausdorff_one(bvhB, A, tol, opt, stream, &rab, 0.0);
  if (ab) *ab = rab;
  if (rc != HD_OK) return rc;
  // h(B, A) at the same absolute tolerance, with l starting from h(A, B)'s lower bound: a
  // sub-triangle of B whose U is below it cannot raise H = max(h(A, B), h(B, A))
  hd_options o2;
  if (opt) o2 = *opt;
  else hd_options_default(&o2);
  o2.tol_mode = HD_TOL_ABS;
  rc = hausdorff_one(bvhA, B, rab.stats.eps_abs, &o2, stream, &rba, rab.lower);
  if (ba) *ba = rba;
  if (rc != HD_OK) return rc;
  out->lower = std::max(rab.lower, rba.lower);
  out->upper = std::max(rab.upper, rba.upper);
  out->status = rab.status != HD_OK ? rab.status : rba.status;
  hd_stats& S = out->stats;
  const hd_stats &X = rab.stats, &Y = rba.stats;
  S.rounds = X.rounds + Y.rounds;
  S.splits = X.splits + Y.splits;
  S.queries = X.queries + Y.queries;
  S.pointtri_evals = X.pointtri_evals + Y.pointtri_evals;
  S.leaf_tests = X.leaf_tests + Y.leaf_tests;
  S.box_tests = X.box_tests + Y.box_tests;
  for (int k = 0; k < 6; ++k) S.discards[k] = X.discards[k] + Y.discards[k];
  S.retired = X.retired + Y.retired;
  S.fp64_escalations = X.fp64_escalations + Y.fp64_escalations;
  S.peak_frontier = std::max(X.peak_frontier, Y.peak_frontier);
  S.pool_vertices = X.pool_vertices + Y.pool_vertices;
  S.long_queries = X.long_queries + Y.long_queries;
  S.kernel_launches = X.kernel_launches + Y.kernel_launches;
  S.d2h_bytes = X.d2h_bytes + Y.d2h_bytes;
  S.promoted = X.promoted + Y.promoted;
  S.node_visits = X.node_visits + Y.node_visits;
  S.long_node_visits = X.long_node_visits + Y.long_node_visits;
  S.long_leaf_tests = X.long_leaf_tests + Y.long_leaf_tests;
  S.queries_cut = X.queries_cut + Y.queries_cut;
  S.eps_abs = X.eps_abs;
  S.dA = X.dA;
  return HD_OK;
}

int hd_hausdorff_batched(const hd_bvh* const* Bs, const hd_mesh* As, int64_t npairs, double tol,
                         const hd_options* opt, void* stream, hd_result* outs) {
  if (!Bs || !As || !outs || npairs < 0) return HD_ERR_INVALID;
  if (npairs == 0) return HD_OK;
  Opts o;
  if (!(tol > 0.0) || resolve_options(opt, &o) != HD_OK) return HD_ERR_INVALID;
  int dev = -1;
  HD_TRY(cudaGetDevice(&dev));
  int64_t nV = 0, nF = 0;
  for (int64_t i = 0; i < npairs; ++i) {
    if (!Bs[i] || Bs[i]->device != dev || check_mesh(&As[i]) != HD_OK) return HD_ERR_INVALID;
    nV += As[i].nV;
    nF += As[i].nF;
  }
  keep_pool_memory();
  std::vector<int64_t> todo;
  // the batched run: one launch per phase for all pairs (pool indices of all pairs' vertices
  // and the face enumeration must stay well inside int)
  if (!(o.flags & (HD_FLAG_BATCH_STREAMS | HD_FLAG_SHARE_MIDPOINTS)) && npairs <= INT32_MAX / 4 && nV <= INT32_MAX / 8 &&
      nF <= INT32_MAX / 8) {
    for (int64_t i = 0; i < npairs; ++i) {
      memset(&outs[i], 0, sizeof outs[i]);
      outs[i].status = HD_ERR_INVALID;
    }
    const int rc = o.precision == HD_FP64 ? run_batch<PolicyD>(Bs, As, npairs, tol, o, (cudaStream_t)stream, outs, &todo)
                                          : run_batch_mixed(Bs, As, npairs, tol, o, (cudaStream_t)stream, outs, &todo);
    // pairs the batch's shared buffers could not finish run again on their own below
    if (rc != HD_OK || todo.empty()) return rc;
  } else {
    todo.resize(npairs);
    for (int64_t i = 0; i < npairs; ++i) todo[i] = i;
  }
  return streams_batch(Bs, As, todo, tol, opt, stream, outs, dev);
}

int hd_nearest(const hd_bvh* B, const void* P, int32_t ptype, int64_t n, int32_t precision, void* stream,
               double* dist, int32_t* idx, double* foot, double* dist_lo) {
  if (!B || (n > 0 && (!P || !dist || !idx || !foot)) || n < 0) return HD_ERR_INVALID;
  if ((ptype != HD_F32 && ptype != HD_F64) || (precision != HD_FP64 && precision != HD_MIXED)) return HD_ERR_INVALID;
  if (n == 0) return HD_OK;
  keep_pool_memory();
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == HD_FP64) return nearest_points_fp64(B, P, ptype, n, s, dist, idx, foot, dist_lo);
  return nearest_points_mixed(B, P, ptype, n, s, dist, idx, foot, dist_lo);
}

int hd_upper_bounds(const hd_bvh* B, const double* T, const double* Td, const int32_t* TI, const double* Tq,
                    int64_t n, double l, const hd_options* opt, void* stream, double* U, int32_t* code) {
  Opts o;
  if (!B || n < 0 || resolve_options(opt, &o) != HD_OK) return HD_ERR_INVALID;
  if (n == 0) return HD_OK;
  if (!T || !Td || !TI || !Tq || !U || !code) return HD_ERR_INVALID;
  RunParams rp;
  rp.eps = 0.0;
  rp.slack = 0.0;
  rp.slack_f = 0.f;
  rp.defer_u4 = 0;
  rp.parent_clamp = 0;
  memcpy(rp.order, o.order, 4);
  rp.n_bounds = o.n_bounds;
  cudaStream_t s = (cudaStream_t)stream;
  if (o.precision == HD_MIXED) return upper_bounds_mixed(B, T, Td, TI, Tq, n, l, rp, s, U, code);
  k_upper_bounds<<<blocks_for(n, 128), 128, 0, s>>>(bvh_dev(B), B->inv, T, Td, TI, Tq, n, l, rp, U, code);
  HD_TRY_LAUNCH();
  return HD_OK;
}

}  // extern "C"
