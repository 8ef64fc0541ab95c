// K1 -- GPU build of the bounding-volume hierarchy over B.
//
// The paper builds libigl's AABB tree over B once and uses it for all distance queries
// (Section 4).  Here the hierarchy is a linear BVH built on the GPU:
//   1. triangle centroids and their bounding box;
//   2. Morton codes of the centroids, 10 to 16 bits per axis (wider for larger B);
//   3. a stable LSD radix sort of (code, triangle) pairs, 8-bit digits;
//   4. the binary radix tree of Karras (HPG 2012) over the sorted codes, ties broken by
//      position;
//   5. node boxes (float, rounded outward so they contain the exact triangles), each the
//      union of the aligned power-of-two blocks of leaves that tile its range;
//   6. traversal nodes: 128 B each, holding up to four child boxes (a binary node with its
//      grandchildren); subtrees of at most leaf_size triangles become leaf ranges.
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <vector>

#include "hd_internal.cuh"

namespace hd {

namespace {

constexpr int kThreads = 256;
#ifndef HD_GRID_MEMSET
#define HD_GRID_MEMSET 0  // 1: clear the hint grid with cudaMemsetAsync instead of a chained kernel
#endif
#ifndef HD_KEEP_TRI64
#define HD_KEEP_TRI64 0  // 1: keep the FP64 copy of B for float32 input too
#endif

// ---------------------------------------------------------------- 1-2: centroids, Morton codes

template <typename T>
__device__ inline D3 load_vertex(const T* V, int64_t i) {
  return {(double)V[3 * i], (double)V[3 * i + 1], (double)V[3 * i + 2]};
}

// A face's three vertices as doubles, or the origin three times when an index is out of range
// or a coordinate is not finite (B is then invalid and flagged by k_prep; the face becomes a
// point so that the tree stays finite and every later kernel stays in bounds until the flag
// is read).
template <typename T>
__device__ inline bool load_face(const T* V, int64_t nV, const int32_t* F, int64_t f, D3& a, D3& b, D3& c) {
  const int32_t i0 = F[3 * f], i1 = F[3 * f + 1], i2 = F[3 * f + 2];
  a = b = c = {0, 0, 0};
  if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= nV || i1 >= nV || i2 >= nV) return false;
  a = load_vertex(V, i0);
  b = load_vertex(V, i1);
  c = load_vertex(V, i2);
  const bool fin = isfinite(a.x) && isfinite(a.y) && isfinite(a.z) && isfinite(b.x) && isfinite(b.y) &&
                   isfinite(b.z) && isfinite(c.x) && isfinite(c.y) && isfinite(c.z);
  if (!fin) a = b = c = {0, 0, 0};
  return fin;
}

// The same for float input, in float: a float vertex is exact as it is, and FP64 arithmetic
// runs at a small fraction of the FP32 rate on GB300 (the build's per-triangle FP64 work
// dominated its time).
struct F3v {
  float x, y, z;
};
__device__ inline bool load_face_f(const float* V, int64_t nV, const int32_t* F, int64_t f, F3v& a, F3v& b, F3v& c) {
  const int32_t i0 = F[3 * f], i1 = F[3 * f + 1], i2 = F[3 * f + 2];
  a = b = c = {0.f, 0.f, 0.f};
  if (i0 < 0 || i1 < 0 || i2 < 0 || i0 >= nV || i1 >= nV || i2 >= nV) return false;
  a = {V[3 * (int64_t)i0], V[3 * (int64_t)i0 + 1], V[3 * (int64_t)i0 + 2]};
  b = {V[3 * (int64_t)i1], V[3 * (int64_t)i1 + 1], V[3 * (int64_t)i1 + 2]};
  c = {V[3 * (int64_t)i2], V[3 * (int64_t)i2 + 1], V[3 * (int64_t)i2 + 2]};
  const bool fin = isfinite(a.x) && isfinite(a.y) && isfinite(a.z) && isfinite(b.x) && isfinite(b.y) &&
                   isfinite(b.z) && isfinite(c.x) && isfinite(c.y) && isfinite(c.z);
  if (!fin) a = b = c = {0.f, 0.f, 0.f};
  return fin;
}

// Validation, the centroids and their bounding box.  Grid-stride, so that the box is reduced
// per thread, then per block, and ends in one atomic per block and bound.  The centroids only
// order the triangles (Morton codes), so float input keeps them in float.
template <typename T>
__global__ void k_prep(const T* V, int64_t nV, const int32_t* F, int64_t nF, float4* cent,
                       unsigned* cbox /*6 ordered floats: min xyz (as ~max), max xyz*/, int* bad) {
  grid_dep_wait();
  grid_dep_launch();
  __shared__ float part[6][kThreads / 32];
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nF; f += (int64_t)gridDim.x * blockDim.x) {
    float mx, my, mz;
    if constexpr (std::is_same<T, float>::value) {
      F3v a, b, c;
      if (!load_face_f(V, nV, F, f, a, b, c)) {
        atomicExch(bad, 1);
        cent[f] = make_float4(0.f, 0.f, 0.f, 0.f);
        continue;
      }
      mx = (a.x + b.x + c.x) * (1.f / 3.f);
      my = (a.y + b.y + c.y) * (1.f / 3.f);
      mz = (a.z + b.z + c.z) * (1.f / 3.f);
    } else {
      D3 a, b, c;
      if (!load_face(V, nV, F, f, a, b, c)) {
        atomicExch(bad, 1);
        cent[f] = make_float4(0.f, 0.f, 0.f, 0.f);
        continue;
      }
      const D3 m = (1.0 / 3.0) * (a + b + c);
      mx = (float)m.x;
      my = (float)m.y;
      mz = (float)m.z;
    }
    lo[0] = fminf(lo[0], mx);
    lo[1] = fminf(lo[1], my);
    lo[2] = fminf(lo[2], mz);
    hi[0] = fmaxf(hi[0], mx);
    hi[1] = fmaxf(hi[1], my);
    hi[2] = fmaxf(hi[2], mz);
    cent[f] = make_float4(mx, my, mz, 0.f);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
      hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
    }
    if (lane == 0) {
      part[k][w] = lo[k];
      part[3 + k][w] = hi[k];
    }
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int k = threadIdx.x;
    float r = k < 3 ? INFINITY : -INFINITY;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) r = k < 3 ? fminf(r, part[k][q]) : fmaxf(r, part[k][q]);
    if (isfinite(r)) {
      if (k < 3) atomicMin(&cbox[k], float_to_ordered(r));
      else atomicMax(&cbox[k], float_to_ordered(r));
    }
  }
}

__device__ inline uint64_t spread16(uint32_t v) {  // 16 bits -> every third bit of 48
  uint64_t x = v & 0xffffu;
  x = (x | (x << 16)) & 0x0000ff0000ffull;
  x = (x | (x << 8)) & 0x00f00f00f00full;
  x = (x | (x << 4)) & 0x0c30c30c30c3ull;
  x = (x | (x << 2)) & 0x249249249249ull;
  return x;
}

// Also zeroes the `ntot` digit totals of the sort passes that follow.
__global__ void k_morton(const float4* cent, int64_t nF, const unsigned* cbox, int bits, int drop, uint64_t* keys,
                         uint32_t* vals, unsigned* tot, int ntot) {
  grid_dep_wait();
  grid_dep_launch();
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t i = f; i < ntot; i += (int64_t)gridDim.x * blockDim.x) tot[i] = 0u;
  if (f >= nF) return;
  const float cells = (float)(1u << bits);
  float4 c = cent[f];
  float cc[3] = {c.x, c.y, c.z};
  uint32_t q[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float lo = ordered_to_float(cbox[k]), hi = ordered_to_float(cbox[3 + k]);
    float ext = hi - lo;
    float u = ext > 0.f ? (cc[k] - lo) * (cells / ext) : 0.5f * cells;
    q[k] = (uint32_t)fminf(fmaxf(u, 0.f), cells - 1.f);
  }
  keys[f] = ((spread16(q[0]) << 2) | (spread16(q[1]) << 1) | spread16(q[2])) >> drop;
  vals[f] = (uint32_t)f;
}

// ---------------------------------------------------------------- 3: stable LSD radix sort

// A block sorts a tile of RS_THREADS * ROUNDS keys; warp w owns ROUNDS * 32 consecutive keys.
// Small inputs use 4 rounds (1024-key tiles) so that more blocks share the work.
constexpr int RS_WARPS = 8, RS_THREADS = RS_WARPS * 32;

// Per-block digit counts: digit-major (hist[d * nblocks + b], scanned by k_rs_scan_digits) or, for
// the fused small-input path, block-major (hist[b * 256 + d], read by every scatter block).
// With `tot` (non-fused path), the block's counts are also added to the pass's digit totals.
template <int ROUNDS, bool FUSED>
__global__ void k_rs_hist(const uint64_t* keys, int64_t n, int shift, unsigned* hist, int nblocks, unsigned* tot) {
  grid_dep_wait();
  grid_dep_launch();
  constexpr int RS_TILE = RS_THREADS * ROUNDS;
  __shared__ unsigned cnt[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * RS_TILE;
  for (int k = threadIdx.x; k < RS_TILE; k += blockDim.x) {
    int64_t i = base + k;
    if (i < n) atomicAdd(&cnt[(keys[i] >> shift) & 0xff], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) {
    if (FUSED) {
      hist[(int64_t)blockIdx.x * 256 + d] = cnt[d];
    } else {
      hist[(int64_t)d * nblocks + blockIdx.x] = cnt[d];
      if (cnt[d]) atomicAdd(&tot[d], cnt[d]);
    }
  }
}

// Largest block count of the fused path: each scatter block then reads all nblocks x 256
// counts itself instead of waiting for a separate scan launch.
constexpr int RS_FUSED_MAX_BLOCKS = 64;
#ifndef HD_RS_ROUNDS
#define HD_RS_ROUNDS 8
#endif
// rounds per warp of the large-input tiles (RS_THREADS * RS_BIG keys); on 2M triangles 8 rounds
// built B in 0.566 ms against 0.586 ms with 16
constexpr int RS_BIG = HD_RS_ROUNDS;
constexpr int kMaxSortPasses = 6;  // 3 x 16-bit Morton keys, 8 bits per pass

// The scatter offsets of one pass, one block per digit d (256 blocks of 256 threads): the
// exclusive scan of digit d's per-block counts (hist[d * nblocks + b], contiguous), plus the
// keys of all smaller digits (the sum of the pass's totals below d).
__global__ void k_rs_scan_digits(unsigned* hist, int nblocks, const unsigned* tot) {
  grid_dep_wait();
  grid_dep_launch();
  __shared__ unsigned wsum[8];
  __shared__ unsigned s_base;
  const int d = blockIdx.x, t = threadIdx.x, w = t >> 5, lane = t & 31;
  // keys of smaller digits
  unsigned x = t < d ? tot[t] : 0u;
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if (lane == 0) wsum[w] = x;
  __syncthreads();
  if (t == 0) {
    unsigned b = 0;
    for (int k = 0; k < 8; ++k) b += wsum[k];
    s_base = b;
  }
  __syncthreads();
  unsigned carry = s_base;
  unsigned* a = hist + (int64_t)d * nblocks;
  for (int c0 = 0; c0 < nblocks; c0 += 256) {
    const int i = c0 + t;
    const unsigned v = i < nblocks ? a[i] : 0u;
    unsigned y = v;  // inclusive warp scan
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned z = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += z;
    }
    __syncthreads();  // wsum is free again
    if (lane == 31) wsum[w] = y;
    __syncthreads();
    unsigned before = 0, all = 0;
    for (int k = 0; k < 8; ++k) {
      before += k < w ? wsum[k] : 0u;
      all += wsum[k];
    }
    if (i < nblocks) a[i] = carry + before + y - v;
    carry += all;
  }
}

// The keys of a tile go first to shared memory in the tile's digit order (each key at its
// digit's block-local start + its warp's offset + its rank in the warp), then out to global
// memory from there, so that consecutive threads write consecutive addresses of one digit's
// run: writing each key straight from its lane scattered 8- and 4-byte stores over up to 256
// runs (several times the bytes in partly written sectors).  Dynamic shared memory: 12 bytes
// per key of the tile.
template <int ROUNDS>
constexpr size_t rs_scatter_smem() {
  return (size_t)RS_THREADS * ROUNDS * (sizeof(uint64_t) + sizeof(uint32_t));
}

template <int ROUNDS, bool FUSED>
__global__ void k_rs_scatter(const uint64_t* kin, const uint32_t* vin, uint64_t* kout, uint32_t* vout, int64_t n,
                             int shift, const unsigned* hist, int nblocks) {
  grid_dep_wait();
  grid_dep_launch();
  constexpr int RS_TILE = RS_THREADS * ROUNDS;
  static_assert(RS_THREADS == 256, "one digit per thread");
  extern __shared__ __align__(16) unsigned char rs_smem[];
  uint64_t* sk = reinterpret_cast<uint64_t*>(rs_smem);
  uint32_t* sv = reinterpret_cast<uint32_t*>(rs_smem + sizeof(uint64_t) * RS_TILE);
  __shared__ unsigned wcnt[RS_WARPS][256];
  __shared__ unsigned doff[256];  // where this block's keys of digit d start in the output
  __shared__ unsigned lofs[256];  // where they start in the tile's digit order
  __shared__ unsigned wsum[RS_WARPS];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (FUSED) {
    // all keys of smaller digits, plus the keys of digit d in earlier blocks
    const int d = threadIdx.x;
    unsigned tot = 0, mine = 0;
    for (int b = 0; b < nblocks; ++b) {
      unsigned c = hist[(int64_t)b * 256 + d];
      tot += c;
      mine += b < (int)blockIdx.x ? c : 0u;
    }
    unsigned x = tot;  // inclusive warp scan, then across the 8 warps
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    unsigned before = 0;
    for (int k = 0; k < w; ++k) before += wsum[k];
    doff[d] = before + x - tot + mine;
  } else {
    doff[threadIdx.x] = hist[(int64_t)threadIdx.x * nblocks + blockIdx.x];
  }
  for (int i = lane; i < 256; i += 32) wcnt[w][i] = 0;
  __syncwarp();
  const unsigned lt = (1u << lane) - 1u;
  const int64_t tile0 = (int64_t)blockIdx.x * RS_TILE;
  const int64_t base = tile0 + w * (RS_TILE / RS_WARPS);
  unsigned rank[ROUNDS];
  uint64_t key[ROUNDS];
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    int64_t i = base + r * 32 + lane;
    bool valid = i < n;
    key[r] = valid ? kin[i] : 0ull;
    unsigned dig = valid ? (unsigned)((key[r] >> shift) & 0xff) : 256u + lane;  // invalid lanes match only themselves
    unsigned peers = __match_any_sync(0xffffffffu, dig);
    unsigned before = __popc(peers & lt);
    unsigned c = valid ? wcnt[w][dig] : 0;
    __syncwarp();
    if (valid && before == 0) wcnt[w][dig] = c + __popc(peers);
    __syncwarp();
    rank[r] = c + before;
  }
  __syncthreads();
  // per digit (one per thread): the warps' offsets (exclusive over warps), then the digit's
  // start in the tile (exclusive scan of the block's digit totals)
  {
    const int d = threadIdx.x;
    unsigned run = 0;
    for (int k = 0; k < RS_WARPS; ++k) {
      unsigned v = wcnt[k][d];
      wcnt[k][d] = run;
      run += v;
    }
    unsigned x = run;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;  // (the fused offsets above read wsum before the last barrier)
    __syncthreads();
    unsigned before = 0;
    for (int k = 0; k < w; ++k) before += wsum[k];
    lofs[d] = before + x - run;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < ROUNDS; ++r) {
    int64_t i = base + r * 32 + lane;
    if (i < n) {
      unsigned dig = (unsigned)((key[r] >> shift) & 0xff);
      unsigned loc = lofs[dig] + wcnt[w][dig] + rank[r];
      sk[loc] = key[r];
      sv[loc] = vin[i];
    }
  }
  __syncthreads();
  const int cnt = (int)min((int64_t)RS_TILE, n - tile0);
  for (int j = threadIdx.x; j < cnt; j += RS_THREADS) {
    const uint64_t k = sk[j];
    const unsigned dig = (unsigned)((k >> shift) & 0xff);
    const unsigned pos = doff[dig] + (unsigned)j - lofs[dig];
    kout[pos] = k;
    vout[pos] = sv[j];
  }
}

// Dynamic shared memory above the default 48 KB for the large-tile scatter, once per device.
template <bool FUSED>
cudaError_t rs_scatter_attr() {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_relaxed) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(k_rs_scatter<RS_BIG, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)rs_scatter_smem<RS_BIG>());
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_relaxed);
  return e;
}

// ---------------------------------------------------------------- weld (option): one id per position

__device__ inline unsigned long long mix64(unsigned long long z) {  // the SplitMix64 finaliser
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// canon[i] = the index of one vertex with exactly the position of vertex i (the same for all
// of them): vertices are inserted into an open-addressing table keyed by their coordinates;
// the first to claim an entry represents its position.  -0 and +0 are the same position.
// table: 2^k ints, zeroed, at least twice the vertices (so a probe always ends).
template <typename T>
__global__ void k_weld(const T* V, int64_t nV, int* table, unsigned long long mask, int* canon) {
  grid_dep_wait();
  grid_dep_launch();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nV) return;
  const double x = (double)V[3 * i] + 0.0, y = (double)V[3 * i + 1] + 0.0, z = (double)V[3 * i + 2] + 0.0;
  unsigned long long h = mix64((unsigned long long)__double_as_longlong(x) ^
                               mix64((unsigned long long)__double_as_longlong(y) ^
                                     mix64((unsigned long long)__double_as_longlong(z))));
  h &= mask;
  int id = (int)i;
  for (unsigned long long probe = 0; probe <= mask; ++probe) {
    const int prev = atomicCAS(&table[h], 0, (int)i + 1);
    if (prev == 0) break;  // this vertex represents its position
    const int64_t j = prev - 1;
    if ((double)V[3 * j] == x && (double)V[3 * j + 1] == y && (double)V[3 * j + 2] == z) {
      id = (int)j;
      break;
    }
    h = (h + 1) & mask;
  }
  canon[i] = id;
}

// ---------------------------------------------------------------- 4: sorted triangles, leaf boxes

__device__ inline float rd(double x) { return __double2float_rd(x); }
__device__ inline float ru(double x) { return __double2float_ru(x); }

template <typename T>
__global__ void k_gather(const T* V, const int32_t* F, const uint32_t* order, int64_t nF, const int* canon, int64_t nV,
                         double* tri64, float4* tri32, int4* tri_vid, int* inv, float4* leafbox /*2 per leaf*/,
                         unsigned* e2_bits) {
  grid_dep_wait();
  grid_dep_launch();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double e2 = 0.0;  // squared distance between a float vertex and its input vertex
  if (i < nF) {
    uint32_t f = order[i];
    double* t = tri64 ? tri64 + 9 * i : nullptr;  // null: float32 input, not kept
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float4 out[3];
    if constexpr (std::is_same<T, float>::value) {
      // float input is its own float copy: no rounding, eta = 0, no FP64 arithmetic
      F3v a, b, c;
      load_face_f(V, nV, F, f, a, b, c);
      const float s[9] = {a.x, a.y, a.z, b.x, b.y, b.z, c.x, c.y, c.z};
      for (int v = 0; v < 3; ++v) {
        for (int k = 0; k < 3; ++k) {
          const float x = s[3 * v + k];
          if (t) t[3 * v + k] = (double)x;
          lo[k] = fminf(lo[k], x);
          hi[k] = fmaxf(hi[k], x);
        }
        out[v] = make_float4(s[3 * v], s[3 * v + 1], s[3 * v + 2], 0.0f);
      }
    } else {
      D3 a, b, c;
      load_face(V, nV, F, f, a, b, c);
      const double s[9] = {a.x, a.y, a.z, b.x, b.y, b.z, c.x, c.y, c.z};
      for (int v = 0; v < 3; ++v) {
        float c[3];
        for (int k = 0; k < 3; ++k) {
          double x = s[3 * v + k];
          if (t) t[3 * v + k] = x;
          lo[k] = fminf(lo[k], rd(x));
          hi[k] = fmaxf(hi[k], ru(x));
          c[k] = (float)x;
        }
        // x - float(x) is exact in double
        double ex = s[3 * v] - c[0], ey = s[3 * v + 1] - c[1], ez = s[3 * v + 2] - c[2];
        e2 = fmax(e2, ex * ex + ey * ey + ez * ez);
        out[v] = make_float4(c[0], c[1], c[2], 0.0f);
      }
    }
    out[0].w = __int_as_float((int)f);
    tri32[3 * i] = out[0];
    tri32[3 * i + 1] = out[1];
    tri32[3 * i + 2] = out[2];
    // vertex ids for the adjacency of u3 (welded ids with canon; an index out of range makes
    // B invalid and is kept as it is)
    int id[3];
    for (int v = 0; v < 3; ++v) {
      const int k = F[3 * f + v];
      id[v] = canon && k >= 0 && k < nV ? canon[k] : k;
    }
    tri_vid[i] = make_int4(id[0], id[1], id[2], (int)f);
    inv[f] = (int)i;
    leafbox[2 * i] = make_float4(lo[0], lo[1], lo[2], 0.0f);
    leafbox[2 * i + 1] = make_float4(hi[0], hi[1], hi[2], 0.0f);
  }
  if constexpr (!std::is_same<T, float>::value) {
    // the largest squared error, rounded up (the host takes its square root): the squares and
    // their sum carry at most 3 * 2^-53 relative error, covered by the margin
    float e2f = __double2float_ru(e2 * (1.0 + 1e-12));
    for (int o = 16; o > 0; o >>= 1) e2f = fmaxf(e2f, __shfl_xor_sync(0xffffffffu, e2f, o));
    if ((threadIdx.x & 31) == 0 && e2f > 0.0f) atomicMax(e2_bits, __float_as_uint(e2f));
  }
}

// ---------------------------------------------------------------- 5: Karras binary radix tree

__device__ inline int delta(const uint64_t* k, int64_t n, int64_t i, int64_t j) {
  if (j < 0 || j >= n) return -1;
  uint64_t a = k[i], b = k[j];
  if (a == b) return 64 + __clz((int)(uint32_t)(i ^ j));
  return __clzll((long long)(a ^ b));
}

// Internal node i covers the sorted range [first, last]; its children are encoded as
// c >= 0 internal, c < 0 leaf ~c.
__global__ void k_karras(const uint64_t* keys, int64_t n, int* left, int* right, int* first, int* last) {
  grid_dep_wait();
  grid_dep_launch();
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  int d = delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1) >= 0 ? 1 : -1;
  int dmin = delta(keys, n, i, i - d);
  int64_t lmax = 2;
  while (delta(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
  int64_t l = 0;
  for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
    if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
  int64_t j = i + l * d;
  int dnode = delta(keys, n, i, j);
  int64_t s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  int64_t g = i + s * d + (d < 0 ? -1 : 0);
  int64_t lo = i < j ? i : j, hi = i < j ? j : i;
  int cl = (lo == g) ? ~(int)g : (int)g;
  int cr = (hi == g + 1) ? ~(int)(g + 1) : (int)(g + 1);
  left[i] = cl;
  right[i] = cr;
  first[i] = (int)lo;
  last[i] = (int)hi;
}

__device__ inline void load_box(const float4* b, float lo[3], float hi[3]) {
  float4 a = __ldcg(b), c = __ldcg(b + 1);
  lo[0] = a.x; lo[1] = a.y; lo[2] = a.z;
  hi[0] = c.x; hi[1] = c.y; hi[2] = c.z;
}

// Traversal reference of child c: a leaf range (first triangle, count <= L) or an inner
// node (index, count 0).
__device__ inline void child_meta(int c, const int* first, const int* last, int L, int& ref, int& cnt) {
  if (c < 0) {
    ref = ~c;
    cnt = 1;
    return;
  }
  int sz = last[c] - first[c] + 1;
  if (sz <= L) {
    ref = first[c];
    cnt = sz;
  } else {
    ref = c;
    cnt = 0;
  }
}

// Slots 2j, 2j + 1 of a 4-wide node from binary child c: c's two children when c is an inner
// node that is split further (covers more than L triangles), else c itself as a leaf range
// and an empty slot.  cbox is c's box; the children's boxes are read from ibox / leafbox.
__device__ inline void wide_slots(int c, const float clo[3], const float chi[3], const int* left, const int* right,
                                  const int* first, const int* last, int L, const float4* leafbox,
                                  const float4* ibox, float lo[2][3], float hi[2][3], unsigned code[2],
                                  unsigned rep[2]) {
  const bool expand = c >= 0 && last[c] - first[c] + 1 > L;
  if (!expand) {
    int r, k;
    child_meta(c, first, last, L, r, k);
    code[0] = node_code(r, k);
    code[1] = kNoChild;
    rep[0] = (unsigned)(c >= 0 ? first[c] : ~c);
    rep[1] = 0u;
    for (int a = 0; a < 3; ++a) {
      lo[0][a] = clo[a];
      hi[0][a] = chi[a];
      lo[1][a] = INFINITY;
      hi[1][a] = -INFINITY;
    }
    return;
  }
  const int g[2] = {left[c], right[c]};
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    int r, k;
    child_meta(g[j], first, last, L, r, k);
    code[j] = node_code(r, k);
    rep[j] = (unsigned)(g[j] >= 0 ? first[g[j]] : ~g[j]);
    load_box(g[j] >= 0 ? ibox + 2 * g[j] : leafbox + 2 * (int64_t)(~g[j]), lo[j], hi[j]);
  }
}

// Boxes of aligned blocks of leaves: level k holds count[k] = ceil(n / 2^k) boxes, box i of
// level k covering leaves [i 2^k, (i + 1) 2^k) (level 0: the leaf boxes themselves).  Any
// node's range [first, last] is then the union of at most 2 log2(n) such blocks, so every
// node's box is found independently (k_node_box) instead of through a bottom-up chain of
// dependent steps as long as the tree is deep.
struct LevelOffsets {
  int off[32];    // first box of level k in the level array (k >= 1)
  int count[32];  // boxes at level k
  int levels;     // the top level (count 1)
};

// Levels k0 + 1 .. k0 + 8 from the m boxes of level k0 at `in`: a block of 256 threads
// reduces 256 consecutive boxes pairwise in shared memory.
__global__ void k_levels(const float4* in, int m, float4* lv, LevelOffsets L, int k0) {
  grid_dep_wait();
  grid_dep_launch();
  __shared__ float sb[6][256];
  const int t = threadIdx.x;
  const int i = blockIdx.x * 256 + t;
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  if (i < m) load_box(in + 2 * (int64_t)i, lo, hi);
  for (int a = 0; a < 3; ++a) {
    sb[a][t] = lo[a];
    sb[3 + a][t] = hi[a];
  }
  for (int j = 1; j <= 8 && k0 + j <= L.levels; ++j) {
    const int width = 256 >> j, k = k0 + j;
    __syncthreads();
    float u[6];
    if (t < width)
      for (int a = 0; a < 3; ++a) {
        u[a] = fminf(sb[a][2 * t], sb[a][2 * t + 1]);
        u[3 + a] = fmaxf(sb[3 + a][2 * t], sb[3 + a][2 * t + 1]);
      }
    __syncthreads();
    if (t < width) {
      for (int a = 0; a < 6; ++a) sb[a][t] = u[a];
      const int g = blockIdx.x * width + t;
      if (g < L.count[k]) {
        lv[2 * ((int64_t)L.off[k] + g)] = make_float4(u[0], u[1], u[2], 0.f);
        lv[2 * ((int64_t)L.off[k] + g) + 1] = make_float4(u[3], u[4], u[5], 0.f);
      }
    }
  }
}

// The box of every inner node, as the union of the aligned blocks that tile its range.
__global__ void k_node_box(int64_t n, const int* first, const int* last, const float4* leafbox, const float4* lv,
                           LevelOffsets L, float4* ibox) {
  grid_dep_wait();
  grid_dep_launch();
  int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (x >= n - 1) return;
  int f = first[x];
  const int l = last[x];
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  while (f <= l) {
    // the largest aligned block that starts at f and ends by l
    const int align = f ? __ffs(f) - 1 : 30, span = 31 - __clz(l - f + 1);
    const int k = min(min(align, span), L.levels);
    float a[3], b[3];
    load_box(k ? lv + 2 * ((int64_t)L.off[k] + (f >> k)) : leafbox + 2 * (int64_t)f, a, b);
    for (int c = 0; c < 3; ++c) {
      lo[c] = fminf(lo[c], a[c]);
      hi[c] = fmaxf(hi[c], b[c]);
    }
    f += 1 << k;
  }
  ibox[2 * x] = make_float4(lo[0], lo[1], lo[2], 0.f);
  ibox[2 * x + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
}

// The 128-byte traversal node of every inner node covering more than L triangles: its
// children, or their children where those are split further, so that the nodes reached from
// the root skip every other level of the binary tree.  (The nodes of the skipped levels are
// written too and never visited.)
__global__ void k_emit(int64_t n, int L, const int* left, const int* right, const int* first, const int* last,
                       const float4* leafbox, const float4* ibox, BvhNode* nodes) {
  grid_dep_wait();
  grid_dep_launch();
  int64_t node = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (node >= n - 1 || last[node] - first[node] + 1 <= L) return;
  float lo0[3], hi0[3], lo1[3], hi1[3];
  int cl = left[node], cr = right[node];
  load_box(cl >= 0 ? ibox + 2 * cl : leafbox + 2 * (int64_t)(~cl), lo0, hi0);
  load_box(cr >= 0 ? ibox + 2 * cr : leafbox + 2 * (int64_t)(~cr), lo1, hi1);
  float lo[4][3], hi[4][3];
  unsigned code[4], rep[4];
  wide_slots(cl, lo0, hi0, left, right, first, last, L, leafbox, ibox, lo, hi, code, rep);
  wide_slots(cr, lo1, hi1, left, right, first, last, L, leafbox, ibox, lo + 2, hi + 2, code + 2, rep + 2);
  BvhNode nd;
  nd.lox = make_float4(lo[0][0], lo[1][0], lo[2][0], lo[3][0]);
  nd.loy = make_float4(lo[0][1], lo[1][1], lo[2][1], lo[3][1]);
  nd.loz = make_float4(lo[0][2], lo[1][2], lo[2][2], lo[3][2]);
  nd.hix = make_float4(hi[0][0], hi[1][0], hi[2][0], hi[3][0]);
  nd.hiy = make_float4(hi[0][1], hi[1][1], hi[2][1], hi[3][1]);
  nd.hiz = make_float4(hi[0][2], hi[1][2], hi[2][2], hi[3][2]);
  nd.code = make_uint4(code[0], code[1], code[2], code[3]);
  nd.rep = make_uint4(rep[0], rep[1], rep[2], rep[3]);
  nodes[node] = nd;
}

// Root for n <= leaf_size: one node whose first child is the whole range.
__global__ void k_root_leaf(int64_t n, const float4* leafbox, BvhNode* nodes) {
  grid_dep_wait();
  grid_dep_launch();
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = 0; i < n; ++i) {
    float a[3], b[3];
    load_box(leafbox + 2 * i, a, b);
    for (int k = 0; k < 3; ++k) {
      lo[k] = fminf(lo[k], a[k]);
      hi[k] = fmaxf(hi[k], b[k]);
    }
  }
  const float I = INFINITY;
  BvhNode nd;
  nd.lox = make_float4(lo[0], I, I, I);
  nd.loy = make_float4(lo[1], I, I, I);
  nd.loz = make_float4(lo[2], I, I, I);
  nd.hix = make_float4(hi[0], -I, -I, -I);
  nd.hiy = make_float4(hi[1], -I, -I, -I);
  nd.hiz = make_float4(hi[2], -I, -I, -I);
  nd.code = make_uint4(node_code(0, (int)n), kNoChild, kNoChild, kNoChild);
  nd.rep = make_uint4(0, 0, 0, 0);
  nodes[0] = nd;
}

// eta (the largest distance between a float vertex of tri32 and its input value, the
// square root of the gathered squared maximum, rounded up) and the validity flag of B.
__global__ void k_build_meta(const unsigned* misc, float* meta, int bits, int gbits) {
  grid_dep_wait();
  grid_dep_launch();
  const double r = sqrt((double)__uint_as_float(misc[7])) * (1.0 + 1e-15);
  meta[0] = __double2float_ru(r);
  meta[1] = __uint_as_float(misc[6] != 0u ? 1u : 0u);
  meta[2] = 0.f;
  meta[3] = 0.f;
  for (int k = 0; k < 6; ++k) meta[4 + k] = ordered_to_float(misc[k]);  // the Morton codes' box
  meta[10] = __int_as_float(bits);
  meta[11] = __int_as_float(gbits);
}

// The hint grid from the sorted codes: -1 everywhere (k_grid_clear), then the first triangle
// of every coarse cell that holds one (a cell's triangles are contiguous in BVH order).
__global__ void k_grid_clear(int* grid, int64_t ncells) {
  grid_dep_wait();
  grid_dep_launch();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ncells; e += (int64_t)gridDim.x * blockDim.x)
    grid[e] = -1;
}
__global__ void k_grid(const uint64_t* keys, int64_t n, int shift, int* grid) {
  grid_dep_wait();
  grid_dep_launch();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t c = keys[i] >> shift;
  if (i == 0 || (keys[i - 1] >> shift) != c) grid[c] = (int)i;
}

template <typename T>
int launch_prep(const hd_mesh* B, const void* V, const int32_t* F, float4* cent, unsigned* cbox, int* bad, int sms,
                cudaStream_t s) {
  launch_chained(k_prep<T>, std::min(blocks_for(B->nF, kThreads), (unsigned)sms * 8), kThreads, 0, s, (const T*)V, B->nV,
                 F, B->nF, cent, cbox, bad);
  HD_TRY_LAUNCH();
  return HD_OK;
}

}  // namespace

int build_bvh(const hd_mesh* B, const Opts& o, cudaStream_t s, hd_bvh** out) {
  const int64_t n = B->nF;
  const size_t vbytes = (size_t)B->nV * 3 * (B->vtype == HD_F64 ? 8 : 4);
  int dev = 0;
  HD_TRY(cudaGetDevice(&dev));

  // inputs on the device
  const void* V = B->V;
  const int32_t* F = B->F;
  void* Vtmp = nullptr;
  int32_t* Ftmp = nullptr;
  if (!B->on_device) {
    HD_TRY(cudaMallocAsync(&Vtmp, vbytes, s));
    HD_TRY(cudaMallocAsync((void**)&Ftmp, (size_t)n * 12, s));
    HD_TRY(cudaMemcpyAsync(Vtmp, B->V, vbytes, cudaMemcpyHostToDevice, s));
    HD_TRY(cudaMemcpyAsync(Ftmp, B->F, (size_t)n * 12, cudaMemcpyHostToDevice, s));
    V = Vtmp;
    F = Ftmp;
  }

  // grid bits per axis: about 2^4 cells per triangle along each axis beyond n^(1/3), at
  // least 10 and at most 16 (3 x 16 = 48-bit codes); the code's lowest 1 or 2 bits are dropped
  // when they would take a sort pass of their own (33 bits -> 32: four passes instead of
  // five; equal codes keep their input order), and the sort runs ceil(key bits / 8) passes
  int bits = 10;
  while (bits < 16 && ((int64_t)1 << (3 * (bits - 4))) < n) ++bits;
  const int drop = (3 * bits) % 8 <= 2 ? (3 * bits) % 8 : 0, key_bits = 3 * bits - drop;
  // the hint grid: about 2 triangles per coarse cell (gbits per axis, at most 10)
  int gbits = 1;
  while (gbits < 10 && gbits < bits - 1 && ((int64_t)1 << (3 * (gbits + 1) + 1)) <= n) ++gbits;

  hd_bvh* h = new hd_bvh();
  h->block = nullptr;
  h->meta = nullptr;
  h->grid = nullptr;
  h->eta = 0.f;
  h->device = dev;
  h->nF = n;
  h->leaf_size = o.leaf_size;
  h->input_f64 = B->vtype == HD_F64;
  h->n_nodes = n > 1 ? n - 1 : 1;
  {
    // the BVH's own arrays: one allocation from the device's stream-ordered pool
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    // the FP64 copy of the triangles only for float64 input (tri32 holds float32 input exactly)
    const size_t b_nodes = up(sizeof(BvhNode) * h->n_nodes), b_t32 = up(sizeof(float4) * 3 * n),
                 b_t64 = (h->input_f64 || HD_KEEP_TRI64) ? up(sizeof(double) * 9 * n) : 0, b_vid = up(sizeof(int4) * n),
                 b_inv = up(sizeof(int) * n),
                 b_meta = up(16 * sizeof(float)), b_grid = up(sizeof(int) << (3 * gbits));
    cudaError_t e = cudaMallocAsync(&h->block, b_nodes + b_t32 + b_t64 + b_vid + b_inv + b_meta + b_grid, s);
    if (e != cudaSuccess) {
      delete h;
      return set_cuda_error(e, "cudaMallocAsync", __FILE__, __LINE__);
    }
    char* c = (char*)h->block;
    h->nodes = (BvhNode*)c;
    h->tri32 = (float4*)(c + b_nodes);
    h->tri64 = (h->input_f64 || HD_KEEP_TRI64) ? (double*)(c + b_nodes + b_t32) : nullptr;
    h->tri_vid = (int4*)(c + b_nodes + b_t32 + b_t64);
    h->inv = (int*)(c + b_nodes + b_t32 + b_t64 + b_vid);
    h->meta = (float*)(c + b_nodes + b_t32 + b_t64 + b_vid + b_inv);
    h->grid = (int*)(c + b_nodes + b_t32 + b_t64 + b_vid + b_inv + b_meta);
    h->grid_bits = gbits;
  }

  // scratch: one block, carved up
  // radix-sort tiles: 1024 keys for small inputs (more blocks), RS_THREADS * RS_BIG above; up to
  // RS_FUSED_MAX_BLOCKS tiles the digit offsets are computed inside the scatter kernel
  const int rs_rounds = n <= (int64_t)RS_FUSED_MAX_BLOCKS * RS_THREADS * 4 ? 4 : RS_BIG;
  const int64_t rs_tile = (int64_t)RS_THREADS * rs_rounds;
  const int nblk = (int)((n + rs_tile - 1) / rs_tile);
  const bool fused = nblk <= RS_FUSED_MAX_BLOCKS;
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    size_t at = off;
    off += (bytes + 255) & ~(size_t)255;
    return at;
  };
  size_t o_cent = carve(16 * n), o_k0 = carve(8 * n), o_k1 = carve(8 * n), o_v0 = carve(4 * n),
         o_v1 = carve(4 * n), o_hist = carve(4 * 256 * (size_t)nblk), o_leafbox = carve(32 * n),
         o_ibox = carve(32 * n), o_lv = carve(32 * (n + 64)), o_int = carve(4 * 4 * n + 64), o_misc = carve(64),
         o_tot = carve(4 * 256 * kMaxSortPasses);
  // weld: canonical vertex ids, and a table of at least twice the vertices
  const bool weld = (o.flags & HD_FLAG_WELD_B) != 0;
  uint64_t weld_entries = 1024;
  while (weld && weld_entries < 2 * (uint64_t)B->nV) weld_entries <<= 1;
  const size_t o_canon = weld ? carve(4 * (size_t)B->nV) : 0, o_wtab = weld ? carve(4 * weld_entries) : 0;
  char* scratch = nullptr;
  HD_TRY(cudaMallocAsync((void**)&scratch, off, s));
  float4* cent = (float4*)(scratch + o_cent);
  uint64_t* k0 = (uint64_t*)(scratch + o_k0);
  uint64_t* k1 = (uint64_t*)(scratch + o_k1);
  uint32_t* v0 = (uint32_t*)(scratch + o_v0);
  uint32_t* v1 = (uint32_t*)(scratch + o_v1);
  unsigned* hist = (unsigned*)(scratch + o_hist);
  float4* leafbox = (float4*)(scratch + o_leafbox);
  float4* ibox = (float4*)(scratch + o_ibox);
  float4* lv = (float4*)(scratch + o_lv);
  int* ints = (int*)(scratch + o_int);
  int *left = ints, *right = ints + n, *first = ints + 2 * n, *last = ints + 3 * n;
  // [0..5] centroid box (ordered bits: minima start at all ones), [6] bad, [7] squared eta bits
  unsigned* misc = (unsigned*)(scratch + o_misc);
  unsigned* tot = (unsigned*)(scratch + o_tot);  // digit totals of each sort pass (unfused path)

  TraceScope trace_build(HD_K_BUILD, s);  // the whole build counts as one launch
  HD_TRY(cudaMemsetAsync(misc, 0xff, 3 * sizeof(unsigned), s));
  HD_TRY(cudaMemsetAsync(misc + 3, 0, 5 * sizeof(unsigned), s));
  int sms = 1;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int rc = B->vtype == HD_F64 ? launch_prep<double>(B, V, F, cent, misc, (int*)(misc + 6), sms, s)
                              : launch_prep<float>(B, V, F, cent, misc, (int*)(misc + 6), sms, s);
  if (rc != HD_OK) return rc;
  launch_chained(k_morton, blocks_for(n, kThreads), kThreads, 0, s, cent, n, misc, bits, drop, k0, v0, tot,
                 256 * kMaxSortPasses);
  HD_TRY_LAUNCH();

  if (!(fused && rs_rounds == 4)) HD_TRY(fused ? rs_scatter_attr<true>() : rs_scatter_attr<false>());
  for (int shift = 0, pass = 0; shift < key_bits; shift += 8, ++pass) {
    if (fused && rs_rounds == 4) {
      launch_chained(k_rs_hist<4, true>, nblk, RS_THREADS, 0, s, k0, n, shift, hist, nblk, (unsigned*)nullptr);
      launch_chained(k_rs_scatter<4, true>, nblk, RS_THREADS, rs_scatter_smem<4>(), s, k0, v0, k1, v1, n, shift, hist,
                     nblk);
    } else if (fused) {
      launch_chained(k_rs_hist<RS_BIG, true>, nblk, RS_THREADS, 0, s, k0, n, shift, hist, nblk, (unsigned*)nullptr);
      launch_chained(k_rs_scatter<RS_BIG, true>, nblk, RS_THREADS, rs_scatter_smem<RS_BIG>(), s, k0, v0, k1, v1, n,
                     shift, hist, nblk);
    } else {
      unsigned* tp = tot + 256 * pass;
      launch_chained(k_rs_hist<RS_BIG, false>, nblk, RS_THREADS, 0, s, k0, n, shift, hist, nblk, tp);
      launch_chained(k_rs_scan_digits, 256, 256, 0, s, hist, nblk, (const unsigned*)tp);
      launch_chained(k_rs_scatter<RS_BIG, false>, nblk, RS_THREADS, rs_scatter_smem<RS_BIG>(), s, k0, v0, k1, v1, n,
                     shift, hist, nblk);
    }
    HD_TRY_LAUNCH();
    std::swap(k0, k1);
    std::swap(v0, v1);
  }

  {
    const int64_t ncells = (int64_t)1 << (3 * gbits);
#if HD_GRID_MEMSET
    HD_TRY(cudaMemsetAsync(h->grid, 0xff, sizeof(int) * ncells, s));
#else
    launch_chained(k_grid_clear, std::min<unsigned>(blocks_for(ncells, kThreads), 1024u), kThreads, 0, s, h->grid, ncells);
#endif
    launch_chained(k_grid, blocks_for(n, kThreads), kThreads, 0, s, (const uint64_t*)k0, n, 3 * (bits - gbits) - drop,
                   h->grid);
    HD_TRY_LAUNCH();
  }

  int* canon = nullptr;
  if (weld) {
    canon = (int*)(scratch + o_canon);
    int* wtab = (int*)(scratch + o_wtab);
    HD_TRY(cudaMemsetAsync(wtab, 0, 4 * weld_entries, s));
    if (B->vtype == HD_F64)
      launch_chained(k_weld<double>, blocks_for(B->nV, kThreads), kThreads, 0, s, (const double*)V, B->nV, wtab,
                     (unsigned long long)(weld_entries - 1), canon);
    else
      launch_chained(k_weld<float>, blocks_for(B->nV, kThreads), kThreads, 0, s, (const float*)V, B->nV, wtab,
                     (unsigned long long)(weld_entries - 1), canon);
  }
  if (B->vtype == HD_F64)
    launch_chained(k_gather<double>, blocks_for(n, kThreads), kThreads, 0, s, (const double*)V, F, v0, n,
                   (const int*)canon, (int64_t)B->nV, h->tri64, h->tri32, h->tri_vid, h->inv, leafbox, misc + 7);
  else
    launch_chained(k_gather<float>, blocks_for(n, kThreads), kThreads, 0, s, (const float*)V, F, v0, n,
                   (const int*)canon, (int64_t)B->nV, h->tri64, h->tri32, h->tri_vid, h->inv, leafbox, misc + 7);
  HD_TRY_LAUNCH();
  if (n > o.leaf_size) {
    launch_chained(k_karras, blocks_for(n - 1, kThreads), kThreads, 0, s, k0, n, left, right, first, last);
    // aligned-block boxes, 8 levels per launch, then every node's box
    LevelOffsets L;
    memset(&L, 0, sizeof L);
    L.count[0] = (int)n;
    int total = 0;
    while (L.count[L.levels] > 1) {
      const int k = ++L.levels;
      L.count[k] = (L.count[k - 1] + 1) / 2;
      L.off[k] = total;
      total += L.count[k];
    }
    for (int k0 = 0; k0 < L.levels; k0 += 8) {
      const float4* in = k0 ? lv + 2 * (int64_t)L.off[k0] : leafbox;
      launch_chained(k_levels, blocks_for(L.count[k0], 256), 256, 0, s, in, L.count[k0], lv, L, k0);
    }
    launch_chained(k_node_box, blocks_for(n - 1, kThreads), kThreads, 0, s, n, first, last, leafbox, lv, L, ibox);
    launch_chained(k_emit, blocks_for(n - 1, kThreads), kThreads, 0, s, n, o.leaf_size, left, right, first, last, leafbox, ibox,
                                                            h->nodes);
  } else {
    launch_chained(k_root_leaf, 1, 1, 0, s, n, leafbox, h->nodes);
  }
  HD_TRY_LAUNCH();

  launch_chained(k_build_meta, 1, 1, 0, s, misc, h->meta, bits, gbits);
  HD_TRY_LAUNCH();
  HD_TRY(cudaFreeAsync(scratch, s));
  if (Vtmp) HD_TRY(cudaFreeAsync(Vtmp, s));
  if (Ftmp) HD_TRY(cudaFreeAsync(Ftmp, s));
  if (!(o.flags & HD_FLAG_ASYNC_BUILD)) {
    float meta[2] = {0.f, 0.f};
    HD_TRY(cudaMemcpyAsync(meta, h->meta, sizeof meta, cudaMemcpyDeviceToHost, s));
    HD_TRY(cudaStreamSynchronize(s));
    h->eta = meta[0];
    uint32_t bad_bits;
    memcpy(&bad_bits, &meta[1], 4);
    if (bad_bits != 0u) {
      hd_free_B(h);
      return HD_ERR_INVALID;
    }
  }
  *out = h;
  return HD_OK;
}

}  // namespace hd
