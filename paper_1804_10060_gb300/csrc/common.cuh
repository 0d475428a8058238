// Shared device/host utilities of the thermoamg CUDA library: error handling,
// stream-ordered allocation, prefix sums, deterministic block reductions and
// small warp-level sorts used by the symbolic (pattern-building) phases.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <stdexcept>
#include <string>

#include <nvtx3/nvToolsExt.h>
#include "thermoamg.h"

namespace tam {

// ---------------------------------------------------------------------------
// Errors: internal code throws tam::Error; the C ABI converts it to a status.
// ---------------------------------------------------------------------------
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void set_last_error(const std::string& msg);

#define TAM_CUDA(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      throw ::tam::Error(e_ == cudaErrorMemoryAllocation ? TAM_ERR_OOM : TAM_ERR_CUDA, \
                         std::string(#call) + ": " + cudaGetErrorString(e_));          \
    }                                                                                  \
  } while (0)

#define TAM_CHECK(cond, code, msg)                                 \
  do {                                                             \
    if (!(cond)) throw ::tam::Error((code), std::string(msg));     \
  } while (0)

// Every kernel launch of the library is followed by TAM_LAUNCH_CHECK(), which
// also counts it (launches recorded into a CUDA graph are counted when the
// graph is launched, see count_graph_launch).
void count_launch();
void count_graph_launch(long long kernel_nodes);
extern thread_local bool g_capturing;

#define TAM_LAUNCH_CHECK()        \
  do {                            \
    TAM_CUDA(cudaGetLastError()); \
    ::tam::count_launch();        \
  } while (0)

// ---------------------------------------------------------------------------
// Stream-ordered device memory (default pool, kept cached between calls).
// ---------------------------------------------------------------------------
void* dev_alloc_bytes(size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

template <typename T>
T* dalloc(size_t n, cudaStream_t s) {
  return static_cast<T*>(dev_alloc_bytes(n * sizeof(T) + 16, s));  // +16: room for aligned bulk copies
}

// Owning device buffer (freed stream-ordered on the stream it was made on).
template <typename T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  DBuf() = default;
  DBuf(size_t n_, cudaStream_t s_) : n(n_), s(s_) { p = n_ ? dalloc<T>(n_, s_) : nullptr; }
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : p(o.p), n(o.n), s(o.s) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept {
    if (this != &o) { reset(); p = o.p; n = o.n; s = o.s; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { reset(); }
  void reset() {
    if (p) dev_free(p, s);
    p = nullptr;
    n = 0;
  }
  void zero() { if (p) TAM_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s)); }
  T* get() const { return p; }
};

// A named NVTX range for the lifetime of the object (host side: what a
// profiler's timeline shows for the library's phases; costs nothing when no
// tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Small pinned host staging area for synchronous scalar read-backs.
struct HostScalars {
  long long* ll = nullptr;
  double* d = nullptr;
};
HostScalars& host_scalars();  // per thread, allocated once

long long read_back_ll(const long long* dptr, cudaStream_t s);
int read_back_int(const int* dptr, cudaStream_t s);
// Two scalars with one synchronisation.
void read_back_ll_int(const long long* a, const int* b, long long* va, int* vb, cudaStream_t s);
void read_back_int2(const int* a, const int* b, int* va, int* vb, cudaStream_t s);
double read_back_double(const double* dptr, cudaStream_t s);

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
inline unsigned grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  return (unsigned)(g < 1 ? 1 : g);
}

// Streaming multiprocessors of the current device (cached per device id).
int sm_count();
// Grid of a grid-stride vector kernel: `per_sm` blocks per SM at most.
inline unsigned stride_grid(long long n, int block, int per_sm) {
  const unsigned cap = (unsigned)sm_count() * (unsigned)per_sm;
  const unsigned g = grid_for(n, block);
  return g < cap ? g : cap;
}

// ---------------------------------------------------------------------------
// Prefix sums: out[0..n] = exclusive scan of in[0..n), out[n] = total.
// `in` and `out` may alias.  Returns nothing; total stays on the device.
// ---------------------------------------------------------------------------
void exclusive_scan_i32(const int* in, int* out, long long n, cudaStream_t s);
void exclusive_scan_i64(const long long* in, long long* out, long long n, cudaStream_t s);

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum (all threads get the result).  `sh` needs 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  double r = sh[0];
  __syncthreads();
  return r;
}

// Deterministic grid reduction: each block stores its partial; the last block
// to finish (ticket) sums the partials in block order and returns true in all
// of its threads with *total set.  The ticket is reset for the next launch.
struct GridReduce {
  double* partials;       // [>= gridDim.x * nvals]
  unsigned int* ticket;   // one counter, zero between launches
};

template <int NV>
__device__ bool grid_reduce(GridReduce gr, const double (&v)[NV], double (&total)[NV], double* sh) {
  __shared__ bool s_last;
  for (int k = 0; k < NV; ++k) {
    double b = block_sum(v[k], sh);
    if (threadIdx.x == 0) gr.partials[(size_t)blockIdx.x * NV + k] = b;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(gr.ticket, 1u);
    s_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  for (int k = 0; k < NV; ++k) {
    double acc = 0.0;
    // fixed order: thread t sums partials t, t+B, ...; then a fixed tree
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
      acc += ((volatile double*)gr.partials)[(size_t)b * NV + k];
    total[k] = block_sum(acc, sh);
  }
  if (threadIdx.x == 0) *gr.ticket = 0u;
  return true;
}

// SplitMix64 finaliser (Steele, Lea & Flood 2014).
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// In-place ascending bitonic sort of buf[0..n2) by one warp (n2 a power of 2,
// pad with INT_MAX).  Optional payload array moves with the keys.
template <bool PAYLOAD>
__device__ void warp_bitonic_sort(int* key, int* pay, int n2) {
  const int lane = threadIdx.x & 31;
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < n2; i += 32) {
        int ixj = i ^ j;
        if (ixj > i) {
          int a = key[i], b = key[ixj];
          bool up = ((i & k) == 0);
          if ((a > b) == up) {
            key[i] = b;
            key[ixj] = a;
            if (PAYLOAD) { int t = pay[i]; pay[i] = pay[ixj]; pay[ixj] = t; }
          }
        }
      }
      __syncwarp();
    }
  }
}

// After sorting, compact unique keys (< INT_MAX) to the front; returns count.
__device__ __forceinline__ int warp_unique_sorted(int* key, int n2) {
  const int lane = threadIdx.x & 31;
  int count = 0;
  for (int base = 0; base < n2; base += 32) {
    int i = base + lane;
    int v = key[i];
    bool keep = (v != 0x7fffffff) && (i == 0 || key[i - 1] != v);
    unsigned m = __ballot_sync(0xffffffffu, keep);
    __syncwarp();
    int pos = count + __popc(m & ((1u << lane) - 1u));
    if (keep) key[pos] = v;  // pos <= i: writes never overtake unread slots of this chunk
    count += __popc(m);
    __syncwarp();
  }
  return count;
}

__device__ __forceinline__ int next_pow2(int v) {
  int p = 32;
  while (p < v) p <<= 1;
  return p;
}

// Binary search of `key` in sorted a[lo, hi); returns index or -1.
__device__ __forceinline__ int bsearch_i32(const int* a, int lo, int hi, int key) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    int v = a[mid];
    if (v == key) return mid;
    if (v < key) lo = mid + 1; else hi = mid;
  }
  return -1;
}

}  // namespace tam
