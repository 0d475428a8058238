// Host-side utilities: error string, stream-ordered allocation, read-backs,
// and the three-phase (block sums, scan of sums, apply) exclusive scan.
#include "common.cuh"

#include <atomic>
#include <mutex>

namespace tam {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};
thread_local bool g_capturing = false;
static thread_local long long g_captured = 0;

void count_launch() {
  if (g_capturing) ++g_captured;
  else g_launches.fetch_add(1, std::memory_order_relaxed);
}
void count_graph_launch(long long kernel_nodes) { g_launches.fetch_add(kernel_nodes, std::memory_order_relaxed); }
long long launches_total() { return g_launches.load(); }
long long captured_and_reset() { long long c = g_captured; g_captured = 0; return c; }

void set_last_error(const std::string& msg) { g_last_error = msg; }

int sm_count() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cached[kMaxDev] = {};
  int dev = 0;
  TAM_CUDA(cudaGetDevice(&dev));
  if (dev >= 0 && dev < kMaxDev) {
    const int c = cached[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int n = 0;
  TAM_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  n = n > 0 ? n : 1;
  if (dev >= 0 && dev < kMaxDev) cached[dev].store(n, std::memory_order_relaxed);
  return n;
}
const char* last_error_cstr() { return g_last_error.c_str(); }

static void configure_pool_once() {
  static std::once_flag flag;
  std::call_once(flag, [] {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = ~0ull;  // keep freed blocks cached in this process
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  });
}

void* dev_alloc_bytes(size_t bytes, cudaStream_t s) {
  configure_pool_once();
  void* p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(e == cudaErrorMemoryAllocation ? TAM_ERR_OOM : TAM_ERR_CUDA,
                "cudaMallocAsync(" + std::to_string(bytes) + " B): " + cudaGetErrorString(e));
  }
  return p;
}

void dev_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

HostScalars& host_scalars() {
  static thread_local HostScalars hs;
  if (!hs.ll) {
    TAM_CUDA(cudaMallocHost(&hs.ll, 8 * sizeof(long long)));
    TAM_CUDA(cudaMallocHost(&hs.d, 8 * sizeof(double)));
  }
  return hs;
}

long long read_back_ll(const long long* dptr, cudaStream_t s) {
  HostScalars& h = host_scalars();
  TAM_CUDA(cudaMemcpyAsync(h.ll, dptr, sizeof(long long), cudaMemcpyDeviceToHost, s));
  TAM_CUDA(cudaStreamSynchronize(s));
  return h.ll[0];
}

void read_back_ll_int(const long long* a, const int* b, long long* va, int* vb, cudaStream_t s) {
  HostScalars& h = host_scalars();
  TAM_CUDA(cudaMemcpyAsync(h.ll, a, sizeof(long long), cudaMemcpyDeviceToHost, s));
  TAM_CUDA(cudaMemcpyAsync(h.ll + 1, b, sizeof(int), cudaMemcpyDeviceToHost, s));
  TAM_CUDA(cudaStreamSynchronize(s));
  *va = h.ll[0];
  *vb = *reinterpret_cast<int*>(h.ll + 1);
}

void read_back_int2(const int* a, const int* b, int* va, int* vb, cudaStream_t s) {
  HostScalars& h = host_scalars();
  TAM_CUDA(cudaMemcpyAsync(h.ll, a, sizeof(int), cudaMemcpyDeviceToHost, s));
  TAM_CUDA(cudaMemcpyAsync(h.ll + 1, b, sizeof(int), cudaMemcpyDeviceToHost, s));
  TAM_CUDA(cudaStreamSynchronize(s));
  *va = *reinterpret_cast<int*>(h.ll);
  *vb = *reinterpret_cast<int*>(h.ll + 1);
}

int read_back_int(const int* dptr, cudaStream_t s) {
  HostScalars& h = host_scalars();
  TAM_CUDA(cudaMemcpyAsync(h.ll, dptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  TAM_CUDA(cudaStreamSynchronize(s));
  return *reinterpret_cast<int*>(h.ll);
}

double read_back_double(const double* dptr, cudaStream_t s) {
  HostScalars& h = host_scalars();
  TAM_CUDA(cudaMemcpyAsync(h.d, dptr, sizeof(double), cudaMemcpyDeviceToHost, s));
  TAM_CUDA(cudaStreamSynchronize(s));
  return h.d[0];
}

// ---------------------------------------------------------------------------
// Exclusive scan.  Phase 1: each block of 1024 threads sums a tile of
// 4096 items.  Phase 2: one block scans the tile sums.  Phase 3: every tile
// is rescanned and offset.
// ---------------------------------------------------------------------------
namespace {
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <typename T>
__device__ T block_exclusive_scan(T v, T* sh, T* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    T w = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  T warp_off = wid > 0 ? sh[wid - 1] : T(0);
  *total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return warp_off + x - v;
}

template <typename T>
__global__ void scan_tile_sums(const T* __restrict__ in, long long n, T* __restrict__ sums) {
  __shared__ T sh[32];
  long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
  T s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k)
    if (base + k < n) s += in[base + k];
  T tot;
  block_exclusive_scan<T>(s, sh, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

template <typename T>
__global__ void scan_sums_single(T* sums, long long m, T* total_out) {
  __shared__ T sh[32];
  T carry = 0;
  for (long long base = 0; base < m; base += SCAN_THREADS) {
    long long i = base + threadIdx.x;
    T v = i < m ? sums[i] : T(0);
    T tot;
    T ex = block_exclusive_scan<T>(v, sh, &tot);
    if (i < m) sums[i] = carry + ex;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total_out = carry;
}

template <typename T>
__global__ void scan_apply(const T* in, T* out, long long n, const T* __restrict__ sums) {
  __shared__ T sh[32];
  long long base = (long long)blockIdx.x * SCAN_TILE + (long long)threadIdx.x * SCAN_ITEMS;
  T v[SCAN_ITEMS];
  T s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    v[k] = (base + k < n) ? in[base + k] : T(0);
    s += v[k];
  }
  T tot;
  T ex = block_exclusive_scan<T>(s, sh, &tot);
  // all reads of this tile are done before any write (in/out may alias)
  __syncthreads();
  T run = sums[blockIdx.x] + ex;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
}

template <typename T>
void exclusive_scan_impl(const T* in, T* out, long long n, cudaStream_t s) {
  long long tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (tiles < 1) tiles = 1;
  DBuf<T> sums((size_t)tiles, s);
  scan_tile_sums<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, n, sums.p);
  TAM_LAUNCH_CHECK();
  scan_sums_single<T><<<1, SCAN_THREADS, 0, s>>>(sums.p, tiles, out + n);
  TAM_LAUNCH_CHECK();
  if (n > 0) {
    scan_apply<T><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, sums.p);
    TAM_LAUNCH_CHECK();
  }
}
}  // namespace

void exclusive_scan_i32(const int* in, int* out, long long n, cudaStream_t s) {
  exclusive_scan_impl<int>(in, out, n, s);
}
void exclusive_scan_i64(const long long* in, long long* out, long long n, cudaStream_t s) {
  exclusive_scan_impl<long long>(in, out, n, s);
}

}  // namespace tam
