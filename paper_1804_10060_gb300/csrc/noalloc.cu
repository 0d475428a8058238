// Allocation-free variant of tam_matrix_residual_norm.
//
// Some callers cannot allocate device memory at the moment they want a
// residual check: code running inside a custom device allocator or memory-pool
// callback (allocating there would re-enter the allocator), applications that
// reserve a fixed device-memory budget at start-up and treat any later
// cudaMalloc as an error (or would simply hit out-of-memory), and latency-
// critical paths that cannot afford the implicit synchronisation of
// cudaMalloc/cudaFree.  For them this file keeps the residual-norm
// reduction's scratch (one partial sum per thread block, the result and the
// last-block ticket) in a file-scope device array instead of allocating it.
//
// Set-up: the first call on each device looks up the array's device address
// with cudaGetSymbolAddress (with that device current) and caches it; make
// that first call before any stream capture begins.  The cached address
// belongs to the device's primary context: after cudaDeviceReset the array
// lives at an address the cache does not know, so a process that resets a
// device must not call this entry point on it again.
//
// The product is plain FP64 (the split copy of K is not used), like
// tam_matrix_residual_norm's.
//
// The array is TAM_NOALLOC_MAX_BLOCKS + 2 doubles (128 KiB) and stays
// resident on every device that loads the library until the process exits.
// It limits the matrix to TAM_NOALLOC_MAX_BLOCKS * 128 block rows.  Every
// call on a device shares it, so calls whose kernels overlap on the GPU (on
// different streams, or from different host threads) race; serialise them.
#include <cmath>
#include <mutex>

#include "handles.cuh"

namespace tam {
namespace {

constexpr int TAM_NOALLOC_MAX_BLOCKS = 16384;
constexpr int MAX_DEVICES = 64;

// [0, MAX_BLOCKS): per-block partials; [MAX_BLOCKS]: result;
// [MAX_BLOCKS + 1]: ticket (an unsigned int in the first 4 bytes).
static __device__ __align__(256) double g_noalloc_scratch[TAM_NOALLOC_MAX_BLOCKS + 2];

std::mutex g_addr_mutex;
double* g_addr[MAX_DEVICES] = {};

// Device address of the scratch array for the current device.  The host-side
// symbol is only a stand-in, so the address is looked up once per device
// (with that device current) and cached.
double* scratch_address() {
  int dev = 0;
  TAM_CUDA(cudaGetDevice(&dev));
  TAM_CHECK(dev >= 0 && dev < MAX_DEVICES, TAM_ERR_UNSUPPORTED, "residual_norm_noalloc: device id too large");
  std::lock_guard<std::mutex> lock(g_addr_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    TAM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_addr[dev] = static_cast<double*>(p);
  }
  return g_addr[dev];
}

template <int BR>
struct EpiResNormStatic {
  const double* b;
  int n_rows;
  GridReduce gr;
  double* out;
  __device__ bool skip() const { return false; }
  __device__ void operator()(int row, const double (&acc)[BR], double* sh) const {
    double s[1] = {0.0};
    if (row < n_rows)
#pragma unroll
      for (int k = 0; k < BR; ++k) {
        double v = b[(size_t)row * BR + k] - acc[k];
        s[0] += v * v;
      }
    double tot[1];
    if (grid_reduce<1>(gr, s, tot, sh) && threadIdx.x == 0) *out = tot[0];
  }
};

}  // namespace
}  // namespace tam

using namespace tam;

extern "C" int tam_matrix_residual_norm_noalloc(tam_matrix K, const double* b, const double* x, double* norm_host,
                                                void* stream) {
  try {
    set_last_error("");
    TAM_CHECK(K && b && x && norm_host, TAM_ERR_INVALID_ARG, "tam_matrix_residual_norm_noalloc: NULL argument");
    TAM_CHECK(K->A.br == 3, TAM_ERR_INVALID_ARG, "tam_matrix_residual_norm_noalloc: 3x3-block (elastic) K only");
    const unsigned grid = sell_grid(K->S);
    TAM_CHECK(grid <= (unsigned)TAM_NOALLOC_MAX_BLOCKS, TAM_ERR_INVALID_ARG,
              "tam_matrix_residual_norm_noalloc: matrix has more than 16384*128 = 2,097,152 block rows "
              "(the static scratch limit); use tam_matrix_residual_norm");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double* scratch = scratch_address();
    unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + TAM_NOALLOC_MAX_BLOCKS + 1);
    double* out = scratch + TAM_NOALLOC_MAX_BLOCKS;
    // the ticket must start at zero (a previous call may have been cut short)
    TAM_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s));
    GridReduce gr{scratch, ticket};
    sell_spmv<3, 3>(K->S, x, EpiResNormStatic<3>{b, K->n_nodes, gr, out}, s, /*df=*/false);
    double r2 = 0.0;
    TAM_CUDA(cudaMemcpyAsync(&r2, out, sizeof(double), cudaMemcpyDeviceToHost, s));
    TAM_CUDA(cudaStreamSynchronize(s));
    *norm_host = std::sqrt(r2);
    return TAM_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return TAM_ERR_INTERNAL;
  }
}
