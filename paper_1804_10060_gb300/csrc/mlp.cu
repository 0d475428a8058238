// Learned CG initial guess: a node-wise multilayer perceptron, trained and
// evaluated with the kernels in this file.
//
// The paper has no learned component.  The network maps per-node features
// (coordinates, temperature, temperature gradient, distance to the clamped
// boundary) to a displacement guess that seeds AMG-PCG; the solver always
// iterates to the tolerance from it, and a guess whose preconditioned
// residual energy <r, M r> is not below that of the zero guess is replaced by
// zero (tam_learned_guess), so the network can cost iterations but never
// accuracy.
//
// Layers: tanh hidden layers, linear output.  Inputs are standardised,
// (x - shift) * scale, inside the first layer; outputs are multiplied by
// out_scale.  Training minimises the mean squared error with Adam.  All
// parameters are FP32 (master copy); inference can read a BF16 copy of the
// weights.  Each dense layer is one tiled kernel: a 64-row tile of the
// activations and the whole layer weight matrix sit in shared memory, and each
// thread produces 8 consecutive outputs of one row.
#include <cmath>
#include <type_traits>
#include <vector>

#include "handles.cuh"

struct tam_mlp_s {
  int n_in = 0, width = 0, depth = 0, n_out = 0;
  std::vector<std::pair<int, int>> shapes;  // (fan-in, fan-out) per layer
  std::vector<long long> offset;            // start of W_l in theta (bias follows)
  long long n_par = 0;
  tam::DBuf<float> theta, grad, m1, m2, shift, scale, out_scale;
  tam::DBuf<__nv_bfloat16> theta16;
  bool theta16_valid = false;
  int adam_t = 0;
  tam::DBuf<float> act;  // activations of the current batch, layer after layer
  size_t act_cap = 0;
  tam::DBuf<float> dbuf[2];
  size_t dcap = 0;
  tam::DBuf<double> red;  // loss reduction
  tam::DBuf<unsigned int> ticket;
};

namespace tam {
namespace {

constexpr int ROWS = 64;   // rows of the activation tile per block
constexpr int THREADS = 256;

template <typename TW>
__device__ __forceinline__ float ld(const TW* p) { return (float)p[0]; }
template <>
__device__ __forceinline__ float ld<__nv_bfloat16>(const __nv_bfloat16* p) { return __bfloat162float(p[0]); }

// out[n x N] = epi(A[n x K] W + bias) with W [K x N] row-major (or W^T when
// TRANS: W stored [N x K]).  MODE: 0 linear, 1 tanh, 2 output (* out_scale),
// 3 backward through tanh: out = (A W^T) * (1 - H^2) with H = `aux`.
// STD: standardise A on load with (a - shift) * scale.
template <typename TW, int MODE, bool TRANS, bool STD>
__global__ void __launch_bounds__(THREADS)
dense_kernel(const float* __restrict__ A, int n, int K, int N, const TW* __restrict__ W,
             const float* __restrict__ bias, const float* __restrict__ shift, const float* __restrict__ scale,
             const float* __restrict__ out_scale, const float* __restrict__ aux, float* __restrict__ out) {
  extern __shared__ float sm[];
  float* Ws = sm;                     // [K][N]
  float* As = sm + (size_t)K * N;     // [ROWS][K]
  for (int e = threadIdx.x; e < K * N; e += THREADS) {
    const int k = e / N, j = e % N;
    Ws[e] = TRANS ? ld(W + (size_t)j * K + k) : ld(W + e);
  }
  const int groups = (N + 7) / 8;
  for (long long r0 = (long long)blockIdx.x * ROWS; r0 < n; r0 += (long long)gridDim.x * ROWS) {
    __syncthreads();
    for (int e = threadIdx.x; e < ROWS * K; e += THREADS) {
      const int r = e / K, k = e % K;
      const long long row = r0 + r;
      float a = row < n ? A[row * K + k] : 0.f;
      if (STD) a = (a - shift[k]) * scale[k];
      As[e] = a;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < ROWS * groups; it += THREADS) {
      const int r = it / groups, c0 = (it % groups) * 8;
      const long long row = r0 + r;
      if (row >= n) continue;
      float acc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = 0.f;
      const float* ar = As + r * K;
      for (int k = 0; k < K; ++k) {
        const float a = ar[k];
        const float* wr = Ws + k * N + c0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (c0 + q < N) acc[q] = fmaf(a, wr[q], acc[q]);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int c = c0 + q;
        if (c >= N) break;
        float z = acc[q] + (bias ? bias[c] : 0.f);
        if (MODE == 1) z = tanhf(z);
        else if (MODE == 2) z *= out_scale[c];
        else if (MODE == 3) {
          const float h = aux[row * N + c];
          z *= (1.f - h * h);
        }
        out[row * N + c] = z;
      }
    }
  }
}

// grad_W[K x N] += H^T D and grad_b[N] += colsum(D) over all n rows; every
// block accumulates its share of rows in registers, then adds once.
__global__ void __launch_bounds__(THREADS)
weight_grad_kernel(const float* __restrict__ H, const float* __restrict__ D, int n, int K, int N,
                   const float* __restrict__ shift, const float* __restrict__ scale, float* __restrict__ gW,
                   float* __restrict__ gb) {
  extern __shared__ float sm[];
  float* Hs = sm;                   // [ROWS][K]
  float* Ds = sm + ROWS * K;        // [ROWS][N]
  const int KN = K * N;
  const int per = (KN + N + THREADS - 1) / THREADS;  // entries of (W, b) owned by this thread
  float acc[80];
#pragma unroll
  for (int q = 0; q < 80; ++q) acc[q] = 0.f;
  for (long long r0 = (long long)blockIdx.x * ROWS; r0 < n; r0 += (long long)gridDim.x * ROWS) {
    __syncthreads();
    for (int e = threadIdx.x; e < ROWS * K; e += THREADS) {
      const int r = e / K, k = e % K;
      const long long row = r0 + r;
      float h = row < n ? H[row * K + k] : 0.f;
      if (shift && row < n) h = (h - shift[k]) * scale[k];
      Hs[e] = h;
    }
    for (int e = threadIdx.x; e < ROWS * N; e += THREADS) {
      const long long row = r0 + e / N;
      Ds[e] = row < n ? D[row * N + e % N] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 80; ++q) {
      if (q >= per) break;
      const int e = threadIdx.x + q * THREADS;
      if (e < KN) {
        const int k = e / N, j = e % N;
        float s = acc[q];
        for (int r = 0; r < ROWS; ++r) s = fmaf(Hs[r * K + k], Ds[r * N + j], s);
        acc[q] = s;
      } else if (e < KN + N) {
        const int j = e - KN;
        float s = acc[q];
        for (int r = 0; r < ROWS; ++r) s += Ds[r * N + j];
        acc[q] = s;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 80; ++q) {
    if (q >= per) break;
    const int e = threadIdx.x + q * THREADS;
    if (e < KN) atomicAdd(&gW[e], acc[q]);
    else if (e < KN + N) atomicAdd(&gb[e - KN], acc[q]);
  }
}

// d = 2 (pred - Y) / (n m) * out_scale;  loss = mean (pred - Y)^2
__global__ void loss_grad_kernel(const float* __restrict__ pred, const float* __restrict__ Y, long long n, int m,
                                 const float* __restrict__ out_scale, float* __restrict__ d, GridReduce gr,
                                 double* __restrict__ loss) {
  __shared__ double sh[32];
  double acc[1] = {0.0};
  const double inv = 1.0 / ((double)n * m);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n * m; i += (long long)gridDim.x * blockDim.x) {
    const float diff = pred[i] - Y[i];
    acc[0] += (double)diff * diff;
    d[i] = (float)(2.0 * diff * inv) * out_scale[i % m];
  }
  double tot[1];
  if (grid_reduce<1>(gr, acc, tot, sh) && threadIdx.x == 0) *loss = tot[0] * inv;
}

// Adam (Kingma & Ba 2015): bias-corrected first/second moments
__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void init_params_kernel(float* __restrict__ theta, long long off, int a, int b, unsigned long long seed) {
  const long long nw = (long long)a * b;
  const float lim = sqrtf(6.f / (float)(a + b));  // Glorot uniform
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nw + b; i += (long long)gridDim.x * blockDim.x) {
    if (i < nw) {
      const uint64_t z = splitmix64(seed ^ (uint64_t)(off + i) * 0x9E3779B97F4A7C15ull);
      const float u = (float)((z >> 40) * (1.0 / 16777216.0));
      theta[off + i] = (2.f * u - 1.f) * lim;
    } else {
      theta[off + i] = 0.f;
    }
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16(in[i]);
}

// ---------------------------------------------------------------------------
// BF16 inference on the tensor cores: out = epi(A W + bias) with BF16 weights
// and BF16-rounded activations, FP32 accumulation (mma.sync m16n8k16).  A
// block of 4 warps takes 64 rows; warp w multiplies rows 16w..16w+15 of the
// tile by all of W.  W is kept transposed (n-major) in shared memory so that
// the two k-consecutive values of a B fragment are one 32-bit word; the A
// tile likewise.  K is padded to a multiple of 16 and N to a multiple of 8
// with zeros (K, N <= 128).
// ---------------------------------------------------------------------------
constexpr int MMA_ROWS = 64;
constexpr int MMA_THREADS = 128;
constexpr int MMA_KMAX = 128, MMA_NMAX = 128;
constexpr int MMA_LD = MMA_KMAX + 8;  // row stride in bf16 elements (staggers the banks)

__device__ __forceinline__ void mma_bf16_16x8x16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                                 unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <int MODE, bool STD>
__global__ void __launch_bounds__(MMA_THREADS)
dense_mma_kernel(const float* __restrict__ A, long long n, int K, int N, const __nv_bfloat16* __restrict__ W,
                 const float* __restrict__ bias, const float* __restrict__ shift, const float* __restrict__ scale,
                 const float* __restrict__ out_scale, float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __nv_bfloat16* Wt = reinterpret_cast<__nv_bfloat16*>(sm_raw);  // [Np][MMA_LD]
  const int Kp = (K + 15) & ~15, Np = (N + 7) & ~7;
  __nv_bfloat16* At = Wt + (size_t)Np * MMA_LD;                  // [MMA_ROWS][MMA_LD]
  for (int e = threadIdx.x; e < Np * Kp; e += MMA_THREADS) {
    const int nn = e / Kp, k = e % Kp;
    Wt[nn * MMA_LD + k] = (nn < N && k < K) ? W[(size_t)k * N + nn] : __float2bfloat16(0.f);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  for (long long r0 = (long long)blockIdx.x * MMA_ROWS; r0 < n; r0 += (long long)gridDim.x * MMA_ROWS) {
    __syncthreads();
    for (int e = threadIdx.x; e < MMA_ROWS * Kp; e += MMA_THREADS) {
      const int r = e / Kp, k = e % Kp;
      const long long row = r0 + r;
      float a = 0.f;
      if (row < n && k < K) {
        a = A[row * K + k];
        if (STD) a = (a - shift[k]) * scale[k];
      }
      At[r * MMA_LD + k] = __float2bfloat16(a);
    }
    __syncthreads();
    float acc[MMA_NMAX / 8][4];
#pragma unroll
    for (int j = 0; j < MMA_NMAX / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
    const __nv_bfloat16* Aw = At + (warp * 16) * MMA_LD;
    for (int k0 = 0; k0 < Kp; k0 += 16) {
      // A fragment: (g, 2t..2t+1), (g+8, 2t..), (g, 2t+8..), (g+8, 2t+8..)
      const unsigned a0 = *reinterpret_cast<const unsigned*>(Aw + g * MMA_LD + k0 + 2 * t);
      const unsigned a1 = *reinterpret_cast<const unsigned*>(Aw + (g + 8) * MMA_LD + k0 + 2 * t);
      const unsigned a2 = *reinterpret_cast<const unsigned*>(Aw + g * MMA_LD + k0 + 2 * t + 8);
      const unsigned a3 = *reinterpret_cast<const unsigned*>(Aw + (g + 8) * MMA_LD + k0 + 2 * t + 8);
#pragma unroll
      for (int j = 0; j < MMA_NMAX / 8; ++j) {
        if (j * 8 >= Np) break;
        // B fragment (column n = 8j + g): k = 2t..2t+1 and 2t+8..2t+9
        const __nv_bfloat16* wb = Wt + (j * 8 + g) * MMA_LD + k0 + 2 * t;
        mma_bf16_16x8x16(acc[j], a0, a1, a2, a3, *reinterpret_cast<const unsigned*>(wb),
                         *reinterpret_cast<const unsigned*>(wb + 8));
      }
    }
    // C fragment: (g, 2t..2t+1) and (g+8, 2t..2t+1) of each 16x8 tile
#pragma unroll
    for (int j = 0; j < MMA_NMAX / 8; ++j) {
      if (j * 8 >= Np) break;
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const long long row = r0 + warp * 16 + g + (h >= 2 ? 8 : 0);
        const int c = j * 8 + 2 * t + (h & 1);
        if (row >= n || c >= N) continue;
        float z = acc[j][h] + (bias ? bias[c] : 0.f);
        if (MODE == 1) z = tanhf(z);
        else if (MODE == 2) z *= out_scale[c];
        out[row * N + c] = z;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// The whole network in one kernel (BF16 inference): every layer's transposed
// BF16 weights and FP32 biases sit in shared memory for the kernel's life;
// each warp takes 16 rows at a time through all layers with the activations
// in registers -- the FP32 accumulators of one layer's 16 x 8 output tiles,
// biased, passed through tanh and rounded to BF16, are exactly the A
// fragments of the next layer's m16n8k16 products (tiles 2m and 2m+1 form
// k-chunk m).  Per row only the n_in inputs are read and the n_out outputs
// written.  Same roundings, products and summation order as the layer-by-
// layer kernel above, so the results are bitwise the same.
// ---------------------------------------------------------------------------
constexpr int FUSED_WARPS = 8;
constexpr int FUSED_MAX_LAYERS = 8;
constexpr int FUSED_WMAX = 128;  // widest layer (inputs and outputs)

struct FusedNet {
  int L;
  int K[FUSED_MAX_LAYERS], N[FUSED_MAX_LAYERS];    // true fan-in / fan-out
  int Kp[FUSED_MAX_LAYERS], Np[FUSED_MAX_LAYERS];  // padded: K to 16, N to 16 (hidden) or 8 (last)
  int wsm[FUSED_MAX_LAYERS], bsm[FUSED_MAX_LAYERS];  // shared-memory offsets (bf16 / float elements)
  long long woff[FUSED_MAX_LAYERS];                // W_l in theta (bias follows)
  int w_elems, b_elems;
};

__device__ __forceinline__ unsigned pack_bf16x2(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const unsigned*>(&v);
}

__global__ void __launch_bounds__(FUSED_WARPS * 32, 2)
mlp_fused_kernel(const float* __restrict__ X, long long n, FusedNet net, const __nv_bfloat16* __restrict__ th16,
                 const float* __restrict__ th, const float* __restrict__ shift, const float* __restrict__ scale,
                 const float* __restrict__ out_scale, float* __restrict__ Y) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __nv_bfloat16* Ws = reinterpret_cast<__nv_bfloat16*>(sm_raw);
  float* Bs = reinterpret_cast<float*>(sm_raw + (((size_t)net.w_elems * 2 + 15) & ~(size_t)15));
  // W_l^T [Np][Kp + 8] (zero-padded) and b_l [Np]
  for (int l = 0; l < net.L; ++l) {
    const int K = net.K[l], N = net.N[l], Kp = net.Kp[l], Np = net.Np[l], ld = Kp + 8;
    const __nv_bfloat16* W = th16 + net.woff[l];
    for (int e = threadIdx.x; e < Np * ld; e += blockDim.x) {
      const int nn = e / ld, k = e - nn * ld;
      Ws[net.wsm[l] + e] = (nn < N && k < K) ? W[(size_t)k * N + nn] : __float2bfloat16(0.f);
    }
    const float* b = th + net.woff[l] + (long long)K * N;
    for (int e = threadIdx.x; e < Np; e += blockDim.x) Bs[net.bsm[l] + e] = e < N ? b[e] : 0.f;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int n_in = net.K[0], n_out = net.N[net.L - 1];
  for (long long r0 = ((long long)blockIdx.x * FUSED_WARPS + warp) * 16; r0 < n;
       r0 += (long long)gridDim.x * FUSED_WARPS * 16) {
    unsigned af[FUSED_WMAX / 16][4];
    // layer 0's A fragments from the standardised inputs of rows r0+g, r0+g+8
    {
      const long long ra = r0 + g, rb = r0 + g + 8;
#pragma unroll
      for (int m = 0; m < FUSED_WMAX / 16; ++m) {
        if (m * 16 >= net.Kp[0]) break;
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          // q: 0,1 (ra, 2t..), 2,3 (rb, 2t..), 4,5 (ra, 2t+8..), 6,7 (rb, 2t+8..)
          const long long row = (q & 2) ? rb : ra;
          const int k = m * 16 + 2 * t + (q & 1) + ((q & 4) ? 8 : 0);
          float a = 0.f;
          if (row < n && k < n_in) a = (X[row * n_in + k] - shift[k]) * scale[k];
          v[q] = a;
        }
        af[m][0] = pack_bf16x2(v[0], v[1]);
        af[m][1] = pack_bf16x2(v[2], v[3]);
        af[m][2] = pack_bf16x2(v[4], v[5]);
        af[m][3] = pack_bf16x2(v[6], v[7]);
      }
    }
    for (int l = 0; l < net.L; ++l) {
      const int Kp = net.Kp[l], Np = net.Np[l], ld = Kp + 8;
      const __nv_bfloat16* Wt = Ws + net.wsm[l];
      float acc[FUSED_WMAX / 8][4];
#pragma unroll
      for (int j = 0; j < FUSED_WMAX / 8; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
      for (int m = 0; m < FUSED_WMAX / 16; ++m) {
        if (m * 16 >= Kp) break;
#pragma unroll
        for (int j = 0; j < FUSED_WMAX / 8; ++j) {
          if (j * 8 >= Np) break;
          const __nv_bfloat16* wb = Wt + (j * 8 + g) * ld + m * 16 + 2 * t;
          mma_bf16_16x8x16(acc[j], af[m][0], af[m][1], af[m][2], af[m][3], *reinterpret_cast<const unsigned*>(wb),
                           *reinterpret_cast<const unsigned*>(wb + 8));
        }
      }
      const float* bl = Bs + net.bsm[l];
      if (l + 1 < net.L) {
        // hidden layer: tanh(acc + b), rounded to BF16, becomes the next A
#pragma unroll
        for (int m = 0; m < FUSED_WMAX / 16; ++m) {
          if (m * 16 >= Np) break;
          float z[2][4];
#pragma unroll
          for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int h = 0; h < 4; ++h) z[u][h] = tanhf(acc[2 * m + u][h] + bl[(2 * m + u) * 8 + 2 * t + (h & 1)]);
          af[m][0] = pack_bf16x2(z[0][0], z[0][1]);
          af[m][1] = pack_bf16x2(z[0][2], z[0][3]);
          af[m][2] = pack_bf16x2(z[1][0], z[1][1]);
          af[m][3] = pack_bf16x2(z[1][2], z[1][3]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < FUSED_WMAX / 8; ++j) {
          if (j * 8 >= Np) break;
#pragma unroll
          for (int h = 0; h < 4; ++h) {
            const long long row = r0 + g + (h >= 2 ? 8 : 0);
            const int c = j * 8 + 2 * t + (h & 1);
            if (row < n && c < n_out) Y[row * n_out + c] = (acc[j][h] + bl[c]) * out_scale[c];
          }
        }
      }
    }
  }
}

// Shapes the fused kernel takes: at most FUSED_MAX_LAYERS layers, every fan-in
// and fan-out at most FUSED_WMAX; false otherwise (layer-by-layer kernels).
bool fused_net(const tam_mlp_s* M, FusedNet& f, size_t& smem) {
  const int L = (int)M->shapes.size();
  if (L < 1 || L > FUSED_MAX_LAYERS) return false;
  f = FusedNet{};
  f.L = L;
  int w = 0, b = 0;
  for (int l = 0; l < L; ++l) {
    const int K = M->shapes[l].first, N = M->shapes[l].second;
    if (K > FUSED_WMAX || N > FUSED_WMAX) return false;
    f.K[l] = K;
    f.N[l] = N;
    f.Kp[l] = (K + 15) & ~15;
    f.Np[l] = l + 1 < L ? (N + 15) & ~15 : (N + 7) & ~7;
    if (l > 0 && f.Kp[l] != f.Np[l - 1]) return false;  // chained widths
    f.wsm[l] = w;
    f.bsm[l] = b;
    f.woff[l] = M->offset[l];
    w += f.Np[l] * (f.Kp[l] + 8);
    b += f.Np[l];
  }
  f.w_elems = w;
  f.b_elems = b;
  smem = (((size_t)w * 2 + 15) & ~(size_t)15) + (size_t)b * 4;
  return smem <= 200 * 1024;
}

size_t dense_mma_smem(int N) {
  return sizeof(__nv_bfloat16) * ((size_t)((N + 7) & ~7) * MMA_LD + (size_t)MMA_ROWS * MMA_LD);
}

unsigned ew_grid(long long n) { return stride_grid(n, 256, 8); }
unsigned row_grid(long long n) { return std::min<unsigned>((unsigned)((n + ROWS - 1) / ROWS), (unsigned)sm_count() * 2u); }

size_t dense_smem(int K, int N) { return sizeof(float) * ((size_t)K * N + (size_t)ROWS * K); }

template <typename TW, int MODE, bool TRANS, bool STD>
void dense(const float* A, long long n, int K, int N, const TW* W, const float* bias, const tam_mlp_s* M,
           const float* aux, float* out, cudaStream_t s) {
  if constexpr (std::is_same<TW, __nv_bfloat16>::value && !TRANS && (MODE == 1 || MODE == 2)) {
    // BF16 inference: tensor cores
    if (K <= MMA_KMAX && N <= MMA_NMAX) {
      const size_t smem = dense_mma_smem(N);
      TAM_CUDA(cudaFuncSetAttribute(dense_mma_kernel<MODE, STD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
      const unsigned grid = std::min<unsigned>((unsigned)((n + MMA_ROWS - 1) / MMA_ROWS), (unsigned)sm_count() * 8u);
      dense_mma_kernel<MODE, STD><<<std::max(1u, grid), MMA_THREADS, smem, s>>>(
          A, n, K, N, W, bias, M->shift.p, M->scale.p, M->out_scale.p, out);
      TAM_LAUNCH_CHECK();
      return;
    }
  }
  const size_t smem = dense_smem(K, N);
  TAM_CUDA(cudaFuncSetAttribute(dense_kernel<TW, MODE, TRANS, STD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  dense_kernel<TW, MODE, TRANS, STD><<<row_grid(n), THREADS, smem, s>>>(
      A, (int)n, K, N, W, bias, M->shift.p, M->scale.p, M->out_scale.p, aux, out);
  TAM_LAUNCH_CHECK();
}

// keep_all: every layer's activations (training needs them for the backward
// pass); otherwise only the two ping-pong buffers are sized.
void ensure_workspace(tam_mlp_s* M, long long n, bool keep_all, cudaStream_t s) {
  size_t need = 0;
  for (auto& sh : M->shapes) need += (size_t)n * sh.second;
  if (keep_all && need > M->act_cap) {
    M->act = DBuf<float>(need, s);
    M->act_cap = need;
  }
  size_t dneed = (size_t)n * std::max(M->width, M->n_out);
  if (dneed > M->dcap) {
    M->dbuf[0] = DBuf<float>(dneed, s);
    M->dbuf[1] = DBuf<float>(dneed, s);
    M->dcap = dneed;
  }
}

// forward into the workspace; returns the output pointer ([n x n_out]).
// keep_all: layer l's output stays in the activation buffer for the backward
// pass; otherwise the layers alternate between the two ping-pong buffers.
template <typename TW>
float* forward(tam_mlp_s* M, const float* X, long long n, const TW* theta, bool keep_all, cudaStream_t s) {
  ensure_workspace(M, n, keep_all, s);
  const float* in = X;
  float* o = keep_all ? M->act.p : M->dbuf[0].p;
  const int L = (int)M->shapes.size();
  for (int l = 0; l < L; ++l) {
    const int a = M->shapes[l].first, b = M->shapes[l].second;
    const TW* W = theta + M->offset[l];
    const float* bias_dummy = nullptr;
    (void)bias_dummy;
    // bias is FP32 in both precisions: read from the master copy
    const float* bias = M->theta.p + M->offset[l] + (long long)a * b;
    const bool last = l == L - 1;
    if (l == 0) {
      if (last) dense<TW, 2, false, true>(in, n, a, b, W, bias, M, nullptr, o, s);
      else dense<TW, 1, false, true>(in, n, a, b, W, bias, M, nullptr, o, s);
    } else {
      if (last) dense<TW, 2, false, false>(in, n, a, b, W, bias, M, nullptr, o, s);
      else dense<TW, 1, false, false>(in, n, a, b, W, bias, M, nullptr, o, s);
    }
    in = o;
    o = keep_all ? o + (size_t)n * b : M->dbuf[(l + 1) & 1].p;
  }
  return const_cast<float*>(in);
}

double loss_and_grad(tam_mlp_s* M, const float* X, const float* Y, long long n, cudaStream_t s) {
  float* pred = forward<float>(M, X, n, M->theta.p, true, s);
  M->grad.zero();
  const int L = (int)M->shapes.size();
  GridReduce gr{reinterpret_cast<double*>(M->red.p), M->ticket.p};
  DBuf<double> loss(1, s);
  float* d = M->dbuf[0].p;
  float* d2 = M->dbuf[1].p;
  loss_grad_kernel<<<ew_grid(n * M->n_out), 256, 0, s>>>(pred, Y, n, M->n_out, M->out_scale.p, d, gr, loss.p);
  TAM_LAUNCH_CHECK();
  // activations of layer l are at act + sum_{l'<l} n * b_l'
  std::vector<float*> acts(L);
  {
    float* o = M->act.p;
    for (int l = 0; l < L; ++l) {
      acts[l] = o;
      o += (size_t)n * M->shapes[l].second;
    }
  }
  for (int l = L - 1; l >= 0; --l) {
    const int a = M->shapes[l].first, b = M->shapes[l].second;
    const float* Hin = l == 0 ? X : acts[l - 1];
    const size_t smem = sizeof(float) * ((size_t)ROWS * a + (size_t)ROWS * b);
    TAM_CUDA(cudaFuncSetAttribute(weight_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    TAM_CHECK((a * b + b + THREADS - 1) / THREADS <= 80, TAM_ERR_UNSUPPORTED, "mlp: layer too wide");
    weight_grad_kernel<<<row_grid(n), THREADS, smem, s>>>(Hin, d, (int)n, a, b, l == 0 ? M->shift.p : nullptr,
                                                          l == 0 ? M->scale.p : nullptr, M->grad.p + M->offset[l],
                                                          M->grad.p + M->offset[l] + (long long)a * b);
    TAM_LAUNCH_CHECK();
    if (l > 0) {
      // d_prev = (d W^T) * (1 - H_{l-1}^2)
      dense<float, 3, true, false>(d, n, b, a, M->theta.p + M->offset[l], nullptr, M, acts[l - 1], d2, s);
      std::swap(d, d2);
    }
  }
  return read_back_double(loss.p, s);
}

void ensure_bf16(tam_mlp_s* M, cudaStream_t s) {
  if (!M->theta16_valid) {
    to_bf16_kernel<<<ew_grid(M->n_par), 256, 0, s>>>(M->theta.p, M->theta16.p, M->n_par);
    TAM_LAUNCH_CHECK();
    M->theta16_valid = true;
  }
}

float* forward_any(tam_mlp_s* M, const float* X, long long n, int bf16, cudaStream_t s) {
  if (!bf16) return forward<float>(M, X, n, M->theta.p, false, s);
  ensure_bf16(M, s);
  return forward<__nv_bfloat16>(M, X, n, M->theta16.p, false, s);
}

}  // namespace

// bf16: 0 FP32 layer by layer; 1 BF16 tensor cores, the whole network in one
// kernel when its shapes allow (else layer by layer); 2 BF16 layer by layer.
void mlp_forward_device(tam_mlp_s* M, long long n, const float* X, float* Y, int bf16, cudaStream_t s) {
  NvtxRange nvtx("tam: network inference");
  FusedNet f;
  size_t smem = 0;
  if (bf16 == 1 && fused_net(M, f, smem)) {
    ensure_bf16(M, s);
    if (n > 0) {
      TAM_CUDA(cudaFuncSetAttribute(mlp_fused_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      const long long tiles = (n + 15) / 16;
      const unsigned grid = (unsigned)std::min<long long>((tiles + FUSED_WARPS - 1) / FUSED_WARPS,
                                                          (long long)sm_count() * 2);
      mlp_fused_kernel<<<std::max(1u, grid), FUSED_WARPS * 32, smem, s>>>(
          X, n, f, M->theta16.p, M->theta.p, M->shift.p, M->scale.p, M->out_scale.p, Y);
      TAM_LAUNCH_CHECK();
    }
    return;
  }
  float* out = forward_any(M, X, n, bf16, s);
  TAM_CUDA(cudaMemcpyAsync(Y, out, 4 * (size_t)n * M->n_out, cudaMemcpyDeviceToDevice, s));
}
int mlp_n_in(tam_mlp_s* M) { return M->n_in; }
int mlp_n_out(tam_mlp_s* M) { return M->n_out; }

}  // namespace tam

using namespace tam;

namespace {
template <class F>
int guarded_mlp(F&& f) {
  try {
    set_last_error("");
    return f();
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return TAM_ERR_INTERNAL;
  }
}
}  // namespace

extern "C" {

int tam_mlp_create(int n_in, int width, int depth, int n_out, unsigned long long seed, tam_mlp* out) {
  return guarded_mlp([&] {
    TAM_CHECK(out && n_in >= 1 && n_in <= 128 && width >= 1 && width <= 128 && depth >= 1 && depth <= 16 &&
                  n_out >= 1 && n_out <= 128,
              TAM_ERR_INVALID_ARG, "tam_mlp_create: sizes out of range (1..128, depth 1..16)");
    auto M = new tam_mlp_s();
    cudaStream_t s = nullptr;
    M->n_in = n_in;
    M->width = width;
    M->depth = depth;
    M->n_out = n_out;
    std::vector<int> dims{n_in};
    for (int i = 0; i < depth; ++i) dims.push_back(width);
    dims.push_back(n_out);
    long long off = 0;
    for (size_t l = 0; l + 1 < dims.size(); ++l) {
      M->shapes.emplace_back(dims[l], dims[l + 1]);
      M->offset.push_back(off);
      off += (long long)dims[l] * dims[l + 1] + dims[l + 1];
    }
    M->n_par = off;
    M->theta = DBuf<float>(off, s);
    M->grad = DBuf<float>(off, s);
    M->m1 = DBuf<float>(off, s);
    M->m2 = DBuf<float>(off, s);
    M->theta16 = DBuf<__nv_bfloat16>(off, s);
    M->m1.zero();
    M->m2.zero();
    for (size_t l = 0; l < M->shapes.size(); ++l)
      init_params_kernel<<<64, 256, 0, s>>>(M->theta.p, M->offset[l], M->shapes[l].first, M->shapes[l].second,
                                            seed);
    TAM_LAUNCH_CHECK();
    M->shift = DBuf<float>(n_in, s);
    M->scale = DBuf<float>(n_in, s);
    M->out_scale = DBuf<float>(n_out, s);
    std::vector<float> zero(n_in, 0.f), one(std::max(n_in, n_out), 1.f);
    TAM_CUDA(cudaMemcpy(M->shift.p, zero.data(), 4 * n_in, cudaMemcpyHostToDevice));
    TAM_CUDA(cudaMemcpy(M->scale.p, one.data(), 4 * n_in, cudaMemcpyHostToDevice));
    TAM_CUDA(cudaMemcpy(M->out_scale.p, one.data(), 4 * n_out, cudaMemcpyHostToDevice));
    M->red = DBuf<double>((size_t)sm_count() * 8 * 2, s);
    M->ticket = DBuf<unsigned int>(1, s);
    M->ticket.zero();
    TAM_CUDA(cudaStreamSynchronize(s));
    *out = M;
    return TAM_OK;
  });
}

int tam_mlp_destroy(tam_mlp M) {
  return guarded_mlp([&] {
    delete M;
    return TAM_OK;
  });
}

int tam_mlp_info(tam_mlp M, long long* n_params, int* n_layers) {
  return guarded_mlp([&] {
    TAM_CHECK(M, TAM_ERR_INVALID_ARG, "tam_mlp_info: NULL handle");
    if (n_params) *n_params = M->n_par;
    if (n_layers) *n_layers = (int)M->shapes.size();
    return TAM_OK;
  });
}

int tam_mlp_set_normalization(tam_mlp M, const float* shift_host, const float* scale_host,
                              const float* out_scale_host) {
  return guarded_mlp([&] {
    TAM_CHECK(M && shift_host && scale_host && out_scale_host, TAM_ERR_INVALID_ARG, "tam_mlp_set_normalization: NULL");
    TAM_CUDA(cudaMemcpy(M->shift.p, shift_host, 4 * M->n_in, cudaMemcpyHostToDevice));
    TAM_CUDA(cudaMemcpy(M->scale.p, scale_host, 4 * M->n_in, cudaMemcpyHostToDevice));
    TAM_CUDA(cudaMemcpy(M->out_scale.p, out_scale_host, 4 * M->n_out, cudaMemcpyHostToDevice));
    return TAM_OK;
  });
}

int tam_mlp_get_params(tam_mlp M, float* theta_host) {
  return guarded_mlp([&] {
    TAM_CHECK(M && theta_host, TAM_ERR_INVALID_ARG, "tam_mlp_get_params: NULL");
    TAM_CUDA(cudaMemcpy(theta_host, M->theta.p, 4 * (size_t)M->n_par, cudaMemcpyDeviceToHost));
    return TAM_OK;
  });
}

int tam_mlp_set_params(tam_mlp M, const float* theta_host) {
  return guarded_mlp([&] {
    TAM_CHECK(M && theta_host, TAM_ERR_INVALID_ARG, "tam_mlp_set_params: NULL");
    TAM_CUDA(cudaMemcpy(M->theta.p, theta_host, 4 * (size_t)M->n_par, cudaMemcpyHostToDevice));
    M->theta16_valid = false;
    return TAM_OK;
  });
}

int tam_mlp_forward(tam_mlp M, long long n, const float* X, float* Y, int bf16, void* stream) {
  return guarded_mlp([&] {
    TAM_CHECK(M && X && Y && n >= 0, TAM_ERR_INVALID_ARG, "tam_mlp_forward: bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (n == 0) return TAM_OK;
    mlp_forward_device(M, n, X, Y, bf16, s);
    return TAM_OK;
  });
}

int tam_mlp_loss_grad(tam_mlp M, long long n, const float* X, const float* Yt, double* loss_host, float* grad_host,
                      void* stream) {
  return guarded_mlp([&] {
    TAM_CHECK(M && X && Yt && n > 0, TAM_ERR_INVALID_ARG, "tam_mlp_loss_grad: bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double L = loss_and_grad(M, X, Yt, n, s);
    if (loss_host) *loss_host = L;
    if (grad_host) {
      TAM_CUDA(cudaMemcpyAsync(grad_host, M->grad.p, 4 * (size_t)M->n_par, cudaMemcpyDeviceToHost, s));
      TAM_CUDA(cudaStreamSynchronize(s));
    }
    return TAM_OK;
  });
}

int tam_mlp_train_step(tam_mlp M, long long n, const float* X, const float* Yt, float lr, double* loss_host,
                       void* stream) {
  return guarded_mlp([&] {
    TAM_CHECK(M && X && Yt && n > 0 && lr > 0.f, TAM_ERR_INVALID_ARG, "tam_mlp_train_step: bad argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double L = loss_and_grad(M, X, Yt, n, s);
    M->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)M->adam_t), c2 = 1.f - powf(b2, (float)M->adam_t);
    adam_kernel<<<ew_grid(M->n_par), 256, 0, s>>>(M->theta.p, M->grad.p, M->m1.p, M->m2.p, M->n_par, lr, b1, b2,
                                                  1e-8f, c1, c2);
    TAM_LAUNCH_CHECK();
    M->theta16_valid = false;
    if (loss_host) *loss_host = L;
    return TAM_OK;
  });
}

}  // extern "C"
