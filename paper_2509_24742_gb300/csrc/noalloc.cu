// srbe_structure_factor_noalloc: the structure factor S(k) = sum_j w_j exp(i k . r_j) for caller
// buffers, with no device allocation at all.  For callers that cannot call cudaMalloc (an MD
// engine that owns every byte of device memory through its own pool, or code running where an
// allocation would stall or break a running pipeline), the per-chunk partial sums live in a
// file-scope __device__ array of fixed size instead of a context buffer.
//
// The array (and the sin/cos table) is part of the library image: every GPU that loads the
// library holds it until the process exits.  Host code never dereferences the symbol; the
// device address is looked up once per device with cudaGetSymbolAddress and passed to the
// kernels.  Every call reuses the same array, so calls that overlap on the GPU (two streams,
// two host threads) race on it.
#include <cmath>
#include <mutex>

#include "srbe_internal.cuh"

namespace srbe {
namespace {

constexpr int kNaThreads = 128;              // 4 warps; a block covers 32 modes x 128 particles
constexpr int kNaMaxModes = 8192;            // largest mode list accepted
constexpr int kNaPartials = 1 << 17;         // 131072 double2 partials = 2 MiB
constexpr int kNaMaxChunks = 1024;
constexpr int kNaMaxDevices = 64;

static __device__ __align__(256) double2 na_scratch[kNaPartials];
static __device__ __align__(256) double2 na_table[kTab];

struct DeviceSetup {
  bool ready = false;
  double2 *scratch = nullptr;
  double2 *table = nullptr;
};
DeviceSetup g_setup[kNaMaxDevices];
std::mutex g_setup_mutex;

// partial[c][k] = sum over particles of chunk c of w_j exp(i k . r_j); r is [n][3], m is [K][3]
__global__ void __launch_bounds__(kNaThreads)
k_na_partial(int64_t n, const double *__restrict__ r, const double *__restrict__ w, int K,
             const int32_t *__restrict__ m3, double3 invL, const double2 *__restrict__ tab, int64_t chunk,
             double2 *__restrict__ partial) {
  __shared__ uint64_t su[3][kNaThreads];
  __shared__ double sw[kNaThreads];
  __shared__ double2 red[4][32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int kidx = blockIdx.y * 32 + lane;
  int4 m = make_int4(0, 0, 0, 0);
  if (kidx < K) m = make_int4(m3[3 * kidx], m3[3 * kidx + 1], m3[3 * kidx + 2], 0);
  const int64_t i0 = (int64_t)blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  double are = 0.0, aim = 0.0;
  for (int64_t base = i0; base < i1; base += kNaThreads) {
    __syncthreads();
    const int64_t i = base + t;
    if (i < i1) {
      su[0][t] = to_turns64(r[3 * i], invL.x);
      su[1][t] = to_turns64(r[3 * i + 1], invL.y);
      su[2][t] = to_turns64(r[3 * i + 2], invL.z);
      sw[t] = w[i];
    }
    __syncthreads();
    const int cnt = (int)min((int64_t)kNaThreads, i1 - base);
    for (int j = warp; j < cnt; j += 4) {
      double c, s;
      sincos_turns(phase64(m, su[0][j], su[1][j], su[2][j]), tab, c, s);
      are = fma(sw[j], c, are);
      aim = fma(sw[j], s, aim);
    }
  }
  red[warp][lane] = make_double2(are, aim);
  __syncthreads();
  if (warp == 0 && kidx < K) {
    double2 a = red[0][lane];
    for (int q = 1; q < 4; ++q) {
      a.x += red[q][lane].x;
      a.y += red[q][lane].y;
    }
    partial[(int64_t)blockIdx.x * K + kidx] = a;
  }
}

// S[k] = sum of the partials in chunk order; warp per mode, fixed shuffle order
__global__ void k_na_reduce(int K, int nchunk, const double2 *__restrict__ partial, double *__restrict__ S) {
  const int lane = threadIdx.x & 31;
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (k >= K) return;
  double re = 0.0, im = 0.0;
  for (int c = lane; c < nchunk; c += 32) {
    const double2 p = partial[(int64_t)c * K + k];
    re += p.x;
    im += p.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) {
    S[2 * k] = re;
    S[2 * k + 1] = im;
  }
}

// Once per device, with that device current: resolve the device addresses of the file-scope
// arrays, fill the sin/cos table (a host-to-symbol copy, no allocation), wait for the device, and
// load both kernels.
int setup_device(DeviceSetup **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return SRBE_ECUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup &s = g_setup[dev];
  if (!s.ready) {
    if (cudaGetSymbolAddress((void **)&s.scratch, na_scratch) != cudaSuccess) return SRBE_ECUDA;
    if (cudaGetSymbolAddress((void **)&s.table, na_table) != cudaSuccess) return SRBE_ECUDA;
    double2 h[kTab];
    for (int j = 0; j < kTab; ++j) {
      const long double a = 2.0L * 3.141592653589793238462643383279502884L * (long double)j / (long double)kTab;
      h[j] = make_double2((double)cosl(a), (double)sinl(a));
    }
    if (cudaMemcpyToSymbol(na_table, h, sizeof(h)) != cudaSuccess) return SRBE_ECUDA;
    // A copy from pageable memory may return before its DMA has landed, and streams created
    // non-blocking do not wait for the legacy stream it ran on: wait for it here, so that a first
    // call on any stream reads a complete table.
    if (cudaDeviceSynchronize() != cudaSuccess) return SRBE_ECUDA;
    // Load both kernels now (lazy module loading would otherwise load them at their first launch,
    // which may come inside a stream capture or a running pipeline).
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_na_partial) != cudaSuccess) return SRBE_ECUDA;
    if (cudaFuncGetAttributes(&fa, k_na_reduce) != cudaSuccess) return SRBE_ECUDA;
    s.ready = true;
  }
  *out = &s;
  return SRBE_OK;
}

}  // namespace
}  // namespace srbe

extern "C" int srbe_structure_factor_noalloc(const double box[3], int64_t n, const double *r_dev,
                                             const double *w_dev, int K, const int32_t *m_dev, double *S_dev,
                                             void *stream) {
  using namespace srbe;
  if (!box || !(box[0] > 0) || !(box[1] > 0) || !(box[2] > 0) || n < 0 || K < 0 || K > kNaMaxModes)
    return SRBE_EINVAL;
  if ((n > 0 && (!r_dev || !w_dev)) || (K > 0 && (!m_dev || !S_dev))) return SRBE_EINVAL;
  DeviceSetup *s = nullptr;
  const int st = setup_device(&s);
  if (st != SRBE_OK) return st;
  if (K == 0) return SRBE_OK;
  cudaStream_t cs = (cudaStream_t)stream;
  // chunks of whole 128-particle batches; at most kNaPartials / K partials fit the scratch array
  const int64_t cap = std::max<int64_t>(1, std::min<int64_t>(kNaMaxChunks, kNaPartials / K));
  int64_t nchunk = n > 0 ? std::min<int64_t>(cap, (n + kNaThreads - 1) / kNaThreads) : 0;
  int64_t chunk = kNaThreads;
  if (nchunk > 0) {
    chunk = (n + nchunk - 1) / nchunk;
    chunk = ((chunk + kNaThreads - 1) / kNaThreads) * kNaThreads;
    nchunk = (n + chunk - 1) / chunk;
    const double3 invL = make_double3(1.0 / box[0], 1.0 / box[1], 1.0 / box[2]);
    dim3 grid((unsigned)nchunk, (unsigned)((K + 31) / 32));
    k_na_partial<<<grid, kNaThreads, 0, cs>>>(n, r_dev, w_dev, K, m_dev, invL, s->table, chunk, s->scratch);
    if (cudaGetLastError() != cudaSuccess) return SRBE_ECUDA;
  }
  k_na_reduce<<<(unsigned)((K * 32 + 255) / 256), 256, 0, cs>>>(K, (int)nchunk, s->scratch, S_dev);
  if (cudaGetLastError() != cudaSuccess) return SRBE_ECUDA;
  return SRBE_OK;
}
