// C ABI of the SRBE library (declared in include/srbe.h): argument checks, host-side mode
// sampling (Eqs. 26-29), mode weights (Eqs. 24-25), the normalisation G (Eq. 27), staging of
// host arrays, and the order of the device passes of Algorithm 1.
#include <cmath>
#include <cstring>
#include <algorithm>
#include <chrono>
#include <mutex>
#include <new>
#include <thread>

#include "srbe_internal.cuh"

namespace srbe {

constexpr double kVolt = 0.694461;   // 1 V as a Coulomb potential in e/nm (96.4853 / 138.935458)
constexpr double kKeHost = 138.935458;

// ------------------------------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11)
// ------------------------------------------------------------------------------------------------
struct Philox4x64 {
  static void mul(uint64_t a, uint64_t b, uint64_t &hi, uint64_t &lo) {
    const unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    hi = (uint64_t)(p >> 64);
    lo = (uint64_t)p;
  }
  static void block(const uint64_t in[4], uint64_t k0, uint64_t k1, uint64_t out[4]) {
    uint64_t x0 = in[0], x1 = in[1], x2 = in[2], x3 = in[3];
    for (int r = 0; r < 10; ++r) {
      uint64_t hA, lA, hB, lB;
      mul(0xD2E7470EE14C6C93ull, x0, hA, lA);
      mul(0xCA5A826395121157ull, x2, hB, lB);
      const uint64_t y0 = hB ^ x1 ^ k0, y2 = hA ^ x3 ^ k1;
      x0 = y0;
      x1 = lB;
      x2 = y2;
      x3 = lA;
      k0 += 0x9E3779B97F4A7C15ull;   // key schedule: Weyl increments between rounds
      k1 += 0xBB67AE8584CAA73Bull;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
  }
};

inline double unit_open0(uint64_t w) { return ((double)(w >> 11) + 1.0) * (1.0 / 9007199254740992.0); }

// The sampling law of Eq. 26 factorises: exp(-k^2/4a^2) = prod_d exp(-pi^2 m_d^2 / (a L_d)^2), a discrete
// Gaussian per dimension of width sigma_d = a L_d / (sqrt 2 pi).
struct ModeSampler {
  double L[3], alpha;
  int M;
  int32_t box[3];
  double sig[3];
  int tabhalf[3];
  std::vector<double> qtab[3];   // q_d(m) of Eq. 28 for |m| <= tabhalf

  void init(const double Lb[3], double a, int Mdet, const int32_t mmax[3]) {
    alpha = a;
    M = Mdet;
    for (int d = 0; d < 3; ++d) {
      L[d] = Lb[d];
      box[d] = mmax[d];
      sig[d] = alpha * L[d] / (std::sqrt(2.0) * kPi);
      tabhalf[d] = (int)std::ceil(12.0 * sig[d]) + 2;
      qtab[d].resize(2 * tabhalf[d] + 1);
      for (int m = -tabhalf[d]; m <= tabhalf[d]; ++m) qtab[d][m + tabhalf[d]] = qd_direct(m, d);
    }
  }
  double qd_direct(int32_t m, int d) const {
    const double s = std::sqrt(2.0) * sig[d];
    return 0.5 * (std::erf((m + 0.5) / s) - std::erf((m - 0.5) / s));
  }
  double qd(int32_t m, int d) const {
    return (m >= -tabhalf[d] && m <= tabhalf[d]) ? qtab[d][m + tabhalf[d]] : qd_direct(m, d);
  }
  bool rejected(const int32_t m[3]) const {
    for (int d = 0; d < 3; ++d)
      if (box[d] > 0 && std::abs(m[d]) > box[d]) return true;
    return m[0] == 0 && m[1] == 0 && std::abs(m[2]) <= M;
  }
  double target(const int32_t m[3]) const {
    double k2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double kd = 2.0 * kPi * m[d] / L[d];
      k2 += kd * kd;
    }
    return std::exp(-k2 / (4.0 * alpha * alpha));
  }
  // proposal j of step `step`: three rounded normals and the acceptance uniform
  void proposal(uint64_t seed, uint64_t step, uint64_t j, int32_t m[3], double &u) const {
    const uint64_t c0[4] = {2 * j, step, 0, 0}, c1[4] = {2 * j + 1, step, 0, 0};
    uint64_t w0[4], w1[4];
    Philox4x64::block(c0, seed, 0x5352424500000001ull, w0);
    Philox4x64::block(c1, seed, 0x5352424500000001ull, w1);
    const double ra = std::sqrt(-2.0 * std::log(unit_open0(w0[0]))), ta = 2.0 * kPi * unit_open0(w0[1]);
    const double rb = std::sqrt(-2.0 * std::log(unit_open0(w0[2]))), tb = 2.0 * kPi * unit_open0(w0[3]);
    const double g[3] = {ra * std::cos(ta), ra * std::sin(ta), rb * std::cos(tb)};
    for (int d = 0; d < 3; ++d) m[d] = (int32_t)std::floor(sig[d] * g[d] + 0.5);
    u = unit_open0(w1[0]);
  }
  // Metropolis chain of Eq. 29 with independent proposals; first admissible proposal starts it
  void metropolis(uint64_t seed, uint64_t step, int P, int32_t *out) const {
    uint64_t j = 0;
    int32_t cur[3];
    double u;
    do {
      proposal(seed, step, j++, cur, u);
    } while (rejected(cur));
    double pc = target(cur), qc = qd(cur[0], 0) * qd(cur[1], 1) * qd(cur[2], 2);
    for (int l = 0; l < P; ++l) {
      if (l > 0) {
        int32_t pr[3];
        proposal(seed, step, j++, pr, u);
        if (!rejected(pr)) {
          const double pp = target(pr), qp = qd(pr[0], 0) * qd(pr[1], 1) * qd(pr[2], 2);
          if (u <= (pp * qc) / (pc * qp)) {
            std::memcpy(cur, pr, sizeof cur);
            pc = pp;
            qc = qp;
          }
        }
      }
      std::memcpy(out + 3 * l, cur, sizeof cur);
    }
  }
  int32_t support(int d) const {
    return box[d] > 0 ? box[d] : (int32_t)std::ceil(alpha * L[d] * std::sqrt(21.0 * std::log(10.0)) / kPi);
  }
  // the per-dimension cumulative distributions of the exact sampler (also the device sampler's)
  void exact_tables(std::vector<double> cdf[3], int32_t sup[3]) const {
    for (int d = 0; d < 3; ++d) {
      sup[d] = support(d);
      cdf[d].resize(2 * sup[d] + 1);
      double acc = 0.0;
      for (int i = 0; i < 2 * sup[d] + 1; ++i) {
        const double kd = 2.0 * kPi * (i - sup[d]) / L[d];
        acc += std::exp(-kd * kd / (4.0 * alpha * alpha));
        cdf[d][i] = acc;
      }
      for (double &v : cdf[d]) v /= acc;
    }
  }
  // exact i.i.d. draws: inverse CDF per dimension, rejection of I u {0}
  void exact(uint64_t seed, uint64_t step, int P, int32_t *out) const {
    std::vector<double> cdf[3];
    int32_t sup[3];
    exact_tables(cdf, sup);
    uint64_t tries = 0;
    for (int l = 0; l < P;) {
      const uint64_t c[4] = {tries++, step, 1, 0};
      uint64_t w[4];
      Philox4x64::block(c, seed, 0x5352424500000002ull, w);
      int32_t m[3];
      for (int d = 0; d < 3; ++d) {
        const double u = unit_open0(w[d]);
        const auto it = std::lower_bound(cdf[d].begin(), cdf[d].end() - 1, u);
        m[d] = (int32_t)(it - cdf[d].begin()) - sup[d];
      }
      if (rejected(m)) continue;
      std::memcpy(out + 3 * l, m, sizeof m);
      ++l;
    }
  }
  // Eq. 27 in product form over dimensions, minus k = 0 and the 2M deterministic modes
  double G() const {
    double th[3];
    for (int d = 0; d < 3; ++d) {
      const int32_t s = support(d);
      double acc = 0.0;
      for (int32_t m = -s; m <= s; ++m) {
        const double x = kPi * m / (alpha * L[d]);
        acc += std::exp(-x * x);
      }
      th[d] = acc;
    }
    double det = 0.0;
    const int top = box[2] > 0 ? std::min(M, (int)box[2]) : M;
    for (int m = 1; m <= top; ++m) {
      const double x = kPi * m / (alpha * L[2]);
      det += std::exp(-x * x);
    }
    return th[0] * th[1] * th[2] - 1.0 - 2.0 * det;
  }
};

}  // namespace srbe

using namespace srbe;

namespace {

// Streams of the critical path (a context's own stream, the capture stream, batch forks) get the
// highest priority, the side stream (lists, ion-ion forces) the lowest, so that where both have
// blocks waiting the block scheduler serves b, the solve and S2 first.
cudaStream_t make_stream(bool critical) {
  int least = 0, greatest = 0;
  SRBE_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  cudaStream_t s = nullptr;
  SRBE_CUDA(cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, critical ? greatest : least));
  return s;
}

int fail(srbe_ctx *c, const Error &e) {
  if (c) c->err = e.msg;
  return e.code;
}

// Every call that may change the state a captured step reads (buffers, sizes, settings) drops the
// step's CUDA graphs; srbe_step and the read-only queries keep them.
template <class Fn>
int guarded(srbe_ctx *c, Fn &&fn, bool keeps_graph = false) {
  if (!c) return SRBE_EINVAL;
  try {
    c->err.clear();
    if (!keeps_graph && c->hx) {
      c->hx->graph_dirty = true;
      c->hx->epoch++;
    }
    fn();
    return SRBE_OK;
  } catch (const Error &e) {
    return fail(c, e);
  } catch (const std::bad_alloc &) {
    return fail(c, Error{SRBE_ENOMEM, "host allocation failed"});
  } catch (const std::exception &e) {
    return fail(c, Error{SRBE_EINVAL, e.what()});
  }
}

bool finite_all(const double *a, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(a[i])) return false;
  return true;
}

// ---- staging kernels
__global__ void k_deinterleave(int64_t n, const double *__restrict__ r, double Lx, double Ly, double *__restrict__ x,
                               double *__restrict__ y, double *__restrict__ z) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double X = r[3 * i], Y = r[3 * i + 1];
  X -= Lx * floor(X / Lx);
  Y -= Ly * floor(Y / Ly);
  if (X >= Lx) X -= Lx;
  if (Y >= Ly) Y -= Ly;
  x[i] = X;
  y[i] = Y;
  z[i] = r[3 * i + 2];
}

__global__ void k_site_turns(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                             const double *__restrict__ z, double3 invL, uint64_t *__restrict__ u) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  u[i] = to_turns64(x[i], invL.x);
  u[n + i] = to_turns64(y[i], invL.y);
  u[2 * n + i] = to_turns64(z[i], invL.z);
}

// FP32 copies of the fixed site positions (the mixed form's b), site order
__global__ void k_site_f4(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                          const double *__restrict__ z, float4 *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_float4((float)x[i], (float)y[i], (float)z[i], 0.f);
}

// y = Q - psi_bar A^-1 e (inverse of Q = y + psi_bar A^-1 e, Eq. 10)
__global__ void k_unproject(int64_t n, const double *__restrict__ Q, const double *__restrict__ we,
                            const double *__restrict__ scal, double *__restrict__ y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = fma(-scal[kScalPsi], we[i], Q[i]);
}

__global__ void k_to_f32(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

__global__ void k_interleave(int64_t n, const double *__restrict__ F, double *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[3 * i] = F[i];
  out[3 * i + 1] = F[n + i];
  out[3 * i + 2] = F[2 * n + i];
}

// the force provider's input: positions [n][3] read from the caller's pinned host buffer (mapped),
// x and y wrapped into [0, L) as srbe_set_positions does, and their fixed-point phase coordinates for
// the ion structure factor.  A non-finite position is replaced by the box origin (so that no kernel
// sees it) and raises the bad-input flag.
__global__ void k_io_load(int64_t n, const double *__restrict__ r, double Lx, double Ly, double3 invL,
                          double *__restrict__ x, double *__restrict__ y, double *__restrict__ z,
                          uint64_t *__restrict__ iu, int *__restrict__ status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double X = r[3 * i], Y = r[3 * i + 1], Z = r[3 * i + 2];
  if (!(isfinite(X) && isfinite(Y) && isfinite(Z))) {
    X = Y = Z = 0.0;
    *(volatile int *)(status + kStatBadInput) = 1;
  }
  X -= Lx * floor(X / Lx);
  Y -= Ly * floor(Y / Ly);
  if (X >= Lx) X -= Lx;
  if (Y >= Ly) Y -= Ly;
  x[i] = X;
  y[i] = Y;
  z[i] = Z;
  iu[i] = to_turns64(X, invL.x);
  iu[n + i] = to_turns64(Y, invL.y);
  iu[2 * n + i] = to_turns64(Z, invL.z);
}

// the force provider's output: F [3][ni] as [ni][3], Q and psi_bar into the caller's pinned buffers
__global__ void k_io_store(int64_t ni, const double *__restrict__ F, double *__restrict__ Fo, int64_t ne,
                           const double *__restrict__ Q, double *__restrict__ Qo, const double *__restrict__ scal,
                           double *__restrict__ psi) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ni || i < ne; i += stride) {
    if (i < ni) {
      Fo[3 * i] = F[i];
      Fo[3 * i + 1] = F[ni + i];
      Fo[3 * i + 2] = F[2 * ni + i];
    }
    if (i < ne && Qo) Qo[i] = Q[i];
    if (i == 0) *psi = scal[kScalPsi];
  }
}

__global__ void k_interleave3(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                              const double *__restrict__ z, double *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[3 * i] = x[i];
  out[3 * i + 1] = y[i];
  out[3 * i + 2] = z[i];
}

}  // namespace

// per-context host state that the kernels never see
struct srbe::HostExt {
  ModeSampler sampler;
  // the exact sampler on the device: its tables (the host sampler's own cumulative distributions)
  bool dev_sampler = false;
  DevBuf<double> dev_cdf;
  int32_t dev_sup[3] = {0, 0, 0};
  DevBuf<int4> dev_step;   // step word for srbe_sample_k_device
  DevBuf<int> dev_err;     // set when the device sampler ran out of tries
  std::vector<double> hq;  // the ion charges last handed to srbe_set_positions (host copy)
  DevBuf<double> aos;      // AoS staging for positions / forces
  bool forces_valid = false;
  // CUDA graphs of one MD step, one per pinned staging slot of the mode list (ping-pong)
  struct Slot {
    int4 *hm = nullptr;           // mapped pinned memory: the host writes, a captured step reads
    double *hw = nullptr;
    const int4 *dhm = nullptr;    // the same buffers as device pointers
    const double *dhw = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
  } slot[2];
  cudaStream_t cap = nullptr;   // capture stream (a legacy default stream cannot be captured)
  // the captured host-I/O force provider (srbe_set_host_io / srbe_forces_host_io): the caller's
  // pinned buffers and their device views, a library-owned mapped word for psi_bar, and one graph
  // per mode-list slot
  double *io_r = nullptr, *io_F = nullptr, *io_Q = nullptr;
  const double *io_dr = nullptr;
  double *io_dF = nullptr, *io_dQ = nullptr;
  double *io_psi = nullptr, *io_dpsi = nullptr;
  cudaGraphExec_t io_exec[2] = {nullptr, nullptr};
  uint64_t io_epoch = ~0ull;
  int io_K = -1;
  int64_t io_kernels = 0;
  uint64_t io_calls = 0;
  // the next call's mode list, sampled (and written to the other slot) while the GPU runs this one
  bool io_pre = false;
  uint64_t io_pre_seed = 0, io_pre_step = 0;
  std::vector<int32_t> io_pre_hm, io_pre_samp;
  std::vector<double> io_pre_hc;
  void drop_io_graphs() {
    for (auto &g : io_exec)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
    io_epoch = ~0ull;
  }
  int graph_K = -1;
  int slot_cap = 0;
  bool graph_dirty = true;
  bool graph_failed = false;
  uint64_t epoch = 0;           // counts calls that may change what a captured step reads
  int64_t graph_kernels = 0;
  void drop_graphs() {
    for (auto &sl : slot)
      if (sl.exec) {
        cudaGraphExecDestroy(sl.exec);
        sl.exec = nullptr;
      }
    graph_dirty = true;
  }
  // phase tracing: a pool of event pairs, drained into per-phase sums when full or on request
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_phase;
  size_t ev_used = 0;
  int open_phase[kPhCount];
  double ms[kPhCount];
  int64_t count[kPhCount];
  ~HostExt() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    drop_graphs();
    drop_io_graphs();
    if (io_psi) cudaFreeHost(io_psi);
    if (cap) cudaStreamDestroy(cap);
    for (auto &sl : slot) {
      if (sl.hm) cudaFreeHost(sl.hm);
      if (sl.hw) cudaFreeHost(sl.hw);
      if (sl.done) cudaEventDestroy(sl.done);
    }
  }
};

namespace {
using Extra = srbe::HostExt;
Extra *extra(srbe_ctx *c) { return c->hx; }

constexpr size_t kEventPool = 4096;   // event pairs per drain

void drain_events(srbe_ctx *c) {
  Extra *e = extra(c);
  if (!e->ev_used) return;
  for (size_t i = 0; i < e->ev_used; ++i) {
    float t = 0.f;
    // phases run on the main and the side stream: wait for each interval's own end event
    SRBE_CUDA(cudaEventSynchronize(e->ev[2 * i + 1]));
    SRBE_CUDA(cudaEventElapsedTime(&t, e->ev[2 * i], e->ev[2 * i + 1]));
    e->ms[e->ev_phase[i]] += t;
    e->count[e->ev_phase[i]]++;
  }
  e->ev_used = 0;
}
}  // namespace

namespace srbe {
void phase_begin(srbe_ctx *c, int ph) {
  if (!c->profiling) return;
  Extra *e = extra(c);
  if (e->ev_used == kEventPool) drain_events(c);
  if (e->ev.empty()) {
    e->ev.resize(2 * kEventPool);
    e->ev_phase.resize(kEventPool);
    for (auto &x : e->ev) SRBE_CUDA(cudaEventCreate(&x));
  }
  e->open_phase[ph] = (int)e->ev_used;
  e->ev_phase[e->ev_used] = ph;
  SRBE_CUDA(cudaEventRecord(e->ev[2 * e->ev_used], c->stream));
  e->ev_used++;
}
void phase_end(srbe_ctx *c, int ph) {
  if (!c->profiling) return;
  Extra *e = extra(c);
  SRBE_CUDA(cudaEventRecord(e->ev[2 * e->open_phase[ph] + 1], c->stream));
}

// A cooperative kernel is only guaranteed to make progress when all its blocks can be resident at
// once; two of them overlapping on one GPU could each hold part of the SMs while waiting for the
// rest.  All cooperative launches (and graph launches that contain them) of the process on one
// device are therefore ordered through one event per device.
cudaEvent_t device_coop_chain() {
  static std::mutex mu;
  static std::vector<cudaEvent_t> ev;
  int dev = 0;
  SRBE_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if ((int)ev.size() <= dev) ev.resize(dev + 1, nullptr);
  if (!ev[dev]) SRBE_CUDA(cudaEventCreateWithFlags(&ev[dev], cudaEventDisableTiming));
  return ev[dev];
}
void coop_before(srbe_ctx *c) {
  SRBE_CUDA(cudaStreamWaitEvent(c->stream, c->coop_chain ? c->coop_chain : device_coop_chain(), 0));
}
void coop_after(srbe_ctx *c) {
  SRBE_CUDA(cudaEventRecord(c->coop_chain ? c->coop_chain : device_coop_chain(), c->stream));
}
}  // namespace srbe

namespace srbe {

void upload_table(srbe_ctx *c) {
  std::vector<double2> h(kTab);
  for (int j = 0; j < kTab; ++j) {
    const long double a = 2.0L * 3.141592653589793238462643383279502884L * (long double)j / (long double)kTab;
    h[j] = make_double2((double)cosl(a), (double)sinl(a));
  }
  c->tab.ensure(kTab);
  SRBE_CUDA(cudaMemcpyAsync(c->tab.p, h.data(), sizeof(double2) * kTab, cudaMemcpyHostToDevice, c->stream));
  SRBE_CUDA(cudaStreamSynchronize(c->stream));
}

void reserve(srbe_ctx *c) {
  const int K = std::max(c->K, 1);
  int64_t ch;
  const int64_t nch = std::max(sfac_chunks(c->ni, c->K, c->sf_occ, &ch), sfac_chunks(c->ne, c->K, c->sf_occ, &ch));
  c->partial.ensure((size_t)std::max<int64_t>(nch, 1) * K);
  c->mpart.ensure((size_t)std::max<int64_t>(nch, 1));
  c->coef.ensure((size_t)K);
  c->coef32.ensure((size_t)K);
  c->Q32.ensure((size_t)std::max<int64_t>(c->ne, 1));
  const size_t nblk = blocks_for(std::max<int64_t>(c->ni, 1), kWarpsPerBlock);
  const size_t neb = blocks_for(std::max<int64_t>(c->ne, 1), 128);
  c->epart.ensure(nblk * 4 + 4 + neb + 8);
  c->scal.ensure(kScalCount);
  const size_t tiles = (size_t)(K + 31) / 32;
  if (c->sfdone.cap < tiles) {
    c->sfdone.ensure(tiles);
    SRBE_CUDA(cudaMemsetAsync(c->sfdone.p, 0, sizeof(int) * tiles, c->stream));
  }
  // ion cell list and Verlet lists
  Cells &cl = c->icells;
  const size_t nn = (size_t)std::max<int64_t>(c->ni, 1), ne = (size_t)std::max<int64_t>(c->ne, 1);
  cl.cell.ensure(nn);
  cl.rank.ensure(nn);
  cl.order.ensure(nn);
  cl.inv.ensure(nn);
  cl.start.ensure((size_t)cl.g.ncell() + 1);
  cl.xs.ensure(nn);
  cl.ys.ensure(nn);
  cl.zs.ensure(nn);
  cl.ws.ensure(nn);
  cl.ts.ensure(nn);
  cl.ms.ensure(nn);
  cl.pf.ensure(nn);
  cl.us.ensure(3 * nn);
  NbrLists &nb = c->nbr;
  if (nb.cap == 0) {
    // twice the expected neighbour count at rc + skin for the mean ion density between the walls
    const double h = std::max(1.0, c->wall_span);
    const double rho = (double)std::max<int64_t>(c->ni, 1) / (c->L[0] * c->L[1] * h);
    const double r = c->rc + nb.skin;
    const double expect = rho * 4.0 / 3.0 * kPi * r * r * r;
    nb.cap = (int)std::min<double>(1 << 20, 32 * std::ceil(std::max(128.0, 2.0 * expect + 64.0) / 32.0));
  }
  nb.ii.ensure(nn * nb.cap);
  nb.ie.ensure(nn * nb.cap);
  nb.ei.ensure(ne * nb.cap);
  nb.ii_n.ensure(nn);
  nb.ie_n.ensure(nn);
  nb.ei_n.ensure(ne);
  nb.xb.ensure(nn);
  nb.yb.ensure(nn);
  nb.pfb.ensure(nn);
  nb.cell_s.ensure(nn);
  nb.flag.ensure(3);
  if (c->lat.nl > 0) c->lat.E.ensure((size_t)K * c->lat.nl);
}

}  // namespace srbe

namespace {

// the word after the mode list carries the MD step number (low, high 32 bits) for the thermostat
inline int4 step_word(uint64_t step) { return make_int4((int)(uint32_t)step, (int)(uint32_t)(step >> 32), 0, 0); }

void upload_modes(srbe_ctx *c) {
  const int K = (int)c->hc.size();
  if ((size_t)K + 1 > c->stage_cap) {
    if (c->h_mode_stage) cudaFreeHost(c->h_mode_stage);
    if (c->h_w_stage) cudaFreeHost(c->h_w_stage);
    c->h_mode_stage = nullptr;
    c->h_w_stage = nullptr;
    SRBE_CUDA(cudaMallocHost((void **)&c->h_mode_stage, sizeof(int4) * (K + 1)));
    SRBE_CUDA(cudaMallocHost((void **)&c->h_w_stage, sizeof(double) * (K + 1)));
    c->stage_cap = (size_t)K + 1;
  }
  // the previous copy out of the pinned buffer must have finished before it is overwritten
  SRBE_CUDA(cudaEventSynchronize(c->stage_done));
  for (int k = 0; k < K; ++k) {
    c->h_mode_stage[k] = make_int4(c->hm[4 * k], c->hm[4 * k + 1], c->hm[4 * k + 2], 0);
    c->h_w_stage[k] = c->hc[k];
  }
  c->h_mode_stage[K] = step_word(c->md_step);
  c->dm.ensure(K + 1);
  c->dc.ensure(std::max(K, 1));
  c->S1.ensure(std::max(K, 1));
  c->S2.ensure(std::max(K, 1));
  phase_begin(c, kPhUpload);
  SRBE_CUDA(cudaMemcpyAsync(c->dm.p, c->h_mode_stage, sizeof(int4) * (K + 1), cudaMemcpyHostToDevice, c->stream));
  if (K > 0)
    SRBE_CUDA(cudaMemcpyAsync(c->dc.p, c->h_w_stage, sizeof(double) * K, cudaMemcpyHostToDevice, c->stream));
  phase_end(c, kPhUpload);
  SRBE_CUDA(cudaEventRecord(c->stage_done, c->stream));
  c->K = K;
  c->have_modes = true;
}

// SRBE mode list (Eqs. 24-25): I folded to +m_z with twice the Ewald weight, then the samples with
// (G / P) 4 pi / (V k^2)
void srbe_host_list(srbe_ctx *c, const int32_t *samp, int P) {
  c->hm.clear();
  c->hc.clear();
  const double V = c->V;
  for (int mz = 1; mz <= c->M; ++mz) {
    const double kz = 2.0 * kPi * mz / c->L[2];
    const double k2 = kz * kz;
    c->hm.insert(c->hm.end(), {0, 0, mz, 0});
    c->hc.push_back(2.0 * 4.0 * kPi / (V * k2) * std::exp(-k2 / (4.0 * c->alpha * c->alpha)));
  }
  c->Kdet = c->M;
  for (int l = 0; l < P; ++l) {
    const int32_t *m = samp + 3 * l;
    double k2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double kd = 2.0 * kPi * m[d] / c->L[d];
      k2 += kd * kd;
    }
    c->hm.insert(c->hm.end(), {m[0], m[1], m[2], 0});
    c->hc.push_back((c->G / P) * 4.0 * kPi / (V * k2));
  }
  c->hsamp.assign(samp, samp + 3 * P);
  c->explicit_list = false;
}

void srbe_list_from_samples(srbe_ctx *c, const int32_t *samp, int P) {
  srbe_host_list(c, samp, P);
  upload_modes(c);
}

// ---- CUDA graph of one MD step ------------------------------------------------------------------
// The device half of a step (mode list read from a mapped pinned slot, kick/drift, the force pass,
// kick) has no host synchronisation and no allocation once the buffers are reserved, so it is
// captured once per slot and replayed; the host fills the other slot while the GPU runs.
void forces_pass(srbe_ctx *c, bool energies, bool after_drift = false, bool check = true);

// the captured step's mode list (K int4 + the step word) and weights, read from a mapped pinned slot
__global__ void k_stage_modes(int K, const int4 *__restrict__ hm, const double *__restrict__ hw,
                              int4 *__restrict__ dm, double *__restrict__ dc) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= K; k += gridDim.x * blockDim.x) {
    dm[k] = hm[k];
    if (k < K) dc[k] = hw[k];
  }
}

// the same for every replica of a batch graph at once, one block per replica
struct StageEntry {
  const int4 *hm;
  const double *hw;
  int4 *dm;
  double *dc;
  int K;
};
__global__ void k_stage_many(const StageEntry *__restrict__ tab) {
  const StageEntry s = tab[blockIdx.x];
  for (int k = threadIdx.x; k <= s.K; k += blockDim.x) {
    s.dm[k] = s.hm[k];
    if (k < s.K) s.dc[k] = s.hw[k];
  }
}

// The exact i.i.d. sampler (inverse CDF per dimension, rejection of I u {0}) on the device, one block:
// tries are numbered as on the host (Philox4x64-10, key (seed, 'SRBE' 2), counter (try, step, 1, 0)),
// 256 per round, accepted ones placed in try order by a block scan, so the list is bitwise the host
// sampler's; weights (G / P) 4 pi / (V k^2) with the host's operations in the host's order.
constexpr int kSampleThreads = 256;
constexpr int kSampleRounds = 1 << 12;     // 1M tries at most (a round accepts nearly all of its 256)
struct DevSampleArgs {
  const int4 *step_src;     // (step low, step high, seed low, seed high)
  int P, M;
  int32_t box[3], sup[3];
  const double *cdf;        // the three tables back to back, 2 sup[d] + 1 entries each
  double L[3], G, V;
  int4 *dm;                 // modes: I at [0, M) (left as they are), samples at [M, M + P), step word at M + P
  double *dc;               // weights, the same layout
  int *err;
};
__device__ __forceinline__ int cdf_search(const double *cdf, int n, double u) {
  // first index in [0, n - 1) with cdf >= u, else n - 1 (the host's lower_bound over [0, n - 1))
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cdf[mid] < u) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}
__global__ void __launch_bounds__(kSampleThreads) k_sample_exact(DevSampleArgs a) {
  __shared__ int scan[kSampleThreads];
  __shared__ int s_count;
  const int t = threadIdx.x;
  const int4 sw = *a.step_src;
  const uint64_t step = (uint64_t)(uint32_t)sw.x | ((uint64_t)(uint32_t)sw.y << 32);
  const uint64_t seed = (uint64_t)(uint32_t)sw.z | ((uint64_t)(uint32_t)sw.w << 32);
  if (t == 0) {
    s_count = 0;
    a.dm[a.M + a.P] = sw;   // the step word of the list (the thermostat reads its step half)
  }
  const double *cd[3] = {a.cdf, a.cdf + 2 * a.sup[0] + 1, a.cdf + 2 * a.sup[0] + 1 + 2 * a.sup[1] + 1};
  __syncthreads();
  for (int round = 0; round < kSampleRounds; ++round) {
    uint64_t w[4];
    philox4x64_dev((uint64_t)round * kSampleThreads + t, step, 1, 0, seed, 0x5352424500000002ull, w);
    int32_t m[3];
    bool ok = true;
    for (int d = 0; d < 3; ++d) {
      const double u = ((double)(w[d] >> 11) + 1.0) * 0x1.0p-53;
      m[d] = cdf_search(cd[d], 2 * a.sup[d] + 1, u) - a.sup[d];
      if (a.box[d] > 0 && abs(m[d]) > a.box[d]) ok = false;
    }
    if (m[0] == 0 && m[1] == 0 && abs(m[2]) <= a.M) ok = false;
    // inclusive block scan of the accept flags (Hillis-Steele)
    scan[t] = ok ? 1 : 0;
    __syncthreads();
    for (int off = 1; off < kSampleThreads; off <<= 1) {
      const int v = t >= off ? scan[t - off] : 0;
      __syncthreads();
      scan[t] += v;
      __syncthreads();
    }
    const int pos = s_count + scan[t] - (ok ? 1 : 0);
    if (ok && pos < a.P) {
      a.dm[a.M + pos] = make_int4(m[0], m[1], m[2], 0);
      double k2 = 0.0;
      for (int d = 0; d < 3; ++d) {
        const double kd = __ddiv_rn(__dmul_rn(2.0 * kPi, (double)m[d]), a.L[d]);
        k2 = __dadd_rn(k2, __dmul_rn(kd, kd));
      }
      a.dc[a.M + pos] = __ddiv_rn(__dmul_rn(__dmul_rn(__ddiv_rn(a.G, (double)a.P), 4.0), kPi), __dmul_rn(a.V, k2));
    }
    __syncthreads();
    if (t == 0) s_count += scan[kSampleThreads - 1];
    __syncthreads();
    if (s_count >= a.P) return;
  }
  if (t == 0) atomicExch(a.err, 1);
}

inline int4 sample_word(uint64_t step, uint64_t seed) {
  return make_int4((int)(uint32_t)step, (int)(uint32_t)(step >> 32), (int)(uint32_t)seed, (int)(uint32_t)(seed >> 32));
}

DevSampleArgs dev_sample_args(srbe_ctx *c, const int4 *step_src) {
  Extra *e = extra(c);
  DevSampleArgs a;
  a.step_src = step_src;
  a.P = c->P;
  a.M = c->M;
  for (int d = 0; d < 3; ++d) {
    a.box[d] = c->mmax[d];
    a.sup[d] = e->dev_sup[d];
    a.L[d] = c->L[d];
  }
  a.cdf = e->dev_cdf.p;
  a.G = c->G;
  a.V = c->V;
  a.dm = c->dm.p;
  a.dc = c->dc.p;
  a.err = e->dev_err.p;
  return a;
}

// the host sampler's cumulative distributions, uploaded for the device sampler
void upload_sampler_tables(srbe_ctx *c) {
  Extra *e = extra(c);
  std::vector<double> cdf[3];
  e->sampler.exact_tables(cdf, e->dev_sup);
  std::vector<double> all;
  for (auto &v : cdf) all.insert(all.end(), v.begin(), v.end());
  double *d = e->dev_cdf.ensure(all.size());
  SRBE_CUDA(cudaMemcpy(d, all.data(), sizeof(double) * all.size(), cudaMemcpyHostToDevice));
  e->dev_step.ensure(1);
  SRBE_CUDA(cudaMemset(e->dev_err.ensure(1), 0, sizeof(int)));
}

void check_dev_sampler(srbe_ctx *c) {
  int h = 0;
  SRBE_CUDA(cudaMemcpyAsync(&h, extra(c)->dev_err.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  SRBE_CUDA(cudaStreamSynchronize(c->stream));
  if (h) {
    SRBE_CUDA(cudaMemset(extra(c)->dev_err.p, 0, sizeof(int)));
    throw Error{SRBE_ENOTCONV, "device sampler: fewer than P admissible modes in 2^20 tries"};
  }
}

// one captured MD step of c; staged: the mode list is already on the device (batch graphs)
void device_step(srbe_ctx *c, int slot, bool staged) {
  Extra *e = extra(c);
  const int K = c->K;
  SRBE_REQUIRE(c->dm.cap > (size_t)K && c->dc.cap >= (size_t)K && e->slot[slot].dhm, SRBE_ESTATE,
               "mode buffers not reserved for a captured step");
  if (!staged) {
    // the mode list comes in through a kernel on the side stream that reads the pinned slot while
    // the opening kick runs (nothing before S1 reads it; the opening kick has no thermostat): the
    // host's list, or with the device sampler only the slot's (step, seed) word
    SRBE_CUDA(cudaEventRecord(c->ev_fork, c->stream));
    SRBE_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    if (e->dev_sampler)
      k_sample_exact<<<1, kSampleThreads, 0, c->side>>>(dev_sample_args(c, e->slot[slot].dhm + K));
    else
      k_stage_modes<<<std::min(blocks_for((int64_t)K + 1, 256), 64u), 256, 0, c->side>>>(K, e->slot[slot].dhm,
                                                                                         e->slot[slot].dhw, c->dm.p,
                                                                                         c->dc.p);
    c->launches++;
    SRBE_CUDA(cudaGetLastError());
    SRBE_CUDA(cudaEventRecord(c->ev_modes, c->side));
  }
  integrate_kick_drift(c, 0.5 * c->dt, true);
  if (!staged) SRBE_CUDA(cudaStreamWaitEvent(c->stream, c->ev_modes, 0));
  forces_pass(c, false, true);
  integrate_kick_drift(c, 0.5 * c->dt, false);
}

// one pass of the host-I/O force provider: mode list from the slot (side stream), positions from the
// caller's mapped buffer, the full force pass, the non-finite check, forces and charges back
void provider_step(srbe_ctx *c, int slot) {
  Extra *e = extra(c);
  const int K = c->K;
  SRBE_REQUIRE(c->dm.cap > (size_t)K && c->dc.cap >= (size_t)K && e->slot[slot].dhm && e->io_dr, SRBE_ESTATE,
               "buffers not reserved for the force provider");
  SRBE_CUDA(cudaEventRecord(c->ev_fork, c->stream));
  SRBE_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
  k_stage_modes<<<std::min(blocks_for((int64_t)K + 1, 256), 64u), 256, 0, c->side>>>(K, e->slot[slot].dhm,
                                                                                     e->slot[slot].dhw, c->dm.p,
                                                                                     c->dc.p);
  SRBE_CUDA(cudaEventRecord(c->ev_modes, c->side));
  uint64_t *iu = c->iu.ensure((size_t)3 * std::max<int64_t>(c->ni, 1));
  const double3 invL = make_double3(1.0 / c->L[0], 1.0 / c->L[1], 1.0 / c->L[2]);
  k_io_load<<<blocks_for(std::max<int64_t>(c->ni, 1), 64), 64, 0, c->stream>>>(
      c->ni, e->io_dr, c->L[0], c->L[1], invL, c->x.p, c->y.p, c->z.p, iu, c->d_status);
  c->launches += 2;
  SRBE_CUDA(cudaGetLastError());
  SRBE_CUDA(cudaStreamWaitEvent(c->stream, c->ev_modes, 0));
  forces_pass(c, false, true);
  check_finite(c, true, true);
  const int64_t nt = std::max<int64_t>(std::max<int64_t>(c->ni, c->ne), 1);
  k_io_store<<<std::min(blocks_for(nt, 256), 304u), 256, 0, c->stream>>>(c->ni, c->F.p, e->io_dF, c->ne, c->Q.p,
                                                                         e->io_dQ, c->scal.p, e->io_dpsi);
  c->launches++;
  SRBE_CUDA(cudaGetLastError());
}

void ensure_slot_buffers(srbe_ctx *c) {
  Extra *e = extra(c);
  SRBE_CUDA(cudaStreamSynchronize(c->stream));
  if (e->slot_cap < c->K) {
    for (auto &sl : e->slot) {
      if (sl.hm) cudaFreeHost(sl.hm);
      if (sl.hw) cudaFreeHost(sl.hw);
      sl.hm = nullptr;
      sl.hw = nullptr;
      sl.dhm = nullptr;
      sl.dhw = nullptr;
    }
    e->slot_cap = 0;
  }
  for (auto &sl : e->slot) {
    if (!sl.hm) {
      SRBE_CUDA(cudaHostAlloc((void **)&sl.hm, sizeof(int4) * (std::max(c->K, 1) + 1), cudaHostAllocMapped));
      SRBE_CUDA(cudaHostGetDevicePointer((void **)&sl.dhm, sl.hm, 0));
    }
    if (!sl.hw) {
      SRBE_CUDA(cudaHostAlloc((void **)&sl.hw, sizeof(double) * std::max(c->K, 1), cudaHostAllocMapped));
      SRBE_CUDA(cudaHostGetDevicePointer((void **)&sl.dhw, sl.hw, 0));
    }
    if (!sl.done) {
      SRBE_CUDA(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
      SRBE_CUDA(cudaEventRecord(sl.done, c->stream));
    }
  }
  e->slot_cap = std::max(e->slot_cap, std::max(c->K, 1));
}

void copy_to_slot(srbe_ctx *c, int slot) {
  Extra *e = extra(c);
  SRBE_REQUIRE((int)c->hc.size() == c->K && c->K <= e->slot_cap, SRBE_ESTATE, "mode count changed under a graph");
  for (int k = 0; k < c->K; ++k) {
    e->slot[slot].hm[k] = make_int4(c->hm[4 * k], c->hm[4 * k + 1], c->hm[4 * k + 2], 0);
    e->slot[slot].hw[k] = c->hc[k];
  }
  e->slot[slot].hm[c->K] = step_word(c->md_step);
}

void fill_slot(srbe_ctx *c, int slot) {
  SRBE_CUDA(cudaEventSynchronize(extra(c)->slot[slot].done));
  copy_to_slot(c, slot);
}

// Captures device_step (provider: provider_step) of every context in ctxs into one executable graph
// per slot.  With width 0
// all run in order on the capture stream; otherwise context r runs on forks[r % width], forked from
// and joined back into the capture stream, so that up to width replicas overlap on the GPU.  The
// cooperative kernels of all of them are chained through one capture-local event, so no two of them
// ever run at the same time.  kernels[r] receives the kernels one replay runs for context r.
// Returns false (and leaves nothing captured) when capture is not possible.
bool capture_graphs(srbe_ctx *const *ctxs, int n, cudaStream_t main, int width, const cudaStream_t *forks,
                    cudaGraphExec_t out[2], int64_t *kernels, DevBuf<StageEntry> *stage_tabs,
                    bool provider = false) {
  std::vector<int64_t> launches0(n);
  for (int r = 0; r < n; ++r) launches0[r] = ctxs[r]->launches;
  std::vector<cudaStream_t> saved(n);
  for (int r = 0; r < n; ++r) saved[r] = ctxs[r]->stream;
  cudaEvent_t fork_ev = nullptr, chain = nullptr;
  std::vector<cudaEvent_t> join(n, nullptr);
  auto release = [&] {
    for (int r = 0; r < n; ++r) {
      ctxs[r]->stream = saved[r];
      ctxs[r]->coop_chain = nullptr;
    }
    if (fork_ev) cudaEventDestroy(fork_ev);
    if (chain) cudaEventDestroy(chain);
    for (auto &j : join)
      if (j) cudaEventDestroy(j);
  };
  bool ok = cudaEventCreateWithFlags(&fork_ev, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&chain, cudaEventDisableTiming) == cudaSuccess;
  for (auto &j : join) ok = ok && cudaEventCreateWithFlags(&j, cudaEventDisableTiming) == cudaSuccess;
  out[0] = out[1] = nullptr;
  for (int slot = 0; slot < 2 && ok; ++slot) {
    cudaGraph_t g = nullptr;
    // with stage tables, every context's mode list of this slot comes in through one kernel at the
    // head of the graph (its pointers are fixed while the graph lives)
    if (stage_tabs) {
      try {
        std::vector<StageEntry> h(n);
        for (int r = 0; r < n; ++r) {
          srbe_ctx *c = ctxs[r];
          const auto &sl = extra(c)->slot[slot];
          SRBE_REQUIRE(sl.dhm && c->dm.cap > (size_t)c->K && c->dc.cap >= (size_t)c->K, SRBE_ESTATE,
                       "mode buffers not reserved for a captured step");
          h[r] = StageEntry{sl.dhm, sl.dhw, c->dm.p, c->dc.p, c->K};
        }
        StageEntry *d = stage_tabs[slot].ensure(n);
        SRBE_CUDA(cudaMemcpy(d, h.data(), sizeof(StageEntry) * n, cudaMemcpyHostToDevice));
      } catch (const Error &) {
        ok = false;
        break;
      }
    }
    if (cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      ok = false;
      break;
    }
    try {
      if (stage_tabs) {
        k_stage_many<<<n, 256, 0, main>>>(stage_tabs[slot].p);
        SRBE_CUDA(cudaGetLastError());
      }
      SRBE_CUDA(cudaEventRecord(chain, main));
      SRBE_CUDA(cudaEventRecord(fork_ev, main));
      for (int r = 0; r < n; ++r) {
        srbe_ctx *c = ctxs[r];
        c->coop_chain = chain;
        if (width > 0) {
          c->stream = forks[r % width];
          SRBE_CUDA(cudaStreamWaitEvent(c->stream, fork_ev, 0));
        } else {
          c->stream = main;
        }
        const int64_t l0 = c->launches;
        if (provider) provider_step(c, slot);
        else device_step(c, slot, stage_tabs != nullptr);
        kernels[r] = c->launches - l0 + (stage_tabs && r == 0 ? 1 : 0);
        if (width > 0) {
          SRBE_CUDA(cudaEventRecord(join[r], c->stream));
          SRBE_CUDA(cudaStreamWaitEvent(main, join[r], 0));
        }
        c->stream = saved[r];
        c->coop_chain = nullptr;
      }
    } catch (const Error &) {
      ok = false;
    }
    const cudaError_t ec = cudaStreamEndCapture(main, &g);
    if (!ok || ec != cudaSuccess || !g || cudaGraphInstantiate(&out[slot], g, 0) != cudaSuccess) ok = false;
    if (g) cudaGraphDestroy(g);
  }
  release();
  // capturing launches nothing
  for (int r = 0; r < n; ++r) ctxs[r]->launches = launches0[r];
  if (!ok) {
    cudaGetLastError();
    for (int k = 0; k < 2; ++k)
      if (out[k]) cudaGraphExecDestroy(out[k]);
    out[0] = out[1] = nullptr;
  }
  return ok;
}

void require_state(srbe_ctx *c, bool pos) {
  SRBE_REQUIRE(c->have_ele, SRBE_ESTATE, "srbe_set_electrode has not been called");
  if (pos) SRBE_REQUIRE(c->have_pos, SRBE_ESTATE, "srbe_set_positions has not been called");
  SRBE_REQUIRE(c->have_modes, SRBE_ESTATE, "no mode list: call srbe_sample_k, srbe_set_k or srbe_set_mode_list");
}

// after_drift: this step's drift has just written the ions' phase coordinates (c->iu)
void charges_pass(srbe_ctx *c, bool after_drift) {
  reserve(c);
  // the neighbour refresh / rebuild (reads x, y, z; writes the sorted copies and lists) runs on the
  // context's side stream beside S1 (reads x, y, z, q) and joins before b, which needs both
  SRBE_CUDA(cudaEventRecord(c->ev_fork, c->stream));
  SRBE_CUDA(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
  const cudaStream_t main = c->stream;
  c->stream = c->side;
  try {
    phase_begin(c, kPhCells);
    neighbor_update(c);
    phase_end(c, kPhCells);
  } catch (...) {
    c->stream = main;
    throw;
  }
  c->stream = main;
  SRBE_CUDA(cudaEventRecord(c->ev_join, c->side));
  phase_begin(c, kPhS1);
  structure_factor(c, c->ni, c->x.p, c->y.p, c->z.p, c->q.p, c->S1.p, nullptr, kScalMion, 0,
                   after_drift ? c->iu.p : nullptr, c->q32.p);
  phase_end(c, kPhS1);
  SRBE_CUDA(cudaStreamWaitEvent(c->stream, c->ev_join, 0));
  phase_begin(c, kPhRhs);
  electrode_rhs(c);
  phase_end(c, kPhRhs);
  phase_begin(c, kPhSolve);
  charge_update(c);
  phase_end(c, kPhSolve);
  // test aid: a NaN in Q[0] before anything reads the charges
  if (c->inject == 2 && c->ne > 0) {
    SRBE_CUDA(cudaMemsetAsync(c->Q.p, 0xff, sizeof(double), c->stream));
    SRBE_CUDA(cudaMemsetAsync(c->Q32.p, 0xff, sizeof(float), c->stream));
  }
}

// check: non-finite forces and charges raise the context's flag (the MD step checks them in its
// closing half kick instead, after_drift; the minimiser tolerates overflowing forces)
void forces_pass(srbe_ctx *c, bool energies, bool after_drift, bool check) {
  charges_pass(c, after_drift);
  if (ion_forces_split(c, energies)) {
    // the ion-ion pairs on the side stream, behind the neighbour update, beside b / solve / S2
    const cudaStream_t main = c->stream;
    c->stream = c->side;
    try {
      phase_begin(c, kPhForcesII);
      ion_forces_ii(c);
      phase_end(c, kPhForcesII);
    } catch (...) {
      c->stream = main;
      throw;
    }
    c->stream = main;
  }
  phase_begin(c, kPhS2);
  if (c->lat.active(c->ne, c->K)) lattice_s2(c, c->S2.p, c->S1.p, kScalMele);
  else structure_factor(c, c->ne, c->ex.p, c->ey.p, c->ez.p, c->Q.p, c->S2.p, c->S1.p, kScalMele, 1, c->eu.p, c->Q32.p);
  phase_end(c, kPhS2);
  phase_begin(c, kPhForces);
  ion_forces(c, energies);
  phase_end(c, kPhForces);
  // test aid: a NaN in F[0] before the check
  if (c->inject == 1 && c->ni > 0) SRBE_CUDA(cudaMemsetAsync(c->F.p, 0xff, sizeof(double), c->stream));
  if (check && !after_drift) check_finite(c, true, true);
  if (energies) {
    phase_begin(c, kPhEnergy);
    energy_scalars(c);
    phase_end(c, kPhEnergy);
  }
}

// host half of a step's mode list: samples (Eqs. 26-29) and weights (Eqs. 24-25) into c->hm / c->hc
void build_host_list(srbe_ctx *c, uint64_t seed, uint64_t step) {
  Extra *e = extra(c);
  std::vector<int32_t> smp((size_t)3 * c->P);
  if (c->sampler == SRBE_SAMPLER_EXACT) e->sampler.exact(seed, step, c->P, smp.data());
  else e->sampler.metropolis(seed, step, c->P, smp.data());
  srbe_host_list(c, smp.data(), c->P);
}

void sample_into(srbe_ctx *c, uint64_t seed, uint64_t step) {
  build_host_list(c, seed, step);
  upload_modes(c);
}

// forces at the starting positions (modes of step md_step), once after any change of the state
void initial_forces(srbe_ctx *c, uint64_t seed0) {
  Extra *e = extra(c);
  if (e->forces_valid) return;
  sample_into(c, seed0, c->md_step);
  forces_pass(c, false);
  e->forces_valid = true;
}

// one velocity-Verlet step of Algorithm 1 through ordinary launches
void eager_step(srbe_ctx *c, uint64_t seed0) {
  c->md_step++;
  sample_into(c, seed0, c->md_step);
  phase_begin(c, kPhIntegrate);
  integrate_kick_drift(c, 0.5 * c->dt, true);
  phase_end(c, kPhIntegrate);
  forces_pass(c, false, true);
  phase_begin(c, kPhIntegrate);
  integrate_kick_drift(c, 0.5 * c->dt, false);
  phase_end(c, kPhIntegrate);
}


// Reports (throws) and clears the device-raised flags: after the work that may raise them has
// finished, or (srbe_step) for whatever the host already sees, without waiting.  notconv = false
// leaves an unconverged iterative solve (whose pass fell back to the direct solve) raised for a later
// call, so that MD keeps stepping.
void report_status(srbe_ctx *c, bool notconv = true) {
  volatile int *h = c->h_status;
  if (!h) return;
  const int nc = notconv ? h[kStatNotConv] : 0, nf = h[kStatNonFiniteF], nq = h[kStatNonFiniteQ],
            nb = h[kStatBadInput], nt = h[kStatTimeout];
  if (!(nc | nf | nq | nb | nt)) return;
  if (notconv) h[kStatNotConv] = 0;
  if (nt) {
    h[kStatTimeout] = 0;
    throw Error{SRBE_ETIMEOUT, "a tensor-core MMA did not complete within its wait limit (its outputs are invalid)"};
  }
  h[kStatNonFiniteF] = 0;
  h[kStatNonFiniteQ] = 0;
  h[kStatBadInput] = 0;
  if (nb)
    throw Error{SRBE_EINVAL, "non-finite position in the host input buffer (replaced by the origin for that pass)"};
  if (nf || nq)
    throw Error{SRBE_ENONFINITE, std::string("non-finite ") + (nf && nq ? "forces and electrode charges"
                                                               : nf   ? "forces"
                                                                      : "electrode charges") +
                                     (nc ? " (and an iterative solve stopped at maxit)" : "")};
  throw Error{SRBE_ENOTCONV, "PCG charge solve stopped at maxit above its tolerance; the charges of that pass "
                             "come from the direct solve"};
}

void download_outputs(srbe_ctx *c, double *F, double *Q, double *psi, double *energy, double *b) {
  Extra *e = extra(c);
  if (F && c->ni > 0) {
    double *aos = e->aos.ensure((size_t)3 * c->ni);
    k_interleave<<<blocks_for(c->ni, 256), 256, 0, c->stream>>>(c->ni, c->F.p, aos);
    c->launches++;
    SRBE_CUDA(cudaGetLastError());
    SRBE_CUDA(cudaMemcpyAsync(F, aos, sizeof(double) * 3 * c->ni, cudaMemcpyDeviceToHost, c->stream));
  }
  if (Q) SRBE_CUDA(cudaMemcpyAsync(Q, c->Q.p, sizeof(double) * c->ne, cudaMemcpyDeviceToHost, c->stream));
  if (b) SRBE_CUDA(cudaMemcpyAsync(b, c->bvec.p, sizeof(double) * c->ne, cudaMemcpyDeviceToHost, c->stream));
  SRBE_CUDA(cudaMemcpyAsync(c->h_scal, c->scal.p, sizeof(double) * kScalCount, cudaMemcpyDeviceToHost, c->stream));
  SRBE_CUDA(cudaStreamSynchronize(c->stream));
  if (b)
    for (int64_t j = 0; j < c->ne; ++j) b[j] /= kVolt;
  if (psi) *psi = c->h_scal[kScalPsi] / kVolt;
  if (energy) {
    const double *s = c->h_scal;
    const double Mz = s[kScalMion] + s[kScalMele];
    const double self = (1.0 / (std::sqrt(2.0 * kPi) * c->eta) - c->alpha / std::sqrt(kPi)) * s[kScalQ2] -
                        c->alpha / std::sqrt(kPi) * s[kScalq2];
    energy[0] = kKeHost * s[kScalEii];
    energy[1] = kKeHost * s[kScalEie];
    energy[2] = kKeHost * s[kScalEee];
    energy[3] = kKeHost * s[kScalUF];
    energy[4] = kKeHost * self;
    energy[5] = kKeHost * 2.0 * kPi / c->V * Mz * Mz;
    energy[6] = s[kScalElj];
    energy[7] = s[kScalEbond];
  }
}

}  // namespace

// ================================================================================================
// C ABI
// ================================================================================================
extern "C" {

int srbe_create(const double box[3], double alpha, double eta, double rc, int P, int kz0, double psi_left,
                double psi_right, srbe_ctx **out) {
  if (!out) return SRBE_EINVAL;
  *out = nullptr;
  if (!box || !(box[0] > 0) || !(box[1] > 0) || !(box[2] > 0) || !std::isfinite(box[0]) || !std::isfinite(box[1]) ||
      !std::isfinite(box[2]) || !(alpha > 0) || !(eta > 0) || !(rc > 0) || P < 0 || kz0 < 0 || (int64_t)P + kz0 > kMaxModes ||
      !std::isfinite(psi_left) || !std::isfinite(psi_right) || !std::isfinite(alpha) || !std::isfinite(eta) ||
      !std::isfinite(rc))
    return SRBE_EINVAL;
  srbe_ctx *c = new (std::nothrow) srbe_ctx();
  if (!c) return SRBE_ENOMEM;
  c->hx = new (std::nothrow) srbe::HostExt();
  if (!c->hx) {
    delete c;
    return SRBE_ENOMEM;
  }
  for (int d = 0; d < 3; ++d) c->L[d] = box[d];
  c->V = box[0] * box[1] * box[2];
  c->alpha = alpha;
  c->eta = eta;
  c->rc = rc;
  c->P = P;
  c->M = kz0;
  c->psi_left = psi_left;
  c->psi_right = psi_right;
  c->dpsi = (psi_right - psi_left) * kVolt;
  int rcode = guarded(c, [&] {
    c->stream = make_stream(true);
    c->own_stream = true;
    SRBE_CUDA(cudaEventCreateWithFlags(&c->stage_done, cudaEventDisableTiming));
    SRBE_CUDA(cudaEventRecord(c->stage_done, c->stream));
    c->side = make_stream(false);
    SRBE_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    SRBE_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    SRBE_CUDA(cudaEventCreateWithFlags(&c->ev_modes, cudaEventDisableTiming));
    SRBE_CUDA(cudaEventCreateWithFlags(&c->ev_ii, cudaEventDisableTiming));
    upload_table(c);
    SRBE_CUDA(cudaHostAlloc((void **)&c->h_status, sizeof(int) * kStatCount, cudaHostAllocMapped));
    std::memset(c->h_status, 0, sizeof(int) * kStatCount);
    SRBE_CUDA(cudaHostGetDevicePointer((void **)&c->d_status, c->h_status, 0));
    c->scal.ensure(kScalCount);
    SRBE_CUDA(cudaMemsetAsync(c->scal.p, 0, sizeof(double) * kScalCount, c->stream));
    c->hx->sampler.init(c->L, c->alpha, c->M, c->mmax);
    c->G = c->hx->sampler.G();
  });
  if (rcode != SRBE_OK) {
    srbe_destroy(c);
    return rcode;
  }
  *out = c;
  return SRBE_OK;
}

int srbe_destroy(srbe_ctx *c) {
  if (!c) return SRBE_OK;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->h_mode_stage) cudaFreeHost(c->h_mode_stage);
  if (c->h_w_stage) cudaFreeHost(c->h_w_stage);
  if (c->side) cudaStreamSynchronize(c->side);
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->stage_done) cudaEventDestroy(c->stage_done);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_modes) cudaEventDestroy(c->ev_modes);
  if (c->ev_ii) cudaEventDestroy(c->ev_ii);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  c->stream = nullptr;
  delete c->hx;
  c->hx = nullptr;
  delete c;
  return SRBE_OK;
}

const char *srbe_last_error(const srbe_ctx *c) { return c ? c->err.c_str() : "null context"; }

int srbe_set_stream(srbe_ctx *c, void *stream) {
  return guarded(c, [&] {
    SRBE_CUDA(cudaStreamSynchronize(c->stream));
    if (stream) {
      if (c->own_stream) SRBE_CUDA(cudaStreamDestroy(c->stream));
      c->stream = (cudaStream_t)stream;
      c->own_stream = false;
    } else if (!c->own_stream) {
      c->stream = make_stream(true);
      c->own_stream = true;
    }
    SRBE_CUDA(cudaEventRecord(c->stage_done, c->stream));
  });
}

int srbe_set_precision(srbe_ctx *c, int mode) {
  return guarded(c, [&] {
    SRBE_REQUIRE(mode == SRBE_FP64 || mode == SRBE_MIXED, SRBE_EINVAL, "unknown precision mode");
    c->precision = mode;
  });
}

int srbe_set_A_params(srbe_ctx *c, double alpha_A, double tol) {
  return guarded(c, [&] {
    SRBE_REQUIRE(std::isfinite(alpha_A) && std::isfinite(tol) && tol < 1.0, SRBE_EINVAL, "bad A parameters");
    SRBE_REQUIRE(!c->have_ele, SRBE_ESTATE, "A parameters must be set before srbe_set_electrode");
    c->alpha_A = alpha_A;
    c->tol_A = tol;
  });
}

int srbe_set_electrode(srbe_ctx *c, int64_t n_ele, const double *R, const int8_t *side) {
  return guarded(c, [&] {
    SRBE_REQUIRE(R && side && n_ele >= 2, SRBE_EINVAL, "need at least two electrode sites");
    SRBE_REQUIRE(n_ele <= (1 << 22), SRBE_EINVAL, "at most 4,194,304 electrode sites are supported");
    SRBE_REQUIRE(finite_all(R, 3 * n_ele), SRBE_EINVAL, "non-finite electrode position");
    int64_t nl = 0, nr = 0;
    for (int64_t j = 0; j < n_ele; ++j) {
      SRBE_REQUIRE(side[j] == 0 || side[j] == 1, SRBE_EINVAL, "side must be 0 (left) or 1 (right)");
      (side[j] ? nr : nl)++;
    }
    SRBE_REQUIRE(nl > 0 && nr > 0, SRBE_EINVAL, "both electrodes need at least one site");
    c->ne = n_ele;
    c->hR.assign(R, R + 3 * n_ele);
    c->hside.assign(side, side + n_ele);
    std::vector<double> x(n_ele), y(n_ele), z(n_ele), d(n_ele);
    for (int64_t j = 0; j < n_ele; ++j) {
      double X = R[3 * j], Y = R[3 * j + 1];
      X -= c->L[0] * std::floor(X / c->L[0]);
      Y -= c->L[1] * std::floor(Y / c->L[1]);
      if (X >= c->L[0]) X -= c->L[0];
      if (Y >= c->L[1]) Y -= c->L[1];
      x[j] = X;
      y[j] = Y;
      z[j] = R[3 * j + 2];
      d[j] = side[j] ? 0.5 : -0.5;
    }
    c->ex.ensure(n_ele);
    c->ey.ensure(n_ele);
    c->ez.ensure(n_ele);
    c->ed.ensure(n_ele);
    c->Q.ensure(n_ele);
    c->bvec.ensure(n_ele);
    SRBE_CUDA(cudaMemcpyAsync(c->ex.p, x.data(), sizeof(double) * n_ele, cudaMemcpyHostToDevice, c->stream));
    SRBE_CUDA(cudaMemcpyAsync(c->ey.p, y.data(), sizeof(double) * n_ele, cudaMemcpyHostToDevice, c->stream));
    SRBE_CUDA(cudaMemcpyAsync(c->ez.p, z.data(), sizeof(double) * n_ele, cudaMemcpyHostToDevice, c->stream));
    SRBE_CUDA(cudaMemcpyAsync(c->ed.p, d.data(), sizeof(double) * n_ele, cudaMemcpyHostToDevice, c->stream));
    SRBE_CUDA(cudaMemsetAsync(c->Q.p, 0, sizeof(double) * n_ele, c->stream));
    // one cell grid for ions and electrode sites: the whole periodic length in z, centred on the walls
    const double zmin = *std::min_element(z.begin(), z.end()), zmax = *std::max_element(z.begin(), z.end());
    const double pad = 0.5 * (c->L[2] - (zmax - zmin));
    c->wall_span = zmax - zmin;
    choose_grid(c, c->ecells.g, zmin - pad, zmax + pad);
    c->icells.g = c->ecells.g;
    build_run_table(c);
    build_cells(c, c->ecells, n_ele, c->ex.p, c->ey.p, c->ez.p, nullptr, nullptr, nullptr, false);
    c->eu.ensure(3 * (size_t)n_ele);
    k_site_turns<<<blocks_for(n_ele, 256), 256, 0, c->stream>>>(n_ele, c->ex.p, c->ey.p, c->ez.p,
                                                               make_double3(1.0 / c->L[0], 1.0 / c->L[1],
                                                                            1.0 / c->L[2]),
                                                               c->eu.p);
    k_site_f4<<<blocks_for(n_ele, 256), 256, 0, c->stream>>>(n_ele, c->ex.p, c->ey.p, c->ez.p,
                                                            c->epf.ensure((size_t)n_ele));
    SRBE_CUDA(cudaGetLastError());
    lattice_setup(c, x, y, z);
    build_A_and_inverse(c);
    c->have_ele = true;
    extra(c)->forces_valid = false;
  });
}

int srbe_set_positions(srbe_ctx *c, int64_t n_ion, const double *r, const double *q) {
  return guarded(c, [&] {
    SRBE_REQUIRE(n_ion >= 0 && (n_ion == 0 || (r && q)), SRBE_EINVAL, "null positions or charges");
    SRBE_REQUIRE(n_ion < (1ll << 23), SRBE_EINVAL, "at most 8,388,607 ions are supported");
    SRBE_REQUIRE(finite_all(r, 3 * n_ion) && finite_all(q, n_ion), SRBE_EINVAL, "non-finite ion position or charge");
    if (c->have_md && n_ion != c->ni) c->have_md = false;
    if (n_ion != c->ni) c->nbr.cap = 0;
    Extra *e = extra(c);
    // the same ions with the same charges (an MD engine handing in each step's positions) keep their
    // Verlet lists: the per-step refresh rebuilds them once some ion has moved more than half the
    // skin since the last build.  Anything else (new count, new charges, first call) rebuilds.
    const bool same_ions = c->have_pos && n_ion == c->ni && e->hq.size() == (size_t)n_ion &&
                           std::equal(q, q + n_ion, e->hq.begin());
    c->ni = n_ion;
    const size_t n = (size_t)std::max<int64_t>(n_ion, 1);
    c->x.ensure(n);
    c->y.ensure(n);
    c->z.ensure(n);
    c->q.ensure(n);
    c->F.ensure(3 * n);
    if (!same_ions) {
      neighbor_force_rebuild(c);
      e->hq.assign(q, q + n_ion);
    }
    if (n_ion > 0) {
      double *aos = e->aos.ensure(3 * n);
      SRBE_CUDA(cudaMemcpyAsync(aos, r, sizeof(double) * 3 * n_ion, cudaMemcpyHostToDevice, c->stream));
      SRBE_CUDA(cudaMemcpyAsync(c->q.p, q, sizeof(double) * n_ion, cudaMemcpyHostToDevice, c->stream));
      k_to_f32<<<blocks_for(n_ion, 256), 256, 0, c->stream>>>(n_ion, c->q.p, c->q32.ensure(n));
      c->launches++;
      k_deinterleave<<<blocks_for(n_ion, 256), 256, 0, c->stream>>>(n_ion, aos, c->L[0], c->L[1], c->x.p, c->y.p,
                                                                   c->z.p);
      c->launches++;
      SRBE_CUDA(cudaGetLastError());
    }
    c->have_pos = true;
    e->forces_valid = false;
  });
}

int srbe_set_positions_dev(srbe_ctx *c, int64_t n_ion, const double *r_dev, const double *q_dev) {
  return guarded(c, [&] {
    SRBE_REQUIRE(n_ion >= 0 && (n_ion == 0 || (r_dev && q_dev)), SRBE_EINVAL, "null positions or charges");
    SRBE_REQUIRE(n_ion < (1ll << 23), SRBE_EINVAL, "at most 8,388,607 ions are supported");
    if (c->have_md && n_ion != c->ni) c->have_md = false;
    if (n_ion != c->ni) c->nbr.cap = 0;
    c->ni = n_ion;
    neighbor_force_rebuild(c);
    extra(c)->hq.clear();   // charges from device memory: the next host call rebuilds
    const size_t n = (size_t)std::max<int64_t>(n_ion, 1);
    c->x.ensure(n);
    c->y.ensure(n);
    c->z.ensure(n);
    c->q.ensure(n);
    c->F.ensure(3 * n);
    if (n_ion > 0) {
      SRBE_CUDA(cudaMemcpyAsync(c->q.p, q_dev, sizeof(double) * n_ion, cudaMemcpyDeviceToDevice, c->stream));
      k_to_f32<<<blocks_for(n_ion, 256), 256, 0, c->stream>>>(n_ion, c->q.p, c->q32.ensure(n));
      c->launches++;
      k_deinterleave<<<blocks_for(n_ion, 256), 256, 0, c->stream>>>(n_ion, r_dev, c->L[0], c->L[1], c->x.p, c->y.p,
                                                                   c->z.p);
      c->launches++;
      SRBE_CUDA(cudaGetLastError());
    }
    c->have_pos = true;
    extra(c)->forces_valid = false;
  });
}

int srbe_get_positions(srbe_ctx *c, double *r, double *v) {
  return guarded(c, [&] {
    SRBE_REQUIRE(c->have_pos, SRBE_ESTATE, "no positions");
    if (c->ni == 0) return;
    double *aos = extra(c)->aos.ensure((size_t)3 * c->ni);
    if (r) {
      k_interleave3<<<blocks_for(c->ni, 256), 256, 0, c->stream>>>(c->ni, c->x.p, c->y.p, c->z.p, aos);
      SRBE_CUDA(cudaMemcpyAsync(r, aos, sizeof(double) * 3 * c->ni, cudaMemcpyDeviceToHost, c->stream));
      SRBE_CUDA(cudaStreamSynchronize(c->stream));
    }
    if (v) {
      SRBE_REQUIRE(c->have_md, SRBE_ESTATE, "no velocities (srbe_set_md)");
      k_interleave3<<<blocks_for(c->ni, 256), 256, 0, c->stream>>>(c->ni, c->vx.p, c->vy.p, c->vz.p, aos);
      SRBE_CUDA(cudaMemcpyAsync(v, aos, sizeof(double) * 3 * c->ni, cudaMemcpyDeviceToHost, c->stream));
      SRBE_CUDA(cudaStreamSynchronize(c->stream));
    }
  }, true);
}

int srbe_set_md(srbe_ctx *c, const double *mass, const double *v, int ntype, const int32_t *itype,
                const int32_t *mol, const double *lj_sigma, const double *lj_eps, int64_t nb, const int32_t *bonds,
                const double *r0, double kb, double dt) {
  return guarded(c, [&] {
    SRBE_REQUIRE(c->have_pos, SRBE_ESTATE, "srbe_set_md needs srbe_set_positions first");
    SRBE_CUDA(cudaStreamSynchronize(c->stream));
    const int64_t n = c->ni;
    SRBE_REQUIRE(n == 0 || (mass && itype && mol), SRBE_EINVAL, "null mass / type / molecule array");
    SRBE_REQUIRE(ntype >= 1 && ntype <= 16 && lj_sigma && lj_eps, SRBE_EINVAL, "bad LJ tables");
    SRBE_REQUIRE(nb >= 0 && (nb == 0 || (bonds && r0)), SRBE_EINVAL, "bad bond list");
    SRBE_REQUIRE(dt > 0 && std::isfinite(dt) && std::isfinite(kb), SRBE_EINVAL, "bad dt or kb");
    std::vector<double> minv(n), lj(2 * ntype * ntype);
    for (int64_t i = 0; i < n; ++i) {
      SRBE_REQUIRE(mass[i] > 0 && std::isfinite(mass[i]), SRBE_EINVAL, "masses must be positive");
      SRBE_REQUIRE(itype[i] >= 0 && itype[i] < ntype - 1, SRBE_EINVAL, "ion type out of range");
      minv[i] = 1.0 / mass[i];
    }
    for (int a = 0; a < ntype * ntype; ++a) {
      lj[2 * a] = lj_sigma[a] * lj_sigma[a];
      lj[2 * a + 1] = lj_eps[a];
    }
    // bonds as a CSR list per ion (each bond stored from both ends)
    std::vector<int32_t> start(n + 1, 0), bj(2 * nb);
    std::vector<double> br(2 * nb);
    for (int64_t b = 0; b < nb; ++b) {
      SRBE_REQUIRE(bonds[2 * b] >= 0 && bonds[2 * b] < n && bonds[2 * b + 1] >= 0 && bonds[2 * b + 1] < n &&
                       bonds[2 * b] != bonds[2 * b + 1],
                   SRBE_EINVAL, "bond index out of range");
      start[bonds[2 * b] + 1]++;
      start[bonds[2 * b + 1] + 1]++;
    }
    for (int64_t i = 0; i < n; ++i) start[i + 1] += start[i];
    std::vector<int32_t> fill(start.begin(), start.end() - 1);
    for (int64_t b = 0; b < nb; ++b) {
      const int32_t i = bonds[2 * b], j = bonds[2 * b + 1];
      bj[fill[i]] = j;
      br[fill[i]++] = r0[b];
      bj[fill[j]] = i;
      br[fill[j]++] = r0[b];
    }
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    c->vx.ensure(nn);
    c->vy.ensure(nn);
    c->vz.ensure(nn);
    c->minv.ensure(nn);
    c->itype.ensure(nn);
    c->mol.ensure(nn);
    c->lj.ensure(lj.size());
    c->bond_start.ensure(n + 1);
    c->bond_j.ensure(std::max<int64_t>(2 * nb, 1));
    c->bond_r0.ensure(std::max<int64_t>(2 * nb, 1));
    if (n > 0) {
      std::vector<double> vx(n, 0.0), vy(n, 0.0), vz(n, 0.0);
      if (v)
        for (int64_t i = 0; i < n; ++i) {
          vx[i] = v[3 * i];
          vy[i] = v[3 * i + 1];
          vz[i] = v[3 * i + 2];
        }
      SRBE_CUDA(cudaMemcpy(c->vx.p, vx.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
      SRBE_CUDA(cudaMemcpy(c->vy.p, vy.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
      SRBE_CUDA(cudaMemcpy(c->vz.p, vz.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
      SRBE_CUDA(cudaMemcpy(c->minv.p, minv.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
      SRBE_CUDA(cudaMemcpy(c->itype.p, itype, sizeof(int32_t) * n, cudaMemcpyHostToDevice));
      SRBE_CUDA(cudaMemcpy(c->mol.p, mol, sizeof(int32_t) * n, cudaMemcpyHostToDevice));
    }
    SRBE_CUDA(cudaMemcpy(c->lj.p, lj.data(), sizeof(double) * lj.size(), cudaMemcpyHostToDevice));
    std::vector<float> lj32(lj.begin(), lj.end());
    c->lj32.ensure(lj32.size() / 2);
    SRBE_CUDA(cudaMemcpy(c->lj32.p, lj32.data(), sizeof(float) * lj32.size(), cudaMemcpyHostToDevice));
    SRBE_CUDA(cudaMemcpy(c->bond_start.p, start.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice));
    if (nb > 0) {
      SRBE_CUDA(cudaMemcpy(c->bond_j.p, bj.data(), sizeof(int32_t) * 2 * nb, cudaMemcpyHostToDevice));
      SRBE_CUDA(cudaMemcpy(c->bond_r0.p, br.data(), sizeof(double) * 2 * nb, cudaMemcpyHostToDevice));
    }
    c->ntype = ntype;
    c->kb = kb;
    c->dt = dt;
    c->have_md = true;
    neighbor_force_rebuild(c);
    extra(c)->forces_valid = false;
  });
}

int srbe_set_sampler(srbe_ctx *c, int kind, const int32_t *mmax) {
  return guarded(c, [&] {
    SRBE_REQUIRE(kind == SRBE_SAMPLER_METROPOLIS || kind == SRBE_SAMPLER_EXACT, SRBE_EINVAL, "unknown sampler");
    c->sampler = kind;
    for (int d = 0; d < 3; ++d) c->mmax[d] = mmax ? std::max(mmax[d], 0) : 0;
    Extra *e = extra(c);
    e->sampler.init(c->L, c->alpha, c->M, c->mmax);
    c->G = e->sampler.G();
    if (e->dev_sampler) {
      if (kind == SRBE_SAMPLER_EXACT) upload_sampler_tables(c);
      else e->dev_sampler = false;
    }
  });
}

int srbe_sample_k(srbe_ctx *c, uint64_t seed, uint64_t step) {
  return guarded(c, [&] { sample_into(c, seed, step); });
}

int srbe_set_device_sampler(srbe_ctx *c, int on) {
  return guarded(c, [&] {
    Extra *e = extra(c);
    if (on) {
      SRBE_REQUIRE(c->sampler == SRBE_SAMPLER_EXACT, SRBE_EINVAL,
                   "the device sampler is the exact one: select SRBE_SAMPLER_EXACT first");
      upload_sampler_tables(c);
    }
    e->dev_sampler = on != 0;
  });
}

int srbe_sample_k_device(srbe_ctx *c, uint64_t seed, uint64_t step, int32_t *m, double *w) {
  return guarded(c, [&] {
    Extra *e = extra(c);
    SRBE_REQUIRE(e->dev_sampler, SRBE_ESTATE, "device sampler not enabled (srbe_set_device_sampler)");
    const int P = c->P, M = c->M;
    // the list's layout (I, then P samples, then the step word) with zero samples for the kernel to
    // overwrite
    std::vector<int32_t> zero((size_t)3 * P, 0);
    srbe_host_list(c, zero.data(), P);
    upload_modes(c);
    const int4 word = sample_word(step, seed);
    SRBE_CUDA(cudaMemcpyAsync(e->dev_step.p, &word, sizeof(int4), cudaMemcpyHostToDevice, c->stream));
    k_sample_exact<<<1, kSampleThreads, 0, c->stream>>>(dev_sample_args(c, e->dev_step.p));
    c->launches++;
    SRBE_CUDA(cudaGetLastError());
    // the list's step word stays the MD step (the thermostat's), as after srbe_sample_k
    const int4 md = step_word(c->md_step);
    SRBE_CUDA(cudaMemcpyAsync(c->dm.p + c->K, &md, sizeof(int4), cudaMemcpyHostToDevice, c->stream));
    std::vector<int4> hm4((size_t)std::max(P, 1));
    std::vector<double> hw((size_t)std::max(P, 1));
    if (P > 0) {
      SRBE_CUDA(cudaMemcpyAsync(hm4.data(), c->dm.p + M, sizeof(int4) * P, cudaMemcpyDeviceToHost, c->stream));
      SRBE_CUDA(cudaMemcpyAsync(hw.data(), c->dc.p + M, sizeof(double) * P, cudaMemcpyDeviceToHost, c->stream));
    }
    SRBE_CUDA(cudaStreamSynchronize(c->stream));
    check_dev_sampler(c);
    // the host copy of the list follows the device's
    for (int l = 0; l < P; ++l) {
      const int32_t v[3] = {hm4[l].x, hm4[l].y, hm4[l].z};
      for (int d = 0; d < 3; ++d) {
        c->hm[4 * (M + l) + d] = v[d];
        c->hsamp[3 * l + d] = v[d];
        if (m) m[3 * l + d] = v[d];
      }
      c->hc[M + l] = hw[l];
      if (w) w[l] = hw[l];
    }
  });
}

int srbe_get_k(const srbe_ctx *cc, int32_t *m, double *G) {
  srbe_ctx *c = const_cast<srbe_ctx *>(cc);
  return guarded(c, [&] {
    SRBE_REQUIRE(c->have_modes && !c->explicit_list, SRBE_ESTATE, "no sampled mode list");
    if (m) std::memcpy(m, c->hsamp.data(), sizeof(int32_t) * c->hsamp.size());
    if (G) *G = c->G;
  }, true);
}

int srbe_set_k(srbe_ctx *c, const int32_t *m, int P) {
  return guarded(c, [&] {
    SRBE_REQUIRE(P >= 0 && (P == 0 || m), SRBE_EINVAL, "bad sampled-mode list");
    SRBE_REQUIRE((int64_t)P + c->M <= kMaxModes, SRBE_EINVAL, "too many modes (at most 2,097,120)");
    for (int l = 0; l < P; ++l)
      SRBE_REQUIRE(!(m[3 * l] == 0 && m[3 * l + 1] == 0 && std::abs(m[3 * l + 2]) <= c->M), SRBE_EINVAL,
                   "sampled mode lies in I u {0}");
    srbe_list_from_samples(c, m, P);
  });
}

int srbe_set_mode_list(srbe_ctx *c, const int32_t *m, const double *w, int K) {
  return guarded(c, [&] {
    SRBE_REQUIRE(K >= 0 && (K == 0 || (m && w)), SRBE_EINVAL, "bad mode list");
    SRBE_REQUIRE(K <= kMaxModes, SRBE_EINVAL, "too many modes (at most 2,097,120)");
    SRBE_REQUIRE(finite_all(w, K), SRBE_EINVAL, "non-finite mode weight");
    c->hm.clear();
    c->hc.assign(w, w + K);
    for (int k = 0; k < K; ++k) {
      SRBE_REQUIRE(m[3 * k] || m[3 * k + 1] || m[3 * k + 2], SRBE_EINVAL, "mode k = 0 is not allowed");
      c->hm.insert(c->hm.end(), {m[3 * k], m[3 * k + 1], m[3 * k + 2], 0});
    }
    c->Kdet = K;
    c->explicit_list = true;
    upload_modes(c);
  });
}

int srbe_solve_electrode_charges(srbe_ctx *c, double *Q, double *psi_bar, double *b) {
  return guarded(c, [&] {
    require_state(c, true);
    charges_pass(c, false);
    check_finite(c, false, true);
    download_outputs(c, nullptr, Q, psi_bar, nullptr, b);
    report_status(c);
  });
}

int srbe_forces(srbe_ctx *c, double *F, double *Q, double *psi_bar, double *energy) {
  return guarded(c, [&] {
    require_state(c, true);
    forces_pass(c, energy != nullptr);
    extra(c)->forces_valid = true;
    download_outputs(c, F, Q, psi_bar, energy, nullptr);
    report_status(c);
  });
}

int srbe_forces_dev(srbe_ctx *c, double *F_dev, double *Q_dev) {
  return guarded(c, [&] {
    require_state(c, true);
    forces_pass(c, false);
    extra(c)->forces_valid = true;
    if (F_dev && c->ni > 0) {
      k_interleave<<<blocks_for(c->ni, 256), 256, 0, c->stream>>>(c->ni, c->F.p, F_dev);
      c->launches++;
      SRBE_CUDA(cudaGetLastError());
    }
    if (Q_dev) SRBE_CUDA(cudaMemcpyAsync(Q_dev, c->Q.p, sizeof(double) * c->ne, cudaMemcpyDeviceToDevice, c->stream));
  });
}

int srbe_set_host_io(srbe_ctx *c, double *r, double *F, double *Q) {
  return guarded(c, [&] {
    SRBE_REQUIRE(c->have_ele && c->have_pos, SRBE_ESTATE, "electrode and positions (charges) are required");
    SRBE_REQUIRE(r && (F || c->ni == 0), SRBE_EINVAL, "null position or force buffer");
    Extra *e = extra(c);
    e->drop_io_graphs();
    // page-locked host memory (cudaHostAlloc or cudaHostRegister) only: plain pageable memory is
    // rejected even where the device could reach it
    auto dev_view = [](void *h, const char *what) {
      cudaPointerAttributes at{};
      if (cudaPointerGetAttributes(&at, h) != cudaSuccess || at.type != cudaMemoryTypeHost || !at.devicePointer) {
        cudaGetLastError();
        throw Error{SRBE_EINVAL, std::string(what) + " is not page-locked host memory mapped for the device "
                                                     "(allocate it with cudaHostAlloc or register it)"};
      }
      return at.devicePointer;
    };
    e->io_dr = (const double *)dev_view(r, "the position buffer");
    e->io_dF = F ? (double *)dev_view(F, "the force buffer") : nullptr;
    e->io_dQ = Q ? (double *)dev_view(Q, "the charge buffer") : nullptr;
    e->io_r = r;
    e->io_F = F;
    e->io_Q = Q;
    if (!e->io_psi) {
      SRBE_CUDA(cudaHostAlloc((void **)&e->io_psi, sizeof(double), cudaHostAllocMapped));
      SRBE_CUDA(cudaHostGetDevicePointer((void **)&e->io_dpsi, e->io_psi, 0));
    }
  });
}

int srbe_forces_host_io(srbe_ctx *c, uint64_t seed, uint64_t step, double *psi_bar) {
  return guarded(c, [&] {
    Extra *e = extra(c);
    SRBE_REQUIRE(e->io_dr, SRBE_ESTATE, "srbe_set_host_io has not been called");
    SRBE_REQUIRE(c->have_ele && c->have_pos, SRBE_ESTATE, "electrode and positions (charges) are required");
    report_status(c);                  // flags of earlier asynchronous calls
    const int slot = (int)(e->io_calls++ & 1);
    // the list presampled by the previous call sits in this slot already when it is this step's
    const bool pre = e->io_pre && e->io_pre_seed == seed && e->io_pre_step == step && !c->explicit_list &&
                     e->io_epoch == e->epoch && e->io_K == c->K && e->slot_cap >= c->K;
    e->io_pre = false;
    if (pre) {
      c->hm.swap(e->io_pre_hm);
      c->hc.swap(e->io_pre_hc);
      c->hsamp.swap(e->io_pre_samp);
    } else {
      build_host_list(c, seed, step);
    }
    if (!c->have_modes || (int)c->hc.size() != c->K) {
      upload_modes(c);                 // a new mode count: sizes the mode buffers (and recaptures)
      c->have_modes = true;
    }
    reserve(c);
    ensure_slot_buffers(c);
    if (!pre) fill_slot(c, slot);
    if (e->io_epoch != e->epoch || e->io_K != c->K || !e->io_exec[slot]) {
      // the first pass after a state change runs the ordinary way (it sizes every buffer), then the
      // pass is captured for the following calls
      provider_step(c, slot);
      e->drop_io_graphs();
      srbe_ctx *one[1] = {c};
      if (!e->cap) e->cap = make_stream(true);
      if (capture_graphs(one, 1, e->cap, 0, nullptr, e->io_exec, &e->io_kernels, nullptr, true)) {
        e->io_epoch = e->epoch;
        e->io_K = c->K;
      }
    } else {
      coop_before(c);
      SRBE_CUDA(cudaGraphLaunch(e->io_exec[slot], c->stream));
      coop_after(c);
      c->launches += e->io_kernels;
    }
    SRBE_CUDA(cudaEventRecord(e->slot[slot].done, c->stream));
    if (e->io_exec[1 - slot] && e->io_epoch == e->epoch && !c->explicit_list) {
      // while the GPU runs: sample step + 1 into the other slot (its last pass has finished), keeping
      // this step's host list as the context's
      e->io_pre_hm = c->hm;
      e->io_pre_hc = c->hc;
      e->io_pre_samp = c->hsamp;
      build_host_list(c, seed, step + 1);
      if ((int)c->hc.size() == c->K) {
        fill_slot(c, 1 - slot);
        e->io_pre = true;
        e->io_pre_seed = seed;
        e->io_pre_step = step + 1;
      }
      c->hm.swap(e->io_pre_hm);
      c->hc.swap(e->io_pre_hc);
      c->hsamp.swap(e->io_pre_samp);
    }
    SRBE_CUDA(cudaStreamSynchronize(c->stream));
    e->forces_valid = true;
    if (psi_bar) *psi_bar = *(volatile double *)e->io_psi / kVolt;
    report_status(c);
  }, true);
}

int srbe_step(srbe_ctx *c, int nsteps, uint64_t seed0) {
  return guarded(c, [&] {
    SRBE_REQUIRE(nsteps >= 0, SRBE_EINVAL, "negative step count");
    SRBE_REQUIRE(c->have_ele && c->have_pos, SRBE_ESTATE, "electrode and positions are required");
    SRBE_REQUIRE(c->have_md, SRBE_ESTATE, "srbe_set_md has not been called");
    Extra *e = extra(c);
    report_status(c, false);     // flags that earlier (asynchronous) steps raised
    initial_forces(c, seed0);
    const bool graphs = !c->profiling && c->use_graphs && !e->graph_failed && nsteps > 0;
    if (graphs && (e->graph_dirty || e->graph_K != c->K)) {
      // one step the ordinary way sizes every buffer the step touches, then the step is captured
      eager_step(c, seed0);
      --nsteps;
      e->drop_graphs();
      reserve(c);
      ensure_slot_buffers(c);
      cudaGraphExec_t ex[2] = {nullptr, nullptr};
      srbe_ctx *one[1] = {c};
      if (!e->cap) e->cap = make_stream(true);
      if (capture_graphs(one, 1, e->cap, 0, nullptr, ex, &e->graph_kernels, nullptr)) {
        e->slot[0].exec = ex[0];
        e->slot[1].exec = ex[1];
        e->graph_dirty = false;
        e->graph_K = c->K;
      } else {
        e->graph_failed = true;
      }
    }
    if (graphs && !e->graph_failed) {
      for (int s = 0; s < nsteps; ++s) {
        report_status(c, false); // what the host sees so far (no wait)
        c->md_step++;
        const int slot = (int)(c->md_step & 1);
        if (e->dev_sampler) {
          // the captured step samples its modes on the device from this word
          SRBE_CUDA(cudaEventSynchronize(e->slot[slot].done));
          e->slot[slot].hm[c->K] = sample_word(c->md_step, seed0);
        } else {
          build_host_list(c, seed0, c->md_step);
          fill_slot(c, slot);
        }
        coop_before(c);
        SRBE_CUDA(cudaGraphLaunch(e->slot[slot].exec, c->stream));
        coop_after(c);
        SRBE_CUDA(cudaEventRecord(e->slot[slot].done, c->stream));
        c->launches += e->graph_kernels;
      }
      return;
    }
    for (int s = 0; s < nsteps; ++s) {
      report_status(c, false);
      eager_step(c, seed0);
    }
    SRBE_CUDA(cudaGetLastError());
  }, true);
}

int srbe_synchronize(srbe_ctx *c, double timeout_s) {
  return guarded(c, [&] {
    SRBE_REQUIRE(!std::isnan(timeout_s), SRBE_EINVAL, "timeout is NaN");
    cudaStream_t ss[2] = {c->stream, c->side};
    if (timeout_s < 0) {
      for (cudaStream_t st : ss) SRBE_CUDA(cudaStreamSynchronize(st));
    } else {
      // bounded wait: poll both streams until they are idle or the limit passes
      const auto t_end = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
      for (;;) {
        bool busy = false;
        for (cudaStream_t st : ss) {
          const cudaError_t q = cudaStreamQuery(st);
          if (q == cudaErrorNotReady) busy = true;
          else SRBE_CUDA(q);
        }
        if (!busy) break;
        if (std::chrono::steady_clock::now() >= t_end)
          throw Error{SRBE_ETIMEOUT, "work still running on the context's streams after the time limit"};
        std::this_thread::sleep_for(std::chrono::microseconds(50));
      }
    }
    report_status(c);
  }, true);
}

int srbe_debug_inject_nonfinite(srbe_ctx *c, int what) {
  return guarded(c, [&] {
    SRBE_REQUIRE(what >= 0 && what <= 2, SRBE_EINVAL, "what must be 0, 1 (F[0]) or 2 (Q[0])");
    c->inject = what;
  });
}

int srbe_set_graphs(srbe_ctx *c, int on) {
  return guarded(c, [&] {
    c->use_graphs = on != 0;
    extra(c)->graph_failed = false;
  });
}

int srbe_graph_state(srbe_ctx *c, int *captured, int64_t *kernels_per_step) {
  return guarded(c, [&] {
    Extra *e = extra(c);
    const bool ok = e->slot[0].exec && !e->graph_dirty && !e->graph_failed;
    if (captured) *captured = ok ? 1 : (e->graph_failed ? -1 : 0);
    if (kernels_per_step) *kernels_per_step = ok ? e->graph_kernels : 0;
  }, true);
}

int srbe_set_profiling(srbe_ctx *c, int on) {
  return guarded(c, [&] {
    Extra *e = extra(c);
    if (on) {
      drain_events(c);
      for (int p = 0; p < kPhCount; ++p) {
        e->ms[p] = 0.0;
        e->count[p] = 0;
      }
    }
    c->profiling = on != 0;
  });
}

int srbe_get_phase_times(srbe_ctx *c, double *ms, int64_t *count) {
  return guarded(c, [&] {
    drain_events(c);
    Extra *e = extra(c);
    for (int p = 0; p < kPhCount; ++p) {
      if (ms) ms[p] = e->ms[p];
      if (count) count[p] = e->count[p];
    }
  }, true);
}

int srbe_minimize(srbe_ctx *c, int nsteps, double a, double dmax, uint64_t seed) {
  return guarded(c, [&] {
    SRBE_REQUIRE(nsteps >= 0 && a > 0 && dmax > 0 && std::isfinite(a) && std::isfinite(dmax), SRBE_EINVAL,
                 "bad minimisation parameters");
    SRBE_REQUIRE(c->have_ele && c->have_pos && c->have_md, SRBE_ESTATE, "electrode, positions and MD terms needed");
    for (int t = 0; t < nsteps; ++t) {
      sample_into(c, seed, (uint64_t)t);
      forces_pass(c, false, false, false);
      steepest_descent_move(c, a, dmax);
    }
    extra(c)->forces_valid = false;
    SRBE_CUDA(cudaStreamSynchronize(c->stream));
    report_status(c);
  });
}

// ---- iterative solve and learned warm start ---------------------------------------------------
int srbe_set_solver(srbe_ctx *c, int kind, double tol, int maxit, int warm) {
  return guarded(c, [&] {
    SRBE_REQUIRE(kind == SRBE_SOLVER_DIRECT || kind == SRBE_SOLVER_PCG || kind == SRBE_SOLVER_LATTICE, SRBE_EINVAL,
                 "unknown solver");
    SRBE_REQUIRE(warm >= SRBE_WARM_ZERO && warm <= SRBE_WARM_MODEL, SRBE_EINVAL, "unknown warm start");
    SRBE_REQUIRE(tol > 0 && tol < 1 && maxit > 0, SRBE_EINVAL, "bad tolerance or iteration limit");
    SRBE_REQUIRE(c->have_ele, SRBE_ESTATE, "srbe_set_electrode must come first");
    SRBE_REQUIRE(kind == SRBE_SOLVER_LATTICE || c->dense, SRBE_ESTATE,
                 "this electrode has no dense A (more than 16,384 sites): only the lattice solver applies");
    SRBE_REQUIRE(kind != SRBE_SOLVER_LATTICE || c->lat.spectral, SRBE_ESTATE,
                 "the lattice solver needs a lattice electrode");
    c->lat_solve = kind == SRBE_SOLVER_LATTICE;
    c->pcg.on = kind == SRBE_SOLVER_PCG;
    c->pcg.tol = tol;
    c->pcg.maxit = maxit;
    c->pcg.warm = warm;
    if (c->pcg.on) pcg_prepare(c);
  });
}

int srbe_get_solver_stats(srbe_ctx *c, int *iterations, double *rel_residual) {
  return guarded(c, [&] {
    SRBE_REQUIRE(c->pcg.on, SRBE_ESTATE, "the iterative solver is not selected");
    int it = 0;
    double r = 0.0;
    SRBE_CUDA(cudaMemcpyAsync(&it, c->pcg.stats.p, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    SRBE_CUDA(cudaMemcpyAsync(&r, c->pcg.res.p, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    SRBE_CUDA(cudaStreamSynchronize(c->stream));
    if (iterations) *iterations = it;
    if (rel_residual) *rel_residual = r;
  }, true);
}

namespace {
void mlp_alloc(srbe_ctx *c) {
  const size_t n = (size_t)mlp_param_count();
  c->mlp.P.ensure(n);
  c->mlp.m1.ensure(n);
  c->mlp.m2.ensure(n);
  c->mlp.grad.ensure(n);
}
void mlp_reset_moments(srbe_ctx *c) {
  const size_t n = (size_t)mlp_param_count();
  SRBE_CUDA(cudaMemsetAsync(c->mlp.m1.p, 0, sizeof(float) * n, c->stream));
  SRBE_CUDA(cudaMemsetAsync(c->mlp.m2.p, 0, sizeof(float) * n, c->stream));
  c->mlp.t = 0;
}
}  // namespace

int srbe_mlp_init(srbe_ctx *c, uint64_t seed) {
  return guarded(c, [&] {
    const int n = mlp_param_count(), nin = mlp_input_width(), nh = 128;
    std::vector<float> P(n, 0.f);
    // Glorot-uniform weights from Philox4x64-10 words, zero biases, identity standardisation
    uint64_t ctr = 0;
    auto uniform = [&](double lim) {
      const uint64_t c4[4] = {ctr++, 0, 0, 0x4d4c5000ull};
      uint64_t w[4];
      Philox4x64::block(c4, seed, 0x5352424500000003ull, w);
      return (float)((2.0 * unit_open0(w[0]) - 1.0) * lim);
    };
    const double l1 = std::sqrt(6.0 / (nin + nh)), l2 = std::sqrt(6.0 / (nh + nh)), l3 = std::sqrt(6.0 / (nh + 1));
    size_t o = 0;
    for (int i = 0; i < nh * nin; ++i) P[o++] = uniform(l1);
    o += nh;
    for (int i = 0; i < nh * nh; ++i) P[o++] = uniform(l2);
    o += nh;
    for (int i = 0; i < nh; ++i) P[o++] = uniform(l3);
    o += 1;
    o += nin;                                   // input means 0
    for (int i = 0; i < nin; ++i) P[o++] = 1.f;  // input spreads 1
    P[o++] = 0.f;                               // target mean
    P[o++] = 1.f;                               // target spread
    mlp_alloc(c);
    SRBE_CUDA(cudaMemcpyAsync(c->mlp.P.p, P.data(), sizeof(float) * n, cudaMemcpyHostToDevice, c->stream));
    mlp_reset_moments(c);
    SRBE_CUDA(cudaStreamSynchronize(c->stream));
    c->mlp.ready = true;
  });
}

int srbe_mlp_get_params(srbe_ctx *c, float *params, int64_t *count) {
  return guarded(c, [&] {
    if (count) *count = mlp_param_count();
    if (!params) return;
    SRBE_REQUIRE(c->mlp.ready, SRBE_ESTATE, "no MLP parameters");
    SRBE_CUDA(cudaMemcpyAsync(params, c->mlp.P.p, sizeof(float) * mlp_param_count(), cudaMemcpyDeviceToHost,
                              c->stream));
    SRBE_CUDA(cudaStreamSynchronize(c->stream));
  }, true);
}

int srbe_mlp_set_params(srbe_ctx *c, const float *params, int64_t count) {
  return guarded(c, [&] {
    SRBE_REQUIRE(params && count == mlp_param_count(), SRBE_EINVAL, "parameter vector of the wrong length");
    for (int64_t i = 0; i < count; ++i) SRBE_REQUIRE(std::isfinite(params[i]), SRBE_EINVAL, "non-finite parameter");
    mlp_alloc(c);
    SRBE_CUDA(cudaMemcpyAsync(c->mlp.P.p, params, sizeof(float) * count, cudaMemcpyHostToDevice, c->stream));
    mlp_reset_moments(c);
    SRBE_CUDA(cudaStreamSynchronize(c->stream));
    c->mlp.ready = true;
  });
}

int srbe_descriptors(srbe_ctx *c, float *D) {
  return guarded(c, [&] {
    SRBE_REQUIRE(D, SRBE_EINVAL, "null output");
    SRBE_REQUIRE(c->have_ele && c->have_pos && c->nbr.cap > 0, SRBE_ESTATE,
                 "descriptors need a charge update or force call first");
    c->mlp.D.ensure((size_t)c->ne * mlp_input_width());
    mlp_descriptors(c, c->mlp.D.p);
    SRBE_CUDA(cudaMemcpyAsync(D, c->mlp.D.p, sizeof(float) * c->ne * mlp_input_width(), cudaMemcpyDeviceToHost,
                              c->stream));
    SRBE_CUDA(cudaStreamSynchronize(c->stream));
  });
}

int srbe_solution(srbe_ctx *c, double *y) {
  return guarded(c, [&] {
    SRBE_REQUIRE(y, SRBE_EINVAL, "null output");
    SRBE_REQUIRE(c->have_ele, SRBE_ESTATE, "no electrode");
    k_unproject<<<blocks_for(c->ne, 256), 256, 0, c->stream>>>(c->ne, c->Q.p, c->we.p, c->scal.p,
                                                              extra(c)->aos.ensure(std::max<int64_t>(c->ne, 1)));
    c->launches++;
    SRBE_CUDA(cudaGetLastError());
    SRBE_CUDA(cudaMemcpyAsync(y, extra(c)->aos.p, sizeof(double) * c->ne, cudaMemcpyDeviceToHost, c->stream));
    SRBE_CUDA(cudaStreamSynchronize(c->stream));
  });
}

namespace {
void upload_rows(srbe_ctx *c, const float *D, const float *T, int64_t n) {
  const int w = mlp_input_width();
  c->mlp.data_D.ensure((size_t)std::max<int64_t>(n, 1) * w);
  SRBE_CUDA(cudaMemcpyAsync(c->mlp.data_D.p, D, sizeof(float) * n * w, cudaMemcpyHostToDevice, c->stream));
  if (T) {
    c->mlp.data_T.ensure((size_t)std::max<int64_t>(n, 1));
    SRBE_CUDA(cudaMemcpyAsync(c->mlp.data_T.p, T, sizeof(float) * n, cudaMemcpyHostToDevice, c->stream));
  }
}
}  // namespace

int srbe_mlp_predict(srbe_ctx *c, const float *D, int64_t n, float *out) {
  return guarded(c, [&] {
    SRBE_REQUIRE(D && out && n >= 0, SRBE_EINVAL, "bad arguments");
    SRBE_REQUIRE(c->mlp.ready, SRBE_ESTATE, "no MLP parameters");
    if (n == 0) return;
    upload_rows(c, D, nullptr, n);
    float *o = c->mlp.grad.ensure(std::max<size_t>((size_t)n, (size_t)mlp_param_count()));
    mlp_forward(c, c->mlp.data_D.p, n, o, nullptr);
    SRBE_CUDA(cudaMemcpyAsync(out, o, sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream));
    SRBE_CUDA(cudaStreamSynchronize(c->stream));
  });
}

int srbe_mlp_predict_dev(srbe_ctx *c, const float *D_dev, int64_t n, float *out_dev) {
  return guarded(c, [&] {
    SRBE_REQUIRE(D_dev && out_dev && n >= 0, SRBE_EINVAL, "bad arguments");
    SRBE_REQUIRE(c->mlp.ready, SRBE_ESTATE, "no MLP parameters");
    mlp_forward(c, D_dev, n, out_dev, nullptr);
  }, true);
}

int srbe_mlp_gradients(srbe_ctx *c, const float *D, const float *target, int64_t n, float *grad, double *loss) {
  return guarded(c, [&] {
    SRBE_REQUIRE(D && target && grad && n > 0, SRBE_EINVAL, "bad arguments");
    SRBE_REQUIRE(c->mlp.ready, SRBE_ESTATE, "no MLP parameters");
    upload_rows(c, D, target, n);
    const double l = mlp_grad_step(c, c->mlp.data_D.p, c->mlp.data_T.p, nullptr, n, c->mlp.grad.p, false, 0.f, 0.f);
    int64_t ntrain = 0;
    // the trainable part is everything before the input mean
    ntrain = mlp_param_count() - 2 * mlp_input_width() - 2;
    SRBE_CUDA(cudaMemcpyAsync(grad, c->mlp.grad.p, sizeof(float) * ntrain, cudaMemcpyDeviceToHost, c->stream));
    SRBE_CUDA(cudaStreamSynchronize(c->stream));
    if (loss) *loss = l;
  });
}

int srbe_mlp_train(srbe_ctx *c, const float *D, const float *target, int64_t n, int epochs, int batch, float lr,
                   float weight_decay, uint64_t seed, double *final_loss) {
  return guarded(c, [&] {
    SRBE_REQUIRE(D && target && n > 1 && epochs > 0 && batch > 0 && lr > 0, SRBE_EINVAL, "bad arguments");
    SRBE_REQUIRE(c->mlp.ready, SRBE_ESTATE, "no MLP parameters (srbe_mlp_init)");
    const int w = mlp_input_width(), np = mlp_param_count();
    // standardisation from the data (mean and spread of every input column and of the target)
    std::vector<float> P(np);
    SRBE_CUDA(cudaMemcpy(P.data(), c->mlp.P.p, sizeof(float) * np, cudaMemcpyDeviceToHost));
    const int oXm = np - 2 * w - 2, oXs = oXm + w, oYm = oXs + w, oYs = oYm + 1;
    for (int k = 0; k < w; ++k) {
      double s = 0.0, s2 = 0.0;
      for (int64_t i = 0; i < n; ++i) {
        const double v = D[i * w + k];
        s += v;
        s2 += v * v;
      }
      const double m = s / n, var = std::max(s2 / n - m * m, 0.0);
      P[oXm + k] = (float)m;
      P[oXs + k] = (float)std::max(std::sqrt(var), 1e-6);
    }
    double s = 0.0, s2 = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      s += target[i];
      s2 += (double)target[i] * target[i];
    }
    const double m = s / n;
    P[oYm] = (float)m;
    P[oYs] = (float)std::max(std::sqrt(std::max(s2 / n - m * m, 0.0)), 1e-12);
    SRBE_CUDA(cudaMemcpy(c->mlp.P.p, P.data(), sizeof(float) * np, cudaMemcpyHostToDevice));
    mlp_reset_moments(c);
    upload_rows(c, D, target, n);
    c->mlp.rows.ensure((size_t)n);
    std::vector<int32_t> perm(n);
    double last = 0.0;
    uint64_t ctr = 0;
    for (int e = 0; e < epochs; ++e) {
      for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
      for (int64_t i = n - 1; i > 0; --i) {   // Fisher-Yates with Philox draws
        const uint64_t c4[4] = {ctr++, (uint64_t)e, 0, 0x53485546ull};
        uint64_t wv[4];
        Philox4x64::block(c4, seed, 0x5352424500000004ull, wv);
        const int64_t j = (int64_t)(wv[0] % (uint64_t)(i + 1));
        std::swap(perm[i], perm[j]);
      }
      SRBE_CUDA(cudaMemcpyAsync(c->mlp.rows.p, perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, c->stream));
      double tot = 0.0;
      int64_t seen = 0;
      for (int64_t b0 = 0; b0 < n; b0 += batch) {
        const int64_t nb = std::min<int64_t>(batch, n - b0);
        const double l = mlp_grad_step(c, c->mlp.data_D.p, c->mlp.data_T.p, c->mlp.rows.p + b0, nb, nullptr, true,
                                       lr, weight_decay);
        tot += l * nb;
        seen += nb;
      }
      last = tot / seen;
    }
    if (final_loss) *final_loss = last;
  });
}

int srbe_get_counters(const srbe_ctx *cc, int64_t *kernel_launches, int64_t *mode_evals) {
  if (!cc) return SRBE_EINVAL;
  if (kernel_launches) *kernel_launches = cc->launches;
  if (mode_evals) *mode_evals = cc->mode_evals;
  return SRBE_OK;
}

int srbe_set_lattice(srbe_ctx *c, int on) {
  return guarded(c, [&] {
    SRBE_REQUIRE(on >= 0 && on <= 2, SRBE_EINVAL, "lattice mode is 0 (never), 1 (when it pays) or 2 (always)");
    c->lat.mode = on;
  });
}

int srbe_lattice_info(srbe_ctx *c, int32_t dims[3]) {
  return guarded(c, [&] {
    SRBE_REQUIRE(dims, SRBE_EINVAL, "null output");
    dims[0] = c->lat.nl;
    dims[1] = c->lat.nx;
    dims[2] = c->lat.ny;
  }, true);
}

int srbe_set_thermostat(srbe_ctx *c, double gamma, double T, uint64_t seed) {
  return guarded(c, [&] {
    SRBE_REQUIRE(std::isfinite(gamma) && gamma >= 0.0 && std::isfinite(T) && T >= 0.0, SRBE_EINVAL,
                 "thermostat needs gamma >= 0 (1/ps) and T >= 0 (K)");
    c->lang_gamma = gamma;
    c->lang_T = T;
    c->lang_seed = seed;
  });
}

int srbe_charge_residual(srbe_ctx *c, double *rel_residual) {
  return guarded(c, [&] {
    require_state(c, true);
    SRBE_REQUIRE(rel_residual, SRBE_EINVAL, "null output");
    double *d = c->resid.ensure((size_t)2 * std::max<int64_t>(c->ne, 1) + 2) + 2 * std::max<int64_t>(c->ne, 1);
    charge_residual(c, d);
    double h[2];
    SRBE_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    SRBE_CUDA(cudaStreamSynchronize(c->stream));
    *rel_residual = h[1] > 0 ? std::sqrt(h[0] / h[1]) : std::sqrt(h[0]);
  }, true);
}

int srbe_set_skin(srbe_ctx *c, double skin) {
  return guarded(c, [&] {
    SRBE_REQUIRE(std::isfinite(skin) && skin > 0.0 && skin <= 1.0, SRBE_EINVAL, "skin must be in (0, 1] nm");
    c->nbr.skin = skin;
    c->nbr.cap = 0;                    // list capacity follows the skin (recomputed by reserve)
    if (c->have_pos) {
      reserve(c);
      neighbor_force_rebuild(c);
    }
  });
}

double srbe_get_skin(const srbe_ctx *c) { return c ? c->nbr.skin : 0.0; }

double srbe_get_alpha_A(const srbe_ctx *c) { return c ? c->alpha_A : 0.0; }

}  // extern "C"

// ---- replicas: snapshots and the batch ----------------------------------------------------------
namespace {

// device copy of the dynamical state of a context (positions, velocities, forces, charges, PCG
// iterate) and its step counter; restoring it also forces a neighbour-list rebuild
struct Snapshot {
  DevBuf<double> buf;
  uint64_t md_step = 0;
  bool forces_valid = false;
  bool pcg = false;
};

void snapshot_io(srbe_ctx *c, Snapshot &sn, bool save) {
  const size_t n = (size_t)c->ni, ne = (size_t)c->ne;
  if (save) sn.pcg = c->pcg.y.p != nullptr;
  const bool pcg = sn.pcg;
  SRBE_REQUIRE(!pcg || c->pcg.y.p, SRBE_ESTATE, "PCG state vanished under a snapshot");
  double *b = save ? sn.buf.ensure(9 * n + ne + (pcg ? ne : 0) + 1) : sn.buf.p;
  struct Part {
    double *p;
    size_t n;
  } parts[] = {{c->x.p, n}, {c->y.p, n}, {c->z.p, n}, {c->vx.p, n}, {c->vy.p, n}, {c->vz.p, n},
               {c->F.p, 3 * n}, {c->Q.p, ne}, {pcg ? c->pcg.y.p : nullptr, pcg ? ne : 0}};
  size_t o = 0;
  for (const Part &pt : parts) {
    if (pt.p && pt.n) {
      if (save) SRBE_CUDA(cudaMemcpyAsync(b + o, pt.p, sizeof(double) * pt.n, cudaMemcpyDeviceToDevice, c->stream));
      else SRBE_CUDA(cudaMemcpyAsync(pt.p, b + o, sizeof(double) * pt.n, cudaMemcpyDeviceToDevice, c->stream));
    }
    o += pt.n;
  }
  if (save) {
    sn.md_step = c->md_step;
    sn.forces_valid = extra(c)->forces_valid;
  } else {
    c->md_step = sn.md_step;
    extra(c)->forces_valid = sn.forces_valid;
    neighbor_force_rebuild(c);
  }
}

}  // namespace

struct srbe_batch {
  std::vector<srbe_ctx *> ctx;
  std::vector<uint64_t> epoch;       // state epochs of the replicas when the graphs were captured
  std::vector<int64_t> kernels;      // kernels per replica in one replay
  cudaStream_t main = nullptr;
  std::vector<cudaStream_t> forks;
  int width = 0;                     // concurrent replica streams (0: one stream, in order)
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaEvent_t done[2] = {nullptr, nullptr};
  cudaEvent_t mark = nullptr;
  DevBuf<double> res;                // residual sums [n][2]
  DevBuf<StageEntry> stage[2];       // per slot: where each replica's mode list comes from and goes
  double *h_res = nullptr;
  uint64_t t = 0;
  bool dirty = true;
  int device = 0;
  int threads = 1;
  std::string err;

  void drop() {
    for (auto &x : exec)
      if (x) {
        cudaGraphExecDestroy(x);
        x = nullptr;
      }
    dirty = true;
  }
  ~srbe_batch() {
    if (main) cudaStreamSynchronize(main);
    drop();
    for (auto &f : forks) cudaStreamDestroy(f);
    for (auto &d : done)
      if (d) cudaEventDestroy(d);
    if (mark) cudaEventDestroy(mark);
    if (h_res) cudaFreeHost(h_res);
    if (main) cudaStreamDestroy(main);
  }
};

namespace {

template <class Fn>
int batch_guarded(srbe_batch *b, Fn &&fn) {
  if (!b) return SRBE_EINVAL;
  try {
    b->err.clear();
    SRBE_CUDA(cudaSetDevice(b->device));
    fn();
    return SRBE_OK;
  } catch (const Error &e) {
    b->err = e.msg;
    return e.code;
  } catch (const std::bad_alloc &) {
    b->err = "host allocation failed";
    return SRBE_ENOMEM;
  } catch (const std::exception &e) {
    b->err = e.what();
    return SRBE_EINVAL;
  }
}

// runs fn(r) for every replica, spread over up to `threads` host threads
template <class Fn>
void for_replicas(int n, int threads, Fn &&fn) {
  if (threads <= 1 || n < 4) {
    for (int r = 0; r < n; ++r) fn(r);
    return;
  }
  const int nt = std::min(threads, n);
  std::vector<std::thread> pool;
  std::vector<std::string> errs(nt);
  std::vector<int> codes(nt, SRBE_OK);
  for (int t = 0; t < nt; ++t)
    pool.emplace_back([&, t] {
      try {
        for (int r = t; r < n; r += nt) fn(r);
      } catch (const Error &e) {
        codes[t] = e.code;
        errs[t] = e.msg;
      } catch (const std::exception &e) {
        codes[t] = SRBE_EINVAL;
        errs[t] = e.what();
      }
    });
  for (auto &th : pool) th.join();
  for (int t = 0; t < nt; ++t)
    if (codes[t] != SRBE_OK) throw Error{codes[t], errs[t]};
}

// orders `to` after everything issued so far on `from`
void stream_after(cudaStream_t to, cudaStream_t from, cudaEvent_t ev) {
  SRBE_CUDA(cudaEventRecord(ev, from));
  SRBE_CUDA(cudaStreamWaitEvent(to, ev, 0));
}

void batch_check_replicas(srbe_batch *b) {
  for (srbe_ctx *c : b->ctx) {
    SRBE_REQUIRE(c->have_ele && c->have_pos && c->have_md, SRBE_ESTATE,
                 "every replica needs electrode, positions and srbe_set_md");
    SRBE_REQUIRE(!c->profiling, SRBE_ESTATE, "switch phase tracing off on the replicas of a batch");
  }
}

// (re)captures the batch graphs after one ordinary step of every replica
void batch_capture(srbe_batch *b, const uint64_t *seeds) {
  const int n = (int)b->ctx.size();
  b->drop();
  for (int r = 0; r < n; ++r) {
    srbe_ctx *c = b->ctx[r];
    stream_after(c->stream, b->main, b->mark);
    initial_forces(c, seeds[r]);
    eager_step(c, seeds[r]);
    reserve(c);
    ensure_slot_buffers(c);    // synchronises the replica's stream
  }
  while ((int)b->forks.size() < b->width) {
    cudaStream_t f = nullptr;
    f = make_stream(true);
    b->forks.push_back(f);
  }
  b->kernels.assign(n, 0);
  SRBE_REQUIRE(capture_graphs(b->ctx.data(), n, b->main, b->width, b->forks.data(), b->exec, b->kernels.data(),
                              b->stage),
               SRBE_ECUDA, "capture of the batch step failed");
  b->epoch.resize(n);
  for (int r = 0; r < n; ++r) {
    b->epoch[r] = extra(b->ctx[r])->epoch;
    extra(b->ctx[r])->graph_dirty = true;     // the replicas' own single-context graphs are stale now
  }
  b->dirty = false;
}

bool batch_stale(const srbe_batch *b) {
  if (b->dirty || !b->exec[0]) return true;
  for (size_t r = 0; r < b->ctx.size(); ++r) {
    const srbe_ctx *c = b->ctx[r];
    if (c->hx->epoch != b->epoch[r] || !c->hx->forces_valid || (int)c->hc.size() != c->K) return true;
  }
  return false;
}

// nsteps MD steps of every replica; the first step after a change of state runs the ordinary way
void batch_run(srbe_batch *b, int nsteps, const uint64_t *seeds) {
  const int n = (int)b->ctx.size();
  if (nsteps <= 0) return;
  for (srbe_ctx *c : b->ctx) {
    stream_after(b->main, c->stream, b->mark);
    // a replica's own step graph may still read its pinned slots
    for (auto &sl : extra(c)->slot)
      if (sl.done) SRBE_CUDA(cudaEventSynchronize(sl.done));
  }
  if (batch_stale(b)) {
    batch_capture(b, seeds);
    --nsteps;
  }
  for (int s = 0; s < nsteps; ++s) {
    const int slot = (int)(b->t & 1);
    b->t++;
    for_replicas(n, b->threads, [&](int r) {
      srbe_ctx *c = b->ctx[r];
      c->md_step++;
      build_host_list(c, seeds[r], c->md_step);
    });
    SRBE_CUDA(cudaEventSynchronize(b->done[slot]));
    for (int r = 0; r < n; ++r) copy_to_slot(b->ctx[r], slot);
    SRBE_CUDA(cudaStreamWaitEvent(b->main, device_coop_chain(), 0));
    SRBE_CUDA(cudaGraphLaunch(b->exec[slot], b->main));
    SRBE_CUDA(cudaEventRecord(device_coop_chain(), b->main));
    SRBE_CUDA(cudaEventRecord(b->done[slot], b->main));
    for (int r = 0; r < n; ++r) b->ctx[r]->launches += b->kernels[r];
  }
  // later work on a replica's own stream sees the batch's results, and its own step graph waits
  // for the batch's reads of the shared pinned slots before refilling them
  SRBE_CUDA(cudaEventRecord(b->mark, b->main));
  for (srbe_ctx *c : b->ctx) {
    SRBE_CUDA(cudaStreamWaitEvent(c->stream, b->mark, 0));
    for (auto &sl : extra(c)->slot)
      if (sl.done) SRBE_CUDA(cudaEventRecord(sl.done, b->main));
  }
}

void batch_residuals(srbe_batch *b, double *out) {
  const int n = (int)b->ctx.size();
  double *d = b->res.ensure((size_t)2 * n);
  for (int r = 0; r < n; ++r) {
    srbe_ctx *c = b->ctx[r];
    stream_after(b->main, c->stream, b->mark);
    const cudaStream_t own = c->stream;
    c->stream = b->main;
    try {
      charge_residual(c, d + 2 * r);
    } catch (...) {
      c->stream = own;
      throw;
    }
    c->stream = own;
  }
  SRBE_CUDA(cudaMemcpyAsync(b->h_res, d, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, b->main));
  SRBE_CUDA(cudaStreamSynchronize(b->main));
  for (int r = 0; r < n; ++r) {
    const double a = b->h_res[2 * r], q = b->h_res[2 * r + 1];
    out[r] = q > 0 ? std::sqrt(a / q) : std::sqrt(a);
  }
}

}  // namespace

extern "C" {

int srbe_batch_create(int n, srbe_ctx *const *ctxs, srbe_batch **out) {
  if (!out) return SRBE_EINVAL;
  *out = nullptr;
  if (n < 1 || !ctxs) return SRBE_EINVAL;
  for (int r = 0; r < n; ++r) {
    if (!ctxs[r]) return SRBE_EINVAL;
    for (int q = 0; q < r; ++q)
      if (ctxs[q] == ctxs[r]) return SRBE_EINVAL;
  }
  srbe_batch *b = new (std::nothrow) srbe_batch;
  if (!b) return SRBE_ENOMEM;
  b->ctx.assign(ctxs, ctxs + n);
  const int rc = batch_guarded(b, [&] {
    SRBE_CUDA(cudaGetDevice(&b->device));
    b->main = make_stream(true);
    for (auto &d : b->done) {
      SRBE_CUDA(cudaEventCreateWithFlags(&d, cudaEventDisableTiming));
      SRBE_CUDA(cudaEventRecord(d, b->main));
    }
    SRBE_CUDA(cudaEventCreateWithFlags(&b->mark, cudaEventDisableTiming));
    SRBE_CUDA(cudaMallocHost((void **)&b->h_res, sizeof(double) * 2 * n));
    b->width = std::min(n, 16);
    const unsigned hw = std::thread::hardware_concurrency();
    b->threads = (int)std::max(1u, std::min(8u, hw ? hw : 1u));
  });
  if (rc != SRBE_OK) {
    delete b;
    return rc;
  }
  *out = b;
  return SRBE_OK;
}

int srbe_batch_destroy(srbe_batch *b) {
  if (!b) return SRBE_EINVAL;
  cudaSetDevice(b->device);
  delete b;
  return SRBE_OK;
}

const char *srbe_batch_last_error(const srbe_batch *b) { return b ? b->err.c_str() : "null batch"; }

int srbe_batch_set_width(srbe_batch *b, int width) {
  return batch_guarded(b, [&] {
    SRBE_REQUIRE(width >= 0, SRBE_EINVAL, "negative width");
    b->width = std::min<int>(width, (int)b->ctx.size());
    b->dirty = true;
  });
}

int srbe_batch_get_width(const srbe_batch *b) { return b ? b->width : -1; }

void *srbe_batch_stream(const srbe_batch *b) { return b ? (void *)b->main : nullptr; }

int srbe_batch_step(srbe_batch *b, int nsteps, const uint64_t *seeds, double *residuals) {
  return batch_guarded(b, [&] {
    SRBE_REQUIRE(nsteps >= 0, SRBE_EINVAL, "negative step count");
    SRBE_REQUIRE(seeds, SRBE_EINVAL, "null seed array");
    batch_check_replicas(b);
    // device flags that earlier (asynchronous) batch steps raised on any replica
    for (size_t r = 0; r < b->ctx.size(); ++r) {
      try {
        report_status(b->ctx[r], false);
      } catch (const Error &e) {
        throw Error{e.code, "replica " + std::to_string(r) + ": " + e.msg};
      }
    }
    batch_run(b, nsteps, seeds);
    if (residuals) batch_residuals(b, residuals);
  });
}

int srbe_autotune_tiles(srbe_ctx *c, int trial_steps, uint64_t seed, const int *occ, int n_occ,
                        double *ms_per_step) {
  return guarded(c, [&] {
    SRBE_REQUIRE(trial_steps >= 1 && occ && n_occ >= 1, SRBE_EINVAL, "need trial steps and candidate tiles");
    SRBE_REQUIRE(c->have_md && c->have_pos && c->have_ele, SRBE_ESTATE, "the context needs an MD state");
    for (int i = 0; i < n_occ; ++i)
      SRBE_REQUIRE(occ[i] >= 1 && occ[i] <= 64, SRBE_EINVAL, "blocks per SM out of [1, 64]");
    const bool prof = c->profiling;
    c->profiling = false;
    initial_forces(c, seed);
    Snapshot snap;
    snapshot_io(c, snap, true);
    cudaEvent_t t0, t1;
    SRBE_CUDA(cudaEventCreate(&t0));
    SRBE_CUDA(cudaEventCreate(&t1));
    double best = 1e300;
    int best_occ = c->sf_occ;
    for (int i = 0; i < n_occ; ++i) {
      c->sf_occ = occ[i];
      reserve(c);
      extra(c)->graph_dirty = true;
      SRBE_REQUIRE(srbe_step(c, 2, seed) == SRBE_OK, SRBE_ECUDA, c->err);
      SRBE_CUDA(cudaEventRecord(t0, c->stream));
      SRBE_REQUIRE(srbe_step(c, trial_steps, seed) == SRBE_OK, SRBE_ECUDA, c->err);
      SRBE_CUDA(cudaEventRecord(t1, c->stream));
      SRBE_CUDA(cudaEventSynchronize(t1));
      float ms = 0.f;
      SRBE_CUDA(cudaEventElapsedTime(&ms, t0, t1));
      if (ms_per_step) ms_per_step[i] = ms / trial_steps;
      if (ms / trial_steps < best) {
        best = ms / trial_steps;
        best_occ = occ[i];
      }
      snapshot_io(c, snap, false);
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    c->sf_occ = best_occ;
    reserve(c);
    extra(c)->graph_dirty = true;
    c->profiling = prof;
  });
}

int srbe_get_tiles(const srbe_ctx *c) { return c ? c->sf_occ : 0; }

int srbe_set_tiles(srbe_ctx *c, int occ) {
  return guarded(c, [&] {
    SRBE_REQUIRE(occ >= 1 && occ <= 64, SRBE_EINVAL, "blocks per SM out of [1, 64]");
    c->sf_occ = occ;                 // the next pass sizes the partial sums for it (reserve)
  });
}

int srbe_batch_autotune(srbe_batch *b, int trial_steps, const uint64_t *seeds, const int *widths, int n_widths,
                        double *ms_per_step) {
  return batch_guarded(b, [&] {
    SRBE_REQUIRE(trial_steps >= 1 && seeds && widths && n_widths >= 1, SRBE_EINVAL,
                 "need trial_steps >= 1, seeds and candidate widths");
    for (int i = 0; i < n_widths; ++i) SRBE_REQUIRE(widths[i] >= 0, SRBE_EINVAL, "negative width");
    batch_check_replicas(b);
    const int n = (int)b->ctx.size();
    std::vector<Snapshot> snap(n);
    for (int r = 0; r < n; ++r) {
      SRBE_CUDA(cudaStreamSynchronize(b->main));
      initial_forces(b->ctx[r], seeds[r]);
      snapshot_io(b->ctx[r], snap[r], true);
    }
    cudaEvent_t t0, t1;
    SRBE_CUDA(cudaEventCreate(&t0));
    SRBE_CUDA(cudaEventCreate(&t1));
    double best = 1e300;
    int best_w = b->width;
    for (int i = 0; i < n_widths; ++i) {
      const int w = std::min(widths[i], n);
      b->width = w;
      b->dirty = true;
      batch_run(b, 2, seeds);                        // ordinary first step, capture, one replay
      SRBE_CUDA(cudaEventRecord(t0, b->main));
      batch_run(b, trial_steps, seeds);
      SRBE_CUDA(cudaEventRecord(t1, b->main));
      SRBE_CUDA(cudaEventSynchronize(t1));
      float ms = 0.f;
      SRBE_CUDA(cudaEventElapsedTime(&ms, t0, t1));
      if (ms / trial_steps < best) {
        best = ms / trial_steps;
        best_w = w;
      }
      if (ms_per_step) ms_per_step[i] = ms / trial_steps;
      for (int r = 0; r < n; ++r) {
        srbe_ctx *c = b->ctx[r];
        SRBE_CUDA(cudaStreamSynchronize(c->stream));
        snapshot_io(c, snap[r], false);
      }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    for (int r = 0; r < n; ++r) SRBE_CUDA(cudaStreamSynchronize(b->ctx[r]->stream));
    b->width = best_w;
    b->dirty = true;
  });
}

int srbe_batch_autotune_tiles(srbe_batch *b, int trial_steps, const uint64_t *seeds, const int *occ, int n_occ,
                              double *ms_per_step) {
  return batch_guarded(b, [&] {
    SRBE_REQUIRE(trial_steps >= 1 && seeds && occ && n_occ >= 1, SRBE_EINVAL,
                 "need trial_steps >= 1, seeds and candidate tiles");
    for (int i = 0; i < n_occ; ++i)
      SRBE_REQUIRE(occ[i] >= 1 && occ[i] <= 64, SRBE_EINVAL, "blocks per SM out of [1, 64]");
    batch_check_replicas(b);
    const int n = (int)b->ctx.size();
    std::vector<Snapshot> snap(n);
    for (int r = 0; r < n; ++r) {
      SRBE_CUDA(cudaStreamSynchronize(b->main));
      initial_forces(b->ctx[r], seeds[r]);
      snapshot_io(b->ctx[r], snap[r], true);
    }
    cudaEvent_t t0, t1;
    SRBE_CUDA(cudaEventCreate(&t0));
    SRBE_CUDA(cudaEventCreate(&t1));
    double best = 1e300;
    int best_occ = b->ctx.empty() ? 8 : b->ctx[0]->sf_occ;
    for (int i = 0; i < n_occ; ++i) {
      // one setting for every replica: each replica's chunking follows its own size from it
      for (int r = 0; r < n; ++r) {
        b->ctx[r]->sf_occ = occ[i];
        reserve(b->ctx[r]);
      }
      b->dirty = true;
      batch_run(b, 2, seeds);                        // ordinary first step, capture, one replay
      SRBE_CUDA(cudaEventRecord(t0, b->main));
      batch_run(b, trial_steps, seeds);
      SRBE_CUDA(cudaEventRecord(t1, b->main));
      SRBE_CUDA(cudaEventSynchronize(t1));
      float ms = 0.f;
      SRBE_CUDA(cudaEventElapsedTime(&ms, t0, t1));
      if (ms / trial_steps < best) {
        best = ms / trial_steps;
        best_occ = occ[i];
      }
      if (ms_per_step) ms_per_step[i] = ms / trial_steps;
      for (int r = 0; r < n; ++r) {
        srbe_ctx *c = b->ctx[r];
        SRBE_CUDA(cudaStreamSynchronize(c->stream));
        snapshot_io(c, snap[r], false);
      }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    for (int r = 0; r < n; ++r) {
      SRBE_CUDA(cudaStreamSynchronize(b->ctx[r]->stream));
      b->ctx[r]->sf_occ = best_occ;
      reserve(b->ctx[r]);
    }
    b->dirty = true;
  });
}

int srbe_autotune_skin(srbe_ctx *c, int trial_steps, uint64_t seed, const double *skins, int n_skins,
                       double *ms_per_step) {
  return guarded(c, [&] {
    SRBE_REQUIRE(trial_steps >= 1 && skins && n_skins >= 1, SRBE_EINVAL, "need trial steps and candidate skins");
    SRBE_REQUIRE(c->have_md && c->have_pos && c->have_ele, SRBE_ESTATE, "the context needs an MD state");
    for (int i = 0; i < n_skins; ++i)
      SRBE_REQUIRE(std::isfinite(skins[i]) && skins[i] > 0.0 && skins[i] <= 1.0, SRBE_EINVAL, "skin out of (0, 1]");
    const bool prof = c->profiling;
    c->profiling = false;
    initial_forces(c, seed);
    Snapshot snap;
    snapshot_io(c, snap, true);
    cudaEvent_t t0, t1;
    SRBE_CUDA(cudaEventCreate(&t0));
    SRBE_CUDA(cudaEventCreate(&t1));
    double best = 1e300, best_skin = c->nbr.skin;
    for (int i = 0; i < n_skins; ++i) {
      c->nbr.skin = skins[i];
      c->nbr.cap = 0;
      reserve(c);
      neighbor_force_rebuild(c);
      extra(c)->graph_dirty = true;
      SRBE_REQUIRE(srbe_step(c, 2, seed) == SRBE_OK, SRBE_ECUDA, c->err);
      SRBE_CUDA(cudaEventRecord(t0, c->stream));
      SRBE_REQUIRE(srbe_step(c, trial_steps, seed) == SRBE_OK, SRBE_ECUDA, c->err);
      SRBE_CUDA(cudaEventRecord(t1, c->stream));
      SRBE_CUDA(cudaEventSynchronize(t1));
      float ms = 0.f;
      SRBE_CUDA(cudaEventElapsedTime(&ms, t0, t1));
      if (ms_per_step) ms_per_step[i] = ms / trial_steps;
      if (ms / trial_steps < best) {
        best = ms / trial_steps;
        best_skin = skins[i];
      }
      snapshot_io(c, snap, false);
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    c->nbr.skin = best_skin;
    c->nbr.cap = 0;
    reserve(c);
    neighbor_force_rebuild(c);
    c->profiling = prof;
  });
}

}  // extern "C"
