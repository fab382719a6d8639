// Internal declarations of the SRBE library: context layout, device buffers, launch helpers and
// the fixed-point phase / sin-cos primitives shared by the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/srbe.h"

namespace srbe {

constexpr double kPi = 3.14159265358979323846;
constexpr double kBoltz = 0.0083144626;     // kJ mol^-1 K^-1
constexpr int64_t kMaxModes = 32 * 65535;   // modes per list: 32-mode tiles on a grid's y dimension
constexpr int64_t kDenseMaxSites = 16384;    // dense A and its inverse (3 x n^2 x 8 B) only up to here
constexpr int64_t kLatSolveMinSites = 8192;  // lattice electrodes from here solve through the spectral form
constexpr int kTabBits = 10;                  // sin/cos table of 1024 entries per turn
constexpr int kTab = 1 << kTabBits;
constexpr int kGatherThreads = 256;           // gather kernels: one warp per particle
constexpr int kWarpsPerBlock = kGatherThreads / 32;

// ------------------------------------------------------------------------------------------------
// error plumbing
// ------------------------------------------------------------------------------------------------
struct Error {
  int code;
  std::string msg;
};

#define SRBE_CUDA(call)                                                                         \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      throw ::srbe::Error{SRBE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)};      \
  } while (0)

#define SRBE_REQUIRE(cond, code, text)                  \
  do {                                                  \
    if (!(cond)) throw ::srbe::Error{(code), (text)};   \
  } while (0)

// ------------------------------------------------------------------------------------------------
// device buffer with grow-only capacity
// ------------------------------------------------------------------------------------------------
template <class T>
struct DevBuf {
  T *p = nullptr;
  size_t cap = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  T *ensure(size_t n) {
    if (n <= cap && p) return p;
    release();
    size_t bytes = (n ? n : 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void **)&p, bytes);
    if (e != cudaSuccess) {
      p = nullptr;
      cudaGetLastError();
      throw Error{SRBE_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e)};
    }
    cap = n ? n : 1;
    return p;
  }
};

// Cell list of a point set: 2D-periodic bins in x, y and open bins in z.
struct CellGrid {
  int nc[3] = {1, 1, 1};       // cells per dimension
  double cs[3] = {1, 1, 1};    // cell edge
  double z0 = 0.0;             // z of the lower edge of cell 0
  int span[3] = {1, 1, 1};     // stencil half-width in cells, so that span * cs >= rc
  int ncell() const { return nc[0] * nc[1] * nc[2]; }
};

// Stencil of every cell as runs of consecutive cells of one x-row sharing an image shift:
// (first cell, number of cells, packed image (ix + 512) | (iy + 512) << 10, 0), per-cell offsets.
struct RunTable {
  DevBuf<int4> runs;
  DevBuf<int32_t> first;
};

// Verlet lists (rc + skin), rebuilt on the device when an ion has moved more than skin / 2 since
// the last build.  Entries pack a sorted index (bits 0-23) and the image shifts (ix + 8, iy + 8) in
// 4 bits each (bits 24-27, 28-31).
struct NbrLists {
  DevBuf<int32_t> ii, ie, ei;        // ion-ion [ni][cap], ion-electrode [ni][cap], electrode-ion [ne][cap]
  DevBuf<int32_t> ii_n, ie_n, ei_n;  // entry counts (can exceed cap: the gathers then walk the stencil)
  int cap = 0;
  DevBuf<double> xb, yb;             // sorted x, y at the last build (unwrapping reference)
  DevBuf<float4> pfb;                // sorted FP32 positions at the last build
  DevBuf<int32_t> cell_s;            // cell of each sorted ion at the last build
  DevBuf<int> flag;                  // [0] rebuild needed, [1] forced by the host, [2] list-task counter
  double skin = 0.1;
};

// Iterative charge solve state (preconditioned CG on A y = dpsi d + b)
struct PcgState {
  bool on = false;
  double tol = 1e-8;
  int maxit = 1000;
  int warm = 0;                      // 0 zero, 1 previous solution, 2 learned model
  DevBuf<double> dinv, y, r, z, p, Ap, part, res;
  DevBuf<int> stats;
  // mixed form: FP32 copy of A and FP32 vectors of the inner iteration (iterative refinement)
  DevBuf<float> A32, r32, z32, p32, Ap32, d32, s32, dinv32, part32;
  bool a32_ready = false;
};

// Learned warm start: MLP parameters, AdamW moments, scratch
struct MlpState {
  bool ready = false;
  int t = 0;
  DevBuf<float> P, m1, m2, gpart, grad, D, data_D, data_T;
  DevBuf<double> lpart;
  DevBuf<double2> Slow;
  DevBuf<int32_t> rows;
};

struct Cells {
  CellGrid g;
  DevBuf<int32_t> cell, rank, start, order;   // order: sorted position -> original index
  DevBuf<int32_t> inv;                        // original index -> sorted position
  DevBuf<double> xs, ys, zs, ws;              // positions / charges in sorted order
  DevBuf<int32_t> ts, ms;                     // type, molecule in sorted order
  DevBuf<float4> pf;                          // FP32 (x, y, z, w) in sorted order for the pre-check
  DevBuf<uint64_t> us;                        // fixed-point phase coordinates [3][n] in sorted order
};

struct HostExt;   // host-only per-context state (sampler, staging), defined in api.cu

}  // namespace srbe

// ------------------------------------------------------------------------------------------------
// the context
// ------------------------------------------------------------------------------------------------
namespace srbe {
// electrode recognised as layers of a rectangular lattice commensurate with the box (nl = 0: not)
constexpr int kLatMaxLayers = 8;
constexpr int kLatMaxN = 960;                  // lattice points per row / column (shared-memory lines)
struct Lattice {
  int nl = 0, nx = 0, ny = 0;
  DevBuf<int32_t> site;                        // [nl][ny][nx] -> site index
  DevBuf<uint64_t> lu;                         // [3][nl] layer origins in turns
  DevBuf<double2> twx, twy;                    // e^{2 pi i t / nx}, e^{2 pi i t / ny}
  DevBuf<double> Zl;                           // layer heights
  DevBuf<double2> T, Qh;                       // [nl][ny][nx] transform scratch
  DevBuf<double> bF;                           // far part of b per site
  DevBuf<double2> E;                           // per-step e^{i phi_l(k)} [K][nl]
  // spectral form of A: A is block-circulant over the lattice, A y = sum_bins w^{-bin.i} M(bin) Yhat(bin)
  // with nl x nl Hermitian blocks M per bin (a, b); Minv holds M^-1 / (nx ny)^2 for the exact solve
  bool spectral = false;
  DevBuf<double2> M, Minv;                     // [ny][nx][nl][nl]
  DevBuf<double> R, Y;                         // per-site scratch (right-hand side, solution)
  DevBuf<double> Rrow;                         // [nl][ne] real-space rows of A at the layer origins
  int mode = 1;                                // 0 never, 1 when it pays (N_ele K large), 2 always
  int64_t min_work = 4000000;                  // N_ele x K from which mode 1 takes the lattice path
  bool active(int64_t ne, int K) const {
    return nl > 0 && (mode == 2 || (mode == 1 && ne * (int64_t)K >= min_work));
  }
};
}  // namespace srbe

struct srbe_ctx {
  // problem parameters
  double L[3] = {0, 0, 0};
  double V = 0;
  double alpha = 0, eta = 0, rc = 0;
  int P = 0, M = 0;
  double psi_left = 0, psi_right = 0;
  double dpsi = 0;              // (psi_right - psi_left) in e/nm
  double alpha_A = 0, tol_A = 1e-17;
  int precision = SRBE_FP64;
  int sampler = SRBE_SAMPLER_METROPOLIS;
  int32_t mmax[3] = {0, 0, 0};
  double G = 0;

  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t side = nullptr;                 // neighbour-list work beside S1 (joined before b)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_modes = nullptr;              // a captured step's mode list staged (side stream)
  cudaEvent_t ev_ii = nullptr;                 // the mixed form's ion-ion force pass done (side stream)
  bool fii_pending = false;                    // that pass was launched for the coming force pass
  srbe::DevBuf<float4> fii;                    // its per-ion forces, sorted order
  std::string err;

  bool have_ele = false, have_pos = false, have_modes = false, have_md = false;

  // electrode (fixed sites)
  int64_t ne = 0;
  srbe::DevBuf<double> ex, ey, ez, ed;         // positions and d (-1/2 | +1/2)
  srbe::DevBuf<uint64_t> eu;                   // fixed-point phase coordinates [3][ne], site order
  srbe::DevBuf<float4> epf;                    // FP32 site positions (x, y, z, 0), site order
  srbe::DevBuf<uint64_t> iu;                   // ion phase coordinates [3][ni] written by the drift of a step
  srbe::DevBuf<double> Bmat;                   // projected inverse J A^-1, ne x ne row-major
  srbe::DevBuf<float2> Bsplit;                 // its (hi, lo) FP32 split (mixed form)
  srbe::DevBuf<double> Amat;                   // A itself (kept for the refinement residual)
  srbe::DevBuf<double> we, qd;                 // A^-1 e and (J A^-1) d
  srbe::DevBuf<double> bvec, Q;                // per-step b and charges
  srbe::DevBuf<float2> bsplit;                 // b as (hi, lo) FP32 pairs (mixed form)
  srbe::DevBuf<float2> wesplit;                // A^-1 e as (hi, lo) FP32 pairs
  double s_e = 0, wd = 0;                      // e^T A^-1 e and (A^-1 e)^T d
  std::vector<double> hR;                      // host copy of R
  double wall_span = 0;                        // z extent of the electrode sites
  std::vector<int8_t> hside;
  srbe::Cells ecells;
  srbe::RunTable runtab;                       // stencil runs of the shared ion / electrode grid
  srbe::NbrLists nbr;                          // Verlet lists of the real-space sums
  srbe::PcgState pcg;                          // iterative charge solve
  srbe::MlpState mlp;                          // learned warm start

  // electrolyte
  int64_t ni = 0;
  srbe::DevBuf<double> x, y, z, q;
  srbe::DevBuf<float> q32;                     // FP32 copy of q (the mixed form's structure factor)
  srbe::DevBuf<double> vx, vy, vz, minv;
  srbe::DevBuf<double> F;                      // [3][ni] SoA force
  srbe::DevBuf<int32_t> itype, mol;
  srbe::DevBuf<int32_t> bond_start, bond_j;
  srbe::DevBuf<double> bond_r0;
  int ntype = 0;
  srbe::DevBuf<double> lj;                     // [ntype*ntype] (sigma^2, 4 eps) pairs as double2
  double kb = 0, dt = 0;
  srbe::Cells icells;

  // modes
  int K = 0;                                   // modes evaluated on the device
  int Kdet = 0;                                // of which deterministic (folded +m_z with weight x2)
  std::vector<int32_t> hm;                     // host mode list [K][4]
  std::vector<double> hc;                      // host weights [K]
  std::vector<int32_t> hsamp;                  // last sampled modes [P][3]
  bool explicit_list = false;
  srbe::DevBuf<int4> dm;
  srbe::DevBuf<double> dc;
  srbe::DevBuf<double2> S1, S2;                // structure factors (S2 holds S1 + S2 after the update)
  srbe::DevBuf<double2> tab;                   // sin/cos table

  // pinned staging for mode lists
  int4 *h_mode_stage = nullptr;
  double *h_w_stage = nullptr;
  size_t stage_cap = 0;
  cudaEvent_t stage_done = nullptr;

  // scratch (sized by srbe::reserve before any launch so that steps allocate nothing)
  srbe::DevBuf<double2> partial;               // structure-factor partials [chunks][K]
  srbe::DevBuf<double> mpart;                  // dipole partials [chunks]
  srbe::DevBuf<double2> coef;                  // per-mode c_k S(k) coefficients [K]
  srbe::DevBuf<float2> coef32;                 // their FP32 copy (mixed form)
  srbe::DevBuf<float> Q32;                     // FP32 copy of the charges (mixed form)
  srbe::DevBuf<float2> lj32;                   // FP32 (sigma^2, eps) table (mixed form)
  srbe::DevBuf<double> scal;                   // device scalars (see kScal* indices)
  srbe::DevBuf<double> epart;                  // per-block energy partials
  srbe::DevBuf<int> flag;                      // device error flag
  srbe::DevBuf<int> sfdone;                    // per mode tile: blocks of the structure factor done (self re-arming)
  srbe::DevBuf<double> resid;                  // per-row squared residuals of the FP64 check
  double h_scal[16];

  srbe::HostExt *hx = nullptr;

  // phase tracing
  bool profiling = false;
  bool use_graphs = true;                      // srbe_step replays a captured CUDA graph per step
  // Cooperative kernels (grid-wide barriers) never overlap one another: each waits on and then
  // records a chain event, the process-wide one of the device, or during a capture a capture-local one
  cudaEvent_t coop_chain = nullptr;

  srbe::Lattice lat;                           // lattice electrode path (Eqs. 15, 24 separated per layer)
  bool dense = true;                           // dense A / projected inverse exist
  bool lat_solve = false;                      // charge update through the spectral form of A
  int sf_occ = 8;                              // structure factor: blocks per SM its chunking keeps (tile)

  // Langevin thermostat (Eq. 39): collision rate (1/ps, 0 = off), temperature (K), noise seed
  double lang_gamma = 0.0, lang_T = 0.0;
  uint64_t lang_seed = 0;

  // device-raised error flags (see srbe_synchronize), one word each so that kernels set them with
  // plain stores: host-mapped pinned memory, read by the host without a copy
  int *h_status = nullptr;                     // host view
  int *d_status = nullptr;                     // device view of the same words
  int inject = 0;                              // test aid: 1 NaN into F[0], 2 NaN into Q[0] after each pass

  // counters
  int64_t launches = 0;
  int64_t mode_evals = 0;
  uint64_t md_step = 0;
};

namespace srbe {

// device error flags (ctx->d_status words)
enum { kStatNotConv = 0, kStatNonFiniteF = 1, kStatNonFiniteQ = 2, kStatBadInput = 3, kStatTimeout = 4, kStatCount = 8 };

// indices into ctx->scal (16 device scalars): dipoles sum q z and sum Q Z, psi_bar (e/nm), then the
// energy accumulators: U_N ion-ion, U_N ion-electrode, LJ, bonds, U_N electrode-electrode,
// 1/2 sum c |S|^2, sum Q^2, sum q^2
enum {
  kScalMion = 0, kScalMele = 1, kScalPsi = 2,
  kScalEnergy = 4, kScalEii = 4, kScalEie = 5, kScalElj = 6, kScalEbond = 7, kScalEee = 8,
  kScalUF = 9, kScalQ2 = 10, kScalq2 = 11, kScalCount = 16
};

// ------------------------------------------------------------------------------------------------
// Philox4x64-10 on the device (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two 64x64->128
// multiplications with the published multipliers and Weyl key increments
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64_dev(uint64_t x0, uint64_t x1, uint64_t x2, uint64_t x3, uint64_t k0,
                                               uint64_t k1, uint64_t out[4]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t hA = __umul64hi(0xD2E7470EE14C6C93ull, x0), lA = 0xD2E7470EE14C6C93ull * x0;
    const uint64_t hB = __umul64hi(0xCA5A826395121157ull, x2), lB = 0xCA5A826395121157ull * x2;
    x0 = hB ^ x1 ^ k0;
    x1 = lB;
    x2 = hA ^ x3 ^ k1;
    x3 = lA;
    k0 += 0x9E3779B97F4A7C15ull;
    k1 += 0xBB67AE8584CAA73Bull;
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}

// ------------------------------------------------------------------------------------------------
// fixed-point phases and sin/cos
// ------------------------------------------------------------------------------------------------
// A coordinate x in a period L is stored as u = frac(x / L) * 2^64 (uint64), so that the phase
// k . r = 2 pi (m_x u_x + m_y u_y + m_z u_z) / 2^64 is exact modulo one turn in integer
// arithmetic, whatever the size of m.
__device__ __forceinline__ uint64_t to_turns64(double x, double invL) {
  double t = x * invL;
  t -= floor(t);
  if (t >= 1.0) t = 0.0;
  return (uint64_t)__double2ull_rz(t * 18446744073709551616.0);
}

__device__ __forceinline__ uint64_t phase64(int4 m, uint64_t ux, uint64_t uy, uint64_t uz) {
  return (uint64_t)(int64_t)m.x * ux + (uint64_t)(int64_t)m.y * uy + (uint64_t)(int64_t)m.z * uz;
}

// cos and sin of 2 pi th / 2^64.  The top 10 bits (rounded) select a table angle
// a_j = 2 pi j / 1024; the remainder x (|x| <= pi / 1024) enters through
// sin x = x - x^3/6 + x^5/120 and cos x - 1 = -x^2/2 + x^4/24 (truncation below 1e-18) and the
// angle-addition formulas.  The remainder is turned into a double exactly by adding it to the
// bit pattern of 1.5 * 2^52.
__device__ __forceinline__ void sincos_turns(uint64_t th, const double2 *__restrict__ tab, double &c, double &s) {
  const uint64_t t = th + (1ull << 53);
  const unsigned idx = (unsigned)(t >> 54);
  const int64_t rem = (int64_t)(th - ((uint64_t)idx << 54));     // in [-2^53, 2^53)
  const int64_t v = rem >> 2;                                      // |v| <= 2^51
  const double xv = __longlong_as_double(0x4338000000000000LL + v) - 6755399441055744.0;
  constexpr double kTurn62 = 2.0 * kPi / 4611686018427387904.0;    // 2 pi / 2^62
  const double x = xv * kTurn62;
  const double x2 = x * x;
  const double sx = fma(x * x2, fma(x2, 1.0 / 120.0, -1.0 / 6.0), x);
  const double cm1 = x2 * fma(x2, 1.0 / 24.0, -0.5);
  const double2 T = __ldg(&tab[idx]);
  c = fma(T.x, cm1, fma(-T.y, sx, T.x));
  s = fma(T.y, cm1, fma(T.x, sx, T.y));
}

// FP32 form: phase in turns from 32-bit fixed point (top half), reduced to [-pi, pi).
__device__ __forceinline__ uint32_t to_turns32(double x, double invL) { return (uint32_t)(to_turns64(x, invL) >> 32); }
// small integer (|v| < 2^22) to float without a conversion instruction: added to the mantissa of
// 1.5 x 2^23, where the float spacing is 1, then the offset removed (exact)
__device__ __forceinline__ float small_int_to_float(int v) {
  return __int_as_float(0x4B400000 + v) - 12582912.0f;
}

// FP32 sin/cos of a 32-bit phase in turns: the top 23 bits (a signed value below 2^22 in
// magnitude, so converted exactly without a conversion instruction) times 2 pi / 2^23; the 7.5e-7
// rad step is below __sincosf's own error on [-pi, pi)
__device__ __forceinline__ void sincos_turns32(uint32_t th, float &c, float &s) {
  constexpr float kTurn23 = (float)(2.0 * kPi / 8388608.0);         // 2 pi / 2^23
  const float a = small_int_to_float((int32_t)th >> 9) * kTurn23;
  __sincosf(a, &s, &c);
}

// ------------------------------------------------------------------------------------------------
// kernels' host launchers (defined in the .cu files)
// ------------------------------------------------------------------------------------------------
void upload_table(srbe_ctx *c);
void build_cells(srbe_ctx *c, Cells &cl, int64_t n, const double *x, const double *y, const double *z,
                 const double *w, const int32_t *typ, const int32_t *mol, bool is_ion);
void choose_grid(const srbe_ctx *c, CellGrid &g, double zlo, double zhi);
void build_run_table(srbe_ctx *c);
void neighbor_update(srbe_ctx *c);
void neighbor_force_rebuild(srbe_ctx *c);
// coef_mode: -1 none, 0 writes (c Re S, c Im S) for the electrode right-hand side, 1 writes
// (c Im S, c Re S) for the ion forces, into ctx->coef / coef32.  u: the particles' fixed-point phase
// coordinates [3][n] if already known (else they come from x, y, z); z is read for M_z either way
void structure_factor(srbe_ctx *c, int64_t n, const double *x, const double *y, const double *z, const double *w,
                      double2 *S, const double2 *S_add, int mslot, int coef_mode, const uint64_t *u = nullptr,
                      const float *w32 = nullptr);
void electrode_rhs(srbe_ctx *c);
void charge_update(srbe_ctx *c);
void pcg_prepare(srbe_ctx *c);
int mlp_param_count();
int mlp_input_width();
void mlp_descriptors(srbe_ctx *c, float *D_dev);
void mlp_forward(srbe_ctx *c, const float *D_dev, int64_t n, float *out_dev, double *out_y_dev);
double mlp_grad_step(srbe_ctx *c, const float *D_dev, const float *T_dev, const int32_t *rows_dev, int64_t n,
                     float *grad_dev, bool apply, float lr, float wd);
void ion_forces(srbe_ctx *c, bool energies);
bool ion_forces_split(const srbe_ctx *c, bool energies);
void ion_forces_ii(srbe_ctx *c);
void integrate_kick_drift(srbe_ctx *c, double fac_kick, bool drift);
void steepest_descent_move(srbe_ctx *c, double a, double dmax);
void build_A_and_inverse(srbe_ctx *c);
void energy_scalars(srbe_ctx *c);
// raises kStatNonFiniteF / kStatNonFiniteQ if any of F [3][ni] (forces = true) or Q [ne] is not finite
void check_finite(srbe_ctx *c, bool forces, bool charges);
enum Phase {
  kPhUpload = 0, kPhCells, kPhS1, kPhRhs, kPhSolve, kPhS2, kPhForces, kPhIntegrate, kPhEnergy, kPhForcesII, kPhCount
};
void lattice_setup(srbe_ctx *c, const std::vector<double> &x, const std::vector<double> &y,
                   const std::vector<double> &z);
void lattice_bfar(srbe_ctx *c);
void lattice_s2(srbe_ctx *c, double2 *S, const double2 *S1, int mslot);
void lattice_spectral_setup(srbe_ctx *c, const std::vector<int4> &modesA, const std::vector<double> &wA,
                            double alpha_A, double rcut, int nimx, int nimy, double self, double slab);
void lattice_solve(srbe_ctx *c, const double *rhs, double *y);
void lattice_apply_A(srbe_ctx *c, const double *x, double *y);
void charge_update_lattice(srbe_ctx *c);
void coop_before(srbe_ctx *c);
void coop_after(srbe_ctx *c);
cudaEvent_t device_coop_chain();
void charge_residual(srbe_ctx *c, double *out_dev);
void phase_begin(srbe_ctx *c, int ph);
void phase_end(srbe_ctx *c, int ph);
void reserve(srbe_ctx *c);
int64_t sfac_chunks(int64_t n, int K, int occ, int64_t *chunk);

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace srbe
