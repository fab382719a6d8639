// The constant-potential charge solve.
//
// One-time (srbe_set_electrode): A of Eq. 18 on the GPU -
//   k-space  (1/V) sum_k 4 pi / k^2 exp(-k^2/4a^2) cos(k.(R_i - R_j)), evaluated as
//            sum over half the lattice of w_k [C_ki C_kj + S_ki S_kj] with per-site cos/sin tables;
//   real     sum over in-plane images of [erfc(a R) - erfc(R / (sqrt 2 eta))] / R within r_A;
//   self     2 (1 / (sqrt(2 pi) eta) - a / sqrt(pi)) on the diagonal;
//   slab     (4 pi / V) Z_i Z_j (the Hessian of the slab energy (2 pi / V) M_z^2);
// then its inverse by Gauss-Jordan elimination (A is symmetric positive definite, so the
// diagonal pivots stay positive), w_e = A^-1 e, s = e^T w_e and the projected inverse
// B = J A^-1 = A^-1 - w_e w_e^T / s (Eq. 11), and q_d = B d.
//
// Per step (Eqs. 9-10):  Q = B b + dpsi q_d,  psi_bar = -(w_e^T b + dpsi w_e^T d) / s,
// one dense FP64 matrix-vector product, one warp per row with a fixed-order shuffle reduction.
#include <cooperative_groups.h>

#include "srbe_internal.cuh"

namespace cg = cooperative_groups;

namespace srbe {

// per-site cos / sin of k . R for the A-modes (mode-major, [K][ne])
__global__ void k_site_trig(int K, int64_t ne, const int4 *__restrict__ modes, const double *__restrict__ ex,
                            const double *__restrict__ ey, const double *__restrict__ ez, double3 invL,
                            const double2 *__restrict__ tab, double *__restrict__ C, double *__restrict__ S) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (j >= ne || k >= K) return;
  double c, s;
  sincos_turns(phase64(modes[k], to_turns64(ex[j], invL.x), to_turns64(ey[j], invL.y), to_turns64(ez[j], invL.z)),
               tab, c, s);
  C[(int64_t)k * ne + j] = c;
  S[(int64_t)k * ne + j] = s;
}

// A[i][j] += sum_k w_k (C_ki C_kj + S_ki S_kj), 64 x 64 output tiles, 16 x 16 threads x (4 x 4)
constexpr int kAT = 64, kAK = 16;
__global__ void __launch_bounds__(256)
k_A_kspace(int K, int64_t ne, const double *__restrict__ w, const double *__restrict__ C,
           const double *__restrict__ S, double *__restrict__ A) {
  __shared__ double ci[kAK][kAT], si[kAK][kAT], cj[kAK][kAT], sj[kAK][kAT];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t i0 = (int64_t)blockIdx.y * kAT, j0 = (int64_t)blockIdx.x * kAT;
  if (j0 + kAT <= i0) return;   // strictly-lower tiles are mirrored at the end
  double acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += kAK) {
    __syncthreads();
    for (int e = threadIdx.x; e < kAK * kAT; e += 256) {
      const int kk = e / kAT, ii = e % kAT;
      const int k = k0 + kk;
      const bool ok = k < K;
      const double wk = ok ? w[k] : 0.0;
      const int64_t gi = i0 + ii, gj = j0 + ii;
      ci[kk][ii] = (ok && gi < ne) ? wk * C[(int64_t)k * ne + gi] : 0.0;
      si[kk][ii] = (ok && gi < ne) ? wk * S[(int64_t)k * ne + gi] : 0.0;
      cj[kk][ii] = (ok && gj < ne) ? C[(int64_t)k * ne + gj] : 0.0;
      sj[kk][ii] = (ok && gj < ne) ? S[(int64_t)k * ne + gj] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kAK; ++kk) {
      double a[4], b[4], c[4], d[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = ci[kk][ty + 16 * u];
        b[u] = si[kk][ty + 16 * u];
        c[u] = cj[kk][tx + 16 * u];
        d[u] = sj[kk][tx + 16 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], c[v], fma(b[u], d[v], acc[u][v]));
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int64_t gi = i0 + ty + 16 * u, gj = j0 + tx + 16 * v;
      if (gi < ne && gj < ne && gj >= gi) A[gi * ne + gj] += acc[u][v];
    }
}

// real-space images, self and slab terms of Eq. 18 (upper triangle incl. diagonal); writes A
__global__ void k_A_real(int64_t ne, const double *__restrict__ ex, const double *__restrict__ ey,
                         const double *__restrict__ ez, double Lx, double Ly, double alpha, double eta, double rcut,
                         int nimx, int nimy, double self, double slab, double *__restrict__ A) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = blockIdx.y;
  if (j >= ne || j < i) return;
  double dx0 = ex[i] - ex[j], dy0 = ey[i] - ey[j];
  const double dz = ez[i] - ez[j];
  dx0 -= Lx * floor(dx0 / Lx + 0.5);
  dy0 -= Ly * floor(dy0 / Ly + 0.5);
  const double rc2 = rcut * rcut, eg = 1.4142135623730951 * eta;
  double acc = 0.0;
  for (int a = -nimx; a <= nimx; ++a)
    for (int b = -nimy; b <= nimy; ++b) {
      const double dx = dx0 + a * Lx, dy = dy0 + b * Ly;
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 > 0.0 && r2 < rc2) {
        const double r = sqrt(r2);
        acc += (erfc(alpha * r) - erfc(r / eg)) / r;
      }
    }
  if (i == j) acc += self;
  acc = fma(slab * ez[i], ez[j], acc);
  A[i * ne + j] = acc;
}

__global__ void k_mirror_upper(int64_t ne, double *__restrict__ A) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = blockIdx.y;
  if (j < i && j < ne) A[i * ne + j] = A[j * ne + i];
}

// Gauss-Jordan step p, part 1: rowp[j] = A[p][j] / A[p][p] (j != p), rowp[p] = 1 / A[p][p];
// colp[i] = A[i][p].  A non-positive pivot raises the flag.
__global__ void k_gj_pivot(int64_t ne, int64_t p, const double *__restrict__ A, double *__restrict__ rowp,
                           double *__restrict__ colp, int *__restrict__ flag) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ne) return;
  const double piv = A[p * ne + p];
  if (!(piv > 0.0)) {
    if (j == 0) atomicExch(flag, 1);
    rowp[j] = 0.0;
    colp[j] = 0.0;
    return;
  }
  const double inv = 1.0 / piv;
  rowp[j] = (j == p) ? inv : A[p * ne + j] * inv;
  colp[j] = A[j * ne + p];
}

// part 2: A[i][j] -= colp[i] rowp[j] (i, j != p); A[p][j] = rowp[j]; A[i][p] = -colp[i] rowp[p]
__global__ void k_gj_update(int64_t ne, int64_t p, double *__restrict__ A, const double *__restrict__ rowp,
                            const double *__restrict__ colp) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = blockIdx.y;
  if (j >= ne) return;
  double *a = A + i * ne + j;
  if (i == p) *a = rowp[j];
  else if (j == p) *a = -colp[i] * rowp[p];
  else *a = fma(-colp[i], rowp[j], *a);
}

// y[i] = sum_j M[i][j] v[j] (+ dpsi * add[i]) for i < nrow; warp per row, fixed-order reduction.
// When wrow != nullptr, "row" nrow is the vector wrow and its result r gives
// psi_bar = -(r + dpsi * wd) / s_e, written to scal[kScalPsi].
template <class T>
__global__ void k_gemv_rows(int64_t nrow, int64_t ncol, const T *__restrict__ M, const double *__restrict__ v,
                            double dpsi, const double *__restrict__ add, double *__restrict__ y,
                            const double *__restrict__ wrow, double wd, double s_e, double *__restrict__ scal,
                            float *__restrict__ y32 = nullptr) {
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row > nrow || (row == nrow && !wrow)) return;
  double acc = 0.0;
  if (row < nrow) {
    const T *r = M + row * ncol;
    for (int64_t j = lane; j < ncol; j += 32) acc = fma((double)r[j], __ldg(v + j), acc);
  } else {
    for (int64_t j = lane; j < ncol; j += 32) acc = fma(wrow[j], __ldg(v + j), acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    if (row < nrow) {
      const double r = add ? fma(dpsi, add[row], acc) : acc;
      y[row] = r;
      if (y32) y32[row] = (float)r;
    }
    else scal[kScalPsi] = -(acc + dpsi * wd) / s_e;
  }
}

// Charge update Q = B b + dpsi q_d and psi_bar = -(w_e . b + dpsi w_e . d) / s_e (Eqs. 9-10), one
// warp per row (row n: the w_e row).  FP64 form: double2 loads, four in flight per lane.
__global__ void __launch_bounds__(256)
k_charges_fp64(int64_t n, const double *__restrict__ B, const double *__restrict__ b, double dpsi,
               const double *__restrict__ qd, const double *__restrict__ we, double wd, double s_e,
               double *__restrict__ Q, float *__restrict__ Q32, double *__restrict__ scal,
               const int *__restrict__ gate) {
  // gate (the fallback after an iterative solve): run only if *gate is set
  if (gate && *gate == 0) return;
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row > n) return;
  const double *r = row < n ? B + row * n : we;
  double a0 = 0.0, a1 = 0.0;
  int64_t j = 0;
  if ((n & 1) == 0) {
    const double2 *r2 = reinterpret_cast<const double2 *>(r);
    const double2 *b2 = reinterpret_cast<const double2 *>(b);
    const int64_t h = n >> 1;
    int64_t k = lane;
    for (; k + 96 < h; k += 128) {
      const double2 m0 = __ldcs(r2 + k), m1 = __ldcs(r2 + k + 32), m2 = __ldcs(r2 + k + 64),
                    m3 = __ldcs(r2 + k + 96);
      const double2 v0 = __ldg(b2 + k), v1 = __ldg(b2 + k + 32), v2 = __ldg(b2 + k + 64), v3 = __ldg(b2 + k + 96);
      a0 = fma(m0.x, v0.x, a0);
      a1 = fma(m0.y, v0.y, a1);
      a0 = fma(m1.x, v1.x, a0);
      a1 = fma(m1.y, v1.y, a1);
      a0 = fma(m2.x, v2.x, a0);
      a1 = fma(m2.y, v2.y, a1);
      a0 = fma(m3.x, v3.x, a0);
      a1 = fma(m3.y, v3.y, a1);
    }
    for (; k < h; k += 32) {
      const double2 m0 = __ldcs(r2 + k), v0 = __ldg(b2 + k);
      a0 = fma(m0.x, v0.x, a0);
      a1 = fma(m0.y, v0.y, a1);
    }
    j = n;
  }
  for (int64_t jj = j + lane; jj < n; jj += 32) a0 = fma(r[jj], __ldg(b + jj), a0);
  double acc = a0 + a1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    if (row < n) {
      const double q = fma(dpsi, qd[row], acc);
      Q[row] = q;
      Q32[row] = (float)q;
    } else {
      scal[kScalPsi] = -(acc + dpsi * wd) / s_e;
    }
  }
}

// Double-float arithmetic (pairs of FP32 with error-free transformations): products by FMA,
// sums by Knuth's TwoSum; about 2^-48 relative accuracy with only FP32 instructions.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_add(DF a, float b) {
  const float s = a.hi + b, bb = s - a.hi, err = (a.hi - (s - bb)) + (b - bb);
  return DF{s, a.lo + err};
}
__device__ __forceinline__ DF df_add_df(DF a, DF b) {
  const float s = a.hi + b.hi, bb = s - a.hi, err = (a.hi - (s - bb)) + (b.hi - bb);
  const float lo = err + a.lo + b.lo;
  const float h = s + lo;
  return DF{h, lo - (h - s)};
}

// Mixed form of the same update: B and b as (hi, lo) FP32 pairs; every term is the exact product
// hi*hi (FMA remainder) plus the cross terms, accumulated as a double-float.  Only the final
// combination with dpsi q_d and psi_bar run in FP64 (one lane per row).  The matrix is streamed
// once per step from HBM, so each row is split over kSplitWarps warps (contiguous column segments)
// to keep enough loads in flight; the segments' double-floats are combined in a fixed order.
constexpr int kSplitWarps = 4;
__global__ void __launch_bounds__(256)
k_charges_split(int64_t n, const float2 *__restrict__ B, const float2 *__restrict__ b, double dpsi,
                const double *__restrict__ qd, const float2 *__restrict__ we, double wd, double s_e,
                double *__restrict__ Q, float *__restrict__ Q32, double *__restrict__ scal,
                const int *__restrict__ gate) {
  __shared__ DF part[256 / 32];
  // gate (the fallback after an iterative solve): the whole block leaves unless *gate is set
  if (gate && *gate == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int seg = warp % kSplitWarps;
  const int64_t row = (int64_t)blockIdx.x * (256 / 32 / kSplitWarps) + warp / kSplitWarps;
  DF acc{0.f, 0.f};
  float lo = 0.f;
  auto term = [&](float2 m, float2 v) {
    const float p = m.x * v.x;
    const float e = fmaf(m.x, v.x, -p);
    lo += e + fmaf(m.x, v.y, m.y * v.x);
    acc = df_add(acc, p);
  };
  if (row <= n) {
    const float2 *r = row < n ? B + row * n : we;
    if ((n & 1) == 0) {
      // even n: rows start on 16-byte boundaries; two entries per 16-byte load
      const float4 *r4 = reinterpret_cast<const float4 *>(r);
      const float4 *b4 = reinterpret_cast<const float4 *>(b);
      const int64_t h = n >> 1, per = (h + kSplitWarps - 1) / kSplitWarps;
      const int64_t k0 = seg * per, k1 = min(h, k0 + per);
      int64_t k = k0 + lane;
      for (; k + 96 < k1; k += 128) {
        float4 m[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) m[u] = __ldcs(r4 + k + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float4 v = __ldg(b4 + k + 32 * u);
          term(make_float2(m[u].x, m[u].y), make_float2(v.x, v.y));
          term(make_float2(m[u].z, m[u].w), make_float2(v.z, v.w));
        }
      }
      for (; k < k1; k += 32) {
        const float4 m = __ldcs(r4 + k), v = __ldg(b4 + k);
        term(make_float2(m.x, m.y), make_float2(v.x, v.y));
        term(make_float2(m.z, m.w), make_float2(v.z, v.w));
      }
    } else {
      const int64_t per = (n + kSplitWarps - 1) / kSplitWarps;
      const int64_t k0 = seg * per, k1 = min(n, k0 + per);
      for (int64_t k = k0 + lane; k < k1; k += 32) term(__ldcs(r + k), __ldg(b + k));
    }
  }
  acc.lo += lo;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DF other{__shfl_xor_sync(0xffffffffu, acc.hi, o), __shfl_xor_sync(0xffffffffu, acc.lo, o)};
    // order the operands by lane so that both partners compute the identical sum
    acc = (lane & o) ? df_add_df(other, acc) : df_add_df(acc, other);
  }
  if (lane == 0) part[warp] = acc;
  __syncthreads();
  if (seg == 0 && lane == 0 && row <= n) {
    DF t = part[warp];
    for (int w = 1; w < kSplitWarps; ++w) t = df_add_df(t, part[warp + w]);
    const double a = (double)t.hi + (double)t.lo;
    if (row < n) {
      const double q = fma(dpsi, qd[row], a);
      Q[row] = q;
      Q32[row] = (float)q;
    } else {
      scal[kScalPsi] = -(a + dpsi * wd) / s_e;
    }
  }
}

__global__ void k_split(int64_t n, const double *__restrict__ a, float2 *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float hi = (float)a[i];
  out[i] = make_float2(hi, (float)(a[i] - (double)hi));
}

__global__ void k_rowsum(int64_t ne, const double *__restrict__ A, double *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= ne) return;
  double acc = 0.0;
  for (int64_t j = lane; j < ne; j += 32) acc += A[row * ne + j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) out[row] = acc;
}

__global__ void k_project(int64_t ne, double *__restrict__ B, const double *__restrict__ w, double inv_s) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t i = blockIdx.y;
  if (j < ne) B[i * ne + j] = fma(-w[i] * inv_s, w[j], B[i * ne + j]);
}

__global__ void k_to_float(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

static double host_dot(const std::vector<double> &a, const std::vector<double> &b) {
  double s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}

void build_A_and_inverse(srbe_ctx *c) {
  const int64_t ne = c->ne;
  c->pcg.a32_ready = false;          // the mixed form's FP32 copy of A follows the new A
  const double Lx = c->L[0], Ly = c->L[1], Lz = c->L[2];
  // alpha_A: in-plane-only real-space images are exact only if erfc(alpha_A * gap) is negligible
  double zmin = 1e300, zmax = -1e300;
  for (int64_t j = 0; j < ne; ++j) {
    zmin = std::min(zmin, c->hR[3 * j + 2]);
    zmax = std::max(zmax, c->hR[3 * j + 2]);
  }
  const double gap = Lz - (zmax - zmin);
  SRBE_REQUIRE(gap > 0.0, SRBE_EINVAL, "electrode sites span the whole periodic length Lz");
  const double tol = c->tol_A > 0 ? c->tol_A : 1e-17;
  const double xk = std::sqrt(-std::log(tol));   // exp(-x^2) = tol
  double xr = 1.0;                               // erfc(xr) = tol
  while (std::erfc(xr) >= tol) xr += 0.01;
  double aA = c->alpha_A;
  if (!(aA > 0.0)) aA = std::max(0.5, (xr + 0.6) / gap);
  c->alpha_A = aA;
  // half lattice: first nonzero of (m_z, m_y, m_x) positive, exp(-k^2/4a^2) >= tol, weight doubled
  const double kmax = 2.0 * aA * xk;
  const int mx = (int)std::floor(kmax * Lx / (2 * kPi)), my = (int)std::floor(kmax * Ly / (2 * kPi)),
            mz = (int)std::floor(kmax * Lz / (2 * kPi));
  std::vector<int4> hm;
  std::vector<double> hw;
  for (int a = -mx; a <= mx; ++a)
    for (int b = -my; b <= my; ++b)
      for (int cc = 0; cc <= mz; ++cc) {
        if (cc == 0 && (b < 0 || (b == 0 && a <= 0))) continue;
        const double kx = 2 * kPi * a / Lx, ky = 2 * kPi * b / Ly, kz = 2 * kPi * cc / Lz;
        const double k2 = kx * kx + ky * ky + kz * kz;
        const double g = std::exp(-k2 / (4 * aA * aA));
        if (g < tol) continue;
        hm.push_back(make_int4(a, b, cc, 0));
        hw.push_back(2.0 * 4.0 * kPi / (c->V * k2) * g);
      }
  const int KA = (int)hm.size();
  const double rcut0 = xr / aA;
  const int nimx0 = (int)std::ceil(rcut0 / Lx) + 1, nimy0 = (int)std::ceil(rcut0 / Ly) + 1;
  const double self0 = 2.0 * (1.0 / (std::sqrt(2.0 * kPi) * c->eta) - aA / std::sqrt(kPi));
  // lattice electrodes: the block-circulant (spectral) form of the same A, built from A's rows at
  // the layer origins and its binned modes; beyond kDenseMaxSites it is the only form of A
  lattice_spectral_setup(c, hm, hw, aA, rcut0, nimx0, nimy0, self0, 4.0 * kPi / c->V);
  c->dense = ne <= kDenseMaxSites;
  if (!c->dense) {
    SRBE_REQUIRE(c->lat.spectral, SRBE_EINVAL,
                 "more than 16,384 electrode sites are supported only for lattice electrodes (dense A would not fit)");
    std::vector<double> ones(ne, 1.0), hwe(ne), hd(ne);
    double *we = c->we.ensure(ne);
    SRBE_CUDA(cudaMemcpyAsync(c->lat.R.p, ones.data(), sizeof(double) * ne, cudaMemcpyHostToDevice, c->stream));
    lattice_solve(c, c->lat.R.p, we);
    SRBE_CUDA(cudaMemcpyAsync(hwe.data(), we, sizeof(double) * ne, cudaMemcpyDeviceToHost, c->stream));
    SRBE_CUDA(cudaStreamSynchronize(c->stream));
    for (int64_t j = 0; j < ne; ++j) hd[j] = c->hside[j] ? 0.5 : -0.5;
    double s = 0.0;
    for (int64_t j = 0; j < ne; ++j) s += hwe[j];
    SRBE_REQUIRE(s > 0.0, SRBE_ENOTCONV, "e^T A^-1 e is not positive");
    c->s_e = s;
    c->wd = host_dot(hwe, hd);
    c->bsplit.ensure(ne);
    c->lat_solve = true;
    return;
  }
  DevBuf<int4> dmA;
  DevBuf<double> dw, Ct, St, rowp, colp;
  dmA.ensure(KA);
  dw.ensure(KA);
  SRBE_CUDA(cudaMemcpyAsync(dmA.p, hm.data(), sizeof(int4) * KA, cudaMemcpyHostToDevice, c->stream));
  SRBE_CUDA(cudaMemcpyAsync(dw.p, hw.data(), sizeof(double) * KA, cudaMemcpyHostToDevice, c->stream));
  double *A = c->Bmat.ensure((size_t)ne * ne);
  const double rcut = xr / aA;
  const int nimx = (int)std::ceil(rcut / Lx) + 1, nimy = (int)std::ceil(rcut / Ly) + 1;
  const double self = 2.0 * (1.0 / (std::sqrt(2.0 * kPi) * c->eta) - aA / std::sqrt(kPi));
  {
    dim3 g(blocks_for(ne, 128), (unsigned)ne);
    k_A_real<<<g, 128, 0, c->stream>>>(ne, c->ex.p, c->ey.p, c->ez.p, Lx, Ly, aA, c->eta, rcut, nimx, nimy, self,
                                       4.0 * kPi / c->V, A);
    c->launches++;
  }
  // k-space in slabs of modes so that the cos/sin tables stay within ~1 GB
  const int64_t kslab = std::max<int64_t>(16, std::min<int64_t>(KA, (int64_t)(1ll << 26) / std::max<int64_t>(ne, 1)));
  Ct.ensure((size_t)kslab * ne);
  St.ensure((size_t)kslab * ne);
  const double3 invL = make_double3(1.0 / Lx, 1.0 / Ly, 1.0 / Lz);
  for (int64_t k0 = 0; k0 < KA; k0 += kslab) {
    const int kn = (int)std::min<int64_t>(kslab, KA - k0);
    dim3 gt(blocks_for(ne, 128), (unsigned)kn);
    k_site_trig<<<gt, 128, 0, c->stream>>>(kn, ne, dmA.p + k0, c->ex.p, c->ey.p, c->ez.p, invL, c->tab.p, Ct.p, St.p);
    const unsigned nt = (unsigned)((ne + kAT - 1) / kAT);
    k_A_kspace<<<dim3(nt, nt), 256, 0, c->stream>>>(kn, ne, dw.p + k0, Ct.p, St.p, A);
    c->launches += 2;
  }
  {
    dim3 g(blocks_for(ne, 128), (unsigned)ne);
    k_mirror_upper<<<g, 128, 0, c->stream>>>(ne, A);
    c->launches++;
  }
  // keep A for residual checks
  double *Akeep = c->Amat.ensure((size_t)ne * ne);
  SRBE_CUDA(cudaMemcpyAsync(Akeep, A, sizeof(double) * ne * ne, cudaMemcpyDeviceToDevice, c->stream));
  // Gauss-Jordan inversion in place
  rowp.ensure(ne);
  colp.ensure(ne);
  int *flag = c->flag.ensure(1);
  SRBE_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
  for (int64_t p = 0; p < ne; ++p) {
    k_gj_pivot<<<blocks_for(ne, 256), 256, 0, c->stream>>>(ne, p, A, rowp.p, colp.p, flag);
    k_gj_update<<<dim3(blocks_for(ne, 256), (unsigned)ne), 256, 0, c->stream>>>(ne, p, A, rowp.p, colp.p);
  }
  c->launches += 2 * ne;
  SRBE_CUDA(cudaGetLastError());
  int hflag = 0;
  SRBE_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  // w_e = A^-1 e, s = e^T w_e, w_e^T d
  double *we = c->we.ensure(ne);
  k_rowsum<<<blocks_for(ne * 32, 256), 256, 0, c->stream>>>(ne, A, we);
  std::vector<double> hwe(ne), hd(ne);
  SRBE_CUDA(cudaMemcpyAsync(hwe.data(), we, sizeof(double) * ne, cudaMemcpyDeviceToHost, c->stream));
  SRBE_CUDA(cudaStreamSynchronize(c->stream));
  SRBE_REQUIRE(hflag == 0, SRBE_ENOTCONV, "A is not positive definite (non-positive pivot in Gauss-Jordan)");
  for (int64_t j = 0; j < ne; ++j) hd[j] = c->hside[j] ? 0.5 : -0.5;
  double s = 0.0;
  for (int64_t j = 0; j < ne; ++j) s += hwe[j];
  SRBE_REQUIRE(s > 0.0, SRBE_ENOTCONV, "e^T A^-1 e is not positive");
  c->s_e = s;
  c->wd = host_dot(hwe, hd);
  // B = A^-1 - w_e w_e^T / s ; q_d = B d
  k_project<<<dim3(blocks_for(ne, 256), (unsigned)ne), 256, 0, c->stream>>>(ne, A, we, 1.0 / s);
  double *qd = c->qd.ensure(ne);
  k_gemv_rows<double><<<blocks_for(ne * 32, 256), 256, 0, c->stream>>>(ne, ne, A, c->ed.p, 0.0, nullptr, qd, nullptr,
                                                                      0.0, 1.0, nullptr);
  float2 *Bs = c->Bsplit.ensure((size_t)ne * ne);
  k_split<<<blocks_for(ne * ne, 256), 256, 0, c->stream>>>(ne * ne, A, Bs);
  k_split<<<blocks_for(ne, 256), 256, 0, c->stream>>>(ne, we, c->wesplit.ensure(ne));
  c->bsplit.ensure(ne);
  c->launches += 4;
  SRBE_CUDA(cudaGetLastError());
  SRBE_CUDA(cudaStreamSynchronize(c->stream));
  // the spectral solve is the default where it beats the dense matrix-vector product
  c->lat_solve = c->lat.spectral && ne >= kLatSolveMinSites;
}

// ------------------------------------------------------------------------------------------------
// Preconditioned conjugate gradients for A y = dpsi d + b (A symmetric positive definite, Eq. 18),
// Jacobi preconditioner, in one cooperative launch: the matrix-vector products run one warp per
// row, every dot product is a fixed-order two-level reduction (block partials, then each block sums
// the partials in block order, so all blocks hold the same value without another barrier), and the
// loop ends on the device when ||r|| <= tol ||v||.  Q and psi_bar follow from Eqs. 9-10:
// psi_bar = -e^T y / (e^T A^-1 e), Q = y + psi_bar A^-1 e.
// ------------------------------------------------------------------------------------------------
struct PcgArgs {
  int64_t n;
  const double *A, *dinv, *b, *d, *we;
  double dpsi, s_e, tol2;
  int maxit;
  double *y, *r, *z, *p, *Ap, *part;
  double *Q, *scal;
  float *Q32;
  int *stats;        // [0] iterations, [1] 1 if stopped at maxit above the tolerance (arms the fallback)
  double *res;       // [0] final relative residual (recomputed)
  int *status;       // the context's host-mapped error flags
  // mixed form (k_pcg_mixed): FP32 A and inner vectors
  const float *A32;
  float *r32, *z32, *p32, *Ap32, *d32, *s32, *part32;
  const float *dinv32;
};

__device__ double grid_dot_sum(const PcgArgs &a, double mine, int slot, cg::grid_group &grid) {
  __shared__ double red[256];
  const int t = threadIdx.x;
  red[t] = mine;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (t < s) red[t] += red[t + s];
    __syncthreads();
  }
  if (t == 0) a.part[slot * gridDim.x + blockIdx.x] = red[0];
  grid.sync();
  __shared__ double total;
  if (t < 32) {
    double acc = 0.0;
    for (unsigned b = t; b < gridDim.x; b += 32) acc += __ldcg(&a.part[slot * gridDim.x + b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (t == 0) total = acc;
  }
  __syncthreads();
  return total;
}

// two sums at once (one grid barrier): slots slot and slot + 1 of the block partials
__device__ double2 grid_dot_sum2(const PcgArgs &a, double m0, double m1, int slot, cg::grid_group &grid) {
  __shared__ double red2[2][256];
  const int t = threadIdx.x;
  red2[0][t] = m0;
  red2[1][t] = m1;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (t < s) {
      red2[0][t] += red2[0][t + s];
      red2[1][t] += red2[1][t + s];
    }
    __syncthreads();
  }
  if (t == 0) {
    a.part[slot * gridDim.x + blockIdx.x] = red2[0][0];
    a.part[(slot + 1) * gridDim.x + blockIdx.x] = red2[1][0];
  }
  grid.sync();
  __shared__ double total2[2];
  if (t < 64) {
    const int k = t >> 5, lane = t & 31;
    double acc = 0.0;
    for (unsigned b = lane; b < gridDim.x; b += 32) acc += __ldcg(&a.part[(slot + k) * gridDim.x + b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) total2[k] = acc;
  }
  __syncthreads();
  return make_double2(total2[0], total2[1]);
}

// Matrix-vector products of the iterative solves.  Block b takes the rows b, b + G, b + 2G, ...
// (G blocks) kGemvRows at a time, and its 8 warps split every row's columns into 8 contiguous
// segments: each lane keeps kGemvRows independent row loads in flight per load of x, which the
// warp-per-row form (one dependent chain per lane) did not.  The 8 segment partials of a row are
// added in segment order.
constexpr int kGemvRows = 11;
constexpr int kGemvUnroll = 3;
template <class V> struct Vec;          // 16-byte vector of the matrix type
template <> struct Vec<float> {
  using T = float4;
  static constexpr int W = 4;
  __device__ static float dot(T m, T v) { return fmaf(m.x, v.x, fmaf(m.y, v.y, fmaf(m.z, v.z, m.w * v.w))); }
};
template <> struct Vec<double> {
  using T = double2;
  static constexpr int W = 2;
  __device__ static double dot(T m, T v) { return fma(m.x, v.x, m.y * v.y); }
};
template <class T>
__device__ void block_rows_gemv(int64_t n, const T *__restrict__ A, const T *__restrict__ x, int64_t r0,
                                T (*part)[kGemvRows]) {
  using V = Vec<T>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t G = gridDim.x;
  T acc[kGemvRows];
#pragma unroll
  for (int k = 0; k < kGemvRows; ++k) acc[k] = 0;
  if (n % V::W == 0) {
    // 16-byte loads (rows start on 16-byte boundaries), kGemvUnroll column steps of all kGemvRows
    // rows issued before any is used: the product is bound by the loads in flight, not by the FMAs
    using VT = typename V::T;
    const int64_t nv = n / V::W, seg = (nv + 7) / 8, c0 = warp * seg, c1 = min(nv, c0 + seg);
    const VT *xv = reinterpret_cast<const VT *>(x);
    const VT zero{};
    for (int64_t j0 = c0 + lane; j0 < c1; j0 += 32 * kGemvUnroll) {
      VT m[kGemvUnroll][kGemvRows], v[kGemvUnroll];
#pragma unroll
      for (int u = 0; u < kGemvUnroll; ++u) {
        const int64_t j = j0 + 32 * u;
        v[u] = j < c1 ? __ldcg(xv + j) : zero;
#pragma unroll
        for (int k = 0; k < kGemvRows; ++k) {
          const int64_t row = r0 + k * G;
          m[u][k] = (j < c1 && row < n) ? __ldcs(reinterpret_cast<const VT *>(A + row * n) + j) : zero;
        }
      }
#pragma unroll
      for (int u = 0; u < kGemvUnroll; ++u)
#pragma unroll
        for (int k = 0; k < kGemvRows; ++k) acc[k] += V::dot(m[u][k], v[u]);
    }
  } else {
    const int64_t seg = (n + 7) / 8, c0 = warp * seg, c1 = min(n, c0 + seg);
    for (int64_t j = c0 + lane; j < c1; j += 32) {
      const T v = __ldcg(x + j);
#pragma unroll
      for (int k = 0; k < kGemvRows; ++k) {
        const int64_t row = r0 + k * G;
        if (row < n) acc[k] = fma(__ldcs(A + row * n + j), v, acc[k]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kGemvRows; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
  }
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < kGemvRows; ++k) part[warp][k] = acc[k];
}

// out = v - A x (minus = true) or A x in FP64
__device__ void grid_gemv(const PcgArgs &a, const double *x, const double *v, double *out, bool minus) {
  __shared__ double part[8][kGemvRows];
  const int64_t G = gridDim.x;
  for (int64_t r0 = blockIdx.x; r0 < a.n; r0 += G * kGemvRows) {
    block_rows_gemv<double>(a.n, a.A, x, r0, part);
    __syncthreads();
    if (threadIdx.x < kGemvRows) {
      const int64_t row = r0 + threadIdx.x * G;
      if (row < a.n) {
        double s = part[0][threadIdx.x];
        for (int w = 1; w < 8; ++w) s += part[w][threadIdx.x];
        out[row] = minus ? v[row] - s : s;
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_pcg(PcgArgs a) {
  cg::grid_group grid = cg::this_grid();
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
  // v = dpsi d + b lives in p for the first product; r = v - A y
  for (int64_t i = gt; i < a.n; i += gs) a.p[i] = fma(a.dpsi, a.d[i], a.b[i]);
  grid.sync();
  grid_gemv(a, a.y, a.p, a.r, true);
  grid.sync();
  double vv = 0.0, rz = 0.0, rr = 0.0;
  for (int64_t i = gt; i < a.n; i += gs) {
    const double v = a.p[i];
    vv += v * v;
  }
  vv = grid_dot_sum(a, vv, 0, grid);
  for (int64_t i = gt; i < a.n; i += gs) {
    const double zi = a.dinv[i] * a.r[i];
    a.z[i] = zi;
    rz += a.r[i] * zi;
    rr += a.r[i] * a.r[i];
  }
  rz = grid_dot_sum(a, rz, 1, grid);
  rr = grid_dot_sum(a, rr, 2, grid);
  for (int64_t i = gt; i < a.n; i += gs) a.p[i] = a.z[i];
  grid.sync();
  int it = 0;
  while (it < a.maxit && rr > a.tol2 * vv) {
    grid_gemv(a, a.p, nullptr, a.Ap, false);
    grid.sync();
    double pap = 0.0;
    for (int64_t i = gt; i < a.n; i += gs) pap += a.p[i] * a.Ap[i];
    pap = grid_dot_sum(a, pap, 3, grid);
    const double alpha = rz / pap;
    double rz1 = 0.0, rr1 = 0.0;
    for (int64_t i = gt; i < a.n; i += gs) {
      a.y[i] = fma(alpha, a.p[i], a.y[i]);
      const double ri = fma(-alpha, a.Ap[i], a.r[i]);
      a.r[i] = ri;
      const double zi = a.dinv[i] * ri;
      a.z[i] = zi;
      rz1 += ri * zi;
      rr1 += ri * ri;
    }
    rz1 = grid_dot_sum(a, rz1, 4 + (it & 1) * 2, grid);
    rr1 = grid_dot_sum(a, rr1, 5 + (it & 1) * 2, grid);
    const double beta = rz1 / rz;
    rz = rz1;
    rr = rr1;
    for (int64_t i = gt; i < a.n; i += gs) a.p[i] = fma(beta, a.p[i], a.z[i]);
    grid.sync();
    ++it;
  }
  // true residual, neutrality projection and psi_bar (Eqs. 9-10)
  for (int64_t i = gt; i < a.n; i += gs) a.z[i] = fma(a.dpsi, a.d[i], a.b[i]);
  grid.sync();
  grid_gemv(a, a.y, a.z, a.r, true);
  grid.sync();
  double r2 = 0.0, ey = 0.0;
  for (int64_t i = gt; i < a.n; i += gs) {
    r2 += a.r[i] * a.r[i];
    ey += a.y[i];
  }
  r2 = grid_dot_sum(a, r2, 8, grid);
  ey = grid_dot_sum(a, ey, 9, grid);
  const double psi = -ey / a.s_e;
  for (int64_t i = gt; i < a.n; i += gs) {
    const double q = fma(psi, a.we[i], a.y[i]);
    a.Q[i] = q;
    a.Q32[i] = (float)q;
  }
  if (gt == 0) {
    a.scal[kScalPsi] = psi;
    a.stats[0] = it;
    a.res[0] = sqrt(r2 / vv);
    // stopped at maxit above the tolerance: raise the host flag and arm the direct fallback
    const int failed = rr > a.tol2 * vv ? 1 : 0;
    a.stats[1] = failed;
    if (failed) *(volatile int *)(a.status + kStatNotConv) = 1;
  }
}

// The mixed form's inner sums: FP32, a warp tree, the 8 warps in order, then the block partials in
// block order (one grid barrier for three sums); two alternating partial slots
__device__ float3 grid_sum3f(const PcgArgs &a, float v0, float v1, float v2, int slot, cg::grid_group &grid) {
  __shared__ float wred[3][8];
  __shared__ float3 tot;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_xor_sync(0xffffffffu, v0, o);
    v1 += __shfl_xor_sync(0xffffffffu, v1, o);
    v2 += __shfl_xor_sync(0xffffffffu, v2, o);
  }
  if (lane == 0) {
    wred[0][warp] = v0;
    wred[1][warp] = v1;
    wred[2][warp] = v2;
  }
  __syncthreads();
  float *P = a.part32 + (size_t)slot * 3 * gridDim.x;
  if (threadIdx.x == 0) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int w = 0; w < 8; ++w) {
      s0 += wred[0][w];
      s1 += wred[1][w];
      s2 += wred[2][w];
    }
    P[blockIdx.x] = s0;
    P[gridDim.x + blockIdx.x] = s1;
    P[2 * gridDim.x + blockIdx.x] = s2;
  }
  grid.sync();
  if (warp == 0) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (unsigned b = lane; b < gridDim.x; b += 32) {
      s0 += __ldcg(P + b);
      s1 += __ldcg(P + gridDim.x + b);
      s2 += __ldcg(P + 2 * gridDim.x + b);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) tot = make_float3(s0, s1, s2);
  }
  __syncthreads();
  return tot;
}

// w = A32 u in FP32 (block rows, warp column segments); returns this thread's share of (w, u)
__device__ float grid_gemv32_dot(const PcgArgs &a, const float *u, float *w) {
  __shared__ float part[8][kGemvRows];
  const int64_t G = gridDim.x;
  float dl = 0.f;
  for (int64_t r0 = blockIdx.x; r0 < a.n; r0 += G * kGemvRows) {
    block_rows_gemv<float>(a.n, a.A32, u, r0, part);
    __syncthreads();
    if (threadIdx.x < kGemvRows) {
      const int64_t row = r0 + threadIdx.x * G;
      if (row < a.n) {
        float s = part[0][threadIdx.x];
        for (int k = 1; k < 8; ++k) s += part[k][threadIdx.x];
        w[row] = s;
        dl = fmaf(s, __ldcg(u + row), dl);
      }
    }
    __syncthreads();
  }
  return dl;
}

// The mixed form's iterative solve: iterative refinement in FP64 around Jacobi-PCG in FP32.  Each
// outer pass forms the FP64 residual r = dpsi d + b - A y with A in FP64 and stops once
// ||r|| <= tol ||dpsi d + b||; otherwise it solves A delta = r on an FP32 copy of A until the inner
// residual has fallen by 1e-4, and adds delta to y in FP64.  The inner solve is the Chronopoulos-Gear
// form of preconditioned CG (Chronopoulos and Gear, J. Comput. Appl. Math. 25, 1989): it applies A to
// the preconditioned residual u = M^-1 r and updates A p by the recurrence s = w + beta s, so the three
// inner products of an iteration, (r, u), (A u, u) and (r, r), share one grid barrier; an iteration
// costs two grid barriers instead of four.  maxit bounds the inner iterations over all passes; the
// iteration count reported is theirs.  Q and psi_bar follow from Eqs. 9-10 as in k_pcg.
__global__ void __launch_bounds__(256, 1) k_pcg_mixed(PcgArgs a) {
  cg::grid_group grid = cg::this_grid();
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
  int slot = 0, fslot = 0;
  double vv = 0.0;
  for (int64_t i = gt; i < a.n; i += gs) {
    const double v = fma(a.dpsi, a.d[i], a.b[i]);
    a.p[i] = v;
    vv += v * v;
  }
  vv = grid_dot_sum(a, vv, slot, grid);
  slot = (slot + 1) & 7;            // its grid barrier also orders the writes of p before the products below
  int it = 0;
  bool converged = false;
  float *x = a.d32, *r = a.r32, *u = a.z32, *w = a.Ap32, *p = a.p32, *s = a.s32;
  for (int outer = 0; outer < 16; ++outer) {
    grid_gemv(a, a.y, a.p, a.r, true);
    grid.sync();
    double rr = 0.0;
    for (int64_t i = gt; i < a.n; i += gs) rr += a.r[i] * a.r[i];
    rr = grid_dot_sum(a, rr, slot, grid);
    slot = (slot + 1) & 7;
    if (rr <= a.tol2 * vv) {
      converged = true;
      break;
    }
    if (it >= a.maxit) break;
    // inner FP32 solve of A delta = r (delta in x)
    float gam = 0.f, rr32 = 0.f;
    for (int64_t i = gt; i < a.n; i += gs) {
      const float ri = (float)a.r[i], ui = a.dinv32[i] * ri;
      r[i] = ri;
      u[i] = ui;
      x[i] = 0.f;
      p[i] = 0.f;
      s[i] = 0.f;
      gam = fmaf(ri, ui, gam);
      rr32 = fmaf(ri, ri, rr32);
    }
    grid.sync();
    float dl = grid_gemv32_dot(a, u, w);
    float3 t = grid_sum3f(a, gam, dl, rr32, fslot, grid);
    fslot ^= 1;
    float gamma = t.x, alpha = t.x / t.y, beta = 0.f;
    const float stop = (float)(1e-8 * rr);   // inner residual 1e-4 of the outer one
    float rrc = t.z;
    while (it < a.maxit && rrc > stop) {
      gam = 0.f;
      rr32 = 0.f;
      for (int64_t i = gt; i < a.n; i += gs) {
        const float pi = fmaf(beta, p[i], u[i]), si = fmaf(beta, s[i], __ldcg(w + i));
        p[i] = pi;
        s[i] = si;
        x[i] = fmaf(alpha, pi, x[i]);
        const float ri = fmaf(-alpha, si, r[i]);
        r[i] = ri;
        const float ui = a.dinv32[i] * ri;
        u[i] = ui;
        gam = fmaf(ri, ui, gam);
        rr32 = fmaf(ri, ri, rr32);
      }
      grid.sync();
      dl = grid_gemv32_dot(a, u, w);
      t = grid_sum3f(a, gam, dl, rr32, fslot, grid);
      fslot ^= 1;
      beta = t.x / gamma;
      alpha = t.x / (t.y - beta * t.x / alpha);
      gamma = t.x;
      rrc = t.z;
      ++it;
    }
    for (int64_t i = gt; i < a.n; i += gs) a.y[i] += (double)x[i];
    grid.sync();
  }
  // true residual, neutrality projection and psi_bar (Eqs. 9-10)
  grid_gemv(a, a.y, a.p, a.r, true);
  grid.sync();
  double r2 = 0.0, ey = 0.0;
  for (int64_t i = gt; i < a.n; i += gs) {
    r2 += a.r[i] * a.r[i];
    ey += a.y[i];
  }
  r2 = grid_dot_sum(a, r2, slot, grid);
    slot = (slot + 1) & 7;
  ey = grid_dot_sum(a, ey, slot, grid);
    slot = (slot + 1) & 7;
  const double psi = -ey / a.s_e;
  for (int64_t i = gt; i < a.n; i += gs) {
    const double q = fma(psi, a.we[i], a.y[i]);
    a.Q[i] = q;
    a.Q32[i] = (float)q;
  }
  if (gt == 0) {
    a.scal[kScalPsi] = psi;
    a.stats[0] = it;
    a.res[0] = sqrt(r2 / vv);
    const int failed = converged || r2 <= a.tol2 * vv ? 0 : 1;
    a.stats[1] = failed;
    if (failed) *(volatile int *)(a.status + kStatNotConv) = 1;
  }
}

__global__ void k_to_float_n(int64_t n, const double *__restrict__ a, float *__restrict__ b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

void charge_update_pcg(srbe_ctx *c) {
  const int64_t n = c->ne;
  const bool mixed = c->precision == SRBE_MIXED;
  static int blocks_per_sm = 0, nsm = 0;
  if (!blocks_per_sm) {
    int dev = 0, b1 = 0, b2 = 0;
    SRBE_CUDA(cudaGetDevice(&dev));
    SRBE_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    SRBE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b1, k_pcg, 256, 0));
    SRBE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_pcg_mixed, 256, 0));
    blocks_per_sm = std::min(b1, b2);
    SRBE_REQUIRE(blocks_per_sm > 0, SRBE_ECUDA, "PCG kernel cannot be resident");
  }
  if (mixed && !c->pcg.a32_ready) {
    // the FP32 copy of A, formed once per electrode (outside any capture: the first pass after a
    // state change runs the ordinary way)
    float *A32 = c->pcg.A32.ensure((size_t)n * n);
    k_to_float_n<<<std::min<unsigned>(blocks_for(n * n, 256), 4096u), 256, 0, c->stream>>>(n * n, c->Amat.p, A32);
    c->pcg.r32.ensure(n);
    c->pcg.z32.ensure(n);
    c->pcg.p32.ensure(n);
    c->pcg.Ap32.ensure(n);
    c->pcg.d32.ensure(n);
    c->pcg.s32.ensure(n);
    k_to_float_n<<<blocks_for(n, 256), 256, 0, c->stream>>>(n, c->pcg.dinv.p, c->pcg.dinv32.ensure(n));
    c->launches += 2;
    SRBE_CUDA(cudaGetLastError());
    c->pcg.a32_ready = true;
  }
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n * 32 + 255) / 256, (int64_t)blocks_per_sm * nsm));
  PcgArgs a;
  a.n = n;
  a.A = c->Amat.p;
  a.dinv = c->pcg.dinv.p;
  a.b = c->bvec.p;
  a.d = c->ed.p;
  a.we = c->we.p;
  a.dpsi = c->dpsi;
  a.s_e = c->s_e;
  a.tol2 = c->pcg.tol * c->pcg.tol;
  a.maxit = c->pcg.maxit;
  a.y = c->pcg.y.p;
  a.r = c->pcg.r.p;
  a.z = c->pcg.z.p;
  a.p = c->pcg.p.p;
  a.Ap = c->pcg.Ap.p;
  a.part = c->pcg.part.ensure((size_t)grid * 10);
  a.A32 = c->pcg.A32.p;
  a.r32 = c->pcg.r32.p;
  a.z32 = c->pcg.z32.p;
  a.p32 = c->pcg.p32.p;
  a.Ap32 = c->pcg.Ap32.p;
  a.d32 = c->pcg.d32.p;
  a.s32 = c->pcg.s32.p;
  a.dinv32 = c->pcg.dinv32.p;
  a.part32 = c->pcg.part32.ensure((size_t)grid * 6);
  a.Q = c->Q.p;
  a.Q32 = c->Q32.p;
  a.scal = c->scal.p;
  a.stats = c->pcg.stats.p;
  a.res = c->pcg.res.p;
  a.status = c->d_status;
  void *args[] = {&a};
  coop_before(c);
  SRBE_CUDA(cudaLaunchCooperativeKernel(mixed ? (const void *)k_pcg_mixed : (const void *)k_pcg, dim3(grid), dim3(256),
                                        args, 0, c->stream));
  coop_after(c);
  c->launches++;
}

__global__ void k_diag_inv(int64_t n, const double *__restrict__ A, double *__restrict__ dinv) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dinv[i] = 1.0 / A[i * n + i];
}

void pcg_prepare(srbe_ctx *c) {
  const int64_t n = c->ne;
  c->pcg.a32_ready = false;
  c->pcg.dinv.ensure(n);
  c->pcg.y.ensure(n);
  c->pcg.r.ensure(n);
  c->pcg.z.ensure(n);
  c->pcg.p.ensure(n);
  c->pcg.Ap.ensure(n);
  c->pcg.stats.ensure(4);
  c->pcg.res.ensure(4);
  k_diag_inv<<<blocks_for(n, 256), 256, 0, c->stream>>>(n, c->Amat.p, c->pcg.dinv.p);
  SRBE_CUDA(cudaMemsetAsync(c->pcg.y.p, 0, sizeof(double) * n, c->stream));
  SRBE_CUDA(cudaGetLastError());
}

// Q and psi_bar through the projected inverse (one matrix-vector product); with a gate, only if *gate
void charge_update_direct(srbe_ctx *c, const int *gate) {
  const int64_t ne = c->ne;
  const unsigned nb = blocks_for((ne + 1) * 32, 256);
  if (c->precision == SRBE_MIXED)
    k_charges_split<<<blocks_for(ne + 1, 256 / 32 / kSplitWarps), 256, 0, c->stream>>>(
        ne, c->Bsplit.p, c->bsplit.p, c->dpsi, c->qd.p, c->wesplit.p, c->wd, c->s_e, c->Q.p, c->Q32.p, c->scal.p,
        gate);
  else
    k_charges_fp64<<<nb, 256, 0, c->stream>>>(ne, c->Bmat.p, c->bvec.p, c->dpsi, c->qd.p, c->we.p, c->wd, c->s_e,
                                              c->Q.p, c->Q32.p, c->scal.p, gate);
  c->launches++;
  SRBE_CUDA(cudaGetLastError());
}

void charge_update(srbe_ctx *c) {
  if (c->lat_solve) {
    charge_update_lattice(c);
    return;
  }
  if (c->pcg.on) {
    if (c->pcg.warm == 0) {
      SRBE_CUDA(cudaMemsetAsync(c->pcg.y.p, 0, sizeof(double) * c->ne, c->stream));
    } else if (c->pcg.warm == 2) {
      SRBE_REQUIRE(c->mlp.ready, SRBE_ESTATE, "learned warm start needs srbe_mlp_init or srbe_mlp_set_params");
      c->mlp.D.ensure((size_t)c->ne * mlp_input_width());
      mlp_descriptors(c, c->mlp.D.p);
      mlp_forward(c, c->mlp.D.p, c->ne, nullptr, c->pcg.y.p);
    }
    charge_update_pcg(c);
    // the direct solve of the same right-hand side, run only when PCG stopped at maxit above tol
    charge_update_direct(c, c->pcg.stats.p + 1);
    return;
  }
  charge_update_direct(c, nullptr);
}

// FP64 check of the constant-potential conditions (Eqs. 9-10) met by the charges in use:
// A Q = dpsi d + b + psi_bar e, so row i of the residual is (A Q)_i - dpsi d_i - b_i - psi_bar.
// Warp per row; the squared residual and the squared right-hand side of each row go to rr[2 i].
__global__ void __launch_bounds__(256)
k_cp_residual_rows(int64_t n, const double *__restrict__ A, const double *__restrict__ Q, const double *__restrict__ d,
                   const double *__restrict__ b, double dpsi, const double *__restrict__ scal,
                   double *__restrict__ rr) {
  const int lane = threadIdx.x & 31;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (row >= n) return;
  const double *a = A + row * n;
  double acc = 0.0;
  for (int64_t j = lane; j < n; j += 32) acc = fma(__ldcs(a + j), __ldg(Q + j), acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    const double rhs = fma(dpsi, d[row], b[row]);
    const double r = acc - rhs - scal[kScalPsi];
    rr[2 * row] = r * r;
    rr[2 * row + 1] = rhs * rhs;
  }
}

// one block: out[0] = sum of squared residuals, out[1] = sum of squared right-hand sides (fixed order)
__global__ void k_cp_residual_sum(int64_t n, const double *__restrict__ rr, double *__restrict__ out) {
  __shared__ double red[2][256];
  const int t = threadIdx.x;
  double a = 0.0, b = 0.0;
  for (int64_t i = t; i < n; i += 256) {
    a += rr[2 * i];
    b += rr[2 * i + 1];
  }
  red[0][t] = a;
  red[1][t] = b;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (t < s) {
      red[0][t] += red[0][t + s];
      red[1][t] += red[1][t + s];
    }
    __syncthreads();
  }
  if (t == 0) {
    out[0] = red[0][0];
    out[1] = red[1][0];
  }
}

// the same residual from a precomputed A Q (spectral form of A, no dense matrix)
__global__ void k_cp_residual_vec(int64_t n, const double *__restrict__ AQ, const double *__restrict__ d,
                                  const double *__restrict__ b, double dpsi, const double *__restrict__ scal,
                                  double *__restrict__ rr) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double rhs = fma(dpsi, d[i], b[i]);
  const double r = AQ[i] - rhs - scal[kScalPsi];
  rr[2 * i] = r * r;
  rr[2 * i + 1] = rhs * rhs;
}

void charge_residual(srbe_ctx *c, double *out_dev) {
  const int64_t n = c->ne;
  double *rr = c->resid.ensure((size_t)2 * std::max<int64_t>(n, 1));
  if (!c->dense) {
    double *aq = c->lat.Y.p;
    lattice_apply_A(c, c->Q.p, aq);
    k_cp_residual_vec<<<blocks_for(n, 256), 256, 0, c->stream>>>(n, aq, c->ed.p, c->bvec.p, c->dpsi, c->scal.p, rr);
    k_cp_residual_sum<<<1, 256, 0, c->stream>>>(n, rr, out_dev);
    c->launches += 2;
    SRBE_CUDA(cudaGetLastError());
    return;
  }
  k_cp_residual_rows<<<blocks_for(n * 32, 256), 256, 0, c->stream>>>(n, c->Amat.p, c->Q.p, c->ed.p, c->bvec.p,
                                                                      c->dpsi, c->scal.p, rr);
  k_cp_residual_sum<<<1, 256, 0, c->stream>>>(n, rr, out_dev);
  c->launches += 2;
  SRBE_CUDA(cudaGetLastError());
}

// 1/2 sum_k c_k |S(k)|^2, sum Q^2, sum q^2 into scal (one block, fixed order)
__global__ void k_energy_scalars(int K, const double *__restrict__ cw, const double2 *__restrict__ S, int64_t ne,
                                 const double *__restrict__ Q, int64_t ni, const double *__restrict__ q,
                                 double *__restrict__ scal) {
  __shared__ double red[3][256];
  const int t = threadIdx.x;
  double a = 0, b = 0, d = 0;
  for (int k = t; k < K; k += 256) a += 0.5 * cw[k] * (S[k].x * S[k].x + S[k].y * S[k].y);
  for (int64_t j = t; j < ne; j += 256) b += Q[j] * Q[j];
  for (int64_t i = t; i < ni; i += 256) d += q[i] * q[i];
  red[0][t] = a;
  red[1][t] = b;
  red[2][t] = d;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (t < s)
      for (int e = 0; e < 3; ++e) red[e][t] += red[e][t + s];
    __syncthreads();
  }
  if (t == 0) {
    scal[kScalUF] = red[0][0];
    scal[kScalQ2] = red[1][0];
    scal[kScalq2] = red[2][0];
  }
}

void energy_scalars(srbe_ctx *c) {
  k_energy_scalars<<<1, 256, 0, c->stream>>>(c->K, c->dc.p, c->S2.p, c->ne, c->Q.p, c->ni, c->q.p, c->scal.p);
  c->launches++;
  SRBE_CUDA(cudaGetLastError());
}

}  // namespace srbe
