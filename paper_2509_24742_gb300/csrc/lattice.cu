// Electrode structure factor and far-field right-hand side for electrodes that are rectangular
// lattices commensurate with the box.
//
// When every layer l of the electrode holds the sites R = (x0_l + ix Lx / nx, y0_l + iy Ly / ny, Z_l),
// 0 <= ix < nx, 0 <= iy < ny, the phase of a mode m factorises:
//   k . R = phi_l(k) + 2 pi (m_x ix / nx + m_y iy / ny),  phi_l(k) = k_x x0_l + k_y y0_l + k_z Z_l,
// so the sums of Eq. 15 and Eq. 24 over the electrode only depend on (m_x mod nx, m_y mod ny):
//   S2(k)  = sum_l e^{i phi_l(k)} Qhat_l[m_y mod ny][m_x mod nx],
//            Qhat_l[b][a] = sum_{ix,iy} Q_l[iy][ix] e^{2 pi i (a ix / nx + b iy / ny)}   (a 2D DFT),
//   b_F,j  = - Re sum_{a,b} W_l[b][a] e^{-2 pi i (a ix / nx + b iy / ny)},
//            W_l[b][a] = sum_{k in bin (a, b)} c_k S1(k) e^{-i phi_l(k)}.
// This replaces the K x N_ele mode-site evaluations of the plain path by two small DFTs per layer
// (O(N_ele (nx + ny))) and O(K x layers) mode work.  Everything here is FP64 in both precision forms
// (the DFT work is a few MFLOP); sums run in a fixed order, so results are reproducible.
#include "srbe_internal.cuh"

#include <algorithm>
#include <cmath>

namespace srbe {

namespace {

struct LatDev {
  int nl, nx, ny;
  const int32_t *site;       // [nl][ny][nx] -> electrode site index
  const uint64_t *lu;        // [3][nl] layer origins in turns
  const double2 *twx, *twy;  // e^{2 pi i t / nx}, e^{2 pi i t / ny}
};

LatDev lat_dev(const srbe_ctx *c) {
  const Lattice &L = c->lat;
  LatDev d;
  d.nl = L.nl;
  d.nx = L.nx;
  d.ny = L.ny;
  d.site = L.site.p;
  d.lu = L.lu.p;
  d.twx = L.twx.p;
  d.twy = L.twy.p;
  return d;
}

__device__ __forceinline__ int pmod(int a, int n) {
  const int r = a % n;
  return r < 0 ? r + n : r;
}

// One 1D DFT of length n per warp ("line"), the line's input staged in shared memory next to the
// twiddle table so that the O(n) inner loop runs at shared-memory latency; lanes take the outputs.
//   kFwdX: rows (l, iy):    T[l][iy][a]  = sum_ix Q[site(l, iy, ix)] w_nx^{a ix}
//   kFwdY: columns (l, a):  Qh[l][b][a]  = sum_iy T[l][iy][a] w_ny^{b iy}
//   kInvY: columns (l, a):  U[l][iy][a]  = sum_b  W[l][b][a] w_ny^{-b iy}
//   kInvX: rows (l, iy):    bF[site(l, iy, ix)] = - Re sum_a U[l][iy][a] w_nx^{-a ix}
//   kInvXp: as kInvX but + Re into a per-site array (the spectral solve's y)
enum { kFwdX = 0, kFwdY = 1, kInvY = 2, kInvX = 3, kInvXp = 4 };
constexpr int kLineWarps = 2;

template <int MODE>
__global__ void __launch_bounds__(32 * kLineWarps)
k_lat_line(LatDev L, const double *__restrict__ Q, const double2 *__restrict__ in, double2 *__restrict__ out,
           double *__restrict__ bF) {
  extern __shared__ double2 sm[];
  constexpr bool along_x = (MODE == kFwdX || MODE == kInvX || MODE == kInvXp);
  constexpr bool conj = (MODE == kInvY || MODE == kInvX || MODE == kInvXp);
  const int n = along_x ? L.nx : L.ny;
  const int64_t lines = along_x ? (int64_t)L.nl * L.ny : (int64_t)L.nl * L.nx;
  double2 *tw = sm;
  const double2 *twg = along_x ? L.twx : L.twy;
  for (int t = threadIdx.x; t < n; t += 32 * kLineWarps) tw[t] = twg[t];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t line = (int64_t)blockIdx.x * kLineWarps + warp;
  double2 *v = sm + n + warp * n;
  if (line < lines) {
    for (int t = lane; t < n; t += 32) {
      double2 x;
      if (MODE == kFwdX) {
        x = make_double2(Q[L.site[line * L.nx + t]], 0.0);
      } else if (MODE == kInvX || MODE == kInvXp) {
        x = in[line * L.nx + t];
      } else {
        const int64_t l = line / L.nx, a = line % L.nx;
        x = in[(l * L.ny + t) * L.nx + a];
      }
      v[t] = x;
    }
  }
  __syncthreads();
  if (line >= lines) return;
  for (int s = lane; s < n; s += 32) {
    double re = 0.0, im = 0.0;
    int p = 0;                                  // (s t) mod n
    for (int t = 0; t < n; ++t) {
      const double2 x = v[t], w = tw[p];
      if (conj) {
        re = fma(x.x, w.x, fma(x.y, w.y, re));
        im = fma(x.y, w.x, fma(-x.x, w.y, im));
      } else {
        re = fma(x.x, w.x, fma(-x.y, w.y, re));
        im = fma(x.x, w.y, fma(x.y, w.x, im));
      }
      p += s;
      if (p >= n) p -= n;
    }
    if (MODE == kFwdX) {
      out[line * L.nx + s] = make_double2(re, im);
    } else if (MODE == kInvX) {
      bF[L.site[line * L.nx + s]] = -re;
    } else if (MODE == kInvXp) {
      bF[L.site[line * L.nx + s]] = re;
    } else {
      const int64_t l = line / L.nx, a = line % L.nx;
      out[(l * L.ny + s) * L.nx + a] = make_double2(re, im);
    }
  }
}

// Q: real per-site input of kFwdX; dst: per-site output of kInvX / kInvXp
template <int MODE>
void launch_line(srbe_ctx *c, const LatDev &L, const double2 *in, double2 *out, const double *Q = nullptr,
                 double *dst = nullptr) {
  constexpr bool along_x = (MODE == kFwdX || MODE == kInvX || MODE == kInvXp);
  const int n = along_x ? L.nx : L.ny;
  const int64_t lines = along_x ? (int64_t)L.nl * L.ny : (int64_t)L.nl * L.nx;
  const size_t smem = sizeof(double2) * (size_t)n * (1 + kLineWarps);
  k_lat_line<MODE><<<blocks_for(lines, kLineWarps), 32 * kLineWarps, smem, c->stream>>>(
      L, Q ? Q : c->Q.p, in, out, dst ? dst : c->lat.bF.p);
  c->launches++;
}

// E[k][l] = e^{i phi_l(k)}: one thread per (mode, layer), once per step (both paths use it)
__global__ void k_lat_phase(LatDev L, int K, const int4 *__restrict__ modes, const double2 *__restrict__ tab,
                            double2 *__restrict__ E) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)K * L.nl) return;
  const int k = (int)(t / L.nl), l = (int)(t % L.nl);
  double cs, sn;
  sincos_turns(phase64(__ldg(&modes[k]), L.lu[l], L.lu[L.nl + l], L.lu[2 * L.nl + l]), tab, cs, sn);
  E[t] = make_double2(cs, sn);
}

// per mode: S2(k) = sum_l E[k][l] Qhat_l[bin(k)] (layers in order), S = S1 + S2 into S, the force
// coefficients (c Im S, c Re S) in FP64 and FP32; thread K: sum_j Q_j Z_j = sum_l Z_l Re Qhat_l[0][0]
__global__ void k_lat_modes(LatDev L, int K, const int4 *__restrict__ modes, const double2 *__restrict__ Qh,
                            const double2 *__restrict__ E, const double *__restrict__ Zl,
                            const double2 *__restrict__ S1, const double *__restrict__ cw, double2 *__restrict__ S,
                            double2 *__restrict__ coef, float2 *__restrict__ coef32, double *__restrict__ scal,
                            int mslot) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > K) return;
  if (k == K) {
    double m = 0.0;
    for (int l = 0; l < L.nl; ++l) m = fma(Zl[l], Qh[(int64_t)l * L.ny * L.nx].x, m);
    scal[mslot] = m;
    return;
  }
  const int4 m = modes[k];
  const int a = pmod(m.x, L.nx), b = pmod(m.y, L.ny);
  double re = 0.0, im = 0.0;
  for (int l = 0; l < L.nl; ++l) {
    const double2 e = E[(int64_t)k * L.nl + l];
    const double2 q = Qh[((int64_t)l * L.ny + b) * L.nx + a];
    re += e.x * q.x - e.y * q.y;
    im += e.x * q.y + e.y * q.x;
  }
  re += S1[k].x;
  im += S1[k].y;
  S[k] = make_double2(re, im);
  const double c = cw[k];
  const double2 v = make_double2(c * im, c * re);
  coef[k] = v;
  coef32[k] = make_float2((float)v.x, (float)v.y);
}

// one warp per bin (a, b): W_l[b][a] = sum over the modes of the bin of (c S1)(k) conj(E[k][l]);
// lanes take the modes in turn, then a fixed butterfly per layer
__global__ void k_lat_bin(LatDev L, int K, const int4 *__restrict__ modes, const double2 *__restrict__ coefS,
                          const double2 *__restrict__ E, double2 *__restrict__ W) {
  const int lane = threadIdx.x & 31;
  const int64_t bin = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (bin >= (int64_t)L.nx * L.ny) return;
  const int a = (int)(bin % L.nx), b = (int)(bin / L.nx);
  double re[kLatMaxLayers], im[kLatMaxLayers];
#pragma unroll
  for (int l = 0; l < kLatMaxLayers; ++l) re[l] = im[l] = 0.0;
#pragma unroll 4
  for (int k = lane; k < K; k += 32) {
    const int4 m = __ldg(&modes[k]);
    if (pmod(m.x, L.nx) != a || pmod(m.y, L.ny) != b) continue;
    const double2 cf = __ldg(&coefS[k]);
#pragma unroll
    for (int l = 0; l < kLatMaxLayers; ++l) {
      if (l >= L.nl) break;
      const double2 e = __ldg(&E[(int64_t)k * L.nl + l]);
      re[l] += cf.x * e.x + cf.y * e.y;        // (x + i y) e^{-i phi}
      im[l] += cf.y * e.x - cf.x * e.y;
    }
  }
#pragma unroll
  for (int l = 0; l < kLatMaxLayers; ++l) {
    if (l >= L.nl) break;
    double x = re[l], y = im[l];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x += __shfl_xor_sync(0xffffffffu, x, o);
      y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    if (lane == 0) W[((int64_t)l * L.ny + b) * L.nx + a] = make_double2(x, y);
  }
}

// twiddle table e^{2 pi i t / n}, t < n, in long double
std::vector<double2> twiddles(int n) {
  std::vector<double2> h(n);
  for (int t = 0; t < n; ++t) {
    const long double a = 2.0L * 3.141592653589793238462643383279502884L * (long double)t / (long double)n;
    h[t] = make_double2((double)cosl(a), (double)sinl(a));
  }
  return h;
}

// site coordinate along one axis on a lattice of n points over the period L, origin o:
// returns the index, or -1 when x is not on the lattice (relative tolerance 1e-9 of the step)
int lattice_index(double x, double o, double L, int n) {
  const double step = L / n;
  double u = (x - o) / step;
  const double r = std::nearbyint(u);
  if (std::fabs(u - r) > 1e-6) return -1;
  long long i = (long long)r % n;
  if (i < 0) i += n;
  return (int)i;
}

}  // namespace

// Recognises a lattice electrode from the host copy of the sites (wrapped into the box): layers of
// equal z, each a full nx x ny rectangular lattice commensurate with Lx, Ly (the same nx, ny in
// every layer, any in-plane origin).  Sets c->lat.nl = 0 when the sites are anything else.
void lattice_setup(srbe_ctx *c, const std::vector<double> &x, const std::vector<double> &y,
                   const std::vector<double> &z) {
  Lattice &L = c->lat;
  L.nl = 0;
  const int64_t ne = (int64_t)x.size();
  std::vector<double> zs(z);
  std::sort(zs.begin(), zs.end());
  std::vector<double> Zl;
  for (double v : zs)
    if (Zl.empty() || v - Zl.back() > 1e-9) Zl.push_back(v);
  const int nl = (int)Zl.size();
  if (nl > kLatMaxLayers || ne % nl) return;
  std::vector<int> layer(ne);
  std::vector<std::vector<int64_t>> members(nl);
  for (int64_t j = 0; j < ne; ++j) {
    const int l = (int)(std::lower_bound(Zl.begin(), Zl.end(), z[j] - 1e-9) - Zl.begin());
    if (l >= nl || std::fabs(z[j] - Zl[l]) > 1e-9) return;
    layer[j] = l;
    members[l].push_back(j);
  }
  // lattice size from the first layer: distinct x and y values
  auto distinct = [](std::vector<double> v, double period) {
    std::sort(v.begin(), v.end());
    int n = 0;
    for (size_t i = 0; i < v.size(); ++i)
      if (i == 0 || v[i] - v[i - 1] > 1e-9 * period) ++n;
    return n;
  };
  std::vector<double> x0v, y0v;
  for (int64_t j : members[0]) {
    x0v.push_back(x[j]);
    y0v.push_back(y[j]);
  }
  const int nx = distinct(x0v, c->L[0]), ny = distinct(y0v, c->L[1]);
  if ((int64_t)nx * ny * nl != ne || nx > kLatMaxN || ny > kLatMaxN) return;
  std::vector<int32_t> site((size_t)ne, -1);
  std::vector<double> ox(nl), oy(nl);
  for (int l = 0; l < nl; ++l) {
    if ((int64_t)members[l].size() != (int64_t)nx * ny) return;
    double mx = 1e300, my = 1e300;
    for (int64_t j : members[l]) {
      mx = std::min(mx, x[j]);
      my = std::min(my, y[j]);
    }
    ox[l] = mx;
    oy[l] = my;
    for (int64_t j : members[l]) {
      const int ix = lattice_index(x[j], mx, c->L[0], nx), iy = lattice_index(y[j], my, c->L[1], ny);
      if (ix < 0 || iy < 0) return;
      int32_t &s = site[((size_t)l * ny + iy) * nx + ix];
      if (s >= 0) return;
      s = (int32_t)j;
    }
  }
  // layer origins in turns (same fixed-point convention as the sites)
  std::vector<uint64_t> lu(3 * (size_t)nl);
  auto turns = [](double v, double period) {
    long double f = (long double)v / (long double)period;
    f -= std::floor((double)f);
    return (uint64_t)(f * 18446744073709551616.0L);
  };
  for (int l = 0; l < nl; ++l) {
    lu[l] = turns(ox[l], c->L[0]);
    lu[nl + l] = turns(oy[l], c->L[1]);
    lu[2 * nl + l] = turns(Zl[l], c->L[2]);
  }
  const auto tx = twiddles(nx), ty = twiddles(ny);
  L.site.ensure(ne);
  L.lu.ensure(lu.size());
  L.twx.ensure(nx);
  L.twy.ensure(ny);
  L.Zl.ensure(nl);
  const size_t cells = (size_t)nl * nx * ny;
  L.T.ensure(cells);
  L.Qh.ensure(cells);
  L.bF.ensure(ne);
  SRBE_CUDA(cudaMemcpyAsync(L.site.p, site.data(), sizeof(int32_t) * ne, cudaMemcpyHostToDevice, c->stream));
  SRBE_CUDA(cudaMemcpyAsync(L.lu.p, lu.data(), sizeof(uint64_t) * lu.size(), cudaMemcpyHostToDevice, c->stream));
  SRBE_CUDA(cudaMemcpyAsync(L.twx.p, tx.data(), sizeof(double2) * nx, cudaMemcpyHostToDevice, c->stream));
  SRBE_CUDA(cudaMemcpyAsync(L.twy.p, ty.data(), sizeof(double2) * ny, cudaMemcpyHostToDevice, c->stream));
  SRBE_CUDA(cudaMemcpyAsync(L.Zl.p, Zl.data(), sizeof(double) * nl, cudaMemcpyHostToDevice, c->stream));
  SRBE_CUDA(cudaStreamSynchronize(c->stream));
  L.nl = nl;
  L.nx = nx;
  L.ny = ny;
}

// b_F of every electrode site into c->lat.bF (coefficients c_k S1(k) from the S1 reduction)
void lattice_bfar(srbe_ctx *c) {
  const LatDev L = lat_dev(c);
  const int64_t cells = (int64_t)L.nl * L.nx * L.ny;
  const int64_t bins = (int64_t)L.nx * L.ny;
  (void)cells;
  double2 *W = c->lat.Qh.p, *U = c->lat.T.p;
  double2 *E = c->lat.E.ensure((size_t)std::max(c->K, 1) * L.nl);
  k_lat_phase<<<blocks_for((int64_t)c->K * L.nl, 128), 128, 0, c->stream>>>(L, c->K, c->dm.p, c->tab.p, E);
  k_lat_bin<<<blocks_for(bins * 32, 128), 128, 0, c->stream>>>(L, c->K, c->dm.p, c->coef.p, E, W);
  launch_line<kInvY>(c, L, W, U);
  launch_line<kInvX>(c, L, U, nullptr);
  c->launches += 2;
  c->mode_evals += (int64_t)c->K * L.nl;
  SRBE_CUDA(cudaGetLastError());
}

// S2 over the electrode and S = S1 + S2 into S (Eq. 15), the force coefficients and sum Q Z;
// reuses the per-step phases E of lattice_bfar (same mode list)
void lattice_s2(srbe_ctx *c, double2 *S, const double2 *S1, int mslot) {
  SRBE_REQUIRE(c->lat.E.p && c->lat.E.cap >= (size_t)c->K * c->lat.nl, SRBE_ESTATE, "lattice phases missing");
  const LatDev L = lat_dev(c);
  const int64_t cells = (int64_t)L.nl * L.nx * L.ny;
  (void)cells;
  launch_line<kFwdX>(c, L, nullptr, c->lat.T.p);
  launch_line<kFwdY>(c, L, c->lat.T.p, c->lat.Qh.p);
  k_lat_modes<<<blocks_for(c->K + 1, 64), 64, 0, c->stream>>>(L, c->K, c->dm.p, c->lat.Qh.p, c->lat.E.p, c->lat.Zl.p,
                                                                S1, c->dc.p, S, c->coef.p, c->coef32.p, c->scal.p,
                                                                mslot);
  c->launches += 1;
  c->mode_evals += (int64_t)c->K * L.nl;
  SRBE_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------------------------------------------
// Spectral form of A for lattice electrodes (an evaluation order of Eqs. 9-10 and 18, exact up to
// rounding).  Every term of A depends on two sites only through their layers and their lattice
// offset (the slab term through the layers alone), so A is block-circulant over (ix, iy) with
// nl x nl blocks: with Yhat = F+ y (the forward transform of the lattice lines) and F- the
// transform back without normalisation, A y = F- (M Yhat) bin by bin, where
//   M(bin) = sum over the modes k of A in the bin of c_k e^{-i (phi_l(k) - phi_l'(k))}
//          + conj(F+ R_l restricted to layer l') / (nx ny),
// R_l being the real-space, self and slab part of the row of A at the origin site of layer l.
// Hence A^-1 rhs = F- (M^-1 F+ rhs) / (nx ny)^2 with one nl x nl inverse per bin: the
// constant-potential solve costs two small transforms per step and no dense matrix.
// ------------------------------------------------------------------------------------------------
namespace {

// R[l][j] = real-space images + self + slab term of A between the origin site of layer l and site j
// (the same terms and cut-offs as the dense build of A)
__global__ void k_lat_real_rows(LatDev L, int64_t ne, const double *__restrict__ ex, const double *__restrict__ ey,
                                const double *__restrict__ ez, double Lx, double Ly, double alpha, double eta,
                                double rcut, int nimx, int nimy, double self, double slab, double *__restrict__ R) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int l = blockIdx.y;
  if (j >= ne) return;
  const int64_t i = L.site[(int64_t)l * L.ny * L.nx];
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
  R[(int64_t)l * ne + j] = acc;
}

// M[bin][l][l'] = conj(Rhat_l[l'][bin]) / (nx ny): the transformed real-space row of origin layer l
__global__ void k_lat_collect_real(LatDev L, int l, const double2 *__restrict__ Rh, double2 *__restrict__ M) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nb = (int64_t)L.nx * L.ny;
  if (t >= nb * L.nl) return;
  const int64_t bin = t % nb;
  const int lp = (int)(t / nb);
  const double2 v = Rh[(int64_t)lp * nb + bin];
  const double inv = 1.0 / (double)nb;
  M[(bin * L.nl + l) * L.nl + lp] = make_double2(v.x * inv, -v.y * inv);
}

// k-space part: thread per (bin, l, l'), the bin's entries (mode of the half lattice, +1 for the
// mode's own bin, -1 for its mirror -k) in list order; half-lattice weights are doubled, so c_k = w / 2
__global__ void k_lat_kspace_M(LatDev L, const int32_t *__restrict__ start, const int2 *__restrict__ ent,
                               const int4 *__restrict__ modes, const double *__restrict__ w,
                               const double2 *__restrict__ tab, double2 *__restrict__ M) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nb = (int64_t)L.nx * L.ny;
  const int nl2 = L.nl * L.nl;
  if (t >= nb * nl2) return;
  const int64_t bin = t / nl2;
  const int l = (int)((t % nl2) / L.nl), lp = (int)(t % L.nl);
  double re = 0.0, im = 0.0;
  for (int e = start[bin]; e < start[bin + 1]; ++e) {
    const int2 en = ent[e];
    const int4 m = modes[en.x];
    // e^{-i s (phi_l - phi_l')} with the phases as exact 64-bit turns
    const uint64_t d = phase64(m, L.lu[l], L.lu[L.nl + l], L.lu[2 * L.nl + l]) -
                       phase64(m, L.lu[lp], L.lu[L.nl + lp], L.lu[2 * L.nl + lp]);
    double cs, sn;
    sincos_turns(d, tab, cs, sn);
    const double c = 0.5 * w[en.x];
    re = fma(c, cs, re);
    im = fma(-c * (double)en.y, sn, im);
  }
  double2 *dst = M + bin * nl2 + l * L.nl + lp;
  *dst = make_double2(dst->x + re, dst->y + im);
}

// per bin: Hermitian part of M, its Cholesky factor, and scale x M^-1 into Minv; a non-positive
// pivot raises flag (A not positive definite)
__global__ void k_lat_invert(LatDev L, const double2 *__restrict__ M, double2 *__restrict__ Minv, double scale,
                             int *__restrict__ flag) {
  const int64_t bin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (bin >= (int64_t)L.nx * L.ny) return;
  const int n = L.nl;
  double2 H[kLatMaxLayers][kLatMaxLayers], X[kLatMaxLayers][kLatMaxLayers];
  const double2 *m = M + bin * n * n;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double2 a = m[i * n + j], b = m[j * n + i];
      H[i][j] = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    }
  // H = C C^H, C lower triangular (overwrites the lower part of H)
  for (int j = 0; j < n; ++j) {
    double dj = H[j][j].x;
    for (int k = 0; k < j; ++k) dj -= H[j][k].x * H[j][k].x + H[j][k].y * H[j][k].y;
    if (!(dj > 0.0)) {
      atomicExch(flag, 1);
      return;
    }
    const double cjj = sqrt(dj);
    H[j][j] = make_double2(cjj, 0.0);
    for (int i = j + 1; i < n; ++i) {
      double re = H[i][j].x, im = H[i][j].y;
      for (int k = 0; k < j; ++k) {   // - C[i][k] conj(C[j][k])
        re -= H[i][k].x * H[j][k].x + H[i][k].y * H[j][k].y;
        im -= H[i][k].y * H[j][k].x - H[i][k].x * H[j][k].y;
      }
      H[i][j] = make_double2(re / cjj, im / cjj);
    }
  }
  // columns of H^-1: solve C z = e_c, then C^H x = z
  for (int c = 0; c < n; ++c) {
    double2 z[kLatMaxLayers];
    for (int i = 0; i < n; ++i) {
      double re = (i == c) ? 1.0 : 0.0, im = 0.0;
      for (int k = 0; k < i; ++k) {
        re -= H[i][k].x * z[k].x - H[i][k].y * z[k].y;
        im -= H[i][k].x * z[k].y + H[i][k].y * z[k].x;
      }
      z[i] = make_double2(re / H[i][i].x, im / H[i][i].x);
    }
    for (int i = n - 1; i >= 0; --i) {
      double re = z[i].x, im = z[i].y;
      for (int k = i + 1; k < n; ++k) {   // - conj(C[k][i]) x[k]
        re -= H[k][i].x * X[k][c].x + H[k][i].y * X[k][c].y;
        im -= H[k][i].x * X[k][c].y - H[k][i].y * X[k][c].x;
      }
      X[i][c] = make_double2(re / H[i][i].x, im / H[i][i].x);
    }
  }
  double2 *o = Minv + bin * n * n;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) o[i * n + j] = make_double2(scale * X[i][j].x, scale * X[i][j].y);
}

// W[l][bin] = sum_l' B[bin][l][l'] Yh[l'][bin] (thread per (bin, l), layers in order)
__global__ void k_lat_binmul(LatDev L, const double2 *__restrict__ B, const double2 *__restrict__ Yh,
                             double2 *__restrict__ W) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nb = (int64_t)L.nx * L.ny;
  if (t >= nb * L.nl) return;
  const int64_t bin = t % nb;
  const int l = (int)(t / nb);
  const double2 *b = B + (bin * L.nl + l) * L.nl;
  double re = 0.0, im = 0.0;
  for (int lp = 0; lp < L.nl; ++lp) {
    const double2 m = b[lp], y = Yh[(int64_t)lp * nb + bin];
    re = fma(m.x, y.x, fma(-m.y, y.y, re));
    im = fma(m.x, y.y, fma(m.y, y.x, im));
  }
  W[(int64_t)l * nb + bin] = make_double2(re, im);
}

__global__ void k_lat_rhs(int64_t ne, double dpsi, const double *__restrict__ d, const double *__restrict__ b,
                          double *__restrict__ r) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < ne) r[j] = fma(dpsi, d[j], b[j]);
}

// one block: psi_bar = -(e^T y) / s (fixed-order sum), Q = y + psi_bar w_e (Eqs. 9-10)
__global__ void __launch_bounds__(1024)
k_lat_finish(int64_t ne, const double *__restrict__ y, const double *__restrict__ we, double s_e,
             double *__restrict__ Q, float *__restrict__ Q32, double *__restrict__ scal) {
  __shared__ double red[1024];
  __shared__ double psi;
  const int t = threadIdx.x;
  double a = 0.0;
  for (int64_t j = t; j < ne; j += 1024) a += y[j];
  red[t] = a;
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if (t < s) red[t] += red[t + s];
    __syncthreads();
  }
  if (t == 0) {
    psi = -red[0] / s_e;
    scal[kScalPsi] = psi;
  }
  __syncthreads();
  const double p = psi;
  for (int64_t j = t; j < ne; j += 1024) {
    const double q = fma(p, we[j], y[j]);
    Q[j] = q;
    Q32[j] = (float)q;
  }
}

// y = F- (B F+ x), B = Minv (solve) or M (apply)
void spectral_apply(srbe_ctx *c, const double2 *B, const double *x, double *y) {
  const LatDev L = lat_dev(c);
  const int64_t cells = (int64_t)L.nl * L.nx * L.ny;
  launch_line<kFwdX>(c, L, nullptr, c->lat.T.p, x);
  launch_line<kFwdY>(c, L, c->lat.T.p, c->lat.Qh.p);
  k_lat_binmul<<<blocks_for(cells, 256), 256, 0, c->stream>>>(L, B, c->lat.Qh.p, c->lat.T.p);
  launch_line<kInvY>(c, L, c->lat.T.p, c->lat.Qh.p);
  launch_line<kInvXp>(c, L, c->lat.Qh.p, nullptr, nullptr, y);
  c->launches++;
  SRBE_CUDA(cudaGetLastError());
}

}  // namespace

void lattice_spectral_setup(srbe_ctx *c, const std::vector<int4> &modesA, const std::vector<double> &wA,
                            double alpha_A, double rcut, int nimx, int nimy, double self, double slab) {
  Lattice &Lt = c->lat;
  Lt.spectral = false;
  if (Lt.nl == 0) return;
  const LatDev L = lat_dev(c);
  const int64_t ne = c->ne, nb = (int64_t)L.nx * L.ny, nl = L.nl;
  double2 *M = Lt.M.ensure((size_t)nb * nl * nl);
  double2 *Minv = Lt.Minv.ensure((size_t)nb * nl * nl);
  double *R = Lt.Rrow.ensure((size_t)nl * ne);
  Lt.R.ensure(ne);
  Lt.Y.ensure(ne);
  // real-space rows at the layer origins, transformed layer by layer
  k_lat_real_rows<<<dim3(blocks_for(ne, 128), (unsigned)nl), 128, 0, c->stream>>>(
      L, ne, c->ex.p, c->ey.p, c->ez.p, c->L[0], c->L[1], alpha_A, c->eta, rcut, nimx, nimy, self, slab, R);
  c->launches++;
  for (int l = 0; l < nl; ++l) {
    launch_line<kFwdX>(c, L, nullptr, Lt.T.p, R + (size_t)l * ne);
    launch_line<kFwdY>(c, L, Lt.T.p, Lt.Qh.p);
    k_lat_collect_real<<<blocks_for(nb * nl, 256), 256, 0, c->stream>>>(L, l, Lt.Qh.p, M);
    c->launches++;
  }
  // k-space part: the half-lattice modes of A binned by (m_x mod nx, m_y mod ny), each also into
  // its mirror's bin; entries kept in mode order
  const int64_t KA = (int64_t)modesA.size();
  std::vector<int32_t> start(nb + 1, 0);
  auto pm = [](int a, int n) { return ((a % n) + n) % n; };
  auto bin_of = [&](int mx, int my) { return (int64_t)pm(my, L.ny) * L.nx + pm(mx, L.nx); };
  for (int64_t t = 0; t < KA; ++t) {
    start[bin_of(modesA[t].x, modesA[t].y) + 1]++;
    start[bin_of(-modesA[t].x, -modesA[t].y) + 1]++;
  }
  for (int64_t b = 0; b < nb; ++b) start[b + 1] += start[b];
  std::vector<int2> ent((size_t)2 * KA);
  std::vector<int32_t> fill(start.begin(), start.end() - 1);
  for (int64_t t = 0; t < KA; ++t) {
    ent[fill[bin_of(modesA[t].x, modesA[t].y)]++] = make_int2((int)t, 1);
    ent[fill[bin_of(-modesA[t].x, -modesA[t].y)]++] = make_int2((int)t, -1);
  }
  DevBuf<int32_t> dstart;
  DevBuf<int2> dent;
  DevBuf<int4> dmodes;
  DevBuf<double> dw;
  dstart.ensure(nb + 1);
  dent.ensure(std::max<int64_t>(2 * KA, 1));
  dmodes.ensure(std::max<int64_t>(KA, 1));
  dw.ensure(std::max<int64_t>(KA, 1));
  SRBE_CUDA(cudaMemcpyAsync(dstart.p, start.data(), sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice, c->stream));
  if (KA > 0) {
    SRBE_CUDA(cudaMemcpyAsync(dent.p, ent.data(), sizeof(int2) * 2 * KA, cudaMemcpyHostToDevice, c->stream));
    SRBE_CUDA(cudaMemcpyAsync(dmodes.p, modesA.data(), sizeof(int4) * KA, cudaMemcpyHostToDevice, c->stream));
    SRBE_CUDA(cudaMemcpyAsync(dw.p, wA.data(), sizeof(double) * KA, cudaMemcpyHostToDevice, c->stream));
  }
  k_lat_kspace_M<<<blocks_for(nb * nl * nl, 128), 128, 0, c->stream>>>(L, dstart.p, dent.p, dmodes.p, dw.p,
                                                                       c->tab.p, M);
  int *flag = c->flag.ensure(1);
  SRBE_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
  k_lat_invert<<<blocks_for(nb, 64), 64, 0, c->stream>>>(L, M, Minv, 1.0 / ((double)nb * (double)nb), flag);
  c->launches += 2;
  SRBE_CUDA(cudaGetLastError());
  int hflag = 0;
  SRBE_CUDA(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  SRBE_CUDA(cudaStreamSynchronize(c->stream));
  SRBE_REQUIRE(hflag == 0, SRBE_ENOTCONV, "A is not positive definite (a lattice block has a non-positive pivot)");
  Lt.spectral = true;
}

void lattice_solve(srbe_ctx *c, const double *rhs, double *y) {
  SRBE_REQUIRE(c->lat.spectral, SRBE_ESTATE, "no spectral form of A");
  spectral_apply(c, c->lat.Minv.p, rhs, y);
}

void lattice_apply_A(srbe_ctx *c, const double *x, double *y) {
  SRBE_REQUIRE(c->lat.spectral, SRBE_ESTATE, "no spectral form of A");
  spectral_apply(c, c->lat.M.p, x, y);
}

// per step: y = A^-1 (dpsi d + b), then psi_bar and Q (Eqs. 9-10)
void charge_update_lattice(srbe_ctx *c) {
  const int64_t ne = c->ne;
  k_lat_rhs<<<blocks_for(ne, 256), 256, 0, c->stream>>>(ne, c->dpsi, c->ed.p, c->bvec.p, c->lat.R.p);
  c->launches++;
  lattice_solve(c, c->lat.R.p, c->lat.Y.p);
  k_lat_finish<<<1, 1024, 0, c->stream>>>(ne, c->lat.Y.p, c->we.p, c->s_e, c->Q.p, c->Q32.p, c->scal.p);
  c->launches++;
  SRBE_CUDA(cudaGetLastError());
}

}  // namespace srbe
