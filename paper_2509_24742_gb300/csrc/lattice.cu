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
enum { kFwdX = 0, kFwdY = 1, kInvY = 2, kInvX = 3 };
constexpr int kLineWarps = 2;

template <int MODE>
__global__ void __launch_bounds__(32 * kLineWarps)
k_lat_line(LatDev L, const double *__restrict__ Q, const double2 *__restrict__ in, double2 *__restrict__ out,
           double *__restrict__ bF) {
  extern __shared__ double2 sm[];
  constexpr bool along_x = (MODE == kFwdX || MODE == kInvX);
  constexpr bool conj = (MODE == kInvY || MODE == kInvX);
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
      } else if (MODE == kInvX) {
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
    } else {
      const int64_t l = line / L.nx, a = line % L.nx;
      out[(l * L.ny + s) * L.nx + a] = make_double2(re, im);
    }
  }
}

template <int MODE>
void launch_line(srbe_ctx *c, const LatDev &L, const double2 *in, double2 *out) {
  constexpr bool along_x = (MODE == kFwdX || MODE == kInvX);
  const int n = along_x ? L.nx : L.ny;
  const int64_t lines = along_x ? (int64_t)L.nl * L.ny : (int64_t)L.nl * L.nx;
  const size_t smem = sizeof(double2) * (size_t)n * (1 + kLineWarps);
  k_lat_line<MODE><<<blocks_for(lines, kLineWarps), 32 * kLineWarps, smem, c->stream>>>(L, c->Q.p, in, out,
                                                                                        c->lat.bF.p);
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
  c->launches += 4;
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
  c->launches += 3;
  c->mode_evals += (int64_t)c->K * L.nl;
  SRBE_CUDA(cudaGetLastError());
}

}  // namespace srbe
