// Near-field part of SRBE and the per-particle gathers:
//  * cell lists (2D-periodic bins in x, y; open bins in z; deterministic order inside a cell);
//  * the electrode right-hand side b_j = b_F,j + b_N,j + b_slab,j (Eq. 24 far part, Eq. 19
//    near part within rc over every in-plane image, slab part -(4 pi / V) Z_j sum_i q_i z_i);
//  * the ion force: SRBE k-space gather (Eq. 25), slab force -(4 pi / V) q_i M_z, real-space
//    Coulomb of Eq. 13 (ion-ion erfc(alpha r)/r, ion-electrode [erfc(alpha r) - erfc(r/eta)]/r),
//    and the MD support terms (LJ 12-6, harmonic bonds);
//  * the velocity-Verlet kick/drift.
// One thread per particle; stencil cells are visited in a fixed order and cells are sorted by
// particle index, so every sum has a fixed order and results are bitwise reproducible.
#include "srbe_internal.cuh"

namespace srbe {

constexpr double kKe = 138.935458;            // kJ mol^-1 nm e^-2
constexpr double kTwoOverSqrtPi = 1.1283791670955126;
constexpr int kGatherThreads = 128;
constexpr int kModeTile = 256;

struct GridDev {
  int nc[3];
  int span[3];
  double cs[3];
  double inv[3];
  double z0;
};

static GridDev to_dev(const CellGrid &g) {
  GridDev d;
  for (int i = 0; i < 3; ++i) {
    d.nc[i] = g.nc[i];
    d.span[i] = g.span[i];
    d.cs[i] = g.cs[i];
    d.inv[i] = 1.0 / g.cs[i];
  }
  d.z0 = g.z0;
  return d;
}

void choose_grid(const srbe_ctx *c, CellGrid &g, double zlo, double zhi) {
  const double target = 0.5 * c->rc;
  for (int d = 0; d < 2; ++d) {
    g.nc[d] = std::max(1, (int)std::floor(c->L[d] / target));
    g.cs[d] = c->L[d] / g.nc[d];
    g.span[d] = (int)std::ceil(c->rc / g.cs[d] - 1e-12);
  }
  const double h = std::max(zhi - zlo, 1e-9);
  g.nc[2] = std::max(1, (int)std::floor(h / target));
  g.cs[2] = h / g.nc[2];
  g.span[2] = (int)std::ceil(c->rc / g.cs[2] - 1e-12);
  g.z0 = zlo;
}

__device__ __forceinline__ int cell_coord(double v, double inv, int n) {
  int ci = (int)floor(v * inv);
  return min(max(ci, 0), n - 1);
}

__global__ void k_cell_count(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                             const double *__restrict__ z, GridDev g, int32_t *__restrict__ cell,
                             int32_t *__restrict__ rank, int32_t *__restrict__ count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int cx = cell_coord(x[i], g.inv[0], g.nc[0]);
  const int cy = cell_coord(y[i], g.inv[1], g.nc[1]);
  const int cz = cell_coord(z[i] - g.z0, g.inv[2], g.nc[2]);
  const int c = (cz * g.nc[1] + cy) * g.nc[0] + cx;
  cell[i] = c;
  rank[i] = atomicAdd(&count[c], 1);
}

// exclusive scan of count[0..ncell) into start[0..ncell], one block of 1024 threads
__global__ void k_scan(int ncell, int32_t *__restrict__ start) {
  __shared__ int32_t part[1024];
  const int t = threadIdx.x;
  const int per = (ncell + 1023) / 1024;
  const int b = t * per, e = min(ncell, b + per);
  int32_t s = 0;
  for (int i = b; i < e; ++i) s += start[i];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int32_t v = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int32_t run = part[t] - s;  // exclusive prefix of this segment
  for (int i = b; i < e; ++i) {
    int32_t v = start[i];
    start[i] = run;
    run += v;
  }
  if (t == 1023) start[ncell] = part[1023];
}

__global__ void k_scatter(int64_t n, const int32_t *__restrict__ cell, const int32_t *__restrict__ rank,
                          const int32_t *__restrict__ start, int32_t *__restrict__ order) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) order[start[cell[i]] + rank[i]] = (int32_t)i;
}

// insertion sort of each cell's entries by particle index (cells hold tens of particles)
__global__ void k_sort_cells(int ncell, const int32_t *__restrict__ start, int32_t *__restrict__ order) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const int b = start[c], e = start[c + 1];
  for (int i = b + 1; i < e; ++i) {
    int32_t v = order[i];
    int j = i - 1;
    while (j >= b && order[j] > v) {
      order[j + 1] = order[j];
      --j;
    }
    order[j + 1] = v;
  }
}

__global__ void k_gather_sorted(int64_t n, const int32_t *__restrict__ order, const double *__restrict__ x,
                                const double *__restrict__ y, const double *__restrict__ z,
                                const double *__restrict__ w, const int32_t *__restrict__ typ,
                                const int32_t *__restrict__ mol, double *__restrict__ xs, double *__restrict__ ys,
                                double *__restrict__ zs, double *__restrict__ ws, int32_t *__restrict__ ts,
                                int32_t *__restrict__ ms, float *__restrict__ xf, float *__restrict__ yf,
                                float *__restrict__ zf) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int32_t i = order[p];
  xs[p] = x[i];
  ys[p] = y[i];
  zs[p] = z[i];
  xf[p] = (float)x[i];
  yf[p] = (float)y[i];
  zf[p] = (float)z[i];
  if (w) ws[p] = w[i];
  if (typ) ts[p] = typ[i];
  if (mol) ms[p] = mol[i];
}

void build_cells(srbe_ctx *c, Cells &cl, int64_t n, const double *x, const double *y, const double *z,
                 const double *w, const int32_t *typ, const int32_t *mol, bool) {
  const int ncell = cl.g.ncell();
  const size_t nn = (size_t)std::max<int64_t>(n, 1);
  cl.cell.ensure(nn);
  cl.rank.ensure(nn);
  cl.order.ensure(nn);
  cl.start.ensure((size_t)ncell + 1);
  cl.xs.ensure(nn);
  cl.ys.ensure(nn);
  cl.zs.ensure(nn);
  cl.ws.ensure(nn);
  cl.ts.ensure(nn);
  cl.ms.ensure(nn);
  cl.xf.ensure(nn);
  cl.yf.ensure(nn);
  cl.zf.ensure(nn);
  SRBE_CUDA(cudaMemsetAsync(cl.start.p, 0, sizeof(int32_t) * ((size_t)ncell + 1), c->stream));
  const GridDev g = to_dev(cl.g);
  if (n > 0) {
    k_cell_count<<<blocks_for(n, 256), 256, 0, c->stream>>>(n, x, y, z, g, cl.cell.p, cl.rank.p, cl.start.p);
    c->launches++;
  }
  k_scan<<<1, 1024, 0, c->stream>>>(ncell, cl.start.p);
  c->launches++;
  if (n > 0) {
    k_scatter<<<blocks_for(n, 256), 256, 0, c->stream>>>(n, cl.cell.p, cl.rank.p, cl.start.p, cl.order.p);
    k_sort_cells<<<blocks_for(ncell, 128), 128, 0, c->stream>>>(ncell, cl.start.p, cl.order.p);
    k_gather_sorted<<<blocks_for(n, 256), 256, 0, c->stream>>>(n, cl.order.p, x, y, z, w, typ, mol, cl.xs.p, cl.ys.p,
                                                              cl.zs.p, cl.ws.p, cl.ts.p, cl.ms.p, cl.xf.p, cl.yf.p,
                                                              cl.zf.p);
    c->launches += 3;
  }
  SRBE_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------------------------------------------
// pair kernels of Eq. 13 (Gaussian units).  mdphi_over_r = -phi'(r) / r so that the force on the
// first particle is q_a q_b mdphi_over_r * (r_a - r_b).
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void pair_ii(double r2, double alpha, double &phi, double &mdphi_r) {
  const double r = sqrt(r2);
  const double ec = erfc(alpha * r);
  const double ex = exp(-alpha * alpha * r2);
  phi = ec / r;
  mdphi_r = (phi + kTwoOverSqrtPi * alpha * ex) / r2;
}

__device__ __forceinline__ void pair_ie(double r2, double alpha, double eta, double &phi, double &mdphi_r) {
  const double r = sqrt(r2);
  const double ec = erfc(alpha * r);
  const double ex = exp(-alpha * alpha * r2);
  double p = ec / r, f = p + kTwoOverSqrtPi * alpha * ex;
  if (r < 6.5 * eta) {  // erfc(6.5) < 1e-19: the Gaussian term vanishes beyond
    const double eg = erfc(r / eta);
    const double exg = exp(-r2 / (eta * eta));
    p -= eg / r;
    f -= eg / r + kTwoOverSqrtPi / eta * exg;
  }
  phi = p;
  mdphi_r = f / r2;
}

__device__ __forceinline__ void pair_ii_f(float r2, float alpha, float &phi, float &mdphi_r) {
  const float r = sqrtf(r2);
  const float ec = erfcf(alpha * r);
  const float ex = __expf(-alpha * alpha * r2);
  phi = ec / r;
  mdphi_r = (phi + (float)kTwoOverSqrtPi * alpha * ex) / r2;
}

__device__ __forceinline__ void pair_ie_f(float r2, float alpha, float eta, float &phi, float &mdphi_r) {
  const float r = sqrtf(r2);
  const float ec = erfcf(alpha * r);
  const float ex = __expf(-alpha * alpha * r2);
  float p = ec / r, f = p + (float)kTwoOverSqrtPi * alpha * ex;
  if (r < 4.5f * eta) {
    const float eg = erfcf(r / eta);
    const float exg = __expf(-r2 / (eta * eta));
    p -= eg / r;
    f -= eg / r + (float)kTwoOverSqrtPi / eta * exg;
  }
  phi = p;
  mdphi_r = f / r2;
}

struct CellsDev {
  GridDev g;
  const int32_t *start, *order;
  const double *xs, *ys, *zs, *ws;
  const int32_t *ts, *ms;
  const float *xf, *yf, *zf;
};

static CellsDev cells_dev(const Cells &cl) {
  CellsDev d;
  d.g = to_dev(cl.g);
  d.start = cl.start.p;
  d.order = cl.order.p;
  d.xs = cl.xs.p;
  d.ys = cl.ys.p;
  d.zs = cl.zs.p;
  d.ws = cl.ws.p;
  d.ts = cl.ts.p;
  d.ms = cl.ms.p;
  d.xf = cl.xf.p;
  d.yf = cl.yf.p;
  d.zf = cl.zf.p;
  return d;
}

// Visits every (neighbour, image) within the stencil of a point: fn(p, sx, sy, ix, iy) with p the
// sorted index, (sx, sy) the image shift to add to the neighbour and (ix, iy) the image index.
template <class Fn>
__device__ __forceinline__ void for_stencil(const CellsDev &C, double x, double y, double z, double Lx, double Ly,
                                            Fn &&fn) {
  const GridDev &g = C.g;
  const int cx = cell_coord(x, g.inv[0], g.nc[0]);
  const int cy = cell_coord(y, g.inv[1], g.nc[1]);
  const int cz = cell_coord(z - g.z0, g.inv[2], g.nc[2]);
  const int z_lo = max(0, cz - g.span[2]), z_hi = min(g.nc[2] - 1, cz + g.span[2]);
  for (int dz = z_lo; dz <= z_hi; ++dz) {
    for (int oy = -g.span[1]; oy <= g.span[1]; ++oy) {
      const int yy = cy + oy;
      const int iy = (yy >= 0) ? yy / g.nc[1] : -((-yy + g.nc[1] - 1) / g.nc[1]);
      const int ccy = yy - iy * g.nc[1];
      for (int ox = -g.span[0]; ox <= g.span[0]; ++ox) {
        const int xx = cx + ox;
        const int ix = (xx >= 0) ? xx / g.nc[0] : -((-xx + g.nc[0] - 1) / g.nc[0]);
        const int ccx = xx - ix * g.nc[0];
        const int cell = (dz * g.nc[1] + ccy) * g.nc[0] + ccx;
        const int b = C.start[cell], e = C.start[cell + 1];
        for (int p = b; p < e; ++p) fn(p, ix * Lx, iy * Ly, ix, iy);
      }
    }
  }
}

// ------------------------------------------------------------------------------------------------
// electrode right-hand side
// ------------------------------------------------------------------------------------------------
// coefS[k] = (c_k Re S1(k), c_k Im S1(k));  b_F,j = - sum_k Re(exp(-i k.R_j) c_k S1) (Eq. 24)
template <bool F32>
__global__ void __launch_bounds__(kGatherThreads)
k_electrode_rhs(int64_t ne, const double *__restrict__ ex, const double *__restrict__ ey,
                const double *__restrict__ ez, int K, const int4 *__restrict__ modes,
                const double2 *__restrict__ coefS, const double2 *__restrict__ gtab, double3 invL, CellsDev ions,
                double Lx, double Ly, double alpha, double eta, double rc, double slab, const double *__restrict__ scal,
                double *__restrict__ b) {
  __shared__ double2 tab[F32 ? 1 : kTab];
  __shared__ int4 sm[kModeTile];
  __shared__ double2 sc[kModeTile];
  const int t = threadIdx.x;
  if (!F32)
    for (int i = t; i < kTab; i += kGatherThreads) tab[i] = gtab[i];
  const int64_t j = (int64_t)blockIdx.x * kGatherThreads + t;
  const bool live = j < ne;
  double X = 0, Y = 0, Z = 0;
  uint64_t ux = 0, uy = 0, uz = 0;
  if (live) {
    X = ex[j];
    Y = ey[j];
    Z = ez[j];
    ux = to_turns64(X, invL.x);
    uy = to_turns64(Y, invL.y);
    uz = to_turns64(Z, invL.z);
  }
  double acc = 0.0;
  float facc = 0.f, fcmp = 0.f;
  for (int k0 = 0; k0 < K; k0 += kModeTile) {
    __syncthreads();
    for (int k = t; k < kModeTile && k0 + k < K; k += kGatherThreads) {
      sm[k] = modes[k0 + k];
      sc[k] = coefS[k0 + k];
    }
    __syncthreads();
    const int cnt = min(kModeTile, K - k0);
    if (live) {
      if (!F32) {
        for (int k = 0; k < cnt; ++k) {
          double cs, sn;
          sincos_turns(phase64(sm[k], ux, uy, uz), tab, cs, sn);
          acc = fma(-sc[k].x, cs, acc);
          acc = fma(-sc[k].y, sn, acc);
        }
      } else {
        const uint32_t vx = (uint32_t)(ux >> 32), vy = (uint32_t)(uy >> 32), vz = (uint32_t)(uz >> 32);
        for (int k = 0; k < cnt; ++k) {
          const int4 m = sm[k];
          float cs, sn;
          sincos_turns32((uint32_t)m.x * vx + (uint32_t)m.y * vy + (uint32_t)m.z * vz, cs, sn);
          const float term = -(float)sc[k].x * cs - (float)sc[k].y * sn;
          const float yv = term - fcmp, tv = facc + yv;
          fcmp = (tv - facc) - yv;
          facc = tv;
        }
      }
    }
  }
  if (F32) acc = (double)facc - (double)fcmp;
  if (!live) return;
  // near part of Eq. 19: - sum_i q_i [erfc(alpha d) - erfc(d/eta)] / d over images within rc
  const double rc2 = rc * rc;
  if (!F32) {
    double near = 0.0;
    for_stencil(ions, X, Y, Z, Lx, Ly, [&](int p, double sx, double sy, int, int) {
      const double dx = X - (ions.xs[p] + sx), dy = Y - (ions.ys[p] + sy), dz = Z - ions.zs[p];
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < rc2 && r2 > 0.0) {
        double phi, md;
        pair_ie(r2, alpha, eta, phi, md);
        near = fma(-ions.ws[p], phi, near);
      }
    });
    acc += near;
  } else {
    const float Xf = (float)X, Yf = (float)Y, Zf = (float)Z, rc2f = (float)rc2;
    float ns = 0.f, nc = 0.f;
    for_stencil(ions, X, Y, Z, Lx, Ly, [&](int p, double sx, double sy, int, int) {
      const float dx = Xf - (ions.xf[p] + (float)sx), dy = Yf - (ions.yf[p] + (float)sy), dz = Zf - ions.zf[p];
      const float r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < rc2f && r2 > 0.f) {
        float phi, md;
        pair_ie_f(r2, (float)alpha, (float)eta, phi, md);
        const float yv = -(float)ions.ws[p] * phi - nc, tv = ns + yv;
        nc = (tv - ns) - yv;
        ns = tv;
      }
    });
    acc += (double)ns - (double)nc;
  }
  // slab part (FP64 in every form): -(4 pi / V) Z_j sum_i q_i z_i
  acc = fma(-slab * Z, scal[kScalMion], acc);
  b[j] = acc;
}

__global__ void k_coef(int K, const double *__restrict__ c, const double2 *__restrict__ S, double2 *__restrict__ out,
                       int swap) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < K) {
    const double2 s = S[k];
    out[k] = swap ? make_double2(c[k] * s.y, c[k] * s.x) : make_double2(c[k] * s.x, c[k] * s.y);
  }
}

void electrode_rhs(srbe_ctx *c) {
  const int K = c->K;
  double2 *coef = c->coef.p;
  if (K > 0) {
    k_coef<<<blocks_for(K, 128), 128, 0, c->stream>>>(K, c->dc.p, c->S1.p, coef, 0);
    c->launches++;
  }
  const double3 invL = make_double3(1.0 / c->L[0], 1.0 / c->L[1], 1.0 / c->L[2]);
  const double slab = 4.0 * kPi / c->V;
  const CellsDev ions = cells_dev(c->icells);
  if (c->precision == SRBE_MIXED)
    k_electrode_rhs<true><<<blocks_for(c->ne, kGatherThreads), kGatherThreads, 0, c->stream>>>(
        c->ne, c->ex.p, c->ey.p, c->ez.p, K, c->dm.p, coef, c->tab.p, invL, ions, c->L[0], c->L[1], c->alpha,
        c->eta, c->rc, slab, c->scal.p, c->bvec.p);
  else
    k_electrode_rhs<false><<<blocks_for(c->ne, kGatherThreads), kGatherThreads, 0, c->stream>>>(
        c->ne, c->ex.p, c->ey.p, c->ez.p, K, c->dm.p, coef, c->tab.p, invL, ions, c->L[0], c->L[1], c->alpha,
        c->eta, c->rc, slab, c->scal.p, c->bvec.p);
  c->launches++;
  c->mode_evals += c->ne * (int64_t)K;
  SRBE_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------------------------------------------
// ion forces
// ------------------------------------------------------------------------------------------------
struct MdDev {
  int ntype;                        // 0 = no LJ / bonds
  const double2 *lj;                // (sigma^2, eps) per type pair
  const int32_t *bond_start, *bond_j;
  const double *bond_r0;
  double kb;
};

// coefF[k] = (c_k Im S(k), c_k Re S(k)) with S = S1 + S2;
// F_i = - q_i sum_k c_k k Im(S exp(-i k . r_i)) = - q_i sum_k k (cIm cos - cRe sin)   (Eq. 25)
template <bool F32>
__global__ void __launch_bounds__(kGatherThreads)
k_ion_forces(int64_t ni, CellsDev ions, CellsDev eles, const double *__restrict__ Q, int K,
             const int4 *__restrict__ modes, const double2 *__restrict__ coefF, const double2 *__restrict__ gtab,
             double3 invL, double Lx, double Ly, double alpha, double eta, double rc, double slab,
             const double *__restrict__ scal, MdDev md, const double *__restrict__ x_orig,
             const double *__restrict__ y_orig, const double *__restrict__ z_orig, double *__restrict__ F,
             double *__restrict__ epart) {
  __shared__ double2 tab[F32 ? 1 : kTab];
  __shared__ int4 sm[kModeTile];
  __shared__ double2 sc[kModeTile];
  __shared__ double red[4][kGatherThreads];
  const int t = threadIdx.x;
  if (!F32)
    for (int i = t; i < kTab; i += kGatherThreads) tab[i] = gtab[i];
  const int64_t p = (int64_t)blockIdx.x * kGatherThreads + t;
  const bool live = p < ni;
  int32_t i = 0;
  double X = 0, Y = 0, Z = 0, qi = 0;
  int ti = 0, mi = -1;
  uint64_t ux = 0, uy = 0, uz = 0;
  if (live) {
    i = ions.order[p];
    X = ions.xs[p];
    Y = ions.ys[p];
    Z = ions.zs[p];
    qi = ions.ws[p];
    ti = ions.ts ? ions.ts[p] : 0;
    mi = ions.ms ? ions.ms[p] : -1;
    ux = to_turns64(X, invL.x);
    uy = to_turns64(Y, invL.y);
    uz = to_turns64(Z, invL.z);
  }
  // ---- k-space gather
  double fk[3] = {0, 0, 0};
  float ff[3] = {0, 0, 0}, fc[3] = {0, 0, 0};
  const double tpx = 2.0 * kPi * invL.x, tpy = 2.0 * kPi * invL.y, tpz = 2.0 * kPi * invL.z;
  for (int k0 = 0; k0 < K; k0 += kModeTile) {
    __syncthreads();
    for (int k = t; k < kModeTile && k0 + k < K; k += kGatherThreads) {
      sm[k] = modes[k0 + k];
      sc[k] = coefF[k0 + k];
    }
    __syncthreads();
    const int cnt = min(kModeTile, K - k0);
    if (live) {
      if (!F32) {
        for (int k = 0; k < cnt; ++k) {
          const int4 m = sm[k];
          double cs, sn;
          sincos_turns(phase64(m, ux, uy, uz), tab, cs, sn);
          const double im = fma(sc[k].x, cs, -sc[k].y * sn);
          fk[0] = fma(tpx * m.x, im, fk[0]);
          fk[1] = fma(tpy * m.y, im, fk[1]);
          fk[2] = fma(tpz * m.z, im, fk[2]);
        }
      } else {
        const uint32_t vx = (uint32_t)(ux >> 32), vy = (uint32_t)(uy >> 32), vz = (uint32_t)(uz >> 32);
        const float kx = (float)tpx, ky = (float)tpy, kz = (float)tpz;
        for (int k = 0; k < cnt; ++k) {
          const int4 m = sm[k];
          float cs, sn;
          sincos_turns32((uint32_t)m.x * vx + (uint32_t)m.y * vy + (uint32_t)m.z * vz, cs, sn);
          const float im = (float)sc[k].x * cs - (float)sc[k].y * sn;
          const float v[3] = {kx * (float)m.x * im, ky * (float)m.y * im, kz * (float)m.z * im};
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const float yv = v[d] - fc[d], tv = ff[d] + yv;
            fc[d] = (tv - ff[d]) - yv;
            ff[d] = tv;
          }
        }
      }
    }
  }
  if (!live) {
    // keep the block-wide reduction below well formed
    for (int e = 0; e < 4; ++e) red[e][t] = 0.0;
  }
  double e_ii = 0, e_ie = 0, e_lj = 0, e_b = 0;
  if (live) {
    if (F32)
      for (int d = 0; d < 3; ++d) fk[d] = (double)ff[d] - (double)fc[d];
    double Fx = -qi * fk[0], Fy = -qi * fk[1], Fz = -qi * fk[2];
    // slab force, FP64 in every form: M_z = sum q_i z_i + sum Q_j Z_j
    Fz = fma(-slab * qi, scal[kScalMion] + scal[kScalMele], Fz);
    // ---- real space
    const double rc2 = rc * rc;
    double rx = 0, ry = 0, rz = 0;      // Coulomb (Gaussian units)
    double lx = 0, ly = 0, lz = 0;      // LJ (kJ/mol/nm)
    if (!F32) {
      for_stencil(ions, X, Y, Z, Lx, Ly, [&](int pp, double sx, double sy, int ix, int iy) {
        if (pp == p && ix == 0 && iy == 0) return;
        const double dx = X - (ions.xs[pp] + sx), dy = Y - (ions.ys[pp] + sy), dz = Z - ions.zs[pp];
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= rc2) return;
        double phi, md2;
        pair_ii(r2, alpha, phi, md2);
        const double s = qi * ions.ws[pp] * md2;
        rx = fma(s, dx, rx);
        ry = fma(s, dy, ry);
        rz = fma(s, dz, rz);
        e_ii = fma(0.5 * qi * ions.ws[pp], phi, e_ii);
        if (md.ntype && ions.ms[pp] != mi) {
          const double2 sg = md.lj[ti * md.ntype + ions.ts[pp]];
          const double sr2 = sg.x / r2, sr6 = sr2 * sr2 * sr2;
          const double fs = 24.0 * sg.y * (2.0 * sr6 * sr6 - sr6) / r2;
          lx = fma(fs, dx, lx);
          ly = fma(fs, dy, ly);
          lz = fma(fs, dz, lz);
          e_lj += 0.5 * 4.0 * sg.y * (sr6 * sr6 - sr6);
        }
      });
      for_stencil(eles, X, Y, Z, Lx, Ly, [&](int pe, double sx, double sy, int, int) {
        const double dx = X - (eles.xs[pe] + sx), dy = Y - (eles.ys[pe] + sy), dz = Z - eles.zs[pe];
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= rc2 || r2 == 0.0) return;
        const double Qj = Q[eles.order[pe]];
        double phi, md2;
        pair_ie(r2, alpha, eta, phi, md2);
        const double s = qi * Qj * md2;
        rx = fma(s, dx, rx);
        ry = fma(s, dy, ry);
        rz = fma(s, dz, rz);
        e_ie = fma(qi * Qj, phi, e_ie);
        if (md.ntype) {
          const double2 sg = md.lj[ti * md.ntype + (md.ntype - 1)];
          const double sr2 = sg.x / r2, sr6 = sr2 * sr2 * sr2;
          const double fs = 24.0 * sg.y * (2.0 * sr6 * sr6 - sr6) / r2;
          lx = fma(fs, dx, lx);
          ly = fma(fs, dy, ly);
          lz = fma(fs, dz, lz);
          e_lj += 4.0 * sg.y * (sr6 * sr6 - sr6);
        }
      });
    } else {
      const float Xf = (float)X, Yf = (float)Y, Zf = (float)Z, rc2f = (float)rc2;
      const float af = (float)alpha, etaf = (float)eta, qf = (float)qi;
      float a[6] = {0, 0, 0, 0, 0, 0}, cmp[6] = {0, 0, 0, 0, 0, 0};
      auto kadd = [&](int d, float v) {
        const float yv = v - cmp[d], tv = a[d] + yv;
        cmp[d] = (tv - a[d]) - yv;
        a[d] = tv;
      };
      float eii = 0.f, eie = 0.f, elj = 0.f;
      for_stencil(ions, X, Y, Z, Lx, Ly, [&](int pp, double sx, double sy, int ix, int iy) {
        if (pp == p && ix == 0 && iy == 0) return;
        const float dx = Xf - (ions.xf[pp] + (float)sx), dy = Yf - (ions.yf[pp] + (float)sy), dz = Zf - ions.zf[pp];
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= rc2f) return;
        float phi, md2;
        pair_ii_f(r2, af, phi, md2);
        const float qq = qf * (float)ions.ws[pp];
        const float s = qq * md2;
        kadd(0, s * dx);
        kadd(1, s * dy);
        kadd(2, s * dz);
        eii += 0.5f * qq * phi;
        if (md.ntype && ions.ms[pp] != mi) {
          const double2 sg = md.lj[ti * md.ntype + ions.ts[pp]];
          const float sr2 = (float)sg.x / r2, sr6 = sr2 * sr2 * sr2;
          const float fs = 24.f * (float)sg.y * (2.f * sr6 * sr6 - sr6) / r2;
          kadd(3, fs * dx);
          kadd(4, fs * dy);
          kadd(5, fs * dz);
          elj += 2.f * (float)sg.y * (sr6 * sr6 - sr6);
        }
      });
      for_stencil(eles, X, Y, Z, Lx, Ly, [&](int pe, double sx, double sy, int, int) {
        const float dx = Xf - (eles.xf[pe] + (float)sx), dy = Yf - (eles.yf[pe] + (float)sy), dz = Zf - eles.zf[pe];
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 >= rc2f || r2 == 0.f) return;
        const float Qj = (float)Q[eles.order[pe]];
        float phi, md2;
        pair_ie_f(r2, af, etaf, phi, md2);
        const float s = qf * Qj * md2;
        kadd(0, s * dx);
        kadd(1, s * dy);
        kadd(2, s * dz);
        eie += qf * Qj * phi;
        if (md.ntype) {
          const double2 sg = md.lj[ti * md.ntype + (md.ntype - 1)];
          const float sr2 = (float)sg.x / r2, sr6 = sr2 * sr2 * sr2;
          const float fs = 24.f * (float)sg.y * (2.f * sr6 * sr6 - sr6) / r2;
          kadd(3, fs * dx);
          kadd(4, fs * dy);
          kadd(5, fs * dz);
          elj += 4.f * (float)sg.y * (sr6 * sr6 - sr6);
        }
      });
      rx = (double)a[0] - cmp[0];
      ry = (double)a[1] - cmp[1];
      rz = (double)a[2] - cmp[2];
      lx = (double)a[3] - cmp[3];
      ly = (double)a[4] - cmp[4];
      lz = (double)a[5] - cmp[5];
      e_ii = eii;
      e_ie = eie;
      e_lj = elj;
    }
    // ---- bonds (FP64; a handful per site)
    double bx = 0, by = 0, bz = 0;
    if (md.ntype && md.bond_start) {
      const double xo = x_orig[i], yo = y_orig[i], zo = z_orig[i];
      for (int b = md.bond_start[i]; b < md.bond_start[i + 1]; ++b) {
        const int j2 = md.bond_j[b];
        double dx = xo - x_orig[j2], dy = yo - y_orig[j2], dz = zo - z_orig[j2];
        dx -= Lx * floor(dx / Lx + 0.5);
        dy -= Ly * floor(dy / Ly + 0.5);
        const double len = sqrt(dx * dx + dy * dy + dz * dz);
        const double ext = len - md.bond_r0[b];
        const double f = -md.kb * ext / len;
        bx = fma(f, dx, bx);
        by = fma(f, dy, by);
        bz = fma(f, dz, bz);
        e_b += 0.25 * md.kb * ext * ext;   // each bond is visited from both ends
      }
    }
    Fx = kKe * (Fx + rx) + lx + bx;
    Fy = kKe * (Fy + ry) + ly + by;
    Fz = kKe * (Fz + rz) + lz + bz;
    F[i] = Fx;
    F[ni + i] = Fy;
    F[2 * ni + i] = Fz;
    red[0][t] = e_ii;
    red[1][t] = e_ie;
    red[2][t] = e_lj;
    red[3][t] = e_b;
  }
  if (epart) {
    __syncthreads();
    for (int s = kGatherThreads / 2; s > 0; s >>= 1) {
      if (t < s)
        for (int e = 0; e < 4; ++e) red[e][t] += red[e][t + s];
      __syncthreads();
    }
    if (t < 4) epart[(int64_t)blockIdx.x * 4 + t] = red[t][0];
  }
}

// electrode-electrode real-space energy 1/2 sum Q_i Q_j [erfc(alpha r) - erfc(r / (sqrt 2 eta))]/r (Eq. 13)
__global__ void k_ee_energy(int64_t ne, CellsDev eles, const double *__restrict__ Q, double Lx, double Ly,
                            double alpha, double eta, double rc, double *__restrict__ out) {
  __shared__ double red[128];
  const int t = threadIdx.x;
  const int64_t p = (int64_t)blockIdx.x * 128 + t;
  double e = 0.0;
  if (p < ne) {
    const double X = eles.xs[p], Y = eles.ys[p], Z = eles.zs[p];
    const double Qi = Q[eles.order[p]];
    const double rc2 = rc * rc, eg = 1.4142135623730951 * eta;
    for_stencil(eles, X, Y, Z, Lx, Ly, [&](int pp, double sx, double sy, int ix, int iy) {
      if (pp == p && ix == 0 && iy == 0) return;
      const double dx = X - (eles.xs[pp] + sx), dy = Y - (eles.ys[pp] + sy), dz = Z - eles.zs[pp];
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 >= rc2 || r2 == 0.0) return;
      const double r = sqrt(r2);
      e += 0.5 * Qi * Q[eles.order[pp]] * (erfc(alpha * r) - erfc(r / eg)) / r;
    });
  }
  red[t] = e;
  __syncthreads();
  for (int s = 64; s > 0; s >>= 1) {
    if (t < s) red[t] += red[t + s];
    __syncthreads();
  }
  if (t == 0) out[blockIdx.x] = red[0];
}

// sums of fixed-size partial arrays into device scalars, in order
__global__ void k_sum_partials(int nblk, int width, const double *__restrict__ part, double *__restrict__ out) {
  const int e = threadIdx.x;
  if (e >= width) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * width + e];
  out[e] = s;
}

void ion_forces(srbe_ctx *c, bool energies) {
  const int K = c->K;
  double2 *coef = c->coef.p;
  if (K > 0) {
    k_coef<<<blocks_for(K, 128), 128, 0, c->stream>>>(K, c->dc.p, c->S2.p, coef, 1);
    c->launches++;
  }
  MdDev md{};
  if (c->have_md) {
    md.ntype = c->ntype;
    md.lj = (const double2 *)c->lj.p;
    md.bond_start = c->bond_start.p;
    md.bond_j = c->bond_j.p;
    md.bond_r0 = c->bond_r0.p;
    md.kb = c->kb;
  }
  const double3 invL = make_double3(1.0 / c->L[0], 1.0 / c->L[1], 1.0 / c->L[2]);
  const double slab = 4.0 * kPi / c->V;
  const unsigned nblk = blocks_for(std::max<int64_t>(c->ni, 1), kGatherThreads);
  double *ep = energies ? c->epart.p : nullptr;
  CellsDev ions = cells_dev(c->icells), eles = cells_dev(c->ecells);
  if (!c->have_md) {
    ions.ts = nullptr;
    ions.ms = nullptr;
  }
  if (c->ni > 0) {
    if (c->precision == SRBE_MIXED)
      k_ion_forces<true><<<nblk, kGatherThreads, 0, c->stream>>>(
          c->ni, ions, eles, c->Q.p, K, c->dm.p, coef, c->tab.p, invL, c->L[0], c->L[1], c->alpha, c->eta, c->rc,
          slab, c->scal.p, md, c->x.p, c->y.p, c->z.p, c->F.p, ep);
    else
      k_ion_forces<false><<<nblk, kGatherThreads, 0, c->stream>>>(
          c->ni, ions, eles, c->Q.p, K, c->dm.p, coef, c->tab.p, invL, c->L[0], c->L[1], c->alpha, c->eta, c->rc,
          slab, c->scal.p, md, c->x.p, c->y.p, c->z.p, c->F.p, ep);
    c->launches++;
    c->mode_evals += c->ni * (int64_t)K;
  }
  if (energies) {
    if (c->ni > 0) {
      k_sum_partials<<<1, 32, 0, c->stream>>>((int)nblk, 4, ep, c->scal.p + kScalEnergy);
    } else {
      SRBE_CUDA(cudaMemsetAsync(c->scal.p + kScalEnergy, 0, 4 * sizeof(double), c->stream));
    }
    const unsigned neb = blocks_for(c->ne, 128);
    double *ee = ep + (size_t)nblk * 4 + 4;   // reserve() sizes epart for both regions
    k_ee_energy<<<neb, 128, 0, c->stream>>>(c->ne, eles, c->Q.p, c->L[0], c->L[1], c->alpha, c->eta, c->rc, ee);
    k_sum_partials<<<1, 32, 0, c->stream>>>((int)neb, 1, ee, c->scal.p + kScalEee);
    c->launches += 3;
  }
  SRBE_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------------------------------------------
// velocity Verlet: v += fac F / m ; optionally r += dt v with x, y wrapped into [0, L)
// ------------------------------------------------------------------------------------------------
__global__ void k_kick_drift(int64_t n, double *__restrict__ x, double *__restrict__ y, double *__restrict__ z,
                             double *__restrict__ vx, double *__restrict__ vy, double *__restrict__ vz,
                             const double *__restrict__ F, const double *__restrict__ minv, double fac, double dt,
                             int drift, double Lx, double Ly) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double w = fac * minv[i];
  double a = fma(w, F[i], vx[i]), b = fma(w, F[n + i], vy[i]), c = fma(w, F[2 * n + i], vz[i]);
  vx[i] = a;
  vy[i] = b;
  vz[i] = c;
  if (drift) {
    double X = fma(dt, a, x[i]), Y = fma(dt, b, y[i]);
    X -= Lx * floor(X / Lx);
    Y -= Ly * floor(Y / Ly);
    if (X >= Lx) X -= Lx;
    if (Y >= Ly) Y -= Ly;
    x[i] = X;
    y[i] = Y;
    z[i] = fma(dt, c, z[i]);
  }
}

void integrate_kick_drift(srbe_ctx *c, double fac_kick, bool drift) {
  if (c->ni == 0) return;
  k_kick_drift<<<blocks_for(c->ni, 256), 256, 0, c->stream>>>(c->ni, c->x.p, c->y.p, c->z.p, c->vx.p, c->vy.p,
                                                             c->vz.p, c->F.p, c->minv.p, fac_kick, c->dt,
                                                             drift ? 1 : 0, c->L[0], c->L[1]);
  c->launches++;
  SRBE_CUDA(cudaGetLastError());
}

}  // namespace srbe
