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
#include <cooperative_groups.h>

#include "srbe_internal.cuh"

namespace cg = cooperative_groups;

namespace srbe {

constexpr double kKe = 138.935458;            // kJ mol^-1 nm e^-2
constexpr double kTwoOverSqrtPi = 1.1283791670955126;

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

// Cells of at least (rc + skin) / 2, so that the stencil of a cell covers rc + skin from any point
// in it: Verlet lists built at rc + skin then hold every pair within rc until an ion has moved
// skin / 2.
void choose_grid(const srbe_ctx *c, CellGrid &g, double zlo, double zhi) {
  const double reach = c->rc + c->nbr.skin;
  const double target = 0.5 * reach;
  for (int d = 0; d < 2; ++d) {
    g.nc[d] = std::max(1, (int)std::floor(c->L[d] / target));
    g.cs[d] = c->L[d] / g.nc[d];
    g.span[d] = (int)std::ceil(reach / g.cs[d] - 1e-12);
    SRBE_REQUIRE(g.span[d] <= 7 * g.nc[d], SRBE_EINVAL, "cutoff too long for the periodic box (more than 7 images)");
  }
  const double h = std::max(zhi - zlo, 1e-9);
  g.nc[2] = std::max(1, (int)std::floor(h / target));
  g.cs[2] = h / g.nc[2];
  g.span[2] = (int)std::ceil(reach / g.cs[2] - 1e-12);
  g.z0 = zlo;
}

static int host_floor_div(int a, int n) { return a >= 0 ? a / n : -((-a + n - 1) / n); }

void build_run_table(srbe_ctx *c) {
  const CellGrid &g = c->ecells.g;
  std::vector<int4> runs;
  std::vector<int32_t> first(g.ncell() + 1, 0);
  for (int cz = 0; cz < g.nc[2]; ++cz)
    for (int cy = 0; cy < g.nc[1]; ++cy)
      for (int cx = 0; cx < g.nc[0]; ++cx) {
        const int cell = (cz * g.nc[1] + cy) * g.nc[0] + cx;
        first[cell] = (int32_t)runs.size();
        for (int zc = std::max(0, cz - g.span[2]); zc <= std::min(g.nc[2] - 1, cz + g.span[2]); ++zc)
          for (int oy = -g.span[1]; oy <= g.span[1]; ++oy) {
            const int yy = cy + oy, iy = host_floor_div(yy, g.nc[1]);
            const int rowbase = (zc * g.nc[1] + (yy - iy * g.nc[1])) * g.nc[0];
            int ox = -g.span[0];
            while (ox <= g.span[0]) {
              const int xx = cx + ox, ix = host_floor_div(xx, g.nc[0]), ccx = xx - ix * g.nc[0];
              const int run = std::min(g.span[0] - ox + 1, g.nc[0] - ccx);
              runs.push_back(make_int4(rowbase + ccx, run, (ix + 512) | ((iy + 512) << 10),
                                       (yy - iy * g.nc[1]) | (zc << 16)));
              ox += run;
            }
          }
      }
  first[g.ncell()] = (int32_t)runs.size();
  c->runtab.runs.ensure(runs.size());
  c->runtab.first.ensure(first.size());
  SRBE_CUDA(cudaMemcpyAsync(c->runtab.runs.p, runs.data(), sizeof(int4) * runs.size(), cudaMemcpyHostToDevice,
                            c->stream));
  SRBE_CUDA(cudaMemcpyAsync(c->runtab.first.p, first.data(), sizeof(int32_t) * first.size(),
                            cudaMemcpyHostToDevice, c->stream));
  SRBE_CUDA(cudaStreamSynchronize(c->stream));
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

// sorts each cell's entries by particle index: one warp per cell; cells of up to 32 entries are
// ranked with shuffles, larger ones fall back to an insertion sort by lane 0
__global__ void k_sort_cells(int ncell, const int32_t *__restrict__ start, int32_t *__restrict__ order) {
  const int lane = threadIdx.x & 31;
  const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (c >= ncell) return;
  const int b = start[c], e = start[c + 1], n = e - b;
  if (n <= 1) return;
  if (n <= 32) {
    const int32_t v = lane < n ? order[b + lane] : 0x7fffffff;
    int rank = 0;
    for (int l = 0; l < 32; ++l) {
      const int32_t w = __shfl_sync(0xffffffffu, v, l);
      rank += (w < v) ? 1 : 0;
    }
    __syncwarp();
    if (lane < n) order[b + rank] = v;
    return;
  }
  if (lane == 0) {
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
}

__global__ void k_gather_sorted(int64_t n, const int32_t *__restrict__ order, const double *__restrict__ x,
                                const double *__restrict__ y, const double *__restrict__ z,
                                const double *__restrict__ w, const int32_t *__restrict__ typ,
                                const int32_t *__restrict__ mol, double *__restrict__ xs, double *__restrict__ ys,
                                double *__restrict__ zs, double *__restrict__ ws, int32_t *__restrict__ ts,
                                int32_t *__restrict__ ms, float4 *__restrict__ pf, uint64_t *__restrict__ us,
                                int32_t *__restrict__ inv, double3 invL) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int32_t i = order[p];
  inv[i] = (int32_t)p;
  us[p] = to_turns64(x[i], invL.x);
  us[n + p] = to_turns64(y[i], invL.y);
  us[2 * n + p] = to_turns64(z[i], invL.z);
  xs[p] = x[i];
  ys[p] = y[i];
  zs[p] = z[i];
  pf[p] = make_float4((float)x[i], (float)y[i], (float)z[i], w ? (float)w[i] : 0.f);
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
  cl.pf.ensure(nn);
  cl.us.ensure(3 * nn);
  cl.inv.ensure(nn);
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
    k_sort_cells<<<blocks_for((int64_t)ncell * 32, 256), 256, 0, c->stream>>>(ncell, cl.start.p, cl.order.p);
    k_gather_sorted<<<blocks_for(n, 256), 256, 0, c->stream>>>(n, cl.order.p, x, y, z, w, typ, mol, cl.xs.p, cl.ys.p,
                                                              cl.zs.p, cl.ws.p, cl.ts.p, cl.ms.p, cl.pf.p, cl.us.p,
                                                              cl.inv.p, make_double3(1.0 / c->L[0], 1.0 / c->L[1],
                                                                           1.0 / c->L[2]));
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

// erfc(x) for x >= 0 from Abramowitz & Stegun 7.1.26 (Hastings' rational approximation,
// |error| <= 1.5e-7 absolute), written against exp(-x^2) so that the force term shares it.
__device__ __forceinline__ float erfc_as(float x, float ex2) {
  // the approximation's own error (1.5e-7) dwarfs the 2-ulp error of the fast reciprocal
  const float t = __fdividef(1.0f, fmaf(0.3275911f, x, 1.0f));
  const float poly = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f),
                                      -0.284496736f), 0.254829592f);
  return poly * ex2;
}

__device__ __forceinline__ void pair_ii_f(float r2, float alpha, float &phi, float &mdphi_r, float &rinv) {
  rinv = rsqrtf(r2);
  const float r = r2 * rinv;
  const float ex = __expf(-alpha * alpha * r2);
  phi = erfc_as(alpha * r, ex) * rinv;
  mdphi_r = (phi + (float)kTwoOverSqrtPi * alpha * ex) * (rinv * rinv);
}

__device__ __forceinline__ void pair_ie_f(float r2, float alpha, float eta, float &phi, float &mdphi_r, float &rinv) {
  rinv = rsqrtf(r2);
  const float r = r2 * rinv;
  const float ex = __expf(-alpha * alpha * r2);
  float p = erfc_as(alpha * r, ex) * rinv, f = p + (float)kTwoOverSqrtPi * alpha * ex;
  if (r < 4.5f * eta) {
    const float eg = erfcf(r / eta);
    const float exg = __expf(-r2 / (eta * eta));
    p -= eg * rinv;
    f -= eg * rinv + (float)kTwoOverSqrtPi / eta * exg;
  }
  phi = p;
  mdphi_r = f * (rinv * rinv);
}

struct CellsDev {
  GridDev g;
  const int32_t *start, *order;
  const double *xs, *ys, *zs, *ws;
  const int32_t *ts, *ms;
  const float4 *pf;
  const uint64_t *us;
  const int32_t *inv;
  const int4 *runs;
  const int32_t *run_first;
  int64_t n;
};

static CellsDev cells_dev(const Cells &cl, const RunTable &rt) {
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
  d.pf = cl.pf.p;
  d.us = cl.us.p;
  d.inv = cl.inv.p;
  d.runs = rt.runs.p;
  d.run_first = rt.first.p;
  d.n = 0;
  return d;
}

// Visits every (neighbour, image) within the stencil of a point, serially: fn(p, sx, sy, ix, iy)
// with p the sorted index, (sx, sy) the image shift to add to the neighbour and (ix, iy) the image
// index.  Used by the energy diagnostics; the hot gathers split the stencil over a warp.
__device__ __forceinline__ int floor_div(int a, int n) { return a >= 0 ? a / n : -((-a + n - 1) / n); }

template <class Fn>
__device__ __forceinline__ void for_stencil(const CellsDev &C, double x, double y, double z, double Lx, double Ly,
                                            Fn &&fn) {
  const GridDev &g = C.g;
  const int cx = cell_coord(x, g.inv[0], g.nc[0]);
  const int cy = cell_coord(y, g.inv[1], g.nc[1]);
  const int cz = cell_coord(z - g.z0, g.inv[2], g.nc[2]);
  const int z_lo = max(0, cz - g.span[2]), z_hi = min(g.nc[2] - 1, cz + g.span[2]);
  for (int zc = z_lo; zc <= z_hi; ++zc) {
    for (int oy = -g.span[1]; oy <= g.span[1]; ++oy) {
      const int yy = cy + oy;
      const int iy = floor_div(yy, g.nc[1]);
      const int ccy = yy - iy * g.nc[1];
      for (int ox = -g.span[0]; ox <= g.span[0]; ++ox) {
        const int xx = cx + ox;
        const int ix = floor_div(xx, g.nc[0]);
        const int ccx = xx - ix * g.nc[0];
        const int cell = (zc * g.nc[1] + ccy) * g.nc[0] + ccx;
        const int b = C.start[cell], e = C.start[cell + 1];
        for (int p = b; p < e; ++p) fn(p, ix * Lx, iy * Ly, ix, iy);
      }
    }
  }
}

// Butterfly sum over a warp.  Each step adds two lanes' values, and a + b == b + a exactly, so
// every lane ends with the same, run-to-run reproducible, value.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct KahanF32 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c, t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
  __device__ __forceinline__ float valuef() const { return s - c; }
};

constexpr int kMaxLjTypes = 16;        // atom types of the LJ table (the FP32 forces keep it in shared memory)

// FP32 pre-check margin: positions below 64 nm carry at most ~4e-6 nm of rounding in FP32
constexpr float kPrecheckMargin = 1e-3f;

struct MdDev {
  int ntype;                        // 0 = no LJ / bonds
  const double2 *lj;                // (sigma^2, eps) per type pair
  const float2 *lj32;               // the same in FP32 (mixed form)
  const int32_t *bond_start, *bond_j;
  const double *bond_r0;
  double kb;
};

// Per-ion constants and accumulators of the real-space pair sums.  Candidate neighbours that pass
// the cutoff test are first compacted into a per-warp queue (index, image) in shared memory, so
// that the pair arithmetic always runs on 32 pairs at once instead of on the ~20% of lanes whose
// candidate falls inside rc.
struct PairSite {
  double X, Y, Z, qi, Lx, Ly, alpha, eta, rc2;
  float Xf, Yf, Zf, qf, Lxf, Lyf, af, etaf;
  float qke;                          // K_E q_i (FP32 form: Coulomb folded into kJ/mol/nm)
  int ti, mi;
  int64_t p;
};

// FP32 form: one plain sum per component of K_E x Coulomb + LJ (each lane adds ~20 terms, then a
// warp tree; errors stay near 1e-6 of the largest term, far inside the form's 1e-3 budget)
struct PairAcc {
  float f0 = 0.f, f1 = 0.f, f2 = 0.f;
  float eii = 0.f, eie = 0.f, elj = 0.f;
  double r[3] = {0, 0, 0}, l[3] = {0, 0, 0};   // FP64 form
  double dii = 0, die = 0, dlj = 0;
};

__device__ __forceinline__ int pack_image(int ix, int iy) { return (ix + 512) | ((iy + 512) << 10); }
__device__ __forceinline__ int image_x(int v) { return (v & 1023) - 512; }
__device__ __forceinline__ int image_y(int v) { return ((v >> 10) & 1023) - 512; }

template <bool F32, bool EN>
__device__ __forceinline__ void pair_ion_ion(const PairSite &S, const CellsDev &ions, const MdDev &md, int2 e,
                                             PairAcc &A) {
  const int pp = e.x, ix = image_x(e.y), iy = image_y(e.y);
  const bool lj = md.ntype && ions.ms[pp] != S.mi;
  if (F32) {
    const float4 o = ions.pf[pp];
    const float dx = S.Xf - (o.x + (float)ix * S.Lxf), dy = S.Yf - (o.y + (float)iy * S.Lyf), dz = S.Zf - o.z;
    const float r2 = dx * dx + dy * dy + dz * dz;
    float phi, md2, rinv;
    pair_ii_f(r2, S.af, phi, md2, rinv);
    float fs = S.qke * o.w * md2;
    if (EN) A.eii += 0.5f * S.qf * o.w * phi;
    if (lj) {
      const float2 sg = md.lj32[S.ti * md.ntype + ions.ts[pp]];
      const float ir2 = rinv * rinv, sr2 = sg.x * ir2, sr6 = sr2 * sr2 * sr2;
      fs += 24.f * sg.y * (2.f * sr6 * sr6 - sr6) * ir2;
      if (EN) A.elj += 2.f * sg.y * (sr6 * sr6 - sr6);
    }
    A.f0 = fmaf(fs, dx, A.f0);
    A.f1 = fmaf(fs, dy, A.f1);
    A.f2 = fmaf(fs, dz, A.f2);
  } else {
    const double dx = S.X - (ions.xs[pp] + ix * S.Lx), dy = S.Y - (ions.ys[pp] + iy * S.Ly), dz = S.Z - ions.zs[pp];
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 >= S.rc2) return;
    double phi, md2;
    pair_ii(r2, S.alpha, phi, md2);
    const double qq = S.qi * ions.ws[pp], s = qq * md2;
    A.r[0] = fma(s, dx, A.r[0]);
    A.r[1] = fma(s, dy, A.r[1]);
    A.r[2] = fma(s, dz, A.r[2]);
    if (EN) A.dii = fma(0.5 * qq, phi, A.dii);
    if (lj) {
      const double2 sg = md.lj[S.ti * md.ntype + ions.ts[pp]];
      const double sr2 = sg.x / r2, sr6 = sr2 * sr2 * sr2;
      const double fs = 24.0 * sg.y * (2.0 * sr6 * sr6 - sr6) / r2;
      A.l[0] = fma(fs, dx, A.l[0]);
      A.l[1] = fma(fs, dy, A.l[1]);
      A.l[2] = fma(fs, dz, A.l[2]);
      if (EN) A.dlj += 0.5 * 4.0 * sg.y * (sr6 * sr6 - sr6);
    }
  }
}

template <bool F32, bool EN>
__device__ __forceinline__ void pair_ion_ele(const PairSite &S, const CellsDev &eles, const MdDev &md,
                                             const double *__restrict__ Q, const float *__restrict__ Q32, int2 e,
                                             PairAcc &A) {
  const int pe = e.x, ix = image_x(e.y), iy = image_y(e.y);
  if (F32) {
    const float4 o = eles.pf[pe];
    const float dx = S.Xf - (o.x + (float)ix * S.Lxf), dy = S.Yf - (o.y + (float)iy * S.Lyf), dz = S.Zf - o.z;
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float Qj = Q32[eles.order[pe]];
    float phi, md2, rinv;
    pair_ie_f(r2, S.af, S.etaf, phi, md2, rinv);
    float fs = S.qke * Qj * md2;
    if (EN) A.eie += S.qf * Qj * phi;
    if (md.ntype) {
      const float2 sg = md.lj32[S.ti * md.ntype + (md.ntype - 1)];
      const float ir2 = rinv * rinv, sr2 = sg.x * ir2, sr6 = sr2 * sr2 * sr2;
      fs += 24.f * sg.y * (2.f * sr6 * sr6 - sr6) * ir2;
      if (EN) A.elj += 4.f * sg.y * (sr6 * sr6 - sr6);
    }
    A.f0 = fmaf(fs, dx, A.f0);
    A.f1 = fmaf(fs, dy, A.f1);
    A.f2 = fmaf(fs, dz, A.f2);
  } else {
    const double dx = S.X - (eles.xs[pe] + ix * S.Lx), dy = S.Y - (eles.ys[pe] + iy * S.Ly), dz = S.Z - eles.zs[pe];
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 >= S.rc2 || r2 == 0.0) return;
    const double Qj = Q[eles.order[pe]];
    double phi, md2;
    pair_ie(r2, S.alpha, S.eta, phi, md2);
    const double s = S.qi * Qj * md2;
    A.r[0] = fma(s, dx, A.r[0]);
    A.r[1] = fma(s, dy, A.r[1]);
    A.r[2] = fma(s, dz, A.r[2]);
    if (EN) A.die = fma(S.qi * Qj, phi, A.die);
    if (md.ntype) {
      const double2 sg = md.lj[S.ti * md.ntype + (md.ntype - 1)];
      const double sr2 = sg.x / r2, sr6 = sr2 * sr2 * sr2;
      const double fs = 24.0 * sg.y * (2.0 * sr6 * sr6 - sr6) / r2;
      A.l[0] = fma(fs, dx, A.l[0]);
      A.l[1] = fma(fs, dy, A.l[1]);
      A.l[2] = fma(fs, dz, A.l[2]);
      if (EN) A.dlj += 4.0 * sg.y * (sr6 * sr6 - sr6);
    }
  }
}

// Walks the stencil of S over the cell list C and compacts candidates with squared distance below
// cut2 (FP32 test) into the warp queue q; calls pair(entry) for every full batch of 32 and once
// more for the rest.  All lanes of the warp take part; skip_self drops the zero image of S.p.
template <class Pair>
__device__ __forceinline__ void compacted_pairs(const PairSite &S, const CellsDev &C, int cell, bool skip_self,
                                                float cut2, int2 *q, int lane, Pair &&pair) {
  int qn = 0;
  const unsigned below = (1u << lane) - 1u;
  const int r1 = C.run_first[cell + 1];
  for (int r = C.run_first[cell]; r < r1; ++r) {
    const int4 R = C.runs[r];
    const int b0 = C.start[R.x], b1 = C.start[R.x + R.y];
    if (b0 == b1) continue;
    const int ix = image_x(R.z), iy = image_y(R.z);
    const float sxf = (float)ix * S.Lxf, syf = (float)iy * S.Lyf;
    const bool zero_image = skip_self && ix == 0 && iy == 0;
    const int img = R.z;
    for (int base = b0; base < b1; base += 32) {
      const int pp = base + lane;
      bool in = false;
      if (pp < b1 && !(zero_image && pp == S.p)) {
        const float4 o = C.pf[pp];
        const float dx = S.Xf - (o.x + sxf), dy = S.Yf - (o.y + syf), dz = S.Zf - o.z;
        const float r2 = dx * dx + dy * dy + dz * dz;
        in = r2 < cut2 && r2 > 0.f;
      }
      const unsigned m = __ballot_sync(0xffffffffu, in);
      if (in) q[qn + __popc(m & below)] = make_int2(pp, img);
      qn += __popc(m);
      if (qn >= 32) {
        __syncwarp();
        pair(q[lane]);
        __syncwarp();
        if (lane < qn - 32) q[lane] = q[lane + 32];
        __syncwarp();
        qn -= 32;
      }
    }
  }
  __syncwarp();
  if (lane < qn) pair(q[lane]);
  __syncwarp();
}

// The same compaction over a Verlet list: entries pack a sorted index (bits 0-22), an LJ-exclusion
// bit (bit 23: the pair lies inside one molecule; ion-ion lists only) and the image shifts ix + 8,
// iy + 8 (bits 24-27, 28-31); consecutive lanes read consecutive entries.
constexpr int32_t kListExcl = 1 << 23;
__device__ __forceinline__ int list_index(int32_t e) { return e & 0x7fffff; }
__device__ __forceinline__ int list_ix(int32_t e) { return ((e >> 24) & 15) - 8; }
__device__ __forceinline__ int list_iy(int32_t e) { return ((unsigned)e >> 28) - 8; }
// image shifts of a list entry as floats without an int-to-float conversion: the 4-bit field ORed
// into the mantissa of 2^23 gives 2^23 + (shift + 8) exactly
__device__ __forceinline__ float list_fx(int32_t e) {
  return __int_as_float(0x4B000000 | (((unsigned)e >> 24) & 15u)) - 8388616.0f;
}
__device__ __forceinline__ float list_fy(int32_t e) {
  return __int_as_float(0x4B000000 | ((unsigned)e >> 28)) - 8388616.0f;
}
__device__ __forceinline__ int32_t list_entry(int idx, int ix, int iy) {
  return (int32_t)((unsigned)idx | ((unsigned)(ix + 8) << 24) | ((unsigned)(iy + 8) << 28));
}

template <class Pair>
__device__ __forceinline__ void compacted_list(const PairSite &S, const CellsDev &C, const int32_t *__restrict__ list,
                                               int count, float cut2, int2 *q, int lane, Pair &&pair) {
  int qn = 0;
  const unsigned below = (1u << lane) - 1u;
  for (int base = 0; base < count; base += 32) {
    const int k = base + lane;
    bool in = false;
    int pp = 0, img = 0;
    if (k < count) {
      const int32_t e = list[k];
      pp = list_index(e);
      const int ix = list_ix(e), iy = list_iy(e);
      const float4 o = C.pf[pp];
      const float dx = S.Xf - (o.x + (float)ix * S.Lxf), dy = S.Yf - (o.y + (float)iy * S.Lyf), dz = S.Zf - o.z;
      const float r2 = dx * dx + dy * dy + dz * dz;
      in = r2 < cut2 && r2 > 0.f;
      img = pack_image(ix, iy);
    }
    const unsigned m = __ballot_sync(0xffffffffu, in);
    if (in) q[qn + __popc(m & below)] = make_int2(pp, img);
    qn += __popc(m);
    if (qn >= 32) {
      __syncwarp();
      pair(q[lane]);
      __syncwarp();
      if (lane < qn - 32) q[lane] = q[lane + 32];
      __syncwarp();
      qn -= 32;
    }
  }
  __syncwarp();
  if (lane < qn) pair(q[lane]);
  __syncwarp();
}

// FP32 passes over one Verlet list (the mixed form's forces): 32 entries per batch with a
// three-stage software pipeline, the entries of batch b+2 and the particle data of batch b+1 in
// flight while batch b computes, so that the two dependent gathers (entry, then particle) overlap
// with arithmetic.  Lanes whose entry lies beyond rc (about a fifth of a list built at rc + skin)
// sit out their batch instead of being compacted.  ljs: the LJ table in shared memory.
template <bool EN>
__device__ __forceinline__ void ii_list_f32(const PairSite &S, const CellsDev &ions, const MdDev &md,
                                            const float2 *ljs, const int32_t *__restrict__ list, int count,
                                            float cut2, int lane, PairAcc &A) {
  const bool mdon = md.ntype != 0;
  auto entry = [&](int k) { return k < count ? __ldg(list + k) : 0; };
  int32_t e0 = entry(lane), e1 = entry(32 + lane);
  int i0 = list_index(e0);
  float4 o0 = ions.pf[i0];
  int m0 = mdon ? ions.ms[i0] : 0, t0 = mdon ? ions.ts[i0] : 0;
  for (int base = 0; base < count; base += 32) {
    const int32_t e2 = entry(base + 64 + lane);
    const int i1 = list_index(e1);
    const float4 o1 = ions.pf[i1];
    const int m1 = mdon ? ions.ms[i1] : 0, t1 = mdon ? ions.ts[i1] : 0;
    // batch b
    const float dx = S.Xf - fmaf(list_fx(e0), S.Lxf, o0.x);
    const float dy = S.Yf - fmaf(list_fy(e0), S.Lyf, o0.y), dz = S.Zf - o0.z;
    const float r2 = dx * dx + dy * dy + dz * dz;
    if (base + lane < count && r2 < cut2 && r2 > 0.f) {
      float phi, md2, rinv;
      pair_ii_f(r2, S.af, phi, md2, rinv);
      float fs = S.qke * o0.w * md2;
      if (EN) A.eii += 0.5f * S.qf * o0.w * phi;
      if (mdon && m0 != S.mi) {
        const float2 sg = ljs[S.ti * md.ntype + t0];
        const float ir2 = rinv * rinv, sr2 = sg.x * ir2, sr6 = sr2 * sr2 * sr2;
        fs += 24.f * sg.y * (2.f * sr6 * sr6 - sr6) * ir2;
        if (EN) A.elj += 2.f * sg.y * (sr6 * sr6 - sr6);
      }
      A.f0 = fmaf(fs, dx, A.f0);
      A.f1 = fmaf(fs, dy, A.f1);
      A.f2 = fmaf(fs, dz, A.f2);
    }
    e0 = e1;
    e1 = e2;
    o0 = o1;
    m0 = m1;
    t0 = t1;
  }
}

template <bool EN>
__device__ __forceinline__ void ie_list_f32(const PairSite &S, const CellsDev &eles, const MdDev &md,
                                            const float2 *ljs, const float *__restrict__ Q32,
                                            const int32_t *__restrict__ list, int count, float cut2, int lane,
                                            PairAcc &A) {
  auto entry = [&](int k) { return k < count ? __ldg(list + k) : 0; };
  int32_t e0 = entry(lane), e1 = entry(32 + lane);
  int j0 = list_index(e0);
  float4 o0 = eles.pf[j0];
  int s0 = eles.order[j0];
  const float2 sg = md.ntype ? ljs[S.ti * md.ntype + (md.ntype - 1)] : make_float2(0.f, 0.f);
  for (int base = 0; base < count; base += 32) {
    const int32_t e2 = entry(base + 64 + lane);
    const int j1 = list_index(e1);
    const float4 o1 = eles.pf[j1];
    const int s1 = eles.order[j1];
    const float dx = S.Xf - fmaf(list_fx(e0), S.Lxf, o0.x);
    const float dy = S.Yf - fmaf(list_fy(e0), S.Lyf, o0.y), dz = S.Zf - o0.z;
    const float r2 = dx * dx + dy * dy + dz * dz;
    if (base + lane < count && r2 < cut2 && r2 > 0.f) {
      const float Qj = __ldg(Q32 + s0);
      float phi, md2, rinv;
      pair_ie_f(r2, S.af, S.etaf, phi, md2, rinv);
      float fs = S.qke * Qj * md2;
      if (EN) A.eie += S.qf * Qj * phi;
      if (md.ntype) {
        const float ir2 = rinv * rinv, sr2 = sg.x * ir2, sr6 = sr2 * sr2 * sr2;
        fs += 24.f * sg.y * (2.f * sr6 * sr6 - sr6) * ir2;
        if (EN) A.elj += 4.f * sg.y * (sr6 * sr6 - sr6);
      }
      A.f0 = fmaf(fs, dx, A.f0);
      A.f1 = fmaf(fs, dy, A.f1);
      A.f2 = fmaf(fs, dz, A.f2);
    }
    e0 = e1;
    e1 = e2;
    o0 = o1;
    s0 = s1;
  }
}

// FP32 pass over an electrode site's Verlet list (the mixed form's near part of b, Eq. 19): the
// same three-stage pipeline as the ion passes, Kahan-compensated sum of -q_i phi_ie
__device__ __forceinline__ void ei_list_f32(const PairSite &S, const CellsDev &ions, const int32_t *__restrict__ list,
                                            int count, float cut2, int lane, KahanF32 &acc) {
  auto entry = [&](int k) { return k < count ? __ldg(list + k) : 0; };
  int32_t e0 = entry(lane), e1 = entry(32 + lane);
  float4 o0 = ions.pf[list_index(e0)];
  for (int base = 0; base < count; base += 32) {
    const int32_t e2 = entry(base + 64 + lane);
    const float4 o1 = ions.pf[list_index(e1)];
    const float dx = S.Xf - fmaf(list_fx(e0), S.Lxf, o0.x);
    const float dy = S.Yf - fmaf(list_fy(e0), S.Lyf, o0.y), dz = S.Zf - o0.z;
    const float r2 = dx * dx + dy * dy + dz * dz;
    if (base + lane < count && r2 < cut2 && r2 > 0.f) {
      float phi, md2, rinv;
      pair_ie_f(r2, S.af, S.etaf, phi, md2, rinv);
      acc.add(-o0.w * phi);
    }
    e0 = e1;
    e1 = e2;
    o0 = o1;
  }
}

// the FP32 copies of the scalar parameters the mixed form needs (converted once on the host)
struct ForceF32 {
  float Lx, Ly, alpha, eta, rc, slab, kb;
};

// Verlet-list view handed to the gathers
struct ListsDev {
  const int32_t *ii, *ie, *ei, *ii_n, *ie_n, *ei_n, *cell_s, *ecell;
  int cap;
};

// ------------------------------------------------------------------------------------------------
// electrode right-hand side: one warp per electrode site, lanes split the modes and the stencil
// ------------------------------------------------------------------------------------------------
// coefS[k] = (c_k Re S1(k), c_k Im S1(k));  b_F,j = - sum_k Re(exp(-i k.R_j) c_k S1) (Eq. 24)
template <bool F32>
__global__ void __launch_bounds__(kGatherThreads)
k_electrode_rhs(int64_t ne, const double *__restrict__ ex, const double *__restrict__ ey,
                const double *__restrict__ ez, const uint64_t *__restrict__ eu, int K, const int4 *__restrict__ modes,
                const double2 *__restrict__ coefS, const float2 *__restrict__ coefS32,
                const double2 *__restrict__ tab, double3 invL, CellsDev ions, ListsDev nl,
                double Lx, double Ly, double alpha, double eta, double rc, double slab, const double *__restrict__ scal,
                double *__restrict__ b, float2 *__restrict__ bsplit, const double *__restrict__ bfar,
                const float4 *__restrict__ epf, ForceF32 pf) {
  __shared__ int2 wq[kWarpsPerBlock][64];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t j = ((int64_t)blockIdx.x * kGatherThreads + threadIdx.x) >> 5;
  if (j >= ne) return;                        // whole warps leave together; no block barrier below
  // the mixed form takes the site and the scalars in FP32 (no FP64 conversion per lane)
  const double X = F32 ? 0.0 : ex[j], Y = F32 ? 0.0 : ey[j], Z = F32 ? 0.0 : ez[j];
  const float4 sf = F32 ? epf[j] : make_float4(0.f, 0.f, 0.f, 0.f);
  const uint64_t ux = eu[j], uy = eu[ne + j], uz = eu[2 * ne + j];
  double acc = 0.0;
  KahanF32 fk;
  if (bfar) {
    // far part precomputed by the lattice transforms
  } else if (!F32) {
    for (int k = lane; k < K; k += 32) {
      double cs, sn;
      sincos_turns(phase64(__ldg(&modes[k]), ux, uy, uz), tab, cs, sn);
      const double2 cf = __ldg(&coefS[k]);
      acc = fma(-cf.x, cs, acc);
      acc = fma(-cf.y, sn, acc);
    }
  } else {
    const uint32_t vx = (uint32_t)(ux >> 32), vy = (uint32_t)(uy >> 32), vz = (uint32_t)(uz >> 32);
    for (int k = lane; k < K; k += 32) {
      const int4 m = __ldg(&modes[k]);
      float cs, sn;
      sincos_turns32((uint32_t)m.x * vx + (uint32_t)m.y * vy + (uint32_t)m.z * vz, cs, sn);
      const float2 cf = __ldg(&coefS32[k]);
      fk.add(-cf.x * cs - cf.y * sn);
    }
  }
  // near part of Eq. 19: - sum_i q_i [erfc(alpha d) - erfc(d/eta)] / d over images within rc,
  // candidates compacted through the warp queue
  PairSite S;
  S.X = X; S.Y = Y; S.Z = Z; S.qi = 0.0; S.Lx = Lx; S.Ly = Ly; S.alpha = alpha; S.eta = eta; S.rc2 = rc * rc;
  if (F32) {
    S.Xf = sf.x; S.Yf = sf.y; S.Zf = sf.z;
    S.Lxf = pf.Lx; S.Lyf = pf.Ly; S.af = pf.alpha; S.etaf = pf.eta;
  } else {
    S.Xf = (float)X; S.Yf = (float)Y; S.Zf = (float)Z;
    S.Lxf = (float)Lx; S.Lyf = (float)Ly; S.af = (float)alpha; S.etaf = (float)eta;
  }
  S.qf = 0.f;
  S.ti = 0; S.mi = -1; S.p = -1;
  const float rcf = F32 ? pf.rc : (float)rc;
  const float cut2 = F32 ? rcf * rcf : (rcf + kPrecheckMargin) * (rcf + kPrecheckMargin);
  KahanF32 fn;
  double near = 0.0;
  auto near_pair = [&](int2 e) {
    const int pp = e.x, ix = image_x(e.y), iy = image_y(e.y);
    if (F32) {
      const float4 o = ions.pf[pp];
      const float dx = S.Xf - (o.x + (float)ix * S.Lxf), dy = S.Yf - (o.y + (float)iy * S.Lyf), dz = S.Zf - o.z;
      float phi, md, rinv;
      pair_ie_f(dx * dx + dy * dy + dz * dz, S.af, S.etaf, phi, md, rinv);
      fn.add(-o.w * phi);
    } else {
      const double dx = X - (ions.xs[pp] + ix * Lx), dy = Y - (ions.ys[pp] + iy * Ly), dz = Z - ions.zs[pp];
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < S.rc2 && r2 > 0.0) {
        double phi, md;
        pair_ie(r2, alpha, eta, phi, md);
        near = fma(-ions.ws[pp], phi, near);
      }
    }
  };
  const int nei = nl.ei_n[j];
  if (F32 && nei <= nl.cap) ei_list_f32(S, ions, nl.ei + j * nl.cap, nei, cut2, lane, fn);
  else if (nei <= nl.cap) compacted_list(S, ions, nl.ei + j * nl.cap, nei, cut2, wq[warp], lane, near_pair);
  else compacted_pairs(S, ions, nl.ecell[j], false, cut2, wq[warp], lane, near_pair);
  if (F32) {
    // FP32 to the end of the warp sum: on this GPU every FP64 warp instruction is costly
    const float accf = warp_sum_f(fk.valuef() + fn.valuef());
    if (lane == 0) {
      const double bj = fma(-slab * ez[j], scal[kScalMion], (double)accf + (bfar ? bfar[j] : 0.0));
      const float hi = (float)bj;
      b[j] = bj;
      bsplit[j] = make_float2(hi, (float)(bj - (double)hi));
    }
  } else {
    acc = warp_sum(acc + near);
    // slab part (FP64 in every form): -(4 pi / V) Z_j sum_i q_i z_i
    if (lane == 0) b[j] = fma(-slab * Z, scal[kScalMion], bfar ? acc + bfar[j] : acc);
  }
}

static ListsDev lists_dev(const srbe_ctx *c) {
  ListsDev d;
  d.ii = c->nbr.ii.p;
  d.ie = c->nbr.ie.p;
  d.ei = c->nbr.ei.p;
  d.ii_n = c->nbr.ii_n.p;
  d.ie_n = c->nbr.ie_n.p;
  d.ei_n = c->nbr.ei_n.p;
  d.cell_s = c->nbr.cell_s.p;
  d.ecell = c->ecells.cell.p;
  d.cap = c->nbr.cap;
  return d;
}

// ------------------------------------------------------------------------------------------------
// Verlet lists of the ions: one cooperative launch per step.
//   phase 0  refresh the sorted copies in the order of the last build, x and y unwrapped next to
//            the build positions (so the stored image shifts stay valid), and flag a rebuild when
//            an ion has moved more than skin / 2;
//   grid sync; if no rebuild: done;
//   phases 1-6  rebuild the cell list (zero, count, scan, scatter, per-cell sort, gather + snapshot);
//   phases 7-8  rebuild the ion-ion / ion-electrode lists (warp per ion) and the electrode-ion
//               lists (warp per electrode site) at rc + skin.
// The barriers are cooperative-groups grid syncs over a co-resident grid.
// ------------------------------------------------------------------------------------------------
struct NbrKernelArgs {
  int64_t n, ne;
  int ncell, cap;
  const double *x, *y, *z, *w;
  const int32_t *typ, *mol;
  int32_t *cell, *rank, *start, *order, *inv, *ts, *ms, *cell_s;
  double *xs, *ys, *zs, *ws, *xb, *yb;
  float4 *pf, *pfb;
  uint64_t *us;
  int32_t *ii, *ie, *ei, *ii_n, *ie_n, *ei_n;
  GridDev g;
  const int4 *runs;
  const int32_t *run_first;
  CellsDev eles;
  const int32_t *ecell;
  const double *ex, *ey, *ez;
  double Lx, Ly;
  double3 invL;
  float cut2, half_skin2;
  float csf[3], z0f;     // cell edges and the grid's lower z in FP32 (stencil pruning)
  int *flag;
};

__device__ __forceinline__ void warp_append(int32_t *list, int cap, int &count, bool in, int32_t entry, int lane) {
  const unsigned m = __ballot_sync(0xffffffffu, in);
  const int pos = count + __popc(m & ((1u << lane) - 1u));
  if (in && pos < cap) list[pos] = entry;
  count += __popc(m);
}

// appends every particle of the runs of `cell` within sqrt(cut2) of (X, Y, Z) to list.  The runs
// and their particle ranges are fetched 32 at a time (lane = run) and broadcast, so that a list
// costs one round of dependent loads for the whole stencil instead of one per run.
// ms (ion-ion lists with molecules): entries of particles of molecule `mol` get the exclusion bit.
__device__ __forceinline__ int build_list(const NbrKernelArgs &a, const int4 *runs, const int32_t *run_first, int cell,
                                          const int32_t *start, const float4 *pf, float X, float Y, float Z,
                                          int64_t self, int32_t *list, int lane, const int32_t *ms = nullptr,
                                          int mol = -1) {
  int count = 0;
  const float Lxf = (float)a.Lx, Lyf = (float)a.Ly;
  // stencil pruning: a run (one row of cells) whose box lies farther than the reach (plus a margin
  // for FP32 rounding of the cell edges) in y and z is skipped, and its cells beyond the reach in x
  // are trimmed; the end cells in z hold any particle beyond them, so they are open-ended
  const float reach = sqrtf(a.cut2) + 1e-3f, reach2 = reach * reach;
  const int rfirst = run_first[cell], nrun = run_first[cell + 1] - rfirst;
  for (int rb = 0; rb < nrun; rb += 32) {
    int mb0 = 0, mb1 = 0, mz = 0;
    if (rb + lane < nrun) {
      const int4 R = runs[rfirst + rb + lane];
      const int ccy = R.w & 0xffff, zc = R.w >> 16;
      const int ix = image_x(R.z), iy = image_y(R.z);
      const float ylo = (float)ccy * a.csf[1] + (float)iy * Lyf, yhi = ylo + a.csf[1];
      const float zlo = a.z0f + (float)zc * a.csf[2], zhi = zlo + a.csf[2];
      const float dy = fmaxf(fmaxf(ylo - Y, Y - yhi), 0.f);
      const float dz = fmaxf(fmaxf(zc > 0 ? zlo - Z : 0.f, zc < a.g.nc[2] - 1 ? Z - zhi : 0.f), 0.f);
      const float d2 = dy * dy + dz * dz;
      if (d2 < reach2) {
        const float xr = sqrtf(reach2 - d2), xs = X - (float)ix * Lxf;
        const int ccx0 = R.x - (zc * a.g.nc[1] + ccy) * a.g.nc[0];
        const int klo = max(0, (int)floorf((xs - xr) / a.csf[0]) - ccx0);
        const int khi = min(R.y - 1, (int)floorf((xs + xr) / a.csf[0]) - ccx0);
        if (klo <= khi) {
          mb0 = start[R.x + klo];
          mb1 = start[R.x + khi + 1];
          mz = R.z;
        }
      }
    }
    const int nq = min(32, nrun - rb);
    for (int q = 0; q < nq; ++q) {
      const int b0 = __shfl_sync(0xffffffffu, mb0, q), b1 = __shfl_sync(0xffffffffu, mb1, q);
      if (b0 == b1) continue;
      const int code = __shfl_sync(0xffffffffu, mz, q);
      const int ix = image_x(code), iy = image_y(code);
      const float sx = (float)ix * Lxf, sy = (float)iy * Lyf;
      const bool zero_image = ix == 0 && iy == 0;
      // two batches of 32 candidates per pass, both loads issued before either test (the entries
      // are appended in candidate order, as one batch at a time would)
      for (int base = b0; base < b1; base += 64) {
        const int pa = base + lane, pb = base + 32 + lane;
        const bool va = pa < b1 && !(zero_image && pa == self), vb = pb < b1 && !(zero_image && pb == self);
        const float4 oa = va ? pf[pa] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 ob = vb ? pf[pb] : make_float4(0.f, 0.f, 0.f, 0.f);
        float dx = X - (oa.x + sx), dy = Y - (oa.y + sy), dz = Z - oa.z;
        const bool ina = va && dx * dx + dy * dy + dz * dz < a.cut2;
        dx = X - (ob.x + sx);
        dy = Y - (ob.y + sy);
        dz = Z - ob.z;
        const bool inb = vb && dx * dx + dy * dy + dz * dz < a.cut2;
        const int32_t exa = ina && ms && ms[pa] == mol ? kListExcl : 0;
        const int32_t exb = inb && ms && ms[pb] == mol ? kListExcl : 0;
        warp_append(list, a.cap, count, ina, list_entry(pa, ix, iy) | exa, lane);
        if (base + 32 < b1) warp_append(list, a.cap, count, inb, list_entry(pb, ix, iy) | exb, lane);
      }
    }
  }
  return count;
}

// Every step: the sorted copies follow the ions (unwrapped against the build positions, so the
// lists' image shifts stay valid) and any ion that moved more than skin / 2 since the build raises
// flag[0]; a forced rebuild (flag[1]) skips the refresh and raises flag[0] itself.  Four threads per
// sorted ion, one per component (the fourth only completes the group): the FP64 unwrap and
// fixed-point conversion of a component is a short chain, and three of them in parallel keep the
// kernel short; the group sums its squared displacements with shuffles for the skin test.
__global__ void __launch_bounds__(256) k_nbr_refresh(NbrKernelArgs a) {
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (__ldcg(&a.flag[1])) {
    if (gtid == 0) a.flag[0] = 1;
    return;
  }
  const int64_t p = gtid >> 2;
  const int d = (int)(gtid & 3);
  float e2 = 0.f;
  if (p < a.n && d < 3) {
    const int32_t i = a.order[p];
    const float4 b = a.pfb[p];
    float ed;
    if (d < 2) {
      // displacement since the build position, back across the periodic wrap (it is far below
      // L / 2 unless the ion was wrapped, then within a skin of +-L): no FP64 division
      const double L = d == 0 ? a.Lx : a.Ly;
      const double base = d == 0 ? a.xb[p] : a.yb[p];
      double dx = (d == 0 ? a.x[i] : a.y[i]) - base;
      if (dx > 0.5 * L) dx -= L;
      else if (dx < -0.5 * L) dx += L;
      const double X = base + dx;
      if (d == 0) {
        a.xs[p] = X;
        a.pf[p].x = (float)X;
        ed = (float)X - b.x;
      } else {
        a.ys[p] = X;
        a.pf[p].y = (float)X;
        ed = (float)X - b.y;
      }
      a.us[d * a.n + p] = to_turns64(X, d == 0 ? a.invL.x : a.invL.y);
    } else {
      const double Z = a.z[i];
      a.zs[p] = Z;
      a.pf[p].z = (float)Z;
      ed = (float)Z - b.z;
      a.us[2 * a.n + p] = to_turns64(Z, a.invL.z);
    }
    e2 = ed * ed;
  }
  // the group of four lanes holds one ion: add its three squared components in the order x, y, z
  const float ey2 = __shfl_down_sync(0xffffffffu, e2, 1), ez2 = __shfl_down_sync(0xffffffffu, e2, 2);
  if (d == 0 && p < a.n && (e2 + ey2) + ez2 > a.half_skin2) atomicOr(&a.flag[0], 1);
}

// The rebuild, one cooperative launch whose phases are separated by grid-wide barriers.  The
// decision (flag[0], final once k_nbr_refresh has run) is read once per block and is the same for
// every block, so without a rebuild the whole grid returns before its first barrier.
__global__ void __launch_bounds__(256) k_neighbor_update(NbrKernelArgs a) {
  cg::grid_group grid = cg::this_grid();
  __shared__ int32_t part[256];
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + tid, gsize = (int64_t)gridDim.x * blockDim.x;
  const int64_t gwarp = gtid >> 5, nwarps = gsize >> 5;
  __shared__ int s_rebuild;
  if (tid == 0) s_rebuild = __ldcg(&a.flag[0]);
  __syncthreads();
  if (!s_rebuild) return;
  // ---- phase 1: zero the cell counts and the list-task counter
  for (int64_t c = gtid; c <= a.ncell; c += gsize) a.start[c] = 0;
  if (gtid == 0) a.flag[2] = 0;
  grid.sync();
  // ---- phase 2: count
  for (int64_t i = gtid; i < a.n; i += gsize) {
    const int cx = cell_coord(a.x[i], a.g.inv[0], a.g.nc[0]);
    const int cy = cell_coord(a.y[i], a.g.inv[1], a.g.nc[1]);
    const int cz = cell_coord(a.z[i] - a.g.z0, a.g.inv[2], a.g.nc[2]);
    const int c = (cz * a.g.nc[1] + cy) * a.g.nc[0] + cx;
    a.cell[i] = c;
    a.rank[i] = atomicAdd(&a.start[c], 1);
  }
  grid.sync();
  // ---- phase 3: exclusive scan (block 0)
  if (blockIdx.x == 0) {
    const int per = (a.ncell + 255) / 256;
    const int b = tid * per, e = min(a.ncell, b + per);
    int32_t s = 0;
    for (int i = b; i < e; ++i) s += a.start[i];
    part[tid] = s;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
      const int32_t v = tid >= off ? part[tid - off] : 0;
      __syncthreads();
      part[tid] += v;
      __syncthreads();
    }
    int32_t run = part[tid] - s;
    for (int i = b; i < e; ++i) {
      const int32_t v = a.start[i];
      a.start[i] = run;
      run += v;
    }
    if (tid == 255) a.start[a.ncell] = part[255];
  }
  grid.sync();
  // ---- phase 4: scatter
  for (int64_t i = gtid; i < a.n; i += gsize) a.order[a.start[a.cell[i]] + a.rank[i]] = (int32_t)i;
  grid.sync();
  // ---- phase 5: sort each cell by particle index (warp per cell)
  for (int64_t c = gwarp; c < a.ncell; c += nwarps) {
    const int b = a.start[c], e = a.start[c + 1], m = e - b;
    if (m <= 1) continue;
    if (m <= 32) {
      const int32_t v = lane < m ? a.order[b + lane] : 0x7fffffff;
      int rank = 0;
      for (int l = 0; l < 32; ++l) rank += (__shfl_sync(0xffffffffu, v, l) < v) ? 1 : 0;
      __syncwarp();
      if (lane < m) a.order[b + rank] = v;
    } else if (lane == 0) {
      for (int i = b + 1; i < e; ++i) {
        const int32_t v = a.order[i];
        int j = i - 1;
        while (j >= b && a.order[j] > v) {
          a.order[j + 1] = a.order[j];
          --j;
        }
        a.order[j + 1] = v;
      }
    }
    __syncwarp();
  }
  grid.sync();
  // ---- phase 6: gather into sorted order and snapshot the build positions
  for (int64_t p = gtid; p < a.n; p += gsize) {
    const int32_t i = a.order[p];
    a.inv[i] = (int32_t)p;
    const double X = a.x[i], Y = a.y[i], Z = a.z[i];
    a.xs[p] = X;
    a.ys[p] = Y;
    a.zs[p] = Z;
    a.xb[p] = X;
    a.yb[p] = Y;
    a.ws[p] = a.w[i];
    if (a.typ) a.ts[p] = a.typ[i];
    if (a.mol) a.ms[p] = a.mol[i];
    const float4 f = make_float4((float)X, (float)Y, (float)Z, (float)a.w[i]);
    a.pf[p] = f;
    a.pfb[p] = f;
    a.us[p] = to_turns64(X, a.invL.x);
    a.us[a.n + p] = to_turns64(Y, a.invL.y);
    a.us[2 * a.n + p] = to_turns64(Z, a.invL.z);
    a.cell_s[p] = a.cell[i];
  }
  grid.sync();
  // ---- phase 7: the ion-ion, ion-electrode and electrode-ion lists as one pool of tasks (one list
  // each), handed to warps through an atomic counter in that order, so that the warps finish together
  // (a list's content does not depend on the warp that builds it)
  (void)gwarp;
  (void)nwarps;
  const int64_t ntask = 2 * a.n + a.ne;
  for (;;) {
    int64_t t = 0;
    if (lane == 0) t = atomicAdd(&a.flag[2], 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= ntask) break;
    if (t < a.n) {
      const int64_t p = t;
      const float4 me = a.pf[p];
      const int nii = build_list(a, a.runs, a.run_first, a.cell_s[p], a.start, a.pf, me.x, me.y, me.z, p,
                                 a.ii + p * a.cap, lane, a.mol ? a.ms : nullptr, a.mol ? a.ms[p] : -1);
      // pad the ion-ion list to a whole number of 32-entry batches with entries that always lie beyond
      // the cutoff (the ion itself seven box lengths away in x and y), so that the mixed form's pass
      // runs without bounds checks; a list that overflowed is walked from the stencil instead
      if (nii <= a.cap) {
        const int padded = min(a.cap, (nii + 31) & ~31);
        if (nii + lane < padded) a.ii[p * a.cap + nii + lane] = list_entry((int)p, 7, 7);
      }
      if (lane == 0) a.ii_n[p] = nii;
    } else if (t < 2 * a.n) {
      const int64_t p = t - a.n;
      const float4 me = a.pf[p];
      const int nie = build_list(a, a.runs, a.run_first, a.cell_s[p], a.eles.start, a.eles.pf, me.x, me.y, me.z, -1,
                                 a.ie + p * a.cap, lane);
      if (lane == 0) a.ie_n[p] = nie;
    } else {
      const int64_t j = t - 2 * a.n;
      const int nei = build_list(a, a.runs, a.run_first, a.ecell[j], a.start, a.pf, (float)a.ex[j], (float)a.ey[j],
                                 (float)a.ez[j], -1, a.ei + j * a.cap, lane);
      if (lane == 0) a.ei_n[j] = nei;
    }
  }
  grid.sync();
  if (gtid == 0) {
    a.flag[0] = 0;
    a.flag[1] = 0;
  }
}

void neighbor_force_rebuild(srbe_ctx *c) {
  int *f = c->nbr.flag.ensure(3);
  const int one[2] = {1, 1};
  SRBE_CUDA(cudaMemcpyAsync(f, one, sizeof(one), cudaMemcpyHostToDevice, c->stream));
  SRBE_CUDA(cudaStreamSynchronize(c->stream));
}

void neighbor_update(srbe_ctx *c) {
  Cells &cl = c->icells;
  NbrLists &nb = c->nbr;
  const int64_t n = c->ni;
  const size_t nn = (size_t)std::max<int64_t>(n, 1);
  const int ncell = cl.g.ncell();
  SRBE_REQUIRE(nb.cap > 0 && nb.ii.cap >= nn * (size_t)nb.cap, SRBE_ESTATE, "neighbor lists not reserved");
  NbrKernelArgs a;
  a.n = n;
  a.ne = c->ne;
  a.ncell = ncell;
  a.cap = nb.cap;
  a.x = c->x.p;
  a.y = c->y.p;
  a.z = c->z.p;
  a.w = c->q.p;
  a.typ = c->have_md ? c->itype.p : nullptr;
  a.mol = c->have_md ? c->mol.p : nullptr;
  a.cell = cl.cell.p;
  a.rank = cl.rank.p;
  a.start = cl.start.p;
  a.order = cl.order.p;
  a.inv = cl.inv.p;
  a.ts = cl.ts.p;
  a.ms = cl.ms.p;
  a.cell_s = nb.cell_s.p;
  a.xs = cl.xs.p;
  a.ys = cl.ys.p;
  a.zs = cl.zs.p;
  a.ws = cl.ws.p;
  a.xb = nb.xb.p;
  a.yb = nb.yb.p;
  a.pf = cl.pf.p;
  a.pfb = nb.pfb.p;
  a.us = cl.us.p;
  a.ii = nb.ii.p;
  a.ie = nb.ie.p;
  a.ei = nb.ei.p;
  a.ii_n = nb.ii_n.p;
  a.ie_n = nb.ie_n.p;
  a.ei_n = nb.ei_n.p;
  a.g = to_dev(cl.g);
  a.runs = c->runtab.runs.p;
  a.run_first = c->runtab.first.p;
  a.eles = cells_dev(c->ecells, c->runtab);
  a.ecell = c->ecells.cell.p;
  a.ex = c->ex.p;
  a.ey = c->ey.p;
  a.ez = c->ez.p;
  a.Lx = c->L[0];
  a.Ly = c->L[1];
  a.invL = make_double3(1.0 / c->L[0], 1.0 / c->L[1], 1.0 / c->L[2]);
  for (int d = 0; d < 3; ++d) a.csf[d] = (float)cl.g.cs[d];
  a.z0f = (float)cl.g.z0;
  const float reach = (float)(c->rc + nb.skin) + (c->precision == SRBE_MIXED ? 0.f : kPrecheckMargin);
  a.cut2 = reach * reach;
  a.half_skin2 = (float)(0.25 * nb.skin * nb.skin);
  a.flag = nb.flag.p;
  static int blocks_per_sm = 0, nsm = 0;
  if (!blocks_per_sm) {
    int dev = 0;
    SRBE_CUDA(cudaGetDevice(&dev));
    SRBE_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    SRBE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_neighbor_update, 256, 0));
    SRBE_REQUIRE(blocks_per_sm > 0, SRBE_ECUDA, "neighbor-update kernel cannot be resident");
  }
  const int want = (int)std::max<int64_t>(1, std::min<int64_t>((std::max<int64_t>(n, c->ne) * 32 + 255) / 256,
                                                                 (int64_t)blocks_per_sm * nsm));
  k_nbr_refresh<<<blocks_for(4 * std::max<int64_t>(n, 1), 128), 128, 0, c->stream>>>(a);
  SRBE_CUDA(cudaGetLastError());
  void *args[] = {&a};
  coop_before(c);
  SRBE_CUDA(cudaLaunchCooperativeKernel((const void *)k_neighbor_update, dim3(want), dim3(256), args, 0, c->stream));
  coop_after(c);
  c->launches += 2;
}

void electrode_rhs(srbe_ctx *c) {
  const int K = c->K;
  const double *bfar = nullptr;
  if (c->lat.active(c->ne, K)) {
    lattice_bfar(c);
    bfar = c->lat.bF.p;
  }
  double2 *coef = c->coef.p;   // written by the S1 reduction
  const double3 invL = make_double3(1.0 / c->L[0], 1.0 / c->L[1], 1.0 / c->L[2]);
  const double slab = 4.0 * kPi / c->V;
  const CellsDev ions = cells_dev(c->icells, c->runtab);
  const unsigned nb = blocks_for(c->ne, kWarpsPerBlock);
  const ForceF32 pf{(float)c->L[0], (float)c->L[1], (float)c->alpha, (float)c->eta, (float)c->rc, (float)slab, 0.f};
  if (c->precision == SRBE_MIXED)
    k_electrode_rhs<true><<<nb, kGatherThreads, 0, c->stream>>>(c->ne, c->ex.p, c->ey.p, c->ez.p, c->eu.p, K, c->dm.p,
                                                               coef,
                                                               c->coef32.p, c->tab.p, invL, ions, lists_dev(c), c->L[0], c->L[1], c->alpha,
                                                               c->eta, c->rc, slab, c->scal.p, c->bvec.p, c->bsplit.p,
                                                               bfar, c->epf.p, pf);
  else
    k_electrode_rhs<false><<<nb, kGatherThreads, 0, c->stream>>>(c->ne, c->ex.p, c->ey.p, c->ez.p, c->eu.p, K, c->dm.p,
                                                               coef,
                                                                c->coef32.p, c->tab.p, invL, ions, lists_dev(c), c->L[0], c->L[1], c->alpha,
                                                                c->eta, c->rc, slab, c->scal.p, c->bvec.p, c->bsplit.p,
                                                                bfar, c->epf.p, pf);
  c->launches++;
  if (!bfar) c->mode_evals += c->ne * (int64_t)K;
  SRBE_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------------------------------------------
// ion forces: one warp per ion, lanes split the modes and the stencil cells
// ------------------------------------------------------------------------------------------------

// coefF[k] = (c_k Im S(k), c_k Re S(k)) with S = S1 + S2;
// F_i = - q_i sum_k c_k k Im(S exp(-i k . r_i)) = - q_i sum_k k (cIm cos - cRe sin)   (Eq. 25)

// exact FP32 -> FP64 widening with integer instructions (FP64-pipe conversions are scarce on this
// GPU): normal numbers re-biased, zeros kept; subnormal, infinite and NaN inputs take the conversion
__device__ __forceinline__ double widen_f32(float f) {
  const uint32_t u = __float_as_uint(f), e = (u >> 23) & 0xffu;
  if (e - 1u < 254u)
    return __longlong_as_double((long long)(((uint64_t)(u >> 31) << 63) | ((uint64_t)(e + 896u) << 52) |
                                            ((uint64_t)(u & 0x7fffffu) << 29)));
  if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)((uint64_t)(u >> 31) << 63));
  return (double)f;
}

// PART 0: the whole force.  PART 2 (mixed form without energies): everything but the ion-ion pairs
// and bonds, plus Fii, their forces from k_ion_ii (sorted order; they need neither Q nor S, so that
// pass runs beside b, the solve and S2)
template <bool F32, bool EN, int PART>
__global__ void __launch_bounds__(kGatherThreads)
k_ion_forces(int64_t ni, CellsDev ions, CellsDev eles, ListsDev nl, const double *__restrict__ Q,
             const float *__restrict__ Q32,
             int K, const int4 *__restrict__ modes, const double2 *__restrict__ coefF,
             const float2 *__restrict__ coefF32, const double2 *__restrict__ tab,
             double3 invL, float3 kvf, double Lx, double Ly, double alpha, double eta, double rc, double slab,
             ForceF32 pf, const double *__restrict__ scal, MdDev md, const double *__restrict__ x_orig,
             const double *__restrict__ y_orig, const double *__restrict__ z_orig, double *__restrict__ F,
             double *__restrict__ epart, const float4 *__restrict__ Fii) {
  static_assert(PART == 0 || (PART == 2 && F32 && !EN), "the split force pass is the mixed form's, without energies");
  __shared__ double red[kWarpsPerBlock][4];
  __shared__ int2 wq[kWarpsPerBlock][64];
  __shared__ float2 ljs[kMaxLjTypes * kMaxLjTypes];
  __shared__ float s_mz;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // blocks take their groups of 8 ions alternately from the two ends of the sorted order: the ions
  // next to the electrode walls (long ion-electrode lists) sit at both ends (cells are z-major), so
  // both walls' groups start early instead of the far wall's ending the launch (each ion's result
  // does not depend on which block computes it)
  const int64_t bq = blockIdx.x >> 1;
  const int64_t bg = (blockIdx.x & 1) ? (int64_t)gridDim.x - 1 - bq : bq;
  const int64_t p = bg * kWarpsPerBlock + warp;
  double e_ii = 0, e_ie = 0, e_lj = 0, e_b = 0;
  if (F32) {
    for (int t = threadIdx.x; t < md.ntype * md.ntype; t += blockDim.x) ljs[t] = md.lj32[t];
    // M_z (an FP64 sum over all charges) in FP32, once per block
    if (threadIdx.x == 0) s_mz = (float)(scal[kScalMion] + scal[kScalMele]);
  }
  __syncthreads();
  if (p < ni) {
    const int32_t i = ions.order[p];
    // PART 2: the ion-ion pass's force for this ion, fetched now and used in the epilogue
    const float4 fii_p = PART == 2 && lane == 0 ? Fii[p] : make_float4(0.f, 0.f, 0.f, 0.f);
    const double X = ions.xs[p], Y = ions.ys[p], Z = ions.zs[p], qi = ions.ws[p];
    const int ti = ions.ts ? ions.ts[p] : 0;
    const int mi = ions.ms ? ions.ms[p] : -1;
    const uint64_t ux = ions.us[p], uy = ions.us[ni + p], uz = ions.us[2 * ni + p];
    const double tpx = 2.0 * kPi * invL.x, tpy = 2.0 * kPi * invL.y, tpz = 2.0 * kPi * invL.z;
    // ---- k-space gather
    double fk[3] = {0, 0, 0};
    float ak0 = 0.f, ak1 = 0.f, ak2 = 0.f;
    if (!F32) {
      for (int k = lane; k < K; k += 32) {
        const int4 m = __ldg(&modes[k]);
        double cs, sn;
        sincos_turns(phase64(m, ux, uy, uz), tab, cs, sn);
        const double2 cf = __ldg(&coefF[k]);
        const double im = fma(cf.x, cs, -cf.y * sn);
        fk[0] = fma(tpx * m.x, im, fk[0]);
        fk[1] = fma(tpy * m.y, im, fk[1]);
        fk[2] = fma(tpz * m.z, im, fk[2]);
      }
    } else {
      const uint32_t vx = (uint32_t)(ux >> 32), vy = (uint32_t)(uy >> 32), vz = (uint32_t)(uz >> 32);
      for (int k = lane; k < K; k += 32) {
        const int4 m = __ldg(&modes[k]);
        float cs, sn;
        sincos_turns32((uint32_t)m.x * vx + (uint32_t)m.y * vy + (uint32_t)m.z * vz, cs, sn);
        const float2 cf = __ldg(&coefF32[k]);
        const float im = cf.x * cs - cf.y * sn;
        ak0 = fmaf(small_int_to_float(m.x), im, ak0);
        ak1 = fmaf(small_int_to_float(m.y), im, ak1);
        ak2 = fmaf(small_int_to_float(m.z), im, ak2);
      }
    }
    // ---- real space: Coulomb of Eq. 13 (Gaussian units) and LJ (kJ/mol/nm), compacted pairs
    PairSite S;
    S.X = X; S.Y = Y; S.Z = Z; S.qi = qi; S.Lx = Lx; S.Ly = Ly; S.alpha = alpha; S.eta = eta; S.rc2 = rc * rc;
    const float4 self = ions.pf[p];
    S.Xf = self.x; S.Yf = self.y; S.Zf = self.z; S.qf = self.w;
    S.Lxf = pf.Lx; S.Lyf = pf.Ly; S.af = pf.alpha; S.etaf = pf.eta;
    S.qke = (float)kKe * self.w;
    S.ti = ti; S.mi = mi; S.p = p;
    const float rcf = F32 ? pf.rc : (float)rc;
    const float cut2 = F32 ? rcf * rcf : (rcf + kPrecheckMargin) * (rcf + kPrecheckMargin);
    PairAcc A;
    int2 *q = wq[warp];
    // Verlet lists; a particle whose list overflowed walks the stencil of its build cell instead
    const int nii = nl.ii_n[p], nie = nl.ie_n[p];
    if (PART == 2) {
      // the ion-ion pairs came from k_ion_ii
    } else if (F32 && nii <= nl.cap)
      ii_list_f32<EN>(S, ions, md, ljs, nl.ii + p * nl.cap, nii, cut2, lane, A);
    else if (nii <= nl.cap)
      compacted_list(S, ions, nl.ii + p * nl.cap, nii, cut2, q, lane,
                     [&](int2 e) { pair_ion_ion<F32, EN>(S, ions, md, e, A); });
    else
      compacted_pairs(S, ions, nl.cell_s[p], true, cut2, q, lane,
                      [&](int2 e) { pair_ion_ion<F32, EN>(S, ions, md, e, A); });
    if (F32 && nie <= nl.cap)
      ie_list_f32<EN>(S, eles, md, ljs, Q32, nl.ie + p * nl.cap, nie, cut2, lane, A);
    else if (nie <= nl.cap)
      compacted_list(S, eles, nl.ie + p * nl.cap, nie, cut2, q, lane,
                     [&](int2 e) { pair_ion_ele<F32, EN>(S, eles, md, Q, Q32, e, A); });
    else
      compacted_pairs(S, eles, nl.cell_s[p], false, cut2, q, lane,
                      [&](int2 e) { pair_ion_ele<F32, EN>(S, eles, md, Q, Q32, e, A); });
    const float Xf = S.Xf, Yf = S.Yf, Zf = S.Zf, qf = S.qf;
    double rr[3] = {A.r[0], A.r[1], A.r[2]}, ll[3] = {A.l[0], A.l[1], A.l[2]};
    e_ii = A.dii;
    e_ie = A.die;
    e_lj = A.dlj;
    float eii = A.eii, eie = A.eie, elj = A.elj;
    if (F32) {
      // FP32 to the end: sums, warp reductions, bonds and the force assembly; only M_z (an FP64
      // reduction over all charges) enters from FP64
      float v[6] = {ak0, ak1, ak2, A.f0, A.f1, A.f2};
#pragma unroll
      for (int d = 0; d < 6; ++d) v[d] = warp_sum_f(v[d]);
      if (EN) {
        eii = warp_sum_f(eii);
        eie = warp_sum_f(eie);
        elj = warp_sum_f(elj);
      }
      if (lane == 0) {
        const float Fx = -qf * kvf.x * v[0];
        const float Fy = -qf * kvf.y * v[1];
        const float Fz = -qf * kvf.z * v[2] - pf.slab * qf * s_mz;
        float bx = 0.f, by = 0.f, bz = 0.f, eb = 0.f;
        if (PART != 2 && md.ntype && md.bond_start) {
          const float Lxf = pf.Lx, Lyf = pf.Ly, kbf = pf.kb;
          for (int b = md.bond_start[i]; b < md.bond_start[i + 1]; ++b) {
            const float4 o = ions.pf[ions.inv[md.bond_j[b]]];
            float dx = Xf - o.x, dy = Yf - o.y, dz = Zf - o.z;
            dx -= Lxf * floorf(dx / Lxf + 0.5f);
            dy -= Lyf * floorf(dy / Lyf + 0.5f);
            const float len = sqrtf(dx * dx + dy * dy + dz * dz);
            const float ext = len - (float)md.bond_r0[b];
            const float f = -kbf * ext / len;
            bx += f * dx;
            by += f * dy;
            bz += f * dz;
            eb += 0.25f * kbf * ext * ext;   // each bond is visited from both ends
          }
        }
        const float ke = (float)kKe;
        if (PART == 2) {
          bx = fii_p.x;
          by = fii_p.y;
          bz = fii_p.z;
        }
        F[i] = widen_f32(ke * Fx + v[3] + bx);
        F[ni + i] = widen_f32(ke * Fy + v[4] + by);
        F[2 * ni + i] = widen_f32(ke * Fz + v[5] + bz);
        e_ii = eii;
        e_ie = eie;
        e_lj = elj;
        e_b = eb;
      }
    } else {
      for (int d = 0; d < 3; ++d) {
        fk[d] = warp_sum(fk[d]);
        rr[d] = warp_sum(rr[d]);
        ll[d] = warp_sum(ll[d]);
      }
      if (EN) {
        e_ii = warp_sum(e_ii);
        e_ie = warp_sum(e_ie);
        e_lj = warp_sum(e_lj);
      }
      if (lane == 0) {
        double Fx = -qi * fk[0], Fy = -qi * fk[1], Fz = -qi * fk[2];
        // slab force: M_z = sum q_i z_i + sum Q_j Z_j
        Fz = fma(-slab * qi, scal[kScalMion] + scal[kScalMele], Fz);
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
        F[i] = kKe * (Fx + rr[0]) + ll[0] + bx;
        F[ni + i] = kKe * (Fy + rr[1]) + ll[1] + by;
        F[2 * ni + i] = kKe * (Fz + rr[2]) + ll[2] + bz;
      }
    }
  }
  if (EN && epart) {
    if (lane == 0) {
      red[warp][0] = e_ii;
      red[warp][1] = e_ie;
      red[warp][2] = e_lj;
      red[warp][3] = e_b;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
      double s = 0.0;
      for (int w = 0; w < kWarpsPerBlock; ++w) s += red[w][threadIdx.x];
      epart[(int64_t)blockIdx.x * 4 + threadIdx.x] = s;
    }
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

namespace {
struct ForceLaunch {
  MdDev md{};
  double3 invL;
  float3 kvf;
  double slab;
  unsigned nblk;
  CellsDev ions, eles;
  ForceF32 pf;
};
ForceLaunch force_launch(srbe_ctx *c) {
  ForceLaunch f;
  if (c->have_md) {
    f.md.ntype = c->ntype;
    f.md.lj = (const double2 *)c->lj.p;
    f.md.lj32 = c->lj32.p;
    f.md.bond_start = c->bond_start.p;
    f.md.bond_j = c->bond_j.p;
    f.md.bond_r0 = c->bond_r0.p;
    f.md.kb = c->kb;
  }
  f.invL = make_double3(1.0 / c->L[0], 1.0 / c->L[1], 1.0 / c->L[2]);
  f.kvf = make_float3((float)(2.0 * kPi / c->L[0]), (float)(2.0 * kPi / c->L[1]), (float)(2.0 * kPi / c->L[2]));
  f.slab = 4.0 * kPi / c->V;
  f.nblk = blocks_for(std::max<int64_t>(c->ni, 1), kWarpsPerBlock);
  f.ions = cells_dev(c->icells, c->runtab);
  f.eles = cells_dev(c->ecells, c->runtab);
  if (!c->have_md) {
    f.ions.ts = nullptr;
    f.ions.ms = nullptr;
  }
  f.pf = ForceF32{(float)c->L[0], (float)c->L[1], (float)c->alpha, (float)c->eta,
                  (float)c->rc,   (float)f.slab, (float)f.md.kb};
  return f;
}
}  // namespace

// The mixed form's ion-ion pass (real-space Coulomb of Eq. 13 between ions, LJ, bonds; no Q, no S):
// one warp per ion over its Verlet list, FP32.  The list is padded to whole 32-entry batches with
// entries beyond the cutoff, so the loop has no bounds checks; an entry carries the LJ exclusion of
// an intramolecular pair, so the only gathers per entry are the neighbour's (x, y, z, q) and, with
// LJ, its type; image shifts come from a 256-entry shared table indexed by the entry's top byte.
// Two-stage software pipeline: the entries of batch b + 2 and the particle data of batch b + 1 are
// in flight while batch b computes.  Per lane the terms are summed in list order, then a warp tree.
// the list of ion p overflowed at its build: walk the stencil of its build cell (kept out of line so
// that the list loop's registers do not carry it)
__device__ __noinline__ float3 ion_ii_stencil(int64_t p, float4 me, int ti, int mi, const CellsDev &ions,
                                               const ListsDev &nl, const MdDev &md, const ForceF32 &pf, int2 *q,
                                               int lane) {
  PairSite S;
  S.Xf = me.x; S.Yf = me.y; S.Zf = me.z; S.qf = me.w; S.Lxf = pf.Lx; S.Lyf = pf.Ly; S.af = pf.alpha;
  S.etaf = pf.eta; S.qke = (float)kKe * me.w; S.ti = ti; S.mi = mi; S.p = p;
  PairAcc A;
  compacted_pairs(S, ions, nl.cell_s[p], true, pf.rc * pf.rc, q, lane,
                  [&](int2 e) { pair_ion_ion<true, false>(S, ions, md, e, A); });
  return make_float3(A.f0, A.f1, A.f2);
}

// one ion's pass (the body of k_ion_ii)
template <bool LJ>
__device__ __forceinline__ void ion_ii_one(int64_t p, int64_t ni, const CellsDev &ions, const ListsDev &nl,
                                           const MdDev &md, const ForceF32 &pf, const float2 *shift,
                                           const float2 *ljs, int2 *wq, int lane, float4 *__restrict__ Fii) {
  if (p >= ni) return;
  const float4 me = ions.pf[p];
  const int ti = LJ ? ions.ts[p] : 0;
  const float2 *ljrow = ljs + ti * md.ntype;
  const float qke = (float)kKe * me.w, af = pf.alpha, cut2 = pf.rc * pf.rc, Lx = pf.Lx, Ly = pf.Ly;
  float f0 = 0.f, f1 = 0.f, f2 = 0.f;
  const int cnt = nl.ii_n[p];
  if (cnt <= nl.cap) {
    const int32_t *list = nl.ii + p * nl.cap;
    const int nb = min(nl.cap, (cnt + 31) & ~31);
    int32_t e0 = nb > 0 ? __ldg(list + lane) : 0, e1 = nb > 32 ? __ldg(list + 32 + lane) : 0;
    float4 o0 = ions.pf[list_index(e0)];
    int t0 = LJ ? ions.ts[list_index(e0)] : 0;
    for (int base = 0; base < nb; base += 32) {
      const int32_t e2 = base + 64 < nb ? __ldg(list + base + 64 + lane) : 0;
      const int j1 = list_index(e1);
      const float4 o1 = ions.pf[j1];
      const int t1 = LJ ? ions.ts[j1] : 0;
      // batch b
      const float2 sh = shift[(unsigned)e0 >> 24];
      const float dx = me.x - fmaf(sh.x, Lx, o0.x), dy = me.y - fmaf(sh.y, Ly, o0.y), dz = me.z - o0.z;
      const float r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < cut2 && r2 > 0.f) {
        float phi, md2, rinv;
        pair_ii_f(r2, af, phi, md2, rinv);
        float fs = qke * o0.w * md2;
        if (LJ && !(e0 & kListExcl)) {
          const float2 sg = ljrow[t0];
          const float ir2 = rinv * rinv, sr2 = sg.x * ir2, sr6 = sr2 * sr2 * sr2;
          fs += sg.y * (2.f * sr6 * sr6 - sr6) * ir2;
        }
        f0 = fmaf(fs, dx, f0);
        f1 = fmaf(fs, dy, f1);
        f2 = fmaf(fs, dz, f2);
      }
      e0 = e1;
      e1 = e2;
      o0 = o1;
      t0 = t1;
    }
  } else {
    const float3 f = ion_ii_stencil(p, me, ti, LJ ? ions.ms[p] : -1, ions, nl, md, pf, wq, lane);
    f0 = f.x;
    f1 = f.y;
    f2 = f.z;
  }
  f0 = warp_sum_f(f0);
  f1 = warp_sum_f(f1);
  f2 = warp_sum_f(f2);
  if (lane == 0) {
    float bx = 0.f, by = 0.f, bz = 0.f;
    if (LJ && md.bond_start) {
      const int32_t i = ions.order[p];
      const float kbf = pf.kb;
      for (int b = md.bond_start[i]; b < md.bond_start[i + 1]; ++b) {
        const float4 o = ions.pf[ions.inv[md.bond_j[b]]];
        float dx = me.x - o.x, dy = me.y - o.y, dz = me.z - o.z;
        dx -= Lx * floorf(dx / Lx + 0.5f);
        dy -= Ly * floorf(dy / Ly + 0.5f);
        const float len = sqrtf(dx * dx + dy * dy + dz * dz);
        const float ext = len - (float)md.bond_r0[b];
        const float f = -kbf * ext / len;
        bx += f * dx;
        by += f * dy;
        bz += f * dz;
      }
    }
    Fii[p] = make_float4(f0 + bx, f1 + by, f2 + bz, 0.f);
  }
}

template <bool LJ>
__global__ void __launch_bounds__(kGatherThreads, 5)
k_ion_ii(int64_t ni, CellsDev ions, ListsDev nl, MdDev md, ForceF32 pf, float4 *__restrict__ Fii) {
  __shared__ float2 shift[256];                     // (ix, iy) image counts as floats, by entry >> 24
  __shared__ float2 ljs[kMaxLjTypes * kMaxLjTypes]; // (sigma^2, 24 eps)
  __shared__ int2 wq[kWarpsPerBlock][64];           // queue of the stencil walk (overflowed lists)
  for (int t = threadIdx.x; t < 256; t += blockDim.x)
    shift[t] = make_float2(small_int_to_float((t & 15) - 8), small_int_to_float((t >> 4) - 8));
  if (LJ)
    for (int t = threadIdx.x; t < md.ntype * md.ntype; t += blockDim.x) {
      const float2 v = md.lj32[t];
      ljs[t] = make_float2(v.x, 24.f * v.y);
    }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // one warp per ion (a grid-stride loop, so any grid size covers every ion)
  for (int64_t p = (int64_t)blockIdx.x * kWarpsPerBlock + warp; p < ni; p += (int64_t)gridDim.x * kWarpsPerBlock)
    ion_ii_one<LJ>(p, ni, ions, nl, md, pf, shift, ljs, wq[warp], lane, Fii);
}

bool ion_forces_split(const srbe_ctx *c, bool energies) {
  return c->precision == SRBE_MIXED && !energies && c->ni > 0;
}

// the mixed form's ion-ion pass (pairs and bonds: no Q, no S) on the side stream, right behind the
// neighbour update there, so that it runs beside b, the charge solve and S2 on the main stream
void ion_forces_ii(srbe_ctx *c) {
  const ForceLaunch f = force_launch(c);
  float4 *fii = c->fii.ensure((size_t)c->ni);
  const ListsDev L = lists_dev(c);
  const int64_t n = c->ni;
  const unsigned nblk = f.nblk;
  if (c->have_md && f.md.ntype)
    k_ion_ii<true><<<nblk, kGatherThreads, 0, c->side>>>(n, f.ions, L, f.md, f.pf, fii);
  else
    k_ion_ii<false><<<nblk, kGatherThreads, 0, c->side>>>(n, f.ions, L, f.md, f.pf, fii);
  c->launches++;
  SRBE_CUDA(cudaGetLastError());
  SRBE_CUDA(cudaEventRecord(c->ev_ii, c->side));
  c->fii_pending = true;
}

void ion_forces(srbe_ctx *c, bool energies) {
  const int K = c->K;
  double2 *coef = c->coef.p;   // written by the S2 reduction (S = S1 + S2)
  MdDev md{};
  if (c->have_md) {
    md.ntype = c->ntype;
    md.lj = (const double2 *)c->lj.p;
    md.lj32 = c->lj32.p;
    md.bond_start = c->bond_start.p;
    md.bond_j = c->bond_j.p;
    md.bond_r0 = c->bond_r0.p;
    md.kb = c->kb;
  }
  const double3 invL = make_double3(1.0 / c->L[0], 1.0 / c->L[1], 1.0 / c->L[2]);
  const float3 kvf = make_float3((float)(2.0 * kPi / c->L[0]), (float)(2.0 * kPi / c->L[1]),
                                 (float)(2.0 * kPi / c->L[2]));
  const double slab = 4.0 * kPi / c->V;
  const unsigned nblk = blocks_for(std::max<int64_t>(c->ni, 1), kWarpsPerBlock);
  double *ep = energies ? c->epart.p : nullptr;
  CellsDev ions = cells_dev(c->icells, c->runtab), eles = cells_dev(c->ecells, c->runtab);
  if (!c->have_md) {
    ions.ts = nullptr;
    ions.ms = nullptr;
  }
  if (c->ni > 0) {
    const bool mixed = c->precision == SRBE_MIXED;
    const bool part2 = c->fii_pending && ion_forces_split(c, energies);
    auto kern = part2 ? k_ion_forces<true, false, 2>
                : mixed ? (energies ? k_ion_forces<true, true, 0> : k_ion_forces<true, false, 0>)
                        : (energies ? k_ion_forces<false, true, 0> : k_ion_forces<false, false, 0>);
    if (part2) SRBE_CUDA(cudaStreamWaitEvent(c->stream, c->ev_ii, 0));
    const ForceF32 pf{(float)c->L[0], (float)c->L[1], (float)c->alpha, (float)c->eta,
                      (float)c->rc,   (float)slab,   (float)md.kb};
    kern<<<nblk, kGatherThreads, 0, c->stream>>>(c->ni, ions, eles, lists_dev(c), c->Q.p, c->Q32.p, K, c->dm.p, coef,
                                                 c->coef32.p, c->tab.p, invL, kvf, c->L[0], c->L[1], c->alpha, c->eta,
                                                 c->rc, slab, pf, c->scal.p, md, c->x.p, c->y.p, c->z.p, c->F.p, ep,
                                                 part2 ? c->fii.p : nullptr);
    c->launches++;
    c->mode_evals += c->ni * (int64_t)K;
  }
  c->fii_pending = false;
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
// Langevin part of Eq. 39 over one step, solved exactly (Ornstein-Uhlenbeck):
// v <- c1 v + sqrt((1 - c1^2) kB T / m) g with c1 = exp(-gamma dt) and g three standard normals per
// ion from Philox4x64-10, key (seed, 'LANG'), counter (step, i, 0, 0), Box-Muller on 53-bit uniforms
// strictly inside (0, 1).  The step number is read from device memory (the word after the mode list)
// so that a replayed graph draws fresh noise every step.
struct Thermo {
  int on = 0;
  int f32 = 0;                        // mixed form: Box-Muller on 24-bit uniforms in FP32
  double c1 = 1.0, s2 = 0.0;          // e^{-gamma dt}, (1 - c1^2) kB T
  uint64_t seed = 0;
  const int4 *step = nullptr;
};

// X - L floor(X / L), then once more if rounding left X at L.  A step moves a particle by far less
// than L, so the usual case is one addition or subtraction of L (the same result as the floor form,
// which runs only for X beyond [-L, 2L): FP64 division is costly on this GPU)
__device__ __forceinline__ double wrap_periodic(double X, double L) {
  if (X >= 0.0 && X < L) return X;
  if (X >= -L && X < 0.0) {
    X += L;
  } else if (X >= L && X < 2.0 * L) {
    X -= L;
  } else {
    X -= L * floor(X / L);
  }
  if (X >= L) X -= L;
  return X;
}

// The closing half kick (status != nullptr) also checks the step's forces and charges: a non-finite
// F of this thread's ion or Q of the electrode site with the same index raises the context's flag.
// One thread per (ion, component): the FP64 update of a component is a short dependent chain, and
// on this GPU an FP64 warp instruction holds its sub-partition for many cycles, so three threads
// per ion shorten the kernel's critical path.  blockIdx.y is the component (0 x, 1 y, 2 z).  Each
// thread draws the same Philox words for its ion and forms its own one of the three normals (the
// arithmetic of each component is unchanged: the results are the same bits as one thread per ion).
__global__ void k_kick_drift(int64_t n, double *__restrict__ x, double *__restrict__ y, double *__restrict__ z,
                             double *__restrict__ vx, double *__restrict__ vy, double *__restrict__ vz,
                             const double *__restrict__ F, const double *__restrict__ minv, double fac, double dt,
                             int drift, double Lx, double Ly, Thermo th, double3 invL, uint64_t *__restrict__ iu,
                             int64_t ne, const double *__restrict__ Q, int *__restrict__ status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int d = blockIdx.y;
  if (d == 0 && status && i < ne && !isfinite(Q[i])) *(volatile int *)(status + kStatNonFiniteQ) = 1;
  if (i >= n) return;
  double *pos = d == 0 ? x : (d == 1 ? y : z);
  double *vel = d == 0 ? vx : (d == 1 ? vy : vz);
  const double w = fac * minv[i];
  const double f = F[d * n + i];
  if (status && !isfinite(f)) *(volatile int *)(status + kStatNonFiniteF) = 1;
  double a = fma(w, f, vel[i]);
  if (th.on) {
    const int4 st = *th.step;
    const uint64_t step = (uint64_t)(uint32_t)st.x | ((uint64_t)(uint32_t)st.y << 32);
    uint64_t wd[4];
    philox4x64_dev(step, (uint64_t)i, 0, 0, th.seed, 0x4C414E47ull, wd);
    // sigma_i times a standard normal: words 0 and 1 give the x and y normals (Box-Muller, cos and
    // sin), words 2 and 3 the z normal (cos)
    const int wr = d < 2 ? 0 : 2;
    double g;
    if (th.f32) {
      // the top 24 bits of the words as FP32 uniforms in (0, 1): the noise needs no more than FP32
      // and every FP64 instruction is costly on this GPU
      const float u0 = ((float)(uint32_t)(wd[wr] >> 40) + 0.5f) * 0x1.0p-24f;
      const float u1 = ((float)(uint32_t)(wd[wr + 1] >> 40) + 0.5f) * 0x1.0p-24f;
      const float r = sqrtf(-2.f * logf(u0));
      float sn, cs;
      sincospif(2.f * u1, &sn, &cs);
      const float sg = sqrtf((float)th.s2 * (float)minv[i]);
      g = (double)(sg * (r * (d == 1 ? sn : cs)));
    } else {
      const double u0 = ((double)(wd[wr] >> 11) + 0.5) * 0x1.0p-53;
      const double u1 = ((double)(wd[wr + 1] >> 11) + 0.5) * 0x1.0p-53;
      const double r = sqrt(-2.0 * log(u0));
      double sn, cs;
      sincospi(2.0 * u1, &sn, &cs);
      const double sig = sqrt(th.s2 * minv[i]);
      g = sig * (r * (d == 1 ? sn : cs));
    }
    a = fma(th.c1, a, g);
  }
  vel[i] = a;
  if (drift) {
    double X = fma(dt, a, pos[i]);
    if (d < 2) X = wrap_periodic(X, d == 0 ? Lx : Ly);
    pos[i] = X;
    // the new position's fixed-point phase coordinate, once per step for the ion structure factor
    iu[d * n + i] = to_turns64(X, d == 0 ? invL.x : (d == 1 ? invL.y : invL.z));
  }
}

__global__ void k_sd_move(int64_t n, double *__restrict__ x, double *__restrict__ y, double *__restrict__ z,
                          const double *__restrict__ F, double a, double dmax, double Lx, double Ly) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double fx = F[i], fy = F[n + i], fz = F[2 * n + i];
  double fn = sqrt(fx * fx + fy * fy + fz * fz);
  double s = fn > 0.0 ? fmin(a, dmax / fn) : 0.0;
  if (!isfinite(fn)) {
    // a force that overflowed (sites on top of each other): the full capped step along the signs of
    // its infinite components; NaN components do not move
    fx = isinf(fx) ? copysign(1.0, fx) : 0.0;
    fy = isinf(fy) ? copysign(1.0, fy) : 0.0;
    fz = isinf(fz) ? copysign(1.0, fz) : 0.0;
    fn = sqrt(fx * fx + fy * fy + fz * fz);
    s = fn > 0.0 ? dmax / fn : 0.0;
  }
  double X = fma(s, fx, x[i]), Y = fma(s, fy, y[i]);
  X -= Lx * floor(X / Lx);
  Y -= Ly * floor(Y / Ly);
  if (X >= Lx) X -= Lx;
  if (Y >= Ly) Y -= Ly;
  x[i] = X;
  y[i] = Y;
  z[i] = fma(s, fz, z[i]);
}

void steepest_descent_move(srbe_ctx *c, double a, double dmax) {
  if (c->ni == 0) return;
  k_sd_move<<<blocks_for(c->ni, 256), 256, 0, c->stream>>>(c->ni, c->x.p, c->y.p, c->z.p, c->F.p, a, dmax, c->L[0],
                                                          c->L[1]);
  c->launches++;
  SRBE_CUDA(cudaGetLastError());
}

void integrate_kick_drift(srbe_ctx *c, double fac_kick, bool drift) {
  if (c->ni == 0) return;
  Thermo th;
  if (!drift && c->lang_gamma > 0.0) {
    // the closing half kick of a step also applies the thermostat; the step number sits in dm[K]
    SRBE_REQUIRE(c->dm.p && c->dm.cap > (size_t)c->K, SRBE_ESTATE, "mode list without its step word");
    th.on = 1;
    th.f32 = c->precision == SRBE_MIXED ? 1 : 0;
    th.c1 = std::exp(-c->lang_gamma * c->dt);
    th.s2 = (1.0 - th.c1 * th.c1) * kBoltz * c->lang_T;
    th.seed = c->lang_seed;
    th.step = c->dm.p + c->K;
  }
  uint64_t *iu = drift ? c->iu.ensure((size_t)3 * c->ni) : nullptr;
  const double3 invL = make_double3(1.0 / c->L[0], 1.0 / c->L[1], 1.0 / c->L[2]);
  // the closing kick checks the step's forces and charges (one thread per ion and per site)
  const int64_t ne = drift ? 0 : c->ne;
  const int64_t nt = std::max<int64_t>(c->ni, ne);
  // 64-thread blocks, one grid row per component: the FP64 arithmetic spreads over every SM even for
  // a few thousand ions
  k_kick_drift<<<dim3(blocks_for(nt, 64), 3), 64, 0, c->stream>>>(c->ni, c->x.p, c->y.p, c->z.p, c->vx.p, c->vy.p,
                                                         c->vz.p, c->F.p, c->minv.p, fac_kick, c->dt,
                                                         drift ? 1 : 0, c->L[0], c->L[1], th, invL, iu, ne, c->Q.p,
                                                         drift ? nullptr : c->d_status);
  c->launches++;
  SRBE_CUDA(cudaGetLastError());
}

// non-finite check of the forces [3][nF / 3] and charges [nQ] of a pass outside the MD step
__global__ void k_check_finite(int64_t nF, const double *__restrict__ F, int64_t nQ, const double *__restrict__ Q,
                               int *__restrict__ status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nF || i < nQ; i += stride) {
    if (i < nF && !isfinite(F[i])) *(volatile int *)(status + kStatNonFiniteF) = 1;
    if (i < nQ && !isfinite(Q[i])) *(volatile int *)(status + kStatNonFiniteQ) = 1;
  }
}

void check_finite(srbe_ctx *c, bool forces, bool charges) {
  const int64_t nF = forces ? 3 * c->ni : 0, nQ = charges ? c->ne : 0;
  if (nF == 0 && nQ == 0) return;
  const unsigned nb = std::min<unsigned>(blocks_for(std::max(nF, nQ), 256), 304);
  k_check_finite<<<nb, 256, 0, c->stream>>>(nF, c->F.p, nQ, c->Q.p, c->d_status);
  c->launches++;
  SRBE_CUDA(cudaGetLastError());
}

}  // namespace srbe
