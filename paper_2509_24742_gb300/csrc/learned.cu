// Learned warm start for the constant-potential solve (the learned form): a per-electrode-site MLP
// (80 -> 128 -> 128 -> 1, SiLU; FP32 parameters, forward GEMMs on the tensor cores) maps local
// electrolyte descriptors to the unprojected solution
// y = A^-1 (dpsi d + b) of the charge update (Eqs. 9-10), which seeds the PCG iteration.
//
// Descriptors of site j (80 floats):
//   0..31   sum over ions with q > 0 within rc of  |q| exp(-(r - mu_b)^2 / (2 s^2)), mu_b = 0.25 + b / 31 nm
//   32..63  the same for ions with q < 0
//   64..79  Re, Im of exp(-i k_z Z_j) S1(k_z) for k_z = 2 pi m / L_z, m = 1..8 (the lowest k_z modes
//           that the symmetry-preserving set I keeps, Eqs. 15 and 24)
// Inputs and the target are standardised with the training set's mean and spread, which are part of
// the parameter vector.  Training minimises the mean squared error with AdamW; the per-site
// backward pass accumulates each block's gradient in shared memory (every thread owns its rows, so
// the sum order is fixed) and a second kernel adds the block gradients in block order and applies
// the AdamW update.
#include "srbe_internal.cuh"
#include "tc.cuh"

namespace srbe {

constexpr int kIn = 80, kH = 128;
constexpr int kNbasis = 32, kNlow = 8;
constexpr float kRbfSigma = 0.035f;
// parameter layout
constexpr int oW1 = 0, oB1 = oW1 + kH * kIn, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH, oB3 = oW3 + kH,
              oXm = oB3 + 1, oXs = oXm + kIn, oYm = oXs + kIn, oYs = oYm + 1, kNparam = oYs + 1;
constexpr int kNtrain = oXm;     // trainable entries come first

__device__ __forceinline__ float silu(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
  const float s = 1.f / (1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

// S_low[m] = sum_i q_i exp(i 2 pi m z_i / L_z), m = 1..8, one block, fixed order
__global__ void k_low_modes(int64_t n, const double *__restrict__ z, const double *__restrict__ q, double invLz,
                            double2 *__restrict__ S) {
  __shared__ double red[2 * kNlow][256];
  const int t = threadIdx.x;
  double a[2 * kNlow];
  for (int m = 0; m < 2 * kNlow; ++m) a[m] = 0.0;
  for (int64_t i = t; i < n; i += 256) {
    const uint64_t u = to_turns64(z[i], invLz);
    for (int m = 0; m < kNlow; ++m) {
      float c, s;
      sincos_turns32((uint32_t)((u * (uint64_t)(m + 1)) >> 32), c, s);
      a[2 * m] += q[i] * c;
      a[2 * m + 1] += q[i] * s;
    }
  }
  for (int m = 0; m < 2 * kNlow; ++m) red[m][t] = a[m];
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (t < s)
      for (int m = 0; m < 2 * kNlow; ++m) red[m][t] += red[m][t + s];
    __syncthreads();
  }
  if (t < kNlow) S[t] = make_double2(red[2 * t][0], red[2 * t + 1][0]);
}

// descriptors, one warp per electrode site; lane b owns basis function b
__global__ void __launch_bounds__(256)
k_descriptors(int64_t ne, const double *__restrict__ ex, const double *__restrict__ ey, const double *__restrict__ ez,
              const float4 *__restrict__ ion_pf, const int32_t *__restrict__ ei, const int32_t *__restrict__ ei_n,
              int cap, float Lx, float Ly, float rc2, const double2 *__restrict__ Slow, double invLz,
              float *__restrict__ D) {
  const int lane = threadIdx.x & 31;
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (j >= ne) return;
  const float X = (float)ex[j], Y = (float)ey[j], Z = (float)ez[j];
  const float mu = 0.25f + lane * (1.0f / 31.0f);
  const float inv2s2 = 1.0f / (2.0f * kRbfSigma * kRbfSigma);
  float pos = 0.f, neg = 0.f;
  const int cnt = min(ei_n[j], cap);
  for (int base = 0; base < cnt; base += 32) {
    const int k = base + lane;
    float r = 0.f, qv = 0.f;
    if (k < cnt) {
      const int32_t e = ei[j * (int64_t)cap + k];
      const int idx = e & 0x7fffff, ix = ((e >> 24) & 15) - 8, iy = ((unsigned)e >> 28) - 8;
      const float4 o = ion_pf[idx];
      const float dx = X - (o.x + ix * Lx), dy = Y - (o.y + iy * Ly), dz = Z - o.z;
      const float r2 = dx * dx + dy * dy + dz * dz;
      if (r2 < rc2) {
        r = sqrtf(r2);
        qv = o.w;
      }
    }
    const int m = min(32, cnt - base);
    for (int l = 0; l < m; ++l) {
      const float rl = __shfl_sync(0xffffffffu, r, l), ql = __shfl_sync(0xffffffffu, qv, l);
      if (ql == 0.f) continue;
      const float g = fabsf(ql) * __expf(-(rl - mu) * (rl - mu) * inv2s2);
      if (ql > 0.f) pos += g;
      else neg += g;
    }
  }
  float *row = D + j * (int64_t)kIn;
  row[lane] = pos;
  row[32 + lane] = neg;
  if (lane < kNlow) {
    // exp(-i k Z) S(k) with k = 2 pi (m + 1) / L_z
    const uint64_t u = to_turns64(ez[j], invLz);
    float c, s;
    sincos_turns32((uint32_t)((u * (uint64_t)(lane + 1)) >> 32), c, s);
    const double2 S = Slow[lane];
    row[64 + 2 * lane] = (float)(c * S.x + s * S.y);
    row[64 + 2 * lane + 1] = (float)(c * S.y - s * S.x);
  }
}

// ------------------------------------------------------------------------------------------------
// forward pass on the tensor cores (tcgen05): 128 rows per tile, Z1 = X W1^T and Z2 = H1 W2^T as
// kind::f16 MMAs into tensor memory with FP32 accumulation.  Every operand is split into BF16
// (hi, lo) and each product taken as hi hi + hi lo + lo hi, which keeps about 16 significand bits
// (the scalar FP32 path keeps 24; the difference stays below 1e-5 of the output here).  One CTA of
// 16 warps per SM, persistent over tiles; in the bias + SiLU epilogues the four warps of a
// tensor-memory lane quarter split the 128 columns of their 32 rows, and thread 0 issues the MMAs.
// ------------------------------------------------------------------------------------------------
constexpr int kTcK1 = kIn / tc::kKstep;    // 5 K steps of layer 1
constexpr int kTcK2 = kH / tc::kKstep;     // 8 K steps of layer 2
constexpr size_t kTcSmem = (size_t)(2 * kTcK1 + 2 * kTcK2) * 2 * tc::kBlockBytes;   // 208 KB
constexpr int kTcPolls = 1 << 20;          // bounded mbarrier waits
static_assert(kIn % tc::kKstep == 0 && kH == tc::kRows, "MLP sizes must match the MMA tiles");

constexpr int kTcThreads = 512;            // 16 warps: 4 per tensor-memory lane quarter
constexpr int kTcGroups = kTcThreads / 128; // column groups of 32 per row in the epilogues

__global__ void __launch_bounds__(kTcThreads, 1)
k_mlp_forward_tc(int64_t n, const float *__restrict__ D, const float *__restrict__ P, float *__restrict__ out,
                 double *__restrict__ out_y, int *__restrict__ status) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __nv_bfloat16 *w1h = reinterpret_cast<__nv_bfloat16 *>(smem);
  __nv_bfloat16 *w1l = w1h + kTcK1 * tc::kBlockElems, *w2h = w1l + kTcK1 * tc::kBlockElems;
  __nv_bfloat16 *w2l = w2h + kTcK2 * tc::kBlockElems, *xh = w2l + kTcK2 * tc::kBlockElems;
  __nv_bfloat16 *xl = xh + kTcK1 * tc::kBlockElems, *hh = xl + kTcK1 * tc::kBlockElems;
  __nv_bfloat16 *hl = hh + kTcK2 * tc::kBlockElems;
  __shared__ float sb1[kH], sb2[kH], sw3[kH], sxm[kIn], sxs[kIn];
  __shared__ float part[kTcGroups][128];       // the output's partial dot products per column group
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tbase;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  // warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (rows of the tile) and columns 32 (w / 4) .. + 31
  const int quarter = warp & 3, grp = warp >> 2, row_t = 32 * quarter + lane, c0 = 32 * grp;
  for (int i = t; i < kH * kIn; i += kTcThreads) {
    const int h = i / kIn, k = i - h * kIn;
    tc::split_bf16(P[oW1 + i], w1h[tc::off(h, k)], w1l[tc::off(h, k)]);
  }
  for (int i = t; i < kH * kH; i += kTcThreads) {
    const int h = i / kH, k = i - h * kH;
    tc::split_bf16(P[oW2 + i], w2h[tc::off(h, k)], w2l[tc::off(h, k)]);
  }
  if (t < kH) {
    sb1[t] = P[oB1 + t];
    sb2[t] = P[oB2 + t];
    sw3[t] = P[oW3 + t];
  }
  if (t < kIn) {
    sxm[t] = P[oXm + t];
    sxs[t] = P[oXs + t];
  }
  const float b3 = P[oB3], ym = P[oYm], ys = P[oYs];
  if (t == 0) tc::mbar_init(&mbar, 1);
  if (warp == 0) tc::tmem_alloc(&tbase, 256);
  tc::fence_async_smem();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t d1 = tbase, d2 = tbase + 128, lanes = (uint32_t)(32 * quarter) << 16;
  const uint32_t idesc = tc::idesc_bf16(128, 128);
  const int64_t ntiles = (n + 127) / 128;
  uint32_t phase = 0;
  bool fail = false;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t row0 = tile * 128;
    // standardised inputs of the tile (rows beyond n are zero): row row_t, 8-wide chunks grp,
    // grp + 4, grp + 8 (16-byte loads and stores)
    {
      const bool live = row0 + row_t < n;
      const float4 *src = reinterpret_cast<const float4 *>(D + (row0 + row_t) * kIn);
      for (int ch = grp; ch < kIn / 8; ch += kTcGroups) {
        const float4 q0 = live ? __ldg(src + 2 * ch) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 q1 = live ? __ldg(src + 2 * ch + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
        float v[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = live ? (v[j] - sxm[8 * ch + j]) / sxs[8 * ch + j] : 0.f;
        tc::store8_split(xh, xl, row_t, 8 * ch, v);
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) {
      for (int s = 0; s < kTcK1; ++s) {
        const uint64_t ah = tc::block_desc(xh + s * tc::kBlockElems), al = tc::block_desc(xl + s * tc::kBlockElems);
        const uint64_t bh = tc::block_desc(w1h + s * tc::kBlockElems), bl = tc::block_desc(w1l + s * tc::kBlockElems);
        tc::mma_bf16(d1, ah, bh, idesc, s > 0);
        tc::mma_bf16(d1, ah, bl, idesc, true);
        tc::mma_bf16(d1, al, bh, idesc, true);
      }
      tc::commit(&mbar);
    }
    fail = __syncthreads_or(!tc::mbar_wait(&mbar, phase, kTcPolls)) != 0;
    if (fail) break;
    phase ^= 1u;
    tc::fence_after_sync();
    // H1 = SiLU(Z1 + b1) for row row_t, columns c0 .. c0 + 31, split into the layer-2 operand
    {
      float v[32];
      tc::ld32(d1 + lanes + (uint32_t)c0, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = silu(v[j] + sb1[c0 + j]);
#pragma unroll
      for (int g = 0; g < 4; ++g) tc::store8_split(hh, hl, row_t, c0 + 8 * g, v + 8 * g);
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (t == 0) {
      for (int s = 0; s < kTcK2; ++s) {
        const uint64_t ah = tc::block_desc(hh + s * tc::kBlockElems), al = tc::block_desc(hl + s * tc::kBlockElems);
        const uint64_t bh = tc::block_desc(w2h + s * tc::kBlockElems), bl = tc::block_desc(w2l + s * tc::kBlockElems);
        tc::mma_bf16(d2, ah, bh, idesc, s > 0);
        tc::mma_bf16(d2, ah, bl, idesc, true);
        tc::mma_bf16(d2, al, bh, idesc, true);
      }
      tc::commit(&mbar);
    }
    fail = __syncthreads_or(!tc::mbar_wait(&mbar, phase, kTcPolls)) != 0;
    if (fail) break;
    phase ^= 1u;
    tc::fence_after_sync();
    // output = W3 . SiLU(Z2 + b2) + b3: partial sums per column group, added in group order
    {
      float v[32];
      tc::ld32(d2 + lanes + (uint32_t)c0, v);
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < 32; ++j) acc = fmaf(sw3[c0 + j], silu(v[j] + sb2[c0 + j]), acc);
      part[grp][row_t] = acc;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (t < 128) {
      float acc = part[0][t];
#pragma unroll
      for (int g = 1; g < kTcGroups; ++g) acc += part[g][t];
      const int64_t row = row0 + t;
      if (row < n) {
        const float y = (acc + b3) * ys + ym;
        if (out) out[row] = y;
        if (out_y) out_y[row] = (double)y;
      }
    }
  }
  if (fail) {
    // an MMA did not complete within the limit: raise the flag, give it one more bounded wait, then
    // release the tensor memory and return
    if (t == 0) *(volatile int *)(status + kStatTimeout) = 1;
    tc::mbar_wait(&mbar, phase, kTcPolls);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tbase, 256);
}

// forward + backward of the standardised MSE loss over rows [blockIdx.x * chunk, ...); the block's
// gradient (trainable entries) goes to gpart[blockIdx.x][kNtrain], its loss to lpart[blockIdx.x]
__global__ void __launch_bounds__(kH)
k_mlp_backward(int64_t n, int64_t chunk, const int32_t *__restrict__ rows, const float *__restrict__ D,
               const float *__restrict__ T, const float *__restrict__ P, float inv_n, float *__restrict__ gpart,
               double *__restrict__ lpart) {
  extern __shared__ float g[];            // kNtrain floats
  __shared__ float x[kIn], z1s[kH], h1[kH], dz2[kH], red[kH / 32];
  const int h = threadIdx.x;
  for (int i = h; i < kNtrain; i += kH) g[i] = 0.f;
  double loss = 0.0;
  __syncthreads();
  const int64_t r0 = (int64_t)blockIdx.x * chunk, r1 = min(n, r0 + chunk);
  for (int64_t rr = r0; rr < r1; ++rr) {
    const int64_t row = rows ? rows[rr] : rr;
    if (h < kIn) x[h] = (D[row * kIn + h] - P[oXm + h]) / P[oXs + h];
    __syncthreads();
    float z1 = P[oB1 + h];
    for (int k = 0; k < kIn; ++k) z1 = fmaf(P[oW1 + h * kIn + k], x[k], z1);
    z1s[h] = z1;
    h1[h] = silu(z1);
    __syncthreads();
    float z2 = P[oB2 + h];
    for (int k = 0; k < kH; ++k) z2 = fmaf(P[oW2 + h * kH + k], h1[k], z2);
    const float a2 = silu(z2);
    float v = P[oW3 + h] * a2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((h & 31) == 0) red[h >> 5] = v;
    __syncthreads();
    const float o3 = red[0] + red[1] + red[2] + red[3] + P[oB3];
    const float t = (T[row] - P[oYm]) / P[oYs];
    const float err = o3 - t;
    if (h == 0) loss += (double)err * err;
    const float dout = 2.f * err * inv_n;
    // layer 3
    g[oW3 + h] += dout * a2;
    if (h == 0) g[oB3] += dout;
    const float d2 = dout * P[oW3 + h] * silu_grad(z2);
    dz2[h] = d2;
    // layer 2: thread h owns row h of W2
    for (int k = 0; k < kH; ++k) g[oW2 + h * kH + k] += d2 * h1[k];
    g[oB2 + h] += d2;
    __syncthreads();
    // layer 1: dh1[h] = sum_k W2[k][h] dz2[k]
    float dh1 = 0.f;
    for (int k = 0; k < kH; ++k) dh1 = fmaf(P[oW2 + k * kH + h], dz2[k], dh1);
    const float d1 = dh1 * silu_grad(z1s[h]);
    for (int k = 0; k < kIn; ++k) g[oW1 + h * kIn + k] += d1 * x[k];
    g[oB1 + h] += d1;
    __syncthreads();
  }
  for (int i = h; i < kNtrain; i += kH) gpart[(int64_t)blockIdx.x * kNtrain + i] = g[i];
  if (h == 0) lpart[blockIdx.x] = loss;
}

// sums the block gradients in block order; optionally applies AdamW (step t >= 1)
__global__ void k_mlp_reduce_adamw(int nblk, const float *__restrict__ gpart, float *__restrict__ grad,
                                   float *__restrict__ P, float *__restrict__ m1, float *__restrict__ m2, int t,
                                   float lr, float wd, int apply) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNtrain) return;
  float s = 0.f;
  for (int b = 0; b < nblk; ++b) s += gpart[(int64_t)b * kNtrain + i];
  if (grad) grad[i] = s;
  if (!apply) return;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float a = b1 * m1[i] + (1.f - b1) * s, v = b2 * m2[i] + (1.f - b2) * s * s;
  m1[i] = a;
  m2[i] = v;
  const float ah = a / (1.f - powf(b1, (float)t)), vh = v / (1.f - powf(b2, (float)t));
  P[i] -= lr * (ah / (sqrtf(vh) + eps) + wd * P[i]);
}

// ------------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------------
int mlp_param_count() { return kNparam; }
int mlp_input_width() { return kIn; }

void mlp_descriptors(srbe_ctx *c, float *D_dev) {
  const int64_t ne = c->ne;
  c->mlp.Slow.ensure(kNlow);
  k_low_modes<<<1, 256, 0, c->stream>>>(c->ni, c->z.p, c->q.p, 1.0 / c->L[2], c->mlp.Slow.p);
  const float rc = (float)c->rc;
  k_descriptors<<<blocks_for(ne * 32, 256), 256, 0, c->stream>>>(
      ne, c->ex.p, c->ey.p, c->ez.p, c->icells.pf.p, c->nbr.ei.p, c->nbr.ei_n.p, c->nbr.cap, (float)c->L[0],
      (float)c->L[1], rc * rc, c->mlp.Slow.p, 1.0 / c->L[2], D_dev);
  c->launches += 2;
  SRBE_CUDA(cudaGetLastError());
}

void mlp_forward(srbe_ctx *c, const float *D_dev, int64_t n, float *out_dev, double *out_y_dev) {
  if (n <= 0) return;
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    SRBE_CUDA(cudaGetDevice(&dev));
    SRBE_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    SRBE_CUDA(cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
  }
  const unsigned grid = (unsigned)std::min<int64_t>((n + 127) / 128, nsm);
  k_mlp_forward_tc<<<grid, kTcThreads, kTcSmem, c->stream>>>(n, D_dev, c->mlp.P.p, out_dev, out_y_dev, c->d_status);
  c->launches++;
  SRBE_CUDA(cudaGetLastError());
}

// gradient (and optionally one AdamW step) over rows (all n rows when rows_dev is null)
double mlp_grad_step(srbe_ctx *c, const float *D_dev, const float *T_dev, const int32_t *rows_dev, int64_t n,
                     float *grad_dev, bool apply, float lr, float wd) {
  auto &m = c->mlp;
  const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>(152, (n + 15) / 16));
  const int64_t chunk = (n + nblk - 1) / nblk;
  m.gpart.ensure((size_t)nblk * kNtrain);
  m.lpart.ensure((size_t)nblk);
  const size_t smem = sizeof(float) * kNtrain;
  static bool attr = false;
  if (!attr) {
    SRBE_CUDA(cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  k_mlp_backward<<<nblk, kH, smem, c->stream>>>(n, chunk, rows_dev, D_dev, T_dev, m.P.p, 1.0f / (float)n, m.gpart.p,
                                                m.lpart.p);
  if (apply) m.t++;
  k_mlp_reduce_adamw<<<blocks_for(kNtrain, 256), 256, 0, c->stream>>>(nblk, m.gpart.p, grad_dev, m.P.p, m.m1.p, m.m2.p,
                                                                      m.t, lr, wd, apply ? 1 : 0);
  c->launches += 2;
  SRBE_CUDA(cudaGetLastError());
  std::vector<double> lp(nblk);
  SRBE_CUDA(cudaMemcpyAsync(lp.data(), m.lpart.p, sizeof(double) * nblk, cudaMemcpyDeviceToHost, c->stream));
  SRBE_CUDA(cudaStreamSynchronize(c->stream));
  double l = 0.0;
  for (double v : lp) l += v;
  return l / (double)n;
}

}  // namespace srbe
