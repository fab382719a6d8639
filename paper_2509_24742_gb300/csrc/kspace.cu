// Fourier-space part of SRBE: structure factors S(k) = sum_j w_j exp(i k . r_j) (Eq. 15) over a
// weighted mode list (the deterministic set I and the P sampled modes, Eqs. 24-25), the
// far-field electrode right-hand side b_F (Eq. 24), and the reductions that finish S.
//
// Layout: positions are SoA doubles; the mode list is int4 (m_x, m_y, m_z, 0) plus one double
// weight c_k per mode.  Phases are exact 64-bit fixed-point turns (srbe_internal.cuh).
//
// S(k) is computed in two deterministic passes: each block sums a fixed chunk of particles for
// a tile of 128 modes (one mode per thread, particles staged in shared memory), writing one
// partial per (chunk, mode); a second kernel adds the partials in chunk order.
#include "srbe_internal.cuh"

namespace srbe {

constexpr int kSfThreads = 128;              // 4 warps; a block covers 32 modes x a particle chunk
constexpr int kSfMaxChunks = 512;

// FP32 Kahan-compensated accumulator (the mixed form's "compensated sums").
struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Double-float (hi, lo) addition by Knuth's TwoSum, FP32 instructions only (~2^-48 relative): the
// mixed form combines its compensated partial sums this way, since on this GPU each FP64 addition
// holds a sub-partition's FP64 pipe for many cycles and the combines form a serial chain.
__device__ __forceinline__ float2 df_sum(float2 a, float2 b) {
  const float s = a.x + b.x, bb = s - a.x, err = (a.x - (s - bb)) + (b.x - bb);
  const float lo = err + a.y + b.y;
  const float h = s + lo;
  return make_float2(h, lo - (h - s));
}

// Finishes mode k (k < K) or, for k == K, the dipole: lanes take chunks lane, lane + 32, ..., then a
// butterfly sum (every lane ends with the same value); lane 0 writes S (+ S_add) and the gather
// coefficients, or the dipole into scal[mslot].  Partials are read through L2 (__ldcg): in the
// fused form they were written by other blocks of the same launch.
struct SfFinish {
  int K, nchunk;
  const double2 *partial;
  const double *mpart;
  double2 *S;
  const double2 *S_add;
  double *scal;
  int mslot;
  const double *cw;
  double2 *coef;
  float2 *coef32;
  int swap;
};

__device__ __forceinline__ void sf_finish(const SfFinish &f, int k, int lane) {
  double re = 0.0, im = 0.0;
  if (k < f.K) {
    for (int c = lane; c < f.nchunk; c += 32) {
      const double2 p = __ldcg(f.partial + (int64_t)c * f.K + k);
      re += p.x;
      im += p.y;
    }
  } else {
    for (int c = lane; c < f.nchunk; c += 32) re += __ldcg(f.mpart + c);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) {
    if (k < f.K) {
      if (f.S_add) {
        re += f.S_add[k].x;
        im += f.S_add[k].y;
      }
      f.S[k] = make_double2(re, im);
      if (f.coef) {
        // per-mode coefficients of the gathers: (c Re S, c Im S) for b, (c Im S, c Re S) for forces
        const double c = f.cw[k];
        const double2 v = f.swap ? make_double2(c * im, c * re) : make_double2(c * re, c * im);
        f.coef[k] = v;
        f.coef32[k] = make_float2((float)v.x, (float)v.y);
      }
    } else {
      f.scal[f.mslot] = re;
    }
  }
}

// partial[c][k] = sum over the particles of chunk c of w_j exp(i k . r_j).  Lane = mode (32 per
// block in y), the four warps take every fourth particle of each staged batch of 128, and the
// four warp sums are added in warp order.  Blocks with blockIdx.y == 0 also sum w z per chunk.
template <bool F32>
__global__ void __launch_bounds__(kSfThreads)
k_sfac_partial(int64_t n, const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
               const uint64_t *__restrict__ u, const double *__restrict__ w, const float *__restrict__ w32, int K,
               const int4 *__restrict__ modes, double3 invL,
               const double2 *__restrict__ tab, int64_t chunk, double2 *__restrict__ partial,
               double *__restrict__ mpart, SfFinish fin, int *__restrict__ done) {
  __shared__ uint64_t su[3][kSfThreads];
  __shared__ double sw[kSfThreads];
  __shared__ float sw32[kSfThreads];          // the weights in FP32 (mixed form), converted once
  __shared__ double2 red[4][32];
  __shared__ double mred[kSfThreads];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int kidx = blockIdx.y * 32 + lane;
  const int4 m = kidx < K ? modes[kidx] : make_int4(0, 0, 0, 0);
  const int64_t i0 = (int64_t)blockIdx.x * chunk;
  const int64_t i1 = min(n, i0 + chunk);
  double are = 0.0, aim = 0.0, mz = 0.0;
  KahanF fre, fim;
  for (int64_t base = i0; base < i1; base += kSfThreads) {
    __syncthreads();
    const int64_t i = base + t;
    if (i < i1) {
      if (u) {
        su[0][t] = u[i];
        su[1][t] = u[n + i];
        su[2][t] = u[2 * n + i];
      } else {
        su[0][t] = to_turns64(x[i], invL.x);
        su[1][t] = to_turns64(y[i], invL.y);
        su[2][t] = to_turns64(z[i], invL.z);
      }
      // the mixed form reads the weights' FP32 copy when there is one: an FP64 conversion per
      // particle would keep this GPU's scarce FP64 pipe busy
      if (!F32) sw[t] = w[i];
      else sw32[t] = w32 ? w32[i] : (float)w[i];
      if (blockIdx.y == 0) mz = fma(w[i], z[i], mz);
    }
    __syncthreads();
    const int cnt = (int)min((int64_t)kSfThreads, i1 - base);
    if (!F32) {
      for (int j = warp; j < cnt; j += 4) {
        double c, s;
        sincos_turns(phase64(m, su[0][j], su[1][j], su[2][j]), tab, c, s);
        are = fma(sw[j], c, are);
        aim = fma(sw[j], s, aim);
      }
    } else {
      for (int j = warp; j < cnt; j += 4) {
        const uint32_t th = (uint32_t)m.x * (uint32_t)(su[0][j] >> 32) + (uint32_t)m.y * (uint32_t)(su[1][j] >> 32) +
                            (uint32_t)m.z * (uint32_t)(su[2][j] >> 32);
        float c, s;
        sincos_turns32(th, c, s);
        const float wf = sw32[j];
        fre.add(wf * c);
        fim.add(wf * s);
      }
    }
  }
  // the mixed form keeps each Kahan sum with its compensation as a double-float (s, -c) and adds the
  // four warps' sums in warp order with FP32 instructions; its partials are (re hi, re lo, im hi,
  // im lo) in the same 16 bytes as the FP64 form's (re, im)
  __shared__ float4 red32[4][32];
  if (F32) red32[warp][lane] = make_float4(fre.s, -fre.c, fim.s, -fim.c);
  else red[warp][lane] = make_double2(are, aim);
  __syncthreads();
  if (warp == 0 && kidx < K) {
    if (F32) {
      float2 re = make_float2(red32[0][lane].x, red32[0][lane].y), im = make_float2(red32[0][lane].z, red32[0][lane].w);
#pragma unroll
      for (int q = 1; q < 4; ++q) {
        re = df_sum(re, make_float2(red32[q][lane].x, red32[q][lane].y));
        im = df_sum(im, make_float2(red32[q][lane].z, red32[q][lane].w));
      }
      reinterpret_cast<float4 *>(partial)[(int64_t)blockIdx.x * K + kidx] = make_float4(re.x, re.y, im.x, im.y);
    } else {
      double2 a = red[0][lane];
#pragma unroll
      for (int q = 1; q < 4; ++q) {
        a.x += red[q][lane].x;
        a.y += red[q][lane].y;
      }
      partial[(int64_t)blockIdx.x * K + kidx] = a;
    }
  }
  if (blockIdx.y == 0) {
    // fixed-order block reduction of sum w z
    mred[t] = mz;
    __syncthreads();
    for (int s = kSfThreads / 2; s > 0; s >>= 1) {
      if (t < s) mred[t] += mred[t + s];
      __syncthreads();
    }
    if (t == 0) mpart[blockIdx.x] = mred[0];
  }
  // the last block to finish a mode tile adds that tile's partials (the same order as
  // k_sfac_reduce, so the result does not depend on which block comes last) and re-arms the counter
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(&done[blockIdx.y], 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // lane = mode of the tile, warp w takes chunks w, w + 4, ... (coalesced 512-byte rows of the
  // partials), then the four warp sums are added in warp order
  // the mode's sum over the chunks, in chunk order (lane = mode, warp w takes chunks w, w + 4, ...,
  // then the four warp sums in warp order), held by warp 0 as (re, im)
  double re = 0.0, im = 0.0;
  if (F32) {
    // double-float sums, FP32 instructions only; one conversion to FP64 per mode
    float2 dre = make_float2(0.f, 0.f), dim = make_float2(0.f, 0.f);
    if (kidx < K) {
      const float4 *p32 = reinterpret_cast<const float4 *>(partial);
      int c = warp;
      for (; c + 28 < fin.nchunk; c += 32) {
        float4 p[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) p[u] = __ldcg(p32 + (int64_t)(c + 4 * u) * K + kidx);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          dre = df_sum(dre, make_float2(p[u].x, p[u].y));
          dim = df_sum(dim, make_float2(p[u].z, p[u].w));
        }
      }
      for (; c < fin.nchunk; c += 4) {
        const float4 p = __ldcg(p32 + (int64_t)c * K + kidx);
        dre = df_sum(dre, make_float2(p.x, p.y));
        dim = df_sum(dim, make_float2(p.z, p.w));
      }
    }
    red32[warp][lane] = make_float4(dre.x, dre.y, dim.x, dim.y);
    __syncthreads();
    if (warp == 0 && kidx < K) {
      float2 sre = make_float2(red32[0][lane].x, red32[0][lane].y);
      float2 sim = make_float2(red32[0][lane].z, red32[0][lane].w);
#pragma unroll
      for (int q = 1; q < 4; ++q) {
        sre = df_sum(sre, make_float2(red32[q][lane].x, red32[q][lane].y));
        sim = df_sum(sim, make_float2(red32[q][lane].z, red32[q][lane].w));
      }
      re = (double)sre.x + (double)sre.y;
      im = (double)sim.x + (double)sim.y;
    }
  } else {
    double2 acc = make_double2(0.0, 0.0);
    if (kidx < K) {
      // eight loads in flight per thread before the adds (same order of additions)
      int c = warp;
      for (; c + 28 < fin.nchunk; c += 32) {
        double2 p[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) p[u] = __ldcg(partial + (int64_t)(c + 4 * u) * K + kidx);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          acc.x += p[u].x;
          acc.y += p[u].y;
        }
      }
      for (; c < fin.nchunk; c += 4) {
        const double2 p = __ldcg(partial + (int64_t)c * K + kidx);
        acc.x += p.x;
        acc.y += p.y;
      }
    }
    red[warp][lane] = acc;
    __syncthreads();
    if (warp == 0 && kidx < K) {
      re = red[0][lane].x;
      im = red[0][lane].y;
#pragma unroll
      for (int q = 1; q < 4; ++q) {
        re += red[q][lane].x;
        im += red[q][lane].y;
      }
    }
  }
  if (warp == 0 && kidx < K) {
    if (fin.S_add) {
      re += fin.S_add[kidx].x;
      im += fin.S_add[kidx].y;
    }
    fin.S[kidx] = make_double2(re, im);
    if (fin.coef) {
      const double c = fin.cw[kidx];
      const double2 v = fin.swap ? make_double2(c * im, c * re) : make_double2(c * re, c * im);
      fin.coef[kidx] = v;
      fin.coef32[kidx] = make_float2((float)v.x, (float)v.y);
    }
  }
  if (blockIdx.y == 0 && warp == 1) sf_finish(fin, K, lane);     // the dipole partials
  if (t == 0) done[blockIdx.y] = 0;
}

// S[k] = sum over chunks of the partials (+ S_add[k]): one warp per mode, lanes take chunks
// lane, lane + 32, ..., then a butterfly sum (every lane ends with the same value).  Warp K sums
// the dipole partials into scal[mslot].
__global__ void k_sfac_reduce(SfFinish f) {
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (k > f.K) return;
  sf_finish(f, k, threadIdx.x & 31);
}

// chunking of the particle sum (the kernel's tile along the particles): whole 128-particle
// batches, at most kSfMaxChunks chunks.  A chunk spans as many batches (up to 8) as keeps at least
// `occ` blocks per SM: each block ends with a few FP64 operations (the partial's compensation and the
// warp sums), which cost 64 cycles of a sub-partition each on this GPU, so longer chunks spread them
// over more particles, while shorter ones give more blocks to hide latency with.  occ is a context
// setting (default 8) that srbe_autotune_tiles / srbe_batch_autotune_tiles choose by timing.
int64_t sfac_chunks(int64_t n, int K, int occ, int64_t *chunk) {
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    SRBE_CUDA(cudaGetDevice(&dev));
    SRBE_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  }
  if (n <= 0) {
    *chunk = kSfThreads;
    return 0;
  }
  const int64_t min_blocks = (int64_t)std::max(1, occ) * nsm;
  const int64_t ktiles = std::max(1, (K + 31) / 32);
  const int64_t batches = (n + kSfThreads - 1) / kSfThreads;
  int64_t per = (batches + kSfMaxChunks - 1) / kSfMaxChunks;
  while (per < 8 && ((batches + 2 * per - 1) / (2 * per)) * ktiles >= min_blocks) per *= 2;
  *chunk = per * kSfThreads;
  return (n + *chunk - 1) / *chunk;
}

void structure_factor(srbe_ctx *c, int64_t n, const double *x, const double *y, const double *z, const double *w,
                      double2 *S, const double2 *S_add, int mslot, int coef_mode, const uint64_t *u,
                      const float *w32) {
  const int K = c->K;
  const int ktiles = std::max(1, (K + 31) / 32);
  int64_t chunk;
  const int64_t nchunk = sfac_chunks(n, K, c->sf_occ, &chunk);
  SRBE_REQUIRE(c->partial.cap >= (size_t)std::max<int64_t>(nchunk * K, 1) &&
                   c->mpart.cap >= (size_t)std::max<int64_t>(nchunk, 1),
               SRBE_ESTATE, "scratch buffers not reserved for this size");
  const double3 invL = make_double3(1.0 / c->L[0], 1.0 / c->L[1], 1.0 / c->L[2]);
  SfFinish f{K, (int)nchunk, c->partial.p, c->mpart.p, S, S_add, c->scal.p, mslot, c->dc.p,
             coef_mode >= 0 ? c->coef.p : nullptr, c->coef32.p, coef_mode > 0 ? 1 : 0};
  if (nchunk > 0) {
    SRBE_REQUIRE(c->sfdone.cap >= (size_t)ktiles, SRBE_ESTATE, "tile counters not reserved for this size");
    dim3 grid((unsigned)nchunk, (unsigned)ktiles);
    if (c->precision == SRBE_MIXED)
      k_sfac_partial<true><<<grid, kSfThreads, 0, c->stream>>>(n, x, y, z, u, w, w32, K, c->dm.p, invL, c->tab.p,
                                                               chunk, c->partial.p, c->mpart.p, f, c->sfdone.p);
    else
      k_sfac_partial<false><<<grid, kSfThreads, 0, c->stream>>>(n, x, y, z, u, w, nullptr, K, c->dm.p, invL,
                                                                c->tab.p, chunk, c->partial.p, c->mpart.p, f,
                                                                c->sfdone.p);
    c->launches++;
    c->mode_evals += n * (int64_t)K;
  } else {
    k_sfac_reduce<<<blocks_for((int64_t)(K + 1) * 32, 256), 256, 0, c->stream>>>(f);
    c->launches++;
  }
  SRBE_CUDA(cudaGetLastError());
}

}  // namespace srbe
