// Second stage of the hierarchy (arXiv:2110.13115 Sec. III.C, "finer reconstruction for every
// sample inside all the triggering bins"; Sec. III.E custom kernel), grouped by bin:
// first-stage candidates are bucketed by bin (count, scan, scatter), then one CTA per bin stages
// the k x w window of beta in shared memory once and every warp reconstructs one candidate
// template over the window, z[m] = sum_k conj(a_tk) beta_k[m] in FP32, keeping the arg-max
// (first on ties) when |z| >= rho_II.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace {

__global__ void k_bin_count(const rb_candidate* __restrict__ cand, const unsigned long long* dev_count, int64_t cap,
                            int bin0, int nb, unsigned* __restrict__ count) {
  const int64_t n = (int64_t)min((unsigned long long)cap, *dev_count);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int b = cand[i].bin - bin0;
    if (b >= 0 && b < nb) atomicAdd(count + b, 1u);
  }
}

// Exclusive scan of count[0, nb) into start[0, nb]; count is reset to zero (it becomes the
// per-bin fill cursor). One CTA of 1024 threads, each owning a contiguous range of bins.
__global__ void __launch_bounds__(1024) k_bin_scan(unsigned* __restrict__ count, unsigned* __restrict__ start, int nb) {
  __shared__ unsigned wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (nb + 1023) / 1024;
  const int lo = min(nb, tid * per), hi = min(nb, lo + per);
  unsigned s = 0;
  for (int i = lo; i < hi; ++i) s += count[i];
  unsigned inc = s;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += y;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const unsigned v = wsum[lane];
    unsigned x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, x, off);
      if (lane >= off) x += y;
    }
    wsum[lane] = x - v;
  }
  __syncthreads();
  unsigned base = wsum[warp] + inc - s;
  for (int i = lo; i < hi; ++i) {
    start[i] = base;
    base += count[i];
    count[i] = 0;
  }
  if (tid == 1023) start[nb] = base;  // the last range ends at nb (possibly empty ranges before it)
}

__global__ void k_bin_scatter(const rb_candidate* __restrict__ cand, const unsigned long long* dev_count, int64_t cap,
                              int bin0, int nb, const unsigned* __restrict__ start, unsigned* __restrict__ cursor,
                              rb_candidate* __restrict__ out) {
  const int64_t n = (int64_t)min((unsigned long long)cap, *dev_count);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const rb_candidate c = cand[i];
    const int b = c.bin - bin0;
    if (b < 0 || b >= nb) continue;
    out[start[b] + atomicAdd(cursor + b, 1u)] = c;
  }
}

template <int W>
__global__ void __launch_bounds__(256) k_stage2_bins(const float2* __restrict__ coeff, int ldk,
                                                     const float2* __restrict__ beta, int k, int T, int64_t half,
                                                     int bin0, int nb, const unsigned* __restrict__ start,
                                                     const rb_candidate* __restrict__ sorted, float thr2,
                                                     int64_t sample_offset, rb_trigger* __restrict__ trig,
                                                     unsigned long long* counter, int64_t cap) {
  extern __shared__ float2 bs[];  // [W][k]: the bin's window of every basis series
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    const unsigned c0 = start[b], c1 = start[b + 1];
    if (c0 == c1) continue;
    __syncthreads();
    const int64_t m0 = (int64_t)(bin0 + b) * W - half;
    for (int idx = threadIdx.x; idx < k * W; idx += blockDim.x) {
      const int kk = idx / W, r = idx - kk * W;
      bs[r * k + kk] = __ldg(beta + (int64_t)kk * half + m0 + r);
    }
    __syncthreads();
    for (unsigned ci = c0 + warp; ci < c1; ci += nwarp) {
      const rb_candidate cd = sorted[ci];
      if (cd.tmpl < 0 || cd.tmpl >= T) continue;
      float2 acc[W];
#pragma unroll
      for (int r = 0; r < W; ++r) acc[r] = make_float2(0.f, 0.f);
      const float2* arow = coeff + (int64_t)cd.tmpl * ldk;
      for (int kk = lane; kk < k; kk += 32) {
        const float2 av = __ldg(arow + kk);
#pragma unroll
        for (int r = 0; r < W; ++r) {
          const float2 bv = bs[r * k + kk];
          acc[r].x = fmaf(av.x, bv.x, fmaf(av.y, bv.y, acc[r].x));
          acc[r].y = fmaf(av.x, bv.y, fmaf(-av.y, bv.x, acc[r].y));
        }
      }
#pragma unroll
      for (int r = 0; r < W; ++r)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          acc[r].x += __shfl_xor_sync(0xffffffffu, acc[r].x, off);
          acc[r].y += __shfl_xor_sync(0xffffffffu, acc[r].y, off);
        }
      if (lane == 0) {
        int best = 0;
        float r2b = cabs2(acc[0]);
        float2 zb = acc[0];
#pragma unroll
        for (int r = 1; r < W; ++r) {
          const float r2 = cabs2(acc[r]);
          if (r2 > r2b) {
            r2b = r2;
            best = r;
            zb = acc[r];
          }
        }
        if (r2b >= thr2) {
          const unsigned long long idx = atomicAdd(counter, 1ull);
          if ((int64_t)idx < cap) {
            rb_trigger t;
            t.sample = sample_offset + (int64_t)cd.bin * W + best;
            t.tmpl = cd.tmpl;
            t.block = cd.block;
            t.snr = sqrtf(r2b);
            t.phase = atan2f(zb.y, zb.x);
            trig[idx] = t;
          }
        }
      }
    }
  }
}

template <int W>
int launch_bins(const rb_filter_desc& d, const rb_basis& b, const rb::Geometry& g, const rb::Workspace& ws,
                rb_trigger* trig, int64_t cap, cudaStream_t st) {
  const int nb = (int)g.n_bins;
  const int smem = W * d.k * (int)sizeof(float2);
  auto kern = k_stage2_bins<W>;
  if (smem > 48 * 1024) RB_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int grid = std::min(nb, 152 * 16);
  kern<<<grid, 256, smem, st>>>(reinterpret_cast<const float2*>(b.coeff), b.k, ws.beta, d.k, d.n_templates, g.n / 2,
                                nb, nb, ws.bin_start, ws.cand_sorted, d.rho_ii * d.rho_ii, d.sample_offset, trig,
                                ws.trig_count, cap);
  RB_LAUNCH_CHECK();
  return RB_OK;
}

}  // namespace

namespace rb {

int stage2_bucketed(const rb_filter_desc& d, const rb_basis& b, const Geometry& g, const Workspace& ws,
                    rb_trigger* trig, int64_t cap, cudaStream_t st) {
  const int nb = (int)g.n_bins;
  const int bin0 = nb;  // valid bins are [n/(2w), n/w)
  if (d.k * d.w * (int)sizeof(float2) > 200 * 1024) {
    set_detail("k * w too large for the second-stage window (%d x %d)", d.k, d.w);
    return RB_ERR_UNSUPPORTED;
  }
  RB_CUDA_TRY(cudaMemsetAsync(ws.bin_count, 0, sizeof(unsigned) * (nb + 1), st));
  k_bin_count<<<152 * 8, 256, 0, st>>>(ws.cand, ws.cand_count, d.cand_capacity, bin0, nb, ws.bin_count);
  RB_LAUNCH_CHECK();
  k_bin_scan<<<1, 1024, 0, st>>>(ws.bin_count, ws.bin_start, nb);
  RB_LAUNCH_CHECK();
  k_bin_scatter<<<152 * 8, 256, 0, st>>>(ws.cand, ws.cand_count, d.cand_capacity, bin0, nb, ws.bin_start,
                                         ws.bin_count, ws.cand_sorted);
  RB_LAUNCH_CHECK();
  switch (d.w) {
    case 1: return launch_bins<1>(d, b, g, ws, trig, cap, st);
    case 2: return launch_bins<2>(d, b, g, ws, trig, cap, st);
    case 4: return launch_bins<4>(d, b, g, ws, trig, cap, st);
    case 8: return launch_bins<8>(d, b, g, ws, trig, cap, st);
    case 16: return launch_bins<16>(d, b, g, ws, trig, cap, st);
  }
  return RB_ERR_BAD_INPUT;
}

}  // namespace rb
