// Hot path of the hierarchical reduced-basis matched filter (arXiv:2110.13115, Sec. III.C/E):
//   a1 whitening forward FFT, a2+a3 basis SNR series with bin averages, the template-method
//   comparator, the FP32 first stage, and operand packing for the tensor-core first stage.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstring>

#include "fft.cuh"
#include "fft2.cuh"
#include "internal.h"

using namespace rbfft;

namespace {

enum { MODE_BANK = 0, MODE_STRAIN = 1, MODE_PLAIN = 2, MODE_FOLD = 3, MODE_LOWPASS = 4 };

// Folded spectrum of the fast first stage (Sec. III.D, Eqs. 10-12) at f' of a length-M = n/w transform:
// Omega(f') = sum_{l < w/2} s_hat[l M + f'] conj(g[l M + f']) gfold[l M + f'] with gfold[j] = G(j) / w and
// G(j) = sum_{r<w} exp(2 pi i j r / n); terms with l >= w/2 fall on the zero half of the one-sided spectrum.
__device__ __forceinline__ float2 fold_at(const float2* __restrict__ shat, const float2* __restrict__ row,
                                          const float2* __restrict__ gfold, int64_t fp, int64_t M, int fold_w) {
  float2 acc = make_float2(0.f, 0.f);
  for (int l = 0; l < fold_w / 2; ++l) {
    const int64_t j = l * M + fp;
    const float2 q = cmulc(__ldg(shat + j), __ldcs(row + j));
    acc = cadd(acc, cmul(q, __ldg(gfold + j)));
  }
  return acc;
}

// gfold[j] = G(j) / w for 0 <= j < n/2, with G(j) = (1 - e^(2 pi i j w / n)) / (1 - e^(2 pi i j / n)) and
// G(0) = w (the geometric sum over the w samples of a bin, in FP64).
__global__ void k_gfold(float2* gfold, int64_t n, int w) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n / 2; j += (int64_t)gridDim.x * blockDim.x) {
    if (j == 0) {
      gfold[0] = make_float2(1.f, 0.f);
      continue;
    }
    double sa, ca, sb, cb;
    sincospi(2.0 * (double)((j * w) % n) / (double)n, &sa, &ca);
    sincospi(2.0 * (double)j / (double)n, &sb, &cb);
    const double nr = 1.0 - ca, ni = -sa, dr = 1.0 - cb, di = -sb;
    const double den = dr * dr + di * di;
    gfold[j] = make_float2((float)((nr * dr + ni * di) / (den * w)), (float)((ni * dr - nr * di) / (den * w)));
  }
}

// ---------------------------------------------------------------------------------------
// Set-up: twiddle tables (FP64 sincospi rounded to FP32) and the whitening weights
//   wt[j] = dt * sqrt(4 df / S_j) for 0 < j < n/2 (0 at DC).
// tables: tab_n1[n1] = exp(2 pi i e/n1), tab_n2[n2] = exp(2 pi i e/n2), tab_fine[n2] = exp(2 pi i e/n)
__global__ void k_init(float2* tab_n1, float2* tab_n2, float2* tab_fine, float2* w2a, float2* w2b, int n1, int n2,
                       float* wt, const double* psd, int64_t half, double dt, double df, unsigned* flags) {
  const int64_t n = (int64_t)n1 * n2;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // stage-2 twiddles of the radix-32 passes: w2[j (S + 1) + r] = exp(2 pi i j r / L), S = L / 32
  for (int e = (int)tid; e < 2 * 32 * 33; e += (int)stride) {
    const int which = e / (32 * 33), rem = e % (32 * 33);
    const int L = which == 0 ? n2 : n1, S = L / 32;
    const int j = rem / (S + 1), r = rem % (S + 1);
    if (S < 1 || j >= 32 || r >= S) continue;
    double s, c;
    sincospi(2.0 * (double)((j * r) % L) / L, &s, &c);
    (which == 0 ? w2a : w2b)[j * (S + 1) + r] = make_float2((float)c, (float)s);
  }
  for (int64_t e = tid; e < n1 + 2 * n2; e += stride) {
    double s, c;
    if (e < n1) {
      sincospi(2.0 * (double)e / n1, &s, &c);
      tab_n1[e] = make_float2((float)c, (float)s);
    } else if (e < n1 + n2) {
      const int64_t i = e - n1;
      sincospi(2.0 * (double)i / n2, &s, &c);
      tab_n2[i] = make_float2((float)c, (float)s);
    } else {
      const int64_t i = e - n1 - n2;
      sincospi(2.0 * (double)i / (double)n, &s, &c);
      tab_fine[i] = make_float2((float)c, (float)s);
    }
  }
  if (wt == nullptr) return;
  for (int64_t j = tid; j < half; j += stride) {
    if (j == 0) {
      wt[0] = 0.f;
      continue;
    }
    const double S = psd[j];
    if (!(S > 0.0) || isinf(S) || isnan(S)) {
      atomicOr(flags, (unsigned)RB_FLAG_BAD_PSD);
      wt[j] = 0.f;
    } else {
      wt[j] = (float)(dt * sqrt(4.0 * df / S));
    }
  }
}

// ---------------------------------------------------------------------------------------
// Pass A of the four-step transform: G columns j1 of length L = n2.
//  MODE_BANK : x[j] = s_hat[j] * conj(rows[vec][j]) for j < n/2 (zero above: the one-sided
//              filter of Eq. 1), inverse sign. rows = basis vectors or unit-norm templates.
//  MODE_STRAIN: x[j] = strain[j], forward sign.
// Output X[vec][j1][m2] (m2 fastest) = w_n^(j1 m2) * inner transform.
template <int MODE, int L, int G>
__global__ void __launch_bounds__(G * L / kE) k_pass_a(const float2* __restrict__ rows,
                                                       const float2* __restrict__ shat,
                                                       const float* __restrict__ strain,
                                                       float2* __restrict__ X,
                                                       const float2* __restrict__ tab_n2,
                                                       const float2* __restrict__ tab_n1,
                                                       const float2* __restrict__ tab_fine, int n1,
                                                       int64_t vec0, const float2* __restrict__ gfold, int fold_w) {
  constexpr int SIGN = MODE == MODE_STRAIN ? -1 : 1;
  constexpr int LOG2L = __builtin_ctz(L);
  extern __shared__ float2 smem[];
  float2* tw = smem;
  float2* sdata = smem + L;
  const int tid = threadIdx.x;
  for (int e = tid; e < L; e += blockDim.x) tw[e] = tab_n2[e];
  __syncthreads();
  const int c = tid % G, tj = tid / G;
  const int j1 = blockIdx.x * G + c;
  const int64_t M = (int64_t)n1 * L, half = M / 2;
  // MODE_FOLD and MODE_LOWPASS transform length M = n / w; their rows are one-sided spectra of n / 2 points
  const int64_t pitch = (MODE == MODE_FOLD || MODE == MODE_LOWPASS) ? M * fold_w / 2 : half;
  const float2* row = rows + (vec0 + blockIdx.y) * pitch;
  float2 v[kE];
  auto load = [&](int j2) -> float2 {
    const int64_t j = (int64_t)j1 + (int64_t)n1 * j2;
    if constexpr (MODE == MODE_STRAIN) {
      return make_float2(__ldg(strain + j), 0.f);
    } else if constexpr (MODE == MODE_FOLD) {
      return fold_at(shat, row, gfold, j, M, fold_w);
    } else if constexpr (MODE == MODE_LOWPASS) {
      return cmulc(__ldg(shat + j), __ldcs(row + j));  // the band below n/w of the one-sided product
    } else {
      if (j2 >= L / 2) return make_float2(0.f, 0.f);
      return cmulc(__ldg(shat + j), __ldcs(row + j));
    }
  };
  column_transform<SIGN, L, G, MODE == MODE_BANK>(v, c, tj, sdata, tw, load);
  __syncthreads();
  // twiddle w_n^(j1 m2): the last pass's outputs are m2 = m2_0(b) + r NS, so each butterfly takes one
  // table value w_n^(j1 m2_0) and the powers of w_n^(j1 NS), shared by the thread's butterflies
  constexpr int RL = LastPass<L>::R, NSL = LastPass<L>::NS;
  auto tw_n = [&](int rr) {  // w_n^rr, rr < n, from the two-level table
    float2 t = cmul(__ldg(tab_n1 + (rr >> LOG2L)), __ldg(tab_fine + (rr & (L - 1))));
    if (SIGN < 0) t.y = -t.y;
    return t;
  };
  float2 sp[RL];
  if constexpr (RL > 1) twiddle_powers<RL>(tw_n(j1 * NSL), sp);
#pragma unroll
  for (int b = 0; b < kE / RL; ++b) {
    const int m20 = final_point<L>(tj, b, 0);
    const float2 base = tw_n(j1 * m20);  // j1 m2 < n
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const float2 t = r == 0 ? base : cmul(base, sp[r]);
      sdata[c * (L + 1) + m20 + r * NSL] = cmul(v[b * RL + r], t);
    }
  }
  __syncthreads();
  float2* xo = X + ((int64_t)blockIdx.y * n1 + (int64_t)blockIdx.x * G) * L;
  for (int idx = tid; idx < G * L; idx += blockDim.x) {
    const int cc = idx >> LOG2L, m2 = idx & (L - 1);
    xo[idx] = sdata[cc * (L + 1) + m2];
  }
}

template <int L, int G>
constexpr int pass_a_smem_bytes() {
  return (L + std::max(Smem<L, G>::data, G * (L + 1))) * 8;
}

// ---------------------------------------------------------------------------------------
// Pass B: G columns m2 of length L = n1, input X[vec][j1][m2]; output sample
// m = m2 + n2 m1 of the long transform.
//  MODE_BANK  : keep m in [n/2, n): beta[vec][m - n/2] and the W-sample bin means
//               beta_avg[vec][(m - n/2)/W] (Eq. 9).
//  MODE_STRAIN: keep m in [0, n/2): s_hat[m] = wt[m] * Y[m] (whitening, Sec. III.E).
//  MODE_PLAIN : keep m in [n/2, n): rho^2 = |Y|^2, window arg-max over W samples,
//               trigger when rho^2 >= thr2 (template method, Eq. 4).
struct PassBArgs {
  const float2* X;
  int n2;
  int64_t vec0;
  float2* beta;
  float2* beta_avg;
  float2* shat;
  const float* wt;
  rb_trigger* trig;
  unsigned long long* counter;
  int64_t cap;
  float thr2;
  int64_t sample_offset;
  int block_id;
  rb_candidate* cand;  // MODE_FOLD output (capacity cap, count at counter)
};

template <int MODE, int L, int W, int G>
__global__ void __launch_bounds__(G * L / kE) k_pass_b(PassBArgs a, const float2* __restrict__ tab_n1) {
  static_assert(G >= W, "a bin's W columns must lie in one CTA");
  constexpr int SIGN = MODE == MODE_STRAIN ? -1 : 1;
  extern __shared__ float2 smem[];
  float2* tw = smem;
  float2* sdata = smem + L;
  const int tid = threadIdx.x;
  for (int e = tid; e < L; e += blockDim.x) tw[e] = tab_n1[e];
  __syncthreads();
  const int c = tid % G, tj = tid / G;
  const int n2 = a.n2;
  const int m2 = blockIdx.x * G + c;
  const float2* xin = a.X + (int64_t)blockIdx.y * L * n2;
  float2 v[kE];
  auto load = [&](int j1) -> float2 { return xin[(int64_t)j1 * n2 + m2]; };
  column_transform<SIGN, L, G>(v, c, tj, sdata, tw, load);
  const int64_t n = (int64_t)L * n2, half = n / 2;
  const int64_t vec = a.vec0 + blockIdx.y;
  // the last pass's outputs are m1 = j + r NS with j < NS = L / RL, so m1 >= L/2 exactly when
  // r >= RL/2: the half that is not kept is known at compile time and never finished or stored
  constexpr int RL = LastPass<L>::R;
  static_assert(RL >= 2 && LastPass<L>::NS * RL == L, "last pass layout");
#pragma unroll
  for (int b = 0; b < kE / RL; ++b)
#pragma unroll
    for (int r = 0; r < RL; ++r) {
      const int m1 = final_point<L>(tj, b, r);
      const int64_t m = m2 + (int64_t)n2 * m1;
      const float2 val = v[b * RL + r];
      if constexpr (MODE == MODE_STRAIN) {
        if (r < RL / 2) a.shat[m] = cscale(val, __ldg(a.wt + m));
      } else if constexpr (MODE == MODE_BANK) {
        if (r < RL / 2) continue;
        float2 s = val;
#pragma unroll
        for (int off = 1; off < W; off <<= 1) {
          s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
          s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
        }
        if (a.beta) __stcs(a.beta + vec * half + (m - half), val);
        if ((c & (W - 1)) == 0) a.beta_avg[vec * (half / W) + (m - half) / W] = cscale(s, 1.0f / W);
      } else if constexpr (MODE == MODE_FOLD) {
        if (r < RL / 2) continue;
        const float r2 = cabs2(val);
        if (r2 >= a.thr2) {
          const unsigned long long idx = atomicAdd(a.counter, 1ull);
          if ((int64_t)idx < a.cap) {
            rb_candidate cd;
            cd.tmpl = (int32_t)vec;
            cd.bin = (int32_t)m;
            cd.snr_avg = sqrtf(r2);
            cd.block = a.block_id;
            a.cand[idx] = cd;
          }
        }
      } else {
        if (r < RL / 2) continue;
        float r2 = cabs2(val);
        int64_t mb = m;
        float2 vb = val;
#pragma unroll
        for (int off = 1; off < W; off <<= 1) {
          const float r2o = __shfl_xor_sync(0xffffffffu, r2, off);
          const int64_t mo = __shfl_xor_sync(0xffffffffu, mb, off);
          const float vx = __shfl_xor_sync(0xffffffffu, vb.x, off);
          const float vy = __shfl_xor_sync(0xffffffffu, vb.y, off);
          if (r2o > r2 || (r2o == r2 && mo < mb)) {
            r2 = r2o;
            mb = mo;
            vb = make_float2(vx, vy);
          }
        }
        if ((c & (W - 1)) == 0 && r2 >= a.thr2) {
          const unsigned long long idx = atomicAdd(a.counter, 1ull);
          if ((int64_t)idx < a.cap) {
            rb_trigger t;
            t.sample = a.sample_offset + mb;
            t.tmpl = (int32_t)vec;
            t.block = a.block_id;
            t.snr = sqrtf(r2);
            t.phase = atan2f(vb.y, vb.x);
            a.trig[idx] = t;
          }
        }
      }
    }
}

template <int L, int G>
constexpr int pass_b_smem_bytes() {
  return (L + Smem<L, G>::data) * 8;
}

// ---------------------------------------------------------------------------------------
// Radix-32 four-step passes of the basis filter and the template method for n >= 2^16 (inner and
// outer lengths 256..1024), persistent: a grid of at most three CTAs per SM walks the work items
// (a group of G columns of one vector) of a chunk. Pass A: column j1 of length L = n2 gets
// x[j2] = s_hat[j] conj(row[j]), j = j1 + n1 j2, zero for j >= n/2 (the one-sided filter of Eq. 1);
// two register stages (the first skipping the zero half); the four-step twiddle w_n^(j1 m2);
// X[vec][j1][m2] stored from registers (no transpose).
//   w_n^(j1 m2) with m2 = j + 32 k: w_n^(j1 j) (two table values per butterfly) times (w_n^(32 j1))^k,
//   the powers by a running product over k.

// w_n^e for 0 <= e < n from the two-level tables (tab_n1[e >> log2 L] = w_n1^(e >> log2 L), tab_fine = w_n^(e mod L))
template <int LOG2L>
__device__ __forceinline__ float2 tw_two_level(const float2* __restrict__ tab_n1, const float2* __restrict__ tab_fine,
                                               int64_t e) {
  constexpr int L = 1 << LOG2L;
  return cmul(__ldg(tab_n1 + (e >> LOG2L)), __ldg(tab_fine + (e & (L - 1))));
}

// VAR bit 0: stage-2 twiddles by running products (fft2.cuh TWR); bit 1: the outputs staged in shared
// memory and stored as whole rows (16-byte stores, 256 contiguous bytes per warp).
template <int L, int G, int FW, int VAR = 0>
__global__ void __launch_bounds__(G * L / 32, FW == 0 ? 3 : 2) k_fa(const float2* __restrict__ rows, const float2* __restrict__ shat,
                                                      float2* __restrict__ X, const float2* __restrict__ tab_n1,
                                                      const float2* __restrict__ tab_fine,
                                                      const float2* __restrict__ w2, int n1, int64_t vec0, int nvec,
                                                      const float2* __restrict__ gfold) {
  using namespace rbfft2;
  constexpr int S = Col<L>::S, NB = Col<L>::NB;
  constexpr int LOG2L = __builtin_ctz(L);
  extern __shared__ float2 xbuf[];  // [exchange_slots<L, G>]
  const int tid = threadIdx.x;
  const int c = tid % G, tj = tid / G;
  const int groups = n1 / G;
  const int64_t n = (int64_t)n1 * L, half = n / 2;
  const int64_t items = (int64_t)groups * nvec;
  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int grp = (int)(item % groups);
    const int64_t vec = item / groups;
    const int j1 = grp * G + c;
    float2 v[32];
    if constexpr (FW > 0) {
      const float2* row = rows + (vec0 + vec) * (n * FW / 2);
#pragma unroll
      for (int r = 0; r < 32; ++r) v[r] = fold_at(shat, row, gfold, (int64_t)j1 + (int64_t)n1 * (tj + S * r), n, FW);
    } else if constexpr (FW < 0) {
      const float2* row = rows + (vec0 + vec) * (n * -FW / 2);
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        const int64_t j = (int64_t)j1 + (int64_t)n1 * (tj + S * r);
        v[r] = cmulc(__ldg(shat + j), __ldcs(row + j));
      }
    } else {
      const float2* row = rows + (vec0 + vec) * half;
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int64_t j = (int64_t)j1 + (int64_t)n1 * (tj + S * r);
        v[r] = cmulc(__ldg(shat + j), __ldcs(row + j));
      }
#pragma unroll
      for (int r = 16; r < 32; ++r) v[r] = make_float2(0.f, 0.f);
    }
    column32<1, L, G, FW == 0, false, (VAR & 1) != 0>(v, c, tj, xbuf, w2);
    const float2 step = tw_two_level<LOG2L>(tab_n1, tab_fine, ((int64_t)32 * j1) & (n - 1));
    if constexpr ((VAR & 2) != 0) {
      // rows of L + 2 slots: the stores of a half-warp (8 columns x 2 consecutive m2) hit distinct banks
      constexpr int PITCH = L + 2;
      static_assert(G * PITCH <= exchange_slots<L, G>(), "staged rows fit the exchange buffer");
      __syncthreads();  // every thread is done reading the exchange buffer
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int j = tj + S * b;
        float2 t = tw_two_level<LOG2L>(tab_n1, tab_fine, (int64_t)j1 * j);  // j1 j < 32 n1 <= n
#pragma unroll
        for (int k = 0; k < S; ++k) {
          xbuf[c * PITCH + j + 32 * k] = cmul(v[b * S + k], t);
          t = cmul(t, step);
        }
      }
      __syncthreads();
      float4* xo = reinterpret_cast<float4*>(X + (vec * n1 + (int64_t)grp * G) * L);
      for (int e = tid; e < G * L / 2; e += blockDim.x) {
        const int cc = e / (L / 2), m = 2 * (e % (L / 2));
        const float2 a0 = xbuf[cc * PITCH + m], a1 = xbuf[cc * PITCH + m + 1];
        xo[e] = make_float4(a0.x, a0.y, a1.x, a1.y);
      }
    } else {
      float2* xo = X + (vec * n1 + j1) * L;
#pragma unroll
      for (int b = 0; b < NB; ++b) {
        const int j = tj + S * b;
        float2 t = tw_two_level<LOG2L>(tab_n1, tab_fine, (int64_t)j1 * j);  // j1 j < 32 n1 <= n
#pragma unroll
        for (int k = 0; k < S; ++k) {
          xo[j + 32 * k] = cmul(v[b * S + k], t);
          t = cmul(t, step);
        }
      }
    }
    __syncthreads();  // the next item's stage-1 stores reuse the exchange buffer
  }
}

template <int L, int G>
constexpr int fa_smem_bytes() {
  return rbfft2::exchange_slots<L, G>() * 8;
}

// Pass B: G columns m2 of length L = n1 from X[vec][j1][m2]; two register stages of which the second
// forms only the upper half (m1 >= L/2, the valid samples m = m2 + n2 m1 >= n/2). The kept outputs
// go to shared memory (rows of G + 1 slots: conflict-free for the bin sums), where W consecutive
// columns (one bin, Eq. 9) are summed (MODE_BANK: beta and the bin means), searched for their arg-max
// (MODE_PLAIN: template-method triggers), or thresholded (MODE_FOLD, W = 1: first-stage candidates).
template <int MODE, int L, int W, int G, int VAR = 0>
__global__ void __launch_bounds__(G * L / 32, G * L / 32 <= 256 ? 3 : 1) k_fb(PassBArgs a,
                                                                             const float2* __restrict__ w2, int nvec) {
  using namespace rbfft2;
  static_assert(G >= W && G % W == 0, "a bin's W columns must lie in one CTA");
  constexpr int S = Col<L>::S, NB = Col<L>::NB, H = L / 2, P = G + 1;
  static_assert(H * P <= exchange_slots<L, G>(), "kept outputs fit the exchange buffer");
  extern __shared__ float2 xbuf[];
  const int tid = threadIdx.x;
  const int c = tid % G, tj = tid / G;
  const int n2 = a.n2;
  const int groups = n2 / G;
  const int64_t n = (int64_t)L * n2, half = n / 2;
  const int64_t items = (int64_t)groups * nvec;
  for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
    const int grp = (int)(item % groups);
    const int64_t iv = item / groups, vec = a.vec0 + iv;
    const int m20 = grp * G, m2 = m20 + c;
    const float2* xin = a.X + iv * L * n2 + m2;
    float2 v[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) v[r] = xin[(int64_t)(tj + S * r) * n2];
    column32<1, L, G, false, true, (VAR & 1) != 0>(v, c, tj, xbuf, w2);
    __syncthreads();  // every thread is done reading the exchange buffer
    // kept outputs: k >= S/2 of butterfly b, m1 = j + 32 k, p = m1 - L/2 in [0, L/2)
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const int j = tj + S * b;
#pragma unroll
      for (int k = S / 2; k < S; ++k) {
        const int p = j + 32 * k - H;
        const float2 val = v[b * S + k];
        if constexpr (MODE == MODE_BANK)
          if (a.beta) __stcs(a.beta + vec * half + (m2 + (int64_t)n2 * p), val);
        xbuf[p * P + c] = val;
      }
    }
    __syncthreads();
    // (G / W) bins of W columns for each of the L/2 kept rows
    constexpr int NBIN = (G / W) * H;
    for (int q = tid; q < NBIN; q += blockDim.x) {
      const int cg = q % (G / W), p = q / (G / W);
      const float2* src = xbuf + p * P + cg * W;
      const int64_t bin = (int64_t)(m20 / W + cg) + (int64_t)(n2 / W) * p;
      if constexpr (MODE == MODE_BANK) {
        float2 s = src[0];
#pragma unroll
        for (int r = 1; r < W; ++r) s = cadd(s, src[r]);
        a.beta_avg[vec * (half / W) + bin] = cscale(s, 1.0f / W);
      } else if constexpr (MODE == MODE_FOLD) {
        static_assert(W == 1, "a folded series has one sample per bin");
        const float r2 = cabs2(src[0]);
        if (r2 >= a.thr2) {
          const unsigned long long idx = atomicAdd(a.counter, 1ull);
          if ((int64_t)idx < a.cap) {
            rb_candidate cd;
            cd.tmpl = (int32_t)vec;
            cd.bin = (int32_t)(half + bin);
            cd.snr_avg = sqrtf(r2);
            cd.block = a.block_id;
            a.cand[idx] = cd;
          }
        }
      } else {
        float best = -1.f;
        int br = 0;
        float2 vb = src[0];
#pragma unroll
        for (int r = 0; r < W; ++r) {
          const float2 z = src[r];
          const float r2 = cabs2(z);
          if (r2 > best) {  // strict: ties keep the smaller sample
            best = r2;
            br = r;
            vb = z;
          }
        }
        if (best >= a.thr2) {
          const unsigned long long idx = atomicAdd(a.counter, 1ull);
          if ((int64_t)idx < a.cap) {
            rb_trigger t;
            t.sample = a.sample_offset + half + bin * W + br;
            t.tmpl = (int32_t)vec;
            t.block = a.block_id;
            t.snr = sqrtf(best);
            t.phase = atan2f(vb.y, vb.x);
            a.trig[idx] = t;
          }
        }
      }
    }
    __syncthreads();  // the next item's stage-1 stores reuse the buffer
  }
}

template <int L, int G>
constexpr int fb_smem_bytes() {
  return rbfft2::exchange_slots<L, G>() * 8;
}

// CTAs of a persistent radix-32 pass: resident CTAs per SM (asked of the runtime once per kernel) x SMs,
// at most the number of work items.
template <class K>
static int persistent_grid(K kernel, int threads, int smem, int64_t items) {
  static int per_sm = 0, sms = 0;
  if (per_sm == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
      per_sm = 1;
    if (sms < 1) sms = 1;
  }
  return (int)std::min<int64_t>(items, (int64_t)per_sm * sms);
}

// ---------------------------------------------------------------------------------------
// First stage in FP32 (SIMT): z_avg[t, i] = sum_k conj(a_tk) beta_avg_k[i] over a 64x64 tile,
// |z_avg|^2 >= thr2 tested in registers, candidates appended (Sec. III.C first stage).
__global__ void __launch_bounds__(256) k_stage1_simt(const float2* __restrict__ coeff, int ldk,
                                                     const float2* __restrict__ bavg, int T, int k,
                                                     int nb, float thr2, int bin0, int block_id,
                                                     rb_candidate* cand, unsigned long long* counter,
                                                     int64_t cap) {
  __shared__ float2 As[16][65];
  __shared__ float2 Bs[16][64];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int t0 = blockIdx.y * 64, i0 = blockIdx.x * 64;
  float2 acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = make_float2(0.f, 0.f);
  for (int k0 = 0; k0 < k; k0 += 16) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = tid + 256 * e;
      const int tt = idx >> 4, kk = idx & 15;
      As[kk][tt] = (t0 + tt < T && k0 + kk < k) ? coeff[(int64_t)(t0 + tt) * ldk + k0 + kk] : make_float2(0.f, 0.f);
      const int kb = idx >> 6, ii = idx & 63;
      Bs[kb][ii] = (k0 + kb < k && i0 + ii < nb) ? bavg[(int64_t)(k0 + kb) * nb + i0 + ii] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float2 av[4], bv[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) av[p] = As[kk][ty + 16 * p];
#pragma unroll
      for (int q = 0; q < 4; ++q) bv[q] = Bs[kk][tx + 16 * q];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[p][q].x = fmaf(av[p].x, bv[q].x, fmaf(av[p].y, bv[q].y, acc[p][q].x));
          acc[p][q].y = fmaf(av[p].x, bv[q].y, fmaf(-av[p].y, bv[q].x, acc[p][q].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int t = t0 + ty + 16 * p, i = i0 + tx + 16 * q;
      if (t < T && i < nb) {
        const float r2 = cabs2(acc[p][q]);
        if (r2 >= thr2) {
          const unsigned long long idx = atomicAdd(counter, 1ull);
          if ((int64_t)idx < cap) {
            rb_candidate cd;
            cd.tmpl = t;
            cd.bin = bin0 + i;
            cd.snr_avg = sqrtf(r2);
            cd.block = block_id;
            cand[idx] = cd;
          }
        }
      }
    }
}

// ---------------------------------------------------------------------------------------
// Operand packing for the tensor-core first stage (16-bit planes, hi then lo).
template <typename T16>
__device__ __forceinline__ T16 to16(float x);
template <>
__device__ __forceinline__ __half to16<__half>(float x) { return __float2half_rn(x); }
template <>
__device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
__device__ __forceinline__ float from16(__half x) { return __half2float(x); }
__device__ __forceinline__ float from16(__nv_bfloat16 x) { return __bfloat162float(x); }

// rows 2t: [Re a_t(0..k), Im a_t(0..k), 0..]; rows 2t+1: [-Im a_t, Re a_t, 0..]
template <typename T16>
__global__ void k_pack_coeff(const float2* __restrict__ coeff, int ldk, int T, int k, int kp,
                             T16* __restrict__ hi, T16* __restrict__ lo) {
  const int64_t total = (int64_t)2 * T * kp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / kp;
    const int col = (int)(idx - row * kp);
    const int64_t t = row >> 1;
    const bool im = row & 1;
    float x = 0.f;
    if (col < k) {
      const float2 a = coeff[t * ldk + col];
      x = im ? -a.y : a.x;
    } else if (col < 2 * k) {
      const float2 a = coeff[t * ldk + col - k];
      x = im ? a.x : a.y;
    }
    const T16 h = to16<T16>(x);
    hi[idx] = h;
    if (lo) lo[idx] = to16<T16>(x - from16(h));
  }
}

// second-stage operand rows t: [Re a_t(0..k), 0.., Im a_t(0..k), 0..] with halves of k16 columns
__global__ void k_pack_s2(const float2* __restrict__ coeff, int ldk, int T, int k, int k16, __half* __restrict__ hi,
                          __half* __restrict__ lo) {
  const int64_t p2 = 2 * (int64_t)k16;
  const int64_t total = (int64_t)T * p2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = idx / p2;
    // row position p = 32 q + 8 t4 + s holds column c = 16 kc + j of [Re a (k16) | Im a (k16)] with
    // kc = 2 q + s / 4 and j = 2 t4 + (s & 1) + 8 ((s >> 1) & 1): the m16n8k16 A-fragment order, so
    // that one 16-byte load gives a lane its registers a0, a2 (or a1, a3) for two K chunks
    const int pos = (int)(idx - t * p2);
    const int q = pos >> 5, t4 = (pos >> 3) & 3, sl = pos & 7;
    const int col = (2 * q + (sl >> 2)) * 16 + 2 * t4 + (sl & 1) + 8 * ((sl >> 1) & 1);
    const bool im = col >= k16;
    const int kk = im ? col - k16 : col;
    float x = 0.f;
    if (kk < k) {
      const float2 a = coeff[t * ldk + kk];
      x = im ? a.y : a.x;
    }
    const __half h = __float2half_rn(x);
    hi[idx] = h;
    lo[idx] = __float2half_rn(x - __half2float(h));
  }
}

// beta_avg [k][nb] complex -> [nb][kp] rows: [Re beta_avg(:, i), Im beta_avg(:, i), 0..]
template <typename T16>
__global__ void __launch_bounds__(256) k_pack_beta(const float2* __restrict__ bavg, int k, int nb, int kp,
                                                   T16* __restrict__ hi, T16* __restrict__ lo) {
  __shared__ float2 tile[32][33];
  const int i0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of 32
  for (int r = ty; r < 32; r += 8) {
    const int kk = k0 + r, ii = i0 + tx;
    tile[r][tx] = (kk < k && ii < nb) ? bavg[(int64_t)kk * nb + ii] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int ii = i0 + r, kk = k0 + tx;
    if (ii >= nb) continue;
    const float2 b = tile[tx][r];
    const int64_t base = (int64_t)ii * kp;
    if (kk < k) {
      const T16 hr = to16<T16>(b.x), hm = to16<T16>(b.y);
      hi[base + kk] = hr;
      hi[base + k + kk] = hm;
      if (lo) {
        lo[base + kk] = to16<T16>(b.x - from16(hr));
        lo[base + k + kk] = to16<T16>(b.y - from16(hm));
      }
    }
    // zero padding columns [2k, kp) once per row (block column 0 only)
    if (blockIdx.y == 0) {
      for (int col = 2 * k + tx; col < kp; col += 32) {
        hi[base + col] = to16<T16>(0.f);
        if (lo) lo[base + col] = to16<T16>(0.f);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Launch helpers (template dispatch on the column length)

template <typename K>
static cudaError_t allow_smem(K kernel, int bytes) {
  if (bytes <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// Columns per CTA of the four-step passes. Inner (pass A) and outer (pass B) lengths of 256 and
// more take the tuned variant's widths; shorter lengths use fixed widths that keep CTAs >= 64 threads.
template <int L>
struct GA {
  static constexpr int value = L >= 512 ? 8 : (L >= 128 ? 16 : 32);
};

template <int MODE, int L, int G>
static int launch_a_LG(const rb::Geometry& g, const float2* rows, const float2* shat, const float* strain,
                       float2* X, const rb::Tables& tb, int64_t vec0, int nvec, cudaStream_t st,
                       const float2* gfold, int fold_w) {
  constexpr int smem = pass_a_smem_bytes<L, G>();
  auto kern = k_pass_a<MODE, L, G>;
  RB_CUDA_TRY(allow_smem(kern, smem));
  dim3 grid(g.n1 / G, nvec);
  kern<<<grid, G * L / kE, smem, st>>>(rows, shat, strain, X, tb.n2, tb.n1, tb.fine, g.n1, vec0, gfold, fold_w);
  RB_LAUNCH_CHECK();
  return RB_OK;
}

template <int MODE, int L>
static int launch_a_L(const rb::Geometry& g, const float2* rows, const float2* shat, const float* strain,
                      float2* X, const rb::Tables& tb, int64_t vec0, int nvec, int ga, cudaStream_t st,
                      const float2* gfold, int fold_w) {
  if constexpr (L >= 256) {
    if (ga == 4 && g.n1 >= 4)
      return launch_a_LG<MODE, L, 4>(g, rows, shat, strain, X, tb, vec0, nvec, st, gfold, fold_w);
    if (ga == 16 && g.n1 >= 16)
      return launch_a_LG<MODE, L, 16>(g, rows, shat, strain, X, tb, vec0, nvec, st, gfold, fold_w);
  }
  return launch_a_LG<MODE, L, GA<L>::value>(g, rows, shat, strain, X, tb, vec0, nvec, st, gfold, fold_w);
}

template <int MODE>
static int launch_a(const rb::Geometry& g, const float2* rows, const float2* shat, const float* strain,
                    float2* X, const rb::Tables& tb, int64_t vec0, int nvec, int ga, cudaStream_t st,
                    const float2* gfold = nullptr, int fold_w = 1) {
  switch (g.n2) {
    case 32: return launch_a_L<MODE, 32>(g, rows, shat, strain, X, tb, vec0, nvec, ga, st, gfold, fold_w);
    case 64: return launch_a_L<MODE, 64>(g, rows, shat, strain, X, tb, vec0, nvec, ga, st, gfold, fold_w);
    case 128: return launch_a_L<MODE, 128>(g, rows, shat, strain, X, tb, vec0, nvec, ga, st, gfold, fold_w);
    case 256: return launch_a_L<MODE, 256>(g, rows, shat, strain, X, tb, vec0, nvec, ga, st, gfold, fold_w);
    case 512: return launch_a_L<MODE, 512>(g, rows, shat, strain, X, tb, vec0, nvec, ga, st, gfold, fold_w);
    case 1024: return launch_a_L<MODE, 1024>(g, rows, shat, strain, X, tb, vec0, nvec, ga, st, gfold, fold_w);
  }
  rb::set_detail("unsupported inner FFT length %d", g.n2);
  return RB_ERR_UNSUPPORTED;
}

template <int MODE, int L, int W, int G>
static int launch_b_LWG(const rb::Geometry& g, const PassBArgs& a, const rb::Tables& tb, int nvec,
                        cudaStream_t st) {
  constexpr int smem = pass_b_smem_bytes<L, G>();
  auto kern = k_pass_b<MODE, L, W, G>;
  RB_CUDA_TRY(allow_smem(kern, smem));
  dim3 grid(g.n2 / G, nvec);
  kern<<<grid, G * L / kE, smem, st>>>(a, tb.n1);
  RB_LAUNCH_CHECK();
  return RB_OK;
}

template <int MODE, int L, int W>
static int launch_b_LW(const rb::Geometry& g, const PassBArgs& a, const rb::Tables& tb, int nvec, int gb,
                       cudaStream_t st) {
  if constexpr (L >= 256 && W <= 8 && MODE != MODE_STRAIN)
    if (gb == 8) return launch_b_LWG<MODE, L, W, 8>(g, a, tb, nvec, st);
  return launch_b_LWG<MODE, L, W, 16>(g, a, tb, nvec, st);
}

template <int MODE, int L>
static int launch_b_L(const rb::Geometry& g, const PassBArgs& a, const rb::Tables& tb, int nvec, int w, int gb,
                      cudaStream_t st) {
  if constexpr (MODE == MODE_STRAIN || MODE == MODE_FOLD) {
    return launch_b_LW<MODE, L, 1>(g, a, tb, nvec, gb, st);
  } else {
    switch (w) {
    case 1: return launch_b_LW<MODE, L, 1>(g, a, tb, nvec, gb, st);
    case 2: return launch_b_LW<MODE, L, 2>(g, a, tb, nvec, gb, st);
    case 4: return launch_b_LW<MODE, L, 4>(g, a, tb, nvec, gb, st);
    case 8: return launch_b_LW<MODE, L, 8>(g, a, tb, nvec, gb, st);
    case 16: return launch_b_LW<MODE, L, 16>(g, a, tb, nvec, gb, st);
  }
    rb::set_detail("unsupported bin width %d", w);
    return RB_ERR_BAD_INPUT;
  }
}

template <int MODE>
static int launch_b(const rb::Geometry& g, const PassBArgs& a, const rb::Tables& tb, int nvec, int w, int gb,
                    cudaStream_t st) {
  switch (g.n1) {
    case 32: return launch_b_L<MODE, 32>(g, a, tb, nvec, w, gb, st);
    case 64: return launch_b_L<MODE, 64>(g, a, tb, nvec, w, gb, st);
    case 128: return launch_b_L<MODE, 128>(g, a, tb, nvec, w, gb, st);
    case 256: return launch_b_L<MODE, 256>(g, a, tb, nvec, w, gb, st);
    case 512: return launch_b_L<MODE, 512>(g, a, tb, nvec, w, gb, st);
    case 1024: return launch_b_L<MODE, 1024>(g, a, tb, nvec, w, gb, st);
  }
  rb::set_detail("unsupported outer FFT length %d", g.n1);
  return RB_ERR_UNSUPPORTED;
}

// Radix-32 passes (n1, n2 >= 256): 256-thread CTAs, G = 256 / (L / 32) columns each (pass B takes
// 512 threads when 8 columns cannot hold a bin of w = 16).
int radix32_variant();  // bits of the VAR template argument in use (host hook rbx_set_fft_radix32)

template <int L, int FW, int VAR>
static int launch_fa_LFV(const rb::Geometry& g, const float2* rows, const float2* shat, float2* X, const rb::Tables& tb,
                         int64_t vec0, int nvec, cudaStream_t st, const float2* gfold) {
  constexpr int G = 256 / (L / 32);
  constexpr int smem = fa_smem_bytes<L, G>();
  auto kern = k_fa<L, G, FW, VAR>;
  RB_CUDA_TRY(allow_smem(kern, smem));
  const int grid = persistent_grid(kern, G * L / 32, smem, (int64_t)(g.n1 / G) * nvec);
  kern<<<grid, G * L / 32, smem, st>>>(rows, shat, X, tb.n1, tb.fine, tb.w2a, g.n1, vec0, nvec, gfold);
  RB_LAUNCH_CHECK();
  return RB_OK;
}

template <int L, int FW>
static int launch_fa_LF(const rb::Geometry& g, const float2* rows, const float2* shat, float2* X, const rb::Tables& tb,
                        int64_t vec0, int nvec, cudaStream_t st, const float2* gfold) {
  if constexpr (FW == 0) {
    switch (radix32_variant()) {
      case 1: return launch_fa_LFV<L, FW, 1>(g, rows, shat, X, tb, vec0, nvec, st, gfold);
      case 2: return launch_fa_LFV<L, FW, 2>(g, rows, shat, X, tb, vec0, nvec, st, gfold);
      case 3: return launch_fa_LFV<L, FW, 3>(g, rows, shat, X, tb, vec0, nvec, st, gfold);
    }
  }
  return launch_fa_LFV<L, FW, 0>(g, rows, shat, X, tb, vec0, nvec, st, gfold);
}

template <int L>
static int launch_fa_L(const rb::Geometry& g, const float2* rows, const float2* shat, float2* X, const rb::Tables& tb,
                       int64_t vec0, int nvec, cudaStream_t st, const float2* gfold, int fold_w) {
  switch (fold_w) {
    case 0: return launch_fa_LF<L, 0>(g, rows, shat, X, tb, vec0, nvec, st, gfold);
    case 2: return launch_fa_LF<L, 2>(g, rows, shat, X, tb, vec0, nvec, st, gfold);
    case 4: return launch_fa_LF<L, 4>(g, rows, shat, X, tb, vec0, nvec, st, gfold);
    case 8: return launch_fa_LF<L, 8>(g, rows, shat, X, tb, vec0, nvec, st, gfold);
    case 16: return launch_fa_LF<L, 16>(g, rows, shat, X, tb, vec0, nvec, st, gfold);
    case -2: return launch_fa_LF<L, -2>(g, rows, shat, X, tb, vec0, nvec, st, gfold);
    case -4: return launch_fa_LF<L, -4>(g, rows, shat, X, tb, vec0, nvec, st, gfold);
    case -8: return launch_fa_LF<L, -8>(g, rows, shat, X, tb, vec0, nvec, st, gfold);
    case -16: return launch_fa_LF<L, -16>(g, rows, shat, X, tb, vec0, nvec, st, gfold);
  }
  rb::set_detail("fold width %d", fold_w);
  return RB_ERR_BAD_INPUT;
}

// fold_w = 0: the one-sided product of the basis filter / template method; 2..16: the folded spectrum;
// -2..-16: the low-pass first stage.
static int launch_fa(const rb::Geometry& g, const float2* rows, const float2* shat, float2* X, const rb::Tables& tb,
                     int64_t vec0, int nvec, cudaStream_t st, const float2* gfold = nullptr, int fold_w = 0) {
  switch (g.n2) {
    case 256: return launch_fa_L<256>(g, rows, shat, X, tb, vec0, nvec, st, gfold, fold_w);
    case 512: return launch_fa_L<512>(g, rows, shat, X, tb, vec0, nvec, st, gfold, fold_w);
    case 1024: return launch_fa_L<1024>(g, rows, shat, X, tb, vec0, nvec, st, gfold, fold_w);
  }
  rb::set_detail("radix-32 pass A: inner length %d", g.n2);
  return RB_ERR_UNSUPPORTED;
}

template <int MODE, int L, int W, int VAR>
static int launch_fb_LWV(const rb::Geometry& g, const PassBArgs& a, const rb::Tables& tb, int nvec, cudaStream_t st) {
  constexpr int G0 = 256 / (L / 32);
  constexpr int G = G0 >= W ? G0 : W;
  constexpr int smem = fb_smem_bytes<L, G>();
  auto kern = k_fb<MODE, L, W, G, VAR>;
  RB_CUDA_TRY(allow_smem(kern, smem));
  const int grid = persistent_grid(kern, G * L / 32, smem, (int64_t)(g.n2 / G) * nvec);
  kern<<<grid, G * L / 32, smem, st>>>(a, tb.w2b, nvec);
  RB_LAUNCH_CHECK();
  return RB_OK;
}

template <int MODE, int L, int W>
static int launch_fb_LW(const rb::Geometry& g, const PassBArgs& a, const rb::Tables& tb, int nvec, cudaStream_t st) {
  if constexpr (MODE == MODE_BANK || MODE == MODE_PLAIN) {
    if (radix32_variant() & 1) return launch_fb_LWV<MODE, L, W, 1>(g, a, tb, nvec, st);
  }
  return launch_fb_LWV<MODE, L, W, 0>(g, a, tb, nvec, st);
}

template <int MODE, int L>
static int launch_fb_L(const rb::Geometry& g, const PassBArgs& a, const rb::Tables& tb, int nvec, int w,
                       cudaStream_t st) {
  if constexpr (MODE == MODE_FOLD) {
    return launch_fb_LW<MODE, L, 1>(g, a, tb, nvec, st);
  } else {
    switch (w) {
    case 1: return launch_fb_LW<MODE, L, 1>(g, a, tb, nvec, st);
    case 2: return launch_fb_LW<MODE, L, 2>(g, a, tb, nvec, st);
    case 4: return launch_fb_LW<MODE, L, 4>(g, a, tb, nvec, st);
    case 8: return launch_fb_LW<MODE, L, 8>(g, a, tb, nvec, st);
    case 16: return launch_fb_LW<MODE, L, 16>(g, a, tb, nvec, st);
  }
    rb::set_detail("unsupported bin width %d", w);
    return RB_ERR_BAD_INPUT;
  }
}

template <int MODE>
static int launch_fb(const rb::Geometry& g, const PassBArgs& a, const rb::Tables& tb, int nvec, int w, cudaStream_t st) {
  switch (g.n1) {
    case 256: return launch_fb_L<MODE, 256>(g, a, tb, nvec, w, st);
    case 512: return launch_fb_L<MODE, 512>(g, a, tb, nvec, w, st);
    case 1024: return launch_fb_L<MODE, 1024>(g, a, tb, nvec, w, st);
  }
  rb::set_detail("radix-32 pass B: outer length %d", g.n1);
  return RB_ERR_UNSUPPORTED;
}

bool use_radix32(const rb::Geometry& g) { return g.n1 >= 256 && g.n2 >= 256 && rb::fft_radix32_enabled(); }

// FFT schedule variants of the basis filter: columns per CTA of pass A and pass B, and the size
// in MB of a four-step chunk's intermediate X (which stays in L2 between the passes).
struct FftVariant {
  int ga, gb, mb;
};
constexpr FftVariant kFftVariants[RB_FFT_VARIANTS] = {{8, 16, 32}, {4, 8, 32}, {4, 16, 32}, {8, 8, 32},
                                                      {4, 8, 64}, {8, 16, 64}, {16, 16, 64}, {8, 16, 96}};

int chunk_vectors(const rb::Geometry& g, const rb::Workspace& ws, const FftVariant& v) {
  const int64_t want = ((int64_t)v.mb << 20) / (g.n * 8);
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, ws.vc));
}

std::mutex g_fft_mu;
std::map<std::pair<int64_t, int>, int> g_fft_choice;  // (n, w) -> variant

int fft_variant_for(int64_t n, int w) {
  std::lock_guard<std::mutex> lk(g_fft_mu);
  auto it = g_fft_choice.find({n, w});
  return it == g_fft_choice.end() ? 0 : it->second;
}

}  // namespace

// =======================================================================================
// Host orchestration (namespace rb, used by the C ABI below and by other translation units)

namespace rb {

int init_tables(const Geometry& g, const Workspace& ws, const double* psd, double fs, cudaStream_t st) {
  const double dt = 1.0 / fs, df = fs / (double)g.n;
  const int64_t work = std::max<int64_t>(g.n1 + 2 * g.n2, psd ? g.n / 2 : 0);
  const int blocks = (int)std::min<int64_t>(1024, (work + 255) / 256);
  k_init<<<blocks, 256, 0, st>>>(ws.tables.n1_w, ws.tables.n2_w, ws.tables.fine_w, ws.tables.w2a_w, ws.tables.w2b_w,
                                 g.n1, g.n2, psd ? ws.wt : nullptr, psd, g.n / 2, dt, df, ws.flags);
  RB_LAUNCH_CHECK();
  return RB_OK;
}

int whiten(const Geometry& g, const Workspace& ws, const float* strain, float2* shat, cudaStream_t st) {
  int rc = launch_a<MODE_STRAIN>(g, nullptr, nullptr, strain, ws.X, ws.tables, 0, 1, 8, st);
  if (rc) return rc;
  PassBArgs a{};
  a.X = ws.X;
  a.n2 = g.n2;
  a.shat = shat;
  a.wt = ws.wt;
  return launch_b<MODE_STRAIN>(g, a, ws.tables, 1, 1, 16, st);
}

static int bank_filter_v(const Geometry& g, const Workspace& ws, const float2* rows, int64_t nvec,
                         const float2* shat, float2* beta, float2* bavg, int w, const FftVariant& v, cudaStream_t st) {
  const int vc = chunk_vectors(g, ws, v);
  const bool r32 = use_radix32(g);
  for (int64_t v0 = 0; v0 < nvec; v0 += vc) {
    const int cnt = (int)std::min<int64_t>(vc, nvec - v0);
    int rc = r32 ? launch_fa(g, rows, shat, ws.X, ws.tables, v0, cnt, st)
                 : launch_a<MODE_BANK>(g, rows, shat, nullptr, ws.X, ws.tables, v0, cnt, v.ga, st);
    if (rc) return rc;
    PassBArgs a{};
    a.X = ws.X;
    a.n2 = g.n2;
    a.vec0 = v0;
    a.beta = beta;
    a.beta_avg = bavg;
    rc = r32 ? launch_fb<MODE_BANK>(g, a, ws.tables, cnt, w, st) : launch_b<MODE_BANK>(g, a, ws.tables, cnt, w, v.gb, st);
    if (rc) return rc;
  }
  return RB_OK;
}

int bank_filter(const Geometry& g, const Workspace& ws, const float2* rows, int64_t nvec, const float2* shat,
                float2* beta, float2* bavg, int w, cudaStream_t st) {
  return bank_filter_v(g, ws, rows, nvec, shat, beta, bavg, w, kFftVariants[fft_variant_for(g.n, w)], st);
}

namespace {
// 0: radix-16 passes; 1 + v: radix-32 passes in variant v (running-product twiddles and staged stores by
// default: 4.63 against 4.99 us per basis vector at n = 2^19 for the radix-16 passes)
std::atomic<int> g_radix32{4};
}
bool fft_radix32_enabled() { return g_radix32.load() != 0; }

int set_fft_variant(const Geometry& g, int w, int variant) {
  if (variant < 0 || variant >= RB_FFT_VARIANTS) {
    set_detail("FFT variant %d outside [0, %d)", variant, RB_FFT_VARIANTS);
    return RB_ERR_BAD_INPUT;
  }
  std::lock_guard<std::mutex> lk(g_fft_mu);
  g_fft_choice[{g.n, w}] = variant;
  return RB_OK;
}

int tune_fft(const Geometry& g, const Workspace& ws, const float2* rows, int64_t nvec, const float2* shat,
             float2* beta, float2* bavg, int w, double* ms, int* chosen, cudaStream_t st) {
  cudaEvent_t e0, e1;
  RB_CUDA_TRY(cudaEventCreate(&e0));
  RB_CUDA_TRY(cudaEventCreate(&e1));
  int rc = RB_OK, best = 0;
  for (int v = 0; v < RB_FFT_VARIANTS && rc == RB_OK; ++v) {
    const int reps = 3;
    rc = bank_filter_v(g, ws, rows, nvec, shat, beta, bavg, w, kFftVariants[v], st);  // warm-up
    if (rc == RB_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = RB_ERR_CUDA;
    for (int r = 0; r < reps && rc == RB_OK; ++r)
      rc = bank_filter_v(g, ws, rows, nvec, shat, beta, bavg, w, kFftVariants[v], st);
    float t = 0.f;
    if (rc == RB_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
      rc = RB_ERR_CUDA;
    if (rc == RB_OK) {
      ms[v] = t / reps;
      if (ms[v] < ms[best]) best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) {
    if (rc == RB_ERR_CUDA) set_detail("FFT tuning timing failed");
    return rc;
  }
  *chosen = best;
  return set_fft_variant(g, w, best);
}

int plain_filter(const Geometry& g, const Workspace& ws, const float2* tmpl, int64_t T, const float2* shat,
                 int w, float thr2, int64_t sample_offset, int block_id, rb_trigger* trig, int64_t cap,
                 cudaStream_t st) {
  const FftVariant& v = kFftVariants[fft_variant_for(g.n, w)];
  const int vc = chunk_vectors(g, ws, v);
  for (int64_t v0 = 0; v0 < T; v0 += vc) {
    const int cnt = (int)std::min<int64_t>(vc, T - v0);
    const bool r32 = use_radix32(g);
    int rc = r32 ? launch_fa(g, tmpl, shat, ws.X, ws.tables, v0, cnt, st)
                 : launch_a<MODE_BANK>(g, tmpl, shat, nullptr, ws.X, ws.tables, v0, cnt, v.ga, st);
    if (rc) return rc;
    PassBArgs a{};
    a.X = ws.X;
    a.n2 = g.n2;
    a.vec0 = v0;
    a.trig = trig;
    a.counter = ws.trig_count;
    a.cap = cap;
    a.thr2 = thr2;
    a.sample_offset = sample_offset;
    a.block_id = block_id;
    rc = r32 ? launch_fb<MODE_PLAIN>(g, a, ws.tables, cnt, w, st) : launch_b<MODE_PLAIN>(g, a, ws.tables, cnt, w, v.gb, st);
    if (rc) return rc;
  }
  return RB_OK;
}

int init_gfold(float2* gfold, int64_t n, int w, cudaStream_t st) {
  k_gfold<<<(int)std::min<int64_t>(1024, (n / 2 + 255) / 256), 256, 0, st>>>(gfold, n, w);
  RB_LAUNCH_CHECK();
  return RB_OK;
}

int folded_stage1(const Geometry& gm, const Workspace& wm, const float2* tmpl, int64_t T, const float2* shat, int w,
                  float thr2, int block_id, rb_candidate* cand, int64_t cap, const float2* gfold, cudaStream_t st,
                  bool lowpass) {
  const FftVariant& v = kFftVariants[fft_variant_for(gm.n, 1)];
  const int vc = chunk_vectors(gm, wm, v);
  const bool r32 = use_radix32(gm);
  for (int64_t v0 = 0; v0 < T; v0 += vc) {
    const int cnt = (int)std::min<int64_t>(vc, T - v0);
    int rc = r32 ? launch_fa(gm, tmpl, shat, wm.X, wm.tables, v0, cnt, st, gfold, lowpass ? -w : w)
             : lowpass ? launch_a<MODE_LOWPASS>(gm, tmpl, shat, nullptr, wm.X, wm.tables, v0, cnt, v.ga, st, gfold, w)
                       : launch_a<MODE_FOLD>(gm, tmpl, shat, nullptr, wm.X, wm.tables, v0, cnt, v.ga, st, gfold, w);
    if (rc) return rc;
    PassBArgs a{};
    a.X = wm.X;
    a.n2 = gm.n2;
    a.vec0 = v0;
    a.cand = cand;
    a.counter = wm.cand_count;
    a.cap = cap;
    a.thr2 = thr2;
    a.block_id = block_id;
    rc = r32 ? launch_fb<MODE_FOLD>(gm, a, wm.tables, cnt, 1, st) : launch_b<MODE_FOLD>(gm, a, wm.tables, cnt, 1, v.gb, st);
    if (rc) return rc;
  }
  return RB_OK;
}

int stage1_simt(const rb_filter_desc& d, const rb_basis& b, const Geometry& g, const Workspace& ws,
                const float2* bavg, rb_candidate* cand, cudaStream_t st) {
  const int nb = (int)g.n_bins;
  dim3 grid((nb + 63) / 64, (d.n_templates + 63) / 64);
  k_stage1_simt<<<grid, 256, 0, st>>>(reinterpret_cast<const float2*>(b.coeff), b.k, bavg, d.n_templates,
                                      d.k, nb, d.rho_i * d.rho_i, nb, d.block_id, cand, ws.cand_count,
                                      d.cand_capacity);
  RB_LAUNCH_CHECK();
  return RB_OK;
}

int pack_beta(const rb_filter_desc& d, const Geometry& g, const float2* bavg, void* hi, void* lo,
              cudaStream_t st) {
  const int nb = (int)g.n_bins;
  dim3 grid((nb + 31) / 32, (d.k + 31) / 32);
  const bool bf = d.precision == RB_PREC_BF16 || d.precision == RB_PREC_BF16_SPLIT;
  if (bf)
    k_pack_beta<__nv_bfloat16><<<grid, 256, 0, st>>>(bavg, d.k, nb, g.kp, (__nv_bfloat16*)hi, (__nv_bfloat16*)lo);
  else
    k_pack_beta<__half><<<grid, 256, 0, st>>>(bavg, d.k, nb, g.kp, (__half*)hi, (__half*)lo);
  RB_LAUNCH_CHECK();
  return RB_OK;
}

int pack_coeff(const rb_filter_desc& d, const rb_basis& b, const Geometry& g, void* out_all, cudaStream_t st) {
  {
    // second-stage operand: rows [Re a_t (k16), Im a_t (k16)] as FP16 hi and lo planes
    const int64_t p2 = (int64_t)d.n_templates * 2 * g.k16;
    auto* h2 = (__half*)out_all;
    k_pack_s2<<<(int)std::min<int64_t>(4096, (p2 + 255) / 256), 256, 0, st>>>(
        reinterpret_cast<const float2*>(b.coeff), b.k, d.n_templates, d.k, g.k16, h2, h2 + p2);
    RB_LAUNCH_CHECK();
  }
  if (d.precision == RB_PREC_FP32) return RB_OK;
  void* out = (char*)out_all + g.s2_bytes;
  const int64_t plane = (int64_t)2 * d.n_templates * g.kp;
  // A in hi and lo planes for every split precision (the B operand is split only for the first two)
  const bool split = d.precision == RB_PREC_FP16_SPLIT || d.precision == RB_PREC_BF16_SPLIT ||
                     d.precision == RB_PREC_FP16_SPLIT_A;
  const bool bf = d.precision == RB_PREC_BF16 || d.precision == RB_PREC_BF16_SPLIT;
  const int blocks = (int)std::min<int64_t>(4096, (plane + 255) / 256);
  if (bf) {
    auto* h = (__nv_bfloat16*)out;
    k_pack_coeff<__nv_bfloat16><<<blocks, 256, 0, st>>>(reinterpret_cast<const float2*>(b.coeff), b.k,
                                                        d.n_templates, d.k, g.kp, h, split ? h + plane : nullptr);
  } else {
    auto* h = (__half*)out;
    k_pack_coeff<__half><<<blocks, 256, 0, st>>>(reinterpret_cast<const float2*>(b.coeff), b.k,
                                                 d.n_templates, d.k, g.kp, h, split ? h + plane : nullptr);
  }
  RB_LAUNCH_CHECK();
  return RB_OK;
}

}  // namespace rb

namespace {
int radix32_variant() { return std::max(0, rb::g_radix32.load() - 1) & 3; }
}  // namespace

// Host-only hook (not part of the C ABI): 0 sends every length through the radix-16 four-step passes;
// 1 + v selects the radix-32 passes (the default wherever both four-step lengths are >= 256) in variant
// v (bit 0: stage-2 twiddles by running products; bit 1: pass A's outputs staged in shared memory);
// for parity tests between the passes and for timing.
extern "C" int rbx_set_fft_radix32(int mode) {
  rb::g_radix32.store(mode < 0 ? 0 : mode);
  return 0;
}
