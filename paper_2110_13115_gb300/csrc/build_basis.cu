// Step a0 (rb_build) and template generation (rb_templates), arXiv:2110.13115 Sec. III.A-B:
// whitened unit-norm stationary-phase templates on the GPU, then a randomised subspace
// iteration with FP64 orthonormalisation and an FP64 Rayleigh-Ritz step for the basis.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "linalg.h"

namespace {

constexpr double kMsunS = 4.925491025543576e-06;  // G M_sun / c^3 [s]
constexpr double kPi = 3.14159265358979323846;

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// Per-frequency FP64 tables: vf[j] = (pi f_j)^(1/3), amp[j] = f_j^(-7/6) sqrt(4 df / S_j).
__global__ void k_freq_tables(int64_t half, double df, const double* psd, double* vf, double* amp, unsigned* flags) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < half; j += (int64_t)gridDim.x * blockDim.x) {
    if (j == 0) {
      vf[0] = 0.0;
      amp[0] = 0.0;
      continue;
    }
    const double f = j * df, S = psd[j];
    if (!(S > 0.0) || isinf(S) || isnan(S)) {
      atomicOr(flags, (unsigned)RB_FLAG_BAD_PSD);
      amp[j] = 0.0;
    } else {
      amp[j] = pow(f, -7.0 / 6.0) * sqrt(4.0 * df / S);
    }
    vf[j] = cbrt(kPi * f);
  }
}

// One CTA per template: sigma^2 = sum over the support of amp^2 (FP64), then the unit-norm row
// g_t[j] / sigma_t = amp[j] exp(-i Psi(f_j)) / sigma_t, Psi in FP64 reduced modulo 2 pi.
__global__ void __launch_bounds__(256) k_templates(int T, int64_t half, double df, double f_low,
                                                   const double* __restrict__ params, int pn,
                                                   const double* __restrict__ vf, const double* __restrict__ amp,
                                                   float2* __restrict__ out, int64_t ld, double* __restrict__ sigma2) {
  __shared__ double red[256];
  const int t = blockIdx.x;
  if (t >= T) return;
  const double m1 = params[4 * t], m2 = params[4 * t + 1], x1 = params[4 * t + 2], x2 = params[4 * t + 3];
  const double mt = m1 + m2, eta = m1 * m2 / (mt * mt), ms = mt * kMsunS;
  const double beta = (x1 * (113.0 * (m1 / mt) * (m1 / mt) + 75.0 * eta) + x2 * (113.0 * (m2 / mt) * (m2 / mt) + 75.0 * eta)) / 12.0;
  const double c0 = 3.0 / (128.0 * eta);
  const double c2 = pn >= 2 ? (20.0 / 9.0) * (743.0 / 336.0 + 11.0 * eta / 4.0) : 0.0;
  const double c3 = pn >= 3 ? 4.0 * beta - 16.0 * kPi : 0.0;
  const double fisco = 1.0 / (pow(6.0, 1.5) * kPi * ms);
  const double m13 = cbrt(ms);
  // support f_low <= j df < fisco, 0 < j < half, with the comparisons done exactly as stated
  int64_t jlo = (int64_t)floor(f_low / df) - 1;
  if (jlo < 1) jlo = 1;
  while (jlo < half && (double)jlo * df < f_low) ++jlo;
  int64_t jhi = (int64_t)floor(fisco / df) + 2;
  if (jhi > half) jhi = half;
  while (jhi > jlo && (double)(jhi - 1) * df >= fisco) --jhi;
  double acc = 0.0;
  for (int64_t j = jlo + threadIdx.x; j < jhi; j += blockDim.x) acc += amp[j] * amp[j];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  const double s2 = red[0];
  if (threadIdx.x == 0) sigma2[t] = s2;
  const double inv = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
  float2* row = out + (int64_t)t * ld;
  for (int64_t j = threadIdx.x; j < half; j += blockDim.x) {
    float2 g = make_float2(0.f, 0.f);
    if (j >= jlo && j < jhi) {
      const double v = m13 * vf[j];
      const double iv = 1.0 / v, iv2 = iv * iv;
      double psi = -0.25 * kPi + c0 * iv2 * iv * (iv2 + c2 + c3 * v);
      psi -= 2.0 * kPi * rint(psi / (2.0 * kPi));
      float sn, cs;
      sincosf((float)psi, &sn, &cs);
      const float a = (float)(amp[j] * inv);
      g = make_float2(a * cs, -a * sn);
    }
    row[j] = g;
  }
}

// Counter-based complex normal draws (splitmix64 hash of (seed, index), Box-Muller).
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
__global__ void k_randn(float2* out, int64_t count, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t h = splitmix64(seed ^ splitmix64((uint64_t)i));
    const double u1 = ((h >> 11) + 1.0) * (1.0 / 9007199254740993.0);
    const double u2 = (splitmix64(h) >> 11) * (1.0 / 9007199254740992.0);
    const double r = sqrt(-2.0 * log(u1));
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    out[i] = make_float2((float)(r * c), (float)(r * s));
  }
}

// out = conj(in) rounded to FP32
__global__ void k_d2f_conj(const double2* in, float2* out, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = make_float2((float)in[i].x, -(float)in[i].y);
}

// ---------------------------------------------------------------------------------------
// Generic strided complex GEMM: C[m, n] (+)= sum_k opA(A)[m, k] opB(B)[k, n] with
// element (m, k) of A at A[m sam + k sak] and (k, n) of B at B[k sbk + n sbn]; op = optional
// conjugation. 64 x 64 tiles, 16-deep K steps, 256 threads with 4 x 4 outputs each.
// Accumulation in ACC (float or double) within a CTA's K-slice; ATOMIC adds the slice's sum
// into a double2 C (split-K).
template <typename ACC>
struct V2;
template <>
struct V2<float> {
  using t = float2;
};
template <>
struct V2<double> {
  using t = double2;
};

template <typename ACC, typename TI>
__device__ __forceinline__ typename V2<ACC>::t ld2(const TI* p, int64_t i, bool conj) {
  const TI v = p[i];
  typename V2<ACC>::t r;
  r.x = (ACC)v.x;
  r.y = conj ? -(ACC)v.y : (ACC)v.y;
  return r;
}

template <typename TA, typename TB, typename TC, typename ACC, bool CA, bool CB, bool ATOMIC>
__global__ void __launch_bounds__(256) k_cgemm(int M, int N, int64_t K, int64_t kchunk, const TA* __restrict__ A,
                                               int64_t sam, int64_t sak, const TB* __restrict__ B, int64_t sbk,
                                               int64_t sbn, TC* __restrict__ C, int64_t scm, int64_t scn) {
  using A2 = typename V2<ACC>::t;
  __shared__ A2 As[16][65];
  __shared__ A2 Bs[16][65];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  const int64_t kb = (int64_t)blockIdx.z * kchunk;
  const int64_t ke = min(K, kb + kchunk);
  A2 acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q].x = acc[p][q].y = (ACC)0;
  const bool a_kfast = sak == 1, b_nfast = sbn == 1;
  for (int64_t k0 = kb; k0 < ke; k0 += 16) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = tid + 256 * e;
      int mm, kk;
      if (a_kfast) {
        kk = idx & 15;
        mm = idx >> 4;
      } else {
        mm = idx & 63;
        kk = idx >> 6;
      }
      A2 va;
      va.x = va.y = (ACC)0;
      if (m0 + mm < M && k0 + kk < ke) va = ld2<ACC>(A, (int64_t)(m0 + mm) * sam + (k0 + kk) * sak, CA);
      As[kk][mm] = va;
      int nn, kb2;
      if (b_nfast) {
        nn = idx & 63;
        kb2 = idx >> 6;
      } else {
        kb2 = idx & 15;
        nn = idx >> 4;
      }
      A2 vb;
      vb.x = vb.y = (ACC)0;
      if (n0 + nn < N && k0 + kb2 < ke) vb = ld2<ACC>(B, (k0 + kb2) * sbk + (int64_t)(n0 + nn) * sbn, CB);
      Bs[kb2][nn] = vb;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      A2 av[4], bv[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) av[p] = As[kk][ty + 16 * p];
#pragma unroll
      for (int q = 0; q < 4; ++q) bv[q] = Bs[kk][tx + 16 * q];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          acc[p][q].x = fma(av[p].x, bv[q].x, fma(-av[p].y, bv[q].y, acc[p][q].x));
          acc[p][q].y = fma(av[p].x, bv[q].y, fma(av[p].y, bv[q].x, acc[p][q].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int m = m0 + ty + 16 * p, n = n0 + tx + 16 * q;
      if (m < M && n < N) {
        TC* c = C + (int64_t)m * scm + (int64_t)n * scn;
        if constexpr (ATOMIC) {
          atomicAdd(&c->x, (double)acc[p][q].x);
          atomicAdd(&c->y, (double)acc[p][q].y);
        } else {
          c->x = (decltype(c->x))acc[p][q].x;
          c->y = (decltype(c->y))acc[p][q].y;
        }
      }
    }
}

template <typename TA, typename TB, typename TC, typename ACC, bool CA, bool CB, bool ATOMIC>
int gemm(int M, int N, int64_t K, const TA* A, int64_t sam, int64_t sak, const TB* B, int64_t sbk, int64_t sbn, TC* C,
         int64_t scm, int64_t scn, cudaStream_t st) {
  const int64_t tiles = (int64_t)((M + 63) / 64) * ((N + 63) / 64);
  int64_t kchunk = K;
  if (ATOMIC) {
    const int64_t want = std::max<int64_t>(1, (152 * 16 + tiles - 1) / tiles);
    kchunk = std::max<int64_t>(256, ((K + want - 1) / want + 15) / 16 * 16);
  }
  const int64_t splits = (K + kchunk - 1) / kchunk;
  dim3 grid((N + 63) / 64, (M + 63) / 64, (unsigned)splits);
  k_cgemm<TA, TB, TC, ACC, CA, CB, ATOMIC><<<grid, 256, 0, st>>>(M, N, K, kchunk, A, sam, sak, B, sbk, sbn, C, scm, scn);
  RB_LAUNCH_CHECK();
  return RB_OK;
}

struct BuildWs {
  unsigned* flags;
  double* params;
  double* vf;
  double* amp;
  float2* G;     // [T][half]
  float2* Om;    // [T][l]
  double2* B;    // [T][l]
  float2* Y;     // [l][half]
  float2* Q;     // [l][half]
  double2* W;    // [l][l]
  float2* Mf;    // [l][l]
  double2* Md;   // [l][l]
  size_t total;
};

void carve_build(int T, int64_t half, int l, char* base, BuildWs* w, bool templates_only) {
  size_t off = 0;
  auto take = [&](size_t b) {
    char* p = base ? base + off : nullptr;
    off += a256(b);
    return p;
  };
  w->flags = (unsigned*)take(256);
  w->params = (double*)take(sizeof(double) * 4 * T);
  w->vf = (double*)take(sizeof(double) * half);
  w->amp = (double*)take(sizeof(double) * half);
  if (!templates_only) {
    w->G = (float2*)take(sizeof(float2) * (size_t)T * half);
    w->Om = (float2*)take(sizeof(float2) * (size_t)T * l);
    w->B = (double2*)take(sizeof(double2) * (size_t)T * l);
    w->Y = (float2*)take(sizeof(float2) * (size_t)l * half);
    w->Q = (float2*)take(sizeof(float2) * (size_t)l * half);
    w->W = (double2*)take(sizeof(double2) * (size_t)l * l);
    w->Mf = (float2*)take(sizeof(float2) * (size_t)l * l);
    w->Md = (double2*)take(sizeof(double2) * (size_t)l * l);
  }
  w->total = off;
}

int check_bank(const rb_bank_desc* b) {
  if (!b || !b->params) {
    rb::set_detail("bank or params is NULL");
    return RB_ERR_BAD_INPUT;
  }
  if (!rb_is_pow2(b->n) || b->n < (1 << 10) || b->n > (1 << 20) || !(b->fs > 0) || !(b->f_low > 0) ||
      b->n_templates < 1 || !(b->pn_order == 0 || b->pn_order == 2 || b->pn_order == 3)) {
    rb::set_detail("bad bank descriptor (n=%lld, fs=%g, f_low=%g, T=%d, pn_order=%d)", (long long)b->n, b->fs,
                   b->f_low, b->n_templates, b->pn_order);
    return RB_ERR_BAD_INPUT;
  }
  for (int t = 0; t < b->n_templates; ++t) {
    const double* p = b->params + 4 * t;
    if (!(p[0] > 0) || !(p[1] > 0) || !std::isfinite(p[0] + p[1] + p[2] + p[3]) || std::fabs(p[2]) > 1 ||
        std::fabs(p[3]) > 1) {
      rb::set_detail("template %d has invalid parameters", t);
      return RB_ERR_BAD_INPUT;
    }
  }
  return RB_OK;
}

int gen_templates(const rb_bank_desc* b, const double* psd, const BuildWs& w, float2* out, double* sigma2,
                  cudaStream_t st) {
  const int64_t half = b->n / 2;
  const double df = b->fs / (double)b->n;
  RB_CUDA_TRY(cudaMemsetAsync(w.flags, 0, 256, st));
  RB_CUDA_TRY(cudaMemcpyAsync(w.params, b->params, sizeof(double) * 4 * b->n_templates, cudaMemcpyHostToDevice, st));
  k_freq_tables<<<(int)std::min<int64_t>(2048, (half + 255) / 256), 256, 0, st>>>(half, df, psd, w.vf, w.amp, w.flags);
  RB_LAUNCH_CHECK();
  k_templates<<<b->n_templates, 256, 0, st>>>(b->n_templates, half, df, b->f_low, w.params, b->pn_order, w.vf, w.amp,
                                               out, half, sigma2);
  RB_LAUNCH_CHECK();
  return RB_OK;
}

using cd = std::complex<double>;

int download(std::vector<cd>& h, const double2* d, size_t count, cudaStream_t st) {
  h.resize(count);
  RB_CUDA_TRY(cudaMemcpyAsync(h.data(), d, sizeof(double2) * count, cudaMemcpyDeviceToHost, st));
  RB_CUDA_TRY(cudaStreamSynchronize(st));
  return RB_OK;
}

int upload(const std::vector<cd>& h, const BuildWs& w, size_t count, cudaStream_t st) {
  std::vector<float> f(2 * count);
  for (size_t i = 0; i < count; ++i) {
    f[2 * i] = (float)h[i].real();
    f[2 * i + 1] = (float)h[i].imag();
  }
  RB_CUDA_TRY(cudaMemcpyAsync(w.Md, h.data(), sizeof(double2) * count, cudaMemcpyHostToDevice, st));
  RB_CUDA_TRY(cudaMemcpyAsync(w.Mf, f.data(), sizeof(float2) * count, cudaMemcpyHostToDevice, st));
  RB_CUDA_TRY(cudaStreamSynchronize(st));
  return RB_OK;
}

// Rows of Y (l x half) -> orthonormal rows in Q by CholeskyQR2 with FP64 Gram matrices
// (shifted on the first pass when the Gram matrix is not numerically positive definite).
int orthonormalise(int l, int64_t half, const BuildWs& w, float2*& Y, float2*& Q, cudaStream_t st) {
  std::vector<cd> Wh, L((size_t)l * l), Li((size_t)l * l);
  for (int pass = 0; pass < 2; ++pass) {
    RB_CUDA_TRY(cudaMemsetAsync(w.W, 0, sizeof(double2) * l * l, st));
    int rc = gemm<float2, float2, double2, double, false, true, true>(l, l, half, Y, half, 1, Y, 1, half, w.W, l, 1, st);
    if (rc) return rc;
    if ((rc = download(Wh, w.W, (size_t)l * l, st))) return rc;
    if (!rb::cholesky(l, Wh.data(), L.data())) {
      double tr = 0.0;
      for (int i = 0; i < l; ++i) tr = std::max(tr, Wh[(size_t)i * l + i].real());
      const double shift = 1e-12 * tr * l;
      for (int i = 0; i < l; ++i) Wh[(size_t)i * l + i] += shift;
      if (!rb::cholesky(l, Wh.data(), L.data())) {
        rb::set_detail("sketch Gram matrix is not positive definite (rank-deficient bank?)");
        return RB_ERR_BAD_INPUT;
      }
    }
    rb::lower_inverse(l, L.data(), Li.data());
    if ((rc = upload(Li, w, (size_t)l * l, st))) return rc;
    rc = gemm<float2, float2, float2, float, false, false, false>(l, (int)half, l, w.Mf, l, 1, Y, half, 1, Q, half, 1, st);
    if (rc) return rc;
    std::swap(Y, Q);
  }
  std::swap(Y, Q);  // result in Q
  return RB_OK;
}

// Largest single-template truncation loss for every basis size: loss[q] = max_t (1 - sum_{j<=q} |a_tj|^2),
// accumulated in FP64, clamped at 0 (rounding can push the captured fraction of a row slightly above
// one). Non-negative doubles order like their bit patterns, so the maxima are unsigned 64-bit atomics:
// one shared-memory maximum per CTA and basis size, then one global atomic per (CTA, size).
__global__ void __launch_bounds__(256) k_max_loss(const float2* __restrict__ coeff, int T, int k,
                                                  unsigned long long* __restrict__ out) {
  extern __shared__ unsigned long long smax[];
  for (int q = threadIdx.x; q < k; q += blockDim.x) smax[q] = 0ull;
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < T) {
    const float2* row = coeff + (int64_t)t * k;
    double cap = 0.0;
    for (int q = 0; q < k; ++q) {
      const float2 a = row[q];
      cap += (double)a.x * a.x + (double)a.y * a.y;
      const double loss = fmax(1.0 - cap, 0.0);
      atomicMax(&smax[q], (unsigned long long)__double_as_longlong(loss));
    }
  }
  __syncthreads();
  for (int q = threadIdx.x; q < k; q += blockDim.x) atomicMax(&out[q], smax[q]);
}

}  // namespace

extern "C" {

int rb_basis_max_loss(const rb_basis* basis, double* loss, void* workspace, size_t workspace_bytes, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (!basis || !basis->coeff || !loss || basis->k < 1 || basis->n_templates < 1) {
    rb::set_detail("NULL basis, coefficients or output, or k, T < 1");
    return RB_ERR_BAD_INPUT;
  }
  const int k = basis->k, T = basis->n_templates;
  if ((size_t)k * 8 > 48 * 1024) {
    rb::set_detail("k = %d above the %d vectors this call handles", k, 48 * 1024 / 8);
    return RB_ERR_UNSUPPORTED;
  }
  if (!workspace || workspace_bytes < (size_t)k * 8 || ((uintptr_t)workspace & 255)) {
    rb::set_detail("workspace too small: need %zu bytes, 256-byte aligned", (size_t)k * 8);
    return RB_ERR_OOM;
  }
  auto* acc = (unsigned long long*)workspace;
  RB_CUDA_TRY(cudaMemsetAsync(acc, 0, (size_t)k * 8, st));
  k_max_loss<<<(T + 255) / 256, 256, (size_t)k * 8, st>>>((const float2*)basis->coeff, T, k, acc);
  RB_LAUNCH_CHECK();
  RB_CUDA_TRY(cudaMemcpyAsync(loss, acc, (size_t)k * 8, cudaMemcpyDeviceToHost, st));
  RB_CUDA_TRY(cudaStreamSynchronize(st));
  return RB_OK;
}

int rb_build_plan(const rb_bank_desc* bank, int32_t k, int32_t oversample, size_t* templates_bytes,
                  size_t* build_bytes) {
  int rc = check_bank(bank);
  if (rc) return rc;
  if (k < 1 || k > bank->n_templates || oversample < 0) {
    rb::set_detail("k = %d must be in [1, T = %d], oversample >= 0", k, bank->n_templates);
    return RB_ERR_BAD_INPUT;
  }
  const int l = std::min(k + oversample, bank->n_templates);
  BuildWs a, b;
  carve_build(bank->n_templates, bank->n / 2, l, nullptr, &a, true);
  carve_build(bank->n_templates, bank->n / 2, l, nullptr, &b, false);
  if (templates_bytes) *templates_bytes = a.total;
  if (build_bytes) *build_bytes = b.total;
  return RB_OK;
}

int rb_templates(const rb_bank_desc* bank, const double* psd, float* out, double* sigma2, void* workspace,
                 size_t workspace_bytes, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int rc = check_bank(bank);
  if (rc) return rc;
  if (!psd || !out || !sigma2) {
    rb::set_detail("NULL array");
    return RB_ERR_BAD_INPUT;
  }
  BuildWs w;
  carve_build(bank->n_templates, bank->n / 2, 1, nullptr, &w, true);
  if (!workspace || workspace_bytes < w.total || ((uintptr_t)workspace & 255)) {
    rb::set_detail("workspace too small: need %zu bytes", w.total);
    return RB_ERR_OOM;
  }
  carve_build(bank->n_templates, bank->n / 2, 1, (char*)workspace, &w, true);
  return gen_templates(bank, psd, w, (float2*)out, sigma2, st);
}

int rb_build(const rb_bank_desc* bank, const double* psd, int32_t k, int32_t oversample, int32_t power_iters,
             uint64_t seed, float* vectors, float* coeff, double* sigma2, double* sv, void* workspace,
             size_t workspace_bytes, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  size_t need = 0;
  int rc = rb_build_plan(bank, k, oversample, nullptr, &need);
  if (rc) return rc;
  if (!psd || !vectors || !coeff || !sigma2 || !sv || power_iters < 0) {
    rb::set_detail("NULL array or negative power_iters");
    return RB_ERR_BAD_INPUT;
  }
  const int T = bank->n_templates;
  const int64_t half = bank->n / 2;
  const int l = std::min(k + oversample, T);
  if (l > 1024) {
    rb::set_detail("sketch width %d exceeds 1024", l);
    return RB_ERR_UNSUPPORTED;
  }
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255)) {
    rb::set_detail("workspace too small: need %zu bytes", need);
    return RB_ERR_OOM;
  }
  BuildWs w;
  carve_build(T, half, l, (char*)workspace, &w, false);
  if ((rc = gen_templates(bank, psd, w, w.G, sigma2, st))) return rc;
  unsigned flags = 0;
  RB_CUDA_TRY(cudaMemcpyAsync(&flags, w.flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  RB_CUDA_TRY(cudaStreamSynchronize(st));
  if (flags & RB_FLAG_BAD_PSD) {
    rb::set_detail("PSD not finite and positive on 0 < j < n/2");
    return RB_ERR_BAD_INPUT;
  }
  // sketch rows Y[i] = sum_t Omega[t][i] g_t (random combinations of the templates)
  k_randn<<<1024, 256, 0, st>>>(w.Om, (int64_t)T * l, seed);
  RB_LAUNCH_CHECK();
  float2* Y = w.Y;
  float2* Q = w.Q;
  if ((rc = gemm<float2, float2, float2, float, false, false, false>(l, (int)half, T, w.Om, 1, l, w.G, half, 1, Y,
                                                                    half, 1, st)))
    return rc;
  for (int it = 0; it <= power_iters; ++it) {
    if ((rc = orthonormalise(l, half, w, Y, Q, st))) return rc;
    // B = G Q^H  (T x l), FP32 products summed in FP64 across K-slices
    RB_CUDA_TRY(cudaMemsetAsync(w.B, 0, sizeof(double2) * (size_t)T * l, st));
    if ((rc = gemm<float2, float2, double2, float, false, true, true>(T, l, half, w.G, half, 1, Q, 1, half, w.B, l, 1,
                                                                     st)))
      return rc;
    if (it == power_iters) break;
    // power step on the row space: Y[i] = sum_t conj(B[t][i]) g_t = q_i (G^H G)
    k_d2f_conj<<<1024, 256, 0, st>>>(w.B, w.Om, (int64_t)T * l);
    RB_LAUNCH_CHECK();
    if ((rc = gemm<float2, float2, float2, float, false, false, false>(l, (int)half, T, w.Om, 1, l, w.G, half, 1, Y,
                                                                      half, 1, st)))
      return rc;
  }
  // Rayleigh-Ritz: B^H B = V diag(s^2) V^H  (FP64)
  RB_CUDA_TRY(cudaMemsetAsync(w.W, 0, sizeof(double2) * l * l, st));
  if ((rc = gemm<double2, double2, double2, double, true, false, true>(l, l, T, w.B, 1, l, w.B, l, 1, w.W, l, 1, st)))
    return rc;
  std::vector<cd> Wh, V((size_t)l * l);
  if ((rc = download(Wh, w.W, (size_t)l * l, st))) return rc;
  std::vector<double> ev(l);
  rb::herm_eig(l, Wh.data(), ev.data(), V.data());
  for (int i = 0; i < k; ++i) sv[i] = std::sqrt(std::max(ev[i], 0.0));
  if ((rc = upload(V, w, (size_t)l * l, st))) return rc;
  // basis rows p_kk = sum_i conj(V[i][kk]) q_i ; coefficients a[t][kk] = sum_i B[t][i] V[i][kk]
  if ((rc = gemm<float2, float2, float2, float, true, false, false>(k, (int)half, l, w.Mf, 1, l, Q, half, 1,
                                                                   (float2*)vectors, half, 1, st)))
    return rc;
  if ((rc = gemm<double2, double2, float2, double, false, false, false>(T, k, l, w.B, l, 1, w.Md, l, 1, (float2*)coeff,
                                                                       k, 1, st)))
    return rc;
  RB_CUDA_TRY(cudaStreamSynchronize(st));
  return RB_OK;
}

}  // extern "C"
