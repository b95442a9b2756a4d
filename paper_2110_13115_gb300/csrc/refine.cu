// Candidate refinement (step a8): J(theta) = |Z(theta)|^2 / sigma^2 of a non-spinning TaylorF2
// template at its own coalescence time, its adjoint with respect to theta = (mc, eta, t_c, phi_c),
// and an in-kernel gradient ascent. The matched filter is Eq. (1) of arXiv:2110.13115 evaluated at
// t_0 = t_c (Eq. 3-4); the paper stops at the triggers, so the ascent rule is this library's own
// (see include/rbmf.h). One CTA per candidate recomputes the whitened template frequency by
// frequency in every pass: Psi in FP64 reduced modulo 2 pi, sin/cos in FP32, sums in FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr double kMsunS = 4.925491025543576e-06;
constexpr double kPi = 3.14159265358979323846;
constexpr double kFref = 100.0;
constexpr double kEtaMin = 0.05;
constexpr int kThreads = 256;

enum { R_EVAL = 0, R_ADJOINT = 1, R_ASCEND = 2 };

struct RefArgs {
  const float2* shat;
  const double* amp;  // f^(-7/6) sqrt(4 df / S_j)
  const double* vf;   // (pi f_j)^(1/3)
  int64_t half;
  double df;
  double f_low;
  int pn;
  const double* theta_in;
  double* theta_out;
  double* J;
  double* Z;
  const double* dJ;
  double* dtheta;
  int64_t n_cand;
  int steps;
  double alpha0, alpha_max;
  unsigned* flags;
};

__global__ void k_refine_tables(int64_t half, double df, const double* psd, double* amp, double* vf, unsigned* flags) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < half; j += (int64_t)gridDim.x * blockDim.x) {
    if (j == 0) {
      amp[0] = 0.0;
      vf[0] = 0.0;
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

// Sum NV doubles over the block; every thread receives the totals.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], off);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) red[warp * NV + i] = v[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w * NV + i];
    v[i] = s;
  }
}

// Z (v[0..1]) and, when GRAD, dZ/dtheta_k (v[2 + 2k .. 3 + 2k]) summed over [jlo, jhi).
template <bool GRAD>
__device__ void evaluate(const RefArgs& a, const double (&th)[4], int64_t jlo, int64_t jhi, double (&v)[10],
                         double* red) {
  const double mc = th[0], eta = th[1], tc = th[2], phic = th[3];
  const double mt = mc * pow(eta, -0.6) * kMsunS;
  const double m13 = cbrt(mt);
  const double c0 = 3.0 / (128.0 * eta);
  const double c2 = a.pn >= 2 ? (20.0 / 9.0) * (743.0 / 336.0 + 11.0 * eta / 4.0) : 0.0;
  const double c3 = a.pn >= 3 ? -16.0 * kPi : 0.0;
  const double dc2 = a.pn >= 2 ? (20.0 / 9.0) * (11.0 / 4.0) : 0.0;
#pragma unroll
  for (int i = 0; i < 10; ++i) v[i] = 0.0;
  for (int64_t j = jlo + threadIdx.x; j < jhi; j += blockDim.x) {
    const double f = j * a.df;
    const double vv = m13 * a.vf[j];
    const double iv = 1.0 / vv, iv2 = iv * iv, iv3 = iv2 * iv, iv5 = iv3 * iv2;
    const double psi_pn = c0 * (iv5 + c2 * iv3 + c3 * iv2);
    double psi = 2.0 * kPi * f * tc - phic - 0.25 * kPi + psi_pn;
    psi -= 2.0 * kPi * rint(psi / (2.0 * kPi));
    float sn, cs;
    sincosf((float)psi, &sn, &cs);
    const float2 sh = a.shat[j];
    const double am = a.amp[j];
    // term = s_hat * conj(g) = s_hat * amp * exp(+i Psi)
    const double tr = am * ((double)sh.x * cs - (double)sh.y * sn);
    const double ti = am * ((double)sh.x * sn + (double)sh.y * cs);
    v[0] += tr;
    v[1] += ti;
    if (GRAD) {
      const double dpsi_dm = (-5.0 * iv5 - 3.0 * c2 * iv3 - 2.0 * c3 * iv2) / (128.0 * eta * mt);
      const double dpsi_deta_m = -psi_pn / eta + c0 * dc2 * iv3;
      const double d[4] = {dpsi_dm * mt / mc, dpsi_deta_m + dpsi_dm * (-0.6 * mt / eta), 2.0 * kPi * f, -1.0};
#pragma unroll
      for (int k = 0; k < 4; ++k) {  // i d term
        v[2 + 2 * k] -= d[k] * ti;
        v[3 + 2 * k] += d[k] * tr;
      }
    }
  }
  block_sum<10>(v, red);
}

__device__ __forceinline__ void support(const RefArgs& a, double mc0, double eta0, int64_t& jlo, int64_t& jhi) {
  const double mt0 = mc0 * pow(eta0, -0.6) * kMsunS;
  const double fcut = 1.0 / (pow(6.0, 1.5) * kPi * mt0);
  jlo = (int64_t)floor(a.f_low / a.df) - 1;
  if (jlo < 1) jlo = 1;
  while (jlo < a.half && (double)jlo * a.df < a.f_low) ++jlo;
  jhi = (int64_t)floor(fcut / a.df) + 2;
  if (jhi > a.half) jhi = a.half;
  while (jhi > jlo && (double)(jhi - 1) * a.df >= fcut) --jhi;
}

template <int MODE>
__global__ void __launch_bounds__(kThreads) k_refine(RefArgs a) {
  __shared__ double red[(kThreads / 32) * 10];
  const int64_t c = blockIdx.x;
  if (c >= a.n_cand) return;
  double th[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) th[i] = a.theta_in[4 * c + i];
  if (!(th[0] > 0.0) || !(th[1] > 0.0) || !(th[1] <= 0.25) || !isfinite(th[2]) || !isfinite(th[3])) {
    if (threadIdx.x == 0) {
      atomicOr(a.flags, (unsigned)RB_FLAG_BAD_STRAIN);
      if (a.J) a.J[c] = __longlong_as_double(0x7ff8000000000000ll);
    }
    return;
  }
  int64_t jlo, jhi;
  support(a, th[0], th[1], jlo, jhi);
  double s2[1] = {0.0};
  for (int64_t j = jlo + threadIdx.x; j < jhi; j += blockDim.x) s2[0] += a.amp[j] * a.amp[j];
  block_sum<1>(s2, red);
  const double sig2 = s2[0];
  double v[10];
  if (MODE == R_EVAL) {
    evaluate<false>(a, th, jlo, jhi, v, red);
    if (threadIdx.x == 0) {
      a.J[c] = (v[0] * v[0] + v[1] * v[1]) / sig2;
      a.Z[2 * c] = v[0];
      a.Z[2 * c + 1] = v[1];
    }
  } else if (MODE == R_ADJOINT) {
    evaluate<true>(a, th, jlo, jhi, v, red);
    const double zr = a.Z[2 * c], zi = a.Z[2 * c + 1], g = a.dJ[c];
    if (threadIdx.x == 0)
#pragma unroll
      for (int k = 0; k < 4; ++k) a.dtheta[4 * c + k] = g * 2.0 * (zr * v[2 + 2 * k] + zi * v[3 + 2 * k]) / sig2;
  } else {
    const double scale[4] = {th[0], 1.0, 1.0 / kFref, 1.0};
    double u[4], grad[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) u[k] = th[k] / scale[k];
    evaluate<true>(a, th, jlo, jhi, v, red);
    double J = (v[0] * v[0] + v[1] * v[1]) / sig2;
#pragma unroll
    for (int k = 0; k < 4; ++k) grad[k] = 2.0 * (v[0] * v[2 + 2 * k] + v[1] * v[3 + 2 * k]) / sig2;
    double alpha = a.alpha0;
    for (int step = 0; step < a.steps; ++step) {
      double gu[4], nrm = 0.0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        gu[k] = grad[k] * scale[k];
        nrm += gu[k] * gu[k];
      }
      nrm = sqrt(nrm);
      if (!(nrm > 0.0)) continue;
      double ut[4], tt[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) ut[k] = u[k] + alpha * gu[k] / nrm;
      ut[1] = fmin(fmax(ut[1], kEtaMin), 0.25);
#pragma unroll
      for (int k = 0; k < 4; ++k) tt[k] = ut[k] * scale[k];
      evaluate<true>(a, tt, jlo, jhi, v, red);
      const double Jt = (v[0] * v[0] + v[1] * v[1]) / sig2;
      if (Jt > J) {
        J = Jt;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          u[k] = ut[k];
          grad[k] = 2.0 * (v[0] * v[2 + 2 * k] + v[1] * v[3 + 2 * k]) / sig2;
        }
        alpha = fmin(2.0 * alpha, a.alpha_max);
      } else {
        alpha *= 0.5;
      }
    }
    if (threadIdx.x == 0) {
#pragma unroll
      for (int k = 0; k < 4; ++k) a.theta_out[4 * c + k] = u[k] * scale[k];
      a.J[c] = J;
    }
  }
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

int prepare(const rb_refine_desc* d, const float* shat, const double* psd, const void* theta, int64_t n_cand,
            void* ws, size_t bytes, RefArgs& a, cudaStream_t st) {
  if (!d || !shat || !psd || !theta || n_cand < 0) {
    rb::set_detail("NULL argument or negative count");
    return RB_ERR_BAD_INPUT;
  }
  if (!rb_is_pow2(d->n) || d->n < (1 << 10) || d->n > (1 << 20) || !(d->fs > 0) || !(d->f_low > 0) ||
      !(d->pn_order == 0 || d->pn_order == 2 || d->pn_order == 3) || d->steps < 0 || !(d->alpha0 > 0) ||
      !(d->alpha_max >= d->alpha0)) {
    rb::set_detail("bad refine descriptor");
    return RB_ERR_BAD_INPUT;
  }
  const size_t need = rb_refine_workspace_bytes(d);
  if (!ws || bytes < need || ((uintptr_t)ws & 255)) {
    rb::set_detail("workspace too small: need %zu bytes", need);
    return RB_ERR_OOM;
  }
  const int64_t half = d->n / 2;
  char* base = (char*)ws;
  a.flags = (unsigned*)base;
  a.amp = (const double*)(base + 256);
  a.vf = (const double*)(base + 256 + a256(sizeof(double) * half));
  a.shat = (const float2*)shat;
  a.half = half;
  a.df = d->fs / (double)d->n;
  a.f_low = d->f_low;
  a.pn = d->pn_order;
  a.n_cand = n_cand;
  a.steps = d->steps;
  a.alpha0 = d->alpha0;
  a.alpha_max = d->alpha_max;
  RB_CUDA_TRY(cudaMemsetAsync(a.flags, 0, 256, st));
  k_refine_tables<<<(int)std::min<int64_t>(1024, (half + 255) / 256), 256, 0, st>>>(
      half, a.df, psd, (double*)a.amp, (double*)a.vf, a.flags);
  RB_LAUNCH_CHECK();
  return RB_OK;
}

template <int MODE>
int run(const RefArgs& a, cudaStream_t st) {
  if (a.n_cand > 0) {
    k_refine<MODE><<<(unsigned)a.n_cand, kThreads, 0, st>>>(a);
    RB_LAUNCH_CHECK();
  }
  unsigned flags = 0;
  RB_CUDA_TRY(cudaMemcpyAsync(&flags, a.flags, sizeof(flags), cudaMemcpyDeviceToHost, st));
  RB_CUDA_TRY(cudaStreamSynchronize(st));
  if (flags & RB_FLAG_BAD_PSD) {
    rb::set_detail("PSD not finite and positive on 0 < j < n/2");
    return RB_ERR_BAD_INPUT;
  }
  if (flags & RB_FLAG_BAD_STRAIN) {
    rb::set_detail("a candidate has mc <= 0, eta outside (0, 0.25] or a non-finite t_c / phi_c");
    return RB_ERR_BAD_INPUT;
  }
  return RB_OK;
}

}  // namespace

extern "C" {

size_t rb_refine_workspace_bytes(const rb_refine_desc* d) {
  if (!d || d->n < 2) return 0;
  return 256 + 2 * a256(sizeof(double) * (size_t)(d->n / 2));
}

int rb_refine_eval(const rb_refine_desc* d, const float* s_hat, const double* psd, const double* theta, double* J,
                   double* Z, int64_t n_cand, void* workspace, size_t workspace_bytes, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  RefArgs a{};
  int rc = prepare(d, s_hat, psd, theta, n_cand, workspace, workspace_bytes, a, st);
  if (rc) return rc;
  if (!J || !Z) {
    rb::set_detail("NULL output");
    return RB_ERR_BAD_INPUT;
  }
  a.theta_in = theta;
  a.J = J;
  a.Z = Z;
  return run<R_EVAL>(a, st);
}

int rb_refine_adjoint(const rb_refine_desc* d, const float* s_hat, const double* psd, const double* theta,
                      const double* Z, const double* dJ, double* dtheta, int64_t n_cand, void* workspace,
                      size_t workspace_bytes, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  RefArgs a{};
  int rc = prepare(d, s_hat, psd, theta, n_cand, workspace, workspace_bytes, a, st);
  if (rc) return rc;
  if (!Z || !dJ || !dtheta) {
    rb::set_detail("NULL argument");
    return RB_ERR_BAD_INPUT;
  }
  a.theta_in = theta;
  a.Z = (double*)Z;
  a.dJ = dJ;
  a.dtheta = dtheta;
  return run<R_ADJOINT>(a, st);
}

int rb_refine(const rb_refine_desc* d, const float* s_hat, const double* psd, double* theta, double* J,
              int64_t n_cand, void* workspace, size_t workspace_bytes, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  RefArgs a{};
  int rc = prepare(d, s_hat, psd, theta, n_cand, workspace, workspace_bytes, a, st);
  if (rc) return rc;
  if (!J) {
    rb::set_detail("NULL output");
    return RB_ERR_BAD_INPUT;
  }
  a.theta_in = theta;
  a.theta_out = theta;
  a.J = J;
  return run<R_ASCEND>(a, st);
}

}  // extern "C"
