// Shared device helpers for the sm_103a hot path (complex arithmetic, status words).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rbmf.h"

#define RB_CUDA_TRY(expr)                                   \
  do {                                                      \
    cudaError_t _e = (expr);                                \
    if (_e != cudaSuccess) {                                \
      rb_set_last_cuda_error(_e, #expr, __FILE__, __LINE__); \
      return RB_ERR_CUDA;                                   \
    }                                                       \
  } while (0)

void rb_count_launch();

#define RB_LAUNCH_CHECK()                                                     \
  do {                                                                        \
    rb_count_launch();                                                        \
    cudaError_t _e = cudaGetLastError();                                      \
    if (_e != cudaSuccess) {                                                  \
      rb_set_last_cuda_error(_e, "kernel launch", __FILE__, __LINE__);        \
      return RB_ERR_CUDA;                                                     \
    }                                                                         \
  } while (0)

void rb_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// Device status words (in workspace): bad input, overflow counters.
enum { RB_FLAG_BAD_PSD = 1, RB_FLAG_BAD_STRAIN = 2, RB_FLAG_TIMEOUT = 4, RB_FLAG_CAND_OVERFLOW = 8 };

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

static inline int rb_ilog2(int64_t x) {
  int r = 0;
  while ((int64_t(1) << r) < x) ++r;
  return r;
}
static inline bool rb_is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }
