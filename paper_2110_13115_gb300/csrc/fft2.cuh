// Radix-32 building blocks for the four-step passes of the long inverse transforms (n >= 2^16).
//
// A column of length L (256, 512 or 1024) is held by S = L/32 threads with 32 complex values each
// and transformed in two register stages with one shared-memory exchange between them:
//   stage 1: thread tj takes x[tj + S r] (r < 32) and does a length-32 DFT, giving y1[32 tj + k];
//   stage 2: butterfly j (j < 32; thread tj owns j = tj + S b, b < 32/S) takes y1[j + 32 r'],
//            r' < S, multiplies by w_L^(j r') and does a length-S DFT, giving Y[j + 32 k'].
// Every shared-memory and twiddle-table address is a per-thread base plus a compile-time offset.
#pragma once
#include "common.cuh"
#include "fft.cuh"

namespace rbfft2 {

using rbfft::mul_i;

// exp(SIGN 2 pi i K / 32) as a compile-time constant
template <int SIGN, int K>
__device__ __forceinline__ float2 w32() {
  constexpr int k = K & 31;
  constexpr float c[32] = {1.0f,
                           0.98078528040323044913f,
                           0.92387953251128675613f,
                           0.83146961230254523708f,
                           0.70710678118654752440f,
                           0.55557023301960222474f,
                           0.38268343236508977173f,
                           0.19509032201612826785f,
                           0.0f,
                           -0.19509032201612826785f,
                           -0.38268343236508977173f,
                           -0.55557023301960222474f,
                           -0.70710678118654752440f,
                           -0.83146961230254523708f,
                           -0.92387953251128675613f,
                           -0.98078528040323044913f,
                           -1.0f,
                           -0.98078528040323044913f,
                           -0.92387953251128675613f,
                           -0.83146961230254523708f,
                           -0.70710678118654752440f,
                           -0.55557023301960222474f,
                           -0.38268343236508977173f,
                           -0.19509032201612826785f,
                           0.0f,
                           0.19509032201612826785f,
                           0.38268343236508977173f,
                           0.55557023301960222474f,
                           0.70710678118654752440f,
                           0.83146961230254523708f,
                           0.92387953251128675613f,
                           0.98078528040323044913f};
  // sin(2 pi k / 32) = cos(2 pi (k - 8) / 32)
  return make_float2(c[k], SIGN * c[(k + 24) & 31]);
}

// a * exp(SIGN 2 pi i K / 32), with the multiplications by 1, +-i and (+-1 +- i)/sqrt(2) spelled out
template <int SIGN, int K>
__device__ __forceinline__ float2 rot32(float2 a) {
  constexpr int k = K & 31;
  if constexpr (k == 0) {
    return a;
  } else if constexpr (k == 8) {
    return mul_i<SIGN>(a);
  } else if constexpr (k == 16) {
    return make_float2(-a.x, -a.y);
  } else if constexpr (k == 24) {
    return mul_i<-SIGN>(a);
  } else if constexpr ((k & 7) == 4) {
    // (c + i s) with |c| = |s| = 1/sqrt(2)
    constexpr float h = 0.70710678118654752440f;
    const float2 w = w32<SIGN, k>();
    const float cr = w.x > 0.f ? h : -h, ci = w.y > 0.f ? h : -h;
    return make_float2(cr * a.x - ci * a.y, cr * a.y + ci * a.x);
  } else {
    const float2 w = w32<SIGN, k>();
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
  }
}

// y[k] = sum_{r<R} v[r] exp(SIGN 2 pi i r k / R) for R in {4, 8, 16}: the existing kernels.
template <int R, int SIGN>
__device__ __forceinline__ void dft_small(float2* v) {
  rbfft::dft<R, SIGN>(v);
}

// Length-32 DFT in place, natural order: DFTs of the even and the odd samples, then
// y[k] = E[k] + w^k O[k], y[k + 16] = E[k] - w^k O[k]. HALF: v[16..31] are zero (a one-sided
// spectrum), so both length-16 DFTs see a zero upper half.
template <int SIGN, bool HALF = false>
__device__ __forceinline__ void dft32(float2 (&v)[32]) {
  float2 e[16], o[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    e[r] = v[2 * r];
    o[r] = v[2 * r + 1];
  }
  if constexpr (HALF) {
    rbfft::dft16_half<SIGN>(e);
    rbfft::dft16_half<SIGN>(o);
  } else {
    rbfft::dft<16, SIGN>(e);
    rbfft::dft<16, SIGN>(o);
  }
  float2 t[16];
  t[0] = o[0];
#define RB_ROT(K) t[K] = rot32<SIGN, K>(o[K]);
  RB_ROT(1) RB_ROT(2) RB_ROT(3) RB_ROT(4) RB_ROT(5) RB_ROT(6) RB_ROT(7) RB_ROT(8)
  RB_ROT(9) RB_ROT(10) RB_ROT(11) RB_ROT(12) RB_ROT(13) RB_ROT(14) RB_ROT(15)
#undef RB_ROT
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    v[k] = cadd(e[k], t[k]);
    v[k + 16] = csub(e[k], t[k]);
  }
}

// Full DFT of length R in {8, 16, 32} on v[0..R).
template <int R, int SIGN>
__device__ __forceinline__ void dft_r(float2* v) {
  if constexpr (R == 32) {
    float2(&a)[32] = *reinterpret_cast<float2(*)[32]>(v);
    dft32<SIGN>(a);
  } else {
    rbfft::dft<R, SIGN>(v);
  }
}

// Upper half of a length-R DFT (R in {8, 16, 32}): on return v[R/2 + k] = y[R/2 + k] for
// k < R/2 (the lower half of v is left undefined). y[R/2 + k] = E[k] - w_R^k O[k] with E, O the
// length-R/2 DFTs of the even and odd samples.
template <int R, int SIGN>
__device__ __forceinline__ void dft_upper(float2* v) {
  constexpr int H = R / 2;
  float2 e[H], o[H];
#pragma unroll
  for (int r = 0; r < H; ++r) {
    e[r] = v[2 * r];
    o[r] = v[2 * r + 1];
  }
  dft_r<H, SIGN>(e);
  dft_r<H, SIGN>(o);
#pragma unroll
  for (int k = 0; k < H; ++k) {
    float2 t;
    // w_R^k = w_32^(k 32 / R)
    switch ((k * (32 / R)) & 31) {
#define RB_CASE(K) \
  case K:          \
    t = rot32<SIGN, K>(o[k]); \
    break;
      RB_CASE(0) RB_CASE(1) RB_CASE(2) RB_CASE(3) RB_CASE(4) RB_CASE(5) RB_CASE(6) RB_CASE(7)
      RB_CASE(8) RB_CASE(9) RB_CASE(10) RB_CASE(11) RB_CASE(12) RB_CASE(13) RB_CASE(14) RB_CASE(15)
#undef RB_CASE
      default: t = o[k]; break;
    }
    v[H + k] = csub(e[k], t);
  }
}

template <int L>
struct Col {
  static constexpr int S = L / 32;  // threads per column = stage-2 radix
  static constexpr int NB = 32 / S; // stage-2 butterflies per thread
  static_assert(L == 256 || L == 512 || L == 1024, "radix-32 columns of 256, 512 or 1024 points");
};

// Shared-memory slot (float2 units) of point p of column c: columns interleaved, one padding point
// after every 32, which keeps both the stage-1 stores (p = 32 tj + k) and the stage-2 loads
// (p = j + 32 r') free of bank conflicts for G in {4, 8, 16, 32}.
template <int G>
__device__ __forceinline__ int slot(int p, int c) {
  return G * (p + (p >> 5)) + c;
}
template <int L, int G>
constexpr int exchange_slots() {
  return G * (L + L / 32);
}

// The column transform from registers (stage-1 inputs v[r] = x[tj + S r]) to registers (stage-2
// outputs); tw2 (global memory, read through the L1 cache) holds tw2[j (S + 1) + r'] = w_L^(j r')
// (SIGN = +1). UPPER: only the upper half of each stage-2 butterfly's outputs is formed
// (v[b S + k'] for k' >= S/2).
// TWR: the stage-2 twiddles of a butterfly are powers of its first one, w_L^j, formed by a running
// product (one table value per butterfly) instead of one table value each.
template <int SIGN, int L, int G, bool HALF, bool UPPER, bool TWR = false>
__device__ __forceinline__ void column32(float2 (&v)[32], int c, int tj, float2* xbuf,
                                         const float2* __restrict__ tw2) {
  static_assert(SIGN == 1, "the stage-2 table holds the inverse transform's twiddles");
  constexpr int S = Col<L>::S, NB = Col<L>::NB;
  dft32<SIGN, HALF>(v);
  // exchange: y1[32 tj + k] out, y1[j + 32 r'] in (j = tj + S b)
  float2* wbase = xbuf + G * 33 * tj + c;
#pragma unroll
  for (int k = 0; k < 32; ++k) wbase[G * k] = v[k];
  __syncthreads();
  const float2* rbase = xbuf + G * tj + c;
#pragma unroll
  for (int b = 0; b < NB; ++b)
#pragma unroll
    for (int r = 0; r < S; ++r) v[b * S + r] = rbase[G * (S * b + 33 * r)];
  const float2* tbase = tw2 + tj * (S + 1);
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if constexpr (TWR) {
      const float2 w1 = __ldg(tbase + S * b * (S + 1) + 1);
      float2 t = w1;
#pragma unroll
      for (int r = 1; r < S; ++r) {
        v[b * S + r] = cmul(v[b * S + r], t);
        t = cmul(t, w1);
      }
    } else {
#pragma unroll
      for (int r = 1; r < S; ++r) v[b * S + r] = cmul(v[b * S + r], __ldg(tbase + S * b * (S + 1) + r));
    }
    if constexpr (UPPER)
      dft_upper<S, SIGN>(&v[b * S]);
    else
      dft_r<S, SIGN>(&v[b * S]);
  }
}

}  // namespace rbfft2
