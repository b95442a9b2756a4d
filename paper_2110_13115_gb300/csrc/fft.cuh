// Batched Stockham FFT building blocks for the four-step long transforms.
//
// A length-n transform is split n = n1 * n2 (four-step): with j = j1 + n1 j2 and
// m = m2 + n2 m1,
//   Y[m2 + n2 m1] = sum_j1 w_n1^(j1 m1) [ w_n^(j1 m2) sum_j2 x[j1 + n1 j2] w_n2^(j2 m2) ],
// w_L = exp(SIGN 2 pi i / L). Pass "A" does the inner length-n2 transforms (one per j1)
// and the twiddle w_n^(j1 m2); pass "B" the outer length-n1 transforms (one per m2).
// Each CTA transforms G columns at once; a column of length L is held by L/16 threads,
// 16 complex values each in registers, and radix-16/8/4/2 Stockham passes exchange
// values through shared memory (autosort: no bit reversal pass).
#pragma once
#include "common.cuh"

namespace rbfft {

constexpr int kE = 16;  // complex values per thread per column

template <int SIGN>
__device__ __forceinline__ float2 mul_i(float2 a) {  // a * (SIGN i)
  return SIGN > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// exp(SIGN i pi m / 8) as a compile-time-indexed constant
template <int SIGN, int M>
__device__ __forceinline__ float2 w16() {
  constexpr int m = M & 15;
  constexpr float c[16] = {1.0f, 0.92387953251128675613f, 0.70710678118654752440f, 0.38268343236508977173f,
                           0.0f, -0.38268343236508977173f, -0.70710678118654752440f, -0.92387953251128675613f,
                           -1.0f, -0.92387953251128675613f, -0.70710678118654752440f, -0.38268343236508977173f,
                           0.0f, 0.38268343236508977173f, 0.70710678118654752440f, 0.92387953251128675613f};
  // sin(m pi/8) = cos((m - 4) pi / 8)
  return make_float2(c[m], SIGN * c[(m + 12) & 15]);
}

template <int SIGN>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <int SIGN>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  float2 s02 = cadd(a0, a2), d02 = csub(a0, a2);
  float2 s13 = cadd(a1, a3), d13 = mul_i<SIGN>(csub(a1, a3));
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, d13);
  a3 = csub(d02, d13);
}

// y[k] = sum_r v[r] exp(SIGN 2 pi i r k / R), in place, natural order.
template <int R, int SIGN>
__device__ __forceinline__ void dft(float2* v);

template <>
__device__ __forceinline__ void dft<1, 1>(float2*) {}
template <>
__device__ __forceinline__ void dft<1, -1>(float2*) {}

template <>
__device__ __forceinline__ void dft<2, 1>(float2* v) { dft2<1>(v[0], v[1]); }
template <>
__device__ __forceinline__ void dft<2, -1>(float2* v) { dft2<-1>(v[0], v[1]); }

template <int SIGN>
__device__ __forceinline__ void dft4v(float2* v) { dft4<SIGN>(v[0], v[1], v[2], v[3]); }
template <>
__device__ __forceinline__ void dft<4, 1>(float2* v) { dft4v<1>(v); }
template <>
__device__ __forceinline__ void dft<4, -1>(float2* v) { dft4v<-1>(v); }

template <int SIGN>
__device__ __forceinline__ void dft8v(float2* v) {
  // radix-2 over two length-4 transforms of the even and odd samples
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<SIGN>(e0, e1, e2, e3);
  dft4<SIGN>(o0, o1, o2, o3);
  o1 = cmul(o1, w16<SIGN, 2>());
  o2 = mul_i<SIGN>(o2);
  o3 = cmul(o3, w16<SIGN, 6>());
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1);
  v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2);
  v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3);
  v[7] = csub(e3, o3);
}
template <>
__device__ __forceinline__ void dft<8, 1>(float2* v) { dft8v<1>(v); }
template <>
__device__ __forceinline__ void dft<8, -1>(float2* v) { dft8v<-1>(v); }

template <int SIGN>
__device__ __forceinline__ void dft16v(float2* v) {
  // 16 = 4 x 4: r = 4 r1 + r2, k = k1 + 4 k2
  // step 1: length-4 transforms over r1 for each r2, results A[r2][k1] at v[r2 + 4 k1]
#pragma unroll
  for (int r2 = 0; r2 < 4; ++r2) dft4<SIGN>(v[r2], v[r2 + 4], v[r2 + 8], v[r2 + 12]);
  // step 2: twiddles w16^(r2 k1)
  v[5] = cmul(v[5], w16<SIGN, 1>());
  v[6] = cmul(v[6], w16<SIGN, 2>());
  v[7] = cmul(v[7], w16<SIGN, 3>());
  v[9] = cmul(v[9], w16<SIGN, 2>());
  v[10] = mul_i<SIGN>(v[10]);
  v[11] = cmul(v[11], w16<SIGN, 6>());
  v[13] = cmul(v[13], w16<SIGN, 3>());
  v[14] = cmul(v[14], w16<SIGN, 6>());
  v[15] = cmul(v[15], w16<SIGN, 9>());
  // step 3: length-4 transforms over r2 for each k1; y[k1 + 4 k2] lands at v[4 k1 + k2]
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<SIGN>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  float2 t[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = t[i];
}
// dft16v for inputs whose upper half v[8..15] is zero (a one-sided spectrum's first pass): the first
// radix-4 stage reduces to (a0 + a1, a0 + SIGN i a1, a0 - a1, a0 - SIGN i a1).
template <int SIGN>
__device__ __forceinline__ void dft16_half(float2* v) {
#pragma unroll
  for (int r2 = 0; r2 < 4; ++r2) {
    const float2 a0 = v[r2], a1 = v[r2 + 4];
    const float2 ia1 = mul_i<SIGN>(a1);
    v[r2] = cadd(a0, a1);
    v[r2 + 4] = cadd(a0, ia1);
    v[r2 + 8] = csub(a0, a1);
    v[r2 + 12] = csub(a0, ia1);
  }
  v[5] = cmul(v[5], w16<SIGN, 1>());
  v[6] = cmul(v[6], w16<SIGN, 2>());
  v[7] = cmul(v[7], w16<SIGN, 3>());
  v[9] = cmul(v[9], w16<SIGN, 2>());
  v[10] = mul_i<SIGN>(v[10]);
  v[11] = cmul(v[11], w16<SIGN, 6>());
  v[13] = cmul(v[13], w16<SIGN, 3>());
  v[14] = cmul(v[14], w16<SIGN, 6>());
  v[15] = cmul(v[15], w16<SIGN, 9>());
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<SIGN>(v[4 * k1], v[4 * k1 + 1], v[4 * k1 + 2], v[4 * k1 + 3]);
  float2 t[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = v[4 * k1 + k2];
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = t[i];
}

template <>
__device__ __forceinline__ void dft<16, 1>(float2* v) { dft16v<1>(v); }
template <>
__device__ __forceinline__ void dft<16, -1>(float2* v) { dft16v<-1>(v); }

// Radix plan for a column length L (power of two, 16..2048): up to three passes.
template <int L>
struct Radix {
  static constexpr int r0 = L >= 16 ? 16 : L;
  static constexpr int l1 = L / r0;
  static constexpr int r1 = l1 >= 16 ? 16 : l1;
  static constexpr int l2 = l1 / r1;
  static constexpr int r2 = l2;  // 1, 2, 4 or 8
  static_assert(r2 <= 16, "column length too long");
};

// Powers t[r] = w^r, r = 1..R-1, of one table twiddle w by binary powering (depth <= 4 products
// for R = 16), so a butterfly reads one table entry instead of R - 1.
template <int R>
__device__ __forceinline__ void twiddle_powers(float2 w, float2 (&t)[R]) {
  t[1] = w;
  if constexpr (R > 2) {
    t[2] = cmul(w, w);
    t[3] = cmul(t[2], w);
  }
  if constexpr (R > 4) {
    t[4] = cmul(t[2], t[2]);
    t[5] = cmul(t[4], w);
    t[6] = cmul(t[4], t[2]);
    t[7] = cmul(t[4], t[3]);
  }
  if constexpr (R > 8) {
    t[8] = cmul(t[4], t[4]);
#pragma unroll
    for (int r = 9; r < 16; ++r) t[r] = cmul(t[8], t[r - 8]);
  }
}

// One Stockham pass of radix R after passes whose radices multiply to NS.
// In:  v[b R + r] = x[j_b + r L/R];  Out: v[b R + r] = y[(j_b/NS) NS R + j_b % NS + r NS],
// with j_b = tj + b (L/kE). tw[e] = exp(+2 pi i e / L).
template <int SIGN, int L, int R, int NS>
__device__ __forceinline__ void radix_pass(float2 (&v)[kE], int tj, const float2* tw) {
#pragma unroll
  for (int b = 0; b < kE / R; ++b) {
    if constexpr (NS > 1) {
      const int j = tj + b * (L / kE);
      const int jm = j & (NS - 1);
      float2 w = tw[jm * (L / (NS * R))];  // exp(2 pi i jm / (NS R))
      if (SIGN < 0) w.y = -w.y;
      float2 t[R];
      twiddle_powers<R>(w, t);
#pragma unroll
      for (int r = 1; r < R; ++r) v[b * R + r] = cmul(v[b * R + r], t[r]);
    }
    dft<R, SIGN>(&v[b * R]);
  }
}

template <int L, int R>
__device__ __forceinline__ int in_pos(int tj, int b, int r) {
  return tj + b * (L / kE) + r * (L / R);
}
template <int L, int R, int NS>
__device__ __forceinline__ int out_pos(int tj, int b, int r) {
  const int j = tj + b * (L / kE);
  return (j / NS) * NS * R + (j & (NS - 1)) + r * NS;
}

// Shared-memory slot of (point, column) for G columns; padded every 32 points.
template <int G>
__device__ __forceinline__ int sidx(int point, int c) {
  return point * G + c + (point >> 5);
}
template <int L, int G>
struct Smem {
  static constexpr int data = L * G + L / 32 + 1;  // float2 slots
};

// The whole column transform: pass 0 reads through `load(point)`, the last pass leaves
// v[b Rl + r] holding output point out_pos<L, Rl, NSl>(tj, b, r). Returns via v.
// HALF: the input points >= L/2 are zero (a one-sided spectrum); with a first pass of radix 16 that
// holds all of a thread's points (R0 = kE), they are exactly the thread's r >= 8 and are neither
// loaded nor added.
template <int SIGN, int L, int G, bool HALF = false, class Load>
__device__ __forceinline__ void column_transform(float2 (&v)[kE], int c, int tj, float2* sdata,
                                                 const float2* tw, Load load) {
  using P = Radix<L>;
  constexpr int R0 = P::r0, R1 = P::r1, R2 = P::r2;
  if constexpr (HALF && R0 == kE && R0 == 16) {
#pragma unroll
    for (int r = 0; r < R0; ++r) v[r] = r < R0 / 2 ? load(in_pos<L, R0>(tj, 0, r)) : make_float2(0.f, 0.f);
    dft16_half<SIGN>(v);
  } else {
#pragma unroll
    for (int b = 0; b < kE / R0; ++b)
#pragma unroll
      for (int r = 0; r < R0; ++r) v[b * R0 + r] = load(in_pos<L, R0>(tj, b, r));
    radix_pass<SIGN, L, R0, 1>(v, tj, tw);
  }
  if constexpr (R1 > 1) {
    __syncthreads();
#pragma unroll
    for (int b = 0; b < kE / R0; ++b)
#pragma unroll
      for (int r = 0; r < R0; ++r) sdata[sidx<G>(out_pos<L, R0, 1>(tj, b, r), c)] = v[b * R0 + r];
    __syncthreads();
#pragma unroll
    for (int b = 0; b < kE / R1; ++b)
#pragma unroll
      for (int r = 0; r < R1; ++r) v[b * R1 + r] = sdata[sidx<G>(in_pos<L, R1>(tj, b, r), c)];
    radix_pass<SIGN, L, R1, R0>(v, tj, tw);
  }
  if constexpr (R2 > 1) {
    __syncthreads();
#pragma unroll
    for (int b = 0; b < kE / R1; ++b)
#pragma unroll
      for (int r = 0; r < R1; ++r) sdata[sidx<G>(out_pos<L, R1, R0>(tj, b, r), c)] = v[b * R1 + r];
    __syncthreads();
#pragma unroll
    for (int b = 0; b < kE / R2; ++b)
#pragma unroll
      for (int r = 0; r < R2; ++r) v[b * R2 + r] = sdata[sidx<G>(in_pos<L, R2>(tj, b, r), c)];
    radix_pass<SIGN, L, R2, R0 * R1>(v, tj, tw);
  }
}

// Radix and stride of the last pass, for mapping v[] to output points.
template <int L>
struct LastPass {
  using P = Radix<L>;
  static constexpr int R = P::r2 > 1 ? P::r2 : (P::r1 > 1 ? P::r1 : P::r0);
  static constexpr int NS = P::r2 > 1 ? P::r0 * P::r1 : (P::r1 > 1 ? P::r0 : 1);
};

template <int L>
__device__ __forceinline__ int final_point(int tj, int b, int r) {
  return out_pos<L, LastPass<L>::R, LastPass<L>::NS>(tj, b, r);
}

}  // namespace rbfft
