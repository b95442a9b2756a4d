// Second stage on tcgen05 tensor cores (arXiv:2110.13115 Sec. III.C second stage, Sec. III.E custom
// kernel): for the records of one group of G = 16 / w bins (a record: one template's candidate bins
// within the group, as a bin mask), z_t[m] = sum_k conj(a_tk) beta_k[m] over the group's S = 16
// samples as one real contraction D[128 records][2N] = A[128][K] . B[K][2N] (N = 2S) with
//   A row  = [Re a_t | Im a_t] (K = 2 k16, FP16 hi and lo planes from rb_pack_coeff, in its column order)
//   B[kk][2r] = Re beta_kk[r] / Im beta_(kk-k16)[r],  B[kk][2r+1] = Im beta_kk[r] / -Re beta_(kk-k16)[r]
// (the first / second half of K) in FP16 hi (columns 0..N-1) and lo (columns N..2N-1), so
// D[., 2r] + D[., N + 2r] and D[., 2r+1] + D[., N + 2r+1] are Re and Im of z at sample r.
// Two products per K step, A_hi . [B_hi | B_lo] and A_lo . [B_hi | B_lo], with FP32 accumulation in
// tensor memory: the split terms hi.hi + hi.lo + lo.hi (+ lo.lo), FP32-accurate.
//
// The arg-max over each bin of a record's mask is reported when |z| >= rho_II. Reading a coefficient
// row once for all of a template's candidate bins of the group cuts the gathers by the number of
// candidates per record (about 1.8 on clustered candidates at w = 8).
// Persistent kernel, one CTA per SM, 544 threads, over the pieces (up to 256 records of one group by
// default, dealt round-robin to the CTAs) that the bucketing produced:
//   warps 0-3  : coefficient producers. Per tile of 128 candidates each warp gathers the coefficient
//                rows of its 32 candidates, K block by K block, with cp.async into an S-deep ring
//                (S = 2..6, as many 32-KB stages as shared memory holds); a stage is published to the
//                MMA by cp.async.mbarrier.arrive when its copies land, so no producer waits on them.
//                The template index of the next tile and the record of the next piece are loaded
//                one tile ahead.
//   warp 4     : tensor-memory allocation and the MMA issuer (one thread), two tiles in flight.
//   warps 5-8  : epilogue: one tensor-memory lane quarter each; arg-max over each bin of the record's
//                mask, rho_II, triggers.
//   warps 9-16 : window producers: the group's B operand (hi and lo windows side by side, 128-byte
//                swizzled K-major), double-buffered, so a piece's window is built while the one before runs.
// Every mbarrier wait is bounded (1 s); a timeout sets RB_FLAG_TIMEOUT and every role stops; copies
// and products in flight are waited for (bounded) and tensor memory is freed before the CTA exits.
//
// Neither the tensor pipe nor L2 is saturated (about a fifth of each on the 10,000-template block):
// the pace is set by the balance of the CTAs' walk over the pieces and by the window builds (one per
// piece), the gathers' round trips through the ring (three 32-KB stages beside the two 56-KB windows
// at k <= 256) overlapping them.
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "internal.h"
#include "tma.cuh"

namespace {

using namespace rbtma;

constexpr int kBM = 128;          // candidates per tile (tensor-memory lanes)
constexpr int kKB = 64;           // K block: 64 FP16 = one 128-byte swizzled row
constexpr int kMaxStagesA = 6;    // coefficient ring depth, at most
constexpr int kAStageBytes = 2 * kBM * 128;
constexpr int kWinThreads = 256;  // window producers (8 warps)
constexpr int kThreadsTc = 288 + kWinThreads;  // 4 + 1 + 4 warps, then the window producers
constexpr unsigned kFull = 0xffffffffu;

struct S2Params {
  const __half* ahi;   // [T][2 k16] coefficient planes (packed column order)
  const __half* alo;
  const float2* beta;  // [k][half] valid half
  int k, k16, kp2, nkb;  // kp2 = 2 k16 rounded up to kKB, nkb = kp2 / kKB
  int stages;            // coefficient ring depth
  int nbuf;              // window buffers (2: a piece's window is built while the one before runs)
  int T;
  int64_t half;
  int bin0;
  const int4* pieces;
  const unsigned* piece_total;
  const rb::SortedCand* sorted;
  float thr2;
  int64_t sample_offset;
  rb_trigger* trig;
  unsigned long long* counter;
  int64_t cap;
  unsigned* flags;
  uint32_t idesc;
  int withhold_copies;  // failure-detection test: the producers issue no copy (rbx_stage2_withhold_copies)
  int tmpl_base;        // added to a trigger's template row (sub-banks filtered into one list)
};

// Byte offset of element e (0..63) of row `row` in a 128-byte swizzled K-major tile.
__device__ __forceinline__ uint32_t sw128_off(int row, int e) {
  return (uint32_t)(row * 128 + ((((e >> 3) ^ (row & 7))) << 4) + ((e & 7) << 1));
}

// One arrival on `bar` once every cp.async this thread issued so far has landed (the barrier's
// expected count includes it); the thread itself does not wait.
__device__ __forceinline__ void cp_async_arrive(uint64_t* bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(saddr(bar)) : "memory");
}

__device__ __forceinline__ int4 piece_at(const S2Params& p, unsigned i, unsigned n) {
  return i < n ? p.pieces[i] : make_int4(0, 0, 0, 0);
}

__device__ __forceinline__ int tiles_of(const int4& pc) { return (int)(((unsigned)pc.z - (unsigned)pc.y + kBM - 1) / kBM); }

template <int W, int N>
__global__ void __launch_bounds__(kThreadsTc, 1) k_stage2_tc(S2Params p) {
  constexpr int S = N / 2, G = S / W;  // samples and bins of a group
  static_assert(G * W == S && G >= 1 && G <= 32 && N % 32 == 0 && 16 % W == 0, "a group is a whole number of bins");
  constexpr int N2 = 2 * N;  // B rows: hi window in 0..N-1, lo window in N..2N-1
  extern __shared__ uint8_t dsm[];
  __shared__ __align__(8) uint64_t afull[kMaxStagesA], aempty[kMaxStagesA], bfull[2], bempty[2], tfull[2], tempty[2],
      drain;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr uint32_t kAcc = N2;                          // tensor-memory columns of one tile
  constexpr uint32_t kCols = 2 * kAcc < 32 ? 32 : 2 * kAcc;  // two tiles in flight
  static_assert(kCols <= 512 && (kCols & (kCols - 1)) == 0, "tensor-memory columns");
  const uint32_t base = (saddr(dsm) + 1023u) & ~1023u;
  constexpr uint32_t A_PLANE = kBM * 128, A_STAGE = kAStageBytes;
  const int NS = p.stages;
  const uint32_t b_tile = N2 * 128, b_buf = (uint32_t)p.nkb * b_tile;
  const uint32_t a0 = base, b0 = base + NS * A_STAGE;
  uint8_t* const gen = dsm + (base - saddr(dsm));  // generic pointer to `base`

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&afull[s], 128);
      mbar_init(&aempty[s], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bfull[i], kWinThreads);
      mbar_init(&bempty[i], 1);
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 4);
    }
    mbar_init(&drain, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const unsigned npieces = *p.piece_total, grid = gridDim.x;
  auto fail = [&]() {
    abort_flag = 1;
    atomicOr(p.flags, (unsigned)RB_FLAG_TIMEOUT);
  };

  if (warp < 4) {
    // ---------------- coefficient producers
    const int tid = threadIdx.x;  // 0..127: the candidate row of every tile
    const int64_t p2 = 2 * (int64_t)p.k16;
    unsigned g = 0;  // K blocks issued so far
    auto tmpl_at = [&](const int4& pc, int tile) {
      const unsigned ci = (unsigned)pc.y + tile * kBM + tid;
      int t = ci < (unsigned)pc.z ? p.sorted[ci].tmpl : -1;
      return t >= p.T ? -1 : t;
    };
    unsigned pc_i = blockIdx.x;
    int4 pc = piece_at(p, pc_i, npieces), pcn = piece_at(p, pc_i + grid, npieces);
    int tile = 0;
    int t = pc_i < npieces ? tmpl_at(pc, 0) : -1;
    // (withhold_copies: no copy and no arrival at all, so the MMA thread's first wait runs out)
    while (pc_i < npieces && !p.withhold_copies && !__any_sync(kFull, abort_flag != 0)) {
      // the next tile, and its template, before this tile's copies
      const bool same = tile + 1 < tiles_of(pc);
      const unsigned nx_i = same ? pc_i : pc_i + grid;
      const int nx_tile = same ? tile + 1 : 0;
      const int t_next = nx_i < npieces ? tmpl_at(same ? pc : pcn, nx_tile) : -1;
      // 8 lanes per row: one warp instruction copies 4 whole 128-byte lines; the warp covers its
      // 32 rows (its own candidates) in 8 instructions per plane
      const __half* rowp[8];
      bool rv[8];
#pragma unroll
      for (int it = 0; it < 8; ++it) {
        const int tr = __shfl_sync(kFull, t, 4 * it + (lane >> 3));
        rv[it] = tr >= 0;
        rowp[it] = p.ahi + (int64_t)max(tr, 0) * p2 + (lane & 7) * 8;
      }
      const int64_t lo_off = (int64_t)p.T * p2;
      bool ok = true;
      for (int kb = 0; kb < p.nkb; ++kb, ++g) {
        const uint32_t s = g % NS, ph = (g / NS) & 1;
        // every lane waits; the outcome is made warp-uniform before the warp-wide steps below
        if (!__all_sync(kFull, mbar_wait(&aempty[s], ph ^ 1, &abort_flag))) {
          if (lane == 0) fail();
          ok = false;
          break;
        }
        const uint32_t dst = a0 + s * A_STAGE;
        const int col = kb * kKB + (lane & 7) * 8;  // first FP16 element of this lane's 16-byte chunk
#pragma unroll
        for (int it = 0; it < 8; ++it) {
          const bool v = rv[it] && col < 2 * p.k16;
          const uint32_t off = sw128_off(32 * warp + 4 * it + (lane >> 3), (lane & 7) * 8);
          const __half* src = rowp[it] + (v ? kb * kKB : 0);
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst + off), "l"(src), "r"(v ? 16 : 0)
                       : "memory");
          asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst + A_PLANE + off), "l"(src + lo_off),
                       "r"(v ? 16 : 0)
                       : "memory");
        }
        cp_async_arrive(&afull[s]);  // the stage is published when its copies land
      }
      if (!ok) break;
      if (!same) {
        pc = pcn;
        pcn = piece_at(p, nx_i + grid, npieces);
      }
      pc_i = nx_i;
      tile = nx_tile;
      t = t_next;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp == 4) {
    // ---------------- MMA issuer
    if (lane == 0) {
      unsigned g = 0, gt = 0, i = 0;
      bool issued = false;
      int4 pcn = piece_at(p, blockIdx.x, npieces);
      for (unsigned pc_i = blockIdx.x; pc_i < npieces && !abort_flag; pc_i += grid, ++i) {
        const int4 pc = pcn;
        pcn = piece_at(p, pc_i + grid, npieces);
        const int pb = i % p.nbuf;
        if (!mbar_wait(&bfull[pb], (i / p.nbuf) & 1, &abort_flag)) {
          fail();
          break;
        }
        tc_fence_after();
        const uint32_t bt = b0 + pb * b_buf;
        const int ntiles = tiles_of(pc);
        bool ok = true;
        for (int tile = 0; tile < ntiles && ok; ++tile, ++gt) {
          const int acc = gt & 1;
          if (!mbar_wait(&tempty[acc], ((gt >> 1) & 1) ^ 1, &abort_flag)) {
            fail();
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)acc * kAcc;
          for (int kb = 0; kb < p.nkb; ++kb, ++g) {
            const uint32_t s = g % NS, ph = (g / NS) & 1;
            if (!mbar_wait(&afull[s], ph, &abort_flag)) {
              fail();
              ok = false;
              break;
            }
            tc_fence_after();
            fence_async_smem();  // the stage's cp.async (generic proxy) writes before the products read it
            const uint32_t ah = a0 + s * A_STAGE, al = ah + A_PLANE;
            const uint32_t bk = bt + kb * b_tile;
#pragma unroll
            for (int kk = 0; kk < kKB / 16; ++kk) {
              const uint32_t off = kk * 32;
              tc_mma(d, sw128_desc(ah + off), sw128_desc(bk + off), p.idesc, (kb | kk) != 0);
              tc_mma(d, sw128_desc(al + off), sw128_desc(bk + off), p.idesc, 1);
            }
            issued = true;
            tc_commit(&aempty[s]);
          }
          if (!ok) break;
          tc_commit(&tfull[acc]);
        }
        if (!ok) break;
        tc_commit(&bempty[pb]);
      }
      if (issued) {
        // every product issued so far has completed before tensor memory is released
        tc_commit(&drain);
        const uint64_t t0 = gtimer();
        while (!mbar_try(&drain, 0) && gtimer() - t0 < kWaitNs) {
        }
      }
    }
  } else if (warp < 9) {
    // ---------------- epilogue: warp 5..8 reads tensor-memory lanes 32 (warp % 4) + [0, 32)
    const int q = warp & 3;
    unsigned gt = 0;
    bool stop = false;
    int4 pcn = piece_at(p, blockIdx.x, npieces);
    for (unsigned pc_i = blockIdx.x; pc_i < npieces && !stop; pc_i += grid) {
      const int4 pc = pcn;
      pcn = piece_at(p, pc_i + grid, npieces);
      const int grp = pc.x;
      const unsigned c0 = (unsigned)pc.y, c1 = (unsigned)pc.z;
      const int ntiles = tiles_of(pc);
      for (int tile = 0; tile < ntiles; ++tile, ++gt) {
        const unsigned ci = c0 + tile * kBM + q * 32 + lane;
        rb::SortedCand cd{-1, 0, 0u};
        if (ci < c1) cd = p.sorted[ci];
        const int acc = gt & 1;
        if (!__all_sync(kFull, mbar_wait(&tfull[acc], (gt >> 1) & 1, &abort_flag))) {
          if (lane == 0) fail();
          stop = true;
          break;
        }
        tc_fence_after();
        // columns 0..N-1: products against the hi window, N..2N-1: against the lo window; read 32
        // columns (16 samples, 16 / W bins) of each at a time
        const uint32_t row = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)acc * kAcc;
#pragma unroll
        for (int h = 0; h < N / 32; ++h) {
          float vh[32], vl[32];
          tc_ld32(row + 32 * h, vh);
          tc_ld32(row + N + 32 * h, vl);
          if (h == N / 32 - 1) {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
          }
#pragma unroll
          for (int j = h * (16 / W); j < (h + 1) * (16 / W); ++j) {
            float best = -1.f, zr = 0.f, zi = 0.f;
            int br = 0;
#pragma unroll
            for (int r = j * W; r < (j + 1) * W; ++r) {
              const int c = 2 * (r - 16 * h);
              const float re = vh[c] + vl[c], im = vh[c + 1] + vl[c + 1];
              const float p2s = fmaf(re, re, im * im);
              if (p2s > best) {
                best = p2s;
                br = r - j * W;
                zr = re;
                zi = im;
              }
            }
            const bool emit = ci < c1 && ((cd.mask >> j) & 1u) && best >= p.thr2;
            const unsigned em = __ballot_sync(kFull, emit);
            if (!em) continue;
            const int leader = __ffs(em) - 1;
            unsigned long long b0c = 0;
            if (lane == leader) b0c = atomicAdd(p.counter, (unsigned long long)__popc(em));
            b0c = __shfl_sync(kFull, b0c, leader);
            if (emit) {
              const unsigned long long idx = b0c + __popc(em & ((1u << lane) - 1u));
              if ((int64_t)idx < p.cap) {
                rb_trigger tg;
                tg.sample = p.sample_offset + (int64_t)(p.bin0 + grp * G + j) * W + br;
                tg.tmpl = p.tmpl_base + cd.tmpl;
                tg.block = cd.block;
                tg.snr = sqrtf(best);
                tg.phase = atan2f(zi, zr);
                p.trig[idx] = tg;
              }
            }
          }
        }
      }
    }
  } else {
    // ---------------- window producers: B operand of each piece's bin, double-buffered
    const int tid = threadIdx.x - 9 * 32;  // 0..kWinThreads-1
    // zero both B buffers once: positions >= 2 k16 are never written again
    for (uint32_t o = tid * 16; o < p.nbuf * b_buf; o += kWinThreads * 16)
      *reinterpret_cast<uint4*>(gen + (b0 - base) + o) = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("bar.sync 1, %0;" ::"n"(kWinThreads) : "memory");
    // one work item: the 16-byte chunk of packed positions 8 ch .. 8 ch + 7 (eight K columns) for
    // sample r, both parts (B rows 2r and 2r + 1), hi and lo: eight beta loads, four 16-byte stores
    const int nchunk = 2 * p.k16 / 8, total = nchunk * S;
    int4 pcn = piece_at(p, blockIdx.x, npieces);
    unsigned i = 0;
    for (unsigned pc_i = blockIdx.x; pc_i < npieces && !abort_flag; pc_i += grid, ++i) {
      const int grp = pcn.x;
      pcn = piece_at(p, pc_i + grid, npieces);
      const int pb = i % p.nbuf;
      if (!mbar_wait(&bempty[pb], ((i / p.nbuf) & 1) ^ 1, &abort_flag)) {
        fail();
        break;
      }
      const int64_t m0 = (int64_t)grp * S;  // valid-half index of the group's first sample
      uint8_t* bt = gen + (b0 - base) + pb * b_buf;
      constexpr int U = 2;
      for (int i0 = tid; i0 < total; i0 += U * kWinThreads) {
        float2 bv[U][8];
#pragma unroll
        for (int u = 0; u < U; ++u) {  // loads first, then the stores (zero past the valid half)
          const int idx = i0 + u * kWinThreads, ch = idx / S, r = idx - ch * S;
          const bool in = idx < total && m0 + r < p.half;
#pragma unroll
          for (int sl = 0; sl < 8; ++sl) {
            // packed position 8 ch + sl holds column (2 q + sl / 4) 16 + 2 t4 + (sl & 1) + 8 ((sl >> 1) & 1)
            const int q = ch >> 2, t4 = ch & 3;
            const int col = (2 * q + (sl >> 2)) * 16 + 2 * t4 + (sl & 1) + 8 * ((sl >> 1) & 1);
            const int kk = col < p.k16 ? col : col - p.k16;
            bv[u][sl] = in && kk < p.k ? __ldg(p.beta + (int64_t)kk * p.half + m0 + r) : make_float2(0.f, 0.f);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = i0 + u * kWinThreads, ch = idx / S, r = idx - ch * S;
          if (idx >= total) break;
          const int q = ch >> 2, t4 = ch & 3;
          uint32_t h[2][4], l[2][4];  // [part][pair of halves]
#pragma unroll
          for (int sl = 0; sl < 8; sl += 2) {
            __half hv[2][2], lv[2][2];
#pragma unroll
            for (int o = 0; o < 2; ++o) {
              const int e = sl + o;
              const int col = (2 * q + (e >> 2)) * 16 + 2 * t4 + (e & 1) + 8 * ((e >> 1) & 1);
              const float2 v = bv[u][e];
              // Re half: (Re, Im) of beta; Im half: (Im, -Re)
              const float x0 = col < p.k16 ? v.x : v.y, x1 = col < p.k16 ? v.y : -v.x;
              hv[0][o] = __float2half_rn(x0);
              lv[0][o] = __float2half_rn(x0 - __half2float(hv[0][o]));
              hv[1][o] = __float2half_rn(x1);
              lv[1][o] = __float2half_rn(x1 - __half2float(hv[1][o]));
            }
#pragma unroll
            for (int part = 0; part < 2; ++part) {
              h[part][sl >> 1] = (uint32_t)__half_as_ushort(hv[part][0]) | ((uint32_t)__half_as_ushort(hv[part][1]) << 16);
              l[part][sl >> 1] = (uint32_t)__half_as_ushort(lv[part][0]) | ((uint32_t)__half_as_ushort(lv[part][1]) << 16);
            }
          }
          const int pos = 8 * ch;
          uint8_t* kt = bt + (uint32_t)(pos / kKB) * b_tile;
#pragma unroll
          for (int part = 0; part < 2; ++part) {
            const int n = 2 * r + part;
            *reinterpret_cast<uint4*>(kt + sw128_off(n, pos % kKB)) = make_uint4(h[part][0], h[part][1], h[part][2], h[part][3]);
            *reinterpret_cast<uint4*>(kt + sw128_off(N + n, pos % kKB)) =
                make_uint4(l[part][0], l[part][1], l[part][2], l[part][3]);
          }
        }
      }
      fence_async_smem();
      mbar_arrive(&bfull[pb]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 4) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kCols)
                 : "memory");
  }
}

// Shared memory of nbuf B windows of N = 2S columns, and the coefficient ring stages that fit beside
// them.
int window_bytes(int k, int N, int nbuf) {
  const int k16 = (k + 15) / 16 * 16, nkb = (2 * k16 + kKB - 1) / kKB;
  return nbuf * nkb * 2 * N * 128;
}
int ring_stages(int k, int N, int nbuf) {
  const int limit = 227 * 1024 - 1024 - 256;  // 256: static barriers
  return std::max(0, std::min(kMaxStagesA, (limit - window_bytes(k, N, nbuf)) / kAStageBytes));
}
std::atomic<int> g_windows{0};  // forced window buffers (0: automatic)

// Window buffers for S samples: two while a ring of three stages still fits beside them, else one.
int window_buffers(int k, int S) {
  const int forced = g_windows.load();
  if (forced) return forced;
  return ring_stages(k, 2 * S, 2) >= 3 ? 2 : 1;
}

template <int W, int N>
int launch_tc2(const rb_filter_desc& d, const rb_basis& b, const rb::Geometry& g, const rb::Workspace& ws,
               const float2* beta, rb_trigger* trig, int64_t cap, unsigned long long* counter, cudaStream_t st,
               int withhold, int tmpl_base) {
  S2Params p;
  p.tmpl_base = tmpl_base;
  p.k16 = (int)g.k16;
  p.k = d.k;
  p.kp2 = (2 * p.k16 + kKB - 1) / kKB * kKB;
  p.nkb = p.kp2 / kKB;
  p.ahi = reinterpret_cast<const __half*>(b.coeff_op);
  p.alo = p.ahi + (int64_t)d.n_templates * 2 * p.k16;
  p.beta = beta;
  p.T = d.n_templates;
  p.half = g.n / 2;
  p.bin0 = (int)g.n_bins;
  p.pieces = ws.pieces;
  p.piece_total = ws.piece_total;
  p.sorted = ws.cand_sorted;
  p.thr2 = d.rho_ii * d.rho_ii;
  p.sample_offset = d.sample_offset;
  p.trig = trig;
  p.counter = counter;
  p.cap = cap;
  p.flags = ws.flags;
  p.withhold_copies = withhold;
  p.idesc = (1u << 4) | ((uint32_t)((2 * N) >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);  // F32 acc, FP16 A/B
  p.nbuf = window_buffers(d.k, N / 2);
  p.stages = ring_stages(d.k, N, p.nbuf);
  if (p.stages < 2) {
    rb::set_detail("k = %d too large for the tensor-core second stage", d.k);
    return RB_ERR_UNSUPPORTED;
  }
  const int smem = p.stages * kAStageBytes + window_bytes(d.k, N, p.nbuf) + 1024;
  auto kern = k_stage2_tc<W, N>;
  RB_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  kern<<<152, kThreadsTc, smem, st>>>(p);
  RB_LAUNCH_CHECK();
  return RB_OK;
}

std::atomic<int> g_withhold2{0};  // launches left whose producers issue no copy (failure-detection test)

}  // namespace

namespace rb {

int stage2_tc_run(const rb_filter_desc& d, const rb_basis& b, const Geometry& g, const Workspace& ws,
                  const float2* beta, rb_trigger* trig, int64_t cap, unsigned long long* counter, cudaStream_t st,
                  int tmpl_base) {
  int left = g_withhold2.load();
  while (left > 0 && !g_withhold2.compare_exchange_weak(left, left - 1)) {
  }
  const int withhold = left > 0 ? 1 : 0;
  const int S = stage2_tc_samples(d);
#define RB_TC2(W_, S_) \
  if (d.w == W_ && S == S_) return launch_tc2<W_, 2 * S_>(d, b, g, ws, beta, trig, cap, counter, st, withhold, tmpl_base);
  RB_TC2(1, 16) RB_TC2(2, 16) RB_TC2(4, 16) RB_TC2(8, 16)
  RB_TC2(2, 32) RB_TC2(4, 32) RB_TC2(8, 32)
#undef RB_TC2
  set_detail("the tensor-core second stage takes w <= 8 and k with room for its coefficient ring");
  return RB_ERR_UNSUPPORTED;
}

int stage2_tc_samples(const rb_filter_desc& d) {
  if (d.w > 8) return 0;
  const int mode = stage2_tc_mode();
  auto fits = [&](int S) { return ring_stages(d.k, 2 * S, window_buffers(d.k, S)) >= 2; };
  if (mode == 16 || mode == 32) return fits(mode) && mode / d.w <= 16 ? mode : 0;
  // automatic: 16 samples. 32-sample groups gather fewer rows (1.1 M against 1.9 M records on the
  // 10,000-template workload at w = 8) but leave room for one window buffer only, and the window
  // builds between pieces then cost more than the gathers save (0.70 ms against 0.62 ms there).
  return fits(16) ? 16 : 0;
}

}  // namespace rb

// Host-only test hook (not part of the C ABI): the next n tcgen05 second-stage launches issue no
// coefficient copies, so the MMA thread's bounded wait runs out; the call reports RB_ERR_TIMEOUT and
// the context stays usable. Used by the failure-detection test; no other code calls it.
extern "C" int rbx_stage2_withhold_copies(int n) {
  g_withhold2.store(n > 0 ? n : 0);
  return 0;
}

// Host-only hook (not part of the C ABI): window buffers of the tcgen05 second stage, 1 or 2 (a
// piece's window built while the one before runs), or 0 for the automatic choice; one buffer leaves
// room for more coefficient-ring stages. RB_ERR_BAD_INPUT for another value.
extern "C" int rbx_set_stage2_tc_windows(int n) {
  if (n < 0 || n > 2) return RB_ERR_BAD_INPUT;
  g_windows.store(n);
  return 0;
}
