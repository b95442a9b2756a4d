// Second stage of the hierarchy (arXiv:2110.13115 Sec. III.C, full-resolution reconstruction of
// every sample inside the triggering bins; Sec. III.E custom kernel), grouped by bin.
//
// 1. First-stage candidates are bucketed by groups of G consecutive bins (G = 1 for this kernel, more
//    for the tcgen05 one): per-group counts and a scatter, both through per-chunk shared-memory
//    histograms, around an exclusive scan. A run of candidates of one template and block in strictly
//    increasing bins of one group (the first stage writes a template's hits of a 32-bin chunk
//    consecutively, in bin order) becomes one record (template, block, mask of its bins in the
//    group), so its coefficient row is gathered once for all of them; the group comes with the work
//    piece.
// 2. The scan cuts each non-empty bin into pieces of at most kStage2Piece candidates, so a bin
//    with thousands of candidates is shared by many CTAs and empty bins cost nothing. For each
//    piece a CTA stages the bin's k x w window of beta (unless it already holds that bin) as
//    16-bit hi + lo tensor-core fragments of the real contraction
//        B[kk][2r]   = kk < k ? Re beta_kk[m0 + r] :  Im beta_(kk-k)[m0 + r]
//        B[kk][2r+1] = kk < k ? Im beta_kk[m0 + r] : -Re beta_(kk-k)[m0 + r],
//    so that [Re a_t, Im a_t] . B gives (Re, Im) of z_t[m0 + r] = sum_k conj(a_tk) beta_k[m0 + r].
//    Each warp reconstructs 16 candidates at a time with mma.sync m16n8k16 (FP16 in, FP32
//    accumulate) using three products hi.hi + hi.lo + lo.hi, which keeps the result at FP32
//    accuracy; the coefficients come pre-split from rb_pack_coeff (rows [Re a, Im a] in FP16
//    hi and lo planes at the start of coeff_op, columns permuted into fragment order so that
//    each lane fetches its A registers for two K chunks with one 16-byte load).
// 3. The arg-max over the bin's w samples (first on ties) is kept when |z| >= rho_II.
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <climits>

#include "common.cuh"
#include "internal.h"

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned kPiece = rb::kStage2Piece;  // candidates per second-stage work item
std::atomic<int> g_stage2_ring{2};  // coefficient ring slots of the mma.sync second stage (0: registers)
// records per work piece of the tcgen05 second stage: 256 (two tiles) balances the persistent CTAs'
// grid-stride walk over the pieces better than 512 at the cost of more window builds (0.539 against
// 0.565 ms on the 10,000-template block; 128: 0.531 ms but a slower scan)
std::atomic<int> g_tc_piece{256};

// Bucketing works on chunks of consecutive candidates. The first stage emits candidates in tile
// order and the tiles in flight share their bins, so a chunk's groups lie in a narrow range: each CTA
// histograms its chunk in shared memory over a window of kWin groups from the chunk's smallest group
// and then issues one global atomic per (chunk, group) instead of one per candidate. Groups outside
// the window (candidate lists in any other order) take one global atomic each. Small chunks (1024
// candidates in the count, 512 in the scatter) keep most CTAs of the grid busy on ~10^6 candidates.
constexpr int kWin = 1024;  // histogram window (groups)

__device__ __forceinline__ int block_min(int v, int* red) {  // blockDim.x == 256
  v = __reduce_min_sync(kFull, v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  int m = red[0];
#pragma unroll
  for (int i = 1; i < 8; ++i) m = min(m, red[i]);
  return m;
}

// Whether candidate c continues the run of its predecessor p: p kept (its bin relative to bin0 in
// [blo, nb)), c's bin in range, the same template and block, the same group of 2^gs bins, and a
// strictly later bin. A run therefore holds at most 2^gs candidates, and with gs = 0 every kept
// candidate starts its own.
__device__ __forceinline__ bool continues_run(const rb_candidate& p, const rb_candidate& c, int bin0, int blo, int nb,
                                              int gs) {
  const int px = p.bin - bin0, cx = c.bin - bin0;
  return px >= blo && px < cx && cx < nb && p.tmpl == c.tmpl && p.block == c.block && (px >> gs) == (cx >> gs);
}

// Whether candidate i (kept) starts a run: one record per run (every candidate when gs = 0).
__device__ __forceinline__ bool run_head(const rb_candidate* __restrict__ cand, int64_t i, const rb_candidate& c,
                                         int bin0, int blo, int nb, int gs) {
  return gs == 0 || i == 0 || !continues_run(cand[i - 1], c, bin0, blo, nb, gs);
}

// Per-group record counts (groups of 2^gs bins) of the candidates [0, min(cap, count)) whose bin
// (relative to bin0) lies in [blo, nb): bins before blo are dropped, as a block whose earlier valid
// samples another block already covers keeps only [blo, nb). 256 threads, chunks of 1024 candidates.
__global__ void __launch_bounds__(256) k_bin_count(const rb_candidate* __restrict__ cand,
                                                   const unsigned long long* dev_count, int64_t cap, int bin0,
                                                   int blo, int nb, int gs, unsigned* __restrict__ count) {
  constexpr int PER = 4, CHUNK = 256 * PER;
  __shared__ unsigned hist[kWin];
  __shared__ int red[8];
  const int64_t n = (int64_t)min((unsigned long long)cap, *dev_count);
  const int tid = threadIdx.x;
  for (int64_t c0 = blockIdx.x * (int64_t)CHUNK; c0 < n; c0 += (int64_t)gridDim.x * CHUNK) {
    int b[PER];
    int mn = INT_MAX;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int64_t i = c0 + j * 256 + tid;
      b[j] = -1;
      if (i < n) {
        const rb_candidate c = cand[i];
        const int x = c.bin - bin0;
        if (x >= blo && x < nb && run_head(cand, i, c, bin0, blo, nb, gs)) b[j] = x >> gs;
      }
      if (b[j] >= 0) mn = min(mn, b[j]);
    }
#pragma unroll
    for (int j = 0; j < kWin / 256; ++j) hist[j * 256 + tid] = 0u;
    const int lo = block_min(mn, red);  // (its __syncthreads also orders the zeroing)
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      if (b[j] < 0) continue;
      const int d = b[j] - lo;
      if (d < kWin) atomicAdd(&hist[d], 1u);
      else atomicAdd(count + b[j], 1u);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kWin / 256; ++j) {
      const unsigned h = hist[j * 256 + tid];
      if (h) atomicAdd(count + lo + j * 256 + tid, h);
    }
    __syncthreads();  // hist and red are reused by the next chunk
  }
}

constexpr int kScanPer = 16;                 // counters per thread and tile
constexpr int kScanTile = 1024 * kScanPer;   // bins per tile (one tile for 2^19-sample blocks at w = 8)
// one padding word per kScanPer: each thread's run of kScanPer counters starts in its own bank
__host__ __device__ constexpr int spad(int x) { return x + x / kScanPer; }
constexpr size_t kScanSmem = 2 * sizeof(unsigned) * (spad(kScanTile) + 1);

// Exclusive scan of count[0, nb) into start[0, nb] plus the piece list; count is reset to zero
// (it becomes the per-bin fill cursor). A bin holding c candidates is cut into ceil(c / kPiece)
// pieces {bin, first, end} of at most kPiece consecutive bucketed candidates, so that the
// second stage can spread a bin with thousands of candidates over many CTAs and skips empty
// bins entirely. Counts and piece counts are scanned together as one 64-bit value (pieces in the
// high word). One CTA of 1024 threads walks the array in tiles of 16384 counters, loading the next
// tile's counters while it processes one. Counters and start[] move with coalesced accesses
// through shared memory; each thread scans 16 consecutive counters; the tile's pieces are written
// one per thread (coalesced), each thread finding its piece's bin by binary search over the tile's
// piece prefix. Also raises
// RB_FLAG_CAND_OVERFLOW when the first stage found more candidates than the buffer holds.
__global__ void __launch_bounds__(1024) k_bin_scan(unsigned* __restrict__ count, unsigned* __restrict__ start, int nb,
                                                   unsigned piece, int4* __restrict__ pieces,
                                                   unsigned* __restrict__ piece_total,
                                                   const unsigned long long* dev_count, int64_t cap,
                                                   unsigned* flags) {
  using u64 = unsigned long long;
  extern __shared__ unsigned scan_smem[];
  unsigned* st_s = scan_smem;                          // global start of every bin of the tile (+ the end)
  unsigned* pp_s = scan_smem + spad(kScanTile) + 1;   // global index of every bin's first piece (+ the end)
  __shared__ u64 wsum[32];
  __shared__ u64 carry_s, carry_next;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto packed = [piece](unsigned c) { return (u64)c | ((u64)((c + piece - 1) / piece) << 32); };
  if (tid == 0) {
    carry_s = 0;
    if (*dev_count > (u64)cap) atomicOr(flags, (unsigned)RB_FLAG_CAND_OVERFLOW);
  }
  unsigned nx[kScanPer];  // the next tile's counters, loaded one tile ahead (and reset)
  auto fetch = [&](int b0) {
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
      const int i = b0 + j * 1024 + tid;
      nx[j] = 0;
      if (i < nb) {
        nx[j] = count[i];
        count[i] = 0;
      }
    }
  };
  fetch(0);
  __syncthreads();
  for (int base = 0; base < nb; base += kScanTile) {
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) st_s[spad(j * 1024 + tid)] = nx[j];
    fetch(base + kScanTile);
    __syncthreads();
    u64 s = 0;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) s += packed(st_s[spad(tid * kScanPer + j)]);
    u64 inc = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const u64 y = __shfl_up_sync(kFull, inc, off);
      if (lane >= off) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
      const u64 x0 = wsum[lane];
      u64 x = x0;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const u64 y = __shfl_up_sync(kFull, x, off);
        if (lane >= off) x += y;
      }
      wsum[lane] = x - x0;
    }
    __syncthreads();
    u64 run = carry_s + wsum[warp] + inc - s;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {  // (this thread's own counters: read, then overwritten)
      const int x = tid * kScanPer + j;
      const unsigned c = st_s[spad(x)];
      st_s[spad(x)] = (unsigned)run;
      pp_s[spad(x)] = (unsigned)(run >> 32);
      run += packed(c);
    }
    if (tid == 1023) {  // bins past nb count 0, so this is the tile's end
      st_s[spad(kScanTile)] = (unsigned)run;
      pp_s[spad(kScanTile)] = (unsigned)(run >> 32);
      carry_next = run;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
      const int x = j * 1024 + tid, i = base + x;
      if (i < nb) start[i] = st_s[spad(x)];
    }
    const unsigned p_end = (unsigned)(carry_next >> 32);
    for (unsigned pi = (unsigned)(carry_s >> 32) + tid; pi < p_end; pi += 1024) {
      int lo = 0, hi = kScanTile;  // pp[lo] <= pi < pp[hi]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pp_s[spad(mid)] <= pi) lo = mid;
        else hi = mid;
      }
      const unsigned c0 = st_s[spad(lo)] + (pi - pp_s[spad(lo)]) * piece;
      const unsigned c1 = min(st_s[spad(lo + 1)], c0 + piece);
      pieces[pi] = make_int4(base + lo, (int)c0, (int)c1, 0);
    }
    __syncthreads();
    if (tid == 0) carry_s = carry_next;
    __syncthreads();
  }
  if (tid == 0) {
    start[nb] = (unsigned)carry_s;
    *piece_total = (unsigned)(carry_s >> 32);
  }
}

// Records into group order, by chunks of 512 candidates (256 threads): each run head gathers its
// run's bin mask (at most 2^gs following candidates); a record's rank among the chunk's records of
// its group comes from a shared-memory atomic, the chunk's base in the group from one global cursor
// atomic per (chunk, group); groups outside the window take one global atomic each.
__global__ void __launch_bounds__(256) k_bin_scatter(const rb_candidate* __restrict__ cand,
                                                     const unsigned long long* dev_count, int64_t cap, int bin0,
                                                     int blo, int nb, int gs, const unsigned* __restrict__ start,
                                                     unsigned* __restrict__ cursor,
                                                     rb::SortedCand* __restrict__ out) {
  constexpr int PER = 2, CHUNK = 256 * PER;
  __shared__ unsigned hist[kWin];
  __shared__ int red[8];
  const int64_t n = (int64_t)min((unsigned long long)cap, *dev_count);
  const int tid = threadIdx.x;
  for (int64_t c0 = blockIdx.x * (int64_t)CHUNK; c0 < n; c0 += (int64_t)gridDim.x * CHUNK) {
    rb_candidate c[PER];
    int b[PER];
    int mn = INT_MAX;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int64_t i = c0 + j * 256 + tid;
      b[j] = -1;
      if (i < n) {
        c[j] = cand[i];
        const int x = c[j].bin - bin0;
        if (x >= blo && x < nb && run_head(cand, i, c[j], bin0, blo, nb, gs)) b[j] = x >> gs;
      }
      if (b[j] >= 0) mn = min(mn, b[j]);
    }
#pragma unroll
    for (int j = 0; j < kWin / 256; ++j) hist[j * 256 + tid] = 0u;
    const int lo = block_min(mn, red);
    unsigned r[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      r[j] = 0;
      if (b[j] >= 0 && b[j] - lo < kWin) r[j] = atomicAdd(&hist[b[j] - lo], 1u);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kWin / 256; ++j) {  // the chunk's base position inside each bin
      const int x = j * 256 + tid;
      const unsigned h = hist[x];
      if (h) hist[x] = atomicAdd(cursor + lo + x, h);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      if (b[j] < 0) continue;
      const int d = b[j] - lo;
      const unsigned pos = d < kWin ? hist[d] + r[j] : atomicAdd(cursor + b[j], 1u);
      const int64_t i = c0 + j * 256 + tid;
      const int gmask = (1 << gs) - 1;
      unsigned mask = 1u << ((c[j].bin - bin0) & gmask);
      rb_candidate prev = c[j];
      for (int r = 1; r < (1 << gs) && i + r < n; ++r) {
        const rb_candidate q = cand[i + r];
        if (!continues_run(prev, q, bin0, blo, nb, gs)) break;
        mask |= 1u << ((q.bin - bin0) & gmask);
        prev = q;
      }
      out[start[b[j]] + pos] = rb::SortedCand{c[j].tmpl, c[j].block, mask};
    }
    __syncthreads();  // hist and red are reused by the next chunk
  }
}

__device__ __forceinline__ uint32_t pack_h2(__half lo, __half hi) {
  return (uint32_t)__half_as_ushort(lo) | ((uint32_t)__half_as_ushort(hi) << 16);
}
// x -> (hi, lo) halves with hi + lo ~ x to about 22 bits
__device__ __forceinline__ void split_h(float x, __half& h, __half& l) {
  h = __float2half_rn(x);
  l = __float2half_rn(x - __half2float(h));
}

__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  // no side effects: the compiler may interleave independent products
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// W samples per bin -> NT = ceil(2W / 8) n-tiles of 8 columns (columns 2r, 2r+1 = Re, Im of sample r).
template <int W>
struct S2 {
  static constexpr int NT = (2 * W + 7) / 8;
};

// Stages the k x W window of beta starting at valid-half index m0 into shared memory, then
// writes its hi and lo tensor-core B fragments; ends with a barrier. The B operand of
// m16n8k16 for lane L holds b0 = (kk = 16 kc + 2 t, +1), b1 = (+8, +9) of column n = 8 nt + g.
template <int W>
__device__ __forceinline__ void stage_window(const float2* __restrict__ beta, int64_t m0, int64_t half, int k,
                                             int k16, float2* win, uint2* frag) {
  constexpr int NT = S2<W>::NT;
  const int pitch = k16 + 1, nkc = 2 * k16 / 16;
  for (int idx = threadIdx.x; idx < k16 * W; idx += blockDim.x) {
    const int kk = idx / W, r = idx - kk * W;
    win[r * pitch + kk] = kk < k ? __ldg(beta + (int64_t)kk * half + m0 + r) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nkc * NT * 32; idx += blockDim.x) {
    const int L = idx & 31, nt = (idx >> 5) % NT, kc = (idx >> 5) / NT;
    const int gg = L >> 2, tt = L & 3;
    const int n = nt * 8 + gg, r = n >> 1, part = n & 1;
    __half hv[4], lv[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int kk = kc * 16 + 2 * tt + (e & 1) + (e >> 1) * 8;
      float x = 0.f;
      if (r < W) {
        const bool im_half = kk >= k16;
        const float2 bv = win[r * pitch + (im_half ? kk - k16 : kk)];
        x = !im_half ? (part ? bv.y : bv.x) : (part ? -bv.x : bv.y);
      }
      split_h(x, hv[e], lv[e]);
    }
    frag[((0 * nkc + kc) * NT + nt) * 32 + L] = make_uint2(pack_h2(hv[0], hv[1]), pack_h2(hv[2], hv[3]));
    frag[((1 * nkc + kc) * NT + nt) * 32 + L] = make_uint2(pack_h2(lv[0], lv[1]), pack_h2(lv[2], lv[3]));
  }
  __syncthreads();
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid) {
  const unsigned dst = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(gmem), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Shared-memory bytes of k_stage2_bins<W, D>: fragments frag[plane][kc][nt][lane] (uint2), then one
// region that holds the bin's window [W][k16 + 1] float2 while it is staged and, while candidates
// are reconstructed, each warp's ring of D coefficient slots [slot][4][lane] (uint4).
template <int W, int D>
constexpr size_t bins_smem(int k16) {
  const size_t fr = sizeof(uint2) * 2 * (2 * k16 / 16) * S2<W>::NT * 32;
  const size_t wn = sizeof(float2) * W * (k16 + 1), ring = sizeof(uint4) * 8 * D * 4 * 32;
  return fr + (wn > ring ? wn : ring);
}

// D = 0: each lane loads its coefficient fragments into registers (two K-chunk pairs unrolled);
// D > 0: each lane streams them through a private ring of D slots in shared memory with cp.async,
// D - 1 K-chunk pairs ahead of the products, so that the gathers of a tile overlap its products
// without holding registers. A lane reads back only what it copied itself, so its own
// cp.async.wait_group orders each slot's fill before its reads, and its reads (consumed by the
// products before the next copy is issued) before the slot's refill.
template <int W, int D>
__global__ void __launch_bounds__(256, 3) k_stage2_bins(const __half* __restrict__ ahi, const __half* __restrict__ alo,
                                                     const float2* __restrict__ beta, int k, int k16, int T,
                                                     int64_t half, int bin0, const int4* __restrict__ pieces,
                                                     const unsigned* __restrict__ piece_total,
                                                     const rb::SortedCand* __restrict__ sorted, float thr2,
                                                     int64_t sample_offset, rb_trigger* __restrict__ trig,
                                                     unsigned long long* counter, int64_t cap, int tmpl_base) {
  constexpr int NT = S2<W>::NT;
  extern __shared__ __align__(16) uint8_t s2mem[];
  const int nkc = 2 * k16 / 16;                     // K chunks: Re half then Im half (even)
  uint2* frag = reinterpret_cast<uint2*>(s2mem);    // [2][nkc][NT][32]
  uint8_t* region = s2mem + sizeof(uint2) * 2 * nkc * NT * 32;
  float2* win = reinterpret_cast<float2*>(region);  // [W][k16 + 1] while a bin is staged
  uint4* ring = reinterpret_cast<uint4*>(region) + (threadIdx.x >> 5) * (D * 4 * 32);  // this warp's slots
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  const unsigned npieces = *piece_total;
  int staged = -1;
  for (unsigned p = blockIdx.x; p < npieces; p += gridDim.x) {
    const int4 pc = pieces[p];
    const int b = pc.x;
    const unsigned c0 = (unsigned)pc.y, c1 = (unsigned)pc.z;
    if (b != staged) {  // block-uniform: the window and its fragments change with the bin
      staged = b;
      __syncthreads();  // every warp is done with the previous bin's fragments
      stage_window<W>(beta, (int64_t)(bin0 + b) * W - half, half, k, k16, win, frag);
    }
    for (unsigned base = c0 + warp * 16; base < c1; base += nwarp * 16) {
      // rows g and g + 8 of the m16 tile are candidates base + g and base + g + 8
      int tr[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const unsigned ci = base + g + 8 * h;
        const int t = ci < c1 ? sorted[ci].tmpl : -1;
        tr[h] = (t >= 0 && t < T) ? t : -1;
      }
      float d[NT][4];
#pragma unroll
      for (int nt = 0; nt < NT; ++nt) d[nt][0] = d[nt][1] = d[nt][2] = d[nt][3] = 0.f;
      // A fragments straight from the packed FP16 hi/lo rows, stored in fragment order: the 16 bytes
      // at 32 q + 8 t4 of a row hold this lane's (a0, a2) for K chunks 2q and 2q + 1
      const int64_t p2 = 2 * (int64_t)k16;
      const uint4* rh0 = reinterpret_cast<const uint4*>(ahi + (int64_t)max(tr[0], 0) * p2) + t4;
      const uint4* rh1 = reinterpret_cast<const uint4*>(ahi + (int64_t)max(tr[1], 0) * p2) + t4;
      const uint4* rl0 = reinterpret_cast<const uint4*>(alo + (int64_t)max(tr[0], 0) * p2) + t4;
      const uint4* rl1 = reinterpret_cast<const uint4*>(alo + (int64_t)max(tr[1], 0) * p2) + t4;
      const bool v0 = tr[0] >= 0, v1 = tr[1] >= 0;
      const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
      const int nq = nkc / 2;
      auto issue = [&](int q) {  // K-chunk pair q into slot q % D (zero-filled for an empty row)
        uint4* sl = ring + (q % (D > 0 ? D : 1)) * 4 * 32 + lane;
        cp_async16(sl + 0 * 32, rh0 + 4 * q, v0);
        cp_async16(sl + 1 * 32, rh1 + 4 * q, v1);
        cp_async16(sl + 2 * 32, rl0 + 4 * q, v0);
        cp_async16(sl + 3 * 32, rl1 + 4 * q, v1);
      };
      if constexpr (D > 0) {
#pragma unroll
        for (int s = 0; s < D - 1; ++s) {
          if (s < nq) issue(s);
          cp_async_commit();
        }
      }
#pragma unroll 2
      for (int q = 0; q < nq; ++q) {
        uint4 h0, h1, l0, l1;
        if constexpr (D > 0) {
          if (q + D - 1 < nq) issue(q + D - 1);
          cp_async_commit();
          cp_async_wait<D - 1>();  // the group of pair q is complete
          const uint4* sl = ring + (q % D) * 4 * 32 + lane;
          h0 = sl[0 * 32];
          h1 = sl[1 * 32];
          l0 = sl[2 * 32];
          l1 = sl[3 * 32];
        } else {
          h0 = v0 ? __ldg(rh0 + 4 * q) : z4;
          h1 = v1 ? __ldg(rh1 + 4 * q) : z4;
          l0 = v0 ? __ldg(rl0 + 4 * q) : z4;
          l1 = v1 ? __ldg(rl1 + 4 * q) : z4;
        }
#pragma unroll
        for (int half_q = 0; half_q < 2; ++half_q) {
          const int kc = 2 * q + half_q;
          const uint32_t ah0 = half_q ? h0.z : h0.x, ah2 = half_q ? h0.w : h0.y;
          const uint32_t ah1 = half_q ? h1.z : h1.x, ah3 = half_q ? h1.w : h1.y;
          const uint32_t al0 = half_q ? l0.z : l0.x, al2 = half_q ? l0.w : l0.y;
          const uint32_t al1 = half_q ? l1.z : l1.x, al3 = half_q ? l1.w : l1.y;
          // the three products of every n-tile, ordered so that consecutive ones are independent
          uint2 bh[NT], bl[NT];
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) {
            bh[nt] = frag[((0 * nkc + kc) * NT + nt) * 32 + lane];
            bl[nt] = frag[((1 * nkc + kc) * NT + nt) * 32 + lane];
          }
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) mma16816(d[nt], ah0, ah1, ah2, ah3, bh[nt].x, bh[nt].y);
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) mma16816(d[nt], ah0, ah1, ah2, ah3, bl[nt].x, bl[nt].y);
#pragma unroll
          for (int nt = 0; nt < NT; ++nt) mma16816(d[nt], al0, al1, al2, al3, bh[nt].x, bh[nt].y);
        }
      }
      // thread (g, t) holds, per n-tile, (Re, Im) of sample r = 4 nt + t for rows g and g + 8
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float best = -1.f, zr = 0.f, zi = 0.f;
        int br = 0;
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          const int r = 4 * nt + t4;
          const float re = d[nt][2 * h], im = d[nt][2 * h + 1];
          const float p2 = fmaf(re, re, im * im);
          if (r < W && p2 > best) {
            best = p2;
            br = r;
            zr = re;
            zi = im;
          }
        }
#pragma unroll
        for (int off = 1; off < 4; off <<= 1) {
          const float ob = __shfl_xor_sync(kFull, best, off);
          const int orr = __shfl_xor_sync(kFull, br, off);
          const float ozr = __shfl_xor_sync(kFull, zr, off);
          const float ozi = __shfl_xor_sync(kFull, zi, off);
          if (ob > best || (ob == best && orr < br)) {
            best = ob;
            br = orr;
            zr = ozr;
            zi = ozi;
          }
        }
        // one counter reservation per warp for its (up to 8) triggers of this half
        const bool emit = t4 == 0 && tr[h] >= 0 && best >= thr2;
        const unsigned em = __ballot_sync(kFull, emit);
        if (!em) continue;
        const int leader = __ffs(em) - 1;
        unsigned long long b0 = 0;
        if (lane == leader) b0 = atomicAdd(counter, (unsigned long long)__popc(em));
        b0 = __shfl_sync(kFull, b0, leader);
        if (emit) {
          const rb::SortedCand cd = sorted[base + g + 8 * h];
          const unsigned long long idx = b0 + __popc(em & ((1u << lane) - 1u));
          if ((int64_t)idx < cap) {
            rb_trigger tg;
            tg.sample = sample_offset + (int64_t)(bin0 + b) * W + br;
            tg.tmpl = tmpl_base + cd.tmpl;
            tg.block = cd.block;
            tg.snr = sqrtf(best);
            tg.phase = atan2f(zi, zr);
            trig[idx] = tg;
          }
        }
      }
    }
  }
}

template <int W, int D>
int launch_bins(const rb_filter_desc& d, const rb_basis& b, const rb::Geometry& g, const rb::Workspace& ws,
                const float2* beta, rb_trigger* trig, int64_t cap, unsigned long long* counter, int tmpl_base,
                cudaStream_t st) {
  const int nb = (int)g.n_bins;
  const int k16 = (d.k + 15) / 16 * 16;
  const int smem = (int)bins_smem<W, D>(k16);
  if (smem > 200 * 1024) {
    rb::set_detail("k * w too large for the second-stage window (%d x %d)", d.k, W);
    return RB_ERR_UNSUPPORTED;
  }
  auto kern = k_stage2_bins<W, D>;
  if (smem > 48 * 1024) RB_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  const int grid = 152 * 8;
  const __half* ahi = reinterpret_cast<const __half*>(b.coeff_op);
  const __half* alo = ahi + (int64_t)d.n_templates * 2 * k16;
  kern<<<grid, 256, smem, st>>>(ahi, alo, beta, d.k, k16, d.n_templates, g.n / 2, nb, ws.pieces, ws.piece_total,
                                ws.cand_sorted, d.rho_ii * d.rho_ii, d.sample_offset, trig, counter, cap, tmpl_base);
  RB_LAUNCH_CHECK();
  return RB_OK;
}

}  // namespace

namespace rb {

int stage2_group(const rb_filter_desc& d) {
  const int samples = stage2_use_tc() ? stage2_tc_samples(d) : 0;
  return samples > 0 ? samples / d.w : 1;
}

int stage2_bucket(const rb_filter_desc& d, const Geometry& g, const Workspace& ws, int bin_lo, cudaStream_t st) {
  const int nb = (int)g.n_bins;
  const int bin0 = nb;  // valid bins are [n/(2w), n/w)
  const int G = stage2_group(d);
  const int gs = __builtin_ctz((unsigned)G);
  const int ng = (nb + G - 1) / G;
  RB_CUDA_TRY(cudaMemsetAsync(ws.bin_count, 0, sizeof(unsigned) * (ng + 1), st));
  k_bin_count<<<152 * 8, 256, 0, st>>>(ws.cand, ws.cand_count, d.cand_capacity, bin0, bin_lo, nb, gs,
                                       ws.bin_count);
  RB_LAUNCH_CHECK();
  RB_CUDA_TRY(cudaFuncSetAttribute(k_bin_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kScanSmem));
  // work pieces: kStage2Piece records per group at most; the tcgen05 kernel builds one window per piece
  // and takes pieces of g_tc_piece records
  const unsigned piece = G > 1 ? (unsigned)g_tc_piece.load() : kPiece;
  k_bin_scan<<<1, 1024, kScanSmem, st>>>(ws.bin_count, ws.bin_start, ng, piece, ws.pieces, ws.piece_total,
                                         ws.cand_count, d.cand_capacity, ws.flags);
  RB_LAUNCH_CHECK();
  k_bin_scatter<<<152 * 8, 256, 0, st>>>(ws.cand, ws.cand_count, d.cand_capacity, bin0, bin_lo, nb, gs,
                                         ws.bin_start, ws.bin_count, ws.cand_sorted);
  RB_LAUNCH_CHECK();
  return RB_OK;
}

int stage2_run(const rb_filter_desc& d, const rb_basis& b, const Geometry& g, const Workspace& ws,
               const float2* beta, rb_trigger* trig, int64_t cap, unsigned long long* counter, cudaStream_t st,
               int tmpl_base) {
  if (stage2_group(d) > 1) return stage2_tc_run(d, b, g, ws, beta, trig, cap, counter, st, tmpl_base);
  const int D = g_stage2_ring.load();
#define RB_BINS(W_, D_) \
  if (d.w == W_ && D == D_) return launch_bins<W_, D_>(d, b, g, ws, beta, trig, cap, counter, tmpl_base, st);
  RB_BINS(1, 0) RB_BINS(1, 2) RB_BINS(1, 3)
  RB_BINS(2, 0) RB_BINS(2, 2) RB_BINS(2, 3)
  RB_BINS(4, 0) RB_BINS(4, 2) RB_BINS(4, 3)
  RB_BINS(8, 0) RB_BINS(8, 2) RB_BINS(8, 3) RB_BINS(8, 4)
  RB_BINS(16, 0) RB_BINS(16, 2) RB_BINS(16, 3)
#undef RB_BINS
  if (d.w == 1 || d.w == 2 || d.w == 4 || d.w == 8 || d.w == 16) {
    set_detail("no second-stage kernel for w = %d with a ring of %d slots", d.w, D);
    return RB_ERR_UNSUPPORTED;
  }
  return RB_ERR_BAD_INPUT;
}

int stage2_bucketed(const rb_filter_desc& d, const rb_basis& b, const Geometry& g, const Workspace& ws,
                    const float2* beta, rb_trigger* trig, int64_t cap, unsigned long long* counter, int bin_lo,
                    cudaStream_t st) {
  int rc = stage2_bucket(d, g, ws, bin_lo, st);
  if (rc) return rc;
  return stage2_run(d, b, g, ws, beta, trig, cap, counter, st);
}

}  // namespace rb

namespace {
std::atomic<int> g_stage2_tc{1};
}

// Host-only hook (not part of the C ABI): slots of the mma.sync second stage's per-lane coefficient
// ring (0: loads into registers; 2, the default, and 3 for every w, also 4 for w = 8).
// RB_ERR_BAD_INPUT otherwise.
extern "C" int rbx_set_stage2_ring(int slots) {
  if (slots != 0 && slots != 2 && slots != 3 && slots != 4) return RB_ERR_BAD_INPUT;
  g_stage2_ring.store(slots);
  return 0;
}

namespace rb {
bool stage2_use_tc() { return g_stage2_tc.load() != 0; }
int stage2_tc_mode() { return g_stage2_tc.load(); }
}  // namespace rb

// Host-only hook (not part of the C ABI): the second-stage kernel. 1 (the default): the tcgen05
// kernel (stage2_tc.cu) over bin groups of the automatic width, 16 or 32: of that many samples,
// where it applies (w <= 8 and a coefficient ring fits beside the windows; the mma.sync kernel
// otherwise); 0: the per-bin mma.sync kernel above. RB_ERR_BAD_INPUT for another value. On the
// 10,000-template, 2^19-sample workload (3.5 M candidates, 1.9 M records in 16-sample groups) the
// second stage takes 0.62 ms on tcgen05, 0.70 ms on mma.sync.
extern "C" int rbx_set_stage2_tc(int mode) {
  if (mode != 0 && mode != 1 && mode != 16 && mode != 32) return RB_ERR_BAD_INPUT;
  g_stage2_tc.store(mode);
  return 0;
}

// Host-only measurement hook (not part of the C ABI): the mma.sync m16n8k16 FP16 -> FP32 issue rate of
// this GPU, the ceiling of the mma.sync second stage. Every warp of 608 CTAs x 256 threads runs `iters`
// rounds of 8 independent register-only products; *per_s receives products per second (0 on error).
namespace {
__global__ void __launch_bounds__(256) k_mma_rate(float* out, int iters) {
  uint32_t a0 = threadIdx.x * 2654435761u, a1 = a0 * 3u, a2 = a0 * 5u, a3 = a0 * 7u, b0 = a0 * 11u, b1 = a0 * 13u;
  float d[8][4] = {};
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) mma16816(d[i], a0, a1, a2, a3, b0, b1);
  }
  float acc = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) acc += d[i][0] + d[i][1] + d[i][2] + d[i][3];
  if (acc == 1.2345f) out[0] = acc;  // keeps the products live
}
}  // namespace

extern "C" int rbx_mma_sync_rate(int iters, double* per_s) {
  if (!per_s || iters < 1 || iters > (1 << 20)) return RB_ERR_BAD_INPUT;
  *per_s = 0.0;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = RB_OK;
  float ms = 0.f;
  if (cudaMalloc(&out, sizeof(float)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    rc = RB_ERR_CUDA;
  } else {
    k_mma_rate<<<608, 256>>>(out, iters);  // warm-up
    cudaEventRecord(e0);
    k_mma_rate<<<608, 256>>>(out, iters);
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.f)
      rc = RB_ERR_CUDA;
    else
      *per_s = 608.0 * 8 * iters * 8 / (ms * 1e-3);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  return rc;
}

// Host-only hook (not part of the C ABI): records per work piece of the tcgen05 second stage, a
// multiple of 128 from rb::kStage2MinPiece up to 4096 (each piece costs one group-window build).
// RB_ERR_BAD_INPUT otherwise.
extern "C" int rbx_set_stage2_tc_piece(int records) {
  if (records < (int)rb::kStage2MinPiece || records > 4096 || records % 128) return RB_ERR_BAD_INPUT;
  g_tc_piece.store(records);
  return 0;
}
