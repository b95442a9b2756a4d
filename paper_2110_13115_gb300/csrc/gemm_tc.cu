// First-stage reconstruction on tcgen05 tensor cores (arXiv:2110.13115 Sec. III.C first stage; the
// product of the bin-averaged basis series with the coefficient matrix of Sec. III.E):
// z_avg[t, i] = sum_k conj(a_tk) beta_avg_k[i] as one real contraction over K = 2k,
//   rows 2t   [Re a_t, Im a_t]   . [Re b_i, Im b_i] = Re z_avg[t, i]
//   rows 2t+1 [-Im a_t, Re a_t]  . [Re b_i, Im b_i] = Im z_avg[t, i],
// with 16-bit operands (one plane each; hi + lo planes of both with three products hi.hi + hi.lo +
// lo.hi; or hi + lo planes of A against one plane of B with two products) and FP32 accumulators in
// tensor memory. The epilogue squares, pairs the Re/Im rows across
// neighbouring lanes, tests |z_avg|^2 >= rho_I^2 and appends candidates; the T x bins array
// never reaches global memory.
//
// Persistent kernel, one CTA per SM, 320 threads:
//   warp 0  : TMA producer (one thread) - 128B-swizzled K-major tiles of A (128 x 64) and
//             B (BN x 64) per plane into a STAGES-deep shared-memory ring;
//   warp 1  : tensor-memory allocation (2 BN columns) and the MMA issuer (one thread),
//             M = 128, N = BN, K = 16 per instruction, two accumulator buffers;
//   warps 2-9: epilogue, two per 32-lane quarter of tensor memory (half the columns each).
// Every mbarrier wait is bounded (1 s of %globaltimer); a timeout sets RB_FLAG_TIMEOUT, makes the
// other roles stop, waits (bounded) for the copies and products in flight, frees tensor memory
// and returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "internal.h"
#include "tma.cuh"

namespace {

using namespace rbtma;

constexpr int BM = 128, BK = 64;
constexpr int kThreads = 320;  // producer warp, MMA warp, 8 epilogue warps

struct TcParams {
  int T;          // templates (rows of A = 2T)
  int N;          // valid bins (rows of B)
  int KB;         // K blocks of 64
  int last_k16;   // 16-wide K steps of the last block that hold data (columns < 2k; the rest is zero)
  int num_m, num_n;
  float thr2;
  int bin0;
  int block_id;
  rb_candidate* cand;
  unsigned long long* counter;
  long long cap;
  unsigned* flags;
  uint32_t idesc;
  int withhold_copies;  // failure-detection test: the producer issues no copy (see rbx_stage1_withhold_copies)
};

// Tile order: row blocks fastest, so the tiles in flight share one B tile (it is read from L2 by
// every CTA while all of A stays L2-resident). Grouping rows x columns measured slower.
__device__ __forceinline__ void tile_coords(int tile, int num_m, int num_n, int& mb, int& nb) {
  mb = tile % num_m;
  nb = tile / num_m;
}

// NA / NB: planes of A / B (1: one 16-bit operand; 2: hi and lo). Products per K step:
// (1, 1) a.b; (2, 2) hi.hi + hi.lo + lo.hi; (2, 1) hi.b + lo.b (A exact to about 22 bits, B rounded).
template <int NA, int NB, int STAGES, int BN>
__global__ void __launch_bounds__(kThreads, 1)
    k_stage1_tc(const __grid_constant__ CUtensorMap tmA0, const __grid_constant__ CUtensorMap tmA1,
                const __grid_constant__ CUtensorMap tmB0, const __grid_constant__ CUtensorMap tmB1, TcParams p) {
  constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
  constexpr uint32_t STAGE_BYTES = NA * A_BYTES + NB * B_BYTES;
  extern __shared__ uint8_t dsmem[];
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], tfull[2], tempty[2], drain;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t smem0 = (saddr(dsmem) + 1023u) & ~1023u;
  const int num_tiles = p.num_m * p.num_n;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], 8);
    }
    mbar_init(&drain, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                 "r"((uint32_t)(2 * BN))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  auto fail = [&]() {
    abort_flag = 1;
    atomicOr(p.flags, (unsigned)RB_FLAG_TIMEOUT);
  };

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int used = 0;  // stages that received at least one load
      // (withhold_copies: no copy at all, so the MMA warp's first wait runs out and every role stops)
      for (int tile = blockIdx.x; tile < num_tiles && !abort_flag && !p.withhold_copies; tile += gridDim.x) {
        int mb, nb;
        tile_coords(tile, p.num_m, p.num_n, mb, nb);
        for (int kb = 0; kb < p.KB; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1, &abort_flag)) {
            fail();
            break;
          }
          const uint32_t sb = smem0 + stage * STAGE_BYTES;
          mbar_expect_tx(&full[stage], STAGE_BYTES);
          tma_load(sb, &tmA0, &full[stage], kb * BK, mb * BM);
          if (NA == 2) tma_load(sb + A_BYTES, &tmA1, &full[stage], kb * BK, mb * BM);
          tma_load(sb + NA * A_BYTES, &tmB0, &full[stage], kb * BK, nb * BN);
          if (NB == 2) tma_load(sb + NA * A_BYTES + B_BYTES, &tmB1, &full[stage], kb * BK, nb * BN);
          used = used < STAGES ? used + 1 : STAGES;
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
      // copies in flight land before the CTA may exit: the last load of each used stage
      for (int i = 0; i < used; ++i) {
        if (--stage < 0) {
          stage = STAGES - 1;
          phase ^= 1;
        }
        const uint64_t t0 = gtimer();
        while (!mbar_try(&full[stage], phase) && gtimer() - t0 < kWaitNs) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int acc = 0;
      uint32_t acc_phase = 0;
      bool issued = false;
      for (int tile = blockIdx.x; tile < num_tiles && !abort_flag; tile += gridDim.x) {
        if (!mbar_wait(&tempty[acc], acc_phase ^ 1, &abort_flag)) {
          fail();
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * BN);
        bool ok = true;
        for (int kb = 0; kb < p.KB; ++kb) {
          if (!mbar_wait(&full[stage], phase, &abort_flag)) {
            fail();
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem0 + stage * STAGE_BYTES;
          const uint32_t a1 = a0 + A_BYTES;
          const uint32_t b0 = a0 + NA * A_BYTES;
          const uint32_t b1 = b0 + B_BYTES;
          // the zero-padded K steps past 2k in the last block add nothing: skipped
          const int nkk = kb == p.KB - 1 ? p.last_k16 : BK / 16;
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk) {
            if (kk >= nkk) break;
            const uint32_t off = kk * 32;
            tc_mma(d, sw128_desc(a0 + off), sw128_desc(b0 + off), p.idesc, (kb | kk) != 0);
            if (NB == 2) tc_mma(d, sw128_desc(a0 + off), sw128_desc(b1 + off), p.idesc, 1);
            if (NA == 2) tc_mma(d, sw128_desc(a1 + off), sw128_desc(b0 + off), p.idesc, 1);
          }
          issued = true;
          tc_commit(&empty[stage]);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        tc_commit(&tfull[acc]);
        if (++acc == 2) {
          acc = 0;
          acc_phase ^= 1;
        }
      }
      if (issued) {
        // every product issued so far has completed before tensor memory is released
        tc_commit(&drain);
        const uint64_t t0 = gtimer();
        while (!mbar_try(&drain, 0) && gtimer() - t0 < kWaitNs) {
        }
      }
    }
  } else {
    // two warps per tensor-memory lane quarter, each owning half of the tile's columns
    const int q = warp & 3;
    const int cbase = ((warp - 2) >> 2) * (BN / 2);
    int acc = 0;
    uint32_t acc_phase = 0;
    const unsigned full_mask = 0xffffffffu;
    for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x) {
      if (!mbar_wait(&tfull[acc], acc_phase, &abort_flag)) {
        if (lane == 0) fail();
        break;
      }
      tc_fence_after();
      int mb, nb;
      tile_coords(tile, p.num_m, p.num_n, mb, nb);
      const int row = mb * BM + q * 32 + lane;
      const int t = row >> 1;
      const bool even = (lane & 1) == 0;
      const bool trow = even && t < p.T;
#pragma unroll 1
      for (int c0 = cbase; c0 < cbase + BN / 2; c0 += 32) {
        float v[32];
        tc_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * BN + c0), v);
        // |z|^2 of the (Re, Im) row pair: rows 2t and 2t+1 sit in neighbouring lanes
        float pmax = 0.f;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          v[j] = v[j] * v[j];
          v[j] += __shfl_xor_sync(full_mask, v[j], 1);
          pmax = fmaxf(pmax, v[j]);
        }
        const int col0 = nb * BN + c0;
        if (!__any_sync(full_mask, trow && col0 < p.N && pmax >= p.thr2)) continue;
        // one counter reservation per warp and chunk: per-lane hit masks, a warp scan of the
        // counts, then each lane writes its hits in column order
        unsigned hits = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j)
          hits |= (unsigned)(trow && col0 + j < p.N && v[j] >= p.thr2) << j;
        const int cnt = __popc(hits);
        int incl = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const int y = __shfl_up_sync(full_mask, incl, off);
          if (lane >= off) incl += y;
        }
        unsigned long long base = 0;
        if (lane == 31) base = atomicAdd(p.counter, (unsigned long long)incl);
        base = __shfl_sync(full_mask, base, 31);
        unsigned long long idx = base + (unsigned long long)(incl - cnt);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if ((hits >> j) & 1u) {
            if ((long long)idx < p.cap) {
              rb_candidate c;
              c.tmpl = t;
              c.bin = p.bin0 + col0 + j;
              c.snr_avg = sqrtf(v[j]);
              c.block = p.block_id;
              p.cand[idx] = c;
            }
            ++idx;
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
      if (++acc == 2) {
        acc = 0;
        acc_phase ^= 1;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)(2 * BN)) : "memory");
  }
}

// --- host side --------------------------------------------------------------------------------

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(ptr);
  });
  return fn;
}

}  // namespace

namespace rb {

int make_map_2d(CUtensorMap* m, CUtensorMapDataType type, int elem_bytes, const void* base, uint64_t dim0,
                uint64_t dim1, uint64_t row_bytes, uint32_t box0, uint32_t box1, CUtensorMapSwizzle swizzle) {
  EncodeTiled enc = encode_fn();
  if (!enc) {
    set_detail("cuTensorMapEncodeTiled unavailable from the driver");
    return RB_ERR_CUDA;
  }
  if (((uintptr_t)base & 15) || row_bytes % 16 || (box0 * elem_bytes) % 16) {
    set_detail("tensor map base, row pitch or box width not 16-byte aligned");
    return RB_ERR_BAD_INPUT;
  }
  cuuint64_t dims[2] = {(cuuint64_t)dim0, (cuuint64_t)dim1};
  cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
  cuuint32_t box[2] = {box0, box1};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, type, 2, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_detail("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return RB_ERR_CUDA;
  }
  return RB_OK;
}

}  // namespace rb

namespace {

// 2D map over a [rows][kp] 16-bit matrix, box of 64 (K) x box_rows, 128-byte swizzle, zero fill.
int make_map(CUtensorMap* m, const void* base, bool bf16, int64_t kp, int64_t rows, int box_rows) {
  EncodeTiled enc = encode_fn();
  if (!enc) {
    rb::set_detail("cuTensorMapEncodeTiled unavailable from the driver");
    return RB_ERR_CUDA;
  }
  if (((uintptr_t)base & 15) || (kp * 2) % 16) {
    rb::set_detail("operand base or row pitch not 16-byte aligned");
    return RB_ERR_BAD_INPUT;
  }
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                   const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    rb::set_detail("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return RB_ERR_CUDA;
  }
  return RB_OK;
}

template <int NA, int NB, int STAGES, int BN>
int launch_tc(const CUtensorMap* maps, const TcParams& p, cudaStream_t st) {
  constexpr int smem = STAGES * (NA * BM * BK * 2 + NB * BN * BK * 2) + 1024;
  static_assert(smem <= 227 * 1024, "shared memory budget");
  auto kern = k_stage1_tc<NA, NB, STAGES, BN>;
  RB_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int dev = 0, sms = 0;
  RB_CUDA_TRY(cudaGetDevice(&dev));
  RB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int tiles = p.num_m * p.num_n;
  const int grid = std::max(1, std::min(tiles, sms));
  kern<<<grid, kThreads, smem, st>>>(maps[0], maps[1], maps[2], maps[3], p);
  RB_LAUNCH_CHECK();
  return RB_OK;
}

// Tile variants (the autotuner's search space): N-tile width and the ring depth that fits.
constexpr int kVariants = 2;
constexpr int kVariantBN[kVariants] = {256, 128};

// planes: 1 (single operands), 2 (A and B split), 3 (A split, B single)
int launch_variant(int v, int planes, const CUtensorMap* maps, const TcParams& p, cudaStream_t st) {
  if (v == 0) {
    if (planes == 2) return launch_tc<2, 2, 2, 256>(maps, p, st);
    if (planes == 3) return launch_tc<2, 1, 3, 256>(maps, p, st);
    return launch_tc<1, 1, 4, 256>(maps, p, st);
  }
  if (planes == 2) return launch_tc<2, 2, 3, 128>(maps, p, st);
  if (planes == 3) return launch_tc<2, 1, 4, 128>(maps, p, st);
  return launch_tc<1, 1, 6, 128>(maps, p, st);
}

int plane_mode(int precision) {
  if (precision == RB_PREC_FP16_SPLIT || precision == RB_PREC_BF16_SPLIT) return 2;
  if (precision == RB_PREC_FP16_SPLIT_A) return 3;
  return 1;
}

struct TuneKey {
  int precision, T;
  int64_t n_bins;
  int kp;
  bool operator<(const TuneKey& o) const {
    return std::tie(precision, T, n_bins, kp) < std::tie(o.precision, o.T, o.n_bins, o.kp);
  }
};
std::mutex g_tune_mu;
std::atomic<int> g_withhold{0};  // launches left whose producer issues no copy (failure-detection test)
std::map<TuneKey, int> g_tuned;

int chosen_variant(const rb_filter_desc& d, const rb::Geometry& g) {
  std::lock_guard<std::mutex> lock(g_tune_mu);
  auto it = g_tuned.find(TuneKey{d.precision, d.n_templates, g.n_bins, g.kp});
  return it == g_tuned.end() ? 0 : it->second;
}

int build_params(const rb_filter_desc& d, const rb_basis& b, const rb::Geometry& g, const rb::Workspace& ws,
                 rb_candidate* cand, int variant, CUtensorMap* maps, TcParams& p) {
  const int BN = kVariantBN[variant];
  const int planes = plane_mode(d.precision);
  const bool split = planes == 2;                  // B in hi and lo planes
  const bool split_a = planes == 2 || planes == 3;  // A in hi and lo planes
  const bool bf = d.precision == RB_PREC_BF16 || d.precision == RB_PREC_BF16_SPLIT;
  const int64_t M = 2 * (int64_t)d.n_templates;
  const uint16_t* a0 = (const uint16_t*)((const char*)b.coeff_op + g.s2_bytes);
  const uint16_t* a1 = split_a ? a0 + M * g.kp : a0;
  int rc;
  if ((rc = make_map(&maps[0], a0, bf, g.kp, M, BM))) return rc;
  if ((rc = make_map(&maps[1], a1, bf, g.kp, M, BM))) return rc;
  if ((rc = make_map(&maps[2], ws.bop_hi, bf, g.kp, g.n_bins, BN))) return rc;
  if ((rc = make_map(&maps[3], split ? ws.bop_lo : ws.bop_hi, bf, g.kp, g.n_bins, BN))) return rc;
  p.T = d.n_templates;
  p.N = (int)g.n_bins;
  p.KB = g.kp / BK;
  p.last_k16 = (2 * d.k - (p.KB - 1) * BK + 15) / 16;  // 1..4
  p.num_m = (int)((M + BM - 1) / BM);
  p.num_n = (int)((g.n_bins + BN - 1) / BN);
  p.thr2 = d.rho_i * d.rho_i;
  p.bin0 = (int)g.n_bins;
  p.block_id = d.block_id;
  p.cand = cand;
  p.counter = ws.cand_count;
  p.cap = d.cand_capacity;
  p.flags = ws.flags;
  const uint32_t fmt = bf ? 1u : 0u;
  p.idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
  p.withhold_copies = 0;
  return RB_OK;
}

}  // namespace

namespace rb {

int stage1_tc(const rb_filter_desc& d, const rb_basis& b, const Geometry& g, const Workspace& ws, rb_candidate* cand,
              cudaStream_t st) {
  const int planes = plane_mode(d.precision);
  const int v = chosen_variant(d, g);
  CUtensorMap maps[4];
  TcParams p;
  int rc = build_params(d, b, g, ws, cand, v, maps, p);
  if (rc) return rc;
  int left = g_withhold.load();
  while (left > 0 && !g_withhold.compare_exchange_weak(left, left - 1)) {
  }
  p.withhold_copies = left > 0 ? 1 : 0;
  return launch_variant(v, planes, maps, p, st);
}

// Time every variant on the packed operands in the workspace (threshold disabled so no candidate is
// written), remember the fastest for this shape and precision, and report the times.
int tune_stage1(const rb_filter_desc& d, const rb_basis& b, const Geometry& g, const Workspace& ws, double* ms,
                int* chosen, cudaStream_t st) {
  const int planes = plane_mode(d.precision);
  cudaEvent_t e0, e1;
  RB_CUDA_TRY(cudaEventCreate(&e0));
  RB_CUDA_TRY(cudaEventCreate(&e1));
  int best = 0, rc = RB_OK;
  double best_ms = 1e30;
  for (int v = 0; v < kVariants && rc == RB_OK; ++v) {
    CUtensorMap maps[4];
    TcParams p;
    if ((rc = build_params(d, b, g, ws, ws.cand, v, maps, p))) break;
    p.thr2 = INFINITY;
    if ((rc = launch_variant(v, planes, maps, p, st))) break;  // warm-up
    const int reps = 3;
    if (cudaEventRecord(e0, st) != cudaSuccess) rc = RB_ERR_CUDA;
    for (int r = 0; r < reps && rc == RB_OK; ++r) rc = launch_variant(v, planes, maps, p, st);
    if (rc) break;
    float t = 0.f;
    if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
      rc = RB_ERR_CUDA;
      break;
    }
    ms[v] = t / reps;
    if (ms[v] < best_ms) {
      best_ms = ms[v];
      best = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[TuneKey{d.precision, d.n_templates, g.n_bins, g.kp}] = best;
  }
  *chosen = best;
  return RB_OK;
}

int stage1_tc_variants() { return kVariants; }

int set_stage1_variant(const rb_filter_desc& d, const Geometry& g, int variant) {
  if (variant < 0 || variant >= kVariants) {
    set_detail("variant %d out of range", variant);
    return RB_ERR_BAD_INPUT;
  }
  std::lock_guard<std::mutex> lock(g_tune_mu);
  g_tuned[TuneKey{d.precision, d.n_templates, g.n_bins, g.kp}] = variant;
  return RB_OK;
}

}  // namespace rb

// Host-only test hook (not part of the C ABI): the next n tensor-core first-stage launches issue no
// copies, so their bounded waits run out; the call reports RB_ERR_TIMEOUT and the context stays
// usable. Used by the failure-detection test; no other code calls it.
extern "C" int rbx_stage1_withhold_copies(int n) {
  g_withhold.store(n > 0 ? n : 0);
  return 0;
}
