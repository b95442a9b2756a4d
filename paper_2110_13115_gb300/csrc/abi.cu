// C ABI entry points (include/rbmf.h): validation, workspace carving, orchestration.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "common.cuh"
#include "internal.h"

#include <algorithm>
#include <map>
#include <mutex>
#include <atomic>
#include <memory>
#include <vector>

namespace {
thread_local char g_detail[512] = "";
std::atomic<uint64_t> g_launches{0};

// Per-thread profiler: one set of RB_STAGES + 1 events per profiled rb_filter call.
struct Profiler {
  bool on = false;
  std::vector<std::vector<cudaEvent_t>> sets;
};
thread_local Profiler g_prof;

struct StageMarks {
  std::vector<cudaEvent_t>* ev = nullptr;
  cudaStream_t st = nullptr;
  int last = -1;
  void begin(cudaStream_t s) {
    if (!g_prof.on) return;
    g_prof.sets.emplace_back(RB_STAGES + 1, nullptr);
    ev = &g_prof.sets.back();
    for (auto& e : *ev) cudaEventCreate(&e);
    st = s;
    cudaEventRecord((*ev)[0], st);
    last = 0;
  }
  // mark the start of `stage` (= the end of the previous one); skipped stages get zero duration
  void to(int stage) {
    if (!ev) return;
    for (int i = last + 1; i <= stage; ++i) cudaEventRecord((*ev)[i], st);
    last = std::max(last, stage);
  }
  void finish() {
    if (!ev) return;
    for (int i = last + 1; i <= RB_STAGES; ++i) cudaEventRecord((*ev)[i], st);
    last = RB_STAGES;
  }
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Status {
  unsigned flags;
  unsigned pad;
  unsigned long long cand;
  unsigned long long trig;
};
}  // namespace

void rb_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void rb_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_detail, sizeof(g_detail), "CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what,
           file, line);
}

namespace rb {

void set_detail(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_detail, sizeof(g_detail), fmt, ap);
  va_end(ap);
}

int make_geometry(const rb_filter_desc& d, Geometry* g) {
  if (!(d.fs > 0.0) || !std::isfinite(d.fs)) {
    set_detail("fs must be finite and > 0");
    return RB_ERR_BAD_INPUT;
  }
  if (!rb_is_pow2(d.n) || d.n < (1 << 10) || d.n > (1 << 20)) {
    set_detail("n = %lld must be a power of two in [2^10, 2^20]", (long long)d.n);
    return RB_ERR_BAD_INPUT;
  }
  if (d.k < 1 || d.n_templates < 1) {
    set_detail("k = %d and n_templates = %d must be >= 1", d.k, d.n_templates);
    return RB_ERR_BAD_INPUT;
  }
  if (!(d.w == 1 || d.w == 2 || d.w == 4 || d.w == 8 || d.w == 16)) {
    set_detail("w = %d must be 1, 2, 4, 8 or 16", d.w);
    return RB_ERR_BAD_INPUT;
  }
  if (!(d.rho_i >= 0.f) || !(d.rho_ii >= 0.f) || !std::isfinite(d.rho_i) || !std::isfinite(d.rho_ii)) {
    set_detail("thresholds must be finite and >= 0");
    return RB_ERR_BAD_INPUT;
  }
  if (d.cand_capacity < 0 || d.cand_capacity > INT32_MAX ||
      (d.mem & ~(RB_MEM_HOST_STRAIN | RB_MEM_HOST_TRIGGERS)) != 0) {
    set_detail("cand_capacity must be in [0, 2^31) and mem may hold only RB_MEM_* bits");
    return RB_ERR_BAD_INPUT;
  }
  if (d.precision < RB_PREC_FP32 || d.precision > RB_PREC_FP16_SPLIT_A) {
    set_detail("unknown precision %d", d.precision);
    return RB_ERR_UNSUPPORTED;
  }
  const int p = rb_ilog2(d.n);
  g->n = d.n;
  g->n1 = 1 << (p / 2);
  g->n2 = 1 << (p - p / 2);
  g->n_bins = d.n / (2 * d.w);
  g->kp = ((2 * d.k + 63) / 64) * 64;
  g->k16 = (d.k + 15) / 16 * 16;
  g->s2_bytes = (size_t)2 * d.n_templates * (2 * g->k16) * 2;
  return RB_OK;
}

size_t coeff_op_bytes(const rb_filter_desc& d, const Geometry& g) {
  // A planes of the first stage: hi and lo for the split precisions (B split or not), else one
  const bool split_a = d.precision == RB_PREC_FP16_SPLIT || d.precision == RB_PREC_BF16_SPLIT ||
                       d.precision == RB_PREC_FP16_SPLIT_A;
  const size_t stage1 = d.precision == RB_PREC_FP32 ? 0 : (split_a ? 2 : 1) * (size_t)2 * d.n_templates * g.kp * 2;
  return g.s2_bytes + stage1;
}

// Bytes of the trigger staging region for host trigger buffers: 96 MB, at least one n-point vector.
size_t host_trig_bytes(const Geometry& g) {
  return std::max<size_t>(size_t(96) << 20, sizeof(float2) * (size_t)g.n) / sizeof(rb_trigger) * sizeof(rb_trigger);
}

void carve(const rb_filter_desc& d, const Geometry& g, char* base, Workspace* ws, bool plain) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += align256(bytes);
    return p;
  };
  char* st = take(256);
  ws->flags = (unsigned*)st;
  ws->cand_count = st ? (unsigned long long*)(st + 8) : nullptr;
  ws->trig_count = st ? (unsigned long long*)(st + 16) : nullptr;
  ws->host_status = (unsigned long long*)st;
  const int64_t half = g.n / 2;
  ws->tables.n1_w = (float2*)take(sizeof(float2) * g.n1);
  ws->tables.n2_w = (float2*)take(sizeof(float2) * g.n2);
  ws->tables.fine_w = (float2*)take(sizeof(float2) * g.n2);
  ws->tables.w2a_w = (float2*)take(sizeof(float2) * w2_entries(g.n2));
  ws->tables.w2b_w = (float2*)take(sizeof(float2) * w2_entries(g.n1));
  ws->tables.n1 = ws->tables.n1_w;
  ws->tables.n2 = ws->tables.n2_w;
  ws->tables.fine = ws->tables.fine_w;
  ws->tables.w2a = ws->tables.w2a_w;
  ws->tables.w2b = ws->tables.w2b_w;
  ws->wt = (float*)take(sizeof(float) * half);
  ws->shat = (float2*)take(sizeof(float2) * half);
  // everything above depends on n only, so sub-banks that share a workspace share it
  if (!plain && (d.mem & RB_MEM_HOST_TRIGGERS)) ws->trig_stage = (rb_trigger*)take(host_trig_bytes(g));
  const int64_t nvec = plain ? d.n_templates : d.k;
  int64_t vc = (int64_t(96) << 20) / (g.n * 8);  // four-step chunks of up to 96 MB (kept in L2)
  vc = std::max<int64_t>(1, std::min<int64_t>(vc, std::min<int64_t>(nvec, 65535)));
  ws->vc = (int)vc;
  ws->X = (float2*)take(sizeof(float2) * g.n * vc);
  if (!plain) {
    ws->beta = (float2*)take(sizeof(float2) * (size_t)d.k * half);
    ws->bavg = (float2*)take(sizeof(float2) * (size_t)d.k * g.n_bins);
    if (d.precision != RB_PREC_FP32) {
      const size_t plane = (size_t)g.n_bins * g.kp * 2;
      ws->bop_hi = take(plane);
      const bool split = d.precision == RB_PREC_FP16_SPLIT || d.precision == RB_PREC_BF16_SPLIT;
      ws->bop_lo = split ? take(plane) : nullptr;
    }
    ws->cand = (rb_candidate*)take(sizeof(rb_candidate) * (size_t)std::max<int64_t>(d.cand_capacity, 1));
    ws->cand_sorted = (SortedCand*)take(sizeof(SortedCand) * (size_t)std::max<int64_t>(d.cand_capacity, 1));
    ws->bin_count = (unsigned*)take(sizeof(unsigned) * (size_t)(g.n_bins + 1));
    ws->bin_start = (unsigned*)take(sizeof(unsigned) * (size_t)(g.n_bins + 1));
    // pieces: sum over groups of ceil(c_g / piece) <= n_bins + capacity / kStage2MinPiece
    ws->pieces = (int4*)take(sizeof(int4) * (size_t)(g.n_bins + d.cand_capacity / kStage2MinPiece + 1));
    ws->piece_total = (unsigned*)take(sizeof(unsigned));
  }
  ws->total = off;
}

}  // namespace rb

using namespace rb;

namespace {

// Triggers rb_filter and rb_filter_banks can stage on the device for a host trigger buffer.
int64_t host_trig_capacity(const Geometry& g, const Workspace&) {
  return (int64_t)(host_trig_bytes(g) / sizeof(rb_trigger));
}

// A non-blocking stream per device for the trigger copies of rb_filter_banks, created on first use
// and kept for the life of the process.
int copy_stream(cudaStream_t* out) {
  static std::mutex mu;
  static std::map<int, cudaStream_t> streams;
  int dev = 0;
  RB_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  auto it = streams.find(dev);
  if (it == streams.end()) {
    cudaStream_t s = nullptr;
    RB_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    it = streams.emplace(dev, s).first;
  }
  *out = it->second;
  return RB_OK;
}

int prepare(const rb_filter_desc* desc, void* workspace, size_t bytes, bool plain, Geometry* g, Workspace* ws,
            cudaStream_t st, bool host_buffers = false) {
  if (!desc) {
    set_detail("desc is NULL");
    return RB_ERR_BAD_INPUT;
  }
  int rc = make_geometry(*desc, g);
  if (rc) return rc;
  if (desc->mem != 0 && !host_buffers) {
    set_detail("desc->mem = %d: host buffers are taken by rb_filter only; this call wants 0", desc->mem);
    return RB_ERR_BAD_INPUT;
  }
  Workspace probe;
  carve(*desc, *g, nullptr, &probe, plain);
  if (!workspace || bytes < probe.total || ((uintptr_t)workspace & 255)) {
    set_detail("workspace %p of %zu bytes; need %zu bytes, 256-byte aligned", workspace, bytes, probe.total);
    return RB_ERR_OOM;
  }
  carve(*desc, *g, (char*)workspace, ws, plain);
  RB_CUDA_TRY(cudaMemsetAsync(ws->flags, 0, 256, st));
  return RB_OK;
}

int read_status(const Workspace& ws, Status* s, cudaStream_t st) {
  RB_CUDA_TRY(cudaMemcpyAsync(s, ws.host_status, sizeof(Status), cudaMemcpyDeviceToHost, st));
  RB_CUDA_TRY(cudaStreamSynchronize(st));
  return RB_OK;
}

int check_basis(const rb_filter_desc& d, const rb_basis* b, bool need_op = false) {
  if (!b || !b->vectors || !b->coeff) {
    set_detail("basis or its arrays are NULL");
    return RB_ERR_BAD_INPUT;
  }
  if (need_op && !b->coeff_op) {
    set_detail("basis->coeff_op is NULL: pack it with rb_pack_coeff first");
    return RB_ERR_BAD_INPUT;
  }
  if (b->k < d.k || b->n_templates != d.n_templates || b->n != d.n) {
    set_detail("basis (k=%d, T=%d, n=%lld) does not match desc (k=%d, T=%d, n=%lld)", b->k, b->n_templates,
               (long long)b->n, d.k, d.n_templates, (long long)d.n);
    return RB_ERR_BAD_INPUT;
  }
  return RB_OK;
}

// Folded first stage: the whitening FFT of length n and the folded transforms of length M = n / w
// share the status block; X holds max(vc M, n) points (the whitening uses one n-point vector).
struct FoldWs {
  Geometry gn, gm;
  Workspace wn, wm;
  float2* gfold = nullptr;
  size_t total = 0;
};

int fold_geometry(const rb_filter_desc& d, FoldWs* f) {
  int rc = make_geometry(d, &f->gn);
  if (rc) return rc;
  const int64_t M = d.n / d.w;
  if (M < (1 << 10)) {
    set_detail("the folded series has n / w = %lld points; at least 1024 are supported", (long long)M);
    return RB_ERR_UNSUPPORTED;
  }
  const int p = rb_ilog2(M);
  f->gm = Geometry{};
  f->gm.n = M;
  f->gm.n1 = 1 << (p / 2);
  f->gm.n2 = 1 << (p - p / 2);
  f->gm.n_bins = M / 2;
  return RB_OK;
}

void carve_fold(const rb_filter_desc& d, char* base, FoldWs* f) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* ptr = base ? base + off : nullptr;
    off += align256(bytes);
    return ptr;
  };
  const Geometry& gn = f->gn;
  const Geometry& gm = f->gm;
  char* st = take(256);
  for (Workspace* w : {&f->wn, &f->wm}) {
    w->flags = (unsigned*)st;
    w->cand_count = st ? (unsigned long long*)(st + 8) : nullptr;
    w->trig_count = st ? (unsigned long long*)(st + 16) : nullptr;
    w->host_status = (unsigned long long*)st;
  }
  auto tables = [&](Workspace* w, const Geometry& g) {
    w->tables.n1_w = (float2*)take(sizeof(float2) * g.n1);
    w->tables.n2_w = (float2*)take(sizeof(float2) * g.n2);
    w->tables.fine_w = (float2*)take(sizeof(float2) * g.n2);
    w->tables.w2a_w = (float2*)take(sizeof(float2) * w2_entries(g.n2));
    w->tables.w2b_w = (float2*)take(sizeof(float2) * w2_entries(g.n1));
    w->tables.n1 = w->tables.n1_w;
    w->tables.n2 = w->tables.n2_w;
    w->tables.fine = w->tables.fine_w;
    w->tables.w2a = w->tables.w2a_w;
    w->tables.w2b = w->tables.w2b_w;
  };
  tables(&f->wn, gn);
  tables(&f->wm, gm);
  f->wn.wt = (float*)take(sizeof(float) * gn.n / 2);
  f->wn.shat = (float2*)take(sizeof(float2) * gn.n / 2);
  f->wm.shat = f->wn.shat;
  f->gfold = (float2*)take(sizeof(float2) * gn.n / 2);
  int64_t vc = (int64_t(96) << 20) / (gm.n * 8);
  vc = std::max<int64_t>(1, std::min<int64_t>(vc, std::min<int64_t>(d.n_templates, 65535)));
  f->wm.vc = (int)vc;
  f->wn.vc = 1;
  f->wm.X = f->wn.X = (float2*)take(sizeof(float2) * std::max<int64_t>(gm.n * vc, gn.n));
  f->total = off;
}

int run_stage1(const rb_filter_desc& d, const rb_basis& b, const Geometry& g, const Workspace& ws,
                      const float2* bavg, rb_candidate* cand, cudaStream_t st, StageMarks* mk = nullptr) {
  if (d.precision == RB_PREC_FP32) {
    if (mk) mk->to(RB_STAGE_FIRST);
    return stage1_simt(d, b, g, ws, bavg, cand, st);
  }
  if (!b.coeff_op || b.coeff_op_precision != d.precision) {
    set_detail("coeff_op missing or packed for precision %d (need %d)", b.coeff_op_precision, d.precision);
    return RB_ERR_BAD_INPUT;
  }
  int rc = pack_beta(d, g, bavg, ws.bop_hi, ws.bop_lo, st);
  if (rc) return rc;
  if (mk) mk->to(RB_STAGE_FIRST);
  return stage1_tc(d, b, g, ws, cand, st);
}

// ---------------------------------------------------------------------------------------
// Batching: a validated copy of the work list, its enqueue (no host synchronisation, so that it
// can be recorded as a CUDA graph) and the final status read.
struct BatchSpec {
  std::vector<rb_filter_desc> descs;
  std::vector<rb_basis> bases;
  std::vector<Geometry> geos;
  std::vector<rb_block> blocks;
  rb_trigger* trig = nullptr;
  int64_t capacity = 0;
  char* workspace = nullptr;
};

int batch_workspace(const rb_filter_desc* descs, int32_t n, std::vector<Geometry>* geos, size_t* bytes) {
  *bytes = 0;
  for (int32_t i = 0; i < n; ++i) {
    Geometry g;
    int rc = make_geometry(descs[i], &g);
    if (rc) return rc;
    Workspace w;
    carve(descs[i], g, nullptr, &w, false);
    *bytes = std::max(*bytes, w.total);
    if (geos) geos->push_back(g);
  }
  return RB_OK;
}

int batch_validate(const rb_filter_desc* descs, const rb_basis* bases, int32_t n_bases, const rb_block* blocks,
                   int64_t n_blocks, rb_trigger* trig, int64_t capacity, void* workspace, size_t bytes,
                   BatchSpec* out) {
  if (!descs || !bases || n_bases < 1 || n_blocks < 0 || (n_blocks > 0 && !blocks) || capacity < 0 ||
      (capacity > 0 && !trig)) {
    set_detail("NULL array or bad count");
    return RB_ERR_BAD_INPUT;
  }
  size_t need = 0;
  int rc = batch_workspace(descs, n_bases, &out->geos, &need);
  if (rc) return rc;
  for (int32_t i = 0; i < n_bases; ++i) {
    if (descs[i].mem != 0) {
      set_detail("descs[%d].mem = %d: batch blocks take device pointers", i, descs[i].mem);
      return RB_ERR_BAD_INPUT;
    }
    if ((rc = check_basis(descs[i], &bases[i], true))) return rc;
    if (bases[i].coeff_op_precision != descs[i].precision) {
      set_detail("bases[%d] was packed for precision %d, descs[%d] asks for %d", i, bases[i].coeff_op_precision, i,
                 descs[i].precision);
      return RB_ERR_BAD_INPUT;
    }
  }
  if (!workspace || bytes < need || ((uintptr_t)workspace & 255)) {
    set_detail("workspace %p of %zu bytes; need %zu bytes, 256-byte aligned", workspace, bytes, need);
    return RB_ERR_OOM;
  }
  for (int64_t i = 0; i < n_blocks; ++i) {
    const rb_block& b = blocks[i];
    if (b.basis < 0 || b.basis >= n_bases || !b.strain || !b.psd) {
      set_detail("blocks[%lld]: basis index %d (of %d) or NULL strain / psd", (long long)i, b.basis, n_bases);
      return RB_ERR_BAD_INPUT;
    }
    const rb_filter_desc& d = descs[b.basis];
    if (b.valid_lo < d.n / 2 || b.valid_lo >= d.n || b.valid_lo % d.w) {
      set_detail("blocks[%lld]: valid_lo %lld must lie in [n/2, n) and be a multiple of w", (long long)i,
                 (long long)b.valid_lo);
      return RB_ERR_BAD_INPUT;
    }
  }
  out->descs.assign(descs, descs + n_bases);
  out->bases.assign(bases, bases + n_bases);
  out->blocks.assign(blocks, blocks + n_blocks);
  out->trig = trig;
  out->capacity = capacity;
  out->workspace = (char*)workspace;
  return RB_OK;
}

// Every block runs the rb_filter pipeline through the one workspace; the status block (flags and
// counters, the first 256 bytes of every carving) is cleared once, so triggers of all blocks share
// one counter and the flags are sticky. Only the candidate count is reset per block.
int batch_enqueue(const BatchSpec& s, cudaStream_t st) {
  Workspace ws0;
  carve(s.descs[0], s.geos[0], s.workspace, &ws0, false);
  RB_CUDA_TRY(cudaMemsetAsync(ws0.flags, 0, 256, st));
  for (const rb_block& blk : s.blocks) {
    rb_filter_desc d = s.descs[blk.basis];
    d.sample_offset = blk.sample_offset;
    d.block_id = blk.block_id;
    const Geometry& g = s.geos[blk.basis];
    const rb_basis& b = s.bases[blk.basis];
    Workspace ws;
    carve(d, g, s.workspace, &ws, false);
    RB_CUDA_TRY(cudaMemsetAsync(ws.cand_count, 0, sizeof(unsigned long long), st));
    int rc;
    if ((rc = init_tables(g, ws, blk.psd, d.fs, st))) return rc;
    if ((rc = whiten(g, ws, blk.strain, ws.shat, st))) return rc;
    if ((rc = bank_filter(g, ws, (const float2*)b.vectors, d.k, ws.shat, ws.beta, ws.bavg, d.w, st))) return rc;
    if ((rc = run_stage1(d, b, g, ws, ws.bavg, ws.cand, st))) return rc;
    const int bin_lo = (int)((blk.valid_lo - d.n / 2) / d.w);
    if ((rc = stage2_bucketed(d, b, g, ws, ws.beta, s.trig, s.capacity, ws.trig_count, bin_lo, st))) return rc;
  }
  return RB_OK;
}

int batch_status(const BatchSpec& s, int64_t* n_trig, cudaStream_t st) {
  Workspace ws0;
  carve(s.descs[0], s.geos[0], s.workspace, &ws0, false);
  Status stt;
  int rc = read_status(ws0, &stt, st);
  if (rc) return rc;
  *n_trig = (int64_t)stt.trig;
  if (stt.flags & RB_FLAG_BAD_PSD) {
    set_detail("a block's PSD is not finite and positive on 0 < j < n/2");
    return RB_ERR_BAD_INPUT;
  }
  if (stt.flags & RB_FLAG_TIMEOUT) {
    set_detail("a bounded device-side wait (tcgen05 first or second stage) timed out");
    return RB_ERR_TIMEOUT;
  }
  if (stt.flags & RB_FLAG_CAND_OVERFLOW) {
    set_detail("a block had more first-stage candidates than its desc's cand_capacity");
    return RB_ERR_OVERFLOW;
  }
  if ((int64_t)stt.trig > s.capacity) {
    set_detail("%llu triggers exceed capacity %lld", stt.trig, (long long)s.capacity);
    return RB_ERR_OVERFLOW;
  }
  return RB_OK;
}

}  // namespace

struct rb_batch {
  BatchSpec spec;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t launches = 0;  // kernels recorded in the graph
};

extern "C" {

const char* rb_strerror(int status) {
  switch (status) {
    case RB_OK: return "ok";
    case RB_ERR_BAD_INPUT: return "bad input";
    case RB_ERR_OOM: return "workspace too small";
    case RB_ERR_OVERFLOW: return "output overflow";
    case RB_ERR_TIMEOUT: return "device wait timed out";
    case RB_ERR_CUDA: return "CUDA error";
    case RB_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* rb_last_error_detail(void) { return g_detail; }

int rb_version(void) { return 100; }

uint64_t rb_kernel_launches(void) { return g_launches.load(); }

int rb_profile_start(void) {
  g_prof.on = true;
  g_prof.sets.clear();
  return RB_OK;
}

int rb_profile_stop(double* stage_ms, int64_t* calls) {
  if (!g_prof.on) {
    set_detail("rb_profile_stop without rb_profile_start");
    return RB_ERR_BAD_INPUT;
  }
  g_prof.on = false;
  std::vector<double> acc(RB_STAGES, 0.0);
  int rc = RB_OK;
  for (auto& set : g_prof.sets) {
    if (cudaEventSynchronize(set[RB_STAGES]) != cudaSuccess) rc = RB_ERR_CUDA;
    for (int i = 0; i < RB_STAGES && rc == RB_OK; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, set[i], set[i + 1]) != cudaSuccess) rc = RB_ERR_CUDA;
      acc[i] += ms;
    }
    for (auto e : set) cudaEventDestroy(e);
  }
  const int64_t n = (int64_t)g_prof.sets.size();
  g_prof.sets.clear();
  if (calls) *calls = n;
  if (stage_ms)
    for (int i = 0; i < RB_STAGES; ++i) stage_ms[i] = n ? acc[i] / n : 0.0;
  if (rc) set_detail("profiling events failed");
  return rc;
}

int rb_filter_plan(const rb_filter_desc* desc, rb_filter_sizes* out) {
  if (!desc || !out) {
    set_detail("NULL argument");
    return RB_ERR_BAD_INPUT;
  }
  Geometry g;
  int rc = make_geometry(*desc, &g);
  if (rc) return rc;
  Workspace a, b;
  carve(*desc, g, nullptr, &a, false);
  carve(*desc, g, nullptr, &b, true);
  out->workspace_bytes = std::max(a.total, b.total);
  out->n_bins = g.n_bins;
  out->n1 = g.n1;
  out->n2 = g.n2;
  out->kp = g.kp;
  out->coeff_op_bytes = coeff_op_bytes(*desc, g);
  out->host_trig_capacity = host_trig_capacity(g, a);
  return RB_OK;
}

int rb_whiten(const rb_filter_desc* desc, const float* strain, const double* psd, float* s_hat, void* workspace,
              size_t workspace_bytes, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  Geometry g;
  Workspace ws;
  int rc = prepare(desc, workspace, workspace_bytes, true, &g, &ws, st);
  if (rc) return rc;
  if (!strain || !psd || !s_hat) {
    set_detail("NULL array");
    return RB_ERR_BAD_INPUT;
  }
  if ((rc = init_tables(g, ws, psd, desc->fs, st))) return rc;
  if ((rc = whiten(g, ws, strain, (float2*)s_hat, st))) return rc;
  Status s;
  if ((rc = read_status(ws, &s, st))) return rc;
  if (s.flags & RB_FLAG_BAD_PSD) {
    set_detail("PSD not finite and positive on 0 < j < n/2");
    return RB_ERR_BAD_INPUT;
  }
  return RB_OK;
}

int rb_basis_filter(const rb_filter_desc* desc, const rb_basis* basis, const float* s_hat, float* beta,
                    float* beta_avg, void* workspace, size_t workspace_bytes, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  Geometry g;
  Workspace ws;
  int rc = prepare(desc, workspace, workspace_bytes, false, &g, &ws, st);
  if (rc) return rc;
  if ((rc = check_basis(*desc, basis))) return rc;
  if (!s_hat || !beta_avg) {
    set_detail("NULL array");
    return RB_ERR_BAD_INPUT;
  }
  if ((rc = init_tables(g, ws, nullptr, desc->fs, st))) return rc;
  return bank_filter(g, ws, (const float2*)basis->vectors, desc->k, (const float2*)s_hat, (float2*)beta,
                     (float2*)beta_avg, desc->w, st);
}

int rb_pack_coeff(const rb_filter_desc* desc, const rb_basis* basis, void* out, void* stream) {
  if (!desc) return RB_ERR_BAD_INPUT;
  Geometry g;
  int rc = make_geometry(*desc, &g);
  if (rc) return rc;
  if ((rc = check_basis(*desc, basis))) return rc;
  if (!out || (reinterpret_cast<uintptr_t>(out) & 255)) {
    set_detail("out is NULL or not 256-byte aligned");
    return RB_ERR_BAD_INPUT;
  }
  return pack_coeff(*desc, *basis, g, out, (cudaStream_t)stream);
}


int rb_stage1(const rb_filter_desc* desc, const rb_basis* basis, const float* beta_avg, rb_candidate* cand,
              int64_t* n_cand, void* workspace, size_t workspace_bytes, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  Geometry g;
  Workspace ws;
  int rc = prepare(desc, workspace, workspace_bytes, false, &g, &ws, st);
  if (rc) return rc;
  if ((rc = check_basis(*desc, basis))) return rc;
  if (!beta_avg || !cand || !n_cand) {
    set_detail("NULL array");
    return RB_ERR_BAD_INPUT;
  }
  if ((rc = run_stage1(*desc, *basis, g, ws, (const float2*)beta_avg, cand, st))) return rc;
  Status s;
  if ((rc = read_status(ws, &s, st))) return rc;
  if (s.flags & RB_FLAG_TIMEOUT) {
    set_detail("a device-side wait of the first stage timed out");
    return RB_ERR_TIMEOUT;
  }
  *n_cand = (int64_t)s.cand;
  return (int64_t)s.cand > desc->cand_capacity ? RB_ERR_OVERFLOW : RB_OK;
}

int rb_set_stage1_variant(const rb_filter_desc* desc, int32_t variant) {
  if (!desc) {
    set_detail("desc is NULL");
    return RB_ERR_BAD_INPUT;
  }
  Geometry g;
  int rc = make_geometry(*desc, &g);
  if (rc) return rc;
  return set_stage1_variant(*desc, g, variant);
}

int rb_set_fft_variant(const rb_filter_desc* desc, int32_t variant) {
  if (!desc) {
    set_detail("desc is NULL");
    return RB_ERR_BAD_INPUT;
  }
  Geometry g;
  int rc = make_geometry(*desc, &g);
  if (rc) return rc;
  return set_fft_variant(g, desc->w, variant);
}

int rb_tune_fft(const rb_filter_desc* desc, const rb_basis* basis, const float* s_hat, double* times_ms,
                int32_t* chosen, void* workspace, size_t workspace_bytes, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  Geometry g;
  Workspace ws;
  int rc = prepare(desc, workspace, workspace_bytes, false, &g, &ws, st);
  if (rc) return rc;
  if ((rc = check_basis(*desc, basis))) return rc;
  if (!s_hat || !times_ms || !chosen) {
    set_detail("NULL argument");
    return RB_ERR_BAD_INPUT;
  }
  if ((rc = init_tables(g, ws, nullptr, desc->fs, st))) return rc;
  for (int v = 0; v < RB_FFT_VARIANTS; ++v) times_ms[v] = -1.0;
  int best = 0;
  if ((rc = tune_fft(g, ws, (const float2*)basis->vectors, desc->k, (const float2*)s_hat, ws.beta, ws.bavg,
                     desc->w, times_ms, &best, st)))
    return rc;
  *chosen = best;
  return RB_OK;
}

int rb_tune_stage1(const rb_filter_desc* desc, const rb_basis* basis, const float* beta_avg, double* times_ms,
                   int32_t* chosen, void* workspace, size_t workspace_bytes, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  Geometry g;
  Workspace ws;
  int rc = prepare(desc, workspace, workspace_bytes, false, &g, &ws, st);
  if (rc) return rc;
  if ((rc = check_basis(*desc, basis))) return rc;
  if (desc->precision == RB_PREC_FP32 || !basis->coeff_op || basis->coeff_op_precision != desc->precision) {
    set_detail("tuning needs a 16-bit precision with a matching packed coeff_op");
    return RB_ERR_BAD_INPUT;
  }
  if (!beta_avg || !times_ms || !chosen) {
    set_detail("NULL argument");
    return RB_ERR_BAD_INPUT;
  }
  if ((rc = pack_beta(*desc, g, (const float2*)beta_avg, ws.bop_hi, ws.bop_lo, st))) return rc;
  for (int v = 0; v < RB_STAGE1_VARIANTS; ++v) times_ms[v] = -1.0;
  int best = 0;
  if ((rc = tune_stage1(*desc, *basis, g, ws, times_ms, &best, st))) return rc;
  *chosen = best;
  return RB_OK;
}

int rb_stage2(const rb_filter_desc* desc, const rb_basis* basis, const float* beta, const rb_candidate* cand,
              int64_t n_cand, rb_trigger* trig, int64_t capacity, int64_t* n_trig, void* workspace,
              size_t workspace_bytes, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  Geometry g;
  Workspace ws;
  int rc = prepare(desc, workspace, workspace_bytes, false, &g, &ws, st);
  if (rc) return rc;
  if ((rc = check_basis(*desc, basis, true))) return rc;
  if (!beta || (n_cand > 0 && !cand) || !n_trig || capacity < 0 || n_cand < 0 || (capacity > 0 && !trig)) {
    set_detail("NULL array or negative count");
    return RB_ERR_BAD_INPUT;
  }
  if (n_cand > desc->cand_capacity) {
    set_detail("n_cand %lld exceeds desc->cand_capacity %lld", (long long)n_cand, (long long)desc->cand_capacity);
    return RB_ERR_BAD_INPUT;
  }
  if (n_cand > 0) {
    const unsigned long long cnt = (unsigned long long)n_cand;
    RB_CUDA_TRY(cudaMemcpyAsync(ws.cand, cand, sizeof(rb_candidate) * n_cand, cudaMemcpyDeviceToDevice, st));
    RB_CUDA_TRY(cudaMemcpyAsync(ws.cand_count, &cnt, sizeof(cnt), cudaMemcpyHostToDevice, st));
    RB_CUDA_TRY(cudaStreamSynchronize(st));  // cnt lives on this stack frame
    if ((rc = stage2_bucketed(*desc, *basis, g, ws, (const float2*)beta, trig, capacity, ws.trig_count, 0, st))) return rc;
  }
  Status s;
  if ((rc = read_status(ws, &s, st))) return rc;
  *n_trig = (int64_t)s.trig;
  if (s.flags & RB_FLAG_TIMEOUT) {
    set_detail("a bounded device-side wait of the tcgen05 second stage timed out");
    return RB_ERR_TIMEOUT;
  }
  return (int64_t)s.trig > capacity ? RB_ERR_OVERFLOW : RB_OK;
}

int rb_filter(const rb_filter_desc* desc, const rb_basis* basis, const float* strain, const double* psd,
              rb_trigger* trig, int64_t capacity, int64_t* n_trig, void* workspace, size_t workspace_bytes,
              void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  Geometry g;
  Workspace ws;
  int rc = prepare(desc, workspace, workspace_bytes, false, &g, &ws, st, true);
  if (rc) return rc;
  if ((rc = check_basis(*desc, basis, true))) return rc;
  if (!strain || !psd || !n_trig || capacity < 0 || (capacity > 0 && !trig)) {
    set_detail("NULL array or negative capacity");
    return RB_ERR_BAD_INPUT;
  }
  // host buffers: the strain is staged in the beta region (written only after the whitening FFT
  // has read it) and the triggers in the staging region
  const bool host_in = desc->mem & RB_MEM_HOST_STRAIN, host_out = desc->mem & RB_MEM_HOST_TRIGGERS;
  if (host_out && capacity > host_trig_capacity(g, ws)) {
    set_detail("capacity %lld exceeds host_trig_capacity %lld", (long long)capacity,
               (long long)host_trig_capacity(g, ws));
    return RB_ERR_BAD_INPUT;
  }
  rb_trigger* trig_d = host_out ? ws.trig_stage : trig;
  StageMarks mk;
  mk.begin(st);
  if (host_in) {
    RB_CUDA_TRY(cudaMemcpyAsync(ws.beta, strain, sizeof(float) * g.n, cudaMemcpyHostToDevice, st));
    strain = reinterpret_cast<const float*>(ws.beta);
  }
  if ((rc = init_tables(g, ws, psd, desc->fs, st))) return rc;
  mk.to(RB_STAGE_WHITEN);
  if ((rc = whiten(g, ws, strain, ws.shat, st))) return rc;
  mk.to(RB_STAGE_BASIS);
  if ((rc = bank_filter(g, ws, (const float2*)basis->vectors, desc->k, ws.shat, ws.beta, ws.bavg, desc->w, st)))
    return rc;
  mk.to(RB_STAGE_PACK);
  if ((rc = run_stage1(*desc, *basis, g, ws, ws.bavg, ws.cand, st, &mk))) return rc;
  mk.to(RB_STAGE_BUCKET);
  if ((rc = stage2_bucket(*desc, g, ws, 0, st))) return rc;
  mk.to(RB_STAGE_SECOND);
  if ((rc = stage2_run(*desc, *basis, g, ws, ws.beta, trig_d, capacity, ws.trig_count, st))) return rc;
  mk.finish();
  Status s;
  if ((rc = read_status(ws, &s, st))) return rc;
  if (host_out && s.trig > 0 && capacity > 0) {
    const int64_t copied = std::min<int64_t>((int64_t)s.trig, capacity);
    RB_CUDA_TRY(cudaMemcpyAsync(trig, trig_d, sizeof(rb_trigger) * copied, cudaMemcpyDeviceToHost, st));
    RB_CUDA_TRY(cudaStreamSynchronize(st));
  }
  if (s.flags & RB_FLAG_BAD_PSD) {
    set_detail("PSD not finite and positive on 0 < j < n/2");
    return RB_ERR_BAD_INPUT;
  }
  if (s.flags & RB_FLAG_TIMEOUT) {
    set_detail("a bounded device-side wait (tcgen05 first or second stage) timed out");
    return RB_ERR_TIMEOUT;
  }
  if ((int64_t)s.cand > desc->cand_capacity) {
    *n_trig = -1;
    set_detail("%llu first-stage candidates exceed cand_capacity %lld", s.cand, (long long)desc->cand_capacity);
    return RB_ERR_OVERFLOW;
  }
  *n_trig = (int64_t)s.trig;
  if ((int64_t)s.trig > capacity) {
    set_detail("%llu triggers exceed capacity %lld", s.trig, (long long)capacity);
    return RB_ERR_OVERFLOW;
  }
  return RB_OK;
}

int rb_banks_plan(const rb_filter_desc* descs, int32_t n_banks, rb_filter_sizes* out) {
  if (!descs || !out || n_banks < 1) {
    set_detail("NULL argument or n_banks < 1");
    return RB_ERR_BAD_INPUT;
  }
  rb_filter_sizes s{};
  int64_t host_cap = INT64_MAX;
  for (int32_t b = 0; b < n_banks; ++b) {
    Geometry g;
    int rc = make_geometry(descs[b], &g);
    if (rc) return rc;
    if (descs[b].n != descs[0].n || descs[b].fs != descs[0].fs || descs[b].w != descs[0].w ||
        descs[b].mem != descs[0].mem) {
      set_detail("descs[%d] differs from descs[0] in n, fs, w or mem", b);
      return RB_ERR_BAD_INPUT;
    }
    Workspace w;
    carve(descs[b], g, nullptr, &w, false);
    s.workspace_bytes = std::max(s.workspace_bytes, w.total);
    s.n_bins = g.n_bins;
    s.n1 = g.n1;
    s.n2 = g.n2;
    s.kp = std::max(s.kp, g.kp);
    host_cap = std::min(host_cap, host_trig_capacity(g, w));
  }
  s.coeff_op_bytes = 0;
  s.host_trig_capacity = host_cap;
  *out = s;
  return RB_OK;
}

int rb_filter_banks(const rb_filter_desc* descs, const rb_basis* bases, int32_t n_banks, const float* strain,
                    const double* psd, rb_trigger* trig, int64_t capacity, int64_t* n_trig, void* workspace,
                    size_t workspace_bytes, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  rb_filter_sizes plan;
  int rc = rb_banks_plan(descs, n_banks, &plan);
  if (rc) return rc;
  if (!bases || !strain || !psd || !n_trig || capacity < 0 || (capacity > 0 && !trig)) {
    set_detail("NULL array or negative capacity");
    return RB_ERR_BAD_INPUT;
  }
  if (!workspace || workspace_bytes < plan.workspace_bytes || ((uintptr_t)workspace & 255)) {
    set_detail("workspace %p of %zu bytes; need %zu bytes, 256-byte aligned", workspace, workspace_bytes,
               plan.workspace_bytes);
    return RB_ERR_OOM;
  }
  int64_t rows = 0;
  for (int32_t b = 0; b < n_banks; ++b) {
    if ((rc = check_basis(descs[b], &bases[b], true))) return rc;
    if (bases[b].coeff_op_precision != descs[b].precision) {
      set_detail("bases[%d] was packed for precision %d, descs[%d] asks for %d", b, bases[b].coeff_op_precision, b,
                 descs[b].precision);
      return RB_ERR_BAD_INPUT;
    }
    rows += descs[b].n_templates;
  }
  if (rows > INT32_MAX) {
    set_detail("the sub-banks hold %lld templates in all (at most 2^31 - 1)", (long long)rows);
    return RB_ERR_BAD_INPUT;
  }
  const bool host_in = descs[0].mem & RB_MEM_HOST_STRAIN, host_out = descs[0].mem & RB_MEM_HOST_TRIGGERS;
  if (host_out && capacity > plan.host_trig_capacity) {
    set_detail("capacity %lld exceeds host_trig_capacity %lld", (long long)capacity,
               (long long)plan.host_trig_capacity);
    return RB_ERR_BAD_INPUT;
  }
  // every carving shares the status block, the tables, the whitening weights and s_hat (their offsets
  // depend on n only), so the block is whitened once; the rest is per sub-bank scratch
  Geometry g0;
  Workspace ws0;
  if ((rc = make_geometry(descs[0], &g0))) return rc;
  carve(descs[0], g0, (char*)workspace, &ws0, false);
  RB_CUDA_TRY(cudaMemsetAsync(ws0.flags, 0, 256, st));
  rb_trigger* trig_d = host_out ? ws0.trig_stage : trig;
  // host triggers: once sub-bank b is done (its event), its triggers go out on a side stream while the
  // sub-banks after it run on `stream`; the staging region is not touched by later sub-banks except
  // past their own count
  cudaStream_t cs = nullptr;
  std::vector<cudaEvent_t> done;
  // on every return: the copies into the caller's host buffer have landed (an early error return
  // included), then the events go
  struct EventGuard {
    std::vector<cudaEvent_t>& ev;
    cudaStream_t& cs;
    ~EventGuard() {
      if (cs) cudaStreamSynchronize(cs);
      for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    }
  } guard{done, cs};
  if (host_out) {
    if ((rc = copy_stream(&cs))) return rc;
    done.resize(n_banks, nullptr);
    for (auto& e : done) RB_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  int64_t copied = 0;
  // copies sub-bank j's new triggers (blocks the host until sub-bank j is done)
  auto flush = [&](int j) -> int {
    unsigned long long cnt = 0;
    RB_CUDA_TRY(cudaStreamWaitEvent(cs, done[j], 0));
    RB_CUDA_TRY(cudaMemcpyAsync(&cnt, ws0.trig_count, sizeof(cnt), cudaMemcpyDeviceToHost, cs));
    RB_CUDA_TRY(cudaStreamSynchronize(cs));
    const int64_t upto = std::min<int64_t>((int64_t)cnt, capacity);
    if (upto > copied)
      RB_CUDA_TRY(cudaMemcpyAsync(trig + copied, trig_d + copied, sizeof(rb_trigger) * (upto - copied),
                                  cudaMemcpyDeviceToHost, cs));
    copied = std::max(copied, upto);
    return RB_OK;
  };
  StageMarks mk;
  mk.begin(st);
  if (host_in) {
    RB_CUDA_TRY(cudaMemcpyAsync(ws0.beta, strain, sizeof(float) * g0.n, cudaMemcpyHostToDevice, st));
    strain = reinterpret_cast<const float*>(ws0.beta);
  }
  if ((rc = init_tables(g0, ws0, psd, descs[0].fs, st))) return rc;
  mk.to(RB_STAGE_WHITEN);
  if ((rc = whiten(g0, ws0, strain, ws0.shat, st))) return rc;
  int64_t base = 0;
  Status s{};
  for (int32_t b = 0; b < n_banks; ++b) {
    rb_filter_desc d = descs[b];
    d.sample_offset = descs[0].sample_offset;
    d.block_id = descs[0].block_id;
    Geometry g;
    Workspace ws;
    make_geometry(d, &g);
    carve(d, g, (char*)workspace, &ws, false);
    // profiling: one event set per sub-bank (the first also holds the set-up and the whitening), so
    // the per-stage means of rb_profile_stop times n_banks are the per-call totals
    if (b > 0) mk.begin(st);
    RB_CUDA_TRY(cudaMemsetAsync(ws.cand_count, 0, sizeof(unsigned long long), st));
    mk.to(RB_STAGE_BASIS);
    if ((rc = bank_filter(g, ws, (const float2*)bases[b].vectors, d.k, ws.shat, ws.beta, ws.bavg, d.w, st))) return rc;
    mk.to(RB_STAGE_PACK);
    if ((rc = run_stage1(d, bases[b], g, ws, ws.bavg, ws.cand, st, &mk))) return rc;
    mk.to(RB_STAGE_BUCKET);
    if ((rc = stage2_bucket(d, g, ws, 0, st))) return rc;
    mk.to(RB_STAGE_SECOND);
    if ((rc = stage2_run(d, bases[b], g, ws, ws.beta, trig_d, capacity, ws.trig_count, st, (int)base))) return rc;
    mk.finish();
    base += d.n_templates;
    if (host_out) {
      RB_CUDA_TRY(cudaEventRecord(done[b], st));
      if (b > 0 && (rc = flush(b - 1))) return rc;  // sub-bank b is queued behind it meanwhile
    }
  }
  if (host_out) {
    if ((rc = flush(n_banks - 1))) return rc;
    RB_CUDA_TRY(cudaStreamSynchronize(cs));
  }
  if ((rc = read_status(ws0, &s, st))) return rc;
  if (s.flags & RB_FLAG_BAD_PSD) {
    set_detail("PSD not finite and positive on 0 < j < n/2");
    return RB_ERR_BAD_INPUT;
  }
  if (s.flags & RB_FLAG_TIMEOUT) {
    set_detail("a bounded device-side wait (tcgen05 first or second stage) timed out");
    return RB_ERR_TIMEOUT;
  }
  if (s.flags & RB_FLAG_CAND_OVERFLOW) {
    *n_trig = -1;
    set_detail("a sub-bank had more first-stage candidates than its desc's cand_capacity");
    return RB_ERR_OVERFLOW;
  }
  *n_trig = (int64_t)s.trig;
  if ((int64_t)s.trig > capacity) {
    set_detail("%llu triggers exceed capacity %lld", s.trig, (long long)capacity);
    return RB_ERR_OVERFLOW;
  }
  return RB_OK;
}

int rb_folded_plan(const rb_filter_desc* desc, size_t* workspace_bytes) {
  if (!desc || !workspace_bytes) {
    set_detail("NULL argument");
    return RB_ERR_BAD_INPUT;
  }
  FoldWs f;
  int rc = fold_geometry(*desc, &f);
  if (rc) return rc;
  if (desc->w < 2) {
    set_detail("the folded first stage needs w >= 2");
    return RB_ERR_BAD_INPUT;
  }
  carve_fold(*desc, nullptr, &f);
  *workspace_bytes = f.total;
  return RB_OK;
}

static int template_first_stage(const rb_filter_desc* desc, const float* templates, const float* strain,
                                const double* psd, rb_candidate* cand, int64_t* n_cand, void* workspace,
                                size_t workspace_bytes, void* stream, bool lowpass) {
  cudaStream_t st = (cudaStream_t)stream;
  size_t need = 0;
  int rc = rb_folded_plan(desc, &need);
  if (rc) return rc;
  if (desc->mem != 0) {
    set_detail("desc->mem = %d: this call takes device pointers", desc->mem);
    return RB_ERR_BAD_INPUT;
  }
  if (!templates || !strain || !psd || !n_cand || (desc->cand_capacity > 0 && !cand)) {
    set_detail("NULL array");
    return RB_ERR_BAD_INPUT;
  }
  if (!workspace || workspace_bytes < need || ((uintptr_t)workspace & 255)) {
    set_detail("workspace %p of %zu bytes; need %zu bytes, 256-byte aligned", workspace, workspace_bytes, need);
    return RB_ERR_OOM;
  }
  FoldWs f;
  fold_geometry(*desc, &f);
  carve_fold(*desc, (char*)workspace, &f);
  RB_CUDA_TRY(cudaMemsetAsync(f.wn.flags, 0, 256, st));
  if ((rc = init_tables(f.gn, f.wn, psd, desc->fs, st))) return rc;
  if ((rc = init_tables(f.gm, f.wm, nullptr, desc->fs, st))) return rc;
  if ((rc = whiten(f.gn, f.wn, strain, f.wn.shat, st))) return rc;
  if (!lowpass && (rc = init_gfold(f.gfold, desc->n, desc->w, st))) return rc;
  if ((rc = folded_stage1(f.gm, f.wm, (const float2*)templates, desc->n_templates, f.wn.shat, desc->w,
                          desc->rho_i * desc->rho_i, desc->block_id, cand, desc->cand_capacity, f.gfold, st,
                          lowpass)))
    return rc;
  Status s;
  if ((rc = read_status(f.wn, &s, st))) return rc;
  if (s.flags & RB_FLAG_BAD_PSD) {
    set_detail("PSD not finite and positive on 0 < j < n/2");
    return RB_ERR_BAD_INPUT;
  }
  *n_cand = (int64_t)s.cand;
  if ((int64_t)s.cand > desc->cand_capacity) {
    set_detail("%llu candidates exceed cand_capacity %lld", s.cand, (long long)desc->cand_capacity);
    return RB_ERR_OVERFLOW;
  }
  return RB_OK;
}

int rb_stage1_folded(const rb_filter_desc* desc, const float* templates, const float* strain, const double* psd,
                     rb_candidate* cand, int64_t* n_cand, void* workspace, size_t workspace_bytes, void* stream) {
  return template_first_stage(desc, templates, strain, psd, cand, n_cand, workspace, workspace_bytes, stream, false);
}

int rb_stage1_lowpass(const rb_filter_desc* desc, const float* templates, const float* strain, const double* psd,
                      rb_candidate* cand, int64_t* n_cand, void* workspace, size_t workspace_bytes, void* stream) {
  return template_first_stage(desc, templates, strain, psd, cand, n_cand, workspace, workspace_bytes, stream, true);
}

int rb_filter_plain(const rb_filter_desc* desc, const float* templates, const float* strain, const double* psd,
                    rb_trigger* trig, int64_t capacity, int64_t* n_trig, void* workspace, size_t workspace_bytes,
                    void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  Geometry g;
  Workspace ws;
  int rc = prepare(desc, workspace, workspace_bytes, true, &g, &ws, st);
  if (rc) return rc;
  if (!templates || !strain || !psd || !n_trig || capacity < 0 || (capacity > 0 && !trig)) {
    set_detail("NULL array or negative capacity");
    return RB_ERR_BAD_INPUT;
  }
  if ((rc = init_tables(g, ws, psd, desc->fs, st))) return rc;
  if ((rc = whiten(g, ws, strain, ws.shat, st))) return rc;
  if ((rc = plain_filter(g, ws, (const float2*)templates, desc->n_templates, ws.shat, desc->w,
                         desc->rho_ii * desc->rho_ii, desc->sample_offset, desc->block_id, trig, capacity, st)))
    return rc;
  Status s;
  if ((rc = read_status(ws, &s, st))) return rc;
  if (s.flags & RB_FLAG_BAD_PSD) {
    set_detail("PSD not finite and positive on 0 < j < n/2");
    return RB_ERR_BAD_INPUT;
  }
  *n_trig = (int64_t)s.trig;
  if ((int64_t)s.trig > capacity) {
    set_detail("%llu triggers exceed capacity %lld", s.trig, (long long)capacity);
    return RB_ERR_OVERFLOW;
  }
  return RB_OK;
}

int rb_batch_plan(const rb_filter_desc* descs, int32_t n_descs, size_t* workspace_bytes) {
  if (!descs || n_descs < 1 || !workspace_bytes) {
    set_detail("NULL argument or n_descs < 1");
    return RB_ERR_BAD_INPUT;
  }
  return batch_workspace(descs, n_descs, nullptr, workspace_bytes);
}

int rb_filter_batch(const rb_filter_desc* descs, const rb_basis* bases, int32_t n_bases, const rb_block* blocks,
                    int64_t n_blocks, rb_trigger* trig, int64_t capacity, int64_t* n_trig, void* workspace,
                    size_t workspace_bytes, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (!n_trig) {
    set_detail("n_trig is NULL");
    return RB_ERR_BAD_INPUT;
  }
  BatchSpec spec;
  int rc = batch_validate(descs, bases, n_bases, blocks, n_blocks, trig, capacity, workspace, workspace_bytes, &spec);
  if (rc) return rc;
  if ((rc = batch_enqueue(spec, st))) return rc;
  return batch_status(spec, n_trig, st);
}

int rb_batch_create(const rb_filter_desc* descs, const rb_basis* bases, int32_t n_bases, const rb_block* blocks,
                    int64_t n_blocks, rb_trigger* trig, int64_t capacity, void* workspace, size_t workspace_bytes,
                    rb_batch** out) {
  if (!out) {
    set_detail("out is NULL");
    return RB_ERR_BAD_INPUT;
  }
  *out = nullptr;
  std::unique_ptr<rb_batch> bt(new rb_batch);
  int rc = batch_validate(descs, bases, n_bases, blocks, n_blocks, trig, capacity, workspace, workspace_bytes,
                          &bt->spec);
  if (rc) return rc;
  // record on a private stream (the caller's may be the legacy default stream, which cannot capture)
  cudaStream_t cs = nullptr;
  RB_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  const uint64_t l0 = g_launches.load();
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cs);
    set_detail("cudaStreamBeginCapture: %s", cudaGetErrorString(e));
    return RB_ERR_CUDA;
  }
  rc = batch_enqueue(bt->spec, cs);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cs, &graph);
  cudaStreamDestroy(cs);
  const uint64_t recorded = g_launches.load() - l0;
  g_launches.fetch_sub(recorded);  // recorded, not launched: counted at each run
  if (rc == RB_OK && (e != cudaSuccess || !graph)) {
    set_detail("stream capture failed: %s", cudaGetErrorString(e));
    rc = RB_ERR_CUDA;
  }
  if (rc == RB_OK) {
    e = cudaGraphInstantiate(&bt->exec, graph, 0);
    if (e != cudaSuccess) {
      set_detail("cudaGraphInstantiate: %s", cudaGetErrorString(e));
      rc = RB_ERR_CUDA;
    }
  }
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc;
  }
  bt->graph = graph;
  bt->launches = recorded;
  *out = bt.release();
  return RB_OK;
}

int rb_batch_run(rb_batch* batch, int64_t* n_trig, void* stream) {
  if (!batch || !n_trig) {
    set_detail("NULL argument");
    return RB_ERR_BAD_INPUT;
  }
  cudaStream_t st = (cudaStream_t)stream;
  RB_CUDA_TRY(cudaGraphLaunch(batch->exec, st));
  g_launches.fetch_add(batch->launches);
  return batch_status(batch->spec, n_trig, st);
}

int rb_batch_destroy(rb_batch* batch) {
  if (!batch) return RB_OK;
  int rc = RB_OK;
  if (batch->exec && cudaGraphExecDestroy(batch->exec) != cudaSuccess) rc = RB_ERR_CUDA;
  if (batch->graph && cudaGraphDestroy(batch->graph) != cudaSuccess) rc = RB_ERR_CUDA;
  delete batch;
  return rc;
}

// ---------------------------------------------------------------------------------------
// Sub-banks along iso-tau0 lines and the basis size for a tolerance (Sec. III.B, Table I). Host only.

int rb_bank_tau0(const rb_bank_desc* bank, double f0, double* tau0) {
  if (!bank || !bank->params || !tau0 || bank->n_templates < 1) {
    set_detail("bank, bank->params or tau0 is NULL, or n_templates < 1");
    return RB_ERR_BAD_INPUT;
  }
  if (!(f0 > 0.0) || !std::isfinite(f0)) {
    set_detail("f0 = %g must be finite and > 0", f0);
    return RB_ERR_BAD_INPUT;
  }
  constexpr double kTsun = 4.925490947641267e-6;  // G M_sun / c^3 [s]
  constexpr double kPi = 3.14159265358979323846;
  for (int t = 0; t < bank->n_templates; ++t) {
    const double m1 = bank->params[4 * t], m2 = bank->params[4 * t + 1];
    if (!(m1 > 0.0) || !(m2 > 0.0) || !std::isfinite(m1) || !std::isfinite(m2)) {
      set_detail("template %d: masses (%g, %g) must be finite and > 0", t, m1, m2);
      return RB_ERR_BAD_INPUT;
    }
    const double M = (m1 + m2) * kTsun, eta = m1 * m2 / ((m1 + m2) * (m1 + m2));
    const double v = std::cbrt(kPi * M * f0), v2 = v * v, v4 = v2 * v2;
    tau0[t] = 5.0 * M / (256.0 * eta * v4 * v4);
  }
  return RB_OK;
}

int rb_bank_split_tau0(const double* tau0, int64_t n_templates, int32_t parts, int64_t* order, int64_t* offsets) {
  if (!tau0 || !order || !offsets || n_templates < 1 || parts < 1 || parts > n_templates) {
    set_detail("NULL pointer, n_templates = %lld < 1 or parts = %d not in [1, n_templates]",
               (long long)n_templates, parts);
    return RB_ERR_BAD_INPUT;
  }
  for (int64_t t = 0; t < n_templates; ++t) {
    if (!std::isfinite(tau0[t])) {
      set_detail("tau0[%lld] is not finite", (long long)t);
      return RB_ERR_BAD_INPUT;
    }
    order[t] = t;
  }
  std::stable_sort(order, order + n_templates, [&](int64_t a, int64_t b) { return tau0[a] < tau0[b]; });
  // floor(p T / parts) = p q + floor(p r / parts) with T = q parts + r: no intermediate overflows
  const int64_t q = n_templates / parts, r = n_templates % parts;
  for (int32_t p = 0; p <= parts; ++p) offsets[p] = (int64_t)p * q + ((int64_t)p * r) / parts;
  return RB_OK;
}

int rb_basis_k_for_loss(const double* sv, int32_t k, int64_t n_templates, double tol, int32_t* k_out,
                        double* loss_out) {
  if (!sv || !k_out || !loss_out || k < 1 || n_templates < 1 || !(tol >= 0.0 && tol < 1.0)) {
    set_detail("NULL pointer, k = %d < 1, n_templates = %lld < 1 or tol = %g not in [0, 1)", k,
               (long long)n_templates, tol);
    return RB_ERR_BAD_INPUT;
  }
  const double T = (double)n_templates;
  double kept = 0.0;
  for (int32_t j = 0; j < k; ++j) {
    if (!(sv[j] >= 0.0) || !std::isfinite(sv[j]) || (j > 0 && sv[j] > sv[j - 1])) {
      set_detail("sv[%d] = %g: singular values must be finite, >= 0 and descending", j, sv[j]);
      return RB_ERR_BAD_INPUT;
    }
    kept += sv[j] * sv[j];
  }
  if (kept > T * (1.0 + 1e-6)) {
    set_detail("sum of sv^2 = %.17g exceeds n_templates = %lld: rows are not unit-normalised", kept,
               (long long)n_templates);
    return RB_ERR_BAD_INPUT;
  }
  kept = 0.0;
  for (int32_t j = 0; j < k; ++j) {
    kept += sv[j] * sv[j];
    const double loss = std::max(0.0, 1.0 - kept / T);
    if (loss <= tol) {
      *k_out = j + 1;
      *loss_out = loss;
      return RB_OK;
    }
  }
  *k_out = k;
  *loss_out = std::max(0.0, 1.0 - kept / T);
  set_detail("the %d singular values leave an Eq. 8 loss of %.3g > tol = %.3g", k, *loss_out, tol);
  return RB_ERR_UNSUPPORTED;
}

}  // extern "C"
