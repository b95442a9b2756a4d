// Internal host-side interfaces shared by the translation units of the library.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>

#include "../../include/rbmf.h"

namespace rb {

// Second-stage work item: at most this many bucketed candidates of one bin.
constexpr unsigned kStage2Piece = 512;
constexpr unsigned kStage2MinPiece = 128;  // the smallest work piece any second stage asks for

struct Geometry {
  int64_t n = 0;       // block length
  int n1 = 0, n2 = 0;  // four-step split n = n1 * n2 (outer x inner)
  int64_t n_bins = 0;  // valid bins n / (2 w)
  int kp = 0;          // 2k rounded up to 64 (first-stage contraction length)
  int k16 = 0;         // k rounded up to 16 (second-stage chunking)
  size_t s2_bytes = 0; // second-stage operand planes at the start of coeff_op
};

struct Tables {
  float2* n1_w = nullptr;    // [n1] exp(2 pi i e / n1)
  float2* n2_w = nullptr;    // [n2] exp(2 pi i e / n2)
  float2* fine_w = nullptr;  // [n2] exp(2 pi i e / n)
  float2* w2a_w = nullptr;   // [32][n2/32 + 1]: exp(2 pi i j r / n2), stage-2 twiddles of the radix-32 pass A
  float2* w2b_w = nullptr;   // [32][n1/32 + 1]: exp(2 pi i j r / n1), the same for pass B
  const float2* n1 = nullptr;
  const float2* n2 = nullptr;
  const float2* fine = nullptr;
  const float2* w2a = nullptr;
  const float2* w2b = nullptr;
};
// float2 entries of a stage-2 twiddle table for a column length L
inline int64_t w2_entries(int L) { return 32 * (int64_t)(L / 32 + 1); }

// A bucketed second-stage record: the template row and block id of a run of candidates in one
// group of bins, and the mask of those bins within the group (bit j: bin j of the group); the group
// comes with the work piece.
struct SortedCand {
  int tmpl;
  int block;
  unsigned mask;
};


// Carving of the caller's workspace (all offsets 256-byte aligned).
struct Workspace {
  unsigned* flags = nullptr;                 // RB_FLAG_* bits
  unsigned long long* cand_count = nullptr;  // first-stage candidates found
  unsigned long long* trig_count = nullptr;  // triggers found
  unsigned long long* host_status = nullptr; // (device) copy-out block: flags, counts
  Tables tables;
  float* wt = nullptr;        // [n/2] whitening weights
  float2* shat = nullptr;     // [n/2] whitened data
  rb_trigger* trig_stage = nullptr;  // device staging of the triggers for RB_MEM_HOST_TRIGGERS (at an
                                     // offset and size that depend on n only)
  float2* X = nullptr;        // [vc][n1][n2] four-step intermediate
  int vc = 1;                 // vectors per four-step chunk
  float2* beta = nullptr;     // [k][n/2]
  float2* bavg = nullptr;     // [k][n_bins]
  void* bop_hi = nullptr;     // [n_bins][kp] 16-bit
  void* bop_lo = nullptr;     // [n_bins][kp] 16-bit (split precisions)
  rb_candidate* cand = nullptr;
  SortedCand* cand_sorted = nullptr;    // candidates grouped by bin for the second stage
  unsigned* bin_count = nullptr;        // [n_bins + 1] per-bin counts, then fill cursors
  unsigned* bin_start = nullptr;        // [n_bins + 1] exclusive prefix sums
  int4* pieces = nullptr;               // second-stage work items {bin, first, end, 0}
  unsigned* piece_total = nullptr;      // number of pieces (device)
  size_t total = 0;
};

void set_detail(const char* fmt, ...);
// 2D TMA descriptor over [dim1][dim0] elements (row pitch row_bytes), box box0 x box1, zero fill.
int make_map_2d(CUtensorMap* m, CUtensorMapDataType type, int elem_bytes, const void* base, uint64_t dim0,
                uint64_t dim1, uint64_t row_bytes, uint32_t box0, uint32_t box1, CUtensorMapSwizzle swizzle);
int make_geometry(const rb_filter_desc& d, Geometry* g);
// base == nullptr: only compute the size (ws->total)
void carve(const rb_filter_desc& d, const Geometry& g, char* base, Workspace* ws, bool plain);
size_t coeff_op_bytes(const rb_filter_desc& d, const Geometry& g);

int init_tables(const Geometry& g, const Workspace& ws, const double* psd, double fs, cudaStream_t st);
int whiten(const Geometry& g, const Workspace& ws, const float* strain, float2* shat, cudaStream_t st);
int bank_filter(const Geometry& g, const Workspace& ws, const float2* rows, int64_t nvec, const float2* shat,
                float2* beta, float2* bavg, int w, cudaStream_t st);
int plain_filter(const Geometry& g, const Workspace& ws, const float2* tmpl, int64_t T, const float2* shat,
                 int w, float thr2, int64_t sample_offset, int block_id, rb_trigger* trig, int64_t cap,
                 cudaStream_t st);
// Whether the radix-32 four-step passes run where they apply (host hook rbx_set_fft_radix32).
bool fft_radix32_enabled();
// FFT schedule variants of the basis filter and the template-method comparator (per n and w)
int set_fft_variant(const Geometry& g, int w, int variant);
int tune_fft(const Geometry& g, const Workspace& ws, const float2* rows, int64_t nvec, const float2* shat,
             float2* beta, float2* bavg, int w, double* ms, int* chosen, cudaStream_t st);
// Fast first stage by the template method (Sec. III.D): gfold[j] = G(j) / w on j < n/2, then per template
// the folded spectrum's inverse transform of length gm.n = n / w, candidates where |<z>_b|^2 >= thr2
// (counted at wm.cand_count, at most cap stored).
int init_gfold(float2* gfold, int64_t n, int w, cudaStream_t st);
// lowpass: the first stage of Sec. III.G instead (the product's lowest n / w bins, no fold).
int folded_stage1(const Geometry& gm, const Workspace& wm, const float2* tmpl, int64_t T, const float2* shat, int w,
                  float thr2, int block_id, rb_candidate* cand, int64_t cap, const float2* gfold, cudaStream_t st,
                  bool lowpass = false);
int stage1_simt(const rb_filter_desc& d, const rb_basis& b, const Geometry& g, const Workspace& ws,
                const float2* bavg, rb_candidate* cand, cudaStream_t st);
int pack_beta(const rb_filter_desc& d, const Geometry& g, const float2* bavg, void* hi, void* lo,
              cudaStream_t st);
int pack_coeff(const rb_filter_desc& d, const rb_basis& b, const Geometry& g, void* out, cudaStream_t st);
int stage1_tc(const rb_filter_desc& d, const rb_basis& b, const Geometry& g, const Workspace& ws,
              rb_candidate* cand, cudaStream_t st);
int tune_stage1(const rb_filter_desc& d, const rb_basis& b, const Geometry& g, const Workspace& ws, double* ms,
                int* chosen, cudaStream_t st);
int stage1_tc_variants();
int set_stage1_variant(const rb_filter_desc& d, const Geometry& g, int variant);
// Second stage on ws.cand (count at ws.cand_count): bucketing by bin, then exact reconstruction;
// triggers are appended at *counter. Bins before bin_lo (relative to the first valid bin) are skipped.
int stage2_bucketed(const rb_filter_desc& d, const rb_basis& b, const Geometry& g, const Workspace& ws,
                    const float2* beta, rb_trigger* trig, int64_t cap, unsigned long long* counter, int bin_lo,
                    cudaStream_t st);
// tcgen05 second stage (w <= 8; RB_ERR_UNSUPPORTED when k does not fit) and its selection
int stage2_tc_run(const rb_filter_desc& d, const rb_basis& b, const Geometry& g, const Workspace& ws,
                  const float2* beta, rb_trigger* trig, int64_t cap, unsigned long long* counter, cudaStream_t st,
                  int tmpl_base = 0);
bool stage2_use_tc();
int stage2_tc_mode();  // 0 off, 1 automatic group width, 16 or 32 samples per group
// Samples per bin group of the tcgen05 second stage for desc (16 or 32), 0 when it cannot run it
// (w > 8, or no room for a coefficient ring beside the windows).
int stage2_tc_samples(const rb_filter_desc& d);
// Bins per group for desc: stage2_tc_samples / w for the tcgen05 second stage, 1 for the mma.sync
// one; the bucketing and the reconstruction of one call see the same value.
int stage2_group(const rb_filter_desc& d);
// The two halves of stage2_bucketed: bucketing of ws.cand by bin group, then the reconstruction.
int stage2_bucket(const rb_filter_desc& d, const Geometry& g, const Workspace& ws, int bin_lo, cudaStream_t st);
// tmpl_base is added to every trigger's template row (sub-banks filtered into one list).
int stage2_run(const rb_filter_desc& d, const rb_basis& b, const Geometry& g, const Workspace& ws,
               const float2* beta, rb_trigger* trig, int64_t cap, unsigned long long* counter, cudaStream_t st,
               int tmpl_base = 0);

}  // namespace rb
