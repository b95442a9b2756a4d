/*
 * rbmf.h - C ABI of the GB300 (sm_103a) hierarchical reduced-basis matched filter.
 *
 * Method: arXiv:2110.13115 (Dhurkunde, Fehrmann, Nitz), "A hierarchical approach to
 * matched filtering using a reduced basis".
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - A block holds n samples at fs Hz (n a power of two, 2^10 <= n <= 2^20); df = fs/n.
 *    Frequencies f_j = j df, j in [0, n/2]. Only 0 < j < n/2 enters any sum
 *    (one-sided matched filter of Eq. (1); DC and Nyquist excluded).
 *  - Blocks overlap by n/2 (Sec. III.F): only block samples m in [n/2, n) are valid and
 *    reported. Trigger sample indices are sample_offset + m.
 *  - Whitened coordinates: x_hat[j] = sqrt(4 df / S_j) x(f_j), with x(f) = dt * DFT(x).
 *    In them the inner product <a|b> of Eq. (1) is sum_j a_hat[j] conj(b_hat[j]).
 *  - Complex arrays are interleaved float pairs (re, im), C order as stated per argument.
 *  - Pointers are DEVICE pointers unless the argument says "host", or unless rb_filter_desc.mem
 *    tags them as host pointers (rb_filter and rb_filter_static only, see RB_MEM_*). All buffers are owned
 *    by the caller; the library allocates no device memory (beyond the CUDA graph objects that
 *    rb_batch_create records): every call that needs scratch space takes a caller-provided
 *    workspace of at least the size rb_filter_plan reports (256-byte aligned).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Calls that return counts
 *    (n_out) synchronise that stream before returning; the others only enqueue work.
 *  - Every function returns RB_OK (0) or a negative RB_ERR_* code; nothing throws.
 *    rb_strerror() names a code, rb_last_error_detail() describes the last failure on the
 *    calling thread (a CUDA error string, which argument was rejected).
 */
#ifndef RBMF_H
#define RBMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  RB_OK = 0,
  RB_ERR_BAD_INPUT = -1,   /* a descriptor field, size or pointer is invalid */
  RB_ERR_OOM = -2,         /* the workspace passed is smaller than rb_filter_plan's size */
  RB_ERR_OVERFLOW = -3,    /* an output or candidate list was too small; *n_out = required */
  RB_ERR_TIMEOUT = -4,     /* a device-side bounded wait gave up */
  RB_ERR_CUDA = -5,        /* a CUDA runtime call or launch failed */
  RB_ERR_UNSUPPORTED = -6  /* valid request the build does not support (size, precision) */
};

/* Stage-1 reconstruction arithmetic (Sec. III.C first stage; precision study). */
enum {
  RB_PREC_FP32 = 0,        /* FP32 SIMT complex GEMM */
  RB_PREC_FP16_SPLIT = 1,  /* tcgen05 FP16 operands split hi+lo, 3 MMAs, FP32 accumulate */
  RB_PREC_BF16_SPLIT = 2,  /* tcgen05 BF16 operands split hi+lo, 3 MMAs, FP32 accumulate */
  RB_PREC_FP16 = 3,        /* tcgen05 single FP16 operands, FP32 accumulate */
  RB_PREC_BF16 = 4,        /* tcgen05 single BF16 operands, FP32 accumulate */
  RB_PREC_FP16_SPLIT_A = 5 /* tcgen05 FP16, coefficients split hi+lo, beta_avg single: 2 MMAs */
};

/* Where rb_filter's strain and trigger buffers live (rb_filter_desc.mem bits; 0 = both on the
 * device). With a host bit set, rb_filter copies through device staging inside its workspace on the
 * caller's stream: the strain in before the whitening FFT, the triggers out after the second stage
 * (the call already synchronises the stream to return the count). Host buffers may be pageable;
 * pinned ones let the copies run at full link speed. */
enum {
  RB_MEM_HOST_STRAIN = 1,   /* strain is a host pointer ([n] float32) */
  RB_MEM_HOST_TRIGGERS = 2  /* trig is a host pointer; capacity <= rb_filter_sizes.host_trig_capacity */
};

/* One block's filtering parameters. */
typedef struct rb_filter_desc {
  double fs;              /* sample rate [Hz] */
  int64_t n;              /* block length: power of two, 2^10..2^20 */
  int32_t k;              /* basis vectors used (rows of rb_basis.vectors) */
  int32_t n_templates;    /* T: rows of rb_basis.coeff */
  int32_t w;              /* bin width in samples (Eq. 9): 1, 2, 4, 8 or 16 */
  int32_t precision;      /* RB_PREC_* for the first stage */
  float rho_i;            /* first-stage threshold on the bin-averaged SNR (Sec. III.C) */
  float rho_ii;           /* second-stage threshold on the full-rate SNR (Sec. III.C) */
  int64_t cand_capacity;  /* first-stage candidate slots kept in the workspace, < 2^31 */
  int64_t sample_offset;  /* global index of block sample 0 */
  int32_t block_id;       /* copied into rb_trigger.block / rb_candidate.block */
  int32_t mem;            /* RB_MEM_* bits (rb_filter, rb_filter_static); 0 for every other call */
} rb_filter_desc;

/* The reduced basis of a template bank (output of rb_build; caller-owned arrays). */
typedef struct rb_basis {
  int32_t k;              /* basis vectors stored */
  int32_t n_templates;    /* T */
  int64_t n;              /* block length the basis was built for */
  const float* vectors;   /* [k][n/2] complex: p_k in whitened coordinates, orthonormal */
  const float* coeff;     /* [T][k] complex: a_tk = <g_t|p_k> / sigma_t (SNR units, Eq. 7) */
  const void* coeff_op;   /* packed stage operands from rb_pack_coeff (needed by rb_filter, rb_stage2) */
  int32_t coeff_op_precision; /* RB_PREC_* coeff_op was packed for */
  int32_t reserved;
} rb_basis;

/* A final trigger (Sec. III.C second stage; also the template method's triggers). */
typedef struct rb_trigger {
  int64_t sample;   /* sample_offset + block sample m of the window's arg-max */
  int32_t tmpl;     /* template row */
  int32_t block;    /* rb_filter_desc.block_id */
  float snr;        /* rho = |z| / sigma */
  float phase;      /* arg z in (-pi, pi] */
} rb_trigger;       /* 24 bytes */

/* A first-stage candidate: a (template, bin) whose bin-averaged SNR reached rho_I. */
typedef struct rb_candidate {
  int32_t tmpl;     /* template row */
  int32_t bin;      /* bin index i of Eq. (9): samples [i w, i w + w) of the block */
  float snr_avg;    /* |sum_k a_tk^* beta^avg_k[i]| */
  int32_t block;    /* rb_filter_desc.block_id */
} rb_candidate;     /* 16 bytes */

/* Sizes derived from a descriptor (host-only, no CUDA call). */
typedef struct rb_filter_sizes {
  size_t workspace_bytes;   /* minimum workspace for rb_filter / rb_filter_plain / stage calls */
  int64_t n_bins;           /* valid bins n/(2w) */
  int32_t n1, n2;           /* four-step split n = n1 * n2 */
  int32_t kp;               /* stage-1 contraction length 2k rounded up to 64 */
  size_t coeff_op_bytes;    /* bytes rb_pack_coeff writes for desc->precision */
  int64_t host_trig_capacity; /* largest rb_filter capacity with RB_MEM_HOST_TRIGGERS: the triggers are
                                 staged in a region of max(96 MB, 8 n bytes) that the workspace holds
                                 (workspace_bytes includes it) when desc->mem has that bit */
} rb_filter_sizes;

/* Name of a status code (static string). */
const char* rb_strerror(int status);
/* Details of the last failure on the calling thread (static per-thread buffer). */
const char* rb_last_error_detail(void);
/* Library version: major*10000 + minor*100 + patch. */
int rb_version(void);

/*
 * rb_filter_plan - validate `desc` and report workspace size and layout parameters.
 * Host only. Errors: RB_ERR_BAD_INPUT (n not a power of two in range, k < 1, T < 1,
 * w not in {1,2,4,8,16}, w > n/2, thresholds negative or NaN, mem with bits other than RB_MEM_*),
 * RB_ERR_UNSUPPORTED (precision unknown).
 */
int rb_filter_plan(const rb_filter_desc* desc, rb_filter_sizes* out /* host */);

/*
 * rb_whiten - step a1: s_hat[j] = sqrt(4 df / S_j) * dt * DFT(strain)[j] for j in [0, n/2)
 * (s_hat[0] = 0), by a forward Stockham FFT with the whitening fused into its last pass.
 * Paper: Sec. III.C (first bullet; data FFT) and Sec. III.E (whitening by S_n^{-1/2}).
 *   strain: [n] float32 time samples.       psd: [n/2 + 1] float64 one-sided PSD S_j
 *   (S_0 may be +inf; S_j for 0 < j < n/2 must be finite and > 0, else RB_ERR_BAD_INPUT,
 *   detected on the device and reported after the stream synchronises).
 *   s_hat: [n/2] complex output.            workspace: rb_filter_plan size.
 */
int rb_whiten(const rb_filter_desc* desc, const float* strain, const double* psd, float* s_hat,
              void* workspace, size_t workspace_bytes, void* stream);

/*
 * rb_basis_filter - steps a2 + a3: basis SNR series and their bin averages.
 *   beta_k[m] = sum_{j<n/2} s_hat[j] conj(p_k[j]) exp(+2 pi i j m / n)  (Eq. 6-7,
 *   Sec. III.C third bullet), stored for the valid half m in [n/2, n) only;
 *   beta_avg_k[i] = (1/w) sum_{r<w} beta_k[i w + r] for valid bins i in [n/(2w), n/w) (Eq. 9).
 * The multiply by conj(p_k) is fused into the first pass of a four-step inverse Stockham FFT;
 * the averaging is fused into its last pass.
 *   s_hat: [n/2] complex (rb_whiten output).  basis->vectors: [k][n/2] complex.
 *   beta: [k][n/2] complex output (index m - n/2), may be NULL to skip storing it.
 *   beta_avg: [k][n/(2w)] complex output (index i - n/(2w)).
 *   Errors: RB_ERR_BAD_INPUT (desc invalid, basis not matching desc, NULL s_hat or beta_avg),
 *   RB_ERR_OOM (workspace smaller than rb_filter_plan's size or not 256-byte aligned).
 */
int rb_basis_filter(const rb_filter_desc* desc, const rb_basis* basis, const float* s_hat,
                    float* beta, float* beta_avg, void* workspace, size_t workspace_bytes,
                    void* stream);

/*
 * rb_pack_coeff - lay out the coefficient operands of both stages from basis->coeff (the
 * a_tk of Eq. 7). Required before rb_filter, rb_stage1 (16-bit precisions) and rb_stage2.
 *   Second-stage part (every precision; first s2 bytes of out): an FP16 hi plane then an FP16
 *   lo plane (lo = fp16(x - hi)), each [T][2 k16] with row t = [Re a_t (k16) | Im a_t (k16)],
 *   k16 = k rounded up to 16, zero padded; hi + lo carries FP32-level accuracy.
 *   First-stage part (16-bit precisions only; after the second-stage part): rows 2t and 2t+1
 *   hold [Re a_t, Im a_t] and [-Im a_t, Re a_t] (k values each, zero padded to kp), so that
 *   one real GEMM row pair gives Re and Im of sum_k a_tk^* beta_k; split precisions store a
 *   hi plane then a lo plane (lo = round(x - hi)).
 *   out: plan.coeff_op_bytes device bytes, 256-byte aligned, owned by the caller and stored
 *   as basis->coeff_op with basis->coeff_op_precision = desc->precision. Enqueue only.
 *   Errors: RB_ERR_BAD_INPUT for a null pointer or a basis that does not match desc.
 */
int rb_pack_coeff(const rb_filter_desc* desc, const rb_basis* basis, void* out, void* stream);

/*
 * rb_stage1 - step a4: first-stage reconstruction z_avg[t,i] = sum_k conj(a_tk) beta_avg_k[i]
 * (Eq. 7 applied to Eq. 9) as one contraction over K = 2k, with |z_avg| >= rho_I tested in the
 * epilogue so the T x bins array never reaches memory (Sec. III.C first stage; Sec. III.E).
 * RB_PREC_FP32 runs an FP32 SIMT kernel; the 16-bit precisions run a tcgen05 kernel whose
 * operands TMA loads into shared memory and whose accumulators live in tensor memory (one, two
 * or three products per K step by precision; every device wait is bounded, RB_ERR_TIMEOUT).
 *   beta_avg: [k][n/(2w)] complex (rb_basis_filter output).
 *   cand: [desc->cand_capacity] output; n_cand (host): number found. Synchronises `stream`.
 *   Errors: RB_ERR_OVERFLOW when more than cand_capacity candidates exist (*n_cand = count,
 *   the first cand_capacity found are stored), RB_ERR_BAD_INPUT when coeff_op is missing
 *   or was packed for another precision.
 */
int rb_stage1(const rb_filter_desc* desc, const rb_basis* basis, const float* beta_avg,
              rb_candidate* cand, int64_t* n_cand, void* workspace, size_t workspace_bytes,
              void* stream);

/*
 * rb_stage2 - step a5: for each candidate (t, i), z_t[m] = sum_k conj(a_tk) beta_k[m] to FP32
 * accuracy for m in [i w, i w + w); emit the arg-max (ties to the smaller m) when |z| >= rho_II
 * (Sec. III.C second stage, Sec. III.E custom kernel). Candidates are bucketed by bin (any
 * input order); for each bin the k x w window of beta is staged once in shared memory as FP16
 * hi + lo tensor-core fragments and a warp reconstructs 16 candidates at a time with mma.sync
 * (three products hi.hi + hi.lo + lo.hi, FP32 accumulation), reading the coefficients that
 * rb_pack_coeff laid out (required: basis->coeff_op).
 *   beta: [k][n/2] complex (valid half, rb_basis_filter output).  cand: [n_cand] device.
 *   trig: [capacity] output; n_trig (host). Synchronises `stream`.
 *   Errors: RB_ERR_OVERFLOW as for rb_stage1; RB_ERR_BAD_INPUT without coeff_op or with n_cand
 *   above desc->cand_capacity; RB_ERR_TIMEOUT when a bounded device wait of the (opt-in) tcgen05
 *   second stage gave up.
 */
int rb_stage2(const rb_filter_desc* desc, const rb_basis* basis, const float* beta,
              const rb_candidate* cand, int64_t n_cand, rb_trigger* trig, int64_t capacity,
              int64_t* n_trig, void* workspace, size_t workspace_bytes, void* stream);

/*
 * rb_filter - the whole hierarchical filter of one block: a1 (rb_whiten), a2+a3
 * (rb_basis_filter), a4 (rb_stage1), a5 (rb_stage2), all on `stream`, beta kept in the
 * workspace. Paper: Sec. III.C (the six bullets) and Sec. III.E.
 *   strain: [n] float32 (host when desc->mem has RB_MEM_HOST_STRAIN). psd: [n/2+1] float64.
 *   trig: [capacity] (host when desc->mem has RB_MEM_HOST_TRIGGERS); n_trig (host).
 *   With host buffers the copies run on `stream` inside the call, so one call takes strain in
 *   host memory to triggers in host memory.
 *   Errors: as the stage calls; RB_ERR_OVERFLOW from either stage sets *n_trig to the
 *   required trigger count when known, else to -1 (candidate list overflowed); RB_ERR_BAD_INPUT
 *   when capacity exceeds host_trig_capacity with RB_MEM_HOST_TRIGGERS.
 */
int rb_filter(const rb_filter_desc* desc, const rb_basis* basis, const float* strain,
              const double* psd, rb_trigger* trig, int64_t capacity, int64_t* n_trig,
              void* workspace, size_t workspace_bytes, void* stream);

/*
 * rb_banks_plan - workspace for rb_filter_banks: the largest rb_filter_plan workspace over the sub-bank
 * descriptors (they share one workspace in turn). n_bins, n1 and n2 as rb_filter_plan (equal for all),
 * kp the largest, coeff_op_bytes 0 (pack each sub-bank with rb_pack_coeff and its own desc),
 * host_trig_capacity the smallest. Host only.
 * Errors: as rb_filter_plan for any desc; RB_ERR_BAD_INPUT when n_banks < 1 or a desc differs from
 * descs[0] in n, fs, w or mem.
 */
int rb_banks_plan(const rb_filter_desc* descs, int32_t n_banks, rb_filter_sizes* out /* host */);

/*
 * rb_filter_banks - one block through the hierarchical filter of a bank cut into sub-banks, each with
 * its own reduced basis: the paper splits its bank along lines of equal chirp time tau0 and gives
 * every part the basis size that its tolerance needs (Sec. III.B, Table I). The strain is whitened
 * once (a1); then for every sub-bank b in order the basis filter (a2 + a3), the first stage (a4) and
 * the second stage (a5) run with descs[b] and bases[b], all appending to one trigger list on `stream`.
 * A trigger's tmpl is its row in the concatenation of the sub-banks' coefficient matrices:
 * sum_{b' < b} descs[b'].n_templates + the row in bases[b].
 *   descs: [n_banks] HOST; same fs, n, w and mem (k, T, precision, rho_i, rho_ii, cand_capacity may
 *     differ); sample_offset and block_id are taken from descs[0]; mem tags strain / trig as host
 *     buffers as for rb_filter.
 *   bases: [n_banks] HOST array; bases[b] matches descs[b] and is packed by rb_pack_coeff for it.
 *   strain, psd, trig, capacity, n_trig: as rb_filter.   workspace: rb_banks_plan size.
 *   With RB_MEM_HOST_TRIGGERS each sub-bank's triggers are copied out on a library-owned side stream
 *   (one per device, kept for the life of the process) while the next sub-bank runs on `stream`; the
 *   call returns when every copy has landed.
 *   Errors: as rb_filter; a sub-bank's candidate overflow sets *n_trig = -1 (RB_ERR_OVERFLOW).
 */
int rb_filter_banks(const rb_filter_desc* descs, const rb_basis* bases, int32_t n_banks, const float* strain,
                    const double* psd, rb_trigger* trig, int64_t capacity, int64_t* n_trig, void* workspace,
                    size_t workspace_bytes, void* stream);

/*
 * rb_stage1_folded - the first stage by the template method instead of the basis (Sec. III.D,
 * Eqs. 10-12): the bin average of a template's SNR series is one inverse DFT of length M = n / w of
 * the folded spectrum
 *   Omega(f') = (1/w) sum_l Q[l M + f'] G(l M + f'),   G(f) = sum_{r<w} exp(2 pi i f r / n),
 * Q[j] = s_hat[j] conj(g_t[j]) on 0 < j < n/2 (zero above, so only l < w/2 contributes), and
 *   <z>_b = sum_{f' < M} Omega(f') exp(2 pi i f' b / M),   b in [M/2, M) (the valid bins of Eq. 9).
 * G is evaluated in closed form, (1 - e^(2 pi i f w / n)) / (1 - e^(2 pi i f / n)) with G(0) = w, in FP64.
 * Candidates (t, b) with |<z>_b| >= rho_I are written as by rb_stage1 (bin = b), in no set order. The
 * strain is whitened inside the call (as rb_filter_plain).
 *   templates: [T][n/2] complex whitened unit-norm templates (g_t / sigma_t, as rb_templates).
 *   strain: [n] float32.  psd: [n/2 + 1] float64.  desc: fs, n, w (2..16), n_templates, rho_i,
 *   cand_capacity, block_id used (k, precision, rho_ii ignored; mem must be 0).
 *   cand: [cand_capacity] output; n_cand (host). workspace: rb_folded_plan size. Synchronises `stream`.
 *   Errors: RB_ERR_BAD_INPUT (w < 2, NULL array, PSD), RB_ERR_UNSUPPORTED (n / w < 1024),
 *   RB_ERR_OOM (workspace), RB_ERR_OVERFLOW (more candidates than cand_capacity; *n_cand = count).
 */
int rb_folded_plan(const rb_filter_desc* desc, size_t* workspace_bytes /* host */);
int rb_stage1_folded(const rb_filter_desc* desc, const float* templates, const float* strain, const double* psd,
                     rb_candidate* cand, int64_t* n_cand, void* workspace, size_t workspace_bytes, void* stream);

/*
 * rb_stage1_lowpass - the low-pass alternative to the first stage that the paper compares with
 * (Sec. III.G): each template's SNR series low-passed to the lowest M = n / w frequency bins of its
 * one-sided spectrum and decimated by w,
 *   z_lp[b] = sum_{j < M} s_hat[j] conj(g_t[j]) exp(2 pi i j b / M),   b in [M/2, M),
 * one inverse DFT of length M per template, candidates where |z_lp[b]| >= rho_I (bin = b, as
 * rb_stage1_folded). Same arguments, workspace (rb_folded_plan) and errors as rb_stage1_folded.
 */
int rb_stage1_lowpass(const rb_filter_desc* desc, const float* templates, const float* strain, const double* psd,
                      rb_candidate* cand, int64_t* n_cand, void* workspace, size_t workspace_bytes, void* stream);

/*
 * rb_filter_plain - the template method (Sec. II, Eq. 4; the baseline of Sec. IV.B.2):
 * per template one inverse FFT of s_hat * conj(h_hat_t), rho = |z| (templates given
 * unit-normalised), per window of w valid samples the arg-max kept when rho >= rho_II.
 * The multiply is fused into the FFT's first pass and the window maximum into its last,
 * so no SNR series reaches memory.
 *   templates: [T][n/2] complex whitened unit-norm templates (g_t / sigma_t).
 *   strain, psd, trig, capacity, n_trig: as rb_filter (desc->k, w, rho_ii used; rho_i ignored).
 *   Errors: RB_ERR_BAD_INPUT (NULL array, negative capacity, PSD not finite and > 0 on 0 < j < n/2),
 *   RB_ERR_OOM (workspace), RB_ERR_OVERFLOW (more triggers than capacity; *n_trig = the count).
 */
int rb_filter_plain(const rb_filter_desc* desc, const float* templates, const float* strain,
                    const double* psd, rb_trigger* trig, int64_t capacity, int64_t* n_trig,
                    void* workspace, size_t workspace_bytes, void* stream);

/*
 * rb_filter_static - rb_filter without any device allocation, for callers that cannot allocate
 * device memory: code running inside a host application that owns the whole GPU memory pool,
 * latency-critical loops where an allocation may block or fail under memory pressure, and
 * plugins whose host forbids allocation calls. (The paper has no counterpart; this is a
 * deployment convenience.)
 *
 * Same arguments, results and errors as rb_filter minus the workspace: the scratch lives in a
 * static device array of RB_STATIC_SCRATCH_BYTES (32 MiB) inside the library, which every GPU that
 * loads the library keeps until the process exits. Problems whose rb_filter_plan workspace exceeds
 * that size are rejected with RB_ERR_UNSUPPORTED (e.g. n = 16384, k = 64, T = 64 fits; the
 * 2^19-sample, k = 256 workload does not). The call itself allocates nothing (no cudaMalloc, no
 * allocating library routine).
 *   - The first call in each CUDA context of a device looks up the array's device address, with
 *     that device current, and keeps it for that context; make that first call before any stream
 *     capture. After cudaDeviceReset the device has a new context, where the module may load at
 *     another address, so the next call is a first call again.
 *   - All calls share the one array and it keeps the last call's contents (every value a call
 *     reads is written or cleared by that call first). Calls that overlap on the GPU - from two
 *     streams or two host threads at once - race on it: serialise them.
 */
#define RB_STATIC_SCRATCH_BYTES (32u << 20)
int rb_filter_static(const rb_filter_desc* desc, const rb_basis* basis, const float* strain, const double* psd,
                     rb_trigger* trig, int64_t capacity, int64_t* n_trig, void* stream);

/*
 * Batching: many blocks - from segments of uneven length, several detectors and several FFT sizes -
 * filtered in one call, each block through the whole rb_filter pipeline (Sec. III.E: the data of
 * many segments is processed per launch so that the device never idles between them). Banks that
 * share a basis are filtered together by concatenating their coefficient rows (the M dimension of
 * the first-stage GEMM), so each block's basis series beta is computed once for all of them.
 *
 * rb_block - one filtering block:
 *   strain: device [n] float32 samples of the block; psd: device [n/2 + 1] float64 one-sided PSD of
 *   its detector (a per-detector scale factor is a scaled PSD).
 *   basis: index into the descs / bases arrays (one entry per FFT size n; entry i's desc describes
 *   bases[i]); its desc's sample_offset and block_id are replaced by the block's own.
 *   valid_lo: first block sample whose triggers are kept, n/2 <= valid_lo < n, a multiple of w:
 *   n/2 for an ordinary block, more for a right-aligned tail block whose leading valid samples the
 *   previous block already covered (no trigger is reported twice).
 */
typedef struct rb_block {
  const float* strain;
  const double* psd;
  int64_t sample_offset;
  int64_t valid_lo;
  int32_t basis;
  int32_t block_id;
} rb_block;

/* rb_batch_plan - workspace bytes for batches over descs[0..n_descs): the largest rb_filter_plan
 * workspace (blocks run one after another through one workspace). Errors as rb_filter_plan. */
int rb_batch_plan(const rb_filter_desc* descs, int32_t n_descs, size_t* workspace_bytes);

/*
 * rb_filter_batch - filter blocks[0..n_blocks) in order, appending every block's triggers to trig
 * (one counter; trigger order across blocks is unspecified) and synchronising once at the end.
 *   descs, bases: n_bases pairs, each bases[i] packed (rb_pack_coeff) for descs[i].
 *   trig: [capacity] device output; n_trig (host): triggers found.
 *   Errors: RB_ERR_BAD_INPUT (a block's basis index, pointers, valid_lo; a basis that does not match
 *   its desc; a PSD that is not finite and positive), RB_ERR_OOM (workspace), RB_ERR_OVERFLOW (some
 *   block had more than its desc's cand_capacity candidates, or more than capacity triggers in all;
 *   *n_trig is the count found), RB_ERR_TIMEOUT, RB_ERR_CUDA.
 */
int rb_filter_batch(const rb_filter_desc* descs, const rb_basis* bases, int32_t n_bases, const rb_block* blocks,
                    int64_t n_blocks, rb_trigger* trig, int64_t capacity, int64_t* n_trig, void* workspace,
                    size_t workspace_bytes, void* stream);

/*
 * rb_batch_create / rb_batch_run / rb_batch_destroy - the same batch recorded once as a CUDA graph
 * and replayed with a single graph launch per run. create validates the arguments as
 * rb_filter_batch does, copies descs, bases and blocks, and records every kernel, memset and
 * copy of the batch on a private stream; the device buffers (strain, psd, coefficients, basis,
 * trig, workspace) are referenced, not copied: keep them alive and at the same addresses until
 * destroy, and refill them between runs to filter new data. Record the batch after the first-stage
 * tile choice (rb_tune_stage1 / rb_set_stage1_variant) it should use.
 *   run: launches the graph on `stream`, then reads the status (synchronises `stream`); results and
 *   errors as rb_filter_batch. Runs on one batch must not overlap.
 *   out (create): a new handle, owned by the caller; destroy frees it (NULL is a no-op).
 */
typedef struct rb_batch rb_batch;
int rb_batch_create(const rb_filter_desc* descs, const rb_basis* bases, int32_t n_bases, const rb_block* blocks,
                    int64_t n_blocks, rb_trigger* trig, int64_t capacity, void* workspace, size_t workspace_bytes,
                    rb_batch** out);
int rb_batch_run(rb_batch* batch, int64_t* n_trig, void* stream);
int rb_batch_destroy(rb_batch* batch);

/*
 * rb_tune_stage1 - autotuner of the tensor-core first stage: packs beta_avg (as rb_stage1 does), times
 * each tile variant of the tcgen05 kernel (N-tile width 256 or 128 columns with the deepest operand
 * ring that fits in shared memory) with the threshold disabled, and remembers the fastest for this
 * (precision, T, n_bins, kp) in a process-wide table that rb_stage1 / rb_filter consult (variant 0
 * when untuned). Measurement support, not in the paper.
 *   beta_avg: [k][n/(2w)] complex device.  times_ms: HOST [RB_STAGE1_VARIANTS] mean ms per launch.
 *   chosen: HOST, the selected variant. Synchronises `stream`.
 *   Errors: RB_ERR_BAD_INPUT (NULL argument, basis not matching desc, an FP32 desc or a coeff_op not
 *   packed for desc's precision), RB_ERR_OOM (workspace), RB_ERR_TIMEOUT (a variant's bounded wait).
 */
#define RB_STAGE1_VARIANTS 2
/* rb_set_stage1_variant - pin the tile variant (0: N-tile 256, 1: N-tile 128) used for desc's shape
 * and precision, overriding the tuner's choice. Host only. Errors: RB_ERR_BAD_INPUT. */
int rb_set_stage1_variant(const rb_filter_desc* desc, int32_t variant);
int rb_tune_stage1(const rb_filter_desc* desc, const rb_basis* basis, const float* beta_avg, double* times_ms,
                   int32_t* chosen, void* workspace, size_t workspace_bytes, void* stream);

/*
 * rb_tune_fft - autotuner of the FFT schedule of the basis filter (rb_basis_filter, and inside
 * rb_filter / rb_filter_batch / rb_filter_plain): times every variant of RB_FFT_VARIANTS (columns
 * per CTA of the two four-step passes, and the size of the chunk of vectors whose intermediate stays
 * in L2) on this desc's basis and s_hat, and remembers the fastest for (n, w) in a process-wide
 * table (variant 0 when untuned). Measurement support, not in the paper.
 *   s_hat: [n/2] complex device (rb_whiten output). times_ms: HOST [RB_FFT_VARIANTS] mean ms of one
 *   basis filter. chosen: HOST, the selected variant. Synchronises `stream`.
 *   Errors: RB_ERR_BAD_INPUT (NULL argument, basis not matching desc), RB_ERR_OOM (workspace).
 */
#define RB_FFT_VARIANTS 8
int rb_tune_fft(const rb_filter_desc* desc, const rb_basis* basis, const float* s_hat, double* times_ms,
                int32_t* chosen, void* workspace, size_t workspace_bytes, void* stream);
/* rb_set_fft_variant - pin the FFT schedule variant used for desc's (n, w). Host only. */
int rb_set_fft_variant(const rb_filter_desc* desc, int32_t variant);

/* Stages of rb_filter timed by the profiler (CUDA events recorded on the call's stream). */
enum {
  RB_STAGE_SETUP = 0,   /* status reset, twiddle tables, whitening weights */
  RB_STAGE_WHITEN = 1,  /* a1 */
  RB_STAGE_BASIS = 2,   /* a2 + a3 */
  RB_STAGE_PACK = 3,    /* first-stage operand packing (16-bit precisions) */
  RB_STAGE_FIRST = 4,   /* a4 contraction with fused threshold */
  RB_STAGE_BUCKET = 5,  /* a5 candidates bucketed by bin */
  RB_STAGE_SECOND = 6,  /* a5 reconstruction of the candidates */
  RB_STAGES = 7
};

/*
 * rb_profile_start / rb_profile_stop - per-stage timing of rb_filter (measurement support; the
 * paper reports in-situ wall time, Sec. IV.B.2). Between start and stop, every rb_filter call on
 * the calling thread records a CUDA event at each stage boundary on its stream. stop synchronises
 * those events and writes the mean milliseconds per stage into stage_ms[RB_STAGES] (host) and the
 * number of profiled calls into *calls (host). Errors: RB_ERR_BAD_INPUT (stop without start).
 */
int rb_profile_start(void);
int rb_profile_stop(double* stage_ms, int64_t* calls);

/* Number of kernels this library has launched in this process (all entry points). */
uint64_t rb_kernel_launches(void);

/* A bank of closed-form stationary-phase chirps h(f) = f^(-7/6) exp(-i Psi(f)) (the
 * synthetic stand-in for the paper's IMRPhenomPv2 bank, Sec. III.B), with
 * Psi = -pi/4 + 3/(128 eta v^5) [1 + (20/9)(743/336 + 11 eta/4) v^2 + (4 beta - 16 pi) v^3],
 * v = (pi M f)^(1/3), supported on f_low <= f < 1/(6^(3/2) pi M), 0 < j < n/2. */
typedef struct rb_bank_desc {
  double fs;              /* sample rate [Hz] */
  int64_t n;              /* block length (as rb_filter_desc.n) */
  double f_low;           /* lower cutoff [Hz] */
  int32_t n_templates;    /* T */
  int32_t pn_order;       /* 0: Newtonian; 2: through 1PN; 3: adds the 1.5PN tail and spin-orbit */
  const double* params;   /* HOST [T][4]: m1, m2 [solar masses], chi1, chi2 (aligned spins) */
} rb_bank_desc;

/*
 * rb_build_plan - workspace sizes for rb_templates and rb_build (host only).
 *   oversample: extra sketch columns beyond k (randomised range finder); l = min(k + oversample, T).
 * Errors: RB_ERR_BAD_INPUT (sizes, n, pn_order, k > T).
 */
int rb_build_plan(const rb_bank_desc* bank, int32_t k, int32_t oversample, size_t* templates_bytes /* host */,
                  size_t* build_bytes /* host */);

/*
 * rb_templates - whitened, unit-normalised templates g_t / sigma_t on j in [0, n/2) (the rows of the
 * template matrix of Sec. III.B, each whitened by the PSD and scaled to norm one), with
 * g_t[j] = sqrt(4 df / S_j) h_t(f_j) and sigma_t^2 = sum_j |g_t[j]|^2 = <h_t|h_t> (Eq. 2) in FP64.
 * The phase is evaluated in FP64, reduced modulo 2 pi, then sin/cos in FP32.
 *   psd: [n/2+1] float64 device.  out: [T][n/2] complex device.  sigma2: [T] float64 device.
 *   workspace: templates_bytes of rb_build_plan. Enqueue only.
 *   Errors: RB_ERR_BAD_INPUT (NULL array, bank sizes or pn_order), RB_ERR_OOM (workspace smaller than
 *   templates_bytes).
 */
int rb_templates(const rb_bank_desc* bank, const double* psd, float* out, double* sigma2, void* workspace,
                 size_t workspace_bytes, void* stream);

/*
 * rb_build - step a0: the reduced basis of a bank (Sec. III.A-B; Eq. 5b; Eq. 7 coefficients).
 * The unit-normalised whitened template matrix G (T x n/2, rows from rb_templates) is decomposed
 * by a randomised subspace iteration: Y = G^H Omega (Omega T x l seeded complex normal), then
 * `power_iters` rounds of Y <- G^H (G Q^H) with Q the orthonormalised Y; orthonormalisation is
 * CholeskyQR2 with FP64 Gram matrices; a Rayleigh-Ritz step (FP64 eigen-decomposition of the
 * l x l matrix B^H B, B = G Q^H, on the host) gives the singular values and the basis
 * p_k = sum_i conj(V[i][k]) q_i. Sketch products run in FP32 with FP64 accumulation across
 * K-slices. Outputs (all caller-owned):
 *   vectors: [k][n/2] complex device, orthonormal rows (the basis P of Eq. 5b).
 *   coeff:   [T][k] complex device, a_tk = <g_t/sigma_t | p_k> (normalised coefficients).
 *   sigma2:  [T] float64 device (exact FP64 template norms).
 *   sv:      [k] float64 HOST, leading singular values of G, descending.
 * Synchronises `stream`. Errors: RB_ERR_BAD_INPUT (k < 1, k > T, bad PSD), RB_ERR_OOM
 * (workspace smaller than build_bytes), RB_ERR_UNSUPPORTED (l > 1024).
 */
int rb_build(const rb_bank_desc* bank, const double* psd, int32_t k, int32_t oversample, int32_t power_iters,
             uint64_t seed, float* vectors, float* coeff, double* sigma2, double* sv, void* workspace,
             size_t workspace_bytes, void* stream);

/*
 * Sub-banks along iso-tau0 lines and the basis size for a tolerance (Sec. III.B, Table I): a large
 * bank is cut into parts of equal template count in the order of the Newtonian chirp time, each
 * part gets its own basis (rb_build), and each basis keeps the fewest vectors whose Eq. 8 loss meets
 * the tolerance. Host only: no device memory, no stream.
 *
 * rb_bank_tau0 - tau0[t] = 5 M / (256 eta v^8) with v = (pi M f0)^(1/3), M = m1 + m2 in seconds
 *   (G M_sun / c^3 = 4.925490947641267e-6 s) and eta = m1 m2 / M^2: the Newtonian chirp time from
 *   frequency f0 to coalescence, tau0 ~ Mc^(-5/3) f0^(-8/3) (Sec. III.B).
 *   bank: its params (HOST [T][4]) and n_templates are read.  tau0: [T] float64 HOST output.
 *   Errors: RB_ERR_BAD_INPUT (NULL pointer, T < 1, f0 not finite and > 0, a mass not > 0).
 */
int rb_bank_tau0(const rb_bank_desc* bank, double f0, double* tau0);

/*
 * rb_bank_split_tau0 - order[] lists the T templates by ascending tau0 (equal values keep their
 *   index order); part p holds order[offsets[p] .. offsets[p+1]) with offsets[p] = floor(p T / parts),
 *   so part sizes differ by at most one and every tau0 of part p is <= every tau0 of part p+1.
 *   tau0: [T] HOST.  order: [T] int64 HOST output.  offsets: [parts + 1] int64 HOST output.
 *   Errors: RB_ERR_BAD_INPUT (NULL pointer, T < 1, parts < 1 or > T, a tau0 not finite).
 */
int rb_bank_split_tau0(const double* tau0, int64_t n_templates, int32_t parts, int64_t* order, int64_t* offsets);

/*
 * rb_basis_k_for_loss - the fewest basis vectors whose Eq. 8 loss meets `tol`: with rows of unit
 *   norm the squared singular values of all T rows sum to T, so keeping k' vectors loses
 *   L(k') = 1 - sum_{j<k'} sv[j]^2 / T, the bank-averaged SNR loss. *k_out = the smallest k' in
 *   [1, k] with L(k') <= tol, and *loss_out = L(*k_out).
 *   sv: [k] HOST, descending, from rb_build.  n_templates: T of that rb_build.
 *   Errors: RB_ERR_BAD_INPUT (NULL pointer, k < 1, T < 1, tol not in [0, 1), sv not descending and
 *   >= 0, or sum sv^2 > T by more than rounding); RB_ERR_UNSUPPORTED when even L(k) > tol, with
 *   *k_out = k and *loss_out = L(k) (build a larger basis).
 */
int rb_basis_k_for_loss(const double* sv, int32_t k, int64_t n_templates, double tol, int32_t* k_out,
                        double* loss_out);

/*
 * rb_basis_max_loss - the worst single-template SNR loss of every basis size: for q in [0, k),
 *   loss[q] = max_t (1 - sum_{j<=q} |a_tj|^2), the relative SNR that template t loses, against the
 *   template method, on its own noiseless signal when only the first q + 1 basis vectors are kept
 *   (rows of unit norm, residual orthogonal to the span: rho_k / rho = 1 - r_t^2, the per-template
 *   quantity that Eq. 8 averages over the bank, Sec. III.B). Sums in FP64; values clamped at 0.
 *   basis->coeff: [T][k] device (rb_build output, rows in SNR units).  loss: [k] float64 HOST output.
 *   workspace: >= 8 k device bytes, 256-byte aligned. Synchronises `stream`.
 *   Errors: RB_ERR_BAD_INPUT (NULL pointer, k or T < 1), RB_ERR_OOM (workspace), RB_ERR_UNSUPPORTED
 *   (k > 6144).
 */
int rb_basis_max_loss(const rb_basis* basis, double* loss, void* workspace, size_t workspace_bytes, void* stream);

/* Candidate refinement (step a8; not in the paper, which stops at the triggers). */
typedef struct rb_refine_desc {
  double fs;          /* sample rate [Hz] */
  int64_t n;          /* block length (power of two, 2^10..2^20) */
  double f_low;       /* lower cutoff [Hz] */
  int32_t pn_order;   /* 0, 2 or 3 (non-spinning TaylorF2 as in rb_bank_desc) */
  int32_t steps;      /* gradient-ascent steps for rb_refine */
  double alpha0;      /* initial step length in scaled coordinates (e.g. 1e-3) */
  double alpha_max;   /* step length cap (e.g. 0.05) */
} rb_refine_desc;

/*
 * For a candidate theta = (mc [M_sun], eta, t_c [s from block start], phi_c) the matched filter of
 * Eq. (1) at the template's own coalescence time (Eq. 3-4 with t_0 inside Psi) is
 *   Z(theta) = sum_j s_hat[j] conj(g_j(theta)),  g_j = sqrt(4 df / S_j) f_j^(-7/6) exp(-i Psi(f_j; theta)),
 *   J(theta) = |Z|^2 / sigma^2,                  sigma^2 = sum_j |g_j|^2,
 * over the support f_low <= f_j < f_isco(theta_start), 0 < j < n/2, frozen at the starting point (so
 * sigma does not depend on theta). Psi is evaluated in FP64 and reduced modulo 2 pi before FP32
 * sin/cos; sums are accumulated in FP64. One CTA per candidate; the template is recomputed in every
 * pass, no per-template series is stored.
 *   s_hat: [n/2] complex device (rb_whiten output).  psd: [n/2+1] float64 device.
 *   theta: [n_cand][4] float64 device.  workspace: at least rb_refine_workspace_bytes(desc) bytes.
 */
size_t rb_refine_workspace_bytes(const rb_refine_desc* desc);

/* rb_refine_eval - J [n_cand] and Z [n_cand] complex (float64 pairs) at theta (the forward pass).
 * Errors: RB_ERR_BAD_INPUT (NULL output, sizes, PSD not finite and > 0 on 0 < j < n/2, a candidate with
 * mc <= 0, eta outside (0, 0.25] or non-finite t_c / phi_c), RB_ERR_OOM (workspace). */
int rb_refine_eval(const rb_refine_desc* desc, const float* s_hat, const double* psd, const double* theta,
                   double* J, double* Z, int64_t n_cand, void* workspace, size_t workspace_bytes, void* stream);

/* rb_refine_adjoint - the backward pass: given dL/dJ [n_cand] and the forward Z, recomputes the
 * templates and returns dL/dtheta [n_cand][4] = dL/dJ * 2 Re(conj(Z) dZ/dtheta) / sigma^2 with
 * dZ/dtheta = sum_j s_hat[j] (i dPsi_j/dtheta) conj(g_j). Errors: as rb_refine_eval. */
int rb_refine_adjoint(const rb_refine_desc* desc, const float* s_hat, const double* psd, const double* theta,
                      const double* Z, const double* dJ, double* dtheta, int64_t n_cand, void* workspace,
                      size_t workspace_bytes, void* stream);

/* rb_refine - desc->steps of normalised gradient ascent of J in scaled coordinates
 * u = (mc/mc_start, eta, t_c * 100 Hz, phi_c): a step of length alpha along the normalised gradient is
 * kept only if J increases (then alpha doubles, capped at alpha_max), otherwise alpha halves; eta is
 * clamped to [0.05, 0.25]. theta is updated in place; J [n_cand] receives the final J.
 * Errors: RB_ERR_BAD_INPUT (sizes, pn_order, eta outside (0, 0.25], mc <= 0). */
int rb_refine(const rb_refine_desc* desc, const float* s_hat, const double* psd, double* theta, double* J,
              int64_t n_cand, void* workspace, size_t workspace_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RBMF_H */
