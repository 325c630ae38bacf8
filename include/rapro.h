/*
 * rapro.h -- C ABI of the GB300 uplink receive path of
 * "Implementation of Massive MIMO Uplink Receiver on RaPro Prototyping Platform"
 * (arXiv 1802.05427): LS channel estimation -> low-complexity sub-block LMMSE
 * channel estimation -> per-subcarrier MMSE detection with Cholesky and QAM demapping.
 *
 * Notation.  The paper's R antennas and S users are M and K here; its N used
 * subcarriers are n_sc; the sub-block size of the partitioned correlation matrix is B.
 *
 * Conventions shared by every entry point
 *  - Array arguments are caller-owned DEVICE memory (the caller allocates and frees,
 *    like the receiver functions of Sec. III-B that read and write caller arrays),
 *    dense, in the layouts given below, subcarrier index fastest.  rapro_c32 is an
 *    interleaved single-precision complex {re, im} (8 bytes).  All arithmetic on the
 *    device is FP32; the LMMSE weights are built in FP64 on the host and rounded.
 *  - Work is enqueued on the caller's stream (a cudaStream_t, passed as rapro_stream;
 *    NULL means the legacy default stream).  Only rapro_plan_create and
 *    rapro_plan_destroy synchronise.  A return of RAPRO_OK means "validated and
 *    enqueued"; device-side results (non-positive-definite pivots, timeouts) are
 *    reported through the info array and rapro_plan_device_status.
 *  - The plan is the only library-owned memory: the weights W_b on the device, a
 *    channel-estimate workspace used by rapro_receive_subframe when h_out is NULL,
 *    the 16-bit forms' staging buffers, and one device status word.  rapro_plan_destroy frees all of it.
 *  - No call throws across the ABI, traps on the device or asserts.  NaN/Inf inputs
 *    propagate to the outputs.  Calls that share a plan may run concurrently on
 *    different streams except rapro_receive_subframe with h_out == NULL, which writes
 *    the plan's workspace, the detector of a RAPRO_PREC_BF16 or _FP16 plan, which keeps its
 *    FP64-fallback list in the plan, and the estimator of such a plan with 16 < B (the
 *    tensor-core GEMM), which stages its rounded LS operand in the plan: serialise those per
 *    plan.
 *
 * Layouts (T = n_pilot_sym slots, D = n_sym / n_pilot_sym - 1 data symbols per slot):
 *   y_pilot, h_ls, h  [T][K][M][n_sc]   pilot observation of user s at antenna m
 *   pilots            [T][K][n_sc]      transmitted pilot of user s (|p| != 0)
 *   y_data            [T*D][M][n_sc]    data OFDM symbols in time order; data symbol n
 *                                       belongs to slot n / D and is detected with
 *                                       that slot's channel estimate
 *   x_eq              [T*D][K][n_sc]    MMSE output x~ of Eq. 22
 *   labels            [T*D][K][n_sc]    hard decision as the q-bit Gray label
 *                                       (uint8, bit b0 = most significant)
 *   llr               [T*D][K][n_sc][q] max-log LLR per bit, b0 first, > 0 favours 0
 *   info              [T][n_sc]         0, or j+1 if pivot j of the Cholesky factor of
 *                                       H^H H + sigma2 I was not positive and finite
 * With pilot_layout == RAPRO_PILOT_COMB (the shared pilot symbol of Sec. II, user s on
 * the tones s, s + S, s + 2S, ... of a comb of spacing S = comb_spacing):
 *   y_pilot           [T][M][n_sc]      received pilot OFDM symbol of each slot
 *   pilots            [T][n_sc]         value sent on each tone by the user owning it
 *   h                 [T][K][M][n_sc]   dense channel estimate, as above
 */
#ifndef RAPRO_H
#define RAPRO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { float re, im; } rapro_c32;

/* Same type as cudaStream_t; this header does not need the CUDA headers. */
typedef struct CUstream_st* rapro_stream;

typedef enum {
  RAPRO_OK = 0,
  RAPRO_ERR_INVALID_ARG = 1,   /* a size, pointer or parameter outside its documented range */
  RAPRO_ERR_CUDA = 2,          /* a CUDA runtime call failed (the message is kept, see below) */
  RAPRO_ERR_NOT_POSDEF = 3,    /* the FP64 host factorisation of R_b + sigma2 I failed */
  RAPRO_ERR_TIMEOUT = 4,       /* a device wait hit its iteration limit (device status) */
  RAPRO_ERR_UNSUPPORTED = 5,   /* a valid request this build does not implement */
  RAPRO_ERR_NOMEM = 6          /* device allocation failed in rapro_plan_create */
} rapro_status;

typedef enum {
  RAPRO_PILOT_ORTHOGONAL = 0,  /* one pilot observation per user on every subcarrier */
  RAPRO_PILOT_COMB = 1         /* the FDM comb of Sec. II, estimated by rapro_ce_comb */
} rapro_pilot_layout;

/* Estimators of the comb layout (Sec. IV-B; groups and windows of Tables I and II). */
typedef enum {
  /* 3W-LMMSE: per pilot tone j of a user, 3 estimates at the tone and S/3, 2S/3 after it
   * from the LS of 3 consecutive tones (window min(max(j-1, 0), P-3)), one of 3 weight
   * matrices shared by all users; zero-order hold to every subcarrier.  3 | S. */
  RAPRO_COMB_3W = 0,
  /* S-W-LMMSE (12W at S = 12): per group j, the S subcarriers jS .. jS+S-1 from the LS of
   * S consecutive tones (window min(max(j-(S-1)/2, 0), P-S)), one of S weight matrices
   * per user. */
  RAPRO_COMB_SW = 1,
  /* Three-fold linearly interpolated LS at the 3W positions (the comparator of Sec. V),
   * the last tone's LS held past it, then zero-order hold.  3 | S. */
  RAPRO_COMB_INTERP3 = 2
} rapro_comb_method;

typedef enum {
  /* Exponential power-delay profile of Sec. III-A (text under Eq. 16) on integer delays:
   * r(d) = sum_{l<n_taps} p_l exp(-j 2 pi l d / n_fft), p_l = exp(-l/tau_rms) / sum. */
  RAPRO_PDP_EXP = 0,
  /* Eq. 16: r(0) = 1, r(d) = (1 - exp(-j 2 pi L d / n_fft)) / (j 2 pi L d / n_fft). */
  RAPRO_PDP_UNIFORM_L = 1
} rapro_pdp_kind;

/* Arithmetic of the sub-block LMMSE filter (Eq. 12). */
typedef enum {
  /* FP32 accuracy: TF32 tensor cores with three split passes (even B <= 16 dividing n_sc,
   * 16-byte aligned arrays) or FP32 FMAs otherwise. */
  RAPRO_PREC_FP32 = 0,
  /* Precision form: one BF16 pass on the tensor cores, FP32 accumulation (W and the LS
   * estimate rounded to BF16; relative filter error ~ 2^-8).  Needs the orthogonal layout,
   * an even B <= 2048 dividing n_sc and 16-byte aligned arrays; rapro_ce_lmmse_subblock and
   * w_override are not available (RAPRO_ERR_UNSUPPORTED).  The detector of such a plan
   * (rapro_detector_form, default RAPRO_DET_REFINED) forms the Gram H^H H + sigma2 I and
   * H^H y on the tensor cores from BF16 operands (FP32 accumulation), factors it in FP32 and
   * takes one FP32 refinement step with the residual H^H (y - H x~) - sigma2 x~ from the
   * FP32 h (16-byte aligned h and y_data and an even n_sc; other arrays take the FP32
   * detector).  Either detector falls back to FP64 for every subcarrier whose FP32
   * Cholesky pivots give (max L_jj / min L_jj)^2 > 1e6 (a lower bound of cond(A)) or fail:
   * Eq. 22 solved again in FP64 by the last CTA, which overwrites that subcarrier's outputs
   * and info. */
  RAPRO_PREC_BF16 = 1,
  /* As RAPRO_PREC_BF16 with FP16 operands (11 significant bits, range +-65504: relative
   * filter error ~ 2^-10 for the O(1) LS estimates and weights of unit-power channels);
   * the same rules and the same FP64 detector fallback. */
  RAPRO_PREC_FP16 = 2
} rapro_precision;

/* How rapro_receive_subframe runs a subframe (no counterpart in the paper, which runs the
 * steps one after the other on each core; the results agree to FP32 rounding). */
typedef enum {
  /* Default: the estimator kernel (into h_out or the plan's workspace), then the detector. */
  RAPRO_RECV_SPLIT = 0,
  /* One kernel does LS (Eq. 9), the sub-block LMMSE (Eq. 12, FP32 FMAs) and the detection
   * (Eq. 20-22) per tile of 16 subcarriers, the estimate of each antenna chunk staying in
   * shared memory (written to h_out only if given).  Applies to orthogonal-layout
   * RAPRO_PREC_FP32 plans with an even B <= 16, even n_sc and 16-byte aligned y_pilot and
   * y_data; other plans and arrays take the two-kernel form.  Faster than the default on
   * small subframes (one launch) and some block sizes; rapro_plan_tune picks the faster. */
  RAPRO_RECV_FUSED = 1
} rapro_receive_form;

/* Detector of a RAPRO_PREC_BF16 / _FP16 plan (no counterpart in the paper).  The refined
 * form follows the precision form as specified; at D data symbols per slot its FP32 residual
 * costs 2 M K D complex multiply-adds per subcarrier, about what the FP32 Gram and matched
 * filter cost (M K (K + 1) / 2 + M K D), so the FP32 form is the faster one at D ~ K/2. */
typedef enum {
  RAPRO_DET_REFINED = 0,   /* tensor-core Gram of 16-bit operands + one FP32 refinement step */
  RAPRO_DET_FP32 = 1       /* the FP32 detector (Gram and matched filter in FP32 FMAs) */
} rapro_detector_form;

#define RAPRO_MAX_PILOT_SYM 8
#define RAPRO_MAX_USERS 16       /* K limit of the register-tiled detector */
#define RAPRO_MAX_DATA_PER_SLOT 12

typedef struct {
  int M;                 /* BS antennas (paper: R), >= 1 */
  int K;                 /* single-antenna users (paper: S), 1..RAPRO_MAX_USERS */
  int n_sc;              /* used subcarriers (paper: N), >= 1 */
  int n_fft;             /* FFT size (paper: N_FFT), >= n_sc; the N of Eq. 16 */
  int n_sym;             /* OFDM symbols per subframe, e.g. 14 */
  int n_pilot_sym;       /* pilot symbols = slots T, 1..RAPRO_MAX_PILOT_SYM; n_sym % T == 0 */
  int pilot_sym_idx[RAPRO_MAX_PILOT_SYM]; /* symbol index of the pilot of slot j; must lie in
                                             [j*n_sym/T, (j+1)*n_sym/T) */
  int pilot_layout;      /* rapro_pilot_layout */
  int subblock;          /* B, 1..n_sc; B == n_sc is the full LMMSE of Eq. 13 */
  double sigma2;         /* noise variance sigma^2 > 0 (pilot power sigma_s^2 = 1), used by
                            both the estimator (Eq. 17) and the detector (Eq. 22) */
  int pdp;               /* rapro_pdp_kind */
  int n_taps;            /* EXP: taps at delays 0..n_taps-1, >= 1 */
  double tau_rms;        /* EXP: decay constant in samples, > 0 */
  double L;              /* UNIFORM_L: assumed channel length in samples, > 0 */
  int qam_bits;          /* q = 2 (QPSK), 4 (16-QAM) or 6 (64-QAM) */
  /* pilot_layout == RAPRO_PILOT_COMB only (ignored otherwise; subblock is then unused): */
  int comb_spacing;      /* S: tone spacing of each user's comb, K <= S <= 16, S | n_sc,
                            P = n_sc / S tones per user, 2 <= P <= 1024, P >= the window */
  int comb_method;       /* rapro_comb_method */
  int precision;         /* rapro_precision of the sub-block filter, default RAPRO_PREC_FP32 */
} rapro_params;

typedef struct rapro_plan rapro_plan;

/* Human-readable name of a status code (static storage). */
const char* rapro_status_string(rapro_status s);

/* Text of the last error recorded by this thread (CUDA message or argument check). */
const char* rapro_last_error(void);

/* Check a parameter set without touching the GPU.  Host only. */
rapro_status rapro_params_validate(const rapro_params* p);

/*
 * Host-only FP64 weights of one sub-block (Eq. 13/17 with R_{H Hls} = R_{HH}):
 *   W = R (R + sigma2 I)^-1,  R[a][b] = r(a - b),  a, b in [0, block_len)
 * built from p's PDP model; written row-major as interleaved {re, im} doubles,
 * w_out[2*(a*block_len + b) + {0,1}].  block_len in [1, 4096].
 * Returns RAPRO_ERR_NOT_POSDEF if R + sigma2 I fails to factor in FP64.
 */
rapro_status rapro_build_weights_host(const rapro_params* p, int block_len, double* w_out);

/*
 * Host-only FP64 weights of the comb estimators (pilot_layout == RAPRO_PILOT_COMB,
 * comb_method 3W or S-W; Sec. IV-B, Eq. 17 with Eq. W1-W3 and P).  Q = 3 (3W) or S (S-W);
 * sets = 1 (3W, shared by all users) or K (S-W, one per user).  w_out receives
 * sets * Q * Q * Q complex doubles, interleaved {re, im}: set k, weight index w (the
 * group's position in its window, Tables I-II: W^(w+1)), row u (estimate), column i
 * (window tone) at 2 * (((k*Q + w)*Q + u)*Q + i).
 * Returns RAPRO_ERR_NOT_POSDEF if R_{Hls Hls} + sigma2 I fails to factor in FP64.
 */
rapro_status rapro_build_comb_weights_host(const rapro_params* p, double* w_out);

/*
 * Validate p, build W_b for the full block size B and for the tail block of
 * n_sc mod B subcarriers (blocks start at subcarrier 0), or the comb weights of
 * rapro_build_comb_weights_host for a comb plan, round them to complex64, copy them to
 * the current device, and allocate the workspace.
 * Synchronous.  *out is NULL on failure.
 */
rapro_status rapro_plan_create(const rapro_params* p, rapro_plan** out);

/* Free the plan and its device memory (synchronises the device first).  NULL is a no-op. */
rapro_status rapro_plan_destroy(rapro_plan* plan);

/* Derived sizes of a plan: slots T, data symbols per slot D, blocks nb, tail size
 * (0 if B divides n_sc).  Any output pointer may be NULL. */
rapro_status rapro_plan_dims(const rapro_plan* plan, int* T, int* D, int* nb, int* tail);

/*
 * Read (and with reset != 0 clear) the plan's device status word: 0, or
 * RAPRO_ERR_TIMEOUT if a kernel gave up waiting on one of its pipeline barriers.
 * Synchronises the plan's status copy with the device.
 */
rapro_status rapro_plan_device_status(rapro_plan* plan, int reset, int* status_out);

/*
 * Step a1 -- LS estimate, Eq. 8-9: h_ls = y_pilot / pilots = y_pilot conj(p) / |p|^2
 * per (slot, user, antenna, subcarrier).  The paper multiplies by the conjugate pilot
 * because its pilots have unit modulus (Sec. IV-C); the division form is exact for any
 * nonzero pilot.  In-place (h_ls == y_pilot) is allowed.
 */
rapro_status rapro_ce_ls(const rapro_plan* plan, const rapro_c32* y_pilot,
                         const rapro_c32* pilots, rapro_c32* h_ls, rapro_stream stream);

/*
 * Step a3 -- sub-block LMMSE filter, Eq. 12 with the fixed weights of Eq. 17:
 *   h[t][s][m][blk] = W_blk * h_ls[t][s][m][blk]
 * for every slot, user and antenna, over the non-overlapping blocks of B contiguous
 * subcarriers (the last block holds n_sc mod B).  w_override, if not NULL, replaces
 * the plan's weights: nb matrices stored one after another, block b's W row-major,
 * B*B entries for full blocks and tail*tail for the tail.  h must not alias h_ls.
 */
rapro_status rapro_ce_lmmse_subblock(const rapro_plan* plan, const rapro_c32* h_ls,
                                     const rapro_c32* w_override, rapro_c32* h,
                                     rapro_stream stream);

/*
 * Steps a1 + a3 in one pass: the LS estimate of Eq. 9 is formed on load and filtered by
 * the sub-block weights of Eq. 12/17 without being stored:
 *   h[t][s][m][blk] = W_blk * (y_pilot[t][s][m][blk] conj(p[t][s][blk]) / |p|^2).
 * w_override as for rapro_ce_lmmse_subblock.  h must not alias y_pilot.
 */
rapro_status rapro_ce_ls_lmmse(const rapro_plan* plan, const rapro_c32* y_pilot,
                               const rapro_c32* pilots, const rapro_c32* w_override,
                               rapro_c32* h, rapro_stream stream);

/*
 * Steps a4-a8 -- MMSE detection, Eq. 20-22, per (slot, subcarrier):
 *   A = H^H H + sigma2 I (Gram), z = H^H y (matched filter), A = L L^H (Cholesky, the
 *   uplo = L factorisation the paper solves with), L L^H x~ = z for every data symbol
 *   of the slot; x_eq = x~.  Demapping: mu_k = 1 - sigma2 [A^-1]_kk, x^ = x~ / mu,
 *   labels = nearest Gray-QAM point of x^, llr_i = (min_{b_i=1}|x^-x|^2 -
 *   min_{b_i=0}|x^-x|^2) / nu with nu = (1 - mu) / mu.
 * labels, llr and info may be NULL (not produced).  A subcarrier whose pivot fails
 * gets info = j+1 and NaN outputs; the others are unaffected.
 */
rapro_status rapro_mmse_detect(const rapro_plan* plan, const rapro_c32* h,
                               const rapro_c32* y_data, rapro_c32* x_eq, uint8_t* labels,
                               float* llr, int32_t* info, rapro_stream stream);

/*
 * Comb-pilot channel estimation (plans with pilot_layout == RAPRO_PILOT_COMB; Sec. II,
 * IV-B): the LS estimate of Eq. 9 on each user's tones, then the plan's comb_method
 * (3W- or S-W-LMMSE: W = R_{H Hls} (R_{Hls Hls} + sigma2 I)^-1 of Eq. 17 with the
 * rectangular cross-correlation of Eq. W1-W3 and P, per group of Tables I and II; or
 * three-fold interpolated LS), and zero-order hold, into the dense h [T][K][M][n_sc] the
 * detector reads.  The weights are built in FP64 at plan creation.  Layouts in the header
 * comment.  Orthogonal-layout plans return RAPRO_ERR_UNSUPPORTED (and comb plans do so
 * for rapro_ce_ls, rapro_ce_lmmse_subblock and rapro_ce_ls_lmmse).
 */
rapro_status rapro_ce_comb(const rapro_plan* plan, const rapro_c32* y_pilot, const rapro_c32* pilots,
                           rapro_c32* h, rapro_stream stream);

/*
 * The whole path (a1, a3, a4-a8) for one subframe on one stream, in the plan's receive form
 * (rapro_receive_form): fused into one kernel where it applies, else rapro_ce_ls_lmmse
 * (rapro_ce_comb for a comb plan) followed by rapro_mmse_detect.  h_out (nullable)
 * receives the channel estimate; when NULL the two-kernel form keeps it in the plan's
 * workspace and the fused form does not store it.  Other arguments as above.
 */
rapro_status rapro_receive_subframe(const rapro_plan* plan, const rapro_c32* y_pilot,
                                    const rapro_c32* pilots, const rapro_c32* y_data,
                                    rapro_c32* h_out, rapro_c32* x_eq, uint8_t* labels,
                                    float* llr, int32_t* info, rapro_stream stream);

/*
 * Autotuner (no counterpart in the paper, whose receiver has one code path): times every
 * combination of the estimator kernels that apply to the plan's shape and these arrays
 * (tensor cores with one or as many CTAs per SM as fit, the tensor-core GEMM for large
 * blocks, streaming, row-segment and tiled kernels; comb plans have one), the detector's warps per role and (where it applies) the
 * fused receive form, each as whole receives with four subframes in flight on streams of
 * the library's (one at a time for BF16 and FP16 plans), 2 warm and 5 timed rounds, and
 * keeps the one with the best throughput in the plan (later calls with arrays a choice does
 * not apply to fall back to the built-in choice).  Overwrites h and x_eq.  Synchronises the stream; not inside a
 * stream capture.  The plan must not be in use by another stream meanwhile.
 */
rapro_status rapro_plan_tune(rapro_plan* plan, const rapro_c32* y_pilot, const rapro_c32* pilots,
                             const rapro_c32* y_data, rapro_c32* h, rapro_c32* x_eq, rapro_stream stream);

/* The plan's kernel choices: estimator kernel (-1 built-in, 0 tensor cores, 1 streaming,
 * 2 row segments, 3 tiled, 4 tensor-core GEMM for even 16 < B <= 2048 dividing n_sc), the detector's
 * warps per role, and the tensor-core estimator's
 * CTAs per SM (0: as many as fit).  A new plan has -1, 1 and 1: one warp per role and one
 * estimator CTA per SM leave room on every SM for an estimator and a detector CTA of two
 * subframes in flight.  Any pointer may be NULL. */
rapro_status rapro_plan_variant(const rapro_plan* plan, int* est_variant, int* det_split, int* est_ctas_per_sm);

/* Set the plan's kernel choices by hand (as rapro_plan_tune would): est_variant -1 (built-in)
 * or 0..4 as above (a choice that does not apply to later calls' arrays falls back to the
 * built-in one), det_split 1 or 2 (at most 2 when the detector has at most 8 roles, else 1),
 * est_ctas_per_sm 0..8.  RAPRO_ERR_INVALID_ARG otherwise.  Not while another stream uses the
 * plan. */
rapro_status rapro_plan_set_variant(rapro_plan* plan, int est_variant, int det_split, int est_ctas_per_sm);

/* Set the plan's receive form (rapro_receive_form; RAPRO_ERR_INVALID_ARG otherwise).  Not
 * while another stream uses the plan. */
rapro_status rapro_plan_set_receive_form(rapro_plan* plan, int form);

/* Set the detector form of a RAPRO_PREC_BF16 / _FP16 plan (rapro_detector_form;
 * RAPRO_ERR_INVALID_ARG for another value, RAPRO_ERR_UNSUPPORTED for an FP32 plan).  Not
 * while another stream uses the plan. */
rapro_status rapro_plan_set_detector_form(rapro_plan* plan, int form);

/* *fused = 1 if rapro_receive_subframe with these y_pilot and y_data pointers runs the fused
 * kernel under the plan's current form, else 0.  No device work. */
rapro_status rapro_receive_is_fused(const rapro_plan* plan, const rapro_c32* y_pilot, const rapro_c32* y_data,
                                    int* fused);

/*
 * Batched heterogeneous receive: many independent subframes, each with its own plan (any
 * shapes, layouts and precisions), in one call.  The library's pool of n_streams CUDA
 * streams (rapro_batch_create, 1..32) runs them side by side: the jobs go longest first
 * (estimated multiply-accumulates) onto the least loaded stream, forked from and joined back
 * into the caller's stream with events, so the call can be captured into one CUDA graph and
 * returns "enqueued" like the single-subframe call.  Jobs that share a plan must pass h_out
 * (the plan's workspace holds one estimate).  Arguments of each job as for
 * rapro_receive_subframe; one bad job returns its status after the jobs before it were
 * enqueued and the streams joined.
 */
typedef struct rapro_batch rapro_batch;
typedef struct {
  const rapro_plan* plan;
  const rapro_c32* y_pilot;
  const rapro_c32* pilots;
  const rapro_c32* y_data;
  rapro_c32* h_out;      /* nullable: the plan's workspace */
  rapro_c32* x_eq;
  uint8_t* labels;       /* nullable */
  float* llr;            /* nullable */
  int32_t* info;         /* nullable */
} rapro_job;
rapro_status rapro_batch_create(int n_streams, rapro_batch** out);
rapro_status rapro_batch_destroy(rapro_batch* batch);   /* synchronises the device; NULL is a no-op */
rapro_status rapro_receive_batch(rapro_batch* batch, const rapro_job* jobs, int n_jobs, rapro_stream stream);

/*
 * Reverse mode of the symbol MSE, for fitting the model parameters of Eq. 13/17 (the paper
 * fixes them by hand: L and SNR_fixed, Sec. IV-C) and sigma2 by gradient descent.  With the
 * forward results h and x_eq of rapro_receive_subframe and known transmitted symbols
 * x_ref [T*D][K][n_sc] (training data):
 *   L = mean over (data symbol, user, subcarrier) of |x_eq - x_ref|^2.
 * Outputs (device; gradients are conjugate Wirtinger gradients G = dL/dX*, i.e.
 * dL = 2 Re sum conj(G) dX):
 *   g_h       [T][K][M][n_sc]  dL/dh*  (detector adjoint of Eq. 22: sum_d y_d lambda_d^H -
 *                              H sum_d (lambda_d x~_d^H + x~_d lambda_d^H), lambda_d = A^-1 g_d)
 *   scalars   [2] floats       L, and dL/dsigma2 through the detector only (W held fixed)
 *   g_w_main  [B][B]           dL/dW* of the shared block weights (sum over rows and blocks of
 *                              g_h,blk h_ls,blk^H, Eq. 12), g_w_tail [tail][tail] likewise
 * FP32 on the device, accumulated with atomics.  Orthogonal plans, B <= 64, n_sc <= 2048
 * (RAPRO_ERR_UNSUPPORTED otherwise).  g_h must not alias an input.
 */
rapro_status rapro_mse_backward(const rapro_plan* plan, const rapro_c32* y_pilot, const rapro_c32* pilots,
                                const rapro_c32* y_data, const rapro_c32* h, const rapro_c32* x_eq,
                                const rapro_c32* x_ref, rapro_c32* g_h, float* scalars, rapro_c32* g_w_main,
                                rapro_c32* g_w_tail, rapro_stream stream);

/*
 * Host-only FP64 chain rule through W = R (R + sigma2 I)^-1 (exponential PDP model):
 * dW/dsigma2 = -W A^-1 and dW/dtau = (I - W) dR/dtau A^-1 with A = R + sigma2 I.
 * g_w_main / g_w_tail: the weight gradients of rapro_mse_backward as interleaved doubles
 * (g_w_tail may be NULL when B divides n_sc).  grad_out[0] = dL/dsigma2 and
 * grad_out[1] = dL/dtau_rms through the estimator; the total dL/dsigma2 adds the
 * detector's term from rapro_mse_backward.
 */
rapro_status rapro_weight_grad_host(const rapro_params* p, const double* g_w_main, const double* g_w_tail,
                                    double* grad_out);

/*
 * Diagnostics of the device-side timeout path (not for production use).  wait_rounds > 0
 * limits each wait between the FP32 detector's TMA load producer and its consumers to that
 * many bounded try-wait rounds (each suspends at most 2 us; 0 restores the default limit of
 * about 2 s); stall_producer != 0 makes the producer post no load, so that the consumers'
 * first wait runs out.  The kernel then records RAPRO_ERR_TIMEOUT in the plan's status word
 * (rapro_plan_device_status), writes no output and no info entry, and returns; copies in
 * flight are always drained with the default limit.  Affects rapro_mmse_detect and
 * rapro_receive_subframe on the TMA path of FP32 plans.  Host only.
 */
rapro_status rapro_plan_set_wait_test(rapro_plan* plan, int stall_producer, uint32_t wait_rounds);

/*
 * Steps a4 + a5 on the tensor cores with 16-bit operands (the precision form's Gram, Eq. 22):
 * per (slot t, subcarrier k) with H_k = h[t][:, :, k] (K users x M antennas) and Y_k the
 * slot's D data symbols at subcarrier k,
 *   gram[t][k][s][c] = (H_k^H H_k + sigma2 I)[s][c]   for c < K,
 *   gram[t][k][s][K + n] = (H_k^H Y_k)[s][n]           for n < D,
 * layout [T][n_sc][K][K + D] complex, caller-owned device memory.  h and y_data are rounded
 * to BF16 (fp16 == 0) or FP16 (fp16 != 0), the products accumulate in FP32 (tcgen05,
 * kind::f16).  Needs 16-byte aligned h and y_data and an even n_sc (RAPRO_ERR_UNSUPPORTED
 * otherwise) and the orthogonal pilot layout's plan shapes.
 */
rapro_status rapro_gram_tc(const rapro_plan* plan, const rapro_c32* h, const rapro_c32* y_data, rapro_c32* gram,
                           int fp16, rapro_stream stream);

/*
 * Measurement utility (not a step of the receive path): the device's FP32 FMA rate.
 * Launches a full-occupancy grid (8 CTAs of 256 threads per SM) in which every thread
 * runs 8 independent FMA recurrences for 16 x trips rounds, on `stream`, timed with CUDA
 * events after one short warm-up launch; waits for it to finish.  *tflops_out receives
 * 2 x FMAs / seconds / 1e12 and *ms_out (nullable) the timed launch's duration.  The SM
 * clock during the launch decides the figure: sample it alongside.  RAPRO_ERR_INVALID_ARG
 * if trips < 1 or tflops_out is NULL.
 */
rapro_status rapro_measure_ffma_peak(int trips, double* tflops_out, double* ms_out, rapro_stream stream);

/*
 * Allocation-free variant of rapro_receive_subframe (the paper has no counterpart; it
 * runs its receiver on host memory it allocates freely).  For callers that cannot
 * allocate device memory when a subframe arrives: real-time slot loops that must not
 * wait on an allocator (cudaMalloc can synchronise the device or take milliseconds,
 * longer than a slot's deadline), processes whose device memory belongs to another
 * framework's pool, and deployments that forbid run-time allocation.
 *  - Needs no plan: p is validated and the weights of its sub-block size are built in
 *    FP64 on the host at every call (the plan's builder, in stack storage) and passed to
 *    the kernel as parameters, so subblock must be <= 32 (RAPRO_ERR_UNSUPPORTED
 *    otherwise).  The comb layout and the 16-bit precision forms are not available here
 *    (RAPRO_ERR_UNSUPPORTED): precision must be RAPRO_PREC_FP32.
 *  - The channel-estimate scratch is a fixed 32 MiB device array inside the library
 *    (held by every GPU that loads the library until the process exits):
 *    n_pilot_sym * K * M * n_sc * 8 bytes must not exceed 32 MiB (RAPRO_ERR_INVALID_ARG
 *    otherwise; the 128 x 12 x 1200 two-slot subframe needs 29.5 MB).
 *  - Allocates and frees no device memory; the only host allocation is the text of an
 *    error message on a rejected call.
 *  - The first call on a device (of this function or rapro_noalloc_status) looks up the
 *    scratch's device address and raises the kernels' shared-memory limits; make that
 *    first call before any stream capture.
 *  - All calls share the scratch and its status word (they keep the last call's
 *    contents; each call clears the status word first): calls that overlap on the GPU
 *    race and give undefined outputs; serialise them.
 *  - A pipeline timeout is recorded in the scratch's status word (read it with
 *    rapro_noalloc_status).  After an estimator timeout the detector writes nothing; after
 *    a detector timeout the affected subcarriers' outputs and info entries are left
 *    unwritten, so a caller may also fill info with a sentinel (e.g. -1) before the call.
 * Inputs, outputs, layouts and results are those of rapro_receive_subframe with
 * h_out == NULL, on the caller's stream.
 */
rapro_status rapro_receive_subframe_noalloc(const rapro_params* p, const rapro_c32* y_pilot,
                                            const rapro_c32* pilots, const rapro_c32* y_data,
                                            rapro_c32* x_eq, uint8_t* labels, float* llr,
                                            int32_t* info, rapro_stream stream);

/*
 * Status word of the allocation-free receive on the current device: enqueues a read of it
 * on `stream` (after the calls enqueued there before), clears it if reset != 0, and waits
 * for the stream.  *status_out: RAPRO_OK, or RAPRO_ERR_TIMEOUT if a pipeline wait of the
 * last rapro_receive_subframe_noalloc call ran out.  Allocates nothing.
 */
rapro_status rapro_noalloc_status(int reset, int* status_out, rapro_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* RAPRO_H */
