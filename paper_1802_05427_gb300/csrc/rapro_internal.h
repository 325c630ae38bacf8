// Internal declarations shared by the host plan, the ABI layer and the kernels.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <complex>
#include <vector>

#include "rapro.h"

namespace rapro {

// Detector tiling: each CTA owns DET_SC consecutive subcarriers of one slot and streams
// the antennas through shared memory DET_MCH at a time.
constexpr int DET_SC = 16;
constexpr int DET_MCH = 8;
constexpr int DET_STAGES = 4;

// Work roles of the detector's accumulation, one warp each (times an antenna split).
// Users form groups of 4 (g = 0 .. NG-1), data symbols groups of 6.  A role is
//   kind 0: the lower triangle of group g's Gram block plus, if r >= 0, the full
//           Gram block of rows group r x columns group c (r > c);
//   kind 1: only the block rows r x columns c;
//   kind 2: matched-filter block of users group g x data symbols c*6 .. c*6+5.
// Every needed entry of A (lower triangle) and z is computed exactly once.
constexpr int DET_MAX_ROLES = 16;
struct DetTiles {
  int n_roles;
  int msplit;  // warps per role, each taking part of every antenna chunk
  int KP;      // padded user rows in the shared-memory stage (4 * NG)
  int DP;      // padded data rows (6 * data groups)
  signed char kind[DET_MAX_ROLES];
  signed char g[DET_MAX_ROLES];
  signed char r[DET_MAX_ROLES];
  signed char c[DET_MAX_ROLES];
};

constexpr int LMMSE_SMALL_MAX = 32;   // B <= this uses the weights-in-parameter kernel

struct Plan {
  rapro_params p;
  int T = 0, D = 0, q = 0;
  int B = 0, nb = 0, tail = 0;     // block size, block count, tail block size (0 = none)
  std::vector<float2> w_main;      // B x B row-major, complex64
  std::vector<float2> w_tail;      // tail x tail
  float2* d_w_main = nullptr;
  float2* d_w_tail = nullptr;
  float2* d_h_work = nullptr;      // [T][K][M][n_sc] estimate workspace
  int* d_status = nullptr;         // device status word
  void* d_w_tc = nullptr;          // tensor-core filter operand (canonical layout), or null
  void* d_w_tcg = nullptr;         // large-B tensor-core GEMM operand (tiles of Wr chunks), or null
  void* d_a_tcg = nullptr;         // 16-bit GEMM forms: staged LS operand (canonical A chunks), or null
  int est_variant = -1;            // estimator kernel (EST_*), -1 = built-in choice; set by rapro_plan_tune
  int recv_form = RAPRO_RECV_SPLIT; // rapro_receive_form of rapro_receive_subframe
  // Tensor-core estimator CTAs per SM (0: as many as fit).  One leaves each SM room for a
  // detector CTA of the next subframe in flight (with one warp per detector role), which
  // raises the throughput of pipelined subframes; set by rapro_plan_tune / _set_variant.
  int est_ctas_per_sm = 1;
  int* d_fix = nullptr;            // precision form: FP64-fallback count, ticket, list [T n_sc]
  float2* d_gram = nullptr;        // precision form: tensor-core Gram | matched filter [T][n_sc][K][K + D]
  int det_form = RAPRO_DET_REFINED; // detector of a 16-bit plan (rapro_detector_form)
  uint32_t wait_rounds = 0;        // diagnostics (rapro_plan_set_wait_test): detector handoff wait limit
  int stall_producer = 0;          //   and a load producer that posts nothing
  bool comb = false;               // comb pilot layout (Sec. II)
  std::vector<float2> w_comb;      // comb weights [sets][Q][Q][Q] (3W: 1 set, S-W: K sets)
  float2* d_w_comb = nullptr;
  DetTiles tiles{};
  int device = 0;
};

// The precision forms with 16-bit filter operands (BF16 or FP16 on the tensor cores).
inline bool half_precision(const rapro_params& p) {
  return p.precision == RAPRO_PREC_BF16 || p.precision == RAPRO_PREC_FP16;
}

// Thread-local last-error text.
void set_error(const std::string& msg);
rapro_status cuda_fail(cudaError_t e, const char* what);

// Frequency correlation r(d) of subcarriers d apart (Eq. 16, or the exponential PDP), FP64.
std::complex<double> corr_fp64(const rapro_params& p, int d);

// Host FP64 weights of one block of len subcarriers: W = R (R + s I)^-1, row-major
// interleaved.  Returns false if R + s I is not positive definite in FP64.
bool build_weights_fp64(const rapro_params& p, int len, std::vector<double>& w);
// The same arithmetic into caller storage, allocating nothing: work holds
// weights_fp64_work(len) complex doubles, w_out 2 len^2 doubles.
constexpr size_t weights_fp64_work(int len) { return size_t(2 * len - 1) + 2 * size_t(len) * len + size_t(len); }
bool weights_fp64_into(const rapro_params& p, int len, std::complex<double>* work, double* w_out);

DetTiles make_det_tiles(int K, int D);

// Comb layout: window Q (3 or S) and the FP64 weights [sets][w][u][i], interleaved.
int comb_window(const rapro_params& p);
bool build_comb_weights_fp64(const rapro_params& p, std::vector<double>& w_out);
cudaError_t launch_comb(const Plan& pl, const float2* y, const float2* pil, float2* h, cudaStream_t st);
cudaError_t prepare_comb(int device);

// One subframe through the estimator and the detector on st (rapro_receive_subframe).
rapro_status receive_on(const Plan* pl, const rapro_c32* y_pilot, const rapro_c32* pilots, const rapro_c32* y_data,
                        rapro_c32* h_out, rapro_c32* x_eq, uint8_t* labels, float* llr, int32_t* info,
                        cudaStream_t st);

// Reverse mode of the symbol MSE (k_adjoint.cu); weights' chain rule on the host.
int adjoint_max_block();
int adjoint_max_subcarriers();
cudaError_t launch_adjoint(const Plan& pl, const float2* y_pilot, const float2* pilots, const float2* y_data,
                           const float2* h, const float2* x_eq, const float2* x_ref, float2* g_h, float* scal,
                           float2* g_wm, float2* g_wt, cudaStream_t st);
cudaError_t prepare_adjoint(int device);
// The detector part of the adjoint (k_adj_detect.cu): G_H, the loss and dL/dsigma2 into scal.
cudaError_t launch_adj_detect(const Plan& pl, const float2* h, const float2* y, const float2* x_eq,
                              const float2* x_ref, float2* g_h, float* scal, cudaStream_t st);
cudaError_t prepare_adj_detect(int device);

// Kernel launchers (return the launch error, if any).
cudaError_t launch_ls(const float2* y, const float2* pil, float2* h, int T, int K, int M,
                      int N, cudaStream_t st);

// LMMSE filter; if pil != nullptr the input is y_pilot and LS is applied on load.
// w_main/w_tail: host copies (small-B kernel) or device pointers (tiled kernel).
cudaError_t launch_lmmse(const Plan& pl, const float2* x, const float2* pil,
                         const float2* d_w_main, const float2* d_w_tail,
                         const float2* h_w_main, const float2* h_w_tail, float2* out,
                         cudaStream_t st);

cudaError_t prepare_detect(int device);
// Precision form: subcarriers with (max L_jj / min L_jj)^2 > kFp64CondLimit are redone in FP64.
constexpr float kFp64CondLimit = 1.0e6f;
cudaError_t prepare_estimate(int device);
cudaError_t prepare_lmmse_tc(int device);
// Estimator kernels a plan can use (the autotuner times the ones that apply).
enum { EST_TC = 0, EST_STREAM = 1, EST_SMALL = 2, EST_TILED = 3, EST_TCG = 4, EST_VARIANTS = 5 };
bool lmmse_variant_ok(const Plan& pl, int v, const float2* x, const float2* pil, const float2* out);
// Detector warps per role of a plan by default: one, so that a detector CTA and an estimator
// CTA of another subframe in flight share an SM (registers allow it only then).
constexpr int kDefaultDetSplit = 1;
cudaError_t launch_lmmse_variant(const Plan& pl, int v, const float2* x, const float2* pil, float2* out,
                                 cudaStream_t st);
// Tensor-core LS + LMMSE (even B <= 16 dividing n_sc, aligned arrays).
bool lmmse_tc_shape_ok(const Plan& pl);
void build_lmmse_tc_weights(const Plan& pl, std::vector<unsigned char>& out);
bool lmmse_tc_ok(const Plan& pl, const float2* y, const float2* pil, const float2* out);
cudaError_t launch_lmmse_tc(const Plan& pl, const float2* y, const float2* pil, float2* out, cudaStream_t st);
// Tensor-core GEMM form for larger blocks (even 16 < B <= 2048 dividing n_sc, FP32 plans,
// aligned arrays); pil may be null (the input is then h_ls).
bool lmmse_tcg_shape_ok(const Plan& pl);
void build_lmmse_tcg_weights(const Plan& pl, std::vector<unsigned char>& out);
bool lmmse_tcg_ok(const Plan& pl, const float2* x, const float2* out);
cudaError_t launch_lmmse_tcg(const Plan& pl, const float2* x, const float2* pil, float2* out, cudaStream_t st);
size_t lmmse_tcg_stage_bytes(const Plan& pl);   // the 16-bit forms' staged operand (0: none)
cudaError_t prepare_lmmse_tcg(int device);

// Gram and matched filter on tcgen05 with 16-bit operands (precision form): G[t][k][s][c] =
// (H^H H + sigma2 I | H^H Y)[s][c] per (slot, subcarrier); needs 16-byte aligned h and y
// and even n_sc (TMA boxes).
bool gram_tc_ok(const Plan& pl, const void* h, const void* y);
cudaError_t launch_gram_tc(const Plan& pl, const float2* h, const float2* y, float2* G, bool fp16,
                           cudaStream_t st);
cudaError_t prepare_gram_tc(int device);

// Precision-form detection: the tensor-core Gram of 16-bit operands, its FP32 Cholesky and
// one FP32 refinement step with the residual from h (k_refine.cu); half-precision plans
// with gram_tc_ok inputs take it.
bool refine_ok(const Plan& pl, const void* h, const void* y);
cudaError_t launch_detect_refine(const Plan& pl, const float2* h, const float2* y, float2* x_eq,
                                 unsigned char* labels, float* llr, int* info, cudaStream_t st);
cudaError_t prepare_refine(int device);

cudaError_t launch_detect(const Plan& pl, const float2* h, const float2* y, float2* x_eq,
                          unsigned char* labels, float* llr, int* info, cudaStream_t st);

// Fused receive form: LS, LMMSE and detection in one kernel (orthogonal FP32 plans, even
// B <= 16, 16-byte aligned y_pilot and y_data); h_out may be null.
bool receive_fused_ok(const Plan& pl, const void* y_pilot, const void* y_data);
cudaError_t launch_receive_fused(const Plan& pl, const float2* y_pilot, const float2* pil, const float2* y_data,
                                 float2* h_out, float2* x_eq, unsigned char* labels, float* llr, int* info,
                                 cudaStream_t st);

// Plan-free launchers used by the allocation-free receive entry point.
cudaError_t launch_ls_lmmse_small_raw(const float2* w_main, const float2* w_tail, int B, int tail,
                                      int nb, int rows, int M, int N, const float2* y,
                                      const float2* pil, float2* out, int* status, cudaStream_t st);
cudaError_t launch_detect_raw(const DetTiles& tiles, int T, int K, int M, int N, int D, int q,
                              float sigma2, int* status, const float2* h, const float2* y,
                              float2* x_eq, unsigned char* labels, float* llr, int* info,
                              cudaStream_t st);

}  // namespace rapro
