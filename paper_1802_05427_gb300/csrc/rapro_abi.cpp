// extern "C" entry points: argument checks, then the kernel launchers.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "rapro_internal.h"

using namespace rapro;

namespace {

rapro_status bad(const char* msg) {
  set_error(msg);
  return RAPRO_ERR_INVALID_ARG;
}

// The plan's weights live on the device that was current at rapro_plan_create.
rapro_status check_device(const Plan* pl) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != pl->device) return bad("current device differs from the plan's device");
  return RAPRO_OK;
}

rapro_status launched(cudaError_t e, const char* what) {
  return e == cudaSuccess ? RAPRO_OK : cuda_fail(e, what);
}

rapro_status orthogonal_only(const Plan* pl) {
  if (!pl->comb) return RAPRO_OK;
  set_error("this estimator reads the orthogonal pilot layout; comb plans use rapro_ce_comb");
  return RAPRO_ERR_UNSUPPORTED;
}

// The BF16 / FP16 forms run only on the tensor-core estimator: LS fused, the plan's
// weights, aligned arrays.
rapro_status bf16_check(const Plan* pl, const void* y, const void* pil, const void* h, const void* w_override) {
  if (!half_precision(pl->p)) return RAPRO_OK;
  if (!pil || w_override) {
    set_error("the BF16 / FP16 forms need the fused LS (pilots) and the plan's weights");
    return RAPRO_ERR_UNSUPPORTED;
  }
  const uintptr_t a = reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(pil) |
                      reinterpret_cast<uintptr_t>(h);
  if (a & 15) {
    set_error("the BF16 / FP16 forms need 16-byte aligned y_pilot, pilots and h");
    return RAPRO_ERR_INVALID_ARG;
  }
  return RAPRO_OK;
}

inline const float2* f2(const rapro_c32* p) { return reinterpret_cast<const float2*>(p); }
inline float2* f2(rapro_c32* p) { return reinterpret_cast<float2*>(p); }
inline cudaStream_t cs(rapro_stream s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

namespace rapro {

// One subframe through the estimator and the detector on stream st (rapro_receive_subframe).
rapro_status receive_on(const Plan* pl, const rapro_c32* y_pilot, const rapro_c32* pilots, const rapro_c32* y_data,
                        rapro_c32* h_out, rapro_c32* x_eq, uint8_t* labels, float* llr, int32_t* info,
                        cudaStream_t st) {
  if (!y_pilot || !pilots || !y_data || !x_eq)
    return bad("y_pilot, pilots, y_data and x_eq must not be NULL");
  rapro_status s = check_device(pl);
  if (s != RAPRO_OK) return s;
  if (pl->recv_form == RAPRO_RECV_FUSED && receive_fused_ok(*pl, y_pilot, y_data))
    return launched(launch_receive_fused(*pl, f2(y_pilot), f2(pilots), f2(y_data), h_out ? f2(h_out) : nullptr,
                                         f2(x_eq), labels, llr, info, st),
                    "fused receive kernel launch");
  float2* h = h_out ? f2(h_out) : pl->d_h_work;
  if ((s = bf16_check(pl, y_pilot, pilots, h, nullptr)) != RAPRO_OK) return s;
  cudaError_t e = pl->comb ? launch_comb(*pl, f2(y_pilot), f2(pilots), h, st)
                           : launch_lmmse(*pl, f2(y_pilot), f2(pilots), pl->d_w_main, pl->d_w_tail,
                                          pl->w_main.data(), pl->w_tail.data(), h, st);
  if (e != cudaSuccess) return cuda_fail(e, "channel estimator launch");
  return launched(launch_detect(*pl, h, f2(y_data), f2(x_eq), labels, llr, info, st), "detection kernel launch");
}

}  // namespace rapro

extern "C" {

rapro_status rapro_ce_ls(const rapro_plan* plan, const rapro_c32* y_pilot, const rapro_c32* pilots,
                         rapro_c32* h_ls, rapro_stream stream) {
  if (!plan) return bad("plan is NULL");
  if (!y_pilot || !pilots || !h_ls) return bad("y_pilot, pilots and h_ls must not be NULL");
  const Plan* pl = reinterpret_cast<const Plan*>(plan);
  rapro_status s = check_device(pl);
  if (s == RAPRO_OK) s = orthogonal_only(pl);
  if (s != RAPRO_OK) return s;
  return launched(launch_ls(f2(y_pilot), f2(pilots), f2(h_ls), pl->T, pl->p.K, pl->p.M, pl->p.n_sc, cs(stream)),
                  "LS kernel launch");
}

rapro_status rapro_ce_lmmse_subblock(const rapro_plan* plan, const rapro_c32* h_ls,
                                     const rapro_c32* w_override, rapro_c32* h, rapro_stream stream) {
  if (!plan) return bad("plan is NULL");
  if (!h_ls || !h) return bad("h_ls and h must not be NULL");
  if (f2(h_ls) == f2(h)) return bad("h must not alias h_ls");
  const Plan* pl = reinterpret_cast<const Plan*>(plan);
  rapro_status s = check_device(pl);
  if (s == RAPRO_OK) s = orthogonal_only(pl);
  if (s == RAPRO_OK) s = bf16_check(pl, h_ls, nullptr, h, w_override);
  if (s != RAPRO_OK) return s;
  const float2* w = w_override ? f2(w_override) : pl->d_w_main;
  return launched(launch_lmmse(*pl, f2(h_ls), nullptr, w, pl->d_w_tail, pl->w_main.data(),
                               pl->w_tail.data(), f2(h), cs(stream)),
                  "LMMSE kernel launch");
}

rapro_status rapro_ce_ls_lmmse(const rapro_plan* plan, const rapro_c32* y_pilot, const rapro_c32* pilots,
                               const rapro_c32* w_override, rapro_c32* h, rapro_stream stream) {
  if (!plan) return bad("plan is NULL");
  if (!y_pilot || !pilots || !h) return bad("y_pilot, pilots and h must not be NULL");
  if (f2(y_pilot) == f2(h)) return bad("h must not alias y_pilot");
  const Plan* pl = reinterpret_cast<const Plan*>(plan);
  rapro_status s = check_device(pl);
  if (s == RAPRO_OK) s = orthogonal_only(pl);
  if (s == RAPRO_OK) s = bf16_check(pl, y_pilot, pilots, h, w_override);
  if (s != RAPRO_OK) return s;
  const float2* w = w_override ? f2(w_override) : pl->d_w_main;
  return launched(launch_lmmse(*pl, f2(y_pilot), f2(pilots), w, pl->d_w_tail, pl->w_main.data(),
                               pl->w_tail.data(), f2(h), cs(stream)),
                  "LS+LMMSE kernel launch");
}

rapro_status rapro_ce_comb(const rapro_plan* plan, const rapro_c32* y_pilot, const rapro_c32* pilots,
                           rapro_c32* h, rapro_stream stream) {
  if (!plan) return bad("plan is NULL");
  if (!y_pilot || !pilots || !h) return bad("y_pilot, pilots and h must not be NULL");
  const Plan* pl = reinterpret_cast<const Plan*>(plan);
  rapro_status s = check_device(pl);
  if (s != RAPRO_OK) return s;
  if (!pl->comb) {
    set_error("rapro_ce_comb needs a plan with pilot_layout == RAPRO_PILOT_COMB");
    return RAPRO_ERR_UNSUPPORTED;
  }
  return launched(launch_comb(*pl, f2(y_pilot), f2(pilots), f2(h), cs(stream)), "comb estimator launch");
}

rapro_status rapro_mmse_detect(const rapro_plan* plan, const rapro_c32* h, const rapro_c32* y_data,
                               rapro_c32* x_eq, uint8_t* labels, float* llr, int32_t* info,
                               rapro_stream stream) {
  if (!plan) return bad("plan is NULL");
  if (!h || !y_data || !x_eq) return bad("h, y_data and x_eq must not be NULL");
  const Plan* pl = reinterpret_cast<const Plan*>(plan);
  rapro_status s = check_device(pl);
  if (s != RAPRO_OK) return s;
  return launched(launch_detect(*pl, f2(h), f2(y_data), f2(x_eq), labels, llr, info, cs(stream)),
                  "detection kernel launch");
}

rapro_status rapro_gram_tc(const rapro_plan* plan, const rapro_c32* h, const rapro_c32* y_data, rapro_c32* gram,
                           int fp16, rapro_stream stream) {
  if (!plan) return bad("plan is NULL");
  if (!h || !y_data || !gram) return bad("h, y_data and gram must not be NULL");
  const Plan* pl = reinterpret_cast<const Plan*>(plan);
  rapro_status s = check_device(pl);
  if (s == RAPRO_OK) s = orthogonal_only(pl);
  if (s != RAPRO_OK) return s;
  if (!gram_tc_ok(*pl, h, y_data)) {
    set_error("the tensor-core Gram needs 16-byte aligned h and y_data and an even n_sc");
    return RAPRO_ERR_UNSUPPORTED;
  }
  return launched(launch_gram_tc(*pl, f2(h), f2(y_data), f2(gram), fp16 != 0, cs(stream)),
                  "tensor-core Gram kernel launch");
}

rapro_status rapro_receive_subframe(const rapro_plan* plan, const rapro_c32* y_pilot,
                                    const rapro_c32* pilots, const rapro_c32* y_data,
                                    rapro_c32* h_out, rapro_c32* x_eq, uint8_t* labels, float* llr,
                                    int32_t* info, rapro_stream stream) {
  if (!plan) return bad("plan is NULL");
  return receive_on(reinterpret_cast<const Plan*>(plan), y_pilot, pilots, y_data, h_out, x_eq, labels, llr, info,
                    cs(stream));
}

rapro_status rapro_mse_backward(const rapro_plan* plan, const rapro_c32* y_pilot, const rapro_c32* pilots,
                                const rapro_c32* y_data, const rapro_c32* h, const rapro_c32* x_eq,
                                const rapro_c32* x_ref, rapro_c32* g_h, float* scalars, rapro_c32* g_w_main,
                                rapro_c32* g_w_tail, rapro_stream stream) {
  if (!plan) return bad("plan is NULL");
  const Plan* pl = reinterpret_cast<const Plan*>(plan);
  if (!y_pilot || !pilots || !y_data || !h || !x_eq || !x_ref || !g_h || !scalars || !g_w_main ||
      (pl->tail && !g_w_tail))
    return bad("every array except g_w_tail (when B divides n_sc) is required");
  const void* g = g_h;
  if (g == y_pilot || g == y_data || g == h || g == x_eq || g == x_ref) return bad("g_h must not alias an input");
  rapro_status s = check_device(pl);
  if (s == RAPRO_OK) s = orthogonal_only(pl);
  if (s != RAPRO_OK) return s;
  if (pl->B > adjoint_max_block() || pl->p.n_sc > adjoint_max_subcarriers()) {
    set_error("the adjoint supports subblock <= 64 and n_sc <= 2048");
    return RAPRO_ERR_UNSUPPORTED;
  }
  return launched(launch_adjoint(*pl, f2(y_pilot), f2(pilots), f2(y_data), f2(h), f2(x_eq), f2(x_ref), f2(g_h),
                                 scalars, f2(g_w_main), f2(g_w_tail), cs(stream)),
                  "adjoint launch");
}

}  // extern "C"
