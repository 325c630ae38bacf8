// Batched heterogeneous receive and the plan autotuner.
//
// The paper runs one slot per core, 18 slot threads at a time (Sec. III-B).  Here a batch of
// independent subframes of uneven shapes (each with its own plan) is spread over a pool of
// CUDA streams, longest jobs first onto the least loaded stream, forked from and joined
// back into the caller's stream with events, so that small jobs that fill only part of the
// GPU run side by side; the whole batch can be captured into one CUDA graph.  The
// autotuner times every estimator kernel that applies to a plan's shape (tensor cores,
// streaming, segment and tiled kernels) and the detector's warps-per-role split on the
// caller's arrays, and keeps the fastest in the plan.
#include <algorithm>
#include <cstdint>
#include <numeric>
#include <set>
#include <vector>

#include "rapro_internal.h"

using namespace rapro;

struct rapro_batch {
  int n = 0;
  int device = 0;
  cudaStream_t s[32] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[32] = {};
};

namespace {

rapro_status bad(const char* msg) {
  set_error(msg);
  return RAPRO_ERR_INVALID_ARG;
}

// Work estimate of one subframe: the estimator's filter MACs plus the detector's Gram and
// matched-filter MACs.
double job_work(const Plan& pl) {
  const rapro_params& p = pl.p;
  const double rows = double(pl.T) * p.K * p.M;
  const double est = rows * p.n_sc * (pl.comb ? 3.0 : double(std::max(1, pl.B)));
  const double det = double(pl.T) * p.n_sc * p.M * (p.K * (p.K + 1) / 2.0 + double(p.K) * pl.D);
  return est + det;
}

// Average time of fn on st over reps launches after warm launches (ms), or a negative
// value if a launch failed.
template <class F>
float time_on(cudaStream_t st, int warm, int reps, F fn) {
  for (int i = 0; i < warm; ++i)
    if (fn() != cudaSuccess) return -1.f;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess) return -1.f;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return -1.f;
  }
  float ms = -1.f;
  bool ok = cudaEventRecord(a, st) == cudaSuccess;
  for (int i = 0; ok && i < reps; ++i) ok = fn() == cudaSuccess;
  if (ok && cudaEventRecord(b, st) == cudaSuccess && cudaEventSynchronize(b) == cudaSuccess &&
      cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
    ms /= float(reps);
  else
    ms = -1.f;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms;
}

}  // namespace

extern "C" {

rapro_status rapro_plan_tune(rapro_plan* plan, const rapro_c32* y_pilot, const rapro_c32* pilots,
                             const rapro_c32* y_data, rapro_c32* h, rapro_c32* x_eq, rapro_stream stream) {
  if (!plan) return bad("plan is NULL");
  if (!y_pilot || !pilots || !y_data || !h || !x_eq) return bad("y_pilot, pilots, y_data, h and x_eq are required");
  Plan* pl = reinterpret_cast<Plan*>(plan);
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != pl->device) return bad("current device differs from the plan's device");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const float2* y = reinterpret_cast<const float2*>(y_pilot);
  const float2* pil = reinterpret_cast<const float2*>(pilots);
  const float2* yd = reinterpret_cast<const float2*>(y_data);
  float2* hh = reinterpret_cast<float2*>(h);
  float2* xx = reinterpret_cast<float2*>(x_eq);
  // Candidates run as whole receives with kInFlight copies in flight on streams of their own
  // (the same inputs and outputs: every copy writes the same values), so that the choice
  // is the one with the best throughput of pipelined subframes.  A BF16 plan's detectors
  // share the FP64-fallback list, so its copies run one at a time.
  constexpr int kWarm = 2, kReps = 5, kInFlight = 4;
  const int in_flight = pl->d_fix ? 1 : kInFlight;
  cudaStream_t side[kInFlight] = {};
  cudaEvent_t fork = nullptr, join[kInFlight] = {};
  auto cleanup = [&] {
    for (int i = 0; i < kInFlight; ++i) {
      if (side[i]) cudaStreamDestroy(side[i]);
      if (join[i]) cudaEventDestroy(join[i]);
    }
    if (fork) cudaEventDestroy(fork);
  };
  e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
  for (int i = 0; i < kInFlight && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "tuning streams");
  }
  // One round: every side stream runs `fn` once, forked from and joined into st.
  auto round = [&](auto fn) -> cudaError_t {
    cudaError_t r = cudaEventRecord(fork, st);
    for (int i = 0; i < in_flight && r == cudaSuccess; ++i) {
      r = cudaStreamWaitEvent(side[i], fork, 0);
      if (r == cudaSuccess) r = fn(side[i]);
      if (r == cudaSuccess) r = cudaEventRecord(join[i], side[i]);
      if (r == cudaSuccess) r = cudaStreamWaitEvent(st, join[i], 0);
    }
    return r;
  };
  auto receive_split = [&](cudaStream_t q) {
    cudaError_t r = pl->comb ? launch_comb(*pl, y, pil, hh, q)
                             : launch_lmmse(*pl, y, pil, pl->d_w_main, pl->d_w_tail, nullptr, nullptr, hh, q);
    return r != cudaSuccess ? r : launch_detect(*pl, hh, yd, xx, nullptr, nullptr, nullptr, q);
  };
  const int max_split = make_det_tiles(pl->p.K, pl->D).msplit;
  float best_ms = -1.f;
  int best_v = pl->est_variant, best_g = pl->est_ctas_per_sm, best_split = pl->tiles.msplit, best_form = RAPRO_RECV_SPLIT;
  auto consider = [&](int v, int g, int split, int form, float ms) {
    if (best_ms < 0.f || ms < best_ms) {
      best_ms = ms;
      best_v = v;
      best_g = g;
      best_split = split;
      best_form = form;
    }
  };
  rapro_status status = RAPRO_OK;
  for (int v = pl->comb ? -1 : 0; v < (pl->comb ? 0 : EST_VARIANTS) && status == RAPRO_OK; ++v) {
    if (v >= 0 && !lmmse_variant_ok(*pl, v, y, pil, hh)) continue;
    for (int g : {1, 0}) {
      if (g == 0 && v != EST_TC) continue;        // the grid choice concerns the tensor-core kernel
      for (int split = 1; split <= max_split; ++split) {
        pl->est_variant = v;
        pl->est_ctas_per_sm = g;
        pl->tiles.msplit = split;
        const float ms = time_on(st, kWarm, kReps, [&] { return round(receive_split); });
        if (ms < 0.f) {
          status = cuda_fail(cudaGetLastError(), "receive candidate during tuning");
          break;
        }
        consider(v, g, split, RAPRO_RECV_SPLIT, ms);
      }
    }
  }
  pl->recv_form = RAPRO_RECV_FUSED;
  const bool mode_fused = status == RAPRO_OK && receive_fused_ok(*pl, y_pilot, y_data);
  for (int split = 1; split <= max_split && mode_fused; ++split) {
    pl->tiles.msplit = split;
    const float ms = time_on(st, kWarm, kReps, [&] {
      return round([&](cudaStream_t q) {
        return launch_receive_fused(*pl, y, pil, yd, nullptr, xx, nullptr, nullptr, nullptr, q);
      });
    });
    if (ms < 0.f) {
      status = cuda_fail(cudaGetLastError(), "fused receive during tuning");
      break;
    }
    consider(best_v, best_g, split, RAPRO_RECV_FUSED, ms);
  }
  pl->est_variant = best_v;
  pl->est_ctas_per_sm = best_g;
  pl->tiles.msplit = best_split;
  pl->recv_form = best_form;
  if (status == RAPRO_OK) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) status = cuda_fail(e, "tuning");
  }
  cleanup();
  return status;
}

rapro_status rapro_plan_set_variant(rapro_plan* plan, int est_variant, int det_split, int est_ctas_per_sm) {
  if (!plan) return bad("plan is NULL");
  Plan* pl = reinterpret_cast<Plan*>(plan);
  if (est_variant < -1 || est_variant >= EST_VARIANTS) return bad("est_variant must be -1 .. 4");
  if (pl->comb && est_variant != -1) return bad("comb plans have one estimator (est_variant -1)");
  const int max_split = make_det_tiles(pl->p.K, pl->D).msplit;
  if (det_split < 1 || det_split > max_split) return bad("det_split out of range for this plan");
  if (est_ctas_per_sm < 0 || est_ctas_per_sm > 8) return bad("est_ctas_per_sm must be 0 .. 8");
  pl->est_variant = est_variant;
  pl->tiles.msplit = det_split;
  pl->est_ctas_per_sm = est_ctas_per_sm;
  return RAPRO_OK;
}

rapro_status rapro_plan_set_detector_form(rapro_plan* plan, int form) {
  if (!plan) return bad("plan is NULL");
  if (form != RAPRO_DET_REFINED && form != RAPRO_DET_FP32) return bad("form must be a rapro_detector_form");
  Plan* pl = reinterpret_cast<Plan*>(plan);
  if (!half_precision(pl->p)) {
    set_error("the detector form applies to RAPRO_PREC_BF16 and RAPRO_PREC_FP16 plans");
    return RAPRO_ERR_UNSUPPORTED;
  }
  pl->det_form = form;
  return RAPRO_OK;
}

rapro_status rapro_plan_set_wait_test(rapro_plan* plan, int stall_producer, uint32_t wait_rounds) {
  if (!plan) return bad("plan is NULL");
  Plan* pl = reinterpret_cast<Plan*>(plan);
  pl->stall_producer = stall_producer != 0;
  pl->wait_rounds = wait_rounds;
  return RAPRO_OK;
}

rapro_status rapro_plan_set_receive_form(rapro_plan* plan, int form) {
  if (!plan) return bad("plan is NULL");
  if (form != RAPRO_RECV_FUSED && form != RAPRO_RECV_SPLIT) return bad("form must be a rapro_receive_form");
  reinterpret_cast<Plan*>(plan)->recv_form = form;
  return RAPRO_OK;
}

rapro_status rapro_receive_is_fused(const rapro_plan* plan, const rapro_c32* y_pilot, const rapro_c32* y_data,
                                    int* fused) {
  if (!plan || !fused) return bad("plan and fused must not be NULL");
  const Plan* pl = reinterpret_cast<const Plan*>(plan);
  *fused = pl->recv_form == RAPRO_RECV_FUSED && receive_fused_ok(*pl, y_pilot, y_data) ? 1 : 0;
  return RAPRO_OK;
}

rapro_status rapro_plan_variant(const rapro_plan* plan, int* est_variant, int* det_split, int* est_ctas_per_sm) {
  if (!plan) return bad("plan is NULL");
  const Plan* pl = reinterpret_cast<const Plan*>(plan);
  if (est_variant) *est_variant = pl->est_variant;
  if (det_split) *det_split = pl->tiles.msplit;
  if (est_ctas_per_sm) *est_ctas_per_sm = pl->est_ctas_per_sm;
  return RAPRO_OK;
}

rapro_status rapro_batch_create(int n_streams, rapro_batch** out) {
  if (!out) return bad("out is NULL");
  *out = nullptr;
  if (n_streams < 1 || n_streams > 32) return bad("n_streams must be in [1, 32]");
  rapro_batch* b = new rapro_batch();
  cudaError_t e = cudaGetDevice(&b->device);
  auto fail = [&](const char* what) {
    for (int i = 0; i < b->n; ++i) {
      cudaStreamDestroy(b->s[i]);
      cudaEventDestroy(b->join[i]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    delete b;
    return cuda_fail(e, what);
  };
  if (e != cudaSuccess) return fail("cudaGetDevice");
  if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess) return fail("event");
  for (int i = 0; i < n_streams; ++i) {
    if ((e = cudaStreamCreateWithFlags(&b->s[i], cudaStreamNonBlocking)) != cudaSuccess) return fail("stream");
    if ((e = cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming)) != cudaSuccess) {
      cudaStreamDestroy(b->s[i]);
      return fail("event");
    }
    b->n = i + 1;
  }
  *out = b;
  return RAPRO_OK;
}

rapro_status rapro_batch_destroy(rapro_batch* b) {
  if (!b) return RAPRO_OK;
  cudaError_t e = cudaDeviceSynchronize();
  for (int i = 0; i < b->n; ++i) {
    cudaStreamDestroy(b->s[i]);
    cudaEventDestroy(b->join[i]);
  }
  cudaEventDestroy(b->fork);
  delete b;
  return e == cudaSuccess ? RAPRO_OK : cuda_fail(e, "rapro_batch_destroy");
}

rapro_status rapro_receive_batch(rapro_batch* b, const rapro_job* jobs, int n_jobs, rapro_stream stream) {
  if (!b) return bad("batch is NULL");
  if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return bad("jobs is NULL");
  if (n_jobs == 0) return RAPRO_OK;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev != b->device) return bad("current device differs from the batch's device");
  std::set<const rapro_plan*> workspace_users;
  std::vector<double> work(n_jobs);
  for (int i = 0; i < n_jobs; ++i) {
    const rapro_job& j = jobs[i];
    if (!j.plan || !j.y_pilot || !j.pilots || !j.y_data || !j.x_eq)
      return bad("every job needs plan, y_pilot, pilots, y_data and x_eq");
    if (!j.h_out && !workspace_users.insert(j.plan).second)
      return bad("jobs sharing a plan must pass h_out (the plan's workspace holds one estimate)");
    work[i] = job_work(*reinterpret_cast<const Plan*>(j.plan));
  }
  // Longest processing time first, each onto the stream with the least work so far.
  std::vector<int> order(n_jobs);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
  std::vector<double> load(b->n, 0.0);
  std::vector<int> where(n_jobs);
  for (int i : order) {
    const int k = int(std::min_element(load.begin(), load.end()) - load.begin());
    where[i] = k;
    load[k] += work[i];
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if ((e = cudaEventRecord(b->fork, st)) != cudaSuccess) return cuda_fail(e, "fork event");
  for (int k = 0; k < b->n; ++k)
    if ((e = cudaStreamWaitEvent(b->s[k], b->fork, 0)) != cudaSuccess) return cuda_fail(e, "fork wait");
  rapro_status s = RAPRO_OK;
  for (int i : order) {
    const rapro_job& j = jobs[i];
    s = receive_on(reinterpret_cast<const Plan*>(j.plan), j.y_pilot, j.pilots, j.y_data, j.h_out, j.x_eq, j.labels,
                   j.llr, j.info, b->s[where[i]]);
    if (s != RAPRO_OK) break;          // still join every stream back
  }
  for (int k = 0; k < b->n; ++k) {
    if ((e = cudaEventRecord(b->join[k], b->s[k])) != cudaSuccess) return cuda_fail(e, "join event");
    if ((e = cudaStreamWaitEvent(st, b->join[k], 0)) != cudaSuccess) return cuda_fail(e, "join wait");
  }
  return s;
}

}  // extern "C"
