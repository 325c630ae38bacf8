// Host side of the MMSE detector: TMA tensor maps, padded-user-count dispatch, set-up.
#include <algorithm>
#include <mutex>

#include "detect_kernel.cuh"

namespace rapro {

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 3-D map over complex64 data [depth][M][N] with boxes of box_x x DET_MCH x box_z.
bool encode_cx_map(CUtensorMap* m, const void* base, int N, int M, int depth, int box_z, int box_x) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[3] = {cuuint64_t(N), cuuint64_t(M), cuuint64_t(depth)};
  cuuint64_t strides[2] = {cuuint64_t(N) * 8, cuuint64_t(N) * M * 8};
  cuuint32_t box[3] = {cuuint32_t(box_x), cuuint32_t(DET_MCH), cuuint32_t(box_z)};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static bool encode_map(CUtensorMap* m, const void* base, int N, int M, int depth, int box_z,
                       int box_x = DET_SC) {
  return encode_cx_map(m, base, N, M, depth, box_z, box_x);
}

static int padded_users(int K) { return K <= 4 ? 4 : K <= 8 ? 8 : K <= 12 ? 12 : 16; }

static size_t smem_bytes(const DetTiles& t, int K, int D, bool tma) {
  const int KT = padded_users(K), DT = D > 6 ? 12 : 6;
  return 1024 + std::max(det_stage_bytes(t) * (tma ? DET_STAGES : 1),
                         det_epilogue_bytes(KT, DT) + det_scratch_bytes(KT, DT));
}

// Largest dynamic shared memory of one CTA on sm_103a (227 KB).
constexpr size_t kSmemOptin = 232448;

// Fused receive form: the pilot box of a tile starts at its first block and must reach the
// end of its last one (full length assumed for a tail block too, its extra weights being
// zero); rows of the box whose width is a multiple of 16 subcarriers would put adjacent
// rows on the same banks, so such a width grows by 2 when n_sc allows.
static int fused_span(int N, int B) {
  int span = 0;
  for (int k0 = 0; k0 < N; k0 += DET_SC) {
    const int x0 = (k0 / B) * B, last = std::min(N, k0 + DET_SC) - 1;
    span = std::max(span, (last / B) * B + B - x0);
  }
  if (span % 16 == 0 && span + 2 <= N) span += 2;
  return span;
}

static size_t fused_smem_bytes(const DetTiles& t, int K, int D, int span, int nst) {
  const int KT = padded_users(K), DT = D > 6 ? 12 : 6;
  return 1024 + std::max(fused_work_bytes(t, K, span, nst), det_epilogue_bytes(KT, DT) + det_scratch_bytes(KT, DT));
}

// Shape rules of the fused form (array alignment is checked per call): orthogonal pilots,
// the FP32 filter, an even block of at most 16 subcarriers, even n_sc, and a pilot box
// that fits (span <= n_sc, at least two stages in shared memory).
static bool fused_shape(const Plan& pl, int* span_out, int* nst_out) {
  const int B = pl.B, N = pl.p.n_sc;
  if (pl.comb || pl.p.precision != RAPRO_PREC_FP32 || B < 2 || B > 16 || (B & 1) || (N & 1)) return false;
  const int span = fused_span(N, B);
  if (span > N || span > 64) return false;
  int nst = DET_STAGES;
  while (nst >= 2 && fused_smem_bytes(pl.tiles, pl.p.K, pl.D, span, nst) > kSmemOptin) --nst;
  if (nst < 2) return false;
  if (span_out) *span_out = span;
  if (nst_out) *nst_out = nst;
  return true;
}

bool receive_fused_ok(const Plan& pl, const void* y_pilot, const void* y_data) {
  const bool aligned = ((reinterpret_cast<uintptr_t>(y_pilot) | reinterpret_cast<uintptr_t>(y_data)) & 15) == 0;
  return aligned && fused_shape(pl, nullptr, nullptr);
}

static cudaError_t dispatch(DetLaunch& L) {
  switch (padded_users(L.P.K)) {
    case 4: return detect_launch_kt<4>(L);
    case 8: return detect_launch_kt<8>(L);
    case 12: return detect_launch_kt<12>(L);
    default: return detect_launch_kt<16>(L);
  }
}

static cudaError_t run(DetParams P, const float2* h, const float2* y, float2* x_eq, unsigned char* labels,
                       float* llr, int* info, cudaStream_t st) {
  DetLaunch L{};
  L.h = h; L.y = y; L.x_eq = x_eq; L.labels = labels; L.llr = llr; L.info = info;
  L.P = P;
  L.stream = st;
  const bool aligned = ((reinterpret_cast<uintptr_t>(h) | reinterpret_cast<uintptr_t>(y)) & 15) == 0;
  L.tma = aligned && (P.N % 2 == 0) && encode_map(&L.map_h, h, P.N, P.M, P.T * P.K, P.K) &&
          encode_map(&L.map_y, y, P.N, P.M, P.T * P.D, P.D);
  L.smem = smem_bytes(P.tiles, P.K, P.D, L.tma);
  return dispatch(L);
}

cudaError_t launch_detect(const Plan& pl, const float2* h, const float2* y, float2* x_eq,
                          unsigned char* labels, float* llr, int* info, cudaStream_t st) {
  // Precision form: Gram on the tensor cores, one FP32 refinement step (shape rules of the
  // tensor-core Gram; other inputs take the FP32 detector with the FP64 fallback).
  if (half_precision(pl.p) && pl.det_form == RAPRO_DET_REFINED && refine_ok(pl, h, y))
    return launch_detect_refine(pl, h, y, x_eq, labels, llr, info, st);
  DetParams P{};
  P.T = pl.T; P.K = pl.p.K; P.M = pl.p.M; P.N = pl.p.n_sc; P.D = pl.D; P.q = pl.q;
  P.sigma2 = float(pl.p.sigma2);
  P.nchunks = (pl.p.M + DET_MCH - 1) / DET_MCH;
  P.tiles = pl.tiles;
  P.status = pl.d_status;
  P.wait_rounds = pl.wait_rounds;
  P.stall_producer = pl.stall_producer;
  if (pl.d_fix) {                       // [0] count, [1] ticket (both reset by the kernel), [2..] list
    P.fix_count = pl.d_fix;
    P.fix_ticket = pl.d_fix + 1;
    P.fix_list = pl.d_fix + 2;
    P.fix_cap = pl.T * pl.p.n_sc;
    P.cond_limit = kFp64CondLimit;
    P.sigma2_d = pl.p.sigma2;
  }
  return run(P, h, y, x_eq, labels, llr, info, st);
}

// The whole subframe in one launch (fused form); the caller has checked receive_fused_ok.
cudaError_t launch_receive_fused(const Plan& pl, const float2* y_pilot, const float2* pil, const float2* y_data,
                                 float2* h_out, float2* x_eq, unsigned char* labels, float* llr, int* info,
                                 cudaStream_t st) {
  int span = 0, nst = 0;
  if (!fused_shape(pl, &span, &nst)) return cudaErrorNotSupported;
  DetLaunch L{};
  DetParams& P = L.P;
  P.T = pl.T; P.K = pl.p.K; P.M = pl.p.M; P.N = pl.p.n_sc; P.D = pl.D; P.q = pl.q;
  P.sigma2 = float(pl.p.sigma2);
  P.nchunks = (pl.p.M + DET_MCH - 1) / DET_MCH;
  P.tiles = pl.tiles;
  P.status = pl.d_status;
  P.pil = pil;
  P.w_main = pl.d_w_main;
  P.w_tail = pl.d_w_tail;
  P.h_out = h_out;
  P.B = pl.B;
  P.nfull = pl.p.n_sc / pl.B;
  P.tail = pl.tail;
  P.span = span;
  P.nst = nst;
  L.y = y_data; L.x_eq = x_eq; L.labels = labels; L.llr = llr; L.info = info;
  L.stream = st;
  L.tma = true;
  L.fused = true;
  if (!encode_map(&L.map_h, y_pilot, P.N, P.M, P.T * P.K, P.K, span) ||
      !encode_map(&L.map_y, y_data, P.N, P.M, P.T * P.D, P.D))
    return cudaErrorInvalidValue;
  L.smem = fused_smem_bytes(P.tiles, P.K, P.D, span, nst);
  return dispatch(L);
}

// Detection without a plan (same kernels): used by the allocation-free receive entry point.
cudaError_t launch_detect_raw(const DetTiles& tiles, int T, int K, int M, int N, int D, int q,
                              float sigma2, int* status, const float2* h, const float2* y,
                              float2* x_eq, unsigned char* labels, float* llr, int* info,
                              cudaStream_t st) {
  DetParams P{};
  P.T = T; P.K = K; P.M = M; P.N = N; P.D = D; P.q = q;
  P.sigma2 = sigma2;
  P.nchunks = (M + DET_MCH - 1) / DET_MCH;
  P.tiles = tiles;
  P.status = status;
  P.skip_if_set = status;               // the estimator before it timed out: leave the outputs
  return run(P, h, y, x_eq, labels, llr, info, st);
}

// Raise the detectors' dynamic shared-memory limit once per device, at plan creation
// (not at launch, which may be inside a CUDA-graph capture).
cudaError_t prepare_detect(int device) {
  static std::once_flag flags[64];
  static cudaError_t result[64];
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  std::call_once(flags[device], [device] {
    DetTiles worst = make_det_tiles(RAPRO_MAX_USERS, RAPRO_MAX_DATA_PER_SLOT);
    const int smem = int(std::max(smem_bytes(worst, RAPRO_MAX_USERS, RAPRO_MAX_DATA_PER_SLOT, true),
                                  smem_bytes(worst, RAPRO_MAX_USERS, RAPRO_MAX_DATA_PER_SLOT, false)));
    const int fsmem = int(kSmemOptin);
    cudaError_t e = detect_prepare_kt<4>(smem, fsmem);
    if (e == cudaSuccess) e = detect_prepare_kt<8>(smem, fsmem);
    if (e == cudaSuccess) e = detect_prepare_kt<12>(smem, fsmem);
    if (e == cudaSuccess) e = detect_prepare_kt<16>(smem, fsmem);
    result[device] = e;
  });
  return result[device];
}

}  // namespace rapro
