// Precision form of the MMSE detector (Eq. 22): the solve of a Gram built from 16-bit
// operands, with one step of FP32 iterative refinement.
//
// Input: G[t][k] = (A_low | z_low) per (slot, subcarrier), the Gram H^H H + sigma2 I and the
// matched filter H^H Y formed on the tensor cores from BF16 or FP16 operands (k_gram_tc.cu).
// Per CTA tile (one slot, DET_SC subcarriers):
//  1. A_low = L L^H (FP32 Cholesky), columns of L^-1, s = sigma2 [A_low^-1]_kk, and
//     x0 = A_low^-1 z_low, one half-warp per subcarrier (the detector's factor/solve code);
//  2. the residual of Eq. 22 from the FP32 channel estimate, streamed through the same TMA
//     ring of 8-antenna chunks as the detector:  r = H^H (y - H x0) - sigma2 x0,
//     e = y - H x0 per (data symbol, antenna, subcarrier) first, then the users' sums;
//  3. x = x0 + A_low^-1 r with the same factor, then demap and store as the detector does.
// Subcarriers whose pivot ratio exceeds the precision form's limit (or whose FP32 factor
// fails) are re-solved in FP64 from h and y by the last CTA, as in the detector.
#include <algorithm>
#include <mutex>

#include "detect_kernel.cuh"

namespace rapro {

namespace {

constexpr int RF_CONS_WARPS = DET_SC / 2;        // one half-warp per subcarrier in the solves
constexpr int RF_CONS = RF_CONS_WARPS * 32;
constexpr int RF_THREADS = RF_CONS + 32;         // + the TMA warp

template <int KT, int DT>
constexpr size_t refine_smem_bytes() {
  const size_t stage = size_t(KT + DT) * DET_MCH * DET_SC * sizeof(float2);
  return 1024 + DET_STAGES * stage + det_off_park(KT, DT) * sizeof(float2) +
         size_t(DT) * DET_MCH * DET_SC * sizeof(float2);
}

}  // namespace

template <int KT, int DT>
__global__ void __launch_bounds__(RF_THREADS, 1)
    refine_kernel(const __grid_constant__ CUtensorMap map_h, const __grid_constant__ CUtensorMap map_y,
                  const float2* __restrict__ h, const float2* __restrict__ y, float2* __restrict__ x_eq,
                  unsigned char* __restrict__ labels, float* __restrict__ llr, int* __restrict__ info,
                  const __grid_constant__ DetParams P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + DET_STAGES;
  int* s_abort = reinterpret_cast<int*>(smem + 128);
  int* s_last = reinterpret_cast<int*>(smem + 136);
  float2* stage0 = reinterpret_cast<float2*>(smem + 1024);
  constexpr int PL = DET_MCH * DET_SC;
  constexpr int AS = KT + 1;
  constexpr int XS = DET_SC + 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x;
  const int t = blockIdx.y, k0 = blockIdx.x * DET_SC;
  const int K = P.K, D = P.D, N = P.N, C = P.K + P.D;
  const int yoff = KT * PL;                             // data rows within a stage
  const int stage_elems = (KT + DT) * PL;
  float2* ep = stage0 + size_t(DET_STAGES) * stage_elems;
  float2* As = ep;                                       // A_low, then L, then L^-1
  float2* Zs = ep + det_off_z(KT);                       // z_low, w, r, w
  float2* Xs = ep + det_off_x(KT, DT);                   // x0, then x
  float* Ss = reinterpret_cast<float*>(ep + det_off_s(KT, DT));
  int* Is = reinterpret_cast<int*>(Ss + KT * XS);
  float2* Cb = ep + det_off_col(KT, DT);
  float2* Es = ep + det_off_park(KT, DT);                // [DT][PL]: e = y - H x0 of a chunk
  const bool consumer = warp < RF_CONS_WARPS;

  if (tid == 0) {
    *s_abort = 0;
    for (int s = 0; s < DET_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], RF_CONS_WARPS);
    }
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == RF_CONS_WARPS) {
    // ------------------------------------------------ TMA warp: every antenna chunk
    if (lane == 0) {
      prefetch_tensormap(&map_h);
      prefetch_tensormap(&map_y);
      const uint32_t tx = uint32_t((K + D) * PL * sizeof(float2));
      int issued = 0;
      for (int c = 0; c < P.nchunks; ++c) {
        const int s = c % DET_STAGES;
        if (c >= DET_STAGES && !mbar_wait_bounded(&empty[s], uint32_t(c / DET_STAGES - 1) & 1u)) {
          atomicExch(s_abort, 1);
          break;
        }
        float2* st = stage0 + size_t(s) * stage_elems;
        mbar_arrive_expect_tx(&full[s], tx);
        tma_load_3d(st, &map_h, &full[s], k0, c * DET_MCH, t * K);
        tma_load_3d(st + yoff, &map_y, &full[s], k0, c * DET_MCH, t * D);
        ++issued;
      }
      // Every issued load lands before the CTA moves on (load j of stage s is phase j / DET_STAGES).
      for (int s = 0; s < DET_STAGES && s < issued; ++s)
        (void)mbar_wait_bounded(&full[s], uint32_t((issued - 1 - s) / DET_STAGES) & 1u);
    }
    __syncwarp();
  } else {
    // ------------------------------------------------ 1. factor A_low, x0 = A_low^-1 z_low
    const float2* G = P.gram + (size_t(t) * N + k0) * K * C;
    for (int e = tid; e < DET_SC * K * C; e += RF_CONS) {
      const int sc = e / (K * C), rem = e - sc * K * C, i = rem / C, c = rem - i * C;
      const bool in = k0 + sc < N;
      const float2 v = in ? G[e] : make_float2(c == i ? 1.f : 0.f, 0.f);   // identity past n_sc
      if (c < K) As[(sc * KT + i) * AS + c] = v;
      else Zs[(sc * KT + i) * DT + (c - K)] = in ? v : make_float2(0.f, 0.f);
    }
    named_bar_sync(1, RF_CONS);
    const int hw = lane >> 4, i = lane & 15, scl = warp * 2 + hw;
    det_factor_solve<KT, DT, true>(i, scl, K, D, t, k0, N, P, As, Zs, Xs, Ss, Is, Cb);
    named_bar_sync(1, RF_CONS);

    // ------------------------------------------------ 2. r = H^H (y - H x0) - sigma2 x0
    // e = y - H x0: thread (subcarrier, antenna of the chunk, half of the symbols); its x0
    // values stay in registers across chunks when they fit.
    constexpr int NB1 = DT / 2;
    constexpr bool CACHE = KT * NB1 <= 36;
    const int e_sc = tid & (DET_SC - 1), e_m = (tid >> 4) & (DET_MCH - 1), e_n0 = (tid >> 7) * NB1;
    float2 xc[CACHE ? KT : 1][CACHE ? NB1 : 1];
    if constexpr (CACHE) {
#pragma unroll
      for (int k = 0; k < KT; ++k)
#pragma unroll
        for (int j = 0; j < NB1; ++j)
          xc[k][j] = (k < K && e_n0 + j < D) ? Xs[((e_n0 + j) * KT + k) * XS + e_sc] : make_float2(0.f, 0.f);
    }
    // r += H^H e: thread pair (subcarrier, 4 users, 3 symbols), one thread per half of the
    // chunk's antennas; the halves meet by a shuffle at the end.
    constexpr int KG = KT / 4, NG2 = DT / 3, COMBOS = DET_SC * KG * NG2;
    constexpr int CPT = (COMBOS + RF_CONS / 2 - 1) / (RF_CONS / 2);
    const int mh = tid & 1, pair = tid >> 1;
    float2 racc[CPT][4][3];
#pragma unroll
    for (int u = 0; u < CPT; ++u)
#pragma unroll
      for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
        for (int j = 0; j < 3; ++j) racc[u][a2][j] = make_float2(0.f, 0.f);
    bool aborted = false;
    for (int c = 0; c < P.nchunks; ++c) {
      const int s = c % DET_STAGES;
      // Every consumer warp passes both barriers of every chunk; a wait that ran out marks
      // the CTA aborted instead of leaving the loop.
      bool ok = !aborted && !*reinterpret_cast<volatile int*>(s_abort) &&
                mbar_wait_bounded(&full[s], uint32_t(c / DET_STAGES) & 1u);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) {
        if (!aborted && lane == 0) atomicExch(s_abort, 1);
        aborted = true;
      }
      const float2* st = stage0 + size_t(s) * stage_elems;
      if (!aborted) {
        const int rem = e_m * DET_SC + e_sc;
        float2 hv[KT];
#pragma unroll
        for (int k = 0; k < KT; ++k) hv[k] = k < K ? st[k * PL + rem] : make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < NB1; ++j) {
          const int n = e_n0 + j;
          if (n < D) {
            float2 e = st[yoff + n * PL + rem];
#pragma unroll
            for (int k = 0; k < KT; ++k) {
              if (k < K) {
                const float2 xv = CACHE ? xc[CACHE ? k : 0][CACHE ? j : 0] : Xs[(n * KT + k) * XS + e_sc];
                e.x -= hv[k].x * xv.x - hv[k].y * xv.y;
                e.y -= hv[k].x * xv.y + hv[k].y * xv.x;
              }
            }
            Es[n * PL + rem] = e;
          }
        }
      }
      named_bar_sync(1, RF_CONS);
      if (!aborted) {
#pragma unroll
        for (int u = 0; u < CPT; ++u) {
          const int cmb = pair + u * (RF_CONS / 2);
          if (cmb < COMBOS) {
            const int sc = cmb & (DET_SC - 1), kg = (cmb >> 4) % KG, ng = (cmb >> 4) / KG;
#pragma unroll
            for (int mm = 0; mm < DET_MCH / 2; ++mm) {
              const int rem = (mh * (DET_MCH / 2) + mm) * DET_SC + sc;
              float2 hv[4], ev[3];
#pragma unroll
              for (int a2 = 0; a2 < 4; ++a2)
                hv[a2] = 4 * kg + a2 < K ? st[(4 * kg + a2) * PL + rem] : make_float2(0.f, 0.f);
#pragma unroll
              for (int j = 0; j < 3; ++j) ev[j] = 3 * ng + j < D ? Es[(3 * ng + j) * PL + rem] : make_float2(0.f, 0.f);
#pragma unroll
              for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
                for (int j = 0; j < 3; ++j) cmac_conj(racc[u][a2][j], hv[a2], ev[j]);
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0 && !aborted) mbar_arrive(&empty[s]);
      named_bar_sync(1, RF_CONS);
    }
    // ------------------------------------------------ 3. x = x0 + A_low^-1 r
#pragma unroll
    for (int u = 0; u < CPT; ++u)
#pragma unroll
      for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          racc[u][a2][j].x += __shfl_xor_sync(0xffffffffu, racc[u][a2][j].x, 1);
          racc[u][a2][j].y += __shfl_xor_sync(0xffffffffu, racc[u][a2][j].y, 1);
        }
    if (!aborted && mh == 0) {
#pragma unroll
      for (int u = 0; u < CPT; ++u) {
        const int cmb = pair + u * (RF_CONS / 2);
        if (cmb < COMBOS) {
          const int sc = cmb & (DET_SC - 1), kg = (cmb >> 4) % KG, ng = (cmb >> 4) / KG;
#pragma unroll
          for (int a2 = 0; a2 < 4; ++a2)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
              const int k = 4 * kg + a2, n = 3 * ng + j;
              if (k < K && n < D) {
                const float2 xv = Xs[(n * KT + k) * XS + sc];
                Zs[(sc * KT + k) * DT + n] =
                    make_float2(racc[u][a2][j].x - P.sigma2 * xv.x, racc[u][a2][j].y - P.sigma2 * xv.y);
              }
            }
        }
      }
    }
    named_bar_sync(1, RF_CONS);
    if (!aborted) det_solve_add<KT, DT>(i, scl, K, D, As, Zs, Xs);
  }

  // FP64 fallback: every CTA counts itself done; the last one re-solves the flagged
  // subcarriers (process) and clears the list for the next launch.
  auto finish_fix = [&](bool process) {
    if (!P.fix_count) return;
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      *s_last = atomicAdd(P.fix_ticket, 1) == int(gridDim.x * gridDim.y) - 1;
    }
    __syncthreads();
    if (!*s_last) return;
    __threadfence();
    if (process) {
      const FixArgs fa{h, y, x_eq, labels, llr, info, P.fix_count, P.fix_list, P.fix_cap,
                       P.T, K, P.M, N, D, P.q, P.sigma2_d};
      fp64_fix_items(fa, reinterpret_cast<FixScratch*>(stage0));
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      *P.fix_count = 0;
      *P.fix_ticket = 0;
      __threadfence();
    }
  };
  __syncthreads();
  if (*s_abort) {
    if (threadIdx.x == 0) atomicExch(P.status, int(RAPRO_ERR_TIMEOUT));
    finish_fix(false);
    return;
  }
  det_demap_store<KT, DT>(t, k0, K, D, N, P.q, Xs, Ss, x_eq, labels, llr);
  if (info && threadIdx.x < DET_SC && k0 + threadIdx.x < N) info[size_t(t) * N + k0 + threadIdx.x] = Is[threadIdx.x];
  finish_fix(true);
}

namespace {

template <int KT, int DT>
cudaError_t refine_go(const DetParams& P, const CUtensorMap& mh, const CUtensorMap& my, const float2* h,
                      const float2* y, float2* x_eq, unsigned char* labels, float* llr, int* info, cudaStream_t st) {
  const dim3 grid((P.N + DET_SC - 1) / DET_SC, P.T), block(RF_THREADS);
  refine_kernel<KT, DT><<<grid, block, refine_smem_bytes<KT, DT>(), st>>>(mh, my, h, y, x_eq, labels, llr, info, P);
  return cudaGetLastError();
}

template <int KT>
cudaError_t refine_kt(const DetParams& P, const CUtensorMap& mh, const CUtensorMap& my, const float2* h,
                      const float2* y, float2* x_eq, unsigned char* labels, float* llr, int* info, cudaStream_t st) {
  if (P.D > 6) return refine_go<KT, 12>(P, mh, my, h, y, x_eq, labels, llr, info, st);
  return refine_go<KT, 6>(P, mh, my, h, y, x_eq, labels, llr, info, st);
}

template <int KT>
cudaError_t refine_prepare_kt() {
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(refine_kernel<KT, 6>, A, int(refine_smem_bytes<KT, 6>()));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(refine_kernel<KT, 12>, A, int(refine_smem_bytes<KT, 12>()));
  return e;
}

static_assert(refine_smem_bytes<16, 12>() <= 232448, "the refine kernel's largest tile fits in shared memory");
static_assert(RF_CONS == 256 && DET_SC == 16 && DET_MCH == 8, "the residual's thread maps assume 256 consumers, 16 x 8 tiles");

}  // namespace

bool refine_ok(const Plan& pl, const void* h, const void* y) {
  return pl.d_gram && !pl.comb && gram_tc_ok(pl, h, y);
}

cudaError_t launch_detect_refine(const Plan& pl, const float2* h, const float2* y, float2* x_eq,
                                 unsigned char* labels, float* llr, int* info, cudaStream_t st) {
  cudaError_t e = launch_gram_tc(pl, h, y, pl.d_gram, pl.p.precision == RAPRO_PREC_FP16, st);
  if (e != cudaSuccess) return e;
  DetParams P{};
  P.T = pl.T; P.K = pl.p.K; P.M = pl.p.M; P.N = pl.p.n_sc; P.D = pl.D; P.q = pl.q;
  P.sigma2 = float(pl.p.sigma2);
  P.nchunks = (pl.p.M + DET_MCH - 1) / DET_MCH;
  P.status = pl.d_status;
  P.gram = pl.d_gram;
  P.fix_count = pl.d_fix;
  P.fix_ticket = pl.d_fix + 1;
  P.fix_list = pl.d_fix + 2;
  P.fix_cap = pl.T * pl.p.n_sc;
  P.cond_limit = kFp64CondLimit;
  P.sigma2_d = pl.p.sigma2;
  CUtensorMap mh, my;
  if (!encode_cx_map(&mh, h, P.N, P.M, P.T * P.K, P.K, DET_SC) ||
      !encode_cx_map(&my, y, P.N, P.M, P.T * P.D, P.D, DET_SC))
    return cudaErrorInvalidValue;
  const int K = P.K;
  if (K <= 4) return refine_kt<4>(P, mh, my, h, y, x_eq, labels, llr, info, st);
  if (K <= 8) return refine_kt<8>(P, mh, my, h, y, x_eq, labels, llr, info, st);
  if (K <= 12) return refine_kt<12>(P, mh, my, h, y, x_eq, labels, llr, info, st);
  return refine_kt<16>(P, mh, my, h, y, x_eq, labels, llr, info, st);
}

cudaError_t prepare_refine(int device) {
  static std::once_flag flags[64];
  static cudaError_t result[64];
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  std::call_once(flags[device], [device] {
    cudaError_t e = refine_prepare_kt<4>();
    if (e == cudaSuccess) e = refine_prepare_kt<8>();
    if (e == cudaSuccess) e = refine_prepare_kt<12>();
    if (e == cudaSuccess) e = refine_prepare_kt<16>();
    result[device] = e;
  });
  return result[device];
}

}  // namespace rapro
