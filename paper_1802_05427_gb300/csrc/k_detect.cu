// MMSE detection (Eq. 20-22) with Cholesky (A = L L^H, uplo = L) and Gray-QAM demapping.
//
// One CTA owns DET_SC consecutive subcarriers of one slot.  The channel estimate
// h[t][s][m][k] and the slot's data symbols y[t*D+n][m][k] stream through shared memory
// DET_MCH antennas at a time (TMA boxes of 16 subcarriers x 8 antennas x K users / D
// symbols, a DET_STAGES-deep mbarrier pipeline).  Each warp owns one 4 x 6 tile of the
// augmented product [H | y]^H-row-block x [H | y]: Gram entries A[i][j] = sum_m conj(h_i) h_j
// and matched-filter entries z[i][n] = sum_m conj(h_i) y_n; lanes 0-15 and 16-31 take
// alternate antenna halves of a chunk and are summed at the end.  Then one half-warp per
// subcarrier factors A + sigma2 I, solves L L^H x = z for every data symbol, computes
// [A^-1]_kk from the columns of L^-1, and slices / computes max-log LLRs.
#include <algorithm>
#include <cudaTypedefs.h>
#include <mutex>

#include "rapro_internal.h"
#include "rapro_ptx.cuh"

namespace rapro {

struct DetParams {
  int T, K, M, N, D, q;
  float sigma2;
  int nchunks;
  DetTiles tiles;
  int* status;
};

constexpr int AZ_STRIDE = 17;   // padded row stride of the per-subcarrier Gram in shared memory

// ---------------------------------------------------------------- demapper helpers
// One PAM dimension with mb bits: v is the component scaled so the levels sit at the odd
// integers (2^mb - 1) - 2u, u = 0..2^mb-1, with Gray label u ^ (u >> 1) read MSB first.
// Returns the hard Gray label and fills dd[p] = min_{bit p = 1} (v-a)^2 - min_{bit p = 0} (v-a)^2.
__device__ __forceinline__ int pam_demap(float v, int mb, float* dd) {
  const int nl = 1 << mb;
  float u = ceilf((float(nl) - v) * 0.5f) - 1.0f;   // nearest level, ties to the upper level
  u = fminf(fmaxf(u, 0.0f), float(nl - 1));
  const int ui = int(u);
  float m0[3] = {3.4e38f, 3.4e38f, 3.4e38f}, m1[3] = {3.4e38f, 3.4e38f, 3.4e38f};
  for (int l = 0; l < nl; ++l) {
    const float a = float(nl - 1 - 2 * l);
    const float e = (v - a) * (v - a);
    const int g = l ^ (l >> 1);
    for (int p = 0; p < mb; ++p) {
      if ((g >> (mb - 1 - p)) & 1) m1[p] = fminf(m1[p], e);
      else m0[p] = fminf(m0[p], e);
    }
  }
  for (int p = 0; p < mb; ++p) dd[p] = m1[p] - m0[p];
  return ui ^ (ui >> 1);
}

// ---------------------------------------------------------------------- the kernel
template <bool USE_TMA>
__global__ void __launch_bounds__(DET_MAX_TILES * 32, 1)
    detect_kernel(const __grid_constant__ CUtensorMap map_h, const __grid_constant__ CUtensorMap map_y,
                  const float2* __restrict__ h, const float2* __restrict__ y,
                  float2* __restrict__ x_eq, unsigned char* __restrict__ labels,
                  float* __restrict__ llr, int* __restrict__ info, const __grid_constant__ DetParams P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  int* s_abort = reinterpret_cast<int*>(smem + 64);
  int* s_info = reinterpret_cast<int*>(smem + 128);            // [DET_SC]
  float2* stage0 = reinterpret_cast<float2*>(smem + 1024);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const int t = blockIdx.y, k0 = blockIdx.x * DET_SC;
  const int K = P.K, D = P.D, M = P.M, N = P.N;
  const int KP6 = P.tiles.KP6, DP6 = P.tiles.DP6;
  const int stage_elems = (KP6 + DP6) * DET_MCH * DET_SC;
  const int nst = USE_TMA ? DET_STAGES : 1;

  // Zero the padding rows (users K..KP6-1, symbols D..DP6-1) of every stage once; the
  // loads below never write them.
  for (int s = 0; s < nst; ++s) {
    float2* st = stage0 + s * stage_elems;
    for (int e = threadIdx.x; e < (KP6 - K) * DET_MCH * DET_SC; e += blockDim.x)
      st[K * DET_MCH * DET_SC + e] = make_float2(0.f, 0.f);
    for (int e = threadIdx.x; e < (DP6 - D) * DET_MCH * DET_SC; e += blockDim.x)
      st[(KP6 + D) * DET_MCH * DET_SC + e] = make_float2(0.f, 0.f);
  }
  if (threadIdx.x < DET_SC) s_info[threadIdx.x] = 0;
  if (threadIdx.x == 0) {
    *s_abort = 0;
    if (USE_TMA) {
      for (int s = 0; s < DET_STAGES; ++s) mbar_init(&bars[s], 1);
      fence_mbar_init();
    }
  }
  __syncthreads();

  const uint32_t stage_tx = uint32_t((K + D) * DET_MCH * DET_SC * sizeof(float2));
  auto issue = [&](int c, int s) {
    float2* st = stage0 + s * stage_elems;
    mbar_arrive_expect_tx(&bars[s], stage_tx);
    tma_load_3d(st, &map_h, &bars[s], k0, c * DET_MCH, t * K);
    tma_load_3d(st + KP6 * DET_MCH * DET_SC, &map_y, &bars[s], k0, c * DET_MCH, t * D);
  };
  if (USE_TMA && threadIdx.x == 0) {
    prefetch_tensormap(&map_h);
    prefetch_tensormap(&map_y);
    for (int c = 0; c < DET_STAGES && c < P.nchunks; ++c) issue(c, c);
  }

  const int a = P.tiles.row_group[warp], coff = P.tiles.col_off[warp];
  const int sc = lane & 15, mh = lane >> 4;
  float2 acc[4][6];
#pragma unroll
  for (int ii = 0; ii < 4; ++ii)
#pragma unroll
    for (int jj = 0; jj < 6; ++jj) acc[ii][jj] = make_float2(0.f, 0.f);

  for (int c = 0; c < P.nchunks; ++c) {
    const int s = USE_TMA ? (c % DET_STAGES) : 0;
    float2* st = stage0 + s * stage_elems;
    if (USE_TMA) {
      if (!mbar_wait_bounded(&bars[s], uint32_t(c / DET_STAGES) & 1u)) atomicExch(s_abort, 1);
    } else {
      // Plain loads with bounds checks (odd n_sc or unaligned pointers).
      const int m0 = c * DET_MCH;
      for (int e = threadIdx.x; e < (K + D) * DET_MCH * DET_SC; e += blockDim.x) {
        const int op = e / (DET_MCH * DET_SC), rem = e % (DET_MCH * DET_SC);
        const int m = m0 + rem / DET_SC, k = k0 + rem % DET_SC;
        float2 v = make_float2(0.f, 0.f);
        if (m < M && k < N)
          v = (op < K) ? h[(size_t(t * K + op) * M + m) * N + k]
                       : y[(size_t(t * D + op - K) * M + m) * N + k];
        const int dst = (op < K) ? op : KP6 + (op - K);
        st[dst * DET_MCH * DET_SC + rem] = v;
      }
      __syncthreads();
    }
#pragma unroll
    for (int mm = 0; mm < DET_MCH / 2; ++mm) {
      const int m = mh * (DET_MCH / 2) + mm;
      float2 r[4], cv[6];
#pragma unroll
      for (int ii = 0; ii < 4; ++ii) r[ii] = st[((4 * a + ii) * DET_MCH + m) * DET_SC + sc];
#pragma unroll
      for (int jj = 0; jj < 6; ++jj) cv[jj] = st[((coff + jj) * DET_MCH + m) * DET_SC + sc];
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int jj = 0; jj < 6; ++jj) cmac_conj(acc[ii][jj], r[ii], cv[jj]);
    }
    __syncthreads();
    if (*s_abort) {
      // A pipeline wait ran out: give the copies in flight a bounded chance to land,
      // record the timeout and leave without touching the outputs.
      if (threadIdx.x == 0) {
        for (int cc = c; cc < P.nchunks && cc < c + DET_STAGES; ++cc)
          (void)mbar_wait_bounded(&bars[cc % DET_STAGES], uint32_t(cc / DET_STAGES) & 1u);
        atomicExch(P.status, int(RAPRO_ERR_TIMEOUT));
      }
      return;
    }
    if (USE_TMA && threadIdx.x == 0 && c + DET_STAGES < P.nchunks) issue(c + DET_STAGES, s);
  }

  // Sum the two antenna halves.
#pragma unroll
  for (int ii = 0; ii < 4; ++ii)
#pragma unroll
    for (int jj = 0; jj < 6; ++jj) {
      acc[ii][jj].x += __shfl_xor_sync(0xffffffffu, acc[ii][jj].x, 16);
      acc[ii][jj].y += __shfl_xor_sync(0xffffffffu, acc[ii][jj].y, 16);
    }

  // The stages are free now: reuse them for A (Gram + sigma2 I), z, 1/L_jj and s_k.
  float2* As = stage0;                                        // [DET_SC][16][AZ_STRIDE]
  float2* Zs = As + DET_SC * 16 * AZ_STRIDE;                  // [DET_SC][16][16]
  float* dinv = reinterpret_cast<float*>(Zs + DET_SC * 16 * 16);   // [DET_SC][16]
  float* sdg = dinv + DET_SC * 16;                            // [DET_SC][16]
  if (mh == 0) {
#pragma unroll
    for (int ii = 0; ii < 4; ++ii) {
      const int i = 4 * a + ii;
      if (i >= K) continue;
#pragma unroll
      for (int jj = 0; jj < 6; ++jj) {
        const int col = coff + jj;
        if (col < KP6) {
          if (col < K) {
            float2 v = acc[ii][jj];
            if (col == i) v.x += P.sigma2;
            As[(sc * 16 + i) * AZ_STRIDE + col] = v;
          }
        } else if (col - KP6 < D) {
          Zs[(sc * 16 + i) * 16 + (col - KP6)] = acc[ii][jj];
        }
      }
    }
  }
  __syncthreads();

  const int hw = lane >> 4, l16 = lane & 15;
  for (int scl = warp * 2 + hw; scl < DET_SC; scl += 2 * nwarps) {
    float2* Am = As + scl * 16 * AZ_STRIDE;
    float* di = dinv + scl * 16;
    // Right-looking Cholesky, lane i owns row i.
    for (int j = 0; j < K; ++j) {
      if (l16 == j) {
        const float d = Am[j * AZ_STRIDE + j].x;
        const bool ok = (d > 0.0f) && (d < 3.0e38f);
        const float lj = ok ? sqrtf(d) : __int_as_float(0x7fc00000);
        if (!ok && s_info[scl] == 0) s_info[scl] = j + 1;
        Am[j * AZ_STRIDE + j] = make_float2(lj, 0.f);
        di[j] = 1.0f / lj;
      }
      __syncwarp();
      const float ij = di[j];
      float2 lij = make_float2(0.f, 0.f);
      if (l16 > j && l16 < K) {
        lij = Am[l16 * AZ_STRIDE + j];
        lij.x *= ij;
        lij.y *= ij;
        Am[l16 * AZ_STRIDE + j] = lij;
      }
      __syncwarp();
      if (l16 > j && l16 < K) {
        for (int l = j + 1; l <= l16; ++l) {
          const float2 llj = Am[l * AZ_STRIDE + j];
          float2 v = Am[l16 * AZ_STRIDE + l];
          // v -= lij * conj(llj)
          v.x -= fmaf(lij.x, llj.x, lij.y * llj.y);
          v.y -= fmaf(lij.y, llj.x, -lij.x * llj.y);
          Am[l16 * AZ_STRIDE + l] = v;
        }
      }
      __syncwarp();
    }
    // Lane kk: column kk of L^-1, s_kk = sigma2 sum_j |[L^-1]_{j,kk}|^2 = sigma2 [A^-1]_kk.
    if (l16 < K) {
      const int kk = l16;
      float2 yv[16];
      float sd = 0.f;
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        yv[j] = make_float2(0.f, 0.f);
        if (j < K && j >= kk) {
          float2 s = make_float2(j == kk ? 1.f : 0.f, 0.f);
#pragma unroll
          for (int l = 0; l < j; ++l) {
            const float2 L = Am[j * AZ_STRIDE + l];
            s.x -= fmaf(L.x, yv[l].x, -L.y * yv[l].y);
            s.y -= fmaf(L.x, yv[l].y, L.y * yv[l].x);
          }
          yv[j] = make_float2(s.x * di[j], s.y * di[j]);
          sd = fmaf(yv[j].x, yv[j].x, fmaf(yv[j].y, yv[j].y, sd));
        }
      }
      sdg[scl * 16 + kk] = P.sigma2 * sd;
    }
    __syncwarp();
    // Lane n: solve L w = z_n, then L^H x = w, for data symbol n of the slot.
    const int kglob = k0 + scl;
    if (l16 < D && kglob < N) {
      const int n = l16;
      float2 w[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        w[j] = make_float2(0.f, 0.f);
        if (j < K) {
          float2 s = Zs[(scl * 16 + j) * 16 + n];
#pragma unroll
          for (int l = 0; l < j; ++l) {
            const float2 L = Am[j * AZ_STRIDE + l];
            s.x -= fmaf(L.x, w[l].x, -L.y * w[l].y);
            s.y -= fmaf(L.x, w[l].y, L.y * w[l].x);
          }
          w[j] = make_float2(s.x * di[j], s.y * di[j]);
        }
      }
#pragma unroll
      for (int j = 15; j >= 0; --j) {
        if (j < K) {
          float2 s = w[j];
#pragma unroll
          for (int l = j + 1; l < 16; ++l) {
            if (l < K) {
              const float2 L = Am[l * AZ_STRIDE + j];   // use conj(L[l][j])
              s.x -= fmaf(L.x, w[l].x, L.y * w[l].y);
              s.y -= fmaf(L.x, w[l].y, -L.y * w[l].x);
            }
          }
          w[j] = make_float2(s.x * di[j], s.y * di[j]);
        }
      }
      const int q = P.q, mb = q >> 1;
      const float scale = (mb == 1) ? 1.41421356237309505f : (mb == 2 ? 3.16227766016837933f : 6.48074069840786023f);
      const size_t dn = size_t(t) * D + n;
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        if (k < K) {
          const size_t o = (dn * K + k) * N + kglob;
          x_eq[o] = w[k];
          if (labels || llr) {
            const float sk = sdg[scl * 16 + k];
            const float mu = 1.0f - sk;
            const float inv_mu = 1.0f / mu;
            const float nu = sk * inv_mu;
            float ddI[3], ddQ[3];
            const int gI = pam_demap(w[k].x * inv_mu * scale, mb, ddI);
            const int gQ = pam_demap(w[k].y * inv_mu * scale, mb, ddQ);
            if (labels) {
              int lab = 0;
              for (int p = 0; p < mb; ++p) {
                lab |= ((gI >> (mb - 1 - p)) & 1) << (q - 1 - 2 * p);
                lab |= ((gQ >> (mb - 1 - p)) & 1) << (q - 2 - 2 * p);
              }
              labels[o] = (unsigned char)lab;
            }
            if (llr) {
              const float g = 1.0f / (nu * scale * scale);
              for (int p = 0; p < mb; ++p) {
                llr[o * q + 2 * p] = ddI[p] * g;
                llr[o * q + 2 * p + 1] = ddQ[p] * g;
              }
            }
          }
        }
      }
    }
    __syncwarp();
    if (l16 == 0 && info && kglob < N) info[size_t(t) * N + kglob] = s_info[scl];
  }
}

// ---------------------------------------------------------------------- launcher
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

// 3-D map over complex64 data [depth][M][N] with boxes of DET_SC x DET_MCH x box_z.
static bool encode_map(CUtensorMap* m, const void* base, int N, int M, int depth, int box_z) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[3] = {cuuint64_t(N), cuuint64_t(M), cuuint64_t(depth)};
  cuuint64_t strides[2] = {cuuint64_t(N) * 8, cuuint64_t(N) * M * 8};
  cuuint32_t box[3] = {cuuint32_t(DET_SC), cuuint32_t(DET_MCH), cuuint32_t(box_z)};
  cuuint32_t es[3] = {1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<void*>(base), dims, strides, box, es,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t detect_smem_bytes(const DetTiles& t, bool tma) {
  const size_t stage = size_t(t.KP6 + t.DP6) * DET_MCH * DET_SC * sizeof(float2);
  const size_t az = size_t(DET_SC) * 16 * AZ_STRIDE * sizeof(float2) +
                    size_t(DET_SC) * 16 * 16 * sizeof(float2) + 2 * size_t(DET_SC) * 16 * sizeof(float);
  return 1024 + std::max(stage * (tma ? DET_STAGES : 1), az);
}

cudaError_t launch_detect(const Plan& pl, const float2* h, const float2* y, float2* x_eq,
                          unsigned char* labels, float* llr, int* info, cudaStream_t st) {
  DetParams P;
  P.T = pl.T; P.K = pl.p.K; P.M = pl.p.M; P.N = pl.p.n_sc; P.D = pl.D; P.q = pl.q;
  P.sigma2 = float(pl.p.sigma2);
  P.nchunks = (pl.p.M + DET_MCH - 1) / DET_MCH;
  P.tiles = pl.tiles;
  P.status = pl.d_status;
  CUtensorMap mh{}, my{};
  const bool aligned = ((reinterpret_cast<uintptr_t>(h) | reinterpret_cast<uintptr_t>(y)) & 15) == 0;
  bool tma = aligned && (P.N % 2 == 0) && encode_map(&mh, h, P.N, P.M, P.T * P.K, P.K) &&
             encode_map(&my, y, P.N, P.M, P.T * P.D, P.D);
  const size_t smem = detect_smem_bytes(pl.tiles, tma);
  dim3 grid((P.N + DET_SC - 1) / DET_SC, P.T);
  dim3 block(32 * pl.tiles.n_tiles);
  if (tma)
    detect_kernel<true><<<grid, block, smem, st>>>(mh, my, h, y, x_eq, labels, llr, info, P);
  else
    detect_kernel<false><<<grid, block, smem, st>>>(mh, my, h, y, x_eq, labels, llr, info, P);
  return cudaGetLastError();
}

// Detection without a plan (same kernel): used by the allocation-free receive entry point.
cudaError_t launch_detect_raw(const DetTiles& tiles, int T, int K, int M, int N, int D, int q,
                              float sigma2, int* status, const float2* h, const float2* y,
                              float2* x_eq, unsigned char* labels, float* llr, int* info,
                              cudaStream_t st) {
  DetParams P;
  P.T = T; P.K = K; P.M = M; P.N = N; P.D = D; P.q = q;
  P.sigma2 = sigma2;
  P.nchunks = (M + DET_MCH - 1) / DET_MCH;
  P.tiles = tiles;
  P.status = status;
  CUtensorMap mh{}, my{};
  const bool aligned = ((reinterpret_cast<uintptr_t>(h) | reinterpret_cast<uintptr_t>(y)) & 15) == 0;
  bool tma = aligned && (N % 2 == 0) && encode_map(&mh, h, N, M, T * K, K) &&
             encode_map(&my, y, N, M, T * D, D);
  const size_t smem = detect_smem_bytes(tiles, tma);
  dim3 grid((N + DET_SC - 1) / DET_SC, T);
  dim3 block(32 * tiles.n_tiles);
  if (tma)
    detect_kernel<true><<<grid, block, smem, st>>>(mh, my, h, y, x_eq, labels, llr, info, P);
  else
    detect_kernel<false><<<grid, block, smem, st>>>(mh, my, h, y, x_eq, labels, llr, info, P);
  return cudaGetLastError();
}

// Raise the dynamic shared-memory limit of the detector once per device, at plan
// creation (not at launch, which may be inside a CUDA-graph capture).
cudaError_t prepare_detect(int device) {
  static std::once_flag flags[64];
  static cudaError_t result[64];
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  std::call_once(flags[device], [device] {
    DetTiles worst = make_det_tiles(RAPRO_MAX_USERS, RAPRO_MAX_DATA_PER_SLOT);
    const int smem = int(std::max(detect_smem_bytes(worst, true), detect_smem_bytes(worst, false)));
    cudaError_t e = cudaFuncSetAttribute(detect_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(detect_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    result[device] = e;
  });
  return result[device];
}

}  // namespace rapro
