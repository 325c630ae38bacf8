// MMSE detection kernel (Eq. 20-22) with Cholesky (A = L L^H, uplo = L) and Gray-QAM
// demapping; templated on the padded user count KT and data-symbol count DT.
//
// One CTA owns DET_SC = 16 consecutive subcarriers of one slot.  The channel estimate
// h[t][s][m][k] and the slot's data symbols y[t*D+n][m][k] stream through shared memory
// DET_MCH = 8 antennas at a time as TMA boxes (16 subcarriers x 8 antennas x K users, and
// x D symbols) in a DET_STAGES-deep mbarrier pipeline.  Each warp owns one 4 x 6 tile of
// the augmented product: rows are users i, columns are users j (Gram entries
// A[i][j] = sum_m conj(h_i) h_j) or data symbols n (matched filter z[i][n] =
// sum_m conj(h_i) y_n); lanes 0-15 and 16-31 take the two antenna halves of a chunk.
//
// Epilogue, one half-warp per subcarrier, lane i holding row i in registers:
//   Cholesky of A + sigma2 I by columns (pivot and column broadcast by shuffles),
//   w = L^-1 z (forward substitution, lane-per-row), the rows of L^-1 (same scheme with
//   the identity), s_k = sigma2 [A^-1]_kk = sigma2 sum_i |[L^-1]_ik|^2 (butterfly column
//   sums), x~ = L^-H w from the rows of L^-1 and w exchanged through shared memory.
// Then all threads demap (x^ = x~ / mu, mu = 1 - s) and store with coalesced writes.
#pragma once

#include <cudaTypedefs.h>

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

struct DetLaunch {
  CUtensorMap map_h, map_y;
  const float2* h;
  const float2* y;
  float2* x_eq;
  unsigned char* labels;
  float* llr;
  int* info;
  DetParams P;
  bool tma;
  size_t smem;
  cudaStream_t stream;
};

// Shared-memory footprint of the epilogue for (KT, DT).
__host__ __device__ constexpr size_t det_epilogue_bytes(int KT, int DT) {
  return size_t(DET_SC) * KT * (KT + 1) * 8 + size_t(DET_SC) * KT * DT * 8 + size_t(DET_SC) * KT * 4 +
         size_t(DET_SC) * 4;
}

// Threads of the largest tile set of a (KT, DT) class: the tile count of make_det_tiles
// at K = KT, D = DT (one warp per tile).
__host__ __device__ constexpr int det_max_threads(int KT, int DT) {
  int n = 0;
  for (int a = 0; a < (KT + 3) / 4; ++a)
    for (int c = 0; c < (KT + 5) / 6; ++c)
      if (6 * c <= 4 * a + 3) ++n;
  return 32 * (n + ((KT + 3) / 4) * ((DT + 5) / 6));
}

inline size_t det_stage_bytes(const DetTiles& t) {
  return size_t(t.KP6 + t.DP6) * DET_MCH * DET_SC * sizeof(float2);
}

// --------------------------------------------------------------- demapper helpers
// One PAM dimension with MB bits.  v is the component scaled so that the levels sit on
// the odd integers (2^MB - 1) - 2u (u = 0..2^MB-1, Gray label u ^ (u >> 1), MSB first).
// Returns the hard Gray label; dd[p] = min_{bit p = 1} (v - a)^2 - min_{bit p = 0} (v - a)^2.
template <int MB>
__device__ __forceinline__ int pam_demap(float v, float (&dd)[MB]) {
  constexpr int NL = 1 << MB;
  float u = ceilf((float(NL) - v) * 0.5f) - 1.0f;   // nearest level; ties to the upper level
  u = fminf(fmaxf(u, 0.0f), float(NL - 1));
  const int ui = int(u);
  float m0[MB], m1[MB];
#pragma unroll
  for (int p = 0; p < MB; ++p) m0[p] = m1[p] = 3.4e38f;
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    const float a = float(NL - 1 - 2 * l);
    const float e = (v - a) * (v - a);
    const int g = l ^ (l >> 1);
#pragma unroll
    for (int p = 0; p < MB; ++p) {
      if ((g >> (MB - 1 - p)) & 1)
        m1[p] = fminf(m1[p], e);
      else
        m0[p] = fminf(m0[p], e);
    }
  }
#pragma unroll
  for (int p = 0; p < MB; ++p) dd[p] = m1[p] - m0[p];
  return ui ^ (ui >> 1);
}

template <int MB>
__device__ __forceinline__ void demap_store(float2 xt, float s, size_t o, unsigned char* labels, float* llr) {
  constexpr int Q = 2 * MB;
  const float scale = (MB == 1) ? 1.41421356237309505f : (MB == 2 ? 3.16227766016837933f : 6.48074069840786023f);
  const float mu = 1.0f - s;
  const float inv_mu = 1.0f / mu;
  const float nu = s * inv_mu;
  float ddI[MB], ddQ[MB];
  const int gI = pam_demap<MB>(xt.x * inv_mu * scale, ddI);
  const int gQ = pam_demap<MB>(xt.y * inv_mu * scale, ddQ);
  if (labels) {
    int lab = 0;
#pragma unroll
    for (int p = 0; p < MB; ++p) {
      lab |= ((gI >> (MB - 1 - p)) & 1) << (Q - 1 - 2 * p);
      lab |= ((gQ >> (MB - 1 - p)) & 1) << (Q - 2 - 2 * p);
    }
    labels[o] = (unsigned char)lab;
  }
  if (llr) {
    const float g = 1.0f / (nu * scale * scale);
#pragma unroll
    for (int p = 0; p < MB; ++p) {
      llr[o * Q + 2 * p] = ddI[p] * g;
      llr[o * Q + 2 * p + 1] = ddQ[p] * g;
    }
  }
}

// ------------------------------------------------------------------------ kernel
template <int KT, int DT, bool USE_TMA>
__global__ void __launch_bounds__(det_max_threads(KT, DT), 1)
    detect_kernel(const __grid_constant__ CUtensorMap map_h, const __grid_constant__ CUtensorMap map_y,
                  const float2* __restrict__ h, const float2* __restrict__ y,
                  float2* __restrict__ x_eq, unsigned char* __restrict__ labels,
                  float* __restrict__ llr, int* __restrict__ info, const __grid_constant__ DetParams P) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  int* s_abort = reinterpret_cast<int*>(smem + 128);
  float2* stage0 = reinterpret_cast<float2*>(smem + 1024);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const int t = blockIdx.y, k0 = blockIdx.x * DET_SC;
  const int K = P.K, D = P.D, M = P.M, N = P.N;
  const int KP6 = P.tiles.KP6, DP6 = P.tiles.DP6;
  const int stage_elems = (KP6 + DP6) * DET_MCH * DET_SC;
  const int nst = USE_TMA ? DET_STAGES : 1;

  // Zero the padding rows (users K..KP6-1, symbols D..DP6-1) of every stage once; the
  // loads never write them.
  for (int s = 0; s < nst; ++s) {
    float2* st = stage0 + s * stage_elems;
    for (int e = threadIdx.x; e < (KP6 - K) * DET_MCH * DET_SC; e += blockDim.x)
      st[K * DET_MCH * DET_SC + e] = make_float2(0.f, 0.f);
    for (int e = threadIdx.x; e < (DP6 - D) * DET_MCH * DET_SC; e += blockDim.x)
      st[(KP6 + D) * DET_MCH * DET_SC + e] = make_float2(0.f, 0.f);
  }
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

  // ------------------------------------------------ accumulation: Gram and z
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
          v = (op < K) ? h[(size_t(t * K + op) * M + m) * N + k] : y[(size_t(t * D + op - K) * M + m) * N + k];
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

#pragma unroll
  for (int ii = 0; ii < 4; ++ii)
#pragma unroll
    for (int jj = 0; jj < 6; ++jj) {
      acc[ii][jj].x += __shfl_xor_sync(0xffffffffu, acc[ii][jj].x, 16);
      acc[ii][jj].y += __shfl_xor_sync(0xffffffffu, acc[ii][jj].y, 16);
    }

  // The stages are free: A (+ sigma2 I) and z go to shared memory.
  constexpr int AS = KT + 1;                                    // padded row stride
  float2* As = stage0;                                          // [DET_SC][KT][AS], later rows of L^-1
  float2* Zs = As + DET_SC * KT * AS;                           // [DET_SC][KT][DT], later w, then x~ [n][k]
  float* Ss = reinterpret_cast<float*>(Zs + DET_SC * KT * DT);  // [DET_SC][KT]  s_k
  int* Is = reinterpret_cast<int*>(Ss + DET_SC * KT);           // [DET_SC]      info
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
            As[(sc * KT + i) * AS + col] = v;
          }
        } else if (col - KP6 < D) {
          Zs[(sc * KT + i) * DT + (col - KP6)] = acc[ii][jj];
        }
      }
    }
  }
  __syncthreads();

  // --------------------------------------------- factorisation and solves
  const int hw = lane >> 4, i = lane & 15, base = hw << 4;
  const unsigned FULL = 0xffffffffu;
  for (int scl = warp * 2 + hw; scl < DET_SC; scl += 2 * nwarps) {
    const bool live = i < K;                 // real user row
    float2 ar[KT], zr[DT];
#pragma unroll
    for (int j = 0; j < KT; ++j) {
      if (live && j <= i) ar[j] = As[(scl * KT + i) * AS + j];
      else ar[j] = make_float2((i < KT && j == i) ? 1.f : 0.f, 0.f);   // padded rows: identity
    }
#pragma unroll
    for (int n = 0; n < DT; ++n) zr[n] = (live && n < D) ? Zs[(scl * KT + i) * DT + n] : make_float2(0.f, 0.f);
    __syncwarp();

    // Cholesky, column j at a time: every lane reads the pivot, so each knows L_jj.
    float inv_l[KT];
    int fail = 0;
#pragma unroll
    for (int j = 0; j < KT; ++j) {
      const float d = __shfl_sync(FULL, ar[j].x, base + j);
      const bool ok = (d > 0.0f) && (d < 3.0e38f);
      if (!ok && fail == 0) fail = j + 1;
      const float lj = sqrtf(d);
      const float il = 1.0f / lj;
      inv_l[j] = il;
      if (i == j) ar[j] = make_float2(lj, 0.f);
      else if (i > j) ar[j] = make_float2(ar[j].x * il, ar[j].y * il);
#pragma unroll
      for (int l = j + 1; l < KT; ++l) {
        float2 c;
        c.x = __shfl_sync(FULL, ar[j].x, base + l);          // L[l][j]
        c.y = __shfl_sync(FULL, ar[j].y, base + l);
        if (i >= l) {                                        // A[i][l] -= L[i][j] conj(L[l][j])
          ar[l].x -= fmaf(ar[j].x, c.x, ar[j].y * c.y);
          ar[l].y -= fmaf(ar[j].y, c.x, -ar[j].x * c.y);
        }
      }
    }
    // w = L^-1 z, lane i ends with w_i.
#pragma unroll
    for (int j = 0; j < KT; ++j) {
#pragma unroll
      for (int n = 0; n < DT; ++n) {
        float2 wj;
        wj.x = __shfl_sync(FULL, zr[n].x, base + j) * inv_l[j];
        wj.y = __shfl_sync(FULL, zr[n].y, base + j) * inv_l[j];
        if (i == j) zr[n] = wj;
        else if (i > j) {
          zr[n].x -= fmaf(ar[j].x, wj.x, -ar[j].y * wj.y);
          zr[n].y -= fmaf(ar[j].x, wj.y, ar[j].y * wj.x);
        }
      }
    }
    // Rows of L^-1 (forward substitution of the identity), lane i ends with row i.
    float2 yr[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) yr[k] = make_float2(k == i ? 1.f : 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < KT; ++j) {
#pragma unroll
      for (int k = 0; k <= j; ++k) {
        float2 yj;
        yj.x = __shfl_sync(FULL, yr[k].x, base + j) * inv_l[j];
        yj.y = __shfl_sync(FULL, yr[k].y, base + j) * inv_l[j];
        if (i == j) yr[k] = yj;
        else if (i > j) {
          yr[k].x -= fmaf(ar[j].x, yj.x, -ar[j].y * yj.y);
          yr[k].y -= fmaf(ar[j].x, yj.y, ar[j].y * yj.x);
        }
      }
    }
    // s_k = sigma2 sum_i |[L^-1]_ik|^2 over the real user rows.
    float sq[KT];
#pragma unroll
    for (int k = 0; k < KT; ++k) sq[k] = live ? fmaf(yr[k].x, yr[k].x, yr[k].y * yr[k].y) : 0.f;
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1)
#pragma unroll
      for (int k = 0; k < KT; ++k) sq[k] += __shfl_xor_sync(FULL, sq[k], off);
    // Exchange rows of L^-1 and w through shared memory for x~ = L^-H w.
    if (i < KT) {
#pragma unroll
      for (int k = 0; k < KT; ++k) As[(scl * KT + i) * AS + k] = yr[k];
#pragma unroll
      for (int n = 0; n < DT; ++n) Zs[(scl * KT + i) * DT + n] = zr[n];
    }
    if (live) {
      float sk = 0.f;
#pragma unroll
      for (int k = 0; k < KT; ++k)
        if (k == i) sk = sq[k];
      Ss[scl * KT + i] = P.sigma2 * sk;
    }
    if (i == 0) Is[scl] = fail;
    __syncwarp();
    float2 xk[DT];
#pragma unroll
    for (int n = 0; n < DT; ++n) xk[n] = make_float2(0.f, 0.f);
    if (live) {
      for (int r = i; r < K; ++r) {
        const float2 Y = As[(scl * KT + r) * AS + i];        // [L^-1]_{r,i}, use its conjugate
#pragma unroll
        for (int n = 0; n < DT; ++n) {
          const float2 w = Zs[(scl * KT + r) * DT + n];
          xk[n].x = fmaf(Y.x, w.x, fmaf(Y.y, w.y, xk[n].x));
          xk[n].y = fmaf(Y.x, w.y, fmaf(-Y.y, w.x, xk[n].y));
        }
      }
    }
    __syncwarp();
    if (live) {
#pragma unroll
      for (int n = 0; n < DT; ++n)
        if (n < D) Zs[(scl * DT + n) * KT + i] = xk[n];       // x~ as [sc][n][k]
    }
    __syncwarp();
  }
  __syncthreads();

  // ------------------------------------------------ demap and coalesced stores
  const int total = D * K * DET_SC;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int scx = idx % DET_SC, k = (idx / DET_SC) % K, n = idx / (DET_SC * K);
    const int kg = k0 + scx;
    if (kg >= N) continue;
    const float2 xt = Zs[(scx * DT + n) * KT + k];
    const size_t o = (size_t(t * D + n) * K + k) * N + kg;
    x_eq[o] = xt;
    if (labels || llr) {
      const float s = Ss[scx * KT + k];
      switch (P.q) {
        case 2: demap_store<1>(xt, s, o, labels, llr); break;
        case 4: demap_store<2>(xt, s, o, labels, llr); break;
        default: demap_store<3>(xt, s, o, labels, llr); break;
      }
    }
  }
  if (info && threadIdx.x < DET_SC && k0 + threadIdx.x < N) info[size_t(t) * N + k0 + threadIdx.x] = Is[threadIdx.x];
}

template <int KT>
cudaError_t detect_launch_kt(const DetLaunch& L);

template <int KT>
cudaError_t detect_prepare_kt(int smem);

// One explicit specialisation per padded user count, each in its own translation unit.
template <> cudaError_t detect_launch_kt<4>(const DetLaunch& L);
template <> cudaError_t detect_launch_kt<8>(const DetLaunch& L);
template <> cudaError_t detect_launch_kt<12>(const DetLaunch& L);
template <> cudaError_t detect_launch_kt<16>(const DetLaunch& L);
template <> cudaError_t detect_prepare_kt<4>(int smem);
template <> cudaError_t detect_prepare_kt<8>(int smem);
template <> cudaError_t detect_prepare_kt<12>(int smem);
template <> cudaError_t detect_prepare_kt<16>(int smem);

// Definitions, instantiated once per KT in its own translation unit.
#define RAPRO_DETECT_DEFINE_KT(KTV)                                                                    \
  template <>                                                                                          \
  cudaError_t detect_launch_kt<KTV>(const DetLaunch& L) {                                              \
    dim3 grid((L.P.N + DET_SC - 1) / DET_SC, L.P.T);                                                   \
    dim3 block(32 * L.P.tiles.n_tiles);                                                                \
    const bool d12 = L.P.D > 6;                                                                        \
    if (L.tma) {                                                                                       \
      if (d12) detect_kernel<KTV, 12, true><<<grid, block, L.smem, L.stream>>>(                        \
          L.map_h, L.map_y, L.h, L.y, L.x_eq, L.labels, L.llr, L.info, L.P);                           \
      else detect_kernel<KTV, 6, true><<<grid, block, L.smem, L.stream>>>(                             \
          L.map_h, L.map_y, L.h, L.y, L.x_eq, L.labels, L.llr, L.info, L.P);                           \
    } else {                                                                                           \
      if (d12) detect_kernel<KTV, 12, false><<<grid, block, L.smem, L.stream>>>(                       \
          L.map_h, L.map_y, L.h, L.y, L.x_eq, L.labels, L.llr, L.info, L.P);                           \
      else detect_kernel<KTV, 6, false><<<grid, block, L.smem, L.stream>>>(                            \
          L.map_h, L.map_y, L.h, L.y, L.x_eq, L.labels, L.llr, L.info, L.P);                           \
    }                                                                                                  \
    return cudaGetLastError();                                                                         \
  }                                                                                                    \
  template <>                                                                                          \
  cudaError_t detect_prepare_kt<KTV>(int smem) {                                                       \
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;                           \
    cudaError_t e = cudaFuncSetAttribute(detect_kernel<KTV, 6, true>, A, smem);                        \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(detect_kernel<KTV, 12, true>, A, smem);             \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(detect_kernel<KTV, 6, false>, A, smem);             \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(detect_kernel<KTV, 12, false>, A, smem);            \
    return e;                                                                                          \
  }

}  // namespace rapro
