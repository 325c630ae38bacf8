// MMSE detection kernel (Eq. 20-22) with Cholesky (A = L L^H, uplo = L) and Gray-QAM
// demapping; templated on the padded user count KT and data-symbol count DT.
//
// One CTA owns DET_SC = 16 consecutive subcarriers of one slot.  The channel estimate
// h[t][s][m][k] and the slot's data symbols y[t*D+n][m][k] stream through shared memory
// DET_MCH = 8 antennas at a time as TMA boxes (16 subcarriers x 8 antennas x K users, and
// x D symbols) in a DET_STAGES-deep mbarrier pipeline.  Each warp owns one role (see
// DetTiles): the lower triangle of a 4-user Gram block plus one off-diagonal block, or a
// 4-user x 6-symbol matched-filter block, so every entry of A[i][j] = sum_m conj(h_i) h_j
// (j <= i) and z[i][n] = sum_m conj(h_i) y_n is computed once.  Lane = subcarrier; the
// antennas of a chunk are split between the two half-warps and, when there are few roles,
// between two warps per role.  A producer warp issues the TMA loads; consumer warps free a
// stage through an mbarrier, so no CTA-wide barrier sits in the antenna loop.
//
// Epilogue, one half-warp per subcarrier, lane i owning row i (all exchanges go through
// shared memory: a broadcast load moves a complex value, a shuffle only half of one):
//   Cholesky of A + sigma2 I by columns (each column published in a small buffer);
//   column i of L^-1 by forward substitution with pending sums and
//   s_i = sigma2 [A^-1]_ii = sigma2 sum_j |L^-1[j][i]|^2; w = L^-1 z lane-per-row and
//   x~ = L^-H w lane-per-column.
// Then all threads demap (x^ = x~ / mu, mu = 1 - s) and store with coalesced writes.
//
// Fused receive form (DET_FUSED): the CTA takes the raw pilot symbols instead of h.  Each
// stage then holds y_pilot for the tile's LMMSE blocks (K users x 8 antennas x `span`
// subcarriers from the first block's start) besides the data symbols; consumer half-warps
// filter the chunk, lane = output subcarrier, with the LS division folded into the lane's
// weight row (h_j = sum_i W[j][i] conj(p_i) / |p_i|^2 y_i, Eq. 9 and 12), write h into a
// double-buffered chunk of shared memory, meet at a named barrier and run the Gram and
// matched filter on it as above.  The estimate never leaves the SM (unless the caller asks
// for it), and the subframe needs one launch.
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
  // FP64 fallback (precision form): subcarriers whose pivot ratio max/min L_jj^2 exceeds
  // cond_limit, or whose FP32 factorisation failed, are appended to fix_list
  // (t * N + subcarrier) for the FP64 kernel.
  int* fix_count;       // null: no fallback
  int* fix_ticket;      // CTAs finished; the last one runs the FP64 solves and resets both
  int* fix_list;
  int fix_cap;
  float cond_limit;
  double sigma2_d;
  // Fused receive form: map_h covers y_pilot [T K][M][N] in boxes of span x DET_MCH x K.
  const float2* pil;      // pilots [T][K][N]
  const float2* w_main;   // W of a full block [B][B], row-major (h_j = sum_i W[j][i] h_ls_i)
  const float2* w_tail;   // W of the tail block [tail][tail], or null
  float2* h_out;          // channel estimate [T][K][M][N], or null (then not written)
  int B, nfull, tail;     // block size, full blocks, tail block length
  int span, nst;          // pilot box width in subcarriers, stage ring depth
  // Precision form (refine kernel): the tensor-core Gram | matched filter [T][N][K][K + D].
  const float2* gram;
  // Diagnostics of the timeout path (rapro_plan_set_wait_test): rounds of the waits between
  // the load producer and the consumers (0: the default limit), and a producer that posts
  // no load, so that a consumer's wait runs out.  Draining copies in flight always waits
  // with the default limit.
  uint32_t wait_rounds;
  int stall_producer;
  // Non-null: the kernel does nothing (outputs and info untouched) when this word is
  // non-zero on entry, i.e. when the kernel before it in the stream recorded a failure.
  const int* skip_if_set;
};

// Kernel forms: plain detection, detection with the FP64 fallback, fused receive.
enum { DET_PLAIN = 0, DET_FIX = 1, DET_FUSED = 2 };

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
  bool fused;
  size_t smem;
  cudaStream_t stream;
};

// Threads of the largest role set of a (KT, DT) class (make_det_tiles at K = KT, D = DT):
// NG triangle roles, the off-diagonal blocks left after pairing one with each triangle,
// NG x data-group blocks; two warps per role when there are at most 8 roles.
__host__ __device__ constexpr int det_max_threads(int KT, int DT) {
  const int ng = (KT + 3) / 4, nr = ng * (ng - 1) / 2, ndg = (DT + 5) / 6;
  const int roles = ng + (nr > ng ? nr - ng : 0) + ng * ndg;
  const int warps = roles * (roles <= 8 ? 2 : 1) + 1;       // + the TMA producer warp
  return 32 * (warps < DET_SC / 2 ? DET_SC / 2 : warps);     // at least one warp per 2 subcarriers
}

inline int det_block_threads(const DetTiles& t) {
  const int warps = t.n_roles * t.msplit + 1;
  return 32 * (warps < DET_SC / 2 ? DET_SC / 2 : warps);
}

// Shared-memory layout of the epilogue (reusing the stage ring), in float2 units:
//   A / L / L^-1  [DET_SC][KT][KT+1]      z / w  [DET_SC][KT][DT]
//   x~ [DT][KT][DET_SC+1]   s [KT][DET_SC+1] (float)   info [DET_SC] (int)
//   column broadcast buffers [DET_SC][2][16]
//   parked partial sums [warps][DET_SC][26]
__host__ __device__ constexpr size_t det_off_z(int KT) { return size_t(DET_SC) * KT * (KT + 1); }
__host__ __device__ constexpr size_t det_off_x(int KT, int DT) { return det_off_z(KT) + size_t(DET_SC) * KT * DT; }
__host__ __device__ constexpr size_t det_off_s(int KT, int DT) { return det_off_x(KT, DT) + size_t(DT) * KT * (DET_SC + 1); }
__host__ __device__ constexpr size_t det_off_col(int KT, int DT) {
  return det_off_s(KT, DT) + (size_t(KT) * (DET_SC + 1) + DET_SC + 1) / 2;
}
__host__ __device__ constexpr size_t det_off_park(int KT, int DT) { return det_off_col(KT, DT) + size_t(DET_SC) * 2 * 16; }
__host__ __device__ constexpr size_t det_epilogue_bytes(int KT, int DT) { return det_off_park(KT, DT) * 8; }
// Parked partial sums: one slot of DET_SC x 26 complex per warp.
__host__ __device__ constexpr size_t det_scratch_bytes(int KT, int DT) {
  return size_t(det_max_threads(KT, DT) / 32) * DET_SC * 26 * 8;
}

inline size_t det_stage_bytes(const DetTiles& t) {
  return size_t(t.KP + t.DP) * DET_MCH * DET_SC * sizeof(float2);
}

// Fused form, in float2 units after the 1 KB header: the ring [nst][K*DET_MCH*span +
// DP*DET_MCH*DET_SC], the filtered chunk [2][KP][DET_MCH][DET_SC], the LS-folded weights
// [K][DET_SC][16] (zero past each block's length).
inline size_t fused_work_bytes(const DetTiles& t, int K, int span, int nst) {
  const size_t stage = size_t(K) * DET_MCH * span + size_t(t.DP) * DET_MCH * DET_SC;
  return (size_t(nst) * stage + 2 * size_t(t.KP) * DET_MCH * DET_SC + size_t(K) * DET_SC * 16) * sizeof(float2);
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
  const float inv_mu = __fdividef(1.0f, mu);
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
    const float g = __fdividef(1.0f, nu * scale * scale);
#pragma unroll
    for (int p = 0; p < MB; ++p) {
      llr[o * Q + 2 * p] = ddI[p] * g;
      llr[o * Q + 2 * p + 1] = ddQ[p] * g;
    }
  }
}

// Hard Gray label alone (no LLR): the nearest level per dimension, ties to the upper level,
// bits interleaved I, Q from the most significant one (the labels of demap_store).
template <int MB>
__device__ __forceinline__ unsigned char hard_label(float2 xt, float s) {
  constexpr int NL = 1 << MB, Q = 2 * MB;
  const float scale = (MB == 1) ? 1.41421356237309505f : (MB == 2 ? 3.16227766016837933f : 6.48074069840786023f);
  const float g = __fdividef(1.0f, 1.0f - s) * scale;
  const float vi = xt.x * g, vq = xt.y * g;
  const int ui = int(fminf(fmaxf(ceilf((float(NL) - vi) * 0.5f) - 1.0f, 0.0f), float(NL - 1)));
  const int uq = int(fminf(fmaxf(ceilf((float(NL) - vq) * 0.5f) - 1.0f, 0.0f), float(NL - 1)));
  const int gi = ui ^ (ui >> 1), gq = uq ^ (uq >> 1);
  int lab = 0;
#pragma unroll
  for (int p = 0; p < MB; ++p) {
    lab |= ((gi >> (MB - 1 - p)) & 1) << (Q - 1 - 2 * p);
    lab |= ((gq >> (MB - 1 - p)) & 1) << (Q - 2 - 2 * p);
  }
  return (unsigned char)lab;
}

}  // namespace rapro

#include "fixup.cuh"

namespace rapro {

// Per subcarrier scl (one half-warp, lane i owns row i) of a detector tile: Cholesky of the
// lower triangle of A in As (sigma2 included), the columns of L^-1 into As, s_i = sigma2
// [A^-1]_ii into Ss, the first failed pivot into Is; then w = L^-1 z (z in Zs) and
// x~ = L^-H w into Xs.  FIX also flags ill-conditioned or failed subcarriers for the FP64
// fallback.  Layouts as in the detector's epilogue (AS = KT + 1, XS = DET_SC + 1).
template <int KT, int DT, bool FIX>
__device__ __forceinline__ void det_factor_solve(const int i, const int scl, const int K, const int D, const int t,
                                                 const int k0, const int N, const DetParams& P, float2* As,
                                                 float2* Zs, float2* Xs, float* Ss, int* Is, float2* Cb) {
  constexpr int AS = KT + 1;
  constexpr int XS = DET_SC + 1;
  const bool live = i < K;                 // real user row
  const bool row = i < KT;                 // row of the padded system
  float2* Am = As + scl * KT * AS;
  float2* Zm = Zs + scl * KT * DT;
  float2* cb = Cb + scl * 32;              // two 16-entry column buffers
  float2 ar[KT];
#pragma unroll
  for (int j = 0; j < KT; ++j) {
    if (live && j <= i) ar[j] = Am[i * AS + j];
    else ar[j] = make_float2((row && j == i) ? 1.f : 0.f, 0.f);   // padded rows: identity
  }

  // Cholesky, column j at a time: rows publish A[.][j] in a column buffer; every lane
  // reads the pivot and the column from it (broadcast loads) and updates its own row.
  float inv_l[KT];
  int fail = 0;
  float dmax = 0.f, dmin = 3.4e38f;        // pivots L_jj^2 of the real users
#pragma unroll
  for (int j = 0; j < KT; ++j) {
    float2* col = cb + (j & 1) * 16;
    if (row) col[i] = ar[j];
    __syncwarp();
    const float d = col[j].x;
    const bool ok = (d > 0.0f) && (d < 3.0e38f);
    if (!ok && fail == 0) fail = j + 1;
    if (j < K) {
      dmax = fmaxf(dmax, d);
      dmin = fminf(dmin, d);
    }
    const float il = rsqrtf(d);                            // 1 / L_jj
    inv_l[j] = il;
    const float2 lij = make_float2(ar[j].x * il, ar[j].y * il);   // L[i][j] for i > j
#pragma unroll
    for (int l = j + 1; l < KT; ++l) {
      const float2 a = col[l];                             // A[l][j]; L[l][j] = a * il
      if (i >= l) {                                        // A[i][l] -= L[i][j] conj(L[l][j])
        ar[l].x -= fmaf(lij.x, a.x, lij.y * a.y) * il;
        ar[l].y -= fmaf(lij.y, a.x, -lij.x * a.y) * il;
      }
    }
    ar[j] = (i == j) ? make_float2(d * il, 0.f) : ((i > j) ? lij : ar[j]);
  }
  if (row) {
#pragma unroll
    for (int j = 0; j < KT; ++j) Am[i * AS + j] = ar[j];   // row i of L
  }
  __syncwarp();
  // Column i of L^-1 by forward substitution with pending sums: once y_j is known, every
  // later row r gets pend[r] += L[r][j] y_j (independent updates, broadcast loads).
  float2 yc[KT], pend[KT];
#pragma unroll
  for (int r = 0; r < KT; ++r) pend[r] = make_float2(0.f, 0.f);
  float sk = 0.f;
#pragma unroll
  for (int j = 0; j < KT; ++j) {
    const float il = inv_l[j];
    yc[j] = (j == i) ? make_float2(il, 0.f)
                     : ((j > i) ? make_float2(-pend[j].x * il, -pend[j].y * il) : make_float2(0.f, 0.f));
    sk = fmaf(yc[j].x, yc[j].x, fmaf(yc[j].y, yc[j].y, sk));
#pragma unroll
    for (int r = j + 1; r < KT; ++r) cmac(pend[r], Am[r * AS + j], yc[j]);
  }
  __syncwarp();
  if (row) {
#pragma unroll
    for (int j = 0; j < KT; ++j) Am[j * AS + i] = yc[j];   // L^-1[j][i]
  }
  if (live) Ss[i * XS + scl] = P.sigma2 * sk;
  if (i == 0) Is[scl] = fail;
  if (FIX && i == 0 && P.fix_count && k0 + scl < N && (fail != 0 || dmax > P.cond_limit * dmin)) {
    const int slot = atomicAdd(P.fix_count, 1);              // (max L_jj / min L_jj)^2 <= cond(A)
    if (slot < P.fix_cap) P.fix_list[slot] = t * N + k0 + scl;
  }
  __syncwarp();
  // w_i = sum_{l <= i} L^-1[i][l] z_l (row i of L^-1 first, then the broadcast z reads).
  float2 yrow[KT], wr[DT];
#pragma unroll
  for (int l = 0; l < KT; ++l) yrow[l] = live ? Am[i * AS + l] : make_float2(0.f, 0.f);
#pragma unroll
  for (int n = 0; n < DT; ++n) wr[n] = make_float2(0.f, 0.f);
#pragma unroll
  for (int l = 0; l < KT; ++l) {
    if (l < K) {
#pragma unroll
      for (int n = 0; n < DT; ++n) cmac(wr[n], yrow[l], Zm[l * DT + n]);
    }
  }
  __syncwarp();
  if (live) {
#pragma unroll
    for (int n = 0; n < DT; ++n) Zm[i * DT + n] = wr[n];
  }
  __syncwarp();
  // x~_i = sum_{j >= i} conj(L^-1[j][i]) w_j  (column i of L^-1 is still in yc).
  float2 xr[DT];
#pragma unroll
  for (int n = 0; n < DT; ++n) xr[n] = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < KT; ++j) {
    if (j < K) {
#pragma unroll
      for (int n = 0; n < DT; ++n) cmac_conj(xr[n], yc[j], Zm[j * DT + n]);
    }
  }
  if (live) {
#pragma unroll
    for (int n = 0; n < DT; ++n)
      if (n < D) Xs[(n * KT + i) * XS + scl] = xr[n];
  }
}

// w = L^-1 r and x~ += L^-H w for subcarrier scl, with the columns of L^-1 in As (as left by
// det_factor_solve) and the right-hand sides r in Zs (overwritten by w).
template <int KT, int DT>
__device__ __forceinline__ void det_solve_add(const int i, const int scl, const int K, const int D, const float2* As,
                                              float2* Zs, float2* Xs) {
  constexpr int AS = KT + 1;
  constexpr int XS = DET_SC + 1;
  const bool live = i < K;
  const float2* Am = As + scl * KT * AS;
  float2* Zm = Zs + scl * KT * DT;
  float2 wr[DT];
#pragma unroll
  for (int n = 0; n < DT; ++n) wr[n] = make_float2(0.f, 0.f);
#pragma unroll
  for (int l = 0; l < KT; ++l) {
    if (l < K && live && l <= i) {
      const float2 a = Am[i * AS + l];                         // L^-1[i][l]
#pragma unroll
      for (int n = 0; n < DT; ++n) cmac(wr[n], a, Zm[l * DT + n]);
    }
  }
  __syncwarp();
  if (live) {
#pragma unroll
    for (int n = 0; n < DT; ++n) Zm[i * DT + n] = wr[n];
  }
  __syncwarp();
  float2 xr[DT];
#pragma unroll
  for (int n = 0; n < DT; ++n) xr[n] = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < KT; ++j) {
    if (j < K && live) {
      const float2 c = Am[j * AS + i];                         // L^-1[j][i], zero above the diagonal
#pragma unroll
      for (int n = 0; n < DT; ++n) cmac_conj(xr[n], c, Zm[j * DT + n]);
    }
  }
  if (live) {
#pragma unroll
    for (int n = 0; n < DT; ++n)
      if (n < D) {
        float2& x = Xs[(n * KT + i) * XS + scl];
        x.x += xr[n].x;
        x.y += xr[n].y;
      }
  }
}

// Demap the tile's x~ (Xs, with s in Ss) and store x_eq, labels and LLRs with coalesced
// writes, all threads of the CTA.
template <int KT, int DT>
__device__ __forceinline__ void det_demap_store(const int t, const int k0, const int K, const int D, const int N,
                                                const int q, const float2* Xs, const float* Ss, float2* x_eq,
                                                unsigned char* labels, float* llr) {
  constexpr int XS = DET_SC + 1;
  // Thread -> subcarrier scx and a group g of (symbol, user) rows; rows advance by the
  // group count (no division by K), and each 16-lane group writes 16 consecutive entries.
  {
    const int scx = threadIdx.x % DET_SC, g0 = threadIdx.x / DET_SC, G = blockDim.x / DET_SC;
    const int kg = k0 + scx;
    if (kg < N && g0 < G) {
      int n = 0, k = g0;
      while (k >= K) { k -= K; ++n; }
      for (; n < D;) {
        const float2 xt = Xs[(n * KT + k) * XS + scx];
        const size_t o = (size_t(t * D + n) * K + k) * N + kg;
        x_eq[o] = xt;
        if (llr) {
          const float s = Ss[k * XS + scx];
          switch (q) {
            case 2: demap_store<1>(xt, s, o, labels, llr); break;
            case 4: demap_store<2>(xt, s, o, labels, llr); break;
            default: demap_store<3>(xt, s, o, labels, llr); break;
          }
        } else if (labels) {
          const float s = Ss[k * XS + scx];
          switch (q) {
            case 2: labels[o] = hard_label<1>(xt, s); break;
            case 4: labels[o] = hard_label<2>(xt, s); break;
            default: labels[o] = hard_label<3>(xt, s); break;
          }
        }
        k += G;
        while (k >= K) { k -= K; ++n; }
      }
    }
  }
}

// ------------------------------------------------------------------------ kernel
// MODE DET_FIX compiles in the FP64 fallback of the precision form (flagging and the last
// CTA's solves), so the FP32 path carries none of that code; DET_FUSED is the fused
// receive form (TMA only).
template <int KT, int DT, bool USE_TMA, int MODE>
__global__ void __launch_bounds__(det_max_threads(KT, DT), 1)
    detect_kernel(const __grid_constant__ CUtensorMap map_h, const __grid_constant__ CUtensorMap map_y,
                  const float2* __restrict__ h, const float2* __restrict__ y,
                  float2* __restrict__ x_eq, unsigned char* __restrict__ labels,
                  float* __restrict__ llr, int* __restrict__ info, const __grid_constant__ DetParams P) {
  constexpr bool FIX = MODE == DET_FIX;
  constexpr bool FUSED = MODE == DET_FUSED;
  static_assert(!FUSED || USE_TMA, "the fused form streams through TMA");
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
  int* s_abort = reinterpret_cast<int*>(smem + 128);
  int* s_issued = reinterpret_cast<int*>(smem + 144);   // loads the producer issued
  float2* stage0 = reinterpret_cast<float2*>(smem + 1024);

  if (P.skip_if_set && *reinterpret_cast<const volatile int*>(P.skip_if_set) != 0) return;   // uniform per CTA
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const int t = blockIdx.y, k0 = blockIdx.x * DET_SC;
  const int K = P.K, D = P.D, M = P.M, N = P.N;
  const int KP = P.tiles.KP, DP = P.tiles.DP;
  constexpr int PL = DET_MCH * DET_SC;                 // one operand row of a stage
  const int span = FUSED ? P.span : 0;
  const int yoff = FUSED ? K * DET_MCH * span : KP * PL;        // data rows within a stage
  const int stage_elems = yoff + DP * PL;
  const int nst = USE_TMA ? (FUSED ? P.nst : DET_STAGES) : 1;
  float2* hs = stage0 + size_t(nst) * stage_elems;     // fused: filtered chunk [2][KP][PL]
  float2* wps = hs + 2 * KP * PL;                      // fused: weights [K][DET_SC][16]
  const int x0 = FUSED ? (k0 / P.B) * P.B : k0;        // first subcarrier of a pilot box

  // Zero the padding rows (users K..KP-1, symbols D..DP-1) of every stage once; the
  // loads never write them.  (Fused: the user padding lives in the filtered chunk.)
  for (int s = 0; s < nst; ++s) {
    float2* st = stage0 + s * stage_elems;
    if (!FUSED)
      for (int e = threadIdx.x; e < (KP - K) * PL; e += blockDim.x) st[K * PL + e] = make_float2(0.f, 0.f);
    for (int e = threadIdx.x; e < (DP - D) * PL; e += blockDim.x) st[yoff + D * PL + e] = make_float2(0.f, 0.f);
  }
  if (FUSED)
    for (int e = threadIdx.x; e < 2 * (KP - K) * PL; e += blockDim.x) {
      const int b = e / ((KP - K) * PL), r = e % ((KP - K) * PL);
      hs[b * KP * PL + K * PL + r] = make_float2(0.f, 0.f);
    }
  // Consumer warps (one or two per role) and, on the TMA path, one producer warp (the last).
  const int n_cons = P.tiles.n_roles * P.tiles.msplit;
  uint64_t* full = bars;                      // [DET_STAGES] TMA bytes landed
  uint64_t* empty = bars + DET_STAGES;        // [DET_STAGES] every consumer warp is done
  if (threadIdx.x == 0) {
    *s_abort = 0;
    *s_issued = 0;
    if (USE_TMA) {
      for (int s = 0; s < DET_STAGES; ++s) {
        mbar_init(&full[s], 1);
        mbar_init(&empty[s], n_cons);
      }
      fence_mbar_init();
    }
  }
  __syncthreads();

  const uint32_t stage_tx = uint32_t((FUSED ? K * DET_MCH * span + D * PL : (K + D) * PL) * sizeof(float2));
  if (USE_TMA && warp == n_cons) {
    // Producer: stream every antenna chunk through the stage ring.
    if (lane == 0) {
      prefetch_tensormap(&map_h);
      prefetch_tensormap(&map_y);
      int issued = 0;
      for (int c = 0; c < P.nchunks && !P.stall_producer; ++c) {
        const int s = c % nst;
        if (c >= nst && !mbar_wait_rounds(&empty[s], uint32_t(c / nst - 1) & 1u, P.wait_rounds)) {
          atomicExch(s_abort, 1);
          break;
        }
        float2* st = stage0 + s * stage_elems;
        mbar_arrive_expect_tx(&full[s], stage_tx);
        tma_load_3d(st, &map_h, &full[s], x0, c * DET_MCH, t * K);
        tma_load_3d(st + yoff, &map_y, &full[s], k0, c * DET_MCH, t * D);
        ++issued;
      }
      *s_issued = issued;
    }
    __syncwarp();
  }

  // ------------------------------------------------ accumulation: Gram and z
  const int R = P.tiles.n_roles;
  const int role = warp % R, mg = warp / R;
  const int kind = P.tiles.kind[role], rg = P.tiles.g[role], rr = P.tiles.r[role], rc = P.tiles.c[role];
  const int sc = lane & 15, mh = lane >> 4;
  const int per = DET_MCH / (2 * P.tiles.msplit);      // antennas of a chunk per half-warp
  const int m_first = (mg * 2 + mh) * per;
  float2 acc[26];
#pragma unroll
  for (int e = 0; e < 26; ++e) acc[e] = make_float2(0.f, 0.f);

  const bool consumer = warp < n_cons;
  // Fused form: the LS-folded weights of the tile, wps[k][j][i] = W[j'][i] conj(p_i) / |p_i|^2
  // for output subcarrier k0 + j at position j' of its block (zero past the block's length
  // and past n_sc), and each lane's input offset within the pilot box.
  int off_j = 0;
  if constexpr (FUSED) {
    if (consumer) {
      for (int e = threadIdx.x; e < K * DET_SC * 16; e += n_cons * 32) {
        const int k = e >> 8, j = (e >> 4) & 15, i = e & 15;
        const int kg = k0 + j;
        float2 v = make_float2(0.f, 0.f);
        if (kg < N) {
          const int b = kg / P.B, jp = kg - b * P.B;
          const bool full_blk = b < P.nfull;
          if (i < (full_blk ? P.B : P.tail)) {
            const float2 w = full_blk ? P.w_main[jp * P.B + i] : P.w_tail[jp * P.tail + i];
            const float2 pl = P.pil[size_t(t * K + k) * N + b * P.B + i];
            const float inv = 1.0f / fmaf(pl.x, pl.x, pl.y * pl.y);
            v = make_float2(fmaf(w.x, pl.x, w.y * pl.y) * inv, fmaf(w.y, pl.x, -w.x * pl.y) * inv);
          }
        }
        wps[e] = v;
      }
      if (k0 + sc < N) off_j = ((k0 + sc) / P.B) * P.B - x0;
      named_bar_sync(1, n_cons * 32);
    }
  }
  float2 wp[16];                                       // fused: weight row of user cur_k
  int cur_k = -1;
  bool aborted = false;

  for (int c = 0; c < P.nchunks; ++c) {
    const int s = USE_TMA ? (c % nst) : 0;
    float2* st = stage0 + s * stage_elems;
    if (USE_TMA) {
      if (!consumer) break;
      if constexpr (FUSED) {
        // Every consumer warp passes the named barrier of every chunk, so a wait that ran
        // out marks the warp aborted instead of leaving the loop.
        bool ok = !aborted && !*reinterpret_cast<volatile int*>(s_abort) &&
                  mbar_wait_rounds(&full[s], uint32_t(c / nst) & 1u, P.wait_rounds);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) {
          if (!aborted && lane == 0) atomicExch(s_abort, 1);
          aborted = true;
        }
      } else if (!mbar_wait_rounds(&full[s], uint32_t(c / nst) & 1u, P.wait_rounds)) {
        atomicExch(s_abort, 1);
        break;
      }
    } else {
      // Plain loads with bounds checks (odd n_sc or unaligned pointers), all threads.
      const int m0 = c * DET_MCH;
      for (int e = threadIdx.x; e < (K + D) * PL; e += blockDim.x) {
        const int op = e / PL, rem = e % PL;
        const int m = m0 + rem / DET_SC, k = k0 + rem % DET_SC;
        float2 v = make_float2(0.f, 0.f);
        if (m < M && k < N)
          v = (op < K) ? h[(size_t(t * K + op) * M + m) * N + k] : y[(size_t(t * D + op - K) * M + m) * N + k];
        const int dst = (op < K) ? op : KP + (op - K);
        st[dst * PL + rem] = v;
      }
      __syncthreads();
    }
    const float2* hsrc = st;                           // the chunk's h rows [KP][PL]
    if constexpr (FUSED) {
      // LS + LMMSE of the chunk: half-warp g takes a run of U consecutive units u = (user
      // u/2, antenna parity u%2) of 4 rows, so that its users (and weight rows) change
      // little; lane sc owns output subcarrier k0 + sc.  The two half-warps of a warp read
      // adjacent rows, which sit on different banks (span % 16 != 0).
      float2* hb = hs + (c & 1) * KP * PL;
      if (!aborted) {
        const int U = (2 * K + 2 * n_cons - 1) / (2 * n_cons), g = warp * 2 + mh;
        for (int i = 0; i < U; ++i) {
          // odd half-warps take each user's parities in the other order (adjacent rows again)
          const int u = g * U + ((U & 1) ? i : (i ^ (g & 1)));
          if (u >= 2 * K) continue;
          const int k = u >> 1, par = u & 1;
          if (k != cur_k) {
            const float4* wr = reinterpret_cast<const float4*>(wps + (k * DET_SC + sc) * 16);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const float4 v = wr[i];
              wp[2 * i] = make_float2(v.x, v.y);
              wp[2 * i + 1] = make_float2(v.z, v.w);
            }
            cur_k = k;
          }
          float2 a[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) a[r] = make_float2(0.f, 0.f);
          const float2* src = st + (k * DET_MCH + par) * span + off_j;
#pragma unroll
          for (int i = 0; i < 16; i += 2) {
            if (i < P.B) {
#pragma unroll
              for (int r = 0; r < 4; ++r) {
                const float4 v = *reinterpret_cast<const float4*>(src + 2 * r * span + i);
                cmac(a[r], wp[i], make_float2(v.x, v.y));
                cmac(a[r], wp[i + 1], make_float2(v.z, v.w));
              }
            }
          }
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const int m = par + 2 * r;
            hb[k * PL + m * DET_SC + sc] = a[r];
            if (P.h_out) {
              const int mgl = c * DET_MCH + m, kg = k0 + sc;
              if (kg < N && mgl < M) P.h_out[(size_t(t * K + k) * M + mgl) * N + kg] = a[r];
            }
          }
        }
      }
      named_bar_sync(1, n_cons * 32);
      hsrc = hb;
    }
    if (consumer && !aborted) {
      const float2* sl = hsrc + sc;
      const float2* yl = st + yoff + sc;
#pragma unroll
      for (int mm = 0; mm < DET_MCH / 2; ++mm) {
        if (mm < per) {
          const int mo = (m_first + mm) * DET_SC;
          if (kind == 2) {
            float2 a4[4], y6[6];
#pragma unroll
            for (int ii = 0; ii < 4; ++ii) a4[ii] = sl[(4 * rg + ii) * PL + mo];
#pragma unroll
            for (int jj = 0; jj < 6; ++jj) y6[jj] = yl[(6 * rc + jj) * PL + mo];
#pragma unroll
            for (int ii = 0; ii < 4; ++ii)
#pragma unroll
              for (int jj = 0; jj < 6; ++jj) cmac_conj(acc[ii * 6 + jj], a4[ii], y6[jj]);
          } else {
            if (kind == 0) {
              float2 t4[4];
#pragma unroll
              for (int ii = 0; ii < 4; ++ii) t4[ii] = sl[(4 * rg + ii) * PL + mo];
#pragma unroll
              for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                for (int jj = 0; jj <= ii; ++jj) cmac_conj(acc[ii * (ii + 1) / 2 + jj], t4[ii], t4[jj]);
            }
            if (rr >= 0) {
              float2 r4[4], c4[4];
#pragma unroll
              for (int ii = 0; ii < 4; ++ii) r4[ii] = sl[(4 * rr + ii) * PL + mo];
#pragma unroll
              for (int jj = 0; jj < 4; ++jj) c4[jj] = sl[(4 * rc + jj) * PL + mo];
#pragma unroll
              for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) cmac_conj(acc[10 + ii * 4 + jj], r4[ii], c4[jj]);
            }
          }
        }
      }
    }
    if (USE_TMA) {
      __syncwarp();
      if (lane == 0 && !aborted) mbar_arrive(&empty[s]);   // this warp is done with the stage
    } else {
      __syncthreads();
    }
  }
  // FP64 fallback (precision form): every CTA counts itself done; the last one re-solves
  // the flagged subcarriers (process) and clears the list for the next launch.
  int* s_last = reinterpret_cast<int*>(smem + 136);
  auto finish_fix = [&](bool process) {
    if constexpr (!FIX) return;
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
                       P.T, K, M, N, D, P.q, P.sigma2_d};
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
    // A pipeline wait ran out: give the copies in flight a bounded chance to land,
    // record the timeout and leave without touching the outputs.
    if (threadIdx.x == 0) {
      // Load j of stage s completes phase j / nst: wait for the last one of each stage.
      const int issued = USE_TMA ? *s_issued : 0;
      for (int s = 0; s < nst && s < issued; ++s)
        (void)mbar_wait_bounded(&full[s], uint32_t((issued - 1 - s) / nst) & 1u);
      atomicExch(P.status, int(RAPRO_ERR_TIMEOUT));
    }
    finish_fix(false);
    return;
  }

  // ---------------- partial sums -> A (+ sigma2 I, lower triangle) and z
  constexpr int AS = KT + 1;                                    // padded row stride
  constexpr int XS = DET_SC + 1;
  float2* As = stage0;                                          // [DET_SC][KT][AS]: A, then L, then L^-1
  float2* Zs = stage0 + det_off_z(KT);                          // [DET_SC][KT][DT]: z, then w
  float2* Xs = stage0 + det_off_x(KT, DT);                      // [DT][KT][XS]: x~
  float* Ss = reinterpret_cast<float*>(stage0 + det_off_s(KT, DT));   // [KT][XS]: s_k
  int* Is = reinterpret_cast<int*>(Ss + KT * XS);              // [DET_SC]: info
  float2* Cb = stage0 + det_off_col(KT, DT);                    // [DET_SC][2][16]: column broadcast
  float2* park = stage0 + det_off_park(KT, DT);                 // [warp][DET_SC][26]
  if (consumer) {
    float2* pw = park + size_t(warp) * DET_SC * 26 + sc * 26;
    if (mh == 1) {
#pragma unroll
      for (int e = 0; e < 26; ++e) pw[e] = acc[e];
    }
    __syncwarp();
    if (mh == 0) {
#pragma unroll
      for (int e = 0; e < 26; ++e) {
        const float2 o = pw[e];
        acc[e].x += o.x;
        acc[e].y += o.y;
      }
    }
  }
  if (P.tiles.msplit == 2) {
    __syncthreads();                       // every warp has read its own slot
    if (consumer && mg == 1 && mh == 0) {
      float2* pw = park + size_t(role) * DET_SC * 26 + sc * 26;
#pragma unroll
      for (int e = 0; e < 26; ++e) pw[e] = acc[e];
    }
    __syncthreads();
    if (consumer && mg == 0 && mh == 0) {
      const float2* pw = park + size_t(role) * DET_SC * 26 + sc * 26;
#pragma unroll
      for (int e = 0; e < 26; ++e) {
        const float2 o = pw[e];
        acc[e].x += o.x;
        acc[e].y += o.y;
      }
    }
  }
  if (consumer && mg == 0 && mh == 0) {
    if (kind == 2) {
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int jj = 0; jj < 6; ++jj) {
          const int i = 4 * rg + ii, n = 6 * rc + jj;
          if (i < K && n < D) Zs[(sc * KT + i) * DT + n] = acc[ii * 6 + jj];
        }
    } else {
      if (kind == 0) {
#pragma unroll
        for (int ii = 0; ii < 4; ++ii)
#pragma unroll
          for (int jj = 0; jj <= ii; ++jj) {
            const int i = 4 * rg + ii, j = 4 * rg + jj;
            float2 v = acc[ii * (ii + 1) / 2 + jj];
            if (ii == jj) v.x += P.sigma2;
            if (i < K) As[(sc * KT + i) * AS + j] = v;
          }
      }
      if (rr >= 0) {
#pragma unroll
        for (int ii = 0; ii < 4; ++ii)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int i = 4 * rr + ii, j = 4 * rc + jj;
            if (i < K && j < K) As[(sc * KT + i) * AS + j] = acc[10 + ii * 4 + jj];
          }
      }
    }
  }
  __syncthreads();

  // --------------------------------------------- factorisation and solves
  // Every CTA has at least DET_SC / 2 warps, so each half-warp takes at most one subcarrier
  // (a single pass keeps the row arrays in registers).  Lane i owns row i.
  const int hw = lane >> 4, i = lane & 15;
  const int scl = warp * 2 + hw;
  if (scl < DET_SC) det_factor_solve<KT, DT, FIX>(i, scl, K, D, t, k0, N, P, As, Zs, Xs, Ss, Is, Cb);
  __syncthreads();

  // ------------------------------------------------ demap and coalesced stores
  det_demap_store<KT, DT>(t, k0, K, D, N, P.q, Xs, Ss, x_eq, labels, llr);
  if (info && threadIdx.x < DET_SC && k0 + threadIdx.x < N) info[size_t(t) * N + k0 + threadIdx.x] = Is[threadIdx.x];
  finish_fix(true);
}

template <int KT>
cudaError_t detect_launch_kt(const DetLaunch& L);

template <int KT>
cudaError_t detect_prepare_kt(int smem, int fused_smem);

// One explicit specialisation per padded user count, each in its own translation unit.
template <> cudaError_t detect_launch_kt<4>(const DetLaunch& L);
template <> cudaError_t detect_launch_kt<8>(const DetLaunch& L);
template <> cudaError_t detect_launch_kt<12>(const DetLaunch& L);
template <> cudaError_t detect_launch_kt<16>(const DetLaunch& L);
template <> cudaError_t detect_prepare_kt<4>(int smem, int fused_smem);
template <> cudaError_t detect_prepare_kt<8>(int smem, int fused_smem);
template <> cudaError_t detect_prepare_kt<12>(int smem, int fused_smem);
template <> cudaError_t detect_prepare_kt<16>(int smem, int fused_smem);

// Definitions, instantiated once per KT in its own translation unit.
#define RAPRO_DETECT_DEFINE_KT(KTV)                                                                    \
  template <>                                                                                          \
  cudaError_t detect_launch_kt<KTV>(const DetLaunch& L) {                                              \
    dim3 grid((L.P.N + DET_SC - 1) / DET_SC, L.P.T);                                                   \
    dim3 block(det_block_threads(L.P.tiles));                                                          \
    const int v = (L.P.D > 6 ? 1 : 0) + (L.tma ? 2 : 0) + (L.P.fix_count ? 4 : 0);                    \
    if (L.fused) {                                                                                     \
      if (L.P.D > 6) RAPRO_DETECT_GO(KTV, 12, true, DET_FUSED);                                        \
      else RAPRO_DETECT_GO(KTV, 6, true, DET_FUSED);                                                   \
      return cudaGetLastError();                                                                       \
    }                                                                                                  \
    switch (v) {                                                                                       \
      case 0: RAPRO_DETECT_GO(KTV, 6, false, DET_PLAIN); break;                                        \
      case 1: RAPRO_DETECT_GO(KTV, 12, false, DET_PLAIN); break;                                       \
      case 2: RAPRO_DETECT_GO(KTV, 6, true, DET_PLAIN); break;                                         \
      case 3: RAPRO_DETECT_GO(KTV, 12, true, DET_PLAIN); break;                                        \
      case 4: RAPRO_DETECT_GO(KTV, 6, false, DET_FIX); break;                                          \
      case 5: RAPRO_DETECT_GO(KTV, 12, false, DET_FIX); break;                                         \
      case 6: RAPRO_DETECT_GO(KTV, 6, true, DET_FIX); break;                                           \
      default: RAPRO_DETECT_GO(KTV, 12, true, DET_FIX); break;                                         \
    }                                                                                                  \
    return cudaGetLastError();                                                                         \
  }                                                                                                    \
  template <>                                                                                          \
  cudaError_t detect_prepare_kt<KTV>(int smem, int fused_smem) {                                       \
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;                           \
    cudaError_t e = cudaFuncSetAttribute(detect_kernel<KTV, 6, true, DET_PLAIN>, A, smem);             \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(detect_kernel<KTV, 12, true, DET_PLAIN>, A, smem);  \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(detect_kernel<KTV, 6, false, DET_PLAIN>, A, smem);  \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(detect_kernel<KTV, 12, false, DET_PLAIN>, A, smem); \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(detect_kernel<KTV, 6, true, DET_FIX>, A, smem);     \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(detect_kernel<KTV, 12, true, DET_FIX>, A, smem);    \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(detect_kernel<KTV, 6, false, DET_FIX>, A, smem);    \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(detect_kernel<KTV, 12, false, DET_FIX>, A, smem);   \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(detect_kernel<KTV, 6, true, DET_FUSED>, A, fused_smem);  \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(detect_kernel<KTV, 12, true, DET_FUSED>, A, fused_smem); \
    return e;                                                                                          \
  }

#define RAPRO_DETECT_GO(KTV, DTV, TMA, MODEV)                                                           \
  detect_kernel<KTV, DTV, TMA, MODEV><<<grid, block, L.smem, L.stream>>>(L.map_h, L.map_y, L.h, L.y,   \
                                                                         L.x_eq, L.labels, L.llr,      \
                                                                         L.info, L.P)

}  // namespace rapro
