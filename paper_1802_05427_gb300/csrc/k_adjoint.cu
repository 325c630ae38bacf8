// Reverse-mode derivative of the receive path's symbol MSE, L = mean |x~ - x|^2 over the
// data symbols, users and subcarriers (x known), for fitting the estimator's model
// parameters (Eq. 13/17) and the detector's sigma2 (Eq. 22).  Gradients are conjugate
// Wirtinger gradients G_X = dL/dX*, so that dL = 2 Re sum conj(G_X) dX.
//
// Detector (Eq. 22, per slot t and subcarrier n; A = H^H H + sigma2 I, x~_d = A^-1 H^H y_d):
//   g_d = (x~_d - x_d) / count,  lambda_d = A^-1 g_d,
//   G_H = sum_d y_d lambda_d^H - H C,   C = sum_d (lambda_d x~_d^H + x~_d lambda_d^H),
//   dL/dsigma2 = -2 Re sum_d lambda_d^H x~_d   (kernel in k_adj_detect.cu).
// Estimator (Eq. 12, per row (t, s, m) and block b; h_blk = W h_ls_blk):
//   G_W = sum_{rows, blocks} G_h,blk h_ls,blk^H   (one sum for the shared W, one for the tail).
#include <algorithm>
#include <cstdint>
#include <mutex>

#include "rapro_internal.h"
#include "rapro_ptx.cuh"

namespace rapro {

namespace {

constexpr int ADJ_THREADS = 256;
constexpr int ADJ_MAX_N = 2048;   // largest n_sc
constexpr int ADJ_MAX_B = 64;

struct AdjEstArgs {
  const float2* y;      // y_pilot [T][K][M][N]
  const float2* pil;    // [T][K][N]
  const float2* g_h;    // [T][K][M][N]
  float2* g_w;          // [Bb][Bb], accumulated with atomics
  int rows, M, N;       // rows = T K M
  int Bb, nb, col0;     // block width, blocks per row, first column of block 0
};

__device__ __forceinline__ void red_add_shared(uint32_t addr, float v) {
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}

// Sum of the CTA's SI x SJ register tiles into G_W: shuffles over the lanes that hold the
// same tile (when the Q tiles of a pair divide the warp), shared-space reductions issued in
// program order (one address register live at a time), then the caller's global atomics.
// `lanes_ok` marks the threads that own a tile; FULL: every tile lies inside the block.
template <int SI, int SJ, bool FULL>
__device__ __forceinline__ void add_tiles(float2 (&acc)[SI][SJ], float2* sw, int Bb, int Q, int qi, int qj,
                                          bool lanes_ok, bool split, int lane) {
  if (split) {
#pragma unroll
    for (int i = 0; i < SI; ++i)
#pragma unroll
      for (int j = 0; j < SJ; ++j)
        for (int o = Q; o < 32; o <<= 1) {
          acc[i][j].x += __shfl_xor_sync(0xffffffffu, acc[i][j].x, o);
          acc[i][j].y += __shfl_xor_sync(0xffffffffu, acc[i][j].y, o);
        }
  }
  if (lanes_ok && (!split || lane < Q)) {
    const uint32_t tile = smem_u32(sw) + uint32_t((qi * SI) * Bb + qj * SJ) * uint32_t(sizeof(float2));
#pragma unroll
    for (int i = 0; i < SI; ++i) {
      const uint32_t row = tile + uint32_t(i * Bb) * uint32_t(sizeof(float2));
#pragma unroll
      for (int j = 0; j < SJ; ++j)
        if (FULL || (qi * SI + i < Bb && qj * SJ + j < Bb)) {
          red_add_shared(row + j * sizeof(float2), acc[i][j].x);
          red_add_shared(row + j * sizeof(float2) + 4, acc[i][j].y);
        }
    }
  }
}

// Direct form, any block width: G_W += g_blk ls_blk^H over the (row, block) pairs.  A pair's
// Bb x Bb product is cut into Q = ceil(Bb / S)^2 tiles of S x S; the Q threads of a pair lane
// hold one tile each in registers and read their g, y and pilot elements straight from
// global memory.  Consecutive pair lanes take consecutive blocks of a row; a CTA walks a
// contiguous range of pairs.
template <int S>
__global__ void __launch_bounds__(ADJ_THREADS, 2) adj_lmmse_kernel(const AdjEstArgs a) {
  extern __shared__ float2 sw[];      // [Bb][Bb]
  const int Bb = a.Bb, nb = a.nb, tid = threadIdx.x;
  const int Bq = (Bb + S - 1) / S, Q = Bq * Bq, lanes = ADJ_THREADS / Q;
  const int pl = tid / Q, q = tid - pl * Q, qi = q / Bq, qj = q - qi * Bq;
  for (int e = tid; e < Bb * Bb; e += ADJ_THREADS) sw[e] = make_float2(0.f, 0.f);
  float2 acc[S][S];
#pragma unroll
  for (int i = 0; i < S; ++i)
#pragma unroll
    for (int j = 0; j < S; ++j) acc[i][j] = make_float2(0.f, 0.f);
  const long long P = (long long)a.rows * nb;
  const long long per_cta = (P + gridDim.x - 1) / gridDim.x;
  const long long p0 = blockIdx.x * per_cta, p1 = min(P, p0 + per_cta);
  if (pl < lanes && p0 + pl < p1) {
    long long p = p0 + pl;
    int r = int(p / nb), b = int(p - (long long)r * nb);
    const int dr = lanes / nb, db = lanes - dr * nb;
    for (; p < p1; p += lanes) {
      const size_t cb = size_t(a.col0) + size_t(b) * Bb;
      const float2* gr = a.g_h + size_t(r) * a.N + cb + qi * S;
      const float2* yr = a.y + size_t(r) * a.N + cb + qj * S;
      const float2* pr = a.pil + size_t(r / a.M) * a.N + cb + qj * S;
      float2 gi[S], yv[S], pv[S];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const bool in_i = qi * S + s < Bb, in_j = qj * S + s < Bb;
        gi[s] = in_i ? gr[s] : make_float2(0.f, 0.f);
        yv[s] = in_j ? yr[s] : make_float2(0.f, 0.f);
        pv[s] = in_j ? pr[s] : make_float2(1.f, 0.f);
      }
#pragma unroll
      for (int s = 0; s < S; ++s) {       // ls = y / p (Eq. 9)
        const float inv = __fdividef(1.0f, fmaf(pv[s].x, pv[s].x, pv[s].y * pv[s].y));
        const float2 y = yv[s], pp = pv[s];
        yv[s] = make_float2(fmaf(y.x, pp.x, y.y * pp.y) * inv, fmaf(y.y, pp.x, -y.x * pp.y) * inv);
      }
#pragma unroll
      for (int i = 0; i < S; ++i)
#pragma unroll
        for (int j = 0; j < S; ++j) cmac_conj(acc[i][j], yv[j], gi[i]);   // += g conj(ls)
      b += db;
      r += dr;
      if (b >= nb) { b -= nb; ++r; }
    }
  }
  __syncthreads();
  add_tiles<S, S, false>(acc, sw, Bb, Q, qi, qj, pl < lanes, (32 % Q) == 0, tid & 31);
  __syncthreads();
  for (int e = tid; e < Bb * Bb; e += ADJ_THREADS) {
    atomicAdd(&a.g_w[e].x, sw[e].x);
    atomicAdd(&a.g_w[e].y, sw[e].y);
  }
}

// Row form for Q <= 32 tiles per pair.  A pair's Bb x Bb product is cut into Q tiles of
// SI x SJ (SI rows of g, SJ columns of ls); lane (pair, tile) of a warp holds one tile, and a
// warp covers a chunk of up to ppw = floor(32 / Q) consecutive blocks of a row.  The row
// units are numbered (t, k, chunk, m) with m fastest and cut into equal contiguous runs, one
// per warp, so that consecutive units of a run share the pilots of (t, k, chunk): a lane
// keeps 1 / p of its SJ columns in registers and renews them only when the run enters the
// next (t, k, chunk).  Lane (pair, tile) loads its SI g and SJ y elements of a row straight
// into registers, ADJ_PF rows ahead of the row it multiplies, and the warp asks L2 for the
// row ADJ_L2_AHEAD units ahead, so that the bytes in flight do not depend on the registers.
// The tiles are summed once, when the run ends.  V4: 16-byte loads of g (SI even, Bb a
// multiple of SI and SJ, 16-byte aligned rows).
constexpr int ADJ_WARPS = ADJ_THREADS / 32;
constexpr int ADJ_PF = 2;          // rows held in registers ahead of the multiply
constexpr int ADJ_L2_AHEAD = 8;    // units ahead of the multiply that are prefetched to L2

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <int SI, int SJ, bool V4>
__global__ void __launch_bounds__(ADJ_THREADS, 2) adj_lmmse_rows_kernel(const AdjEstArgs a) {
  extern __shared__ __align__(16) float2 sw[];          // [Bb][Bb]
  const int Bb = a.Bb, nb = a.nb, M = a.M, N = a.N, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Bqi = (Bb + SI - 1) / SI, Bqj = (Bb + SJ - 1) / SJ, Q = Bqi * Bqj, ppw = 32 / Q;
  const int cpr = (nb + ppw - 1) / ppw;                 // chunks per row
  const int pp = lane / Q, q = lane - pp * Q, qi = q / Bqj, qj = q - qi * Bqj;
  for (int e = tid; e < Bb * Bb; e += ADJ_THREADS) sw[e] = make_float2(0.f, 0.f);
  float2 acc[SI][SJ];
#pragma unroll
  for (int i = 0; i < SI; ++i)
#pragma unroll
    for (int j = 0; j < SJ; ++j) acc[i][j] = make_float2(0.f, 0.f);
  __syncthreads();                                      // sw is zero before any task ends
  const int U = (a.rows / M) * cpr * M;                 // < 2^31: checked by the launcher
  const int nw = gridDim.x * ADJ_WARPS, per_w = (U + nw - 1) / nw;
  const int u0 = min(U, (int(blockIdx.x) * ADJ_WARPS + warp) * per_w), n = min(U, u0 + per_w) - u0;
  // Start of task tkc's chunk in its antenna row m = 0 (elements), and its number of blocks.
  auto task_base = [&](int tkc, size_t& off, int& nv) {
    const int tk = tkc / cpr, c = tkc - tk * cpr;
    off = size_t(tk) * M * N + a.col0 + size_t(c) * ppw * Bb;
    nv = min(ppw, nb - c * ppw);
  };
  int ltk = 0, lm = 0, lnv = 0;                         // next unit to load: task, antenna, blocks
  size_t loff = 0;                                      // its chunk's first element
  float2 lw[SJ];                                        // 1 / p of the lane's columns there
  auto task_pilots = [&]() {
    const int tk = ltk / cpr, c = ltk - tk * cpr;
    const float2* pr = a.pil + size_t(tk) * N + a.col0 + size_t(c * ppw + pp) * Bb + qj * SJ;
#pragma unroll
    for (int s = 0; s < SJ; ++s) {
      const bool live = pp < lnv && (V4 || qj * SJ + s < Bb);
      const float2 p = live ? __ldg(pr + s) : make_float2(1.f, 0.f);
      const float inv = live ? __fdividef(1.0f, fmaf(p.x, p.x, p.y * p.y)) : 0.f;   // dead lane: ls = 0
      lw[s] = make_float2(p.x * inv, -p.y * inv);
    }
  };
  int ptk = 0, pm = 0, pnv = 0;                         // next unit to prefetch to L2
  size_t poff = 0;
  float2 G[ADJ_PF][SI], Y[ADJ_PF][SJ];
  auto load = [&](float2 (&g)[SI], float2 (&y)[SJ]) {
    // A lane past the chunk's last block reads that block (in bounds) and has ls = 0.
    const size_t at = loff + size_t(min(pp, lnv - 1)) * Bb;
    const float2* gr = a.g_h + at + qi * SI;
    const float2* yr = a.y + at + qj * SJ;
    if (V4) {
#pragma unroll
      for (int s = 0; s < SI; s += 2) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(gr + s));
        g[s] = make_float2(v.x, v.y);
        g[s + 1] = make_float2(v.z, v.w);
      }
#pragma unroll
      for (int s = 0; s < SJ; ++s) y[s] = __ldg(yr + s);
    } else {
#pragma unroll
      for (int s = 0; s < SI; ++s) g[s] = qi * SI + s < Bb ? __ldg(gr + s) : make_float2(0.f, 0.f);
#pragma unroll
      for (int s = 0; s < SJ; ++s) y[s] = qj * SJ + s < Bb ? __ldg(yr + s) : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int s = 0; s < SJ; ++s) y[s] = cmul(y[s], lw[s]);   // ls = y / p (Eq. 9)
    loff += N;
    if (++lm == M) {
      lm = 0;
      task_base(++ltk, loff, lnv);
      task_pilots();
    }
  };
  // Lanes 0..15 touch the unit's g run every 128 bytes and at its last byte, lanes 16..31
  // its y run.
  auto prefetch_unit = [&]() {
    const int bytes = pnv * Bb * int(sizeof(float2)), at = (lane & 15) * 128;
    const char* base = reinterpret_cast<const char*>((lane < 16 ? a.g_h : a.y) + poff);
    if (at < bytes + 127) prefetch_l2(base + min(at, bytes - 1));   // addresses inside the run
    poff += N;
    if (++pm == M) {
      pm = 0;
      task_base(++ptk, poff, pnv);
    }
  };
  if (n > 0) {
    ltk = ptk = u0 / M;
    lm = pm = u0 - ltk * M;
    task_base(ltk, loff, lnv);
    task_pilots();
    loff += size_t(lm) * N;
    task_base(ptk, poff, pnv);
    poff += size_t(pm) * N;
    for (int k = 0; k < ADJ_L2_AHEAD && k < n; ++k) prefetch_unit();
#pragma unroll
    for (int s = 0; s < ADJ_PF; ++s)
      if (s < n) load(G[s], Y[s]);
    for (int k0 = 0; k0 < n; k0 += ADJ_PF) {
#pragma unroll
      for (int s = 0; s < ADJ_PF; ++s) {
        const int k = k0 + s;
        if (k < n) {
#pragma unroll
          for (int i = 0; i < SI; ++i)
#pragma unroll
            for (int j = 0; j < SJ; ++j) cmac_conj(acc[i][j], Y[s][j], G[s][i]);   // += g conj(ls)
          if (k + ADJ_PF < n) load(G[s], Y[s]);
          if (k + ADJ_L2_AHEAD < n) prefetch_unit();
        }
      }
    }
  }
  add_tiles<SI, SJ, V4>(acc, sw, Bb, Q, qi, qj, pp < ppw, (32 % Q) == 0, lane);
  __syncthreads();
  for (int e = tid; e < Bb * Bb; e += ADJ_THREADS) {
    atomicAdd(&a.g_w[e].x, sw[e].x);
    atomicAdd(&a.g_w[e].y, sw[e].y);
  }
}

template <int SI, int SJ>
bool rows_fit(const AdjEstArgs& a) {
  const int Bqi = (a.Bb + SI - 1) / SI, Bqj = (a.Bb + SJ - 1) / SJ;
  return a.nb > 1 && Bqi * Bqj <= 32 && (long long)a.rows * a.nb < (1LL << 31);
}

template <int SI, int SJ>
cudaError_t launch_rows(const AdjEstArgs& a, int ctas, int sms, cudaStream_t st) {
  const auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  const bool v4 = SI % 2 == 0 && a.Bb % SI == 0 && a.Bb % SJ == 0 && al16(a.g_h) && a.N % 2 == 0 &&
                  a.col0 % 2 == 0;
  const size_t smem = size_t(a.Bb) * a.Bb * sizeof(float2);
  ctas = std::min(ctas, 2 * sms);                   // one wave: each warp walks one run of units
  if (v4)
    adj_lmmse_rows_kernel<SI, SJ, true><<<ctas, ADJ_THREADS, smem, st>>>(a);
  else
    adj_lmmse_rows_kernel<SI, SJ, false><<<ctas, ADJ_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

// Row form with 6 x 3 tiles where they tile the block (Bb a multiple of 6), else 4 x 4; the
// direct form where a pair needs more than 32 tiles or a row holds a single block.
cudaError_t launch_adj_lmmse(const AdjEstArgs& a, int ctas, int sms, cudaStream_t st) {
  const size_t smem = size_t(a.Bb) * a.Bb * sizeof(float2);
  if (a.Bb % 6 == 0 && rows_fit<6, 3>(a)) return launch_rows<6, 3>(a, ctas, sms, st);
  if (rows_fit<4, 4>(a)) return launch_rows<4, 4>(a, ctas, sms, st);
  if (a.Bb == 6 || a.Bb == 12 || a.Bb == 24)
    adj_lmmse_kernel<6><<<ctas, ADJ_THREADS, smem, st>>>(a);
  else
    adj_lmmse_kernel<4><<<ctas, ADJ_THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace

int adjoint_max_block() { return ADJ_MAX_B; }
int adjoint_max_subcarriers() { return ADJ_MAX_N; }

cudaError_t launch_adjoint(const Plan& pl, const float2* y_pilot, const float2* pilots, const float2* y_data,
                           const float2* h, const float2* x_eq, const float2* x_ref, float2* g_h, float* scal,
                           float2* g_wm, float2* g_wt, cudaStream_t st) {
  const rapro_params& p = pl.p;
  const int T = pl.T, K = p.K, M = p.M, N = p.n_sc;
  cudaError_t e;
  if ((e = cudaMemsetAsync(scal, 0, 2 * sizeof(float), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(g_wm, 0, size_t(pl.B) * pl.B * sizeof(float2), st)) != cudaSuccess) return e;
  if (pl.tail && (e = cudaMemsetAsync(g_wt, 0, size_t(pl.tail) * pl.tail * sizeof(float2), st)) != cudaSuccess)
    return e;
  if ((e = launch_adj_detect(pl, h, y_data, x_eq, x_ref, g_h, scal, st)) != cudaSuccess) return e;
  static std::once_flag once[64];
  static int sm_count[64];
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::call_once(once[dev], [dev] {
    sm_count[dev] = 148;
    cudaDeviceGetAttribute(&sm_count[dev], cudaDevAttrMultiProcessorCount, dev);
  });
  const int sms = sm_count[dev], rows = T * K * M, nbf = N / pl.B;
  const long long pairs = (long long)rows * nbf;
  const int ctas = int(std::min<long long>(2LL * sms, std::max<long long>(1, pairs / 64)));
  if (nbf > 0 &&
      (e = launch_adj_lmmse(AdjEstArgs{y_pilot, pilots, g_h, g_wm, rows, M, N, pl.B, nbf, 0}, ctas, sms, st)) !=
          cudaSuccess)
    return e;
  if (pl.tail) {
    const int tctas = std::max(1, std::min(2 * sms, rows / 64));
    if ((e = launch_adj_lmmse(AdjEstArgs{y_pilot, pilots, g_h, g_wt, rows, M, N, pl.tail, 1, nbf * pl.B}, tctas,
                              sms, st)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

cudaError_t prepare_adjoint(int device) { return prepare_adj_detect(device); }

}  // namespace rapro
