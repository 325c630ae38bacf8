// Channel estimation kernels: LS (Eq. 9) and the sub-block LMMSE filter (Eq. 12, 17).
//
// Data: rows r = (slot t, user s, antenna m) of n_sc complex64 subcarriers each; block b
// covers subcarriers [b*B, b*B + B_b) with B_b = B, or n_sc mod B for the last block.
// The filter is out[r][blk] = W_b * in[r][blk]: for every block a complex
// (rows x B_b) x (B_b x B_b)^T product, FP32 FFMA with FP32 accumulation.
#include <algorithm>

#include "rapro_internal.h"
#include "rapro_ptx.cuh"

namespace rapro {

// ----------------------------------------------------------------------------- LS
// h = y conj(p) / |p|^2 on every (t, s, m, k); one thread per subcarrier of one row.
__global__ void __launch_bounds__(256) ls_kernel(const float2* y, const float2* __restrict__ pil,
                                                 float2* h, int M, int N) {
  const int row = blockIdx.y;                       // (t*K + s)*M + m
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const size_t i = size_t(row) * N + k;
  const float2 p = pil[size_t(row / M) * N + k];
  const float2 v = y[i];
  const float inv = 1.0f / fmaf(p.x, p.x, p.y * p.y);
  h[i] = make_float2(fmaf(v.x, p.x, v.y * p.y) * inv, fmaf(v.y, p.x, -v.x * p.y) * inv);
}

cudaError_t launch_ls(const float2* y, const float2* pil, float2* h, int T, int K, int M, int N,
                      cudaStream_t st) {
  const int rows = T * K * M;
  if (rows == 0 || N == 0) return cudaSuccess;
  dim3 grid((N + 255) / 256, rows);
  ls_kernel<<<grid, 256, 0, st>>>(y, pil, h, M, N);
  return cudaGetLastError();
}

// ----------------------------------------------------- LMMSE, small blocks (B <= 32)
// The block's weights travel in the kernel parameters, so every W[i][j] is a
// constant-bank operand of the FFMAs and costs no load instruction.  One thread filters
// one block of one row; lanes are consecutive rows, so pilots (same user) broadcast.
template <int BM>
struct WSmall {
  float2 w[BM * BM];   // full-size block, zero padded to BM x BM
  float2 wt[BM * BM];  // tail block, zero padded
};

template <int BM>
__device__ __forceinline__ void apply_w(const float2 (&W)[BM * BM], const float2 (&v)[BM],
                                        float2 (&acc)[BM]) {
#pragma unroll
  for (int i = 0; i < BM; ++i) {
    float2 a = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < BM; ++j) cmac(a, W[i * BM + j], v[j]);
    acc[i] = a;
  }
}

template <int BM, bool LS>
__global__ void __launch_bounds__(256) lmmse_small_kernel(const float2* __restrict__ x,
                                                          const float2* __restrict__ pil,
                                                          float2* __restrict__ out, int rows,
                                                          int M, int N, int B, int nb, int tail,
                                                          const __grid_constant__ WSmall<BM> W) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (row >= rows) return;
  const bool is_tail = (tail != 0) && (b == nb - 1);
  const int Bb = is_tail ? tail : B;
  const size_t base = size_t(row) * N + size_t(b) * B;
  float2 v[BM];
#pragma unroll
  for (int j = 0; j < BM; ++j) v[j] = (j < Bb) ? x[base + j] : make_float2(0.f, 0.f);
  if (LS) {
    const size_t pb = size_t(row / M) * N + size_t(b) * B;
#pragma unroll
    for (int j = 0; j < BM; ++j) {
      if (j < Bb) {
        const float2 p = pil[pb + j];
        const float inv = 1.0f / fmaf(p.x, p.x, p.y * p.y);
        const float2 y = v[j];
        v[j] = make_float2(fmaf(y.x, p.x, y.y * p.y) * inv, fmaf(y.y, p.x, -y.x * p.y) * inv);
      }
    }
  }
  float2 acc[BM];
  if (!is_tail)
    apply_w<BM>(W.w, v, acc);
  else
    apply_w<BM>(W.wt, v, acc);
#pragma unroll
  for (int i = 0; i < BM; ++i)
    if (i < Bb) out[base + i] = acc[i];
}

template <int BM>
static cudaError_t launch_small(const Plan& pl, const float2* x, const float2* pil, float2* out,
                                cudaStream_t st) {
  WSmall<BM> W;
  for (int i = 0; i < BM * BM; ++i) W.w[i] = W.wt[i] = make_float2(0.f, 0.f);
  for (int i = 0; i < pl.B; ++i)
    for (int j = 0; j < pl.B; ++j) W.w[i * BM + j] = pl.w_main[size_t(i) * pl.B + j];
  for (int i = 0; i < pl.tail; ++i)
    for (int j = 0; j < pl.tail; ++j) W.wt[i * BM + j] = pl.w_tail[size_t(i) * pl.tail + j];
  const int rows = pl.T * pl.p.K * pl.p.M;
  dim3 grid((rows + 127) / 128, pl.nb);
  if (pil)
    lmmse_small_kernel<BM, true><<<grid, 128, 0, st>>>(x, pil, out, rows, pl.p.M, pl.p.n_sc, pl.B,
                                                      pl.nb, pl.tail, W);
  else
    lmmse_small_kernel<BM, false><<<grid, 128, 0, st>>>(x, pil, out, rows, pl.p.M, pl.p.n_sc, pl.B,
                                                       pl.nb, pl.tail, W);
  return cudaGetLastError();
}

// ------------------------------------------------------ LMMSE, tiled (any block size)
// CTA tile: 64 rows x 64 outputs of one block, k-loop over the block's inputs in steps
// of 16.  Thread (tx, ty) owns rows ty + 16 ii and outputs tx + 16 kk (ii, kk < 4), so
// the shared-memory reads of W are conflict-free and the stores are coalesced.
// per_block: block b's W sits at w + b*B*B (tail after the full blocks); otherwise all
// full blocks share w and the tail uses wt.
template <bool LS>
__global__ void __launch_bounds__(256) lmmse_tiled_kernel(const float2* __restrict__ x,
                                                          const float2* __restrict__ pil,
                                                          float2* __restrict__ out,
                                                          const float2* __restrict__ w,
                                                          const float2* __restrict__ wt,
                                                          int per_block, int rows, int M, int N,
                                                          int B, int nb, int tail) {
  constexpr int TM = 64, TN = 64, TK = 16;
  __shared__ float2 Xs[TK][TM + 1];
  __shared__ float2 Ws[TK][TN + 1];
  const int b = blockIdx.z;
  const bool is_tail = (tail != 0) && (b == nb - 1);
  const int Bb = is_tail ? tail : B;
  const float2* Wb = per_block ? (w + size_t(b) * B * B) : (is_tail ? wt : w);
  const int row0 = blockIdx.x * TM, i0 = blockIdx.y * TN;
  if (i0 >= Bb) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const size_t colbase = size_t(b) * B;
  float2 acc[4][4];
#pragma unroll
  for (int ii = 0; ii < 4; ++ii)
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) acc[ii][kk] = make_float2(0.f, 0.f);

  for (int j0 = 0; j0 < Bb; j0 += TK) {
    for (int e = tid; e < TM * TK; e += 256) {
      const int r = e / TK, jj = e % TK;
      const int row = row0 + r, j = j0 + jj;
      float2 v = make_float2(0.f, 0.f);
      if (row < rows && j < Bb) {
        v = x[size_t(row) * N + colbase + j];
        if (LS) {
          const float2 p = pil[size_t(row / M) * N + colbase + j];
          const float inv = 1.0f / fmaf(p.x, p.x, p.y * p.y);
          v = make_float2(fmaf(v.x, p.x, v.y * p.y) * inv, fmaf(v.y, p.x, -v.x * p.y) * inv);
        }
      }
      Xs[jj][r] = v;
    }
    for (int e = tid; e < TN * TK; e += 256) {
      const int c = e / TK, jj = e % TK;
      const int i = i0 + c, j = j0 + jj;
      Ws[jj][c] = (i < Bb && j < Bb) ? Wb[size_t(i) * Bb + j] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < TK; ++jj) {
      float2 a[4], wv[4];
#pragma unroll
      for (int ii = 0; ii < 4; ++ii) a[ii] = Xs[jj][ty + 16 * ii];
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) wv[kk] = Ws[jj][tx + 16 * kk];
#pragma unroll
      for (int ii = 0; ii < 4; ++ii)
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) cmac(acc[ii][kk], wv[kk], a[ii]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int ii = 0; ii < 4; ++ii) {
    const int row = row0 + ty + 16 * ii;
    if (row >= rows) continue;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const int i = i0 + tx + 16 * kk;
      if (i < Bb) out[size_t(row) * N + colbase + i] = acc[ii][kk];
    }
  }
}

static cudaError_t launch_tiled(const Plan& pl, const float2* x, const float2* pil, const float2* w,
                                const float2* wt, int per_block, float2* out, cudaStream_t st) {
  const int rows = pl.T * pl.p.K * pl.p.M;
  dim3 grid((rows + 63) / 64, (pl.B + 63) / 64, pl.nb);
  if (pil)
    lmmse_tiled_kernel<true><<<grid, 256, 0, st>>>(x, pil, out, w, wt, per_block, rows, pl.p.M,
                                                   pl.p.n_sc, pl.B, pl.nb, pl.tail);
  else
    lmmse_tiled_kernel<false><<<grid, 256, 0, st>>>(x, pil, out, w, wt, per_block, rows, pl.p.M,
                                                    pl.p.n_sc, pl.B, pl.nb, pl.tail);
  return cudaGetLastError();
}

// Small-block LS + LMMSE without a plan: host weights w_main (B x B) and w_tail
// (tail x tail), row-major.  Used by the allocation-free receive entry point.
template <int BM>
static cudaError_t launch_small_raw(const float2* w_main, const float2* w_tail, int B, int tail,
                                    int nb, int rows, int M, int N, const float2* y,
                                    const float2* pil, float2* out, cudaStream_t st) {
  WSmall<BM> W;
  for (int i = 0; i < BM * BM; ++i) W.w[i] = W.wt[i] = make_float2(0.f, 0.f);
  for (int i = 0; i < B; ++i)
    for (int j = 0; j < B; ++j) W.w[i * BM + j] = w_main[i * B + j];
  for (int i = 0; i < tail; ++i)
    for (int j = 0; j < tail; ++j) W.wt[i * BM + j] = w_tail[i * tail + j];
  dim3 grid((rows + 127) / 128, nb);
  lmmse_small_kernel<BM, true><<<grid, 128, 0, st>>>(y, pil, out, rows, M, N, B, nb, tail, W);
  return cudaGetLastError();
}

cudaError_t launch_ls_lmmse_small_raw(const float2* w_main, const float2* w_tail, int B, int tail,
                                      int nb, int rows, int M, int N, const float2* y,
                                      const float2* pil, float2* out, cudaStream_t st) {
  if (B <= 4) return launch_small_raw<4>(w_main, w_tail, B, tail, nb, rows, M, N, y, pil, out, st);
  if (B <= 8) return launch_small_raw<8>(w_main, w_tail, B, tail, nb, rows, M, N, y, pil, out, st);
  if (B <= 12) return launch_small_raw<12>(w_main, w_tail, B, tail, nb, rows, M, N, y, pil, out, st);
  if (B <= 16) return launch_small_raw<16>(w_main, w_tail, B, tail, nb, rows, M, N, y, pil, out, st);
  if (B <= 24) return launch_small_raw<24>(w_main, w_tail, B, tail, nb, rows, M, N, y, pil, out, st);
  if (B <= LMMSE_SMALL_MAX)
    return launch_small_raw<32>(w_main, w_tail, B, tail, nb, rows, M, N, y, pil, out, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_lmmse(const Plan& pl, const float2* x, const float2* pil,
                         const float2* d_w_main, const float2* d_w_tail,
                         const float2* /*h_w_main*/, const float2* /*h_w_tail*/, float2* out,
                         cudaStream_t st) {
  // d_w_main != plan weights means a caller override with one W per block.
  const bool override_w = d_w_main != pl.d_w_main;
  if (override_w) return launch_tiled(pl, x, pil, d_w_main, nullptr, 1, out, st);
  const int B = pl.B;
  if (B <= 4) return launch_small<4>(pl, x, pil, out, st);
  if (B <= 8) return launch_small<8>(pl, x, pil, out, st);
  if (B <= 12) return launch_small<12>(pl, x, pil, out, st);
  if (B <= 16) return launch_small<16>(pl, x, pil, out, st);
  if (B <= 24) return launch_small<24>(pl, x, pil, out, st);
  if (B <= LMMSE_SMALL_MAX) return launch_small<32>(pl, x, pil, out, st);
  return launch_tiled(pl, x, pil, d_w_main, d_w_tail, 0, out, st);
}

}  // namespace rapro
