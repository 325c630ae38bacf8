// Channel estimation kernels: LS (Eq. 9) and the sub-block LMMSE filter (Eq. 12, 17).
//
// Data: rows r = (slot t, user s, antenna m) of n_sc complex64 subcarriers each; block b
// covers subcarriers [b*B, b*B + B_b) with B_b = B, or n_sc mod B for the last block.
// The filter is out[r][blk] = W_b * in[r][blk]: for every block a complex
// (rows x B_b) x (B_b x B_b)^T product, FP32 FFMA with FP32 accumulation.
#include <algorithm>
#include <mutex>

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
// One CTA per segment of up to SEG_BLOCKS blocks of one row (t, s, m).  The segment's
// subcarriers arrive with coalesced loads (LS applied on the way in) into shared memory,
// one padded slot of BM + 1 entries per block (conflict-free per half-warp); each thread
// then filters one block from registers with the weights in the kernel parameters, so
// every W[i][j] is a constant-bank operand of the FFMAs, and writes it back in place; the
// segment leaves with coalesced stores.
constexpr int SEG_BLOCKS = 128;
constexpr int SMALL_THREADS = 128;

template <int BM>
struct WSmall {
  float2 w[BM * BM];   // full-size block, zero padded to BM x BM
  float2 wt[BM * BM];  // tail block, zero padded
};

// acc = W v with the input index outermost, so the BM accumulators update independently.
template <int BM>
__device__ __forceinline__ void apply_w(const float2 (&W)[BM * BM], const float2 (&v)[BM],
                                        float2 (&acc)[BM]) {
#pragma unroll
  for (int i = 0; i < BM; ++i) acc[i] = make_float2(0.f, 0.f);
#pragma unroll
  for (int j = 0; j < BM; ++j)
#pragma unroll
    for (int i = 0; i < BM; ++i) cmac(acc[i], W[i * BM + j], v[j]);
}

template <int BM, bool LS>
__global__ void __launch_bounds__(SMALL_THREADS) lmmse_small_kernel(const float2* __restrict__ x,
                                                                    const float2* __restrict__ pil,
                                                                    float2* __restrict__ out, int M, int N,
                                                                    int B, int nb, int tail,
                                                                    const __grid_constant__ WSmall<BM> W) {
  __shared__ float2 xs[SEG_BLOCKS * (BM + 1)];
  const int row = blockIdx.y;
  const int b0 = blockIdx.x * SEG_BLOCKS;
  const int nbl = min(SEG_BLOCKS, nb - b0);
  const int e0 = b0 * B;
  const int n_el = min(N - e0, nbl * B);
  const float2* xr = x + size_t(row) * N + e0;
  const float2* pr = pil + size_t(row / M) * N + e0;
  float2* orow = out + size_t(row) * N + e0;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int dblk = nt / B, dj = nt % B;

  {  // element e of the segment -> (block e / B, offset e % B), tracked incrementally
    int blk = tid / B, j = tid % B;
#pragma unroll 4
    for (int e = tid; e < n_el; e += nt) {
      float2 v = xr[e];
      if (LS) {
        const float2 p = pr[e];
        const float inv = 1.0f / fmaf(p.x, p.x, p.y * p.y);
        v = make_float2(fmaf(v.x, p.x, v.y * p.y) * inv, fmaf(v.y, p.x, -v.x * p.y) * inv);
      }
      xs[blk * (BM + 1) + j] = v;
      blk += dblk;
      j += dj;
      if (j >= B) { j -= B; ++blk; }
    }
  }
  __syncthreads();
  for (int bl = tid; bl < nbl; bl += nt) {
    const int b = b0 + bl;
    const bool is_tail = (tail != 0) && (b == nb - 1);
    const int Bb = is_tail ? tail : B;
    float2 v[BM], acc[BM];
#pragma unroll
    for (int j = 0; j < BM; ++j) v[j] = (j < Bb) ? xs[bl * (BM + 1) + j] : make_float2(0.f, 0.f);
    if (!is_tail)
      apply_w<BM>(W.w, v, acc);
    else
      apply_w<BM>(W.wt, v, acc);
#pragma unroll
    for (int i = 0; i < BM; ++i)
      if (i < Bb) xs[bl * (BM + 1) + i] = acc[i];
  }
  __syncthreads();
  {
    int blk = tid / B, j = tid % B;
#pragma unroll 4
    for (int e = tid; e < n_el; e += nt) {
      orow[e] = xs[blk * (BM + 1) + j];
      blk += dblk;
      j += dj;
      if (j >= B) { j -= B; ++blk; }
    }
  }
}

// Streaming variant for rows that bulk copies can move (n_sc and B even, 16-byte aligned
// arrays, at most STREAM_MAX_THREADS blocks per row): one CTA filters STREAM_ROWS
// consecutive antenna rows of one (slot, user).  Its pilot row is loaded once and turned
// into conj(p) / |p|^2; row buffers are filled and drained by 1-D bulk copies in a
// STREAM_BUF-deep ring, so loads stay in flight while the CTA computes.  Thread b owns
// block b of every row and keeps that block's pilot factors in registers.
constexpr int STREAM_ROWS = 8;
constexpr int STREAM_BUF = 3;
constexpr int STREAM_MAX_THREADS = 512;
// Threads (= blocks per row) a streaming CTA may have for padded block size BM.
__host__ __device__ constexpr int stream_max_threads(int BM) { return BM <= 12 ? STREAM_MAX_THREADS : 256; }

template <int BM>
__device__ __forceinline__ void apply_stream(const WSmall<BM>& W, bool tail, const float2 (&v)[BM], float2 (&acc)[BM]) {
  if (!tail) apply_w<BM>(W.w, v, acc);
  else apply_w<BM>(W.wt, v, acc);
}

template <int BM>
__global__ void __launch_bounds__(stream_max_threads(BM)) lmmse_stream_kernel(
    const float2* __restrict__ y, const float2* __restrict__ pil, float2* __restrict__ out, int M, int N,
    int B, int nb, int tail, int* status, const __grid_constant__ WSmall<BM> W) {
  static_assert(BM % 2 == 0, "blocks move as pairs of complex values");
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);            // [0]: pilot, [1 + b]: row buffer b
  int* s_abort = reinterpret_cast<int*>(smem + 64);
  float2* pc = reinterpret_cast<float2*>(smem + 128);             // pilot row -> conj(p)/|p|^2
  float2* buf = pc + N;                                          // [STREAM_BUF][N]
  const int ts = blockIdx.y;                                     // t*K + s
  const int m0 = blockIdx.x * STREAM_ROWS;
  const int nrows = min(STREAM_ROWS, M - m0);
  const size_t row0 = size_t(ts) * M + m0;
  const uint32_t row_bytes = uint32_t(N) * sizeof(float2);
  const int tid = threadIdx.x;

  if (tid == 0) {
    *s_abort = 0;
    for (int b = 0; b <= STREAM_BUF; ++b) mbar_init(&bars[b], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (tid == 0) {
    mbar_arrive_expect_tx(&bars[0], row_bytes);
    bulk_load(pc, pil + size_t(ts) * N, row_bytes, &bars[0]);
    for (int r = 0; r < STREAM_BUF && r < nrows; ++r) {
      mbar_arrive_expect_tx(&bars[1 + r], row_bytes);
      bulk_load(buf + size_t(r) * N, y + (row0 + r) * N, row_bytes, &bars[1 + r]);
    }
  }
  const int b = tid;
  const bool active = b < nb;
  const bool is_tail = (tail != 0) && (b == nb - 1);
  const int Bb = is_tail ? tail : B;                             // even
  const int e0 = b * B;                                          // even
  float2 pcr[BM];
  if (!mbar_wait_bounded(&bars[0], 0)) atomicExch(s_abort, 1);
#pragma unroll
  for (int jp = 0; jp < BM / 2; ++jp) {
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    if (active && 2 * jp < Bb) q = reinterpret_cast<const float4*>(pc + e0)[jp];
    float inv = __fdividef(1.0f, fmaf(q.x, q.x, q.y * q.y));
    pcr[2 * jp] = (active && 2 * jp < Bb) ? make_float2(q.x * inv, -q.y * inv) : make_float2(0.f, 0.f);
    inv = __fdividef(1.0f, fmaf(q.z, q.z, q.w * q.w));
    pcr[2 * jp + 1] = (active && 2 * jp < Bb) ? make_float2(q.z * inv, -q.w * inv) : make_float2(0.f, 0.f);
  }
  for (int r = 0; r < nrows; ++r) {
    const int slot = r % STREAM_BUF;
    float2* row = buf + size_t(slot) * N;
    if (!mbar_wait_bounded(&bars[1 + slot], uint32_t(r / STREAM_BUF) & 1u)) atomicExch(s_abort, 1);
    if (active) {
      float2 v[BM], acc[BM];
      float4* row4 = reinterpret_cast<float4*>(row + e0);
#pragma unroll
      for (int jp = 0; jp < BM / 2; ++jp) {
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (2 * jp < Bb) q = row4[jp];
        const float2 c0 = pcr[2 * jp], c1 = pcr[2 * jp + 1];
        v[2 * jp] = make_float2(fmaf(q.x, c0.x, -q.y * c0.y), fmaf(q.x, c0.y, q.y * c0.x));
        v[2 * jp + 1] = make_float2(fmaf(q.z, c1.x, -q.w * c1.y), fmaf(q.z, c1.y, q.w * c1.x));
      }
      apply_stream<BM>(W, is_tail, v, acc);
#pragma unroll
      for (int jp = 0; jp < BM / 2; ++jp)
        if (2 * jp < Bb) row4[jp] = make_float4(acc[2 * jp].x, acc[2 * jp].y, acc[2 * jp + 1].x, acc[2 * jp + 1].y);
    }
    fence_proxy_async_shared();
    __syncthreads();
    if (*s_abort) {
      if (tid == 0) {
        bulk_wait_all();
        atomicExch(status, int(RAPRO_ERR_TIMEOUT));
      }
      return;
    }
    if (tid == 0) {
      bulk_store(out + (row0 + r) * N, row, row_bytes);
      bulk_commit();
      const int rn = r + STREAM_BUF;
      if (rn < nrows) {
        bulk_wait_read<0>();                 // the store of this buffer has read it
        mbar_arrive_expect_tx(&bars[1 + slot], row_bytes);
        bulk_load(row, y + (row0 + rn) * N, row_bytes, &bars[1 + slot]);
      }
    }
  }
  if (tid == 0) bulk_wait_all();
}

size_t lmmse_stream_smem(int N) { return 128 + size_t(N) * sizeof(float2) * (1 + STREAM_BUF); }

template <int BM>
static void fill_small(WSmall<BM>& W, const float2* w_main, const float2* w_tail, int B, int tail) {
  for (int i = 0; i < BM * BM; ++i) W.w[i] = W.wt[i] = make_float2(0.f, 0.f);
  for (int i = 0; i < B; ++i)
    for (int j = 0; j < B; ++j) W.w[i * BM + j] = w_main[size_t(i) * B + j];
  for (int i = 0; i < tail; ++i)
    for (int j = 0; j < tail; ++j) W.wt[i * BM + j] = w_tail[size_t(i) * tail + j];
}

static bool stream_ok(const float2* y, const float2* pil, const float2* out, int N, int B, int nb) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(pil) |
                      reinterpret_cast<uintptr_t>(out);
  const int bm = B <= 4 ? 4 : B <= 8 ? 8 : B <= 12 ? 12 : B <= 16 ? 16 : B <= 24 ? 24 : 32;
  return (a & 15) == 0 && N % 2 == 0 && B % 2 == 0 && nb <= stream_max_threads(bm) &&
         lmmse_stream_smem(N) <= size_t(200) * 1024;
}

template <int BM>
static cudaError_t launch_stream(const WSmall<BM>& W0, const float2* y, const float2* pil, float2* out,
                                 int T, int K, int M, int N, int B, int nb, int tail, int* status,
                                 cudaStream_t st) {
  const WSmall<BM>& W = W0;
  const size_t smem = lmmse_stream_smem(N);
  dim3 grid((M + STREAM_ROWS - 1) / STREAM_ROWS, T * K);
  const int threads = std::max(32, (nb + 31) / 32 * 32);
  lmmse_stream_kernel<BM><<<grid, threads, smem, st>>>(y, pil, out, M, N, B, nb, tail, status, W);
  return cudaGetLastError();
}

template <int BM>
static cudaError_t launch_small(const Plan& pl, const float2* x, const float2* pil, float2* out,
                                cudaStream_t st, bool allow_stream = true) {
  WSmall<BM> W;
  fill_small<BM>(W, pl.w_main.data(), pl.w_tail.data(), pl.B, pl.tail);
  if (allow_stream && pil && stream_ok(x, pil, out, pl.p.n_sc, pl.B, pl.nb))
    return launch_stream<BM>(W, x, pil, out, pl.T, pl.p.K, pl.p.M, pl.p.n_sc, pl.B, pl.nb, pl.tail,
                             pl.d_status, st);
  const int rows = pl.T * pl.p.K * pl.p.M;
  dim3 grid((pl.nb + SEG_BLOCKS - 1) / SEG_BLOCKS, rows);
  if (pil)
    lmmse_small_kernel<BM, true><<<grid, SMALL_THREADS, 0, st>>>(x, pil, out, pl.p.M, pl.p.n_sc, pl.B,
                                                                pl.nb, pl.tail, W);
  else
    lmmse_small_kernel<BM, false><<<grid, SMALL_THREADS, 0, st>>>(x, pil, out, pl.p.M, pl.p.n_sc, pl.B,
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
                                    const float2* pil, float2* out, int* status, cudaStream_t st) {
  WSmall<BM> W;
  fill_small<BM>(W, w_main, w_tail, B, tail);
  if (status && stream_ok(y, pil, out, N, B, nb))
    return launch_stream<BM>(W, y, pil, out, 1, rows / M, M, N, B, nb, tail, status, st);
  dim3 grid((nb + SEG_BLOCKS - 1) / SEG_BLOCKS, rows);
  lmmse_small_kernel<BM, true><<<grid, SMALL_THREADS, 0, st>>>(y, pil, out, M, N, B, nb, tail, W);
  return cudaGetLastError();
}

cudaError_t launch_ls_lmmse_small_raw(const float2* w_main, const float2* w_tail, int B, int tail,
                                      int nb, int rows, int M, int N, const float2* y,
                                      const float2* pil, float2* out, int* status, cudaStream_t st) {
  if (B <= 4) return launch_small_raw<4>(w_main, w_tail, B, tail, nb, rows, M, N, y, pil, out, status, st);
  if (B <= 8) return launch_small_raw<8>(w_main, w_tail, B, tail, nb, rows, M, N, y, pil, out, status, st);
  if (B <= 12) return launch_small_raw<12>(w_main, w_tail, B, tail, nb, rows, M, N, y, pil, out, status, st);
  if (B <= 16) return launch_small_raw<16>(w_main, w_tail, B, tail, nb, rows, M, N, y, pil, out, status, st);
  if (B <= 24) return launch_small_raw<24>(w_main, w_tail, B, tail, nb, rows, M, N, y, pil, out, status, st);
  if (B <= LMMSE_SMALL_MAX)
    return launch_small_raw<32>(w_main, w_tail, B, tail, nb, rows, M, N, y, pil, out, status, st);
  return cudaErrorInvalidValue;
}

// Raise the streaming kernels' dynamic shared-memory limit once per device, at plan
// creation (not at launch, which may be inside a CUDA-graph capture).
cudaError_t prepare_estimate(int device) {
  static std::once_flag flags[64];
  static cudaError_t result[64];
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  std::call_once(flags[device], [device] {
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    const int lim = 200 * 1024;
    cudaError_t e = cudaFuncSetAttribute(lmmse_stream_kernel<4>, A, lim);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lmmse_stream_kernel<8>, A, lim);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lmmse_stream_kernel<12>, A, lim);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lmmse_stream_kernel<16>, A, lim);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lmmse_stream_kernel<24>, A, lim);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(lmmse_stream_kernel<32>, A, lim);
    result[device] = e;
  });
  return result[device];
}

cudaError_t launch_lmmse(const Plan& pl, const float2* x, const float2* pil,
                         const float2* d_w_main, const float2* d_w_tail,
                         const float2* /*h_w_main*/, const float2* /*h_w_tail*/, float2* out,
                         cudaStream_t st) {
  // d_w_main != plan weights means a caller override with one W per block.
  const bool override_w = d_w_main != pl.d_w_main;
  if (override_w) return launch_tiled(pl, x, pil, d_w_main, nullptr, 1, out, st);
  return launch_lmmse_variant(pl, pl.est_variant, x, pil, out, st);
}

bool lmmse_variant_ok(const Plan& pl, int v, const float2* x, const float2* pil, const float2* out) {
  if (half_precision(pl.p))
    return (v == EST_TC && lmmse_tc_ok(pl, x, pil, out)) || (v == EST_TCG && pil && lmmse_tcg_ok(pl, x, out));
  switch (v) {
    case EST_TC: return lmmse_tc_ok(pl, x, pil, out);
    case EST_STREAM: return pil && pl.B <= LMMSE_SMALL_MAX && stream_ok(x, pil, out, pl.p.n_sc, pl.B, pl.nb);
    case EST_SMALL: return pl.B <= LMMSE_SMALL_MAX;
    case EST_TILED: return true;
    case EST_TCG: return lmmse_tcg_ok(pl, x, out);
    default: return false;
  }
}

// Variant v (EST_*), or the built-in choice for v < 0 or a variant that does not apply to
// these arrays: tensor cores, then the streaming / segment kernels, then the tiled one.
cudaError_t launch_lmmse_variant(const Plan& pl, int v, const float2* x, const float2* pil, float2* out,
                                 cudaStream_t st) {
  if (v < 0 || !lmmse_variant_ok(pl, v, x, pil, out)) {
    if (lmmse_tc_ok(pl, x, pil, out)) return launch_lmmse_tc(pl, x, pil, out, st);
    if (half_precision(pl.p))   // the 16-bit forms run on the tensor cores or not at all
      return pil && lmmse_tcg_ok(pl, x, out) ? launch_lmmse_tcg(pl, x, pil, out, st) : cudaErrorNotSupported;
    if (lmmse_tcg_ok(pl, x, out)) return launch_lmmse_tcg(pl, x, pil, out, st);
    v = pl.B <= LMMSE_SMALL_MAX ? EST_STREAM : EST_TILED;
  }
  if (v == EST_TC) return launch_lmmse_tc(pl, x, pil, out, st);
  if (v == EST_TCG) return launch_lmmse_tcg(pl, x, pil, out, st);
  if (v == EST_TILED) return launch_tiled(pl, x, pil, pl.d_w_main, pl.d_w_tail, 0, out, st);
  const bool stream = v == EST_STREAM;
  const int B = pl.B;
  if (B <= 4) return launch_small<4>(pl, x, pil, out, st, stream);
  if (B <= 8) return launch_small<8>(pl, x, pil, out, st, stream);
  if (B <= 12) return launch_small<12>(pl, x, pil, out, st, stream);
  if (B <= 16) return launch_small<16>(pl, x, pil, out, st, stream);
  if (B <= 24) return launch_small<24>(pl, x, pil, out, st, stream);
  return launch_small<32>(pl, x, pil, out, st, stream);
}

}  // namespace rapro
