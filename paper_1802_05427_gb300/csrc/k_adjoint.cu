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
#include <mutex>

#include "rapro_internal.h"

namespace rapro {

namespace {

constexpr int ADJ_EST_UNROLL = 4;
constexpr int ADJ_THREADS = 256;
constexpr int ADJ_ROWS = 4;       // estimator rows staged at a time
constexpr int ADJ_MAX_N = 2048;   // largest n_sc
constexpr int ADJ_MAX_B = 64;
constexpr int ADJ_W_PER_THREAD = ADJ_MAX_B * ADJ_MAX_B / ADJ_THREADS;

__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {     // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

struct AdjEstArgs {
  const float2* y;      // y_pilot [T][K][M][N]
  const float2* pil;    // [T][K][N]
  const float2* g_h;    // [T][K][M][N]
  float2* g_wm;         // [B][B]
  float2* g_wt;         // [tail][tail] or null
  int rows, M, N, B, nbf, tail;   // rows = T K M; nbf = full blocks
};

// Rows are staged in shared memory ADJ_ROWS at a time.  B <= 16: thread (i, lane) owns
// row i of G_W for the (row, block) pairs lane, lane + L, ... (L = 256 / B lanes), so each
// pair costs it 1 + B shared loads and B complex MACs; the lanes' partial rows are summed
// through shared memory at the end.  16 < B <= 64: thread per entry of G_W.
constexpr int ADJ_FAST_B = 16;

__global__ void __launch_bounds__(ADJ_THREADS, 2) adj_lmmse_kernel(const AdjEstArgs a) {
  extern __shared__ float2 sm[];
  const int N = a.N, B = a.B, tail = a.tail, tid = threadIdx.x;
  float2* gh = sm;                       // [ADJ_ROWS][N]
  float2* ls = sm + ADJ_ROWS * N;        // [ADJ_ROWS][N]
  float2* part = ls + ADJ_ROWS * N;      // [L][B][B] lane partials (fast path)
  const bool fast = B <= ADJ_FAST_B;
  const int L = fast ? ADJ_THREADS / B : 1;
  const int fi = tid % B, lane = tid / B;          // fast path: row of G_W, lane
  float2 acc[ADJ_FAST_B];
#pragma unroll
  for (int j = 0; j < ADJ_FAST_B; ++j) acc[j] = make_float2(0.f, 0.f);
  float2 am[ADJ_W_PER_THREAD], at[ADJ_W_PER_THREAD];
#pragma unroll
  for (int q = 0; q < ADJ_W_PER_THREAD; ++q) am[q] = at[q] = make_float2(0.f, 0.f);
  const int per_cta = ADJ_ROWS * ((a.rows + ADJ_ROWS * gridDim.x - 1) / (ADJ_ROWS * gridDim.x));
  const int r_begin = blockIdx.x * per_cta, r_end = min(a.rows, r_begin + per_cta);
  for (int r0 = r_begin; r0 < r_end; r0 += ADJ_ROWS) {
    const int nr = min(ADJ_ROWS, r_end - r0);
    for (int base = tid; base < nr * N; base += blockDim.x * ADJ_EST_UNROLL) {
      float2 gv[ADJ_EST_UNROLL], yv[ADJ_EST_UNROLL], pv[ADJ_EST_UNROLL];
#pragma unroll
      for (int u = 0; u < ADJ_EST_UNROLL; ++u) {
        const int e = base + u * blockDim.x;
        gv[u] = yv[u] = make_float2(0.f, 0.f);
        pv[u] = make_float2(1.f, 0.f);
        if (e < nr * N) {
          const int rr = e / N, n = e - rr * N, r = r0 + rr;
          gv[u] = a.g_h[size_t(r) * N + n];
          yv[u] = a.y[size_t(r) * N + n];
          pv[u] = a.pil[size_t(r / a.M) * N + n];
        }
      }
#pragma unroll
      for (int u = 0; u < ADJ_EST_UNROLL; ++u) {
        const int e = base + u * blockDim.x;
        if (e < nr * N) {
          const float2 p = pv[u], y = yv[u];
          const float inv = __fdividef(1.0f, fmaf(p.x, p.x, p.y * p.y));
          gh[e] = gv[u];
          ls[e] = make_float2(fmaf(y.x, p.x, y.y * p.y) * inv, fmaf(y.y, p.x, -y.x * p.y) * inv);  // Eq. 9
        }
      }
    }
    __syncthreads();
    if (fast) {
      if (lane < L) {
        const int pairs = nr * a.nbf;
        for (int q = lane; q < pairs; q += L) {
          const int rr = q / a.nbf, b = q - rr * a.nbf;
          const float2 g = gh[rr * N + b * B + fi];
          const float2* x = ls + rr * N + b * B;
#pragma unroll
          for (int j = 0; j < ADJ_FAST_B; ++j)
            if (j < B) acc[j] = cadd(acc[j], cmulc(g, x[j]));
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < ADJ_W_PER_THREAD; ++q) {
        const int e = tid + q * ADJ_THREADS;
        if (e < B * B) {
          const int i = e / B, j = e - i * B;
          float2 sacc = am[q];
          for (int rr = 0; rr < nr; ++rr)
            for (int b = 0; b < a.nbf; ++b) sacc = cadd(sacc, cmulc(gh[rr * N + b * B + i], ls[rr * N + b * B + j]));
          am[q] = sacc;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < ADJ_W_PER_THREAD; ++q) {     // the tail block
      const int e = tid + q * ADJ_THREADS;
      if (e < tail * tail) {
        const int i = e / tail, j = e - i * tail, b0 = a.nbf * B;
        for (int rr = 0; rr < nr; ++rr) at[q] = cadd(at[q], cmulc(gh[rr * N + b0 + i], ls[rr * N + b0 + j]));
      }
    }
    __syncthreads();
  }
  if (fast) {
    if (lane < L) {
#pragma unroll
      for (int j = 0; j < ADJ_FAST_B; ++j)
        if (j < B) part[(lane * B + fi) * B + j] = acc[j];
    }
    __syncthreads();
    for (int e = tid; e < B * B; e += blockDim.x) {
      float2 sum = make_float2(0.f, 0.f);
      for (int l = 0; l < L; ++l) sum = cadd(sum, part[l * B * B + e]);
      atomicAdd(&a.g_wm[e].x, sum.x);
      atomicAdd(&a.g_wm[e].y, sum.y);
    }
  } else {
#pragma unroll
    for (int q = 0; q < ADJ_W_PER_THREAD; ++q) {
      const int e = tid + q * ADJ_THREADS;
      if (e < B * B) {
        atomicAdd(&a.g_wm[e].x, am[q].x);
        atomicAdd(&a.g_wm[e].y, am[q].y);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < ADJ_W_PER_THREAD; ++q) {
    const int e = tid + q * ADJ_THREADS;
    if (e < tail * tail) {
      atomicAdd(&a.g_wt[e].x, at[q].x);
      atomicAdd(&a.g_wt[e].y, at[q].y);
    }
  }
}

size_t adj_est_smem(int N, int B) {
  const size_t lanes = B <= ADJ_FAST_B ? size_t(ADJ_THREADS / B) : 0;
  return (2 * size_t(ADJ_ROWS) * N + lanes * B * B) * sizeof(float2);
}

}  // namespace

int adjoint_max_block() { return ADJ_MAX_B; }
int adjoint_max_subcarriers() { return ADJ_MAX_N; }

cudaError_t launch_adjoint(const Plan& pl, const float2* y_pilot, const float2* pilots, const float2* y_data,
                           const float2* h, const float2* x_eq, const float2* x_ref, float2* g_h, float* scal,
                           float2* g_wm, float2* g_wt, cudaStream_t st) {
  const rapro_params& p = pl.p;
  const int T = pl.T, D = pl.D, K = p.K, M = p.M, N = p.n_sc;
  cudaError_t e;
  if ((e = cudaMemsetAsync(scal, 0, 2 * sizeof(float), st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(g_wm, 0, size_t(pl.B) * pl.B * sizeof(float2), st)) != cudaSuccess) return e;
  if (pl.tail && (e = cudaMemsetAsync(g_wt, 0, size_t(pl.tail) * pl.tail * sizeof(float2), st)) != cudaSuccess)
    return e;
  if ((e = launch_adj_detect(pl, h, y_data, x_eq, x_ref, g_h, scal, st)) != cudaSuccess) return e;
  AdjEstArgs ae{y_pilot, pilots, g_h, g_wm, g_wt, T * K * M, M, N, pl.B, N / pl.B, pl.tail};
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int row_groups = (T * K * M + ADJ_ROWS - 1) / ADJ_ROWS;
  adj_lmmse_kernel<<<std::min(row_groups, 2 * sms), ADJ_THREADS, adj_est_smem(N, pl.B), st>>>(ae);
  return cudaGetLastError();
}

cudaError_t prepare_adjoint(int device) {
  static std::once_flag flags[64];
  static cudaError_t result[64];
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  std::call_once(flags[device], [device] {
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = prepare_adj_detect(device);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(adj_lmmse_kernel, A, int(adj_est_smem(ADJ_MAX_N, ADJ_FAST_B)));
    result[device] = e;
  });
  return result[device];
}

}  // namespace rapro
