// Reverse-mode derivative of the receive path's symbol MSE, L = mean |x~ - x|^2 over the
// data symbols, users and subcarriers (x known), for fitting the estimator's model
// parameters (Eq. 13/17) and the detector's sigma2 (Eq. 22).  Gradients are conjugate
// Wirtinger gradients G_X = dL/dX*, so that dL = 2 Re sum conj(G_X) dX.
//
// Detector (Eq. 22, per slot t and subcarrier n; A = H^H H + sigma2 I, x~_d = A^-1 H^H y_d):
//   g_d = (x~_d - x_d) / count,  lambda_d = A^-1 g_d,
//   G_H = sum_d y_d lambda_d^H - H C,   C = sum_d (lambda_d x~_d^H + x~_d lambda_d^H),
//   dL/dsigma2 = -2 Re sum_d lambda_d^H x~_d.
// Estimator (Eq. 12, per row (t, s, m) and block b; h_blk = W h_ls_blk):
//   G_W = sum_{rows, blocks} G_h,blk h_ls,blk^H   (one sum for the shared W, one for the tail).
#include <algorithm>
#include <mutex>

#include "rapro_internal.h"

namespace rapro {

namespace {

constexpr int ADJ_SC = 16;        // subcarriers per detector-adjoint CTA
constexpr int ADJ_MC = 8;         // antennas per staged chunk
constexpr int ADJ_THREADS = 256;
constexpr int ADJ_ROWS = 16;      // estimator rows per CTA
constexpr int ADJ_MAXK = 16;
constexpr int ADJ_GRAM_PER_THREAD = (ADJ_SC * ADJ_MAXK * (ADJ_MAXK + 1) / 2 + ADJ_THREADS - 1) / ADJ_THREADS;
constexpr int ADJ_MAX_B = 64;
constexpr int ADJ_W_PER_THREAD = ADJ_MAX_B * ADJ_MAX_B / ADJ_THREADS;

__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {     // a * conj(b)
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cmul_(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

struct AdjDetArgs {
  const float2* h;      // [T][K][M][N]
  const float2* y;      // [T*D][M][N]
  const float2* x_eq;   // [T*D][K][N]
  const float2* x_ref;  // [T*D][K][N]
  float2* g_h;          // [T][K][M][N]
  float* scal;          // [0] += loss, [1] += dL/dsigma2 (detector)
  int K, M, N, D;
  float sigma2, scale;  // scale = 1 / (T D K N)
};

// Lower-triangle pair index -> (i, j), i >= j.
__device__ __forceinline__ void tri_pair(int p, int& i, int& j) {
  i = 0;
  while ((i + 1) * (i + 2) / 2 <= p) ++i;
  j = p - i * (i + 1) / 2;
}

__global__ void __launch_bounds__(ADJ_THREADS) adj_detect_kernel(const AdjDetArgs a) {
  extern __shared__ float2 sm[];
  const int K = a.K, M = a.M, N = a.N, D = a.D;
  const int t = blockIdx.y, k0 = blockIdx.x * ADJ_SC, tid = threadIdx.x;
  float2* Hc = sm;                                   // [K][ADJ_MC][ADJ_SC]
  float2* Yc = Hc + K * ADJ_MC * ADJ_SC;             // [D][ADJ_MC][ADJ_SC]
  float2* A = Yc + D * ADJ_MC * ADJ_SC;              // [ADJ_SC][K][K]   Gram, then its factor
  float2* C = A + ADJ_SC * K * K;                    // [ADJ_SC][K][K]
  float2* Lm = C + ADJ_SC * K * K;                   // [ADJ_SC][K][D]   g, then lambda
  float2* Xs = Lm + ADJ_SC * K * D;                  // [ADJ_SC][D][K]   x~
  const int npair = K * (K + 1) / 2;

  auto load_chunk = [&](int m0, bool with_y) {
    for (int e = tid; e < K * ADJ_MC * ADJ_SC; e += blockDim.x) {
      const int n = e % ADJ_SC, ml = (e / ADJ_SC) % ADJ_MC, k = e / (ADJ_SC * ADJ_MC);
      const int m = m0 + ml, sc = k0 + n;
      Hc[e] = (m < M && sc < N) ? a.h[((size_t(t) * K + k) * M + m) * N + sc] : make_float2(0.f, 0.f);
    }
    if (with_y)
      for (int e = tid; e < D * ADJ_MC * ADJ_SC; e += blockDim.x) {
        const int n = e % ADJ_SC, ml = (e / ADJ_SC) % ADJ_MC, d = e / (ADJ_SC * ADJ_MC);
        const int m = m0 + ml, sc = k0 + n;
        Yc[e] = (m < M && sc < N) ? a.y[((size_t(t) * D + d) * M + m) * N + sc] : make_float2(0.f, 0.f);
      }
  };

  // ---------------------------------------------------------------- Gram (Eq. 22)
  float2 acc[ADJ_GRAM_PER_THREAD];
#pragma unroll
  for (int q = 0; q < ADJ_GRAM_PER_THREAD; ++q) acc[q] = make_float2(0.f, 0.f);
  for (int m0 = 0; m0 < M; m0 += ADJ_MC) {
    load_chunk(m0, false);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < ADJ_GRAM_PER_THREAD; ++q) {
      const int e = tid + q * ADJ_THREADS;
      if (e < ADJ_SC * npair) {
        const int n = e % ADJ_SC;
        int i, j;
        tri_pair(e / ADJ_SC, i, j);
        for (int ml = 0; ml < ADJ_MC; ++ml) {
          const float2 hi = Hc[(i * ADJ_MC + ml) * ADJ_SC + n], hj = Hc[(j * ADJ_MC + ml) * ADJ_SC + n];
          acc[q] = cadd(acc[q], cmulc(hj, hi));    // conj(H[m][i]) H[m][j]
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < ADJ_GRAM_PER_THREAD; ++q) {
    const int e = tid + q * ADJ_THREADS;
    if (e < ADJ_SC * npair) {
      const int n = e % ADJ_SC;
      int i, j;
      tri_pair(e / ADJ_SC, i, j);
      float2 v = acc[q];
      if (i == j) v.x += a.sigma2;
      A[(n * K + i) * K + j] = v;
      A[(n * K + j) * K + i] = make_float2(v.x, -v.y);
    }
  }
  // x~ and g = (x~ - x) / count
  for (int e = tid; e < ADJ_SC * D * K; e += blockDim.x) {
    const int n = e % ADJ_SC, k = (e / ADJ_SC) % K, d = e / (ADJ_SC * K);
    const int sc = k0 + n;
    float2 xv = make_float2(0.f, 0.f), xr = make_float2(0.f, 0.f);
    if (sc < N) {
      const size_t idx = (size_t(t) * D + d) * K * size_t(N) + size_t(k) * N + sc;
      xv = a.x_eq[idx];
      xr = a.x_ref[idx];
    }
    Xs[(n * D + d) * K + k] = xv;
    const float2 g = csub(xv, xr);
    Lm[(n * K + k) * D + d] = make_float2(g.x * a.scale, g.y * a.scale);
  }
  __syncthreads();

  // ---------------------------------- per subcarrier: factor, lambda = A^-1 g, C, sums
  if (tid < ADJ_SC && k0 + tid < N) {
    const int n = tid;
    float2* An = A + n * K * K;
    float2* Ln = Lm + n * K * D;
    const float2* Xn = Xs + n * D * K;
    float loss = 0.f, gs = 0.f;
    for (int d = 0; d < D; ++d)
      for (int k = 0; k < K; ++k) {
        const float2 g = Ln[k * D + d];
        loss += (g.x * g.x + g.y * g.y) / a.scale;
      }
    // A = L L^H in the lower triangle (FP32, as in the forward pass).
    for (int j = 0; j < K; ++j) {
      float dj = An[j * K + j].x;
      for (int m = 0; m < j; ++m) dj -= An[j * K + m].x * An[j * K + m].x + An[j * K + m].y * An[j * K + m].y;
      const float ljj = sqrtf(dj), inv = 1.0f / ljj;
      An[j * K + j] = make_float2(ljj, 0.f);
      for (int i = j + 1; i < K; ++i) {
        float2 s = An[i * K + j];
        for (int m = 0; m < j; ++m) s = csub(s, cmulc(An[i * K + m], An[j * K + m]));
        An[i * K + j] = make_float2(s.x * inv, s.y * inv);
      }
    }
    for (int d = 0; d < D; ++d) {
      for (int i = 0; i < K; ++i) {                  // L w = g
        float2 s = Ln[i * D + d];
        for (int m = 0; m < i; ++m) s = csub(s, cmul_(An[i * K + m], Ln[m * D + d]));
        const float inv = 1.0f / An[i * K + i].x;
        Ln[i * D + d] = make_float2(s.x * inv, s.y * inv);
      }
      for (int i = K - 1; i >= 0; --i) {             // L^H lambda = w
        float2 s = Ln[i * D + d];
        for (int m = i + 1; m < K; ++m) s = csub(s, cmulc(Ln[m * D + d], An[m * K + i]));
        const float inv = 1.0f / An[i * K + i].x;
        Ln[i * D + d] = make_float2(s.x * inv, s.y * inv);
      }
      for (int k = 0; k < K; ++k) {                  // -2 Re lambda^H x~
        const float2 l = Ln[k * D + d], x = Xn[d * K + k];
        gs -= 2.f * (l.x * x.x + l.y * x.y);
      }
    }
    float2* Cn = C + n * K * K;
    for (int i = 0; i < K; ++i)
      for (int j = 0; j < K; ++j) {
        float2 s = make_float2(0.f, 0.f);
        for (int d = 0; d < D; ++d)
          s = cadd(s, cadd(cmulc(Ln[i * D + d], Xn[d * K + j]), cmulc(Xn[d * K + i], Ln[j * D + d])));
        Cn[i * K + j] = s;
      }
    atomicAdd(&a.scal[0], loss);
    atomicAdd(&a.scal[1], gs);
  }
  __syncthreads();

  // ------------------------------------------- G_H = Y Lambda^H - H C, per antenna chunk
  for (int m0 = 0; m0 < M; m0 += ADJ_MC) {
    load_chunk(m0, true);
    __syncthreads();
    for (int e = tid; e < K * ADJ_MC * ADJ_SC; e += blockDim.x) {
      const int n = e % ADJ_SC, ml = (e / ADJ_SC) % ADJ_MC, k = e / (ADJ_SC * ADJ_MC);
      const int m = m0 + ml, sc = k0 + n;
      if (m >= M || sc >= N) continue;
      float2 g = make_float2(0.f, 0.f);
      const float2* Ln = Lm + n * K * D;
      const float2* Cn = C + n * K * K;
      for (int d = 0; d < D; ++d) g = cadd(g, cmulc(Yc[(d * ADJ_MC + ml) * ADJ_SC + n], Ln[k * D + d]));
      for (int j = 0; j < K; ++j) g = csub(g, cmul_(Hc[(j * ADJ_MC + ml) * ADJ_SC + n], Cn[j * K + k]));
      a.g_h[((size_t(t) * K + k) * M + m) * N + sc] = g;
    }
    __syncthreads();
  }
}

struct AdjEstArgs {
  const float2* y;      // y_pilot [T][K][M][N]
  const float2* pil;    // [T][K][N]
  const float2* g_h;    // [T][K][M][N]
  float2* g_wm;         // [B][B]
  float2* g_wt;         // [tail][tail] or null
  int rows, M, N, B, nbf, tail;   // rows = T K M; nbf = full blocks
};

__global__ void __launch_bounds__(ADJ_THREADS) adj_lmmse_kernel(const AdjEstArgs a) {
  extern __shared__ float2 sm[];
  const int N = a.N, B = a.B, tail = a.tail, tid = threadIdx.x;
  float2* gh = sm;          // [N]
  float2* ls = sm + N;      // [N]
  float2 am[ADJ_W_PER_THREAD], at[ADJ_W_PER_THREAD];
#pragma unroll
  for (int q = 0; q < ADJ_W_PER_THREAD; ++q) am[q] = at[q] = make_float2(0.f, 0.f);
  const int r0 = blockIdx.x * ADJ_ROWS;
  for (int r = r0; r < min(r0 + ADJ_ROWS, a.rows); ++r) {
    const float2* prow = a.pil + size_t(r / a.M) * N;
    for (int n = tid; n < N; n += blockDim.x) {
      gh[n] = a.g_h[size_t(r) * N + n];
      const float2 yv = a.y[size_t(r) * N + n], p = prow[n];
      const float inv = 1.0f / fmaf(p.x, p.x, p.y * p.y);
      ls[n] = make_float2(fmaf(yv.x, p.x, yv.y * p.y) * inv, fmaf(yv.y, p.x, -yv.x * p.y) * inv);  // Eq. 9
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < ADJ_W_PER_THREAD; ++q) {
      const int e = tid + q * ADJ_THREADS;
      if (e < B * B) {
        const int i = e / B, j = e - i * B;
        float2 s = am[q];
        for (int b = 0; b < a.nbf; ++b) s = cadd(s, cmulc(gh[b * B + i], ls[b * B + j]));
        am[q] = s;
      }
      if (e < tail * tail) {
        const int i = e / tail, j = e - i * tail, b0 = a.nbf * B;
        at[q] = cadd(at[q], cmulc(gh[b0 + i], ls[b0 + j]));
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < ADJ_W_PER_THREAD; ++q) {
    const int e = tid + q * ADJ_THREADS;
    if (e < B * B) {
      atomicAdd(&a.g_wm[e].x, am[q].x);
      atomicAdd(&a.g_wm[e].y, am[q].y);
    }
    if (e < tail * tail) {
      atomicAdd(&a.g_wt[e].x, at[q].x);
      atomicAdd(&a.g_wt[e].y, at[q].y);
    }
  }
}

size_t adj_det_smem(int K, int D) {
  return (size_t(K) * ADJ_MC * ADJ_SC + size_t(D) * ADJ_MC * ADJ_SC + 2 * size_t(ADJ_SC) * K * K +
          2 * size_t(ADJ_SC) * K * D) * sizeof(float2);
}

}  // namespace

int adjoint_max_block() { return ADJ_MAX_B; }

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
  AdjDetArgs ad{h, y_data, x_eq, x_ref, g_h, scal, K, M, N, D, float(p.sigma2),
                float(1.0 / (double(T) * D * K * N))};
  adj_detect_kernel<<<dim3((N + ADJ_SC - 1) / ADJ_SC, T), ADJ_THREADS, adj_det_smem(K, D), st>>>(ad);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  AdjEstArgs ae{y_pilot, pilots, g_h, g_wm, g_wt, T * K * M, M, N, pl.B, N / pl.B, pl.tail};
  adj_lmmse_kernel<<<(T * K * M + ADJ_ROWS - 1) / ADJ_ROWS, ADJ_THREADS, 2 * size_t(N) * sizeof(float2), st>>>(ae);
  return cudaGetLastError();
}

cudaError_t prepare_adjoint(int device) {
  static std::once_flag flags[64];
  static cudaError_t result[64];
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  std::call_once(flags[device], [device] {
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute(adj_detect_kernel, A, int(adj_det_smem(ADJ_MAXK, RAPRO_MAX_DATA_PER_SLOT)));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(adj_lmmse_kernel, A, 2 * 8192 * int(sizeof(float2)));
    result[device] = e;
  });
  return result[device];
}

}  // namespace rapro
