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

constexpr int ADJ_SC = 8;         // subcarriers per detector-adjoint CTA
constexpr int ADJ_MC = 16;        // antennas per staged chunk
constexpr int ADJ_UNROLL = 8;     // loads in flight per thread while staging
constexpr int ADJ_EST_UNROLL = 4;
constexpr int ADJ_THREADS = 256;
constexpr int ADJ_ROWS = 4;       // estimator rows staged at a time
constexpr int ADJ_MAX_N = 2048;   // largest n_sc
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

// Shared-memory arrays keep the subcarrier index fastest ([...][ADJ_SC]), so that the
// subcarriers of a warp's accesses fall in distinct banks.
__global__ void __launch_bounds__(ADJ_THREADS, 1) adj_detect_kernel(const AdjDetArgs a) {
  extern __shared__ float2 sm[];
  const int K = a.K, M = a.M, N = a.N, D = a.D;
  const int t = blockIdx.y, k0 = blockIdx.x * ADJ_SC, tid = threadIdx.x;
  float2* Hc = sm;                                   // [K][ADJ_MC][ADJ_SC]
  float2* Yc = Hc + K * ADJ_MC * ADJ_SC;             // [D][ADJ_MC][ADJ_SC]
  float2* A = Yc + D * ADJ_MC * ADJ_SC;              // [K][K][ADJ_SC]   Gram, then its factor
  float2* C = A + ADJ_SC * K * K;                    // [K][K][ADJ_SC]
  float2* Lm = C + ADJ_SC * K * K;                   // [K][D][ADJ_SC]   g, then lambda
  float2* Xs = Lm + ADJ_SC * K * D;                  // [D][K][ADJ_SC]   x~
  float* red = reinterpret_cast<float*>(Xs + ADJ_SC * D * K);   // [2][ADJ_THREADS / 32]
  const int npair = K * (K + 1) / 2;
  auto AT = [&](int i, int j, int n) -> float2& { return A[(i * K + j) * ADJ_SC + n]; };
  auto LT = [&](int k, int d, int n) -> float2& { return Lm[(k * D + d) * ADJ_SC + n]; };
  auto XT = [&](int d, int k, int n) -> float2& { return Xs[(d * K + k) * ADJ_SC + n]; };
  auto CT = [&](int i, int j, int n) -> float2& { return C[(i * K + j) * ADJ_SC + n]; };

  // Staged with ADJ_UNROLL independent loads in flight per thread.
  auto load_chunk = [&](int m0, bool with_y) {
    const int nh = K * ADJ_MC * ADJ_SC, ny = with_y ? D * ADJ_MC * ADJ_SC : 0;
    for (int base = tid; base < nh + ny; base += blockDim.x * ADJ_UNROLL) {
      float2 v[ADJ_UNROLL];
#pragma unroll
      for (int u = 0; u < ADJ_UNROLL; ++u) {
        const int e = base + u * blockDim.x;
        v[u] = make_float2(0.f, 0.f);
        if (e < nh) {
          const int n = e % ADJ_SC, ml = (e / ADJ_SC) % ADJ_MC, k = e / (ADJ_SC * ADJ_MC);
          const int m = m0 + ml, sc = k0 + n;
          if (m < M && sc < N) v[u] = a.h[((size_t(t) * K + k) * M + m) * N + sc];
        } else if (e < nh + ny) {
          const int f = e - nh;
          const int n = f % ADJ_SC, ml = (f / ADJ_SC) % ADJ_MC, d = f / (ADJ_SC * ADJ_MC);
          const int m = m0 + ml, sc = k0 + n;
          if (m < M && sc < N) v[u] = a.y[((size_t(t) * D + d) * M + m) * N + sc];
        }
      }
#pragma unroll
      for (int u = 0; u < ADJ_UNROLL; ++u) {
        const int e = base + u * blockDim.x;
        if (e < nh + ny) Hc[e] = v[u];           // Yc follows Hc directly
      }
    }
  };

  // ---------------------------------------------------------------- Gram (Eq. 22)
  float2 acc[ADJ_GRAM_PER_THREAD];
  int pi_[ADJ_GRAM_PER_THREAD], pj_[ADJ_GRAM_PER_THREAD];
#pragma unroll
  for (int q = 0; q < ADJ_GRAM_PER_THREAD; ++q) {
    acc[q] = make_float2(0.f, 0.f);
    const int e = tid + q * ADJ_THREADS;
    int i = 0, j = 0;
    if (e < ADJ_SC * npair) tri_pair(e / ADJ_SC, i, j);
    pi_[q] = i;
    pj_[q] = j;
  }
  for (int m0 = 0; m0 < M; m0 += ADJ_MC) {
    load_chunk(m0, false);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < ADJ_GRAM_PER_THREAD; ++q) {
      const int e = tid + q * ADJ_THREADS;
      if (e < ADJ_SC * npair) {
        const int n = e % ADJ_SC, i = pi_[q], j = pj_[q];
#pragma unroll
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
      const int n = e % ADJ_SC, i = pi_[q], j = pj_[q];
      float2 v = acc[q];
      if (i == j) v.x += a.sigma2;
      AT(i, j, n) = v;
      AT(j, i, n) = make_float2(v.x, -v.y);
    }
  }
  // x~ and g = (x~ - x) / count; the loss on the way
  float loss = 0.f, gs = 0.f;
  for (int e = tid; e < ADJ_SC * D * K; e += blockDim.x) {
    const int n = e % ADJ_SC, k = (e / ADJ_SC) % K, d = e / (ADJ_SC * K);
    const int sc = k0 + n;
    float2 xv = make_float2(0.f, 0.f), xr = make_float2(0.f, 0.f);
    if (sc < N) {
      const size_t idx = (size_t(t) * D + d) * K * size_t(N) + size_t(k) * N + sc;
      xv = a.x_eq[idx];
      xr = a.x_ref[idx];
    }
    XT(d, k, n) = xv;
    const float2 g = csub(xv, xr);
    loss += (g.x * g.x + g.y * g.y) * a.scale;
    LT(k, d, n) = make_float2(g.x * a.scale, g.y * a.scale);
  }
  __syncthreads();

  // ------------------------ A = L L^H per subcarrier (FP32, as in the forward pass)
  if (tid < ADJ_SC) {
    const int n = tid;
    for (int j = 0; j < K; ++j) {
      float dj = AT(j, j, n).x;
      for (int m = 0; m < j; ++m) {
        const float2 l = AT(j, m, n);
        dj -= l.x * l.x + l.y * l.y;
      }
      const float ljj = sqrtf(dj), inv = 1.0f / ljj;
      AT(j, j, n) = make_float2(ljj, 0.f);
      for (int i = j + 1; i < K; ++i) {
        float2 s = AT(i, j, n);
        for (int m = 0; m < j; ++m) s = csub(s, cmulc(AT(i, m, n), AT(j, m, n)));
        AT(i, j, n) = make_float2(s.x * inv, s.y * inv);
      }
    }
  }
  __syncthreads();
  // ----------------- lambda_d = A^-1 g_d, one thread per (subcarrier, data symbol)
  for (int e = tid; e < ADJ_SC * D; e += blockDim.x) {
    const int n = e % ADJ_SC, d = e / ADJ_SC;
    if (k0 + n >= N) continue;
    for (int i = 0; i < K; ++i) {                    // L w = g
      float2 s = LT(i, d, n);
      for (int m = 0; m < i; ++m) s = csub(s, cmul_(AT(i, m, n), LT(m, d, n)));
      const float inv = 1.0f / AT(i, i, n).x;
      LT(i, d, n) = make_float2(s.x * inv, s.y * inv);
    }
    for (int i = K - 1; i >= 0; --i) {               // L^H lambda = w
      float2 s = LT(i, d, n);
      for (int m = i + 1; m < K; ++m) s = csub(s, cmulc(LT(m, d, n), AT(m, i, n)));
      const float inv = 1.0f / AT(i, i, n).x;
      LT(i, d, n) = make_float2(s.x * inv, s.y * inv);
    }
    for (int k = 0; k < K; ++k) {                    // -2 Re lambda^H x~
      const float2 l = LT(k, d, n), x = XT(d, k, n);
      gs -= 2.f * (l.x * x.x + l.y * x.y);
    }
  }
  __syncthreads();
  // --------------------------- C = sum_d (lambda_d x~_d^H + x~_d lambda_d^H), K x K
  for (int e = tid; e < ADJ_SC * K * K; e += blockDim.x) {
    const int n = e % ADJ_SC, j = (e / ADJ_SC) % K, i = e / (ADJ_SC * K);
    float2 s = make_float2(0.f, 0.f);
    for (int d = 0; d < D; ++d)
      s = cadd(s, cadd(cmulc(LT(i, d, n), XT(d, j, n)), cmulc(XT(d, i, n), LT(j, d, n))));
    CT(i, j, n) = s;
  }
  // block sums of the loss and dL/dsigma2, one atomic each per CTA
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    loss += __shfl_xor_sync(0xffffffffu, loss, o);
    gs += __shfl_xor_sync(0xffffffffu, gs, o);
  }
  if ((tid & 31) == 0) {
    red[tid >> 5] = loss;
    red[ADJ_THREADS / 32 + (tid >> 5)] = gs;
  }
  __syncthreads();
  if (tid == 0) {
    float l = 0.f, g = 0.f;
    for (int w = 0; w < ADJ_THREADS / 32; ++w) {
      l += red[w];
      g += red[ADJ_THREADS / 32 + w];
    }
    atomicAdd(&a.scal[0], l);
    atomicAdd(&a.scal[1], g);
  }

  // ------------------------------------------- G_H = Y Lambda^H - H C, per antenna chunk
  for (int m0 = 0; m0 < M; m0 += ADJ_MC) {
    load_chunk(m0, true);
    __syncthreads();
    for (int e = tid; e < K * ADJ_MC * ADJ_SC; e += blockDim.x) {
      const int n = e % ADJ_SC, ml = (e / ADJ_SC) % ADJ_MC, k = e / (ADJ_SC * ADJ_MC);
      const int m = m0 + ml, sc = k0 + n;
      if (m >= M || sc >= N) continue;
      float2 g = make_float2(0.f, 0.f);
      for (int d = 0; d < D; ++d) g = cadd(g, cmulc(Yc[(d * ADJ_MC + ml) * ADJ_SC + n], LT(k, d, n)));
      for (int j = 0; j < K; ++j) g = csub(g, cmul_(Hc[(j * ADJ_MC + ml) * ADJ_SC + n], CT(j, k, n)));
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

size_t adj_det_smem(int K, int D) {
  return (size_t(K) * ADJ_MC * ADJ_SC + size_t(D) * ADJ_MC * ADJ_SC + 2 * size_t(ADJ_SC) * K * K +
          2 * size_t(ADJ_SC) * K * D) * sizeof(float2) + 2 * (ADJ_THREADS / 32) * sizeof(float);
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
  AdjDetArgs ad{h, y_data, x_eq, x_ref, g_h, scal, K, M, N, D, float(p.sigma2),
                float(1.0 / (double(T) * D * K * N))};
  adj_detect_kernel<<<dim3((N + ADJ_SC - 1) / ADJ_SC, T), ADJ_THREADS, adj_det_smem(K, D), st>>>(ad);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
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
    cudaError_t e = cudaFuncSetAttribute(adj_detect_kernel, A, int(adj_det_smem(ADJ_MAXK, RAPRO_MAX_DATA_PER_SLOT)));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(adj_lmmse_kernel, A, int(adj_est_smem(ADJ_MAX_N, ADJ_FAST_B)));
    result[device] = e;
  });
  return result[device];
}

}  // namespace rapro
