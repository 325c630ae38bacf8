// Detector adjoint of the symbol MSE (reverse mode of Eq. 22), templated on the padded user
// count KT and data-symbol count DT like the detector.
//
// Loss L = scale sum |x~ - x|^2 over (data symbol, user, subcarrier), scale = 1 / count.  With
// g_d = scale (x~_d - x_d) and A = H^H H + sigma2 I per (slot, subcarrier), the conjugate
// Wirtinger gradients (dL = 2 Re sum conj(G) dX) are
//   lambda_d = A^-1 g_d,   C = sum_d (lambda_d x~_d^H + x~_d lambda_d^H),
//   G_H = sum_d y_d lambda_d^H - H C,   dL/dsigma2 = -2 Re sum_d lambda_d^H x~_d.
//
// One CTA per (slot, DET_SC = 16 subcarriers), 256 threads:
//  1. Gram pass: 8-antenna chunks of h, double-buffered through registers (the loads of the
//     next chunk are in flight while the current one is used); thread (subcarrier, 4 x 4
//     block of the lower triangle, share of the chunk's antennas) accumulates its block in
//     registers; the shares are summed through shared memory into A + sigma2 I;
//  2. g from x~ and x, the loss; lambda = A^-1 g by the detector's own factor / solve code
//     (Cholesky, L^-1, two triangular solves; one half-warp per subcarrier);
//  3. C per subcarrier and dL/dsigma2;
//  4. G_H pass: chunks of h and y again; thread (subcarrier, user, share of the antennas)
//     keeps its user's weights conj(lambda_k,d) and C[j][k] in registers and writes its
//     entries of G_H.
#include <algorithm>
#include <mutex>

#include "detect_kernel.cuh"

namespace rapro {

namespace {

constexpr int AD_SC = DET_SC;            // subcarriers per CTA (16)
constexpr int AD_MC = DET_MCH;           // antennas per chunk (8)
constexpr int AD_THREADS = 256;
constexpr int AD_PL = AD_SC * AD_MC;     // one row of a chunk: [antenna][subcarrier]

struct AdjDetParams {
  const float2* h;      // [T][K][M][N]
  const float2* y;      // [T*D][M][N]
  const float2* x_eq;   // [T*D][K][N]
  const float2* x_ref;  // [T*D][K][N]
  float2* g_h;          // [T][K][M][N]
  float* scal;          // [0] += loss, [1] += dL/dsigma2 (detector)
  int K, M, N, D;
  float sigma2, scale;  // scale = 1 / (T D K N)
};

// Lower-triangle 4 x 4 blocks of a KT x KT matrix: NB = G (G + 1) / 2 for G = KT / 4.
template <int KT>
struct GramBlocks {
  static constexpr int G = KT / 4;
  static constexpr int NB = G * (G + 1) / 2;
  // antennas of a chunk per thread: the chunk's 8 antennas split over MQ shares so that
  // AD_SC * NB * MQ work items fit in one pass of 256 threads
  static constexpr int MQ = (AD_SC * NB * 8 <= AD_THREADS) ? 8 : (AD_SC * NB * 4 <= AD_THREADS) ? 4
                          : (AD_SC * NB * 2 <= AD_THREADS) ? 2 : 1;
  static constexpr int ITEMS = AD_SC * NB * MQ;
};

// G_H pass: (subcarrier, user) items split over MQ2 shares of the chunk's antennas.
template <int KT>
struct GhItems {
  static constexpr int MQ2 = (AD_SC * KT * 8 <= AD_THREADS) ? 8 : (AD_SC * KT * 4 <= AD_THREADS) ? 4
                           : (AD_SC * KT * 2 <= AD_THREADS) ? 2 : 1;
  static constexpr int ITEMS = AD_SC * KT * MQ2;
};

// Shared memory (float2 units): the chunk double buffer [2][KT + DT][AD_PL] (the Gram
// shares [MQ][AD_SC][NB][16] reuse it after the Gram pass), the detector's epilogue region
// (A, z = g, x = lambda, s, info, column buffers, parked sums), x~ [DT][KT][AD_SC] and
// C [KT][KT][AD_SC], then the block sums of the loss and dL/dsigma2.
template <int KT, int DT>
constexpr size_t ad_off_epi() {
  const size_t chunk = 2 * size_t(KT + DT) * AD_PL;
  const size_t shares = size_t(GramBlocks<KT>::MQ) * AD_SC * GramBlocks<KT>::NB * 16;
  return chunk > shares ? chunk : shares;
}
template <int KT, int DT>
constexpr size_t ad_off_xt() { return ad_off_epi<KT, DT>() + det_off_park(KT, DT); }
template <int KT, int DT>
constexpr size_t ad_off_c() { return ad_off_xt<KT, DT>() + size_t(DT) * KT * AD_SC; }
template <int KT, int DT>
constexpr size_t ad_off_red() { return ad_off_c<KT, DT>() + size_t(KT) * KT * AD_SC; }
template <int KT, int DT>
constexpr size_t ad_smem_bytes() { return ad_off_red<KT, DT>() * sizeof(float2) + 2 * (AD_THREADS / 32) * sizeof(float); }

static_assert(ad_smem_bytes<16, 12>() <= 232448, "the largest detector-adjoint tile fits in shared memory");

// One chunk of h (and, with Y, of y) for subcarriers k0.. of slot t, antennas m0..m0+7:
// each thread loads its elements e = tid + 256 u of [rows][antenna][subcarrier] into
// registers (zero outside the arrays); store() puts them into a shared buffer.
template <int KT, int DT, bool Y>
struct ChunkRegs {
  static constexpr int ROWS = KT + (Y ? DT : 0);
  static constexpr int PER = (ROWS * AD_PL + AD_THREADS - 1) / AD_THREADS;
  float2 v[PER];
  __device__ __forceinline__ void load(const AdjDetParams& a, int t, int k0, int m0) {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + u * AD_THREADS;
      const int n = e & (AD_SC - 1), ml = (e >> 4) & (AD_MC - 1), r = e >> 7;
      const int m = m0 + ml, sc = k0 + n;
      v[u] = make_float2(0.f, 0.f);
      if (r < ROWS && m < a.M && sc < a.N) {
        if (r < KT) {
          if (r < a.K) v[u] = a.h[((size_t(t) * a.K + r) * a.M + m) * a.N + sc];
        } else if (r - KT < a.D) {
          v[u] = a.y[((size_t(t) * a.D + (r - KT)) * a.M + m) * a.N + sc];
        }
      }
    }
  }
  __device__ __forceinline__ void store(float2* buf) const {
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = threadIdx.x + u * AD_THREADS;
      if (e < ROWS * AD_PL) buf[e] = v[u];
    }
  }
};

}  // namespace

template <int KT, int DT>
__global__ void __launch_bounds__(AD_THREADS, 1) adj_det_kernel(const __grid_constant__ AdjDetParams a) {
  extern __shared__ __align__(16) float2 sm[];
  using GB = GramBlocks<KT>;
  using GI = GhItems<KT>;
  constexpr int AS = KT + 1;
  constexpr int XS = DET_SC + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int t = blockIdx.y, k0 = blockIdx.x * AD_SC;
  const int K = a.K, D = a.D, M = a.M, N = a.N;
  const int nch = (M + AD_MC - 1) / AD_MC;
  float2* chunk = sm;                                     // [2][KT + DT][AD_PL]
  float2* ep = sm + ad_off_epi<KT, DT>();
  float2* As = ep;                                        // A, then L, then L^-1
  float2* Zs = ep + det_off_z(KT);                        // g, then w
  float2* Xs = ep + det_off_x(KT, DT);                    // lambda [DT][KT][XS]
  float* Ss = reinterpret_cast<float*>(ep + det_off_s(KT, DT));
  int* Is = reinterpret_cast<int*>(Ss + KT * XS);
  float2* Cb = ep + det_off_col(KT, DT);
  float2* Xt = sm + ad_off_xt<KT, DT>();                  // x~ [DT][KT][AD_SC]
  float2* Cm = sm + ad_off_c<KT, DT>();                   // C [KT][KT][AD_SC]
  float* red = reinterpret_cast<float*>(sm + ad_off_red<KT, DT>());
  constexpr int HROWS = KT + DT;                          // rows of a chunk buffer

  // ------------------------------------------------------------ 1. Gram pass
  float2 acc[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) acc[e] = make_float2(0.f, 0.f);
  const bool g_item = tid < GB::ITEMS;
  const int g_n = tid & (AD_SC - 1), g_rest = tid >> 4;
  const int g_blk = g_rest % GB::NB, g_mq = g_rest / GB::NB;
  int bi = 0, bj = 0;                                     // block (bi, bj), bi >= bj
  {
    int b = g_blk;
    while (b > bi) {
      b -= bi + 1;
      ++bi;
    }
    bj = b;
  }
  {
    ChunkRegs<KT, DT, false> cr;
    cr.load(a, t, k0, 0);
    cr.store(chunk);
    __syncthreads();
    for (int c = 0; c < nch; ++c) {
      const float2* cur = chunk + size_t(c & 1) * HROWS * AD_PL;
      if (c + 1 < nch) cr.load(a, t, k0, (c + 1) * AD_MC);
      if (g_item) {
#pragma unroll
        for (int mm = 0; mm < AD_MC / GB::MQ; ++mm) {
          const int ml = g_mq + mm * GB::MQ;
          float2 hi[4], hj[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            hi[r] = cur[(4 * bi + r) * AD_PL + ml * AD_SC + g_n];
            hj[r] = cur[(4 * bj + r) * AD_PL + ml * AD_SC + g_n];
          }
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int q = 0; q < 4; ++q) cmac_conj(acc[r * 4 + q], hi[r], hj[q]);   // A[i][j] += conj(h_i) h_j
        }
      }
      if (c + 1 < nch) cr.store(chunk + size_t((c + 1) & 1) * HROWS * AD_PL);
      __syncthreads();
    }
  }
  // the antenna shares summed into A + sigma2 I (lower triangle, the detector's layout)
  float2* shares = sm;                                    // [MQ][AD_SC][NB][16], over the chunks
  if (g_item) {
#pragma unroll
    for (int e = 0; e < 16; ++e) shares[((size_t(g_mq) * AD_SC + g_n) * GB::NB + g_blk) * 16 + e] = acc[e];
  }
  __syncthreads();
  for (int e = tid; e < AD_SC * GB::NB * 16; e += AD_THREADS) {
    const int rq = e & 15, n = (e >> 4) & (AD_SC - 1), blk = e >> 8;
    float2 v = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < GB::MQ; ++q) {
      const float2 s = shares[((size_t(q) * AD_SC + n) * GB::NB + blk) * 16 + rq];
      v.x += s.x;
      v.y += s.y;
    }
    int b2 = blk, i0 = 0;
    while (b2 > i0) {
      b2 -= i0 + 1;
      ++i0;
    }
    const int i = 4 * i0 + (rq >> 2), j = 4 * b2 + (rq & 3);
    if (i < K && j <= i) {
      if (i == j) v.x += a.sigma2;
      As[(n * KT + i) * AS + j] = v;
    }
  }
  // ------------------------------------------------------------ 2. g, loss, lambda = A^-1 g
  float loss = 0.f, gs = 0.f;
  for (int e = tid; e < AD_SC * KT * DT; e += AD_THREADS) {
    const int n = e & (AD_SC - 1), k = (e >> 4) % KT, d = (e >> 4) / KT;
    const int sc = k0 + n;
    float2 xv = make_float2(0.f, 0.f), g = make_float2(0.f, 0.f);
    if (k < K && d < D && sc < N) {
      const size_t idx = (size_t(t) * D + d) * K * size_t(N) + size_t(k) * N + sc;
      xv = a.x_eq[idx];
      const float2 xr = a.x_ref[idx];
      g = make_float2(xv.x - xr.x, xv.y - xr.y);
      loss += (g.x * g.x + g.y * g.y) * a.scale;
    }
    Xt[(d * KT + k) * AD_SC + n] = xv;
    Zs[(n * KT + k) * DT + d] = make_float2(g.x * a.scale, g.y * a.scale);
  }
  __syncthreads();
  {
    DetParams P{};                                        // no FP64 fallback in the adjoint
    P.sigma2 = a.sigma2;
    det_factor_solve<KT, DT, false>(lane & 15, warp * 2 + (lane >> 4), K, D, t, k0, N, P, As, Zs, Xs, Ss, Is, Cb);
  }
  __syncthreads();
  // ------------------------------------------------------------ 3. dL/dsigma2, C
  for (int e = tid; e < AD_SC * KT * DT; e += AD_THREADS) {
    const int n = e & (AD_SC - 1), k = (e >> 4) % KT, d = (e >> 4) / KT;
    if (k < K && d < D && k0 + n < N) {
      const float2 l = Xs[(d * KT + k) * XS + n], x = Xt[(d * KT + k) * AD_SC + n];
      gs -= 2.f * (l.x * x.x + l.y * x.y);                // -2 Re lambda^H x~
    }
  }
  for (int e = tid; e < AD_SC * KT * KT; e += AD_THREADS) {
    const int n = e & (AD_SC - 1), k = (e >> 4) % KT, j = (e >> 4) / KT;
    float2 s = make_float2(0.f, 0.f);
    if (j < K && k < K) {
      for (int d = 0; d < D; ++d) {
        const float2 lj = Xs[(d * KT + j) * XS + n], lk = Xs[(d * KT + k) * XS + n];
        const float2 xj = Xt[(d * KT + j) * AD_SC + n], xk = Xt[(d * KT + k) * AD_SC + n];
        cmac_conj_rev(s, lj, xk);                         // lambda_j conj(x~_k)
        cmac_conj_rev(s, xj, lk);                         // x~_j conj(lambda_k)
      }
    }
    Cm[(j * KT + k) * AD_SC + n] = s;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    loss += __shfl_xor_sync(0xffffffffu, loss, o);
    gs += __shfl_xor_sync(0xffffffffu, gs, o);
  }
  if (lane == 0) {
    red[warp] = loss;
    red[AD_THREADS / 32 + warp] = gs;
  }
  __syncthreads();
  if (tid == 0) {
    float l = 0.f, g = 0.f;
    for (int w = 0; w < AD_THREADS / 32; ++w) {
      l += red[w];
      g += red[AD_THREADS / 32 + w];
    }
    atomicAdd(&a.scal[0], l);
    atomicAdd(&a.scal[1], g);
  }
  // ------------------------------------------------------------ 4. G_H = Y Lambda^H - H C
  const bool h_item = tid < GI::ITEMS;
  const int h_n = tid & (AD_SC - 1), h_k = (tid >> 4) % KT, h_mq = (tid >> 4) / KT;
  const bool h_live = h_item && h_k < K;
  float2 lam[DT], cw[KT];                                 // conj(lambda_k,d) and C[j][k] of this user
#pragma unroll
  for (int d = 0; d < DT; ++d) {
    const float2 l = (h_live && d < D) ? Xs[(d * KT + h_k) * XS + h_n] : make_float2(0.f, 0.f);
    lam[d] = make_float2(l.x, -l.y);
  }
#pragma unroll
  for (int j = 0; j < KT; ++j) cw[j] = (h_live && j < K) ? Cm[(j * KT + h_k) * AD_SC + h_n] : make_float2(0.f, 0.f);
  {
    ChunkRegs<KT, DT, true> cr;
    cr.load(a, t, k0, 0);
    cr.store(chunk);
    __syncthreads();
    for (int c = 0; c < nch; ++c) {
      const float2* cur = chunk + size_t(c & 1) * HROWS * AD_PL;
      if (c + 1 < nch) cr.load(a, t, k0, (c + 1) * AD_MC);
      if (h_live) {
#pragma unroll
        for (int mm = 0; mm < AD_MC / GI::MQ2; ++mm) {
          const int ml = h_mq + mm * GI::MQ2;
          const int m = c * AD_MC + ml, sc = k0 + h_n;
          float2 g = make_float2(0.f, 0.f);
#pragma unroll
          for (int d = 0; d < DT; ++d) cmac(g, cur[(KT + d) * AD_PL + ml * AD_SC + h_n], lam[d]);
          float2 hc = make_float2(0.f, 0.f);
#pragma unroll
          for (int j = 0; j < KT; ++j) cmac(hc, cur[j * AD_PL + ml * AD_SC + h_n], cw[j]);
          if (m < M && sc < N) a.g_h[((size_t(t) * K + h_k) * M + m) * N + sc] = make_float2(g.x - hc.x, g.y - hc.y);
        }
      }
      if (c + 1 < nch) cr.store(chunk + size_t((c + 1) & 1) * HROWS * AD_PL);
      __syncthreads();
    }
  }
}

namespace {

template <int KT, int DT>
cudaError_t ad_go(const AdjDetParams& a, int T, cudaStream_t st) {
  adj_det_kernel<KT, DT><<<dim3((a.N + AD_SC - 1) / AD_SC, T), AD_THREADS, ad_smem_bytes<KT, DT>(), st>>>(a);
  return cudaGetLastError();
}

template <int KT>
cudaError_t ad_kt(const AdjDetParams& a, int T, cudaStream_t st) {
  return a.D > 6 ? ad_go<KT, 12>(a, T, st) : ad_go<KT, 6>(a, T, st);
}

template <int KT>
cudaError_t ad_prepare_kt() {
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute(adj_det_kernel<KT, 6>, A, int(ad_smem_bytes<KT, 6>()));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(adj_det_kernel<KT, 12>, A, int(ad_smem_bytes<KT, 12>()));
  return e;
}

}  // namespace

cudaError_t launch_adj_detect(const Plan& pl, const float2* h, const float2* y, const float2* x_eq,
                              const float2* x_ref, float2* g_h, float* scal, cudaStream_t st) {
  const int T = pl.T, D = pl.D, K = pl.p.K, M = pl.p.M, N = pl.p.n_sc;
  const AdjDetParams a{h, y, x_eq, x_ref, g_h, scal, K, M, N, D, float(pl.p.sigma2),
                       float(1.0 / (double(T) * D * K * N))};
  if (K <= 4) return ad_kt<4>(a, T, st);
  if (K <= 8) return ad_kt<8>(a, T, st);
  if (K <= 12) return ad_kt<12>(a, T, st);
  return ad_kt<16>(a, T, st);
}

cudaError_t prepare_adj_detect(int device) {
  static std::once_flag flags[64];
  static cudaError_t result[64];
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  std::call_once(flags[device], [device] {
    cudaError_t e = ad_prepare_kt<4>();
    if (e == cudaSuccess) e = ad_prepare_kt<8>();
    if (e == cudaSuccess) e = ad_prepare_kt<12>();
    if (e == cudaSuccess) e = ad_prepare_kt<16>();
    result[device] = e;
  });
  return result[device];
}

}  // namespace rapro
