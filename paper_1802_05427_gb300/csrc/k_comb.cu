// Comb-pilot channel estimation (Sec. II, IV-B): the LS estimate on each user's own tones
// (Eq. 9), then 3W- or S-W-LMMSE per group (Eq. 12 with the weights of Eq. 17, W1-W3, P;
// groups and windows of Tables I and II) or three-fold linearly interpolated LS, and the
// zero-order hold, giving the dense h [T][K][M][n_sc] the detector reads.
//
// One CTA per (slot, user, COMB_ROWS antennas).  It stages its user's weights and the LS
// values of its rows in shared memory (the tones are S subcarriers apart in y_pilot; the K
// users' CTAs read the same pilot rows, which L2 serves), then one thread per output
// subcarrier finds its group, window and weight row, keeps that row in registers and
// applies it to every staged antenna row, so the stores of a warp are consecutive.
#include <algorithm>
#include <mutex>

#include "rapro_internal.h"

namespace rapro {

namespace {

constexpr int COMB_THREADS = 256;
constexpr int COMB_ROWS = 8;          // antenna rows per CTA
constexpr int COMB_MAX_S = 16;        // largest comb spacing (S-W window)
constexpr int COMB_MAX_P = 1024;      // largest number of tones per user

struct CombArgs {
  const float2* y;      // [T][M][N]
  const float2* pil;    // [T][N]
  const float2* w;      // [sets][Q][Q][Q]
  float2* h;            // [T][K][M][N]
  int M, K, N, S, P;
};

__device__ __forceinline__ void cmac(float2& acc, float2 a, float2 b) {
  acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
  acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}

// METHOD: RAPRO_COMB_3W, RAPRO_COMB_SW or RAPRO_COMB_INTERP3; Q = 3 or S (<= QMAX).
template <int METHOD, int QMAX>
__global__ void __launch_bounds__(COMB_THREADS) comb_kernel(const CombArgs a) {
  extern __shared__ float2 sm[];
  const int t = blockIdx.z, k = blockIdx.y, m0 = blockIdx.x * COMB_ROWS;
  const int rows = min(COMB_ROWS, a.M - m0);
  const int S = a.S, P = a.P, N = a.N;
  const int Q = METHOD == RAPRO_COMB_SW ? S : 3;
  const int nw = METHOD == RAPRO_COMB_INTERP3 ? 0 : Q * Q * Q;
  float2* ws = sm;                       // this user's weights [Q][Q][Q]
  float2* ls = sm + nw;                  // [COMB_ROWS][P]
  const float2* wsrc = a.w + (METHOD == RAPRO_COMB_SW ? size_t(k) * nw : 0);
  for (int e = threadIdx.x; e < nw; e += blockDim.x) ws[e] = wsrc[e];
  // Eq. 9 on user k's tones n = k + iS: y conj(p) / |p|^2 (rows past the last antenna: 0).
  for (int e = threadIdx.x; e < COMB_ROWS * P; e += blockDim.x) {
    const int r = e / P, i = e - r * P;
    if (r >= rows) {
      ls[e] = make_float2(0.f, 0.f);
      continue;
    }
    const int n = k + i * S;
    const float2 yv = a.y[(size_t(t) * a.M + m0 + r) * N + n];
    const float2 pv = a.pil[size_t(t) * N + n];
    const float inv = 1.0f / fmaf(pv.x, pv.x, pv.y * pv.y);
    ls[r * P + i] = make_float2(fmaf(yv.x, pv.x, yv.y * pv.y) * inv, fmaf(yv.y, pv.x, -yv.x * pv.y) * inv);
  }
  __syncthreads();
  float2* hout = a.h + ((size_t(t) * a.K + k) * a.M + m0) * N;
  for (int n = threadIdx.x; n < N; n += blockDim.x) {
    if (METHOD == RAPRO_COMB_SW) {
      // Table II: group j = n / S, window of S tones from i0, weight index j - i0.
      const int j = n / S, u = n - j * S;
      const int i0 = min(max(j - (S - 1) / 2, 0), P - S);
      const float2* wr = ws + ((j - i0) * S + u) * S;
      float2 wv[QMAX];
#pragma unroll
      for (int i = 0; i < QMAX; ++i) wv[i] = i < S ? wr[i] : make_float2(0.f, 0.f);
      // All staged rows at once: COMB_ROWS independent accumulation chains (rows past the
      // last antenna are zero and not stored).
      float2 acc[COMB_ROWS];
#pragma unroll
      for (int r = 0; r < COMB_ROWS; ++r) acc[r] = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < QMAX; ++i)
        if (i < S) {
#pragma unroll
          for (int r = 0; r < COMB_ROWS; ++r) cmac(acc[r], wv[i], ls[r * P + i0 + i]);
        }
#pragma unroll
      for (int r = 0; r < COMB_ROWS; ++r)
        if (r < rows) hout[size_t(r) * N + n] = acc[r];
    } else {
      // Zero-order hold onto the 3W positions k + v S/3 (v = 3j + u): the last one <= n,
      // the first one before the user's first tone.
      const int s3 = S / 3;
      const int v = min(n < k ? 0 : (n - k) / s3, 3 * P - 1);
      const int j = v / 3, u = v - 3 * j;
      if (METHOD == RAPRO_COMB_3W) {
        // Table I: window of 3 tones from i0 = min(max(j - 1, 0), P - 3), weight j - i0.
        const int i0 = min(max(j - 1, 0), P - 3);
        const float2* wr = ws + ((j - i0) * 3 + u) * 3;
        const float2 w0 = wr[0], w1 = wr[1], w2 = wr[2];
        for (int r = 0; r < rows; ++r) {
          const float2* x = ls + r * P + i0;
          float2 acc = make_float2(0.f, 0.f);
          cmac(acc, w0, x[0]);
          cmac(acc, w1, x[1]);
          cmac(acc, w2, x[2]);
          hout[size_t(r) * N + n] = acc;
        }
      } else {
        // Three-fold linear interpolation between tones j and j + 1; past the last tone
        // its LS is held.
        const bool last = j + 1 >= P;
        const float f = last ? 0.f : float(u) / 3.0f, g = 1.0f - f;
        const int j1 = last ? j : j + 1;
        for (int r = 0; r < rows; ++r) {
          const float2 x0 = ls[r * P + j], x1 = ls[r * P + j1];
          hout[size_t(r) * N + n] = make_float2(fmaf(g, x0.x, f * x1.x), fmaf(g, x0.y, f * x1.y));
        }
      }
    }
  }
}

size_t comb_smem(int method, int S, int P) {
  const int Q = method == RAPRO_COMB_SW ? S : 3;
  const size_t nw = method == RAPRO_COMB_INTERP3 ? 0 : size_t(Q) * Q * Q;
  return (nw + size_t(COMB_ROWS) * P) * sizeof(float2);
}

}  // namespace

cudaError_t launch_comb(const Plan& pl, const float2* y, const float2* pil, float2* h, cudaStream_t st) {
  const rapro_params& p = pl.p;
  CombArgs a{y, pil, pl.d_w_comb, h, p.M, p.K, p.n_sc, p.comb_spacing, p.n_sc / p.comb_spacing};
  const dim3 grid((p.M + COMB_ROWS - 1) / COMB_ROWS, p.K, pl.T);
  const size_t smem = comb_smem(p.comb_method, a.S, a.P);
  switch (p.comb_method) {
    case RAPRO_COMB_3W: comb_kernel<RAPRO_COMB_3W, 3><<<grid, COMB_THREADS, smem, st>>>(a); break;
    case RAPRO_COMB_SW: comb_kernel<RAPRO_COMB_SW, COMB_MAX_S><<<grid, COMB_THREADS, smem, st>>>(a); break;
    default: comb_kernel<RAPRO_COMB_INTERP3, 3><<<grid, COMB_THREADS, smem, st>>>(a); break;
  }
  return cudaGetLastError();
}

cudaError_t prepare_comb(int device) {
  static std::once_flag flags[64];
  static cudaError_t result[64];
  if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
  std::call_once(flags[device], [device] {
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
    const int big = int(comb_smem(RAPRO_COMB_SW, COMB_MAX_S, COMB_MAX_P));
    cudaError_t e = cudaFuncSetAttribute(comb_kernel<RAPRO_COMB_SW, COMB_MAX_S>, A, big);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(comb_kernel<RAPRO_COMB_3W, 3>, A, int(comb_smem(RAPRO_COMB_3W, 3, COMB_MAX_P)));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(comb_kernel<RAPRO_COMB_INTERP3, 3>, A,
                               int(comb_smem(RAPRO_COMB_INTERP3, 3, COMB_MAX_P)));
    result[device] = e;
  });
  return result[device];
}

}  // namespace rapro
