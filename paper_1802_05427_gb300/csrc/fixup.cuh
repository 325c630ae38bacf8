// FP64 fallback of the precision form: the subcarriers the detector flagged as ill
// conditioned (pivot ratio (max L_jj / min L_jj)^2 above the limit, a lower bound of
// cond(A), or a failed FP32 factorisation) are solved again, Eq. 22 in FP64:
// A = H^H H + sigma2 I and z_d = H^H y_d summed in FP64 from the FP32 inputs, A = L L^H,
// s_k = sigma2 sum_j |L^-1[j][k]|^2, x~_d = A^-1 z_d; the FP32 outputs (x_eq, labels, LLRs,
// info) of those subcarriers are overwritten.  Run by the detector's last CTA to finish.
#pragma once

#include "rapro_internal.h"

// Included by detect_kernel.cuh after demap_store.

namespace rapro {

constexpr int FIX_MAXK = 16;

struct FixArgs {
  const float2* h;
  const float2* y;
  float2* x_eq;
  unsigned char* labels;
  float* llr;
  int* info;
  const int* count;
  const int* list;
  int cap, T, K, M, N, D, q;
  double sigma2;
};

// Shared scratch of the FP64 solves (16-byte aligned).
struct FixScratch {
  double2 A[FIX_MAXK][FIX_MAXK];
  double2 Z[FIX_MAXK][RAPRO_MAX_DATA_PER_SLOT];
  double S[FIX_MAXK];
  int fail;
};

// Every flagged subcarrier, by all threads of the calling CTA.
static __device__ __noinline__ void fp64_fix_items(const FixArgs a, FixScratch* sc) {
  auto& A = sc->A;
  auto& Z = sc->Z;
  auto& S = sc->S;
  int& fail_s = sc->fail;
  const int K = a.K, D = a.D, M = a.M, N = a.N, tid = threadIdx.x;
  const int n_items = min(*a.count, a.cap);
  const int npair = K * (K + 1) / 2;
  for (int item = 0; item < n_items; ++item) {
    const int code = a.list[item], t = code / N, n = code - t * N;
    // Gram (lower triangle) and matched filter in FP64
    for (int e = tid; e < npair + K * D; e += blockDim.x) {
      double sr = 0.0, si = 0.0;
      if (e < npair) {
        int i = 0;
        while ((i + 1) * (i + 2) / 2 <= e) ++i;
        const int j = e - i * (i + 1) / 2;
        for (int m = 0; m < M; ++m) {
          const float2 hi = a.h[((size_t(t) * K + i) * M + m) * N + n];
          const float2 hj = a.h[((size_t(t) * K + j) * M + m) * N + n];
          sr += double(hi.x) * hj.x + double(hi.y) * hj.y;     // conj(h_i) h_j
          si += double(hi.x) * hj.y - double(hi.y) * hj.x;
        }
        if (i == j) sr += a.sigma2;
        A[i][j] = make_double2(sr, si);
      } else {
        const int f = e - npair, k = f / D, d = f - k * D;
        for (int m = 0; m < M; ++m) {
          const float2 hk = a.h[((size_t(t) * K + k) * M + m) * N + n];
          const float2 yv = a.y[((size_t(t) * D + d) * M + m) * N + n];
          sr += double(hk.x) * yv.x + double(hk.y) * yv.y;     // conj(h_k) y_d
          si += double(hk.x) * yv.y - double(hk.y) * yv.x;
        }
        Z[k][d] = make_double2(sr, si);
      }
    }
    __syncthreads();
    if (tid == 0) {
      int fail = 0;
      for (int j = 0; j < K && !fail; ++j) {                     // A = L L^H (lower)
        double dj = A[j][j].x;
        for (int m = 0; m < j; ++m) dj -= A[j][m].x * A[j][m].x + A[j][m].y * A[j][m].y;
        if (!(dj > 0.0)) {
          fail = j + 1;
          break;
        }
        const double ljj = sqrt(dj);
        A[j][j] = make_double2(ljj, 0.0);
        for (int i = j + 1; i < K; ++i) {
          double2 s = A[i][j];
          for (int m = 0; m < j; ++m) {                          // s -= L_im conj(L_jm)
            s.x -= A[i][m].x * A[j][m].x + A[i][m].y * A[j][m].y;
            s.y -= A[i][m].y * A[j][m].x - A[i][m].x * A[j][m].y;
          }
          A[i][j] = make_double2(s.x / ljj, s.y / ljj);
        }
      }
      fail_s = fail;
      if (!fail) {
        // s_k = sigma2 sum_j |L^-1[j][k]|^2: column k of L^-1 by forward substitution
        for (int k = 0; k < K; ++k) {
          double2 col[FIX_MAXK];
          double acc = 0.0;
          for (int j = 0; j < K; ++j) {
            double2 v = make_double2(j == k ? 1.0 : 0.0, 0.0);
            for (int m = k; m < j; ++m) {
              v.x -= A[j][m].x * col[m].x - A[j][m].y * col[m].y;
              v.y -= A[j][m].x * col[m].y + A[j][m].y * col[m].x;
            }
            col[j] = j < k ? make_double2(0.0, 0.0) : make_double2(v.x / A[j][j].x, v.y / A[j][j].x);
            acc += col[j].x * col[j].x + col[j].y * col[j].y;
          }
          S[k] = a.sigma2 * acc;
        }
        for (int d = 0; d < D; ++d) {                            // L w = z, L^H x = w
          double2 w[FIX_MAXK];
          for (int i = 0; i < K; ++i) {
            double2 s = Z[i][d];
            for (int m = 0; m < i; ++m) {
              s.x -= A[i][m].x * w[m].x - A[i][m].y * w[m].y;
              s.y -= A[i][m].x * w[m].y + A[i][m].y * w[m].x;
            }
            w[i] = make_double2(s.x / A[i][i].x, s.y / A[i][i].x);
          }
          for (int i = K - 1; i >= 0; --i) {
            double2 s = w[i];
            for (int m = i + 1; m < K; ++m) {                    // s -= conj(L_mi) x_m
              s.x -= A[m][i].x * Z[m][d].x + A[m][i].y * Z[m][d].y;
              s.y -= A[m][i].x * Z[m][d].y - A[m][i].y * Z[m][d].x;
            }
            Z[i][d] = make_double2(s.x / A[i][i].x, s.y / A[i][i].x);
          }
        }
      }
    }
    __syncthreads();
    if (fail_s == 0) {
      for (int e = tid; e < K * D; e += blockDim.x) {
        const int k = e / D, d = e - k * D;
        const size_t o = (size_t(t * D + d) * K + k) * N + n;
        const float2 xt = make_float2(float(Z[k][d].x), float(Z[k][d].y));
        a.x_eq[o] = xt;
        if (a.labels || a.llr) {
          const float s = float(S[k]);
          switch (a.q) {
            case 2: demap_store<1>(xt, s, o, a.labels, a.llr); break;
            case 4: demap_store<2>(xt, s, o, a.labels, a.llr); break;
            default: demap_store<3>(xt, s, o, a.labels, a.llr); break;
          }
        }
      }
    }
    if (tid == 0 && a.info) a.info[size_t(t) * N + n] = fail_s;
    __syncthreads();
  }
}

}  // namespace rapro
