// Host side of the library: parameter checks, FP64 sub-block LMMSE weights, plans.
//
// The weights follow Eq. 13/17 with orthogonal per-user pilots, where the LS estimate
// sits on every subcarrier and R_{H Hls} = R_{HH} = R:  W = R (R + sigma2 I)^-1.
// Because A = R + sigma2 I and R are Hermitian, W^H = A^-1 R, so W is obtained from one
// Cholesky factorisation A = L L^H and two triangular solves per column of R.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "rapro_internal.h"

namespace rapro {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

rapro_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? RAPRO_ERR_NOMEM : RAPRO_ERR_CUDA;
}

using cd = std::complex<double>;

// Frequency correlation r(d) between subcarriers d apart (Eq. 16 or the exponential PDP).
cd corr_fp64(const rapro_params& p, int d) {
  const double two_pi = 6.283185307179586476925286766559;
  if (p.pdp == RAPRO_PDP_EXP) {
    double norm = 0.0;
    for (int l = 0; l < p.n_taps; ++l) norm += std::exp(-l / p.tau_rms);
    cd acc(0.0, 0.0);
    for (int l = 0; l < p.n_taps; ++l) {
      const double ph = -two_pi * double(l) * double(d) / double(p.n_fft);
      acc += (std::exp(-l / p.tau_rms) / norm) * cd(std::cos(ph), std::sin(ph));
    }
    return acc;
  }
  if (d == 0) return cd(1.0, 0.0);
  const double x = two_pi * p.L * double(d) / double(p.n_fft);
  // (1 - e^{-jx}) / (jx)
  const cd num(1.0 - std::cos(x), std::sin(x));
  return num / cd(0.0, x);
}

bool weights_fp64_into(const rapro_params& p, int n, std::complex<double>* work, double* w_out) {
  // work: r(d) for d in (-n, n), then L, X (n x n each), then y (n)
  cd* r = work;
  cd* L = r + (2 * n - 1);
  cd* X = L + size_t(n) * n;
  cd* y = X + size_t(n) * n;
  for (int d = -(n - 1); d <= n - 1; ++d) r[d + n - 1] = corr_fp64(p, d);
  auto R = [&](int a, int b) { return r[a - b + n - 1]; };

  // A = R + sigma2 I, Cholesky in place (lower triangle), column-major access by rows.
  for (int i = 0; i < n; ++i)
    for (int j = 0; j <= i; ++j) L[size_t(i) * n + j] = R(i, j) + (i == j ? p.sigma2 : 0.0);
  for (int j = 0; j < n; ++j) {
    cd* Lj = &L[size_t(j) * n];
    double d = Lj[j].real();
    for (int k = 0; k < j; ++k) d -= std::norm(Lj[k]);
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    const double ljj = std::sqrt(d);
    Lj[j] = cd(ljj, 0.0);
    for (int i = j + 1; i < n; ++i) {
      cd* Li = &L[size_t(i) * n];
      cd s = Li[j];
      for (int k = 0; k < j; ++k) s -= Li[k] * std::conj(Lj[k]);
      Li[j] = s / ljj;
    }
  }
  // X = A^-1 R column by column (L y = r_col, L^H x = y); then W = X^H.
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) {
      cd s = R(i, c);
      const cd* Li = &L[size_t(i) * n];
      for (int k = 0; k < i; ++k) s -= Li[k] * y[k];
      y[i] = s / Li[i].real();
    }
    for (int i = n - 1; i >= 0; --i) {
      cd s = y[i];
      for (int k = i + 1; k < n; ++k) s -= std::conj(L[size_t(k) * n + i]) * X[size_t(k) * n + c];
      X[size_t(i) * n + c] = s / L[size_t(i) * n + i].real();
    }
  }
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      const cd v = std::conj(X[size_t(b) * n + a]);   // W[a][b] = conj(X[b][a])
      w_out[2 * (size_t(a) * n + b)] = v.real();
      w_out[2 * (size_t(a) * n + b) + 1] = v.imag();
    }
  return true;
}

bool build_weights_fp64(const rapro_params& p, int n, std::vector<double>& w_out) {
  std::vector<cd> work(weights_fp64_work(n));
  w_out.assign(size_t(2) * n * n, 0.0);
  return weights_fp64_into(p, n, work.data(), w_out.data());
}

int comb_window(const rapro_params& p) {
  return p.comb_method == RAPRO_COMB_SW ? p.comb_spacing : 3;
}

bool build_comb_weights_fp64(const rapro_params& p, std::vector<double>& w_out) {
  // Sec. IV-B: per weight index w (group position within its window) a Q x Q matrix
  // W = R_o (R_i + sigma2 I)^-1, R_i[a][b] = r((a - b) S) over the window's tones and
  // R_o[u][i] = r(out_u - tone_i):  (w - i) S + u S/3 for 3W (any user), (w - i) S + u - k
  // for S-W and user k.  Solved as for the sub-blocks: A = L L^H, X = A^-1 R_o^H, W = X^H.
  const int S = p.comb_spacing, Q = comb_window(p);
  const bool sw = p.comb_method == RAPRO_COMB_SW;
  const int sets = sw ? p.K : 1;
  std::vector<cd> L(size_t(Q) * Q), X(size_t(Q) * Q), y(Q);
  for (int i = 0; i < Q; ++i)
    for (int j = 0; j <= i; ++j) L[size_t(i) * Q + j] = corr_fp64(p, (i - j) * S) + (i == j ? p.sigma2 : 0.0);
  for (int j = 0; j < Q; ++j) {
    cd* Lj = &L[size_t(j) * Q];
    double d = Lj[j].real();
    for (int k = 0; k < j; ++k) d -= std::norm(Lj[k]);
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    const double ljj = std::sqrt(d);
    Lj[j] = cd(ljj, 0.0);
    for (int i = j + 1; i < Q; ++i) {
      cd* Li = &L[size_t(i) * Q];
      cd s = Li[j];
      for (int k = 0; k < j; ++k) s -= Li[k] * std::conj(Lj[k]);
      Li[j] = s / ljj;
    }
  }
  w_out.assign(size_t(2) * sets * Q * Q * Q, 0.0);
  for (int k = 0; k < sets; ++k)
    for (int w = 0; w < Q; ++w) {
      auto off = [&](int u, int i) { return sw ? (w - i) * S + u - k : (w - i) * S + u * (S / 3); };
      // column c of R_o^H: conj(R_o[c][i]) over i; solve L y = col, L^H x = y.
      for (int c = 0; c < Q; ++c) {
        for (int i = 0; i < Q; ++i) {
          cd s = std::conj(corr_fp64(p, off(c, i)));
          const cd* Li = &L[size_t(i) * Q];
          for (int m = 0; m < i; ++m) s -= Li[m] * y[m];
          y[i] = s / Li[i].real();
        }
        for (int i = Q - 1; i >= 0; --i) {
          cd s = y[i];
          for (int m = i + 1; m < Q; ++m) s -= std::conj(L[size_t(m) * Q + i]) * X[size_t(m) * Q + c];
          X[size_t(i) * Q + c] = s / L[size_t(i) * Q + i].real();
        }
      }
      double* dst = &w_out[size_t(2) * ((size_t(k) * Q + w) * Q) * Q];
      for (int u = 0; u < Q; ++u)
        for (int i = 0; i < Q; ++i) {
          const cd v = std::conj(X[size_t(i) * Q + u]);   // W[u][i] = conj(X[i][u])
          dst[2 * (size_t(u) * Q + i)] = v.real();
          dst[2 * (size_t(u) * Q + i) + 1] = v.imag();
        }
    }
  return true;
}

DetTiles make_det_tiles(int K, int D) {
  DetTiles t{};
  const int ng = (K + 3) / 4, ndg = (D + 5) / 6;
  t.KP = 4 * ng;
  t.DP = 6 * ndg;
  int n = 0;
  auto add = [&](int kind, int g, int r, int c) {
    t.kind[n] = (signed char)kind; t.g[n] = (signed char)g; t.r[n] = (signed char)r; t.c[n] = (signed char)c;
    ++n;
  };
  // Off-diagonal Gram blocks (r > c): pair one with each triangle, the rest alone.
  int rects[DET_MAX_ROLES][2], nr = 0;
  for (int r = 1; r < ng; ++r)
    for (int c = 0; c < r; ++c) { rects[nr][0] = r; rects[nr][1] = c; ++nr; }
  bool used[DET_MAX_ROLES] = {};
  for (int g = 0; g < ng; ++g) {
    int pick = -1;
    for (int k = 0; k < nr && pick < 0; ++k)   // prefer a block sharing rows or columns with g
      if (!used[k] && (rects[k][0] == g || rects[k][1] == g)) pick = k;
    if (pick >= 0) { used[pick] = true; add(0, g, rects[pick][0], rects[pick][1]); }
    else add(0, g, -1, -1);
  }
  for (int k = 0; k < nr; ++k)
    if (!used[k]) add(1, -1, rects[k][0], rects[k][1]);
  for (int g = 0; g < ng; ++g)
    for (int c = 0; c < ndg; ++c) add(2, g, -1, c);
  t.n_roles = n;
  t.msplit = n <= 8 ? 2 : 1;
  return t;
}

static rapro_status invalid(const char* msg) {
  set_error(msg);
  return RAPRO_ERR_INVALID_ARG;
}

}  // namespace rapro

using namespace rapro;

extern "C" {

const char* rapro_status_string(rapro_status s) {
  switch (s) {
    case RAPRO_OK: return "RAPRO_OK";
    case RAPRO_ERR_INVALID_ARG: return "RAPRO_ERR_INVALID_ARG";
    case RAPRO_ERR_CUDA: return "RAPRO_ERR_CUDA";
    case RAPRO_ERR_NOT_POSDEF: return "RAPRO_ERR_NOT_POSDEF";
    case RAPRO_ERR_TIMEOUT: return "RAPRO_ERR_TIMEOUT";
    case RAPRO_ERR_UNSUPPORTED: return "RAPRO_ERR_UNSUPPORTED";
    case RAPRO_ERR_NOMEM: return "RAPRO_ERR_NOMEM";
  }
  return "RAPRO_ERR_UNKNOWN";
}

const char* rapro_last_error(void) { return g_last_error.c_str(); }

rapro_status rapro_params_validate(const rapro_params* p) {
  if (!p) return invalid("params is NULL");
  if (p->M < 1) return invalid("M must be >= 1");
  if (p->K < 1 || p->K > RAPRO_MAX_USERS) return invalid("K must be in [1, RAPRO_MAX_USERS]");
  if (p->n_sc < 1) return invalid("n_sc must be >= 1");
  if (p->n_fft < p->n_sc) return invalid("n_fft must be >= n_sc");
  if (p->n_pilot_sym < 1 || p->n_pilot_sym > RAPRO_MAX_PILOT_SYM)
    return invalid("n_pilot_sym must be in [1, RAPRO_MAX_PILOT_SYM]");
  if (p->n_sym < 2 * p->n_pilot_sym || p->n_sym % p->n_pilot_sym != 0)
    return invalid("n_sym must be a multiple of n_pilot_sym with >= 1 data symbol per slot");
  const int slot_len = p->n_sym / p->n_pilot_sym;
  if (slot_len - 1 > RAPRO_MAX_DATA_PER_SLOT)
    return invalid("more than RAPRO_MAX_DATA_PER_SLOT data symbols per slot");
  for (int j = 0; j < p->n_pilot_sym; ++j)
    if (p->pilot_sym_idx[j] < j * slot_len || p->pilot_sym_idx[j] >= (j + 1) * slot_len)
      return invalid("pilot_sym_idx[j] must lie inside slot j");
  if (p->pilot_layout == RAPRO_PILOT_COMB) {
    const int S = p->comb_spacing;
    if (S < p->K || S > 16) return invalid("comb_spacing must be in [K, 16]");
    if (p->n_sc % S != 0) return invalid("comb_spacing must divide n_sc");
    const int P = p->n_sc / S;
    if (P > 1024) return invalid("more than 1024 pilot tones per user");
    if (p->comb_method == RAPRO_COMB_SW) {
      if (P < S) return invalid("S-W-LMMSE needs at least comb_spacing tones per user");
    } else if (p->comb_method == RAPRO_COMB_3W || p->comb_method == RAPRO_COMB_INTERP3) {
      if (S % 3 != 0) return invalid("3W-LMMSE and interpolated LS need 3 | comb_spacing");
      if (P < 3) return invalid("3W-LMMSE and interpolated LS need at least 3 tones per user");
    } else {
      return invalid("unknown comb_method");
    }
  } else if (p->pilot_layout == RAPRO_PILOT_ORTHOGONAL) {
    if (p->subblock < 1 || p->subblock > p->n_sc) return invalid("subblock must be in [1, n_sc]");
  } else {
    return invalid("unknown pilot_layout");
  }
  if (!(p->sigma2 > 0.0) || !std::isfinite(p->sigma2)) return invalid("sigma2 must be finite and > 0");
  if (p->pdp == RAPRO_PDP_EXP) {
    if (p->n_taps < 1) return invalid("n_taps must be >= 1");
    if (!(p->tau_rms > 0.0) || !std::isfinite(p->tau_rms)) return invalid("tau_rms must be > 0");
  } else if (p->pdp == RAPRO_PDP_UNIFORM_L) {
    if (!(p->L > 0.0) || !std::isfinite(p->L)) return invalid("L must be > 0");
  } else {
    return invalid("unknown pdp kind");
  }
  if (p->qam_bits != 2 && p->qam_bits != 4 && p->qam_bits != 6) return invalid("qam_bits must be 2, 4 or 6");
  if (half_precision(*p)) {
    if (p->pilot_layout != RAPRO_PILOT_ORTHOGONAL || p->subblock % 2 != 0 || p->subblock > 2048 ||
        p->n_sc % p->subblock != 0) {
      set_error("the BF16 / FP16 forms filter on the tensor cores: orthogonal pilots, even subblock <= 2048 dividing n_sc");
      return RAPRO_ERR_UNSUPPORTED;
    }
  } else if (p->precision != RAPRO_PREC_FP32) {
    return invalid("unknown precision");
  }
  const double elems = double(p->n_pilot_sym) * p->K * p->M * p->n_sc;
  if (elems > 2147483647.0) return invalid("T*K*M*n_sc must fit in int32");
  return RAPRO_OK;
}

rapro_status rapro_build_weights_host(const rapro_params* p, int block_len, double* w_out) {
  rapro_status s = rapro_params_validate(p);
  if (s != RAPRO_OK) return s;
  if (block_len < 1 || block_len > 4096) return invalid("block_len must be in [1, 4096]");
  if (!w_out) return invalid("w_out is NULL");
  std::vector<double> w;
  if (!build_weights_fp64(*p, block_len, w)) {
    set_error("R + sigma2 I is not positive definite in FP64");
    return RAPRO_ERR_NOT_POSDEF;
  }
  std::memcpy(w_out, w.data(), w.size() * sizeof(double));
  return RAPRO_OK;
}

rapro_status rapro_weight_grad_host(const rapro_params* p, const double* g_w_main, const double* g_w_tail,
                                    double* grad_out) {
  rapro_status s = rapro_params_validate(p);
  if (s != RAPRO_OK) return s;
  if (p->pilot_layout != RAPRO_PILOT_ORTHOGONAL || p->pdp != RAPRO_PDP_EXP) {
    set_error("the weight gradient covers the sub-block weights of the exponential PDP model");
    return RAPRO_ERR_UNSUPPORTED;
  }
  const int B = p->subblock, tail = p->n_sc % B;
  if (!g_w_main || !grad_out || (tail && !g_w_tail)) return invalid("g_w_main, grad_out (and g_w_tail) are required");
  if (B > 512) return invalid("block size above 512");
  // dp_l/dtau = p_l (l - lbar) / tau^2 for p_l = exp(-l/tau) / sum; r'(d) = sum_l dp_l e^{-j 2 pi l d / n_fft}.
  const double two_pi = 6.283185307179586476925286766559;
  std::vector<double> pl(p->n_taps);
  double norm = 0.0, lbar = 0.0;
  for (int l = 0; l < p->n_taps; ++l) norm += (pl[l] = std::exp(-l / p->tau_rms));
  for (int l = 0; l < p->n_taps; ++l) lbar += (pl[l] /= norm) * l;
  auto dcorr = [&](int d) {
    cd acc(0.0, 0.0);
    for (int l = 0; l < p->n_taps; ++l) {
      const double ph = -two_pi * double(l) * double(d) / double(p->n_fft);
      acc += (pl[l] * (l - lbar) / (p->tau_rms * p->tau_rms)) * cd(std::cos(ph), std::sin(ph));
    }
    return acc;
  };
  double g_s2 = 0.0, g_tau = 0.0;
  for (int part = 0; part < (tail ? 2 : 1); ++part) {
    const int n = part ? tail : B;
    const double* G = part ? g_w_tail : g_w_main;
    // A = R + sigma2 I = L L^H; Ainv by solves on the identity; W = R Ainv.
    std::vector<cd> R(size_t(n) * n), dR(size_t(n) * n), L(size_t(n) * n), Ai(size_t(n) * n), y(n);
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        R[size_t(a) * n + b] = corr_fp64(*p, a - b);
        dR[size_t(a) * n + b] = dcorr(a - b);
      }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j <= i; ++j) L[size_t(i) * n + j] = R[size_t(i) * n + j] + (i == j ? p->sigma2 : 0.0);
    for (int j = 0; j < n; ++j) {
      cd* Lj = &L[size_t(j) * n];
      double d = Lj[j].real();
      for (int k = 0; k < j; ++k) d -= std::norm(Lj[k]);
      if (!(d > 0.0) || !std::isfinite(d)) {
        set_error("R + sigma2 I is not positive definite in FP64");
        return RAPRO_ERR_NOT_POSDEF;
      }
      const double ljj = std::sqrt(d);
      Lj[j] = cd(ljj, 0.0);
      for (int i = j + 1; i < n; ++i) {
        cd* Li = &L[size_t(i) * n];
        cd sum = Li[j];
        for (int k = 0; k < j; ++k) sum -= Li[k] * std::conj(Lj[k]);
        Li[j] = sum / ljj;
      }
    }
    for (int c = 0; c < n; ++c) {
      for (int i = 0; i < n; ++i) {
        cd sum = (i == c) ? cd(1.0, 0.0) : cd(0.0, 0.0);
        for (int k = 0; k < i; ++k) sum -= L[size_t(i) * n + k] * y[k];
        y[i] = sum / L[size_t(i) * n + i].real();
      }
      for (int i = n - 1; i >= 0; --i) {
        cd sum = y[i];
        for (int k = i + 1; k < n; ++k) sum -= std::conj(L[size_t(k) * n + i]) * Ai[size_t(k) * n + c];
        Ai[size_t(i) * n + c] = sum / L[size_t(i) * n + i].real();
      }
    }
    auto mul = [n](const std::vector<cd>& X, const std::vector<cd>& Y) {
      std::vector<cd> Z(size_t(n) * n, cd(0.0, 0.0));
      for (int i = 0; i < n; ++i)
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j) Z[size_t(i) * n + j] += X[size_t(i) * n + k] * Y[size_t(k) * n + j];
      return Z;
    };
    const std::vector<cd> W = mul(R, Ai);
    const std::vector<cd> dWs = mul(W, Ai);                 // dW/dsigma2 = -W Ainv
    std::vector<cd> ImW(size_t(n) * n);
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) ImW[size_t(i) * n + j] = (i == j ? 1.0 : 0.0) - W[size_t(i) * n + j];
    const std::vector<cd> dWt = mul(mul(ImW, dR), Ai);      // dW/dtau = (I - W) dR Ainv
    for (size_t e = 0; e < size_t(n) * n; ++e) {
      const cd g(G[2 * e], G[2 * e + 1]);
      g_s2 += 2.0 * (std::conj(g) * (-dWs[e])).real();
      g_tau += 2.0 * (std::conj(g) * dWt[e]).real();
    }
  }
  grad_out[0] = g_s2;
  grad_out[1] = g_tau;
  return RAPRO_OK;
}

rapro_status rapro_build_comb_weights_host(const rapro_params* p, double* w_out) {
  rapro_status s = rapro_params_validate(p);
  if (s != RAPRO_OK) return s;
  if (p->pilot_layout != RAPRO_PILOT_COMB || p->comb_method == RAPRO_COMB_INTERP3)
    return invalid("weights exist for the comb layout's 3W and S-W methods only");
  if (!w_out) return invalid("w_out is NULL");
  std::vector<double> w;
  if (!build_comb_weights_fp64(*p, w)) {
    set_error("R_{Hls Hls} + sigma2 I is not positive definite in FP64");
    return RAPRO_ERR_NOT_POSDEF;
  }
  std::memcpy(w_out, w.data(), w.size() * sizeof(double));
  return RAPRO_OK;
}

rapro_status rapro_plan_create(const rapro_params* p, rapro_plan** out) {
  if (!out) return invalid("out is NULL");
  *out = nullptr;
  rapro_status s = rapro_params_validate(p);
  if (s != RAPRO_OK) return s;
  Plan* pl = new Plan();
  pl->p = *p;
  pl->T = p->n_pilot_sym;
  pl->D = p->n_sym / p->n_pilot_sym - 1;
  pl->q = p->qam_bits;
  pl->comb = p->pilot_layout == RAPRO_PILOT_COMB;
  if (!pl->comb) {
    pl->B = p->subblock;
    pl->nb = (p->n_sc + p->subblock - 1) / p->subblock;
    pl->tail = p->n_sc % p->subblock;
  }
  pl->tiles = make_det_tiles(p->K, pl->D);
  pl->tiles.msplit = kDefaultDetSplit;

  auto to_c64 = [](const std::vector<double>& w) {
    std::vector<float2> o(w.size() / 2);
    for (size_t i = 0; i < o.size(); ++i) o[i] = make_float2(float(w[2 * i]), float(w[2 * i + 1]));
    return o;
  };
  std::vector<double> w;
  if (pl->comb) {
    if (p->comb_method != RAPRO_COMB_INTERP3) {
      if (!build_comb_weights_fp64(*p, w)) {
        delete pl;
        set_error("R_{Hls Hls} + sigma2 I is not positive definite in FP64");
        return RAPRO_ERR_NOT_POSDEF;
      }
      pl->w_comb = to_c64(w);
    }
  } else if (!build_weights_fp64(*p, pl->B, w)) {
    delete pl;
    set_error("R_b + sigma2 I is not positive definite in FP64");
    return RAPRO_ERR_NOT_POSDEF;
  } else {
    pl->w_main = to_c64(w);
  }
  if (pl->tail) {
    if (!build_weights_fp64(*p, pl->tail, w)) {
      delete pl;
      set_error("tail R_b + sigma2 I is not positive definite in FP64");
      return RAPRO_ERR_NOT_POSDEF;
    }
    pl->w_tail = to_c64(w);
  }
  cudaError_t e = cudaGetDevice(&pl->device);
  if (e != cudaSuccess) { delete pl; return cuda_fail(e, "cudaGetDevice"); }
  if ((e = prepare_detect(pl->device)) != cudaSuccess) { delete pl; return cuda_fail(e, "detector set-up"); }
  if ((e = prepare_estimate(pl->device)) != cudaSuccess) { delete pl; return cuda_fail(e, "estimator set-up"); }
  if ((e = prepare_lmmse_tc(pl->device)) != cudaSuccess) { delete pl; return cuda_fail(e, "tensor-core estimator set-up"); }
  if ((e = prepare_lmmse_tcg(pl->device)) != cudaSuccess) { delete pl; return cuda_fail(e, "tensor-core GEMM set-up"); }
  if ((e = prepare_gram_tc(pl->device)) != cudaSuccess) { delete pl; return cuda_fail(e, "tensor-core Gram set-up"); }
  if ((e = prepare_refine(pl->device)) != cudaSuccess) { delete pl; return cuda_fail(e, "refined detector set-up"); }
  if ((e = prepare_comb(pl->device)) != cudaSuccess) { delete pl; return cuda_fail(e, "comb estimator set-up"); }
  if ((e = prepare_adjoint(pl->device)) != cudaSuccess) { delete pl; return cuda_fail(e, "adjoint set-up"); }
  const size_t h_elems = size_t(pl->T) * p->K * p->M * p->n_sc;
  auto fail = [&](cudaError_t err, const char* what) {
    cudaFree(pl->d_w_main); cudaFree(pl->d_w_tail); cudaFree(pl->d_h_work); cudaFree(pl->d_status);
    cudaFree(pl->d_w_tc); cudaFree(pl->d_w_tcg); cudaFree(pl->d_w_comb); cudaFree(pl->d_fix); cudaFree(pl->d_gram);
    cudaFree(pl->d_a_tcg);
    delete pl;
    return cuda_fail(err, what);
  };
  if (!pl->w_main.empty() &&
      (e = cudaMalloc(&pl->d_w_main, pl->w_main.size() * sizeof(float2))) != cudaSuccess) return fail(e, "cudaMalloc W");
  if (!pl->w_comb.empty()) {
    if ((e = cudaMalloc(&pl->d_w_comb, pl->w_comb.size() * sizeof(float2))) != cudaSuccess)
      return fail(e, "cudaMalloc W (comb)");
    if ((e = cudaMemcpy(pl->d_w_comb, pl->w_comb.data(), pl->w_comb.size() * sizeof(float2),
                        cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e, "cudaMemcpy W (comb)");
  }
  if (pl->tail && (e = cudaMalloc(&pl->d_w_tail, pl->w_tail.size() * sizeof(float2))) != cudaSuccess)
    return fail(e, "cudaMalloc W tail");
  if ((e = cudaMalloc(&pl->d_h_work, h_elems * sizeof(float2))) != cudaSuccess) return fail(e, "cudaMalloc workspace");
  if ((e = cudaMalloc(&pl->d_status, sizeof(int))) != cudaSuccess) return fail(e, "cudaMalloc status");
  if (!pl->w_main.empty() && (e = cudaMemcpy(pl->d_w_main, pl->w_main.data(), pl->w_main.size() * sizeof(float2),
                                             cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e, "cudaMemcpy W");
  if (pl->tail && (e = cudaMemcpy(pl->d_w_tail, pl->w_tail.data(), pl->w_tail.size() * sizeof(float2),
                                  cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e, "cudaMemcpy W tail");
  if ((e = cudaMemset(pl->d_status, 0, sizeof(int))) != cudaSuccess) return fail(e, "cudaMemset status");
  if (half_precision(*p)) {
    if ((e = cudaMalloc(&pl->d_fix, (2 + size_t(pl->T) * p->n_sc) * sizeof(int))) != cudaSuccess)
      return fail(e, "cudaMalloc FP64-fallback list");
    if ((e = cudaMemset(pl->d_fix, 0, 2 * sizeof(int))) != cudaSuccess) return fail(e, "cudaMemset FP64-fallback count");
    // The tensor-core Gram and matched filter of the refined detector: [T][n_sc][K][K + D].
    if (!pl->comb &&
        (e = cudaMalloc(&pl->d_gram, size_t(pl->T) * p->n_sc * p->K * (p->K + pl->D) * sizeof(float2))) != cudaSuccess)
      return fail(e, "cudaMalloc Gram workspace");
  }
  if (!pl->comb && lmmse_tc_shape_ok(*pl)) {
    std::vector<unsigned char> wtc;
    build_lmmse_tc_weights(*pl, wtc);
    if ((e = cudaMalloc(&pl->d_w_tc, wtc.size())) != cudaSuccess) return fail(e, "cudaMalloc W (tensor cores)");
    if ((e = cudaMemcpy(pl->d_w_tc, wtc.data(), wtc.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail(e, "cudaMemcpy W (tensor cores)");
  }
  if (lmmse_tcg_shape_ok(*pl)) {
    std::vector<unsigned char> wtg;
    build_lmmse_tcg_weights(*pl, wtg);
    if ((e = cudaMalloc(&pl->d_w_tcg, wtg.size())) != cudaSuccess) return fail(e, "cudaMalloc W (tensor-core GEMM)");
    if ((e = cudaMemcpy(pl->d_w_tcg, wtg.data(), wtg.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
      return fail(e, "cudaMemcpy W (tensor-core GEMM)");
    const size_t a_bytes = lmmse_tcg_stage_bytes(*pl);
    if (a_bytes && (e = cudaMalloc(&pl->d_a_tcg, a_bytes)) != cudaSuccess)
      return fail(e, "cudaMalloc staged operand (tensor-core GEMM)");
  }
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e, "plan upload");
  *out = reinterpret_cast<rapro_plan*>(pl);
  return RAPRO_OK;
}

rapro_status rapro_plan_destroy(rapro_plan* plan) {
  if (!plan) return RAPRO_OK;
  Plan* pl = reinterpret_cast<Plan*>(plan);
  cudaError_t e = cudaDeviceSynchronize();
  cudaFree(pl->d_w_main);
  cudaFree(pl->d_w_tail);
  cudaFree(pl->d_h_work);
  cudaFree(pl->d_status);
  cudaFree(pl->d_w_tc);
  cudaFree(pl->d_w_tcg);
  cudaFree(pl->d_w_comb);
  cudaFree(pl->d_fix);
  cudaFree(pl->d_gram);
  cudaFree(pl->d_a_tcg);
  delete pl;
  return e == cudaSuccess ? RAPRO_OK : cuda_fail(e, "rapro_plan_destroy");
}

rapro_status rapro_plan_dims(const rapro_plan* plan, int* T, int* D, int* nb, int* tail) {
  if (!plan) return invalid("plan is NULL");
  const Plan* pl = reinterpret_cast<const Plan*>(plan);
  if (T) *T = pl->T;
  if (D) *D = pl->D;
  if (nb) *nb = pl->nb;
  if (tail) *tail = pl->tail;
  return RAPRO_OK;
}

rapro_status rapro_plan_device_status(rapro_plan* plan, int reset, int* status_out) {
  if (!plan || !status_out) return invalid("plan or status_out is NULL");
  Plan* pl = reinterpret_cast<Plan*>(plan);
  int v = 0;
  cudaError_t e = cudaMemcpy(&v, pl->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read device status");
  if (reset && (e = cudaMemset(pl->d_status, 0, sizeof(int))) != cudaSuccess) return cuda_fail(e, "reset status");
  *status_out = v;
  return RAPRO_OK;
}

}  // extern "C"
