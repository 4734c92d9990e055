// Host-side plan of the RSFT hot path (FP64): sigma draws (Def. 1), windows
// (§III-C.1, §IV-B), beta(sigma) and first-stage thresholds (eq. (alpha_beta),
// eq. (tpd)), and the second-stage threshold design of eq. (opt).
#include "plan_host.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>

namespace rsft {
namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }

// e^{j pi num / den}, with num reduced modulo 2 den first (exact integer reduction).
cplx cis_pi(int64_t num, int64_t den) {
  int64_t r = num % (2 * den);
  if (r < 0) r += 2 * den;
  return std::polar(1.0, kPi * static_cast<double>(r) / static_cast<double>(den));
}

// In-place iterative radix-2 FFT, forward kernel e^{-j 2 pi k n / N}, unnormalised.
void fft_pow2(std::vector<cplx>& a) {
  const size_t n = a.size();
  for (size_t i = 1, j = 0; i < n; ++i) {
    size_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (size_t len = 2; len <= n; len <<= 1) {
    const size_t half = len / 2;
    std::vector<cplx> tw(half);
    for (size_t k = 0; k < half; ++k) tw[k] = cis_pi(-2 * static_cast<int64_t>(k), static_cast<int64_t>(len));
    for (size_t s = 0; s < n; s += len) {
      for (size_t k = 0; k < half; ++k) {
        cplx u = a[s + k], v = a[s + k + half] * tw[k];
        a[s + k] = u + v;
        a[s + k + half] = u - v;
      }
    }
  }
}

// Chebyshev polynomial of the first kind T_order(x).
double cheb_t(int64_t order, double x) {
  if (std::fabs(x) <= 1.0) return std::cos(static_cast<double>(order) * std::acos(x));
  double v = std::cosh(static_cast<double>(order) * std::acosh(std::fabs(x)));
  return (x < 0 && (order & 1)) ? -v : v;
}

double q_tail(double x) { return 0.5 * std::erfc(x / std::sqrt(2.0)); }


template <class F>
double bisect(F f, double lo, double hi, int iters) {
  double flo = f(lo);
  for (int i = 0; i < iters; ++i) {
    double mid = 0.5 * (lo + hi);
    double fm = f(mid);
    if ((fm > 0) == (flo > 0)) {
      lo = mid;
      flo = fm;
    } else {
      hi = mid;
    }
  }
  return 0.5 * (lo + hi);
}

std::vector<cplx> flat_window(int64_t n, int64_t m, int kind, double atten_db, int64_t support) {
  // w-bar(t) = g c(t) sum_{p<m} e^{-j 2 pi p t / n}; the sum is the Dirichlet kernel
  // e^{-j pi (m-1) t / n} sin(pi m t / n) / sin(pi t / n) (m at t = 0).
  std::vector<cplx> raw(n);
  std::vector<double> taper(n, 0.0);
  if (kind == RSFT_FLAT_IDEAL) {
    std::fill(taper.begin(), taper.end(), 1.0);
  } else {
    int64_t s = support > 0 ? support : n;
    int64_t half = (s - 2) / 2;
    std::vector<double> c = chebyshev_window(2 * half + 1, atten_db);
    for (int64_t t = -half; t <= half; ++t) taper[((t % n) + n) % n] = c[t + half];
  }
  for (int64_t t = 0; t < n; ++t) {
    cplx d;
    if (t == 0) {
      d = cplx(static_cast<double>(m), 0.0);
    } else {
      double num = std::imag(cis_pi(m * t, n));  // sin(pi m t / n)
      double den = std::imag(cis_pi(t, n));      // sin(pi t / n)
      d = cis_pi(-(m - 1) * t, n) * (num / den);
    }
    raw[t] = taper[t] * d;
  }
  std::vector<cplx> spec = raw;
  fft_pow2(spec);
  double g = 1.0 / (std::real(spec[(n - (m / 2)) % n]) / static_cast<double>(n));
  for (auto& v : raw) v *= g;
  return raw;
}

}  // namespace

// P(V > mu) for V ~ Binomial(L, p): the terms C(L, v) p^v (1 - p)^(L - v), v = mu + 1..L, in
// logarithms (lgamma, log1p) so that neither the coefficients nor the powers overflow.
double binomial_tail(int L, double p, int mu) {
  if (mu >= L) return 0.0;
  if (!(p > 0.0)) return mu < 0 ? 1.0 : 0.0;
  if (!(p < 1.0)) return 1.0;
  const double lp = std::log(p), lq = std::log1p(-p), lgl = std::lgamma(L + 1.0);
  double acc = 0.0;
  for (int v = std::max(mu + 1, 0); v <= L; ++v)
    acc += std::exp(lgl - std::lgamma(v + 1.0) - std::lgamma(L - v + 1.0) + v * lp + (L - v) * lq);
  return std::min(acc, 1.0);
}

uint64_t splitmix64_at(uint64_t seed, uint64_t index) {
  uint64_t z = seed + (index + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int64_t inverse_mod_pow2(int64_t sigma, int64_t n) {
  // Newton: x <- x (2 - s x) doubles the correct low bits; s itself is right to 3 bits.
  uint64_t s = static_cast<uint64_t>(sigma), x = s;
  for (int i = 0; i < 6; ++i) x *= 2 - s * x;
  return static_cast<int64_t>(x & static_cast<uint64_t>(n - 1));
}

std::vector<double> chebyshev_window(int64_t len, double atten_db) {
  std::vector<double> w(len, 1.0);
  if (len <= 1) return w;
  const int64_t order = len - 1;
  const double x0 = std::cosh(std::acosh(std::pow(10.0, atten_db / 20.0)) / static_cast<double>(order));
  std::vector<double> amp(len);
  for (int64_t k = 0; k < len; ++k) amp[k] = cheb_t(order, x0 * std::real(cis_pi(k, len)));
  // w[m] = (1/len) sum_k amp_k cos(pi k (2m - len + 1) / len): the inverse DFT of the
  // sampled response with the linear phase of a window centred at (len - 1) / 2.
  std::vector<double> ctab(2 * len);
  for (int64_t i = 0; i < 2 * len; ++i) ctab[i] = std::real(cis_pi(i, len));
  double peak = -std::numeric_limits<double>::infinity();
  for (int64_t mm = 0; mm < len; ++mm) {
    const int64_t step = ((2 * mm - len + 1) % (2 * len) + 2 * len) % (2 * len);
    double acc = 0.0;
    int64_t idx = 0;
    for (int64_t k = 0; k < len; ++k) {
      acc += amp[k] * ctab[idx];
      idx += step;
      if (idx >= 2 * len) idx -= 2 * len;
    }
    w[mm] = acc / static_cast<double>(len);
    peak = std::max(peak, w[mm]);
  }
  for (auto& v : w) v /= peak;
  return w;
}

double window_6db_bins(const std::vector<double>& w) {
  const int64_t n = static_cast<int64_t>(w.size());
  auto mag = [&](double nu) {
    cplx acc(0.0, 0.0);
    for (int64_t t = 0; t < n; ++t) acc += w[t] * std::polar(1.0, -2.0 * kPi * nu * static_cast<double>(t) / static_cast<double>(n));
    return std::abs(acc);
  };
  const double half = 0.5 * mag(0.0);
  double lo = 0.0, hi = -1.0;
  for (int i = 1; i <= 16 * n; ++i) {
    double nu = i / 16.0;
    if (mag(nu) < half) {
      hi = nu;
      break;
    }
    lo = nu;
  }
  if (hi < 0) return static_cast<double>(n);
  for (int i = 0; i < 100; ++i) {
    double mid = 0.5 * (lo + hi);
    if (mag(mid) < half) hi = mid; else lo = mid;
  }
  return lo + hi;  // full width = 2 * midpoint
}

rsft_status validate_desc(const rsft_desc& d, std::string& err) {
  if (d.ndim > 4) {
    err = "ndim > 4 is not supported";
    return RSFT_ERR_UNSUPPORTED;
  }
  if (d.ndim < 1) {
    err = "ndim must be in [1, 4]";
    return RSFT_ERR_INVALID_ARG;
  }
  double total = 1.0;
  for (int i = 0; i < d.ndim; ++i) {
    if (d.n[i] < 2 || !is_pow2(d.n[i]) || d.n[i] > (int64_t(1) << 30)) {
      err = "n[" + std::to_string(i) + "] must be a power of two in [2, 2^30]";
      return RSFT_ERR_INVALID_ARG;
    }
    if (!is_pow2(d.b[i]) || d.b[i] > d.n[i]) {
      err = "b[" + std::to_string(i) + "] must be a power of two dividing n";
      return RSFT_ERR_INVALID_ARG;
    }
    if (d.flat_support[i] != 0 && (d.flat_support[i] < 2 || d.flat_support[i] > d.n[i] || (d.flat_support[i] & 1))) {
      err = "flat_support[" + std::to_string(i) + "] must be 0 or even in [2, n]";
      return RSFT_ERR_INVALID_ARG;
    }
    total *= static_cast<double>(d.n[i]);
  }
  if (total > 8589934592.0) {
    err = "cube larger than 2^33 elements";
    return RSFT_ERR_UNSUPPORTED;
  }
  if (d.loops < 1 || d.loops > 255) {
    err = "loops must be in [1, 255] (votes are counted in 8 bits)";
    return RSFT_ERR_INVALID_ARG;
  }
  if (d.window != RSFT_WIN_RECT && d.window != RSFT_WIN_CHEB) {
    err = "unknown window";
    return RSFT_ERR_INVALID_ARG;
  }
  if (d.flat != RSFT_FLAT_IDEAL && d.flat != RSFT_FLAT_CHEB) {
    err = "unknown flat window";
    return RSFT_ERR_INVALID_ARG;
  }
  if ((d.window == RSFT_WIN_CHEB || d.flat == RSFT_FLAT_CHEB) && !(d.atten_db > 0.0 && d.atten_db <= 400.0)) {
    err = "atten_db must be in (0, 400]";
    return RSFT_ERR_INVALID_ARG;
  }
  if (!std::isfinite(d.noise_var)) {
    err = "noise_var must be finite (> 0 known noise, <= 0 estimate mode)";
    return RSFT_ERR_INVALID_ARG;
  }
  if (d.design_mode != RSFT_DESIGN_NORMAL && d.design_mode != RSFT_DESIGN_BINOMIAL) {
    err = "unknown design_mode";
    return RSFT_ERR_INVALID_ARG;
  }
  if (d.p_fa1_override > 0.0 && !(d.p_fa1_override < 1.0)) {
    err = "p_fa1_override must be in (0, 1)";
    return RSFT_ERR_INVALID_ARG;
  }
  if (d.mu_override >= d.loops) {
    err = "mu_override must be < loops";
    return RSFT_ERR_INVALID_ARG;
  }
  const bool need_design = !(d.p_fa1_override > 0.0) || d.mu_override < 0;
  if (need_design) {
    if (!(d.p_fa > 0.0 && d.p_fa < 1.0) || !(d.p_d > 0.0 && d.p_d < 1.0) || d.k_max < 1) {
      err = "p_fa, p_d must be in (0, 1) and k_max >= 1";
      return RSFT_ERR_INVALID_ARG;
    }
  }
  if (d.sigma) {
    for (int l = 0; l < d.loops; ++l)
      for (int i = 0; i < d.ndim; ++i) {
        int64_t s = d.sigma[l * d.ndim + i];
        if (s <= 0 || s >= d.n[i] || !(s & 1)) {
          err = "sigma entries must be odd and in (0, n_d)";
          return RSFT_ERR_INVALID_ARG;
        }
      }
  }
  if (d.vote_mode != RSFT_VOTES_ROWS && d.vote_mode != RSFT_VOTES_SCATTER) {
    err = "unknown vote_mode";
    return RSFT_ERR_INVALID_ARG;
  }
  if (d.max_located < 0) {
    err = "max_located must be >= 0";
    return RSFT_ERR_INVALID_ARG;
  }
  return RSFT_OK;
}

rsft_status build_host_plan(const rsft_desc& d, HostPlan& p, std::string& err) {
  rsft_status st = validate_desc(d, err);
  if (st != RSFT_OK) return st;
  p = HostPlan();
  p.desc = d;
  p.desc.sigma = nullptr;
  p.ndim = d.ndim;
  p.loops = d.loops;
  for (int i = 0; i < p.ndim; ++i) {
    p.n[i] = d.n[i];
    p.b[i] = d.b[i];
    p.m[i] = d.n[i] / d.b[i];
    p.total_n *= p.n[i];
    p.total_b *= p.b[i];
  }
  const int L = p.loops, D = p.ndim;
  // sigma: odd and uniform in [N_d] from SplitMix64 output number l*D + d (Def. 1).
  p.sigma.resize(L * D);
  p.sigma_inv.resize(L * D);
  for (int l = 0; l < L; ++l)
    for (int i = 0; i < D; ++i) {
      int64_t s = d.sigma ? d.sigma[l * D + i]
                          : static_cast<int64_t>((splitmix64_at(d.seed, static_cast<uint64_t>(l) * D + i) %
                                                  static_cast<uint64_t>(p.n[i])) | 1u);
      p.sigma[l * D + i] = s;
      p.sigma_inv[l * D + i] = inverse_mod_pow2(s, p.n[i]);
    }
  // windows
  p.wsum = 1.0;
  p.eta_m = 1.0;
  for (int i = 0; i < D; ++i) {
    if (d.window == RSFT_WIN_CHEB) p.w[i] = chebyshev_window(p.n[i], d.atten_db);
    else p.w[i] = std::vector<double>(p.n[i], 1.0);
    p.wbar[i] = flat_window(p.n[i], p.m[i], d.flat, d.atten_db, d.flat_support[i]);
    double s = 0.0;
    for (double v : p.w[i]) s += v;
    p.wsum *= s;
    p.eta_m *= window_6db_bins(p.w[i]);
    std::vector<cplx> spec = p.wbar[i];
    fft_pow2(spec);
    p.gain_pass[i].resize(p.m[i]);
    for (int64_t v = 0; v < p.m[i]; ++v) p.gain_pass[i][v] = spec[(p.n[i] - v) % p.n[i]] / static_cast<double>(p.n[i]);
  }
  // beta(sigma_l) = prod_d sum_t |w-bar_d(t)|^2 w_d(sigma t mod N_d)^2
  p.beta.resize(L);
  for (int l = 0; l < L; ++l) {
    double bt = 1.0;
    for (int i = 0; i < D; ++i) {
      const int64_t n = p.n[i], s = p.sigma[l * D + i];
      double acc = 0.0;
      for (int64_t t = 0; t < n; ++t) {
        double wv = p.w[i][(s * t) & (n - 1)];
        acc += std::norm(p.wbar[i][t]) * wv * wv;
      }
      bt *= acc;
    }
    p.beta[l] = bt;
  }
  // second-stage design, eq. (opt): enumerate mu in [L]
  if (d.k_max >= 1 && static_cast<double>(d.k_max) * p.eta_m >= static_cast<double>(p.total_b))
    p.warnings |= RSFT_WARN_SPARSITY_LIMIT;
  double pfa1 = d.p_fa1_override;
  int mu = d.mu_override;
  if (!(pfa1 > 0.0) || mu < 0) {
    const double F = static_cast<double>(L) * d.k_max * p.eta_m / static_cast<double>(p.total_b);
    if (F >= static_cast<double>(L)) {
      // Remark 2: with K eta_m >= B the vote statistics under both hypotheses coincide
      err = "eq. (opt) is infeasible: K_max * eta_m >= B (Remark 2)";
      return RSFT_ERR_DESIGN;
    }
    int best_mu = -1;
    double best_snr = std::numeric_limits<double>::infinity(), best_q = 0, best_pd = 0;
    const bool binom = d.design_mode == RSFT_DESIGN_BINOMIAL;
    const double rho = F / static_cast<double>(L);  // per-loop chance of sharing a target's bucket
    for (int cand = 0; cand < L; ++cand) {
      // Claim 2 (Normal) or its binomial law: P_d = P(votes of a true cell > mu)
      auto fpd = [&](double pd) {
        if (binom) return binomial_tail(L, pd, cand) - d.p_d;
        return q_tail((cand - L * pd) / std::sqrt(L * pd * (1 - pd))) - d.p_d;
      };
      double lo = 1e-15, hi = 1 - 1e-15;
      if ((fpd(lo) > 0) == (fpd(hi) > 0)) continue;
      const double pd = bisect(fpd, lo, hi, 200);
      const double hit = d.eta_p > 0 ? std::min(1.0, d.eta_p * pd) : 1.0;
      // Claim 3 (Normal) or its binomial law: P_fa = P(votes of an off-target cell > mu)
      auto fq = [&](double q) {
        if (binom) return binomial_tail(L, rho * hit + (1.0 - rho) * q, cand) - d.p_fa;
        double mean = F * hit + (L - F) * q;
        double var = F * hit * (1 - hit) + (L - F) * q * (1 - q);
        return q_tail((cand - mean) / std::sqrt(var)) - d.p_fa;
      };
      double qlo = 1e-300, qhi = 1 - 1e-12;
      if (binom && fq(0.0) >= 0) continue;  // the targets' buckets alone exceed P_fa at this mu
      if ((fq(qlo) > 0) == (fq(qhi) > 0)) continue;
      const double q = bisect(fq, qlo, qhi, 400);
      if (q >= pd) continue;
      const double snr = std::log(q) / std::log(pd) - 1.0;  // times beta-bar / alpha-bar
      if (snr < best_snr) {
        best_snr = snr;
        best_mu = cand;
        best_q = q;
        best_pd = pd;
      }
    }
    if (best_mu < 0) {
      err = "eq. (opt) has no feasible second-stage threshold for these p_fa, p_d, k_max";
      return RSFT_ERR_DESIGN;
    }
    if (!(pfa1 > 0.0)) pfa1 = best_q;
    if (mu < 0) mu = best_mu;
    p.pd_bar = best_pd;
  }
  p.pfa1 = pfa1;
  p.mu = mu;
  p.gamma.resize(L);
  double beta_mean = 0.0;
  if (d.beta_mode == RSFT_BETA_MEAN) {
    beta_mean = 1.0;
    for (int i = 0; i < D; ++i) {
      const int64_t n = p.n[i];
      double tot = 0.0;
      for (int64_t s = 1; s < n; s += 2) {
        double acc = 0.0;
        for (int64_t t = 0; t < n; ++t) {
          double wv = p.w[i][(s * t) & (n - 1)];
          acc += std::norm(p.wbar[i][t]) * wv * wv;
        }
        tot += acc;
      }
      beta_mean *= tot / static_cast<double>(n / 2);
    }
  }
  p.estimate_noise = !(d.noise_var > 0.0);
  // estimate mode: gamma_l = -(lowermedian(P_l) / ln 2) ln Pfa1-bar is formed by each execute from
  // its own bucket powers; the factor -ln Pfa1-bar / ln 2 is fixed here
  p.floor_factor = -std::log(pfa1) / std::log(2.0);
  for (int l = 0; l < L; ++l)
    p.gamma[l] = p.estimate_noise ? std::numeric_limits<double>::quiet_NaN()
                                  : -d.noise_var * (d.beta_mode == RSFT_BETA_MEAN ? beta_mean : p.beta[l]) *
                                        std::log(pfa1);
  return RSFT_OK;
}

double design_snr_db(const HostPlan& p) {
  // SNR*_min = (beta-bar / alpha-bar)(ln Pfa1 / ln Pd - 1) (from eq. (bpd)), alpha for a
  // tone at N_d/16 + 1/2 bins in every dimension, averaged over odd sigma (Claim 1 peak bucket).
  if (!(p.pd_bar > 0.0)) return std::numeric_limits<double>::quiet_NaN();
  double abar = 1.0, bbar = 1.0;
  for (int i = 0; i < p.ndim; ++i) {
    const int64_t n = p.n[i], b = p.b[i];
    const int64_t f0 = n / 16;  // floor of the tone bin
    double asum = 0.0, bsum = 0.0;
    for (int64_t s = 1; s < n; s += 2) {
      std::vector<cplx> fold(b, cplx(0, 0));
      double bacc = 0.0;
      for (int64_t t = 0; t < n; ++t) {
        int64_t st = (s * t) & (n - 1);
        // e^{j omega st} with omega = 2 pi (f0 + 1/2) / n  ->  e^{j pi (2 f0 + 1) st / n}
        cplx v = p.wbar[i][t] * p.w[i][st] * cis_pi((2 * f0 + 1) * st, n);
        fold[t & (b - 1)] += v;
        bacc += std::norm(p.wbar[i][t]) * p.w[i][st] * p.w[i][st];
      }
      int64_t peak = (((s * f0) & (n - 1)) * b) / n;
      cplx acc(0, 0);
      for (int64_t j = 0; j < b; ++j) acc += fold[j] * cis_pi(-2 * peak * j, b);
      asum += std::norm(acc);
      bsum += bacc;
    }
    abar *= asum / static_cast<double>(n / 2);
    bbar *= bsum / static_cast<double>(n / 2);
  }
  double snr = (bbar / abar) * (std::log(p.pfa1) / std::log(p.pd_bar) - 1.0);
  return 10.0 * std::log10(snr);
}

}  // namespace rsft
