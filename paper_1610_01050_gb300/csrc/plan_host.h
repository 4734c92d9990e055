// Host-side plan of the RSFT hot path: parameter validation, sigma draws,
// windows, per-loop thresholds and the second-stage threshold design.
// Everything here is plain C++17 in FP64 and touches no GPU.
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "rsft.h"

namespace rsft {

using cplx = std::complex<double>;

struct HostPlan {
  rsft_desc desc{};
  int ndim = 0;
  int loops = 0;
  int64_t n[4] = {1, 1, 1, 1};
  int64_t b[4] = {1, 1, 1, 1};
  int64_t m[4] = {1, 1, 1, 1};
  int64_t total_n = 1;
  int64_t total_b = 1;
  std::vector<int64_t> sigma;      // [L][D] odd multipliers (Def. 1)
  std::vector<int64_t> sigma_inv;  // [L][D] inverses mod N_d (eq. (mod_inv))
  std::vector<double> w[4];        // pre-permutation window taps (§III-C.1)
  std::vector<cplx> wbar[4];       // flat-window taps (§IV-B)
  std::vector<cplx> gain_pass[4];  // G_d(-v mod N_d) for pass-band offset v in [M_d]
  double wsum = 1.0;               // prod_d sum_t w_d(t)
  std::vector<double> beta;        // [L] beta(sigma_l) (eq. (alpha_beta))
  std::vector<double> gamma;       // [L] first-stage thresholds (NaN in estimate mode)
  bool estimate_noise = false;     // noise_var <= 0: each loop's noise floor from its bucket powers
  double floor_factor = 0.0;       // -ln Pfa1-bar / ln 2: gamma_l = lowermedian(P_l) times this
  int mu = 0;                      // second-stage threshold: votes > mu
  double pfa1 = 0.0;               // first-stage Pfa1-bar
  double pd_bar = 0.0;             // Pd-bar of the design (0 when overridden)
  double eta_m = 0.0;              // prod_d 6-dB bandwidth of w_d in bins
  int warnings = 0;
};

rsft_status validate_desc(const rsft_desc& d, std::string& err);
rsft_status build_host_plan(const rsft_desc& d, HostPlan& p, std::string& err);

// SplitMix64 output number `index` of the sequence started at `seed`.
uint64_t splitmix64_at(uint64_t seed, uint64_t index);
// Inverse of an odd sigma modulo 2^k by Newton iteration, reduced mod n.
int64_t inverse_mod_pow2(int64_t sigma, int64_t n);

// P(V > mu) for V ~ Binomial(L, p) (the binomial vote law of the second-stage design).
double binomial_tail(int L, double p, int mu);
// Dolph-Chebyshev window of length len, side lobes at -atten_db, peak 1.
std::vector<double> chebyshev_window(int64_t len, double atten_db);
// 6-dB bandwidth of a window in bins (bisection on the DTFT).
double window_6db_bins(const std::vector<double>& w);
// SNR*_min of eq. (opt) in dB for a half-bin tone at N_d/16 + 1/2 per dimension.
double design_snr_db(const HostPlan& p);

}  // namespace rsft
