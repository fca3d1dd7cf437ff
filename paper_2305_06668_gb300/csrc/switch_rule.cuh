// When the mixed form leaves FP32 (reading R22; host code, no device work).
//
// Fed once per FP32 iteration with r_i, the largest residual norm of the k sought pairs.
// With a fixed threshold (switch_tol > 0) it leaves at the first r_i <= switch_tol.
// Otherwise it leaves once the FP32 phase has reached its rounding floor:
//   * after r_i fell below 1% of its first value, a sudden loss of a fast rate: over the
//     three iterations i-5 .. i-2 it fell by a factor <= 0.6 per iteration on geometric
//     average, then two iterations in a row (i-1 and i) cut it by less than 25% each;
//   * or no 10% improvement on the best r for 2 iterations (once the best is below 1% of
//     the first value) or for 5 iterations (at any level).
#pragma once

namespace lobpcg {

struct MixedSwitch {
  double switch_tol = 0.0;
  double first_rk = -1.0, best_rk = 1e300;
  int since_best = 0;
  double rk_hist[5] = {0.0, 0.0, 0.0, 0.0, 0.0};  // r_{i-5} .. r_{i-1}
  int nhist = 0;

  // r_i of this iteration; true: leave FP32 after it.
  bool step(double rk) {
    if (first_rk < 0.0) first_rk = rk;
    bool rate_lost = false;
    if (nhist >= 5 && rk <= 1e-2 * first_rk) {
      const bool fast = rk_hist[3] <= 0.216 * rk_hist[0];  // (r_{i-2} / r_{i-5})^(1/3) <= 0.6
      rate_lost = fast && rk_hist[4] > 0.75 * rk_hist[3] && rk > 0.75 * rk_hist[4];
    }
    if (nhist < 5) {
      rk_hist[nhist++] = rk;
    } else {
      for (int h = 0; h < 4; ++h) rk_hist[h] = rk_hist[h + 1];
      rk_hist[4] = rk;
    }
    if (switch_tol > 0.0) return rk <= switch_tol;
    if (rate_lost) return true;
    if (rk < 0.9 * best_rk) {
      best_rk = rk, since_best = 0;
      return false;
    }
    return ++since_best >= 5 || (since_best >= 2 && best_rk <= 1e-2 * first_rk);
  }
};

}  // namespace lobpcg
