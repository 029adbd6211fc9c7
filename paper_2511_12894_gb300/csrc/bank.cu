// Template-bank structuring (Sec. III.A), on the host: sets of one reference and its dependent
// templates, each set's durations within a spread limit and its size within a size limit.
//   tau  = -t(f_low), t(f) = Psi'(f) / (2 pi) with t_c = 0 (Eq. A2): time from f_low to merger.
//   Stage 1: the bank in chirp-mass order (mc = (m1 m2)^(3/5) / (m1 + m2)^(1/5); equal values in
//            bank order) is halved (first half = floor of half) until each set's
//            max tau - min tau is within the spread limit.
//   Stage 2: each set in eta order (eta = m1 m2 / (m1 + m2)^2; equal values in bank order) is
//            halved until it holds at most the size limit.
//   Reference: the minimiser of sum_j |tau_i - tau_j| over the set; sums within 1e-9 of each
//            other (relative) tie (in one dimension all templates between the two middle
//            durations reach the minimum) and the lowest bank index wins.
// Sets are numbered depth first, first half first.
#include <algorithm>
#include <cmath>
#include <functional>
#include <vector>

#include "tf2.cuh"

namespace rf {

namespace {

// Halve idx until keep(set) holds, appending the sets depth first.
void halves(const std::vector<int>& idx, const std::function<bool(const std::vector<int>&)>& keep,
            std::vector<std::vector<int>>& out) {
  if (idx.size() <= 1 || keep(idx)) {
    out.push_back(idx);
    return;
  }
  const size_t h = idx.size() / 2;
  halves(std::vector<int>(idx.begin(), idx.begin() + h), keep, out);
  halves(std::vector<int>(idx.begin() + h, idx.end()), keep, out);
}

int reference_of(const std::vector<int>& idx, const std::vector<double>& tau) {
  int best = -1;
  double best_sum = INFINITY;
  for (int i : idx) {
    double s = 0.0;
    for (int j : idx) s += std::fabs(tau[i] - tau[j]);
    if (best < 0 || s < best_sum - 1e-9 * best_sum) {
      best = i;
      best_sum = s;
    } else if (std::fabs(s - best_sum) <= 1e-9 * best_sum && i < best) {
      best = i;
      best_sum = std::min(s, best_sum);
    }
  }
  return best;
}

}  // namespace

void bank_structure_impl(const rf_template* bank, int32_t count, double f_low, int pn_order, double max_spread,
                         int32_t max_size, int32_t* set_of, int32_t* ref_of_set, int32_t* n_sets,
                         double* duration_out) {
  *n_sets = 0;
  if (count == 0) return;
  std::vector<double> mc(count), eta(count), tau(count);
  for (int i = 0; i < count; ++i) {
    const double m1 = bank[i].m1, m2 = bank[i].m2;
    mc[i] = std::pow(m1 * m2, 0.6) / std::pow(m1 + m2, 0.2);
    eta[i] = m1 * m2 / ((m1 + m2) * (m1 + m2));
    rf_template t = bank[i];
    t.tc = 0.0;
    tau[i] = -(tf2_dphase(make_tf2(t, pn_order), f_low) / kTwoPi);
  }
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return mc[a] < mc[b] || (mc[a] == mc[b] && a < b); });
  std::vector<std::vector<int>> by_mc, sets;
  halves(order,
         [&](const std::vector<int>& s) {
           double lo = INFINITY, hi = -INFINITY;
           for (int i : s) {
             lo = std::min(lo, tau[i]);
             hi = std::max(hi, tau[i]);
           }
           return hi - lo <= max_spread;
         },
         by_mc);
  for (auto& s : by_mc) {
    std::vector<int> e = s;
    std::sort(e.begin(), e.end(), [&](int a, int b) { return eta[a] < eta[b] || (eta[a] == eta[b] && a < b); });
    halves(e, [&](const std::vector<int>& x) { return (int64_t)x.size() <= max_size; }, sets);
  }
  for (size_t g = 0; g < sets.size(); ++g) {
    for (int i : sets[g]) set_of[i] = (int32_t)g;
    ref_of_set[g] = reference_of(sets[g], tau);
  }
  *n_sets = (int32_t)sets.size();
  if (duration_out)
    for (int i = 0; i < count; ++i) duration_out[i] = tau[i];
}

}  // namespace rf
