// Coverage-driven active-space sampling (Numerical Implementation, Algorithm 1) on the host: the
// greedy cover is sequential (each candidate is judged against what earlier ones covered), so it
// runs once per problem on the CPU before the flow is set up.  Contract: include/qflow.h.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <new>
#include <vector>

#include "qflow_internal.h"

namespace {

// SplitMix64 (Steele, Lea and Flood, 2014): Weyl-sequence state, variant-13 mixing of the output.
struct SplitMix64 {
  uint64_t state;
  uint64_t next() {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
};

// k distinct elements of 0..m-1 in ascending order: partial Fisher-Yates from the identity.
void draw(SplitMix64& rng, int m, int k, std::vector<int>& scratch, int* out) {
  scratch.resize((size_t)m);
  for (int i = 0; i < m; ++i) scratch[(size_t)i] = i;
  for (int i = 0; i < k; ++i) {
    const int j = i + (int)(rng.next() % (uint64_t)(m - i));
    std::swap(scratch[(size_t)i], scratch[(size_t)j]);
  }
  for (int i = 0; i < k; ++i) out[i] = scratch[(size_t)i];
  std::sort(out, out + k);
}

struct Kept {
  double de;
  int occ[3], vir[3];
};

}  // namespace

extern "C" int qflow_sample_spaces(int32_t nocc, int32_t nvir, int32_t no, int32_t nv, const double* eps,
                                   uint64_t seed, qflow_space* out, int64_t capacity, int64_t* count,
                                   int64_t* draws) {
  if (!eps || !count || nocc < 2 || nvir < 2 || nocc + nvir > 128 || no < 2 || nv < 2 || no > 3 || nv > 3 ||
      no > nocc || nv > nvir || capacity < 0 || (capacity > 0 && !out))
    return QFLOW_ERR_ARG;
  for (int p = 0; p < nocc + nvir; ++p)
    if (!isfinite(eps[p])) return QFLOW_ERR_ARG;
  try {
    // pair indices of the minimal coverage set C_min = {(o1 < o2, v1 < v2)}
    std::vector<int> pair_o((size_t)nocc * nocc, -1), pair_v((size_t)nvir * nvir, -1);
    int npo = 0, npv = 0;
    for (int a = 0; a < nocc; ++a)
      for (int b = a + 1; b < nocc; ++b) pair_o[(size_t)a * nocc + b] = npo++;
    for (int a = 0; a < nvir; ++a)
      for (int b = a + 1; b < nvir; ++b) pair_v[(size_t)a * nvir + b] = npv++;
    std::vector<uint8_t> covered((size_t)npo * npv, 0);
    int64_t remaining = (int64_t)npo * npv;
    SplitMix64 rng{seed};
    std::vector<int> scratch;
    std::vector<Kept> kept;
    std::vector<size_t> fresh;
    int64_t n_draws = 0;
    // every candidate has a positive chance to cover a remaining tuple; the bound only guards
    // against a broken generator
    const int64_t max_draws = (int64_t)1 << 40;
    while (remaining > 0 && n_draws < max_draws) {
      Kept k{};
      draw(rng, nocc, no, scratch, k.occ);
      draw(rng, nvir, nv, scratch, k.vir);
      ++n_draws;
      fresh.clear();
      for (int i = 0; i < no; ++i)
        for (int j = i + 1; j < no; ++j)
          for (int a = 0; a < nv; ++a)
            for (int b = a + 1; b < nv; ++b) {
              const size_t x = (size_t)pair_o[(size_t)k.occ[i] * nocc + k.occ[j]];
              const size_t y = (size_t)pair_v[(size_t)k.vir[a] * nvir + k.vir[b]];
              if (!covered[x * (size_t)npv + y]) fresh.push_back(x * (size_t)npv + y);
            }
      if (fresh.empty()) continue;  // covers nothing new: discarded
      for (size_t t : fresh) covered[t] = 1;
      remaining -= (int64_t)fresh.size();
      double sv = 0.0, so = 0.0;
      for (int a = 0; a < nv; ++a) sv = sv + eps[nocc + k.vir[a]];
      for (int i = 0; i < no; ++i) so = so + eps[k.occ[i]];
      k.de = sv - so;
      kept.push_back(k);
    }
    if (remaining > 0) return QFLOW_ERR_NOCONV;
    std::stable_sort(kept.begin(), kept.end(), [](const Kept& x, const Kept& y) { return x.de < y.de; });
    *count = (int64_t)kept.size();
    if (draws) *draws = n_draws;
    if ((int64_t)kept.size() > capacity) return QFLOW_ERR_TOO_LARGE;
    for (size_t r = 0; r < kept.size(); ++r) {
      qflow_space& q = out[r];
      q.no = no;
      q.nv = nv;
      for (int t = 0; t < 6; ++t) q.orb[t] = -1;
      for (int i = 0; i < no; ++i) q.orb[i] = kept[r].occ[i];
      for (int a = 0; a < nv; ++a) q.orb[no + a] = nocc + kept[r].vir[a];
    }
  } catch (const std::bad_alloc&) {
    return QFLOW_ERR_OOM;
  }
  return QFLOW_OK;
}
