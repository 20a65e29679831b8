// Host harness for the fixed-point reduction arithmetic of the solver
// (paper_2003_00082_gb300/csrc/cgp_fixed.h).  Reads groups of doubles (as
// hex bit patterns) from stdin: a line "G n" starts a group of n values.
// Each group is summed relative to its own largest exponent, the group sums
// are aligned to the overall largest exponent and added, exactly as the
// GPU does per warp, per block and across blocks.  Prints the bit pattern
// of the converted total.
//
// A first line "R red" selects the tagged form: every group sum (one
// block's partial) goes through a tagged slot of reduction `red` and back
// before the groups are added.  Exit status 3: a slot did not read as
// current; 4: a slot built from halves of two stores, or a zeroed slot,
// read as current.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "cgp_fixed.h"

using namespace cgp::fx;

int main() {
  std::vector<std::vector<double>> groups;
  char tag[8];
  int n;
  int red = -1;
  while (std::scanf("%7s %d", tag, &n) == 2) {
    if (tag[0] == 'R') {
      red = n;
      continue;
    }
    std::vector<double> g(n);
    for (int i = 0; i < n; ++i) {
      unsigned long long b;
      if (std::scanf("%llx", &b) != 1) return 2;
      g[i] = from_bits(b);
    }
    groups.push_back(g);
  }
  std::vector<I128> gsum;
  std::vector<int> gexp;
  int E = 1;
  for (auto& g : groups) {
    int e = 1;
    for (double v : g) e = exponent_of(v) > e ? exponent_of(v) : e;
    I128 s = 0;
    if (e < kBadExp)
      for (double v : g) s = add(s, image(v, e));
    gsum.push_back(s);
    gexp.push_back(e);
    E = e > E ? e : E;
  }
  if (red >= 0) {
    I128 t = 0;
    for (size_t i = 0; i < gsum.size(); ++i) {
      uint64_t lo, hi, lo2, hi2;
      pack_tagged(gsum[i], gexp[i], red, lo, hi);
      pack_tagged(gsum[i] + 12345, gexp[i], red - 2, lo2, hi2);   // the bank's previous store
      if (!tagged_current(lo, hi, red)) return 3;
      if (tagged_current(lo2, hi, red) || tagged_current(lo, hi2, red) || tagged_current(0, 0, red)) return 4;
      if (tagged_exponent(hi) != gexp[i]) return 3;
      if (E < kBadExp) t = add(t, sar(tagged_mantissa(lo, hi), E - gexp[i]));
    }
    std::printf("%016llx\n", (unsigned long long)dbits(E < kBadExp ? to_double(t, E + kTagShift) : to_double(0, kBadExp)));
    return 0;
  }
  I128 t = 0;
  if (E < kBadExp)
    for (size_t i = 0; i < gsum.size(); ++i) t = add(t, sar(gsum[i], E - gexp[i]));
  std::printf("%016llx\n", (unsigned long long)dbits(to_double(t, E)));
  return 0;
}
