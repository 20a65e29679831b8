// Host harness for the fixed-point reduction arithmetic of the solver
// (paper_2003_00082_gb300/csrc/cgp_fixed.h).  Reads groups of doubles (as
// hex bit patterns) from stdin: a line "G n" starts a group of n values.
// Each group is summed relative to its own largest exponent, the group sums
// are aligned to the overall largest exponent and added, exactly as the
// GPU does per warp, per block and across blocks.  Prints the bit pattern
// of the converted total.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "cgp_fixed.h"

using namespace cgp::fx;

int main() {
  std::vector<std::vector<double>> groups;
  char tag[8];
  int n;
  while (std::scanf("%7s %d", tag, &n) == 2) {
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
  I128 t = 0;
  if (E < kBadExp)
    for (size_t i = 0; i < gsum.size(); ++i) t = add(t, sar(gsum[i], E - gexp[i]));
  std::printf("%016llx\n", (unsigned long long)dbits(to_double(t, E)));
  return 0;
}
