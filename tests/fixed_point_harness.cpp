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
//
// A line "W w" (with "R red") selects instead the 64-bit tagged form of the
// solver's iterations: groups are warps (64-bit images relative to the
// warp's largest exponent, summed exactly), every w consecutive warps a
// block (warp sums aligned to the block's largest exponent with 5 bits of
// headroom, summed), every block's sum through an unshifted tagged slot,
// and the slots added as the solver's poll does.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "cgp_fixed.h"

using namespace cgp::fx;

int main() {
  std::vector<std::vector<double>> groups;
  char tag[8];
  int n;
  int red = -1, wpb = 0;
  while (std::scanf("%7s %d", tag, &n) == 2) {
    if (tag[0] == 'R') {
      red = n;
      continue;
    }
    if (tag[0] == 'W') {
      wpb = n;
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
  if (wpb > 0 && red >= 0) {
    // warps
    std::vector<int64_t> ws;
    std::vector<int> we;
    for (auto& g : groups) {
      int e = 1;
      for (double v : g) e = exponent_of(v) > e ? exponent_of(v) : e;
      int64_t s = 0;
      if (e < kBadExp)
        for (double v : g) s += image64(v, e);
      ws.push_back(s);
      we.push_back(e);
    }
    // blocks, their slots, and the poll's sum
    std::vector<uint64_t> los, his;
    int Eg = 1;
    for (size_t b0 = 0; b0 < ws.size(); b0 += (size_t)wpb) {
      const size_t b1 = b0 + (size_t)wpb < ws.size() ? b0 + (size_t)wpb : ws.size();
      int Eb = 1;
      for (size_t w = b0; w < b1; ++w) Eb = we[w] > Eb ? we[w] : Eb;
      int64_t S = 0;
      if (Eb < kBadExp)
        for (size_t w = b0; w < b1; ++w) {
          const int s = Eb - we[w] + 5;
          S += ws[w] >> (s > 63 ? 63 : s);
        }
      uint64_t lo, hi, lo2, hi2;
      pack_tagged((I128)S, Eb, red, lo, hi, 0);
      pack_tagged((I128)S + 777, Eb, red - 2, lo2, hi2, 0);
      if (!tagged_current(lo, hi, red)) return 3;
      if (tagged_current(lo2, hi, red) || tagged_current(lo, hi2, red) || tagged_current(0, 0, red)) return 4;
      if (tagged_exponent(hi) != Eb || tagged_mantissa(lo, hi) != (I128)S) return 3;
      los.push_back(lo);
      his.push_back(hi);
      Eg = Eb > Eg ? Eb : Eg;
    }
    I128 t = 0;
    if (Eg < kBadExp)
      for (size_t b = 0; b < los.size(); ++b) t = add(t, sar(tagged_mantissa(los[b], his[b]), Eg - tagged_exponent(his[b])));
    std::printf("%016llx\n", (unsigned long long)dbits(Eg < kBadExp ? to_double(t, Eg + 55) : to_double(0, kBadExp)));
    return 0;
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
