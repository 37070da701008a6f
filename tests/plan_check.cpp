// Host-only driver of the FFT planning code (csrc/plan.h) for the CPU tests:
// prints, as one JSON object per line, the plan of each length given on the
// command line (as L:E pairs) -- radices, stage table, the twiddle table in
// double precision -- and the tile choices for a few row counts. Compiled
// with g++ by tests/test_plan_host.py; it launches nothing.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "plan.h"

int main(int argc, char** argv) {
  for (int a = 1; a < argc; ++a) {
    int L = 0, E = 0;
    if (std::sscanf(argv[a], "%d:%d", &L, &E) != 2) return 2;
    int rad[gad::kMaxStages];
    const int n = gad::radices_for(L, E, rad);
    std::printf("{\"L\": %d, \"E\": %d, \"radices\": [", L, E);
    for (int i = 0; i < n; ++i) std::printf("%s%d", i ? ", " : "", rad[i]);
    std::printf("]");
    if (n > 0) {
      std::vector<double> tw(2 * (size_t)L);
      gad::plan_twiddles<double>(rad, n, tw.data());
      gad::FftPlan fp;
      const bool ok = gad::make_fft_from(L, rad, n, tw.data(), fp);
      std::printf(", \"plan_ok\": %s, \"stages\": [", ok ? "true" : "false");
      for (int q = 0; q < fp.nst; ++q)
        std::printf("%s[%d, %d, %d]", q ? ", " : "", fp.st[q].radix, fp.st[q].ns, fp.st[q].tw_off);
      std::printf("], \"twiddles\": [");
      for (int i = 0; i < 2 * (L - 1); ++i) std::printf("%s%.17g", i ? ", " : "", tw[i]);
      std::printf("]");
      int rrev[gad::kMaxStages];
      const int nr = gad::plan_radices(L, E, true, rrev);
      std::printf(", \"reversed\": [");
      for (int i = 0; i < nr; ++i) std::printf("%s%d", i ? ", " : "", rrev[i]);
      std::vector<double> twr(2 * (size_t)L);
      gad::plan_twiddles<double>(rrev, nr, twr.data());
      std::printf("], \"reversed_twiddles\": [");
      for (int i = 0; i < 2 * (L - 1); ++i) std::printf("%s%.17g", i ? ", " : "", twr[i]);
      std::printf("]");
    }
    std::printf(", \"tiles\": [");
    const int divs[4] = {0, 1, 16, 4096};
    for (int d = 0; d < 4; ++d) {
      gad::TileShape ts;
      const bool ok = gad::choose_tile(L, E, L + 1, divs[d], 8, ts);
      std::printf("%s[%d, %d, %d, %d, %d, %zu]", d ? ", " : "", divs[d], ok ? 1 : 0, ts.W, ts.T, ts.ld, ts.smem);
    }
    std::printf("]}\n");
  }
  return 0;
}
