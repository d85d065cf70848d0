// Prints the launch-shape candidates of the tensor-core contraction for the
// shapes given on the command line (M n_pad nk sm_count a_bytes b_bytes ...),
// one line per candidate: "variant nfast splits kbs valid", the default
// first, and an empty line after each shape.
#include <cstdio>
#include <cstdlib>

#include "tc_tune.h"

int main(int argc, char** argv) {
  using namespace sccsd;
  for (int i = 1; i + 5 < argc; i += 6) {
    TcShape s;
    s.M = std::atoll(argv[i]);
    s.n_pad = std::atoll(argv[i + 1]);
    s.nk = std::atoi(argv[i + 2]);
    s.sm_count = std::atoi(argv[i + 3]);
    const double ab = std::atof(argv[i + 4]), bb = std::atof(argv[i + 5]);
    const long long mt = (s.M + 127) / 128, nt = s.n_pad / 256;
    for (const TcConfig& c : tc_candidates(s, mt, nt, ab, bb))
      std::printf("%d %d %d %d %d\n", c.variant, c.nfast, c.splits, c.kbs,
                  (int)tc_config_valid(c, s.nk, nt));
    std::printf("\n");
  }
  return 0;
}
