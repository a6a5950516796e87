// Host driver of the autotuner's rules (sbp_tune.h) for tests/test_host_tune.py.
// Usage: tune_driver ni nj viscous critical n_sm [strip,rows,rows_upd=ms ...]
// Prints the eligible candidates ("eligible s,r,u ...") and, given times for some of them, the
// kept one ("pick s,r,u"). The widths and the staging flag are the library's (marching strips
// of 58 columns, column-marching strips of 116 and 244, TMA flag 0x10000, 32-column tiles).
#include <cstdio>
#include <cstdlib>
#include <utility>
#include <vector>

#include "sbp_tune.h"

using namespace sbp;

int main(int argc, char **argv) {
  if (argc < 6) return 2;
  const TuneMesh m{std::atoi(argv[1]), std::atoi(argv[2]), std::atoi(argv[3]) != 0, 32, 0x10000, 58};
  const bool critical = std::atoi(argv[4]) != 0;
  const int n_sm = std::atoi(argv[5]);
  const std::vector<TuneCand> cands = tune_candidates(58, 116, 244, 0x10000);
  const std::vector<int> el = tune_eligible(cands.data(), (int)cands.size(), m, critical, n_sm);
  std::printf("eligible");
  for (int i : el) std::printf(" %d,%d,%d", cands[i].strip, cands[i].rows, cands[i].rows_upd);
  std::printf("\n");
  std::vector<std::pair<float, int>> timed;
  for (int a = 6; a < argc; ++a) {
    int s, r, u;
    float ms;
    if (std::sscanf(argv[a], "%d,%d,%d=%f", &s, &r, &u, &ms) != 4) return 2;
    int found = -1;
    for (int i : el)
      if (cands[i].strip == s && cands[i].rows == r && cands[i].rows_upd == u) found = i;
    if (found < 0) return 3;  // timing for a candidate that is not eligible
    timed.push_back({ms, found});
  }
  if (!timed.empty()) {
    const int p = tune_pick(cands.data(), timed, m, critical);
    std::printf("pick %d,%d,%d\n", cands[p].strip, cands[p].rows, cands[p].rows_upd);
  }
  return 0;
}
