// Test harness (host only): the autotuner's candidate schedules and its pick
// among measured times (fake timings given on the command line; "inf" for a
// candidate that failed).  Prints one JSON line.
//   usage: sched_check mg(0|1) t0 t1 ...
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "plan.h"

using namespace exx;

int main(int argc, char **argv)
{
    if (argc < 2) return 2;
    const bool mg = std::atoi(argv[1]) != 0;
    const std::vector<exx_schedule> c = schedule_candidates(mg, 0.7);
    std::vector<double> ms;
    for (int k = 2; k < argc; ++k) ms.push_back(std::strtod(argv[k], nullptr));
    const int pick = ms.empty() ? -1 : pick_schedule(ms.data(), (int)ms.size());
    std::printf("{\"n\": %zu, \"pick\": %d, \"cand\": [", c.size(), pick);
    for (size_t k = 0; k < c.size(); ++k)
        std::printf("%s[%d, %.2f, %d]", k ? ", " : "", c[k].precond, c[k].omega, c[k].inner_shift);
    std::printf("]}\n");
    return 0;
}
