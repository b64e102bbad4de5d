// Host-only checks of the Newton load schedule (LoadSchedule in pfem_internal.h): uncut
// levels are exactly k / n, a cut halves the increment from the last converged level, the
// increment doubles back after each converged level, and cuts stop at the limit or at the
// smallest increment. Prints "ok" and exits 0, or names the failed check and exits 1.
#include <cstdio>

#include "pfem_internal.h"

using pfem::LoadSchedule;

static int fails = 0;
static void check(bool c, const char* what) {
  if (!c) {
    std::printf("FAILED: %s\n", what);
    ++fails;
  }
}

int main() {
  for (int n : {1, 2, 3, 5, 7, 20}) {  // no cuts: the fractions k / n, then the last level
    LoadSchedule s;
    s.start(n);
    for (int k = 1; k <= n; ++k) {
      check(s.fraction() == (double)k / (double)n, "uncut fraction equals k / n");
      check(s.last() == (k == n), "last level only at the full load");
      if (!s.last()) s.converged();
    }
    check(s.cuts == 0, "no cuts without failures");
  }
  {  // cut at the first level of 5: 1/10, then 1/5 + ... regrowth to the 1/5 grid
    LoadSchedule s;
    s.start(5);
    check(s.cut(), "first cut allowed");
    check(s.fraction() == 0.1, "half of the first increment");
    s.converged();  // at 0.1, increment back to 1/5
    check(s.fraction() == 0.3, "doubled increment after a converged level");
    s.converged();
    check(s.fraction() == 0.5, "full increment again");
    while (!s.last()) s.converged();
    check(s.fraction() == 1.0, "ends at the full load");
    check(s.cuts == 1, "one cut counted");
  }
  {  // repeated failures at one level: 6 halvings reach the smallest increment (1/64 step)
    LoadSchedule s;
    s.start(1);
    int n = 0;
    while (s.cut()) ++n;
    check(n == 6, "six cuts down to the smallest increment");
    check(s.fraction() == 1.0 / 64.0, "smallest increment is 1/64 of a step");
    check(s.cuts == 6, "cuts counted");
  }
  {  // the per-solve limit
    LoadSchedule s;
    s.start(2);
    int n = 0;
    for (int round = 0; round < 10; ++round) {  // fail, converge, fail, converge, ...
      if (!s.cut()) break;
      ++n;
      if (!s.last()) s.converged();
    }
    check(n <= pfem::kMaxLoadCuts && s.cuts <= pfem::kMaxLoadCuts, "at most kMaxLoadCuts cuts");
  }
  if (fails == 0) std::printf("ok\n");
  return fails == 0 ? 0 : 1;
}
