// Prints the fold schedule the plan would choose for each geometry given on stdin, with its
// thread placement and epilogue tables, for tests/test_fold_schedule_host.py.
// Input lines: ndim loops sms n_0 .. n_{ndim-1} b_0 .. b_{ndim-1}
// Output per geometry: one line "key=value ..." (lists comma-separated), or "none".
#include <cstdio>
#include <vector>

#include "fold_schedule.h"

int main() {
  int ndim = 0, loops = 0, sms = 0;
  while (std::scanf("%d %d %d", &ndim, &loops, &sms) == 3) {
    rsft::Geometry g{};
    g.ndim = ndim;
    g.loops = loops;
    for (int d = 0; d < rsft::kMaxDim; ++d) g.n[d] = g.b[d] = g.m[d] = 1;
    long long v = 0;
    bool ok = true;
    for (int d = 0; d < 2 * ndim; ++d) {
      ok = ok && std::scanf("%lld", &v) == 1;
      (d < ndim ? g.n[d] : g.b[d - ndim]) = static_cast<int64_t>(v);
    }
    if (!ok) return 1;
    for (int d = 0; d < ndim; ++d) g.m[d] = g.n[d] / g.b[d];
    rsft::FoldSchedule fs{};
    if (!rsft::choose_fold_schedule(g, sms, fs)) {
      std::printf("none\n");
      continue;
    }
    std::vector<unsigned short> slots, digits;
    const char* why = rsft::fold_epilogue_tables(g.n, g.b, ndim, fs, slots, digits);
    std::printf("d_in=%d width=%d col_chunks=%d classes=%d rows_per_class=%d cps=%d crow=%d xcount=%d direct=%d "
                "lane_perm=%u red_mask=%d leaders=%d slots_per_x=%d error=%s slots=",
                fs.d_in, fs.width, fs.col_chunks, fs.classes, fs.rows_per_class, fs.cps, fs.crow, fs.xcount,
                fs.direct, fs.lane_perm, fs.red_mask, fs.leaders, fs.slots_per_x, why ? "yes" : "no");
    for (size_t i = 0; i < slots.size(); ++i) std::printf(i ? ",%u" : "%u", slots[i]);
    std::printf(" digits=");
    for (size_t i = 0; i < digits.size(); ++i) std::printf(i ? ",%u" : "%u", digits[i]);
    std::printf("\n");
  }
  return 0;
}
