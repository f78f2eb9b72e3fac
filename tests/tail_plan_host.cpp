// Host-side check of the fine-chunked tail plan (TailPlan, tail_plan in
// rad_impl.h): reads lines "tensor_core n n_tiles ck n_chunks grid bins_per_tile"
// from standard input and prints, per line, "tiles0 ck0 n_chunks0 tiles1 ck1
// n_chunks1 items fine_floats level1_offset".  Driven by
// tests/test_tail_plan_cpu.py.
#include <cstdio>

#include "rad_impl.h"

int main() {
  static_assert(radimpl::kTailLevels == 2, "the output has two levels");
  int tc, n_tiles, ck, n_chunks, bins_per_tile;
  long long n, grid;
  while (std::scanf("%d %lld %d %d %d %lld %d", &tc, &n, &n_tiles, &ck, &n_chunks, &grid,
                    &bins_per_tile) == 7) {
    const radimpl::TailPlan t = radimpl::tail_plan(tc != 0, n, n_tiles, ck, n_chunks, grid);
    std::printf("%d %d %d %d %d %d %lld %lld %lld\n", t.lv[0].tiles, t.lv[0].ck, t.lv[0].n_chunks,
                t.lv[1].tiles, t.lv[1].ck, t.lv[1].n_chunks, t.items(n_tiles, n_chunks),
                t.fine_floats(bins_per_tile), t.level_offset(1, bins_per_tile));
  }
  return 0;
}
