// Host-side check of the fine-chunked tail plan (TailPlan, tail_plan in
// rad_impl.h): reads lines "tensor_core n n_tiles ck n_chunks grid bins_per_tile"
// from standard input and prints, per line, "tiles ck_f n_chunks_f items
// fine_floats".  Driven by tests/test_tail_plan_cpu.py.
#include <cstdio>

#include "rad_impl.h"

int main() {
  int tc, n_tiles, ck, n_chunks, bins_per_tile;
  long long n, grid;
  while (std::scanf("%d %lld %d %d %d %lld %d", &tc, &n, &n_tiles, &ck, &n_chunks, &grid,
                    &bins_per_tile) == 7) {
    const radimpl::TailPlan t = radimpl::tail_plan(tc != 0, n, n_tiles, ck, n_chunks, grid);
    std::printf("%d %d %d %lld %lld\n", t.tiles, t.ck, t.n_chunks, t.items(n_tiles, n_chunks),
                t.fine_floats(bins_per_tile));
  }
  return 0;
}
