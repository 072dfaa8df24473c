// Host check of the warp tiling of apply stages (no GPU).
//
// The stage kernels write every output row of a stage from exactly one warp
// tile, which is what makes the apply deterministic without atomics, and their
// warp shuffles need every lane of a warp to run the same number of row passes.
// This harness draws seeded random stages of block descriptors (uneven shapes,
// empty blocks, odd and even column counts) and tiles them with the library's
// make_tiles for every autotuner candidate (tile budgets of 4, 16 and 64 KB x 2,
// 4 or 8 16-byte vectors per lane and row) and the default, then checks:
//   * the tiles of each block cover its rows 0 .. M-1 once, in order, and blocks
//     with no rows get no tile;
//   * g (lanes per row) is a power of two <= 32 and nr a positive multiple of 32/g;
//   * a lane streams at most the target number of 16-byte vectors per row unless
//     g = 32 already;
//   * a tile holds at most the budget of factor bytes (at least one pass of 32/g
//     rows, and never less than the 2 KB floor).
// Prints "ok <stages checked>" and exits 0, or the first violation.
#include <cstdio>
#include <cstdint>
#include <vector>

#include "internal.h"

using namespace vie;

static uint64_t g_state = 0x9e3779b97f4a7c15ull;
static uint32_t rnd(uint32_t n) {  // splitmix64, reduced to [0, n)
  uint64_t z = (g_state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  return (uint32_t)(z % n);
}

static bool check(const std::vector<OpDesc>& ops, const std::vector<Tile>& tiles, int64_t budget, int vec,
                  const char* what) {
  std::vector<int64_t> next(ops.size(), 0);  // next uncovered row of each block
  for (const Tile& t : tiles) {
    if (t.op < 0 || t.op >= (int)ops.size()) { std::printf("FAIL %s: tile of no block\n", what); return false; }
    const OpDesc& o = ops[t.op];
    const int g = t.g;
    if (g < 1 || g > 32 || (g & (g - 1))) { std::printf("FAIL %s: g = %d\n", what, g); return false; }
    const int rp = 32 / g;
    if (t.nr <= 0 || t.nr % rp) { std::printf("FAIL %s: nr = %d with g = %d\n", what, t.nr, g); return false; }
    if (t.r0 != next[t.op] || t.r0 >= o.M) {
      std::printf("FAIL %s: block %d tile starts at %d, expected %lld\n", what, t.op, t.r0, (long long)next[t.op]);
      return false;
    }
    const int64_t rows = std::min<int64_t>(t.nr, o.M - t.r0);
    next[t.op] = t.r0 + rows;
    const int per = (o.K + 1) / 2;  // 16-byte vectors per row (complex FP32)
    if (g < 32 && (int64_t)vec * g < per) { std::printf("FAIL %s: g = %d too small for K = %d\n", what, g, o.K); return false; }
    const int64_t row_bytes = (int64_t)o.ld * 8;
    const int64_t cap = std::max<int64_t>(std::max<int64_t>(2048, budget), rp * row_bytes);
    if (rows * row_bytes > cap) {
      std::printf("FAIL %s: tile of %lld bytes over the budget %lld\n", what, (long long)(rows * row_bytes),
                  (long long)cap);
      return false;
    }
  }
  for (size_t i = 0; i < ops.size(); ++i)
    if (next[i] != std::max<int64_t>(0, ops[i].M)) {
      std::printf("FAIL %s: block %zu covered to row %lld of %d\n", what, i, (long long)next[i], ops[i].M);
      return false;
    }
  return true;
}

int main() {
  const int64_t budgets[3] = {4096, 16384, 65536};
  const int vecs[3] = {2, 4, 8};
  int checked = 0;
  for (int trial = 0; trial < 200; ++trial) {
    std::vector<OpDesc> ops;
    const int nops = 1 + (int)rnd(trial % 4 == 0 ? 2000 : 60);
    int64_t off = 0;
    for (int i = 0; i < nops; ++i) {
      OpDesc o{};
      const uint32_t kind = rnd(10);
      o.M = kind == 0 ? 0 : (kind < 4 ? 1 + (int)rnd(8) : 1 + (int)rnd(kind < 8 ? 200 : 3000));
      o.K = kind == 9 ? 1 + (int)rnd(4000) : (int)rnd(300);
      o.ld = (o.K + 1) & ~1;
      o.mat_off = off;
      off += (int64_t)o.M * o.ld;
      ops.push_back(o);
    }
    std::vector<Tile> tiles;
    make_tiles(ops, tiles);
    if (!check(ops, tiles, 16384, 4, "default tiling")) return 1;
    ++checked;
    for (int64_t b : budgets)
      for (int v : vecs) {
        make_tiles(ops, tiles, b, v);
        if (!check(ops, tiles, b, v, "candidate tiling")) return 1;
        ++checked;
      }
  }
  std::printf("ok %d\n", checked);
  return 0;
}
