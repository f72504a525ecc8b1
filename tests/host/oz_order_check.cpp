// Host check of csrc/oz_order.cuh, the work order of the split-precision
// GEMM: for full and lower C, tile grids up to 48 x 48, band widths 1 .. 9
// and 4096, and both forms (one CTA per tile; clusters of two on tile-row
// pairs), the items 0 .. oz_item_count - 1 cover every output tile exactly
// once (for a lower C the tiles with tm >= tn), name no tile outside the
// grid, and (pair form) never name the same pair twice.
#include <cstdio>
#include <vector>

#include OZ_ORDER_HEADER

using namespace qmlgb;

static int fail(const char *what, int tm, int tn, int lower, int pairs, int band, int item) {
  std::printf("FAIL %s tiles=%dx%d lower=%d pairs=%d band=%d item=%d\n", what, tm, tn, lower, pairs,
              band, item);
  return 1;
}

static int check(int tiles_m, int tiles_n, int lower, int pairs, int band) {
  std::vector<int> hit((size_t)tiles_m * tiles_n, 0);
  const int count = oz_item_count(tiles_m, tiles_n, lower, pairs);
  if (pairs) {
    const int T2 = (tiles_m + 1) / 2;
    std::vector<int> seen((size_t)T2 * tiles_n, 0);
    for (int idx = 0; idx < count; ++idx) {
      int TM = -1, tn = -1;
      oz_pair_of(tiles_m, tiles_n, lower, band, idx, TM, tn);
      if (TM < 0 || TM >= T2 || tn < 0 || tn >= tiles_n) return fail("pair outside", tiles_m, tiles_n, lower, pairs, band, idx);
      if (lower && (tn > 2 * TM + 1 || tn >= tiles_m)) return fail("pair above the diagonal", tiles_m, tiles_n, lower, pairs, band, idx);
      if (seen[(size_t)TM * tiles_n + tn]++) return fail("pair twice", tiles_m, tiles_n, lower, pairs, band, idx);
      for (int r = 0; r < 2; ++r) {
        const int tm = 2 * TM + r;
        if (tm >= tiles_m || (lower && tn > tm)) continue;  // computed on zeros, not stored
        ++hit[(size_t)tm * tiles_n + tn];
      }
    }
  } else {
    for (int bid = 0; bid < count; ++bid) {
      int tm = -1, tn = -1;
      oz_tile_of(lower, tiles_n, bid, tm, tn);
      if (tm < 0 || tm >= tiles_m || tn < 0 || tn >= tiles_n || (lower && tn > tm))
        return fail("tile outside", tiles_m, tiles_n, lower, pairs, band, bid);
      ++hit[(size_t)tm * tiles_n + tn];
    }
  }
  for (int tm = 0; tm < tiles_m; ++tm)
    for (int tn = 0; tn < tiles_n; ++tn) {
      const int want = (lower && tn > tm) ? 0 : 1;
      if (hit[(size_t)tm * tiles_n + tn] != want) return fail("tile not covered once", tiles_m, tiles_n, lower, pairs, band, tm * tiles_n + tn);
    }
  return 0;
}

int main() {
  int cases = 0;
  for (int lower = 0; lower < 2; ++lower)
    for (int tiles_m = 1; tiles_m <= 48; ++tiles_m)
      for (int tiles_n = 1; tiles_n <= 48; ++tiles_n) {
        if (lower && tiles_n != tiles_m) continue;  // a lower C is square
        for (int pairs = 0; pairs < 2; ++pairs) {
          if (pairs && tiles_m < 2) continue;  // the launch takes one CTA per tile there
          for (int band : {1, 2, 3, 4, 5, 6, 7, 8, 9, 4096}) {
            if (check(tiles_m, tiles_n, lower, pairs, band)) return 1;
            ++cases;
            if (!pairs) break;  // the band only orders pairs
          }
        }
      }
  std::printf("%d cases OK\n", cases);
  return 0;
}
