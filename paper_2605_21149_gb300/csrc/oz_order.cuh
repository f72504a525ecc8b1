// Work order of the persistent split-precision GEMM (ozaki.cu): which output
// tiles of 128 x 128 a work item covers, and how many items a launch has.
// Shared by the kernel and a host check that compiles this header with a
// plain C++ compiler.
//
// One CTA per item (single form): item bid is tile (tm, tn), row by row; for
// a lower C only the tiles with tm >= tn.  Clusters of two (pair form): item
// idx is pair (TM, tn), tile rows 2 TM and 2 TM + 1 of tile column tn (one B
// tile shared by both CTAs).  For a lower C only the pairs with
// tn <= 2 TM + 1 and tn < tiles_m; a tile of a pair above the diagonal or
// past the last tile row is computed on zeros or discarded and stores
// nothing.  Pairs come in bands of `band` row pairs, inside a band column by
// column and the band's row pairs within each column.  The persistent grid
// takes the items in waves of one pair per cluster, which all stream K in
// step, and a wave over a compact band of rows and columns reads fewer
// distinct digit panels from DRAM than one along whole rows (about 25 panels
// a wave instead of about 45 at k = 6900).
#pragma once

#include <math.h>

#ifdef __CUDACC__
#define QMLGB_HD __host__ __device__ __forceinline__
#else
#define QMLGB_HD inline
#endif

namespace qmlgb {

// single form: tile of item bid
QMLGB_HD void oz_tile_of(int lower, int tiles_n, int bid, int &tm, int &tn) {
  if (!lower) {
    tm = bid / tiles_n;
    tn = bid % tiles_n;
    return;
  }
  // lower-triangle tiles (tm >= tn), row by row
  int r = (int)((sqrt(8.0 * bid + 1.0) - 1.0) * 0.5);
  while ((r + 1) * (r + 2) / 2 <= bid) ++r;
  while (r * (r + 1) / 2 > bid) --r;
  tm = r;
  tn = bid - r * (r + 1) / 2;
}

// pair form, lower C: pairs of column tn in the band of row pairs [t0, t1)
QMLGB_HD int oz_band_col_count(int tn, int t0, int t1) {
  const int need = tn >= 1 ? tn / 2 : 0;  // the smallest TM with 2 TM + 1 >= tn
  const int lo = need > t0 ? need : t0;
  return t1 > lo ? t1 - lo : 0;
}

// pair form: pair (TM, tn) of item idx
QMLGB_HD void oz_pair_of(int tiles_m, int tiles_n, int lower, int band, int idx, int &TM, int &tn) {
  const int T2 = (tiles_m + 1) / 2;
  for (int t0 = 0; t0 < T2; t0 += band) {
    const int t1 = t0 + band < T2 ? t0 + band : T2;
    // columns of this band: all of C, or for a lower C those up to the last
    // row pair's diagonal (and inside the matrix)
    const int ncol = lower ? (2 * t1 < tiles_m ? 2 * t1 : tiles_m) : tiles_n;
    if (!lower) {
      const int cnt = (t1 - t0) * ncol;
      if (idx < cnt) {
        tn = idx / (t1 - t0);
        TM = t0 + idx % (t1 - t0);
        return;
      }
      idx -= cnt;
      continue;
    }
    for (int c = 0; c < ncol; ++c) {
      const int cc = oz_band_col_count(c, t0, t1);
      if (idx < cc) {
        tn = c;
        TM = t1 - cc + idx;
        return;
      }
      idx -= cc;
    }
  }
  TM = T2;  // past the last item (not reached for idx below oz_item_count)
  tn = 0;
}

// items of a launch: tiles (single form) or tile-row pairs (pair form)
QMLGB_HD int oz_item_count(int tiles_m, int tiles_n, int lower, int pairs) {
  if (!pairs) return lower ? tiles_m * (tiles_m + 1) / 2 : tiles_m * tiles_n;
  const int T2 = (tiles_m + 1) / 2;
  return lower ? (tiles_m % 2 == 0 ? T2 * (T2 + 1) : (T2 - 1) * T2 + tiles_m) : T2 * tiles_n;
}

}  // namespace qmlgb
