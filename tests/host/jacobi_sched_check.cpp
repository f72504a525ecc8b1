// Host check of csrc/jacobi_sched.cuh, the index arithmetic of the
// float32 Jacobi phase, for every even order up to 160, the workloads' orders
// and the largest ones (to 640), with clusters of 8 and 16 CTAs:
//  * the pair ranges of the CTAs cover 0 .. h - 1 and j32_owner agrees;
//  * moving the columns with j32_dest_P / j32_dest_Q each round is a
//    permutation of the (pair, side) places, puts in every place the column
//    of the player the round-robin schedule names for the next round, and
//    brings every column home after a sweep of n - 1 rounds;
//  * in every round the writes that j32_next_inputs names fill each next-
//    round pair's a_pp, a_qq and a_qp exactly once, each from the right entry
//    (row and column player).
#include <algorithm>
#include <cstdio>
#include <vector>

#include JACOBI_SCHED_HEADER

using namespace qmlgb;

static int fail(const char *what, int n, int cn, int r, int a) {
  std::printf("FAIL %s n=%d cn=%d round=%d pair=%d\n", what, n, cn, r, a);
  return 1;
}

static int check_order(int n, int cn) {
  const int h = n / 2;
  // ownership
  if (j32_lo(0, h, cn) != 0 || j32_lo(cn, h, cn) != h) return fail("range ends", n, cn, -1, -1);
  for (int c = 0; c < cn; ++c)
    if (h >= cn && j32_lo(c + 1, h, cn) <= j32_lo(c, h, cn)) return fail("empty CTA", n, cn, -1, c);
  for (int a = 0; a < h; ++a) {
    const int c = j32_owner(a, h, cn);
    if (c < 0 || c >= cn || a < j32_lo(c, h, cn) || a >= j32_lo(c + 1, h, cn))
      return fail("owner", n, cn, -1, a);
  }
  // holder[2 a + side]: the player whose column sits at (pair a, side)
  std::vector<int> holder(n), next(n), home(n);
  for (int a = 0; a < h; ++a) {
    holder[2 * a] = a;
    holder[2 * a + 1] = n - 1 - a;
    if (jac_player(a, 0, n) != a || jac_player(n - 1 - a, 0, n) != n - 1 - a)
      return fail("round 0 players", n, cn, 0, a);
  }
  home = holder;
  for (int r = 0; r < n - 1; ++r) {
    // columns move
    std::fill(next.begin(), next.end(), -1);
    for (int a = 0; a < h; ++a) {
      int dp, ds;
      j32_dest_P(a, dp, ds);
      if (next[2 * dp + ds] != -1) return fail("P destination taken twice", n, cn, r, a);
      next[2 * dp + ds] = holder[2 * a];
      j32_dest_Q(a, h, dp, ds);
      if (next[2 * dp + ds] != -1) return fail("Q destination taken twice", n, cn, r, a);
      next[2 * dp + ds] = holder[2 * a + 1];
    }
    for (int a = 0; a < h; ++a)
      if (next[2 * a] != jac_player(a, r + 1, n) || next[2 * a + 1] != jac_player(n - 1 - a, r + 1, n))
        return fail("column not at its next-round slot", n, cn, r, a);
    // next-round rotation inputs: written[3 a' + slot] = (row, column player)
    std::vector<int> wrow(3 * h, -1), wcol(3 * h, -1), cnt(3 * h, 0);
    for (int a = 0; a < h; ++a) {
      const int colP = holder[2 * a], colQ = holder[2 * a + 1];
      int dpa, dps, dqa, dqs;
      j32_dest_P(a, dpa, dps);
      j32_dest_Q(a, h, dqa, dqs);
      const int rqP = dps == 0 ? jac_player(n - 1 - dpa, r + 1, n) : -1;
      const int rqQ = dqs == 0 ? jac_player(h, r + 1, n) : -1;
      for (int b = 0; b < h; ++b) {
        const int pb = jac_player(b, r, n), qb = jac_player(n - 1 - b, r, n);
        int tp[4], ts[4], te[4];
        const int m = j32_next_inputs(a, b, h, pb, qb, rqP, rqQ, tp, ts, te);
        if (m < 0 || m > 4) return fail("write count", n, cn, r, a);
        for (int i = 0; i < m; ++i) {
          const int row = (te[i] == 0 || te[i] == 2) ? pb : qb;
          const int col = te[i] < 2 ? colP : colQ;
          const int k = 3 * tp[i] + ts[i];
          ++cnt[k];
          wrow[k] = row;
          wcol[k] = col;
        }
      }
    }
    for (int a = 0; a < h; ++a) {
      const int p2 = jac_player(a, r + 1, n), q2 = jac_player(n - 1 - a, r + 1, n);
      const int want_row[3] = {p2, q2, q2}, want_col[3] = {p2, q2, p2};
      for (int s = 0; s < 3; ++s) {
        const int k = 3 * a + s;
        if (cnt[k] != 1) return fail("input written not exactly once", n, cn, r, a);
        if (wrow[k] != want_row[s] || wcol[k] != want_col[s]) return fail("wrong input entry", n, cn, r, a);
      }
    }
    holder = next;
  }
  if (holder != home) return fail("columns not home after a sweep", n, cn, n - 1, -1);
  return 0;
}

int main() {
  // every even order up to 160, then the orders of the workloads (TQU l <= 47:
  // 276; QU l <= 95: 282; TQU l <= 95: 564) and the largest ones
  std::vector<int> orders;
  for (int n = 4; n <= 160; n += 2) orders.push_back(n);
  for (int n : {202, 276, 282, 330, 438, 564, 638, 640}) orders.push_back(n);
  int cases = 0;
  for (int cn : {8, 16})
    for (int n : orders) {
      if (n / 2 < cn) continue;  // every CTA owns at least one pair
      if (check_order(n, cn)) return 1;
      ++cases;
    }
  std::printf("%d orders OK\n", cases);
  return 0;
}
