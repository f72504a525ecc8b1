// Index arithmetic of the parallel cyclic Jacobi schedule, shared by the
// eigensolver kernels (eig.cu) and a host check that compiles this header
// with a plain C++ compiler.
//
// Round-robin (circle) schedule on n = 2h players: slot x of round r holds
// player(x, r); slots a and n - 1 - a (a < h) form pair a; player 0 never
// moves and the others advance one slot a round along 1 .. n - 1, so after
// n - 1 rounds (one sweep) every pair of players has met once and slot x
// holds player x again.
//
// The float32 phase keeps, for each pair a, the column of the player in slot
// a (side P) and in slot n - 1 - a (side Q).  Between rounds the column in
// slot y moves to slot y - 1 (y >= 2), slot 1's to slot n - 1, and slot 0's
// stays; in pairs and sides that is j32_dest_P / j32_dest_Q below.  Pairs
// are owned by the CTAs of one cluster in contiguous ranges.
#pragma once

#ifdef __CUDACC__
#define QMLGB_HD __host__ __device__ __forceinline__
#else
#define QMLGB_HD inline
#endif

namespace qmlgb {

QMLGB_HD int jac_player(int x, int r, int n) {
  return x == 0 ? 0 : ((x - 1 + r) % (n - 1)) + 1;
}

// pairs [j32_lo(c), j32_lo(c + 1)) belong to CTA c of cn
QMLGB_HD int j32_lo(int c, int h, int cn) { return c * h / cn; }
// the CTA that owns pair a (the c with j32_lo(c) <= a < j32_lo(c + 1))
QMLGB_HD int j32_owner(int a, int h, int cn) { return ((a + 1) * cn + h - 1) / h - 1; }

// where pair a's P column (slot a) sits in the next round: P(a - 1), except
// P(0) -> P(0) and P(1) -> Q(0); side 0 is P, 1 is Q
QMLGB_HD void j32_dest_P(int a, int &pair, int &side) {
  pair = a <= 1 ? 0 : a - 1;
  side = a == 1 ? 1 : 0;
}
// where pair a's Q column (slot n - 1 - a) sits in the next round: Q(a + 1),
// except Q(h - 1) -> P(h - 1)
QMLGB_HD void j32_dest_Q(int a, int h, int &pair, int &side) {
  pair = a == h - 1 ? h - 1 : a + 1;
  side = a == h - 1 ? 0 : 1;
}

// The next round's rotation inputs among the four entries that the task of
// pair a's columns and pair b's rows writes in a round (rows pb, qb, the
// players of pair b): up to four (target pair tp, slot ts, entry te), with
// slot 0 = a_pp, 1 = a_qq, 2 = a_qp of the target pair and entry 0 = row pb
// of the P column, 1 = row qb of the P column, 2 = row pb of the Q column,
// 3 = row qb of the Q column.  The diagonal of both columns lies in the
// pair's own block (b == a); a column that becomes a P column also carries
// a_qp, at the row of its next partner: rqP for pair a's P column (used when
// it stays a P column), rqQ for its Q column (used when it becomes P(h - 1)).
// Returns how many.
QMLGB_HD int j32_next_inputs(int a, int b, int h, int pb, int qb, int rqP, int rqQ, int (&tp)[4],
                             int (&ts)[4], int (&te)[4]) {
  int dpa, dps, dqa, dqs;
  j32_dest_P(a, dpa, dps);
  j32_dest_Q(a, h, dqa, dqs);
  int m = 0;
  if (b == a) {
    tp[m] = dpa, ts[m] = dps, te[m] = 0, ++m;  // P column: a_pp of P(dpa), or a_qq of Q(0)
    tp[m] = dqa, ts[m] = dqs, te[m] = 3, ++m;  // Q column: a_qq of Q(dqa), or a_pp of P(h - 1)
  }
  if (dps == 0) {
    if (pb == rqP) tp[m] = dpa, ts[m] = 2, te[m] = 0, ++m;
    else if (qb == rqP) tp[m] = dpa, ts[m] = 2, te[m] = 1, ++m;
  }
  if (dqs == 0) {
    if (pb == rqQ) tp[m] = dqa, ts[m] = 2, te[m] = 2, ++m;
    else if (qb == rqQ) tp[m] = dqa, ts[m] = 2, te[m] = 3, ++m;
  }
  return m;
}

}  // namespace qmlgb
