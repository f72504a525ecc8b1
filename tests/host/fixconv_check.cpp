// Host check of csrc/fixconv.cuh: fixed_to_double_bits(acc, E, neg) against
// the C++ conversion (double)acc scaled by ldexp, bit for bit, on edge cases
// and on random int64 values of every magnitude.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include FIXCONV_HEADER

static uint64_t bits_of(double x) {
  uint64_t b;
  std::memcpy(&b, &x, 8);
  return b;
}

static int check(int64_t acc, int E, bool neg) {
  uint64_t got = 0;
  const bool ok = qmlgb::fixed_to_double_bits(acc, E, neg, got);
  double ref = std::ldexp((double)acc, E);  // (double) rounds to nearest even
  if (neg) ref = -ref;
  const uint64_t rb = bits_of(ref);
  const int rexp = (int)((rb >> 52) & 0x7FF);
  const bool ref_normal = (acc == 0) || (rexp > 0 && rexp < 2047);
  if (ok != ref_normal) {
    std::printf("range mismatch acc=%lld E=%d neg=%d\n", (long long)acc, E, (int)neg);
    return 1;
  }
  if (ok && got != rb) {
    std::printf("bits mismatch acc=%lld E=%d neg=%d got=%016llx ref=%016llx\n", (long long)acc, E,
                (int)neg, (unsigned long long)got, (unsigned long long)rb);
    return 1;
  }
  return 0;
}

int main() {
  int bad = 0;
  const int64_t edges[] = {0, 1, -1, 2, 3, (1LL << 53) - 1, 1LL << 53, (1LL << 53) + 1,
                           (1LL << 53) + 2, (1LL << 53) + 3, (1LL << 54) + 2, (1LL << 54) + 6,
                           (1LL << 62), INT64_MAX, INT64_MIN, INT64_MIN + 1, -(1LL << 53) - 1};
  for (int64_t a : edges)
    for (int E : {-1100, -1074, -100, -40, 0, 7, 900, 1000})
      for (bool neg : {false, true}) bad += check(a, E, neg);
  std::mt19937_64 g(12345);
  for (int i = 0; i < 2000000 && bad < 10; ++i) {
    const int sh = (int)(g() % 64);
    int64_t a = (int64_t)(g() >> sh);
    if (g() & 1) a = -a;
    const int E = (int)(g() % 200) - 120;
    bad += check(a, E, (g() & 1) != 0);
  }
  // ties: values whose lowest bits fall exactly half way
  for (int k = 54; k < 63 && bad < 10; ++k)
    for (int j = 0; j < 1000; ++j) {
      const int64_t base = (int64_t)((g() >> (64 - k)) | (1ULL << (k - 1)));
      const int64_t tie = (base & ~((1LL << (k - 53)) - 1)) | (1LL << (k - 54));
      bad += check(tie, 0, false) + check(-tie, 3, true);
    }
  std::printf("%s\n", bad ? "FAIL" : "OK");
  return bad ? 1 : 0;
}
