// Host check of the float-float helpers of csrc/dfloat.cuh.  The test driver
// pastes the header's body (between its namespace braces) into DFLOAT_BODY;
// the CUDA intrinsics it uses are mapped here to IEEE float32 operations in
// round-to-nearest (compiled with -ffp-contract=off), which is what the
// device intrinsics compute.  Prints the worst relative errors and exits
// nonzero when a bound is broken.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#define __device__
#define __host__
#define __forceinline__ inline
static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fsub_rn(float a, float b) { return a - b; }
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fmaf_rn(float a, float b, float c) { return std::fma(a, b, c); }
static inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
static inline int __double2hiint(double x) { uint64_t u; std::memcpy(&u, &x, 8); return (int)(u >> 32); }
static inline int __double2loint(double x) { uint64_t u; std::memcpy(&u, &x, 8); return (int)(uint32_t)u; }
static inline double __hiloint2double(int h, int l) {
  const uint64_t u = ((uint64_t)(uint32_t)h << 32) | (uint32_t)l;
  double x; std::memcpy(&x, &u, 8); return x;
}
static inline float __int_as_float(int i) { float f; std::memcpy(&f, &i, 4); return f; }
static inline int __float_as_int(float f) { int i; std::memcpy(&i, &f, 4); return i; }
static inline float __uint2float_rn(unsigned u) { return (float)u; }

namespace qmlgb {
#include DFLOAT_BODY
}
using namespace qmlgb;

static long double val(dfl v) { return (long double)v.h + (long double)v.l; }

int main() {
  std::mt19937_64 g(20261203);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  double conv = 0, back = 0, mul = 0, fms = 0, rs = 0, norm = 0;
  for (int it = 0; it < 200000; ++it) {
    const int s = (int)(g() % 61) - 30;
    const double x = U(g) * std::ldexp(1.0, (int)(g() % 81) - 40);
    if (x == 0.0) continue;
    const dfl v = df_from_double(x, s);
    conv = std::fmax(conv, (double)std::fabs((val(v) * std::ldexp(1.0L, s) - x) / x));
    back = std::fmax(back, std::fabs((df_to_double(v, s) - x) / x));
    // canonical form: |l| <= ulp(h) / 2
    norm = std::fmax(norm, (double)(std::fabs(v.l) / std::ldexp(1.0f, std::ilogb(v.h) - 24)));
    const dfl a = df_from_double(U(g), 0), y = df_from_double(U(g), 0), z = df_from_double(U(g), 0);
    const long double A = val(a), Y = val(y), Z = val(z);
    mul = std::fmax(mul, (double)std::fabs((val(df_mul(y, z)) - Y * Z) / (Y * Z)));
    fms = std::fmax(fms, (double)(std::fabs(val(df_fms(a, y, z)) - (A - Y * Z)) /
                                  (std::fabs(A) + std::fabs(Y * Z))));
    const dfl d = df_from_double(1.0 + 3.0 * std::fabs(U(g)), 0);
    rs = std::fmax(rs, (double)std::fabs(val(df_rsqrt(d)) * std::sqrt(val(d)) - 1.0L));
  }
  std::printf("conv %.3g back %.3g norm %.3g mul %.3g fms %.3g rsqrt %.3g\n", conv, back, norm, mul,
              fms, rs);
  int bad = 0;
  bad |= !(conv <= 0x1p-47);   // truncated 24 + rounded 24 bits, renormalised
  bad |= !(back <= 0x1p-47);   // one float64 rounding on top
  bad |= !(norm <= 1.0);
  bad |= !(mul <= 0x1p-45);
  bad |= !(fms <= 0x1p-45);
  bad |= !(rs <= 0x1p-45);
  // special values
  const dfl zero = df_from_double(0.0, 5), neg = df_from_double(-1.5, 1);
  bad |= !(zero.h == 0.0f && zero.l == 0.0f);
  bad |= !(neg.h == -0.75f && neg.l == 0.0f && df_to_double(neg, 1) == -1.5);
  bad |= !std::isnan(df_from_double(NAN, 0).h);
  bad |= !std::isnan(df_from_double(INFINITY, 0).h);
  bad |= !(df_from_double(std::ldexp(1.0, -200), 0).h == 0.0f);  // below 2^-126: 0
  bad |= !(packed_off(0, 64) == 0 && packed_off(1, 64) == 64 && packed_off(63, 64) == 2079 &&
           packed_off(64, 64) == 2080);
  std::printf(bad ? "FAIL\n" : "ok\n");
  return bad;
}
