// Split-precision float64 GEMM on tcgen05 tensor cores (Ozaki-style).
//
//   C <- alpha op(A) op(B) + beta C,  op(A) m x K, op(B) K x n, float64 in/out.
//
// Each row i of op(A) is scaled by 2^-e_i (|x| <= 2^e_i) and written as S
// signed digits of beta bits: x 2^-e_i = sum_s a_s 2^(-beta s) with |a_1| <=
// 2^beta, |a_s| <= 2^(beta-1) (s >= 2), every digit an integer that bf16 holds
// exactly; the same for the columns of op(B) with exponents f_j.  Then
//   C_ij = 2^(e_i+f_j) sum_{s+t <= S+1} 2^(-beta(s+t)) (A_s B_t^T)_ij
// (products below the truncation level are dropped).  Every digit product
// A_s B_t^T is an integer matrix, and all pairs of one level L = s + t carry
// the same weight, so they accumulate into one FP32 TMEM accumulator; over a
// K-chunk of 1536 (S <= 8) or 1024 elements the level sum stays below 2^24, so the
// tensor-core accumulation is exact whatever its order or rounding mode.
// Each exact (level, chunk) sum is converted to int32 and added, shifted left
// by shift_L = shift_top - beta (L - 2) bits (right, rounded, when negative),
// into one int64 fixed-point accumulator per output held in registers; the
// total stays below 2^62.  One int64 -> float64 conversion per output; the
// scaling by a power of two is an integer add to the exponent field, and the
// digit slicing reads the float64 bit patterns with integer operations (the
// float64 pipe of this part is narrow).
//
// Schedule.  The levels are taken in groups of four, largest first (6..9,
// then 10..11, then 2..5; see group_at), each level of a group in its own
// 128-column FP32 accumulator (the four use all 512 TMEM columns).  For a
// group, every K step of 16 loads each digit tile the group needs once --
// A_1..A_d and B_1..B_d, d = min(S, last level - 1), 4 KB each -- and runs
// every digit pair of the group's levels on them,
// so a loaded tile serves all the pairs it belongs to (S = 8: 24 tile loads
// per K step for 36 products, where one load per operand and pair would take
// 72).  The tensor core reads a 128 x 128 x 16 product's 8 KB of operands from
// shared memory at its full rate; what bounds the product is delivering the
// tiles from L2, hence the reuse.
//
// Kernel layout: one CTA per 128 x 128 output tile, 384 threads.
//   warp 0   TMA producer (one lane): 128 x 16 bf16 digit tiles, 32-byte
//            swizzle, a ring of stages of up to stage_tiles tiles per operand
//            (one or more K steps), guarded by mbarriers;
//   warp 1   TMEM allocator and MMA issuer (one lane): tcgen05.mma kind::f16
//            M=128 N=128 K=16 into the group's level accumulators; after each
//            exact chunk it commits them to the epilogue and waits until they
//            are read before the next chunk overwrites them;
//   warps 2-3 idle (they complete warpgroup 0 for the register split);
//   warps 4-11 epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (tile rows)
//            and 64 columns (half (w - 4) / 4 of the tile) of each level.
// Every mbarrier wait is bounded (2 s of %globaltimer): on expiry the CTA records
// QML_ETIMEOUT, drains what it issued, frees TMEM and returns.
#include "fixconv.cuh"
#include "oz_order.cuh"
#include "internal.cuh"
#include "ptx.cuh"

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

namespace qmlgb {

namespace {

constexpr int OBM = 128, OBN = 128, OBK = 64;  // output tile; K padding of the digit planes
constexpr int KS = 16;                          // K per MMA instruction and per TMA box
constexpr int kDigitTile = OBM * KS * 2;        // 4 KB: one 128 x 16 bf16 digit tile
constexpr int kGroupLevels = 4;                 // levels per group: 4 x 128 TMEM columns
// Three warpgroups.  Warpgroup 0: warp 0 the TMA producer, warp 1 the TMEM
// allocator and MMA issuer, warps 2-3 idle.  Warpgroups 1 and 2 (warps
// 4-11): kEpiWarps epilogue warps, each one TMEM lane quarter (32 tile rows)
// by kEpiCols columns, so a thread holds kEpiCols int64 accumulators.  The
// block starts at kLaunchRegs registers a thread (12 warps, three on each SM
// sub-partition of 16384 registers: 65536 / 384 rounded down to 8); then
// warpgroup 0 gives registers back (setmaxnreg.dec to kIssueRegs) and the
// epilogue takes them (setmaxnreg.inc to kEpiRegs), so that its 64 int64 sums
// stay in registers.  The split adds up exactly:
// 128 kIssueRegs + 256 kEpiRegs = 384 kLaunchRegs.
constexpr int kEpiWarps = 8, kEpiCols = 128 * 4 / kEpiWarps;
constexpr int kThreads = 128 + 32 * kEpiWarps;
constexpr int kLaunchRegs = 168, kIssueRegs = 56, kEpiRegs = 224;
static_assert(128 * kIssueRegs + 256 * kEpiRegs == kThreads * kLaunchRegs,
              "register split must equal the launch's registers");
static_assert(kThreads * kLaunchRegs <= 65536, "launch registers exceed the SM");
// K elements per exact chunk.  All digit pairs (s, t) of one level L = s + t
// accumulate in the same FP32 accumulator: with beta = 6, |a_1|, |b_1| <= 2^6
// and the other digits <= 2^5, so a level-L sum over c elements is at most
// c 2^10 (n_L + 2) for the n_L <= S pairs of a level L >= 3, and level 2 at
// most c 2^12.  With S <= 8 (n_L <= 8) a chunk of 1536 stays below
// 1536 2^10 10 < 2^24; with S = 9, 10 a chunk of 1024 below 2^10 2^10 12 <
// 2^24: exact either way.
__host__ __device__ constexpr int chunk_elems(int S) { return S <= 8 ? 1536 : 1024; }
// most digits per operand element (beta S <= 62 with beta = 6)
constexpr int kMaxSlices = 10;

// ------------------------------------------------------------ PTX helpers --
// (TMA, tcgen05 and shared-memory descriptor helpers: ptx.cuh)

// instruction descriptor, kind::f16: D f32, A and B bf16, both K-major, N, M
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OBN >> 3) << 17) |
                            ((uint32_t)(OBM >> 4) << 24);

// K-major bf16 tile of 16-element (32-byte) rows with the 32-byte swizzle
// (8-row atoms of 256 B): start address, LBO 16 B (unused: one MMA's K is the
// whole swizzle row), SBO 256 B, descriptor version 1, layout type 6.
__device__ __forceinline__ uint64_t smem_desc_sw32(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(256 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)6 << 61;
  return d;
}

struct OzParams {
  int64_t M, N;            // logical output size
  int Mpad, Npad, nk16;    // padded rows of the digit arrays; K steps of 16
  int S, beta;             // digits, bits per digit
  int stage_tiles;         // digit tiles per operand a ring stage holds
  int nstages;             // ring depth
  int shift_top;           // left shift of level-2 chunk sums in the int64 accumulator
  int tiles_m, tiles_n, lower;
  int band;                // row pairs per band of the pair order (>= 1)
  int ntiles;              // work items (tiles, or tile pairs); the grid takes them round-robin
  double alpha, betac;
  int alpha_pow2, alpha_exp, alpha_neg;  // alpha = (-1)^neg 2^exp when alpha_pow2
  // 0: C is not read (beta = 0); 1: v + C (beta = 1); 2: fma(beta, C, v).  A
  // float64 compare is a float64-pipe instruction (tens of clocks a warp on
  // this part), so the output takes this integer instead of testing beta.
  int beta_mode;
  int prefetch_c;  // fetch each output tile's C into L2 when the tile starts
  double *C;
  int64_t ldc;
  const int *ea, *eb;
  DevStatus *status;
  // failure-path test (tuning key test_wait_timeout): the producer issues no
  // copies and every wait gives up after wait_ns, so each CTA takes its
  // timeout exit; normal calls have wait_ns = kWaitNs and no_loads = 0
  uint64_t wait_ns;
  int no_loads;
};

// acc 2^E as a float64, sign flipped when neg, by integer operations
// (fixconv.cuh); false when the result would leave the normal range, and the
// caller then uses ldexp.
__device__ __forceinline__ bool fixed_to_double(long long acc, int E, bool neg, double &out) {
  uint64_t bits;
  if (!fixed_to_double_bits(acc, E, neg, bits)) return false;
  out = __longlong_as_double((long long)bits);
  return true;
}

// the tile (single form) or tile-row pair (pair form) of a work item
// (oz_order.cuh)
__device__ __forceinline__ void tile_of(const OzParams &p, int bid, int &tm, int &tn) {
  oz_tile_of(p.lower, p.tiles_n, bid, tm, tn);
}
__device__ __forceinline__ void pair_of(const OzParams &p, int idx, int &TM, int &tn) {
  oz_pair_of(p.tiles_m, p.tiles_n, p.lower, p.band, idx, TM, tn);
}
// This CTA's rank in its pair, its first work item and the stride between
// its items (read from special registers where used: held in registers
// across the role loops they pushed the 56-register warpgroup into spills).
template <int CL>
__device__ __forceinline__ int pair_rank() {
  return CL == 2 ? (int)cluster_ctarank() : 0;
}
template <int CL>
__device__ __forceinline__ int item_first() {
  return CL == 2 ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
}
template <int CL>
__device__ __forceinline__ int item_stride() {
  return CL == 2 ? (int)(gridDim.x >> 1) : (int)gridDim.x;
}
// the output tile of this CTA for work item `item` (a tile, or a pair for CL = 2)
template <int CL>
__device__ __forceinline__ void item_tile(const OzParams &p, int item, int rank, int &tm, int &tn) {
  if (CL == 1) {
    tile_of(p, item, tm, tn);
  } else {
    int TM;
    pair_of(p, item, TM, tn);
    tm = 2 * TM + rank;
  }
}

// Level group g: levels lb .. le (at most kGroupLevels), digits 1 .. nd of
// each operand, and the K steps a ring stage holds for it.
struct Group {
  int lb, le, nd, sps;
};
__device__ __forceinline__ Group group_of(const OzParams &p, int S, int g) {
  Group G;
  G.lb = 2 + kGroupLevels * g;
  G.le = min(S + 1, G.lb + kGroupLevels - 1);
  G.nd = min(S, G.le - 1);
  G.sps = max(1, p.stage_tiles / G.nd);
  return G;
}
// The order the groups are taken in: group 1 (levels 6..9, the most digit
// pairs) first, group 0 (levels 2..5) last.  The epilogue writes a finished
// tile out before it reads the next tile's first group, and the MMAs of that
// group cannot start on accumulators still unread; with the largest group
// first they keep the tensor core busy for longer than the output takes.  The
// int64 sums are the same whatever the order.
__device__ __forceinline__ int group_at(int i, int ngroups) {
  if (ngroups == 1) return 0;
  return i == 0 ? 1 : (i == ngroups - 1 ? 0 : i + 1);
}

// Every digit product of levels LB..LE (S digits) for one K step, in
// level-major order: pair (s, t) reads digit tile s - 1 of A and t - 1 of B,
// at descriptor offsets of 256 (4 KB >> 4) per tile from the step's first
// tiles (da, db).  Unrolled at compile time, so the issuing thread spends a
// few instructions per MMA: with loop bounds, flags and descriptors computed
// at run time it could not keep up with the tensor core (about 95 clocks of
// issue per 64-clock MMA).  The first pair of each level writes its
// accumulator when acc0 is 0 (first K step of a chunk), later pairs add.
template <int LB, int LE, int S>
__device__ __forceinline__ void issue_step(uint32_t tbase, uint64_t da, uint64_t db,
                                           uint32_t acc0) {
#pragma unroll
  for (int L = LB; L <= LE; ++L) {
#pragma unroll
    for (int s = (L - S > 1 ? L - S : 1); s <= (L - 1 < S ? L - 1 : S); ++s) {
      const int t = L - s;
      const bool first = (s == (L - S > 1 ? L - S : 1));
      mma_bf16_off(tbase + 128 * (L - LB), da, (uint64_t)(256 * (s - 1)), db,
                   (uint64_t)(256 * (t - 1)), kIdesc, first ? acc0 : 1u);
    }
  }
}

// TMA loads of one stage: nsteps K steps, each one box of ND digit tiles
// (digits 1..ND, 128 rows, 16 elements of K) per operand from a 3-D map over
// the digit planes (K, rows, digit); the box lands as ND consecutive 4 KB tiles.
template <int ND>
__device__ __forceinline__ void load_stage(const CUtensorMap *tmA, const CUtensorMap *tmB,
                                           uint32_t sa, uint32_t sb, uint32_t bar, int k16,
                                           int nsteps, int m0, int n0) {
  for (int j = 0; j < nsteps; ++j) {
    const uint32_t off = (uint32_t)(j * ND) * kDigitTile;
    tma_load_3d(sa + off, tmA, bar, (k16 + j) * KS, m0, 0);
    tma_load_3d(sb + off, tmB, bar, (k16 + j) * KS, n0, 0);
  }
}

// Output of 8 consecutive columns of one row: C[gi + gj ldc] = alpha 2^(e)
// acc + beta C for the live entries (gj < N, and gj <= gi for a lower C).  Not
// inlined: its 8 calls share one copy of the code, which stays in the
// instruction cache (unrolled 64 times, the output code ran once per tile and
// was fetched cold).  The 8 C values are read before any is written, so
// their loads are in flight together; the 8 column exponents f_j come in as
// arguments (the caller has them by warp shuffle), not as loads between the
// stores.
__device__ __noinline__ void store_out8(const OzParams &p, int64_t gi, int64_t gj0, int ebase,
                                        long long a0, long long a1, long long a2, long long a3,
                                        long long a4, long long a5, long long a6, long long a7,
                                        int f0, int f1, int f2, int f3, int f4, int f5, int f6,
                                        int f7) {
  const long long av[8] = {a0, a1, a2, a3, a4, a5, a6, a7};
  const int fv[8] = {f0, f1, f2, f3, f4, f5, f6, f7};
  const int eshift = p.alpha_pow2 ? p.alpha_exp : 0;
  const bool aneg = p.alpha_pow2 && p.alpha_neg;
  const int bmode = p.beta_mode;
  double cv[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int64_t gj = gj0 + u;
    const bool live = gj < p.N && !(p.lower && gi < gj);
    cv[u] = (live && bmode != 0) ? p.C[gi + gj * p.ldc] : 0.0;
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int64_t gj = gj0 + u;
    if (gj >= p.N || (p.lower && gi < gj)) continue;
    const int eb = fv[u];
    double v;
    if (fixed_to_double(av[u], ebase + eb + eshift, aneg, v)) {
      if (!p.alpha_pow2) v *= p.alpha;
    } else {
      v = p.alpha * ldexp((double)av[u], ebase + eb);
    }
    if (bmode == 1) v += cv[u];
    else if (bmode == 2) v = fma(p.betac, cv[u], v);
    p.C[gi + gj * p.ldc] = v;
  }
}

// SC = 8: the default digit count with the unrolled schedule above; SC = 0:
// any S (run-time loops).  Persistent: each CTA takes tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...; the producer runs on into the next tile's
// data and the MMAs of the next tile start as soon as the epilogue has read
// the accumulators, while the epilogue converts and stores the finished tile
// from its registers.
//
// CL = 2: clusters of two CTAs on the tile rows 2 TM, 2 TM + 1 of one tile
// column, which need the same B digit tiles.  Each CTA loads its own A tiles
// and half of the B digits, multicast into both CTAs' shared memory at the
// same offsets (the stage's full barrier in each CTA expects all of its
// bytes), so B leaves L2 once for the two tiles: a quarter less L2 traffic,
// which is what bounds the long-K products.  A stage is free again only when
// both CTAs' MMAs are done with it: the MMA commits arrive on the empty
// barriers of both CTAs (two arrivals a phase).  Cluster barriers order the
// barrier initialisation before any remote arrival and keep both CTAs alive
// until neither can reach the other's shared memory.
template <int SC, int CL>
__global__ void __launch_bounds__(kThreads, 1)
    ozaki_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB,
                      const __grid_constant__ CUtensorMap tmA4,
                      const __grid_constant__ CUtensorMap tmB4,
                      const __grid_constant__ CUtensorMap tmA8,
                      const __grid_constant__ CUtensorMap tmB8,
                      const __grid_constant__ CUtensorMap tmB2, OzParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the swizzled tiles
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int NST = p.nstages;
  const int stage_bytes = 2 * p.stage_tiles * kDigitTile;  // A tiles, then B tiles
  uint64_t *bars = (uint64_t *)(smem + (size_t)NST * stage_bytes);
  // bars: [0,NST) full, [NST,2NST) empty, 2NST acc_full, 2NST+1 acc_empty, 2NST+2 drain
  uint32_t *tmem_holder = (uint32_t *)(bars + 2 * NST + 3);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  DevStatus *st = p.status;
  const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[NST]);
  const uint32_t accf = smem_u32(&bars[2 * NST]), acce = smem_u32(&bars[2 * NST + 1]);
  const uint32_t drain = smem_u32(&bars[2 * NST + 2]);

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, CL);
    }
    mbar_init(accf, 1);
    mbar_init(acce, 32 * kEpiWarps);
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_holder), kGroupLevels * 128);
  tc_fence_before();
  __syncthreads();
  if (CL == 2) cluster_sync_all();  // both CTAs' barriers exist before any remote arrival
  tc_fence_after();
  const uint32_t tbase = *tmem_holder;

  const int S = SC ? SC : p.S;
  const int ngroups = (S + kGroupLevels - 1) / kGroupLevels;  // levels 2 .. S+1
  const int csteps = chunk_elems(S) / KS;  // K steps per exact chunk
  const int nchunks = (p.nk16 + csteps - 1) / csteps;

  if (warp < 4) {
  // warpgroup 0 hands registers to the epilogue warpgroups
  asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kIssueRegs));
  if (warp == 0) {
    // ------------------------------------------------------- TMA producer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int last_phase[4] = {-1, -1, -1, -1};
      bool ok = (*((volatile int *)&st->code) == 0) && !p.no_loads;
      for (int item = item_first<CL>(); item < p.ntiles && ok; item += item_stride<CL>()) {
        int tm, tn;
        item_tile<CL>(p, item, pair_rank<CL>(), tm, tn);
        const int m0 = tm * OBM, n0 = tn * OBN;
        for (int gi = 0; gi < ngroups && ok; ++gi) {
          const int g = group_at(gi, ngroups);
          const Group G = group_of(p, S, g);
          for (int c = 0; c < nchunks && ok; ++c) {
            const int k0 = c * csteps, k1 = min(k0 + csteps, p.nk16);
            for (int ks = k0; ks < k1; ks += G.sps) {
              const int nsteps = min(G.sps, k1 - ks);
              if (!mbar_wait(empty0 + 8 * stage, phase ^ 1, st, p.wait_ns)) { ok = false; break; }
              mbar_expect_tx(full0 + 8 * stage, 2u * G.nd * nsteps * kDigitTile);
              const uint32_t sa = smem_u32(smem + (size_t)stage * stage_bytes);
              const uint32_t sb = sa + p.stage_tiles * kDigitTile;
              const uint32_t fb = full0 + 8 * stage;
              if (CL == 2 && SC == 8) {
                // own A box; B digits [rank h, rank h + h) for both CTAs
                const int h = G.nd >> 1, rank = pair_rank<CL>();
                const CUtensorMap *mA = G.nd == 4 ? &tmA4 : &tmA8;
                const CUtensorMap *mBh = G.nd == 4 ? &tmB2 : &tmB4;
                for (int j = 0; j < nsteps; ++j) {
                  const uint32_t off = (uint32_t)(j * G.nd) * kDigitTile;
                  tma_load_3d(sa + off, mA, fb, (ks + j) * KS, m0, 0);
                  tma_load_3d_mc(sb + off + (uint32_t)(rank * h) * kDigitTile, mBh, fb,
                                 (ks + j) * KS, n0, rank * h, (uint16_t)3);
                }
              } else if (SC == 8 && G.nd == 4) {
                load_stage<4>(&tmA4, &tmB4, sa, sb, fb, ks, nsteps, m0, n0);
              } else if (SC == 8) {
                load_stage<8>(&tmA8, &tmB8, sa, sb, fb, ks, nsteps, m0, n0);
              } else {
                for (int j = 0; j < nsteps; ++j)
                  for (int d = 0; d < G.nd; ++d) {
                    const uint32_t off = (uint32_t)(j * G.nd + d) * kDigitTile;
                    tma_load_2d(sa + off, &tmA, fb, (ks + j) * KS, d * p.Mpad + m0);
                    if (CL == 1)
                      tma_load_2d(sb + off, &tmB, fb, (ks + j) * KS, d * p.Npad + n0);
                    else if ((d & 1) == pair_rank<CL>())  // B digit d from CTA d mod 2, to both
                      tma_load_2d_mc(sb + off, &tmB, fb, (ks + j) * KS, d * p.Npad + n0,
                                     (uint16_t)3);
                  }
              }
              last_phase[stage] = (int)phase;
              if (++stage == NST) { stage = 0; phase ^= 1; }
            }
          }
        }
      }
      if (!ok) {
        // drain: wait (bounded) until the last load issued into each slot has
        // landed, so no copy is still writing shared memory when the CTA exits
        for (int q = 0; q < NST; ++q) {
          if (last_phase[q] < 0) continue;
          mbar_drain_wait(full0 + 8 * q, (uint32_t)last_phase[q]);
        }
      }
    }
  } else if (warp == 1) {
    // -------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      uint32_t q = 0;  // chunk flushes so far
      bool ok = (*((volatile int *)&st->code) == 0);
      for (int item = item_first<CL>(); item < p.ntiles && ok; item += item_stride<CL>()) {
        for (int gi = 0; gi < ngroups && ok; ++gi) {
          const int g = group_at(gi, ngroups);
          const Group G = group_of(p, S, g);
          for (int c = 0; c < nchunks && ok; ++c) {
            // the epilogue must have read the accumulators of the previous chunk
            if (q >= 1 && !mbar_wait(acce, (q - 1) & 1, st, p.wait_ns)) { ok = false; break; }
            tc_fence_after();
            const int k0 = c * csteps, k1 = min(k0 + csteps, p.nk16);
            for (int ks = k0; ks < k1 && ok; ks += G.sps) {
              const int nsteps = min(G.sps, k1 - ks);
              if (!mbar_wait(full0 + 8 * stage, phase, st, p.wait_ns)) { ok = false; break; }
              tc_fence_after();
              const uint32_t sa = smem_u32(smem + (size_t)stage * stage_bytes);
              const uint32_t sb = sa + p.stage_tiles * kDigitTile;
              const uint64_t da0 = smem_desc_sw32(sa), db0 = smem_desc_sw32(sb);
              for (int j = 0; j < nsteps; ++j) {
                const uint32_t acc0 = (ks == k0 && j == 0) ? 0u : 1u;
                if (SC == 8 && g == 0) {
                  issue_step<2, 5, 8>(tbase, da0 + (uint64_t)(256 * 4 * j),
                                      db0 + (uint64_t)(256 * 4 * j), acc0);
                } else if (SC == 8) {
                  issue_step<6, 9, 8>(tbase, da0 + (uint64_t)(256 * 8 * j),
                                      db0 + (uint64_t)(256 * 8 * j), acc0);
                } else {
                  for (int L = G.lb; L <= G.le; ++L) {
                    const int s0 = max(1, L - S);
                    for (int s = s0; s <= min(S, L - 1); ++s) {
                      const int t = L - s;
                      mma_bf16(tbase + 128 * (L - G.lb),
                               da0 + (uint64_t)(256 * (j * G.nd + s - 1)),
                               db0 + (uint64_t)(256 * (j * G.nd + t - 1)), kIdesc,
                               s == s0 ? acc0 : 1u);
                    }
                  }
                }
              }
              // frees the smem slot when these MMAs finish (in both CTAs of a pair)
              if (CL == 2)
                mma_commit_mc(empty0 + 8 * stage, (uint16_t)3);
              else
                mma_commit(empty0 + 8 * stage);
              if (++stage == NST) { stage = 0; phase ^= 1; }
            }
            if (!ok) break;
            mma_commit(accf);  // the group's (level, chunk) sums ready for the epilogue
            ++q;
          }
        }
      }
      // wait for every MMA this thread issued before TMEM is released
      mma_commit(drain);
      mbar_drain_wait(drain, 0);
    }
  }
  } else {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kEpiRegs));
    // ---------------------------------------------------------- epilogue
    const int quad = warp & 3;            // TMEM lane quarter this warp may access
    const int half = (warp - 4) >> 2;     // which kEpiCols columns of the tile
    const int row = quad * 32 + lane;
    const uint32_t lane_base = tbase + ((uint32_t)(quad * 32) << 16) + kEpiCols * half;
    uint32_t q = 0;
    bool ok = true;
    for (int item = item_first<CL>(); item < p.ntiles && ok; item += item_stride<CL>()) {
      int tm, tn;
      item_tile<CL>(p, item, pair_rank<CL>(), tm, tn);
      const int m0 = tm * OBM, n0 = tn * OBN;
      // the column exponents f_j of this warp's kEpiCols columns, two a lane
      const int64_t gjl = n0 + kEpiCols * half + lane;
      const int f_lo = gjl < p.N ? p.eb[gjl] : 0;
      const int f_hi = gjl + 32 < p.N ? p.eb[gjl + 32] : 0;
      // beta C is read only when the tile is written out, after all of its
      // MMAs; fetch this thread's C entries into L2 now, so that those reads
      // wait on L2 rather than on DRAM
      if (p.prefetch_c && m0 + row < p.M) {
        const int64_t pi = m0 + row;
        for (int j = 0; j < kEpiCols; ++j) {
          const int64_t pj = n0 + kEpiCols * half + j;
          if (pj >= p.N || (p.lower && pi < pj)) break;
          asm volatile("prefetch.global.L2 [%0];" ::"l"(__cvta_generic_to_global(p.C + pi + pj * p.ldc)));
        }
      }
      long long acc[kEpiCols];
#pragma unroll
      for (int j = 0; j < kEpiCols; ++j) acc[j] = 0;
      for (int gi = 0; gi < ngroups && ok; ++gi) {
        const Group G = group_of(p, S, group_at(gi, ngroups));
        for (int c = 0; c < nchunks; ++c) {
          int okw = 1;
          if (lane == 0) okw = mbar_wait(accf, q & 1, st, p.wait_ns) ? 1 : 0;
          okw = __shfl_sync(0xffffffffu, okw, 0);
          __syncwarp();
          if (!okw) { ok = false; break; }
          tc_fence_after();
          for (int L = G.lb; L <= G.le; ++L) {
            const int sh = p.shift_top - p.beta * (L - 2);
            const uint32_t lbase = lane_base + 128 * (L - G.lb);
#pragma unroll
            for (int cb = 0; cb < kEpiCols / 16; ++cb) {
              uint32_t a[16];
              tmem_ld16(lbase + 16 * cb, a);
              if (sh >= 0) {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                  acc[16 * cb + j] += (long long)__float2int_rn(__uint_as_float(a[j])) << sh;
              } else {
                const int r = -sh;
                const long long rnd = 1LL << (r - 1);
#pragma unroll
                for (int j = 0; j < 16; ++j)
                  acc[16 * cb + j] += ((long long)__float2int_rn(__uint_as_float(a[j])) + rnd) >> r;
              }
            }
          }
          tc_fence_before();
          mbar_arrive(acce);  // the accumulators may be overwritten from here on
          ++q;
        }
      }
      if (!ok) break;
      // output: alpha 2^(e_i + f_j - 2 beta - shift_top) acc + beta C, while
      // the MMAs of the next tile already run
      // (every lane takes part in the shuffles; rows past M store nothing)
      const int64_t gi = m0 + row;
      const bool live_row = gi < p.M;
      const int ebase = live_row ? p.ea[gi] - 2 * p.beta - p.shift_top : 0;
      const int64_t gj0 = n0 + kEpiCols * half;
#pragma unroll
      for (int g = 0; g < kEpiCols / 8; ++g) {
        int f[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int cix = 8 * g + u;
          f[u] = __shfl_sync(0xffffffffu, cix < 32 ? f_lo : f_hi, cix & 31);
        }
        if (live_row)
          store_out8(p, gi, gj0 + 8 * g, ebase, acc[8 * g], acc[8 * g + 1], acc[8 * g + 2],
                     acc[8 * g + 3], acc[8 * g + 4], acc[8 * g + 5], acc[8 * g + 6],
                     acc[8 * g + 7], f[0], f[1], f[2], f[3], f[4], f[5], f[6], f[7]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  // neither CTA of a pair leaves while the other may still write its shared
  // memory or arrive on its barriers
  if (CL == 2) cluster_sync_all();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tbase, kGroupLevels * 128);
}

// ------------------------------------------------------------- digits ----
// Row maxima of |x| as float64 bit patterns with the sign cleared (for
// non-negative float64 values the integer order is the numeric order).
// Rows strided, k contiguous: one warp per row, lanes stride over k.
__global__ void rowmax_kcontig_kernel(const double *X, int64_t R, int64_t K, int64_t sr,
                                      unsigned long long *bits, int Rpad) {
  const int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= Rpad) return;
  unsigned long long mb = 0;
  if (r < R)
    for (int64_t k = lane; k < K; k += 32) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(X[r * sr + k]) &
                                   0x7FFFFFFFFFFFFFFFull;
      mb = b > mb ? b : mb;
    }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, mb, o);
    mb = t > mb ? t : mb;
  }
  if (lane == 0) bits[r] = mb;
}

// Rows contiguous (column-major operand): block (x, y) covers 32 rows and 256
// values of k; a warp reads 32 consecutive rows at one k (coalesced), the 8
// warps take every 8th k, and the block's maximum per row joins the others
// with atomicMax (bits zeroed beforehand).
__global__ void rowmax_rcontig_kernel(const double *X, int64_t R, int64_t K, int64_t sk,
                                      unsigned long long *bits) {
  __shared__ unsigned long long part[8][32];
  const int rl = threadIdx.x & 31, kg = threadIdx.x >> 5;
  const int64_t r = (int64_t)blockIdx.x * 32 + rl;
  const int64_t kc0 = (int64_t)blockIdx.y * 256, kc1 = (kc0 + 256 < K) ? kc0 + 256 : K;
  unsigned long long mb = 0;
  if (r < R)
    for (int64_t k = kc0 + kg; k < kc1; k += 8) {
      const unsigned long long b = (unsigned long long)__double_as_longlong(X[r + k * sk]) &
                                   0x7FFFFFFFFFFFFFFFull;
      mb = b > mb ? b : mb;
    }
  part[kg][rl] = mb;
  __syncthreads();
  if (kg == 0 && r < R) {
    for (int q = 1; q < 8; ++q) mb = part[q][rl] > mb ? part[q][rl] : mb;
    if (mb) atomicMax(&bits[r], mb);
  }
}

// exponent e of a row maximum m (frexp convention: m < 2^e, 0 for m = 0)
__device__ __forceinline__ int exponent_of(unsigned long long m) {
  if (m == 0) return 0;
  const int E = (int)(m >> 52);
  if (E == 0) {  // subnormal maximum
    int ex = 0;
    frexp(__longlong_as_double((long long)m), &ex);
    return ex;
  }
  return E - 1022;  // m = 1.f 2^(E-1023) = (1.f / 2) 2^(E-1022)
}

// round(x 2^sh) to the nearest integer, ties to even (as __double2ll_rn of
// ldexp(x, sh) would), by integer operations on the float64 bit pattern; the
// caller guarantees |x| 2^sh < 2^62
__device__ __forceinline__ long long scaled_round(double x, int sh) {
  const long long bits = __double_as_longlong(x);
  const int bexp = (int)((bits >> 52) & 0x7FF);
  unsigned long long m = (unsigned long long)(bits & ((1ll << 52) - 1));
  if (bexp == 0 && m == 0) return 0;
  if (bexp != 0) m |= 1ull << 52;
  // x = m 2^(e2), e2 = max(bexp, 1) - 1075
  const int t = (bexp != 0 ? bexp : 1) - 1075 + sh;
  unsigned long long q;
  if (t >= 0) {
    q = m << t;
  } else if (t < -63) {
    q = 0;
  } else {
    const int d = -t;
    q = m >> d;
    const unsigned long long rem = m & ((1ull << d) - 1ull), half = 1ull << (d - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
  }
  return bits < 0 ? -(long long)q : (long long)q;
}

// The S digits of two adjacent elements x0, x1 (k, k + 1) of row r with row
// exponent er into the digit planes D[s][r][k] (rows Rpad, Kpad per row):
// F = round(x 2^(beta S - er)) as an integer, then signed digits from the
// bottom, each in [-2^(beta-1), 2^(beta-1)), the top one in [-2^beta, 2^beta].
// Digit i (from the bottom, i < S - 1) by the signed base-2^beta recurrence
// d = ((F + 2^(beta-1)) mod 2^beta) - 2^(beta-1), F <- (F - d) / 2^beta, run
// on chunks of up to 4 digits in 32-bit arithmetic (the chunk's carry joins
// the rest of F at its end); digit S - 1 is what remains.
__device__ __forceinline__ void slice_pair(double x0, double x1, int er, int S, int beta,
                                           __nv_bfloat16 *D, int Rpad, int Kpad, int64_t r,
                                           int64_t k) {
  long long Fh[2];
  int lo[2] = {0, 0};
  Fh[0] = scaled_round(x0, beta * S - er);
  Fh[1] = scaled_round(x1, beta * S - er);
  const int half = 1 << (beta - 1), mask = (1 << beta) - 1;
#pragma unroll
  for (int i = 0; i < kMaxSlices; ++i) {
    if (i >= S) break;
    int d[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (i < S - 1) {
        if ((i & 3) == 0) {
          const int nd = (S - 1 - i) < 4 ? (S - 1 - i) : 4;
          const int nb = beta * nd;
          lo[h] = (int)(Fh[h] & ((1LL << nb) - 1));
          Fh[h] >>= nb;
        }
        d[h] = ((lo[h] + half) & mask) - half;
        lo[h] = (lo[h] - d[h]) >> beta;
        if ((i & 3) == 3 || i == S - 2) Fh[h] += lo[h];
      } else {
        d[h] = (int)Fh[h];
      }
    }
    // digit i from the bottom is digit s = S - i of the expansion
    __nv_bfloat162 v = __floats2bfloat162_rn((float)d[0], (float)d[1]);
    *(__nv_bfloat162 *)(D + ((int64_t)(S - i - 1) * Rpad + r) * Kpad + k) = v;
  }
}

// One 32 x 64 tile of X (rows r0.., k0..; element (r, k) at X[r sr + k sk],
// zero outside R x K) into shared memory, read coalesced along whichever of
// r and k is contiguous.
__device__ __forceinline__ void load_tile32x64(double (*tile)[65], const double *X, int64_t R,
                                               int64_t K, int64_t sr, int64_t sk, int64_t r0,
                                               int64_t k0) {
  const int tid = threadIdx.x;  // 256 threads
  if (sk == 1) {
    // k contiguous: 64 consecutive k per row
    for (int t = tid; t < 32 * 64; t += 256) {
      const int rr = t / 64, kk = t % 64;
      const int64_t r = r0 + rr, k = k0 + kk;
      tile[rr][kk] = (r < R && k < K) ? X[r * sr + k] : 0.0;
    }
  } else {
    // r contiguous: 32 consecutive r per k
    for (int t = tid; t < 32 * 64; t += 256) {
      const int rr = t % 32, kk = t / 32;
      const int64_t r = r0 + rr, k = k0 + kk;
      tile[rr][kk] = (r < R && k < K) ? X[r + k * sk] : 0.0;
    }
  }
}

// digits of one logical matrix X (R x K) into D[s][r][k] (bf16, rows Rpad,
// K-contiguous rows of Kpad), from row maxima already in bits: one 32 x 64
// tile per block via shared memory, so both the read and the K-contiguous
// write coalesce.
__global__ void slice_kernel(const double *X, int64_t R, int64_t K, int64_t sr, int64_t sk,
                             const unsigned long long *bits, int *e, int S, int beta,
                             __nv_bfloat16 *D, int Rpad, int Kpad) {
  __shared__ double tile[32][65];
  const int64_t r0 = (int64_t)blockIdx.y * 32, k0 = (int64_t)blockIdx.x * 64;
  load_tile32x64(tile, X, R, K, sr, sk, r0, k0);
  __syncthreads();
  // each thread: one row rq, two adjacent k (kp, kp + 1)
  const int tid = threadIdx.x, rr = tid / 32, kp = (tid % 32) * 2;
  for (int rq = rr; rq < 32; rq += 8) {
    const int64_t r = r0 + rq;
    if (r >= Rpad) continue;
    const int er = (r < R) ? exponent_of(bits[r]) : 0;
    if (blockIdx.x == 0 && kp == 0) e[r] = er;
    slice_pair(tile[rq][kp], tile[rq][kp + 1], er, S, beta, D, Rpad, Kpad, r, k0 + kp);
  }
}

// ------------------------------------------------------- tensor maps -----
// digit planes (rows x kpad bf16): 128 x 16 boxes, 32-byte swizzle
bool make_map(CUtensorMap *map, void *base, int64_t rows, int64_t kpad) {
  return make_map_bf16(map, base, kpad, rows, kpad * 2, KS, OBM, 32);
}

int64_t rup(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace

// ------------------------------------------------ shared tensor-map builder --
namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}
}  // namespace

bool make_map_bf16(CUtensorMap *map, const void *base, int64_t inner, int64_t rows,
                   int64_t row_bytes, int box_inner, int box_rows, int swizzle_bytes) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  CUtensorMapSwizzle sw = CU_TENSOR_MAP_SWIZZLE_128B;
  if (swizzle_bytes == 64) sw = CU_TENSOR_MAP_SWIZZLE_64B;
  else if (swizzle_bytes == 32) sw = CU_TENSOR_MAP_SWIZZLE_32B;
  else if (swizzle_bytes != 128) return false;
  cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
  cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides,
             box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

namespace {
// the digit planes as a 3-D tensor (K, rows, digit): boxes of `depth` digits x
// 128 rows x 16 elements of K, 32-byte swizzle
bool make_map3(CUtensorMap *map, void *base, int64_t rpad, int64_t kpad, int S, int depth) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[3] = {(cuuint64_t)kpad, (cuuint64_t)rpad, (cuuint64_t)S};
  cuuint64_t strides[2] = {(cuuint64_t)(kpad * 2), (cuuint64_t)(rpad * kpad * 2)};
  cuuint32_t box[3] = {(cuuint32_t)KS, (cuuint32_t)OBM, (cuuint32_t)depth};
  cuuint32_t estr[3] = {1, 1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

void ozaki_choose(int64_t K, int nslices, int &S, int &beta) {
  // beta: digit bits (exact chunk 2^(24 - 2 beta) elements); S digits cover
  // about 48 bits unless the caller asks for another count
  beta = 6;
  (void)K;
  S = nslices > 0 ? nslices : 8;
  if (S * beta > 62) S = 62 / beta;
}

size_t ozaki_workspace_bytes(int64_t M, int64_t N, int64_t K, int nslices, bool shared_operand) {
  int S, beta;
  ozaki_choose(K, nslices, S, beta);
  const int64_t Mpad = rup(M, OBM), Npad = rup(N, OBN), Kpad = rup(K, OBK);
  size_t b = rup((size_t)S * Mpad * Kpad * 2, 1024) + rup(12 * (size_t)Mpad, 1024);
  if (!shared_operand) b += rup((size_t)S * Npad * Kpad * 2, 1024) + rup(12 * (size_t)Npad, 1024);
  return b;
}

// row maxima of one operand (element (r, k) at X[r sr + k sk], one of the
// strides 1) into bits[0 .. Rpad), padding rows 0
void launch_rowmax(const double *X, int64_t R, int64_t K, int64_t sr, int64_t sk,
                   unsigned long long *bits, int64_t Rpad, cudaStream_t st) {
  if (sr == 1) {
    cudaMemsetAsync(bits, 0, (size_t)Rpad * sizeof(unsigned long long), st);
    dim3 g((unsigned)((Rpad + 31) / 32), (unsigned)((K + 255) / 256));
    rowmax_rcontig_kernel<<<g, 256, 0, st>>>(X, R, K, sk, bits);
  } else {
    rowmax_kcontig_kernel<<<(unsigned)((Rpad + 7) / 8), 256, 0, st>>>(X, R, K, sr, bits,
                                                                      (int)Rpad);
  }
  count_launch();
}

// ring stages: stage_tiles digit tiles per operand (all digits of one K step
// for the widest group; several K steps for narrower groups)
__host__ __device__ constexpr size_t oz_smem_c(int stage_tiles, int nstages) {
  return 1024 + (size_t)nstages * 2 * stage_tiles * kDigitTile + (2 * nstages + 3) * 8 + 16;
}
// the largest configuration: S = 8, three stages of eight digit tiles per operand
constexpr int kMaxSmem = (int)oz_smem_c(8, 3);
static_assert(oz_smem_c(8, 3) <= 232448, "split kernel exceeds 227 KB of shared memory");
static_assert(oz_smem_c(10, 2) <= oz_smem_c(8, 3), "S = 10 layout must fit the attribute");

size_t oz_smem(int stage_tiles, int nstages) { return oz_smem_c(stage_tiles, nstages); }

// Launch attributes of the four instantiations, set once: the shared-memory
// size, and the check that the warpgroups' register split (setmaxnreg) adds
// up to exactly kLaunchRegs a thread (a build that launches with any other
// count is refused rather than run: an increase that cannot be met never
// returns).  Also the most clusters of two that can be resident at once.
template <int SC, int CL>
cudaError_t oz_prepare(int &max_items) {
  cudaError_t e = cudaFuncSetAttribute(ozaki_gemm_kernel<SC, CL>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxSmem);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, ozaki_gemm_kernel<SC, CL>);
  if (e != cudaSuccess) return e;
  if (fa.numRegs != kLaunchRegs) return cudaErrorInvalidConfiguration;
  int dev = 0, nsm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
    return e;
  if (CL == 1) {
    max_items = nsm;
    return cudaSuccess;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * (unsigned)nsm);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = kMaxSmem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int ncl = 0;
  e = cudaOccupancyMaxActiveClusters(&ncl, ozaki_gemm_kernel<SC, CL>, &cfg);
  if (e != cudaSuccess) return e;
  max_items = ncl > 0 ? ncl : 1;
  return cudaSuccess;
}

template <int SC, int CL>
cudaError_t launch_oz_t(int nitems, int reserve_sms, const CUtensorMap &mA, const CUtensorMap &mB,
                        const CUtensorMap *m3, const OzParams &p, size_t smem, cudaStream_t st) {
  static int max_items = 0;
  static cudaError_t prep = cudaErrorNotReady;
  static std::once_flag once;
  std::call_once(once, [] { prep = oz_prepare<SC, CL>(max_items); });
  if (prep != cudaSuccess) return prep;
  // persistent: one CTA per SM (one fits: 512 TMEM columns, ~197 KB of
  // shared memory), the CTAs (or pairs) taking every grid-th work item;
  // reserve_sms SMs (rounded up to whole pairs) stay free for other streams
  int cap = max_items - (reserve_sms + CL - 1) / CL;
  if (cap < 1) cap = 1;
  const int items = nitems < cap ? nitems : cap;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(CL * items));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const CUtensorMap &a4 = SC == 8 ? m3[0] : mA, &b4 = SC == 8 ? m3[1] : mB;
  const CUtensorMap &a8 = SC == 8 ? m3[2] : mA, &b8 = SC == 8 ? m3[3] : mB;
  const CUtensorMap &b2 = SC == 8 ? m3[4] : mB;
  cudaError_t e = cudaLaunchKernelEx(&cfg, ozaki_gemm_kernel<SC, CL>, mA, mB, a4, b4, a8, b8, b2, p);
  count_launch();
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_oz(int nitems, bool pairs, int reserve_sms, const CUtensorMap &mA,
                      const CUtensorMap &mB, const CUtensorMap *m3, const OzParams &p,
                      cudaStream_t st) {
  const size_t smem = oz_smem(p.stage_tiles, p.nstages);
  if (smem > (size_t)kMaxSmem) return cudaErrorInvalidValue;
  const int rsv = reserve_sms > 0 ? reserve_sms : 0;
  if (p.S == 8)
    return pairs ? launch_oz_t<8, 2>(nitems, rsv, mA, mB, m3, p, smem, st)
                 : launch_oz_t<8, 1>(nitems, rsv, mA, mB, m3, p, smem, st);
  return pairs ? launch_oz_t<0, 2>(nitems, rsv, mA, mB, m3, p, smem, st)
               : launch_oz_t<0, 1>(nitems, rsv, mA, mB, m3, p, smem, st);
}

cudaError_t ozaki_gemm(int ta, int tb, int64_t M, int64_t N, int64_t K, double alpha,
                       const double *A, int64_t lda, const double *B, int64_t ldb, double beta_c,
                       double *C, int64_t ldc, int lower, int nslices, void *work,
                       DevStatus *status, cudaStream_t st, int reserve_sms) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  int S, beta;
  ozaki_choose(K, nslices, S, beta);
  const int64_t Mpad = rup(M, OBM), Npad = rup(N, OBN), Kpad = rup(K, OBK);
  // op(A) and op(B)^T are the same logical matrix when A == B and exactly one
  // of them is transposed (X^T X, G G^T): slice it once
  const bool shared = (A == B && lda == ldb && ta != tb && M == N);
  unsigned char *w = (unsigned char *)work;
  __nv_bfloat16 *DA = (__nv_bfloat16 *)w;
  w += rup((size_t)S * Mpad * Kpad * 2, 1024);
  int *ea = (int *)w;
  unsigned long long *ma = (unsigned long long *)(w + 4 * (size_t)Mpad);  // Mpad % 128 == 0
  w += rup(12 * (size_t)Mpad, 1024);
  __nv_bfloat16 *DB = DA;
  int *eb = ea;
  unsigned long long *mb = ma;
  if (!shared) {
    DB = (__nv_bfloat16 *)w;
    w += rup((size_t)S * Npad * Kpad * 2, 1024);
    eb = (int *)w;
    mb = (unsigned long long *)(w + 4 * (size_t)Npad);
  }
  // op(A)[i,k] = A[i + k lda] (ta = 0) or A[k + i lda]
  const int64_t asr = ta ? lda : 1, ask = ta ? 1 : lda;
  // op(B) column j, entry k: B[k + j ldb] (tb = 0) or B[j + k ldb]
  const int64_t bsr = tb ? 1 : ldb, bsk = tb ? ldb : 1;
  {
    launch_rowmax(A, M, K, asr, ask, ma, Mpad, st);
    dim3 gs((unsigned)(Kpad / 64), (unsigned)(Mpad / 32));
    slice_kernel<<<gs, 256, 0, st>>>(A, M, K, asr, ask, ma, ea, S, beta, DA, (int)Mpad, (int)Kpad);
    count_launch();
    if (!shared) {
      launch_rowmax(B, N, K, bsr, bsk, mb, Npad, st);
      dim3 gb((unsigned)(Kpad / 64), (unsigned)(Npad / 32));
      slice_kernel<<<gb, 256, 0, st>>>(B, N, K, bsr, bsk, mb, eb, S, beta, DB, (int)Npad,
                                       (int)Kpad);
      count_launch();
    }
  }
  CUtensorMap mA, mB, m3[5];
  if (!make_map(&mA, DA, (int64_t)S * Mpad, Kpad) || !make_map(&mB, DB, (int64_t)S * Npad, Kpad))
    return cudaErrorInvalidValue;
  if (S == 8 && (!make_map3(&m3[0], DA, Mpad, Kpad, S, 4) || !make_map3(&m3[1], DB, Npad, Kpad, S, 4) ||
                 !make_map3(&m3[2], DA, Mpad, Kpad, S, 8) || !make_map3(&m3[3], DB, Npad, Kpad, S, 8) ||
                 !make_map3(&m3[4], DB, Npad, Kpad, S, 2)))
    return cudaErrorInvalidValue;
  OzParams p;
  p.M = M;
  p.N = N;
  p.Mpad = (int)Mpad;
  p.Npad = (int)Npad;
  p.nk16 = (int)(Kpad / KS);
  p.S = S;
  p.beta = beta;
  // a stage holds every digit of one K step for the widest group (8 tiles per
  // operand for S <= 8: 64 KB, three stages); S = 9, 10 take S tiles, two stages
  p.stage_tiles = S > 8 ? S : 8;
  p.nstages = S > 8 ? 2 : (tune_get("ozaki_stages", 3) == 2 ? 2 : 3);
  {
    // level-2 chunk sums are below 2^(2 beta) c <= 2^22.6 (c = 1536 elements),
    // level L >= 3 sums below c 2^10 (L + 1) (a shift of beta (L - 2) bits
    // further down): with nchunks <= 2^lg chunks the int64 total stays below
    // 2^(shift_top + 22.6 + lg) x 1.02 <= 2^61.7
    const int csteps = chunk_elems(S) / KS;
    const int nchunks = (p.nk16 + csteps - 1) / csteps;
    int lg = 0;
    while ((1 << lg) < nchunks) ++lg;
    p.shift_top = 39 - lg;
  }
  p.tiles_n = (int)(Npad / OBN);
  p.lower = lower;
  p.alpha = alpha;
  p.betac = beta_c;
  p.beta_mode = beta_c == 0.0 ? 0 : (beta_c == 1.0 ? 1 : 2);
  p.prefetch_c = (p.beta_mode != 0 && tune_get("ozaki_prefetch_c", 1) != 0) ? 1 : 0;
  {
    int ax = 0;
    const double fr = frexp(alpha, &ax);  // alpha = fr 2^ax, |fr| in [0.5, 1)
    p.alpha_pow2 = (fr == 0.5 || fr == -0.5) ? 1 : 0;
    p.alpha_exp = ax - 1;
    p.alpha_neg = alpha < 0.0 ? 1 : 0;
  }
  p.C = C;
  p.ldc = ldc;
  p.ea = ea;
  p.eb = eb;
  p.status = status;
  p.no_loads = tune_get("test_wait_timeout", 0) != 0 ? 1 : 0;
  p.wait_ns = p.no_loads ? 1000000ull : kWaitNs;  // 1 ms in the failure-path test
  const int tiles_m = (int)(Mpad / OBM);
  p.tiles_m = tiles_m;
  {
    const int64_t b = tune_get("ozaki_band", 6);
    p.band = b < 1 ? 1 : (b > 4096 ? 4096 : (int)b);
  }
  // clusters of two on tile-row pairs (B shared through multicast) unless
  // switched off or the output has a single tile row
  const bool pairs = tune_get("ozaki_pairs", 1) != 0 && tiles_m >= 2;
  p.ntiles = oz_item_count(tiles_m, p.tiles_n, lower ? 1 : 0, pairs ? 1 : 0);
  return launch_oz(p.ntiles, pairs, reserve_sms, mA, mB, m3, p, st);
}

}  // namespace qmlgb
