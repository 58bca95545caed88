// Tensor-core forms of the aligned contraction (Alg. 2, contraction step) on
// sm_103a: TMA -> shared memory -> tcgen05.mma with accumulators in TMEM ->
// tcgen05.ld epilogue that writes W's standard reduced form directly (the
// output step of Alg. 2 fused into the epilogue).
//
// Split-BF16 form (Ozaki-style; the paper has no mixed-precision path).
//   Operands arrive as S BF16 slices, slice i holding balanced digits
//   a_i * 2^(-8i), |a_i| <= 128, plus one binary exponent per aligned row.
//   Slice-pair products a_i b_j (|.| <= 2^14) are summed on the tensor core in
//   FP32 by diagonal d = i + j, for d <= S-1:
//     TMEM acc0: d = 0, acc1: d = 1, acc2: d = 2   (exact, see below)
//     TMEM acc3: d >= 3                             (rounded; weight <= 2^-24)
//   The epilogue warps drain acc2 after every 64 columns of K (kKChunk), acc1
//   after every 128 and acc0 after every 256, while the tensor core keeps
//   working on the d >= 3 pairs: diagonal d has d + 1 pairs per K step, so a
//   drain carries at most 3 x 64, 2 x 128 or 1 x 256 products of 2^14, i.e.
//   <= 2^22: an exact integer that FP32 represents and that a magic-number add
//   turns into an int32.  The
//   integers are summed in three int32 registers per output element; at the
//   end they and acc3 are combined in one int64 that is rounded once to
//   float64 with the row and column exponents applied (integer arithmetic
//   only: GB300 has little float64 throughput).
// TF32 form: one FP32 operand per side (rounded to TF32), kind::tf32,
//   one 128 x 256 accumulator, FP32 -> float64 in the epilogue.
//
// CTA: 384 threads.  warp 0 = TMA producer, warp 1 = MMA issuer and TMEM
// owner, warps 2-3 idle, warps 4..11 = epilogue (two warps per 32-lane TMEM
// quadrant, one per half of the tile's columns).  Warpgroup 0 gives registers
// to the two epilogue warpgroups (setmaxnreg 56 / 224), which hold the int32
// running sums of their 64 columns.  Optional split-K: each K range adds its
// exact int64 partial sums into a workspace with integer atomics (order-free,
// so the result is deterministic) and a finalize kernel rounds them.  Tiles
// 128 x 128 (split: 64-byte K rows of 32 BF16, SWIZZLE_64B, two stages) or
// 128 x 256 (TF32: 128-byte K rows of 32 FP32, SWIZZLE_128B, four stages), all
// 512 TMEM columns allocated (4 x 128 FP32 accumulators in the split form).
// Every wait is bounded: on expiry the kernel records DEVERR_TIMEOUT in the
// workspace error word, drains its own copies and MMAs, frees TMEM, returns.
#include <cuda.h>
#include <cstdint>
#include <cstdio>
#include <type_traits>
#include <utility>

#include "symctr_internal.h"

namespace symctr {

namespace {

constexpr int TM = 128;
constexpr int NTHREADS = 384;
constexpr int EPI_WARP0 = 4;
constexpr int kExpBias = 4096;     // row exponents are stored biased (0 = all-zero row)
// Every kFoldChunks exact drains, the rounded accumulator of diagonals >= 3 is
// folded as well: its part in units of 2^-16 moves into the int32 running sum
// of diagonal 2 and only the remainder (|r| <= 2^-17) stays in TMEM, so the
// tensor core keeps accumulating into a small value.  This bounds the drift of
// its FP32 accumulation over long K.
constexpr int kFoldChunks = 16;

// Exact accumulators drained after chunk c (bit d = diagonal d): diagonal 2
// after every chunk, 1 after every second, 0 after every fourth (c = -1: none
// were filled yet, all start fresh).
__host__ __device__ constexpr uint32_t drained_after(int c) {
  return c < 0 ? 7u : (4u | (((c + 1) % 2 == 0) ? 2u : 0u) | (((c + 1) % 4 == 0) ? 1u : 0u));
}
constexpr long long kTimeoutCycles = 4000000000ll;  // ~2 s per wait at 2 GHz

enum Mode { MODE_SPLIT = 0, MODE_TF32 = 1 };

// Tile shapes per form: the split form 128 x 128 (four accumulators fill
// TMEM), the TF32 form 128 x 256 (one accumulator; the wider B tile doubles
// the MMA work per byte staged, which bounds TF32 at 128 x 128).
// K bytes per tile row and stage: 64 (32 BF16, SWIZZLE_64B) in the split form,
// whose 5 + 5 slice tiles make 80 KB a stage; 128 (32 FP32, SWIZZLE_128B) in
// the TF32 form, so that a stage carries four K8 MMAs and the issuing thread's
// per-stage waits and commits are amortised over more tensor work.
template <int KIND>
struct TileCfg {
  static constexpr int N = KIND == MODE_TF32 ? 256 : 128;    // output columns per CTA
  static constexpr int ROW_BYTES = KIND == MODE_TF32 ? 128 : 64;
  static constexpr int KSTEPS = ROW_BYTES / 32;              // MMA K steps per stage
  static constexpr int A_BYTES = TM * ROW_BYTES;             // per slice, per stage
  static constexpr int B_BYTES = N * ROW_BYTES;
  static constexpr int LD = N + 1;                           // staging row stride (elements)
  static constexpr size_t EPI_BYTES = (size_t)TM * LD * (KIND == MODE_SPLIT ? 8 : 4);
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(su32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

struct Ctl {
  volatile int abort;
  unsigned* err;
};

// Bounded wait: true when the phase completed; false on timeout or abort.
// The budget is counted in SM clock cycles (clock64 is cheap to read; about
// 2 s at the maximum SM clock, longer at lower clocks).
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, Ctl* ctl,
                                           long long limit = kTimeoutCycles) {
  if (mbar_test(bar, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (mbar_test(bar, parity)) return true;
    if (ctl->abort) return false;
    if (clock64() - t0 > limit) {
      atomicOr(ctl->err, (unsigned)DEVERR_TIMEOUT);
      ctl->abort = 1;
      return false;
    }
  }
}

// Same, for threads with nothing else to do: the hardware suspends them
// between polls (suspend-time hint), so they do not take issue slots from
// the producer and MMA threads.
__device__ __forceinline__ bool mbar_test_sleep(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity), "r"(1000000u)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool wait_phase_sleep(uint64_t* bar, uint32_t parity, Ctl* ctl) {
  const long long t0 = clock64();
  for (;;) {
    if (mbar_test_sleep(bar, parity)) return true;
    if (ctl->abort) return false;
    if (clock64() - t0 > kTimeoutCycles) {
      atomicOr(ctl->err, (unsigned)DEVERR_TIMEOUT);
      ctl->abort = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_3d(const CUtensorMap* map, uint64_t* bar, void* dst,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(su32(dst)),
      "l"(map), "r"(su32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   su32(bar))
               : "memory");
}
// 4 consecutive 32-bit TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}

// 16 consecutive 32-bit TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// 8 consecutive 32-bit TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                 "=r"(r[7])
               : "r"(taddr));
}
template <int W>
__device__ __forceinline__ void tmem_ld_w(uint32_t taddr, uint32_t* r) {
  if constexpr (W == 16) tmem_ld16(taddr, r);
  else if constexpr (W == 8) tmem_ld8(taddr, r);
  else tmem_ld4(taddr, r);
}
// Zeros into W consecutive 32-bit TMEM columns of this warp's 32 lanes.
template <int W>
__device__ __forceinline__ void tmem_zero_w(uint32_t taddr) {
  const uint32_t z = 0u;
  if constexpr (W == 16) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
        "r"(z)
        : "memory");
  } else {
    static_assert(W == 8, "8 or 16 columns");
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
                 "r"(z)
                 : "memory");
  }
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, const uint32_t* r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr),
               "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3])
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, rows of ROW_BYTES swizzled over
// their width (SWIZZLE_64B for 64-byte rows, SWIZZLE_128B for 128-byte rows),
// 8-row groups 8 * ROW_BYTES apart.
template <int KIND>
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  constexpr int RB = TileCfg<KIND>::ROW_BYTES;
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)((8 * RB) >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version (tcgen05)
  d |= (uint64_t)(RB == 128 ? 2 : 4) << 61;   // SWIZZLE_128B / SWIZZLE_64B
  return d;
}

// Instruction descriptor: FP32 accumulate, K-major A and B, M = 128,
// N = the form's tile width.
template <int KIND, int N = TileCfg<KIND>::N>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | ((KIND == MODE_SPLIT ? 1u : 2u) << 7) | ((KIND == MODE_SPLIT ? 1u : 2u) << 10) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

// RN(R * 2^e) as float64 using integer operations only (ties to even).
// Fast path: |R| < 2^53 and a normal result need no rounding, only a shift.
__device__ __forceinline__ double i64_scaled_slow(long long Rv, int e) {
  uint64_t sgn = Rv < 0 ? (1ull << 63) : 0ull;
  uint64_t m = Rv < 0 ? (uint64_t)(-Rv) : (uint64_t)Rv;
  int nb = 64 - __clzll((long long)m);
  int be = e + nb - 1 + 1023;  // biased exponent of the leading bit
  if (be >= 2047) return __longlong_as_double((long long)(sgn | 0x7FF0000000000000ull));
  if (be <= 0) {
    // subnormal: value / 2^-1074 = m * 2^(e + 1074)
    int k = -(e + 1074);
    uint64_t q;
    if (k <= 0) {
      q = m << (-k);
    } else if (k >= 64) {
      q = 0;
      if (k == 64 && m > (1ull << 63)) q = 1;
    } else {
      q = m >> k;
      uint64_t rem = m & ((1ull << k) - 1), half = 1ull << (k - 1);
      if (rem > half || (rem == half && (q & 1))) ++q;
    }
    return __longlong_as_double((long long)(sgn | q));
  }
  int shift = nb - 53;
  uint64_t q;
  if (shift > 0) {
    q = m >> shift;
    uint64_t rem = m & ((1ull << shift) - 1), half = 1ull << (shift - 1);
    if (rem > half || (rem == half && (q & 1))) ++q;
    if (q == (1ull << 53)) {
      q >>= 1;
      ++be;
      if (be >= 2047) return __longlong_as_double((long long)(sgn | 0x7FF0000000000000ull));
    }
  } else {
    q = m << (-shift);
  }
  return __longlong_as_double((long long)(sgn | ((uint64_t)be << 52) | (q & ((1ull << 52) - 1))));
}

__device__ __forceinline__ double i64_scaled(long long Rv, int e) {
  if (Rv == 0) return 0.0;
  const uint64_t m = Rv < 0 ? (uint64_t)(-Rv) : (uint64_t)Rv;
  if (m < (1ull << 53)) {
    const int nb = 64 - __clzll((long long)m);
    const int be = e + nb - 1 + 1023;
    if (be > 0 && be < 2047) {
      const uint64_t q = m << (53 - nb);
      const uint64_t sgn = Rv < 0 ? (1ull << 63) : 0ull;
      return __longlong_as_double((long long)(sgn | ((uint64_t)be << 52) | (q & ((1ull << 52) - 1))));
    }
  }
  return i64_scaled_slow(Rv, e);
}

// Out-of-line copies for the rare entries of a batch (keeps the batch code small).
__device__ __noinline__ double i64_scaled_rare(long long Rv, int e) { return i64_scaled_slow(Rv, e); }

// The common case of i64_scaled without branches (selects only), so that a
// batch of conversions interleaves: exact for Rv = 0, or |Rv| < 2^53 with a
// normal result; `slow` is set for every other Rv.
__device__ __forceinline__ double i64_scaled_common(long long Rv, int e, bool& slow) {
  const uint64_t sm = (uint64_t)(Rv >> 63);   // all ones for Rv < 0
  const uint64_t m = ((uint64_t)Rv ^ sm) - sm;
  const int nb = 64 - __clzll((long long)m);
  const int be = e + nb - 1 + 1023;
  const uint64_t q = m << ((53 - nb) & 63);
  const uint64_t bits = (sm << 63) | ((uint64_t)(unsigned)be << 52) | (q & ((1ull << 52) - 1));
  slow = Rv != 0 && ((m >> 53) != 0 || (unsigned)(be - 1) >= 2046u);
  return Rv == 0 ? 0.0 : __longlong_as_double((long long)bits);
}

// RN(Rv[j] * 2^e[j]) for a batch: the common case for all, the general routine
// only for the entries that need it.
template <int B>
__device__ __forceinline__ void i64_scaled_batch(const long long (&Rv)[B], const int (&e)[B], double (&d)[B]) {
  unsigned slow_mask = 0;
#pragma unroll
  for (int j = 0; j < B; ++j) {
    bool sl;
    d[j] = i64_scaled_common(Rv[j], e[j], sl);
    slow_mask |= (unsigned)sl << j;
  }
  if (slow_mask) {
#pragma unroll
    for (int j = 0; j < B; ++j)
      if ((slow_mask >> j) & 1u) d[j] = i64_scaled_rare(Rv[j], e[j]);
  }
}

// Fire-and-forget 64-bit integer add in L2 (no value returned).
__device__ __forceinline__ void red_add_u64(unsigned long long* a, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(a), "l"(v) : "memory");
}

// Exact float32 -> float64 with integer operations.
__device__ __forceinline__ double f32_to_f64(uint32_t u) {
  uint64_t sgn = (uint64_t)(u >> 31) << 63;
  uint32_t e = (u >> 23) & 0xFF, m = u & 0x7FFFFF;
  if (e == 0) {
    if (m == 0) return __longlong_as_double((long long)sgn);
    double v = i64_scaled((long long)m, -149);
    return sgn ? -v : v;
  }
  if (e == 255) return __longlong_as_double((long long)(sgn | 0x7FF0000000000000ull | ((uint64_t)m << 29)));
  return __longlong_as_double((long long)(sgn | ((uint64_t)(e - 127 + 1023) << 52) | ((uint64_t)m << 29)));
}

__device__ __noinline__ double f32_to_f64_rare(uint32_t u) { return f32_to_f64(u); }

// f32_to_f64 for a batch: normal numbers and zeros without branches, the
// general routine for subnormals, infinities and NaNs.
template <int B>
__device__ __forceinline__ void f32_to_f64_batch(const uint32_t (&u)[B], double (&d)[B]) {
  unsigned slow_mask = 0;
#pragma unroll
  for (int j = 0; j < B; ++j) {
    const uint32_t e = (u[j] >> 23) & 0xFFu;
    const uint64_t sgn = (uint64_t)(u[j] >> 31) << 63;
    const uint64_t bits = sgn | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(u[j] & 0x7FFFFFu) << 29);
    const bool zero = (u[j] << 1) == 0;
    slow_mask |= (unsigned)(!zero && (e == 0 || e == 255)) << j;
    d[j] = __longlong_as_double((long long)(zero ? sgn : bits));
  }
  if (slow_mask) {
#pragma unroll
    for (int j = 0; j < B; ++j)
      if ((slow_mask >> j) & 1u) d[j] = f32_to_f64_rare(u[j]);
  }
}

// Map-back stores of a batch of results of one column (rows m_first, + rstep,
// ...): plain stores, or (complex products) adds, with the problem's sign; the
// output mode is uniform, so the plain path loads nothing from W.
// Rows or columns with offset -1 (general plans: absent from W) are not stored.
template <int B, bool GEN>
__device__ __forceinline__ void store_batch(const Problem& p, double* w, const int64_t (&ro)[B],
                                            int64_t co, const double (&d)[B], int64_t m_first,
                                            int rstep) {
  if (co < 0) return;
  if constexpr (!GEN) {
#pragma unroll
    for (int j = 0; j < B; ++j)
      if (m_first + rstep * j < p.M && ro[j] >= 0) w[ro[j] + co] = d[j];
  } else if (!p.accumulate) {
#pragma unroll
    for (int j = 0; j < B; ++j)
      if (m_first + rstep * j < p.M && ro[j] >= 0) w[(int64_t)p.es * (ro[j] + co)] = signed_result(p, d[j]);
  } else {
#pragma unroll
    for (int j = 0; j < B; ++j)
      if (m_first + rstep * j < p.M && ro[j] >= 0) w[(int64_t)p.es * (ro[j] + co)] += signed_result(p, d[j]);
  }
}

// Descriptor offset of slice tile `i`, K step `kk` (16-byte units).
template <int KIND>
__host__ __device__ constexpr uint64_t dofs(int i, int kk) {
  return (uint64_t)((i * TM * TileCfg<KIND>::ROW_BYTES + kk * 32) >> 4);
}

// Compile-time loop: f(std::integral_constant<int, 0>) ... f(..<N-1>).
template <typename F, int... Is>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, Is...>) {
  (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// One MMA on slice tiles (I, J) at K step KK: the descriptor offsets are
// immediates, so the issuing thread keeps only the two stage bases live.
template <int KIND, int I, int J, int KK>
__device__ __forceinline__ void mma_ij(uint32_t tacc, uint64_t da, uint64_t db, uint32_t id,
                                       uint32_t acc) {
  constexpr unsigned long long oa = dofs<KIND>(I, KK), ob = dofs<KIND>(J, KK);
  if (KIND == MODE_SPLIT) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t.reg .b64 a, b;\n\t"
        "add.u64 a, %1, %5;\n\tadd.u64 b, %2, %6;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], a, b, %3, p;\n\t}\n" ::"r"(tacc),
        "l"(da), "l"(db), "r"(id), "r"(acc), "n"(oa), "n"(ob)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t.reg .b64 a, b;\n\t"
        "add.u64 a, %1, %5;\n\tadd.u64 b, %2, %6;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], a, b, %3, p;\n\t}\n" ::"r"(tacc),
        "l"(da), "l"(db), "r"(id), "r"(acc), "n"(oa), "n"(ob)
        : "memory");
  }
}

// TF32 form (one "slice"): the MMAs of a stage into accumulator 0; bit 0 of
// `fresh` makes the first overwrite it.
template <int KIND, int S>
__device__ __forceinline__ void issue_top(uint32_t tmem, uint64_t da, uint64_t db, uint32_t id,
                                          uint32_t fresh) {
  static_for<3>([&](auto D) {
    if constexpr (D.value <= S - 1) {
      static_for<D.value + 1>([&](auto I) {
        static_for<TileCfg<KIND>::KSTEPS>([&](auto KK) {
          constexpr bool first = I.value == 0 && KK.value == 0;
          mma_ij<KIND, I.value, D.value - I.value, KK.value>(
              tmem + 128u * D.value, da, db, id, (first && ((fresh >> D.value) & 1u)) ? 0u : 1u);
        });
      });
    }
  });
}

// Split form, slice pairs (i, j) with i + j <= S - 1, one MMA each or two at
// once: pairs (i, j) and (i, j + 1) whose targets are consecutive
// accumulators (diagonals i + j and i + j + 1 <= 3, accumulator 3 holding every
// diagonal >= 3) share one N = 256 MMA over B slices j and j + 1, which lie
// one after the other in shared memory: the A slice is read once for both.
// "top" entries touch an exact accumulator (diagonal <= 2), "low" entries only
// accumulator 3.  Every MMA accumulates; the epilogue zeroes the accumulators
// at the start of the tile and after each drain.
struct PairSched {
  int n_top = 0, n_low = 0;
  int ti[21] = {}, tj[21] = {}, tw[21] = {};   // top: A slice, first B slice, 2 = combined
  int li[21] = {}, lj[21] = {};
};
__host__ __device__ constexpr PairSched pair_sched(int S) {
  PairSched r;
  for (int i = 0; i < S; ++i) {
    for (int j = 0; i + j <= S - 1; ++j) {
      const bool combine = i + j <= 2 && i + j + 1 <= S - 1;
      if (combine) {
        r.ti[r.n_top] = i, r.tj[r.n_top] = j, r.tw[r.n_top] = 2, ++r.n_top;
        ++j;
      } else if (i + j <= 2) {
        r.ti[r.n_top] = i, r.tj[r.n_top] = j, r.tw[r.n_top] = 1, ++r.n_top;
      } else {
        r.li[r.n_low] = i, r.lj[r.n_low] = j, ++r.n_low;
      }
    }
  }
  return r;
}

template <int S>
__device__ __forceinline__ void issue_top_acc(uint32_t tmem, uint64_t da, uint64_t db, uint32_t id128,
                                              uint32_t id256) {
  constexpr PairSched P = pair_sched(S);
  static_for<P.n_top>([&](auto T) {
    constexpr int I = P.ti[T.value], J = P.tj[T.value], D = I + J;
    static_for<TileCfg<MODE_SPLIT>::KSTEPS>([&](auto KK) {
      mma_ij<MODE_SPLIT, I, J, KK.value>(tmem + 128u * D, da, db, P.tw[T.value] == 2 ? id256 : id128, 1u);
    });
  });
}

template <int S>
__device__ __forceinline__ void issue_low_acc(uint32_t tmem, uint64_t da, uint64_t db, uint32_t id128) {
  constexpr PairSched P = pair_sched(S);
  static_for<P.n_low>([&](auto T) {
    constexpr int I = P.li[T.value], J = P.lj[T.value];
    static_for<TileCfg<MODE_SPLIT>::KSTEPS>([&](auto KK) {
      mma_ij<MODE_SPLIT, I, J, KK.value>(tmem + 384u, da, db, id128, 1u);
    });
  });
}

struct TcArgs {
  Problem p;
  int S;             // slices (1 for TF32)
  int n_kb;          // K stages
  int ebytes;        // element bytes of the operand tiles (2 or 4)
  const int32_t* eu; // row exponents of U (split form)
  const int32_t* ev; // row exponents of V
  double* w;
  unsigned* err;
  int ksplit;        // K ranges (grid.z = n_q * ksplit)
  int kb_per_split;  // stages per K range (a multiple of 2)
  unsigned long long* wacc;  // [n_q][M][N] int64 partial sums when ksplit > 1 (zeroed)
  const int64_t* wrow;       // [n_q][M] offsets of W's rows in its reduced form
  const int64_t* wcol;       // [n_q][N] offsets of W's columns
};

// Epilogue staging: the results of the tile in shared memory (the operand
// stages are free by then), rows padded by one entry.
template <int KIND, int S, int STAGES>
__host__ __device__ constexpr size_t tile_region_bytes() {
  using C = TileCfg<KIND>;
  return (size_t)STAGES * S * (C::A_BYTES + C::B_BYTES) > C::EPI_BYTES
             ? (size_t)STAGES * S * (C::A_BYTES + C::B_BYTES)
             : C::EPI_BYTES;
}

// GEN: the general output mode (complex element stride, sign, accumulate);
// real contractions use the plain instance, whose epilogue is unchanged.
template <int KIND, int S, int STAGES, bool GEN>
__global__ void __launch_bounds__(NTHREADS, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tma_a, const __grid_constant__ CUtensorMap tma_b,
                   const __grid_constant__ TcArgs args) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const Problem& p = args.p;
  using Cfg = TileCfg<KIND>;
  constexpr int TNk = Cfg::N;
  constexpr int STAGE_LD = Cfg::LD;
  uint8_t* tiles = smem;  // [STAGES][S A tiles, S B tiles], later the epilogue staging
  uint8_t* ctl_base = smem + tile_region_bytes<KIND, S, STAGES>();
  uint64_t* full = (uint64_t*)ctl_base;
  uint64_t* empty = full + STAGES;
  uint64_t* top_full = empty + STAGES;
  uint64_t* top_empty = top_full + 1;
  uint64_t* acc_full = top_empty + 1;
  uint64_t* drain = acc_full + 1;
  uint64_t* low_full = drain + 1;
  uint64_t* low_empty = low_full + 1;
  uint64_t* zero_done = low_empty + 1;          // split form: accumulators zeroed
  int64_t* coff = (int64_t*)(zero_done + 1);   // [TNk] W column offsets
  int32_t* cexp = (int32_t*)(coff + TNk);       // [TNk] column exponents
  int64_t* roffs = (int64_t*)(cexp + TNk);       // [TM] W row offsets
  int32_t* rexps = (int32_t*)(roffs + TM);       // [TM] row exponents
  uint32_t* tmem_slot = (uint32_t*)(rexps + TM);
  Ctl* ctl = (Ctl*)(tmem_slot + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n0 = (int64_t)blockIdx.x * TNk, m0 = (int64_t)blockIdx.y * TM;
  const int b = blockIdx.z / args.ksplit;
  const int ks = blockIdx.z % args.ksplit;
  const int Q = batch_irrep(p, b);
  const int kb0 = ks * args.kb_per_split;
  const int kb1 = min(args.n_kb, kb0 + args.kb_per_split);
  const int n_kb = kb1 - kb0;
  const int n_chunks = KIND == MODE_SPLIT ? (n_kb + 1) / 2 : 1;
  const int stage_bytes = S * (Cfg::A_BYTES + Cfg::B_BYTES);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(top_full, 1);
    mbar_init(top_empty, 8);
    mbar_init(acc_full, 1);
    mbar_init(drain, 1);
    mbar_init(low_full, 1);
    mbar_init(low_empty, 8);
    mbar_init(zero_done, 8);
    ctl->abort = 0;
    ctl->err = args.err;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     su32(tmem_slot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // W's offset tables are constants of the plan: read before the wait.
  if (threadIdx.x >= EPI_WARP0 * 32 && threadIdx.x < EPI_WARP0 * 32 + TNk) {
    const int c = threadIdx.x - EPI_WARP0 * 32;
    const int64_t n = n0 + c, m = m0 + c;
    coff[c] = n < p.N ? args.wcol[(int64_t)b * p.N + n] : 0;
    if (c < TM) roffs[c] = m < p.M ? args.wrow[(int64_t)b * p.M + m] : 0;
  }
  // Launched as a programmatic dependent of the operand preparation: the setup
  // above overlaps its tail; everything below reads its outputs.
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (threadIdx.x >= EPI_WARP0 * 32 && threadIdx.x < EPI_WARP0 * 32 + TNk) {
    const int c = threadIdx.x - EPI_WARP0 * 32;
    const int64_t n = n0 + c, m = m0 + c;
    if (KIND == MODE_SPLIT) {
      cexp[c] = n < p.N ? args.ev[(int64_t)b * p.N + n] - kExpBias : 0;
      if (c < TM) rexps[c] = m < p.M ? args.eu[(int64_t)b * p.M + m] - kExpBias : 0;
    } else {
      cexp[c] = 0;
      if (c < TM) rexps[c] = 0;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp < EPI_WARP0) asm volatile("setmaxnreg.dec.sync.aligned.u32 56;");
  if (warp == 0) {
    // ------------------------------------------------------------ producer
    int issued = 0;
    if (lane == 0) {
      for (int kb = 0; kb < n_kb; ++kb) {
        int st = kb % STAGES;
        uint32_t ph = (kb / STAGES) & 1;
        if (!wait_phase(&empty[st], ph ^ 1, ctl)) break;
        mbar_expect_tx(&full[st], stage_bytes);
        uint8_t* sa = tiles + (size_t)st * stage_bytes;
        uint8_t* sb = sa + S * Cfg::A_BYTES;
        int kc = (kb0 + kb) * (Cfg::ROW_BYTES / args.ebytes);
        for (int i = 0; i < S; ++i) {
          tma_load_3d(&tma_a, &full[st], sa + i * Cfg::A_BYTES, kc, (int)m0, i * p.n_q + b);
          tma_load_3d(&tma_b, &full[st], sb + i * Cfg::B_BYTES, kc, (int)n0, i * p.n_q + b);
        }
        ++issued;
      }
      if (ctl->abort) {
        // let the copies this thread issued land before the CTA exits
        int first = issued > STAGES ? issued - STAGES : 0;
        for (int kb = first; kb < issued; ++kb)
          wait_phase(&full[kb % STAGES], (kb / STAGES) & 1, ctl, kTimeoutCycles / 2);
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id = idesc<KIND>();
      const uint32_t ab = su32(tiles);
      for (int kb = 0; kb < n_kb; ++kb) {
        int st = kb % STAGES;
        uint32_t ph = (kb / STAGES) & 1;
        if (!wait_phase(&full[st], ph, ctl)) break;
        tc_fence_after();
        const uint64_t da = sdesc<KIND>(ab + st * stage_bytes);
        const uint64_t db = sdesc<KIND>(ab + st * stage_bytes + S * Cfg::A_BYTES);
        const bool cfirst = KIND == MODE_TF32 ? (kb == 0) : (kb % 2 == 0);
        const int chunk = KIND == MODE_TF32 ? 0 : kb / 2;
        const bool final_chunk = chunk == n_chunks - 1;
        bool ok = true;
        // fold of accumulator 3 after chunk c: (c + 1) % kFoldChunks == 0, not the last chunk
        constexpr bool has_low = KIND == MODE_SPLIT && S >= 4;
        if (KIND == MODE_SPLIT && kb == 0) {
          // the epilogue warps have zeroed the accumulators
          ok = wait_phase(zero_done, 0, ctl);
          tc_fence_after();
        }
        if (KIND == MODE_TF32) {
          if (ok) issue_top<KIND, S>(tmem, da, db, id, kb == 0 ? 7u : 0u);
        } else if (cfirst) {
          if (has_low && chunk > 0 && chunk % kFoldChunks == 0) {
            ok = ok && wait_phase(low_empty, (uint32_t)(chunk / kFoldChunks - 1) & 1, ctl);
            tc_fence_after();
          }
          if (ok) issue_low_acc<S>(tmem, da, db, id);
          if (chunk > 0) {
            ok = ok && wait_phase(top_empty, (chunk - 1) & 1, ctl);
            tc_fence_after();
          }
          if (ok) issue_top_acc<S>(tmem, da, db, id, idesc<KIND, 256>());
        } else {
          issue_top_acc<S>(tmem, da, db, id, idesc<KIND, 256>());
          if (!final_chunk) tc_commit(top_full);
          issue_low_acc<S>(tmem, da, db, id);
          if (has_low && !final_chunk && (chunk + 1) % kFoldChunks == 0) tc_commit(low_full);
        }
        tc_commit(&empty[st]);
        if (!ok) break;
      }
      tc_commit(acc_full);
      tc_commit(drain);
      wait_phase(drain, 0, ctl, kTimeoutCycles / 2);
    }
  } else if (warp >= EPI_WARP0) {
    // ------------------------------------------------------------ epilogue
    asm volatile("setmaxnreg.inc.sync.aligned.u32 224;");
    const int ew = warp - EPI_WARP0;      // 0..7
    const int quad = warp & 3;            // TMEM lane quadrant this warp may access
    const int half = ew >> 2;             // column half
    const int row = quad * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * (TNk / 2));
    // Running sums of the exact diagonals d = 0, 1, 2 in their own units
    // (1, 2^-8, 2^-16).  Diagonal d has d + 1 slice pairs of |a_i b_j| <= 2^14
    // per K step and is drained every 4, 2, 1 chunks of 64 K (d = 0, 1, 2): at
    // most 256 * 2^14, 2 * 128 * 2^14, 3 * 64 * 2^14 <= 2^22 per drain, which
    // the magic-number drain and the FP32 accumulator hold exactly; int32 holds
    // the sums of 512 chunks, i.e. K up to 32768 per K range (longer K is split).
    int32_t s0[64], s1[64], s2[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) s0[j] = s1[j] = s2[j] = 0;
    const float M0 = 12582912.0f;              // 1.5 * 2^23: ulp 1
    const float M1 = 12582912.0f / 256.0f;     // ulp 2^-8
    const float M2 = 12582912.0f / 65536.0f;   // ulp 2^-16
    const int32_t B0 = (int32_t)__float_as_uint(M0), B1 = (int32_t)__float_as_uint(M1),
                  B2 = (int32_t)__float_as_uint(M2);
    constexpr bool live1 = S >= 2, live2 = S >= 3, live3 = S >= 4;
    // after chunk c: the accumulators in drained_after(c) (always diagonal 2's;
    // every 2nd chunk diagonal 1's, every 4th diagonal 0's), as three
    // straight-line variants
    // W columns per TMEM load and wait: 16 when only diagonal 2 is drained
    // (the common case), 8 otherwise (registers: the running sums take 192)
    auto drain_top = [&](auto D0c, auto D1c) {
      constexpr bool d0 = decltype(D0c)::value, d1 = live1 && decltype(D1c)::value, d2 = live2;
      constexpr int W = (!d0 && !d1) ? 16 : 8;
#pragma unroll
      for (int pc = 0; pc < 64 / W; ++pc) {
        uint32_t a0[W], a1[W], a2[W];
        (void)a0, (void)a1, (void)a2;   // unused in the variants that skip a diagonal
        if constexpr (d0) tmem_ld_w<W>(lane_base + 0 + pc * W, a0);
        if constexpr (d1) tmem_ld_w<W>(lane_base + 128 + pc * W, a1);
        if constexpr (d2) tmem_ld_w<W>(lane_base + 256 + pc * W, a2);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < W; ++j) {
          if constexpr (d0) s0[pc * W + j] += (int32_t)__float_as_uint(__uint_as_float(a0[j]) + M0) - B0;
          if constexpr (d1) s1[pc * W + j] += (int32_t)__float_as_uint(__uint_as_float(a1[j]) + M1) - B1;
          if constexpr (d2) s2[pc * W + j] += (int32_t)__float_as_uint(__uint_as_float(a2[j]) + M2) - B2;
        }
        // the MMAs accumulate: a drained accumulator restarts from zero
        if constexpr (d0) tmem_zero_w<W>(lane_base + 0 + pc * W);
        if constexpr (d1) tmem_zero_w<W>(lane_base + 128 + pc * W);
        if constexpr (d2) tmem_zero_w<W>(lane_base + 256 + pc * W);
      }
      tmem_wait_st();
    };
    bool ok = true;
    if (KIND == MODE_SPLIT) {
      // the accumulators start from zero (every MMA accumulates)
#pragma unroll
      for (int acc = 0; acc < 4; ++acc)
#pragma unroll
        for (int pc = 0; pc < 4; ++pc) tmem_zero_w<16>(lane_base + 128 * acc + pc * 16);
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(zero_done);
      for (int c = 0; c + 1 < n_chunks; ++c) {
        if (!wait_phase_sleep(top_full, c & 1, ctl)) {
          ok = false;
          break;
        }
        tc_fence_after();
        switch (drained_after(c)) {
          case 7u: drain_top(std::true_type{}, std::true_type{}); break;
          case 6u: drain_top(std::false_type{}, std::true_type{}); break;
          default: drain_top(std::false_type{}, std::false_type{}); break;
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(top_empty);
        if (live3 && (c + 1) % kFoldChunks == 0) {
          if (!wait_phase_sleep(low_full, (uint32_t)(c / kFoldChunks) & 1, ctl)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int pc = 0; pc < 16; ++pc) {
            uint32_t a3[4];
            tmem_ld4(lane_base + 384 + pc * 4, a3);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const float x = __uint_as_float(a3[j]);
              const float r = __fmaf_rn(x, 65536.0f, M0);        // round(x * 2^16) + 1.5*2^23
              s2[pc * 4 + j] += (int32_t)__float_as_uint(r) - B0;
              const float back = (r - M0) * (1.0f / 65536.0f);   // exact
              a3[j] = __float_as_uint(x - back);                 // exact remainder
            }
            tmem_st4(lane_base + 384 + pc * 4, a3);
          }
          tmem_wait_st();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(low_empty);
        }
      }
    }
    if (ok) ok = wait_phase_sleep(acc_full, 0, ctl);
    ok = ok && !ctl->abort;
    if (ok) {
      tc_fence_after();
      if (KIND == MODE_SPLIT) {
        // last chunk's exact diagonals and acc3, four columns at a time (the
        // running sums of finished columns die early), staged as int64
        int64_t* st64 = (int64_t*)tiles + row * STAGE_LD + half * 64;
#pragma unroll
        for (int pc = 0; pc < 16; ++pc) {
          uint32_t a0[4], a1[4], a2[4], a3[4];
          tmem_ld4(lane_base + 0 + pc * 4, a0);
          if (live1) tmem_ld4(lane_base + 128 + pc * 4, a1);
          if (live2) tmem_ld4(lane_base + 256 + pc * 4, a2);
          if (live3) tmem_ld4(lane_base + 384 + pc * 4, a3);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int jj = pc * 4 + j;
            int32_t t0 = s0[jj] + (int32_t)__float_as_uint(__uint_as_float(a0[j]) + M0) - B0;
            int32_t t1 = live1 ? s1[jj] + (int32_t)__float_as_uint(__uint_as_float(a1[j]) + M1) - B1 : 0;
            int32_t t2 = live2 ? s2[jj] + (int32_t)__float_as_uint(__uint_as_float(a2[j]) + M2) - B2 : 0;
            // round(acc3 * 2^24) with FP32 operations only (no 64-bit
            // conversion: those run on GB300's narrow float64 pipe).  |acc3|
            // < 64 (at most kFoldChunks chunks since the last fold), so
            // h = round(acc3 * 2^16) is a magic-number conversion, the
            // remainder acc3 - h 2^-16 is exact and |.| <= 2^-17, and
            // round(acc3 * 2^24) = 2^8 h + round(remainder * 2^24).
            long long low = 0;
            if (live3) {
              const float x = __uint_as_float(a3[j]);
              const float r = __fmaf_rn(x, 65536.0f, M0);
              const float rem = x - (r - M0) * (1.0f / 65536.0f);
              const int32_t h = (int32_t)__float_as_uint(r) - B0;
              const int32_t l = (int32_t)__float_as_uint(__fmaf_rn(rem, 16777216.0f, M0)) - B0;
              low = ((long long)h << 8) + l;
            }
            st64[jj] = ((long long)t0 << 24) + ((long long)t1 << 16) + ((long long)t2 << 8) + low;
          }
        }
      } else {
        uint32_t* st32 = (uint32_t*)tiles + row * STAGE_LD + half * (TNk / 2);
#pragma unroll
        for (int pc = 0; pc < TNk / 32; ++pc) {
          uint32_t a0[16];
          tmem_ld16(lane_base + pc * 16, a0);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) st32[pc * 16 + j] = a0[j];
        }
      }
    }
    tc_fence_before();
    // all 256 epilogue threads meet here, whatever path they took
    asm volatile("bar.sync 1, 256;" ::: "memory");
    const int t = threadIdx.x - EPI_WARP0 * 32;
    // Thread t writes column c = t % TNk of rows t / TNk, t / TNk + RSTEP, ...: the
    // column's offset and exponent stay in registers, and each batch issues
    // all of its shared-memory (or L2) loads before any global store, so the
    // loads of a batch overlap instead of waiting behind the stores.
    constexpr int RSTEP = 256 / TNk;
    constexpr int BATCH = 8;
    static_assert(TM % (RSTEP * BATCH) == 0 && 256 % TNk == 0, "epilogue row walk");
    const int c = t % TNk;
    const bool col_ok = n0 + c < p.N;
    const int64_t co = coff[c];
    const int ce = cexp[c] - 36;
    const int64_t acc_col = ((int64_t)b * p.M + m0) * p.N + n0 + c;   // wacc index of row 0
    if (ok && col_ok) {
#pragma unroll 1
      for (int rb = t / TNk; rb < TM; rb += RSTEP * BATCH) {
        if (KIND == MODE_SPLIT) {
          long long Rv[BATCH];
#pragma unroll
          for (int j = 0; j < BATCH; ++j) Rv[j] = ((const long long*)tiles)[(rb + RSTEP * j) * STAGE_LD + c];
          if (args.ksplit > 1) {
#pragma unroll
            for (int j = 0; j < BATCH; ++j) {
              const int r = rb + RSTEP * j;
              if (m0 + r < p.M) red_add_u64(args.wacc + acc_col + (int64_t)r * p.N, (unsigned long long)Rv[j]);
            }
          } else {
            int64_t ro[BATCH];
            int ex[BATCH];
#pragma unroll
            for (int j = 0; j < BATCH; ++j) {
              ro[j] = roffs[rb + RSTEP * j];
              ex[j] = rexps[rb + RSTEP * j] + ce;
            }
            double d[BATCH];
            i64_scaled_batch<BATCH>(Rv, ex, d);
            store_batch<BATCH, GEN>(p, args.w, ro, co, d, m0 + rb, RSTEP);
          }
        } else {
          uint32_t a[BATCH];
          int64_t ro[BATCH];
#pragma unroll
          for (int j = 0; j < BATCH; ++j) {
            a[j] = ((const uint32_t*)tiles)[(rb + RSTEP * j) * STAGE_LD + c];
            ro[j] = roffs[rb + RSTEP * j];
          }
          double d[BATCH];
          f32_to_f64_batch<BATCH>(a, d);
          store_batch<BATCH, GEN>(p, args.w, ro, co, d, m0 + rb, RSTEP);
        }
      }
    }
  }
  // a split-K rounding kernel behind this one may start its launch now
  asm volatile("griddepcontrol.launch_dependents;");
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// Failure-detection self-test: one CTA waits, through the same bounded wait as
// the GEMM's pipeline, on an mbarrier that nothing arrives on.  The wait gives
// up after `limit` cycles, records DEVERR_TIMEOUT in the error word and the
// kernel returns normally (no trap, the context stays usable).
__global__ void bounded_wait_selftest_kernel(unsigned* err, long long limit) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ Ctl ctl;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    ctl.abort = 0;
    ctl.err = err;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) wait_phase(&bar, 0, &ctl, limit);
  __syncthreads();
}

// Split-K rounding: once every K range of the GEMM has added its exact int64
// partial sums into wacc ([n_q][M][N]), each thread takes one column n and
// kRoundRows consecutive rows of one irrep, rounds R * 2^(row exponent +
// column exponent - 36) once to float64 (the same integer-only rounding as the
// GEMM's own epilogue) and stores it through the offset tables.  Launched
// behind the GEMM with programmatic serialization; griddepcontrol.wait makes
// the GEMM's partial sums visible.  Skipped when a GEMM wait timed out (the
// sums are incomplete; the error word already reports it).
constexpr int kRoundRows = 4;
constexpr int kRoundThreads = 256;

template <bool GEN>
__global__ void __launch_bounds__(kRoundThreads) splitk_round_kernel(
    Problem p, const unsigned long long* __restrict__ wacc, const int32_t* __restrict__ eu,
    const int32_t* __restrict__ ev, const int64_t* __restrict__ wrow,
    const int64_t* __restrict__ wcol, double* w, const unsigned* err) {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (*(const volatile unsigned*)err & DEVERR_TIMEOUT) return;
  const int64_t M = p.M, N = p.N;
  const int64_t row_groups = (M + kRoundRows - 1) / kRoundRows;
  const int64_t total = (int64_t)p.n_q * row_groups * N;
  // 32-bit index arithmetic where it fits (64-bit integer division runs on
  // GB300's narrow float64 pipe)
  const bool narrow = total <= 0x7FFFFFFF;
  for (int64_t i = (int64_t)blockIdx.x * kRoundThreads + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * kRoundThreads) {
    int64_t n, b, m0;
    if (narrow) {
      const uint32_t i32 = (uint32_t)i, n32 = (uint32_t)N, g = i32 / n32, rg = (uint32_t)row_groups;
      n = i32 - g * n32;
      b = g / rg;
      m0 = (int64_t)(g - (uint32_t)b * rg) * kRoundRows;
    } else {
      const int64_t g = i / N;
      n = i - g * N;
      b = g / row_groups;
      m0 = (g - b * row_groups) * kRoundRows;
    }
    const int64_t co = wcol[b * N + n];
    const int ce = ev[b * N + n] - kExpBias - 36;
    long long Rv[kRoundRows];
    int64_t ro[kRoundRows];
    int ex[kRoundRows];
#pragma unroll
    for (int j = 0; j < kRoundRows; ++j) {
      const int64_t m = m0 + j;
      const bool in = m < M;
      Rv[j] = in ? (long long)__ldcg(wacc + (b * M + m) * N + n) : 0ll;
      ro[j] = in ? wrow[b * M + m] : 0;
      ex[j] = (in ? eu[b * M + m] - kExpBias : 0) + ce;
    }
    double d[kRoundRows];
    i64_scaled_batch<kRoundRows>(Rv, ex, d);
    store_batch<kRoundRows, GEN>(p, w, ro, co, d, m0, 1);
  }
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)ptr;
  }
  return fn;
}

bool encode_map(CUtensorMap* map, const void* base, bool is_f32, int64_t kpad, int64_t rows,
                int64_t planes, int box_rows);

// 3-D map over [planes][rows][kpad] with a (64-byte, box_rows, 1) box.  The
// encoding is a pure function of its arguments, so the last few are kept per
// host thread (a contraction called again on the same workspace reuses them).
bool make_map(CUtensorMap* map, const void* base, bool is_f32, int64_t kpad, int64_t rows,
              int64_t planes, int box_rows) {
  struct Entry {
    const void* base;
    bool f32;
    int64_t kpad, rows, planes;
    int box_rows;
    CUtensorMap map;
  };
  constexpr int kEntries = 8;
  thread_local Entry cache[kEntries];
  thread_local int used = 0, next = 0;
  for (int i = 0; i < used; ++i) {
    const Entry& e = cache[i];
    if (e.base == base && e.f32 == is_f32 && e.kpad == kpad && e.rows == rows && e.planes == planes &&
        e.box_rows == box_rows) {
      *map = e.map;
      return true;
    }
  }
  if (!encode_map(map, base, is_f32, kpad, rows, planes, box_rows)) return false;
  cache[next] = Entry{base, is_f32, kpad, rows, planes, box_rows, *map};
  next = (next + 1) % kEntries;
  if (used < kEntries) ++used;
  return true;
}

bool encode_map(CUtensorMap* map, const void* base, bool is_f32, int64_t kpad, int64_t rows,
                int64_t planes, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  int eb = is_f32 ? 4 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)kpad, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)(kpad * eb), (cuuint64_t)(kpad * eb * rows)};
  // 128-byte rows with SWIZZLE_128B (TF32), 64-byte rows with SWIZZLE_64B (split)
  const int rb = is_f32 ? TileCfg<MODE_TF32>::ROW_BYTES : TileCfg<MODE_SPLIT>::ROW_BYTES;
  cuuint32_t box[3] = {(cuuint32_t)(rb / eb), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, is_f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  rb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

template <int KIND, int S, int STAGES, bool GEN>
cudaError_t launch_tc_mode(const Problem& p, const Tables& tab, const void* a, const void* bop, const int32_t* eu,
                      const int32_t* ev, int64_t kpad, double* w, unsigned* err, int ksplit,
                      unsigned long long* wacc, cudaStream_t st) {
  const bool f32 = KIND == MODE_TF32;
  CUtensorMap ma, mb;
  if (!make_map(&ma, a, f32, kpad, p.M, (int64_t)S * p.n_q, TM) ||
      !make_map(&mb, bop, f32, kpad, p.N, (int64_t)S * p.n_q, TileCfg<KIND>::N))
    return cudaErrorInvalidValue;
  TcArgs args;
  args.p = p;
  args.S = S;
  args.ebytes = f32 ? 4 : 2;
  args.n_kb = (int)(kpad * args.ebytes / TileCfg<KIND>::ROW_BYTES);
  args.eu = eu;
  args.ev = ev;
  args.w = w;
  args.err = err;
  args.ksplit = ksplit < 1 ? 1 : ksplit;
  args.kb_per_split = ((args.n_kb + args.ksplit - 1) / args.ksplit + 1) / 2 * 2;
  if (args.kb_per_split < 2) args.kb_per_split = 2;
  args.ksplit = (args.n_kb + args.kb_per_split - 1) / args.kb_per_split;
  args.wacc = wacc;
  args.wrow = tab.wrow;
  args.wcol = tab.wcol;
  constexpr int TNk = TileCfg<KIND>::N;
  size_t smem = 1024 + tile_region_bytes<KIND, S, STAGES>() + 8 * (2 * STAGES + 7) + 8 * TNk + 4 * TNk +
                8 * TM + 4 * TM + 16 + 64;
  auto kern = gemm_tc_kernel<KIND, S, STAGES, GEN>;
  thread_local bool attr_set[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (!attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  int64_t gx = (p.N + TNk - 1) / TNk, gy = (p.M + TM - 1) / TM;
  if (gx > 0x7FFFFFFF || gy > 65535 || (int64_t)p.n_q * args.ksplit > 65535)
    return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)(p.n_q * args.ksplit));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(NTHREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t le = cudaLaunchKernelEx(&cfg, kern, ma, mb, args);
  ++g_kernel_launches;
  if (le != cudaSuccess || KIND != MODE_SPLIT || args.ksplit == 1) return le;
  // the rounding of the split-K sums, one thread per kRoundRows outputs
  const int64_t work = (int64_t)p.n_q * ((p.M + kRoundRows - 1) / kRoundRows) * p.N;
  int sms = 148;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = (work + kRoundThreads - 1) / kRoundThreads;
  cudaLaunchConfig_t rc = cfg;
  rc.gridDim = dim3((unsigned)(blocks < (int64_t)sms * 8 ? blocks : (int64_t)sms * 8));
  rc.blockDim = dim3(kRoundThreads);
  rc.dynamicSmemBytes = 0;
  le = cudaLaunchKernelEx(&rc, splitk_round_kernel<GEN>, p, (const unsigned long long*)wacc, eu, ev,
                          tab.wrow, tab.wcol, w, (const unsigned*)err);
  ++g_kernel_launches;
  return le;
}

template <int KIND, int S, int STAGES>
cudaError_t launch_tc(const Problem& p, const Tables& tab, const void* a, const void* bop, const int32_t* eu,
                      const int32_t* ev, int64_t kpad, double* w, unsigned* err, int ksplit,
                      unsigned long long* wacc, cudaStream_t st) {
  if (p.es == 1 && !p.negate && !p.accumulate)
    return launch_tc_mode<KIND, S, STAGES, false>(p, tab, a, bop, eu, ev, kpad, w, err, ksplit, wacc,
                                                  st);
  return launch_tc_mode<KIND, S, STAGES, true>(p, tab, a, bop, eu, ev, kpad, w, err, ksplit, wacc,
                                               st);
}

}  // namespace

cudaError_t launch_gemm_split(const Problem& p, const Tables& tab, int n_slices, const uint16_t* us,
                              const uint16_t* vs, const int32_t* eu, const int32_t* ev,
                              int64_t kpad, double* w, unsigned* err, int ksplit,
                              unsigned long long* wacc, cudaStream_t st) {
  switch (n_slices) {
    case 2: return launch_tc<MODE_SPLIT, 2, 2>(p, tab, us, vs, eu, ev, kpad, w, err, ksplit, wacc, st);
    case 3: return launch_tc<MODE_SPLIT, 3, 2>(p, tab, us, vs, eu, ev, kpad, w, err, ksplit, wacc, st);
    case 4: return launch_tc<MODE_SPLIT, 4, 2>(p, tab, us, vs, eu, ev, kpad, w, err, ksplit, wacc, st);
    case 5: return launch_tc<MODE_SPLIT, 5, 2>(p, tab, us, vs, eu, ev, kpad, w, err, ksplit, wacc, st);
    case 6: return launch_tc<MODE_SPLIT, 6, 2>(p, tab, us, vs, eu, ev, kpad, w, err, ksplit, wacc, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_gemm_tf32(const Problem& p, const Tables& tab, const float* u, const float* v,
                             int64_t kpad, double* w, unsigned* err, cudaStream_t st) {
  return launch_tc<MODE_TF32, 1, 4>(p, tab, u, v, nullptr, nullptr, kpad, w, err, 1, nullptr, st);
}

cudaError_t launch_bounded_wait_selftest(unsigned* err, long long limit_cycles, cudaStream_t st) {
  bounded_wait_selftest_kernel<<<1, 32, 0, st>>>(err, limit_cycles);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace symctr
