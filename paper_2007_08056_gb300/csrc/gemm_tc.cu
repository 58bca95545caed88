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
//   Every 64 columns of K (kKChunk) the epilogue warps drain acc0..acc2 while
//   the tensor core keeps working on the d >= 3 pairs: at most 3 pairs x 64 x
//   2^14 <= 2^22 per drain, so each drained value is an exact integer that
//   FP32 represents and that a magic-number add turns into an int32.  The
//   integers are summed in one int64 per output element; at the end acc3 is
//   folded in and the int64 is rounded once to float64 with the row and
//   column exponents applied (integer arithmetic only: GB300 has little
//   float64 throughput).
// TF32 form: one FP32 operand per side (rounded to TF32), kind::tf32,
//   one accumulator, FP32 -> float64 in the epilogue.
//
// CTA: 384 threads.  warp 0 = TMA producer, warp 1 = MMA issuer and TMEM
// owner, warps 2-3 idle, warps 4..11 = epilogue (two warps per 32-lane TMEM
// quadrant, one per half of the 128 columns).  Warpgroup 0 gives registers
// to the two epilogue warpgroups (setmaxnreg 40 / 232), which hold the int64
// running sums of their 64 columns.  Optional split-K: each K range adds its
// exact int64 partial sums into a workspace with integer atomics (order-free,
// so the result is deterministic) and a finalize kernel rounds them.  Tile 128 x 128, 64-byte K rows (32 BF16 or 16
// FP32), SWIZZLE_64B, all 512 TMEM columns (4 x 128 FP32 accumulators).
// Every wait is bounded: on expiry the kernel records DEVERR_TIMEOUT in the
// workspace error word, drains its own copies and MMAs, frees TMEM, returns.
#include <cuda.h>
#include <cstdint>
#include <cstdio>

#include "symctr_internal.h"

namespace symctr {

namespace {

constexpr int TM = 128, TN = 128;
constexpr int ROW_BYTES = 64;                  // K bytes per tile row per stage
constexpr int TILE_BYTES = TM * ROW_BYTES;     // 8 KB per operand tile per stage
constexpr int NTHREADS = 384;
constexpr int EPI_WARP0 = 4;
constexpr int kExpBias = 4096;     // row exponents are stored biased (0 = all-zero row)
constexpr uint64_t kTimeoutNs = 2000000000ull;  // 2 s per wait

enum Mode { MODE_SPLIT = 0, MODE_TF32 = 1 };

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
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
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t parity, Ctl* ctl,
                                        uint64_t limit = kTimeoutNs) {
  if (mbar_test(bar, parity)) return true;
  uint64_t t0 = globaltimer();
  for (;;) {
    for (int i = 0; i < 32; ++i)
      if (mbar_test(bar, parity)) return true;
    if (ctl->abort) return false;
    if (globaltimer() - t0 > limit) {
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
template <int KIND>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc) {
  if (KIND == MODE_SPLIT) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}

// 8 consecutive 32-bit TMEM columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
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
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, SWIZZLE_64B, 8-row groups 512 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version (tcgen05)
  d |= (uint64_t)4 << 61;             // SWIZZLE_64B
  return d;
}

// Instruction descriptor: FP32 accumulate, K-major A and B, M = 128, N = 128.
template <int KIND>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | ((KIND == MODE_SPLIT ? 1u : 2u) << 7) | ((KIND == MODE_SPLIT ? 1u : 2u) << 10) |
         ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

// RN(R * 2^e) as float64 using integer operations only (ties to even).
__device__ __forceinline__ double i64_scaled(long long Rv, int e) {
  if (Rv == 0) return 0.0;
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

struct PairList {
  int n;
  int8_t i[21], j[21], acc[21];
};

struct TcArgs {
  Problem p;
  int S;             // slices (1 for TF32)
  int n_kb;          // K stages
  int ebytes;        // element bytes of the operand tiles (2 or 4)
  const int32_t* eu; // row exponents of U (split form)
  const int32_t* ev; // row exponents of V
  double* w;
  unsigned* err;
  PairList top, low;
  int acc_live;      // bit mask of accumulators written by at least one MMA
  int ksplit;        // K ranges (grid.z = n_q * ksplit)
  int kb_per_split;  // stages per K range (a multiple of 2)
  unsigned long long* wacc;  // [n_q][M][N] int64 partial sums when ksplit > 1
};

template <int KIND, int STAGES>
__global__ void __launch_bounds__(NTHREADS, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tma_a, const __grid_constant__ CUtensorMap tma_b,
                   const __grid_constant__ TcArgs args) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int S = args.S;
  const Problem& p = args.p;
  uint8_t* tiles = smem;  // [STAGES][2][S][TILE_BYTES]
  uint8_t* ctl_base = smem + (size_t)STAGES * 2 * S * TILE_BYTES;
  uint64_t* full = (uint64_t*)ctl_base;
  uint64_t* empty = full + STAGES;
  uint64_t* top_full = empty + STAGES;
  uint64_t* top_empty = top_full + 1;
  uint64_t* acc_full = top_empty + 1;
  uint64_t* drain = acc_full + 1;
  int64_t* coff = (int64_t*)(drain + 1);       // [TN] W column offsets
  int32_t* cexp = (int32_t*)(coff + TN);        // [TN] column exponents
  uint32_t* tmem_slot = (uint32_t*)(cexp + TN);
  Ctl* ctl = (Ctl*)(tmem_slot + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n0 = (int64_t)blockIdx.x * TN, m0 = (int64_t)blockIdx.y * TM;
  const int b = blockIdx.z / args.ksplit;
  const int ks = blockIdx.z % args.ksplit;
  const int Q = batch_irrep(p, b);
  const int kb0 = ks * args.kb_per_split;
  const int kb1 = min(args.n_kb, kb0 + args.kb_per_split);
  const int n_kb = kb1 - kb0;
  const int n_chunks = KIND == MODE_SPLIT ? (n_kb + 1) / 2 : 1;
  const int stage_bytes = 2 * S * TILE_BYTES;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(top_full, 1);
    mbar_init(top_empty, 8);
    mbar_init(acc_full, 1);
    mbar_init(drain, 1);
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
  if (threadIdx.x >= EPI_WARP0 * 32 && threadIdx.x < EPI_WARP0 * 32 + TN) {
    int c = threadIdx.x - EPI_WARP0 * 32;
    int64_t n = n0 + c;
    coff[c] = n < p.N ? axis_offset(p.w.cols, p.g, Q, n) : 0;
    cexp[c] = (KIND == MODE_SPLIT && n < p.N) ? args.ev[(int64_t)b * p.N + n] - kExpBias : 0;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp < EPI_WARP0) asm volatile("setmaxnreg.dec.sync.aligned.u32 40;");
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
        uint8_t* sb = sa + S * TILE_BYTES;
        int kc = (kb0 + kb) * (ROW_BYTES / args.ebytes);
        for (int i = 0; i < S; ++i) {
          tma_load_3d(&tma_a, &full[st], sa + i * TILE_BYTES, kc, (int)m0, i * p.n_q + b);
          tma_load_3d(&tma_b, &full[st], sb + i * TILE_BYTES, kc, (int)n0, i * p.n_q + b);
        }
        ++issued;
      }
      if (ctl->abort) {
        // let the copies this thread issued land before the CTA exits
        int first = issued > STAGES ? issued - STAGES : 0;
        for (int kb = first; kb < issued; ++kb)
          wait_phase(&full[kb % STAGES], (kb / STAGES) & 1, ctl, kTimeoutNs / 2);
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
        const uint32_t sa = ab + st * stage_bytes;
        const uint32_t sb = sa + S * TILE_BYTES;
        const bool cfirst = KIND == MODE_TF32 ? (kb == 0) : (kb % 2 == 0);
        const int chunk = KIND == MODE_TF32 ? 0 : kb / 2;
        const bool final_chunk = chunk == n_chunks - 1;
        auto issue = [&](const PairList& L, bool fresh) {
          bool seen[4] = {false, false, false, false};
          for (int q = 0; q < L.n; ++q) {
            int a = L.acc[q];
            uint32_t d = tmem + 128u * a;
            for (int kk = 0; kk < 2; ++kk) {
              uint32_t accum = (fresh && !seen[a] && kk == 0) ? 0u : 1u;
              tc_mma<KIND>(d, sdesc(sa + L.i[q] * TILE_BYTES + kk * 32),
                           sdesc(sb + L.j[q] * TILE_BYTES + kk * 32), id, accum);
            }
            seen[a] = true;
          }
        };
        bool ok = true;
        if (cfirst) {
          issue(args.low, kb == 0);
          if (chunk > 0) {
            ok = wait_phase(top_empty, (chunk - 1) & 1, ctl);
            tc_fence_after();
          }
          if (ok) issue(args.top, true);
        } else {
          issue(args.top, false);
          if (!final_chunk) tc_commit(top_full);
          issue(args.low, false);
        }
        tc_commit(&empty[st]);
        if (!ok) break;
      }
      tc_commit(acc_full);
      tc_commit(drain);
      wait_phase(drain, 0, ctl, kTimeoutNs / 2);
    }
  } else if (warp >= EPI_WARP0) {
    // ------------------------------------------------------------ epilogue
    asm volatile("setmaxnreg.inc.sync.aligned.u32 232;");
    const int ew = warp - EPI_WARP0;      // 0..7
    const int quad = warp & 3;            // TMEM lane quadrant this warp may access
    const int half = ew >> 2;             // column half
    const int row = quad * 32 + lane;
    const int64_t m = m0 + row;
    const uint32_t lane_base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * 64);
    int64_t racc[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) racc[j] = 0;
    const float M0 = 12582912.0f;              // 1.5 * 2^23
    const float M1 = 12582912.0f / 256.0f;     // unit 2^-8
    const float M2 = 12582912.0f / 65536.0f;   // unit 2^-16
    const uint32_t B0 = __float_as_uint(M0), B1 = __float_as_uint(M1), B2 = __float_as_uint(M2);
    const uint32_t C01 = B0 * 256u + B1;
    const bool live1 = (args.acc_live >> 1) & 1, live2 = (args.acc_live >> 2) & 1,
               live3 = (args.acc_live >> 3) & 1;
    auto drain_top = [&]() {
#pragma unroll
      for (int pc = 0; pc < 8; ++pc) {
        uint32_t a0[8], a1[8], a2[8];
        tmem_ld8(lane_base + 0 + pc * 8, a0);
        if (live1) tmem_ld8(lane_base + 128 + pc * 8, a1);
        if (live2) tmem_ld8(lane_base + 256 + pc * 8, a2);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          uint32_t v0 = __float_as_uint(__uint_as_float(a0[j]) + M0);
          uint32_t v1 = live1 ? __float_as_uint(__uint_as_float(a1[j]) + M1) : B1;
          uint32_t v2 = live2 ? __float_as_uint(__uint_as_float(a2[j]) + M2) : B2;
          int32_t x = (int32_t)(v0 * 256u + v1 - C01);
          int32_t y = (int32_t)(v2 - B2);
          racc[pc * 8 + j] += (int64_t)x * 256 + y;
        }
      }
    };
    bool ok = true;
    if (KIND == MODE_SPLIT) {
      for (int c = 0; c + 1 < n_chunks; ++c) {
        if (!wait_phase(top_full, c & 1, ctl)) {
          ok = false;
          break;
        }
        tc_fence_after();
        drain_top();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(top_empty);
      }
    }
    if (ok) ok = wait_phase(acc_full, 0, ctl);
    if (ok && !ctl->abort) {
      tc_fence_after();
      const bool row_ok = m < p.M;
      const int64_t roff = row_ok ? axis_offset(p.w.rows, p.g, Q, m) : 0;
      double* wout = args.w + roff;
      if (KIND == MODE_SPLIT) {
        drain_top();
        const int32_t er = row_ok ? args.eu[(int64_t)b * p.M + m] - kExpBias : 0;
        unsigned long long* wacc = args.wacc + ((int64_t)b * p.M + m) * p.N + n0;
#pragma unroll
        for (int pc = 0; pc < 4; ++pc) {
          uint32_t a3[16];
          if (live3) {
            tmem_ld16(lane_base + 384 + pc * 16, a3);
            tmem_wait_ld();
          }
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            int c = half * 64 + pc * 16 + j;
            long long low = live3 ? __float2ll_rn(__uint_as_float(a3[j]) * 16777216.0f) : 0ll;
            long long Rv = (long long)(racc[pc * 16 + j] << 8) + low;
            if (row_ok && n0 + c < p.N) {
              if (args.ksplit > 1) atomicAdd(wacc + c, (unsigned long long)Rv);
              else wout[coff[c]] = i64_scaled(Rv, er + cexp[c] - 36);
            }
          }
        }
      } else {
#pragma unroll
        for (int pc = 0; pc < 4; ++pc) {
          uint32_t a0[16];
          tmem_ld16(lane_base + pc * 16, a0);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            int c = half * 64 + pc * 16 + j;
            if (row_ok && n0 + c < p.N) wout[coff[c]] = f32_to_f64(a0[j]);
          }
        }
      }
    }
    tc_fence_before();
  }
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

// Split-K finalize: round the summed int64 partials once and map them back.
__global__ void __launch_bounds__(256) split_finalize_kernel(Problem p,
                                                             const unsigned long long* __restrict__ wacc,
                                                             const int32_t* __restrict__ eu,
                                                             const int32_t* __restrict__ ev,
                                                             double* __restrict__ w) {
  const int64_t total = (int64_t)p.n_q * p.M * p.N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = i / (p.M * p.N);
    int64_t r = i - b * p.M * p.N;
    int64_t m = r / p.N, n = r % p.N;
    int Q = batch_irrep(p, (int)b);
    int e = (eu[b * p.M + m] - kExpBias) + (ev[b * p.N + n] - kExpBias) - 36;
    w[axis_offset(p.w.rows, p.g, Q, m) + axis_offset(p.w.cols, p.g, Q, n)] =
        i64_scaled((long long)wacc[i], e);
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

// 3-D map over [planes][rows][kpad] with a (64-byte, 128-row, 1) box.
bool make_map(CUtensorMap* map, const void* base, bool is_f32, int64_t kpad, int64_t rows,
              int64_t planes) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  int eb = is_f32 ? 4 : 2;
  cuuint64_t dims[3] = {(cuuint64_t)kpad, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)(kpad * eb), (cuuint64_t)(kpad * eb * rows)};
  cuuint32_t box[3] = {(cuuint32_t)(ROW_BYTES / eb), (cuuint32_t)TM, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(map, is_f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                  const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

void build_pairs(int S, PairList* top, PairList* low, int* live) {
  top->n = low->n = 0;
  *live = 0;
  for (int d = 0; d <= S - 1; ++d) {
    for (int i = 0; i <= d; ++i) {
      int j = d - i;
      if (i >= S || j >= S) continue;
      PairList* L = d <= 2 ? top : low;
      int acc = d <= 2 ? d : 3;
      L->i[L->n] = (int8_t)i;
      L->j[L->n] = (int8_t)j;
      L->acc[L->n] = (int8_t)acc;
      ++L->n;
      *live |= 1 << acc;
    }
  }
}

template <int KIND, int STAGES>
cudaError_t launch_tc(const Problem& p, int S, const void* a, const void* bop, const int32_t* eu,
                      const int32_t* ev, int64_t kpad, double* w, unsigned* err, int ksplit,
                      unsigned long long* wacc, cudaStream_t st) {
  const bool f32 = KIND == MODE_TF32;
  CUtensorMap ma, mb;
  if (!make_map(&ma, a, f32, kpad, p.M, (int64_t)S * p.n_q) ||
      !make_map(&mb, bop, f32, kpad, p.N, (int64_t)S * p.n_q))
    return cudaErrorInvalidValue;
  TcArgs args;
  args.p = p;
  args.S = S;
  args.ebytes = f32 ? 4 : 2;
  args.n_kb = (int)(kpad * args.ebytes / ROW_BYTES);
  args.eu = eu;
  args.ev = ev;
  args.w = w;
  args.err = err;
  args.ksplit = ksplit < 1 ? 1 : ksplit;
  args.kb_per_split = ((args.n_kb + args.ksplit - 1) / args.ksplit + 1) / 2 * 2;
  if (args.kb_per_split < 2) args.kb_per_split = 2;
  args.ksplit = (args.n_kb + args.kb_per_split - 1) / args.kb_per_split;
  args.wacc = wacc;
  if (args.ksplit > 1) {
    cudaError_t e0 = cudaMemsetAsync(wacc, 0, sizeof(unsigned long long) * p.n_q * p.M * p.N, st);
    if (e0 != cudaSuccess) return e0;
  }
  if (KIND == MODE_SPLIT) {
    build_pairs(S, &args.top, &args.low, &args.acc_live);
  } else {
    args.top.n = 1;
    args.top.i[0] = args.top.j[0] = args.top.acc[0] = 0;
    args.low.n = 0;
    args.acc_live = 1;
  }
  size_t smem = 1024 + (size_t)STAGES * 2 * S * TILE_BYTES + 8 * (2 * STAGES + 4) + 8 * TN +
                4 * TN + 16 + 64;
  auto kern = gemm_tc_kernel<KIND, STAGES>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int64_t gx = (p.N + TN - 1) / TN, gy = (p.M + TM - 1) / TM;
  if (gx > 0x7FFFFFFF || gy > 65535 || (int64_t)p.n_q * args.ksplit > 65535)
    return cudaErrorInvalidConfiguration;
  dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)(p.n_q * args.ksplit));
  kern<<<grid, NTHREADS, smem, st>>>(ma, mb, args);
  ++g_kernel_launches;
  if (args.ksplit > 1) {
    int64_t total = (int64_t)p.n_q * p.M * p.N;
    int64_t blocks = (total + 255) / 256;
    split_finalize_kernel<<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(p, wacc, eu, ev, w);
    ++g_kernel_launches;
  }
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gemm_split(const Problem& p, int n_slices, const uint16_t* us,
                              const uint16_t* vs, const int32_t* eu, const int32_t* ev,
                              int64_t kpad, double* w, unsigned* err, int ksplit,
                              unsigned long long* wacc, cudaStream_t st) {
  return launch_tc<MODE_SPLIT, 2>(p, n_slices, us, vs, eu, ev, kpad, w, err, ksplit, wacc, st);
}

cudaError_t launch_gemm_tf32(const Problem& p, const float* u, const float* v, int64_t kpad,
                             double* w, unsigned* err, cudaStream_t st) {
  return launch_tc<MODE_TF32, 6>(p, 1, u, v, nullptr, nullptr, kpad, w, err, 1, nullptr, st);
}

}  // namespace symctr
