// Alignment transforms of Algorithm 2 (input transformations of U and V, the
// output step of W) as separable gathers, and the operand preparation of the
// two tensor-core precision forms.
//
// The paper performs these steps as dense einsums with generalized Kronecker
// deltas (Sec. 3), at O(G) extra cost, and notes that a mechanism using the
// structure of the deltas avoids that factor (Sec. 5.1.1).  Here each aligned
// element (Q, r, c) is read from reduced-form offset row_off(Q, r) +
// col_off(Q, c): constant work per element, pure data movement, bit-exact.
#include <cstdint>

#include "symctr_internal.h"

namespace symctr {

namespace {

constexpr int TILE = 32;
constexpr int THREADS = 256;

// Which side of a map carries the reduced form's unit stride (coalescing).
__host__ inline bool rows_fast(const OperandMap& m) {
  return m.rows.n > 0 && m.rows.bstride[m.rows.n - 1] == 1;
}

// True when columns 2j and 2j+1 of every row are adjacent in memory and the
// even one sits at an even offset: the innermost column digit has stride 1 and
// an even extent, and every other stride of rows and columns is even.
__host__ inline bool pairs_aligned(const OperandMap& m) {
  const AxisMap& c = m.cols;
  if (c.n == 0 || c.bstride[c.n - 1] != 1 || (c.D[c.n - 1] & 1)) return false;
  for (int i = 0; i < c.n; ++i) {
    if (i < c.n - 1 && (c.bstride[i] & 1)) return false;
    if (c.sstride[i] & 1) return false;
  }
  for (int i = 0; i < m.rows.n; ++i)
    if ((m.rows.bstride[i] & 1) || (m.rows.sstride[i] & 1)) return false;
  return true;
}

__global__ void fill_zero_kernel(double* __restrict__ w, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) w[i] = 0.0;
}

// Gather (direction +1: reduced -> aligned) or scatter (-1: aligned -> reduced)
// of one operand, 32x32 tiles through shared memory so that both sides are
// accessed along their contiguous axis.
__global__ void __launch_bounds__(THREADS) align_kernel(Problem p, OperandMap m, int64_t R,
                                                        int64_t Cn, int direction, bool fast_rows,
                                                        const double* __restrict__ src,
                                                        double* __restrict__ dst) {
  __shared__ double tile[TILE][TILE + 1];
  __shared__ int64_t roff[TILE], coff[TILE];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t rt = (R + TILE - 1) / TILE, ct = (Cn + TILE - 1) / TILE;
  const int64_t ntiles = rt * ct * p.n_q;
  for (int64_t tI = blockIdx.x; tI < ntiles; tI += gridDim.x) {
    int64_t b = tI / (rt * ct);
    int64_t rem = tI - b * rt * ct;
    int64_t r0 = (rem / ct) * TILE, c0 = (rem % ct) * TILE;
    int Q = batch_irrep(p, (int)b);
    __syncthreads();
    if (threadIdx.x < TILE) {
      int64_t r = r0 + threadIdx.x;
      roff[threadIdx.x] = r < R ? axis_offset(m.rows, p.g, Q, r) : 0;
    } else if (threadIdx.x < 2 * TILE) {
      int64_t c = c0 + threadIdx.x - TILE;
      coff[threadIdx.x - TILE] = c < Cn ? axis_offset(m.cols, p.g, Q, c) : 0;
    }
    __syncthreads();
    const int64_t abase = (b * R) * Cn;
    if (direction > 0) {
      for (int k = ty; k < TILE; k += THREADS / 32) {
        int rr = fast_rows ? tx : k, cc = fast_rows ? k : tx;
        if (r0 + rr < R && c0 + cc < Cn) tile[rr][cc] = src[roff[rr] + coff[cc]];
      }
      __syncthreads();
      for (int k = ty; k < TILE; k += THREADS / 32) {
        if (r0 + k < R && c0 + tx < Cn) dst[abase + (r0 + k) * Cn + c0 + tx] = tile[k][tx];
      }
    } else {
      for (int k = ty; k < TILE; k += THREADS / 32) {
        if (r0 + k < R && c0 + tx < Cn) tile[k][tx] = src[abase + (r0 + k) * Cn + c0 + tx];
      }
      __syncthreads();
      for (int k = ty; k < TILE; k += THREADS / 32) {
        int rr = fast_rows ? tx : k, cc = fast_rows ? k : tx;
        if (r0 + rr < R && c0 + cc < Cn) dst[roff[rr] + coff[cc]] = tile[rr][cc];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Split-BF16 operand preparation (Ozaki-style splitting, integer arithmetic
// only: GB300 has very little float64 throughput).
//
// For aligned row r with largest binary exponent E_r (|x| < 2^(E_r+1)), each
// entry is written as y = x / 2^(E_r+1) in (-1, 1) and rounded to the integer
// X = round(y * 2^(8S-1)), |X| <= 2^(8S-1).  X is cut into S balanced base-256
// digits a_0..a_{S-1} with a_i in [-128, 128], so y ~= sum_i a_i 2^(-7-8i) with
// error <= 2^(-8S).  Slice i stores a_i * 2^(-8i) as BF16 (exact: a_i has at
// most 8 significant bits), so that every slice-pair product lands at its own
// scale 2^(-8(i+j)) and |a_i b_j| <= 2^14.
// ---------------------------------------------------------------------------

constexpr int32_t kZeroRowExp = -2000;

__device__ __forceinline__ int32_t exponent_of(double x, unsigned* bad) {
  uint64_t bits = (uint64_t)__double_as_longlong(x);
  int ef = (int)((bits >> 52) & 0x7FF);
  uint64_t mant = bits & ((1ull << 52) - 1);
  if (ef == 0x7FF) {
    *bad = 1;
    return kZeroRowExp;
  }
  if (ef != 0) return ef - 1023;
  if (mant == 0) return kZeroRowExp;
  return (63 - __clzll((long long)mant)) - 1074;
}

// X = round(x * 2^(8S - 2 - E)), |X| <= 2^(8S-1).  Round half away from zero.
__device__ __forceinline__ int64_t fixed_point(double x, int32_t E, int S) {
  uint64_t bits = (uint64_t)__double_as_longlong(x);
  int ef = (int)((bits >> 52) & 0x7FF);
  uint64_t mant = bits & ((1ull << 52) - 1);
  int ex;
  if (ef != 0) {
    mant |= 1ull << 52;
    ex = ef - 1075;
  } else {
    ex = -1074;
  }
  if (mant == 0 || E == kZeroRowExp) return 0;
  int sh = ex + 8 * S - 2 - E;
  uint64_t X;
  if (sh >= 0) {
    X = sh >= 63 ? 0 : (mant << sh);  // subnormal rows: |X| <= 2^(8S-1) still holds
  } else {
    int k = -sh;
    X = k > 54 ? 0 : ((mant + (1ull << (k - 1))) >> k);
  }
  int64_t v = (int64_t)X;
  return (bits >> 63) ? -v : v;
}

// Balanced base-256 digits by byte extraction: with B = 0x80 * (256^S - 1)/255,
// Y = X + B has bytes (a_k + 128) for the low S-1 digits and (a_top + 128) in
// [0, 256] above them (no carries: every shifted digit lies in [0, 255]).
__host__ __device__ constexpr uint64_t digit_bias(int S) {
  uint64_t b = 0;
  for (int k = 0; k < S; ++k) b |= (uint64_t)0x80 << (8 * k);
  return b;
}

// BF16 bits of (u - 128) * 2^(-8 i) for a biased digit u in [0, 256], with
// full-rate operations only: 0x4B000000 | u is the float 2^23 + u, so one
// subtraction gives u - 128 exactly; the scale is an exponent decrement.
__device__ __forceinline__ uint32_t bf16_of_biased(uint32_t u, int i) {
  const float f = __uint_as_float(0x4B000000u | u) - 8388736.0f;
  const uint32_t b = __float_as_uint(f) >> 16;
  return b ? b - ((uint32_t)i << 10) : 0u;
}

__device__ __forceinline__ uint16_t digit_bf16(int a, int slice) {
  if (a == 0) return 0;
  float f = (float)a;                                  // exact, |a| <= 128
  f = __fmul_rn(f, __int_as_float((127 - 8 * slice) << 23));  // * 2^(-8 slice), exact
  return (uint16_t)(__float_as_uint(f) >> 16);         // low 16 bits are zero
}

// Row exponents, stored biased: E + kExpBias for a row whose largest entry
// lies in [2^E, 2^(E+1)), 0 for an all-zero row.
constexpr int32_t kExpBias = 4096;
constexpr int SCAN_COLS = 256;
constexpr int SLICE_COLS = 64;

// Bounded grid-wide barrier of the cooperative prep launch (all CTAs are
// co-resident).  `ctr` is zeroed before the launch; barrier number `phase`
// completes when phase * gridDim.x arrivals have been counted.  On a wait of
// more than ~2 s the error word gets DEVERR_TIMEOUT and the CTA goes on.
__device__ __forceinline__ void grid_barrier(unsigned* ctr, unsigned phase, unsigned* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
    const unsigned target = phase * gridDim.x;
    const long long t0 = clock64();
    for (;;) {
      unsigned seen;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(seen) : "l"(ctr) : "memory");
      if (seen >= target) break;
      if (clock64() - t0 > 4000000000ll) {
        atomicOr(err, (unsigned)DEVERR_TIMEOUT);
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
}

struct PrepArgs {
  Problem p;
  Tables t;
  int split;                 // 1: exponent scan + BF16 slices, 0: TF32 copy
  int S;
  int64_t kpad;
  const double* src[2];      // U, V standard reduced forms
  void* dst[2];              // slices (split) or float32 operands (TF32)
  int32_t* exps[2];
  bool fast_rows[2];
  bool pair_ok[2];           // column-contiguous with every offset of an even column even
  unsigned* err;
  unsigned* barrier;
  unsigned long long* zero64;  // split-K partial sums, zeroed here
  int64_t zero64_n;
  unsigned* zero32;            // split-K tile counters, zeroed here
  int64_t zero32_n;
};

__device__ __forceinline__ void operand_dims(const Problem& p, int op, int64_t* R, int64_t* Cn) {
  *R = op == 0 ? p.M : p.N;
  *Cn = p.K;
}

// One 32 x 256 tile of the exponent scan.
__device__ void scan_tile(const PrepArgs& a, int op, int64_t tile, int64_t* roff, int64_t* coff,
                          int32_t* rmax) {
  const Problem& p = a.p;
  int64_t R, Cn;
  operand_dims(p, op, &R, &Cn);
  const int64_t* rtab = op == 0 ? a.t.urow : a.t.vrow;
  const int64_t* ctab = op == 0 ? a.t.ucol : a.t.vcol;
  const double* src = a.src[op];
  int32_t* exps = a.exps[op];
  const bool fast_rows = a.fast_rows[op];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t rt = (R + TILE - 1) / TILE, ct = (Cn + SCAN_COLS - 1) / SCAN_COLS;
  const int64_t b = tile / (rt * ct);
  const int64_t rem = tile - b * rt * ct;
  const int64_t r0 = (rem / ct) * TILE, c0 = (rem % ct) * SCAN_COLS;
  __syncthreads();
  if (threadIdx.x < TILE) {
    int64_t r = r0 + threadIdx.x;
    roff[threadIdx.x] = r < R ? rtab[b * R + r] : 0;
    rmax[threadIdx.x] = 0;
  }
  {
    int64_t c = c0 + threadIdx.x;
    coff[threadIdx.x] = c < Cn ? ctab[b * Cn + c] : 0;
  }
  __syncthreads();
  unsigned bad = 0;
  constexpr int PER = SCAN_COLS / (THREADS / 32);
  if (fast_rows) {
    const bool rok = r0 + tx < R;
    int32_t mx = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      double x[PER / 2];
#pragma unroll
      for (int i = 0; i < PER / 2; ++i) {
        int cc = ty + (h * (PER / 2) + i) * (THREADS / 32);
        x[i] = (rok && c0 + cc < Cn) ? src[roff[tx] + coff[cc]] : 0.0;
      }
#pragma unroll
      for (int i = 0; i < PER / 2; ++i) {
        int32_t e = exponent_of(x[i], &bad);
        mx = max(mx, e == kZeroRowExp ? 0 : e + kExpBias);
      }
    }
    atomicMax(&rmax[tx], mx);
  } else {
#pragma unroll
    for (int rg = 0; rg < TILE / (THREADS / 32); ++rg) {
      int rr = ty + rg * (THREADS / 32);
      const bool rok = r0 + rr < R;
      double x[SCAN_COLS / 32];
#pragma unroll
      for (int i = 0; i < SCAN_COLS / 32; ++i) {
        int cc = tx + 32 * i;
        x[i] = (rok && c0 + cc < Cn) ? src[roff[rr] + coff[cc]] : 0.0;
      }
      int32_t mx = 0;
#pragma unroll
      for (int i = 0; i < SCAN_COLS / 32; ++i) {
        int32_t e = exponent_of(x[i], &bad);
        mx = max(mx, e == kZeroRowExp ? 0 : e + kExpBias);
      }
      for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (tx == 0) rmax[rr] = max(rmax[rr], mx);
    }
  }
  if (bad) atomicOr(a.err, (unsigned)DEVERR_NONFINITE);
  __syncthreads();
  if (threadIdx.x < TILE && r0 + threadIdx.x < R && rmax[threadIdx.x] > 0)
    atomicMax(&exps[b * R + r0 + threadIdx.x], rmax[threadIdx.x]);
}

// Writes the S slices of two adjacent columns (c, c+1) of one row.
template <int S>
__device__ __forceinline__ void put_slices_pair(double x0, double x1, int32_t E, uint32_t* dst,
                                                int64_t stride) {
  const uint64_t y0 = (uint64_t)(fixed_point(x0, E, S) + (int64_t)digit_bias(S));
  const uint64_t y1 = (uint64_t)(fixed_point(x1, E, S) + (int64_t)digit_bias(S));
#pragma unroll
  for (int i = 0; i < S; ++i) {
    const int k = S - 1 - i;  // byte position of slice i's digit
    const uint32_t u0 = i == 0 ? (uint32_t)(y0 >> (8 * k)) : (uint32_t)(y0 >> (8 * k)) & 255u;
    const uint32_t u1 = i == 0 ? (uint32_t)(y1 >> (8 * k)) : (uint32_t)(y1 >> (8 * k)) & 255u;
    dst[(int64_t)i * stride] = bf16_of_biased(u0, i) | (bf16_of_biased(u1, i) << 16);
  }
}

template <int S>
__device__ __forceinline__ void put_slices_one(double x, int32_t E, uint16_t* dst, int64_t stride) {
  const uint64_t y = (uint64_t)(fixed_point(x, E, S) + (int64_t)digit_bias(S));
#pragma unroll
  for (int i = 0; i < S; ++i) {
    const int k = S - 1 - i;
    const uint32_t u = i == 0 ? (uint32_t)(y >> (8 * k)) : (uint32_t)(y >> (8 * k)) & 255u;
    dst[(int64_t)i * stride] = (uint16_t)bf16_of_biased(u, i);
  }
}

__device__ __forceinline__ float tf32_round(double x) {
  uint32_t u = __float_as_uint(__double2float_rn(x));
  if ((u & 0x7F800000u) != 0x7F800000u) u = (u + 0xFFFu + ((u >> 13) & 1u)) & ~0x1FFFu;
  return __uint_as_float(u);
}

// One 32 x 64 tile of the padded aligned operand.  Column-contiguous operands
// are read along the columns straight from global memory (16-byte loads when
// every offset is even), row-contiguous ones go through shared memory so that
// both the gather and the slice stores are coalesced.
template <int S>
__device__ void slice_tile(const PrepArgs& a, int op, int64_t tile, int64_t* roff, int64_t* coff,
                           int32_t* rexp, double (*tilebuf)[SLICE_COLS + 1]) {
  const Problem& p = a.p;
  int64_t R, Cn;
  operand_dims(p, op, &R, &Cn);
  const int64_t kpad = a.kpad;
  const int64_t* rtab = op == 0 ? a.t.urow : a.t.vrow;
  const int64_t* ctab = op == 0 ? a.t.ucol : a.t.vcol;
  const double* src = a.src[op];
  const bool fast_rows = a.fast_rows[op];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t rt = (R + TILE - 1) / TILE, ct = (kpad + SLICE_COLS - 1) / SLICE_COLS;
  const int64_t b = tile / (rt * ct);
  const int64_t rem = tile - b * rt * ct;
  const int64_t r0 = (rem / ct) * TILE, c0 = (rem % ct) * SLICE_COLS;
  const bool split = a.split;
  const int64_t slice_stride = (int64_t)p.n_q * R * kpad;   // elements
  if (!fast_rows) {
    // lanes walk column pairs; warps walk rows; no shared memory
    const int64_t c = c0 + 2 * tx;
    const bool pair = a.pair_ok[op];
    int64_t co0 = 0, co1 = 0;
    if (c < Cn) co0 = ctab[b * Cn + c];
    if (!pair && c + 1 < Cn) co1 = ctab[b * Cn + c + 1];
#pragma unroll
    for (int rg = 0; rg < TILE / (THREADS / 32); ++rg) {
      const int64_t r = r0 + ty + rg * (THREADS / 32);
      if (r >= R || c >= kpad) continue;
      const int64_t ro = rtab[b * R + r];
      double x0 = 0.0, x1 = 0.0;
      if (pair) {
        if (c < Cn) {
          const double2 v2 = *reinterpret_cast<const double2*>(src + ro + co0);
          x0 = v2.x;
          x1 = v2.y;
        }
      } else {
        if (c < Cn) x0 = src[ro + co0];
        if (c + 1 < Cn) x1 = src[ro + co1];
      }
      const int64_t e_at = (b * R + r) * kpad + c;
      if (split) {
        const int32_t st = a.exps[op][b * R + r];
        const int32_t E = st == 0 ? kZeroRowExp : st - kExpBias;
        put_slices_pair<S>(x0, x1, E, (uint32_t*)a.dst[op] + e_at / 2, slice_stride / 2);
      } else {
        float2 f;
        f.x = tf32_round(x0);
        f.y = tf32_round(x1);
        reinterpret_cast<float2*>(a.dst[op])[e_at / 2] = f;
      }
    }
    return;
  }
  __syncthreads();
  if (threadIdx.x < TILE) {
    int64_t r = r0 + threadIdx.x;
    roff[threadIdx.x] = r < R ? rtab[b * R + r] : 0;
    if (split) {
      int32_t st = r < R ? a.exps[op][b * R + r] : 0;
      rexp[threadIdx.x] = st == 0 ? kZeroRowExp : st - kExpBias;
    }
  } else if (threadIdx.x < TILE + SLICE_COLS) {
    int64_t c = c0 + threadIdx.x - TILE;
    coff[threadIdx.x - TILE] = c < Cn ? ctab[b * Cn + c] : 0;
  }
  __syncthreads();
  {
    double x[SLICE_COLS / (THREADS / 32)];
    const bool rok = r0 + tx < R;
#pragma unroll
    for (int i = 0; i < SLICE_COLS / (THREADS / 32); ++i) {
      int cc = ty + i * (THREADS / 32);
      x[i] = (rok && c0 + cc < Cn) ? src[roff[tx] + coff[cc]] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < SLICE_COLS / (THREADS / 32); ++i) tilebuf[tx][ty + i * (THREADS / 32)] = x[i];
  }
  __syncthreads();
  // each thread: one row, two adjacent columns -> one uint32 per slice
  for (int rr = ty; rr < TILE; rr += THREADS / 32) {
    int64_t r = r0 + rr, c = c0 + 2 * tx;
    if (r >= R || c >= kpad) continue;
    const int64_t e_at = (b * R + r) * kpad + c;
    if (split) {
      put_slices_pair<S>(tilebuf[rr][2 * tx], tilebuf[rr][2 * tx + 1], rexp[rr],
                         (uint32_t*)a.dst[op] + e_at / 2, slice_stride / 2);
    } else {
      float2 f;
      f.x = tf32_round(tilebuf[rr][2 * tx]);
      f.y = tf32_round(tilebuf[rr][2 * tx + 1]);
      reinterpret_cast<float2*>(a.dst[op])[e_at / 2] = f;
    }
  }
}

// Operand preparation of one contraction in one cooperative launch:
//   phase 0  offset tables of the six index maps; zero the row exponents and
//            the split-K accumulators;
//   phase 1  (split form) per-row exponent maxima of U and V;
//   phase 2  BF16 slices (split) or TF32 copies of U and V.
__global__ void __launch_bounds__(THREADS, 4) prep_kernel(PrepArgs a) {
  __shared__ int64_t roff[TILE], coff[SCAN_COLS];
  __shared__ int32_t rbuf[TILE];
  __shared__ double tilebuf[TILE][SLICE_COLS + 1];
  const Problem& p = a.p;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // phase 0
  {
    const int64_t segs[6] = {p.M, p.K, p.N, p.K, p.M, p.N};
    int64_t* dsts[6] = {a.t.urow, a.t.ucol, a.t.vrow, a.t.vcol, a.t.wrow, a.t.wcol};
    int64_t total = 0;
    for (int i = 0; i < 6; ++i) total += segs[i] * p.n_q;
    for (int64_t e = gtid; e < total; e += gthreads) {
      int64_t rem = e;
      int which = 0;
      while (rem >= segs[which] * p.n_q) {
        rem -= segs[which] * p.n_q;
        ++which;
      }
      int64_t b = rem / segs[which], r = rem % segs[which];
      int Q = batch_irrep(p, (int)b);
      const AxisMap& m = which == 0 ? p.u.rows : which == 1 ? p.u.cols : which == 2 ? p.v.rows
                       : which == 3 ? p.v.cols : which == 4 ? p.w.rows : p.w.cols;
      dsts[which][rem] = axis_offset(m, p.g, Q, r);
    }
    if (a.split) {
      for (int64_t e = gtid; e < (int64_t)p.n_q * p.M; e += gthreads) a.exps[0][e] = 0;
      for (int64_t e = gtid; e < (int64_t)p.n_q * p.N; e += gthreads) a.exps[1][e] = 0;
    }
    for (int64_t e = gtid; e < a.zero64_n; e += gthreads) a.zero64[e] = 0ull;
    for (int64_t e = gtid; e < a.zero32_n; e += gthreads) a.zero32[e] = 0u;
  }
  grid_barrier(a.barrier, 1, a.err);
  unsigned next = 2;
  if (a.split) {
    int64_t tiles[2];
    for (int op = 0; op < 2; ++op) {
      int64_t R, Cn;
      operand_dims(p, op, &R, &Cn);
      tiles[op] = ((R + TILE - 1) / TILE) * ((Cn + SCAN_COLS - 1) / SCAN_COLS) * p.n_q;
    }
    for (int64_t t = blockIdx.x; t < tiles[0] + tiles[1]; t += gridDim.x) {
      int op = t < tiles[0] ? 0 : 1;
      scan_tile(a, op, op == 0 ? t : t - tiles[0], roff, coff, rbuf);
    }
    grid_barrier(a.barrier, next++, a.err);
  }
  // the GEMM that consumes these operands may start its setup now
  asm volatile("griddepcontrol.launch_dependents;");
  {
    int64_t tiles[2];
    for (int op = 0; op < 2; ++op) {
      int64_t R, Cn;
      operand_dims(p, op, &R, &Cn);
      tiles[op] = ((R + TILE - 1) / TILE) * ((a.kpad + SLICE_COLS - 1) / SLICE_COLS) * p.n_q;
    }
    for (int64_t t = blockIdx.x; t < tiles[0] + tiles[1]; t += gridDim.x) {
      int op = t < tiles[0] ? 0 : 1;
      int64_t tt = op == 0 ? t : t - tiles[0];
      switch (a.split ? a.S : 1) {
        case 1: slice_tile<1>(a, op, tt, roff, coff, rbuf, tilebuf); break;
        case 2: slice_tile<2>(a, op, tt, roff, coff, rbuf, tilebuf); break;
        case 3: slice_tile<3>(a, op, tt, roff, coff, rbuf, tilebuf); break;
        case 4: slice_tile<4>(a, op, tt, roff, coff, rbuf, tilebuf); break;
        case 5: slice_tile<5>(a, op, tt, roff, coff, rbuf, tilebuf); break;
        default: slice_tile<6>(a, op, tt, roff, coff, rbuf, tilebuf); break;
      }
    }
  }
}

int grid_for(int64_t tiles) {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t cap = (int64_t)sms * 8;
  return (int)(tiles < cap ? (tiles > 0 ? tiles : 1) : cap);
}

const OperandMap& operand_map(const Problem& p, int operand) {
  return operand == 0 ? p.u : operand == 1 ? p.v : p.w;
}

void operand_extent(const Problem& p, int operand, int64_t* R, int64_t* Cn) {
  if (operand == 0) { *R = p.M; *Cn = p.K; }
  else if (operand == 1) { *R = p.N; *Cn = p.K; }
  else { *R = p.M; *Cn = p.N; }
}

}  // namespace

cudaError_t launch_fill_zero(double* w, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  fill_zero_kernel<<<grid_for(blocks), 256, 0, st>>>(w, n);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_align_f64(const Problem& p, int operand, int direction, const double* src,
                             double* dst, cudaStream_t st) {
  int64_t R, Cn;
  operand_extent(p, operand, &R, &Cn);
  if (R == 0 || Cn == 0 || p.n_q == 0) return cudaSuccess;
  const OperandMap& m = operand_map(p, operand);
  int64_t tiles = ((R + TILE - 1) / TILE) * ((Cn + TILE - 1) / TILE) * p.n_q;
  align_kernel<<<grid_for(tiles), THREADS, 0, st>>>(p, m, R, Cn, direction, rows_fast(m), src, dst);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_prep(const Problem& p, const Tables& t, bool split, int n_slices,
                        const double* u, const double* v, void* ua, void* va, int32_t* eu,
                        int32_t* ev, int64_t kpad, unsigned* err, unsigned* barrier,
                        unsigned long long* zero64, int64_t zero64_n, unsigned* zero32,
                        int64_t zero32_n, cudaStream_t st) {
  static int max_blocks = 0;
  if (max_blocks == 0) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, prep_kernel, THREADS, 0);
    if (e != cudaSuccess) return e;
    max_blocks = sms * (per < 4 ? per : 4);
  }
  int64_t work = 0;
  {
    int64_t rt_u = (p.M + TILE - 1) / TILE, rt_v = (p.N + TILE - 1) / TILE;
    int64_t ct = (kpad + SLICE_COLS - 1) / SLICE_COLS;
    work = (rt_u + rt_v) * ct * p.n_q;
  }
  int grid = (int)(work < max_blocks ? (work > 0 ? work : 1) : max_blocks);
  PrepArgs a;
  a.p = p;
  a.t = t;
  a.split = split ? 1 : 0;
  a.S = n_slices;
  a.kpad = kpad;
  a.src[0] = u;
  a.src[1] = v;
  a.dst[0] = ua;
  a.dst[1] = va;
  a.exps[0] = eu;
  a.exps[1] = ev;
  a.fast_rows[0] = rows_fast(p.u);
  a.fast_rows[1] = rows_fast(p.v);
  a.pair_ok[0] = !a.fast_rows[0] && pairs_aligned(p.u);
  a.pair_ok[1] = !a.fast_rows[1] && pairs_aligned(p.v);
  a.err = err;
  a.barrier = barrier;
  a.zero64 = zero64;
  a.zero64_n = zero64_n;
  a.zero32 = zero32;
  a.zero32_n = zero32_n;
  void* params[] = {&a};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)prep_kernel, dim3(grid), dim3(THREADS),
                                              params, 0, st);
  ++g_kernel_launches;
  return e;
}

}  // namespace symctr
