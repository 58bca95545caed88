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

#include <cuda_bf16.h>

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
  // (never asked for general plans: a padded column pair may be half absent)
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
                                                        const int64_t* __restrict__ rtab,
                                                        const int64_t* __restrict__ ctab,
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
    // general plans: offsets from the tables, -1 marking an absent row/column
    if (threadIdx.x < TILE) {
      int64_t r = r0 + threadIdx.x;
      roff[threadIdx.x] = r < R ? (rtab ? rtab[b * R + r] : axis_offset(m.rows, p.g, Q, r)) : 0;
    } else if (threadIdx.x < 2 * TILE) {
      int64_t c = c0 + threadIdx.x - TILE;
      coff[threadIdx.x - TILE] = c < Cn ? (ctab ? ctab[b * Cn + c] : axis_offset(m.cols, p.g, Q, c)) : 0;
    }
    __syncthreads();
    const int64_t abase = (b * R) * Cn;
    if (direction > 0) {
      for (int k = ty; k < TILE; k += THREADS / 32) {
        int rr = fast_rows ? tx : k, cc = fast_rows ? k : tx;
        if (r0 + rr < R && c0 + cc < Cn)
          tile[rr][cc] = (roff[rr] >= 0 && coff[cc] >= 0) ? src[roff[rr] + coff[cc]] : 0.0;
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
        if (r0 + rr < R && c0 + cc < Cn && roff[rr] >= 0 && coff[cc] >= 0)
          dst[roff[rr] + coff[cc]] = tile[rr][cc];
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

// Row exponents, stored biased: E + kExpBias for a row whose largest entry
// lies in [2^E, 2^(E+1)) (E clamped below at 8S - 1076, see row_key), 0 for an
// all-zero row.
constexpr int32_t kExpBias = 4096;
constexpr int SCAN_COLS = 256;
constexpr int SLICE_COLS = 64;
constexpr int SLICE_GROUP = 4;   // 64-column sub-tiles per slice work unit

// |x| as its IEEE bit pattern: the order of these integers is the order of
// the magnitudes, so a row maximum needs only integer max operations.
__device__ __forceinline__ uint64_t abs_bits(double x) {
  return (uint64_t)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// Running maximum of |x| bit patterns kept as two 32-bit maxima: of the high
// words (sign dropped) and of the low words.  Whenever some high word is
// nonzero the row's scale depends on the high word of the largest entry only;
// when all are zero the largest pattern is the largest low word.  Two 32-bit
// integer max operations per entry instead of a 64-bit one.
struct Max2 {
  uint32_t hi = 0u, lo = 0u;
  __device__ __forceinline__ void add(double x) {
    hi = max(hi, (uint32_t)__double2hiint(x) & 0x7FFFFFFFu);
    lo = max(lo, (uint32_t)__double2loint(x));
  }
  __device__ __forceinline__ void merge_xor(int o) {
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    lo = max(lo, __shfl_xor_sync(0xffffffffu, lo, o));
  }
  __device__ __forceinline__ uint64_t pattern() const { return hi != 0u ? (uint64_t)hi << 32 : (uint64_t)lo; }
};

// Biased row exponent key from the largest |x| bit pattern of a row: 0 for an
// all-zero row; nonfinite entries set `bad`.  E is clamped below at 8S - 1076:
// a row whose largest entry is smaller holds only subnormals, which are exact
// integers at that scale (multiples of 2^-1074), so nothing is lost, and every
// entry then needs a right shift only (fixed_point).
template <int S>
__device__ __forceinline__ int32_t row_key(uint64_t ab, unsigned& bad) {
  if (ab == 0) return 0;
  if (ab >= 0x7FF0000000000000ull) {
    bad = 1;
    return 0;
  }
  const int ef = (int)(ab >> 52);
  const int e = ef != 0 ? ef - 1023 : (63 - __clzll((long long)ab)) - 1074;
  return max(e, 8 * S - 1076) + kExpBias;
}

// X = round(x * 2^(8S - 2 - E)), |X| <= 2^(8S-1), round half away from zero,
// given k0 = E + 1077 - 8S for the row (so that X = round(m * 2^-k) with
// k = k0 - max(e_f, 1) >= 0 for the integer mantissa m and exponent field
// e_f).  A zero row passes k0 >= 64 + 2047.  Selects only, no branches.
__device__ __forceinline__ int64_t fixed_point(double x, int k0) {
  const uint64_t bits = (uint64_t)__double_as_longlong(x);
  const int ef = (int)((bits >> 52) & 0x7FF);
  const uint64_t mant = (bits & ((1ull << 52) - 1)) | ((uint64_t)(ef != 0) << 52);
  const int k = min(k0 - max(ef, 1), 63);
  const uint64_t X = (mant + ((1ull << k) >> 1)) >> k;   // 0 once k >= 54
  const uint64_t sm = 0ull - (bits >> 63);               // all ones for a negative entry
  return (int64_t)((X ^ sm) - sm);
}

__device__ __forceinline__ int row_k0(int32_t key, int S) {
  return key == 0 ? 4096 : key - kExpBias + 1077 - 8 * S;
}

// Balanced base-256 digits by byte extraction: with B = 0x80 * (256^S - 1)/255,
// Y = X + B has bytes (a_k + 128) for the low S-1 digits and (a_top + 128) in
// [0, 256] above them (no carries: every shifted digit lies in [0, 255]).
__host__ __device__ constexpr uint64_t digit_bias(int S) {
  uint64_t b = 0;
  for (int k = 0; k < S; ++k) b |= (uint64_t)0x80 << (8 * k);
  return b;
}

// Slice i's value (a - 128) * 2^(-8 i) as a float, for the biased digit
// a + 128 held in byte k = S-1-i of y (the top digit, which may be 256, is
// everything above the low S-1 bytes).  The byte is moved under the exponent of
// 2^23 by one byte permute, giving the float 2^23 + u; one FMA then scales by
// 2^(-8 i) and subtracts (2^23 + 128) 2^(-8 i).  Product and sum are exact, so
// the result is exact (and +0 for a zero digit).
template <int S, int I>
__device__ __forceinline__ float digit_value(uint64_t y) {
  constexpr int k = S - 1 - I;
  uint32_t w;
  if (I == 0) {
    w = 0x4B000000u | (uint32_t)(y >> (8 * k));
  } else if (k < 4) {
    w = __byte_perm((uint32_t)y, 0x4B000000u, 0x7540 | k);
  } else {
    w = __byte_perm((uint32_t)(y >> 32), 0x4B000000u, 0x7540 | (k - 4));
  }
  const float scale = __int_as_float((127 - 8 * I) << 23);
  return __fmaf_rn(__uint_as_float(w), scale, -8388736.0f * scale);
}

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
  int64_t kpad;
  int parts;                 // column blocks of the exponent scan (prep_scan_parts)
  const double* src[2];      // U, V standard reduced forms
  void* dst[2];              // slices (split) or float32 operands (TF32)
  int32_t* exps[2];          // biased row exponents read by the GEMM
  int32_t* part[2];          // [parts][n_q * R] partial row maxima (parts > 1)
  bool fast_rows[2];
  bool pair_ok[2];           // column-contiguous with every offset of an even column even
  unsigned* err;
  unsigned* barrier;
  unsigned long long* zero64;  // split-K partial sums, zeroed here
  int64_t zero64_n;
  bool skip[2];              // operands prepared by the single-read kernel instead
};

__device__ __forceinline__ void operand_dims(const Problem& p, int op, int64_t* R, int64_t* Cn) {
  *R = op == 0 ? p.M : p.N;
  *Cn = p.K;
}

// Exponent scan of 32 rows over one column block: the offsets of up to
// kScanWidth columns at once, then the loads.
template <int S>
__device__ void scan_tile(const PrepArgs& a, int op, uint32_t tile, int64_t* roff, int64_t* coff,
                          unsigned long long* rmax) {
  const Problem& p = a.p;
  int64_t R, Cn;
  operand_dims(p, op, &R, &Cn);
  const int64_t* rtab = op == 0 ? a.t.urow : a.t.vrow;
  const int64_t* ctab = op == 0 ? a.t.ucol : a.t.vcol;
  const double* src = a.src[op];
  const bool fast_rows = a.fast_rows[op];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const uint32_t P = (uint32_t)a.parts;
  // column blocks start on multiples of 32 columns: the pair path loads two
  // adjacent columns with one 16-byte load, which needs an even first column
  // (a trailing block may be short or empty; an empty one writes key 0)
  const int64_t width = ((Cn + P - 1) / P + 31) / 32 * 32;
  const uint32_t rt = (uint32_t)((R + TILE - 1) / TILE);
  const uint32_t b = tile / (rt * P);
  const uint32_t rem = tile - b * rt * P;
  const int64_t r0 = (int64_t)(rem / P) * TILE;
  const uint32_t j = rem % P;
  const int64_t cb = j * width, ce = min(Cn, cb + width);
  __syncthreads();
  if (threadIdx.x < TILE) {
    const int64_t r = r0 + threadIdx.x;
    roff[threadIdx.x] = r < R ? rtab[(int64_t)b * R + r] : 0;
    rmax[threadIdx.x] = 0;
  }
  // general plans: an absent row (offset -1) or column reads as zero
  const bool masked = p.general != 0;
  constexpr int PER = SCAN_COLS / (THREADS / 32);
  constexpr int RPW = TILE / (THREADS / 32);   // rows per warp (column paths)
  Max2 mx;                  // fast rows: this thread's row (tx)
  Max2 mxr[RPW];            // column paths: this lane's share of its warp's rows
  for (int64_t sb = cb; sb < ce; sb += kScanWidth) {
    const int64_t se = min(ce, sb + kScanWidth);
#pragma unroll
    for (int i = 0; i < kScanWidth / THREADS; ++i) {
      const int64_t c = sb + threadIdx.x + i * THREADS;
      coff[threadIdx.x + i * THREADS] = c < se ? ctab[(int64_t)b * Cn + c] : 0;
    }
    __syncthreads();
    for (int64_t c0 = sb; c0 < se; c0 += SCAN_COLS) {
      const int64_t* co = coff + (c0 - sb);
      if (fast_rows) {
        // lanes walk rows (contiguous), warps walk columns
        const bool rok = r0 + tx < R && (!masked || roff[tx] >= 0);
        const double* rowp = src + (int64_t)p.es * roff[tx];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          double x[PER / 2];
#pragma unroll
          for (int i = 0; i < PER / 2; ++i) {
            const int cc = ty + (h * (PER / 2) + i) * (THREADS / 32);
            x[i] = (rok && c0 + cc < se && (!masked || co[cc] >= 0)) ? rowp[(int64_t)p.es * co[cc]] : 0.0;
          }
#pragma unroll
          for (int i = 0; i < PER / 2; ++i) mx.add(x[i]);
        }
      } else if (a.pair_ok[op]) {
        // lanes walk column pairs (16-byte loads), warps walk rows; per-row
        // maxima stay in registers until the end of the tile
#pragma unroll
        for (int h = 0; h < RPW; ++h) {
          const int rr = ty + h * (THREADS / 32);
          const bool rok = r0 + rr < R;
          const double* rowp = src + (int64_t)p.es * roff[rr];
          double2 x[SCAN_COLS / 64];
#pragma unroll
          for (int i = 0; i < SCAN_COLS / 64; ++i) {
            const int cc = 2 * tx + 64 * i;
            x[i] = (rok && c0 + cc < se) ? *reinterpret_cast<const double2*>(rowp + co[cc])
                                         : make_double2(0.0, 0.0);
          }
#pragma unroll
          for (int i = 0; i < SCAN_COLS / 64; ++i)
            mxr[h].add(x[i].x), mxr[h].add(x[i].y);
        }
      } else {
        // lanes walk columns (contiguous), warps walk rows
#pragma unroll
        for (int h = 0; h < RPW; ++h) {
          const int rr = ty + h * (THREADS / 32);
          const bool rok = r0 + rr < R && (!masked || roff[rr] >= 0);
          const double* rowp = src + (int64_t)p.es * roff[rr];
          double x[SCAN_COLS / 32];
#pragma unroll
          for (int i = 0; i < SCAN_COLS / 32; ++i) {
            const int cc = tx + 32 * i;
            x[i] = (rok && c0 + cc < se && (!masked || co[cc] >= 0)) ? rowp[(int64_t)p.es * co[cc]] : 0.0;
          }
#pragma unroll
          for (int i = 0; i < SCAN_COLS / 32; ++i) mxr[h].add(x[i]);
        }
      }
    }
    __syncthreads();
  }
  if (!fast_rows) {
#pragma unroll
    for (int h = 0; h < RPW; ++h) {
      Max2 v = mxr[h];
      for (int o = 16; o > 0; o >>= 1) v.merge_xor(o);
      if (tx == 0) rmax[ty + h * (THREADS / 32)] = v.pattern();   // row belongs to this warp alone
    }
  }
  // the max of the patterns is the pattern of the merged maxima
  if (fast_rows) atomicMax(&rmax[tx], (unsigned long long)mx.pattern());
  __syncthreads();
  if (threadIdx.x < TILE && r0 + threadIdx.x < R) {
    unsigned bad = 0;
    const int32_t key = row_key<S>(rmax[threadIdx.x], bad);
    if (bad) atomicOr(a.err, (unsigned)DEVERR_NONFINITE);
    int32_t* out = P > 1 ? a.part[op] + (int64_t)j * p.n_q * R : a.exps[op];
    out[(int64_t)b * R + r0 + threadIdx.x] = key;
  }
}

// Writes the S slices of two adjacent columns (c, c+1) of one row: one
// packed BF16 pair per slice (the conversion is exact, every digit value has
// at most 8 significant bits).
template <int S, int I = 0>
__device__ __forceinline__ void put_digits(uint64_t y0, uint64_t y1, uint32_t* dst, int64_t stride) {
  if constexpr (I < S) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(digit_value<S, I>(y0), digit_value<S, I>(y1));
    dst[(int64_t)I * stride] = *reinterpret_cast<const uint32_t*>(&h);
    put_digits<S, I + 1>(y0, y1, dst, stride);
  }
}

template <int S>
__device__ __forceinline__ void put_slices_pair(double x0, double x1, int k0, uint32_t* dst,
                                                int64_t stride) {
  const uint64_t y0 = (uint64_t)(fixed_point(x0, k0) + (int64_t)digit_bias(S));
  const uint64_t y1 = (uint64_t)(fixed_point(x1, k0) + (int64_t)digit_bias(S));
  put_digits<S>(y0, y1, dst, stride);
}

// Four adjacent columns of one row: per slice, four BF16 digits in one 8-byte
// store (dst and stride in units of uint2).
template <int S, int I = 0>
__device__ __forceinline__ void put_digits_quad(const uint64_t (&y)[4], uint2* dst, int64_t stride) {
  if constexpr (I < S) {
    const __nv_bfloat162 lo = __floats2bfloat162_rn(digit_value<S, I>(y[0]), digit_value<S, I>(y[1]));
    const __nv_bfloat162 hi = __floats2bfloat162_rn(digit_value<S, I>(y[2]), digit_value<S, I>(y[3]));
    dst[(int64_t)I * stride] =
        make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
    put_digits_quad<S, I + 1>(y, dst, stride);
  }
}

template <int S>
__device__ __forceinline__ void put_slices_quad(const double (&x)[4], int k0, uint2* dst, int64_t stride) {
  uint64_t y[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) y[j] = (uint64_t)(fixed_point(x[j], k0) + (int64_t)digit_bias(S));
  put_digits_quad<S>(y, dst, stride);
}

__device__ __forceinline__ float tf32_round(double x) {
  uint32_t u = __float_as_uint(__double2float_rn(x));
  if ((u & 0x7F800000u) != 0x7F800000u) u = (u + 0xFFFu + ((u >> 13) & 1u)) & ~0x1FFFu;
  return __uint_as_float(u);
}

template <int S>
__device__ __forceinline__ void put_pair(const PrepArgs& a, int op, double x0, double x1, int k0,
                                         int64_t e_at, int64_t slice_stride) {
  if constexpr (S > 0) {
    put_slices_pair<S>(x0, x1, k0, (uint32_t*)a.dst[op] + e_at / 2, slice_stride / 2);
  } else {
    float2 f;
    f.x = tf32_round(x0);
    f.y = tf32_round(x1);
    reinterpret_cast<float2*>(a.dst[op])[e_at / 2] = f;
  }
}

// One work unit of the padded aligned operand: 32 rows by SLICE_GROUP x 64
// columns (S slices; S = 0: the TF32 copy).  Column-contiguous operands are
// read along the columns straight from global memory (16-byte loads when every
// offset is even), row-contiguous ones go through shared memory, 64 columns at
// a time, so that both the gather and the slice stores are coalesced.  The row
// exponents are the maxima over the scan's column blocks; the units of the
// first column group store them for the GEMM.
template <int S>
__device__ void slice_unit(const PrepArgs& a, int op, uint32_t unit, int64_t* roff, int64_t* coff,
                           int32_t* rk0, double (*tilebuf)[SLICE_COLS + 1]) {
  constexpr int UCOLS = SLICE_GROUP * SLICE_COLS;
  const Problem& p = a.p;
  int64_t R, Cn;
  operand_dims(p, op, &R, &Cn);
  const int64_t kpad = a.kpad;
  const int64_t* rtab = op == 0 ? a.t.urow : a.t.vrow;
  const int64_t* ctab = op == 0 ? a.t.ucol : a.t.vcol;
  const double* src = a.src[op];
  const bool fast_rows = a.fast_rows[op];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const uint32_t rt = (uint32_t)((R + TILE - 1) / TILE), ct = (uint32_t)((kpad + UCOLS - 1) / UCOLS);
  const uint32_t b = unit / (rt * ct);
  const uint32_t rem = unit - b * rt * ct;
  const int64_t r0 = (int64_t)(rem / ct) * TILE, cu = (int64_t)(rem % ct) * UCOLS;
  const int64_t slice_stride = (int64_t)p.n_q * R * kpad;   // elements
  const int64_t brow = (int64_t)b * R;
  __syncthreads();
  if (threadIdx.x < TILE) {
    const int64_t r = r0 + threadIdx.x;
    roff[threadIdx.x] = r < R ? rtab[brow + r] : 0;
    if constexpr (S > 0) {
      int32_t key = 0;
      if (r < R) {
        if (a.parts > 1) {
          const int64_t nR = (int64_t)p.n_q * R;
          for (int j = 0; j < a.parts; ++j) key = max(key, a.part[op][j * nR + brow + r]);
          if (cu == 0) a.exps[op][brow + r] = key;
        } else {
          key = a.exps[op][brow + r];
        }
      }
      rk0[threadIdx.x] = row_k0(key, S);
    }
  } else if (fast_rows) {
    for (int i = threadIdx.x - TILE; i < UCOLS; i += THREADS - TILE) {
      const int64_t c = cu + i;
      coff[i] = c < Cn ? ctab[(int64_t)b * Cn + c] : 0;
    }
  }
  __syncthreads();
  if (!fast_rows && a.pair_ok[op]) {
    // lanes walk column pairs with 16-byte loads, warps walk rows; the column
    // offsets of all sub-tiles are loaded first, then two sub-tiles' data
    // (eight 16-byte loads per lane) go out before any of it is sliced
    int64_t co[SLICE_GROUP];
#pragma unroll
    for (int g = 0; g < SLICE_GROUP; ++g) {
      const int64_t c = cu + g * SLICE_COLS + 2 * tx;
      co[g] = c < Cn ? ctab[(int64_t)b * Cn + c] : 0;
    }
    constexpr int RPW = TILE / (THREADS / 32);
#pragma unroll
    for (int g0 = 0; g0 < SLICE_GROUP; g0 += 2) {
      double2 x[2][RPW];
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const int64_t c = cu + (g0 + g) * SLICE_COLS + 2 * tx;
#pragma unroll
        for (int rg = 0; rg < RPW; ++rg) {
          const int rr = ty + rg * (THREADS / 32);
          x[g][rg] = (c < Cn && r0 + rr < R)
                         ? *reinterpret_cast<const double2*>(src + (int64_t)p.es * roff[rr] + co[g0 + g])
                         : make_double2(0.0, 0.0);
        }
      }
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const int64_t c = cu + (g0 + g) * SLICE_COLS + 2 * tx;
        if (c >= kpad) continue;
#pragma unroll
        for (int rg = 0; rg < RPW; ++rg) {
          const int rr = ty + rg * (THREADS / 32);
          const int64_t r = r0 + rr;
          if (r >= R) continue;
          put_pair<S>(a, op, x[g][rg].x, x[g][rg].y, S > 0 ? rk0[rr] : 0, (brow + r) * kpad + c,
                      slice_stride);
        }
      }
    }
    return;
  }
  const bool masked = p.general != 0;   // absent rows/columns (offset -1) read as zero
  if (!fast_rows) {
    // lanes walk column pairs, warps walk rows; no shared-memory transpose
    const bool pair = a.pair_ok[op];
#pragma unroll 1
    for (int sub = 0; sub < SLICE_GROUP; ++sub) {
      const int64_t c = cu + sub * SLICE_COLS + 2 * tx;
      if (c >= kpad) break;
      int64_t co0 = 0, co1 = 0;
      if (c < Cn) co0 = ctab[(int64_t)b * Cn + c];
      if (!pair && c + 1 < Cn) co1 = ctab[(int64_t)b * Cn + c + 1];
#pragma unroll
      for (int rg = 0; rg < TILE / (THREADS / 32); ++rg) {
        const int rr = ty + rg * (THREADS / 32);
        const int64_t r = r0 + rr;
        if (r >= R) continue;
        const double* rowp = src + (int64_t)p.es * roff[rr];
        double x0 = 0.0, x1 = 0.0;
        if (pair) {
          if (c < Cn) {
            const double2 v2 = *reinterpret_cast<const double2*>(rowp + co0);
            x0 = v2.x;
            x1 = v2.y;
          }
        } else if (!masked || roff[rr] >= 0) {
          if (c < Cn && (!masked || co0 >= 0)) x0 = rowp[(int64_t)p.es * co0];
          if (c + 1 < Cn && (!masked || co1 >= 0)) x1 = rowp[(int64_t)p.es * co1];
        }
        put_pair<S>(a, op, x0, x1, S > 0 ? rk0[rr] : 0, (brow + r) * kpad + c, slice_stride);
      }
    }
    return;
  }
  const bool rok = r0 + tx < R && (!masked || roff[tx] >= 0);
  const double* rowp = src + (int64_t)p.es * roff[tx];
#pragma unroll 1
  for (int sub = 0; sub < SLICE_GROUP; ++sub) {
    const int64_t c0 = cu + sub * SLICE_COLS;
    if (c0 >= kpad) break;
    if (sub > 0) __syncthreads();   // the previous sub-tile's reads of tilebuf are done
    {
      double x[SLICE_COLS / (THREADS / 32)];
#pragma unroll
      for (int i = 0; i < SLICE_COLS / (THREADS / 32); ++i) {
        const int cc = ty + i * (THREADS / 32);
        const int64_t cof = coff[sub * SLICE_COLS + cc];
        x[i] = (rok && c0 + cc < Cn && (!masked || cof >= 0)) ? rowp[(int64_t)p.es * cof] : 0.0;
      }
#pragma unroll
      for (int i = 0; i < SLICE_COLS / (THREADS / 32); ++i) tilebuf[tx][ty + i * (THREADS / 32)] = x[i];
    }
    __syncthreads();
    // each thread: one row, two adjacent columns -> one uint32 per slice
#pragma unroll
    for (int rg = 0; rg < TILE / (THREADS / 32); ++rg) {
      const int rr = ty + rg * (THREADS / 32);
      const int64_t r = r0 + rr, c = c0 + 2 * tx;
      if (r >= R || c >= kpad) continue;
      put_pair<S>(a, op, tilebuf[rr][2 * tx], tilebuf[rr][2 * tx + 1], S > 0 ? rk0[rr] : 0,
                  (brow + r) * kpad + c, slice_stride);
    }
  }
}

// Operand preparation of one contraction in one cooperative launch (the
// offset tables are already in the workspace):
//   phase 1  zeroed split-K accumulators and (split form) the per-row
//            exponent maxima of U and V;
//   phase 2  BF16 slices (split) or TF32 copies of U and V.
template <int S>
__global__ void __launch_bounds__(THREADS, 4) prep_kernel(PrepArgs a) {
  __shared__ int64_t roff[TILE], coff[kScanWidth];
  __shared__ unsigned long long rmax[TILE];
  __shared__ int32_t rk0[TILE];
  __shared__ double tilebuf[TILE][SLICE_COLS + 1];
  const Problem& p = a.p;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t i = gtid; i < a.zero64_n; i += gthreads) a.zero64[i] = 0ull;
  if (S > 0) {
    const uint32_t tiles0 = a.skip[0] ? 0u : (uint32_t)(((p.M + TILE - 1) / TILE) * a.parts * p.n_q);
    const uint32_t tiles1 = a.skip[1] ? 0u : (uint32_t)(((p.N + TILE - 1) / TILE) * a.parts * p.n_q);
    for (uint32_t t = blockIdx.x; t < tiles0 + tiles1; t += gridDim.x) {
      const int op = t < tiles0 ? 0 : 1;
      scan_tile<S>(a, op, op == 0 ? t : t - tiles0, roff, coff, rmax);
    }
    grid_barrier(a.barrier, 1, a.err);
  }
  // the GEMM that consumes these operands may start its setup now
  asm volatile("griddepcontrol.launch_dependents;");
  {
    constexpr int UCOLS = SLICE_GROUP * SLICE_COLS;
    uint32_t units[2];
    for (int op = 0; op < 2; ++op) {
      int64_t R, Cn;
      operand_dims(p, op, &R, &Cn);
      units[op] = a.skip[op] ? 0u : (uint32_t)(((R + TILE - 1) / TILE) * ((a.kpad + UCOLS - 1) / UCOLS) * p.n_q);
    }
    for (uint32_t t = blockIdx.x; t < units[0] + units[1]; t += gridDim.x) {
      const int op = t < units[0] ? 0 : 1;
      slice_unit<S>(a, op, op == 0 ? t : t - units[0], roff, coff, rk0, tilebuf);
    }
  }
}

// ---------------------------------------------------------------------------
// Single-read operand preparation (split form).  The exponent of an aligned
// row must be known before any of its digits, so the two-phase kernel above
// reads each operand twice.  When a row is made of runs of L contiguous
// reduced-form entries (the column map's innermost block digits have
// unit-stride layout) and fits in shared memory, one CTA per SM instead
// streams whole rows into shared memory with bulk copies (one per run, on an
// mbarrier, up to kRsMaxBufs rows in flight), takes the row maximum there and writes
// the row's digits from there: every operand entry crosses HBM once.
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 512;
constexpr int kRsMaxBufs = 6;          // rows in flight per CTA (as shared memory allows)
constexpr size_t kRsSmem = 200 * 1024;  // shared memory for the row buffers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

struct RowStreamArgs {
  int64_t R, K, kpad, L;    // rows per batch, columns, padded columns, run length
  int n_q;
  const int64_t* rtab;      // [n_q][R] row offsets
  const int64_t* ctab;      // [n_q][K] column offsets (run starts read at multiples of L)
  const double* src;
  uint32_t* dst;            // BF16 digit pairs: [S][n_q][R][kpad / 2]
  int64_t slice_stride;     // n_q * R * kpad (elements)
  int32_t* exps;            // [n_q][R] biased row exponents
  unsigned* err;
  int nbuf;                 // row buffers (<= kRsMaxBufs)
  int64_t seg;              // cluster form: columns per CTA (rank r holds [r seg, (r+1) seg))
};

// Bounded wait on a bulk-copy barrier (about 2 s of SM clock); false on expiry.
__device__ __forceinline__ bool rs_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(100000u)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > 4000000000ll) return false;
  }
}

// Warp 0: queue the bulk copies of row g into buffer `slot` (lane 0 posts the
// byte count first; lanes then issue one run each, 32 at a time).
__device__ __forceinline__ void rs_issue(const RowStreamArgs& a, int64_t g, double* buf, uint64_t* bar,
                                         int lane) {
  const int64_t b = g / a.R;
  const int64_t roff = a.rtab[g];
  if (lane == 0)
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"((uint32_t)(a.K * 8))
                 : "memory");
  __syncwarp();
  const int64_t nruns = a.K / a.L;
  for (int64_t j = lane; j < nruns; j += 32) {
    const double* from = a.src + roff + a.ctab[b * a.K + j * a.L];
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(buf + j * a.L)),
        "l"(from), "r"((uint32_t)(a.L * 8)), "r"(smem_u32(bar))
        : "memory");
  }
}

// Maximum of the high words of a row (sign dropped: the exponent and the top
// 20 mantissa bits decide the row's scale whenever they are not all zero)
// into *m: a shared-memory atomic per warp.
__device__ __forceinline__ void rs_hi_max(const double* row, int64_t K, uint32_t* m, int tid, int lane) {
  const uint32_t* hw = reinterpret_cast<const uint32_t*>(row) + 1;
  uint32_t mh = 0;
#pragma unroll 4
  for (int64_t c = tid; c < K; c += RS_THREADS) mh = max(mh, hw[2 * c] & 0x7FFFFFFFu);
  for (int o = 16; o > 0; o >>= 1) mh = max(mh, __shfl_xor_sync(0xffffffffu, mh, o));
  if (lane == 0) atomicMax(m, mh);
}

// The row's scale from its high-word maximum m (read by every thread after a
// barrier, so the branch is uniform): all high words zero (a zero row, or
// entries below 2^-1042 only) takes the exact maximum of the whole bit
// patterns, with one more barrier.  Thread 0 stores the exponent.
template <int S>
__device__ __forceinline__ int rs_row_k0(const RowStreamArgs& a, const double* row, int64_t g, uint32_t m,
                                         unsigned long long* red, int tid, int warp, int lane) {
  uint64_t ab = (uint64_t)m << 32;
  if (m == 0) {
    uint64_t mx = 0;
    for (int64_t c = tid; c < a.K; c += RS_THREADS) mx = max(mx, abs_bits(row[c]));
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    for (int w = 0; w < RS_THREADS / 32; ++w) ab = max(ab, (uint64_t)red[w]);
  }
  unsigned bad = 0;
  const int32_t key = row_key<S>(ab, bad);
  if (tid == 0) {
    if (bad) atomicOr(a.err, (unsigned)DEVERR_NONFINITE);
    a.exps[g] = key;
  }
  return row_k0(key, S);
}

// Software-pipelined over the CTA's rows: iteration i writes the digits of
// row i and takes the maximum of row i + 1 (whose copy was queued nbuf - 1
// rows earlier), then one barrier frees row i's buffer for its refill and
// publishes row i + 1's maximum.  The maxima rotate over three shared words,
// each cleared two barriers before its next use.
template <int S>
__global__ void __launch_bounds__(RS_THREADS, 1) rowstream_kernel(const __grid_constant__ RowStreamArgs a) {
  extern __shared__ __align__(128) uint8_t rs_smem[];
  __shared__ __align__(8) uint64_t bars[kRsMaxBufs];
  __shared__ unsigned long long red[RS_THREADS / 32];
  __shared__ uint32_t mxs[3];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t buf_elems = (a.K + 15) / 16 * 16;   // 128-byte aligned buffers
  double* bufs = (double*)rs_smem;
  const int64_t rows = (int64_t)a.n_q * a.R;
  const int nbuf = a.nbuf;
  if (tid == 0) {
    for (int i = 0; i < nbuf; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 3) mxs[tid] = 0u;
  __syncthreads();
  if (warp == 0)
    for (int s = 0; s < nbuf; ++s) {
      const int64_t g = blockIdx.x + (int64_t)s * gridDim.x;
      if (g < rows) rs_issue(a, g, bufs + s * buf_elems, &bars[s], lane);
    }
  int64_t g = blockIdx.x;
  int it = 0;
  bool abort = false;
  int first_pending = 0;   // on abort: the first row whose copy may be in flight
  int k0 = 0;
  if (g < rows) {
    // row 0's maximum
    const bool ok = rs_wait(&bars[0], 0u);
    if (ok) rs_hi_max(bufs, a.K, &mxs[0], tid, lane);
    if (!ok && lane == 0) atomicOr(a.err, (unsigned)DEVERR_TIMEOUT);
    abort = __syncthreads_or(!ok);
    if (!abort) k0 = rs_row_k0<S>(a, bufs, g, *(volatile uint32_t*)&mxs[0], red, tid, warp, lane);
  }
  for (; !abort && g < rows; g += gridDim.x, ++it) {
    const int slot = it % nbuf;
    const double* row = bufs + slot * buf_elems;
    // the digits of row it, four adjacent columns per thread and step (zeros
    // beyond K)
    uint2* d = reinterpret_cast<uint2*>(a.dst) + g * (a.kpad / 4);
    for (int64_t q = tid; q < a.kpad / 4; q += RS_THREADS) {
      const int64_t c = 4 * q;
      double x[4];
      if (c + 4 <= a.K) {
        const double2 v0 = *reinterpret_cast<const double2*>(row + c);
        const double2 v1 = *reinterpret_cast<const double2*>(row + c + 2);
        x[0] = v0.x, x[1] = v0.y, x[2] = v1.x, x[3] = v1.y;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) x[e] = c + e < a.K ? row[c + e] : 0.0;
      }
      put_slices_quad<S>(x, k0, d + q, a.slice_stride / 4);
    }
    // the maximum of row it + 1
    const int64_t g1 = g + gridDim.x;
    const int slot1 = (it + 1) % nbuf;
    bool ok = true;
    if (g1 < rows) {
      ok = rs_wait(&bars[slot1], (uint32_t)((it + 1) / nbuf) & 1u);
      if (ok) rs_hi_max(bufs + slot1 * buf_elems, a.K, &mxs[(it + 1) % 3], tid, lane);
      if (!ok && lane == 0) atomicOr(a.err, (unsigned)DEVERR_TIMEOUT);
    }
    // row it's buffer is free; row it + 1's maximum is complete
    abort = __syncthreads_or(!ok);
    if (abort) {
      first_pending = it + 1;
      break;
    }
    if (tid == 0) mxs[it % 3] = 0u;   // row it + 3 collects here, after the next barrier
    const int64_t gn = g + (int64_t)nbuf * gridDim.x;
    if (warp == 0 && gn < rows) rs_issue(a, gn, bufs + slot * buf_elems, &bars[slot], lane);
    if (g1 < rows)
      k0 = rs_row_k0<S>(a, bufs + slot1 * buf_elems, g1, *(volatile uint32_t*)&mxs[(it + 1) % 3], red, tid,
                        warp, lane);
  }
  // the GEMM behind this kernel may start its launch
  asm volatile("griddepcontrol.launch_dependents;");
  if (abort && tid == 0) {
    // let the copies still in flight land before the CTA exits (bounded)
    for (int k = first_pending; k < it + nbuf; ++k) {
      const int64_t gk = blockIdx.x + (int64_t)k * gridDim.x;
      if (gk >= rows) break;
      rs_wait(&bars[k % nbuf], (uint32_t)(k / nbuf) & 1u);
    }
  }
}

// ---------------------------------------------------------------------------
// Rows longer than one CTA's shared memory (K > kRowStreamMaxK): a cluster of C
// CTAs holds each row, CTA r its columns [r seg, (r+1) seg).  Each CTA streams
// its segment with bulk copies (the run pieces inside the segment), takes the
// maximum of its high words, and the cluster barrier lets every CTA read the
// other segments' maxima from distributed shared memory: the row's scale is
// the same in every CTA, each writes the digits of its own segment, and every
// entry crosses HBM once.  Pipelined like the one-CTA kernel (the digits of
// row i and the maxima of row i + 1 between one cluster barrier); a failed
// copy wait is published in the same rotating slots, so the whole cluster
// leaves the loop together.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cl_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// a 32-bit / 64-bit word of CTA `rank`'s shared memory at this CTA's address of it
__device__ __forceinline__ uint32_t cl_ld32(const void* p, uint32_t rank) {
  uint32_t v;
  asm volatile(
      "{\n\t.reg .b32 ra;\n\tmapa.shared::cluster.u32 ra, %1, %2;\n\t"
      "ld.shared::cluster.u32 %0, [ra];\n\t}\n"
      : "=r"(v)
      : "r"(smem_u32(p)), "r"(rank)
      : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long cl_ld64(const void* p, uint32_t rank) {
  unsigned long long v;
  asm volatile(
      "{\n\t.reg .b32 ra;\n\tmapa.shared::cluster.u32 ra, %1, %2;\n\t"
      "ld.shared::cluster.u64 %0, [ra];\n\t}\n"
      : "=l"(v)
      : "r"(smem_u32(p)), "r"(rank)
      : "memory");
  return v;
}

// Warp 0: the bulk copies of row g's columns [s0, s1) into buf (the pieces of
// the runs of L contiguous entries that overlap the segment).
__device__ __forceinline__ void cl_issue(const RowStreamArgs& a, int64_t g, int64_t s0, int64_t s1, double* buf,
                                         uint64_t* bar, int lane) {
  const int64_t b = g / a.R;
  const int64_t roff = a.rtab[g];
  if (lane == 0)
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"((uint32_t)((s1 - s0) * 8))
                 : "memory");
  __syncwarp();
  for (int64_t j = s0 / a.L + lane; j * a.L < s1; j += 32) {
    const int64_t c0 = max(j * a.L, s0), c1 = min((j + 1) * a.L, s1);
    const double* from = a.src + roff + a.ctab[b * a.K + j * a.L] + (c0 - j * a.L);
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(buf + (c0 - s0))),
        "l"(from), "r"((uint32_t)((c1 - c0) * 8)), "r"(smem_u32(bar))
        : "memory");
  }
}

// Warp 0 reads slot x's maximum and copy-failure flag of every CTA of the
// cluster (one remote load per lane) and leaves their maximum and OR in
// this CTA's shared memory for all its threads (after the CTA barrier).
__device__ __forceinline__ void cl_gather(const uint32_t* mx, const uint32_t* fl, uint32_t C, int warp, int lane,
                                          uint32_t* gm, uint32_t* gf) {
  if (warp == 0) {
    uint32_t m = 0u, f = 0u;
    if ((uint32_t)lane < C) {
      m = cl_ld32(mx, (uint32_t)lane);
      f = cl_ld32(fl, (uint32_t)lane);
    }
    for (int o = 16; o > 0; o >>= 1) {
      m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
      f |= __shfl_xor_sync(0xffffffffu, f, o);
    }
    if (lane == 0) *gm = m, *gf = f;
  }
  __syncthreads();
}

// The row's scale from the cluster's high-word maximum m (the same in every
// CTA, so the branch is uniform); m = 0: the exact maximum of the whole bit
// patterns, exchanged through red64 with one more cluster barrier.  CTA 0
// stores the exponent.
template <int S>
__device__ __forceinline__ int cl_row_k0(const RowStreamArgs& a, const double* seg_buf, int64_t n, int64_t g,
                                         uint32_t m, unsigned long long* redw, unsigned long long* red64,
                                         uint32_t C, uint32_t rank, int tid, int warp, int lane) {
  uint64_t ab = (uint64_t)m << 32;
  if (m == 0) {
    uint64_t mx = 0;
    for (int64_t c = tid; c < n; c += RS_THREADS) mx = max(mx, abs_bits(seg_buf[c]));
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)mx, o));
    if (lane == 0) redw[warp] = mx;
    __syncthreads();
    if (tid == 0) {
      uint64_t v = 0;
      for (int w = 0; w < RS_THREADS / 32; ++w) v = max(v, (uint64_t)redw[w]);
      *red64 = v;
    }
    cl_sync();
    if (warp == 0) {
      uint64_t v = (uint32_t)lane < C ? (uint64_t)cl_ld64(red64, (uint32_t)lane) : 0ull;
      for (int o = 16; o > 0; o >>= 1) v = max(v, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)v, o));
      if (lane == 0) redw[0] = v;
    }
    __syncthreads();
    ab = max(ab, (uint64_t)redw[0]);
  }
  unsigned bad = 0;
  const int32_t key = row_key<S>(ab, bad);
  if (rank == 0 && tid == 0) {
    if (bad) atomicOr(a.err, (unsigned)DEVERR_NONFINITE);
    a.exps[g] = key;
  }
  return row_k0(key, S);
}

template <int S>
__global__ void __launch_bounds__(RS_THREADS, 1) rowcluster_kernel(const __grid_constant__ RowStreamArgs a) {
  extern __shared__ __align__(128) uint8_t rs_smem[];
  __shared__ __align__(8) uint64_t bars[kRsMaxBufs];
  __shared__ unsigned long long redw[RS_THREADS / 32];
  __shared__ unsigned long long red64;
  __shared__ uint32_t mxs[3];
  __shared__ uint32_t flg[3];
  __shared__ uint32_t gm, gf;   // the cluster's maximum and failure flag of the slot just gathered
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t C = cl_size(), rank = cl_rank();
  const int64_t cid = blockIdx.x / C, ncl = gridDim.x / C;
  const int64_t s0 = (int64_t)rank * a.seg, s1 = min(a.K, s0 + a.seg);
  const int64_t n = s1 > s0 ? s1 - s0 : 0;                  // this CTA's columns of a row
  const int64_t q0 = s0 / 4, q1 = rank == C - 1 ? a.kpad / 4 : s1 / 4;   // its digit quads
  const int64_t buf_elems = (a.seg + 15) / 16 * 16;
  double* bufs = (double*)rs_smem;
  const int64_t rows = (int64_t)a.n_q * a.R;
  const int nbuf = a.nbuf;
  if (tid == 0) {
    for (int i = 0; i < nbuf; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < 3) mxs[tid] = 0u, flg[tid] = 0u;
  cl_sync();
  if (warp == 0 && n > 0)
    for (int s = 0; s < nbuf; ++s) {
      const int64_t g = cid + (int64_t)s * ncl;
      if (g < rows) cl_issue(a, g, s0, s1, bufs + s * buf_elems, &bars[s], lane);
    }
  int64_t g = cid;
  int it = 0;
  bool abort = false;
  int first_pending = 0;
  int k0 = 0;
  if (g < rows) {
    const bool ok = n == 0 || rs_wait(&bars[0], 0u);
    if (ok && n > 0) rs_hi_max(bufs, n, &mxs[0], tid, lane);
    if (!ok) flg[0] = 1u;
    cl_sync();
    cl_gather(&mxs[0], &flg[0], C, warp, lane, &gm, &gf);
    abort = gf != 0u;
    if (abort) {
      if (tid == 0 && !ok) atomicOr(a.err, (unsigned)DEVERR_TIMEOUT);
    } else {
      k0 = cl_row_k0<S>(a, bufs, n, g, gm, redw, &red64, C, rank, tid, warp, lane);
    }
  }
  for (; !abort && g < rows; g += ncl, ++it) {
    const int slot = it % nbuf;
    const double* row = bufs + slot * buf_elems;
    // the digits of this CTA's segment of row it (the last CTA also writes the
    // zero digits of the padding columns K..kpad-1)
    uint2* d = reinterpret_cast<uint2*>(a.dst) + g * (a.kpad / 4);
    for (int64_t q = q0 + tid; q < q1; q += RS_THREADS) {
      const int64_t c = 4 * q;
      double x[4];
      if (c + 4 <= s1) {
        const double2 v0 = *reinterpret_cast<const double2*>(row + (c - s0));
        const double2 v1 = *reinterpret_cast<const double2*>(row + (c - s0) + 2);
        x[0] = v0.x, x[1] = v0.y, x[2] = v1.x, x[3] = v1.y;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) x[e] = c + e < s1 ? row[c + e - s0] : 0.0;
      }
      put_slices_quad<S>(x, k0, d + q, a.slice_stride / 4);
    }
    // the maxima of row it + 1
    const int64_t g1 = g + ncl;
    const int slot1 = (it + 1) % nbuf;
    bool ok = true;
    if (g1 < rows && n > 0) {
      ok = rs_wait(&bars[slot1], (uint32_t)((it + 1) / nbuf) & 1u);
      if (ok) rs_hi_max(bufs + slot1 * buf_elems, n, &mxs[(it + 1) % 3], tid, lane);
      if (!ok) flg[(it + 1) % 3] = 1u;
    }
    // row it's buffers are free in every CTA; row it + 1's maxima are complete
    cl_sync();
    cl_gather(&mxs[(it + 1) % 3], &flg[(it + 1) % 3], C, warp, lane, &gm, &gf);
    if (gf != 0u) {
      if (tid == 0 && !ok) atomicOr(a.err, (unsigned)DEVERR_TIMEOUT);
      abort = true;
      first_pending = it + 1;
      break;
    }
    // row it + 3 collects in slot it % 3, after the next cluster barrier
    if (tid == 0) mxs[it % 3] = 0u, flg[it % 3] = 0u;
    const int64_t gn = g + (int64_t)nbuf * ncl;
    if (warp == 0 && n > 0 && gn < rows) cl_issue(a, gn, s0, s1, bufs + slot * buf_elems, &bars[slot], lane);
    if (g1 < rows) k0 = cl_row_k0<S>(a, bufs + slot1 * buf_elems, n, g1, gm, redw, &red64, C, rank, tid, warp, lane);
  }
  // the GEMM behind this kernel may start its launch
  asm volatile("griddepcontrol.launch_dependents;");
  if (abort && tid == 0 && n > 0) {
    // let this CTA's copies still in flight land (bounded)
    for (int k = first_pending; k < it + nbuf; ++k) {
      const int64_t gk = cid + (int64_t)k * ncl;
      if (gk >= rows) break;
      rs_wait(&bars[k % nbuf], (uint32_t)(k / nbuf) & 1u);
    }
  }
  // no CTA leaves while another may still read its shared memory
  cl_sync();
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

// ---------------------------------------------------------------------------
// Single-read preparation of short rows (split form, K <= kRowTileMaxK).  One
// CTA holds 2^rlog whole aligned rows in shared memory: it gathers them once
// (consecutive threads on consecutive rows when the rows are the reduced form's
// unit-stride side, else on consecutive columns), takes each row's maximum
// there and writes the row's digits from there.  No grid barrier: the
// operands' preparation is one plain launch.
// ---------------------------------------------------------------------------
constexpr int RT_THREADS = 512;

// 8-byte asynchronous copy global -> shared; src_bytes 0 fills zeros (reads nothing)
__device__ __forceinline__ void cp_async8(void* dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}

struct RowTileArgs {
  Problem p;
  Tables t;
  int64_t kpad;
  int rlog;                  // rows per CTA = 2^rlog
  uint32_t units[2];         // (irrep, row block) units of U and of V (0: not prepared here)
  const double* src[2];
  uint32_t* dst[2];          // BF16 digit pairs: [S][n_q][R][kpad / 2]
  int32_t* exps[2];          // [n_q][R] biased row exponents
  bool fast_rows[2];
  size_t buf_off;            // byte offset of the row buffer in shared memory
  unsigned* err;
  unsigned long long* zero64;  // split-K partial sums, zeroed here
  int64_t zero64_n;
};

template <int S>
__global__ void __launch_bounds__(RT_THREADS) rowtile_kernel(const __grid_constant__ RowTileArgs a) {
  extern __shared__ __align__(16) uint8_t rt_smem[];
  const Problem& p = a.p;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int R = 1 << a.rlog;
  const int Kc = (int)p.K;
  const int kpad = (int)a.kpad;
  // row pitch kpad + 2 doubles: 16-byte aligned pairs for the digit pass, and
  // row-strided stores of the gather spread over the banks
  const int LD = kpad + 2;
  int64_t* coff = (int64_t*)rt_smem;
  int64_t* roff = coff + Kc;
  unsigned long long* rmx = (unsigned long long*)(roff + R);
  int32_t* rk0 = (int32_t*)(rmx + R);
  // index split j = r * n + c by a float reciprocal: exact while j / n <= 64
  // and n <= 4096 (the error, below 2^-17, stays under the 0.5 / n margin)
  const float inv_q = 1.0f / (float)(kpad >> 2);
  // row walks over columns: wpr warps per row when R < 16, else a warp per row
  constexpr int NW = RT_THREADS / 32;
  const int wpr = R < NW ? NW / R : 1;
  const int sub = warp % wpr;
  double* buf = (double*)(rt_smem + a.buf_off);
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + tid; i < a.zero64_n; i += gthreads) a.zero64[i] = 0ull;
  // every CTA of this grid is resident once all have passed here: the GEMM
  // behind it may start its setup
  asm volatile("griddepcontrol.launch_dependents;");
  const uint32_t total = a.units[0] + a.units[1];
  for (uint32_t unit = blockIdx.x; unit < total; unit += gridDim.x) {
    const int op = unit < a.units[0] ? 0 : 1;
    const uint32_t un = op == 0 ? unit : unit - a.units[0];
    const int64_t Rtot = op == 0 ? p.M : p.N;
    const uint32_t rblocks = (uint32_t)((Rtot + R - 1) >> a.rlog);
    const uint32_t b = un / rblocks;
    const int64_t r0 = (int64_t)(un - b * rblocks) << a.rlog;
    const int64_t* rtab = (op == 0 ? a.t.urow : a.t.vrow) + (int64_t)b * Rtot;
    const int64_t* ctab = (op == 0 ? a.t.ucol : a.t.vcol) + (int64_t)b * Kc;
    const double* src = a.src[op];
    __syncthreads();   // the previous unit is done with shared memory
    // offsets, then the rows: asynchronous 8-byte copies into shared memory,
    // every copy of a thread in flight at once (an absent row or column,
    // offset -1 in general plans, and rows past the end are zero-filled)
    for (int k = tid; k < Kc; k += RT_THREADS) cp_async8(coff + k, ctab + k, 8u);
    for (int r = tid; r < R; r += RT_THREADS) {
      if (r0 + r < Rtot) cp_async8(roff + r, rtab + r0 + r, 8u);
      else roff[r] = -1;
      rmx[r] = 0ull;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (a.fast_rows[op]) {
      // consecutive threads on consecutive rows (the unit-stride side); a
      // thread keeps one row (R divides the block) and walks its columns
      const int r = tid & (R - 1);
      const int64_t ro = roff[r];
      const double* rowp = src + (ro >= 0 ? ro : 0);
      double* brow = buf + r * LD;
#pragma unroll 4
      for (int k = tid >> a.rlog; k < Kc; k += RT_THREADS >> a.rlog) {
        const int64_t co = coff[k];
        const bool ok = ro >= 0 && co >= 0;
        cp_async8(brow + k, ok ? rowp + co : src, ok ? 8u : 0u);
      }
    } else {
      // lanes on consecutive columns, wpr warps per row
      for (int r = warp / wpr; r < R; r += NW / wpr) {
        const int64_t ro = roff[r];
        const double* rowp = src + (ro >= 0 ? ro : 0);
        double* brow = buf + r * LD;
#pragma unroll 4
        for (int k = sub * 32 + lane; k < Kc; k += 32 * wpr) {
          const int64_t co = coff[k];
          const bool ok = ro >= 0 && co >= 0;
          cp_async8(brow + k, ok ? rowp + co : src, ok ? 8u : 0u);
        }
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    // row maxima over the high words (sign dropped: the exponent and the top
    // 20 mantissa bits decide the row's scale whenever they are not all zero)
    for (int r = warp / wpr; r < R; r += NW / wpr) {
      const uint32_t* hw = reinterpret_cast<const uint32_t*>(buf + r * LD) + 1;
      uint32_t m = 0;
#pragma unroll 4
      for (int k = sub * 32 + lane; k < Kc; k += 32 * wpr) m = max(m, hw[2 * k] & 0x7FFFFFFFu);
      for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) atomicMax(&rmx[r], (unsigned long long)m << 32);
    }
    __syncthreads();
    // rows whose high words are all zero (zero rows, or entries below 2^-1042
    // only): the exact maximum of the whole bit patterns
    for (int r = warp / wpr; r < R; r += NW / wpr) {
      if (rmx[r] != 0ull) continue;
      uint64_t m = 0;
      for (int k = sub * 32 + lane; k < Kc; k += 32 * wpr) m = max(m, abs_bits(buf[r * LD + k]));
      for (int o = 16; o > 0; o >>= 1)
        m = max(m, (uint64_t)__shfl_xor_sync(0xffffffffu, (unsigned long long)m, o));
      if (lane == 0 && m != 0) atomicMax(&rmx[r], (unsigned long long)m);
    }
    __syncthreads();
    for (int r = tid; r < R; r += RT_THREADS) {
      unsigned bad = 0;
      const int32_t key = row_key<S>(rmx[r], bad);
      if (bad) atomicOr(a.err, (unsigned)DEVERR_NONFINITE);
      if (r0 + r < Rtot) a.exps[op][(int64_t)b * Rtot + r0 + r] = key;
      rk0[r] = row_k0(key, S);
    }
    __syncthreads();
    // digits: consecutive threads on consecutive groups of four columns of a
    // row (the padding columns K..kpad-1 get zero digits)
    const int Q4 = kpad >> 2;
    const int64_t sstride = (int64_t)p.n_q * Rtot * Q4;   // uint2 quads per slice
    uint2* dst = reinterpret_cast<uint2*>(a.dst[op]) + ((int64_t)b * Rtot + r0) * Q4;
    const int rows_here = (int)min((int64_t)R, Rtot - r0);
    for (int j = tid; j < rows_here * Q4; j += RT_THREADS) {
      const int r = __float2int_rz(((float)j + 0.5f) * inv_q);
      const int c = 4 * (j - r * Q4);
      const double2* at = reinterpret_cast<const double2*>(buf + r * LD + c);
      double x[4];
      if (c + 4 <= Kc) {
        const double2 v0 = at[0], v1 = at[1];
        x[0] = v0.x, x[1] = v0.y, x[2] = v1.x, x[3] = v1.y;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) x[e] = c + e < Kc ? buf[r * LD + c + e] : 0.0;
      }
      put_slices_quad<S>(x, rk0[r], dst + j, sstride);
    }
  }
}

}  // namespace

int rowtile_rows_log2(int64_t kpad) {
  int rl = 0;
  while (rl < 6 && ((kpad << (rl + 1)) <= kRowTileElems)) ++rl;   // K = 4096: 2 rows
  return rl;
}

// column offsets, row offsets, row maxima, row scale keys, then the rows
static size_t rowtile_head_bytes(int64_t K, int64_t R) {
  return ((size_t)(K + 2 * R) * 8 + (size_t)R * 4 + 15) / 16 * 16;
}

size_t rowtile_smem_bytes(int64_t K, int64_t kpad) {
  const int64_t R = (int64_t)1 << rowtile_rows_log2(kpad);
  return rowtile_head_bytes(K, R) + (size_t)R * (kpad + 2) * 8;
}

cudaError_t launch_rowtile(const Problem& p, const Tables& t, int n_slices, const bool* on,
                           const double* u, const double* v, void* ua, void* va, int32_t* eu,
                           int32_t* ev, int64_t kpad, unsigned* err, unsigned long long* zero64,
                           int64_t zero64_n, cudaStream_t st) {
  if (n_slices < 1 || n_slices > kMaxSlices || p.es != 1 || p.K < 1 || kpad > kRowTileMaxK ||
      kpad % 32 != 0 || kpad < p.K)
    return cudaErrorInvalidValue;
  void (*kern)(RowTileArgs) = nullptr;
  switch (n_slices) {
    case 1: kern = rowtile_kernel<1>; break;
    case 2: kern = rowtile_kernel<2>; break;
    case 3: kern = rowtile_kernel<3>; break;
    case 4: kern = rowtile_kernel<4>; break;
    case 5: kern = rowtile_kernel<5>; break;
    default: kern = rowtile_kernel<6>; break;
  }
  RowTileArgs a;
  a.p = p;
  a.t = t;
  a.kpad = kpad;
  a.rlog = rowtile_rows_log2(kpad);
  const int64_t R = (int64_t)1 << a.rlog;
  const int64_t units[2] = {on[0] ? (int64_t)p.n_q * ((p.M + R - 1) / R) : 0,
                            on[1] ? (int64_t)p.n_q * ((p.N + R - 1) / R) : 0};
  if (units[0] + units[1] > 0x7FFFFFFFll) return cudaErrorInvalidValue;
  a.units[0] = (uint32_t)units[0];
  a.units[1] = (uint32_t)units[1];
  a.src[0] = u;
  a.src[1] = v;
  a.dst[0] = (uint32_t*)ua;
  a.dst[1] = (uint32_t*)va;
  a.exps[0] = eu;
  a.exps[1] = ev;
  a.fast_rows[0] = rows_fast(p.u);
  a.fast_rows[1] = rows_fast(p.v);
  a.buf_off = rowtile_head_bytes(p.K, R);
  a.err = err;
  a.zero64 = zero64;
  a.zero64_n = zero64_n;
  const size_t smem = rowtile_smem_bytes(p.K, kpad);
  // the attribute and the occupancy are taken once per instance and device
  // (kept per host thread)
  thread_local size_t set_for[kMaxSlices + 1][16] = {};
  thread_local int resident[kMaxSlices + 1][16] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 16) return cudaErrorInvalidDevice;
  if (set_for[n_slices][dev] < smem) {
    e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    set_for[n_slices][dev] = smem;
    resident[n_slices][dev] = 0;
  }
  if (resident[n_slices][dev] == 0) {
    int sms = 0, per = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, RT_THREADS, smem);
    if (e != cudaSuccess) return e;
    resident[n_slices][dev] = sms * (per > 0 ? per : 1);
  }
  const int64_t work = units[0] + units[1];
  const int64_t zero_ctas = (zero64_n + RT_THREADS - 1) / RT_THREADS;
  int64_t grid = work > 0 ? work : (zero_ctas > 0 ? zero_ctas : 1);
  if (grid > resident[n_slices][dev]) grid = resident[n_slices][dev];
  kern<<<(unsigned)grid, RT_THREADS, smem, st>>>(a);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_fill_zero(double* w, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  fill_zero_kernel<<<grid_for(blocks), 256, 0, st>>>(w, n);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_align_f64(const Problem& p, int operand, int direction, const double* src,
                             double* dst, const Tables* t, cudaStream_t st) {
  int64_t R, Cn;
  operand_extent(p, operand, &R, &Cn);
  if (R == 0 || Cn == 0 || p.n_q == 0) return cudaSuccess;
  const OperandMap& m = operand_map(p, operand);
  const int64_t* rtab = t ? (operand == 0 ? t->urow : operand == 1 ? t->vrow : t->wrow) : nullptr;
  const int64_t* ctab = t ? (operand == 0 ? t->ucol : operand == 1 ? t->vcol : t->wcol) : nullptr;
  int64_t tiles = ((R + TILE - 1) / TILE) * ((Cn + TILE - 1) / TILE) * p.n_q;
  align_kernel<<<grid_for(tiles), THREADS, 0, st>>>(p, m, R, Cn, direction, rows_fast(m), rtab, ctab,
                                                     src, dst);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_rowstream(const Problem& p, const Tables& t, int op, int n_slices, int64_t run,
                             const double* src, void* slices, int32_t* exps, int64_t kpad,
                             unsigned* err, cudaStream_t st) {
  if (n_slices < 2 || n_slices > kMaxSlices || p.es != 1 || p.general) return cudaErrorInvalidValue;
  const int64_t R = op == 0 ? p.M : p.N, K = p.K;
  if (run <= 0 || K % run != 0 || (run * 8) % 16 != 0 || K > kRowClusterMaxK) return cudaErrorInvalidValue;
  // rows beyond one CTA's buffers: clusters of C CTAs, CTA r holding columns
  // [r seg, (r+1) seg) (seg a multiple of 4, so every piece of a run stays even)
  const int C = (int)((K + kRowStreamMaxK - 1) / kRowStreamMaxK);
  const int64_t seg = C > 1 ? ((K + C - 1) / C + 3) / 4 * 4 : K;
  void (*kern)(RowStreamArgs) = nullptr;
  switch (n_slices) {
    case 2: kern = C > 1 ? rowcluster_kernel<2> : rowstream_kernel<2>; break;
    case 3: kern = C > 1 ? rowcluster_kernel<3> : rowstream_kernel<3>; break;
    case 4: kern = C > 1 ? rowcluster_kernel<4> : rowstream_kernel<4>; break;
    case 5: kern = C > 1 ? rowcluster_kernel<5> : rowstream_kernel<5>; break;
    default: kern = C > 1 ? rowcluster_kernel<6> : rowstream_kernel<6>; break;
  }
  const size_t row_bytes = (size_t)((seg + 15) / 16 * 16) * sizeof(double);
  int nbuf = (int)(kRsSmem / row_bytes);
  if (nbuf > kRsMaxBufs) nbuf = kRsMaxBufs;
  if (nbuf < 2) return cudaErrorInvalidValue;
  const size_t smem = (size_t)nbuf * row_bytes;
  // the attribute is set once per instance and device (kept per host thread)
  thread_local size_t set_for[2][kMaxSlices + 1][16] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 16) return cudaErrorInvalidDevice;
  if (set_for[C > 1][n_slices][dev] < smem) {
    e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    set_for[C > 1][n_slices][dev] = smem;
  }
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  RowStreamArgs a;
  a.R = R;
  a.K = K;
  a.kpad = kpad;
  a.L = run;
  a.n_q = p.n_q;
  a.rtab = op == 0 ? t.urow : t.vrow;
  a.ctab = op == 0 ? t.ucol : t.vcol;
  a.src = src;
  a.dst = (uint32_t*)slices;
  a.slice_stride = (int64_t)p.n_q * R * kpad;
  a.exps = exps;
  a.err = err;
  a.nbuf = nbuf;
  a.seg = seg;
  const int64_t rows = (int64_t)p.n_q * R;
  if (C == 1) {
    const int grid = (int)(rows < sms ? (rows > 0 ? rows : 1) : sms);
    kern<<<grid, RS_THREADS, smem, st>>>(a);
    ++g_kernel_launches;
    return cudaGetLastError();
  }
  // as many clusters as can be resident at once (a persistent loop over the
  // rows, each row in one cluster): clusters that had to wait for a second wave
  // would finish their rows after the rest
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(RS_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  thread_local int resident[kMaxSlices + 1][9][16] = {};
  int& res = resident[n_slices][C][dev];
  if (res == 0) {
    cfg.gridDim = dim3((unsigned)((sms / C) * C));
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, (const void*)kern, &cfg);
    if (e != cudaSuccess) return e;
    res = n > 0 ? n : 1;
  }
  int64_t clusters = res;
  if (clusters > rows) clusters = rows > 0 ? rows : 1;
  cfg.gridDim = dim3((unsigned)(clusters * C));
  e = cudaLaunchKernelEx(&cfg, kern, a);
  ++g_kernel_launches;
  return e;
}

cudaError_t launch_prep(const Problem& p, const Tables& t, bool split, int n_slices,
                        const double* u, const double* v, void* ua, void* va, int32_t* eu,
                        int32_t* ev, int32_t* partials, int64_t kpad, unsigned* err, unsigned* barrier,
                        unsigned long long* zero64, int64_t zero64_n, const bool* skip,
                        cudaStream_t st) {
  const int S = split ? n_slices : 0;
  if (S < 0 || S > kMaxSlices) return cudaErrorInvalidValue;
  void (*kern)(PrepArgs) = nullptr;
  switch (S) {
    case 0: kern = prep_kernel<0>; break;
    case 1: kern = prep_kernel<1>; break;
    case 2: kern = prep_kernel<2>; break;
    case 3: kern = prep_kernel<3>; break;
    case 4: kern = prep_kernel<4>; break;
    case 5: kern = prep_kernel<5>; break;
    default: kern = prep_kernel<6>; break;
  }
  // co-resident CTAs of the cooperative launch, per instance and device (kept
  // per host thread: no shared mutable state between threads)
  thread_local int max_blocks[kMaxSlices + 1][16] = {};
  int dev = 0;
  {
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 16) return cudaErrorInvalidDevice;
  }
  if (max_blocks[S][dev] == 0) {
    int sms = 0, per = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, THREADS, 0);
    if (e != cudaSuccess) return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    max_blocks[S][dev] = sms * (per < 4 ? per : 4);
  }
  const int cap = max_blocks[S][dev];
  int64_t work = 0;
  {
    int64_t rt_u = (p.M + TILE - 1) / TILE, rt_v = (p.N + TILE - 1) / TILE;
    int64_t ct = (kpad + SLICE_GROUP * SLICE_COLS - 1) / (SLICE_GROUP * SLICE_COLS);
    work = (rt_u + rt_v) * ct * p.n_q;
    if (work > 0xFFFFFFFFll / 2 || (rt_u + rt_v) * (int64_t)prep_scan_parts(p) * p.n_q > 0xFFFFFFFFll / 2)
      return cudaErrorInvalidValue;
  }
  int grid = (int)(work < cap ? (work > 0 ? work : 1) : cap);
  PrepArgs a;
  a.p = p;
  a.t = t;
  a.kpad = kpad;
  a.parts = S > 0 ? prep_scan_parts(p) : 1;
  if (a.parts > 1 && !partials) return cudaErrorInvalidValue;
  a.src[0] = u;
  a.src[1] = v;
  a.dst[0] = ua;
  a.dst[1] = va;
  a.exps[0] = eu;
  a.exps[1] = ev;
  a.part[0] = partials;
  a.part[1] = partials ? partials + (int64_t)a.parts * p.n_q * p.M : nullptr;
  a.fast_rows[0] = rows_fast(p.u);
  a.fast_rows[1] = rows_fast(p.v);
  // 16-byte pair loads need adjacent real entries (not interleaved complex ones)
  a.pair_ok[0] = p.es == 1 && !p.general && !a.fast_rows[0] && pairs_aligned(p.u);
  a.pair_ok[1] = p.es == 1 && !p.general && !a.fast_rows[1] && pairs_aligned(p.v);
  a.err = err;
  a.barrier = barrier;
  a.zero64 = zero64;
  a.zero64_n = zero64_n;
  a.skip[0] = skip && skip[0];
  a.skip[1] = skip && skip[1];
  void* params[] = {&a};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)kern, dim3(grid), dim3(THREADS),
                                              params, 0, st);
  ++g_kernel_launches;
  return e;
}

}  // namespace symctr
