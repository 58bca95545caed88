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

__device__ __forceinline__ uint16_t digit_bf16(int a, int slice) {
  if (a == 0) return 0;
  float f = (float)a;                                  // exact, |a| <= 128
  f = __fmul_rn(f, __int_as_float((127 - 8 * slice) << 23));  // * 2^(-8 slice), exact
  return (uint16_t)(__float_as_uint(f) >> 16);         // low 16 bits are zero
}

// Offset tables: one thread per (batch, index) of the six index maps.
__global__ void __launch_bounds__(THREADS) tables_kernel(Problem p, Tables t) {
  const int64_t segs[6] = {p.M, p.K, p.N, p.K, p.M, p.N};
  int64_t total = 0;
  for (int i = 0; i < 6; ++i) total += segs[i] * p.n_q;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t rem = e;
    int which = 0;
    while (rem >= segs[which] * p.n_q) {
      rem -= segs[which] * p.n_q;
      ++which;
    }
    int64_t b = rem / segs[which], r = rem % segs[which];
    int Q = batch_irrep(p, (int)b);
    const AxisMap& a = which == 0 ? p.u.rows : which == 1 ? p.u.cols : which == 2 ? p.v.rows
                     : which == 3 ? p.v.cols : which == 4 ? p.w.rows : p.w.cols;
    int64_t* dst = which == 0 ? t.urow : which == 1 ? t.ucol : which == 2 ? t.vrow
                 : which == 3 ? t.vcol : which == 4 ? t.wrow : t.wcol;
    dst[rem] = axis_offset(a, p.g, Q, r);
  }
}

// Row exponents, stored biased: E + kExpBias for a row whose largest entry
// lies in [2^E, 2^(E+1)), 0 for an all-zero row (the buffer is zeroed first).
constexpr int32_t kExpBias = 4096;
constexpr int SCAN_COLS = 256;

// Exponent scan: tiles of 32 rows x 256 columns, per-row maxima combined with
// atomicMax in global memory, so any row length spreads over many CTAs.
__global__ void __launch_bounds__(THREADS) exp_scan_kernel(Problem p, const int64_t* __restrict__ rtab,
                                                           const int64_t* __restrict__ ctab, int64_t R,
                                                           int64_t Cn, bool fast_rows,
                                                           const double* __restrict__ src,
                                                           int32_t* __restrict__ exps,
                                                           unsigned* __restrict__ err) {
  __shared__ int64_t roff[TILE], coff[SCAN_COLS];
  __shared__ int32_t rmax[TILE];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t rt = (R + TILE - 1) / TILE, ct = (Cn + SCAN_COLS - 1) / SCAN_COLS;
  const int64_t ntiles = rt * ct * p.n_q;
  for (int64_t tI = blockIdx.x; tI < ntiles; tI += gridDim.x) {
    int64_t b = tI / (rt * ct);
    int64_t rem = tI - b * rt * ct;
    int64_t r0 = (rem / ct) * TILE, c0 = (rem % ct) * SCAN_COLS;
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
    constexpr int PER = SCAN_COLS / (THREADS / 32);   // 32 loads per thread, issued together
    if (fast_rows) {
      // lanes walk rows (contiguous), warps walk columns
      double x[PER];
      const bool rok = r0 + tx < R;
#pragma unroll
      for (int i = 0; i < PER; ++i) {
        int cc = ty + i * (THREADS / 32);
        x[i] = (rok && c0 + cc < Cn) ? src[roff[tx] + coff[cc]] : 0.0;
      }
      int32_t mx = 0;
#pragma unroll
      for (int i = 0; i < PER; ++i) {
        int32_t e = exponent_of(x[i], &bad);
        mx = max(mx, e == kZeroRowExp ? 0 : e + kExpBias);
      }
      atomicMax(&rmax[tx], mx);
    } else {
      // lanes walk columns (contiguous), warps walk rows
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
    if (bad) atomicOr(err, (unsigned)DEVERR_NONFINITE);
    __syncthreads();
    if (threadIdx.x < TILE && r0 + threadIdx.x < R && rmax[threadIdx.x] > 0)
      atomicMax(&exps[b * R + r0 + threadIdx.x], rmax[threadIdx.x]);
  }
}

constexpr int SLICE_COLS = 64;

// Slicing: tiles of 32 rows x 64 columns of the padded aligned operand; the
// source tile goes through shared memory so that the reduced form is read
// along its contiguous axis and every slice row is written as 128-byte runs.
__global__ void __launch_bounds__(THREADS) slice_kernel(Problem p, const int64_t* __restrict__ rtab,
                                                        const int64_t* __restrict__ ctab, int64_t R,
                                                        int64_t Cn, int64_t kpad, bool fast_rows,
                                                        int S, const double* __restrict__ src,
                                                        const int32_t* __restrict__ exps,
                                                        uint32_t* __restrict__ slices) {
  __shared__ double tile[TILE][SLICE_COLS + 1];
  __shared__ int64_t roff[TILE], coff[SLICE_COLS];
  __shared__ int32_t rexp[TILE];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t rt = (R + TILE - 1) / TILE, ct = (kpad + SLICE_COLS - 1) / SLICE_COLS;
  const int64_t ntiles = rt * ct * p.n_q;
  const int64_t slice_stride = (int64_t)p.n_q * R * kpad / 2;  // in uint32 pairs
  for (int64_t tI = blockIdx.x; tI < ntiles; tI += gridDim.x) {
    int64_t b = tI / (rt * ct);
    int64_t rem = tI - b * rt * ct;
    int64_t r0 = (rem / ct) * TILE, c0 = (rem % ct) * SLICE_COLS;
    __syncthreads();
    if (threadIdx.x < TILE) {
      int64_t r = r0 + threadIdx.x;
      roff[threadIdx.x] = r < R ? rtab[b * R + r] : 0;
      int32_t st = r < R ? exps[b * R + r] : 0;
      rexp[threadIdx.x] = st == 0 ? kZeroRowExp : st - kExpBias;
    } else if (threadIdx.x < TILE + SLICE_COLS) {
      int64_t c = c0 + threadIdx.x - TILE;
      coff[threadIdx.x - TILE] = c < Cn ? ctab[b * Cn + c] : 0;
    }
    __syncthreads();
    if (fast_rows) {
      double x[SLICE_COLS / (THREADS / 32)];
      const bool rok = r0 + tx < R;
#pragma unroll
      for (int i = 0; i < SLICE_COLS / (THREADS / 32); ++i) {
        int cc = ty + i * (THREADS / 32);
        x[i] = (rok && c0 + cc < Cn) ? src[roff[tx] + coff[cc]] : 0.0;
      }
#pragma unroll
      for (int i = 0; i < SLICE_COLS / (THREADS / 32); ++i) tile[tx][ty + i * (THREADS / 32)] = x[i];
    } else {
      double x[TILE / (THREADS / 32)][SLICE_COLS / 32];
#pragma unroll
      for (int rg = 0; rg < TILE / (THREADS / 32); ++rg)
#pragma unroll
        for (int i = 0; i < SLICE_COLS / 32; ++i) {
          int rr = ty + rg * (THREADS / 32), cc = tx + 32 * i;
          x[rg][i] = (r0 + rr < R && c0 + cc < Cn) ? src[roff[rr] + coff[cc]] : 0.0;
        }
#pragma unroll
      for (int rg = 0; rg < TILE / (THREADS / 32); ++rg)
#pragma unroll
        for (int i = 0; i < SLICE_COLS / 32; ++i) tile[ty + rg * (THREADS / 32)][tx + 32 * i] = x[rg][i];
    }
    __syncthreads();
    // each thread: one row, two adjacent columns -> one uint32 per slice
    for (int rr = ty; rr < TILE; rr += THREADS / 32) {
      int64_t r = r0 + rr, c = c0 + 2 * tx;
      if (r >= R || c >= kpad) continue;
      int64_t X0 = fixed_point(tile[rr][2 * tx], rexp[rr], S);
      int64_t X1 = fixed_point(tile[rr][2 * tx + 1], rexp[rr], S);
      uint32_t* dst = slices + ((b * R + r) * kpad + c) / 2;
      for (int i = S - 1; i >= 1; --i) {
        int a0 = (int)(((X0 + 128) & 255) - 128);
        int a1 = (int)(((X1 + 128) & 255) - 128);
        X0 = (X0 - a0) >> 8;
        X1 = (X1 - a1) >> 8;
        dst[(int64_t)i * slice_stride] = (uint32_t)digit_bf16(a0, i) | ((uint32_t)digit_bf16(a1, i) << 16);
      }
      dst[0] = (uint32_t)digit_bf16((int)X0, 0) | ((uint32_t)digit_bf16((int)X1, 0) << 16);
    }
  }
}

// TF32 form: aligned float32 operand rounded to TF32 (round to nearest even
// on the 10-bit mantissa), zero padded to kpad columns.
__global__ void __launch_bounds__(THREADS) tf32_kernel(Problem p, const int64_t* __restrict__ rtab,
                                                       const int64_t* __restrict__ ctab, int64_t R,
                                                       int64_t Cn, int64_t kpad, bool fast_rows,
                                                       const double* __restrict__ src,
                                                       float* __restrict__ dst) {
  __shared__ float tile[TILE][TILE + 1];
  __shared__ int64_t roff[TILE], coff[TILE];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t rt = (R + TILE - 1) / TILE, ct = (kpad + TILE - 1) / TILE;
  const int64_t ntiles = rt * ct * p.n_q;
  for (int64_t tI = blockIdx.x; tI < ntiles; tI += gridDim.x) {
    int64_t b = tI / (rt * ct);
    int64_t rem = tI - b * rt * ct;
    int64_t r0 = (rem / ct) * TILE, c0 = (rem % ct) * TILE;
    __syncthreads();
    if (threadIdx.x < TILE) {
      int64_t r = r0 + threadIdx.x;
      roff[threadIdx.x] = r < R ? rtab[b * R + r] : 0;
    } else if (threadIdx.x < 2 * TILE) {
      int64_t c = c0 + threadIdx.x - TILE;
      coff[threadIdx.x - TILE] = c < Cn ? ctab[b * Cn + c] : 0;
    }
    __syncthreads();
    for (int k = ty; k < TILE; k += THREADS / 32) {
      int rr = fast_rows ? tx : k, cc = fast_rows ? k : tx;
      float f = 0.f;
      if (r0 + rr < R && c0 + cc < Cn) {
        f = __double2float_rn(src[roff[rr] + coff[cc]]);
        uint32_t u = __float_as_uint(f);
        if ((u & 0x7F800000u) != 0x7F800000u) {
          u = (u + 0xFFFu + ((u >> 13) & 1u)) & ~0x1FFFu;
          f = __uint_as_float(u);
        }
      }
      tile[rr][cc] = f;
    }
    __syncthreads();
    for (int k = ty; k < TILE; k += THREADS / 32) {
      if (r0 + k < R && c0 + tx < kpad) dst[(b * R + r0 + k) * kpad + c0 + tx] = tile[k][tx];
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

cudaError_t launch_tables(const Problem& p, const Tables& t, cudaStream_t st) {
  int64_t total = tables_entries(p);
  if (total == 0) return cudaSuccess;
  tables_kernel<<<grid_for((total + THREADS - 1) / THREADS), THREADS, 0, st>>>(p, t);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_split_operand(const Problem& p, const Tables& t, int operand, int n_slices,
                                 const double* src, uint16_t* slices, int64_t kpad, int32_t* exps,
                                 unsigned* err, cudaStream_t st) {
  int64_t R, Cn;
  operand_extent(p, operand, &R, &Cn);
  const OperandMap& m = operand_map(p, operand);
  const int64_t* rt = operand == 0 ? t.urow : t.vrow;
  const int64_t* ct = operand == 0 ? t.ucol : t.vcol;
  cudaError_t e = cudaMemsetAsync(exps, 0, sizeof(int32_t) * R * p.n_q, st);
  if (e != cudaSuccess) return e;
  int64_t t1 = ((R + TILE - 1) / TILE) * ((Cn + SCAN_COLS - 1) / SCAN_COLS) * p.n_q;
  exp_scan_kernel<<<grid_for(t1), THREADS, 0, st>>>(p, rt, ct, R, Cn, rows_fast(m), src, exps, err);
  ++g_kernel_launches;
  int64_t t2 = ((R + TILE - 1) / TILE) * ((kpad + SLICE_COLS - 1) / SLICE_COLS) * p.n_q;
  slice_kernel<<<grid_for(t2), THREADS, 0, st>>>(p, rt, ct, R, Cn, kpad, rows_fast(m), n_slices, src,
                                                  exps, (uint32_t*)slices);
  ++g_kernel_launches;
  return cudaGetLastError();
}

cudaError_t launch_tf32_operand(const Problem& p, const Tables& t, int operand, const double* src,
                                float* dst, int64_t kpad, cudaStream_t st) {
  int64_t R, Cn;
  operand_extent(p, operand, &R, &Cn);
  const OperandMap& m = operand_map(p, operand);
  const int64_t* rt = operand == 0 ? t.urow : t.vrow;
  const int64_t* ct = operand == 0 ? t.ucol : t.vcol;
  int64_t tiles = ((R + TILE - 1) / TILE) * ((kpad + TILE - 1) / TILE) * p.n_q;
  tf32_kernel<<<grid_for(tiles), THREADS, 0, st>>>(p, rt, ct, R, Cn, kpad, rows_fast(m), src, dst);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace symctr
