// Float64 form of the aligned contraction (Alg. 2, contraction step):
//   W_hat[Q, m, n] = sum_kappa U_hat[Q, m, kappa] V_hat[Q, n, kappa]
// with the input transformations fused into the operand loads (each tile
// element is gathered from the standard reduced form through the separable
// index maps) and the output step fused into the epilogue (each result is
// written straight to W's standard reduced form).  GB300 has very little
// float64 throughput, so the aligned operands are never materialised: the
// loads are free next to the FMAs.
//
// Three kernels: a 64x64 register-tiled kernel for GEMM-shaped problems, a
// warp-per-row dot-product kernel for skinny ones (a few rows or columns),
// both with optional split-K through atomicAdd into a zeroed output (or onto
// the existing output in accumulate mode), and a thread-per-row kernel for
// skinny problems with a short contracted extent (the adjoints of a GEMV:
// an outer product, K = 1, or K = 2), where lanes walking K would idle.
#include <cstdint>

#include "symctr_internal.h"

namespace symctr {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, THREADS = 256;

// axis_offset as one out-of-line device function: every kernel below computes
// offsets in a dozen places (per instance of the short-side row count), and
// inlining the mixed-radix arithmetic at each of them multiplied the code size
// and the compile time without changing the speed (none of these calls sits in
// an innermost loop).
__device__ __noinline__ int64_t aoff(const AxisMap& a, const GroupDesc& g, int Q, int64_t r) {
  return axis_offset(a, g, Q, r);
}

__host__ __device__ inline bool map_rows_fast(const AxisMap& rows) {
  return rows.n > 0 && rows.bstride[rows.n - 1] == 1;
}

// General plans pass their offset tables (t.urow != NULL): offsets come from
// them, -1 marking an absent aligned row or column (read as zero, not stored).
__global__ void __launch_bounds__(THREADS) gemm_f64_tiled(const __grid_constant__ Problem p, int ksplit, bool u_rows_fast,
                                                          bool v_rows_fast, const Tables t,
                                                          const double* __restrict__ U,
                                                          const double* __restrict__ V,
                                                          double* __restrict__ W) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  __shared__ int64_t uoff[BM], voff[BN], kuoff[BK], kvoff[BK], woffr[BM], woffc[BN];
  const int tid = threadIdx.x;
  const int tr = tid / 16, tc = tid % 16;
  const int64_t mt = (p.M + BM - 1) / BM, nt = (p.N + BN - 1) / BN;
  const int64_t kchunk = ((p.K + ksplit - 1) / ksplit + BK - 1) / BK * BK;
  const int64_t ntiles = mt * nt * p.n_q * ksplit;
  for (int64_t tI = blockIdx.x; tI < ntiles; tI += gridDim.x) {
    int64_t ks = tI % ksplit;
    int64_t t2 = tI / ksplit;
    int64_t b = t2 / (mt * nt);
    int64_t rem = t2 - b * mt * nt;
    int64_t m0 = (rem / nt) * BM, n0 = (rem % nt) * BN;
    int Q = batch_irrep(p, (int)b);
    int64_t kbeg = ks * kchunk, kend = kbeg + kchunk < p.K ? kbeg + kchunk : p.K;
    __syncthreads();
    const bool tab = t.urow != nullptr;
    if (tid < BM) {
      int64_t m = m0 + tid;
      uoff[tid] = m >= p.M ? 0 : tab ? t.urow[b * p.M + m] : aoff(p.u.rows, p.g, Q, m);
      woffr[tid] = m >= p.M ? 0 : tab ? t.wrow[b * p.M + m] : aoff(p.w.rows, p.g, Q, m);
    } else if (tid < BM + BN) {
      int64_t n = n0 + tid - BM;
      voff[tid - BM] = n >= p.N ? 0 : tab ? t.vrow[b * p.N + n] : aoff(p.v.rows, p.g, Q, n);
      woffc[tid - BM] = n >= p.N ? 0 : tab ? t.wcol[b * p.N + n] : aoff(p.w.cols, p.g, Q, n);
    }
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
      __syncthreads();
      if (tid < BK) {
        int64_t k = k0 + tid;
        kuoff[tid] = k >= kend ? 0 : tab ? t.ucol[b * p.K + k] : aoff(p.u.cols, p.g, Q, k);
      } else if (tid >= 32 && tid < 32 + BK) {
        int64_t k = k0 + tid - 32;
        kvoff[tid - 32] = k >= kend ? 0 : tab ? t.vcol[b * p.K + k] : aoff(p.v.cols, p.g, Q, k);
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < (BM * BK) / THREADS; ++j) {
        int e = tid + j * THREADS;
        int mm = u_rows_fast ? e % BM : e / BK;
        int kk = u_rows_fast ? e / BM : e % BK;
        double x = 0.0;
        if (m0 + mm < p.M && k0 + kk < kend && uoff[mm] >= 0 && kuoff[kk] >= 0)
          x = U[p.es * (uoff[mm] + kuoff[kk])];
        As[kk][mm] = x;
      }
#pragma unroll
      for (int j = 0; j < (BN * BK) / THREADS; ++j) {
        int e = tid + j * THREADS;
        int nn = v_rows_fast ? e % BN : e / BK;
        int kk = v_rows_fast ? e / BN : e % BK;
        double x = 0.0;
        if (n0 + nn < p.N && k0 + kk < kend && voff[nn] >= 0 && kvoff[kk] >= 0)
          x = V[p.es * (voff[nn] + kvoff[kk])];
        Bs[kk][nn] = x;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][tr + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tc + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int mm = tr + 16 * i;
      if (m0 + mm >= p.M || woffr[mm] < 0) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int nn = tc + 16 * j;
        if (n0 + nn >= p.N || woffc[nn] < 0) continue;
        double* dst = W + p.es * (woffr[mm] + woffc[nn]);
        if (ksplit > 1) atomicAdd(dst, signed_result(p, acc[i][j]));
        else store_w(p, dst, acc[i][j]);
      }
    }
  }
}

// Skinny problems: the "long" side L (rows of U or of V, whichever is larger)
// is spread over warps, the "short" side (<= 8 rows) is held in registers;
// lanes stride over kappa.  Optional split-K over kappa ranges.
//
// Column offsets: kappa = o * I + i, where I (the "inner" extent) is the
// product of the fastest block dims of the column map up to kInnerMax.  The
// offset is then aoff(o * I) + inner(i), inner(i) being the block part
// of i alone (independent of Q); each block tabulates inner() in shared
// memory, and a warp computes the offsets aoff(o * I) of the inner blocks of
// its K range 16 at a time, one per lane, instead of one mixed-radix
// decomposition per element.
constexpr int SKINNY_MAX = 8;
constexpr int kInnerMax = 2048;

// Product of the fastest block dims that the two column maps share, up to
// kInnerMax (both maps index the same kappa, so their dims agree).
__device__ __forceinline__ int64_t inner_extent(const AxisMap& a, const AxisMap& b) {
  int64_t e = 1;
  for (int i = a.n - 1, j = b.n - 1; i >= 0 && j >= 0; --i, --j) {
    if (a.D[i] != b.D[j] || e * a.D[i] > kInnerMax) break;
    e *= a.D[i];
  }
  return e;
}

// A 64-bit integer division is a long emulated instruction sequence:
// quotients of values below 2^32 are taken in 32 bits.
__device__ __forceinline__ int64_t div_idx(int64_t a, int64_t b) {
  if (((uint64_t)a | (uint64_t)b) <= 0xFFFFFFFFull) return (int64_t)((uint32_t)a / (uint32_t)b);
  return a / b;
}

// scale * inner(i) for i < I: the block digits of i over the fastest block
// axes (scale: the element stride, so that the table holds array indices).
// I <= kInnerMax, so the digits are taken in 32 bits.
__device__ void fill_inner(const AxisMap& a, int64_t I, int64_t scale, int64_t* tab) {
  for (int i = threadIdx.x; i < (int)I; i += blockDim.x) {
    uint32_t r = (uint32_t)i;
    int64_t off = 0;
    for (int d = a.n - 1; d >= 0 && r > 0; --d) {
      const uint32_t D = (uint32_t)a.D[d], q = r / D;
      off += (int64_t)(r - q * D) * a.bstride[d];
      r = q;
    }
    tab[i] = off * scale;
  }
}

// Elements per lane whose loads (one of L, NS of S) are all issued before
// their FMAs: fewer for more short-side rows, so that the registers they
// take stay about the same.
template <int NS>
struct SkinnyUnroll {
  static constexpr int value = NS <= 2 ? 4 : 2;
};

// NS = the short side's row count (one instance per count, so that no
// float64 instruction of an absent row is issued: GB300's float64 pipe is
// narrow and issues predicated-off instructions all the same).
//
// Work items: (irrep, long-side row, K range), the K ranges whole inner
// blocks; the launcher sizes ksplit so that the items about fill the
// resident warps once, which pays the offset arithmetic of an item (a
// dependent chain of modular arithmetic under a product group) once per warp.
template <int NS>
__global__ void __launch_bounds__(THREADS, 3)
    gemm_f64_skinny(const __grid_constant__ Problem p, bool long_is_u, int ksplit, const double* __restrict__ U,
                    const double* __restrict__ V, double* __restrict__ W) {
  __shared__ int64_t tab_l[kInnerMax], tab_s[kInnerMax];
  const AxisMap& Lrows = long_is_u ? p.u.rows : p.v.rows;
  const AxisMap& Lcols = long_is_u ? p.u.cols : p.v.cols;
  const AxisMap& Srows = long_is_u ? p.v.rows : p.u.rows;
  const AxisMap& Scols = long_is_u ? p.v.cols : p.u.cols;
  // W's axis along the long side and along the short side
  const AxisMap& Wl = long_is_u ? p.w.rows : p.w.cols;
  const AxisMap& Ws = long_is_u ? p.w.cols : p.w.rows;
  const double* Lp = long_is_u ? U : V;
  const double* Sp = long_is_u ? V : U;
  const int64_t nL = long_is_u ? p.M : p.N;
  const int64_t es = p.es;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t I = inner_extent(Lcols, Scols);
  fill_inner(Lcols, I, es, tab_l);
  fill_inner(Scols, I, es, tab_s);
  __syncthreads();
  // K ranges of whole inner blocks (K is a multiple of I)
  const int64_t nb = div_idx(p.K, I);
  const int64_t per = div_idx(nb + ksplit - 1, ksplit);
  const int64_t parts = div_idx(nb + per - 1, per);
  const int64_t items = nL * p.n_q * parts;
  for (int64_t it = warp; it < items; it += nwarps) {
    const int64_t t2 = div_idx(it, parts);
    const int64_t ks = it - t2 * parts;
    const int64_t b = div_idx(t2, nL);
    const int64_t l = t2 - b * nL;
    const int Q = batch_irrep(p, (int)b);
    // the row offsets, one per lane: lane 0 L's row, lanes 1..NS the short
    // rows in S, lane NS+1 the long row along W, lanes NS+2..2NS+1 the short
    // rows along W (the other lanes repeat lane 0's)
    const AxisMap* rm = &Lrows;
    int64_t rr = l;
    if (lane >= 1 && lane <= NS) {
      rm = &Srows;
      rr = lane - 1;
    } else if (lane == NS + 1) {
      rm = &Wl;
    } else if (lane >= NS + 2 && lane <= 2 * NS + 1) {
      rm = &Ws;
      rr = lane - NS - 2;
    }
    const int64_t ro = aoff(*rm, p.g, Q, rr);
    const int64_t loff = es * __shfl_sync(0xffffffffu, ro, 0);
    int64_t soff[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) soff[s] = es * __shfl_sync(0xffffffffu, ro, 1 + s);
    double acc[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) acc[s] = 0.0;
    const int64_t ob0 = ks * per, ob1 = ob0 + per < nb ? ob0 + per : nb;
    if (I >= 32) {
      // inner blocks 16 at a time: lanes 0-15 compute the L offsets of blocks
      // g0 + lane, lanes 16-31 the S offsets of blocks g0 + lane - 16
      for (int64_t g0 = ob0; g0 < ob1; g0 += 16) {
        const int64_t ob = g0 + (lane & 15);
        const int64_t co = ob < ob1 ? aoff(lane < 16 ? Lcols : Scols, p.g, Q, ob * I) : 0;
        const int nbk = ob1 - g0 < 16 ? (int)(ob1 - g0) : 16;
        for (int j = 0; j < nbk; ++j) {
          const double* Lb = Lp + (loff + es * __shfl_sync(0xffffffffu, co, j));
          const int64_t sb = es * __shfl_sync(0xffffffffu, co, 16 + j);
          const double* Sb[NS];
#pragma unroll
          for (int s = 0; s < NS; ++s) Sb[s] = Sp + (soff[s] + sb);
          constexpr int kU = SkinnyUnroll<NS>::value;
          for (int i0 = 0; i0 < (int)I; i0 += 32 * kU) {
            if (i0 + 32 * kU <= (int)I) {
              double x[kU], y[NS][kU];
#pragma unroll
              for (int u = 0; u < kU; ++u) {
                const int i = i0 + 32 * u + lane;
                const int64_t tl = tab_l[i], ts = tab_s[i];
                x[u] = Lb[tl];
#pragma unroll
                for (int s = 0; s < NS; ++s) y[s][u] = Sb[s][ts];
              }
#pragma unroll
              for (int u = 0; u < kU; ++u) {
#pragma unroll
                for (int s = 0; s < NS; ++s) acc[s] = fma(x[u], y[s][u], acc[s]);
              }
            } else {
              // the ragged end of an inner block (I not a multiple of 32 kU)
              for (int i = i0 + lane; i < (int)I; i += 32) {
                const double x = Lb[tab_l[i]];
#pragma unroll
                for (int s = 0; s < NS; ++s) acc[s] = fma(x, Sb[s][tab_s[i]], acc[s]);
              }
            }
          }
        }
      }
    } else {
      // short inner blocks: lanes walk the elements, recomputing the two
      // inner-block offsets when the block changes
      const int64_t kend = ob1 * I;
      int64_t k = ob0 * I + lane;
      int64_t o = div_idx(k, I), i = k - o * I;
      int64_t lo = es * aoff(Lcols, p.g, Q, o * I), so = es * aoff(Scols, p.g, Q, o * I);
      for (; k < kend; k += 32) {
        const double x = Lp[loff + lo + tab_l[i]];
        const int64_t sc = so + tab_s[i];
#pragma unroll
        for (int s = 0; s < NS; ++s) acc[s] = fma(x, Sp[soff[s] + sc], acc[s]);
        i += 32;
        if (i >= I) {
          o += i / I;
          i %= I;
          if (k + 32 < kend) {
            lo = es * aoff(Lcols, p.g, Q, o * I);
            so = es * aoff(Scols, p.g, Q, o * I);
          }
        }
      }
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      double a = acc[s];
      for (int o2 = 16; o2 > 0; o2 >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o2);
      acc[s] = a;
    }
    const int64_t wlo = __shfl_sync(0xffffffffu, ro, NS + 1);
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int64_t wso = __shfl_sync(0xffffffffu, ro, NS + 2 + s);
      if (lane == 0) {
        double* dst = W + es * (wlo + wso);
        if (ksplit > 1) atomicAdd(dst, signed_result(p, acc[s]));
        else store_w(p, dst, acc[s]);
      }
    }
  }
}

// Skinny problems with K <= kShortK: one thread per row of the long side, on
// a persistent grid whose blocks take kShortRows consecutive rows (a chunk)
// at a time.  The short side's values and the long side's column offsets
// depend only on the irrep, so a block stages them in shared memory when the
// irrep changes.  Row offsets in
// L and W use the inner-block split of the skinny kernel above (l = o * I +
// i): a table of inner(i) per map, and aoff(o * I) for the inner blocks of a
// chunk computed by as many threads at once, spread over the warps (the
// index arithmetic of one offset is a long dependent chain under a product
// group, so it is never left to a single thread).  A thread issues the loads
// of a few rows (ShortUnroll) before their FMAs.
constexpr int kShortK = 32;
constexpr int kShortRows = 4096;
constexpr int kShortSlots = kShortRows / 32 + 2;

// Rows per thread whose loads are all issued before their FMAs.
template <int KT>
struct ShortUnroll {
  static constexpr int value = KT == 1 ? 8 : (KT == 2 ? 4 : 2);
};

// Step (o, i) = divmod(l, I) by THREADS rows without dividing.
__device__ __forceinline__ void step_rows(int I, int& o, int& i) {
  i += THREADS;
  while (i >= I) {
    i -= I;
    ++o;
  }
}

// A W entry of the short-K kernel, whose staged short-side values carry the
// problem's sign (exact: x * (-s) = -(x * s)).  Accumulation is a float64
// atomic add (a single writer per entry: the same rounded sum).
__device__ __forceinline__ void put_w(int accumulate, double* dst, double x) {
  if (accumulate)
    atomicAdd(dst, x);
  else
    *dst = x;
}

// KT: K itself when it is 1 or 2 (the loads of a row unrolled), 0 for any
// K <= kShortK (a loop over K).
template <int NS, int KT>
__global__ void __launch_bounds__(THREADS, 4)
    gemm_f64_shortk(const __grid_constant__ Problem p, bool long_is_u, const double* __restrict__ U,
                    const double* __restrict__ V, double* __restrict__ W) {
  __shared__ double sval[SKINNY_MAX][kShortK];
  __shared__ int64_t lco[kShortK], scol[kShortK];
  __shared__ int64_t wso[SKINNY_MAX], srow[SKINNY_MAX];
  __shared__ int64_t tab_lr[kInnerMax], tab_w[kInnerMax];
  __shared__ int64_t ob_l[kShortSlots], ob_w[kShortSlots];
  const AxisMap& Lrows = long_is_u ? p.u.rows : p.v.rows;
  const AxisMap& Lcols = long_is_u ? p.u.cols : p.v.cols;
  const AxisMap& Srows = long_is_u ? p.v.rows : p.u.rows;
  const AxisMap& Scols = long_is_u ? p.v.cols : p.u.cols;
  const AxisMap& Wl = long_is_u ? p.w.rows : p.w.cols;
  const AxisMap& Ws = long_is_u ? p.w.cols : p.w.rows;
  const double* Lp = long_is_u ? U : V;
  const double* Sp = long_is_u ? V : U;
  const int64_t nL = long_is_u ? p.M : p.N;
  const int64_t es = p.es;
  constexpr int RU = ShortUnroll<KT>::value;
  constexpr int KX = KT > 0 ? KT : 1;
  const int K = KT ? KT : (int)p.K;
  const int64_t per_q = (nL + kShortRows - 1) / kShortRows;
  // the rows of L and W's axis along the long side index the same modes
  const int64_t I = inner_extent(Lrows, Wl);
  const bool tabulated = I >= 32;   // then a chunk touches <= kShortSlots inner blocks
  if (tabulated) {
    fill_inner(Lrows, I, es, tab_lr);
    fill_inner(Wl, I, es, tab_w);
  }
  // this thread's share of a chunk's offsets: task t falls to lane t / 8 of
  // warp t % 8, so that every warp computes about as many
  const int task0 = (threadIdx.x & 31) * (THREADS / 32) + (threadIdx.x >> 5);
  int staged = -1;
  for (int64_t blk = blockIdx.x; blk < per_q * p.n_q; blk += gridDim.x) {
    const int b = (int)div_idx(blk, per_q);
    const int64_t l0 = (blk - (int64_t)b * per_q) * kShortRows;
    const int64_t lend = l0 + kShortRows < nL ? l0 + kShortRows : nL;
    const int64_t o0 = div_idx(l0, I);
    const int Q = batch_irrep(p, b);
    __syncthreads();   // the previous chunk's readers are done
    // one offset per task: on a new irrep first the short rows in S, S's and
    // L's columns and the short rows along W (2 NS + 2 K), then L's and W's
    // offsets of the chunk's inner blocks (alternating)
    const bool stage = b != staged;
    const int n_s = stage ? 2 * NS + 2 * K : 0;
    const int n_t = n_s + (tabulated ? 2 * (int)(div_idx(lend - 1, I) - o0 + 1) : 0);
    for (int t = task0; t < n_t; t += THREADS) {
      const AxisMap* m;
      int64_t r, sc = es;
      int64_t* dst;
      if (t >= n_s) {
        const int j = (t - n_s) / 2;
        m = ((t - n_s) & 1) ? &Wl : &Lrows;
        r = (o0 + j) * I;
        dst = ((t - n_s) & 1) ? &ob_w[j] : &ob_l[j];
      } else if (t < NS) {
        m = &Srows;
        r = t;
        sc = 1;
        dst = &srow[t];
      } else if (t < NS + K) {
        m = &Scols;
        r = t - NS;
        sc = 1;
        dst = &scol[t - NS];
      } else if (t < NS + 2 * K) {
        m = &Lcols;
        r = t - NS - K;
        dst = &lco[t - NS - K];
      } else {
        m = &Ws;
        r = t - NS - 2 * K;
        dst = &wso[t - NS - 2 * K];
      }
      *dst = sc * aoff(*m, p.g, Q, r);
    }
    __syncthreads();
    if (stage) {
      for (int i = threadIdx.x; i < NS * K; i += THREADS) {
        const int sr = i / K, k = i - sr * K;
        sval[sr][k] = signed_result(p, Sp[es * (srow[sr] + scol[k])]);
      }
      staged = b;
      __syncthreads();
    }
    // a row's two columns of L (two short rows of W) adjacent in memory
    const bool pair_l = K == 2 && lco[1] == lco[0] + 1;
    const bool pair_w = NS == 2 && wso[1] == wso[0] + 1;
    if (!tabulated) {
      // short inner blocks: the offsets of each row from scratch
      for (int64_t l = l0 + threadIdx.x; l < lend; l += THREADS) {
        const int64_t lo = es * aoff(Lrows, p.g, Q, l), wo = es * aoff(Wl, p.g, Q, l);
        double acc[NS];
#pragma unroll
        for (int sr = 0; sr < NS; ++sr) acc[sr] = 0.0;
        for (int k = 0; k < K; ++k) {
          const double x = Lp[lo + lco[k]];
#pragma unroll
          for (int sr = 0; sr < NS; ++sr) acc[sr] = fma(x, sval[sr][k], acc[sr]);
        }
#pragma unroll
        for (int sr = 0; sr < NS; ++sr) put_w(p.accumulate, W + (wo + wso[sr]), acc[sr]);
      }
      continue;
    }
    // (o - o0, i) of the thread's first row by one division; rows and inner
    // positions within a chunk in 32 bits (a chunk spans kShortRows rows)
    const int nrows = (int)(lend - l0), Ii = (int)I;
    int orel = (int)(div_idx(l0 + threadIdx.x, I) - o0);
    int i = (int)(l0 + threadIdx.x - (o0 + orel) * I);
    for (int t = threadIdx.x; t < nrows; t += THREADS * RU) {
      // RU rows: every load first, then the products and stores, the W
      // offsets found again from the saved (o - o0, i)
      const int os = orel, is = i;
      if (KT > 0) {
        double x[RU][KX];
#pragma unroll
        for (int r = 0; r < RU; ++r) {
          const bool ok = t + r * THREADS < nrows;
          const int64_t lo = ok ? ob_l[orel] + tab_lr[i] : 0;
          const double* src = Lp + (lo + lco[0]);
          if (KX == 2 && ok && pair_l && ((uintptr_t)src & 15) == 0) {
            // a row's two entries adjacent: one 16-byte load
            const double2 v2 = *reinterpret_cast<const double2*>(src);
            x[r][0] = v2.x;
            x[r][KX - 1] = v2.y;
          } else {
#pragma unroll
            for (int k = 0; k < KX; ++k) x[r][k] = ok ? Lp[lo + lco[k]] : 0.0;
          }
          if (ok) step_rows(Ii, orel, i);
        }
        int o2 = os, i2 = is;
#pragma unroll
        for (int r = 0; r < RU; ++r) {
          if (t + r * THREADS >= nrows) break;
          const int64_t wo = ob_w[o2] + tab_w[i2];
          double a[NS];
#pragma unroll
          for (int sr = 0; sr < NS; ++sr) {
            // the sum starts from the first product (not an FMA onto 0.0:
            // the float64 pipe is the bound here)
            a[sr] = x[r][0] * sval[sr][0];
#pragma unroll
            for (int k = 1; k < KX; ++k) a[sr] = fma(x[r][k], sval[sr][k], a[sr]);
          }
          double* dst = W + (wo + wso[0]);
          if (NS == 2 && pair_w && !p.accumulate && ((uintptr_t)dst & 15) == 0) {
            // the row's two results adjacent: one 16-byte store
            *reinterpret_cast<double2*>(dst) = make_double2(a[0], a[NS - 1]);
          } else {
#pragma unroll
            for (int sr = 0; sr < NS; ++sr) put_w(p.accumulate, W + (wo + wso[sr]), a[sr]);
          }
          step_rows(Ii, o2, i2);
        }
      } else {
        int64_t wo[RU];
        int64_t lo[RU];
#pragma unroll
        for (int r = 0; r < RU; ++r) {
          const bool ok = t + r * THREADS < nrows;
          lo[r] = ok ? ob_l[orel] + tab_lr[i] : -1;
          wo[r] = ok ? ob_w[orel] + tab_w[i] : 0;
          if (ok) step_rows(Ii, orel, i);
        }
        double acc[RU][NS];
#pragma unroll
        for (int r = 0; r < RU; ++r)
#pragma unroll
          for (int sr = 0; sr < NS; ++sr) acc[r][sr] = 0.0;
        for (int k = 0; k < K; ++k) {
          double x[RU];
#pragma unroll
          for (int r = 0; r < RU; ++r) x[r] = lo[r] >= 0 ? Lp[lo[r] + lco[k]] : 0.0;
#pragma unroll
          for (int r = 0; r < RU; ++r)
#pragma unroll
            for (int sr = 0; sr < NS; ++sr) acc[r][sr] = fma(x[r], sval[sr][k], acc[r][sr]);
        }
#pragma unroll
        for (int r = 0; r < RU; ++r) {
          if (lo[r] < 0) break;
#pragma unroll
          for (int sr = 0; sr < NS; ++sr) put_w(p.accumulate, W + (wo[r] + wso[sr]), acc[r][sr]);
        }
      }
    }
  }
}

int sm_count() {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

// Zero the entries of W that a split-K launch accumulates into.
__global__ void zero_w_entries(const __grid_constant__ Problem p, double* __restrict__ W) {
  int64_t total = (int64_t)p.n_q * p.M * p.N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = i / (p.M * p.N);
    int64_t r = i - b * p.M * p.N;
    int64_t m = r / p.N, n = r % p.N;
    int Q = batch_irrep(p, (int)b);
    W[p.es * (aoff(p.w.rows, p.g, Q, m) + aoff(p.w.cols, p.g, Q, n))] = 0.0;
  }
}

// Resident blocks per SM of a kernel instance (cached per device).
template <typename Kernel>
int blocks_per_sm(Kernel kernel, int* cache) {
  int dev = 0;
  cudaGetDevice(&dev);
  int& c = cache[dev & 63];
  if (c == 0) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, THREADS, 0) != cudaSuccess || n < 1) n = 1;
    c = n;
  }
  return c;
}

template <int NS, int KT>
void launch_shortk_kt(int sms, int64_t chunks, cudaStream_t st, const Problem& p, bool long_is_u, const double* u,
                      const double* v, double* w) {
  // a persistent grid: a block stages an irrep's values once and walks its chunks
  static int cache[64] = {};
  const int64_t resident = (int64_t)blocks_per_sm(gemm_f64_shortk<NS, KT>, cache) * sms;
  const int grid = (int)(chunks < resident ? chunks : resident);
  gemm_f64_shortk<NS, KT><<<grid, THREADS, 0, st>>>(p, long_is_u, u, v, w);
}

template <int NS>
void launch_shortk_ns(int kt, int sms, int64_t chunks, cudaStream_t st, const Problem& p, bool long_is_u,
                      const double* u, const double* v, double* w) {
  if (kt == 1) launch_shortk_kt<NS, 1>(sms, chunks, st, p, long_is_u, u, v, w);
  else if (kt == 2) launch_shortk_kt<NS, 2>(sms, chunks, st, p, long_is_u, u, v, w);
  else launch_shortk_kt<NS, 0>(sms, chunks, st, p, long_is_u, u, v, w);
}

// Resident warps of the skinny kernel's instance for NS short-side rows
// (cached per device).
template <int NS>
int64_t skinny_resident_warps(int sms) {
  static int cache[64] = {};
  return (int64_t)blocks_per_sm(gemm_f64_skinny<NS>, cache) * sms * (THREADS / 32);
}

template <int NS>
void launch_skinny_ns(int sms, cudaStream_t st, const Problem& p, bool long_is_u, const double* u,
                      const double* v, double* w) {
  const int64_t nL = long_is_u ? p.M : p.N;
  const int64_t rows = nL * p.n_q;
  const int64_t resident = skinny_resident_warps<NS>(sms);
  // one item per resident warp where the rows are fewer, K ranges of at
  // least 512 entries
  int64_t ksplit = 1;
  if (rows < resident) {
    ksplit = resident / rows;
    const int64_t most = p.K / 512 > 1 ? p.K / 512 : 1;
    if (ksplit > most) ksplit = most;
  }
  if (ksplit > 1 && !p.accumulate) {
    zero_w_entries<<<sms * 4, 256, 0, st>>>(p, w);
    ++g_kernel_launches;
  }
  const int64_t items = rows * ksplit;   // at most; the kernel rounds K ranges to inner blocks
  const int64_t blocks = (items * 32 + THREADS - 1) / THREADS;
  const int64_t cap = resident / (THREADS / 32);
  const int grid = (int)(blocks < cap ? blocks : cap);
  gemm_f64_skinny<NS><<<grid, THREADS, 0, st>>>(p, long_is_u, (int)ksplit, u, v, w);
}

}  // namespace

cudaError_t launch_gemm_f64(const Problem& p, const double* u, const double* v, double* w,
                            const Tables* tables, cudaStream_t st) {
  if (p.n_q == 0 || p.M == 0 || p.N == 0) return cudaSuccess;
  const int sms = sm_count();
  const int64_t target = (int64_t)sms * 2;
  // general plans take the tiled kernel with their tables (every shape)
  bool skinny = !tables && (p.M < 16 || p.N < 16);
  if (skinny && (p.M <= SKINNY_MAX || p.N <= SKINNY_MAX)) {
    bool long_is_u = p.N <= SKINNY_MAX ? true : false;
    // both sides short: an item reads one long-side row and every short-side
    // row along its K range, nL * (1 + nS) rows in all, fewest with the
    // shorter side as the long one
    if (p.M <= SKINNY_MAX && p.N <= SKINNY_MAX) long_is_u = p.M <= p.N;
    const int nS = (int)(long_is_u ? p.N : p.M);
    if (p.K <= kShortK) {
      const int64_t nL = long_is_u ? p.M : p.N;
      const int64_t chunks = (nL + kShortRows - 1) / kShortRows * p.n_q;
      const int kt = p.K == 1 ? 1 : (p.K == 2 ? 2 : 0);
      switch (nS) {
        case 1: launch_shortk_ns<1>(kt, sms, chunks, st, p, long_is_u, u, v, w); break;
        case 2: launch_shortk_ns<2>(kt, sms, chunks, st, p, long_is_u, u, v, w); break;
        case 3: launch_shortk_ns<3>(kt, sms, chunks, st, p, long_is_u, u, v, w); break;
        case 4: launch_shortk_ns<4>(kt, sms, chunks, st, p, long_is_u, u, v, w); break;
        case 5: launch_shortk_ns<5>(kt, sms, chunks, st, p, long_is_u, u, v, w); break;
        case 6: launch_shortk_ns<6>(kt, sms, chunks, st, p, long_is_u, u, v, w); break;
        case 7: launch_shortk_ns<7>(kt, sms, chunks, st, p, long_is_u, u, v, w); break;
        default: launch_shortk_ns<8>(kt, sms, chunks, st, p, long_is_u, u, v, w); break;
      }
      ++g_kernel_launches;
      return cudaGetLastError();
    }
    switch (nS) {
      case 1: launch_skinny_ns<1>(sms, st, p, long_is_u, u, v, w); break;
      case 2: launch_skinny_ns<2>(sms, st, p, long_is_u, u, v, w); break;
      case 3: launch_skinny_ns<3>(sms, st, p, long_is_u, u, v, w); break;
      case 4: launch_skinny_ns<4>(sms, st, p, long_is_u, u, v, w); break;
      case 5: launch_skinny_ns<5>(sms, st, p, long_is_u, u, v, w); break;
      case 6: launch_skinny_ns<6>(sms, st, p, long_is_u, u, v, w); break;
      case 7: launch_skinny_ns<7>(sms, st, p, long_is_u, u, v, w); break;
      default: launch_skinny_ns<8>(sms, st, p, long_is_u, u, v, w); break;
    }
    ++g_kernel_launches;
    return cudaGetLastError();
  }
  int64_t tiles = ((p.M + BM - 1) / BM) * ((p.N + BN - 1) / BN) * p.n_q;
  int ksplit = 1;
  while (tiles * ksplit < target && p.K / (ksplit * 2) >= 512) ksplit *= 2;
  // (a general plan's W is zeroed as a whole before its contraction)
  if (ksplit > 1 && !p.accumulate && !tables) {
    zero_w_entries<<<sms * 4, 256, 0, st>>>(p, w);
    ++g_kernel_launches;
  }
  Tables t{};
  if (tables) t = *tables;
  int64_t blocks = tiles * ksplit;
  int64_t cap = (int64_t)sms * 4;
  gemm_f64_tiled<<<(int)(blocks < cap ? blocks : cap), THREADS, 0, st>>>(
      p, ksplit, map_rows_fast(p.u.rows), map_rows_fast(p.v.rows), t, u, v, w);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace symctr
