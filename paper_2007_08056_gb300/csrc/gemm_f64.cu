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
// memory and each lane recomputes aoff(o * I) only when o changes
// (every I / 32 steps), instead of one mixed-radix decomposition per element.
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

// inner(i) for i < I: the block digits of i over the fastest block axes.
__device__ void fill_inner(const AxisMap& a, int64_t I, int64_t* tab) {
  for (int64_t i = threadIdx.x; i < I; i += blockDim.x) {
    int64_t r = i, off = 0;
    for (int d = a.n - 1; d >= 0 && r > 0; --d) {
      off += (r % a.D[d]) * a.bstride[d];
      r /= a.D[d];
    }
    tab[i] = off;
  }
}

// NS = the short side's row count (one instance per count, so that no
// float64 instruction of an absent row is issued: GB300's float64 pipe is
// narrow and issues predicated-off instructions all the same).
template <int NS>
__global__ void __launch_bounds__(THREADS) gemm_f64_skinny(const __grid_constant__ Problem p, bool long_is_u, int ksplit,
                                                           const double* __restrict__ U,
                                                           const double* __restrict__ V,
                                                           double* __restrict__ W) {
  __shared__ int64_t tab_l[kInnerMax], tab_s[kInnerMax];
  const AxisMap& Lrows = long_is_u ? p.u.rows : p.v.rows;
  const AxisMap& Lcols = long_is_u ? p.u.cols : p.v.cols;
  const AxisMap& Srows = long_is_u ? p.v.rows : p.u.rows;
  const AxisMap& Scols = long_is_u ? p.v.cols : p.u.cols;
  const double* Lp = long_is_u ? U : V;
  const double* Sp = long_is_u ? V : U;
  const int64_t nL = long_is_u ? p.M : p.N;
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t I = inner_extent(Lcols, Scols);
  // K ranges start on multiples of I (K itself is one), so that a range
  // covers whole inner blocks when I >= 32
  const int64_t kchunk = ((p.K + ksplit - 1) / ksplit + I - 1) / I * I;
  const int64_t items = nL * p.n_q * ksplit;
  fill_inner(Lcols, I, tab_l);
  fill_inner(Scols, I, tab_s);
  __syncthreads();
  for (int64_t it = warp; it < items; it += nwarps) {
    int64_t ks = it % ksplit;
    int64_t t2 = it / ksplit;
    int64_t b = t2 / nL;
    int64_t l = t2 - b * nL;
    int Q = batch_irrep(p, (int)b);
    int64_t kbeg = ks * kchunk, kend = kbeg + kchunk < p.K ? kbeg + kchunk : p.K;
    int64_t loff = aoff(Lrows, p.g, Q, l);
    int64_t soff[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) soff[s] = aoff(Srows, p.g, Q, s);
    double acc[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) acc[s] = 0.0;
    if (I >= 32) {
      // whole inner blocks (kend is a multiple of I): lane j computes the two
      // offsets of inner block ob + j, for 32 blocks at once, and the warp
      // walks them with kUnroll independent loads per lane in flight
      constexpr int kUnroll = 4;
      for (int64_t ob = kbeg / I; ob * I < kend; ob += 32) {
        const int64_t oj = ob + lane;
        const bool own = oj * I < kend;
        const int64_t lo_j = own ? loff + aoff(Lcols, p.g, Q, oj * I) : 0;
        const int64_t so_j = own ? aoff(Scols, p.g, Q, oj * I) : 0;
        const int64_t left = (kend - ob * I) / I;
        const int nb = left < 32 ? (int)left : 32;
        for (int j = 0; j < nb; ++j) {
          const int64_t lo = __shfl_sync(0xffffffffu, lo_j, j);
          const int64_t so = __shfl_sync(0xffffffffu, so_j, j);
          for (int64_t i0 = lane; i0 < I; i0 += 32 * kUnroll) {
            double x[kUnroll];
            int64_t sc[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
              const int64_t i = i0 + 32 * u;
              const bool in = i < I;
              x[u] = in ? Lp[p.es * (lo + tab_l[i])] : 0.0;
              sc[u] = in ? so + tab_s[i] : -1;
            }
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
              for (int s = 0; s < NS; ++s)
                if (sc[u] >= 0) acc[s] = fma(x[u], Sp[p.es * (soff[s] + sc[u])], acc[s]);
            }
          }
        }
      }
    } else {
      int64_t k = kbeg + lane;
      int64_t o = k / I, i = k - o * I;
      int64_t lo = aoff(Lcols, p.g, Q, o * I), so = aoff(Scols, p.g, Q, o * I);
      for (; k < kend; k += 32) {
        const double x = Lp[p.es * (loff + lo + tab_l[i])];
        const int64_t sc = so + tab_s[i];
#pragma unroll
        for (int s = 0; s < NS; ++s)
          acc[s] = fma(x, Sp[p.es * (soff[s] + sc)], acc[s]);
        i += 32;
        if (i >= I) {
          o += i / I;
          i %= I;
          if (k + 32 < kend) {
            lo = aoff(Lcols, p.g, Q, o * I);
            so = aoff(Scols, p.g, Q, o * I);
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
    if (lane == 0) {
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        int64_t m = long_is_u ? l : s, n = long_is_u ? s : l;
        double* dst = W + p.es * (aoff(p.w.rows, p.g, Q, m) + aoff(p.w.cols, p.g, Q, n));
        if (ksplit > 1) atomicAdd(dst, signed_result(p, acc[s]));
        else store_w(p, dst, acc[s]);
      }
    }
  }
}

// Skinny problems with K <= kShortK: one thread per row of the long side, a
// block taking kShortRows consecutive rows at a time (kShortRows / THREADS
// per thread).  The short side's values and the long side's column offsets
// depend only on the irrep, so a block stages them in shared memory when the
// irrep changes.  Row offsets in L and W use the inner-block split of the
// skinny kernel above (l = o * I + i): a table of inner(i) per map, and
// aoff(o * I) for the inner blocks of a chunk computed by as many
// threads at once (the index arithmetic of one offset is a long dependent
// chain under a product group, so it is never left to a single thread).
constexpr int kShortK = 32;
constexpr int kShortRows = 4096;
constexpr int kShortSlots = kShortRows / 32 + 2;

template <int NS>
__global__ void __launch_bounds__(THREADS) gemm_f64_shortk(const __grid_constant__ Problem p, bool long_is_u,
                                                           const double* __restrict__ U,
                                                           const double* __restrict__ V,
                                                           double* __restrict__ W) {
  __shared__ double sval[SKINNY_MAX][kShortK];
  __shared__ int64_t lco[kShortK];
  __shared__ int64_t wso[SKINNY_MAX];
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
  constexpr int nS = NS;   // the launcher picks the instance with NS == the short side
  const int K = (int)p.K;
  const int64_t per_q = (nL + kShortRows - 1) / kShortRows;
  // the rows of L and W's axis along the long side index the same modes
  const int64_t I = inner_extent(Lrows, Wl);
  const bool tabulated = I >= 32;   // then a chunk touches <= kShortSlots inner blocks
  if (tabulated) {
    fill_inner(Lrows, I, tab_lr);
    fill_inner(Wl, I, tab_w);
  }
  int staged = -1;
  for (int64_t blk = blockIdx.x; blk < per_q * p.n_q; blk += gridDim.x) {
    const int b = (int)(blk / per_q);
    const int64_t l0 = (blk - (int64_t)b * per_q) * kShortRows;
    const int64_t lend = l0 + kShortRows < nL ? l0 + kShortRows : nL;
    const int64_t o0 = l0 / I;
    const int Q = batch_irrep(p, b);
    __syncthreads();   // the previous chunk's readers are done
    if (b != staged) {
      for (int i = threadIdx.x; i < nS * K; i += THREADS) {
        const int sr = i / K, k = i - sr * K;
        sval[sr][k] = Sp[p.es * (aoff(Srows, p.g, Q, sr) + aoff(Scols, p.g, Q, k))];
      }
      for (int k = threadIdx.x; k < K; k += THREADS) lco[k] = aoff(Lcols, p.g, Q, k);
      for (int sr = threadIdx.x; sr < nS; sr += THREADS) wso[sr] = aoff(Ws, p.g, Q, sr);
      staged = b;
    }
    if (tabulated) {
      const int64_t n_o = (lend - 1) / I - o0 + 1;
      for (int64_t j = threadIdx.x; j < n_o; j += THREADS) {
        ob_l[j] = aoff(Lrows, p.g, Q, (o0 + j) * I);
        ob_w[j] = aoff(Wl, p.g, Q, (o0 + j) * I);
      }
    }
    __syncthreads();
    // (o, i) of the thread's first row by one division; later rows step by
    // THREADS without dividing (64-bit integer division runs on GB300's
    // narrow float64 pipe)
    int64_t o = tabulated ? (l0 + threadIdx.x) / I : 0;
    int64_t i = tabulated ? l0 + threadIdx.x - o * I : 0;
    for (int64_t l = l0 + threadIdx.x; l < lend; l += THREADS) {
      int64_t loff, woff;
      if (tabulated) {
        loff = ob_l[o - o0] + tab_lr[i];
        woff = ob_w[o - o0] + tab_w[i];
        i += THREADS;
        while (i >= I) {
          i -= I;
          ++o;
        }
      } else {
        loff = aoff(Lrows, p.g, Q, l);
        woff = aoff(Wl, p.g, Q, l);
      }
      double acc[NS];
#pragma unroll
      for (int sr = 0; sr < NS; ++sr) acc[sr] = 0.0;
      for (int k = 0; k < K; ++k) {
        const double x = Lp[p.es * (loff + lco[k])];
#pragma unroll
        for (int sr = 0; sr < NS; ++sr)
          acc[sr] = fma(x, sval[sr][k], acc[sr]);
      }
#pragma unroll
      for (int sr = 0; sr < NS; ++sr)
        store_w(p, W + p.es * (woff + wso[sr]), acc[sr]);
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
    if (p.K <= kShortK) {
      const int64_t nL = long_is_u ? p.M : p.N;
      const int64_t blocks = (nL + kShortRows - 1) / kShortRows * p.n_q;
      const int64_t cap = (int64_t)sms * 16;
      const int grid = (int)(blocks < cap ? blocks : cap), nS = (int)(long_is_u ? p.N : p.M);
      switch (nS) {
        case 1: gemm_f64_shortk<1><<<grid, THREADS, 0, st>>>(p, long_is_u, u, v, w); break;
        case 2: gemm_f64_shortk<2><<<grid, THREADS, 0, st>>>(p, long_is_u, u, v, w); break;
        case 3: gemm_f64_shortk<3><<<grid, THREADS, 0, st>>>(p, long_is_u, u, v, w); break;
        case 4: gemm_f64_shortk<4><<<grid, THREADS, 0, st>>>(p, long_is_u, u, v, w); break;
        case 5: gemm_f64_shortk<5><<<grid, THREADS, 0, st>>>(p, long_is_u, u, v, w); break;
        case 6: gemm_f64_shortk<6><<<grid, THREADS, 0, st>>>(p, long_is_u, u, v, w); break;
        case 7: gemm_f64_shortk<7><<<grid, THREADS, 0, st>>>(p, long_is_u, u, v, w); break;
        default: gemm_f64_shortk<8><<<grid, THREADS, 0, st>>>(p, long_is_u, u, v, w); break;
      }
      ++g_kernel_launches;
      return cudaGetLastError();
    }
    int64_t nL = long_is_u ? p.M : p.N;
    int64_t warps = nL * p.n_q;
    int ksplit = 1;
    int64_t want_warps = (int64_t)sms * (THREADS / 32) * 4;
    while (warps * ksplit < want_warps && p.K / (ksplit * 2) >= 256) ksplit *= 2;
    if (ksplit > 1 && !p.accumulate) {
      zero_w_entries<<<sms * 4, 256, 0, st>>>(p, w);
      ++g_kernel_launches;
    }
    int64_t blocks = (warps * ksplit * 32 + THREADS - 1) / THREADS;
    int64_t cap = (int64_t)sms * 16;
    const int grid = (int)(blocks < cap ? blocks : cap), nS = (int)(long_is_u ? p.N : p.M);
    switch (nS) {
      case 1: gemm_f64_skinny<1><<<grid, THREADS, 0, st>>>(p, long_is_u, ksplit, u, v, w); break;
      case 2: gemm_f64_skinny<2><<<grid, THREADS, 0, st>>>(p, long_is_u, ksplit, u, v, w); break;
      case 3: gemm_f64_skinny<3><<<grid, THREADS, 0, st>>>(p, long_is_u, ksplit, u, v, w); break;
      case 4: gemm_f64_skinny<4><<<grid, THREADS, 0, st>>>(p, long_is_u, ksplit, u, v, w); break;
      case 5: gemm_f64_skinny<5><<<grid, THREADS, 0, st>>>(p, long_is_u, ksplit, u, v, w); break;
      case 6: gemm_f64_skinny<6><<<grid, THREADS, 0, st>>>(p, long_is_u, ksplit, u, v, w); break;
      case 7: gemm_f64_skinny<7><<<grid, THREADS, 0, st>>>(p, long_is_u, ksplit, u, v, w); break;
      default: gemm_f64_skinny<8><<<grid, THREADS, 0, st>>>(p, long_is_u, ksplit, u, v, w); break;
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
