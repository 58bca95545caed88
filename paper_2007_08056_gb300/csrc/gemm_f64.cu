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

__host__ __device__ inline bool map_rows_fast(const AxisMap& rows) {
  return rows.n > 0 && rows.bstride[rows.n - 1] == 1;
}

__global__ void __launch_bounds__(THREADS) gemm_f64_tiled(Problem p, int ksplit, bool u_rows_fast,
                                                          bool v_rows_fast,
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
    if (tid < BM) {
      int64_t m = m0 + tid;
      uoff[tid] = m < p.M ? axis_offset(p.u.rows, p.g, Q, m) : 0;
      woffr[tid] = m < p.M ? axis_offset(p.w.rows, p.g, Q, m) : 0;
    } else if (tid < BM + BN) {
      int64_t n = n0 + tid - BM;
      voff[tid - BM] = n < p.N ? axis_offset(p.v.rows, p.g, Q, n) : 0;
      woffc[tid - BM] = n < p.N ? axis_offset(p.w.cols, p.g, Q, n) : 0;
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
        kuoff[tid] = k < kend ? axis_offset(p.u.cols, p.g, Q, k) : 0;
      } else if (tid >= 32 && tid < 32 + BK) {
        int64_t k = k0 + tid - 32;
        kvoff[tid - 32] = k < kend ? axis_offset(p.v.cols, p.g, Q, k) : 0;
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < (BM * BK) / THREADS; ++j) {
        int e = tid + j * THREADS;
        int mm = u_rows_fast ? e % BM : e / BK;
        int kk = u_rows_fast ? e / BM : e % BK;
        double x = 0.0;
        if (m0 + mm < p.M && k0 + kk < kend) x = U[p.es * (uoff[mm] + kuoff[kk])];
        As[kk][mm] = x;
      }
#pragma unroll
      for (int j = 0; j < (BN * BK) / THREADS; ++j) {
        int e = tid + j * THREADS;
        int nn = v_rows_fast ? e % BN : e / BK;
        int kk = v_rows_fast ? e / BN : e % BK;
        double x = 0.0;
        if (n0 + nn < p.N && k0 + kk < kend) x = V[p.es * (voff[nn] + kvoff[kk])];
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
      if (m0 + mm >= p.M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int nn = tc + 16 * j;
        if (n0 + nn >= p.N) continue;
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
constexpr int SKINNY_MAX = 8;

__global__ void __launch_bounds__(THREADS) gemm_f64_skinny(Problem p, bool long_is_u, int ksplit,
                                                           const double* __restrict__ U,
                                                           const double* __restrict__ V,
                                                           double* __restrict__ W) {
  const AxisMap& Lrows = long_is_u ? p.u.rows : p.v.rows;
  const AxisMap& Lcols = long_is_u ? p.u.cols : p.v.cols;
  const AxisMap& Srows = long_is_u ? p.v.rows : p.u.rows;
  const AxisMap& Scols = long_is_u ? p.v.cols : p.u.cols;
  const double* Lp = long_is_u ? U : V;
  const double* Sp = long_is_u ? V : U;
  const int64_t nL = long_is_u ? p.M : p.N;
  const int nS = (int)(long_is_u ? p.N : p.M);
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t kchunk = (p.K + ksplit - 1) / ksplit;
  const int64_t items = nL * p.n_q * ksplit;
  for (int64_t it = warp; it < items; it += nwarps) {
    int64_t ks = it % ksplit;
    int64_t t2 = it / ksplit;
    int64_t b = t2 / nL;
    int64_t l = t2 - b * nL;
    int Q = batch_irrep(p, (int)b);
    int64_t kbeg = ks * kchunk, kend = kbeg + kchunk < p.K ? kbeg + kchunk : p.K;
    int64_t loff = axis_offset(Lrows, p.g, Q, l);
    int64_t soff[SKINNY_MAX];
#pragma unroll
    for (int s = 0; s < SKINNY_MAX; ++s) soff[s] = s < nS ? axis_offset(Srows, p.g, Q, s) : 0;
    double acc[SKINNY_MAX];
#pragma unroll
    for (int s = 0; s < SKINNY_MAX; ++s) acc[s] = 0.0;
    for (int64_t k = kbeg + lane; k < kend; k += 32) {
      double x = Lp[p.es * (loff + axis_offset(Lcols, p.g, Q, k))];
      int64_t sc = axis_offset(Scols, p.g, Q, k);
#pragma unroll
      for (int s = 0; s < SKINNY_MAX; ++s)
        if (s < nS) acc[s] = fma(x, Sp[p.es * (soff[s] + sc)], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < SKINNY_MAX; ++s) {
      double a = acc[s];
      for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      acc[s] = a;
    }
    if (lane == 0) {
      for (int s = 0; s < nS; ++s) {
        int64_t m = long_is_u ? l : s, n = long_is_u ? s : l;
        double* dst = W + p.es * (axis_offset(p.w.rows, p.g, Q, m) + axis_offset(p.w.cols, p.g, Q, n));
        if (ksplit > 1) atomicAdd(dst, signed_result(p, acc[s]));
        else store_w(p, dst, acc[s]);
      }
    }
  }
}

// Skinny problems with K <= kShortK: one thread per row of the long side.  The
// short side's values and the long side's column offsets depend only on the
// irrep, so each block stages them in shared memory once per irrep; a thread
// then computes two offsets (its row in L and in W) and K loads.
constexpr int kShortK = 32;

__global__ void __launch_bounds__(THREADS) gemm_f64_shortk(Problem p, bool long_is_u,
                                                           const double* __restrict__ U,
                                                           const double* __restrict__ V,
                                                           double* __restrict__ W) {
  __shared__ double sval[SKINNY_MAX][kShortK];
  __shared__ int64_t lco[kShortK];
  __shared__ int64_t wso[SKINNY_MAX];
  const AxisMap& Lrows = long_is_u ? p.u.rows : p.v.rows;
  const AxisMap& Lcols = long_is_u ? p.u.cols : p.v.cols;
  const AxisMap& Srows = long_is_u ? p.v.rows : p.u.rows;
  const AxisMap& Scols = long_is_u ? p.v.cols : p.u.cols;
  const AxisMap& Wl = long_is_u ? p.w.rows : p.w.cols;
  const AxisMap& Ws = long_is_u ? p.w.cols : p.w.rows;
  const double* Lp = long_is_u ? U : V;
  const double* Sp = long_is_u ? V : U;
  const int64_t nL = long_is_u ? p.M : p.N;
  const int nS = (int)(long_is_u ? p.N : p.M);
  const int K = (int)p.K;
  const int64_t per_q = (nL + THREADS - 1) / THREADS;
  for (int64_t blk = blockIdx.x; blk < per_q * p.n_q; blk += gridDim.x) {
    const int b = (int)(blk / per_q);
    const int64_t l = (blk - (int64_t)b * per_q) * THREADS + threadIdx.x;
    const int Q = batch_irrep(p, b);
    __syncthreads();   // the previous irrep's readers are done
    for (int i = threadIdx.x; i < nS * K; i += THREADS) {
      const int sr = i / K, k = i - sr * K;
      sval[sr][k] = Sp[p.es * (axis_offset(Srows, p.g, Q, sr) + axis_offset(Scols, p.g, Q, k))];
    }
    for (int k = threadIdx.x; k < K; k += THREADS) lco[k] = axis_offset(Lcols, p.g, Q, k);
    for (int sr = threadIdx.x; sr < nS; sr += THREADS) wso[sr] = axis_offset(Ws, p.g, Q, sr);
    __syncthreads();
    if (l < nL) {
      const int64_t loff = axis_offset(Lrows, p.g, Q, l);
      const int64_t woff = axis_offset(Wl, p.g, Q, l);
      double acc[SKINNY_MAX];
#pragma unroll
      for (int sr = 0; sr < SKINNY_MAX; ++sr) acc[sr] = 0.0;
      for (int k = 0; k < K; ++k) {
        const double x = Lp[p.es * (loff + lco[k])];
#pragma unroll
        for (int sr = 0; sr < SKINNY_MAX; ++sr)
          if (sr < nS) acc[sr] = fma(x, sval[sr][k], acc[sr]);
      }
#pragma unroll
      for (int sr = 0; sr < SKINNY_MAX; ++sr)
        if (sr < nS) store_w(p, W + p.es * (woff + wso[sr]), acc[sr]);
    }
  }
}

int sm_count() {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

// Zero the entries of W that a split-K launch accumulates into.
__global__ void zero_w_entries(Problem p, double* __restrict__ W) {
  int64_t total = (int64_t)p.n_q * p.M * p.N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = i / (p.M * p.N);
    int64_t r = i - b * p.M * p.N;
    int64_t m = r / p.N, n = r % p.N;
    int Q = batch_irrep(p, (int)b);
    W[p.es * (axis_offset(p.w.rows, p.g, Q, m) + axis_offset(p.w.cols, p.g, Q, n))] = 0.0;
  }
}

}  // namespace

cudaError_t launch_gemm_f64(const Problem& p, const double* u, const double* v, double* w,
                            cudaStream_t st) {
  if (p.n_q == 0 || p.M == 0 || p.N == 0) return cudaSuccess;
  const int sms = sm_count();
  const int64_t target = (int64_t)sms * 2;
  bool skinny = p.M < 16 || p.N < 16;
  if (skinny && (p.M <= SKINNY_MAX || p.N <= SKINNY_MAX)) {
    bool long_is_u = p.N <= SKINNY_MAX ? true : false;
    if (p.M <= SKINNY_MAX && p.N <= SKINNY_MAX) long_is_u = p.M >= p.N;
    if (p.K <= kShortK) {
      const int64_t nL = long_is_u ? p.M : p.N;
      const int64_t blocks = (nL + THREADS - 1) / THREADS * p.n_q;
      const int64_t cap = (int64_t)sms * 16;
      gemm_f64_shortk<<<(int)(blocks < cap ? blocks : cap), THREADS, 0, st>>>(p, long_is_u, u, v, w);
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
    gemm_f64_skinny<<<(int)(blocks < cap ? blocks : cap), THREADS, 0, st>>>(p, long_is_u, ksplit, u,
                                                                             v, w);
    ++g_kernel_launches;
    return cudaGetLastError();
  }
  int64_t tiles = ((p.M + BM - 1) / BM) * ((p.N + BN - 1) / BN) * p.n_q;
  int ksplit = 1;
  while (tiles * ksplit < target && p.K / (ksplit * 2) >= 512) ksplit *= 2;
  if (ksplit > 1 && !p.accumulate) {
    zero_w_entries<<<sms * 4, 256, 0, st>>>(p, w);
    ++g_kernel_launches;
  }
  int64_t blocks = tiles * ksplit;
  int64_t cap = (int64_t)sms * 4;
  gemm_f64_tiled<<<(int)(blocks < cap ? blocks : cap), THREADS, 0, st>>>(
      p, ksplit, map_rows_fast(p.u.rows), map_rows_fast(p.v.rows), u, v, w);
  ++g_kernel_launches;
  return cudaGetLastError();
}

}  // namespace symctr
