// Internal declarations shared by the planner (plan.cpp) and the CUDA kernels.
//
// Index maps.  Every transformation of Algorithm 2 (std reduced form <->
// aligned form, for U, V and W) is a *separable* gather: an aligned element
// (Q, r, c) lives at reduced-form offset row_off(Q, r) + col_off(Q, c).  This
// holds because the implicit sector of the row modes depends only on Q and the
// explicit row sectors, and likewise for the column modes (uniqueness of Q in
// the proof of Sec. 2.3).  An AxisMap describes one side.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "symctr.h"

#if defined(__CUDACC__)
#define SC_HD __host__ __device__ __forceinline__
#else
#define SC_HD inline
#endif

namespace symctr {

// Z_m1 x ... x Z_mr, labels flattened mixed-radix, first modulus most significant.
struct GroupDesc {
  int n;
  int mod[SYMCTR_MAX_MODULI];
  int order;
};

SC_HD int g_add(const GroupDesc& g, int a, int b) {
  if (g.n == 1) { int r = a + b; return r >= g.order ? r - g.order : r; }
  int out = 0, scale = 1;
  for (int i = g.n - 1; i >= 0; --i) {
    int m = g.mod[i];
    int x = (a % m + b % m) % m;
    out += x * scale;
    scale *= m;
    a /= m;
    b /= m;
  }
  return out;
}

SC_HD int g_neg(const GroupDesc& g, int a) {
  if (g.n == 1) return a == 0 ? 0 : g.order - a;
  int out = 0, scale = 1;
  for (int i = g.n - 1; i >= 0; --i) {
    int m = g.mod[i];
    int x = a % m;
    out += (x == 0 ? 0 : m - x) * scale;
    scale *= m;
    a /= m;
  }
  return out;
}

SC_HD int g_signed(const GroupDesc& g, int sign, int a) { return sign > 0 ? a : g_neg(g, a); }

// One side (rows or columns) of an aligned operand.
struct AxisMap {
  int n;                                // modes in this group
  int64_t size;                         // G^(n-1) * prod D  (1 if n == 0)
  int D[SYMCTR_MAX_ORDER];
  int sign[SYMCTR_MAX_ORDER];           // law coefficients used to solve the implicit sector
  int64_t sstride[SYMCTR_MAX_ORDER];    // reduced-form stride of the sector axis (0: not stored)
  int64_t bstride[SYMCTR_MAX_ORDER];    // reduced-form stride of the block axis
  int qa;                               // sum_i sign_i q_i == qa*Q + z  (qa = +-1)
  int z;
};

// Offset contribution of aligned index r at irrep Q.  Axes below 2^31
// entries (all practical ones) take 32-bit divisions.
//
// Under a product group Z_m1 x ... x Z_mr the conservation law holds factor by
// factor, so the sector labels are split into their factor digits straight
// from r (one division per factor), the signed digit sums are kept per factor
// without reduction, and the implicit sector's digits are reduced once at the
// end: a handful of divisions per mode instead of the label arithmetic of
// g_add / g_neg at every step.
template <typename I>
SC_HD int64_t axis_offset_t(const AxisMap& a, const GroupDesc& g, int Q, I r) {
  int64_t off = 0;
  for (int i = a.n - 1; i >= 0; --i) {
    const I d = (I)a.D[i];
    const I q = r / d;
    off += (int64_t)(r - q * d) * a.bstride[i];
    r = q;
  }
  if (g.n == 1) {
    int partial = 0;
    for (int i = a.n - 2; i >= 0; --i) {
      const I q = r / (I)g.order;
      const int s = (int)(r - q * (I)g.order);
      r = q;
      off += (int64_t)s * a.sstride[i];
      partial = g_add(g, partial, g_signed(g, a.sign[i], s));
    }
    int target = g_add(g, g_signed(g, a.qa, Q), a.z);
    int last = g_signed(g, a.sign[a.n - 1], g_add(g, target, g_neg(g, partial)));
    off += (int64_t)last * a.sstride[a.n - 1];
    return off;
  }
  // part[k]: the signed digit sum of factor g.n - 1 - k (indexed by the
  // unrolled counter, so that it stays in registers)
  int part[SYMCTR_MAX_MODULI];
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
  for (int k = 0; k < SYMCTR_MAX_MODULI; ++k) part[k] = 0;
  for (int i = a.n - 2; i >= 0; --i) {
    int s = 0, scale = 1;
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
    for (int k = 0; k < SYMCTR_MAX_MODULI; ++k) {
      if (k < g.n) {
        const int mf = g.mod[g.n - 1 - k];
        const I m = (I)mf;
        const I q = r / m;
        const int d = (int)(r - q * m);
        r = q;
        s += d * scale;
        scale *= mf;
        part[k] += a.sign[i] > 0 ? d : -d;
      }
    }
    off += (int64_t)s * a.sstride[i];
  }
  // digit f of the implicit sector: sign_last * (qa * Q_f + z_f - part_f) mod m_f
  int last = 0, scale = 1, qr = Q, zr = a.z;
#if defined(__CUDA_ARCH__)
#pragma unroll
#endif
  for (int k = 0; k < SYMCTR_MAX_MODULI; ++k) {
    if (k < g.n) {
      const int m = g.mod[g.n - 1 - k];
      const int qf = qr % m, zf = zr % m;
      qr /= m;
      zr /= m;
      int x = (a.qa > 0 ? qf : -qf) + zf - part[k];
      if (!(a.sign[a.n - 1] > 0)) x = -x;
      x %= m;
      if (x < 0) x += m;
      last += x * scale;
      scale *= m;
    }
  }
  off += (int64_t)last * a.sstride[a.n - 1];
  return off;
}

SC_HD int64_t axis_offset(const AxisMap& a, const GroupDesc& g, int Q, int64_t r) {
  if (a.n == 0) return 0;
  if (a.size <= 0x7FFFFFFF) return axis_offset_t<uint32_t>(a, g, Q, (uint32_t)r);
  return axis_offset_t<int64_t>(a, g, Q, r);
}

struct OperandMap {
  AxisMap rows, cols;
};

// Everything a kernel needs to locate the aligned GEMM problem.
struct Problem {
  GroupDesc g;
  int n_q;            // batches (irreps carrying work)
  int q_single;       // the irrep of a single-irrep problem, else -1
  int q_base;         // batch index of this pass's batch 0 (Q-streaming)
  int q0 = 0;         // batch b is irrep q0 + b * q_step (mod G) when q_single < 0
  int q_step = 1;
  // General symmetry (sub-group coefficients or padded sectors): the index
  // maps live only in the offset tables, where an absent aligned row or
  // column (an implicit-sector equation without a solution, or a padding
  // position) has offset -1; kernels read it as zero and never store it.
  int general = 0;
  int64_t M, N, K;
  OperandMap u, v, w; // U: rows = free-U, cols = contracted; V: rows = free-V, cols = contracted;
                      // W: rows = free-U, cols = free-V
  // element stride of U, V and W in doubles: 1 for real data, 2 when the
  // reduced forms hold interleaved complex entries and the pointers address
  // their real or imaginary parts
  int es = 1;
  int negate = 0;     // W = (-)result, or W += (-)result when accumulate
  int accumulate = 0;
};

#ifdef __CUDACC__
// The result with the problem's sign: a flip of the sign bit, as an integer
// XOR in inline PTX.  Written in C++, the conditional XOR may be folded into a
// float64 negation, which GB300 issues on its narrow float64 pipe for every
// stored value.
__device__ __forceinline__ double signed_result(const Problem& p, double x) {
  const unsigned mask = p.negate ? 0x80000000u : 0u;
  unsigned hi = (unsigned)__double2hiint(x);
  asm("xor.b32 %0, %0, %1;" : "+r"(hi) : "r"(mask));
  return __hiloint2double((int)hi, __double2loint(x));
}

// Store of one result into W under the problem's output mode.  The
// accumulating store is a float64 atomic add (performed in L2, each entry
// with a single writer: the same rounded sum), so that neither mode puts a
// float64 add on the narrow float64 pipe.
__device__ __forceinline__ void store_w(const Problem& p, double* dst, double x) {
  x = signed_result(p, x);
  if (p.accumulate)
    atomicAdd(dst, x);
  else
    *dst = x;
}
#endif

SC_HD int batch_irrep(const Problem& p, int b) {
  return p.q_single >= 0 ? p.q_single : (p.q0 + (p.q_base + b) * p.q_step) % p.g.order;
}

// Offset tables of the aligned forms for one contraction pass: row_off /
// col_off of every (batch, index), int64.  They are computed once per plan on
// the host and read in place through the device view of page-locked host
// memory, or copied into the workspace where that view is unavailable.
struct Tables {
  const int64_t* urow;  // [n_q][M]
  const int64_t* ucol;  // [n_q][K]
  const int64_t* vrow;  // [n_q][N]
  const int64_t* vcol;  // [n_q][K]
  const int64_t* wrow;  // [n_q][M]
  const int64_t* wcol;  // [n_q][N]
};

SC_HD int64_t tables_entries(const Problem& p) {
  return (int64_t)p.n_q * (2 * p.M + 2 * p.N + 2 * p.K);
}

// Exponent scan of the operand preparation: aligned rows are scanned in
// tiles of 32 rows by at most kScanWidth columns, the K range cut into
// `prep_scan_parts` column blocks (also enough of them to give the GPU some
// 8192 tiles); each block writes its own partial row maxima ([parts][n_q *
// (M + N)] int32 in the workspace, when parts > 1).
constexpr int kScanWidth = 1024;
inline int prep_scan_parts(const Problem& p) {
  const int64_t row_tiles = ((p.M + 31) / 32 + (p.N + 31) / 32) * (int64_t)p.n_q;
  const int64_t col_blocks = (p.K + 255) / 256;
  int64_t parts = row_tiles > 0 ? (8192 + row_tiles - 1) / row_tiles : 1;
  const int64_t by_width = (p.K + kScanWidth - 1) / kScanWidth;
  if (parts < by_width) parts = by_width;
  if (parts > col_blocks) parts = col_blocks;
  if (parts > 64) parts = 64;
  return parts < 1 ? 1 : (int)parts;
}

inline int64_t prep_partials_entries(const Problem& p) {
  const int parts = prep_scan_parts(p);
  return parts > 1 ? (int64_t)parts * p.n_q * (p.M + p.N) : 0;
}

// Device error word codes (first uint32 of the workspace).
enum : unsigned { DEVERR_NONE = 0, DEVERR_TIMEOUT = 1, DEVERR_NONFINITE = 2 };

// Split-precision constants.
constexpr int kSliceBits = 8;       // bits per balanced BF16 digit
constexpr int kMaxSlices = 6;
constexpr int kKBlock = 32;         // K per pipeline stage (64-byte rows of BF16)
constexpr int kKChunk = 64;         // K between exact flushes of the top accumulators

// Kernels launched on this host thread (every launcher adds its launches).
extern thread_local long long g_kernel_launches;

// ---- kernel launchers (return cudaError_t of the launch) ----
// `tables` (general plans only, else NULL): the offset tables of all batches.
cudaError_t launch_align_f64(const Problem& p, int operand, int direction, const double* src,
                             double* dst, const Tables* tables, cudaStream_t st);
cudaError_t launch_gemm_f64(const Problem& p, const double* u, const double* v, double* w,
                            const Tables* tables, cudaStream_t st);
cudaError_t launch_fill_zero(double* w, int64_t n, cudaStream_t st);
// skip[op]: operand op is prepared by launch_rowstream or launch_rowtile
// instead (NULL: neither)
cudaError_t launch_prep(const Problem& p, const Tables& t, bool split, int n_slices,
                        const double* u, const double* v, void* ua, void* va, int32_t* eu,
                        int32_t* ev, int32_t* partials, int64_t kpad, unsigned* err, unsigned* barrier,
                        unsigned long long* zero64, int64_t zero64_n, const bool* skip,
                        cudaStream_t st);
// Single-read split-form preparation of operand op (0 = U, 1 = V) whose
// aligned rows are runs of `run` contiguous reduced-form entries and at most
// kRowClusterMaxK long (plan-time eligibility: row_run in plan.cpp); rows
// longer than kRowStreamMaxK take the cluster form.
constexpr int64_t kRowStreamMaxK = 8192;
// Longer rows (up to kRowClusterMaxK) are held by a cluster of up to 8 CTAs,
// each streaming one segment of every row.
constexpr int64_t kRowClusterMaxK = 8 * kRowStreamMaxK;
cudaError_t launch_rowstream(const Problem& p, const Tables& t, int op, int n_slices, int64_t run,
                             const double* src, void* slices, int32_t* exps, int64_t kpad,
                             unsigned* err, cudaStream_t st);
// Single-read split-form preparation of short rows: the operands with on[op]
// set, K <= kRowTileMaxK (padded), 2^rowtile_rows_log2(kpad) whole rows per
// CTA in rowtile_smem_bytes of shared memory; also zeroes zero64 (the split-K
// sums) when no other preparation kernel runs.
constexpr int64_t kRowTileMaxK = 4096;
constexpr int64_t kRowTileElems = 8192;   // aligned entries held per CTA (at most; at least 2 rows)
int rowtile_rows_log2(int64_t kpad);
size_t rowtile_smem_bytes(int64_t K, int64_t kpad);
cudaError_t launch_rowtile(const Problem& p, const Tables& t, int n_slices, const bool* on,
                           const double* u, const double* v, void* ua, void* va, int32_t* eu,
                           int32_t* ev, int64_t kpad, unsigned* err, unsigned long long* zero64,
                           int64_t zero64_n, cudaStream_t st);
cudaError_t launch_bounded_wait_selftest(unsigned* err, long long limit_cycles, cudaStream_t st);
cudaError_t launch_gemm_split(const Problem& p, const Tables& t, int n_slices, const uint16_t* us,
                              const uint16_t* vs, const int32_t* eu, const int32_t* ev,
                              int64_t kpad, double* w, unsigned* err, int ksplit,
                              unsigned long long* wacc, cudaStream_t st);
cudaError_t launch_gemm_tf32(const Problem& p, const Tables& t, const float* u, const float* v,
                             int64_t kpad, double* w, unsigned* err, cudaStream_t st);

// K ranges of the split-BF16 GEMM: enough CTAs to fill the GPU when the
// problem has few 128x128 tiles (deterministic: independent of the device).
// A K range holds at most kMaxChunksPerRange exact drains (int32 running sums).
constexpr int64_t kMaxChunksPerRange = 512;

inline int split_k_ranges(const Problem& p, int64_t kpad) {
  int64_t tiles = ((p.M + 127) / 128) * ((p.N + 127) / 128) * (int64_t)p.n_q;
  int64_t chunks = (kpad + kKChunk - 1) / kKChunk;
  int64_t per = chunks;                         // chunks per range
  if (tiles < 80 && chunks >= 4) {
    int64_t want = (160 + tiles - 1) / tiles;
    per = (chunks + want - 1) / want;
    if (per < 2) per = 2;
  }
  if (per > kMaxChunksPerRange) per = kMaxChunksPerRange;
  return (int)((chunks + per - 1) / per);
}

// The contraction of symctr_contract on a given workspace, the plan's workspace
// size, and the error-detail recorder (defined in plan.cpp).
symctr_status contract_into_workspace(const symctr_plan* P, const double* u, const double* v,
                                      double* w, void* ws, size_t ws_bytes, cudaStream_t st);
uint64_t plan_workspace_bytes(const symctr_plan* P);
uint64_t plan_workspace_bytes_min(const symctr_plan* P);
symctr_status record_error(symctr_status st, const char* detail);
// Device address of the static scratch array on the current device (looked
// up once per device, defined in static_scratch.cu), or NULL with *st set.
void* static_scratch_address(symctr_status* st);

// Shape test of the tensor-core forms: both output sides at least 8 long.
// Below that the aligned GEMM is a GEMV or an outer product; the float64
// kernels then read each long-side entry once, while the split form would
// also write its slices and fill 128-row MMA tiles with a few rows.  Any K
// (padded to 32 with zeros) takes the tensor cores.
inline bool tensor_core_shape(const Problem& p) { return p.M >= 8 && p.N >= 8 && p.K >= 1; }

}  // namespace symctr
