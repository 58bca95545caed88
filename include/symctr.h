/*
 * symctr.h -- C ABI of the irrep-aligned contraction library for tensors with
 * cyclic-group (Z_G, or product of cyclic groups) symmetry, GB300 / sm_103a.
 *
 * The operation (Sec. 2.2, Eq. ctr and Algorithm 2 of "Automatic Transformation
 * of Irreducible Representations for Efficient Contraction of Tensors with
 * Cyclic Group Symmetry"):
 *
 *   W[i.., j..] = sum_{k..} U[i.., k..] V[k.., j..]
 *
 * where each tensor vanishes unless its sector labels obey a conservation law
 * sum_mu c_mu q_mu == Z (mod G), c_mu = +-1 (Eq. symtsr).  Operands and result
 * are passed in STANDARD REDUCED FORM: a C-contiguous float64 array of shape
 * [G]*(N-1) + [D_0, ..., D_{N-1}] whose first N-1 axes are the sector labels of
 * modes 0..N-2 and whose last N axes are the in-block indices; the sector of
 * the last mode is implicit, q_{N-1} = c_{N-1} (Z - sum_{mu<N-1} c_mu q_mu)
 * (Sec. 2.1 and its footnote; API listing of Sec. 3, shape [G,G,G,N,N,N,N]).
 * For a product group Z_m1 x ... x Z_mr a sector label is the mixed-radix
 * flattening of its components, first modulus most significant.
 *
 * Internally each operand is remapped to an aligned form indexed by an
 * auxiliary irrep Q (Sec. 2.1 / Alg. 2): U_hat[Q][m][kappa], V_hat[Q][n][kappa],
 * W_hat[Q][m][n], so that the contraction is one batched GEMM over Q, and the
 * result is mapped back to W's standard reduced form.  Q is defined as
 * Q = sum_{k contracted} c^U_k q_k (mod G).  The aligned layouts are:
 *   m     = (q of free-U modes except the last, b of all free-U modes)
 *   kappa = (q of contracted modes except the last, b of all contracted modes)
 *   n     = (q of free-V modes except the last, b of all free-V modes)
 * sector digits before block digits, C order, modes in the order they appear
 * in U (free-U, contracted) or V (free-V); only the irreps Q that can carry
 * nonzero entries are stored (symctr_plan_info.n_q of them, ascending).
 *
 * Conventions of every call
 *   Ownership : the caller owns every device pointer, the workspace and the
 *               stream.  A plan owns host memory only: its metadata and, for
 *               the tensor-core forms, the offset tables of the aligned forms
 *               (computed at plan creation and page-locked on the first
 *               contraction; read in place when small, else copied into the
 *               workspace by every contraction, unless the caller has
 *               attached a device copy with symctr_plan_attach_tables).  No
 *               call allocates device memory.
 *   Errors    : every call returns a status and never throws across the ABI.
 *               Kernels never trap: a device-side failure (a bounded wait that
 *               expired, a non-finite input) is recorded in the first word of
 *               the workspace and reported by symctr_check_device_error.
 *   Asynchrony: every call that takes a stream is asynchronous on it (the
 *               stream is a cudaStream_t; NULL = legacy default stream).
 *   Data      : float64, C-contiguous, device memory, 16-byte aligned; outputs
 *               are fully overwritten.  Inputs must be finite.
 */
#ifndef SYMCTR_H
#define SYMCTR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SYMCTR_API __attribute__((visibility("default")))
#else
#define SYMCTR_API
#endif

#define SYMCTR_MAX_ORDER 8      /* modes per tensor */
#define SYMCTR_MAX_MODULI 4     /* cyclic factors of the group */
#define SYMCTR_MAX_GROUP 256    /* order of the group */

typedef struct symctr_plan symctr_plan;   /* opaque */

typedef enum {
  SYMCTR_OK = 0,
  SYMCTR_ERR_EINSUM = 1,        /* malformed einsum, repeated or trace/batch labels */
  SYMCTR_ERR_SIGNS = 2,         /* contracted coefficients do not agree up to one sign */
  SYMCTR_ERR_SHAPE = 3,         /* sector dims of a contracted mode differ; bad modulus */
  SYMCTR_ERR_CHARGE = 4,        /* a given output law contradicts the derived one */
  SYMCTR_ERR_UNSUPPORTED = 5,   /* order > 8, group > 256, ... */
  SYMCTR_ERR_NULLPTR = 6,
  SYMCTR_ERR_WORKSPACE = 7,     /* workspace smaller than symctr_plan_info.workspace_bytes */
  SYMCTR_ERR_CUDA = 8,          /* a CUDA runtime/driver call failed */
  SYMCTR_ERR_DEVICE_TIMEOUT = 9,/* a kernel's bounded wait expired */
  SYMCTR_ERR_OVERFLOW = 10,     /* an extent or offset exceeds 64-bit / kernel limits */
  SYMCTR_ERR_NONFINITE = 11,    /* a non-finite input reached the split-precision form */
  SYMCTR_ERR_ARGUMENT = 12      /* any other invalid argument */
} symctr_status;

typedef enum {
  SYMCTR_FP64 = 0,        /* float64 FMA throughout */
  SYMCTR_SPLIT_BF16 = 1,  /* Ozaki-style BF16 slices on tcgen05, exact FP32 partial
                             sums, integer recombination, one rounding to float64 */
  SYMCTR_TF32 = 2         /* operands rounded to TF32 on tcgen05, FP32 accumulation */
} symctr_precision;

typedef struct {
  int32_t order_u, order_v, order_w;
  int32_t s, t, v;              /* free-U, free-V and contracted mode counts (Eq. ctr) */
  int32_t sigma;                /* c^V_k = sigma c^U_k on contracted modes (+-1) */
  int32_t n_moduli;
  int32_t moduli[SYMCTR_MAX_MODULI];
  int32_t group_order;          /* G = product of moduli */
  int32_t precision;            /* symctr_precision */
  int32_t n_slices;             /* BF16 slices per operand (split form), else 0 */
  int8_t signs_w[SYMCTR_MAX_ORDER];
  int32_t charge_w[SYMCTR_MAX_MODULI];
  int64_t dims_w[SYMCTR_MAX_ORDER];
  int64_t numel_u, numel_v, numel_w;   /* elements of the standard reduced forms */
  int64_t M, N, K;              /* aligned GEMM extents per irrep Q */
  int32_t n_q;                  /* irreps Q that carry work (0, 1 or G; general plans: the
                                   irreps of a progression, see q_first / q_step) */
  int32_t q_single;             /* the irrep when n_q == 1, else -1 */
  int64_t aligned_numel_u;      /* n_q * M * K */
  int64_t aligned_numel_v;      /* n_q * N * K */
  int64_t aligned_numel_w;      /* n_q * M * N */
  double useful_flops;          /* 2 * n_q * M * N * K: symmetry-reduced GEMM flops */
  double transform_bytes;       /* algorithmic bytes of the alignment transforms */
  uint64_t workspace_bytes;     /* device workspace for one pass over all irreps Q */
  uint64_t workspace_bytes_backward; /* device workspace symctr_contract_backward needs */
  uint64_t workspace_bytes_min; /* smallest accepted workspace: the contraction then runs
                                   one pass per group of irreps that fits (Q-streaming) */
  uint64_t table_bytes;         /* device buffer symctr_plan_attach_tables takes (0: the
                                   plan has no offset tables, e.g. the float64 form) */
  int32_t tensor_core;          /* 1: the GEMM of the precision form runs on tcgen05;
                                   0: it runs on the float64 CUDA-core kernels (the float64
                                   form, or an aligned GEMM with M or N below 8, e.g. a GEMV,
                                   where the tensor-core forms would gain nothing; the
                                   result is then exact to float64 rounding) */
  int32_t general;              /* 1: some mode has fewer than G sectors or non-uniform
                                   sector sizes (symctr_plan_create_general) */
  int32_t q_first, q_step;      /* batch b of the aligned forms is irrep
                                   Q = q_first + b * q_step (mod G), b < n_q (q_step = 0
                                   when n_q <= 1; 0 and 1 for every plan of
                                   symctr_plan_create with n_q = G) */
  int32_t sectors_w[SYMCTR_MAX_ORDER]; /* sector count of each mode of W */
  int32_t single_read_prep;     /* split form: bit 0 (U) / bit 1 (V) set when that operand's
                                   aligned rows are long contiguous runs and its slices are
                                   prepared by the single-read kernel (one HBM read); bit 2
                                   (U) / bit 3 (V) set when that operand's whole rows are
                                   read once by the short-row kernel instead: K (padded) at
                                   most 4096, or at most 2048 for rows that are the reduced
                                   form's unit-stride side or long runs (real data; complex
                                   data takes the two-phase kernel) */
  int32_t chained;              /* 1 after symctr_plan_chain re-laid the plan out (numel_u,
                                   numel_v, numel_w then count the chained layouts) */
  int64_t zero_fill_numel;      /* entries of W a contraction zeroes before the GEMM writes
                                   the rest (Alg. 2's output step: entries of irreps that
                                   carry no work are zero): 0 when the irreps cover W;
                                   numel_w for general plans; otherwise the sector blocks
                                   of W that no irrep writes (uniform plans of at most 8192
                                   sector combinations; numel_w beyond) */
} symctr_plan_info;

/* One operand in the general form of Eq. symtsr, for symctr_plan_create_general.
 *  signs       : [order] sign of each mode's coefficient (+1 / -1).
 *  charge      : [n_moduli] remainder Z.
 *  dims        : [order] block size D of each mode; with non-uniform sectors the
 *                padded size (every block is stored padded to D).
 *  sectors     : [order] sector count H of each mode (H divides G; the mode's
 *                sectors are 0..H-1 and its coefficient is sign * G / H, so its
 *                charges form the subgroup of order H), or NULL for H = G on every
 *                mode.  H < G needs a single cyclic factor (n_moduli = 1).
 *  sector_dims : the true block size d(q) in [0, D] of every sector, mode after
 *                mode ([H_0 + ... + H_{order-1}] entries), or NULL for uniform
 *                blocks (Sec. 1: non-uniform blocks are padded with zeros to a
 *                fixed size).
 * The standard reduced form is then a float64 array of shape
 * [H_0, ..., H_{N-2}] + [D_0, ..., D_{N-1}] (sector of the last mode implicit,
 * solving c_{N-1} q_{N-1} == Z - sum_{mu<N-1} c_mu q_mu (mod G)).  Entries that
 * are not part of the tensor -- padding positions b >= d(q), and explicit sector
 * tuples for which that equation has no solution -- are read as zero (whatever
 * they hold) and written as zero. */
typedef struct {
  const int8_t* signs;
  const int32_t* charge;
  const int64_t* dims;
  const int32_t* sectors;
  const int64_t* sector_dims;
} symctr_operand;

/* Build a plan for W = einsum(spec, U, V).
 *  einsum   : "u_labels,v_labels->w_labels" (letters; each label at most once per
 *             operand; the output lists exactly the free labels, in any order).
 *  moduli   : n_moduli cyclic factors (product G <= 256), e.g. {3} or {2,3}.
 *  signs_*  : per-mode coefficient +1/-1 of each operand's law (Eq. symtsr).
 *  charge_* : n_moduli components of each operand's remainder Z.
 *  dims_*   : per-mode sector (block) dimension D_mu >= 1.
 *  signs_w_or_null / charge_w_or_null : optional check of the output law; the
 *             derived law (c^U on free-U modes, -sigma c^V on free-V modes,
 *             Z_U - sigma Z_V) or its global negation is accepted.
 *  prec, n_slices : precision form; n_slices = 0 picks the default (5).
 * Returns SYMCTR_OK and *out, or an error status and *out = NULL.  Host only. */
SYMCTR_API symctr_status symctr_plan_create(const char* einsum, int n_moduli, const int32_t* moduli,
                                 const int8_t* signs_u, const int32_t* charge_u,
                                 const int8_t* signs_v, const int32_t* charge_v,
                                 const int64_t* dims_u, const int64_t* dims_v,
                                 const int8_t* signs_w_or_null, const int32_t* charge_w_or_null,
                                 symctr_precision prec, int n_slices, symctr_plan** out);

/* symctr_plan_create for operands in the general form of Eq. symtsr: modes with
 * H | G sectors and coefficient +-G/H, and non-uniform sector sizes held in
 * zero-padded blocks (symctr_operand).  Contracted modes must agree in D, H and
 * sector sizes.  W's modes inherit them from the operand modes they come from,
 * and its law is derived as in symctr_plan_create (signs_w / charge_w optional
 * checks).  Every precision form runs with the same kernels as for plain
 * plans; the index maps of the aligned forms are always read from the offset
 * tables (absent rows and columns marked there), and W is zeroed as a whole
 * before each contraction.  Returns as symctr_plan_create (SYMCTR_ERR_SHAPE
 * for a sector count that does not divide G or a size outside [0, D],
 * SYMCTR_ERR_UNSUPPORTED for H < G with a product group).  Host only. */
SYMCTR_API symctr_status symctr_plan_create_general(const char* einsum, int n_moduli,
                                                   const int32_t* moduli, const symctr_operand* u,
                                                   const symctr_operand* v,
                                                   const int8_t* signs_w_or_null,
                                                   const int32_t* charge_w_or_null,
                                                   symctr_precision prec, int n_slices,
                                                   symctr_plan** out);

/* Contraction chains that stay aligned (Sec. 2.1: the aligned result W_hat,
 * with its extra symmetry mode Q, is itself a reduced form of W and can be
 * remapped to any other; Alg. 2's output step is then skipped).  Re-lays a
 * plan out so that:
 *  - w_aligned != 0: the result is written as W_hat[b][m][n], float64, C order,
 *    n_q x M x N (batch b is irrep q_first + b q_step; m and n as in the aligned
 *    layouts above), with no map back to W's standard reduced form;
 *  - u_from (v_from) != NULL: U (V) is passed as that plan's aligned result
 *    W_hat (written by it with w_aligned) instead of a standard reduced form.
 *    That plan's output modes must be this operand's modes in the same order,
 *    with the same group, law (or its global negation), sector counts and
 *    sizes; its free-U modes (which fix its irrep) must all be free modes or
 *    all contracted modes of this contraction (else SYMCTR_ERR_UNSUPPORTED).
 * Every form then reads its index maps from the offset tables (the kernels are
 * the same); numel_u / numel_v / numel_w and the workspace sizes of
 * symctr_plan_query follow the new layouts.  Call once, before the plan's
 * first contraction or table attachment (SYMCTR_ERR_ARGUMENT otherwise); the
 * source plans only lend their layouts and may be destroyed afterwards.  A
 * chained plan has no backward (symctr_contract_backward returns
 * SYMCTR_ERR_UNSUPPORTED).  Returns SYMCTR_OK, SYMCTR_ERR_NULLPTR,
 * SYMCTR_ERR_SHAPE (a source that is not the operand), SYMCTR_ERR_UNSUPPORTED,
 * SYMCTR_ERR_ARGUMENT or SYMCTR_ERR_OVERFLOW.  Host only. */
SYMCTR_API symctr_status symctr_plan_chain(symctr_plan* plan, const symctr_plan* u_from,
                                          const symctr_plan* v_from, int w_aligned);

/* Fill *out with the plan's derived quantities.  Host only. */
SYMCTR_API symctr_status symctr_plan_query(const symctr_plan* plan, symctr_plan_info* out);

/* Give the plan a device-resident copy of its offset tables (the row and column
 * offsets of Alg. 2's aligned operands in the standard reduced forms, computed
 * on the host at plan creation, including those of the backward's two
 * contractions).  Without it each contraction reads the tables from
 * page-locked host memory (up to 1 MiB, over the CPU-GPU link) or copies them
 * into the workspace; with it the kernels read them from HBM.
 *  tables : caller-owned device memory (256-byte aligned) of at least
 *           table_bytes bytes, on the device that is current during the call;
 *           NULL detaches (the plan reverts to the host tables).
 *  stream : the copy is queued on it; the caller orders contractions on other
 *           streams after it (e.g. synchronises the stream once).
 * The caller keeps the buffer allocated and unmodified until it detaches or
 * destroys the plan and the contractions issued until then have completed.  Contractions running on another device than the
 * buffer's keep using the host tables.  Not to be called while a contraction
 * with this plan is being issued on another host thread.
 * Returns SYMCTR_OK (also when table_bytes is 0: nothing to copy),
 * SYMCTR_ERR_NULLPTR (plan), SYMCTR_ERR_WORKSPACE (bytes < table_bytes),
 * SYMCTR_ERR_ARGUMENT (misaligned) or SYMCTR_ERR_CUDA. */
SYMCTR_API symctr_status symctr_plan_attach_tables(symctr_plan* plan, void* tables, size_t bytes,
                                                  void* stream);

/* Bit-exact alignment transforms (Alg. 2 input transformations and output step).
 *  operand   : 0 = U, 1 = V, 2 = W.
 *  direction : +1 standard reduced form (src) -> aligned form (dst);
 *              -1 aligned form (src) -> standard reduced form (dst; entries whose
 *              irrep Q carries no work are written as 0).
 *  Aligned sizes are aligned_numel_{u,v,w}; reduced sizes numel_{u,v,w}; a side
 *  with no entries may be NULL.  General plans: absent aligned entries are
 *  written as 0 (+1) or skipped (-1, the reduced form being zeroed first). */
SYMCTR_API symctr_status symctr_align(const symctr_plan* plan, int operand, int direction,
                           const double* src, double* dst, void* stream);

/* W = einsum(U, V) in the plan's precision form, from and to standard reduced forms.
 *  workspace : device scratch (256-byte aligned) of at least workspace_bytes_min bytes;
 *              with less than workspace_bytes the irreps Q are processed in several
 *              passes, each holding the aligned operands of as many irreps as fit.  Its
 *              first word receives device-side error codes. */
SYMCTR_API symctr_status symctr_contract(const symctr_plan* plan, const double* u_red, const double* v_red,
                              double* w_red, void* workspace, size_t workspace_bytes,
                              void* stream);

/* Complex tensors (Sec. 1: tensor entries may be complex).  u_red, v_red and
 * w_red hold interleaved complex128 reduced forms (real, imaginary pairs of
 * float64; numel_u / numel_v / numel_w complex entries each).  Computes
 *   W = einsum(op_u(U), op_v(V)),  op = complex conjugate where conj_u / conj_v
 * is nonzero.  The plan describes the operands as contracted: the conjugate of
 * a tensor with law (c, Z) carries the law (-c, -Z), so a plan for a
 * conjugated operand is created with that operand's signs and charge negated
 * (its reduced array is the same).  Runs as four real contractions of the
 * plan's precision form on the real and imaginary parts (four times the real
 * work), with the same workspace and error reporting as symctr_contract.
 * Returns as symctr_contract. */
SYMCTR_API symctr_status symctr_contract_complex(const symctr_plan* plan, int conj_u, int conj_v,
                                                const double* u_red, const double* v_red,
                                                double* w_red, void* workspace,
                                                size_t workspace_bytes, void* stream);

/* symctr_contract without a caller-provided workspace, for callers that cannot
 * allocate device memory (they are handed only their input and output buffers,
 * or run where no allocator may be called).  The paper has no counterpart: this
 * is a deployment convenience.  The scratch is one static device array of
 * 64 MiB that every GPU loading this code holds until exit.  Plans whose
 * workspace_bytes_min exceeds it get SYMCTR_ERR_WORKSPACE; plans whose
 * workspace_bytes exceeds it but whose workspace_bytes_min fits run in several
 * passes over the irreps Q.  All calls share that array: calls that overlap on
 * the GPU race (use one stream).  The first call on a device looks up the
 * array's address (cudaGetSymbolAddress, device current) and should come
 * before any stream capture; that cached address does not survive
 * cudaDeviceReset or a switch to another context on the device.  Device-side
 * failures are recorded in the array's first word: symctr_check_device_error
 * with a NULL workspace reads and clears it.  No memory is allocated or freed
 * (the first contraction of a plan, through either entry point, page-locks the
 * plan's own host offset tables). */
SYMCTR_API symctr_status symctr_contract_static_scratch(const symctr_plan* plan,
                                                        const double* u_red, const double* v_red,
                                                        double* w_red, void* stream);

/* Gradients of a scalar loss L through W = einsum(U, V), given gW = dL/dW:
 *   gU = einsum(w_labels, v_labels -> u_labels)(gW, V)   (written if grad_u_red != NULL)
 *   gV = einsum(u_labels, w_labels -> v_labels)(U, gW)   (written if grad_v_red != NULL)
 * Both are irrep-aligned contractions in the plan's precision form; the aligned
 * operands are recomputed from the standard forms (nothing is saved from the
 * forward).  gU is in U's layout and gV in V's layout. */
SYMCTR_API symctr_status symctr_contract_backward(const symctr_plan* plan, const double* grad_w_red,
                                       const double* u_red, const double* v_red,
                                       double* grad_u_red, double* grad_v_red,
                                       void* workspace, size_t workspace_bytes, void* stream);

/* Synchronise `stream`, read the device error word from `workspace` and clear it.
 * workspace = NULL reads the word of symctr_contract_static_scratch's static
 * array on the current device.
 * Returns SYMCTR_OK, SYMCTR_ERR_DEVICE_TIMEOUT, SYMCTR_ERR_NONFINITE or SYMCTR_ERR_CUDA. */
SYMCTR_API symctr_status symctr_check_device_error(const symctr_plan* plan, void* workspace, void* stream);

/* Failure-detection self-test (the paper has no counterpart).  Launches, on
 * `stream`, one small kernel that waits through the library's bounded-wait
 * routine (the one every pipeline wait of the tensor-core GEMM uses) on a
 * barrier that nothing completes.  After wait_cycles SM clock cycles (clamped
 * to [1e3, 2e9]; 2e6 is about 1 ms) the wait gives up, sets the timeout code in
 * the first word of `workspace` (at least 256 bytes, device memory) and the
 * kernel returns; symctr_check_device_error(plan, workspace, stream) then
 * returns SYMCTR_ERR_DEVICE_TIMEOUT.  Nothing traps; the context stays usable.
 * Returns SYMCTR_OK once launched, SYMCTR_ERR_NULLPTR, SYMCTR_ERR_WORKSPACE or
 * SYMCTR_ERR_CUDA. */
SYMCTR_API symctr_status symctr_selftest_bounded_wait(void* workspace, size_t workspace_bytes,
                                                     int64_t wait_cycles, void* stream);

/* Phase timing for measurement.  enable = 1 creates CUDA events on the plan;
 * each later symctr_contract on it records them on the call's stream around
 * the operand preparation (split / TF32 transforms) and the GEMM launch.
 * enable = 0 destroys them.  Host only; allocates no device memory. */
SYMCTR_API symctr_status symctr_profile_enable(symctr_plan* plan, int enable);

/* Durations in milliseconds of the two phases of the last symctr_contract on
 * the plan (prep_ms = 0 for the float64 form) and the number of kernels that
 * call launched (launches may be NULL).  Waits for the events. */
SYMCTR_API symctr_status symctr_profile_read(const symctr_plan* plan, float* prep_ms,
                                             float* gemm_ms, int* launches);

/* Human-readable name of a status. */
SYMCTR_API const char* symctr_status_string(symctr_status status);

/* Text of the last error raised on the calling host thread (empty if none). */
SYMCTR_API const char* symctr_last_error_detail(void);

/* Release a plan (NULL is ignored).  If its offset tables were page-locked,
 * this first waits, on each stream that used them, for the last contraction
 * (or table attachment) that read them; no other work is waited for.  A plan
 * must not be destroyed while another host thread is issuing calls with it. */
SYMCTR_API void symctr_plan_destroy(symctr_plan* plan);

#ifdef __cplusplus
}
#endif
#endif /* SYMCTR_H */
