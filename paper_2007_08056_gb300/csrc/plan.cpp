// Planner and C ABI: einsum parsing, the charge algebra of Algorithm 2,
// aligned-layout index maps, workspace layout and kernel dispatch.
//
// Charge algebra (Sec. 2.2, Alg. 2 coefficient vectors and deltas, with the
// sign-flip allowance of the remark after Eq. ctr):
//   sigma      : c^V_k = sigma * c^U_k on every contracted mode k (sigma = -1
//                when nothing is contracted);
//   Q          : sum_{k in C} c^U_k q_k                      (mod G)
//   free U     : sum_{F_U} c^U q == Z_U - Q
//   contracted : sum_C c^V q == sigma * Q
//   free V     : sum_{F_V} c^V q == Z_V - sigma * Q
//   output law : c^W = (c^U on F_U, -sigma c^V on F_V), Z_W = Z_U - sigma Z_V
// (the last follows by eliminating Q, as in the proof of Sec. 2.3).
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "fill.h"
#include "symctr_internal.h"

using namespace symctr;

thread_local long long symctr::g_kernel_launches = 0;

namespace {

thread_local std::string g_detail;

symctr_status fail(symctr_status st, const std::string& msg) {
  g_detail = msg;
  return st;
}

constexpr int64_t kLimit = (int64_t)1 << 61;

bool mul_ok(int64_t a, int64_t b, int64_t* out) {
  if (a < 0 || b < 0) return false;
  if (a != 0 && b > kLimit / a) return false;
  *out = a * b;
  return true;
}

int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Byte offsets of one pass's workspace regions (a pass covers n_q irreps).
struct Layout {
  uint64_t off_tab = 0, off_a = 0, off_b = 0, off_ea = 0, off_eb = 0, off_acc = 0;
  uint64_t off_part = 0;
  uint64_t bytes = 256;
  int ksplit = 1;
  bool ok = true;
};

Layout make_layout(const Problem& pr, bool tensor_core, bool general, symctr_precision prec,
                   int n_slices, int64_t kpad) {
  Layout L;
  uint64_t off = 256;
  auto region = [&](int64_t bytes) {
    uint64_t at = off;
    off += (uint64_t)round_up(bytes, 256);
    return at;
  };
  if (!tensor_core && general) {
    // the float64 form of a general plan reads its tables only
    L.off_tab = region(tables_entries(pr) * 8);
  } else if (tensor_core) {
    const int64_t nq = pr.n_q;
    L.off_tab = region(tables_entries(pr) * 8);
    int64_t ra = 0, rb = 0;
    if (!mul_ok(nq * pr.M, kpad, &ra) || !mul_ok(nq * pr.N, kpad, &rb)) {
      L.ok = false;
      return L;
    }
    if (prec == SYMCTR_SPLIT_BF16) {
      L.off_a = region(ra * 2 * n_slices);
      L.off_b = region(rb * 2 * n_slices);
      L.off_ea = region(nq * pr.M * 4);
      L.off_eb = region(nq * pr.N * 4);
      if (prep_partials_entries(pr) > 0) L.off_part = region(prep_partials_entries(pr) * 4);
      L.ksplit = split_k_ranges(pr, kpad);
      if (L.ksplit > 1) L.off_acc = region(nq * pr.M * pr.N * 8);
    } else {
      L.off_a = region(ra * 4);
      L.off_b = region(rb * 4);
    }
  }
  L.bytes = off;
  return L;
}

struct Tensor {
  std::string labels;
  int sign[SYMCTR_MAX_ORDER];
  int z;  // flattened remainder
  int64_t dim[SYMCTR_MAX_ORDER];
  // sector count H of each mode (H | G; the coefficient is sign * G / H,
  // Eq. symtsr) and the true block size of each sector when the blocks are
  // non-uniform (padded to dim; empty: uniform)
  int H[SYMCTR_MAX_ORDER];
  std::vector<int64_t> sd[SYMCTR_MAX_ORDER];
  int order() const { return (int)labels.size(); }
  bool general(int G) const {
    for (int i = 0; i < order(); ++i)
      if (H[i] != G || !sd[i].empty()) return true;
    return false;
  }
};

// Reduced-form strides of one tensor: sector axes of modes 0..N-2 (H_i
// sectors each), then blocks.
void reduced_strides(const Tensor& t, int64_t* sstride, int64_t* bstride) {
  int n = t.order();
  int64_t acc = 1;
  for (int i = n - 1; i >= 0; --i) {
    bstride[i] = acc;
    acc *= t.dim[i];
  }
  for (int i = n - 1; i >= 0; --i) {
    if (i == n - 1) {
      sstride[i] = 0;
      continue;
    }
    sstride[i] = acc;
    acc *= t.H[i];
  }
}

int64_t reduced_numel(const Tensor& t) {
  int n = t.order();
  int64_t acc = 1;
  for (int i = 0; i < n; ++i) mul_ok(acc, t.dim[i], &acc);
  for (int i = 0; i + 1 < n; ++i) mul_ok(acc, t.H[i], &acc);
  return acc;
}

// One side (rows or columns) of an aligned operand in the general form: the
// modes' sector counts, coefficient signs, strides and true block sizes.
// Host only: general plans read their index maps from the offset tables.
struct GenAxis {
  int n = 0;
  int H[SYMCTR_MAX_ORDER], sign[SYMCTR_MAX_ORDER];
  int64_t D[SYMCTR_MAX_ORDER], sstride[SYMCTR_MAX_ORDER], bstride[SYMCTR_MAX_ORDER];
  const std::vector<int64_t>* sd[SYMCTR_MAX_ORDER];
  int qa = 1, z = 0;
  int64_t size = 1;
};

// Sectors q and block indices b of aligned index r at irrep Q over the modes
// of one side, the last mode's sector solving sum_i c_i q_i == qa Q + z
// (mod G), c_i = sign_i G / H_i.  False when the entry is absent: that
// equation has no solution (it needs a multiple of G / H_last) or a block
// index lies beyond its sector's true size (padding).  Product groups have
// H = G on every mode and solve componentwise.
bool gen_decode(const GenAxis& a, const GroupDesc& g, int Q, int64_t r, int* q, int64_t* b) {
  const int target = g_add(g, g_signed(g, a.qa, Q), a.z);
  if (a.n == 0) return target == 0;
  for (int i = a.n - 1; i >= 0; --i) {
    b[i] = r % a.D[i];
    r /= a.D[i];
  }
  for (int i = a.n - 2; i >= 0; --i) {
    q[i] = (int)(r % a.H[i]);
    r /= a.H[i];
  }
  const int last = a.n - 1;
  if (g.n == 1) {
    const int G = g.order;
    int partial = 0;
    for (int i = 0; i < last; ++i) partial = (partial + a.sign[i] * (G / a.H[i]) * q[i]) % G;
    const int rhs = ((target - partial) % G + G) % G;
    const int x = ((a.sign[last] * rhs) % G + G) % G;
    const int step = G / a.H[last];
    if (x % step != 0) return false;
    q[last] = x / step;
  } else {
    int partial = 0;
    for (int i = 0; i < last; ++i) partial = g_add(g, partial, g_signed(g, a.sign[i], q[i]));
    q[last] = g_signed(g, a.sign[last], g_add(g, target, g_neg(g, partial)));
  }
  for (int i = 0; i < a.n; ++i)
    if (a.sd[i] && b[i] >= (*a.sd[i])[q[i]]) return false;
  return true;
}

// Reduced-form offset of aligned index r at irrep Q, or -1 when the entry is
// absent (gen_decode).
int64_t gen_offset(const GenAxis& a, const GroupDesc& g, int Q, int64_t r) {
  int q[SYMCTR_MAX_ORDER];
  int64_t b[SYMCTR_MAX_ORDER];
  if (!gen_decode(a, g, Q, r, q, b)) return -1;
  int64_t off = 0;
  for (int i = 0; i < a.n; ++i) off += (int64_t)q[i] * a.sstride[i] + b[i] * a.bstride[i];
  return off;
}

// One side of an operand read from another plan's aligned result W_hat[b][m][n]
// (contraction chains, symctr_plan_chain): for each of the side's modes, the
// strides of its sector and block digits in that layout (0 for a sector the
// layout leaves implicit), and, when the source's free-U modes all fall on
// this side, the batch term: the source irrep Q_src = z - sum coef_i q_i
// selects batch b = (Q_src - q0) / step, weighted by M_src * N_src.
struct ChainSide {
  int64_t sstride[SYMCTR_MAX_ORDER], bstride[SYMCTR_MAX_ORDER];
  bool batch = false;
  int coef[SYMCTR_MAX_ORDER];   // source coefficients on this side's modes (0: not free-U there)
  int z = 0;
  int q_single = -1, q0 = 0, q_step = 1, n_q = 0;
  int64_t batch_stride = 0;
};

int64_t chain_offset(const GenAxis& a, const ChainSide& c, const GroupDesc& g, int Q, int64_t r) {
  int q[SYMCTR_MAX_ORDER];
  int64_t b[SYMCTR_MAX_ORDER];
  if (!gen_decode(a, g, Q, r, q, b)) return -1;
  int64_t off = 0;
  for (int i = 0; i < a.n; ++i) off += (int64_t)q[i] * c.sstride[i] + b[i] * c.bstride[i];
  if (c.batch) {
    int qs = c.z;
    for (int i = 0; i < a.n; ++i) {
      if (c.coef[i] == 0) continue;
      if (g.n == 1)
        qs = ((qs - c.coef[i] * q[i]) % g.order + g.order) % g.order;
      else
        qs = g_add(g, qs, g_signed(g, -c.coef[i], q[i]));
    }
    int bi;
    if (c.q_single >= 0) {
      bi = qs == c.q_single ? 0 : -1;
    } else {
      const int d = ((qs - c.q0) % g.order + g.order) % g.order;
      bi = (d % c.q_step == 0 && d / c.q_step < c.n_q) ? d / c.q_step : -1;
    }
    if (bi < 0) return -1;
    off += (int64_t)bi * c.batch_stride;
  }
  return off;
}

}  // namespace

struct symctr_plan {
  Tensor u, v, w;
  GroupDesc g;
  int s = 0, t = 0, vv = 0, sigma = -1;
  std::vector<int> FU, C, FV;  // mode positions: FU, C in U; FV in V
  Problem prob;
  int64_t numel_u = 0, numel_v = 0, numel_w = 0;
  symctr_precision prec = SYMCTR_FP64;
  int n_slices = 0;
  int64_t kpad = 0;
  // workspace: all irreps in one pass, or the smallest pass (one irrep)
  uint64_t ws_bytes = 256, ws_bytes_min = 256;
  bool tensor_core = false;
  // sub-group coefficients or padded sectors on some mode: every form reads
  // its index maps from the offset tables (absent entries -1)
  bool general = false;
  // split form: run length of the single-read preparation of U and V (0: the
  // operand takes the two-phase preparation)
  int64_t row_run[2] = {0, 0};
  // split form, K <= kRowTileMaxK: operand op's whole aligned rows fit one
  // CTA's shared memory and it takes the short-row single-read kernel
  bool row_tile[2] = {false, false};
  // contraction chains (symctr_plan_chain): U and/or V read from another
  // plan's aligned result, and/or W written as W_hat; no backward.  A chained
  // plan is table-driven (general) without having absent entries of its own.
  bool chained = false;
  // W holds entries no aligned element covers (padding, sector tuples without
  // a solution): zeroed as a whole before each contraction
  bool fill_all = false;
  // uniform plans whose irreps do not cover W: the sector combinations of W
  // that the contraction writes whole (bit c of fill_written), each fill_bv
  // doubles; the zero fill skips them (fill_bv == 0: zero all of W)
  int64_t fill_bv = 0, fill_combos = 0;
  std::vector<uint32_t> fill_written;
  symctr_plan* bwd_u = nullptr;
  symctr_plan* bwd_v = nullptr;
  bool prof = false;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  mutable int last_launches = 0;
  // offset tables of all irreps (tensor-core forms and general plans),
  // computed once on the host in the workspace layout of a single pass;
  // page-locked on first use
  std::vector<int64_t> htab;
  mutable std::once_flag pin_once;
  mutable bool pinned = false;
  mutable const int64_t* dtab = nullptr;   // device view of the page-locked tables
  // the last contraction that read the page-locked tables, per (device,
  // stream): destroying the plan waits for these events only
  struct Use {
    int dev;
    cudaStream_t st;
    cudaEvent_t ev;
  };
  mutable std::mutex use_mu;
  mutable std::vector<Use> uses;
  // caller-owned device copy of htab (symctr_plan_attach_tables) and its device
  const int64_t* dev_tab = nullptr;
  int dev_tab_device = -1;
};

namespace {

// Offset tables up to this size are read in place from page-locked host memory.
constexpr size_t kMappedTablesMax = 1 << 20;

int g_label(const GroupDesc& g, const int32_t* comps) {
  int q = 0;
  for (int i = 0; i < g.n; ++i) {
    int m = g.mod[i];
    int c = ((comps[i] % m) + m) % m;
    q = q * m + c;
  }
  return q;
}

void g_comps(const GroupDesc& g, int q, int32_t* comps) {
  for (int i = g.n - 1; i >= 0; --i) {
    comps[i] = q % g.mod[i];
    q /= g.mod[i];
  }
}

AxisMap make_axis(const Tensor& t, const std::vector<int>& modes, const int* law_sign, int qa,
                  int z) {
  AxisMap a;
  std::memset(&a, 0, sizeof(a));
  int64_t ss[SYMCTR_MAX_ORDER], bs[SYMCTR_MAX_ORDER];
  reduced_strides(t, ss, bs);
  a.n = (int)modes.size();
  int64_t size = 1;
  for (int i = 0; i < a.n; ++i) {
    int mu = modes[i];
    a.D[i] = (int)t.dim[mu];
    a.sign[i] = law_sign[i];
    a.sstride[i] = ss[mu];
    a.bstride[i] = bs[mu];
    size *= t.dim[mu];
    if (i + 1 < a.n) size *= t.H[mu];
  }
  a.size = size;
  a.qa = qa;
  a.z = z;
  return a;
}

GenAxis make_gen_axis(const Tensor& t, const std::vector<int>& modes, const int* law_sign, int qa,
                      int z) {
  GenAxis a;
  int64_t ss[SYMCTR_MAX_ORDER], bs[SYMCTR_MAX_ORDER];
  reduced_strides(t, ss, bs);
  a.n = (int)modes.size();
  for (int i = 0; i < a.n; ++i) {
    int mu = modes[i];
    a.H[i] = t.H[mu];
    a.sign[i] = law_sign[i];
    a.D[i] = t.dim[mu];
    a.sstride[i] = ss[mu];
    a.bstride[i] = bs[mu];
    a.sd[i] = t.sd[mu].empty() ? nullptr : &t.sd[mu];
    a.size *= t.dim[mu];
    if (i + 1 < a.n) a.size *= t.H[mu];
  }
  a.qa = qa;
  a.z = z;
  return a;
}

// One operand as the plan builder receives it (see symctr_operand).
struct OpDesc {
  const int8_t* signs = nullptr;
  const int32_t* charge = nullptr;
  const int64_t* dims = nullptr;
  const int32_t* sectors = nullptr;      // NULL: G sectors on every mode
  const int64_t* sector_dims = nullptr;  // NULL: uniform blocks
};

// An OpDesc view of a tensor of a plan, with its own storage (backward plans).
struct OwnedDesc {
  int8_t signs[SYMCTR_MAX_ORDER];
  int32_t charge[SYMCTR_MAX_MODULI];
  int64_t dims[SYMCTR_MAX_ORDER];
  int32_t sectors[SYMCTR_MAX_ORDER];
  std::vector<int64_t> sd;
  OpDesc desc;
  OwnedDesc(const Tensor& t, const GroupDesc& g) {
    bool any_sd = false;
    for (int i = 0; i < t.order(); ++i) {
      signs[i] = (int8_t)t.sign[i];
      dims[i] = t.dim[i];
      sectors[i] = t.H[i];
      any_sd = any_sd || !t.sd[i].empty();
    }
    if (any_sd)
      for (int i = 0; i < t.order(); ++i)
        for (int q = 0; q < t.H[i]; ++q) sd.push_back(t.sd[i].empty() ? t.dim[i] : t.sd[i][q]);
    g_comps(g, t.z, charge);
    desc.signs = signs;
    desc.charge = charge;
    desc.dims = dims;
    desc.sectors = sectors;
    desc.sector_dims = any_sd ? sd.data() : nullptr;
  }
};

int64_t gcd64(int64_t a, int64_t b) {
  while (b) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

symctr_status build(const char* einsum, int n_moduli, const int32_t* moduli, const OpDesc& du_,
                    const OpDesc& dv_, const int8_t* sw, const int32_t* zw, symctr_precision prec,
                    int n_slices, bool with_backward, symctr_plan** out) {
  if (!out) return fail(SYMCTR_ERR_NULLPTR, "out is NULL");
  *out = nullptr;
  if (!einsum || !moduli || !du_.charge || !dv_.charge) return fail(SYMCTR_ERR_NULLPTR, "NULL argument");
  if (n_moduli < 1 || n_moduli > SYMCTR_MAX_MODULI)
    return fail(SYMCTR_ERR_UNSUPPORTED, "n_moduli must be in [1, 4]");
  if (prec != SYMCTR_FP64 && prec != SYMCTR_SPLIT_BF16 && prec != SYMCTR_TF32)
    return fail(SYMCTR_ERR_ARGUMENT, "unknown precision form");
  if (n_slices < 0 || n_slices > kMaxSlices)
    return fail(SYMCTR_ERR_ARGUMENT, "n_slices must be in [0, 6]");

  // ---- einsum ----
  std::string spec;
  for (const char* c = einsum; *c; ++c)
    if (*c != ' ') spec.push_back(*c);
  size_t arrow = spec.find("->");
  size_t comma = spec.find(',');
  if (arrow == std::string::npos || comma == std::string::npos || comma > arrow ||
      spec.find(',', comma + 1) != std::string::npos)
    return fail(SYMCTR_ERR_EINSUM, "expected 'u,v->w'");
  std::string lu = spec.substr(0, comma), lv = spec.substr(comma + 1, arrow - comma - 1),
              lw = spec.substr(arrow + 2);
  for (const std::string* lab : {&lu, &lv, &lw}) {
    if ((int)lab->size() > SYMCTR_MAX_ORDER)
      return fail(SYMCTR_ERR_UNSUPPORTED, "order > 8");
    for (size_t i = 0; i < lab->size(); ++i) {
      char c = (*lab)[i];
      if (!((c >= 'a' && c <= 'z') || (c >= 'A' && c <= 'Z')))
        return fail(SYMCTR_ERR_EINSUM, "labels must be letters");
      if (lab->find(c, i + 1) != std::string::npos)
        return fail(SYMCTR_ERR_EINSUM, "repeated label inside one operand (trace)");
    }
  }
  for (char c : lw) {
    bool inu = lu.find(c) != std::string::npos, inv = lv.find(c) != std::string::npos;
    if (inu && inv) return fail(SYMCTR_ERR_EINSUM, "batch label (in U, V and W)");
    if (!inu && !inv) return fail(SYMCTR_ERR_EINSUM, "output label absent from inputs");
  }
  for (char c : lu)
    if (lv.find(c) == std::string::npos && lw.find(c) == std::string::npos)
      return fail(SYMCTR_ERR_EINSUM, "free label of U missing from the output");
  for (char c : lv)
    if (lu.find(c) == std::string::npos && lw.find(c) == std::string::npos)
      return fail(SYMCTR_ERR_EINSUM, "free label of V missing from the output");
  if ((!du_.signs || !du_.dims) && !lu.empty()) return fail(SYMCTR_ERR_NULLPTR, "signs_u/dims_u NULL");
  if ((!dv_.signs || !dv_.dims) && !lv.empty()) return fail(SYMCTR_ERR_NULLPTR, "signs_v/dims_v NULL");

  symctr_plan* P = new (std::nothrow) symctr_plan();
  if (!P) return fail(SYMCTR_ERR_ARGUMENT, "out of host memory");
  auto bail = [&](symctr_status st, const std::string& m) {
    delete P;
    return fail(st, m);
  };

  // ---- group ----
  P->g.n = n_moduli;
  int64_t G = 1;
  for (int i = 0; i < n_moduli; ++i) {
    if (moduli[i] < 1) return bail(SYMCTR_ERR_SHAPE, "moduli must be >= 1");
    P->g.mod[i] = moduli[i];
    G *= moduli[i];
    if (G > SYMCTR_MAX_GROUP) return bail(SYMCTR_ERR_UNSUPPORTED, "group order > 256");
  }
  P->g.order = (int)G;
  const GroupDesc& g = P->g;

  // ---- operands: signs, block sizes, sector counts (Eq. symtsr), sector sizes ----
  P->u.labels = lu;
  P->v.labels = lv;
  P->w.labels = lw;
  auto load = [&](Tensor& t, const OpDesc& d, const char* name) -> std::string {
    int64_t at = 0;
    for (int i = 0; i < t.order(); ++i) {
      if (d.signs[i] != 1 && d.signs[i] != -1) return std::string("signs must be +1/-1 (") + name + ")";
      if (d.dims[i] < 1 || d.dims[i] > (1 << 30)) return std::string("sector dim out of range (") + name + ")";
      t.sign[i] = d.signs[i];
      t.dim[i] = d.dims[i];
      t.H[i] = d.sectors ? d.sectors[i] : (int)G;
      if (t.H[i] < 1 || t.H[i] > G || G % t.H[i] != 0)
        return std::string("sector counts must divide the group order (") + name + ")";
      if (t.H[i] != G && n_moduli != 1)
        return std::string("unsupported: sub-group coefficients need a single cyclic factor (") + name + ")";
      if (d.sector_dims) {
        bool uniform = true;
        for (int q = 0; q < t.H[i]; ++q) {
          const int64_t x = d.sector_dims[at + q];
          if (x < 0 || x > t.dim[i]) return std::string("sector sizes must lie in [0, D] (") + name + ")";
          uniform = uniform && x == t.dim[i];
        }
        if (!uniform) t.sd[i].assign(d.sector_dims + at, d.sector_dims + at + t.H[i]);
        at += t.H[i];
      }
    }
    return "";
  };
  {
    std::string m = load(P->u, du_, "U");
    if (m.empty()) m = load(P->v, dv_, "V");
    if (!m.empty())
      return bail(m.rfind("unsupported", 0) == 0 ? SYMCTR_ERR_UNSUPPORTED
                  : m.rfind("signs", 0) == 0     ? SYMCTR_ERR_SIGNS
                                                 : SYMCTR_ERR_SHAPE,
                  m);
  }
  P->u.z = g_label(g, du_.charge);
  P->v.z = g_label(g, dv_.charge);

  // ---- mode classes and sigma ----
  int sigma = 0;
  for (int i = 0; i < (int)lu.size(); ++i) {
    size_t j = lv.find(lu[i]);
    if (j == std::string::npos) {
      P->FU.push_back(i);
      continue;
    }
    P->C.push_back(i);
    if (P->u.dim[i] != P->v.dim[j] || P->u.H[i] != P->v.H[j] || P->u.sd[i] != P->v.sd[j])
      return bail(SYMCTR_ERR_SHAPE, std::string("sectors or their sizes differ on contracted mode ") + lu[i]);
    int r = P->u.sign[i] * P->v.sign[j];
    if (sigma == 0) sigma = r;
    else if (sigma != r)
      return bail(SYMCTR_ERR_SIGNS, "contracted coefficients must agree up to one global sign");
  }
  for (int j = 0; j < (int)lv.size(); ++j)
    if (lu.find(lv[j]) == std::string::npos) P->FV.push_back(j);
  if (sigma == 0) sigma = -1;
  P->sigma = sigma;
  P->s = (int)P->FU.size();
  P->t = (int)P->FV.size();
  P->vv = (int)P->C.size();

  // ---- output law ----
  // With nothing contracted (v = 0) both sigma = +1 and sigma = -1 give a valid
  // law for the outer product, and both reduced forms hold the same numbers
  // (the two laws agree wherever U's and V's laws both hold); a requested
  // output law then selects sigma.
  auto derive = [&](int sg) {
    for (int i = 0; i < (int)lw.size(); ++i) {
      size_t a = lu.find(lw[i]);
      const Tensor* src;
      int mu;
      if (a != std::string::npos) {
        P->w.sign[i] = P->u.sign[a];
        src = &P->u;
        mu = (int)a;
      } else {
        size_t b = lv.find(lw[i]);
        P->w.sign[i] = -sg * P->v.sign[b];
        src = &P->v;
        mu = (int)b;
      }
      P->w.dim[i] = src->dim[mu];
      P->w.H[i] = src->H[mu];
      P->w.sd[i] = src->sd[mu];
    }
    P->w.z = g_add(g, P->u.z, g_signed(g, -sg, P->v.z));
  };
  auto matches = [&](const int8_t* sw_, const int32_t* zw_) {
    int zgiven = g_label(g, zw_);
    bool same = zgiven == P->w.z, neg = zgiven == g_neg(g, P->w.z);
    for (int i = 0; i < (int)lw.size(); ++i) {
      same = same && sw_[i] == P->w.sign[i];
      neg = neg && sw_[i] == -P->w.sign[i];
    }
    return same || neg;
  };
  derive(sigma);
  if (sw || zw) {
    if (!sw || !zw) return bail(SYMCTR_ERR_NULLPTR, "give both signs_w and charge_w, or neither");
    if (!matches(sw, zw) && P->C.empty()) {
      sigma = -sigma;
      P->sigma = sigma;
      derive(sigma);
    }
    if (!matches(sw, zw)) return bail(SYMCTR_ERR_CHARGE, "given output law contradicts the derived law");
  }
  P->general = P->u.general((int)G) || P->v.general((int)G) || P->w.general((int)G);
  P->fill_all = P->general;

  // ---- sizes ----
  P->numel_u = reduced_numel(P->u);
  P->numel_v = reduced_numel(P->v);
  P->numel_w = reduced_numel(P->w);
  if (P->numel_u >= kLimit || P->numel_v >= kLimit || P->numel_w >= kLimit)
    return bail(SYMCTR_ERR_OVERFLOW, "tensor too large");

  // ---- index maps ----
  std::vector<int> FV_in_V = P->FV, C_in_V, FU_in_W, FV_in_W;
  int sgn_fu[SYMCTR_MAX_ORDER], sgn_cu[SYMCTR_MAX_ORDER], sgn_cv[SYMCTR_MAX_ORDER],
      sgn_fv[SYMCTR_MAX_ORDER];
  for (size_t i = 0; i < P->FU.size(); ++i) {
    sgn_fu[i] = P->u.sign[P->FU[i]];
    FU_in_W.push_back((int)lw.find(lu[P->FU[i]]));
  }
  for (size_t i = 0; i < P->C.size(); ++i) {
    sgn_cu[i] = P->u.sign[P->C[i]];
    int j = (int)lv.find(lu[P->C[i]]);
    C_in_V.push_back(j);
    sgn_cv[i] = P->v.sign[j];
  }
  for (size_t i = 0; i < P->FV.size(); ++i) {
    sgn_fv[i] = P->v.sign[P->FV[i]];
    FV_in_W.push_back((int)lw.find(lv[P->FV[i]]));
  }
  Problem& pr = P->prob;
  pr.g = g;
  pr.u.rows = make_axis(P->u, P->FU, sgn_fu, -1, P->u.z);
  pr.u.cols = make_axis(P->u, P->C, sgn_cu, +1, 0);
  pr.v.rows = make_axis(P->v, FV_in_V, sgn_fv, -sigma, P->v.z);
  pr.v.cols = make_axis(P->v, C_in_V, sgn_cv, sigma, 0);
  pr.w.rows = make_axis(P->w, FU_in_W, sgn_fu, -1, P->u.z);
  pr.w.cols = make_axis(P->w, FV_in_W, sgn_fv, -sigma, P->v.z);
  pr.M = pr.u.rows.size;
  pr.N = pr.v.rows.size;
  pr.K = pr.u.cols.size;
  pr.general = P->general ? 1 : 0;
  GenAxis gax[6];
  if (P->general) {
    gax[0] = make_gen_axis(P->u, P->FU, sgn_fu, -1, P->u.z);
    gax[1] = make_gen_axis(P->u, P->C, sgn_cu, +1, 0);
    gax[2] = make_gen_axis(P->v, FV_in_V, sgn_fv, -sigma, P->v.z);
    gax[3] = make_gen_axis(P->v, C_in_V, sgn_cv, sigma, 0);
    gax[4] = make_gen_axis(P->w, FU_in_W, sgn_fu, -1, P->u.z);
    gax[5] = make_gen_axis(P->w, FV_in_W, sgn_fv, -sigma, P->v.z);
  }

  // ---- irreps carrying work ----
  std::vector<int> works;
  for (int Q = 0; Q < (int)G; ++Q) {
    bool ok = true;
    if (!P->general) {
      if (P->s == 0) ok = ok && g_add(g, P->u.z, g_neg(g, Q)) == 0;
      if (P->vv == 0) ok = ok && Q == 0;
      if (P->t == 0) ok = ok && g_add(g, P->v.z, g_neg(g, g_signed(g, sigma, Q))) == 0;
    } else {
      // some U row, some contracted column and some V row exist at this Q
      for (int k : {0, 1, 2}) {
        bool any = false;
        for (int64_t r = 0; r < gax[k].size && !any; ++r) any = gen_offset(gax[k], g, Q, r) >= 0;
        ok = ok && any;
      }
    }
    if (ok) works.push_back(Q);
  }
  pr.n_q = (int)works.size();
  pr.q_single = pr.n_q == 1 ? works[0] : -1;
  pr.q0 = 0;
  pr.q_step = 1;
  if (pr.n_q > 1) {
    // the batches: the progression q0 + b * step (mod G) through all of them
    // (a coset of a subgroup of Z_G for a single cyclic factor; extra irreps
    // of an irregular set carry absent rows only)
    int64_t step = G;
    for (int q : works) step = gcd64(step, (int64_t)(q - works[0] + G) % G);
    pr.q0 = works[0];
    pr.q_step = (int)step;
    pr.n_q = (int)(G / step);
    if (!P->general && pr.n_q != (int)G) return bail(SYMCTR_ERR_ARGUMENT, "internal: Q set");
  }

  // ---- precision form and workspace ----
  P->prec = prec;
  P->tensor_core = prec != SYMCTR_FP64 && pr.n_q > 0 && tensor_core_shape(pr);
  P->n_slices = prec == SYMCTR_SPLIT_BF16 ? (n_slices == 0 ? 5 : n_slices) : 0;
  if (prec == SYMCTR_SPLIT_BF16 && P->n_slices < 2)
    return bail(SYMCTR_ERR_ARGUMENT, "split form needs at least 2 slices");
  P->kpad = round_up(pr.K, kKBlock);
  pr.q_base = 0;
  if (P->tensor_core || (P->general && pr.n_q > 0)) {
    // the six offset tables [U rows | U cols | V rows | V cols | W rows | W cols],
    // each [n_q][extent]: the same function of the plan on every call
    const int64_t total = tables_entries(pr);
    if (total > (int64_t)1 << 28) return bail(SYMCTR_ERR_OVERFLOW, "offset tables too large");
    try {
      P->htab.resize((size_t)total);
    } catch (const std::bad_alloc&) {
      return bail(SYMCTR_ERR_OVERFLOW, "offset tables: host allocation failed");
    }
    int64_t* t = P->htab.data();
    const AxisMap* maps[6] = {&pr.u.rows, &pr.u.cols, &pr.v.rows, &pr.v.cols, &pr.w.rows, &pr.w.cols};
    const int64_t ext[6] = {pr.M, pr.K, pr.N, pr.K, pr.M, pr.N};
    for (int k = 0; k < 6; ++k)
      for (int b = 0; b < pr.n_q; ++b)
        for (int64_t r = 0; r < ext[k]; ++r)
          *t++ = P->general ? gen_offset(gax[k], pr.g, batch_irrep(pr, b), r)
                            : axis_offset(*maps[k], pr.g, batch_irrep(pr, b), r);
  }
  {
    Layout full = make_layout(pr, P->tensor_core, P->general, prec, P->n_slices, P->kpad);
    if (!full.ok) return bail(SYMCTR_ERR_OVERFLOW, "aligned operand too large");
    P->ws_bytes = full.bytes;
    P->ws_bytes_min = full.bytes;
    if (P->tensor_core && pr.q_single < 0 && pr.n_q > 1) {
      Problem one = pr;
      one.n_q = 1;
      P->ws_bytes_min = make_layout(one, true, P->general, prec, P->n_slices, P->kpad).bytes;
    }
  }

  // Zero fill of the irreps that carry no work (uniform plans): a sector
  // combination of W (its stored sector labels) is written at every block
  // position by one irrep's row and column sector patterns, or not at all.
  // The combinations written are found from the patterns' first entries and
  // checked to hold exactly the n_q M N entries the contraction writes.
  if (!P->general && (int64_t)pr.n_q * pr.M * pr.N < P->numel_w) {
    int64_t bv = 1;
    for (int i = 0; i < P->w.order(); ++i) bv *= P->w.dim[i];
    const int64_t n_combo = bv > 0 ? P->numel_w / bv : 0;
    if (n_combo > 0 && n_combo <= kFillMaskCombos && n_combo * bv == P->numel_w) {
      std::vector<uint32_t> mask((size_t)(n_combo + 31) / 32, 0u);
      const AxisMap& R = pr.w.rows;
      const AxisMap& Cm = pr.w.cols;
      int64_t rb = 1, cb = 1;
      for (int i = 0; i < R.n; ++i) rb *= R.D[i];
      for (int i = 0; i < Cm.n; ++i) cb *= Cm.D[i];
      const int64_t rp = R.size / rb, cp = Cm.size / cb;
      bool ok = rp * rb == pr.M && cp * cb == pr.N;
      for (int b = 0; b < pr.n_q && ok; ++b) {
        const int Q = batch_irrep(pr, b);
        for (int64_t i = 0; i < rp && ok; ++i) {
          const int64_t ro = axis_offset(R, pr.g, Q, i * rb);
          for (int64_t j = 0; j < cp && ok; ++j) {
            const int64_t c = (ro + axis_offset(Cm, pr.g, Q, j * cb)) / bv;
            ok = c >= 0 && c < n_combo;
            if (ok) mask[(size_t)(c >> 5)] |= 1u << (c & 31);
          }
        }
      }
      int64_t written = 0;
      for (uint32_t m : mask) written += __builtin_popcount(m);
      if (ok && written * bv == (int64_t)pr.n_q * pr.M * pr.N) {
        P->fill_bv = bv;
        P->fill_combos = n_combo;
        P->fill_written.swap(mask);
      }
    }
  }

  // Single-read preparation (split form): an operand whose aligned rows are
  // column-contiguous runs of at least 128 entries, at most kRowClusterMaxK
  // long (clusters of CTAs beyond kRowStreamMaxK), every run start and row
  // offset even (16-byte bulk copies), and
  // large enough (>= 32 MB) to be bandwidth-bound.
  if (P->tensor_core && prec == SYMCTR_SPLIT_BF16 && !P->general) {
    const AxisMap* rows[2] = {&pr.u.rows, &pr.v.rows};
    const AxisMap* cols[2] = {&pr.u.cols, &pr.v.cols};
    const int64_t R[2] = {pr.M, pr.N};
    const int64_t* rtab[2] = {P->htab.data(), P->htab.data() + (int64_t)pr.n_q * (pr.M + pr.K)};
    const int64_t* ctab[2] = {P->htab.data() + (int64_t)pr.n_q * pr.M,
                              P->htab.data() + (int64_t)pr.n_q * (pr.M + pr.K + pr.N)};
    for (int op = 0; op < 2; ++op) {
      const AxisMap& c = *cols[op];
      const bool rows_contig = rows[op]->n > 0 && rows[op]->bstride[rows[op]->n - 1] == 1;
      if (rows_contig || c.n == 0 || c.bstride[c.n - 1] != 1) continue;
      int64_t L = c.D[c.n - 1];
      for (int i = c.n - 2; i >= 0 && c.bstride[i] == L; --i) L *= c.D[i];
      if (L < 128 || L % 2 != 0 || pr.K % L != 0 || pr.K > kRowClusterMaxK) continue;
      if ((int64_t)pr.n_q * R[op] * pr.K < ((int64_t)4 << 20)) continue;
      bool even = true;
      for (int64_t i = 0; i < (int64_t)pr.n_q * R[op] && even; ++i) even = rtab[op][i] % 2 == 0;
      for (int64_t b = 0; b < pr.n_q && even; ++b)
        for (int64_t j = 0; j < pr.K && even; j += L) even = ctab[op][b * pr.K + j] % 2 == 0;
      if (even) P->row_run[op] = L;
    }
  }

  // Short rows (split form): operands whose padded K is at most kRowTileMaxK
  // are read once by the short-row kernel (whole rows per CTA, no grid
  // barrier), with the exceptions below.
  if (P->tensor_core && prec == SYMCTR_SPLIT_BF16 && P->kpad <= kRowTileMaxK) {
    const AxisMap* rows[2] = {&pr.u.rows, &pr.v.rows};
    for (int op = 0; op < 2; ++op) {
      // rows that are the reduced form's unit-stride side are gathered across
      // rows, at least 4 per CTA (32-byte sectors): K <= 2048; rows of
      // contiguous runs up to K = 2048 also go here (the bulk-copy kernel, one
      // row per step, pays off on longer rows)
      const bool rows_contig = rows[op]->n > 0 && rows[op]->bstride[rows[op]->n - 1] == 1;
      if (rows_contig && P->kpad > kRowTileMaxK / 2) continue;
      if (P->row_run[op] > 0 && P->kpad > kRowTileMaxK / 2) continue;
      P->row_tile[op] = true;
      P->row_run[op] = 0;
    }
  }

  if (with_backward) {
    // gU = einsum(lw,lv->lu)(gW, V): result carries U's law.
    OwnedDesc dw(P->w, g), du(P->u, g), dv(P->v, g);
    std::string su_spec = lw + "," + lv + "->" + lu;
    std::string sv_spec = lu + "," + lw + "->" + lv;
    symctr_status st = build(su_spec.c_str(), n_moduli, moduli, dw.desc, dv.desc, du.signs, du.charge,
                             prec, P->n_slices, false, &P->bwd_u);
    if (st != SYMCTR_OK) return bail(st, "backward plan (dU): " + g_detail);
    st = build(sv_spec.c_str(), n_moduli, moduli, du.desc, dw.desc, dv.signs, dv.charge, prec,
               P->n_slices, false, &P->bwd_v);
    if (st != SYMCTR_OK) {
      symctr_plan_destroy(P->bwd_u);
      P->bwd_u = nullptr;
      return bail(st, "backward plan (dV): " + g_detail);
    }
  }
  *out = P;
  g_detail.clear();
  return SYMCTR_OK;
}

symctr_status cuda_status(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return SYMCTR_OK;
  return fail(SYMCTR_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Kernels and copies queued on `st` read the plan's page-locked tables: record
// the point after which the plan may release them (one event per device and
// stream, re-recorded by every such call).
symctr_status mark_table_use(const symctr_plan* P, cudaStream_t st) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "current device");
  std::lock_guard<std::mutex> lock(P->use_mu);
  cudaEvent_t ev = nullptr;
  for (const auto& u : P->uses)
    if (u.dev == dev && u.st == st) ev = u.ev;
  if (!ev) {
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_status(e, "table-use event");
    P->uses.push_back({dev, st, ev});
  }
  return cuda_status(cudaEventRecord(ev, st), "table-use event");
}

// How one real contraction reads and writes: element stride (2 when the
// pointers address the real or imaginary parts of interleaved complex data),
// output mode W = (-)R or W += (-)R, whether the workspace's error word
// is cleared first, and how many doubles of W are zeroed up front (the entries
// of irreps that carry no work; -1: W's reduced form).
struct RunMode {
  int es = 1;
  int negate = 0;
  int accumulate = 0;
  bool clear_err = true;
  int64_t fill_n = -1;
};

symctr_status run_contract_body(const symctr_plan* P, const double* u, const double* v,
                                double* w, void* ws, size_t ws_bytes, cudaStream_t st,
                                const RunMode& mode);

symctr_status run_contract(const symctr_plan* P, const double* u, const double* v, double* w,
                           void* ws, size_t ws_bytes, cudaStream_t st,
                           const RunMode& mode = RunMode()) {
  long long before = g_kernel_launches;
  symctr_status s = run_contract_body(P, u, v, w, ws, ws_bytes, st, mode);
  P->last_launches = (int)(g_kernel_launches - before);
  return s;
}

// Page-lock the host tables once, so that their copies are plain DMA reads and
// small ones can be read in place (without it they are staged through pageable
// memory, also correct).
void pin_tables(const symctr_plan* P) {
  std::call_once(P->pin_once, [P] {
    if (!P->htab.empty() &&
        cudaHostRegister((void*)P->htab.data(), P->htab.size() * sizeof(int64_t),
                         cudaHostRegisterPortable | cudaHostRegisterMapped) == cudaSuccess) {
      P->pinned = true;
      void* d = nullptr;
      if (cudaHostGetDevicePointer(&d, (void*)P->htab.data(), 0) == cudaSuccess) P->dtab = (const int64_t*)d;
    }
    cudaGetLastError();
  });
}

// Whether the caller-attached device tables live on the current device.
bool tables_attached(const symctr_plan* P) {
  if (!P->dev_tab) return false;
  int dev = -1;
  return cudaGetDevice(&dev) == cudaSuccess && dev == P->dev_tab_device;
}

// The tables of one pass (batches q0 .. q0 + pc.n_q - 1): the attached device
// copy, the small page-locked host tables read in place (reads over the
// CPU-GPU link are not cached on the GPU, so larger tables, re-read by many
// tiles, are copied to HBM instead), or a copy into the workspace at off_tab.
symctr_status pass_tables(const symctr_plan* P, const Problem& pc, int q0, bool attached, char* base,
                          uint64_t off_tab, cudaStream_t st, Tables* tab) {
  const Problem& pr = P->prob;
  const int64_t ext[6] = {pr.M, pr.K, pr.N, pr.K, pr.M, pr.N};
  const int64_t* in_place = attached ? P->dev_tab
                            : (P->dtab && P->htab.size() * sizeof(int64_t) <= kMappedTablesMax)
                                ? P->dtab
                                : nullptr;
  if (in_place) {
    const int64_t* src = in_place;
    const int64_t** dst[6] = {&tab->urow, &tab->ucol, &tab->vrow, &tab->vcol, &tab->wrow, &tab->wcol};
    for (int k = 0; k < 6; ++k) {
      *dst[k] = src + (int64_t)q0 * ext[k];
      src += (int64_t)pr.n_q * ext[k];
    }
    return SYMCTR_OK;
  }
  // one copy for a single pass, one per table otherwise
  int64_t* t0 = (int64_t*)(base + off_tab);
  tab->urow = t0;
  tab->ucol = tab->urow + (int64_t)pc.n_q * pc.M;
  tab->vrow = tab->ucol + (int64_t)pc.n_q * pc.K;
  tab->vcol = tab->vrow + (int64_t)pc.n_q * pc.N;
  tab->wrow = tab->vcol + (int64_t)pc.n_q * pc.K;
  tab->wcol = tab->wrow + (int64_t)pc.n_q * pc.M;
  cudaError_t e = cudaSuccess;
  if (pc.n_q == pr.n_q) {
    e = cudaMemcpyAsync(t0, P->htab.data(), P->htab.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st);
  } else {
    const int64_t* src = P->htab.data();
    int64_t* dst = t0;
    for (int k = 0; k < 6 && e == cudaSuccess; ++k) {
      e = cudaMemcpyAsync(dst, src + (int64_t)q0 * ext[k], (size_t)(pc.n_q * ext[k]) * sizeof(int64_t),
                          cudaMemcpyHostToDevice, st);
      src += (int64_t)pr.n_q * ext[k];
      dst += (int64_t)pc.n_q * ext[k];
    }
  }
  return cuda_status(e, "offset tables");
}

symctr_status run_contract_body(const symctr_plan* P, const double* u, const double* v,
                                double* w, void* ws, size_t ws_bytes, cudaStream_t st,
                                const RunMode& mode) {
  Problem prob = P->prob;
  prob.es = mode.es;
  prob.negate = mode.negate;
  prob.accumulate = mode.accumulate;
  const Problem& pr = prob;
  if (!w || (!u && P->numel_u) || (!v && P->numel_v))
    return fail(SYMCTR_ERR_NULLPTR, "NULL tensor pointer");
  if (!ws || ws_bytes < P->ws_bytes_min)
    return fail(SYMCTR_ERR_WORKSPACE, "workspace smaller than workspace_bytes_min");
  char* base = (char*)ws;
  unsigned* err = (unsigned*)base;
  // header: error word (byte 0) and the prep kernel's grid-barrier counter (byte 64)
  cudaError_t e = mode.clear_err ? cudaMemsetAsync(err, 0, 128, st) : cudaMemsetAsync(base + 64, 0, 64, st);
  if (e != cudaSuccess) return cuda_status(e, "clear workspace header");
  // Entries of W whose irrep Q carries no work are zero, and so are, in a
  // general plan, its padding and the entries whose implicit sector has no
  // solution: those plans zero W as a whole first.
  const int64_t fill_n = mode.fill_n < 0 ? P->numel_w : mode.fill_n;
  if ((P->fill_all || (int64_t)pr.n_q * pr.M * pr.N < P->numel_w) && fill_n > 0) {
    // W's own reduced form, real entries: only the sector blocks no irrep writes
    if (P->fill_bv > 0 && !P->fill_all && !P->general && mode.fill_n < 0 && mode.es == 1)
      e = launch_fill_dead(w, P->fill_bv, P->fill_combos, P->fill_written.data(), st);
    else
      e = launch_fill_zero(w, fill_n, st);
    if (e != cudaSuccess) return cuda_status(e, "zero fill");
  }
  if (pr.n_q == 0) return SYMCTR_OK;
  if (P->prof) cudaEventRecord(P->ev[0], st);
  const bool attached = tables_attached(P);
  if (!attached && !P->htab.empty()) pin_tables(P);
  if (!P->tensor_core) {
    if (P->prof) cudaEventRecord(P->ev[1], st);
    if (P->general) {
      const Layout L = make_layout(pr, false, true, P->prec, P->n_slices, P->kpad);
      Tables tab;
      symctr_status s = pass_tables(P, pr, 0, attached, base, L.off_tab, st, &tab);
      if (s != SYMCTR_OK) return s;
      // the table-driven kernel accumulates split K ranges onto a zeroed W (a
      // chained plan's W has not been zeroed above)
      if (!P->fill_all && !mode.accumulate && fill_n > 0) {
        e = launch_fill_zero(w, fill_n, st);
        if (e != cudaSuccess) return cuda_status(e, "zero fill");
      }
      e = launch_gemm_f64(pr, u, v, w, &tab, st);
    } else {
      e = launch_gemm_f64(pr, u, v, w, nullptr, st);
    }
    if (P->prof) cudaEventRecord(P->ev[2], st);
    if (e != cudaSuccess) return cuda_status(e, "gemm_f64");
    if (P->general && !attached && P->pinned) return mark_table_use(P, st);
    return SYMCTR_OK;
  }
  // Q-streaming: as many irreps per pass as the workspace holds.
  int per_pass = pr.n_q;
  if (ws_bytes < P->ws_bytes) {
    per_pass = 0;
    for (int c = pr.n_q - 1; c >= 1 && per_pass == 0; --c) {
      Problem pc = pr;
      pc.n_q = c;
      if (make_layout(pc, true, P->general, P->prec, P->n_slices, P->kpad).bytes <= ws_bytes) per_pass = c;
    }
    if (per_pass == 0) return fail(SYMCTR_ERR_WORKSPACE, "workspace smaller than workspace_bytes_min");
  }
  unsigned* barrier = (unsigned*)(base + 64);
  const bool split = P->prec == SYMCTR_SPLIT_BF16;
  for (int q0 = 0; q0 < pr.n_q; q0 += per_pass) {
    Problem pc = pr;
    if (per_pass < pr.n_q) {
      pc.n_q = per_pass < pr.n_q - q0 ? per_pass : pr.n_q - q0;
      pc.q_base = q0;
      if (q0 > 0) {
        e = cudaMemsetAsync(barrier, 0, 64, st);
        if (e != cudaSuccess) return cuda_status(e, "clear barrier");
      }
    }
    const Layout L = make_layout(pc, true, P->general, P->prec, P->n_slices, P->kpad);
    Tables tab;
    symctr_status s = pass_tables(P, pc, q0, attached, base, L.off_tab, st, &tab);
    if (s != SYMCTR_OK) return s;
    unsigned long long* acc = L.ksplit > 1 ? (unsigned long long*)(base + L.off_acc) : nullptr;
    const int64_t acc_n = L.ksplit > 1 ? (int64_t)pc.n_q * pc.M * pc.N : 0;
    int32_t* ea = split ? (int32_t*)(base + L.off_ea) : nullptr;
    int32_t* eb = split ? (int32_t*)(base + L.off_eb) : nullptr;
    int32_t* part = split && L.off_part ? (int32_t*)(base + L.off_part) : nullptr;
    // operands with row runs take the single-read kernel (real data only)
    const bool rs[2] = {split && pr.es == 1 && P->row_run[0] > 0, split && pr.es == 1 && P->row_run[1] > 0};
    // short rows take the short-row kernel (real data only)
    const bool rt[2] = {split && pr.es == 1 && P->row_tile[0], split && pr.es == 1 && P->row_tile[1]};
    const bool skip[2] = {rs[0] || rt[0], rs[1] || rt[1]};
    // the two-phase kernel runs for an operand left to it, or to zero the
    // split-K sums when no short-row kernel runs
    const bool two_phase = !skip[0] || !skip[1] || !(rt[0] || rt[1]);
    if (two_phase) {
      e = launch_prep(pc, tab, split, P->n_slices, u, v, base + L.off_a, base + L.off_b, ea, eb, part,
                      P->kpad, err, barrier, acc, acc_n, skip, st);
      if (e != cudaSuccess) return cuda_status(e, "operand preparation");
    }
    if (rt[0] || rt[1]) {
      e = launch_rowtile(pc, tab, P->n_slices, rt, u, v, base + L.off_a, base + L.off_b, ea, eb, P->kpad,
                         err, two_phase ? nullptr : acc, two_phase ? 0 : acc_n, st);
      if (e != cudaSuccess) return cuda_status(e, "operand preparation (short rows)");
    }
    for (int op = 0; op < 2; ++op) {
      if (!rs[op]) continue;
      e = launch_rowstream(pc, tab, op, P->n_slices, P->row_run[op], op == 0 ? u : v,
                           base + (op == 0 ? L.off_a : L.off_b), op == 0 ? ea : eb, P->kpad, err, st);
      if (e != cudaSuccess) return cuda_status(e, "operand preparation (single read)");
    }
    if (P->prof && q0 == 0) cudaEventRecord(P->ev[1], st);
    if (split)
      e = launch_gemm_split(pc, tab, P->n_slices, (const uint16_t*)(base + L.off_a),
                            (const uint16_t*)(base + L.off_b), ea, eb, P->kpad, w, err, L.ksplit,
                            acc, st);
    else
      e = launch_gemm_tf32(pc, tab, (const float*)(base + L.off_a),
                           (const float*)(base + L.off_b), P->kpad, w, err, st);
    if (e != cudaSuccess) return cuda_status(e, split ? "gemm_split" : "gemm_tf32");
  }
  if (P->prof) cudaEventRecord(P->ev[2], st);
  if (!attached && P->pinned) return mark_table_use(P, st);
  return SYMCTR_OK;
}

}  // namespace

namespace symctr {

symctr_status contract_into_workspace(const symctr_plan* P, const double* u, const double* v,
                                      double* w, void* ws, size_t ws_bytes, cudaStream_t st) {
  if (!P) return fail(SYMCTR_ERR_NULLPTR, "NULL plan");
  return run_contract(P, u, v, w, ws, ws_bytes, st);
}

uint64_t plan_workspace_bytes(const symctr_plan* P) { return P ? P->ws_bytes : 0; }

uint64_t plan_workspace_bytes_min(const symctr_plan* P) { return P ? P->ws_bytes_min : 0; }

symctr_status record_error(symctr_status st, const char* detail) { return fail(st, detail); }

}  // namespace symctr

static uint64_t own_table_bytes(const symctr_plan* P) {
  return (uint64_t)round_up((int64_t)(P->htab.size() * sizeof(int64_t)), 256);
}

// The plan's tables, then the backward plans' (recursively), each 256-byte aligned.
static uint64_t all_table_bytes(const symctr_plan* P) {
  if (!P) return 0;
  return own_table_bytes(P) + all_table_bytes(P->bwd_u) + all_table_bytes(P->bwd_v);
}

static symctr_status attach_tables(symctr_plan* P, uint8_t* buf, int dev, cudaStream_t st) {
  if (!P) return SYMCTR_OK;
  if (!buf) {
    P->dev_tab = nullptr;
    P->dev_tab_device = -1;
  } else if (!P->htab.empty()) {
    cudaError_t e = cudaMemcpyAsync(buf, P->htab.data(), P->htab.size() * sizeof(int64_t),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_status(e, "attach offset tables");
    if (P->pinned) {
      symctr_status r = mark_table_use(P, st);
      if (r != SYMCTR_OK) return r;
    }
    P->dev_tab = (const int64_t*)buf;
    P->dev_tab_device = dev;
  }
  uint8_t* next = buf ? buf + own_table_bytes(P) : nullptr;
  symctr_status r = attach_tables(P->bwd_u, next, dev, st);
  if (r != SYMCTR_OK) return r;
  return attach_tables(P->bwd_v, next ? next + all_table_bytes(P->bwd_u) : nullptr, dev, st);
}

// The six standard index maps of a plan in the general form (host).
static void plan_axes(const symctr_plan* P, GenAxis* gax) {
  const std::string &lu = P->u.labels, &lv = P->v.labels, &lw = P->w.labels;
  std::vector<int> FV_in_V = P->FV, C_in_V, FU_in_W, FV_in_W;
  int sgn_fu[SYMCTR_MAX_ORDER], sgn_cu[SYMCTR_MAX_ORDER], sgn_cv[SYMCTR_MAX_ORDER],
      sgn_fv[SYMCTR_MAX_ORDER];
  for (size_t i = 0; i < P->FU.size(); ++i) {
    sgn_fu[i] = P->u.sign[P->FU[i]];
    FU_in_W.push_back((int)lw.find(lu[P->FU[i]]));
  }
  for (size_t i = 0; i < P->C.size(); ++i) {
    sgn_cu[i] = P->u.sign[P->C[i]];
    int j = (int)lv.find(lu[P->C[i]]);
    C_in_V.push_back(j);
    sgn_cv[i] = P->v.sign[j];
  }
  for (size_t i = 0; i < P->FV.size(); ++i) {
    sgn_fv[i] = P->v.sign[P->FV[i]];
    FV_in_W.push_back((int)lw.find(lv[P->FV[i]]));
  }
  gax[0] = make_gen_axis(P->u, P->FU, sgn_fu, -1, P->u.z);
  gax[1] = make_gen_axis(P->u, P->C, sgn_cu, +1, 0);
  gax[2] = make_gen_axis(P->v, FV_in_V, sgn_fv, -P->sigma, P->v.z);
  gax[3] = make_gen_axis(P->v, C_in_V, sgn_cv, P->sigma, 0);
  gax[4] = make_gen_axis(P->w, FU_in_W, sgn_fu, -1, P->u.z);
  gax[5] = make_gen_axis(P->w, FV_in_W, sgn_fv, -P->sigma, P->v.z);
}

// The two sides of an operand (its modes `rows`, `cols`, positions in the
// operand) read from `src`'s aligned result, whose output modes are the
// operand's modes in order.  Returns false when the source's free-U modes
// (which fix its irrep) are split between the two sides.
static bool chain_sides(const symctr_plan* src, const std::vector<int>& rows,
                        const std::vector<int>& cols, ChainSide* cr, ChainSide* cc) {
  const int G = src->g.order;
  const std::string &lw = src->w.labels, &lu = src->u.labels, &lv = src->v.labels;
  const int s = (int)src->FU.size(), t = (int)src->FV.size();
  // W positions of the source's free-U and free-V modes, in its aligned order
  std::vector<int> fu_w, fv_w;
  for (int i : src->FU) fu_w.push_back((int)lw.find(lu[i]));
  for (int j : src->FV) fv_w.push_back((int)lw.find(lv[j]));
  // mixed-radix strides of m = (sectors of free-U but the last, their blocks), n likewise
  auto strides = [&](const std::vector<int>& modes) {
    std::vector<int64_t> rad;
    for (size_t i = 0; i + 1 < modes.size(); ++i) rad.push_back(src->w.H[modes[i]]);
    for (int p : modes) rad.push_back(src->w.dim[p]);
    std::vector<int64_t> st(rad.size());
    int64_t acc = 1;
    for (int k = (int)rad.size() - 1; k >= 0; --k) {
      st[k] = acc;
      acc *= rad[k];
    }
    return st;
  };
  const std::vector<int64_t> ms = strides(fu_w), ns = strides(fv_w);
  const int64_t Nsrc = src->prob.N;
  auto fill = [&](const std::vector<int>& modes, ChainSide* c) {
    for (size_t k = 0; k < modes.size(); ++k) {
      const int p = modes[k];   // W position of the source = operand position
      c->coef[k] = 0;
      for (int i = 0; i < s; ++i)
        if (fu_w[i] == p) {
          c->sstride[k] = i < s - 1 ? ms[i] * Nsrc : 0;
          c->bstride[k] = ms[(s - 1) + i] * Nsrc;
          c->coef[k] = src->u.sign[src->FU[i]] * (G / src->u.H[src->FU[i]]);
        }
      for (int j = 0; j < t; ++j)
        if (fv_w[j] == p) {
          c->sstride[k] = j < t - 1 ? ns[j] : 0;
          c->bstride[k] = ns[(t - 1) + j];
        }
    }
    c->batch = false;
    c->z = src->u.z;
    c->q_single = src->prob.q_single;
    c->q0 = src->prob.q0;
    c->q_step = src->prob.q_step;
    c->n_q = src->prob.n_q;
    c->batch_stride = src->prob.M * src->prob.N;
  };
  fill(rows, cr);
  fill(cols, cc);
  int in_rows = 0, in_cols = 0;
  for (int p : fu_w) {
    for (int r : rows) in_rows += r == p;
    for (int c : cols) in_cols += c == p;
  }
  if (in_rows && in_cols) return false;
  (in_cols ? cc : cr)->batch = true;
  return true;
}

extern "C" {

symctr_status symctr_plan_create(const char* einsum, int n_moduli, const int32_t* moduli,
                                 const int8_t* signs_u, const int32_t* charge_u,
                                 const int8_t* signs_v, const int32_t* charge_v,
                                 const int64_t* dims_u, const int64_t* dims_v,
                                 const int8_t* signs_w_or_null, const int32_t* charge_w_or_null,
                                 symctr_precision prec, int n_slices, symctr_plan** out) {
  OpDesc du, dv;
  du.signs = signs_u;
  du.charge = charge_u;
  du.dims = dims_u;
  dv.signs = signs_v;
  dv.charge = charge_v;
  dv.dims = dims_v;
  return build(einsum, n_moduli, moduli, du, dv, signs_w_or_null, charge_w_or_null, prec, n_slices,
               true, out);
}

symctr_status symctr_plan_create_general(const char* einsum, int n_moduli, const int32_t* moduli,
                                         const symctr_operand* u, const symctr_operand* v,
                                         const int8_t* signs_w_or_null,
                                         const int32_t* charge_w_or_null, symctr_precision prec,
                                         int n_slices, symctr_plan** out) {
  if (out) *out = nullptr;
  if (!u || !v) return fail(SYMCTR_ERR_NULLPTR, "NULL operand descriptor");
  OpDesc du, dv;
  du.signs = u->signs;
  du.charge = u->charge;
  du.dims = u->dims;
  du.sectors = u->sectors;
  du.sector_dims = u->sector_dims;
  dv.signs = v->signs;
  dv.charge = v->charge;
  dv.dims = v->dims;
  dv.sectors = v->sectors;
  dv.sector_dims = v->sector_dims;
  return build(einsum, n_moduli, moduli, du, dv, signs_w_or_null, charge_w_or_null, prec, n_slices,
               true, out);
}

symctr_status symctr_plan_query(const symctr_plan* P, symctr_plan_info* o) {
  if (!P || !o) return fail(SYMCTR_ERR_NULLPTR, "NULL argument");
  std::memset(o, 0, sizeof(*o));
  const Problem& pr = P->prob;
  o->order_u = P->u.order();
  o->order_v = P->v.order();
  o->order_w = P->w.order();
  o->s = P->s;
  o->t = P->t;
  o->v = P->vv;
  o->sigma = P->sigma;
  o->n_moduli = P->g.n;
  for (int i = 0; i < P->g.n; ++i) o->moduli[i] = P->g.mod[i];
  o->group_order = P->g.order;
  o->precision = (int32_t)P->prec;
  o->n_slices = P->n_slices;
  for (int i = 0; i < P->w.order(); ++i) {
    o->signs_w[i] = (int8_t)P->w.sign[i];
    o->dims_w[i] = P->w.dim[i];
  }
  g_comps(P->g, P->w.z, o->charge_w);
  o->numel_u = P->numel_u;
  o->numel_v = P->numel_v;
  o->numel_w = P->numel_w;
  o->M = pr.M;
  o->N = pr.N;
  o->K = pr.K;
  o->n_q = pr.n_q;
  o->q_single = pr.q_single;
  o->aligned_numel_u = (int64_t)pr.n_q * pr.M * pr.K;
  o->aligned_numel_v = (int64_t)pr.n_q * pr.N * pr.K;
  o->aligned_numel_w = (int64_t)pr.n_q * pr.M * pr.N;
  o->useful_flops = 2.0 * (double)pr.n_q * (double)pr.M * (double)pr.N * (double)pr.K;
  // transforms move each operand element once in and once out (8 B each way)
  o->transform_bytes = 16.0 * (double)(o->aligned_numel_u + o->aligned_numel_v + o->aligned_numel_w);
  o->workspace_bytes = P->ws_bytes;
  o->workspace_bytes_min = P->ws_bytes_min;
  uint64_t wb = 256;
  if (P->bwd_u && P->bwd_u->ws_bytes > wb) wb = P->bwd_u->ws_bytes;
  if (P->bwd_v && P->bwd_v->ws_bytes > wb) wb = P->bwd_v->ws_bytes;
  o->workspace_bytes_backward = wb;
  o->table_bytes = all_table_bytes(P);
  o->tensor_core = P->tensor_core ? 1 : 0;
  o->general = P->fill_all ? 1 : 0;
  o->q_first = pr.q_single >= 0 ? pr.q_single : pr.q0;
  o->q_step = pr.q_single >= 0 ? 0 : pr.q_step;
  for (int i = 0; i < P->w.order(); ++i) o->sectors_w[i] = P->w.H[i];
  o->single_read_prep = (P->row_run[0] > 0 ? 1 : 0) | (P->row_run[1] > 0 ? 2 : 0) |
                        (P->row_tile[0] ? 4 : 0) | (P->row_tile[1] ? 8 : 0);
  o->chained = P->chained ? 1 : 0;
  // what a contraction zeroes first (real W in its own reduced form): the
  // sector blocks no irrep writes, all of W, or nothing
  o->zero_fill_numel = 0;
  if (P->fill_all || (int64_t)pr.n_q * pr.M * pr.N < P->numel_w) {
    if (P->fill_bv > 0 && !P->fill_all && !P->general) {
      int64_t written = 0;
      for (uint32_t m : P->fill_written) written += __builtin_popcount(m);
      o->zero_fill_numel = (P->fill_combos - written) * P->fill_bv;
    } else {
      o->zero_fill_numel = P->numel_w;
    }
  }
  return SYMCTR_OK;
}

symctr_status symctr_plan_attach_tables(symctr_plan* P, void* tables, size_t bytes, void* stream) {
  if (!P) return fail(SYMCTR_ERR_NULLPTR, "NULL plan");
  if (!tables) return attach_tables(P, nullptr, -1, nullptr);
  if ((uint64_t)bytes < all_table_bytes(P)) return fail(SYMCTR_ERR_WORKSPACE, "table buffer too small");
  if ((uintptr_t)tables % 256 != 0) return fail(SYMCTR_ERR_ARGUMENT, "table buffer not 256-byte aligned");
  if (all_table_bytes(P) == 0) return SYMCTR_OK;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "current device");
  // detach first: a failed copy leaves no half-attached plan behind
  attach_tables(P, nullptr, -1, nullptr);
  symctr_status r = attach_tables(P, (uint8_t*)tables, dev, (cudaStream_t)stream);
  if (r != SYMCTR_OK) attach_tables(P, nullptr, -1, nullptr);
  return r;
}

symctr_status symctr_align(const symctr_plan* P, int operand, int direction, const double* src,
                           double* dst, void* stream) {
  if (!P) return fail(SYMCTR_ERR_NULLPTR, "NULL plan");
  if (operand < 0 || operand > 2 || (direction != 1 && direction != -1))
    return fail(SYMCTR_ERR_ARGUMENT, "operand in {0,1,2}, direction in {+1,-1}");
  const Problem& pr = P->prob;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t covered = operand == 0 ? (int64_t)pr.n_q * pr.M * pr.K
                          : operand == 1 ? (int64_t)pr.n_q * pr.N * pr.K
                                         : (int64_t)pr.n_q * pr.M * pr.N;
  const int64_t total = operand == 0 ? P->numel_u : operand == 1 ? P->numel_v : P->numel_w;
  // an empty side (no irrep carries work: the aligned form has no entries) may be NULL
  if ((!src && (direction > 0 ? total : covered) > 0) || (!dst && (direction > 0 ? covered : total) > 0))
    return fail(SYMCTR_ERR_NULLPTR, "NULL argument");
  if (direction == -1) {
    if (P->fill_all || covered < total) {
      cudaError_t e = launch_fill_zero(dst, total, st);
      if (e != cudaSuccess) return cuda_status(e, "zero fill");
    }
  }
  if (pr.n_q == 0) return SYMCTR_OK;
  if (!P->general)
    return cuda_status(launch_align_f64(pr, operand, direction, src, dst, nullptr, st), "align");
  // general plans: the index maps are the tables (attached, else the
  // page-locked host tables read in place)
  Tables tab;
  const bool attached = tables_attached(P);
  if (!attached) pin_tables(P);
  const int64_t* t0 = attached ? P->dev_tab : P->dtab;
  if (!t0) return fail(SYMCTR_ERR_CUDA, "offset tables could not be mapped; attach them first");
  tab.urow = t0;
  tab.ucol = tab.urow + (int64_t)pr.n_q * pr.M;
  tab.vrow = tab.ucol + (int64_t)pr.n_q * pr.K;
  tab.vcol = tab.vrow + (int64_t)pr.n_q * pr.N;
  tab.wrow = tab.vcol + (int64_t)pr.n_q * pr.K;
  tab.wcol = tab.wrow + (int64_t)pr.n_q * pr.M;
  symctr_status r = cuda_status(launch_align_f64(pr, operand, direction, src, dst, &tab, st), "align");
  if (r == SYMCTR_OK && !attached) r = mark_table_use(P, st);
  return r;
}

symctr_status symctr_contract(const symctr_plan* P, const double* u, const double* v, double* w,
                              void* ws, size_t ws_bytes, void* stream) {
  if (!P) return fail(SYMCTR_ERR_NULLPTR, "NULL plan");
  return run_contract(P, u, v, w, ws, ws_bytes, (cudaStream_t)stream);
}

symctr_status symctr_contract_backward(const symctr_plan* P, const double* gw, const double* u,
                                       const double* v, double* gu, double* gv, void* ws,
                                       size_t ws_bytes, void* stream) {
  if (!P || !gw) return fail(SYMCTR_ERR_NULLPTR, "NULL argument");
  if (P->chained) return fail(SYMCTR_ERR_UNSUPPORTED, "a chained plan has no backward");
  if (!P->bwd_u || !P->bwd_v) return fail(SYMCTR_ERR_ARGUMENT, "plan has no backward");
  cudaStream_t st = (cudaStream_t)stream;
  if (gu) {
    symctr_status s = run_contract(P->bwd_u, gw, v, gu, ws, ws_bytes, st);
    if (s != SYMCTR_OK) return s;
  }
  if (gv) {
    RunMode m;
    m.clear_err = gu == nullptr;   // keep a device error of the first contraction
    symctr_status s = run_contract(P->bwd_v, u, gw, gv, ws, ws_bytes, st, m);
    if (s != SYMCTR_OK) return s;
  }
  return SYMCTR_OK;
}

symctr_status symctr_contract_complex(const symctr_plan* P, int conj_u, int conj_v, const double* u,
                                      const double* v, double* w, void* ws, size_t ws_bytes,
                                      void* stream) {
  if (!P) return fail(SYMCTR_ERR_NULLPTR, "NULL plan");
  if (!w || !u || !v) return fail(SYMCTR_ERR_NULLPTR, "NULL tensor pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const double su = conj_u ? -1.0 : 1.0, sv = conj_v ? -1.0 : 1.0;
  // (Ur + i su Ui)(Vr + i sv Vi) = Ur Vr - su sv Ui Vi + i (sv Ur Vi + su Ui Vr):
  // four real contractions on the real (+0) and imaginary (+1) parts
  struct Term {
    int ui, vi, wi;
    double sign;
    int accumulate;
  };
  const Term terms[4] = {{0, 0, 0, 1.0, 0}, {1, 1, 0, -su * sv, 1}, {0, 1, 1, sv, 0}, {1, 0, 1, su, 1}};
  for (int k = 0; k < 4; ++k) {
    RunMode m;
    m.es = 2;
    m.negate = terms[k].sign < 0 ? 1 : 0;
    m.accumulate = terms[k].accumulate;
    m.clear_err = k == 0;
    m.fill_n = k == 0 ? 2 * P->numel_w : 0;   // both parts of W once
    symctr_status s = run_contract(P, u + terms[k].ui, v + terms[k].vi, w + terms[k].wi, ws, ws_bytes,
                                   st, m);
    if (s != SYMCTR_OK) return s;
  }
  return SYMCTR_OK;
}

symctr_status symctr_check_device_error(const symctr_plan* P, void* ws, void* stream) {
  (void)P;
  if (!ws) {
    // the static scratch array of symctr_contract_static_scratch on this device
    symctr_status st = SYMCTR_OK;
    ws = static_scratch_address(&st);
    if (!ws) return st;
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, ws, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "read device error word");
  e = cudaMemsetAsync(ws, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return cuda_status(e, "clear device error word");
  if (h & DEVERR_TIMEOUT) return fail(SYMCTR_ERR_DEVICE_TIMEOUT, "a kernel's bounded wait expired");
  if (h & DEVERR_NONFINITE) return fail(SYMCTR_ERR_NONFINITE, "non-finite input");
  return SYMCTR_OK;
}

symctr_status symctr_selftest_bounded_wait(void* ws, size_t ws_bytes, int64_t wait_cycles,
                                           void* stream) {
  if (!ws) return fail(SYMCTR_ERR_NULLPTR, "NULL workspace");
  if (ws_bytes < 256) return fail(SYMCTR_ERR_WORKSPACE, "workspace smaller than its 256-byte header");
  if (wait_cycles < 1000) wait_cycles = 1000;
  if (wait_cycles > 2000000000ll) wait_cycles = 2000000000ll;
  return cuda_status(launch_bounded_wait_selftest((unsigned*)ws, (long long)wait_cycles,
                                                  (cudaStream_t)stream),
                     "bounded-wait self-test");
}

const char* symctr_status_string(symctr_status s) {
  switch (s) {
    case SYMCTR_OK: return "SYMCTR_OK";
    case SYMCTR_ERR_EINSUM: return "SYMCTR_ERR_EINSUM";
    case SYMCTR_ERR_SIGNS: return "SYMCTR_ERR_SIGNS";
    case SYMCTR_ERR_SHAPE: return "SYMCTR_ERR_SHAPE";
    case SYMCTR_ERR_CHARGE: return "SYMCTR_ERR_CHARGE";
    case SYMCTR_ERR_UNSUPPORTED: return "SYMCTR_ERR_UNSUPPORTED";
    case SYMCTR_ERR_NULLPTR: return "SYMCTR_ERR_NULLPTR";
    case SYMCTR_ERR_WORKSPACE: return "SYMCTR_ERR_WORKSPACE";
    case SYMCTR_ERR_CUDA: return "SYMCTR_ERR_CUDA";
    case SYMCTR_ERR_DEVICE_TIMEOUT: return "SYMCTR_ERR_DEVICE_TIMEOUT";
    case SYMCTR_ERR_OVERFLOW: return "SYMCTR_ERR_OVERFLOW";
    case SYMCTR_ERR_NONFINITE: return "SYMCTR_ERR_NONFINITE";
    case SYMCTR_ERR_ARGUMENT: return "SYMCTR_ERR_ARGUMENT";
  }
  return "SYMCTR_UNKNOWN";
}

const char* symctr_last_error_detail(void) { return g_detail.c_str(); }

symctr_status symctr_profile_enable(symctr_plan* P, int enable) {
  if (!P) return fail(SYMCTR_ERR_NULLPTR, "NULL plan");
  if (enable && !P->prof) {
    for (int i = 0; i < 3; ++i) {
      cudaError_t e = cudaEventCreate(&P->ev[i]);
      if (e != cudaSuccess) return cuda_status(e, "cudaEventCreate");
    }
    P->prof = true;
  } else if (!enable && P->prof) {
    for (int i = 0; i < 3; ++i) cudaEventDestroy(P->ev[i]);
    P->prof = false;
  }
  return SYMCTR_OK;
}

symctr_status symctr_profile_read(const symctr_plan* P, float* prep_ms, float* gemm_ms,
                                  int* launches) {
  if (!P || !prep_ms || !gemm_ms) return fail(SYMCTR_ERR_NULLPTR, "NULL argument");
  if (launches) *launches = P->last_launches;
  if (!P->prof) return fail(SYMCTR_ERR_ARGUMENT, "profiling not enabled");
  cudaError_t e = cudaEventSynchronize(P->ev[2]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(prep_ms, P->ev[0], P->ev[1]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(gemm_ms, P->ev[1], P->ev[2]);
  return cuda_status(e, "profile read");
}

symctr_status symctr_plan_chain(symctr_plan* P, const symctr_plan* u_from, const symctr_plan* v_from,
                                int w_aligned) {
  if (!P) return fail(SYMCTR_ERR_NULLPTR, "NULL plan");
  if (!u_from && !v_from && !w_aligned) return SYMCTR_OK;
  if (P->chained || P->pinned || P->dev_tab)
    return fail(SYMCTR_ERR_ARGUMENT, "chain a plan once, before its first contraction or table attachment");
  const GroupDesc& g = P->g;
  auto same_tensor = [&](const symctr_plan* src, const Tensor& t) -> bool {
    if (src->g.n != g.n || src->g.order != g.order) return false;
    for (int i = 0; i < g.n; ++i)
      if (src->g.mod[i] != g.mod[i]) return false;
    const Tensor& w = src->w;
    if (w.order() != t.order()) return false;
    bool same = w.z == t.z, neg = w.z == g_neg(g, t.z);
    for (int i = 0; i < t.order(); ++i) {
      if (w.dim[i] != t.dim[i] || w.H[i] != t.H[i] || w.sd[i] != t.sd[i]) return false;
      same = same && w.sign[i] == t.sign[i];
      neg = neg && w.sign[i] == -t.sign[i];
    }
    return same || neg;
  };
  if (u_from && !same_tensor(u_from, P->u))
    return fail(SYMCTR_ERR_SHAPE, "u_from's result is not this plan's U (modes, sectors, sizes or law differ)");
  if (v_from && !same_tensor(v_from, P->v))
    return fail(SYMCTR_ERR_SHAPE, "v_from's result is not this plan's V (modes, sectors, sizes or law differ)");
  ChainSide cs[4];
  std::vector<int> C_in_V;
  for (int i : P->C) C_in_V.push_back((int)P->v.labels.find(P->u.labels[i]));
  if (u_from && !chain_sides(u_from, P->FU, P->C, &cs[0], &cs[1]))
    return fail(SYMCTR_ERR_UNSUPPORTED, "u_from's free-U modes are split between U's free and contracted modes");
  if (v_from && !chain_sides(v_from, P->FV, C_in_V, &cs[2], &cs[3]))
    return fail(SYMCTR_ERR_UNSUPPORTED, "v_from's free-U modes are split between V's free and contracted modes");
  Problem& pr = P->prob;
  GenAxis gax[6];
  plan_axes(P, gax);
  if (pr.n_q > 0) {
    const int64_t total = tables_entries(pr);
    if (total > (int64_t)1 << 28) return fail(SYMCTR_ERR_OVERFLOW, "offset tables too large");
    std::vector<int64_t> tab;
    try {
      tab.resize((size_t)total);
    } catch (const std::bad_alloc&) {
      return fail(SYMCTR_ERR_OVERFLOW, "offset tables: host allocation failed");
    }
    int64_t* t = tab.data();
    const int64_t ext[6] = {pr.M, pr.K, pr.N, pr.K, pr.M, pr.N};
    for (int k = 0; k < 6; ++k)
      for (int b = 0; b < pr.n_q; ++b) {
        const int Q = batch_irrep(pr, b);
        for (int64_t r = 0; r < ext[k]; ++r) {
          int64_t off;
          if (k < 2 && u_from)
            off = chain_offset(gax[k], cs[k], g, Q, r);
          else if (k >= 2 && k < 4 && v_from)
            off = chain_offset(gax[k], cs[k], g, Q, r);
          else if (k >= 4 && w_aligned)   // W_hat[b][m][n]: rows (b M + m) N, columns n
            off = gen_offset(gax[k], g, Q, r) < 0 ? -1 : (k == 4 ? ((int64_t)b * pr.M + r) * pr.N : r);
          else
            off = gen_offset(gax[k], g, Q, r);
          *t++ = off;
        }
      }
    P->htab.swap(tab);
  }
  P->chained = true;
  P->general = true;
  pr.general = 1;
  P->row_run[0] = P->row_run[1] = 0;
  if (u_from) P->numel_u = (int64_t)u_from->prob.n_q * u_from->prob.M * u_from->prob.N;
  if (v_from) P->numel_v = (int64_t)v_from->prob.n_q * v_from->prob.M * v_from->prob.N;
  if (w_aligned) P->numel_w = (int64_t)pr.n_q * pr.M * pr.N;
  Layout full = make_layout(pr, P->tensor_core, true, P->prec, P->n_slices, P->kpad);
  if (!full.ok) return fail(SYMCTR_ERR_OVERFLOW, "aligned operand too large");
  P->ws_bytes = P->ws_bytes_min = full.bytes;
  if (P->tensor_core && pr.q_single < 0 && pr.n_q > 1) {
    Problem one = pr;
    one.n_q = 1;
    P->ws_bytes_min = make_layout(one, true, true, P->prec, P->n_slices, P->kpad).bytes;
  }
  return SYMCTR_OK;
}

void symctr_plan_destroy(symctr_plan* P) {
  if (!P) return;
  symctr_profile_enable(P, 0);
  if (P->pinned) {
    // wait for the last contraction that read the page-locked tables on each
    // stream that used them (nothing else on the device is waited for)
    for (const auto& u : P->uses) {
      cudaEventSynchronize(u.ev);
      cudaEventDestroy(u.ev);
    }
    P->uses.clear();
    cudaHostUnregister((void*)P->htab.data());
    cudaGetLastError();
  }
  symctr_plan_destroy(P->bwd_u);
  symctr_plan_destroy(P->bwd_v);
  delete P;
}

}  // extern "C"
