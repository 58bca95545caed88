// Host check of axis_offset (the separable index map of an aligned operand
// side, Sec. 2.3 / Alg. 2) against a brute-force definition: the explicit
// sector labels and block digits are read off the aligned index, and the
// implicit sector is found by trying every label of the group against the
// conservation law, factor by factor.  Random groups (one to three cyclic
// factors), random maps, every irrep, and every index of small maps (2048
// random ones of larger maps); both the 32-bit and the 64-bit instantiation.  Prints "ok <cases>" and exits 0, or reports the
// first mismatch and exits 1.
#include <cstdio>
#include <cstdint>
#include <random>

#include "symctr_internal.h"

using namespace symctr;

namespace {

int digit(const GroupDesc& g, int label, int f) {
  for (int k = g.n - 1; k > f; --k) label /= g.mod[k];
  return label % g.mod[f];
}

int64_t brute(const AxisMap& a, const GroupDesc& g, int Q, int64_t r) {
  int64_t off = 0;
  for (int i = a.n - 1; i >= 0; --i) {
    off += (r % a.D[i]) * a.bstride[i];
    r /= a.D[i];
  }
  int s[SYMCTR_MAX_ORDER];
  for (int i = a.n - 2; i >= 0; --i) {
    s[i] = (int)(r % g.order);
    r /= g.order;
    off += s[i] * a.sstride[i];
  }
  int found = -1;
  for (int t = 0; t < g.order && found < 0; ++t) {
    bool ok = true;
    for (int f = 0; f < g.n && ok; ++f) {
      int sum = (a.sign[a.n - 1] > 0 ? 1 : -1) * digit(g, t, f) - (a.qa > 0 ? 1 : -1) * digit(g, Q, f) -
                digit(g, a.z, f);
      for (int i = 0; i < a.n - 1; ++i) sum += (a.sign[i] > 0 ? 1 : -1) * digit(g, s[i], f);
      ok = ((sum % g.mod[f]) + g.mod[f]) % g.mod[f] == 0;
    }
    if (ok) found = t;
  }
  return off + found * a.sstride[a.n - 1];
}

}  // namespace

int main() {
  std::mt19937 rng(20070856);
  auto uni = [&](int lo, int hi) { return std::uniform_int_distribution<int>(lo, hi)(rng); };
  long cases = 0;
  for (int trial = 0; trial < 400; ++trial) {
    GroupDesc g{};
    g.n = uni(1, 3);
    g.order = 1;
    for (int f = 0; f < g.n; ++f) {
      g.mod[f] = uni(2, 5);
      g.order *= g.mod[f];
    }
    AxisMap a{};
    a.n = uni(1, 4);
    a.size = 1;
    for (int i = 0; i < a.n; ++i) {
      a.D[i] = uni(1, 4);
      a.sign[i] = uni(0, 1) ? 1 : -1;
      a.sstride[i] = uni(0, 3) == 0 ? 0 : uni(1, 100000);
      a.bstride[i] = uni(1, 1000);
      a.size *= a.D[i];
      if (i + 1 < a.n) a.size *= g.order;
    }
    a.qa = uni(0, 1) ? 1 : -1;
    a.z = uni(0, g.order - 1);
    // every index of small maps, 2048 random ones of larger maps
    const bool all = a.size <= 2048;
    std::uniform_int_distribution<int64_t> pick(0, a.size - 1);
    for (int Q = 0; Q < g.order; ++Q) {
      for (int64_t j = 0; j < (all ? a.size : 2048); ++j) {
        const int64_t r = all ? j : pick(rng);
        const int64_t want = brute(a, g, Q, r);
        const int64_t got = axis_offset(a, g, Q, r);
        const int64_t got64 = axis_offset_t<int64_t>(a, g, Q, r);
        ++cases;
        if (got != want || got64 != want) {
          std::printf("mismatch: trial %d group n=%d order=%d Q=%d r=%lld want %lld got %lld / %lld\n", trial,
                      g.n, g.order, Q, (long long)r, (long long)want, (long long)got, (long long)got64);
          return 1;
        }
      }
    }
  }
  std::printf("ok %ld\n", cases);
  return 0;
}
