// Host schedulers: rotation lists and Hamiltonians -> tile passes + groups.
//
// Rotation lists keep their order (the circuit order of the product formula
// after Eq. ucc); only runs of consecutive, mutually commuting rotations with
// the same xmask are merged into one group, and consecutive groups whose
// xmasks span at most T dimensions (with the low chunk qubits) share one pass
// over HBM.
//
// Hamiltonian terms may be visited in any order (Eq. qubit-ham-detail is a
// plain sum), so their xmask groups are packed into passes greedily, on tiles
// spanned by unit qubit vectors, to minimise the number of passes.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <stdexcept>

#include "q2_internal.h"

namespace q2 {

namespace {

inline int popc64(uint64_t v) { return __builtin_popcountll(v); }
inline int parity64(uint64_t v) { return __builtin_parityll(v); }
inline int high_bit(uint64_t v) { return 63 - __builtin_clzll(v); }

// GF(2) span of a few vectors, with the coordinates of any member in terms of
// the inserted (original) basis vectors.
struct Gf2Basis {
  std::vector<uint64_t> orig;   // basis vectors as inserted
  std::vector<uint64_t> red;    // reduced rows, distinct highest bits, descending
  std::vector<uint32_t> comb;   // red[i] = XOR of orig[l] over bits l of comb[i]

  int rank() const { return (int)orig.size(); }

  uint64_t reduce(uint64_t v, uint32_t &c) const {
    c = 0;
    for (size_t i = 0; i < red.size(); ++i) {
      if ((v >> high_bit(red[i])) & 1) {
        v ^= red[i];
        c ^= comb[i];
      }
    }
    return v;
  }
  bool contains(uint64_t v) const {
    uint32_t c;
    return reduce(v, c) == 0;
  }
  uint32_t coords(uint64_t v) const {
    uint32_t c;
    if (reduce(v, c) != 0) throw std::logic_error("coords of a vector outside the span");
    return c;
  }
  bool add(uint64_t v) {
    uint32_t c;
    uint64_t rem = reduce(v, c);
    if (rem == 0) return false;
    int l = (int)orig.size();
    orig.push_back(v);
    uint32_t cc = c ^ (1u << l);
    int hb = high_bit(rem);
    size_t pos = 0;
    while (pos < red.size() && high_bit(red[pos]) > hb) ++pos;
    red.insert(red.begin() + pos, rem);
    comb.insert(comb.begin() + pos, cc);
    return true;
  }
  uint64_t pivot_mask() const {
    uint64_t m = 0;
    for (uint64_t r : red) m |= 1ull << high_bit(r);
    return m;
  }
};

struct RawGroup {
  uint64_t x;
  uint8_t kind;
  std::vector<int64_t> members;   // term / rotation indices
  Gf2Basis basis;                 // span of the members' zmasks
};

int align_up_int(int v, int a) { return (v + a - 1) / a * a; }

uint64_t nmask_of(int n) { return n >= 64 ? ~0ull : ((1ull << n) - 1ull); }

// Local basis of a pass: e_0..e_{C-1} first (C as large as the span allows),
// then the generators reduced modulo the low unit vectors, filled up to T
// dimensions with the lowest independent unit vectors.
struct Tiling {
  uint64_t w[T_LIMIT];
  uint64_t umask;
  int T, C;
  Gf2Basis wb;   // basis w_0..w_{T-1} in order, for coordinates

  uint64_t packz(uint64_t z) const {
    uint64_t lo = 0;
    for (int b = 0; b < T; ++b) lo |= (uint64_t)parity64(w[b] & z) << b;
    return (extract_bits(z, umask) << T) | lo;
  }
  uint32_t local_coords(uint64_t x) const { return wb.coords(x); }
};

Tiling make_tiling(int n, int T, int Cmin, const std::vector<uint64_t> &gens) {
  Gf2Basis span;
  for (int q = 0; q < Cmin; ++q) span.add(1ull << q);
  for (uint64_t g : gens) span.add(g);
  if (span.rank() > T) throw std::logic_error("pass generators exceed the tile dimension");
  for (int q = 0; q < n && span.rank() < T; ++q) span.add(1ull << q);
  int C = 0;
  while (C < T && C < n && span.contains(1ull << C)) ++C;
  Tiling t;
  std::memset(t.w, 0, sizeof(t.w));
  t.T = T;
  t.C = C;
  const uint64_t low = (C >= 64) ? ~0ull : ((1ull << C) - 1);
  for (int b = 0; b < C; ++b) {
    t.w[b] = 1ull << b;
    t.wb.add(t.w[b]);
  }
  int b = C;
  for (uint64_t v : span.orig) {
    if (b >= T) break;
    uint64_t r = v & ~low;
    if (r == 0) continue;
    if (t.wb.add(r)) t.w[b++] = r;
  }
  if (b != T) throw std::logic_error("tiling basis incomplete");
  t.umask = nmask_of(n) & ~t.wb.pivot_mask();
  return t;
}

// Code of a local index for a group: bits parity(l & bp_k), local part only.
uint32_t local_code(const GroupDesc &d, uint64_t l, int T) {
  const uint64_t lm = (1ull << T) - 1;
  uint32_t c = 0;
  for (int k = 0; k < d.r; ++k) c |= (uint32_t)parity64(l & d.bp[k] & lm) << k;
  return c;
}

// Device descriptor of one group inside a pass (pair-enumeration tables
// included; block tables are filled by form_blocks).
GroupDesc make_desc(const RawGroup &g, const Tiling &tl, uint32_t lut_off) {
  GroupDesc d;
  std::memset(&d, 0, sizeof(d));
  const int T = tl.T;
  d.kind = g.kind;
  d.r = (uint8_t)g.basis.rank();
  d.lut = lut_off;
  for (int l = 0; l < d.r; ++l) d.bp[l] = tl.packz(g.basis.orig[l]);
  const bool diag = (g.kind == KIND_DIAG);
  d.xl = diag ? 0u : tl.local_coords(g.x);
  d.pivot = diag ? 0 : (uint8_t)high_bit(d.xl);
  const int64_t per_tile = diag ? (1ll << T) : (1ll << (T - 1));
  const int64_t P = std::max<int64_t>(1, per_tile / NT);
  if (P > P_MAX || (!diag && P > 16)) throw std::logic_error("tile too large for the per-thread tables");
  for (int64_t j = 0; j < P; ++j) {
    uint32_t v = (uint32_t)(NT * j);
    if (!diag) {
      v = insert_zero(v, d.pivot);
      d.pu[j] = (uint16_t)v;
    }
    d.pjcode[j] = (uint8_t)local_code(d, v, T);
  }
  for (int lane = 0; lane < 32; ++lane) {
    const uint32_t v = diag ? (uint32_t)lane : insert_zero((uint32_t)lane, d.pivot);
    d.plane[lane] = (uint8_t)local_code(d, v, T);
  }
  for (int w = 0; w < NT / 32; ++w) {
    const uint32_t v = diag ? (uint32_t)(32 * w) : insert_zero((uint32_t)(32 * w), d.pivot);
    d.pwarp[w] = (uint8_t)local_code(d, v, T);
  }
  return d;
}

// base(s): s with zero bits inserted at the (ascending) pivots.
uint32_t block_base(uint32_t s, const BlockDesc &b) {
  for (int i = 0; i < b.d; ++i) s = insert_zero(s, b.piv[i]);
  return s;
}

// Partition groups[first, last) of a pass into register blocks of span <= dmax.
// With reorder, groups are first arranged greedily so that blocks stay small
// (allowed for Hamiltonian terms, whose sum is order-free).
void form_blocks(std::vector<GroupDesc> &groups, size_t first, size_t last, int T, int dmax,
                 bool reorder, std::vector<BlockDesc> &blocks) {
  if (reorder) {
    std::vector<GroupDesc> rest(groups.begin() + first, groups.begin() + last), out;
    std::vector<char> used(rest.size(), 0);
    size_t left = rest.size();
    while (left) {
      Gf2Basis span;
      for (;;) {
        size_t best = rest.size();
        int best_add = 99;
        for (size_t i = 0; i < rest.size(); ++i) {
          if (used[i]) continue;
          const uint64_t xl = rest[i].xl;
          const int add = (xl == 0 || span.contains(xl)) ? 0 : 1;
          if (span.rank() + add > dmax) continue;
          if (add < best_add) {
            best = i;
            best_add = add;
            if (add == 0) break;
          }
        }
        if (best == rest.size()) break;
        used[best] = 1;
        --left;
        if (rest[best].xl) span.add(rest[best].xl);
        out.push_back(rest[best]);
      }
    }
    std::copy(out.begin(), out.end(), groups.begin() + first);
  }
  size_t g = first;
  while (g < last) {
    Gf2Basis span;
    size_t e = g;
    while (e < last) {
      const uint64_t xl = groups[e].xl;
      if (xl && !span.contains(xl) && span.rank() >= dmax) break;
      if (xl) span.add(xl);
      ++e;
    }
    // Basis of the block: the groups' own xmasks in order of appearance, so a
    // group that opens a new dimension pairs combos along one basis bit.
    // Pivots are the highest bits of the echelon rows: the basis restricted
    // to them is invertible, so base(s) ^ comb[c] enumerates the tile once.
    std::vector<uint64_t> v = span.orig;
    std::vector<int> piv;
    for (uint64_t r : span.red) piv.push_back(high_bit(r));
    if (v.empty()) {                      // diagonal-only block: any one local direction
      v.push_back(1);
      piv.push_back(0);
    }
    std::sort(piv.begin(), piv.end());
    BlockDesc b;
    std::memset(&b, 0, sizeof(b));
    b.d = (uint8_t)v.size();
    for (int i = 0; i < b.d; ++i) b.piv[i] = (uint8_t)piv[i];
    for (uint32_t c = 0; c < (1u << b.d); ++c) {
      uint64_t o = 0;
      for (int i = 0; i < b.d; ++i)
        if ((c >> i) & 1) o ^= v[i];
      b.comb[c] = (uint16_t)o;
    }
    const int64_t ncos = 1ll << (T - b.d);
    const int64_t J = std::max<int64_t>(1, ncos / NT);
    if (J > 16) throw std::logic_error("too many cosets per thread");
    for (int64_t j = 0; j < J; ++j) b.uj[j] = (uint16_t)block_base((uint32_t)(NT * j), b);
    b.g_begin = (uint16_t)(g - first);
    b.g_end = (uint16_t)(e - first);
    for (size_t kk = g; kk < e; ++kk) {
      GroupDesc &d = groups[kk];
      // coordinates of xl in the basis v
      d.a = d.xl ? (uint8_t)span.coords(d.xl) : (uint8_t)0;
      const int k = (int)(kk - g);
      if (k == b.canon && k < b.d && d.kind == KIND_REAL && d.a == (1u << k)) ++b.canon;
      for (uint32_t c = 0; c < (1u << b.d); ++c) d.bccode[c] = (uint8_t)local_code(d, b.comb[c], T);
      for (int64_t j = 0; j < J; ++j) d.bjcode[j] = (uint8_t)local_code(d, b.uj[j], T);
      for (int lane = 0; lane < 32; ++lane) d.blane[lane] = (uint8_t)local_code(d, block_base(lane, b), T);
      for (int w = 0; w < NT / 32; ++w) d.bwarp[w] = (uint8_t)local_code(d, block_base(32 * w, b), T);
    }
    blocks.push_back(b);
    g = e;
  }
}

int block_dmax(int T, int cap = D_MAX) { return std::max(1, std::min(cap, T - 8)); }

PassDesc make_pass(const Tiling &tl) {
  PassDesc pd;
  std::memset(&pd, 0, sizeof(pd));
  for (int b = 0; b < T_LIMIT; ++b) pd.w[b] = tl.w[b];
  pd.umask = tl.umask;
  pd.T = tl.T;
  pd.C = tl.C;
  return pd;
}

}  // namespace

int64_t count_x_groups(int64_t n_terms, const uint64_t *x) {
  std::vector<uint64_t> v(x, x + n_terms);
  std::sort(v.begin(), v.end());
  return (int64_t)(std::unique(v.begin(), v.end()) - v.begin());
}

// --------------------------------------------------------------- rotations

RotPlan build_rot_plan(int n, int64_t n_rot, const uint64_t *x, const uint64_t *z, int Tmax,
                       int Cmin) {
  RotPlan P;
  P.n = n;
  const int T = std::min(Tmax, n);
  P.T = T;
  const int C = std::min(Cmin, T);

  // 1. groups of consecutive commuting rotations with one xmask
  std::vector<RawGroup> groups;
  for (int64_t k = 0; k < n_rot; ++k) {
    const int ny = popc64(x[k] & z[k]);
    const uint8_t kind = x[k] == 0 ? KIND_DIAG : ((ny & 1) ? KIND_REAL : KIND_XROT);
    bool join = false;
    if (!groups.empty()) {
      RawGroup &g = groups.back();
      if (g.x == x[k] && g.kind == kind && (int)g.members.size() < M_MAX &&
          (g.basis.contains(z[k]) || g.basis.rank() < R_MAX_ROT))
        join = true;
    }
    if (!join) {
      groups.emplace_back();
      groups.back().x = x[k];
      groups.back().kind = kind;
    }
    groups.back().members.push_back(k);
    groups.back().basis.add(z[k]);
  }

  // 2. passes: consecutive groups whose xmasks span <= T dimensions with e_0..e_{C-1}
  struct PassRange {
    size_t gb, ge;
    std::vector<uint64_t> gens;
  };
  std::vector<PassRange> ranges;
  {
    Gf2Basis W;
    for (int q = 0; q < C; ++q) W.add(1ull << q);
    PassRange cur{0, 0, {}};
    int rots = 0, luts = 0;
    for (size_t g = 0; g < groups.size(); ++g) {
      const uint64_t xg = groups[g].x;
      const int m = (int)groups[g].members.size();
      const int nl = 1 << groups[g].basis.rank();
      const int lut_at = align_up_int(luts, nl);   // every group's table starts at a multiple of 2^r
      const bool fits = (xg == 0 || W.contains(xg) || W.rank() < T) && rots + m <= RP_MAX &&
                        (int)(g - cur.gb) < G_STAGE && lut_at + nl <= LUT_STAGE;
      if (!fits && g > cur.gb) {
        cur.ge = g;
        ranges.push_back(cur);
        cur = PassRange{g, 0, {}};
        W = Gf2Basis();
        for (int q = 0; q < C; ++q) W.add(1ull << q);
        rots = 0;
        luts = 0;
      }
      if (xg != 0 && W.add(xg)) cur.gens.push_back(xg);
      rots += m;
      luts = align_up_int(luts, nl) + nl;
    }
    if (cur.gb < groups.size()) {
      cur.ge = groups.size();
      ranges.push_back(cur);
    }
  }

  // 3. descriptors
  P.rot_coord.resize(n_rot);
  P.rot_sigma.resize(n_rot);
  P.signmask.resize(n_rot);
  uint32_t lut = 0;
  for (const PassRange &pr : ranges) {
    const Tiling tl = make_tiling(n, T, C, pr.gens);
    PassDesc pd = make_pass(tl);
    pd.g_begin = (int)P.groups.size();
    pd.rot_begin = (int)groups[pr.gb].members.front();
    lut = (uint32_t)align_up_int((int)lut, 1 << R_MAX_ROT);
    for (size_t g = pr.gb; g < pr.ge; ++g) {
      const RawGroup &rg = groups[g];
      lut = (uint32_t)align_up_int((int)lut, 1 << rg.basis.rank());
      GroupDesc d = make_desc(rg, tl, lut);
      d.m = (uint8_t)rg.members.size();
      d.rot0 = (uint32_t)(rg.members.front() - pd.rot_begin);
      P.groups.push_back(d);
      P.grp_rot_begin.push_back((int)rg.members.front());
      const uint32_t ncode = 1u << d.r;
      for (int64_t k : rg.members) {
        const int ny = popc64(x[k] & z[k]);
        int sigma = 1;
        if (rg.kind == KIND_REAL) sigma = (ny % 4 == 1) ? 1 : -1;
        else if (rg.kind == KIND_XROT) sigma = (ny % 4 == 0) ? 1 : -1;
        const uint32_t co = rg.basis.coords(z[k]);
        P.rot_coord[k] = (uint8_t)co;
        P.rot_sigma[k] = (int8_t)sigma;
        uint64_t sm = 0;
        for (uint32_t c = 0; c < ncode; ++c) {
          const int s = sigma * (parity64(c & co) ? -1 : 1);
          if (s < 0) sm |= 1ull << c;
        }
        P.signmask[k] = sm;
      }
      lut += ncode;
    }
    pd.g_end = (int)P.groups.size();
    pd.lut_begin = (int)P.groups[pd.g_begin].lut;
    pd.lut_count = (int)lut - pd.lut_begin;
    pd.b_begin = (int)P.blocks.size();
    form_blocks(P.groups, pd.g_begin, pd.g_end, T, block_dmax(T), false, P.blocks);
    pd.b_end = (int)P.blocks.size();
    pd.rot_end = (int)(groups[pr.ge - 1].members.back() + 1);
    P.max_pass_rots = std::max(P.max_pass_rots, pd.rot_end - pd.rot_begin);
    bool canon4 = pd.g_end - pd.g_begin <= 16 && pd.b_end > pd.b_begin;
    for (int b = pd.b_begin; b < pd.b_end && canon4; ++b) {
      const BlockDesc &bd = P.blocks[b];
      canon4 = bd.d == 4 && bd.canon == 4 && bd.g_end - bd.g_begin == 4;
    }
    P.pass_canon4.push_back(canon4 ? 1 : 0);
    P.passes.push_back(pd);
  }
  P.lut_entries = lut;
  return P;
}

void set_param_weights(RotPlan &p, const int32_t *param, const double *coef) {
  const size_t n_rot = p.signmask.size();
  p.fold.assign(coef, coef + n_rot);
  p.wlut.clear();
  for (size_t g = 0; g < p.groups.size(); ++g) {
    GroupDesc &d = p.groups[g];
    const int k0 = p.grp_rot_begin[g];
    bool one = true;
    for (int k = k0 + 1; k < k0 + d.m; ++k) one = one && param[k] == param[k0];
    d.one_param = one ? 1 : 0;
    d.wlut = 0;
    if (!one) continue;
    d.wlut = (uint32_t)p.wlut.size();
    const uint32_t ncode = 1u << d.r;
    for (uint32_t c = 0; c < ncode; ++c) {
      double w = 0.0;
      for (int k = k0; k < k0 + d.m; ++k) w += ((p.signmask[k] >> c) & 1) ? -coef[k] : coef[k];
      p.wlut.push_back(w);
    }
    p.fold[k0] = 1.0;
    for (int k = k0 + 1; k < k0 + d.m; ++k) p.fold[k] = 0.0;
  }
  p.pass_one_param.assign(p.passes.size(), 1);
  for (size_t i = 0; i < p.passes.size(); ++i)
    for (int g = p.passes[i].g_begin; g < p.passes[i].g_end; ++g)
      if (!p.groups[g].one_param) p.pass_one_param[i] = 0;
}

void RotPlan::build_lut(const double *phi, double *lut2) const {
  for (size_t g = 0; g < groups.size(); ++g) {
    const GroupDesc &d = groups[g];
    const uint32_t ncode = 1u << d.r;
    const int k0 = grp_rot_begin[g];
    for (uint32_t c = 0; c < ncode; ++c) {
      double beta = 0.0;
      for (int k = k0; k < k0 + d.m; ++k) {
        const double half = 0.5 * phi[k];
        beta += ((signmask[k] >> c) & 1) ? -half : half;
      }
      lut2[2 * (d.lut + c)] = std::cos(beta);
      lut2[2 * (d.lut + c) + 1] = std::sin(beta);
    }
  }
}

// --------------------------------------------------------------- Hamiltonian

HamPlan build_ham_plan(int n, int64_t n_terms, const uint64_t *x, const uint64_t *z,
                       const double *c, int Tmax, int Cmin, int lut_stage) {
  HamPlan H;
  H.n = n;
  const int T = std::min(Tmax, n);
  H.T = T;
  const int C = std::min(Cmin, T);
  const uint64_t lowmask = (C >= 64) ? ~0ull : ((1ull << C) - 1);

  std::vector<int64_t> order(n_terms);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    return x[a] != x[b] ? x[a] < x[b] : z[a] < z[b];
  });

  // 1. subgroups: same xmask, code rank <= R_MAX
  std::vector<RawGroup> groups;
  for (int64_t t : order) {
    bool join = false;
    if (!groups.empty()) {
      RawGroup &g = groups.back();
      if (g.x == x[t] && (g.basis.contains(z[t]) || g.basis.rank() < R_MAX)) join = true;
    }
    if (!join) {
      groups.emplace_back();
      groups.back().x = x[t];
      groups.back().kind = x[t] == 0 ? KIND_DIAG : KIND_PAIR;
    }
    groups.back().members.push_back(t);
    groups.back().basis.add(z[t]);
  }

  // 2a. groups whose xmask has more qubits than a tile has room for: tiles
  // spanned by the xmasks themselves (one dimension per independent xmask)
  std::vector<char> done(groups.size(), 0);
  size_t remaining = groups.size();
  std::vector<std::vector<size_t>> pass_groups;
  std::vector<std::vector<uint64_t>> pass_gens;
  {
    Gf2Basis W;
    std::vector<size_t> cur;
    std::vector<uint64_t> gens;
    auto reset = [&]() {
      W = Gf2Basis();
      for (int q = 0; q < C; ++q) W.add(1ull << q);
      cur.clear();
      gens.clear();
    };
    reset();
    int luts = 0;
    for (size_t g = 0; g < groups.size(); ++g) {
      if (popc64(groups[g].x | lowmask) <= T) continue;
      const int nl = 1 << groups[g].basis.rank();
      if ((!W.contains(groups[g].x) && W.rank() >= T) || (int)cur.size() >= G_STAGE ||
          align_up_int(luts, nl) + nl > lut_stage) {
        luts = 0;
        pass_groups.push_back(cur);
        pass_gens.push_back(gens);
        reset();
      }
      if (W.add(groups[g].x)) gens.push_back(groups[g].x);
      cur.push_back(g);
      luts = align_up_int(luts, nl) + nl;
      done[g] = 1;
      --remaining;
    }
    if (!cur.empty()) {
      pass_groups.push_back(cur);
      pass_gens.push_back(gens);
    }
  }

  // 2b. greedy packing of the other subgroups into passes over unit-qubit tiles
  while (remaining > 0) {
    uint64_t L = lowmask;
    std::vector<size_t> chosen;
    int luts = 0;
    bool full = false;
    for (;;) {
      for (size_t g = 0; g < groups.size() && !full; ++g)
        if (!done[g] && (groups[g].x & ~L) == 0) {
          const int nl = 1 << groups[g].basis.rank();
          if ((int)chosen.size() >= G_STAGE || align_up_int(luts, nl) + nl > lut_stage) {
            full = true;
            break;
          }
          done[g] = 1;
          --remaining;
          chosen.push_back(g);
          luts = align_up_int(luts, nl) + nl;
        }
      if (remaining == 0 || full) break;
      int freq[64] = {0};
      for (size_t g = 0; g < groups.size(); ++g)
        if (!done[g]) {
          uint64_t v = groups[g].x & ~L;
          while (v) {
            ++freq[__builtin_ctzll(v)];
            v &= v - 1;
          }
        }
      size_t best = groups.size();
      int best_new = 65;
      long best_score = -1;
      for (size_t g = 0; g < groups.size(); ++g) {
        if (done[g]) continue;
        const uint64_t nb = groups[g].x & ~L;
        const int nnew = popc64(nb);
        if (popc64(L | nb) > T) continue;
        long score = 0;
        uint64_t v = nb;
        while (v) {
          score += freq[__builtin_ctzll(v)];
          v &= v - 1;
        }
        if (nnew < best_new || (nnew == best_new && score > best_score)) {
          best = g;
          best_new = nnew;
          best_score = score;
        }
      }
      if (best == groups.size()) break;
      L |= groups[best].x;
    }
    if (chosen.empty()) throw std::logic_error("Hamiltonian group does not fit a tile");
    std::stable_sort(chosen.begin(), chosen.end(), [&](size_t a, size_t b) {
      return groups[a].kind < groups[b].kind || (groups[a].kind == groups[b].kind && a < b);
    });
    pass_groups.push_back(chosen);
    std::vector<uint64_t> gens;
    for (int q = 0; q < n; ++q)
      if ((L >> q) & 1) gens.push_back(1ull << q);
    pass_gens.push_back(gens);
  }

  // 3. descriptors and LUT of combined coefficients (R, Q) per code
  uint32_t lut = 0;
  std::vector<size_t> raw_of;   // raw group of each descriptor, in descriptor order
  for (size_t p = 0; p < pass_groups.size(); ++p) {
    const Tiling tl = make_tiling(n, T, C, pass_gens[p]);
    PassDesc pd = make_pass(tl);
    pd.g_begin = (int)H.groups.size();
    pd.rot_begin = pd.rot_end = 0;
    lut = (uint32_t)align_up_int((int)lut, 1 << R_MAX);
    for (size_t g : pass_groups[p]) {
      raw_of.push_back(g);
      const RawGroup &rg = groups[g];
      lut = (uint32_t)align_up_int((int)lut, 1 << rg.basis.rank());
      GroupDesc d = make_desc(rg, tl, lut);
      // Every member with an even Y count gives a real pair coefficient
      // (Q = 0 at every code): such groups run the real-coefficient path.
      bool any_odd = false;
      for (int64_t t : rg.members) any_odd |= (popc64(x[t] & z[t]) & 1) != 0;
      if (d.kind == KIND_PAIR && !any_odd) d.kind = KIND_REAL;
      H.groups.push_back(d);
      const uint32_t ncode = 1u << d.r;
      H.lut2.resize(2 * (size_t)(lut + ncode), 0.0);
      for (int64_t t : rg.members) {
        const int ny = popc64(x[t] & z[t]);
        const uint32_t co = rg.basis.coords(z[t]);
        for (uint32_t cd = 0; cd < ncode; ++cd) {
          const int par = parity64(cd & co);
          if ((ny & 1) == 0) {
            const int s = ((ny / 2) + par) & 1;
            H.lut2[2 * (size_t)(lut + cd)] += s ? -c[t] : c[t];
          } else {
            const int s = (par + (ny % 4 == 3)) & 1;
            H.lut2[2 * (size_t)(lut + cd) + 1] += s ? -c[t] : c[t];
          }
        }
      }
      lut += ncode;
    }
    pd.g_end = (int)H.groups.size();
    pd.lut_begin = (int)H.groups[pd.g_begin].lut;
    pd.lut_count = (int)lut - pd.lut_begin;
    pd.b_begin = (int)H.blocks.size();
    // block formation may reorder the pass's descriptors: carry each one's raw group along
    // (the LUT offset identifies a descriptor uniquely within a pass)
    std::vector<std::pair<uint32_t, size_t>> before;
    for (int g = pd.g_begin; g < pd.g_end; ++g) before.push_back({H.groups[g].lut, raw_of[g]});
    form_blocks(H.groups, pd.g_begin, pd.g_end, T, block_dmax(T, D_MAX_EXPECT), true, H.blocks);
    std::sort(before.begin(), before.end());
    for (int g = pd.g_begin; g < pd.g_end; ++g) {
      auto it = std::lower_bound(before.begin(), before.end(), std::make_pair(H.groups[g].lut, (size_t)0));
      raw_of[g] = it->second;
    }
    pd.b_end = (int)H.blocks.size();
    bool lean = true;
    for (int g = pd.g_begin; g < pd.g_end; ++g)
      lean = lean && (H.groups[g].kind == KIND_REAL || H.groups[g].kind == KIND_DIAG);
    for (int b = pd.b_begin; b < pd.b_end; ++b) lean = lean && H.blocks[b].d <= 3;
    H.pass_lean.push_back(lean ? 1 : 0);
    H.passes.push_back(pd);
  }
  H.lut_entries = lut;
  H.term_begin.assign(1, 0);
  for (size_t g = 0; g < H.groups.size(); ++g) {
    const RawGroup &rg = groups[raw_of[g]];
    H.term_idx.insert(H.term_idx.end(), rg.members.begin(), rg.members.end());
    H.term_begin.push_back((int64_t)H.term_idx.size());
  }
  return H;
}

void restrict_to_shard(HamPlan &p, int shard, int n_shards) {
  if (n_shards <= 1) return;
  const size_t np = p.passes.size();
  std::vector<double> cost(np, 1.0);
  for (size_t i = 0; i < np; ++i)
    for (int g = p.passes[i].g_begin; g < p.passes[i].g_end; ++g) cost[i] += p.groups[g].kind == KIND_DIAG ? 2.0 : 1.0;
  std::vector<size_t> order(np);
  std::iota(order.begin(), order.end(), (size_t)0);
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
  std::vector<double> load(n_shards, 0.0);
  std::vector<int> owner(np, 0);
  for (size_t i : order) {
    int best = 0;
    for (int s = 1; s < n_shards; ++s)
      if (load[s] < load[best]) best = s;
    owner[i] = best;
    load[best] += cost[i];
  }
  std::vector<PassDesc> keep;
  std::vector<uint8_t> keep_lean;
  for (size_t i = 0; i < np; ++i)
    if (owner[i] == shard) {
      keep.push_back(p.passes[i]);
      keep_lean.push_back(i < p.pass_lean.size() ? p.pass_lean[i] : 0);
    }
  p.passes.swap(keep);
  p.pass_lean.swap(keep_lean);
}

std::vector<float> HamPlan::lut_f32() const {
  std::vector<float> f(lut2.size());
  for (size_t i = 0; i < lut2.size(); ++i) f[i] = (float)lut2[i];
  for (const GroupDesc &g : groups) {
    if (g.kind != KIND_REAL && g.kind != KIND_DIAG) continue;
    for (uint32_t c = 0; c < (1u << g.r); ++c) f[2 * (size_t)(g.lut + c) + 1] = f[2 * (size_t)(g.lut + c)];
  }
  return f;
}

}  // namespace q2
