/*
 * COMPASS oracle -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.
 *
 * A plain, slow, single-threaded CPU restatement of what the hot path computes:
 * the push-down Fast-AGMS sketch build and the sketch-merging join-size estimate of
 * Izenov, Datta, Rusu, Shin, "COMPASS: Online Sketch-based Query Optimization for
 * In-Memory Databases" (arXiv 2102.02440).  Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or constant with the CUDA library; the two are compared on the same inputs.
 *
 * Arithmetic is exact: hashes in unsigned __int128, counters in int32 (the paper uses
 * 4-byte counters, Sec. 6.1 "Implementation"), estimates in arbitrary-precision signed
 * integers (int128 fast path, promoted to a limb vector on overflow), one rounding to
 * double at the very end.
 *
 * Pinned by tests/test_oracle_*.py against: Python big-int hash arithmetic, brute-force
 * filters and exact join sizes, linearity, per-row sum of signs, identity-hash histograms,
 * the worked merge values of Sec. 4.2, the brute-force contraction enumerator, the
 * explicit 3-chain double sum of Sec. 4.1, seed-averaged unbiasedness, and finite
 * differences for the MLP.  The accuracy of merged estimates against true multi-way join
 * sizes in random-hash mode is parity unpinned: the paper calls merging a heuristic.
 */
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

typedef __int128 i128;
typedef unsigned __int128 u128;

namespace {

const uint64_t kP = (1ULL << 61) - 1;  // Mersenne prime 2^61 - 1

/* ------------------------------------------------------------------ hashing */

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): state += golden gamma, then the
 * variant-13 finaliser.  Used only to derive hash parameters from a seed. */
struct SplitMix64 {
  uint64_t state;
  uint64_t next() {
    state += 0x9E3779B97F4A7C15ULL;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
  }
};

uint64_t draw61(SplitMix64& g) {
  uint64_t v = g.next() >> 3;  // 61 random bits
  return v == kP ? 0 : v;      // field element in [0, p)
}

/* key -> field element: the residue of the (sign-extended) key modulo p, in [0, p).
 * Injective on (-p, p), so every int32 key and nearly every int64 key is its own
 * element; an int32 and an int64 column holding the same value hash identically. */
uint64_t field_of_key(int64_t key) {
  int64_t r = key % (int64_t)kP;  // C++ remainder: sign of the dividend, |r| < p
  if (r < 0) r += (int64_t)kP;
  return (uint64_t)r;
}

/* Carter-Wegman: bucket h(x) = ((a x + b) mod p) mod w  (2-wise independent),
 * sign xi(x) from the parity of (c3 x^3 + c2 x^2 + c1 x + c0) mod p (4-wise). */
void hash_eval(const uint64_t* hp, int w, int64_t key, int* bucket, int* sign) {
  const u128 x = field_of_key(key);
  const u128 lin = ((u128)hp[0] * x + hp[1]) % kP;
  *bucket = (int)(uint64_t)(lin % (u128)w);
  const u128 x2 = (x * x) % kP;
  const u128 x3 = (x2 * x) % kP;
  const u128 poly = ((u128)hp[5] * x3 + (u128)hp[4] * x2 + (u128)hp[3] * x + hp[2]) % kP;
  *sign = (((uint64_t)poly) & 1) ? -1 : +1;
}

/* --------------------------------------------------------------- big integers */

struct Big {
  int s = 0;                 // -1, 0, +1
  std::vector<uint32_t> m;   // magnitude, little endian base 2^32, no leading zero limbs
};

void trim(std::vector<uint32_t>& m) {
  while (!m.empty() && m.back() == 0) m.pop_back();
}

Big big_from_i128(i128 v) {
  Big b;
  if (v == 0) return b;
  b.s = v < 0 ? -1 : 1;
  u128 u = v < 0 ? (u128)(-(v + 1)) + 1 : (u128)v;
  while (u) {
    b.m.push_back((uint32_t)u);
    u >>= 32;
  }
  return b;
}

int cmp_mag(const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) {
  if (a.size() != b.size()) return a.size() < b.size() ? -1 : 1;
  for (size_t i = a.size(); i-- > 0;)
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  return 0;
}

std::vector<uint32_t> add_mag(const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) {
  std::vector<uint32_t> r(std::max(a.size(), b.size()) + 1, 0);
  uint64_t c = 0;
  for (size_t i = 0; i < r.size(); i++) {
    uint64_t t = c;
    if (i < a.size()) t += a[i];
    if (i < b.size()) t += b[i];
    r[i] = (uint32_t)t;
    c = t >> 32;
  }
  trim(r);
  return r;
}

std::vector<uint32_t> sub_mag(const std::vector<uint32_t>& a, const std::vector<uint32_t>& b) {  // a >= b
  std::vector<uint32_t> r(a.size(), 0);
  int64_t br = 0;
  for (size_t i = 0; i < a.size(); i++) {
    int64_t t = (int64_t)a[i] - br - (i < b.size() ? (int64_t)b[i] : 0);
    br = t < 0 ? 1 : 0;
    r[i] = (uint32_t)(t + (br << 32));
  }
  trim(r);
  return r;
}

Big big_add(const Big& x, const Big& y) {
  if (x.s == 0) return y;
  if (y.s == 0) return x;
  Big r;
  if (x.s == y.s) {
    r.s = x.s;
    r.m = add_mag(x.m, y.m);
    return r;
  }
  int c = cmp_mag(x.m, y.m);
  if (c == 0) return r;
  if (c > 0) {
    r.s = x.s;
    r.m = sub_mag(x.m, y.m);
  } else {
    r.s = y.s;
    r.m = sub_mag(y.m, x.m);
  }
  return r;
}

Big big_mul(const Big& x, const Big& y) {
  Big r;
  if (x.s == 0 || y.s == 0) return r;
  std::vector<uint32_t> m(x.m.size() + y.m.size(), 0);
  for (size_t i = 0; i < x.m.size(); i++) {
    uint64_t c = 0;
    for (size_t j = 0; j < y.m.size(); j++) {
      uint64_t t = (uint64_t)x.m[i] * y.m[j] + m[i + j] + c;
      m[i + j] = (uint32_t)t;
      c = t >> 32;
    }
    size_t k = i + y.m.size();
    while (c) {
      uint64_t t = (uint64_t)m[k] + c;
      m[k] = (uint32_t)t;
      c = t >> 32;
      k++;
    }
  }
  trim(m);
  r.s = x.s * y.s;
  r.m = std::move(m);
  return r;
}

bool big_to_i128(const Big& b, i128* out) {
  if (b.s == 0) {
    *out = 0;
    return true;
  }
  if (b.m.size() > 4) return false;
  u128 u = 0;
  for (size_t i = b.m.size(); i-- > 0;) u = (u << 32) | b.m[i];
  const u128 lim = (u128)1 << 127;
  if (b.s > 0) {
    if (u >= lim) return false;
    *out = (i128)u;
  } else {
    if (u > lim) return false;
    *out = u == lim ? (i128)(-((i128)(lim - 1))) - 1 : -(i128)u;
  }
  return true;
}

/* Round-to-nearest-even conversion of an exact integer to IEEE-754 binary64,
 * written from the definition: keep the top 53 significant bits, look at the
 * remainder against one half ulp, break exact ties to an even significand. */
double big_to_double(const Big& b) {
  if (b.s == 0) return 0.0;
  int top = (int)b.m.size() * 32 - 1;
  while (!((b.m[top / 32] >> (top % 32)) & 1)) top--;
  // top = index of the most significant set bit; the value has top+1 bits.
  auto bit = [&](int k) -> int { return k < 0 ? 0 : (int)((b.m[k / 32] >> (k % 32)) & 1); };
  if (top < 53) {
    double r = 0.0;
    for (int k = top; k >= 0; k--) r = r * 2.0 + bit(k);
    return b.s * r;
  }
  uint64_t sig = 0;  // 53 bits: positions top .. top-52
  for (int k = top; k > top - 53; k--) sig = (sig << 1) | (uint64_t)bit(k);
  const int half = bit(top - 53);
  bool sticky = false;
  for (int k = top - 54; k >= 0 && !sticky; k--) sticky = bit(k) != 0;
  if (half && (sticky || (sig & 1))) sig++;
  int exp = top - 52;
  if (sig == (1ULL << 53)) {
    sig >>= 1;
    exp++;
  }
  return b.s * std::ldexp((double)sig, exp);
}

std::string big_to_dec(const Big& b) {
  if (b.s == 0) return "0";
  std::vector<uint32_t> m = b.m;
  std::string digits;
  while (!m.empty()) {
    uint64_t rem = 0;
    for (size_t i = m.size(); i-- > 0;) {
      uint64_t cur = (rem << 32) | m[i];
      m[i] = (uint32_t)(cur / 1000000000ULL);
      rem = cur % 1000000000ULL;
    }
    trim(m);
    for (int k = 0; k < 9; k++) {
      digits.push_back((char)('0' + rem % 10));
      rem /= 10;
      if (m.empty() && rem == 0) break;
    }
  }
  while (digits.size() > 1 && digits.back() == '0') digits.pop_back();
  if (b.s < 0) digits.push_back('-');
  std::reverse(digits.begin(), digits.end());
  return digits;
}

/* Exact signed number: int128 while it fits, big integer otherwise. */
struct Num {
  bool isbig = false;
  i128 v = 0;
  Big b;
};

Num num_i(i128 v) {
  Num n;
  n.v = v;
  return n;
}
Big num_big(const Num& n) { return n.isbig ? n.b : big_from_i128(n.v); }
Num num_norm(Big b) {
  i128 v;
  if (big_to_i128(b, &v)) return num_i(v);
  Num n;
  n.isbig = true;
  n.b = std::move(b);
  return n;
}
Num num_add(const Num& x, const Num& y) {
  if (!x.isbig && !y.isbig) {
    i128 r;
    if (!__builtin_add_overflow(x.v, y.v, &r)) return num_i(r);
  }
  return num_norm(big_add(num_big(x), num_big(y)));
}
Num num_neg(const Num& x) {
  Big b = num_big(x);
  b.s = -b.s;
  return num_norm(b);
}
Num num_mul(const Num& x, const Num& y) {
  if (!x.isbig && !y.isbig) {
    i128 r;
    if (!__builtin_mul_overflow(x.v, y.v, &r)) return num_i(r);
  }
  return num_norm(big_mul(num_big(x), num_big(y)));
}
int num_sign(const Num& x) { return x.isbig ? x.b.s : (x.v > 0) - (x.v < 0); }
int num_cmp(const Num& x, const Num& y) { return num_sign(num_add(x, num_neg(y))); }
double num_to_double(const Num& x) { return big_to_double(num_big(x)); }

/* ------------------------------------------------------- sketch-merging estimate */

struct Graph {
  int nt, ne;
  const int32_t* eu;
  const int32_t* ev;
  const int32_t* const* sk;  // sk[2*e + end] -> int32 [d][w]; end 0 = eu side, 1 = ev side
  int d, w;
};

/* One table's part of the contraction (Sec. 4.2, sketch merging, iterated over the
 * table's relevant edges in ascending edge id).  The merged tensor of the table is
 * T[j_1..j_k] = s_l[j_l] with l the smallest index attaining min_l |s_l[j_l]|
 * (the "<=" of the merge equation keeps the left operand on ties).  Summing T times
 * the incoming messages over every index except the output edge's, split by which l
 * attains the minimum, gives threshold sums over the incoming messages:
 *   G_l^>(tau) = sum of m_l[j] over |s_l[j]| >  tau,
 *   G_l^>=(tau) = sum of m_l[j] over |s_l[j]| >= tau.
 * Edge l' loses to the winner l iff |s_l'| > |s_l| (l' < l) or >= (l' > l).
 * p = index of the output edge, or -1 at the root (then a single scalar is returned). */
struct EdgeIn {
  const int32_t* s;          // this table's sketch row for the edge (length w)
  const std::vector<Num>* m; // incoming message (length w); null for the output edge
  std::vector<int64_t> abs_sorted;
  std::vector<int> ord;      // bucket indices sorted by (|s|, index)
  std::vector<Num> suffix;   // suffix[q] = sum_{r >= q} m[ord[r]]
};

int64_t iabs32(int32_t v) { return v < 0 ? -(int64_t)v : (int64_t)v; }

Num G(const EdgeIn& e, bool strict, int64_t tau) {
  size_t q = strict ? std::upper_bound(e.abs_sorted.begin(), e.abs_sorted.end(), tau) - e.abs_sorted.begin()
                    : std::lower_bound(e.abs_sorted.begin(), e.abs_sorted.end(), tau) - e.abs_sorted.begin();
  return e.suffix[q];
}

void prepare(EdgeIn& e, int w) {
  e.ord.resize(w);
  for (int j = 0; j < w; j++) e.ord[j] = j;
  std::sort(e.ord.begin(), e.ord.end(), [&](int a, int b) {
    int64_t x = iabs32(e.s[a]), y = iabs32(e.s[b]);
    return x != y ? x < y : a < b;
  });
  e.abs_sorted.resize(w);
  for (int q = 0; q < w; q++) e.abs_sorted[q] = iabs32(e.s[e.ord[q]]);
  if (e.m) {
    e.suffix.assign(w + 1, num_i(0));
    for (int q = w - 1; q >= 0; q--) e.suffix[q] = num_add(e.suffix[q + 1], (*e.m)[e.ord[q]]);
  }
}

/* returns the message vector (p >= 0) or a one-element vector with the root scalar */
std::vector<Num> table_rule(std::vector<EdgeIn>& in, int p, int w) {
  const int k = (int)in.size();
  for (int l = 0; l < k; l++) prepare(in[l], w);
  // q_l[j] = s_l[j] m_l[j] prod_{l' != l, p} G_l'^{cmp(l',l)}(|s_l[j]|), prefix sums in |s_l| order
  std::vector<std::vector<Num>> pre(k);
  Num root_sum = num_i(0);
  for (int l = 0; l < k; l++) {
    if (l == p) continue;
    std::vector<Num> q(w);
    for (int j = 0; j < w; j++) {
      Num t = num_mul(num_i(in[l].s[j]), (*in[l].m)[j]);
      const int64_t tau = iabs32(in[l].s[j]);
      for (int l2 = 0; l2 < k && num_sign(t) != 0; l2++) {
        if (l2 == l || l2 == p) continue;
        t = num_mul(t, G(in[l2], /*strict=*/l2 < l, tau));
      }
      q[j] = t;
    }
    if (p < 0) {
      for (int j = 0; j < w; j++) root_sum = num_add(root_sum, q[j]);
      continue;
    }
    pre[l].assign(w + 1, num_i(0));
    for (int r = 0; r < w; r++) pre[l][r + 1] = num_add(pre[l][r], q[in[l].ord[r]]);
  }
  if (p < 0) return std::vector<Num>(1, root_sum);
  std::vector<Num> out(w);
  for (int jp = 0; jp < w; jp++) {
    const int64_t tau = iabs32(in[p].s[jp]);
    // winner = output edge p
    Num t = num_i(in[p].s[jp]);
    for (int l = 0; l < k && num_sign(t) != 0; l++) {
      if (l == p) continue;
      t = num_mul(t, G(in[l], /*strict=*/l < p, tau));
    }
    // winner = input edge l, restricted by the output edge: |s_l| < tau if l > p, <= tau if l < p
    for (int l = 0; l < k; l++) {
      if (l == p) continue;
      const auto& as = in[l].abs_sorted;
      size_t cnt = l > p ? std::lower_bound(as.begin(), as.end(), tau) - as.begin()
                         : std::upper_bound(as.begin(), as.end(), tau) - as.begin();
      t = num_add(t, pre[l][cnt]);
    }
    out[jp] = t;
  }
  return out;
}

struct Plan {
  std::vector<int> tables;       // BFS order from the lowest table id
  std::vector<int> parent_edge;  // per table (-1 at root / outside)
  std::vector<int> edges;        // induced edges, ascending
  std::vector<char> tree;        // per edge
  std::vector<int> nontree;      // induced edges not in the BFS tree, ascending
};

int make_plan(const Graph& g, uint64_t mask, Plan* pl) {
  if (mask == 0 || g.nt > 64 || (g.nt < 64 && (mask >> g.nt) != 0)) return -1;
  pl->parent_edge.assign(g.nt, -1);
  pl->tree.assign(g.ne, 0);
  for (int e = 0; e < g.ne; e++) {
    if (g.eu[e] < 0 || g.eu[e] >= g.nt || g.ev[e] < 0 || g.ev[e] >= g.nt || g.eu[e] == g.ev[e]) return -1;
    if (((mask >> g.eu[e]) & 1) && ((mask >> g.ev[e]) & 1)) pl->edges.push_back(e);
  }
  int root = 0;
  while (!((mask >> root) & 1)) root++;
  std::vector<char> seen(g.nt, 0);
  seen[root] = 1;
  pl->tables.push_back(root);
  for (size_t h = 0; h < pl->tables.size(); h++) {
    const int t = pl->tables[h];
    for (int e : pl->edges) {
      int o = g.eu[e] == t ? g.ev[e] : (g.ev[e] == t ? g.eu[e] : -1);
      if (o < 0 || seen[o]) continue;
      seen[o] = 1;
      pl->parent_edge[o] = e;
      pl->tree[e] = 1;
      pl->tables.push_back(o);
    }
  }
  if ((int)pl->tables.size() != __builtin_popcountll(mask)) return -1;  // not connected
  for (int e : pl->edges)
    if (!pl->tree[e]) pl->nontree.push_back(e);
  return 0;
}

const int32_t* sketch_row(const Graph& g, int e, int t, int row) {
  const int end = g.eu[e] == t ? 0 : 1;
  return g.sk[2 * e + end] + (size_t)row * g.w;
}

/* Tree contraction for one sketch row with the non-tree edge indices fixed to cond[]. */
Num contract_tree(const Graph& g, const Plan& pl, int row, const std::vector<int>& cond) {
  std::vector<std::vector<Num>> msg(g.nt);
  std::vector<std::vector<Num>> unit(pl.nontree.size());
  for (size_t c = 0; c < pl.nontree.size(); c++) {
    unit[c].assign(g.w, num_i(0));
    unit[c][cond[c]] = num_i(1);
  }
  for (size_t h = pl.tables.size(); h-- > 0;) {
    const int t = pl.tables[h];
    std::vector<EdgeIn> in;
    int p = -1;
    for (int e : pl.edges) {
      if (g.eu[e] != t && g.ev[e] != t) continue;
      EdgeIn x;
      x.s = sketch_row(g, e, t, row);
      x.m = nullptr;
      if (e == pl.parent_edge[t]) {
        p = (int)in.size();
      } else if (pl.tree[e]) {
        const int child = g.eu[e] == t ? g.ev[e] : g.eu[e];
        x.m = &msg[child];
      } else {
        size_t c = std::find(pl.nontree.begin(), pl.nontree.end(), e) - pl.nontree.begin();
        x.m = &unit[c];
      }
      in.push_back(std::move(x));
    }
    std::vector<Num> out = table_rule(in, p, g.w);
    if (p < 0) return out[0];
    msg[t] = std::move(out);
  }
  return num_i(0);
}

/* Sum over every assignment of the non-tree edge indices (cycle conditioning). */
Num contract(const Graph& g, const Plan& pl, int row) {
  std::vector<int> cond(pl.nontree.size(), 0);
  Num total = num_i(0);
  if (pl.nontree.empty()) return contract_tree(g, pl, row, cond);
  while (true) {
    total = num_add(total, contract_tree(g, pl, row, cond));
    size_t c = 0;
    while (c < cond.size() && ++cond[c] == g.w) cond[c++] = 0;
    if (c == cond.size()) break;
  }
  return total;
}

/* The definition itself, by enumeration of every edge-index assignment: the product of
 * the merged tensors of all tables of the sub-plan, summed.  Exponential; tiny w only. */
Num brute_force(const Graph& g, const Plan& pl, int row) {
  const size_t ne = pl.edges.size();
  std::vector<int> j(ne, 0);
  std::vector<int> pos(g.ne, -1);
  for (size_t i = 0; i < ne; i++) pos[pl.edges[i]] = (int)i;
  Num total = num_i(0);
  while (true) {
    Num prod = num_i(1);
    for (int t : pl.tables) {
      int64_t best = -1;
      int32_t val = 0;
      for (int e : pl.edges) {  // ascending edge id: first strict minimum wins
        if (g.eu[e] != t && g.ev[e] != t) continue;
        const int32_t v = sketch_row(g, e, t, row)[j[pos[e]]];
        if (best < 0 || iabs32(v) < best) {
          best = iabs32(v);
          val = v;
        }
      }
      prod = num_mul(prod, num_i(val));
    }
    total = num_add(total, prod);
    size_t c = 0;
    while (c < ne && ++j[c] == g.w) j[c++] = 0;
    if (c == ne) break;
  }
  return total;
}

/* median of the row estimates (Sec. 3.2): middle value for odd d, exact mean of the two
 * middle values for even d; one rounding to double. */
double median_of(std::vector<Num> v) {
  std::sort(v.begin(), v.end(), [](const Num& a, const Num& b) { return num_cmp(a, b) < 0; });
  const size_t d = v.size();
  if (d % 2 == 1) return num_to_double(v[d / 2]);
  return num_to_double(num_add(v[d / 2 - 1], v[d / 2])) / 2.0;  // halving is exact
}

/* ------------------------------------------------------------------ MLP helpers */

float bf16_round(float f) {  // IEEE binary32 -> bfloat16, round to nearest even
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) {  // inf / nan: truncate, keep nan quiet
    if (u & 0x007FFFFFu) u |= 0x00400000u;
    u &= 0xFFFF0000u;
  } else {
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7FFFu + lsb;
    u &= 0xFFFF0000u;
  }
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

}  // namespace

/* ======================================================================= C ABI */
extern "C" {

int orc_version(void) { return 1; }

/* Raw SplitMix64 outputs, for pinning the generator against published values. */
int orc_splitmix64(uint64_t seed, int n, uint64_t* out) {
  SplitMix64 g{seed};
  for (int i = 0; i < n; i++) out[i] = g.next();
  return 0;
}

/* Hash parameters: per edge e (ascending), per row i (ascending), fields a, b, c0, c1,
 * c2, c3, each the top 61 bits of the next SplitMix64 output (value p maps to 0);
 * a = 0 is replaced by 1.  out[(e*d + i)*6 + f]. */
int orc_hash_params(uint64_t seed, int n_edges, int d, uint64_t* out) {
  if (n_edges < 0 || d <= 0 || !out) return -1;
  SplitMix64 g{seed};
  for (int e = 0; e < n_edges; e++)
    for (int i = 0; i < d; i++) {
      uint64_t* h = out + ((size_t)e * d + i) * 6;
      for (int f = 0; f < 6; f++) h[f] = draw61(g);
      if (h[0] == 0) h[0] = 1;
    }
  return 0;
}

int orc_hash_eval(const uint64_t* hp, int w, int64_t n, const int64_t* keys, int32_t* bucket, int32_t* sign) {
  if (w <= 0 || !hp) return -1;
  for (int64_t r = 0; r < n; r++) {
    int b, s;
    hash_eval(hp, w, keys[r], &b, &s);
    bucket[r] = b;
    sign[r] = s;
  }
  return 0;
}

/* Push-down selection + Fast-AGMS update (Sec. 2 "Partitioned query execution";
 * Sec. 3.2 counter update C[i][h_i(x)] += xi_i(x)).  For each tuple in row order: the
 * conjunction of predicates (RANGE lo <= v < hi, EQ v == lo, IN bit v of a bitmap) is
 * evaluated; a survivor adds xi to bucket h in every row of every sketch of the table.
 * counters: [n_sketches][d][w] int32, zeroed first unless accumulate != 0.
 * Returns 0, or -1 on an invalid argument. */
int orc_build(int64_t n_rows, int n_cols, const void* const* cols, const int32_t* col_dtype, int n_preds,
              const int32_t* pred_col, const int32_t* pred_op, const int64_t* pred_lo, const int64_t* pred_hi,
              const uint32_t* const* pred_bitmap, const int64_t* pred_nbits, int n_sketches, const int32_t* key_col,
              const int32_t* edge_id, int n_edges, int d, int w, const uint64_t* hash, int accumulate,
              int32_t* counters, int64_t* survivors) {
  if (n_rows < 0 || n_rows > 2147483647LL || d <= 0 || w <= 0 || n_sketches < 0) return -1;
  for (int s = 0; s < n_sketches; s++)
    if (key_col[s] < 0 || key_col[s] >= n_cols || edge_id[s] < 0 || edge_id[s] >= n_edges) return -1;
  for (int q = 0; q < n_preds; q++)
    if (pred_col[q] < 0 || pred_col[q] >= n_cols || pred_op[q] < 0 || pred_op[q] > 2) return -1;
  auto value = [&](int c, int64_t r) -> int64_t {
    return col_dtype[c] == 0 ? (int64_t)((const int32_t*)cols[c])[r] : ((const int64_t*)cols[c])[r];
  };
  const size_t total = (size_t)n_sketches * d * w;
  if (!accumulate) {
    std::memset(counters, 0, total * sizeof(int32_t));
    *survivors = 0;
  }
  for (int64_t r = 0; r < n_rows; r++) {
    bool keep = true;
    for (int q = 0; q < n_preds && keep; q++) {
      const int64_t v = value(pred_col[q], r);
      if (pred_op[q] == 0) keep = pred_lo[q] <= v && v < pred_hi[q];
      else if (pred_op[q] == 1) keep = v == pred_lo[q];
      else keep = v >= 0 && v < pred_nbits[q] && ((pred_bitmap[q][v >> 5] >> (v & 31)) & 1u);
    }
    if (!keep) continue;
    *survivors += 1;
    for (int s = 0; s < n_sketches; s++) {
      const int64_t key = value(key_col[s], r);
      for (int i = 0; i < d; i++) {
        int b, sg;
        hash_eval(hash + ((size_t)edge_id[s] * d + i) * 6, w, key, &b, &sg);
        uint32_t* c = (uint32_t*)counters + ((size_t)s * d + i) * w + b;
        *c = *c + (uint32_t)sg;  // int32 wrap-exact
      }
    }
  }
  return 0;
}

/* Estimate of one sub-plan (bit t of mask = table t).  |S| = 1: the exact survivor
 * count (push-down gives exact selectivities).  |S| >= 2: per sketch row, the full
 * contraction of the merged tensors over the induced edges (method 0: spanning-tree
 * message passing with cycle conditioning; method 1: brute-force enumeration), then the
 * median over rows.  row_dec: d * 2048 chars of decimal row estimates (each NUL-terminated;
 * a row that needs more digits makes the call fail with -3); row_dbl: [d].
 * Returns 0, -1 invalid / not connected, -2 too large for method 1. */
int orc_estimate(int n_tables, int n_edges, const int32_t* edge_u, const int32_t* edge_v,
                 const int32_t* const* sketches, const int64_t* survivors, int d, int w, uint64_t mask, int method,
                 char* row_dec, double* row_dbl, double* est) {
  if (d <= 0 || w <= 0 || n_tables <= 0 || n_edges < 0) return -1;
  Graph g{n_tables, n_edges, edge_u, edge_v, sketches, d, w};
  Plan pl;
  if (make_plan(g, mask, &pl) != 0) return -1;
  std::vector<Num> rows(d);
  if (pl.tables.size() == 1) {
    for (int i = 0; i < d; i++) rows[i] = num_i(survivors[pl.tables[0]]);
  } else {
    if (method == 1) {
      double space = std::pow((double)w, (double)pl.edges.size());
      if (space > 5e7) return -2;
    }
    for (int i = 0; i < d; i++) rows[i] = method == 1 ? brute_force(g, pl, i) : contract(g, pl, i);
  }
  for (int i = 0; i < d; i++) {
    if (row_dbl) row_dbl[i] = num_to_double(rows[i]);
    if (row_dec) {
      std::string s = big_to_dec(num_big(rows[i]));
      if (s.size() > 2047) return -3;
      std::strncpy(row_dec + (size_t)i * 2048, s.c_str(), 2047);
      row_dec[(size_t)i * 2048 + 2047] = 0;
    }
  }
  *est = median_of(rows);
  return 0;
}

/* Exact double of a decimal integer string (the oracle's own rounding), for tests. */
double orc_dec_to_double(const char* s) {
  Big b;
  int sign = 1;
  if (*s == '-') {
    sign = -1;
    s++;
  }
  for (; *s; s++) {
    b = big_add(big_mul(b, big_from_i128(10)), big_from_i128(*s - '0'));
  }
  if (b.s) b.s = sign;
  return big_to_double(b);
}

/* Exact two-way join size of two key multisets (histogram dot product).
 * out_dec: 64 chars decimal. */
int orc_join2(int64_t na, const int64_t* a, int64_t nb, const int64_t* b, char* out_dec, double* out_dbl) {
  std::vector<int64_t> x(a, a + na), y(b, b + nb);
  std::sort(x.begin(), x.end());
  std::sort(y.begin(), y.end());
  u128 total = 0;
  size_t i = 0, j = 0;
  while (i < x.size() && j < y.size()) {
    if (x[i] < y[j]) i++;
    else if (y[j] < x[i]) j++;
    else {
      const int64_t k = x[i];
      uint64_t ca = 0, cb = 0;
      while (i < x.size() && x[i] == k) ca++, i++;
      while (j < y.size() && y[j] == k) cb++, j++;
      total += (u128)ca * cb;
    }
  }
  Big bb = big_from_i128((i128)total);
  std::string s = big_to_dec(bb);
  std::strncpy(out_dec, s.c_str(), 63);
  out_dec[63] = 0;
  *out_dbl = big_to_double(bb);
  return 0;
}

/* Exact two-way join size of two key multisets with every key in [0, domain): the dot
 * product of the two key histograms, O(na + nb + domain).  Returns -1 for a key outside the
 * domain.  *out = the size (below 2^128 for any na, nb < 2^63). */
int orc_join2_dense(int64_t na, const int32_t* a, int64_t nb, const int32_t* b, int64_t domain, uint64_t* out_lo,
                    uint64_t* out_hi) {
  if (domain < 1) return -1;
  std::vector<uint64_t> ha((size_t)domain, 0), hb((size_t)domain, 0);
  for (int64_t i = 0; i < na; i++) {
    if (a[i] < 0 || a[i] >= domain) return -1;
    ha[(size_t)a[i]]++;
  }
  for (int64_t i = 0; i < nb; i++) {
    if (b[i] < 0 || b[i] >= domain) return -1;
    hb[(size_t)b[i]]++;
  }
  u128 total = 0;
  for (int64_t k = 0; k < domain; k++) total += (u128)ha[(size_t)k] * hb[(size_t)k];
  *out_lo = (uint64_t)total;
  *out_hi = (uint64_t)(total >> 64);
  return 0;
}

/* Exact multi-way join size by nested loops (tiny tables only).  Table t has n_rows[t]
 * tuples; keys[2*e + end] is the join-key column of endpoint `end` of edge e, aligned
 * with that table's tuples.  A tuple combination counts iff every edge's two keys match. */
int orc_join_brute(int n_tables, int n_edges, const int32_t* edge_u, const int32_t* edge_v, const int64_t* n_rows,
                   const int64_t* const* keys, uint64_t mask, char* out_dec, double* out_dbl) {
  std::vector<int> ts;
  for (int t = 0; t < n_tables; t++)
    if ((mask >> t) & 1) ts.push_back(t);
  std::vector<int64_t> pick(n_tables, -1);
  Big total;
  double space = 1;
  for (int t : ts) space *= (double)std::max<int64_t>(n_rows[t], 1);
  if (space > 2e8) return -2;
  // iterative odometer over the selected tables
  std::vector<int64_t> idx(ts.size(), 0);
  for (int t : ts)
    if (n_rows[t] == 0) {
      std::strncpy(out_dec, "0", 63);
      *out_dbl = 0;
      return 0;
    }
  uint64_t count = 0;
  while (true) {
    for (size_t q = 0; q < ts.size(); q++) pick[ts[q]] = idx[q];
    bool ok = true;
    for (int e = 0; e < n_edges && ok; e++) {
      if (!((mask >> edge_u[e]) & 1) || !((mask >> edge_v[e]) & 1)) continue;
      ok = keys[2 * e][pick[edge_u[e]]] == keys[2 * e + 1][pick[edge_v[e]]];
    }
    count += ok;
    size_t c = 0;
    while (c < ts.size() && ++idx[c] == n_rows[ts[c]]) idx[c++] = 0;
    if (c == ts.size()) break;
  }
  total = big_from_i128((i128)count);
  std::string s = big_to_dec(total);
  std::strncpy(out_dec, s.c_str(), 63);
  out_dec[63] = 0;
  *out_dbl = big_to_double(total);
  return 0;
}

/* ------------------------------------------------------------- learned combiner
 * Not in the paper (it takes the median over rows, Sec. 3.2).  A 2-layer perceptron
 * y = W2 relu(W1 x + b1) + b2, dims nin -> nh -> 1.  Parameters are kept in fp32
 * ("master") and rounded to bfloat16 (nearest even) for every forward and backward
 * pass; the oracle then evaluates in fp64 on those rounded values.
 * params layout (fp32): W1[nh][nin], b1[nh], W2[nh], b2[1]. */
int orc_bf16_round(int64_t n, const float* in, float* out) {
  for (int64_t i = 0; i < n; i++) out[i] = bf16_round(in[i]);
  return 0;
}

int orc_mlp_forward(int nin, int nh, int skip, const float* params, int64_t n, const float* x, double* y) {
  const float* W1 = params;
  const float* b1 = W1 + (size_t)nh * nin;
  const float* W2 = b1 + nh;
  const float* b2 = W2 + nh;
  for (int64_t r = 0; r < n; r++) {
    double acc = bf16_round(b2[0]);
    if (skip >= 0) acc += std::max(0.0, (double)x[r * nin + skip]);
    for (int h = 0; h < nh; h++) {
      double z = bf16_round(b1[h]);
      for (int c = 0; c < nin; c++) z += (double)bf16_round(W1[(size_t)h * nin + c]) * (double)x[r * nin + c];
      if (z > 0) acc += (double)bf16_round(W2[h]) * z;
    }
    y[r] = acc;
  }
  return 0;
}

/* loss = (1/n) sum (y - t)^2 and its gradient with respect to the bf16-rounded
 * parameters (applied to the fp32 master copy). grad has the params layout. */
/* loss_kind 0: mean of (y - t)^2.  loss_kind 1: mean Huber loss with threshold delta,
 * 0.5 e^2 for |e| <= delta and delta (|e| - 0.5 delta) beyond (L1-like tails, so the fit
 * follows the conditional median of the target rather than its mean). */
int orc_mlp_loss_grad(int nin, int nh, int skip, int loss_kind, double delta, const float* params, int64_t n,
                      const float* x, const float* t, double* loss, double* grad) {
  const float* W1 = params;
  const float* b1 = W1 + (size_t)nh * nin;
  const float* W2 = b1 + nh;
  const float* b2 = W2 + nh;
  const size_t np = (size_t)nh * nin + 2 * nh + 1;
  std::fill(grad, grad + np, 0.0);
  double* gW1 = grad;
  double* gb1 = gW1 + (size_t)nh * nin;
  double* gW2 = gb1 + nh;
  double* gb2 = gW2 + nh;
  std::vector<double> z(nh);
  double L = 0;
  for (int64_t r = 0; r < n; r++) {
    double y = bf16_round(b2[0]);
    if (skip >= 0) y += std::max(0.0, (double)x[r * nin + skip]);
    for (int h = 0; h < nh; h++) {
      double zz = bf16_round(b1[h]);
      for (int c = 0; c < nin; c++) zz += (double)bf16_round(W1[(size_t)h * nin + c]) * (double)x[r * nin + c];
      z[h] = zz;
      if (zz > 0) y += (double)bf16_round(W2[h]) * zz;
    }
    const double err = y - (double)t[r];
    double dy;
    if (loss_kind == 1) {
      const double a = std::fabs(err);
      L += a <= delta ? 0.5 * err * err : delta * (a - 0.5 * delta);
      dy = (a <= delta ? err : (err > 0 ? delta : -delta)) / (double)n;
    } else {
      L += err * err;
      dy = 2.0 * err / (double)n;
    }
    gb2[0] += dy;
    for (int h = 0; h < nh; h++) {
      if (z[h] <= 0) continue;
      gW2[h] += dy * z[h];
      const double dz = dy * (double)bf16_round(W2[h]);
      gb1[h] += dz;
      for (int c = 0; c < nin; c++) gW1[(size_t)h * nin + c] += dz * (double)x[r * nin + c];
    }
  }
  *loss = L / (double)n;
  return 0;
}

/* One Adam step (Kingma & Ba 2015) on the fp32 master parameters, in fp64. */
int orc_adam_step(int64_t np, float* params, double* m, double* v, const double* grad, double lr, double b1, double b2,
                  double eps, int step) {
  const double c1 = 1.0 - std::pow(b1, step), c2 = 1.0 - std::pow(b2, step);
  for (int64_t i = 0; i < np; i++) {
    m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
    v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
    const double mh = m[i] / c1, vh = v[i] / c2;
    params[i] = (float)((double)params[i] - lr * mh / (std::sqrt(vh) + eps));
  }
  return 0;
}

}  // extern "C"
