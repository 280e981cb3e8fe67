// CPU oracle for exact treewidth by breadth-first elimination-ordering DP.
//
// TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
// CUDA path is checked against.  Only the test suite, the smoke check and the
// CPU-baseline leg of the benchmark may load it; the product path never does.
// It shares no code, header or constant table with the CUDA library.
//
// What it computes (van der Zanden & Bodlaender, "Computing Treewidth on the
// GPU", arXiv 1709.09990):
//   * Section 2: for a set S of eliminated vertices and a vertex v outside S,
//     Q(S, v) is the set of vertices u outside S u {v} for which G has a path
//     from v to u whose inner vertices all belong to S; |Q(S, v)| is the
//     degree v has once S has been eliminated.  An ordering's width is the
//     largest such degree along it, and tw(G) is the smallest width.
//   * Section 3.1: the treewidth test at bound k keeps, for i = 0, 1, ...,
//     the family L_i of i-vertex sets that can be eliminated first without a
//     degree above k.  L_0 holds the empty set, and L_{i+1} is the family of
//     sets S u {v} with S in L_i, v outside S and |Q(S, v)| <= k.  Since any
//     k+1 vertices can be eliminated last in any order, tw <= k exactly when
//     L_{n-k-1} is not empty.  The treewidth is the first k that passes.
//
// Readings taken where the paper is silent or ambiguous:
//   R1  Q(S, v) never contains v itself (the definition speaks of paths to
//       other vertices; a path that returns to v is not one).
//   R2  The levels run i = 0 .. n-k-1; an empty level ends the run (every
//       later level would be empty too) and is the last one reported.
//   R3  k >= n-1 answers yes with the single level {empty set}.
//   R4  The families are exact sets (the paper's Bloom filter is lossy).
//
// One counter is not part of the paper's method: with COUNT_CANONICAL the
// run also counts the pairs (S, v) with |Q(S, v)| <= k whose v lies in the
// component of G[S u {v}] that holds the lowest vertex of S u {v}.  Those are
// the pairs the CUDA path submits to its duplicate-removal table; the count is
// computed here from that definition so the GPU's count can be checked.
//
// Independent pins (exercised by tests/test_oracle_*.py):
//   * brute force over all n! orderings with an explicit elimination game
//     (remove v, turn its neighbourhood into a clique; Section 2, second
//     paragraph) for n <= 10;
//   * a subset DP over all 2^n masks that tracks the eliminated graph
//     explicitly (fill-in edges) instead of path reachability, n <= 22.
//
// Layout of every adjacency argument: n rows of W = ceil(n/64) little-endian
// uint64 words; bit c of row r is set iff rc is an edge.  n <= 128.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <unordered_map>
#include <unordered_set>
#include <vector>

namespace {

constexpr int kMaxN = 128;

// A vertex set of at most 128 vertices (bit v of word v/64).
struct Key {
  uint64_t w[2];
  bool operator==(const Key& o) const { return w[0] == o.w[0] && w[1] == o.w[1]; }
};

// splitmix64 output function (Steele, Lea & Flood 2014), used as the set
// fingerprint and as the hash of the unordered containers.
uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Fingerprint of a vertex set: mix64(w0 ^ mix64(w1)).
uint64_t set_fingerprint(const Key& s) { return mix64(s.w[0] ^ mix64(s.w[1])); }

struct KeyHash {
  size_t operator()(const Key& k) const { return (size_t)set_fingerprint(k); }
};

const Key kNoVertex{{0, 0}};

bool has(const Key& s, int v) { return (s.w[v >> 6] >> (v & 63)) & 1ULL; }
Key with(Key s, int v) {
  s.w[v >> 6] |= 1ULL << (v & 63);
  return s;
}
Key without(Key s, int v) {
  s.w[v >> 6] &= ~(1ULL << (v & 63));
  return s;
}
Key set_union(const Key& a, const Key& b) { return Key{{a.w[0] | b.w[0], a.w[1] | b.w[1]}}; }
Key set_meet(const Key& a, const Key& b) { return Key{{a.w[0] & b.w[0], a.w[1] & b.w[1]}}; }
Key set_minus(const Key& a, const Key& b) { return Key{{a.w[0] & ~b.w[0], a.w[1] & ~b.w[1]}}; }
bool is_empty(const Key& s) { return (s.w[0] | s.w[1]) == 0; }

int popcount_key(const Key& s) { return __builtin_popcountll(s.w[0]) + __builtin_popcountll(s.w[1]); }

int lowest_vertex(const Key& s) { return s.w[0] ? __builtin_ctzll(s.w[0]) : 64 + __builtin_ctzll(s.w[1]); }

struct Graph {
  int n = 0;
  std::vector<std::vector<int>> nbr;        // adjacency lists, increasing order
  std::vector<std::vector<char>> mat;       // adjacency matrix
  std::vector<Key> nset;                    // N(v) as a vertex set
};

int words_for(int n) { return n <= 64 ? 1 : (n + 63) / 64; }

// Rebuilds the adjacency lists and neighbour sets from the matrix.
void derive_lists(Graph* g) {
  g->nbr.assign(g->n, {});
  g->nset.assign(g->n, kNoVertex);
  for (int r = 0; r < g->n; ++r)
    for (int c = 0; c < g->n; ++c)
      if (g->mat[r][c]) {
        g->nbr[r].push_back(c);
        g->nset[r] = with(g->nset[r], c);
      }
}

// Returns false on an invalid graph (asymmetric row, self-loop, bits >= n).
bool load_graph(const uint64_t* adj, int n, Graph* g) {
  if (n < 1 || n > kMaxN || adj == nullptr) return false;
  const int W = words_for(n);
  g->n = n;
  g->mat.assign(n, std::vector<char>(n, 0));
  for (int r = 0; r < n; ++r) {
    for (int c = 0; c < W * 64; ++c) {
      const bool bit = (adj[(size_t)r * W + (c >> 6)] >> (c & 63)) & 1ULL;
      if (!bit) continue;
      if (c >= n || c == r) return false;
      g->mat[r][c] = 1;
    }
  }
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c)
      if (g->mat[r][c] != g->mat[c][r]) return false;
  derive_lists(g);
  return true;
}

// The union of N(x) over the vertices x of X.
Key neighbours_of(const Graph& g, const Key& X) {
  Key out = kNoVertex;
  for (int x = 0; x < g.n; ++x)
    if (has(X, x)) out = set_union(out, g.nset[x]);
  return out;
}

// The vertices of `inside` that v reaches by a path whose vertices after v
// all lie in `inside`, collected by path length: the ones at distance 1,
// then those adjacent to a collected one, and so on until nothing is added.
Key reach_within(const Graph& g, const Key& inside, int v) {
  Key reached = set_meet(g.nset[v], inside);
  Key newest = reached;
  while (!is_empty(newest)) {
    newest = set_minus(set_meet(neighbours_of(g, newest), inside), reached);
    reached = set_union(reached, newest);
  }
  return reached;
}

// Q(S, v) of Section 2: a path from v to u with every inner vertex in S is
// v - x_1 - ... - x_m - u with x_1 .. x_m in S (m = 0 allowed), so u is a
// neighbour of v or of a vertex of S that v reaches through S.  Reading R1
// leaves v out; vertices of S are never in Q.
Key q_set(const Graph& g, const Key& S, int v) {
  const Key inner = reach_within(g, S, v);
  const Key ends = set_union(g.nset[v], neighbours_of(g, inner));
  return without(set_minus(ends, S), v);
}

int q_size(const Graph& g, const Key& S, int v) { return popcount_key(q_set(g, S, v)); }

// Whether v lies in the component of G[S u {v}] that contains the lowest
// vertex of S u {v}.
bool in_lowest_component(const Graph& g, const Key& S, int v) {
  const Key T = with(S, v);
  const int low = lowest_vertex(T);
  return low == v || has(reach_within(g, T, v), low);
}

struct DecideOut {
  int yes = 0;
  int levels = 0;
  std::vector<int64_t> level_size;
  std::vector<uint64_t> fp_sum, fp_xor;
  int64_t states_expanded = 0;
  int64_t candidates = 0;
  int64_t feasible = 0;
  int64_t canonical = 0;   // counted when asked (see the header)
  std::vector<int> order;  // filled when want_order and yes
};

int mmw_bound(const Graph& g, const Key& S, int stop_above);

// A level L_i: every set, mapped to one vertex v whose removal leaves a set
// of L_{i-1} from which it was obtained (-1 for the empty set).
using Level = std::unordered_map<Key, int, KeyHash>;

// What a run of the test may change (everything off is the plain method).
struct RunRule {
  const std::vector<char>* allowed = nullptr;  // only these vertices may join a set
  bool mmw_prune = false;                       // Section 3.3 bound on each set
  bool count_canonical = false;
};

// L_{i+1} from L_i (Section 3.1): every S u {v} with v outside S and
// |Q(S, v)| <= k, keeping for each new set the first v that produced it.
// Adds the counters of this step to *out.
Level grow_level(const Graph& g, int k, const Level& Li, const RunRule& rule, DecideOut* out) {
  Level next;
  for (const auto& entry : Li) {
    const Key& S = entry.first;
    std::vector<int> outside;
    for (int v = 0; v < g.n; ++v)
      if (!has(S, v) && (!rule.allowed || (*rule.allowed)[v])) outside.push_back(v);
    out->candidates += (int64_t)outside.size();
    if (rule.mmw_prune && mmw_bound(g, S, k) > k) continue;
    for (int v : outside) {
      if (q_size(g, S, v) > k) continue;
      ++out->feasible;
      if (rule.count_canonical && in_lowest_component(g, S, v)) ++out->canonical;
      next.emplace(with(S, v), v);  // keeps the first producer
    }
  }
  out->states_expanded += (int64_t)Li.size();
  return next;
}

// The test at bound k with exact sets (reading R4).  With max_level >= 0 the
// run stops after building level max_level (the first levels of a run too
// large to finish here; yes is then not decided).  When keep is given it
// receives every level built (level 0 first).
void decide(const Graph& g, int k, bool want_order, DecideOut* out, const std::vector<char>* allowed = nullptr,
            bool mmw_prune = false, bool count_canonical = false, int max_level = -1,
            std::vector<Level>* keep = nullptr) {
  const int n = g.n;
  out->level_size.assign(n + 1, 0);
  out->fp_sum.assign(n + 1, 0);
  out->fp_xor.assign(n + 1, 0);
  out->order.clear();
  RunRule rule;
  rule.allowed = allowed;
  rule.mmw_prune = mmw_prune;
  rule.count_canonical = count_canonical;

  std::vector<Level> L(1);
  L[0].emplace(kNoVertex, -1);
  auto record = [&](int i) {
    uint64_t s = 0, x = 0;
    for (const auto& e : L[i]) {
      const uint64_t f = set_fingerprint(e.first);
      s += f;
      x ^= f;
    }
    out->level_size[i] = (int64_t)L[i].size();
    out->fp_sum[i] = s;
    out->fp_xor[i] = x;
  };
  record(0);
  const int top = n - k - 1;  // the level whose non-emptiness answers yes
  const int stop = max_level >= 0 ? std::min(top, max_level) : top;
  while ((int)L.size() - 1 < stop && !L.back().empty()) {
    Level next = grow_level(g, k, L.back(), rule, out);
    if (!want_order && !keep) L.back().clear();  // only the newest level is still needed
    L.push_back(std::move(next));
    record((int)L.size() - 1);
  }
  const int last = (int)L.size() - 1;
  out->levels = last + 1;
  out->yes = L[last].empty() ? 0 : 1;

  if (want_order && out->yes) {
    // From any set of the last level, drop the recorded producers one level
    // at a time; they are the first vertices of the ordering, in reverse.
    Key S = L[last].begin()->first;
    const Key final_set = S;
    std::vector<int> first(last, -1);
    for (int j = last; j >= 1; --j) {
      const int v = L[j].at(S);
      first[j - 1] = v;
      S = without(S, v);
    }
    out->order = first;
    for (int v = 0; v < n; ++v)
      if (!has(final_set, v)) out->order.push_back(v);
  }
  if (keep) *keep = std::move(L);
}

// Width of an ordering through Q (Section 2's definition).
int width_by_q(const Graph& g, const int* order) {
  const int n = g.n;
  std::vector<char> seen(n, 0);
  for (int j = 0; j < n; ++j) {
    if (order[j] < 0 || order[j] >= n || seen[order[j]]) return -1;
    seen[order[j]] = 1;
  }
  Key prefix{{0, 0}};
  int width = 0;
  for (int j = 0; j < n; ++j) {
    const int v = order[j];
    width = std::max(width, q_size(g, prefix, v));
    prefix = with(prefix, v);
  }
  return width;
}

// Width of an ordering by the explicit elimination game: remove v, turn its
// remaining neighbourhood into a clique (Section 2, second paragraph).
int width_by_elimination(const Graph& g, const int* order) {
  const int n = g.n;
  std::vector<std::vector<char>> m = g.mat;
  std::vector<char> gone(n, 0);
  int width = 0;
  for (int j = 0; j < n; ++j) {
    const int v = order[j];
    if (v < 0 || v >= n || gone[v]) return -1;
    std::vector<int> nb;
    for (int u = 0; u < n; ++u)
      if (!gone[u] && u != v && m[v][u]) nb.push_back(u);
    width = std::max(width, (int)nb.size());
    for (int a : nb)
      for (int b : nb)
        if (a != b) m[a][b] = 1;
    gone[v] = 1;
  }
  return width;
}

}  // namespace

extern "C" {

int orc_max_n() { return kMaxN; }

uint64_t orc_set_fingerprint(uint64_t w0, uint64_t w1) { return set_fingerprint(Key{{w0, w1}}); }

// Validates an adjacency: 1 if it is a simple undirected graph, else 0.
int orc_valid_graph(const uint64_t* adj, int n) {
  Graph g;
  return load_graph(adj, n, &g) ? 1 : 0;
}

// |Q(S, v)| (Section 2).  S is given as two words.
int orc_q_size(const uint64_t* adj, int n, uint64_t s0, uint64_t s1, int v) {
  Graph g;
  if (!load_graph(adj, n, &g) || v < 0 || v >= n) return -1;
  return q_size(g, Key{{s0, s1}}, v);
}

// Q(S, v) as two words.
int orc_q_set(const uint64_t* adj, int n, uint64_t s0, uint64_t s1, int v, uint64_t* q_out) {
  Graph g;
  if (!load_graph(adj, n, &g) || v < 0 || v >= n) return -1;
  const Key q = q_set(g, Key{{s0, s1}}, v);
  q_out[0] = q.w[0];
  q_out[1] = q.w[1];
  return 0;
}

// One run of the Section 3.1 test (Listing 1) at bound k.  Arrays level_size / fp_sum / fp_xor have
// n+1 entries (entries past the last level are zero).  counters[0..2] =
// states expanded, candidates, feasible candidates.  order (n entries, or
// NULL) receives an elimination ordering of width <= k when the answer is
// yes.  Returns 1 (yes), 0 (no) or -1 (invalid input).
int orc_decide(const uint64_t* adj, int n, int k, int64_t* level_size, uint64_t* fp_sum,
               uint64_t* fp_xor, int* levels, int64_t* counters, int32_t* order) {
  Graph g;
  if (!load_graph(adj, n, &g) || k < 0) return -1;
  DecideOut out;
  decide(g, k, order != nullptr, &out);
  for (int i = 0; i <= n; ++i) {
    if (level_size) level_size[i] = out.level_size[i];
    if (fp_sum) fp_sum[i] = out.fp_sum[i];
    if (fp_xor) fp_xor[i] = out.fp_xor[i];
  }
  if (levels) *levels = out.levels;
  if (counters) {
    counters[0] = out.states_expanded;
    counters[1] = out.candidates;
    counters[2] = out.feasible;
  }
  if (order && out.yes)
    for (int j = 0; j < n; ++j) order[j] = out.order[j];
  return out.yes;
}

// Iterative deepening (Section 3.1) from k_start upward; the first
// yes is the treewidth.  counters[0..2] are summed over every k tried;
// counters[3] = number of k tried.  Returns tw or -1.
int orc_solve(const uint64_t* adj, int n, int k_start, int32_t* order, int64_t* counters) {
  Graph g;
  if (!load_graph(adj, n, &g) || k_start < 0) return -1;
  int64_t tot[4] = {0, 0, 0, 0};
  for (int k = k_start; k < n; ++k) {
    DecideOut out;
    decide(g, k, order != nullptr, &out);
    tot[0] += out.states_expanded;
    tot[1] += out.candidates;
    tot[2] += out.feasible;
    tot[3] += 1;
    if (out.yes) {
      if (order)
        for (int j = 0; j < n; ++j) order[j] = out.order[j];
      if (counters) std::memcpy(counters, tot, sizeof(tot));
      return k;
    }
  }
  return -1;  // unreachable for a valid graph: k = n-1 always answers yes
}

// Width of an ordering via Q; -1 if order is not a permutation of 0..n-1.
int orc_width_q(const uint64_t* adj, int n, const int32_t* order) {
  Graph g;
  if (!load_graph(adj, n, &g)) return -1;
  std::vector<int> o(order, order + n);
  return width_by_q(g, o.data());
}

// Width of an ordering via the elimination game.
int orc_width_elim(const uint64_t* adj, int n, const int32_t* order) {
  Graph g;
  if (!load_graph(adj, n, &g)) return -1;
  std::vector<int> o(order, order + n);
  return width_by_elimination(g, o.data());
}

// Brute force over all n! orderings (elimination game), n <= 10.
int orc_brute_force_tw(const uint64_t* adj, int n) {
  Graph g;
  if (!load_graph(adj, n, &g) || n > 10) return -1;
  std::vector<int> perm(n);
  for (int i = 0; i < n; ++i) perm[i] = i;
  int best = n;
  do {
    best = std::min(best, width_by_elimination(g, perm.data()));
  } while (std::next_permutation(perm.begin(), perm.end()));
  return best;
}

// Subset DP over all 2^n vertex masks, n <= 22, independent of the search
// above: it keeps, for every feasible mask S, the graph that remains after
// eliminating S (adjacency rows over V \ S with fill-in edges), built by
// eliminating one vertex at a time.  feasible[S u {v}] holds iff S is feasible
// and v has degree <= k in that graph.  Reports the sizes and fingerprints of
// the levels 0 .. n-k-1 with the same truncation at the first empty level.
// Returns 1/0 (yes/no) or -1.
int orc_subset_dp(const uint64_t* adj, int n, int k, int64_t* level_size, uint64_t* fp_sum,
                  uint64_t* fp_xor, int* levels) {
  Graph g;
  if (!load_graph(adj, n, &g) || n > 22 || k < 0) return -1;
  const uint32_t full = (n == 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
  const size_t masks = (size_t)1 << n;
  std::vector<uint8_t> feasible(masks, 0);
  // rows[mask * n + u] = neighbours of u in the graph after eliminating mask.
  std::vector<uint32_t> rows(masks * (size_t)n, 0);
  std::vector<uint8_t> built(masks, 0);
  for (int u = 0; u < n; ++u) {
    uint32_t r = 0;
    for (int v : g.nbr[u]) r |= 1u << v;
    rows[u] = r;
  }
  built[0] = 1;
  feasible[0] = 1;
  const int top_level = std::max(0, n - k - 1);
  for (size_t m = 0; m < masks; ++m) {
    if (!feasible[m]) continue;
    const int pc = __builtin_popcount((uint32_t)m);
    if (pc >= top_level) continue;
    const uint32_t* R = &rows[m * n];
    for (int v = 0; v < n; ++v) {
      if ((m >> v) & 1u) continue;
      const int deg = __builtin_popcount(R[v]);
      if (deg > k) continue;
      const size_t m2 = m | ((size_t)1 << v);
      feasible[m2] = 1;
      if (!built[m2]) {
        // Eliminate v from the graph of m: its neighbourhood becomes a clique.
        uint32_t* R2 = &rows[m2 * n];
        const uint32_t nb = R[v];
        for (int u = 0; u < n; ++u) {
          if ((m2 >> u) & 1u) {
            R2[u] = 0;
            continue;
          }
          uint32_t r = R[u] & ~(1u << v);
          if ((nb >> u) & 1u) r |= nb & ~(1u << u);
          R2[u] = r & full;
        }
        built[m2] = 1;
      }
    }
  }
  std::vector<int64_t> cnt(n + 1, 0);
  std::vector<uint64_t> fs(n + 1, 0), fx(n + 1, 0);
  for (size_t m = 0; m < masks; ++m) {
    if (!feasible[m]) continue;
    const int pc = __builtin_popcount((uint32_t)m);
    if (pc > top_level) continue;
    cnt[pc] += 1;
    const uint64_t f = set_fingerprint(Key{{(uint64_t)m, 0}});
    fs[pc] += f;
    fx[pc] ^= f;
  }
  int last = 0;
  while (last < top_level && cnt[last + 1] > 0) ++last;
  if (last < top_level) ++last;  // include the first empty level
  for (int i = 0; i <= n; ++i) {
    const bool in = i <= last;
    if (level_size) level_size[i] = in ? cnt[i] : 0;
    if (fp_sum) fp_sum[i] = in ? fs[i] : 0;
    if (fp_xor) fp_xor[i] = in ? fx[i] : 0;
  }
  if (levels) *levels = last + 1;
  return cnt[top_level] > 0 ? 1 : 0;
}

// Tree decomposition from an ordering: bag(v) = {v} u Q(prefix(v), v);
// parent(v) = the vertex of Q(prefix(v), v) that comes first in the order
// after v; a vertex with empty Q hangs below the last vertex of the order,
// which is the root (parent -1).  bags: n rows of W words.  Returns the width.
int orc_td_from_order(const uint64_t* adj, int n, const int32_t* order, int32_t* parent,
                      uint64_t* bags) {
  Graph g;
  if (!load_graph(adj, n, &g)) return -1;
  const int W = words_for(n);
  std::vector<int> pos(n, -1);
  for (int j = 0; j < n; ++j) {
    if (order[j] < 0 || order[j] >= n || pos[order[j]] >= 0) return -1;
    pos[order[j]] = j;
  }
  Key prefix{{0, 0}};
  int width = 0;
  for (int j = 0; j < n; ++j) {
    const int v = order[j];
    const Key q = q_set(g, prefix, v);
    const Key bag = with(q, v);
    for (int w = 0; w < W; ++w) bags[(size_t)v * W + w] = bag.w[w];
    width = std::max(width, popcount_key(bag) - 1);
    int best = -1;
    for (int u = 0; u < n; ++u)
      if (has(q, u) && (best < 0 || pos[u] < pos[best])) best = u;
    if (best < 0) best = (j == n - 1) ? -1 : order[n - 1];
    parent[v] = best;
    prefix = with(prefix, v);
  }
  return width;
}

// Checks a tree decomposition given as one bag per vertex plus parent
// pointers: the parent pointers form a single rooted tree, every vertex lies
// in a bag, every edge lies in a bag, and for every vertex x the bags holding
// x are connected in the tree.  Returns the width, or -1 if any check fails.
int orc_verify_td(const uint64_t* adj, int n, const int32_t* parent, const uint64_t* bags) {
  Graph g;
  if (!load_graph(adj, n, &g)) return -1;
  const int W = words_for(n);
  auto in_bag = [&](int b, int x) { return (bags[(size_t)b * W + (x >> 6)] >> (x & 63)) & 1ULL; };
  int roots = 0;
  for (int b = 0; b < n; ++b) {
    if (parent[b] == -1)
      ++roots;
    else if (parent[b] < 0 || parent[b] >= n || parent[b] == b)
      return -1;
  }
  if (roots != 1) return -1;
  // Acyclic: every node reaches the root within n steps.
  for (int b = 0; b < n; ++b) {
    int c = b, steps = 0;
    while (parent[c] != -1) {
      c = parent[c];
      if (++steps > n) return -1;
    }
  }
  for (int x = 0; x < n; ++x) {
    bool found = false;
    for (int b = 0; b < n && !found; ++b) found = in_bag(b, x);
    if (!found) return -1;
  }
  for (int u = 0; u < n; ++u)
    for (int v : g.nbr[u]) {
      bool found = false;
      for (int b = 0; b < n && !found; ++b) found = in_bag(b, u) && in_bag(b, v);
      if (!found) return -1;
    }
  // Running intersection: among the bags holding x exactly one has a parent
  // that does not hold x (or is the root).
  for (int x = 0; x < n; ++x) {
    int tops = 0;
    for (int b = 0; b < n; ++b) {
      if (!in_bag(b, x)) continue;
      if (parent[b] == -1 || !in_bag(parent[b], x)) ++tops;
    }
    if (tops != 1) return -1;
  }
  int width = 0;
  for (int b = 0; b < n; ++b) {
    int c = 0;
    for (int x = 0; x < n; ++x) c += in_bag(b, x) ? 1 : 0;
    width = std::max(width, c - 1);
  }
  return width;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The first two optimisations of Section 3.1 (opt-in; they change the sets
// explored but not the answer):
//  * clique skip: a maximum clique C can be eliminated last, so vertices of C
//    are never added to a set; a clique with more than k+1 vertices answers
//    no at once.  C is the maximum clique whose sorted vertex list is
//    lexicographically smallest.
//  * disjoint paths: for decide(k), every non-adjacent pair u, v joined by at
//    least k+1 internally vertex-disjoint paths in G gets the edge uv.
namespace {

// Exhaustive search over vertices in increasing order, trying "take v"
// before "skip v"; a clique replaces the best one only when it is strictly
// larger, so the first maximum clique found is the lexicographically smallest.
void clique_search(const Graph& g, std::vector<int>& cur, int next, std::vector<int>& best) {
  const int n = g.n;
  int possible = (int)cur.size();
  for (int v = next; v < n; ++v) {
    bool ok = true;
    for (int u : cur) ok = ok && g.mat[u][v];
    if (ok) ++possible;
  }
  if (possible <= (int)best.size()) return;
  if ((int)cur.size() > (int)best.size()) best = cur;
  for (int v = next; v < n; ++v) {
    bool ok = true;
    for (int u : cur) ok = ok && g.mat[u][v];
    if (!ok) continue;
    cur.push_back(v);
    clique_search(g, cur, v + 1, best);
    cur.pop_back();
  }
}

// Minor-min-width of the graph H that remains after eliminating S
// (Section 3.3), with the second-smallest degree as the bound of each step:
// H has the vertices outside S and an edge uw iff w is in Q(S, u).  While H
// has at least two vertices: take a minimum-degree vertex v (lowest index),
// record the second-smallest degree of H, delete v if it is isolated, else
// contract v into its minimum-degree neighbour (lowest index).  Returns the
// largest recorded degree (callers only compare it with stop_above, so the
// search may stop once it exceeds that).
int mmw_bound(const Graph& g, const Key& S, int stop_above) {
  const int n = g.n;
  std::vector<std::vector<char>> h(n, std::vector<char>(n, 0));
  std::vector<char> alive(n, 0);
  for (int u = 0; u < n; ++u) {
    if (has(S, u)) continue;
    alive[u] = 1;
    const Key q = q_set(g, S, u);
    for (int w = 0; w < n; ++w)
      if (has(q, w)) h[u][w] = 1;
  }
  int lb = 0;
  for (;;) {
    std::vector<int> deg(n, -1);
    int count = 0;
    for (int u = 0; u < n; ++u) {
      if (!alive[u]) continue;
      ++count;
      int d = 0;
      for (int w = 0; w < n; ++w) d += (alive[w] && h[u][w]) ? 1 : 0;
      deg[u] = d;
    }
    if (count < 2) break;
    int v = -1;
    for (int u = 0; u < n; ++u)
      if (alive[u] && (v < 0 || deg[u] < deg[v])) v = u;
    int second = -1;
    for (int u = 0; u < n; ++u)
      if (alive[u] && u != v && (second < 0 || deg[u] < second)) second = deg[u];
    lb = std::max(lb, second);
    if (lb > stop_above) return lb;
    if (deg[v] == 0) {
      alive[v] = 0;
      continue;
    }
    int into = -1;
    for (int u = 0; u < n; ++u)
      if (alive[u] && h[v][u] && (into < 0 || deg[u] < deg[into])) into = u;
    for (int w = 0; w < n; ++w)
      if (alive[w] && h[v][w] && w != into) h[into][w] = h[w][into] = 1;
    alive[v] = 0;
  }
  return lb;
}

std::vector<int> first_max_clique(const Graph& g) {
  std::vector<int> cur, best;
  clique_search(g, cur, 0, best);
  return best;
}

// Number of internally vertex-disjoint u-v paths, counted up to limit:
// augmenting paths (depth-first) in the graph with every vertex other than
// u and v split into an in- and an out-node joined by a unit arc.
int disjoint_paths(const Graph& g, int u, int v, int limit) {
  const int n = g.n;
  const int N = 2 * n;  // node x_in = 2x, x_out = 2x+1
  std::vector<std::vector<int>> cap(N, std::vector<int>(N, 0));
  for (int x = 0; x < n; ++x) cap[2 * x][2 * x + 1] = (x == u || x == v) ? (1 << 20) : 1;
  for (int a = 0; a < n; ++a)
    for (int b : g.nbr[a]) cap[2 * a + 1][2 * b] = 1 << 20;
  const int src = 2 * u + 1, dst = 2 * v;
  int flow = 0;
  while (flow < limit) {
    std::vector<int> prev(N, -1);
    std::vector<int> stack{src};
    prev[src] = src;
    while (!stack.empty() && prev[dst] < 0) {
      const int x = stack.back();
      stack.pop_back();
      for (int y = 0; y < N; ++y)
        if (cap[x][y] > 0 && prev[y] < 0) {
          prev[y] = x;
          stack.push_back(y);
        }
    }
    if (prev[dst] < 0) break;
    for (int y = dst; y != src; y = prev[y]) {
      cap[prev[y]][y] -= 1;
      cap[y][prev[y]] += 1;
    }
    ++flow;
  }
  return flow;
}

}  // namespace

extern "C" {

// The minor-min-width bound of the graph left after eliminating S.
int orc_mmw_bound(const uint64_t* adj, int n, uint64_t s0, uint64_t s1) {
  Graph g;
  if (!load_graph(adj, n, &g)) return -1;
  return mmw_bound(g, Key{{s0, s1}}, n);
}

// The clique of the clique-skip option: writes its vertices (sorted) and
// returns its size.
int orc_max_clique(const uint64_t* adj, int n, int32_t* out) {
  Graph g;
  if (!load_graph(adj, n, &g)) return -1;
  const std::vector<int> c = first_max_clique(g);
  for (size_t i = 0; i < c.size(); ++i) out[i] = c[i];
  return (int)c.size();
}

// Internally vertex-disjoint u-v paths, counted up to limit.
int orc_disjoint_paths(const uint64_t* adj, int n, int u, int v, int limit) {
  Graph g;
  if (!load_graph(adj, n, &g) || u == v || u < 0 || v < 0 || u >= n || v >= n) return -1;
  return disjoint_paths(g, u, v, limit);
}

// The first levels 0 .. max_level of orc_decide (with count_canonical, the
// canonical pairs are counted into counters[3]); for runs too large to
// finish.  Returns the number of levels built, or -1 for invalid input.
int orc_decide_prefix(const uint64_t* adj, int n, int k, int max_level, int64_t* level_size, uint64_t* fp_sum,
                      uint64_t* fp_xor, int64_t* counters, int count_canonical) {
  Graph g;
  if (!load_graph(adj, n, &g) || k < 0 || max_level < 0) return -1;
  DecideOut out;
  decide(g, k, false, &out, nullptr, false, count_canonical != 0, max_level);
  for (int i = 0; i <= n; ++i) {
    if (level_size) level_size[i] = out.level_size[i];
    if (fp_sum) fp_sum[i] = out.fp_sum[i];
    if (fp_xor) fp_xor[i] = out.fp_xor[i];
  }
  if (counters) {
    counters[0] = out.states_expanded;
    counters[1] = out.candidates;
    counters[2] = out.feasible;
    counters[3] = out.canonical;
  }
  return out.levels;
}

// The sets of level `level` of the run at bound k (the run stops after that
// level; a level past the end of the run is empty).  Writes up to cap sets,
// each as W = ceil(n/64) words, in no particular order, and returns the
// level's size, or -1 for invalid input.
int64_t orc_level_keys(const uint64_t* adj, int n, int k, int level, uint64_t* keys, int64_t cap) {
  Graph g;
  if (!load_graph(adj, n, &g) || k < 0 || level < 0) return -1;
  DecideOut out;
  std::vector<Level> L;
  decide(g, k, false, &out, nullptr, false, false, level, &L);
  if (level >= (int)L.size()) return 0;
  const int W = words_for(n);
  int64_t j = 0;
  for (const auto& e : L[level]) {
    if (j < cap)
      for (int w = 0; w < W; ++w) keys[j * W + w] = e.first.w[w];
    ++j;
  }
  return j;
}

// orc_decide with the options of Sections 3.1 and 3.3: bit 0 of opts =
// clique skip, bit 1 = disjoint-path edges, bit 2 = minor-min-width pruning
// (on the graph with the added edges).  Same outputs as orc_decide; with the
// clique skip, candidates count only vertices outside C.  Bit 3 counts the
// canonical pairs (see the header) into counters[3], which must then exist.
int orc_decide_opts(const uint64_t* adj, int n, int k, int opts, int64_t* level_size, uint64_t* fp_sum,
                    uint64_t* fp_xor, int* levels, int64_t* counters, int32_t* order) {
  Graph g0;
  if (!load_graph(adj, n, &g0) || k < 0) return -1;
  Graph g = g0;
  if (opts & 2) {
    for (int u = 0; u < n; ++u)
      for (int v = u + 1; v < n; ++v)
        if (!g0.mat[u][v] && disjoint_paths(g0, u, v, k + 1) >= k + 1) g.mat[u][v] = g.mat[v][u] = 1;
    derive_lists(&g);
  }
  DecideOut out;
  std::vector<char> allowed(n, 1);
  const std::vector<char>* filter = nullptr;
  bool immediate_no = false;
  if (opts & 1) {
    const std::vector<int> c = first_max_clique(g0);
    for (int v : c) allowed[v] = 0;
    filter = &allowed;
    immediate_no = (int)c.size() > k + 1;  // tw >= |C| - 1 > k
  }
  if (immediate_no) {
    out.level_size.assign(n + 1, 0);
    out.fp_sum.assign(n + 1, 0);
    out.fp_xor.assign(n + 1, 0);
    out.level_size[0] = 1;
    out.levels = 1;
    out.yes = 0;
  } else {
    decide(g, k, order != nullptr, &out, filter, (opts & 4) != 0, (opts & 8) != 0);
  }
  for (int i = 0; i <= n; ++i) {
    if (level_size) level_size[i] = out.level_size[i];
    if (fp_sum) fp_sum[i] = out.fp_sum[i];
    if (fp_xor) fp_xor[i] = out.fp_xor[i];
  }
  if (levels) *levels = out.levels;
  if (counters) {
    counters[0] = out.states_expanded;
    counters[1] = out.candidates;
    counters[2] = out.feasible;
    if (opts & 8) counters[3] = out.canonical;
  }
  if (order && out.yes)
    for (int j = 0; j < n; ++j) order[j] = out.order[j];
  return out.yes;
}

}  // extern "C"
