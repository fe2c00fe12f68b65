// Oracle: a plain, slow, obviously correct CPU restatement of exact
// hyper-triangle counting (Yin et al., "Efficient Computation of
// Hyper-triangles on Hypergraphs", PVLDB 18(3)).
//
// TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
// this file: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg
// use it.  It shares no code, table or header with the CUDA library.
//
// What it computes (all exact integers):
//   * per-pattern hyper-triangle counts H[1..20] and the total T (Def. 2.4);
//   * hyperwedge statistics: W = |wedges|, W_t (intersection type), W_c
//     (inclusion type) (Def. 2.2, Def. 2.3);
//   * connected triples sum_i C(|N(e_i)|, 2) and open hyper-triangles (Def. 5.1);
//   * the same histogram split by owner, the member of each hyper-triangle ranked
//     lowest in the order (|N(e)|, id) (oracle_count_owned).
//
// Two enumerations:
//   * mode 0 follows Exact-bs (Algorithm 1): build the projection graph
//     N(e_i) = { e_j : e_i and e_j share a vertex } (Sec. 2), then for every
//     e_i and every pair {e_j, e_k} of its neighbours with i < min(j, k), test
//     e_j and e_k for a common vertex and classify the triple.  Only the pairs
//     with j, k > i are visited, which is the same set Algorithm 1 keeps after
//     its i < min{j,k} test.
//   * mode 1 is brute force over all C(|E|, 3) triples (tiny inputs only).
//
// Classification (Def. 2.4): a triple {e_i, e_j, e_k} has seven Venn regions
//   (a) e_i only  (b) e_j only  (c) e_k only  (d) e_i and e_j, not e_k
//   (e) e_j and e_k, not e_i  (f) e_k and e_i, not e_j  (g) all three.
// The pattern is decided by which regions are non-empty, up to relabelling
// the three hyperedges.  The paper's pattern figure is not available, so the
// numbering below is a reading of the text: pattern 1 is the CCC class, 2-5
// TCC, 6-8 TTC, 9-20 TTT (Sec. 2), 9-16 have region (g) non-empty and 17-20
// have it empty (Sec. 3.2).  Inside each class the numbers are fixed by the
// O(1) rules of Algorithm 5 (patterns 1-8) and by the case study of Sec. 6.2
// (co-authorship triangles of patterns 10 and 12, e-mail triangles of
// pattern 5); the order of 9, 11 and 13-20 is parity unpinned (the paper
// shows them only in a figure): ascending number of non-empty pairwise
// regions (d, e, f), then ascending number of non-empty single regions.
#include <algorithm>
#include <array>
#include <cmath>
#include <chrono>
#include <cstdint>
#include <cstring>
#include <set>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// Region letters of each pattern in one labelling of (e_i, e_j, e_k).
const char* const kPatternRegions[20] = {
    "adg",      // 1  CCC: chain e_k inside e_j inside e_i
    "abg",      // 2  TCC: e_k equal to e_i cap e_j
    "abdg",     // 3  TCC: e_k strictly inside e_i cap e_j
    "deg",      // 4  TCC: e_j equal to e_i cup e_k
    "bdeg",     // 5  TCC: e_j strictly contains e_i cup e_k
    "acdg",     // 6  TTC
    "adeg",     // 7  TTC
    "abdeg",    // 8  TTC
    "abcg",     // 9  DenseTTT
    "abcdg",    // 10 DenseTTT
    "acdeg",    // 11 DenseTTT
    "abcdeg",   // 12 DenseTTT
    "defg",     // 13 DenseTTT
    "adefg",    // 14 DenseTTT
    "abdefg",   // 15 DenseTTT
    "abcdefg",  // 16 DenseTTT
    "def",      // 17 SparseTTT
    "adef",     // 18 SparseTTT
    "abdef",    // 19 SparseTTT
    "abcdef",   // 20 SparseTTT
};

// Which of the three sets (i, j, k) contain each region a..g.
const int kRegionIn[7][3] = {
    {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {0, 1, 1}, {1, 0, 1}, {1, 1, 1}};

int region_of(int in_i, int in_j, int in_k) {
  for (int r = 0; r < 7; ++r)
    if (kRegionIn[r][0] == in_i && kRegionIn[r][1] == in_j && kRegionIn[r][2] == in_k) return r;
  return -1;
}

// Relabel a region bit mask: set number s of the new labelling is set perm[s] of the old.
int relabel(int mask, const int perm[3]) {
  int out = 0;
  for (int r = 0; r < 7; ++r) {
    if (!(mask >> r & 1)) continue;
    int in_new[3];
    for (int s = 0; s < 3; ++s) in_new[s] = kRegionIn[r][perm[s]];
    out |= 1 << region_of(in_new[0], in_new[1], in_new[2]);
  }
  return out;
}

// mask -> pattern number (0 = not a pattern), built once from kPatternRegions
struct PatternMap {
  int of_mask[128];
  int conflict;
  PatternMap() : conflict(0) {
    std::memset(of_mask, 0, sizeof(of_mask));
    const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int p = 0; p < 20; ++p) {
      int m = 0;
      for (const char* c = kPatternRegions[p]; *c; ++c) m |= 1 << (*c - 'a');
      for (const auto& pr : perms) {
        int lm = relabel(m, pr);
        if (of_mask[lm] != 0 && of_mask[lm] != p + 1) conflict = 1;
        of_mask[lm] = p + 1;
      }
    }
  }
};
const PatternMap& pattern_map() {
  static PatternMap pm;
  return pm;
}

// Canonical form of a labelled region mask: the smallest mask value over the six
// relabellings of the three hyperedges.  Two hyper-triangles get the same canonical
// mask exactly when their sets of non-empty regions agree up to relabelling, which is
// what a pattern is (Sec. 2); the histogram over canonical masks therefore does not
// depend on how the twenty patterns are numbered.
struct CanonMap {
  int of_mask[128];
  CanonMap() {
    const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int m = 0; m < 128; ++m) {
      int best = m;
      for (const auto& pr : perms) best = std::min(best, relabel(m, pr));
      of_mask[m] = best;
    }
  }
};
const CanonMap& canon_map() {
  static CanonMap cm;
  return cm;
}

using VSet = std::set<int32_t>;

// Seven-region non-emptiness mask of (A, B, C), written from the definitions.
int region_mask(const VSet& A, const VSet& B, const VSet& C) {
  int mask = 0;
  for (int32_t x : A) mask |= 1 << region_of(1, B.count(x) ? 1 : 0, C.count(x) ? 1 : 0);
  for (int32_t x : B)
    if (!A.count(x)) mask |= 1 << region_of(0, 1, C.count(x) ? 1 : 0);
  for (int32_t x : C)
    if (!A.count(x) && !B.count(x)) mask |= 1 << region_of(0, 0, 1);
  return mask;
}

bool intersects(const VSet& A, const VSet& B) {
  for (int32_t x : A)
    if (B.count(x)) return true;
  return false;
}

size_t common(const VSet& A, const VSet& B) {
  size_t n = 0;
  for (int32_t x : A) n += B.count(x);
  return n;
}

struct Graph {
  int32_t nv = 0, ne = 0;
  std::vector<VSet> e;                      // hyperedge vertex sets
  std::vector<std::vector<int32_t>> Ev;     // E_v: hyperedges containing v, ascending
};

int load(Graph& g, int32_t nv, int32_t ne, const int64_t* e_ptr, const int32_t* e_idx) {
  g.nv = nv;
  g.ne = ne;
  g.e.assign(ne, VSet());
  g.Ev.assign(nv, {});
  for (int32_t i = 0; i < ne; ++i) {
    if (e_ptr[i + 1] <= e_ptr[i]) return -2;                  // empty hyperedge
    for (int64_t p = e_ptr[i]; p < e_ptr[i + 1]; ++p) {
      int32_t v = e_idx[p];
      if (v < 0 || v >= nv) return -3;
      if (!g.e[i].insert(v).second) return -4;                 // repeated vertex
      g.Ev[v].push_back(i);
    }
  }
  return 0;
}

// N(e_i) as an ascending vector, from the union of E_v over v in e_i.
std::vector<int32_t> neighbours(const Graph& g, int32_t i) {
  std::set<int32_t> n;
  for (int32_t v : g.e[i])
    for (int32_t j : g.Ev[v])
      if (j != i) n.insert(j);
  return std::vector<int32_t>(n.begin(), n.end());
}

bool adjacent(const std::vector<std::vector<int32_t>>& N, int32_t j, int32_t k) {
  return std::binary_search(N[j].begin(), N[j].end(), k);
}

}  // namespace

extern "C" {

// stats layout
enum { ST_W = 0, ST_WT, ST_WC, ST_CONNECTED, ST_OPEN, ST_MAXDEG, ST_T, ST_DUP, ST_N };

int oracle_pattern_table_ok() { return pattern_map().conflict ? 0 : 1; }

// Pattern number (1..20) of one labelled region mask; 0 if none.
int oracle_pattern_of_mask(int mask) {
  if (mask < 0 || mask > 127) return 0;
  return pattern_map().of_mask[mask];
}

// Region mask of three explicit vertex lists.
int oracle_region_mask(const int32_t* a, int na, const int32_t* b, int nb, const int32_t* c,
                       int nc) {
  VSet A(a, a + na), B(b, b + nb), C(c, c + nc);
  return region_mask(A, B, C);
}

// Line-graph degrees |N(e_i)| (Sec. 2: the hyperedges sharing a vertex with e_i) into
// deg[ne].  Returns 0 or a negative input error as oracle_count.
int oracle_degrees(int32_t nv, int32_t ne, const int64_t* e_ptr, const int32_t* e_idx,
                   int32_t* deg) {
  if (!deg || nv < 0 || ne < 0) return -6;
  Graph g;
  int rc = load(g, nv, ne, e_ptr, e_idx);
  if (rc) return rc;
#pragma omp parallel for schedule(dynamic, 256)
  for (int32_t i = 0; i < ne; ++i) deg[i] = (int32_t)neighbours(g, i).size();
  return 0;
}

// Canonical form (smallest over the six relabellings) of a labelled region mask.
int oracle_canonical_mask(int mask) {
  if (mask < 0 || mask > 127) return -1;
  return canon_map().of_mask[mask];
}

// Pattern of three explicit vertex lists: 1..20; 0 if not a hyper-triangle;
// -1 if two of the sets are equal (the paper assumes distinct hyperedges).
int oracle_classify(const int32_t* a, int na, const int32_t* b, int nb, const int32_t* c,
                    int nc) {
  VSet A(a, a + na), B(b, b + nb), C(c, c + nc);
  if (A == B || B == C || A == C) return -1;
  if (!intersects(A, B) || !intersects(B, C) || !intersects(A, C)) return 0;
  return pattern_map().of_mask[region_mask(A, B, C)];
}

// Exact counts.  mode 0: Exact-bs shaped; mode 1: all triples.
// Only triangles whose smallest hyperedge id lies in [i_lo, i_hi) are counted
// (pass 0, ne for the whole graph); wedge statistics always cover the needed part.
// counts[21]: [0] = T, [p] = H[p].  stats[ST_N] as in the enum above.
// masks[128] (may be NULL): masks[m] = hyper-triangles whose region mask, in its
// canonical form (oracle_canonical_mask), is m; zero at non-canonical m.
// Returns 0, or a negative input error (-2 empty hyperedge, -3 vertex out of
// range, -4 repeated vertex, -5 duplicate hyperedge, -6 bad argument,
// -7 pattern table inconsistent, -8 unclassifiable triple).
int oracle_count(int32_t nv, int32_t ne, const int64_t* e_ptr, const int32_t* e_idx, int mode,
                 int nthreads, int32_t i_lo, int32_t i_hi, uint64_t* counts, uint64_t* stats,
                 uint64_t* masks, double* seconds) {
  auto t0 = std::chrono::steady_clock::now();
  if (!counts || !stats || nv < 0 || ne < 0 || i_lo < 0 || i_hi > ne || i_lo > i_hi) return -6;
  if (!oracle_pattern_table_ok()) return -7;
  std::memset(counts, 0, sizeof(uint64_t) * 21);
  std::memset(stats, 0, sizeof(uint64_t) * ST_N);
  if (masks) std::memset(masks, 0, sizeof(uint64_t) * 128);
  const auto& cm = canon_map();
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  Graph g;
  int rc = load(g, nv, ne, e_ptr, e_idx);
  if (rc) return rc;
  const auto& pm = pattern_map();
  int bad = 0;

  if (mode == 1) {
    // brute force: every unordered triple of distinct hyperedges
    uint64_t H[21] = {0};
    uint64_t M[128] = {0};
    uint64_t open = 0, connected = 0, W = 0, Wc = 0;
    uint64_t maxdeg = 0;
    for (int32_t i = 0; i < ne; ++i) {
      uint64_t deg = 0;
      for (int32_t j = 0; j < ne; ++j) {
        if (j == i || !intersects(g.e[i], g.e[j])) continue;
        ++deg;
        if (g.e[i] == g.e[j]) return -5;
        if (j > i) {
          ++W;
          size_t w = common(g.e[i], g.e[j]);
          if (w == std::min(g.e[i].size(), g.e[j].size())) ++Wc;
        }
      }
      maxdeg = std::max(maxdeg, deg);
      connected += deg * (deg - (deg ? 1 : 0)) / 2;
    }
    for (int32_t i = i_lo; i < i_hi; ++i)
      for (int32_t j = i + 1; j < ne; ++j)
        for (int32_t k = j + 1; k < ne; ++k) {
          int ij = intersects(g.e[i], g.e[j]), jk = intersects(g.e[j], g.e[k]),
              ik = intersects(g.e[i], g.e[k]);
          int n = ij + jk + ik;
          if (n == 2) ++open;
          if (n != 3) continue;
          const int m = region_mask(g.e[i], g.e[j], g.e[k]);
          int p = pm.of_mask[m];
          if (p == 0) { bad = 1; continue; }
          ++H[p];
          ++M[cm.of_mask[m]];
        }
    for (int p = 1; p <= 20; ++p) { counts[p] = H[p]; counts[0] += H[p]; }
    if (masks) std::memcpy(masks, M, sizeof(M));
    stats[ST_W] = W; stats[ST_WC] = Wc; stats[ST_WT] = W - Wc;
    stats[ST_CONNECTED] = connected; stats[ST_OPEN] = open; stats[ST_MAXDEG] = maxdeg;
    stats[ST_T] = counts[0];
    if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return bad ? -8 : 0;
  }
  if (mode != 0) return -6;

  // Projection graph (Sec. 2 / Algorithm 1): N(e_x) for every hyperedge that the
  // requested range needs: the range itself and the larger-id neighbours of it.
  const bool whole = (i_lo == 0 && i_hi == ne);
  std::vector<std::vector<int32_t>> N(ne);
  std::vector<char> need(ne, whole ? 1 : 0);
  if (!whole) {
    for (int32_t i = i_lo; i < i_hi; ++i) {
      need[i] = 1;
      for (int32_t v : g.e[i])
        for (int32_t j : g.Ev[v])
          if (j > i) need[j] = 1;
    }
  }
#pragma omp parallel for schedule(dynamic, 256)
  for (int32_t x = 0; x < ne; ++x)
    if (need[x]) N[x] = neighbours(g, x);

  uint64_t W = 0, Wc = 0, connected = 0, maxdeg = 0;
  int dup = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : W, Wc, connected) reduction(max : maxdeg) reduction(| : dup)
  for (int32_t x = 0; x < ne; ++x) {
    if (!need[x]) continue;
    uint64_t d = N[x].size();
    connected += d * (d - (d ? 1 : 0)) / 2;
    maxdeg = std::max(maxdeg, d);
    for (int32_t y : N[x]) {
      if (y < x) continue;
      ++W;
      size_t w = common(g.e[x], g.e[y]);                      // omega_xy (Def. 2.2)
      if (w == g.e[x].size() && w == g.e[y].size()) dup = 1;   // equal hyperedges
      if (w == std::min(g.e[x].size(), g.e[y].size())) ++Wc;  // inclusion type (Def. 2.3)
    }
  }
  if (dup) return -5;

  int nth = 1;
#ifdef _OPENMP
  nth = omp_get_max_threads();
#endif
  std::vector<uint64_t> Hs((size_t)nth * 21, 0), Ms((size_t)nth * 128, 0);
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    uint64_t* H = &Hs[(size_t)tid * 21];
    uint64_t* M = &Ms[(size_t)tid * 128];
#pragma omp for schedule(dynamic, 64) reduction(| : bad)
    for (int32_t i = i_lo; i < i_hi; ++i) {
      const auto& Ni = N[i];
      for (size_t a = 0; a < Ni.size(); ++a) {
        int32_t j = Ni[a];
        if (j <= i) continue;
        for (size_t b = a + 1; b < Ni.size(); ++b) {
          int32_t k = Ni[b];                                     // i < j < k
          if (!adjacent(N, j, k)) continue;                      // e_j cap e_k empty
          const int m = region_mask(g.e[i], g.e[j], g.e[k]);
          int p = pm.of_mask[m];
          if (p == 0) { bad = 1; continue; }
          ++H[p];
          ++M[cm.of_mask[m]];
        }
      }
    }
  }
  for (int t = 0; t < nth; ++t) {
    for (int p = 1; p <= 20; ++p) counts[p] += Hs[(size_t)t * 21 + p];
    if (masks)
      for (int m = 0; m < 128; ++m) masks[m] += Ms[(size_t)t * 128 + m];
  }
  for (int p = 1; p <= 20; ++p) counts[0] += counts[p];
  stats[ST_W] = W; stats[ST_WC] = Wc; stats[ST_WT] = W - Wc;
  stats[ST_CONNECTED] = connected; stats[ST_MAXDEG] = maxdeg; stats[ST_T] = counts[0];
  // every closed triple is counted three times in sum C(deg, 2), every open one once
  stats[ST_OPEN] = whole ? connected - 3 * counts[0] : 0;
  if (seconds) *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return bad ? -8 : 0;
}

// Hyper-triangles by owner.  Order the hyperedges by (|N(e)|, id), |N(e)| the number of
// other hyperedges sharing a vertex with e (Sec. 2).  Every hyper-triangle {e_u, e_v, e_w}
// (Def. 2.4) has exactly one member ranked lowest in that order: its owner.  For each
// requested owner u = owners[k]:
//   above[k]            the neighbours of e_u ranked above it;
//   masks[128 k + m]    the hyper-triangles owned by u whose region mask, in canonical
//                       form (oracle_canonical_mask), is m.
// The degrees of e_u's neighbours are counted with a mark array: for each of them, every
// id met in the E_y lists of its vertices is counted the first time it is met.
// Returns 0, a negative input error as oracle_count, -6 for an owner out of range, or
// -8 (unclassifiable triple).
int oracle_count_owned(int32_t nv, int32_t ne, const int64_t* e_ptr, const int32_t* e_idx,
                       const int32_t* owners, int32_t n, int nthreads, int32_t* above,
                       uint64_t* masks) {
  if (nv < 0 || ne < 0 || n < 0 || (n > 0 && (!owners || !above || !masks))) return -6;
  if (!oracle_pattern_table_ok()) return -7;
  for (int32_t k = 0; k < n; ++k)
    if (owners[k] < 0 || owners[k] >= ne) return -6;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  Graph g;
  int rc = load(g, nv, ne, e_ptr, e_idx);
  if (rc) return rc;
  const auto& pm = pattern_map();
  const auto& cm = canon_map();
  int nth = 1;
#ifdef _OPENMP
  nth = omp_get_max_threads();
#endif
  int bad = 0;
  for (int32_t k = 0; k < n; ++k) {
    const int32_t u = owners[k];
    const std::vector<int32_t> Nu = neighbours(g, u);
    const int64_t du = (int64_t)Nu.size();
    // |N(e_x)| of every neighbour x
    std::vector<int64_t> dx(Nu.size(), 0);
#pragma omp parallel
    {
      std::vector<int32_t> mark((size_t)ne, -1);
#pragma omp for schedule(dynamic, 16)
      for (size_t a = 0; a < Nu.size(); ++a) {
        const int32_t x = Nu[a];
        int64_t d = 0;
        for (int32_t v : g.e[x])
          for (int32_t j : g.Ev[v])
            if (j != x && mark[j] != x) {
              mark[j] = x;
              ++d;
            }
        dx[a] = d;
      }
    }
    // the neighbours ranked above u, ascending id
    std::vector<int32_t> R;
    for (size_t a = 0; a < Nu.size(); ++a)
      if (dx[a] > du || (dx[a] == du && Nu[a] > u)) R.push_back(Nu[a]);
    above[k] = (int32_t)R.size();
    // every pair {v, w} of them whose hyperedges intersect closes a hyper-triangle
    std::vector<uint64_t> Ms((size_t)nth * 128, 0);
#pragma omp parallel
    {
      int tid = 0;
#ifdef _OPENMP
      tid = omp_get_thread_num();
#endif
      uint64_t* M = &Ms[(size_t)tid * 128];
#pragma omp for schedule(dynamic, 8) reduction(| : bad)
      for (size_t a = 0; a < R.size(); ++a)
        for (size_t b = a + 1; b < R.size(); ++b) {
          if (!intersects(g.e[R[a]], g.e[R[b]])) continue;
          const int m = region_mask(g.e[u], g.e[R[a]], g.e[R[b]]);
          if (pm.of_mask[m] == 0) {
            bad = 1;
            continue;
          }
          ++M[cm.of_mask[m]];
        }
    }
    uint64_t* out = masks + 128 * (size_t)k;
    for (int m = 0; m < 128; ++m) {
      out[m] = 0;
      for (int t = 0; t < nth; ++t) out[m] += Ms[(size_t)t * 128 + m];
    }
  }
  return bad ? -8 : 0;
}

// ---------------------------------------------------------------- Appro-bs (Algorithm 6)
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
// 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplications on a 4-word
// counter under a 2-word key that is bumped by the Weyl constants between rounds.
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0, n1 = (uint32_t)p1;
    const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1, n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// The sub-hypergraph G' of Algorithms 6 and 7 (their first step: sigma|E| hyperedges drawn
// uniformly at random).  Reading: hyperedge i gets the priority
// r_i = x1 << 32 | x0 of Philox4x32-10(counter = (i, 0, 1, 0), key = (seed lo, seed hi));
// G' keeps the ceil(sigma * |E|) hyperedges with the smallest (r_i, i), renumbered
// 0 .. |E'|-1 in ascending original id (so the order O is kept).  sigma = 1 keeps all.
// Writes the kept ids, ascending, to kept[] (capacity ne) and returns how many.
int32_t oracle_subgraph(int32_t ne, uint64_t seed, double sigma, int32_t* kept) {
  if (ne < 0 || !(sigma > 0.0) || sigma > 1.0) return -1;
  const int32_t keep = sigma == 1.0 ? ne : (int32_t)std::ceil(sigma * (double)ne);
  std::vector<std::pair<uint64_t, int32_t>> pr((size_t)ne);
  for (int32_t i = 0; i < ne; ++i) {
    uint64_t r = 0;
    if (sigma != 1.0) {
      const uint32_t ctr[4] = {(uint32_t)i, 0u, 1u, 0u};
      const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
      uint32_t x[4];
      oracle_philox4x32_10(ctr, key, x);
      r = ((uint64_t)x[1] << 32) | x[0];
    }
    pr[(size_t)i] = {r, i};
  }
  std::sort(pr.begin(), pr.end());
  std::vector<int32_t> ids;
  for (int32_t k = 0; k < keep; ++k) ids.push_back(pr[(size_t)k].second);
  std::sort(ids.begin(), ids.end());
  for (int32_t k = 0; k < keep; ++k) kept[k] = ids[(size_t)k];
  return keep;
}

}  // extern "C"

namespace {

// CSR of G' (oracle_subgraph) with its hyperedges renumbered in ascending original id.
int sub_csr(int32_t ne, const int64_t* e_ptr, const int32_t* e_idx, uint64_t seed, double sigma,
            std::vector<int64_t>& sp, std::vector<int32_t>& si) {
  std::vector<int32_t> kept((size_t)std::max(ne, 1));
  const int32_t n = oracle_subgraph(ne, seed, sigma, kept.data());
  if (n < 0) return -1;
  sp.assign(1, 0);
  si.clear();
  for (int32_t k = 0; k < n; ++k) {
    const int32_t i = kept[(size_t)k];
    for (int64_t q = e_ptr[i]; q < e_ptr[i + 1]; ++q) si.push_back(e_idx[q]);
    sp.push_back((int64_t)si.size());
  }
  return 0;
}

}  // namespace

extern "C" {

// Hyperwedge sampling estimate (Algorithm 6):
//   the hyperwedges are numbered in the order O of Sec. 2 (i ascending, then j
//   ascending, i < j); sample n draws x = Philox4x32-10(counter = (n lo, n hi, 0, 0),
//   key = (seed lo, seed hi)), r = x1 << 32 | x0 and takes hyperwedge
//   m = floor(r * W / 2^64) (with replacement); the hyper-triangles counted for
//   hyperwedge (i, j) are those {i, j, k} with k > j, i.e. the ones whose smallest
//   hyperwedge in O is (i, j); raw[p] sums them over the samples and
//   est[p] = raw[p] * (W / samples) / sigma^3 (p = 0 is the total).
// With sigma < 1 all of this runs on the sub-hypergraph G' of oracle_subgraph
// (W is then the number of hyperwedges of G').
// identity_draws = 1 replaces the draw by m = n (every wedge once when the
// samples are 0 .. W-1) - the special case that pins the estimate to the count.
int oracle_sample_estimate(int32_t nv, int32_t ne, const int64_t* e_ptr, const int32_t* e_idx,
                           uint64_t seed, uint64_t first, uint64_t num, double sigma,
                           int identity_draws, int nthreads, uint64_t* raw, double* est,
                           uint64_t* wedges) {
  if (!raw || !est || num == 0) return -6;
  if (!oracle_pattern_table_ok()) return -7;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  std::vector<int64_t> sub_ptr;
  std::vector<int32_t> sub_idx;
  if (sigma != 1.0) {
    if (sub_csr(ne, e_ptr, e_idx, seed, sigma, sub_ptr, sub_idx)) return -6;
    ne = (int32_t)sub_ptr.size() - 1;
    e_ptr = sub_ptr.data();
    e_idx = sub_idx.data();
  }
  Graph g;
  int rc = load(g, nv, ne, e_ptr, e_idx);
  if (rc) return rc;
  std::vector<std::vector<int32_t>> N(ne);
#pragma omp parallel for schedule(dynamic, 256)
  for (int32_t x = 0; x < ne; ++x) N[x] = neighbours(g, x);
  // wedges in O order: prefix over i of |{j in N(i) : j > i}|
  std::vector<uint64_t> start(ne + 1, 0);
  for (int32_t i = 0; i < ne; ++i) {
    uint64_t up = 0;
    for (int32_t j : N[i]) up += j > i;
    start[i + 1] = start[i] + up;
  }
  const uint64_t W = start[ne];
  if (wedges) *wedges = W;
  std::memset(raw, 0, sizeof(uint64_t) * 21);
  if (W == 0) {
    for (int p = 0; p <= 20; ++p) est[p] = 0.0;
    return 0;
  }
  const auto& pm = pattern_map();
  int nth = 1;
#ifdef _OPENMP
  nth = omp_get_max_threads();
#endif
  std::vector<uint64_t> Hs((size_t)nth * 21, 0);
  int bad = 0;
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    uint64_t* H = &Hs[(size_t)tid * 21];
#pragma omp for schedule(dynamic, 1024) reduction(| : bad)
    for (int64_t s = 0; s < (int64_t)num; ++s) {
      const uint64_t n = first + (uint64_t)s;
      uint64_t m;
      if (identity_draws) {
        m = n;
        if (m >= W) continue;
      } else {
        const uint32_t ctr[4] = {(uint32_t)n, (uint32_t)(n >> 32), 0u, 0u};
        const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        uint32_t x[4];
        oracle_philox4x32_10(ctr, key, x);
        const uint64_t r = ((uint64_t)x[1] << 32) | x[0];
        m = (uint64_t)(((unsigned __int128)r * W) >> 64);
      }
      // the m-th hyperwedge (i, j) in O
      const int32_t i = (int32_t)(std::upper_bound(start.begin(), start.end(), m) - start.begin()) - 1;
      uint64_t rank = m - start[i];
      int32_t j = -1;
      for (int32_t x : N[i])
        if (x > i && rank-- == 0) { j = x; break; }
      // every hyperwedge (i, k) after (i, j) in O whose k meets e_j closes a triangle
      for (int32_t k : N[i]) {
        if (k <= j || !adjacent(N, j, k)) continue;
        const int p = pm.of_mask[region_mask(g.e[i], g.e[j], g.e[k])];
        if (p == 0) { bad = 1; continue; }
        ++H[p];
      }
    }
  }
  for (int t = 0; t < nth; ++t)
    for (int p = 1; p <= 20; ++p) raw[p] += Hs[(size_t)t * 21 + p];
  for (int p = 1; p <= 20; ++p) raw[0] += raw[p];
  const double scale = (double)W / (double)num;
  const double s3 = sigma * sigma * sigma;
  for (int p = 0; p <= 20; ++p) est[p] = ((double)raw[p] * scale) / s3;
  return bad ? -8 : 0;
}

// Appro-adv (Algorithm 7).  On G' (oracle_subgraph), the hyperwedges split into
// W^t (intersection type) and W^c (inclusion type) (Def. 2.3), each in the order O.
// The alpha samples are shared out as Algorithm 7 states, floors of exact integer quotients:
//   alpha_1 = |W^t|^2 alpha / |W|^2     TTT class, drawn from W^t
//   alpha_2 = |W^c|^2 alpha / |W|^2     CCC class, drawn from W^c
//   alpha_3 = |W^t||W^c| alpha / |W|^2  TTC class, drawn from W^t
//   alpha_4 = |W^t||W^c| alpha / |W|^2  TCC class, drawn from W^c.
// Sample s (0 .. alpha_x - 1) of set x draws n = first + s from Philox4x32-10
// (counter = (n lo, n hi, 1 + x, 0), key = seed), r = x1 << 32 | x0, and takes the
// m-th hyperwedge of its type, m = floor(r |W^type| / 2^64).  For the drawn (i, j)
// every k adjacent to both closes a hyper-triangle; it is counted when its class
// (from its pattern: 1 CCC, 2-5 TCC, 6-8 TTC, 9-20 TTT) is the set's class and
// (i, j) is, among the triangle's hyperwedges of the drawn type, the first in O
// (reading: the triangle's owner, so that every triangle of the class is counted
// once over W^type).  est[p] = raw[p] * (|W^type| / alpha_x) / sigma^3 for p in the
// set's class; est[0] = sum of est[1..20] in order.  class_mask (bit 0 CCC, 1 TCC,
// 2 TTC, 3 TTT) selects the sets that are drawn (targeted estimation).
// identity_draws = 1 draws every hyperwedge of the type once (alpha_x = |W^type|,
// m = s): the estimate is then the exact count of each selected class.
// info[8] = W, W_t, W_c, alpha_1..alpha_4, |E'|.
int oracle_sample_estimate_adv(int32_t nv, int32_t ne, const int64_t* e_ptr,
                               const int32_t* e_idx, uint64_t seed, uint64_t first, uint64_t num,
                               double sigma, int class_mask, int identity_draws, int nthreads,
                               uint64_t* raw, double* est, uint64_t* info) {
  if (!raw || !est || !info) return -6;
  if (!oracle_pattern_table_ok()) return -7;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  std::vector<int64_t> sub_ptr;
  std::vector<int32_t> sub_idx;
  if (sigma != 1.0) {
    if (sub_csr(ne, e_ptr, e_idx, seed, sigma, sub_ptr, sub_idx)) return -6;
    ne = (int32_t)sub_ptr.size() - 1;
    e_ptr = sub_ptr.data();
    e_idx = sub_idx.data();
  }
  Graph g;
  int rc = load(g, nv, ne, e_ptr, e_idx);
  if (rc) return rc;
  std::vector<std::vector<int32_t>> N(ne);
#pragma omp parallel for schedule(dynamic, 256)
  for (int32_t x = 0; x < ne; ++x) N[x] = neighbours(g, x);
  // inclusion type of a hyperwedge (Def. 2.3): the intersection is the smaller hyperedge
  auto inclusion = [&](int32_t a, int32_t b) {
    size_t common = 0;
    for (int32_t v : g.e[a]) common += g.e[b].count(v);
    return common == std::min(g.e[a].size(), g.e[b].size());
  };
  // per type, the wedges (i, j), j > i, in O: row starts and the row lists
  std::vector<std::vector<int32_t>> up[2];   // [0] intersection, [1] inclusion
  up[0].assign(ne, {});
  up[1].assign(ne, {});
#pragma omp parallel for schedule(dynamic, 256)
  for (int32_t i = 0; i < ne; ++i)
    for (int32_t j : N[i])
      if (j > i) up[inclusion(i, j) ? 1 : 0][i].push_back(j);
  std::vector<uint64_t> start[2];
  for (int t = 0; t < 2; ++t) {
    start[t].assign(ne + 1, 0);
    for (int32_t i = 0; i < ne; ++i) start[t][i + 1] = start[t][i] + up[t][i].size();
  }
  const uint64_t Wt = start[0][ne], Wc = start[1][ne], W = Wt + Wc;
  uint64_t alpha[4] = {0, 0, 0, 0};
  if (W > 0) {
    const unsigned __int128 den = (unsigned __int128)W * W;
    alpha[0] = (uint64_t)((unsigned __int128)Wt * Wt * num / den);
    alpha[1] = (uint64_t)((unsigned __int128)Wc * Wc * num / den);
    alpha[2] = alpha[3] = (uint64_t)((unsigned __int128)Wt * Wc * num / den);
  }
  const int set_type[4] = {0, 1, 0, 1};     // the type each set draws from
  const int set_class[4] = {3, 0, 2, 1};    // TTT, CCC, TTC, TCC
  static const int kClassOf[21] = {-1, 0, 1, 1, 1, 1, 2, 2, 2, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3, 3};
  if (identity_draws)
    for (int x = 0; x < 4; ++x) alpha[x] = start[set_type[x]][ne];
  info[0] = W; info[1] = Wt; info[2] = Wc;
  for (int x = 0; x < 4; ++x) info[3 + x] = alpha[x];
  info[7] = (uint64_t)ne;
  std::memset(raw, 0, sizeof(uint64_t) * 21);
  for (int p = 0; p <= 20; ++p) est[p] = 0.0;
  const auto& pm = pattern_map();
  int bad = 0;
  for (int x = 0; x < 4; ++x) {
    if (!(class_mask >> set_class[x] & 1) || alpha[x] == 0) continue;
    const int t = set_type[x];
    const uint64_t Wx = start[t][ne];
    uint64_t H[21] = {0};
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : H[:21]) reduction(| : bad)
    for (int64_t s = 0; s < (int64_t)alpha[x]; ++s) {
      uint64_t m;
      if (identity_draws) {
        m = (uint64_t)s;
      } else {
        const uint64_t n = first + (uint64_t)s;
        const uint32_t ctr[4] = {(uint32_t)n, (uint32_t)(n >> 32), (uint32_t)(1 + x), 0u};
        const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        uint32_t xr[4];
        oracle_philox4x32_10(ctr, key, xr);
        const uint64_t r = ((uint64_t)xr[1] << 32) | xr[0];
        m = (uint64_t)(((unsigned __int128)r * Wx) >> 64);
      }
      const int32_t i =
          (int32_t)(std::upper_bound(start[t].begin(), start[t].end(), m) - start[t].begin()) - 1;
      const int32_t j = up[t][i][(size_t)(m - start[t][i])];
      for (int32_t k : N[i]) {
        if (k == j || !adjacent(N, j, k)) continue;
        const int p = pm.of_mask[region_mask(g.e[i], g.e[j], g.e[k])];
        if (p == 0) { bad = 1; continue; }
        if (kClassOf[p] != set_class[x]) continue;
        // the triangle's hyperwedges in O: (a,b) < (a,c) < (b,c) for a < b < c
        int32_t v[3] = {i, j, k};
        std::sort(v, v + 3);
        const int32_t pairs[3][2] = {{v[0], v[1]}, {v[0], v[2]}, {v[1], v[2]}};
        for (auto& pq : pairs) {
          if ((inclusion(pq[0], pq[1]) ? 1 : 0) != t) continue;
          if (pq[0] == std::min(i, j) && pq[1] == std::max(i, j)) ++H[p];
          break;   // only the first hyperwedge of the drawn type owns the triangle
        }
      }
    }
    const double scale = (double)Wx / (double)alpha[x];
    const double s3 = sigma * sigma * sigma;
    for (int p = 1; p <= 20; ++p) {
      if (kClassOf[p] != set_class[x]) continue;
      raw[p] = H[p];
      est[p] = ((double)H[p] * scale) / s3;
    }
  }
  for (int p = 1; p <= 20; ++p) {
    raw[0] += raw[p];
    est[0] += est[p];
  }
  return bad ? -8 : 0;
}

// The hyper-triangles of one pattern (the problem statement of Sec. 2: compute the
// hyper-triangles of a given pattern p; 0 = every pattern), as triples i < j < k in
// lexicographic order.  mode 0 enumerates like Exact-bs (Algorithm 1), mode 1 tries every
// triple.  The first min(total, capacity) triples go to out[3 * t ..]; *total = how many.
int oracle_enumerate(int32_t nv, int32_t ne, const int64_t* e_ptr, const int32_t* e_idx, int mode,
                     int pattern, int nthreads, int32_t* out, uint64_t capacity,
                     uint64_t* total) {
  if (!total || pattern < 0 || pattern > 20 || (capacity > 0 && !out)) return -6;
  if (!oracle_pattern_table_ok()) return -7;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
  Graph g;
  int rc = load(g, nv, ne, e_ptr, e_idx);
  if (rc) return rc;
  const auto& pm = pattern_map();
  std::vector<std::vector<int32_t>> N(ne);
#pragma omp parallel for schedule(dynamic, 256)
  for (int32_t x = 0; x < ne; ++x) N[x] = neighbours(g, x);
  int nth = 1;
#ifdef _OPENMP
  nth = omp_get_max_threads();
#endif
  std::vector<std::vector<std::array<int32_t, 3>>> found((size_t)nth);
  int bad = 0;
#pragma omp parallel
  {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    auto& mine = found[(size_t)tid];
#pragma omp for schedule(dynamic, 16) reduction(| : bad)
    for (int32_t i = 0; i < ne; ++i) {
      if (mode == 1) {   // every triple i < j < k
        for (int32_t j = i + 1; j < ne; ++j)
          for (int32_t k = j + 1; k < ne; ++k) {
            if (!adjacent(N, i, j) || !adjacent(N, j, k) || !adjacent(N, i, k)) continue;
            const int p = pm.of_mask[region_mask(g.e[i], g.e[j], g.e[k])];
            if (p == 0) { bad = 1; continue; }
            if (pattern == 0 || p == pattern) mine.push_back({i, j, k});
          }
      } else {           // pairs of neighbours of e_i above i that meet
        const auto& Ni = N[i];
        for (size_t a = 0; a < Ni.size(); ++a) {
          const int32_t j = Ni[a];
          if (j <= i) continue;
          for (size_t b = a + 1; b < Ni.size(); ++b) {
            const int32_t k = Ni[b];
            if (!adjacent(N, j, k)) continue;
            const int p = pm.of_mask[region_mask(g.e[i], g.e[j], g.e[k])];
            if (p == 0) { bad = 1; continue; }
            if (pattern == 0 || p == pattern) mine.push_back({i, j, k});
          }
        }
      }
    }
  }
  std::vector<std::array<int32_t, 3>> all;
  for (auto& f : found) all.insert(all.end(), f.begin(), f.end());
  std::sort(all.begin(), all.end());
  *total = all.size();
  for (uint64_t t = 0; t < std::min<uint64_t>(capacity, all.size()); ++t)
    for (int c = 0; c < 3; ++c) out[3 * t + (uint64_t)c] = all[(size_t)t][(size_t)c];
  return bad ? -8 : 0;
}

int oracle_max_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
