/*
 * hg.h - C ABI of the GB300 exact hyper-triangle counting library (libhg).
 *
 * Method: Yin et al., "Efficient Computation of Hyper-triangles on
 * Hypergraphs", PVLDB 18(3), 2024.  Step one builds every hyperwedge (a pair of
 * hyperedges sharing >= 1 vertex, Def. 2.2) with omega_ij = |e_i cap e_j|
 * (Sec. 3.1, Algorithm 2); step two closes hyperwedges into hyper-triangles
 * (Def. 2.4), classifies each by the emptiness of its seven Venn regions and
 * reduces into per-pattern counts H[p] (Sec. 2, Table 1) and the fine-grained
 * clustering coefficient (Def. 5.1).
 *
 * Conventions for every entry point:
 *   - Ids are int32, offsets int64.  A hypergraph is given as a hyperedge->vertex
 *     CSR: edge_ptr[|E|+1] (edge_ptr[0] = 0, non-decreasing, edge_ptr[|E|] = nnz)
 *     and edge_vtx[nnz]; row i lists the vertices of e_i strictly ascending.
 *   - Every call returns an hg_status; none aborts, prints or traps.  CUDA errors
 *     of asynchronous work surface at the next call that synchronises.
 *   - One handle is used by one host thread at a time; all device work of a handle
 *     is ordered on the CUDA stream given at load time.
 *   - Device memory of a handle comes from the allocator installed with
 *     hg_set_allocator at the time of the call (default: cudaMallocAsync on the
 *     handle's stream) and is released by hg_free.
 */
#ifndef HG_H_
#define HG_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hg_graph hg_graph; /* opaque; owns the device copy of one hypergraph */

typedef enum hg_status {
  HG_OK = 0,
  HG_ERR_INVALID_ARG = 1,          /* null pointer, negative size, bad edge_ptr shape */
  HG_ERR_EMPTY_HYPEREDGE = 2,      /* a hyperedge with no vertex (Def. 2.1 forbids it) */
  HG_ERR_DUP_VERTEX = 3,           /* a vertex listed twice in one hyperedge */
  HG_ERR_VERTEX_RANGE = 4,         /* vertex id outside [0, num_vertices) */
  HG_ERR_UNSORTED = 5,             /* a hyperedge's vertex list is not ascending */
  HG_ERR_DUPLICATE_HYPEREDGE = 6,  /* two equal hyperedges (the paper assumes none, Sec. 2) */
  HG_ERR_OOM = 7,                  /* the allocator returned no memory */
  HG_ERR_CUDA = 8,                 /* a CUDA runtime call failed */
  HG_ERR_TIMEOUT = 9,              /* a bounded device wait gave up */
  HG_ERR_STATE = 10,               /* call out of order (e.g. counting before hg_build_wedges) */
  HG_ERR_UNSUPPORTED = 11,         /* input beyond this build's limits */
  HG_ERR_NO_DEVICE = 12,           /* no usable sm_103 device */
  HG_ERR_INTERNAL = 13,            /* a consistency check of the library failed */
  HG_ERR_CANCELLED = 14            /* a served query was cancelled before it ran */
} hg_status;

/*
 * Device allocator hooks.  alloc returns a device pointer of at least `bytes`
 * bytes usable on `stream` (a cudaStream_t), or NULL; free releases it.  ctx is
 * passed back unchanged.  Passing two NULLs restores the default
 * (cudaMallocAsync / cudaFreeAsync on the handle's stream).  The setting is
 * process-wide and is read at each allocation.
 */
typedef void* (*hg_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*hg_free_fn)(void* ptr, size_t bytes, void* stream, void* ctx);
hg_status hg_set_allocator(hg_alloc_fn alloc, hg_free_fn free_fn, void* ctx);

/*
 * Load and validate a hypergraph (Def. 2.1; Sec. 3.1 builds the per-vertex lists
 * E_v, Algorithm 2).
 *   num_vertices, num_edges  |V| >= 1 and |E| >= 0.
 *   edge_ptr, edge_vtx       the hyperedge->vertex CSR described above; host
 *                            pointers if inputs_on_device == 0, device pointers
 *                            otherwise.  They stay owned by the caller and are
 *                            copied; they may be freed when the call returns.
 *   cuda_stream              cudaStream_t for all work of the handle (NULL = legacy
 *                            default stream).
 *   out                      receives the new handle on HG_OK, NULL otherwise.
 * Builds the vertex->hyperedge lists on the device.  Returns HG_ERR_EMPTY_HYPEREDGE,
 * HG_ERR_DUP_VERTEX, HG_ERR_UNSORTED or HG_ERR_VERTEX_RANGE for malformed input,
 * before any counting work.  Synchronises the stream.
 */
hg_status hg_load_csr(int32_t num_vertices, int32_t num_edges, const int64_t* edge_ptr,
                      const int32_t* edge_vtx, int inputs_on_device, void* cuda_stream,
                      hg_graph** out);

/* Optional tuning of hg_build_wedges; zero fields mean "choose automatically". */
typedef struct hg_tuning {
  int32_t dense_min_size;  /* hyperedges with at least this many vertices form the
                              dense tensor-core tile set; -1 disables the dense path */
  int32_t dense_max_count; /* cap on the size of the dense set (0 = 1% of |E|) */
  int32_t close_mode;      /* step two team shape: 0 = by out-degree and |e_u| (warp
                              teams where they fit), 1 = global-table teams for every
                              hyperedge, 2 = warp and block teams build their tables,
                              then hand every hyperedge over to the global-table teams
                              (the path a team whose cuckoo stash overflows takes);
                              counts do not depend on it */
  int32_t orient_exact;    /* 1 = oriented rows in an exact layout (W entries, one extra
                              counting pass); 0 = room for deg(i) per row (2W entries)
                              while that fits 8 GB.  Counts do not depend on it */
  int32_t gather_light_max; /* step one: rows gathering at most this many incidences take
                               one warp, larger ones a block (0 = the largest a warp's table
                               holds: 512 in the packed layout, 256 otherwise; 32..512,
                               capped at that largest) */
  int32_t warp_team_max;   /* step two: largest out-degree closed by a one-warp team; larger
                              ones take block teams (0 = 256; 64, 128 or 256) */
  int32_t reserved[2];
} hg_tuning;

typedef struct hg_wedge_stats {
  uint64_t W;           /* hyperwedges: unordered pairs of hyperedges sharing a vertex */
  uint64_t W_t;         /* intersection type (Def. 2.3) */
  uint64_t W_c;         /* inclusion type: one hyperedge contains the other */
  uint64_t connected;   /* sum over hyperedges of C(deg, 2), deg = |N(e_i)| (Sec. 2) */
  uint64_t max_deg;     /* max |N(e_i)| */
  uint64_t max_out_deg; /* max out-degree after degree ordering */
  uint64_t dense_edges; /* hyperedges handled by the dense tile path */
  uint64_t reserved;
} hg_wedge_stats;

/*
 * Step one (Sec. 3.1, Algorithm 2): omega_ij = |e_i cap e_j| for every hyperwedge,
 * its type (Def. 2.3), then the degree-ordered orientation used by step two.
 * opt may be NULL.  out may be NULL.  Rejects equal hyperedges with
 * HG_ERR_DUPLICATE_HYPEREDGE.  May be called again; it rebuilds.  Synchronises.
 * A tuning field out of its range (close_mode not 0-2, orient_exact not 0-1) is
 * rejected with HG_ERR_INVALID_ARG before anything changes: a built handle stays
 * built.  HG_ERR_UNSUPPORTED for a hyperedge whose vertices lie in 2^30 or more
 * hyperedges in all (sum over its vertices v of |E_v| - 1).  Any other error leaves the handle unbuilt (counting then answers
 * HG_ERR_STATE until a build succeeds).
 */
hg_status hg_build_wedges(hg_graph* g, const hg_tuning* opt, hg_wedge_stats* out);

/*
 * Autotuner (no counterpart in the paper: the paper's parameters are its algorithms'
 * class split, not kernel shapes).  Picks, for this hypergraph, the hg_tuning fields
 * whose best value depends on the input - warp_team_max (64/128/256), gather_light_max
 * (128/256/default), orient_exact (0/1) and, for hyperedges of 32+ vertices, dense_min_size
 * (automatic / off / 64) - by coordinate descent: from the defaults, each field in turn
 * tries its other values with the rest at the best so far and keeps one that lowers the
 * device time of hg_build_wedges + hg_count_patterns (CUDA events on the handle's
 * stream).  Every candidate's counts, canonical mask histogram and wedge statistics must
 * agree (HG_ERR_INTERNAL otherwise).  The choice is kept on the handle and used by later
 * hg_build_wedges calls given opt = NULL; the handle is left built and counted with it.
 *   out  may be NULL; else the choice, and every candidate tried with its time and counts.
 * HG_ERR_UNSUPPORTED for a wave handle of a batch (see hg_batch_autotune).  Synchronises.
 */
#define HG_AUTOTUNE_MAX 16
typedef struct hg_autotune_result {
  hg_tuning best;                         /* the chosen tuning */
  float best_ms;                          /* its step one + step two time, ms */
  int32_t best_index;                     /* its position in tried[] */
  int32_t num_tried;                      /* candidates timed */
  int32_t reserved;
  hg_tuning tried[HG_AUTOTUNE_MAX];       /* in the order they ran; tried[0] = defaults */
  float ms[HG_AUTOTUNE_MAX];
  uint64_t counts[HG_AUTOTUNE_MAX][21];   /* each candidate's hg_count_patterns result */
} hg_autotune_result;
hg_status hg_autotune(hg_graph* g, hg_autotune_result* out);

/*
 * Step two (Sec. 3.2-3.3; Algorithms 3-5 compute the same counts per class):
 * every hyper-triangle {e_i, e_j, e_k} (three pairwise-intersecting hyperedges,
 * Def. 2.4) is found once and classified into pattern p in 1..20 from the
 * emptiness of its seven Venn regions (Sec. 2).
 *   counts[21]  out: counts[0] = total hyper-triangles, counts[p] = H[p].
 * Requires hg_build_wedges.  Synchronises.
 */
hg_status hg_count_patterns(hg_graph* g, uint64_t counts[21]);

/*
 * The pattern of every hyper-triangle before any numbering (Sec. 2: a pattern is the
 * set of non-empty Venn regions up to relabelling the three hyperedges).  masks[m] =
 * hyper-triangles counted by the last hg_count_patterns whose region mask (bit r =
 * region r of (a)..(g) non-empty), in canonical form (the smallest of its six
 * relabellings, see hg_canonical_masks), is m; 0 at every non-canonical m.  H[p] is the
 * sum of masks[m] over the canonical m of pattern p (hg_pattern_table).
 *   masks[128]  out.
 * Requires hg_count_patterns (HG_ERR_STATE before).  No device work.
 */
hg_status hg_mask_histogram(hg_graph* g, uint64_t masks[128]);

/*
 * Step two restricted to owners.  The closure orders the hyperedges by (|N(e)|, id),
 * |N(e)| the number of other hyperedges sharing a vertex with e (Sec. 2), and finds each
 * hyper-triangle (Def. 2.4) from its lowest-ranked member, its owner.  This call runs
 * only the teams of the listed owners, with the same kernels and team shapes as
 * hg_count_patterns, so any part of a large hypergraph can be checked against a
 * reference that counts the same owners one by one.
 *   owners[num_owners]  in, host: hyperedge ids in [0, |E|); repeats count once.
 *   counts[21]          out: as hg_count_patterns, over the owned hyper-triangles.
 *   masks[128]          out (may be NULL): as hg_mask_histogram, over the same.
 * HG_ERR_INVALID_ARG for an id out of range; HG_ERR_UNSUPPORTED for a wave handle of a
 * batch.  Requires hg_build_wedges; afterwards the handle is built but not counted
 * (hg_mask_histogram and hg_clustering_coeff want a new hg_count_patterns).  Synchronises.
 */
hg_status hg_count_owned(hg_graph* g, const int32_t* owners, int32_t num_owners,
                         uint64_t counts[21], uint64_t masks[128]);

/*
 * Out-degree of every hyperedge in the orientation step two uses: the number of its
 * neighbours ranked above it in (|N(e)|, id) (see hg_count_owned).
 *   out_degree[|E|]  out, host.
 * Requires hg_build_wedges.  Synchronises.
 */
hg_status hg_out_degrees(hg_graph* g, int32_t* out_degree);

/*
 * Hyperwedge-sampling estimate of the per-pattern counts (Sec. 4.1, Algorithm 6,
 * "Appro-bs"), with vertex-sampling rate sigma = 1.
 * The W hyperwedges (i, j), i < j, are numbered in the order O of Sec. 2 (by i,
 * then j).  Sample n, for n = first_sample .. first_sample + num_samples - 1,
 * draws hyperwedge m = floor(r * W / 2^64), where r = x1 * 2^32 + x0 and
 * (x0, x1, x2, x3) is the Philox4x32-10 block (Salmon et al., SC'11) of counter
 * (n mod 2^32, n div 2^32, 0, 0) under key (seed mod 2^32, seed div 2^32).
 * For the drawn (i, j) every k > j adjacent to both closes a hyper-triangle; it
 * is classified as in hg_count_patterns and counted.
 *   raw[21]  out: raw[0] = hyper-triangles found over all samples, raw[p] per pattern.
 *   est[21]  out: est[p] = raw[p] * (W / num_samples) / sigma^3 in IEEE double
 *                 (0 when num_samples == 0).
 * Disjoint sample ranges with the same seed are independent draws, so split runs
 * sum to one run over the union (raw exactly).  Builds the sorted neighbour rows
 * on the first call after hg_build_wedges (W extra entries of device memory).
 * sigma in (0, 1] (the sigma|E| draw of Algorithm 6): with sigma < 1 everything above runs on
 * the sub-hypergraph G' of the ceil(sigma |E|) hyperedges with the smallest
 * priorities r_i = x1 * 2^32 + x0 of Philox4x32-10(counter (i, 0, 1, 0), key as
 * above) (ties by id), renumbered in id order; W is then G''s, and est[p] =
 * raw[p] * (W / num_samples) / sigma^3.  G' is built on the device and kept on the
 * handle for the last (seed, sigma).
 * Requires hg_build_wedges.  sigma outside (0, 1] is HG_ERR_INVALID_ARG; a wave handle
 * of a batch is HG_ERR_UNSUPPORTED.  A hyperedge with more than 16,384 neighbours of
 * larger index is HG_ERR_UNSUPPORTED.  Synchronises.
 */
hg_status hg_sample_estimate(hg_graph* g, uint64_t seed, uint64_t first_sample,
                             uint64_t num_samples, double sigma, uint64_t raw[21],
                             double est[21]);

/*
 * Class-targeted sampling estimate (Sec. 4.2, Algorithm 7, "Appro-adv").  On G (or on
 * G' for sigma < 1, as above) the hyperwedges split into W^t (intersection type) and
 * W^c (inclusion type) (Def. 2.3), each numbered in the order O.  The num_samples = alpha
 * draws are shared out as Algorithm 7 states, as exact integer floors:
 *   set 1: alpha_1 = |W^t|^2 alpha / |W|^2 draws from W^t, counting the TTT class (9-20)
 *   set 2: alpha_2 = |W^c|^2 alpha / |W|^2 draws from W^c, counting CCC (1)
 *   set 3: alpha_3 = |W^t||W^c| alpha / |W|^2 draws from W^t, counting TTC (6-8)
 *   set 4: alpha_4 = alpha_3 draws from W^c, counting TCC (2-5).
 * Draw s of set x uses n = first_sample + s and Philox4x32-10(counter (n lo, n hi, 1 + x,
 * 0), key (seed lo, seed hi)); r = x1 * 2^32 + x0 picks the hyperwedge
 * m = floor(r |W^type| / 2^64) of that type.  For the drawn (i, j), every k adjacent to
 * both closes a hyper-triangle, counted when it is of the set's class and (i, j) is, among
 * its hyperwedges of the drawn type, the first in O (so each triangle of the class is
 * counted once over W^type).
 *   class_mask  bit 0 CCC, 1 TCC, 2 TTC, 3 TTT: the sets drawn (targeted estimation);
 *               unselected classes stay 0.
 *   raw[21], est[21]  out: per pattern; est[p] = raw[p] (|W^type| / alpha_x) / sigma^3 in
 *               IEEE double; raw[0], est[0] = the sums over p = 1..20 in order.
 *   info[8]     out (may be NULL): W, W^t, W^c, alpha_1..alpha_4, |E'|.
 * Builds, on the first call after hg_build_wedges, the upper rows split by type and every
 * neighbour row sorted (3W more entries).  Limits and errors as hg_sample_estimate, plus
 * every neighbour row at most 16,384 long; class_mask > 15 is HG_ERR_INVALID_ARG.
 */
hg_status hg_sample_estimate_adv(hg_graph* g, uint64_t seed, uint64_t first_sample,
                                 uint64_t num_samples, double sigma, uint32_t class_mask,
                                 uint64_t raw[21], double est[21], uint64_t info[8]);

/*
 * The hyper-triangles of one pattern (Sec. 2, problem statement: compute the
 * hyper-triangles of a given pattern p).  Every hyper-triangle {e_i, e_j, e_k},
 * i < j < k, of pattern `pattern` (1..20; 0 = every pattern) is found once, from its
 * smallest hyperwedge (i, j) in the order O, and written as the three ids (i, j, k).
 *   triples   [capacity][3] int32, on the device (triples_on_device = 1) or the host;
 *             the first min(total, capacity) triples found are written, in no fixed
 *             order (each triple ascending).
 *   total     out: the number of hyper-triangles of the pattern (= H[pattern], or T).
 * Uses the sorted upper rows of hg_sample_estimate (built on first use).  Requires
 * hg_build_wedges; a wave handle of a batch is HG_ERR_UNSUPPORTED.  Synchronises.
 */
hg_status hg_enumerate_pattern(hg_graph* g, int32_t pattern, int32_t* triples, uint64_t capacity,
                               int triples_on_device, uint64_t* total);

/*
 * Fine-grained hypergraph clustering coefficient (Def. 5.1):
 *   cc = 3 * sum_{p=1..20} eps[p-1] * H[p] / open,
 * evaluated on the host in IEEE double with the sum taken in order p = 1..20;
 * open = hyper-triples with exactly two of their three pairs connected
 * ("open hyper-triangles"), = connected - 3 * total.  cc is NaN when open == 0.
 * eps: 20 weights in [0, 1] (not checked).  Any output pointer may be NULL.
 * Requires hg_count_patterns on the same handle.  No device work.
 */
hg_status hg_clustering_coeff(hg_graph* g, const double eps[20], double* cc,
                              uint64_t* open_triples, uint64_t* connected_triples);

/*
 * Work done by the last hg_count_patterns or hg_count_owned of a handle (counted by the
 * kernels):
 *   probes       sum over oriented wedges u->v of |out(v)|: out-list entries
 *                streamed and looked up in u's table (every hyper-triangle is
 *                one successful probe);
 *   gathers      entries of E_y read to build the Omega_ux vertex masks;
 *   out_entries  entries of the teams' own out-lists out(u) (= oriented wedges
 *                of hyperedges with out-degree >= 2);
 *   teams        hyperedges u that owned a closing team (out-degree >= 2);
 *   bucket_*     the same per team shape: warp teams for out-degree <= 64, <= 128,
 *                <= 256 (indices 0-2); block teams with shared-memory tables for <= 1024,
 *                <= 2048 and <= 6144 (<= 4096 when omega or ids need the 8-byte row
 *                layout) (3-5); block teams with global-memory tables for hyperedges of
 *                more than 32 vertices with out-degree <= 4096 and for what the other
 *                teams hand over (6); thread-block clusters sharing global-memory tables
 *                for larger out-degrees (7).
 */
typedef struct hg_close_stats {
  uint64_t probes;
  uint64_t gathers;
  uint64_t out_entries;
  uint64_t teams;
  uint64_t bucket_teams[8];
  uint64_t bucket_probes[8];
  uint64_t bucket_gathers[8];
  uint64_t bucket_out_entries[8];
} hg_close_stats;
hg_status hg_close_stats_get(hg_graph* g, hg_close_stats* out);

/* Process-wide number of kernel launches libhg has issued so far. */
hg_status hg_kernel_launches(uint64_t* n);

/*
 * A bounded device wait, the discipline every wait in libhg's kernels follows (no
 * counterpart in the paper): one thread polls the int32 at device address flag, with
 * back-off, until it is non-zero (HG_OK) or limit_us microseconds of the GPU's global
 * timer have passed (HG_ERR_TIMEOUT; the context stays usable).  Runs on cuda_stream
 * and synchronises it.  Nothing in libhg sets the flag: whatever should set it must have
 * done so before the call (no kernel of libhg ever waits on another launch).
 * HG_ERR_INVALID_ARG for a NULL flag or a negative limit.
 */
hg_status hg_wait_flag(const int32_t* flag, int32_t limit_us, void* cuda_stream);

/*
 * Line-graph degrees without allocating.  The paper has no counterpart: this is
 * for callers that cannot allocate device memory while they run - a service whose
 * device memory is a fixed arena owned by someone else (reserved up front, or the
 * pool of another framework), where a cudaMalloc would fail or stall the other
 * streams on the device.  The call makes ordinary CUDA runtime calls (a memset, a
 * launch, copies, a stream synchronisation), so it is made from plain host code,
 * never from inside a host function enqueued on a stream.  It computes what the
 * count pass of hg_build_wedges computes, from buffers the caller owns:
 *   num_edges            |E| >= 0
 *   edge_ptr, edge_vtx   device hyperedge->vertex CSR (as for hg_load_csr; rows
 *                        ascending, already valid - this call does not validate)
 *   vertex_ptr,          device vertex->hyperedge CSR of the same hypergraph
 *   vertex_edge          (vertex_ptr[|V|+1] int64, vertex_edge[nnz] int32, any order
 *                        inside a list)
 *   degrees              device int32[|E|] out: |N(e_i)|, hyperedges sharing a vertex
 *                        with e_i
 *   inclusion_wedges     device uint64 out: inclusion-type hyperwedges (Def. 2.3)
 *   cuda_stream          stream for the work; the call synchronises it.
 * Scratch is one file-scope device array of 32 MiB (128 tables of 32,768 slots)
 * that every device which loads this code keeps until the process exits.  A
 * hyperedge whose vertices lie in more than 16,384 other (hyperedge, vertex)
 * incidences does not fit a table: the call returns HG_ERR_UNSUPPORTED (and
 * degrees are then incomplete).  Equal hyperedges give HG_ERR_DUPLICATE_HYPEREDGE.
 * The array is placed on a device when the library's device code is loaded there
 * (under lazy module loading: at the first call on that device).  The first call on
 * a device also looks up the array's device address (with that device current).  Calls
 * share the array and its previous contents: the call clears what must start at zero,
 * and two calls whose work overlaps on the same GPU (for example on two streams)
 * race on the array and corrupt each other.  No cudaMalloc, cudaFree or
 * allocating library call is made.
 */
hg_status hg_wedge_degrees_noalloc(int32_t num_edges, const int64_t* edge_ptr,
                                   const int32_t* edge_vtx, const int64_t* vertex_ptr,
                                   const int32_t* vertex_edge, int32_t* degrees,
                                   unsigned long long* inclusion_wedges, void* cuda_stream);

/* Release the handle and every device buffer it owns (stream-ordered).
 * The wave handles of a batch belong to the batch: HG_ERR_STATE for them. */
hg_status hg_free(hg_graph* g);

/*
 * Batches of independent hypergraphs.  The paper counts one hypergraph at a
 * time; a batch counts many in the same kernel launches.  Members get disjoint
 * vertex ranges, so the union's line graph is the disjoint union of theirs, every
 * hyperwedge and hyper-triangle (Defs. 2.2, 2.4) lies in one member, and the
 * closure kernels add each hyper-triangle to its member's 20 pattern bins.  Each
 * member's results equal those of hg_load_csr / hg_build_wedges /
 * hg_count_patterns on that member alone.
 *
 * Consecutive members are grouped into waves of at most max_wave_edges
 * hyperedges (0 = 2^24 - 1, the limit of packed neighbour ids; a larger member
 * is a wave of its own); each wave is one union handle resident on the device.
 *
 *   num_graphs    G >= 1.
 *   num_vertices  [G] host: |V_m| >= 1.
 *   edge_off      [G+1] host: member m owns hyperedges edge_off[m] .. edge_off[m+1]-1
 *                 of the concatenated CSR; edge_off[0] = 0, non-decreasing; empty
 *                 members are allowed.
 *   edge_ptr      [edge_off[G]+1] int64, host or device (inputs_on_device): offsets
 *                 into edge_vtx, edge_ptr[0] = 0, non-decreasing.
 *   edge_vtx      vertex ids LOCAL to the member (0 .. |V_m|-1), each hyperedge
 *                 ascending and duplicate-free; an id outside its member's range is
 *                 HG_ERR_VERTEX_RANGE.  Other input errors as in hg_load_csr.
 * The caller keeps its arrays; the batch holds device copies in union ids.
 * Synchronises.  Free with hg_batch_free.
 */
typedef struct hg_batch hg_batch;
hg_status hg_load_batch(int32_t num_graphs, const int32_t* num_vertices, const int64_t* edge_off,
                        const int64_t* edge_ptr, const int32_t* edge_vtx, int inputs_on_device,
                        int64_t max_wave_edges, void* cuda_stream, hg_batch** out);

/*
 * The same for members stored apart: member m's CSR is edge_ptrs[m][0 .. num_edges[m]]
 * (offsets from 0) and edge_vtxs[m] (member-local ids), all on the host or all on the
 * device.  The pointer arrays themselves are host arrays.  The members are gathered
 * into the waves with one copy per member.
 */
hg_status hg_load_batch_members(int32_t num_graphs, const int32_t* num_vertices,
                                const int32_t* num_edges, const int64_t* const* edge_ptrs,
                                const int32_t* const* edge_vtxs, int inputs_on_device,
                                int64_t max_wave_edges, void* cuda_stream, hg_batch** out);

/* The autotuner of hg_autotune run on one wave of the batch (wave = -1: the wave with the
 * most hyperedges); its choice is kept by every wave and used by hg_batch_build_wedges
 * given opt = NULL.  The batch must be built again afterwards.  Synchronises. */
hg_status hg_batch_autotune(hg_batch* b, int32_t wave, hg_autotune_result* out);

/* Step one (as hg_build_wedges) on every wave.  opt may be NULL; an out-of-range
 * tuning is rejected with HG_ERR_INVALID_ARG before anything changes.  Synchronises. */
hg_status hg_batch_build_wedges(hg_batch* b, const hg_tuning* opt);

/*
 * Step two (as hg_count_patterns) on every wave.
 *   counts  [G][21] out (may be NULL): counts[21 m] = member m's total, counts[21 m + p] = H[p].
 *   stats   [G] out (may be NULL): W, W_t, W_c, connected, max_deg of member m
 *           (max_out_deg and dense_edges are 0 per member).
 * Requires hg_batch_build_wedges.  Synchronises.
 */
hg_status hg_batch_count_patterns(hg_batch* b, uint64_t* counts, hg_wedge_stats* stats);

/* Per member, as hg_mask_histogram: masks [G][128] out.  Requires
 * hg_batch_count_patterns.  No device work. */
hg_status hg_batch_mask_histogram(hg_batch* b, uint64_t* masks);

/* Def. 5.1 per member, as hg_clustering_coeff: cc, open, connected are [G] (each may
 * be NULL).  Requires hg_batch_count_patterns.  No device work. */
hg_status hg_batch_clustering_coeff(hg_batch* b, const double eps[20], double* cc,
                                    uint64_t* open_triples, uint64_t* connected_triples);

/* Number of waves, and wave k's handle (borrowed: for hg_set_timing, hg_kernel_times,
 * hg_close_stats_get) with its first member and member count. */
hg_status hg_batch_waves(hg_batch* b, int32_t* num_waves);
hg_status hg_batch_wave(hg_batch* b, int32_t k, hg_graph** wave, int32_t* first_member,
                        int32_t* num_members);

/* Release the batch, its waves and their device buffers. */
hg_status hg_batch_free(hg_batch* b);

/*
 * Serving: count, clustering-coefficient and sampled-estimate queries on hypergraphs
 * kept resident on the device, answered with continuous batching.  (No counterpart
 * in the paper, which answers one query on one hypergraph at a time.)
 *
 * Queries are admitted in arrival order.  A free worker takes the oldest waiting
 * query with everything that can share its launches: an exact query takes every
 * waiting exact query whose hypergraph is in the batch or still fits
 * (max_batch_graphs, the device-memory budget), and the batch runs as one
 * hg_load_batch_members / hg_batch_build_wedges / hg_batch_count_patterns with each
 * distinct hypergraph evaluated once; an estimate query takes the waiting estimate
 * queries on its hypergraph, which share one load and step one.  `workers` batches
 * run at the same time, each on its own CUDA stream; a batch waits while its memory
 * estimate does not fit the budget (unless nothing else is running).  Every answer
 * equals the one the plain calls give for that query alone.
 *
 * Threads: submit / wait / drain / stats may be called from any thread.  The
 * server's own threads allocate with cudaMallocAsync whatever hg_set_allocator set.
 */
typedef struct hg_server hg_server;

typedef struct {
  int32_t workers;            /* concurrent batches, each with its own stream (0 = 4) */
  int32_t max_batch_graphs;   /* distinct hypergraphs in one exact batch (0 = 64) */
  int64_t memory_budget;      /* device bytes of the batches in flight (0 = half of free) */
  int32_t max_batch_queries;  /* queries in one batch (0 = no limit for exact batches, 256
                                 for estimate groups); 1 = no batching */
  int32_t reserved[3];
} hg_server_options;

typedef enum {
  HG_Q_COUNTS = 0,       /* the 21 counts of hg_count_patterns */
  HG_Q_CLUSTERING = 1,   /* the counts and Def. 5.1 with weights eps */
  HG_Q_ESTIMATE = 2      /* hg_sample_estimate(seed, first_sample, num_samples, 1.0) */
} hg_query_kind;

typedef struct {
  int32_t kind;          /* hg_query_kind */
  int32_t graph;         /* id from hg_server_add_graph */
  uint64_t seed, first_sample, num_samples;   /* HG_Q_ESTIMATE */
  double eps[20];        /* HG_Q_CLUSTERING */
} hg_query;

typedef struct {
  hg_status status;
  int32_t kind, graph;
  uint64_t counts[21];   /* exact counts, or the raw sample counts of an estimate */
  double est[21];        /* HG_Q_ESTIMATE */
  double cc;             /* HG_Q_CLUSTERING: cc, open, connected as hg_clustering_coeff */
  uint64_t open, connected;
  double t_submit, t_start, t_done;   /* seconds since hg_server_create */
  int32_t batch_queries, batch_graphs, worker, reserved;
} hg_result;

typedef struct {
  uint64_t submitted, batches, exact_batches, queries_batched;
  uint64_t max_in_flight_bytes, max_concurrent_batches, budget_bytes;
  double now;            /* seconds since hg_server_create */
} hg_server_stats;

/* Start the workers on the current device.  opt may be NULL (defaults). */
hg_status hg_server_create(const hg_server_options* opt, hg_server** out);

/*
 * Register a hypergraph: its CSR (as hg_load_csr; host or device) is copied into
 * server-owned device memory and stays there until hg_server_destroy.  Validates it
 * and runs step one once to size its memory estimate.  Synchronises.
 */
hg_status hg_server_add_graph(hg_server* s, int32_t num_vertices, int32_t num_edges,
                              const int64_t* edge_ptr, const int32_t* edge_vtx,
                              int inputs_on_device, int32_t* graph_id);

/* Queue a query (copied); returns at once with a ticket for hg_server_wait. */
hg_status hg_server_submit(hg_server* s, const hg_query* q, uint64_t* ticket);

/* Block until the ticket's query is answered, then hand its result over (each ticket
 * once; an unknown or collected ticket is HG_ERR_INVALID_ARG).  The query's own
 * outcome is out->status. */
hg_status hg_server_wait(hg_server* s, uint64_t ticket, hg_result* out);

/* Block until nothing is queued or running. */
hg_status hg_server_drain(hg_server* s);

/* Cancel a query that no worker has taken yet: it leaves the queue and its result
 * (collected by hg_server_wait as usual) has status HG_ERR_CANCELLED.  HG_ERR_STATE when
 * the query is already running or answered (its answer stands); HG_ERR_INVALID_ARG for
 * an unknown or collected ticket. */
hg_status hg_server_cancel(hg_server* s, uint64_t ticket);

hg_status hg_server_stats_get(hg_server* s, hg_server_stats* out);

/* Answer what is queued, stop the workers, free the resident hypergraphs. */
hg_status hg_server_destroy(hg_server* s);

/*
 * The library's pattern table: lut[m] = pattern 1..20 of a labelled region mask
 * m (bit r set = region r of (a)..(g) non-empty, Sec. 2), 0 where m is not a
 * hyper-triangle of three distinct hyperedges.  Host only; no device needed.
 */
hg_status hg_pattern_table(uint8_t lut[128]);

/*
 * The library's canonical forms: canon[m] = the smallest region mask among the six
 * relabellings of the three hyperedges of labelled mask m (Sec. 2: hyper-triangles of
 * the same pattern, and only those, share a canonical mask).  Host only.
 */
hg_status hg_canonical_masks(uint8_t canon[128]);

/*
 * Reads made by the last hg_sample_estimate on this handle (its G' for sigma < 1):
 * work[0] row-pointer reads (8 bytes each) of the row searches, work[1] upper-row entries
 * read (4 bytes packed, 8 unpacked) by the walks and searches, work[2] vertex ids
 * (4 bytes) read by the 3-way merges.  For roofline accounting.
 */
hg_status hg_sample_work_get(hg_graph* g, uint64_t work[3]);

/* Static description of a status code. */
const char* hg_status_str(hg_status s);

/*
 * Per-kernel device times of the last hg_build_wedges / hg_count_patterns on
 * this handle, when timing was switched on with hg_set_timing(g, 1) (CUDA events
 * on the handle's stream around each launch).  names[i] points to static
 * strings; ms[i] is the summed time of that kernel in the last call.  *n is the
 * capacity in and the number written out.
 */
hg_status hg_set_timing(hg_graph* g, int enable);
hg_status hg_kernel_times(hg_graph* g, const char** names, float* ms, int32_t* launches,
                          int32_t* n);

#ifdef __cplusplus
}
#endif

#endif /* HG_H_ */
