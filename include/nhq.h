/*
 * nhq.h -- C ABI of the GB300 (sm_103a) native hybrid-query library.
 *
 * The library answers hybrid queries (Def. 4 of arXiv 2203.13601): top-k objects
 * that are near a query vector AND share its structured attributes, by searching
 * a composite proximity-graph index under the fusion distance (Eq. 6).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Plain pointers and sizes only.  A pointer argument may be device memory
 *   (including memory allocated by another runtime such as PyTorch's caching
 *   allocator) or host memory, except where a call says "device".  The library
 *   detects which with cudaPointerGetAttributes.  Calls that receive host input
 *   or output pointers copy through library-owned device staging and return
 *   only after host outputs are written (the call synchronises `stream`).
 * - `stream` is a cudaStream_t (NULL = legacy default stream).  With device
 *   pointers every call only enqueues work and returns; outputs are valid once
 *   the stream has been synchronised.
 * - Ownership: the caller owns every array it passes.  An nhq_index owns its
 *   device copies (vectors, packed attributes, graph) and its scratch buffers;
 *   it is released by nhq_free.  Indices are not thread-safe: one host thread
 *   per index at a time.
 * - Errors: every call returns nhq_status; nothing aborts or throws across the
 *   ABI.  nhq_last_error() returns a message for the last failing call on the
 *   calling thread.  Invalid sizes or values return NHQ_ERR_ARG before any
 *   work is enqueued; a failing CUDA call returns NHQ_ERR_CUDA; a failed
 *   device allocation returns NHQ_ERR_OOM.
 * - Notation (paper): N objects, d vector dimension, m attributes (1..32, each an
 *   ordinal code 0..255, Sec. 3.2 "ordinal encoding"), R graph out-degree
 *   (the paper's k in Sec. 4), k results, ef search-pool size.
 * - Result order: ascending by (Gamma, id).  `dists` hold Gamma (Eq. 6), not
 *   delta.  Missing results (fewer than k reachable) have id 0xFFFFFFFF,
 *   Gamma +inf and chi 255.
 */
#ifndef NHQ_H
#define NHQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum nhq_status {
    NHQ_OK = 0,
    NHQ_ERR_ARG = 1,
    NHQ_ERR_OOM = 2,
    NHQ_ERR_CUDA = 3,
    NHQ_ERR_ITER_LIMIT = 4, /* per-query status only: expansion cap reached */
    NHQ_ERR_IO = 5
} nhq_status;

/* Weights of the fusion distance Gamma = w_v * delta + w_l * chi (Eq. 6). */
typedef enum nhq_weight_mode {
    NHQ_W_PROPORTIONAL = 0, /* w_v = 1, w_l = delta / m: the recommended setting of Sec. 3.2 */
    NHQ_W_CONSTANT = 1,     /* w_v, w_l as given (Sec. 6.5, curve v)                         */
    NHQ_W_HARMONIC = 3,     /* curves i/ii of Sec. 6.5: Gamma = 2 delta h / (delta + h), h = chi
                               (w_l = 0, curve i) or h = 1 for chi = 0 and w_l * chi otherwise
                               (w_l = c >= 1, curve ii); w_v is unused                      */
    NHQ_W_FILTER = 2        /* brute force only: Gamma = delta if chi = 0, else excluded; the
                               hybrid ground truth of Sec. 6.1                               */
} nhq_weight_mode;

typedef struct nhq_weights {
    int32_t mode; /* nhq_weight_mode */
    float w_v;
    float w_l;
} nhq_weights;

/* Element type of the vector copy used to score candidates during search (a
 * project addition; the paper scores in f32).  Each component of the object
 * vectors is rounded to nearest-even into the copy (FP8 saturates at +-448); the
 * query stays f32 and distances accumulate in f32.  With `rerank` the final pool
 * is re-scored with the f32 vectors and the first k of that order are returned. */
typedef enum nhq_vec_dtype {
    NHQ_VEC_F32 = 0,
    NHQ_VEC_BF16 = 1,
    NHQ_VEC_FP8E4M3 = 2,
    NHQ_VEC_F16 = 3 /* IEEE binary16 (rounded to nearest even, overflow to +-inf) */
} nhq_vec_dtype;

/* Element type of the vectors a caller passes to nhq_index_create_typed /
 * nhq_build_typed (the index keeps an f32 copy for every kernel; an F16 or BF16 input
 * also becomes the index's scoring copy of that type, which is then exact). */
typedef enum nhq_dtype { NHQ_F32 = 0, NHQ_F16 = 1, NHQ_BF16 = 2 } nhq_dtype;

typedef struct nhq_build_params {
    int32_t K;           /* candidate-set size l of Sec. 4.1 (exact K nearest by Gamma); 0 -> 64 */
    int32_t reverse;     /* 1: second selection pass over N(v) plus reverse sources (default)   */
    int32_t reverse_cap; /* at most this many reverse sources per vertex; 0 -> 64               */
    int32_t knn_dtype;   /* 0: exact f32 candidates (nhq_knn); 1: bf16 tensor cores (nhq_knn_bf16);
                            2: NN-descent (nhq_knn_nndescent, 12 iterations at most)           */
} nhq_build_params;

/* How the seed set B of Alg. 2 is chosen (the paper draws it at random). */
typedef enum nhq_seed_mode {
    NHQ_SEED_RANDOM = 0,    /* first min(ef, 32) distinct ids of splitmix64(seed ^ mix64(q)) mod N,
                               at most 64 draws                                              */
    NHQ_SEED_ATTRIBUTE = 1, /* P = objects whose attributes all equal the query's, ascending id;
                               c = |P| >= 1: S = min(ef, 32, c), B = {P[floor(j*c/S)] : j < S};
                               c = 0: as NHQ_SEED_RANDOM                                     */
    NHQ_SEED_GIVEN = 2,     /* B = the valid distinct ids of seeds[q][0..n_seeds)            */
    NHQ_SEED_ATTRIBUTE_NEAR = 3, /* P as above; of its M = min(256, c) members P[floor(j*c/M)]
                               the min(ef, 32) nearest to the query by (delta^2 of the f32
                               rows summed in index order, id); c = 0 as NHQ_SEED_RANDOM.
                               For tuples spread over many clusters, where evenly spaced
                               members rarely include the query's own                       */
    NHQ_SEED_CELL_NEAREST = 4, /* entry cells (nhq_index_build_cells): the T = entry_cells cells
                               of largest score q.c - |c|^2/2 (f32, products summed in index
                               order; ties: smaller cell), i.e. nearest centroids (exactly so
                               when the arithmetic is exact, e.g. integer components); P and
                               c as above,
                               S = min(ef, 32, c); B = the first S members of P in those cells
                               (nearest cell first, ascending ids within a cell), then while
                               fewer than S the evenly spaced P[floor(j*c/S2)], j < S2 = S - |B|
                               (an id listed twice is evaluated once); c = 0 as
                               NHQ_SEED_RANDOM.  Closed queries only (wildcard = 0)          */
    NHQ_SEED_CELL_LEARNED = 5  /* as NHQ_SEED_CELL_NEAREST with the T cells of largest logit
                               (ties: smaller cell) under the entry model `entry_model`       */
} nhq_seed_mode;

/* Learned early stop (a project addition; the paper's search has no learned
 * part): a 2-layer perceptron with NHQ_MLP_INPUTS inputs, NHQ_MLP_HIDDEN ReLU
 * units and one logit.  Parameters are one flat f32 vector:
 * W1[NHQ_MLP_INPUTS][NHQ_MLP_HIDDEN] (input-major) | b1 | W2 | b2. */
#define NHQ_MLP_INPUTS 8
#define NHQ_MLP_HIDDEN 64
#define NHQ_MLP_PARAMS (NHQ_MLP_INPUTS * NHQ_MLP_HIDDEN + 2 * NHQ_MLP_HIDDEN + 1)

/* Learned entry point (a project addition): a 2-layer perceptron that scores the E entry
 * cells of an index from a query vector q (d values): x = s q, NHQ_ENTRY_HIDDEN ReLU
 * units, one logit per cell.  Parameters are one flat f32 vector of
 * nhq_entry_param_count(d, E) values: s (a fixed input scale, not trained) |
 * W1[d][NHQ_ENTRY_HIDDEN] (input-major) | b1 | W2[NHQ_ENTRY_HIDDEN][E] (hidden-major) | b2.
 * Inference (the search's seed pass, nhq_entry_forward) reads fp16 weights and
 * accumulates in f32. */
#define NHQ_ENTRY_HIDDEN 64

typedef struct nhq_search_params {
    uint64_t seed;           /* random seeds and S1 neighbour subsets derive from splitmix64(seed) */
    int32_t h;               /* two-stage routing: S1 visits ceil(R/h) neighbours; 1 = off     */
    int32_t max_iters;       /* expansion cap per query; 0 -> 1<<20                             */
    int32_t warps_per_block; /* 0 -> auto                                                      */
    int32_t hash_bits;       /* visited-filter size 2^hash_bits per query; 0 -> auto          */
    int32_t vec_dtype;       /* nhq_vec_dtype used for candidate scoring                       */
    int32_t rerank;          /* with BF16/FP8 scoring: re-score the final pool in f32          */
    int32_t seed_mode;       /* nhq_seed_mode                                                   */
    int32_t n_seeds;         /* NHQ_SEED_GIVEN: row width of `seeds`, 1..64                     */
    const uint32_t *seeds;   /* NHQ_SEED_GIVEN: [Q][n_seeds] ids (device or host), 0xFFFFFFFF
                                entries are skipped                                           */
    const float *stop_model; /* device, NHQ_MLP_PARAMS f32, or NULL: no learned stop         */
    float stop_threshold;    /* stop when sigmoid(logit) > this probability                   */
    int32_t stop_min;        /* first expansion count at which the model is consulted          */
    int32_t stop_every;      /* consult it every this many expansions (>= 1 when a model is set) */
    int32_t wildcard;        /* 1: a query code 255 places no constraint on its attribute (a
                                partial constraint; the paper's hybrid query constrains every
                                attribute): it never counts toward chi.  Under the attribute
                                seed modes such a query's completions (each open attribute
                                set to 0..its largest code among the objects, the lowest
                                attribute fastest; at most 64) give P as their runs one
                                after another, and the seed mode's rule (evenly spaced, or
                                nearest of 256 sampled) picks B from it; more completions,
                                or no member: the random stream of NHQ_SEED_RANDOM.
                                0: 255 is an ordinary code                                  */
    int32_t warps_per_query; /* 0 or 1: one warp per query; 2 or 4: that many warps share each
                                expansion's distance evaluations (rows in flight per query
                                grow with it, queries in flight per SM shrink); results are
                                the same for every value                                     */
    const float *entry_model; /* NHQ_SEED_CELL_LEARNED: device, nhq_entry_param_count(d, E) f32 */
    int32_t entry_cells;     /* NHQ_SEED_CELL_*: T, the cells taken per query, 1..min(8, E); 0 -> 2 */
    int32_t *cells_out;      /* NHQ_SEED_CELL_*: device [Q][T] receiving each query's cells, or
                                NULL                                                          */
    int32_t tile_rows;       /* rows each team of 8 lanes evaluates per distance pass: 0 or 2
                                (8 rows per warp and pass), 4 (16 rows: an expansion's
                                candidates in one pass, fewer resident warps; one warp per
                                query only); rows wider than the fixed-chunk forms always
                                take 2; results are the same on integer components, within
                                f32 rounding otherwise                                     */
} nhq_search_params;

typedef struct nhq_index nhq_index;

/* Message of the last failing call on this thread ("" if none). */
const char *nhq_last_error(void);

/* ABI version of this header (1). */
int32_t nhq_version(void);

/*
 * Object set S of Def. 1: copies vectors[N][d] (f32, row-major) into index-owned
 * HBM (rows padded to a multiple of 16 elements) and packs attributes[N][m] (u8
 * ordinal codes, Sec. 3.2) into one u32 per object: m <= 4 codes take a byte each
 * (as nhq_pack_attributes); more codes take, in order, fields of the fewest bits
 * that hold 0..c_j + 1, c_j the largest code of attribute j among the objects, so
 * that a query code above c_j (which no object has) still counts as a mismatch.
 * chi is exact either way.  `w` fixes the fusion distance (Eq. 6) used by build
 * and search.  The graph is empty until nhq_index_build / nhq_index_set_graph.
 * Errors: N < 1, d < 1, m outside 1..32, fields needing more than 32 bits in all,
 * a non-finite vector component, or w_v/w_l negative or non-finite -> NHQ_ERR_ARG.
 */
nhq_status nhq_index_create(const float *vectors, int64_t N, int32_t d, const uint8_t *attributes,
                            int32_t m, nhq_weights w, void *stream, nhq_index **out);

/* nhq_index_create for vectors of element type `dtype` (nhq_dtype): the values are
 * widened to f32 exactly, and for NHQ_F16 / NHQ_BF16 the index's f16 / bf16 scoring copy
 * (nhq_search_params::vec_dtype NHQ_VEC_F16 / NHQ_VEC_BF16) is those same values, so
 * searching with it reads rows of 2 d bytes and scores exactly as f32.
 * Errors: as nhq_index_create; dtype not an nhq_dtype. */
nhq_status nhq_index_create_typed(const void *vectors, int32_t dtype, int64_t N, int32_t d,
                                  const uint8_t *attributes, int32_t m, nhq_weights w,
                                  void *stream, nhq_index **out);

/* Releases the index and all its device memory.  NULL is a no-op. */
void nhq_free(nhq_index *index);

/* Shape of an index (any output pointer may be NULL).  R = 0 before a graph exists. */
nhq_status nhq_index_info(const nhq_index *index, int64_t *N, int32_t *d, int32_t *m, int32_t *R);

/*
 * Ordinal attribute packing (Sec. 3.2): packed[i] = sum_j attributes[i][j] << 8j for
 * n rows of m (1..4) u8 codes.  Device pointers only.
 */
nhq_status nhq_pack_attributes(const uint8_t *attributes, int64_t n, int32_t m, uint32_t *packed,
                               void *stream);

/*
 * Candidate sets C(u) of Sec. 4.1 (the paper refines random candidates by
 * NN-descent; this computes their limit, the exact K nearest): for every object
 * u, the K objects v != u with smallest (Gamma(u, v), v).  cand_ids[N][K] u32,
 * cand_dist[N][K] f32 (may be NULL).  Errors: K outside 1..256 or K >= N.
 */
nhq_status nhq_knn(const nhq_index *index, int32_t K, uint32_t *cand_ids, float *cand_dist,
                   void *stream);

/*
 * The same candidate sets with the dot products on the tensor cores: every
 * object row is rounded to bf16 (nearest even, padded with zeros to a multiple
 * of 64 dimensions) and delta^2 = |u|^2 + |v|^2 - 2 u.v is formed from the
 * rounded rows with f32 accumulation; Gamma and the (Gamma, v) order are then
 * exactly as in nhq_knn.  Rows whose components are integers 0..255 with d <= 128
 * round exactly and give nhq_knn's result bit for bit; other rows give the
 * exact candidates of their bf16 roundings.  Errors: K outside 1..64 or K >= N;
 * NHQ_ERR_CUDA if the tensor-core pipeline stalls (its waits are bounded).
 */
nhq_status nhq_knn_bf16(const nhq_index *index, int32_t K, uint32_t *cand_ids, float *cand_dist,
                        void *stream);

/*
 * Candidate sets by NN-descent (Sec. 4.3: NPG_kgraph refines random neighbour lists by
 * NN-descent instead of computing the exact K nearest): random initial lists, then
 * iterations of sampling (16 new and 16 old records per vertex plus as many reverse
 * ones), local joins (Gamma of every new x new and new x old pair of a vertex's
 * candidates, each offered to the pair's two lists through a 128-slot table per vertex
 * that keeps the best record per slot) and merges, until fewer than delta * N * K records
 * change (delta = 1e-3) or after max_iters iterations.  Graph quality against the exact
 * sets: 0.96 at N = 20,000 and 0.89-0.92 at N = 1M after 12 iterations.  Same outputs as nhq_knn (rows ascending by
 * (Gamma, id), 0xFFFFFFFF / +inf padded); every Gamma is exact, but the lists are
 * approximate (their graph quality, Eq. 7, against the exact sets is what the method
 * trades for speed) and may differ between runs, since updates race.  *iterations
 * (may be NULL) receives the number of iterations run.  Allocates its working memory
 * (about N * (9 K + 1290) bytes) for the call.
 * Errors: K outside 1..min(64, N-1), max_iters outside 1..100.
 */
nhq_status nhq_knn_nndescent(const nhq_index *index, int32_t K, int32_t max_iters, uint64_t seed,
                             uint32_t *cand_ids, float *cand_dist, int32_t *iterations,
                             void *stream);

/*
 * Landing-zone edge selection (Sec. 4.1, Def. 6) for every vertex u over the
 * candidate list cand_ids[N][L] (0xFFFFFFFF, u itself and repeats are skipped):
 * candidates are sorted by (Gamma(p, u), p); the nearest joins N(u); each next p
 * joins iff for every j already in N(u): Gamma(p, u) < Gamma(p, j) and
 * Gamma(p, u) > Gamma(u, j); stop at R.  Writes nbr_out[N][R], unused slots
 * 0xFFFFFFFF.  Errors: L outside 1..128, R outside 1..64.
 */
nhq_status nhq_edge_select(const nhq_index *index, const uint32_t *cand_ids, int32_t L, int32_t R,
                           uint32_t *nbr_out, void *stream);

/*
 * Reverse-edge candidates for a second selection pass (the paper states no
 * reverse-edge step; this is the library's reading): out[v] (width R + cap) =
 * N(v) in slot order, then the `cap` smallest ids u with v in N(u) and u not in
 * N(v), ascending; 0xFFFFFFFF pads.  nbr[N][R] as written by nhq_edge_select.
 * Errors: R outside 1..64, cap outside 0..64.
 */
nhq_status nhq_reverse_candidates(const nhq_index *index, const uint32_t *nbr, int32_t R,
                                  int32_t cap, uint32_t *out, void *stream);

/* Installs a graph nbr[N][R] (copied) as the index's composite-index adjacency. */
nhq_status nhq_index_set_graph(nhq_index *index, const uint32_t *nbr, int32_t R, void *stream);

/* Copies the index's adjacency into nbr[N][R]. */
nhq_status nhq_index_get_graph(const nhq_index *index, uint32_t *nbr, void *stream);

/*
 * Composite-index build (Sec. 5.1 with the NPG_kgraph recipe of Sec. 4.3):
 * exact candidate sets (nhq_knn, K), landing-zone selection to degree R, then
 * (params->reverse) a second selection over nhq_reverse_candidates.  params may
 * be NULL for the defaults.  Errors: as nhq_knn / nhq_edge_select.
 */
nhq_status nhq_index_build(nhq_index *index, int32_t degree, const nhq_build_params *params,
                           void *stream);

/*
 * Incremental build (NPG_nsw of Sec. 4.3), batched into insertion waves: vertex 0 alone,
 * then waves [s, e) of 1, 2, 4, ... vertices (at most wave_max).  Every vertex of a wave
 * searches the graph of [0, s) (Alg. 2 with k = ef = L from min(32, s) entry points: the
 * consecutive ids (h + j) mod s, h = splitmix64(seed ^ mix64(v))[0] mod s) and keeps a
 * landing-zone selection of the result (Def. 6, degree R); then every earlier vertex u it
 * selected re-selects from N(u) plus its new sources (ascending ids, at most rev_cap).
 * entry = 1 takes the entry points by attributes instead: the earlier vertices whose
 * attributes all equal v's, ascending, at most 32 evenly spaced (P[floor(j c / S)]), the
 * id rule when there is none (under constant weights the graph separates by tuple, and
 * the id rule rarely reaches v's own).  Every wave sees the graph as it was when the wave
 * began, so the result is deterministic.  Replaces the index's graph.
 * Errors: degree outside 1..64, L outside degree..128, degree + rev_cap > 128,
 * wave_max outside 1..65536, entry not 0 or 1.
 */
nhq_status nhq_index_build_nsw(nhq_index *index, int32_t degree, int32_t L, int32_t wave_max,
                               int32_t rev_cap, int32_t entry, uint64_t seed, void *stream);

/*
 * Entry cells (a project addition; the paper draws the seed set B of Alg. 2 at random):
 * E centroids, the objects floor(j N / E) for j < E; every object's cell is its nearest
 * centroid by (delta, j) (Eq. 1 in f32, the exact top-1 of a plain-L2 brute force over the
 * centroid rows); the objects are also ordered by (attribute word, cell, id) so that the
 * seed modes NHQ_SEED_CELL_* find a tuple's members in a cell with one binary search.
 * Replaces earlier cells.  Not saved by nhq_save.  Errors: E outside 1..min(N, 65535).
 */
nhq_status nhq_index_build_cells(nhq_index *index, int32_t E, void *stream);

/* *E (may be NULL) = the number of entry cells (0 before nhq_index_build_cells) and
 * cell_of[N] (may be NULL; device or host) = every object's cell. */
nhq_status nhq_index_cells(const nhq_index *index, int32_t *E, uint32_t *cell_of, void *stream);

/* Number of parameters of the entry model for d dimensions and E cells. */
int64_t nhq_entry_param_count(int32_t d, int32_t E);

/* Entry-model logits[n][E] of queries[n][d] with the fp16-rounded weights the search reads
 * (f32 accumulation, the seed pass's arithmetic).  Device pointers.
 * Errors: d < 1, E outside 1..65535. */
nhq_status nhq_entry_forward(const float *params, int32_t d, int32_t E, const float *queries,
                             int64_t n, float *logits, void *stream);

/* Mean softmax cross-entropy over n samples (labels in 0..E-1; other labels contribute
 * nothing) and its gradient w.r.t. the f32 parameters (grad[0], the scale's entry, is 0),
 * written to grad[nhq_entry_param_count(d, E)] and *loss.  Device pointers. */
nhq_status nhq_entry_grad(const float *params, int32_t d, int32_t E, const float *queries,
                          const int32_t *labels, int64_t n, float *grad, float *loss,
                          void *stream);

/* Trains params in place with Adam (beta1 0.9, beta2 0.999; the scale is kept) on batches
 * of `batch` consecutive samples for `epochs` passes.  Device pointers.
 * Errors: batch outside 1..65536, epochs < 0. */
nhq_status nhq_entry_train(float *params, int32_t d, int32_t E, const float *queries,
                           const int32_t *labels, int64_t n, int32_t epochs, int32_t batch,
                           float lr, void *stream);

/* Training labels: labels[q] = the cell of ids[q][0] (the first result of a search), or -1
 * where that id is 0xFFFFFFFF.  ids[n][k].  Device pointers.  Errors: no cells. */
nhq_status nhq_entry_labels(const nhq_index *index, const uint32_t *ids, int32_t k, int64_t n,
                            int32_t *labels, void *stream);

/* nhq_build for vectors of element type `dtype`: nhq_index_create_typed + nhq_index_build. */
nhq_status nhq_build_typed(const void *vectors, int32_t dtype, int64_t N, int32_t d,
                           const uint8_t *attributes, int32_t m, int32_t degree, nhq_weights w,
                           const nhq_build_params *params, void *stream, nhq_index **out);

/* build(vectors, attributes, degree, weights): nhq_index_create + nhq_index_build. */
nhq_status nhq_build(const float *vectors, int64_t N, int32_t d, const uint8_t *attributes,
                     int32_t m, int32_t degree, nhq_weights w, const nhq_build_params *params,
                     void *stream, nhq_index **out);

/*
 * Exact top-k by (Gamma, id) over all N objects (Def. 2 with Gamma in place of
 * delta).  queries[Q][d] f32, query_attributes[Q][m] u8.  `w` overrides the
 * index weights when not NULL (NHQ_W_FILTER gives the hybrid ground truth of
 * Sec. 6.1).  ids[Q][k] u32, dists[Q][k] f32, chi[Q][k] u8 (may be NULL).
 * Errors: k outside 1..256.
 */
/* nhq_brute_force with the wildcard rule of nhq_search_params::wildcard (0 or 1). */
nhq_status nhq_brute_force_wildcard(const nhq_index *index, const float *queries,
                                    const uint8_t *query_attributes, int64_t Q, int32_t k,
                                    const nhq_weights *w, int32_t wildcard, uint32_t *ids,
                                    float *dists, uint8_t *chi, void *stream);
nhq_status nhq_brute_force(const nhq_index *index, const float *queries,
                           const uint8_t *query_attributes, int64_t Q, int32_t k,
                           const nhq_weights *w, uint32_t *ids, float *dists, uint8_t *chi,
                           void *stream);

/*
 * Merge of per-shard top-k lists: the paper's parallel form (Sec. 6.1, the object set
 * split into P shards with one graph each, every shard searched for every query, the
 * results combined).  Shard p holds the objects with global ids offsets[p] + local
 * id; its list for query q is row q of the p-th [Q][k_in] block, sorted by
 * (Gamma, local id) as nhq_search and nhq_brute_force return it.  Output row q is
 * the k_out smallest records of all P rows by (Gamma, global id), ids made global;
 * shorter results are padded with 0xFFFFFFFF / +inf / chi 255.
 *   ids[P][Q][k_in] u32 (0xFFFFFFFF = none), dists[P][Q][k_in] f32,
 *   chi[P][Q][k_in] u8 (may be NULL; then out_chi must be NULL), offsets[P] u32.
 *   out_ids[Q][k_out] u32, out_dists[Q][k_out] f32, out_chi[Q][k_out] u8 (or NULL).
 * Pointers may be device or host memory (host arrays are staged; the call then
 * synchronises).  Errors: P outside 1..4096, k_in or k_out outside 1..1024, Q < 0,
 * a global id that does not fit in 32 bits is not detected (the caller's offsets
 * must keep offsets[p] + local id below 0xFFFFFFFF).
 */
nhq_status nhq_merge_topk(int32_t P, int64_t Q, int32_t k_in, int32_t k_out,
                          const uint32_t *ids, const float *dists, const uint8_t *chi,
                          const uint32_t *offsets, uint32_t *out_ids, float *out_dists,
                          uint8_t *out_chi, void *stream);

/*
 * Post-filter of a result list (the "search, then filter" strategy the paper compares
 * NHQ against, Sec. 2 and Sec. 6.2): row q of out is the first k_out records of row
 * q of the input whose chi is 0 (attributes equal to the query's), in input order;
 * shorter results are padded with 0xFFFFFFFF / +inf.
 *   ids[Q][k_in] u32 (0xFFFFFFFF = none), dists[Q][k_in] f32, chi[Q][k_in] u8,
 *   out_ids[Q][k_out] u32, out_dists[Q][k_out] f32.
 * Pointers may be device or host memory.  Errors: k_in or k_out outside 1..1024, Q < 0.
 */
nhq_status nhq_postfilter(int64_t Q, int32_t k_in, int32_t k_out, const uint32_t *ids,
                          const float *dists, const uint8_t *chi, uint32_t *out_ids,
                          float *out_dists, void *stream);

/*
 * search(queries, query_attributes, k, ef): joint pruning (Alg. 2) on the
 * composite index, ef-bounded, with the two-stage routing of Sec. 4.2 / 5.2
 * when params->h > 1.  Per query: a pool of ef records sorted by (Gamma, id);
 * repeatedly expand the nearest unexpanded record and evaluate its neighbours
 * not evaluated before; stop when every record is expanded; return the first k.
 * Seeds: params->seed_mode (nhq_seed_mode; q = row index within this call).
 * Outputs: ids/dists/chi [Q][k]; status[Q] (NHQ_OK or NHQ_ERR_ITER_LIMIT),
 * ndc[Q] (vector-distance evaluations) and expansions[Q] (expanded vertices)
 * may be NULL.  Errors: no graph, k < 1, ef < k, ef > 1024, Q < 0.  Q = 0 is a
 * no-op.
 */
nhq_status nhq_search(const nhq_index *index, const float *queries,
                      const uint8_t *query_attributes, int64_t Q, int32_t k, int32_t ef,
                      const nhq_search_params *params, uint32_t *ids, float *dists, uint8_t *chi,
                      int32_t *status, int32_t *ndc, int32_t *expansions, void *stream);

/*
 * Heterogeneous batch in one launch: query q uses k_arr[q] and ef_arr[q]
 * (device or host int32 arrays); outputs are [Q][k_max] with row q holding
 * k_arr[q] results followed by padding.  Same semantics as nhq_search per
 * query.  Errors: any k_arr[q] outside 1..k_max, ef_arr[q] outside
 * k_arr[q]..1024.
 */
nhq_status nhq_search_batched(const nhq_index *index, const float *queries,
                              const uint8_t *query_attributes, int64_t Q, const int32_t *k_arr,
                              const int32_t *ef_arr, int32_t k_max,
                              const nhq_search_params *params, uint32_t *ids, float *dists,
                              uint8_t *chi, int32_t *status, int32_t *ndc, int32_t *expansions,
                              void *stream);

/*
 * Allocation-free brute-force top-k.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they call the
 * library (their memory is owned by another allocator or pool, or their hot path
 * must not touch an allocator).  It computes the same result as nhq_brute_force
 * but takes raw arrays instead of an index and allocates nothing:
 *   vectors[N][d] f32 (d a multiple of 4, 16-byte aligned), packed_attributes[N]
 *   and packed_query_attributes[Q] (u32 words as written by nhq_pack_attributes),
 *   queries[Q][d] f32, outputs ids/dists/chi[Q][k] (dists, chi may be NULL);
 *   every pointer must be device memory.
 * Its working memory is a fixed 16 MiB array inside the library.  Device memory for
 * it is committed on each GPU when the library's code is first used there (under
 * CUDA's lazy module loading that can be this call's first use on the device) and
 * stays until the process exits.  The first call on a device also looks up the
 * array's device address.  So make one call on each device at start-up -- a call
 * with Q = 0 does only this set-up -- before the caller's own allocator reserves
 * the device's memory and before any stream capture.
 * A call whose split lists would need more than 16 MiB (about Q * 32 * k * 8
 * bytes for small batches) returns NHQ_ERR_ARG with the required size; nothing
 * is written then.  Weights follow nhq_brute_force's rules (NHQ_W_FILTER allowed).
 * Calls share the array: calls that overlap on the GPU (other streams or host
 * threads) race and must be serialised by the caller.
 */
nhq_status nhq_brute_force_noalloc(const float *vectors, const uint32_t *packed_attributes,
                                   int64_t N, int32_t d, int32_t m, const float *queries,
                                   const uint32_t *packed_query_attributes, int64_t Q, int32_t k,
                                   nhq_weights w, uint32_t *ids, float *dists, uint8_t *chi,
                                   void *stream);

/*
 * Autotuner (a project addition): times nhq_search on this batch for every launch
 * shape -- warps per query in {1, 2, 4}, rows per team and pass (tile_rows) in {2, 4},
 * warps per block in {2, 4, 8} (at least the warps per query) and visited-filter sizes
 * 2^b for b from the smallest legal size up to three above it -- with CUDA events (one
 * warm-up and three timed runs each), and writes the fastest into
 * params->warps_per_query / tile_rows / warps_per_block / hash_bits (the other fields
 * are used as given).  Every shape returns the same results on integer components
 * (tile_rows changes the f32 summation order of float rows).  *best_ms (may be NULL)
 * receives its time per call.  Device pointers; the outputs are overwritten by the
 * trial runs.
 */
nhq_status nhq_autotune_search(const nhq_index *index, const float *queries,
                               const uint8_t *query_attributes, int64_t Q, int32_t k, int32_t ef,
                               nhq_search_params *params, uint32_t *ids, float *best_ms,
                               void *stream);

/* nhq_autotune_search for a heterogeneous batch: the same launch shapes, timed on
 * nhq_search_batched with these k_arr / ef_arr (device). */
nhq_status nhq_autotune_batched(const nhq_index *index, const float *queries,
                                const uint8_t *query_attributes, int64_t Q,
                                const int32_t *k_arr, const int32_t *ef_arr, int32_t k_max,
                                nhq_search_params *params, uint32_t *ids, float *best_ms,
                                void *stream);

/*
 * Beam-width tuning (a project addition): the smallest ef of ef_list[0..n_ef)
 * (ascending, each in k..1024) whose recall against truth[Q][k] reaches `target`, then
 * the fastest launch shape for that ef (as nhq_autotune_search).  Recall of query q is
 * |ids_q & truth_q| / |truth_q| with 0xFFFFFFFF entries of truth_q not counted, averaged
 * over the queries with at least one truth entry (Eq. 3; with the filter-mode ground
 * truth of nhq_brute_force this is the hybrid recall of Sec. 6.1).  When no ef reaches
 * the target the largest is taken.  Writes *ef_out, *recall_out (may be NULL) and the
 * launch-shape fields of params; *best_ms as nhq_autotune_search.  Device pointers.
 * Errors: n_ef outside 1..64, an ef outside k..1024 or not ascending, target outside
 * (0, 1].
 */
nhq_status nhq_autotune_beam(const nhq_index *index, const float *queries,
                             const uint8_t *query_attributes, int64_t Q, int32_t k,
                             const int32_t *ef_list, int32_t n_ef, const uint32_t *truth,
                             float target, nhq_search_params *params, uint32_t *ids,
                             int32_t *ef_out, float *recall_out, float *best_ms, void *stream);

/* Mean recall of ids[Q][k] against truth[Q][k_truth] as nhq_autotune_beam computes it
 * (ids beyond the first k_truth columns are not read; k_truth <= k).  Device pointers;
 * *recall is written on the host, so the call synchronises `stream`. */
nhq_status nhq_recall(const uint32_t *ids, int32_t k, const uint32_t *truth, int32_t k_truth,
                      int64_t Q, float *recall, void *stream);

/*
 * Captured search (a project addition): records one nhq_search call (counter
 * reset, seed pre-pass, search kernel) into an instantiated CUDA graph that
 * nhq_search_graph_launch replays on any stream with the same pointers; update
 * the query buffers in place between launches.  Device pointers only; the
 * lazily built index parts (reduced-precision copies, attribute table, scratch)
 * are built by the capture call itself before capturing.  Free with
 * nhq_search_graph_free.
 */
typedef struct nhq_search_graph nhq_search_graph;
nhq_status nhq_search_graph_create(const nhq_index *index, const float *queries,
                                   const uint8_t *query_attributes, int64_t Q, int32_t k,
                                   int32_t ef, const nhq_search_params *params, uint32_t *ids,
                                   float *dists, uint8_t *chi, nhq_search_graph **out);
/* The captured form of nhq_search_batched.  k_arr / ef_arr are checked once, here, and
 * the pool is sized for the largest ef; between launches the caller may rewrite the
 * query buffers and the per-query values in place, keeping every k in 1..k_max and every
 * ef in k..(the largest ef at creation).  Device pointers only. */
nhq_status nhq_search_graph_create_batched(const nhq_index *index, const float *queries,
                                           const uint8_t *query_attributes, int64_t Q,
                                           const int32_t *k_arr, const int32_t *ef_arr,
                                           int32_t k_max, const nhq_search_params *params,
                                           uint32_t *ids, float *dists, uint8_t *chi,
                                           nhq_search_graph **out);
nhq_status nhq_search_graph_launch(nhq_search_graph *graph, void *stream);
void nhq_search_graph_free(nhq_search_graph *graph);

/*
 * Learned early stop, training data.  Runs nhq_search (params->stop_model is
 * ignored) and, at every expansion count c >= params->stop_min with
 * (c - stop_min) % stop_every == 0 while the pool holds >= k records, records the
 * model's NHQ_MLP_INPUTS features (beam statistics: expansions so far, spread of
 * the top-k, distance of the pool's last record, depth and distance of the next
 * parent, records inserted by the last expansion, expansions since the top-k last
 * changed, pool fill) into features[cap][NHQ_MLP_INPUTS], the query row into
 * query[cap], and labels[cap] = 1 if stopping there would return the same top-k
 * ids in the same order as the full search, else 0.  *n_traces receives the
 * number of records produced (records beyond cap are dropped).  Device pointers.
 */
nhq_status nhq_search_trace(const nhq_index *index, const float *queries,
                            const uint8_t *query_attributes, int64_t Q, int32_t k, int32_t ef,
                            const nhq_search_params *params, float *features, uint8_t *labels,
                            int32_t *query, int64_t cap, int64_t *n_traces, void *stream);

/* Model logits for features[n][NHQ_MLP_INPUTS] with the fp16-rounded weights the
 * search reads (f32 accumulation).  Device pointers. */
nhq_status nhq_mlp_forward(const float *params, const float *features, int64_t n, float *logits,
                           void *stream);

/* Mean binary cross-entropy with logits over n samples (labels 0/1 as f32) and its
 * gradient w.r.t. the f32 parameters, written to grad[NHQ_MLP_PARAMS] and *loss.
 * Device pointers. */
nhq_status nhq_mlp_grad(const float *params, const float *features, const float *labels,
                        int64_t n, float *grad, float *loss, void *stream);

/* Trains params in place with Adam (beta1 0.9, beta2 0.999) on batches of `batch`
 * consecutive samples for `epochs` passes.  Device pointers. */
nhq_status nhq_mlp_train(float *params, const float *features, const float *labels, int64_t n,
                         int32_t epochs, int32_t batch, float lr, void *stream);

/*
 * Index persistence: header {magic "NHQIDX01", version, N, d, m, R, weights}, in
 * version 2 followed by the attribute layout (32 field shifts, 32 field widths, u8),
 * then vectors (f32, unpadded rows), packed attributes (u32) and the graph (u32).
 * nhq_save writes version 2; nhq_load reads versions 1 (a byte per attribute) and 2.
 * Errors: unreadable/unwritable file or bad header -> NHQ_ERR_IO.
 */
nhq_status nhq_save(const nhq_index *index, const char *path);
nhq_status nhq_load(const char *path, void *stream, nhq_index **out);

#ifdef __cplusplus
}
#endif

#endif /* NHQ_H */
