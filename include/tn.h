/*
 * tn.h -- C ABI of libtn: exact inference on discrete graphical models by
 * contracting the model's factor tensors along a binary contraction tree on
 * one GB300 GPU (sm_103a).
 *
 * Method (arXiv 2405.14060, "Probabilistic Inference in the Era of Tensor
 * Networks and Differential Programming"):
 *   - a model is the tensor network (Lambda, T, {}) of its factors
 *     (Sec. "Tensor networks for probabilistic modeling", Def. "Tensor Network");
 *   - PR   p(e) = con(Lambda \ E, T_e, {})                          (Eq. pr)
 *   - MAR  p(Q_i | e) from the gradients of unity tensors 1_{Q_i} added to the
 *          network, one forward and one reverse pass                 (Sec. MAR,
 *          Thm. "Tensor network differentiation", Eq. einback)
 *   - MPE  tcon of the log-tensors in the max-plus semiring and the
 *          configuration by back-propagating Boolean masks            (Sec. MPE,
 *          Eq. log-map, Eq. tropical-back)
 *   - MMAP sum-contract groups of tensors that hold every summed
 *          variable, then MPE over the query variables                (Sec. MMAP)
 *   - sampling: backward sampling through the cached contraction tree
 *          (Sec. "Generative modeling", Eq. sample, Eq. condition-prob)
 *   - joint marginals p(Q | e) of a variable set: the contraction with Q
 *          left open                                                  (Eq. evidence)
 *
 * Conventions
 *   - Variables are 0..nvars-1 with domain sizes card[v] >= 1.
 *   - Factor tables are row-major with the LAST scope variable fastest
 *     (UAI convention), non-negative and finite.
 *   - Evidence vectors are int32 [nvars]: observed value, or -1 if free.
 *   - Logarithms are natural.
 *   - Output buffers are owned by the caller.  Functions without the _dev
 *     suffix take HOST pointers and copy through the library's stream.  The
 *     _dev variants take DEVICE pointers.  With opts->cuda_stream set they
 *     only enqueue their work on that stream (outputs are valid once the
 *     stream reaches that point; a device-side wait that gave up is reported
 *     by the next synchronous call); without it they run on the model's own
 *     stream and synchronise before returning.
 *   - No exception crosses the ABI.  Every call returns a tn_status; on
 *     failure tn_last_error() describes the cause (thread-local string, valid
 *     until the next call on the same thread).
 *   - A model is not thread-safe: calls on one tn_model must not overlap.
 */
#ifndef TN_H
#define TN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tn_model tn_model;   /* opaque, owned by the library */

typedef enum {
    TN_OK = 0,
    TN_E_ARG = 1,          /* invalid argument (also: p(e) = 0 for MAR/MAP/sample) */
    TN_E_PARSE = 2,        /* malformed UAI text */
    TN_E_ORDER = 3,        /* invalid contraction tree */
    TN_E_OOM = 4,          /* device memory or the HBM budget exhausted */
    TN_E_CUDA = 5,         /* a CUDA call failed */
    TN_E_TIMEOUT = 6,      /* a bounded device-side wait gave up */
    TN_E_UNSUPPORTED = 7   /* valid request outside what the library supports */
} tn_status;

typedef enum {
    TN_FP64 = 0,   /* every tensor and every operation in double */
    TN_FP32 = 1,   /* float tensors, FP32 CUDA-core arithmetic */
    TN_TF32 = 2,   /* float tensors; dense GEMM nodes on tcgen05 kind::tf32 */
    TN_BF16 = 3    /* float tensors; dense GEMM nodes on tcgen05 kind::f16 (bf16) */
} tn_prec;

typedef struct {
    tn_prec prec;               /* default TN_FP64 */
    int64_t hbm_budget_bytes;   /* 0 = no limit beyond the device's memory */
    int max_slices;             /* reserved (slicing is set by tn_set_order) */
    int autotune;               /* 1: on a program's first use, time a few launch shapes
                                   (graph lanes, streaming-kernel blocks per SM) and
                                   keep the fastest (cached per model and program) */
    void *cuda_stream;          /* cudaStream_t for the _dev variants; NULL = default */
} tn_options;                   /* a NULL options pointer means all defaults */

/* ------------------------------------------------------------ model */

/* Parse a UAI-format MARKOV or BAYES file (Sec. "Performance benchmarks" uses the UAI
 * competition format).  *out receives a new model (free with tn_free_model).
 * Errors: TN_E_ARG (NULL arguments, unreadable file), TN_E_PARSE. */
tn_status tn_load_model(const char *uai_path, tn_model **out);

/* Read a UAI-format evidence file for model m: either one block
 * "<nobs> v1 x1 v2 x2 ..." (one evidence set) or "<nsets>" followed by nsets
 * such blocks (the competition's multi-sample form).  Writes the first
 * min(max_sets, nsets) sets to evid[set][nvars] (-1 = unobserved, the layout
 * tn_pr / tn_mar take) and the number of sets in the file to *nsets (call
 * with max_sets = 0 to size the buffer).  Host only.  Errors: TN_E_ARG
 * (NULL arguments, unreadable file), TN_E_PARSE (malformed file, variable or
 * value out of range, a variable observed twice in one set). */
tn_status tn_read_evidence(const tn_model *m, const char *path, int max_sets, int32_t *evid,
                           int *nsets);

/* Read a UAI-format MMAP query file "<nq> v1 ... vq" for model m: writes the
 * first min(max_q, nq) query variables to query (the order tn_mmap takes)
 * and nq to *nq.  Host only.  Errors as tn_read_evidence (TN_E_PARSE also
 * for a repeated variable). */
tn_status tn_read_query(const tn_model *m, const char *path, int max_q, int32_t *query, int *nq);

/* Build a model from arrays.  Factor f has scope
 * scope_vars[scope_off[f] .. scope_off[f+1]) and its table starts at
 * tables + (sum of the sizes of factors 0..f-1).  All arrays are host
 * memory and are copied.  Errors: TN_E_ARG (bad domain size, scope variable
 * out of range or repeated, negative or non-finite table entry). */
tn_status tn_load_model_arrays(int nvars, const int *card, int nfactors,
                               const int *scope_off, const int *scope_vars,
                               const double *tables, tn_model **out);

void tn_free_model(tn_model *m);

/* ------------------------------------------------------- contraction order */

/*
 * Leaves of the contraction tree: ids 0..nfactors-1 are the factors, ids
 * nfactors..nfactors+nvars-1 are the per-variable unity/evidence vectors
 * (Sec. MAR step 1: one unity tensor per variable; an observed variable's
 * vector is the indicator of its value, which equals slicing, Eq. pr).
 * nleaves = nfactors + nvars.  Internal node i (0 <= i < nleaves-1) has id
 * nleaves + i and children left[i], right[i], which must be ids of leaves or
 * of earlier internal nodes; every id except the root is used exactly once
 * (Sec. Tensor networks, binary contraction trees).  The last node is the root.
 *
 * nnodes = 0 with left = right = NULL selects the built-in greedy order
 * (repeatedly contract the connected pair with the smallest size increase).
 * slice_vars[0..nslice) are variables fixed per slice: they are removed from
 * every tensor, the tree is contracted once per assignment of them (at most
 * 2^24 assignments) and the results are combined on the device: log-sum-exp
 * of log Z for PR, Z-weighted marginals for MAR (a sliced variable's
 * marginal is the Z-share of its values).  Slicing bounds the largest
 * intermediate by the product of the sliced domains; sampling draws the
 * assignment of the sliced variables first (probability Z_a / Z, a second
 * forward pass per drawn assignment); MPE and MMAP reject a sliced tree
 * (TN_E_UNSUPPORTED).  tn_tree_stats then reports the
 * per-slice space complexity and the total time over all slices.
 * Errors: TN_E_ORDER (a malformed tree), TN_E_ARG (bad slice variables).
 */
tn_status tn_set_order(tn_model *m, int nnodes, const int *left, const int *right,
                       int nslice, const int *slice_vars);

/* Build a tree from a variable elimination order (a permutation of a subset
 * of 0..nvars-1; variables not listed are eliminated last in id order): the
 * tensors holding each variable are merged smallest-first and the variable
 * is summed at the last merge.  Writes nleaves-1 entries to left/right. */
tn_status tn_tree_from_elimination(const tn_model *m, int nelim, const int *order,
                                   int *left, int *right);

/* Search a contraction tree: method 0 = greedy (as tn_set_order's default),
 * 1 = randomised min-fill / min-degree elimination with `restarts` restarts
 * keeping the tree of least time complexity whose space complexity is
 * minimal, 2 = method 1 followed by `restarts` rounds of simulated annealing
 * over local rotations of the tree (objective: log2 of the total
 * multiply-add count plus a penalty on space complexity above the best seen
 * minus one), in the spirit of the tree-annealing finders the paper cites for
 * its orders (Sec. Tensor networks); 3 = recursive bisection of the tensor
 * hypergraph (one vertex per tensor, one hyperedge per variable weighted by
 * log2 of its domain; Fiduccia-Mattheyses passes from max(4, restarts)
 * random balanced starts per split), kept when it beats method 1's tree,
 * followed by the annealing of method 2; 4 = the better of methods 1 and 3's
 * starting trees, then `restarts` rounds of the same annealing evaluated
 * incrementally (a rotation changes the labels of one node and the costs of
 * two, so each round affords 2000 rotations per leaf).
 * Host only; deterministic for a seed.
 * Writes nleaves-1 entries to left/right. */
tn_status tn_optimize_order(const tn_model *m, int method, int restarts, uint64_t seed,
                            int *left, int *right);

/* Equivalent tree with runs of absorption steps re-associated.  The
 * contraction is associative (Sec. Tensor networks: every binary tree gives
 * the same result; only the cost changes), so a run of steps in which a large
 * tensor absorbs small ones one at a time, Y_i = con(Y_(i-1), W_i), is
 * rewritten as V = con(W_1, ..., W_k) followed by one step Y_k = con(Y_0, V):
 * the large tensor is read and written once per run instead of once per
 * step.  Runs are chosen per chain by dynamic programming over a time model
 * of the streaming kernels (bytes, FLOPs, a fixed cost per launch).  Input:
 * a tree in tn_set_order's form (nleaves-1 entries each); output: the new
 * tree, post-ordered, in left_out/right_out (nleaves-1 entries each; may
 * alias neither input).  Host only.  TN_E_ORDER if the input is not a valid
 * tree.  The result is unchanged where no run pays off. */
tn_status tn_reassociate(const tn_model *m, const int *left, const int *right,
                         int *left_out, int *right_out);

/* Slice variables for a tree (left/right as tn_set_order's; NULL: the current
 * tree): greedily adds the label of the current largest intermediate whose
 * slicing gives the smallest space complexity (ties: the smallest total
 * multiply-add count over all slices) until the per-slice space complexity
 * is at most target_sc_log2 (log2 entries) or max_vars variables are chosen
 * (slicing, Sec. Tensor networks: fixing a label splits the contraction into
 * independent ones, one per value).  Writes at most max_vars variables to
 * vars and their count to *nvars_out; pass them to tn_set_order.  Host only.
 * Errors: TN_E_ARG (NULL outputs), TN_E_ORDER (an invalid tree). */
tn_status tn_choose_slices(const tn_model *m, const int *left, const int *right,
                           double target_sc_log2, int max_vars, int *vars, int *nvars_out);

/* Complexities of the current tree for `batch` evidence sets:
 * out[0] = log2 of the total multiply-add count (time complexity, paper:
 * product over the union of the labels of each pairwise contraction),
 * out[1] = log2 of the largest intermediate's entry count (space complexity),
 * out[2] = log2 of the total entries read and written (read-write complexity),
 * out[3] = number of internal nodes, out[4] = forward FLOPs (2 per multiply-add),
 * out[5] = forward algorithmic bytes at the given precision. */
tn_status tn_tree_stats(const tn_model *m, int batch, tn_prec prec, double *out);

/* ------------------------------------------------------------- tasks */

/* PR: logz[b] = log p(e_b) for each of `batch` evidence sets evid[b][nvars]
 * (Eq. pr).  log p(e) = -inf when the evidence is impossible.  The evidence
 * sets run as one batched contraction (a batch label on every unity vector);
 * when that does not fit the device memory or opts->hbm_budget_bytes, they
 * run in the largest power-of-two sub-batches that do (same for tn_mar). */
tn_status tn_pr(tn_model *m, int batch, const int32_t *evid, const tn_options *opts,
                double *logz);

/* MAR: logz as tn_pr, and marg[b][sum card] = p(v = x | e_b) for every
 * variable (an observed variable gets the indicator of its value).  One
 * forward and one reverse (adjoint) pass over the tree (Sec. MAR).  The
 * reverse pass reads the forward intermediates; when keeping all of them
 * does not fit the device memory or opts->hbm_budget_bytes even for one
 * evidence set, the largest ones (never a parent and its child) are not
 * kept: the reverse pass recomputes each from its kept operands just before
 * it is read (checkpointing; the extra work shows as class 8 of tn_profile).
 * Errors: TN_E_ARG when some p(e_b) = 0; TN_E_OOM when even that does not
 * fit. */
tn_status tn_mar(tn_model *m, int batch, const int32_t *evid, const tn_options *opts,
                 double *logz, double *marg);

/* Joint marginal of a set of variables Q = query[0..nq) (distinct, observed
 * ones allowed): joint[q] = p(Q = q | e) over the joint domain of Q, row-major
 * with the last query variable fastest (prod of their domain sizes entries,
 * at most 65536), and logz = log p(e).  p(Q, e) is the contraction of the
 * network with Q left open (Eq. evidence); the query labels are sliced and
 * each slice -- the evidence extended by Q = q, a PR of Eq. pr -- is one row
 * of a single batched contraction along the model's tree (sub-batched under
 * the memory budget as tn_pr).  Assignments that contradict an observed
 * query variable get 0 without being run.  In reduced precision the error
 * of joint[q] follows the per-row log Z error.
 * Errors: TN_E_ARG for a bad or repeated query variable, a joint domain
 * above 65536 assignments, or p(e) = 0. */
tn_status tn_joint_mar(tn_model *m, const int32_t *evid, int nq, const int32_t *query,
                       const tn_options *opts, double *logz, double *joint);

/* MPE: assign[nvars] maximises prod_f T_f given the evidence (observed
 * variables keep their value); logp = log of that maximum (Eq. log-map).
 * Ties go to the lowest flat index at each contraction.
 * Errors: TN_E_ARG when p(e) = 0. */
tn_status tn_map(tn_model *m, const int32_t *evid, const tn_options *opts,
                 int32_t *assign, double *logp);

/* MMAP: assign[nq] maximises sum_m p(q, m, e) over the query variables
 * query[0..nq); logp = log of that maximum (Eq. mmap), by the two-phase
 * method of Sec. MMAP (sum-contract groups, then max-plus over the query).
 * The summed phase runs in FP64 when prec = TN_FP64, else in FP32 with
 * power-of-two rescaling; the max-plus phase runs in FP64 / FP32 likewise.
 * The model keeps the programs of its last call: a call with the same query
 * set, the same observed variables and the same precision only replays them
 * with the new evidence values.
 * Errors: TN_E_ARG (query overlaps evidence, p(e) = 0), TN_E_OOM. */
tn_status tn_mmap(tn_model *m, const int32_t *evid, int nq, const int32_t *query,
                  const tn_options *opts, int32_t *assign, double *logp);

/* Sampling: n exact samples of all variables from p(Lambda \ E | e) by
 * backward sampling through the contraction tree (Sec. Generative modeling,
 * Eq. condition-prob).  samples[n][nvars] (observed variables keep their
 * value; domain sizes must be <= 127).  Random numbers: Philox4x32-10
 * keyed by `seed`, one counter per (sample, node).
 * Errors: TN_E_ARG when p(e) = 0. */
tn_status tn_sample(tn_model *m, const int32_t *evid, uint64_t seed, int64_t n,
                    const tn_options *opts, int8_t *samples);

/* Device-pointer variants.  evid, logz, marg, factor_tables and grad live in
 * device memory.  If factor_tables is non-NULL it replaces the model's
 * tables for this call and later calls (same layout as tn_load_model_arrays,
 * double); with tables_are_log != 0 its entries are the natural logarithms
 * of the tables (exponentiated when the leaves are built).  The model's own
 * tables come back on the next call without factor_tables.
 * tn_mar_dev additionally writes, if grad is non-NULL, grad[b][sum of
 * factor table sizes] = d log p(e_b) / d log T_f[x] = the factor marginal
 * p(scope_f = x | e_b) (Thm. "Tensor network differentiation" applied to
 * each factor). */
tn_status tn_pr_dev(tn_model *m, int batch, const int32_t *evid,
                    const double *factor_tables, int tables_are_log,
                    const tn_options *opts, double *logz);
tn_status tn_mar_dev(tn_model *m, int batch, const int32_t *evid,
                     const double *factor_tables, int tables_are_log,
                     const tn_options *opts, double *logz, double *marg, double *grad);

/* Facts about the program that tn_pr (task 0) or tn_mar (task 1) runs for
 * `batch` evidence sets with these options (it is built, autotuned when
 * opts->autotune is set, and cached, as a task call would).  out[8]:
 *   0 bytes of its tensor arena, 1 bytes that arena takes when every forward
 *   tensor is kept, 2 forward tensors the MAR reverse pass recomputes
 *   (checkpointing), 3 kernel launches per pass, 4 streams (lanes) of its
 *   captured graph, 5 blocks per SM of the streaming absorb kernels (0: the
 *   default), 6 1 if the launch shapes were chosen by the autotuner, 7 the
 *   evidence sets per pass (the sub-batch that fits the memory). */
tn_status tn_program_stats(tn_model *m, int task, int batch, const tn_options *opts,
                           double *out);

/* PR (task 0) or PR + MAR (task 1) for several models in one graph launch:
 * each model's program (built and cached as tn_pr / tn_mar would, for
 * batch[i] evidence sets evid[i] in tn_pr's layout, NULL = no evidence)
 * becomes a branch of one CUDA graph, so models of uneven treewidth run
 * concurrently on the device, behind a single launch on opts->cuda_stream
 * (else the first model's stream).  Results as tn_pr / tn_mar, into host
 * buffers logz[i][batch[i]] and, for task 1, marg[i][batch[i]][sum card].
 * The models must be distinct, on one device, unsliced, and each batch
 * must fit the device memory at once (no sub-batching).  Errors as tn_mar;
 * TN_E_UNSUPPORTED for a sliced model. */
tn_status tn_solve_multi(int task, int nmodels, tn_model *const *models, const int *batch,
                         const int32_t *const *evid, const tn_options *opts,
                         double *const *logz, double *const *marg);

/* Device-side duration of the last task's kernels in milliseconds
 * (CUDA events around the launch on the task's stream). */
double tn_last_device_ms(const tn_model *m);

/* Number of kernel launches the last task issued (graph nodes counted). */
int64_t tn_last_launch_count(const tn_model *m);

/* Profile one PR (task 0) or PR + MAR (task 1) pass kernel by kernel (each
 * launch timed with CUDA events on the model's stream, outside any graph),
 * averaged over `reps` passes.  out[9][4] per kernel class: milliseconds,
 * launches, algorithmic FLOPs (2 per multiply-add of a contraction) and
 * algorithmic bytes (operands and result once).  Classes: 0 leaves and
 * finalisation (not timed, reported as 0), 1 streaming absorb, 2 streaming
 * reduction (or split-K), 3 tcgen05 GEMM, 4 CUDA-core GEMM, 5 operand
 * preparation / scatter, 6 generic strided contraction, 7 batched strided
 * GEMM, 8 recomputation: forward steps that a checkpointed MAR program
 * re-runs in its backward pass (their FLOPs and bytes are extra work, not
 * part of the algorithmic count of the other classes). */
tn_status tn_profile(tn_model *m, int task, int batch, const int32_t *evid,
                     const tn_options *opts, int reps, double *out);

/* Like tn_profile for one pass, but per launch in launch order:
 * steps[i][4] = class, milliseconds, algorithmic FLOPs, algorithmic bytes
 * for i < min(cap, *nsteps); *nsteps receives the number of launches. */
tn_status tn_profile_steps(tn_model *m, int task, int batch, const int32_t *evid,
                           const tn_options *opts, int cap, double *steps, int *nsteps);

const char *tn_last_error(void);

/* ---------------------------------------------------- pairwise contraction */

/*
 * One pairwise contraction con({A, B} -> C) (Def. "Tensor Network",
 * Eq. contraction-definition) on device buffers, with the labels of each
 * operand given as small integers (storage order, last fastest) and
 * sizes[label] the dimension of each label (labels 0..nlabels-1).
 *   semiring 0: C = sum over the labels not in C of A * B
 *   semiring 1: C = max over those labels of A + B (Eq. tropical), and if
 *               argmax is non-NULL, argmax[c] = the flat index (first
 *               eliminated label slowest, in the order: labels of A not in
 *               C in A's order, then labels of B in neither A nor C in B's
 *               order) of the first maximising assignment.
 * dtype: 0 = double, 1 = float.  A sum-product contraction whose row, column
 * and summed label groups each hold at least 64 entries (and with no label
 * summed inside one operand alone) runs as a batched GEMM: TN_TF32 / TN_BF16
 * on tcgen05 tensor cores (float data only), TN_FP32 / TN_FP64 on a CUDA-core
 * tiled GEMM; other sum-product contractions with no label summed inside one
 * operand run on a batched strided GEMM over the label groups (CUDA cores,
 * operands read in place through per-group offset tables); everything else
 * runs on the strided contraction kernels.  No
 * rescaling is applied.  The call allocates its scratch memory (operand
 * workspaces, split-K partial sums) stream-ordered from the CUDA memory pool
 * and synchronises `cuda_stream` before returning.
 */
tn_status tn_contract_dev(int nlabels, const int *sizes,
                          int na, const int *labels_a, const void *A,
                          int nb, const int *labels_b, const void *B,
                          int nc, const int *labels_c, void *C,
                          int semiring, int dtype, tn_prec prec, int32_t *argmax,
                          void *cuda_stream);

/* ------------------------------------------------ allocation-free variant */

/* Size of the fixed device scratch used by tn_contract_dev_noalloc. */
#define TN_NOALLOC_SCRATCH_BYTES (8u << 20)

/*
 * The same pairwise contraction as tn_contract_dev (same arguments, same
 * results up to floating-point summation order), on the strided contraction
 * kernels (split over the summed space where it is long, one pass per output
 * entry otherwise), without allocating any device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot let a library
 * allocate GPU memory -- an application that owns all device memory through
 * its own pool, or a latency-critical loop where cudaMalloc / cudaFree, which
 * may synchronise the device, are not acceptable.
 *
 * The split-K partial sums live in one file-scope device array of
 * TN_NOALLOC_SCRATCH_BYTES bytes that every GPU loading the library holds
 * until the process exits.  An output of more than TN_NOALLOC_SCRATCH_BYTES /
 * (element size + 4) entries is rejected with TN_E_ARG and a message naming
 * the limit; nothing is launched then.
 *
 * The first call on each device looks up the array's device address (once,
 * with that device current), so make the first call on a device before any
 * stream capture.  All calls in the process share the array and it keeps the
 * last call's contents (no part of it needs to start at zero: a call reads
 * only partials it wrote itself).  Calls whose kernels can overlap on the GPU
 * -- on different streams without ordering, or from several host threads --
 * race on the array and must be serialised by the caller.  The call
 * synchronises `cuda_stream` before returning.  prec is not taken: the
 * contraction kernels compute in the data type (dtype 0 double, 1 float).
 */
tn_status tn_contract_dev_noalloc(int nlabels, const int *sizes,
                                  int na, const int *labels_a, const void *A,
                                  int nb, const int *labels_b, const void *B,
                                  int nc, const int *labels_c, void *C,
                                  int semiring, int dtype, int32_t *argmax,
                                  void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* TN_H */
