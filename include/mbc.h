/* mbc.h - C ABI of libmbc: multi-baryon two-point correlators on GB300 (sm_103a).
 *
 * Computes the correlator of arXiv 2201.04269, Eq. 1,
 *
 *     C = sum_{(a, a') in I} W^{a}_{a'} <q(a_1)...q(a_n) qbar(a'_1)...qbar(a'_n)>,
 *
 * for quark-only operators with n_u up and n_d down quarks, with every quark at one
 * sink site x and every antiquark at one source point, summed over the sink sites of
 * each time slice (zero momentum).  The quark-level Wick contraction is evaluated in
 * its determinant form (Sec. 1): after the caller has written the slots of every term
 * in flavour-grouped order (all up slots, then all down slots) and folded the
 * reordering signs into the weights,
 *
 *     C_x(t) = scale * sum_{(a, a') in I} W(a, a') det U_x[a_u, a'_u] det D_x[a_d, a'_d],
 *
 * with scale carrying (-1)^{n(n-1)/2} and any normalisation.  Three algorithms:
 * the direct index-set sweep (MBC_ALGO_DIRECT), factor trees (Sec. 4,
 * MBC_ALGO_TREE) and a plan extracted from a tensor e-graph (Sec. 5, MBC_ALGO_EGRAPH);
 * three arithmetics: complex double (MBC_PREC_FP64), complex FP32 pairs with
 * compensated products and double accumulation (MBC_PREC_MIXED, "double-float"), and
 * complex FP32 with compensated sums and a per-site error guard (MBC_PREC_FP32, e-graph
 * plans only; see mbc_plan_set_guard).
 *
 * Conventions for every call:
 *  - Spin-colour index i = 3 * spin + colour in 0..11.  A propagator field is a device
 *    array of complex double (interleaved re, im), layout [set][t][site][12][12],
 *    row = sink index, column = source index; it is owned by the caller.
 *  - Calls never throw; they return an mbc_status.  Failed calls leave outputs
 *    unchanged and record a message readable through mbc_last_error(ctx).
 *  - Device work is enqueued on the caller's stream and is asynchronous.  No call
 *    synchronises the device except where stated.
 *  - A plan is immutable after creation.  The evaluation calls of one context share
 *    its scratch pool (per-site partial sums, per-block K slots, the work counter, the
 *    block buffers), so their device work must not overlap: issue them on one stream,
 *    or give each stream its own context (and plans).  A context is used by one host
 *    thread at a time.
 */
#ifndef MBC_H
#define MBC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* mbc_stream;   /* a cudaStream_t; NULL = the legacy default stream */

typedef enum {
    MBC_OK = 0,
    MBC_INVALID_ARG = 1,   /* null pointer, negative size, inconsistent offsets, bad enum */
    MBC_UNSUPPORTED = 2,   /* n_u or n_d outside 0..6, index outside 0..11, algorithm not
                              available for this kind of plan */
    MBC_OOM = 3,           /* host or device allocation failed */
    MBC_CUDA = 4,          /* a CUDA runtime call failed (message names it) */
    MBC_TIMEOUT = 5,       /* a bounded device wait gave up */
    MBC_NUMERIC = 6,       /* non-finite input or result */
    MBC_IO = 7             /* plan file missing, truncated or of another version */
} mbc_status;

typedef enum { MBC_ALGO_DIRECT = 0, MBC_ALGO_TREE = 1, MBC_ALGO_EGRAPH = 2 } mbc_algo;
typedef enum { MBC_PREC_FP64 = 0, MBC_PREC_MIXED = 1, MBC_PREC_FP32 = 2 } mbc_prec;

typedef struct mbc_ctx mbc_ctx;
typedef struct mbc_plan mbc_plan;

/* ------------------------------------------------------------------------------------
 * Context.  mbc_create binds a context to a CUDA device; the context owns its plans'
 * device memory.  device = -1 makes a host-only context: plans are built and can be
 * inspected, saved and loaded, but evaluation calls return MBC_UNSUPPORTED (no CUDA
 * call is made).  mbc_destroy frees everything the context owns (plans included).
 * ---------------------------------------------------------------------------------- */
mbc_status mbc_create(mbc_ctx** ctx, int device);
void mbc_destroy(mbc_ctx* ctx);
/* Message of the last failed call on this context (never NULL; "" if none).  The
 * string is owned by the context and valid until its next call. */
const char* mbc_last_error(const mbc_ctx* ctx);
/* Library version, e.g. "mbc 1.0". */
const char* mbc_version(void);

/* ------------------------------------------------------------------------------------
 * Operator library: the baryon and multi-baryon operators of Sec. 1 and Eq. 2
 * (proton, neutron, D_I, D_II, 3He_I, 3He_II) expanded into sink terms.
 *
 * Each operator is expanded into ordered products of quark fields; each product is
 * written in flavour-grouped slot order with the sign of that Grassmann reordering
 * folded into its weight; identical slot tuples are merged.  Weights are returned
 * unnormalised (Gaussian integers, so merging is exact); *scale receives
 * (-1)^{n(n-1)/2} |norm|^2 for the correlator of the operator with itself.  Readings
 * where the paper is silent: Dirac basis with C = gamma_4 gamma_2; the free spin index
 * (proton, neutron, 3He) is projected with P_+ = (1 + gamma_4)/2 and traced; the
 * source uses the conjugated sink weights.  MBC_OP_HE3_II_S is a stand-in for 3He_II
 * (its printed terms 1, 2, 5 with normalisation 2/sqrt(6)), because the printed D_II
 * and 3He_II vanish identically.
 *
 * Call with idx == NULL to query sizes: *n_terms receives the total term count.
 * Otherwise idx must hold n_terms * (n_u + n_d) bytes, w 2 * n_terms doubles,
 * offsets n_free + 1 entries (terms of free index j are offsets[j]..offsets[j+1]-1),
 * proj 2 * n_free * n_free doubles (row-major complex P_jj').
 * ---------------------------------------------------------------------------------- */
typedef enum {
    MBC_OP_PROTON = 0, MBC_OP_NEUTRON = 1, MBC_OP_DINUCLEON_I = 2, MBC_OP_DINUCLEON_II = 3,
    MBC_OP_HE3_I = 4, MBC_OP_HE3_II = 5, MBC_OP_HE3_II_S = 6
} mbc_operator;

mbc_status mbc_operator_terms(int op, int* n_u, int* n_d, int* n_free, int64_t* n_terms,
                              int8_t* idx, double* w, int64_t* offsets, double* proj, double* scale);

/* ------------------------------------------------------------------------------------
 * Plans.
 *
 * mbc_plan_create: a factored weight (Eq. 1 with W factorised over sink and source)
 *     W(a, a') = sum_{j, j'} P_jj' s_j(a) conj(r_j'(a')),
 * j, j' in 0..n_free-1.  snk_idx [n_snk][n_u + n_d] int8 slot indices (flavour
 * grouped), snk_w [n_snk] complex double, snk_off [n_free + 1]; the same for the
 * source; proj [n_free][n_free] complex double; scale a complex double multiplying C
 * (pass {(-1)^{n(n-1)/2}, 0} for the plain Wick sign).  All pointers are host memory,
 * read during the call only.
 *
 * The planner (host, once per plan; Sec. 3-5) canonicalises every term (ascending
 * slot sets per flavour with the sorting sign, repeated indices dropped: the
 * Index-List pruning), merges multiplicities, builds the linearised factor tree and
 * runs the minor e-graph, then uploads what the chosen algorithm needs to the device.
 *
 * mbc_plan_from_terms: explicit index set, term t = (a_t, a'_t, W_t) with
 * a = sink[t][n_u + n_d], a' = source[t][n_u + n_d], W [n_terms] complex double.
 * Supports MBC_ALGO_DIRECT and MBC_ALGO_TREE (MBC_UNSUPPORTED otherwise).
 * ---------------------------------------------------------------------------------- */
typedef struct {
    int n_u, n_d, n_free;
    const int8_t* snk_idx; const double* snk_w; const int64_t* snk_off;
    const int8_t* src_idx; const double* src_w; const int64_t* src_off;
    const double* proj;
    double scale[2];
} mbc_problem;

mbc_status mbc_plan_create(mbc_ctx* ctx, const mbc_problem* problem, int algo, int prec, mbc_plan** out);
mbc_status mbc_plan_from_terms(mbc_ctx* ctx, int n_u, int n_d, int64_t n_terms,
                               const int8_t* sink, const int8_t* source, const double* W,
                               const double* scale, int algo, int prec, mbc_plan** out);
void mbc_plan_destroy(mbc_plan* plan);

/* Plan statistics (host values): */
typedef struct {
    int n_u, n_d, algo, prec;
    int64_t index_size;          /* |I|: (sink, source) term pairs of the direct sweep */
    int64_t canonical_terms;     /* merged canonical (R_u, R_d, C_u, C_d) terms (tree leaves) */
    int64_t rows_u, rows_d, cols_u, cols_d;   /* distinct ascending slot sets */
    int64_t minors_u, minors_d;  /* distinct minors the canonical form needs */
    int64_t tree_nodes;          /* vertices of the linearised factor tree (root included) */
    int64_t egraph_classes, egraph_nodes;     /* saturated minor e-graph size */
    double flops_per_site;       /* algorithmic flops of this plan's algorithm, per site */
    double direct_flops_per_site;/* the direct sweep's flops, per site (for comparison) */
    int64_t scratch_bytes_per_site; /* device scratch the algorithm uses per in-flight site */
} mbc_plan_info;
mbc_status mbc_plan_get_info(const mbc_plan* plan, mbc_plan_info* info);

/* Linearised factor tree of the plan (Sec. 4, Fig. 5): factors[n_nodes] (factors[0]
 * is the root and is -1; up minor m is m, down minor m is minors_u + m), children
 * [n_nodes], coefficients [n_leaves] complex double (scale not applied).  Pass NULL
 * arrays to query n_nodes / n_leaves.  Minor m of flavour f is (rows, cols) given by
 * mbc_plan_get_minor. */
mbc_status mbc_plan_get_tree(const mbc_plan* plan, int64_t* n_nodes, int64_t* n_leaves,
                             int32_t* factors, int32_t* children, double* coefficients);
mbc_status mbc_plan_get_minor(const mbc_plan* plan, int flavour, int64_t m, int8_t* rows, int8_t* cols);

/* Serialise a plan (problem, canonical lists, tree, e-graph plan) to a versioned file,
 * and load it back (the planner is not re-run). */
mbc_status mbc_plan_save(const mbc_plan* plan, const char* path);
mbc_status mbc_plan_load(mbc_ctx* ctx, const char* path, mbc_plan** out);

/* ------------------------------------------------------------------------------------
 * Evaluation.
 *
 * mbc_correlator: C[s][t] = scale * sum_{x < V3} C_x(s, t) for every set s < n_sets and
 * time slice t < T.  U, D: device pointers, complex double [n_sets][T][V3][12][12]
 * (caller-owned).  C: device pointer, complex double [n_sets][T] (written, not
 * accumulated).  site_out: optional device pointer, complex double [n_sets][T][V3]
 * receiving scale * C_x per site, or NULL.  The site sum is taken in double with
 * compensated (TwoSum) accumulation in a fixed order, so results are bit-reproducible
 * for a given plan, sizes and device.  Temporary device memory is taken from the
 * context's pool (grown on demand with cudaMalloc outside any stream capture).
 * ---------------------------------------------------------------------------------- */
mbc_status mbc_correlator(mbc_plan* plan, const void* U, const void* D, int n_sets, int T, int64_t V3,
                          void* C, void* site_out, mbc_stream stream);

/* Nonzero sink momentum (the e^{-i p.x} projection of Sec. 2): as mbc_correlator on an
 * L^3 lattice (V3 = L^3), with C[s][t] = scale * sum_x e^{-i 2 pi p.x / L} C_x(s, t) and
 * site x of a slice at (x mod L, (x / L) mod L, x / L^2); p: three integers (host
 * memory), NULL for zero momentum; site_out (optional) receives the site values without
 * the phase. */
mbc_status mbc_correlator_momentum(mbc_plan* plan, const void* U, const void* D, int n_sets, int T, int L,
                                   const int* p, void* C, void* site_out, mbc_stream stream);

/* End to end from host memory: copies U, D (host, pinned or pageable, same layout) to
 * the context's device buffers, evaluates, copies C back to host memory C_host, on
 * the given stream, and synchronises that stream before returning.  Large calls are
 * split into up to 8 chunks of whole time slices: the copy of a chunk runs on a second
 * stream of the context while the previous chunk is evaluated on the given one (pinned
 * host memory lets the copies overlap); the results equal a single evaluation. */
mbc_status mbc_correlator_host(mbc_plan* plan, const void* U_host, const void* D_host, int n_sets, int T,
                               int64_t V3, void* C_host, mbc_stream stream);

/* Batched evaluation: several (plan, fields, output) items -- different operators,
 * propagator sets and lattice sizes -- in one persistent launch per precision, load
 * balanced over (item, site) work units by an atomic counter (no inter-block waiting),
 * followed by one small site-sum launch per item.  Items must use MBC_ALGO_EGRAPH plans
 * of this context.  mbc_batch_reserve sizes the device buffers and uploads the item
 * table (synchronously); mbc_batch with the same item array (same plans, pointers and
 * sizes) then allocates nothing and can be captured in a CUDA graph.  Called with other
 * items outside a capture, mbc_batch reserves them first; inside a capture it fails
 * with MBC_OOM.  MBC_PREC_FP32 items run as one FP32 launch over all their units (with
 * the largest walker count and cluster size among them; items of fewer leave warps or
 * blocks idle), one slice-guard launch and one double-float launch over the units the
 * guards list; a plan whose guard settings or kernel shape changed since the
 * reservation is reserved again (MBC_OOM inside a capture, as above). */
typedef struct {
    mbc_plan* plan;
    const void* U;
    const void* D;
    int n_sets, T;
    int64_t V3;
    void* C;                    /* device complex double [n_sets][T] */
    void* site_out;             /* optional device complex double [n_sets][T][V3]: per-site
                                   values (as mbc_correlator's site_out), or NULL */
} mbc_work;
mbc_status mbc_batch_reserve(mbc_ctx* ctx, const mbc_work* items, int n_items);
mbc_status mbc_batch(mbc_ctx* ctx, const mbc_work* items, int n_items, mbc_stream stream);

/* ------------------------------------------------------------------------------------
 * The FP32 arithmetic of e-graph plans (MBC_PREC_FP32).
 *
 * The minors (Laplace steps of the extracted column trees, Sec. 5), the G stage and the
 * pair products run in complex FP32 on each site's propagators scaled by exact powers
 * of two; every thread sums its parts with TwoSum compensation and the site sum is a
 * compensated double sum.  FP32 rounding (2^-24 per operation) reaches the results
 * amplified by cancellation (the floating-point problem cited in Sec. 1): within a
 * site's sum, and across the sites of a time slice in C(t).  Two guards decide which
 * sites the double-float kernel (the arithmetic of MBC_PREC_MIXED) recomputes, in a
 * second launch on the same stream before the site sum:
 *  - per site (only when per-site values are returned, site_out != NULL): with
 *        s_x = sqrt(sum over the site's (A leaf, B row set) parts of |part|^2),
 *    a site with s_x / |C_x| > site_threshold (or a non-finite value) is recomputed.
 *    The FP32 error of a site measured about 1e-7 x s_x (median); the default
 *    threshold 2 (about a quarter of the He-3 sites recomputed) kept every per-site
 *    error of a 97k-site sample below 1e-6.  +inf recomputes no site, <= 0 every site.
 *  - per time slice (always): the error of C(t) from the FP32 sites is estimated as
 *    2.5e-7 x sqrt(sum_x s_x^2) (independent rounding errors), and when that exceeds
 *    slice_tolerance x |C(t)| (with the sink momentum phase, if any) the slice's FP32
 *    sites of largest s_x are recomputed: those above the largest threshold for which
 *    the sites left in FP32 estimate at most half the tolerance.  Default 1e-6; +inf
 *    switches it off.
 *
 * mbc_plan_set_guard / mbc_plan_get_guard: the plan's site threshold and slice tolerance
 * (host calls, effective for evaluations issued afterwards).  mbc_fp32_recomputed: the
 * number of sites that the last MBC_PREC_FP32 evaluation of this context recomputed
 * (synchronises the device; 0 if none ran; after a chunked mbc_correlator_host, its
 * last chunk's).  Results are bit-reproducible for a given
 * plan, guards, sizes and device.
 * ---------------------------------------------------------------------------------- */
mbc_status mbc_plan_set_guard(mbc_plan* plan, double site_threshold, double slice_tolerance);
mbc_status mbc_plan_get_guard(const mbc_plan* plan, double* site_threshold, double* slice_tolerance);
mbc_status mbc_fp32_recomputed(mbc_ctx* ctx, int64_t* n_sites);

/* ------------------------------------------------------------------------------------
 * Tensor e-graph (Sec. 5) of a tensor-network expression: the e-graph (U, M, H) of the
 * expression's splits E -> sigma -> E1 E2 under the two restrictions of Sec. 5 (each part
 * contracts an index internally; one part holds a tensor whose indices are all contracted
 * in E), saturated up to node_limit e-nodes, extracted by the objective of Sec. 5 (the
 * children's excess parents from distinct e-classes times their flops, ties to the
 * smaller cost).  Canonical forms rename summed labels s0, s1, ... and open labels o0,
 * o1, ... over every factor order and every slot order of the antisymmetric tensors.
 *
 * expression: "name(i,j,k) name(l,m) ..." (host string; a label used twice is summed, none
 * more than twice; 1 to 8 tensors); antisymmetric: names of antisymmetric tensors,
 * space separated (or NULL); dim: index range for the flop counts.  plan (host buffer of
 * plan_len bytes, or NULL to query *plan_needed) receives the extracted plan as text: a
 * first line "root <id> sign <+1|-1>" (the expression equals that sign times the root
 * class's canonical form), then one line per e-class reached from the root:
 *     class <id> <canonical form> cost <flops> : leaf
 *     class <id> <canonical form> cost <flops> : prod <id1> [labels] <id2> [labels] sign <+1|-1>
 * (labels: the class's canonical labels of the two children's open slots; sign: the
 * relative sign of the children's canonicalisations).  *n_classes, *n_enodes: the
 * saturated e-graph's size.  Host-only; works on a device -1 context.
 * ---------------------------------------------------------------------------------- */
mbc_status mbc_tensor_egraph(mbc_ctx* ctx, const char* expression, const char* antisymmetric, int64_t node_limit,
                             int dim, char* plan, int64_t plan_len, int64_t* plan_needed, int64_t* n_classes,
                             int64_t* n_enodes);

/* ------------------------------------------------------------------------------------
 * Launch schedule and autotuning.  A schedule is (threads per block, blocks per SM,
 * sites per work unit); mbc_autotune times the candidate schedules of the plan's
 * kernel on the given fields (the plan's current schedule first, then the candidate
 * grid; every candidate evaluates the n_sites sites as one time slice four times, the
 * first untimed), keeps the fastest in the plan and in the context's cache keyed by the
 * plan signature (a plan made later with the same signature starts from it), and reports
 * it.  Candidates that do not fit or fail to launch are skipped; on an error the plan
 * keeps its original schedule.  Synchronises the stream.
 *
 * For an MBC_PREC_FP32 e-graph plan the schedule is the FP32 kernel's shape: threads =
 * 128 x walkers (128..768; a walker is a group of 128 threads walking its part of the
 * column trees), blocks_per_sm = blocks per site (1 or 2: a thread-block cluster whose
 * blocks share the site's B table), sites_per_unit = A leaves per leaf batch (1..3, 1
 * when more than two free indices are in use).  Setting a new shape rebuilds the plan's
 * FP32 arrays on the device (synchronising the device; MBC_UNSUPPORTED when the shape
 * needs more shared memory than a block has): CUDA graphs that captured calls of the
 * plan must be captured again, and the context's mbc_batch_reserve is redone by the next
 * mbc_batch.
 * ---------------------------------------------------------------------------------- */
typedef struct { int threads; int blocks_per_sm; int sites_per_unit; } mbc_schedule;
mbc_status mbc_autotune(mbc_plan* plan, const void* U, const void* D, int64_t n_sites, mbc_stream stream,
                        mbc_schedule* best);
mbc_status mbc_set_schedule(mbc_plan* plan, const mbc_schedule* s);
mbc_status mbc_get_schedule(const mbc_plan* plan, mbc_schedule* s);

/* ------------------------------------------------------------------------------------
 * Evaluation without device allocation.  The paper has no counterpart to this entry
 * point; it serves callers that may not allocate device memory at the moment they
 * evaluate: services whose device memory is carved out once at start up and must not
 * grow (an allocation could fail or take memory promised to another tenant), plug-ins
 * inside a host application that owns every device allocation, and real-time loops
 * that cannot afford an allocation's latency and implicit synchronisation.
 *
 * mbc_correlator_noalloc computes exactly what mbc_correlator computes (C only, no
 * per-site output) for an MBC_ALGO_EGRAPH plan, with every temporary (work counter,
 * per-site partial sums, the kernel's K slots) taken from one fixed device array of
 * MBC_NOALLOC_SCRATCH_BYTES bytes built into the library; it calls no cudaMalloc,
 * cudaFree or other allocating routine.  (MBC_PREC_FP32 plans are evaluated here in
 * the double-float arithmetic of MBC_PREC_MIXED, so their results agree with
 * mbc_correlator's to the FP32 path's tolerance, not bit for bit; for the other plans
 * they are identical.)  The caller still supplies the fields
 * U, D and the output C (device memory, same layouts as mbc_correlator); the plan must
 * have been created beforehand (plan creation allocates).
 *  - Every GPU that loads this part of the library holds the array until the process
 *    exits.  The first call on a device looks up the array's device address (with that
 *    device current) and keeps it for the life of the process; a device reset
 *    (cudaDeviceReset) invalidates it, and the entry point is then not usable again in
 *    that process.
 *  - All calls share the array and it keeps the last call's contents (the work counter
 *    is cleared on the stream at each call; nothing else needs to start at zero).
 *    Calls whose device work overlaps (different streams, or different host threads on
 *    one device) race on the array: serialise them on one stream.
 *  - A call needing more than the array holds (32 bytes per sink site plus one K slot
 *    of the plan, |cols_B| x |rows_B| x 16 bytes, plus 256) returns MBC_UNSUPPORTED
 *    and a message giving the sizes; fewer K slots than blocks reduce the grid instead.
 *    Plans with an empty canonical term set (C = 0) are not size-limited.
 * ---------------------------------------------------------------------------------- */
#define MBC_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
mbc_status mbc_correlator_noalloc(mbc_plan* plan, const void* U, const void* D, int n_sets, int T, int64_t V3,
                                  void* C, mbc_stream stream);

/* ------------------------------------------------------------------------------------
 * Hadron blocks (Sec. 2) and the block form of the correlator (Secs. 3-4).
 *
 * The block of a baryon B = eps_abc (q1_a^T G q2_b) q3_c^alpha with q3 = q1, at sink
 * site x (the proton block equation of Sec. 2):
 *     f(x; s1, s2, s3)_alpha = < B_alpha(x) qbar1(s1) qbar2(s2) qbar3(s3) >
 *       = eps_abc G_{beta gamma} [ Q1[(a beta), s3] Q1[(c alpha), s1]
 *                                  - Q1[(a beta), s1] Q1[(c alpha), s3] ] Q2[(b gamma), s2]
 * with Q1, Q2 the propagators of flavours q1, q2 at x, row (colour a, spin beta) =
 * 3 beta + a and source indices s = 3 spin + colour.  Types: P (q1 = u, q2 = d) and N
 * (q1 = d, q2 = u), each with G = C gamma_5, C gamma_5 P_+ or C gamma_5 P_-.  Entry
 * eta = ((s1 * 12 + s2) * 12 + s3) * 4 + alpha; MBC_BLOCK_ENTRIES entries per block.
 * Arithmetic: complex double.
 *
 * mbc_hadron_blocks: per-site blocks of one type, f [n_sites][MBC_BLOCK_ENTRIES] complex
 * double (device, written), from U, D [n_sites][12][12] (device).
 *
 * mbc_hadron_blocks_projected: F[s][t] = sum_x e^{-i 2 pi p.x / L} f(x) over the L^3
 * sink sites of each time slice, site i of the field layout at x = (i mod L,
 * (i / L) mod L, i / L^2); p: three integers (host memory) or NULL for zero momentum;
 * U, D [n_sets][T][L^3][12][12]; F [n_sets][T][MBC_BLOCK_ENTRIES] complex double
 * (device, written).  Partial sums over fixed tiles of sites are combined in a fixed
 * order with compensated sums (bit-reproducible for given sizes and device).
 *
 * Block plans (host planner, once per operator): the expanded block form of an
 * operator of the library (Sec. 3).  The sink operator is a sum of products of A
 * baryons whose spins are tied by the operator's tensors; the source operator is the
 * one of mbc_operator_terms (conjugated sink weights), first put in canonical form
 * (ascending slot sets, sorting sign; the contraction is antisymmetric in same-flavour
 * source fields).  Wick's theorem hands the source fields to the sink baryons in N_w
 * ways per product (9 for dinucleon I, 360 for 3He), each with the sign of the source
 * reordering times (-1)^{A(A-1)/2}; every term becomes a string of A block entries,
 * ordered canonically (ascending type, then eta) and merged with its multiplicity; the
 * merged terms form a factor tree (Sec. 4).
 *
 * mbc_block_correlator evaluates, for every set s and time slice t,
 *     C[s][t] = sum_k w_k prod_i F^{h_ik}[s][t](eta_ik)
 * with every sink baryon projected to momentum p (p, U, D, C as above; C device complex
 * double [n_sets][T], written): the paper's block setting.  On an L = 1 lattice it
 * equals the local-sink correlator of mbc_correlator.  prec: MBC_PREC_FP64 (complex
 * double throughout) or MBC_PREC_MIXED (double-float arithmetic: the projected blocks
 * with power-of-two site scaling, the factor tree over blocks scaled per slice; the
 * tile and slice sums in compensated double).
 * ---------------------------------------------------------------------------------- */
#define MBC_BLOCK_ENTRIES 6912
typedef enum {
    MBC_BLOCK_P = 0, MBC_BLOCK_N = 1, MBC_BLOCK_P_PLUS = 2, MBC_BLOCK_P_MINUS = 3,
    MBC_BLOCK_N_PLUS = 4, MBC_BLOCK_N_MINUS = 5
} mbc_block_type;
typedef struct mbc_block_plan mbc_block_plan;

mbc_status mbc_hadron_blocks(mbc_ctx* ctx, int type, const void* U, const void* D, int64_t n_sites, void* f,
                             mbc_stream stream);
mbc_status mbc_hadron_blocks_projected(mbc_ctx* ctx, int type, const void* U, const void* D, int n_sets, int T,
                                       int L, const int* p, void* F, mbc_stream stream);

mbc_status mbc_block_plan_create(mbc_ctx* ctx, int op, int prec, mbc_block_plan** out);
void mbc_block_plan_destroy(mbc_block_plan* plan);
typedef struct {
    int n_baryons;               /* A */
    int n_products;              /* baryon products of the sink operator */
    int n_w[8];                  /* source assignments (N_w) of the first 8 products */
    int64_t expanded_terms;      /* terms before merging */
    int64_t merged_terms;        /* after merging: the factor tree's leaves */
    int64_t factors;             /* distinct block entries the terms use */
    int64_t level_nodes[4];      /* factor-tree vertices per level (level A-1: leaves) */
    double block_flops_per_site; /* projected blocks of the used entries, per sink site */
    double tree_flops_per_slice; /* factor-tree evaluation, per time slice */
    int64_t shared_sums;         /* the factor tree's level-(A-2) vertices hash-consed by their
                                    leaf sums (Sec. 5's congruence on the block terms): distinct
                                    sums with equal factor and weight lists (A >= 2, else 0) */
    int64_t shared_sum_terms;    /* leaf terms of those distinct sums */
} mbc_block_plan_info;
mbc_status mbc_block_plan_get_info(const mbc_block_plan* plan, mbc_block_plan_info* info);
/* Merged terms: ids [merged_terms][A] (type * MBC_BLOCK_ENTRIES + eta, ascending within
 * a term), w [merged_terms][2] complex double (normalisation included); host memory. */
mbc_status mbc_block_plan_get_terms(const mbc_block_plan* plan, int32_t* ids, double* w);
/* Multiplicity of every merged term (how many expanded terms it merges; Sec. 3 and the
 * multiplicity histograms of its Fig. 2): int32 [merged_terms], host memory, in the order
 * of mbc_block_plan_get_terms. */
mbc_status mbc_block_plan_get_multiplicities(const mbc_block_plan* plan, int32_t* multiplicity);
mbc_status mbc_block_correlator(mbc_block_plan* plan, const void* U, const void* D, int n_sets, int T, int L,
                                const int* p, void* C, mbc_stream stream);
/* The block form of the local-sink correlator: C[s][t] = sum_x C_x with
 *     C_x = sum_k w_k prod_i f^{h_ik}(x; eta_ik),
 * every baryon at the same sink site x -- the same quantity as mbc_correlator for the
 * operator (U, D [n_sets][T][V3][12][12], C [n_sets][T], site_out optional
 * [n_sets][T][V3], as for mbc_correlator).  One block of threads per site builds the
 * site's blocks in shared memory and walks the block factor tree over them.  FP64 plans;
 * MBC_UNSUPPORTED when the plan's block entries do not fit shared memory. */
mbc_status mbc_block_correlator_local(mbc_block_plan* plan, const void* U, const void* D, int n_sets, int T,
                                      int64_t V3, void* C, void* site_out, mbc_stream stream);

/* Number of device kernel launches made by this context since it was created (every
 * launch of every mbc call counts once). */
int64_t mbc_launch_count(const mbc_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* MBC_H */
