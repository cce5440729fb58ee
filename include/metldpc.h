/*
 * metldpc.h -- C ABI of the batched MET-LDPC belief-propagation decoder
 * (libmetldpc.so, CUDA for sm_103a).
 *
 * The decoder performs the error-correction step of reverse reconciliation
 * in continuous-variable QKD as described in arXiv:1711.01783: Bob sends
 * the syndrome s = H x of his bits (Methods, Step 1); Alice decodes her soft
 * observation of x with flooding sum-product belief propagation (Methods,
 * Steps 2-5, Eqs. 1-5), many codewords at once (Results, "High speed error
 * correction with MET-LDPC codes").
 *
 * Conventions shared by every entry point:
 *  - Return value: MLD_OK (0) or a negative MLD_E* status.  The text of the
 *    last error raised on the calling thread is returned by mld_last_error().
 *  - Ownership: buffers passed in are owned by the caller and never freed by
 *    the library.  Opaque handles are freed by their *_destroy function.
 *  - Streams: every call that touches the device takes a cudaStream_t passed
 *    as `void *stream` (NULL = the legacy default stream).  Work is enqueued
 *    on that stream; the library never synchronizes the device.  With host
 *    buffers (no MLD_DEVICE_PTRS) the results are valid once that stream has
 *    been synchronized, and the caller leaves the buffers untouched until
 *    then: page-locked, mapped host buffers (cudaHostAlloc, cudaHostRegister,
 *    torch pin_memory) are read and written in place by the kernels over the
 *    host link; other host buffers are copied through the library's own.
 *  - Device: handles are bound to the CUDA device that was current when they
 *    were created; calls must be made with that device current.
 *  - LLRs follow L = ln p(x=0)/p(x=1); a bit is decided 1 iff its posterior
 *    is negative (a posterior of exactly 0 decides 0).  This is the LLR form
 *    of the ratio q(1)/q(0) and of the decision "c_i = 1 iff q_i > 1" in
 *    Methods, Step 5.
 *  - Bits, syndromes and flags are one uint8_t (0 or 1) per value; arrays
 *    indexed [codeword][node] are row-major with the node index fastest, in
 *    the caller's node numbering.
 */
#ifndef METLDPC_H
#define METLDPC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define MLD_OK        0
#define MLD_EINVAL   (-1)  /* bad argument (null pointer, size, flag, dtype)   */
#define MLD_ENOMEM   (-2)  /* host or device allocation failed                  */
#define MLD_ECUDA    (-3)  /* a CUDA runtime call or kernel launch failed        */
#define MLD_ETIMEOUT (-4)  /* a bounded device-side wait gave up (reported by
                              mld_decode_status; see mld_opts.staging)        */
#define MLD_EGRAPH   (-5)  /* malformed Tanner graph (index out of range, ...)   */

/* ---- edge-message storage type (mld_opts.msg_dtype) ---------------------- */
#define MLD_MSG_F32 0      /* check-to-variable messages stored as float       */
#define MLD_MSG_F16 1      /* stored as IEEE half (round to nearest even);
                              all arithmetic stays in float                    */

/* ---- decode flags -------------------------------------------------------- */
#define MLD_EARLY_TERM  0x1u  /* stop each codeword at the first iteration l >= 1
                                 whose hard decision satisfies H x = s
                                 (Methods, Step 5)                             */
#define MLD_DEVICE_PTRS 0x2u  /* all data pointers of the call are device
                                 memory; otherwise they are host memory, used
                                 in place when page-locked and mapped, else
                                 staged through the library's own buffers     */

typedef struct mld_graph mld_graph;
typedef struct mld_decoder mld_decoder;

/* Text of the last error raised on the calling thread ("" if none).  The
 * pointer stays valid until the next library call on this thread. */
const char *mld_last_error(void);

/* Library version string, e.g. "metldpc 0.1.0 sm_103a". */
const char *mld_version(void);

/* ---- Tanner graph --------------------------------------------------------
 * mld_graph_create: build the decoder's graph store from an edge list and
 * upload it to the current device.  H has n_cn rows (checks) and n_vn columns
 * (variable nodes, VNs); edge k joins VN edge_vn[k] and check edge_cn[k]
 * (Methods: R_j = VNs of check j, C_i = checks of VN i).
 *   edge_vn, edge_cn : host int32 [n_edges], 0 <= edge_vn < n_vn,
 *                      0 <= edge_cn < n_cn; each (VN, check) pair at most once.
 *   edge_type        : host uint8 [n_edges] in [0, MLD_MAX_EDGE_TYPES) or NULL
 *                      (all 0); it selects the weight of weighted BP only.
 * VNs of degree 1 carry no stored message: their variable-to-check message
 * is always their channel LLR, so they are left out of the iterations and
 * their posteriors are formed from the last check update (the "ignored VNs"
 * of Table 1 and the Discussion).  Errors: MLD_EINVAL for null/negative
 * arguments, MLD_EGRAPH for an out-of-range index, a repeated pair or more
 * than 2^30 edges, MLD_ENOMEM, MLD_ECUDA.  *out is set only on success. */
#define MLD_MAX_EDGE_TYPES 8
int mld_graph_create(const int32_t *edge_vn, const int32_t *edge_cn,
                     const uint8_t *edge_type, int64_t n_edges,
                     int32_t n_vn, int32_t n_cn, mld_graph **out);
int mld_graph_destroy(mld_graph *g);

typedef struct {
    int32_t n_vn, n_cn;
    int64_t n_edges;
    int32_t n_core;        /* VNs of degree != 1 (updated every iteration)   */
    int32_t n_deg1;        /* VNs of degree 1 (skipped during iterations)     */
    int64_t e_core;        /* edges between checks and core VNs = stored
                              messages = n_edges - n_deg1 (Table 1, "edges
                              to pass messages")                             */
    int32_t max_check_deg; /* max check degree (core + degree-1 edges)       */
    int32_t max_vn_deg;
} mld_graph_stats;
int mld_graph_stats_get(const mld_graph *g, mld_graph_stats *out);

/* The graph store's device index arrays, for tools that inspect or verify it
 * (device pointers into the library's own memory, int32, valid until
 * mld_graph_destroy).  Internal numbering: core edges check-major (cptr
 * [n_cn + 1], col [e_core]: core VN of each edge), degree-1 slots (dptr
 * [n_cn + 1]), the VN-major view (vptr [n_core + 1], vedge [e_core]), the
 * internal index of every caller VN (unit [n_vn]) and every caller check's
 * internal index (cint [n_cn]).  Writing through them corrupts the graph:
 * decoders created with `checked` detect that before decoding.  Errors:
 * MLD_EINVAL. */
typedef struct {
    const int32_t *cptr, *col, *dptr, *vptr, *vedge, *unit, *cint;
    int64_t n_cptr, n_col, n_dptr, n_vptr, n_vedge, n_unit, n_cint;
} mld_index_arrays;
int mld_graph_index_arrays(const mld_graph *g, mld_index_arrays *out);

/* ---- layers for the layered (serial) schedule -----------------------------
 * The layered schedule updates the checks one after another, each from the
 * latest messages of the others (the check and variable updates of Methods,
 * Steps 3-4, taken check by check instead of all at once; the paper runs the
 * flooding schedule).  Checks that share no VN of degree >= 2 give the same
 * result in either order, so the serial order is given as layers of such
 * checks: layer 0's checks first (in any order among themselves), then
 * layer 1's, and so on.
 * mld_graph_set_layers: layer_of_check = host int32 [n_cn], in the caller's
 *   check numbering, values in [0, n_layers); or NULL to build the default:
 *   the checks of each shape (edges to VNs of degree >= 2, degree-1 VNs) split
 *   by first fit, in check order, into layers whose checks share no such VN,
 *   layers numbered shape after shape.  Replaces any earlier layering; must
 *   not run while a decode on the graph is in flight.  Errors: MLD_EINVAL
 *   (null graph, layer out of range), MLD_EGRAPH (two checks of one layer
 *   share a VN of degree >= 2), MLD_ENOMEM, MLD_ECUDA.
 * mld_graph_layers_get: the current layering (layer_of_check may be NULL to
 *   read only *n_layers); MLD_EINVAL if the graph has none. */
int mld_graph_set_layers(mld_graph *g, const int32_t *layer_of_check, int32_t n_layers);
int mld_graph_layers_get(const mld_graph *g, int32_t *layer_of_check, int32_t *n_layers);

/* ---- synthetic code ensemble ----------------------------------------------
 * The seeded multi-edge-type ensemble the decoder is benchmarked on, built on
 * the host.  (The paper decodes PEG-built MET codes whose degree
 * distributions come from an external reference, Results and Table 1; this
 * family has their shape.)  n_c = round(core_frac n) core VNs with 2 (the
 * first 40 %) or 3 type-1 edges to m1 = n_c - round(rate n) type-1 checks and
 * d2 type-2 edges to m2 = n - n_c type-2 checks; m2 degree-1 VNs, one per
 * type-2 check; m = m1 + m2 = n - round(rate n) checks (the rate relation of
 * the Methods).  Check sockets of each edge type are dealt evenly, shuffled
 * and paired with VN sockets; repeated pairs are re-paired; VN and check
 * labels are shuffled.  Random numbers: xoshiro256** seeded by splitmix64
 * from (seed, n, d2).  Deterministic in the arguments on every machine.
 * mld_ensemble_size  : edges and checks of (rate, n, d2, core_frac).  Host only.
 * mld_ensemble_edges : the edge list into caller host buffers of `capacity`
 *                      entries (>= the edge count), sorted by (check, VN);
 *                      edge_type (may be NULL): 0 = type-1, 1 = type-2 of a
 *                      core VN, 2 = degree-1 VN.  Host only.
 * mld_graph_generate : mld_ensemble_edges with core_frac 0.20 / 0.12 / 0.06
 *                      for rate 0.1 / 0.05 / 0.02 (other rates: MLD_EINVAL),
 *                      then mld_graph_create.
 * Errors: MLD_EINVAL (arguments, degenerate sizes, capacity), MLD_EGRAPH
 * (re-pairing did not settle), and those of mld_graph_create. */
int mld_ensemble_size(double rate, int32_t n, int32_t d2, double core_frac,
                      int64_t *n_edges, int32_t *n_cn);
int mld_ensemble_edges(double rate, int32_t n, int32_t d2, double core_frac, uint64_t seed,
                       int32_t *edge_vn, int32_t *edge_cn, uint8_t *edge_type, int64_t capacity);
int mld_graph_generate(double rate, int32_t n, int32_t d2, uint64_t seed, mld_graph **out);

/* ---- progressive edge growth (PEG) ----------------------------------------
 * mld_peg_edges: the edge list of a multi-edge-type Tanner graph built by
 * progressive edge growth from VN degrees per edge type (the paper's codes
 * are PEG-built from multi-edge-type degree distributions, Results and
 * Table 1).  Host only.
 *   deg        : host int32 [n_types][n_vn], edges of each type per VN.
 *   mask       : host uint32 [n_cn]; bit t set if check c accepts type t.
 *   prio       : host int32 [n_cn] tie-break priorities, or NULL (index).
 *   outputs    : edge_vn, edge_cn int32 and edge_type uint8 [capacity] (>=
 *                the total degree), in placement order; *n_edges the count.
 * Rule: VNs in order of increasing total degree (ties by index), each VN's
 * edges type by type; an edge of type t goes to a check accepting t that is
 * not yet a neighbour of the VN, among the farthest from it in the graph
 * built so far (unreachable ones if any, else those at the largest
 * breadth-first level, the VN's neighbours being level 1), and among those
 * the lowest current degree, then the lowest priority.  Each placement costs
 * one breadth-first search (stopped once every check accepting t is
 * reached), so construction time grows with the square of the edge count.
 * Errors: MLD_EINVAL (arguments, capacity, more than 2^30 edges, 1 <= n_types
 * <= MLD_MAX_EDGE_TYPES), MLD_EGRAPH (no check left for an edge). */
int mld_peg_edges(int32_t n_vn, int32_t n_types, const int32_t *deg, int32_t n_cn, const uint32_t *mask,
                  const int32_t *prio, int64_t capacity, int32_t *edge_vn, int32_t *edge_cn,
                  uint8_t *edge_type, int64_t *n_edges);

/* ---- decoder --------------------------------------------------------------
 * mld_decoder_create: allocate the device state for decoding up to
 * opts->max_batch codewords of graph g at once.  The graph must outlive the
 * decoder.  Codewords are interleaved in slabs of `slab_width` (the paper's
 * "raw key permutation", Results): the message of one edge for one slab is a
 * contiguous run of slab_width values, so every graph gather is a full cache
 * line.  opts fields:
 *   msg_dtype  : MLD_MSG_F32 or MLD_MSG_F16.
 *   max_batch  : >= 1.
 *   lmax       : LLR clamp (> 0; 0 selects 25).  Channel LLRs, messages and
 *                the arguments of phi are kept within it (see mld_decode).
 *   slab_width : 8, 16, 32 or 64 codewords per slab; 0 selects 32 for F32
 *                and 64 for F16.
 *   vn_update  : how the variable update of Eq. 4 forms the posteriors
 *                L_v = L_ch(v) + sum_{e in C_v} r_e:
 *                MLD_VN_GATHER (0, default): a separate pass gathers each
 *                  VN's messages in a fixed order (deterministic results);
 *                MLD_VN_ACCUMULATE (1): the check update adds every new
 *                  message, as stored, to the next iteration's posteriors
 *                  with atomic adds, so the messages are read once less per
 *                  iteration; the order of the additions varies from run to
 *                  run, so posteriors may differ in the last float bits.  It
 *                  applies to fixed-iteration decoding (calls with
 *                  MLD_EARLY_TERM use the gather), needs the default slab
 *                  width and a graph whose checks all have at most 8 edges and
 *                  at most one degree-1 VN (MLD_EINVAL otherwise), and takes
 *                  two more posterior arrays of device memory.
 *   schedule   : MLD_SCHED_FLOODING (0, default): every check, then every
 *                  VN, per iteration (Methods, Steps 3-4);
 *                MLD_SCHED_LAYERED (1): the checks are updated one layer at a
 *                  time (see mld_graph_set_layers), each from the messages
 *                  its predecessors in the same iteration have just sent,
 *                  and the posteriors follow every layer (no separate
 *                  variable update).  One iteration updates every check
 *                  once.  Needs the default slab width and MLD_VN_GATHER
 *                  (MLD_EINVAL otherwise); if the graph has no layering yet,
 *                  the default one is built here.  Plans (mld_plan_create)
 *                  and mld_decode_noalloc run flooding.
 *   check_rule : MLD_CHECK_SUM_PRODUCT (0, default): Eqs. 2-3 in the phi form;
 *                MLD_CHECK_MIN_SUM (1): offset min-sum, an approximation of
 *                  Eqs. 2-3 that keeps the sign rule (syndrome sign included)
 *                  and takes as magnitude max(min of the other |q| - ms_offset,
 *                  0): no phi evaluations, at a cost in frame error rate.
 *                  Needs the default slab width, the flooding schedule and
 *                  MLD_VN_GATHER (MLD_EINVAL otherwise).  Plans and
 *                  mld_decode_noalloc run sum-product.
 *   ms_offset  : the min-sum offset in nats, >= 0 (ignored by sum-product).
 *   checked    : 0 (default) or 1: before every decode call a kernel checks
 *                every index of the graph's device arrays (and the layered
 *                tables of a layered decoder) against its range; the call
 *                waits for that check (it is no longer asynchronous) and, if
 *                the store is corrupted, returns MLD_EGRAPH naming the array,
 *                index and value without launching any decoding kernel.
 *                The result is kept for mld_decode_status.  A debugging aid
 *                for programs that may write stray device memory; plans do
 *                not check.
 *   staging    : MLD_STAGE_DIRECT (default): the check update reads its
 *                operands from device memory as it goes.  MLD_STAGE_BULK:
 *                where it applies (half messages at slab width 64,
 *                sum-product, flooding, MLD_VN_GATHER, checks of at most six
 *                terms with at most one degree-1 VN, and not the
 *                decisions-only early-termination pass), the operands of
 *                each group of 8 checks are brought into shared memory by
 *                bulk copies one group ahead of the arithmetic, one copy per
 *                posterior row; MLD_STAGE_BULK_LSU: the same, with the
 *                posterior rows copied 16 bytes per thread by cp.async.
 *                Results are bit-identical to MLD_STAGE_DIRECT (and slower
 *                on GB300: the direct kernel is instruction-bound).  Waits
 *                are bounded (2 s): a copy that never completes makes the
 *                decode's results invalid and mld_decode_status return
 *                MLD_ETIMEOUT.
 * Errors: MLD_EINVAL, MLD_ENOMEM, MLD_ECUDA. */
#define MLD_VN_GATHER         0
#define MLD_VN_ACCUMULATE     1
#define MLD_SCHED_FLOODING    0
#define MLD_SCHED_LAYERED     1
#define MLD_CHECK_SUM_PRODUCT 0
#define MLD_CHECK_MIN_SUM     1
#define MLD_STAGE_DIRECT      0
#define MLD_STAGE_BULK        1
#define MLD_STAGE_BULK_LSU    2
typedef struct {
    int32_t msg_dtype;
    int32_t max_batch;
    float lmax;
    int32_t slab_width;
    int32_t vn_update;
    int32_t schedule;
    int32_t check_rule;
    float ms_offset;
    int32_t checked;
    int32_t staging;
    int32_t reserved[6];  /* must be zero */
} mld_opts;
int mld_decoder_create(const mld_graph *g, const mld_opts *opts, mld_decoder **out);
int mld_decoder_destroy(mld_decoder *d);

/* mld_decode: sum-product BP on `batch` codewords (Methods, Steps 2-5).
 *   llr        : float [batch][n_vn], channel LLRs 2y/sigma^2 (Eq. 1 in LLR
 *                form), clamped to [-lmax, lmax] on entry.
 *   syndrome   : uint8 [batch][n_cn], Bob's syndrome s = H x (Step 1).
 *   batch      : 0 <= batch <= max_batch (0 does nothing).
 *   max_iters  : >= 0 flooding iterations; one iteration = check update
 *                (Eqs. 2-3, with the factor (1 - 2 s_j) of check j) then
 *                variable update (Eq. 4).  Per iteration, for check c and
 *                core edge e = (v, c):
 *                  q_e = clamp(L_v - r_e, lmax)   (degree-1 VN: q = L_ch(v))
 *                  r_e = (1-2s_c) prod_{e' != e} sgn q_e'
 *                        * phi(clamp(sum_{e' != e} phi(clamp(|q_e'|))))
 *                  L_v = L_ch(v) + sum_{e in C_v} r_e        (Eqs. 4-5)
 *                with phi(x) = -ln tanh(x/2) evaluated in float and its
 *                arguments kept in [phi(lmax), lmax].
 *   flags      : MLD_EARLY_TERM, MLD_DEVICE_PTRS.
 *   bits_out   : uint8 [batch][n_vn], hard decisions x = [L < 0] (Step 5).
 *   post_out   : float [batch][n_vn] posteriors L (Eq. 5), or NULL.
 *   converged  : uint8 [batch], 1 iff H bits = s.  Without MLD_EARLY_TERM
 *                exactly max_iters iterations run and this is still set.
 *   iters_used : int32 [batch]; max_iters without MLD_EARLY_TERM; with it,
 *                the first l >= 1 with H x^l = s (outputs are x^l, L^l), else
 *                max_iters.
 * Errors: MLD_EINVAL (null pointer, batch > max_batch, negative max_iters,
 * unknown flag), MLD_ECUDA.  A device-detected error, if any, is reported
 * by mld_decode_status once the stream has completed. */
int mld_decode(mld_decoder *d, const float *llr, const uint8_t *syndrome,
               int32_t batch, int32_t max_iters, uint32_t flags,
               uint8_t *bits_out, float *post_out, uint8_t *converged,
               int32_t *iters_used, void *stream);

/* mld_decode_y: as mld_decode, from Alice's BIAWGN observation
 * y = (1 - 2x) + sigma z instead of LLRs; the channel LLR 2 y / sigma_b^2
 * (Eq. 1 in LLR form) is formed on the device.
 *   y     : float [batch][n_vn];  sigma : float [batch], each > 0 (host or
 *   device memory like the other pointers).  A sigma <= 0 yields LLR 0 for
 *   that codeword's bits (no information) rather than an error. */
int mld_decode_y(mld_decoder *d, const float *y, const float *sigma,
                 const uint8_t *syndrome, int32_t batch, int32_t max_iters,
                 uint32_t flags, uint8_t *bits_out, float *post_out,
                 uint8_t *converged, int32_t *iters_used, void *stream);

/* Status of the decoder's device-side checks: MLD_OK, or MLD_EGRAPH when
 * the check of a decoder created with `checked` found the graph store
 * corrupted in its last decode call (array, index and value in
 * mld_last_error()), or MLD_ETIMEOUT when a staged check update
 * (MLD_STAGE_BULK) gave up waiting for a copy in some earlier call (sticky:
 * that decoder's later results are not to be trusted).  Reads the device
 * status word with a blocking copy; call after the stream is idle. */
int mld_decode_status(mld_decoder *d);

/* Test of the timeout path of the staged check update: with bytes > 0, every
 * later staged check-update launch of this decoder makes one block expect
 * `bytes` more than its first stage's copies bring, so that block's bounded
 * wait (2 s) runs out, it records MLD_ETIMEOUT in the status word and leaves
 * without storing (the decode's results are then invalid); 0 turns it off.
 * No fault is raised and the context stays usable.  Decoders without staging
 * ignore it.  A change waits for the device to be idle (it drops the
 * decoder's captured early-termination loops).  Errors: MLD_EINVAL (null
 * decoder, bytes outside [0, 65536]), MLD_ECUDA. */
int mld_decoder_test_stall(mld_decoder *d, int32_t bytes);

/* ---- uneven batches: several graphs in one launch --------------------------
 * A job is a batch of codewords of one graph, decoded with its own decoder
 * (which fixes the graph, message storage type, slab width and working
 * memory) and its own iteration cap.  A plan turns a list of jobs into one
 * schedule: in every iteration, one launch per kernel shape covers the work
 * of all jobs that are still iterating (their caps differ), so codes of
 * different rates and lengths share the GPU; the schedule is captured once
 * into a CUDA graph and mld_plan_launch replays it with a single launch.
 * This generalises the paper's multi-codeword decoding (Results, "High speed
 * error correction with MET-LDPC codes"), which decodes one code at a time.
 * Semantics per codeword are those of mld_decode_y / mld_decode with the
 * job's max_iters; with MLD_EARLY_TERM each codeword stops at its first
 * syndrome match (Methods, Step 5) and a slab whose codewords have all
 * stopped is skipped.
 *   decoder    : from mld_decoder_create; at most one job per decoder.
 *   in         : device float [batch][n_vn]: observations y if sigma != NULL
 *                (LLR = 2y/sigma^2 formed on the device), else channel LLRs.
 *   sigma      : device float [batch] or NULL.
 *   syndrome   : device uint8 [batch][n_cn].
 *   batch      : 1 <= batch <= the decoder's max_batch.
 *   max_iters  : >= 0.
 *   bits_out, post_out (or NULL), converged, iters_used: device outputs as
 *                for mld_decode.
 * All pointers are device memory (MLD_DEVICE_PTRS is implied).  The plan
 * records the pointers: they and the decoders must stay valid while the plan
 * is used, and a plan's launches must not overlap with other work on the same
 * decoders.  Errors: MLD_EINVAL (bad job, shared decoder, flag), MLD_ENOMEM,
 * MLD_ECUDA. */
typedef struct {
    mld_decoder *decoder;
    const float *in;
    const float *sigma;
    const uint8_t *syndrome;
    int32_t batch;
    int32_t max_iters;
    uint8_t *bits_out;
    float *post_out;
    uint8_t *converged;
    int32_t *iters_used;
} mld_job;
typedef struct mld_plan mld_plan;
int mld_plan_create(const mld_job *jobs, int32_t n_jobs, uint32_t flags, mld_plan **out);
/* Enqueue the plan's CUDA graph on `stream` (one launch). */
int mld_plan_launch(mld_plan *p, void *stream);
/* Number of kernel launches inside the plan's graph. */
int mld_plan_stats(const mld_plan *p, int64_t *launches);
int mld_plan_destroy(mld_plan *p);
/* Create a plan, launch it on `stream`, wait for the stream, destroy it. */
int mld_decode_multi(const mld_job *jobs, int32_t n_jobs, uint32_t flags, void *stream);

/* ---- differentiable weighted BP --------------------------------------------
 * Weighted BP scales every variable-to-check message of iteration t by a
 * learnable weight w[t][type(e)] (type = the edge_type given at graph
 * creation): in the LLR form of Methods Eq. 4,
 *   q_e^t = clamp(w[t][type(e)] * (L_ch(v) + sum_{e' != e} r_{e'}^{t-1})),
 * followed by the check update of Eqs. 2-3 (syndrome sign, phi, clamps);
 * all weights 1 is plain BP.  The soft output is the posterior of Eq. 5
 * after T iterations.  The adjoint gives dloss/dw and dloss/dLLR for any
 * loss of the soft output; it recomputes segments of ckpt_k iterations from
 * messages stored every ckpt_k iterations (ckpt_k = 1 stores every one).
 *
 * mld_wbp_forward:
 *   d        : decoder with MLD_MSG_F32 storage (its working memory is used;
 *              no other call may use d until the tape is destroyed).
 *   llr      : device float [batch][n_vn] channel LLRs (clamped to lmax).
 *   syndrome : device uint8 [batch][n_cn].   1 <= batch <= max_batch.
 *   w        : device float [T][n_types], 1 <= n_types <= MLD_MAX_EDGE_TYPES,
 *              every edge type of the graph < n_types.
 *   T >= 1 iterations; ckpt_k >= 1.
 *   soft_out : device float [batch][n_vn] posteriors after iteration T.
 *   tape     : receives the tape for mld_wbp_backward, or NULL (no tape).
 * mld_wbp_backward: dsoft = dloss/dsoft_out (device float [batch][n_vn]);
 *   writes dw (device float [T][n_types]) and dllr (device float
 *   [batch][n_vn], 0 where the LLR was clamped).  May be called more than once.
 * mld_tape_destroy: the decoder keeps the tape's device buffers (without
 *   waiting for the device) and reuses them in its next mld_wbp_forward of
 *   the same shape (batch slabs, T, ckpt_k, n_types), so a training loop
 *   allocates once; that forward must be ordered after the backward's work
 *   (same stream, or synchronised).  The decoder frees them when destroyed.
 *   With a tape, the forward's iterations and the adjoint's segments run as
 *   CUDA graphs over the tape's buffers, captured (on the decoder's own
 *   capture stream) at the tape's first use and replayed later; if this
 *   thread cannot capture, they are launched directly.
 * Checks of degree above 16 are refused (MLD_EINVAL).  Errors: MLD_EINVAL,
 * MLD_ENOMEM, MLD_ECUDA. */
typedef struct mld_tape mld_tape;
int mld_wbp_forward(mld_decoder *d, const float *llr, const uint8_t *syndrome, int32_t batch,
                    const float *w, int32_t n_types, int32_t T, int32_t ckpt_k,
                    float *soft_out, mld_tape **tape, void *stream);
int mld_wbp_backward(mld_tape *t, const float *dsoft, float *dw, float *dllr, void *stream);
int mld_tape_destroy(mld_tape *t);

/* ---- kernel timing (measurement hook) -------------------------------------
 * mld_decoder_timing_enable(d, every): every = 0 turns timing off; every = N
 * >= 1 makes later decode calls on d record a pair of CUDA events on their
 * stream around the kernels of every N-th iteration (one pair around all
 * check-update launches of that iteration, one around its variable update,
 * one around its syndrome check) and around the entry and exit layout
 * kernels.  mld_decoder_timing_read waits for those events and returns, per
 * kernel class since the last read: the summed device time of the timed
 * regions (*_ms), their number (*_timed), and the number of kernels launched
 * while timing was on (*_launches, sampled or not); then it clears them.
 * Classes: check update (Eqs. 2-3), variable update (Eqs. 4-5), syndrome
 * check (Step 5), layout (interleave / de-interleave / bit packing).
 * Timing changes no result.  Errors: MLD_EINVAL, MLD_ECUDA. */
typedef struct {
    double check_ms, var_ms, syndrome_ms, layout_ms;
    int64_t check_launches, var_launches, syndrome_launches, layout_launches;
    int64_t check_timed, var_timed, syndrome_timed, layout_timed;
} mld_timing;
int mld_decoder_timing_enable(mld_decoder *d, int every);
int mld_decoder_timing_read(mld_decoder *d, mld_timing *out);

/* ---- decoding without any device allocation ------------------------------
 * (The paper has no counterpart to this entry point: it concerns how the
 * library obtains memory, not the decoding method.)
 *
 * mld_decode_noalloc decodes like mld_decode, but without a decoder object
 * and without allocating anything: its working memory (messages, posteriors,
 * interleaved inputs, syndrome and decision bits, per-codeword flags) is
 * carved from one file-scope device array of MLD_NOALLOC_SCRATCH_BYTES that
 * the library reserves on every GPU it is loaded on, for the life of the
 * process.  It serves callers that cannot call cudaMalloc: hosts whose device
 * memory is owned entirely by their own allocator or capped at start-up (a
 * framework's caching pool, a fixed real-time budget), and code paths where
 * an allocation is not allowed or where the implicit device synchronisation
 * of cudaMalloc/cudaFree would stall other streams.  It calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *   g          : a graph from mld_graph_create (created beforehand).
 *   msg_dtype  : MLD_MSG_F32 (slabs of 32 codewords) or MLD_MSG_F16 (64).
 *   llr, syndrome, bits_out, post_out (or NULL), converged, iters_used:
 *                DEVICE pointers laid out as for mld_decode; the call reads
 *                and writes only these and the scratch array.  MLD_DEVICE_PTRS
 *                may be given in flags and is implied.
 *   flags      : MLD_EARLY_TERM and/or MLD_DEVICE_PTRS.
 * The LLR clamp is 25.  Results are those of mld_decode with the same graph,
 * dtype, default slab width and inputs.
 * Limit: the working set for (graph, batch, msg_dtype) must fit in
 * MLD_NOALLOC_SCRATCH_BYTES; otherwise the call returns MLD_EINVAL and
 * mld_last_error() states the bytes needed.  (A rate-0.1 graph with n = 4096
 * needs about 4.5 MiB per slab of 64 codewords with half messages.)
 * Set-up: the first call on each device, made with that device current,
 * looks up the array's device address (cudaGetSymbolAddress) and caches it;
 * make that first call before any stream capture on the device.  Under lazy
 * module loading (CUDA_MODULE_LOADING=LAZY, the default of current CUDA) the
 * array is only reserved when the library's module is loaded on the device,
 * which may be that first call: make one warm-up call per device (any valid
 * call, e.g. batch 1 with max_iters 0) before handing the device's remaining
 * memory to another allocator, so that the 32 MiB are taken while they are
 * still free.  If they cannot be, the call fails with MLD_ECUDA and a text
 * naming the scratch array.  The cached address belongs to the device's
 * primary context: after cudaDeviceReset (or any teardown of that context)
 * it is stale, and this entry point must not be called again in the process.
 * Sharing: every call on a device uses the same array, which keeps the last
 * call's contents; each call clears what must start at zero.  Calls whose
 * work overlaps on the GPU (different streams, or host threads racing)
 * corrupt each other: serialize them.
 * Errors: MLD_EINVAL (null pointer, bad dtype/flag/size, scratch too small),
 * MLD_ECUDA. */
#define MLD_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int mld_decode_noalloc(const mld_graph *g, int32_t msg_dtype, const float *llr,
                       const uint8_t *syndrome, int32_t batch, int32_t max_iters,
                       uint32_t flags, uint8_t *bits_out, float *post_out,
                       uint8_t *converged, int32_t *iters_used, void *stream);

/* ---- multidimensional reconciliation front end (d = 8) --------------------
 * The step before decoding in the paper's reconciliation (Results,
 * "Information reconciliation for CV-QKD system"; Fig. 1): Bob's and Alice's
 * correlated Gaussian samples y = x + z become Bob's bits and Alice's LLRs of
 * them by rotating blocks of 8 samples onto a virtual binary-input AWGN
 * channel (the paper cites the method; these are its definitions).  A_i is
 * the matrix of left multiplication by the basis octonion e_i, octonions
 * being pairs of quaternions (1, i, j, k) with the Cayley-Dickson product
 * (a, b)(c, d) = (ac - conj(d) b, da + b conj(c)).
 * mld_md_bob: per block of 8 samples y and 8 bits b (uint8 0/1, the bits
 *   Bob will send the syndrome of): ynorm = |y|, u = (1 - 2b)/sqrt 8,
 *   alpha_i = <A_i y/|y|, u>, so that M = sum_i alpha_i A_i is orthogonal and
 *   M y/|y| = u.  A block of zeros is taken as direction e_0.
 *   y: float [count], bits: uint8 [count], alpha_out: float [count] (8 per
 *   block), ynorm_out: float [count/8]; count a multiple of 8.
 * mld_md_alice: LLR_k = 2 |y| (M x)_k / (sqrt 8 sigma_z^2) per block (the
 *   LLR of Bob's bit on the virtual channel; for Gaussian modulation only the
 *   noise variance sigma_z^2 of y = x + z enters), for `rows` rows of
 *   `row_len` samples (a multiple of 8), e.g. [codeword][n], with one noise
 *   variance per row: x, alpha, llr_out float [rows][row_len], ynorm
 *   [rows][row_len/8], noise_var [rows].  The LLRs feed mld_decode.
 * All pointers are device memory; y, x, alpha and outputs 16-byte aligned,
 * bits 8-byte aligned (MLD_EINVAL otherwise).  Errors: MLD_EINVAL, MLD_ECUDA. */
int mld_md_bob(const float *y, const uint8_t *bits, int64_t count, float *alpha_out, float *ynorm_out,
               void *stream);
int mld_md_alice(const float *x, const float *alpha, const float *ynorm, const float *noise_var, int32_t rows,
                 int64_t row_len, float *llr_out, void *stream);

/* ---- phi evaluation (verification hook) ----------------------------------
 * Evaluates on the device the float phi(x) = -ln tanh(x/2) that the check
 * update uses (the LLR-domain message map that the closing paragraph of the
 * Methods proposes to tabulate), for n inputs clamped to [phi(lmax), lmax]
 * with lmax = 25.  msg_dtype selects the variant a decoder of that message
 * storage type uses: MLD_MSG_F32 (relative error below 2e-6, about 1.5e-7
 * from the fit) or MLD_MSG_F16 (a shorter fit, relative error 2.0e-4, below
 * half's 2^-11 = 4.9e-4 rounding of every stored message).
 * x and out are device float pointers [n].  Errors: MLD_EINVAL, MLD_ECUDA. */
int mld_phi_eval(int32_t msg_dtype, const float *x, float *out, int64_t n, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* METLDPC_H */
