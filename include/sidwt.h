/*
 * sidwt.h -- C ABI of libsidwt, the GB300 (sm_103a) library for
 * multiresolution correlation of complex signals in the shift-invariant DWT
 * (SIDWT) domain by lifting (Bhattacharya & Mahapatra, "A Novel Application of
 * Lifting Scheme for Multiresolution Correlation of Complex Radar Signals").
 *
 * Problem (Sec. II, eq. 5-6; Sec. IV, eq. 20-20a).  A stored matching signal
 * x and received signals y, each N complex samples, are compared at every
 * circular lag D in [0, N) and at every dyadic scale j = 0..J:
 *
 *     r_j[D] = sum_k conj(X_{j,D}[k]) * Y_j[k]
 *
 * where X_{j,D} is the level-j primal (x-side) analysis of x delayed by D and
 * Y_j the level-j dual (y-side) analysis of y (scale 0: the signals
 * themselves).  The library evaluates the paper's DWT-domain form: for j < J
 * the level-(j+1) approximation and detail bands of the stored signal's SIDWT
 * tree (the shift-circulant block matrices of eq. 6 / 20) against the
 * received pulse's level-(j+1) bands; for j = J the level-J approximations
 * only (eq. 20a).  Real lifting steps act on Re and Im separately (eq. 19).
 *
 * Filters and sides (Sec. III):
 *   SIDWT_D4           causal Daubechies-4 lifting, eq. 17, on both sides;
 *                      polyphase pair (v[2n], v[2n-1]).
 *   SIDWT_LEGALL53     LeGall 5/3: x side P~(z^-1) and y side P^T(z^-1) of
 *                      Sec. III-C Case I; pair (v[2n], v[2n+1]).
 *   SIDWT_CDF97        CDF 9/7 with the rational Table I constants: x side
 *                      P~(z^-1), y side P^T(z^-1) of Sec. III-C Case II.
 *   SIDWT_CDF97_INT    reversible integer 9/7: the steps of Table I with
 *                      dyadic constants a = -3/2, b = -1/16, g = 205/256
 *                      (~ 4/5), d = 15/32, each update rounded to the nearest
 *                      integer (floor(c s + 1/2)), scalings dropped (x on one
 *                      side, 1/x on the other cancel in the pairing); int16
 *                      I/Q in, int32 coefficients, bit-exact.
 *   SIDWT_LEGALL53_INT reversible integer 5/3 (Sec. I, V-B): floor-rounded
 *                      steps, diagonal scalings dropped; inputs int16 I/Q,
 *                      coefficients int32, bit-exact.
 * Boundary handling is periodic at every level.
 *
 * Conventions shared by every entry point:
 *   - Complex data is interleaved (re, im) float32 ("complex64").  Integer
 *     plans take int16 (I, Q) pairs and produce int32 (re, im) pairs.
 *   - Pointers named *_dev are CUDA device pointers owned by the caller and
 *     must stay valid until the stream work that uses them has finished.
 *     Pointers named *_host are host pointers read or written before the call
 *     returns.
 *   - Calls enqueue work on `stream` (0 = the legacy default stream) and
 *     return without synchronising unless stated.  Errors detectable on the
 *     host return at once with a status; asynchronous device errors surface
 *     as SIDWT_ECUDA from a later call.  sidwt_last_error() describes the
 *     last failure of the calling thread.  No C++ exception crosses the ABI.
 *   - A plan is not thread-safe: serialise calls on one plan.
 */
#ifndef SIDWT_H
#define SIDWT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st *sidwt_stream; /* same type as cudaStream_t */

typedef enum {
    SIDWT_D4 = 0,
    SIDWT_LEGALL53 = 1,
    SIDWT_CDF97 = 2,
    SIDWT_LEGALL53_INT = 3,
    SIDWT_CDF97_INT = 4
} sidwt_filter;

typedef enum {
    SIDWT_PREC_FP32 = 0,  /* plain FP32 CUDA-core path ("plain")                      */
    SIDWT_PREC_BF16X3 = 1, /* tcgen05 tensor cores, bf16 hi+lo split (hi*hi + hi*lo + lo*hi),
                              FP32 accumulate; scales whose band is shorter than 64 or
                              not a multiple of 64 run on the FP32 path            */
    SIDWT_PREC_TF32X3 = 2  /* tcgen05 tensor cores, 3xTF32 split (hi*hi + hi*lo + lo*hi of
                              TF32-rounded parts), FP32 accumulate: FP32-grade accuracy;
                              plans only (sidwt_correlate); scales whose band is
                              shorter than 64 or not a multiple of 64 run on the FP32 path */
} sidwt_precision;

typedef enum {
    SIDWT_OK = 0,
    SIDWT_EINVAL = 1,      /* bad argument                                 */
    SIDWT_ENOMEM = 2,      /* device or host allocation failed             */
    SIDWT_ECUDA = 3,       /* a CUDA call failed (message has the detail)  */
    SIDWT_ETIMEOUT = 4,    /* a bounded wait ran out                       */
    SIDWT_EBUSY = 5,       /* resource in use                              */
    SIDWT_EUNSUPPORTED = 6 /* valid request this build does not implement  */
} sidwt_status;

typedef struct sidwt_plan sidwt_plan; /* opaque; owns the reference store and workspaces */

/* Library version string, e.g. "libsidwt 0.1 sm_103a". */
const char *sidwt_version(void);

/* Thread-local description of the last failure ("" if none). */
const char *sidwt_last_error(void);

/* Create a plan for pulses of N complex samples analysed to J dyadic levels
 * with filter f (Sec. II: L = 2^J samples; multiples of 2^J are accepted).
 * EINVAL unless 1 <= J <= 15, N % 2^J == 0, N >= 2^J and N <= 2^26.
 * *out receives the plan; destroy it with sidwt_plan_destroy. */
sidwt_status sidwt_plan_create(sidwt_filter f, int64_t N, int J, sidwt_plan **out);

/* Release the plan, its reference store and workspaces.  Synchronises the
 * device first.  NULL is accepted. */
sidwt_status sidwt_plan_destroy(sidwt_plan *p);

/* Pre-size the reference store for max_refs references and the workspaces
 * for batches of up to max_batch pulses, so that later calls allocate
 * nothing (needed before stream capture). */
sidwt_status sidwt_plan_reserve(sidwt_plan *p, int32_t max_refs, int64_t max_batch);

/* Number of stored references. */
int32_t sidwt_plan_num_refs(const sidwt_plan *p);

/* CDF 9/7 plans: use the member of the 9/7 family with free parameter t
 * (Sec. III-C Case II: a = (1 - 2t) / (4 (t - 1)), b = -(t - 1)^2,
 * g = 1 / (4 t (t - 1)), d = t^3 - (7/4) t^2 + t, x = sqrt(2) / t; t = 5/4
 * gives Table I, t = 0 restores it).  Both sides use the same t, so the
 * dual pairing and perfect reconstruction hold for every t.  EINVAL unless
 * the plan is CDF 9/7 and 0.780 < t < 1.852, t != 1; EBUSY once a reference
 * is stored. */
sidwt_status sidwt_plan_set_cdf97_t(sidwt_plan *p, double t);

/* Store a matching signal x (Sec. II eq. 5, Fig. 1 and 5): computes its SIDWT
 * tree -- for every level l = 1..J and variant v < 2^l, the level-l
 * approximation A and detail B of x delayed by v -- and the FP64 energies
 * ||X_{l,v}||^2 (eq. 1), and keeps them on the device.
 * x_dev: complex64[N] (float plans) or int16[N][2] (integer plan), 8- resp.
 * 4-byte aligned.  *ref_id_out receives the new reference's id (0, 1, ...).
 * The store may grow (a device allocation) unless reserved. */
sidwt_status sidwt_store_reference(sidwt_plan *p, const void *x_dev, int32_t *ref_id_out,
                                   sidwt_stream stream);

/* Copy reference ref_id's SIDWT tree and energies to caller buffers (either
 * may be NULL).  tree_dev layout: level l = 1..J at element offset 2N(l-1):
 * A[2^l][N >> l] then B[2^l][N >> l]; complex64 for float plans, int32 pairs
 * for the integer plan.  energies_dev: double[2^(J+1) - 1], level l variant v
 * at 2^l - 1 + v (level 0 is x itself). */
sidwt_status sidwt_reference_tree(sidwt_plan *p, int32_t ref_id, void *tree_dev, double *energies_dev,
                                  sidwt_stream stream);

/* Dual-basis analysis of B received pulses (Sec. III, Fig. 3(b) / 4(b)):
 * all J levels in one pass.  y_dev: [B][N] complex64 (float plans) or
 * int16[B][N][2] (integer plan).  Results stay in the plan's workspace; if
 * pyr_dev is not NULL they are also copied there as [B][2N - 2(N >> J)]
 * elements (complex64 or int32 pairs), level l at offset 2N - 4(N >> l):
 * c_l[N >> l] then d_l[N >> l].  energies_dev (optional): double[B][J+1],
 * ||c_j||^2 with c_0 = y. */
sidwt_status sidwt_analyze(sidwt_plan *p, const void *y_dev, int64_t B, void *pyr_dev, double *energies_dev,
                           sidwt_stream stream);

/* Correlate B received pulses, pulse b against stored reference
 * ref_ids_dev[b], at all N lags and all J+1 scales (eq. 20 / 20a), and
 * locate the peak of every (pulse, scale).  Runs the received analysis, the
 * correlation and the peak epilogue; results are read with sidwt_peaks.
 * ref_ids_dev: int32[B]; an id outside [0, num_refs) marks that pulse
 *   invalid (its peaks read lag -1) and is reported by sidwt_check.
 * y_dev: as for sidwt_analyze.
 * prec: SIDWT_PREC_FP32, SIDWT_PREC_BF16X3 or SIDWT_PREC_TF32X3.  Batches of at most 16
 *   pulses run in FP32 on the CUDA cores whatever prec says (a tile of 64 or
 *   128 pulses would be mostly empty): for N <= 8192 one CTA per (pulse,
 *   scale, variant, 32 delays) with the contraction split over its warps
 *   (the latency path), else the batch-of-one kernel of the ragged path, whose
 *   work list the first call with a given B builds.
 * r_dev: optional complex64[B][J+1][N], r_j[D] at [b][j][D]; NULL skips it
 *   (the full output is large: B (J+1) N 8 bytes). */
sidwt_status sidwt_correlate(sidwt_plan *p, const int32_t *ref_ids_dev, const void *y_dev, int64_t B,
                             sidwt_precision prec, void *r_dev, sidwt_stream stream);

/* sidwt_correlate without the received analysis: the pulses are those of
 * the plan's last analysis (sidwt_analyze, sidwt_correlate or
 * sidwt_correlate_c2f), whose pyramids and energies the plan still holds, so
 * that one batch is correlated against several stored signals while each
 * pulse is decomposed once (Sec. IV: the received signal's SIDWT feeds the
 * products with every stored signal).  B must equal that analysis's batch
 * (B = 0 does nothing); SIDWT_EINVAL otherwise, or when the plan's workspace
 * was reallocated since (a larger batch, sidwt_plan_reserve).  Other arguments and results as for
 * sidwt_correlate; calls on one plan must be ordered on one stream. */
sidwt_status sidwt_correlate_again(sidwt_plan *p, const int32_t *ref_ids_dev, int64_t B, sidwt_precision prec,
                                   void *r_dev, sidwt_stream stream);

/* Peaks of the last sidwt_correlate on this plan (B must match it), per
 * pulse b and scale j at [b][j]: lag_dev int32 (delay D of the stored signal
 * with the largest |r_j[D]|, smallest D on ties; -1 for an invalid pulse),
 * mag_dev float |r_j[lag]|, norm_dev double |r_j[lag]| /
 * sqrt(E_x[j][lag mod 2^j] E_y[j]) with the FP64 energies of eq. 1.  Any of
 * the three may be NULL. */
sidwt_status sidwt_peaks(sidwt_plan *p, int64_t B, int32_t *lag_dev, float *mag_dev, double *norm_dev,
                         sidwt_stream stream);

/* End-to-end call on host buffers: copies ref_ids_host and y_host to the
 * device (through pinned staging owned by the plan), correlates, and copies
 * the peaks back; returns after the stream has finished.  Any output pointer
 * may be NULL.  Same layouts as sidwt_correlate / sidwt_peaks. */
sidwt_status sidwt_correlate_host(sidwt_plan *p, const int32_t *ref_ids_host, const void *y_host, int64_t B,
                                  sidwt_precision prec, int32_t *lag_host, float *mag_host, double *norm_host,
                                  sidwt_stream stream);

/* Asynchronous form of sidwt_correlate_host for page-locked host buffers
 * (every non-NULL host pointer must be pinned, else SIDWT_EINVAL): the input
 * copies run on a copy stream owned by the plan, ordered after the previous
 * call's compute on this plan has read the plan's device copy of the inputs;
 * the correlation and the peak copies to the host run on `stream`, after the
 * input copies.  Returns once everything is enqueued: the outputs are valid,
 * and the host inputs may be reused, after `stream` has been synchronised.
 * Calls on different plans that share one stream overlap one call's input
 * copy with the previous call's correlation, while the correlations
 * themselves stay in stream order (they do not compete for the SMs).  Same
 * layouts as sidwt_correlate / sidwt_peaks. */
sidwt_status sidwt_correlate_host_async(sidwt_plan *p, const int32_t *ref_ids_host, const void *y_host, int64_t B,
                                        sidwt_precision prec, int32_t *lag_host, float *mag_host, double *norm_host,
                                        sidwt_stream stream);

/* Forget every stored reference (ids restart at 0); the store's capacity is
 * kept, so storing again allocates nothing. */
sidwt_status sidwt_reset_references(sidwt_plan *p);

/* Per-stage GPU time of this plan's calls, measured with CUDA events that the
 * library records on the call's stream around each stage while timing is
 * enabled.  Milliseconds summed over the calls since the last reset;
 * `launches` counts the library's kernel launches in those calls. */
typedef struct {
    double store_ms;     /* SIDWT tree of stored references                 */
    double group_ms;     /* grouping a batch by reference                   */
    double analyze_ms;   /* received dual-basis analysis                    */
    double correlate_ms; /* all-lag, all-scale correlation                  */
    double peaks_ms;     /* peak epilogue                                   */
    int64_t correlate_calls;
    int64_t launches;
} sidwt_timing;

/* Enable (1) or disable (0) stage timing on this plan. */
sidwt_status sidwt_set_timing(sidwt_plan *p, int enable);

/* Synchronise the recorded events and return the sums; reset != 0 clears
 * them afterwards. */
sidwt_status sidwt_read_timing(sidwt_plan *p, sidwt_timing *out, int reset);

/* Synchronise `stream` and report device-side errors recorded by earlier
 * calls on this plan: SIDWT_EINVAL for an out-of-range reference id,
 * SIDWT_ETIMEOUT if a tensor-core CTA or the pipelined received analysis
 * gave up on one of its bounded waits (the message says which; the results
 * are then incomplete); SIDWT_OK otherwise.  The record is cleared. */
sidwt_status sidwt_check(sidwt_plan *p, sidwt_stream stream);

/* Test hook (the paper has no counterpart): makes a bounded device wait run
 * out on purpose, so that a caller can test its handling of SIDWT_ETIMEOUT
 * without faulting the GPU.  Process-wide; read at each later launch of the
 * kernels it names; what = 0 restores normal operation.
 *   SIDWT_STALL_ANALYSIS: the pipelined received analysis (plan pulses that
 *     fit its shared memory, y_dev 16-byte aligned; ragged pulses of every
 *     length but those too long for a tail's shared memory) issues no input
 *     copy, so its first wait gives up after 200 ms; it records the timeout
 *     (sidwt_check / sidwt_ragged_check: SIDWT_ETIMEOUT; a serving request:
 *     status SIDWT_ETIMEOUT; sidwt_correlate_static: every peak record of the
 *     call is lag -1, |r| 0, norm 0) and returns with nothing in flight.
 *   SIDWT_STALL_TC_SELFTEST: sidwt_tc_selftest issues neither its MMA nor
 *     the commit, so its wait gives up after 200 ms and sets bit 4 of its err
 *     word; the kernel still releases its tensor memory.
 * EINVAL for unknown bits. */
#define SIDWT_STALL_ANALYSIS 1u
#define SIDWT_STALL_TC_SELFTEST 2u
sidwt_status sidwt_debug_stall(uint32_t what);

/* ---------------------------------------------------------------------------
 * Ragged batches: pulses of uneven length N, depth J and filter, each against
 * its own stored signal, correlated by persistent launches (all lags, all
 * J+1 scales, peaks), optionally replayed as one CUDA graph.  Every pair is a
 * batch of one.  In FP32 (the default) the correlation runs on the CUDA
 * cores: a work list over (pair, scale, variant, block of delays), ordered by
 * cost (largest first) and pulled by a persistent grid.  With
 * sidwt_ragged_set_precision(SIDWT_PREC_BF16X3) the scales whose bands have
 * at least 64 samples run as tcgen05 GEMMs instead (see there).  Float
 * filters only (D4, LeGall 5/3, CDF 9/7).  An object is not thread-safe and
 * holds one batch in flight; a graph refers to the object's buffers, so a
 * later call that grows them (more or longer references, a larger batch)
 * invalidates it.
 * ------------------------------------------------------------------------- */
typedef struct sidwt_ragged sidwt_ragged;

/* Create an empty ragged object.  Tile shapes come from the tuning cache
 * named by the environment variable SIDWT_TUNE_CACHE when it exists
 * (lines "log2(band length) shifts-per-thread"), else from defaults. */
sidwt_status sidwt_ragged_create(sidwt_ragged **out);
sidwt_status sidwt_ragged_destroy(sidwt_ragged *r);

/* Pre-size the reference store (tree_elems = sum of 2 J N over the stored
 * signals; their energies are sized to match), the received pyramid
 * (pyr_elems = sum of 2N - 2(N >> J) over a batch) and the peak slots
 * (slots = sum of J + 1 over a batch). */
sidwt_status sidwt_ragged_reserve(sidwt_ragged *r, int64_t tree_elems, int64_t pyr_elems, int64_t slots);

int32_t sidwt_ragged_num_refs(const sidwt_ragged *r);

/* Store one signal x_dev (complex64[N]) for filter f and depth J (same rules
 * as sidwt_plan_create); its SIDWT tree and energies stay resident. */
sidwt_status sidwt_ragged_store_reference(sidwt_ragged *r, sidwt_filter f, int64_t N, int J, const void *x_dev,
                                          int32_t *ref_id_out, sidwt_stream stream);

/* Store n signals at once (same rules per item as
 * sidwt_ragged_store_reference): item i is the complex64 signal of N_host[i]
 * samples at element x_offsets_host[i] of x_dev (x_elems elements; x_dev
 * 8-byte aligned), stored for filter filters_host[i] and depth J_host[i]
 * (Sec. II: the even and odd children at every level, Fig. 1 and 5).  All
 * the items' trees are built together, one launch per level and filter for
 * every 64 items, instead of one per level per item.  ref_ids_out[i]
 * receives item i's reference id.  The host arrays are read before the call
 * returns; x_dev must stay valid until the stream reaches the call. */
sidwt_status sidwt_ragged_store_references(sidwt_ragged *r, int64_t n, const int32_t *filters_host,
                                           const int64_t *N_host, const int32_t *J_host, const void *x_dev,
                                           const int64_t *x_offsets_host, int64_t x_elems, int32_t *ref_ids_out,
                                           sidwt_stream stream);

/* Correlate n_items pulses: item i is the complex64 pulse starting at element
 * y_offsets_host[i] of y_dev (even offsets: 16-byte aligned pulses), whose
 * length, depth and filter are those of reference ref_ids_host[i]; y_dev
 * holds y_elems complex64 elements and every pulse must lie inside it (else
 * SIDWT_EINVAL).  Peaks land in slots: item i's scales 0..J_i at slot
 * sum_{i' < i} (J_i' + 1).  The host arrays are read before the call
 * returns. */
sidwt_status sidwt_ragged_correlate(sidwt_ragged *r, int64_t n_items, const int32_t *ref_ids_host,
                                    const int64_t *y_offsets_host, const void *y_dev, int64_t y_elems,
                                    sidwt_stream stream);

/* How the tensor-core tiles' contractions are scheduled (not in the paper:
 * a latency measure).  mode 0 (default): a tile whose contraction is more
 * than twice the batch's total divided by twice the SM count is cut into
 * parts of about that share, at least 8 K-blocks of 64 samples each (never
 * across the two bands of eq. 20), each run by its own CTA; their
 * accumulators are summed in a fixed order by a second kernel that then
 * forms the peaks (and r), so a lone long pulse spreads over the GPU while a
 * large batch of short tiles is left as it is.  mode 1: never; mode 2: every tile long enough (for
 * tests).  Results agree within the stated bounds (the parts are summed in
 * FP32 outside the tensor cores).  EINVAL for another mode. */
sidwt_status sidwt_ragged_set_split(sidwt_ragged *r, int mode);

/* sidwt_ragged_correlate that also writes the correlation at every lag and
 * every scale, r_j[D] for D = 0..N_i-1 (eq. 20 for j < J_i, eq. 20a for
 * j = J_i), of every item: item i's rows start at complex64 element
 * sum_{i' < i} (J_i' + 1) N_i' of r_dev, scale j's row at + j N_i.  r_dev
 * (caller-owned, 8-byte aligned) must hold r_elems >= that sum over the
 * batch, else SIDWT_EINVAL; r_dev = NULL is sidwt_ragged_correlate.  The
 * writes are scattered (meant for checking, not for the bulk path). */
sidwt_status sidwt_ragged_correlate_r(sidwt_ragged *r, int64_t n_items, const int32_t *ref_ids_host,
                                      const int64_t *y_offsets_host, const void *y_dev, int64_t y_elems, void *r_dev,
                                      int64_t r_elems, sidwt_stream stream);

/* Build and instantiate a CUDA graph of the whole batch (lifting, the
 * persistent correlation, peaks) for this item layout and pulse buffer; the
 * layout is copied to device memory owned by the graph.  Replay with
 * sidwt_ragged_graph_launch after refilling y_dev in place.  launches_out
 * (optional) receives the number of kernels in the graph. */
sidwt_status sidwt_ragged_graph_create(sidwt_ragged *r, int64_t n_items, const int32_t *ref_ids_host,
                                       const int64_t *y_offsets_host, const void *y_dev, int64_t y_elems,
                                       int32_t *launches_out);
sidwt_status sidwt_ragged_graph_launch(sidwt_ragged *r, sidwt_stream stream);

/* Copy the last batch's peaks (n_slots = its sum of J_i + 1; same meaning as
 * sidwt_peaks).  Any output may be NULL. */
sidwt_status sidwt_ragged_peaks(sidwt_ragged *r, int64_t n_slots, int32_t *lag_dev, float *mag_dev, double *norm_dev,
                                sidwt_stream stream);

/* Autotune the correlation tiles and write the choice to cache_path (or
 * SIDWT_TUNE_CACHE; NULL and unset: not written; sidwt_ragged_create reads
 * SIDWT_TUNE_CACHE).  CUDA-core tiles: the shifts per thread for band
 * lengths 2^8 .. 2^15, each candidate (1, 2, 4, 8) timed on a synthetic
 * pair.  Tensor-core tiles: for band lengths 2^6 .. 2^14, every tile width S
 * (256, 192, 128, 64 advances) timed on a synthetic pair's tiles replicated over
 * the SMs; the weight of a width is its time per padded MMA element relative
 * to S = 256, and a reference stored afterwards takes, per scale, the width
 * of least weighted padded work (references stored before keep theirs).
 * Allocates and synchronises; call outside stream capture.  SIDWT_ETIMEOUT
 * if a timed kernel's bounded wait ran out. */
sidwt_status sidwt_ragged_autotune(sidwt_ragged *r, const char *cache_path, sidwt_stream stream);

/* The tensor-core width weights in use: w[k * 25 + b] for width 256 (k = 0),
 * 128 (1), 64 (2), 192 (3) and bands of 2^b .. 2^(b+1) - 1 samples. */
sidwt_status sidwt_ragged_tc_weights(const sidwt_ragged *r, float *w /* [4 * 25] */);

/* Stage timing of direct sidwt_ragged_correlate calls (not graph replays),
 * same meaning as sidwt_set_timing / sidwt_read_timing: analyze_ms (lifting),
 * correlate_ms (the persistent correlation kernel), peaks_ms. */
sidwt_status sidwt_ragged_set_timing(sidwt_ragged *r, int enable);
sidwt_status sidwt_ragged_read_timing(sidwt_ragged *r, sidwt_timing *out, int reset);

/* Forget every stored reference (ids restart at 0; capacity kept).  Must not
 * be called while a batch using them is in flight. */
sidwt_status sidwt_ragged_reset_references(sidwt_ragged *r);

/* Precision of later stores and correlations: SIDWT_PREC_FP32 (default; the
 * CUDA-core kernel above) or SIDWT_PREC_BF16X3.  With BF16X3 each stored
 * signal also keeps, for every scale whose band K' is at least 64 samples,
 * its variants packed for the tensor cores (bf16 hi and lo, about 32 N bytes
 * per such scale), and correlations run those scales as GEMMs on tcgen05:
 * rows are the stored variants advanced by multiples of S (S = 64, 128, 192
 * or 256 chosen per scale), columns the received band advanced by 0..S-1, so that
 * one received pulse fills whole tiles (eq. 20 / 20a unchanged; bands that
 * are not a multiple of 64 use the equivalent zero-padded linear form).
 * Shorter bands, and signals stored before the switch, stay on the CUDA
 * cores.  Error bound as for sidwt_correlate with BF16X3.
 * SIDWT_EUNSUPPORTED for SIDWT_PREC_TF32X3. */
sidwt_status sidwt_ragged_set_precision(sidwt_ragged *r, sidwt_precision prec);

/* Synchronise `stream` and report device-side failures of earlier batches:
 * SIDWT_ETIMEOUT if a tensor-core CTA or the received analysis gave up on a
 * bounded wait (the message says which; the results are incomplete),
 * SIDWT_OK otherwise.  The record is cleared. */
sidwt_status sidwt_ragged_check(sidwt_ragged *r, sidwt_stream stream);

/* The current choice: mq_by_log2_band[k] shifts per thread for bands of
 * length in [2^k, 2^(k+1)) (32 entries). */
sidwt_status sidwt_ragged_tuning(const sidwt_ragged *r, int32_t *mq_by_log2_band);

/* ---------------------------------------------------------------------------
 * Serving loop.  Requests (one received complex64 pulse each, against one of
 * the resident reference waveforms, with its own N, J and float filter)
 * arrive at any time; a server thread batches them continuously.  The device
 * is split into `lanes` CUDA streams with pre-reserved buffers; whenever a
 * lane is idle the thread takes queued requests in arrival order while they
 * fit the lane's share of memory_cap_bytes (request footprint about
 * (32 + 16 J) N bytes), zero-pads each request's waveform to its N, builds
 * the SIDWT trees and runs the ragged correlation, so batches overlap on the
 * device.  Each lane keeps the stored trees it built, keyed by (waveform,
 * filter, N, J), until its pre-reserved stores are full (then it starts
 * afresh): a request whose key is resident on its lane skips the stored-side
 * analysis.  A request larger than a lane's share is rejected (SIDWT_ENOMEM).
 * Latency runs from sidwt_server_submit to the moment the server thread
 * sees the lane's completion event.
 * ------------------------------------------------------------------------- */
typedef struct sidwt_server sidwt_server;

typedef struct {
    int32_t lanes;            /* concurrent batches (CUDA streams), 1..64          */
    int32_t max_batch;        /* requests per batch                                */
    int32_t max_j;            /* largest J a request may use (<= 15)               */
    int64_t memory_cap_bytes; /* admission cap over all in-flight batches          */
    int64_t max_lane_samples; /* sum of N one lane can hold (buffers pre-reserved) */
    int32_t precision;        /* SIDWT_PREC_FP32 or SIDWT_PREC_BF16X3 (the tensor-core
                                 batch-of-one path of sidwt_ragged_set_precision; the
                                 footprint then also counts its packed operands)     */
} sidwt_server_config;

typedef struct {
    int64_t completed, rejected, batches, max_batch, samples, queued;
    double p50_ms, p99_ms, max_ms; /* latency of completed requests              */
    double span_s;                 /* first arrival to last completion            */
    int64_t ref_hits;              /* requests whose stored SIDWT tree was already
                                      resident on their lane (no re-analysis)    */
    int64_t ref_stores;            /* stored trees built for requests            */
} sidwt_server_stats;

sidwt_status sidwt_server_create(const sidwt_server_config *cfg, sidwt_server **out);

/* Make a reference waveform (complex64[len], host) resident; before start. */
sidwt_status sidwt_server_add_waveform(sidwt_server *s, const void *x_host, int64_t len, int32_t *wave_id);

/* Start the server thread (uses the device current at this call). */
sidwt_status sidwt_server_start(sidwt_server *s);

/* Queue one request: y_host points at N complex64 samples (pinned memory
 * copies fastest) and must stay valid until the request finishes.  Returns
 * at once with the request id. */
sidwt_status sidwt_server_submit(sidwt_server *s, int32_t wave_id, sidwt_filter f, int64_t N, int J,
                                 const void *y_host, int64_t *request_id);

/* Bounded waits: SIDWT_ETIMEOUT if not finished within timeout_s; otherwise
 * the request's own status (SIDWT_ENOMEM if it was rejected, SIDWT_ETIMEOUT
 * if a bounded device wait of its batch ran out: every request of that batch
 * fails, and the lane's stored signals are rebuilt for later batches). */
sidwt_status sidwt_server_wait(sidwt_server *s, int64_t request_id, double timeout_s);
sidwt_status sidwt_server_drain(sidwt_server *s, double timeout_s);

/* A finished request's peaks (J+1 entries each, as sidwt_peaks) and latency. */
sidwt_status sidwt_server_result(sidwt_server *s, int64_t request_id, int32_t *lag_host, float *mag_host,
                                 double *norm_host, double *latency_ms);

/* Release a finished request's record. */
sidwt_status sidwt_server_forget(sidwt_server *s, int64_t request_id);

/* Counters and latency percentiles since the last reset. */
sidwt_status sidwt_server_read_stats(sidwt_server *s, sidwt_server_stats *out, int reset);

/* Finish queued and in-flight requests, stop the thread, free everything. */
sidwt_status sidwt_server_destroy(sidwt_server *s);

/* ---------------------------------------------------------------------------
 * Coarse-to-fine formation (Sec. IV eq. 21, Sec. V-B).
 * ------------------------------------------------------------------------- */

/* Eq. 21: one level of inverse y-side (dual) lifting -- the received
 * pyramid's approximation c_{l-1} from its level-l bands (c_l, d_l), i.e. the
 * synthesis that forms the finer resolution from the coarser one (perfect
 * reconstruction of one sidwt_analyze level).  B rows; row b reads H complex64
 * values at lo_dev + b * in_stride and at hi_dev + b * in_stride (so a
 * pyramid level can be read in place: lo = pyramid + 2N - 4H, hi = lo + H,
 * in_stride = the pyramid row length) and writes 2H values at
 * out_dev + b * 2H.  Float filters only (SIDWT_EUNSUPPORTED for the integer
 * filter); EINVAL unless 1 <= H <= 2^25, 0 <= B <= 65535, in_stride >= H and
 * the buffers are 8-byte aligned. */
sidwt_status sidwt_synthesize(sidwt_filter f, int64_t H, int64_t B, const void *lo_dev, const void *hi_dev,
                              int64_t in_stride, void *out_dev, sidwt_stream stream);

/* Coarse-to-fine peak search of B received pulses (Sec. V-B: the coarse scale
 * is correlated first and the finer ones are formed from it; Sec. IV: the
 * peak lag is the same at every scale within the scale's resolution).  Runs
 * the received analysis, correlates scale J at every delay D (eq. 20a), and
 * for j = J-1 down to 0 only at the delays within w_j = half_window 2^(j+1)
 * of the scale-(j+1) peak (circularly; all delays once 2 w_j + 1 >= N),
 * taking the largest |r_j| there (smallest delay on ties).  Per pulse about
 * N^2 / 2^J + 4 half_window N J complex products instead of about 2 N^2.
 * Output lag_dev int32[B][J+1] (delays; -1 for an invalid reference id,
 * reported by sidwt_check) and mag_dev float[B][J+1] (|r_j| there).  FP32.
 * Overwrites the plan's received pyramid; does not touch the peaks of
 * sidwt_correlate.  EINVAL for half_window < 1. */
sidwt_status sidwt_correlate_c2f(sidwt_plan *p, const int32_t *ref_ids_dev, const void *y_dev, int64_t B,
                                 int half_window, int32_t *lag_dev, float *mag_dev, sidwt_stream stream);

/* Per-scale target detection (Sec. V-A, Fig. 6: point targets that a scale
 * resolves show as separate peaks of |r_j| above a dB level; nearby targets
 * merge at coarser scales).  r_dev: complex64[rows][N], e.g. the r_dev of
 * sidwt_correlate ([B][J+1][N], rows = B (J+1)).  In each row, a detection is
 * a delay D whose |r[D]| is a local maximum along the delay axis
 * (circularly: greater than |r[D-1]|, not less than |r[D+1]|, so a flat top
 * counts once) and at least the row's largest |r| times
 * 10^(-threshold_db / 20).  count_dev int32[rows] receives the number of
 * detections; lag_dev int32[rows][max_det] and mag_dev float[rows][max_det]
 * the first max_det of them in increasing delay (|r| there).  FP32.
 * EINVAL for negative sizes or threshold, NULL buffers. */
sidwt_status sidwt_detect(const void *r_dev, int64_t rows, int64_t N, float threshold_db, int max_det,
                          int32_t *count_dev, int32_t *lag_dev, float *mag_dev, sidwt_stream stream);

/* Diagnostic: one tcgen05 MMA (M = 128, N = 64, K = 16, bf16 in, f32 out)
 * on fixed integer-valued operands laid out exactly as the tensor-core
 * correlation lays them out (K-major A; the overlapping MN-major window as
 * B), so that a host check can confirm the operand layouts on a given GPU.
 * out_dev: float[128][64]; err_dev: int32 flag, bit 4 set if the bounded
 * wait for the MMA ran out.  Operands: A[m][k] = ((7m + 3k) mod 11) - 5,
 * window planes P in {1, 2} with W_P[t] = ((5t + 17P) mod 13) - 6 and
 * B[k][n] = W_{1 + k/8}[8 (k mod 8) + n]. */
sidwt_status sidwt_tc_selftest(float *out_dev, int32_t *err_dev, sidwt_stream stream);

/* Allocation-free correlation against one stored signal.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory, for example a real-time receive loop that must not call
 * cudaMalloc once it runs (an allocation can synchronise the device and stall
 * for an unbounded time) or an application whose device memory belongs to
 * another allocator.  It stores x_dev (one complex64[N] or int16[N][2]
 * signal), correlates the B pulses of y_dev against it at all lags and scales
 * on the FP32 path, and writes the peaks to lag_dev / mag_dev / norm_dev
 * ([B][J+1], same meaning as sidwt_peaks; none may be NULL).
 * All intermediates live in one 16 MiB static device array inside the
 * library, which every GPU that loads the library holds until the process
 * exits; the call allocates nothing.  A call that needs more than 16 MiB
 * (roughly 16 N (B + J) bytes, twice that for the integer filter) returns
 * SIDWT_EINVAL with the size in the message; 1 <= B <= 65535.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  The address is kept for
 * the life of the process: after cudaDeviceReset (or anything else that
 * replaces the device's primary context) this entry point must not be called
 * again on that device.  Every call reuses the same array, so calls that
 * overlap on the GPU (other streams, other host threads) race and corrupt
 * each other: serialise them on one stream.  The call's own device error
 * record lives in the array too: if the received analysis gave up on its
 * bounded wait for an input copy, every peak record of the call is written as
 * lag -1, |r| 0, norm 0 (see sidwt_debug_stall). */
sidwt_status sidwt_correlate_static(sidwt_filter f, int64_t N, int J, const void *x_dev, const void *y_dev,
                                    int64_t B, int32_t *lag_dev, float *mag_dev, double *norm_dev,
                                    sidwt_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* SIDWT_H */
