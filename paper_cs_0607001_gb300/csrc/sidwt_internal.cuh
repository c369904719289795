// Internal declarations of libsidwt: lifting programs, plan state and the
// kernel launchers shared between translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "sidwt.h"

namespace sidwt {

// ---------------------------------------------------------------------------
// Programmatic dependent launch: a kernel launched with launch_dependent()
// may start while the previous kernel on the stream is still running; it
// calls pdl_wait() before it reads anything that kernel writes (the wait
// returns once that grid has completed and its writes are visible; launched
// normally, the wait returns at once).  pdl_release() lets the next such
// kernel start early.
// ---------------------------------------------------------------------------
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename... K, typename... A>
cudaError_t launch_dependent(void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<A &&>(args)...);
}

// The peak record of entry i = b (J + 1) + j from its packed key (|r|^2 bits
// high, ~D low): lag D, |r| and |r| over the FP64 energies (eq. 1); an
// invalid id, a zero key or a set *fail gives lag -1.  The key is reset to
// zero for the next call.
__device__ __forceinline__ void finalize_entry(int64_t i, unsigned long long *keys, const int32_t *ids, int nrefs,
                                               const double *xen, int64_t xen_len, const double *yen, int J,
                                               int32_t *lag, float *mag, double *norm, const int32_t *fail) {
    const int64_t b = i / (J + 1);
    const int j = (int)(i % (J + 1));
    const int r = ids[b];
    const unsigned long long k = __ldcg(keys + i);
    keys[i] = 0ull;
    if (r < 0 || r >= nrefs || k == 0ull || (fail && *fail)) {
        lag[i] = -1;
        mag[i] = 0.f;
        norm[i] = 0.0;
        return;
    }
    const uint32_t D = 0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFull);
    const float m = sqrtf(__uint_as_float((uint32_t)(k >> 32)));
    lag[i] = (int32_t)D;
    mag[i] = m;
    const double ex = xen[(int64_t)r * xen_len + ((1 << j) - 1) + (D & ((1u << j) - 1u))];
    const double den = sqrt(ex * yen[i]);
    norm[i] = den > 0.0 ? (double)m / den : 0.0;
}
#endif

enum Side { SIDE_X = 0, SIDE_Y = 1 };  // x: primal analysis P~(z^-1); y: dual P^T(z^-1)

// ---------------------------------------------------------------------------
// Lifting programs.  One analysis level of a periodic phase pair (E, O):
// steps X[n] += c0[s] * Y[n] + c1[s] * Y[n + nb[s]] with X = O (target 1) or
// E (target 0) and Y the other phase, then lo = ce E[n] and hi = co O[n]
// (D4: hi = co (E[n] + O[n-1])).  The structure is compile-time
// (LiftShape); the coefficients are computed on the host in double precision
// (LiftCoef) and passed by value.
//   LeGall 5/3, Sec. III-C Case I:  x: O -= (E[n]+E[n+1])/2, E += (O[n]+O[n-1])/4,
//     scale (1, 1/2);  y: E += (O[n]+O[n-1])/2, O -= (E[n]+E[n+1])/4, scale (1, 2).
//   CDF 9/7, Sec. III-C Case II with Table I: four steps a, b, g, d and the
//     scaling x (x side) or their negations in reverse roles (y side).
//   Causal D4, eq. 17 (both sides): O -= sqrt3 E; E += (sqrt3/4) O[n] +
//     ((sqrt3-2)/4) O[n-1]; lo = K1 E, hi = K2 (E[n] + O[n-1]); the odd phase is
//     v[2n-1].
// ---------------------------------------------------------------------------
struct LiftCoef {
    float c0[4], c1[4];
    float ce, co;
};

template <int F, int S>
struct LiftShape;

// target(s): 1 if step s updates the odd phase, 0 if the even phase.
// nb(s): offset of the second neighbour in the other phase (+1 or -1).
template <>
struct LiftShape<SIDWT_LEGALL53, SIDE_X> {
    static constexpr int nsteps = 2;
    __host__ __device__ static constexpr int target(int s) { return s == 0 ? 1 : 0; }
    __host__ __device__ static constexpr int nb(int s) { return s == 0 ? +1 : -1; }
    static constexpr bool d4 = false;
};
template <>
struct LiftShape<SIDWT_LEGALL53, SIDE_Y> {
    static constexpr int nsteps = 2;
    __host__ __device__ static constexpr int target(int s) { return s == 0 ? 0 : 1; }
    __host__ __device__ static constexpr int nb(int s) { return s == 0 ? -1 : +1; }
    static constexpr bool d4 = false;
};
template <>
struct LiftShape<SIDWT_CDF97, SIDE_X> {
    static constexpr int nsteps = 4;
    __host__ __device__ static constexpr int target(int s) { return (s & 1) ? 0 : 1; }
    __host__ __device__ static constexpr int nb(int s) { return (s & 1) ? -1 : +1; }
    static constexpr bool d4 = false;
};
template <>
struct LiftShape<SIDWT_CDF97, SIDE_Y> {
    static constexpr int nsteps = 4;
    __host__ __device__ static constexpr int target(int s) { return (s & 1) ? 1 : 0; }
    __host__ __device__ static constexpr int nb(int s) { return (s & 1) ? +1 : -1; }
    static constexpr bool d4 = false;
};
template <int S>
struct LiftShape<SIDWT_D4, S> {
    static constexpr int nsteps = 2;
    __host__ __device__ static constexpr int target(int s) { return s == 0 ? 1 : 0; }
    __host__ __device__ static constexpr int nb(int s) { return s == 0 ? +1 : -1; }
    static constexpr bool d4 = true;
};

// Host-side coefficient tables (double math, rounded once to float).
LiftCoef lift_coef(int filter, int side);
LiftCoef lift_coef_97t(double t, int side);

// One pulse of a ragged batch for the lifting kernels (element offsets).
struct RaggedLift {
    int64_t y_off;    // pulse start in the packed received buffer
    int64_t pyr_off;  // pyramid row start
    int64_t yen_off;  // energies start (J+1 values)
    int32_t N, J;
};

// Long pulses of a ragged batch, in tiles: tile k lifts levels 1..L of
// samples [t0, t0 + Tc) of its pulse (with a periodic halo) and leaves the
// energy partials of levels 0..L at part[part_off ..]; the pulse's tail then
// sums them and lifts levels L + 1..J from c_L.
constexpr int kTileSamples = 4096;
constexpr int kTileHalo = 256;   // samples each side: covers 5 levels of the 5-pair windows
constexpr int kTileLevels = 5;
struct RaggedTile {
    int64_t y_off, pyr_off, part_off;
    int32_t N, L, t0, Tc;
};
struct RaggedTail {
    RaggedLift it;
    int64_t part_off;  // the pulse's first tile's partials
    int32_t ntiles, L;
};

// Device item lists of a ragged batch by filter (0 D4, 1 5/3, 2 9/7) and path.
struct RaggedLiftGroups {
    const RaggedTile *tiles[3] = {nullptr, nullptr, nullptr};
    int n_tiles[3] = {0, 0, 0};
    const RaggedTail *tails[3] = {nullptr, nullptr, nullptr};
    int n_tails[3] = {0, 0, 0};
    int64_t maxN_tail[3] = {0, 0, 0};  // the longest c_L a tail lifts
    // pipelined persistent kernel (double buffer fits), [size class][filter]:
    // the shared buffers follow the class's longest pulse, so short pulses run
    // more CTAs per SM
    const RaggedLift *pipe[3][3] = {};
    int n_pipe[3][3] = {};
    int64_t maxN_pipe[3][3] = {};
    const RaggedLift *lng[3] = {nullptr, nullptr, nullptr};
    int n_long[3] = {0, 0, 0};
    int64_t maxN_long[3] = {0, 0, 0};
    int maxJ_long[3] = {0, 0, 0};
};

// ---------------------------------------------------------------------------
// Plan state.
// ---------------------------------------------------------------------------
struct TileList {  // per correlate: pulse tiles grouped by reference
    int32_t *perm = nullptr;        // [B] pulse indices grouped by reference
    int32_t *perm_prev = nullptr;   // the previous call's order (the two swap; null: not kept)
    int32_t *perm_base = nullptr;   // the allocation holding both
    int32_t *tile_ref = nullptr;    // [max_tiles]
    int32_t *tile_start = nullptr;  // [max_tiles] offset into perm
    int32_t *tile_count = nullptr;  // [max_tiles]
    int32_t *ntiles = nullptr;      // [3]: tiles, pulses with a valid id, grouping changed since the last call
    int32_t *cursor = nullptr;      // [cap_refs] scratch
    int64_t max_tiles = 0;
};

}  // namespace sidwt

struct sidwt_plan {
    int filter = 0;
    int64_t N = 0;
    int J = 0;
    bool is_int = false;
    double t97 = 0.0;  // CDF 9/7 free parameter t (0: Table I)

    // reference store
    int32_t nrefs = 0, cap_refs = 0;
    int64_t tree_elems = 0;        // 2 J N elements per reference
    float2 *tree_f = nullptr;      // [cap][tree_elems] (float view; integer plan: converted copy)
    int2 *tree_i = nullptr;        // [cap][tree_elems] integer plan only
    double *xen = nullptr;         // [cap][2^(J+1) - 1]
    int64_t xen_len = 0;

    // workspaces (sized for cap_batch pulses)
    int64_t cap_batch = 0;
    int64_t pyr_elems = 0;         // 2N - 2(N >> J) elements per pulse
    float2 *pyr_f = nullptr;       // [cap_batch][pyr_elems]
    int2 *pyr_i = nullptr;         // integer plan only
    double *yen = nullptr;         // [cap_batch][J+1]
    unsigned long long *keys = nullptr;  // [cap_batch][J+1] packed peak keys
    bool keys_clean = false;             // every key is zero (the kernels that read keys reset them)
    int32_t *lag = nullptr;
    float *mag = nullptr;
    double *norm = nullptr;
    int32_t *ref_ids = nullptr;    // copy of the last correlate's ids
    int32_t *err = nullptr;        // device error record
    sidwt::TileList tiles;
    int64_t last_B = -1;
    int64_t analyzed_B = -1;  // pulses whose pyramid and energies the plan holds (sidwt_correlate_again)
    int64_t analysis_gen = 0;  // counts analyses: the packed received operands record the one they came from
    int64_t tc_rx_gen = -1, tc_rx_B = -1;      // BF16x3 received operands: analysis and batch packed
    int64_t tc32_rx_gen = -1, tc32_rx_B = -1;  // the same for 3xTF32

    // sidwt_correlate_host: pinned host staging and device copies of the inputs
    void *h_stage = nullptr;
    size_t h_stage_bytes = 0;
    void *d_in = nullptr;
    size_t d_in_bytes = 0;
    // sidwt_correlate_host_async: the input copies run on the plan's own copy
    // stream; in_ready orders the compute after them, in_free the next call's
    // copies after the compute that read d_in
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t in_ready = nullptr, in_free = nullptr;

    // tensor-core operands (per scale j): packed reference windows and the
    // received bf16 hi/lo planes in grouped order
    void *tc_ref[16] = {};
    void *tc_ahi[16] = {};
    void *tc_alo[16] = {};
    int32_t tc_cap_refs = 0;
    int64_t tc_cap_batch = 0;
    int32_t tc_packed = 0;
    // 3xTF32 operands (per scale j): stored windows, received hi / lo planes
    void *tc32_ref[16] = {};
    void *tc32_bhi[16] = {};
    void *tc32_blo[16] = {};
    int32_t tc32_cap_refs = 0;
    int64_t tc32_cap_batch = 0;
    int32_t tc32_packed = 0;

    // stage timing: events recorded around each stage while enabled
    bool timing = false;
    struct Mark {
        int stage;  // 0 store, 1 group, 2 analyze, 3 correlate, 4 peaks
        cudaEvent_t a, b;
    };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> event_pool;
    int64_t timed_correlate_calls = 0;
    int64_t timed_launches = 0;

    void *small = nullptr;  // small-batch work list (ragged.cu)
};

namespace sidwt {

// stage timing (no-ops unless the plan's timing is on)
struct StageTimer {
    sidwt_plan *p;
    int stage;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    StageTimer(sidwt_plan *p, int stage, cudaStream_t s, int launches);
    ~StageTimer();
};

// the plan's lifting coefficients (its filter, and t for a CDF 9/7 plan)
LiftCoef plan_coef(const sidwt_plan *p, int side);

// plan workspaces and pulse-buffer checks shared with other entry points
sidwt_status ensure_plan_batch(sidwt_plan *p, int64_t B);
sidwt_status check_plan_pulses(sidwt_plan *p, const void *y_dev, int64_t B);

// error plumbing
void set_error(const std::string &msg);
sidwt_status cuda_fail(cudaError_t e, const char *what);

// bits of a plan's device error record
constexpr int32_t kErrBadRefId = 1;       // a pulse named a reference outside [0, num_refs)
constexpr int32_t kErrTcWait = 2;         // a tensor-core correlation CTA gave up on a bounded wait
constexpr int32_t kErrSelftestWait = 4;   // sidwt_tc_selftest's wait for its MMA gave up
constexpr int32_t kErrAnalysisWait = 8;   // the pipelined received analysis gave up waiting for an input copy

// sidwt_debug_stall's flags, read at each launch of a kernel they apply to
uint32_t debug_stall_flags();

// ---- lifting.cu ----
// SIDWT tree of one stored pulse (x_dev: complex64[N] or int16x2[N]) into
// reference slot ref of the plan, plus its energies.
sidwt_status build_reference_tree(sidwt_plan *p, const void *x_dev, int32_t ref, cudaStream_t s);
// Stored trees of up to kTreeBatch float signals of one filter in one pass
// (kernel parameters carry the descriptors): item k's pulse at x + x_off,
// its tree (2 J N elements) at tree + tree_off, its energies at
// xen + xen_off.  J from 1 to 15.
struct TreeItem {
    int64_t x_off, tree_off, xen_off;
    int32_t N, J;
};
constexpr int kTreeBatch = 64;
struct TreeBatch {
    int32_t n, pad;
    TreeItem it[kTreeBatch];           // sorted by decreasing J
    int64_t nprefix[kTreeBatch + 1];   // sum of N over the items before k
    int64_t eprefix[kTreeBatch + 1];   // sum of 2^(J+1) - 1 (energy blocks) before k
};
sidwt_status build_reference_trees(int filter, const float2 *x, float2 *tree, double *xen, const TreeItem *items,
                                   int n, cudaStream_t s, int *launches);
// Received analysis of B pulses into the plan's pyramid workspace (+ energies).
sidwt_status analyze_batch(sidwt_plan *p, const void *y_dev, int64_t B, cudaStream_t s);
int analyze_launch_count(const sidwt_plan *p);
// Ragged batch: all listed pulses, each with its own N, J and filter.
// part: the tiles' energy partials (kTileLevels + 1 per tile); err: the
// object's device error record (the pipelined kernel's bounded waits)
sidwt_status analyze_ragged(const float2 *y, const RaggedLiftGroups &g, float2 *pyr, double *yen, double *part,
                            int32_t *err, cudaStream_t s, int *launches);
int64_t tile_tail_max_n();
// Longest float pulse the pipelined analysis takes with two input buffers,
// and the upper ends of its size classes (the last one is that maximum).
int64_t analyze_pipe_max_n();
constexpr int kPipeClasses = 3;
int64_t analyze_pipe_class_max(int k);
cudaError_t prepare_ragged_kernels();
cudaError_t prepare_analysis_kernels();
cudaError_t prepare_tc_kernels();
// Sets every kernel's shared-memory budget once per device (outside any
// stream capture); called by plan and ragged-object creation.
sidwt_status prepare_kernels();

// ---- corr_simt.cu ----
sidwt_status group_pulses(sidwt_plan *p, const int32_t *ref_ids_dev, int64_t B, int tile_pulses,
                          cudaStream_t s);
// scale_mask: bit j set = correlate scale j here; group_tile: pulses per grouping tile
sidwt_status correlate_simt(sidwt_plan *p, int64_t B, float2 *r_dev, cudaStream_t s, uint32_t scale_mask = 0xffffffffu,
                            int group_tile = 64);
int simt_tile_pulses();

// ---- ragged.cu: batches of a few pulses on the batch-of-one kernel ----
constexpr int64_t kSmallBatch = 16;
sidwt_status prepare_small(sidwt_plan *p, int64_t B);
sidwt_status correlate_small(sidwt_plan *p, const int32_t *ref_ids_dev, int64_t B, float2 *R, cudaStream_t s);
int small_launch_count(const sidwt_plan *p);
// the latency kernel also records the ids and invalid-id errors (no grouping pass)
bool small_uses_latency_kernel(const sidwt_plan *p);
void free_small(sidwt_plan *p);

// ---- corr_tc.cu ----
sidwt_status correlate_tc(sidwt_plan *p, int64_t B, float2 *r_dev, cudaStream_t s);
uint32_t tc_scale_mask(const sidwt_plan *p);
int tc_group_tile();
int tc_launch_count(const sidwt_plan *p);
void free_tc(sidwt_plan *p);
// Peak records from the keys.  With invalidate_on_error, every record of the
// batch is written as no peak (lag -1, |r| 0, norm 0) if the plan's error
// record is set when the epilogue runs (callers that have no sidwt_check).
sidwt_status finalize_peaks(sidwt_plan *p, int64_t B, cudaStream_t s, bool invalidate_on_error = false);
// Copy the last batch's n peak entries to the caller's buffers (any may be null) in one launch.
sidwt_status copy_peaks(const sidwt_plan *p, int64_t n, int32_t *lag, float *mag, double *norm, cudaStream_t s);

// ---- corr_tc32.cu (3xTF32) ----
sidwt_status correlate_tc32(sidwt_plan *p, int64_t B, float2 *r_dev, cudaStream_t s);
uint32_t tc32_scale_mask(const sidwt_plan *p);
int tc32_group_tile();
int tc32_launch_count(const sidwt_plan *p);
void free_tc32(sidwt_plan *p);
cudaError_t prepare_tc32_kernels();
cudaError_t prepare_detect_kernels();

// ---- ragged_tc.cu: batch-of-one pairs on the tensor cores ----
namespace rtc {

// Operand geometry of one (pulse length N, depth J, scale j) on the
// tensor cores.  Rows of the GEMM are (variant v, shift block i) of the
// stored side, columns S consecutive advances; see ragged_tc.cu.
struct Shape {
    int j, lev, nb, nv;
    int64_t Kp;   // band length K'
    int S;        // advances per tile column block (MMA N) and per row
    int Lr;       // S / 8: polyphase samples per stored row
    int k0;       // first contraction index: 0 (circular, K' % 64 == 0) or -S (zero-padded)
    int nkb;      // K-blocks of 64 per band
    int gv;       // 8-row groups per variant
    int Rs;       // stored rows of Lr samples per (band, hi/lo, variant, chunk)
    int tiles;    // 128-row tiles of this (pair, scale)
    int64_t a_elems;  // stored operand, bf16 elements
};

struct TcTile {
    int32_t map;   // maps[2 map]: stored operand (maps[2 map + 1] unused)
    int32_t tile;  // first 8-row group = 16 tile
    int32_t nkb, Kp, gv, nv;
    int16_t nb, lev, S, k0;  // k0: first contraction index (0 circular, -S zero-padded)
    int64_t slot;   // peak key of this (pair, scale)
    int64_t u_off;  // received band 0 of this scale in the pyramid buffer (band 1 follows at + Kp)
    // peak key formed from band 0 alone before band 1 is added (scale J, whose
    // eq. 20a product is band 0 of scale J - 1's eq. 20 product), or -1
    int64_t slot_mid;
    // optional r output: complex64 offsets of the N-lag rows of slot and slot_mid
    int64_t r_at = -1, r_mid = -1;
    // split contraction: this work item runs the K-blocks f0 .. f0 + fcnt - 1
    // of the flattened (band, K-block) sequence (fcnt < 0: all of them); with
    // part_off >= 0 its accumulators go to the partials buffer ([S][128]
    // complex64 at part_off) for tc_split_reduce instead of peak keys
    int32_t f0 = 0, fcnt = -1;
    int64_t part_off = -1;
};

// A tile whose contraction was split into parts: the reduction sums its
// parts (the band-0 ones first: their sum alone is scale J's product when
// slot_mid >= 0) and forms the peaks as the epilogue would.
struct TcSplit {
    int64_t slot, slot_mid, r_at, r_mid, part_first;
    int32_t nparts, nparts0;  // all parts, and those of band 0 (the first nparts0)
    int32_t tile, gv, nv, Kp, lev, S;
};


// Relative cost per padded MMA element of each tile width (index 0: S = 256,
// 1: 128, 2: 64, 3: 192) by floor(log2 K'): defaults, or measured by the
// autotuner.
constexpr int kTcBuckets = 25;
constexpr int kTcWidths = 4;
constexpr int kTcWidth[kTcWidths] = {256, 128, 64, 192};
struct TcWeights {
    float w[kTcWidths][kTcBuckets];
};
void default_weights(TcWeights *t);
// The shape of scale j with tile width S (false: band outside the tensor-core range).
bool shape_with(int64_t N, int J, int j, int S, Shape *sh);  // S in kTcWidth
// The cheapest width under the weights (nullptr: defaults).
bool shape_for(int64_t N, int J, int j, Shape *sh, const TcWeights *w = nullptr);
// Stored tensor-core operand elements (bf16) of one (N, J) signal, rounded up
// per scale as the ragged object lays them out.
int64_t operand_elems(int64_t N, int J);
// Stored operand of every tensor-core scale of one signal whose SIDWT tree
// starts at tree; a_off[j] = element offset in abuf (-1: scale not packed),
// S_of[j] its tile width.
sidwt_status pack_stored(const float2 *tree, int64_t N, int J, const int64_t *a_off, const int16_t *S_of, void *abuf,
                         cudaStream_t s);
// The same for many signals whose trees start at tree + tree_off, in as few
// launches as the kernel-parameter tables allow.
struct PackItem {
    int64_t tree_off, N;
    int J;
    const int64_t *a_off;
    const int16_t *S_of;
};
sidwt_status pack_stored_batch(const float2 *tree, const PackItem *items, int n, void *abuf, cudaStream_t s,
                               int *launches);
sidwt_status encode_maps(void *two_maps, const void *a_base, const void *b_base, const Shape &sh);
size_t map_bytes();
// R: optional complex64 r output (each tile writes its rows at r_at / r_mid), or null;
// part: the partials buffer of split tiles (null when none is split)
sidwt_status launch_corr(const void *maps, const TcTile *tiles, int ntiles, const float2 *pyr, unsigned long long *keys,
                         int32_t *err, int sms, cudaStream_t s, float2 *R = nullptr, float2 *part = nullptr);
// Peaks (and r) of the split tiles from their parts.
sidwt_status launch_split_reduce(const TcSplit *splits, int nsplits, int maxS, const float2 *part,
                                 unsigned long long *keys, float2 *R, cudaStream_t s);
cudaError_t prepare_kernels();

}  // namespace rtc

// ---- ragged.cu: pre-size a ragged object's tensor-core operand buffers ----
sidwt_status ragged_reserve_tc(sidwt_ragged *r, int64_t stored_elems);
// whether the reserved stores hold that many more elements without growing
bool ragged_room(const sidwt_ragged *r, int64_t tree_elems, int64_t xen_elems, int64_t tc_elems);
// the device error record of a ragged object (kErr* bits; the serving loop
// copies it out with each batch's results)
int32_t *ragged_error_record(sidwt_ragged *r);
}  // namespace sidwt
