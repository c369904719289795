// C ABI of libsidwt: plans, the reference store, workspaces and the entry
// points declared in include/sidwt.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <atomic>
#include <new>
#include <string>

#include "sidwt_internal.cuh"

namespace sidwt {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

static std::atomic<uint32_t> g_debug_stall{0};

uint32_t debug_stall_flags() { return g_debug_stall.load(std::memory_order_relaxed); }

sidwt_status cuda_fail(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return SIDWT_ECUDA;
}

template <typename T>
static sidwt_status dalloc(T **ptr, size_t count, const char *what) {
    *ptr = nullptr;
    if (count == 0) return SIDWT_OK;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(ptr), count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        g_last_error = std::string("device allocation failed: ") + what + " (" + std::to_string(count * sizeof(T)) +
                       " bytes): " + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? SIDWT_ENOMEM : SIDWT_ECUDA;
    }
    return SIDWT_OK;
}

template <typename T>
static void dfree(T *&ptr) {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
}

static void free_batch(sidwt_plan *p) {
    dfree(p->pyr_f);
    dfree(p->pyr_i);
    dfree(p->yen);
    dfree(p->keys);
    dfree(p->lag);
    dfree(p->mag);
    dfree(p->norm);
    dfree(p->ref_ids);
    dfree(p->tiles.perm_base);
    p->tiles.perm = p->tiles.perm_prev = nullptr;
    dfree(p->tiles.tile_ref);
    dfree(p->tiles.tile_start);
    dfree(p->tiles.tile_count);
    p->cap_batch = 0;
    p->tiles.max_tiles = 0;
}

// Size every per-batch buffer for B pulses (and the tile list for the current
// number of references).
static sidwt_status ensure_batch(sidwt_plan *p, int64_t B) {
    const int64_t need_tiles = (B + 31) / 32 + std::max<int64_t>(p->cap_refs, 1);
    if (B <= p->cap_batch && need_tiles <= p->tiles.max_tiles) return SIDWT_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronise before workspace growth");
    const int64_t cap = std::max<int64_t>(B, p->cap_batch);
    free_batch(p);
    p->analyzed_B = -1;
    sidwt_status st = SIDWT_OK;
    const int64_t nk = cap * (p->J + 1);
    if ((st = dalloc(&p->pyr_f, (size_t)(cap * p->pyr_elems), "received pyramid")) ||
        (p->is_int && (st = dalloc(&p->pyr_i, (size_t)(cap * p->pyr_elems), "integer pyramid"))) ||
        (st = dalloc(&p->yen, (size_t)nk, "received energies")) || (st = dalloc(&p->keys, (size_t)nk, "peak keys")) ||
        (st = dalloc(&p->lag, (size_t)nk, "peak lags")) || (st = dalloc(&p->mag, (size_t)nk, "peak magnitudes")) ||
        (st = dalloc(&p->norm, (size_t)nk, "peak norms")) || (st = dalloc(&p->ref_ids, (size_t)cap, "reference ids")) ||
        (st = dalloc(&p->tiles.perm_base, (size_t)(2 * cap), "pulse order")) ||
        (st = dalloc(&p->tiles.tile_ref, (size_t)need_tiles, "tile list")) ||
        (st = dalloc(&p->tiles.tile_start, (size_t)need_tiles, "tile list")) ||
        (st = dalloc(&p->tiles.tile_count, (size_t)need_tiles, "tile list"))) {
        free_batch(p);
        return st;
    }
    // both order buffers start out as "no pulse" (-1), so that the first
    // grouping reads as changed
    if (cudaMemset(p->tiles.perm_base, 0xFF, (size_t)(2 * cap) * sizeof(int32_t)) != cudaSuccess) {
        free_batch(p);
        return cuda_fail(cudaGetLastError(), "memset");
    }
    p->tiles.perm = p->tiles.perm_base;
    p->tiles.perm_prev = p->tiles.perm_base + cap;
    p->cap_batch = cap;
    p->tiles.max_tiles = need_tiles;
    p->keys_clean = false;
    return SIDWT_OK;
}

static sidwt_status ensure_refs(sidwt_plan *p, int32_t need) {
    if (need <= p->cap_refs) return SIDWT_OK;
    const int32_t cap = std::max<int32_t>(need, std::max<int32_t>(4, 2 * p->cap_refs));
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronise before store growth");
    float2 *tf = nullptr;
    int2 *ti = nullptr;
    double *xe = nullptr;
    int32_t *cur = nullptr;
    sidwt_status st;
    if ((st = dalloc(&tf, (size_t)cap * p->tree_elems, "reference store")) ||
        (p->is_int && (st = dalloc(&ti, (size_t)cap * p->tree_elems, "integer reference store"))) ||
        (st = dalloc(&xe, (size_t)cap * p->xen_len, "reference energies")) ||
        (st = dalloc(&cur, (size_t)cap, "grouping scratch"))) {
        dfree(tf);
        dfree(ti);
        dfree(xe);
        dfree(cur);
        return st;
    }
    if (p->nrefs > 0) {
        cudaMemcpy(tf, p->tree_f, (size_t)p->nrefs * p->tree_elems * sizeof(float2), cudaMemcpyDeviceToDevice);
        if (p->is_int)
            cudaMemcpy(ti, p->tree_i, (size_t)p->nrefs * p->tree_elems * sizeof(int2), cudaMemcpyDeviceToDevice);
        cudaMemcpy(xe, p->xen, (size_t)p->nrefs * p->xen_len * sizeof(double), cudaMemcpyDeviceToDevice);
    }
    e = cudaGetLastError();
    dfree(p->tree_f);
    dfree(p->tree_i);
    dfree(p->xen);
    dfree(p->tiles.cursor);
    p->tree_f = tf;
    p->tree_i = ti;
    p->xen = xe;
    p->tiles.cursor = cur;
    p->cap_refs = cap;
    if (e != cudaSuccess) return cuda_fail(e, "store growth copy");
    // the tile list bound depends on the number of references
    if (p->cap_batch > 0) {
        const int64_t B = p->cap_batch;
        return ensure_batch(p, B);
    }
    return SIDWT_OK;
}

static cudaEvent_t take_event(sidwt_plan *p) {
    if (!p->event_pool.empty()) {
        cudaEvent_t e = p->event_pool.back();
        p->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

StageTimer::StageTimer(sidwt_plan *p_, int stage_, cudaStream_t s_, int launches) : p(p_), stage(stage_), s(s_) {
    if (!p->timing) return;
    p->timed_launches += launches;
    a = take_event(p);
    if (a) cudaEventRecord(a, s);
}

StageTimer::~StageTimer() {
    if (!p->timing || !a) return;
    cudaEvent_t b = take_event(p);
    if (!b) {
        p->event_pool.push_back(a);
        return;
    }
    cudaEventRecord(b, s);
    p->marks.push_back({stage, a, b});
}

sidwt_status prepare_kernels() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && done[dev]) return SIDWT_OK;
    e = prepare_analysis_kernels();
    if (e == cudaSuccess) e = prepare_tc_kernels();
    if (e == cudaSuccess) e = rtc::prepare_kernels();
    if (e == cudaSuccess) e = prepare_tc32_kernels();
    if (e == cudaSuccess) e = prepare_detect_kernels();
    if (e != cudaSuccess) return cuda_fail(e, "kernel shared-memory attributes");
    if (dev >= 0 && dev < 64) done[dev] = true;
    return SIDWT_OK;
}

// Device buffer for the inputs of the host-buffer entry points, owned by the
// plan; growing it waits for the device (the old buffer may still be read).
static sidwt_status ensure_host_inputs(sidwt_plan *p, size_t need) {
    if (need <= p->d_in_bytes) return SIDWT_OK;
    cudaDeviceSynchronize();
    if (p->d_in) cudaFree(p->d_in);
    p->d_in = nullptr;
    p->d_in_bytes = 0;
    if (cudaMalloc(&p->d_in, need) != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation failed for host-call inputs");
        return SIDWT_ENOMEM;
    }
    p->d_in_bytes = need;
    return SIDWT_OK;
}

static bool is_pinned_host(const void *ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

}  // namespace sidwt

using namespace sidwt;

#define CHECK_PLAN(p)                          \
    do {                                       \
        if (!(p)) {                            \
            set_error("plan is NULL");         \
            return SIDWT_EINVAL;               \
        }                                      \
    } while (0)

extern "C" {

const char *sidwt_version(void) { return "libsidwt 0.1 sm_103a"; }

const char *sidwt_last_error(void) { return g_last_error.c_str(); }

sidwt_status sidwt_debug_stall(uint32_t what) {
    if (what & ~(SIDWT_STALL_ANALYSIS | SIDWT_STALL_TC_SELFTEST)) {
        set_error("sidwt_debug_stall: unknown flag");
        return SIDWT_EINVAL;
    }
    g_debug_stall.store(what, std::memory_order_relaxed);
    return SIDWT_OK;
}

sidwt_status sidwt_plan_create(sidwt_filter f, int64_t N, int J, sidwt_plan **out) {
    if (!out) {
        set_error("out is NULL");
        return SIDWT_EINVAL;
    }
    *out = nullptr;
    if ((int)f < 0 || (int)f > 4) {
        set_error("unknown filter");
        return SIDWT_EINVAL;
    }
    if (J < 1 || J > 15 || N < 2 || N > (int64_t(1) << 26) || N % (int64_t(1) << J) != 0) {
        set_error("need 1 <= J <= 15, N a multiple of 2^J, N <= 2^26");
        return SIDWT_EINVAL;
    }
    sidwt_status pst = prepare_kernels();
    if (pst) return pst;
    sidwt_plan *p = new (std::nothrow) sidwt_plan();
    if (!p) {
        set_error("host allocation failed");
        return SIDWT_ENOMEM;
    }
    p->filter = (int)f;
    p->N = N;
    p->J = J;
    p->is_int = (f == SIDWT_LEGALL53_INT || f == SIDWT_CDF97_INT);
    p->tree_elems = 2 * (int64_t)J * N;
    p->xen_len = (int64_t(2) << J) - 1;
    p->pyr_elems = 2 * N - 2 * (N >> J);
    sidwt_status st = dalloc(&p->err, 1, "error record");
    if (st == SIDWT_OK && (st = dalloc(&p->tiles.ntiles, 3, "tile count")) == SIDWT_OK) {
        cudaError_t e = cudaMemset(p->err, 0, sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMemset(p->tiles.ntiles, 0, 3 * sizeof(int32_t));
        if (e != cudaSuccess) st = cuda_fail(e, "memset");
    }
    if (st != SIDWT_OK) {
        dfree(p->err);
        dfree(p->tiles.ntiles);
        delete p;
        return st;
    }
    *out = p;
    return SIDWT_OK;
}

sidwt_status sidwt_plan_destroy(sidwt_plan *p) {
    if (!p) return SIDWT_OK;
    cudaDeviceSynchronize();
    free_batch(p);
    free_tc(p);
    free_tc32(p);
    free_small(p);
    dfree(p->tree_f);
    dfree(p->tree_i);
    dfree(p->xen);
    dfree(p->tiles.cursor);
    dfree(p->tiles.ntiles);
    dfree(p->err);
    if (p->h_stage) cudaFreeHost(p->h_stage);
    if (p->d_in) cudaFree(p->d_in);
    if (p->in_ready) cudaEventDestroy(p->in_ready);
    if (p->in_free) cudaEventDestroy(p->in_free);
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    for (auto &m : p->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (auto e : p->event_pool) cudaEventDestroy(e);
    delete p;
    return SIDWT_OK;
}

sidwt_status sidwt_plan_reserve(sidwt_plan *p, int32_t max_refs, int64_t max_batch) {
    CHECK_PLAN(p);
    if (max_refs < 0 || max_batch < 0) {
        set_error("negative reservation");
        return SIDWT_EINVAL;
    }
    sidwt_status st = ensure_refs(p, std::max<int32_t>(max_refs, 1));
    if (st) return st;
    if (max_batch > 0) return ensure_batch(p, max_batch);
    return SIDWT_OK;
}

int32_t sidwt_plan_num_refs(const sidwt_plan *p) { return p ? p->nrefs : -1; }

sidwt_status sidwt_store_reference(sidwt_plan *p, const void *x_dev, int32_t *ref_id_out, sidwt_stream stream) {
    CHECK_PLAN(p);
    if (!x_dev || !ref_id_out) {
        set_error("x_dev and ref_id_out must not be NULL");
        return SIDWT_EINVAL;
    }
    const uintptr_t align = p->is_int ? 4 : 8;
    if (reinterpret_cast<uintptr_t>(x_dev) % align) {
        set_error("x_dev is misaligned");
        return SIDWT_EINVAL;
    }
    sidwt_status st = ensure_refs(p, p->nrefs + 1);
    if (st) return st;
    const int32_t id = p->nrefs;
    {
        StageTimer t(p, 0, reinterpret_cast<cudaStream_t>(stream), p->J + 1);
        st = build_reference_tree(p, x_dev, id, reinterpret_cast<cudaStream_t>(stream));
    }
    if (st) return st;
    p->nrefs = id + 1;
    *ref_id_out = id;
    return SIDWT_OK;
}

sidwt_status sidwt_reference_tree(sidwt_plan *p, int32_t ref_id, void *tree_dev, double *energies_dev,
                                  sidwt_stream stream) {
    CHECK_PLAN(p);
    if (ref_id < 0 || ref_id >= p->nrefs) {
        set_error("reference id out of range");
        return SIDWT_EINVAL;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (tree_dev) {
        if (p->is_int)
            e = cudaMemcpyAsync(tree_dev, p->tree_i + (int64_t)ref_id * p->tree_elems, p->tree_elems * sizeof(int2),
                                cudaMemcpyDeviceToDevice, s);
        else
            e = cudaMemcpyAsync(tree_dev, p->tree_f + (int64_t)ref_id * p->tree_elems,
                                p->tree_elems * sizeof(float2), cudaMemcpyDeviceToDevice, s);
    }
    if (e == cudaSuccess && energies_dev)
        e = cudaMemcpyAsync(energies_dev, p->xen + (int64_t)ref_id * p->xen_len, p->xen_len * sizeof(double),
                            cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "tree copy");
}

static sidwt_status check_pulses(sidwt_plan *p, const void *y_dev, int64_t B) {
    if (B < 0 || B > (int64_t(1) << 31) - 1) {
        set_error("batch size out of range");
        return SIDWT_EINVAL;
    }
    if (B > 0 && !y_dev) {
        set_error("y_dev is NULL");
        return SIDWT_EINVAL;
    }
    const uintptr_t align = p->is_int ? 8 : 16;
    if (reinterpret_cast<uintptr_t>(y_dev) % align) {
        set_error("y_dev must be 16-byte (float) / 8-byte (integer) aligned");
        return SIDWT_EINVAL;
    }
    return SIDWT_OK;
}

}  // extern "C"

namespace sidwt {
sidwt_status ensure_plan_batch(sidwt_plan *p, int64_t B) { return ensure_batch(p, std::max<int64_t>(B, 1)); }
sidwt_status check_plan_pulses(sidwt_plan *p, const void *y_dev, int64_t B) { return check_pulses(p, y_dev, B); }
}  // namespace sidwt

extern "C" {

sidwt_status sidwt_plan_set_cdf97_t(sidwt_plan *p, double t) {
    CHECK_PLAN(p);
    if (p->filter != SIDWT_CDF97) {
        set_error("the free parameter t belongs to CDF 9/7 plans");
        return SIDWT_EINVAL;
    }
    if (t != 0.0 && !(t > 0.780 && t < 1.852 && std::fabs(t - 1.0) > 1e-6)) {
        set_error("need 0.780 < t < 1.852, t != 1 (or 0 for Table I)");
        return SIDWT_EINVAL;
    }
    if (p->nrefs > 0) {
        set_error("set t before storing references");
        return SIDWT_EBUSY;
    }
    p->t97 = t;
    return SIDWT_OK;
}

sidwt_status sidwt_analyze(sidwt_plan *p, const void *y_dev, int64_t B, void *pyr_dev, double *energies_dev,
                           sidwt_stream stream) {
    CHECK_PLAN(p);
    sidwt_status st = check_pulses(p, y_dev, B);
    if (st) return st;
    if ((st = ensure_batch(p, std::max<int64_t>(B, 1)))) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    {
        StageTimer t(p, 2, s, B > 0 ? analyze_launch_count(p) : 0);
        if ((st = analyze_batch(p, y_dev, B, s))) return st;
        p->analyzed_B = B;
        ++p->analysis_gen;
    }
    cudaError_t e = cudaSuccess;
    if (pyr_dev && B > 0) {
        if (p->is_int)
            e = cudaMemcpyAsync(pyr_dev, p->pyr_i, B * p->pyr_elems * sizeof(int2), cudaMemcpyDeviceToDevice, s);
        else
            e = cudaMemcpyAsync(pyr_dev, p->pyr_f, B * p->pyr_elems * sizeof(float2), cudaMemcpyDeviceToDevice, s);
    }
    if (e == cudaSuccess && energies_dev && B > 0)
        e = cudaMemcpyAsync(energies_dev, p->yen, B * (p->J + 1) * sizeof(double), cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "analysis copy-out");
}

// The body of sidwt_correlate and sidwt_correlate_again: `again` correlates
// the pulses of the plan's last analysis (no analysis launch, y_dev unused).
static sidwt_status correlate_impl(sidwt_plan *p, const int32_t *ref_ids_dev, const void *y_dev, int64_t B,
                                   sidwt_precision prec, void *r_dev, sidwt_stream stream, bool again) {
    sidwt_status st = SIDWT_OK;
    if (B > 0 && !ref_ids_dev) {
        set_error("ref_ids_dev is NULL");
        return SIDWT_EINVAL;
    }
    if (prec != SIDWT_PREC_FP32 && prec != SIDWT_PREC_BF16X3 && prec != SIDWT_PREC_TF32X3) {
        set_error("unknown precision");
        return SIDWT_EINVAL;
    }
    const bool tc = (prec == SIDWT_PREC_BF16X3);
    const bool tc32 = (prec == SIDWT_PREC_TF32X3);
    if (p->nrefs == 0 && B > 0) {
        set_error("no stored reference");
        return SIDWT_EINVAL;
    }
    if (again && B > 0 && B != p->analyzed_B) {
        set_error("B does not match the pulses of the plan's last analysis (sidwt_analyze or sidwt_correlate)");
        return SIDWT_EINVAL;
    }
    if ((st = ensure_batch(p, std::max<int64_t>(B, 1)))) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    p->last_B = B;
    if (B == 0) return SIDWT_OK;
    if (p->timing) ++p->timed_correlate_calls;
    const bool small = B <= kSmallBatch;
    if (small && !small_uses_latency_kernel(p) && (st = prepare_small(p, B))) return st;
    if (!(small && small_uses_latency_kernel(p))) {
        StageTimer t(p, 1, s, 1);
        const int gt = tc ? tc_group_tile() : (tc32 ? tc32_group_tile() : simt_tile_pulses());
        if ((st = group_pulses(p, ref_ids_dev, B, gt, s))) return st;
    }
    // keys are left zero by the kernel that reads them (finalize); clear them
    // only after an interrupted call or a fresh allocation, ahead of the
    // analysis (the correlation kernels may start before the analysis ends)
    if (!p->keys_clean) {
        cudaError_t e = cudaMemsetAsync(p->keys, 0, p->cap_batch * (p->J + 1) * sizeof(unsigned long long), s);
        if (e != cudaSuccess) return cuda_fail(e, "memset");
    }
    if (!again) {
        StageTimer t(p, 2, s, analyze_launch_count(p));
        if ((st = analyze_batch(p, y_dev, B, s))) return st;
        p->analyzed_B = B;
        ++p->analysis_gen;
    }
    p->keys_clean = false;
    {
        StageTimer t(p, 3, s, small ? small_launch_count(p) : (tc ? tc_launch_count(p) : (tc32 ? tc32_launch_count(p) : 1)));
        if (small) {
            if ((st = correlate_small(p, ref_ids_dev, B, reinterpret_cast<float2 *>(r_dev), s))) return st;
        } else if (tc) {
            if ((st = correlate_tc(p, B, reinterpret_cast<float2 *>(r_dev), s))) return st;
        } else if (tc32) {
            if ((st = correlate_tc32(p, B, reinterpret_cast<float2 *>(r_dev), s))) return st;
        } else if ((st = correlate_simt(p, B, reinterpret_cast<float2 *>(r_dev), s))) {
            return st;
        }
    }
    {
        StageTimer t(p, 4, s, 1);
        if ((st = finalize_peaks(p, B, s))) return st;
    }
    p->keys_clean = true;
    return SIDWT_OK;
}

sidwt_status sidwt_correlate(sidwt_plan *p, const int32_t *ref_ids_dev, const void *y_dev, int64_t B,
                             sidwt_precision prec, void *r_dev, sidwt_stream stream) {
    CHECK_PLAN(p);
    sidwt_status st = check_pulses(p, y_dev, B);
    if (st) return st;
    return correlate_impl(p, ref_ids_dev, y_dev, B, prec, r_dev, stream, false);
}

sidwt_status sidwt_correlate_again(sidwt_plan *p, const int32_t *ref_ids_dev, int64_t B, sidwt_precision prec,
                                   void *r_dev, sidwt_stream stream) {
    CHECK_PLAN(p);
    if (B < 0) {
        set_error("negative batch");
        return SIDWT_EINVAL;
    }
    return correlate_impl(p, ref_ids_dev, nullptr, B, prec, r_dev, stream, true);
}

sidwt_status sidwt_peaks(sidwt_plan *p, int64_t B, int32_t *lag_dev, float *mag_dev, double *norm_dev,
                         sidwt_stream stream) {
    CHECK_PLAN(p);
    if (B != p->last_B) {
        set_error("B does not match the last sidwt_correlate on this plan");
        return SIDWT_EINVAL;
    }
    if (B == 0) return SIDWT_OK;
    return copy_peaks(p, B * (p->J + 1), lag_dev, mag_dev, norm_dev, reinterpret_cast<cudaStream_t>(stream));
}

sidwt_status sidwt_correlate_host_async(sidwt_plan *p, const int32_t *ref_ids_host, const void *y_host, int64_t B,
                                        sidwt_precision prec, int32_t *lag_host, float *mag_host, double *norm_host,
                                        sidwt_stream stream) {
    CHECK_PLAN(p);
    if (B < 0 || (B > 0 && (!ref_ids_host || !y_host))) {
        set_error("bad host buffers");
        return SIDWT_EINVAL;
    }
    if (B > 0 && (!is_pinned_host(y_host) || !is_pinned_host(ref_ids_host) ||
                  (lag_host && !is_pinned_host(lag_host)) || (mag_host && !is_pinned_host(mag_host)) ||
                  (norm_host && !is_pinned_host(norm_host)))) {
        set_error("sidwt_correlate_host_async needs page-locked host buffers (cudaMallocHost / cudaHostRegister)");
        return SIDWT_EINVAL;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t ybytes = (size_t)B * p->N * (p->is_int ? 4 : 8);
    const size_t ibytes = (size_t)B * sizeof(int32_t);
    sidwt_status st = ensure_host_inputs(p, ybytes + ibytes + 256);
    if (st) return st;
    if (!p->copy_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->in_ready, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->in_free, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "copy stream / events");
    }
    char *dy = static_cast<char *>(p->d_in);
    int32_t *dids = reinterpret_cast<int32_t *>(dy + ((ybytes + 255) / 256) * 256);
    // the copies wait for the compute of the previous call on this plan to have
    // read d_in (an event never recorded lets them start at once), then run
    // beside whatever the compute stream is doing
    cudaError_t e = cudaStreamWaitEvent(p->copy_stream, p->in_free, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dy, y_host, ybytes, cudaMemcpyHostToDevice, p->copy_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dids, ref_ids_host, ibytes, cudaMemcpyHostToDevice, p->copy_stream);
    if (e == cudaSuccess) e = cudaEventRecord(p->in_ready, p->copy_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->in_ready, 0);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    st = sidwt_correlate(p, dids, dy, B, prec, nullptr, stream);
    if (st) return st;
    e = cudaEventRecord(p->in_free, s);
    const size_t n = (size_t)B * (p->J + 1);
    if (e == cudaSuccess && lag_host) e = cudaMemcpyAsync(lag_host, p->lag, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && mag_host) e = cudaMemcpyAsync(mag_host, p->mag, n * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && norm_host)
        e = cudaMemcpyAsync(norm_host, p->norm, n * sizeof(double), cudaMemcpyDeviceToHost, s);
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "device-to-host copy");
}

sidwt_status sidwt_correlate_host(sidwt_plan *p, const int32_t *ref_ids_host, const void *y_host, int64_t B,
                                  sidwt_precision prec, int32_t *lag_host, float *mag_host, double *norm_host,
                                  sidwt_stream stream) {
    CHECK_PLAN(p);
    if (B < 0 || (B > 0 && (!ref_ids_host || !y_host))) {
        set_error("bad host buffers");
        return SIDWT_EINVAL;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t ybytes = (size_t)B * p->N * (p->is_int ? 4 : 8);
    const size_t ibytes = (size_t)B * sizeof(int32_t);
    sidwt_status st0 = ensure_host_inputs(p, ybytes + ibytes + 256);
    if (st0) return st0;
    char *dy = static_cast<char *>(p->d_in);
    int32_t *dids = reinterpret_cast<int32_t *>(dy + ((ybytes + 255) / 256) * 256);
    const void *ysrc = y_host;
    const void *isrc = ref_ids_host;
    // pageable inputs go through the plan's pinned staging buffer
    if (!is_pinned_host(y_host) || !is_pinned_host(ref_ids_host)) {
        if (p->h_stage_bytes < ybytes + ibytes) {
            if (p->h_stage) cudaFreeHost(p->h_stage);
            p->h_stage = nullptr;
            p->h_stage_bytes = 0;
            if (cudaMallocHost(&p->h_stage, ybytes + ibytes) != cudaSuccess) {
                cudaGetLastError();
                set_error("pinned staging allocation failed");
                return SIDWT_ENOMEM;
            }
            p->h_stage_bytes = ybytes + ibytes;
        }
        std::memcpy(p->h_stage, y_host, ybytes);
        std::memcpy(static_cast<char *>(p->h_stage) + ybytes, ref_ids_host, ibytes);
        ysrc = p->h_stage;
        isrc = static_cast<char *>(p->h_stage) + ybytes;
    }
    cudaError_t e = cudaMemcpyAsync(dy, ysrc, ybytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dids, isrc, ibytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
    sidwt_status st = sidwt_correlate(p, dids, dy, B, prec, nullptr, stream);
    if (st) return st;
    const size_t n = (size_t)B * (p->J + 1);
    if (lag_host) e = cudaMemcpyAsync(lag_host, p->lag, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && mag_host) e = cudaMemcpyAsync(mag_host, p->mag, n * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && norm_host)
        e = cudaMemcpyAsync(norm_host, p->norm, n * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "device-to-host copy");
}

sidwt_status sidwt_reset_references(sidwt_plan *p) {
    CHECK_PLAN(p);
    p->nrefs = 0;
    p->tc_packed = 0;
    p->tc32_packed = 0;
    return SIDWT_OK;
}

sidwt_status sidwt_set_timing(sidwt_plan *p, int enable) {
    CHECK_PLAN(p);
    p->timing = enable != 0;
    return SIDWT_OK;
}

sidwt_status sidwt_read_timing(sidwt_plan *p, sidwt_timing *out, int reset) {
    CHECK_PLAN(p);
    if (!out) {
        set_error("out is NULL");
        return SIDWT_EINVAL;
    }
    double ms[5] = {0, 0, 0, 0, 0};
    for (auto &m : p->marks) {
        cudaError_t e = cudaEventSynchronize(m.b);
        if (e != cudaSuccess) return cuda_fail(e, "timing event");
        float t = 0.f;
        cudaEventElapsedTime(&t, m.a, m.b);
        ms[m.stage] += t;
    }
    out->store_ms = ms[0];
    out->group_ms = ms[1];
    out->analyze_ms = ms[2];
    out->correlate_ms = ms[3];
    out->peaks_ms = ms[4];
    out->correlate_calls = p->timed_correlate_calls;
    out->launches = p->timed_launches;
    if (reset) {
        for (auto &m : p->marks) {
            p->event_pool.push_back(m.a);
            p->event_pool.push_back(m.b);
        }
        p->marks.clear();
        p->timed_correlate_calls = 0;
        p->timed_launches = 0;
    }
    return SIDWT_OK;
}

sidwt_status sidwt_check(sidwt_plan *p, sidwt_stream stream) {
    CHECK_PLAN(p);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int32_t h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, p->err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "check");
    if (h) {
        cudaMemsetAsync(p->err, 0, sizeof(int32_t), s);
        cudaStreamSynchronize(s);
        if (h & kErrTcWait) {
            set_error("a tensor-core correlation CTA gave up on a bounded wait; its results are incomplete");
            return SIDWT_ETIMEOUT;
        }
        if (h & kErrAnalysisWait) {
            set_error("the received analysis gave up waiting for an input copy; the pyramid and the peaks are incomplete");
            return SIDWT_ETIMEOUT;
        }
        set_error("a correlate call received a reference id outside [0, num_refs)");
        return SIDWT_EINVAL;
    }
    return SIDWT_OK;
}

}  // extern "C"
