// Serving loop: correlation requests (one received pulse each, against one
// of the resident reference waveforms, with its own length N, depth J and
// filter) arrive at any time; a server thread batches them continuously.
//
// The device is split into lanes (CUDA streams), each with a pre-reserved
// ragged object and buffers.  Whenever a lane is idle the thread forms a
// batch from the queue in arrival order, admitting requests while they fit
// the lane's share of the memory cap, and enqueues the batch: pulse copies
// in, each request's waveform zero-padded to its N, the SIDWT trees, the
// ragged correlation, peaks out.  Requests that arrive while other lanes are
// busy join the next idle lane, so batches overlap on the device.  A request
// larger than a lane's share is rejected.  Every host wait is bounded.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sidwt_internal.cuh"

using namespace sidwt;
using Clock = std::chrono::steady_clock;

namespace {

struct Request {
    int64_t id;
    int32_t wave;
    int filter;
    int64_t N;
    int J;
    const void *y_host;
    Clock::time_point arrival, done;
    int64_t bytes = 0;
    sidwt_status status = SIDWT_OK;
    bool finished = false;
    std::vector<int32_t> lag;
    std::vector<float> mag;
    std::vector<double> norm;
};

int64_t footprint(int64_t N, int J, int precision) {
    // pulse, padded reference, SIDWT tree, pyramid, peak slots
    int64_t b = 8 * N + 8 * N + 16 * (int64_t)J * N + 16 * N + 64 * (J + 1);
    if (precision == SIDWT_PREC_BF16X3) b += 2 * rtc::operand_elems(N, J);  // packed stored operand (bf16)
    return b;
}

// The waveforms of a batch's new stored signals, each zero-padded to its
// request's N at its offset of the lane's signal buffer: grid.y = item.
constexpr int kPadBatch = 64;
struct PadBatch {
    const float2 *wave[kPadBatch];
    int64_t wlen[kPadBatch], off[kPadBatch], N[kPadBatch];
};

__global__ void pad_batch_kernel(const __grid_constant__ PadBatch b, float2 *__restrict__ x) {
    const int k = blockIdx.y;
    const float2 *w = b.wave[k];
    const int64_t wl = b.wlen[k], N = b.N[k];
    float2 *o = x + b.off[k];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = i < wl ? w[i] : make_float2(0.f, 0.f);
}

struct Lane {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    sidwt_ragged *rg = nullptr;
    float2 *y = nullptr, *x = nullptr;
    int64_t cap_samples = 0;
    int32_t *lag_d = nullptr;
    float *mag_d = nullptr;
    double *norm_d = nullptr;
    int32_t *lag_h = nullptr;
    float *mag_h = nullptr;
    double *norm_h = nullptr;
    int32_t *err_h = nullptr;  // the ragged object's device error record, copied out with each batch
    int64_t cap_slots = 0;
    bool busy = false;
    std::vector<Request *> batch;
    int64_t bytes = 0;
    // stored signals resident in this lane's ragged object, keyed by
    // (waveform, filter, N, J): a repeated request reuses its SIDWT tree
    std::unordered_map<uint64_t, int32_t> cache;
};

uint64_t ref_key(int32_t wave, int filter, int64_t N, int J) {
    return (uint64_t)(uint32_t)wave | ((uint64_t)filter << 20) | ((uint64_t)J << 24) | ((uint64_t)N << 32);
}

}  // namespace

struct sidwt_server {
    sidwt_server_config cfg;
    std::vector<Lane> lanes;
    std::vector<float2 *> waves;
    std::vector<int64_t> wave_len;
    std::mutex mu;
    std::condition_variable cv_submit, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<int64_t, Request *> reqs;
    int64_t next_id = 0;
    std::thread th;
    bool running = false, stop = false;
    int64_t in_flight_bytes = 0;
    // statistics
    std::vector<double> lat_ms;
    int64_t completed = 0, rejected = 0, batches = 0, samples = 0;
    Clock::time_point first_arrival, last_done;
    bool any = false;
    int64_t max_batch_seen = 0;
    int64_t ref_hits = 0, ref_stores = 0;
};

namespace {

void complete_lane(sidwt_server *s, Lane &L) {
    const auto now = Clock::now();
    int64_t slot = 0;
    std::lock_guard<std::mutex> lock(s->mu);
    for (Request *r : L.batch) {
        const int n = r->J + 1;
        r->lag.assign(L.lag_h + slot, L.lag_h + slot + n);
        r->mag.assign(L.mag_h + slot, L.mag_h + slot + n);
        r->norm.assign(L.norm_h + slot, L.norm_h + slot + n);
        slot += n;
        r->done = now;
        r->finished = true;
        s->lat_ms.push_back(std::chrono::duration<double, std::milli>(now - r->arrival).count());
        s->samples += r->N;
        ++s->completed;
    }
    s->last_done = now;
    s->in_flight_bytes -= L.bytes;
    L.bytes = 0;
    L.batch.clear();
    L.busy = false;
    s->cv_done.notify_all();
}

void fail_lane(sidwt_server *s, Lane &L, sidwt_status st) {
    std::lock_guard<std::mutex> lock(s->mu);
    for (Request *r : L.batch) {
        r->status = st;
        r->finished = true;
        r->done = Clock::now();
    }
    s->in_flight_bytes -= L.bytes;
    L.bytes = 0;
    L.batch.clear();
    L.busy = false;
    // what the failed batch stored may be incomplete
    L.cache.clear();
    sidwt_ragged_reset_references(L.rg);
    s->cv_done.notify_all();
}

// Elements one more stored signal takes in a lane's ragged object.
void store_needs(const sidwt_server *s, int64_t N, int J, int64_t *tree, int64_t *xen, int64_t *tc) {
    *tree = 2 * (int64_t)J * N;
    *xen = (int64_t(2) << J) - 1;
    *tc = s->cfg.precision == SIDWT_PREC_BF16X3 ? rtc::operand_elems(N, J) : 0;
}

// Enqueue a formed batch on a lane (server thread only).
sidwt_status launch_lane(sidwt_server *s, Lane &L) {
    cudaStream_t st = L.stream;
    // the batch's signals not yet resident must fit the lane's reserved
    // stores; otherwise start the cache afresh (nothing of it is in flight:
    // the lane is idle)
    {
        int64_t t = 0, x = 0, c = 0;
        std::unordered_map<uint64_t, int> seen;
        for (Request *r : L.batch) {
            const uint64_t k = ref_key(r->wave, r->filter, r->N, r->J);
            if (L.cache.count(k) || seen.count(k)) continue;
            seen[k] = 1;
            int64_t a, b2, d;
            store_needs(s, r->N, r->J, &a, &b2, &d);
            t += a;
            x += b2;
            c += d;
        }
        if (!ragged_room(L.rg, t, x, c)) {
            sidwt_ragged_reset_references(L.rg);
            L.cache.clear();
        }
    }
    std::vector<int32_t> ids;
    std::vector<int64_t> offs;
    // signals not yet resident: padded into the lane's signal buffer at the
    // request's offset and stored together (one batched tree build)
    std::vector<int32_t> nf, nJ;
    std::vector<int64_t> nN, noff;
    std::vector<uint64_t> nkey;
    std::unordered_map<uint64_t, int> pending;  // key -> index in the new signals
    std::vector<int> wait_new;                  // per request: index of the new signal it waits for, or -1
    PadBatch pb;
    int npad = 0;
    int64_t maxN = 0;
    int64_t off = 0, slots = 0, hits = 0, misses = 0;
    for (Request *r : L.batch) {
        cudaError_t e = cudaMemcpyAsync(L.y + off, r->y_host, (size_t)r->N * 8, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "request pulse copy");
        const uint64_t key = ref_key(r->wave, r->filter, r->N, r->J);
        auto it = L.cache.find(key);
        int32_t rid = -1;
        int wn = -1;
        if (it != L.cache.end()) {
            rid = it->second;
            ++hits;
        } else if (pending.count(key)) {
            wn = pending[key];
            ++hits;
        } else {
            wn = (int)nkey.size();
            pending[key] = wn;
            nkey.push_back(key);
            nf.push_back(r->filter);
            nN.push_back(r->N);
            nJ.push_back(r->J);
            noff.push_back(off);
            pb.wave[npad] = s->waves[(size_t)r->wave];
            pb.wlen[npad] = std::min<int64_t>(s->wave_len[(size_t)r->wave], r->N);
            pb.off[npad] = off;
            pb.N[npad] = r->N;
            maxN = std::max(maxN, r->N);
            ++npad;
            ++misses;
            if (npad == kPadBatch) {
                pad_batch_kernel<<<dim3((unsigned)std::min<int64_t>(64, (maxN + 255) / 256), (unsigned)npad), 256, 0,
                                   st>>>(pb, L.x);
                npad = 0;
                maxN = 0;
            }
        }
        ids.push_back(rid);
        wait_new.push_back(wn);
        offs.push_back(off);
        off += r->N;
        slots += r->J + 1;
    }
    if (npad > 0)
        pad_batch_kernel<<<dim3((unsigned)std::min<int64_t>(64, (maxN + 255) / 256), (unsigned)npad), 256, 0, st>>>(
            pb, L.x);
    if (!nkey.empty()) {
        std::vector<int32_t> nid(nkey.size());
        sidwt_status ss = sidwt_ragged_store_references(L.rg, (int64_t)nkey.size(), nf.data(), nN.data(), nJ.data(),
                                                        L.x, noff.data(), off, nid.data(),
                                                        reinterpret_cast<sidwt_stream>(st));
        if (ss) return ss;
        for (size_t k = 0; k < nkey.size(); ++k) L.cache[nkey[k]] = nid[k];
        for (size_t b = 0; b < ids.size(); ++b)
            if (wait_new[b] >= 0) ids[b] = nid[(size_t)wait_new[b]];
    }
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->ref_hits += hits;
        s->ref_stores += misses;
    }
    sidwt_status ss = sidwt_ragged_correlate(L.rg, (int64_t)ids.size(), ids.data(), offs.data(), L.y, off,
                                             reinterpret_cast<sidwt_stream>(st));
    if (ss) return ss;
    ss = sidwt_ragged_peaks(L.rg, slots, L.lag_d, L.mag_d, L.norm_d, reinterpret_cast<sidwt_stream>(st));
    if (ss) return ss;
    cudaError_t e = cudaMemcpyAsync(L.lag_h, L.lag_d, slots * sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L.mag_h, L.mag_d, slots * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L.norm_h, L.norm_d, slots * sizeof(double), cudaMemcpyDeviceToHost, st);
    // a bounded device wait that ran out (bits of the record) fails the batch
    int32_t *rec = ragged_error_record(L.rg);
    if (e == cudaSuccess) e = cudaMemcpyAsync(L.err_h, rec, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(rec, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = cudaEventRecord(L.done, st);
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "request result copy");
}

void serve(sidwt_server *s) {
    const int64_t lane_budget = s->cfg.memory_cap_bytes / std::max(1, s->cfg.lanes);
    for (;;) {
        bool progressed = false;
        for (Lane &L : s->lanes) {
            if (L.busy) {
                cudaError_t q = cudaEventQuery(L.done);
                if (q == cudaSuccess && *L.err_h) {
                    fail_lane(s, L, SIDWT_ETIMEOUT);
                    progressed = true;
                } else if (q == cudaSuccess) {
                    complete_lane(s, L);
                    progressed = true;
                } else if (q != cudaErrorNotReady) {
                    fail_lane(s, L, cuda_fail(q, "lane"));
                }
            }
        }
        for (Lane &L : s->lanes) {
            if (L.busy) continue;
            {
                std::lock_guard<std::mutex> lock(s->mu);
                int64_t bytes = 0, samples = 0, slots = 0;
                while (!s->queue.empty() && (int64_t)L.batch.size() < s->cfg.max_batch) {
                    Request *r = s->queue.front();
                    const int64_t fb = footprint(r->N, r->J, s->cfg.precision);
                    if (fb > lane_budget || r->N > L.cap_samples || r->J + 1 > L.cap_slots) {
                        // can never fit a lane: reject
                        s->queue.pop_front();
                        r->status = SIDWT_ENOMEM;
                        r->finished = true;
                        r->done = Clock::now();
                        ++s->rejected;
                        s->cv_done.notify_all();
                        continue;
                    }
                    if (bytes + fb > lane_budget || samples + r->N > L.cap_samples || slots + r->J + 1 > L.cap_slots ||
                        s->in_flight_bytes + bytes + fb > s->cfg.memory_cap_bytes)
                        break;
                    s->queue.pop_front();
                    L.batch.push_back(r);
                    bytes += fb;
                    samples += r->N;
                    slots += r->J + 1;
                }
                if (L.batch.empty()) continue;
                L.bytes = bytes;
                s->in_flight_bytes += bytes;
                ++s->batches;
                s->max_batch_seen = std::max<int64_t>(s->max_batch_seen, (int64_t)L.batch.size());
                L.busy = true;
            }
            sidwt_status st = launch_lane(s, L);
            if (st) fail_lane(s, L, st);
            progressed = true;
        }
        std::unique_lock<std::mutex> lock(s->mu);
        if (s->stop) {
            bool idle = true;
            for (Lane &L : s->lanes) idle = idle && !L.busy;
            if (idle && s->queue.empty()) break;
        }
        if (!progressed) {
            bool any_busy = false;
            for (Lane &L : s->lanes) any_busy = any_busy || L.busy;
            // idle: sleep until a submission; busy lanes: poll again shortly
            if (!any_busy)
                s->cv_submit.wait_for(lock, std::chrono::milliseconds(5));
            else {
                lock.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
        }
    }
}

}  // namespace

extern "C" {

sidwt_status sidwt_server_create(const sidwt_server_config *cfg, sidwt_server **out) {
    if (!cfg || !out || cfg->lanes < 1 || cfg->lanes > 64 || cfg->memory_cap_bytes <= 0 || cfg->max_batch < 1 ||
        cfg->max_lane_samples < 2 || cfg->max_j < 1 || cfg->max_j > 15 ||
        (cfg->precision != SIDWT_PREC_FP32 && cfg->precision != SIDWT_PREC_BF16X3)) {
        set_error("bad server configuration");
        return SIDWT_EINVAL;
    }
    *out = nullptr;
    sidwt_server *s = new (std::nothrow) sidwt_server();
    if (!s) {
        set_error("host allocation failed");
        return SIDWT_ENOMEM;
    }
    s->cfg = *cfg;
    s->lanes.resize((size_t)cfg->lanes);
    const int64_t cap = cfg->max_lane_samples;
    const int64_t slots = (int64_t)cfg->max_batch * (cfg->max_j + 1);
    for (Lane &L : s->lanes) {
        sidwt_status st = sidwt_ragged_create(&L.rg);
        if (!st) st = sidwt_ragged_reserve(L.rg, 2 * (int64_t)cfg->max_j * cap, 2 * cap, slots);
        if (!st) st = sidwt_ragged_set_precision(L.rg, (sidwt_precision)cfg->precision);
        if (!st && cfg->precision == SIDWT_PREC_BF16X3) {
            const int64_t a = rtc::operand_elems(cap - cap % (int64_t(1) << cfg->max_j), cfg->max_j);
            st = ragged_reserve_tc(L.rg, a + a / 2);
        }
        if (st || cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMalloc(&L.y, cap * sizeof(float2)) != cudaSuccess || cudaMalloc(&L.x, cap * sizeof(float2)) != cudaSuccess ||
            cudaMalloc(&L.lag_d, slots * sizeof(int32_t)) != cudaSuccess ||
            cudaMalloc(&L.mag_d, slots * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&L.norm_d, slots * sizeof(double)) != cudaSuccess ||
            cudaMallocHost(&L.lag_h, slots * sizeof(int32_t)) != cudaSuccess ||
            cudaMallocHost(&L.mag_h, slots * sizeof(float)) != cudaSuccess ||
            cudaMallocHost(&L.norm_h, slots * sizeof(double)) != cudaSuccess ||
            cudaMallocHost(&L.err_h, sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            sidwt_server_destroy(s);
            if (!st) set_error("server allocation failed");
            return st ? st : SIDWT_ENOMEM;
        }
        L.cap_samples = cap;
        L.cap_slots = slots;
    }
    *out = s;
    return SIDWT_OK;
}

sidwt_status sidwt_server_add_waveform(sidwt_server *s, const void *x_host, int64_t len, int32_t *wave_id) {
    if (!s || !x_host || len < 1 || !wave_id) {
        set_error("bad waveform");
        return SIDWT_EINVAL;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->running) {
        set_error("add waveforms before sidwt_server_start");
        return SIDWT_EBUSY;
    }
    float2 *d = nullptr;
    if (cudaMalloc(&d, len * sizeof(float2)) != cudaSuccess) {
        cudaGetLastError();
        set_error("waveform allocation failed");
        return SIDWT_ENOMEM;
    }
    cudaError_t e = cudaMemcpy(d, x_host, len * sizeof(float2), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "waveform copy");
    }
    s->waves.push_back(d);
    s->wave_len.push_back(len);
    *wave_id = (int32_t)s->waves.size() - 1;
    return SIDWT_OK;
}

sidwt_status sidwt_server_start(sidwt_server *s) {
    if (!s) {
        set_error("NULL server");
        return SIDWT_EINVAL;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->running) return SIDWT_OK;
    s->stop = false;
    s->running = true;
    int dev = 0;
    cudaGetDevice(&dev);
    s->th = std::thread([s, dev] {
        cudaSetDevice(dev);
        serve(s);
    });
    return SIDWT_OK;
}

sidwt_status sidwt_server_submit(sidwt_server *s, int32_t wave_id, sidwt_filter f, int64_t N, int J,
                                 const void *y_host, int64_t *request_id) {
    if (!s || !y_host || !request_id) {
        set_error("NULL argument");
        return SIDWT_EINVAL;
    }
    if ((int)f < 0 || (int)f > 2 || J < 1 || J > s->cfg.max_j || N < 2 || N % (int64_t(1) << J) != 0) {
        set_error("bad request shape (float filter, 1 <= J <= max_j, N a multiple of 2^J)");
        return SIDWT_EINVAL;
    }
    Request *r = new (std::nothrow) Request();
    if (!r) {
        set_error("host allocation failed");
        return SIDWT_ENOMEM;
    }
    r->wave = wave_id;
    r->filter = (int)f;
    r->N = N;
    r->J = J;
    r->y_host = y_host;
    r->arrival = Clock::now();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        if (wave_id < 0 || wave_id >= (int32_t)s->waves.size()) {
            delete r;
            set_error("unknown waveform");
            return SIDWT_EINVAL;
        }
        r->id = s->next_id++;
        if (!s->any) {
            s->first_arrival = r->arrival;
            s->any = true;
        }
        s->reqs[r->id] = r;
        s->queue.push_back(r);
    }
    s->cv_submit.notify_one();
    *request_id = r->id;
    return SIDWT_OK;
}

sidwt_status sidwt_server_wait(sidwt_server *s, int64_t request_id, double timeout_s) {
    if (!s) {
        set_error("NULL server");
        return SIDWT_EINVAL;
    }
    std::unique_lock<std::mutex> lock(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) {
        set_error("unknown request");
        return SIDWT_EINVAL;
    }
    Request *r = it->second;
    const bool ok = s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), [r] { return r->finished; });
    if (!ok) {
        set_error("request did not finish within the timeout");
        return SIDWT_ETIMEOUT;
    }
    return r->status;
}

sidwt_status sidwt_server_result(sidwt_server *s, int64_t request_id, int32_t *lag_host, float *mag_host,
                                 double *norm_host, double *latency_ms) {
    if (!s) {
        set_error("NULL server");
        return SIDWT_EINVAL;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) {
        set_error("unknown request");
        return SIDWT_EINVAL;
    }
    Request *r = it->second;
    if (!r->finished) {
        set_error("request still in flight");
        return SIDWT_EBUSY;
    }
    if (r->status) {
        set_error(r->status == SIDWT_ENOMEM     ? "request rejected: larger than a lane's share of the memory cap"
                  : r->status == SIDWT_ETIMEOUT ? "request failed: a bounded device wait of its batch ran out"
                                                : "request failed");
        return r->status;
    }
    const size_t n = r->lag.size();
    if (lag_host) std::memcpy(lag_host, r->lag.data(), n * sizeof(int32_t));
    if (mag_host) std::memcpy(mag_host, r->mag.data(), n * sizeof(float));
    if (norm_host) std::memcpy(norm_host, r->norm.data(), n * sizeof(double));
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->done - r->arrival).count();
    return SIDWT_OK;
}

sidwt_status sidwt_server_drain(sidwt_server *s, double timeout_s) {
    if (!s) {
        set_error("NULL server");
        return SIDWT_EINVAL;
    }
    std::unique_lock<std::mutex> lock(s->mu);
    const bool ok = s->cv_done.wait_for(lock, std::chrono::duration<double>(timeout_s), [s] {
        for (auto &kv : s->reqs)
            if (!kv.second->finished) return false;
        return true;
    });
    if (!ok) {
        set_error("requests still in flight after the timeout");
        return SIDWT_ETIMEOUT;
    }
    return SIDWT_OK;
}

sidwt_status sidwt_server_read_stats(sidwt_server *s, sidwt_server_stats *out, int reset) {
    if (!s || !out) {
        set_error("NULL argument");
        return SIDWT_EINVAL;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->completed = s->completed;
    out->rejected = s->rejected;
    out->batches = s->batches;
    out->max_batch = s->max_batch_seen;
    out->samples = s->samples;
    out->queued = (int64_t)s->queue.size();
    out->ref_hits = s->ref_hits;
    out->ref_stores = s->ref_stores;
    if (!s->lat_ms.empty()) {
        std::vector<double> v = s->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) { return v[(size_t)std::min<double>(v.size() - 1, p * (v.size() - 1) + 0.5)]; };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = v.back();
    }
    if (s->any && s->completed > 0)
        out->span_s = std::chrono::duration<double>(s->last_done - s->first_arrival).count();
    if (reset) {
        s->lat_ms.clear();
        s->completed = s->rejected = s->batches = s->samples = s->max_batch_seen = 0;
        s->ref_hits = s->ref_stores = 0;
        s->any = false;
        for (auto &kv : s->reqs)
            if (!kv.second->finished) {
                s->any = true;
                s->first_arrival = kv.second->arrival;
                break;
            }
    }
    return SIDWT_OK;
}

sidwt_status sidwt_server_forget(sidwt_server *s, int64_t request_id) {
    if (!s) {
        set_error("NULL server");
        return SIDWT_EINVAL;
    }
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end() || !it->second->finished) {
        set_error("unknown or unfinished request");
        return SIDWT_EINVAL;
    }
    delete it->second;
    s->reqs.erase(it);
    return SIDWT_OK;
}

sidwt_status sidwt_server_destroy(sidwt_server *s) {
    if (!s) return SIDWT_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_submit.notify_all();
    if (s->th.joinable()) s->th.join();
    cudaDeviceSynchronize();
    for (Lane &L : s->lanes) {
        if (L.rg) sidwt_ragged_destroy(L.rg);
        if (L.stream) cudaStreamDestroy(L.stream);
        if (L.done) cudaEventDestroy(L.done);
        cudaFree(L.y);
        cudaFree(L.x);
        cudaFree(L.lag_d);
        cudaFree(L.mag_d);
        cudaFree(L.norm_d);
        if (L.lag_h) cudaFreeHost(L.lag_h);
        if (L.mag_h) cudaFreeHost(L.mag_h);
        if (L.norm_h) cudaFreeHost(L.norm_h);
        if (L.err_h) cudaFreeHost(L.err_h);
    }
    for (float2 *w : s->waves) cudaFree(w);
    for (auto &kv : s->reqs) delete kv.second;
    delete s;
    return SIDWT_OK;
}

}  // extern "C"
