// Ragged batches: thousands of pulses of uneven length N, depth J and
// filter, each against its own stored signal, in one persistent correlation
// launch (optionally replayed as a CUDA graph), with tile shapes chosen by an
// autotuner.
//
// Every pair is a batch of one, so the correlation runs on the CUDA cores: a
// work item is a block of circular shifts of one (pair, scale, variant) for
// bands of 256 samples or more (each thread keeps MQ consecutive shifts and
// slides an MQ-sample window along k, MQ picked per band-length bucket by the
// autotuner), or several whole variants of a short band (one shift per
// thread).  Work items are ordered by cost, largest first, and pulled by a
// persistent grid from a device counter.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sidwt_internal.cuh"

namespace sidwt {
namespace rg {

constexpr int kT = 256;     // threads per CTA
constexpr int kTK = 64;     // k per staged chunk
constexpr int kMaxMQ = 8;   // shifts per thread, large bands
constexpr int kSmallBand = 256;
constexpr int kWin = kT * kMaxMQ + kTK;  // window samples per chunk (upper bound)

struct Item {
    int64_t pyr_off;   // received pyramid row (float2 elements)
    int64_t tree_off;  // stored SIDWT tree start
    int64_t xen_off;   // stored energies start
    int64_t slot;      // first of the J+1 peak slots (and received energies)
    int32_t N, J, ref, pad;
    int64_t r_off;     // complex64 offset of this pulse's J+1 rows of N lags in the optional r output
};

struct Work {
    int32_t item;
    int16_t j;
    int16_t mq;    // shifts per thread (large band) or 0 (short band: nvar whole variants)
    int32_t v0;    // first variant
    int32_t nvar;  // variants (short band)
    int32_t q0;    // first shift (large band)
    int32_t pad;
};

__device__ __forceinline__ int wpad(int t) { return t + (t >> 3); }

__device__ __forceinline__ unsigned long long peak_key(float2 a, uint32_t D) {
    const float m2 = a.x * a.x + a.y * a.y;
    return ((unsigned long long)__float_as_uint(m2) << 32) | (unsigned long long)(0xFFFFFFFFu - D);
}

__device__ __forceinline__ unsigned long long block_max_key(unsigned long long k, unsigned long long *red) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, k, o);
        k = t > k ? t : k;
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = k;
    __syncthreads();
    unsigned long long m = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < kT / 32; ++i) m = red[i] > m ? red[i] : m;
    return m;
}

// Long band: shifts q0 + t*MQ + l of variant v; r[q] = sum_k conj(w[k - q]) u[k].
template <int MQ>
__device__ __forceinline__ void large_tile(const Item &it, const Work &wk, int lev, int Kp, int nb, const float2 *__restrict__ tree,
                           const float2 *__restrict__ pyr, float2 *us, float2 *ws, unsigned long long *red,
                           unsigned long long *keys, float2 *R) {
    constexpr int TQ = kT * MQ;
    const int tid = threadIdx.x;
    const int N = it.N;
    const int q0 = wk.q0, v = wk.v0;
    const float2 *wa = tree + it.tree_off + 2 * (int64_t)N * (lev - 1) + (int64_t)v * Kp;
    const float2 *ua = pyr + it.pyr_off + 2 * (int64_t)N - 4 * (int64_t)Kp;
    float2 acc[MQ];
#pragma unroll
    for (int l = 0; l < MQ; ++l) acc[l] = make_float2(0.f, 0.f);
    const int base = TQ - 1 - tid * MQ;
    for (int band = 0; band < nb; ++band) {
        const float2 *w = wa + (int64_t)band * N;
        const float2 *u = ua + (int64_t)band * Kp;
        for (int k0 = 0; k0 < Kp; k0 += kTK) {
            __syncthreads();
            for (int t = tid; t < kTK; t += kT) us[t] = (k0 + t < Kp) ? u[k0 + t] : make_float2(0.f, 0.f);
            int idx = (k0 - q0 - (TQ - 1)) % Kp;
            if (idx < 0) idx += Kp;
            idx += tid;
            for (int t = tid; t < TQ + kTK - 1; t += kT) {
                while (idx >= Kp) idx -= Kp;
                ws[wpad(t)] = w[idx];
                idx += kT;
            }
            __syncthreads();
            float2 wv[MQ];
#pragma unroll
            for (int l = 0; l < MQ; ++l) wv[l] = ws[wpad(base - l)];
#pragma unroll 8
            for (int kk = 0; kk < kTK; ++kk) {
                if (kk > 0) {
#pragma unroll
                    for (int l = MQ - 1; l > 0; --l) wv[l] = wv[l - 1];
                    wv[0] = ws[wpad(base + kk)];
                }
                const float2 uv = us[kk];
#pragma unroll
                for (int l = 0; l < MQ; ++l) {
                    acc[l].x = fmaf(wv[l].x, uv.x, fmaf(wv[l].y, uv.y, acc[l].x));
                    acc[l].y = fmaf(wv[l].x, uv.y, fmaf(-wv[l].y, uv.x, acc[l].y));
                }
            }
        }
    }
    unsigned long long best = 0ull;
#pragma unroll
    for (int l = 0; l < MQ; ++l) {
        const int q = q0 + tid * MQ + l;
        if (q < Kp) {
            const uint32_t D = ((uint32_t)q << lev) + (uint32_t)v;
            const unsigned long long k = peak_key(acc[l], D);
            best = k > best ? k : best;
            if (R) R[it.r_off + (int64_t)wk.j * N + D] = acc[l];
        }
    }
    best = block_max_key(best, red);
    if (threadIdx.x == 0 && best) atomicMax(&keys[it.slot + wk.j], best);
}

// Short band: variants v0 .. v0+nvar-1, one shift per thread.
__device__ __forceinline__ void small_tile(const Item &it, const Work &wk, int lev, int Kp, int nb, const float2 *__restrict__ tree,
                           const float2 *__restrict__ pyr, float2 *sm, unsigned long long *red,
                           unsigned long long *keys, float2 *R) {
    const int tid = threadIdx.x;
    const int N = it.N;
    const int nvar = wk.nvar;
    float2 *u = sm;                   // nb * Kp
    float2 *w = sm + nb * Kp;         // [band][variant][Kp]
    const float2 *ua = pyr + it.pyr_off + 2 * (int64_t)N - 4 * (int64_t)Kp;
    const float2 *wa = tree + it.tree_off + 2 * (int64_t)N * (lev - 1) + (int64_t)wk.v0 * Kp;
    __syncthreads();
    for (int t = tid; t < nb * Kp; t += kT) u[t] = ua[t];
    for (int t = tid; t < nb * nvar * Kp; t += kT) {
        const int band = t / (nvar * Kp), r = t % (nvar * Kp);
        w[t] = wa[(int64_t)band * N + r];
    }
    __syncthreads();
    unsigned long long best = 0ull;
    if (tid < nvar * Kp) {
        const int vi = tid / Kp, q = tid % Kp;
        float2 acc = make_float2(0.f, 0.f);
        for (int band = 0; band < nb; ++band) {
            const float2 *wb = w + (band * nvar + vi) * Kp;
            const float2 *ub = u + band * Kp;
            int idx = (Kp - q) % Kp;  // (k - q) mod Kp at k = 0
            for (int k = 0; k < Kp; ++k) {
                const float2 wv = wb[idx], uv = ub[k];
                acc.x = fmaf(wv.x, uv.x, fmaf(wv.y, uv.y, acc.x));
                acc.y = fmaf(wv.x, uv.y, fmaf(-wv.y, uv.x, acc.y));
                if (++idx == Kp) idx = 0;
            }
        }
        const uint32_t D = ((uint32_t)q << lev) + (uint32_t)(wk.v0 + vi);
        best = peak_key(acc, D);
        if (R) R[it.r_off + (int64_t)wk.j * N + D] = acc;
    }
    best = block_max_key(best, red);
    if (threadIdx.x == 0 && best) atomicMax(&keys[it.slot + wk.j], best);
}

__global__ void __launch_bounds__(kT, 2) corr_ragged_kernel(const Item *__restrict__ items, const Work *__restrict__ work,
                                                         int nwork, int *counter, const float2 *__restrict__ tree,
                                                         const float2 *__restrict__ pyr,
                                                         unsigned long long *__restrict__ keys, float2 *R) {
    __shared__ float2 us[kTK];
    __shared__ float2 ws[kWin + kWin / 8 + 8];
    __shared__ unsigned long long red[kT / 32];
    __shared__ int s_w;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_w = atomicAdd(counter, 1);
        __syncthreads();
        const int w = s_w;
        if (w >= nwork) break;
        const Work wk = work[w];
        const Item it = items[wk.item];
        if (it.N == 0) continue;  // a pulse with an invalid reference id (uniform per CTA)
        const int lev = wk.j < it.J ? wk.j + 1 : it.J;
        const int Kp = it.N >> lev;
        const int nb = wk.j < it.J ? 2 : 1;
        switch (wk.mq) {
        case 0: small_tile(it, wk, lev, Kp, nb, tree, pyr, ws, red, keys, R); break;
        case 1: large_tile<1>(it, wk, lev, Kp, nb, tree, pyr, us, ws, red, keys, R); break;
        case 2: large_tile<2>(it, wk, lev, Kp, nb, tree, pyr, us, ws, red, keys, R); break;
        case 4: large_tile<4>(it, wk, lev, Kp, nb, tree, pyr, us, ws, red, keys, R); break;
        default: large_tile<8>(it, wk, lev, Kp, nb, tree, pyr, us, ws, red, keys, R); break;
        }
    }
}

__global__ void finalize_ragged_kernel(const unsigned long long *__restrict__ keys, const int32_t *__restrict__ slot_item,
                                       const Item *__restrict__ items, const double *__restrict__ xen,
                                       const double *__restrict__ yen, int64_t nslots, int32_t *__restrict__ lag,
                                       float *__restrict__ mag, double *__restrict__ norm) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslots) return;
    const Item it = items[slot_item[s]];
    const int j = (int)(s - it.slot);
    const unsigned long long k = keys[s];
    if (k == 0ull) {
        lag[s] = -1;
        mag[s] = 0.f;
        norm[s] = 0.0;
        return;
    }
    const uint32_t D = 0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFull);
    const float m = sqrtf(__uint_as_float((uint32_t)(k >> 32)));
    lag[s] = (int32_t)D;
    mag[s] = m;
    const double den = sqrt(xen[it.xen_off + ((1 << j) - 1) + (D & ((1u << j) - 1u))] * yen[s]);
    norm[s] = den > 0.0 ? (double)m / den : 0.0;
}

// Items of a uniform plan batch: pulse b uses reference ref_ids[b].
__global__ void plan_items_kernel(const int32_t *__restrict__ ref_ids, int B, int nrefs, int N, int J,
                                  int64_t pyr_elems, int64_t tree_elems, int64_t xen_len, Item *__restrict__ items) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const int r = ref_ids[b];
    const bool ok = r >= 0 && r < nrefs;
    items[b] = Item{(int64_t)b * pyr_elems, ok ? (int64_t)r * tree_elems : 0, ok ? (int64_t)r * xen_len : 0,
                    (int64_t)b * (J + 1), ok ? N : 0, J, r, 0, (int64_t)b * (J + 1) * N};
}

// Latency path for a few short pulses of a plan: every (pulse, scale,
// variant, block of 32 delays) is its own CTA, and its 8 warps split the
// contraction (k) into 8 slices, so that even one pulse spreads over the
// whole GPU.  r_j[2^l q + v] = sum_k conj(w_v[(k - q) mod K']) u[k] per band
// (eq. 20 / 20a with the variant delayed by q).
struct LatScale {
    int32_t j, lev, Kp, nv, nqb, first;
};
struct LatTable {
    LatScale t[16];
    int n;
};
constexpr int kLatMaxN = 8192;
constexpr int kLatStageW = 4096;  // stored-band samples a CTA stages (both bands of a variant)
constexpr int kLatChunk = 1024;   // received samples staged at a time

__global__ void __launch_bounds__(256) corr_latency_kernel(const float2 *__restrict__ tree, int64_t tree_elems,
                                                           const float2 *__restrict__ pyr, int64_t pyr_elems,
                                                           const int32_t *__restrict__ ref_ids, int nrefs, int64_t N,
                                                           int J, LatTable tab, unsigned long long *__restrict__ keys,
                                                           float2 *__restrict__ R, int32_t *__restrict__ saved,
                                                           int32_t *__restrict__ err) {
    __shared__ float2 part[8][33];
    __shared__ float2 lat_sm[kLatStageW + kLatChunk];  // 40 KB
    pdl_wait();  // the analysis kernel's pyramid and energies
    pdl_release();
    const int b = blockIdx.y;
    const int ref = ref_ids[b];
    if (blockIdx.x == 0 && threadIdx.x == 0) {  // the ids the peak epilogue reads, and the error record
        saved[b] = ref;
        if (ref < 0 || ref >= nrefs) atomicOr(err, kErrBadRefId);
    }
    if (ref < 0 || ref >= nrefs) return;  // invalid pulse: its keys stay 0 (lag -1)
    const int task = blockIdx.x;
    int k = 0;
    while (k + 1 < tab.n && task >= tab.t[k + 1].first) ++k;
    const LatScale z = tab.t[k];
    const int local = task - z.first;
    const int v = local / z.nqb, qb = local % z.nqb;
    const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
    const int q = qb * 32 + lane;
    const int Kp = z.Kp;
    const int nb = z.j < J ? 2 : 1;
    const int K = nb * Kp;
    const float2 *u0 = pyr + (int64_t)b * pyr_elems + 2 * N - 4 * (int64_t)Kp;
    const float2 *w0 = tree + (int64_t)ref * tree_elems + 2 * N * (int64_t)(z.lev - 1) + (int64_t)v * Kp;
    const int qq = q < Kp ? q : 0;
    float ar = 0.f, ai = 0.f;
    if (nb * Kp <= kLatStageW) {
        // the variant's band(s) and the received band, chunk by chunk, in
        // shared memory (coalesced loads, one L2 round trip per chunk); slice
        // s takes its eighth of each chunk, which for K <= kLatChunk is the
        // same partition of k as the direct form below
        float2 *ws = lat_sm, *us = lat_sm + kLatStageW;
        for (int t = threadIdx.x; t < nb * Kp; t += blockDim.x) {
            const int band = t >= Kp ? 1 : 0;
            ws[t] = w0[(int64_t)band * N + (t - band * Kp)];
        }
        for (int c0 = 0; c0 < K; c0 += kLatChunk) {
            const int cnt = min(kLatChunk, K - c0);
            for (int t = threadIdx.x; t < cnt; t += blockDim.x) us[t] = u0[c0 + t];
            __syncthreads();
            const int per = (cnt + 7) / 8;
            const int a0 = slice * per, a1 = min(cnt, a0 + per);
            for (int i = a0; i < a1; ++i) {
                const int kk = c0 + i;
                const int band = kk >= Kp ? 1 : 0;
                int idx = kk - band * Kp - qq;
                if (idx < 0) idx += Kp;
                const float2 wv = ws[band * Kp + idx];
                const float2 uv = us[i];
                ar = fmaf(wv.x, uv.x, fmaf(wv.y, uv.y, ar));
                ai = fmaf(wv.x, uv.y, fmaf(-wv.y, uv.x, ai));
            }
            __syncthreads();  // the chunk's reads end before the next chunk overwrites it
        }
    } else {
        const int per = (K + 7) / 8;
        const int k0 = slice * per, k1 = min(K, k0 + per);
        for (int kk = k0; kk < k1; ++kk) {
            const int band = kk >= Kp ? 1 : 0;
            int idx = kk - band * Kp - qq;
            if (idx < 0) idx += Kp;
            const float2 wv = w0[(int64_t)band * N + idx];
            const float2 uv = u0[kk];
            ar = fmaf(wv.x, uv.x, fmaf(wv.y, uv.y, ar));
            ai = fmaf(wv.x, uv.y, fmaf(-wv.y, uv.x, ai));
        }
    }
    part[slice][lane] = make_float2(ar, ai);
    __syncthreads();
    if (slice == 0) {
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            sr += part[i][lane].x;
            si += part[i][lane].y;
        }
        unsigned long long key = 0ull;
        if (q < Kp) {
            const uint32_t D = ((uint32_t)q << z.lev) + (uint32_t)v;
            key = peak_key(make_float2(sr, si), D);
            if (R) R[((int64_t)b * (J + 1) + z.j) * N + D] = make_float2(sr, si);
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, key, o);
            key = t > key ? t : key;
        }
        if (lane == 0 && key) atomicMax(&keys[(int64_t)b * (J + 1) + z.j], key);
    }
}

__global__ void fill_kernel(float2 *x, int64_t n, uint32_t seed) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t h = (uint32_t)i * 2654435761u ^ seed;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    x[i] = make_float2((float)(h & 0xffff) / 32768.f - 1.f, (float)(h >> 16) / 32768.f - 1.f);
}

}  // namespace rg
}  // namespace sidwt

using namespace sidwt;

struct RefInfo {
    int filter;
    int64_t N;
    int J;
    int64_t tree_off, xen_off;
    int64_t tc_off[16];  // stored tensor-core operand of scale j (bf16 elements), -1: none
    int16_t tc_S[16];    // its tile width, fixed when it was packed
};

struct RaggedLayout {  // everything a batch needs on the device, built on the host
    std::vector<rg::Item> items;
    std::vector<rg::Work> work;
    std::vector<RaggedLift> lift[2 + kPipeClasses][3];  // [path: unused, long, pipelined by size class][filter]
    std::vector<RaggedTile> tiles[3];    // tiled long pulses, by filter
    std::vector<RaggedTail> tails[3];
    int64_t maxN_tail[3] = {0, 0, 0};
    int64_t part_elems = 0;
    std::vector<int32_t> slot_item;
    // tensor-core part: one received-operand entry and two tensor maps per
    // (pair, scale), tiles in cost order
    std::vector<rtc::TcTile> tc_tiles;
    std::vector<rtc::TcSplit> tc_splits;  // tiles whose contraction runs as several parts
    int64_t tc_part_elems = 0;            // complex64 elements of those parts' accumulators
    int tc_split_maxS = 0;
    // one entry per tensor-core (pair, scale): its shape and stored operand
    std::vector<rtc::Shape> recv_shape;
    std::vector<int64_t> recv_a_off;
    std::vector<unsigned char> maps;
    int64_t pyr_elems = 0, slots = 0;
    int64_t r_elems = 0;  // complex64 elements of the optional r output: sum of (J_i + 1) N_i
    int64_t maxN[2 + kPipeClasses][3] = {};
    int maxJ_long[3] = {0, 0, 0};
};

struct DevLayout {  // device copy of a RaggedLayout
    rg::Item *items = nullptr;
    rg::Work *work = nullptr;
    RaggedLift *lift = nullptr;
    int32_t *slot_item = nullptr;
    rtc::TcTile *tc_tiles = nullptr;
    unsigned char *maps = nullptr;
    RaggedTile *lt = nullptr;   // tiled long pulses (all filters, filter-major)
    RaggedTail *ltail = nullptr;
    rtc::TcSplit *splits = nullptr;
    int64_t cap_items = 0, cap_work = 0, cap_lift = 0, cap_slots = 0, cap_tiles = 0, cap_maps = 0, cap_lt = 0,
            cap_ltail = 0, cap_splits = 0;
    int n_splits = 0, split_maxS = 0;
    RaggedLiftGroups groups;
    int nwork = 0, n_tc_tiles = 0;
};

struct sidwt_ragged {
    std::vector<RefInfo> refs;
    float2 *tree = nullptr;
    int64_t tree_cap = 0, tree_used = 0;
    // tensor-core path (SIDWT_PREC_BF16X3): stored operands of the references
    // packed at store time (the received windows are expanded on chip), error flag
    int prec = SIDWT_PREC_FP32;
    // split contractions (sidwt_ragged_set_split): 0 when a batch has too few
    // tiles to fill the GPU, 1 never, 2 every tile long enough (tests)
    int split_mode = 0;
    float2 *tcpart = nullptr;
    int64_t tcpart_cap = 0;
    __nv_bfloat16 *tc_a = nullptr;
    int64_t tc_a_cap = 0, tc_a_used = 0;
    int32_t *err = nullptr;
    double *xen = nullptr;
    int64_t xen_cap = 0, xen_used = 0;
    // batch workspace
    float2 *pyr = nullptr;
    int64_t pyr_cap = 0;
    double *yen = nullptr;
    double *part = nullptr;  // energy partials of the tiled long pulses
    int64_t part_cap = 0;
    unsigned long long *keys = nullptr;
    int32_t *lag = nullptr;
    float *mag = nullptr;
    double *norm = nullptr;
    int64_t slot_cap = 0;
    int *counter = nullptr;
    DevLayout dl;       // layout of direct correlate calls
    DevLayout gl;       // layout owned by the captured graph
    void *h_stage = nullptr;
    size_t h_stage_bytes = 0;
    cudaEvent_t stage_done = nullptr;  // recorded after the last upload's copies from h_stage
    int64_t last_slots = -1;
    // graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t graph_slots = 0;
    int graph_launches = 0;
    // tuning: shifts per thread by floor(log2(band length)); tensor-core tile
    // width weights (applied to references stored afterwards)
    int mq_for[32];
    rtc::TcWeights tcw;
    int sms = 0;
    // stage timing of direct calls (CUDA events), as for plans
    bool timing = false;
    std::vector<cudaEvent_t> ev;  // 4 per timed call: before lift, corr, peaks, after
    double t_ms[3] = {0, 0, 0};
    int64_t timed_calls = 0, timed_launches = 0;
};

namespace {

template <typename T>
sidwt_status grow(T **p, int64_t *cap, int64_t need, int64_t keep, const char *what) {
    if (need <= *cap) return SIDWT_OK;
    const int64_t nc = std::max<int64_t>(need, *cap * 2);
    T *q = nullptr;
    if (cudaMalloc(&q, (size_t)nc * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("device allocation failed: ") + what);
        return SIDWT_ENOMEM;
    }
    if (*p) {
        if (keep > 0) cudaMemcpy(q, *p, (size_t)keep * sizeof(T), cudaMemcpyDeviceToDevice);
        cudaFree(*p);
    }
    *p = q;
    *cap = nc;
    return SIDWT_OK;
}

int default_mq(int lg) { return lg >= 11 ? 8 : (lg >= 10 ? 4 : (lg >= 9 ? 2 : 1)); }

// A tile whose contraction (2 K' samples at the long scales) is long against
// the batch's whole work keeps its SM busy after the others have finished:
// such tiles are cut into parts of at least kMinPartKB K-blocks, never across the
// band boundary, each a work item of its own whose accumulators go to the
// partials buffer; tc_split_reduce then sums them and forms the peaks.
constexpr int kMinPartKB = 8;
constexpr int kMaxParts = 64;

void split_long_tiles(const sidwt_ragged *r, std::vector<std::pair<int64_t, rtc::TcTile>> &tct, RaggedLayout &L) {
    if (tct.empty() || r->split_mode == 1) return;
    int64_t total_kb = 0;
    for (const auto &x : tct) total_kb += (int64_t)x.second.nb * x.second.nkb;
    const int64_t items = 2 * (int64_t)std::max(1, r->sms);
    // K-blocks per work item that would spread the batch over about `items`
    // items; a tile with more than twice that is cut (a large batch, whose
    // tiles are many and short against the batch, cuts none)
    const int64_t target = std::max<int64_t>(kMinPartKB, (total_kb + items - 1) / items);
    std::vector<std::pair<int64_t, rtc::TcTile>> out;
    out.reserve(tct.size());
    for (const auto &x : tct) {
        const rtc::TcTile &w = x.second;
        const int nb = w.nb, nkb = w.nkb, F = nb * nkb;
        int P = r->split_mode == 2 ? F / kMinPartKB : (F >= 2 * target ? (int)((F + target - 1) / target) : 1);
        P = std::min(P, kMaxParts);
        const int per_band = (P + nb - 1) / nb;  // parts per band
        if (P < 2 || nkb / per_band < kMinPartKB) {
            out.push_back(x);
            continue;
        }
        rtc::TcSplit sp;
        sp.slot = w.slot;
        sp.slot_mid = w.slot_mid;
        sp.r_at = w.r_at;
        sp.r_mid = w.r_mid;
        sp.part_first = L.tc_part_elems;
        sp.nparts = per_band * nb;
        sp.nparts0 = per_band;  // band 0's parts come first
        sp.tile = w.tile;
        sp.gv = w.gv;
        sp.nv = w.nv;
        sp.Kp = w.Kp;
        sp.lev = w.lev;
        sp.S = w.S;
        for (int b = 0; b < nb; ++b)
            for (int k = 0; k < per_band; ++k) {
                const int k0 = (int)((int64_t)nkb * k / per_band), k1 = (int)((int64_t)nkb * (k + 1) / per_band);
                rtc::TcTile part = w;
                part.slot_mid = -1;
                part.f0 = b * nkb + k0;
                part.fcnt = k1 - k0;
                part.part_off = L.tc_part_elems;
                L.tc_part_elems += (int64_t)w.S * 128;
                out.push_back({(int64_t)part.fcnt * w.S, part});
            }
        L.tc_splits.push_back(sp);
        L.tc_split_maxS = std::max<int>(L.tc_split_maxS, w.S);
    }
    tct.swap(out);
}

// Builds the device-side description of a batch on the host.
sidwt_status build_layout(const sidwt_ragged *r, int64_t n, const int32_t *ref_ids, const int64_t *y_off,
                          int64_t y_elems, RaggedLayout &L) {
    L = RaggedLayout();
    L.items.resize((size_t)n);
    const int64_t pipe_max = analyze_pipe_max_n();
    for (int64_t i = 0; i < n; ++i) {
        const int32_t rid = ref_ids[i];
        if (rid < 0 || rid >= (int32_t)r->refs.size()) {
            set_error("reference id out of range in item " + std::to_string(i));
            return SIDWT_EINVAL;
        }
        if (y_off[i] < 0 || (y_off[i] & 1)) {
            set_error("pulse offsets must be even and non-negative (16-byte aligned pulses)");
            return SIDWT_EINVAL;
        }
        const RefInfo &ri = r->refs[(size_t)rid];
        if (y_off[i] + ri.N > y_elems) {
            set_error("item " + std::to_string(i) + " runs past the end of the pulse buffer");
            return SIDWT_EINVAL;
        }
        rg::Item &it = L.items[(size_t)i];
        it.pyr_off = L.pyr_elems;
        it.tree_off = ri.tree_off;
        it.xen_off = ri.xen_off;
        it.slot = L.slots;
        it.N = (int32_t)ri.N;
        it.J = ri.J;
        it.ref = rid;
        it.pad = 0;
        it.r_off = L.r_elems;
        L.r_elems += (int64_t)(ri.J + 1) * ri.N;
        RaggedLift lf{y_off[i], L.pyr_elems, L.slots, (int32_t)ri.N, ri.J};
        const int Lv = std::min(ri.J, kTileLevels);
        const bool tiled = ri.N > pipe_max && (ri.J == Lv || (ri.N >> Lv) <= tile_tail_max_n());
        if (tiled) {
            const int nt = (int)((ri.N + kTileSamples - 1) / kTileSamples);
            for (int k = 0; k < nt; ++k) {
                const int64_t t0 = (int64_t)k * kTileSamples;
                L.tiles[ri.filter].push_back(RaggedTile{y_off[i], L.pyr_elems, L.part_elems + (int64_t)k * (kTileLevels + 1),
                                                        (int32_t)ri.N, Lv, (int32_t)t0,
                                                        (int32_t)std::min<int64_t>(kTileSamples, ri.N - t0)});
            }
            L.tails[ri.filter].push_back(RaggedTail{lf, L.part_elems, nt, Lv});
            if (ri.J > Lv) L.maxN_tail[ri.filter] = std::max<int64_t>(L.maxN_tail[ri.filter], ri.N >> Lv);
            L.part_elems += (int64_t)nt * (kTileLevels + 1);
        }
        int path = 1;  // per-level windows: pulses too long for the tiles' tail
        for (int k = kPipeClasses - 1; k >= 0; --k)
            if (ri.N <= analyze_pipe_class_max(k)) path = 2 + k;
        if (!tiled) L.lift[path][ri.filter].push_back(lf);
        if (!tiled) {
            L.maxN[path][ri.filter] = std::max<int64_t>(L.maxN[path][ri.filter], ri.N);
            if (path == 1) L.maxJ_long[ri.filter] = std::max(L.maxJ_long[ri.filter], ri.J);
        }
        for (int j = 0; j <= ri.J; ++j) L.slot_item.push_back((int32_t)i);
        L.pyr_elems += 2 * ri.N - 2 * (ri.N >> ri.J);
        L.slots += ri.J + 1;
    }
    // the pipelined kernel's persistent CTAs take the pulses in list order: longest first
    for (int k = 2; k < 2 + kPipeClasses; ++k)
        for (int f = 0; f < 3; ++f)
            std::stable_sort(L.lift[k][f].begin(), L.lift[k][f].end(),
                             [](const RaggedLift &a, const RaggedLift &b) { return a.N > b.N; });
    // work items, bucketed by log2 of their cost, largest first
    std::vector<std::vector<rg::Work>> buckets(64);
    std::vector<std::pair<int64_t, rtc::TcTile>> tct;  // (cost, tile)
    for (int64_t i = 0; i < n; ++i) {
        const rg::Item &it = L.items[(size_t)i];
        const RefInfo &ri = r->refs[(size_t)it.ref];
        // scale J (eq. 20a) is band 0 of scale J - 1 (eq. 20) at the same level: its
        // peak is formed by the scale J - 1 tiles before they add band 1
        const bool mergeJ = r->prec == SIDWT_PREC_BF16X3 && it.J >= 1 && it.J < 16 && ri.tc_off[it.J] >= 0 &&
                            ri.tc_off[it.J - 1] >= 0 && ri.tc_S[it.J] == ri.tc_S[it.J - 1];
        for (int j = 0; j <= it.J; ++j) {
            if (j == it.J && mergeJ) continue;
            rtc::Shape sh;
            if (r->prec == SIDWT_PREC_BF16X3 && j < 16 && ri.tc_off[j] >= 0 &&
                rtc::shape_with(it.N, it.J, j, ri.tc_S[j], &sh)) {
                const int e = (int)L.recv_shape.size();
                L.recv_shape.push_back(sh);
                L.recv_a_off.push_back(ri.tc_off[j]);
                for (int t = 0; t < sh.tiles; ++t) {
                    rtc::TcTile w;
                    w.map = e;
                    w.tile = t;
                    w.nkb = sh.nkb;
                    w.Kp = (int32_t)sh.Kp;
                    w.gv = sh.gv;
                    w.nv = sh.nv;
                    w.nb = (int16_t)sh.nb;
                    w.lev = (int16_t)sh.lev;
                    w.S = (int16_t)sh.S;
                    w.k0 = (int16_t)sh.k0;
                    w.slot = it.slot + j;
                    w.u_off = it.pyr_off + 2 * (int64_t)it.N - 4 * sh.Kp;
                    w.slot_mid = (mergeJ && j == it.J - 1) ? it.slot + it.J : -1;
                    w.r_at = it.r_off + (int64_t)j * it.N;
                    w.r_mid = it.r_off + (int64_t)it.J * it.N;
                    tct.push_back({(int64_t)sh.nb * sh.nkb * sh.S, w});
                }
                continue;
            }
            const int lev = j < it.J ? j + 1 : it.J;
            const int64_t Kp = (int64_t)it.N >> lev;
            const int nb = j < it.J ? 2 : 1;
            const int nv = 1 << lev;
            if (Kp >= rg::kSmallBand) {
                int lg = 0;
                while ((int64_t(2) << lg) <= Kp) ++lg;
                int mq = r->mq_for[std::min(lg, 31)];
                while (mq > 1 && (int64_t)rg::kT * mq > Kp) mq >>= 1;
                const int64_t TQ = (int64_t)rg::kT * mq;
                const double cost = (double)TQ * nb * Kp;
                int b = std::max(0, std::min(63, (int)std::log2(std::max(1.0, cost))));
                for (int v = 0; v < nv; ++v)
                    for (int64_t q0 = 0; q0 < Kp; q0 += TQ)
                        buckets[b].push_back({(int32_t)i, (int16_t)j, (int16_t)mq, v, 1, (int32_t)q0, 0});
            } else {
                const int nvar = std::max<int>(1, (int)(rg::kT / Kp));
                for (int v0 = 0; v0 < nv; v0 += nvar) {
                    const int cnt = std::min(nvar, nv - v0);
                    const double cost = (double)cnt * Kp * nb * Kp;
                    int b = std::max(0, std::min(63, (int)std::log2(std::max(1.0, cost))));
                    buckets[b].push_back({(int32_t)i, (int16_t)j, 0, v0, cnt, 0, 0});
                }
            }
        }
    }
    for (int b = 63; b >= 0; --b) L.work.insert(L.work.end(), buckets[b].begin(), buckets[b].end());
    split_long_tiles(r, tct, L);
    std::stable_sort(tct.begin(), tct.end(), [](const std::pair<int64_t, rtc::TcTile> &a,
                                                const std::pair<int64_t, rtc::TcTile> &b) { return a.first > b.first; });
    L.tc_tiles.reserve(tct.size());
    for (const auto &x : tct) L.tc_tiles.push_back(x.second);
    if (L.work.size() > 0x7fffffff || L.tc_tiles.size() > 0x7fffffff || L.recv_shape.size() > 0x7fffffff) {
        set_error("too many work items");
        return SIDWT_EINVAL;
    }
    return SIDWT_OK;
}

sidwt_status ensure_dev(DevLayout &d, const RaggedLayout &L) {
    int64_t nl = 0;
    for (int p = 0; p < 2 + kPipeClasses; ++p)
        for (int f = 0; f < 3; ++f) nl += (int64_t)L.lift[p][f].size();
    sidwt_status st;
    if ((st = grow(&d.items, &d.cap_items, (int64_t)L.items.size(), 0, "ragged items")) ||
        (st = grow(&d.work, &d.cap_work, (int64_t)L.work.size(), 0, "ragged work list")) ||
        (st = grow(&d.lift, &d.cap_lift, nl, 0, "ragged lifting list")) ||
        (st = grow(&d.slot_item, &d.cap_slots, L.slots, 0, "ragged slot map")) ||
        (st = grow(&d.tc_tiles, &d.cap_tiles, (int64_t)L.tc_tiles.size(), 0, "tensor-core tile list")) ||
        (st = grow(&d.maps, &d.cap_maps, (int64_t)L.maps.size(), 0, "tensor maps")))
        return st;
    int64_t nt = 0, ntl = 0;
    for (int f = 0; f < 3; ++f) {
        nt += (int64_t)L.tiles[f].size();
        ntl += (int64_t)L.tails[f].size();
    }
    if ((st = grow(&d.lt, &d.cap_lt, nt, 0, "ragged analysis tiles")) ||
        (st = grow(&d.ltail, &d.cap_ltail, ntl, 0, "ragged analysis tails")) ||
        (st = grow(&d.splits, &d.cap_splits, (int64_t)L.tc_splits.size(), 0, "split tensor-core tiles")))
        return st;
    return SIDWT_OK;
}

// Tensor maps of the layout's tensor-core entries (needs the object's
// operand buffers, so after ensure_workspace).
sidwt_status encode_layout_maps(const sidwt_ragged *r, RaggedLayout &L) {
    const size_t mb = rtc::map_bytes();
    L.maps.assign(L.recv_shape.size() * 2 * mb, 0);
    for (size_t e = 0; e < L.recv_shape.size(); ++e) {
        sidwt_status st = rtc::encode_maps(L.maps.data() + e * 2 * mb, r->tc_a + L.recv_a_off[e], nullptr,
                                           L.recv_shape[e]);
        if (st) return st;
    }
    return SIDWT_OK;
}

// Copies a layout to the device (synchronously when stage is null).
sidwt_status upload(sidwt_ragged *r, DevLayout &d, const RaggedLayout &L, cudaStream_t s, bool sync) {
    sidwt_status st = ensure_dev(d, L);
    if (st) return st;
    std::vector<RaggedLift> lift;
    int64_t base = 0;
    RaggedLiftGroups g;
    for (int p = 0; p < 2 + kPipeClasses; ++p)
        for (int f = 0; f < 3; ++f) {
            const auto &v = L.lift[p][f];
            if (p >= 2) {
                g.pipe[p - 2][f] = d.lift + base;
                g.n_pipe[p - 2][f] = (int)v.size();
                g.maxN_pipe[p - 2][f] = L.maxN[p][f];
            } else if (p == 1) {
                g.lng[f] = d.lift + base;
                g.n_long[f] = (int)v.size();
                g.maxN_long[f] = L.maxN[1][f];
                g.maxJ_long[f] = L.maxJ_long[f];
            }
            lift.insert(lift.end(), v.begin(), v.end());
            base += (int64_t)v.size();
        }
    std::vector<RaggedTile> tiles;
    std::vector<RaggedTail> tails;
    for (int f = 0; f < 3; ++f) {
        g.tiles[f] = d.lt + tiles.size();
        g.n_tiles[f] = (int)L.tiles[f].size();
        g.tails[f] = d.ltail + tails.size();
        g.n_tails[f] = (int)L.tails[f].size();
        g.maxN_tail[f] = L.maxN_tail[f];
        tiles.insert(tiles.end(), L.tiles[f].begin(), L.tiles[f].end());
        tails.insert(tails.end(), L.tails[f].begin(), L.tails[f].end());
    }
    d.groups = g;
    d.n_splits = (int)L.tc_splits.size();
    d.split_maxS = L.tc_split_maxS;
    d.nwork = (int)L.work.size();
    d.n_tc_tiles = (int)L.tc_tiles.size();
    const size_t b1 = L.items.size() * sizeof(rg::Item), b2 = L.work.size() * sizeof(rg::Work);
    const size_t b3 = lift.size() * sizeof(RaggedLift), b4 = L.slot_item.size() * sizeof(int32_t);
    const size_t b5 = L.tc_tiles.size() * sizeof(rtc::TcTile);
    const size_t b7 = L.maps.size();
    const size_t b8 = tiles.size() * sizeof(RaggedTile), b9 = tails.size() * sizeof(RaggedTail);
    const size_t b10 = L.tc_splits.size() * sizeof(rtc::TcSplit);
    cudaError_t e = cudaSuccess;
    if (sync) {
        if (b1) e = cudaMemcpy(d.items, L.items.data(), b1, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && b2) e = cudaMemcpy(d.work, L.work.data(), b2, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && b3) e = cudaMemcpy(d.lift, lift.data(), b3, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && b4) e = cudaMemcpy(d.slot_item, L.slot_item.data(), b4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && b5) e = cudaMemcpy(d.tc_tiles, L.tc_tiles.data(), b5, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && b7) e = cudaMemcpy(d.maps, L.maps.data(), b7, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && b8) e = cudaMemcpy(d.lt, tiles.data(), b8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && b9) e = cudaMemcpy(d.ltail, tails.data(), b9, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && b10) e = cudaMemcpy(d.splits, L.tc_splits.data(), b10, cudaMemcpyHostToDevice);
        return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "ragged layout upload");
    }
    // asynchronous: through the object's pinned staging buffer (the previous
    // upload has been consumed once the stream reaches this point)
    const size_t tot = b1 + b2 + b3 + b4 + b5 + b7 + b8 + b9 + b10 + 9 * 16;
    if (tot > r->h_stage_bytes) {
        cudaStreamSynchronize(s);
        if (r->h_stage) cudaFreeHost(r->h_stage);
        r->h_stage = nullptr;
        r->h_stage_bytes = 0;
        if (cudaMallocHost(&r->h_stage, tot * 2) != cudaSuccess) {
            cudaGetLastError();
            set_error("pinned staging allocation failed");
            return SIDWT_ENOMEM;
        }
        r->h_stage_bytes = tot * 2;
    } else if (r->stage_done) {
        // the staging buffer may still feed the previous upload's copies: wait
        // for those alone, not for the rest of the stream
        cudaEventSynchronize(r->stage_done);
    }
    char *h = static_cast<char *>(r->h_stage);
    size_t o = 0;
    auto put = [&](void *dst, const void *src, size_t n) {
        if (!n || e != cudaSuccess) return;
        std::memcpy(h + o, src, n);
        e = cudaMemcpyAsync(dst, h + o, n, cudaMemcpyHostToDevice, s);
        o += (n + 15) & ~size_t(15);
    };
    put(d.items, L.items.data(), b1);
    put(d.work, L.work.data(), b2);
    put(d.lift, lift.data(), b3);
    put(d.slot_item, L.slot_item.data(), b4);
    put(d.tc_tiles, L.tc_tiles.data(), b5);
    put(d.maps, L.maps.data(), b7);
    put(d.lt, tiles.data(), b8);
    put(d.ltail, tails.data(), b9);
    put(d.splits, L.tc_splits.data(), b10);
    if (e == cudaSuccess && !r->stage_done) e = cudaEventCreateWithFlags(&r->stage_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(r->stage_done, s);
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "ragged layout upload");
}

sidwt_status ensure_workspace(sidwt_ragged *r, const RaggedLayout &L) {
    sidwt_status st;
    if ((st = grow(&r->pyr, &r->pyr_cap, L.pyr_elems, 0, "ragged pyramid"))) return st;
    if ((st = grow(&r->part, &r->part_cap, L.part_elems, 0, "ragged analysis partials"))) return st;
    if ((st = grow(&r->tcpart, &r->tcpart_cap, L.tc_part_elems, 0, "split-contraction partials"))) return st;
    if (L.slots > r->slot_cap) {
        int64_t c0 = r->slot_cap, c1 = r->slot_cap, c2 = r->slot_cap, c3 = r->slot_cap, c4 = r->slot_cap;
        if ((st = grow(&r->yen, &c0, L.slots, 0, "ragged energies")) ||
            (st = grow(&r->keys, &c1, L.slots, 0, "ragged keys")) || (st = grow(&r->lag, &c2, L.slots, 0, "ragged lags")) ||
            (st = grow(&r->mag, &c3, L.slots, 0, "ragged magnitudes")) ||
            (st = grow(&r->norm, &c4, L.slots, 0, "ragged norms")))
            return st;
        r->slot_cap = c0;
    }
    if (!r->counter && cudaMalloc(&r->counter, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation failed: work counter");
        return SIDWT_ENOMEM;
    }
    return SIDWT_OK;
}

// The launches of one batch (all capturable; events only outside capture).
sidwt_status enqueue(sidwt_ragged *r, const DevLayout &d, int64_t slots, int64_t nitems, const float2 *y, cudaStream_t s,
                     int *launches, float2 *R = nullptr) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    const bool timed = r->timing && cap == cudaStreamCaptureStatusNone;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    if (timed)
        for (int i = 0; i < 4; ++i)
            if (cudaEventCreate(&ev[i]) != cudaSuccess) {
                cudaGetLastError();
                return cuda_fail(cudaErrorMemoryAllocation, "timing events");
            }
    if (timed) cudaEventRecord(ev[0], s);
    int nl = 0;
    sidwt_status st = analyze_ragged(y, d.groups, r->pyr, r->yen, r->part, r->err, s, &nl);
    if (st) return st;
    cudaError_t e = cudaMemsetAsync(r->keys, 0, (size_t)slots * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(r->counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "ragged memset");
    if (timed) cudaEventRecord(ev[1], s);
    if (d.n_tc_tiles > 0) {
        if ((st = rtc::launch_corr(d.maps, d.tc_tiles, d.n_tc_tiles, r->pyr, r->keys, r->err, r->sms, s, R,
                                   d.n_splits > 0 ? r->tcpart : nullptr)))
            return st;
        nl += 1;
        if (d.n_splits > 0) {
            if ((st = rtc::launch_split_reduce(d.splits, d.n_splits, d.split_maxS, r->tcpart, r->keys, R, s)))
                return st;
            nl += 1;
        }
    }
    if (d.nwork > 0) {
        rg::corr_ragged_kernel<<<r->sms * 2, rg::kT, 0, s>>>(d.items, d.work, d.nwork, r->counter, r->tree, r->pyr,
                                                              r->keys, R);
        ++nl;
    }
    if (timed) cudaEventRecord(ev[2], s);
    if (slots > 0) {
        rg::finalize_ragged_kernel<<<(unsigned)((slots + 255) / 256), 256, 0, s>>>(
            r->keys, d.slot_item, d.items, r->xen, r->yen, slots, r->lag, r->mag, r->norm);
        ++nl;
    }
    if (timed) {
        cudaEventRecord(ev[3], s);
        r->ev.insert(r->ev.end(), ev, ev + 4);
        ++r->timed_calls;
        r->timed_launches += nl;
    }
    (void)nitems;
    if (launches) *launches = nl;
    e = cudaGetLastError();
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "ragged correlation launch");
}

// Cache file lines: "<log2 band> <shifts per thread>" for the CUDA-core
// tiles, "tc <tile width> <log2 band> <weight>" for the tensor-core tiles.
void load_tuning(sidwt_ragged *r, const char *path) {
    for (int i = 0; i < 32; ++i) r->mq_for[i] = default_mq(i);
    rtc::default_weights(&r->tcw);
    if (!path) path = std::getenv("SIDWT_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char line[128];
    while (std::fgets(line, sizeof line, f)) {
        int lg, mq, S;
        float w;
        if (std::sscanf(line, "tc %d %d %f", &S, &lg, &w) == 3) {
            int k = -1;
            for (int q = 0; q < rtc::kTcWidths; ++q)
                if (rtc::kTcWidth[q] == S) k = q;
            if (k >= 0 && lg >= 0 && lg < rtc::kTcBuckets && w > 0.1f && w < 100.f) r->tcw.w[k][lg] = w;
        } else if (std::sscanf(line, "%d %d", &lg, &mq) == 2) {
            if (lg >= 0 && lg < 32 && (mq == 1 || mq == 2 || mq == 4 || mq == 8)) r->mq_for[lg] = mq;
        }
    }
    std::fclose(f);
}

}  // namespace

namespace sidwt {

// Small batches of a uniform plan: every pulse is a batch of one on the
// persistent kernel (a 64-pulse SIMT tile would be mostly empty).
struct PlanSmall {
    rg::Item *items = nullptr;
    rg::Work *work = nullptr;
    int *counter = nullptr;
    int64_t built_B = -1;
    int nwork = 0;
};

void free_small(sidwt_plan *p) {
    PlanSmall *ps = static_cast<PlanSmall *>(p->small);
    if (!ps) return;
    cudaFree(ps->items);
    cudaFree(ps->work);
    cudaFree(ps->counter);
    delete ps;
    p->small = nullptr;
}

// Allocates and fills the device work list for batches of B pulses (outside
// any capture: later calls with the same B reuse it).
sidwt_status prepare_small(sidwt_plan *p, int64_t B) {
    PlanSmall *ps = static_cast<PlanSmall *>(p->small);
    if (ps && ps->built_B == B) return SIDWT_OK;
    free_small(p);
    ps = new (std::nothrow) PlanSmall();
    if (!ps) {
        set_error("host allocation failed");
        return SIDWT_ENOMEM;
    }
    p->small = ps;
    std::vector<rg::Work> one;
    for (int j = 0; j <= p->J; ++j) {
        const int lev = j < p->J ? j + 1 : p->J;
        const int64_t Kp = p->N >> lev;
        const int nv = 1 << lev;
        if (Kp >= rg::kSmallBand) {
            int lg = 0;
            while ((int64_t(2) << lg) <= Kp) ++lg;
            int mq = default_mq(std::min(lg, 31));
            while (mq > 1 && (int64_t)rg::kT * mq > Kp) mq >>= 1;
            const int64_t TQ = (int64_t)rg::kT * mq;
            for (int v = 0; v < nv; ++v)
                for (int64_t q0 = 0; q0 < Kp; q0 += TQ) one.push_back({0, (int16_t)j, (int16_t)mq, v, 1, (int32_t)q0, 0});
        } else {
            const int nvar = std::max<int>(1, (int)(rg::kT / Kp));
            for (int v0 = 0; v0 < nv; v0 += nvar) one.push_back({0, (int16_t)j, 0, v0, std::min(nvar, nv - v0), 0, 0});
        }
    }
    std::vector<rg::Work> all;
    all.reserve(one.size() * (size_t)B);
    for (const auto &w : one)  // the largest work of every pulse first
        for (int64_t b = 0; b < B; ++b) {
            rg::Work x = w;
            x.item = (int32_t)b;
            all.push_back(x);
        }
    if (cudaMalloc(&ps->items, (size_t)B * sizeof(rg::Item)) != cudaSuccess ||
        cudaMalloc(&ps->work, all.size() * sizeof(rg::Work)) != cudaSuccess ||
        cudaMalloc(&ps->counter, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        free_small(p);
        set_error("device allocation failed: small-batch work list");
        return SIDWT_ENOMEM;
    }
    cudaError_t e = cudaMemcpy(ps->work, all.data(), all.size() * sizeof(rg::Work), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "small-batch work list upload");
    ps->nwork = (int)all.size();
    ps->built_B = B;
    return SIDWT_OK;
}

bool small_uses_latency_kernel(const sidwt_plan *p) { return p->N <= rg::kLatMaxN && p->J < 16; }
int small_launch_count(const sidwt_plan *p) { return small_uses_latency_kernel(p) ? 1 : 2; }

sidwt_status correlate_small(sidwt_plan *p, const int32_t *ref_ids_dev, int64_t B, float2 *R, cudaStream_t s) {
    if (small_uses_latency_kernel(p)) {
        rg::LatTable tab;
        std::memset(&tab, 0, sizeof(tab));
        int total = 0;
        for (int j = 0; j <= p->J; ++j) {
            rg::LatScale &z = tab.t[tab.n++];
            z.j = j;
            z.lev = j < p->J ? j + 1 : p->J;
            z.Kp = (int32_t)(p->N >> z.lev);
            z.nv = 1 << z.lev;
            z.nqb = (z.Kp + 31) / 32;
            z.first = total;
            total += z.nv * z.nqb;
        }
        cudaError_t e = launch_dependent(rg::corr_latency_kernel, dim3((unsigned)total, (unsigned)B), dim3(256), 0, s,
                                         (const float2 *)p->tree_f, p->tree_elems, (const float2 *)p->pyr_f,
                                         p->pyr_elems, ref_ids_dev, p->nrefs, p->N, p->J, tab, p->keys, R, p->ref_ids,
                                         p->err);
        if (e == cudaSuccess) e = cudaGetLastError();
        return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "small-batch correlation launch");
    }
    PlanSmall *ps = static_cast<PlanSmall *>(p->small);
    if (!ps || ps->built_B != B) {
        set_error("small-batch work list not prepared");
        return SIDWT_EINVAL;
    }
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    rg::plan_items_kernel<<<1, 32, 0, s>>>(ref_ids_dev, (int)B, p->nrefs, (int)p->N, p->J, p->pyr_elems,
                                           p->tree_elems, p->xen_len, ps->items);
    cudaError_t e = cudaMemsetAsync(ps->counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    const int grid = std::min<int>(sms * 2, std::max(1, ps->nwork));
    rg::corr_ragged_kernel<<<grid, rg::kT, 0, s>>>(ps->items, ps->work, ps->nwork, ps->counter, p->tree_f, p->pyr_f,
                                                    p->keys, R);
    e = cudaGetLastError();
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "small-batch correlation launch");
}

}  // namespace sidwt

bool sidwt::ragged_room(const sidwt_ragged *r, int64_t tree_elems, int64_t xen_elems, int64_t tc_elems) {
    return r->tree_used + tree_elems <= r->tree_cap && r->xen_used + xen_elems <= r->xen_cap &&
           r->tc_a_used + tc_elems <= r->tc_a_cap;
}

sidwt_status sidwt::ragged_reserve_tc(sidwt_ragged *r, int64_t stored_elems) {
    return grow(&r->tc_a, &r->tc_a_cap, stored_elems, r->tc_a_used, "stored tensor-core operands");
}

extern "C" {

sidwt_status sidwt_ragged_create(sidwt_ragged **out) {
    if (!out) {
        set_error("out is NULL");
        return SIDWT_EINVAL;
    }
    *out = nullptr;
    sidwt_ragged *r = new (std::nothrow) sidwt_ragged();
    if (!r) {
        set_error("host allocation failed");
        return SIDWT_ENOMEM;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&r->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        r->sms = 152;
    }
    load_tuning(r, nullptr);
    sidwt_status pst = prepare_kernels();
    if (pst) {
        delete r;
        return pst;
    }
    if (cudaMalloc(&r->err, sizeof(int32_t)) != cudaSuccess || cudaMemset(r->err, 0, sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        sidwt_ragged_destroy(r);
        set_error("device allocation failed: error flag");
        return SIDWT_ENOMEM;
    }
    *out = r;
    return SIDWT_OK;
}

sidwt_status sidwt_ragged_destroy(sidwt_ragged *r) {
    if (!r) return SIDWT_OK;
    cudaDeviceSynchronize();
    if (r->exec) cudaGraphExecDestroy(r->exec);
    if (r->graph) cudaGraphDestroy(r->graph);
    for (DevLayout *d : {&r->dl, &r->gl}) {
        cudaFree(d->items);
        cudaFree(d->work);
        cudaFree(d->lift);
        cudaFree(d->slot_item);
        cudaFree(d->tc_tiles);
        cudaFree(d->maps);
        cudaFree(d->lt);
        cudaFree(d->ltail);
        cudaFree(d->splits);
    }
    cudaFree(r->tc_a);
    cudaFree(r->err);
    cudaFree(r->tree);
    cudaFree(r->xen);
    cudaFree(r->pyr);
    cudaFree(r->yen);
    cudaFree(r->part);
    cudaFree(r->tcpart);
    cudaFree(r->keys);
    cudaFree(r->lag);
    cudaFree(r->mag);
    cudaFree(r->norm);
    cudaFree(r->counter);
    for (auto e : r->ev) cudaEventDestroy(e);
    if (r->stage_done) cudaEventDestroy(r->stage_done);
    if (r->h_stage) cudaFreeHost(r->h_stage);
    delete r;
    return SIDWT_OK;
}

sidwt_status sidwt_ragged_reserve(sidwt_ragged *r, int64_t tree_elems, int64_t pyr_elems, int64_t slots) {
    if (!r || tree_elems < 0 || pyr_elems < 0 || slots < 0) {
        set_error("bad reservation");
        return SIDWT_EINVAL;
    }
    cudaDeviceSynchronize();
    sidwt_status st;
    if ((st = grow(&r->tree, &r->tree_cap, tree_elems, r->tree_used, "ragged reference store"))) return st;
    // a reference's energies (2^(J+1) - 1 values) never exceed its tree (2 J N >= 2^(J+1) elements)
    if ((st = grow(&r->xen, &r->xen_cap, tree_elems, r->xen_used, "ragged reference energies"))) return st;
    RaggedLayout L;
    L.pyr_elems = pyr_elems;
    L.slots = slots;
    // the tiled analysis keeps kTileLevels + 1 partials per tile: at most one tile per
    // kTileSamples samples plus one per pulse (a pyramid row holds about 2 N elements)
    L.part_elems = (kTileLevels + 1) * (pyr_elems / (2 * kTileSamples) + slots + 1);
    return ensure_workspace(r, L);
}

int32_t sidwt_ragged_num_refs(const sidwt_ragged *r) { return r ? (int32_t)r->refs.size() : -1; }

sidwt_status sidwt_ragged_store_reference(sidwt_ragged *r, sidwt_filter f, int64_t N, int J, const void *x_dev,
                                          int32_t *ref_id_out, sidwt_stream stream) {
    if (!r || !x_dev || !ref_id_out) {
        set_error("NULL argument");
        return SIDWT_EINVAL;
    }
    if ((int)f < 0 || (int)f > 2) {
        set_error("ragged batches take the float filters (D4, LeGall 5/3, CDF 9/7)");
        return ((int)f == 3 || (int)f == 4) ? SIDWT_EUNSUPPORTED : SIDWT_EINVAL;
    }
    if (J < 1 || J > 15 || N < 2 || N > (int64_t(1) << 26) || N % (int64_t(1) << J) != 0) {
        set_error("need 1 <= J <= 15, N a multiple of 2^J, N <= 2^26");
        return SIDWT_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(x_dev) % 8) {
        set_error("x_dev is misaligned");
        return SIDWT_EINVAL;
    }
    const int64_t te = 2 * (int64_t)J * N, xe = (int64_t(2) << J) - 1;
    if (r->tree_used + te > r->tree_cap || r->xen_used + xe > r->xen_cap) cudaDeviceSynchronize();
    sidwt_status st;
    if ((st = grow(&r->tree, &r->tree_cap, r->tree_used + te, r->tree_used, "ragged reference store")) ||
        (st = grow(&r->xen, &r->xen_cap, r->xen_used + xe, r->xen_used, "ragged reference energies")))
        return st;
    sidwt_plan p;  // describes one reference slot; owns nothing
    p.filter = (int)f;
    p.N = N;
    p.J = J;
    p.tree_elems = te;
    p.xen_len = xe;
    p.tree_f = r->tree + r->tree_used;
    p.xen = r->xen + r->xen_used;
    if ((st = build_reference_tree(&p, x_dev, 0, reinterpret_cast<cudaStream_t>(stream)))) return st;
    RefInfo ri{(int)f, N, J, r->tree_used, r->xen_used, {}, {}};
    for (int j = 0; j < 16; ++j) {
        ri.tc_off[j] = -1;
        ri.tc_S[j] = 0;
    }
    if (r->prec == SIDWT_PREC_BF16X3) {
        // stored tensor-core operands of the scales whose bands are long enough
        int64_t need = r->tc_a_used;
        for (int j = 0; j <= J && j < 16; ++j) {
            rtc::Shape sh;
            if (!rtc::shape_for(N, J, j, &sh, &r->tcw)) continue;
            ri.tc_off[j] = need;
            ri.tc_S[j] = (int16_t)sh.S;
            need += (sh.a_elems + 63) / 64 * 64;
        }
        if (need > r->tc_a_used) {
            if (need > r->tc_a_cap) cudaDeviceSynchronize();
            if ((st = grow(&r->tc_a, &r->tc_a_cap, need, r->tc_a_used, "stored tensor-core operands"))) return st;
            if ((st = rtc::pack_stored(p.tree_f, N, J, ri.tc_off, ri.tc_S, r->tc_a,
                                       reinterpret_cast<cudaStream_t>(stream))))
                return st;
            r->tc_a_used = need;
        }
    }
    r->refs.push_back(ri);
    r->tree_used += te;
    r->xen_used += xe;
    *ref_id_out = (int32_t)r->refs.size() - 1;
    return SIDWT_OK;
}

sidwt_status sidwt_ragged_store_references(sidwt_ragged *r, int64_t n, const int32_t *filters_host,
                                           const int64_t *N_host, const int32_t *J_host, const void *x_dev,
                                           const int64_t *x_offsets_host, int64_t x_elems, int32_t *ref_ids_out,
                                           sidwt_stream stream) {
    if (!r || n < 0 || (n > 0 && (!filters_host || !N_host || !J_host || !x_dev || !x_offsets_host || !ref_ids_out))) {
        set_error("NULL argument");
        return SIDWT_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(x_dev) % 8) {
        set_error("x_dev is misaligned");
        return SIDWT_EINVAL;
    }
    int64_t te_all = 0, xe_all = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int f = filters_host[i], J = J_host[i];
        const int64_t N = N_host[i];
        if (f < 0 || f > 2) {
            set_error("item " + std::to_string(i) + ": ragged batches take the float filters (D4, LeGall 5/3, CDF 9/7)");
            return (f == 3 || f == 4) ? SIDWT_EUNSUPPORTED : SIDWT_EINVAL;
        }
        if (J < 1 || J > 15 || N < 2 || N > (int64_t(1) << 26) || N % (int64_t(1) << J) != 0) {
            set_error("item " + std::to_string(i) + ": need 1 <= J <= 15, N a multiple of 2^J, N <= 2^26");
            return SIDWT_EINVAL;
        }
        if (x_offsets_host[i] < 0 || x_offsets_host[i] + N > x_elems) {
            set_error("item " + std::to_string(i) + " runs past the end of the signal buffer");
            return SIDWT_EINVAL;
        }
        te_all += 2 * (int64_t)J * N;
        xe_all += (int64_t(2) << J) - 1;
    }
    if (n == 0) return SIDWT_OK;
    if (r->tree_used + te_all > r->tree_cap || r->xen_used + xe_all > r->xen_cap) cudaDeviceSynchronize();
    sidwt_status st;
    if ((st = grow(&r->tree, &r->tree_cap, r->tree_used + te_all, r->tree_used, "ragged reference store")) ||
        (st = grow(&r->xen, &r->xen_cap, r->xen_used + xe_all, r->xen_used, "ragged reference energies")))
        return st;
    // offsets of every tree, energy row and stored tensor-core operand
    std::vector<RefInfo> infos((size_t)n);
    std::vector<TreeItem> by_filter[3];
    int64_t tree_at = r->tree_used, xen_at = r->xen_used, tc_at = r->tc_a_used;
    for (int64_t i = 0; i < n; ++i) {
        const int f = filters_host[i], J = J_host[i];
        const int64_t N = N_host[i];
        RefInfo &ri = infos[(size_t)i];
        ri = RefInfo{f, N, J, tree_at, xen_at, {}, {}};
        for (int j = 0; j < 16; ++j) {
            ri.tc_off[j] = -1;
            ri.tc_S[j] = 0;
        }
        if (r->prec == SIDWT_PREC_BF16X3)
            for (int j = 0; j <= J && j < 16; ++j) {
                rtc::Shape sh;
                if (!rtc::shape_for(N, J, j, &sh, &r->tcw)) continue;
                ri.tc_off[j] = tc_at;
                ri.tc_S[j] = (int16_t)sh.S;
                tc_at += (sh.a_elems + 63) / 64 * 64;
            }
        by_filter[f].push_back(TreeItem{x_offsets_host[i], tree_at, xen_at, (int32_t)N, J});
        tree_at += 2 * (int64_t)J * N;
        xen_at += (int64_t(2) << J) - 1;
    }
    if (tc_at > r->tc_a_used) {
        if (tc_at > r->tc_a_cap) cudaDeviceSynchronize();
        if ((st = grow(&r->tc_a, &r->tc_a_cap, tc_at, r->tc_a_used, "stored tensor-core operands"))) return st;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float2 *x = static_cast<const float2 *>(x_dev);
    for (int f = 0; f < 3; ++f)
        if (!by_filter[f].empty() &&
            (st = build_reference_trees(f, x, r->tree, r->xen, by_filter[f].data(), (int)by_filter[f].size(), s,
                                        nullptr)))
            return st;
    if (tc_at > r->tc_a_used) {
        std::vector<rtc::PackItem> pk;
        pk.reserve((size_t)n);
        for (const RefInfo &ri : infos) pk.push_back(rtc::PackItem{ri.tree_off, ri.N, ri.J, ri.tc_off, ri.tc_S});
        if ((st = rtc::pack_stored_batch(r->tree, pk.data(), (int)pk.size(), r->tc_a, s, nullptr))) return st;
    }
    for (int64_t i = 0; i < n; ++i) {
        ref_ids_out[i] = (int32_t)r->refs.size();
        r->refs.push_back(infos[(size_t)i]);
    }
    r->tree_used = tree_at;
    r->xen_used = xen_at;
    r->tc_a_used = tc_at;
    return SIDWT_OK;
}

sidwt_status sidwt_ragged_set_split(sidwt_ragged *r, int mode) {
    if (!r || mode < 0 || mode > 2) {
        set_error("need a ragged object and mode 0 (automatic), 1 (never) or 2 (always)");
        return SIDWT_EINVAL;
    }
    r->split_mode = mode;
    return SIDWT_OK;
}

sidwt_status sidwt_ragged_correlate_r(sidwt_ragged *r, int64_t n_items, const int32_t *ref_ids_host,
                                      const int64_t *y_offsets_host, const void *y_dev, int64_t y_elems, void *r_dev,
                                      int64_t r_elems, sidwt_stream stream) {
    if (!r || n_items < 0 || (n_items > 0 && (!ref_ids_host || !y_offsets_host || !y_dev))) {
        set_error("bad arguments");
        return SIDWT_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(y_dev) % 16 || reinterpret_cast<uintptr_t>(r_dev) % 8) {
        set_error("y_dev must be 16-byte aligned (r_dev 8-byte aligned)");
        return SIDWT_EINVAL;
    }
    RaggedLayout L;
    sidwt_status st = build_layout(r, n_items, ref_ids_host, y_offsets_host, y_elems, L);
    if (st) return st;
    if (r_dev && r_elems < L.r_elems) {
        set_error("r_dev holds " + std::to_string(r_elems) + " elements; this batch writes " +
                  std::to_string(L.r_elems) + " (the sum of (J_i + 1) N_i)");
        return SIDWT_EINVAL;
    }
    if ((st = ensure_workspace(r, L)) || (st = encode_layout_maps(r, L))) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if ((st = upload(r, r->dl, L, s, false))) return st;
    r->last_slots = L.slots;
    return enqueue(r, r->dl, L.slots, n_items, static_cast<const float2 *>(y_dev), s, nullptr,
                   static_cast<float2 *>(r_dev));
}

sidwt_status sidwt_ragged_correlate(sidwt_ragged *r, int64_t n_items, const int32_t *ref_ids_host,
                                    const int64_t *y_offsets_host, const void *y_dev, int64_t y_elems,
                                    sidwt_stream stream) {
    return sidwt_ragged_correlate_r(r, n_items, ref_ids_host, y_offsets_host, y_dev, y_elems, nullptr, 0, stream);
}

sidwt_status sidwt_ragged_graph_create(sidwt_ragged *r, int64_t n_items, const int32_t *ref_ids_host,
                                       const int64_t *y_offsets_host, const void *y_dev, int64_t y_elems,
                                       int32_t *launches_out) {
    if (!r || n_items < 0 || (n_items > 0 && (!ref_ids_host || !y_offsets_host || !y_dev))) {
        set_error("bad arguments");
        return SIDWT_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(y_dev) % 16) {
        set_error("y_dev must be 16-byte aligned");
        return SIDWT_EINVAL;
    }
    RaggedLayout L;
    sidwt_status st = build_layout(r, n_items, ref_ids_host, y_offsets_host, y_elems, L);
    if (st) return st;
    if ((st = ensure_workspace(r, L)) || (st = encode_layout_maps(r, L))) return st;
    if ((st = upload(r, r->gl, L, nullptr, true))) return st;
    if (r->exec) cudaGraphExecDestroy(r->exec);
    if (r->graph) cudaGraphDestroy(r->graph);
    r->exec = nullptr;
    r->graph = nullptr;
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return cuda_fail(cudaGetLastError(), "stream");
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        return cuda_fail(e, "begin capture");
    }
    int nl = 0;
    st = enqueue(r, r->gl, L.slots, n_items, static_cast<const float2 *>(y_dev), cs, &nl);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    if (st) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    e = cudaGraphInstantiate(&r->exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e, "graph instantiate");
    }
    r->graph = g;
    r->graph_slots = L.slots;
    r->graph_launches = nl;
    if (launches_out) *launches_out = nl;
    return SIDWT_OK;
}

sidwt_status sidwt_ragged_graph_launch(sidwt_ragged *r, sidwt_stream stream) {
    if (!r || !r->exec) {
        set_error("no graph: call sidwt_ragged_graph_create first");
        return SIDWT_EINVAL;
    }
    cudaError_t e = cudaGraphLaunch(r->exec, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    r->last_slots = r->graph_slots;
    return SIDWT_OK;
}

sidwt_status sidwt_ragged_peaks(sidwt_ragged *r, int64_t n_slots, int32_t *lag_dev, float *mag_dev, double *norm_dev,
                                sidwt_stream stream) {
    if (!r || n_slots != r->last_slots) {
        set_error("n_slots must equal the sum of J_i + 1 over the last batch");
        return SIDWT_EINVAL;
    }
    if (n_slots == 0) return SIDWT_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (lag_dev) e = cudaMemcpyAsync(lag_dev, r->lag, n_slots * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && mag_dev)
        e = cudaMemcpyAsync(mag_dev, r->mag, n_slots * sizeof(float), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && norm_dev)
        e = cudaMemcpyAsync(norm_dev, r->norm, n_slots * sizeof(double), cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "ragged peak copy");
}

namespace {

// Tensor-core tile widths: for each band bucket 2^lg (lg 6..14; longer bands
// keep the 2^14 weights) one synthetic pair at scale 3 of J = 4 (N = 2^(lg+4):
// 16 variants, so every tile is full; both bands, circular form) is packed
// with every width and its tiles, replicated to keep every SM busy, are timed
// on the persistent kernel.  A width's weight is its time per padded MMA
// element (tiles x 128 rows x S columns x K) relative to width 256.
sidwt_status tune_tc(sidwt_ragged *r, cudaStream_t s, std::string *report) {
    const int lg_lo = 6, lg_hi = 14;
    const int *widths = rtc::kTcWidth;
    int64_t amax = 0, tmax = 0;
    for (int lg = lg_lo; lg <= lg_hi; ++lg)
        for (int k = 0; k < rtc::kTcWidths; ++k) {
            const int S = widths[k];
            rtc::Shape sh;
            if (!rtc::shape_with(int64_t(16) << lg, 4, 3, S, &sh)) continue;
            amax = std::max(amax, sh.a_elems);
        }
    for (int lg = lg_lo; lg <= lg_hi; ++lg)
        tmax = std::max<int64_t>(tmax, (int64_t)r->sms * std::min(64, std::max(2, 1 << std::max(0, 16 - lg))));
    const int64_t Nmax = int64_t(16) << lg_hi;
    float2 *tree = nullptr, *pyr = nullptr;
    __nv_bfloat16 *abuf = nullptr;
    unsigned char *maps = nullptr;
    rtc::TcTile *dt = nullptr;
    unsigned long long *keys = nullptr;
    int32_t *err = nullptr;
    const size_t mb = rtc::map_bytes();
    auto release = [&]() {
        cudaFree(tree);
        cudaFree(pyr);
        cudaFree(abuf);
        cudaFree(maps);
        cudaFree(dt);
        cudaFree(keys);
        cudaFree(err);
    };
    if (cudaMalloc(&tree, 8 * Nmax * sizeof(float2)) != cudaSuccess ||  // 2 J N, J = 4
        cudaMalloc(&pyr, 2 * Nmax * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&abuf, amax * sizeof(__nv_bfloat16)) != cudaSuccess || cudaMalloc(&maps, 2 * mb) != cudaSuccess ||
        cudaMalloc(&dt, tmax * sizeof(rtc::TcTile)) != cudaSuccess ||
        cudaMalloc(&keys, sizeof(unsigned long long)) != cudaSuccess || cudaMalloc(&err, sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        release();
        set_error("autotune allocation failed");
        return SIDWT_ENOMEM;
    }
    rg::fill_kernel<<<(unsigned)((8 * Nmax + 255) / 256), 256, 0, s>>>(tree, 8 * Nmax, 3u);
    rg::fill_kernel<<<(unsigned)((2 * Nmax + 255) / 256), 256, 0, s>>>(pyr, 2 * Nmax, 4u);
    cudaMemsetAsync(err, 0, sizeof(int32_t), s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<unsigned char> hmaps(2 * mb);
    sidwt_status st = SIDWT_OK;
    rtc::TcWeights w = r->tcw;
    for (int lg = lg_lo; lg <= lg_hi && !st; ++lg) {
        const int64_t Kp = int64_t(1) << lg, N = 16 * Kp;
        double per[rtc::kTcWidths] = {};
        for (int k = 0; k < rtc::kTcWidths && !st; ++k) {
            const int S = widths[k];
            rtc::Shape sh;
            rtc::shape_with(N, 4, 3, S, &sh);
            int64_t a_off[16];
            int16_t S_of[16];
            for (int j = 0; j < 16; ++j) {
                a_off[j] = -1;
                S_of[j] = 0;
            }
            a_off[3] = 0;
            S_of[3] = (int16_t)S;
            if ((st = rtc::pack_stored(tree, N, 4, a_off, S_of, abuf, s))) break;
            if ((st = rtc::encode_maps(hmaps.data(), abuf, nullptr, sh))) break;
            cudaMemcpyAsync(maps, hmaps.data(), 2 * mb, cudaMemcpyHostToDevice, s);
            const int n = r->sms * std::min(64, std::max(2, 1 << std::max(0, 16 - lg)));
            std::vector<rtc::TcTile> tl((size_t)n);
            for (int t = 0; t < n; ++t) {
                rtc::TcTile &x = tl[(size_t)t];
                x.map = 0;
                x.tile = t % sh.tiles;
                x.nkb = sh.nkb;
                x.Kp = (int32_t)Kp;
                x.gv = sh.gv;
                x.nv = sh.nv;
                x.nb = (int16_t)sh.nb;
                x.lev = (int16_t)sh.lev;
                x.S = (int16_t)S;
                x.k0 = (int16_t)sh.k0;
                x.slot = 0;
                x.u_off = 2 * N - 4 * Kp;  // level sh.lev of the synthetic pyramid
                x.slot_mid = -1;
            }
            cudaMemcpyAsync(dt, tl.data(), (size_t)n * sizeof(rtc::TcTile), cudaMemcpyHostToDevice, s);
            cudaStreamSynchronize(s);  // the host staging buffers are reused
            float tot = 0.f;
            for (int rep = 0; rep < 4 && !st; ++rep) {
                cudaEventRecord(e0, s);
                st = rtc::launch_corr(maps, dt, n, pyr, keys, err, r->sms, s);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) tot += ms;
            }
            per[k] = (double)tot / ((double)n * S * sh.nkb);
        }
        if (st) break;
        for (int k = 0; k < rtc::kTcWidths; ++k) {
            const float v = per[0] > 0 ? (float)(per[k] / per[0]) : w.w[k][lg];
            w.w[k][lg] = std::min(50.f, std::max(0.2f, v));
            *report += "tc " + std::to_string(widths[k]) + " " + std::to_string(lg) + " " + std::to_string(w.w[k][lg]) + "\n";
        }
    }
    int32_t herr = 0;
    if (!st) {
        cudaMemcpy(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(e, "tensor-core autotune");
        else if (herr) {
            set_error("tensor-core autotune: a kernel wait timed out");
            st = SIDWT_ETIMEOUT;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    release();
    if (st) return st;
    for (int lg = lg_hi + 1; lg < rtc::kTcBuckets; ++lg)
        for (int k = 0; k < rtc::kTcWidths; ++k) w.w[k][lg] = w.w[k][lg_hi];
    for (int lg = 0; lg < lg_lo; ++lg)
        for (int k = 0; k < rtc::kTcWidths; ++k) w.w[k][lg] = w.w[k][lg_lo];
    r->tcw = w;
    return SIDWT_OK;
}

}  // namespace

sidwt_status sidwt_ragged_autotune(sidwt_ragged *r, const char *cache_path, sidwt_stream stream) {
    if (!r) {
        set_error("NULL argument");
        return SIDWT_EINVAL;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // one synthetic pair per bucket: band length Kp = 2^lg at scale 0 (J = 1)
    const int lg_lo = 8, lg_hi = 15;
    const int64_t Nmax = int64_t(2) << lg_hi;
    float2 *tree = nullptr, *pyr = nullptr;
    unsigned long long *keys = nullptr;
    int *counter = nullptr;
    rg::Item *ditem = nullptr;
    rg::Work *dwork = nullptr;
    // each candidate runs the pair's work items replicated until the largest
    // shift count gives every SM four items: throughput, as in a real batch,
    // rather than the latency of one pair
    const int64_t lags_target = (int64_t)4 * r->sms * rg::kT * rg::kMaxMQ;
    const int64_t max_work = 2 * lags_target / rg::kT + 2 * Nmax / rg::kT + 64;
    if (cudaMalloc(&tree, 2 * Nmax * sizeof(float2)) != cudaSuccess || cudaMalloc(&pyr, 2 * Nmax * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&keys, 4 * sizeof(unsigned long long)) != cudaSuccess || cudaMalloc(&counter, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&ditem, sizeof(rg::Item)) != cudaSuccess || cudaMalloc(&dwork, max_work * sizeof(rg::Work)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(tree);
        cudaFree(pyr);
        cudaFree(keys);
        cudaFree(counter);
        cudaFree(ditem);
        cudaFree(dwork);
        set_error("autotune allocation failed");
        return SIDWT_ENOMEM;
    }
    rg::fill_kernel<<<(unsigned)((2 * Nmax + 255) / 256), 256, 0, s>>>(tree, 2 * Nmax, 1u);
    rg::fill_kernel<<<(unsigned)((2 * Nmax + 255) / 256), 256, 0, s>>>(pyr, 2 * Nmax, 2u);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::string report;
    for (int lg = lg_lo; lg <= lg_hi; ++lg) {
        const int64_t Kp = int64_t(1) << lg, N = 2 * Kp;
        rg::Item it{0, 0, 0, 0, (int32_t)N, 1, 0, 0, 0};
        cudaMemcpyAsync(ditem, &it, sizeof(it), cudaMemcpyHostToDevice, s);
        float best_ms = 1e30f;
        int best_mq = default_mq(lg);
        for (int mq : {1, 2, 4, 8}) {
            const int64_t TQ = (int64_t)rg::kT * mq;
            if (TQ > Kp) continue;
            std::vector<rg::Work> w;
            const int64_t reps = std::max<int64_t>(1, (lags_target + 2 * Kp - 1) / (2 * Kp));
            for (int64_t k = 0; k < reps; ++k)
                for (int v = 0; v < 2; ++v)
                    for (int64_t q0 = 0; q0 < Kp; q0 += TQ) w.push_back({0, 0, (int16_t)mq, v, 1, (int32_t)q0, 0});
            if ((int64_t)w.size() > max_work) continue;  // cannot happen: max_work bounds reps x items
            cudaMemcpyAsync(dwork, w.data(), w.size() * sizeof(rg::Work), cudaMemcpyHostToDevice, s);
            cudaStreamSynchronize(s);
            float tot = 0.f;
            for (int rep = 0; rep < 4; ++rep) {
                cudaMemsetAsync(counter, 0, sizeof(int), s);
                cudaEventRecord(e0, s);
                rg::corr_ragged_kernel<<<r->sms * 2, rg::kT, 0, s>>>(ditem, dwork, (int)w.size(), counter, tree, pyr, keys,
                                                                      nullptr);
                cudaEventRecord(e1, s);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) tot += ms;
            }
            if (tot < best_ms) {
                best_ms = tot;
                best_mq = mq;
            }
        }
        r->mq_for[lg] = best_mq;
        report += std::to_string(lg) + " " + std::to_string(best_mq) + "\n";
    }
    for (int lg = lg_hi + 1; lg < 32; ++lg) r->mq_for[lg] = r->mq_for[lg_hi];
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(tree);
    cudaFree(pyr);
    cudaFree(keys);
    cudaFree(counter);
    cudaFree(ditem);
    cudaFree(dwork);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    sidwt_status st = tune_tc(r, s, &report);
    if (st) return st;
    if (!cache_path) cache_path = std::getenv("SIDWT_TUNE_CACHE");
    if (cache_path) {
        FILE *f = std::fopen(cache_path, "w");
        if (f) {
            std::fputs(report.c_str(), f);
            std::fclose(f);
        }
    }
    return SIDWT_OK;
}

sidwt_status sidwt_ragged_set_timing(sidwt_ragged *r, int enable) {
    if (!r) {
        set_error("NULL argument");
        return SIDWT_EINVAL;
    }
    r->timing = enable != 0;
    return SIDWT_OK;
}

sidwt_status sidwt_ragged_read_timing(sidwt_ragged *r, sidwt_timing *out, int reset) {
    if (!r || !out) {
        set_error("NULL argument");
        return SIDWT_EINVAL;
    }
    for (size_t i = 0; i + 3 < r->ev.size(); i += 4) {
        cudaError_t e = cudaEventSynchronize(r->ev[i + 3]);
        if (e != cudaSuccess) return cuda_fail(e, "timing event");
        float a = 0.f, b = 0.f, c = 0.f;
        cudaEventElapsedTime(&a, r->ev[i], r->ev[i + 1]);
        cudaEventElapsedTime(&b, r->ev[i + 1], r->ev[i + 2]);
        cudaEventElapsedTime(&c, r->ev[i + 2], r->ev[i + 3]);
        r->t_ms[0] += a;
        r->t_ms[1] += b;
        r->t_ms[2] += c;
    }
    for (auto e : r->ev) cudaEventDestroy(e);
    r->ev.clear();
    std::memset(out, 0, sizeof(*out));
    out->analyze_ms = r->t_ms[0];
    out->correlate_ms = r->t_ms[1];
    out->peaks_ms = r->t_ms[2];
    out->correlate_calls = r->timed_calls;
    out->launches = r->timed_launches;
    if (reset) {
        r->t_ms[0] = r->t_ms[1] = r->t_ms[2] = 0.0;
        r->timed_calls = r->timed_launches = 0;
    }
    return SIDWT_OK;
}

sidwt_status sidwt_ragged_reset_references(sidwt_ragged *r) {
    if (!r) {
        set_error("NULL argument");
        return SIDWT_EINVAL;
    }
    r->refs.clear();
    r->tree_used = 0;
    r->xen_used = 0;
    r->tc_a_used = 0;
    return SIDWT_OK;
}

sidwt_status sidwt_ragged_set_precision(sidwt_ragged *r, sidwt_precision prec) {
    if (!r) {
        set_error("NULL argument");
        return SIDWT_EINVAL;
    }
    if (prec == SIDWT_PREC_TF32X3) {
        set_error("3xTF32 is not implemented for ragged batches");
        return SIDWT_EUNSUPPORTED;
    }
    if (prec != SIDWT_PREC_FP32 && prec != SIDWT_PREC_BF16X3) {
        set_error("unknown precision");
        return SIDWT_EINVAL;
    }
    r->prec = (int)prec;
    return SIDWT_OK;
}

sidwt_status sidwt_ragged_check(sidwt_ragged *r, sidwt_stream stream) {
    if (!r) {
        set_error("NULL argument");
        return SIDWT_EINVAL;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int32_t h = 0;
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemcpy(&h, r->err, sizeof(h), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(r->err, 0, sizeof(int32_t));
    if (e != cudaSuccess) return cuda_fail(e, "ragged check");
    if (h & kErrTcWait) {
        set_error("a tensor-core CTA gave up on a bounded wait; results are incomplete");
        return SIDWT_ETIMEOUT;
    }
    if (h & kErrAnalysisWait) {
        set_error("the received analysis gave up waiting for an input copy; the pyramids and the peaks are incomplete");
        return SIDWT_ETIMEOUT;
    }
    return SIDWT_OK;
}

sidwt_status sidwt_ragged_tuning(const sidwt_ragged *r, int32_t *mq_by_log2_band /* [32] */) {
    if (!r || !mq_by_log2_band) {
        set_error("NULL argument");
        return SIDWT_EINVAL;
    }
    for (int i = 0; i < 32; ++i) mq_by_log2_band[i] = r->mq_for[i];
    return SIDWT_OK;
}

sidwt_status sidwt_ragged_tc_weights(const sidwt_ragged *r, float *w) {
    if (!r || !w) {
        set_error("NULL argument");
        return SIDWT_EINVAL;
    }
    for (int k = 0; k < rtc::kTcWidths; ++k)
        for (int b = 0; b < rtc::kTcBuckets; ++b) w[k * rtc::kTcBuckets + b] = r->tcw.w[k][b];
    return SIDWT_OK;
}

}  // extern "C"

int32_t *sidwt::ragged_error_record(sidwt_ragged *r) { return r->err; }
