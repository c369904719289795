// Per-scale target detection on the correlation (Sec. V-A, Fig. 6): in every
// row of |r_j| (one pulse, one scale) the local maxima along the delay axis
// (circularly: above the previous delay, not below the next) that lie within
// the threshold of the row's largest magnitude, in increasing delay.  One
// CTA per row.
#include <cuda_runtime.h>

#include <cmath>

#include "sidwt_internal.cuh"

namespace sidwt {
namespace {

constexpr int kDetThreads = 256;

__device__ __forceinline__ float mag2(float2 v) { return fmaf(v.x, v.x, v.y * v.y); }

__global__ void __launch_bounds__(kDetThreads) detect_kernel(const float2 *__restrict__ R, int64_t N, float ratio2,
                                                             int max_det, int32_t *__restrict__ count,
                                                             int32_t *__restrict__ det_lag, float *__restrict__ det_mag) {
    __shared__ float red[kDetThreads / 32];
    __shared__ int scan[kDetThreads / 32];
    const int64_t row = blockIdx.x;
    const float2 *r = R + row * N;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    float mx = 0.f;
    for (int64_t D = tid; D < N; D += blockDim.x) mx = fmaxf(mx, mag2(r[D]));
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    mx = 0.f;
    for (int w = 0; w < nw; ++w) mx = fmaxf(mx, red[w]);
    const float level = mx * ratio2;
    // thread t owns the delays [t chunk, (t + 1) chunk)
    const int64_t chunk = (N + blockDim.x - 1) / blockDim.x;
    const int64_t d0 = tid * chunk, d1 = d0 + chunk < N ? d0 + chunk : N;
    int mine = 0;
    if (mx > 0.f && d0 < d1) {
        float prev = mag2(r[(d0 + N - 1) % N]), cur = mag2(r[d0]);
        for (int64_t D = d0; D < d1; ++D) {
            const float nxt = mag2(r[(D + 1) % N]);
            if (cur > prev && cur >= nxt && cur >= level) ++mine;
            prev = cur;
            cur = nxt;
        }
    }
    // exclusive prefix sum of the per-thread counts, in thread (= delay) order
    int incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) scan[warp] = incl;
    __syncthreads();
    int before = 0, total = 0;
    for (int w = 0; w < nw; ++w) {
        if (w < warp) before += scan[w];
        total += scan[w];
    }
    int pos = before + incl - mine;
    if (mx > 0.f && d0 < d1 && mine && pos < max_det) {
        float prev = mag2(r[(d0 + N - 1) % N]), cur = mag2(r[d0]);
        for (int64_t D = d0; D < d1 && pos < max_det; ++D) {
            const float nxt = mag2(r[(D + 1) % N]);
            if (cur > prev && cur >= nxt && cur >= level) {
                det_lag[row * max_det + pos] = (int32_t)D;
                det_mag[row * max_det + pos] = sqrtf(cur);
                ++pos;
            }
            prev = cur;
            cur = nxt;
        }
    }
    if (tid == 0) count[row] = total;
}

// Rows of up to kDetSmemN delays: |r|^2 staged in shared memory by coalesced
// loads (the row is read from DRAM once); delays tested in rounds of 256
// (D = 256 k + thread), compacted in delay order by warp ballots and a scan
// of the per-(round, warp) counts.
constexpr int kDetSmemN = 16384;
constexpr int kDetRounds = kDetSmemN / kDetThreads;

__global__ void __launch_bounds__(kDetThreads) detect_smem_kernel(const float2 *__restrict__ R, int N, float ratio2,
                                                                  int max_det, int32_t *__restrict__ count,
                                                                  int32_t *__restrict__ det_lag,
                                                                  float *__restrict__ det_mag) {
    extern __shared__ float m2[];
    __shared__ float red[kDetThreads / 32];
    __shared__ int cnt[kDetRounds * (kDetThreads / 32)];
    __shared__ int total_s;
    const int64_t row = blockIdx.x;
    const float2 *r = R + row * (int64_t)N;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kDetThreads / 32;
    float mx = 0.f;
    for (int D = tid; D < N; D += kDetThreads) {
        const float v = mag2(r[D]);
        m2[D] = v;
        mx = fmaxf(mx, v);
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    mx = 0.f;
    for (int w = 0; w < NW; ++w) mx = fmaxf(mx, red[w]);
    const float level = mx * ratio2;
    const int rounds = (N + kDetThreads - 1) / kDetThreads;
    auto hit_at = [&](int D) -> bool {
        if (D >= N || !(mx > 0.f)) return false;
        const float cur = m2[D];
        const float prev = m2[D == 0 ? N - 1 : D - 1];
        const float nxt = m2[D + 1 == N ? 0 : D + 1];
        return cur > prev && cur >= nxt && cur >= level;
    };
    for (int k = 0; k < rounds; ++k) {
        const unsigned bal = __ballot_sync(0xffffffffu, hit_at(k * kDetThreads + tid));
        if (lane == 0) cnt[k * NW + warp] = __popc(bal);
    }
    __syncthreads();
    if (warp == 0) {  // exclusive scan of rounds * NW counts, in (round, warp) = delay order
        const int n = rounds * NW;
        const int per = (n + 31) / 32;
        const int a = lane * per, b = min(n, a + per);
        int sum = 0;
        for (int i = a; i < b; ++i) sum += cnt[i];
        int incl = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int run = incl - sum;
        for (int i = a; i < b; ++i) {
            const int c = cnt[i];
            cnt[i] = run;
            run += c;
        }
        if (lane == 31) total_s = incl;
    }
    __syncthreads();
    for (int k = 0; k < rounds; ++k) {
        const int D = k * kDetThreads + tid;
        const bool hit = hit_at(D);
        const unsigned bal = __ballot_sync(0xffffffffu, hit);
        const int pos = cnt[k * NW + warp] + __popc(bal & ((1u << lane) - 1u));
        if (hit && pos < max_det) {
            det_lag[row * max_det + pos] = D;
            det_mag[row * max_det + pos] = sqrtf(m2[D]);
        }
    }
    if (tid == 0) count[row] = total_s;
}

}  // namespace

cudaError_t prepare_detect_kernels() {
    return cudaFuncSetAttribute(detect_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kDetSmemN * (int)sizeof(float));
}

}  // namespace sidwt

using namespace sidwt;

extern "C" sidwt_status sidwt_detect(const void *r_dev, int64_t rows, int64_t N, float threshold_db, int max_det,
                                     int32_t *count_dev, int32_t *lag_dev, float *mag_dev, sidwt_stream stream) {
    if (rows < 0 || rows > 0x7fffffff || N < 1 || max_det < 0 || !(threshold_db >= 0.f) ||
        (rows > 0 && (!r_dev || !count_dev || (max_det > 0 && (!lag_dev || !mag_dev))))) {
        set_error("bad detection arguments");
        return SIDWT_EINVAL;
    }
    if (rows == 0) return SIDWT_OK;
    if (reinterpret_cast<uintptr_t>(r_dev) % 8) {
        set_error("r_dev must be 8-byte aligned");
        return SIDWT_EINVAL;
    }
    sidwt_status st = prepare_kernels();
    if (st) return st;
    const float ratio2 = (float)std::pow(10.0, -(double)threshold_db / 10.0);  // (10^(-T/20))^2
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (N <= kDetSmemN)
        detect_smem_kernel<<<(unsigned)rows, kDetThreads, (size_t)N * sizeof(float), s>>>(
            static_cast<const float2 *>(r_dev), (int)N, ratio2, max_det, count_dev, lag_dev, mag_dev);
    else
        detect_kernel<<<(unsigned)rows, kDetThreads, 0, s>>>(static_cast<const float2 *>(r_dev), N, ratio2, max_det,
                                                              count_dev, lag_dev, mag_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "detection launch");
}
