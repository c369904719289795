// Per-scale target detection on the correlation (Sec. V-A, Fig. 6): in every
// row of |r_j| (one pulse, one scale) the local maxima along the delay axis
// (circularly: above the previous delay, not below the next) that lie within
// the threshold of the row's largest magnitude, in increasing delay.  One
// CTA per row: a max reduction, then a chunked scan in delay order with a
// block-wide prefix sum, so the output order is the delay order.
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

}  // namespace
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
    const float ratio2 = (float)std::pow(10.0, -(double)threshold_db / 10.0);  // (10^(-T/20))^2
    detect_kernel<<<(unsigned)rows, kDetThreads, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        static_cast<const float2 *>(r_dev), N, ratio2, max_det, count_dev, lag_dev, mag_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "detection launch");
}
