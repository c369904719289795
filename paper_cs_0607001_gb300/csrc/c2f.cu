// Coarse-to-fine formation (Sec. IV eq. 21, Sec. V-B).
//
// sidwt_synthesize: one level of inverse y-side lifting, c_{l-1} from
// (c_l, d_l) -- eq. 21, the synthesis that forms the finer resolution from
// the coarser one.  One thread per output pair runs the inverse steps on a
// 5-pair window of the coarse bands.
//
// sidwt_correlate_c2f: correlate the coarsest scale J at every delay (the
// batched FP32 kernel with only scale J selected), then each finer scale j
// only at the delays within h 2^(j+1) of the scale-(j+1) peak (the peak lag
// is scale-invariant within the scale's resolution), so the cost is about
// N^2 / 2^J + 4 h N J complex products per pulse instead of about 2 N^2.
// The window search runs one CTA per pulse.
#include <cuda_runtime.h>

#include <algorithm>

#include "sidwt_internal.cuh"

namespace sidwt {
namespace {

__device__ __forceinline__ float2 axpy2n(float2 t, float c0, float2 a, float c1, float2 b) {
    // t - (c0 a + c1 b)
    return make_float2(t.x - fmaf(c0, a.x, c1 * b.x), t.y - fmaf(c0, a.y, c1 * b.y));
}

__device__ __forceinline__ int wrapi(int m, int H) {
    m %= H;
    return m < 0 ? m + H : m;
}

// Inverse of one y-side analysis level: lo = ce E, hi = co O (D4: hi =
// co (E[n] + O[n-1])) after the lifting steps; undo the scaling, then the
// steps in reverse order with the opposite sign.  Output: v[2n] = E[n] and
// v[2n+1] = O[n] (D4: v[2n-1] = O[n]).
template <int F>
__global__ void synth_kernel(const float2 *__restrict__ lo, const float2 *__restrict__ hi, int64_t in_stride, int H,
                             int B, float2 *__restrict__ out, LiftCoef c) {
    using Sh = LiftShape<F, SIDE_Y>;
    constexpr bool D4 = Sh::d4;
    constexpr int R = 2, M = 2 * R + 1;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (n >= H || b >= B) return;
    const float2 *L = lo + (int64_t)b * in_stride;
    const float2 *Hh = hi + (int64_t)b * in_stride;
    const float ice = 1.0f / c.ce, ico = 1.0f / c.co;
    float2 E[M], O[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
        const float2 l = L[wrapi(n - R + i, H)];
        E[i] = make_float2(l.x * ice, l.y * ice);
    }
#pragma unroll
    for (int i = 0; i < M; ++i) {
        if (D4) {
            // hi[m] = co (E[m] + O[m - 1])  =>  O[m] = hi[m + 1] / co - E[m + 1]
            const float2 h = Hh[wrapi(n - R + i + 1, H)];
            const float2 e1 = i + 1 < M ? E[i + 1] : make_float2(0.f, 0.f);
            O[i] = make_float2(h.x * ico - e1.x, h.y * ico - e1.y);
        } else {
            const float2 h = Hh[wrapi(n - R + i, H)];
            O[i] = make_float2(h.x * ico, h.y * ico);
        }
    }
#pragma unroll
    for (int s = Sh::nsteps - 1; s >= 0; --s) {
        const float c0 = c.c0[s], c1 = c.c1[s];
        if (Sh::target(s) == 1) {
            if (Sh::nb(s) > 0) {
#pragma unroll
                for (int i = 0; i < M - 1; ++i) O[i] = axpy2n(O[i], c0, E[i], c1, E[i + 1]);
            } else {
#pragma unroll
                for (int i = M - 1; i >= 1; --i) O[i] = axpy2n(O[i], c0, E[i], c1, E[i - 1]);
            }
        } else {
            if (Sh::nb(s) > 0) {
#pragma unroll
                for (int i = 0; i < M - 1; ++i) E[i] = axpy2n(E[i], c0, O[i], c1, O[i + 1]);
            } else {
#pragma unroll
                for (int i = M - 1; i >= 1; --i) E[i] = axpy2n(E[i], c0, O[i], c1, O[i - 1]);
            }
        }
    }
    float2 *o = out + (int64_t)b * 2 * H;
    o[2 * n] = E[R];
    if (D4)
        o[wrapi(2 * n - 1, 2 * H)] = O[R];
    else
        o[2 * n + 1] = O[R];
}

__device__ __forceinline__ unsigned long long c2f_key(float re, float im, uint32_t D) {
    return ((unsigned long long)__float_as_uint(re * re + im * im) << 32) | (unsigned long long)(0xFFFFFFFFu - D);
}

constexpr int kC2fThreads = 512;
constexpr int kC2fChunk = 256;  // delays per pass of the window (their band partial sums in shared memory)

// One pulse per CTA, after the scale-J correlation at every delay has left
// its peak key in keys[b][J].  For j = J-1 down to 0 one warp per (delay of
// the window, band) (lanes over k, coalesced):
// r_j[2^l q + v] = sum over the bands of conj(w_v[(k - q) mod K']) u[k]
// (the variant delayed by q).
__global__ void __launch_bounds__(kC2fThreads) c2f_kernel(const float2 *__restrict__ tree, int64_t tree_elems,
                                                          const float2 *__restrict__ pyr, int64_t pyr_elems,
                                                          const int32_t *__restrict__ ref_ids, int nrefs, int64_t N,
                                                          int J, int h, const unsigned long long *__restrict__ keys,
                                                          int32_t *__restrict__ lag, float *__restrict__ mag) {
    __shared__ unsigned long long wkey[kC2fThreads / 32];
    __shared__ float2 part[2 * kC2fChunk];
    const int b = blockIdx.x;
    const int ref = ref_ids[b];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const unsigned long long kJ = keys[(int64_t)b * (J + 1) + J];
    if (ref < 0 || ref >= nrefs || kJ == 0ull) {  // invalid pulse (recorded by the grouping pass)
        if (tid <= J) {
            lag[(int64_t)b * (J + 1) + tid] = -1;
            mag[(int64_t)b * (J + 1) + tid] = 0.f;
        }
        return;
    }
    const float2 *T = tree + (int64_t)ref * tree_elems;
    const float2 *P = pyr + (int64_t)b * pyr_elems;
    uint32_t Dc = 0xFFFFFFFFu - (uint32_t)(kJ & 0xFFFFFFFFull);
    if (tid == 0) {
        lag[(int64_t)b * (J + 1) + J] = (int32_t)Dc;
        mag[(int64_t)b * (J + 1) + J] = sqrtf(__uint_as_float((uint32_t)(kJ >> 32)));
    }
    for (int j = J - 1; j >= 0; --j) {
        const int lev = j + 1;
        const int Kp = (int)(N >> lev);
        const float2 *u = P + 2 * N - 4 * (int64_t)Kp;  // c_{j+1} then d_{j+1}
        const float2 *A = T + 2 * N * (int64_t)(lev - 1);
        const int64_t w = (int64_t)h << (j + 1);
        const int64_t cnt = 2 * w + 1 >= N ? N : 2 * w + 1;
        const int64_t start = 2 * w + 1 >= N ? 0 : (int64_t)Dc - w;
        unsigned long long best = 0ull;
        for (int64_t base = 0; base < cnt; base += kC2fChunk) {
            const int nl = (int)(cnt - base < kC2fChunk ? cnt - base : kC2fChunk);
            // one warp per (delay, band): the delayed variant splits into two
            // unwrapped runs, k in [q, K') reads w[k - q], k in [0, q) w[k - q + K']
            for (int it = warp; it < 2 * nl; it += nw) {
                int64_t D = (start + base + (it >> 1)) % N;
                if (D < 0) D += N;
                const int band = it & 1;
                const int q = (int)(D >> lev), v = (int)(D & ((1 << lev) - 1));
                const float2 *wb = A + (int64_t)band * N + (int64_t)v * Kp;
                const float2 *ub = u + (int64_t)band * Kp;
                float ar = 0.f, ai = 0.f;
                for (int k = q + lane; k < Kp; k += 32) {
                    const float2 wv = wb[k - q], uv = ub[k];
                    ar = fmaf(wv.x, uv.x, fmaf(wv.y, uv.y, ar));
                    ai = fmaf(wv.x, uv.y, fmaf(-wv.y, uv.x, ai));
                }
                for (int k = lane; k < q; k += 32) {
                    const float2 wv = wb[k - q + Kp], uv = ub[k];
                    ar = fmaf(wv.x, uv.x, fmaf(wv.y, uv.y, ar));
                    ai = fmaf(wv.x, uv.y, fmaf(-wv.y, uv.x, ai));
                }
                for (int o = 16; o > 0; o >>= 1) {
                    ar += __shfl_xor_sync(0xffffffffu, ar, o);
                    ai += __shfl_xor_sync(0xffffffffu, ai, o);
                }
                if (lane == 0) part[it] = make_float2(ar, ai);
            }
            __syncthreads();
            for (int l = tid; l < nl; l += blockDim.x) {
                int64_t D = (start + base + l) % N;
                if (D < 0) D += N;
                const float2 a0 = part[2 * l], a1 = part[2 * l + 1];
                const unsigned long long key = c2f_key(a0.x + a1.x, a0.y + a1.y, (uint32_t)D);
                best = key > best ? key : best;
            }
            __syncthreads();
        }
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long t = __shfl_xor_sync(0xffffffffu, best, o);
            best = t > best ? t : best;
        }
        if (lane == 0) wkey[warp] = best;
        __syncthreads();
        unsigned long long m = 0ull;
        for (int i = 0; i < nw; ++i) m = wkey[i] > m ? wkey[i] : m;
        __syncthreads();
        Dc = 0xFFFFFFFFu - (uint32_t)(m & 0xFFFFFFFFull);
        if (tid == 0) {
            lag[(int64_t)b * (J + 1) + j] = m ? (int32_t)Dc : -1;
            mag[(int64_t)b * (J + 1) + j] = sqrtf(__uint_as_float((uint32_t)(m >> 32)));
        }
    }
}

template <int F>
cudaError_t launch_synth(const float2 *lo, const float2 *hi, int64_t stride, int H, int B, float2 *out, cudaStream_t s) {
    dim3 g((unsigned)((H + 127) / 128), (unsigned)B);
    synth_kernel<F><<<g, 128, 0, s>>>(lo, hi, stride, H, B, out, lift_coef(F, SIDE_Y));
    return cudaGetLastError();
}

}  // namespace
}  // namespace sidwt

using namespace sidwt;

extern "C" {

sidwt_status sidwt_synthesize(sidwt_filter f, int64_t H, int64_t B, const void *lo_dev, const void *hi_dev,
                              int64_t in_stride, void *out_dev, sidwt_stream stream) {
    if ((int)f == SIDWT_LEGALL53_INT || (int)f == SIDWT_CDF97_INT) {
        set_error("synthesis takes the float filters");
        return SIDWT_EUNSUPPORTED;
    }
    if ((int)f < 0 || (int)f > 2 || H < 1 || H > (int64_t(1) << 25) || B < 0 || B > 65535 || in_stride < H ||
        (B > 0 && (!lo_dev || !hi_dev || !out_dev))) {
        set_error("bad synthesis arguments");
        return SIDWT_EINVAL;
    }
    if (B == 0) return SIDWT_OK;
    if ((reinterpret_cast<uintptr_t>(lo_dev) | reinterpret_cast<uintptr_t>(hi_dev) |
         reinterpret_cast<uintptr_t>(out_dev)) % 8) {
        set_error("misaligned complex64 buffers");
        return SIDWT_EINVAL;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const float2 *lo = static_cast<const float2 *>(lo_dev), *hi = static_cast<const float2 *>(hi_dev);
    float2 *out = static_cast<float2 *>(out_dev);
    cudaError_t e;
    switch (f) {
    case SIDWT_D4: e = launch_synth<SIDWT_D4>(lo, hi, in_stride, (int)H, (int)B, out, s); break;
    case SIDWT_LEGALL53: e = launch_synth<SIDWT_LEGALL53>(lo, hi, in_stride, (int)H, (int)B, out, s); break;
    default: e = launch_synth<SIDWT_CDF97>(lo, hi, in_stride, (int)H, (int)B, out, s); break;
    }
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "synthesis launch");
}

sidwt_status sidwt_correlate_c2f(sidwt_plan *p, const int32_t *ref_ids_dev, const void *y_dev, int64_t B,
                                 int half_window, int32_t *lag_dev, float *mag_dev, sidwt_stream stream) {
    if (!p) {
        set_error("plan is NULL");
        return SIDWT_EINVAL;
    }
    if (B < 0 || B > 0x7fffffff || half_window < 1 || (B > 0 && (!ref_ids_dev || !y_dev || !lag_dev || !mag_dev))) {
        set_error("bad coarse-to-fine arguments");
        return SIDWT_EINVAL;
    }
    if (B == 0) return SIDWT_OK;
    if (p->nrefs == 0) {
        set_error("no stored reference");
        return SIDWT_EINVAL;
    }
    if (p->N > (int64_t(1) << 30) / std::max(1, half_window)) {
        set_error("window too large");
        return SIDWT_EINVAL;
    }
    sidwt_status st = check_plan_pulses(p, y_dev, B);
    if (st || (st = ensure_plan_batch(p, B))) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // scale J at every delay on the FP32 correlation kernel (its peak key per
    // pulse), then the windows of the finer scales
    if ((st = group_pulses(p, ref_ids_dev, B, simt_tile_pulses(), s)) || (st = analyze_batch(p, y_dev, B, s)))
        return st;
    p->analyzed_B = B;
    ++p->analysis_gen;
    p->keys_clean = false;  // scale J's keys are left set
    cudaError_t e = cudaMemsetAsync(p->keys, 0, B * (p->J + 1) * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    if ((st = correlate_simt(p, B, nullptr, s, 1u << p->J))) return st;
    c2f_kernel<<<(unsigned)B, kC2fThreads, 0, s>>>(p->tree_f, p->tree_elems, p->pyr_f, p->pyr_elems, p->ref_ids,
                                                   p->nrefs, p->N, p->J, half_window, p->keys, lag_dev, mag_dev);
    e = cudaGetLastError();
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "coarse-to-fine launch");
}

}  // extern "C"
