// Lifting kernels: the received (dual-basis) analysis of a batch of pulses,
// all J levels in one pass through shared memory, and the stored signal's
// SIDWT tree (even and odd children at every level).
//
// Received analysis (Sec. III, Fig. 3(b) / 4(b); eq. 17 for D4): one CTA per
// pulse.  The pulse is read once with 128-bit loads straight into its two
// polyphase phases (the split is fused into the load), each lifting step runs
// over the level in shared memory, and the scaled outputs go to HBM while the
// approximation is written, already split into the next level's phases, into
// the other half of a 1.5 N ping-pong buffer.  Levels ping-pong between the
// regions [0, N) and [N, 1.5 N).
//
// SIDWT tree (Sec. II, Fig. 1 and 5): level j -> j+1 for all 2^j variants and
// both children at once; every thread recomputes one output pair from an
// 11-sample window of its input (the lifting steps have support <= 9), so a
// level is one fully parallel launch.  The same window kernel is the
// received-side path for pulses too long for shared memory.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "sidwt_internal.cuh"

namespace sidwt {

LiftCoef lift_coef(int filter, int side) {
    LiftCoef c{};
    if (filter == SIDWT_LEGALL53 || filter == SIDWT_LEGALL53_INT) {
        if (side == SIDE_X) {  // P~(z^-1) = diag(1, 1/2) U((1+z^-1)/4) P(-(1+z)/2)
            c.c0[0] = c.c1[0] = -0.5f;
            c.c0[1] = c.c1[1] = 0.25f;
            c.ce = 1.0f;
            c.co = 0.5f;
        } else {  // P^T(z^-1) = diag(1, 2) P(-(1+z)/4) U((1+z^-1)/2)
            c.c0[0] = c.c1[0] = 0.5f;
            c.c0[1] = c.c1[1] = -0.25f;
            c.ce = 1.0f;
            c.co = 2.0f;
        }
    } else if (filter == SIDWT_CDF97) {  // Table I, t = 5/4
        const double a = -1.5, b = -1.0 / 16.0, g = 4.0 / 5.0, d = 15.0 / 32.0;
        const double x = 4.0 * std::sqrt(2.0) / 5.0;
        const double st[4] = {a, b, g, d};
        for (int s = 0; s < 4; ++s) {
            double v = (side == SIDE_X) ? st[s] : -st[s];
            c.c0[s] = c.c1[s] = (float)v;
        }
        c.ce = (float)((side == SIDE_X) ? x : 1.0 / x);
        c.co = (float)((side == SIDE_X) ? 1.0 / x : x);
    } else {  // causal D4, eq. 17
        const double s3 = std::sqrt(3.0), s2 = std::sqrt(2.0);
        c.c0[0] = (float)(-s3);
        c.c1[0] = 0.0f;
        c.c0[1] = (float)(s3 / 4.0);
        c.c1[1] = (float)((s3 - 2.0) / 4.0);
        c.ce = (float)((s3 + 1.0) / s2);
        c.co = (float)((s3 - 1.0) / s2);
    }
    return c;
}

// CDF 9/7 with free parameter t (Sec. III-C Case II): a = (1 - 2t) / (4 (t - 1)),
// b = -(t - 1)^2, g = 1 / (4 t (t - 1)), d = t^3 - 7/4 t^2 + t, x = sqrt(2) / t;
// the same step structure as Table I (t = 5/4).
LiftCoef lift_coef_97t(double t, int side) {
    LiftCoef c{};
    const double a = (1.0 - 2.0 * t) / (4.0 * (t - 1.0)), b = -(t - 1.0) * (t - 1.0);
    const double g = 1.0 / (4.0 * t * (t - 1.0)), d = t * t * t - 1.75 * t * t + t;
    const double x = std::sqrt(2.0) / t;
    const double st[4] = {a, b, g, d};
    for (int s = 0; s < 4; ++s) {
        const double v = (side == SIDE_X) ? st[s] : -st[s];
        c.c0[s] = c.c1[s] = (float)v;
    }
    c.ce = (float)((side == SIDE_X) ? x : 1.0 / x);
    c.co = (float)((side == SIDE_X) ? 1.0 / x : x);
    return c;
}

LiftCoef plan_coef(const sidwt_plan *p, int side) {
    return (p->filter == SIDWT_CDF97 && p->t97 != 0.0) ? lift_coef_97t(p->t97, side) : lift_coef(p->filter, side);
}

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 axpy2(float2 x, float c0, float2 y0, float c1, float2 y1) {
    x.x = fmaf(c1, y1.x, fmaf(c0, y0.x, x.x));
    x.y = fmaf(c1, y1.y, fmaf(c0, y0.y, x.y));
    return x;
}
__device__ __forceinline__ float2 scale2(float s, float2 v) { return make_float2(s * v.x, s * v.y); }
__device__ __forceinline__ int wrapi(int64_t i, int64_t m) {
    int64_t r = i % m;
    return (int)(r < 0 ? r + m : r);
}

template <typename T>
__device__ __forceinline__ float2 to_f2(T v);
template <>
__device__ __forceinline__ float2 to_f2<float2>(float2 v) { return v; }
template <>
__device__ __forceinline__ float2 to_f2<int2>(int2 v) { return make_float2((float)v.x, (float)v.y); }

template <typename T>
__device__ __forceinline__ int2 to_i2(T v);
template <>
__device__ __forceinline__ int2 to_i2<short2>(short2 v) { return make_int2(v.x, v.y); }
template <>
__device__ __forceinline__ int2 to_i2<int2>(int2 v) { return v; }


// Energy accumulator (eq. 1).  The FP64 pipe of this part runs at a small
// fraction of FP32, so the sums are kept as unevaluated pairs of floats
// (hi + lo, Knuth's TwoSum), which carry about 48 significant bits; squares
// are formed in FP32 from the FP32 coefficients.  Only the final value of a
// block sum is converted to double.
struct EnAcc {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float s = hi + x;
        const float bb = s - hi;
        const float e = (hi - (s - bb)) + (x - bb);
        hi = s;
        lo += e;
    }
    __device__ __forceinline__ void add(const EnAcc &o) {
        add(o.hi);
        lo += o.lo;
    }
    __device__ __forceinline__ double total() const { return (double)hi + (double)lo; }
};
__device__ __forceinline__ float sq2(float2 v) { return fmaf(v.x, v.x, v.y * v.y); }
__device__ __forceinline__ long long sq2i(int2 v) { return (long long)v.x * v.x + (long long)v.y * v.y; }

// Deterministic block sum of one pair-of-floats accumulator per thread
// (blockDim.x multiple of 32); the result, in double, is valid in thread 0.
__device__ double block_sum(EnAcc v, float2 *red) {
    for (int o = 16; o > 0; o >>= 1) {
        EnAcc t;
        t.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
        t.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
        v.add(t);
    }
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = make_float2(v.hi, v.lo);
    __syncthreads();
    EnAcc t;
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; ++i) {
            EnAcc u;
            u.hi = red[i].x;
            u.lo = red[i].y;
            t.add(u);
        }
    return t.total();
}

// Deterministic block sum of one int64 per thread, returned as double.
__device__ double block_sum_i64(long long v, long long *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    long long t = 0;
    if (threadIdx.x == 0)
        for (int i = 0; i < nw; ++i) t += red[i];
    return (double)t;  // valid in thread 0
}

// ---------------------------------------------------------------------------
// Integer 5/3 steps (floor division by arithmetic shift; Sec. I / V-B).
// x side: O -= (E[n] + E[n+1]) >> 1;  E += (O[n-1] + O[n] + 2) >> 2.
// y side: E += (O[n] + O[n-1] + 1) >> 1;  O -= (E[n] + E[n+1] + 2) >> 2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int2 isub_shr(int2 x, int2 a, int2 b, int add, int sh) {
    return make_int2(x.x - ((a.x + b.x + add) >> sh), x.y - ((a.y + b.y + add) >> sh));
}
__device__ __forceinline__ int2 iadd_shr(int2 x, int2 a, int2 b, int add, int sh) {
    return make_int2(x.x + ((a.x + b.x + add) >> sh), x.y + ((a.y + b.y + add) >> sh));
}

// ---------------------------------------------------------------------------
// Window lifting (register arrays, one output pair per thread).
// E[i], O[i] hold the phases at n - R + i.  After the steps the centre R is
// exact (each step consumes at most one neighbour on one side).
// ---------------------------------------------------------------------------
template <int F, int S, int R>
__device__ __forceinline__ void lift_window(float2 (&E)[2 * R + 1], float2 (&O)[2 * R + 1], const LiftCoef &c) {
    using Sh = LiftShape<F, S>;
#pragma unroll
    for (int s = 0; s < Sh::nsteps; ++s) {
        const float c0 = c.c0[s], c1 = c.c1[s];
        if (Sh::target(s) == 1) {
            if (Sh::nb(s) > 0) {
#pragma unroll
                for (int i = 0; i < 2 * R; ++i) O[i] = axpy2(O[i], c0, E[i], c1, E[i + 1]);
            } else {
#pragma unroll
                for (int i = 2 * R; i >= 1; --i) O[i] = axpy2(O[i], c0, E[i], c1, E[i - 1]);
            }
        } else {
            if (Sh::nb(s) > 0) {
#pragma unroll
                for (int i = 0; i < 2 * R; ++i) E[i] = axpy2(E[i], c0, O[i], c1, O[i + 1]);
            } else {
#pragma unroll
                for (int i = 2 * R; i >= 1; --i) E[i] = axpy2(E[i], c0, O[i], c1, O[i - 1]);
            }
        }
    }
}

template <int S, int R>
__device__ __forceinline__ void int53_window(int2 (&E)[2 * R + 1], int2 (&O)[2 * R + 1]) {
    if (S == SIDE_X) {
#pragma unroll
        for (int i = 0; i < 2 * R; ++i) O[i] = isub_shr(O[i], E[i], E[i + 1], 0, 1);
#pragma unroll
        for (int i = 2 * R; i >= 1; --i) E[i] = iadd_shr(E[i], O[i - 1], O[i], 2, 2);
    } else {
#pragma unroll
        for (int i = 2 * R; i >= 1; --i) E[i] = iadd_shr(E[i], O[i], O[i - 1], 1, 1);
#pragma unroll
        for (int i = 0; i < 2 * R; ++i) O[i] = isub_shr(O[i], E[i], E[i + 1], 2, 2);
    }
}

// Integer CDF 9/7 (dyadic Table I steps, rounded updates, no scaling):
// R(c s) = floor((k s + 2^(m-1)) / 2^m) for c = k / 2^m, with a = -3/2,
// b = -1/16, g = 205/256, d = 15/32 (x side; the y side negates them and
// updates the other phase first).
__device__ __forceinline__ int rdy(int k, int m, int s) {
    return (int)(((long long)k * s + (1ll << (m - 1))) >> m);  // arithmetic shift: floor
}
__device__ __forceinline__ int2 iupd(int2 t, int k, int m, int2 p, int2 q) {
    return make_int2(t.x + rdy(k, m, p.x + q.x), t.y + rdy(k, m, p.y + q.y));
}

template <int S, int R>
__device__ __forceinline__ void int97_window(int2 (&E)[2 * R + 1], int2 (&O)[2 * R + 1]) {
    constexpr int K[4] = {-3, -1, 205, 15}, M[4] = {1, 4, 8, 5};
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const bool odd = (S == SIDE_X) ? (s % 2 == 0) : (s % 2 == 1);
        const int k = (S == SIDE_X) ? K[s] : -K[s];
        if (odd) {
#pragma unroll
            for (int i = 0; i < 2 * R; ++i) O[i] = iupd(O[i], k, M[s], E[i], E[i + 1]);
        } else {
#pragma unroll
            for (int i = 2 * R; i >= 1; --i) E[i] = iupd(E[i], k, M[s], O[i], O[i - 1]);
        }
    }
}

// The integer filter's window steps (F: SIDWT_LEGALL53_INT or SIDWT_CDF97_INT).
template <int F, int S, int R>
__device__ __forceinline__ void int_window(int2 (&E)[2 * R + 1], int2 (&O)[2 * R + 1]) {
    if constexpr (F == SIDWT_CDF97_INT)
        int97_window<S, R>(E, O);
    else
        int53_window<S, R>(E, O);
}

__host__ __device__ constexpr bool is_int_filter(int F) { return F == SIDWT_LEGALL53_INT || F == SIDWT_CDF97_INT; }

constexpr int WR = 5;  // window radius

// One analysis level over many rows by per-output recomputation.
// Row r (of nrows) of `in` has K samples at in + r * in_stride; child 1 reads
// the row delayed by one sample.  Output row (r + child * nrows) of length
// K/2 goes to lo/hi at row stride out_stride.
// Output pair n of one analysis level of the periodic row v (K samples),
// delayed by `child` samples: the window of 2 WR + 1 phase pairs around n,
// lifted in registers.
template <int F, int S, typename TIn>
__device__ __forceinline__ void window_pair(const TIn *__restrict__ v, int64_t K, int64_t n, int child,
                                            const LiftCoef &c, float2 &l, float2 &h) {
    using Sh = LiftShape<F, S>;
    float2 E[2 * WR + 1], O[2 * WR + 1];
    // E[i] sits at base + 2 i and O[i] at base + 2 i -+ 1: a window that does
    // not reach past either end of the row reads it directly, the others wrap
    // (periodic extension, any number of times for rows shorter than it)
    const int64_t base = 2 * (n - WR) - child;
    if (base - 1 >= 0 && base + 4 * WR + 1 < K) {
        const TIn *p = v + base;
#pragma unroll
        for (int i = 0; i <= 2 * WR; ++i) {
            E[i] = to_f2(p[2 * i]);
            O[i] = to_f2(p[Sh::d4 ? 2 * i - 1 : 2 * i + 1]);
        }
    } else {
#pragma unroll
        for (int i = 0; i <= 2 * WR; ++i) {
            const int64_t m = n - WR + i;
            E[i] = to_f2(v[wrapi(2 * m - child, K)]);
            O[i] = to_f2(v[wrapi(Sh::d4 ? 2 * m - 1 - child : 2 * m + 1 - child, K)]);
        }
    }
    lift_window<F, S, WR>(E, O, c);
    l = scale2(c.ce, E[WR]);
    if (Sh::d4) h = scale2(c.co, make_float2(E[WR].x + O[WR - 1].x, E[WR].y + O[WR - 1].y));
    else h = scale2(c.co, O[WR]);
}

template <int F, int S, typename TIn>
__global__ void level_window_f(const TIn *__restrict__ in, int64_t in_stride, int nrows, int nchild, int64_t K,
                               float2 *__restrict__ lo, float2 *__restrict__ hi, int64_t out_stride, LiftCoef c) {
    const int64_t H = K / 2;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= H) return;
    const int rc = blockIdx.y;
    const int row = rc % nrows, child = rc / nrows;
    if (child >= nchild) return;
    float2 l, h;
    window_pair<F, S>(in + (int64_t)row * in_stride, K, n, child, c, l, h);
    const int64_t orow = (int64_t)(row + child * nrows) * out_stride;
    lo[orow + n] = l;
    hi[orow + n] = h;
}

// Stored SIDWT trees of many signals at once (x side, float filters): one
// launch per level for every tree of the batch.  Item k's level j + 1 is
// N_k outputs (2^(j+1) variant rows of N_k / 2^(j+1), in the A and the B
// band), one thread each; the items are sorted by decreasing J, so the
// items still lifting at level j are the first n_active, and a thread finds
// its item by binary search in the prefix sums of N.
template <int F>
__global__ void tree_level_batch_kernel(const float2 *__restrict__ x, float2 *__restrict__ tree,
                                        const __grid_constant__ TreeBatch b, int j, int n_active, LiftCoef c) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= b.nprefix[n_active]) return;
    int lo_k = 0, hi_k = n_active - 1;
    while (lo_k < hi_k) {  // last k with nprefix[k] <= t
        const int mid = (lo_k + hi_k + 1) >> 1;
        if (b.nprefix[mid] <= t) lo_k = mid;
        else hi_k = mid - 1;
    }
    const TreeItem it = b.it[lo_k];
    // 32-bit index arithmetic (an item's outputs per level number N < 2^31);
    // the 2^j rows of a child are a power of two
    const int64_t N = it.N;
    const int32_t local = (int32_t)(t - b.nprefix[lo_k]);
    const int32_t K = (int32_t)(N >> j), H = K / 2;
    const int32_t orow = local / H, n = local - orow * H;
    const int row = orow & ((1 << j) - 1), child = orow >> j;
    const float2 *v = j == 0 ? x + it.x_off : tree + it.tree_off + 2 * N * (int64_t)(j - 1) + (int64_t)row * K;
    float2 l, h;
    window_pair<F, SIDE_X>(v, K, n, child, c, l, h);
    float2 *A = tree + it.tree_off + 2 * N * (int64_t)j;
    A[orow * H + n] = l;
    A[N + orow * H + n] = h;
}

// Energies of a stored tree: row r of out (levels l = 0..J, variants
// v < 2^l, r = 2^l - 1 + v) is ||c_l^v||^2 over K = N >> l samples (x itself
// at l = 0).  Rows of K >= kEnBigRow samples are summed by a whole block, the
// others by one warp each (eight a block), so that the many short rows of the
// deep levels do not each hold a block.  Which form sums a row depends on K
// alone, so a tree's energies come out the same from the single-signal and
// the batched launches.
constexpr int kEnBigRow = 4096;

__host__ __device__ inline int energy_big_rows(int64_t N, int J) {
    int n = 0;
    for (int l = 0; l <= J && (N >> l) >= kEnBigRow; ++l) n += 1 << l;
    return n;
}
__host__ __device__ inline int64_t energy_blocks(int64_t N, int J) {
    const int rows = (2 << J) - 1, big = energy_big_rows(N, J);
    return big + (rows - big + 7) / 8;
}

// One warp's sum of |X[k]|^2: lanes stride the row with four FP32-pair
// accumulators each, then a fixed compensated tree; valid in lane 0.
__device__ __forceinline__ double warp_row_energy(const float2 *__restrict__ X, int64_t K) {
    const int lane = threadIdx.x & 31;
    EnAcc a0, a1, a2, a3;
    int64_t k = lane;
    for (; k + 96 < K; k += 128) {
        a0.add(sq2(X[k]));
        a1.add(sq2(X[k + 32]));
        a2.add(sq2(X[k + 64]));
        a3.add(sq2(X[k + 96]));
    }
    for (; k < K; k += 32) a0.add(sq2(X[k]));
    a0.add(a1);
    a2.add(a3);
    a0.add(a2);
    for (int o = 16; o > 0; o >>= 1) {
        EnAcc t;
        t.hi = __shfl_down_sync(0xffffffffu, a0.hi, o);
        t.lo = __shfl_down_sync(0xffffffffu, a0.lo, o);
        a0.add(t);
    }
    return a0.total();
}

// Energy block bl of one tree (x: the signal, tr: its tree, out: its
// 2^(J+1) - 1 energies); blockDim.x = 256.
__device__ __forceinline__ void tree_energy_block(const float2 *__restrict__ x, const float2 *__restrict__ tr,
                                                  int64_t N, int J, int bl, double *__restrict__ out, float2 *red) {
    const int big = energy_big_rows(N, J), rows = (2 << J) - 1;
    const bool whole = bl < big;  // uniform over the block
    const int r = whole ? bl : big + (bl - big) * 8 + (int)(threadIdx.x >> 5);
    if (!whole && r >= rows) return;
    int l = 0;
    while ((2 << l) - 1 <= r) ++l;
    const int v = r - ((1 << l) - 1);
    const int64_t K = N >> l;
    const float2 *X = l == 0 ? x : tr + 2 * N * (int64_t)(l - 1) + (int64_t)v * K;
    if (whole) {
        EnAcc acc;
        for (int64_t k = threadIdx.x; k < K; k += blockDim.x) acc.add(sq2(X[k]));
        const double t = block_sum(acc, red);
        if (threadIdx.x == 0) out[r] = t;
    } else {
        const double t = warp_row_energy(X, K);
        if ((threadIdx.x & 31) == 0) out[r] = t;
    }
}

// Energies of the batch's trees: block e -> item k (prefix sums of
// energy_blocks per item), then tree_energy_block.
__global__ void tree_energy_batch_kernel(const float2 *__restrict__ x, const float2 *__restrict__ tree,
                                         double *__restrict__ xen, const __grid_constant__ TreeBatch b) {
    __shared__ float2 red[32];
    const int64_t e = blockIdx.x;
    int lo_k = 0, hi_k = b.n - 1;
    while (lo_k < hi_k) {
        const int mid = (lo_k + hi_k + 1) >> 1;
        if (b.eprefix[mid] <= e) lo_k = mid;
        else hi_k = mid - 1;
    }
    const TreeItem it = b.it[lo_k];
    tree_energy_block(x + it.x_off, tree + it.tree_off, it.N, it.J, (int)(e - b.eprefix[lo_k]), xen + it.xen_off,
                      red);
}

template <int F, int S, typename TIn>
__global__ void level_window_i(const TIn *__restrict__ in, int64_t in_stride, int nrows, int nchild, int64_t K,
                               int2 *__restrict__ lo, int2 *__restrict__ hi, int64_t out_stride,
                               float2 *__restrict__ lo_f, float2 *__restrict__ hi_f) {
    const int64_t H = K / 2;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= H) return;
    const int rc = blockIdx.y;
    const int row = rc % nrows, child = rc / nrows;
    if (child >= nchild) return;
    const TIn *v = in + (int64_t)row * in_stride;
    int2 E[2 * WR + 1], O[2 * WR + 1];
#pragma unroll
    for (int i = 0; i <= 2 * WR; ++i) {
        const int64_t m = n - WR + i;
        E[i] = to_i2(v[wrapi(2 * m - child, K)]);
        O[i] = to_i2(v[wrapi(2 * m + 1 - child, K)]);
    }
    int_window<F, S, WR>(E, O);
    const int64_t o = (int64_t)(row + child * nrows) * out_stride + n;
    lo[o] = E[WR];
    hi[o] = O[WR];
    if (lo_f) {
        lo_f[o] = to_f2(E[WR]);
        hi_f[o] = to_f2(O[WR]);
    }
}

// Energies ||X_{l,v}||^2 of one reference: block b -> (level l, variant v)
// with b = 2^l - 1 + v.  Level 0 reads x, level l >= 1 the stored A band.
template <typename TIn, typename TTree>
__global__ void ref_energy_kernel(const TIn *__restrict__ x, const TTree *__restrict__ tree, int64_t N,
                                  double *__restrict__ out);

// One float tree's energies: energy_blocks(N, J) blocks of 256 threads.
__global__ void ref_energy_f_kernel(const float2 *__restrict__ x, const float2 *__restrict__ tree, int64_t N, int J,
                                    double *__restrict__ out) {
    __shared__ float2 red[32];
    tree_energy_block(x, tree, N, J, blockIdx.x, out, red);
}

template <>
__global__ void ref_energy_kernel<short2, int2>(const short2 *__restrict__ x, const int2 *__restrict__ tree,
                                               int64_t N, double *__restrict__ out) {
    __shared__ long long red[32];
    const int b = blockIdx.x;
    int l = 0;
    while ((2 << l) - 1 <= b) ++l;
    const int v = b - ((1 << l) - 1);
    const int64_t K = N >> l;
    long long acc = 0;
    if (l == 0) {
        for (int64_t k = threadIdx.x; k < K; k += blockDim.x) acc += sq2i(make_int2(x[k].x, x[k].y));
    } else {
        const int2 *A = tree + 2 * N * (int64_t)(l - 1) + (int64_t)v * K;
        for (int64_t k = threadIdx.x; k < K; k += blockDim.x) acc += sq2i(A[k]);
    }
    const double t = block_sum_i64(acc, red);
    if (threadIdx.x == 0) out[b] = t;
}

// ---------------------------------------------------------------------------
// Received analysis, all levels in one pass through shared memory.
// Level l reads its input (the level l-1 approximation, natural order) from
// one region and writes its approximation to the other; every thread
// computes whole output pairs (c_l[n], d_l[n]) by running the lifting steps
// in registers on a 5-pair window read as 128-bit (even, odd) loads, so a
// level needs a single barrier.
// ---------------------------------------------------------------------------
constexpr int kAnalyzeThreads = 512;

__device__ __forceinline__ int wrap_small(int m, int H) {
    if (m < 0) m += H;
    if (m >= H) m -= H;
    if ((unsigned)m >= (unsigned)H) m = ((m % H) + H) % H;  // tiny levels (H < 3)
    return m;
}

template <int F>
__device__ __forceinline__ void out_pair_f(const float2 *in, int H, int n, const LiftCoef &c, float2 &lo, float2 &hi) {
    constexpr bool D4 = (F == SIDWT_D4);
    const float4 *q = reinterpret_cast<const float4 *>(in);  // q[m] = (in[2m], in[2m+1])
    float2 E[5], O[5];
    if (D4) {
        float4 prev = q[wrap_small(n - 3, H)];
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const float4 cur = q[wrap_small(n - 2 + i, H)];
            E[i] = make_float2(cur.x, cur.y);
            O[i] = make_float2(prev.z, prev.w);  // odd phase of D4: v[2m-1]
            prev = cur;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const float4 cur = q[wrap_small(n - 2 + i, H)];
            E[i] = make_float2(cur.x, cur.y);
            O[i] = make_float2(cur.z, cur.w);
        }
    }
    lift_window<F, SIDE_Y, 2>(E, O, c);
    lo = scale2(c.ce, E[2]);
    if (D4) hi = scale2(c.co, make_float2(E[2].x + O[1].x, E[2].y + O[1].y));
    else hi = scale2(c.co, O[2]);
}

template <int F>
__device__ __forceinline__ void out_pair_i(const int2 *in, int H, int n, int2 &lo, int2 &hi) {
    const int4 *q = reinterpret_cast<const int4 *>(in);
    int2 E[5], O[5];
    const bool interior = n >= 2 && n + 2 < H;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const int4 cur = q[interior ? n - 2 + i : wrap_small(n - 2 + i, H)];
        E[i] = make_int2(cur.x, cur.y);
        O[i] = make_int2(cur.z, cur.w);
    }
    int_window<F, SIDE_Y, 2>(E, O);
    lo = E[2];
    hi = O[2];
}

// All J levels of one pulse by one CTA.  y: the pulse (complex64 or int16
// I/Q); pyr_f / pyr_i: its pyramid row; yen: its J+1 energies.  Shared
// memory: 1.5 N elements of T (float2 or int2).
template <int F, typename T>
__device__ __forceinline__ void analyze_one(const void *__restrict__ y, int64_t N, int J, float2 *__restrict__ pyr_f,
                                            int2 *__restrict__ pyr_i, double *__restrict__ yen, const LiftCoef &c,
                                            T *sm, float2 *red, long long *redi) {
    constexpr bool INT = is_int_filter(F);
    const int Nh = (int)(N / 2);
    EnAcc en;
    long long eni = 0;

    // level-0 load, 128-bit (float) or 64-bit (int16 I/Q) per sample pair
    if constexpr (INT) {
        const short4 *y4 = reinterpret_cast<const short4 *>(y);
        int4 *d4 = reinterpret_cast<int4 *>(sm);
        for (int n = threadIdx.x; n < Nh; n += blockDim.x) {
            const short4 v = y4[n];
            d4[n] = make_int4(v.x, v.y, v.z, v.w);
            eni += sq2i(make_int2(v.x, v.y)) + sq2i(make_int2(v.z, v.w));
        }
    } else {
        const float4 *y4 = reinterpret_cast<const float4 *>(y);
        float4 *d4 = reinterpret_cast<float4 *>(sm);
        for (int n = threadIdx.x; n < Nh; n += blockDim.x) {
            const float4 v = y4[n];
            d4[n] = v;
            en.add(sq2(make_float2(v.x, v.y)));
            en.add(sq2(make_float2(v.z, v.w)));
        }
    }
    {
        const double t = INT ? block_sum_i64(eni, redi) : block_sum(en, red);
        if (threadIdx.x == 0) yen[0] = t;
    }
    __syncthreads();

    for (int l = 1; l <= J; ++l) {
        const int H = (int)(N >> l);
        const T *in = sm + ((l & 1) ? 0 : N);
        T *out = sm + ((l & 1) ? N : 0);
        const int64_t off = 2 * N - 4 * (int64_t)H;
        en = EnAcc();
        eni = 0;
        for (int n = threadIdx.x; n < H; n += blockDim.x) {
            T lo, hi;
            if constexpr (INT) {
                out_pair_i<F>(reinterpret_cast<const int2 *>(in), H, n, lo, hi);
                pyr_i[off + n] = lo;
                pyr_i[off + H + n] = hi;
                pyr_f[off + n] = to_f2(lo);
                pyr_f[off + H + n] = to_f2(hi);
                eni += sq2i(lo);
            } else {
                out_pair_f<F>(reinterpret_cast<const float2 *>(in), H, n, c, lo, hi);
                pyr_f[off + n] = lo;
                pyr_f[off + H + n] = hi;
                en.add(sq2(lo));
            }
            out[n] = lo;
        }
        const double t = INT ? block_sum_i64(eni, redi) : block_sum(en, red);
        if (threadIdx.x == 0) yen[l] = t;
        __syncthreads();
    }
}

// One CTA per pulse of a uniform batch.
template <int F, typename T>
__global__ void __launch_bounds__(kAnalyzeThreads) analyze_smem_kernel(const void *__restrict__ y_in, int64_t N, int J,
                                                                       float2 *__restrict__ pyr_f,
                                                                       int2 *__restrict__ pyr_i, int64_t pyr_elems,
                                                                       double *__restrict__ yen, LiftCoef c) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ float2 red[32];
    __shared__ long long redi[32];
    constexpr bool INT = is_int_filter(F);
    const int64_t b = blockIdx.x;
    const char *y = reinterpret_cast<const char *>(y_in) + b * N * (INT ? 4 : 8);
    analyze_one<F, T>(y, N, J, pyr_f + b * pyr_elems, INT ? pyr_i + b * pyr_elems : nullptr, yen + b * (J + 1), c,
                      reinterpret_cast<T *>(smraw), red, redi);
}

// ---------------------------------------------------------------------------
// Pipelined received analysis of a uniform batch: a persistent grid, each CTA
// walking pulses b, b + G, ...  While the levels of one pulse run, a bulk
// copy (TMA, cp.async.bulk) brings the next pulse into the other of two
// input buffers, so the HBM reads stay in flight across the whole kernel.
// Shared memory: two raw input buffers (N samples of the input type) and a
// level-1 buffer W of N/2 elements of T; level l >= 2 alternates between W
// and the current input buffer (free once level 1 has read it).  Energies:
// warp partial sums per level, one cross-warp sum per pulse.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool pipe_wait(uint64_t *bar, uint32_t parity) {
    uint64_t t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 200ull * 1000 * 1000) return false;  // 200 ms
    }
}

__device__ __forceinline__ void pipe_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Level-1 window of the integer path straight from the int16 I/Q input.
template <int F>
__device__ __forceinline__ void out_pair_i16(const short2 *in, int H, int n, int2 &lo, int2 &hi) {
    const short4 *q = reinterpret_cast<const short4 *>(in);
    int2 E[5], O[5];
    const bool interior = n >= 2 && n + 2 < H;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const short4 cur = q[interior ? n - 2 + i : wrap_small(n - 2 + i, H)];
        E[i] = make_int2(cur.x, cur.y);
        O[i] = make_int2(cur.z, cur.w);
    }
    int_window<F, SIDE_Y, 2>(E, O);
    lo = E[2];
    hi = O[2];
}

constexpr int kPipeMaxLevels = 16;
constexpr int kPipeThreads = 512;

template <int F, typename T, bool RAGGED = false>
__global__ void __launch_bounds__(kPipeThreads) analyze_pipe_kernel(const void *__restrict__ y_in, int64_t N, int J,
                                                                       int64_t B, float2 *__restrict__ pyr_f,
                                                                       int2 *__restrict__ pyr_i, int64_t pyr_elems,
                                                                       double *__restrict__ yen, LiftCoef c,
                                                                       int32_t *__restrict__ err, int nbuf,
                                                                       int stall,
                                                                       const RaggedLift *__restrict__ items) {
    constexpr bool INT = is_int_filter(F);
    constexpr int IN_BYTES = INT ? 4 : 8;
    extern __shared__ __align__(16) unsigned char smraw[];  // 16-byte aligned: enough for the bulk copies
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float2 redf[kPipeMaxLevels][kPipeThreads / 32];
    __shared__ long long redi[kPipeMaxLevels][kPipeThreads / 32];
    __shared__ int sfail;
    // RAGGED: item b of `items` has its own N, J and places (pulse, pyramid
    // row, energies); the shared buffers are sized for N, the longest of them
    const uint32_t bytes = (uint32_t)(N * IN_BYTES);
    const size_t inb = ((size_t)bytes + 127) & ~(size_t)127;
    unsigned char *const buf0 = smraw, *const buf1 = smraw + inb;
    T *W = reinterpret_cast<T *>(smraw + nbuf * inb);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const char *y = reinterpret_cast<const char *>(y_in);
    const int64_t G = gridDim.x;
    pdl_release();  // the correlation kernel may be scheduled now; it waits for this grid's writes

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sfail = 0;
    }
    __syncthreads();
    // stall (test hook, sidwt_debug_stall): no copy is issued, so the first
    // wait runs out and the CTA records the timeout with nothing in flight
    auto src = [&](int64_t q) { return RAGGED ? y + items[q].y_off * IN_BYTES : y + q * (int64_t)bytes; };
    auto len = [&](int64_t q) { return RAGGED ? (uint32_t)(items[q].N * IN_BYTES) : bytes; };
    if (tid == 0 && !stall) pipe_load(buf0, src(blockIdx.x), len(blockIdx.x), &bar[0]);
    int i = 0;
    int64_t issued = stall ? 0 : 1, landed = 0;  // copies issued / waited for (thread 0's bookkeeping)
    for (int64_t b = blockIdx.x; b < B; b += G, ++i) {
        // two buffers: pulse i in buffer i % 2, the next one loading meanwhile;
        // one buffer: pulse i loads once pulse i - 1 is done (other CTAs on the
        // SM overlap it)
        const int s = nbuf == 2 ? (i & 1) : 0;
        unsigned char *const cur = s ? buf1 : buf0;
        if (tid == 0 && !stall) {
            // the buffer written next held a finished pulse, whose accesses ended at the last barrier
            if (nbuf == 2 && b + G < B) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                pipe_load(s ? buf0 : buf1, src(b + G), len(b + G), &bar[s ^ 1]);
                ++issued;
            } else if (nbuf == 1 && i > 0) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                pipe_load(buf0, src(b), len(b), &bar[0]);
                ++issued;
            }
        }
        if (!pipe_wait(&bar[s], (uint32_t)(nbuf == 2 ? ((i >> 1) & 1) : (i & 1)))) sfail = 1;
        __syncthreads();
        if (sfail) break;
        if (tid == 0) ++landed;
        const int64_t Nb = RAGGED ? (int64_t)items[b].N : N;
        const int Jb = RAGGED ? items[b].J : J;
        const int Nhb = (int)(Nb / 2);
        float2 *pf = RAGGED ? pyr_f + items[b].pyr_off : pyr_f + b * pyr_elems;
        int2 *pi = INT ? pyr_i + b * pyr_elems : nullptr;
        double *yb = RAGGED ? yen + items[b].yen_off : yen + b * (J + 1);

        // level-0 energy from the landed input
        {
            long long eni = 0;
            if constexpr (INT) {
                const short4 *q = reinterpret_cast<const short4 *>(cur);
                for (int n = tid; n < Nhb; n += blockDim.x) {
                    const short4 v = q[n];
                    eni += sq2i(make_int2(v.x, v.y)) + sq2i(make_int2(v.z, v.w));
                }
                for (int o = 16; o > 0; o >>= 1) eni += __shfl_xor_sync(0xffffffffu, eni, o);
                if (lane == 0) redi[0][warp] = eni;
            } else {
                const float4 *q = reinterpret_cast<const float4 *>(cur);
                float ens = 0.f;
                for (int n = tid; n < Nhb; n += blockDim.x) {
                    const float4 v = q[n];
                    ens = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, ens))));
                }
                // a thread's partial is a plain FP32 sum of N / 256 squares
                // at most; the warp tree adds five roundings more, so the
                // compensated sum is kept for the cross-warp total only
                for (int o = 16; o > 0; o >>= 1) ens += __shfl_xor_sync(0xffffffffu, ens, o);
                if (lane == 0) redf[0][warp] = make_float2(ens, 0.f);
            }
        }
        for (int l = 1; l <= Jb; ++l) {
            const int H = (int)(Nb >> l);
            const int64_t off = 2 * Nb - 4 * (int64_t)H;
            T *out = (l & 1) ? W : reinterpret_cast<T *>(cur);
            const T *in = (l & 1) ? reinterpret_cast<const T *>(cur) : W;
            EnAcc en;
            long long eni = 0;
            if constexpr (!INT) {
                // one output pair per thread and window; interior windows skip the
                // periodic wrap, and the energy is a plain per-thread sum (at most
                // a few dozen terms) made exact-ish by the compensated warp reduction
                constexpr bool D4 = (F == SIDWT_D4);
                const float4 *q = reinterpret_cast<const float4 *>(in);
                float2 *po = reinterpret_cast<float2 *>(out);
                float2 *pl = pf + off, *ph = pf + off + H;
                float ens = 0.f;
                for (int n = tid; n < H; n += blockDim.x) {
                    float2 E[5], O[5];
                    if (n >= 3 && n + 2 < H) {
                        float4 prev = D4 ? q[n - 3] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                        for (int i = 0; i < 5; ++i) {
                            const float4 cur = q[n - 2 + i];
                            E[i] = make_float2(cur.x, cur.y);
                            O[i] = D4 ? make_float2(prev.z, prev.w) : make_float2(cur.z, cur.w);
                            prev = cur;
                        }
                    } else {
                        float4 prev = D4 ? q[wrap_small(n - 3, H)] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                        for (int i = 0; i < 5; ++i) {
                            const float4 cur = q[wrap_small(n - 2 + i, H)];
                            E[i] = make_float2(cur.x, cur.y);
                            O[i] = D4 ? make_float2(prev.z, prev.w) : make_float2(cur.z, cur.w);  // D4 odd phase: v[2m-1]
                            prev = cur;
                        }
                    }
                    lift_window<F, SIDE_Y, 2>(E, O, c);
                    const float2 lo = scale2(c.ce, E[2]);
                    const float2 hi = D4 ? scale2(c.co, make_float2(E[2].x + O[1].x, E[2].y + O[1].y)) : scale2(c.co, O[2]);
                    pl[n] = lo;
                    ph[n] = hi;
                    po[n] = lo;
                    ens = fmaf(lo.x, lo.x, fmaf(lo.y, lo.y, ens));
                }
                en.add(ens);
            } else
            for (int n = tid; n < H; n += blockDim.x) {
                T lo, hi;
                if constexpr (INT) {
                    if (l == 1)
                        out_pair_i16<F>(reinterpret_cast<const short2 *>(cur), H, n, lo, hi);
                    else
                        out_pair_i<F>(reinterpret_cast<const int2 *>(in), H, n, lo, hi);
                    pi[off + n] = lo;
                    pi[off + H + n] = hi;
                    pf[off + n] = to_f2(lo);
                    pf[off + H + n] = to_f2(hi);
                    eni += sq2i(lo);
                } else {
                    out_pair_f<F>(reinterpret_cast<const float2 *>(in), H, n, c, lo, hi);
                    pf[off + n] = lo;
                    pf[off + H + n] = hi;
                    en.add(sq2(lo));
                }
                out[n] = lo;
            }
            if constexpr (INT) {
                for (int o = 16; o > 0; o >>= 1) eni += __shfl_xor_sync(0xffffffffu, eni, o);
                if (lane == 0) redi[l][warp] = eni;
            } else {
                float v = en.hi + en.lo;  // one plain FP32 partial (see level 0)
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == 0) redf[l][warp] = make_float2(v, 0.f);
            }
            __syncthreads();
        }
        if (tid <= Jb) {
            if constexpr (INT) {
                long long t = 0;
                for (int w = 0; w < nw; ++w) t += redi[tid][w];
                yb[tid] = (double)t;
            } else {
                EnAcc t;
                for (int w = 0; w < nw; ++w) {
                    EnAcc u;
                    u.hi = redf[tid][w].x;
                    u.lo = redf[tid][w].y;
                    t.add(u);
                }
                yb[tid] = t.total();
            }
        }
        // J = 0 cannot happen (J >= 1): the level loop's last barrier orders
        // every read of cur and W before the next prefetch into cur
    }
    if (tid == 0 && sfail) {
        // let this CTA's own copies land before its shared memory is released
        for (int64_t k = landed; k < issued; ++k)
            pipe_wait(&bar[nbuf == 2 ? (k & 1) : 0], (uint32_t)(nbuf == 2 ? ((k >> 1) & 1) : (k & 1)));
        atomicOr(err, kErrAnalysisWait);
    }
}

// Energies of the received pyramid for the window path (c_l read back).
__global__ void pyr_energy_kernel(const float2 *__restrict__ y, const float2 *__restrict__ pyr_f,
                                  const int2 *__restrict__ pyr_i, const short2 *__restrict__ y_i, int64_t N, int J,
                                  int64_t pyr_elems, double *__restrict__ yen) {
    __shared__ float2 red[32];
    __shared__ long long redi[32];
    const int64_t b = blockIdx.x;
    const int l = blockIdx.y;
    const int64_t K = N >> l;
    const int64_t off = b * pyr_elems + 2 * N - 4 * K;
    if (pyr_i) {
        long long acc = 0;
        if (l == 0) {
            for (int64_t k = threadIdx.x; k < K; k += blockDim.x) {
                const short2 t = y_i[b * N + k];
                acc += sq2i(make_int2(t.x, t.y));
            }
        } else {
            for (int64_t k = threadIdx.x; k < K; k += blockDim.x) acc += sq2i(pyr_i[off + k]);
        }
        const double t = block_sum_i64(acc, redi);
        if (threadIdx.x == 0) yen[b * (J + 1) + l] = t;
    } else {
        EnAcc acc;
        if (l == 0) {
            for (int64_t k = threadIdx.x; k < K; k += blockDim.x) acc.add(sq2(y[b * N + k]));
        } else {
            for (int64_t k = threadIdx.x; k < K; k += blockDim.x) acc.add(sq2(pyr_f[off + k]));
        }
        const double t = block_sum(acc, red);
        if (threadIdx.x == 0) yen[b * (J + 1) + l] = t;
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static constexpr int kSmemLimit = 227 * 1024 - 1024;  // dynamic budget; 1 KB left for static shared memory
// the pipelined kernel's static shared memory: barriers and 2 x 16 x 16 partial energies
static constexpr int kPipeSmemLimit = 227 * 1024 - 8 * 1024;

template <int F, typename TIn>
static void launch_level_f(int side, const TIn *in, int64_t in_stride, int nrows, int nchild, int64_t K,
                           float2 *lo, float2 *hi, int64_t out_stride, const LiftCoef &c, cudaStream_t s) {
    const int64_t H = K / 2;
    dim3 grid((unsigned)((H + 127) / 128), (unsigned)(nrows * nchild));
    if (side == SIDE_X)
        level_window_f<F, SIDE_X, TIn><<<grid, 128, 0, s>>>(in, in_stride, nrows, nchild, K, lo, hi, out_stride, c);
    else
        level_window_f<F, SIDE_Y, TIn><<<grid, 128, 0, s>>>(in, in_stride, nrows, nchild, K, lo, hi, out_stride, c);
}

template <typename TIn>
static void launch_level_any(int filter, int side, const TIn *in, int64_t in_stride, int nrows, int nchild,
                             int64_t K, float2 *lo, float2 *hi, int64_t out_stride, const LiftCoef &c,
                             cudaStream_t s) {
    switch (filter) {
    case SIDWT_D4: launch_level_f<SIDWT_D4>(side, in, in_stride, nrows, nchild, K, lo, hi, out_stride, c, s); break;
    case SIDWT_LEGALL53:
        launch_level_f<SIDWT_LEGALL53>(side, in, in_stride, nrows, nchild, K, lo, hi, out_stride, c, s);
        break;
    default: launch_level_f<SIDWT_CDF97>(side, in, in_stride, nrows, nchild, K, lo, hi, out_stride, c, s); break;
    }
}

template <typename TIn>
static void launch_level_int(int filter, int side, const TIn *in, int64_t in_stride, int nrows, int nchild, int64_t K, int2 *lo,
                             int2 *hi, int64_t out_stride, float2 *lo_f, float2 *hi_f, cudaStream_t s) {
    const int64_t H = K / 2;
    dim3 grid((unsigned)((H + 127) / 128), (unsigned)(nrows * nchild));
    if (side == SIDE_X)
        if (filter == SIDWT_CDF97_INT)
            level_window_i<SIDWT_CDF97_INT, SIDE_X, TIn>
                <<<grid, 128, 0, s>>>(in, in_stride, nrows, nchild, K, lo, hi, out_stride, lo_f, hi_f);
        else
            level_window_i<SIDWT_LEGALL53_INT, SIDE_X, TIn>
                <<<grid, 128, 0, s>>>(in, in_stride, nrows, nchild, K, lo, hi, out_stride, lo_f, hi_f);
    else if (filter == SIDWT_CDF97_INT)
        level_window_i<SIDWT_CDF97_INT, SIDE_Y, TIn>
            <<<grid, 128, 0, s>>>(in, in_stride, nrows, nchild, K, lo, hi, out_stride, lo_f, hi_f);
    else
        level_window_i<SIDWT_LEGALL53_INT, SIDE_Y, TIn>
            <<<grid, 128, 0, s>>>(in, in_stride, nrows, nchild, K, lo, hi, out_stride, lo_f, hi_f);
}

sidwt_status build_reference_tree(sidwt_plan *p, const void *x_dev, int32_t ref, cudaStream_t s) {
    const int64_t N = p->N;
    const int J = p->J;
    const LiftCoef c = plan_coef(p, SIDE_X);
    float2 *tf = p->tree_f + (int64_t)ref * p->tree_elems;
    double *xe = p->xen + (int64_t)ref * p->xen_len;
    if (!p->is_int) {
        for (int j = 0; j < J; ++j) {
            const int64_t K = N >> j;
            const int nv = 1 << j;
            float2 *A = tf + 2 * N * (int64_t)j;  // level j+1 block
            float2 *B = A + N;
            if (j == 0)
                launch_level_any(p->filter, SIDE_X, reinterpret_cast<const float2 *>(x_dev), 0, 1, 2, K, A, B, K / 2, c,
                                 s);
            else
                launch_level_any(p->filter, SIDE_X, tf + 2 * N * (int64_t)(j - 1), K, nv, 2, K, A, B, K / 2, c, s);
        }
        ref_energy_f_kernel<<<(unsigned)energy_blocks(N, J), 256, 0, s>>>(reinterpret_cast<const float2 *>(x_dev), tf,
                                                                           N, J, xe);
    } else {
        int2 *ti = p->tree_i + (int64_t)ref * p->tree_elems;
        for (int j = 0; j < J; ++j) {
            const int64_t K = N >> j;
            const int nv = 1 << j;
            int2 *A = ti + 2 * N * (int64_t)j;
            int2 *B = A + N;
            float2 *Af = tf + 2 * N * (int64_t)j;
            float2 *Bf = Af + N;
            if (j == 0)
                launch_level_int(p->filter, SIDE_X, reinterpret_cast<const short2 *>(x_dev), 0, 1, 2, K, A, B, K / 2, Af, Bf,
                                 s);
            else
                launch_level_int(p->filter, SIDE_X, ti + 2 * N * (int64_t)(j - 1), K, nv, 2, K, A, B, K / 2, Af, Bf, s);
        }
        ref_energy_kernel<short2, int2><<<(1 << (J + 1)) - 1, 256, 0, s>>>(
            reinterpret_cast<const short2 *>(x_dev), ti, N, xe);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "reference tree launch");
}

template <int F>
static cudaError_t launch_tree_batch(const float2 *x, float2 *tree, double *xen, const TreeBatch &b, int maxJ,
                                     cudaStream_t s) {
    const LiftCoef c = lift_coef(F, SIDE_X);
    int active = b.n;
    for (int j = 0; j < maxJ; ++j) {
        while (active > 0 && b.it[active - 1].J <= j) --active;  // sorted by decreasing J
        const int64_t total = b.nprefix[active];
        if (total == 0) break;
        tree_level_batch_kernel<F><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(x, tree, b, j, active, c);
    }
    tree_energy_batch_kernel<<<(unsigned)b.eprefix[b.n], 256, 0, s>>>(x, tree, xen, b);
    return cudaGetLastError();
}

sidwt_status build_reference_trees(int filter, const float2 *x, float2 *tree, double *xen, const TreeItem *items,
                                   int n, cudaStream_t s, int *launches) {
    int nl = 0;
    for (int k0 = 0; k0 < n; k0 += kTreeBatch) {
        TreeBatch b;
        std::memset(&b, 0, sizeof(b));
        b.n = std::min(kTreeBatch, n - k0);
        for (int k = 0; k < b.n; ++k) b.it[k] = items[k0 + k];
        std::stable_sort(b.it, b.it + b.n, [](const TreeItem &a, const TreeItem &c) { return a.J > c.J; });
        for (int k = 0; k < b.n; ++k) {
            b.nprefix[k + 1] = b.nprefix[k] + b.it[k].N;
            b.eprefix[k + 1] = b.eprefix[k] + energy_blocks(b.it[k].N, b.it[k].J);
        }
        const int maxJ = b.it[0].J;
        if (b.eprefix[b.n] > 0x7fffffff || (b.nprefix[b.n] + 255) / 256 > 0x7fffffff) {
            set_error("tree batch too large for one launch");
            return SIDWT_EINVAL;
        }
        cudaError_t e;
        switch (filter) {
        case SIDWT_D4: e = launch_tree_batch<SIDWT_D4>(x, tree, xen, b, maxJ, s); break;
        case SIDWT_LEGALL53: e = launch_tree_batch<SIDWT_LEGALL53>(x, tree, xen, b, maxJ, s); break;
        case SIDWT_CDF97: e = launch_tree_batch<SIDWT_CDF97>(x, tree, xen, b, maxJ, s); break;
        default: set_error("batched trees take the float filters"); return SIDWT_EINVAL;
        }
        if (e != cudaSuccess) return cuda_fail(e, "batched reference trees");
        nl += maxJ + 1;
    }
    if (launches) *launches = nl;
    return SIDWT_OK;
}

template <int F, typename T>
static cudaError_t launch_smem(sidwt_plan *p, const void *y, int64_t B, cudaStream_t s, const LiftCoef &c) {
    const size_t smem = (size_t)(p->N + p->N / 2) * sizeof(T);
    analyze_smem_kernel<F, T><<<(unsigned)B, kAnalyzeThreads, smem, s>>>(y, p->N, p->J, p->pyr_f, p->pyr_i,
                                                                       p->pyr_elems, p->yen, c);
    return cudaGetLastError();
}

// Shared-memory budgets of the analysis kernels, set once per device (see
// prepare_kernels) so that no launch needs an attribute call.
cudaError_t prepare_analysis_kernels() {
    cudaError_t e = cudaFuncSetAttribute(analyze_smem_kernel<SIDWT_D4, float2>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(analyze_smem_kernel<SIDWT_LEGALL53, float2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(analyze_smem_kernel<SIDWT_CDF97, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(analyze_smem_kernel<SIDWT_LEGALL53_INT, int2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(analyze_pipe_kernel<SIDWT_D4, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kPipeSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(analyze_pipe_kernel<SIDWT_LEGALL53, float2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kPipeSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(analyze_pipe_kernel<SIDWT_CDF97, float2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kPipeSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(analyze_pipe_kernel<SIDWT_LEGALL53_INT, int2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kPipeSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(analyze_pipe_kernel<SIDWT_CDF97_INT, int2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kPipeSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(analyze_smem_kernel<SIDWT_CDF97_INT, int2>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e == cudaSuccess) e = prepare_ragged_kernels();
    return e;
}

int analyze_launch_count(const sidwt_plan *p) {
    const size_t smem = (size_t)(p->N + p->N / 2) * 8;
    return smem <= (size_t)kSmemLimit ? 1 : p->J + 1;
}

sidwt_status analyze_batch(sidwt_plan *p, const void *y_dev, int64_t B, cudaStream_t s) {
    if (B == 0) return SIDWT_OK;
    const int64_t N = p->N;
    const int J = p->J;
    const LiftCoef c = plan_coef(p, SIDE_Y);
    const size_t smem = (size_t)(N + N / 2) * 8;
    cudaError_t e = cudaSuccess;
    const size_t in_bytes = (size_t)N * (p->is_int ? 4 : 8);
    // two CTAs per SM with two input buffers each (prefetch within the CTA)
    // when they fit; else two CTAs with one buffer (each overlaps the other's
    // loads); else one CTA with two buffers
    const size_t inb = (in_bytes + 127) & ~(size_t)127;
    const size_t one_smem = inb + (size_t)(N / 2) * 8;
    const size_t two_smem = one_smem + inb;
    const size_t sm_bytes = 228 * 1024, per_cta = 9 * 1024;
    const int nbuf = 2 * (two_smem + per_cta) <= sm_bytes ? 2 : (2 * (one_smem + per_cta) <= sm_bytes ? 1 : 2);
    const size_t pipe_smem = nbuf * inb + (size_t)(N / 2) * 8;
    const uintptr_t yal = reinterpret_cast<uintptr_t>(y_dev);
    if (pipe_smem <= (size_t)kPipeSmemLimit && in_bytes % 16 == 0 && yal % 16 == 0 && J < kPipeMaxLevels) {
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int per_sm = std::max(1, std::min(2048 / kPipeThreads, (int)((size_t)(228 * 1024) / (pipe_smem + 9 * 1024))));
        const int64_t grid = std::min<int64_t>(B, (int64_t)sms * per_sm);
        const int stall = (debug_stall_flags() & SIDWT_STALL_ANALYSIS) ? 1 : 0;
        switch (p->filter) {
        case SIDWT_D4:
            analyze_pipe_kernel<SIDWT_D4, float2><<<(unsigned)grid, kPipeThreads, pipe_smem, s>>>(
                y_dev, N, J, B, p->pyr_f, p->pyr_i, p->pyr_elems, p->yen, c, p->err, nbuf, stall, nullptr);
            break;
        case SIDWT_LEGALL53:
            analyze_pipe_kernel<SIDWT_LEGALL53, float2><<<(unsigned)grid, kPipeThreads, pipe_smem, s>>>(
                y_dev, N, J, B, p->pyr_f, p->pyr_i, p->pyr_elems, p->yen, c, p->err, nbuf, stall, nullptr);
            break;
        case SIDWT_CDF97:
            analyze_pipe_kernel<SIDWT_CDF97, float2><<<(unsigned)grid, kPipeThreads, pipe_smem, s>>>(
                y_dev, N, J, B, p->pyr_f, p->pyr_i, p->pyr_elems, p->yen, c, p->err, nbuf, stall, nullptr);
            break;
        case SIDWT_CDF97_INT:
            analyze_pipe_kernel<SIDWT_CDF97_INT, int2><<<(unsigned)grid, kPipeThreads, pipe_smem, s>>>(
                y_dev, N, J, B, p->pyr_f, p->pyr_i, p->pyr_elems, p->yen, c, p->err, nbuf, stall, nullptr);
            break;
        default:
            analyze_pipe_kernel<SIDWT_LEGALL53_INT, int2><<<(unsigned)grid, kPipeThreads, pipe_smem, s>>>(
                y_dev, N, J, B, p->pyr_f, p->pyr_i, p->pyr_elems, p->yen, c, p->err, nbuf, stall, nullptr);
            break;
        }
        e = cudaGetLastError();
        return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "analysis launch");
    }
    if (smem <= (size_t)kSmemLimit && B <= 0x7fffffff) {
        switch (p->filter) {
        case SIDWT_D4: e = launch_smem<SIDWT_D4, float2>(p, y_dev, B, s, c); break;
        case SIDWT_LEGALL53: e = launch_smem<SIDWT_LEGALL53, float2>(p, y_dev, B, s, c); break;
        case SIDWT_CDF97: e = launch_smem<SIDWT_CDF97, float2>(p, y_dev, B, s, c); break;
        case SIDWT_CDF97_INT: e = launch_smem<SIDWT_CDF97_INT, int2>(p, y_dev, B, s, c); break;
        default: e = launch_smem<SIDWT_LEGALL53_INT, int2>(p, y_dev, B, s, c); break;
        }
        return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "analysis launch");
    }
    // long pulses: one launch per level through HBM
    for (int l = 1; l <= J; ++l) {
        const int64_t K = N >> (l - 1);
        const int64_t off = 2 * N - 4 * (N >> l);
        const int64_t prev = 2 * N - 4 * K;  // c_{l-1} offset (l >= 2)
        if (!p->is_int) {
            const float2 *in = (l == 1) ? reinterpret_cast<const float2 *>(y_dev) : p->pyr_f + prev;
            launch_level_any(p->filter, SIDE_Y, in, l == 1 ? N : p->pyr_elems, (int)B, 1, K, p->pyr_f + off,
                             p->pyr_f + off + (N >> l), p->pyr_elems, c, s);
        } else if (l == 1) {
            launch_level_int(p->filter, SIDE_Y, reinterpret_cast<const short2 *>(y_dev), N, (int)B, 1, K, p->pyr_i + off,
                             p->pyr_i + off + (N >> l), p->pyr_elems, p->pyr_f + off, p->pyr_f + off + (N >> l), s);
        } else {
            launch_level_int(p->filter, SIDE_Y, p->pyr_i + prev, p->pyr_elems, (int)B, 1, K, p->pyr_i + off,
                             p->pyr_i + off + (N >> l), p->pyr_elems, p->pyr_f + off, p->pyr_f + off + (N >> l), s);
        }
    }
    dim3 g((unsigned)B, (unsigned)(J + 1));
    pyr_energy_kernel<<<g, 256, 0, s>>>(p->is_int ? nullptr : reinterpret_cast<const float2 *>(y_dev), p->pyr_f,
                                        p->is_int ? p->pyr_i : nullptr,
                                        p->is_int ? reinterpret_cast<const short2 *>(y_dev) : nullptr, N, J,
                                        p->pyr_elems, p->yen);
    e = cudaGetLastError();
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "analysis (window path) launch");
}

// ---------------------------------------------------------------------------
// Ragged batches
// ---------------------------------------------------------------------------
// two input buffers of N complex64 and the level-1 buffer of N / 2
int64_t analyze_pipe_max_n() { return (int64_t)kPipeSmemLimit / 20 / 128 * 128; }
// up to 2048 samples four CTAs fit an SM, up to 5120 two
int64_t analyze_pipe_class_max(int k) { return k == 0 ? 2048 : (k == 1 ? 5120 : analyze_pipe_max_n()); }

// Per-level window lifting of long pulses: block (x, item) computes outputs
// x*128.. of item's level l from its level l-1 approximation (y at l = 1).
template <int F>
__global__ void ragged_level_kernel(const float2 *__restrict__ y, const RaggedLift *__restrict__ items,
                                    float2 *__restrict__ pyr, int l, LiftCoef c) {
    const RaggedLift it = items[blockIdx.y];
    if (l > it.J) return;
    const int64_t N = it.N;
    const int64_t K = N >> (l - 1), H = K / 2;
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= H) return;
    const float2 *v = (l == 1) ? y + it.y_off : pyr + it.pyr_off + (2 * N - 4 * K);
    using Sh = LiftShape<F, SIDE_Y>;
    float2 E[2 * WR + 1], O[2 * WR + 1];
#pragma unroll
    for (int i = 0; i <= 2 * WR; ++i) {
        const int64_t m = n - WR + i;
        E[i] = v[wrapi(2 * m, K)];
        O[i] = v[wrapi(Sh::d4 ? 2 * m - 1 : 2 * m + 1, K)];
    }
    lift_window<F, SIDE_Y, WR>(E, O, c);
    const float2 lo = scale2(c.ce, E[WR]);
    float2 hi;
    if (Sh::d4) hi = scale2(c.co, make_float2(E[WR].x + O[WR - 1].x, E[WR].y + O[WR - 1].y));
    else hi = scale2(c.co, O[WR]);
    float2 *o = pyr + it.pyr_off + (2 * N - 4 * H);
    o[n] = lo;
    o[H + n] = hi;
}

// Energies of long ragged pulses: block (level l, item).
__global__ void ragged_energy_kernel(const float2 *__restrict__ y, const RaggedLift *__restrict__ items,
                                     const float2 *__restrict__ pyr, double *__restrict__ yen) {
    __shared__ float2 red[32];
    const RaggedLift it = items[blockIdx.y];
    const int l = blockIdx.x;
    if (l > it.J) return;
    const int64_t K = it.N >> l;
    const float2 *v = l == 0 ? y + it.y_off : pyr + it.pyr_off + (2 * it.N - 4 * K);
    EnAcc acc;
    for (int64_t k = threadIdx.x; k < K; k += blockDim.x) acc.add(sq2(v[k]));
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) yen[it.yen_off + l] = t;
}


// Long pulses of a ragged batch, in tiles of kTileSamples samples.  A
// persistent CTA walks the tiles b, b + G, ...: while the levels of one tile
// run, bulk copies (cp.async.bulk) bring the next tile's samples and a
// periodic halo of kTileHalo on each side into the other of two input
// buffers, so the HBM reads stay in flight across the kernel.  Levels 1..L
// run in shared memory: each level's valid range shrinks by the windows'
// reach, and the halo keeps the tile's own range valid down to level 5.
// Each level writes the tile's own part to the pyramid.  Output pair n of a level
// reads the input pairs n - 3 .. n + 2; the level's buffer holds pairs
// [p0, p1) and the outputs are [n0, n1) = [p0 + 3, p1 - 3) rounded inwards to
// even n.  Level 1 writes the work buffer W, level 2 the current input buffer
// (free once level 1 has read it), and so on alternately.  Energies: a plain
// FP32 partial per thread (a few terms) summed per warp for each level, and
// the warps' sums added (compensated) once per tile into the tile's partials.
constexpr int kTileThreads = 512;
constexpr int kTileIn = kTileSamples + 2 * kTileHalo;     // samples of one input buffer
constexpr int kTileSmem = (2 * kTileIn + kTileIn / 2) * 8;  // two input buffers and W

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Samples [s0, s0 + cnt) of the periodic pulse (N samples) into dst.  N > cnt,
// so the range wraps once at most: one or two copies.  s0, N and cnt are even
// and the pulse starts 16-byte aligned, so every copy starts on a 16-byte
// boundary and moves a multiple of 16 bytes.
__device__ __forceinline__ void tile_load(float2 *dst, const float2 *pulse, int64_t N, int64_t s0, int cnt,
                                          uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"((uint32_t)cnt * 8u)
                 : "memory");
    const int64_t a = s0 < 0 ? s0 + N : s0;
    const int first = N - a < cnt ? (int)(N - a) : cnt;  // samples before the wrap
    bulk_copy_g2s(dst, pulse + a, (uint32_t)first * 8u, bar);
    if (first < cnt) bulk_copy_g2s(dst + first, pulse, (uint32_t)(cnt - first) * 8u, bar);
}

template <int F>
__global__ void __launch_bounds__(kTileThreads, 2) ragged_tile_kernel(const float2 *__restrict__ y,
                                                                   const RaggedTile *__restrict__ tiles, int ntiles,
                                                                   float2 *__restrict__ pyr, double *__restrict__ part,
                                                                   LiftCoef c, int32_t *__restrict__ err, int stall) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float redf[kTileLevels + 1][kTileThreads / 32];
    __shared__ int sfail;
    constexpr bool D4 = (F == SIDWT_D4);
    float2 *const buf0 = reinterpret_cast<float2 *>(smraw), *const buf1 = buf0 + kTileIn, *const W = buf1 + kTileIn;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x;
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sfail = 0;
    }
    __syncthreads();
    // stall (test hook, sidwt_debug_stall): no copy is issued, so the first
    // wait runs out and the CTA records the timeout with nothing in flight
    auto load = [&](int b, float2 *dst, uint64_t *br) {
        const RaggedTile w = tiles[b];
        tile_load(dst, y + w.y_off, w.N, (int64_t)w.t0 - kTileHalo, w.Tc + 2 * kTileHalo, br);
    };
    if (tid == 0 && !stall) load(blockIdx.x, buf0, &bar[0]);  // the grid has at most ntiles CTAs
    int issued = stall ? 0 : 1, landed = 0;  // copies issued / waited for (thread 0's bookkeeping)
    int i = 0;
    for (int b = blockIdx.x; b < ntiles; b += G, ++i) {
        const int s = i & 1;
        float2 *const cur = s ? buf1 : buf0;
        if (tid == 0 && !stall && b + G < ntiles) {
            // the other buffer held tile i - 1, whose accesses ended at its last barrier
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            load(b + G, s ? buf0 : buf1, &bar[s ^ 1]);
            ++issued;
        }
        if (!pipe_wait(&bar[s], (uint32_t)((i >> 1) & 1))) sfail = 1;
        __syncthreads();
        if (sfail) break;
        if (tid == 0) ++landed;
        const RaggedTile t = tiles[b];
        const int64_t N = t.N;
        float2 *in = cur, *out = W;
        int64_t s0 = (int64_t)t.t0 - kTileHalo;  // first sample of the level held in `in`
        int cnt = t.Tc + 2 * kTileHalo;
        for (int l = 1; l <= t.L; ++l) {
            const int64_t p0 = s0 / 2, p1 = (s0 + cnt) / 2;
            int64_t n0 = p0 + 3, n1 = p1 - 3;
            n0 += n0 & 1;
            n1 -= n1 & 1;
            const int64_t K = N >> l, core0 = (int64_t)t.t0 >> l;
            // outputs are indexed from n0 in 32 bits (a tile level holds at most kTileIn samples)
            const int m_end = (int)(n1 - n0), kofs = (int)(n0 - p0);
            const int c0 = (int)(core0 - n0), c1 = c0 + (t.Tc >> l);
            float2 *pl = pyr + t.pyr_off + 2 * N - 4 * K + n0, *ph = pl + K;
            const float4 *q = reinterpret_cast<const float4 *>(in) + kofs;
            // e0: the energy of the tile's own samples (level 0), from level 1's
            // windows: the centre pair of output m is the input pair n0 + m, so
            // the core outputs' centres are exactly the tile's own pairs
            float e = 0.f, e0 = 0.f;
            for (int m = tid; m < m_end; m += kTileThreads) {
                float2 E[5], O[5];
                float4 prev = D4 ? q[m - 3] : make_float4(0.f, 0.f, 0.f, 0.f), ctr;
#pragma unroll
                for (int k = 0; k < 5; ++k) {
                    const float4 cv = q[m - 2 + k];
                    E[k] = make_float2(cv.x, cv.y);
                    O[k] = D4 ? make_float2(prev.z, prev.w) : make_float2(cv.z, cv.w);  // D4 odd phase: v[2m-1]
                    prev = cv;
                    if (k == 2) ctr = cv;
                }
                lift_window<F, SIDE_Y, 2>(E, O, c);
                const float2 lo = scale2(c.ce, E[2]);
                const float2 hi = D4 ? scale2(c.co, make_float2(E[2].x + O[1].x, E[2].y + O[1].y)) : scale2(c.co, O[2]);
                out[m] = lo;
                if (m >= c0 && m < c1) {
                    pl[m] = lo;
                    ph[m] = hi;
                    e = fmaf(lo.x, lo.x, fmaf(lo.y, lo.y, e));
                    if (l == 1) e0 = fmaf(ctr.x, ctr.x, fmaf(ctr.y, ctr.y, fmaf(ctr.z, ctr.z, fmaf(ctr.w, ctr.w, e0))));
                }
            }
            for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
            if (lane == 0) redf[l][warp] = e;
            if (l == 1) {
                for (int o = 16; o > 0; o >>= 1) e0 += __shfl_xor_sync(0xffffffffu, e0, o);
                if (lane == 0) redf[0][warp] = e0;
            }
            float2 *tmp = in;
            in = out;
            out = tmp;
            s0 = n0;
            cnt = m_end;
            __syncthreads();  // this level's reads of `in` end before the next level overwrites it
        }
        if (tid <= t.L) {
            EnAcc a;
            for (int w = 0; w < kTileThreads / 32; ++w) a.add(redf[tid][w]);
            part[t.part_off + tid] = a.total();
        }
        // the next iteration's wait and barrier order these reads of redf
        // before its level-0 writes
    }
    if (tid == 0 && sfail) {
        // let this CTA's own copies land before its shared memory is released
        for (int k = landed; k < issued; ++k) pipe_wait(&bar[k & 1], (uint32_t)((k >> 1) & 1));
        atomicOr(err, kErrAnalysisWait);
    }
}

// The tails of the tiled pulses: the energies of levels 0..L from the tiles'
// partials (summed in tile order), then levels L + 1..J from c_L in shared
// memory (the pyramid and energy pointers shifted so that its level l lands
// at level L + l).
template <int F>
__global__ void __launch_bounds__(kAnalyzeThreads) ragged_tail_kernel(const RaggedTail *__restrict__ tails,
                                                                      const double *__restrict__ part,
                                                                      float2 *__restrict__ pyr,
                                                                      double *__restrict__ yen, LiftCoef c) {
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ float2 red[32];
    __shared__ long long redi[32];
    const RaggedTail tl = tails[blockIdx.x];
    const int L = tl.L, J = tl.it.J;
    const int last = J > L ? L - 1 : L;  // level L's energy comes from the lifting below when it goes on
    if ((int)threadIdx.x <= last) {
        double e = 0.0;
        for (int k = 0; k < tl.ntiles; ++k) e += part[tl.part_off + (int64_t)k * (kTileLevels + 1) + threadIdx.x];
        yen[tl.it.yen_off + threadIdx.x] = e;
    }
    if (J > L) {
        const int64_t N = tl.it.N, N2 = N >> L;
        float2 *base = pyr + tl.it.pyr_off;
        analyze_one<F, float2>(base + 2 * N - 4 * N2, N2, J - L, base + 2 * N - 2 * N2, nullptr,
                               yen + tl.it.yen_off + L, c, reinterpret_cast<float2 *>(smraw), red, redi);
    }
}

template <int F>
static cudaError_t launch_ragged_tiles(const RaggedTile *tiles, int ntiles, const RaggedTail *tails, int ntails,
                                       int64_t maxN2, const float2 *y, float2 *pyr, double *yen, double *part,
                                       int32_t *err, cudaStream_t s) {
    const LiftCoef c = lift_coef(F, SIDE_Y);
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::min(ntiles, 2 * sms);  // persistent: two CTAs per SM
    const int stall = (debug_stall_flags() & SIDWT_STALL_ANALYSIS) ? 1 : 0;
    ragged_tile_kernel<F><<<grid, kTileThreads, kTileSmem, s>>>(y, tiles, ntiles, pyr, part, c, err, stall);
    ragged_tail_kernel<F><<<ntails, kAnalyzeThreads, (size_t)(maxN2 + maxN2 / 2) * 8, s>>>(tails, part, pyr, yen, c);
    return cudaGetLastError();
}

int64_t tile_tail_max_n() { return (int64_t)kSmemLimit / 12; }

// The ragged kernels get the whole shared-memory budget once, outside any
// stream capture, so that launching them needs no attribute call.
cudaError_t prepare_ragged_kernels() {
    cudaError_t e = cudaFuncSetAttribute(ragged_tile_kernel<SIDWT_D4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ragged_tile_kernel<SIDWT_LEGALL53>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ragged_tile_kernel<SIDWT_CDF97>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ragged_tail_kernel<SIDWT_D4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ragged_tail_kernel<SIDWT_LEGALL53>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ragged_tail_kernel<SIDWT_CDF97>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(analyze_pipe_kernel<SIDWT_D4, float2, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kPipeSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(analyze_pipe_kernel<SIDWT_LEGALL53, float2, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kPipeSmemLimit);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(analyze_pipe_kernel<SIDWT_CDF97, float2, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kPipeSmemLimit);
    return e;
}

// Pulses of a ragged batch whose double buffer fits: the pipelined kernel
// over the item list (persistent CTAs, the next pulse bulk-copied while the
// current one lifts), its shared buffers sized for the longest of them.
template <int F>
static cudaError_t launch_ragged_pipe(const float2 *y, const RaggedLift *items, int n, int64_t maxN, float2 *pyr,
                                      double *yen, int32_t *err, cudaStream_t s) {
    const size_t inb = ((size_t)maxN * 8 + 127) & ~(size_t)127;
    const size_t smem = 2 * inb + (size_t)(maxN / 2) * 8;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = std::max(1, std::min(2048 / kPipeThreads, (int)((size_t)(228 * 1024) / (smem + 9 * 1024))));
    const int grid = (int)std::min<int64_t>(n, (int64_t)sms * per_sm);
    const int stall = (debug_stall_flags() & SIDWT_STALL_ANALYSIS) ? 1 : 0;
    analyze_pipe_kernel<F, float2, true><<<grid, kPipeThreads, smem, s>>>(
        y, maxN, 15, n, pyr, nullptr, 0, yen, lift_coef(F, SIDE_Y), err, 2, stall, items);
    return cudaGetLastError();
}

template <int F>
static cudaError_t launch_ragged_window(const float2 *y, const RaggedLift *items, int n, int64_t maxN, int maxJ,
                                        float2 *pyr, double *yen, cudaStream_t s) {
    const LiftCoef c = lift_coef(F, SIDE_Y);
    for (int l = 1; l <= maxJ; ++l) {
        const int64_t H = maxN >> l;
        dim3 g((unsigned)((H + 127) / 128), (unsigned)n);
        ragged_level_kernel<F><<<g, 128, 0, s>>>(y, items, pyr, l, c);
    }
    dim3 g((unsigned)(maxJ + 1), (unsigned)n);
    ragged_energy_kernel<<<g, 256, 0, s>>>(y, items, pyr, yen);
    return cudaGetLastError();
}

// The received analysis of a ragged batch, by filter: pulses up to
// analyze_pipe_max_n() on the pipelined kernel (one launch per size class),
// longer ones in tiles plus a tail per pulse, and pulses too long for a
// tail's shared memory (N >> 5 above tile_tail_max_n(), J > 5) one launch per
// level (window path).
sidwt_status analyze_ragged(const float2 *y, const RaggedLiftGroups &g, float2 *pyr, double *yen, double *part,
                            int32_t *err, cudaStream_t s, int *launches) {
    cudaError_t e = cudaSuccess;
    int nl = 0;
    for (int f = 0; f < 3 && e == cudaSuccess; ++f) {
        if (g.n_tiles[f] > 0) {
            switch (f) {
            case SIDWT_D4:
                e = launch_ragged_tiles<SIDWT_D4>(g.tiles[f], g.n_tiles[f], g.tails[f], g.n_tails[f], g.maxN_tail[f], y,
                                                  pyr, yen, part, err, s);
                break;
            case SIDWT_LEGALL53:
                e = launch_ragged_tiles<SIDWT_LEGALL53>(g.tiles[f], g.n_tiles[f], g.tails[f], g.n_tails[f],
                                                        g.maxN_tail[f], y, pyr, yen, part, err, s);
                break;
            default:
                e = launch_ragged_tiles<SIDWT_CDF97>(g.tiles[f], g.n_tiles[f], g.tails[f], g.n_tails[f], g.maxN_tail[f],
                                                     y, pyr, yen, part, err, s);
            }
            nl += 2;
        }
        for (int k = 0; k < kPipeClasses && e == cudaSuccess; ++k) {
            if (g.n_pipe[k][f] == 0) continue;
            const RaggedLift *it = g.pipe[k][f];
            const int n = g.n_pipe[k][f];
            const int64_t mx = g.maxN_pipe[k][f];
            switch (f) {
            case SIDWT_D4: e = launch_ragged_pipe<SIDWT_D4>(y, it, n, mx, pyr, yen, err, s); break;
            case SIDWT_LEGALL53: e = launch_ragged_pipe<SIDWT_LEGALL53>(y, it, n, mx, pyr, yen, err, s); break;
            default: e = launch_ragged_pipe<SIDWT_CDF97>(y, it, n, mx, pyr, yen, err, s);
            }
            ++nl;
        }
        if (e == cudaSuccess && g.n_long[f] > 0) {
            switch (f) {
            case SIDWT_D4:
                e = launch_ragged_window<SIDWT_D4>(y, g.lng[f], g.n_long[f], g.maxN_long[f], g.maxJ_long[f], pyr, yen, s);
                break;
            case SIDWT_LEGALL53:
                e = launch_ragged_window<SIDWT_LEGALL53>(y, g.lng[f], g.n_long[f], g.maxN_long[f], g.maxJ_long[f], pyr,
                                                         yen, s);
                break;
            default:
                e = launch_ragged_window<SIDWT_CDF97>(y, g.lng[f], g.n_long[f], g.maxN_long[f], g.maxJ_long[f], pyr,
                                                      yen, s);
            }
            nl += g.maxJ_long[f] + 1;
        }
    }
    if (launches) *launches = nl;
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "ragged analysis launch");
}

}  // namespace sidwt
