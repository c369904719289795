// Batch-of-one correlation on the tcgen05 tensor cores (bf16 hi+lo split,
// three products, FP32 accumulation in TMEM) for ragged batches and the
// serving loop, where every received pulse has its own stored signal.
//
// With one received band u per stored signal the product of eq. 20 / 20a is
// a matrix-vector product per variant, R_v[p] = sum_k conj(w_v[(k+p) mod K'])
// u[k].  It becomes a GEMM by moving part of the advance p into the rows:
// with p = S i - n (0 <= n < S) and k -> k + n,
//     R_v[S i - n] = sum_k conj(w_v[k + S i]) u[k + n],
// so row (v, i) of the stored operand is variant v advanced by S i, column n
// of the received operand is u advanced by n, and every row shares the one
// received operand.  The rows of all 2^lev variants (ceil(K'/S) each, padded
// to groups of 8) fill the 128-row tiles; a tile has S columns.
//
// Both operands are windows, never materialised as matrices:
//   * stored rows: for each residue c of k mod 8 the polyphase sequence
//     P_c[s] = w[(k0 + c + 8 s) mod K'] is cut into rows of S/8 samples, so
//     that row r of a K-block starting at sample 8 kb is row i + (8 kb)/(S/8)
//     of that reshaped array.  The packed operand keeps, for every reshaped
//     row and block of 8 samples, its 16 chunks (residue x Re/Im) of 8
//     samples together (256 bytes), so that two 5-D TMA boxes {64 elements,
//     1 block, 8 rows, hi+lo, 1} per 8-row group move whole 128-byte rows
//     into the K-major A tile, in the 128-byte swizzled layout
//     [chunk half][group][hi/lo][8 rows][128 B] (4 KB per group: 512
//     copy rows per K-block where 16-byte rows took 4096, a quarter of the
//     L2 throughput);
//   * received columns: the overlapping MN-major window of the batched kernel
//     (8 shifted copies U_c[t] = u[t + c + k0], planes Re, Im, -Re), built
//     in shared memory for each K-block by four expansion warps straight from
//     the received pyramid (no packed copy in HBM: the copies and planes are
//     12x the band's bytes).
// Band lengths that are a multiple of 64 use the circular form (k0 = 0, the
// received copies wrap).  Other lengths use the equivalent linear form: the
// received band is zero outside [0, K'), the contraction runs over
// k in [-S, ceil(K'/64) 64), and the stored rows stay periodic.
//
// Persistent grid, one CTA per SM, tiles in cost order strided over the
// CTAs.  Roles (320 threads): warp 0 TMA producer of the stored operand
// (2-stage ring), warp 1 TMEM allocation and MMA issue, warps 2-5 epilogue
// (peak keys), warps 6-9 received-window expansion into the same ring (a
// stage is full once its copies have landed and the four warps have
// arrived).  The producer and the expansion warps run ahead into the next
// tile; the MMA warp starts a tile once the epilogue has drained the
// accumulators.  Scale J has no tiles of its own: its product (eq. 20a) is
// band 0 of scale J - 1's (eq. 20) at the same level, so a scale J - 1 tile
// with a slot_mid hands its accumulators to the epilogue after band 0 (peak
// of scale J) and adds band 1 once they have been read.  Every wait is
// bounded.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "tc_common.cuh"

namespace sidwt {
namespace rtc {

using namespace sidwt::tc;

constexpr int kThreads = 320;
constexpr int kGroupBytes = 4096;             // per 8-row group: 2 chunk halves x hi/lo x 8 rows x 128 B
constexpr int kStageA = 16 * kGroupBytes;     // 65536
constexpr int kHalfBytes = kStageA / 2;       // chunks 0-7 (residues 0-3), then 8-15: [group][hi/lo][8][128 B]
static_assert(kHalfBytes % 1024 == 0, "128-byte swizzle atoms on 1 KB boundaries");
constexpr int kMaxBRow = (256 + 64) * 2;      // 640 bytes per window row at S = 256
constexpr int kStageB = 2 * 24 * kMaxBRow;    // 30720
constexpr int kBRegion = 2 * kStageB;
constexpr int kARegion = 2 * kStageA;
constexpr int kBarOff = kBRegion + kARegion;  // 192512
static_assert(kBRegion % 1024 == 0, "the stored-operand ring starts on a 1 KB boundary");
// what the kernel uses (rings, barriers, 1 KB alignment slack), so that a
// CUDA-core CTA of the ragged kernel (about 20 KB) fits beside it on an SM
constexpr int kSmemBytes = kBarOff + 128 + 1024;
constexpr int kTmemCols = 512;
constexpr int64_t kMinBand = 64;              // shorter bands stay on the CUDA cores
constexpr int64_t kMaxBand = int64_t(1) << 24;

__device__ __forceinline__ void tma_load_5d(void *dst, const void *map, uint64_t *bar, int c0, int c1, int c2, int c3,
                                            int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(saddr(bar))
        : "memory");
}

// The tensor maps live in global memory and are rewritten between batches
// by copies from the host: order those writes before the TMA unit reads the
// descriptors (tensor-map proxy acquire).
__device__ __forceinline__ void tensormap_acquire(const void *map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
                 : "memory");
}

// Wait on a phase that completes only after a whole tile's main loop: the
// limit counts from the last K-block the MMA thread issued (*progress), so
// that long tiles (and slowed-down runs under a profiler) do not trip it.
__device__ __forceinline__ bool mbar_wait_progress(uint64_t *b, uint32_t parity, volatile int *progress) {
    uint64_t t0 = now_ns();
    int last = *progress;
    while (!mbar_test(b, parity)) {
        const int p = *progress;
        if (p != last) {
            last = p;
            t0 = now_ns();
        } else if (now_ns() - t0 > kWaitNs) {
            return false;
        }
    }
    return true;
}

// Number of 8-row groups of tile t that hold rows of an existing variant.
__device__ __forceinline__ int valid_groups(const TcTile &w) {
    const int g0 = 16 * w.tile, total = w.nv * w.gv;
    return max(0, min(16, total - g0));
}

// The received operand of one K-block: for the 8 residues c the window
// U_c[64 kb + t] = u[64 kb + t + c + k0], t < S + 64 (wrapped mod K' in the
// circular form, zero outside [0, K') in the padded one), as bf16 hi and lo
// of the planes Re, Im, -Re: rows (hi/lo) * 24 + 3 c + plane of S + 64
// samples.  Written by the four expansion warps straight from the received
// pyramid (8 samples and 16-byte stores per work item).
__device__ __forceinline__ void expand_window(unsigned char *stB, const float2 *__restrict__ u, int Kp, int k0, int S,
                                              int kb, int tw, int nthreads) {
    const int rowlen = S + 64, ngrp = rowlen >> 3;
    const uint32_t bRow = (uint32_t)rowlen * 2;
    for (int item = tw; item < 8 * ngrp; item += nthreads) {
        const int c = item / ngrp, g = item - c * ngrp;
        int idx = 64 * kb + 8 * g + c + k0;
        if (k0 == 0) idx %= Kp;
        __align__(16) __nv_bfloat16 h[3][8], l[3][8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            float2 x = make_float2(0.f, 0.f);
            if (k0 == 0) {
                x = u[idx];
                idx = idx + 1 == Kp ? 0 : idx + 1;
            } else {
                if (idx >= 0 && idx < Kp) x = u[idx];
                ++idx;
            }
            split_bf16(x.x, h[0][q], l[0][q]);
            split_bf16(x.y, h[1][q], l[1][q]);
            split_bf16(-x.x, h[2][q], l[2][q]);
        }
#pragma unroll
        for (int pl = 0; pl < 3; ++pl) {
            const uint32_t off = (uint32_t)(3 * c + pl) * bRow + 16u * (uint32_t)g;
            *reinterpret_cast<uint4 *>(stB + off) = *reinterpret_cast<const uint4 *>(h[pl]);
            *reinterpret_cast<uint4 *>(stB + 24 * bRow + off) = *reinterpret_cast<const uint4 *>(l[pl]);
        }
    }
}

// The (band b, K-block kb) steps of a work item: all nb x nkb of a whole tile,
// or, for one part of a split contraction, the contiguous run f0 .. f0 + fcnt - 1
// of f = nkb b + kb.  Bands b0 .. b1; band b0 starts at kb0, band b1 ends
// before kb1.
struct StepRange {
    int b0, b1, kb0, kb1;
    __device__ __forceinline__ int kb_begin(int b) const { return b == b0 ? kb0 : 0; }
    __device__ __forceinline__ int kb_end(int b, int nkb) const { return b == b1 ? kb1 : nkb; }
};

template <bool PARTS>
__device__ __forceinline__ StepRange step_range(const TcTile &w) {
    if (!PARTS || w.fcnt < 0) return {0, w.nb - 1, 0, w.nkb};
    const int fe = w.f0 + w.fcnt, b1 = (fe - 1) / w.nkb, b0 = w.f0 / w.nkb;
    return {b0, b1, w.f0 - b0 * w.nkb, fe - b1 * w.nkb};
}

// WITH_R: also write r at every lag; PARTS: some work items are parts of a
// split contraction (separate instances, so that the bulk path's epilogue is
// unchanged)
template <bool WITH_R, bool PARTS>
__global__ void __launch_bounds__(kThreads, 1)
    corr_pair_tc_kernel(const CUtensorMap *__restrict__ maps, const TcTile *__restrict__ tiles, int ntiles,
                        const float2 *__restrict__ pyr, unsigned long long *__restrict__ keys,
                        int32_t *__restrict__ err, float2 *__restrict__ R, float2 *__restrict__ part) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *sB = base;
    unsigned char *sA = base + kBRegion;
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + kBarOff);
    uint64_t *full = bar, *empty = bar + 2, *accf = bar + 4, *tfree = bar + 5, *drain = bar + 6;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 8);
    // [0] error, [1] stages issued, [2] stages consumed, [3] K-blocks issued to the tensor cores so far
    volatile int *sflag = reinterpret_cast<volatile int *>(tmem_slot + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if ((int)blockIdx.x >= ntiles) return;  // uniform: before any barrier or TMEM use

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&full[i], 1 + 4);  // the producer's expect_tx and one arrival per expansion warp
            mbar_init(&empty[i], 1);
        }
        mbar_init(accf, 1);
        mbar_init(tfree, 128);
        mbar_init(drain, 1);
        sflag[0] = 0;
        sflag[1] = 0;
        sflag[2] = 0;
        sflag[3] = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int it = 0;
            for (int t = blockIdx.x; t < ntiles && !sflag[0]; t += gridDim.x) {
                const TcTile w = tiles[t];
                const CUtensorMap *mA = maps + 2 * (int64_t)w.map;
                const int Lr = w.S >> 3;
                const int ng = valid_groups(w);
                tensormap_acquire(mA);
                const uint32_t tx = (uint32_t)(ng * kGroupBytes);
                const StepRange sr = step_range<PARTS>(w);
                for (int b = sr.b0; b <= sr.b1 && !sflag[0]; ++b)
                    for (int kb = sr.kb_begin(b); kb < sr.kb_end(b, w.nkb); ++kb) {
                        const int s = it & 1;
                        if (it >= 2 && !mbar_wait(&empty[s], ((it >> 1) - 1) & 1)) {
                            sflag[0] = 1;
                            break;
                        }
                        if (sflag[0]) break;
                        mbar_expect_tx(&full[s], tx);
                        unsigned char *stA = sA + s * kStageA;
                        const int col = (8 * kb) % Lr, rsh = (8 * kb) / Lr;
                        for (int g = 0; g < ng; ++g) {
                            const int G = 16 * w.tile + g;
                            const int v = G / w.gv, i0 = 8 * (G % w.gv);
                            // chunk halves h: elements 64 h .. 64 h + 63 of the (row, block) record
                            for (int h = 0; h < 2; ++h)
                                tma_load_5d(stA + h * kHalfBytes + g * 2048, mA, &full[s], 64 * h, col >> 3, i0 + rsh,
                                            0, b * w.nv + v);
                        }
                        ++it;
                    }
            }
            sflag[1] = it;
        }
    } else if (warp >= 6) {
        // expansion warps: the received windows of the same K-blocks, in the same order
        const int tw = threadIdx.x - 6 * 32;
        int it = 0;
        for (int t = blockIdx.x; t < ntiles && !sflag[0]; t += gridDim.x) {
            const TcTile w = tiles[t];
            const StepRange sr = step_range<PARTS>(w);
            for (int b = sr.b0; b <= sr.b1 && !sflag[0]; ++b)
                for (int kb = sr.kb_begin(b); kb < sr.kb_end(b, w.nkb); ++kb) {
                    const int s = it & 1;
                    if (it >= 2 && !mbar_wait(&empty[s], ((it >> 1) - 1) & 1)) {
                        sflag[0] = 1;
                        break;
                    }
                    if (sflag[0]) break;
                    expand_window(sB + s * kStageB, pyr + w.u_off + (int64_t)b * w.Kp, w.Kp, w.k0, w.S, kb, tw, 128);
                    // the tensor cores read these stores through the async proxy
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&full[s]);
                    ++it;
                }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0, ec = 0;  // ec: accumulator hand-overs to the epilogue so far
            for (int t = blockIdx.x; t < ntiles && !sflag[0]; t += gridDim.x) {
                const TcTile w = tiles[t];
                if (ec > 0) {
                    if (!mbar_wait(tfree, (ec - 1) & 1)) {
                        sflag[0] = 1;
                        break;
                    }
                    tc_fence_after();
                }
                const uint32_t idesc = idesc_bf16(128, w.S);
                const uint32_t bRow = (uint32_t)(w.S + 64) * 2;
                bool first = true;
                const StepRange sr = step_range<PARTS>(w);
                for (int b = sr.b0; b <= sr.b1 && !sflag[0]; ++b) {
                    if (b == 1 && b > sr.b0 && w.slot_mid >= 0) {
                        // band 0 alone is the coarser scale's product: hand it to the
                        // epilogue and add band 1 once the epilogue has read it
                        mma_commit(accf);
                        ++ec;
                        if (!mbar_wait(tfree, (ec - 1) & 1)) {
                            sflag[0] = 1;
                            break;
                        }
                        tc_fence_after();
                    }
                    for (int kb = sr.kb_begin(b); kb < sr.kb_end(b, w.nkb); ++kb) {
                        const int s = it & 1;
                        if (!mbar_wait(&full[s], (it >> 1) & 1)) {
                            sflag[0] = 1;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t aHi = saddr(sA + s * kStageA), aLo = aHi + 1024;
                        const uint32_t bHi = saddr(sB + s * kStageB), bLo = bHi + 24 * bRow;
#pragma unroll 1
                        for (int c = 0; c < 8; ++c) {
                            // A: chunks (c, Re), (c, Im) are the 32 bytes at 32 (c % 4) of the 128-byte
                            // rows of chunk half c / 4; 8-row atoms 2 KB apart (hi and lo interleaved)
                            const uint32_t ao = (uint32_t)(c >> 2) * kHalfBytes + (uint32_t)(c & 3) * 32u;
                            const uint64_t ah = sdesc_sw128(aHi + ao, 2048);
                            const uint64_t al = sdesc_sw128(aLo + ao, 2048);
#pragma unroll
                            for (int acc = 0; acc < 2; ++acc) {
                                // window rows c*3 + {0: Re u, 1: Im u, 2: -Re u}; Re uses (Re u, Im u),
                                // Im uses (Im u, -Re u): next plane one row (bRow) further along K
                                const uint32_t row = c * 3 + acc;
                                const uint64_t bh = sdesc(bHi + row * bRow, bRow, 16);
                                const uint64_t bl = sdesc(bLo + row * bRow, bRow, 16);
                                const uint32_t d = tmem + acc * 256;
                                mma_bf16(d, ah, bh, idesc, first ? 0u : 1u);
                                mma_bf16(d, ah, bl, idesc, 1u);
                                mma_bf16(d, al, bh, idesc, 1u);
                            }
                            first = false;
                        }
                        mma_commit(&empty[s]);
                        ++it;
                        sflag[3] = it;
                    }
                }
                if (sflag[0]) break;
                mma_commit(accf);  // arrives once every MMA of this tile has completed
                ++ec;
            }
            sflag[2] = it;
            mma_commit(drain);  // every MMA issued by this CTA has completed
            if (!mbar_wait(drain, 0)) sflag[0] = 1;
        }
    } else if (warp >= 2 && warp < 6) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = tile rows
        const int q4 = warp & 3;
        const int m = q4 * 32 + lane;
        int ec = 0;  // accumulator hand-overs read so far
        bool stop = false;
        for (int t = blockIdx.x; t < ntiles && !stop; t += gridDim.x)
          for (int pass = tiles[t].slot_mid >= 0 ? 0 : 1; pass < 2; ++pass, ++ec) {
            // pass 0: band 0 alone (peak of slot_mid); pass 1: the whole product (slot)
            const TcTile w = tiles[t];
            const bool ok = mbar_wait_progress(accf, ec & 1, &sflag[3]);
            tc_fence_after();
            if (!__all_sync(0xffffffffu, ok && !sflag[0])) {  // warp-uniform before the aligned TMEM loads
                sflag[0] = 1;
                stop = true;
                break;
            }
            const int G = 16 * w.tile + (m >> 3);
            const int v = G / w.gv;
            const int i = 8 * (G % w.gv) + (m & 7);
            const bool valid = v < w.nv;
            const int Kp = w.Kp;
            // advance of column n: p = S i - n (mod K'); delay q = -p mod K'
            int pm = (int)(((int64_t)w.S * i) % Kp);
            unsigned long long best = 0ull;
            // optional r output (every (row, column) is a correct advance; rows past
            // ceil(K'/S) and the wrapped columns repeat advances already written)
            float2 *Rrow = (WITH_R && valid) ? R + (pass ? w.r_at : w.r_mid) : nullptr;
            const uint32_t tl = tmem + ((uint32_t)(q4 * 32) << 16);
            if (PARTS && w.part_off >= 0) {
                // one part of a split contraction: the raw accumulators, column-major
                // [S][128], for tc_split_reduce (which forms the peaks)
                float2 *P = part + w.part_off + m;
                for (int c0 = 0; c0 < w.S; c0 += 32) {
                    uint32_t re[32], im[32];
                    TMEM_LD32(tl + c0, re);
                    TMEM_LD32(tl + 256 + c0, im);
                    tmem_wait_ld();
#pragma unroll
                    for (int n = 0; n < 32; ++n)
                        P[(int64_t)(c0 + n) * 128] = make_float2(__uint_as_float(re[n]), __uint_as_float(im[n]));
                }
                tc_fence_before();
                mbar_arrive(tfree);
                continue;
            }
            for (int c0 = 0; c0 < w.S; c0 += 32) {
                uint32_t re[32], im[32];
                TMEM_LD32(tl + c0, re);
                TMEM_LD32(tl + 256 + c0, im);
                tmem_wait_ld();
#pragma unroll
                for (int n = 0; n < 32; ++n) {
                    const float xr = __uint_as_float(re[n]), xi = __uint_as_float(im[n]);
                    const float m2 = xr * xr + xi * xi;
                    const int q = pm == 0 ? 0 : Kp - pm;
                    const uint32_t D = ((uint32_t)q << w.lev) + (uint32_t)v;
                    const unsigned long long key =
                        ((unsigned long long)__float_as_uint(m2) << 32) | (unsigned long long)(0xFFFFFFFFu - D);
                    best = key > best ? key : best;
                    if (WITH_R && Rrow) Rrow[D] = make_float2(xr, xi);
                    pm = pm == 0 ? Kp - 1 : pm - 1;
                }
            }
            tc_fence_before();
            mbar_arrive(tfree);
            if (valid && best) atomicMax(&keys[pass ? w.slot : w.slot_mid], best);
          }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0 && sflag[0]) {
        // let this CTA's own copies land before its shared memory is released
        for (int k = sflag[2]; k < sflag[1]; ++k) mbar_wait(&full[k & 1], (k >> 1) & 1);
        atomicOr(err, kErrTcWait);
    }
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// Split contractions: block (x = split tile, y = pair of columns) sums the
// tile's parts for its 2 x 128 elements in a fixed order (band-0 parts
// first; their partial sum is scale J's product when slot_mid >= 0) and forms
// the peak keys exactly as the epilogue does (one atomicMax per warp).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) tc_split_reduce_kernel(const TcSplit *__restrict__ splits,
                                                              const float2 *__restrict__ part,
                                                              unsigned long long *__restrict__ keys,
                                                              float2 *__restrict__ R) {
    const TcSplit sp = splits[blockIdx.x];
    const int n = 2 * blockIdx.y + (threadIdx.x >> 7);  // column (advance offset within the tile)
    const int m = threadIdx.x & 127;                    // row
    if (n >= sp.S) return;                               // warp-uniform: a warp holds one column
    const int G = 16 * sp.tile + (m >> 3);
    const int v = G / sp.gv;
    const int i = 8 * (G % sp.gv) + (m & 7);
    const bool valid = v < sp.nv;
    const int64_t stride = (int64_t)sp.S * 128;
    const float2 *p = part + sp.part_first + (int64_t)n * 128 + m;
    float2 mid = make_float2(0.f, 0.f);
    for (int k = 0; k < sp.nparts0; ++k) {
        const float2 x = p[k * stride];
        mid.x += x.x;
        mid.y += x.y;
    }
    float2 all = mid;
    for (int k = sp.nparts0; k < sp.nparts; ++k) {
        const float2 x = p[k * stride];
        all.x += x.x;
        all.y += x.y;
    }
    // advance of column n: p = S i - n (mod K'); delay q = -p mod K'
    int pm = (int)((((int64_t)sp.S * i - n) % sp.Kp + sp.Kp) % sp.Kp);
    const int q = pm == 0 ? 0 : sp.Kp - pm;
    const uint32_t D = ((uint32_t)q << sp.lev) + (uint32_t)v;
    auto key_of = [&](float2 a) {
        const float m2 = a.x * a.x + a.y * a.y;
        return ((unsigned long long)__float_as_uint(m2) << 32) | (unsigned long long)(0xFFFFFFFFu - D);
    };
    unsigned long long kall = valid ? key_of(all) : 0ull;
    unsigned long long kmid = (valid && sp.slot_mid >= 0) ? key_of(mid) : 0ull;
    if (R && valid) {
        R[sp.r_at + D] = all;
        if (sp.slot_mid >= 0) R[sp.r_mid + D] = mid;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xffffffffu, kall, o);
        const unsigned long long b = __shfl_xor_sync(0xffffffffu, kmid, o);
        kall = a > kall ? a : kall;
        kmid = b > kmid ? b : kmid;
    }
    if ((threadIdx.x & 31) == 0) {
        if (kall) atomicMax(&keys[sp.slot], kall);
        if (kmid) atomicMax(&keys[sp.slot_mid], kmid);
    }
}

// ---------------------------------------------------------------------------
// Operand packing
// ---------------------------------------------------------------------------
struct StoreScale {
    int64_t out_off;   // element offset in the stored-operand buffer
    int64_t first;     // first flat index of this scale in the launch
    int64_t count;     // elements of this scale
    int64_t level_off; // 2 N (lev - 1): level lev in the SIDWT tree
    int32_t Kp, nv, Lr, Rs, k0;  // Rs reshaped rows of Lr polyphase samples
};
struct StoreScales {
    StoreScale s[16];
    int n;
};

// Chunk pair q of one scale's packed stored operand: the hi and the lo chunk
// (8 elements, one 16-byte store each) of the same (variant, row, block,
// residue, plane), written at `o` (the scale's first element).  The bands of
// the scale's level start at tree[z.level_off] and are N elements apart.
__device__ __forceinline__ void stored_pair(const float2 *__restrict__ tree, int64_t N, const StoreScale &z,
                                            int64_t q, __nv_bfloat16 *__restrict__ o);

// Stored operand of one signal: element [b nv + v][h][row][blk][2 c + plane][e]
// = hi (h = 0) or lo part of plane(w_{v,b}[(k0 + c + 8 s) mod K']), plane 0
// Re, 1 Im, at polyphase sample s = row Lr + 8 blk + e.  A thread writes the
// hi and lo chunks of one (..., c, plane): 8 samples e read once, split
// once, and every index but s computed once.  Scale counts are multiples of
// 128 elements (16 per chunk pair), so pairs never straddle scales.
__global__ void pack_stored_kernel(const float2 *__restrict__ tree, int64_t N, StoreScales sc, int64_t pairs,
                                   __nv_bfloat16 *__restrict__ out) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < pairs; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = 16 * q;
        int k = 0;
        while (k + 1 < sc.n && e >= sc.s[k + 1].first) ++k;
        const StoreScale &z = sc.s[k];
        stored_pair(tree, N, z, (e - z.first) >> 4, out + z.out_off);
    }
}

// The stored operands of many signals in one launch: entry k is one scale
// of one signal (level_off absolute in the tree buffer, N its band stride);
// entries ordered by `first`, found by binary search.
constexpr int kPackBatch = 240;
struct StoreScaleB {
    StoreScale z;
    int64_t N;
};
struct PackBatch {
    int32_t n, pad;
    StoreScaleB s[kPackBatch];
};

__global__ void pack_stored_batch_kernel(const float2 *__restrict__ tree, const __grid_constant__ PackBatch b,
                                         int64_t pairs, __nv_bfloat16 *__restrict__ out) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < pairs; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = 16 * q;
        int lo = 0, hi = b.n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (b.s[mid].z.first <= e) lo = mid;
            else hi = mid - 1;
        }
        const StoreScale &z = b.s[lo].z;
        stored_pair(tree, b.s[lo].N, z, (e - z.first) >> 4, out + z.out_off);
    }
}

__device__ __forceinline__ void stored_pair(const float2 *__restrict__ tree, int64_t N, const StoreScale &z,
                                            int64_t q64, __nv_bfloat16 *__restrict__ o) {
    // 32-bit index arithmetic: a scale holds fewer than 2^31 chunks (checked
    // when the launch is built), and its polyphase samples s and sequence
    // indices stay below 2^31
    const uint32_t q = (uint32_t)q64;
    const int ch = (int)(q & 15);
    const uint32_t nblk = (uint32_t)z.Lr >> 3;
    uint32_t rest = q >> 4;
    const int blk = (int)(rest % nblk);
    rest /= nblk;
    const int row = (int)(rest % (uint32_t)z.Rs);
    const int vb = (int)(rest / (uint32_t)z.Rs);
    const int b = vb / z.nv, v = vb - b * z.nv;
    const int c = ch >> 1, plane = ch & 1;
    const int s0 = row * z.Lr + 8 * blk;
    int idx = (z.k0 + c + 8 * s0) % z.Kp;
    if (idx < 0) idx += z.Kp;
    const float2 *w = tree + z.level_off + (int64_t)b * N + (int64_t)v * z.Kp;
    // sample s0 + e reads index idx + 8 e (mod K'); K' >= 64 > 8 e, so one wrap at most
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
        int i0 = idx + 8 * e, i1 = i0 + 8;
        if (i0 >= z.Kp) i0 -= z.Kp;
        if (i1 >= z.Kp) i1 -= z.Kp;
        const float2 x0 = w[i0], x1 = w[i1];
        __nv_bfloat16 h0, l0, h1, l1;
        split_bf16(plane ? x0.y : x0.x, h0, l0);
        split_bf16(plane ? x1.y : x1.x, h1, l1);
        hw[e >> 1] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        lw[e >> 1] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    // chunk (vb, h, row, blk, ch) starts at element 8 (((2 vb + h) Rs + row) nblk 16 + 16 blk + ch)
    const int64_t per_h = (int64_t)z.Rs * nblk * 128;  // elements of one (vb, h) slab
    const int64_t at = (int64_t)vb * 2 * per_h + ((int64_t)row * nblk + blk) * 128 + 8 * ch;
    *reinterpret_cast<uint4 *>(o + at) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4 *>(o + at + per_h) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
// Untuned weights: typical values the autotuner measures on a GB300 (the
// narrower tiles issue as many TMA boxes per K-block as S = 256 for less MMA
// work each).
void default_weights(TcWeights *t) {
    for (int b = 0; b < kTcBuckets; ++b) {
        t->w[0][b] = 1.0f;
        t->w[1][b] = 1.75f;
        t->w[2][b] = 3.2f;
        t->w[3][b] = 1.2f;
    }
}

static void fill_shape(int64_t N, int J, int j, int S, Shape *sh) {
    sh->j = j;
    sh->lev = j < J ? j + 1 : J;
    sh->nb = j < J ? 2 : 1;
    sh->nv = 1 << sh->lev;
    sh->Kp = N >> sh->lev;
    sh->S = S;
    sh->Lr = S / 8;
    const bool circ = sh->Kp % 64 == 0;
    sh->k0 = circ ? 0 : -S;
    sh->nkb = circ ? (int)(sh->Kp / 64) : (int)(((sh->Kp + 63) / 64 * 64 + S) / 64);
    const int64_t rpv = (sh->Kp + S - 1) / S;
    sh->gv = (int)((rpv + 7) / 8);
    const int64_t groups = (int64_t)sh->nv * sh->gv;
    sh->tiles = (int)((groups + 15) / 16);
    sh->Rs = sh->gv * 8 + (8 * sh->nkb + sh->Lr - 1) / sh->Lr;
    sh->a_elems = (int64_t)2 * sh->nb * sh->nv * 16 * sh->Rs * sh->Lr;
}

bool shape_with(int64_t N, int J, int j, int S, Shape *sh) {
    const int lev = j < J ? j + 1 : J;
    const int64_t Kp = N >> lev;
    if (Kp < kMinBand || Kp > kMaxBand || (S != 256 && S != 192 && S != 128 && S != 64)) return false;
    fill_shape(N, J, j, S, sh);
    return true;
}

// Tensor-core shape of scale j, or false when the band is too short (it
// stays on the CUDA cores).  S (256, 192, 128 or 64) minimises the padded MMA
// work, weighted by each width's cost per padded element in the band's
// log2 bucket (defaults, or measured by the autotuner).
bool shape_for(int64_t N, int J, int j, Shape *sh, const TcWeights *w) {
    const int lev = j < J ? j + 1 : J;
    const int64_t Kp = N >> lev;
    if (Kp < kMinBand || Kp > kMaxBand) return false;
    TcWeights def;
    if (!w) {
        default_weights(&def);
        w = &def;
    }
    int b = 0;
    while (b + 1 < kTcBuckets && (int64_t(2) << b) <= Kp) ++b;  // floor(log2 Kp)
    double best = 1e300;
    for (int k = 0; k < kTcWidths; ++k) {
        Shape t;
        fill_shape(N, J, j, kTcWidth[k], &t);
        const double cost = (double)t.tiles * kTcWidth[k] * t.nkb * w->w[k][b];
        if (cost < best) {
            best = cost;
            *sh = t;
        }
    }
    return true;
}

int64_t operand_elems(int64_t N, int J) {
    int64_t a = 0;
    for (int j = 0; j <= J && j < 16; ++j) {
        Shape sh;
        if (!shape_for(N, J, j, &sh)) continue;
        a += (sh.a_elems + 63) / 64 * 64;
    }
    return a;
}

sidwt_status pack_stored(const float2 *tree, int64_t N, int J, const int64_t *a_off, const int16_t *S_of, void *abuf,
                         cudaStream_t s) {
    StoreScales sc;
    std::memset(&sc, 0, sizeof(sc));
    int64_t total = 0;
    for (int j = 0; j <= J && j < 16; ++j) {
        Shape sh;
        if (a_off[j] < 0 || !shape_with(N, J, j, S_of[j], &sh)) continue;
        StoreScale &z = sc.s[sc.n++];
        if (sh.a_elems / 8 >= (int64_t(1) << 31) || (int64_t)sh.Rs * sh.Lr * 8 + 64 >= (int64_t(1) << 31)) {
            set_error("band too long for the stored-operand packing");
            return SIDWT_EINVAL;
        }
        z.out_off = a_off[j];
        z.first = total;
        z.count = sh.a_elems;
        z.level_off = 2 * N * (int64_t)(sh.lev - 1);
        z.Kp = (int32_t)sh.Kp;
        z.nv = sh.nv;
        z.Lr = sh.Lr;
        z.Rs = sh.Rs;
        z.k0 = sh.k0;
        total += sh.a_elems;
    }
    if (total == 0) return SIDWT_OK;
    const int64_t pairs = total / 16;  // scale counts are multiples of 128 elements
    const int64_t blocks = std::min<int64_t>((pairs + 255) / 256, 152 * 16);
    pack_stored_kernel<<<(unsigned)blocks, 256, 0, s>>>(tree, N, sc, pairs, static_cast<__nv_bfloat16 *>(abuf));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "stored tensor-core operand packing");
}

sidwt_status pack_stored_batch(const float2 *tree, const PackItem *items, int n, void *abuf, cudaStream_t s,
                               int *launches) {
    PackBatch b;
    std::memset(&b, 0, sizeof(b));
    int64_t total = 0;
    int nl = 0;
    auto flush = [&]() -> sidwt_status {
        if (b.n == 0) return SIDWT_OK;
        const int64_t pairs = total / 16;
        const int64_t blocks = std::min<int64_t>((pairs + 255) / 256, 152 * 16);
        pack_stored_batch_kernel<<<(unsigned)blocks, 256, 0, s>>>(tree, b, pairs,
                                                                   static_cast<__nv_bfloat16 *>(abuf));
        cudaError_t e = cudaGetLastError();
        ++nl;
        b.n = 0;
        total = 0;
        return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "batched stored tensor-core operand packing");
    };
    for (int k = 0; k < n; ++k) {
        const PackItem &it = items[k];
        for (int j = 0; j <= it.J && j < 16; ++j) {
            Shape sh;
            if (it.a_off[j] < 0 || !shape_with(it.N, it.J, j, it.S_of[j], &sh)) continue;
            if (b.n == kPackBatch) {
                sidwt_status st = flush();
                if (st) return st;
            }
            if (sh.a_elems / 8 >= (int64_t(1) << 31) || (int64_t)sh.Rs * sh.Lr * 8 + 64 >= (int64_t(1) << 31)) {
                set_error("band too long for the stored-operand packing");
                return SIDWT_EINVAL;
            }
            StoreScaleB &e = b.s[b.n++];
            e.N = it.N;
            StoreScale &z = e.z;
            z.out_off = it.a_off[j];
            z.first = total;
            z.count = sh.a_elems;
            z.level_off = it.tree_off + 2 * it.N * (int64_t)(sh.lev - 1);
            z.Kp = (int32_t)sh.Kp;
            z.nv = sh.nv;
            z.Lr = sh.Lr;
            z.Rs = sh.Rs;
            z.k0 = sh.k0;
            total += sh.a_elems;
        }
    }
    sidwt_status st = flush();
    if (launches) *launches = nl;
    return st;
}

size_t map_bytes() { return sizeof(CUtensorMap); }

sidwt_status encode_maps(void *two_maps, const void *a_base, const void *b_base, const Shape &sh) {
    CUtensorMap *m = static_cast<CUtensorMap *>(two_maps);
    // dims: 128 elements of a (row, block) record, Lr / 8 blocks, Rs rows,
    // hi/lo, band x variant; a box is one chunk half of 8 rows, hi and lo
    const uint64_t blk = (uint64_t)sh.Lr / 8;
    const uint64_t da[5] = {128, blk, (uint64_t)sh.Rs, 2, (uint64_t)sh.nv * sh.nb};
    const uint64_t sa[4] = {256, 256 * blk, 256 * blk * sh.Rs, 512 * blk * sh.Rs};
    const uint32_t ba[5] = {64, 1, 8, 2, 1};
    (void)b_base;  // the received windows are expanded in shared memory by the kernel
    std::memset(&m[1], 0, sizeof(CUtensorMap));
    return encode_nd(&m[0], const_cast<void *>(a_base), 5, da, sa, ba, CU_TENSOR_MAP_SWIZZLE_128B);
}


sidwt_status launch_corr(const void *maps, const TcTile *tiles, int ntiles, const float2 *pyr, unsigned long long *keys,
                         int32_t *err, int sms, cudaStream_t s, float2 *R, float2 *part) {
    if (ntiles <= 0) return SIDWT_OK;
    const int grid = std::min(sms, ntiles);
    const CUtensorMap *m = static_cast<const CUtensorMap *>(maps);
    if (R && part)
        corr_pair_tc_kernel<true, true><<<grid, kThreads, kSmemBytes, s>>>(m, tiles, ntiles, pyr, keys, err, R, part);
    else if (R)
        corr_pair_tc_kernel<true, false><<<grid, kThreads, kSmemBytes, s>>>(m, tiles, ntiles, pyr, keys, err, R, part);
    else if (part)
        corr_pair_tc_kernel<false, true><<<grid, kThreads, kSmemBytes, s>>>(m, tiles, ntiles, pyr, keys, err, R, part);
    else
        corr_pair_tc_kernel<false, false><<<grid, kThreads, kSmemBytes, s>>>(m, tiles, ntiles, pyr, keys, err, R, part);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "tensor-core pair correlation launch");
}

sidwt_status launch_split_reduce(const TcSplit *splits, int nsplits, int maxS, const float2 *part,
                                 unsigned long long *keys, float2 *R, cudaStream_t s) {
    if (nsplits <= 0) return SIDWT_OK;
    tc_split_reduce_kernel<<<dim3((unsigned)nsplits, (unsigned)((maxS + 1) / 2)), 256, 0, s>>>(splits, part, keys, R);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "split-contraction reduction launch");
}

cudaError_t prepare_kernels() {
    cudaError_t e = cudaFuncSetAttribute(corr_pair_tc_kernel<false, false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(corr_pair_tc_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(corr_pair_tc_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(corr_pair_tc_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kSmemBytes);
    return e;
}

}  // namespace rtc
}  // namespace sidwt
