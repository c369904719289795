// Per-scale all-lag correlation on the tcgen05 tensor cores with a bf16
// hi+lo split (three products hi*hi + hi*lo + lo*hi, FP32 accumulation in
// TMEM).
//
// The products are the shift-circulant block products of eq. 20 / 20a in
// "advance" form: for a variant band w (length K') and received band u,
//     C[m][p] = sum_k conj(w[(k + p) mod K']) u_m[k]
// with m a pulse and p = 0..K'-1 the circular advance (the delay is
// q = -p mod K', D = 2^l q + v).  One CTA computes 128 pulses x N_T
// consecutive advances (N_T = 256 where K' allows).
//
// The circulant operand is never materialised.  For the 8 residues c of k
// mod 8 the library keeps 8 shifted copies W_c[t] = w[t + c] of each band
// (doubled for the wrap); in shared memory a 320-element window of W_c is an
// MN-major, non-swizzled B operand whose 8 x 8 core matrices overlap at
// 16-byte steps: element (k = c + 8a, n) sits at 2 (8a + n) bytes, i.e. lag
// n+1 is the next 2 bytes and k+8 the next 16 bytes.  The received side is
// stored polyphase-by-8 ([chunk][pulse][8]) so that A is a plain K-major tile.
// Complex arithmetic uses two accumulators: Re = <(ur, ui), (wr, wi)> and
// Im = <(ur, ui), (-wi, wr)>; the planes (-wi, wr, wi) sit 640 B apart so
// both come from one descriptor stride.
//
// Roles (192 threads): warp 0 issues TMA loads into a 2-stage ring, warp 1
// allocates TMEM and issues the MMAs, warps 2-5 read the accumulators and
// reduce the peaks.  Scales J - 1 and J share level J, and scale J's product
// (eq. 20a) is band 0 of scale J - 1's (eq. 20): with TcArgs::fold the scale
// J - 1 launch hands its accumulators to the epilogue after band 0 (scale J's
// peaks), waits on `tfree` until they have been read, then adds band 1.
// Every wait is bounded; on a timeout the CTA records an error, drains its
// own copies and frees TMEM.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "tc_common.cuh"

namespace sidwt {
namespace tc {

constexpr int kThreads = 192;
constexpr int kTM = 128;                            // pulses per tile
constexpr int kBoxChunks = 40;                      // 320 window elements per row
constexpr int kWinRowBytes = kBoxChunks * 16;       // 640
constexpr int kBRows = 24;                          // 8 shifted copies x 3 planes
constexpr int kBBytes = kBRows * kWinRowBytes;      // 15360 (hi or lo)
constexpr int kABytes = 16 * kTM * 16;              // 32768 (hi or lo): [16 chunks][128 rows][16 B]
constexpr int kStageB = 2 * kBBytes;                // 30720
constexpr int kStageA = 2 * kABytes;                // 65536
constexpr int kStageTx = kStageA + kStageB;         // 96256 bytes per stage
constexpr int kBRegion = 2 * kStageB;               // B ring first (low addresses)
constexpr int kARegion = 2 * kStageA;
constexpr int kBarOff = kBRegion + kARegion;        // 192512
constexpr int kSmemBytes = 227 * 1024;              // whole budget: one CTA per SM, every read in bounds
constexpr int kTmemCols = 512;

struct TcArgs {
    int64_t N;
    int J, j, lev;
    int Kp;          // band length at level lev
    int nv;          // variants 2^lev
    int nbands;      // 2 for j < J, 1 for j = J
    int ntile_n;     // advances per tile (MMA N)
    int nlt;         // advance tiles per variant
    int nkb;         // K-blocks of 64
    int kb_per_band; // Kp / 64
    int fold;        // 1: j = J - 1 also forms scale J (eq. 20a) from band 0 before adding band 1
    int rows_per_ref;
    const int32_t *perm;
    const int32_t *tile_ref;
    const int32_t *tile_start;
    const int32_t *tile_count;
    const int32_t *ntiles;
    unsigned long long *keys;
    float2 *R;
    int32_t *err;
};

__global__ void __launch_bounds__(kThreads, 1)
    corr_tc_kernel(const __grid_constant__ CUtensorMap mapA_hi, const __grid_constant__ CUtensorMap mapA_lo,
                   const __grid_constant__ CUtensorMap mapB, const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *sB = base;
    unsigned char *sA = base + kBRegion;
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + kBarOff);  // full[2], empty[2], accf, tfree
    uint64_t *full = bar, *empty = bar + 2, *accf = bar + 4, *tfree = bar + 5;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 8);
    volatile int *sflag = reinterpret_cast<volatile int *>(tmem_slot + 4);  // [0] error, [1] issued, [2] consumed

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx = blockIdx.x;
    const int lt = bx % a.nlt;
    const int v = (bx / a.nlt) % a.nv;
    const int pt = bx / (a.nlt * a.nv);
    if (pt >= a.ntiles[0]) return;  // uniform: before any barrier or TMEM use
    const int row0 = a.tile_start[pt];
    const int cnt = a.tile_count[pt];
    const int ref = a.tile_ref[pt];
    const int p0 = lt * a.ntile_n;

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(accf, 1);
        mbar_init(tfree, 128);
        sflag[0] = 0;
        sflag[1] = 0;
        sflag[2] = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int kb = 0; kb < a.nkb; ++kb) {
                const int s = kb & 1;
                if (kb >= 2 && !mbar_wait(&empty[s], ((kb >> 1) - 1) & 1)) {
                    sflag[0] = 1;
                    break;
                }
                if (sflag[0]) break;
                const int band = kb / a.kb_per_band;
                const int kap0 = (kb % a.kb_per_band) * 64;
                mbar_expect_tx(&full[s], kStageTx);
                unsigned char *stA = sA + s * kStageA;
                unsigned char *stB = sB + s * kStageB;
                tma_load_3d(stA, &mapA_hi, &full[s], 0, row0, kb * 16);
                tma_load_3d(stA + kABytes, &mapA_lo, &full[s], 0, row0, kb * 16);
                const int rowbase = ref * a.rows_per_ref + ((band * a.nv + v) * 2) * kBRows;
                const int chunk0 = (kap0 + p0) >> 3;
                tma_load_3d(stB, &mapB, &full[s], 0, chunk0, rowbase);
                tma_load_3d(stB + kBBytes, &mapB, &full[s], 0, chunk0, rowbase + kBRows);
                ++issued;
            }
            sflag[1] = issued;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(kTM, a.ntile_n);
            int consumed = 0;
            for (int kb = 0; kb < a.nkb; ++kb) {
                const int s = kb & 1;
                if (a.fold && kb == a.kb_per_band) {
                    // band 0 alone is scale J's product (eq. 20a): hand it to the epilogue,
                    // add band 1 once the epilogue has read it
                    mma_commit(accf);
                    if (!mbar_wait(tfree, 0)) {
                        sflag[0] = 1;
                        break;
                    }
                    tc_fence_after();
                }
                if (!mbar_wait(&full[s], (kb >> 1) & 1)) {
                    sflag[0] = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t aHi = saddr(sA + s * kStageA), aLo = aHi + kABytes;
                const uint32_t bHi = saddr(sB + s * kStageB), bLo = bHi + kBBytes;
#pragma unroll 1
                for (int c = 0; c < 8; ++c) {
                    // A: chunk (c, re) then (c, im) 2048 B apart along K; 8-row groups 128 B apart
                    const uint64_t ah = sdesc(aHi + c * 4096, 2048, 128);
                    const uint64_t al = sdesc(aLo + c * 4096, 2048, 128);
#pragma unroll
                    for (int acc = 0; acc < 2; ++acc) {
                        // B rows c*3 + {0: -wi, 1: wr, 2: wi}; Re uses (wr, wi), Im uses (-wi, wr);
                        // K direction 640 B (next plane), MN direction 16 B (next 8 advances)
                        const uint32_t row = c * 3 + (acc == 0 ? 1 : 0);
                        const uint64_t bh = sdesc(bHi + row * kWinRowBytes, kWinRowBytes, 16);
                        const uint64_t bl = sdesc(bLo + row * kWinRowBytes, kWinRowBytes, 16);
                        const uint32_t d = tmem + acc * 256;
                        const uint32_t first = (kb == 0 && c == 0) ? 0u : 1u;
                        mma_bf16(d, ah, bh, idesc, first);
                        mma_bf16(d, ah, bl, idesc, 1u);
                        mma_bf16(d, al, bh, idesc, 1u);
                    }
                }
                mma_commit(&empty[s]);
                ++consumed;
            }
            sflag[2] = consumed;
            mma_commit(accf);  // arrives once every MMA issued above has completed
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31; with a.fold
        // first band 0 alone (scale J = a.j + 1), then the whole product (a.j)
        const int q4 = warp & 3;
        const int m = q4 * 32 + lane;
        for (int pass = a.fold ? 0 : 1; pass < 2; ++pass) {
        const int jo = pass ? a.j : a.j + 1;
        const bool ok = mbar_wait(accf, a.fold ? (uint32_t)pass : 0u);
        tc_fence_after();
        if (!ok) sflag[0] = 1;
        if (ok && !sflag[0]) {
            const bool valid = m < cnt;
            const int64_t b = valid ? a.perm[row0 + m] : 0;
            unsigned long long best = 0ull;
            const uint32_t tl = tmem + ((uint32_t)(q4 * 32) << 16);
            for (int c0 = 0; c0 < a.ntile_n; c0 += 32) {
                uint32_t re[32], im[32];
                TMEM_LD32(tl + c0, re);
                TMEM_LD32(tl + 256 + c0, im);
                tmem_wait_ld();
#pragma unroll
                for (int n = 0; n < 32; ++n) {
                    const float xr = __uint_as_float(re[n]), xi = __uint_as_float(im[n]);
                    const float m2 = xr * xr + xi * xi;
                    const int p = p0 + c0 + n;
                    const int q = p == 0 ? 0 : a.Kp - p;
                    const uint32_t D = ((uint32_t)q << a.lev) + (uint32_t)v;
                    const unsigned long long key =
                        ((unsigned long long)__float_as_uint(m2) << 32) | (unsigned long long)(0xFFFFFFFFu - D);
                    best = key > best ? key : best;
                    if (a.R && valid) a.R[(b * (a.J + 1) + jo) * a.N + D] = make_float2(xr, xi);
                }
            }
            if (valid && best) atomicMax(&a.keys[b * (a.J + 1) + jo], best);
        }
        if (pass == 0) {
            tc_fence_before();
            mbar_arrive(tfree);
        }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0 && sflag[0]) {
        // let this CTA's own copies land before its shared memory is released
        for (int kb = sflag[2]; kb < sflag[1]; ++kb) mbar_wait(&full[kb & 1], (kb >> 1) & 1);
        atomicOr(a.err, kErrTcWait);
    }
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// Short contractions (K_j <= 128 samples, advance tiles <= 128): the received
// tile of 128 pulses is the same for every variant of the scale, so one CTA
// keeps it resident (both K-blocks, loaded once) and runs kMultiVar variants
// in turn, streaming only their stored windows through a 3-stage ring.  The
// accumulators of consecutive variants rotate through 512 / (2 N_T) TMEM
// slots, so the epilogue of one variant overlaps the MMAs of the next.
// ---------------------------------------------------------------------------
constexpr int kMultiVar = 8;                                 // variants per CTA
constexpr int kMStagesB = 3;
constexpr int kMARegion = 2 * kStageA;                       // resident A, K-blocks 0 and 1
constexpr int kMBarOff = kMARegion + kMStagesB * kStageB;    // 223232
constexpr int kMSmemBytes = kMBarOff + 256 + 1024;
static_assert(kMSmemBytes <= 227 * 1024, "shared memory budget");

__global__ void __launch_bounds__(kThreads, 1)
    corr_tc_multi_kernel(const __grid_constant__ CUtensorMap mapA_hi, const __grid_constant__ CUtensorMap mapA_lo,
                         const __grid_constant__ CUtensorMap mapB, const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *sA = base;
    unsigned char *sB = base + kMARegion;
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + kMBarOff);
    // fullA, fullB[3], emptyB[3], accf[4], tfree[4]
    uint64_t *fullA = bar, *fullB = bar + 1, *emptyB = bar + 4, *accf = bar + 7, *tfree = bar + 11;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 16);
    // [0] error, [1] B stages issued, [2] B stages consumed, [3] A issued, [4] progress
    volatile int *sflag = reinterpret_cast<volatile int *>(tmem_slot + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nvg = (a.nv + kMultiVar - 1) / kMultiVar;
    const int bx = blockIdx.x;
    const int lt = bx % a.nlt;
    const int vg = (bx / a.nlt) % nvg;
    const int pt = bx / (a.nlt * nvg);
    if (pt >= a.ntiles[0]) return;  // uniform: before any barrier or TMEM use
    const int row0 = a.tile_start[pt];
    const int cnt = a.tile_count[pt];
    const int ref = a.tile_ref[pt];
    const int p0 = lt * a.ntile_n;
    const int v0 = vg * kMultiVar;
    const int nvar = min(kMultiVar, a.nv - v0);
    const int nslots = 512 / (2 * a.ntile_n);  // 2 (N_T = 128) or 4 (N_T = 64)

    if (threadIdx.x == 0) {
        mbar_init(fullA, 1);
        for (int i = 0; i < kMStagesB; ++i) {
            mbar_init(&fullB[i], 1);
            mbar_init(&emptyB[i], 1);
        }
        for (int i = 0; i < 4; ++i) {
            mbar_init(&accf[i], 1);
            mbar_init(&tfree[i], 128);
        }
        for (int i = 0; i < 5; ++i) sflag[i] = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            mbar_expect_tx(fullA, (uint32_t)(a.nkb * kStageA));
            for (int kb = 0; kb < a.nkb; ++kb) {
                tma_load_3d(sA + kb * kStageA, &mapA_hi, fullA, 0, row0, kb * 16);
                tma_load_3d(sA + kb * kStageA + kABytes, &mapA_lo, fullA, 0, row0, kb * 16);
            }
            sflag[3] = 1;
            int it = 0;
            for (int g = 0; g < nvar && !sflag[0]; ++g)
                for (int kb = 0; kb < a.nkb; ++kb, ++it) {
                    const int s = it % kMStagesB, use = it / kMStagesB;
                    if (use > 0 && !mbar_wait(&emptyB[s], (use - 1) & 1)) {
                        sflag[0] = 1;
                        break;
                    }
                    if (sflag[0]) break;
                    const int band = kb / a.kb_per_band;
                    const int kap0 = (kb % a.kb_per_band) * 64;
                    mbar_expect_tx(&fullB[s], kStageB);
                    unsigned char *stB = sB + s * kStageB;
                    const int rowbase = ref * a.rows_per_ref + ((band * a.nv + v0 + g) * 2) * kBRows;
                    const int chunk0 = (kap0 + p0) >> 3;
                    tma_load_3d(stB, &mapB, &fullB[s], 0, chunk0, rowbase);
                    tma_load_3d(stB + kBBytes, &mapB, &fullB[s], 0, chunk0, rowbase + kBRows);
                    sflag[1] = it + 1;
                }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(kTM, a.ntile_n);
            bool okA = mbar_wait(fullA, 0);
            if (!okA) sflag[0] = 1;
            tc_fence_after();
            int it = 0;
            for (int g = 0; g < nvar && okA && !sflag[0]; ++g) {
                const int slot = g % nslots, use = g / nslots;
                if (use > 0) {
                    if (!mbar_wait(&tfree[slot], (use - 1) & 1)) {
                        sflag[0] = 1;
                        break;
                    }
                    tc_fence_after();
                }
                const uint32_t dre = tmem + (uint32_t)(slot * 2 * a.ntile_n), dim = dre + (uint32_t)a.ntile_n;
                for (int kb = 0; kb < a.nkb; ++kb, ++it) {
                    const int s = it % kMStagesB;
                    if (!mbar_wait(&fullB[s], (it / kMStagesB) & 1)) {
                        sflag[0] = 1;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t aHi = saddr(sA + kb * kStageA), aLo = aHi + kABytes;
                    const uint32_t bHi = saddr(sB + s * kStageB), bLo = bHi + kBBytes;
#pragma unroll 1
                    for (int c = 0; c < 8; ++c) {
                        const uint64_t ah = sdesc(aHi + c * 4096, 2048, 128);
                        const uint64_t al = sdesc(aLo + c * 4096, 2048, 128);
#pragma unroll
                        for (int acc = 0; acc < 2; ++acc) {
                            const uint32_t row = c * 3 + (acc == 0 ? 1 : 0);
                            const uint64_t bh = sdesc(bHi + row * kWinRowBytes, kWinRowBytes, 16);
                            const uint64_t bl = sdesc(bLo + row * kWinRowBytes, kWinRowBytes, 16);
                            const uint32_t d = acc == 0 ? dre : dim;
                            const uint32_t first = (kb == 0 && c == 0) ? 0u : 1u;
                            mma_bf16(d, ah, bh, idesc, first);
                            mma_bf16(d, ah, bl, idesc, 1u);
                            mma_bf16(d, al, bh, idesc, 1u);
                        }
                    }
                    mma_commit(&emptyB[s]);
                    sflag[2] = it + 1;
                    sflag[4] = it + 1;
                }
                if (sflag[0]) break;
                mma_commit(&accf[slot]);  // this variant's MMAs have completed
            }
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = pulses of the tile
        const int q4 = warp & 3;
        const int m = q4 * 32 + lane;
        const bool valid = m < cnt;
        const int64_t b = valid ? a.perm[row0 + m] : 0;
        const uint32_t tl = tmem + ((uint32_t)(q4 * 32) << 16);
        for (int g = 0; g < nvar; ++g) {
            const int slot = g % nslots, use = g / nslots;
            uint64_t t0 = now_ns();
            int last = sflag[4];
            bool ok = true;
            while (!mbar_test(&accf[slot], use & 1)) {  // bounded from the MMA thread's last progress
                const int pr = sflag[4];
                if (pr != last) {
                    last = pr;
                    t0 = now_ns();
                } else if (now_ns() - t0 > kWaitNs || sflag[0]) {
                    ok = false;
                    break;
                }
            }
            tc_fence_after();
            if (!__all_sync(0xffffffffu, ok && !sflag[0])) {
                sflag[0] = 1;
                break;
            }
            const int v = v0 + g;
            unsigned long long best = 0ull;
            const uint32_t col = (uint32_t)(slot * 2 * a.ntile_n);
            for (int c0 = 0; c0 < a.ntile_n; c0 += 32) {
                uint32_t re[32], im[32];
                TMEM_LD32(tl + col + c0, re);
                TMEM_LD32(tl + col + a.ntile_n + c0, im);
                tmem_wait_ld();
#pragma unroll
                for (int n = 0; n < 32; ++n) {
                    const float xr = __uint_as_float(re[n]), xi = __uint_as_float(im[n]);
                    const float m2 = xr * xr + xi * xi;
                    const int p = p0 + c0 + n;
                    const int q = p == 0 ? 0 : a.Kp - p;
                    const uint32_t D = ((uint32_t)q << a.lev) + (uint32_t)v;
                    const unsigned long long key =
                        ((unsigned long long)__float_as_uint(m2) << 32) | (unsigned long long)(0xFFFFFFFFu - D);
                    best = key > best ? key : best;
                    if (a.R && valid) a.R[(b * (a.J + 1) + a.j) * a.N + D] = make_float2(xr, xi);
                }
            }
            tc_fence_before();
            mbar_arrive(&tfree[slot]);
            if (valid && best) atomicMax(&a.keys[b * (a.J + 1) + a.j], best);
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0 && sflag[0]) {
        // let this CTA's own copies land before its shared memory is released
        if (sflag[3]) mbar_wait(fullA, 0);
        for (int k = sflag[2]; k < sflag[1]; ++k) mbar_wait(&fullB[k % kMStagesB], (k / kMStagesB) & 1);
        atomicOr(a.err, kErrTcWait);
    }
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// Packing kernels
// ---------------------------------------------------------------------------

// Reference windows for one scale: row r = ((ref * nbands + band) * nv + v) * 48
// + hilo * 24 + c * 3 + plane holds Lc elements W[t] = plane(w[(t + c) mod K'])
// (plane 0: -Im, 1: Re, 2: Im), hi or lo part.  A block takes the hi and the
// lo row of one (ref, band, v, c, plane); a thread 8 consecutive t (Lc and
// K' are multiples of 64, so every chunk is one 16-byte store and its
// indices wrap at most once).
__global__ void pack_ref_kernel(const float2 *__restrict__ tree, int64_t tree_elems, int64_t N, int lev, int nbands,
                                int ref0, int nrefs, int Lc, __nv_bfloat16 *__restrict__ out) {
    const int Kp = (int)(N >> lev), nv = 1 << lev;
    const int pairs_per_ref = nbands * nv * 24;
    const int64_t rp = (int64_t)blockIdx.x + (int64_t)ref0 * pairs_per_ref;
    const int ref = (int)(rp / pairs_per_ref);
    if (ref >= ref0 + nrefs) return;
    int rem = (int)(rp % pairs_per_ref);
    const int plane = rem % 3;
    rem /= 3;
    const int c = rem % 8;
    rem /= 8;
    const int vv = rem % nv;
    const int band = rem / nv;
    const float2 *w = tree + (int64_t)ref * tree_elems + 2 * N * (int64_t)(lev - 1) + (int64_t)band * N + (int64_t)vv * Kp;
    const int64_t row_hi = (((int64_t)ref * nbands + band) * nv + vv) * 48 + c * 3 + plane;
    __nv_bfloat16 *oh = out + row_hi * Lc, *ol = out + (row_hi + 24) * Lc;
    for (int q = threadIdx.x; q < Lc / 8; q += blockDim.x) {
        const int t0 = 8 * q;
        int idx = (t0 + c) % Kp;
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            const float2 x0 = w[idx];
            if (++idx == Kp) idx = 0;
            const float2 x1 = w[idx];
            if (++idx == Kp) idx = 0;
            const float v0 = plane == 0 ? -x0.y : (plane == 1 ? x0.x : x0.y);
            const float v1 = plane == 0 ? -x1.y : (plane == 1 ? x1.x : x1.y);
            __nv_bfloat16 h0, l0, h1, l1;
            split_bf16(v0, h0, l0);
            split_bf16(v1, h1, l1);
            hw[e >> 1] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            lw[e >> 1] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        }
        *reinterpret_cast<uint4 *>(oh + t0) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(ol + t0) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
}

// Received operand for one scale, rows in grouped order: chunk index
// kb * 16 + 2c + plane (plane 0 Re, 1 Im), row = grouped position, 8 values
// u[kb*64 + c + 8a], a = 0..7.  Each CTA transposes 32 rows x one K-block.
// same_input: the buffers already hold this pyramid packed for this batch
// size; the packing is skipped when the grouping is unchanged too (ntiles[2],
// written by the grouping kernel of this call).
__global__ void __launch_bounds__(256) pack_rx_kernel(const float2 *__restrict__ pyr, int64_t pyr_elems, int64_t off,
                                                      const int32_t *__restrict__ perm, const int32_t *__restrict__ ntiles,
                                                      int rows, __nv_bfloat16 *__restrict__ ahi,
                                                      __nv_bfloat16 *__restrict__ alo, int same_input) {
    __shared__ float2 tile[32][65];
    if (same_input && ntiles[2] == 0) return;  // uniform over the grid
    const int kb = blockIdx.x;
    const int r0 = blockIdx.y * 32;
    const int nvalid = ntiles[1];
    // 32 rows x 64 samples as 16-byte loads of two samples (rows start on even samples)
#pragma unroll
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
        const int i = e >> 5, k2 = e & 31;
        const int r = r0 + i;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < nvalid)
            v = *reinterpret_cast<const float4 *>(pyr + (int64_t)perm[r] * pyr_elems + off + (int64_t)kb * 64 + 2 * k2);
        tile[i][2 * k2] = make_float2(v.x, v.y);
        tile[i][2 * k2 + 1] = make_float2(v.z, v.w);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 16 * 32; e += 256) {
        const int cp = e >> 5, i = e & 31;
        const int r = r0 + i;
        if (r >= rows) continue;
        const int c = cp >> 1, plane = cp & 1;
        __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
        for (int a8 = 0; a8 < 8; ++a8) {
            const float2 v = tile[i][c + 8 * a8];
            split_bf16(plane ? v.y : v.x, h[a8], l[a8]);
        }
        const int64_t o = (((int64_t)kb * 16 + cp) * rows + r) * 8;
        *reinterpret_cast<uint4 *>(ahi + o) = *reinterpret_cast<const uint4 *>(h);
        *reinterpret_cast<uint4 *>(alo + o) = *reinterpret_cast<const uint4 *>(l);
    }
}

// ---------------------------------------------------------------------------
// Self-test of the operand layouts: one MMA (M = 128, N = 64, K = 16) on
// integer-valued data staged by plain stores, A K-major and B the overlapping
// MN-major window, exactly as the correlation kernel addresses them.
// out: [128][64] floats.
// ---------------------------------------------------------------------------
constexpr int kSelftestSmem = 64 * 1024;

__global__ void __launch_bounds__(128, 1) tc_selftest_kernel(float *out, int32_t *err, int stall) {
    extern __shared__ __align__(1024) unsigned char sm[];  // 64 KB: every reading of the strides stays inside
    __shared__ uint64_t bar;
    __shared__ uint32_t slot;
    unsigned char *sa = sm;                 // [2 chunks][128 rows][8] bf16
    unsigned char *sb = sm + 4096;          // 3 rows x 320 bf16
    __nv_bfloat16 *A = reinterpret_cast<__nv_bfloat16 *>(sa);
    __nv_bfloat16 *W = reinterpret_cast<__nv_bfloat16 *>(sb);
    for (int e = threadIdx.x; e < 2 * 128 * 8; e += 128) {
        const int chunk = e / 1024, row = (e / 8) % 128, a8 = e % 8;
        const int k = chunk * 8 + a8;
        A[e] = __float2bfloat16_rn((float)(((row * 7 + k * 3) % 11) - 5));
    }
    for (int e = threadIdx.x; e < 3 * 320; e += 128) {
        const int pl = e / 320, t = e % 320;
        W[e] = __float2bfloat16_rn((float)(((t * 5 + pl * 17) % 13) - 6));
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    if (warp == 0) tmem_alloc(&slot, 64);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // plain stores -> tensor-core reads
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = slot;
    // stall (test hook, sidwt_debug_stall): neither the MMA nor its commit is
    // issued, so the wait below runs out with nothing in flight, and TMEM is
    // still released at the end
    if (threadIdx.x == 0 && !stall) {
        const uint64_t ad = sdesc(saddr(sa), 2048, 128);
        const uint64_t bd = sdesc(saddr(sb + 640), 640, 16);  // planes 1 and 2
        mma_bf16(tmem, ad, bd, idesc_bf16(128, 64), 0u);
        mma_commit(&bar);
    }
    const bool ok = mbar_wait(&bar, 0);
    tc_fence_after();
    if (!ok && threadIdx.x == 0) atomicOr(err, kErrSelftestWait);
    if (ok) {
        const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < 64; c0 += 32) {
            uint32_t r[32];
            TMEM_LD32(tl + c0, r);
            tmem_wait_ld();
            for (int n = 0; n < 32; ++n) out[(warp * 32 + lane) * 64 + c0 + n] = __uint_as_float(r[n]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, 64);
}


}  // namespace tc

// Scales the tensor-core path takes: band length a multiple of 64.
uint32_t tc_scale_mask(const sidwt_plan *p) {
    uint32_t m = 0;
    for (int j = 0; j <= p->J; ++j) {
        const int lev = j < p->J ? j + 1 : p->J;
        const int64_t Kp = p->N >> lev;
        if (Kp >= 64 && Kp % 64 == 0 && Kp <= (int64_t(1) << 24)) m |= 1u << j;
    }
    return m;
}

static int tc_ntile(int64_t Kp) { return Kp % 256 == 0 ? 256 : (Kp % 128 == 0 ? 128 : 64); }

// Scale J (eq. 20a) is band 0 of scale J - 1 (eq. 20), both at level J: the
// scale J - 1 launch forms both when both are tensor-core scales and it runs
// the one-tile kernel (K' >= 128; K' = 64 takes the short-contraction kernel).
static bool tc_fold_last(const sidwt_plan *p, uint32_t mask) {
    const int J = p->J;
    if (J < 1 || !(mask & (1u << J)) || !(mask & (1u << (J - 1)))) return false;
    return (p->N >> J) >= 128;
}
static int tc_lc(int64_t Kp) { return (int)(2 * Kp + 320); }
static int tc_rows_per_ref(const sidwt_plan *p, int j) {
    const int lev = j < p->J ? j + 1 : p->J;
    return (j < p->J ? 2 : 1) * (1 << lev) * 48;
}

void free_tc(sidwt_plan *p) {
    for (int j = 0; j < 16; ++j) {
        if (p->tc_ref[j]) cudaFree(p->tc_ref[j]);
        if (p->tc_ahi[j]) cudaFree(p->tc_ahi[j]);
        if (p->tc_alo[j]) cudaFree(p->tc_alo[j]);
        p->tc_ref[j] = p->tc_ahi[j] = p->tc_alo[j] = nullptr;
    }
    p->tc_cap_refs = 0;
    p->tc_cap_batch = 0;
    p->tc_packed = 0;
    p->tc_rx_gen = -1;
}

// Allocate the packed operands for the current reference and batch capacity.
static sidwt_status ensure_tc(sidwt_plan *p) {
    if (p->tc_cap_refs >= p->cap_refs && p->tc_cap_batch >= p->cap_batch) return SIDWT_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronise before tensor-core buffers");
    free_tc(p);
    const uint32_t mask = tc_scale_mask(p);
    for (int j = 0; j <= p->J; ++j) {
        if (!(mask & (1u << j))) continue;
        const int lev = j < p->J ? j + 1 : p->J;
        const int64_t Kp = p->N >> lev;
        const int64_t Kj = (j < p->J ? 2 : 1) * Kp;
        const size_t rb = (size_t)p->cap_refs * tc_rows_per_ref(p, j) * tc_lc(Kp) * 2;
        const size_t ab = (size_t)(Kj / 64) * 16 * p->cap_batch * 16;
        if (cudaMalloc(&p->tc_ref[j], rb) != cudaSuccess || cudaMalloc(&p->tc_ahi[j], ab) != cudaSuccess ||
            cudaMalloc(&p->tc_alo[j], ab) != cudaSuccess) {
            cudaGetLastError();
            free_tc(p);
            set_error("device allocation failed for the tensor-core operands");
            return SIDWT_ENOMEM;
        }
    }
    p->tc_cap_refs = p->cap_refs;
    p->tc_cap_batch = p->cap_batch;
    p->tc_packed = 0;
    return SIDWT_OK;
}

sidwt_status correlate_tc(sidwt_plan *p, int64_t B, float2 *r_dev, cudaStream_t s) {
    sidwt_status st = ensure_tc(p);
    if (st) return st;
    const uint32_t mask = tc_scale_mask(p);
    const int64_t N = p->N;
    const int J = p->J;
    // stored references not yet packed
    if (p->tc_packed < p->nrefs) {
        for (int j = 0; j <= J; ++j) {
            if (!(mask & (1u << j))) continue;
            const int lev = j < J ? j + 1 : J;
            const int nb = j < J ? 2 : 1;
            // one block per (hi, lo) row pair
            const int64_t rows = (int64_t)(p->nrefs - p->tc_packed) * tc_rows_per_ref(p, j) / 2;
            tc::pack_ref_kernel<<<(unsigned)rows, 256, 0, s>>>(p->tree_f, p->tree_elems, N, lev, nb, p->tc_packed,
                                                  p->nrefs - p->tc_packed, tc_lc(N >> lev),
                                                  reinterpret_cast<__nv_bfloat16 *>(p->tc_ref[j]));
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "reference packing launch");
        p->tc_packed = p->nrefs;
    }
    const int64_t max_pt = (B + tc::kTM - 1) / tc::kTM + std::min<int64_t>(p->nrefs, B);
    const bool fold = tc_fold_last(p, mask);
    // the received operands already hold this analysis's pyramid for B pulses
    // (sidwt_correlate_again on the same batch): repacked only if the grouping changed
    const bool same_input = p->tc_rx_gen == p->analysis_gen && p->tc_rx_B == B;
    p->tc_rx_gen = p->analysis_gen;
    p->tc_rx_B = B;
    for (int j = 0; j <= J; ++j) {
        if (!(mask & (1u << j))) continue;
        if (fold && j == J) continue;  // formed by the scale J - 1 launch
        const int lev = j < J ? j + 1 : J;
        const int64_t Kp = N >> lev;
        const int nb = j < J ? 2 : 1;
        const int64_t Kj = nb * Kp;
        const int64_t nchunks = Kj / 64 * 16;
        __nv_bfloat16 *ahi = reinterpret_cast<__nv_bfloat16 *>(p->tc_ahi[j]);
        __nv_bfloat16 *alo = reinterpret_cast<__nv_bfloat16 *>(p->tc_alo[j]);
        {
            dim3 g((unsigned)(Kj / 64), (unsigned)((B + 31) / 32));
            tc::pack_rx_kernel<<<g, 256, 0, s>>>(p->pyr_f, p->pyr_elems, 2 * N - 4 * Kp, p->tiles.perm,
                                                 p->tiles.ntiles, (int)B, ahi, alo, same_input ? 1 : 0);
        }
        CUtensorMap mA_hi, mA_lo, mB;
        if ((st = tc::encode_3d(&mA_hi, ahi, 8, (uint64_t)B, (uint64_t)nchunks, 16, 16 * (uint64_t)B, 8, tc::kTM, 16)) ||
            (st = tc::encode_3d(&mA_lo, alo, 8, (uint64_t)B, (uint64_t)nchunks, 16, 16 * (uint64_t)B, 8, tc::kTM, 16)))
            return st;
        const int Lc = tc_lc(Kp);
        const int rpr = tc_rows_per_ref(p, j);
        if ((st = tc::encode_3d(&mB, p->tc_ref[j], 8, (uint64_t)(Lc / 8), (uint64_t)p->nrefs * rpr, 16,
                                (uint64_t)Lc * 2, 8, tc::kBoxChunks, tc::kBRows)))
            return st;
        tc::TcArgs a{};
        a.N = N;
        a.J = J;
        a.j = j;
        a.lev = lev;
        a.Kp = (int)Kp;
        a.nv = 1 << lev;
        a.nbands = nb;
        a.ntile_n = tc_ntile(Kp);
        a.nlt = (int)(Kp / a.ntile_n);
        a.nkb = (int)(Kj / 64);
        a.kb_per_band = (int)(Kp / 64);
        a.fold = (fold && j == J - 1) ? 1 : 0;
        a.rows_per_ref = rpr;
        a.perm = p->tiles.perm;
        a.tile_ref = p->tiles.tile_ref;
        a.tile_start = p->tiles.tile_start;
        a.tile_count = p->tiles.tile_count;
        a.ntiles = p->tiles.ntiles;
        a.keys = p->keys;
        a.R = r_dev;
        a.err = p->err;
        // short contractions: the received tile stays resident over several variants
        const bool multi = a.nkb <= 2 && a.ntile_n <= 128;
        if (multi && a.fold) {
            set_error("internal: scale J folded into a short-contraction launch");
            return SIDWT_EINVAL;
        }
        const int64_t grid =
            max_pt * a.nlt * (multi ? (a.nv + tc::kMultiVar - 1) / tc::kMultiVar : (int64_t)a.nv);
        if (grid > 0x7fffffff) {
            set_error("batch too large for one tensor-core launch");
            return SIDWT_EINVAL;
        }
        if (multi)
            tc::corr_tc_multi_kernel<<<(unsigned)grid, tc::kThreads, tc::kMSmemBytes, s>>>(mA_hi, mA_lo, mB, a);
        else
            tc::corr_tc_kernel<<<(unsigned)grid, tc::kThreads, tc::kSmemBytes, s>>>(mA_hi, mA_lo, mB, a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "tensor-core correlation launch");
    }
    // scales too short for 64-wide K-blocks run on the CUDA cores
    const uint32_t rest = ((1u << (J + 1)) - 1u) & ~mask;
    if (rest) return correlate_simt(p, B, r_dev, s, rest, tc::kTM);
    return SIDWT_OK;
}

int tc_group_tile() { return tc::kTM; }

cudaError_t prepare_tc_kernels() {
    cudaError_t e =
        cudaFuncSetAttribute(tc::corr_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc::corr_tc_multi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tc::kMSmemBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc::tc_selftest_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 tc::kSelftestSmem);
    return e;
}

int tc_launch_count(const sidwt_plan *p) {
    const uint32_t mask = tc_scale_mask(p);
    const bool pack_refs = p->tc_packed < p->nrefs;
    int n = 0;
    for (int j = 0; j <= p->J; ++j)
        if (mask & (1u << j)) n += pack_refs ? 3 : 2;  // (reference pack) + received pack + correlation
    if (tc_fold_last(p, mask)) n -= 2;                 // scale J: no received pack, no launch of its own
    if (((1u << (p->J + 1)) - 1u) & ~mask) n += 1;
    return n;
}

}  // namespace sidwt

extern "C" sidwt_status sidwt_tc_selftest(float *out_dev, int32_t *err_dev, sidwt_stream stream) {
    using namespace sidwt;
    if (!out_dev || !err_dev) {
        set_error("out_dev and err_dev must not be NULL");
        return SIDWT_EINVAL;
    }
    sidwt_status st = prepare_kernels();
    if (st) return st;
    const int stall = (debug_stall_flags() & SIDWT_STALL_TC_SELFTEST) ? 1 : 0;
    tc::tc_selftest_kernel<<<1, 128, tc::kSelftestSmem, reinterpret_cast<cudaStream_t>(stream)>>>(out_dev, err_dev,
                                                                                                 stall);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "self-test launch");
}
