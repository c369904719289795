// Per-scale all-lag correlation on the tcgen05 tensor cores with a 3xTF32
// split (a = a_hi + a_lo, both rounded to TF32; products hi*hi + hi*lo +
// lo*hi, FP32 accumulation in TMEM): FP32-grade accuracy at tensor-core
// speed.
//
// Same products as the bf16 path (eq. 20 / 20a in advance form,
// C[p][m] = sum_k conj(w[(k + p) mod K']) u_m[k]) with the roles of the
// operands exchanged and only K-major layouts:
//   * A (M = 128 rows) is the stored variant's window: row i is the advance
//     p = p0 + r + 4 i, so with a copy W_r[t] = w[t + r] shifted by the
//     residue r, element (i, k) sits at W_r[t0 + 4 i + k]: consecutive rows
//     are 16 bytes apart and the K-major core matrices overlap (LBO 16 B,
//     SBO 128 B).  One CTA owns one residue r and 128 advances spaced by 4
//     (512 consecutive advances per r-quadruple of CTAs).
//     Bands shorter than 512 put G variants in one tile instead: variant g's
//     window (K'/4 + 4 chunks) starts at row g (K'/4 + 4) of the same
//     overlapping layout, so rows g (K'/4 + 4) + i, i < K'/4, are its advances
//     r + 4 i and the 4 rows between windows are discarded.
//   * B (N = 256 columns) is 256 received pulses of one reference, K-major
//     in the 64-byte swizzled layout ([k/16][Re|Im][pulse][16 samples]: one
//     64-byte row per pulse and plane), so the TMA box moves 64-byte rows
//     rather than 16-byte core-matrix rows.
// Re and Im: Re += A(wr) B(ur) + A(wi) B(ui), Im += A(wr) B(ui) + A(-wi) B(ur);
// each with the three split products: 24 MMAs (M 128, N 256, K 8) per stage
// of 16 samples.  The epilogue reduces the peak of every pulse over the
// CTA's advances with a warp transpose-reduction and one atomicMax per
// (warp, pulse).  Roles and bounded waits as in the bf16 kernel.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "tc_common.cuh"

namespace sidwt {
namespace tc32 {

using namespace sidwt::tc;

constexpr int kThreads = 192;
constexpr int kTN = 256;                        // pulses per tile (MMA N)
constexpr int kKB = 16;                         // samples per stage
constexpr int kLagBlock = 512;                  // advances per (r-quadruple of) CTA
constexpr int kWinChunks = 132;                 // window chunks of 4 samples: 4*127 + 15 < 528
constexpr int kWinRowBytes = kWinChunks * 16;   // 2112
constexpr int kARows = 3;                       // planes -Im, Re, Im of one residue
constexpr int kABytes = 6528;                   // 3 planes x 2176 B (2112 B rounded up to 128)
constexpr int kBBytes = 2 * kTN * 64;           // [Re|Im][256 pulses][64 B, swizzled] = 32768
constexpr int kStage = (2 * kBBytes + 2 * kABytes + 1023) / 1024 * 1024;  // B hi, B lo, A hi, A lo: 78848
static_assert(kARows * ((kWinRowBytes + 127) / 128 * 128) <= kABytes, "three plane windows per hi/lo region");
static_assert(kStage % 1024 == 0 && kBBytes % 1024 == 0 && kABytes % 128 == 0,
              "TMA destinations 128-byte aligned, swizzled B planes on 1024-byte boundaries");
constexpr int kBarOff = 2 * kStage;             // 157696
constexpr int kSmemBytes = kBarOff + 128 + 1024;
constexpr int kTmemCols = 512;
constexpr int kRowsPerVariant = 24;             // hi/lo x 4 residues x 3 planes

// Instruction descriptor, kind::tf32: D f32, A and B tf32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d),
        "l"(a), "l"(b), "r"(idesc), "r"(accum)
        : "memory");
}

// Round to TF32 (nearest, ties away from zero): the hi part, then the lo part
// of the remainder.
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}

struct Args {
    int64_t N;
    int J, j, lev;
    int Kp, nv, nbands, nlb;  // band length, variants, bands, 512-advance blocks per variant
    int kb_per_band;          // K' / 16
    int rows_per_ref;
    int G, cg, nvg;           // variants per tile, window chunks per variant, variant groups
    const int32_t *perm;
    const int32_t *tile_ref;
    const int32_t *tile_start;
    const int32_t *tile_count;
    const int32_t *ntiles;
    unsigned long long *keys;
    float2 *R;
    int32_t *err;
};

__device__ __forceinline__ unsigned long long kmax(unsigned long long a, unsigned long long b) { return a > b ? a : b; }

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1, int c2,
                                            int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(saddr(bar))
        : "memory");
}

__global__ void __launch_bounds__(kThreads, 1)
    corr_tc32_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB_hi,
                     const __grid_constant__ CUtensorMap mapB_lo, const Args a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + kBarOff);  // full[2], empty[2], accf
    uint64_t *full = bar, *empty = bar + 2, *accf = bar + 4;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + 8);
    volatile int *sflag = reinterpret_cast<volatile int *>(tmem_slot + 4);  // [0] error, [1] issued, [2] consumed, [3] progress

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bx = blockIdx.x;
    const int lb = bx % a.nlb;
    const int r = (bx / a.nlb) & 3;
    const int v0 = ((bx / (a.nlb * 4)) % a.nvg) * a.G;  // first variant of the tile
    const int pt = bx / (a.nlb * 4 * a.nvg);
    // one plane's windows: G * cg chunks, the plane regions 128-byte aligned (TMA destinations)
    const uint32_t box_bytes = (uint32_t)(a.G * a.cg * 16);
    const uint32_t pitch = (box_bytes + 127u) & ~127u;
    if (pt >= a.ntiles[0]) return;  // uniform: before any barrier or TMEM use
    const int row0 = a.tile_start[pt];
    const int cnt = a.tile_count[pt];
    const int ref = a.tile_ref[pt];
    const int p0 = lb * kLagBlock;
    const int nkb = a.nbands * a.kb_per_band;

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(accf, 1);
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
            int issued = 0;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb & 1;
                if (kb >= 2 && !mbar_wait(&empty[s], ((kb >> 1) - 1) & 1)) {
                    sflag[0] = 1;
                    break;
                }
                if (sflag[0]) break;
                const int band = kb / a.kb_per_band;
                const int kap0 = (kb % a.kb_per_band) * kKB;
                unsigned char *st = base + s * kStage;
                mbar_expect_tx(&full[s], 2 * kBBytes + 2 * kARows * box_bytes);
                const int z0 = ((band * a.Kp + kap0) >> 4) * 2;
                tma_load_3d(st, &mapB_hi, &full[s], 0, row0, z0);
                tma_load_3d(st + kBBytes, &mapB_lo, &full[s], 0, row0, z0);
                // A: per (hi/lo, plane) the windows of the tile's G variants, back to back
                const int vblock = ref * (a.rows_per_ref / kRowsPerVariant) + band * a.nv + v0;
                const int chunk0 = (kap0 + p0) >> 2;
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int q = 0; q < kARows; ++q)
                        tma_load_4d(st + 2 * kBBytes + h * kABytes + q * pitch, &mapA, &full[s], 0, chunk0,
                                    h * 12 + r * kARows + q, vblock);
                ++issued;
            }
            sflag[1] = issued;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(128, kTN);
            int consumed = 0;
            for (int kb = 0; kb < nkb; ++kb) {
                const int s = kb & 1;
                if (!mbar_wait(&full[s], (kb >> 1) & 1)) {
                    sflag[0] = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t sb = saddr(base + s * kStage);
                const uint32_t bHi = sb, bLo = sb + kBBytes;
                const uint32_t aHi = sb + 2 * kBBytes, aLo = aHi + kABytes;
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    // A rows: 0 -Im w, 1 Re w, 2 Im w; K-direction 16 B (next 4 samples), 8 advances 128 B
                    const uint32_t ao = (uint32_t)ks * 32;
                    const uint64_t ah[3] = {sdesc(aHi + ao, 16, 128), sdesc(aHi + pitch + ao, 16, 128),
                                            sdesc(aHi + 2 * pitch + ao, 16, 128)};
                    const uint64_t al[3] = {sdesc(aLo + ao, 16, 128), sdesc(aLo + pitch + ao, 16, 128),
                                            sdesc(aLo + 2 * pitch + ao, 16, 128)};
                    // B planes Re u / Im u: [plane][256 pulses][64 B swizzled], 16 KB apart; the K half
                    // ks is the row's second 32 bytes; 8 pulses 512 B
                    const uint32_t bo = (uint32_t)ks * 32;
                    const uint64_t bh[2] = {sdesc_sw64(bHi + bo, 512), sdesc_sw64(bHi + kTN * 64 + bo, 512)};
                    const uint64_t bl[2] = {sdesc_sw64(bLo + bo, 512), sdesc_sw64(bLo + kTN * 64 + bo, 512)};
                    // (accumulator, A row, B plane): Re += wr ur + wi ui, Im += wr ui + (-wi) ur
                    const int acc_of[4] = {0, 0, 1, 1}, arow[4] = {1, 2, 1, 0}, bpl[4] = {0, 1, 1, 0};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint32_t d = tmem + acc_of[q] * 256;
                        const uint32_t first = (kb == 0 && ks == 0 && (q == 0 || q == 2)) ? 0u : 1u;
                        mma_tf32(d, ah[arow[q]], bh[bpl[q]], idesc, first);
                        mma_tf32(d, ah[arow[q]], bl[bpl[q]], idesc, 1u);
                        mma_tf32(d, al[arow[q]], bh[bpl[q]], idesc, 1u);
                    }
                }
                mma_commit(&empty[s]);
                ++consumed;
                sflag[3] = consumed;
            }
            sflag[2] = consumed;
            mma_commit(accf);  // arrives once every MMA issued above has completed
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = advances m
        const int q4 = warp & 3;
        const int m = q4 * 32 + lane;
        uint64_t t0 = now_ns();
        int last = sflag[3];
        bool ok = true;
        while (!mbar_test(accf, 0)) {  // bounded from the MMA thread's last progress
            const int pr = sflag[3];
            if (pr != last) {
                last = pr;
                t0 = now_ns();
            } else if (now_ns() - t0 > kWaitNs) {
                ok = false;
                break;
            }
        }
        tc_fence_after();
        if (!__all_sync(0xffffffffu, ok && !sflag[0])) {
            sflag[0] = 1;
        } else {
            // row m: variant v0 + g, advance p0 + r + 4 i (rows between windows are discarded)
            const int g = m / a.cg, i = m - g * a.cg;
            const bool valid = g < a.G && v0 + g < a.nv && p0 + r + 4 * i < a.Kp;
            const int p = p0 + r + 4 * i;
            const int pm = p % a.Kp;
            const int q = pm == 0 ? 0 : a.Kp - pm;
            const uint32_t D = ((uint32_t)q << a.lev) + (uint32_t)(v0 + g);
            const uint32_t tl = tmem + ((uint32_t)(q4 * 32) << 16);
            for (int c0 = 0; c0 < kTN; c0 += 32) {
                uint32_t re[32], im[32];
                TMEM_LD32(tl + c0, re);
                TMEM_LD32(tl + 256 + c0, im);
                tmem_wait_ld();
                unsigned long long key[32];
#pragma unroll
                for (int n = 0; n < 32; ++n) {
                    const float xr = __uint_as_float(re[n]), xi = __uint_as_float(im[n]);
                    key[n] = valid ? ((unsigned long long)__float_as_uint(xr * xr + xi * xi) << 32) |
                                         (unsigned long long)(0xFFFFFFFFu - D)
                                   : 0ull;
                    if (a.R && valid && c0 + n < cnt) {
                        const int64_t b = a.perm[row0 + c0 + n];
                        a.R[(b * (a.J + 1) + a.j) * a.N + D] = make_float2(xr, xi);
                    }
                }
                // transpose-reduce: afterwards lane i holds the max over the warp's
                // 32 advances for pulse c0 + i
#pragma unroll
                for (int sh = 16; sh >= 1; sh >>= 1) {
                    const bool upper = (lane & sh) != 0;
#pragma unroll
                    for (int i = 0; i < sh; ++i) {
                        const unsigned long long send = upper ? key[i] : key[i + sh];
                        const unsigned long long keep = upper ? key[i + sh] : key[i];
                        key[i] = kmax(keep, __shfl_xor_sync(0xffffffffu, send, sh));
                    }
                }
                if (c0 + lane < cnt && key[0]) {
                    const int64_t b = a.perm[row0 + c0 + lane];
                    atomicMax(&a.keys[b * (a.J + 1) + a.j], key[0]);
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0 && sflag[0]) {
        for (int kb = sflag[2]; kb < sflag[1]; ++kb) mbar_wait(&full[kb & 1], (kb >> 1) & 1);
        atomicOr(a.err, kErrTcWait);
    }
    __syncthreads();
    if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

// Stored windows: row ((ref * nbands + band) * nv + v) * 24 + hilo * 12 + r * 3
// + plane holds Lc TF32 values W[t] = plane(w[(t + r) mod K']) (plane 0: -Im,
// 1: Re, 2: Im), hi or lo part.
__global__ void pack_ref32_kernel(const float2 *__restrict__ tree, int64_t tree_elems, int64_t N, int lev, int nbands,
                                  int ref0, int Lc, uint32_t *__restrict__ out) {
    const int Kp = (int)(N >> lev), nv = 1 << lev;
    const int rows_per_ref = nbands * nv * kRowsPerVariant;
    const int64_t row = (int64_t)blockIdx.x + (int64_t)ref0 * rows_per_ref;
    const int ref = (int)(row / rows_per_ref);
    int rem = (int)(row % rows_per_ref);
    const int plane = rem % 3;
    rem /= 3;
    const int r = rem % 4;
    rem /= 4;
    const int hilo = rem % 2;
    rem /= 2;
    const int vv = rem % nv;
    const int band = rem / nv;
    const float2 *w = tree + (int64_t)ref * tree_elems + 2 * N * (int64_t)(lev - 1) + (int64_t)band * N + (int64_t)vv * Kp;
    uint32_t *o = out + row * Lc;
    for (int t = threadIdx.x; t < Lc; t += blockDim.x) {
        const float2 x = w[(t + r) % Kp];
        const float val = plane == 0 ? -x.y : (plane == 1 ? x.x : x.y);
        uint32_t hi, lo;
        split_tf32(val, hi, lo);
        o[t] = hilo ? lo : hi;
    }
}

// Received operand of one scale: row ((k / 16) * 2 + plane) of 16 TF32 values
// u_plane[16 (k / 16) .. + 15] per pulse (grouped order) of the concatenated
// bands (plane 0 Re, 1 Im), 64 bytes a pulse.  Block: 64 samples x 32 rows.
// same_input: the buffers already hold this pyramid packed for this batch
// size; the packing is skipped when the grouping is unchanged too (ntiles[2]).
__global__ void __launch_bounds__(256) pack_rx32_kernel(const float2 *__restrict__ pyr, int64_t pyr_elems, int64_t off,
                                                        const int32_t *__restrict__ perm,
                                                        const int32_t *__restrict__ ntiles, int rows,
                                                        uint32_t *__restrict__ bhi, uint32_t *__restrict__ blo,
                                                        int same_input) {
    __shared__ float2 tile[32][65];
    if (same_input && ntiles[2] == 0) return;  // uniform over the grid
    const int kb = blockIdx.x;  // 64 samples
    const int r0 = blockIdx.y * 32;
    const int nvalid = ntiles[1];
    for (int e = threadIdx.x; e < 32 * 64; e += 256) {
        const int i = e >> 6, k = e & 63;
        const int r = r0 + i;
        float2 v = make_float2(0.f, 0.f);
        if (r < nvalid) v = pyr[(int64_t)perm[r] * pyr_elems + off + (int64_t)kb * 64 + k];
        tile[i][k] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {  // 16 k-chunks x 2 planes x 32 rows
        const int cp = e >> 5, i = e & 31;
        const int r = r0 + i;
        if (r >= rows) continue;
        const int kc = cp >> 1, plane = cp & 1;  // kc: 4 samples of the block's 64
        uint4 h, l;
        uint32_t *hp = reinterpret_cast<uint32_t *>(&h), *lp = reinterpret_cast<uint32_t *>(&l);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float2 v = tile[i][kc * 4 + q];
            split_tf32(plane ? v.y : v.x, hp[q], lp[q]);
        }
        const int64_t kq = (int64_t)kb * 4 + (kc >> 2);  // 16-sample row index
        const int64_t o = ((kq * 2 + plane) * rows + r) * 16 + (kc & 3) * 4;
        *reinterpret_cast<uint4 *>(bhi + o) = h;
        *reinterpret_cast<uint4 *>(blo + o) = l;
    }
}

}  // namespace tc32

// Scales the 3xTF32 path takes: band length a multiple of 64 (16-sample
// stages and 64-sample packing blocks).
uint32_t tc32_scale_mask(const sidwt_plan *p) {
    uint32_t m = 0;
    for (int j = 0; j <= p->J; ++j) {
        const int lev = j < p->J ? j + 1 : p->J;
        const int64_t Kp = p->N >> lev;
        if (Kp >= 64 && Kp % 64 == 0 && Kp <= (int64_t(1) << 24)) m |= 1u << j;
    }
    return m;
}

static int tc32_lc(int64_t Kp) { return (int)(2 * Kp + 4 * tc32::kWinChunks); }

// Variants per tile for a band of Kp samples: one (rows = 128 advances of a
// 512-advance block) unless Kp < 512; then G windows of Kp/4 + 4 chunks, the
// last window's advances within the 128 rows and all windows within the
// 132-chunk plane.
static void tc32_group(int64_t Kp, int nv, int *G, int *cg) {
    *G = 1;
    *cg = tc32::kWinChunks;
    if (Kp >= tc32::kLagBlock) return;
    const int c = (int)(Kp / 4 + 4);
    int g = 1;
    while ((g + 1) * c <= tc32::kWinChunks && g * c + (int)(Kp / 4) <= 128 && g + 1 <= nv) ++g;
    *G = g;
    *cg = c;
}
static int tc32_rows_per_ref(const sidwt_plan *p, int j) {
    const int lev = j < p->J ? j + 1 : p->J;
    return (j < p->J ? 2 : 1) * (1 << lev) * tc32::kRowsPerVariant;
}

void free_tc32(sidwt_plan *p) {
    for (int j = 0; j < 16; ++j) {
        if (p->tc32_ref[j]) cudaFree(p->tc32_ref[j]);
        if (p->tc32_bhi[j]) cudaFree(p->tc32_bhi[j]);
        if (p->tc32_blo[j]) cudaFree(p->tc32_blo[j]);
        p->tc32_ref[j] = p->tc32_bhi[j] = p->tc32_blo[j] = nullptr;
    }
    p->tc32_cap_refs = 0;
    p->tc32_cap_batch = 0;
    p->tc32_packed = 0;
    p->tc32_rx_gen = -1;
}

static sidwt_status ensure_tc32(sidwt_plan *p) {
    if (p->tc32_cap_refs >= p->cap_refs && p->tc32_cap_batch >= p->cap_batch) return SIDWT_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronise before tensor-core buffers");
    free_tc32(p);
    const uint32_t mask = tc32_scale_mask(p);
    for (int j = 0; j <= p->J; ++j) {
        if (!(mask & (1u << j))) continue;
        const int lev = j < p->J ? j + 1 : p->J;
        const int64_t Kp = p->N >> lev;
        const int64_t Kj = (j < p->J ? 2 : 1) * Kp;
        const size_t rb = (size_t)p->cap_refs * tc32_rows_per_ref(p, j) * tc32_lc(Kp) * 4;
        const size_t bb = (size_t)Kj * 2 * p->cap_batch * 4;
        if (cudaMalloc(&p->tc32_ref[j], rb) != cudaSuccess || cudaMalloc(&p->tc32_bhi[j], bb) != cudaSuccess ||
            cudaMalloc(&p->tc32_blo[j], bb) != cudaSuccess) {
            cudaGetLastError();
            free_tc32(p);
            set_error("device allocation failed for the 3xTF32 operands");
            return SIDWT_ENOMEM;
        }
    }
    p->tc32_cap_refs = p->cap_refs;
    p->tc32_cap_batch = p->cap_batch;
    p->tc32_packed = 0;
    return SIDWT_OK;
}

sidwt_status correlate_tc32(sidwt_plan *p, int64_t B, float2 *r_dev, cudaStream_t s) {
    sidwt_status st = ensure_tc32(p);
    if (st) return st;
    const uint32_t mask = tc32_scale_mask(p);
    const int64_t N = p->N;
    const int J = p->J;
    if (p->tc32_packed < p->nrefs) {
        for (int j = 0; j <= J; ++j) {
            if (!(mask & (1u << j))) continue;
            const int lev = j < J ? j + 1 : J;
            const int nb = j < J ? 2 : 1;
            const int64_t rows = (int64_t)(p->nrefs - p->tc32_packed) * tc32_rows_per_ref(p, j);
            tc32::pack_ref32_kernel<<<(unsigned)rows, 256, 0, s>>>(p->tree_f, p->tree_elems, N, lev, nb, p->tc32_packed,
                                                                  tc32_lc(N >> lev),
                                                                  static_cast<uint32_t *>(p->tc32_ref[j]));
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "reference packing launch");
        p->tc32_packed = p->nrefs;
    }
    const int64_t max_pt = (B + tc32::kTN - 1) / tc32::kTN + std::min<int64_t>(p->nrefs, B);
    // as for BF16x3: an unchanged pyramid and grouping keep their packed operands
    const bool same_input = p->tc32_rx_gen == p->analysis_gen && p->tc32_rx_B == B;
    p->tc32_rx_gen = p->analysis_gen;
    p->tc32_rx_B = B;
    for (int j = 0; j <= J; ++j) {
        if (!(mask & (1u << j))) continue;
        const int lev = j < J ? j + 1 : J;
        const int64_t Kp = N >> lev;
        const int nb = j < J ? 2 : 1;
        const int64_t Kj = nb * Kp;
        uint32_t *bhi = static_cast<uint32_t *>(p->tc32_bhi[j]);
        uint32_t *blo = static_cast<uint32_t *>(p->tc32_blo[j]);
        {
            dim3 g((unsigned)(Kj / 64), (unsigned)((B + 31) / 32));
            tc32::pack_rx32_kernel<<<g, 256, 0, s>>>(p->pyr_f, p->pyr_elems, 2 * N - 4 * Kp, p->tiles.perm,
                                                     p->tiles.ntiles, (int)B, bhi, blo, same_input ? 1 : 0);
        }
        // TF32 data is moved as pairs of 16-bit units: a 64-byte row is 32 units
        CUtensorMap mA, mBh, mBl;
        {
            const uint64_t dims[3] = {32, (uint64_t)B, (uint64_t)Kj / 16 * 2};
            const uint64_t strides[2] = {64, 64 * (uint64_t)B};
            const uint32_t box[3] = {32, tc32::kTN, 2};
            if ((st = tc::encode_nd(&mBh, bhi, 3, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_64B)) ||
                (st = tc::encode_nd(&mBl, blo, 3, dims, strides, box, CU_TENSOR_MAP_SWIZZLE_64B)))
                return st;
        }
        const int Lc = tc32_lc(Kp);
        const int rpr = tc32_rows_per_ref(p, j);
        int G = 1, cg = tc32::kWinChunks;
        tc32_group(Kp, 1 << lev, &G, &cg);
        {
            // [variant block][24 rows: hi/lo, residue, plane][Lc / 4 chunks][16 B]; box: one row of G blocks
            const uint64_t dims[4] = {8, (uint64_t)(Lc / 4), (uint64_t)tc32::kRowsPerVariant,
                                      (uint64_t)p->nrefs * rpr / tc32::kRowsPerVariant};
            const uint64_t strides[3] = {16, (uint64_t)Lc * 4, (uint64_t)Lc * 4 * tc32::kRowsPerVariant};
            const uint32_t box[4] = {8, (uint32_t)cg, 1, (uint32_t)G};
            if ((st = tc::encode_nd(&mA, p->tc32_ref[j], 4, dims, strides, box))) return st;
        }
        tc32::Args a{};
        a.N = N;
        a.J = J;
        a.j = j;
        a.lev = lev;
        a.Kp = (int)Kp;
        a.nv = 1 << lev;
        a.nbands = nb;
        a.nlb = (int)((Kp + tc32::kLagBlock - 1) / tc32::kLagBlock);
        a.kb_per_band = (int)(Kp / tc32::kKB);
        a.rows_per_ref = rpr;
        a.G = G;
        a.cg = cg;
        a.nvg = (a.nv + G - 1) / G;
        a.perm = p->tiles.perm;
        a.tile_ref = p->tiles.tile_ref;
        a.tile_start = p->tiles.tile_start;
        a.tile_count = p->tiles.tile_count;
        a.ntiles = p->tiles.ntiles;
        a.keys = p->keys;
        a.R = r_dev;
        a.err = p->err;
        const int64_t grid = max_pt * a.nvg * 4 * a.nlb;
        if (grid > 0x7fffffff) {
            set_error("batch too large for one tensor-core launch");
            return SIDWT_EINVAL;
        }
        tc32::corr_tc32_kernel<<<(unsigned)grid, tc32::kThreads, tc32::kSmemBytes, s>>>(mA, mBh, mBl, a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "3xTF32 correlation launch");
    }
    const uint32_t rest = ((1u << (J + 1)) - 1u) & ~mask;
    if (rest) return correlate_simt(p, B, r_dev, s, rest, tc32::kTN);
    return SIDWT_OK;
}

int tc32_group_tile() { return tc32::kTN; }

int tc32_launch_count(const sidwt_plan *p) {
    const uint32_t mask = tc32_scale_mask(p);
    const bool pack_refs = p->tc32_packed < p->nrefs;
    int n = 0;
    for (int j = 0; j <= p->J; ++j)
        if (mask & (1u << j)) n += pack_refs ? 3 : 2;
    if (((1u << (p->J + 1)) - 1u) & ~mask) n += 1;
    return n;
}

cudaError_t prepare_tc32_kernels() {
    return cudaFuncSetAttribute(tc32::corr_tc32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, tc32::kSmemBytes);
}

}  // namespace sidwt
