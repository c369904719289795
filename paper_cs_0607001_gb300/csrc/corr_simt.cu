// Per-scale all-lag correlation on the CUDA cores (the "plain" FP32 path),
// the grouping of a batch by reference, and the peak epilogue.
//
// For scale j < J the stored signal enters through its level-(j+1) SIDWT
// bands: lag D = 2^(j+1) q + v uses variant v's approximation A_v and detail
// B_v rolled by q (the shift-circulant matrices of eq. 6 / 20), so
//   r_j[D] = sum_k conj(A_v[k-q]) c_{j+1}[k] + conj(B_v[k-q]) d_{j+1}[k];
// scale J uses the level-J approximations only (eq. 20a).
//
// A CTA owns one (scale, variant, block of TQ consecutive q) and TP pulses of
// one reference.  Per K-step it stages TP x TK received coefficients and the
// TQ + TK - 1 samples of the variant's window in shared memory.  Each thread
// keeps an MP x MQ block of complex accumulators and slides an MQ-sample
// register window along k (one new shared load per k), so every k costs MP
// received loads and one window load for 4 MP MQ FMAs.
#include <algorithm>

#include "sidwt_internal.cuh"

namespace sidwt {

namespace {

constexpr int TP = 64, TQ = 128, TK = 32, MP = 4, MQ = 8;
constexpr int kThreads = (TP / MP) * (TQ / MQ);  // 256
static_assert(kThreads == 256, "thread layout");
constexpr int kMaxScales = 16;

struct ScaleTab {
    int nscales;                         // entries (a subset of the scales 0..J)
    int scale[kMaxScales];               // scale j of entry e
    int64_t tile_begin[kMaxScales + 1];  // prefix over (variant, q-tile) blocks per entry
    int qtiles[kMaxScales];
    int nsub;                            // pulse sub-tiles of TP per grouping tile
};

__device__ __forceinline__ int wsidx(int t) { return t + (t >> 3); }  // pad 1 per 8: conflict-free window reads

__global__ void __launch_bounds__(kThreads, 2)
    corr_simt_kernel(const float2 *__restrict__ pyr, int64_t pyr_elems, const float2 *__restrict__ tree,
                     int64_t tree_elems, int64_t N, int J, const int32_t *__restrict__ perm,
                     const int32_t *__restrict__ tile_ref, const int32_t *__restrict__ tile_start,
                     const int32_t *__restrict__ tile_count, const int32_t *__restrict__ ntiles, ScaleTab tab,
                     unsigned long long *__restrict__ keys, float2 *__restrict__ R) {
    __shared__ float2 ys[TP][TK + 1];
    __shared__ float2 ws[(TQ + TK) + (TQ + TK) / 8 + 1];
    __shared__ int64_t rowoff[TP];

    const int pt = blockIdx.y / tab.nsub;
    const int sub = blockIdx.y % tab.nsub;
    if (pt >= *ntiles) return;
    const int64_t bx = blockIdx.x;
    int e = 0;
    while (e + 1 < tab.nscales && bx >= tab.tile_begin[e + 1]) ++e;
    const int j = tab.scale[e];
    const int64_t local = bx - tab.tile_begin[e];
    const int qt = (int)(local % tab.qtiles[e]);
    const int var = (int)(local / tab.qtiles[e]);
    const int lev = j < J ? j + 1 : J;
    const int64_t Kp = N >> lev;
    const int nbands = j < J ? 2 : 1;
    const int64_t q0 = (int64_t)qt * TQ;

    const int ref = tile_ref[pt];
    const int start = tile_start[pt] + sub * TP;
    const int cnt = min(TP, tile_count[pt] - sub * TP);
    if (cnt <= 0) return;
    const float2 *Aband = tree + (int64_t)ref * tree_elems + 2 * N * (int64_t)(lev - 1) + (int64_t)var * Kp;
    const int64_t off_c = 2 * N - 4 * Kp;

    const int tid = threadIdx.x;
    const int tq = tid & 15, tp = tid >> 4;
    if (tid < TP) rowoff[tid] = tid < cnt ? (int64_t)perm[start + tid] * pyr_elems : -1;

    float2 acc[MP][MQ];
#pragma unroll
    for (int i = 0; i < MP; ++i)
#pragma unroll
        for (int l = 0; l < MQ; ++l) acc[i][l] = make_float2(0.f, 0.f);

    const int base = TQ - 1 - tq * MQ;
    for (int band = 0; band < nbands; ++band) {
        const float2 *w = band ? Aband + N : Aband;
        const int64_t yoff = off_c + band * Kp;
        for (int64_t k0 = 0; k0 < Kp; k0 += TK) {
            __syncthreads();
            for (int e = tid; e < TP * TK; e += kThreads) {
                const int i = e / TK, kk = e % TK;
                const int64_t ro = rowoff[i];
                float2 v = make_float2(0.f, 0.f);
                if (ro >= 0 && k0 + kk < Kp) v = pyr[ro + yoff + k0 + kk];
                ys[i][kk] = v;
            }
            for (int t = tid; t < TQ + TK - 1; t += kThreads) {
                int64_t u = (k0 - q0 - (TQ - 1) + t) % Kp;
                if (u < 0) u += Kp;
                ws[wsidx(t)] = w[u];
            }
            __syncthreads();
            float2 wv[MQ];
#pragma unroll
            for (int l = 0; l < MQ; ++l) wv[l] = ws[wsidx(base - l)];
#pragma unroll 8
            for (int kk = 0; kk < TK; ++kk) {
                if (kk > 0) {
#pragma unroll
                    for (int l = MQ - 1; l > 0; --l) wv[l] = wv[l - 1];
                    wv[0] = ws[wsidx(base + kk)];
                }
#pragma unroll
                for (int i = 0; i < MP; ++i) {
                    const float2 yv = ys[tp * MP + i][kk];
#pragma unroll
                    for (int l = 0; l < MQ; ++l) {
                        // conj(w) * y
                        acc[i][l].x = fmaf(wv[l].x, yv.x, fmaf(wv[l].y, yv.y, acc[i][l].x));
                        acc[i][l].y = fmaf(wv[l].x, yv.y, fmaf(-wv[l].y, yv.x, acc[i][l].y));
                    }
                }
            }
        }
    }

    // epilogue: optional full output, per-pulse peak over this CTA's lags
#pragma unroll
    for (int i = 0; i < MP; ++i) {
        const int pl = tp * MP + i;
        const bool valid = pl < cnt;
        const int64_t b = valid ? perm[start + pl] : 0;
        unsigned long long best = 0ull;
#pragma unroll
        for (int l = 0; l < MQ; ++l) {
            const int64_t q = q0 + tq * MQ + l;
            if (valid && q < Kp) {
                const int64_t D = (q << lev) + var;
                const float m2 = acc[i][l].x * acc[i][l].x + acc[i][l].y * acc[i][l].y;
                const unsigned long long key =
                    ((unsigned long long)__float_as_uint(m2) << 32) | (unsigned long long)(0xFFFFFFFFu - (uint32_t)D);
                best = key > best ? key : best;
                if (R) R[(b * (J + 1) + j) * N + D] = acc[i][l];
            }
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
            best = other > best ? other : best;
        }
        if (valid && tq == 0 && best) atomicMax(&keys[b * (J + 1) + j], best);
    }
}

// Groups the batch by reference: perm lists pulse indices reference by
// reference; every pulse tile holds up to tile_pulses pulses of one reference.
// Pulses with an out-of-range id are left out and recorded in *err.
constexpr int kGroupSmemRefs = 4096;  // references whose cursors the stable placement keeps in shared memory

__global__ void __launch_bounds__(1024) group_kernel(const int32_t *__restrict__ ref_ids, int B, int nrefs, int TPp,
                                                     int32_t *__restrict__ cursor, int32_t *__restrict__ perm,
                                                     const int32_t *__restrict__ perm_old,
                                                     int32_t *__restrict__ tile_ref, int32_t *__restrict__ tile_start,
                                                     int32_t *__restrict__ tile_count, int32_t *__restrict__ ntiles,
                                                     int32_t *__restrict__ saved, int32_t *__restrict__ err) {
    __shared__ int wsum_c[32], wsum_t[32];
    __shared__ int carry_c, carry_t, old_nvalid, changed;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int r = tid; r < nrefs; r += blockDim.x) cursor[r] = 0;
    if (tid == 0) {
        carry_c = 0;
        carry_t = 0;
        old_nvalid = ntiles[1];
        changed = 0;
    }
    __syncthreads();
    for (int b = tid; b < B; b += blockDim.x) {
        const int r = ref_ids[b];
        saved[b] = r;
        if (r >= 0 && r < nrefs) atomicAdd(&cursor[r], 1);
        else atomicOr(err, kErrBadRefId);
    }
    __syncthreads();
    for (int base = 0; base < nrefs; base += blockDim.x) {
        const int r = base + tid;
        const int c = r < nrefs ? cursor[r] : 0;
        const int t = (c + TPp - 1) / TPp;
        int ic = c, it = t;  // inclusive warp scans
        for (int o = 1; o < 32; o <<= 1) {
            const int vc = __shfl_up_sync(0xffffffffu, ic, o), vt = __shfl_up_sync(0xffffffffu, it, o);
            if (lane >= o) {
                ic += vc;
                it += vt;
            }
        }
        if (lane == 31) {
            wsum_c[wid] = ic;
            wsum_t[wid] = it;
        }
        __syncthreads();
        if (wid == 0) {
            int sc = lane < (int)(blockDim.x >> 5) ? wsum_c[lane] : 0;
            int st = lane < (int)(blockDim.x >> 5) ? wsum_t[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                const int vc = __shfl_up_sync(0xffffffffu, sc, o), vt = __shfl_up_sync(0xffffffffu, st, o);
                if (lane >= o) {
                    sc += vc;
                    st += vt;
                }
            }
            wsum_c[lane] = sc;
            wsum_t[lane] = st;
        }
        __syncthreads();
        const int pc = (wid ? wsum_c[wid - 1] : 0) + ic - c;  // exclusive
        const int ptl = (wid ? wsum_t[wid - 1] : 0) + it - t;
        const int gs = carry_c + pc, ts = carry_t + ptl;
        if (r < nrefs) {
            cursor[r] = gs;
            for (int i = 0; i < t; ++i) {
                tile_ref[ts + i] = r;
                tile_start[ts + i] = gs + i * TPp;
                tile_count[ts + i] = min(TPp, c - i * TPp);
            }
        }
        __syncthreads();
        if (tid == blockDim.x - 1) {
            carry_c = gs + c;
            carry_t = ts + t;
        }
        __syncthreads();
    }
    if (tid == 0) {
        ntiles[0] = carry_t;
        ntiles[1] = carry_c;  // pulses with a valid reference id
    }
    // stable grouping: a reference's pulses in increasing b.  Chunk by chunk
    // and warp by warp in order, the lanes that share a reference take
    // consecutive places from its cursor (the last of them advances it), the
    // cursors in shared memory when the references fit.  The result is the
    // same in every call with the same ids.
    __shared__ int scur[kGroupSmemRefs];
    int *cur = nrefs <= kGroupSmemRefs ? scur : cursor;
    if (nrefs <= kGroupSmemRefs)
        for (int r = tid; r < nrefs; r += blockDim.x) scur[r] = cursor[r];
    __syncthreads();
    const int nw = (int)(blockDim.x >> 5);
    for (int base = 0; base < B; base += blockDim.x) {
        const int b = base + tid;
        const int r = b < B ? ref_ids[b] : -1;
        const bool ok = r >= 0 && r < nrefs;
        const unsigned peers = __match_any_sync(0xffffffffu, ok ? r : -1);
        const int before = __popc(peers & ((1u << lane) - 1u));
        for (int w = 0; w < nw; ++w) {
            if (wid == w && ok) {
                const int pos = cur[r] + before;
                __syncwarp(peers);  // every lane of the group has read the cursor
                perm[pos] = b;
                if (before == __popc(peers) - 1) cur[r] = pos + 1;
            }
            __syncthreads();
        }
    }
    // ntiles[2]: whether the grouping (or the count of valid pulses) changed
    // since the previous call (perm_old: its order; none: assume it did), so
    // that an unchanged received operand need not be packed again
    if (!perm_old) changed = 1;
    else
        for (int i = tid; i < carry_c; i += blockDim.x)
            if (perm[i] != perm_old[i]) changed = 1;
    __syncthreads();
    if (tid == 0) ntiles[2] = (changed || old_nvalid != carry_c) ? 1 : 0;
}

// Reads each peak key once and resets it to zero, so that the next call on
// the plan starts from cleared keys without a separate memset.
__global__ void finalize_kernel(unsigned long long *__restrict__ keys, const int32_t *__restrict__ ids,
                                int nrefs, const double *__restrict__ xen, int64_t xen_len,
                                const double *__restrict__ yen, int64_t B, int J, int32_t *__restrict__ lag,
                                float *__restrict__ mag, double *__restrict__ norm,
                                const int32_t *__restrict__ fail) {
    pdl_wait();  // the correlation kernel's keys
    pdl_release();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * (J + 1)) return;
    finalize_entry(i, keys, ids, nrefs, xen, xen_len, yen, J, lag, mag, norm, fail);
}

}  // namespace

sidwt_status group_pulses(sidwt_plan *p, const int32_t *ref_ids_dev, int64_t B, int tile_pulses, cudaStream_t s) {
    // the two order buffers swap: this call's order beside the previous one's
    if (p->tiles.perm_prev) std::swap(p->tiles.perm, p->tiles.perm_prev);
    group_kernel<<<1, 1024, 0, s>>>(ref_ids_dev, (int)B, p->nrefs, tile_pulses, p->tiles.cursor, p->tiles.perm,
                                    p->tiles.perm_prev,
                                    p->tiles.tile_ref, p->tiles.tile_start, p->tiles.tile_count, p->tiles.ntiles,
                                    p->ref_ids, p->err);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "group launch");
}

sidwt_status correlate_simt(sidwt_plan *p, int64_t B, float2 *r_dev, cudaStream_t s, uint32_t scale_mask,
                            int group_tile) {
    const int64_t N = p->N;
    const int J = p->J;
    ScaleTab tab{};
    int64_t acc = 0;
    int ne = 0;
    for (int j = 0; j <= J; ++j) {
        if (!(scale_mask & (1u << j))) continue;
        const int lev = j < J ? j + 1 : J;
        const int64_t Kp = N >> lev;
        tab.scale[ne] = j;
        tab.qtiles[ne] = (int)((Kp + TQ - 1) / TQ);
        tab.tile_begin[ne] = acc;
        acc += (int64_t)tab.qtiles[ne] << lev;
        ++ne;
    }
    if (ne == 0) return SIDWT_OK;
    tab.nscales = ne;
    tab.tile_begin[ne] = acc;
    tab.nsub = (group_tile + TP - 1) / TP;
    const int64_t max_pt = (B + group_tile - 1) / group_tile + std::min<int64_t>(p->nrefs, B);
    if (acc > 0x7fffffff || max_pt * tab.nsub > 65535) {
        set_error("batch too large for one launch of the FP32 correlation");
        return SIDWT_EINVAL;
    }
    dim3 grid((unsigned)acc, (unsigned)(max_pt * tab.nsub));
    corr_simt_kernel<<<grid, kThreads, 0, s>>>(p->pyr_f, p->pyr_elems, p->tree_f, p->tree_elems, N, J,
                                               p->tiles.perm, p->tiles.tile_ref, p->tiles.tile_start,
                                               p->tiles.tile_count, p->tiles.ntiles, tab, p->keys, r_dev);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "FP32 correlation launch");
}

sidwt_status finalize_peaks(sidwt_plan *p, int64_t B, cudaStream_t s, bool invalidate_on_error) {
    const int64_t n = B * (p->J + 1);
    if (n == 0) return SIDWT_OK;
    cudaError_t e = launch_dependent(finalize_kernel, dim3((unsigned)((n + 255) / 256)), dim3(256), 0, s, p->keys,
                                     (const int32_t *)p->ref_ids, p->nrefs, (const double *)p->xen, p->xen_len,
                                     (const double *)p->yen, B, p->J, p->lag, p->mag, p->norm,
                                     (const int32_t *)(invalidate_on_error ? p->err : nullptr));
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "peak epilogue launch");
}

namespace {
__global__ void copy_peaks_kernel(const int32_t *__restrict__ lag, const float *__restrict__ mag,
                                  const double *__restrict__ norm, int64_t n, int32_t *__restrict__ lag_out,
                                  float *__restrict__ mag_out, double *__restrict__ norm_out) {
    pdl_wait();  // the peak epilogue's outputs
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (lag_out) lag_out[i] = lag[i];
        if (mag_out) mag_out[i] = mag[i];
        if (norm_out) norm_out[i] = norm[i];
    }
}
}  // namespace

sidwt_status copy_peaks(const sidwt_plan *p, int64_t n, int32_t *lag, float *mag, double *norm, cudaStream_t s) {
    if (n == 0 || (!lag && !mag && !norm)) return SIDWT_OK;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    cudaError_t e = launch_dependent(copy_peaks_kernel, dim3((unsigned)blocks), dim3(256), 0, s,
                                     (const int32_t *)p->lag, (const float *)p->mag, (const double *)p->norm, n, lag,
                                     mag, norm);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? SIDWT_OK : cuda_fail(e, "peak copy");
}

int simt_tile_pulses() { return TP; }

}  // namespace sidwt
