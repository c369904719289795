// sidwt_correlate_static: the correlation of a batch against one stored
// signal without any device allocation.  Every intermediate (the stored
// signal's SIDWT tree, the received pyramid, energies, peak keys, the tile
// list) lives in one file-scope device array of fixed size; the caller passes
// only inputs and outputs.  The same kernels as sidwt_correlate run on it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "sidwt_internal.cuh"

using namespace sidwt;

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB, held by every GPU that loads the library
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_addr_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The symbol's
// host-side name is only a stand-in, so the address is looked up once per
// device (with that device current) and cached.  A device reset
// (cudaDeviceReset) or a new primary context leaves the cached address stale:
// calls after one would write to memory that no longer exists.
sidwt_status scratch_address(unsigned char **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal out of range for the static scratch table");
        return SIDWT_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static scratch");
        g_addr[dev] = ptr;
    }
    *out = static_cast<unsigned char *>(g_addr[dev]);
    return SIDWT_OK;
}

struct Carve {
    unsigned char *base;
    size_t off = 0;
    template <typename T>
    T *take(size_t count) {
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += ((count * sizeof(T) + 255) / 256) * 256;
        return p;
    }
};

// Lays out every buffer of one call in the scratch (base == nullptr only
// measures).  Returns the bytes needed.
size_t layout(sidwt_plan &p, unsigned char *base, int64_t B, int32_t **ids_in) {
    Carve c{base};
    p.tree_f = c.take<float2>((size_t)p.tree_elems);
    p.tree_i = p.is_int ? c.take<int2>((size_t)p.tree_elems) : nullptr;
    p.xen = c.take<double>((size_t)p.xen_len);
    p.pyr_f = c.take<float2>((size_t)(B * p.pyr_elems));
    p.pyr_i = p.is_int ? c.take<int2>((size_t)(B * p.pyr_elems)) : nullptr;
    p.yen = c.take<double>((size_t)(B * (p.J + 1)));
    p.keys = c.take<unsigned long long>((size_t)(B * (p.J + 1)));
    *ids_in = c.take<int32_t>((size_t)B);
    p.ref_ids = c.take<int32_t>((size_t)B);
    p.tiles.perm = c.take<int32_t>((size_t)B);
    p.tiles.max_tiles = (B + simt_tile_pulses() - 1) / simt_tile_pulses() + 1;
    p.tiles.tile_ref = c.take<int32_t>((size_t)p.tiles.max_tiles);
    p.tiles.tile_start = c.take<int32_t>((size_t)p.tiles.max_tiles);
    p.tiles.tile_count = c.take<int32_t>((size_t)p.tiles.max_tiles);
    p.tiles.ntiles = c.take<int32_t>(3);
    p.tiles.cursor = c.take<int32_t>(1);
    p.err = c.take<int32_t>(1);
    return c.off;
}

}  // namespace

extern "C" sidwt_status sidwt_correlate_static(sidwt_filter f, int64_t N, int J, const void *x_dev,
                                               const void *y_dev, int64_t B, int32_t *lag_dev, float *mag_dev,
                                               double *norm_dev, sidwt_stream stream) {
    if ((int)f < 0 || (int)f > 4) {
        set_error("unknown filter");
        return SIDWT_EINVAL;
    }
    if (J < 1 || J > 15 || N < 2 || N > (int64_t(1) << 26) || N % (int64_t(1) << J) != 0) {
        set_error("need 1 <= J <= 15, N a multiple of 2^J, N <= 2^26");
        return SIDWT_EINVAL;
    }
    if (B < 1 || B > 65535 || !x_dev || !y_dev || !lag_dev || !mag_dev || !norm_dev) {
        set_error("need 1 <= B <= 65535 and non-NULL x, y, lag, mag and norm");
        return SIDWT_EINVAL;
    }
    const bool is_int = (f == SIDWT_LEGALL53_INT || f == SIDWT_CDF97_INT);
    if (reinterpret_cast<uintptr_t>(x_dev) % (is_int ? 4 : 8) ||
        reinterpret_cast<uintptr_t>(y_dev) % (is_int ? 8 : 16)) {
        set_error("x_dev / y_dev misaligned");
        return SIDWT_EINVAL;
    }
    sidwt_plan p;  // describes the scratch; owns nothing
    p.filter = (int)f;
    p.N = N;
    p.J = J;
    p.is_int = is_int;
    p.tree_elems = 2 * (int64_t)J * N;
    p.xen_len = (int64_t(2) << J) - 1;
    p.pyr_elems = 2 * N - 2 * (N >> J);
    int32_t *ids_in = nullptr;
    const size_t need = layout(p, nullptr, B, &ids_in);
    if (need > kStaticScratchBytes) {
        set_error("sidwt_correlate_static: this call needs " + std::to_string(need) + " bytes of scratch, more than the " +
                  std::to_string(kStaticScratchBytes) + "-byte static array; use sidwt_correlate or a smaller batch");
        return SIDWT_EINVAL;
    }
    sidwt_status st = prepare_kernels();
    if (st) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *base = nullptr;
    st = scratch_address(&base);
    if (st) return st;
    layout(p, base, B, &ids_in);
    p.nrefs = 1;
    p.cap_refs = 1;
    p.cap_batch = B;
    p.lag = lag_dev;
    p.mag = mag_dev;
    p.norm = norm_dev;
    p.last_B = B;
    // the array keeps the previous call's contents: zero what must start at zero
    cudaError_t e = cudaMemsetAsync(ids_in, 0, (size_t)B * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.keys, 0, (size_t)B * (J + 1) * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.err, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return cuda_fail(e, "scratch clear");
    if ((st = build_reference_tree(&p, x_dev, 0, s))) return st;
    if ((st = group_pulses(&p, ids_in, B, simt_tile_pulses(), s))) return st;
    if ((st = analyze_batch(&p, y_dev, B, s))) return st;
    if ((st = correlate_simt(&p, B, nullptr, s))) return st;
    // no sidwt_check reaches this scratch: a recorded error (the analysis gave
    // up on a bounded wait) turns every record of the call into "no peak"
    return finalize_peaks(&p, B, s, true);
}
