// Device-wide scans, reductions and a stable LSD radix sort.
//
// These are the building blocks of the degree ranking (Definition 3 via the
// bin sort named in the proof of Theorem 2), the renumbering of Definition 4
// and the per-start work prefix sums.
#include <climits>

#include "bfc_internal.cuh"

namespace bfc {

namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;     // 4096 elements per block

constexpr int kSortThreads = 256;                         // 8 warps
constexpr int kSortItems = 8;                             // per thread
constexpr int kSortTile = kSortThreads * kSortItems;      // 2048 keys per tile
constexpr int kSortWarpSpan = kSortTile / (kSortThreads / 32);  // 256 consecutive keys per warp

struct OpSum {
    template <typename T>
    __device__ static T apply(T a, T b) { return a + b; }
    template <typename T>
    __device__ static T identity() { return T(0); }
};
struct OpMax {
    template <typename T>
    __device__ static T apply(T a, T b) { return a > b ? a : b; }
    template <typename T>
    __device__ static T identity() { return T(INT_MIN); }
};

template <typename T>
__device__ __forceinline__ T shfl_up(T v, int d) {
    return __shfl_up_sync(0xffffffffu, v, d);
}

// Inclusive scan of one value per thread across the block.  Returns the
// inclusive prefix of this thread; *total receives the block aggregate.
template <typename T, typename Op>
__device__ T block_inclusive(T v, T *warp_buf, T *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T o = shfl_up(v, d);
        if (lane >= d) v = Op::apply(o, v);
    }
    if (lane == 31) warp_buf[warp] = v;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nwarps ? warp_buf[lane] : Op::template identity<T>();
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            T o = shfl_up(w, d);
            if (lane >= d) w = Op::apply(o, w);
        }
        if (lane < nwarps) warp_buf[lane] = w;
    }
    __syncthreads();
    if (warp > 0) v = Op::apply(warp_buf[warp - 1], v);
    *total = warp_buf[nwarps - 1];
    __syncthreads();
    return v;
}

template <typename T, typename Op>
__global__ void __launch_bounds__(kScanThreads) k_tile_reduce(const T *__restrict__ in,
                                                               T *__restrict__ sums, int64_t n) {
    __shared__ T warp_buf[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    T v = Op::template identity<T>();
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        int64_t k = base + i;
        if (k < n) v = Op::apply(v, in[k]);
    }
    T total;
    block_inclusive<T, Op>(v, warp_buf, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// Scans one tile.  Exclusive: out[k] = op of in[0..k), out[n] = aggregate.
// Inclusive: out[k] = op of in[0..k].  `carry` (nullable) holds the
// exclusive scan of the tile aggregates.
template <typename T, typename Op, bool kInclusive>
__global__ void __launch_bounds__(kScanThreads) k_tile_scan(const T *in, T *out,
                                                             const T *__restrict__ carry,
                                                             int64_t n) {
    __shared__ T tile[kScanTile];
    __shared__ T warp_buf[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        int64_t k = base + i;
        tile[i] = k < n ? in[k] : Op::template identity<T>();
    }
    __syncthreads();
    T loc[kScanItems];
    T run = Op::template identity<T>();
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        loc[j] = tile[threadIdx.x * kScanItems + j];
        run = Op::apply(run, loc[j]);
    }
    T total;
    T incl = block_inclusive<T, Op>(run, warp_buf, &total);
    T prefix = carry ? carry[blockIdx.x] : Op::template identity<T>();
    // The exclusive prefix of this thread's first item is the left
    // neighbour's inclusive value (no subtraction, so it works for max too).
    __shared__ T incl_buf[kScanThreads];
    incl_buf[threadIdx.x] = incl;
    __syncthreads();
    T x = threadIdx.x == 0 ? prefix : Op::apply(prefix, incl_buf[threadIdx.x - 1]);
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        T y = Op::apply(x, loc[j]);
        tile[threadIdx.x * kScanItems + j] = kInclusive ? y : x;
        x = y;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
        int64_t k = base + i;
        if (k < n) out[k] = tile[i];
    }
    if (!kInclusive) {
        // the block holding element n-1 writes the aggregate at out[n]
        if (base <= n - 1 && n - 1 < base + kScanTile && threadIdx.x == 0)
            out[n] = Op::apply(prefix, total);
    }
}

template <typename T>
size_t tmp_levels(int64_t n) {
    if (n <= kScanTile) return 0;
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    return (size_t)(2 * nb + 1) + tmp_levels<T>(nb);
}

template <typename T, typename Op, bool kInclusive>
cudaError_t scan_impl(const T *in, T *out, int64_t n, T *tmp, cudaStream_t s) {
    if (n <= 0) {
        if (!kInclusive) return cudaMemsetAsync(out, 0, sizeof(T), s);
        return cudaSuccess;
    }
    int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        k_tile_scan<T, Op, kInclusive><<<1, kScanThreads, 0, s>>>(in, out, nullptr, n); note_launch();
        return cudaGetLastError();
    }
    T *sums = tmp, *sums_scan = tmp + nb, *rest = tmp + 2 * nb + 1;
    k_tile_reduce<T, Op><<<(unsigned)nb, kScanThreads, 0, s>>>(in, sums, n); note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_impl<T, Op, false>(sums, sums_scan, nb, rest, s);
    if (e != cudaSuccess) return e;
    k_tile_scan<T, Op, kInclusive><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, sums_scan, n); note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Radix sort
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint64_t *__restrict__ keys,
                                                              int64_t n, int shift,
                                                              uint32_t *__restrict__ hist,
                                                              int64_t ntiles) {
    __shared__ uint32_t cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll 4
    for (int i = 0; i < kSortItems; ++i) {
        int64_t k = base + (int64_t)i * kSortThreads + threadIdx.x;
        if (k < n) atomicAdd(&cnt[(keys[k] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter of one tile: within a warp, keys are ranked in order with
// __match_any_sync peer groups; warps are then ordered by a per-digit prefix
// over warps, digits by a prefix over the tile's digit counts, and the tile is
// first laid out digit-major in shared memory, so that the global writes of
// each digit's keys are consecutive (coalesced) rather than one per key.
constexpr int kScatterSmem = (kSortThreads / 32) * 256 * 4 + 2 * 256 * 4 + kSortTile * (8 + 4);

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const uint64_t *__restrict__ kin, const int32_t *__restrict__ vin, uint64_t *__restrict__ kout,
    int32_t *__restrict__ vout, int64_t n, int shift, const uint32_t *__restrict__ hist_scan,
    int64_t ntiles) {
    constexpr int kWarps = kSortThreads / 32;
    static_assert(kSortThreads == 256, "one thread per digit");
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *skey = reinterpret_cast<uint64_t *>(smem);                       // [kSortTile]
    int32_t *sval = reinterpret_cast<int32_t *>(skey + kSortTile);             // [kSortTile]
    uint32_t (*wcnt)[256] = reinterpret_cast<uint32_t (*)[256]>(sval + kSortTile);  // [kWarps][256]
    uint32_t *dstart = &wcnt[kWarps][0];                                         // [256]
    uint32_t *gbase = dstart + 256;                                              // [256]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kWarps * 256; i += kSortThreads) (&wcnt[0][0])[i] = 0;
    gbase[threadIdx.x] = hist_scan[(int64_t)threadIdx.x * ntiles + blockIdx.x];
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    const int64_t base = tile0 + (int64_t)warp * kSortWarpSpan;
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint64_t key[kSortItems];
    int32_t val[kSortItems];
    uint32_t rk[kSortItems];
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        int64_t k = base + i * 32 + lane;
        bool valid = k < n;
        key[i] = valid ? kin[k] : 0;
        val[i] = valid ? vin[k] : 0;
    }
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        const bool valid = base + i * 32 + lane < n;
        uint32_t d = valid ? (uint32_t)((key[i] >> shift) & 0xff) : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t cur = valid ? wcnt[warp][d] : 0;
        rk[i] = cur + __popc(peers & lt_mask);
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = cur + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // thread t owns digit t: prefix over warps, then over digits
    uint32_t run = 0;
    for (int w = 0; w < kWarps; ++w) {
        uint32_t t = wcnt[w][threadIdx.x];
        wcnt[w][threadIdx.x] = run;
        run += t;
    }
    {
        uint32_t incl = run;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += o;
        }
        if (lane == 31) dstart[warp] = incl;   // warp totals (dstart reused below)
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += dstart[w];
        __syncthreads();
        dstart[threadIdx.x] = before + incl - run;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kSortItems; ++i) {
        if (base + i * 32 + lane < n) {
            const uint32_t d = (uint32_t)((key[i] >> shift) & 0xff);
            const uint32_t lp = dstart[d] + wcnt[warp][d] + rk[i];
            skey[lp] = key[i];
            sval[lp] = val[i];
        }
    }
    __syncthreads();
    const int cnt = (int)min((int64_t)kSortTile, n - tile0);
    for (int j = threadIdx.x; j < cnt; j += kSortThreads) {
        const uint64_t kk = skey[j];
        const uint32_t d = (uint32_t)((kk >> shift) & 0xff);
        const int64_t pos = (int64_t)gbase[d] + (j - (int)dstart[d]);
        kout[pos] = kk;
        vout[pos] = sval[j];
    }
}

__global__ void k_reduce_max_i32(const int32_t *__restrict__ in, int64_t n, int32_t *out) {
    int32_t m = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        m = max(m, in[k]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, d));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(out, m);
}

__global__ void k_reduce_max_u64(const uint64_t *__restrict__ in, int64_t n,
                                 unsigned long long *out) {
    unsigned long long m = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)in[k]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, d));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(out, m);
}

}  // namespace

template <typename T>
size_t scan_tmp_elems(int64_t n) {
    return tmp_levels<T>(n) + 1;
}

template <typename T>
cudaError_t scan_exclusive(const T *in, T *out, int64_t n, T *tmp, cudaStream_t s) {
    return scan_impl<T, OpSum, false>(in, out, n, tmp, s);
}

template size_t scan_tmp_elems<uint32_t>(int64_t);
template size_t scan_tmp_elems<int64_t>(int64_t);
template size_t scan_tmp_elems<uint64_t>(int64_t);
template cudaError_t scan_exclusive<uint32_t>(const uint32_t *, uint32_t *, int64_t, uint32_t *,
                                              cudaStream_t);
template cudaError_t scan_exclusive<int64_t>(const int64_t *, int64_t *, int64_t, int64_t *,
                                             cudaStream_t);
template cudaError_t scan_exclusive<uint64_t>(const uint64_t *, uint64_t *, int64_t, uint64_t *,
                                              cudaStream_t);

size_t max_scan_tmp_elems(int64_t n) { return tmp_levels<int32_t>(n) + 1; }

cudaError_t max_scan_inclusive(const int32_t *in, int32_t *out, int64_t n, int32_t *tmp,
                               cudaStream_t s) {
    return scan_impl<int32_t, OpMax, true>(in, out, n, tmp, s);
}

size_t max_scan_i64_tmp_elems(int64_t n) { return tmp_levels<int64_t>(n) + 1; }

cudaError_t max_scan_inclusive_i64(const int64_t *in, int64_t *out, int64_t n, int64_t *tmp,
                                   cudaStream_t s) {
    return scan_impl<int64_t, OpMax, true>(in, out, n, tmp, s);
}

size_t radix_hist_elems(int64_t n) {
    int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    if (ntiles < 1) ntiles = 1;
    return (size_t)(256 * ntiles + 1);
}

cudaError_t radix_sort_pairs(uint64_t *k0, int32_t *v0, uint64_t *k1, int32_t *v1, int64_t n,
                             int begin_bit, int end_bit, uint32_t *hist, uint32_t *scan_tmp,
                             cudaStream_t s, int *which) {
    *which = 0;
    if (n <= 1 || end_bit <= begin_bit) return cudaSuccess;
    const int64_t ntiles = (n + kSortTile - 1) / kSortTile;
    {
        static bool attr_set[64] = {false};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
        if (!attr_set[dev]) {
            e = cudaFuncSetAttribute(k_radix_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kScatterSmem);
            if (e != cudaSuccess) return e;
            attr_set[dev] = true;
        }
    }
    uint64_t *ki = k0, *ko = k1;
    int32_t *vi = v0, *vo = v1;
    for (int shift = begin_bit; shift < end_bit; shift += 8) {
        k_radix_hist<<<(unsigned)ntiles, kSortThreads, 0, s>>>(ki, n, shift, hist, ntiles); note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = scan_impl<uint32_t, OpSum, false>(hist, hist, 256 * ntiles, scan_tmp, s);
        if (e != cudaSuccess) return e;
        k_radix_scatter<<<(unsigned)ntiles, kSortThreads, kScatterSmem, s>>>(ki, vi, ko, vo, n, shift,
                                                                              hist, ntiles); note_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        uint64_t *tk = ki; ki = ko; ko = tk;
        int32_t *tv = vi; vi = vo; vo = tv;
        *which ^= 1;
    }
    return cudaSuccess;
}

cudaError_t reduce_max_i32(const int32_t *in, int64_t n, int32_t *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int32_t), s);
    if (e != cudaSuccess || n <= 0) return e;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_reduce_max_i32<<<blocks, 256, 0, s>>>(in, n, out); note_launch();
    return cudaGetLastError();
}

cudaError_t reduce_max_u64(const uint64_t *in, int64_t n, unsigned long long *out,
                           cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n <= 0) return e;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    k_reduce_max_u64<<<blocks, 256, 0, s>>>(in, n, out); note_launch();
    return cudaGetLastError();
}

}  // namespace bfc
