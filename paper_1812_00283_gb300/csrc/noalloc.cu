// bfc_count_small_noalloc: an exact butterfly count for small graphs that
// allocates nothing.
//
// Who needs it: code that may not call cudaMalloc or any allocating routine
// at the point where it counts -- for example a caller whose memory is fully
// reserved up front by its own allocator and that may not grow the device
// footprint, or a real-time loop that must not hit the driver's allocator
// (which can synchronise the device).  The regular entry points
// (bfc_prepare and friends) allocate the renumbered graph from a pool, so
// they are not usable there.
//
// How: every byte of working memory this entry point needs lives in one
// file-scope __device__ array of fixed size (below), which every GPU that
// loads the library holds until the process exits.  The caller passes only
// inputs and outputs.  The whole count is one cooperative kernel: it clears
// the scratch it uses, checks the CSR, builds the L-side lists, and counts
// with Algorithm 2's priority filters (no sorted lists; each neighbour is
// tested against the start's priority).
#include <cooperative_groups.h>

#include <mutex>

#include "bfc_internal.cuh"

namespace cg = cooperative_groups;

namespace bfc {
namespace {

constexpr int kNaThreads = 1024;                  // one CTA of 32 warps per SM
constexpr int kNaWarps = kNaThreads / 32;
constexpr int kNaSmemBytes = 192 * 1024;          // dynamic shared memory: the dense counters
constexpr int32_t kNaMaxVertices = 65536;        // |U| + |L|
constexpr int32_t kNaMaxLayer = kNaSmemBytes / 4; // 49,152 per layer (one dense 32-bit counter array)
constexpr int64_t kNaMaxEdges = 1 << 20;         // 1,048,576 edges
// words: [0,2) 64-bit accumulator | [2] error flags | [3] pad | deg[n] | loff[l+1] | lfill[l] | ladj[m]
constexpr int64_t kNaWords = 4 + 3ll * kNaMaxVertices + 1 + kNaMaxEdges;

}  // namespace
}  // namespace bfc

// The shared scratch of bfc_count_small_noalloc (about 4.8 MB).
static __device__ __align__(256) int32_t g_noalloc_scratch[bfc::kNaWords];

namespace bfc {
namespace {

// p(a) < p(b) in Definition 3's order, ids in the global id space
// (L vertex v -> v, U vertex u -> l + u)
__device__ __forceinline__ bool lower_priority(const int32_t *deg, int32_t a, int32_t b) {
    const int32_t da = deg[a], db = deg[b];
    return da < db || (da == db && a < b);
}

__global__ void __launch_bounds__(kNaThreads, 1)
k_count_noalloc(int32_t r, int32_t l, int32_t m, const int32_t *__restrict__ off_u,
                const int32_t *__restrict__ adj_u, int32_t *scratch,
                unsigned long long *total_out, int32_t *status_out) {
    cg::grid_group grid = cg::this_grid();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem_raw);
    __shared__ unsigned long long red[32];
    __shared__ int32_t carry;

    const int32_t n = r + l;
    unsigned long long *acc_g = reinterpret_cast<unsigned long long *>(scratch);
    int32_t *err = scratch + 2;
    int32_t *deg = scratch + 4;
    int32_t *loff = deg + n;
    int32_t *lfill = loff + l + 1;
    int32_t *ladj = lfill + l;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // clear what must start at zero (the scratch keeps the previous call's contents)
    if (gtid == 0) { *acc_g = 0; *err = 0; }
    for (int64_t i = gtid; i < n; i += gstride) deg[i] = 0;
    for (int64_t i = gtid; i < l; i += gstride) lfill[i] = 0;
    grid.sync();

    // the CSR must be a CSR before anything indexes with it
    for (int64_t u = gtid; u <= r; u += gstride) {
        if (u == 0 && off_u[0] != 0) atomicOr(err, 1);
        if (u < r && off_u[u + 1] < off_u[u]) atomicOr(err, 1);
        if (u == r && off_u[r] != m) atomicOr(err, 1);
    }
    for (int64_t k = gtid; k < m; k += gstride) {
        const int32_t v = adj_u[k];
        if (v < 0 || v >= l) atomicOr(err, 2);
    }
    grid.sync();
    const bool bad = *((volatile int32_t *)err) != 0;

    // degrees, in the global id space
    if (!bad) {
        for (int64_t u = gtid; u < r; u += gstride) deg[l + u] = off_u[u + 1] - off_u[u];
        for (int64_t k = gtid; k < m; k += gstride) atomicAdd(&deg[adj_u[k]], 1);
    }
    grid.sync();

    // L-side offsets: one block scans deg[0, l)
    if (!bad && blockIdx.x == 0) {
        if (threadIdx.x == 0) carry = 0;
        __syncthreads();
        for (int32_t base = 0; base < l; base += kNaThreads) {
            const int32_t i = base + threadIdx.x;
            int32_t x = i < l ? deg[i] : 0;
            int32_t v = x;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                int32_t o = __shfl_up_sync(0xffffffffu, v, d);
                if (lane >= d) v += o;
            }
            __shared__ int32_t wsum[32];
            if (lane == 31) wsum[warp] = v;
            __syncthreads();
            if (warp == 0) {
                int32_t w = wsum[lane];
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    int32_t o = __shfl_up_sync(0xffffffffu, w, d);
                    if (lane >= d) w += o;
                }
                wsum[lane] = w;
            }
            __syncthreads();
            const int32_t incl = v + (warp > 0 ? wsum[warp - 1] : 0);
            if (i < l) loff[i] = carry + incl - x;
            __syncthreads();
            if (threadIdx.x == kNaThreads - 1) carry += incl;
            __syncthreads();
        }
        if (threadIdx.x == 0) loff[l] = carry;
    }
    grid.sync();

    // L-side lists (any order: every neighbour is tested against the filter)
    if (!bad) {
        for (int64_t u = gtid; u < r; u += gstride)
            for (int32_t k = off_u[u]; k < off_u[u + 1]; ++k) {
                const int32_t v = adj_u[k];
                ladj[loff[v] + atomicAdd(&lfill[v], 1)] = (int32_t)u;
            }
    }
    grid.sync();

    // Algorithm 2: for every start x, middles v with p(v) < p(x), ends w with
    // p(w) < p(x); Σ old over the increments of count_wedge(w) = Σ C(count, 2)
    unsigned long long acc = 0;
    if (!bad) {
        for (int32_t x = blockIdx.x; x < n; x += gridDim.x) {
            const bool in_u = x >= l;
            const int32_t layer = in_u ? r : l;
            const int32_t mb = in_u ? off_u[x - l] : loff[x];
            const int32_t me = in_u ? off_u[x - l + 1] : loff[x + 1];
            // a start none of whose neighbours has lower priority has no
            // wedges: skip its clear and its walk (most light starts)
            bool any = false;
            for (int32_t j = mb + threadIdx.x; j < me && !any; j += kNaThreads)
                any = lower_priority(deg, in_u ? adj_u[j] : l + ladj[j], x);
            if (!__syncthreads_or(any)) continue;
            uint4 *c4 = reinterpret_cast<uint4 *>(cnt);
            for (int32_t i = threadIdx.x; i < (layer + 3) / 4; i += kNaThreads)
                c4[i] = make_uint4(0, 0, 0, 0);
            __syncthreads();
            for (int32_t j = mb + warp; j < me; j += kNaWarps) {
                const int32_t v = in_u ? adj_u[j] : l + ladj[j];       // middle, global id
                if (!lower_priority(deg, v, x)) continue;
                const int32_t eb = in_u ? loff[v] : off_u[v - l];
                const int32_t ee = in_u ? loff[v + 1] : off_u[v - l + 1];
                for (int32_t k = eb + lane; k < ee; k += 32) {
                    const int32_t w = in_u ? l + ladj[k] : adj_u[k];   // end, global id
                    if (lower_priority(deg, w, x)) acc += atomicAdd(&cnt[in_u ? w - l : w], 1u);
                }
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (warp == 0) {
        unsigned long long t = red[lane];
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) t += __shfl_xor_sync(0xffffffffu, t, d);
        if (lane == 0 && t) atomicAdd(acc_g, t);
    }
    grid.sync();
    if (gtid == 0) {
        *total_out = bad ? 0ull : *((volatile unsigned long long *)acc_g);
        if (status_out) *status_out = bad ? BFC_ERR_INVALID_GRAPH : BFC_OK;
    }
}

std::mutex g_na_mutex;
int32_t *g_na_ptr[64] = {};
int g_na_grid[64] = {};

// Once per device, with that device current: the device address of the
// scratch array (the host-side name is only a stand-in), the kernel's shared
// memory attribute and the co-resident grid size.
int noalloc_setup(int dev, int32_t **ptr, int *grid) {
    std::lock_guard<std::mutex> lk(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        e = cudaFuncSetAttribute(k_count_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kNaSmemBytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(k_count_noalloc)");
        int sms = 0, per_sm = 0, coop = 0;
        e = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
        if (!coop) { set_last_error("device cannot launch cooperative kernels"); return BFC_ERR_CUDA; }
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_noalloc, kNaThreads,
                                                          kNaSmemBytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        if (per_sm < 1) { set_last_error("k_count_noalloc does not fit on an SM"); return BFC_ERR_CUDA; }
        g_na_grid[dev] = sms * per_sm;
        g_na_ptr[dev] = static_cast<int32_t *>(p);
    }
    *ptr = g_na_ptr[dev];
    *grid = g_na_grid[dev];
    return BFC_OK;
}

}  // namespace
}  // namespace bfc

extern "C" int bfc_count_small_noalloc(int32_t num_u, int32_t num_l, int64_t num_edges,
                                       const int32_t *off_u_dev, const int32_t *adj_u_dev,
                                       void *stream, uint64_t *total_dev, int32_t *status_dev) {
    bfc::set_last_error("");
    if (!off_u_dev || !total_dev || (num_edges > 0 && !adj_u_dev) || num_u < 0 || num_l < 0 ||
        num_edges < 0) {
        bfc::set_last_error("bfc_count_small_noalloc: null pointer or negative size");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    if ((int64_t)num_u + num_l > bfc::kNaMaxVertices || num_u > bfc::kNaMaxLayer ||
        num_l > bfc::kNaMaxLayer || num_edges > bfc::kNaMaxEdges) {
        bfc::set_last_error("bfc_count_small_noalloc: graph too large (limits: |U|, |L| <= 49152, "
                            "|U| + |L| <= 65536, edges <= 1048576)");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    int dev = 0;
    BFC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { bfc::set_last_error("device index out of range"); return BFC_ERR_CUDA; }
    int32_t *scratch = nullptr;
    int grid = 0;
    int rc = bfc::noalloc_setup(dev, &scratch, &grid);
    if (rc) return rc;
    int32_t r = num_u, l = num_l, m = (int32_t)num_edges;
    unsigned long long *tot = reinterpret_cast<unsigned long long *>(total_dev);
    void *args[] = {&r, &l, &m, (void *)&off_u_dev, (void *)&adj_u_dev, &scratch, &tot, &status_dev};
    BFC_CUDA(cudaLaunchCooperativeKernel((const void *)bfc::k_count_noalloc, dim3(grid),
                                         dim3(bfc::kNaThreads), args, bfc::kNaSmemBytes,
                                         static_cast<cudaStream_t>(stream)));
    bfc::note_launch();
    return BFC_OK;
}
