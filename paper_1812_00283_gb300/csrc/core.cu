// The dense high-priority core counted by a matrix product on the tensor
// cores (a hybrid of Algorithm 2 with a masked core product).
//
// Split of the count.  Take the K vertices of highest priority (Definition 3)
// as the core C.  A core start u and a core end w (same layer, p(w) < p(u))
// share count_wedge(w) = a + b middles below u: a of them in the core, b not.
// By Lemma 1 the pair holds C(a + b, 2) = C(b, 2) + a·b + C(a, 2) butterflies.
// The walk of Algorithm 2 skips every wedge whose start, middle and end are
// all in the core, so for such a pair it counts only the b middles outside
// the core and its running sum yields C(b, 2); the count kernel then adds
// a·b + C(a, 2) for every core pair from its counters (b) and from the
// product below (a).  Pairs with an end or a start outside the core are
// untouched.
//
// The product.  In G* the core of a layer is the top of its id range (ids
// ascend in priority within a layer).  Let B be the 0/1 biadjacency between
// the U core (rows) and the L core (columns), and Bm the same with only the
// entries (u, v) with p(v) < p(u) kept (v among the first cut[u] neighbours
// of u).  Then a(u, w) = Σ_v Bm[u][v]·B[w][v] = (Bm · Bᵀ)[u][w] for two U core
// vertices, and the same with the layers swapped for the L core.  The 0/1
// operands are exact in bf16 and the sums (at most the core size of the
// other layer, below 2^16) are exact in fp32.
//
// The kernel is a tcgen05 GEMM for sm_103a: one CTA per 128 x 128 output
// tile of the lower triangle (w < u), operand tiles of 128 rows x 64 bf16
// brought into shared memory by TMA (128-byte swizzle) through a 4-stage
// mbarrier ring, one thread issuing tcgen05.mma (M = 128, N = 128, K = 16,
// fp32 accumulators in tensor memory), the four warps reading the tile back
// with tcgen05.ld and storing it as uint16.  Row tile t of Bm only has
// non-zeros below column cL(last row of t), so its contraction stops there.
// Every wait is bounded: a wait that gives up sets an error bit, the CTA
// drains what it started and frees its tensor memory.
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include "bfc_internal.cuh"

namespace bfc {
namespace {

constexpr int kT = 256;
constexpr int kTile = 128;        // output tile (rows and columns)
constexpr int kKBlock = 64;       // bf16 elements per operand row in one stage (128 bytes)
constexpr int kStages = 4;
constexpr int kStageBytes = 2 * kTile * kKBlock * 2;   // A and B tiles: 32 KB
constexpr int kGemmThreads = 128;
constexpr int kTmemCols = 128;    // fp32 accumulator columns
constexpr int kGemmSmem = kStages * kStageBytes + 1024;   // + alignment slack
constexpr uint64_t kWaitLimitNs = 2000000000ull;       // a wait gives up after 2 s

int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------
// Preparation kernels (graph-static)
// ---------------------------------------------------------------------------

// Global top-k by Definition 3.  In G* the priority order is (degree, id):
// within a layer ids ascend in (degree, original id), L ids come before U
// ids, and a U vertex wins a degree tie against an L vertex (U ids > L ids).
// The top k is the top ku of U and the top k - ku of L; ku is found by a
// binary search on the two descending sequences.
__device__ __forceinline__ bool key_less(const int32_t *deg, int32_t a, int32_t b) {
    const int32_t da = deg[a], db = deg[b];
    return da < db || (da == db && a < b);
}

__global__ void k_core_split(const int32_t *__restrict__ deg_star, int32_t r, int32_t l, int32_t k,
                             int32_t *out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int32_t n = r + l;
    int32_t lo = k > l ? k - l : 0, hi = k < r ? k : r;
    // t U vertices are too few while the (t+1)-th largest U key beats the
    // (k-t)-th largest L key
    while (lo < hi) {
        const int32_t t = (lo + hi) >> 1;
        const int32_t u = n - 1 - t;             // (t+1)-th largest of U
        const int32_t v = l - (k - t);           // (k-t)-th largest of L
        if (key_less(deg_star, v, u)) lo = t + 1; else hi = t;
    }
    out[0] = lo;          // core size in U
    out[1] = k - lo;      // core size in L
}

// ccut[x] for a core vertex x: the neighbours of x outside the core of the
// other layer, which form the prefix of x's ascending list.
__global__ void k_core_ccut(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                            int32_t l, int32_t n, int32_t lo_u, int32_t lo_l, int32_t *ccut) {
    const int32_t k_l = l - lo_l, k_u = n - lo_u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)k_l + k_u;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = i < k_l ? lo_l + (int32_t)i : lo_u + (int32_t)(i - k_l);
        const int32_t thr = x < l ? lo_u : lo_l;     // first core id of the other layer
        const int64_t b = off[x];
        int64_t lo = 0, hi = off[x + 1] - b;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (adj[b + mid] < thr) lo = mid + 1; else hi = mid;
        }
        ccut[x] = (int32_t)lo;
    }
}

// Rows of B and Bm for one layer's core, one warp per core vertex x: its core
// neighbours are list positions [ccut[x], deg); those below cut[x] have lower
// priority than x.  The matrices are zeroed before.  Each row also raises its
// row tile's contraction limit (in 64-column blocks, zeroed before) to cover
// its last lower-priority core neighbour, at list position cut[x] - 1.
__global__ void k_core_rows(const int64_t *__restrict__ off, const int32_t *__restrict__ adj,
                            const int32_t *__restrict__ cut, const int32_t *__restrict__ ccut,
                            int32_t row_lo, int32_t rows, int32_t col_lo, int32_t ld,
                            uint16_t *bmat, uint16_t *bmask, int32_t *kb) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint16_t one = 0x3F80;   // bf16 1.0
    for (int64_t i = w0; i < rows; i += nw) {
        const int32_t x = row_lo + (int32_t)i;
        const int64_t b = off[x], d = off[x + 1] - b;
        const int32_t c = cut[x], cc = ccut[x];
        for (int64_t k = cc + lane; k < d; k += 32) {
            const int32_t col = adj[b + k] - col_lo;
            bmat[i * ld + col] = one;
            if (k < c) bmask[i * ld + col] = one;
        }
        if (lane == 0 && c > cc)
            atomicMax(kb + i / kTile, (adj[b + c - 1] - col_lo + kKBlock) / kKBlock);
    }
}

// ---------------------------------------------------------------------------
// PTX wrappers (sm_100 family: mbarrier, TMA, tcgen05)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ uint64_t now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits until the phase of the given parity has completed; false if it gave
// up after kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = now_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (now_ns() - t0 > kWaitLimitNs) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int32_t x, int32_t y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile written by TMA
// with the 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart
// (stride byte offset), leading byte offset unused for this layout (1),
// descriptor version 1, layout type 2 = 128-byte swizzle.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                  // leading byte offset (16 B, unused)
    d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
    d |= (uint64_t)1 << 46;                  // version
    d |= (uint64_t)2 << 61;                  // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: fp32 accumulators (bits 4-5 = 1),
// A and B bf16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTile >> 3) << 17) |
                            ((uint32_t)(kTile >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// 32 lanes x 32 columns of fp32 from tensor memory: thread i gets row
// (lane base + i), columns [col, col + 32).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ---------------------------------------------------------------------------
// The masked core product: C[u][w] = Σ_v A[u][v]·B[w][v] for the tiles of the
// lower triangle, as uint16.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kGemmThreads, 1)
k_core_gemm(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
            const int32_t *__restrict__ kblocks, uint16_t *out, int32_t ld_out, int *err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], accf;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // tile (tm, tn) of the lower triangle: t = tm (tm + 1) / 2 + tn, tn <= tm
    const int64_t t = blockIdx.x;
    int32_t tm = (int32_t)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((int64_t)(tm + 1) * (tm + 2) / 2 <= t) ++tm;
    while ((int64_t)tm * (tm + 1) / 2 > t) --tm;
    const int32_t tn = (int32_t)(t - (int64_t)tm * (tm + 1) / 2);
    const int32_t nk = kblocks[tm];

    // 1024-byte aligned stages (the swizzle atom)
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;
    auto stage_a = [&](int s) { return base + (uint32_t)s * kStageBytes; };
    auto stage_b = [&](int s) { return base + (uint32_t)s * kStageBytes + kTile * kKBlock * 2; };

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(&accf), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();   // warp 0 reconverges before its .sync.aligned allocation
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (nk > 0) {
        if (warp == 0 && lane == 0) {
            // producer: TMA loads of the A rows of tile tm and the B rows of tile tn
            int issued = 0;
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % kStages;
                if (kb >= kStages && !mbar_wait(smem_u32(&empty[s]), (uint32_t)((kb / kStages) - 1) & 1u)) {
                    atomicOr(err, kErrTimeout);
                    abort_flag = 1;
                    break;
                }
                if (*((volatile int *)&abort_flag)) break;
                mbar_expect_tx(smem_u32(&full[s]), kStageBytes);
                tma_load_2d(stage_a(s), &map_a, smem_u32(&full[s]), kb * kKBlock, tm * kTile);
                tma_load_2d(stage_b(s), &map_b, smem_u32(&full[s]), kb * kKBlock, tn * kTile);
                ++issued;
            }
            // copies still in flight complete before the CTA can exit
            for (int kb = std::max(0, issued - kStages); kb < issued; ++kb)
                mbar_wait(smem_u32(&full[kb % kStages]), (uint32_t)(kb / kStages) & 1u);
        } else if (warp == 1 && lane == 0) {
            // MMA issuer: four K = 16 steps per stage, advancing 32 bytes
            // inside the 128-byte swizzled rows
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % kStages;
                if (!mbar_wait(smem_u32(&full[s]), (uint32_t)(kb / kStages) & 1u)) {
                    atomicOr(err, kErrTimeout);
                    abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const uint64_t da = sw128_desc(stage_a(s)), db = sw128_desc(stage_b(s));
#pragma unroll
                for (int k = 0; k < kKBlock / 16; ++k)
                    mma_bf16(tmem, da + (uint64_t)(k * 2), db + (uint64_t)(k * 2), (kb | k) ? 1u : 0u);
                mma_commit(smem_u32(&empty[s]));   // the stage is free once these MMAs are done
            }
            mma_commit(smem_u32(&accf));           // every MMA issued so far is done
        }
        __syncwarp();
        // epilogue: warp w reads accumulator rows 32w .. 32w + 31
        const bool ok = mbar_wait(smem_u32(&accf), 0);
        if (!ok && lane == 0) atomicOr(err, kErrTimeout);
        __syncwarp();   // the lanes may leave the wait apart; tcgen05.ld is .sync.aligned
        tc_fence_after();
        const int64_t row = (int64_t)tm * kTile + warp * 32 + lane;
#pragma unroll 1
        for (int c = 0; c < kTile / 32; ++c) {
            uint32_t v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), v);
            uint32_t packed[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const uint32_t lo = (uint32_t)__float2uint_rn(__uint_as_float(v[2 * j]));
                const uint32_t hi = (uint32_t)__float2uint_rn(__uint_as_float(v[2 * j + 1]));
                packed[j] = (lo & 0xFFFFu) | (hi << 16);
            }
            uint4 *dst = reinterpret_cast<uint4 *>(out + row * ld_out + (int64_t)tn * kTile + c * 32);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
        }
    } else {
        // no middle of this row tile lies in the core below its rows: a = 0
        const int64_t row = (int64_t)tm * kTile + warp * 32 + lane;
        uint4 *dst = reinterpret_cast<uint4 *>(out + row * ld_out + (int64_t)tn * kTile);
#pragma unroll
        for (int q = 0; q < kTile * 2 / 16; ++q) dst[q] = make_uint4(0, 0, 0, 0);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_encode_mutex;
EncodeTiledFn g_encode = nullptr;

int get_encode(EncodeTiledFn *fn) {
    std::lock_guard<std::mutex> lk(g_encode_mutex);
    if (!g_encode) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
            set_last_error("cuTensorMapEncodeTiled is not available");
            return BFC_ERR_CUDA;
        }
        g_encode = reinterpret_cast<EncodeTiledFn>(p);
    }
    *fn = g_encode;
    return BFC_OK;
}

// Tensor map of a row-major bf16 matrix (rows x cols, cols a multiple of 64,
// base 256-byte aligned), boxes of 128 rows x 64 columns, 128-byte swizzle.
int make_map(CUtensorMap *map, const uint16_t *base, int64_t rows, int64_t cols) {
    EncodeTiledFn enc;
    int rc = get_encode(&enc);
    if (rc) return rc;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kKBlock, (cuuint32_t)kTile};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t *>(base), dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_last_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
        return BFC_ERR_CUDA;
    }
    return BFC_OK;
}

int blocks(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>(cdiv(n, kT), 1), 152 * 32); }

CUtensorMap *map_of(Graph *g, int i) {
    static_assert(sizeof(CUtensorMap) == sizeof(g->core_map_bytes[0]), "tensor map size");
    return reinterpret_cast<CUtensorMap *>(g->core_map_bytes[i]);
}

}  // namespace

// Chooses the core (top core_vertices of Definition 3's order, split between
// the layers), builds B and Bm of both layers' cores and the tile limits.
// Called by prepare while the G* degrees are still at hand; synchronises s.
int core_prepare(Graph *g, cudaStream_t s, const int32_t *deg_star, int32_t core_vertices, bool automatic) {
    const int32_t k = std::min<int32_t>(core_vertices, g->n);
    if (k <= 0 || g->m == 0) return BFC_OK;
    int32_t *split = nullptr;
    Allocs tmp;
    tmp.stream = s;
    struct Guard { Allocs *a; ~Guard() { a->release(); } } guard{&tmp};
    if (tmp.get(&split, 2)) return BFC_ERR_OUT_OF_MEMORY;
    k_core_split<<<1, 1, 0, s>>>(deg_star, g->r, g->l, k, split);
    note_launch();
    BFC_CUDA(cudaGetLastError());
    int32_t h[2] = {0, 0};
    BFC_CUDA(cudaMemcpyAsync(h, split, sizeof(h), cudaMemcpyDeviceToHost, s));
    BFC_CUDA(cudaStreamSynchronize(s));
    const int32_t ku = h[0], kl = h[1];
    // the automatic core needs both layers in it: with a thin side the core
    // block holds few wedges and the product would be pure overhead
    if (automatic && (ku < kCoreAutoMinLayer || kl < kCoreAutoMinLayer)) return BFC_OK;
    if (ku > 65535 || kl > 65535) {
        set_last_error("core_vertices too large: a layer's core holds at most 65,535 vertices");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    g->core_u = ku;
    g->core_l = kl;
    g->core_lo_u = g->n - ku;
    g->core_lo_l = g->l - kl;
    g->core_ld_u = (int32_t)(cdiv(std::max(ku, 1), kTile) * kTile);
    g->core_ld_l = (int32_t)(cdiv(std::max(kl, 1), kTile) * kTile);
    const int64_t pu = g->core_ld_u, pl = g->core_ld_l;
    auto get = [&](auto **p, int64_t cnt) { return g->mem.get(p, (size_t)std::max<int64_t>(cnt, 1)); };
    if (get(&g->ccut, g->n) || get(&g->core_bu, pu * pl) || get(&g->core_bum, pu * pl) ||
        get(&g->core_bl, pl * pu) || get(&g->core_blm, pl * pu) || get(&g->core_au, pu * pu) ||
        get(&g->core_al, pl * pl) || get(&g->core_kb_u, pu / kTile) || get(&g->core_kb_l, pl / kTile)) {
        set_last_error("device allocation failed: core matrices");
        return BFC_ERR_OUT_OF_MEMORY;
    }
    BFC_CUDA(cudaMemsetAsync(g->core_bu, 0, (size_t)(pu * pl) * 2, s));
    BFC_CUDA(cudaMemsetAsync(g->core_bum, 0, (size_t)(pu * pl) * 2, s));
    BFC_CUDA(cudaMemsetAsync(g->core_bl, 0, (size_t)(pl * pu) * 2, s));
    BFC_CUDA(cudaMemsetAsync(g->core_blm, 0, (size_t)(pl * pu) * 2, s));
    k_core_ccut<<<blocks((int64_t)ku + kl), kT, 0, s>>>(g->off, g->adj, g->l, g->n, g->core_lo_u,
                                                        g->core_lo_l, g->ccut);
    note_launch();
    BFC_CUDA(cudaGetLastError());
    BFC_CUDA(cudaMemsetAsync(g->core_kb_u, 0, sizeof(int32_t) * (size_t)(pu / kTile), s));
    BFC_CUDA(cudaMemsetAsync(g->core_kb_l, 0, sizeof(int32_t) * (size_t)(pl / kTile), s));
    if (ku > 0) {
        k_core_rows<<<blocks((int64_t)ku * 32), kT, 0, s>>>(g->off, g->adj, g->cut, g->ccut, g->core_lo_u, ku,
                                                             g->core_lo_l, (int32_t)pl, g->core_bu, g->core_bum,
                                                             g->core_kb_u);
        note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    if (kl > 0) {
        k_core_rows<<<blocks((int64_t)kl * 32), kT, 0, s>>>(g->off, g->adj, g->cut, g->ccut, g->core_lo_l, kl,
                                                             g->core_lo_u, (int32_t)pu, g->core_bl, g->core_blm,
                                                             g->core_kb_l);
        note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    int rc = make_map(map_of(g, 0), g->core_bum, pu, pl);   // U starts: Bm rows
    if (!rc) rc = make_map(map_of(g, 1), g->core_bu, pu, pl);
    if (!rc) rc = make_map(map_of(g, 2), g->core_blm, pl, pu);   // L starts
    if (!rc) rc = make_map(map_of(g, 3), g->core_bl, pl, pu);
    if (rc) return rc;
    BFC_CUDA(cudaStreamSynchronize(s));
    return BFC_OK;
}

// The products a(u, w) of both cores, on s (asynchronous).
int core_product(Graph *g, cudaStream_t s) {
    static std::mutex mu;
    static bool attr_done[64] = {false};
    {
        std::lock_guard<std::mutex> lk(mu);
        if (g->device < 0 || g->device >= 64) return BFC_ERR_INVALID_ARGUMENT;
        if (!attr_done[g->device]) {
            BFC_CUDA(cudaFuncSetAttribute(k_core_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem));
            attr_done[g->device] = true;
        }
    }
    const int64_t tu = g->core_ld_u / kTile, tl = g->core_ld_l / kTile;
    if (g->core_u > 0) {
        k_core_gemm<<<(unsigned)(tu * (tu + 1) / 2), kGemmThreads, kGemmSmem, s>>>(
            *map_of(g, 0), *map_of(g, 1), g->core_kb_u, g->core_au, g->core_ld_u, g->err);
        note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    if (g->core_l > 0) {
        k_core_gemm<<<(unsigned)(tl * (tl + 1) / 2), kGemmThreads, kGemmSmem, s>>>(
            *map_of(g, 2), *map_of(g, 3), g->core_kb_l, g->core_al, g->core_ld_l, g->err);
        note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    return BFC_OK;
}

}  // namespace bfc
