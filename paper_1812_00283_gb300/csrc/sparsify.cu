// Approximate counting by edge sparsification (Section 7: the exact counter
// is the inner block of a sampling estimator, run on sampled graphs).
//
// Every sample keeps each edge independently with probability p.  A
// butterfly survives a sample iff its four edges do, so E[⋈(G_j)] = p^4 ⋈(G)
// and the mean of the samples' exact counts divided by p^4 estimates ⋈(G).
//
// The samples are built side by side as one disjoint union (sample j's U
// vertices at j·|U|.., its L vertices at j·|L|..), which is then prepared and
// counted as a batch: one set of sorts and scans for all samples and one
// persistent count launch with a total per sample.
//
// Keep rule (the same on every platform): sample j keeps the edge at U-side
// slot e iff the (j·m + e + 1)-th output of SplitMix64 seeded with `seed` is
// below floor(p · 2^64); p = 1 keeps every edge.  SplitMix64 is the generator
// of Steele, Lea and Flood (OOPSLA 2014).
#include <algorithm>
#include <cmath>

#include "bfc_internal.cuh"

namespace bfc {
namespace {

constexpr int kT = 256;

unsigned grid_for(int64_t threads) {
    return (unsigned)std::min<int64_t>(std::max<int64_t>((threads + kT - 1) / kT, 1), 152 * 32);
}

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
    uint64_t z = seed + k * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct SampleRule {
    uint64_t seed, threshold;
    int keep_all;
};

// offsets of a CSR: off[0] = 0, off[r] = m, non-decreasing (bit 0 of *bad)
__global__ void k_sp_check_offsets(const int32_t *__restrict__ off, int32_t r, int64_t m, int *bad) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u <= r;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = off[u];
        const bool ok = (u == 0 ? o == 0 : o >= off[u - 1]) && (u < r || o == m);
        if (!ok) atomicOr(bad, 1);
    }
}

// One warp per row (j, u) of the union: lanes draw for the row's slots, a
// ballot gives the kept slots.  kWrite = false: the kept count of the row
// (and, for sample 0, a check of the L ids, bit 1 of *bad); kWrite = true:
// the kept L ids, shifted to sample j's range, at the row's offset.
template <bool kWrite>
__global__ void k_sp_rows(const int32_t *__restrict__ off, const int32_t *__restrict__ adj, int32_t r,
                          int32_t l, int64_t m, int32_t samples, SampleRule rule, int64_t *__restrict__ cnt,
                          const int64_t *__restrict__ uoff, int32_t *__restrict__ uoff32,
                          int32_t *__restrict__ uadj, int *bad) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t rows = (int64_t)samples * r;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t row = w0; row < rows; row += nw) {
        const int64_t j = row / r;
        const int32_t u = (int32_t)(row - j * r);
        const int32_t e0 = off[u], e1 = off[u + 1];
        const uint64_t k0 = (uint64_t)j * (uint64_t)m + 1;   // draw number of slot 0
        const int32_t shift = (int32_t)(j * l);
        int64_t at = kWrite ? uoff[row] : 0;
        int32_t kept = 0;
        for (int64_t b = e0; b < e1; b += 32) {   // warp-uniform
            const int64_t e = b + lane;
            const bool in = e < e1;
            const int32_t v = in ? adj[e] : 0;
            const bool keep = in && (rule.keep_all || splitmix64_at(rule.seed, k0 + (uint64_t)e) < rule.threshold);
            if (!kWrite && j == 0 && in && (v < 0 || v >= l)) atomicOr(bad, 2);
            const uint32_t bal = __ballot_sync(0xffffffffu, keep);
            if (kWrite && keep) uadj[at + kept + __popc(bal & lt)] = v + shift;
            kept += __popc(bal);
        }
        if (lane == 0) {
            if (kWrite) uoff32[row] = (int32_t)at;
            else cnt[row] = kept;
        }
    }
}

// the union's last offset, the sample ranges and the kept edges per sample
__global__ void k_sp_ranges(const int64_t *__restrict__ uoff, int32_t r, int32_t l, int32_t samples,
                            int32_t *uoff32, int32_t *us, int32_t *ls, uint64_t *sample_edges) {
    for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j <= samples; j += gridDim.x * blockDim.x) {
        us[j] = (int32_t)((int64_t)j * r);
        ls[j] = (int32_t)((int64_t)j * l);
        if (j == samples) uoff32[(int64_t)samples * r] = (int32_t)uoff[(int64_t)samples * r];
        if (sample_edges && j < samples)
            sample_edges[j] = (uint64_t)(uoff[(int64_t)(j + 1) * r] - uoff[(int64_t)j * r]);
    }
}

// estimate = Σ c_j / (samples · p^4); standard error = sd(c_j) / p^4 / sqrt(samples)
__global__ void k_sp_estimate(const uint64_t *__restrict__ counts, int32_t samples, double p, double *out) {
    __shared__ unsigned long long s_sum[kT];
    __shared__ double s_sq[kT];
    unsigned long long acc = 0;
    for (int32_t j = threadIdx.x; j < samples; j += blockDim.x) acc += counts[j];
    s_sum[threadIdx.x] = acc;
    __syncthreads();
    for (int d = kT / 2; d > 0; d >>= 1) {
        if (threadIdx.x < d) s_sum[threadIdx.x] += s_sum[threadIdx.x + d];
        __syncthreads();
    }
    const unsigned long long total = s_sum[0];
    const double mean = (double)total / (double)samples;
    double sq = 0.0;
    for (int32_t j = threadIdx.x; j < samples; j += blockDim.x) {
        const double d = (double)counts[j] - mean;
        sq += d * d;
    }
    s_sq[threadIdx.x] = sq;
    __syncthreads();
    for (int d = kT / 2; d > 0; d >>= 1) {
        if (threadIdx.x < d) s_sq[threadIdx.x] += s_sq[threadIdx.x + d];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double p4 = (p * p) * (p * p);
        out[0] = (double)total / ((double)samples * p4);
        out[1] = samples > 1 ? sqrt(s_sq[0] / (double)(samples - 1) / (double)samples) / p4 : (double)NAN;
    }
}

}  // namespace
}  // namespace bfc

extern "C" int bfc_prepare_sparsified(int32_t num_u, int32_t num_l, int64_t num_edges,
                                      const int32_t *off_u_dev, const int32_t *adj_u_dev, double p,
                                      uint64_t seed, int32_t num_samples, const bfc_options *opt,
                                      void *stream, uint64_t *sample_edges_dev, bfc_graph **out) {
    bfc::set_last_error("");
    if (!out) { bfc::set_last_error("null argument"); return BFC_ERR_INVALID_ARGUMENT; }
    *out = nullptr;
    if (num_u < 0 || num_l < 0 || num_edges < 0 || num_edges > 2147483647LL || !off_u_dev ||
        (num_edges > 0 && !adj_u_dev)) {
        bfc::set_last_error("invalid CSR arguments");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    if (!(p > 0.0 && p <= 1.0)) { bfc::set_last_error("keep probability must lie in (0, 1]"); return BFC_ERR_INVALID_ARGUMENT; }
    if (num_samples < 1 || (int64_t)num_samples * ((int64_t)num_u + num_l) > 2147483646LL) {
        bfc::set_last_error("num_samples must be >= 1 with num_samples * (|U| + |L|) below 2^31 - 1");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // p · 2^64 is exact in binary floating point; the conversion truncates
    const bfc::SampleRule rule{seed, p < 1.0 ? (uint64_t)std::ldexp(p, 64) : 0ull, p == 1.0 ? 1 : 0};
    bfc::Allocs a;
    a.stream = s;
    struct Guard { bfc::Allocs *a; ~Guard() { a->release(); } } guard{&a};
    const int64_t rows = (int64_t)num_samples * num_u;
    int *bad;
    int64_t *cnt, *uoff, *scan_tmp;
    int32_t *uoff32, *us, *ls;
    if (a.get(&bad, 1) || a.get(&cnt, rows + 1) || a.get(&uoff, rows + 1) ||
        a.get(&scan_tmp, bfc::scan_tmp_elems<int64_t>(rows)) || a.get(&uoff32, rows + 1) ||
        a.get(&us, (size_t)num_samples + 1) || a.get(&ls, (size_t)num_samples + 1)) {
        bfc::set_last_error("device allocation failed: sample offsets");
        return BFC_ERR_OUT_OF_MEMORY;
    }
    BFC_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    bfc::k_sp_check_offsets<<<bfc::grid_for((int64_t)num_u + 1), bfc::kT, 0, s>>>(off_u_dev, num_u, num_edges, bad);
    bfc::note_launch();
    BFC_CUDA(cudaGetLastError());
    int hbad = 0;
    BFC_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    BFC_CUDA(cudaStreamSynchronize(s));
    if (hbad) { bfc::set_last_error("offsets are not a CSR of num_edges slots"); return BFC_ERR_INVALID_GRAPH; }
    const unsigned rgrid = bfc::grid_for(rows * 32);
    if (rows > 0) {
        bfc::k_sp_rows<false><<<rgrid, bfc::kT, 0, s>>>(off_u_dev, adj_u_dev, num_u, num_l, num_edges, num_samples,
                                                        rule, cnt, nullptr, nullptr, nullptr, bad);
        bfc::note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    BFC_CUDA(bfc::scan_exclusive<int64_t>(cnt, uoff, rows, scan_tmp, s));
    int64_t kept = 0;
    BFC_CUDA(cudaMemcpyAsync(&kept, uoff + rows, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    BFC_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    BFC_CUDA(cudaStreamSynchronize(s));
    if (hbad) { bfc::set_last_error("an L id lies outside [0, num_l)"); return BFC_ERR_INVALID_GRAPH; }
    if (kept > 2147483647LL) {
        bfc::set_last_error("the samples hold more than 2^31 - 1 edges together: use fewer samples");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    int32_t *uadj;
    if (a.get(&uadj, (size_t)std::max<int64_t>(kept, 1))) {
        bfc::set_last_error("device allocation failed: sampled edges");
        return BFC_ERR_OUT_OF_MEMORY;
    }
    if (rows > 0) {
        bfc::k_sp_rows<true><<<rgrid, bfc::kT, 0, s>>>(off_u_dev, adj_u_dev, num_u, num_l, num_edges, num_samples,
                                                       rule, nullptr, uoff, uoff32, uadj, bad);
        bfc::note_launch();
        BFC_CUDA(cudaGetLastError());
    }
    bfc::k_sp_ranges<<<bfc::grid_for((int64_t)num_samples + 1), bfc::kT, 0, s>>>(
        uoff, num_u, num_l, num_samples, uoff32, us, ls, sample_edges_dev);
    bfc::note_launch();
    BFC_CUDA(cudaGetLastError());
    const bfc_csr u{(int32_t)rows, (int32_t)((int64_t)num_samples * num_l), kept, uoff32, uadj};
    const bfc_batch b{num_samples, us, ls};
    // the union's arrays go back to the pool in stream order after the prepare
    return bfc_prepare_batch(&u, &b, opt, stream, out);
}

extern "C" int bfc_sparsified_estimate(const uint64_t *sample_counts_dev, int32_t num_samples, double p,
                                       void *stream, double *estimate_dev) {
    bfc::set_last_error("");
    if (!sample_counts_dev || !estimate_dev || num_samples < 1) {
        bfc::set_last_error("null argument or num_samples < 1");
        return BFC_ERR_INVALID_ARGUMENT;
    }
    if (!(p > 0.0 && p <= 1.0)) { bfc::set_last_error("keep probability must lie in (0, 1]"); return BFC_ERR_INVALID_ARGUMENT; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    bfc::k_sp_estimate<<<1, bfc::kT, 0, s>>>(sample_counts_dev, num_samples, p, estimate_dev);
    bfc::note_launch();
    BFC_CUDA(cudaGetLastError());
    return BFC_OK;
}

extern "C" int bfc_estimate_sparsified(int32_t num_u, int32_t num_l, int64_t num_edges,
                                       const int32_t *off_u_dev, const int32_t *adj_u_dev, double p,
                                       uint64_t seed, int32_t num_samples, const bfc_options *opt,
                                       void *stream, uint64_t *sample_counts_dev, double *estimate_dev) {
    bfc::set_last_error("");
    if (!sample_counts_dev) { bfc::set_last_error("null argument"); return BFC_ERR_INVALID_ARGUMENT; }
    bfc_graph *g = nullptr;
    int rc = bfc_prepare_sparsified(num_u, num_l, num_edges, off_u_dev, adj_u_dev, p, seed, num_samples, opt,
                                    stream, nullptr, &g);
    if (rc != BFC_OK) return rc;
    rc = bfc_count_batch(g, stream, sample_counts_dev, nullptr);
    if (rc == BFC_OK && estimate_dev) rc = bfc_sparsified_estimate(sample_counts_dev, num_samples, p, stream, estimate_dev);
    const int rs = bfc_sync(g, stream);
    bfc_release(g);
    return rc != BFC_OK ? rc : rs;
}
