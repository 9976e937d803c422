// a3: stable LSD radix sort of (uint64 key, uint32 value) pairs and the
// per-tile [start, end) ranges of the sorted keys.
//
// One kernel reads the keys once and counts the digits of every pass (8-bit
// digits); a one-block kernel turns the counts into each pass's digit bases.
// Each pass is then a single kernel with a decoupled look-back: a block takes
// the next partition of 4096 pairs from a counter (partitions are handed out
// in launch order, so every predecessor is already running), ranks its items
// stably (warp match on the digit, per-warp running counters, prefix over
// warps), publishes its per-digit counts, reads its predecessors' published
// counts back to the first inclusive prefix (a bounded wait on each flag) to
// learn where its run of every digit starts, and writes its items out through
// shared memory so that runs of one digit leave the block as contiguous,
// coalesced stores. The number of passes is made even so the result ends in
// the caller's buffers.
#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace psi {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems; // 4096 pairs per block
constexpr int kBins = 256;

// Pair count of the call: *d_n clamped to the buffers' capacity (more pairs
// than the buffers hold is a capacity error, raised once by the first pass).
__device__ __forceinline__ int64_t clamped_count(const int64_t *d_n, int64_t cap)
{
    const int64_t n = *d_n;
    return n < 0 ? 0 : (n > cap ? cap : n);
}

constexpr int kMaxPasses = 8; // 64-bit keys in 8-bit digits

struct PassPlan {
    int passes;
    int shift[kMaxPasses];
    int bits[kMaxPasses];
};

// Digit counts of every pass in one read of the keys: per block in shared
// memory, then added to hist[pass][256] (zeroed by the caller).
__global__ void __launch_bounds__(kThreads) hist_kernel(const uint64_t *__restrict__ keys,
                                                        const int64_t *__restrict__ d_n, int64_t cap, PassPlan plan,
                                                        uint32_t *__restrict__ hist, DevStatus *status)
{
    __shared__ uint32_t h[kMaxPasses][kBins];
    for (int k = threadIdx.x; k < kMaxPasses * kBins; k += kThreads) (&h[0][0])[k] = 0;
    __syncthreads();
    const int64_t n = clamped_count(d_n, cap);
    if (status && blockIdx.x == 0 && threadIdx.x == 0 && *d_n > cap) {
        raise_status(status, PSI_ERR_CAPACITY);
        atomicMax(&status->required_pairs, static_cast<unsigned long long>(*d_n));
    }
    for (int64_t idx = static_cast<int64_t>(blockIdx.x) * kThreads + threadIdx.x; idx < n;
         idx += static_cast<int64_t>(gridDim.x) * kThreads) {
        const uint64_t k = keys[idx];
        for (int ps = 0; ps < plan.passes; ++ps) {
            const uint64_t mask = (1ull << plan.bits[ps]) - 1ull;
            atomicAdd(&h[ps][static_cast<uint32_t>((k >> plan.shift[ps]) & mask)], 1u);
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < plan.passes * kBins; k += kThreads) {
        const uint32_t c = (&h[0][0])[k];
        if (c) atomicAdd(hist + k, c);
    }
}

// hist[pass][256] -> exclusive prefix per pass, in place (one block)
__global__ void __launch_bounds__(kBins) digit_scan_kernel(uint32_t *hist, int passes)
{
    __shared__ uint32_t wsum[kBins / 32];
    const int d = threadIdx.x, lane = d & 31, w = d >> 5;
    for (int ps = 0; ps < passes; ++ps) {
        const uint32_t c = hist[ps * kBins + d];
        uint32_t inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        if (lane == 31) wsum[w] = inc;
        __syncthreads();
        uint32_t before = 0;
        for (int k = 0; k < w; ++k) before += wsum[k];
        hist[ps * kBins + d] = before + inc - c;
        __syncthreads();
    }
}

// look-back status word of (partition, digit), one array shared by the passes:
// flag in bits 62-63, the pass (1-based, up to 8) in bits 58-61, the count
// below; a word of an earlier pass reads as not yet published
constexpr unsigned long long kFlagAgg = 1ull << 62;  // this partition's own count
constexpr unsigned long long kFlagIncl = 2ull << 62; // count of all partitions up to this one
constexpr unsigned long long kTagMask = 15ull << 58;
constexpr unsigned long long kValueMask = (1ull << 58) - 1ull;
__device__ __forceinline__ unsigned long long pass_tag(int ps) { return static_cast<unsigned long long>(ps + 1) << 58; }

struct ScatterSmem {
    uint32_t warp_cnt[kWarps][kBins];
    uint32_t digit_start[kBins];       // start of each digit in the block's local order
    unsigned long long digit_base[kBins]; // global output offset of the block's first item of each digit
    uint32_t warp_tot[kWarps + 1];
    uint64_t xkeys[kTile];
    uint32_t xvals[kTile];
};

__global__ void __launch_bounds__(kThreads) onesweep_kernel(const uint64_t *__restrict__ keys_in,
                                                            const uint32_t *__restrict__ vals_in,
                                                            uint64_t *__restrict__ keys_out,
                                                            uint32_t *__restrict__ vals_out,
                                                            const int64_t *__restrict__ d_n, int64_t cap, int ps,
                                                            int shift, int bits, const uint32_t *__restrict__ digit_base,
                                                            unsigned long long *status_words,
                                                            unsigned int *part_counter, DevStatus *status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScatterSmem &S = *reinterpret_cast<ScatterSmem *>(smem_raw);
    __shared__ uint32_t s_part;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_part = atomicAdd(part_counter, 1u);
    __syncthreads();
    const int64_t part = s_part;
    const int64_t n = clamped_count(d_n, cap);
    const int64_t blk0 = part * kTile;
    if (blk0 >= n) return; // partitions are handed out in order: no valid one waits for this
    const uint64_t mask = (bits >= 64) ? ~0ull : ((1ull << bits) - 1ull);
    for (int k = threadIdx.x; k < kWarps * kBins; k += kThreads) (&S.warp_cnt[0][0])[k] = 0;
    __syncthreads();

    // warp-striped items: item i of lane l is at blk0 + wid*512 + i*32 + l
    uint64_t key[kItems];
    uint32_t val[kItems];
    uint32_t rank[kItems];
    const uint32_t lt = (1u << lane) - 1u;
    // all of the thread's loads first, so that they are in flight together
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int64_t idx = blk0 + wid * (32 * kItems) + i * 32 + lane;
        const bool ok = idx < n;
        key[i] = ok ? __ldcs(keys_in + idx) : 0ull;
        val[i] = ok ? __ldcs(vals_in + idx) : 0u;
    }
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int64_t idx = blk0 + wid * (32 * kItems) + i * 32 + lane;
        const bool ok = idx < n;
        const uint32_t d = ok ? static_cast<uint32_t>((key[i] >> shift) & mask) : (kBins + lane);
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = 0;
        if (ok) before = S.warp_cnt[wid][d];
        __syncwarp();
        if (ok && (peers & lt) == 0) S.warp_cnt[wid][d] = before + __popc(peers);
        __syncwarp();
        rank[i] = before + __popc(peers & lt);
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, and the block's digit count
    uint32_t cnt = 0;
    {
        const int d = threadIdx.x; // kThreads == kBins
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t c = S.warp_cnt[w][d];
            S.warp_cnt[w][d] = run;
            run += c;
        }
        cnt = run;
    }
    // publish this partition's count of digit d, then read the predecessors'
    // back to the first inclusive prefix: the block's run of digit d starts at
    // digit_base[d] + (items of digit d in all earlier partitions)
    {
        const int d = threadIdx.x;
        volatile unsigned long long *row = status_words + part * kBins;
        unsigned long long excl = 0;
        const unsigned long long tag = pass_tag(ps);
        if (part == 0) {
            row[d] = kFlagIncl | tag | cnt;
        } else {
            row[d] = kFlagAgg | tag | cnt;
            const unsigned long long limit = wait_limit(status);
            unsigned long long t0 = 0;
            for (int64_t q = part - 1; q >= 0;) {
                const unsigned long long w = reinterpret_cast<volatile unsigned long long *>(status_words)[q * kBins + d];
                if ((w & (kFlagAgg | kFlagIncl)) == 0 || (w & kTagMask) != tag) {
                    const unsigned long long now = global_ns();
                    if (t0 == 0) t0 = now;
                    else if (now - t0 > limit) {
                        if (status) {
                            atomicCAS(&status->wait_site, 0, kSiteSort);
                            raise_status(status, PSI_ERR_TIMEOUT);
                        }
                        break;
                    }
                    continue;
                }
                t0 = 0;
                excl += w & kValueMask;
                if (w & kFlagIncl) break;
                --q;
            }
            row[d] = kFlagIncl | tag | (excl + cnt);
        }
        S.digit_base[d] = static_cast<unsigned long long>(digit_base[d]) + excl;
    }
    // exclusive scan of the digit counts over the block (256 digits, one per thread)
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) S.warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const uint32_t t = lane < kWarps ? S.warp_tot[lane] : 0u;
        uint32_t ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += u;
        }
        if (lane < kWarps) S.warp_tot[lane] = ti - t;
    }
    __syncthreads();
    S.digit_start[threadIdx.x] = S.warp_tot[wid] + inc - cnt;
    __syncthreads();
    // local (block) position, exchange through shared memory
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const int64_t idx = blk0 + wid * (32 * kItems) + i * 32 + lane;
        if (idx < n) {
            const uint32_t d = static_cast<uint32_t>((key[i] >> shift) & mask);
            const uint32_t lp = S.digit_start[d] + S.warp_cnt[wid][d] + rank[i];
            S.xkeys[lp] = key[i];
            S.xvals[lp] = val[i];
        }
    }
    __syncthreads();
    const int nvalid = static_cast<int>(std::min<int64_t>(kTile, n - blk0));
    for (int j = threadIdx.x; j < nvalid; j += kThreads) {
        const uint64_t k = S.xkeys[j];
        const uint32_t d = static_cast<uint32_t>((k >> shift) & mask);
        const unsigned long long pos = S.digit_base[d] + static_cast<unsigned long long>(j - static_cast<int>(S.digit_start[d]));
        keys_out[pos] = k;
        vals_out[pos] = S.xvals[j];
    }
}

__global__ void __launch_bounds__(256) ranges_kernel(const uint64_t *__restrict__ keys, const int64_t *__restrict__ d_n,
                                                     int64_t cap, uint32_t *__restrict__ ranges, int64_t n_tiles,
                                                     DevStatus *status)
{
    const int64_t n = clamped_count(d_n, cap);
    const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t t = keys[i] >> 32;
    if (t >= static_cast<uint64_t>(n_tiles)) {
        raise_status(status, PSI_ERR_INVALID_ARG);
        return;
    }
    if (i == 0 || (keys[i - 1] >> 32) != t) ranges[2 * t] = static_cast<uint32_t>(i);
    if (i == n - 1 || (keys[i + 1] >> 32) != t) ranges[2 * t + 1] = static_cast<uint32_t>(i + 1);
}

// Launch order of the compositing CTAs: tiles by descending list length
// (64 buckets, two per octave; empty tiles last), so the longest tiles start
// first instead of forming the kernel's tail. Order inside a bucket is
// arbitrary (a schedule only: every tile's result is independent of it).
__device__ __forceinline__ int cost_bucket(uint32_t len)
{
    if (len == 0) return 63;
    const int l2 = 31 - __clz(len);
    const int half = (l2 > 0) ? static_cast<int>((len >> (l2 - 1)) & 1u) : 0;
    return 62 - min(2 * l2 + half, 62);
}

__global__ void __launch_bounds__(1024) tile_order_kernel(const uint32_t *__restrict__ ranges, int64_t n_tiles,
                                                          uint32_t *__restrict__ order)
{
    __shared__ unsigned int hist[64];
    if (threadIdx.x < 64) hist[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t t = threadIdx.x; t < n_tiles; t += blockDim.x)
        atomicAdd(&hist[cost_bucket(ranges[2 * t + 1] - ranges[2 * t])], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int run = 0;
        for (int b = 0; b < 64; ++b) {
            const unsigned int c = hist[b];
            hist[b] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int64_t t = threadIdx.x; t < n_tiles; t += blockDim.x) {
        const unsigned int pos = atomicAdd(&hist[cost_bucket(ranges[2 * t + 1] - ranges[2 * t])], 1u);
        order[pos] = static_cast<uint32_t>(t);
    }
}

} // namespace

namespace {
int64_t sort_partitions(int64_t capacity) { return (std::max<int64_t>(capacity, 1) + kTile - 1) / kTile; }
} // namespace

// alternate keys and values, then (zeroed per call) the digit counts of every
// pass, the partition counters and the look-back status words
size_t sort_workspace_bytes(int64_t capacity)
{
    const int64_t cap = std::max<int64_t>(capacity, 1);
    return align_up(cap * 8, 256) + align_up(cap * 4, 256) + align_up(kMaxPasses * kBins * 4 + kMaxPasses * 4, 256) +
           align_up(sort_partitions(cap) * kBins * 8, 256);
}

cudaError_t launch_sort(uint64_t *keys, uint32_t *vals, const int64_t *d_num_pairs, int64_t capacity, int begin_bit,
                        int end_bit, uint32_t *tile_ranges, int64_t n_tiles_total, void *ws, DevStatus *status,
                        cudaStream_t st)
{
    const int64_t cap = std::max<int64_t>(capacity, 1);
    const int64_t nparts = sort_partitions(cap);
    char *p = static_cast<char *>(ws);
    auto *alt_keys = reinterpret_cast<uint64_t *>(p);
    p += align_up(cap * 8, 256);
    auto *alt_vals = reinterpret_cast<uint32_t *>(p);
    p += align_up(cap * 4, 256);
    char *zero0 = p;
    auto *hist = reinterpret_cast<uint32_t *>(p);
    auto *counters = reinterpret_cast<unsigned int *>(p + kMaxPasses * kBins * 4);
    p += align_up(kMaxPasses * kBins * 4 + kMaxPasses * 4, 256);
    auto *status_words = reinterpret_cast<unsigned long long *>(p);
    p += align_up(nparts * kBins * 8, 256);
    cudaError_t e = cudaMemsetAsync(zero0, 0, static_cast<size_t>(p - zero0), st);
    if (e != cudaSuccess) return e;

    const int nbits = std::max(end_bit - begin_bit, 1);
    PassPlan plan{};
    plan.passes = std::max(2, (nbits + 7) / 8);
    if (plan.passes & 1) ++plan.passes;
    const int dbits = (nbits + plan.passes - 1) / plan.passes;
    for (int ps = 0; ps < plan.passes; ++ps) {
        const int shift = begin_bit + ps * dbits;
        const int bits = std::max(0, std::min(dbits, end_bit - shift));
        plan.shift[ps] = bits == 0 ? 0 : shift; // identity pass (keeps the pass count even)
        plan.bits[ps] = bits;
    }
    e = cudaFuncSetAttribute(onesweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sizeof(ScatterSmem)));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned hgrid = static_cast<unsigned>(std::max<int64_t>(1, std::min<int64_t>(nparts * kItems, sms * 8)));
    hist_kernel<<<hgrid, kThreads, 0, st>>>(keys, d_num_pairs, cap, plan, hist, status);
    digit_scan_kernel<<<1, kBins, 0, st>>>(hist, plan.passes);
    uint64_t *kin = keys, *kout = alt_keys;
    uint32_t *vin = vals, *vout = alt_vals;
    for (int ps = 0; ps < plan.passes; ++ps) {
        onesweep_kernel<<<static_cast<unsigned>(nparts), kThreads, sizeof(ScatterSmem), st>>>(
            kin, vin, kout, vout, d_num_pairs, cap, ps, plan.shift[ps], plan.bits[ps], hist + ps * kBins, status_words,
            counters + ps, status);
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    if (tile_ranges && n_tiles_total > 0) {
        e = cudaMemsetAsync(tile_ranges, 0, static_cast<size_t>(n_tiles_total) * 8, st);
        if (e != cudaSuccess) return e;
        ranges_kernel<<<static_cast<unsigned>((cap + 255) / 256), 256, 0, st>>>(keys, d_num_pairs, cap, tile_ranges,
                                                                               n_tiles_total, status);
        tile_order_kernel<<<1, 1024, 0, st>>>(tile_ranges, n_tiles_total, tile_ranges + 2 * n_tiles_total);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------
// Variant with library-owned scratch, for callers that cannot allocate device
// memory. The scratch is a file-scope device array: the driver allocates it
// when the module is loaded on a device and every device that loads the
// library keeps it until the process exits. Host code must not use the
// array's name as a pointer (on the host it names a host-side stand-in); the
// device address is looked up once per device with cudaGetSymbolAddress.
namespace {

constexpr size_t kNoAllocScratchBytes = PSI_SORT_NOALLOC_SCRATCH_BYTES; // 13 MiB: sort scratch for 2^20 pairs
static_assert(kNoAllocScratchBytes >= 12u * PSI_SORT_NOALLOC_MAX_PAIRS, "scratch must hold the alternate key and value buffers");
static __device__ __align__(256) unsigned char g_sort_scratch[kNoAllocScratchBytes];

std::mutex g_scratch_mu;
void *g_scratch_ptr[PSI_MAX_DEVICES_NOALLOC] = {};

} // namespace

cudaError_t launch_sort_noalloc(uint64_t *keys, uint32_t *vals, const int64_t *d_num_pairs, int64_t capacity,
                                int begin_bit, int end_bit, uint32_t *tile_ranges, int64_t n_tiles_total,
                                DevStatus *status, cudaStream_t st, const char **why)
{
    if (capacity > PSI_SORT_NOALLOC_MAX_PAIRS) {
        *why = "capacity exceeds PSI_SORT_NOALLOC_MAX_PAIRS (use psi_sort_keys with a caller workspace)";
        return cudaErrorInvalidValue;
    }
    if (sort_workspace_bytes(capacity) > kNoAllocScratchBytes) {
        *why = "static scratch too small for this capacity";
        return cudaErrorInvalidValue;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= PSI_MAX_DEVICES_NOALLOC) {
        *why = "device index beyond the no-allocation table";
        return cudaErrorInvalidValue;
    }
    void *ptr = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_ptr[dev]) {
            // first call on this device (the current device): look up the
            // array's device address; not capturable, so make this first call
            // outside any stream capture
            e = cudaGetSymbolAddress(&ptr, g_sort_scratch);
            if (e != cudaSuccess) {
                *why = "cudaGetSymbolAddress of the static sort scratch failed";
                return e;
            }
            g_scratch_ptr[dev] = ptr;
        }
        ptr = g_scratch_ptr[dev];
    }
    return launch_sort(keys, vals, d_num_pairs, capacity, begin_bit, end_bit, tile_ranges, n_tiles_total, ptr, status,
                       st);
}

} // namespace psi
