// a2: tile intersection and (tile|depth, record) key emission, plus the
// device-wide exclusive scan it needs.
//
// After the scan of per-record tile counts, every visible record writes one
// pair per touched tile, in record order, tiles row-major: key =
// (global tile << 32) | float bits of the camera depth (positive, so the bit
// pattern orders like the value), value = record index. Which tiles a record
// touches is decided by the same float32 sequence that counted them (Sec. 5,
// Precise Tile Intersection; EXACT refines each tile row to the ellipse).
#include "discrete.cuh"

namespace psi {

// ------------------------------------------------------------------ scan
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems; // 4096

template <typename T>
__device__ __forceinline__ T block_exclusive_sum(T v, T *warp_tot, T &block_total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T n = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += n;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        T t = lane < (kScanThreads / 32) ? warp_tot[lane] : T(0);
        T ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T n = __shfl_up_sync(0xffffffffu, ti, o);
            if (lane >= o) ti += n;
        }
        if (lane < (kScanThreads / 32)) warp_tot[lane] = ti - t;
        if (lane == (kScanThreads / 32) - 1) warp_tot[kScanThreads / 32] = ti;
    }
    __syncthreads();
    const T res = warp_tot[wid] + inc - v;
    block_total = warp_tot[kScanThreads / 32];
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const uint32_t *__restrict__ in, int64_t n,
                                                                   unsigned long long *__restrict__ block_sums)
{
    __shared__ unsigned long long warp_tot[kScanThreads / 32 + 1];
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile;
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t idx = base + static_cast<int64_t>(k) * kScanThreads + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    unsigned long long tot;
    block_exclusive_sum<unsigned long long>(s, warp_tot, tot);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// one block: exclusive scan of the block sums (any count, chunked), total out
__global__ void __launch_bounds__(kScanThreads) scan_blocks_kernel(unsigned long long *__restrict__ sums, int64_t nb,
                                                                   unsigned long long *__restrict__ d_total)
{
    __shared__ unsigned long long warp_tot[kScanThreads / 32 + 1];
    unsigned long long carry = 0;
    for (int64_t c = 0; c < nb; c += kScanThreads) {
        const int64_t idx = c + threadIdx.x;
        const unsigned long long v = idx < nb ? sums[idx] : 0ull;
        unsigned long long tot;
        const unsigned long long ex = block_exclusive_sum<unsigned long long>(v, warp_tot, tot);
        if (idx < nb) sums[idx] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *d_total = carry;
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const uint32_t *__restrict__ in, int64_t n,
                                                                  const unsigned long long *__restrict__ block_off,
                                                                  unsigned long long *__restrict__ out)
{
    __shared__ unsigned long long warp_tot[kScanThreads / 32 + 1];
    // blocked arrangement: thread t owns items [t*16, t*16+16) of the tile
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + static_cast<int64_t>(threadIdx.x) * kScanItems;
    uint32_t v[kScanItems];
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0u;
        s += v[k];
    }
    unsigned long long tot;
    unsigned long long run = block_exclusive_sum<unsigned long long>(s, warp_tot, tot) + block_off[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

} // namespace

size_t scan_workspace_bytes(int64_t n)
{
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    return align_up(static_cast<size_t>(std::max<int64_t>(nb, 1)) * 8, 256);
}

cudaError_t launch_scan_u32(const uint32_t *in, unsigned long long *out, int64_t n, unsigned long long *d_total,
                            void *ws, cudaStream_t st)
{
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    auto *sums = static_cast<unsigned long long *>(ws);
    if (nb == 0) {
        return cudaMemsetAsync(d_total, 0, 8, st);
    }
    scan_reduce_kernel<<<static_cast<unsigned>(nb), kScanThreads, 0, st>>>(in, n, sums);
    scan_blocks_kernel<<<1, kScanThreads, 0, st>>>(sums, nb, d_total);
    if (out) scan_apply_kernel<<<static_cast<unsigned>(nb), kScanThreads, 0, st>>>(in, n, sums, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ emit
namespace {

using namespace disc;

__global__ void finalize_count_kernel(const unsigned long long *__restrict__ total, int64_t capacity,
                                      int64_t *__restrict__ d_num_pairs, DevStatus *status)
{
    const unsigned long long t = *total;
    if (t > static_cast<unsigned long long>(capacity)) {
        raise_status(status, PSI_ERR_CAPACITY);
        atomicMax(&status->required_pairs, t);
        *d_num_pairs = capacity;
    } else {
        *d_num_pairs = static_cast<int64_t>(t);
    }
}

__global__ void __launch_bounds__(256) emit_kernel(const __grid_constant__ FrameParams fp,
                                                   const float4 *__restrict__ bins, const uint32_t *__restrict__ counts,
                                                   const unsigned long long *__restrict__ offsets,
                                                   uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                                                   int64_t capacity)
{
    const int64_t total = fp.n * fp.n_views;
    const int64_t r = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (r >= total) return;
    const uint32_t cnt = counts[r];
    if (cnt == 0) return;
    unsigned long long off = offsets[r];
    if (off >= static_cast<unsigned long long>(capacity)) return;
    const int v = static_cast<int>(r / fp.n);
    const ViewParams &cam = fp.v[v];
    float depth;
    const bool lp = fp.lowpass != 0;
    const Bin b = load_bin(bins + bin_stride(lp) * r, depth, lp);
    const uint64_t dbits = __float_as_uint(depth);
    const int tw = fp.tile_w, th = fp.tile_h;
    const uint32_t val = static_cast<uint32_t>(r);
    for (int ty = b.py0 / th; ty <= b.py1 / th; ++ty) {
        int c0, c1;
        if (!row_tiles(b, fp.mode, ty, tw, th, c0, c1)) continue;
        const uint32_t rowbase = cam.tile_base + static_cast<uint32_t>(ty * cam.tiles_x);
        for (int tx = c0; tx <= c1; ++tx) {
            if (off >= static_cast<unsigned long long>(capacity)) return;
            keys[off] = (static_cast<uint64_t>(rowbase + static_cast<uint32_t>(tx)) << 32) | dbits;
            vals[off] = val;
            ++off;
        }
    }
}

} // namespace

size_t intersect_workspace_bytes(int64_t n_records)
{
    return align_up(static_cast<size_t>(std::max<int64_t>(n_records, 1)) * 8, 256) + scan_workspace_bytes(n_records) +
           256;
}

cudaError_t launch_intersect(const FrameParams &fp, const float4 *bin_records, const uint32_t *tiles_touched,
                             uint64_t *keys, uint32_t *vals, int64_t capacity, int64_t *d_num_pairs, void *ws,
                             DevStatus *status, cudaStream_t st)
{
    const int64_t R = fp.n * fp.n_views;
    char *p = static_cast<char *>(ws);
    auto *offsets = reinterpret_cast<unsigned long long *>(p);
    p += align_up(static_cast<size_t>(std::max<int64_t>(R, 1)) * 8, 256);
    void *scan_ws = p;
    p += scan_workspace_bytes(R);
    auto *total = reinterpret_cast<unsigned long long *>(p);
    cudaError_t e = launch_scan_u32(tiles_touched, offsets, R, total, scan_ws, st);
    if (e != cudaSuccess) return e;
    finalize_count_kernel<<<1, 1, 0, st>>>(total, capacity, d_num_pairs, status);
    if (R > 0) {
        emit_kernel<<<static_cast<unsigned>((R + 255) / 256), 256, 0, st>>>(fp, bin_records, tiles_touched, offsets,
                                                                           keys, vals, capacity);
    }
    return cudaGetLastError();
}

} // namespace psi
