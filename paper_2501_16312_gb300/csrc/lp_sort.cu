// Global sorting and tiling (Sec. 3.2 "Global Sorting and Tiling"): exclusive
// scan of per-record tile counts, key emission, a hand-written stable LSD
// radix sort of 64-bit (tile << 32 | depth) keys over the used bits, and the
// per-tile ranges of the sorted list.
//
// Every kernel that depends on the tile-list length E reads it from device
// memory, so the same launch sequence works when E is only known on the
// device (inside a CUDA graph); the host supplies an upper bound for grids.
#include "lp_device.cuh"
#include "lp_internal.h"

namespace lp {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;   // 4096 elements per block

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive block scan of one value per thread; returns the block total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t& total) {
    __shared__ uint32_t warp_sums[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t incl = warp_incl_scan(x);
    if (lane == 31) warp_sums[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < kScanThreads / 32 ? warp_sums[lane] : 0u;
        s = warp_incl_scan(s);
        if (lane < kScanThreads / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    const uint32_t before = w > 0 ? warp_sums[w - 1] : 0u;
    total = warp_sums[kScanThreads / 32 - 1];
    __syncthreads();
    return before + incl - x;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ in, long long n,
                                                              uint32_t* __restrict__ block_sums) {
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += in[base + k];
    uint32_t total;
    block_excl_scan(s, total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

// Single block: exclusive scan of the block sums in place; total -> *sum_out.
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(uint32_t* __restrict__ sums, int nb,
                                                            uint32_t* __restrict__ sum_out) {
    uint32_t carry = 0;
    for (int base = 0; base < nb; base += kScanThreads) {
        const int i = base + threadIdx.x;
        const uint32_t x = i < nb ? sums[i] : 0u;
        uint32_t total;
        const uint32_t ex = block_excl_scan(x, total);
        if (i < nb) sums[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0 && sum_out) *sum_out = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t* __restrict__ in, long long n,
                                                            const uint32_t* __restrict__ block_off,
                                                            uint32_t* __restrict__ out) {
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? in[base + k] : 0u;
        s += v[k];
    }
    uint32_t total;
    uint32_t run = block_excl_scan(s, total) + block_off[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

// ------------------------------------------------------------- key emission
// Each record's tile rectangle is (first global tile id, row stride, width,
// height).  A lane writes the entries of a small rectangle itself; larger
// rectangles are written by the whole warp, one record at a time, so that a
// near-camera primitive covering thousands of tiles does not serialise on one
// thread and its writes stay coalesced.
constexpr uint32_t kEmitLaneMax = 8;

template <typename WriteFn>
__device__ __forceinline__ void emit_rect(const int4 t, long long off, uint32_t cnt, uint32_t first_q,
                                          uint32_t step, WriteFn write) {
    for (uint32_t q = first_q; q < cnt; q += step) {
        const uint32_t row = q / (uint32_t)t.z, col = q - row * (uint32_t)t.z;
        write(off + q, (uint32_t)t.x + row * (uint32_t)t.y + col);
    }
}

__global__ void __launch_bounds__(256) k_emit(const uint32_t* __restrict__ counts,
                                              const uint32_t* __restrict__ offsets,
                                              const int4* __restrict__ trect,
                                              const uint32_t* __restrict__ zbits,
                                              long long n_records, uint64_t* __restrict__ keys,
                                              uint32_t* __restrict__ vals, long long cap,
                                              int* __restrict__ status) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t cnt = 0;
    long long off = 0;
    int4 t = make_int4(0, 0, 0, 0);
    uint32_t z = 0;
    if (r < n_records) {
        cnt = counts[r];
        if (cnt) {
            off = offsets[r];
            if (off + cnt > cap) {
                atomicOr(status, kStatusCapacity);
                cnt = 0;
            } else {
                t = trect[r];
                z = zbits[r];
            }
        }
    }
    const bool have = cnt > 0;
    if (have && cnt <= kEmitLaneMax)
        emit_rect(t, off, cnt, 0, 1, [&](long long q, uint32_t tile) {
            keys[q] = ((uint64_t)tile << 32) | z;
            vals[q] = (uint32_t)r;
        });
    const int lane = threadIdx.x & 31;
    unsigned big = __ballot_sync(0xffffffffu, have && cnt > kEmitLaneMax);
    while (big) {
        const int src = __ffs(big) - 1;
        big &= big - 1;
        const uint32_t c = __shfl_sync(0xffffffffu, cnt, src);
        const long long o = __shfl_sync(0xffffffffu, off, src);
        const uint32_t zz = __shfl_sync(0xffffffffu, z, src);
        const long long rr = __shfl_sync(0xffffffffu, r, src);
        int4 tt;
        tt.x = __shfl_sync(0xffffffffu, t.x, src);
        tt.y = __shfl_sync(0xffffffffu, t.y, src);
        tt.z = __shfl_sync(0xffffffffu, t.z, src);
        tt.w = __shfl_sync(0xffffffffu, t.w, src);
        emit_rect(tt, o, c, lane, 32, [&](long long q, uint32_t tile) {
            keys[q] = ((uint64_t)tile << 32) | zz;
            vals[q] = (uint32_t)rr;
        });
    }
}

// ---------------------------------------------------------- LSD radix sort
// Digit width 8.  A block owns a contiguous chunk of kSortChunk items; warp w
// of the block owns the w-th contiguous sub-chunk, which keeps the pass
// stable: ranks follow (block, warp, round, lane) = input order.
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortPerWarp = 512;
constexpr int kSortChunk = kSortWarps * kSortPerWarp;   // 4096
constexpr int kRadix = 256;

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const K* __restrict__ keys,
                                                             const uint32_t* __restrict__ n_dev,
                                                             long long bound, int shift, int nblocks,
                                                             uint32_t* __restrict__ hist) {
    __shared__ uint32_t h[kRadix];
    h[threadIdx.x] = 0;
    __syncthreads();
    const long long n = n_dev ? min((long long)*n_dev, bound) : bound;
    const long long base = (long long)blockIdx.x * kSortChunk;
    for (int k = threadIdx.x; k < kSortChunk; k += kSortThreads) {
        const long long q = base + k;
        if (q < n) atomicAdd(&h[(uint32_t)(keys[q] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const K* __restrict__ kin, const uint32_t* __restrict__ vin,
    K* __restrict__ kout, uint32_t* __restrict__ vout, const uint32_t* __restrict__ n_dev,
    long long bound, int shift, int nblocks, const uint32_t* __restrict__ offs) {
    __shared__ uint32_t cnt[kSortWarps][kRadix];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long n = n_dev ? min((long long)*n_dev, bound) : bound;
    const long long wbase = (long long)blockIdx.x * kSortChunk + (long long)w * kSortPerWarp;
    for (int d = lane; d < kRadix; d += 32) cnt[w][d] = 0;
    __syncwarp();
    // per-warp digit counts
    for (int k = lane; k < kSortPerWarp; k += 32) {
        const long long q = wbase + k;
        if (q < n) atomicAdd(&cnt[w][(uint32_t)(kin[q] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    // running offsets: global digit base of this block + earlier warps' counts
    {
        const int d = threadIdx.x;   // kSortThreads == kRadix
        uint32_t run = offs[(size_t)d * nblocks + blockIdx.x];
#pragma unroll
        for (int ww = 0; ww < kSortWarps; ++ww) {
            const uint32_t c = cnt[ww][d];
            cnt[ww][d] = run;
            run += c;
        }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int k = 0; k < kSortPerWarp; k += 32) {
        const long long q = wbase + k + lane;
        const bool ok = q < n;
        K key = 0;
        uint32_t val = 0, digit = kRadix;   // out-of-range lanes form their own group
        if (ok) {
            key = kin[q];
            val = vin[q];
            digit = (uint32_t)(key >> shift) & (kRadix - 1);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, digit);
        const int rank = __popc(peers & lt);
        uint32_t pos = 0;
        if (ok) pos = cnt[w][digit] + rank;
        __syncwarp();
        if (ok && rank == 0) cnt[w][digit] += __popc(peers);
        __syncwarp();
        if (ok) {
            kout[pos] = key;
            vout[pos] = val;
        }
    }
}

// ------------------------------------------------ two-stage (depth, tile) sort
// Stage 1 orders the records by the binary32 bits of their centre depth
// (records that emit nothing get the largest key); stage 2 emits every record's
// tiles in that order with a 32-bit tile key and stably sorts the tile ids.
// Both sorts are stable, so entries end in (tile, depth, record) order --
// exactly the order of the one-pass 64-bit (tile << 32 | depth) sort.
__global__ void __launch_bounds__(256) k_depth_keys(const uint32_t* __restrict__ counts,
                                                    const uint32_t* __restrict__ zbits, long long n,
                                                    uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    keys[r] = counts[r] ? zbits[r] : 0xffffffffu;
    vals[r] = (uint32_t)r;
}

__global__ void __launch_bounds__(256) k_gather_counts(const uint32_t* __restrict__ counts,
                                                       const uint32_t* __restrict__ order, long long n,
                                                       uint32_t* __restrict__ out) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) out[k] = counts[order[k]];
}

__global__ void __launch_bounds__(256) k_emit_sorted(const uint32_t* __restrict__ order,
                                                     const uint32_t* __restrict__ counts_sorted,
                                                     const uint32_t* __restrict__ offsets,
                                                     const int4* __restrict__ trect,
                                                     long long n_records, uint32_t* __restrict__ keys,
                                                     uint32_t* __restrict__ vals, long long cap,
                                                     int* __restrict__ status) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t cnt = 0, r = 0;
    long long off = 0;
    int4 t = make_int4(0, 0, 0, 0);
    if (k < n_records) {
        cnt = counts_sorted[k];
        if (cnt) {
            off = offsets[k];
            if (off + cnt > cap) {
                atomicOr(status, kStatusCapacity);
                cnt = 0;
            } else {
                r = order[k];
                t = trect[r];
            }
        }
    }
    const bool have = cnt > 0;
    if (have && cnt <= kEmitLaneMax)
        emit_rect(t, off, cnt, 0, 1, [&](long long q, uint32_t tile) {
            keys[q] = tile;
            vals[q] = r;
        });
    const int lane = threadIdx.x & 31;
    unsigned big = __ballot_sync(0xffffffffu, have && cnt > kEmitLaneMax);
    while (big) {
        const int src = __ffs(big) - 1;
        big &= big - 1;
        const uint32_t c = __shfl_sync(0xffffffffu, cnt, src);
        const long long o = __shfl_sync(0xffffffffu, off, src);
        const uint32_t rr = __shfl_sync(0xffffffffu, r, src);
        int4 tt;
        tt.x = __shfl_sync(0xffffffffu, t.x, src);
        tt.y = __shfl_sync(0xffffffffu, t.y, src);
        tt.z = __shfl_sync(0xffffffffu, t.z, src);
        tt.w = __shfl_sync(0xffffffffu, t.w, src);
        emit_rect(tt, o, c, lane, 32, [&](long long q, uint32_t tile) {
            keys[q] = tile;
            vals[q] = rr;
        });
    }
}

// Skipped entirely when the emission overflowed: the list then holds stale
// entries whose tile ids need not be valid, and all ranges stay empty.
template <typename K, int SHIFT>
__global__ void __launch_bounds__(256) k_ranges(const K* __restrict__ keys,
                                                const uint32_t* __restrict__ n_dev, long long bound,
                                                const int* __restrict__ status,
                                                uint2* __restrict__ ranges) {
    if (*status & kStatusCapacity) return;
    const long long n = min((long long)*n_dev, bound);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const uint32_t t = (uint32_t)(keys[i] >> SHIFT);
        if (i == 0 || (uint32_t)(keys[i - 1] >> SHIFT) != t) ranges[t].x = (uint32_t)i;
        if (i == n - 1 || (uint32_t)(keys[i + 1] >> SHIFT) != t) ranges[t].y = (uint32_t)(i + 1);
    }
}

}  // namespace

int scan_blocks(long long n) { return (int)((n + kScanTile - 1) / kScanTile); }

cudaError_t launch_scan(const uint32_t* in, long long n, uint32_t* out, uint32_t* block_sums,
                        uint32_t* total, cudaStream_t st) {
    const int nb = scan_blocks(n);
    if (nb == 0) {
        if (total) return cudaMemsetAsync(total, 0, sizeof(uint32_t), st);
        return cudaSuccess;
    }
    k_scan_reduce<<<nb, kScanThreads, 0, st>>>(in, n, block_sums);
    k_scan_sums<<<1, kScanThreads, 0, st>>>(block_sums, nb, total);
    k_scan_down<<<nb, kScanThreads, 0, st>>>(in, n, block_sums, out);
    return cudaGetLastError();
}

cudaError_t launch_emit(const uint32_t* counts, const uint32_t* offsets, const int4* trect,
                        const uint32_t* zbits, int n, long long n_records, const CamsParam& cams,
                        uint64_t* keys, uint32_t* vals, long long cap, int* status, cudaStream_t st) {
    (void)n;
    (void)cams;
    if (n_records == 0) return cudaSuccess;
    const int grid = (int)((n_records + 255) / 256);
    k_emit<<<grid, 256, 0, st>>>(counts, offsets, trect, zbits, n_records, keys, vals, cap, status);
    return cudaGetLastError();
}

int sort_blocks(long long bound) { return (int)((bound + kSortChunk - 1) / kSortChunk); }

template <typename K>
static cudaError_t radix_sort_t(K* k0, uint32_t* v0, K* k1, uint32_t* v1, const uint32_t* n_dev,
                                long long bound, int key_bits, uint32_t* hist, uint32_t* scan_tmp,
                                int* passes_out, cudaStream_t st) {
    const int nb = sort_blocks(bound);
    int passes = 0;
    if (nb > 0) {
        K* kin = k0; uint32_t* vin = v0;
        K* kout = k1; uint32_t* vout = v1;
        for (int shift = 0; shift < key_bits; shift += 8) {
            k_radix_hist<K><<<nb, kSortThreads, 0, st>>>(kin, n_dev, bound, shift, nb, hist);
            cudaError_t e = launch_scan(hist, (long long)kRadix * nb, hist, scan_tmp, nullptr, st);
            if (e != cudaSuccess) return e;
            k_radix_scatter<K><<<nb, kSortThreads, 0, st>>>(kin, vin, kout, vout, n_dev, bound, shift, nb,
                                                            hist);
            K* tk = kin; kin = kout; kout = tk;
            uint32_t* tv = vin; vin = vout; vout = tv;
            ++passes;
        }
    }
    *passes_out = passes;
    return cudaGetLastError();
}

cudaError_t launch_radix_sort(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1,
                              const uint32_t* n_dev, long long bound, int key_bits,
                              uint32_t* hist, uint32_t* scan_tmp, int* passes_out, cudaStream_t st) {
    return radix_sort_t<uint64_t>(k0, v0, k1, v1, n_dev, bound, key_bits, hist, scan_tmp, passes_out, st);
}

cudaError_t launch_radix_sort32(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1,
                                const uint32_t* n_dev, long long bound, int key_bits,
                                uint32_t* hist, uint32_t* scan_tmp, int* passes_out, cudaStream_t st) {
    return radix_sort_t<uint32_t>(k0, v0, k1, v1, n_dev, bound, key_bits, hist, scan_tmp, passes_out, st);
}

size_t sort_hist_elems(long long bound) { return (size_t)kRadix * (size_t)sort_blocks(bound); }

cudaError_t launch_depth_keys(const uint32_t* counts, const uint32_t* zbits, long long n, uint32_t* keys,
                              uint32_t* vals, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_depth_keys<<<(int)((n + 255) / 256), 256, 0, st>>>(counts, zbits, n, keys, vals);
    return cudaGetLastError();
}

cudaError_t launch_gather_counts(const uint32_t* counts, const uint32_t* order, long long n, uint32_t* out,
                                 cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_gather_counts<<<(int)((n + 255) / 256), 256, 0, st>>>(counts, order, n, out);
    return cudaGetLastError();
}

cudaError_t launch_emit_sorted(const uint32_t* order, const uint32_t* counts_sorted, const uint32_t* offsets,
                               const int4* trect, int n, long long n_records, const CamsParam& cams,
                               uint32_t* keys, uint32_t* vals, long long cap, int* status, cudaStream_t st) {
    (void)n;
    (void)cams;
    if (n_records == 0) return cudaSuccess;
    k_emit_sorted<<<(int)((n_records + 255) / 256), 256, 0, st>>>(order, counts_sorted, offsets, trect,
                                                                  n_records, keys, vals, cap, status);
    return cudaGetLastError();
}

static int ranges_grid(long long bound, int sms) {
    const long long want = (bound + 255) / 256;
    return (int)(want < (long long)sms * 8 ? want : (long long)sms * 8);
}

cudaError_t launch_ranges(const uint64_t* keys, const uint32_t* n_dev, long long bound,
                          const int* status, uint2* ranges, int sms, cudaStream_t st) {
    if (bound == 0) return cudaSuccess;
    k_ranges<uint64_t, 32><<<ranges_grid(bound, sms), 256, 0, st>>>(keys, n_dev, bound, status, ranges);
    return cudaGetLastError();
}

cudaError_t launch_ranges32(const uint32_t* keys, const uint32_t* n_dev, long long bound,
                            const int* status, uint2* ranges, int sms, cudaStream_t st) {
    if (bound == 0) return cudaSuccess;
    k_ranges<uint32_t, 0><<<ranges_grid(bound, sms), 256, 0, st>>>(keys, n_dev, bound, status, ranges);
    return cudaGetLastError();
}

}  // namespace lp
