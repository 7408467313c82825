// Global sorting and tiling (Sec. 3.2 "Global Sorting and Tiling"): exclusive
// scan of per-record tile counts, key emission, a hand-written stable LSD
// radix sort of 64-bit (tile << 32 | depth) keys over the used bits, and the
// per-tile ranges of the sorted list.
//
// Every kernel that depends on the tile-list length E reads it from device
// memory, so the same launch sequence works when E is only known on the
// device (inside a CUDA graph); the host supplies an upper bound for grids.
#include <atomic>
#include <cstdint>

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

// A thread's kScanItems consecutive elements, with 16-byte loads when the
// whole run is in range and the array is 16-byte aligned.
__device__ __forceinline__ void scan_load(const uint32_t* __restrict__ in, long long n, long long base,
                                          bool vec, uint32_t v[kScanItems]) {
    if (vec && base + kScanItems <= n) {
        const uint4* p = reinterpret_cast<const uint4*>(in + base);
#pragma unroll
        for (int k = 0; k < kScanItems / 4; ++k) {
            const uint4 x = p[k];
            v[4 * k] = x.x; v[4 * k + 1] = x.y; v[4 * k + 2] = x.z; v[4 * k + 3] = x.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) v[k] = base + k < n ? in[base + k] : 0u;
    }
}

// Sum of one 64-bit value per thread over the block (every thread gets it).
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long x) {
    __shared__ unsigned long long warp_tot[kScanThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) warp_tot[w] = x;
    __syncthreads();
    unsigned long long t = 0;
#pragma unroll
    for (int k = 0; k < kScanThreads / 32; ++k) t += warp_tot[k];
    __syncthreads();
    return t;
}

// Block totals in 64 bits, saturated to 2^32 - 1 (a block of 4096 counts
// can exceed 32 bits; the sums kernel then reports the overflow).
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ in, long long n,
                                                              uint32_t* __restrict__ block_sums) {
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    scan_load(in, n, base, ((uintptr_t)in & 15) == 0, v);
    unsigned long long s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) s += v[k];
    const unsigned long long total = block_sum_u64(s);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total < kListOverflow ? (uint32_t)total : kListOverflow;
}

// Single block: exclusive scan of the block sums in place; the total goes to
// *sum_out.  The running total is kept in 64 bits: once it reaches 2^32 - 1
// the offsets have wrapped, so *sum_out gets kListOverflow and, when status
// is given, kStatusCapacity is latched.
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(uint32_t* __restrict__ sums, int nb,
                                                            uint32_t* __restrict__ sum_out,
                                                            int* __restrict__ status) {
    unsigned long long carry = 0;
    for (int base = 0; base < nb; base += kScanThreads) {
        const int i = base + threadIdx.x;
        const uint32_t x = i < nb ? sums[i] : 0u;
        uint32_t total;
        const uint32_t ex = block_excl_scan(x, total);
        if (i < nb) sums[i] = (uint32_t)carry + ex;
        carry += block_sum_u64(x);
    }
    if (threadIdx.x == 0 && sum_out) {
        if (carry >= kListOverflow) {
            *sum_out = kListOverflow;
            if (status) atomicOr(status, kStatusCapacity);
        } else {
            *sum_out = (uint32_t)carry;
        }
    }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t* __restrict__ in, long long n,
                                                            const uint32_t* __restrict__ block_off,
                                                            uint32_t* __restrict__ out) {
    const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    const bool vec = (((uintptr_t)in | (uintptr_t)out) & 15) == 0;
    uint32_t v[kScanItems];
    scan_load(in, n, base, vec, v);
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) s += v[k];
    uint32_t total;
    uint32_t run = block_excl_scan(s, total) + block_off[blockIdx.x];
    if (vec && base + kScanItems <= n) {
        uint4* p = reinterpret_cast<uint4*>(out + base);
#pragma unroll
        for (int k = 0; k < kScanItems / 4; ++k) {
            uint4 x;
            x.x = run; run += v[4 * k];
            x.y = run; run += v[4 * k + 1];
            x.z = run; run += v[4 * k + 2];
            x.w = run; run += v[4 * k + 3];
            p[k] = x;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (base + k < n) out[base + k] = run;
            run += v[k];
        }
    }
}

// ------------------------------------------------------------- key emission
// Each record's tile rectangle is (first global tile id, row stride, width,
// height); its entries occupy [offset, offset + count) of the list.  Work is
// split by merge path over records and entries together: record k sits at
// merged position k + offset[k], entry j after every record starting at or
// before j, and block b takes merged positions [b T, (b + 1) T).  So a block
// writes at most T entries however unevenly tiles are spread over records (in
// depth order the near-camera records covering thousands of tiles come
// together), and its writes are coalesced: thread t writes entries j0 + t,
// j0 + t + 256, ... and finds the owning record by binary search over the
// block's record offsets in shared memory.
constexpr int kEmitBlock = 256;
constexpr int kEmitItems = 1024;   // T: records + entries per block

// part[b] = number of records whose merged position precedes b T.
__global__ void __launch_bounds__(256) k_emit_partition(const uint32_t* __restrict__ offsets, long long R,
                                                        const uint32_t* __restrict__ n_dev, long long bound,
                                                        int nb, uint32_t* __restrict__ part) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nb) return;
    if (*n_dev == kListOverflow) return;   // offsets wrapped: nothing is emitted
    const long long E = min((long long)*n_dev, bound);
    const long long d = min((long long)b * kEmitItems, R + E);
    long long lo = 0, hi = R;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (mid + (long long)offsets[mid] < d) lo = mid + 1;
        else hi = mid;
    }
    part[b] = (uint32_t)lo;
}

// SORTED: the key is the 32-bit tile id, and list position k holds record
// order[k] (stage 2 of the two-stage sort), or record k when order is null
// (the per-tile sort); otherwise position k is record k and the key is
// (tile << 32) | depth bits.
template <bool SORTED>
__global__ void __launch_bounds__(kEmitBlock) k_emit_lb(const uint32_t* __restrict__ order,
                                                        const uint32_t* __restrict__ counts,
                                                        const uint32_t* __restrict__ offsets,
                                                        const int4* __restrict__ trect,
                                                        const uint32_t* __restrict__ zbits, long long R,
                                                        const uint32_t* __restrict__ n_dev, long long bound,
                                                        const uint32_t* __restrict__ part,
                                                        uint32_t* __restrict__ keys32,
                                                        uint64_t* __restrict__ keys64,
                                                        uint32_t* __restrict__ vals, long long cap,
                                                        int* __restrict__ status) {
    __shared__ uint32_t s_off[kEmitItems + 1];
    __shared__ int4 s_rect[kEmitItems + 1];
    __shared__ uint32_t s_rec[kEmitItems + 1];
    __shared__ uint32_t s_z[SORTED ? 1 : kEmitItems + 1];
    const int b = blockIdx.x, tid = threadIdx.x;
    const long long Ed = (long long)*n_dev;
    if (Ed == kListOverflow) return;         // latched by the scan; offsets wrapped
    if (b == 0 && tid == 0 && Ed > cap) atomicOr(status, kStatusCapacity);
    const long long E = min(Ed, bound);
    const long long d0 = (long long)b * kEmitItems;
    if (d0 >= R + E) return;   // uniform over the block
    const long long d1 = min(d0 + kEmitItems, R + E);
    const long long i0 = part[b], i1 = part[b + 1];
    const long long j0 = d0 - i0, j1 = min(d1 - i1, cap);
    // the record owning entry j0 may start before d0: records ks .. i1 - 1
    const long long ks = i0 > 0 ? i0 - 1 : 0;
    const int nrec = (int)(i1 - ks);   // <= kEmitItems + 1
    for (int t = tid; t < nrec; t += kEmitBlock) {
        const long long k = ks + t;
        const uint32_t cnt = counts[k];
        const uint32_t r = SORTED && order ? order[k] : (uint32_t)k;
        s_off[t] = offsets[k];
        s_rec[t] = r;
        if (cnt) {
            s_rect[t] = trect[r];
            if (!SORTED) s_z[t] = zbits[r];
        }
    }
    __syncthreads();
    for (long long j = j0 + tid; j < j1; j += kEmitBlock) {
        // the last record whose offset is <= j owns entry j (records with no
        // tiles share their offset with the next record)
        const uint32_t ju = (uint32_t)j;
        int lo = 0, hi = nrec - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= ju) lo = mid;
            else hi = mid - 1;
        }
        const int4 t = s_rect[lo];
        const uint32_t q = ju - s_off[lo];
        const uint32_t row = q / (uint32_t)t.z, col = q - row * (uint32_t)t.z;
        const uint32_t tile = (uint32_t)t.x + row * (uint32_t)t.y + col;
        if (SORTED) keys32[j] = tile;
        else keys64[j] = ((uint64_t)tile << 32) | s_z[lo];
        vals[j] = s_rec[lo];
    }
}

// ---------------------------------------------------------- LSD radix sort
// Digit width RB = 4, 6, 8 or 11 bits (a tuning choice).  A block owns a
// contiguous chunk of kSortChunk items; warp w of the block owns the w-th
// contiguous sub-chunk, which keeps the pass stable: ranks follow (block,
// warp, round, lane) = input order.
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortPerWarp = 512;
constexpr int kSortChunk = kSortWarps * kSortPerWarp;   // 4096
constexpr int kScatterIPT = kSortPerWarp / 32;   // items per lane
constexpr int kRadixMaxBits = 11;
// onesweep status words: flag in the top two bits, a count below
constexpr uint32_t kFlagAgg = 1u << 30, kFlagInc = 2u << 30, kFlagMask = 3u << 30, kValMask = (1u << 30) - 1u;
constexpr long long kSweepWaitCycles = 2000000000ll;   // about a second: bound of one look-back wait
constexpr long long kSweepMaxItems = 1ll << 30;         // counts must fit in the status words
constexpr int kLookWindow = 8;                          // earlier blocks read per look-back step

// Digit counts of one block's chunk: each warp counts its sub-chunk into its
// own shared histogram (less contention than one histogram per block); with
// 11-bit digits the block shares one histogram (the bins rarely collide).
template <typename K, int RB>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const K* __restrict__ keys,
                                                             const uint32_t* __restrict__ n_dev,
                                                             long long bound, int shift, int nblocks,
                                                             uint32_t* __restrict__ hist) {
    constexpr int R = 1 << RB;
    constexpr int NH = RB > 8 ? 1 : kSortWarps;
    __shared__ uint32_t h[NH][R];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int d = tid; d < NH * R; d += kSortThreads) (&h[0][0])[d] = 0;
    __syncthreads();
    const long long n = n_dev ? list_len(n_dev, bound) : bound;
    const long long wbase = (long long)blockIdx.x * kSortChunk + (long long)w * kSortPerWarp;
    uint32_t dig[kScatterIPT];
#pragma unroll
    for (int r = 0; r < kScatterIPT; ++r) {
        const long long q = wbase + r * 32 + lane;
        dig[r] = q < n ? ((uint32_t)(keys[q] >> shift) & (R - 1)) : (uint32_t)R;
    }
#pragma unroll
    for (int r = 0; r < kScatterIPT; ++r)
        if (dig[r] < R) atomicAdd(&h[NH > 1 ? w : 0][dig[r]], 1u);
    __syncthreads();
    for (int d = tid; d < R; d += kSortThreads) {
        uint32_t t = 0;
#pragma unroll
        for (int ww = 0; ww < NH; ++ww) t += h[ww][d];
        hist[(size_t)d * nblocks + blockIdx.x] = t;
    }
}

// Lanes of the warp whose digit equals this lane's (digits < 2^(RB+1); the
// value 2^RB marks "no item"): one ballot per digit bit.  Measured faster than
// __match_any_sync on sm_103 when the kernel streams from DRAM.
template <int RB>
__device__ __forceinline__ unsigned digit_peers(uint32_t d) {
    unsigned m = 0xffffffffu;
#pragma unroll
    for (int b = 0; b <= RB; ++b) {
        const unsigned bit = (d >> b) & 1u;
        const unsigned bb = __ballot_sync(0xffffffffu, bit);
        m &= bit ? bb : ~bb;
    }
    return m;
}

// One pass of the stable scatter.  Each warp ranks its 512 items round by
// round (digit_peers groups equal digits; a per-warp counter per digit gives
// the running rank), the block turns the (warp, digit) counts into block-local
// starts in digit order, the items are placed in shared memory in that order,
// and the block writes them out in index order: consecutive threads then write
// consecutive addresses of each digit's run.  Keys and values are read once.

template <typename K, int RB>
constexpr size_t scatter_smem_bytes() {
    return (size_t)kSortChunk * (sizeof(K) + sizeof(uint32_t)) + (size_t)kSortWarps * (1 << RB) * 4 +
           (size_t)(1 << RB) * 4;
}

// SWEEP (one pass of the onesweep form): blocks take their chunk by a
// dynamic block id, so that a block only ever waits for blocks that have
// started, publish their digit counts, and find the counts of all earlier
// blocks by decoupled look-back; the digits' global starts come from the
// histogram of all passes made up front.  Otherwise offs holds the scanned
// (digit, block) histogram of this pass.
template <typename K, int RB, bool SWEEP>
__global__ void __launch_bounds__(kSortThreads, sizeof(K) == 4 ? 4 : 3) k_radix_scatter(
    const K* __restrict__ kin, const uint32_t* __restrict__ vin,
    K* __restrict__ kout, uint32_t* __restrict__ vout, const uint32_t* __restrict__ n_dev,
    long long bound, int shift, int nblocks, const uint32_t* __restrict__ offs,
    const uint32_t* __restrict__ digit_base, uint32_t* __restrict__ status, uint32_t* __restrict__ counter,
    int* __restrict__ err, int stall_block) {
    constexpr int R = 1 << RB;
    constexpr uint32_t DMASK = (2u << RB) - 1u;        // digit field of a packed item (sentinel included)
    constexpr int DPT = R > kSortThreads ? R / kSortThreads : 1;   // digits per thread in the block scan
    extern __shared__ __align__(16) unsigned char smem[];
    K* skeys = reinterpret_cast<K*>(smem);
    uint32_t* svals = reinterpret_cast<uint32_t*>(smem + sizeof(K) * kSortChunk);
    uint32_t* wcnt = svals + kSortChunk;       // [kSortWarps][R]
    uint32_t* gbase = wcnt + kSortWarps * R;   // [R]
    __shared__ uint32_t wsum[kSortWarps];
    __shared__ uint32_t s_bid;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const long long n = n_dev ? list_len(n_dev, bound) : bound;
    uint32_t bid = blockIdx.x;
    if constexpr (SWEEP) {
        if (tid == 0) s_bid = atomicAdd(counter, 1u);
        __syncthreads();
        bid = s_bid;
    }
    const long long bbase = (long long)bid * kSortChunk;
    if (bbase >= n) return;   // uniform over the block (never waited for: its id is past every chunk)
    for (int d = lane; d < R; d += 32) wcnt[w * R + d] = 0;
    __syncwarp();

    const long long wbase = bbase + (long long)w * kSortPerWarp;
    K key[kScatterIPT];
    uint32_t pk[kScatterIPT];   // pk = digit | warp-local rank << (RB + 1)
#pragma unroll
    for (int r = 0; r < kScatterIPT; ++r) {
        const long long q = wbase + r * 32 + lane;
        const bool ok = q < n;
        key[r] = ok ? kin[q] : K(0);
        pk[r] = ok ? ((uint32_t)(key[r] >> shift) & (R - 1)) : (uint32_t)R;   // R: no item
    }
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kScatterIPT; ++r) {
        const uint32_t d = pk[r];
        const unsigned peers = digit_peers<RB>(d);
        const uint32_t rank = __popc(peers & lt);
        uint32_t base = 0;
        if (d < R) base = wcnt[w * R + d];
        __syncwarp();
        if (d < R && rank == 0) wcnt[w * R + d] = base + __popc(peers);
        __syncwarp();
        pk[r] = d | ((base + rank) << (RB + 1));
    }
    __syncthreads();

    // thread t: digits [t DPT, t DPT + DPT): starts of (warp, d) within digit
    // d, the digits' totals, then the block-local start of each digit
    uint32_t tot[DPT];
    uint32_t tsum = 0;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        const int d = tid * DPT + q;
        uint32_t run = 0;
        if (d < R) {
#pragma unroll
            for (int ww = 0; ww < kSortWarps; ++ww) {
                const uint32_t c = wcnt[ww * R + d];
                wcnt[ww * R + d] = run;
                run += c;
            }
        }
        tot[q] = run;
        tsum += run;
    }
    uint32_t x = tsum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    uint32_t dstart = x - tsum;
    for (int ww = 0; ww < w; ++ww) dstart += wsum[ww];
    uint32_t before[DPT];   // SWEEP: items of digit d in all earlier blocks
    if constexpr (SWEEP) {
        // publish this block's count of each digit (inclusive at once for the
        // first block), then walk back over earlier blocks until one that
        // has published its inclusive count; every wait is bounded in time
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            const int d = tid * DPT + q;
            if (d < R && (int)bid != stall_block)
                *(volatile uint32_t*)(status + (size_t)bid * R + d) = (bid == 0 ? kFlagInc : kFlagAgg) | tot[q];
        }
#pragma unroll
        for (int q = 0; q < DPT; ++q) {
            const int d = tid * DPT + q;
            uint32_t pre = 0u;
            if (d < R && bid > 0) {
                // kLookWindow earlier blocks' words are loaded together (one
                // round trip to L2 instead of one per block), then taken in
                // order; a word not yet published is re-read until it is
                bool found = false;
                for (long long j0 = (long long)bid - 1; j0 >= 0 && !found; j0 -= kLookWindow) {
                    uint32_t win[kLookWindow];
#pragma unroll
                    for (int u = 0; u < kLookWindow; ++u)
                        win[u] = j0 - u >= 0 ? *((const volatile uint32_t*)status + (size_t)(j0 - u) * R + d)
                                             : kFlagInc;
#pragma unroll
                    for (int u = 0; u < kLookWindow; ++u) {
                        if (found) break;
                        uint32_t v = win[u];
                        if (!(v & kFlagMask)) {
                            const volatile uint32_t* sp = status + (size_t)(j0 - u) * R + d;
                            const long long t0 = clock64();
                            while (!((v = *sp) & kFlagMask)) {
                                if (clock64() - t0 > kSweepWaitCycles) {
                                    atomicOr(err, kStatusTimeout);   // the output is invalid, never out of bounds
                                    v = kFlagInc;
                                    break;
                                }
                                __nanosleep(64);
                            }
                        }
                        pre += v & kValMask;
                        found = (v & kFlagInc) != 0u;
                    }
                }
                if ((int)bid != stall_block)
                    *(volatile uint32_t*)(status + (size_t)bid * R + d) = kFlagInc | ((pre + tot[q]) & kValMask);
            }
            before[q] = pre;
        }
    }
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        const int d = tid * DPT + q;
        if (d < R) {
#pragma unroll
            for (int ww = 0; ww < kSortWarps; ++ww) wcnt[ww * R + d] += dstart;
            // global position of block-local index i of digit d: gbase[d] + i (mod 2^32)
            if constexpr (SWEEP) gbase[d] = digit_base[d] + before[q] - dstart;
            else gbase[d] = offs[(size_t)d * nblocks + blockIdx.x] - dstart;
        }
        dstart += tot[q];
    }
    __syncthreads();

    // values are read only now, while the keys' ranks are known
#pragma unroll
    for (int r = 0; r < kScatterIPT; ++r) {
        const uint32_t dd = pk[r] & DMASK;
        if (dd < R) {
            const uint32_t p = wcnt[w * R + dd] + (pk[r] >> (RB + 1));
            skeys[p] = key[r];
            svals[p] = vin[wbase + r * 32 + lane];
        }
    }
    __syncthreads();
    const int cnt = (int)min((long long)kSortChunk, n - bbase);
    for (int i = tid; i < cnt; i += kSortThreads) {
        const K k = skeys[i];
        const uint32_t g = gbase[(uint32_t)(k >> shift) & (R - 1)] + (uint32_t)i;
        if (!SWEEP || (long long)g < n) {   // a timed-out look-back leaves g unknown: stay in bounds
            kout[g] = k;
            vout[g] = svals[i];
        }
    }
}

// Onesweep: the histograms of every digit place at once (one read of the
// keys), then their exclusive scans, one block per place.
template <typename K, int RB>
__global__ void __launch_bounds__(kSortThreads) k_sweep_hist(const K* __restrict__ keys,
                                                             const uint32_t* __restrict__ n_dev, long long bound,
                                                             int passes, uint32_t* __restrict__ ghist) {
    constexpr int R = 1 << RB;
    extern __shared__ uint32_t sh[];   // [passes][R]
    const int tid = threadIdx.x;
    for (int i = tid; i < passes * R; i += kSortThreads) sh[i] = 0u;
    __syncthreads();
    const long long n = n_dev ? list_len(n_dev, bound) : bound;
    for (long long q = (long long)blockIdx.x * kSortThreads + tid; q < n; q += (long long)gridDim.x * kSortThreads) {
        const K k = keys[q];
        for (int p = 0; p < passes; ++p) atomicAdd(&sh[p * R + ((uint32_t)(k >> (p * RB)) & (R - 1))], 1u);
    }
    __syncthreads();
    for (int i = tid; i < passes * R; i += kSortThreads)
        if (sh[i]) atomicAdd(&ghist[i], sh[i]);
}

template <int RB>
__global__ void __launch_bounds__(kSortThreads) k_sweep_base(const uint32_t* __restrict__ ghist,
                                                             uint32_t* __restrict__ gbase) {
    constexpr int R = 1 << RB;
    constexpr int DPT = R > kSortThreads ? R / kSortThreads : 1;
    __shared__ uint32_t wsum[kSortWarps];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t* h = ghist + (size_t)blockIdx.x * R;
    uint32_t c[DPT], t = 0u;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        const int d = tid * DPT + q;
        c[q] = d < R ? h[d] : 0u;
        t += c[q];
    }
    uint32_t x = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    uint32_t run = x - t;
    for (int ww = 0; ww < w; ++ww) run += wsum[ww];
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        const int d = tid * DPT + q;
        if (d < R) gbase[(size_t)blockIdx.x * R + d] = run;
        run += c[q];
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

// Skipped entirely when the emission overflowed or a sort wait expired: the
// list then holds stale entries whose tile ids need not be valid, and all
// ranges stay empty.
template <typename K, int SHIFT>
__global__ void __launch_bounds__(256) k_ranges(const K* __restrict__ keys,
                                                const uint32_t* __restrict__ n_dev, long long bound,
                                                const int* __restrict__ status,
                                                uint2* __restrict__ ranges) {
    if (*status & (kStatusCapacity | kStatusTimeout)) return;
    const long long n = list_len(n_dev, bound);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const uint32_t t = (uint32_t)(keys[i] >> SHIFT);
        if (i == 0 || (uint32_t)(keys[i - 1] >> SHIFT) != t) ranges[t].x = (uint32_t)i;
        if (i == n - 1 || (uint32_t)(keys[i + 1] >> SHIFT) != t) ranges[t].y = (uint32_t)(i + 1);
    }
}

// ------------------------------------------------- longest-list-first order
// The persistent blends take tiles from one queue; taking the tiles with
// the longest lists first keeps a long tile from starting last and running
// alone at the end.  Tiles are counting-sorted by floor(log2(list length))
// into kOrderBuckets buckets, longest bucket first, empty tiles last; the
// order within a bucket is whatever the block atomics give (each tile's
// result does not depend on when it is processed).
constexpr int kOrderBuckets = 34;   // 0: empty, 1 + floor(log2(len)) for len >= 1
constexpr int kOrderThreads = 256;

__device__ __forceinline__ int order_bucket(uint2 r) {
    const uint32_t len = r.y - r.x;
    return len == 0u ? 0 : 32 - __clz(len);   // 1 .. 33
}

__global__ void __launch_bounds__(kOrderThreads) k_order_count(const uint2* __restrict__ ranges, int T,
                                                               uint32_t* __restrict__ cnt) {
    __shared__ uint32_t h[kOrderBuckets];
    if (threadIdx.x < kOrderBuckets) h[threadIdx.x] = 0;
    __syncthreads();
    const int t = blockIdx.x * kOrderThreads + threadIdx.x;
    if (t < T) atomicAdd(&h[order_bucket(ranges[t])], 1u);
    __syncthreads();
    if (threadIdx.x < kOrderBuckets && h[threadIdx.x]) atomicAdd(&cnt[threadIdx.x], h[threadIdx.x]);
}

// One warp: cursor[b] = number of tiles in buckets longer than b (the empty
// bucket 0 goes last); the counts are cleared for the next call.
__global__ void __launch_bounds__(32) k_order_base(uint32_t* __restrict__ cnt, uint32_t* __restrict__ cursor) {
    const int lane = threadIdx.x;
    // lane l handles buckets 33 - l and, for l < 2, 1 - l (descending order)
    const int b0 = kOrderBuckets - 1 - lane;
    const uint32_t c0 = cnt[b0];
    const uint32_t c1 = lane < 2 ? cnt[1 - lane] : 0u;
    uint32_t x = c0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    const uint32_t total32 = __shfl_sync(0xffffffffu, x, 31);
    cursor[b0] = x - c0;
    const uint32_t c1a = __shfl_sync(0xffffffffu, c1, 0);   // bucket 1, then bucket 0
    if (lane == 0) cursor[1] = total32;
    if (lane == 1) cursor[0] = total32 + c1a;
    __syncwarp();
    cnt[b0] = 0u;
    if (lane < 2) cnt[1 - lane] = 0u;
}

__global__ void __launch_bounds__(kOrderThreads) k_order_scatter(const uint2* __restrict__ ranges, int T,
                                                                 uint32_t* __restrict__ cursor,
                                                                 uint32_t* __restrict__ order) {
    __shared__ uint32_t h[kOrderBuckets];
    __shared__ uint32_t base[kOrderBuckets];
    if (threadIdx.x < kOrderBuckets) h[threadIdx.x] = 0;
    __syncthreads();
    const int t = blockIdx.x * kOrderThreads + threadIdx.x;
    int b = 0;
    uint32_t rank = 0;
    if (t < T) {
        b = order_bucket(ranges[t]);
        rank = atomicAdd(&h[b], 1u);
    }
    __syncthreads();
    if (threadIdx.x < kOrderBuckets && h[threadIdx.x]) base[threadIdx.x] = atomicAdd(&cursor[threadIdx.x], h[threadIdx.x]);
    __syncthreads();
    if (t < T) order[base[b] + rank] = (uint32_t)t;
}

}  // namespace

cudaError_t launch_tile_order(const uint2* ranges, long long tiles, uint32_t* order, uint32_t* scratch,
                              cudaStream_t st) {
    if (tiles <= 0) return cudaSuccess;
    const int T = (int)tiles;
    const int nb = (T + kOrderThreads - 1) / kOrderThreads;
    k_order_count<<<nb, kOrderThreads, 0, st>>>(ranges, T, scratch);
    k_order_base<<<1, 32, 0, st>>>(scratch, scratch + kOrderBuckets);
    k_order_scatter<<<nb, kOrderThreads, 0, st>>>(ranges, T, scratch + kOrderBuckets, order);
    return cudaGetLastError();
}

int scan_blocks(long long n) { return (int)((n + kScanTile - 1) / kScanTile); }

cudaError_t launch_scan(const uint32_t* in, long long n, uint32_t* out, uint32_t* block_sums,
                        uint32_t* total, cudaStream_t st, int* status) {
    const int nb = scan_blocks(n);
    if (nb == 0) {
        if (total) return cudaMemsetAsync(total, 0, sizeof(uint32_t), st);
        return cudaSuccess;
    }
    k_scan_reduce<<<nb, kScanThreads, 0, st>>>(in, n, block_sums);
    k_scan_sums<<<1, kScanThreads, 0, st>>>(block_sums, nb, total, status);
    k_scan_down<<<nb, kScanThreads, 0, st>>>(in, n, block_sums, out);
    return cudaGetLastError();
}

int emit_blocks(long long n_records, long long bound) {
    return (int)((n_records + bound + kEmitItems - 1) / kEmitItems);
}

template <bool SORTED>
static cudaError_t emit_t(const uint32_t* order, const uint32_t* counts, const uint32_t* offsets,
                          const int4* trect, const uint32_t* zbits, long long n_records, const uint32_t* n_dev,
                          long long bound, uint32_t* part, uint32_t* keys32, uint64_t* keys64, uint32_t* vals,
                          long long cap, int* status, cudaStream_t st) {
    if (n_records == 0) return cudaSuccess;
    const int nb = emit_blocks(n_records, bound);
    k_emit_partition<<<(nb + 1 + 255) / 256, 256, 0, st>>>(offsets, n_records, n_dev, bound, nb, part);
    k_emit_lb<SORTED><<<nb, kEmitBlock, 0, st>>>(order, counts, offsets, trect, zbits, n_records, n_dev, bound,
                                                 part, keys32, keys64, vals, cap, status);
    return cudaGetLastError();
}

cudaError_t launch_emit(const uint32_t* counts, const uint32_t* offsets, const int4* trect,
                        const uint32_t* zbits, long long n_records, const uint32_t* n_dev, long long bound,
                        uint32_t* part, uint64_t* keys, uint32_t* vals, long long cap, int* status,
                        cudaStream_t st) {
    return emit_t<false>(nullptr, counts, offsets, trect, zbits, n_records, n_dev, bound, part, nullptr, keys,
                         vals, cap, status, st);
}

int sort_blocks(long long bound) { return (int)((bound + kSortChunk - 1) / kSortChunk); }

// The scatter's shared memory exceeds the 48 KB default for 64-bit keys and
// for wide digits: opt in once per device.
template <typename K, int RB, bool SWEEP>
static cudaError_t scatter_attr() {
    constexpr size_t bytes = scatter_smem_bytes<K, RB>();
    if (bytes <= 48 * 1024) return cudaSuccess;
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load() & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(k_radix_scatter<K, RB, SWEEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done.fetch_or(bit);
    return e;
}

// Workspace words of the onesweep form: the histograms and digit bases of up
// to kMaxPasses places, one block counter per place, one status word per
// (block, digit) reused by every pass.
constexpr int kMaxPasses = 16;
size_t sweep_ws_words(int nb, int R) { return (size_t)2 * kMaxPasses * R + kMaxPasses + (size_t)nb * R; }

template <typename K, int RB>
static cudaError_t radix_sort_t(K* k0, uint32_t* v0, K* k1, uint32_t* v1, const uint32_t* n_dev,
                                long long bound, int key_bits, uint32_t* hist, uint32_t* scan_tmp,
                                const SortCtl& ctl, int* passes_out, cudaStream_t st) {
    constexpr int R = 1 << RB;
    const int nb = sort_blocks(bound);
    int passes = 0;
    if (nb > 0) {
        K* kin = k0; uint32_t* vin = v0;
        K* kout = k1; uint32_t* vout = v1;
        if (ctl.onesweep && bound < kSweepMaxItems) {
            cudaError_t ea = scatter_attr<K, RB, true>();
            if (ea != cudaSuccess) return ea;
            const int np = (key_bits + RB - 1) / RB;
            uint32_t* ghist = hist;
            uint32_t* gbase = ghist + (size_t)kMaxPasses * R;
            uint32_t* counter = gbase + (size_t)kMaxPasses * R;
            uint32_t* status = counter + kMaxPasses;
            cudaError_t e = cudaMemsetAsync(ghist, 0, sizeof(uint32_t) * ((size_t)2 * kMaxPasses * R + kMaxPasses), st);
            if (e != cudaSuccess) return e;
            const int hb = nb < ctl.sms * 4 ? nb : ctl.sms * 4;
            k_sweep_hist<K, RB><<<hb, kSortThreads, sizeof(uint32_t) * np * R, st>>>(kin, n_dev, bound, np, ghist);
            k_sweep_base<RB><<<np, kSortThreads, 0, st>>>(ghist, gbase);
            for (int p = 0; p < np; ++p) {
                e = cudaMemsetAsync(status, 0, sizeof(uint32_t) * (size_t)nb * R, st);
                if (e != cudaSuccess) return e;
                k_radix_scatter<K, RB, true><<<nb, kSortThreads, scatter_smem_bytes<K, RB>(), st>>>(
                    kin, vin, kout, vout, n_dev, bound, p * RB, nb, nullptr, gbase + (size_t)p * R, status,
                    counter + p, ctl.status, p == 0 ? ctl.stall_block : -1);
                K* tk = kin; kin = kout; kout = tk;
                uint32_t* tv = vin; vin = vout; vout = tv;
                ++passes;
            }
        } else {
            cudaError_t ea = scatter_attr<K, RB, false>();
            if (ea != cudaSuccess) return ea;
            for (int shift = 0; shift < key_bits; shift += RB) {
                k_radix_hist<K, RB><<<nb, kSortThreads, 0, st>>>(kin, n_dev, bound, shift, nb, hist);
                cudaError_t e = launch_scan(hist, (long long)R * nb, hist, scan_tmp, nullptr, st);
                if (e != cudaSuccess) return e;
                k_radix_scatter<K, RB, false><<<nb, kSortThreads, scatter_smem_bytes<K, RB>(), st>>>(
                    kin, vin, kout, vout, n_dev, bound, shift, nb, hist, nullptr, nullptr, nullptr, nullptr, -1);
                K* tk = kin; kin = kout; kout = tk;
                uint32_t* tv = vin; vin = vout; vout = tv;
                ++passes;
            }
        }
    }
    *passes_out = passes;
    return cudaGetLastError();
}

// radix_bits is the widest digit allowed: the sort takes the fewest passes
// that digits of that width need for key_bits, and spreads the key bits
// evenly over them (18-bit keys at most 8 bits wide: three passes of 6 bits;
// at most 11: two passes of 9), never below 4 bits a digit.
int digit_bits(int key_bits, int radix_bits) {
    if (key_bits <= 0) return radix_bits;
    const int np = (key_bits + radix_bits - 1) / radix_bits;
    const int w = (key_bits + np - 1) / np;
    return w < 4 ? 4 : w;
}

template <typename K>
static cudaError_t radix_sort_rb(K* k0, uint32_t* v0, K* k1, uint32_t* v1, const uint32_t* n_dev,
                                 long long bound, int key_bits, int radix_bits, uint32_t* hist,
                                 uint32_t* scan_tmp, const SortCtl& ctl, int* passes_out, cudaStream_t st) {
    if (radix_bits < 4 || radix_bits > kRadixMaxBits) return cudaErrorInvalidValue;
#define LP_SORT_W(W) \
    case W: return radix_sort_t<K, W>(k0, v0, k1, v1, n_dev, bound, key_bits, hist, scan_tmp, ctl, passes_out, st);
    switch (digit_bits(key_bits, radix_bits)) {
        LP_SORT_W(4) LP_SORT_W(5) LP_SORT_W(6) LP_SORT_W(7) LP_SORT_W(8) LP_SORT_W(9) LP_SORT_W(10) LP_SORT_W(11)
        default: return cudaErrorInvalidValue;
    }
#undef LP_SORT_W
}

cudaError_t launch_radix_sort(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1,
                              const uint32_t* n_dev, long long bound, int key_bits, int radix_bits,
                              uint32_t* hist, uint32_t* scan_tmp, const SortCtl& ctl, int* passes_out,
                              cudaStream_t st) {
    return radix_sort_rb<uint64_t>(k0, v0, k1, v1, n_dev, bound, key_bits, radix_bits, hist, scan_tmp, ctl,
                                   passes_out, st);
}

cudaError_t launch_radix_sort32(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1,
                                const uint32_t* n_dev, long long bound, int key_bits, int radix_bits,
                                uint32_t* hist, uint32_t* scan_tmp, const SortCtl& ctl, int* passes_out,
                                cudaStream_t st) {
    return radix_sort_rb<uint32_t>(k0, v0, k1, v1, n_dev, bound, key_bits, radix_bits, hist, scan_tmp, ctl,
                                   passes_out, st);
}

// Workspace words of a sort of up to `bound` items at any digit width: the
// onesweep form's histograms, bases, counters and status words, or the
// per-pass (digit, block) histogram of the form used past 2^30 items.
size_t sort_hist_elems(long long bound) {
    return sweep_ws_words(sort_blocks(bound), 1 << kRadixMaxBits);
}

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
                               const int4* trect, long long n_records, const uint32_t* n_dev, long long bound,
                               uint32_t* part, uint32_t* keys, uint32_t* vals, long long cap, int* status,
                               cudaStream_t st) {
    return emit_t<true>(order, counts_sorted, offsets, trect, nullptr, n_records, n_dev, bound, part, keys,
                        nullptr, vals, cap, status, st);
}

// ------------------------------------------------ per-tile depth sort (mode 2)
// Sort mode 2 emits every record's entries in record order and stably sorts
// them by tile id, so that each tile's run of the list is in record order;
// sorting each run stably by its records' depth bits then gives (tile, depth,
// record) order, the order of modes 0 and 1.  A warp sorts a run of up to
// kTileWarpCap entries in shared memory (LSD radix, 8-bit digits, the digits
// that do not vary across the run skipped; four warps per block, 9 KB each);
// longer runs are listed and k_tile_sort_long gives each one block, which
// sorts it in shared memory up to kTileBlockCap entries and through global
// scratch in chunks beyond, whatever its length.
constexpr int kTileSortThreads = 128;
constexpr int kTileWarpCap = 512;
constexpr int kTileLongThreads = 256;
constexpr int kTileBlockCap = 2048;
constexpr size_t kTileLongSmem = (size_t)4 * kTileBlockCap * sizeof(uint32_t);

// Stable LSD sort of n <= kTileWarpCap (key, value) pairs in a warp's shared
// memory (ka, va; kb, vb a second buffer; cnt 256 counters).  Returns the
// buffer pair that holds the result (0: ka/va, 1: kb/vb).
__device__ int warp_radix_sort(uint32_t* ka, uint32_t* va, uint32_t* kb, uint32_t* vb, uint32_t* cnt, int n,
                               int lane) {
    uint32_t o = 0u, a = 0xffffffffu;
    for (int i = lane; i < n; i += 32) { o |= ka[i]; a &= ka[i]; }
    const uint32_t diff = __reduce_or_sync(0xffffffffu, o) & ~__reduce_and_sync(0xffffffffu, a);
    int in = 0;
    const unsigned lt = (1u << lane) - 1u;
    for (int shift = 0; shift < 32; shift += 8) {
        if (((diff >> shift) & 255u) == 0u) continue;   // one digit value across the run: already in order
        uint32_t* ks = in ? kb : ka; uint32_t* vs = in ? vb : va;
        uint32_t* kd = in ? ka : kb; uint32_t* vd = in ? va : vb;
#pragma unroll
        for (int q = 0; q < 8; ++q) cnt[lane * 8 + q] = 0u;
        __syncwarp();
        for (int i = lane; i < n; i += 32) atomicAdd(&cnt[(ks[i] >> shift) & 255u], 1u);
        __syncwarp();
        // exclusive scan of the 256 counts: lane l holds digits 8l .. 8l + 7
        uint32_t c[8], tot = 0u;
#pragma unroll
        for (int q = 0; q < 8; ++q) { c[q] = cnt[lane * 8 + q]; tot += c[q]; }
        uint32_t x = tot;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        x -= tot;
#pragma unroll
        for (int q = 0; q < 8; ++q) { cnt[lane * 8 + q] = x; x += c[q]; }
        __syncwarp();
        // rounds of 32 entries in order; equal digits keep their order
        for (int base = 0; base < n; base += 32) {
            const int i = base + lane;
            const bool ok = i < n;
            const uint32_t key = ok ? ks[i] : 0u, val = ok ? vs[i] : 0u;
            const uint32_t d = ok ? (key >> shift) & 255u : 256u;
            const unsigned peers = digit_peers<8>(d);
            const uint32_t rank = __popc(peers & lt);
            const uint32_t off = ok ? cnt[d] : 0u;
            __syncwarp();
            if (ok && rank == 0) cnt[d] = off + __popc(peers);
            __syncwarp();
            if (ok) { kd[off + rank] = key; vd[off + rank] = val; }
        }
        __syncwarp();
        in ^= 1;
    }
    return in;
}

// One warp per tile (tiles from a queue).  Runs longer than kTileWarpCap go
// to long_list.  Skipped when the list overflowed or a sort wait expired (the
// ranges are then all empty).
__global__ void __launch_bounds__(kTileSortThreads) k_tile_sort(uint32_t* __restrict__ vals,
                                                                const uint2* __restrict__ ranges, int T,
                                                                const uint32_t* __restrict__ zbits,
                                                                int* __restrict__ counters,
                                                                uint32_t* __restrict__ long_list,
                                                                const int* __restrict__ status) {
    constexpr int NW = kTileSortThreads / 32;
    __shared__ uint32_t s_buf[NW][4][kTileWarpCap];
    __shared__ uint32_t s_cnt[NW][256];
    if (*status & (kStatusCapacity | kStatusTimeout)) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (;;) {
        int t = 0;
        if (lane == 0) t = atomicAdd(counters, 1);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= T) break;
        const uint2 rg = ranges[t];
        const int n = (int)(rg.y - rg.x);
        if (n <= 1) continue;
        if (n > kTileWarpCap) {
            if (lane == 0) long_list[atomicAdd(counters + 1, 1)] = (uint32_t)t;
            continue;
        }
        uint32_t* ka = s_buf[w][0]; uint32_t* va = s_buf[w][1];
        for (int i = lane; i < n; i += 32) {
            const uint32_t v = vals[rg.x + i];
            va[i] = v;
            ka[i] = zbits[v];
        }
        __syncwarp();
        const int in = warp_radix_sort(ka, va, s_buf[w][2], s_buf[w][3], s_cnt[w], n, lane);
        const uint32_t* vr = in ? s_buf[w][3] : va;
        for (int i = lane; i < n; i += 32) vals[rg.x + i] = vr[i];
        __syncwarp();
    }
}

// One LSD pass of a block over n entries (values v, keys key(v) by the
// functor): digit counts, their scan, then chunks of kTileLongThreads entries
// in order, each ranked by warp, then across the block's warps, so that equal
// digits keep their order.  src and dst are global arrays; key() gathers
// each entry's key again on every pass.
template <typename KeyF>
__device__ void block_lsd_pass(const uint32_t* src, uint32_t* dst, long long n, int shift, KeyF key,
                               uint32_t* s_base, uint32_t (*s_wcnt)[256]) {
    constexpr int NW = kTileLongThreads / 32;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    s_base[tid] = 0u;
    __syncthreads();
    for (long long i = tid; i < n; i += kTileLongThreads)
        atomicAdd(&s_base[(key(src[i]) >> shift) & 255u], 1u);
    __syncthreads();
    if (w == 0) {   // exclusive scan of the 256 counts, 8 per lane
        uint32_t c[8], tot = 0u;
#pragma unroll
        for (int q = 0; q < 8; ++q) { c[q] = s_base[lane * 8 + q]; tot += c[q]; }
        uint32_t x = tot;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        x -= tot;
#pragma unroll
        for (int q = 0; q < 8; ++q) { s_base[lane * 8 + q] = x; x += c[q]; }
    }
    __syncthreads();
    for (long long c0 = 0; c0 < n; c0 += kTileLongThreads) {
        const long long i = c0 + tid;
        const bool ok = i < n;
        const uint32_t v = ok ? src[i] : 0u;
        const uint32_t k = ok ? key(v) : 0u;
        const uint32_t d = ok ? (k >> shift) & 255u : 256u;
        const unsigned peers = digit_peers<8>(d);
        const uint32_t rank = __popc(peers & lt);
#pragma unroll
        for (int ww = 0; ww < NW; ++ww) s_wcnt[ww][tid] = 0u;   // thread t: digit t of every warp
        __syncthreads();
        if (ok && rank == 0) s_wcnt[w][d] = __popc(peers);
        __syncthreads();
        if (ok) {
            uint32_t pos = s_base[d] + rank;
            for (int ww = 0; ww < w; ++ww) pos += s_wcnt[ww][d];
            dst[pos] = v;
        }
        __syncthreads();
        uint32_t add = 0u;
#pragma unroll
        for (int ww = 0; ww < NW; ++ww) add += s_wcnt[ww][tid];
        s_base[tid] += add;
        __syncthreads();
    }
}

// One LSD pass of a block over a run of n <= kTileBlockCap entries in shared
// memory (keys ks, values vs -> kd, vd), as one chunk: warp w ranks the w-th
// contiguous eighth of the run round by round (equal digits found by ballots,
// a running count per (warp, digit) in s_wcnt), the per-digit starts come
// from one block scan, and each entry goes to its digit's start plus the
// counts of earlier warps plus its rank within the warp.  Equal digits keep
// their order.  Four block barriers per pass.
__device__ void block_lsd_pass_smem(const uint32_t* ks, const uint32_t* vs, uint32_t* kd, uint32_t* vd, int n,
                                    int shift, uint32_t* s_base, uint32_t (*s_wcnt)[256], uint32_t* s_wsum) {
    constexpr int NW = kTileLongThreads / 32;
    constexpr int RMAX = kTileBlockCap / kTileLongThreads;   // rounds per warp at most
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int per_warp = ((n + NW - 1) / NW + 31) & ~31;     // whole rounds
    const int rounds = per_warp / 32;
#pragma unroll
    for (int ww = 0; ww < NW; ++ww) s_wcnt[ww][tid] = 0u;
    __syncthreads();
    uint32_t pk[RMAX];   // digit | rank within (warp, digit) << 9
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
        pk[r] = 256u;
        if (r < rounds) {
            const int i = w * per_warp + r * 32 + lane;
            const uint32_t d = i < n ? (ks[i] >> shift) & 255u : 256u;
            const unsigned peers = digit_peers<8>(d);
            const uint32_t rank = __popc(peers & lt);
            const uint32_t base = d < 256u ? s_wcnt[w][d] : 0u;
            __syncwarp();
            if (d < 256u && rank == 0) s_wcnt[w][d] = base + __popc(peers);
            __syncwarp();
            pk[r] = d | ((base + rank) << 9);
        }
    }
    __syncthreads();
    // thread t, digit t: starts of the warps within the digit, then the
    // digit's start over the run (exclusive scan of the digit totals)
    uint32_t run = 0u;
#pragma unroll
    for (int ww = 0; ww < NW; ++ww) {
        const uint32_t c = s_wcnt[ww][tid];
        s_wcnt[ww][tid] = run;
        run += c;
    }
    uint32_t x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_wsum[w] = x;
    __syncthreads();
    uint32_t start = x - run;
    for (int ww = 0; ww < w; ++ww) start += s_wsum[ww];
    s_base[tid] = start;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RMAX; ++r) {
        const uint32_t d = pk[r] & 511u;
        if (r < rounds && d < 256u) {
            const int i = w * per_warp + r * 32 + lane;
            const uint32_t pos = s_base[d] + s_wcnt[w][d] + (pk[r] >> 9);
            kd[pos] = ks[i];
            vd[pos] = vs[i];
        }
    }
    __syncthreads();
}

// One block per listed long run, sorted stably by depth bits: runs of up to
// kTileBlockCap entries in shared memory (dynamic, keys moving with the
// values; block_lsd_pass_smem, one chunk per pass), longer ones through the
// global scratch arrays sa and sb (the run's own positions [rg.x, rg.y) of
// each; block_lsd_pass in chunks, the depth bits gathered again in each pass).

__global__ void __launch_bounds__(kTileLongThreads) k_tile_sort_long(uint32_t* __restrict__ vals,
                                                                     const uint2* __restrict__ ranges,
                                                                     const uint32_t* __restrict__ zbits,
                                                                     const int* __restrict__ counters,
                                                                     const uint32_t* __restrict__ long_list,
                                                                     uint32_t* __restrict__ sa,
                                                                     uint32_t* __restrict__ sb,
                                                                     const int* __restrict__ status) {
    constexpr int NW = kTileLongThreads / 32;
    extern __shared__ __align__(16) uint32_t s_run[];   // values, keys; second values, keys
    __shared__ uint32_t s_base[256];
    __shared__ uint32_t s_wcnt[NW][256];
    __shared__ uint32_t s_wsum[NW];
    __shared__ uint32_t s_or, s_and;
    if (*status & (kStatusCapacity | kStatusTimeout)) return;
    const int tid = threadIdx.x, lane = tid & 31;
    const int nlong = counters[1];
    auto key = [zbits](uint32_t v) { return zbits[v]; };
    for (int li = blockIdx.x; li < nlong; li += gridDim.x) {
        const uint2 rg = ranges[long_list[li]];
        const long long n = (long long)(rg.y - rg.x);
        const bool in_smem = n <= kTileBlockCap;   // uniform over the block
        uint32_t* v0 = in_smem ? s_run : sa + rg.x;
        uint32_t* v1 = in_smem ? s_run + 2 * kTileBlockCap : sb + rg.x;
        uint32_t* k0 = s_run + kTileBlockCap;
        uint32_t* k1 = s_run + 3 * kTileBlockCap;
        if (tid == 0) { s_or = 0u; s_and = 0xffffffffu; }
        __syncthreads();
        uint32_t o = 0u, a = 0xffffffffu;
        for (long long i = tid; i < n; i += kTileLongThreads) {
            const uint32_t v = vals[rg.x + i];
            const uint32_t z = zbits[v];
            v0[i] = v;
            if (in_smem) k0[i] = z;
            o |= z; a &= z;
        }
        o = __reduce_or_sync(0xffffffffu, o);
        a = __reduce_and_sync(0xffffffffu, a);
        if (lane == 0) { atomicOr(&s_or, o); atomicAnd(&s_and, a); }
        __syncthreads();
        const uint32_t diff = s_or & ~s_and;
        for (int shift = 0; shift < 32; shift += 8) {
            if (((diff >> shift) & 255u) == 0u) continue;   // uniform over the block
            if (in_smem) block_lsd_pass_smem(k0, v0, k1, v1, (int)n, shift, s_base, s_wcnt, s_wsum);
            else block_lsd_pass(v0, v1, n, shift, key, s_base, s_wcnt);
            uint32_t* t = v0; v0 = v1; v1 = t;
            t = k0; k0 = k1; k1 = t;
        }
        for (long long i = tid; i < n; i += kTileLongThreads) vals[rg.x + i] = v0[i];
        __syncthreads();
    }
}

cudaError_t launch_tile_sort(uint32_t* vals, const uint2* ranges, long long tiles, const uint32_t* zbits,
                             int* counters, uint32_t* long_list, uint32_t* scratch_a, uint32_t* scratch_b,
                             const int* status, int sms, cudaStream_t st) {
    if (tiles <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(counters, 0, 2 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    const long long want = (tiles + 3) / 4;
    const int grid = (int)(want < (long long)sms * 8 ? want : (long long)sms * 8);
    k_tile_sort<<<grid, kTileSortThreads, 0, st>>>(vals, ranges, (int)tiles, zbits, counters, long_list, status);
    // 32 KB of dynamic shared memory: within the default limit, no attribute to set
    static_assert(kTileLongSmem + 10 * 1024 <= 48 * 1024, "dynamic + static shared memory of k_tile_sort_long");
    k_tile_sort_long<<<sms * 5, kTileLongThreads, kTileLongSmem, st>>>(vals, ranges, zbits, counters, long_list,
                                                                       scratch_a, scratch_b, status);
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
