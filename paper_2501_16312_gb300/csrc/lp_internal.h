// Host-side launchers shared between the kernel translation units and the
// C ABI implementation.  Not part of the public interface.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lp {

// (tile edge, pixels per thread) pairs the ray-space blends are built for: at
// least one full warp per tile, at most 512 threads per block.
constexpr bool tile_pix_ok(int tile, int pix) {
    return (tile == 8 && (pix == 1 || pix == 2)) || (tile == 16 && (pix == 1 || pix == 2 || pix == 4)) ||
           (tile == 32 && (pix == 2 || pix == 4));
}

struct CamsParam;
struct PrimsDev;

// meta: one word per record, the record's face order (as in its word 3),
// read by the chain; may be null when no chain follows.
cudaError_t launch_preprocess(int V, int deg, const PrimsDev& P, const CamsParam& cams, float* rec,
                              uint32_t* counts, int4* trect, uint32_t* zbits, uint32_t* meta, cudaStream_t st);

// acc: the backward's accumulators, planes [R][3F] then colour [R][4].
cudaError_t launch_chain(int V, int deg, const PrimsDev& P, const CamsParam& cams, const uint32_t* meta,
                         const uint32_t* counts, const float* acc, float* dc, float* dv, float* dop,
                         float* dsh, int accumulate, int split, cudaStream_t st);

int scan_blocks(long long n);
// Exclusive scan of n 32-bit counts.  total (optional): their sum, or
// kListOverflow when it reaches 2^32 - 1, in which case kStatusCapacity is
// latched in status (optional).
cudaError_t launch_scan(const uint32_t* in, long long n, uint32_t* out, uint32_t* block_sums,
                        uint32_t* total, cudaStream_t st, int* status = nullptr);

// Key emission.  n_dev: the list length E on the device (written by the
// scan), bound: an upper bound of E for grid sizing, part: emit_blocks + 1
// words of scratch, cap: capacity of keys/vals.
int emit_blocks(long long n_records, long long bound);
cudaError_t launch_emit(const uint32_t* counts, const uint32_t* offsets, const int4* trect,
                        const uint32_t* zbits, long long n_records, const uint32_t* n_dev, long long bound,
                        uint32_t* part, uint64_t* keys, uint32_t* vals, long long cap, int* status,
                        cudaStream_t st);

int sort_blocks(long long bound);
size_t sort_hist_elems(long long bound);
// Radix sort control: SMs (grid of the histogram pass), the status word a
// timed-out look-back latches kStatusTimeout in, and a block of the first
// pass that publishes nothing (-1: none; a test of the bounded wait).
struct SortCtl {
    int sms;
    int* status;
    int stall_block;
    bool onesweep;   // below 2^30 items: the onesweep form (else the per-pass form)
};

// radix_bits: digit width, 4, 6, 8 or 11 (cudaErrorInvalidValue otherwise);
// hist holds sort_hist_elems(bound) words, enough for any width.  The sort
// runs either a histogram, a scan and a scatter per digit place, or (when
// ctl.onesweep and below 2^30 items) the onesweep form: one histogram pass
// for all digit places, then one kernel per place with a decoupled look-back
// whose waits are bounded.
cudaError_t launch_radix_sort(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1,
                              const uint32_t* n_dev, long long bound, int key_bits, int radix_bits,
                              uint32_t* hist, uint32_t* scan_tmp, const SortCtl& ctl, int* passes_out,
                              cudaStream_t st);

cudaError_t launch_ranges(const uint64_t* keys, const uint32_t* n_dev, long long bound,
                          const int* status, uint2* ranges, int sms, cudaStream_t st);

// two-stage sort: records by depth, then entries by 32-bit tile id
cudaError_t launch_radix_sort32(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1,
                                const uint32_t* n_dev, long long bound, int key_bits, int radix_bits,
                                uint32_t* hist, uint32_t* scan_tmp, const SortCtl& ctl, int* passes_out,
                                cudaStream_t st);
cudaError_t launch_depth_keys(const uint32_t* counts, const uint32_t* zbits, long long n, uint32_t* keys,
                              uint32_t* vals, cudaStream_t st);
cudaError_t launch_gather_counts(const uint32_t* counts, const uint32_t* order, long long n, uint32_t* out,
                                 cudaStream_t st);
cudaError_t launch_emit_sorted(const uint32_t* order, const uint32_t* counts_sorted, const uint32_t* offsets,
                               const int4* trect, long long n_records, const uint32_t* n_dev, long long bound,
                               uint32_t* part, uint32_t* keys, uint32_t* vals, long long cap, int* status,
                               cudaStream_t st);
// Sort mode 2, after the tile sort and the ranges: each tile's run of vals
// (record indices, in record order) sorted stably by the records' depth bits.
// counters: 2 device ints (zeroed here); long_list: room for one id per tile;
// scratch_a, scratch_b: 4-byte scratch of the list's length each.
cudaError_t launch_tile_sort(uint32_t* vals, const uint2* ranges, long long tiles, const uint32_t* zbits,
                             int* counters, uint32_t* long_list, uint32_t* scratch_a, uint32_t* scratch_b,
                             const int* status, int sms, cudaStream_t st);
cudaError_t launch_ranges32(const uint32_t* keys, const uint32_t* n_dev, long long bound,
                            const int* status, uint2* ranges, int sms, cudaStream_t st);

// Longest-list-first tile order (order: tiles words; scratch: 68 words,
// zero before the first call, left zero by each call).
cudaError_t launch_tile_order(const uint2* ranges, long long tiles, uint32_t* order, uint32_t* scratch,
                              cudaStream_t st);

struct BlendArgs {
    int grid;
    const float* rec;
    const uint32_t* vals;
    const uint2* ranges;
    const CamsParam* cams;
    float bg[3];
    float* image;          // forward output
    const float* dimage;   // backward input
    uint32_t* last;
    float* tl;
    float* acc;            // plane accumulators [R][3F]
    float* acc_col;        // colour and density accumulators [R][4]
    int* tile_counter;
    unsigned long long* pair_counts;
    bool count;
    float* depth;          // depth pass output (forward kernel in depth mode when non-null)
    const uint32_t* order = nullptr;   // queue position -> tile (null: tiles in index order)
    uint32_t contrib_stride = 0;   // words per lane-group row of the contributor mask
    uint32_t* contrib;     // per lane group g of warp w of a tile, one bit per tile-list entry:
                           // some pixel of that group blended the entry (written by the
                           // forward when non-null, read by the backward).  Word x of group g
                           // is at contrib + w * G * contrib_stride + x * G + g,
                           // with G = lane_groups (groups interleaved word by word); the
                           // exact-span blends keep one row per warp, at w * contrib_stride
};

// Blends for one tile edge each (lp_blend_{fwd,bwd}_t{8,16,32}.cu).
cudaError_t launch_blend_fwd_t8(int V, int batch, int pix, const BlendArgs& a, cudaStream_t st);
cudaError_t launch_blend_fwd_t16(int V, int batch, int pix, const BlendArgs& a, cudaStream_t st);
cudaError_t launch_blend_fwd_t32(int V, int batch, int pix, const BlendArgs& a, cudaStream_t st);
cudaError_t launch_blend_bwd_t8(int V, int batch, int pix, const BlendArgs& a, cudaStream_t st);
cudaError_t launch_blend_bwd_t16(int V, int batch, int pix, const BlendArgs& a, cudaStream_t st);
cudaError_t launch_blend_bwd_t32(int V, int batch, int pix, const BlendArgs& a, cudaStream_t st);
int blend_fwd_occupancy_t8(int V, int batch, int pix);   // resident blocks per SM
int blend_fwd_occupancy_t16(int V, int batch, int pix);
int blend_fwd_occupancy_t32(int V, int batch, int pix);
int blend_bwd_occupancy_t8(int V, int batch, int pix);
int blend_bwd_occupancy_t16(int V, int batch, int pix);
int blend_bwd_occupancy_t32(int V, int batch, int pix);

inline cudaError_t launch_blend_fwd(int tile, int V, int batch, int pix, const BlendArgs& a, cudaStream_t st) {
    return tile == 8 ? launch_blend_fwd_t8(V, batch, pix, a, st)
         : tile == 32 ? launch_blend_fwd_t32(V, batch, pix, a, st) : launch_blend_fwd_t16(V, batch, pix, a, st);
}
inline cudaError_t launch_blend_bwd(int tile, int V, int batch, int pix, const BlendArgs& a, cudaStream_t st) {
    return tile == 8 ? launch_blend_bwd_t8(V, batch, pix, a, st)
         : tile == 32 ? launch_blend_bwd_t32(V, batch, pix, a, st) : launch_blend_bwd_t16(V, batch, pix, a, st);
}
inline int blend_fwd_occupancy(int tile, int V, int batch, int pix) {
    return tile == 8 ? blend_fwd_occupancy_t8(V, batch, pix)
         : tile == 32 ? blend_fwd_occupancy_t32(V, batch, pix) : blend_fwd_occupancy_t16(V, batch, pix);
}
inline int blend_bwd_occupancy(int tile, int V, int batch, int pix) {
    return tile == 8 ? blend_bwd_occupancy_t8(V, batch, pix)
         : tile == 32 ? blend_bwd_occupancy_t32(V, batch, pix) : blend_bwd_occupancy_t16(V, batch, pix);
}
// warps per tile of the ray-space blends
inline int blend_warps(int tile, int pix) { return tile * tile / pix / 32; }
// Lane groups per warp of the ray-space blends: the forward writes one
// contributor-mask row per group (quadrants of the warp's pixel rectangle),
// and each group of the backward walks its own row.
constexpr int kLaneGroupsMax = 4;
constexpr int lane_groups(int tile, int pix) { return 4; }
inline int blend_mask_rows(int tile, int pix) { return blend_warps(tile, pix) * lane_groups(tile, pix); }

// exact spans (no ray-space approximation): own records, accumulators and kernels
int rec_floats_x(int V);
int acc_floats_x(int V);
cudaError_t launch_preprocess_x(int V, int deg, const PrimsDev& P, const CamsParam& cams, float* rec,
                                uint32_t* counts, int4* trect, uint32_t* zbits, cudaStream_t st);
cudaError_t launch_chain_x(int V, int deg, const PrimsDev& P, const CamsParam& cams, const float* rec,
                           const uint32_t* counts, const float* acc, float* dc, float* dv, float* dop, float* dsh,
                           int accumulate, cudaStream_t st);
cudaError_t launch_blend_fwd_x(int tile, int V, const BlendArgs& a, cudaStream_t st);
cudaError_t launch_blend_bwd_x(int tile, int V, const BlendArgs& a, cudaStream_t st);
int blend_x_occupancy(int tile, int V, bool fwd);
// pixels per thread and warps per tile of the exact-span blends
inline int blend_x_pix(int tile) { return tile == 8 ? 2 : 4; }
inline int blend_x_warps(int tile) { return tile * tile / blend_x_pix(tile) / 32; }

}  // namespace lp
