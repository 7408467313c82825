// Host-side launchers shared between the kernel translation units and the
// C ABI implementation.  Not part of the public interface.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lp {

struct CamsParam;
struct PrimsDev;

cudaError_t launch_preprocess(int V, int deg, const PrimsDev& P, const CamsParam& cams, float* rec,
                              uint32_t* counts, int4* trect, uint32_t* zbits, cudaStream_t st);

cudaError_t launch_chain(int V, int deg, const PrimsDev& P, const CamsParam& cams, const float* rec,
                         const uint32_t* counts, const float* acc, float* dc, float* dv, float* dop,
                         float* dsh, int accumulate, int split, cudaStream_t st);

int scan_blocks(long long n);
cudaError_t launch_scan(const uint32_t* in, long long n, uint32_t* out, uint32_t* block_sums,
                        uint32_t* total, cudaStream_t st);

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
cudaError_t launch_radix_sort(uint64_t* k0, uint32_t* v0, uint64_t* k1, uint32_t* v1,
                              const uint32_t* n_dev, long long bound, int key_bits, uint32_t* hist,
                              uint32_t* scan_tmp, int* passes_out, cudaStream_t st);

cudaError_t launch_ranges(const uint64_t* keys, const uint32_t* n_dev, long long bound,
                          const int* status, uint2* ranges, int sms, cudaStream_t st);

// two-stage sort: records by depth, then entries by 32-bit tile id
cudaError_t launch_radix_sort32(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1,
                                const uint32_t* n_dev, long long bound, int key_bits,
                                uint32_t* hist, uint32_t* scan_tmp, int* passes_out, cudaStream_t st);
cudaError_t launch_depth_keys(const uint32_t* counts, const uint32_t* zbits, long long n, uint32_t* keys,
                              uint32_t* vals, cudaStream_t st);
cudaError_t launch_gather_counts(const uint32_t* counts, const uint32_t* order, long long n, uint32_t* out,
                                 cudaStream_t st);
cudaError_t launch_emit_sorted(const uint32_t* order, const uint32_t* counts_sorted, const uint32_t* offsets,
                               const int4* trect, long long n_records, const uint32_t* n_dev, long long bound,
                               uint32_t* part, uint32_t* keys, uint32_t* vals, long long cap, int* status,
                               cudaStream_t st);
cudaError_t launch_ranges32(const uint32_t* keys, const uint32_t* n_dev, long long bound,
                            const int* status, uint2* ranges, int sms, cudaStream_t st);

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
    float* acc;
    int* tile_counter;
    unsigned long long* pair_counts;
    bool count;
    float* depth;          // depth pass output (forward kernel in depth mode when non-null)
    uint32_t contrib_stride = 0;   // words per warp of the contributor mask
    int sparse_lanes = 8;          // backward: per-lane atomics up to this many contributing lanes
    uint32_t* contrib;     // per warp w of a tile (its bits at contrib + w * contrib_stride), one
                           // bit per tile-list entry: some pixel of that warp blended the entry
                           // (written by the forward when non-null, read by the backward)
};

cudaError_t launch_blend_fwd(int V, int batch, int pix, const BlendArgs& a, cudaStream_t st);
cudaError_t launch_blend_bwd(int V, int batch, int pix, const BlendArgs& a, cudaStream_t st);
int blend_fwd_occupancy(int V, int batch, int pix);   // resident blocks per SM
int blend_bwd_occupancy(int V, int batch, int pix);

// exact spans (no ray-space approximation): own records, accumulators and kernels
int rec_floats_x(int V);
int acc_floats_x(int V);
cudaError_t launch_preprocess_x(int V, int deg, const PrimsDev& P, const CamsParam& cams, float* rec,
                                uint32_t* counts, int4* trect, uint32_t* zbits, cudaStream_t st);
cudaError_t launch_chain_x(int V, int deg, const PrimsDev& P, const CamsParam& cams, const float* rec,
                           const uint32_t* counts, const float* acc, float* dc, float* dv, float* dop, float* dsh,
                           int accumulate, cudaStream_t st);
cudaError_t launch_blend_fwd_x(int V, const BlendArgs& a, cudaStream_t st);
cudaError_t launch_blend_bwd_x(int V, const BlendArgs& a, cudaStream_t st);
int blend_x_occupancy(int V, bool fwd);

}  // namespace lp
