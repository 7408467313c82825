// C ABI of the LinPrim rasterizer: context, workspace and launch sequence.
//
// lp_render_forward enqueues, on the caller's stream:
//   A1 preprocess (all cameras x primitives) -> A2 scan of tile counts and key
//   emission -> A3 stable radix sort of (tile << 32 | depth) keys -> A4 tile
//   ranges -> A5 persistent front-to-back blend over the tiles of all cameras.
// lp_render_backward enqueues A6 (back-to-front blend backward) and A7 (chain
// to world-space centre/vertices, opacity and SH, summed over cameras).
#include <cuda_runtime.h>

#include <algorithm>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "linprim.h"
#include "lp_device.cuh"
#include "lp_internal.h"

namespace {

// Grow-only device allocation.  With the context's guard mode on, each
// allocation carries a canary zone of kGuardBytes past its capacity, filled
// with kGuardByte; lp_check_guards reports any byte there that changed.
template <typename T> struct DevBuf {
    T* p = nullptr;
    size_t cap = 0;     // elements
    size_t guard = 0;   // bytes of canary zone after cap elements (0: none)
};

constexpr size_t kGuardBytes = 4096;
constexpr unsigned char kGuardByte = 0xA5;

}  // namespace

struct lp_ctx {
    int device = 0;
    int sms = 0;
    lp_tuning tune{16, 64, 0, 0, 4, 0, 8, 0, 0};
    float aa_kernel = 0.f;      // 2D filter size in pixels (0 = off)
    bool exact = false;         // spans along the true perspective ray
    bool fwd_exact = false;     // mode of the last forward
    uint32_t contrib_stride = 0;
    lp_tuning fwd_tune{16, 64, 0, 0, 4, 0, 8, 0, 0};   // schedule of the last forward (its tiles, mask layout)
    // densification statistics gathered by forward and backward (null: off)
    float* st_grad_sum = nullptr;
    uint32_t* st_grad_count = nullptr;
    uint32_t* st_px_max = nullptr;
    long long st_n = 0;
    char err[512] = {0};

    DevBuf<float> rec;
    DevBuf<uint32_t> counts, offsets, zbits, scan_tmp, hist, last, emit_part, contrib;
    DevBuf<int4> trect;
    DevBuf<uint64_t> keys0, keys1;
    DevBuf<uint32_t> vals0, vals1;
    DevBuf<uint2> ranges;
    DevBuf<float> tl, acc, scratch_image;
    DevBuf<uint32_t> dkeys0, dkeys1, dvals0, dvals1, counts_sorted;   // two-stage sort
    DevBuf<uint32_t> tsort;   // per-tile sort: long-run list (one id per tile) and two counters
    DevBuf<uint32_t> tile_order;     // longest-list-first queue order of the tiles
    DevBuf<uint32_t> meta;           // per-record face order (ray-space records), read by the chain
    uint32_t* d_order_scratch = nullptr;   // bucket counts and cursors of the order
    int* d_status = nullptr;         // latched status bits
    uint32_t* d_E = nullptr;         // tile-list length of the last forward
    int* d_tile_counter = nullptr;   // [0] forward queue, [1] backward queue
    unsigned long long* d_pairs = nullptr;
    uint32_t* h_E = nullptr;         // pinned

    // state of the last forward
    bool have_fwd = false;
    lp_prims prims{};
    lp::CamsParam cams{};
    float bg[3] = {0.f, 0.f, 0.f};
    long long records = 0, pixels = 0, tiles = 0, E_bound = 0, E_host = -1;
    int key_bits = 0, sort_passes = 0;
    int launches_fwd = 0;
    bool result_in_1 = false;
    bool keys32 = false;        // tile list keyed by 32-bit tile ids (two-stage sort)

    // stage timing: events 0..5 bracket the forward stages, 6..8 the backward
    bool timing = false;
    cudaEvent_t ev[9] = {};
    bool fwd_timed = false, bwd_timed = false;

    bool guard = false;   // canary zones on later allocations (lp_set_debug_guard)
    int stall_block = -1; // a sort block that publishes nothing (lp_debug_sort_stall)

    // every grow-only buffer, with a name (guard checks, release)
    template <typename F> void each_buf(F&& f) {
        f(rec, "records"); f(counts, "counts"); f(offsets, "offsets"); f(zbits, "zbits");
        f(scan_tmp, "scan blocks"); f(hist, "histograms"); f(last, "pixel state"); f(emit_part, "emit partition");
        f(contrib, "contributor mask"); f(trect, "tile rects"); f(keys0, "keys"); f(keys1, "keys");
        f(vals0, "values"); f(vals1, "values"); f(ranges, "tile ranges"); f(tl, "pixel state");
        f(acc, "gradient accumulators"); f(scratch_image, "scratch image"); f(dkeys0, "depth keys");
        f(dkeys1, "depth keys"); f(dvals0, "depth values"); f(dvals1, "depth values");
        f(counts_sorted, "sorted counts"); f(tile_order, "tile order"); f(meta, "face orders");
        f(tsort, "tile sort list");
    }
};

namespace {

lp_status fail(lp_ctx* ctx, lp_status s, const char* fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return s;
}

#define LP_CUDA(call)                                                                        \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail(ctx, LP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_));          \
    } while (0)

#define LP_TRY(expr)                    \
    do {                                \
        lp_status s_ = (expr);          \
        if (s_ != LP_OK) return s_;     \
    } while (0)

bool capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
    return cs != cudaStreamCaptureStatusNone;
}

template <typename T>
lp_status ensure(lp_ctx* ctx, DevBuf<T>& b, long long n, bool cap_mode, const char* what) {
    const size_t want = (size_t)(n > 0 ? n : 1);
    if (b.cap >= want) return LP_OK;
    if (cap_mode)
        return fail(ctx, LP_ERR_CAPACITY,
                    "%s needs %lld elements but %zu are reserved; call lp_reserve before capture",
                    what, (long long)want, b.cap);
    if (b.p) {
        cudaError_t e = cudaFree(b.p);
        if (e != cudaSuccess) return fail(ctx, LP_ERR_CUDA, "cudaFree: %s", cudaGetErrorString(e));
        b.p = nullptr;
        b.cap = 0;
    }
    const size_t grow = want + want / 4;
    const size_t guard = ctx->guard ? kGuardBytes : 0;
    cudaError_t e = cudaMalloc((void**)&b.p, grow * sizeof(T) + guard);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, LP_ERR_CUDA, "cudaMalloc(%s, %zu bytes): %s", what, grow * sizeof(T) + guard,
                    cudaGetErrorString(e));
    }
    b.cap = grow;
    b.guard = guard;
    if (guard) {
        // filled and finished before any later launch can touch the buffer
        e = cudaMemset(reinterpret_cast<unsigned char*>(b.p) + grow * sizeof(T), kGuardByte, guard);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return fail(ctx, LP_ERR_CUDA, "guard fill: %s", cudaGetErrorString(e));
    }
    return LP_OK;
}

template <typename T> void release(DevBuf<T>& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    b.guard = 0;
}

int rec_floats(int V) { return V == 6 ? lp::Rec<6>::kFloats : lp::Rec<4>::kFloats; }
int acc_floats(int V) { return V == 6 ? lp::Acc<6>::kFloats : lp::Acc<4>::kFloats; }
int rec_floats_mode(int V, bool exact) { return exact ? lp::rec_floats_x(V) : rec_floats(V); }
int acc_floats_mode(int V, bool exact) { return exact ? lp::acc_floats_x(V) : acc_floats(V); }
// the largest record / accumulator of either kind and mode (for lp_reserve)
int rec_floats_max() { return std::max(rec_floats(6), lp::rec_floats_x(6)); }
int acc_floats_max() { return std::max(acc_floats(6), lp::acc_floats_x(6)); }

lp_status check_prims(lp_ctx* ctx, const lp_prims* p) {
    if (!p) return fail(ctx, LP_ERR_INVALID, "prims is NULL");
    if (p->kind != LP_OCTAHEDRON && p->kind != LP_TETRAHEDRON)
        return fail(ctx, LP_ERR_INVALID, "kind %d is neither LP_OCTAHEDRON nor LP_TETRAHEDRON", p->kind);
    if (p->n < 0) return fail(ctx, LP_ERR_INVALID, "n = %d < 0", p->n);
    if (p->sh_degree < 0 || p->sh_degree > 3)
        return fail(ctx, LP_ERR_INVALID, "sh_degree %d outside 0..3", p->sh_degree);
    if (p->n > 0 && (!p->centre || !p->verts || !p->opacity || !p->sh))
        return fail(ctx, LP_ERR_INVALID, "a primitive array is NULL");
    return LP_OK;
}

lp_status build_cams(lp_ctx* ctx, const lp_camera* cams, int n_cams, int tile, lp::CamsParam& out,
                     long long& pixels, long long& tiles) {
    if (!cams) return fail(ctx, LP_ERR_INVALID, "cams is NULL");
    if (n_cams < 1 || n_cams > LP_MAX_CAMERAS)
        return fail(ctx, LP_ERR_INVALID, "n_cams = %d outside 1..%d", n_cams, LP_MAX_CAMERAS);
    memset(&out, 0, sizeof(out));
    out.n = n_cams;
    out.tile = tile;
    long long tb = 0, pb = 0;
    for (int c = 0; c < n_cams; ++c) {
        const lp_camera& s = cams[c];
        if (s.width < 1 || s.height < 1 || s.width > 65536 || s.height > 65536)
            return fail(ctx, LP_ERR_INVALID, "camera %d has size %dx%d", c, s.width, s.height);
        lp::CamDev& d = out.cam[c];
        double R[3][3], T[3];
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) {
                R[i][j] = s.viewmat[4 * i + j];
                d.R[3 * i + j] = s.viewmat[4 * i + j];
            }
            T[i] = s.viewmat[4 * i + 3];
            d.T[i] = s.viewmat[4 * i + 3];
        }
        for (int j = 0; j < 3; ++j)
            d.campos[j] = (float)(-(R[0][j] * T[0] + R[1][j] * T[1] + R[2][j] * T[2]));
        d.fx = s.fx; d.fy = s.fy; d.cx = s.cx; d.cy = s.cy;
        d.width = s.width; d.height = s.height;
        d.tiles_x = (s.width + tile - 1) / tile;
        d.tiles_y = (s.height + tile - 1) / tile;
        d.tile_base = (int)tb;
        d.pix_base = (int)pb;
        tb += (long long)d.tiles_x * d.tiles_y;
        pb += (long long)s.width * s.height;
    }
    if (pb > (1ll << 30) || tb > (1ll << 30))
        return fail(ctx, LP_ERR_INVALID, "too many pixels (%lld) or tiles (%lld)", pb, tb);
    out.total_tiles = (int)tb;
    out.total_pixels = (int)pb;
    pixels = pb;
    tiles = tb;
    return LP_OK;
}

void mark(lp_ctx* ctx, cudaStream_t st, int i, bool cap_mode) {
    if (!ctx->timing) return;
    cudaEventRecordWithFlags(ctx->ev[i], st, cap_mode ? cudaEventRecordExternal : cudaEventRecordDefault);
}

// Persistent blend grid for schedule t: resident blocks per SM (tuned, or
// what fits) x SMs, never more blocks than tiles.
int blend_grid(const lp_ctx* ctx, const lp_tuning& t, int V, bool fwd, long long tiles, bool exact = false) {
    int bps = t.blocks_per_sm;
    if (exact) {
        bps = lp::blend_x_occupancy(t.tile, V, fwd);
        if (bps <= 0) bps = 1;
    } else if (bps <= 0) {
        bps = fwd ? lp::blend_fwd_occupancy(t.tile, V, t.batch, t.pixels_per_thread)
                  : lp::blend_bwd_occupancy(t.tile, V, t.batch, t.pixels_per_thread);
        if (bps <= 0) bps = 1;
    }
    const long long g = (long long)ctx->sms * bps;
    return (int)(tiles < g ? tiles : g);
}

// Rows of the contributor mask per tile for a schedule (one per lane group
// of each warp; one per warp for the exact-span blends); kMaskRowsMax bounds
// every supported schedule.
constexpr int kMaskRowsMax = 16 * lp::kLaneGroupsMax;
int mask_rows(const lp_tuning& t, bool exact) {
    return exact ? lp::blend_x_warps(t.tile) : lp::blend_mask_rows(t.tile, t.pixels_per_thread);
}

int bits_for(long long n) {   // bits needed to represent values 0 .. n-1
    int b = 0;
    while ((1ll << b) < n) ++b;
    return b;
}

}  // namespace

extern "C" {

const char* lp_status_string(lp_status s) {
    switch (s) {
        case LP_OK: return "LP_OK";
        case LP_ERR_INVALID: return "LP_ERR_INVALID";
        case LP_ERR_CAPACITY: return "LP_ERR_CAPACITY";
        case LP_ERR_CUDA: return "LP_ERR_CUDA";
        case LP_ERR_TIMEOUT: return "LP_ERR_TIMEOUT";
        case LP_ERR_UNSUPPORTED: return "LP_ERR_UNSUPPORTED";
        case LP_ERR_STATE: return "LP_ERR_STATE";
    }
    return "LP_ERR_UNKNOWN";
}

const char* lp_last_error(lp_ctx* ctx) { return ctx ? ctx->err : "no context"; }

lp_status lp_create(lp_ctx** out, int device) {
    if (!out) return LP_ERR_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return LP_ERR_CUDA;
    }
    lp_ctx* ctx = new lp_ctx();
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_E, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_tile_counter, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_pairs, 4 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_order_scratch, 68 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_order_scratch, 0, 68 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->h_E, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_E, 0, sizeof(uint32_t));
    if (e != cudaSuccess) {
        cudaGetLastError();
        lp_destroy(ctx);
        return LP_ERR_CUDA;
    }
    *out = ctx;
    return LP_OK;
}

void lp_destroy(lp_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    ctx->each_buf([](auto& b, const char*) { release(b); });
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->d_E) cudaFree(ctx->d_E);
    if (ctx->d_tile_counter) cudaFree(ctx->d_tile_counter);
    if (ctx->d_pairs) cudaFree(ctx->d_pairs);
    if (ctx->d_order_scratch) cudaFree(ctx->d_order_scratch);
    if (ctx->h_E) cudaFreeHost(ctx->h_E);
    for (cudaEvent_t& e : ctx->ev)
        if (e) cudaEventDestroy(e);
    delete ctx;
}

lp_status lp_set_tuning(lp_ctx* ctx, const lp_tuning* t) {
    if (!ctx || !t) return LP_ERR_INVALID;
    if (t->tile != 8 && t->tile != 16 && t->tile != 32)
        return fail(ctx, LP_ERR_INVALID, "tile %d not in {8, 16, 32}", t->tile);
    if (t->batch != 32 && t->batch != 64 && t->batch != 128)
        return fail(ctx, LP_ERR_INVALID, "batch %d not in {32, 64, 128}", t->batch);
    if (t->blocks_per_sm < 0 || t->blocks_per_sm > 32)
        return fail(ctx, LP_ERR_INVALID, "blocks_per_sm %d outside 0..32", t->blocks_per_sm);
    if (t->pixels_per_thread != 1 && t->pixels_per_thread != 2 && t->pixels_per_thread != 4)
        return fail(ctx, LP_ERR_INVALID, "pixels_per_thread %d not in {1, 2, 4}", t->pixels_per_thread);
    if (!lp::tile_pix_ok(t->tile, t->pixels_per_thread))
        return fail(ctx, LP_ERR_INVALID, "pixels_per_thread %d is not built for %dx%d tiles (8: 1, 2; 16: 1, 2, 4; "
                    "32: 2, 4)", t->pixels_per_thread, t->tile, t->tile);
    if (t->sort_mode < 0 || t->sort_mode > 2)
        return fail(ctx, LP_ERR_INVALID, "sort_mode %d not in {0, 1, 2}", t->sort_mode);
    if (t->chain_split != 0 && t->chain_split != 1)
        return fail(ctx, LP_ERR_INVALID, "chain_split %d not in {0, 1}", t->chain_split);
    if (t->radix_bits != 4 && t->radix_bits != 6 && t->radix_bits != 8 && t->radix_bits != 11)
        return fail(ctx, LP_ERR_INVALID, "radix_bits %d not in {4, 6, 8, 11}", t->radix_bits);
    if (t->tile_order != 0 && t->tile_order != 1)
        return fail(ctx, LP_ERR_INVALID, "tile_order %d not in {0, 1}", t->tile_order);
    if (t->onesweep != 0 && t->onesweep != 1)
        return fail(ctx, LP_ERR_INVALID, "onesweep %d not in {0, 1}", t->onesweep);
    ctx->tune = *t;
    return LP_OK;
}

lp_status lp_get_tuning(lp_ctx* ctx, lp_tuning* t) {
    if (!ctx || !t) return LP_ERR_INVALID;
    *t = ctx->tune;
    return LP_OK;
}

lp_status lp_set_filter_2d(lp_ctx* ctx, float kernel_px) {
    if (!ctx) return LP_ERR_INVALID;
    if (!(kernel_px >= 0.f && kernel_px <= 16.f))
        return fail(ctx, LP_ERR_INVALID, "2D filter size %g outside [0, 16] px", (double)kernel_px);
    ctx->aa_kernel = kernel_px;
    return LP_OK;
}

lp_status lp_set_densify_stats(lp_ctx* ctx, float* grad_sum, unsigned int* grad_count,
                               unsigned int* px_max, long long n) {
    if (!ctx) return LP_ERR_INVALID;
    const bool none = !grad_sum && !grad_count && !px_max;
    if (!none && (!grad_sum || !grad_count || !px_max || n < 0))
        return fail(ctx, LP_ERR_INVALID, "densification statistics need all three arrays and n >= 0");
    ctx->st_grad_sum = grad_sum;
    ctx->st_grad_count = grad_count;
    ctx->st_px_max = px_max;
    ctx->st_n = none ? 0 : n;
    return LP_OK;
}

lp_status lp_set_exact(lp_ctx* ctx, int exact) {
    if (!ctx) return LP_ERR_INVALID;
    ctx->exact = exact != 0;
    return LP_OK;
}

lp_status lp_get_exact(lp_ctx* ctx, int* exact) {
    if (!ctx || !exact) return LP_ERR_INVALID;
    *exact = ctx->exact ? 1 : 0;
    return LP_OK;
}

lp_status lp_get_filter_2d(lp_ctx* ctx, float* kernel_px) {
    if (!ctx || !kernel_px) return LP_ERR_INVALID;
    *kernel_px = ctx->aa_kernel;
    return LP_OK;
}

static lp_status reserve_impl(lp_ctx* ctx, long long records, long long entries, long long pixels,
                              long long tiles, int V) {
    const int rf = V ? rec_floats_mode(V, ctx->exact) : rec_floats_max();
    LP_TRY(ensure(ctx, ctx->rec, records * rf, false, "records"));
    LP_TRY(ensure(ctx, ctx->counts, records, false, "counts"));
    LP_TRY(ensure(ctx, ctx->meta, records, false, "face orders"));
    LP_TRY(ensure(ctx, ctx->offsets, records, false, "offsets"));
    LP_TRY(ensure(ctx, ctx->zbits, records, false, "zbits"));
    LP_TRY(ensure(ctx, ctx->trect, records, false, "tile rects"));
    LP_TRY(ensure(ctx, ctx->keys0, entries, false, "keys"));
    LP_TRY(ensure(ctx, ctx->keys1, entries, false, "keys"));
    LP_TRY(ensure(ctx, ctx->vals0, entries, false, "values"));
    LP_TRY(ensure(ctx, ctx->vals1, entries, false, "values"));
    LP_TRY(ensure(ctx, ctx->dkeys0, records, false, "depth keys"));
    LP_TRY(ensure(ctx, ctx->dkeys1, records, false, "depth keys"));
    LP_TRY(ensure(ctx, ctx->dvals0, records, false, "depth values"));
    LP_TRY(ensure(ctx, ctx->dvals1, records, false, "depth values"));
    LP_TRY(ensure(ctx, ctx->counts_sorted, records, false, "sorted counts"));
    // a captured forward sorts up to the smallest key/value capacity, which
    // the allocator may have rounded up past `entries`
    long long kcap = (long long)ctx->keys0.cap;
    if ((long long)ctx->keys1.cap < kcap) kcap = ctx->keys1.cap;
    if ((long long)ctx->vals0.cap < kcap) kcap = ctx->vals0.cap;
    if ((long long)ctx->vals1.cap < kcap) kcap = ctx->vals1.cap;
    const long long hmax = kcap > records ? kcap : records;
    LP_TRY(ensure(ctx, ctx->hist, (long long)lp::sort_hist_elems(hmax), false, "histograms"));
    long long sb = lp::scan_blocks(records);
    long long sb2 = lp::scan_blocks((long long)lp::sort_hist_elems(hmax));
    LP_TRY(ensure(ctx, ctx->scan_tmp, sb > sb2 ? sb : sb2, false, "scan blocks"));
    LP_TRY(ensure(ctx, ctx->emit_part, (long long)lp::emit_blocks(records, kcap) + 1, false, "emit partition"));
    LP_TRY(ensure(ctx, ctx->contrib, (kcap / 32 + 2) * kMaskRowsMax, false, "contributor mask"));
    LP_TRY(ensure(ctx, ctx->ranges, tiles, false, "tile ranges"));
    LP_TRY(ensure(ctx, ctx->tile_order, tiles, false, "tile order"));
    LP_TRY(ensure(ctx, ctx->tsort, (tiles > 0 ? tiles : 1) + 2, false, "tile sort list"));
    LP_TRY(ensure(ctx, ctx->last, pixels, false, "pixel state"));
    LP_TRY(ensure(ctx, ctx->tl, pixels, false, "pixel state"));
    const int af = V ? acc_floats_mode(V, ctx->exact) : acc_floats_max();
    LP_TRY(ensure(ctx, ctx->acc, records * af, false, "gradient accumulators"));
    return LP_OK;
}

lp_status lp_reserve(lp_ctx* ctx, long long max_records, long long max_entries, long long max_pixels,
                     long long max_tiles) {
    if (!ctx) return LP_ERR_INVALID;
    if (max_records < 0 || max_entries < 0 || max_pixels < 0 || max_tiles < 0 ||
        max_entries > 0xffffffffll)
        return fail(ctx, LP_ERR_INVALID, "bad reserve sizes");
    LP_CUDA(cudaSetDevice(ctx->device));
    return reserve_impl(ctx, max_records, max_entries, max_pixels, max_tiles, 0);
}

lp_status lp_render_forward(lp_ctx* ctx, const lp_prims* prims, const lp_camera* cams, int n_cams,
                            const float bg[3], float* images, void* stream) {
    if (!ctx) return LP_ERR_INVALID;
    ctx->err[0] = 0;
    LP_TRY(check_prims(ctx, prims));
    if (!bg) return fail(ctx, LP_ERR_INVALID, "bg is NULL");
    if (!images) return fail(ctx, LP_ERR_INVALID, "images is NULL");
    LP_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const bool cap_mode = capturing(st);
    const int V = prims->kind;
    lp::CamsParam cp;
    long long pixels = 0, tiles = 0;
    LP_TRY(build_cams(ctx, cams, n_cams, ctx->tune.tile, cp, pixels, tiles));
    // the 2D filter's vertex move, rounded once to binary32 from the size (the
    // exact mode has no filter)
    const bool exact = ctx->exact;
    cp.aa_half = exact ? 0.f : (float)(0.5 * (double)ctx->aa_kernel);
    cp.aa_full = exact ? 0.f : ctx->aa_kernel;
    const long long records = (long long)n_cams * prims->n;
    if (records > 0x7fffffffll) return fail(ctx, LP_ERR_INVALID, "too many records (%lld)", records);
    ctx->have_fwd = false;

    LP_TRY(ensure(ctx, ctx->rec, records * rec_floats_mode(V, exact), cap_mode, "records"));
    LP_TRY(ensure(ctx, ctx->counts, records, cap_mode, "counts"));
    LP_TRY(ensure(ctx, ctx->offsets, records, cap_mode, "offsets"));
    LP_TRY(ensure(ctx, ctx->zbits, records, cap_mode, "zbits"));
    LP_TRY(ensure(ctx, ctx->trect, records, cap_mode, "tile rects"));
    LP_TRY(ensure(ctx, ctx->scan_tmp, lp::scan_blocks(records), cap_mode, "scan blocks"));
    LP_TRY(ensure(ctx, ctx->ranges, tiles, cap_mode, "tile ranges"));
    LP_TRY(ensure(ctx, ctx->last, pixels, cap_mode, "pixel state"));
    LP_TRY(ensure(ctx, ctx->tl, pixels, cap_mode, "pixel state"));

    lp::PrimsDev P{prims->n, prims->centre, prims->verts, prims->opacity, prims->sh};
    if (ctx->st_px_max) {
        if (prims->n > ctx->st_n)
            return fail(ctx, LP_ERR_INVALID, "densification statistics hold %lld primitives, the call has %d",
                        ctx->st_n, prims->n);
        P.px_max = ctx->st_px_max;
    }
    mark(ctx, st, 0, cap_mode);
    if (exact)
        LP_CUDA(lp::launch_preprocess_x(V, prims->sh_degree, P, cp, ctx->rec.p, ctx->counts.p, ctx->trect.p,
                                        ctx->zbits.p, st));
    else {
        LP_TRY(ensure(ctx, ctx->meta, records, cap_mode, "face orders"));
        LP_CUDA(lp::launch_preprocess(V, prims->sh_degree, P, cp, ctx->rec.p, ctx->counts.p, ctx->trect.p,
                                      ctx->zbits.p, ctx->meta.p, st));
    }
    mark(ctx, st, 1, cap_mode);
    const int mode = ctx->tune.sort_mode;
    int passes = 0, passes1 = 0;
    const uint32_t* order = nullptr;   // mode 1: records in depth order
    if (mode == 1) {
        LP_TRY(ensure(ctx, ctx->dkeys0, records, cap_mode, "depth keys"));
        LP_TRY(ensure(ctx, ctx->dkeys1, records, cap_mode, "depth keys"));
        LP_TRY(ensure(ctx, ctx->dvals0, records, cap_mode, "depth values"));
        LP_TRY(ensure(ctx, ctx->dvals1, records, cap_mode, "depth values"));
        LP_TRY(ensure(ctx, ctx->counts_sorted, records, cap_mode, "sorted counts"));
        LP_TRY(ensure(ctx, ctx->hist, (long long)lp::sort_hist_elems(records), cap_mode, "histograms"));
        LP_TRY(ensure(ctx, ctx->scan_tmp, lp::scan_blocks((long long)lp::sort_hist_elems(records)),
                      cap_mode, "scan blocks"));
        // stage 1: records by centre depth
        LP_CUDA(lp::launch_depth_keys(ctx->counts.p, ctx->zbits.p, records, ctx->dkeys0.p, ctx->dvals0.p, st));
        LP_CUDA(lp::launch_radix_sort32(ctx->dkeys0.p, ctx->dvals0.p, ctx->dkeys1.p, ctx->dvals1.p, nullptr,
                                        records, 32, ctx->tune.radix_bits, ctx->hist.p, ctx->scan_tmp.p,
                                        lp::SortCtl{ctx->sms, ctx->d_status, -1, ctx->tune.onesweep != 0}, &passes1, st));
        order = (passes1 & 1) ? ctx->dvals1.p : ctx->dvals0.p;
        LP_CUDA(lp::launch_gather_counts(ctx->counts.p, order, records, ctx->counts_sorted.p, st));
        LP_CUDA(lp::launch_scan(ctx->counts_sorted.p, records, ctx->offsets.p, ctx->scan_tmp.p, ctx->d_E,
                                st, ctx->d_status));
    } else {
        LP_CUDA(lp::launch_scan(ctx->counts.p, records, ctx->offsets.p, ctx->scan_tmp.p, ctx->d_E, st,
                                ctx->d_status));
    }

    long long bound;
    if (!cap_mode) {
        LP_CUDA(cudaMemcpyAsync(ctx->h_E, ctx->d_E, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
        LP_CUDA(cudaStreamSynchronize(st));
        bound = *ctx->h_E;
        if (*ctx->h_E == lp::kListOverflow) {
            // the scan latched the capacity bit too; clear it, this call reports it
            LP_CUDA(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
            ctx->E_host = -1;
            return fail(ctx, LP_ERR_CAPACITY, "tile list of 2^32 - 1 or more entries");
        }
        ctx->E_host = bound;
        LP_TRY(ensure(ctx, ctx->keys0, bound, false, "keys"));
        LP_TRY(ensure(ctx, ctx->keys1, bound, false, "keys"));
        LP_TRY(ensure(ctx, ctx->vals0, bound, false, "values"));
        LP_TRY(ensure(ctx, ctx->vals1, bound, false, "values"));
    } else {
        bound = (long long)ctx->keys0.cap;
        if ((long long)ctx->keys1.cap < bound) bound = ctx->keys1.cap;
        if ((long long)ctx->vals0.cap < bound) bound = ctx->vals0.cap;
        if ((long long)ctx->vals1.cap < bound) bound = ctx->vals1.cap;
        ctx->E_host = -1;
    }
    LP_TRY(ensure(ctx, ctx->hist, (long long)lp::sort_hist_elems(bound), cap_mode, "histograms"));
    LP_TRY(ensure(ctx, ctx->scan_tmp, lp::scan_blocks((long long)lp::sort_hist_elems(bound)), cap_mode,
                  "scan blocks"));
    LP_TRY(ensure(ctx, ctx->emit_part, (long long)lp::emit_blocks(records, bound) + 1, cap_mode,
                  "emit partition"));
    const int mrows = mask_rows(ctx->tune, exact);
    LP_TRY(ensure(ctx, ctx->contrib, (bound / 32 + 2) * mrows, cap_mode, "contributor mask"));
    ctx->contrib_stride = (uint32_t)(bound / 32 + 2);

    const int tile_bits = bits_for(tiles);
    int key_bits;
    const uint32_t* svals;
    if (mode != 0) {
        // mode 1, stage 2: entries in depth order, stably sorted by their tile
        // id.  Mode 2: entries in record order, stably sorted by tile id, then
        // each tile's run by depth.
        uint32_t* t0 = reinterpret_cast<uint32_t*>(ctx->keys0.p);
        uint32_t* t1 = reinterpret_cast<uint32_t*>(ctx->keys1.p);
        if (mode == 2)
            LP_TRY(ensure(ctx, ctx->tsort, (tiles > 0 ? tiles : 1) + 2, cap_mode, "tile sort list"));
        LP_CUDA(lp::launch_emit_sorted(mode == 1 ? order : nullptr, mode == 1 ? ctx->counts_sorted.p : ctx->counts.p,
                                       ctx->offsets.p, ctx->trect.p, records, ctx->d_E, bound, ctx->emit_part.p, t0,
                                       ctx->vals0.p, bound, ctx->d_status, st));
        mark(ctx, st, 2, cap_mode);
        key_bits = tile_bits;
        LP_CUDA(lp::launch_radix_sort32(t0, ctx->vals0.p, t1, ctx->vals1.p, ctx->d_E, bound, key_bits,
                                        ctx->tune.radix_bits, ctx->hist.p, ctx->scan_tmp.p,
                                        lp::SortCtl{ctx->sms, ctx->d_status, ctx->stall_block, ctx->tune.onesweep != 0}, &passes,
                                        st));
        const bool in1 = (passes & 1) != 0;
        svals = in1 ? ctx->vals1.p : ctx->vals0.p;
        mark(ctx, st, 3, cap_mode);
        LP_CUDA(cudaMemsetAsync(ctx->ranges.p, 0, (size_t)(tiles > 0 ? tiles : 1) * sizeof(uint2), st));
        LP_CUDA(lp::launch_ranges32(in1 ? t1 : t0, ctx->d_E, bound, ctx->d_status, ctx->ranges.p, ctx->sms,
                                    st));
        if (mode == 2) {
            // scratch: the key buffer that does not hold the sorted tile ids,
            // as two 4-byte arrays of the list's length
            uint32_t* sa = reinterpret_cast<uint32_t*>(in1 ? ctx->keys0.p : ctx->keys1.p);
            const long long tiles_alloc = tiles > 0 ? tiles : 1;
            LP_CUDA(lp::launch_tile_sort(in1 ? ctx->vals1.p : ctx->vals0.p, ctx->ranges.p, tiles, ctx->zbits.p,
                                         reinterpret_cast<int*>(ctx->tsort.p + tiles_alloc), ctx->tsort.p, sa,
                                         sa + bound, ctx->d_status, ctx->sms, st));
        }
        ctx->result_in_1 = in1;
    } else {
        LP_CUDA(lp::launch_emit(ctx->counts.p, ctx->offsets.p, ctx->trect.p, ctx->zbits.p, records, ctx->d_E,
                                bound, ctx->emit_part.p, ctx->keys0.p, ctx->vals0.p, bound, ctx->d_status, st));
        mark(ctx, st, 2, cap_mode);
        key_bits = 32 + tile_bits;
        LP_CUDA(lp::launch_radix_sort(ctx->keys0.p, ctx->vals0.p, ctx->keys1.p, ctx->vals1.p, ctx->d_E,
                                      bound, key_bits, ctx->tune.radix_bits, ctx->hist.p, ctx->scan_tmp.p,
                                      lp::SortCtl{ctx->sms, ctx->d_status, ctx->stall_block, ctx->tune.onesweep != 0}, &passes,
                                        st));
        const bool in1 = (passes & 1) != 0;
        svals = in1 ? ctx->vals1.p : ctx->vals0.p;
        mark(ctx, st, 3, cap_mode);
        LP_CUDA(cudaMemsetAsync(ctx->ranges.p, 0, (size_t)(tiles > 0 ? tiles : 1) * sizeof(uint2), st));
        LP_CUDA(lp::launch_ranges(in1 ? ctx->keys1.p : ctx->keys0.p, ctx->d_E, bound, ctx->d_status,
                                  ctx->ranges.p, ctx->sms, st));
        ctx->result_in_1 = in1;
    }
    if (ctx->tune.tile_order) {
        LP_TRY(ensure(ctx, ctx->tile_order, tiles, cap_mode, "tile order"));
        LP_CUDA(lp::launch_tile_order(ctx->ranges.p, tiles, ctx->tile_order.p, ctx->d_order_scratch, st));
    }
    mark(ctx, st, 4, cap_mode);

    lp::BlendArgs a{};
    a.grid = blend_grid(ctx, ctx->tune, V, true, tiles, exact);
    a.order = ctx->tune.tile_order ? ctx->tile_order.p : nullptr;
    a.rec = ctx->rec.p;
    a.vals = svals;
    a.ranges = ctx->ranges.p;
    a.cams = &cp;
    a.bg[0] = bg[0]; a.bg[1] = bg[1]; a.bg[2] = bg[2];
    a.image = images;
    a.last = ctx->last.p;
    a.tl = ctx->tl.p;
    a.tile_counter = ctx->d_tile_counter;
    a.pair_counts = ctx->d_pairs;
    a.count = false;
    a.contrib = ctx->contrib.p;
    a.contrib_stride = ctx->contrib_stride;
    LP_CUDA(cudaMemsetAsync(ctx->contrib.p, 0, (size_t)(bound / 32 + 2) * mrows * sizeof(uint32_t), st));
    LP_CUDA(cudaMemsetAsync(ctx->d_tile_counter, 0, sizeof(int), st));
    if (a.grid > 0) {
        if (exact) LP_CUDA(lp::launch_blend_fwd_x(ctx->tune.tile, V, a, st));
        else LP_CUDA(lp::launch_blend_fwd(ctx->tune.tile, V, ctx->tune.batch, ctx->tune.pixels_per_thread, a, st));
    }
    mark(ctx, st, 5, cap_mode);
    ctx->fwd_timed = ctx->timing;
    // kernels of a sort in the onesweep form: histogram and bases, then one per pass
    const bool sweep = ctx->tune.onesweep != 0;
    auto sort_kernels = [sweep](int p, long long n) { return p == 0 ? 0 : (sweep && n < (1ll << 30) ? 2 + p : 5 * p); };
    ctx->launches_fwd = 1 + (records > 0 ? 3 : 0) + (records > 0 ? 1 : 0) + sort_kernels(passes, bound) +
                        sort_kernels(passes1, records) +
                        (mode == 1 && records > 0 ? 2 : 0) + (bound > 0 ? 1 : 0) + (a.grid > 0 ? 1 : 0) +
                        (mode == 2 && tiles > 0 ? 2 : 0) +
                        (ctx->tune.tile_order && tiles > 0 ? 3 : 0);

    ctx->have_fwd = true;
    ctx->prims = *prims;
    ctx->cams = cp;
    ctx->bg[0] = bg[0]; ctx->bg[1] = bg[1]; ctx->bg[2] = bg[2];
    ctx->records = records;
    ctx->pixels = pixels;
    ctx->tiles = tiles;
    ctx->E_bound = bound;
    ctx->key_bits = key_bits;
    ctx->sort_passes = passes1 + passes;
    ctx->keys32 = mode != 0;
    ctx->fwd_exact = exact;
    ctx->fwd_tune = ctx->tune;
    return LP_OK;
}

lp_status lp_render_backward(lp_ctx* ctx, const float* dL_dimages, float* dcentre, float* dverts,
                             float* dopacity, float* dsh, int accumulate, void* stream) {
    if (!ctx) return LP_ERR_INVALID;
    ctx->err[0] = 0;
    if (!ctx->have_fwd) return fail(ctx, LP_ERR_STATE, "lp_render_backward without a forward");
    const lp_prims& pr = ctx->prims;
    if (!dL_dimages) return fail(ctx, LP_ERR_INVALID, "dL_dimages is NULL");
    if (pr.n > 0 && (!dcentre || !dverts || !dopacity || !dsh))
        return fail(ctx, LP_ERR_INVALID, "a gradient output is NULL");
    LP_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const bool cap_mode = capturing(st);
    const int V = pr.kind;
    mark(ctx, st, 6, cap_mode);
    const bool exact = ctx->fwd_exact;
    const long long acc_n = (ctx->records > 0 ? ctx->records : 1) * acc_floats_mode(V, exact);
    LP_TRY(ensure(ctx, ctx->acc, acc_n, cap_mode, "gradient accumulators"));
    LP_CUDA(cudaMemsetAsync(ctx->acc.p, 0, (size_t)acc_n * sizeof(float), st));

    lp::BlendArgs a{};
    const lp_tuning& ft = ctx->fwd_tune;   // the backward walks the forward's tiles and masks
    a.grid = blend_grid(ctx, ft, ctx->prims.kind, false, ctx->tiles, exact);
    a.order = ft.tile_order ? ctx->tile_order.p : nullptr;
    a.rec = ctx->rec.p;
    a.vals = ctx->result_in_1 ? ctx->vals1.p : ctx->vals0.p;
    a.ranges = ctx->ranges.p;
    a.cams = &ctx->cams;
    a.bg[0] = ctx->bg[0]; a.bg[1] = ctx->bg[1]; a.bg[2] = ctx->bg[2];
    a.dimage = dL_dimages;
    a.last = ctx->last.p;
    a.tl = ctx->tl.p;
    a.acc = ctx->acc.p;
    // the colour block follows the plane block (ray-space accumulators)
    a.acc_col = exact ? nullptr
                      : ctx->acc.p + (size_t)ctx->records * (V == 6 ? lp::Acc<6>::kPlane : lp::Acc<4>::kPlane);
    a.contrib = ctx->contrib.p;
    a.contrib_stride = ctx->contrib_stride;
    a.tile_counter = ctx->d_tile_counter + 1;
    LP_CUDA(cudaMemsetAsync(ctx->d_tile_counter + 1, 0, sizeof(int), st));
    if (a.grid > 0) {
        if (exact) LP_CUDA(lp::launch_blend_bwd_x(ft.tile, V, a, st));
        else LP_CUDA(lp::launch_blend_bwd(ft.tile, V, ft.batch, ft.pixels_per_thread, a, st));
    }
    mark(ctx, st, 7, cap_mode);

    lp::PrimsDev P{pr.n, pr.centre, pr.verts, pr.opacity, pr.sh};
    if (ctx->st_grad_sum) {
        if (pr.n > ctx->st_n)
            return fail(ctx, LP_ERR_INVALID, "densification statistics hold %lld primitives, the call has %d",
                        ctx->st_n, pr.n);
        P.grad_sum = ctx->st_grad_sum;
        P.grad_count = ctx->st_grad_count;
    }
    if (exact)
        LP_CUDA(lp::launch_chain_x(V, pr.sh_degree, P, ctx->cams, ctx->rec.p, ctx->counts.p, ctx->acc.p, dcentre,
                                   dverts, dopacity, dsh, accumulate, st));
    else
        LP_CUDA(lp::launch_chain(V, pr.sh_degree, P, ctx->cams, ctx->meta.p, ctx->counts.p, ctx->acc.p, dcentre,
                                 dverts, dopacity, dsh, accumulate, ctx->tune.chain_split, st));
    mark(ctx, st, 8, cap_mode);
    ctx->bwd_timed = ctx->timing;
    return LP_OK;
}

lp_status lp_sync_status(lp_ctx* ctx, void* stream) {
    if (!ctx) return LP_ERR_INVALID;
    LP_CUDA(cudaSetDevice(ctx->device));
    LP_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int s = 0;
    LP_CUDA(cudaMemcpy(&s, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    LP_CUDA(cudaMemset(ctx->d_status, 0, sizeof(int)));
    if (s & lp::kStatusCapacity)
        return fail(ctx, LP_ERR_CAPACITY, "tile list exceeded the reserved capacity");
    if (s & lp::kStatusTimeout) return fail(ctx, LP_ERR_TIMEOUT, "a device-side wait expired");
    return LP_OK;
}

lp_status lp_get_stats(lp_ctx* ctx, lp_stats* out) {
    if (!ctx || !out) return LP_ERR_INVALID;
    out->records = ctx->records;
    out->entries = ctx->E_host;
    if (ctx->have_fwd && ctx->E_host < 0) {
        uint32_t e = 0;
        LP_CUDA(cudaSetDevice(ctx->device));
        LP_CUDA(cudaDeviceSynchronize());
        LP_CUDA(cudaMemcpy(&e, ctx->d_E, sizeof(uint32_t), cudaMemcpyDeviceToHost));
        out->entries = e;
    }
    out->tiles = ctx->tiles;
    out->pixels = ctx->pixels;
    out->sort_passes = ctx->sort_passes;
    out->key_bits = ctx->key_bits;
    out->launches_fwd = ctx->launches_fwd;
    out->launches_bwd = (ctx->tiles > 0 ? 1 : 0) + (ctx->prims.n > 0 ? 1 : 0);
    return LP_OK;
}

lp_status lp_set_timing(lp_ctx* ctx, int enabled) {
    if (!ctx) return LP_ERR_INVALID;
    LP_CUDA(cudaSetDevice(ctx->device));
    if (enabled)
        for (cudaEvent_t& e : ctx->ev)
            if (!e) LP_CUDA(cudaEventCreate(&e));
    ctx->timing = enabled != 0;
    return LP_OK;
}

lp_status lp_stage_times(lp_ctx* ctx, float* ms) {
    if (!ctx || !ms) return LP_ERR_INVALID;
    for (int i = 0; i < LP_NUM_STAGES; ++i) ms[i] = 0.f;
    if (!ctx->timing) return fail(ctx, LP_ERR_STATE, "timing is not enabled");
    LP_CUDA(cudaSetDevice(ctx->device));
    if (ctx->fwd_timed) {
        LP_CUDA(cudaEventSynchronize(ctx->ev[5]));
        for (int i = 0; i < 5; ++i) LP_CUDA(cudaEventElapsedTime(&ms[i], ctx->ev[i], ctx->ev[i + 1]));
    }
    if (ctx->bwd_timed) {
        LP_CUDA(cudaEventSynchronize(ctx->ev[8]));
        LP_CUDA(cudaEventElapsedTime(&ms[LP_STAGE_BLEND_BWD], ctx->ev[6], ctx->ev[7]));
        LP_CUDA(cudaEventElapsedTime(&ms[LP_STAGE_CHAIN], ctx->ev[7], ctx->ev[8]));
    }
    return LP_OK;
}

lp_status lp_debug_scan(lp_ctx* ctx, const unsigned int* counts, long long n, unsigned int* offsets,
                        unsigned int* total, void* stream) {
    if (!ctx || n < 0 || (n > 0 && (!counts || !offsets)) || !total) return LP_ERR_INVALID;
    LP_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    LP_TRY(ensure(ctx, ctx->scan_tmp, lp::scan_blocks(n) + 1, false, "scan blocks"));
    int s = 0;
    LP_CUDA(cudaMemcpyAsync(&s, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    LP_CUDA(cudaStreamSynchronize(st));
    if (s) return fail(ctx, LP_ERR_INVALID, "a status is latched; read it with lp_sync_status first");
    LP_CUDA(lp::launch_scan(counts, n, offsets, ctx->scan_tmp.p, ctx->d_E, st, ctx->d_status));
    LP_CUDA(cudaMemcpyAsync(ctx->h_E, ctx->d_E, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    LP_CUDA(cudaMemcpyAsync(&s, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    LP_CUDA(cudaStreamSynchronize(st));
    *total = *ctx->h_E;
    ctx->E_host = -1;
    ctx->have_fwd = false;
    if (s & lp::kStatusCapacity) {
        LP_CUDA(cudaMemset(ctx->d_status, 0, sizeof(int)));
        return fail(ctx, LP_ERR_CAPACITY, "scan total of 2^32 - 1 or more");
    }
    return LP_OK;
}

lp_status lp_debug_sort_stall(lp_ctx* ctx, int block) {
    if (!ctx || block < -1) return LP_ERR_INVALID;
    ctx->stall_block = block;
    return LP_OK;
}

lp_status lp_set_debug_guard(lp_ctx* ctx, int enabled) {
    if (!ctx) return LP_ERR_INVALID;
    ctx->guard = enabled != 0;
    return LP_OK;
}

lp_status lp_check_guards(lp_ctx* ctx, long long* checked, long long* damaged) {
    if (!ctx || !checked || !damaged) return LP_ERR_INVALID;
    LP_CUDA(cudaSetDevice(ctx->device));
    LP_CUDA(cudaDeviceSynchronize());
    *checked = 0;
    *damaged = 0;
    unsigned char host[kGuardBytes];
    lp_status st = LP_OK;
    const char* first = nullptr;
    ctx->each_buf([&](auto& b, const char* name) {
        if (st != LP_OK || !b.p || !b.guard) return;
        const unsigned char* zone = reinterpret_cast<const unsigned char*>(b.p + b.cap);
        if (cudaMemcpy(host, zone, b.guard, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            st = fail(ctx, LP_ERR_CUDA, "guard read of %s failed", name);
            return;
        }
        ++*checked;
        for (size_t q = 0; q < b.guard; ++q)
            if (host[q] != kGuardByte) {
                ++*damaged;
                if (!first) first = name;
            }
    });
    if (st == LP_OK && first) fail(ctx, LP_OK, "guard zone of %s written", first);
    return st;
}

lp_status lp_debug_keys(lp_ctx* ctx, unsigned long long* keys, unsigned int* vals, long long cap,
                        long long* n) {
    if (!ctx || !n) return LP_ERR_INVALID;
    if (!ctx->have_fwd) return fail(ctx, LP_ERR_STATE, "no forward");
    LP_CUDA(cudaSetDevice(ctx->device));
    LP_CUDA(cudaDeviceSynchronize());
    uint32_t e = 0;
    LP_CUDA(cudaMemcpy(&e, ctx->d_E, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    *n = e;
    long long m = e < cap ? e : cap;
    if (m > ctx->E_bound) m = ctx->E_bound;
    const uint32_t* dvals = ctx->result_in_1 ? ctx->vals1.p : ctx->vals0.p;
    if (m > 0 && vals) LP_CUDA(cudaMemcpy(vals, dvals, (size_t)m * 4, cudaMemcpyDeviceToHost));
    if (m > 0 && keys) {
        if (!ctx->keys32) {
            LP_CUDA(cudaMemcpy(keys, ctx->result_in_1 ? ctx->keys1.p : ctx->keys0.p, (size_t)m * 8,
                               cudaMemcpyDeviceToHost));
        } else {
            // the list is keyed by tile id only; the depth half is the record's depth bits
            uint32_t* tk = (uint32_t*)malloc((size_t)m * 4);
            uint32_t* tv = (uint32_t*)malloc((size_t)m * 4);
            uint32_t* zb = (uint32_t*)malloc((size_t)(ctx->records > 0 ? ctx->records : 1) * 4);
            if (!tk || !tv || !zb) {
                free(tk); free(tv); free(zb);
                return fail(ctx, LP_ERR_INVALID, "host allocation failed");
            }
            const uint64_t* src = ctx->result_in_1 ? ctx->keys1.p : ctx->keys0.p;
            cudaError_t e1 = cudaMemcpy(tk, src, (size_t)m * 4, cudaMemcpyDeviceToHost);
            cudaError_t e2 = cudaMemcpy(tv, dvals, (size_t)m * 4, cudaMemcpyDeviceToHost);
            cudaError_t e3 = cudaMemcpy(zb, ctx->zbits.p, (size_t)ctx->records * 4, cudaMemcpyDeviceToHost);
            if (e1 == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess)
                for (long long q = 0; q < m; ++q)
                    keys[q] = ((unsigned long long)tk[q] << 32) | zb[tv[q]];
            free(tk); free(tv); free(zb);
            if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
                return fail(ctx, LP_ERR_CUDA, "debug key copy failed");
        }
    }
    return LP_OK;
}

lp_status lp_debug_counts(lp_ctx* ctx, unsigned int* counts, long long cap) {
    if (!ctx || !counts) return LP_ERR_INVALID;
    if (!ctx->have_fwd) return fail(ctx, LP_ERR_STATE, "no forward");
    LP_CUDA(cudaSetDevice(ctx->device));
    LP_CUDA(cudaDeviceSynchronize());
    const long long m = ctx->records < cap ? ctx->records : cap;
    if (m > 0) LP_CUDA(cudaMemcpy(counts, ctx->counts.p, (size_t)m * 4, cudaMemcpyDeviceToHost));
    return LP_OK;
}

lp_status lp_debug_pixel_state(lp_ctx* ctx, unsigned int* last, float* T_last, long long cap) {
    if (!ctx) return LP_ERR_INVALID;
    if (!ctx->have_fwd) return fail(ctx, LP_ERR_STATE, "no forward");
    LP_CUDA(cudaSetDevice(ctx->device));
    LP_CUDA(cudaDeviceSynchronize());
    const long long m = ctx->pixels < cap ? ctx->pixels : cap;
    if (m > 0 && last) LP_CUDA(cudaMemcpy(last, ctx->last.p, (size_t)m * 4, cudaMemcpyDeviceToHost));
    if (m > 0 && T_last) LP_CUDA(cudaMemcpy(T_last, ctx->tl.p, (size_t)m * 4, cudaMemcpyDeviceToHost));
    return LP_OK;
}

lp_status lp_render_depth(lp_ctx* ctx, float* depth, void* stream) {
    if (!ctx) return LP_ERR_INVALID;
    if (!depth) return fail(ctx, LP_ERR_INVALID, "depth is NULL");
    if (!ctx->have_fwd) return fail(ctx, LP_ERR_STATE, "no forward");
    LP_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    lp::BlendArgs a{};
    const lp_tuning& ft = ctx->fwd_tune;
    a.grid = blend_grid(ctx, ft, ctx->prims.kind, true, ctx->tiles, ctx->fwd_exact);
    a.order = ft.tile_order ? ctx->tile_order.p : nullptr;
    a.rec = ctx->rec.p;
    a.vals = ctx->result_in_1 ? ctx->vals1.p : ctx->vals0.p;
    a.ranges = ctx->ranges.p;
    a.cams = &ctx->cams;
    a.tile_counter = ctx->d_tile_counter;
    a.pair_counts = ctx->d_pairs;
    a.depth = depth;
    LP_CUDA(cudaMemsetAsync(ctx->d_tile_counter, 0, sizeof(int), st));
    if (a.grid > 0 && ctx->fwd_exact)
        LP_CUDA(lp::launch_blend_fwd_x(ft.tile, ctx->prims.kind, a, st));
    else if (a.grid > 0)
        LP_CUDA(lp::launch_blend_fwd(ft.tile, ctx->prims.kind, ft.batch, ft.pixels_per_thread, a, st));
    else if (ctx->pixels > 0)
        LP_CUDA(cudaMemsetAsync(depth, 0, (size_t)ctx->pixels * sizeof(float), st));
    return LP_OK;
}

lp_status lp_count_pairs(lp_ctx* ctx, long long* counts) {
    if (!ctx || !counts) return LP_ERR_INVALID;
    if (!ctx->have_fwd) return fail(ctx, LP_ERR_STATE, "no forward");
    LP_CUDA(cudaSetDevice(ctx->device));
    LP_CUDA(cudaDeviceSynchronize());
    LP_TRY(ensure(ctx, ctx->scratch_image, 3 * ctx->pixels, false, "scratch image"));
    lp::BlendArgs a{};
    const lp_tuning& ft = ctx->fwd_tune;
    a.grid = blend_grid(ctx, ft, ctx->prims.kind, true, ctx->tiles, ctx->fwd_exact);
    a.order = ft.tile_order ? ctx->tile_order.p : nullptr;
    a.rec = ctx->rec.p;
    a.vals = ctx->result_in_1 ? ctx->vals1.p : ctx->vals0.p;
    a.ranges = ctx->ranges.p;
    a.cams = &ctx->cams;
    a.bg[0] = ctx->bg[0]; a.bg[1] = ctx->bg[1]; a.bg[2] = ctx->bg[2];
    a.image = ctx->scratch_image.p;
    a.last = ctx->last.p;
    a.tl = ctx->tl.p;
    a.tile_counter = ctx->d_tile_counter;
    a.pair_counts = ctx->d_pairs;
    a.count = true;
    LP_CUDA(cudaMemset(ctx->d_pairs, 0, 4 * sizeof(unsigned long long)));
    LP_CUDA(cudaMemset(ctx->d_tile_counter, 0, sizeof(int)));
    if (a.grid > 0 && ctx->fwd_exact) LP_CUDA(lp::launch_blend_fwd_x(ft.tile, ctx->prims.kind, a, 0));
    else if (a.grid > 0)
        LP_CUDA(lp::launch_blend_fwd(ft.tile, ctx->prims.kind, ft.batch, ft.pixels_per_thread, a, 0));
    LP_CUDA(cudaDeviceSynchronize());
    unsigned long long h[4] = {0, 0, 0, 0};
    LP_CUDA(cudaMemcpy(h, ctx->d_pairs, sizeof(h), cudaMemcpyDeviceToHost));
    for (int q = 0; q < 4; ++q) counts[q] = (long long)h[q];
    return LP_OK;
}

}  // extern "C"
