// Allocation-free forward render of one camera.
//
// Some callers cannot call cudaMalloc: memory-budgeted services whose device
// memory is owned by a pool or an allocator they may not bypass, and embedded
// or real-time hosts that forbid allocation after start-up.
// lp_render_forward_noalloc renders one camera with the same kernels as
// lp_render_forward, but every scratch buffer it needs lives in one
// file-scope __device__ array of fixed size, so the call itself never
// allocates device (or pinned host) memory.  It reads the tile-list length
// back after the key scan and the device status word at the end, so it
// synchronises the caller's stream twice.
//
// The array belongs to the library image: every GPU that loads the library
// holds it until the process exits.  All calls share it, so two calls whose
// work overlaps on the GPU (different streams, or different host threads)
// race; serialise them.  The array keeps the previous call's contents; each
// call clears what must start at zero.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "linprim.h"
#include "lp_device.cuh"
#include "lp_internal.h"

namespace {

// Limits of the allocation-free path.
constexpr long long kMaxPrims = 16384;      // primitives (one camera)
constexpr long long kMaxPixels = 512 * 512; // width * height
constexpr long long kMaxTiles = 2048;       // 16x16 tiles of the image
constexpr long long kMaxEntries = 262144;   // tile-list length E

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte offsets of the sub-buffers carved from the scratch array.
constexpr size_t kRecBytes = align256(kMaxPrims * lp::Rec<6>::kFloats * 4);
constexpr size_t kCountBytes = align256(kMaxPrims * 4);
constexpr size_t kRectBytes = align256(kMaxPrims * 16);
constexpr size_t kKeyBytes = align256(kMaxEntries * 8);
constexpr size_t kValBytes = align256(kMaxEntries * 4);
// the sort's workspace at 8-bit digits: histograms, digit bases and block
// counters of up to 16 passes, then one status word per (block, digit)
constexpr size_t kHistElems = 2 * 16 * 256 + 16 + 256 * ((kMaxEntries + 4095) / 4096);
constexpr size_t kHistBytes = align256(kHistElems * 4);
constexpr size_t kScanTmpBytes = align256(((kHistElems + 4095) / 4096 + 16) * 4);
constexpr size_t kRangeBytes = align256(kMaxTiles * 8);
constexpr size_t kPixBytes = align256(kMaxPixels * 4);
constexpr size_t kPartBytes = align256(((kMaxPrims + kMaxEntries + 1023) / 1024 + 2) * 4);
constexpr size_t kMiscBytes = 256;

constexpr size_t kOffRec = 0;
constexpr size_t kOffCounts = kOffRec + kRecBytes;
constexpr size_t kOffOffsets = kOffCounts + kCountBytes;
constexpr size_t kOffZbits = kOffOffsets + kCountBytes;
constexpr size_t kOffRect = kOffZbits + kCountBytes;
constexpr size_t kOffKeys0 = kOffRect + kRectBytes;
constexpr size_t kOffKeys1 = kOffKeys0 + kKeyBytes;
constexpr size_t kOffVals0 = kOffKeys1 + kKeyBytes;
constexpr size_t kOffVals1 = kOffVals0 + kValBytes;
constexpr size_t kOffHist = kOffVals1 + kValBytes;
constexpr size_t kOffScanTmp = kOffHist + kHistBytes;
constexpr size_t kOffRanges = kOffScanTmp + kScanTmpBytes;
constexpr size_t kOffLast = kOffRanges + kRangeBytes;
constexpr size_t kOffTl = kOffLast + kPixBytes;
constexpr size_t kOffPart = kOffTl + kPixBytes;
constexpr size_t kOffMisc = kOffPart + kPartBytes;   // E, status, tile counter, 4 pair counters
constexpr size_t kScratchBytes = kOffMisc + kMiscBytes;   // about 10.6 MiB

// The scratch itself.  In host code `g_scratch` names a host-side stand-in,
// not device memory: only the address from cudaGetSymbolAddress may be passed
// to kernels.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char* g_base[kMaxDevices] = {};

// Once per device, with that device current: the device address of the array.
lp_status scratch_base(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return LP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_base[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return LP_ERR_CUDA;
        }
        g_base[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_base[dev];
    return LP_OK;
}

int bits_for(long long n) {
    int b = 0;
    while ((1ll << b) < n) ++b;
    return b;
}

}  // namespace

extern "C" lp_status lp_render_forward_noalloc(const lp_prims* prims, const lp_camera* cam,
                                               const float bg[3], float* image, void* stream) {
    if (!prims || !cam || !bg || !image) return LP_ERR_INVALID;
    if (prims->kind != LP_OCTAHEDRON && prims->kind != LP_TETRAHEDRON) return LP_ERR_INVALID;
    if (prims->n < 0 || prims->sh_degree < 0 || prims->sh_degree > 3) return LP_ERR_INVALID;
    if (prims->n > 0 && (!prims->centre || !prims->verts || !prims->opacity || !prims->sh))
        return LP_ERR_INVALID;
    if (cam->width < 1 || cam->height < 1) return LP_ERR_INVALID;
    // sizes checked before any arithmetic on them
    if (prims->n > kMaxPrims || cam->width > kMaxPixels || cam->height > kMaxPixels) return LP_ERR_CAPACITY;
    const long long pixels = (long long)cam->width * cam->height;
    const int tile = 16;
    const int tiles_x = (cam->width + tile - 1) / tile, tiles_y = (cam->height + tile - 1) / tile;
    const long long tiles = (long long)tiles_x * tiles_y;
    if (pixels > kMaxPixels || tiles > kMaxTiles) return LP_ERR_CAPACITY;

    // the stream must belong to the current device, whose copy of the
    // scratch array the kernels are given
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sdev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaStreamGetDevice(st, &sdev) != cudaSuccess) {
        cudaGetLastError();
        return LP_ERR_CUDA;
    }
    if (sdev != dev) return LP_ERR_INVALID;
    unsigned char* base = nullptr;
    lp_status s = scratch_base(dev, &base);
    if (s != LP_OK) return s;
    float* rec = reinterpret_cast<float*>(base + kOffRec);
    uint32_t* counts = reinterpret_cast<uint32_t*>(base + kOffCounts);
    uint32_t* offsets = reinterpret_cast<uint32_t*>(base + kOffOffsets);
    uint32_t* zbits = reinterpret_cast<uint32_t*>(base + kOffZbits);
    int4* trect = reinterpret_cast<int4*>(base + kOffRect);
    uint64_t* keys0 = reinterpret_cast<uint64_t*>(base + kOffKeys0);
    uint64_t* keys1 = reinterpret_cast<uint64_t*>(base + kOffKeys1);
    uint32_t* vals0 = reinterpret_cast<uint32_t*>(base + kOffVals0);
    uint32_t* vals1 = reinterpret_cast<uint32_t*>(base + kOffVals1);
    uint32_t* hist = reinterpret_cast<uint32_t*>(base + kOffHist);
    uint32_t* scan_tmp = reinterpret_cast<uint32_t*>(base + kOffScanTmp);
    uint2* ranges = reinterpret_cast<uint2*>(base + kOffRanges);
    uint32_t* last = reinterpret_cast<uint32_t*>(base + kOffLast);
    float* tl = reinterpret_cast<float*>(base + kOffTl);
    uint32_t* part = reinterpret_cast<uint32_t*>(base + kOffPart);
    uint32_t* d_E = reinterpret_cast<uint32_t*>(base + kOffMisc);
    int* d_status = reinterpret_cast<int*>(base + kOffMisc + 4);
    int* d_tile_counter = reinterpret_cast<int*>(base + kOffMisc + 8);
    unsigned long long* d_pairs = reinterpret_cast<unsigned long long*>(base + kOffMisc + 16);   // 4 counters

    // camera, digested as for lp_render_forward
    lp::CamsParam cp;
    memset(&cp, 0, sizeof(cp));
    cp.n = 1;
    cp.tile = tile;
    cp.total_tiles = (int)tiles;
    cp.total_pixels = (int)pixels;
    lp::CamDev& d = cp.cam[0];
    double R[3][3], T[3];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            R[i][j] = cam->viewmat[4 * i + j];
            d.R[3 * i + j] = cam->viewmat[4 * i + j];
        }
        T[i] = cam->viewmat[4 * i + 3];
        d.T[i] = cam->viewmat[4 * i + 3];
    }
    for (int j = 0; j < 3; ++j) d.campos[j] = (float)(-(R[0][j] * T[0] + R[1][j] * T[1] + R[2][j] * T[2]));
    d.fx = cam->fx; d.fy = cam->fy; d.cx = cam->cx; d.cy = cam->cy;
    d.width = cam->width; d.height = cam->height;
    d.tiles_x = tiles_x; d.tiles_y = tiles_y;
    d.tile_base = 0; d.pix_base = 0;

    const int V = prims->kind;
    const long long records = prims->n;
    lp::PrimsDev P{prims->n, prims->centre, prims->verts, prims->opacity, prims->sh};
#define NA_CUDA(call)                          \
    do {                                       \
        if ((call) != cudaSuccess) {           \
            cudaGetLastError();                \
            return LP_ERR_CUDA;                \
        }                                      \
    } while (0)
    // the status word and the tile queue must start at zero
    NA_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), st));
    NA_CUDA(lp::launch_preprocess(V, prims->sh_degree, P, cp, rec, counts, trect, zbits, nullptr, st));
    NA_CUDA(lp::launch_scan(counts, records, offsets, scan_tmp, d_E, st));
    uint32_t E = 0;
    NA_CUDA(cudaMemcpyAsync(&E, d_E, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    if ((long long)E > kMaxEntries) return LP_ERR_CAPACITY;
    if (lp::emit_blocks(records, E) + 1 > (long long)(kPartBytes / 4)) return LP_ERR_CAPACITY;
    NA_CUDA(lp::launch_emit(counts, offsets, trect, zbits, records, d_E, E, part, keys0, vals0, kMaxEntries,
                            d_status, st));
    int passes = 0;
    int sms = 0;
    NA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    NA_CUDA(lp::launch_radix_sort(keys0, vals0, keys1, vals1, d_E, E, 32 + bits_for(tiles), 8, hist, scan_tmp,
                                  lp::SortCtl{sms, d_status, -1, false}, &passes, st));
    const bool in1 = (passes & 1) != 0;
    NA_CUDA(cudaMemsetAsync(ranges, 0, (size_t)tiles * sizeof(uint2), st));
    NA_CUDA(lp::launch_ranges(in1 ? keys1 : keys0, d_E, E, d_status, ranges, sms, st));
    lp::BlendArgs a{};
    const int pix = 4, batch = 64;
    int bps = lp::blend_fwd_occupancy(tile, V, batch, pix);
    if (bps <= 0) bps = 1;
    a.grid = (int)(tiles < (long long)sms * bps ? tiles : (long long)sms * bps);
    a.rec = rec;
    a.vals = in1 ? vals1 : vals0;
    a.ranges = ranges;
    a.cams = &cp;
    a.bg[0] = bg[0]; a.bg[1] = bg[1]; a.bg[2] = bg[2];
    a.image = image;
    a.last = last;
    a.tl = tl;
    a.tile_counter = d_tile_counter;
    a.pair_counts = d_pairs;
    a.count = false;
    NA_CUDA(cudaMemsetAsync(d_tile_counter, 0, sizeof(int), st));
    NA_CUDA(lp::launch_blend_fwd(tile, V, batch, pix, a, st));
    // the status the emission and range kernels latch on the device
    int status = 0;
    NA_CUDA(cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
#undef NA_CUDA
    if (status & lp::kStatusCapacity) return LP_ERR_CAPACITY;
    if (status & lp::kStatusTimeout) return LP_ERR_TIMEOUT;
    return LP_OK;
}
