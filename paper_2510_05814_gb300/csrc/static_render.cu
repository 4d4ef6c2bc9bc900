// smoe_render_static: bin and render one model without any device
// allocation, for callers that cannot call cudaMalloc (for example a plugin
// that lives inside a host application which owns every device allocation,
// or code running where the allocator must not be touched).  The caller
// passes the parameters and the output image; every intermediate buffer
// (prepared kernel records, tile rectangles, per-tile counters, the prefix
// sums and the (tile, kernel) lists) lives in one file-scope device array of
// fixed size that every GPU loading this library holds until the process
// exits.
#include <mutex>

#include "smoe_internal.cuh"

namespace {

using namespace smoe;

// Limits of the static scratch.
constexpr int64_t kStaticMaxK = 32768;          // kernels
constexpr int64_t kStaticMaxTiles = 16384;      // tiles of the output raster
constexpr int64_t kStaticMaxPairs = 524288;     // (tile, kernel) pairs
constexpr size_t kScratchBytes = 8u << 20;

constexpr size_t up(size_t x) { return (x + 255) & ~size_t(255); }
// Region offsets inside the scratch (records sized for the widest record,
// 16 floats: RGB with linear experts).
constexpr size_t kRec = 0;
constexpr size_t kRect = kRec + up(sizeof(float) * 16 * kStaticMaxK);
constexpr size_t kTileCnt = kRect + up(sizeof(int4) * kStaticMaxK);
constexpr size_t kCursor = kTileCnt + up(sizeof(int32_t) * kStaticMaxTiles);
constexpr size_t kLongQ = kCursor + up(sizeof(int32_t) * kStaticMaxTiles);
constexpr size_t kNLong = kLongQ + up(sizeof(int32_t) * kStaticMaxTiles);
constexpr size_t kBsum = kNLong + up(sizeof(int32_t));
constexpr size_t kTileOff = kBsum + up(sizeof(long long) * ((kStaticMaxTiles + 4095) / 4096));
constexpr size_t kNPairs = kTileOff + up(sizeof(int32_t) * (kStaticMaxTiles + 1));
constexpr size_t kPairTmp = kNPairs + up(sizeof(int64_t));
constexpr size_t kPairK = kPairTmp + up(sizeof(int32_t) * kStaticMaxPairs);
constexpr size_t kEnd = kPairK + up(sizeof(int32_t) * kStaticMaxPairs);
static_assert(kEnd <= kScratchBytes, "static scratch layout exceeds its size");

// The scratch.  In host code this name is only a stand-in for the device
// symbol: its device address comes from cudaGetSymbolAddress below.
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch per device.  Outside stream capture it is
// looked up again on every call (a cheap driver query), so a context that
// was torn down and re-created (for example after cudaDeviceReset) cannot
// leave a stale address behind; a call under capture uses the address of the
// last call outside capture on that device.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

smoe_status scratch_address(cudaStream_t st, void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return SMOE_ERR_CUDA;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return SMOE_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (cap == cudaStreamCaptureStatusNone || !g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return SMOE_ERR_CUDA;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return SMOE_OK;
}

}  // namespace

extern "C" SMOE_API smoe_status smoe_render_static(const smoe_desc *d, const smoe_params *p,
                                                   float *y, float *inv_d, int32_t *status,
                                                   void *stream) {
    // The same raster checks as every other entry point (including the
    // largest cutoff, beyond which an included pair's gate would flush to 0).
    if (!desc_valid(d) || !p || !y || !status) return SMOE_ERR_ARG;
    if (p->K < 0 || (p->K > 0 && (!p->mu || !p->chol || !p->ea)) ||
        ((p->eW != nullptr) != (d->expert == 1) && p->K > 0))
        return SMOE_ERR_ARG;
    const int tiles_x = (d->W + d->tile - 1) / d->tile;
    const int tiles_y = (d->H + d->tile - 1) / d->tile;
    const int64_t tiles = (int64_t)tiles_x * tiles_y;
    // Beyond the static scratch: refuse (the caller needs smoe_bin + smoe_render).
    if (p->K > kStaticMaxK || tiles > kStaticMaxTiles) return SMOE_ERR_WORKSPACE;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *base = nullptr;
    smoe_status s = scratch_address(st, &base);
    if (s != SMOE_OK) return s;
    char *b = static_cast<char *>(base);

    Geo g{};
    g.C = d->C;
    g.T = d->tile;
    g.linear = d->expert;
    g.S = rec_stride(d->C, d->expert);
    g.GS = acc_stride(d->C, d->expert);
    g.rbf = d->gate;
    g.qmax = d->qmax;
    g.scale = d->scale;
    g.B = 1;
    g.K_total = p->K;
    g.tiles_total = tiles;
    g.one.W = d->W;
    g.one.H = d->H;
    g.one.tiles_x = tiles_x;
    g.one.tiles_y = tiles_y;
    g.one.K = p->K;
    g.one.iters = 1;
    g.one.p = *p;

    Bufs w{};
    w.rec = reinterpret_cast<float *>(b + kRec);
    w.rect = reinterpret_cast<int4 *>(b + kRect);
    w.tile_cnt = reinterpret_cast<int32_t *>(b + kTileCnt);
    w.cursor = reinterpret_cast<int32_t *>(b + kCursor);
    w.long_q = reinterpret_cast<int32_t *>(b + kLongQ);
    w.n_long = reinterpret_cast<int32_t *>(b + kNLong);
    w.bsum = reinterpret_cast<long long *>(b + kBsum);
    w.tile_off = reinterpret_cast<int32_t *>(b + kTileOff);
    w.n_pairs = reinterpret_cast<int64_t *>(b + kNPairs);
    w.pair_tmp = reinterpret_cast<int32_t *>(b + kPairTmp);
    w.pair_k = reinterpret_cast<int32_t *>(b + kPairK);
    w.acc = nullptr;
    w.pair_cap = kStaticMaxPairs;
    w.status = status;

    // The previous call's contents are stale: the status starts at 0, the
    // per-tile counters are zeroed by the binning sequence itself (as are the
    // scatter cursors and the long-list queue counter); every other region
    // is fully written before it is read.
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t), st);
    if (e == cudaSuccess) e = launch_bin(g, w, st);
    if (e == cudaSuccess) e = launch_render(g, w, y, inv_d, st);
    return e == cudaSuccess ? SMOE_OK : SMOE_ERR_CUDA;
}
