// noalloc.cu -- csgv_encode_bricks_noalloc: the brick encoder without any
// device allocation, for callers that cannot call cudaMalloc.
//
// Who needs it: programs whose device memory is handed out by their own pool
// (a renderer or framework that reserves the GPU's memory up front, where a
// raw cudaMalloc fails or fragments the pool), and latency-sensitive loops
// that cannot afford cudaFree's implicit device-wide synchronisation.  The
// regular csgv_encode_bricks allocates per-brick scratch and the packed
// arrays on every call; this entry point instead works in one fixed scratch
// array that is part of the library image, and writes into output arrays the
// caller provides.
//
// The scratch is a file-scope __device__ array of kNoAllocScratchBytes
// (32 MiB), present on every GPU that loads the library until the process
// exits.  It holds the per-brick buffers of the encoder, so a call accepts at
// most a fixed number of bricks (b = 64: 11, b = 32: 99, b = 16: 790, b = 8: 6004,
// b = 4: 29025, b = 2: 52101) and rejects larger volumes with
// CSGV_ERR_INVALID_ARG.  Every call shares the array and it keeps the last
// call's contents: the counters that must start at zero are cleared at the
// start of each call, and two calls whose work overlaps on the GPU (different
// streams, or different host threads) race on it and must not be issued.
//
// Host code cannot use the array's name as a device address; its device
// address is looked up with cudaGetSymbolAddress once per device, on the
// first call made while that device is current, and cached.  That first call
// should therefore come before any stream capture on the calling thread.
#include <cstdio>
#include <mutex>

#include "encode_api.cuh"
#include "../../include/csgv.h"

namespace csgv {
void set_last_error(const char *msg);  // api.cu: message returned by csgv_last_error()
}

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;
constexpr size_t kAlign = 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_dev[kMaxDevices];
std::mutex g_scratch_mu;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// Byte layout of the scratch for C bricks: header (tables, totals, largest palette), then the
// per-brick areas of the encoder.  Returns the bytes used.
size_t carve(const csgv::EncGeom &G, size_t C, unsigned char *base, csgv::EncScratch *SC, uint32_t **freq,
             uint64_t **tot, uint32_t **maxpal) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
        unsigned char *p = base ? base + o : nullptr;
        o = align_up(o + bytes);
        return p;
    };
    unsigned char *f = take(32 * 4), *t = take(3 * 8), *m = take(3 * 4);
    unsigned char *sz = take(C * 8 * 4), *pal = take(C * G.pal_cap * 4);
    unsigned char *wi = take(C * (G.int_cap + 64) * 2), *wl = take(C * (G.leaf_cap + 64) * 2);
    unsigned char *op = take(C * G.ops_cap), *lv = take(C * G.lvl_bytes);
    if (base) {
        *freq = (uint32_t *)f;
        *tot = (uint64_t *)t;
        *maxpal = (uint32_t *)m;
        SC->sizes = (uint32_t *)sz;
        SC->pal = (uint32_t *)pal;
        SC->w_int = (uint16_t *)wi;
        SC->w_leaf = (uint16_t *)wl;
        SC->ops = op;
        SC->lvl = lv;
    }
    return o;
}

size_t max_bricks(const csgv::EncGeom &G) {
    size_t lo = 0, hi = 1;
    while (carve(G, hi, nullptr, nullptr, nullptr, nullptr, nullptr) <= kNoAllocScratchBytes) hi *= 2;
    while (hi - lo > 1) {
        const size_t mid = (lo + hi) / 2;
        if (carve(G, mid, nullptr, nullptr, nullptr, nullptr, nullptr) <= kNoAllocScratchBytes) lo = mid;
        else hi = mid;
    }
    return lo;
}

int err(int code, const char *msg) {
    csgv::set_last_error(msg);
    return code;
}

}  // namespace

extern "C" {

int csgv_encode_bricks_noalloc(const uint32_t *vol_dev, const uint64_t dims[3], uint32_t b,
                               const csgv_freq_table *table, const csgv_config *cfg, uint64_t *pal_off_dev,
                               uint32_t *pal_dev, uint64_t pal_capacity, uint64_t *int_off_dev,
                               uint16_t *int_words_dev, uint64_t int_capacity, uint64_t *leaf_off_dev,
                               uint16_t *leaf_words_dev, uint64_t leaf_capacity, uint32_t *n_int_sym_dev,
                               uint32_t *n_leaf_sym_dev, uint64_t totals[3], void *stream) {
    char msg[256];
    uint32_t N = 0;
    while (N <= (uint32_t)csgv::kMaxN && (1u << N) != b) N++;
    if (N < 1 || N > (uint32_t)csgv::kMaxN) return err(CSGV_ERR_INVALID_ARG, "brick size must be 2, 4, 8, 16, 32 or 64");
    if (!vol_dev || !dims || !table || !totals || !pal_off_dev || !pal_dev || !int_off_dev || !int_words_dev ||
        !leaf_off_dev || !leaf_words_dev || !n_int_sym_dev || !n_leaf_sym_dev)
        return err(CSGV_ERR_INVALID_ARG, "NULL argument");
    for (int t = 0; t < 2; t++) {
        uint32_t sum = 0;
        for (int s = 0; s < 16; s++) {
            if (table->freq[16 * t + s] == 0) return err(CSGV_ERR_INVALID_ARG, "frequency tables need f >= 1");
            sum += table->freq[16 * t + s];
        }
        if (sum != csgv::kM) return err(CSGV_ERR_INVALID_ARG, "frequency tables must sum to 4096");
    }
    const uint32_t K_max = cfg ? cfg->K_max : 32, S_min = cfg ? cfg->S_min : 256;
    if (K_max < 1 || K_max > 32 || S_min < 1) return err(CSGV_ERR_INVALID_ARG, "K_max must be 1..32, S_min >= 1");
    csgv::EncVol EV;
    EV.vol = vol_dev;
    const csgv::EncGeom G = csgv::make_geom(N, K_max, S_min);
    const size_t cmax = max_bricks(G);
    uint64_t n = 1;
    bool wrapped = false;
    for (int a = 0; a < 3; a++) {
        if (dims[a] == 0 || dims[a] > (1ull << 31)) return err(CSGV_ERR_INVALID_ARG, "bad dimension");
        EV.dims[a] = dims[a];
        EV.nb[a] = (dims[a] + b - 1) / b;
        wrapped |= __builtin_mul_overflow(n, EV.nb[a], &n);  // up to 2^90 bricks: must not wrap to a small n
    }
    if (wrapped) {
        snprintf(msg, sizeof msg,
                 "volume has %llu x %llu x %llu bricks of %u^3; the allocation-free encoder's %zu MiB scratch holds "
                 "at most %zu", (unsigned long long)EV.nb[0], (unsigned long long)EV.nb[1],
                 (unsigned long long)EV.nb[2], b, kNoAllocScratchBytes >> 20, cmax);
        return err(CSGV_ERR_INVALID_ARG, msg);
    }
    if (n > cmax) {
        snprintf(msg, sizeof msg,
                 "volume has %llu bricks of %u^3; the allocation-free encoder's %zu MiB scratch holds at most %zu",
                 (unsigned long long)n, b, kNoAllocScratchBytes >> 20, cmax);
        return err(CSGV_ERR_INVALID_ARG, msg);
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return err(CSGV_ERR_CUDA, "no current CUDA device");
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_dev[dev]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                snprintf(msg, sizeof msg, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
                return err(CSGV_ERR_CUDA, msg);
            }
            g_scratch_dev[dev] = p;
        }
        base = g_scratch_dev[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    csgv::EncScratch SC{};
    uint32_t *freq_d = nullptr, *maxpal_d = nullptr;
    uint64_t *tot_d = nullptr;
    carve(G, n, (unsigned char *)base, &SC, &freq_d, &tot_d, &maxpal_d);
    cudaError_t e = cudaMemcpyAsync(freq_d, table->freq, 32 * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(tot_d, 0, 3 * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(maxpal_d, 0, 3 * 4, st);
    if (e == cudaSuccess) e = csgv::launch_encode(EV, G, 0, 1, (uint32_t)n, freq_d, SC, nullptr, st);
    if (e == cudaSuccess)
        e = csgv::launch_scan(SC.sizes, (uint32_t)n, 0, pal_off_dev, int_off_dev, leaf_off_dev, tot_d, maxpal_d, nullptr,
                              st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(totals, tot_d, 3 * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "encode: %s", cudaGetErrorString(e));
        return err(CSGV_ERR_CUDA, msg);
    }
    if (totals[0] > pal_capacity || totals[1] > int_capacity || totals[2] > leaf_capacity) {
        snprintf(msg, sizeof msg,
                 "output arrays too small: need %llu palette labels, %llu interior and %llu leaf words",
                 (unsigned long long)totals[0], (unsigned long long)totals[1], (unsigned long long)totals[2]);
        return err(CSGV_ERR_INVALID_ARG, msg);
    }
    e = csgv::launch_compact(G, SC, 0, (uint32_t)n, pal_off_dev, int_off_dev, leaf_off_dev, pal_dev, int_words_dev,
                             leaf_words_dev, n_int_sym_dev, n_leaf_sym_dev, st);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "compact: %s", cudaGetErrorString(e));
        return err(CSGV_ERR_CUDA, msg);
    }
    return CSGV_OK;
}

}  // extern "C"
