// api.cu -- C ABI of libcsgv (declared in include/csgv.h): argument checks,
// device allocations owned by volume handles, and kernel launches.
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>
#include <atomic>
#include <mutex>

#include "csgv_internal.cuh"
#include "../../include/csgv.h"

// kernels' launchers (decode.cu, encode.cu)
namespace csgv {
cudaError_t launch_decode_slice(const VolDev &V, uint32_t max_pal, const RecJob &J, uint32_t *out, const uint64_t *out_off,
                                int32_t *status, const DecodeShape &S, cudaStream_t st);
}  // namespace csgv

#include "encode_api.cuh"

struct csgv_volume {
    uint32_t N;
    uint64_t dims[3], grid[3], n_bricks;
    uint32_t K_max, S_min, max_palette;
    uint32_t freq[32];
    uint64_t n_pal, n_iw, n_lw;
    uint64_t *pal_off, *int_off, *leaf_off;
    uint32_t *pal;
    uint16_t *int_words, *leaf_words;
    uint32_t *n_int_sym, *n_leaf_sym;
    uint32_t *lut;
    uint32_t max_int_sym, max_leaf_sym;  // largest per-brick symbol counts: size the decode workspace
    uint16_t *leaf_host = nullptr;        // leaf words in mapped host memory (csgv_volume_leaves_to_host)
    uint64_t dec_ws_bytes = 192ull << 20;  // decode configuration (csgv_decode_autotune)
    csgv::DecodeShape dec_shape;
    cudaEvent_t ready = nullptr;  // recorded when the arrays are complete on the stream that made them
};

namespace {

// word arrays carry this many spare 16-bit words at the end: the decoder stages stream words with
// 16-byte loads aligned down from the stream start, which may touch up to 15 bytes past the last word
constexpr uint64_t kWordPad = 16;
thread_local std::string g_err;

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(CSGV_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

// Per-device stream-ordered pool for volume arrays and decode workspaces; it keeps up to kPoolKeep bytes
// between calls.  Concurrent calls on different streams get their own allocations.
constexpr uint64_t kPoolKeep = 1ull << 30;
constexpr int kPoolDevices = 64;
cudaMemPool_t g_pools[kPoolDevices];
std::mutex g_pool_mu;

int dev_pool(cudaMemPool_t *pool) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kPoolDevices) return fail(CSGV_ERR_INVALID_ARG, "device index %d too large", dev);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps p;
        memset(&p, 0, sizeof p);
        p.allocType = cudaMemAllocationTypePinned;
        p.location.type = cudaMemLocationTypeDevice;
        p.location.id = dev;
        cudaMemPool_t mp;
        CK(cudaMemPoolCreate(&mp, &p));
        uint64_t keep = kPoolKeep;
        CK(cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep));
        g_pools[dev] = mp;
    }
    *pool = g_pools[dev];
    return CSGV_OK;
}

bool pow2_brick(uint32_t b, uint32_t &N) {
    for (N = 1; N <= (uint32_t)csgv::kMaxN; N++)
        if ((1u << N) == b) return true;
    return false;
}

bool valid_table(const uint32_t *f) {
    for (int t = 0; t < 2; t++) {
        uint32_t sum = 0;
        for (int s = 0; s < 16; s++) {
            if (f[16 * t + s] == 0 || f[16 * t + s] > csgv::kM) return false;
            sum += f[16 * t + s];
        }
        if (sum != csgv::kM) return false;
    }
    return true;
}

// Volume arrays come from a per-device stream-ordered pool (see dev_pool), so encoding a volume costs no
// device-wide synchronisation; they are returned when the volume is destroyed.
cudaError_t vol_free_arrays(csgv_volume *v, cudaStream_t st = 0) {
    if (v->ready) cudaEventDestroy(v->ready);
    v->ready = nullptr;
    void *arr[] = {v->pal_off, v->int_off, v->leaf_off, v->pal,       v->int_words,
                   v->leaf_host ? nullptr : v->leaf_words, v->n_int_sym, v->n_leaf_sym, v->lut};
    cudaError_t err = cudaSuccess;
    for (void *a : arr)
        if (a) {
            const cudaError_t e = cudaFreeAsync(a, st);
            if (e != cudaSuccess && err == cudaSuccess) err = e;
        }
    if (v->leaf_host) cudaFreeHost(v->leaf_host);
    v->leaf_host = nullptr;
    return err;
}

// decode table (2 x 4096 packed entries) from the frequencies (freq_dev when given, else t), on the device
__global__ void build_lut_kernel(csgv_freq_table t, const uint32_t *freq_dev, uint32_t *lut) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * csgv::kM) return;
    const uint32_t tb = i / csgv::kM, slot = i % csgv::kM;
    const uint32_t *f = (freq_dev ? freq_dev : t.freq) + 16 * tb;
    uint32_t cum = 0, s = 0;
    while (s < 15 && cum + f[s] <= slot) cum += f[s++];
    lut[i] = csgv::lut_pack(s, f[s], slot - cum);
}

// Both tables from the nibble counts on the device, one warp: lane 16t + s holds symbol s of table t.  Same
// result as normalise_table: f = 1 + floor(c (M - 16) / total), and the r leftover units go to the symbols of
// rank < r, rank = the number of symbols with a larger count or an equal count and a lower index (the order
// in which normalise_table hands them out).
__global__ void __launch_bounds__(32) freq_from_counts_kernel(const unsigned long long *cnt, uint32_t *freq) {
    const uint32_t lane = threadIdx.x, s = lane & 15;
    const unsigned long long c = cnt[lane];
    unsigned long long total = c;
    for (int d = 1; d < 16; d <<= 1) total += __shfl_xor_sync(csgv::kFull, total, d);
    const unsigned long long lim = ~0ull / (csgv::kM - 16);
    unsigned long long q = 0;
    if (total != 0)
        q = c <= lim ? c * (csgv::kM - 16) / total
                     : (unsigned long long)((unsigned __int128)c * (csgv::kM - 16) / total);
    uint32_t f = 1u + (uint32_t)q;
    uint32_t sum = f;
    for (int d = 1; d < 16; d <<= 1) sum += __shfl_xor_sync(csgv::kFull, sum, d);
    uint32_t rank = 0;
    for (uint32_t o = 0; o < 16; o++) {
        const unsigned long long co = __shfl_sync(csgv::kFull, c, (lane & 16u) | o);
        rank += (co > c || (co == c && o < s)) ? 1u : 0u;
    }
    f += rank < csgv::kM - sum ? 1u : 0u;
    freq[lane] = total == 0 ? csgv::kM / 16 : f;
}

// allocate and fill the volume's decode table on `st` from v->freq, or from freq_dev (device) when given
int vol_lut(csgv_volume *v, const uint32_t *freq_dev, cudaStream_t st) {
    cudaMemPool_t pool;
    int rc = dev_pool(&pool);
    if (rc) return rc;
    CK(cudaMallocFromPoolAsync((void **)&v->lut, 2 * csgv::kM * 4, pool, st));
    csgv_freq_table t;
    memcpy(t.freq, v->freq, sizeof t.freq);
    {
        csgv::ProfScope ps("build_lut", st);
        build_lut_kernel<<<2 * csgv::kM / 256, 256, 0, st>>>(t, freq_dev, v->lut);
    }
    CK(cudaGetLastError());
    return CSGV_OK;
}

// mark the volume complete in the order of `st`: calls on other streams wait for this event
int vol_ready(csgv_volume *v, cudaStream_t st) {
    if (!v->ready) CK(cudaEventCreateWithFlags(&v->ready, cudaEventDisableTiming));
    CK(cudaEventRecord(v->ready, st));
    return CSGV_OK;
}

csgv::VolDev dev_view(const csgv_volume *v) {
    csgv::VolDev V;
    V.pal_off = v->pal_off; V.int_off = v->int_off; V.leaf_off = v->leaf_off;
    V.pal = v->pal; V.int_words = v->int_words; V.leaf_words = v->leaf_words;
    V.n_int_sym = v->n_int_sym; V.n_leaf_sym = v->n_leaf_sym;
    V.lut = v->lut;
    V.n_bricks = v->n_bricks;
    V.N = v->N; V.K_max = v->K_max; V.S_min = v->S_min;
    return V;
}


int check_dims(const uint64_t dims[3], uint32_t b, uint32_t &N) {
    if (!dims) return fail(CSGV_ERR_INVALID_ARG, "dims is NULL");
    if (!pow2_brick(b, N)) return fail(CSGV_ERR_INVALID_ARG, "brick size %u is not a power of two in [2, 64]", b);
    for (int a = 0; a < 3; a++)
        if (dims[a] == 0 || dims[a] > (1ull << 31)) return fail(CSGV_ERR_INVALID_ARG, "bad dimension %d", a);
    return CSGV_OK;
}

// Encoder scratch, kept per device between calls so that encoding does not allocate and free
// gigabytes (cudaFree synchronises the whole device) on every call.  Guarded by g_arena_mu for the
// whole encode call; the next call's stream waits for g_arena_done (the previous call's last kernel
// on the arena) before it writes the arena again.
constexpr int kArenaDevices = 64;
struct Arena {
    void *p = nullptr;
    size_t bytes = 0;
};
Arena g_arena[kArenaDevices];
std::mutex g_arena_mu;
cudaEvent_t g_arena_done[kArenaDevices];  // recorded after the last kernel of an encode that read the arena
void *g_readback[kArenaDevices];          // pinned host copy of an encode's per-batch results
cudaEvent_t g_readback_done[kArenaDevices];  // recorded after the copy into g_readback

cudaError_t arena_get(int dev, size_t bytes, void **out) {
    Arena &A = g_arena[dev];
    if (A.bytes < bytes) {
        if (A.p) cudaFree(A.p);
        A.p = nullptr;
        A.bytes = 0;
        cudaError_t e = cudaMalloc(&A.p, bytes);
        if (e != cudaSuccess) return e;
        A.bytes = bytes;
    }
    *out = A.p;
    return cudaSuccess;
}

int grow(void **p, uint64_t &cap, uint64_t need, size_t elem, uint64_t used, cudaStream_t st, bool exact) {
    if (need <= cap) return CSGV_OK;
    uint64_t nc = cap ? cap : 1024;
    while (nc < need) nc = nc + nc / 2 + 1024;
    if (exact) nc = need;
    cudaMemPool_t pool;
    int rc = dev_pool(&pool);
    if (rc) return rc;
    void *q = nullptr;
    CK(cudaMallocFromPoolAsync(&q, nc * elem, pool, st));
    if (*p && used) CK(cudaMemcpyAsync(q, *p, used * elem, cudaMemcpyDeviceToDevice, st));
    if (*p) CK(cudaFreeAsync(*p, st));
    *p = q;
    cap = nc;
    return CSGV_OK;
}

}  // namespace

namespace csgv {
// lets other translation units of the library report a message through csgv_last_error()
void set_last_error(const char *msg) { g_err = msg; }
// a volume's device arrays, its completion event and its grid, for the other translation units
VolDev volume_view(const csgv_volume *v) { return dev_view(v); }
cudaEvent_t volume_ready(const csgv_volume *v) { return v->ready; }
void volume_grid(const csgv_volume *v, uint64_t dims[3], uint64_t grid[3]) {
    for (int a = 0; a < 3; a++) {
        dims[a] = v->dims[a];
        grid[a] = v->grid[a];
    }
}
}  // namespace csgv

namespace csgv {
namespace {
std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
struct ProfRec {
    const char *name;
    cudaEvent_t e0, e1;
    int dev;  // device the events belong to
};
std::vector<ProfRec> g_prof;
std::vector<std::pair<int, cudaEvent_t>> g_prof_free;  // (device, event) ready for reuse
}  // namespace
bool prof_on() { return g_prof_on.load(std::memory_order_relaxed); }
cudaEvent_t prof_event() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        for (size_t i = g_prof_free.size(); i-- > 0;)
            if (g_prof_free[i].first == dev) {
                cudaEvent_t e = g_prof_free[i].second;
                g_prof_free[i] = g_prof_free.back();
                g_prof_free.pop_back();
                return e;
            }
    }
    cudaEvent_t e = nullptr;
    return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
}
void prof_record(const char *name, cudaEvent_t e0, cudaEvent_t e1) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.push_back({name, e0, e1, dev});
}
}  // namespace csgv

extern "C" {

const char *csgv_last_error(void) { return g_err.c_str(); }

int csgv_freq_table_from_counts(const uint64_t counts[32], csgv_freq_table *out) {
    if (!counts || !out) return fail(CSGV_ERR_INVALID_ARG, "NULL argument");
    unsigned long long c[32];
    memcpy(c, counts, sizeof c);  // counts may alias out->counts
    for (int t = 0; t < 2; t++) csgv::normalise_table(c + 16 * t, out->freq + 16 * t);
    memcpy(out->counts, c, sizeof c);
    return CSGV_OK;
}

int csgv_build_freq_table(const uint32_t *vol_dev, const uint64_t dims[3], uint32_t b, uint32_t sample_stride,
                          csgv_freq_table *out, void *stream) {
    uint32_t N;
    int rc = check_dims(dims, b, N);
    if (rc) return rc;
    if (!vol_dev || !out) return fail(CSGV_ERR_INVALID_ARG, "NULL volume or output");
    if (sample_stride == 0) return fail(CSGV_ERR_INVALID_ARG, "sample_stride must be >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    csgv::EncVol EV;
    EV.vol = vol_dev;
    uint64_t n = 1;
    for (int a = 0; a < 3; a++) {
        EV.dims[a] = dims[a];
        EV.nb[a] = (dims[a] + b - 1) / b;
        n *= EV.nb[a];
    }
    const uint64_t n_sampled = (n + sample_stride - 1) / sample_stride;
    csgv::EncGeom G = csgv::make_geom(N, 32, 256);
    unsigned long long *cnt = nullptr;
    cudaMemPool_t pool;
    rc = dev_pool(&pool);
    if (rc) return rc;
    CK(cudaMallocFromPoolAsync((void **)&cnt, 32 * 8, pool, st));
    CK(cudaMemsetAsync(cnt, 0, 32 * 8, st));
    csgv::EncScratch SC{};
    // sampled bricks per count-mode launch (op scratch, and for b = 64 the level arrays, per brick)
    const uint64_t per_batch = std::min<uint64_t>(4096, ((uint64_t)1 << 31) / (G.ops_cap + G.lvl_bytes));
    const uint64_t nb = std::min<uint64_t>(per_batch, n_sampled);
    CK(cudaMallocFromPoolAsync((void **)&SC.ops, nb * G.ops_cap, pool, st));
    if (G.lvl_bytes) CK(cudaMallocFromPoolAsync((void **)&SC.lvl, nb * G.lvl_bytes, pool, st));
    for (uint64_t first = 0; first < n_sampled; first += per_batch) {
        const uint32_t m = (uint32_t)std::min<uint64_t>(per_batch, n_sampled - first);
        cudaError_t e = csgv::launch_encode(EV, G, first * sample_stride, sample_stride, m, nullptr, SC, cnt, st);
        if (e != cudaSuccess) {
            cudaFreeAsync(SC.ops, st);
            if (SC.lvl) cudaFreeAsync(SC.lvl, st);
            cudaFreeAsync(cnt, st);
            return cuda_fail(e, "encode (count mode)");
        }
    }
    cudaFreeAsync(SC.ops, st);
    if (SC.lvl) cudaFreeAsync(SC.lvl, st);
    cudaError_t e = cudaMemcpyAsync(out->counts, cnt, 32 * 8, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(cnt, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "frequency prepass");
    return csgv_freq_table_from_counts(out->counts, out);
}

// What the host reads back after each encode batch, in one copy: running totals, prepass counts, maxima,
// tables.  Lives in the arena (device) and in pinned memory (host).
struct Readback {
    unsigned long long tot[3], cnt[32];
    uint32_t maxes[4], freq[32];
    unsigned long long scan[csgv::kScanScratchBytes / 8];  // the size scan's block totals (device only)
};

// A volume being encoded: its bricks are appended batch by batch (one call, or a stream encoder across calls).
struct EncRun {
    csgv_volume *v = nullptr;
    csgv::EncGeom G{};
    uint64_t cap_p = 0, cap_i = 0, cap_l = 0;  // allocated palette labels / interior words / leaf words
    uint64_t tot[3] = {0, 0, 0};               // used so far
    uint32_t maxes[3] = {0, 0, 0};             // largest palette, interior and leaf symbol counts so far
};

// bricks per encode batch: the scratch of a batch takes at most a quarter of free memory (6 GB at most)
static uint64_t enc_batch_bricks(const csgv::EncGeom &G, uint64_t n) {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const size_t budget = std::min<size_t>(free_b / 4, (size_t)6 << 30);
    const uint64_t C = std::max<uint64_t>(1, std::min<uint64_t>(n, budget / csgv::scratch_bytes_per_brick(G)));
    return std::min<uint64_t>(C, 65535);
}

// the per-brick index arrays of a volume (offsets, symbol counts), from the pool
static int vol_alloc_index(csgv_volume *v, cudaStream_t st) {
    cudaMemPool_t pool;
    int rc = dev_pool(&pool);
    if (rc) return rc;
    const uint64_t n = v->n_bricks;
    CK(cudaMallocFromPoolAsync((void **)&v->pal_off, (n + 1) * 8, pool, st));
    CK(cudaMallocFromPoolAsync((void **)&v->int_off, (n + 1) * 8, pool, st));
    CK(cudaMallocFromPoolAsync((void **)&v->leaf_off, (n + 1) * 8, pool, st));
    CK(cudaMallocFromPoolAsync((void **)&v->n_int_sym, n * 4, pool, st));
    CK(cudaMallocFromPoolAsync((void **)&v->n_leaf_sym, n * 4, pool, st));
    return CSGV_OK;
}

// Encode bricks ev_first .. ev_first + m - 1 of EV (brick ids of EV's grid) as the volume's bricks glob_first ..,
// in batches of C.  table: the tables; NULL: tables normalised on the device from the nibbles of every
// sample_stride-th brick of this run (a single batch; they are returned in *made and set in the volume).
// build_lut: build the volume's decode table once the tables are final.  Synchronises st once per batch.
static int encode_run(EncRun &R, const csgv::EncVol &EV, uint64_t ev_first, uint64_t glob_first, uint64_t m,
                      uint64_t C, const csgv_freq_table *table, uint32_t sample_stride, csgv_freq_table *made,
                      bool build_lut, cudaStream_t st) {
    csgv_volume *v = R.v;
    const csgv::EncGeom &G = R.G;
    int rc = CSGV_OK, dev = -1;
    auto bail = [&](int code) {
        // kernels already queued may still use the arena: the next encode waits for them
        if (dev >= 0 && g_arena_done[dev]) cudaEventRecord(g_arena_done[dev], st);
        return code;
    };
#define CKE(call)                                          \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return bail(cuda_fail(e_, #call)); \
    } while (0)
    std::lock_guard<std::mutex> arena_lock(g_arena_mu);
    int d_ = 0;
    CKE(cudaGetDevice(&d_));
    if (d_ < 0 || d_ >= kArenaDevices) return fail(CSGV_ERR_INVALID_ARG, "device index %d too large", d_);
    dev = d_;
    // carve the batch scratch out of the arena (256-byte aligned pieces)
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_pal = take(C * G.pal_cap * 4);
    const size_t o_wi = take(C * (G.int_cap + 64) * 2), o_wl = take(C * (G.leaf_cap + 64) * 2);
    const size_t o_sz = take(C * 8 * 4), o_rb = take(sizeof(Readback)), o_ops = take(C * G.ops_cap);
    const size_t o_lvl = take(C * G.lvl_bytes);
    void *arena = nullptr;
    CKE(arena_get(dev, off, &arena));
    unsigned char *A = (unsigned char *)arena;
    csgv::EncScratch SC{};
    SC.pal = (uint32_t *)(A + o_pal);
    SC.w_int = (uint16_t *)(A + o_wi);
    SC.w_leaf = (uint16_t *)(A + o_wl);
    SC.sizes = (uint32_t *)(A + o_sz);
    SC.ops = A + o_ops;
    SC.lvl = A + o_lvl;
    Readback *rb_d = (Readback *)(A + o_rb);
    if (!g_readback[dev]) CKE(cudaMallocHost(&g_readback[dev], sizeof(Readback)));
    if (!g_readback_done[dev]) CKE(cudaEventCreateWithFlags(&g_readback_done[dev], cudaEventDisableTiming));
    Readback &rb = *(Readback *)g_readback[dev];
    if (g_arena_done[dev]) CKE(cudaStreamWaitEvent(st, g_arena_done[dev], 0));  // the previous encode is done with it
    else CKE(cudaEventCreateWithFlags(&g_arena_done[dev], cudaEventDisableTiming));
    memset(&rb, 0, sizeof rb);
    for (int a = 0; a < 3; a++) rb.tot[a] = R.tot[a];  // the scan continues from the running totals
    if (table) memcpy(rb.freq, table->freq, sizeof rb.freq);
    CKE(cudaMemcpyAsync(rb_d, &rb, sizeof rb, cudaMemcpyHostToDevice, st));
    for (uint64_t j = 0; j < m; j += C) {
        const uint32_t mm = (uint32_t)std::min<uint64_t>(C, m - j);
        const uint64_t gfirst = glob_first + j;
        if (table) {
            CKE(csgv::launch_encode(EV, G, ev_first + j, 1, mm, rb_d->freq, SC, nullptr, st));
        } else {
            // op streams first (they do not depend on the tables), then the prepass counts from them, the
            // tables from the counts, and the entropy coding, all on the device
            CKE(csgv::launch_encode(EV, G, ev_first + j, 1, mm, nullptr, SC, nullptr, st));
            CKE(csgv::launch_nibble_hist(G, SC, mm, sample_stride, rb_d->cnt, st));
            {
                csgv::ProfScope ps("freq_tables", st);
                freq_from_counts_kernel<<<1, 32, 0, st>>>(rb_d->cnt, rb_d->freq);
            }
            CKE(cudaGetLastError());
            CKE(csgv::launch_rans_encode(G, SC, mm, rb_d->freq, st));
        }
        CKE(csgv::launch_scan(SC.sizes, mm, gfirst, v->pal_off, v->int_off, v->leaf_off, (uint64_t *)rb_d->tot,
                              rb_d->maxes, rb_d->scan, st));
        const bool final_batch = j + mm >= m;
        const uint64_t prev[3] = {R.tot[0], R.tot[1], R.tot[2]};
        CKE(cudaMemcpyAsync(&rb, rb_d, sizeof rb, cudaMemcpyDeviceToHost, st));
        CKE(cudaEventRecord(g_readback_done[dev], st));
        // the decode table is built while the host reads the totals back (the tables are final)
        if (build_lut && final_batch && (rc = vol_lut(v, rb_d->freq, st))) return bail(rc);
        CKE(cudaEventSynchronize(g_readback_done[dev]));
        for (int a = 0; a < 3; a++) {
            R.tot[a] = rb.tot[a];
            R.maxes[a] = std::max(R.maxes[a], rb.maxes[a]);
        }
        if (!table) {  // the sampled tables (one batch only)
            memcpy(made->counts, rb.cnt, sizeof made->counts);
            memcpy(made->freq, rb.freq, sizeof made->freq);
            memcpy(v->freq, made->freq, sizeof v->freq);
        }
        // the whole volume in one batch: arrays sized exactly; otherwise grown geometrically
        const bool exact = gfirst == 0 && mm == v->n_bricks;
        int g;
        if ((g = grow((void **)&v->pal, R.cap_p, std::max<uint64_t>(R.tot[0], 1), 4, prev[0], st, exact)) ||
            (g = grow((void **)&v->int_words, R.cap_i, R.tot[1] + kWordPad, 2, prev[1], st, exact)) ||
            (g = grow((void **)&v->leaf_words, R.cap_l, R.tot[2] + kWordPad, 2, prev[2], st, exact)))
            return bail(g);
        CKE(csgv::launch_compact(G, SC, gfirst, mm, v->pal_off, v->int_off, v->leaf_off, v->pal, v->int_words,
                                 v->leaf_words, v->n_int_sym, v->n_leaf_sym, st));
    }
    CKE(cudaEventRecord(g_arena_done[dev], st));
#undef CKE
    return CSGV_OK;
}

// the volume's totals and maxima from a finished run
static void run_finish(EncRun &R) {
    csgv_volume *v = R.v;
    v->max_palette = R.maxes[0];
    v->max_int_sym = R.maxes[1];
    v->max_leaf_sym = R.maxes[2];
    v->n_pal = R.tot[0];
    v->n_iw = R.tot[1];
    v->n_lw = R.tot[2];
}

// Encode with the given tables, or (table == NULL) with tables normalised from the nibble counts of every
// sample_stride-th brick of this encode (written to *table_out when given).
static int encode_impl(const uint32_t *vol_dev, const uint64_t dims[3], uint32_t b, const csgv_freq_table *table,
                       uint32_t sample_stride, const csgv_config *cfg, csgv_freq_table *table_out,
                       csgv_volume **out, void *stream) {
    uint32_t N;
    int rc = check_dims(dims, b, N);
    if (rc) return rc;
    if (!vol_dev || !out) return fail(CSGV_ERR_INVALID_ARG, "NULL argument");
    if (table && !valid_table(table->freq)) return fail(CSGV_ERR_INVALID_ARG, "frequency tables must sum to 4096 with f >= 1");
    if (!table && sample_stride == 0) return fail(CSGV_ERR_INVALID_ARG, "sample_stride must be >= 1");
    const uint32_t K_max = cfg ? cfg->K_max : 32, S_min = cfg ? cfg->S_min : 256;
    if (K_max < 1 || K_max > 32 || S_min < 1) return fail(CSGV_ERR_INVALID_ARG, "K_max must be 1..32, S_min >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    *out = nullptr;

    csgv_volume *v = new csgv_volume();
    v->N = N;
    v->K_max = K_max;
    v->S_min = S_min;
    csgv::EncVol EV;
    EV.vol = vol_dev;
    v->n_bricks = 1;
    for (int a = 0; a < 3; a++) {
        v->dims[a] = dims[a];
        v->grid[a] = EV.nb[a] = (dims[a] + b - 1) / b;
        EV.dims[a] = dims[a];
        v->n_bricks *= v->grid[a];
    }
    const uint64_t n = v->n_bricks;
    EncRun R;
    R.v = v;
    R.G = csgv::make_geom(N, K_max, S_min);
    const uint64_t C = enc_batch_bricks(R.G, n);
    csgv_freq_table made;
    if (!table && C < n) {  // more than one batch: the tables are needed before the first one is coded
        delete v;
        rc = csgv_build_freq_table(vol_dev, dims, b, sample_stride, &made, stream);
        if (rc) return rc;
        if (table_out) *table_out = made;
        return encode_impl(vol_dev, dims, b, &made, 1, cfg, nullptr, out, stream);
    }
    if (table) memcpy(v->freq, table->freq, sizeof v->freq);
    rc = vol_alloc_index(v, st);
    if (!rc) rc = encode_run(R, EV, 0, 0, n, C, table, sample_stride, &made, true, st);
    if (!rc) {
        run_finish(R);
        if (!table && table_out) *table_out = made;
        rc = vol_ready(v, st);
    }
    if (rc) {
        vol_free_arrays(v);
        delete v;
        return rc;
    }
    *out = v;
    return CSGV_OK;
}

int csgv_encode_bricks(const uint32_t *vol_dev, const uint64_t dims[3], uint32_t b, const csgv_freq_table *table,
                       const csgv_config *cfg, csgv_volume **out, void *stream) {
    if (!table) return fail(CSGV_ERR_INVALID_ARG, "NULL argument");
    return encode_impl(vol_dev, dims, b, table, 1, cfg, nullptr, out, stream);
}

int csgv_encode_bricks_sampled(const uint32_t *vol_dev, const uint64_t dims[3], uint32_t b, uint32_t sample_stride,
                               const csgv_config *cfg, csgv_freq_table *table_out, csgv_volume **out, void *stream) {
    return encode_impl(vol_dev, dims, b, nullptr, sample_stride, cfg, table_out, out, stream);
}

struct csgv_stream_encoder {
    EncRun R;
    csgv_freq_table table;
    uint32_t b = 0;
    uint64_t next = 0;  // bricks added so far
};

int csgv_stream_encoder_create(const uint64_t dims[3], uint32_t b, const csgv_freq_table *table,
                               const csgv_config *cfg, csgv_stream_encoder **out, void *stream) {
    uint32_t N;
    int rc = check_dims(dims, b, N);
    if (rc) return rc;
    if (!table || !out) return fail(CSGV_ERR_INVALID_ARG, "NULL argument");
    if (!valid_table(table->freq)) return fail(CSGV_ERR_INVALID_ARG, "frequency tables must sum to 4096 with f >= 1");
    const uint32_t K_max = cfg ? cfg->K_max : 32, S_min = cfg ? cfg->S_min : 256;
    if (K_max < 1 || K_max > 32 || S_min < 1) return fail(CSGV_ERR_INVALID_ARG, "K_max must be 1..32, S_min >= 1");
    *out = nullptr;
    csgv_volume *v = new csgv_volume();
    v->N = N;
    v->K_max = K_max;
    v->S_min = S_min;
    v->n_bricks = 1;
    for (int a = 0; a < 3; a++) {
        v->dims[a] = dims[a];
        v->grid[a] = (dims[a] + b - 1) / b;
        v->n_bricks *= v->grid[a];
    }
    memcpy(v->freq, table->freq, sizeof v->freq);
    rc = vol_alloc_index(v, (cudaStream_t)stream);
    if (rc) {
        vol_free_arrays(v);
        delete v;
        return rc;
    }
    csgv_stream_encoder *e = new csgv_stream_encoder();
    e->R.v = v;
    e->R.G = csgv::make_geom(N, K_max, S_min);
    e->table = *table;
    e->b = b;
    *out = e;
    return CSGV_OK;
}

int csgv_stream_encoder_add(csgv_stream_encoder *enc, const uint32_t *bricks_dev, uint64_t first, uint32_t m,
                            void *stream) {
    if (!enc || !enc->R.v) return fail(CSGV_ERR_INVALID_ARG, "NULL or finished encoder");
    if (m == 0) return CSGV_OK;
    if (!bricks_dev) return fail(CSGV_ERR_INVALID_ARG, "NULL bricks");
    if (first != enc->next) return fail(CSGV_ERR_INVALID_ARG, "bricks must come in order: expected brick %llu, got %llu",
                                        (unsigned long long)enc->next, (unsigned long long)first);
    if (first + m > enc->R.v->n_bricks) return fail(CSGV_ERR_INVALID_ARG, "bricks past the end of the volume");
    if (((uintptr_t)bricks_dev & 15u) != 0) return fail(CSGV_ERR_INVALID_ARG, "bricks_dev must be 16-byte aligned");
    // the batch seen as a volume of m bricks stacked along z: its brick i is the batch's brick i
    csgv::EncVol EV;
    EV.vol = bricks_dev;
    EV.dims[0] = EV.dims[1] = enc->b;
    EV.dims[2] = (uint64_t)enc->b * m;
    EV.nb[0] = EV.nb[1] = 1;
    EV.nb[2] = m;
    const uint64_t C = enc_batch_bricks(enc->R.G, m);
    const int rc = encode_run(enc->R, EV, 0, first, m, C, &enc->table, 1, nullptr, false, (cudaStream_t)stream);
    if (rc) return rc;
    enc->next += m;
    return CSGV_OK;
}

int csgv_stream_encoder_finish(csgv_stream_encoder *enc, csgv_volume **out, void *stream) {
    if (!enc || !enc->R.v || !out) return fail(CSGV_ERR_INVALID_ARG, "NULL argument or finished encoder");
    csgv_volume *v = enc->R.v;
    if (enc->next != v->n_bricks)
        return fail(CSGV_ERR_INVALID_ARG, "%llu of %llu bricks added", (unsigned long long)enc->next,
                    (unsigned long long)v->n_bricks);
    run_finish(enc->R);
    cudaStream_t st = (cudaStream_t)stream;
    int rc = vol_lut(v, nullptr, st);
    if (!rc) rc = vol_ready(v, st);
    if (rc) return rc;
    enc->R.v = nullptr;
    delete enc;
    *out = v;
    return CSGV_OK;
}

void csgv_stream_encoder_destroy(csgv_stream_encoder *enc) {
    if (!enc) return;
    if (enc->R.v) {
        cudaDeviceSynchronize();
        vol_free_arrays(enc->R.v);
        delete enc->R.v;
    }
    delete enc;
}

int csgv_count_bricks(const uint32_t *bricks_dev, uint32_t m, uint32_t b, uint64_t counts[32], void *stream) {
    if (!counts) return fail(CSGV_ERR_INVALID_ARG, "NULL counts");
    if (m == 0) return CSGV_OK;
    if (!bricks_dev) return fail(CSGV_ERR_INVALID_ARG, "NULL bricks");
    const uint64_t dims[3] = {b, b, (uint64_t)b * m};  // the bricks stacked along z
    csgv_freq_table t;
    const int rc = csgv_build_freq_table(bricks_dev, dims, b, 1, &t, stream);
    if (rc) return rc;
    for (int k = 0; k < 32; k++) counts[k] += t.counts[k];
    return CSGV_OK;
}

static int decode_args(const csgv_volume *vol, const uint32_t *ids, const uint8_t *lods, uint32_t n, uint32_t *out,
                       const uint64_t *off, int32_t *status) {
    if (!vol) return fail(CSGV_ERR_INVALID_ARG, "NULL volume");
    if (n == 0) return CSGV_OK;
    if (!ids || !lods || !out || !off || !status) return fail(CSGV_ERR_INVALID_ARG, "NULL request array");
    return CSGV_OK;
}

// Decode requests [r0, r0 + n) in slices whose op records fit the workspace (stream-ordered allocation).
static int decode_range(const csgv_volume *v, const uint32_t *ids, const uint8_t *lods, uint32_t n, uint32_t *out,
                        const uint64_t *off, int32_t *status, bool one_per_launch, cudaStream_t st) {
    int dev = 0, sms = 148;
    CK(cudaGetDevice(&dev));
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaMemPool_t pool;
    int rc = dev_pool(&pool);
    if (rc) return rc;
    // a request's workspace: interior records at 0, leaf records at leaf_at (one byte per op record, at
    // most one per symbol), then the P_a counts before every 8th record of each stream (uint16)
    auto a16 = [](uint64_t x) { return (x + 15) & ~15ull; };
    const uint64_t leaf_at = ((uint64_t)v->max_int_sym + 7) & ~7ull;
    const uint64_t t8_at = a16(leaf_at + (((uint64_t)v->max_leaf_sym + 7) & ~7ull));
    const uint64_t t8_leaf_at = t8_at + a16((leaf_at / 8 + 1) * 2);
    uint64_t stride = t8_leaf_at + a16(((t8_at - leaf_at) / 8 + 1) * 2);
    // b = 64: the request's level arrays (uint32 palette indices, constant flags) and parent list too
    uint64_t lev_at = 0, flag_at = 0, list_at = 0;
    if (v->N >= 6) {
        uint64_t nodes = 0;
        for (uint32_t l = 0; l <= v->N; l++) nodes += 1ull << (3 * (v->N - l));
        lev_at = stride;
        flag_at = lev_at + a16(nodes * 4);
        list_at = flag_at + a16(nodes);
        stride = list_at + a16((1ull << (3 * (v->N - 1))) * 4);
    }
    // b = 64 requests carry their level arrays (about 2 MB each): a larger budget keeps a slice above the
    // SM count
    const uint64_t budget = v->N >= 6 ? std::max<uint64_t>(v->dec_ws_bytes, 2ull << 30) : v->dec_ws_bytes;
    uint64_t S = one_per_launch ? 1 : std::max<uint64_t>(1, std::min<uint64_t>(n, budget / stride));
    const size_t info_bytes = ((size_t)S * 8 + 255) & ~(size_t)255;
    const size_t bytes = 256 + info_bytes + (size_t)S * stride + (size_t)S * 16;  // + the rebuild split's lists
    // the volume may come from another stream; a captured graph cannot depend on uncaptured work, so a
    // decode being captured does not wait (the graph is launched once the volume is complete)
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(st, &cap));
    if (v->ready && cap == cudaStreamCaptureStatusNone) CK(cudaStreamWaitEvent(st, v->ready, 0));
    void *ws = nullptr;
    CK(cudaMallocFromPoolAsync(&ws, bytes, pool, st));
    csgv::RecJob J{};
    J.counter = (uint32_t *)ws;
    J.info = (uint32_t *)((uint8_t *)ws + 256);
    J.recs = (uint8_t *)ws + 256 + info_bytes;
    J.lists = (uint32_t *)((uint8_t *)ws + 256 + info_bytes + (size_t)S * stride);
    J.stride = stride;
    J.leaf_at = leaf_at;
    J.t8_at = t8_at;
    J.t8_leaf_at = t8_leaf_at;
    J.lev_at = lev_at;
    J.flag_at = flag_at;
    J.list_at = list_at;
    J.compact_nodes = v->dec_shape.compact_nodes;
    cudaError_t e = cudaSuccess;
    for (uint64_t r0 = 0; r0 < n && e == cudaSuccess; r0 += S) {
        J.n = (uint32_t)std::min<uint64_t>(S, n - r0);
        J.ids = ids + r0;
        J.lods = lods + r0;
        e = csgv::launch_decode_slice(dev_view(v), v->max_palette, J, out, off + r0, status + r0, v->dec_shape, st);
    }
    cudaError_t ef = cudaFreeAsync(ws, st);
    if (e != cudaSuccess) return cuda_fail(e, "decode launch");
    if (ef != cudaSuccess) return cuda_fail(ef, "cudaFreeAsync");
    return CSGV_OK;
}

int csgv_decode_bricks(const csgv_volume *vol, const uint32_t *brick_ids_dev, const uint8_t *lods_dev, uint32_t n,
                       uint32_t *out_dev, const uint64_t *out_offsets_dev, int32_t *status_dev, void *stream) {
    int rc = decode_args(vol, brick_ids_dev, lods_dev, n, out_dev, out_offsets_dev, status_dev);
    if (rc || n == 0) return rc;
    return decode_range(vol, brick_ids_dev, lods_dev, n, out_dev, out_offsets_dev, status_dev, false,
                        (cudaStream_t)stream);
}

int csgv_decode_bricks_plain(const csgv_volume *vol, const uint32_t *brick_ids_dev, const uint8_t *lods_dev,
                             uint32_t n, uint32_t *out_dev, const uint64_t *out_offsets_dev, int32_t *status_dev,
                             void *stream) {
    int rc = decode_args(vol, brick_ids_dev, lods_dev, n, out_dev, out_offsets_dev, status_dev);
    if (rc || n == 0) return rc;
    return decode_range(vol, brick_ids_dev, lods_dev, n, out_dev, out_offsets_dev, status_dev, true,
                        (cudaStream_t)stream);
}

int csgv_volume_leaves_to_host(csgv_volume *v) {
    if (!v) return fail(CSGV_ERR_INVALID_ARG, "NULL volume");
    if (v->leaf_host) return CSGV_OK;
    const size_t bytes = (v->n_lw + kWordPad) * 2;
    CK(cudaDeviceSynchronize());
    void *h = nullptr;
    if (cudaHostAlloc(&h, bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess || !h)
        return fail(CSGV_ERR_OOM, "cannot allocate %zu bytes of mapped host memory", bytes);
    void *dptr = nullptr;
    cudaError_t e = cudaMemcpy(h, v->leaf_words, bytes, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&dptr, h, 0);
    if (e != cudaSuccess) {
        cudaFreeHost(h);
        return cuda_fail(e, "leaves to host");
    }
    cudaFreeAsync(v->leaf_words, 0);
    CK(cudaDeviceSynchronize());
    v->leaf_words = (uint16_t *)dptr;
    v->leaf_host = (uint16_t *)h;
    return CSGV_OK;
}

int csgv_volume_leaves_to_device(csgv_volume *v) {
    if (!v) return fail(CSGV_ERR_INVALID_ARG, "NULL volume");
    if (!v->leaf_host) return CSGV_OK;
    const size_t bytes = (v->n_lw + kWordPad) * 2;
    cudaMemPool_t pool;
    int rc = dev_pool(&pool);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());
    void *d = nullptr;
    CK(cudaMallocFromPoolAsync(&d, bytes, pool, 0));
    CK(cudaMemcpy(d, v->leaf_host, bytes, cudaMemcpyHostToDevice));
    cudaFreeHost(v->leaf_host);
    v->leaf_host = nullptr;
    v->leaf_words = (uint16_t *)d;
    return CSGV_OK;
}

namespace {
csgv_decode_tuning tuning_of(const csgv_volume *v) {
    csgv_decode_tuning t{};
    t.workspace_bytes = v->dec_ws_bytes;
    t.rans_ctas_per_sm = v->dec_shape.rec_per_sm;
    t.ring_words = v->dec_shape.ring_words;
    t.rebuild_threads = v->dec_shape.leafc_threads;
    t.medium_threads = v->dec_shape.medium_threads;
    t.compact_nodes = v->dec_shape.compact_nodes;
    t.ms = 0.0;
    return t;
}
bool tuning_valid(const csgv_decode_tuning &t) {
    return t.workspace_bytes >= (1ull << 20) && t.rans_ctas_per_sm >= 4 && t.rans_ctas_per_sm <= 6 &&
           (t.ring_words == 128 || t.ring_words == 256 || t.ring_words == 512) &&
           (t.rebuild_threads == 128 || t.rebuild_threads == 256) &&
           (t.medium_threads == 64 || t.medium_threads == 128 || t.medium_threads == 256) && t.compact_nodes <= csgv::kLeafCap &&
           !(t.ring_words == 512 && t.rans_ctas_per_sm == 6);  // 6 x 40 KB of shared memory do not fit an SM
}
void apply_tuning(csgv_volume *v, const csgv_decode_tuning &t) {
    v->dec_ws_bytes = t.workspace_bytes;
    v->dec_shape.rec_per_sm = t.rans_ctas_per_sm;
    v->dec_shape.ring_words = t.ring_words;
    v->dec_shape.leafc_threads = t.rebuild_threads;
    v->dec_shape.medium_threads = t.medium_threads;
    v->dec_shape.compact_nodes = t.compact_nodes;
}
}  // namespace

int csgv_decode_get_tuning(const csgv_volume *vol, csgv_decode_tuning *t) {
    if (!vol || !t) return fail(CSGV_ERR_INVALID_ARG, "NULL argument");
    *t = tuning_of(vol);
    return CSGV_OK;
}

int csgv_decode_set_tuning(csgv_volume *vol, const csgv_decode_tuning *t) {
    if (!vol || !t) return fail(CSGV_ERR_INVALID_ARG, "NULL argument");
    if (!tuning_valid(*t))
        return fail(CSGV_ERR_INVALID_ARG, "decode tuning out of range (workspace %llu B, %u rANS CTAs per SM, ring %u "
                    "words, rebuild %u threads, LOD 1 kernel %u threads, compact layout up to %u nodes)",
                    (unsigned long long)t->workspace_bytes, t->rans_ctas_per_sm, t->ring_words, t->rebuild_threads,
                    t->medium_threads, t->compact_nodes);
    apply_tuning(vol, *t);
    return CSGV_OK;
}

int csgv_decode_autotune(csgv_volume *vol, const uint32_t *brick_ids_dev, const uint8_t *lods_dev, uint32_t n,
                         uint32_t *out_dev, const uint64_t *out_offsets_dev, int32_t *status_dev, void *stream,
                         csgv_decode_tuning *best) {
    int rc = decode_args(vol, brick_ids_dev, lods_dev, n, out_dev, out_offsets_dev, status_dev);
    if (rc) return rc;
    if (!best) return fail(CSGV_ERR_INVALID_ARG, "NULL output");
    cudaStream_t st = (cudaStream_t)stream;
    csgv_decode_tuning b = tuning_of(vol);
    if (n == 0) {
        *best = b;
        return CSGV_OK;
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    // median of kRuns timed runs after one warm-up run of the candidate
    constexpr int kRuns = 5;
    auto time_of = [&](const csgv_decode_tuning &t, double &ms) {
        apply_tuning(vol, t);
        float v[kRuns];
        for (int k = 0; k <= kRuns && rc == CSGV_OK; k++) {
            cudaEventRecord(e0, st);
            rc = decode_range(vol, brick_ids_dev, lods_dev, n, out_dev, out_offsets_dev, status_dev, false, st);
            cudaEventRecord(e1, st);
            float x = 0.f;
            if (rc == CSGV_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&x, e0, e1) != cudaSuccess))
                rc = fail(CSGV_ERR_CUDA, "autotune timing failed");
            if (k > 0) v[k - 1] = x;
        }
        std::sort(v, v + kRuns);
        ms = v[kRuns / 2];
    };
    // one knob at a time, each search starting from the best point so far: the rANS kernel's ring depth and
    // CTAs per SM, the rebuild's threads per request (warps per brick) for LOD 0 requests, the LOD 0 requests
    // that take the compact layout (4 or 8 warps) rather than the full one (8 warps), the threads per LOD 1
    // request, then the workspace per slice (the number of slices)
    time_of(b, b.ms);
    auto search = [&](auto set, std::initializer_list<uint32_t> vals) {
        for (uint32_t x : vals) {
            csgv_decode_tuning c = b;
            set(c, x);
            if (!tuning_valid(c) || rc != CSGV_OK) continue;
            time_of(c, c.ms);
            if (rc == CSGV_OK && c.ms < b.ms) b = c;
        }
    };
    for (uint32_t ring : {128u, 256u, 512u})
        search([&](csgv_decode_tuning &c, uint32_t x) { c.ring_words = ring; c.rans_ctas_per_sm = x; }, {4u, 5u, 6u});
    search([](csgv_decode_tuning &c, uint32_t x) { c.rebuild_threads = x; }, {128u, 256u});
    search([](csgv_decode_tuning &c, uint32_t x) { c.compact_nodes = x; }, {0u, 256u, 512u, 1024u, csgv::kLeafCap});
    search([](csgv_decode_tuning &c, uint32_t x) { c.medium_threads = x; }, {64u, 128u, 256u});
    search([](csgv_decode_tuning &c, uint32_t x) { c.workspace_bytes = (uint64_t)x << 20; }, {64u, 192u, 512u, 1024u});
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    apply_tuning(vol, b);
    if (rc) return rc;
    *best = b;
    return CSGV_OK;
}

int csgv_volume_info_get(const csgv_volume *v, csgv_volume_info *info) {
    if (!v || !info) return fail(CSGV_ERR_INVALID_ARG, "NULL argument");
    memset(info, 0, sizeof *info);
    info->N = v->N;
    for (int a = 0; a < 3; a++) {
        info->dims[a] = v->dims[a];
        info->grid[a] = v->grid[a];
    }
    info->n_bricks = v->n_bricks;
    info->K_max = v->K_max;
    info->S_min = v->S_min;
    info->max_palette = v->max_palette;
    info->palette_labels = v->n_pal;
    info->int_words = v->n_iw;
    info->leaf_words = v->n_lw;
    info->compressed_bytes = v->n_pal * 4 + (v->n_iw + v->n_lw) * 2 + v->n_bricks * (3 * 8 + 2 * 4);
    memcpy(info->freq, v->freq, sizeof info->freq);
    return CSGV_OK;
}

int csgv_volume_export(const csgv_volume *v, uint64_t *pal_off_host, uint32_t *pal_host, uint64_t *int_off_host,
                       uint16_t *int_words_host, uint64_t *leaf_off_host, uint16_t *leaf_words_host,
                       uint32_t *n_int_sym_host, uint32_t *n_leaf_sym_host) {
    if (!v) return fail(CSGV_ERR_INVALID_ARG, "NULL volume");
    const uint64_t n = v->n_bricks;
    CK(cudaDeviceSynchronize());
    if (pal_off_host) CK(cudaMemcpy(pal_off_host, v->pal_off, (n + 1) * 8, cudaMemcpyDeviceToHost));
    if (int_off_host) CK(cudaMemcpy(int_off_host, v->int_off, (n + 1) * 8, cudaMemcpyDeviceToHost));
    if (leaf_off_host) CK(cudaMemcpy(leaf_off_host, v->leaf_off, (n + 1) * 8, cudaMemcpyDeviceToHost));
    if (pal_host && v->n_pal) CK(cudaMemcpy(pal_host, v->pal, v->n_pal * 4, cudaMemcpyDeviceToHost));
    if (int_words_host && v->n_iw) CK(cudaMemcpy(int_words_host, v->int_words, v->n_iw * 2, cudaMemcpyDeviceToHost));
    if (leaf_words_host && v->n_lw)
        CK(cudaMemcpy(leaf_words_host, v->leaf_words, v->n_lw * 2, cudaMemcpyDeviceToHost));
    if (n_int_sym_host) CK(cudaMemcpy(n_int_sym_host, v->n_int_sym, n * 4, cudaMemcpyDeviceToHost));
    if (n_leaf_sym_host) CK(cudaMemcpy(n_leaf_sym_host, v->n_leaf_sym, n * 4, cudaMemcpyDeviceToHost));
    return CSGV_OK;
}

int csgv_volume_import(uint32_t N, const uint64_t dims[3], uint32_t K_max, uint32_t S_min, const uint32_t freq[32],
                       const uint64_t *pal_off_host, const uint32_t *pal_host, const uint64_t *int_off_host,
                       const uint16_t *int_words_host, const uint64_t *leaf_off_host, const uint16_t *leaf_words_host,
                       const uint32_t *n_int_sym_host, const uint32_t *n_leaf_sym_host, csgv_volume **out) {
    uint32_t NN;
    int rc = check_dims(dims, N >= 1 && N <= (uint32_t)csgv::kMaxN ? (1u << N) : 0u, NN);
    if (rc) return rc;
    if (!out || !freq || !pal_off_host || !int_off_host || !leaf_off_host || !n_int_sym_host || !n_leaf_sym_host)
        return fail(CSGV_ERR_INVALID_ARG, "NULL argument");
    if (!valid_table(freq)) return fail(CSGV_ERR_INVALID_ARG, "frequency tables must sum to 4096 with f >= 1");
    if (K_max < 1 || K_max > 32 || S_min < 1) return fail(CSGV_ERR_INVALID_ARG, "K_max must be 1..32, S_min >= 1");
    csgv_volume *v = new csgv_volume();
    v->N = N;
    v->K_max = K_max;
    v->S_min = S_min;
    memcpy(v->freq, freq, sizeof v->freq);
    const uint32_t b = 1u << N;
    v->n_bricks = 1;
    for (int a = 0; a < 3; a++) {
        v->dims[a] = dims[a];
        v->grid[a] = (dims[a] + b - 1) / b;
        v->n_bricks *= v->grid[a];
    }
    const uint64_t n = v->n_bricks;
    v->n_pal = pal_off_host[n];
    v->n_iw = int_off_host[n];
    v->n_lw = leaf_off_host[n];
    uint32_t maxp = 0;
    for (uint64_t i = 0; i < n; i++) {
        if (pal_off_host[i + 1] < pal_off_host[i] || int_off_host[i + 1] < int_off_host[i] ||
            leaf_off_host[i + 1] < leaf_off_host[i]) {
            delete v;
            return fail(CSGV_ERR_INVALID_ARG, "offsets must be non-decreasing");
        }
        maxp = std::max<uint32_t>(maxp, (uint32_t)(pal_off_host[i + 1] - pal_off_host[i]));
        v->max_int_sym = std::max(v->max_int_sym, n_int_sym_host[i]);
        v->max_leaf_sym = std::max(v->max_leaf_sym, n_leaf_sym_host[i]);
    }
    v->max_palette = maxp;
    cudaMemPool_t pool;
    rc = dev_pool(&pool);
    if (rc) {
        delete v;
        return rc;
    }
    auto up = [&](void **d, const void *h, size_t bytes) -> cudaError_t {
        cudaError_t e = cudaMallocFromPoolAsync(d, bytes + 2 * kWordPad, pool, 0);
        if (e == cudaSuccess && bytes && h) e = cudaMemcpy(*d, h, bytes, cudaMemcpyHostToDevice);
        return e;
    };
    cudaError_t e = up((void **)&v->pal_off, pal_off_host, (n + 1) * 8);
    if (e == cudaSuccess) e = up((void **)&v->int_off, int_off_host, (n + 1) * 8);
    if (e == cudaSuccess) e = up((void **)&v->leaf_off, leaf_off_host, (n + 1) * 8);
    if (e == cudaSuccess) e = up((void **)&v->pal, pal_host, v->n_pal * 4);
    if (e == cudaSuccess) e = up((void **)&v->int_words, int_words_host, v->n_iw * 2);
    if (e == cudaSuccess) e = up((void **)&v->leaf_words, leaf_words_host, v->n_lw * 2);
    if (e == cudaSuccess) e = up((void **)&v->n_int_sym, n_int_sym_host, n * 4);
    if (e == cudaSuccess) e = up((void **)&v->n_leaf_sym, n_leaf_sym_host, n * 4);
    if (e != cudaSuccess) {
        vol_free_arrays(v);
        delete v;
        return cuda_fail(e, "volume import");
    }
    rc = vol_lut(v, nullptr, 0);
    if (!rc) rc = vol_ready(v, 0);
    if (!rc && cudaStreamSynchronize(0) != cudaSuccess) rc = fail(CSGV_ERR_CUDA, "volume import: decode table");
    if (rc) {
        vol_free_arrays(v);
        delete v;
        return rc;
    }
    *out = v;
    return CSGV_OK;
}

int csgv_profile_enable(int on) {
    csgv::g_prof_on = on != 0;
    return CSGV_OK;
}

int csgv_profile_reserve(uint32_t n_events) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    std::vector<cudaEvent_t> made;
    made.reserve(n_events);
    cudaError_t err = cudaSuccess;
    for (uint32_t i = 0; i < n_events && err == cudaSuccess; i++) {
        cudaEvent_t e = nullptr;
        err = cudaEventCreate(&e);
        if (err == cudaSuccess) made.push_back(e);
    }
    {
        std::lock_guard<std::mutex> lk(csgv::g_prof_mu);
        for (cudaEvent_t e : made) csgv::g_prof_free.push_back({dev, e});
    }
    if (err != cudaSuccess) return cuda_fail(err, "cudaEventCreate");
    return CSGV_OK;
}

int csgv_profile_read(uint32_t max_kernels, char *names, double *total_ms, uint32_t *launches, uint32_t *n_kernels) {
    if (!names || !total_ms || !launches || !n_kernels) return fail(CSGV_ERR_INVALID_ARG, "NULL output");
    CK(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> lk(csgv::g_prof_mu);
    std::vector<std::string> keys;
    std::vector<double> ms;
    std::vector<uint32_t> cnt;
    cudaError_t err = cudaSuccess;
    for (const auto &r : csgv::g_prof) {
        float t = 0.f;
        cudaError_t e = cudaEventElapsedTime(&t, r.e0, r.e1);
        if (e != cudaSuccess && err == cudaSuccess) err = e;
        csgv::g_prof_free.push_back({r.dev, r.e0});
        csgv::g_prof_free.push_back({r.dev, r.e1});
        size_t k = 0;
        while (k < keys.size() && keys[k] != r.name) k++;
        if (k == keys.size()) {
            keys.push_back(r.name);
            ms.push_back(0.0);
            cnt.push_back(0);
        }
        ms[k] += t;
        cnt[k] += 1;
    }
    csgv::g_prof.clear();
    if (err != cudaSuccess) return cuda_fail(err, "cudaEventElapsedTime");
    const uint32_t nk = (uint32_t)std::min<size_t>(keys.size(), max_kernels);
    for (uint32_t k = 0; k < nk; k++) {
        snprintf(names + 48 * (size_t)k, 48, "%s", keys[k].c_str());
        total_ms[k] = ms[k];
        launches[k] = cnt[k];
    }
    *n_kernels = nk;
    return CSGV_OK;
}

int csgv_volume_destroy_async(csgv_volume *vol, void *stream) {
    if (!vol) return CSGV_OK;
    if (vol->leaf_host) {  // freeing page-locked host memory synchronises anyway
        csgv_volume_destroy(vol);
        return CSGV_OK;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = vol->ready ? cudaStreamWaitEvent(st, vol->ready, 0) : cudaSuccess;
    const cudaError_t ef = vol_free_arrays(vol, st);
    delete vol;
    if (e == cudaSuccess) e = ef;
    return e == cudaSuccess ? CSGV_OK : cuda_fail(e, "csgv_volume_destroy_async");
}

void csgv_volume_destroy(csgv_volume *vol) {
    if (!vol) return;
    cudaDeviceSynchronize();
    vol_free_arrays(vol);
    delete vol;
}

}  // extern "C"
