// csgv_internal.cuh -- constants and device-side structs of libcsgv (CUDA
// side only).  The stream format is the one documented in include/csgv.h.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace csgv {

// rANS parameters (Sec. 3.3; reading R9): 32-bit state, 12-bit scale,
// lower bound 2^16, 16-bit renormalisation words.
constexpr uint32_t kScaleBits = 12;
constexpr uint32_t kM = 1u << kScaleBits;
constexpr uint32_t kL = 1u << 16;

// operation codes (reading R6)
enum : uint32_t { OP_RP = 0, OP_RX = 1, OP_RY = 2, OP_RZ = 3, OP_P0 = 4, OP_PD = 5, OP_PA = 6 };

constexpr int kMaxN = 6;         // b <= 64 (b = 64 keeps its level arrays in global memory)
constexpr uint32_t kFull = 0xFFFFFFFFu;

// per-request status codes written by the decoder (same values as the ABI)
constexpr int32_t kStOk = 0, kStCorrupt = 4, kStRange = 7;

// Morton masks of the x / y / z bits (x = bit 0, R5), up to 6 bits per axis; every use masks them with the
// bits of the level at hand
constexpr uint32_t kMX = 0x9249u, kMY = 0x12492u, kMZ = 0x24924u;

// Decode workspace of one slice of requests.  Request i owns recs + i * stride: interior records at 0, leaf
// records at leaf_at, the P_a counts before every 8th record (uint16) of the two streams at t8_at and
// t8_leaf_at, and for b = 64 its level arrays (uint32 palette indices at lev_at, constant flags at flag_at,
// the listed parents at list_at); info[2i + s] = record count of stream s | a flag if malformed.
struct RecJob {
    const uint32_t *ids;
    const uint8_t *lods;
    uint32_t n;
    uint8_t *recs;
    uint64_t stride, leaf_at, t8_at, t8_leaf_at;
    uint64_t lev_at, flag_at, list_at;  // b = 64 only
    uint32_t *info;
    uint32_t *counter;  // 64 words: [0] work counter of the rANS kernel; [16..21] list counts and work counters of the
                        // rebuild split; [24..25] oversized LOD 0 requests and their work counter
    uint32_t *lists;    // 4 x n request indices (the rebuild split's three lists, then oversized LOD 0 requests)
    uint32_t compact_nodes;  // 32^3 bricks: LOD 0 requests with more non-constant L1 nodes take the full layout
};

// Device view of a compressed volume (passed to kernels by value).
struct VolDev {
    const uint64_t *pal_off, *int_off, *leaf_off;  // n_bricks + 1 each
    const uint32_t *pal;
    const uint16_t *int_words, *leaf_words;
    const uint32_t *n_int_sym, *n_leaf_sym;
    const uint32_t *lut;                           // 2 x 4096 packed decode entries
    uint64_t n_bricks;
    uint32_t N, K_max, S_min;
};

// Packed decode table entry for slot s of a table: symbol (4 bits) |
// frequency (13 bits) << 4 | (s - cum[symbol]) (12 bits) << 17.
__host__ __device__ inline uint32_t lut_pack(uint32_t sym, uint32_t f, uint32_t bias) {
    return sym | (f << 4) | (bias << 17);
}

// One frequency table (16 symbols) normalised to M from nibble counts (Sec. 3.3; reading R11):
// f = 1 + floor(c * (M - 16) / total), and the fewer than 16 units left over go one each to the largest
// counts (ties to the lower symbol).  All-zero counts give the uniform table.  Host and device.
__host__ __device__ inline void normalise_table(const unsigned long long *ct, uint32_t *f) {
    unsigned long long total = 0;
    for (int s = 0; s < 16; s++) total += ct[s];
    if (total == 0) {
        for (int s = 0; s < 16; s++) f[s] = kM / 16;
        return;
    }
    uint32_t sum = 0;
    for (int s = 0; s < 16; s++) {
        const unsigned __int128 q = (unsigned __int128)ct[s] * (kM - 16) / total;
        f[s] = 1u + (uint32_t)q;
        sum += f[s];
    }
    uint32_t used = 0;
    for (uint32_t k = 0; k < kM - sum; k++) {
        int best = -1;
        for (int s = 0; s < 16; s++)
            if (!((used >> s) & 1u) && (best < 0 || ct[s] > ct[best])) best = s;
        used |= 1u << best;
        f[best] += 1;
    }
}

// number of interleaved states for a stream of n symbols (R10)
__host__ __device__ inline uint32_t lanes_for(uint32_t n, uint32_t K_max, uint32_t S_min) {
    if (n == 0) return 0;
    uint32_t k = n / S_min;
    if (k < 1) k = 1;
    if (k > K_max) k = K_max;
    return k;
}

// Launch shape of a decode (csgv_decode_autotune searches it; kept per volume)
// The compact leaf layout of 32^3 LOD 0 requests holds the children of at most this many non-constant L1 nodes
// (20.8 KB of shared memory with the levels above: 10 CTAs of 128 threads per SM)
constexpr uint32_t kLeafCap = 1280;

struct DecodeShape {
    uint32_t rec_per_sm = 4;        // rANS record kernel: CTAs of 8 warps per SM (4..6)
    uint32_t ring_words = 512;      // rANS record kernel: stream words staged per warp (128, 256, 512)
    uint32_t leafc_threads = 128;   // 32^3 bricks, compact leaf layout: threads per request (128, 256)
    uint32_t compact_nodes = kLeafCap;  // 32^3 bricks: LOD 0 requests with at most this many non-constant L1 nodes take
                                    // the compact layout, the others the full one (256 threads, 8 warps)
    uint32_t medium_threads = 128;  // 32^3 bricks, LOD 1 requests of large mixed batches (64, 128, 256)
};

// Kernel timing (csgv_profile_*): while enabled, a ProfScope around a launch records CUDA events on the
// launching stream before and after it (api.cu keeps the records).
// Events come from a per-device free list that csgv_profile_read refills, so that timing a launch costs
// two event records and no event creation.
bool prof_on();
cudaEvent_t prof_event();  // nullptr if no event could be made
void prof_record(const char *name, cudaEvent_t e0, cudaEvent_t e1);
struct ProfScope {
    const char *name;
    cudaStream_t st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ProfScope(const char *n, cudaStream_t s) : name(n), st(s) {
        if (prof_on() && (e0 = prof_event()) && (e1 = prof_event())) cudaEventRecord(e0, st);
    }
    ~ProfScope() {
        if (!e0 || !e1) return;
        cudaEventRecord(e1, st);
        prof_record(name, e0, e1);
    }
};

}  // namespace csgv
