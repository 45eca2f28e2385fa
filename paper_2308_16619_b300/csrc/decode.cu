// decode.cu -- batched brick decoding (Alg. 1 of the paper) for sm_103a.
//
// A batch of requests (brick id, target LOD t) is decoded in slices of requests; a slice takes two
// launches:
//
//   rans_records (one warp per rANS stream; persistent CTAs hold both decode tables in shared memory;
//     for bricks of 16^3 and smaller, rans_records_packed: several short streams per warp, see there).
//     The K interleaved states of a stream live in lanes 0..K-1; a step decodes K symbols and the lanes
//     that renormalise take consecutive words, in lane order (ballot + popc), from a ring window of the
//     stream staged in shared memory by 16-byte loads (Sec. 3.3, readings R9/R10).  Each delta nibble
//     is folded into the P_delta op before it, so the warp writes exactly one op record per coded
//     child, in stream order (byte: op | stop << 3 | delta << 4), plus the number of P_a records before
//     every 8th record (the palette position i_p there, reading R3), and checks the stream's end (every
//     state back at L, every word read).
//
//   rebuild (one CTA per request).  Alg. 1 level by level, in parallel over the nodes of a level.  With one
//     record per child, the 8 records of the j-th non-constant parent of a level sit at 8j, and i_p at them
//     is known, so a level takes barrier-separated passes:
//       1. the children of constant parents take their parent's palette index (the stop-bit semantics), and
//          the non-constant parents of the level are listed in Morton (= stream) order;
//       2. one thread per listed parent decodes its 8 records at once, byte-wise in two registers
//          (kids8_u8): R_p keeps the parent's index, R_a toward +axis reads the neighbour's parent
//          (reading R4), palette ops index the palette (R1, R3), and R_a toward -axis is written as a
//          sentinel naming the axis (and noted per listed parent);
//       3. the sentinels are resolved, in rounds by the child index's bit count or by following a list of
//          them: a chain has at most 3 hops, since each hop lands on a child index with one more bit set.
//     Levels with at most 64 parents take a thread per parent (uint16 indices: a thread per child).  The
//     levels are held as palette indices in shared memory (uint8 when every palette has <= 253 entries,
//     else uint16): all of them, L0 included, in the full layout (rebuild, 256 threads); for LOD 0 of 32^3
//     bricks the compact layout (rebuild_leafc, 128 threads) holds L0 only under the non-constant L1 nodes.
//     Level t is then written as x-fastest labels with 16-byte streaming stores.  The kernels launched for
//     one brick size take N as a template argument, so level offsets and layouts are constants.
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "csgv_internal.cuh"

namespace csgv {


namespace {

constexpr uint32_t kRecBad = 0x80000000u;
constexpr uint32_t kRecWarps = 8;     // rans_records: warps per CTA (8-warp CTAs, 4 to 6 per SM)
constexpr uint32_t kRbThreads = 256;  // rebuild: threads per CTA
constexpr uint32_t kRbWarps = kRbThreads / 32;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ uint32_t lt_of(uint32_t lane) { return (1u << lane) - 1u; }

// ------------------------------------------------------------------ rans_records

// Decode one stream (whole warp) into records and P_a counts; returns the record count, | kRecBad if
// malformed.  Decoding stops once `need` records are out (a coarse LOD uses only the stream's first
// levels); the end of the stream is then not checked.
//
// Coding order (reading R10): op j of the stream is on state j mod K, a P_delta's delta nibble on its op's
// state; a step decodes the ops of its K states in state order, then the deltas of its P_delta ops in state
// order.  Lane k holds state k, so a step is one warp-wide op decode plus, when a P_delta came out, one
// more decode by those lanes; each lane then writes its own record (op | stop << 3 | delta << 4).  The op
// count is not stored: in the stream's last steps (fewer than 2K symbols left) a lane decodes an op only if
// its op and the deltas owed by the lanes before it still fit in the symbols left.
//
// The stream's words are staged in a ring of kWin words in shared memory (word a, counted from the
// 16-byte boundary at or below the stream's start, sits at a % kWin), refilled half a ring at a time
// with 16-byte loads that stay inside the stream's 16-byte chunks.  A malformed stream may read stale
// ring words, never memory outside the ring; the final check (every word read, every state back at L)
// rejects it.  The P_a count before every 8th record only changes at a P_a record, so the counts are
// written in runs: the steps without P_delta / P_a write only their records.
template <uint32_t kWin>  // ring words per warp: 128, 256 or 512 (a step reads at most 64)
__device__ uint32_t decode_stream(const uint16_t *w, uint32_t n_words, uint32_t n_sym, uint32_t K_max,
                                  uint32_t S_min, const uint32_t *lut, uint16_t *win, uint8_t *rec, uint16_t *t8,
                                  uint64_t cap, uint32_t need, uint32_t lane) {
    if (n_sym == 0) {
        if (lane == 0) t8[0] = 0;
        return n_words == 0 ? 0u : kRecBad;
    }
    const uint32_t K = lanes_for(n_sym, K_max, S_min);
    if (n_sym > cap || n_words < 2 * K) return kRecBad;
    static_assert(kWin >= 128 && (kWin & (kWin - 1)) == 0, "half a ring must hold a step's 64 words");
    constexpr uint32_t kRingChunks = kWin / 8, kHalf = kRingChunks / 2;
    const uint32_t lt = lanemask_lt();
    const uintptr_t g0 = reinterpret_cast<uintptr_t>(w) & ~(uintptr_t)15;
    const uint32_t sh = (uint32_t)(reinterpret_cast<uintptr_t>(w) - g0) >> 1;  // words before the stream (0..7)
    const uint32_t n_chunks = (sh + n_words + 7) / 8;  // 16-byte chunks holding the stream
    const uint4 *src = reinterpret_cast<const uint4 *>(g0);
    uint4 *ring = reinterpret_cast<uint4 *>(win);
    __syncwarp();  // the previous stream's reads of the ring are done
    for (uint32_t c = lane; c < kRingChunks && c < n_chunks; c += 32) ring[c] = __ldg(src + c);
    // a step reads at most 2K <= 64 words: refill once pos passes lim
    uint32_t filled = kRingChunks;  // chunks staged so far
    uint32_t lim = filled < n_chunks ? 8 * filled - 64 : 0xFFFFFFFFu;
    __syncwarp();
    uint32_t x = kL;
    if (lane < K) x = (uint32_t)win[sh + 2 * lane] | ((uint32_t)win[sh + 2 * lane + 1] << 16);
    uint32_t pos = sh + 2 * K, left = n_sym, otail = 0, pa_run = 0, t8n = 0;
    bool stuck = false;
    const bool actK = lane < K;
    auto refill = [&]() {  // stage the next half ring over the half already read
        __syncwarp();
        const uint32_t c = filled + lane;
        if (lane < kHalf && c < n_chunks) ring[c % kRingChunks] = __ldg(src + c);
        filled += kHalf;
        lim = filled < n_chunks ? 8 * filled - 64 : 0xFFFFFFFFu;
        __syncwarp();
    };
    // The step after the ops' decode when a P_delta or P_a came out: the deltas of the P_delta lanes, in lane
    // order, then the records and the P_a counts.
    auto general = [&](uint32_t sym, bool act, uint32_t n) {
        const bool pd = act && (sym & 7u) == OP_PD;
        const uint32_t pdm = __ballot_sync(kFull, pd);
        uint32_t dl = 0;
        if (pdm) {
            const uint32_t e2 = lut[x & (kM - 1u)];
            dl = e2 & 15u;
            const uint32_t xn2 = ((e2 >> 4) & 0x1FFFu) * (x >> kScaleBits) + (e2 >> 17);
            const bool nrm2 = pd && xn2 < kL;
            const uint32_t m2 = __ballot_sync(kFull, nrm2);
            const uint32_t wv2 = win[(pos + __popc(m2 & lt)) % kWin];
            x = pd ? (nrm2 ? ((xn2 << 16) | wv2) : xn2) : x;
            pos += __popc(m2);
        }
        // the P_a counts of the records before this step are all pa_run
        for (uint32_t j = t8n + lane; 8 * j < otail; j += 32) t8[j] = (uint16_t)pa_run;
        const uint32_t pam = __ballot_sync(kFull, act && (sym & 7u) == OP_PA);
        if (act) {
            const uint32_t r = otail + lane;
            rec[r] = (uint8_t)(sym | (pd ? dl << 4 : 0u));
            if ((r & 7u) == 0) t8[r >> 3] = (uint16_t)min(pa_run + __popc(pam & lt), 0xFFFFu);
        }
        pa_run = min(pa_run + __popc(pam), 0xFFFFu);  // saturated: a count past any palette is caught later
        otail += n;
        left -= n + __popc(pdm);
        t8n = (otail + 7) / 8;
    };
    // full steps: at least 2K symbols left, so every lane below K decodes an op
    auto full_step = [&]() {
        if (pos > lim) refill();
        const uint32_t e = lut[x & (kM - 1u)];
        const uint32_t sym = e & 15u;
        const uint32_t xn = ((e >> 4) & 0x1FFFu) * (x >> kScaleBits) + (e >> 17);
        const bool nrm = actK && xn < kL;
        const uint32_t m = __ballot_sync(kFull, nrm);
        const uint32_t wv = win[(pos + __popc(m & lt)) % kWin];
        x = nrm ? ((xn << 16) | wv) : xn;  // lanes >= K: never read
        pos += __popc(m);
        if (__ballot_sync(kFull, actK && (sym & 7u) >= OP_PD)) {  // a P_delta or P_a (or 7)
            general(sym, actK, K);
        } else {
            if (actK) rec[otail + lane] = (uint8_t)sym;
            otail += K;
            left -= K;
        }
    };
    // two at a time while two full steps are sure (a step takes at most 2K symbols) and the first cannot
    // reach `need`
    while (left >= 4 * K && otail + K < need) {
        full_step();
        full_step();
    }
    while (left >= 2 * K && otail < need) full_step();
    // the last steps: a lane decodes an op only if it and the deltas owed by the lanes before it fit
    while (left > 0 && otail < need) {
        if (pos > lim) refill();
        const bool cand = actK && lane < left;
        const uint32_t e = lut[x & (kM - 1u)];
        const uint32_t sym = e & 15u;
        const uint32_t xn = ((e >> 4) & 0x1FFFu) * (x >> kScaleBits) + (e >> 17);
        const uint32_t pdc = __ballot_sync(kFull, cand && (sym & 7u) == OP_PD);
        const uint32_t need_k = lane + 1 + __popc(pdc & ((2u << lane) - 1u));
        const uint32_t n = __popc(__ballot_sync(kFull, cand && need_k <= left));
        if (n == 0) {  // a P_delta whose delta is not in the stream: malformed
            stuck = true;
            break;
        }
        const bool act = lane < n;
        const bool nrm = act && xn < kL;
        const uint32_t m = __ballot_sync(kFull, nrm);
        const uint32_t wv = win[(pos + __popc(m & lt)) % kWin];
        x = act ? (nrm ? ((xn << 16) | wv) : xn) : x;
        pos += __popc(m);
        general(sym, act, n);
    }
    // the counts not yet written: every 8th record from t8n on, and the one just past the last record
    for (uint32_t j = t8n + lane; 8 * j <= otail; j += 32) t8[j] = (uint16_t)pa_run;
    if (stuck) return otail | kRecBad;
    if (left > 0) return pos <= sh + n_words ? otail : (otail | kRecBad);  // stopped early: a prefix
    const bool lane_ok = lane >= K || x == kL;
    const bool ok = __all_sync(kFull, lane_ok) && pos == sh + n_words;
    __syncwarp();
    return ok ? otail : (otail | kRecBad);
}

template <uint32_t kWin, bool kListed = false>  // kListed: a large mixed-LOD slice, its streams taken from the class lists
__global__ void __launch_bounds__(kRecWarps * 32, 6) rans_records(VolDev V, RecJob J) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *lut_s = (uint32_t *)smem;
    for (uint32_t i = threadIdx.x; i < 2 * kM / 4; i += blockDim.x)
        ((uint4 *)lut_s)[i] = __ldg((const uint4 *)V.lut + i);
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint16_t *win = (uint16_t *)(smem + 2 * kM * 4) + warp * kWin;
    // listed queue (large mixed-LOD slices): the two streams of every LOD 0 request, then the interior streams
    // of the LOD 1 requests, then those of the coarser ones, so that the long streams go first and no warp
    // draws the leaf stream of a request that has none to decode
    uint32_t c0 = J.n, c1 = 0, c2 = 0;
    if (kListed) {
        c0 = J.counter[16];
        c1 = J.counter[17];
        c2 = J.counter[18];
    }
    const uint32_t q_end = kListed ? 2 * c0 + c1 + c2 : 2 * J.n;
    for (;;) {
        uint32_t q = 0;
        if (lane == 0) q = atomicAdd(J.counter, 1u);
        q = __shfl_sync(kFull, q, 0);
        if (q >= q_end) break;
        uint32_t i = q >> 1, s = q & 1u;
        if (kListed) {
            if (q < 2 * c0) {
                i = J.lists[q >> 1];
            } else {
                const uint32_t k = q - 2 * c0;
                i = k < c1 ? J.lists[J.n + k] : J.lists[2 * J.n + (k - c1)];
                s = 0;
            }
        }
        const uint32_t id = J.ids[i], t = J.lods[i];
        // interior stream: needed below the root (t < N); leaf stream: needed for t == 0
        if (id >= V.n_bricks || t > V.N || (s == 0 ? t >= V.N : t != 0)) continue;
        const uint64_t *offs = s ? V.leaf_off : V.int_off;
        const uint64_t w0 = offs[id];
        const uint32_t n_words = (uint32_t)(offs[id + 1] - w0);
        const uint32_t n_sym = s ? V.n_leaf_sym[id] : V.n_int_sym[id];
        uint8_t *base = J.recs + (uint64_t)i * J.stride;
        uint8_t *rec = base + (s ? J.leaf_at : 0);
        uint16_t *t8 = (uint16_t *)(base + (s ? J.t8_leaf_at : J.t8_at));
        const uint64_t cap = s ? J.t8_at - J.leaf_at : J.leaf_at;  // the records' room: 8 * (t8 entries - 1)
        // LOD t >= 2 uses the interior levels N-1 .. t only: at most 8 records per node of levels N .. t+1
        const uint32_t need = (s == 0 && t >= 2) ? 8u * (((1u << (3 * (V.N - t))) - 1u) / 7u) : 0xFFFFFFFFu;
        const uint32_t r = decode_stream<kWin>((s ? V.leaf_words : V.int_words) + w0, n_words, n_sym, V.K_max, V.S_min,
                                         lut_s + s * kM, win, rec, t8, cap, need, lane);
        if (lane == 0) J.info[2 * i + s] = r;
    }
}

// Short streams (bricks of 16^3 and smaller have K = 1..4 states per stream at the default S_min) leave most
// lanes of a one-stream warp idle, so for them the streams go to warps in groups: a warp takes streams from
// the queue (all interior streams, then all leaf streams) while their K lanes fit in its 32, at most kPkSegs
// of them, each with K <= 16 (a stream with more states is decoded alone), and decodes the group in one loop:
// a step decodes min(K, symbols left) symbols of every stream of the group, each stream on its own run of
// lanes (its segment).  Every per-stream quantity (word position, record tail, P_a count, ...) is held by
// all lanes of the stream's segment; warp votes are masked to the segment; a step with a P_delta or P_a in
// any stream takes the general path for all of them.  Since K = clamp(n / S_min, 1, K_max), the streams with
// K >= 2 take between S_min and 1.5 S_min steps, so the streams of a group end close together.  Each stream
// has its own ring of words (kPkRing words, or the warp's whole area when it is alone), staged as in
// decode_stream.  Same records, counts and statuses as rans_records.
constexpr uint32_t kPkSegs = 8;          // streams per warp at most
constexpr uint32_t kPkRing = 64;         // ring words per stream of a group (uint16)
constexpr uint32_t kPkMaxK = 16;         // most states of a stream that shares its warp
constexpr uint32_t kPkWarpWords = 512;   // ring words per warp
constexpr uint32_t kNoStream = 0xFFFFFFFFu;

__global__ void __launch_bounds__(kRecWarps * 32, 5) rans_records_packed(VolDev V, RecJob J) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *lut_s = (uint32_t *)smem;
    for (uint32_t i = threadIdx.x; i < 2 * kM / 4; i += blockDim.x)
        ((uint4 *)lut_s)[i] = __ldg((const uint4 *)V.lut + i);
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, lt = lanemask_lt();
    uint16_t *rings = (uint16_t *)(smem + 2 * kM * 4) + warp * kPkWarpWords;
    const uint32_t n_q = 2 * J.n;
    uint32_t nxt = kNoStream;  // a stream taken from the queue and not yet placed
    for (;;) {
        // ---- form a group (warp-uniform); lane g keeps the queue index of the group's stream g
        uint32_t my_q = 0, nseg = 0, used = 0, ends = 0;  // ends: bit e set for the last lane e of a segment
        while (nseg < kPkSegs) {
            if (nxt == kNoStream) {
                uint32_t q = 0;
                if (lane == 0) q = atomicAdd(J.counter, 1u);
                nxt = __shfl_sync(kFull, q, 0);
            }
            if (nxt >= n_q) break;
            const uint32_t s = nxt >= J.n ? 1u : 0u, i = nxt - s * J.n;
            const uint32_t id = J.ids[i], t = J.lods[i];
            // interior stream: needed below the root (t < N); leaf stream: needed for t == 0
            if (id >= V.n_bricks || t > V.N || (s == 0 ? t >= V.N : t != 0)) {
                nxt = kNoStream;
                continue;
            }
            const uint64_t *offs = s ? V.leaf_off : V.int_off;
            const uint32_t n_words = (uint32_t)(offs[id + 1] - offs[id]);
            const uint32_t n_sym = s ? V.n_leaf_sym[id] : V.n_int_sym[id];
            const uint32_t K = lanes_for(n_sym, V.K_max, V.S_min);
            const uint64_t cap = s ? J.t8_at - J.leaf_at : J.leaf_at;  // the records' room: 8 * (t8 entries - 1)
            if (n_sym == 0 || n_sym > cap || n_words < 2 * K || K > 32) {  // settled without decoding
                if (lane == 0) {
                    uint8_t *base = J.recs + (uint64_t)i * J.stride;
                    if (n_sym == 0) *(uint16_t *)(base + (s ? J.t8_leaf_at : J.t8_at)) = 0;
                    J.info[2 * i + s] = (n_sym == 0 && n_words == 0) ? 0u : kRecBad;
                }
                nxt = kNoStream;
                continue;
            }
            if (nseg > 0 && (K > kPkMaxK || used + K > 32)) break;  // kept for the next group
            if (lane == nseg) my_q = nxt;
            used += K;
            ends |= 1u << (used - 1);
            nseg++;
            nxt = kNoStream;
            if (K > kPkMaxK) break;  // decoded alone
        }
        if (nseg == 0) break;  // the queue is empty

        // ---- this lane's stream
        const bool mine = lane < used;  // the lane belongs to a stream of the group
        const uint32_t before = ends & lt;
        const uint32_t seg = __popc(before), sb = before ? 32 - __clz(before) : 0u;  // its stream, first lane
        const uint32_t q = __shfl_sync(kFull, my_q, mine ? seg : 0u);  // seg < nseg <= kPkSegs
        const uint32_t s = q >= J.n ? 1u : 0u, i = q - s * J.n;
        const uint32_t rwords = nseg == 1 ? kPkWarpWords : kPkRing, rchunks = rwords / 8, rhalf = rchunks / 2;
        uint32_t K = 1, n_words = 0, sh = 0, n_chunks = 0, need = 0, remaining = 0;
        const uint4 *src = nullptr;
        uint8_t *rec = nullptr;
        uint16_t *t8 = nullptr;
        const uint32_t *lut = lut_s + s * kM;
        uint16_t *win = rings + (mine ? seg : 0u) * kPkRing;
        if (mine) {
            const uint32_t id = J.ids[i], t = J.lods[i];
            const uint64_t *offs = s ? V.leaf_off : V.int_off;
            const uint64_t w0 = offs[id];
            n_words = (uint32_t)(offs[id + 1] - w0);
            remaining = s ? V.n_leaf_sym[id] : V.n_int_sym[id];
            K = lanes_for(remaining, V.K_max, V.S_min);
            const uint16_t *w = (s ? V.leaf_words : V.int_words) + w0;
            const uintptr_t g0 = reinterpret_cast<uintptr_t>(w) & ~(uintptr_t)15;
            sh = (uint32_t)(reinterpret_cast<uintptr_t>(w) - g0) >> 1;  // words before the stream (0..7)
            n_chunks = (sh + n_words + 7) / 8;                          // 16-byte chunks holding the stream
            src = reinterpret_cast<const uint4 *>(g0);
            uint8_t *base = J.recs + (uint64_t)i * J.stride;
            rec = base + (s ? J.leaf_at : 0);
            t8 = (uint16_t *)(base + (s ? J.t8_leaf_at : J.t8_at));
            // LOD t >= 2 uses the interior levels N-1 .. t only: at most 8 records per node of levels N .. t+1
            need = (s == 0 && t >= 2) ? 8u * (((1u << (3 * (V.N - t))) - 1u) / 7u) : 0xFFFFFFFFu;
        }
        const uint32_t j = lane - sb;  // lane within the segment
        const uint32_t smask = mine ? (K >= 32 ? kFull : ((1u << K) - 1u) << sb) : 0u;
        uint4 *ring = reinterpret_cast<uint4 *>(win);
        __syncwarp();  // the previous group's reads of the rings are done
        if (mine)
            for (uint32_t c = j; c < rchunks && c < n_chunks; c += K) ring[c] = __ldg(src + c);
        // a step reads at most 2K words of a stream, 2K <= half a ring: refill once pos passes lim
        uint32_t filled = rchunks;  // chunks staged so far
        uint32_t lim = filled < n_chunks ? 8 * filled - 2 * K : 0xFFFFFFFFu;
        __syncwarp();
        uint32_t x = kL;
        if (mine) x = (uint32_t)win[sh + 2 * j] | ((uint32_t)win[sh + 2 * j + 1] << 16);
        uint32_t pos = sh + 2 * K, otail = 0, pa_run = 0, t8n = 0;
        bool stuck = false;

        // ---- decode the group: per step, each stream's ops on its lanes, then its deltas (reading R10)
        for (;;) {
            const bool run = mine && remaining > 0 && otail < need && !stuck;
            if (!__any_sync(kFull, run)) break;
            if (__any_sync(kFull, run && pos > lim)) {
                __syncwarp();
                if (run && pos > lim) {  // stage the next half ring over the half already read
                    for (uint32_t c = j; c < rhalf; c += K)
                        if (filled + c < n_chunks) ring[(filled + c) & (rchunks - 1u)] = __ldg(src + filled + c);
                    filled += rhalf;
                    lim = filled < n_chunks ? 8 * filled - 2 * K : 0xFFFFFFFFu;
                }
                __syncwarp();
            }
            bool act = run && j < K && j < remaining;
            const uint32_t e = lut[x & (kM - 1u)];
            const uint32_t sym = e & 15u;
            const uint32_t xn = ((e >> 4) & 0x1FFFu) * (x >> kScaleBits) + (e >> 17);
            uint32_t n = run ? K : 0u;
            if (__any_sync(kFull, run && remaining < 2 * K)) {
                // a stream's last steps: the lanes whose op and the deltas owed before it fit in what is left
                const uint32_t pdm = __ballot_sync(kFull, act && (sym & 7u) == OP_PD) & smask;
                const uint32_t need_k = j + 1 + __popc(pdm & ((2u << lane) - 1u));
                const uint32_t fit = __ballot_sync(kFull, act && need_k <= remaining) & smask;
                if (run && remaining < 2 * K) {
                    n = __popc(fit);
                    stuck = n == 0;  // a P_delta whose delta is not in the stream: malformed
                }
            }
            act = act && j < n;
            const bool nrm = act && xn < kL;
            const uint32_t m = __ballot_sync(kFull, nrm) & smask;
            const uint32_t wv = win[(pos + __popc(m & lt)) & (rwords - 1u)];
            x = act ? (nrm ? ((xn << 16) | wv) : xn) : x;
            pos += __popc(m);
            const uint32_t rare = __ballot_sync(kFull, act && (sym & 7u) >= OP_PD);  // P_delta, P_a (or 7)
            if (rare == 0) {  // common case, every stream of the group: no delta to decode, no P_a
                if (act) rec[otail + j] = (uint8_t)sym;
                otail += n;
                remaining -= n;
                continue;
            }
            // every stream of the group takes the general step (exact for the common case too)
            const bool pd = act && (sym & 7u) == OP_PD;
            const uint32_t pdm = __ballot_sync(kFull, pd) & smask;
            uint32_t dl = 0;
            if (__any_sync(kFull, pd)) {  // the deltas of the P_delta ops, in lane order per stream
                const uint32_t e2 = lut[x & (kM - 1u)];
                dl = e2 & 15u;
                const uint32_t xn2 = ((e2 >> 4) & 0x1FFFu) * (x >> kScaleBits) + (e2 >> 17);
                const bool nrm2 = pd && xn2 < kL;
                const uint32_t m2 = __ballot_sync(kFull, nrm2) & smask;
                const uint32_t wv2 = win[(pos + __popc(m2 & lt)) & (rwords - 1u)];
                x = pd ? (nrm2 ? ((xn2 << 16) | wv2) : xn2) : x;
                pos += __popc(m2);
            }
            // the P_a counts of the records before this step are all pa_run
            if (run)
                for (uint32_t k = t8n + j; 8 * k < otail; k += K) t8[k] = (uint16_t)pa_run;
            const uint32_t pam = __ballot_sync(kFull, act && (sym & 7u) == OP_PA) & smask;
            if (act) {
                const uint32_t r = otail + j;
                rec[r] = (uint8_t)(sym | (pd ? dl << 4 : 0u));
                if ((r & 7u) == 0) t8[r >> 3] = (uint16_t)min(pa_run + __popc(pam & lt), 0xFFFFu);
            }
            if (run) {
                pa_run = min(pa_run + __popc(pam), 0xFFFFu);  // saturated: a count past any palette is caught later
                otail += n;
                remaining -= n + __popc(pdm);
                t8n = (otail + 7) / 8;
            }
        }

        // ---- results: the counts not yet written (every 8th record from t8n on, and the one just past the
        // last record), then the record count and the checks of the stream's end
        if (mine)
            for (uint32_t k = t8n + j; 8 * k <= otail; k += K) t8[k] = (uint16_t)pa_run;
        const uint32_t badx = __ballot_sync(kFull, mine && j < K && x != kL) & smask;
        if (mine && j == 0) {
            uint32_t r;
            if (stuck) r = otail | kRecBad;
            else if (remaining > 0) r = pos <= sh + n_words ? otail : (otail | kRecBad);  // stopped early: a prefix
            else r = (badx == 0 && pos == sh + n_words) ? otail : (otail | kRecBad);
            J.info[2 * i + s] = r;
        }
    }
}

// ------------------------------------------------------------------ rebuild

template <typename IdxT>
struct RbTraits;
template <>
struct RbTraits<uint8_t> {
    static constexpr uint32_t kSent = 0xFDu;  // 0xFD, 0xFE, 0xFF: unresolved R_x-, R_y-, R_z-
    static constexpr uint32_t kRep = 0x01010101u;
};
template <>
struct RbTraits<uint16_t> {
    static constexpr uint32_t kSent = 0xFFFDu;
    static constexpr uint32_t kRep = 0x00010001u;
};
template <>
struct RbTraits<uint32_t> {  // the b = 64 kernel only
    static constexpr uint32_t kSent = 0xFFFFFFFDu;
};

constexpr uint32_t kSmallPar = 64;  // levels with at most this many parents are rebuilt one thread per child

// m - e_a / m + e_a on the Morton grid (caller checks the range)
__device__ __forceinline__ uint32_t mdec(uint32_t m, uint32_t ma) { return (((m & ma) - 1u) & ma) | (m & ~ma); }
__device__ __forceinline__ uint32_t minc(uint32_t m, uint32_t ma) { return (((m | ~ma) + 1u) & ma) | (m & ~ma); }

__host__ __device__ __forceinline__ uint32_t spread5(uint32_t v) {
    return (v & 1u) | ((v & 2u) << 2) | ((v & 4u) << 4) | ((v & 8u) << 6) | ((v & 16u) << 8);
}

// bit 7 of each byte of v gathered into bits 0..3
__device__ __forceinline__ uint32_t gather4(uint32_t v) { return (((v >> 7) & 0x01010101u) * 0x00204081u) >> 21 & 15u; }

// Per-byte masks of 8 op records: ops other than R_p, P_a ops, stop bits (bit c = record c)
__device__ __forceinline__ void rec_masks(uint64_t r8, uint32_t &nr, uint32_t &pa, uint32_t &st) {
    const uint32_t lo = (uint32_t)r8, hi = (uint32_t)(r8 >> 32);
    const uint32_t ol = lo & 0x07070707u, oh = hi & 0x07070707u;
    nr = gather4(ol + 0x7F7F7F7Fu) | gather4(oh + 0x7F7F7F7Fu) << 4;
    pa = gather4(~((ol ^ 0x06060606u) + 0x7F7F7F7Fu)) | gather4(~((oh ^ 0x06060606u) + 0x7F7F7F7Fu)) << 4;
    st = gather4(lo << 4) | gather4(hi << 4) << 4;
}

__device__ __forceinline__ uint32_t bsel(uint32_t a, uint32_t b, uint32_t m) { return (a & ~m) | (b & m); }
// bit 7 set in the bytes where a < b, for bytes b < 0x80
__device__ __forceinline__ uint32_t bytes_lt(uint32_t a, uint32_t b) {
    return ~(((a | 0x80808080u) - b) | a) & 0x80808080u;
}

// The 8 children of a non-constant node with uint8 indices, from its 8 op records at once (child c in byte
// c % 4 of word c / 4, byte-wise SIMD in two registers; the same values as one child at a time, Alg. 1): R_p
// the node's index pk; R_a toward +axis (the child's a-bit set) the index of the node's +a neighbour
// (px, py, pz; R4); R_a toward -axis the sentinel kSent + a; P_0 / P_a / P_delta the palette index i_p, i_p + 1,
// i_p - 1 - delta, i_p being ipl plus the node's P_a records before the child (R1, R3).  Sets `minus` (bit c:
// an R_a child toward -axis) and the stop bits `st`; returns false if the records cannot belong to this node:
// op 7, a stop bit on the leaf level, a step out of the brick (lo3 / hi3: the node on the low / high face of
// axis a, bit a), a P_a past the palette or a P_delta before its first entry.
__device__ __forceinline__ bool kids8_u8(uint64_t r8, uint32_t ipl, uint32_t pk, uint32_t px, uint32_t py, uint32_t pz,
                                         uint32_t lo3, uint32_t hi3, uint32_t np, bool leaf, uint2 &v8,
                                         uint32_t &minus, uint32_t &st) {
    constexpr uint32_t B1 = 0x01010101u, BX = 0xFF00FF00u, BY = 0xFFFF0000u, S = RbTraits<uint8_t>::kSent;
    const uint32_t w0 = (uint32_t)r8, w1 = (uint32_t)(r8 >> 32);
    // the 4 ops of a word as the 4 selector nibbles of a byte permute, which then maps every op through an
    // 8-entry byte table: 0xFF (or 1) for the ops of a class, 0 for the others
    const uint32_t o0 = w0 & 0x07070707u, o1 = w1 & 0x07070707u;
    const uint32_t c0 = __byte_perm(o0 | (o0 >> 4), 0u, 0x4420u), c1 = __byte_perm(o1 | (o1 >> 4), 0u, 0x4420u);
    const uint32_t x0 = __byte_perm(0x0000FF00u, 0u, c0), x1 = __byte_perm(0x0000FF00u, 0u, c1);  // R_x (op 1)
    const uint32_t y0 = __byte_perm(0x00FF0000u, 0u, c0), y1 = __byte_perm(0x00FF0000u, 0u, c1);  // R_y (op 2)
    const uint32_t z0 = __byte_perm(0xFF000000u, 0u, c0), z1 = __byte_perm(0xFF000000u, 0u, c1);  // R_z (op 3)
    const uint32_t d0 = __byte_perm(0u, 0x0000FF00u, c0), d1 = __byte_perm(0u, 0x0000FF00u, c1);  // P_delta (5)
    const uint32_t a0 = __byte_perm(0u, 0x00010000u, c0), a1 = __byte_perm(0u, 0x00010000u, c1);  // P_a (6): 1
    const uint32_t p0 = __byte_perm(0u, 0xFFFFFFFFu, c0), p1 = __byte_perm(0u, 0xFFFFFFFFu, c1);  // ops 4..7
    // i_p before each child: byte sums of the P_a bytes before it (at most 7: no carries)
    const uint32_t na0 = (a0 * B1) >> 24, na1 = (a1 * B1) >> 24;
    const uint32_t i0 = ipl * B1 + a0 * 0x01010100u, i1 = (ipl + na0) * B1 + a1 * 0x01010100u;
    const uint32_t e0 = B1 + ((w0 >> 4) & 0x0F0F0F0Fu), e1 = B1 + ((w1 >> 4) & 0x0F0F0F0Fu);  // 1 + delta
    uint32_t v0 = pk * B1, v1 = pk * B1;
    v0 = bsel(v0, px * B1, x0 & BX);
    v0 = bsel(v0, S * B1, x0 & ~BX);
    v1 = bsel(v1, px * B1, x1 & BX);
    v1 = bsel(v1, S * B1, x1 & ~BX);
    v0 = bsel(v0, py * B1, y0 & BY);
    v0 = bsel(v0, (S + 1) * B1, y0 & ~BY);
    v1 = bsel(v1, py * B1, y1 & BY);
    v1 = bsel(v1, (S + 1) * B1, y1 & ~BY);
    v0 = bsel(v0, (S + 2) * B1, z0);  // children 0..3 lie toward -z
    v1 = bsel(v1, pz * B1, z1);        // children 4..7 toward +z
    v0 = bsel(v0, i0 + a0 - (d0 & e0), p0);
    v1 = bsel(v1, i1 + a1 - (d1 & e1), p1);
    v8 = make_uint2(v0, v1);
    minus = gather4((x0 & ~BX) | (y0 & ~BY) | z0) | gather4((x1 & ~BX) | (y1 & ~BY)) << 4;
    st = gather4(w0 << 4) | gather4(w1 << 4) << 4;
    const uint32_t xs = x0 | x1, ys = y0 | y1;
    const bool bad = (__byte_perm(0u, 0xFF000000u, c0) | __byte_perm(0u, 0xFF000000u, c1)) != 0 ||  // op 7
                     (leaf && ((w0 | w1) & 0x08080808u) != 0) ||
                     ((hi3 & 1u) && (xs & BX)) || ((lo3 & 1u) && (xs & ~BX)) || ((hi3 & 2u) && (ys & BY)) ||
                     ((lo3 & 2u) && (ys & ~BY)) || ((hi3 & 4u) && z1) || ((lo3 & 4u) && z0) ||
                     ((a0 | a1) && ipl + na0 + na1 >= np) || ((bytes_lt(i0, e0) & d0) | (bytes_lt(i1, e1) & d1)) != 0;
    return !bad;
}

// The -axis children of a level are resolved in three rounds.  A child c whose a-bit is 0 and whose op is R_a
// reads the node before it along a, which is child c | (1 << a) of the neighbouring parent: a child index with
// one more bit set.  Children with all three bits set are never -axis children, so resolving the -axis children
// with two bits set, then one, then none, each round reads only values that are final (R4).
__device__ __forceinline__ uint32_t sent_round(uint32_t r) {  // child indices {3, 5, 6}, {1, 2, 4}, {0}
    return (0x011668u >> (8 * r)) & 0xFFu;
}

// Final index of node q of a level whose value w is a -axis sentinel: follow the chain (at most 3 hops).
template <typename IdxT>
__device__ __forceinline__ uint32_t chase(const volatile IdxT *L, uint32_t q, uint32_t w, uint32_t lbits) {
    const uint32_t sent = RbTraits<IdxT>::kSent;
    for (int hop = 0; hop < 4 && w >= sent; hop++) {
        q = mdec(q, kMX << (w - sent)) & lbits;
        w = L[q];
    }
    return w < sent ? w : 0u;
}

// shared-memory layout of a rebuild CTA for a brick of side 2^N (byte offsets)
struct RbLayout {
    uint32_t lev, cm, act, mls, misc, pal, total;
    uint32_t lev_shift;          // entries of the levels below the first one held (levels start at lev - shift)
    uint32_t stage, stage_bytes;  // where the interior records and their P_a counts are staged
    // compact leaf level (rb_layout_leafc): the children of the listed L1 nodes, their list, their -axis
    // masks, and the rank of every 32 L1 nodes
    uint32_t e0, act0, mls0, rk;
};
// const bytes of level l (1..N-1): one byte per parent (bit c = child c constant), 16-byte aligned levels
__host__ __device__ __forceinline__ uint32_t cm_off(uint32_t N, uint32_t l) {
    uint32_t o = 0;
    for (uint32_t L = N - 1; L > l; L--) o += ((1u << (3 * (N - L - 1))) + 15u) & ~15u;
    return o;
}
struct RbMisc {
    uint32_t wcnt[kRbWarps];  // listed parents per warp (pass 1)
    uint32_t msk[16];         // small levels: children toward -axis per 32-child step
    uint32_t bad, pad[3];
};
template <typename IdxT>
__host__ __device__ constexpr RbLayout rb_layout(uint32_t N) {
    uint32_t nodes = 0;
    for (uint32_t l = 0; l <= N; l++) nodes += 1u << (3 * (N - l));
    const uint32_t maxpar = 1u << (3 * (N - 1));  // parents of the leaf level
    RbLayout L{};
    L.lev = 0;
    L.cm = (nodes * (uint32_t)sizeof(IdxT) + 15u) & ~15u;
    L.act = L.cm + cm_off(N, 0);
    L.mls = L.act + ((maxpar * 2u + 15u) & ~15u);
    L.misc = L.mls + ((maxpar + 15u) & ~15u);
    L.pal = L.misc + (((uint32_t)sizeof(RbMisc) + 15u) & ~15u);
    L.total = L.pal + (sizeof(IdxT) == 1 ? 256u * 4u : 0u);
    L.lev_shift = 0;
    L.stage = L.lev;  // the L0 area, free until the leaf level
    L.stage_bytes = (1u << (3 * N)) * (uint32_t)sizeof(IdxT);
    return L;
}

// Layout for a request at LOD t >= lmin (1 or 2): levels lmin..N only, the staged interior records (at most
// the records of levels N-1..lmin, plus one step of the rANS kernel for lmin = 2, which stops once they are
// out) in a region of their own, and parent lists only for level 1's 8^(N-2) parents (lmin = 1: level 1 is
// the one level with over 64 parents).
constexpr uint32_t kStageCoarse = 1024, kStageMedium = 6144;
template <typename IdxT>
__host__ __device__ constexpr RbLayout rb_layout_part(uint32_t N, uint32_t lmin) {
    uint32_t nodes = 0, below = 0;
    for (uint32_t l = 0; l <= N; l++) {
        if (l >= lmin) nodes += 1u << (3 * (N - l));
        else below += 1u << (3 * (N - l));
    }
    const uint32_t maxpar = lmin >= 2 ? 0u : 1u << (3 * (N - 2));
    RbLayout L{};
    L.lev = 0;
    L.lev_shift = below;
    L.stage = (nodes * (uint32_t)sizeof(IdxT) + 15u) & ~15u;
    L.stage_bytes = lmin >= 2 ? kStageCoarse : kStageMedium;
    L.cm = L.stage + L.stage_bytes;
    L.act = L.cm + cm_off(N, 0);
    L.mls = L.act + ((maxpar * 2u + 15u) & ~15u);
    L.misc = L.mls + ((maxpar + 15u) & ~15u);
    L.pal = L.misc + (((uint32_t)sizeof(RbMisc) + 15u) & ~15u);
    L.total = L.pal + (sizeof(IdxT) == 1 ? 256u * 4u : 0u);
    return L;
}

// Layout of the compact leaf level (LOD 0 of a brick, uint8 indices): levels 1..N as in rb_layout_part(N, 1);
// L0 is not held whole.  Its nodes under a constant L1 node are that node's index (read from L1 when needed);
// only the 8 children of each non-constant ("listed") L1 node are held, in listed (Morton) order, at most
// kLeafCap nodes.  They share one region with the staged interior records and the level-1 parent lists, which
// are dead once level 1 is rebuilt.  A request with more listed L1 nodes (more than 8 kLeafCap leaf records)
// goes to the full-layout kernel.  kLeafCap (csgv_internal.cuh): 1280 nodes, 20.8 KB, 10 CTAs of 128 threads per SM
// (on voronoi512 b=32 0.143 -> 0.138 ms against 1792 nodes, 26.4 KB and 8 CTAs; 1536 nodes and 9 CTAs 0.138).
template <typename IdxT>
__host__ __device__ constexpr RbLayout rb_layout_leafc(uint32_t N) {
    uint32_t nodes = 0;
    for (uint32_t l = 1; l <= N; l++) nodes += 1u << (3 * (N - l));
    RbLayout L{};
    L.lev = 0;
    L.lev_shift = 1u << (3 * N);
    L.cm = (nodes + 15u) & ~15u;
    L.misc = L.cm + cm_off(N, 0);
    L.pal = L.misc + (((uint32_t)sizeof(RbMisc) + 15u) & ~15u);
    const uint32_t x = L.pal + 256u * 4u;
    // region x: interior stage, level-1 lists (up to level 1) | L0 children, list, masks, ranks (level 0)
    L.stage = x;
    L.stage_bytes = kStageMedium;
    const uint32_t maxpar1 = 1u << (3 * (N - 2));  // parents of level 1
    L.act = x + kStageMedium;
    L.mls = L.act + ((maxpar1 * 2u + 15u) & ~15u);
    const uint32_t upper_end = L.mls + ((maxpar1 + 15u) & ~15u);
    L.e0 = x;
    L.act0 = L.e0 + 8u * kLeafCap;
    L.mls0 = L.act0 + 2u * kLeafCap;
    L.rk = L.mls0 + ((kLeafCap + 15u) & ~15u);
    const uint32_t leaf_end = L.rk + (((1u << (3 * (N - 1))) / 32u) * 2u + 15u & ~15u);
    L.total = upper_end > leaf_end ? upper_end : leaf_end;
    return L;
}

// offset (entries) of level l in the level array: L0 first, then L1 .. LN
__device__ __forceinline__ uint32_t lev_off(uint32_t N, uint32_t l) {
    uint32_t u = 0;
#pragma unroll
    for (uint32_t k = 0; k < (uint32_t)kMaxN; k++)
        if (k < l) u += 1u << (3 * (N - k));
    return u;
}

// Four consecutive labels out, streaming: one 16-byte store where the output is 16-byte aligned (al, the
// output's address mod 16, is 0), two 8-byte stores where it is 8-byte aligned, else four 4-byte stores.  The
// sectors written are the same; only the number of store instructions differs.
__device__ __forceinline__ void store4(uint32_t *p, uint32_t al, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    if (al == 0) {
        __stcs((uint4 *)p, make_uint4(a, b, c, d));
    } else if (al == 8) {
        __stcs((uint2 *)p, make_uint2(a, b));
        __stcs((uint2 *)p + 1, make_uint2(c, d));
    } else {
        __stcs(p, a);
        __stcs(p + 1, b);
        __stcs(p + 2, c);
        __stcs(p + 3, d);
    }
}

// every voxel of a side^3 block gets one label (kT threads); al = the output's address mod 16 (a multiple of 4):
// the labels before the first 16-byte boundary and after the last one are written one by one
template <uint32_t kT>
__device__ __forceinline__ void store_const(uint32_t label, uint32_t side, uint32_t *out, uint32_t al) {
    const uint32_t n = side * side * side;
    const uint32_t head = min(n, ((16u - al) & 15u) >> 2);
    const uint32_t body = (n - head) / 4;
    const uint4 o = make_uint4(label, label, label, label);
    uint4 *ov = (uint4 *)(out + head);
    for (uint32_t i = threadIdx.x; i < body; i += kT) __stcs(ov + i, o);
    const uint32_t tail = head + 4 * body;
    if (threadIdx.x < head) out[threadIdx.x] = label;
    else if (threadIdx.x - head < n - tail) out[tail + threadIdx.x - head] = label;
}

template <typename IdxT, int kPal>  // kPal: 0 palette in lanes (<= 32 entries), 1 in shared memory, 2 global
__device__ __forceinline__ uint32_t lab(uint32_t v, uint32_t pal_reg, const uint32_t *pal_s, const uint32_t *pal,
                                        uint32_t np) {
    if (kPal == 0) return __shfl_sync(kFull, pal_reg, v);  // the source lane is v mod 32
    if (kPal == 1) return pal_s[v & 0xFFu];
    return __ldg(pal + min(v & 0xFFFFu, np - 1));
}

// Write level t (Morton order, side = 2^s) as x-fastest labels.  A unit is 16 consecutive Morton nodes, a
// 4 x 2 x 2 block (Morton bits x0 y0 z0 x1): one 16-byte shared-memory load per thread (two for uint16
// indices) and four 16-byte rows out.  Units go to threads x-fastest, so that the threads of a warp
// complete whole 128-byte rows; their loads are at most 2-way bank conflicts.
template <typename IdxT, int kPal, uint32_t kT>
__device__ __forceinline__ void store_level(const IdxT *C, uint32_t s, uint32_t *out, uint32_t al, uint32_t pal_reg,
                                            const uint32_t *pal_s, const uint32_t *pal, uint32_t np) {
    const uint32_t side = 1u << s;
    if (side >= 4) {
        const uint32_t units = 1u << (3 * s - 4);
        const uint32_t xb = s - 2, yb = s - 1;  // bits of the unit's x and y index
        for (uint32_t u0 = 0; u0 < units; u0 += kT) {
            const uint32_t u = u0 + threadIdx.x;
            const bool in = u < units;
            const uint32_t uu = in ? u : 0u;
            const uint32_t x0 = 4 * (uu & ((1u << xb) - 1u)), y0 = 2 * ((uu >> xb) & ((1u << yb) - 1u)),
                           z0 = 2 * (uu >> (xb + yb));
            const uint32_t m = spread5(x0) | (spread5(y0) << 1) | (spread5(z0) << 2);
            // row (dy, dz) holds Morton offsets o, o+1, o+8, o+9 with o = 2 dy + 4 dz
            uint32_t r[4][4];
            if constexpr (sizeof(IdxT) == 1) {
                const uint4 q = *(const uint4 *)(C + m);
                const uint32_t lo[2] = {q.x, q.y}, hi[2] = {q.z, q.w};  // Morton offsets 0..7, 8..15
#pragma unroll
                for (uint32_t k = 0; k < 4; k++) {  // k = dy + 2 dz: word k/2, byte pair (k % 2) * 2
                    const uint32_t a = lo[k >> 1] >> (16 * (k & 1u)), c = hi[k >> 1] >> (16 * (k & 1u));
                    r[k][0] = lab<IdxT, kPal>(a, pal_reg, pal_s, pal, np);
                    r[k][1] = lab<IdxT, kPal>(a >> 8, pal_reg, pal_s, pal, np);
                    r[k][2] = lab<IdxT, kPal>(c, pal_reg, pal_s, pal, np);
                    r[k][3] = lab<IdxT, kPal>(c >> 8, pal_reg, pal_s, pal, np);
                }
            } else {
                const uint4 q0 = *(const uint4 *)(C + m), q1 = *(const uint4 *)(C + m + 8);
                const uint32_t lo[4] = {q0.x, q0.y, q0.z, q0.w}, hi[4] = {q1.x, q1.y, q1.z, q1.w};
#pragma unroll
                for (uint32_t k = 0; k < 4; k++) {  // k = dy + 2 dz: word k holds offsets 2k, 2k+1
                    r[k][0] = lab<IdxT, kPal>(lo[k], pal_reg, pal_s, pal, np);
                    r[k][1] = lab<IdxT, kPal>(lo[k] >> 16, pal_reg, pal_s, pal, np);
                    r[k][2] = lab<IdxT, kPal>(hi[k], pal_reg, pal_s, pal, np);
                    r[k][3] = lab<IdxT, kPal>(hi[k] >> 16, pal_reg, pal_s, pal, np);
                }
            }
            if (in) {
                uint32_t *o = out + ((size_t)z0 * side + y0) * side + x0;
#pragma unroll
                for (uint32_t k = 0; k < 4; k++)
                    store4(o + (size_t)(k >> 1) * side * side + (k & 1u) * side, al, r[k][0], r[k][1], r[k][2],
                           r[k][3]);
            }
        }
    } else {
        const uint32_t n = side * side * side;
        for (uint32_t i0 = 0; i0 < n; i0 += kT) {
            const uint32_t i = i0 + threadIdx.x;
            const uint32_t ii = i < n ? i : 0u;
            const uint32_t x = ii & (side - 1), y = (ii >> s) & (side - 1), z = ii >> (2 * s);
            const uint32_t v = C[spread5(x) | (spread5(y) << 1) | (spread5(z) << 2)];
            const uint32_t l = lab<IdxT, kPal>(v, pal_reg, pal_s, pal, np);
            if (i < n) out[i] = l;
        }
    }
}

// Levels with at most kSmallPar parents (the top of the tree): one thread per child in Morton order,
// the whole CTA.  The j-th non-constant parent's records sit at 8j; j, i_p and the stop bits come from
// the active-parent mask and warp ballots over a parent's 8 lanes.  With uint8 indices a thread takes a whole
// parent instead (kids8_u8).  Arguments as for rebuild_level.
template <typename IdxT, bool kSmemRec, uint32_t kT>
__device__ __forceinline__ bool rebuild_small_level(uint8_t *smem, const RbLayout &Ly, uint32_t N, uint32_t l,
                                                    const uint8_t *R, const uint16_t *T8, uint32_t n_left,
                                                    uint32_t ip0, uint32_t np, uint32_t &n_act) {
    typedef RbTraits<IdxT> T;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    IdxT *lev = (IdxT *)(smem + Ly.lev) - Ly.lev_shift;
    uint8_t *cm = smem + Ly.cm;
    RbMisc *ms = (RbMisc *)(smem + Ly.misc);
    const uint32_t npar = 1u << (3 * (N - l - 1));  // 1, 8 or 64
    IdxT *P = lev + lev_off(N, l + 1);
    IdxT *C = lev + lev_off(N, l);
    const uint8_t *cmP = (l + 1 < N) ? cm + cm_off(N, l + 1) : nullptr;  // the root is never constant here
    uint8_t *cmC = l >= 1 ? cm + cm_off(N, l) : nullptr;
    const uint32_t pbits = npar - 1, cbits = 8 * npar - 1;
    const uint32_t sent = T::kSent;
    const uint64_t amask = !cmP ? 1ull : npar == 8 ? (~(uint64_t)cmP[0] & 0xFFull) : ~*(const uint64_t *)cmP;
    n_act = __popcll(amask);
    if (8 * n_act > n_left) return false;  // uniform
    if constexpr (sizeof(IdxT) == 1) {  // uint8 indices: a thread per parent, its 8 children at once (kids8_u8)
        uint8_t *mb = reinterpret_cast<uint8_t *>(ms->msk);  // -axis children of parent k (bit c)
        bool bad = false;
        for (uint32_t k = threadIdx.x; k < npar; k += kT) {
            uint2 v8;
            uint32_t minus = 0, st = 0xFFu;
            if ((amask >> k) & 1ull) {
                const uint32_t j = __popcll(amask & ((1ull << k) - 1ull));
                const uint64_t r8 = kSmemRec ? *(const uint64_t *)(R + 8 * j) : __ldg((const unsigned long long *)(R + 8 * j));
                const uint32_t ipl = ip0 + (kSmemRec ? T8[j] : __ldg(T8 + j));
                const uint32_t lo3 = ((k & kMX & pbits) == 0 ? 1u : 0u) | ((k & kMY & pbits) == 0 ? 2u : 0u) |
                                     ((k & kMZ & pbits) == 0 ? 4u : 0u);
                const uint32_t hi3 = ((k & kMX & pbits) == (kMX & pbits) ? 1u : 0u) |
                                     ((k & kMY & pbits) == (kMY & pbits) ? 2u : 0u) |
                                     ((k & kMZ & pbits) == (kMZ & pbits) ? 4u : 0u);
                const uint32_t px = P[minc(k, kMX) & pbits], py = P[minc(k, kMY) & pbits], pz = P[minc(k, kMZ) & pbits];
                bad |= !kids8_u8(r8, ipl, P[k], px, py, pz, lo3, hi3, np, !cmC, v8, minus, st);
            } else {  // a constant parent: its children repeat it
                const uint32_t r = 0x01010101u * (uint32_t)P[k];
                v8 = make_uint2(r, r);
            }
            *(uint2 *)(C + 8 * k) = v8;
            if (cmC) cmC[k] = (uint8_t)st;
            mb[k] = (uint8_t)minus;
        }
        if (threadIdx.x == 0) ms->bad = 0;
        __syncthreads();
        if (bad) ms->bad = 1;
        volatile IdxT *Cv = C;
        for (uint32_t k = threadIdx.x; k < npar; k += kT) {
            uint32_t m = mb[k];
            while (m) {
                const uint32_t c = __ffs(m) - 1;
                m &= m - 1;
                const uint32_t q = 8 * k + c;
                Cv[q] = (IdxT)chase<IdxT>(Cv, q, Cv[q], cbits);
            }
        }
        __syncthreads();
        return ms->bad == 0;
    }
    const uint32_t nch = 8 * npar, steps = (nch + 31) / 32;
    const uint32_t grp = 0xFFu << (lane & 24u), lt = lanemask_lt();
    bool bad = false;
    for (uint32_t s = warp; s < steps; s += (kT / 32)) {
        const uint32_t q = 32 * s + lane;
        const bool in = q < nch;
        const uint32_t k = (q >> 3) & pbits, c = q & 7u;
        const bool act = in && ((amask >> k) & 1ull);
        uint32_t o = 0, ipl = 0;
        if (act) {
            const uint32_t j = __popcll(amask & ((1ull << k) - 1ull));
            o = kSmemRec ? R[8 * j + c] : __ldg(R + 8 * j + c);
            ipl = ip0 + (kSmemRec ? T8[j] : __ldg(T8 + j));
        }
        const uint32_t op = o & 7u, delta = o >> 4;
        const uint32_t pam = __ballot_sync(kFull, act && op == OP_PA);
        const uint32_t stm = __ballot_sync(kFull, act && (o & 8u));
        const uint32_t ipc = ipl + __popc(pam & grp & lt);
        const bool rx = act && op >= OP_RX && op <= OP_RZ;
        const uint32_t a = (op - OP_RX) & 3u, ma = kMX << a;
        const bool plus = rx && ((c >> a) & 1u);
        const bool minus = rx && !plus;
        uint32_t v = P[k];  // constant parent, or R_p
        if (act && op >= OP_P0) v = ipc + (op == OP_PA ? 1u : 0u) - (op == OP_PD ? 1u + delta : 0u);
        if (plus) v = P[minc(k, ma) & pbits];
        if (minus) v = sent + a;
        bad |= act && ((plus && (k & ma & pbits) == (ma & pbits)) || (minus && (q & ma & cbits) == 0) || op == 7u ||
                       (op == OP_PD && ipc < 1 + delta) || (op == OP_PA && ipc + 1 >= np) || (!cmC && (o & 8u)));
        if (in) C[q] = (IdxT)v;
        if (cmC && in && c == 0) cmC[k] = act ? (uint8_t)(stm >> (lane & 24u)) : (uint8_t)0xFF;
        const uint32_t mm = __ballot_sync(kFull, minus);
        if (lane == 0) ms->msk[s] = mm;
    }
    if (threadIdx.x == 0) ms->bad = 0;
    __syncthreads();
    if (bad) ms->bad = 1;
    volatile IdxT *Cv = C;
    for (uint32_t s = warp; s < steps; s += (kT / 32)) {
        if ((ms->msk[s] >> lane) & 1u) {
            const uint32_t q = 32 * s + lane;
            Cv[q] = (IdxT)chase<IdxT>(Cv, q, Cv[q], cbits);
        }
    }
    __syncthreads();
    return ms->bad == 0;
}

// Rebuild children level l from its parents, one thread per listed (non-constant) parent, the whole CTA
// (see the file comment); returns false if the records are malformed.  R: this level's records (in
// shared memory if kSmemRec); T8: P_a counts before every 8th record of the stream from R's first
// record on; n_left: records of the stream from R on; ip0: i_p at the stream's start.  Sets n_act
// (listed parents: 8 * n_act records were used).
template <typename IdxT, bool kSmemRec, uint32_t kT>
__device__ __forceinline__ bool rebuild_level(uint8_t *smem, const RbLayout &Ly, uint32_t N, uint32_t l,
                                              const uint8_t *R, const uint16_t *T8, uint32_t n_left, uint32_t ip0,
                                              uint32_t np, uint32_t &n_act) {
    typedef RbTraits<IdxT> T;
    constexpr uint32_t nw = kT / 32;  // needs nb = npar / 32 >= nw: npar >= 512 here, 64 <= kT <= 256
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    IdxT *lev = (IdxT *)(smem + Ly.lev) - Ly.lev_shift;
    uint8_t *cm = smem + Ly.cm;
    uint16_t *act = (uint16_t *)(smem + Ly.act);
    RbMisc *ms = (RbMisc *)(smem + Ly.misc);
    const uint32_t npar = 1u << (3 * (N - l - 1));  // >= 512
    IdxT *P = lev + lev_off(N, l + 1);
    IdxT *C = lev + lev_off(N, l);
    const uint8_t *cmP = cm + cm_off(N, l + 1);  // l + 1 < N here
    uint8_t *cmC = l >= 1 ? cm + cm_off(N, l) : nullptr;
    const uint32_t pbits = npar - 1;  // Morton code bits of the parent level
    const uint32_t sent = T::kSent;

    // pass 1: children take the parent's index; each warp lists the non-constant parents of its
    // contiguous range of 32-parent blocks
    const uint32_t nb = npar / 32, bpw = nb / nw;
    const uint32_t b0 = warp * bpw, b1 = b0 + bpw;
    uint16_t *mylist = act + 32 * b0;
    uint32_t cnt = 0;
    for (uint32_t b = b0; b < b1; b++) {
        const uint32_t k = 32 * b + lane;
        const uint32_t cw = *(const uint32_t *)(cmP + 4 * b);  // const bits of parents 32b .. 32b+31
        const bool pc = (cw >> lane) & 1u;
        const uint32_t r = T::kRep * (uint32_t)P[k];
        if (sizeof(IdxT) == 1) {
            if (pc) *(uint2 *)(C + 8 * k) = make_uint2(r, r);  // a listed parent's 8 children come from pass 2
        } else {
            *(uint4 *)(C + 8 * k) = make_uint4(r, r, r, r);
        }
        if (cmC && pc) cmC[k] = 0xFF;
        if (!pc) mylist[cnt + __popc(~cw & lt_of(lane))] = (uint16_t)k;
        cnt += __popc(~cw);
    }
    if (lane == 0) ms->wcnt[warp] = cnt;
    __syncthreads();

    // pass 2: one thread per listed parent decodes its records whose op is not R_p
    uint32_t wbase[nw], wofs[nw];  // first listed index of each warp's list; act index - listed index there
    n_act = 0;
#pragma unroll
    for (uint32_t v = 0; v < nw; v++) {
        wbase[v] = n_act;
        wofs[v] = 32 * bpw * v - n_act;
        n_act += ms->wcnt[v];
    }
    if (8 * n_act > n_left) return false;  // uniform: every thread sees the same counts
    const uint32_t nlb = (n_act + 31) / 32;
    uint8_t *mm = smem + Ly.mls;  // children toward -axis of listed parent j (bit c = child c)
    bool bad = false;
    auto parent_of = [&](uint32_t j) -> uint32_t {  // listed parent j lies in the list of the last warp starting at or before j
        uint32_t o = wofs[0];
#pragma unroll
        for (uint32_t v = 1; v < nw; v++) o = j >= wbase[v] ? wofs[v] : o;
        return act[j + o];
    };
    for (uint32_t b = warp; b < nlb; b += nw) {
        const uint32_t j = 32 * b + lane;
        if (j >= n_act) break;
        const uint32_t k = parent_of(j);
        const uint64_t r8 = kSmemRec ? *(const uint64_t *)(R + 8 * j) : __ldg((const unsigned long long *)(R + 8 * j));
        const uint32_t ipl = ip0 + (kSmemRec ? T8[j] : __ldg(T8 + j));
        if constexpr (sizeof(IdxT) == 1) {  // the 8 children at once
            const uint32_t lo3 = ((k & kMX & pbits) == 0 ? 1u : 0u) | ((k & kMY & pbits) == 0 ? 2u : 0u) |
                                 ((k & kMZ & pbits) == 0 ? 4u : 0u);
            const uint32_t hi3 = ((k & kMX & pbits) == (kMX & pbits) ? 1u : 0u) |
                                 ((k & kMY & pbits) == (kMY & pbits) ? 2u : 0u) |
                                 ((k & kMZ & pbits) == (kMZ & pbits) ? 4u : 0u);
            const uint32_t px = P[minc(k, kMX) & pbits], py = P[minc(k, kMY) & pbits], pz = P[minc(k, kMZ) & pbits];
            uint2 v8;
            uint32_t minus_m, st;
            bad |= !kids8_u8(r8, ipl, P[k], px, py, pz, lo3, hi3, np, !cmC, v8, minus_m, st);
            if (cmC) cmC[k] = (uint8_t)st;
            *(uint2 *)(C + 8 * k) = v8;
            mm[j] = (uint8_t)minus_m;
            continue;
        }
        uint32_t nr, pm, st;
        rec_masks(r8, nr, pm, st);
        if (cmC) cmC[k] = (uint8_t)st;
        // checks that hold for the whole parent: no op 7, leaf stop bits 0, the last P_a inside the palette
        const uint32_t lo = (uint32_t)r8, hi = (uint32_t)(r8 >> 32);
        bad |= (((lo & 0x07070707u) + 0x01010101u) & 0x08080808u) != 0 ||
               (((hi & 0x07070707u) + 0x01010101u) & 0x08080808u) != 0 || (!cmC && st != 0) ||
               (pm != 0 && ipl + __popc(pm) >= np);
        // per axis: parent on the brick's low face (-axis leaves the brick), on its high face (+axis)
        const uint32_t lo3 = ((k & kMX & pbits) == 0 ? 1u : 0u) | ((k & kMY & pbits) == 0 ? 2u : 0u) |
                             ((k & kMZ & pbits) == 0 ? 4u : 0u);
        const uint32_t hi3 = ((k & kMX & pbits) == (kMX & pbits) ? 1u : 0u) |
                             ((k & kMY & pbits) == (kMY & pbits) ? 2u : 0u) |
                             ((k & kMZ & pbits) == (kMZ & pbits) ? 4u : 0u);
        uint32_t minus_m = 0;
        while (nr) {
            const uint32_t c = __ffs(nr) - 1;
            nr &= nr - 1;
            const uint32_t o = ((c & 4u ? hi : lo) >> (8 * (c & 3u))) & 0xFFu;
            const uint32_t op = o & 7u, delta = o >> 4;
            const uint32_t ipc = ipl + __popc(pm & ((1u << c) - 1u));
            const bool rx = op <= OP_RZ;  // R_x, R_y, R_z (op != R_p here)
            const uint32_t a = (op - OP_RX) & 3u;
            const bool plus = rx && ((c >> a) & 1u);
            const bool minus = rx && !plus;
            const uint32_t pv = P[minc(k, kMX << a) & pbits];  // +axis: the neighbour's parent (R4)
            uint32_t v = ipc + (op == OP_PA ? 1u : 0u) - (op == OP_PD ? 1u + delta : 0u);  // R1, R3
            v = plus ? pv : minus ? sent + a : v;
            bad |= (plus && ((hi3 >> a) & 1u)) || (minus && ((lo3 >> a) & 1u)) || (op == OP_PD && ipc < 1 + delta);
            C[8 * k + c] = (IdxT)v;
            minus_m |= (minus ? 1u : 0u) << c;
        }
        mm[j] = (uint8_t)minus_m;
    }
    if (threadIdx.x == 0) ms->bad = 0;
    __syncthreads();
    if (bad) ms->bad = 1;

    // pass 3: resolve the -axis children of this warp's listed parents in rounds (see sent_round)
    const uint32_t cbits = 8 * npar - 1;
#pragma unroll 1
    for (uint32_t r = 0; r < 3; r++) {
        for (uint32_t b = warp; b < nlb; b += nw) {
            const uint32_t j = 32 * b + lane;
            uint32_t m = j < n_act ? mm[j] & sent_round(r) : 0u;
            if (!m) continue;
            const uint32_t k = parent_of(j);
            while (m) {
                const uint32_t c = __ffs(m) - 1;
                m &= m - 1;
                const uint32_t q = 8 * k + c;
                const uint32_t w = C[mdec(q, kMX << ((uint32_t)C[q] - sent)) & cbits];
                C[q] = (IdxT)(w < sent ? w : 0u);
            }
        }
        __syncthreads();
    }
    return ms->bad == 0;
}

// The leaf level in the compact layout (rb_layout_leafc), the whole CTA; returns false if the records are
// malformed.  Same decisions as rebuild_level for l = 0, but the children of constant L1 nodes are never
// written: pass A ranks the non-constant L1 nodes (their constant bits are level 1's cm bytes read as 32-bit
// words, bit i = node 32w + i) and lists them; pass B gives one thread per listed node j, which decodes its 8
// records into the 8 children at E[8j] (one 8-byte store); pass C resolves the -axis sentinels, a neighbour
// under a constant L1 node being that node's index and any other E[8 rank + child].  Arguments as for
// rebuild_level; sets n_act.
template <uint32_t kT>
__device__ __forceinline__ bool rebuild_leaf_compact(uint8_t *smem, const RbLayout &Ly, uint32_t N, const uint8_t *R,
                                                     const uint16_t *T8, uint32_t n_left, uint32_t ip0, uint32_t np,
                                                     uint32_t &n_act) {
    typedef uint8_t IdxT;
    typedef RbTraits<IdxT> T;
    constexpr uint32_t nw = kT / 32;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const IdxT *P = (const IdxT *)(smem + Ly.lev) - Ly.lev_shift + lev_off(N, 1);  // L1
    const uint32_t *cw = (const uint32_t *)(smem + Ly.cm + cm_off(N, 1));          // constant bits of L1 nodes
    uint16_t *act = (uint16_t *)(smem + Ly.act0);
    uint8_t *mm = smem + Ly.mls0;
    uint16_t *rk = (uint16_t *)(smem + Ly.rk);
    IdxT *E = (IdxT *)(smem + Ly.e0);
    RbMisc *ms = (RbMisc *)(smem + Ly.misc);
    const uint32_t npar = 1u << (3 * (N - 1)), pbits = npar - 1, cbits = 8 * npar - 1;
    const uint32_t nwords = npar / 32, wpt = (nwords + kT - 1) / kT;  // a contiguous run of words per thread
    const uint32_t w0 = min(threadIdx.x * wpt, nwords), w1 = min(w0 + wpt, nwords);
    const uint32_t sent = T::kSent;

    // pass A: rank and list the non-constant L1 nodes
    uint32_t c = 0;
    for (uint32_t w = w0; w < w1; w++) c += __popc(~cw[w]);
    uint32_t incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t u = __shfl_up_sync(kFull, incl, d);
        if (lane >= (uint32_t)d) incl += u;
    }
    if (lane == 31) ms->wcnt[warp] = incl;
    __syncthreads();
    uint32_t wb = 0;
    n_act = 0;
#pragma unroll
    for (uint32_t v = 0; v < nw; v++) {
        const uint32_t x = ms->wcnt[v];
        wb += v < warp ? x : 0u;
        n_act += x;
    }
    if (8 * n_act > n_left || n_act > kLeafCap) return false;  // uniform
    uint32_t run = wb + incl - c;
    for (uint32_t w = w0; w < w1; w++) {
        uint32_t nc = ~cw[w];
        rk[w] = (uint16_t)run;
        while (nc) {
            act[run++] = (uint16_t)(32 * w + __ffs(nc) - 1);
            nc &= nc - 1;
        }
    }
    if (threadIdx.x == 0) {
        ms->bad = 0;
        ms->pad[0] = 0;  // pass B's list of -axis children
    }
    __syncthreads();

    // pass B: one thread per listed node decodes its 8 records at once (kids8_u8) into E[8j .. 8j + 7].  Its
    // -axis children are also appended to a list (node << 3 | child) in the part of the E area past the listed
    // nodes, for pass C; the list's length is counted even when it does not fit.
    bool bad = false;
    uint16_t *lst = (uint16_t *)(E + 8 * n_act);
    const uint32_t lst_cap = 4 * (kLeafCap - n_act);
    for (uint32_t j0 = 0; j0 < n_act; j0 += kT) {
      const uint32_t j = j0 + threadIdx.x;
      uint32_t minus_m = 0;
      if (j < n_act) {
        const uint32_t k = act[j];
        const uint64_t r8 = __ldg((const unsigned long long *)(R + 8 * j));
        const uint32_t ipl = ip0 + __ldg(T8 + j);
        const uint32_t lo3 = ((k & kMX & pbits) == 0 ? 1u : 0u) | ((k & kMY & pbits) == 0 ? 2u : 0u) |
                             ((k & kMZ & pbits) == 0 ? 4u : 0u);
        const uint32_t hi3 = ((k & kMX & pbits) == (kMX & pbits) ? 1u : 0u) |
                             ((k & kMY & pbits) == (kMY & pbits) ? 2u : 0u) |
                             ((k & kMZ & pbits) == (kMZ & pbits) ? 4u : 0u);
        const uint32_t px = P[minc(k, kMX) & pbits], py = P[minc(k, kMY) & pbits], pz = P[minc(k, kMZ) & pbits];
        uint2 v8;
        uint32_t st;
        bad |= !kids8_u8(r8, ipl, P[k], px, py, pz, lo3, hi3, np, true, v8, minus_m, st);
        *(uint2 *)(E + 8 * j) = v8;
        mm[j] = (uint8_t)minus_m;
      }
      // append this warp's -axis children to the list: one atomic per warp
      const uint32_t c = __popc(minus_m);
      uint32_t incl = c;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
          const uint32_t u = __shfl_up_sync(kFull, incl, d);
          if (lane >= (uint32_t)d) incl += u;
      }
      uint32_t base = 0;
      if (lane == 31 && incl) base = atomicAdd(&ms->pad[0], incl);
      base = __shfl_sync(kFull, base, 31) + incl - c;
      while (minus_m) {
          const uint32_t ch = __ffs(minus_m) - 1;
          minus_m &= minus_m - 1;
          if (base < lst_cap) lst[base] = (uint16_t)((j << 3) | ch);
          base++;
      }
    }
    __syncthreads();
    if (bad) ms->bad = 1;

    // pass C: resolve the -axis children.  A neighbour under a constant L1 node is that node's index, any other
    // E[8 rank + child].  When the list fits, one list entry per thread, each following its chain (at most 3 hops:
    // each lands on a child index with one more bit set; a target another thread is resolving reads either its
    // sentinel, which the chain then follows, or its final index); otherwise per listed node in rounds (see
    // sent_round), where every read is final.
    const uint32_t n_lst = ms->pad[0];
    if (n_lst <= lst_cap) {
        volatile IdxT *Ev = E;
        for (uint32_t e = threadIdx.x; e < n_lst; e += kT) {
            const uint32_t ent = lst[e], j = ent >> 3, ch = ent & 7u;
            uint32_t q = 8 * (uint32_t)act[j] + ch, w = Ev[8 * j + ch];
            for (int hop = 0; hop < 4 && w >= sent; hop++) {
                q = mdec(q, kMX << (w - sent)) & cbits;
                const uint32_t k2 = q >> 3, word = cw[k2 >> 5], bit = k2 & 31u;
                w = ((word >> bit) & 1u) ? (uint32_t)P[k2]
                                         : (uint32_t)Ev[8 * (rk[k2 >> 5] + __popc(~word & ((1u << bit) - 1u))) + (q & 7u)];
            }
            Ev[8 * j + ch] = (IdxT)(w < sent ? w : 0u);
        }
        __syncthreads();
        return ms->bad == 0;
    }
#pragma unroll 1
    for (uint32_t r = 0; r < 3; r++) {
        for (uint32_t j = threadIdx.x; j < n_act; j += kT) {
            uint32_t m = mm[j] & sent_round(r);
            if (!m) continue;
            const uint32_t k = act[j];
            while (m) {
                const uint32_t ch = __ffs(m) - 1;
                m &= m - 1;
                const uint32_t q = mdec(8 * k + ch, kMX << (E[8 * j + ch] - sent)) & cbits;
                const uint32_t k2 = q >> 3, word = cw[k2 >> 5], bit = k2 & 31u;
                const uint32_t w = ((word >> bit) & 1u) ? (uint32_t)P[k2]
                                                        : (uint32_t)E[8 * (rk[k2 >> 5] + __popc(~word & ((1u << bit) - 1u))) + (q & 7u)];
                E[8 * j + ch] = (IdxT)(w < sent ? w : 0u);
            }
        }
        __syncthreads();
    }
    return ms->bad == 0;
}

// Store the leaf level of the compact layout as x-fastest labels: store_level's 16-node units (4 x 2 x 2
// voxels: two x-neighbouring L1 nodes, four 16-byte rows), units x-fastest over the threads so that a warp's
// stores fill whole 128-byte lines.  A thread's units share their x and y (unit index = thread + kT i), so
// only the z part of the Morton base moves.  The children of a node come from E (non-constant node, at its
// rank) or repeat its L1 index; both are loaded and one is selected (the rank of a constant node points
// inside the E area, or at its end), so that the lanes of a warp take one path.
template <int kPal, uint32_t kT>
__device__ __forceinline__ void store_leaf_compact(uint8_t *smem, const RbLayout &Ly, uint32_t N, uint32_t *out, uint32_t al,
                                                   uint32_t pal_reg, const uint32_t *pal_s, const uint32_t *pal,
                                                   uint32_t np) {
    typedef uint8_t IdxT;
    static_assert(kT % 128 == 0, "whole z-layer pairs of 32^3 units per pass of the CTA");
    const IdxT *P = (const IdxT *)(smem + Ly.lev) - Ly.lev_shift + lev_off(N, 1);
    const uint32_t *cw = (const uint32_t *)(smem + Ly.cm + cm_off(N, 1));
    const uint16_t *rk = (const uint16_t *)(smem + Ly.rk);
    const IdxT *E = (const IdxT *)(smem + Ly.e0);
    const uint32_t s = N, side = 1u << s;
    // the 8 children of the x-neighbouring L1 nodes k0 (even) and k0 + 1, four words (Morton offsets 0..15)
    auto kids2 = [&](uint32_t k0, uint32_t (&w)[4]) {
        const uint32_t word = cw[k0 >> 5], bit = k0 & 31u;
        const uint32_t r0 = rk[k0 >> 5] + __popc(~word & ((1u << bit) - 1u));
        const bool c0 = (word >> bit) & 1u, c1 = (word >> (bit + 1)) & 1u;
        const uint32_t r1 = r0 + (c0 ? 0u : 1u);
        const uint32_t p2 = *(const uint16_t *)(P + k0);  // L1 indices of k0, k0 + 1
        const uint2 e0 = *(const uint2 *)(E + 8 * r0), e1 = *(const uint2 *)(E + 8 * r1);
        const uint32_t rep0 = 0x01010101u * (p2 & 0xFFu), rep1 = 0x01010101u * (p2 >> 8);
        w[0] = c0 ? rep0 : e0.x;
        w[1] = c0 ? rep0 : e0.y;
        w[2] = c1 ? rep1 : e1.x;
        w[3] = c1 ? rep1 : e1.y;
    };
    const uint32_t units = 1u << (3 * s - 4);
    const uint32_t xb = s - 2, yb = s - 1;
    // kT is a multiple of the units of one z-layer pair (2^(xb + yb) = 128 for N = 5): x0 and y0 per thread
    const uint32_t u = threadIdx.x;
    const uint32_t x0 = 4 * (u & ((1u << xb) - 1u)), y0 = 2 * ((u >> xb) & ((1u << yb) - 1u));
    const uint32_t mxy = spread5(x0) | (spread5(y0) << 1);
    const uint32_t zstep = kT >> (xb + yb);  // z0 advances by 2 zstep per iteration
    uint32_t z0 = 2 * (u >> (xb + yb));
    for (uint32_t u0 = 0; u0 < units; u0 += kT, z0 += 2 * zstep) {
        const uint32_t m = mxy | (spread5(z0) << 2);
        uint32_t w[4];
        kids2(m >> 3, w);
        uint32_t r[4][4];
#pragma unroll
        for (uint32_t k = 0; k < 4; k++) {  // k = dy + 2 dz: word k/2, byte pair (k % 2) * 2
            const uint32_t aa = w[k >> 1] >> (16 * (k & 1u)), cc = w[2 + (k >> 1)] >> (16 * (k & 1u));
            r[k][0] = lab<IdxT, kPal>(aa, pal_reg, pal_s, pal, np);
            r[k][1] = lab<IdxT, kPal>(aa >> 8, pal_reg, pal_s, pal, np);
            r[k][2] = lab<IdxT, kPal>(cc, pal_reg, pal_s, pal, np);
            r[k][3] = lab<IdxT, kPal>(cc >> 8, pal_reg, pal_s, pal, np);
        }
        uint32_t *o = out + ((size_t)z0 * side + y0) * side + x0;
#pragma unroll
        for (uint32_t k = 0; k < 4; k++)
            store4(o + (size_t)(k >> 1) * side * side + (k & 1u) * side, al, r[k][0], r[k][1], r[k][2], r[k][3]);
    }
}

constexpr int32_t kStToFull = -2;  // internal: the request needs the full-layout kernel

// kT: threads per CTA (64..256; the leaf-level pass needs 64 or more); kLmin: 0, or 1 / 2 for requests at LOD
// >= kLmin only, in the compact layout rb_layout_part
// kLeafC: the compact leaf level (rb_layout_leafc, uint8 indices); a LOD 0 request with more non-constant L1
// nodes than kLeafCap (the layout's room) or J.compact_nodes (the launch shape's choice) returns kStToFull
// untouched (nothing written).
// kN: the brick's N when the kernel is only launched for one brick size, else 0; with it the level loop is
// unrolled and every level offset and layout folds to a constant (rebuild_leafc on voronoi512 b=32: 148 M ->
// 125 M warp instructions, 0.185 -> 0.170 ms)
template <typename IdxT, uint32_t kT, uint32_t kLmin = 0, bool kLeafC = false, uint32_t kN = 0>
__device__ int32_t rebuild_request(const VolDev &V, const RecJob &J, uint8_t *smem, uint32_t i, uint32_t *out) {
    const uint32_t N = kN ? kN : V.N;
    if (kN && V.N != kN) return kStCorrupt;  // launched for another brick size
    const uint32_t id = J.ids[i], t = J.lods[i];
    if (id >= V.n_bricks || t > N) return kStRange;
    if (kLmin && t < kLmin) return kStCorrupt;  // the caller's lists are wrong
    const RbLayout Ly = kLeafC ? rb_layout_leafc<IdxT>(N) : kLmin ? rb_layout_part<IdxT>(N, kLmin) : rb_layout<IdxT>(N);
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t p0 = V.pal_off[id];
    const uint32_t np = (uint32_t)(V.pal_off[id + 1] - p0);
    const uint32_t *pal = V.pal + p0;
    const uint32_t n_int = V.n_int_sym[id], n_leaf = V.n_leaf_sym[id];
    if (np == 0 || np > RbTraits<IdxT>::kSent) return kStCorrupt;
    const uint32_t al = (uint32_t)(reinterpret_cast<uintptr_t>(out) & 15u);  // a multiple of 4
    const uint32_t side = 1u << (N - t);

    // homogeneous brick: no symbols, every LOD is palette[0] (reading R2)
    if (n_int == 0 && n_leaf == 0) {
        if (V.int_off[id + 1] != V.int_off[id] || V.leaf_off[id + 1] != V.leaf_off[id]) return kStCorrupt;
        store_const<kT>(__ldg(pal), side, out, al);
        return kStOk;
    }
    if (t == N) {  // the root: palette index 0 (Alg. 1 initialisation)
        if (threadIdx.x == 0) out[0] = __ldg(pal);
        return kStOk;
    }
    const uint32_t info_int = J.info[2 * i], info_leaf = t == 0 ? J.info[2 * i + 1] : 0u;
    if ((info_int | info_leaf) & kRecBad) return kStCorrupt;
    if (kLeafC && t == 0 && info_leaf > 8 * min(kLeafCap, J.compact_nodes)) return kStToFull;
    const uint8_t *base = J.recs + (uint64_t)i * J.stride;
    const uint16_t *t8i = (const uint16_t *)(base + J.t8_at), *t8l = (const uint16_t *)(base + J.t8_leaf_at);

    IdxT *lev = (IdxT *)(smem + Ly.lev) - Ly.lev_shift;
    uint32_t *pal_s = (uint32_t *)(smem + Ly.pal);
    // The interior stream (at most 8 records per parent of an interior level) and its P_a counts are
    // staged in the L0 area, which is free until the leaf level (coarse requests: a region of their own).
    if (info_int > 8 * (((1u << (3 * (N - 1))) - 1u) / 7u)) return kStCorrupt;
    uint8_t *srec = smem + Ly.stage;
    const uint32_t ri16 = (info_int + 15u) & ~15u;
    const uint32_t t8b = ((info_int / 8 + 1) * 2 + 15u) & ~15u;
    if (info_int > 0 && ri16 + t8b > Ly.stage_bytes) return kStCorrupt;
    const uint16_t *st8 = (const uint16_t *)(srec + ri16);
    if (info_int > 0) {
        for (uint32_t q = threadIdx.x; q < ri16 / 16; q += kT) ((uint4 *)srec)[q] = __ldg((const uint4 *)base + q);
        for (uint32_t q = threadIdx.x; q < t8b / 16; q += kT)
            ((uint4 *)(srec + ri16))[q] = __ldg((const uint4 *)(base + J.t8_at) + q);
    }
    if (sizeof(IdxT) == 1)
        for (uint32_t k = threadIdx.x; k < np; k += kT) pal_s[k] = __ldg(pal + k);
    const uint32_t pal_reg = lane < np ? __ldg(pal + lane) : 0u;
    if (threadIdx.x == 0) lev[lev_off(N, N)] = 0;
    __syncthreads();

    uint32_t used = 0;  // records of the current stream consumed
#pragma unroll
    for (int l = (int)N - 1; l >= (int)t; l--) {
        const bool small = (1u << (3 * (N - l - 1))) <= kSmallPar;
        uint32_t n_act;
        bool good;
        if (l == 0) {  // the leaf stream follows the complete interior stream
            if (used != info_int) return kStCorrupt;
            const uint32_t ip0 = __ldg(t8i + info_int / 8);
            if constexpr (kLeafC)
                good = rebuild_leaf_compact<kT>(smem, Ly, N, base + J.leaf_at, t8l, info_leaf, ip0, np, n_act);
            else if (small)
                good = rebuild_small_level<IdxT, false, kT>(smem, Ly, N, 0u, base + J.leaf_at, t8l, info_leaf, ip0,
                                                            np, n_act);
            else if constexpr (kT >= 64)
                good = rebuild_level<IdxT, false, kT>(smem, Ly, N, 0u, base + J.leaf_at, t8l, info_leaf, ip0, np, n_act);
            else
                good = false;
            used = 8 * n_act;
        } else {
            if (l == 1 && t == 0) {  // warm L1 with the leaf stream's records and P_a counts
                const uint8_t *lr = base + J.leaf_at;
                for (uint32_t q = 128 * threadIdx.x; q < info_leaf; q += 128 * kT)
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(lr + q));
                const uint8_t *lt8 = (const uint8_t *)t8l;
                for (uint32_t q = 128 * threadIdx.x; q < 2 * (info_leaf / 8 + 1); q += 128 * kT)
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(lt8 + q));
            }
            if (small)
                good = rebuild_small_level<IdxT, true, kT>(smem, Ly, N, (uint32_t)l, srec + used, st8 + used / 8,
                                                           info_int - used, 0u, np, n_act);
            else if constexpr (kT >= 64)
                good = rebuild_level<IdxT, true, kT>(smem, Ly, N, (uint32_t)l, srec + used, st8 + used / 8,
                                                     info_int - used, 0u, np, n_act);
            else
                good = false;
            used += 8 * n_act;
        }
        if (!good) return kStCorrupt;
    }
    if ((t == 1 && used != info_int) || (t == 0 && used != info_leaf)) return kStCorrupt;

    if constexpr (kLeafC) {
        if (t == 0) {
            if (np <= 32) store_leaf_compact<0, kT>(smem, Ly, N, out, al, pal_reg, pal_s, pal, np);
            else store_leaf_compact<1, kT>(smem, Ly, N, out, al, pal_reg, pal_s, pal, np);
            return kStOk;
        }
    }
    const IdxT *C = lev + lev_off(N, t);
    const uint32_t s = N - t;
    if (np <= 32) store_level<IdxT, 0, kT>(C, s, out, al, pal_reg, pal_s, pal, np);
    else if (sizeof(IdxT) == 1) store_level<IdxT, 1, kT>(C, s, out, al, pal_reg, pal_s, pal, np);
    else store_level<IdxT, 2, kT>(C, s, out, al, pal_reg, pal_s, pal, np);
    return kStOk;
}

template <typename IdxT>
__global__ void __launch_bounds__(kRbThreads, 4) rebuild(VolDev V, RecJob J, uint32_t *__restrict__ out,
                                                      const uint64_t *__restrict__ out_off,
                                                      int32_t *__restrict__ status) {
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t i = blockIdx.x;
    const int32_t st = rebuild_request<IdxT, kRbThreads>(V, J, smem, i, out + out_off[i]);
    if (threadIdx.x == 0) status[i] = st;
}

// The same for bricks of 16^3: 64-thread CTAs (the leaf level's 512 parents in 2 warps), 24 per SM at 40
// registers a thread (7.5 KB of shared memory each).  For the 32768 bricks of a 512^3 volume: 0.27 ms, against
// 0.30 (128 threads, 16 per SM), 0.45 (256 threads, 8 per SM) and 0.59 ms (256 threads, 4 per SM).
constexpr uint32_t kRbSmallThreads = 64;
template <typename IdxT>
__global__ void __launch_bounds__(kRbSmallThreads, 24) rebuild_small_brick(VolDev V, RecJob J, uint32_t *__restrict__ out,
                                                                   const uint64_t *__restrict__ out_off,
                                                                   int32_t *__restrict__ status) {
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t i = blockIdx.x;
    const int32_t st = rebuild_request<IdxT, kRbSmallThreads, 0, false, 4>(V, J, smem, i, out + out_off[i]);
    if (threadIdx.x == 0) status[i] = st;
}

// Bricks of 8^3 and smaller (no level with over 64 parents): a CTA of kRbTinyThreads threads per request, 32
// CTAs per SM, since a 512-voxel brick keeps few threads busy.
constexpr uint32_t kRbTinyThreads = 64;

template <typename IdxT>
__global__ void __launch_bounds__(kRbTinyThreads, 32) rebuild_tiny_brick(VolDev V, RecJob J, uint32_t *__restrict__ out,
                                                                   const uint64_t *__restrict__ out_off,
                                                                   int32_t *__restrict__ status) {
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t i = blockIdx.x;
    const int32_t st = rebuild_request<IdxT, kRbTinyThreads>(V, J, smem, i, out + out_off[i]);
    if (threadIdx.x == 0) status[i] = st;
}

// Large mixed-LOD batches of 32^3 bricks: split_lods lists the requests by class (LOD 0, LOD 1, LOD >= 2)
// before the rANS kernel, which then takes its streams class by class (the longest first), and one kernel per
// class rebuilds its list: rebuild_listed_leafc in the compact leaf layout (its few
// oversized requests then by rebuild_listed, as rebuild does); rebuild_medium (LOD 1) with
// 128-thread CTAs in a layout without L0 (14 KB), 14 per SM; rebuild_coarse (LOD >= 2) with 64-thread CTAs
// in a layout of levels 2..N (3.4 KB), 32 per SM, since such a request has at most 64 parents per level,
// where a 256-thread CTA with the full 51 KB layout ran 4 per SM.  The three kernels are persistent (see
// rebuild_list).
constexpr uint32_t kRbCoarseThreads = 64;
constexpr uint32_t kSplitMin = 8192;  // requests per slice from which the split pays for its extra launches

// one atomic per warp and class (a warp's requests of a class take consecutive list entries)
__global__ void split_lods(RecJob J, uint32_t N, uint32_t *lists, uint32_t *counts) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x, lane = threadIdx.x & 31, lt = lanemask_lt();
    const bool in = i < J.n;
    const uint32_t t = in ? (uint32_t)J.lods[i] : 0u;
    const uint32_t c = (t >= 2 && t <= N) ? 2u : t == 1 ? 1u : 0u;
#pragma unroll
    for (uint32_t k = 0; k < 3; k++) {
        const uint32_t m = __ballot_sync(kFull, in && c == k);
        if (m == 0) continue;
        const uint32_t leader = __ffs(m) - 1;
        uint32_t base = 0;
        if (lane == leader) base = atomicAdd(&counts[k], (uint32_t)__popc(m));
        base = __shfl_sync(kFull, base, leader);
        if (in && c == k) lists[k * J.n + base + __popc(m & lt)] = i;
    }
}

// One list of the split: persistent CTAs take the list's requests one at a time (a counter per list), so a
// grid is sized to the CTAs that fit on the GPU, not to the batch.  kLeafC: the compact leaf layout, whose
// oversized requests are appended to `full` (count in *n_full) for rebuild_listed.
template <typename IdxT, uint32_t kT, uint32_t kLmin, bool kLeafC = false, uint32_t kN = 0>
__device__ __forceinline__ void rebuild_list(const VolDev &V, const RecJob &J, uint32_t *out, const uint64_t *out_off,
                                             int32_t *status, const uint32_t *list, const uint32_t *count,
                                             uint32_t *next, uint8_t *smem, uint32_t *full = nullptr,
                                             uint32_t *n_full = nullptr) {
    __shared__ uint32_t sh_j;
    const uint32_t n = *count;
    for (;;) {
        if (threadIdx.x == 0) sh_j = atomicAdd(next, 1u);
        __syncthreads();
        const uint32_t j = sh_j;
        __syncthreads();
        if (j >= n) return;
        const uint32_t i = list[j];
        const int32_t st = rebuild_request<IdxT, kT, kLmin, kLeafC, kN>(V, J, smem, i, out + out_off[i]);
        if (threadIdx.x == 0) {
            if (kLeafC && st == kStToFull) full[atomicAdd(n_full, 1u)] = i;
            else status[i] = st;
        }
        __syncthreads();  // the next request reuses the shared memory
    }
}

// The LOD 0 list of a large mixed batch of 32^3 bricks in the compact leaf layout (as rebuild_leafc, persistent)
template <uint32_t kT>
__global__ void __launch_bounds__(kT, kT == 128 ? 10 : 1024 / kT) rebuild_listed_leafc(VolDev V, RecJob J, uint32_t *__restrict__ out,
                                                                    const uint64_t *__restrict__ out_off,
                                                                    int32_t *__restrict__ status, const uint32_t *list,
                                                                    const uint32_t *count, uint32_t *next,
                                                                    uint32_t *full, uint32_t *n_full) {
    extern __shared__ __align__(16) uint8_t smem[];
    rebuild_list<uint8_t, kT, 0, true, 5>(V, J, out, out_off, status, list, count, next, smem, full, n_full);
}

template <typename IdxT>
__global__ void __launch_bounds__(kRbThreads, 4) rebuild_listed(VolDev V, RecJob J, uint32_t *__restrict__ out,
                                                             const uint64_t *__restrict__ out_off,
                                                             int32_t *__restrict__ status, const uint32_t *list,
                                                             const uint32_t *count, uint32_t *next) {
    extern __shared__ __align__(16) uint8_t smem[];
    rebuild_list<IdxT, kRbThreads, 0, false, 5>(V, J, out, out_off, status, list, count, next, smem);
}

template <typename IdxT, uint32_t kT>  // kT: 64, 128 (default) or 256 threads, the autotuner's choice
__global__ void __launch_bounds__(kT, kT == 64 ? 16 : 1792 / kT) rebuild_medium(VolDev V, RecJob J, uint32_t *__restrict__ out,
                                                                  const uint64_t *__restrict__ out_off,
                                                                  int32_t *__restrict__ status, const uint32_t *list,
                                                                  const uint32_t *count, uint32_t *next) {
    extern __shared__ __align__(16) uint8_t smem[];
    rebuild_list<IdxT, kT, 1, false, 5>(V, J, out, out_off, status, list, count, next, smem);
}

template <typename IdxT>
__global__ void __launch_bounds__(kRbCoarseThreads, 32) rebuild_coarse(VolDev V, RecJob J, uint32_t *__restrict__ out,
                                                                  const uint64_t *__restrict__ out_off,
                                                                  int32_t *__restrict__ status, const uint32_t *list,
                                                                  const uint32_t *count, uint32_t *next) {
    extern __shared__ __align__(16) uint8_t smem[];
    rebuild_list<IdxT, kRbCoarseThreads, 2, false, 5>(V, J, out, out_off, status, list, count, next, smem);
}

// Requests of 32^3 bricks with uint8 indices at any LOD, in the compact leaf layout (rb_layout_leafc, 20.8 KB):
// 128-thread CTAs, 10 per SM, 2.5 times the bricks in flight of rebuild's 51 KB layout (or 256-thread CTAs, 4 per
// SM: the autotuner's choice of warps per brick).  A LOD 0 request with more than kLeafCap non-constant L1
// nodes is appended to `full` (count in *n_full) for rebuild_listed.
template <uint32_t kT>
__global__ void __launch_bounds__(kT, kT == 128 ? 10 : 1024 / kT) rebuild_leafc(VolDev V, RecJob J, uint32_t *__restrict__ out,
                                                             const uint64_t *__restrict__ out_off,
                                                             int32_t *__restrict__ status, uint32_t *full,
                                                             uint32_t *n_full) {
    extern __shared__ __align__(16) uint8_t smem[];
    const uint32_t i = blockIdx.x;
    const int32_t st = rebuild_request<uint8_t, kT, 0, true, 5>(V, J, smem, i, out + out_off[i]);
    if (threadIdx.x == 0) {
        if (st == kStToFull) full[atomicAdd(n_full, 1u)] = i;
        else status[i] = st;
    }
}

// ------------------------------------------------------------------ rebuild for b = 64 (global memory)
//
// The levels of a 64^3 brick (299 593 palette indices) do not fit in shared memory: they live in the
// request's workspace (lev_at), with one constant flag per node (flag_at) and the listed parents of the level
// being rebuilt (list_at).  The indices are uint8 when every palette has at most 253 entries, uint16 up to
// 65 533, else uint32 (a 64^3 palette may pass 2^16 entries), so that the levels of the bricks in flight
// mostly stay in L2.  One CTA of kGwThreads threads per request, level by level: the non-constant parents are
// listed by a block scan; every record of the level is decoded by the thread owning its run of records, with
// i_p from a block scan of the P_a counts (so no sampled P_a counts are needed); children of constant parents
// copy their parent; -axis sentinels are then followed (at most 3 hops, as in the shared-memory kernel), 16
// bytes of a level tested at a time.  Level t is stored as in store_level: 16 Morton-consecutive nodes per
// thread step, four 16-byte rows out.  Same results and status codes as rebuild.

constexpr uint32_t kGwThreads = 1024;
constexpr uint32_t kGwPalSmem = 1024;  // palettes up to this many entries are staged in shared memory

__host__ __device__ __forceinline__ uint32_t spread6(uint32_t v) {
    return (v & 1u) | ((v & 2u) << 2) | ((v & 4u) << 4) | ((v & 8u) << 6) | ((v & 16u) << 8) | ((v & 32u) << 10);
}

// exclusive block scan of one value per thread; red: 33 words of shared memory
__device__ __forceinline__ uint32_t gw_scan(uint32_t v, uint32_t *red, uint32_t &total) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t u = __shfl_up_sync(kFull, incl, d);
        if (lane >= (uint32_t)d) incl += u;
    }
    if (lane == 31) red[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < nw ? red[lane] : 0u;
        uint32_t x = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t u = __shfl_up_sync(kFull, x, d);
            if (lane >= (uint32_t)d) x += u;
        }
        red[lane] = x - w;
        if (lane == 31) red[32] = x;
    }
    __syncthreads();
    const uint32_t r = red[warp] + incl - v;
    total = red[32];
    __syncthreads();
    return r;
}

// any -axis sentinel among the indices packed in 16 bytes
__device__ __forceinline__ bool gw_any_sent(uint4 q, uint8_t) {
    return ((q.x & ((q.x & 0x7F7F7F7Fu) + 0x03030303u)) | (q.y & ((q.y & 0x7F7F7F7Fu) + 0x03030303u)) |
            (q.z & ((q.z & 0x7F7F7F7Fu) + 0x03030303u)) | (q.w & ((q.w & 0x7F7F7F7Fu) + 0x03030303u))) &
           0x80808080u;
}
__device__ __forceinline__ bool gw_any_sent(uint4 q, uint16_t) {
    return ((q.x & ((q.x & 0x7FFF7FFFu) + 0x00030003u)) | (q.y & ((q.y & 0x7FFF7FFFu) + 0x00030003u)) |
            (q.z & ((q.z & 0x7FFF7FFFu) + 0x00030003u)) | (q.w & ((q.w & 0x7FFF7FFFu) + 0x00030003u))) &
           0x80008000u;
}
__device__ __forceinline__ bool gw_any_sent(uint4 q, uint32_t) {
    return q.x >= 0xFFFFFFFDu || q.y >= 0xFFFFFFFDu || q.z >= 0xFFFFFFFDu || q.w >= 0xFFFFFFFDu;
}

// node e of a 16-byte group of indices
template <typename IdxT>
__device__ __forceinline__ uint32_t gw_elem(const uint32_t (&w)[4], uint32_t e) {
    if (sizeof(IdxT) == 1) return (w[e >> 2] >> (8 * (e & 3u))) & 0xFFu;
    if (sizeof(IdxT) == 2) return (w[e >> 1] >> (16 * (e & 1u))) & 0xFFFFu;
    return w[e];
}

template <typename IdxT>
__device__ int32_t rebuild_global_request(const VolDev &V, const RecJob &J, uint32_t i, uint32_t *out,
                                          uint32_t *red, uint32_t &sh_bad, uint32_t *pal_s) {
    const uint32_t sent = RbTraits<IdxT>::kSent;
    const uint32_t N = V.N, nt = blockDim.x, tid = threadIdx.x;
    const uint32_t id = J.ids[i], t = J.lods[i];
    if (id >= V.n_bricks || t > N) return kStRange;
    const uint64_t p0 = V.pal_off[id], np64 = V.pal_off[id + 1] - p0;
    if (np64 == 0 || np64 > sent) return kStCorrupt;
    const uint32_t np = (uint32_t)np64;
    const uint32_t *pal = V.pal + p0;
    const uint32_t n_int = V.n_int_sym[id], n_leaf = V.n_leaf_sym[id];
    const uint32_t s = N - t, side = 1u << s, nvox = side * side * side;
    if (n_int == 0 && n_leaf == 0) {  // homogeneous brick (reading R2)
        if (V.int_off[id + 1] != V.int_off[id] || V.leaf_off[id + 1] != V.leaf_off[id]) return kStCorrupt;
        const uint32_t l0 = __ldg(pal);
        for (uint32_t q = tid; q < nvox; q += nt) out[q] = l0;
        return kStOk;
    }
    if (t == N) {
        if (tid == 0) out[0] = __ldg(pal);
        return kStOk;
    }
    const uint32_t info_int = J.info[2 * i], info_leaf = t == 0 ? J.info[2 * i + 1] : 0u;
    if ((info_int | info_leaf) & kRecBad) return kStCorrupt;
    uint8_t *base = J.recs + (uint64_t)i * J.stride;
    IdxT *lev = (IdxT *)(base + J.lev_at);
    uint8_t *flg = base + J.flag_at;
    uint32_t *lst = (uint32_t *)(base + J.list_at);
    const bool pal_in_smem = np <= kGwPalSmem;
    if (pal_in_smem)
        for (uint32_t k = tid; k < np; k += nt) pal_s[k] = __ldg(pal + k);
    if (tid == 0) {
        lev[lev_off(N, N)] = 0;  // the root: palette index 0, not constant (the brick has symbols)
        flg[lev_off(N, N)] = 0;
    }
    __syncthreads();
    uint32_t used = 0, ip = 0;
    for (int li = (int)N - 1; li >= (int)t; li--) {
        const uint32_t l = (uint32_t)li;
        const uint32_t npar = 1u << (3 * (N - l - 1)), nch = 8 * npar, pbits = npar - 1, cbits = nch - 1;
        const IdxT *P = lev + lev_off(N, l + 1);
        IdxT *C = lev + lev_off(N, l);
        const uint8_t *fP = flg + lev_off(N, l + 1);
        uint8_t *fC = flg + lev_off(N, l);
        const uint8_t *R = base + used;
        uint32_t n_left = info_int - used;
        if (l == 0) {  // the leaf stream follows the complete interior stream
            if (used != info_int) return kStCorrupt;
            R = base + J.leaf_at;
            n_left = info_leaf;
            used = 0;
        }
        // the non-constant parents, in Morton order
        uint32_t n_act;
        {
            const uint32_t per = (npar + nt - 1) / nt, k0 = min(tid * per, npar), k1 = min(k0 + per, npar);
            uint32_t c = 0;
            if (per % 16 == 0) {  // 16 flags (0 or 1 each) per load; the range starts on a 16-byte boundary
                for (uint32_t k = k0; k < k1; k += 16) {
                    const uint4 f = *(const uint4 *)(fP + k);
                    c += 16 - __popc(f.x) - __popc(f.y) - __popc(f.z) - __popc(f.w);
                }
            } else {
                for (uint32_t k = k0; k < k1; k++) c += fP[k] == 0 ? 1u : 0u;
            }
            uint32_t j = gw_scan(c, red, n_act);
            if (per % 16 == 0) {
                for (uint32_t k = k0; k < k1; k += 16) {
                    const uint4 f = *(const uint4 *)(fP + k);
                    const uint32_t w[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
                    for (uint32_t e = 0; e < 16; e++)
                        if (((w[e >> 2] >> (8 * (e & 3u))) & 0xFFu) == 0) lst[j++] = k + e;
                }
            } else {
                for (uint32_t k = k0; k < k1; k++)
                    if (fP[k] == 0) lst[j++] = k;
            }
        }
        if (8 * n_act > n_left) return kStCorrupt;
        if (tid == 0) sh_bad = 0;
        __syncthreads();
        // every record of the level: i_p before it = ip + the P_a records before it in this level.  Warp w takes
        // a contiguous range of records, 32 consecutive ones per step (one per lane), so that the record loads
        // and the children's stores of a step are contiguous; i_p from a block scan of the warps' P_a counts
        // and a ballot per step.
        const uint32_t nrec = 8 * n_act;
        bool bad = false;
        uint32_t n_pa;
        {
            const uint32_t lane = tid & 31, warp = tid >> 5, nw = nt >> 5, lt = lanemask_lt();
            const uint32_t chunk = ((nrec + nw - 1) / nw + 31) & ~31u;
            const uint32_t r0 = min(warp * chunk, nrec), r1 = min(r0 + chunk, nrec);
            uint32_t c = 0;
            for (uint32_t r = r0 + lane; r < r1; r += 32) c += (R[r] & 7u) == OP_PA ? 1u : 0u;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(kFull, c, d);
            const uint32_t before = gw_scan(lane == 0 ? c : 0u, red, n_pa);  // lane 0: P_a of the warps before
            uint32_t ipc = ip + __shfl_sync(kFull, before, 0);
            for (uint32_t rr = r0; rr < r1; rr += 32) {
                const uint32_t r = rr + lane;
                const bool in = r < r1;
                const uint32_t o = in ? (uint32_t)R[r] : 0u, op = o & 7u, stop = (o >> 3) & 1u, delta = o >> 4;
                const uint32_t pam = __ballot_sync(kFull, in && op == OP_PA);
                const uint32_t ipr = ipc + __popc(pam & lt);
                ipc += __popc(pam);
                if (!in) continue;
                const uint32_t k = lst[r >> 3], c8 = r & 7u, q = 8 * k + c8;
                uint32_t v = P[k];  // R_p
                if (op >= OP_RX && op <= OP_RZ) {
                    const uint32_t a = op - OP_RX, ma = kMX << a;
                    if ((c8 >> a) & 1u) {  // +axis: the neighbour's parent (R4)
                        if ((k & ma & pbits) == (ma & pbits)) bad = true;
                        else v = P[minc(k, ma) & pbits];
                    } else {  // -axis: the node before it on this level, resolved below
                        if ((q & ma & cbits) == 0) bad = true;
                        v = sent + a;
                    }
                } else if (op >= OP_P0) {
                    if (op == 7u || (op == OP_PD && ipr < 1 + delta) || (op == OP_PA && ipr + 1 >= np)) bad = true;
                    v = ipr + (op == OP_PA ? 1u : 0u) - (op == OP_PD ? 1u + delta : 0u);
                }
                if (l == 0 && stop) bad = true;  // leaf records carry no stop bit
                C[q] = (IdxT)v;
                if (l >= 1) fC[q] = (uint8_t)stop;
            }
        }
        // children of constant parents repeat their parent (8 children: one 8 / 16 / 32-byte store)
        for (uint32_t k = tid; k < npar; k += nt)
            if (fP[k]) {
                const uint32_t v = P[k];
                if (sizeof(IdxT) == 1) {
                    const uint32_t r4 = 0x01010101u * v;
                    *(uint2 *)(C + 8 * k) = make_uint2(r4, r4);
                } else if (sizeof(IdxT) == 2) {
                    const uint32_t r2 = 0x00010001u * v;
                    *(uint4 *)(C + 8 * k) = make_uint4(r2, r2, r2, r2);
                } else {
                    *(uint4 *)(C + 8 * k) = make_uint4(v, v, v, v);
                    *(uint4 *)(C + 8 * k + 4) = make_uint4(v, v, v, v);
                }
                if (l >= 1) *(uint2 *)(fC + 8 * k) = make_uint2(0x01010101u, 0x01010101u);
            }
        if (bad) sh_bad = 1;
        __syncthreads();
        // follow the -axis sentinels, 16 bytes of the level at a time (the 8-node level: one node at a time)
        volatile IdxT *Cv = C;
        auto resolve = [&](uint32_t q) {
            uint32_t w = Cv[q];
            if (w >= sent) {
                uint32_t qq = q;
                for (int hop = 0; hop < 4 && w >= sent; hop++) {
                    qq = mdec(qq, kMX << (w - sent)) & cbits;
                    w = Cv[qq];
                }
                if (w >= sent) sh_bad = 1;
                else Cv[q] = (IdxT)w;
            }
        };
        constexpr uint32_t per16 = 16 / sizeof(IdxT);
        if (nch >= per16) {
            for (uint32_t g = tid; g < nch / per16; g += nt) {
                const uint4 q4 = __ldcg((const uint4 *)(C + per16 * g));  // L2: other threads resolve nodes meanwhile
                if (gw_any_sent(q4, (IdxT)0))
                    for (uint32_t e = 0; e < per16; e++) resolve(per16 * g + e);
            }
        } else {
            for (uint32_t q = tid; q < nch; q += nt) resolve(q);
        }
        __syncthreads();
        if (sh_bad) return kStCorrupt;
        ip += n_pa;
        used += nrec;
    }
    if ((t == 1 && used != info_int) || (t == 0 && used != info_leaf)) return kStCorrupt;
    const IdxT *Ct = lev + lev_off(N, t);
    auto lab = [&](uint32_t v) { return pal_in_smem ? pal_s[min(v, np - 1)] : __ldg(pal + min(v, np - 1)); };
    const uint32_t al = (uint32_t)(reinterpret_cast<uintptr_t>(out) & 15u);
    if (side >= 4) {
        // a unit is 16 Morton-consecutive nodes, a 4 x 2 x 2 block (Morton bits x0 y0 z0 x1); row (dy, dz)
        // holds Morton offsets o, o+1, o+8, o+9 with o = 2 dy + 4 dz
        const uint32_t units = nvox / 16, xb = s - 2, yb = s - 1;
        for (uint32_t u = tid; u < units; u += nt) {
            const uint32_t x0 = 4 * (u & ((1u << xb) - 1u)), y0 = 2 * ((u >> xb) & ((1u << yb) - 1u)),
                           z0 = 2 * (u >> (xb + yb));
            const uint32_t m = spread6(x0) | (spread6(y0) << 1) | (spread6(z0) << 2);
            uint32_t n16[16];
#pragma unroll
            for (uint32_t h = 0; h < sizeof(IdxT); h++) {
                const uint4 q4 = *(const uint4 *)(Ct + m + h * (16 / sizeof(IdxT)));
                const uint32_t w[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
                for (uint32_t e = 0; e < 16 / sizeof(IdxT); e++) n16[h * (16 / sizeof(IdxT)) + e] = gw_elem<IdxT>(w, e);
            }
            uint32_t *o = out + ((size_t)z0 * side + y0) * side + x0;
#pragma unroll
            for (uint32_t k = 0; k < 4; k++) {  // k = dy + 2 dz
                const uint32_t b0 = 2 * k;
                store4(o + (size_t)(k >> 1) * side * side + (k & 1u) * side, al, lab(n16[b0]), lab(n16[b0 + 1]),
                       lab(n16[b0 + 8]), lab(n16[b0 + 9]));
            }
        }
    } else {
        for (uint32_t q = tid; q < nvox; q += nt) {
            const uint32_t x = q & (side - 1), y = (q >> s) & (side - 1), z = q >> (2 * s);
            out[q] = lab(Ct[spread6(x) | (spread6(y) << 1) | (spread6(z) << 2)]);
        }
    }
    return kStOk;
}

template <typename IdxT>
__global__ void __launch_bounds__(kGwThreads) rebuild_global(VolDev V, RecJob J, uint32_t *__restrict__ out,
                                                             const uint64_t *__restrict__ out_off,
                                                             int32_t *__restrict__ status) {
    __shared__ uint32_t red[33];
    __shared__ uint32_t sh_bad;
    __shared__ uint32_t pal_s[kGwPalSmem];
    const uint32_t i = blockIdx.x;
    const int32_t st = rebuild_global_request<IdxT>(V, J, i, out + out_off[i], red, sh_bad, pal_s);
    if (threadIdx.x == 0) status[i] = st;
}

}  // namespace

// ---------------------------------------------------------------- launchers (host)

// cudaFuncSetAttribute once per device, kernel, attribute and value: the attributes last for the process,
// and setting them again on every decode only costs host time ahead of the launches
static cudaError_t func_attr(const void *fn, cudaFuncAttribute a, int value) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int>, int> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_tuple(dev, fn, (int)a);
    const auto it = done.find(key);
    if (it != done.end() && it->second == value) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, a, value);
    if (e == cudaSuccess) done[key] = value;
    return e;
}

uint32_t rans_records_smem_bytes(uint32_t ring_words) { return 2 * kM * 4 + kRecWarps * ring_words * 2; }
uint32_t rans_records_packed_smem_bytes() { return 2 * kM * 4 + kRecWarps * kPkWarpWords * 2; }

uint32_t rebuild_smem_bytes(uint32_t N, bool wide) {
    return wide ? rb_layout<uint16_t>(N).total : rb_layout<uint8_t>(N).total;
}

// Decode requests [0, J.n) of a slice: records, then the rebuild (statuses and outputs already offset), in the
// launch shape S (rANS grid and ring depth, threads per request of the 32^3 kernels).
cudaError_t launch_decode_slice(const VolDev &V, uint32_t max_pal, const RecJob &J, uint32_t *out, const uint64_t *out_off,
                                int32_t *status, const DecodeShape &S, cudaStream_t st) {
    if (J.n == 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint32_t g = sms > 0 ? (uint32_t)sms : 1u;
    // bricks of 16^3 and smaller: streams of a few states, decoded several to a warp
    const bool packed = V.N <= 4;
    const uint32_t ring = S.ring_words == 128 || S.ring_words == 512 ? S.ring_words : 256u;
    const bool split = !packed && V.N == 5 && max_pal <= RbTraits<uint8_t>::kSent && J.lists && J.n >= kSplitMin;
    auto rk = split ? (ring == 128   ? rans_records<128, true>
                       : ring == 512 ? rans_records<512, true>
                                     : rans_records<256, true>)
                    : (ring == 128 ? rans_records<128> : ring == 512 ? rans_records<512> : rans_records<256>);
    const uint32_t smem_a = packed ? rans_records_packed_smem_bytes() : rans_records_smem_bytes(ring);
    cudaError_t e = func_attr((const void *)(packed ? rans_records_packed : rk), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_a);
    if (e == cudaSuccess && !packed)  // the largest shared-memory carve-out: up to 6 CTAs per SM
        e = func_attr((const void *)rk, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    // every counter of the slice at once: the rANS work counter, the split's list counts and work counters
    // (counter[16..21]) and the oversized-request count and work counter (counter[24..25])
    e = cudaMemsetAsync(J.counter, 0, 128, st);
    if (e != cudaSuccess) return e;
    const bool wide = max_pal > RbTraits<uint8_t>::kSent;  // uint16 palette indices
    // large mixed-LOD slices of 32^3 bricks (split): the requests listed by LOD class first, for the rANS
    // kernel's queue and for the rebuild kernels of the classes
    if (split) {
        split_lods<<<(J.n + 255) / 256, 256, 0, st>>>(J, V.N, J.lists, J.counter + 16);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const uint32_t need = (2 * J.n + kRecWarps - 1) / kRecWarps;
    const uint32_t rec_blocks = max(1u, min(S.rec_per_sm, 6u)) * g;
    {
        ProfScope ps("rans_records", st);
        if (packed) rans_records_packed<<<min(rec_blocks, need), kRecWarps * 32, smem_a, st>>>(V, J);
        else rk<<<min(rec_blocks, need), kRecWarps * 32, smem_a, st>>>(V, J);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (V.N >= 6) {  // b = 64: levels in the workspace
        ProfScope ps("rebuild", st);
        if (max_pal <= RbTraits<uint8_t>::kSent) rebuild_global<uint8_t><<<J.n, kGwThreads, 0, st>>>(V, J, out, out_off, status);
        else if (max_pal <= RbTraits<uint16_t>::kSent)
            rebuild_global<uint16_t><<<J.n, kGwThreads, 0, st>>>(V, J, out, out_off, status);
        else rebuild_global<uint32_t><<<J.n, kGwThreads, 0, st>>>(V, J, out, out_off, status);
        return cudaGetLastError();
    }
    const uint32_t smem_b = rebuild_smem_bytes(V.N, wide);
    if (wide) {
        e = func_attr((const void *)rebuild<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_b);
        if (e != cudaSuccess) return e;
        ProfScope ps("rebuild", st);
        rebuild<uint16_t><<<J.n, kRbThreads, smem_b, st>>>(V, J, out, out_off, status);
    } else {
        if (split) {  // large batch: fine and coarse requests apart (listed above)
            uint32_t *counts = J.counter + 16, *lists = J.lists;
            const uint32_t smem_m = rb_layout_part<uint8_t>(V.N, 1).total, smem_c = rb_layout_part<uint8_t>(V.N, 2).total;
            e = func_attr((const void *)rebuild_listed<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_b);
            if (e == cudaSuccess) e = func_attr((const void *)rebuild_coarse<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_c);
            if (e != cudaSuccess) return e;
            const uint32_t mt = S.medium_threads == 64 || S.medium_threads == 256 ? S.medium_threads : 128u;
            auto mk = mt == 64 ? rebuild_medium<uint8_t, 64> : mt == 256 ? rebuild_medium<uint8_t, 256>
                                                                         : rebuild_medium<uint8_t, 128>;
            e = func_attr((const void *)mk, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_m);
            if (e != cudaSuccess) return e;
            int per_m = 0;  // persistent grid: the CTAs that fit
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_m, mk, (int)mt, smem_m) != cudaSuccess || per_m < 1)
                per_m = 1;
            // LOD 0: the compact leaf layout (persistent), its oversized requests then by rebuild_listed
            const uint32_t smem_l = rb_layout_leafc<uint8_t>(V.N).total;
            const uint32_t lt = S.leafc_threads == 256 ? 256u : 128u;
            auto lk = lt == 256 ? rebuild_listed_leafc<256> : rebuild_listed_leafc<128>;
            uint32_t *n_full = J.counter + 24;  // count, then the work counter of rebuild_listed
            e = func_attr((const void *)lk, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_l);
            if (e == cudaSuccess) e = func_attr((const void *)lk, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            if (e != cudaSuccess) return e;
            int per_l = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_l, lk, (int)lt, smem_l) != cudaSuccess || per_l < 1)
                per_l = 1;
            ProfScope ps("rebuild", st);
            if (S.compact_nodes == 0) {  // every LOD 0 request in the full layout: its list goes there directly
                rebuild_listed<uint8_t><<<min(J.n, 4 * g), kRbThreads, smem_b, st>>>(V, J, out, out_off, status, lists,
                                                                                 counts, counts + 3);
            } else {
                lk<<<min(J.n, (uint32_t)per_l * g), lt, smem_l, st>>>(V, J, out, out_off, status, lists, counts,
                                                                       counts + 3, lists + 3 * J.n, n_full);
                rebuild_listed<uint8_t><<<min(J.n, 4 * g), kRbThreads, smem_b, st>>>(V, J, out, out_off, status,
                                                                                 lists + 3 * J.n, n_full, n_full + 1);
            }
            mk<<<min(J.n, (uint32_t)per_m * g), mt, smem_m, st>>>(V, J, out, out_off, status, lists + J.n, counts + 1,
                                                                  counts + 4);
            rebuild_coarse<uint8_t><<<min(J.n, 32 * g), kRbCoarseThreads, smem_c, st>>>(
                V, J, out, out_off, status, lists + 2 * J.n, counts + 2, counts + 5);
            return cudaGetLastError();
        }
        if (V.N <= 3) {
            e = func_attr((const void *)rebuild_tiny_brick<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_b);
            if (e != cudaSuccess) return e;
            ProfScope ps("rebuild", st);
            rebuild_tiny_brick<uint8_t><<<J.n, kRbTinyThreads, smem_b, st>>>(V, J, out, out_off, status);
            return cudaGetLastError();
        }
        if (V.N <= 4) {
            e = func_attr((const void *)rebuild_small_brick<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_b);
            if (e != cudaSuccess) return e;
            ProfScope ps("rebuild", st);
            rebuild_small_brick<uint8_t><<<J.n, kRbSmallThreads, smem_b, st>>>(V, J, out, out_off, status);
            return cudaGetLastError();
        }
        if (V.N == 5) {  // 32^3 bricks: the compact leaf layout, the few requests it cannot hold in rebuild_listed
            const uint32_t smem_l = rb_layout_leafc<uint8_t>(V.N).total;
            const uint32_t lt = S.leafc_threads == 256 ? 256u : 128u;
            auto lk = lt == 256 ? rebuild_leafc<256> : rebuild_leafc<128>;
            uint32_t *n_full = J.counter + 24;  // count, then the work counter of rebuild_listed
            e = func_attr((const void *)lk, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_l);
            if (e == cudaSuccess)  // the largest shared-memory carve-out: 10 CTAs per SM at 128 threads
                e = func_attr((const void *)lk, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
            if (e == cudaSuccess)
                e = func_attr((const void *)rebuild_listed<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_b);
            if (e != cudaSuccess) return e;
            ProfScope ps("rebuild", st);
            lk<<<J.n, lt, smem_l, st>>>(V, J, out, out_off, status, J.lists, n_full);
            rebuild_listed<uint8_t><<<min(J.n, 4 * g), kRbThreads, smem_b, st>>>(V, J, out, out_off, status, J.lists,
                                                                             n_full, n_full + 1);
            return cudaGetLastError();
        }
        e = func_attr((const void *)rebuild<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_b);
        if (e != cudaSuccess) return e;
        ProfScope ps("rebuild", st);
        rebuild<uint8_t><<<J.n, kRbThreads, smem_b, st>>>(V, J, out, out_off, status);
    }
    return cudaGetLastError();
}

}  // namespace csgv
