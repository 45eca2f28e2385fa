// decode.cu -- batched brick decoding (Alg. 1 of the paper) for sm_103a.
//
// One warp decodes one request (brick id, target LOD t) end to end:
//   1. rANS: the K interleaved states of a stream live in lanes 0..K-1; a
//      step decodes K symbols, lanes that need a renormalisation word take
//      consecutive words in lane order (ballot + popc) from a window of the
//      stream staged in shared memory by 16-byte loads (Sec. 3.3, readings
//      R9/R10).  Each delta nibble is folded into its P_delta op, so the
//      step appends one op record per child to a ring in shared memory.
//   2. Reconstruction, level by level (Alg. 1): the children of all parents
//      are first filled with the parent's label (stop-bit semantics: a
//      constant parent's sub-block takes its label); then the active
//      (non-constant) parents are taken four at a time, lane i handling
//      child i&7 of parent i>>3: the op record decides the child's palette
//      index.  Neighbour reuse toward -axis reads the same level (earlier in
//      Z-order); chains of such references are at most 3 long (each hop sets
//      one more child bit) and are resolved by pointer chasing inside the
//      step.  Toward +axis the neighbour's parent is read (reading R4).
//   3. Labels are stored as palette[index] in x-fastest order with 16-byte
//      vector stores.
// Palette indices, not labels, are kept in shared memory (uint8 when every
// palette has <= 253 entries, else uint16).  For b = 32 the leaf level is
// processed in eight 16^3 chunks in Z-order; the -x/-y/-z faces of finished
// chunks are kept for later chunks' neighbour references.
//
// The persistent kernel takes requests from a global work counter (atomic
// add per warp); the plain kernel decodes one request per launch.
#include "csgv_internal.cuh"

namespace csgv {

namespace {

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Morton code helpers for up to 5 bits per axis (x at bit 0, reading R5)
__device__ __forceinline__ uint32_t spread5(uint32_t v) {
    return (v & 1u) | ((v & 2u) << 2) | ((v & 4u) << 4) | ((v & 8u) << 6) | ((v & 16u) << 8);
}
__device__ __forceinline__ uint32_t morton3(uint32_t x, uint32_t y, uint32_t z) {
    return spread5(x) | (spread5(y) << 1) | (spread5(z) << 2);
}
// m - e_a / m + e_a on the Morton grid (caller checks the range)
__device__ __forceinline__ uint32_t mdec(uint32_t m, uint32_t ma) { return (((m & ma) - 1u) & ma) | (m & ~ma); }
__device__ __forceinline__ uint32_t minc(uint32_t m, uint32_t ma) { return (((m | ~ma) + 1u) & ma) | (m & ~ma); }

template <typename IdxT>
struct Traits;
template <>
struct Traits<uint8_t> {
    static constexpr uint32_t kSent = 0xFDu;  // 0xFD,0xFE,0xFF: unresolved R_x-, R_y-, R_z-
    static constexpr uint32_t kMaxPal = 0xFDu;
};
template <>
struct Traits<uint16_t> {
    static constexpr uint32_t kSent = 0xFFFDu;
    static constexpr uint32_t kMaxPal = 0xFFFDu;
};

// shared-memory layout of one warp (entries of IdxT unless noted)
constexpr uint32_t kUpN = 4688;      // levels 1..5 of a 32^3 brick: 4096+512+64+8+1 = 4681
constexpr uint32_t kChunkN = 4096;   // one 16^3 chunk of level 0 (x fastest)
constexpr uint32_t kXfN = 256, kYfN = 512, kZfN = 1024;  // faces of finished chunks toward -x, -y, -z
constexpr uint32_t kMaskWords = 148; // const bits of levels 1..5
constexpr uint32_t kGroup = 64;      // parents per list (uint32 entries: parent | block base << 16)
constexpr uint32_t kQueueN = 64;     // queued children whose op is not R_p (two words each)
constexpr uint32_t kOpsN = 256;      // op ring (bytes: op | stop<<3 | delta<<4)
constexpr uint32_t kWinWords = 256;  // staged stream words (uint16)

template <typename IdxT>
__host__ __device__ constexpr uint32_t warp_smem_bytes() {
    return ((kUpN + kChunkN + kXfN + kYfN + kZfN) * (uint32_t)sizeof(IdxT) + kMaskWords * 4 + kGroup * 4 +
            kQueueN * 8 + kWinWords * 2 + kOpsN + 15u) & ~15u;
}

template <typename IdxT>
struct WarpMem {
    IdxT *up, *chunk, *xf, *yf, *zf;
    uint32_t *cmask, *list;
    uint2 *queue;
    uint16_t *win;
    uint8_t *ops;
    __device__ explicit WarpMem(uint8_t *base) {
        up = (IdxT *)base;
        chunk = up + kUpN;
        xf = chunk + kChunkN;
        yf = xf + kXfN;
        zf = yf + kYfN;
        cmask = (uint32_t *)(zf + kZfN);  // 16-byte aligned: the IdxT arrays above total a multiple of 16 bytes
        queue = (uint2 *)(cmask + kMaskWords);
        win = (uint16_t *)(queue + kQueueN);
        list = (uint32_t *)(win + kWinWords);
        ops = (uint8_t *)(list + kGroup);
    }
};

// offset of level l (1..N) in `up`, and of its const bits in `cmask` (words)
__device__ __forceinline__ uint32_t up_off(uint32_t N, uint32_t l) {
    uint32_t u = 0;
#pragma unroll
    for (uint32_t k = 1; k <= (uint32_t)kMaxN; k++)
        if (k < l) u += 1u << (3 * (N - k));
    return u;
}
__device__ __forceinline__ uint32_t mask_off(uint32_t N, uint32_t l) {
    uint32_t w = 0;
#pragma unroll
    for (uint32_t k = 1; k <= (uint32_t)kMaxN; k++)
        if (k < l) w += (N - k >= 2) ? (1u << (3 * (N - k) - 5)) : 1u;
    return w;
}

// rANS stream of one brick: x is this lane's state (lanes < K), the rest is uniform.
// Decoded symbols are folded into op records (a P_delta carries its delta) in the op ring.
struct Stream {
    const uint16_t *w;     // stream words in global memory
    uint32_t n_words, pos, K, remaining, x;
    int32_t wb;            // absolute word index held in win[0] (may be negative: alignment slack)
    uint32_t wn;           // valid words in the window
    uint32_t stage_at;     // restage once pos passes this (a step reads at most 32 words)
    uint32_t ohead, otail, pend;  // op ring; pend = 1: op otail-1 still waits for its delta
    bool bad;
};

// stage stream words from s.pos into the window with 16-byte loads (aligned down)
__device__ __forceinline__ void stage(Stream &s, uint16_t *win, uint32_t lane) {
    const uintptr_t g = reinterpret_cast<uintptr_t>(s.w + s.pos);
    const uintptr_t g0 = g & ~(uintptr_t)15;
    const uintptr_t gend = reinterpret_cast<uintptr_t>(s.w + s.n_words);
    for (uint32_t c = lane; c < kWinWords / 8; c += 32) {
        const uintptr_t a = g0 + 16 * (uintptr_t)c;
        if (a < gend) reinterpret_cast<uint4 *>(win)[c] = __ldg(reinterpret_cast<const uint4 *>(a));
    }
    s.wb = (int32_t)s.pos - (int32_t)((g - g0) >> 1);
    s.wn = min(kWinWords, (uint32_t)((int32_t)s.n_words - s.wb));
    const uint32_t end = (uint32_t)(s.wb + (int32_t)s.wn);
    s.stage_at = end < s.n_words ? end - 32 : 0xFFFFFFFFu;
    __syncwarp();
}

__device__ __forceinline__ void stream_init(Stream &s, uint16_t *win, const uint16_t *w, uint32_t n_words,
                                            uint32_t n_sym, uint32_t K_max, uint32_t S_min, uint32_t lane) {
    s.w = w;
    s.n_words = n_words;
    s.remaining = n_sym;
    s.K = lanes_for(n_sym, K_max, S_min);
    s.bad = false;
    s.x = kL;
    s.pos = 0;
    s.ohead = s.otail = s.pend = 0;
    s.wb = 0;
    s.wn = 0;
    s.stage_at = 0xFFFFFFFFu;
    if (n_sym == 0) {
        s.bad = n_words != 0;
        return;
    }
    if (n_words < 2 * s.K) {
        s.bad = true;
        s.remaining = 0;
        return;
    }
    stage(s, win, lane);
    if (lane < s.K) s.x = (uint32_t)win[2 * lane - s.wb] | ((uint32_t)win[2 * lane + 1 - s.wb] << 16);
    s.pos = 2 * s.K;
}

// decode rANS steps until `want` complete op records are waiting or the stream is exhausted
__device__ __forceinline__ void produce(Stream &s, uint8_t *ops, uint16_t *win, const uint32_t *lut, uint32_t want,
                                        uint32_t lane) {
    const uint32_t lt = lanemask_lt();
    uint32_t x = s.x, pos = s.pos, otail = s.otail, remaining = s.remaining, pend = s.pend;
    const uint32_t ohead = s.ohead, K = s.K, last = s.n_words - 1;  // K > 0 and n_words >= 2K whenever remaining > 0
    while (otail - ohead - pend < want && remaining > 0) {
        if (pos > s.stage_at) {
            if (pos > s.n_words) {  // corrupt: the words ran out
                s.bad = true;
                break;
            }
            s.pos = pos;
            stage(s, win, lane);
        }
        const uint32_t n = min(K, remaining);
        const bool act = lane < n;
        // every lane runs the step (branch-free); lanes past n keep their state
        const uint32_t e = lut[x & (kM - 1u)];
        const uint32_t sym = e & 15u;
        const uint32_t xn = ((e >> 4) & 0x1FFFu) * (x >> kScaleBits) + (e >> 17);
        const bool need = act && xn < kL;
        const uint32_t m = __ballot_sync(kFull, need);
        const uint32_t off = min(pos + __popc(m & lt), last);
        const uint32_t wv = win[min(max((int32_t)off - s.wb, 0), (int32_t)kWinWords - 1)];  // in-window for every lane
        x = act ? (need ? ((xn << 16) | wv) : xn) : x;
        pos += __popc(m);
        remaining -= n;
        uint32_t cand = __ballot_sync(kFull, act && (sym & 7u) == OP_PD);
        if ((cand | pend) == 0) {
            // common case: every symbol of the step is an op
            if (act) ops[(otail + lane) & (kOpsN - 1)] = (uint8_t)sym;
            otail += n;
            continue;
        }
        // which symbols are delta nibbles: the one after each P_delta op
        uint64_t dm = pend;  // bit i: symbol i of this step is a delta
        cand &= ~(uint32_t)dm;
        while (cand) {
            const uint32_t i = __ffs(cand) - 1;
            cand &= cand - 1;
            if (!((dm >> i) & 1ull)) {
                dm |= 2ull << i;
                cand &= ~(uint32_t)(2ull << i);
            }
        }
        const uint32_t nxt = __shfl_down_sync(kFull, sym, 1);
        if (pend && lane == 0) ops[(otail - 1) & (kOpsN - 1)] |= (uint8_t)(sym << 4);
        const uint32_t actm = n >= 32 ? kFull : ((1u << n) - 1u);
        const uint32_t opm = actm & ~(uint32_t)dm;
        if ((opm >> lane) & 1u) {
            const bool pd = (sym & 7u) == OP_PD && lane + 1 < n;
            ops[(otail + __popc(opm & lt)) & (kOpsN - 1)] = (uint8_t)(sym | (pd ? nxt << 4 : 0u));
        }
        otail += __popc(opm);
        pend = (uint32_t)((dm >> n) & 1ull);
    }
    s.x = x;
    s.pos = pos;
    s.otail = otail;
    s.remaining = remaining;
    s.pend = pend;
    if (pos > s.n_words) s.bad = true;
    __syncwarp();
}

// true iff every symbol was decoded and consumed and every state is back at L (full decode)
__device__ __forceinline__ bool stream_done_ok(const Stream &s, uint32_t lane) {
    const bool lane_ok = lane >= s.K || s.x == kL;
    return __all_sync(kFull, lane_ok) && !s.bad && s.remaining == 0 && s.ohead == s.otail && !s.pend &&
           s.pos == s.n_words;
}

// take n_ops op records from the ring (lane k < n_ops gets record k); false if the stream ran out
__device__ __forceinline__ bool take_ops(Stream &s, const uint8_t *ops, uint32_t n_ops, uint32_t lane, uint32_t &o) {
    if (s.otail - s.ohead - s.pend < n_ops) return false;
    o = lane < n_ops ? (uint32_t)ops[(s.ohead + lane) & (kOpsN - 1)] : 0u;
    s.ohead += n_ops;
    return true;
}

// labels of 4 indices, from the palette held one entry per lane (kRegPal) or from global memory
template <bool kRegPal>
__device__ __forceinline__ uint4 labels4(uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3, uint32_t pal_reg,
                                         const uint32_t *pal, uint32_t np) {
    uint4 o;
    if (kRegPal) {
        o.x = __shfl_sync(kFull, pal_reg, v0 & 31);
        o.y = __shfl_sync(kFull, pal_reg, v1 & 31);
        o.z = __shfl_sync(kFull, pal_reg, v2 & 31);
        o.w = __shfl_sync(kFull, pal_reg, v3 & 31);
    } else {
        o.x = __ldg(pal + min(v0, np - 1));
        o.y = __ldg(pal + min(v1, np - 1));
        o.z = __ldg(pal + min(v2, np - 1));
        o.w = __ldg(pal + min(v3, np - 1));
    }
    return o;
}

// Store a level held in Morton order (side <= 16) as x-fastest labels with row pitch `pitch`.
template <typename IdxT, bool kRegPal>
__device__ __forceinline__ void store_morton_impl(const IdxT *buf, uint32_t side, uint32_t *out, uint32_t pitch,
                                                  uint32_t pal_reg, const uint32_t *pal, uint32_t np, bool vec,
                                                  uint32_t lane) {
    const uint32_t n = side * side * side;
    if (vec && side >= 4) {
        const uint32_t sh = __ffs(side) - 1;
        const uint32_t x4 = lane & ((side >> 2) - 1);
        const uint32_t sx = spread5(4 * x4);
        for (uint32_t base = 0; base < n / 4; base += 32) {
            const uint32_t i = min(base + lane, n / 4 - 1);
            const uint32_t y = (i >> (sh - 2)) & (side - 1), z = i >> (2 * sh - 2);
            const uint32_t m0 = sx | (spread5(y) << 1) | (spread5(z) << 2);
            uint32_t v0, v1, v2, v3;
            if (sizeof(IdxT) == 1) {
                const uint32_t a = *(const uint16_t *)(buf + m0), b = *(const uint16_t *)(buf + m0 + 8);
                v0 = a & 0xFF; v1 = a >> 8; v2 = b & 0xFF; v3 = b >> 8;
            } else {
                const uint32_t a = *(const uint32_t *)(buf + m0), b = *(const uint32_t *)(buf + m0 + 8);
                v0 = a & 0xFFFF; v1 = a >> 16; v2 = b & 0xFFFF; v3 = b >> 16;
            }
            const uint4 o = labels4<kRegPal>(v0, v1, v2, v3, pal_reg, pal, np);
            if (base + lane < n / 4) __stcs((uint4 *)(out + ((size_t)z * pitch + y) * pitch + 4 * x4), o);
        }
    } else {
        for (uint32_t base = 0; base < n; base += 32) {
            const uint32_t i = base + lane;
            const uint32_t ii = i < n ? i : 0;
            const uint32_t x = ii & (side - 1), y = (ii / side) & (side - 1), z = ii / (side * side);
            const uint32_t v = buf[morton3(x, y, z)];
            const uint32_t lab = kRegPal ? __shfl_sync(kFull, pal_reg, v & 31) : __ldg(pal + min(v, np - 1));
            if (i < n) out[((size_t)z * pitch + y) * pitch + x] = lab;
        }
    }
}

// Store a chunk held x-fastest (side cs = 2^ls) as labels with row pitch `pitch`.
template <typename IdxT, bool kRegPal>
__device__ __forceinline__ void store_linear_impl(const IdxT *buf, uint32_t cs, uint32_t ls, uint32_t *out,
                                                  uint32_t pitch, uint32_t pal_reg, const uint32_t *pal, uint32_t np,
                                                  bool vec, uint32_t lane) {
    const uint32_t n = cs * cs * cs;
    if (vec && cs >= 4) {
        for (uint32_t base = 0; base < n / 4; base += 32) {
            const uint32_t lin = 4 * min(base + lane, n / 4 - 1);
            const uint32_t x = lin & (cs - 1), y = (lin >> ls) & (cs - 1), z = lin >> (2 * ls);
            uint32_t v0, v1, v2, v3;
            if (sizeof(IdxT) == 1) {
                const uint32_t a = *(const uint32_t *)(buf + lin);
                v0 = a & 0xFF; v1 = (a >> 8) & 0xFF; v2 = (a >> 16) & 0xFF; v3 = a >> 24;
            } else {
                const uint2 a = *(const uint2 *)(buf + lin);
                v0 = a.x & 0xFFFF; v1 = a.x >> 16; v2 = a.y & 0xFFFF; v3 = a.y >> 16;
            }
            const uint4 o = labels4<kRegPal>(v0, v1, v2, v3, pal_reg, pal, np);
            if (base + lane < n / 4) __stcs((uint4 *)(out + ((size_t)z * pitch + y) * pitch + x), o);
        }
    } else {
        for (uint32_t base = 0; base < n; base += 32) {
            const uint32_t i = base + lane;
            const uint32_t ii = i < n ? i : 0;
            const uint32_t x = ii & (cs - 1), y = (ii >> ls) & (cs - 1), z = ii >> (2 * ls);
            const uint32_t v = buf[ii];
            const uint32_t lab = kRegPal ? __shfl_sync(kFull, pal_reg, v & 31) : __ldg(pal + min(v, np - 1));
            if (i < n) out[((size_t)z * pitch + y) * pitch + x] = lab;
        }
    }
}

// every voxel of a (side^3, pitch) block gets one label
__device__ __forceinline__ void store_const(uint32_t label, uint32_t side, uint32_t *out, bool vec, uint32_t lane) {
    const uint32_t n = side * side * side;
    if (vec && side >= 4) {
        const uint4 o = make_uint4(label, label, label, label);
        for (uint32_t i = lane; i < n / 4; i += 32) __stcs((uint4 *)out + i, o);
    } else {
        for (uint32_t i = lane; i < n; i += 32) out[i] = label;
    }
}

// Decode one request into out (already offset).  Returns a status code.
template <typename IdxT>
__device__ int32_t decode_request(const VolDev &V, const uint32_t *lut_s, WarpMem<IdxT> &M, uint32_t id, uint32_t t,
                                  uint32_t *out, uint32_t lane) {
    typedef Traits<IdxT> T;
    const uint32_t N = V.N;
    if (id >= V.n_bricks || t > N) return kStRange;
    const uint32_t b = 1u << N;
    const uint64_t p0 = V.pal_off[id];
    const uint32_t np = (uint32_t)(V.pal_off[id + 1] - p0);
    const uint32_t *pal = V.pal + p0;
    const uint32_t n_int = V.n_int_sym[id], n_leaf = V.n_leaf_sym[id];
    if (np == 0 || np > T::kMaxPal) return kStCorrupt;
    const uint32_t pal_reg = lane < np ? __ldg(pal + lane) : 0u;
    const bool vec_ok = ((reinterpret_cast<uintptr_t>(out) & 15u) == 0);
    const bool reg_pal = np <= 32;

    // homogeneous brick: no symbols, every LOD is palette[0] (reading R2)
    if (n_int == 0 && n_leaf == 0) {
        if (V.int_off[id + 1] != V.int_off[id] || V.leaf_off[id + 1] != V.leaf_off[id]) return kStCorrupt;
        store_const(__shfl_sync(kFull, pal_reg, 0), b >> t, out, vec_ok, lane);
        return kStOk;
    }
    // root (level N): palette index 0 (Alg. 1 initialisation), not constant
    if (lane == 0) {
        M.up[up_off(N, N)] = 0;
        M.cmask[mask_off(N, N)] = 0u;
    }
    __syncwarp();
    if (t == N) {
        if (lane == 0) out[0] = pal_reg;
        return kStOk;
    }

    const uint32_t K_max = V.K_max, S_min = V.S_min;
    uint32_t ip = 0;  // palette index of the last P_a (i_p)
    const uint32_t sent = T::kSent;
    const uint32_t c = lane & 7u;

    // value of one coded child (Sec. 3.2): R_p and R_a toward +axis read the parent level (pv), R_a
    // toward -axis is left as a sentinel for the chase, palette ops index the palette (R1, R3)
    auto child_value = [&](uint32_t op, uint32_t delta, uint32_t ipb, uint32_t pv, bool plus, bool minus,
                           uint32_t a) -> uint32_t {
        if (op == OP_RP || plus) return pv;
        if (minus) return sent + a;
        if (op == OP_P0) return ipb;
        if (op == OP_PD) return ipb - 1 - delta;
        return ipb + 1;
    };

    // Children whose op is R_p already hold their parent's label after the fill, so only the other
    // children are queued (uint2: child index | op << 12 | delta << 15 | c << 19, palette index i_p |
    // parent << 16) and evaluated 32 at a time.  Queued children are evaluated in stream order, so a
    // -axis target is either final or evaluated in the same batch (resolved by the chase).
    uint32_t qhead = 0, qtail = 0;

    // ---- interior levels N-1 .. max(t,1): Morton order, all levels of the brick in `up`
    Stream S;
    stream_init(S, M.win, V.int_words + V.int_off[id], (uint32_t)(V.int_off[id + 1] - V.int_off[id]), n_int, K_max,
                S_min, lane);
    if (S.bad) return kStCorrupt;
    const uint32_t lmin = t > 0 ? t : 1u;
    for (uint32_t l = N - 1; l >= lmin && l < N; l--) {
        const uint32_t npar = 1u << (3 * (N - l - 1));
        const uint32_t pbits = npar - 1;  // parent-level Morton code bits
        const IdxT *par = M.up + up_off(N, l + 1);
        const uint32_t *cm_par = M.cmask + mask_off(N, l + 1);
        IdxT *dst = M.up + up_off(N, l);
        uint8_t *cm_dst = (uint8_t *)(M.cmask + mask_off(N, l));
        // evaluate up to 32 queued children (interior level: Morton layout)
        auto flush = [&](uint32_t cnt) -> bool {
            const bool in = lane < cnt;
            const uint2 qe = in ? M.queue[(qhead + lane) & (kQueueN - 1)] : make_uint2(0u, 0u);
            qhead += cnt;
            const uint32_t q = qe.x & 0xFFFu, op = (qe.x >> 12) & 7u, delta = (qe.x >> 15) & 15u, cc = qe.x >> 19;
            const uint32_t ipb = qe.y & 0xFFFFu, k = qe.y >> 16;
            const bool rx = op >= OP_RX && op <= OP_RZ;
            const uint32_t a = rx ? op - OP_RX : 0u;
            const uint32_t ma = kMX << a;
            const bool plus = rx && ((cc >> a) & 1u);
            const bool minus = rx && !plus;
            const bool plus_out = plus && ((k & ma & pbits) == (ma & pbits));
            const uint32_t pv = par[(plus && !plus_out) ? minc(k, ma) : k];
            const bool minus_out = minus && (q & ma & (8 * npar - 1)) == 0;
            const uint32_t v = child_value(op, delta, ipb, pv, plus, minus, a);
            const bool bad = in && (plus_out || minus_out || op == 7u || op == OP_RP ||
                                    (op == OP_PD && ipb < 1 + delta) || (op == OP_PA && ipb + 1 >= np));
            if (in) dst[q] = (IdxT)(bad ? 0u : v);
            if (__any_sync(kFull, bad)) return false;
            const bool chase = in && minus;
            if (__any_sync(kFull, chase)) {
                __syncwarp();
                // same-level references form chains of <= 3 hops (each hop sets one more child bit)
                if (chase) {
                    uint32_t cur = q, ax = a, w = 0;
                    for (int hop = 0; hop < 4; hop++) {
                        cur = mdec(cur, kMX << ax);
                        w = dst[cur];
                        if (w < sent) break;
                        ax = w - sent;
                    }
                    dst[q] = (IdxT)w;
                }
            }
            __syncwarp();
            return true;
        };
        for (uint32_t g0 = 0; g0 < npar; g0 += kGroup) {
            // (a) children take the parent's label (a constant parent keeps it); list the active parents
            uint32_t n_act = 0;
            for (uint32_t g = g0; g < g0 + kGroup && g < npar; g += 32) {
                const uint32_t k = g + lane;
                bool active = false;
                if (k < npar) {
                    const uint32_t v = par[k];
                    const bool pc = (cm_par[k >> 5] >> (k & 31)) & 1u;
                    active = !pc;
                    if (sizeof(IdxT) == 1) {
                        *(uint64_t *)(dst + 8 * k) = 0x0101010101010101ull * v;
                    } else {
                        const uint32_t r = 0x00010001u * v;
                        *(uint4 *)(dst + 8 * k) = make_uint4(r, r, r, r);
                    }
                    cm_dst[k] = pc ? 0xFF : 0x00;
                }
                const uint32_t am = __ballot_sync(kFull, active);
                if (active) M.list[n_act + __popc(am & lanemask_lt())] = k;
                n_act += __popc(am);
            }
            __syncwarp();
            // (b) read four active parents' ops (32) per step; queue the children that are not R_p
            for (uint32_t r0 = 0; r0 < n_act; r0 += 4) {
                const uint32_t n_ops = 8 * min(4u, n_act - r0);
                produce(S, M.ops, M.win, lut_s, n_ops, lane);
                uint32_t o;
                if (!take_ops(S, M.ops, n_ops, lane, o)) return kStCorrupt;
                const bool is_op = lane < n_ops;
                const uint32_t op = o & 7u;
                const uint32_t pam = __ballot_sync(kFull, is_op && op == OP_PA);
                const uint32_t ipb = ip + __popc(pam & lanemask_lt());
                ip += __popc(pam);
                const uint32_t sm = __ballot_sync(kFull, is_op && ((o >> 3) & 1u));
                const bool nr = is_op && op != OP_RP;
                const uint32_t nm = __ballot_sync(kFull, nr);
                if (is_op && (c == 0 || nr)) {
                    const uint32_t k = M.list[r0 + (lane >> 3)];
                    if (c == 0) cm_dst[k] = (uint8_t)(sm >> (lane & ~7u));
                    if (nr)
                        M.queue[(qtail + __popc(nm & lanemask_lt())) & (kQueueN - 1)] =
                            make_uint2((8 * k + c) | (op << 12) | ((o >> 4) << 15) | (c << 19), ipb | (k << 16));
                }
                qtail += __popc(nm);
                __syncwarp();
                if (qtail - qhead >= 32 && !flush(32)) return kStCorrupt;
            }
        }
        while (qtail != qhead)
            if (!flush(min(32u, qtail - qhead))) return kStCorrupt;
    }
    if (t >= 1) {
        if (t == 1 && !stream_done_ok(S, lane)) return kStCorrupt;
        const uint32_t side = b >> t;
        if (reg_pal) store_morton_impl<IdxT, true>(M.up + up_off(N, t), side, out, side, pal_reg, pal, np, vec_ok, lane);
        else store_morton_impl<IdxT, false>(M.up + up_off(N, t), side, out, side, pal_reg, pal, np, vec_ok, lane);
        return kStOk;
    }
    if (!stream_done_ok(S, lane)) return kStCorrupt;

    // ---- leaf level in chunks of side cs = min(b, 16) in Z-order, each held x-fastest in M.chunk
    Stream Lf;
    stream_init(Lf, M.win, V.leaf_words + V.leaf_off[id], (uint32_t)(V.leaf_off[id + 1] - V.leaf_off[id]), n_leaf,
                K_max, S_min, lane);
    if (Lf.bad) return kStCorrupt;
    const uint32_t ls = N < 4 ? N : 4u;             // log2 chunk side
    const uint32_t cs = 1u << ls;
    const uint32_t cbits = N - ls;                  // chunks per axis = 2^cbits (at most 2)
    const uint32_t n_chunks = 1u << (3 * cbits);
    const uint32_t npar = 1u << (3 * (ls - 1));     // L1 parents per chunk (<= 512)
    const uint32_t pbits = (1u << (3 * (N - 1))) - 1u;  // L1 Morton code bits
    const IdxT *par = M.up + up_off(N, 1);
    const uint32_t *cm_par = M.cmask + mask_off(N, 1);
    IdxT *dst = M.chunk;
    const uint32_t coff = (c & 1u) + (((c >> 1) & 1u) << ls) + ((c >> 2) << (2 * ls));  // child offset in the chunk
    for (uint32_t o = 0; o < n_chunks; o++) {
        const uint32_t pp0 = o * npar;
        const uint32_t ox = o & 1u, oy = (o >> 1) & 1u, oz = o >> 2;
        // evaluate up to 32 queued children (leaf chunk: x-fastest layout)
        auto flush = [&](uint32_t cnt) -> bool {
            const bool in = lane < cnt;
            const uint2 qe = in ? M.queue[(qhead + lane) & (kQueueN - 1)] : make_uint2(0u, 0u);
            qhead += cnt;
            const uint32_t qi = qe.x & 0xFFFu, op = (qe.x >> 12) & 7u, delta = (qe.x >> 15) & 15u, cc = qe.x >> 19;
            const uint32_t ipb = qe.y & 0xFFFFu, pp = pp0 + (qe.y >> 16);
            const bool rx = op >= OP_RX && op <= OP_RZ;
            const uint32_t a = rx ? op - OP_RX : 0u;
            const uint32_t ma = kMX << a;
            const bool plus = rx && ((cc >> a) & 1u);
            const bool minus = rx && !plus;
            const bool plus_out = plus && ((pp & ma & pbits) == (ma & pbits));
            const uint32_t pv = par[(plus && !plus_out) ? minc(pp, ma) : pp];
            const bool edge = ((qi >> (ls * a)) & (cs - 1)) == 0;
            const bool minus_out = minus && edge && !((o >> a) & 1u);
            const uint32_t v = child_value(op, delta, ipb, pv, plus, minus, a);
            const bool bad = in && (plus_out || minus_out || op == 7u || op == OP_RP ||
                                    (op == OP_PD && ipb < 1 + delta) || (op == OP_PA && ipb + 1 >= np));
            if (in) dst[qi] = (IdxT)(bad ? 0u : v);
            if (__any_sync(kFull, bad)) return false;
            const bool chase = in && minus;
            if (__any_sync(kFull, chase)) {
                __syncwarp();
                if (chase) {
                    uint32_t cur = qi, ax = a, w = 0;
                    for (int hop = 0; hop < 4; hop++) {
                        if (((cur >> (ls * ax)) & (cs - 1)) == 0) {
                            // crosses into an earlier chunk: its face holds final indices
                            const uint32_t x = cur & (cs - 1), y = (cur >> ls) & (cs - 1), z = cur >> (2 * ls);
                            if (ax == 0) w = M.xf[y + 16 * z];
                            else if (ax == 1) w = M.yf[(ox * 16 + x) + 32 * z];
                            else w = M.zf[(ox * 16 + x) + 32 * (oy * 16 + y)];
                            break;
                        }
                        cur -= 1u << (ls * ax);
                        w = dst[cur];
                        if (w < sent) break;
                        ax = w - sent;
                    }
                    dst[qi] = (IdxT)w;
                }
            }
            __syncwarp();
            return true;
        };
        for (uint32_t g0 = 0; g0 < npar; g0 += kGroup) {
            // (a) 2x2x2 blocks take the parent's label; list active parents with their block's linear base
            uint32_t n_act = 0;
            for (uint32_t g = g0; g < g0 + kGroup && g < npar; g += 32) {
                const uint32_t k = g + lane;
                bool active = false;
                uint32_t lb = 0;
                if (k < npar) {
                    const uint32_t pp = pp0 + k;
                    const uint32_t v = par[pp];
                    active = !((cm_par[pp >> 5] >> (pp & 31)) & 1u);
                    const uint32_t px = (k & 1u) | ((k >> 2) & 2u) | ((k >> 4) & 4u);
                    const uint32_t py = ((k >> 1) & 1u) | ((k >> 3) & 2u) | ((k >> 5) & 4u);
                    const uint32_t pz = ((k >> 2) & 1u) | ((k >> 4) & 2u) | ((k >> 6) & 4u);
                    lb = 2 * px + (2 * py << ls) + (2 * pz << (2 * ls));
                    if (sizeof(IdxT) == 1) {
                        const uint16_t r = (uint16_t)(0x0101u * v);
                        *(uint16_t *)(dst + lb) = r;
                        *(uint16_t *)(dst + lb + cs) = r;
                        *(uint16_t *)(dst + lb + cs * cs) = r;
                        *(uint16_t *)(dst + lb + cs + cs * cs) = r;
                    } else {
                        const uint32_t r = 0x00010001u * v;
                        *(uint32_t *)(dst + lb) = r;
                        *(uint32_t *)(dst + lb + cs) = r;
                        *(uint32_t *)(dst + lb + cs * cs) = r;
                        *(uint32_t *)(dst + lb + cs + cs * cs) = r;
                    }
                }
                const uint32_t am = __ballot_sync(kFull, active);
                if (active) M.list[n_act + __popc(am & lanemask_lt())] = k | (lb << 16);
                n_act += __popc(am);
            }
            __syncwarp();
            // (b) read four active parents' ops per step; queue the children that are not R_p
            for (uint32_t r0 = 0; r0 < n_act; r0 += 4) {
                const uint32_t n_ops = 8 * min(4u, n_act - r0);
                produce(Lf, M.ops, M.win, lut_s + kM, n_ops, lane);
                uint32_t o8;
                if (!take_ops(Lf, M.ops, n_ops, lane, o8)) return kStCorrupt;
                const bool is_op = lane < n_ops;
                const uint32_t op = o8 & 7u;
                const uint32_t pam = __ballot_sync(kFull, is_op && op == OP_PA);
                const uint32_t ipb = ip + __popc(pam & lanemask_lt());
                ip += __popc(pam);
                if (__any_sync(kFull, is_op && ((o8 >> 3) & 1u))) return kStCorrupt;  // leaf stop bits are 0
                const bool nr = is_op && op != OP_RP;
                const uint32_t nm = __ballot_sync(kFull, nr);
                if (nr) {
                    const uint32_t e = M.list[r0 + (lane >> 3)];
                    M.queue[(qtail + __popc(nm & lanemask_lt())) & (kQueueN - 1)] =
                        make_uint2(((e >> 16) + coff) | (op << 12) | ((o8 >> 4) << 15) | (c << 19),
                                   ipb | ((e & 0xFFFFu) << 16));
                }
                qtail += __popc(nm);
                __syncwarp();
                if (qtail - qhead >= 32 && !flush(32)) return kStCorrupt;
            }
        }
        while (qtail != qhead)
            if (!flush(min(32u, qtail - qhead))) return kStCorrupt;
        uint32_t *cout = out + ((size_t)(oz * cs) * b + oy * cs) * b + ox * cs;
        if (reg_pal) store_linear_impl<IdxT, true>(dst, cs, ls, cout, b, pal_reg, pal, np, vec_ok, lane);
        else store_linear_impl<IdxT, false>(dst, cs, ls, cout, b, pal_reg, pal, np, vec_ok, lane);
        if (n_chunks > 1) {
            // keep the faces later chunks may reference (-x, -y, -z neighbours)
            for (uint32_t i = lane; i < 256; i += 32) {
                const uint32_t u = i & 15, w = i >> 4;
                if (!ox) M.xf[u + 16 * w] = dst[15 + 16 * u + 256 * w];
                if (!oy) M.yf[(ox * 16 + u) + 32 * w] = dst[u + 16 * 15 + 256 * w];
                if (!oz) M.zf[(ox * 16 + u) + 32 * (oy * 16 + w)] = dst[u + 16 * w + 256 * 15];
            }
        }
        __syncwarp();
    }
    if (!stream_done_ok(Lf, lane)) return kStCorrupt;
    return kStOk;
}

template <typename IdxT>
__device__ __forceinline__ void load_lut(uint32_t *lut_s, const uint32_t *lut) {
    for (uint32_t i = threadIdx.x; i < 2 * kM / 4; i += blockDim.x)
        ((uint4 *)lut_s)[i] = __ldg((const uint4 *)lut + i);
    __syncthreads();
}

template <typename IdxT>
__global__ void __launch_bounds__(1024, 1)
    decode_persistent(VolDev V, const uint32_t *__restrict__ ids, const uint8_t *__restrict__ lods, uint32_t n,
                      uint32_t *__restrict__ out, const uint64_t *__restrict__ out_off, int32_t *__restrict__ status,
                      uint32_t *__restrict__ work) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *lut_s = (uint32_t *)smem;
    load_lut<IdxT>(lut_s, V.lut);
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpMem<IdxT> M(smem + 2 * kM * 4 + warp * warp_smem_bytes<IdxT>());
    for (;;) {
        uint32_t r = 0;
        if (lane == 0) r = atomicAdd(work, 1u);
        r = __shfl_sync(kFull, r, 0);
        if (r >= n) break;
        const int32_t st = decode_request<IdxT>(V, lut_s, M, ids[r], lods[r], out + out_off[r], lane);
        if (lane == 0) status[r] = st;
        __syncwarp();
    }
}

template <typename IdxT>
__global__ void __launch_bounds__(32, 1)
    decode_single(VolDev V, const uint32_t *__restrict__ ids, const uint8_t *__restrict__ lods, uint32_t r,
                  uint32_t *__restrict__ out, const uint64_t *__restrict__ out_off, int32_t *__restrict__ status) {
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t *lut_s = (uint32_t *)smem;
    load_lut<IdxT>(lut_s, V.lut);
    WarpMem<IdxT> M(smem + 2 * kM * 4);
    const int32_t st = decode_request<IdxT>(V, lut_s, M, ids[r], lods[r], out + out_off[r], threadIdx.x);
    if (threadIdx.x == 0) status[r] = st;
}

}  // namespace

// ---------------------------------------------------------------- launchers (host)

uint32_t decode_smem_bytes(bool wide, uint32_t warps) {
    return 2 * kM * 4 + warps * (wide ? warp_smem_bytes<uint16_t>() : warp_smem_bytes<uint8_t>());
}

cudaError_t launch_decode_persistent(const VolDev &V, bool wide, const uint32_t *ids, const uint8_t *lods, uint32_t n,
                                     uint32_t *out, const uint64_t *out_off, int32_t *status, uint32_t *work,
                                     uint32_t warps, uint32_t blocks, cudaStream_t st) {
    const uint32_t smem = decode_smem_bytes(wide, warps);
    cudaError_t e;
    if (wide) {
        e = cudaFuncSetAttribute(decode_persistent<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        decode_persistent<uint16_t><<<blocks, warps * 32, smem, st>>>(V, ids, lods, n, out, out_off, status, work);
    } else {
        e = cudaFuncSetAttribute(decode_persistent<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        decode_persistent<uint8_t><<<blocks, warps * 32, smem, st>>>(V, ids, lods, n, out, out_off, status, work);
    }
    return cudaGetLastError();
}

cudaError_t launch_decode_single(const VolDev &V, bool wide, const uint32_t *ids, const uint8_t *lods, uint32_t r,
                                 uint32_t *out, const uint64_t *out_off, int32_t *status, cudaStream_t st) {
    const uint32_t smem = decode_smem_bytes(wide, 1);
    if (wide) {
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(decode_single<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 smem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        decode_single<uint16_t><<<1, 32, smem, st>>>(V, ids, lods, r, out, out_off, status);
    } else {
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(decode_single<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 smem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        decode_single<uint8_t><<<1, 32, smem, st>>>(V, ids, lods, r, out, out_off, status);
    }
    return cudaGetLastError();
}

}  // namespace csgv
