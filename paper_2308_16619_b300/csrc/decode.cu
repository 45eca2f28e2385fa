// decode.cu -- batched brick decoding (Alg. 1 of the paper) for sm_103a.
//
// One warp decodes one request (brick id, target LOD t) end to end:
//   1. rANS: the K interleaved states of a stream live in lanes 0..K-1; a
//      step decodes K symbols, lanes that need a renormalisation word take
//      consecutive words in lane order (ballot + popc), symbols go to a
//      128-entry ring in shared memory (Sec. 3.3, readings R9/R10).
//   2. Reconstruction, level by level (Alg. 1): the children of all parents
//      are first filled with the parent's label (stop-bit semantics: a
//      constant parent's sub-block takes its label); then the active
//      (non-constant) parents are taken four at a time, lane i handling
//      child i&7 of parent i>>3: the op nibble decides the child's palette
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
__device__ __forceinline__ uint32_t axis_mask(uint32_t a) { return a == 0 ? kMX : (a == 1 ? kMY : kMZ); }
// m - e_a / m + e_a on the Morton grid (caller checks the range)
__device__ __forceinline__ uint32_t mdec(uint32_t m, uint32_t ma) { return (((m & ma) - 1u) & ma) | (m & ~ma); }
__device__ __forceinline__ uint32_t minc(uint32_t m, uint32_t ma) { return (((m | ~ma) + 1u) & ma) | (m & ~ma); }

// position of the (k+1)-th set bit of x (k < popc(x)), by halving
__device__ __forceinline__ uint32_t nth_set32(uint32_t x, uint32_t k) {
    uint32_t pos = 0;
#pragma unroll
    for (uint32_t s = 16; s > 0; s >>= 1) {
        const uint32_t c = __popc(x & ((1u << s) - 1u));
        if (k >= c) {
            k -= c;
            x >>= s;
            pos += s;
        }
    }
    return pos;
}
__device__ __forceinline__ uint32_t nth_set64(uint64_t z, uint32_t k) {
    const uint32_t lo = (uint32_t)z, cl = __popc(lo);
    if (k < cl) return nth_set32(lo, k);
    return 32u + nth_set32((uint32_t)(z >> 32), k - cl);
}

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
constexpr uint32_t kChunkN = 4096;   // one 16^3 chunk of level 0
constexpr uint32_t kXfN = 256, kYfN = 512, kZfN = 1024;
constexpr uint32_t kMaskWords = 148; // const bits of levels 1..5
constexpr uint32_t kListN = 512;     // active parents of one level / chunk (uint16)
constexpr uint32_t kRingN = 128;     // symbol ring (bytes)

template <typename IdxT>
__host__ __device__ constexpr uint32_t warp_smem_bytes() {
    return ((kUpN + kChunkN + kXfN + kYfN + kZfN) * (uint32_t)sizeof(IdxT) + kMaskWords * 4 + kListN * 2 + kRingN +
            15u) & ~15u;
}

template <typename IdxT>
struct WarpMem {
    IdxT *up, *chunk, *xf, *yf, *zf;
    uint32_t *cmask;
    uint16_t *list;
    uint8_t *ring;
    __device__ explicit WarpMem(uint8_t *base) {
        up = (IdxT *)base;
        chunk = up + kUpN;
        xf = chunk + kChunkN;
        yf = xf + kXfN;
        zf = yf + kYfN;
        cmask = (uint32_t *)(zf + kZfN);
        list = (uint16_t *)(cmask + kMaskWords);
        ring = (uint8_t *)(list + kListN);
    }
};

// rANS stream state: x is this lane's state (lanes < K), the rest is uniform
struct Stream {
    const uint16_t *w;
    uint32_t n_words, pos, K, remaining, head, tail, x;
    bool bad;
};

__device__ __forceinline__ void stream_init(Stream &s, const uint16_t *w, uint32_t n_words, uint32_t n_sym,
                                            uint32_t K_max, uint32_t S_min, uint32_t lane) {
    s.w = w;
    s.n_words = n_words;
    s.remaining = n_sym;
    s.head = s.tail = 0;
    s.K = lanes_for(n_sym, K_max, S_min);
    s.bad = false;
    s.x = kL;
    s.pos = 2 * s.K;
    if (n_sym == 0) {
        s.bad = n_words != 0;
        s.pos = 0;
        return;
    }
    if (n_words < 2 * s.K) {
        s.bad = true;
        s.remaining = 0;
        return;
    }
    if (lane < s.K) s.x = (uint32_t)__ldg(w + 2 * lane) | ((uint32_t)__ldg(w + 2 * lane + 1) << 16);
}

// decode rANS steps into the ring until `want` symbols are buffered or the stream is exhausted
__device__ __forceinline__ void stream_fill(Stream &s, uint8_t *ring, const uint32_t *lut, uint32_t want,
                                            uint32_t lane) {
    while (s.tail - s.head < want && s.remaining > 0) {
        const uint32_t n = min(s.K, s.remaining);
        const bool act = lane < n;
        uint32_t sym = 0;
        if (act) {
            const uint32_t slot = s.x & (kM - 1u);
            const uint32_t e = lut[slot];
            sym = e & 15u;
            s.x = ((e >> 4) & 0x1FFFu) * (s.x >> kScaleBits) + (e >> 17);
        }
        const bool need = act && s.x < kL;
        const uint32_t m = __ballot_sync(kFull, need);
        if (need) {
            const uint32_t off = s.pos + __popc(m & lanemask_lt());
            const uint32_t wv = off < s.n_words ? (uint32_t)__ldg(s.w + off) : 0u;
            s.x = (s.x << 16) | wv;
        }
        s.pos += __popc(m);
        if (act) ring[(s.tail + lane) & (kRingN - 1)] = (uint8_t)sym;
        s.tail += n;
        s.remaining -= n;
    }
    if (s.pos > s.n_words) s.bad = true;
    __syncwarp();
}

// true iff every symbol was consumed and every state is back at L (full decode)
__device__ __forceinline__ bool stream_done_ok(const Stream &s, uint32_t lane) {
    const bool lane_ok = lane >= s.K || s.x == kL;
    return __all_sync(kFull, lane_ok) && !s.bad && s.remaining == 0 && s.head == s.tail && s.pos == s.n_words;
}

// Take the next n_ops (<= 32) operations and their delta nibbles from the
// ring.  Lane k < n_ops receives op nibble and delta of operation k.
// Returns false if the stream ran out.
__device__ __forceinline__ bool take_ops(Stream &s, const uint8_t *ring, uint32_t n_ops, uint32_t lane, uint32_t &nib,
                                         uint32_t &delta) {
    const uint32_t avail = s.tail - s.head;
    const uint32_t s_lo = lane < avail ? ring[(s.head + lane) & (kRingN - 1)] : 7u;
    const uint32_t s_hi = lane + 32 < avail ? ring[(s.head + 32 + lane) & (kRingN - 1)] : 7u;
    const uint32_t c_lo = __ballot_sync(kFull, lane < avail && (s_lo & 7u) == OP_PD);
    const uint32_t c_hi = __ballot_sync(kFull, lane + 32 < avail && (s_hi & 7u) == OP_PD);
    uint64_t cand = (uint64_t)c_lo | ((uint64_t)c_hi << 32);
    uint64_t dm = 0;  // positions holding delta nibbles
    while (cand) {
        const uint32_t i = __ffsll((long long)cand) - 1;
        cand &= cand - 1;
        if (!((dm >> i) & 1ull) && i < 63) {
            dm |= 2ull << i;
            cand &= ~(2ull << i);
        }
    }
    uint32_t pos, last_pos;
    const uint32_t low = (uint32_t)dm & ((n_ops >= 32) ? kFull : ((1u << n_ops) - 1u));
    if (low == 0) {
        pos = lane;
        last_pos = n_ops - 1;
    } else {
        const uint64_t z = ~dm;
        pos = lane < n_ops ? nth_set64(z, lane) : 0u;
        last_pos = nth_set64(z, n_ops - 1);
    }
    const uint32_t consumed = last_pos + 1 + (uint32_t)((dm >> (last_pos + 1)) & 1ull);
    const uint32_t p1 = pos + 1;
    const uint32_t a = __shfl_sync(kFull, s_lo, pos & 31), b = __shfl_sync(kFull, s_hi, pos & 31);
    const uint32_t d_lo = __shfl_sync(kFull, s_lo, p1 & 31), d_hi = __shfl_sync(kFull, s_hi, p1 & 31);
    nib = pos < 32 ? a : b;
    delta = p1 < 32 ? d_lo : d_hi;
    if (consumed > avail) return false;
    s.head += consumed;
    return true;
}

template <typename IdxT>
__device__ __forceinline__ void store_block(const IdxT *buf, uint32_t side, uint32_t *out, uint32_t pitch,
                                            uint32_t pal_reg, const uint32_t *pal, uint32_t np, bool vec,
                                            uint32_t lane) {
    auto label = [&](uint32_t idx) -> uint32_t {
        const uint32_t v = __shfl_sync(kFull, pal_reg, idx & 31);
        return np <= 32 ? v : __ldg(pal + min(idx, np - 1));
    };
    const uint32_t n = side * side * side;
    if (vec) {
        const uint32_t sh = __ffs(side) - 1;  // log2 side
        const uint32_t q = side >> 2;         // uint4 per row
        for (uint32_t base = 0; base < n / 4; base += 32) {
            const uint32_t i = min(base + lane, n / 4 - 1);
            const uint32_t x4 = i & (q - 1), y = (i >> (sh - 2)) & (side - 1), z = i >> (2 * sh - 2);
            const uint32_t m0 = morton3(4 * x4, y, z);
            uint32_t v0, v1, v2, v3;
            if (sizeof(IdxT) == 1) {
                const uint32_t a = *(const uint16_t *)(buf + m0), b = *(const uint16_t *)(buf + m0 + 8);
                v0 = a & 0xFF; v1 = a >> 8; v2 = b & 0xFF; v3 = b >> 8;
            } else {
                const uint32_t a = *(const uint32_t *)(buf + m0), b = *(const uint32_t *)(buf + m0 + 8);
                v0 = a & 0xFFFF; v1 = a >> 16; v2 = b & 0xFFFF; v3 = b >> 16;
            }
            uint4 o;
            o.x = label(v0); o.y = label(v1); o.z = label(v2); o.w = label(v3);
            if (base + lane < n / 4) __stcs((uint4 *)(out + ((size_t)z * pitch + y) * pitch + 4 * x4), o);
        }
    } else {
        for (uint32_t base = 0; base < n; base += 32) {
            const uint32_t i = base + lane;
            const uint32_t ii = i < n ? i : 0;
            const uint32_t x = ii & (side - 1), y = (ii / side) & (side - 1), z = ii / (side * side);
            const uint32_t lab = label(buf[morton3(x, y, z)]);
            if (i < n) out[((size_t)z * pitch + y) * pitch + x] = lab;
        }
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
    const bool brick_const = (n_int == 0 && n_leaf == 0);
    const bool vec_ok = ((reinterpret_cast<uintptr_t>(out) & 15u) == 0);

    // level offsets inside `up` and `cmask` (levels 1..N)
    uint32_t uoff[kMaxN + 2], woff[kMaxN + 2];
    {
        uint32_t u = 0, w = 0;
        for (uint32_t l = 1; l <= N; l++) {
            uoff[l] = u;
            woff[l] = w;
            const uint32_t c = (b >> l) * (b >> l) * (b >> l);
            u += c;
            w += c >= 32 ? c / 32 : 1;
        }
    }
    // root (level N): palette index 0 (Alg. 1 initialisation)
    if (lane == 0) {
        M.up[uoff[N]] = 0;
        M.cmask[woff[N]] = brick_const ? 1u : 0u;
    }
    __syncwarp();
    if (t == N) {
        if (lane == 0) out[0] = pal_reg;
        return kStOk;
    }

    const uint32_t K_max = V.K_max, S_min = V.S_min;
    const uint32_t *lut_int = lut_s, *lut_leaf = lut_s + kM;
    int32_t status = kStOk;
    uint32_t ip = 0;  // palette index of the last P_a (i_p)

    // one level (or chunk) of Alg. 1: parents [pp0, pp0 + npar) on level l+1 (Morton), children on level l.
    // par: parent labels (indexed pp), cm_par: parent const bits, dst: child buffer indexed (8*(pp - pp0) + c)
    // cm_dst: child const bytes (levels >= 1) or null; face lookups for the -axis targets at level 0 chunks.
    auto run_level = [&](Stream &S, const uint32_t *lut, const IdxT *par, const uint32_t *cm_par, uint32_t pp0,
                         uint32_t npar, uint32_t side_par_bits, IdxT *dst, uint8_t *cm_dst, bool leaf,
                         uint32_t chunk_o, uint32_t chunk_bits) -> bool {
        // (a) fill children with the parent's label, const bytes, list of active parents
        uint32_t n_act = 0;
        for (uint32_t g = 0; g < npar; g += 32) {
            const uint32_t k = g + lane;
            bool active = false;
            if (k < npar) {
                const uint32_t pp = pp0 + k;
                const uint32_t v = par[pp];
                const bool pc = (cm_par[pp >> 5] >> (pp & 31)) & 1u;
                active = !pc;
                if (sizeof(IdxT) == 1) {
                    *(uint64_t *)(dst + 8 * k) = 0x0101010101010101ull * v;
                } else {
                    const uint64_t r = 0x0001000100010001ull * v;
                    *(uint4 *)(dst + 8 * k) = make_uint4((uint32_t)r, (uint32_t)(r >> 32), (uint32_t)r,
                                                         (uint32_t)(r >> 32));
                }
                if (cm_dst) cm_dst[k] = pc ? 0xFF : 0x00;
            }
            const uint32_t am = __ballot_sync(kFull, active);
            if (active) M.list[n_act + __popc(am & lanemask_lt())] = (uint16_t)k;
            n_act += __popc(am);
        }
        __syncwarp();
        // (b) decode the active parents' children, four parents per step
        const uint32_t sent = T::kSent;
        const uint32_t cmask_all = (1u << (3 * (side_par_bits + 1))) - 1u;  // Morton bits of the child level
        for (uint32_t r0 = 0; r0 < n_act; r0 += 4) {
            const uint32_t npr = min(4u, n_act - r0);
            const uint32_t n_ops = 8 * npr;
            stream_fill(S, M.ring, lut, 2 * n_ops, lane);
            uint32_t nib, delta;
            if (!take_ops(S, M.ring, n_ops, lane, nib, delta)) return false;
            const bool is_op = lane < n_ops;
            const uint32_t op = nib & 7u, stop = nib >> 3;
            // palette index bookkeeping: i_p moves on P_a only (R3)
            const uint32_t pam = __ballot_sync(kFull, is_op && op == OP_PA);
            const uint32_t ipb = ip + __popc(pam & lanemask_lt());
            ip += __popc(pam);
            const uint32_t k = M.list[r0 + (lane >> 3)];  // parent (relative to pp0)
            const uint32_t c = lane & 7u;
            const uint32_t pp = pp0 + k;       // parent Morton code on its level
            const uint32_t q = 8 * k + c;      // child index into dst
            bool bad = false;
            uint32_t v = 0;
            if (is_op) {
                if (op == OP_RP) {
                    v = par[pp];
                } else if (op <= OP_RZ) {
                    const uint32_t a = op - OP_RX;
                    const uint32_t ma = axis_mask(a);
                    if ((c >> a) & 1u) {
                        // +axis: the neighbour is later in Z-order, use its parent (R4)
                        const uint32_t pm = ma & ((1u << (3 * side_par_bits)) - 1u);
                        const uint32_t gp = leaf ? (pp | (chunk_o << (3 * side_par_bits))) : pp;
                        const uint32_t gma = leaf ? (ma & ((1u << (3 * (side_par_bits + chunk_bits))) - 1u)) : pm;
                        if ((gp & gma) == gma) {
                            bad = true;  // outside the brick
                        } else {
                            const uint32_t np_ = minc(gp, ma);
                            v = par[np_];
                        }
                    } else {
                        // -axis: same level, earlier in Z-order; resolved below
                        const uint32_t qa = q & ma & cmask_all;
                        const bool chunk_edge = leaf && qa == 0;
                        if (chunk_edge && !((chunk_o >> a) & 1u)) bad = true;  // brick boundary
                        if (!leaf && qa == 0) bad = true;
                        v = sent + a;
                    }
                } else if (op == OP_P0) {
                    v = ipb;
                } else if (op == OP_PD) {
                    if (ipb < 1 + delta) bad = true;
                    v = ipb - 1 - delta;
                } else if (op == OP_PA) {
                    v = ipb + 1;
                    if (v >= np) bad = true;
                } else {
                    bad = true;
                }
                if (leaf && stop) bad = true;
                if (bad) v = 0;
                dst[q] = (IdxT)v;
            }
            // stop bits of the children of each parent: one byte per parent
            if (cm_dst) {
                const uint32_t sm = __ballot_sync(kFull, is_op && stop);
                if (is_op && c == 0) cm_dst[k] = (uint8_t)(sm >> (lane & ~7u));
            }
            if (__any_sync(kFull, bad)) return false;
            __syncwarp();
            // resolve same-level references (chains of <= 3 hops)
            if (is_op && v >= sent) {
                uint32_t cur = q, a = v - sent, w = 0;
                for (int hop = 0; hop < 4; hop++) {
                    const uint32_t ma = axis_mask(a);
                    if (leaf && (cur & ma & cmask_all) == 0) {
                        // crosses into the previous chunk: its face holds final labels
                        const uint32_t cx = chunk_o & 1, cy = (chunk_o >> 1) & 1, cz = chunk_o >> 2;
                        uint32_t x = 0, y = 0, z = 0;
                        for (uint32_t bit = 0; bit < 4; bit++) {
                            x |= ((cur >> (3 * bit)) & 1u) << bit;
                            y |= ((cur >> (3 * bit + 1)) & 1u) << bit;
                            z |= ((cur >> (3 * bit + 2)) & 1u) << bit;
                        }
                        if (a == 0) w = M.xf[y + 16 * z];
                        else if (a == 1) w = M.yf[(cx * 16 + x) + 32 * z];
                        else w = M.zf[(cx * 16 + x) + 32 * (cy * 16 + y)];
                        (void)cz;
                        break;
                    }
                    cur = mdec(cur, ma);
                    w = dst[cur];
                    if (w < sent) break;
                    a = w - sent;
                }
                dst[q] = (IdxT)w;
            }
            __syncwarp();
        }
        return true;
    };

    // interior levels N-1 .. max(t,1)
    Stream S;
    stream_init(S, V.int_words + V.int_off[id], (uint32_t)(V.int_off[id + 1] - V.int_off[id]), n_int, K_max, S_min,
                lane);
    if (S.bad) return kStCorrupt;
    const uint32_t lmin = t > 0 ? t : 1u;
    for (uint32_t l = N - 1; l >= lmin && l < N; l--) {
        const uint32_t npar = (b >> (l + 1)) * (b >> (l + 1)) * (b >> (l + 1));
        const uint32_t side_par_bits = N - (l + 1);
        IdxT *dst = M.up + uoff[l];
        if (!run_level(S, lut_int, M.up + uoff[l + 1], M.cmask + woff[l + 1], 0, npar, side_par_bits, dst,
                       (uint8_t *)(M.cmask + woff[l]), false, 0, 0))
            return kStCorrupt;
    }
    if (t >= 1) {
        if (t == 1 && !stream_done_ok(S, lane)) return kStCorrupt;
        const uint32_t side = b >> t;
        store_block<IdxT>(M.up + uoff[t], side, out, side, pal_reg, pal, np, vec_ok && side >= 4, lane);
        return status;
    }
    if (!stream_done_ok(S, lane)) return kStCorrupt;

    // leaf level in chunks of side min(b, 16)
    Stream Lf;
    stream_init(Lf, V.leaf_words + V.leaf_off[id], (uint32_t)(V.leaf_off[id + 1] - V.leaf_off[id]), n_leaf, K_max,
                S_min, lane);
    if (Lf.bad) return kStCorrupt;
    const uint32_t cside = b < 16 ? b : 16u;
    const uint32_t cbits = N - (b < 16 ? N : 4u);  // chunks per axis = 2^cbits
    const uint32_t n_chunks = 1u << (3 * cbits);
    const uint32_t par_per_chunk = (cside / 2) * (cside / 2) * (cside / 2);
    const uint32_t side_par_bits = (b < 16 ? N : 4u) - 1;  // log2 of parent-chunk side
    const IdxT *l1 = M.up + uoff[1];
    const uint32_t *cm1 = M.cmask + woff[1];
    for (uint32_t o = 0; o < n_chunks; o++) {
        if (!run_level(Lf, lut_leaf, l1, cm1, o * par_per_chunk, par_per_chunk, side_par_bits, M.chunk, nullptr,
                       true, o, cbits))
            return kStCorrupt;
        const uint32_t ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
        uint32_t *cout = out + ((size_t)(oz * cside) * b + oy * cside) * b + ox * cside;
        store_block<IdxT>(M.chunk, cside, cout, b, pal_reg, pal, np, vec_ok && cside >= 4, lane);
        if (n_chunks > 1) {
            // keep the faces later chunks may reference (-x, -y, -z neighbours)
            for (uint32_t i = lane; i < 256; i += 32) {
                const uint32_t u = i & 15, v = i >> 4;
                if (!ox) M.xf[u + 16 * v] = M.chunk[morton3(15, u, v)];
                if (!oy) M.yf[(ox * 16 + u) + 32 * v] = M.chunk[morton3(u, 15, v)];
                if (!oz) M.zf[(ox * 16 + u) + 32 * (oy * 16 + v)] = M.chunk[morton3(u, v, 15)];
            }
        }
        __syncwarp();
    }
    if (!stream_done_ok(Lf, lane)) return kStCorrupt;
    return status;
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
