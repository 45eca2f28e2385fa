// encode.cu -- brick encoder (Alg. 2 of the paper), frequency prepass and
// packing for sm_103a.
//
// encode_kernel: one CTA of 256 threads per brick (128 for bricks of 16^3 and smaller), specialised on the
// brick size for 32^3 and 16^3:
//   A. pyramid (Sec. 3.1): L1 from the volume (16-byte row loads for bricks
//      inside an aligned volume), L2..LN in shared memory; each node is the
//      most frequent of its 8 children, ties to the first occurrence in the
//      child array (Sec. 3.4), plus a constant-subtree flag.
//   B. the active (non-constant) parents of every level ranked in stream
//      order (level by level from the root, Morton order within a level);
//      one thread per active parent picks, for each of its 8 children, the
//      first applicable reuse operation R_p, R_x, R_y, R_z (Sec. 3.2, reading
//      R4) and writes the 8 op bytes (op | stop << 3) at 8 x its rank;
//      children no reuse fits are gathered for the palette pass.
//   C. palette pass: the gathered children in stream order, walked by one
//      warp with the last 17 palette entries in registers (lane i holds
//      palette[i_p-i]): a ballot finds P_0 (lane 0) or the smallest P_delta
//      (lanes 1..16); otherwise P_a appends the label (Sec. 3.2,
//      bestOperation order); the op byte gets the delta (delta << 4).
//   D. each stream's symbol count (its ops plus a delta nibble per P_delta,
//      reading R18); in the prepass the nibbles are counted (Sec. 3.4).
// rans_encode_kernel: one warp per stream, K interleaved states in lanes,
//   the op bytes coded from the last step down (a P_delta's delta on its op's
//   state, reading R10); renormalisation words are pushed downward from the
//   top of the scratch area so that the decoder reads them forward in lane
//   order (Sec. 3.3, readings R9/R10).
// A scan kernel turns per-brick sizes into offsets and a compaction kernel
// packs palettes and words into the volume's arrays.
#include "encode_api.cuh"

namespace csgv {

constexpr uint32_t kEncThreads = 256;
constexpr uint32_t kEncWarps = kEncThreads / 32;
constexpr uint32_t kNeedPal = 7;       // op placeholder: no reuse operation applies
constexpr uint32_t kRansEncWarps = 8;   // rans_encode_kernel: one stream per warp (8-warp CTAs spread evenly over the SMs)
constexpr uint32_t kRansEncWin = 2048;  // staged symbols per warp (bytes)

namespace {

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
// Drop the 128-byte L2 lines that lie wholly inside [lo, hi) without writing them back: scratch nobody reads
// again (the lanes of a warp take every 32nd line)
__device__ __forceinline__ void discard_l2(uintptr_t lo, uintptr_t hi, uint32_t lane) {
    const uintptr_t a0 = (lo + 127) & ~(uintptr_t)127, a1 = hi & ~(uintptr_t)127;
    for (uintptr_t a = a0 + 128 * (uintptr_t)lane; a < a1; a += 128 * 32)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(a) : "memory");
}
// 6-bit coordinate <-> every third bit of a Morton code
__device__ __forceinline__ uint32_t spread6(uint32_t v) {
    return (v & 1u) | ((v & 2u) << 2) | ((v & 4u) << 4) | ((v & 8u) << 6) | ((v & 16u) << 8) | ((v & 32u) << 10);
}
__device__ __forceinline__ uint32_t morton3(uint32_t x, uint32_t y, uint32_t z) {
    return spread6(x) | (spread6(y) << 1) | (spread6(z) << 2);
}
__device__ __forceinline__ uint32_t compact6(uint32_t m) {
    return (m & 1u) | ((m >> 2) & 2u) | ((m >> 4) & 4u) | ((m >> 6) & 8u) | ((m >> 8) & 16u) | ((m >> 10) & 32u);
}
__device__ __forceinline__ uint32_t mdec(uint32_t m, uint32_t ma) { return (((m & ma) - 1u) & ma) | (m & ~ma); }
__device__ __forceinline__ uint32_t minc(uint32_t m, uint32_t ma) { return (((m | ~ma) + 1u) & ma) | (m & ~ma); }

// Most frequent of 8 labels, ties to the first occurrence (Sec. 3.4): the distinct values are visited in
// order of first occurrence and a later one wins only with a strictly larger count.  The positions are
// visited in a fixed order (no selection of the value by index); a position already counted is skipped,
// and the walk stops once the positions left cannot outnumber the best count.
__device__ __forceinline__ uint32_t mode8(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, uint32_t w4, uint32_t w5,
                                         uint32_t w6, uint32_t w7, bool &all_equal) {
    const uint32_t w[8] = {w0, w1, w2, w3, w4, w5, w6, w7};
    uint32_t m0 = 1u;  // the positions holding w0
#pragma unroll
    for (uint32_t j = 1; j < 8; j++) m0 |= (w[j] == w0 ? 1u : 0u) << j;
    all_equal = m0 == 0xFFu;
    uint32_t rem = 0xFFu & ~m0, best = w0, bestc = __popc(m0);
#pragma unroll
    for (uint32_t c = 1; c < 8; c++) {
        if (__popc(rem) <= bestc) break;  // rem only shrinks and bestc only grows
        if ((rem >> c) & 1u) {
            const uint32_t v = w[c];
            uint32_t m = 0;
#pragma unroll
            for (uint32_t j = c; j < 8; j++) m |= (w[j] == v ? 1u : 0u) << j;
            const uint32_t cnt = __popc(m);
            if (cnt > bestc) {
                bestc = cnt;
                best = v;
            }
            rem &= ~m;
        }
    }
    return best;
}

struct Brick {
    const uint32_t *vol;
    uint64_t X, Y, Z;
    uint64_t gx0, gy0, gz0;  // brick origin
    const uint32_t *base;    // voxel (gx0, gy0, gz0)
    uint64_t sy, sz;         // element strides of y and z
    bool interior;           // no clamping needed
    __device__ __forceinline__ uint32_t at(uint32_t x, uint32_t y, uint32_t z) const {
        if (interior) return __ldg(base + x + sy * y + sz * z);
        uint64_t gx = gx0 + x, gy = gy0 + y, gz = gz0 + z;
        gx = gx < X ? gx : X - 1;
        gy = gy < Y ? gy : Y - 1;
        gz = gz < Z ? gz : Z - 1;
        return __ldg(vol + gx + X * (gy + Y * gz));
    }
};

// Working arrays of the encoder CTA: the level arrays (labels, const flags and active parents of levels 1..N)
// in shared memory, or for b = 64 (too large) in the brick's global scratch `lvl`; the scan scratch and the
// palette gather list always in shared memory.
struct EncSmem {
    uint32_t *lab;     // up_nodes labels, levels 1..N
    uint8_t *cst;      // up_nodes const flags
    uint16_t *list;    // active parents, ranked in stream order
    uint32_t *red;     // block scan scratch (64 words)
    uint2 *plist;      // children that need a palette op: (op index, label), 256 at a time
    __device__ EncSmem(uint8_t *s, const EncGeom &G, uint8_t *lvl) {
        uint8_t *L = G.lvl_bytes ? lvl : s;
        lab = (uint32_t *)L;
        cst = L + r16(G.up_nodes * 4);
        list = (uint16_t *)(cst + r16(G.up_nodes));
        red = (uint32_t *)(G.lvl_bytes ? s : (uint8_t *)list + r16(G.up_nodes * 2));
        plist = (uint2 *)(red + 64);
    }
    __host__ __device__ static uint32_t r16(uint32_t x) { return (x + 15u) & ~15u; }
};

// bytes of the level arrays of one brick
__host__ __device__ inline uint32_t enc_level_bytes(uint32_t up_nodes) {
    return EncSmem::r16(up_nodes * 4) + EncSmem::r16(up_nodes) + EncSmem::r16(up_nodes * 2);
}

__host__ __device__ inline uint32_t enc_smem_bytes(uint32_t up_nodes, bool levels_in_global) {
    return (levels_in_global ? 0u : enc_level_bytes(up_nodes)) + 64 * 4 + 256 * 8;
}

// exclusive block scan of one value per warp (warp totals in `red`), returns warp's offset and the total
template <uint32_t kW>
__device__ __forceinline__ uint32_t block_excl_warp(uint32_t *red, uint32_t warp_total, uint32_t &total) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = warp_total;
    __syncthreads();
    uint32_t off = 0, tot = 0;
    for (uint32_t w = 0; w < kW; w++) {
        const uint32_t v = red[w];
        if (w < warp) off += v;
        tot += v;
    }
    __syncthreads();
    total = tot;
    return off;
}

// offset of level l (1..N) in the level arrays (the same as EncGeom::off, without indexing a kernel parameter)
__device__ __forceinline__ uint32_t loff(uint32_t N, uint32_t l) {
    uint32_t u = 0;
#pragma unroll
    for (uint32_t k = 1; k <= (uint32_t)kMaxN; k++)
        if (k < l) u += 1u << (3 * (N - k));
    return u;
}

// label of node q (Morton) on level l of the brick
__device__ __forceinline__ uint32_t node_label(const Brick &B, const EncSmem &S, const EncGeom &G, uint32_t l,
                                               uint32_t q) {
    if (l == 0) return B.at(compact6(q), compact6(q >> 1), compact6(q >> 2));
    return S.lab[loff(G.N, l) + q];
}

// Palette operations (Sec. 3.2) of up to 32 children in stream order, one per lane (lane k < kn: child k with
// label `lab`), for warp 0 of the encoder.  The window `win` holds palette[i_p - f] in lane f (f <= 16; valid
// for f <= ip).  Returns lane k's op (P_0, P_delta | delta << 4 or P_a), writes the P_a labels to pal (if
// given) at np, np + 1, ..., and moves the window, ip and np past the chunk.
// The chunk is resolved at once: a child whose label is neither in the window nor carried by an earlier child
// of the chunk is a P_a; every other child finds its label at depth f = (the label's depth in the window, or
// the appends since the label's first child in the chunk) plus the P_a before it.  If some f exceeds 16 (appends
// in this chunk pushed a label out of the window) the chunk is walked child by child instead.  tmp: 32 words of
// shared memory.
__device__ __forceinline__ uint32_t palette_chunk(uint32_t lab, uint32_t kn, uint32_t &win, uint32_t &ip,
                                                  uint32_t &np, uint32_t *pal, uint32_t *tmp) {
    const uint32_t lane = threadIdx.x & 31;
    const bool valid = lane < kn;
    uint32_t pw = 32;  // depth of this child's label in the window (32: not in it)
#pragma unroll
    for (uint32_t f = 0; f <= 16; f++) {
        const uint32_t w = __shfl_sync(kFull, win, f);
        pw = (pw == 32 && f <= ip && w == lab) ? f : pw;
    }
    const uint32_t vmask = __ballot_sync(kFull, valid);
    const uint32_t same = __match_any_sync(kFull, lab) & vmask;
    const uint32_t first = __ffs(same) - 1;  // first child of the chunk with this label
    const bool app = valid && pw == 32 && first == lane;
    const uint32_t amask = __ballot_sync(kFull, app);
    const uint32_t a_before = __popc(amask & lanemask_lt());
    uint32_t f = 0;
    if (valid && !app) f = pw != 32 ? a_before + pw : a_before - __popc(amask & ((1u << first) - 1u)) - 1u;
    if (__ballot_sync(kFull, valid && !app && f > 16) == 0) {
        const uint32_t A = __popc(amask);
        if (pal && app) pal[np + a_before] = lab;
        if (app && A - 1u - a_before < 17u) tmp[A - 1u - a_before] = lab;
        __syncwarp();
        const uint32_t old = __shfl_sync(kFull, win, (lane - A) & 31u);
        win = lane < A ? tmp[lane & 31u] : old;
        __syncwarp();
        ip += A;
        np += A;
        return app ? OP_PA : (f == 0 ? OP_P0 : (OP_PD | ((f - 1u) << 4)));
    }
    uint32_t res = 0;
    for (uint32_t k = 0; k < kn; k++) {
        const uint32_t vk = __shfl_sync(kFull, lab, k);
        const bool match = lane <= 16 && lane <= ip && win == vk;
        const uint32_t mm = __ballot_sync(kFull, match);
        uint32_t r;
        if (mm) {
            const uint32_t fm = __ffs(mm) - 1;
            r = fm == 0 ? OP_P0 : (OP_PD | ((fm - 1) << 4));
        } else {
            r = OP_PA;
            const uint32_t up = __shfl_up_sync(kFull, win, 1);
            win = lane == 0 ? vk : up;
            if (pal && lane == 0) pal[np] = vk;
            ip += 1;
            np += 1;
        }
        res = lane == k ? r : res;
    }
    return res;
}

// Encode (or, when count != nullptr, only count the nibbles of) one brick: phases A-D.
// kT: threads per CTA (64..256); kN: the brick's N when the kernel is launched for that brick size only
// (at most 5: the level arrays in shared memory), else 0; with it the brick's geometry and every level offset
// fold to constants (encode_kernel on voronoi512 b=32: 194 M -> 163 M warp instructions, 0.279 -> 0.247 ms)
template <uint32_t kT, uint32_t kN = 0>
__device__ __forceinline__ void encode_brick(EncVol EV, EncGeom G, uint64_t brick0, uint64_t brick_stride,
                                             uint32_t n_in_batch, EncScratch SC, unsigned long long *count) {
    static_assert(kN <= 5, "bricks of 64^3 keep their level arrays in global memory");
    extern __shared__ __align__(16) uint8_t smem_raw[];
    if constexpr (kN != 0) {
        if (G.N != kN) return;  // launched for another brick size
        G.N = kN;
        G.b = 1u << kN;
        uint32_t u = 0;
#pragma unroll
        for (uint32_t l = 1; l <= kN; l++) u += 1u << (3 * (kN - l));
        G.up_nodes = u;
        G.lvl_bytes = 0;
    }
    EncSmem S(smem_raw, G, SC.lvl + (size_t)blockIdx.x * G.lvl_bytes);
    __shared__ uint32_t hist[32];
    __shared__ uint32_t sh_np;
    __shared__ uint32_t sh_npc;                 // children that need a palette op (phase B)
    __shared__ uint32_t sh_pd[2 * kEncWarps];   // P_delta ops per warp range of phase D, per stream (phase C)
    __shared__ uint32_t lvl_rank[kMaxN + 2];  // rank of the first active parent of level l; [0]: all of them
    __shared__ uint32_t lvl_sp[kMaxN + 2];    // active parents stored before level l (level 1 first)
    uint32_t n_act_total;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t slot = blockIdx.x;
    if (slot >= n_in_batch) return;
    const uint64_t id = brick0 + (uint64_t)slot * brick_stride;
    const uint32_t N = G.N, b = G.b;

    Brick B;
    B.vol = EV.vol;
    B.X = EV.dims[0]; B.Y = EV.dims[1]; B.Z = EV.dims[2];
    const uint64_t bx = id % EV.nb[0], by = (id / EV.nb[0]) % EV.nb[1], bz = id / (EV.nb[0] * EV.nb[1]);
    B.gx0 = bx * b; B.gy0 = by * b; B.gz0 = bz * b;
    B.interior = B.gx0 + b <= B.X && B.gy0 + b <= B.Y && B.gz0 + b <= B.Z;
    B.sy = B.X;
    B.sz = B.X * B.Y;
    B.base = B.vol + B.gx0 + B.X * (B.gy0 + B.Y * B.gz0);
    if (tid < 32) hist[tid] = 0;
    if (tid == 0) sh_npc = 0;
    // op bytes (op | stop<<3 | delta<<4) of every coded child in stream order, in this brick's scratch
    // (written and read by this CTA only, so plain loads after a barrier see them)
    uint8_t *ops = SC.ops + (size_t)slot * G.ops_cap;

    // ---- A. pyramid
    {
        const uint32_t h = N - 1;  // log2 of the L1 side
        const bool vec = B.interior && N >= 2 && (B.X & 3u) == 0 && (reinterpret_cast<uintptr_t>(B.vol) & 15u) == 0;
        if (vec && kT >= 256) {
            // two x-neighbouring L1 nodes per thread: four 16-byte rows (y, z) of 4 voxels.  Pairs go to threads
            // x-fastest (px = x / 4 of the brick's 32-voxel rows, then y / 2, then z / 2), so that each load of a
            // warp reads whole 128-byte rows, and the rows of a thread's next pair are loaded before the modes of
            // this pair are computed (the loads of one pair are in flight while the previous pair is reduced).
            const uint32_t npairs = 1u << (3 * h - 1);
            const uint32_t xb = h - 1;  // bits of px (pairs per L1 row)
            auto rows = [&](uint32_t i, uint4 (&q)[4]) {
                const uint32_t px = i & ((1u << xb) - 1u), y = (i >> xb) & ((1u << h) - 1u), z = i >> (xb + h);
                const uint32_t *r = B.base + B.sz * (2 * z) + B.sy * (2 * y) + 4 * px;
                q[0] = __ldg((const uint4 *)r);
                q[1] = __ldg((const uint4 *)(r + B.sy));
                q[2] = __ldg((const uint4 *)(r + B.sz));
                q[3] = __ldg((const uint4 *)(r + B.sz + B.sy));
            };
            uint4 cur[4], nxt[4];
            if (tid < npairs) rows(tid, cur);
            for (uint32_t i = tid; i < npairs; i += kT) {
                if (i + kT < npairs) rows(i + kT, nxt);
                const uint32_t px = i & ((1u << xb) - 1u), y = (i >> xb) & ((1u << h) - 1u), z = i >> (xb + h);
                bool e0, e1;
                const uint32_t m = loff(G.N, 1) + morton3(2 * px, y, z);
                S.lab[m] = mode8(cur[0].x, cur[0].y, cur[1].x, cur[1].y, cur[2].x, cur[2].y, cur[3].x, cur[3].y, e0);
                S.cst[m] = e0;
                S.lab[m + 1] = mode8(cur[0].z, cur[0].w, cur[1].z, cur[1].w, cur[2].z, cur[2].w, cur[3].z, cur[3].w, e1);
                S.cst[m + 1] = e1;
#pragma unroll
                for (int k = 0; k < 4; k++) cur[k] = nxt[k];
            }
        } else if (vec) {
            // small CTAs (bricks of 16^3 and smaller, registers bounded): Morton pairs 2i, 2i+1 per thread,
            // without the prefetch
            const uint32_t npairs = 1u << (3 * h - 1);
#pragma unroll 2
            for (uint32_t i = tid; i < npairs; i += kT) {
                const uint32_t m2 = 2 * i;
                const uint32_t x = compact6(m2), y = compact6(m2 >> 1), z = compact6(m2 >> 2);  // x even
                const uint32_t *r = B.base + B.sz * (2 * z) + B.sy * (2 * y) + 2 * x;
                const uint4 a = __ldg((const uint4 *)r), bb = __ldg((const uint4 *)(r + B.sy)),
                            c = __ldg((const uint4 *)(r + B.sz)), d = __ldg((const uint4 *)(r + B.sz + B.sy));
                bool e0, e1;
                const uint32_t m = loff(G.N, 1) + m2;
                S.lab[m] = mode8(a.x, a.y, bb.x, bb.y, c.x, c.y, d.x, d.y, e0);
                S.cst[m] = e0;
                S.lab[m + 1] = mode8(a.z, a.w, bb.z, bb.w, c.z, c.w, d.z, d.w, e1);
                S.cst[m + 1] = e1;
            }
        } else {
            const uint32_t n1 = 1u << (3 * h);
            for (uint32_t i = tid; i < n1; i += kT) {
                const uint32_t x = i & ((1u << h) - 1u), y = (i >> h) & ((1u << h) - 1u), z = i >> (2 * h);
                bool eq;
                const uint32_t m = loff(G.N, 1) + morton3(x, y, z);
                S.lab[m] = mode8(B.at(2 * x, 2 * y, 2 * z), B.at(2 * x + 1, 2 * y, 2 * z), B.at(2 * x, 2 * y + 1, 2 * z),
                                 B.at(2 * x + 1, 2 * y + 1, 2 * z), B.at(2 * x, 2 * y, 2 * z + 1),
                                 B.at(2 * x + 1, 2 * y, 2 * z + 1), B.at(2 * x, 2 * y + 1, 2 * z + 1),
                                 B.at(2 * x + 1, 2 * y + 1, 2 * z + 1), eq);
                S.cst[m] = eq;
            }
        }
        __syncthreads();
        // levels of more than 64 nodes by the whole CTA, the smaller ones by warp 0 alone (no CTA barriers)
#pragma unroll
        for (uint32_t l = 2; l <= N; l++) {
            const uint32_t nl = 1u << (3 * (N - l));
            const bool big = nl > 64;
            if (!big && warp != 0) break;
            for (uint32_t i = big ? tid : lane; i < nl; i += big ? kT : 32u) {
                const uint4 wa = *(const uint4 *)(S.lab + loff(G.N, l - 1) + 8 * i),
                            wb = *(const uint4 *)(S.lab + loff(G.N, l - 1) + 8 * i + 4);
                const uint2 cs = *(const uint2 *)(S.cst + loff(G.N, l - 1) + 8 * i);  // 8 flags, 0 or 1 each
                const bool allc = (cs.x & cs.y) == 0x01010101u;
                bool eq;
                S.lab[loff(G.N, l) + i] = mode8(wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w, eq);
                S.cst[loff(G.N, l) + i] = eq && allc;
            }
            if (big) __syncthreads();
            else __syncwarp();
        }
        __syncthreads();
    }

    // ---- B. active parents and reuse operations (Alg. 2 traversal).  The op array lists the children of the
    // active (non-constant) parents level by level from the root down, 8 per parent, parents in Morton order
    // within a level.  Ranking the active parents in that order (rank of a parent of level l = the active
    // parents of the levels above plus those before it on level l) puts its children's ops at 8r .. 8r + 7,
    // so every level is coded in one pass.  The flags are counted in their storage order (level 1 first),
    // 16 per 16-byte load, by contiguous runs of chunks per thread.
    {
        const uint32_t ne = G.up_nodes, nq = (ne + 15) >> 4, cpt = (nq + kT - 1) / kT;
        const uint32_t q0 = min(tid * cpt, nq), q1 = min(q0 + cpt, nq);
        // active (flag 0) bytes of chunk q as a 16-bit mask, bytes at or past ne excluded
        auto act_mask = [&](uint32_t q) {
            const uint4 f = *(const uint4 *)(S.cst + 16 * q);
            const uint32_t w[4] = {f.x, f.y, f.z, f.w};
            uint32_t m = 0;
#pragma unroll
            for (int k = 0; k < 4; k++) m |= (((~w[k] & 0x01010101u) * 0x00204081u) >> 21 & 15u) << (4 * k);  // byte i -> bit i
            const uint32_t valid = 16 * q + 16 <= ne ? 0xFFFFu : (1u << (ne - 16 * q)) - 1u;
            return m & valid;
        };
        // one brick size: a thread's chunk masks are computed once and kept in registers
        constexpr uint32_t kCpt = kN ? ((((1u << (3 * kN)) - 1u) / 7u + 15u) / 16u + kT - 1u) / kT : 1u;
        uint32_t mk[kCpt];
        uint32_t cnt = 0;
        if constexpr (kN != 0) {
#pragma unroll
            for (uint32_t j = 0; j < kCpt; j++) {
                mk[j] = q0 + j < q1 ? act_mask(q0 + j) : 0u;
                cnt += __popc(mk[j]);
            }
        } else {
            for (uint32_t q = q0; q < q1; q++) cnt += __popc(act_mask(q));
        }
        uint32_t incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t u = __shfl_up_sync(kFull, incl, d);
            if (lane >= (uint32_t)d) incl += u;
        }
        uint32_t n_act_all;
        const uint32_t wb = block_excl_warp<kT / 32>(S.red, __shfl_sync(kFull, incl, 31), n_act_all);
        const uint32_t base = wb + incl - cnt;  // active flags before this thread's first chunk
        // level starts in storage order (levels 2..N); lvl_sp[l]: active flags before level l's first node
        uint32_t bnd[kMaxN + 1];
#pragma unroll
        for (uint32_t l = 1; l <= (uint32_t)kMaxN; l++) bnd[l] = l <= N ? loff(G.N, l) : ne;
        {
            uint32_t run = base;
#pragma unroll
            for (uint32_t j = 0; j < (kN ? kCpt : q1 - q0); j++) {
                const uint32_t q = q0 + j;
                if (q >= q1) break;
                const uint32_t m = kN ? mk[j] : act_mask(q);
#pragma unroll
                for (uint32_t l = 2; l <= (uint32_t)kMaxN; l++)
                    if (l <= N && bnd[l] >= 16 * q && bnd[l] < 16 * q + 16)
                        lvl_sp[l] = run + __popc(m & ((1u << (bnd[l] - 16 * q)) - 1u));
                run += __popc(m);
            }
        }
        if (tid == 0) {
            lvl_sp[1] = 0;
            lvl_sp[N + 1] = n_act_all;
        }
        __syncthreads();
        // stream rank of each active parent: S.list[rank] = its index within its level
        uint32_t run = base;
#pragma unroll
        for (uint32_t j = 0; j < (kN ? kCpt : q1 - q0); j++) {
            const uint32_t q = q0 + j;
            if (q >= q1) break;
            uint32_t m = kN ? mk[j] : act_mask(q);
            if (kN) {  // a chunk inside one level (all but the chunks where a level starts past their first node)
                uint32_t lq = 1, lb = 0;
                bool inside = false;
#pragma unroll
                for (uint32_t L = 2; L <= (uint32_t)kMaxN; L++) {
                    if (L <= N && 16 * q >= bnd[L]) {
                        lq = L;
                        lb = bnd[L];
                    }
                    inside |= L <= N && bnd[L] > 16 * q && bnd[L] < 16 * q + 16;
                }
                if (!inside) {
                    uint32_t r = n_act_all - lvl_sp[lq + 1] + run - lvl_sp[lq];
                    const uint32_t e0 = 16 * q - lb;
                    run += __popc(m);
                    while (m) {
                        S.list[r++] = (uint16_t)(e0 + __ffs(m) - 1);
                        m &= m - 1;
                    }
                    continue;
                }
            }
            while (m) {
                const uint32_t k = __ffs(m) - 1, e = 16 * q + k;
                m &= m - 1;
                uint32_t l = 1, lb = 0;
#pragma unroll
                for (uint32_t L = 2; L <= (uint32_t)kMaxN; L++)
                    if (L <= N && e >= bnd[L]) {
                        l = L;
                        lb = bnd[L];
                    }
                const uint32_t r = n_act_all - lvl_sp[l + 1] + run - lvl_sp[l];
                S.list[r] = (uint16_t)(e - lb);
                run++;
            }
        }
        if (tid <= N) lvl_rank[tid] = tid == 0 ? n_act_all : n_act_all - lvl_sp[tid + 1];  // first rank of level
        __syncthreads();
        n_act_total = n_act_all;
    }
    const uint32_t n_ops = 8 * n_act_total, n_int_ops = 8 * lvl_rank[1];
    // the parent of rank r on level l
    auto parent_ops = [&](uint32_t r, uint32_t l) {
        const uint32_t lc = l - 1;
        const uint32_t p = S.list[r];
        // one thread per active parent: its 8 children, the parents next to it toward +axis, and the nodes
        // before its children toward -axis (children of the parent before it along that axis) are loaded
        // once; the 8 ops are chosen in registers and stored as one 8-byte word
        const uint32_t pbits = (1u << (3 * (N - l))) - 1u;  // Morton code bits of the parent level
        const uint32_t pmx = kMX & pbits, pmy = kMY & pbits, pmz = kMZ & pbits;
        const uint32_t *Lp = S.lab + loff(G.N, l);
        {
            const uint32_t pl = Lp[p];
            // faces of the brick: no -axis neighbour on the low face, no +axis neighbour on the high face
            const bool lox = (p & pmx) == 0, loy = (p & pmy) == 0, loz = (p & pmz) == 0;
            const bool hix = (p & pmx) == pmx, hiy = (p & pmy) == pmy, hiz = (p & pmz) == pmz;
            const uint32_t ppx = Lp[minc(p, pmx)], ppy = Lp[minc(p, pmy)], ppz = Lp[minc(p, pmz)];
            uint32_t v[8], nx[8], ny[8], nz[8];  // nx[c]: the -x neighbour of child c (c with x-bit 0)
            if (lc >= 1) {
                const uint32_t *L = S.lab + loff(G.N, lc);
                const uint4 a4 = *(const uint4 *)(L + 8 * p), b4 = *(const uint4 *)(L + 8 * p + 4);
                v[0] = a4.x; v[1] = a4.y; v[2] = a4.z; v[3] = a4.w;
                v[4] = b4.x; v[5] = b4.y; v[6] = b4.z; v[7] = b4.w;
                const uint32_t *Lx = L + 8 * mdec(p, pmx), *Ly = L + 8 * mdec(p, pmy), *Lz = L + 8 * mdec(p, pmz);
#pragma unroll
                for (uint32_t c = 0; c < 8; c++) {
                    nx[c] = Lx[c | 1u];
                    ny[c] = Ly[c | 2u];
                    nz[c] = Lz[c | 4u];
                }
            } else {
                const uint32_t x0 = 2 * compact6(p), y0 = 2 * compact6(p >> 1), z0 = 2 * compact6(p >> 2);
                if (B.interior && (B.X & 1u) == 0 && (reinterpret_cast<uintptr_t>(B.vol) & 7u) == 0) {
                    // rows of two voxels (x0 is even, rows 8-byte aligned): the 8 children in four 8-byte loads,
                    // their -x neighbours from the 8 bytes before each row, -y and -z from the rows before; a -axis
                    // neighbour node that is constant (81 % of the L1 nodes here) has its label in every voxel, so
                    // its voxels are not loaded
                    const uint8_t *Cp = S.cst + loff(G.N, l);
                    const uint32_t qx = mdec(p, pmx), qy = mdec(p, pmy), qz = mdec(p, pmz);
                    const bool kx = !lox && Cp[qx], ky = !loy && Cp[qy], kz = !loz && Cp[qz];
                    const uint32_t lx = Lp[qx], ly = Lp[qy], lz = Lp[qz];
                    const uint32_t *r0 = B.base + B.sz * z0 + B.sy * y0 + x0;
#pragma unroll
                    for (uint32_t k = 0; k < 4; k++) {  // k = dy + 2 dz, children 2k and 2k + 1
                        const uint32_t *rk = r0 + ((k & 1u) ? B.sy : 0u) + ((k & 2u) ? B.sz : 0u);
                        const uint2 a = __ldg(reinterpret_cast<const uint2 *>(rk));
                        v[2 * k] = a.x;
                        v[2 * k + 1] = a.y;
                        nx[2 * k] = lox ? 0u : kx ? lx : __ldg(reinterpret_cast<const uint2 *>(rk - 2)).y;
                        nx[2 * k + 1] = 0u;
                        if ((k & 1u) == 0) {  // y-bit 0: the row before along y
                            const uint2 m = loy ? make_uint2(0u, 0u)
                                            : ky  ? make_uint2(ly, ly)
                                                  : __ldg(reinterpret_cast<const uint2 *>(rk - B.sy));
                            ny[2 * k] = m.x;
                            ny[2 * k + 1] = m.y;
                        } else {
                            ny[2 * k] = ny[2 * k + 1] = 0u;
                        }
                        if ((k & 2u) == 0) {  // z-bit 0: the row before along z
                            const uint2 m = loz ? make_uint2(0u, 0u)
                                            : kz  ? make_uint2(lz, lz)
                                                  : __ldg(reinterpret_cast<const uint2 *>(rk - B.sz));
                            nz[2 * k] = m.x;
                            nz[2 * k + 1] = m.y;
                        } else {
                            nz[2 * k] = nz[2 * k + 1] = 0u;
                        }
                    }
                } else if (B.interior) {
                    const uint32_t *r = B.base + B.sz * z0 + B.sy * y0 + x0;
                    const int64_t sy = (int64_t)B.sy, sz = (int64_t)B.sz;
#pragma unroll
                    for (uint32_t c = 0; c < 8; c++) {
                        const int64_t o = (int64_t)(c & 1u) + sy * ((c >> 1) & 1u) + sz * (c >> 2);
                        v[c] = __ldg(r + o);
                        nx[c] = (c & 1u) ? 0u : __ldg(r + o - (lox ? 0 : 1));
                        ny[c] = (c & 2u) ? 0u : __ldg(r + o - (loy ? 0 : sy));
                        nz[c] = (c & 4u) ? 0u : __ldg(r + o - (loz ? 0 : sz));
                    }
                } else {
#pragma unroll
                    for (uint32_t c = 0; c < 8; c++) {
                        const uint32_t x = x0 + (c & 1u), y = y0 + ((c >> 1) & 1u), z = z0 + (c >> 2);
                        v[c] = B.at(x, y, z);
                        nx[c] = (c & 1u) ? 0u : B.at(lox ? x : x - 1, y, z);
                        ny[c] = (c & 2u) ? 0u : B.at(x, loy ? y : y - 1, z);
                        nz[c] = (c & 4u) ? 0u : B.at(x, y, loz ? z : z - 1);
                    }
                }
            }
            uint2 st2 = make_uint2(0u, 0u);
            if (lc >= 1) st2 = *(const uint2 *)(S.cst + loff(G.N, lc) + 8 * p);  // flags 0 / 1, one byte each
            uint32_t w[2] = {0u, 0u}, need = 0;
#pragma unroll
            for (uint32_t c = 0; c < 8; c++) {
                const bool bx = c & 1u, by = c & 2u, bz = c & 4u;
                const bool okx = bx ? !hix : !lox, oky = by ? !hiy : !loy, okz = bz ? !hiz : !loz;
                const uint32_t vx = bx ? ppx : nx[c], vy = by ? ppy : ny[c], vz = bz ? ppz : nz[c];
                // first applicable reuse: R_p, R_x, R_y, R_z (bestOperation order)
                const uint32_t op = v[c] == pl ? OP_RP
                                    : (okx && vx == v[c]) ? OP_RX
                                    : (oky && vy == v[c]) ? OP_RY
                                    : (okz && vz == v[c]) ? OP_RZ
                                    : kNeedPal;
                const uint32_t stop = ((c < 4 ? st2.x : st2.y) >> (8 * (c & 3u))) & 1u;
                w[c >> 2] |= (op | (stop << 3)) << (8 * (c & 3u));
                need |= (op == kNeedPal ? 1u : 0u) << c;
            }
            if (need) {  // the children no reuse fits, gathered with their labels for the palette pass (first 256)
                uint32_t at = atomicAdd(&sh_npc, (uint32_t)__popc(need));
#pragma unroll
                for (uint32_t c = 0; c < 8; c++)
                    if ((need >> c) & 1u) {
                        const uint32_t stop = ((c < 4 ? st2.x : st2.y) >> (8 * (c & 3u))) & 1u;
                        if (at < 256) S.plist[at] = make_uint2((8 * r + c) << 1 | stop, v[c]);  // op index, stop bit
                        at++;
                    }
            }
            *(uint2 *)(ops + 8 * r) = make_uint2(w[0], w[1]);
        }
    };
    // thread t takes the ranks r = t (mod kT): the parents above level 1 first (their level by rank), then
    // those of level 1, whose children are voxels (a loop of its own, specialised on the level)
    const uint32_t r_leaf = lvl_rank[1];
    for (uint32_t r = tid; r < r_leaf; r += kT) {
        uint32_t l = N;
        for (uint32_t L = 2; L < N; L++)
            if (r >= lvl_rank[L]) {
                l = L;
                break;
            }
        parent_ops(r, l);
    }
    for (uint32_t r = r_leaf + (tid + kT - r_leaf % kT) % kT; r < n_act_total; r += kT) parent_ops(r, 1u);
    __syncthreads();

    // each warp takes a contiguous range of the op array in phases C and D
    const uint32_t per = ((n_ops + (kT / 32) - 1) / (kT / 32) + 127) & ~127u;  // a multiple of 128 ops
    const uint32_t j0 = min(warp * per, n_ops), j1 = min(j0 + per, n_ops);

    // ---- C. palette pass in stream order: warp 0 walks the children no reuse fits, with the last 17 palette
    // entries in registers (lane i holds palette[i_p - i]).  Phase B gathered up to 256 of them with their
    // labels; they are put in stream order by rank and the walk also counts the P_delta ops per warp range
    // of phase D.  Bricks with more go through the gathering below, 256 at a time.
    const uint32_t n_need = sh_npc;
    const bool fast = n_need <= 256 && n_need <= kT;  // one thread per gathered child ranks it
    if (fast) {
        uint2 mine = make_uint2(0u, 0u);
        uint32_t rank = 0;
        if (tid < n_need) {
            mine = S.plist[tid];
#pragma unroll 8
            for (uint32_t k = 0; k < n_need; k++) rank += S.plist[k].x < mine.x ? 1u : 0u;
        }
        if (tid < 2 * (kT / 32)) sh_pd[tid] = 0;
        __syncthreads();
        if (tid < n_need) S.plist[rank] = mine;
        __syncthreads();
        if (warp == 0) {
            const uint32_t root = S.lab[loff(G.N, N)];
            uint32_t win = root;
            uint32_t ip = 0, np = 1;
            uint32_t *pal = count ? nullptr : SC.pal + (size_t)slot * G.pal_cap;
            if (pal && lane == 0) pal[0] = root;
            for (uint32_t k0 = 0; k0 < n_need; k0 += 32) {
                const uint32_t kn = min(32u, n_need - k0);
                const uint2 mine2 = lane < kn ? S.plist[k0 + lane] : make_uint2(0u, 0u);
                const uint32_t res = palette_chunk(mine2.y, kn, win, ip, np, pal, S.red);
                if (lane < kn) {
                    const uint32_t oi = mine2.x >> 1;  // the op's index; its stop bit came along from phase B
                    ops[oi] = (uint8_t)(((mine2.x & 1u) << 3) | res);
                    if ((res & 7u) == OP_PD) atomicAdd(&sh_pd[(oi >= n_int_ops ? (kT / 32) : 0u) + oi / per], 1u);
                }
            }
            if (lane == 0) sh_np = np;
        }
        __syncthreads();
    } else     {
        uint32_t cnt = 0;
        for (uint32_t g = j0; g < j1; g += 32) {
            const uint32_t j = g + lane;
            cnt += __popc(__ballot_sync(kFull, j < j1 && (ops[j] & 7u) == kNeedPal));
        }
        uint32_t total;
        const uint32_t wbase = block_excl_warp<kT / 32>(S.red, cnt, total);
        const uint32_t root = S.lab[loff(G.N, N)];
        uint32_t win = root;
        uint32_t ip = 0, np = 1;  // i_p and palette size (kept by warp 0)
        uint32_t *pal = count ? nullptr : SC.pal + (size_t)slot * G.pal_cap;
        if (pal && tid == 0) pal[0] = root;
        for (uint32_t r0 = 0; r0 < total; r0 += 256) {
            // gather this round's children (op index) in stream order ...
            if (wbase < r0 + 256 && wbase + cnt > r0) {
                uint32_t rank = wbase;
                for (uint32_t g = j0; g < j1; g += 32) {
                    const uint32_t j = g + lane;
                    // ranks count every child gathered in any round: children of earlier rounds already carry
                    // their palette op (P_0, P_delta or P_a), the others still the placeholder
                    const bool need = j < j1 && (ops[j] & 7u) >= OP_P0;
                    const uint32_t m = __ballot_sync(kFull, need);
                    const uint32_t rk = rank + __popc(m & lanemask_lt());
                    if (need && rk >= r0 && rk < r0 + 256) S.plist[rk - r0].x = j;
                    rank += __popc(m);
                }
            }
            __syncwarp();
            // ... then their labels, one child per lane (the loads overlap)
            const uint32_t e0 = max(wbase, r0), e1 = min(wbase + cnt, r0 + 256);
            for (uint32_t e = e0 + lane; e < e1; e += 32) {
                const uint32_t j = S.plist[e - r0].x, r = j >> 3;
                uint32_t l = N;
                for (uint32_t L = 1; L < N; L++)
                    if (r >= lvl_rank[L]) {
                        l = L;
                        break;
                    }
                const uint32_t p = S.list[r];
                S.plist[e - r0].y = node_label(B, S, G, l - 1, 8 * p + (j & 7u));
            }
            __syncthreads();
            if (warp == 0) {
                // 32 children at a time in lane registers; lane k keeps child k's op for one write-back
                const uint32_t nk = min(256u, total - r0);
                for (uint32_t k0 = 0; k0 < nk; k0 += 32) {
                    const uint32_t kn = min(32u, nk - k0);
                    const uint2 mine = lane < kn ? S.plist[k0 + lane] : make_uint2(0u, 0u);
                    const uint32_t res = palette_chunk(mine.y, kn, win, ip, np, pal, S.red);
                    if (lane < kn) ops[mine.x] = (uint8_t)((ops[mine.x] & 8u) | res);
                }
            }
            __syncthreads();
        }
        if (tid == 0) sh_np = np;
    }
    __syncthreads();

    // ---- D. symbol counts: a stream's ops plus its P_delta ops (each adds a delta nibble); in count mode (the
    // frequency prepass) the nibbles themselves are counted.  The rANS kernels code the op bytes directly.
    uint32_t sym_tot[2];
    {
        const uint32_t *pdc = sh_pd;  // P_delta per warp range: counted by the walk, or here
        if (!fast) {
            uint32_t pdi = 0, pdl = 0;
            for (uint32_t g = j0; g < j1; g += 32) {
                const uint32_t j = g + lane;
                const bool pd = j < j1 && (ops[j] & 7u) == OP_PD;
                pdi += __popc(__ballot_sync(kFull, pd && j < n_int_ops));
                pdl += __popc(__ballot_sync(kFull, pd && j >= n_int_ops));
            }
            if (lane == 0) {
                sh_pd[warp] = pdi;
                sh_pd[(kT / 32) + warp] = pdl;
            }
            __syncthreads();
        }
        uint32_t toti = 0, totl = 0;
        for (uint32_t w2 = 0; w2 < (kT / 32); w2++) {
            toti += pdc[w2];
            totl += pdc[(kT / 32) + w2];
        }
        sym_tot[0] = n_int_ops + toti;
        sym_tot[1] = n_ops - n_int_ops + totl;
        if (count)
            for (uint32_t j = j0 + lane; j < j1; j += 32) {
                const uint32_t o = ops[j], leaf = j >= n_int_ops ? 16u : 0u;
                atomicAdd(&hist[leaf + (o & 15u)], 1u);
                if ((o & 7u) == OP_PD) atomicAdd(&hist[leaf + (o >> 4)], 1u);
            }
    }
    if (count) {
        __syncthreads();
        if (tid < 32 && hist[tid]) atomicAdd(count + tid, (unsigned long long)hist[tid]);
        return;
    }
    if (tid == 0) {
        uint32_t *sz = SC.sizes + (size_t)slot * 8;
        sz[0] = sh_np;
        sz[1] = sym_tot[0];
        sz[2] = sym_tot[1];
        sz[7] = (n_int_ops >> 3) | (((n_ops - n_int_ops) >> 3) << 16);  // active parents per stream (< 2^16)
    }
}

// 4 CTAs per SM (64 registers): the compiler's own choice for this body, kept as a bound so that edits
// elsewhere in it do not drop the kernel to 3 CTAs per SM
template <uint32_t kN>  // 5 for bricks of 32^3, 0 (any size) for larger ones
__global__ void __launch_bounds__(kEncThreads, 4)
    encode_kernel(EncVol EV, EncGeom G, uint64_t brick0, uint64_t brick_stride, uint32_t n_in_batch,
                  EncScratch SC, unsigned long long *count) {
    encode_brick<kEncThreads, kN>(EV, G, brick0, brick_stride, n_in_batch, SC, count);
}

// The same for bricks of 16^3 and smaller, which need little shared memory (6.4 KB at 16^3): 128-thread CTAs,
// 16 per SM at 32 registers a thread.  For the 32768 bricks of a 512^3 volume at 16^3: 0.51 ms, against 0.53
// (64 threads, 24 per SM), 0.60 (256 threads, 8 per SM) and 0.71 ms (256 threads, 4 per SM).
constexpr uint32_t kEncSmallThreads = 128;
template <uint32_t kN>  // 4 for bricks of 16^3, 0 (any size) for smaller ones
__global__ void __launch_bounds__(kEncSmallThreads, 16)
    encode_kernel_small(EncVol EV, EncGeom G, uint64_t brick0, uint64_t brick_stride, uint32_t n_in_batch,
                        EncScratch SC, unsigned long long *count) {
    encode_brick<kEncSmallThreads, kN>(EV, G, brick0, brick_stride, n_in_batch, SC, count);
}

// ---- E. rANS, one warp per stream (brick slot q / 2, stream q % 2), from the op bytes of the encode kernel
// (op | stop << 3 | delta << 4, in stream order).  Coding order (reading R10): op j on state j mod K, a
// P_delta's delta nibble on its op's state; a step holds K ops in state order, then the deltas of its P_delta
// ops in state order.  Lane k holds state k and codes the steps from the last one down: in a step, first the
// deltas (lanes of P_delta ops), then the ops, each of the two a warp-wide substep whose renormalisation words
// are pushed downward from the top of the scratch area so that the decoder reads them forward in lane order.
// The ops are staged in shared memory window by window from the end.

// One coding substep: lanes with `act` code `sym` into their state x (Sec. 3.3, R9); renormalisation words go
// below `top`, in lane order.
__device__ __forceinline__ void rans_code_substep(uint32_t &x, uint32_t &top, uint16_t *words, uint32_t sym, bool act,
                                                  uint32_t fc_reg, uint32_t m_reg, uint32_t smask, uint32_t lt) {
    // the lanes hold f | c << 16 (f <= 4096, c < 4096) and the reciprocal m of f for their symbol
    const uint32_t fc = __shfl_sync(kFull, fc_reg, sym), f = fc & 0xFFFFu, c = fc >> 16;
    const uint32_t mf = __shfl_sync(kFull, m_reg, sym);
    // renormalise before coding: keep x below f * 2^20 (one 16-bit word at most)
    const bool emit = act && x >= (f << 20);
    const uint32_t m = __ballot_sync(kFull, emit) & smask;
    if (emit) {
        words[top - __popc(m) + __popc(m & lt)] = (uint16_t)(x & 0xFFFFu);
        x >>= 16;
    }
    top -= __popc(m);
    if (act) {
        // x / f by multiplication with a reciprocal (division by an invariant integer, Granlund and
        // Montgomery 1994): with m = floor((2^32 - 1) / f) = 2^32 / f - e, 0 < e <= 1, the high word of x m is
        // x / f - x e / 2^32 rounded down, i.e. the quotient or one less for every x < 2^32; one remainder
        // check makes it exact
        uint32_t qt = __umulhi(x, mf);
        uint32_t r = x - qt * f;
        if (r >= f) { qt += 1; r -= f; }
        x = qt * kM + r + c;
    }
}

// 32 registers, 7 CTAs per SM: the 1024 CTAs of 4096 bricks' streams run as one wave (39 registers and 6 CTAs
// left a second wave of 136 CTAs; 0.128 -> 0.125 ms on voronoi512 b=32)
__global__ void __launch_bounds__(kRansEncWarps * 32, 7)
    rans_encode_kernel(EncGeom G, EncScratch SC, uint32_t n_in_batch, const uint32_t *freq) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t q = blockIdx.x * kRansEncWarps + warp;
    if (q >= 2 * n_in_batch) return;
    const uint32_t slot = q >> 1, st = q & 1u;
    uint32_t *sz = SC.sizes + (size_t)slot * 8;
    const uint32_t n = sz[1 + st];
    const uint32_t apc = sz[7];  // active parents per stream: 8 ops each
    const uint32_t first = st == 0 ? 0u : 8u * (apc & 0xFFFFu);             // the stream's first op in the brick
    const uint32_t n_ops = st == 0 ? 8u * (apc & 0xFFFFu) : 8u * (apc >> 16);
    const uint8_t *ops = SC.ops + (size_t)slot * G.ops_cap;  // 16-byte aligned, ops_cap a multiple of 16
    const uint32_t cap = (st == 0 ? G.int_cap : G.leaf_cap) + 64;
    uint16_t *words = (st == 0 ? SC.w_int : SC.w_leaf) + (size_t)slot * cap;
    uint8_t *wsm = smem_raw + warp * kRansEncWin;
    const uint32_t *F = freq + 16 * st;
    const uint32_t f_reg = lane < 16 ? F[lane] : 1u;
    const uint32_t m_reg = 0xFFFFFFFFu / f_reg;  // reciprocal of f for the quotient x / f
    uint32_t c_reg = 0;
    for (uint32_t s2 = 0; s2 < 16; s2++) c_reg += (s2 < lane) ? F[s2] : 0u;
    const uint32_t fc_reg = f_reg | (c_reg << 16);
    const uint32_t K = lanes_for(n, G.K_max, G.S_min);
    const uint32_t lt = lanemask_lt();
    uint32_t top = cap;
    if (n > 0) {
        uint32_t x = kL;
        const uint32_t steps = (n_ops + K - 1) / K;
        const uint32_t win_steps = (kRansEncWin - 16) / K;  // steps per staged window (16 bytes of alignment slack)
        // windows of steps from the end: [s_lo, s_hi) covers ops [s_lo*K, min(n_ops, s_hi*K)) of the stream
        for (uint32_t s_hi = steps; s_hi > 0;) {
            const uint32_t s_lo = s_hi > win_steps ? s_hi - win_steps : 0u;
            const uint32_t lo16 = (first + s_lo * K) & ~15u, op_hi = first + min(n_ops, s_hi * K);
            __syncwarp();
            for (uint32_t c16 = lane; lo16 + 16 * c16 < op_hi; c16 += 32)
                reinterpret_cast<uint4 *>(wsm)[c16] = __ldcg(reinterpret_cast<const uint4 *>(ops + lo16) + c16);
            __syncwarp();
            for (uint32_t s2 = s_hi; s2-- > s_lo;) {
                const uint32_t i = s2 * K + lane;
                const bool act = lane < K && i < n_ops;
                const uint32_t o = act ? (uint32_t)wsm[first + i - lo16] : 0u;
                const bool pd = act && (o & 7u) == OP_PD;
                if (__any_sync(kFull, pd)) rans_code_substep(x, top, words, o >> 4, pd, fc_reg, m_reg, kFull, lt);
                rans_code_substep(x, top, words, o & 15u, act, fc_reg, m_reg, kFull, lt);
            }
            // this window's op bytes are read for the last time (the op array is dead after this kernel); the
            // lines shared with the next window down or with the brick's other stream are kept
            discard_l2(reinterpret_cast<uintptr_t>(ops + first + s_lo * K), reinterpret_cast<uintptr_t>(ops + op_hi), lane);
            s_hi = s_lo;
        }
        // final states ahead of the words, state 0 first, low half first
        if (lane < K) {
            words[top - 2 * K + 2 * lane] = (uint16_t)(x & 0xFFFFu);
            words[top - 2 * K + 2 * lane + 1] = (uint16_t)(x >> 16);
        }
        top -= 2 * K;
    }
    if (lane == 0) {
        sz[3 + st] = cap - top;  // words
        sz[5 + st] = top;        // start inside the scratch area
    }
}

// rans_encode_kernel for bricks of 16^3 and smaller, whose streams have few states (K = 1..4 at the default
// S_min): a warp takes kEpkSegs consecutive streams (16 at 16^3, 32 at 8^3 and smaller) and codes as many of
// them at once as their K lanes fit in 32, each on its own run of lanes (its segment) with its own window of
// staged op bytes; a step codes, on every stream that has steps left, the deltas of its P_delta ops and then
// its ops (the streams' steps run from their ends, so shorter streams finish earlier).  Lanes 0..15 hold the
// interior table, lanes 16..31 the leaf table.  Same words as rans_encode_kernel.
template <uint32_t kEpkSegs>  // streams per warp; each stream of a group stages kRansEncWin / kEpkSegs bytes
__global__ void __launch_bounds__(kRansEncWarps * 32)
    rans_encode_packed(EncGeom G, EncScratch SC, uint32_t n_in_batch, const uint32_t *freq) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, lt = lanemask_lt();
    const uint32_t q0 = (blockIdx.x * kRansEncWarps + warp) * kEpkSegs, n_q = 2 * n_in_batch;
    if (q0 >= n_q) return;
    const uint32_t tab = lane >> 4, tsym = lane & 15u;  // this lane's table entry
    const uint32_t *F = freq + 16 * tab;
    const uint32_t f_reg = F[tsym];
    const uint32_t m_reg = 0xFFFFFFFFu / (f_reg ? f_reg : 1u);  // reciprocal of f for the quotient x / f
    uint32_t c_reg = 0;
    for (uint32_t s2 = 0; s2 < 16; s2++) c_reg += (s2 < tsym) ? F[s2] : 0u;
    const uint32_t fc_reg = f_reg | (c_reg << 16);
    uint8_t *wbase = smem_raw + warp * kRansEncWin;
    const uint32_t g_end = min(kEpkSegs, n_q - q0);
    uint32_t g = 0;
    while (g < g_end) {
        // ---- a group: the next streams of the warp's share while their lanes fit (warp-uniform)
        uint32_t my_q = 0, nseg = 0, used = 0, ends = 0;  // ends: bit e set for the last lane e of a segment
        while (g < g_end) {
            const uint32_t q = q0 + g, slot = q >> 1, st = q & 1u;
            const uint32_t n = SC.sizes[(size_t)slot * 8 + 1 + st];
            if (n == 0) {  // nothing to code: no words
                if (lane == 0) {
                    const uint32_t cap = (st == 0 ? G.int_cap : G.leaf_cap) + 64;
                    SC.sizes[(size_t)slot * 8 + 3 + st] = 0;
                    SC.sizes[(size_t)slot * 8 + 5 + st] = cap;
                }
                g++;
                continue;
            }
            const uint32_t K = lanes_for(n, G.K_max, G.S_min);
            if (used + K > 32) break;  // next group (a group's first stream always fits: K <= 32)
            if (lane == nseg) my_q = q;
            used += K;
            ends |= 1u << (used - 1);
            nseg++;
            g++;
        }
        if (nseg == 0) break;
        // ---- this lane's stream
        const bool mine = lane < used;
        const uint32_t before = ends & lt;
        const uint32_t seg = __popc(before), sb = before ? 32 - __clz(before) : 0u;
        const uint32_t q = __shfl_sync(kFull, my_q, mine ? seg : 0u);
        const uint32_t slot = q >> 1, st = q & 1u, j = lane - sb;
        uint32_t n = 0, K = 1, cap = 0, first = 0, n_ops = 0;
        uint16_t *words = nullptr;
        const uint8_t *ops = nullptr;
        if (mine) {
            n = SC.sizes[(size_t)slot * 8 + 1 + st];
            K = lanes_for(n, G.K_max, G.S_min);
            cap = (st == 0 ? G.int_cap : G.leaf_cap) + 64;
            words = (st == 0 ? SC.w_int : SC.w_leaf) + (size_t)slot * cap;
            const uint32_t apc = SC.sizes[(size_t)slot * 8 + 7];  // active parents per stream: 8 ops each
            first = st == 0 ? 0u : 8u * (apc & 0xFFFFu);
            n_ops = st == 0 ? 8u * (apc & 0xFFFFu) : 8u * (apc >> 16);
            ops = SC.ops + (size_t)slot * G.ops_cap;  // 16-byte aligned
        }
        const uint32_t smask = mine ? (K >= 32 ? kFull : ((1u << K) - 1u) << sb) : 0u;
        // the window of a lone stream is the warp's whole area
        const uint32_t win_bytes = nseg == 1 ? kRansEncWin : (kRansEncWin / kEpkSegs);
        uint8_t *wsm = wbase + (mine ? seg : 0u) * (kRansEncWin / kEpkSegs);
        const uint32_t win_steps = (win_bytes - 16) / K;  // steps per staged window (16 bytes of alignment slack)
        uint32_t x = kL, top = cap;
        uint32_t s_hi = mine ? (n_ops + K - 1) / K : 0u;  // steps left: the next step coded is s_hi - 1
        uint32_t s_lo = s_hi, lo16 = 0;                   // staged: steps [s_lo, s_hi of the window)
        for (;;) {
            const bool run = s_hi > 0;
            if (!__any_sync(kFull, run)) break;
            if (__any_sync(kFull, run && s_hi == s_lo)) {  // stage the window of steps below s_hi
                __syncwarp();
                if (run && s_hi == s_lo) {
                    s_lo = s_hi > win_steps ? s_hi - win_steps : 0u;
                    lo16 = (first + s_lo * K) & ~15u;
                    const uint32_t op_hi = first + min(n_ops, s_hi * K);
                    for (uint32_t c16 = j; lo16 + 16 * c16 < op_hi; c16 += K)
                        reinterpret_cast<uint4 *>(wsm)[c16] = __ldcg(reinterpret_cast<const uint4 *>(ops + lo16) + c16);
                }
                __syncwarp();
            }
            const uint32_t i = (s_hi - 1) * K + j;
            const bool act = run && j < K && i < n_ops;
            const uint32_t o = act ? (uint32_t)wsm[first + i - lo16] : 0u;
            const bool pd = act && (o & 7u) == OP_PD;
            // the deltas first, then the ops: the reverse of the decoder's order (entry 16 st + s of the tables)
            if (__any_sync(kFull, pd))
                rans_code_substep(x, top, words, (o >> 4) + 16 * st, pd, fc_reg, m_reg, smask, lt);
            rans_code_substep(x, top, words, (o & 15u) + 16 * st, act, fc_reg, m_reg, smask, lt);
            if (run) s_hi--;
        }
        // final states ahead of the words, state 0 first, low half first
        if (mine) {
            words[top - 2 * K + 2 * j] = (uint16_t)(x & 0xFFFFu);
            words[top - 2 * K + 2 * j + 1] = (uint16_t)(x >> 16);
            top -= 2 * K;
            if (j == 0) {
                SC.sizes[(size_t)slot * 8 + 3 + st] = cap - top;  // words
                SC.sizes[(size_t)slot * 8 + 5 + st] = top;        // start inside the scratch area
            }
        }
        __syncwarp();
    }
}

// Nibble counts (interior then leaf) of the bricks of a batch whose slot is a multiple of `stride`: the counts
// of the frequency prepass (Sec. 3.3), taken from an encode's op bytes.  Every op byte counts its nibble
// (op | stop << 3), a P_delta also its delta nibble; the ops before the interior op count belong to the
// interior stream.  Grid (sampled bricks, kHistSplit), 16 bytes per load, per-warp histograms in shared memory.
constexpr uint32_t kHistSplit = 8;

__global__ void __launch_bounds__(256) op_hist_kernel(EncGeom G, EncScratch SC, uint32_t stride,
                                                      unsigned long long *counts) {
    __shared__ uint32_t h[8][32];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    h[warp][lane] = 0;
    __syncthreads();
    const uint32_t slot = blockIdx.x * stride;
    const uint32_t apc = SC.sizes[(size_t)slot * 8 + 7];
    const uint32_t n_int_ops = 8u * (apc & 0xFFFFu), n_ops = n_int_ops + 8u * (apc >> 16);
    const uint4 *src = (const uint4 *)(SC.ops + (size_t)slot * G.ops_cap);
    const uint32_t t0 = blockIdx.y * blockDim.x + threadIdx.x, step = kHistSplit * blockDim.x;
    for (uint32_t i = t0; 16 * i < n_ops; i += step) {
        const uint4 v = src[i];
        const uint32_t wd[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (uint32_t k = 0; k < 16; k++) {
            const uint32_t j = 16 * i + k;
            if (j < n_ops) {
                const uint32_t o = (wd[k >> 2] >> (8 * (k & 3u))) & 255u, part = j < n_int_ops ? 0u : 16u;
                atomicAdd(&h[warp][part + (o & 15u)], 1u);
                if ((o & 7u) == OP_PD) atomicAdd(&h[warp][part + (o >> 4)], 1u);
            }
        }
    }
    __syncthreads();
    if (warp == 0) {
        uint32_t c = 0;
#pragma unroll
        for (uint32_t w2 = 0; w2 < 8; w2++) c += h[w2][lane];
        if (c) atomicAdd(counts + lane, (unsigned long long)c);
    }
}

// Exclusive scan of per-brick sizes (palette labels, interior words, leaf words) of one batch into the
// volume's offset arrays, continuing from the running totals in tot[0..2]; writes the new totals.  Also
// raises maxes[0..2] (when given) to the batch's largest palette, interior and leaf symbol counts.  One CTA:
// thread t takes the contiguous run of bricks [t * per, (t + 1) * per), sums it, and the block scans the
// 1024 sums.
__global__ void __launch_bounds__(1024) scan_sizes_kernel(const uint32_t *sizes, uint32_t n, uint64_t first,
                                                          uint64_t *pal_off, uint64_t *int_off, uint64_t *leaf_off,
                                                          uint64_t *tot, uint32_t *maxes) {
    __shared__ unsigned long long part[3][32];
    __shared__ uint32_t mx[3][32];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t per = (n + 1023) / 1024, i0 = min(n, tid * per), i1 = min(n, i0 + per);
    unsigned long long sum[3] = {0, 0, 0};
    uint32_t big[3] = {0, 0, 0};
#pragma unroll 4
    for (uint32_t i = i0; i < i1; i++) {
        const uint4 q = *(const uint4 *)(sizes + 8 * (size_t)i);  // n_pal, n_int_sym, n_leaf_sym, n_int_words
        const uint32_t nwl = sizes[8 * (size_t)i + 4];
        sum[0] += q.x;
        sum[1] += q.w;
        sum[2] += nwl;
        big[0] = max(big[0], q.x);
        big[1] = max(big[1], q.y);
        big[2] = max(big[2], q.z);
    }
    unsigned long long inc[3] = {sum[0], sum[1], sum[2]};
#pragma unroll
    for (int a = 0; a < 3; a++) {
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long u = __shfl_up_sync(kFull, inc[a], d);
            if (lane >= (uint32_t)d) inc[a] += u;
        }
        big[a] = __reduce_max_sync(kFull, big[a]);
    }
    if (lane == 31)
        for (int a = 0; a < 3; a++) part[a][warp] = inc[a];
    if (lane == 0)
        for (int a = 0; a < 3; a++) mx[a][warp] = big[a];
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the 32 warp totals, in place
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const unsigned long long t = part[a][lane];
            unsigned long long x = t;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long u = __shfl_up_sync(kFull, x, d);
                if (lane >= (uint32_t)d) x += u;
            }
            part[a][lane] = x - t;
        }
    }
    __syncthreads();
    unsigned long long run[3];
    for (int a = 0; a < 3; a++) run[a] = tot[a] + part[a][warp] + inc[a] - sum[a];  // before this thread's first brick
    for (uint32_t i = i0; i < i1; i++) {
        const uint4 q = *(const uint4 *)(sizes + 8 * (size_t)i);
        const uint32_t nwl = sizes[8 * (size_t)i + 4];
        pal_off[first + i] = run[0];
        int_off[first + i] = run[1];
        leaf_off[first + i] = run[2];
        run[0] += q.x;
        run[1] += q.w;
        run[2] += nwl;
    }
    __syncthreads();  // every thread has read tot[] before thread 1023 moves it
    if (tid == 1023) {  // holds the batch's inclusive totals
        for (int a = 0; a < 3; a++) tot[a] = run[a];
        pal_off[first + n] = run[0];
        int_off[first + n] = run[1];
        leaf_off[first + n] = run[2];
    }
    if (tid < 3 && maxes) {
        uint32_t m = maxes[tid];
        for (uint32_t w = 0; w < 32; w++) m = max(m, mx[tid][w]);
        maxes[tid] = m;
    }
}

// Two-pass size scan for large batches (blocks of kScanBlock bricks, a thread per brick).  Pass 1: each block's
// totals (palette labels, interior words, leaf words) and maxima (palette, interior and leaf symbol counts)
// into blk[b]; block 0 also copies the running totals to blk[kScanMaxBlocks] (pass 2 reads that copy and its
// last block writes the new totals).  Pass 2: each block starts from the running totals plus the blocks
// before it and writes its offsets.  blk: (kScanMaxBlocks + 1) x 4 u64.
constexpr uint32_t kScanBlock = 1024, kScanMaxBlocks = 64;

__device__ __forceinline__ void scan_vals(const uint32_t *sizes, uint32_t i, uint32_t n, unsigned long long v[3],
                                          uint32_t mx[3]) {
    v[0] = v[1] = v[2] = 0;
    mx[0] = mx[1] = mx[2] = 0;
    if (i < n) {
        const uint4 q = *(const uint4 *)(sizes + 8 * (size_t)i);  // n_pal, n_int_sym, n_leaf_sym, n_int_words
        v[0] = q.x;
        v[1] = q.w;
        v[2] = sizes[8 * (size_t)i + 4];
        mx[0] = q.x;
        mx[1] = q.y;
        mx[2] = q.z;
    }
}

__global__ void __launch_bounds__(kScanBlock) scan_blocks_kernel(const uint32_t *sizes, uint32_t n,
                                                                 const uint64_t *tot, unsigned long long *blk) {
    __shared__ unsigned long long ps[3][32];
    __shared__ uint32_t pm[3][32];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long v[3];
    uint32_t mx[3];
    scan_vals(sizes, blockIdx.x * kScanBlock + tid, n, v, mx);
#pragma unroll
    for (int a = 0; a < 3; a++) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) v[a] += __shfl_xor_sync(kFull, v[a], d);
        mx[a] = __reduce_max_sync(kFull, mx[a]);
        if (lane == 0) {
            ps[a][warp] = v[a];
            pm[a][warp] = mx[a];
        }
    }
    __syncthreads();
    if (tid < 3) {
        unsigned long long sum = 0;
        uint32_t m = 0;
        for (uint32_t w = 0; w < kScanBlock / 32; w++) {
            sum += ps[tid][w];
            m = max(m, pm[tid][w]);
        }
        blk[4 * blockIdx.x + tid] = sum;
        blk[4 * (kScanMaxBlocks + 1) + 4 * blockIdx.x + tid] = m;  // maxima after the sums
        if (blockIdx.x == 0) blk[4 * kScanMaxBlocks + tid] = tot[tid];
    }
}

__global__ void __launch_bounds__(kScanBlock) scan_write_kernel(const uint32_t *sizes, uint32_t n, uint64_t first,
                                                                uint64_t *pal_off, uint64_t *int_off,
                                                                uint64_t *leaf_off, uint64_t *tot, uint32_t *maxes,
                                                                const unsigned long long *blk) {
    __shared__ unsigned long long part[3][32], base[3];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, b = blockIdx.x;
    if (tid < 3) {  // running totals plus the blocks before this one
        unsigned long long s = blk[4 * kScanMaxBlocks + tid];
        for (uint32_t k = 0; k < b; k++) s += blk[4 * k + tid];
        base[tid] = s;
    }
    unsigned long long v[3], inc[3];
    uint32_t mx[3];
    const uint32_t i = b * kScanBlock + tid;
    scan_vals(sizes, i, n, v, mx);
#pragma unroll
    for (int a = 0; a < 3; a++) {
        inc[a] = v[a];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long u = __shfl_up_sync(kFull, inc[a], d);
            if (lane >= (uint32_t)d) inc[a] += u;
        }
        if (lane == 31) part[a][warp] = inc[a];
    }
    __syncthreads();
    if (warp == 0) {  // exclusive scan of the warp totals, in place
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const unsigned long long t = part[a][lane];
            unsigned long long x = t;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long u = __shfl_up_sync(kFull, x, d);
                if (lane >= (uint32_t)d) x += u;
            }
            part[a][lane] = x - t;
        }
    }
    __syncthreads();
    unsigned long long o[3];
#pragma unroll
    for (int a = 0; a < 3; a++) o[a] = base[a] + part[a][warp] + inc[a] - v[a];
    if (i < n) {
        pal_off[first + i] = o[0];
        int_off[first + i] = o[1];
        leaf_off[first + i] = o[2];
    }
    if (b == gridDim.x - 1 && i == n - 1) {  // the batch's last brick: new totals and the end offsets
        for (int a = 0; a < 3; a++) tot[a] = o[a] + v[a];
        pal_off[first + n] = o[0] + v[0];
        int_off[first + n] = o[1] + v[1];
        leaf_off[first + n] = o[2] + v[2];
    }
    if (b == gridDim.x - 1 && tid < 3 && maxes) {
        uint32_t m = maxes[tid];
        for (uint32_t k = 0; k < gridDim.x; k++) m = max(m, (uint32_t)blk[4 * (kScanMaxBlocks + 1) + 4 * k + tid]);
        maxes[tid] = m;
    }
}

// Copy each brick's palette and words from scratch to the packed arrays: one warp per run (a brick's palette,
// interior words or leaf words), eight loads in flight per lane.  The runs are short (about 2 KB a brick on
// the benchmark volumes), so the kernel is bound by the latency of its dependent loads rather than by
// bandwidth, and a brick's three runs go to three warps instead of one after another.
constexpr uint32_t kCompactWarps = 8;

template <typename T>
__device__ __forceinline__ void copy_run(T *__restrict__ d, const T *__restrict__ s, uint32_t n, uint32_t lane) {
    uint32_t k = lane;
    for (; k + 224 < n; k += 256) {
        T a[8];
#pragma unroll
        for (uint32_t j = 0; j < 8; j++) a[j] = s[k + 32 * j];
#pragma unroll
        for (uint32_t j = 0; j < 8; j++) d[k + 32 * j] = a[j];
    }
    for (; k < n; k += 32) d[k] = s[k];
}

__global__ void __launch_bounds__(kCompactWarps * 32) compact_kernel(EncGeom G, EncScratch SC, uint64_t first, uint32_t n,
                                                                     const uint64_t *pal_off, const uint64_t *int_off,
                                                                     const uint64_t *leaf_off, uint32_t *pal,
                                                                     uint16_t *int_words, uint16_t *leaf_words,
                                                                     uint32_t *n_int_sym, uint32_t *n_leaf_sym) {
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t task = (uint64_t)blockIdx.x * kCompactWarps + (threadIdx.x >> 5);
    if (task >= 3ull * n) return;
    const uint32_t slot = (uint32_t)(task / 3), run = (uint32_t)(task % 3);
    const uint32_t *sz = SC.sizes + (size_t)slot * 8;  // n_pal, n_int_sym, n_leaf_sym, words, word starts
    const uint64_t id = first + slot;
    if (run == 0) {
        copy_run(pal + pal_off[id], SC.pal + (size_t)slot * G.pal_cap, sz[0], lane);
    } else if (run == 1) {
        copy_run(int_words + int_off[id], SC.w_int + (size_t)slot * (G.int_cap + 64) + sz[5], sz[3], lane);
        if (lane == 0) n_int_sym[id] = sz[1];
    } else {
        copy_run(leaf_words + leaf_off[id], SC.w_leaf + (size_t)slot * (G.leaf_cap + 64) + sz[6], sz[4], lane);
        if (lane == 0) n_leaf_sym[id] = sz[2];
    }
}

}  // namespace

// ---------------------------------------------------------------- host helpers

EncGeom make_geom(uint32_t N, uint32_t K_max, uint32_t S_min) {
    EncGeom G{};
    G.N = N;
    G.b = 1u << N;
    uint32_t u = 0;
    for (uint32_t l = 1; l <= N; l++) {
        G.off[l] = u;
        u += (G.b >> l) * (G.b >> l) * (G.b >> l);
    }
    G.up_nodes = u;
    const uint32_t b3 = G.b * G.b * G.b;
    // every node but the root can be coded (>= 256: rANS staging); a multiple of 16 so that each brick's op
    // array starts on a 16-byte boundary (phase D stages it with 16-byte loads)
    G.ops_cap = ((u + b3 - 1 > 256u ? u + b3 - 1 : 256u) + 15u) & ~15u;
    G.pal_cap = u + b3;             // palette: root + one per P_a
    G.int_cap = (2 * (u - 1) + 2 + 15) & ~15u;  // interior nibbles at most (op + delta each), 16-byte pitch
    G.leaf_cap = (2 * b3 + 15) & ~15u;
    G.lvl_bytes = N >= 6 ? enc_level_bytes(G.up_nodes) : 0u;  // b = 64: level arrays in global scratch
    G.smem = enc_smem_bytes(G.up_nodes, G.lvl_bytes != 0);
    G.K_max = K_max;
    G.S_min = S_min;
    return G;
}

size_t scratch_bytes_per_brick(const EncGeom &G) {
    return (size_t)G.pal_cap * 4 + (size_t)(G.int_cap + 64) * 2 + (size_t)(G.leaf_cap + 64) * 2 + 8 * 4 + 64 +
           G.ops_cap + G.lvl_bytes;
}

cudaError_t launch_encode(const EncVol &EV, const EncGeom &G, uint64_t brick0, uint64_t stride, uint32_t n,
                          const uint32_t *freq, const EncScratch &SC, unsigned long long *count, cudaStream_t st) {
    // bricks of 16^3 and smaller: more CTAs per SM (encode_kernel_small)
    const bool small = G.N <= 4;
    // the brick sizes of the benchmarks (32^3, 16^3) take kernels specialised for them
    auto k = small ? (G.N == 4 ? encode_kernel_small<4> : encode_kernel_small<0>)
                   : (G.N == 5 ? encode_kernel<5> : encode_kernel<0>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, G.smem);
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    {
        ProfScope ps(count ? "encode_count" : "encode", st);
        k<<<n, small ? kEncSmallThreads : kEncThreads, G.smem, st>>>(EV, G, brick0, stride, n, SC, count);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess || count || !freq) return e;  // no tables yet: the caller codes later
    return launch_rans_encode(G, SC, n, freq, st);
}

cudaError_t launch_rans_encode(const EncGeom &G, const EncScratch &SC, uint32_t n, const uint32_t *freq,
                               cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    cudaError_t e;
    const uint32_t smem_e = kRansEncWarps * kRansEncWin;
    // bricks of 16^3 and smaller: streams of a few states, coded several to a warp
    const bool packed = G.N <= 4;
    // streams per warp: 16 at 16^3 (0.27 ms for 32768 bricks, against 0.31 with 8 and 0.39 with 32), 32 below
    // (8^3: 0.09 ms, against 0.19 with 8)
    const uint32_t segs = G.N <= 3 ? 32u : 16u;
    auto kp = segs == 32 ? rans_encode_packed<32> : rans_encode_packed<16>;
    e = cudaFuncSetAttribute(packed ? kp : rans_encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_e);
    if (e != cudaSuccess) return e;
    {
        ProfScope ps("rans_encode", st);
        if (packed) {
            const uint32_t per_cta = kRansEncWarps * segs;
            kp<<<(2 * n + per_cta - 1) / per_cta, kRansEncWarps * 32, smem_e, st>>>(G, SC, n, freq);
        } else {
            rans_encode_kernel<<<(2 * n + kRansEncWarps - 1) / kRansEncWarps, kRansEncWarps * 32, smem_e, st>>>(
                G, SC, n, freq);
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_nibble_hist(const EncGeom &G, const EncScratch &SC, uint32_t n, uint32_t stride,
                               unsigned long long *counts, cudaStream_t st) {
    const uint32_t sampled = (n + stride - 1) / stride;
    if (sampled == 0) return cudaSuccess;
    {
        ProfScope ps("nibble_hist", st);
        op_hist_kernel<<<dim3(sampled, kHistSplit), 256, 0, st>>>(G, SC, stride, counts);
    }
    return cudaGetLastError();
}

cudaError_t launch_scan(const uint32_t *sizes, uint32_t n, uint64_t first, uint64_t *pal_off, uint64_t *int_off,
                        uint64_t *leaf_off, uint64_t *tot, uint32_t *maxes, unsigned long long *blk, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const uint32_t nblk = (n + kScanBlock - 1) / kScanBlock;
    if (!blk || nblk > kScanMaxBlocks || nblk == 1) {  // one CTA
        ProfScope ps("scan_sizes", st);
        scan_sizes_kernel<<<1, 1024, 0, st>>>(sizes, n, first, pal_off, int_off, leaf_off, tot, maxes);
        return cudaGetLastError();
    }
    {
        ProfScope ps("scan_blocks", st);
        scan_blocks_kernel<<<nblk, kScanBlock, 0, st>>>(sizes, n, tot, blk);
    }
    {
        ProfScope ps("scan_sizes", st);
        scan_write_kernel<<<nblk, kScanBlock, 0, st>>>(sizes, n, first, pal_off, int_off, leaf_off, tot, maxes, blk);
    }
    return cudaGetLastError();
}

cudaError_t launch_compact(const EncGeom &G, const EncScratch &SC, uint64_t first, uint32_t n, const uint64_t *pal_off,
                           const uint64_t *int_off, const uint64_t *leaf_off, uint32_t *pal, uint16_t *int_words,
                           uint16_t *leaf_words, uint32_t *n_int_sym, uint32_t *n_leaf_sym, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    {
        ProfScope ps("compact", st);
        compact_kernel<<<(unsigned)((3ull * n + kCompactWarps - 1) / kCompactWarps), kCompactWarps * 32, 0, st>>>(
            G, SC, first, n, pal_off, int_off, leaf_off, pal, int_words, leaf_words, n_int_sym, n_leaf_sym);
    }
    return cudaGetLastError();
}


}  // namespace csgv
