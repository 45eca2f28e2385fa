// encode.cu -- brick encoder (Alg. 2 of the paper), frequency prepass and
// packing for sm_103a.
//
// One CTA encodes one brick:
//   A. pyramid (Sec. 3.1): L1 from the volume in global memory, L2..LN in
//      shared memory; each node is the most frequent of its 8 children, ties
//      to the first occurrence in the child array (Sec. 3.4), plus a
//      constant-subtree flag.
//   B. per level, the list of active (non-constant) parents in Morton order
//      and, for each of their children in parallel, the first applicable
//      reuse operation R_p, R_x, R_y, R_z (Sec. 3.2, reading R4); children
//      no reuse fits are marked for the palette pass.
//   C. palette pass: one warp walks the marked children in stream order with
//      the last 17 palette entries in registers (lane i holds palette[i_p-i]):
//      a ballot finds P_0 (lane 0) or the smallest P_delta (lanes 1..16);
//      otherwise P_a appends the label (Sec. 3.2, bestOperation order).
//   D. nibble positions (one extra nibble after each P_delta, reading R18)
//      by warp scans; interior and leaf nibbles written to scratch, or only
//      counted in the prepass (Sec. 3.4).
//   E. rANS: one warp per stream, K interleaved states in lanes, symbols in
//      reverse; renormalisation words are pushed downward from the top of
//      the scratch area so that the decoder reads them forward in lane order
//      (Sec. 3.3, readings R9/R10).
// A scan kernel turns per-brick sizes into offsets and a compaction kernel
// packs palettes and words into the volume's arrays.
#include "encode_api.cuh"

namespace csgv {

constexpr uint32_t kEncThreads = 256;
constexpr uint32_t kEncWarps = kEncThreads / 32;
constexpr uint32_t kNeedPal = 7;  // op placeholder: no reuse operation applies

namespace {

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ uint32_t spread5(uint32_t v) {
    return (v & 1u) | ((v & 2u) << 2) | ((v & 4u) << 4) | ((v & 8u) << 6) | ((v & 16u) << 8);
}
__device__ __forceinline__ uint32_t morton3(uint32_t x, uint32_t y, uint32_t z) {
    return spread5(x) | (spread5(y) << 1) | (spread5(z) << 2);
}
__device__ __forceinline__ uint32_t compact5(uint32_t m) {
    return (m & 1u) | ((m >> 2) & 2u) | ((m >> 4) & 4u) | ((m >> 6) & 8u) | ((m >> 8) & 16u);
}
__device__ __forceinline__ uint32_t mdec(uint32_t m, uint32_t ma) { return (((m & ma) - 1u) & ma) | (m & ~ma); }
__device__ __forceinline__ uint32_t minc(uint32_t m, uint32_t ma) { return (((m | ~ma) + 1u) & ma) | (m & ~ma); }

// most frequent of 8 labels, ties to the first occurrence (Sec. 3.4)
__device__ __forceinline__ uint32_t mode8(const uint32_t w[8], bool &all_equal) {
    uint32_t best = w[0];
    int best_cnt = 0;
#pragma unroll
    for (int c = 0; c < 8; c++) {
        int cnt = 0;
#pragma unroll
        for (int d = 0; d < 8; d++) cnt += (w[d] == w[c]);
        if (cnt > best_cnt) {
            best_cnt = cnt;
            best = w[c];
        }
    }
    all_equal = best_cnt == 8;
    return best;
}

struct Brick {
    const uint32_t *vol;
    uint64_t X, Y, Z;
    uint64_t gx0, gy0, gz0;  // brick origin
    bool interior;           // no clamping needed
    __device__ __forceinline__ uint32_t at(uint32_t x, uint32_t y, uint32_t z) const {
        uint64_t gx = gx0 + x, gy = gy0 + y, gz = gz0 + z;
        if (!interior) {
            gx = gx < X ? gx : X - 1;
            gy = gy < Y ? gy : Y - 1;
            gz = gz < Z ? gz : Z - 1;
        }
        return __ldg(vol + gx + X * (gy + Y * gz));
    }
};

// shared memory of the encoder CTA
struct EncSmem {
    uint32_t *lab;     // up_nodes labels, levels 1..N
    uint8_t *cst;      // up_nodes const flags
    uint16_t *list;    // active parents per parent level (same offsets as lab)
    uint8_t *ops;      // ops_cap op bytes: op | stop<<3 | delta<<4
    uint32_t *red;     // block scan scratch (64 words)
    uint2 *plist;      // children that need a palette op: (op index, label), one 256-op chunk at a time
    __device__ EncSmem(uint8_t *s, const EncGeom &G) {
        // every region starts on a 16-byte boundary (the rANS phase stages symbols with 16-byte stores)
        lab = (uint32_t *)s;
        cst = (uint8_t *)s + r16(G.up_nodes * 4);
        list = (uint16_t *)(cst + r16(G.up_nodes));
        ops = (uint8_t *)list + r16(G.up_nodes * 2);
        red = (uint32_t *)(ops + r16(G.ops_cap));
        plist = (uint2 *)(red + 64);
    }
    __host__ __device__ static uint32_t r16(uint32_t x) { return (x + 15u) & ~15u; }
};

__host__ __device__ inline uint32_t enc_smem_bytes(uint32_t up_nodes, uint32_t ops_cap) {
    return EncSmem::r16(up_nodes * 4) + EncSmem::r16(up_nodes) + EncSmem::r16(up_nodes * 2) + EncSmem::r16(ops_cap) +
           64 * 4 + 256 * 8;
}

// exclusive block scan of one value per warp (warp totals in `red`), returns warp's offset and the total
__device__ __forceinline__ uint32_t block_excl_warp(uint32_t *red, uint32_t warp_total, uint32_t &total) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = warp_total;
    __syncthreads();
    uint32_t off = 0, tot = 0;
    for (uint32_t w = 0; w < kEncWarps; w++) {
        const uint32_t v = red[w];
        if (w < warp) off += v;
        tot += v;
    }
    __syncthreads();
    total = tot;
    return off;
}

// label of node q (Morton) on level l of the brick
__device__ __forceinline__ uint32_t node_label(const Brick &B, const EncSmem &S, const EncGeom &G, uint32_t l,
                                               uint32_t q) {
    if (l == 0) return B.at(compact5(q), compact5(q >> 1), compact5(q >> 2));
    return S.lab[G.off[l] + q];
}

// Encode (or, when count != nullptr, only count the nibbles of) one brick.
__global__ void __launch_bounds__(kEncThreads)
    encode_kernel(EncVol EV, EncGeom G, uint64_t brick0, uint64_t brick_stride, uint32_t n_in_batch,
                  const uint32_t *freq, EncScratch SC, unsigned long long *count) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    EncSmem S(smem_raw, G);
    __shared__ uint32_t hist[32];
    __shared__ uint32_t sh_np;
    __shared__ uint32_t lvl_base[kMaxN + 2], lvl_nact[kMaxN + 2];  // ops of children of parent level l
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
    if (tid < 32) hist[tid] = 0;

    // ---- A. pyramid
    {
        const uint32_t B1 = b >> 1, n1 = B1 * B1 * B1;
#pragma unroll 2
        for (uint32_t i = tid; i < n1; i += kEncThreads) {
            const uint32_t x = i % B1, y = (i / B1) % B1, z = i / (B1 * B1);
            uint32_t w[8];
#pragma unroll
            for (int c = 0; c < 8; c++) w[c] = B.at(2 * x + (c & 1), 2 * y + ((c >> 1) & 1), 2 * z + ((c >> 2) & 1));
            bool eq;
            const uint32_t m = morton3(x, y, z);
            S.lab[G.off[1] + m] = mode8(w, eq);
            S.cst[G.off[1] + m] = eq;
        }
        __syncthreads();
        for (uint32_t l = 2; l <= N; l++) {
            const uint32_t Bl = b >> l, nl = Bl * Bl * Bl;
            for (uint32_t i = tid; i < nl; i += kEncThreads) {
                uint32_t w[8];
                bool allc = true;
#pragma unroll
                for (int c = 0; c < 8; c++) {
                    w[c] = S.lab[G.off[l - 1] + 8 * i + c];
                    allc = allc && S.cst[G.off[l - 1] + 8 * i + c];
                }
                bool eq;
                S.lab[G.off[l] + i] = mode8(w, eq);
                S.cst[G.off[l] + i] = eq && allc;
            }
            __syncthreads();
        }
    }

    // ---- B. active parent lists and reuse operations, level by level (Alg. 2 traversal)
    uint32_t n_ops = 0, n_int_ops = 0;
    for (uint32_t l = N; l >= 1; l--) {
        const uint32_t Bl = b >> l, nl = Bl * Bl * Bl;
        // compact the active parents of level l (Morton order)
        uint32_t n_act = 0;
        for (uint32_t g = 0; g < nl; g += kEncThreads) {
            const uint32_t i = g + tid;
            const bool act = i < nl && !S.cst[G.off[l] + i];
            const uint32_t m = __ballot_sync(kFull, act);
            uint32_t tot;
            const uint32_t woff = block_excl_warp(S.red, __popc(m), tot);
            if (act) S.list[G.off[l] + n_act + woff + __popc(m & lanemask_lt())] = (uint16_t)i;
            n_act += tot;
        }
        __syncthreads();
        const uint32_t lc = l - 1;
        const uint32_t nops_l = 8 * n_act;
        if (tid == 0) {
            lvl_base[l] = n_ops;
            lvl_nact[l] = n_act;
        }
        const uint32_t cbits = (1u << (3 * (N - lc))) - 1u;  // Morton code bits of the child level
        for (uint32_t j = tid; j < nops_l; j += kEncThreads) {
            const uint32_t p = S.list[G.off[l] + (j >> 3)], c = j & 7u;
            const uint32_t q = 8 * p + c;
            // every label the choice can look at, loaded up front (independent loads); a neighbour index
            // that would leave the brick wraps to an in-brick node and is ignored through ok[]
            uint32_t nv[3];
            bool ok[3];
#pragma unroll
            for (uint32_t a = 0; a < 3; a++) {
                const uint32_t ma = (kMX << a) & cbits;
                const bool minus = ((c >> a) & 1u) == 0;
                ok[a] = minus ? (q & ma) != 0 : (q & ma) != ma;
                nv[a] = minus ? node_label(B, S, G, lc, mdec(q, ma)) : S.lab[G.off[l] + (minc(q, ma) >> 3)];
            }
            const uint32_t v = node_label(B, S, G, lc, q);
            const uint32_t parent = S.lab[G.off[l] + p];
            const uint32_t stop = lc >= 1 ? (uint32_t)S.cst[G.off[lc] + q] : 0u;
            // first applicable reuse: R_p, R_x, R_y, R_z (bestOperation order)
            const uint32_t op = v == parent ? OP_RP
                                : (ok[0] && nv[0] == v) ? OP_RX
                                : (ok[1] && nv[1] == v) ? OP_RY
                                : (ok[2] && nv[2] == v) ? OP_RZ
                                : kNeedPal;
            S.ops[n_ops + j] = (uint8_t)(op | (stop << 3));
        }
        n_ops += nops_l;
        if (lc >= 1) n_int_ops = n_ops;
        __syncthreads();
    }

    // ---- C. palette pass in stream order: all warps collect the children no reuse fits (with their
    // labels), 256 ops at a time; warp 0 then walks them in order with the last 17 palette entries in
    // registers (lane i holds palette[i_p - i])
    {
        const uint32_t root = S.lab[G.off[N]];
        uint32_t win = root;
        uint32_t ip = 0, np = 1;  // i_p and palette size (kept by warp 0)
        uint32_t *pal = count ? nullptr : SC.pal + (size_t)slot * G.pal_cap;
        if (pal && tid == 0) pal[0] = root;
        for (uint32_t g = 0; g < n_ops; g += kEncThreads) {
            const uint32_t j = g + tid;
            const bool need = j < n_ops && (S.ops[j] & 7u) == kNeedPal;
            const uint32_t m = __ballot_sync(kFull, need);
            uint32_t tot;
            const uint32_t woff = block_excl_warp(S.red, __popc(m), tot);
            if (tot == 0) continue;
            if (need) {
                uint32_t l = 1;
                for (uint32_t L = N; L >= 2; L--)
                    if (j >= lvl_base[L] && j < lvl_base[L] + 8 * lvl_nact[L]) l = L;
                const uint32_t base = lvl_base[l];
                const uint32_t p = S.list[G.off[l] + ((j - base) >> 3)];
                S.plist[woff + __popc(m & lanemask_lt())] = make_uint2(j, node_label(B, S, G, l - 1, 8 * p + ((j - base) & 7u)));
            }
            __syncthreads();
            if (warp == 0) {
                for (uint32_t k = 0; k < tot; k++) {
                    const uint2 e = S.plist[k];
                    const uint32_t vk = e.y;
                    const bool match = lane <= 16 && lane <= ip && win == vk;
                    const uint32_t mm = __ballot_sync(kFull, match);
                    uint32_t op, delta = 0;
                    if (mm) {
                        const uint32_t f = __ffs(mm) - 1;
                        op = f == 0 ? OP_P0 : OP_PD;
                        delta = f == 0 ? 0u : f - 1;
                    } else {
                        op = OP_PA;
                        const uint32_t up = __shfl_up_sync(kFull, win, 1);
                        win = lane == 0 ? vk : up;
                        if (pal && lane == 0) pal[np] = vk;
                        ip += 1;
                        np += 1;
                    }
                    if (lane == 0) S.ops[e.x] = (uint8_t)((S.ops[e.x] & 8u) | op | (delta << 4));
                }
            }
            __syncthreads();
        }
        if (tid == 0) sh_np = np;
    }
    __syncthreads();

    // ---- D. nibble positions: per op 1 nibble, +1 after P_delta; each warp takes a contiguous range
    uint32_t sym_tot[2];
    {
        const uint32_t per = ((n_ops + kEncWarps - 1) / kEncWarps + 31) & ~31u;
        const uint32_t j0 = warp * per, j1 = min(n_ops, j0 + per);
        // pass 1: symbols of this warp's range in each stream
        uint32_t cnt[2] = {0, 0};
        for (uint32_t g = j0; g < j1; g += 32) {
            const uint32_t j = g + lane;
            const bool in = j < j1;
            const uint32_t o = in ? S.ops[j] : 0u;
            const uint32_t s = in ? 1u + ((o & 7u) == OP_PD) : 0u;
            const bool leaf = j >= n_int_ops;
            uint32_t tot = s;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) tot += __shfl_xor_sync(kFull, tot, d);
            uint32_t tl = leaf ? s : 0u;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) tl += __shfl_xor_sync(kFull, tl, d);
            cnt[1] += tl;
            cnt[0] += tot - tl;
        }
        uint32_t base[2];
        for (int st = 0; st < 2; st++) base[st] = block_excl_warp(S.red, cnt[st], sym_tot[st]);
        // pass 2: write or count
        uint32_t run[2] = {base[0], base[1]};
        uint8_t *nib[2] = {nullptr, nullptr};
        if (!count) {
            nib[0] = SC.nib_int + (size_t)slot * G.int_cap;
            nib[1] = SC.nib_leaf + (size_t)slot * G.leaf_cap;
        }
        for (uint32_t g = j0; g < j1; g += 32) {
            const uint32_t j = g + lane;
            const bool in = j < j1;
            const uint32_t o = in ? S.ops[j] : 0u;
            const uint32_t op = o & 7u;
            const bool pd = in && op == OP_PD;
            const uint32_t s = in ? 1u + pd : 0u;
            const uint32_t st = j >= n_int_ops ? 1u : 0u;
            // inclusive scan of s among lanes of the same stream (streams split the range at most once)
            uint32_t inc = s;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t u = __shfl_up_sync(kFull, inc, d);
                const uint32_t ust = __shfl_up_sync(kFull, st, d);
                if (lane >= (uint32_t)d && ust == st) inc += u;
            }
            const uint32_t pos = run[st] + inc - s;
            const uint32_t nibble = op | (o & 8u);
            const uint32_t delta = o >> 4;
            if (in) {
                if (count) {
                    atomicAdd(&hist[16 * st + nibble], 1u);
                    if (pd) atomicAdd(&hist[16 * st + delta], 1u);
                } else {
                    nib[st][pos] = (uint8_t)nibble;
                    if (pd) nib[st][pos + 1] = (uint8_t)delta;
                }
            }
            // advance both runs by this tile's totals per stream
            uint32_t t0 = st == 0 ? s : 0u, t1 = st == 1 ? s : 0u;
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) {
                t0 += __shfl_xor_sync(kFull, t0, d);
                t1 += __shfl_xor_sync(kFull, t1, d);
            }
            run[0] += t0;
            run[1] += t1;
        }
    }
    if (count) {
        __syncthreads();
        if (tid < 32 && hist[tid]) atomicAdd(count + tid, (unsigned long long)hist[tid]);
        return;
    }
    __syncthreads();  // nibbles visible to the rANS warps

    // ---- E. rANS, one warp per stream; the symbols are staged in shared memory (the op array is free now)
    if (warp < 2) {
        const uint32_t st = warp;
        const uint32_t n = sym_tot[st];
        const uint32_t cap = (st == 0 ? G.int_cap : G.leaf_cap) + 64;
        uint16_t *words = (st == 0 ? SC.w_int : SC.w_leaf) + (size_t)slot * cap;
        const uint8_t *nib = st == 0 ? SC.nib_int + (size_t)slot * G.int_cap : SC.nib_leaf + (size_t)slot * G.leaf_cap;
        const uint32_t half = (G.ops_cap / 2) & ~15u;  // staging bytes per stream
        uint8_t *wsm = S.ops + st * half;
        const uint32_t *F = freq + 16 * st;
        const uint32_t f_reg = lane < 16 ? F[lane] : 1u;
        const float rcp_reg = 1.0f / (float)f_reg;
        uint32_t c_reg = 0;
        for (uint32_t s2 = 0; s2 < 16; s2++) c_reg += (s2 < lane) ? F[s2] : 0u;
        const uint32_t K = lanes_for(n, G.K_max, G.S_min);
        uint32_t top = cap;
        if (n > 0) {
            uint32_t x = kL;
            const uint32_t steps = (n + K - 1) / K;
            const uint32_t win_steps = (half - 16) / K;  // steps per staged window (16 bytes of alignment slack)
            // windows of steps from the end: [s_lo, s_hi) covers symbols [s_lo*K, min(n, s_hi*K))
            for (uint32_t s_hi = steps; s_hi > 0;) {
                const uint32_t s_lo = s_hi > win_steps ? s_hi - win_steps : 0u;
                const uint32_t lo16 = (s_lo * K) & ~15u, sym_hi = min(n, s_hi * K);
                for (uint32_t c16 = lane; lo16 + 16 * c16 < sym_hi; c16 += 32)
                    reinterpret_cast<uint4 *>(wsm)[c16] = __ldcg(reinterpret_cast<const uint4 *>(nib + lo16) + c16);
                __syncwarp();
                for (uint32_t s2 = s_hi; s2-- > s_lo;) {
                    const uint32_t i = s2 * K + lane;
                    const bool act = lane < K && i < n;
                    const uint32_t sym = act ? (uint32_t)wsm[i - lo16] : 0u;
                    const uint32_t f = __shfl_sync(kFull, f_reg, sym), c = __shfl_sync(kFull, c_reg, sym);
                    const float rf = __shfl_sync(kFull, rcp_reg, sym);
                    // renormalise before coding: keep x below f * 2^20 (one 16-bit word at most)
                    const bool emit = act && x >= (f << 20);
                    const uint32_t m = __ballot_sync(kFull, emit);
                    if (emit) {
                        words[top - __popc(m) + __popc(m & lanemask_lt())] = (uint16_t)(x & 0xFFFFu);
                        x >>= 16;
                    }
                    top -= __popc(m);
                    if (act) {
                        // x / f through a float reciprocal: here x < f * 2^20, so the estimate is within one of
                        // the quotient; the integer remainder check makes it exact
                        uint32_t qt = __float2uint_rz(__uint2float_rz(x) * rf);
                        int32_t r = (int32_t)(x - qt * f);
                        if (r < 0) { qt -= 1; r += (int32_t)f; }
                        if (r < 0) { qt -= 1; r += (int32_t)f; }
                        if (r >= (int32_t)f) { qt += 1; r -= (int32_t)f; }
                        if (r >= (int32_t)f) { qt += 1; r -= (int32_t)f; }
                        x = qt * kM + (uint32_t)r + c;
                    }
                }
                __syncwarp();
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
            uint32_t *sz = SC.sizes + (size_t)slot * 8;
            sz[3 + st] = cap - top;  // words
            sz[5 + st] = top;        // start inside the scratch area
        }
    }
    if (tid == 0) {
        uint32_t *sz = SC.sizes + (size_t)slot * 8;
        sz[0] = sh_np;
        sz[1] = sym_tot[0];
        sz[2] = sym_tot[1];
        sz[7] = 0;
    }
}

// Exclusive scan of per-brick sizes (palette labels, interior words, leaf words) of one batch into the
// volume's offset arrays, continuing from the running totals in tot[0..2]; writes the new totals.
__global__ void __launch_bounds__(1024) scan_sizes_kernel(const uint32_t *sizes, uint32_t n, uint64_t first,
                                                          uint64_t *pal_off, uint64_t *int_off, uint64_t *leaf_off,
                                                          uint64_t *tot) {
    __shared__ unsigned long long part[3][32];
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned long long run[3] = {tot[0], tot[1], tot[2]};
    for (uint32_t g = 0; g < n; g += 1024) {
        const uint32_t i = g + tid;
        unsigned long long v[3] = {0, 0, 0};
        if (i < n) {
            v[0] = sizes[8 * (size_t)i + 0];
            v[1] = sizes[8 * (size_t)i + 3];
            v[2] = sizes[8 * (size_t)i + 4];
        }
        unsigned long long inc[3] = {v[0], v[1], v[2]};
#pragma unroll
        for (int a = 0; a < 3; a++)
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long u = __shfl_up_sync(kFull, inc[a], d);
                if (lane >= (uint32_t)d) inc[a] += u;
            }
        if (lane == 31)
            for (int a = 0; a < 3; a++) part[a][warp] = inc[a];
        __syncthreads();
        unsigned long long wo[3] = {0, 0, 0}, bt[3] = {0, 0, 0};
        for (uint32_t w = 0; w < 32; w++)
            for (int a = 0; a < 3; a++) {
                if (w < warp) wo[a] += part[a][w];
                bt[a] += part[a][w];
            }
        if (i < n) {
            pal_off[first + i] = run[0] + wo[0] + inc[0] - v[0];
            int_off[first + i] = run[1] + wo[1] + inc[1] - v[1];
            leaf_off[first + i] = run[2] + wo[2] + inc[2] - v[2];
        }
        for (int a = 0; a < 3; a++) run[a] += bt[a];
        __syncthreads();
    }
    if (tid == 0) {
        tot[0] = run[0];
        tot[1] = run[1];
        tot[2] = run[2];
        pal_off[first + n] = run[0];
        int_off[first + n] = run[1];
        leaf_off[first + n] = run[2];
    }
}

// Copy each brick's palette and words from scratch to the packed arrays.
__global__ void __launch_bounds__(256) compact_kernel(EncGeom G, EncScratch SC, uint64_t first, const uint64_t *pal_off,
                                                      const uint64_t *int_off, const uint64_t *leaf_off, uint32_t *pal,
                                                      uint16_t *int_words, uint16_t *leaf_words, uint32_t *n_int_sym,
                                                      uint32_t *n_leaf_sym, uint32_t *max_pal) {
    const uint32_t slot = blockIdx.x;
    const uint32_t *sz = SC.sizes + (size_t)slot * 8;
    const uint64_t id = first + slot;
    const uint32_t np = sz[0], nwi = sz[3], nwl = sz[4], si = sz[5], sl = sz[6];
    const uint32_t *ps = SC.pal + (size_t)slot * G.pal_cap;
    const uint16_t *wi = SC.w_int + (size_t)slot * (G.int_cap + 64) + si;
    const uint16_t *wl = SC.w_leaf + (size_t)slot * (G.leaf_cap + 64) + sl;
    uint32_t *pd = pal + pal_off[id];
    uint16_t *di = int_words + int_off[id], *dl = leaf_words + leaf_off[id];
    for (uint32_t k = threadIdx.x; k < np; k += blockDim.x) pd[k] = ps[k];
    for (uint32_t k = threadIdx.x; k < nwi; k += blockDim.x) di[k] = wi[k];
    for (uint32_t k = threadIdx.x; k < nwl; k += blockDim.x) dl[k] = wl[k];
    if (threadIdx.x == 0) {
        n_int_sym[id] = sz[1];
        n_leaf_sym[id] = sz[2];
        atomicMax(max_pal, np);  // max_pal[0..2]: largest palette, interior and leaf symbol counts
        atomicMax(max_pal + 1, sz[1]);
        atomicMax(max_pal + 2, sz[2]);
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
    G.ops_cap = u + b3 - 1 > 256u ? u + b3 - 1 : 256u;  // every node but the root can be coded (>= 256: rANS staging)
    G.pal_cap = u + b3;             // palette: root + one per P_a
    G.int_cap = (2 * (u - 1) + 2 + 15) & ~15u;  // interior nibbles (op + delta each), 16-byte pitch
    G.leaf_cap = (2 * b3 + 15) & ~15u;
    G.smem = enc_smem_bytes(G.up_nodes, G.ops_cap);
    G.K_max = K_max;
    G.S_min = S_min;
    return G;
}

size_t scratch_bytes_per_brick(const EncGeom &G) {
    return (size_t)G.pal_cap * 4 + G.int_cap + G.leaf_cap + (size_t)(G.int_cap + 64) * 2 +
           (size_t)(G.leaf_cap + 64) * 2 + 8 * 4 + 64;
}

cudaError_t launch_encode(const EncVol &EV, const EncGeom &G, uint64_t brick0, uint64_t stride, uint32_t n,
                          const uint32_t *freq, const EncScratch &SC, unsigned long long *count, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, G.smem);
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    encode_kernel<<<n, kEncThreads, G.smem, st>>>(EV, G, brick0, stride, n, freq, SC, count);
    return cudaGetLastError();
}

cudaError_t launch_scan(const uint32_t *sizes, uint32_t n, uint64_t first, uint64_t *pal_off, uint64_t *int_off,
                        uint64_t *leaf_off, uint64_t *tot, cudaStream_t st) {
    scan_sizes_kernel<<<1, 1024, 0, st>>>(sizes, n, first, pal_off, int_off, leaf_off, tot);
    return cudaGetLastError();
}

cudaError_t launch_compact(const EncGeom &G, const EncScratch &SC, uint64_t first, uint32_t n, const uint64_t *pal_off,
                           const uint64_t *int_off, const uint64_t *leaf_off, uint32_t *pal, uint16_t *int_words,
                           uint16_t *leaf_words, uint32_t *n_int_sym, uint32_t *n_leaf_sym, uint32_t *max_pal,
                           cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    compact_kernel<<<n, 256, 0, st>>>(G, SC, first, pal_off, int_off, leaf_off, pal, int_words, leaf_words, n_int_sym,
                                      n_leaf_sym, max_pal);
    return cudaGetLastError();
}


}  // namespace csgv
