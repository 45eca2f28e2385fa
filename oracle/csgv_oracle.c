/*
 * csgv_oracle.c -- plain, slow CPU oracle of the compressed segmentation
 * volume (CSV) brick codec of Piochowiak & Dachsbacher, "Fast Compressed
 * Segmentation Volumes for Scientific Visualization" (IEEE TVCG 2023).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code:
 * only the tests, __graft_entry__.smoke() and the CPU-baseline leg of bench.py
 * load it.  It shares no code, header, table or constant with the CUDA
 * library; the two meet only through the byte layout described below, which
 * each side implements on its own.
 *
 * What it computes, step by step in the paper's order:
 *   - bricking, b = 2^N, clamp-to-edge padding ............ Sec. 3.1
 *   - resolution pyramid L_0..L_N, mode of 8 children,
 *     ties to the first occurrence in the child array,
 *     "constantChildren" (stop) flags ...................... Sec. 3.1, 3.4
 *   - brick encoding: coarse-to-fine Morton traversal, the
 *     seven operations tried in the order
 *     R_p, R_x, R_y, R_z, P_0, P_delta, P_a ................ Sec. 3.2, Alg. 2, 3.4
 *   - brick decoding to a level of detail t ............... Alg. 1, Sec. 3.4
 *   - two static nibble frequency tables (interior / leaf)
 *     from a prepass over every s-th brick .................. Sec. 3.3, 3.4
 *   - rANS entropy coding of the nibble streams ............ Sec. 3.3
 *
 * Readings where the paper is silent or inconsistent (numbered as in the
 * design notes of this repository):
 *   R1  P_delta refers to palette[i_p - 1 - delta] (Sec. 3.2 text); P_0 is
 *       palette[i_p].
 *   R2  No nibble for the root: a brick is homogeneous iff it has no symbols;
 *       then its palette is the single root label.
 *   R3  i_p moves only on P_a.
 *   R4  R_a (a in x,y,z) looks out of the 2^3 sibling block: if the child's
 *       a-bit is 0 it reads the same-level node at -1 along a (earlier in
 *       Z-order, already decoded); if the a-bit is 1 the node at +1 is not yet
 *       decoded, so it reads that node's parent on the coarser level.  A
 *       neighbour outside the brick makes the operation inapplicable.
 *   R5  Morton child index c = x | y<<1 | z<<2 at every level.
 *   R6  op codes R_p=0 R_x=1 R_y=2 R_z=3 P_0=4 P_delta=5 P_a=6 (7 invalid);
 *       nibble = op | stop<<3; a P_delta nibble is followed by its delta
 *       nibble in the same stream (decode order).
 *   R9  rANS: 32-bit state, scale M = 4096, lower bound L = 2^16, 16-bit
 *       words, at most one word per symbol.
 *   R10 K interleaved states per stream, K = clamp(n / S_min, 1, K_max)
 *       with n the stream's nibble count.  The j-th op nibble of the stream
 *       uses state j mod K, and the delta nibble of a P_delta op uses the
 *       same state as its op.  Coding order, step by step: step t holds the
 *       ops tK .. tK+K-1 in state order, then the delta nibbles of those of
 *       them that are P_delta, again in state order.  Stream = K final
 *       states (low half first, state 0 first) followed by the
 *       renormalisation words in coding order.  With K = 1 the coding order
 *       is the nibble order itself.
 *   R11 table: f_s = 1 + floor(count_s * (M - 16) / total), the remaining
 *       r < 16 units go +1 to the r largest counts (ties: lower symbol);
 *       total = 0 gives f_s = 256.
 *   R12 prepass samples bricks with id % stride == 0.
 *
 * The oracle keeps every pyramid level in its own array.  The paper's
 * decoder writes all levels in place into one output block (Sec. 3.4); that
 * saves memory but yields the same labels.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ------------------------------------------------------------------ */
/* error codes (oracle-local)                                          */
/* ------------------------------------------------------------------ */
#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_CORRUPT 2
#define ORC_ERR_NOMEM 3

/* operation codes, reading R6 */
enum { OP_RP = 0, OP_RX = 1, OP_RY = 2, OP_RZ = 3, OP_P0 = 4, OP_PD = 5, OP_PA = 6 };

#define RANS_SCALE_BITS 12u
#define RANS_M (1u << RANS_SCALE_BITS)
#define RANS_L (1u << 16)

/* ------------------------------------------------------------------ */
/* small helpers                                                       */
/* ------------------------------------------------------------------ */

/* Morton index -> coordinate: bit 3k of m is bit k of x, 3k+1 of y, 3k+2 of z (R5). */
static void morton_decode(uint64_t m, uint32_t *x, uint32_t *y, uint32_t *z) {
    uint32_t xx = 0, yy = 0, zz = 0;
    for (int k = 0; k < 21; k++) {
        xx |= (uint32_t)((m >> (3 * k)) & 1u) << k;
        yy |= (uint32_t)((m >> (3 * k + 1)) & 1u) << k;
        zz |= (uint32_t)((m >> (3 * k + 2)) & 1u) << k;
    }
    *x = xx; *y = yy; *z = zz;
}

/* number of nodes of a level with side B */
static uint64_t cube(uint64_t B) { return B * B * B; }

/* offset of level l in the concatenated pyramid arrays (level 0 first) */
static uint64_t level_offset(int N, int l) {
    uint64_t off = 0;
    for (int k = 0; k < l; k++) off += cube((uint64_t)1 << (N - k));
    return off;
}

uint64_t csgvo_pyramid_nodes(int N) { return level_offset(N, N + 1); }

/* ------------------------------------------------------------------ */
/* Sec. 3.1: resolution pyramid                                        */
/* ------------------------------------------------------------------ */

/*
 * Build L_0..L_N of one brick (x-fastest b^3 labels).  lab/cst hold the
 * levels concatenated, level 0 first, each level x-fastest with side b>>l.
 * L_l[p] is the most frequent label among the 8 children of p on L_{l-1};
 * among equally frequent labels the one occurring first in the child array
 * (child index c, R5) wins (Sec. 3.4).  cst[p] = 1 iff every voxel under p has
 * the same label ("constantChildren"); on L_0 it is 1 by definition.
 */
int csgvo_pyramid(const uint32_t *brick, int N, uint32_t *lab, uint8_t *cst) {
    if (N < 1 || N > 6) return ORC_ERR_ARG;
    uint32_t b = 1u << N;
    memcpy(lab, brick, sizeof(uint32_t) * cube(b));
    memset(cst, 1, cube(b));
    for (int l = 1; l <= N; l++) {
        uint32_t B = b >> l, Bc = B * 2;
        uint32_t *L = lab + level_offset(N, l);
        uint8_t *C = cst + level_offset(N, l);
        const uint32_t *Lc = lab + level_offset(N, l - 1);
        const uint8_t *Cc = cst + level_offset(N, l - 1);
        for (uint32_t z = 0; z < B; z++)
            for (uint32_t y = 0; y < B; y++)
                for (uint32_t x = 0; x < B; x++) {
                    uint32_t w[8];
                    int all_const = 1;
                    for (int c = 0; c < 8; c++) {
                        uint32_t cx = 2 * x + (c & 1), cy = 2 * y + ((c >> 1) & 1), cz = 2 * z + ((c >> 2) & 1);
                        uint64_t qi = cx + (uint64_t)Bc * (cy + (uint64_t)Bc * cz);
                        w[c] = Lc[qi];
                        all_const &= Cc[qi];
                    }
                    uint32_t best = w[0];
                    int best_cnt = 0;
                    for (int c = 0; c < 8; c++) {
                        int cnt = 0;
                        for (int d = 0; d < 8; d++) cnt += (w[d] == w[c]);
                        if (cnt > best_cnt) { best_cnt = cnt; best = w[c]; }
                    }
                    uint64_t pi = x + (uint64_t)B * (y + (uint64_t)B * z);
                    L[pi] = best;
                    C[pi] = (uint8_t)(all_const && best_cnt == 8);
                }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Sec. 3.2 / Alg. 2: brick encoding                                   */
/* ------------------------------------------------------------------ */

typedef struct {
    uint8_t *nib;
    uint32_t n, cap;
} nibbuf;

static int put_nib(nibbuf *s, uint32_t v) {
    if (s->n >= s->cap) return ORC_ERR_ARG;
    s->nib[s->n++] = (uint8_t)v;
    return ORC_OK;
}

/*
 * Value that neighbour reuse along axis a gives child (qx,qy,qz) on level
 * lc = l-1, per reading R4.  Returns 0 if the operation is not applicable
 * (neighbour outside the brick), 1 with *val set otherwise.
 */
static int neighbour_value(const uint32_t *lab, int N, int lc, uint32_t qx, uint32_t qy, uint32_t qz,
                           int axis, uint32_t *val) {
    uint32_t Bc = (1u << N) >> lc;
    uint32_t q[3] = {qx, qy, qz};
    uint32_t bit = q[axis] & 1u;
    if (bit == 0) {
        /* -1 along axis: same level, earlier in Z-order */
        if (q[axis] == 0) return 0;
        q[axis] -= 1;
        const uint32_t *L = lab + level_offset(N, lc);
        *val = L[q[0] + (uint64_t)Bc * (q[1] + (uint64_t)Bc * q[2])];
        return 1;
    }
    /* +1 along axis: not yet decoded, use its parent on level lc+1 */
    if (q[axis] + 1 >= Bc) return 0;
    q[axis] += 1;
    uint32_t Bp = Bc / 2;
    const uint32_t *Lp = lab + level_offset(N, lc + 1);
    *val = Lp[(q[0] >> 1) + (uint64_t)Bp * ((q[1] >> 1) + (uint64_t)Bp * (q[2] >> 1))];
    return 1;
}

/*
 * Encode one brick (Alg. 2).  Outputs the palette and two nibble streams:
 * children on levels >= 1 go to the interior stream, children on level 0 to
 * the leaf stream (Sec. 3.3: two tables, leaf stop bits always 0).
 * Capacities: palette >= pyramid nodes, int_nib >= 2 * interior children,
 * leaf_nib >= 2 * b^3.
 */
int csgvo_encode_brick(const uint32_t *brick, int N,
                       uint32_t *palette, uint32_t pal_cap, uint32_t *n_palette,
                       uint8_t *int_nib, uint32_t int_cap, uint32_t *n_int,
                       uint8_t *leaf_nib, uint32_t leaf_cap, uint32_t *n_leaf,
                       uint64_t op_counts[7]) {
    if (N < 1 || N > 6) return ORC_ERR_ARG;
    uint64_t nodes = csgvo_pyramid_nodes(N);
    uint32_t *lab = (uint32_t *)malloc(nodes * sizeof(uint32_t));
    uint8_t *cst = (uint8_t *)malloc(nodes);
    if (!lab || !cst) { free(lab); free(cst); return ORC_ERR_NOMEM; }
    int rc = csgvo_pyramid(brick, N, lab, cst);
    if (rc) { free(lab); free(cst); return rc; }

    nibbuf sint = {int_nib, 0, int_cap}, sleaf = {leaf_nib, 0, leaf_cap};
    uint32_t np = 0;
    /* palette <- root label; i_p = 0 (Sec. 3.2) */
    palette[np++] = lab[level_offset(N, N)];
    uint32_t ip = 0;

    for (int l = N; l >= 1 && rc == ORC_OK; l--) {
        uint32_t B = (1u << N) >> l;
        const uint32_t *L = lab + level_offset(N, l);
        const uint8_t *C = cst + level_offset(N, l);
        const uint32_t *Lc = lab + level_offset(N, l - 1);
        const uint8_t *Cc = cst + level_offset(N, l - 1);
        uint32_t Bc = 2 * B;
        nibbuf *out = (l - 1 >= 1) ? &sint : &sleaf;
        for (uint64_t m = 0; m < cube(B) && rc == ORC_OK; m++) {
            uint32_t px, py, pz;
            morton_decode(m, &px, &py, &pz);
            uint64_t pi = px + (uint64_t)B * (py + (uint64_t)B * pz);
            if (C[pi]) continue; /* constantChildren: nothing below is coded */
            uint32_t parent = L[pi];
            for (int c = 0; c < 8 && rc == ORC_OK; c++) {
                uint32_t qx = 2 * px + (c & 1), qy = 2 * py + ((c >> 1) & 1), qz = 2 * pz + ((c >> 2) & 1);
                uint64_t qi = qx + (uint64_t)Bc * (qy + (uint64_t)Bc * qz);
                uint32_t v = Lc[qi];
                uint32_t stop = (l - 1 >= 1) ? Cc[qi] : 0u;
                /* bestOperation: first applicable of R_p, R_x, R_y, R_z, P_0, P_delta, P_a */
                int op = -1;
                uint32_t delta = 0;
                if (v == parent) op = OP_RP;
                for (int a = 0; a < 3 && op < 0; a++) {
                    uint32_t nv;
                    if (neighbour_value(lab, N, l - 1, qx, qy, qz, a, &nv) && nv == v) op = OP_RX + a;
                }
                if (op < 0 && palette[ip] == v) op = OP_P0;
                for (uint32_t d = 0; d < 16 && op < 0; d++) {
                    if (ip >= 1 + d && palette[ip - 1 - d] == v) { op = OP_PD; delta = d; }
                }
                if (op < 0) {
                    op = OP_PA;
                    if (np >= pal_cap) { rc = ORC_ERR_ARG; break; }
                    palette[np++] = v;
                    ip += 1;
                }
                if (op_counts) op_counts[op]++;
                rc = put_nib(out, (uint32_t)op | (stop << 3));
                if (rc == ORC_OK && op == OP_PD) rc = put_nib(out, delta);
            }
        }
    }
    *n_palette = np;
    *n_int = sint.n;
    *n_leaf = sleaf.n;
    free(lab);
    free(cst);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Alg. 1: brick decoding to level of detail t                         */
/* ------------------------------------------------------------------ */

typedef struct {
    const uint8_t *nib;
    uint32_t n, pos;
} nibreader;

static int get_nib(nibreader *r, uint32_t *v) {
    if (r->pos >= r->n) return ORC_ERR_CORRUPT;
    *v = r->nib[r->pos++];
    return ORC_OK;
}

/*
 * Decode one brick from its palette and nibble streams to LOD t
 * (0 <= t <= N); out receives (b>>t)^3 labels, x-fastest.  The leaf stream is
 * only read for t == 0.  Returns ORC_ERR_CORRUPT for any stream that does not
 * follow the format (invalid op, stop bit on a leaf, palette index out of
 * range, neighbour outside the brick, stream too short or not fully used).
 */
int csgvo_decode_brick(const uint32_t *palette, uint32_t n_palette,
                       const uint8_t *int_nib, uint32_t n_int,
                       const uint8_t *leaf_nib, uint32_t n_leaf,
                       int N, int t, uint32_t *out) {
    if (N < 1 || N > 6 || t < 0 || t > N || n_palette < 1) return ORC_ERR_ARG;
    uint64_t nodes = csgvo_pyramid_nodes(N);
    uint32_t *lab = (uint32_t *)calloc(nodes, sizeof(uint32_t));
    uint8_t *cst = (uint8_t *)calloc(nodes, 1);
    if (!lab || !cst) { free(lab); free(cst); return ORC_ERR_NOMEM; }
    int rc = ORC_OK;
    nibreader rint = {int_nib, n_int, 0}, rleaf = {leaf_nib, n_leaf, 0};

    /* out[0] = palette[i_p], i_p = 0; a brick without symbols is constant (R2) */
    uint32_t ip = 0;
    lab[level_offset(N, N)] = palette[0];
    cst[level_offset(N, N)] = (uint8_t)(n_int == 0 && n_leaf == 0);

    for (int l = N; l >= t + 1 && rc == ORC_OK; l--) {
        uint32_t B = (1u << N) >> l, Bc = 2 * B;
        const uint32_t *L = lab + level_offset(N, l);
        const uint8_t *C = cst + level_offset(N, l);
        uint32_t *Lc = lab + level_offset(N, l - 1);
        uint8_t *Cc = cst + level_offset(N, l - 1);
        nibreader *in = (l - 1 >= 1) ? &rint : &rleaf;
        for (uint64_t m = 0; m < cube(B) && rc == ORC_OK; m++) {
            uint32_t px, py, pz;
            morton_decode(m, &px, &py, &pz);
            uint64_t pi = px + (uint64_t)B * (py + (uint64_t)B * pz);
            uint32_t parent = L[pi];
            for (int c = 0; c < 8 && rc == ORC_OK; c++) {
                uint32_t qx = 2 * px + (c & 1), qy = 2 * py + ((c >> 1) & 1), qz = 2 * pz + ((c >> 2) & 1);
                uint64_t qi = qx + (uint64_t)Bc * (qy + (uint64_t)Bc * qz);
                if (C[pi]) {
                    /* constant area: the sub-block takes the parent's label */
                    Lc[qi] = parent;
                    Cc[qi] = 1;
                    continue;
                }
                uint32_t nib, v = 0;
                rc = get_nib(in, &nib);
                if (rc) break;
                uint32_t op = nib & 7u, stop = nib >> 3;
                if (stop && l - 1 == 0) { rc = ORC_ERR_CORRUPT; break; }
                switch (op) {
                case OP_RP: v = parent; break;
                case OP_RX: case OP_RY: case OP_RZ: {
                    int a = (int)op - OP_RX;
                    if (!neighbour_value(lab, N, l - 1, qx, qy, qz, a, &v)) rc = ORC_ERR_CORRUPT;
                    break;
                }
                case OP_P0: v = palette[ip]; break;
                case OP_PD: {
                    uint32_t d;
                    rc = get_nib(in, &d);
                    if (rc == ORC_OK && ip < 1 + d) rc = ORC_ERR_CORRUPT;
                    if (rc == ORC_OK) v = palette[ip - 1 - d];
                    break;
                }
                case OP_PA:
                    if (ip + 1 >= n_palette) { rc = ORC_ERR_CORRUPT; break; }
                    ip += 1;
                    v = palette[ip];
                    break;
                default: rc = ORC_ERR_CORRUPT; break;
                }
                Lc[qi] = v;
                Cc[qi] = (uint8_t)stop;
            }
        }
    }
    /* every symbol of a fully walked stream must have been used */
    if (rc == ORC_OK && t <= 1 && rint.pos != rint.n) rc = ORC_ERR_CORRUPT;
    if (rc == ORC_OK && t == 0 && rleaf.pos != rleaf.n) rc = ORC_ERR_CORRUPT;
    if (rc == ORC_OK) memcpy(out, lab + level_offset(N, t), sizeof(uint32_t) * cube((1u << N) >> t));
    free(lab);
    free(cst);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Sec. 3.3: static frequency tables                                   */
/* ------------------------------------------------------------------ */

/*
 * Normalise 16 nibble counts to frequencies summing to M = 4096, each >= 1 (R11).
 * Exact for any counts whose sum fits in 64 bits: the product count * 4080 is
 * formed in 128 bits before the division.
 */
void csgvo_normalize(const uint64_t counts[16], uint32_t freq[16]) {
    uint64_t total = 0;
    for (int s = 0; s < 16; s++) total += counts[s];
    if (total == 0) {
        for (int s = 0; s < 16; s++) freq[s] = RANS_M / 16;
        return;
    }
    uint32_t sum = 0;
    for (int s = 0; s < 16; s++) {
        unsigned __int128 scaled = (unsigned __int128)counts[s] * (RANS_M - 16);
        freq[s] = 1u + (uint32_t)(scaled / total);
        sum += freq[s];
    }
    uint32_t r = RANS_M - sum; /* 0 <= r < 16 */
    int used[16] = {0};
    for (uint32_t k = 0; k < r; k++) {
        int best = -1;
        for (int s = 0; s < 16; s++) {
            if (used[s]) continue;
            if (best < 0 || counts[s] > counts[best]) best = s;
        }
        used[best] = 1;
        freq[best] += 1;
    }
}

/* ------------------------------------------------------------------ */
/* Sec. 3.3: rANS over the nibble stream                               */
/* ------------------------------------------------------------------ */

/* number of interleaved states for a stream of n symbols (R10) */
uint32_t csgvo_lanes(uint32_t n, uint32_t K_max, uint32_t S_min) {
    if (n == 0) return 0;
    uint32_t k = n / S_min;
    if (k < 1) k = 1;
    if (k > K_max) k = K_max;
    return k;
}

/* cumulative frequency start of symbol s */
static uint32_t cum_of(const uint32_t freq[16], uint32_t s) {
    uint32_t c = 0;
    for (uint32_t r = 0; r < s; r++) c += freq[r];
    return c;
}

/*
 * The coder itself (Sec. 3.3, R9): n symbols in coding order, symbol i coded
 * with state lane[i].  Encoding runs from the last symbol to the first, so
 * that the decoder reads forward; words receives the K final states, then
 * the renormalisation words in the order the decoder takes them.
 */
static int rans_encode_order(const uint8_t *sym, const uint32_t *lane, uint32_t n, uint32_t K,
                             const uint32_t freq[16], uint16_t *words, uint32_t cap, uint32_t *n_words) {
    uint32_t *x = (uint32_t *)malloc(sizeof(uint32_t) * K);
    uint16_t *emit = (uint16_t *)malloc(sizeof(uint16_t) * (n + 1));
    if (!x || !emit) { free(x); free(emit); return ORC_ERR_NOMEM; }
    for (uint32_t k = 0; k < K; k++) x[k] = RANS_L;
    uint32_t ne = 0;
    for (uint32_t i = n; i-- > 0;) {
        uint32_t k = lane[i], s = sym[i];
        uint32_t f = freq[s], c = cum_of(freq, s);
        /* renormalise: keep x below f * 2^20 = ((L >> scale) << 16) * f */
        uint64_t bound = ((uint64_t)(RANS_L >> RANS_SCALE_BITS) << 16) * f;
        if ((uint64_t)x[k] >= bound) {
            emit[ne++] = (uint16_t)(x[k] & 0xFFFFu);
            x[k] >>= 16;
        }
        x[k] = (x[k] / f) * RANS_M + (x[k] % f) + c;
    }
    uint32_t total = 2 * K + ne;
    if (total > cap) { free(x); free(emit); return ORC_ERR_ARG; }
    for (uint32_t k = 0; k < K; k++) {
        words[2 * k] = (uint16_t)(x[k] & 0xFFFFu);
        words[2 * k + 1] = (uint16_t)(x[k] >> 16);
    }
    for (uint32_t j = 0; j < ne; j++) words[2 * K + j] = emit[ne - 1 - j];
    *n_words = total;
    free(x);
    free(emit);
    return ORC_OK;
}

/* decode one symbol with state *x, reading a renormalisation word when needed */
static int rans_decode_one(uint32_t *x, const uint32_t freq[16], const uint16_t *words, uint32_t n_words,
                           uint32_t *pos, uint8_t *out) {
    uint32_t slot = *x & (RANS_M - 1);
    uint32_t s = 0;
    while (s + 1 < 16 && cum_of(freq, s + 1) <= slot) s++;
    *out = (uint8_t)s;
    *x = freq[s] * (*x >> RANS_SCALE_BITS) + slot - cum_of(freq, s);
    if (*x < RANS_L) {
        if (*pos >= n_words) return ORC_ERR_CORRUPT;
        *x = (*x << 16) | words[(*pos)++];
    }
    return ORC_OK;
}

/*
 * Encode a nibble stream of n symbols (stream order: each P_delta op nibble
 * followed by its delta nibble, R6) with K interleaved states under the
 * coding order of R10.  Empty input gives an empty stream.
 */
int csgvo_rans_encode(const uint8_t *sym, uint32_t n, uint32_t K, const uint32_t freq[16],
                      uint16_t *words, uint32_t cap, uint32_t *n_words) {
    *n_words = 0;
    if (n == 0) return ORC_OK;
    if (K == 0 || K > n) return ORC_ERR_ARG;
    /* the ops: stream position of each op nibble */
    uint32_t *op_at = (uint32_t *)malloc(sizeof(uint32_t) * n);
    uint8_t *cs = (uint8_t *)malloc(n);
    uint32_t *cl = (uint32_t *)malloc(sizeof(uint32_t) * n);
    if (!op_at || !cs || !cl) { free(op_at); free(cs); free(cl); return ORC_ERR_NOMEM; }
    uint32_t m = 0;
    int rc = ORC_OK;
    for (uint32_t i = 0; i < n; i++) {
        op_at[m++] = i;
        if ((sym[i] & 7u) == OP_PD) {
            if (i + 1 >= n) { rc = ORC_ERR_ARG; break; } /* a P_delta needs its delta nibble */
            i++;
        }
    }
    /* coding order: per step of K ops, the ops in state order, then their deltas */
    uint32_t c = 0;
    for (uint32_t t0 = 0; rc == ORC_OK && t0 < m; t0 += K) {
        uint32_t t1 = t0 + K < m ? t0 + K : m;
        for (uint32_t j = t0; j < t1; j++) { cs[c] = sym[op_at[j]]; cl[c++] = j - t0; }
        for (uint32_t j = t0; j < t1; j++)
            if ((sym[op_at[j]] & 7u) == OP_PD) { cs[c] = sym[op_at[j] + 1]; cl[c++] = j - t0; }
    }
    if (rc == ORC_OK) rc = rans_encode_order(cs, cl, n, K, freq, words, cap, n_words);
    free(op_at); free(cs); free(cl);
    return rc;
}

/*
 * Decode the first m of the n symbols (stream order) of a K-state stream.
 * Steps follow the coding order of R10: in state order, a state decodes an
 * op nibble while more symbols remain than the delta nibbles owed to the
 * step's P_delta ops so far; then each P_delta op's state decodes its delta
 * nibble.  Whole steps are decoded until the first m stream symbols are out.
 * When m == n the end of the stream is checked: every state must be back at
 * L and every word used; otherwise ORC_ERR_CORRUPT.
 */
int csgvo_rans_decode(const uint16_t *words, uint32_t n_words, uint32_t n, uint32_t m, uint32_t K,
                      const uint32_t freq[16], uint8_t *sym) {
    if (m > n) return ORC_ERR_ARG;
    if (n == 0) return n_words == 0 ? ORC_OK : ORC_ERR_CORRUPT;
    if (K == 0 || K > n || n_words < 2 * K) return ORC_ERR_CORRUPT;
    uint32_t *x = (uint32_t *)malloc(sizeof(uint32_t) * K);
    uint8_t *op = (uint8_t *)malloc(K), *dl = (uint8_t *)malloc(K);
    uint8_t *st = (uint8_t *)malloc(n + 1);
    if (!x || !op || !dl || !st) { free(x); free(op); free(dl); free(st); return ORC_ERR_NOMEM; }
    for (uint32_t k = 0; k < K; k++) x[k] = (uint32_t)words[2 * k] | ((uint32_t)words[2 * k + 1] << 16);
    uint32_t pos = 2 * K, used = 0, out = 0;
    int rc = ORC_OK;
    while (rc == ORC_OK && out < m) {
        uint32_t nops = 0, owed = 0;
        for (uint32_t k = 0; k < K && rc == ORC_OK; k++) {
            if (used + owed >= n) break;
            rc = rans_decode_one(&x[k], freq, words, n_words, &pos, &op[k]);
            used++;
            nops++;
            if ((op[k] & 7u) == OP_PD) owed++;
        }
        if (rc == ORC_OK && nops == 0) rc = ORC_ERR_CORRUPT;
        for (uint32_t k = 0; k < nops && rc == ORC_OK; k++)
            if ((op[k] & 7u) == OP_PD) {
                if (used >= n) { rc = ORC_ERR_CORRUPT; break; } /* a delta past the stream's symbols */
                rc = rans_decode_one(&x[k], freq, words, n_words, &pos, &dl[k]);
                used++;
            }
        for (uint32_t k = 0; k < nops && rc == ORC_OK; k++) {
            st[out++] = op[k];
            if ((op[k] & 7u) == OP_PD) st[out++] = dl[k];
        }
    }
    if (rc == ORC_OK) {
        memcpy(sym, st, m);
        if (m == n) {
            for (uint32_t k = 0; k < K; k++)
                if (x[k] != RANS_L) rc = ORC_ERR_CORRUPT;
            if (pos != n_words) rc = ORC_ERR_CORRUPT;
        }
    }
    free(x); free(op); free(dl); free(st);
    return rc;
}

/* ------------------------------------------------------------------ */
/* volume level: bricking, prepass, per-brick encode, concatenation    */
/* ------------------------------------------------------------------ */

typedef struct {
    int N;
    uint64_t dims[3];
    uint64_t nb[3];
    uint64_t n_bricks;
    uint32_t K_max, S_min;
    uint32_t freq_int[16], freq_leaf[16];
    /* per-brick results before concatenation */
    uint32_t **pal;
    uint32_t *n_pal;
    uint16_t **wint, **wleaf;
    uint32_t *n_wint, *n_wleaf;
    uint32_t *n_int_sym, *n_leaf_sym;
    uint64_t op_counts[7];
} csgvo_volume;

/* copy brick (bx,by,bz) out of the volume, padding by clamp-to-edge (R8) */
static void extract_brick(const uint32_t *vol, const uint64_t dims[3], int N, uint64_t bx, uint64_t by,
                          uint64_t bz, uint32_t *brick) {
    uint64_t b = 1ull << N;
    for (uint64_t z = 0; z < b; z++)
        for (uint64_t y = 0; y < b; y++)
            for (uint64_t x = 0; x < b; x++) {
                uint64_t gx = bx * b + x, gy = by * b + y, gz = bz * b + z;
                if (gx >= dims[0]) gx = dims[0] - 1;
                if (gy >= dims[1]) gy = dims[1] - 1;
                if (gz >= dims[2]) gz = dims[2] - 1;
                brick[x + b * (y + b * z)] = vol[gx + dims[0] * (gy + dims[1] * gz)];
            }
}

typedef struct {
    csgvo_volume *v;
    const uint32_t *vol;
    int phase; /* 0 = prepass counting, 1 = encode */
    uint64_t stride;
    uint64_t next; /* shared brick counter */
    pthread_mutex_t mu;
    uint64_t cnt_int[16], cnt_leaf[16];
    int rc;
} vol_job;

static void *vol_worker(void *arg) {
    vol_job *J = (vol_job *)arg;
    csgvo_volume *v = J->v;
    int N = v->N;
    uint64_t b3 = cube(1ull << N), nodes = csgvo_pyramid_nodes(N);
    uint64_t int_cap = 2 * (nodes - b3), leaf_cap = 2 * b3;
    uint32_t *brick = (uint32_t *)malloc(sizeof(uint32_t) * b3);
    uint32_t *pal = (uint32_t *)malloc(sizeof(uint32_t) * nodes);
    uint8_t *ni = (uint8_t *)malloc(int_cap + 1), *nl = (uint8_t *)malloc(leaf_cap + 1);
    uint16_t *wi = (uint16_t *)malloc(sizeof(uint16_t) * (int_cap + 64 + 1));
    uint16_t *wl = (uint16_t *)malloc(sizeof(uint16_t) * (leaf_cap + 64 + 1));
    uint64_t ci[16] = {0}, cl[16] = {0}, ops[7] = {0};
    int rc = (brick && pal && ni && nl && wi && wl) ? ORC_OK : ORC_ERR_NOMEM;
    while (rc == ORC_OK) {
        pthread_mutex_lock(&J->mu);
        uint64_t id = J->next;
        J->next += (J->phase == 0) ? J->stride : 1;
        pthread_mutex_unlock(&J->mu);
        if (id >= v->n_bricks) break;
        uint64_t bx = id % v->nb[0], by = (id / v->nb[0]) % v->nb[1], bz = id / (v->nb[0] * v->nb[1]);
        extract_brick(J->vol, v->dims, N, bx, by, bz, brick);
        uint32_t np, nint, nleaf;
        rc = csgvo_encode_brick(brick, N, pal, (uint32_t)nodes, &np, ni, (uint32_t)int_cap, &nint, nl,
                                (uint32_t)leaf_cap, &nleaf, J->phase == 1 ? ops : NULL);
        if (rc) break;
        if (J->phase == 0) {
            for (uint32_t i = 0; i < nint; i++) ci[ni[i]]++;
            for (uint32_t i = 0; i < nleaf; i++) cl[nl[i]]++;
            continue;
        }
        uint32_t nwi, nwl;
        rc = csgvo_rans_encode(ni, nint, csgvo_lanes(nint, v->K_max, v->S_min), v->freq_int, wi,
                               (uint32_t)(int_cap + 64), &nwi);
        if (rc == ORC_OK)
            rc = csgvo_rans_encode(nl, nleaf, csgvo_lanes(nleaf, v->K_max, v->S_min), v->freq_leaf, wl,
                                   (uint32_t)(leaf_cap + 64), &nwl);
        if (rc) break;
        v->pal[id] = (uint32_t *)malloc(sizeof(uint32_t) * np);
        v->wint[id] = (uint16_t *)malloc(sizeof(uint16_t) * (nwi ? nwi : 1));
        v->wleaf[id] = (uint16_t *)malloc(sizeof(uint16_t) * (nwl ? nwl : 1));
        if (!v->pal[id] || !v->wint[id] || !v->wleaf[id]) { rc = ORC_ERR_NOMEM; break; }
        memcpy(v->pal[id], pal, sizeof(uint32_t) * np);
        memcpy(v->wint[id], wi, sizeof(uint16_t) * nwi);
        memcpy(v->wleaf[id], wl, sizeof(uint16_t) * nwl);
        v->n_pal[id] = np;
        v->n_wint[id] = nwi;
        v->n_wleaf[id] = nwl;
        v->n_int_sym[id] = nint;
        v->n_leaf_sym[id] = nleaf;
    }
    pthread_mutex_lock(&J->mu);
    for (int s = 0; s < 16; s++) { J->cnt_int[s] += ci[s]; J->cnt_leaf[s] += cl[s]; }
    for (int o = 0; o < 7; o++) v->op_counts[o] += ops[o];
    if (rc && !J->rc) J->rc = rc;
    pthread_mutex_unlock(&J->mu);
    free(brick); free(pal); free(ni); free(nl); free(wi); free(wl);
    return NULL;
}

static int run_phase(csgvo_volume *v, const uint32_t *vol, int phase, uint64_t stride, int n_threads,
                     uint64_t cnt_int[16], uint64_t cnt_leaf[16]) {
    vol_job J;
    memset(&J, 0, sizeof J);
    J.v = v; J.vol = vol; J.phase = phase; J.stride = stride ? stride : 1;
    pthread_mutex_init(&J.mu, NULL);
    if (n_threads < 1) n_threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * n_threads);
    for (int i = 0; i < n_threads; i++) pthread_create(&th[i], NULL, vol_worker, &J);
    for (int i = 0; i < n_threads; i++) pthread_join(th[i], NULL);
    free(th);
    pthread_mutex_destroy(&J.mu);
    if (cnt_int) memcpy(cnt_int, J.cnt_int, sizeof J.cnt_int);
    if (cnt_leaf) memcpy(cnt_leaf, J.cnt_leaf, sizeof J.cnt_leaf);
    return J.rc;
}

void csgvo_volume_free(csgvo_volume *v) {
    if (!v) return;
    for (uint64_t i = 0; i < v->n_bricks; i++) {
        if (v->pal) free(v->pal[i]);
        if (v->wint) free(v->wint[i]);
        if (v->wleaf) free(v->wleaf[i]);
    }
    free(v->pal); free(v->wint); free(v->wleaf);
    free(v->n_pal); free(v->n_wint); free(v->n_wleaf);
    free(v->n_int_sym); free(v->n_leaf_sym);
    free(v);
}

/*
 * Prepass (Sec. 3.4): run the brick encoder over every stride-th brick and
 * count the nibbles of the interior and leaf streams.
 */
int csgvo_count_nibbles(const uint32_t *vol, const uint64_t dims[3], int N, uint64_t stride, int n_threads,
                        uint64_t cnt_int[16], uint64_t cnt_leaf[16]) {
    csgvo_volume tmp;
    memset(&tmp, 0, sizeof tmp);
    tmp.N = N;
    uint64_t b = 1ull << N;
    for (int a = 0; a < 3; a++) { tmp.dims[a] = dims[a]; tmp.nb[a] = (dims[a] + b - 1) / b; }
    tmp.n_bricks = tmp.nb[0] * tmp.nb[1] * tmp.nb[2];
    return run_phase(&tmp, vol, 0, stride, n_threads, cnt_int, cnt_leaf);
}

/*
 * Encode a whole volume (x-fastest, dims[0] fastest).  If freq is non-NULL
 * its 32 entries (interior table, then leaf table) are used as given;
 * otherwise the tables come from the prepass over every stride-th brick.
 */
csgvo_volume *csgvo_encode_volume(const uint32_t *vol, const uint64_t dims[3], int N, uint64_t stride,
                                  uint32_t K_max, uint32_t S_min, const uint32_t *freq, int n_threads,
                                  int *rc_out) {
    int rc = ORC_OK;
    if (N < 1 || N > 6 || K_max < 1 || S_min < 1 || !dims[0] || !dims[1] || !dims[2]) {
        if (rc_out) *rc_out = ORC_ERR_ARG;
        return NULL;
    }
    csgvo_volume *v = (csgvo_volume *)calloc(1, sizeof(csgvo_volume));
    v->N = N;
    uint64_t b = 1ull << N;
    for (int a = 0; a < 3; a++) { v->dims[a] = dims[a]; v->nb[a] = (dims[a] + b - 1) / b; }
    v->n_bricks = v->nb[0] * v->nb[1] * v->nb[2];
    v->K_max = K_max;
    v->S_min = S_min;
    if (freq) {
        memcpy(v->freq_int, freq, 16 * sizeof(uint32_t));
        memcpy(v->freq_leaf, freq + 16, 16 * sizeof(uint32_t));
    } else {
        uint64_t ci[16], cl[16];
        rc = csgvo_count_nibbles(vol, dims, N, stride, n_threads, ci, cl);
        csgvo_normalize(ci, v->freq_int);
        csgvo_normalize(cl, v->freq_leaf);
    }
    uint64_t n = v->n_bricks;
    v->pal = (uint32_t **)calloc(n, sizeof(void *));
    v->wint = (uint16_t **)calloc(n, sizeof(void *));
    v->wleaf = (uint16_t **)calloc(n, sizeof(void *));
    v->n_pal = (uint32_t *)calloc(n, 4);
    v->n_wint = (uint32_t *)calloc(n, 4);
    v->n_wleaf = (uint32_t *)calloc(n, 4);
    v->n_int_sym = (uint32_t *)calloc(n, 4);
    v->n_leaf_sym = (uint32_t *)calloc(n, 4);
    if (rc == ORC_OK) rc = run_phase(v, vol, 1, 1, n_threads, NULL, NULL);
    if (rc_out) *rc_out = rc;
    if (rc) { csgvo_volume_free(v); return NULL; }
    return v;
}

/* sizes: [n_bricks, palette labels, interior words, leaf words] */
void csgvo_volume_sizes(const csgvo_volume *v, uint64_t out[4]) {
    uint64_t sp = 0, si = 0, sl = 0;
    for (uint64_t i = 0; i < v->n_bricks; i++) { sp += v->n_pal[i]; si += v->n_wint[i]; sl += v->n_wleaf[i]; }
    out[0] = v->n_bricks; out[1] = sp; out[2] = si; out[3] = sl;
}

/* freq: 32 entries (interior then leaf); op_counts: 7 entries */
void csgvo_volume_tables(const csgvo_volume *v, uint32_t freq[32], uint64_t op_counts[7]) {
    memcpy(freq, v->freq_int, 16 * 4);
    memcpy(freq + 16, v->freq_leaf, 16 * 4);
    if (op_counts) memcpy(op_counts, v->op_counts, 7 * 8);
}

/*
 * Concatenate the per-brick results in brick-id order.  Offsets are
 * exclusive prefix sums with n_bricks + 1 entries (palette offsets in
 * labels, word offsets in 16-bit words).
 */
void csgvo_volume_export(const csgvo_volume *v, uint64_t *pal_off, uint32_t *pal, uint64_t *int_off,
                         uint16_t *int_words, uint64_t *leaf_off, uint16_t *leaf_words, uint32_t *n_int_sym,
                         uint32_t *n_leaf_sym) {
    uint64_t sp = 0, si = 0, sl = 0;
    for (uint64_t i = 0; i < v->n_bricks; i++) {
        pal_off[i] = sp; int_off[i] = si; leaf_off[i] = sl;
        memcpy(pal + sp, v->pal[i], 4 * (size_t)v->n_pal[i]);
        memcpy(int_words + si, v->wint[i], 2 * (size_t)v->n_wint[i]);
        memcpy(leaf_words + sl, v->wleaf[i], 2 * (size_t)v->n_wleaf[i]);
        sp += v->n_pal[i]; si += v->n_wint[i]; sl += v->n_wleaf[i];
        n_int_sym[i] = v->n_int_sym[i];
        n_leaf_sym[i] = v->n_leaf_sym[i];
    }
    pal_off[v->n_bricks] = sp; int_off[v->n_bricks] = si; leaf_off[v->n_bricks] = sl;
}

/* ------------------------------------------------------------------ */
/* decoding a batch of bricks from the concatenated arrays             */
/* ------------------------------------------------------------------ */

typedef struct {
    int N;
    uint32_t K_max, S_min;
    const uint32_t *freq;
    const uint64_t *pal_off, *int_off, *leaf_off;
    const uint32_t *pal;
    const uint16_t *int_words, *leaf_words;
    const uint32_t *n_int_sym, *n_leaf_sym;
    uint64_t n_bricks;
    const uint32_t *brick_ids;
    const uint8_t *lods;
    uint64_t n_req;
    uint32_t *out;
    const uint64_t *out_off;
    int32_t *status;
    uint64_t next;
    pthread_mutex_t mu;
} dec_job;

/* decode one request: rANS both streams (leaf only for t == 0), then Alg. 1 */
static int decode_one(dec_job *J, uint32_t id, int t, uint32_t *out, uint8_t *ni, uint8_t *nl) {
    if (id >= J->n_bricks || t < 0 || t > J->N) return ORC_ERR_ARG;
    uint32_t nint = J->n_int_sym[id], nleaf = J->n_leaf_sym[id];
    const uint16_t *wi = J->int_words + J->int_off[id];
    const uint16_t *wl = J->leaf_words + J->leaf_off[id];
    uint32_t nwi = (uint32_t)(J->int_off[id + 1] - J->int_off[id]);
    uint32_t nwl = (uint32_t)(J->leaf_off[id + 1] - J->leaf_off[id]);
    int rc = csgvo_rans_decode(wi, nwi, nint, nint, csgvo_lanes(nint, J->K_max, J->S_min), J->freq, ni);
    if (rc == ORC_OK && t == 0)
        rc = csgvo_rans_decode(wl, nwl, nleaf, nleaf, csgvo_lanes(nleaf, J->K_max, J->S_min), J->freq + 16, nl);
    if (rc) return rc;
    /* a brick with symbols must have a full root-children set; the decoder checks consumption */
    return csgvo_decode_brick(J->pal + J->pal_off[id], (uint32_t)(J->pal_off[id + 1] - J->pal_off[id]), ni, nint,
                              nl, t == 0 ? nleaf : 0, J->N, t, out);
}

static void *dec_worker(void *arg) {
    dec_job *J = (dec_job *)arg;
    uint64_t b3 = cube(1ull << J->N), nodes = csgvo_pyramid_nodes(J->N);
    uint8_t *ni = (uint8_t *)malloc(2 * (nodes - b3) + 1), *nl = (uint8_t *)malloc(2 * b3 + 1);
    for (;;) {
        pthread_mutex_lock(&J->mu);
        uint64_t r = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (r >= J->n_req) break;
        uint32_t id = J->brick_ids[r];
        int t = J->lods[r];
        int rc;
        if (id < J->n_bricks && (J->n_int_sym[id] > 2 * (nodes - b3) || J->n_leaf_sym[id] > 2 * b3))
            rc = ORC_ERR_CORRUPT;
        else
            rc = decode_one(J, id, t, J->out + J->out_off[r], ni, nl);
        J->status[r] = rc;
    }
    free(ni);
    free(nl);
    return NULL;
}

/*
 * Decode n_req requests (brick id, LOD) from concatenated arrays into
 * out + out_off[r] ((b>>t)^3 labels each); status[r] = 0 or an error code.
 * freq holds the interior table then the leaf table.
 */
int csgvo_decode_bricks(int N, uint32_t K_max, uint32_t S_min, const uint32_t *freq, uint64_t n_bricks,
                        const uint64_t *pal_off, const uint32_t *pal, const uint64_t *int_off,
                        const uint16_t *int_words, const uint64_t *leaf_off, const uint16_t *leaf_words,
                        const uint32_t *n_int_sym, const uint32_t *n_leaf_sym, const uint32_t *brick_ids,
                        const uint8_t *lods, uint64_t n_req, uint32_t *out, const uint64_t *out_off,
                        int32_t *status, int n_threads) {
    if (N < 1 || N > 6 || K_max < 1 || S_min < 1) return ORC_ERR_ARG;
    dec_job J;
    memset(&J, 0, sizeof J);
    J.N = N; J.K_max = K_max; J.S_min = S_min; J.freq = freq;
    J.pal_off = pal_off; J.pal = pal; J.int_off = int_off; J.int_words = int_words;
    J.leaf_off = leaf_off; J.leaf_words = leaf_words; J.n_int_sym = n_int_sym; J.n_leaf_sym = n_leaf_sym;
    J.n_bricks = n_bricks; J.brick_ids = brick_ids; J.lods = lods; J.n_req = n_req;
    J.out = out; J.out_off = out_off; J.status = status;
    pthread_mutex_init(&J.mu, NULL);
    if (n_threads < 1) n_threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * n_threads);
    for (int i = 0; i < n_threads; i++) pthread_create(&th[i], NULL, dec_worker, &J);
    for (int i = 0; i < n_threads; i++) pthread_join(th[i], NULL);
    free(th);
    pthread_mutex_destroy(&J.mu);
    return ORC_OK;
}
