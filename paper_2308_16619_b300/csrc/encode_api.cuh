// encode_api.cuh -- encoder structs and launchers shared by encode.cu and api.cu.
#pragma once
#include "csgv_internal.cuh"

namespace csgv {

// per-N geometry shared by the encoder kernels
struct EncGeom {
    uint32_t N, b;
    uint32_t off[kMaxN + 2];  // offset of level l (1..N) in the level arrays (Morton order within a level)
    uint32_t up_nodes;        // sum over l >= 1 of (b>>l)^3
    uint32_t ops_cap;         // coded children at most: nodes - 1
    uint32_t pal_cap, int_cap, leaf_cap;  // per brick: palette labels, interior and leaf nibbles at most
    uint32_t smem;            // dynamic shared memory bytes
    uint32_t lvl_bytes;       // level arrays in global scratch per brick (b = 64), else 0
    uint32_t K_max, S_min;    // interleaving rule (R10)
};

// per-brick scratch of one encode batch of C bricks
struct EncScratch {
    uint32_t *pal;      // C x pal_cap
    uint16_t *w_int;    // C x (int_cap + 64)
    uint16_t *w_leaf;   // C x (leaf_cap + 64)
    uint32_t *sizes;    // C x 8: n_pal, n_int_sym, n_leaf_sym, n_int_words, n_leaf_words, int_start, leaf_start,
                        // interior op count / 8 | leaf op count / 8 << 16
    uint8_t *ops;       // C x ops_cap: op bytes (op | stop << 3 | delta << 4) of the brick in stream order
    uint8_t *lvl;       // C x lvl_bytes: level arrays (b = 64 only)
};

struct EncVol {
    const uint32_t *vol;
    uint64_t dims[3];
    uint64_t nb[3];
};

EncGeom make_geom(uint32_t N, uint32_t K_max, uint32_t S_min);
size_t scratch_bytes_per_brick(const EncGeom &G);
cudaError_t launch_encode(const EncVol &EV, const EncGeom &G, uint64_t brick0, uint64_t stride, uint32_t n,
                          const uint32_t *freq, const EncScratch &SC, unsigned long long *count, cudaStream_t st);
cudaError_t launch_rans_encode(const EncGeom &G, const EncScratch &SC, uint32_t n, const uint32_t *freq,
                               cudaStream_t st);
cudaError_t launch_nibble_hist(const EncGeom &G, const EncScratch &SC, uint32_t n, uint32_t stride,
                               unsigned long long *counts, cudaStream_t st);
cudaError_t launch_scan(const uint32_t *sizes, uint32_t n, uint64_t first, uint64_t *pal_off, uint64_t *int_off,
                        uint64_t *leaf_off, uint64_t *tot, uint32_t *maxes, unsigned long long *blk, cudaStream_t st);
// bytes of the scratch that launch_scan's two-pass scan needs (blk)
constexpr size_t kScanScratchBytes = (64 + 1) * 4 * 8 * 2;
cudaError_t launch_compact(const EncGeom &G, const EncScratch &SC, uint64_t first, uint32_t n, const uint64_t *pal_off,
                           const uint64_t *int_off, const uint64_t *leaf_off, uint32_t *pal, uint16_t *int_words,
                           uint16_t *leaf_words, uint32_t *n_int_sym, uint32_t *n_leaf_sym, cudaStream_t st);

}  // namespace csgv
