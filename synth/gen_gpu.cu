// gen_gpu.cu -- device versions of seeded synthetic generators that are too
// large to make on the host (the 2048 x 2048 x 1024 serving volume).  Same
// integer formulas as gen.c, so a small volume made here equals gen.c's.
// No codec arithmetic here.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr int64_t kFP = 256;
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t hash2(uint64_t a, uint64_t b) {
    return mix64(mix64(a + kGolden) ^ (b * kGolden + 0x632BE59BD9B4E019ull));
}
__device__ __forceinline__ uint32_t label_of(uint64_t seed, uint64_t id) {
    const uint32_t v = (uint32_t)hash2(seed ^ 0x5EED1AB1ull, id);
    return v ? v : 1u;
}

__global__ void worley_kernel(uint32_t *vol, uint64_t X, uint64_t Y, uint64_t Z, int64_t C, uint64_t seed,
                              uint64_t z0, uint64_t nz) {
    const uint64_t n = X * Y * nz;
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x = t % X, y = (t / X) % Y, z = z0 + t / (X * Y);
        const int64_t p0 = (int64_t)x * kFP + kFP / 2, p1 = (int64_t)y * kFP + kFP / 2, p2 = (int64_t)z * kFP + kFP / 2;
        const int64_t ci = (int64_t)x / C, cj = (int64_t)y / C, ck = (int64_t)z / C;
        int64_t best = INT64_MAX, bi = 0, bj = 0, bk = 0;
        for (int64_t i = ci - 1; i <= ci + 1; i++)
            for (int64_t j = cj - 1; j <= cj + 1; j++)
                for (int64_t k = ck - 1; k <= ck + 1; k++) {
                    const uint64_t key = ((uint64_t)(i + 1) << 42) ^ ((uint64_t)(j + 1) << 21) ^ (uint64_t)(k + 1);
                    const uint64_t h = hash2(seed ^ 0x3A0E1Eull, key);
                    const int64_t f0 = i * C * kFP + (int64_t)((h & 0xFFFFFull) % (uint64_t)(C * kFP));
                    const int64_t f1 = j * C * kFP + (int64_t)(((h >> 20) & 0xFFFFFull) % (uint64_t)(C * kFP));
                    const int64_t f2 = k * C * kFP + (int64_t)(((h >> 40) & 0xFFFFFull) % (uint64_t)(C * kFP));
                    const int64_t d0 = f0 - p0, d1 = f1 - p1, d2 = f2 - p2;
                    const int64_t d = d0 * d0 + d1 * d1 + d2 * d2;
                    if (d < best) {
                        best = d;
                        bi = i;
                        bj = j;
                        bk = k;
                    }
                }
        const uint64_t cell = ((uint64_t)(bi + 1) << 42) ^ ((uint64_t)(bj + 1) << 21) ^ (uint64_t)(bk + 1);
        vol[x + X * (y + Y * z)] = label_of(seed, cell);
    }
}

}  // namespace

extern "C" __attribute__((visibility("default"))) int synth_worley_dev(uint32_t *vol_dev, uint64_t X, uint64_t Y,
                                                                        uint64_t Z, uint32_t cell, uint64_t seed,
                                                                        void *stream) {
    if (!vol_dev || !cell || !X || !Y || !Z) return 1;
    const uint64_t slab = 64;  // z slices per launch
    for (uint64_t z0 = 0; z0 < Z; z0 += slab) {
        const uint64_t nz = Z - z0 < slab ? Z - z0 : slab;
        worley_kernel<<<148 * 8, 256, 0, (cudaStream_t)stream>>>(vol_dev, X, Y, Z, (int64_t)cell, seed, z0, nz);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
